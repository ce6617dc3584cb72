// Relative-scale solve (Eq. 14) with an aggregation-multigrid preconditioner on
// the quotient graph: `scale_precond = 1`, K <= 8192 (one CTA), an option off
// by default.  The system and its answer are those of k_scale_cg (the same PCG,
// tolerance, energy and stop test); only the preconditioner differs.
//
// Setup, every iteration (the weights of Eqs. 5 and 11 change with t, and
// aggregates taken from other weights straddle the edges the outlier weights
// cut): on level l every node joins its strongest neighbour (largest weight,
// ties to the smaller index); the connected components of those edges
// (union-find, roots = smallest member) are the nodes of level l + 1, numbered
// by the rank of their root.  Coarse pairs are the level-l pairs whose ends
// fall in different aggregates, merged in a hash table, their weights summed
// (the Galerkin product P^T A P of the piecewise-constant prolongation P keeps
// the graph-Laplacian form).  Levels stop at <= SMG_DENSE nodes, when a level
// shrinks by less than 10 %, or at SMG_LMAX levels.  The coarsest level, when
// small enough, is solved by a dense Cholesky factor of (L + eps I) held in
// shared memory; otherwise by damped Jacobi sweeps.
//
// V-cycle: damped Jacobi (omega 0.7) from zero, residual, restriction (sum over
// the aggregate), coarse correction, prolongation, one damped Jacobi step: a
// symmetric operator, as PCG needs.  All in FP64, all in one CTA of 1024
// threads synchronised by __syncthreads; scratch lives in global memory (L2).
#include <algorithm>

#include "ni_internal.cuh"

#define SMG_LMAX 8
#define SMG_DENSE 32
#define SMG_THREADS 1024
#define SMG_OMEGA 0.7
#define SMG_COARSE_SWEEPS 30
#define SMG_EMPTY 0xffffffffffffffffull

struct ScaleMgScratch {
  int ncap = 0, pcap = 0, ecap = 0, hcap = 0;
  double *nd = nullptr, *ninv = nullptr, *nx = nullptr, *nb = nullptr, *nr = nullptr;
  int *nagg = nullptr, *npar = nullptr, *nbest = nullptr, *nrank = nullptr;
  int *plo = nullptr, *phi = nullptr, *pslot = nullptr;
  double* pw = nullptr;
  int* crow = nullptr;
  int* ccol = nullptr;
  double* cw = nullptr;
  unsigned long long* hkey = nullptr;
  int* hidx = nullptr;
};

struct SmgLevel {
  int n, np;          // nodes, pairs
  int noff, poff;     // offsets into the node pool and the coarse pair pool (level 0 pairs are the partition's)
  int roff, eoff;     // offsets of the level's CSR row pointers and entries (levels >= 1)
};

struct ScaleMgArgs {
  DevState* st;
  const int* row_ptr;     // level 0 CSR of the quotient Laplacian (off-diagonal weights csr_w)
  const int* csr_col;
  const double* csr_w;
  const int* p_lo;        // level 0 pairs; weight p_acc[3 p]
  const int* p_hi;
  const double* p_acc;
  const double* diag;
  const double* g;
  const double* gabs;
  double *s, *r, *z, *pp, *qq;
  double* soff;
  double tol2;
  int maxit, T;
  double dE_max;
  ScaleMgScratch m;
};

// ---------------------------------------------------------------------------
// CTA-wide helpers (every thread of the CTA calls them)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double smg_sum(double v, double* sh) { return block_sum_d(v, sh); }

// exclusive scan of flag(i) over i in [0, n) into out[i]; returns the total
template <class F>
__device__ int smg_scan(int n, F flag, int* out, int* shi) {
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int beg = min(n, (int)threadIdx.x * per), end = min(n, beg + per);
  int c = 0;
  for (int i = beg; i < end; ++i) c += flag(i);
  int tot;
  int base = block_excl_scan_i(c, shi, &tot);
  for (int i = beg; i < end; ++i) {
    out[i] = base;
    base += flag(i);
  }
  __syncthreads();
  return tot;
}

struct SmgCsr {
  const int* rp;
  const int* col;
  const double* w;
};

__device__ __forceinline__ SmgCsr smg_csr(const ScaleMgArgs& A, const SmgLevel& lv, int l) {
  if (l == 0) return SmgCsr{A.row_ptr, A.csr_col, A.csr_w};
  return SmgCsr{A.m.crow + lv.roff, A.m.ccol + lv.eoff, A.m.cw + lv.eoff};
}

// q = L x on one level (rows of <= 32 entries a thread, longer rows a warp);
// out = b - L x when b is given
__device__ void smg_apply(const SmgCsr c, int n, const double* x, const double* b, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int e0 = c.rp[i], e1 = c.rp[i + 1];
    if (e1 - e0 > 32) continue;
    const double xi = x[i];
    double acc = 0.0;
    for (int j = e0; j < e1; ++j) acc += c.w[j] * (xi - x[c.col[j]]);
    out[i] = b ? b[i] - acc : acc;
  }
  for (int i = wid; i < n; i += nw) {
    const int e0 = c.rp[i], e1 = c.rp[i + 1];
    if (e1 - e0 <= 32) continue;
    const double xi = x[i];
    double acc = 0.0;
    for (int j = e0 + lane; j < e1; j += 32) acc += c.w[j] * (xi - x[c.col[j]]);
    acc = warp_sum_d(acc);
    if (lane == 0) out[i] = b ? b[i] - acc : acc;
  }
  __syncthreads();
}

// strongest neighbour of every node (largest weight, ties to the smaller index; -1 if none)
__device__ void smg_strongest(const SmgCsr c, int n, int* best) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int e0 = c.rp[i], e1 = c.rp[i + 1];
    if (e1 - e0 > 32) continue;
    double bw = 0.0;
    int bj = -1;
    for (int j = e0; j < e1; ++j) {
      const double w = c.w[j];
      const int cj = c.col[j];
      if (w > bw || (w == bw && bj >= 0 && cj < bj)) { bw = w; bj = cj; }
    }
    best[i] = bw > 0.0 ? bj : -1;
  }
  for (int i = wid; i < n; i += nw) {
    const int e0 = c.rp[i], e1 = c.rp[i + 1];
    if (e1 - e0 <= 32) continue;
    double bw = 0.0;
    int bj = 0x7fffffff;
    for (int j = e0 + lane; j < e1; j += 32) {
      const double w = c.w[j];
      const int cj = c.col[j];
      if (w > bw || (w == bw && cj < bj)) { bw = w; bj = cj; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double w2 = __shfl_xor_sync(NI_FULL, bw, o);
      const int j2 = __shfl_xor_sync(NI_FULL, bj, o);
      if (w2 > bw || (w2 == bw && j2 < bj)) { bw = w2; bj = j2; }
    }
    if (lane == 0) best[i] = bw > 0.0 ? bj : -1;
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned smg_hash(unsigned long long key, int bits) {
  return (unsigned)((key * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

// ---------------------------------------------------------------------------
// the solve
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SMG_THREADS) k_scale_mgcg(ScaleMgArgs A) {
  __shared__ double sh[40];
  __shared__ int shi[40];
  __shared__ SmgLevel lev[SMG_LMAX];
  __shared__ int s_L, s_stop, s_dense;
  __shared__ double chol[SMG_DENSE * SMG_DENSE];
  DevState* st = A.st;
  if (*(volatile int*)&st->converged) return;
  const int K = st->K, P = st->nP;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  const ScaleMgScratch& m = A.m;

  // ---- level 0 ----
  for (int c = tid; c < K; c += nthr) {
    const double d = A.diag[c];
    m.nd[c] = d;
    m.ninv[c] = d > 0.0 ? 1.0 / d : 0.0;
  }
  if (tid == 0) {
    lev[0] = SmgLevel{K, P, 0, 0, 0, 0};
    s_L = 0;
  }
  __syncthreads();

  // ---- hierarchy ----
  for (int L = 0; L + 1 < SMG_LMAX; ++L) {
    const SmgLevel cur = lev[L];
    if (cur.n <= SMG_DENSE) break;
    const SmgCsr c = smg_csr(A, cur, L);
    int* best = m.nbest + cur.noff;
    int* par = m.npar + cur.noff;
    smg_strongest(c, cur.n, best);
    for (int i = tid; i < cur.n; i += nthr) par[i] = i;
    __syncthreads();
    for (int i = tid; i < cur.n; i += nthr)
      if (best[i] >= 0) uf_unite(par, i, best[i]);
    __syncthreads();
    for (int i = tid; i < cur.n; i += nthr) par[i] = uf_find(par, i);
    __syncthreads();
    int* rank = m.nrank + cur.noff;
    const int nc = smg_scan(cur.n, [&](int i) { return par[i] == i ? 1 : 0; }, rank, shi);
    // stop: too little coarsening, or the pools would overflow
    if (tid == 0) {
      const SmgLevel nl{nc, 0, cur.noff + cur.n, 0, 0, 0};
      s_stop = (nc > (cur.n * 9) / 10) || (nl.noff + nc > m.ncap) || nc < 1;
    }
    __syncthreads();
    if (s_stop) break;
    int* agg = m.nagg + cur.noff;
    for (int i = tid; i < cur.n; i += nthr) agg[i] = rank[par[i]];
    // hash table of coarse pairs: at least 2 slots per level-L pair
    int bits = 10;
    while ((1 << bits) < 2 * cur.np && bits < 30) ++bits;
    const int hs = 1 << bits;
    if (tid == 0) s_stop = hs > m.hcap;
    for (int h = tid; h < min(hs, m.hcap); h += nthr) m.hkey[h] = SMG_EMPTY;
    __syncthreads();
    if (s_stop) break;
    int* slot = (L == 0) ? m.pslot : m.pslot + m.ecap + cur.poff;
    for (int q = tid; q < cur.np; q += nthr) {
      const int lo = (L == 0) ? A.p_lo[q] : m.plo[cur.poff + q];
      const int hi = (L == 0) ? A.p_hi[q] : m.phi[cur.poff + q];
      const int a = agg[lo], b = agg[hi];
      int sl = -1;
      if (a != b) {
        const unsigned long long key = ((unsigned long long)min(a, b) << 32) | (unsigned)max(a, b);
        unsigned h = smg_hash(key, bits);
        for (int probe = 0; probe < hs; ++probe) {
          const unsigned long long old = atomicCAS(&m.hkey[h], SMG_EMPTY, key);
          if (old == SMG_EMPTY || old == key) { sl = (int)h; break; }
          h = (h + 1) & (hs - 1);
        }
      }
      slot[q] = sl;
    }
    __syncthreads();
    const int ncp = smg_scan(hs, [&](int h) { return m.hkey[h] != SMG_EMPTY ? 1 : 0; }, m.hidx, shi);
    // the new level's pools
    const int poff = (L == 0) ? 0 : cur.poff + cur.np;
    const int roff = (L == 0) ? 0 : cur.roff + cur.n + 1;
    const int eoff = (L == 0) ? 0 : cur.eoff + 2 * cur.np;
    if (tid == 0) s_stop = (poff + ncp > m.pcap) || (roff + nc + 1 > m.ncap + SMG_LMAX) || (eoff + 2 * ncp > 2 * m.pcap);
    __syncthreads();
    if (s_stop) break;
    for (int h = tid; h < hs; h += nthr) {
      const unsigned long long key = m.hkey[h];
      if (key == SMG_EMPTY) continue;
      const int idx = m.hidx[h];
      m.plo[poff + idx] = (int)(key >> 32);
      m.phi[poff + idx] = (int)(key & 0xffffffffull);
      m.pw[poff + idx] = 0.0;
    }
    int* cnt = m.nbest + cur.noff + cur.n;   // scratch: counters of the new level's rows
    for (int a = tid; a < nc; a += nthr) cnt[a] = 0;
    __syncthreads();
    for (int q = tid; q < cur.np; q += nthr) {
      const int sl = slot[q];
      if (sl < 0) continue;
      const double w = (L == 0) ? A.p_acc[3 * q] : m.pw[cur.poff + q];
      if (w != 0.0) atomicAdd(&m.pw[poff + m.hidx[sl]], w);
    }
    for (int p = tid; p < ncp; p += nthr) {
      atomicAdd(&cnt[m.plo[poff + p]], 1);
      atomicAdd(&cnt[m.phi[poff + p]], 1);
    }
    __syncthreads();
    int* rp = m.crow + roff;
    const int nent = smg_scan(nc, [&](int a) { return cnt[a]; }, rp, shi);
    if (tid == 0) rp[nc] = nent;
    for (int a = tid; a < nc; a += nthr) cnt[a] = rp[a];   // cursors
    __syncthreads();
    for (int p = tid; p < ncp; p += nthr) {
      const int a = m.plo[poff + p], b = m.phi[poff + p];
      const double w = m.pw[poff + p];
      const int ea = atomicAdd(&cnt[a], 1), eb = atomicAdd(&cnt[b], 1);
      m.ccol[eoff + ea] = b;
      m.cw[eoff + ea] = w;
      m.ccol[eoff + eb] = a;
      m.cw[eoff + eb] = w;
    }
    __syncthreads();
    const int noff = cur.noff + cur.n;
    for (int a = tid; a < nc; a += nthr) {
      double d = 0.0;
      for (int j = rp[a]; j < rp[a + 1]; ++j) d += m.cw[eoff + j];
      m.nd[noff + a] = d;
      m.ninv[noff + a] = d > 0.0 ? 1.0 / d : 0.0;
    }
    if (tid == 0) {
      lev[L + 1] = SmgLevel{nc, ncp, noff, poff, roff, eoff};
      s_L = L + 1;
    }
    __syncthreads();
  }
  const int Lc = s_L;
  const SmgLevel cl = lev[Lc];

  // ---- coarsest level: dense Cholesky of (L + eps I) when small enough ----
  if (tid == 0) s_dense = (cl.n <= SMG_DENSE) ? 1 : 0;
  __syncthreads();
  if (s_dense) {
    const int n = cl.n;
    for (int e = tid; e < SMG_DENSE * SMG_DENSE; e += nthr) chol[e] = 0.0;
    __syncthreads();
    double dmax = 0.0;
    for (int i = 0; i < n; ++i) dmax = fmax(dmax, m.nd[cl.noff + i]);
    const double eps = 1e-8 * (dmax > 0.0 ? dmax : 1.0);
    const SmgCsr c = smg_csr(A, cl, Lc);
    for (int i = tid; i < n; i += nthr) {
      // an isolated node (a whole connected block in one aggregate) gets x = 0
      const double di = m.nd[cl.noff + i];
      chol[i * SMG_DENSE + i] = di > 0.0 ? di + eps : 1.0;
      for (int j = c.rp[i]; j < c.rp[i + 1]; ++j) chol[i * SMG_DENSE + c.col[j]] -= c.w[j];
    }
    __syncthreads();
    if (wid == 0) {   // right-looking Cholesky, lane i owns row i; the lower triangle is kept
      for (int k = 0; k < n; ++k) {
        const double pkk = sqrt(fmax(chol[k * SMG_DENSE + k], eps));
        __syncwarp();
        if (lane == k) chol[k * SMG_DENSE + k] = pkk;
        __syncwarp();
        const double lik = (lane > k && lane < n) ? chol[lane * SMG_DENSE + k] / pkk : 0.0;
        __syncwarp();
        if (lane > k && lane < n) chol[lane * SMG_DENSE + k] = lik;
        __syncwarp();
        for (int j = k + 1; j < n; ++j) {
          const double ljk = __shfl_sync(NI_FULL, lik, j);
          if (lane >= j && lane < n) chol[lane * SMG_DENSE + j] -= lik * ljk;
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }

  // ---- PCG (the same recurrence and stop test as k_scale_cg) ----
  auto vcycle = [&](const double* rin, double* zout) {
    // level 0 vectors: b = rin, x = zout; coarse vectors in the node pool
    for (int l = 0; l <= Lc; ++l) {
      const SmgLevel lv = lev[l];
      if (l > 0)
        for (int i = tid; i < lv.n; i += nthr) m.nb[lv.noff + i] = 0.0;
    }
    __syncthreads();
    for (int l = 0; l < Lc; ++l) {
      const SmgLevel lv = lev[l];
      const double* b = (l == 0) ? rin : m.nb + lv.noff;
      double* x = (l == 0) ? zout : m.nx + lv.noff;
      for (int i = tid; i < lv.n; i += nthr) x[i] = SMG_OMEGA * m.ninv[lv.noff + i] * b[i];
      __syncthreads();
      smg_apply(smg_csr(A, lv, l), lv.n, x, b, m.nr + lv.noff);
      const SmgLevel nl = lev[l + 1];
      for (int i = tid; i < lv.n; i += nthr) {
        const double ri = m.nr[lv.noff + i];
        if (ri != 0.0) atomicAdd(&m.nb[nl.noff + m.nagg[lv.noff + i]], ri);
      }
      __syncthreads();
    }
    {
      const double* b = (Lc == 0) ? rin : m.nb + cl.noff;
      double* x = (Lc == 0) ? zout : m.nx + cl.noff;
      if (s_dense) {
        const int n = cl.n;
        if (wid == 0) {
          double y = (lane < n && m.nd[cl.noff + lane] > 0.0) ? b[lane] : 0.0;
          for (int k = 0; k < n; ++k) {   // forward: L y = b
            const double lkk = chol[k * SMG_DENSE + k];
            const double yk = __shfl_sync(NI_FULL, y, k) / lkk;
            if (lane == k) y = yk;
            if (lane > k && lane < n) y -= chol[lane * SMG_DENSE + k] * yk;
          }
          for (int k = n - 1; k >= 0; --k) {   // backward: L^T x = y
            const double lkk = chol[k * SMG_DENSE + k];
            const double xk = __shfl_sync(NI_FULL, y, k) / lkk;
            if (lane == k) y = xk;
            if (lane < k) y -= chol[k * SMG_DENSE + lane] * xk;
          }
          if (lane < n) x[lane] = y;
        }
        __syncthreads();
      } else {
        for (int i = tid; i < cl.n; i += nthr) x[i] = SMG_OMEGA * m.ninv[cl.noff + i] * b[i];
        __syncthreads();
        for (int sw = 1; sw < SMG_COARSE_SWEEPS; ++sw) {
          smg_apply(smg_csr(A, cl, Lc), cl.n, x, b, m.nr + cl.noff);
          for (int i = tid; i < cl.n; i += nthr) x[i] += SMG_OMEGA * m.ninv[cl.noff + i] * m.nr[cl.noff + i];
          __syncthreads();
        }
      }
    }
    for (int l = Lc - 1; l >= 0; --l) {
      const SmgLevel lv = lev[l], nl = lev[l + 1];
      const double* b = (l == 0) ? rin : m.nb + lv.noff;
      double* x = (l == 0) ? zout : m.nx + lv.noff;
      const double* xc = m.nx + nl.noff;
      for (int i = tid; i < lv.n; i += nthr) x[i] += xc[m.nagg[lv.noff + i]];
      __syncthreads();
      smg_apply(smg_csr(A, lv, l), lv.n, x, b, m.nr + lv.noff);
      for (int i = tid; i < lv.n; i += nthr) x[i] += SMG_OMEGA * m.ninv[lv.noff + i] * m.nr[lv.noff + i];
      __syncthreads();
    }
  };

  double ga2 = 0, gg = 0;
  for (int c = tid; c < K; c += nthr) {
    const double rc = A.g[c];
    A.s[c] = 0.0;
    A.r[c] = rc;
    ga2 += A.gabs[c] * A.gabs[c];
    gg += rc * rc;
  }
  ga2 = smg_sum(ga2, sh);
  gg = smg_sum(gg, sh);
  vcycle(A.r, A.z);
  double rz = 0;
  for (int c = tid; c < K; c += nthr) {
    A.pp[c] = A.z[c];
    rz += A.r[c] * A.z[c];
  }
  rz = smg_sum(rz, sh);
  const double floor2 = (64.0 * 1.1102230246251565e-16) * (64.0 * 1.1102230246251565e-16) * ga2;
  const double stop2 = fmax(A.tol2 * gg, floor2);
  int it = 0;
  bool done = !(gg > 0.0) || gg <= stop2;
  const SmgCsr c0 = smg_csr(A, lev[0], 0);
  while (!done && it < A.maxit) {
    smg_apply(c0, K, A.pp, nullptr, A.qq);
    double pq = 0;
    for (int c = tid; c < K; c += nthr) pq += A.pp[c] * A.qq[c];
    pq = smg_sum(pq, sh);
    const double alpha = pq > 0.0 ? rz / pq : 0.0;
    double rr = 0;
    for (int c = tid; c < K; c += nthr) {
      A.s[c] += alpha * A.pp[c];
      const double rc = A.r[c] - alpha * A.qq[c];
      A.r[c] = rc;
      rr += rc * rc;
    }
    rr = smg_sum(rr, sh);
    ++it;
    done = rr <= stop2 || !(pq > 0.0);
    if (done) break;
    vcycle(A.r, A.z);
    double rzn = 0;
    for (int c = tid; c < K; c += nthr) rzn += A.r[c] * A.z[c];
    rzn = smg_sum(rzn, sh);
    const double beta = rz > 0.0 ? rzn / rz : 0.0;
    rz = rzn;
    for (int c = tid; c < K; c += nthr) A.pp[c] = A.z[c] + beta * A.pp[c];
    __syncthreads();
  }
  // energy of the solved system, update, stop test (as in k_scale_cg)
  double en = 0;
  for (int p = tid; p < P; p += nthr) {
    const double D = A.s[A.p_lo[p]] - A.s[A.p_hi[p]];
    en += A.p_acc[3 * p] * D * D + 2.0 * A.p_acc[3 * p + 1] * D + A.p_acc[3 * p + 2];
  }
  en = smg_sum(en, sh);
  for (int c = tid; c < K; c += nthr) A.soff[c] += A.s[c];
  if (tid == 0) {
    const int t = st->t + 1;
    st->t = t;
    if (t <= NI_MAX_T) st->E[t] = en;
    st->scale_cg_last = it;
    if (it > st->scale_cg_iters) st->scale_cg_iters = it;
    if (it >= A.maxit && !done) st->err |= NI_DEV_ERR_SCALE_NOCONV;
    bool conv = t >= A.T;
    if (!conv && t >= 4 && t <= NI_MAX_T) {
      const double e0 = st->E[t - 1];
      conv = (e0 < 1e-300) || (fabs(en - e0) / e0 < A.dE_max);
    }
    st->converged = conv ? 1 : 0;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
void free_scale_mg(ni_handle* h) {
  ScaleMgScratch* m = h->smg;
  if (!m) return;
  void* ps[] = {m->nd, m->ninv, m->nx, m->nb, m->nr, m->nagg, m->npar, m->nbest, m->nrank, m->plo, m->phi,
                m->pslot, m->pw, m->crow, m->ccol, m->cw, m->hkey, m->hidx};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete m;
  h->smg = nullptr;
}

static cudaError_t scale_mg_capacity(ni_handle* h) {
  const int ncap = 3 * h->Kcap + 64, pcap = 2 * h->Ecap + 64, ecap = h->Ecap;
  int hcap = 1024;
  while (hcap < 2 * h->Ecap && hcap < (1 << 30)) hcap <<= 1;
  ScaleMgScratch* m = h->smg;
  if (m && m->ncap >= ncap && m->pcap >= pcap && m->ecap >= ecap && m->hcap >= hcap) return cudaSuccess;
  free_scale_mg(h);
  m = h->smg = new ScaleMgScratch();
  cudaError_t e = cudaSuccess;
  double** dv[] = {&m->nd, &m->ninv, &m->nx, &m->nb, &m->nr};
  for (double** p : dv)
    if (e == cudaSuccess) e = cudaMalloc((void**)p, (size_t)ncap * sizeof(double));
  int** iv[] = {&m->nagg, &m->npar, &m->nrank};
  for (int** p : iv)
    if (e == cudaSuccess) e = cudaMalloc((void**)p, (size_t)ncap * sizeof(int));
  // nbest also holds the next level's row counters
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->nbest, (size_t)2 * ncap * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->plo, (size_t)pcap * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->phi, (size_t)pcap * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->pslot, ((size_t)pcap + ecap) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->pw, (size_t)pcap * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->crow, ((size_t)ncap + SMG_LMAX) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->ccol, (size_t)2 * pcap * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->cw, (size_t)2 * pcap * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->hkey, (size_t)hcap * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->hidx, (size_t)hcap * sizeof(int));
  if (e != cudaSuccess) {
    free_scale_mg(h);
    return e;
  }
  m->ncap = ncap;
  m->pcap = pcap;
  m->ecap = ecap;
  m->hcap = hcap;
  return cudaSuccess;
}

bool scale_mg_usable(ni_handle* h) { return h->cfg.scale_precond == 1 && h->Kcap <= 8192; }

// Scratch sized by the component and edge capacities; called on the host after
// the first partition build, outside any stream capture.
ni_status scale_mg_prepare(ni_handle* h) {
  if (!scale_mg_usable(h)) return NI_OK;
  return ni_cuda_check(h, scale_mg_capacity(h), "scale multigrid scratch");
}

ni_status scale_mg_launch(ni_handle* h, double* diag, double* g, double* gabs, double* sv, cudaStream_t s) {
  if (!h->smg) return ni_fail(h, NI_ERR_STATE, "scale multigrid scratch missing");
  ScaleMgArgs a;
  a.st = h->st;
  a.row_ptr = h->row_ptr; a.csr_col = h->csr_col; a.csr_w = h->csr_w;
  a.p_lo = h->p_lo; a.p_hi = h->p_hi; a.p_acc = h->p_acc;
  a.diag = diag; a.g = g; a.gabs = gabs;
  const size_t kc = (size_t)h->Kcap;
  a.s = sv; a.r = sv + kc; a.z = sv + 2 * kc; a.pp = sv + 3 * kc; a.qq = sv + 4 * kc;
  a.soff = h->soff;
  a.tol2 = h->cfg.scale_rtol * h->cfg.scale_rtol;
  a.maxit = h->cfg.scale_maxit > 0 ? h->cfg.scale_maxit : std::min(4 * h->Kcap + 100, 200000);
  a.T = h->cfg.T;
  a.dE_max = h->cfg.dE_max;
  a.m = *h->smg;
  k_scale_mgcg<<<1, SMG_THREADS, 0, s>>>(a); NI_COUNT(h);
  return ni_cuda_check(h, cudaGetLastError(), "scale multigrid PCG");
}
