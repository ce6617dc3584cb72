// Component fill (Sec. 3.3, Eqs. 9-10; rows a3-a4) and the per-pixel output (row a8).
//
// Setup (k_edge_setup, k_diag_rhs): for every edge (a, b) to the right or below
// of a valid pixel a,
//   omega~_{b->a} (Eq. 3)  -- perspective: with A = n_a.tau_a, B = n_b.tau_b and
//       d_a = n_a.(tau_b - tau_a), d_b = n_b.(tau_b - tau_a), the midpoint ray
//       tau_m = (tau_a + tau_b) / 2 turns Eq. 3 into
//       log(1 + (d_a B + A d_b) / (A (2 B - d_b))),
//       an algebraically identical form that avoids cancelling two nearly
//       equal products in float32;  orthographic: (n_ax/n_az + n_bx/n_bz) / 2
//       (n_y for vertical edges);
//   gamma_{b->a} = f n_a.tau_a (Eq. 6), f = f_x horizontally, f_y vertically;
//   the fill weight of an intra-component edge at z~ = 0, where w^BiNI = 1/2:
//       w_ab = W_{b->a} + W_{a->b} = (gamma_{b->a}^2 + gamma_{a->b}^2) / 2,
//   which is the edge's entry in A_c^T W_c A_c (rows of both directions);
//   right-hand side b_a = sum_b w_ab omega~_{b->a} (= A_c^T W_c b_c);
//   Jacobi diagonal d_a = sum_b w_ab.
//
// Solve: Jacobi-preconditioned CG on the block-diagonal weighted Laplacian,
//   matrix-free 5-point stencil in float32, reductions in float64 (or float32
//   warp/CTA trees, precision = 1):
//   plain   (batched = 0): one global CG; three kernels per iteration,
//           iteration chunks replayed from a CUDA graph;
//   batched (batched = 1): one cooperative persistent launch with a step
//           length, direction update and convergence mask per component.
// Both start from x0 (0 or the warm start), project the right-hand side and the
// result to zero mean per component (the gauge CG from 0 reaches).
#include <algorithm>
#include <vector>

#include "ni_internal.cuh"

static int grid_px(ni_handle* h, long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  long long cap = (long long)h->num_sms * 8;
  return (int)std::max(1LL, std::min(b, cap));
}

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
__global__ void k_edge_setup(const float4* __restrict__ nrm, const uint8_t* __restrict__ mask,
                             const int* __restrict__ labels, int H, int W, int persp, float fx,
                             float fy, float cx, float cy, float2* __restrict__ omega,
                             float* __restrict__ ntau, float2* __restrict__ wfill) {
  const int N = H * W;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    float2 om = make_float2(0.f, 0.f), w = make_float2(0.f, 0.f);
    float A = 0.f;
    if (mask[a]) {
      const int u = a % W, v = a / W;
      const float4 na = ldg4(&nrm[a]);
      const float tax = persp ? (u - cx) / fx : 0.f, tay = persp ? (v - cy) / fy : 0.f;
      A = persp ? (na.x * tax + na.y * tay + na.z) : na.z;
      const int la = labels[a];
      if (u + 1 < W && mask[a + 1]) {
        const float4 nb = ldg4(&nrm[a + 1]);
        float B;
        if (persp) {
          const float tbx = (u + 1 - cx) / fx;
          B = nb.x * tbx + nb.y * tay + nb.z;
          const float da = na.x / fx, db = nb.x / fx;
          const float qv = (da * B + A * db) / (A * (2.f * B - db));
          om.x = (qv > -1.f) ? log1pf(qv) : logf(fabsf(1.f + qv));
          if (labels[a + 1] == la) w.x = 0.5f * fx * fx * (A * A + B * B);
        } else {
          B = nb.z;
          om.x = 0.5f * (na.x / na.z + nb.x / nb.z);
          if (labels[a + 1] == la) w.x = 0.5f * (A * A + B * B);
        }
      }
      if (v + 1 < H && mask[a + W]) {
        const float4 nb = ldg4(&nrm[a + W]);
        float B;
        if (persp) {
          const float tby = (v + 1 - cy) / fy;
          B = nb.x * tax + nb.y * tby + nb.z;
          const float da = na.y / fy, db = nb.y / fy;
          const float qv = (da * B + A * db) / (A * (2.f * B - db));
          om.y = (qv > -1.f) ? log1pf(qv) : logf(fabsf(1.f + qv));
          if (labels[a + W] == la) w.y = 0.5f * fy * fy * (A * A + B * B);
        } else {
          B = nb.z;
          om.y = 0.5f * (na.y / na.z + nb.y / nb.z);
          if (labels[a + W] == la) w.y = 0.5f * (A * A + B * B);
        }
      }
    }
    omega[a] = om;
    ntau[a] = A;
    wfill[a] = w;
  }
}

// Jacobi inverse diagonal and right-hand side b_a = sum_b w_ab omega~_{b->a}.
__global__ void k_diag_rhs(const float2* __restrict__ wfill, const float2* __restrict__ omega, int H,
                           int W, float* __restrict__ invd, float* __restrict__ rhs) {
  const int N = H * W;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    const int u = a % W, v = a / W;
    const float2 w = wfill[a], om = omega[a];
    float wl = 0.f, wu = 0.f, ol = 0.f, ou = 0.f;
    if (u > 0) { wl = wfill[a - 1].x; ol = omega[a - 1].x; }
    if (v > 0) { wu = wfill[a - W].y; ou = omega[a - W].y; }
    const float d = w.x + w.y + wl + wu;
    invd[a] = d > 0.f ? 1.0f / d : 0.f;
    // omega~_{l->a} = -omega~_{a->l} (antisymmetry of Eq. 3)
    rhs[a] = w.x * om.x + w.y * om.y - wl * ol - wu * ou;
  }
}

// BiNI reweighting sweep of the fill (n_fill_irls > 1): directed weights at the
// current z~ (Eq. 5), the opposite neighbour restricted to the component.
__device__ __forceinline__ float bini_w(float gam, float za, float zb, float zo, bool has_o, float k) {
  float g2 = gam * gam;
  float dop = has_o ? (zo - za) * (zo - za) : 0.f;
  float arg = g2 * (dop - (zb - za) * (zb - za));
  return g2 / (1.f + expf(-k * arg));
}

__global__ void k_fill_reweight(const float* __restrict__ ntau, const int* __restrict__ labels,
                                const float* __restrict__ x, int H, int W, int persp, float fx,
                                float fy, float k, float2* __restrict__ wfill) {
  const int N = H * W;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    float2 w = wfill[a];
    const int la = labels[a];
    const int u = a % W, v = a / W;
    if (la >= 0 && w.x > 0.f) {
      const int b = a + 1;
      float f = persp ? fx : 1.f;
      float gba = f * ntau[a], gab = f * ntau[b];
      bool ho_a = (u > 0) && labels[a - 1] == la;
      bool ho_b = (u + 2 < W) && labels[b + 1] == la;
      w.x = bini_w(gba, x[a], x[b], ho_a ? x[a - 1] : 0.f, ho_a, k) +
            bini_w(gab, x[b], x[a], ho_b ? x[b + 1] : 0.f, ho_b, k);
    }
    if (la >= 0 && w.y > 0.f) {
      const int b = a + W;
      float f = persp ? fy : 1.f;
      float gba = f * ntau[a], gab = f * ntau[b];
      bool ho_a = (v > 0) && labels[a - W] == la;
      bool ho_b = (v + 2 < H) && labels[b + W] == la;
      w.y = bini_w(gba, x[a], x[b], ho_a ? x[a - W] : 0.f, ho_a, k) +
            bini_w(gab, x[b], x[a], ho_b ? x[b + W] : 0.f, ho_b, k);
    }
    wfill[a] = w;
  }
}

// Per-component sums (slot0 += val, slot1 += 1) over valid pixels.
__global__ void k_comp_sum(const int* __restrict__ labels, const float* __restrict__ val, int N,
                           double* __restrict__ acc) {
  const int stride = gridDim.x * blockDim.x;
  const int nIter = (N + stride - 1) / stride;
  for (int it = 0; it < nIter; ++it) {
    int i = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
    int c = (i < N) ? labels[i] : -1;
    double v[2] = {c >= 0 ? (double)val[i] : 0.0, c >= 0 ? 1.0 : 0.0};
    seg_add_d<2>(acc, 2, c, v);
  }
}

__global__ void k_comp_sub_mean(const int* __restrict__ labels, int N, const double* __restrict__ acc,
                                float* __restrict__ val) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int c = labels[i];
    if (c >= 0) {
      double cnt = acc[2 * (size_t)c + 1];
      if (cnt > 0) val[i] = (float)((double)val[i] - acc[2 * (size_t)c] / cnt);
    }
  }
}

// ---------------------------------------------------------------------------
// stencil helpers
// ---------------------------------------------------------------------------
struct Stencil {
  float wr, wd, wl, wu;
};

__device__ __forceinline__ Stencil load_stencil(const float2* __restrict__ wfill, int a, int u, int v,
                                                int W) {
  const float2 w = wfill[a];
  Stencil s;
  s.wr = w.x;
  s.wd = w.y;
  s.wl = (u > 0) ? wfill[a - 1].x : 0.f;
  s.wu = (v > 0) ? wfill[a - W].y : 0.f;
  return s;
}

// (A p)_a = sum_b w_ab (p_a - p_b), evaluated on the differences: the form
// d_a p_a - sum_b w_ab p_b cancels catastrophically in float32 once p is smooth,
// which leaves q = A p inconsistent with p^T A p and stalls CG.
__device__ __forceinline__ float apply_stencil(const Stencil& s, const float* __restrict__ p, int a,
                                               int W, float pa) {
  float acc = 0.f;
  if (s.wr != 0.f) acc += s.wr * (pa - p[a + 1]);
  if (s.wd != 0.f) acc += s.wd * (pa - p[a + W]);
  if (s.wl != 0.f) acc += s.wl * (pa - p[a - 1]);
  if (s.wu != 0.f) acc += s.wu * (pa - p[a - W]);
  return acc;
}

// ---------------------------------------------------------------------------
// plain Jacobi-PCG (global step lengths)
// ---------------------------------------------------------------------------
template <typename Acc>
__device__ __forceinline__ void block_atomic_add(double* dst, Acc v, double* sh) {
  double t = block_sum_d((double)v, sh);
  if (threadIdx.x == 0 && t != 0.0) atomicAdd(dst, t);
}

template <typename Acc>
__global__ void k_cg_init(const float2* __restrict__ wfill, const float* __restrict__ invd,
                          const float* __restrict__ rhs, const float* __restrict__ x,
                          float* __restrict__ r, float* __restrict__ p, int H, int W, DevState* st) {
  __shared__ double sh[33];
  const int N = H * W;
  Acc rz = 0, rr = 0, bb = 0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    const int u = a % W, v = a / W;
    Stencil s = load_stencil(wfill, a, u, v, W);
    float ra = rhs[a] - apply_stencil(s, x, a, W, x[a]);
    if (invd[a] == 0.f) ra = 0.f;
    float z = ra * invd[a];
    r[a] = ra;
    p[a] = z;
    rz += (Acc)(ra * z);
    rr += (Acc)(ra * ra);
    bb += (Acc)(rhs[a] * rhs[a]);
  }
  block_atomic_add(&st->cg[CG_RZ], rz, sh);
  block_atomic_add(&st->cg[CG_RR], rr, sh);
  block_atomic_add(&st->cg[CG_BB], bb, sh);
}

__global__ void k_cg_init_done(DevState* st, double tol2) {
  st->cg_it = 0;
  st->cg_done = (st->cg[CG_BB] <= 0.0) || (st->cg[CG_RR] <= tol2 * st->cg[CG_BB]);
  st->cg[CG_RR] = 0.0;
  st->cg[CG_PAP] = 0.0;
  st->cg[CG_RZNEW] = 0.0;
}

template <typename Acc>
__global__ void k_cg_spmv(const float2* __restrict__ wfill, const float* __restrict__ p,
                          float* __restrict__ q, int H, int W, DevState* st) {
  __shared__ double sh[33];
  if (*(volatile int*)&st->cg_done) return;
  const int N = H * W;
  Acc pap = 0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    const int u = a % W, v = a / W;
    Stencil s = load_stencil(wfill, a, u, v, W);
    const float pa = p[a];
    q[a] = apply_stencil(s, p, a, W, pa);
    // p^T A p as the sum over edges of w (p_a - p_b)^2 (no cancellation)
    if (s.wr != 0.f) { float d = pa - p[a + 1]; pap += (Acc)(s.wr * d * d); }
    if (s.wd != 0.f) { float d = pa - p[a + W]; pap += (Acc)(s.wd * d * d); }
  }
  block_atomic_add(&st->cg[CG_PAP], pap, sh);
}

template <typename Acc>
__global__ void k_cg_update(const float* __restrict__ invd, const float* __restrict__ p,
                            const float* __restrict__ q, float* __restrict__ x, float* __restrict__ r,
                            int N, DevState* st) {
  __shared__ double sh[33];
  if (*(volatile int*)&st->cg_done) return;
  const double pap = *(volatile double*)&st->cg[CG_PAP];
  const float alpha = pap > 0.0 ? (float)(*(volatile double*)&st->cg[CG_RZ] / pap) : 0.f;
  Acc rz = 0, rr = 0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    const float pa = p[a];
    x[a] += alpha * pa;
    const float ra = r[a] - alpha * q[a];
    r[a] = ra;
    const float z = ra * invd[a];
    rz += (Acc)(ra * z);
    rr += (Acc)(ra * ra);
  }
  block_atomic_add(&st->cg[CG_RZNEW], rz, sh);
  block_atomic_add(&st->cg[CG_RR], rr, sh);
}

__global__ void k_cg_dir(const float* __restrict__ invd, const float* __restrict__ r,
                         float* __restrict__ p, int N, DevState* st, unsigned int* counter,
                         double tol2, int maxit) {
  if (*(volatile int*)&st->cg_done) return;
  const double rz = *(volatile double*)&st->cg[CG_RZ];
  const float beta = rz > 0.0 ? (float)(*(volatile double*)&st->cg[CG_RZNEW] / rz) : 0.f;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x)
    p[a] = r[a] * invd[a] + beta * p[a];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    if (prev == gridDim.x - 1) {   // last block: scalar bookkeeping for the next iteration
      volatile double* c = st->cg;
      double rr = c[CG_RR];
      const double pap = c[CG_PAP];
      c[CG_RZ] = c[CG_RZNEW];
      c[CG_RZNEW] = 0.0;
      c[CG_PAP] = 0.0;
      c[CG_RR] = 0.0;
      int it = st->cg_it + 1;
      st->cg_it = it;
      // stop at the tolerance, at the iteration limit, or when the recurrence
      // has stagnated (p^T A p no longer positive: p lies in the null space)
      if (rr <= tol2 * c[CG_BB] || it >= maxit || !(pap > 0.0) || !(rr == rr)) st->cg_done = 1;
      *counter = 0u;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
// batched persistent Jacobi-PCG: per-component step lengths and masks
// ---------------------------------------------------------------------------
// Per-component slots in cacc (each Kcap doubles):
//   0,1 rz (iteration parity)   2,3 p^T A p   4,5 rz_new   6,7 r^T r   8 b^T b
//   9 sum x   10 count
// cflag: [0, Kcap) active flag parity 0, [Kcap, 2 Kcap) parity 1, [2 Kcap, 3 Kcap) iterations
struct PcgArgs {
  const float2* wfill;
  const float* invd;
  const float* rhs;
  const int* labels;
  float* x;
  float* r;
  float* p;
  float* q;
  double* cacc;
  int* cflag;
  DevState* st;
  int* active_cnt;   // [2]
  int H, W, K, Kcap;
  int maxit;
  double tol2;
};

template <bool FP64>
__device__ __forceinline__ void seg_add_one(double* acc, int key, float a) {
  if (FP64) {
    double v[1] = {(double)a};
    seg_add_d<1>(acc, 1, key, v);
  } else {
    float v[1] = {a};
    seg_add_f<1>(acc, 1, key, v);
  }
}

template <bool FP64>
__global__ void __launch_bounds__(256) k_pcg_batched(PcgArgs A) {
  const int H = A.H, W = A.W, N = H * W, K = A.K, Kc = A.Kcap;
  double* rzb0 = A.cacc + 0 * (size_t)Kc;
  double* pap0 = A.cacc + 2 * (size_t)Kc;
  double* rzn0 = A.cacc + 4 * (size_t)Kc;
  double* rr0 = A.cacc + 6 * (size_t)Kc;
  double* bb = A.cacc + 8 * (size_t)Kc;
  double* sx = A.cacc + 9 * (size_t)Kc;
  int* iters = A.cflag + 2 * (size_t)Kc;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthr = gridDim.x * blockDim.x;
  const int nIter = (N + nthr - 1) / nthr;   // uniform trip count for the warp-level reductions
  int* err = &A.st->err;

  // prologue: r = b - A x0, p = z = D^-1 r, per-component r.z, r.r, b.b
  for (int it = 0; it < nIter; ++it) {
    const int a = it * nthr + tid;
    int c = -1;
    float rz = 0.f, rr = 0.f, bsq = 0.f;
    if (a < N) {
      c = A.labels[a];
      if (c >= 0) {
        const int u = a % W, v = a / W;
        Stencil s = load_stencil(A.wfill, a, u, v, W);
        const float id = A.invd[a];
        float ra = A.rhs[a] - apply_stencil(s, A.x, a, W, A.x[a]);
        if (id == 0.f) ra = 0.f;
        const float z = ra * id;
        A.r[a] = ra;
        A.p[a] = z;
        rz = ra * z;
        rr = ra * ra;
        bsq = A.rhs[a] * A.rhs[a];
      }
    }
    seg_add_one<FP64>(rzb0, c, rz);
    seg_add_one<FP64>(rr0 + Kc, c, rr);
    seg_add_one<FP64>(bb, c, bsq);
  }
  if (!grid_barrier(&A.st->bar, err)) return;
  for (int c = tid; c < K; c += nthr) {
    int act = (bb[c] > 0.0) && (rr0[Kc + c] > A.tol2 * bb[c]);
    A.cflag[c] = act;
    iters[c] = 0;
    if (act) atomicAdd(&A.active_cnt[1], 1);
  }
  if (!grid_barrier(&A.st->bar, err)) return;

  int it_done = 0;
  for (int iter = 0; iter < A.maxit; ++iter) {
    const int k = iter & 1, kp = k ^ 1;
    if (*(volatile int*)&A.active_cnt[kp] == 0) break;
    const int* fl = A.cflag + (size_t)k * Kc;
    // phase A: q = A p, per-component p^T A p
    for (int it = 0; it < nIter; ++it) {
      const int a = it * nthr + tid;
      int c = -1;
      float pap = 0.f;
      if (a < N) {
        int lc = A.labels[a];
        if (lc >= 0 && fl[lc]) {
          c = lc;
          const int u = a % W, v = a / W;
          Stencil s = load_stencil(A.wfill, a, u, v, W);
          const float pa = A.p[a];
          A.q[a] = apply_stencil(s, A.p, a, W, pa);
          if (s.wr != 0.f) { float d = pa - A.p[a + 1]; pap += s.wr * d * d; }
          if (s.wd != 0.f) { float d = pa - A.p[a + W]; pap += s.wd * d * d; }
        }
      }
      seg_add_one<FP64>(pap0 + (size_t)k * Kc, c, pap);
    }
    if (!grid_barrier(&A.st->bar, err)) return;
    // phase B: x += alpha p, r -= alpha q, per-component r.z and r.r
    for (int c = tid; c < K; c += nthr) pap0[(size_t)kp * Kc + c] = 0.0;
    if (tid == 0) A.active_cnt[kp] = 0;
    for (int it = 0; it < nIter; ++it) {
      const int a = it * nthr + tid;
      int c = -1;
      float rz = 0.f, rr = 0.f;
      if (a < N) {
        int lc = A.labels[a];
        if (lc >= 0 && fl[lc]) {
          c = lc;
          const double pap = pap0[(size_t)k * Kc + c];
          const float alpha = pap > 0.0 ? (float)(rzb0[(size_t)k * Kc + c] / pap) : 0.f;
          const float pa = A.p[a];
          A.x[a] += alpha * pa;
          const float ra = A.r[a] - alpha * A.q[a];
          A.r[a] = ra;
          rz = ra * ra * A.invd[a];
          rr = ra * ra;
        }
      }
      seg_add_one<FP64>(rzn0 + (size_t)k * Kc, c, rz);
      seg_add_one<FP64>(rr0 + (size_t)k * Kc, c, rr);
    }
    if (!grid_barrier(&A.st->bar, err)) return;
    // phase D: p = z + beta p; next masks
    for (int it = 0; it < nIter; ++it) {
      const int a = it * nthr + tid;
      if (a < N) {
        int c = A.labels[a];
        if (c >= 0 && fl[c]) {
          const double rzo = rzb0[(size_t)k * Kc + c];
          const float beta = rzo > 0.0 ? (float)(rzn0[(size_t)k * Kc + c] / rzo) : 0.f;
          A.p[a] = A.r[a] * A.invd[a] + beta * A.p[a];
        }
      }
    }
    for (int c = tid; c < K; c += nthr) {
      int act = fl[c];
      int nact = 0;
      if (act) {
        rzb0[(size_t)kp * Kc + c] = rzn0[(size_t)k * Kc + c];
        iters[c] += 1;
        nact = rr0[(size_t)k * Kc + c] > A.tol2 * bb[c];
      }
      A.cflag[(size_t)kp * Kc + c] = nact;
      rzn0[(size_t)kp * Kc + c] = 0.0;
      rr0[(size_t)kp * Kc + c] = 0.0;
      if (nact) atomicAdd(&A.active_cnt[k], 1);
    }
    it_done = iter + 1;
    if (!grid_barrier(&A.st->bar, err)) return;
  }
  // epilogue: statistics and zero mean per component (the gauge of CG from 0)
  const int kfin = it_done & 1;
  for (int c = tid; c < K; c += nthr) {
    atomicMax(&A.st->fill_iters, iters[c]);
    if (A.cflag[(size_t)kfin * Kc + c]) {
      atomicAdd(&A.st->fill_unconv, 1);
      atomicOr(err, NI_DEV_ERR_FILL_NOCONV);
    }
  }
  for (int it = 0; it < nIter; ++it) {
    const int a = it * nthr + tid;
    int c = (a < N) ? A.labels[a] : -1;
    double v[2] = {c >= 0 ? (double)A.x[a] : 0.0, c >= 0 ? 1.0 : 0.0};
    seg_add_d<2>(sx, 1, c, v, (size_t)Kc);   // sum x -> slot 9, count -> slot 10
  }
  if (!grid_barrier(&A.st->bar, err)) return;
  for (int a = tid; a < N; a += nthr) {
    int c = A.labels[a];
    if (c >= 0) {
      double cnt = sx[(size_t)Kc + c];
      if (cnt > 0) A.x[a] = (float)((double)A.x[a] - sx[c] / cnt);
    }
  }
  for (int c = tid; c < K; c += nthr)
    if (iters[c] > 0)
      atomicAdd(&A.st->fill_px_iters, (unsigned long long)iters[c] * (unsigned long long)sx[(size_t)Kc + c]);
}

ni_status fill_setup_launch(ni_handle* h, cudaStream_t s) {
  const int N = h->N;
  k_edge_setup<<<grid_px(h, N), 256, 0, s>>>(h->normals, h->mask, h->labels, h->H, h->W, h->persp,
                                               h->fx, h->fy, h->cx, h->cy, h->omega, h->ntau, h->wfill); NI_COUNT(h);
  k_diag_rhs<<<grid_px(h, N), 256, 0, s>>>(h->wfill, h->omega, h->H, h->W, h->invd, h->b); NI_COUNT(h);
  return ni_cuda_check(h, cudaGetLastError(), "fill setup");
}

static ni_status project_rhs(ni_handle* h, float* v, cudaStream_t s) {
  cudaMemsetAsync(h->cacc, 0, sizeof(double) * 2 * (size_t)h->Kcap, s);
  k_comp_sum<<<grid_px(h, h->N), 256, 0, s>>>(h->labels, v, h->N, h->cacc); NI_COUNT(h);
  k_comp_sub_mean<<<grid_px(h, h->N), 256, 0, s>>>(h->labels, h->N, h->cacc, v); NI_COUNT(h);
  return ni_cuda_check(h, cudaGetLastError(), "component mean");
}

static ni_status plain_solve(ni_handle* h, cudaStream_t s) {
  const int N = h->N, H = h->H, W = h->W;
  const double tol2 = h->cfg.cg_rtol * h->cfg.cg_rtol;
  const int maxit = h->cfg.cg_maxit;
  const int g = grid_px(h, N);
  unsigned int* counter = reinterpret_cast<unsigned int*>(&h->st->bar2);
  cudaMemsetAsync(&h->st->cg[0], 0, sizeof(double) * 8, s);
  cudaMemsetAsync(&h->st->bar2, 0, sizeof(GridBar), s);
  const bool f64 = h->cfg.precision == 0;
  if (f64) k_cg_init<double><<<g, 256, 0, s>>>(h->wfill, h->invd, h->b, h->x, h->r, h->p, H, W, h->st);
  else k_cg_init<float><<<g, 256, 0, s>>>(h->wfill, h->invd, h->b, h->x, h->r, h->p, H, W, h->st);
  NI_COUNT(h);
  k_cg_init_done<<<1, 1, 0, s>>>(h->st, tol2); NI_COUNT(h);
  ni_status rc = ni_cuda_check(h, cudaGetLastError(), "plain PCG init");
  if (rc != NI_OK) return rc;
  const int CHUNK = 32;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // capture one chunk of iterations; replay it until the device flag says done
  cudaStream_t cs;
  cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  const long long launches_before = h->launches;
  for (int i = 0; i < CHUNK; ++i) {
    if (f64) k_cg_spmv<double><<<g, 256, 0, cs>>>(h->wfill, h->p, h->q, H, W, h->st);
    else k_cg_spmv<float><<<g, 256, 0, cs>>>(h->wfill, h->p, h->q, H, W, h->st);
    NI_COUNT(h);
    if (f64) k_cg_update<double><<<g, 256, 0, cs>>>(h->invd, h->p, h->q, h->x, h->r, N, h->st);
    else k_cg_update<float><<<g, 256, 0, cs>>>(h->invd, h->p, h->q, h->x, h->r, N, h->st);
    NI_COUNT(h);
    k_cg_dir<<<g, 256, 0, cs>>>(h->invd, h->r, h->p, N, h->st, counter, tol2, maxit); NI_COUNT(h);
  }

  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  const long long per_chunk = h->launches - launches_before;
  h->launches = launches_before;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  rc = ni_cuda_check(h, e, "plain PCG graph");
  if (rc == NI_OK) {
    for (int done_it = 0; done_it < maxit; done_it += CHUNK) {
      cudaGraphLaunch(exec, s);
      h->launches += per_chunk;
      cudaMemcpyAsync(&h->st_host->cg_done, &h->st->cg_done, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) break;
      if (h->st_host->cg_done) break;
    }
    rc = ni_cuda_check(h, e, "plain PCG");
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  return rc;
}

__global__ void k_plain_stats(DevState* st, int maxit, double tol2) {
  st->fill_iters = st->cg_it;
  st->fill_px_iters = (unsigned long long)st->n_valid * (unsigned long long)st->cg_it;
  if (!(st->cg_done) || st->cg_it >= maxit) {
    st->fill_unconv = 1;
    st->err |= NI_DEV_ERR_FILL_NOCONV;
  }
}

static ni_status batched_solve(ni_handle* h, cudaStream_t s) {
  const bool f64 = h->cfg.precision == 0;
  void* fn = f64 ? (void*)k_pcg_batched<true> : (void*)k_pcg_batched<false>;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0);
  if (per_sm < 1) return ni_fail(h, NI_ERR_CUDA, "batched PCG: kernel cannot be resident");
  int grid = h->num_sms * std::min(per_sm, 4);
  long long need = ((long long)h->N + 255) / 256;
  if (grid > need) grid = (int)std::max(1LL, need);
  cudaMemsetAsync(h->cacc, 0, sizeof(double) * 11 * (size_t)h->Kcap, s);
  cudaMemsetAsync(&h->st->bar, 0, sizeof(GridBar), s);
  int* active_cnt = reinterpret_cast<int*>(&h->st->bar2);
  cudaMemsetAsync(active_cnt, 0, sizeof(GridBar), s);
  PcgArgs a;
  a.wfill = h->wfill; a.invd = h->invd; a.rhs = h->b; a.labels = h->labels;
  a.x = h->x; a.r = h->r; a.p = h->p; a.q = h->q;
  a.cacc = h->cacc; a.cflag = h->cflag; a.st = h->st; a.active_cnt = active_cnt;
  a.H = h->H; a.W = h->W; a.K = h->K_host; a.Kcap = h->Kcap;
  a.maxit = h->cfg.cg_maxit; a.tol2 = h->cfg.cg_rtol * h->cfg.cg_rtol;
  void* args[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(256), args, 0, s);
  NI_COUNT(h);
  return ni_cuda_check(h, e, "batched PCG launch");
}

ni_status fill_solve_launch(ni_handle* h, cudaStream_t s) {
  ni_status rc = project_rhs(h, h->b, s);
  if (rc != NI_OK) return rc;
  for (int sweep = 0; sweep < std::max(1, h->cfg.n_fill_irls); ++sweep) {
    if (sweep > 0) {
      k_fill_reweight<<<grid_px(h, h->N), 256, 0, s>>>(h->ntau, h->labels, h->x, h->H, h->W, h->persp,
                                                        h->fx, h->fy, (float)h->cfg.k, h->wfill); NI_COUNT(h);
      k_diag_rhs<<<grid_px(h, h->N), 256, 0, s>>>(h->wfill, h->omega, h->H, h->W, h->invd, h->b); NI_COUNT(h);
      rc = project_rhs(h, h->b, s);
      if (rc != NI_OK) return rc;
    }
    cudaMemsetAsync(&h->st->fill_iters, 0, 2 * sizeof(int), s);
    cudaMemsetAsync(&h->st->fill_px_iters, 0, sizeof(unsigned long long), s);
    cudaEventRecord(h->ev[5], s);
    if (h->cfg.batched) {
      rc = batched_solve(h, s);
      cudaEventRecord(h->ev[6], s);
    } else {
      rc = plain_solve(h, s);
      cudaEventRecord(h->ev[6], s);
      if (rc == NI_OK) {
        k_plain_stats<<<1, 1, 0, s>>>(h->st, h->cfg.cg_maxit, h->cfg.cg_rtol * h->cfg.cg_rtol); NI_COUNT(h);
        rc = project_rhs(h, h->x, s);
      }
    }
    if (rc != NI_OK) return rc;
  }
  return ni_cuda_check(h, cudaGetLastError(), "fill solve");
}

// ---------------------------------------------------------------------------
// log-depth import / export and the output (row a8)
// ---------------------------------------------------------------------------
__global__ void k_export(const float* __restrict__ x, const int* __restrict__ labels,
                         const double* __restrict__ soff, int N, float* __restrict__ out) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    int c = labels[a];
    out[a] = c >= 0 ? (float)((double)x[a] + soff[c]) : 0.f;
  }
}

__global__ void k_import(const float* __restrict__ in, const int* __restrict__ labels, int N,
                         float* __restrict__ x) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x)
    x[a] = labels[a] >= 0 ? in[a] : 0.f;
}

__global__ void k_output(const float* __restrict__ x, const int* __restrict__ labels,
                         const double* __restrict__ soff, int N, int persp, float* __restrict__ depth) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    int c = labels[a];
    float v = __int_as_float(0x7fc00000);
    if (c >= 0) {
      double z = (double)x[a] + soff[c];
      v = persp ? (float)exp(z) : (float)z;
    }
    depth[a] = v;
  }
}

void export_logdepth_launch(ni_handle* h, float* out, cudaStream_t s) {
  k_export<<<grid_px(h, h->N), 256, 0, s>>>(h->x, h->labels, h->soff, h->N, out); NI_COUNT(h);
}

void import_logdepth_launch(ni_handle* h, const float* in, cudaStream_t s) {
  k_import<<<grid_px(h, h->N), 256, 0, s>>>(in, h->labels, h->N, h->x); NI_COUNT(h);
  cudaMemsetAsync(h->soff, 0, sizeof(double) * (size_t)h->Kcap, s);
}

void output_depth_launch(ni_handle* h, float* depth, cudaStream_t s) {
  k_output<<<grid_px(h, h->N), 256, 0, s>>>(h->x, h->labels, h->soff, h->N, h->persp, depth); NI_COUNT(h);
}
