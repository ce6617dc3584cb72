// Relative-scale optimisation and merging (Sec. 3.4-3.5, Algorithm 1; rows a5-a6).
//
// Partition structures (rebuilt after seeding and after every merge):
//   E_inter   inter-component edges as edge ids 2 a + dir (dir 0 right, 1 down),
//             in increasing id order (stream compaction); with 8-connectivity
//             4 a + dir (2 lower-right, 3 lower-left);
//   pairs     the distinct component pairs (lo < hi) that inter edges join:
//             edges are sorted by the key lo * K + hi with a stable LSD radix
//             sort, so each pair's edges are one contiguous run;
//   CSR       rows of the K x K quotient Laplacian (both orientations of every
//             pair, sorted by row).
// One iteration t (all on the device, capturable in a CUDA graph):
//   k_edge_accum   per inter edge: chi = z~_a - z~_b - omega~_{b->a} (Eq. 4),
//                  weight of the two directed rows (1 + 1 for t <= 1; else
//                  (W_{b->a} + W_{a->b}) W^out(|chi|), Eqs. 5, 11), reduced per
//                  pair into (w_p, h_p = sum w chi oriented lo -> hi, q_p = sum w chi^2);
//   k_node_assemble diagonal and right-hand side of A_m^T W A_m s = A_m^T W b_m (Eq. 14);
//   k_scale_cg     Jacobi-PCG in float64, then E_t (energy of the system just
//                  solved), the stop test, and the update of Eqs. 7-8 applied to
//                  a per-component float64 offset (z~_a = x_a + soff[pi(a)]), so
//                  the per-pixel log-depth is only touched when merging.
// Merge (Sec. 3.5): per component the incident inter edge with the smallest
//   float32 |chi| (ties: smaller edge id) by 64-bit atomicMin of
//   (bits(|chi|) << 32 | edge id); union-find over components; new label =
//   rank of the group's smallest old label; pixels relabelled and their offsets
//   folded into x relative to the group's representative.
#include <algorithm>

#include "ni_internal.cuh"

// kernels defined in ni_seed.cu
__global__ void k_scan_blocks(int* blk, int nblocks, int* total_out);

static int grid_lin(ni_handle* h, long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  long long cap = (long long)h->num_sms * 8;
  return (int)std::max(1LL, std::min(b, cap));
}

__device__ __forceinline__ void chunk_rng(int n, int& beg, int& end) {
  int chunk = (n + gridDim.x - 1) / gridDim.x;
  beg = min(n, blockIdx.x * chunk);
  end = min(n, beg + chunk);
}

__device__ __forceinline__ bool gated(const int* gate) { return gate && (*(volatile const int*)gate == 0); }

// ---------------------------------------------------------------------------
// generic chunked compaction: F::count(i) items for element i, F::emit(i, pos, cnt)
// ---------------------------------------------------------------------------
template <class F>
__global__ void k_chunk_count(F f, const int* n_ptr, int* blk, const int* gate) {
  __shared__ int sh[40];
  if (gated(gate)) return;
  int n = *n_ptr, beg, end;
  chunk_rng(n, beg, end);
  int c = 0;
  for (int i = beg + threadIdx.x; i < end; i += blockDim.x) c += f.count(i);
  c = block_sum_i(c, sh);
  if (threadIdx.x == 0) blk[blockIdx.x] = c;
}

template <class F>
__global__ void k_chunk_emit(F f, const int* n_ptr, const int* blk, const int* gate) {
  __shared__ int sh[40];
  if (gated(gate)) return;
  int n = *n_ptr, beg, end;
  chunk_rng(n, beg, end);
  int base = blk[blockIdx.x];
  for (int t0 = beg; t0 < end; t0 += blockDim.x) {
    int i = t0 + threadIdx.x;
    int cnt = (i < end) ? f.count(i) : 0;
    int tot;
    int ex = block_excl_scan_i(cnt, sh, &tot);
    if (i < end) f.emit(i, base + ex, cnt);
    base += tot;
  }
}

__global__ void k_scan_blocks_gated(int* blk, int nblocks, int* total_out, const int* gate) {
  __shared__ int sh[40];
  if (gated(gate)) return;
  int v = (threadIdx.x < nblocks) ? blk[threadIdx.x] : 0;
  int tot;
  int ex = block_excl_scan_i(v, sh, &tot);
  if (threadIdx.x < nblocks) blk[threadIdx.x] = ex;
  if (threadIdx.x == 0) *total_out = tot;
}

template <class F>
static void compact(ni_handle* h, F f, const int* n_ptr, int* total_out, const int* gate, cudaStream_t s) {
  k_chunk_count<F><<<NI_SCAN_BLOCKS, NI_SCAN_THREADS, 0, s>>>(f, n_ptr, h->blk, gate); NI_COUNT(h);
  k_scan_blocks_gated<<<1, 1024, 0, s>>>(h->blk, NI_SCAN_BLOCKS, total_out, gate); NI_COUNT(h);
  k_chunk_emit<F><<<NI_SCAN_BLOCKS, NI_SCAN_THREADS, 0, s>>>(f, n_ptr, h->blk, gate); NI_COUNT(h);
}

// Edge ids: CONN 4: e = 2 a + dir (0 right, 1 down); CONN 8: e = 4 a + dir
// (2 lower-right, 3 lower-left).  b = a + step(dir).
template <int CONN>
__device__ __forceinline__ int edge_a(int e) { return CONN == 8 ? (e >> 2) : (e >> 1); }
template <int CONN>
__device__ __forceinline__ int edge_dir(int e) { return CONN == 8 ? (e & 3) : (e & 1); }
template <int CONN>
__device__ __forceinline__ int edge_step(int dir, int W) {
  if constexpr (CONN == 8) return dir == 0 ? 1 : (dir == 1 ? W : (dir == 2 ? W + 1 : W - 1));
  return dir ? W : 1;
}

// inter edges from the pixel grid (first partition)
template <int CONN>
struct InterFromPixels {
  const int* labels;
  int H, W;
  int* out;
  __device__ int count(int a) const {
    int la = labels[a];
    if (la < 0) return 0;
    int u = a % W, v = a / W, c = 0;
    if (u + 1 < W) { int lb = labels[a + 1]; c += (lb >= 0 && lb != la); }
    if (v + 1 < H) { int lb = labels[a + W]; c += (lb >= 0 && lb != la); }
    if constexpr (CONN == 8) {
      if (u + 1 < W && v + 1 < H) { int lb = labels[a + W + 1]; c += (lb >= 0 && lb != la); }
      if (u >= 1 && v + 1 < H) { int lb = labels[a + W - 1]; c += (lb >= 0 && lb != la); }
    }
    return c;
  }
  __device__ void emit(int a, int pos, int cnt) const {
    if (!cnt) return;
    int la = labels[a], u = a % W, v = a / W;
    if constexpr (CONN == 8) {
      if (u + 1 < W) { int lb = labels[a + 1]; if (lb >= 0 && lb != la) out[pos++] = 4 * a; }
      if (v + 1 < H) { int lb = labels[a + W]; if (lb >= 0 && lb != la) out[pos++] = 4 * a + 1; }
      if (u + 1 < W && v + 1 < H) { int lb = labels[a + W + 1]; if (lb >= 0 && lb != la) out[pos++] = 4 * a + 2; }
      if (u >= 1 && v + 1 < H) { int lb = labels[a + W - 1]; if (lb >= 0 && lb != la) out[pos++] = 4 * a + 3; }
    } else {
      if (u + 1 < W) { int lb = labels[a + 1]; if (lb >= 0 && lb != la) out[pos++] = 2 * a; }
      if (v + 1 < H) { int lb = labels[a + W]; if (lb >= 0 && lb != la) out[pos++] = 2 * a + 1; }
    }
  }
};

// inter edges that survive a merge (labels already rewritten)
template <int CONN>
struct InterFilter {
  const int* labels;
  const int* in;
  int* out;
  int W;
  __device__ int count(int j) const {
    int e = in[j], a = edge_a<CONN>(e), b = a + edge_step<CONN>(edge_dir<CONN>(e), W);
    return labels[a] != labels[b];
  }
  __device__ void emit(int j, int pos, int cnt) const {
    if (cnt) out[pos] = in[j];
  }
};

// pair heads over edges sorted by key
struct PairHeads {
  const unsigned long long* key;
  const DevState* st;
  int* e_pair;
  int* p_lo;
  int* p_hi;
  __device__ int count(int j) const { return (j == 0) || (key[j] != key[j - 1]); }
  __device__ void emit(int j, int pos, int cnt) const {
    e_pair[j] = pos + cnt - 1;
    if (cnt) {
      unsigned long long K = (unsigned long long)st->K;
      p_lo[pos] = (int)(key[j] / K);
      p_hi[pos] = (int)(key[j] % K);
    }
  }
};

// roots of a union-find forest over n = K nodes
struct KRoots {
  const int* parent;
  int* out;
  __device__ int count(int c) const { return parent[c] == c; }
  __device__ void emit(int c, int pos, int cnt) const {
    if (cnt) out[c] = pos;
  }
};

// ---------------------------------------------------------------------------
// stable LSD radix sort of (uint64 key, int value), 8-bit digits
// ---------------------------------------------------------------------------
__global__ void k_radix_hist(const unsigned long long* __restrict__ keys, const int* n_ptr, int shift,
                             int* __restrict__ hist, const int* gate) {
  __shared__ int hcount[256];
  if (gated(gate)) return;
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hcount[d] = 0;
  __syncthreads();
  int n = *n_ptr, beg, end;
  chunk_rng(n, beg, end);
  for (int i = beg + threadIdx.x; i < end; i += blockDim.x)
    atomicAdd(&hcount[(int)((keys[i] >> shift) & 255ull)], 1);
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d * gridDim.x + blockIdx.x] = hcount[d];
}

// single-block exclusive scan of n <= 1024 * 64 ints in place: each warp owns a
// contiguous segment and walks it 32 elements at a time (coalesced), a block
// scan of the warp totals gives the segment offsets
__global__ void k_scan_big(int* __restrict__ a, int n, const int* gate) {
  __shared__ int wsum[32];
  if (gated(gate)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int seg = (n + nw - 1) / nw;
  const int beg = min(n, warp * seg), end = min(n, beg + seg);
  int tot = 0;
#pragma unroll 8
  for (int i = beg + lane; i < end; i += 32) tot += a[i];
  tot = warp_sum_i(tot);
  if (lane == 0) wsum[warp] = tot;
  __syncthreads();
  if (warp == 0) {
    const int v = lane < nw ? wsum[lane] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(NI_FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane < nw) wsum[lane] = x - v;
  }
  __syncthreads();
  int run = wsum[warp];
  for (int i0 = beg; i0 < end; i0 += 32) {
    const int i = i0 + lane;
    const int v = i < end ? a[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(NI_FULL, x, o);
      if (lane >= o) x += y;
    }
    if (i < end) a[i] = run + x - v;
    run += __shfl_sync(NI_FULL, x, 31);
  }
}

__global__ void __launch_bounds__(NI_SORT_THREADS)
k_radix_scatter(const unsigned long long* __restrict__ kin, const int* __restrict__ vin,
                unsigned long long* __restrict__ kout, int* __restrict__ vout, const int* n_ptr, int shift,
                const int* __restrict__ hist, const int* gate) {
  constexpr int NW = NI_SORT_THREADS / 32;
  __shared__ int base[256];
  __shared__ int wcnt[NW][256];
  if (gated(gate)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int n = *n_ptr, beg, end;
  chunk_rng(n, beg, end);
  for (int d = threadIdx.x; d < 256; d += blockDim.x) base[d] = hist[d * gridDim.x + blockIdx.x];
  for (int t0 = beg; t0 < end; t0 += blockDim.x) {
    for (int j = threadIdx.x; j < NW * 256; j += blockDim.x) (&wcnt[0][0])[j] = 0;
    __syncthreads();
    const int i = t0 + threadIdx.x;
    const bool valid = i < end;
    unsigned long long key = valid ? kin[i] : 0ull;
    const int d = valid ? (int)((key >> shift) & 255ull) : 256;
    const unsigned peers = __match_any_sync(NI_FULL, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int off = 0;
      for (int w = 0; w < warp; ++w) off += wcnt[w][d];
      const int pos = base[d] + off + rank;
      kout[pos] = key;
      vout[pos] = vin[i];
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < 256; dd += blockDim.x) {
      int tot = 0;
      for (int w = 0; w < NW; ++w) tot += wcnt[w][dd];
      base[dd] += tot;
    }
    __syncthreads();
  }
}

__global__ void k_copy_kv(const unsigned long long* __restrict__ kin, const int* __restrict__ vin,
                          unsigned long long* __restrict__ kout, int* __restrict__ vout, const int* n_ptr,
                          const int* gate) {
  if (gated(gate)) return;
  int n = *n_ptr;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    kout[i] = kin[i];
    vout[i] = vin[i];
  }
}

static void radix_sort(ni_handle* h, unsigned long long* k0, int* v0, unsigned long long* k1, int* v1,
                       const int* n_ptr, int passes, const int* gate, cudaStream_t s) {
  const int B = NI_SORT_BLOCKS;
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = 8 * ps;
    unsigned long long* ki = (ps & 1) ? k1 : k0;
    int* vi = (ps & 1) ? v1 : v0;
    unsigned long long* ko = (ps & 1) ? k0 : k1;
    int* vo = (ps & 1) ? v0 : v1;
    k_radix_hist<<<B, NI_SORT_THREADS, 0, s>>>(ki, n_ptr, shift, h->radix_hist, gate); NI_COUNT(h);
    k_scan_big<<<1, 1024, 0, s>>>(h->radix_hist, 256 * B, gate); NI_COUNT(h);
    k_radix_scatter<<<B, NI_SORT_THREADS, 0, s>>>(ki, vi, ko, vo, n_ptr, shift, h->radix_hist, gate); NI_COUNT(h);
  }
  if (passes & 1) k_copy_kv<<<grid_lin(h, h->Ecap * 2LL), 256, 0, s>>>(k1, v1, k0, v0, n_ptr, gate);
}

// ---------------------------------------------------------------------------
// partition structures
// ---------------------------------------------------------------------------
template <int CONN>
__global__ void k_edge_keys(const int* __restrict__ e_id, const int* __restrict__ labels, int W,
                            DevState* st, unsigned long long* __restrict__ key, int* __restrict__ val,
                            const int* gate) {
  if (gated(gate)) return;
  const int n = st->nE;
  const unsigned long long K = (unsigned long long)st->K;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    int e = e_id[j], a = edge_a<CONN>(e), b = a + edge_step<CONN>(edge_dir<CONN>(e), W);
    unsigned long long la = (unsigned long long)labels[a], lb = (unsigned long long)labels[b];
    unsigned long long lo = la < lb ? la : lb, hi = la < lb ? lb : la;
    key[j] = lo * K + hi;
    val[j] = j;
  }
}

__global__ void k_csr_entries(const int* __restrict__ p_lo, const int* __restrict__ p_hi, DevState* st,
                              unsigned long long* __restrict__ key, int* __restrict__ val, int* n2,
                              const int* gate) {
  if (gated(gate)) return;
  const int P = st->nP;
  const unsigned long long K = (unsigned long long)st->K;
  if (blockIdx.x == 0 && threadIdx.x == 0) *n2 = 2 * P;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    unsigned long long lo = (unsigned long long)p_lo[p], hi = (unsigned long long)p_hi[p];
    key[2 * p] = lo * K + hi;
    val[2 * p] = p;
    key[2 * p + 1] = hi * K + lo;
    val[2 * p + 1] = p;
  }
}

__global__ void k_csr_finish(const unsigned long long* __restrict__ key, const int* __restrict__ val,
                             DevState* st, int* __restrict__ col, int* __restrict__ pr,
                             int* __restrict__ row_ptr, const int* gate) {
  if (gated(gate)) return;
  const int n = 2 * st->nP, K = st->K;
  const unsigned long long KK = (unsigned long long)K;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    col[j] = (int)(key[j] % KK);
    pr[j] = val[j];
  }
  // row_ptr[c] = first entry whose row >= c (entries are sorted by row)
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= K; c += gridDim.x * blockDim.x) {
    int lo = 0, hi = n;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if ((int)(key[mid] / KK) < c) lo = mid + 1;
      else hi = mid;
    }
    row_ptr[c] = lo;
  }
}

__global__ void k_copy_int(const int* __restrict__ in, int* __restrict__ out, const int* n_ptr, const int* gate) {
  if (gated(gate)) return;
  int n = *n_ptr;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = in[i];
}

__global__ void k_copy1(const int* in, int* out, const int* gate) {
  if (gated(gate)) return;
  *out = *in;
}

static void build_pairs(ni_handle* h, const int* gate, cudaStream_t s) {
  DevState* st = h->st;
  const int g = grid_lin(h, h->Ecap);
  if (h->cfg.connectivity == 8)
    k_edge_keys<8><<<g, 256, 0, s>>>(h->e_id, h->labels, h->W, st, h->e_key, h->e_val, gate);
  else
    k_edge_keys<4><<<g, 256, 0, s>>>(h->e_id, h->labels, h->W, st, h->e_key, h->e_val, gate);
  NI_COUNT(h);
  radix_sort(h, h->e_key, h->e_val, h->e_key2, h->e_val2, &st->nE, h->sort_passes, gate, s);
  PairHeads ph{h->e_key, st, h->e_pair, h->p_lo, h->p_hi};
  compact(h, ph, &st->nE, &st->nP, gate, s);
  int* n2 = h->d_count;
  k_csr_entries<<<g, 256, 0, s>>>(h->p_lo, h->p_hi, st, h->e_key2, h->e_val2, n2, gate); NI_COUNT(h);
  // sort the 2P CSR entries in the second buffers (the first ones hold the edge order)
  radix_sort(h, h->e_key2, h->e_val2, h->c_key, h->c_val, n2, h->sort_passes, gate, s);
  k_csr_finish<<<g, 256, 0, s>>>(h->e_key2, h->e_val2, st, h->csr_col, h->csr_pair, h->row_ptr, gate); NI_COUNT(h);
}

template <int CONN>
static ni_status partition_build(ni_handle* h, int first, cudaStream_t s) {
  DevState* st = h->st;
  if (first) {
    // count, size the edge buffers, then emit
    InterFromPixels<CONN> f{h->labels, h->H, h->W, nullptr};
    int* nptr = h->d_count + 1;
    cudaMemcpyAsync(nptr, &h->N, sizeof(int), cudaMemcpyHostToDevice, s);
    k_chunk_count<InterFromPixels<CONN>><<<NI_SCAN_BLOCKS, NI_SCAN_THREADS, 0, s>>>(f, nptr, h->blk, nullptr);
    NI_COUNT(h);
    k_scan_blocks_gated<<<1, 1024, 0, s>>>(h->blk, NI_SCAN_BLOCKS, &st->nE, nullptr); NI_COUNT(h);
    cudaMemcpyAsync(&h->st_host->nE, &st->nE, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ni_cuda_check(h, e, "inter-edge count");
    ni_status rc = ensure_edge_capacity(h, h->st_host->nE);
    if (rc != NI_OK) return rc;
    f.out = h->e_id;
    k_chunk_emit<InterFromPixels<CONN>><<<NI_SCAN_BLOCKS, NI_SCAN_THREADS, 0, s>>>(f, nptr, h->blk, nullptr);
    NI_COUNT(h);
    build_pairs(h, nullptr, s);
  } else {
    InterFilter<CONN> f{h->labels, h->e_id, h->e_id2, h->W};
    int* nold = h->d_count + 2;
    k_copy1<<<1, 1, 0, s>>>(&st->nE, nold, &st->gate); NI_COUNT(h);
    compact(h, f, nold, &st->nE, &st->gate, s);
    k_copy_int<<<grid_lin(h, h->Ecap), 256, 0, s>>>(h->e_id2, h->e_id, &st->nE, &st->gate); NI_COUNT(h);
    build_pairs(h, &st->gate, s);
  }
  return ni_cuda_check(h, cudaGetLastError(), "partition build");
}

ni_status partition_build_launch(ni_handle* h, int first, cudaStream_t s) {
  return h->cfg.connectivity == 8 ? partition_build<8>(h, first, s) : partition_build<4>(h, first, s);
}

// ---------------------------------------------------------------------------
// one relative-scale iteration
// ---------------------------------------------------------------------------
struct EdgeArgs {
  const int* e_id;
  const int* e_val;
  const int* e_pair;
  const int* p_lo;
  const int* labels;
  const float* x;
  const double* soff;
  const float2* omega;
  const float2* omega_d;   // diagonal edges (8-connectivity), else NULL
  const float* ntau;
  double* p_acc;
  DevState* st;
  int H, W, persp;
  double fx, fy, k, Lt, Ut, U;
  int hard;
};

__device__ __forceinline__ double sigm(double x, double k) { return 1.0 / (1.0 + exp(-k * x)); }

__global__ void k_pair_zero(double* __restrict__ acc, DevState* st) {
  if (st->converged) return;
  const int n = 3 * st->nP;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc[i] = 0.0;
}

template <int CONN>
__global__ void k_edge_accum(EdgeArgs A) {
  DevState* st = A.st;
  if (st->converged) return;
  const int n = st->nE, t = st->t, W = A.W, H = A.H;
  const int nthr = gridDim.x * blockDim.x;
  const int nIter = (n + nthr - 1) / nthr;
  for (int it = 0; it < nIter; ++it) {
    const int j = it * nthr + blockIdx.x * blockDim.x + threadIdx.x;
    int pair = -1;
    double v[3] = {0.0, 0.0, 0.0};
    if (j < n) {
      pair = A.e_pair[j];
      const int e = A.e_id[A.e_val[j]];
      const int a = edge_a<CONN>(e), dir = edge_dir<CONN>(e), step = edge_step<CONN>(dir, W), b = a + step;
      const int ca = A.labels[a], cb = A.labels[b];
      const double za = (double)A.x[a] + A.soff[ca];
      const double zb = (double)A.x[b] + A.soff[cb];
      double omv;
      if constexpr (CONN == 8) {
        const float2 om2 = dir >= 2 ? A.omega_d[a] : A.omega[a];
        omv = (double)((dir & 1) ? om2.y : om2.x);
      } else {
        const float2 om2 = A.omega[a];
        omv = (double)(dir ? om2.y : om2.x);
      }
      const double rho = za - zb - omv;
      double w;
      if (t <= 1) {
        w = 2.0;   // two rows of unit weight (alignment iterations)
      } else {
        const int u = a % W, vv = a / W;
        double f;
        bool has_oa, has_ob;
        if constexpr (CONN == 8) {
          // f = sqrt(f_x f_y) on diagonals; -b of a diagonal edge is a - (b - a)
          f = A.persp ? (dir == 0 ? A.fx : (dir == 1 ? A.fy : sqrt(A.fx * A.fy))) : 1.0;
          has_oa = dir == 0 ? (u > 0) : dir == 1 ? (vv > 0) : dir == 2 ? (u > 0 && vv > 0) : (u + 1 < W && vv > 0);
          has_ob = dir == 0 ? (u + 2 < W) : dir == 1 ? (vv + 2 < H)
                   : dir == 2 ? (u + 2 < W && vv + 2 < H) : (u >= 2 && vv + 2 < H);
        } else {
          f = A.persp ? (dir ? A.fy : A.fx) : 1.0;
          // opposite neighbour of a (away from b) and of b (away from a)
          has_oa = dir ? (vv > 0) : (u > 0);
          has_ob = dir ? (vv + 2 < H) : (u + 2 < W);
        }
        const double gba = f * (double)A.ntau[a], gab = f * (double)A.ntau[b];
        double doa = 0.0, dob = 0.0;
        if (has_oa) {
          int o = a - step, co = A.labels[o];
          if (co >= 0) { double zo = (double)A.x[o] + A.soff[co]; doa = (zo - za) * (zo - za); }
        }
        if (has_ob) {
          int o = b + step, co = A.labels[o];
          if (co >= 0) { double zo = (double)A.x[o] + A.soff[co]; dob = (zo - zb) * (zo - zb); }
        }
        const double d2 = (zb - za) * (zb - za);
        const double g2a = gba * gba, g2b = gab * gab;
        const double wba = g2a * sigm(g2a * (doa - d2), A.k);
        const double wab = g2b * sigm(g2b * (dob - d2), A.k);
        const double ar = fmax(fabs(rho), 1e-30);
        double wout;
        if (A.hard) wout = ar < A.U ? 1.0 : 0.0;
        else wout = sigm(4.0 / (A.Lt - A.Ut) * (2.0 * log10(ar) - (A.Lt + A.Ut)), 1.0);
        w = (wba + wab) * wout;
      }
      const double sg = (ca == A.p_lo[pair]) ? rho : -rho;   // chi oriented lo -> hi
      v[0] = w;
      v[1] = w * sg;
      v[2] = w * rho * rho;
    }
    seg_add_d<3>(A.p_acc, 3, pair, v);
  }
}

// Also gabs_c = sum |h_p|: the size of the terms that cancel in g_c, which sets
// the rounding floor of the right-hand side.
__global__ void k_node_assemble(const int* __restrict__ row_ptr, const int* __restrict__ csr_pair,
                                const int* __restrict__ p_lo, const double* __restrict__ p_acc,
                                DevState* st, double* __restrict__ diag, double* __restrict__ g,
                                double* __restrict__ gabs, double* __restrict__ csr_w) {
  if (st->converged) return;
  const int K = st->K;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int c = gw; c < K; c += nw) {   // one warp per row (power-law degrees)
    double d = 0.0, gs = 0.0, ga = 0.0;
    for (int j = row_ptr[c] + lane; j < row_ptr[c + 1]; j += 32) {
      int p = csr_pair[j];
      const double wp = p_acc[3 * p];
      csr_w[j] = wp;   // the entry's weight for the SpMVs of this iteration
      d += wp;
      const double hp = p_acc[3 * p + 1];
      gs += (p_lo[p] == c) ? -hp : hp;
      ga += fabs(hp);
    }
    d = warp_sum_d(d);
    gs = warp_sum_d(gs);
    ga = warp_sum_d(ga);
    if (lane == 0) {
      diag[c] = d;
      g[c] = gs;
      gabs[c] = ga;
    }
  }
}

struct ScaleArgs {
  DevState* st;
  const int* row_ptr;
  const int* csr_col;
  const double* csr_w;
  const int* csr_pair;
  const int* p_lo;
  const int* p_hi;
  const double* p_acc;
  double* diag;        // the Jacobi diagonal; replaced by its inverse at the start of the solve
  const double* g;
  const double* gabs;
  double* s;
  double* r;
  double* z;
  double* pp;
  double* qq;
  double* red;    // 3 slots x 4 doubles
  double* soff;
  double tol2;
  int maxit;
  int T;
  double dE_max;
};

// CTA sum of three values, the same additions as three block_sum_d calls.  A
// warp whose values are all zero (its rows lie past the last component) or sit
// in lane 0 alone (a long row's result) skips its shuffle trees, which are most
// of the FP64 instructions of an iteration when K is small against the CTA.
__device__ __forceinline__ void block_sum3_d(double& a, double& b, double& c, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const unsigned m = __ballot_sync(NI_FULL, a != 0.0 || b != 0.0 || c != 0.0);
  if (m & ~1u) {
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    c = warp_sum_d(c);
  }
  __syncthreads();
  if (lane == 0) {
    sh[3 * wid] = a;
    sh[3 * wid + 1] = b;
    sh[3 * wid + 2] = c;
  }
  __syncthreads();
  if (wid == 0) {
    double x = lane < nw ? sh[3 * lane] : 0.0, y = lane < nw ? sh[3 * lane + 1] : 0.0,
           z = lane < nw ? sh[3 * lane + 2] : 0.0;
    x = warp_sum_d(x);
    y = warp_sum_d(y);
    z = warp_sum_d(z);
    if (lane == 0) {
      sh[96] = x;
      sh[97] = y;
      sh[98] = z;
    }
  }
  __syncthreads();
  a = sh[96];
  b = sh[97];
  c = sh[98];
}

// Grid-wide sum of three values.  gridDim 1: a block reduction.  Otherwise
// partial sums go to rotating slots (slot m % 3 at call m; block 0 clears slot
// (m + 1) % 3, last read two calls ago) followed by a bounded grid barrier.
__device__ __forceinline__ bool grid_sum3(double& a, double& b, double& c, double* red, int& ncall,
                                          DevState* st, double* sh) {
  double ba = a, bb = b, bc = c;
  block_sum3_d(ba, bb, bc, sh);
  if (gridDim.x == 1) {
    a = ba; b = bb; c = bc;
    return true;
  }
  double* R = red + 4 * (ncall % 3);
  if (threadIdx.x == 0) {
    if (blockIdx.x == 0) {
      double* Z = red + 4 * ((ncall + 1) % 3);
      Z[0] = 0.0; Z[1] = 0.0; Z[2] = 0.0;
    }
    if (ba != 0.0) atomicAdd(&R[0], ba);
    if (bb != 0.0) atomicAdd(&R[1], bb);
    if (bc != 0.0) atomicAdd(&R[2], bc);
  }
  ncall++;
  if (!grid_barrier(&st->bar, &st->err)) return false;
  volatile double* VR = R;
  a = VR[0]; b = VR[1]; c = VR[2];
  return true;
}

__device__ __forceinline__ bool gsync(DevState* st) {
  if (gridDim.x == 1) { __syncthreads(); return true; }
  return grid_barrier(&st->bar, &st->err);
}

__global__ void __launch_bounds__(1024) k_scale_cg(ScaleArgs A) {
  __shared__ double sh[99];
  DevState* st = A.st;
  if (*(volatile int*)&st->converged) return;
  const int K = st->K, P = st->nP;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  int ncall = 0;
  double rz = 0, ga2 = 0, gg = 0;
  for (int c = tid; c < K; c += nthr) {
    const double d = A.diag[c], rc = A.g[c];
    const double id = d > 0.0 ? 1.0 / d : 0.0;   // one FP64 division per component and solve
    A.diag[c] = id;
    const double zc = rc * id;
    A.s[c] = 0.0;
    A.r[c] = rc;
    A.z[c] = zc;
    A.pp[c] = zc;
    rz += rc * zc;
    ga2 += A.gabs[c] * A.gabs[c];
    gg += rc * rc;
  }
  if (!grid_sum3(rz, ga2, gg, A.red, ncall, st, sh)) return;
  // stop at the relative tolerance, or once the residual is at the rounding
  // level of the terms that cancel in g (a system that is already solved has a
  // right-hand side made of rounding noise)
  const double floor2 = (64.0 * 1.1102230246251565e-16) * (64.0 * 1.1102230246251565e-16) * ga2;
  const double stop2 = fmax(A.tol2 * gg, floor2);
  int it = 0;
  bool done = !(gg > 0.0) || gg <= stop2;
  // q = L p.  Rows of at most 32 entries take a thread each, longer rows a warp
  // each: the quotient graph's degrees follow the component sizes (a large
  // component borders thousands of small ones).  Entry weights come from csr_w.
  const int lane = threadIdx.x & 31, wid = tid >> 5, nwarp = nthr >> 5;
  while (!done && it < A.maxit) {
    double pq = 0, d1 = 0, d2 = 0;
    for (int c = tid; c < K; c += nthr) {
      const int b = A.row_ptr[c], e = A.row_ptr[c + 1];
      if (e - b > 32) continue;
      const double pc = A.pp[c];
      double acc = 0.0;
#pragma unroll 4
      for (int j = b; j < e; ++j) acc += A.csr_w[j] * (pc - A.pp[A.csr_col[j]]);
      A.qq[c] = acc;
      pq += pc * acc;
    }
    for (int c = wid; c < K; c += nwarp) {   // warp-uniform
      const int b = A.row_ptr[c], e = A.row_ptr[c + 1];
      if (e - b <= 32) continue;
      const double pc = A.pp[c];
      double acc = 0.0;
#pragma unroll 4
      for (int j = b + lane; j < e; j += 32) acc += A.csr_w[j] * (pc - A.pp[A.csr_col[j]]);
      acc = warp_sum_d(acc);
      if (lane == 0) {
        A.qq[c] = acc;
        pq += pc * acc;
      }
    }
    if (!grid_sum3(pq, d1, d2, A.red, ncall, st, sh)) return;
    const double alpha = pq > 0.0 ? rz / pq : 0.0;
    double rzn = 0, rrn = 0, d3 = 0;
    for (int c = tid; c < K; c += nthr) {
      A.s[c] += alpha * A.pp[c];
      const double rc = A.r[c] - alpha * A.qq[c];
      A.r[c] = rc;
      const double zc = rc * A.diag[c];
      A.z[c] = zc;
      rzn += rc * zc;
      rrn += rc * rc;
    }
    if (!grid_sum3(rzn, rrn, d3, A.red, ncall, st, sh)) return;
    const double beta = rz > 0.0 ? rzn / rz : 0.0;
    rz = rzn;
    ++it;
    done = rrn <= stop2 || !(pq > 0.0);
    if (!done) {
      for (int c = tid; c < K; c += nthr) A.pp[c] = A.z[c] + beta * A.pp[c];
      if (!gsync(st)) return;
    }
  }
  // energy of the solved system: sum_p w_p D^2 + 2 h_p D + q_p, D = s_lo - s_hi
  double en = 0, e1 = 0, e2 = 0;
  for (int p = tid; p < P; p += nthr) {
    const double D = A.s[A.p_lo[p]] - A.s[A.p_hi[p]];
    en += A.p_acc[3 * p] * D * D + 2.0 * A.p_acc[3 * p + 1] * D + A.p_acc[3 * p + 2];
  }
  if (!grid_sum3(en, e1, e2, A.red, ncall, st, sh)) return;
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

// one CTA (no grid barrier) up to 8192 components; beyond, about 8 rows per warp
// over several CTAs
int scale_cg_grid(ni_handle* h) {
  if (h->Kcap <= 8192) return 1;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scale_cg, 1024, 0);
  int g = h->num_sms * std::max(1, std::min(per_sm, 2));
  int need = (h->Kcap + 255) / 256;
  return std::max(1, std::min(g, need));
}

ni_status scale_iteration_launch(ni_handle* h, cudaStream_t s) {
  DevState* st = h->st;
  const int ge = grid_lin(h, h->Ecap);
  k_pair_zero<<<ge, 256, 0, s>>>(h->p_acc, st); NI_COUNT(h);
  EdgeArgs ea;
  ea.e_id = h->e_id; ea.e_val = h->e_val; ea.e_pair = h->e_pair; ea.p_lo = h->p_lo;
  ea.labels = h->labels; ea.x = h->x; ea.soff = h->soff; ea.omega = h->omega; ea.omega_d = h->omega_d;
  ea.ntau = h->ntau;
  ea.p_acc = h->p_acc; ea.st = st; ea.H = h->H; ea.W = h->W; ea.persp = h->persp;
  ea.fx = h->cfg.cam.fx; ea.fy = h->cfg.cam.fy; ea.k = h->cfg.k;
  ea.Lt = log10(h->cfg.L); ea.Ut = log10(h->cfg.U); ea.U = h->cfg.U; ea.hard = h->cfg.hard_outliers;
  if (h->cfg.connectivity == 8) k_edge_accum<8><<<ge, 256, 0, s>>>(ea);
  else k_edge_accum<4><<<ge, 256, 0, s>>>(ea);
  NI_COUNT(h);
  k_node_assemble<<<grid_lin(h, 32LL * h->Kcap), 256, 0, s>>>(h->row_ptr, h->csr_pair, h->p_lo, h->p_acc, st,
                                                        h->sd, h->sv + 5 * (size_t)h->Kcap,
                                                        h->sv + 6 * (size_t)h->Kcap, h->csr_w); NI_COUNT(h);
  ScaleArgs sa;
  sa.st = st; sa.row_ptr = h->row_ptr; sa.csr_col = h->csr_col; sa.csr_w = h->csr_w; sa.csr_pair = h->csr_pair;
  sa.p_lo = h->p_lo; sa.p_hi = h->p_hi; sa.p_acc = h->p_acc; sa.diag = h->sd;
  sa.g = h->sv + 5 * (size_t)h->Kcap;
  sa.gabs = h->sv + 6 * (size_t)h->Kcap;
  sa.s = h->sv; sa.r = h->sv + (size_t)h->Kcap; sa.z = h->sv + 2 * (size_t)h->Kcap;
  sa.pp = h->sv + 3 * (size_t)h->Kcap; sa.qq = h->sv + 4 * (size_t)h->Kcap;
  sa.red = h->cacc;   // 12 doubles of scratch (component accumulators are free here)
  sa.soff = h->soff;
  sa.tol2 = h->cfg.scale_rtol * h->cfg.scale_rtol;
  sa.maxit = h->cfg.scale_maxit > 0 ? h->cfg.scale_maxit : std::min(4 * h->Kcap + 100, 200000);
  sa.T = h->cfg.T;
  sa.dE_max = h->cfg.dE_max;
  const int grid = scale_cg_grid(h);
  if (grid == 1) {
    k_scale_cg<<<1, 1024, 0, s>>>(sa); NI_COUNT(h);
  } else {
    cudaMemsetAsync(h->cacc, 0, 12 * sizeof(double), s);
    cudaMemsetAsync(&st->bar, 0, sizeof(GridBar), s);
    void* args[] = {&sa};
    cudaError_t e = cudaLaunchCooperativeKernel((void*)k_scale_cg, dim3(grid), dim3(1024), args, 0, s);
    NI_COUNT(h);
    if (e != cudaSuccess) return ni_cuda_check(h, e, "scale PCG launch");
  }
  return ni_cuda_check(h, cudaGetLastError(), "scale iteration");
}

// ---------------------------------------------------------------------------
// merging
// ---------------------------------------------------------------------------
__global__ void k_merge_gate(DevState* st, int tgate, int force) {
  st->gate = force ? 1 : (st->t == tgate ? 1 : 0);
}

__global__ void k_merge_init(DevState* st, unsigned long long* __restrict__ key, int* __restrict__ kparent) {
  if (!st->gate) return;
  const int K = st->K;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x) {
    key[c] = ~0ull;
    kparent[c] = c;
  }
}

// chi_abs (caller-given |chi|): [H][W][2] (right, down) with 4-connectivity,
// [H][W][4] (right, down, lower-right, lower-left) with 8.
template <int CONN>
__global__ void k_merge_keys(const int* __restrict__ e_id, const int* __restrict__ labels,
                             const float* __restrict__ x, const double* __restrict__ soff,
                             const float2* __restrict__ omega, const float2* __restrict__ omega_d,
                             const float* __restrict__ chi_abs, int W, DevState* st,
                             unsigned long long* __restrict__ key) {
  if (!st->gate) return;
  const int n = st->nE;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int e = e_id[j], a = edge_a<CONN>(e), dir = edge_dir<CONN>(e), b = a + edge_step<CONN>(dir, W);
    const int ca = labels[a], cb = labels[b];
    float chi;
    if (chi_abs) {
      chi = fabsf(chi_abs[(CONN == 8 ? 4 : 2) * (size_t)a + dir]);
    } else {
      float2 om;
      if constexpr (CONN == 8) om = dir >= 2 ? omega_d[a] : omega[a];
      else om = omega[a];
      const double rho = ((double)x[a] + soff[ca]) - ((double)x[b] + soff[cb]) - (double)((dir & 1) ? om.y : om.x);
      chi = (float)fabs(rho);
    }
    const unsigned long long k = ((unsigned long long)__float_as_uint(chi) << 32) | (unsigned int)e;
    atomicMin(&key[ca], k);
    atomicMin(&key[cb], k);
  }
}

template <int CONN>
__global__ void k_merge_link(const unsigned long long* __restrict__ key, const int* __restrict__ labels,
                             int W, DevState* st, int* __restrict__ kparent) {
  if (!st->gate) return;
  const int K = st->K;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x) {
    const unsigned long long k = key[c];
    if (k == ~0ull) continue;
    const int e = (int)(k & 0xffffffffull), a = edge_a<CONN>(e), b = a + edge_step<CONN>(edge_dir<CONN>(e), W);
    const int ca = labels[a], cb = labels[b];
    uf_unite(kparent, c, ca == c ? cb : ca);
  }
}

__global__ void k_merge_compress(DevState* st, int* __restrict__ kparent) {
  if (!st->gate) return;
  const int K = st->K;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x) {
    int p = kparent[c];
    if (p != c) kparent[c] = uf_find(kparent, c);
  }
}

// kmap[c] = new label of old component c; soff2[new] = offset of the group's root
__global__ void k_merge_map(DevState* st, const int* __restrict__ kparent, int* __restrict__ kmap,
                            const double* __restrict__ soff, double* __restrict__ soff2) {
  if (!st->gate) return;
  const int K = st->K;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x) {
    int r = kparent[c];
    if (r == c) soff2[kmap[c]] = soff[c];
  }
}

__global__ void k_merge_map2(DevState* st, const int* __restrict__ kparent, int* __restrict__ kmap) {
  if (!st->gate) return;
  const int K = st->K;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x) {
    int r = kparent[c];
    if (r != c) kmap[c] = kmap[r];
  }
}

__global__ void k_merge_relabel(DevState* st, const int* __restrict__ kparent, const int* __restrict__ kmap,
                                const double* __restrict__ soff, int N, int* __restrict__ labels,
                                float* __restrict__ x) {
  if (!st->gate) return;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    const int c = labels[a];
    if (c < 0) continue;
    const int r = kparent[c];
    if (r != c) x[a] = (float)((double)x[a] + (soff[c] - soff[r]));
    labels[a] = kmap[c];
  }
}

__global__ void k_merge_finish(DevState* st, const int* __restrict__ knew, const double* __restrict__ soff2,
                               double* __restrict__ soff) {
  if (!st->gate) return;
  const int Kn = *knew;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < Kn; c += gridDim.x * blockDim.x) soff[c] = soff2[c];
}

__global__ void k_merge_setk(DevState* st, const int* __restrict__ knew) {
  if (!st->gate) return;
  st->K = *knew;
  st->merges += 1;
}

ni_status merge_launch(ni_handle* h, const float* chi_abs, cudaStream_t s) {
  DevState* st = h->st;
  const int gk = grid_lin(h, h->Kcap), ge = grid_lin(h, h->Ecap), gp = grid_lin(h, h->N);
  int* knew = h->d_count + 3;
  k_merge_init<<<gk, 256, 0, s>>>(st, h->kkey, h->kparent); NI_COUNT(h);
  if (h->cfg.connectivity == 8) {
    k_merge_keys<8><<<ge, 256, 0, s>>>(h->e_id, h->labels, h->x, h->soff, h->omega, h->omega_d, chi_abs, h->W, st,
                                       h->kkey); NI_COUNT(h);
    k_merge_link<8><<<gk, 256, 0, s>>>(h->kkey, h->labels, h->W, st, h->kparent); NI_COUNT(h);
  } else {
    k_merge_keys<4><<<ge, 256, 0, s>>>(h->e_id, h->labels, h->x, h->soff, h->omega, nullptr, chi_abs, h->W, st,
                                       h->kkey); NI_COUNT(h);
    k_merge_link<4><<<gk, 256, 0, s>>>(h->kkey, h->labels, h->W, st, h->kparent); NI_COUNT(h);
  }
  k_merge_compress<<<gk, 256, 0, s>>>(st, h->kparent); NI_COUNT(h);
  KRoots kr{h->kparent, h->kmap};
  compact(h, kr, &st->K, knew, &st->gate, s);
  k_merge_map<<<gk, 256, 0, s>>>(st, h->kparent, h->kmap, h->soff, h->soff2); NI_COUNT(h);
  k_merge_map2<<<gk, 256, 0, s>>>(st, h->kparent, h->kmap); NI_COUNT(h);
  k_merge_relabel<<<gp, 256, 0, s>>>(st, h->kparent, h->kmap, h->soff, h->N, h->labels, h->x); NI_COUNT(h);
  k_merge_finish<<<gk, 256, 0, s>>>(st, knew, h->soff2, h->soff); NI_COUNT(h);
  k_merge_setk<<<1, 1, 0, s>>>(st, knew); NI_COUNT(h);
  ni_status rc = ni_cuda_check(h, cudaGetLastError(), "merge");
  if (rc != NI_OK) return rc;
  return partition_build_launch(h, 0, s);
}

void merge_gate_launch(ni_handle* h, int tgate, int force, cudaStream_t s) {
  k_merge_gate<<<1, 1, 0, s>>>(h->st, tgate, force); NI_COUNT(h);
}
