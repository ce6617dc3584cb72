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
//   k_scale_cg     Jacobi-PCG in float64 (single-reduction form, exact
//                  fixed-point inner products; one thread-block cluster or a
//                  cooperative grid), then E_t (energy of the system just
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
  int bini_res;            // residual-based BiNI weights
  const float4* lw;        // learned continuity per pixel and direction (t <= 1), or NULL
};

// omega~ stored for the edge (p, p + step(dir)): omega~_{(p + step) -> p}
template <int CONN>
__device__ __forceinline__ double edge_omega(const EdgeArgs& A, int p, int dir) {
  if constexpr (CONN == 8) {
    const float2 o = dir >= 2 ? A.omega_d[p] : A.omega[p];
    return (double)((dir & 1) ? o.y : o.x);
  }
  const float2 o = A.omega[p];
  return (double)(dir ? o.y : o.x);
}

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
        if (A.lw && dir < 2) {
          // learned: row b->a weighted by a's continuity towards b, row a->b by b's towards a
          const float4 pa = A.lw[a], pb = A.lw[b];
          const float wa = dir ? pa.y : pa.x, wb = dir ? pb.w : pb.z;
          w = (double)fmaxf(wa, 1e-3f) + (double)fmaxf(wb, 1e-3f);
        }
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
        // the opposite side of a is the edge (a - step, a), of b the edge (b, b + step)
        if (has_oa) {
          int o = a - step, co = A.labels[o];
          if (co >= 0) {
            const double zo = (double)A.x[o] + A.soff[co];
            // residual chi_{o->a} = z_a - z_o - omega~_{o->a}, omega~_{o->a} = -omega~_{a->o}
            const double e = A.bini_res ? za - zo + edge_omega<CONN>(A, o, dir) : zo - za;
            doa = e * e;
          }
        }
        if (has_ob) {
          int o = b + step, co = A.labels[o];
          if (co >= 0) {
            const double zo = (double)A.x[o] + A.soff[co];
            // residual chi_{o->b} = z_b - z_o - omega~_{o->b}
            const double e = A.bini_res ? zb - zo - edge_omega<CONN>(A, b, dir) : zo - zb;
            dob = e * e;
          }
        }
        // the edge's own side: raw (z_b - z_a)^2, or its residual chi^2 (the same for both rows)
        const double d2 = A.bini_res ? rho * rho : (zb - za) * (zb - za);
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

// Writes the inverse of the Jacobi diagonal.  Also gabs_c = sum |h_p|: the size
// of the terms that cancel in g_c, which sets the rounding floor of the
// right-hand side.
__global__ void k_node_assemble(const int* __restrict__ row_ptr, const int* __restrict__ csr_pair,
                                const int* __restrict__ p_lo, const double* __restrict__ p_acc,
                                DevState* st, double* __restrict__ invd, double* __restrict__ g,
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
      invd[c] = d > 0.0 ? 1.0 / d : 0.0;   // one FP64 division per component and iteration
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
  const double* invd;  // inverse Jacobi diagonal (0 for a row without entries)
  const double* g;
  const double* gabs;
  double* x;           // the solution s~ of Eq. 14
  double* p;           // search direction
  double* r[2];        // residual
  double* q[2];        // q = L p
  double* w[2];        // w = L u, u = D^-1 r
  double* u;           // cluster mode: u of every row, read by the neighbouring rows
  long long* red;      // grid mode: per-CTA partial sums, 2 slots x gridDim x 4 x (q, e)
  double* soff;
  double tol2;
  int maxit;
  int T;
  double dE_max;
  int smem_bytes;      // dynamic shared memory of the launch (CSR cache)
};

// ---- exact sums.  FP64 issues at about 2 lanes per clock per SM on this part
// (a dependent FP64 add or FMA waits 64 cycles), so a shuffle tree of FP64
// additions costs 64 cycles a level per value.  Sums here are taken in 64-bit
// fixed point: a warp finds the largest exponent E of its terms (an integer
// max), turns every term into an integer multiple of 2^(E - 1022 - S) and adds
// the integers exactly; warps, CTAs and the cluster or grid then combine their
// (integer, exponent) pairs by aligning them to the largest exponent with an
// integer shift.  One conversion back to FP64 at the end.  S = 62 - ceil(log2
// of the number of terms), so no integer sum can overflow.  Each term and each
// alignment is rounded to the grain 2^(E - 1022 - S), 2^-S of the largest
// term.  The result does not depend on the order of the terms or on which warp
// adds what: every CTA of a grid or cluster that combines the same partials
// holds the same bits.
struct Fx {
  long long q;   // value q 2^(e - 1022 - S); e = 0: zero, e = 2047: not finite
  int e;
};

__device__ __forceinline__ int fx_exp(double x) {   // biased exponent; subnormal 1, zero 0, inf/nan 2047
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  const int e = (int)(b >> 52);
  return (e == 0 && b != 0ull) ? 1 : e;
}

// x 2^(S - (E - 1022)) rounded to the nearest integer; requires fx_exp(x) <= E < 2047
__device__ __forceinline__ long long fx_quant(double x, int E, int S) {
  const long long bits = __double_as_longlong(x);
  const unsigned long long b = (unsigned long long)bits & 0x7fffffffffffffffull;
  int e = (int)(b >> 52);
  unsigned long long m = b & 0xfffffffffffffull;
  if (e == 0) {
    if (m == 0ull) return 0;
    e = 1;
  } else {
    m |= 0x10000000000000ull;   // x = m 2^(e - 1075)
  }
  const int sh = e - E + S - 53;   // <= S - 53 <= 9
  long long q;
  if (sh >= 0) q = (long long)(m << sh);
  else if (sh > -62) q = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
  else q = 0;
  return bits < 0 ? -q : q;
}

// q 2^-de rounded (de >= 0); |q| < 2^62
__device__ __forceinline__ long long fx_shift(long long q, int de) {
  if (de == 0) return q;
  if (de > 62) return 0;
  return (q + (1ll << (de - 1))) >> de;
}

__device__ __forceinline__ double fx_double(Fx a, int S) {
  if (a.e == 0) return 0.0;
  if (a.e == 2047) return __longlong_as_double(0x7ff8000000000000ll);
  return scalbn((double)a.q, a.e - 1022 - S);
}

__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(NI_FULL, v, o));
  return v;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(NI_FULL, v, o);
  return v;
}

// the terms of the 32 lanes -> one Fx, in every lane
__device__ __forceinline__ Fx warp_fx(double v, int S) {
  const int E = warp_max_i(fx_exp(v));
  if (E == 0 || E == 2047) return Fx{0, E};
  return Fx{warp_sum_ll(fx_quant(v, E, S)), E};
}

// the partials of the 32 lanes (Fx{0, 0} for none) -> one Fx, in every lane
__device__ __forceinline__ Fx warp_fx_combine(Fx a) {
  const int E = warp_max_i(a.e);
  if (E == 0 || E == 2047) return Fx{0, E};
  return Fx{warp_sum_ll(a.e == 0 ? 0ll : fx_shift(a.q, E - a.e)), E};
}

// CTA sum of NV values per thread; the result in every thread.
// shq / she: 33 * NV entries of shared memory
template <int NV>
__device__ __forceinline__ void block_fx(const double (&v)[NV], Fx (&out)[NV], int S, long long* shq, int* she) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const Fx f = warp_fx(v[k], S);
    if (lane == 0) {
      shq[wid * NV + k] = f.q;
      she[wid * NV + k] = f.e;
    }
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const Fx f = warp_fx_combine(lane < nw ? Fx{shq[lane * NV + k], she[lane * NV + k]} : Fx{0, 0});
      if (lane == 0) {
        shq[32 * NV + k] = f.q;
        she[32 * NV + k] = f.e;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = Fx{shq[32 * NV + k], she[32 * NV + k]};
}

// ---- one thread-block cluster (MODE 1): a single cluster of up to 16 CTAs on
// as many SMs; the FP64 work is spread over them and synchronisation is the
// hardware cluster barrier.  A cluster-wide sum: every CTA publishes its
// partial in its own shared memory, a cluster barrier, then warp 0 of every
// CTA reads all partials through distributed shared memory and combines them.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

__device__ __forceinline__ unsigned cluster_ctas() {
  unsigned n;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
  return n;
}

__device__ __forceinline__ unsigned dsmem_addr(const void* p, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ long long dsmem_ld_s64(const long long* p, unsigned rank) {
  long long v;
  asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(v) : "r"(dsmem_addr(p, rank)) : "memory");
  return v;
}

__device__ __forceinline__ int dsmem_ld_s32(const int* p, unsigned rank) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(dsmem_addr(p, rank)) : "memory");
  return v;
}

struct RedShared {
  long long q[33 * 4];
  int e[33 * 4];
  long long slot_q[2 * 4];   // cluster mode: this CTA's published partials, two slots used in turn
  int slot_e[2 * 4];
};

// Sum over the cluster (MODE 1) or the grid (MODE 0; one CTA: the CTA sum);
// the result in every thread.  A slot or global partial is rewritten two sums
// later, after another barrier, when every CTA has read it.
template <int MODE, int NV>
__device__ __forceinline__ bool reduce_fx(const double (&v)[NV], Fx (&out)[NV], int S, RedShared& R,
                                          long long* gred, int& ncall, DevState* st) {
  block_fx<NV>(v, out, S, R.q, R.e);
  if constexpr (MODE == 1) {
    const int s4 = 4 * (ncall & 1);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        R.slot_q[s4 + k] = out[k].q;
        R.slot_e[s4 + k] = out[k].e;
      }
    }
    ++ncall;
    cluster_barrier();   // every thread of this CTA is also past its reads of the broadcast entries
    if (threadIdx.x < 32) {
      const unsigned lane = threadIdx.x, nc = cluster_ctas();
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        Fx a{0, 0};
        if (lane < nc) a = Fx{dsmem_ld_s64(&R.slot_q[s4 + k], lane), dsmem_ld_s32(&R.slot_e[s4 + k], lane)};
        const Fx f = warp_fx_combine(a);
        if (lane == 0) {
          R.q[32 * NV + k] = f.q;
          R.e[32 * NV + k] = f.e;
        }
      }
    }
  } else {
    if (gridDim.x == 1) return true;
    const int nb = gridDim.x;
    long long* G = gred + (size_t)(ncall & 1) * nb * 8;
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        G[blockIdx.x * 8 + 2 * k] = out[k].q;
        G[blockIdx.x * 8 + 2 * k + 1] = out[k].e;
      }
    }
    ++ncall;
    if (!grid_barrier(&st->bar, &st->err)) return false;
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        // fold this lane's CTAs (aligned to their largest exponent), then the lanes
        int e = 0;
        for (int b = lane; b < nb; b += 32) e = max(e, (int)__ldcg(&G[b * 8 + 2 * k + 1]));
        long long q = 0;
        if (e != 2047) {
          for (int b = lane; b < nb; b += 32) {
            const int eb = (int)__ldcg(&G[b * 8 + 2 * k + 1]);
            if (eb != 0) q += fx_shift(__ldcg(&G[b * 8 + 2 * k]), e - eb);
          }
        }
        const Fx f = warp_fx_combine(Fx{q, e});
        if (lane == 0) {
          R.q[32 * NV + k] = f.q;
          R.e[32 * NV + k] = f.e;
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = Fx{R.q[32 * NV + k], R.e[32 * NV + k]};
  return true;
}

// The rows a CTA owns are one contiguous range [lo, hi); thread t owns rows
// lo + t + k blockDim.  The CTA's slice of the CSR (row pointers made local,
// column indices, weights) is copied into shared memory when it fits.
struct RowSlice {
  int lo, hi, base;
  bool cached;
  const int* rp;      // local row pointers (cached) or the global ones
  const int* col;
  const double* wgt;
};

// w_c = sum_j w_cj (u_c - u_j) for the rows this thread owns, in a warp-uniform
// traversal: a warp visits 32 consecutive rows together; rows of at most 32
// entries take one thread, longer ones (the quotient graph's degrees follow the
// component sizes: a large component borders hundreds of small ones) are then
// done by the whole warp one after the other.  uj(j) gives u_j; row(c, u_c, w_c)
// is called once per owned row c, by its owning thread, and returns the row's
// three inner-product terms, summed into s0, s1, s2.
struct Terms3 {
  double a, b, c;
};

template <class UJ, class ROW>
__device__ __forceinline__ void spmv_rows(const RowSlice& RS, UJ uj, ROW row, double& s0, double& s1, double& s2) {
  const int lane = threadIdx.x & 31;
  for (int c0 = RS.lo + threadIdx.x - lane; c0 < RS.hi; c0 += blockDim.x) {   // warp-uniform
    const int c = c0 + lane;
    const bool own = c < RS.hi;
    int b = 0, e = 0;
    double uc = 0.0;
    if (own) {
      const int i = RS.cached ? c - RS.lo : c;
      b = RS.rp[i];
      e = RS.rp[i + 1];
      uc = uj(c);
    }
    const bool lng = e - b > 32;
    double acc = 0.0;
    if (own && !lng) {
#pragma unroll 4
      for (int j = b; j < e; ++j) acc += RS.wgt[j] * (uc - uj(RS.col[j]));
    }
    unsigned m = __ballot_sync(NI_FULL, lng);
    while (m) {
      const int l = __ffs(m) - 1;
      m &= m - 1;
      const int rb = __shfl_sync(NI_FULL, b, l), re = __shfl_sync(NI_FULL, e, l);
      const double ur = __shfl_sync(NI_FULL, uc, l);
      double a2 = 0.0;
#pragma unroll 4
      for (int j = rb + lane; j < re; j += 32) a2 += RS.wgt[j] * (ur - uj(RS.col[j]));
      a2 = warp_sum_d(a2);
      if (lane == l) acc = a2;
    }
    if (own) {
      const Terms3 t = row(c, uc, acc);
      s0 += t.a;
      s1 += t.b;
      s2 += t.c;
    }
  }
}

// The relative-scale solve s~ <- cg(A^T W A, A^T W b) (Eq. 14) on the quotient
// Laplacian L (CSR, FP64), Jacobi-preconditioned, from s~ = 0, in the
// single-reduction form of Chronopoulos and Gear: with u = D^-1 r and w = L u,
// one iteration is
//   p = u + beta p,  q = w + beta q  (q = L p),  x += alpha p,  r -= alpha q,
//   u = D^-1 r,  w = L u,  gamma = r.u,  delta = w.u,  rho = r.r,
//   beta' = gamma' / gamma,  alpha' = gamma' / (delta' - beta' gamma' / alpha),
// so the three inner products share one grid-wide sum.
//   MODE 0 (one CTA or a cooperative grid): one pass per iteration.  Each row
//     recomputes its neighbours' new u from their r, w and q of the previous
//     iteration (the same FMAs their owners evaluate, so the same bits); r, q
//     and w are double-buffered so no pass reads what it writes.
//   MODE 1 (one cluster): two passes per iteration, the row updates (storing
//     u) and then w = L u with the inner products, a cluster barrier between.
// Thread 0 turns the sums into the scalars (two independent divisions an
// iteration) and broadcasts them.
// threads of a cluster-mode CTA: each thread owns about K / (16 x 512) rows, so
// fewer of its rows' dependent loads (L2 gathers of the neighbours' u) queue
// behind one another than with 256
#define NI_SCALE_CL_THREADS 512
template <int MODE>
__global__ void __launch_bounds__(MODE == 1 ? NI_SCALE_CL_THREADS : 256, 1) k_scale_cg(ScaleArgs A) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ RedShared R;
  __shared__ double sc[4];   // alpha, beta, done
  DevState* st = A.st;
  if (*(volatile int*)&st->converged) return;
  const int K = st->K, P = st->nP;
  int ncall = 0;
  // fixed-point grain: the number of terms of a sum is at most the launch's threads
  const int S = 62 - (32 - __clz(gridDim.x * blockDim.x - 1));
  // this CTA's rows and CSR slice
  RowSlice RS;
  {
    const int per = (K + gridDim.x - 1) / gridDim.x;
    RS.lo = min(K, blockIdx.x * per);
    RS.hi = min(K, RS.lo + per);
    RS.base = A.row_ptr[RS.lo];
    const int nnz = A.row_ptr[RS.hi] - RS.base;
    const long long need = 4ll * (RS.hi - RS.lo + 2) + 12ll * nnz + 16;
    RS.cached = need <= (long long)A.smem_bytes;
    if (RS.cached) {
      int* rp = reinterpret_cast<int*>(dyn);
      double* wv = reinterpret_cast<double*>(dyn + ((4 * (RS.hi - RS.lo + 2) + 15) & ~15));
      int* cl = reinterpret_cast<int*>(wv + nnz);
      for (int i = threadIdx.x; i <= RS.hi - RS.lo; i += blockDim.x) rp[i] = A.row_ptr[RS.lo + i] - RS.base;
      for (int j = threadIdx.x; j < nnz; j += blockDim.x) {
        wv[j] = A.csr_w[RS.base + j];
        cl[j] = A.csr_col[RS.base + j];
      }
      RS.rp = rp;
      RS.col = cl;
      RS.wgt = wv;
      __syncthreads();
    } else {
      RS.rp = A.row_ptr;
      RS.col = A.csr_col;
      RS.wgt = A.csr_w;
    }
  }
  const double* __restrict__ invd = A.invd;
  // x0 = 0: r0 = g, u0 = D^-1 g, w0 = L u0 (g and D are inputs: no sync needed)
  double i0 = 0.0, i1 = 0.0, i2 = 0.0;   // gamma, delta, rho
  spmv_rows(RS, [&](int j) { return invd[j] * A.g[j]; },
            [&](int c, double uc, double wc) {
              const double gc = A.g[c];
              A.x[c] = 0.0;
              A.p[c] = 0.0;
              A.r[0][c] = gc;
              A.q[0][c] = 0.0;
              A.w[0][c] = wc;
              return Terms3{gc * uc, wc * uc, gc * gc};
            }, i0, i1, i2);
  double ga = 0.0;
  for (int c = RS.lo + threadIdx.x; c < RS.hi; c += blockDim.x) ga += A.gabs[c] * A.gabs[c];
  // thread 0 keeps gamma, 1 / gamma and 1 / alpha of the previous iteration
  double gamma = 0.0, rgamma = 0.0, ralpha = 0.0;
  {
    const double v4[4] = {i0, i1, i2, ga};   // gamma, delta, rho, sum gabs^2
    Fx f4[4];
    if (!reduce_fx<MODE, 4>(v4, f4, S, R, A.red, ncall, st)) return;
    if (threadIdx.x == 0) {
      const double gm = fx_double(f4[0], S), dl = fx_double(f4[1], S), rh = fx_double(f4[2], S);
      // stop at the relative tolerance, or once the residual is at the rounding
      // level of the terms that cancel in g (a system that is already solved has
      // a right-hand side made of rounding noise)
      const double floor2 = (64.0 * 1.1102230246251565e-16) * (64.0 * 1.1102230246251565e-16) * fx_double(f4[3], S);
      const double stop2 = fmax(A.tol2 * rh, floor2);
      const bool ok = dl > 0.0 && gm > 0.0;
      sc[0] = ok ? gm / dl : 0.0;
      sc[1] = 0.0;
      sc[2] = (!(rh > 0.0) || rh <= stop2 || !ok) ? 1.0 : 0.0;
      sc[3] = stop2;
      gamma = gm;
      rgamma = ok ? 1.0 / gm : 0.0;
      ralpha = ok ? dl / gm : 0.0;
    }
    __syncthreads();
  }
  double alpha = sc[0], beta = 0.0;
  const double stop2 = sc[3];
  bool done = sc[2] != 0.0;
  int it = 0, b = 0;
  while (!done && it < A.maxit) {
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;   // gamma', delta', rho'
    if constexpr (MODE == 0) {
      const double* __restrict__ ro = b ? A.r[1] : A.r[0];
      const double* __restrict__ qo = b ? A.q[1] : A.q[0];
      const double* __restrict__ wo = b ? A.w[1] : A.w[0];
      double* __restrict__ rn = b ? A.r[0] : A.r[1];
      double* __restrict__ qn = b ? A.q[0] : A.q[1];
      double* __restrict__ wn = b ? A.w[0] : A.w[1];
      spmv_rows(RS, [&](int j) { return invd[j] * fma(-alpha, fma(beta, qo[j], wo[j]), ro[j]); },
                [&](int c, double uc, double wc) {
                  const double qc = fma(beta, qo[c], wo[c]);
                  const double rc = fma(-alpha, qc, ro[c]);
                  const double pc = fma(beta, A.p[c], invd[c] * ro[c]);
                  A.x[c] = fma(alpha, pc, A.x[c]);
                  A.p[c] = pc;
                  qn[c] = qc;
                  rn[c] = rc;
                  wn[c] = wc;
                  return Terms3{rc * uc, wc * uc, rc * rc};
                }, t0, t1, t2);
      b ^= 1;
    } else {
      double* __restrict__ r = A.r[0];
      double* __restrict__ q = A.q[0];
      double* __restrict__ w = A.w[0];
      double* __restrict__ u = A.u;
      for (int c = RS.lo + threadIdx.x; c < RS.hi; c += blockDim.x) {
        const double qc = fma(beta, q[c], w[c]);
        const double rc = fma(-alpha, qc, r[c]);
        const double pc = fma(beta, A.p[c], invd[c] * r[c]);
        A.x[c] = fma(alpha, pc, A.x[c]);
        A.p[c] = pc;
        q[c] = qc;
        r[c] = rc;
        u[c] = invd[c] * rc;
      }
      cluster_barrier();
      spmv_rows(RS, [&](int j) { return u[j]; },
                [&](int c, double uc, double wc) {
                  const double rc = r[c];
                  w[c] = wc;
                  return Terms3{rc * uc, wc * uc, rc * rc};
                }, t0, t1, t2);
    }
    const double v3[3] = {t0, t1, t2};
    Fx f3[3];
    if (!reduce_fx<MODE, 3>(v3, f3, S, R, A.red, ncall, st)) return;
    if (threadIdx.x == 0) {
      const double gm = fx_double(f3[0], S), dl = fx_double(f3[1], S), rh = fx_double(f3[2], S);
      const double bt = gm * rgamma;                  // gamma' / gamma
      const double den = dl - bt * gm * ralpha;       // delta' - beta' gamma' / alpha
      const bool ok = den > 0.0 && gm > 0.0;
      const double rden = ok ? 1.0 / den : 0.0;       // the two divisions are independent
      const double rgm = ok ? 1.0 / gm : 0.0;
      sc[0] = gm * rden;
      sc[1] = bt;
      sc[2] = (rh <= stop2 || !ok) ? 1.0 : 0.0;
      gamma = gm;
      rgamma = rgm;
      ralpha = den * rgm;                             // 1 / alpha'
    }
    __syncthreads();
    alpha = sc[0];
    beta = sc[1];
    done = sc[2] != 0.0;   // sc is rewritten only after the next sum's CTA barriers
    ++it;
  }
  // energy of the solved system: sum_p w_p D^2 + 2 h_p D + q_p, D = s_lo - s_hi
  double en = 0.0;
  {
    const int per = (P + gridDim.x - 1) / gridDim.x;
    const int p0 = min(P, (int)blockIdx.x * per), p1 = min(P, p0 + per);
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
      const double D = A.x[A.p_lo[p]] - A.x[A.p_hi[p]];
      en += A.p_acc[3 * p] * D * D + 2.0 * A.p_acc[3 * p + 1] * D + A.p_acc[3 * p + 2];
    }
  }
  const double v1[1] = {en};
  Fx f1[1];
  if (!reduce_fx<MODE, 1>(v1, f1, S, R, A.red, ncall, st)) return;
  // no CTA of a cluster may exit while another still reads its shared memory
  if constexpr (MODE == 1) cluster_barrier();
  for (int c = RS.lo + threadIdx.x; c < RS.hi; c += blockDim.x) A.soff[c] += A.x[c];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double E = fx_double(f1[0], S);
    const int t = st->t + 1;
    st->t = t;
    if (t <= NI_MAX_T) st->E[t] = E;
    st->scale_cg_last = it;
    st->scale_cg_total += (unsigned long long)it;
    if (it > st->scale_cg_iters) st->scale_cg_iters = it;
    if (it >= A.maxit && !done) st->err |= NI_DEV_ERR_SCALE_NOCONV;
    bool conv = t >= A.T;
    if (!conv && t >= 4 && t <= NI_MAX_T) {
      const double e0 = st->E[t - 1];
      conv = (e0 < 1e-300) || (fabs(E - e0) / e0 < A.dE_max);
    }
    st->converged = conv ? 1 : 0;
  }
}

#define NI_SCALE_THREADS 256
// dynamic shared memory of a scale PCG CTA: its slice of the quotient CSR
#define NI_SCALE_SMEM (192 * 1024)

static void scale_kernel_attrs() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute((const void*)k_scale_cg<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, NI_SCALE_SMEM);
  cudaFuncSetAttribute((const void*)k_scale_cg<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, NI_SCALE_SMEM);
  cudaFuncSetAttribute((const void*)k_scale_cg<1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaGetLastError();
  done = true;
}
// MODE 0: one CTA of 256 threads per 256 components, at most one per SM (the
// FP64 rate is per SM), cooperatively launched when there is more than one
int scale_cg_grid(ni_handle* h) {
  scale_kernel_attrs();
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scale_cg<0>, NI_SCALE_THREADS, NI_SCALE_SMEM);
  if (per_sm < 1) return 1;
  const int need = (h->Kcap + NI_SCALE_THREADS - 1) / NI_SCALE_THREADS;
  return std::max(1, std::min(h->num_sms, need));
}

// Cluster-mode scale PCG: CTAs of NI_SCALE_CL_THREADS threads, 16 per cluster (a non-portable
// size) where the device can schedule that, else 8, else none.

static cudaLaunchConfig_t cluster_cfg(int nc, cudaLaunchAttribute* at, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(NI_SCALE_CL_THREADS);
  cfg.dynamicSmemBytes = NI_SCALE_SMEM;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = nc;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

int scale_cluster_size(ni_handle* h) {
  if (h->scale_cluster >= 0) return h->scale_cluster;
  h->scale_cluster = 0;
  scale_kernel_attrs();
  for (int nc = 16; nc >= 8; nc /= 2) {
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_cfg(nc, at, 0);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (const void*)k_scale_cg<1>, &cfg) == cudaSuccess && n >= 1) {
      h->scale_cluster = nc;
      break;
    }
    cudaGetLastError();
  }
  return h->scale_cluster;
}

// the cluster unless the caller asks for the grid (measured faster on every map
// here, from 885 to 26193 components) or the device cannot schedule it
static bool use_scale_cluster(ni_handle* h) {
  if (h->cfg.scale_solver == 2) return false;
  return scale_cluster_size(h) > 0;
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
  ea.bini_res = h->cfg.bini_residual;
  ea.lw = h->cfg.learned_weights ? h->lw : nullptr;
  if (h->cfg.connectivity == 8) k_edge_accum<8><<<ge, 256, 0, s>>>(ea);
  else k_edge_accum<4><<<ge, 256, 0, s>>>(ea);
  NI_COUNT(h);
  k_node_assemble<<<grid_lin(h, 32LL * h->Kcap), 256, 0, s>>>(h->row_ptr, h->csr_pair, h->p_lo, h->p_acc, st,
                                                        h->sd, h->sv + 5 * (size_t)h->Kcap,
                                                        h->sv + 6 * (size_t)h->Kcap, h->csr_w); NI_COUNT(h);
  ScaleArgs sa;
  const size_t kc = (size_t)h->Kcap;
  sa.st = st; sa.row_ptr = h->row_ptr; sa.csr_col = h->csr_col; sa.csr_w = h->csr_w; sa.csr_pair = h->csr_pair;
  sa.p_lo = h->p_lo; sa.p_hi = h->p_hi; sa.p_acc = h->p_acc; sa.invd = h->sd;
  // h->sv: x, r0, r1, p, q0, g, gabs, q1, w0, w1, u (Kcap doubles each)
  sa.g = h->sv + 5 * kc;
  sa.gabs = h->sv + 6 * kc;
  sa.x = h->sv;
  sa.r[0] = h->sv + kc; sa.r[1] = h->sv + 2 * kc;
  sa.p = h->sv + 3 * kc;
  sa.q[0] = h->sv + 4 * kc; sa.q[1] = h->sv + 7 * kc;
  sa.w[0] = h->sv + 8 * kc; sa.w[1] = h->sv + 9 * kc;
  sa.u = h->sv + 10 * kc;
  sa.red = reinterpret_cast<long long*>(h->cacc);   // 2 x grid x 8 (the component accumulators are free here)
  sa.smem_bytes = NI_SCALE_SMEM;
  sa.soff = h->soff;
  sa.tol2 = h->cfg.scale_rtol * h->cfg.scale_rtol;
  sa.maxit = h->cfg.scale_maxit > 0 ? h->cfg.scale_maxit : std::min(4 * h->Kcap + 100, 200000);
  sa.T = h->cfg.T;
  sa.dE_max = h->cfg.dE_max;
  if (use_scale_cluster(h)) {
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_cfg(h->scale_cluster, at, s);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_scale_cg<1>, sa);
    NI_COUNT(h);
    if (e != cudaSuccess) return ni_cuda_check(h, e, "scale PCG cluster launch");
    return ni_cuda_check(h, cudaGetLastError(), "scale iteration");
  }
  const int grid = scale_cg_grid(h);
  if (grid == 1) {
    k_scale_cg<0><<<1, NI_SCALE_THREADS, NI_SCALE_SMEM, s>>>(sa); NI_COUNT(h);
  } else {
    cudaMemsetAsync(&st->bar, 0, sizeof(GridBar), s);
    void* args[] = {&sa};
    cudaError_t e = cudaLaunchCooperativeKernel((void*)k_scale_cg<0>, dim3(grid), dim3(NI_SCALE_THREADS), args,
                                                NI_SCALE_SMEM, s);
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
