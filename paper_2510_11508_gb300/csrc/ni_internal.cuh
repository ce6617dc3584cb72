// Internal declarations shared by the translation units of libni (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ni.h"

#define NI_WARP 32
#define NI_FULL 0xffffffffu

// ----------------------------------------------------------------------------
// device-side error bits (DevState::err)
// ----------------------------------------------------------------------------
#define NI_DEV_ERR_TIMEOUT 1
#define NI_DEV_ERR_BAD_NORMAL 2
#define NI_DEV_ERR_FILL_NOCONV 4
#define NI_DEV_ERR_SCALE_NOCONV 8
#define NI_DEV_ERR_OVERFLOW 16

// A bounded spin: ~2 s at 2 GHz before a wait gives up and flags a timeout.
#define NI_SPIN_LIMIT_CYCLES (4000000000LL)

#define NI_MAX_T 256
#define NI_MG_MAX_LEVELS 24   // multigrid levels of the fill (2^24 > any image side)

// kernel-launch counter of a handle (graph replays add their captured count)
#define NI_COUNT(h) ((h)->launches++)

struct GridBar {
  unsigned int count;
  unsigned int gen;
};

// Scalars that live on the device so that loops can run (and be captured in a
// CUDA graph) without host round trips.
struct DevState {
  int K;           // components of the current partition
  int K0;          // components after seeding
  int nE;          // inter-component edges of the current partition
  int nP;          // distinct component pairs joined by inter edges
  int t;           // relative-scale iterations done
  int converged;   // stop test of Algorithm 1 fired
  int merges;      // merges done
  int err;         // NI_DEV_ERR_* bits
  int n_bad_normals;
  int fill_iters;
  int fill_unconv;
  int scale_cg_iters;
  int scale_cg_last;
  int cg_done;     // plain fill PCG: converged flag
  int cg_it;       // plain fill PCG: iterations
  int gate;        // merge kernels of this iteration run (1) or not (0)
  int n_valid;     // valid pixels of the map
  int warm_fallbacks;  // components whose warm start was scaled to zero (cold start)
  unsigned long long fill_px_iters;  // sum over components of size x PCG iterations
  unsigned long long scale_cg_total; // scale-PCG iterations summed over the loop
  double E[NI_MAX_T + 1];  // E[0] = eps, E[t] after iteration t
  double cg[8];            // plain fill PCG scalars
  GridBar bar;             // software grid barrier of persistent kernels
  GridBar bar2;
};

// Plain PCG scalar slots in DevState::cg
#define CG_RZ 0
#define CG_RZNEW 1
#define CG_PAP 2
#define CG_RR 3
#define CG_BB 4

struct ni_cnn;

// One row of a tuning table (ni_load_tuning): the knobs for maps of at most
// max_px grid pixels and max_k0 components after seeding.
struct TuneRow {
  long long max_px;
  long long max_k0;
  int ctas_per_sm;
  int mg_cta_cells;
  double mg_omega;
  int scale_solver;
};

struct ni_handle {
  ni_config cfg;
  ni_config cfg_user;          // the configuration as given: 0 knobs are the tuning table's to set
  std::vector<TuneRow> tune;
  float4* lw = nullptr;        // network's continuity of the right, down, left, up edge per pixel
  int dev = 0;
  int num_sms = 0;
  int scale_cluster = -1;      // CTAs of the cluster-mode scale PCG (-1 not yet queried, 0 unavailable)
  int H = 0, W = 0;
  int N = 0;
  int Npad = 0;                // N rounded up to a multiple of 1024 (allocation size)
  int ntiles = 0;              // 32 x 32 tiles of the batched PCG
  int ntx = 0;                 // tiles per tile row
  double cos_theta = 2.0;   // > 1 keeps no edge (theta_c = None)
  float fx = 1, fy = 1, cx = 0, cy = 0;
  int persp = 1;

  // caller-owned inputs kept between stage calls
  const float4* normals = nullptr;
  const uint8_t* mask = nullptr;

  // per-pixel workspace
  int32_t* labels = nullptr;   // current partition pi (-1 invalid)
  int32_t* parent = nullptr;   // union-find scratch / previous labels
  float2* omega = nullptr;     // omega~_{b->a} of the right (x) and down (y) edge
  float* ntau = nullptr;       // n_a . tau_a (n_az for orthographic)
  float* wr = nullptr;         // combined fill weight of the edge to the right
  float* wd = nullptr;         // combined fill weight of the edge below
  // 8-connectivity only (NULL otherwise): the diagonal edges of pixel a, to the
  // lower-right (a + W + 1) and lower-left (a + W - 1) neighbour
  float2* omega_d = nullptr;   // omega~_{b->a} of the lower-right (x) and lower-left (y) edge
  float* wdr = nullptr;        // combined fill weight of the lower-right edge
  float* wdl = nullptr;        // combined fill weight of the lower-left edge
  float* invd = nullptr;       // 1 / Jacobi diagonal (0 where the diagonal is 0)
  float* x = nullptr;          // log-depth relative to the component offset
  float* r = nullptr;
  float* p = nullptr;
  float* p2 = nullptr;
  float* q = nullptr;
  float* b = nullptr;          // right-hand side of the fill normal equations

  int* tile_lab = nullptr;     // uniform label of each tile or -1
  int* tiles = nullptr;        // active tile lists of the batched PCG [2][ntiles] x (tile, label)

  // scan scratch
  int* blk = nullptr;          // block partial sums (NI_SCAN_BLOCKS + 1)
  int* d_count = nullptr;

  // component-sized (capacity Kcap)
  int Kcap = 0;
  double* soff = nullptr;      // per-component log-depth offset (lazy Eq. 8 update)
  double* soff2 = nullptr;
  double* cacc = nullptr;      // per-component accumulators [6 * Kcap]
  int* cflag = nullptr;        // per-component flags / iteration counts [2 * Kcap]
  int* kparent = nullptr;      // union-find over components
  int* kmap = nullptr;         // old label -> new label
  unsigned long long* kkey = nullptr;  // merge keys
  double* sv = nullptr;        // scale PCG vectors [7 * Kcap]: s, r, z, p, q, g, |g| terms
  double* sd = nullptr;        // diagonal of the quotient Laplacian
  int* row_ptr = nullptr;      // CSR of the quotient graph [Kcap + 1]

  // edge-sized (capacity Ecap)
  int Ecap = 0;
  int* e_id = nullptr;         // inter edge ids (2 * a + dir), partition order
  int* e_id2 = nullptr;
  unsigned long long* e_key = nullptr;   // sort keys
  unsigned long long* e_key2 = nullptr;
  int* e_val = nullptr;        // sort values
  int* e_val2 = nullptr;
  int* e_pair = nullptr;       // pair index per sorted edge
  int* p_lo = nullptr;         // pair endpoints (lo < hi)
  int* p_hi = nullptr;
  double* p_acc = nullptr;     // per pair: w, h, q  [3 * Ecap]
  unsigned long long* c_key = nullptr;   // sort scratch of the CSR entries [2 * Ecap]
  int* c_val = nullptr;
  int* csr_col = nullptr;      // [2 * Ecap]
  int* csr_pair = nullptr;     // [2 * Ecap]
  double* csr_w = nullptr;     // [2 * Ecap] pair weight of each CSR entry (per scale iteration)
  int* radix_hist = nullptr;   // [256 * NI_SORT_BLOCKS]

  // multigrid hierarchy of the fill (precond = 1): coarse levels 1..mg_L in pools
  int mg_L = 0;
  int mg_h[NI_MG_MAX_LEVELS + 1] = {}, mg_w[NI_MG_MAX_LEVELS + 1] = {};
  long long mg_off[NI_MG_MAX_LEVELS + 1] = {};
  long long mg_cells = 0;      // pool size (0: not allocated)
  int* mg_lab = nullptr;
  float* mg_wr = nullptr;
  float* mg_wd = nullptr;
  float* mg_d = nullptr;       // leak: diagonal minus the cell's edge weights
  float* mg_invd = nullptr;
  float* mg_b = nullptr;       // restricted residuals
  float* mg_e = nullptr;       // coarse corrections
  uint8_t* mg_inc = nullptr;   // cell aggregated into its parent
  uint8_t* inc0 = nullptr;     // the same for the pixels
  GridBar* mg_bar = nullptr;   // barriers of the coarse-level passes [2 * (NI_MG_MAX_LEVELS + 1)]
  int* mg_iter = nullptr;      // per-phase multigrid solve: iteration index and done flag
  int2* mg_tact = nullptr;     // persistent multigrid solve: active tile lists, two by iteration parity
  int fill_fallbacks = 0;      // components the Jacobi fallback re-solved in this call
  float* z = nullptr;          // preconditioned residual

  DevState* st = nullptr;      // device
  DevState* st_host = nullptr; // pinned mirror

  cudaEvent_t ev[8] = {};
  int stage = 0;               // 0 created, 1 seeded, 2 filled
  int K_host = 0;
  int t_host = 0;
  int sort_passes = 0;
  std::string err;

  long long launches = 0;          // kernels launched through this handle
  long long scale_graph_count = 0; // kernels in the relative-scale graph
  float ms_fill_solve = 0.f;       // PCG kernel time of the last fill

  // CUDA graph of the relative-scale loop
  cudaGraphExec_t scale_graph = nullptr;
  long long graph_key[6] = {-1, -1, -1, -1, -1, -1};

  // learned warm start (ni_load_net)
  ni_cnn* net = nullptr;
  float* tile_in = nullptr;
  float* tile_out = nullptr;

  // scratch of ni_min_made (allocated on first use)
  struct MadeScratch* made = nullptr;

  // device copies for ni_integrate_host
  float4* in_normals = nullptr;
  uint8_t* in_mask = nullptr;
  float* out_depth = nullptr;
};

// ----------------------------------------------------------------------------
// launch geometry
// ----------------------------------------------------------------------------
#define NI_MG_MAX_LEVELS 24
#define NI_TILE_PX 1024
#define NI_TILE_W 32
#define NI_TILE_H 32
#define NI_TILE_THREADS 256
// Seeding tile of k_seed_local (one CTA of NI_SEED_TSW x NI_SEED_TSH threads per
// tile); every launch of the seeding kernels takes its tile shape from here.
#define NI_SEED_TSW 32
#define NI_SEED_TSH 16
#define NI_SCAN_BLOCKS 1024
#define NI_SCAN_THREADS 512
#define NI_SORT_BLOCKS 256
#define NI_SORT_THREADS 256

// ----------------------------------------------------------------------------
// host helpers implemented in ni_api.cu
// ----------------------------------------------------------------------------
ni_status ni_fail(ni_handle* h, ni_status s, const std::string& msg);
ni_status ni_cuda_check(ni_handle* h, cudaError_t e, const char* what);

// ni_seed.cu
ni_status seed_launch(ni_handle* h, cudaStream_t s);
// exclusive scan of the flags produced by `Pred`, see ni_seed.cu
void scan_blocks_launch(int* blk, int nblocks, int* total_out, cudaStream_t s);

// ni_fill.cu
ni_status fill_setup_launch(ni_handle* h, cudaStream_t s);
ni_status fill_solve_launch(ni_handle* h, cudaStream_t s);
ni_status mg_solve_launch(ni_handle* h, cudaStream_t s);
void free_mg(ni_handle* h);
void export_logdepth_launch(ni_handle* h, float* out, cudaStream_t s);
void import_logdepth_launch(ni_handle* h, const float* in, cudaStream_t s);
void output_depth_launch(ni_handle* h, float* depth, cudaStream_t s);

// ni_scale.cu
ni_status partition_build_launch(ni_handle* h, int first, cudaStream_t s);
ni_status scale_iteration_launch(ni_handle* h, cudaStream_t s);
ni_status merge_launch(ni_handle* h, const float* chi_abs, cudaStream_t s);
int scale_cg_grid(ni_handle* h);
void merge_gate_launch(ni_handle* h, int tgate, int force, cudaStream_t s);
ni_status ensure_edge_capacity(ni_handle* h, int nE);
ni_status ensure_component_capacity(ni_handle* h, int K);

// ni_made.cu
void free_made(ni_handle* h);

// ni_cnn.cu
ni_status warm_start_launch(ni_handle* h, cudaStream_t s);

// ----------------------------------------------------------------------------
// device helpers
// ----------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(NI_FULL, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(NI_FULL, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(NI_FULL, v, o);
  return v;
}

// Block-wide sum (all threads call; result valid in every thread).
// `sh` must hold at least blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum_d(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int block_sum_i(int v, int* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum_i(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0;
  if (wid == 0) t = warp_sum_i(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  int r = sh[0];
  __syncthreads();
  return r;
}

// Exclusive block scan of ints; returns the exclusive prefix, *total = block sum.
__device__ __forceinline__ int block_excl_scan_i(int v, int* sh, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(NI_FULL, incl, o);
    if (lane >= o) incl += y;
  }
  __syncthreads();
  if (lane == 31) sh[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int t = (lane < nw) ? sh[lane] : 0;
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(NI_FULL, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < nw) sh[lane] = ti - t;   // exclusive warp offsets
    if (lane == 31) sh[32] = ti;        // block total
  }
  __syncthreads();
  int res = sh[wid] + incl - v;
  *total = sh[32];
  __syncthreads();
  return res;
}

// Segmented (by equal consecutive `key` across the lanes of a warp) sum of up to
// three values; the last lane of each run adds the run's sums into
// acc[key * stride + j * jstride].  Lanes with key < 0 contribute nothing.
// All 32 lanes must call it.
template <int NV>
__device__ __forceinline__ void seg_add_d(double* acc, int stride, int key, double (&v)[NV],
                                          size_t jstride = 1) {
  const unsigned lane = threadIdx.x & 31;
  int prev = __shfl_up_sync(NI_FULL, key, 1);
  int next = __shfl_down_sync(NI_FULL, key, 1);
  bool head = (lane == 0) || (prev != key);
  bool tail = (lane == 31) || (next != key);
  unsigned heads = __ballot_sync(NI_FULL, head);
  unsigned below = heads & ((2u << lane) - 1u);   // heads at lanes <= lane
  int my_head = 31 - __clz(below);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double y = __shfl_up_sync(NI_FULL, v[j], o);
      if ((int)lane - o >= my_head) v[j] += y;
    }
  }
  if (tail && key >= 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j)
      if (v[j] != 0.0) atomicAdd(&acc[(size_t)key * stride + j * jstride], v[j]);
  }
}

template <int NV>
__device__ __forceinline__ void seg_add_f(double* acc, int stride, int key, float (&v)[NV],
                                          size_t jstride = 1) {
  const unsigned lane = threadIdx.x & 31;
  int prev = __shfl_up_sync(NI_FULL, key, 1);
  int next = __shfl_down_sync(NI_FULL, key, 1);
  bool head = (lane == 0) || (prev != key);
  bool tail = (lane == 31) || (next != key);
  unsigned heads = __ballot_sync(NI_FULL, head);
  unsigned below = heads & ((2u << lane) - 1u);
  int my_head = 31 - __clz(below);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      float y = __shfl_up_sync(NI_FULL, v[j], o);
      if ((int)lane - o >= my_head) v[j] += y;
    }
  }
  if (tail && key >= 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j)
      if (v[j] != 0.0f) atomicAdd(&acc[(size_t)key * stride + j * jstride], (double)v[j]);
  }
}

// Union-find root walk (read-only).  Parents only ever point to smaller
// indices, so a tree's root is its smallest member and every walk ends.
__device__ __forceinline__ int uf_find(const int* P, int x) {
  int p = P[x];
  while (p != x) {
    x = p;
    p = P[x];
  }
  return x;
}

// Link the trees of a and b, the larger root under the smaller one.
__device__ __forceinline__ void uf_unite(int* P, int a, int b) {
  while (true) {
    a = uf_find(P, a);
    b = uf_find(P, b);
    if (a == b) return;
    if (a > b) { int t = a; a = b; b = t; }
    int old = atomicMin(&P[b], a);
    if (old == b) return;     // b was a root and now hangs under a
    b = old;                  // b had been linked meanwhile; retry from its parent
  }
}

// Software grid barrier for cooperatively launched kernels.  Every wait is
// bounded: after NI_SPIN_LIMIT_CYCLES the block flags NI_DEV_ERR_TIMEOUT and
// returns false (as it does when another block has flagged a timeout), so the
// caller returns instead of hanging.
// grid_barrier_n: the same among the first n blocks (only they call it).
__device__ __forceinline__ bool grid_barrier_n(GridBar* bar, unsigned int n, int* err) {
  __shared__ int s_fail;
  __syncthreads();
  if (threadIdx.x == 0) {
    int fail = 0;
    volatile unsigned int* vgen = &bar->gen;
    unsigned int g = *vgen;
    __threadfence();
    unsigned int arrived = atomicAdd(&bar->count, 1u) + 1u;
    if (arrived == n) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long t0 = clock64();
      while (*vgen == g) {
        if (*(volatile int*)err & NI_DEV_ERR_TIMEOUT) { fail = 1; break; }
        if (clock64() - t0 > NI_SPIN_LIMIT_CYCLES) {
          atomicOr(err, NI_DEV_ERR_TIMEOUT);
          fail = 1;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    s_fail = fail;
  }
  __syncthreads();
  int f = s_fail;
  __syncthreads();
  return f == 0;
}

__device__ __forceinline__ bool grid_barrier(GridBar* bar, int* err) {
  return grid_barrier_n(bar, gridDim.x, err);
}

__device__ __forceinline__ float2 ldg2(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

#endif  // __CUDACC__
