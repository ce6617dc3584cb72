// Quality diagnostic ni_min_made: the smallest mean absolute depth error that
// one scale per component can reach (supplementary material, the section on the
// components found for different theta_c), and with a single component the
// error after the best global scale.
//
// Per component c the error E_c(s) = sum_i w_i |s - r_i| is convex and
// piecewise linear: perspective r = g / d, w = d (|s d - g| = d |s - r|),
// orthographic offsets r = g - d, w = 1.  Its minimum lies at the smallest s
// with W_le(s) = sum_{r_i <= s} w_i >= W_c / 2.  All components are bisected
// at once: a pass over the pixels adds W_le(mid_c) per component (warp-
// aggregated FP64 atomics), then one thread per component halves its bracket
// [lo, hi] (W_le(lo) < W_c / 2 <= W_le(hi)).  Bisection ends when no double
// lies strictly between lo and hi, so hi is the breakpoint itself, or after
// NI_MADE_MAX_PASSES halvings.  A last pass sums |s d - g| (|d + s - g|) at
// s = hi.
#include <math.h>

#include <algorithm>

#include "ni_internal.cuh"

#define NI_MADE_MAX_PASSES 160
#define NI_MADE_CHUNK 16

struct MadeScratch {
  long long ncap = 0;
  int kcap = 0;
  int* key = nullptr;          // per pixel: component, or -1 if the pixel does not count
  double* r = nullptr;         // per pixel: g / d (perspective) or g - d
  double* w = nullptr;         // per pixel: d (perspective) or 1
  double* lo = nullptr;        // per component bracket and sums
  double* hi = nullptr;
  double* wle = nullptr;
  double* wsum = nullptr;
  double* err = nullptr;
  unsigned long long* rmin = nullptr;
  unsigned long long* rmax = nullptr;
  int* cnt = nullptr;
  int* done = nullptr;
  int* flags = nullptr;        // [0] label >= K seen, [1] components still bisecting
  double* made = nullptr;      // result
};

void free_made(ni_handle* h) {
  MadeScratch* m = h->made;
  if (!m) return;
  void* ps[] = {m->key, m->r, m->w, m->lo, m->hi, m->wle, m->wsum, m->err, m->rmin, m->rmax,
                m->cnt, m->done, m->flags, m->made};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete m;
  h->made = nullptr;
}

static cudaError_t made_capacity(ni_handle* h, long long n, int K) {
  if (!h->made) h->made = new MadeScratch();
  MadeScratch* m = h->made;
  cudaError_t e = cudaSuccess;
  if (n > m->ncap) {
    cudaFree(m->key); cudaFree(m->r); cudaFree(m->w);
    m->key = nullptr; m->r = nullptr; m->w = nullptr; m->ncap = 0;
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->key, n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->r, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->w, n * sizeof(double));
    if (e != cudaSuccess) return e;
    m->ncap = n;
  }
  if (K > m->kcap) {
    double** ds[] = {&m->lo, &m->hi, &m->wle, &m->wsum, &m->err};
    for (double** p : ds) { cudaFree(*p); *p = nullptr; }
    cudaFree(m->rmin); cudaFree(m->rmax); cudaFree(m->cnt); cudaFree(m->done);
    m->rmin = m->rmax = nullptr; m->cnt = m->done = nullptr; m->kcap = 0;
    for (double** p : ds)
      if (e == cudaSuccess) e = cudaMalloc((void**)p, (size_t)K * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->rmin, (size_t)K * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->rmax, (size_t)K * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->cnt, (size_t)K * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->done, (size_t)K * sizeof(int));
    if (e != cudaSuccess) return e;
    m->kcap = K;
  }
  if (!m->flags) e = cudaMalloc((void**)&m->flags, 2 * sizeof(int));
  if (e == cudaSuccess && !m->made) e = cudaMalloc((void**)&m->made, sizeof(double));
  return e;
}

// order-preserving map of doubles to unsigned keys (for atomicMin / atomicMax)
__device__ __forceinline__ unsigned long long ord_key(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_val(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// The warp's lanes with key >= 0 all share one key k0 (k0 = -1: no lane has one).
__device__ __forceinline__ bool warp_one_key(int key, int& k0) {
  const unsigned vm = __ballot_sync(NI_FULL, key >= 0);
  k0 = vm ? __shfl_sync(NI_FULL, key, __ffs(vm) - 1) : -1;
  return __all_sync(NI_FULL, key < 0 || key == k0);
}

// add v of every lane with key >= 0 to dst[key]; all 32 lanes call
__device__ __forceinline__ void warp_add_d(double* dst, int key, double v) {
  int k0;
  if (warp_one_key(key, k0)) {
    if (k0 < 0) return;
    const double t = warp_sum_d(key >= 0 ? v : 0.0);
    if ((threadIdx.x & 31) == 0 && t != 0.0) atomicAdd(dst + k0, t);
  } else if (key >= 0 && v != 0.0) {
    atomicAdd(dst + key, v);
  }
}

__device__ __forceinline__ double depth_of(float z, int z_is_log, int persp) {
  return (persp && z_is_log) ? exp((double)z) : (double)z;
}

struct MadeArgs {
  const float* z;
  const int32_t* labels;   // NULL: one component
  const float* gt;
  long long N;
  int K;
  int persp;
  int z_is_log;
  MadeScratch m;
};

// ratios, weights, per-component weight sums, counts and ratio range
__global__ void k_made_prep(MadeArgs A) {
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < A.N; i0 += stride) {
    const long long i = i0 + lane;
    int key = -1;
    double r = 0.0, w = 0.0;
    if (i < A.N) {
      int c = A.labels ? A.labels[i] : 0;
      if (c >= A.K) {          // out of range: flagged for the host, never used as an index
        atomicOr(A.m.flags, 1);
        c = -1;
      }
      if (c >= 0) {
        const double d = depth_of(A.z[i], A.z_is_log, A.persp), g = (double)A.gt[i];
        bool ok = isfinite(d) && isfinite(g);
        if (A.persp) ok = ok && d > 0.0 && g > 0.0;
        if (ok) {
          key = c;
          r = A.persp ? g / d : g - d;
          w = A.persp ? d : 1.0;
        }
      }
      A.m.key[i] = key;
      A.m.r[i] = r;
      A.m.w[i] = w;
    }
    int k0;
    if (warp_one_key(key, k0)) {
      if (k0 < 0) continue;
      const bool on = key >= 0;
      const double ws = warp_sum_d(on ? w : 0.0);
      const int n = __popc(__ballot_sync(NI_FULL, on));
      unsigned long long mn = on ? ord_key(r) : ~0ull, mx = on ? ord_key(r) : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(NI_FULL, mn, o));
        mx = max(mx, __shfl_xor_sync(NI_FULL, mx, o));
      }
      if (lane == 0) {
        atomicAdd(A.m.wsum + k0, ws);
        atomicAdd(A.m.cnt + k0, n);
        atomicMin(A.m.rmin + k0, mn);
        atomicMax(A.m.rmax + k0, mx);
      }
    } else if (key >= 0) {
      atomicAdd(A.m.wsum + key, w);
      atomicAdd(A.m.cnt + key, 1);
      atomicMin(A.m.rmin + key, ord_key(r));
      atomicMax(A.m.rmax + key, ord_key(r));
    }
  }
}

// initial brackets: W_le(lo) = 0 < W_c / 2 and W_le(hi) = W_c
__global__ void k_made_bracket(MadeArgs A) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < A.K; c += gridDim.x * blockDim.x) {
    A.m.wle[c] = 0.0;
    A.m.err[c] = 0.0;
    if (A.m.cnt[c] == 0) {
      A.m.done[c] = 1;
      A.m.lo[c] = A.m.hi[c] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    const double rmin = ord_val(A.m.rmin[c]), rmax = ord_val(A.m.rmax[c]);
    A.m.done[c] = 0;
    A.m.lo[c] = A.persp ? 0.0 : rmin - fmax(1.0, fabs(rmin));
    A.m.hi[c] = rmax;
  }
}

__global__ void k_made_count(MadeArgs A) {
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < A.N; i0 += stride) {
    const long long i = i0 + lane;
    int key = i < A.N ? A.m.key[i] : -1;
    double v = 0.0;
    if (key >= 0) {
      if (A.m.done[key]) {
        key = -1;
      } else {
        const double mid = 0.5 * (A.m.lo[key] + A.m.hi[key]);
        v = A.m.r[i] <= mid ? A.m.w[i] : 0.0;
      }
    }
    warp_add_d(A.m.wle, key, v);
  }
}

__global__ void k_made_step(MadeArgs A) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < A.K; c += gridDim.x * blockDim.x) {
    if (A.m.done[c]) continue;
    const double lo = A.m.lo[c], hi = A.m.hi[c], mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) {
      A.m.done[c] = 1;      // no double between lo and hi: hi is the breakpoint
    } else {
      if (A.m.wle[c] >= 0.5 * A.m.wsum[c]) A.m.hi[c] = mid;
      else A.m.lo[c] = mid;
      atomicAdd(A.m.flags + 1, 1);
    }
    A.m.wle[c] = 0.0;
  }
}

__global__ void k_made_err(MadeArgs A) {
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < A.N; i0 += stride) {
    const long long i = i0 + lane;
    const int key = i < A.N ? A.m.key[i] : -1;
    double e = 0.0;
    if (key >= 0) {
      const double s = A.m.hi[key], d = depth_of(A.z[i], A.z_is_log, A.persp), g = (double)A.gt[i];
      e = A.persp ? fabs(s * d - g) : fabs(d + s - g);
    }
    warp_add_d(A.m.err, key, e);
  }
}

// MADE = sum_c E_c / sum_c n_c (one CTA); per-component outputs
__global__ void __launch_bounds__(1024) k_made_final(MadeArgs A, double* comp_made, double* comp_scale) {
  __shared__ double sh[33];
  __shared__ int shi[33];
  double e = 0.0;
  int n = 0;
  for (int c = threadIdx.x; c < A.K; c += blockDim.x) {
    const int nc = A.m.cnt[c];
    e += A.m.err[c];
    n += nc;
    if (comp_made) comp_made[c] = nc > 0 ? A.m.err[c] / nc : 0.0;
    if (comp_scale) comp_scale[c] = A.m.hi[c];
  }
  e = block_sum_d(e, sh);
  n = block_sum_i(n, shi);
  if (threadIdx.x == 0) *A.m.made = n > 0 ? e / n : __longlong_as_double(0x7ff8000000000000LL);
}

extern "C" ni_status ni_min_made(ni_handle* h, const float* z, int z_is_log, const int32_t* labels, int32_t K,
                                 const float* depth_gt, double* made_out, double* comp_made_out,
                                 double* comp_scale_out, ni_stream_t stream) {
  if (!h) return NI_ERR_INVALID_ARG;
  if (!z || !depth_gt || !made_out) return ni_fail(h, NI_ERR_INVALID_ARG, "z, depth_gt and made_out are required");
  if (!labels) K = 1;
  if (K < 1 || (long long)K > (long long)h->N)
    return ni_fail(h, NI_ERR_INVALID_ARG, "K must be in [1, H * W]");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = made_capacity(h, h->N, K);
  if (e != cudaSuccess) {
    free_made(h);
    return ni_cuda_check(h, e, "min MADE scratch");
  }
  MadeArgs A;
  A.z = z; A.labels = labels; A.gt = depth_gt; A.N = h->N; A.K = K;
  A.persp = h->persp; A.z_is_log = z_is_log ? 1 : 0; A.m = *h->made;
  cudaMemsetAsync(A.m.wsum, 0, (size_t)K * sizeof(double), s);
  cudaMemsetAsync(A.m.cnt, 0, (size_t)K * sizeof(int), s);
  cudaMemsetAsync(A.m.rmin, 0xff, (size_t)K * sizeof(unsigned long long), s);
  cudaMemsetAsync(A.m.rmax, 0, (size_t)K * sizeof(unsigned long long), s);
  cudaMemsetAsync(A.m.flags, 0, 2 * sizeof(int), s);
  const int gp = std::max(1, std::min((int)((h->N + 255) / 256), h->num_sms * 8));
  const int gk = std::max(1, std::min((K + 255) / 256, h->num_sms * 4));
  k_made_prep<<<gp, 256, 0, s>>>(A); NI_COUNT(h);
  k_made_bracket<<<gk, 256, 0, s>>>(A); NI_COUNT(h);
  int flags[2] = {0, 0};
  for (int pass = 0; pass < NI_MADE_MAX_PASSES; pass += NI_MADE_CHUNK) {
    cudaMemsetAsync(A.m.flags + 1, 0, sizeof(int), s);
    for (int j = 0; j < NI_MADE_CHUNK; ++j) {
      k_made_count<<<gp, 256, 0, s>>>(A); NI_COUNT(h);
      k_made_step<<<gk, 256, 0, s>>>(A); NI_COUNT(h);
    }
    e = cudaMemcpyAsync(flags, A.m.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ni_cuda_check(h, e, "min MADE bisection");
    if (flags[0]) return ni_fail(h, NI_ERR_INVALID_ARG, "a label is >= K");
    if (flags[1] == 0) break;   // every bracket has closed
  }
  k_made_err<<<gp, 256, 0, s>>>(A); NI_COUNT(h);
  k_made_final<<<1, 1024, 0, s>>>(A, comp_made_out, comp_scale_out); NI_COUNT(h);
  e = cudaMemcpyAsync(made_out, A.m.made, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return ni_cuda_check(h, e, "min MADE");
}
