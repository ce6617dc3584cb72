// Tile-group helpers shared by the fill PCG kernels: a CTA of 256 threads works on
// a 32x32-pixel tile, each thread on 4 consecutive pixels of one tile row; per-
// component sums of a tile are reduced in warps (optionally compensated) and added
// to FP64 accumulators with one atomic per CTA and label.
#pragma once
#include "ni_internal.cuh"

struct G4 {
  int a;     // raster index of the first pixel
  int row, col;
  int nval;  // pixels of the group inside the image (0..4)
};

__device__ __forceinline__ G4 group_of(int t, int ntx, int H, int W) {
  G4 g;
  g.row = (t / ntx) * NI_TILE_H + (threadIdx.x >> 3);
  g.col = (t % ntx) * NI_TILE_W + ((threadIdx.x & 7) << 2);
  g.nval = g.row < H ? max(0, min(4, W - g.col)) : 0;
  g.a = g.row * W + g.col;
  return g;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float f4get(const float4& v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}
__device__ __forceinline__ void f4set(float4& v, int j, float s) {
  if (j == 0) v.x = s; else if (j == 1) v.y = s; else if (j == 2) v.z = s; else v.w = s;
}

// the 4 values of a group at raster index a (nval of them inside the image)
template <bool ALIGNED>
__device__ __forceinline__ float4 ldg(const float* p, int a, int nval) {
  if (ALIGNED && nval == 4) return ld4(p + a);
  return make_float4(nval > 0 ? p[a] : 0.f, nval > 1 ? p[a + 1] : 0.f, nval > 2 ? p[a + 2] : 0.f,
                     nval > 3 ? p[a + 3] : 0.f);
}
template <bool ALIGNED>
__device__ __forceinline__ void stg(float* p, int a, int nval, float4 v) {
  if (ALIGNED && nval == 4) { st4(p + a, v); return; }
  if (nval > 0) p[a] = v.x;
  if (nval > 1) p[a + 1] = v.y;
  if (nval > 2) p[a + 2] = v.z;
  if (nval > 3) p[a + 3] = v.w;
}
template <bool ALIGNED>
__device__ __forceinline__ void ldlab(const int* l, int a, int nval, int (&lab)[4]) {
  if (ALIGNED && nval == 4) {
    const int4 v = *reinterpret_cast<const int4*>(l + a);
    lab[0] = v.x; lab[1] = v.y; lab[2] = v.z; lab[3] = v.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) lab[j] = j < nval ? l[a + j] : -1;
  }
}

#define TAB_SLOTS 64

// Two-sum of float pairs (Knuth): hi + lo carries ~48 bits, the "compensated
// FP32" reduction (no FP64 instructions per pixel).
__device__ __forceinline__ void ff_add(float& hi, float& lo, float h2, float l2) {
  const float s = hi + h2;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (h2 - bp);
  lo = lo + l2 + e;
  hi = s;
}

// Warp total as a float pair (hi, lo); lo = 0 without compensation.  Callers
// convert to double only in the lane that uses the result.
template <bool COMP>
__device__ __forceinline__ float2 warp_total(float v) {
  if (COMP) {
    float hi = v, lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ff_add(hi, lo, __shfl_xor_sync(NI_FULL, hi, o), __shfl_xor_sync(NI_FULL, lo, o));
    return make_float2(hi, lo);
  }
  return make_float2(warp_sum_f(v), 0.f);
}

// Add `t` to the CTA's shared table entry of label `key` (linear probing over
// TAB_SLOTS slots); straight to dst[j] + key when the table is full.
template <int NV>
__device__ __forceinline__ void table_add(int key, int j, double t, double* const (&dst)[NV], int* s_key,
                                          double* s_val) {
  int h = key & (TAB_SLOTS - 1), slot = -1;
  for (int probe = 0; probe < TAB_SLOTS; ++probe) {
    const int old = atomicCAS(&s_key[h], -1, key);
    if (old == -1 || old == key) { slot = h; break; }
    h = (h + 1) & (TAB_SLOTS - 1);
  }
  if (slot >= 0) atomicAdd(&s_val[slot * 3 + j], t);
  else atomicAdd(dst[j] + key, t);
}

// Add NV per-thread values into dst[v][label].  `key` is the label all of the
// thread's contributing pixels share (-1: nothing to add; threads with pixels of
// several labels add per pixel before calling, and pass -1).  ul >= 0: the whole
// tile is one component.  Warp trees in float (float-float when COMP), the
// per-warp totals in double.  All threads of the CTA call it.
// par = 0 or 1 (the parity of the caller's tile step; 16 * NV doubles of sh):
// a one-label tile's warp totals go to half `par` of sh, so the next tile, which
// writes the other half, needs no second CTA barrier to wait for the adding
// thread; par = -1: one half and two barriers.
template <bool COMP, int NV>
__device__ __forceinline__ void tile_accum(int ul, int key, const float (&v)[NV], double* const (&dst)[NV],
                                           int* s_key, double* s_val, double* sh, int par = -1) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (ul >= 0) {
    float2 w[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) w[j] = warp_total<COMP>(v[j]);
    if (par > 0) sh += 8 * NV;
    if (lane == 0)
#pragma unroll
      for (int j = 0; j < NV; ++j) sh[wid * NV + j] = (double)w[j].x + (double)w[j].y;
    __syncthreads();
    if (threadIdx.x < NV) {   // pairwise over the (at most 8) warps: 3 dependent FP64 adds, not 7
      const int nw = (int)(blockDim.x >> 5);
      double u[8];
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) u[ww] = ww < nw ? sh[ww * NV + threadIdx.x] : 0.0;
      const double t = ((u[0] + u[1]) + (u[2] + u[3])) + ((u[4] + u[5]) + (u[6] + u[7]));
      if (t != 0.0) atomicAdd(dst[threadIdx.x] + ul, t);
    }
    if (par < 0) __syncthreads();
    return;
  }
  // warp-segmented runs of equal keys
  const int prev = __shfl_up_sync(NI_FULL, key, 1);
  const int next = __shfl_down_sync(NI_FULL, key, 1);
  const bool head = (lane == 0) || (prev != key);
  const bool tail = (lane == 31) || (next != key);
  const unsigned heads = __ballot_sync(NI_FULL, head);
  const int my_head = 31 - __clz(heads & ((2u << lane) - 1u));
  float2 acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    float hi = v[j], lo = 0.f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float h2 = __shfl_up_sync(NI_FULL, hi, o);
      const float l2 = COMP ? __shfl_up_sync(NI_FULL, lo, o) : 0.f;
      if (lane - o >= my_head) {
        if (COMP) ff_add(hi, lo, h2, l2);
        else hi += h2;
      }
    }
    acc[j] = make_float2(hi, lo);
  }
  if (tail && key >= 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      const double t = (double)acc[j].x + (double)acc[j].y;
      if (t != 0.0) table_add<NV>(key, j, t, dst, s_key, s_val);
    }
  }
  __syncthreads();
  if (threadIdx.x < TAB_SLOTS) {
    const int k = s_key[threadIdx.x];
    if (k >= 0) {
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const double t = s_val[threadIdx.x * 3 + j];
        if (t != 0.0) atomicAdd(dst[j] + k, t);
        s_val[threadIdx.x * 3 + j] = 0.0;
      }
      s_key[threadIdx.x] = -1;
    }
  }
  __syncthreads();
}

// Per-tile cache of per-component scalars: each distinct label of the tile gets a
// shared-memory slot; slot owners compute the label's scalars once (FP64), the
// pixels read floats.  sl[j] = slot of pixel j, -1 for no label, -2 if the table
// overflowed (the pixel then computes its own scalars).
__device__ __forceinline__ void tile_slots(int ul, const int (&lab)[4], int (&sl)[4], int* s_lab) {
  if (ul >= 0) {
    if (threadIdx.x == 0) s_lab[0] = ul;
    for (int i = 1 + threadIdx.x; i < TAB_SLOTS; i += blockDim.x) s_lab[i] = -1;
#pragma unroll
    for (int j = 0; j < 4; ++j) sl[j] = lab[j] >= 0 ? 0 : -1;
    __syncthreads();
    return;
  }
  if (threadIdx.x < TAB_SLOTS) s_lab[threadIdx.x] = -1;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    sl[j] = -1;
    if (lab[j] < 0) continue;
    if (j > 0 && lab[j] == lab[j - 1]) { sl[j] = sl[j - 1]; continue; }
    int h = lab[j] & (TAB_SLOTS - 1);
    sl[j] = -2;
    for (int probe = 0; probe < TAB_SLOTS; ++probe) {
      const int old = atomicCAS(&s_lab[h], -1, lab[j]);
      if (old == -1 || old == lab[j]) { sl[j] = h; break; }
      h = (h + 1) & (TAB_SLOTS - 1);
    }
  }
  __syncthreads();
}

// key of a thread's contributing pixels (-1 none, -2 several labels)
__device__ __forceinline__ int group_key(const int (&lab)[4], const bool (&on)[4]) {
  int key = -1;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (on[j]) key = (key == -1 || key == lab[j]) ? lab[j] : -2;
  return key;
}

template <int NV>
__device__ __forceinline__ void group_values(int key, const int (&lab)[4], const bool (&on)[4],
                                             const float (&pv)[NV][4], double* const (&dst)[NV],
                                             float (&v)[NV]) {
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.f;
  if (key >= 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) v[i] += on[j] ? pv[i][j] : 0.f;
  } else if (key == -2) {   // pixels of several labels: add them one by one
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (on[j])
#pragma unroll
        for (int i = 0; i < NV; ++i)
          if (pv[i][j] != 0.f) atomicAdd(dst[i] + lab[j], (double)pv[i][j]);
  }
}
