// Learned warm start (not in the paper; an extension beyond it): a 6-layer
// 3x3 convolutional network trained and run with BF16 tensor-core kernels.
//
// The forward and dgrad convolutions are implicit GEMMs on the tcgen05 tensor
// cores with the accumulator in tensor memory (ni_cnn_tc.cu):
//   forward  out = relu(conv_valid(in, W) + b)            (layers 1-5), linear (6)
//   dgrad    g_{l-1} = conv_valid(pad2(g_l), flip(W)^T) * [act_{l-1} > 0]
// The weight gradient, a GEMM whose reduction runs over the pixels, stays on
// mma.sync.m16n8k16 (BF16 inputs, FP32 accumulation):
//   wgrad    dW[tap] (cout x cin) = sum_px g[px] act[px + tap]^T  (K = pixels)
// Channel counts are padded for the 16-wide K steps: the 4 input channels to 16,
// the 5 output channels to 8 (forward) and 16 (gradient of the last layer).
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/ni_cnn.h"
#include "ni_internal.cuh"

typedef __nv_bfloat16 bf16;

// ni_cnn_tc.cu
cudaError_t conv3x3_tc(const bf16* in, int B, int Hi, int ci, int co, int wco, int mode, const bf16* w,
                       const float* bias, int nbias, void* out, const bf16* act_mask, int* err, int num_sms,
                       cudaStream_t s);

namespace {

constexpr int NL = 6;
constexpr int CIN[NL] = {4, 32, 32, 32, 32, 32};
constexpr int COUT[NL] = {32, 32, 32, 32, 32, 5};
constexpr int CINP[NL] = {16, 32, 32, 32, 32, 32};    // padded input channels (kernel layout)
constexpr int COUTP[NL] = {32, 32, 32, 32, 32, 8};    // padded output channels
constexpr int HALO = 6;

constexpr int w_size(int l) { return 9 * CIN[l] * COUT[l]; }
constexpr int layer_params(int l) { return w_size(l) + COUT[l]; }
int param_offset(int l) {
  int o = 0;
  for (int i = 0; i < l; ++i) o += layer_params(i);
  return o;
}
int num_params() { return param_offset(NL); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t pack_raw(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}


// ---------------------------------------------------------------------------
// weight gradient: dW[tap][co][ci] += sum over output pixels of g[px][co] * act[px + tap][ci]
// g: [B][Ho][Wo][GC] bf16 (GC >= CO rows used: M tiles of 16), act: [B][Ho+2][Wo+2][CI]
// One CTA per (pixel chunk, tap); the partial tile is reduced in shared memory and
// added to the FP32 gradient in the parameter layout W[dy][dx][ci][co].
// ---------------------------------------------------------------------------
template <int CI, int GC, int CO_REAL, int CI_REAL>
__global__ void __launch_bounds__(128) k_wgrad(const bf16* __restrict__ gr, const bf16* __restrict__ act, int B,
                                                int Ho, int Wo, float* __restrict__ dW) {
  constexpr int MT = GC / 16, NT = CI / 8;
  __shared__ float red[MT * 16 * CI];
  const int tap = blockIdx.y, dy = tap / 3, dx = tap % 3;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int Wi = Wo + 2, Hi = Ho + 2;
  for (int i = threadIdx.x; i < MT * 16 * CI; i += blockDim.x) red[i] = 0.f;
  __syncthreads();
  float acc[MT][NT][4];
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[m][j][0] = acc[m][j][1] = acc[m][j][2] = acc[m][j][3] = 0.f;
  const int nseg = (Wo + 15) / 16;
  const long long items = (long long)B * Ho * nseg;
  const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long it = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < items; it += wstride) {
    const int seg = (int)(it % nseg);
    const long long ny = it / nseg;
    const int y = (int)(ny % Ho), n = (int)(ny / Ho);
    const int x0 = seg * 16;
    // k index = pixel x0 + k of row y; A[m = co][k], B[k][n = ci]
    const int k0 = 2 * t, k1 = 2 * t + 1, k2 = 2 * t + 8, k3 = 2 * t + 9;
    const bool ok0 = x0 + k0 < Wo, ok1 = x0 + k1 < Wo, ok2 = x0 + k2 < Wo, ok3 = x0 + k3 < Wo;
    const bf16* grow = gr + (((long long)n * Ho + y) * Wo + x0) * GC;
    const bf16* arow = act + (((long long)n * Hi + y + dy) * Wi + x0 + dx) * CI;
    const bf16 z = __float2bfloat16(0.f);
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      const int co = m * 16 + g;
      const uint32_t a0 = pack_raw(ok0 ? grow[(long long)k0 * GC + co] : z, ok1 ? grow[(long long)k1 * GC + co] : z);
      const uint32_t a1 = pack_raw(ok0 ? grow[(long long)k0 * GC + co + 8] : z, ok1 ? grow[(long long)k1 * GC + co + 8] : z);
      const uint32_t a2 = pack_raw(ok2 ? grow[(long long)k2 * GC + co] : z, ok3 ? grow[(long long)k3 * GC + co] : z);
      const uint32_t a3 = pack_raw(ok2 ? grow[(long long)k2 * GC + co + 8] : z, ok3 ? grow[(long long)k3 * GC + co + 8] : z);
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int ci = j * 8 + g;
        const uint32_t b0 = pack_raw(ok0 ? arow[(long long)k0 * CI + ci] : z, ok1 ? arow[(long long)k1 * CI + ci] : z);
        const uint32_t b1 = pack_raw(ok2 ? arow[(long long)k2 * CI + ci] : z, ok3 ? arow[(long long)k3 * CI + ci] : z);
        mma_bf16(acc[m][j], a0, a1, a2, a3, b0, b1);
      }
    }
  }
  // accumulate the warps' tiles in shared memory: C row = co, column = ci
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int co = m * 16 + g, ci = j * 8 + 2 * t;
      atomicAdd(&red[co * CI + ci], acc[m][j][0]);
      atomicAdd(&red[co * CI + ci + 1], acc[m][j][1]);
      atomicAdd(&red[(co + 8) * CI + ci], acc[m][j][2]);
      atomicAdd(&red[(co + 8) * CI + ci + 1], acc[m][j][3]);
    }
  __syncthreads();
  for (int i = threadIdx.x; i < CO_REAL * CI_REAL; i += blockDim.x) {
    const int co = i % CO_REAL, ci = i / CO_REAL;
    const float v = red[co * CI + ci];
    if (v != 0.f) atomicAdd(&dW[((long long)tap * CI_REAL + ci) * CO_REAL + co], v);
  }
}

template <int GC, int CO_REAL>
__global__ void k_bias_grad(const bf16* __restrict__ gr, long long npx, float* __restrict__ db) {
  __shared__ float s[CO_REAL];
  for (int i = threadIdx.x; i < CO_REAL; i += blockDim.x) s[i] = 0.f;
  __syncthreads();
  float acc[CO_REAL];
#pragma unroll
  for (int c = 0; c < CO_REAL; ++c) acc[c] = 0.f;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < CO_REAL; ++c) acc[c] += __bfloat162float(gr[p * GC + c]);
#pragma unroll
  for (int c = 0; c < CO_REAL; ++c) {
    float v = warp_sum_f(acc[c]);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s[c], v);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < CO_REAL; i += blockDim.x) atomicAdd(&db[i], s[i]);
}

// ---------------------------------------------------------------------------
// input packing, padding, loss
// ---------------------------------------------------------------------------
__global__ void k_pack_input(const float* __restrict__ in, long long npx, bf16* __restrict__ out) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += (long long)gridDim.x * blockDim.x) {
    const float4 v = reinterpret_cast<const float4*>(in)[p];
    uint32_t* o = reinterpret_cast<uint32_t*>(out + p * 16);
    o[0] = pack_bf16(v.x, v.y);
    o[1] = pack_bf16(v.z, v.w);
#pragma unroll
    for (int i = 2; i < 8; ++i) o[i] = 0u;
  }
}

// dst [B][H+4][W+4][C] = src [B][H][W][C] with a zero border of 2 (C even)
__global__ void k_pad2(const bf16* __restrict__ src, int B, int H, int W, int C, bf16* __restrict__ dst) {
  const int Hp = H + 4, Wp = W + 4, C2 = C / 2;
  const long long total = (long long)B * Hp * Wp * C2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int c2 = (int)(i % C2);
    long long r = i / C2;
    const int x = (int)(r % Wp);
    r /= Wp;
    const int y = (int)(r % Hp), n = (int)(r / Hp);
    uint32_t v = 0u;
    if (y >= 2 && y < H + 2 && x >= 2 && x < W + 2)
      v = reinterpret_cast<const uint32_t*>(src)[(((long long)n * H + y - 2) * W + x - 2) * C2 + c2];
    reinterpret_cast<uint32_t*>(dst)[i] = v;
  }
}

__device__ __forceinline__ float softplus(float x) { return x > 0.f ? x + log1pf(expf(-x)) : log1pf(expf(x)); }

// counts of depth edges and weight terms
__global__ void k_loss_count(const int* __restrict__ lab, int B, int T, unsigned long long* cnt) {
  unsigned long long nd = 0, nw = 0;
  const long long npx = (long long)B * T * T;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(p % T), y = (int)((p / T) % T);
    const int la = lab[p];
    if (la < 0) continue;
    if (x + 1 < T && lab[p + 1] == la) nd++;
    if (y + 1 < T && lab[p + T] == la) nd++;
    nw += (x + 1 < T && lab[p + 1] >= 0) + (y + 1 < T && lab[p + T] >= 0) + (x > 0 && lab[p - 1] >= 0) +
          (y > 0 && lab[p - T] >= 0);
  }
  for (int o = 16; o > 0; o >>= 1) {
    nd += __shfl_xor_sync(NI_FULL, nd, o);
    nw += __shfl_xor_sync(NI_FULL, nw, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&cnt[0], nd);
    atomicAdd(&cnt[1], nw);
  }
}

// loss sums (double) and d loss / d output (bf16, 16 channels: z, 4 logits, zeros)
__global__ void k_loss_grad(const float* __restrict__ pred, const float* __restrict__ tz, const int* __restrict__ lab,
                            const float* __restrict__ tw, int B, int T, float w_weight,
                            const unsigned long long* __restrict__ cnt, double* loss, bf16* __restrict__ g6) {
  const float inv_d = cnt[0] ? 1.f / (float)cnt[0] : 0.f;
  const float inv_w = cnt[1] ? 1.f / (float)cnt[1] : 0.f;
  double ld = 0.0, lw = 0.0;
  const long long npx = (long long)B * T * T;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(p % T), y = (int)((p / T) % T);
    const int la = lab[p];
    float g[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) g[c] = 0.f;
    if (la >= 0) {
      const float za = pred[p * 8], ta = tz[p];
      // depth: own right/down edges (loss) and all four edges (gradient)
      const long long nb[4] = {p + 1, p + T, p - 1, p - T};
      const bool has[4] = {x + 1 < T, y + 1 < T, x > 0, y > 0};
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        if (!has[d]) continue;
        const int lb = lab[nb[d]];
        if (lb == la) {
          const float dd = (za - pred[nb[d] * 8]) - (ta - tz[nb[d]]);
          g[0] += 2.f * dd * inv_d;
          if (d < 2) ld += (double)dd * dd;
        }
        if (lb >= 0) {   // weight logit of direction d
          const float lg = pred[p * 8 + 1 + d], wt = tw[p * 4 + d];
          lw += (double)(softplus(lg) - wt * lg);
          g[1 + d] = w_weight * inv_w * (1.f / (1.f + expf(-lg)) - wt);
        }
      }
    }
    uint32_t* o = reinterpret_cast<uint32_t*>(g6 + p * 16);
#pragma unroll
    for (int c = 0; c < 8; ++c) o[c] = pack_bf16(g[2 * c], g[2 * c + 1]);
  }
  ld = warp_sum_d(ld);
  lw = warp_sum_d(lw);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&loss[0], ld);
    atomicAdd(&loss[1], lw);
  }
}

// Adam on FP32 master parameters
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// FP32 parameters -> BF16 kernel layouts: forward wf[tap][co][ci] and dgrad
// wd[tap'][ci][co] = W[8 - tap'] (flipped), both zero-padded.
__global__ void k_repack(const float* __restrict__ W, int cin, int cout, int cinp, int coutp, bf16* __restrict__ wf,
                         int dg_ci_p, int dg_co_p, bf16* __restrict__ wdg) {
  const int nf = 9 * coutp * cinp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
    const int ci = i % cinp, co = (i / cinp) % coutp, tap = i / (cinp * coutp);
    const float v = (ci < cin && co < cout) ? W[((long long)tap * cin + ci) * cout + co] : 0.f;
    wf[i] = __float2bfloat16(v);
  }
  if (!wdg) return;
  // dgrad conv: output channel = ci of the layer (dg_co_p), input channel = co (dg_ci_p)
  const int nd = 9 * dg_co_p * dg_ci_p;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += gridDim.x * blockDim.x) {
    const int k = i % dg_ci_p, nn = (i / dg_ci_p) % dg_co_p, tap = i / (dg_ci_p * dg_co_p);
    const int src_tap = 8 - tap;
    const float v = (k < cout && nn < cin) ? W[((long long)src_tap * cin + nn) * cout + k] : 0.f;
    wdg[i] = __float2bfloat16(v);
  }
}

// BiNI edge-weight targets
__global__ void k_edge_targets(const float4* __restrict__ nrm, const uint8_t* __restrict__ mask,
                               const float* __restrict__ z, int H, int W, int persp, float fx, float fy, float cx,
                               float cy, float k, float* __restrict__ out) {
  const int N = H * W;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    const int u = a % W, v = a / W;
    float o[4] = {0.f, 0.f, 0.f, 0.f};
    if (mask[a]) {
      const float4 n = nrm[a];
      const float nt = persp ? n.x * (u - cx) / fx + n.y * (v - cy) / fy + n.z : n.z;
      const int du[4] = {1, 0, -1, 0}, dv[4] = {0, 1, 0, -1};
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        const int ub = u + du[d], vb = v + dv[d];
        if (ub < 0 || ub >= W || vb < 0 || vb >= H) continue;
        const int b = vb * W + ub;
        if (!mask[b]) continue;
        const float f = persp ? (d % 2 == 0 ? fx : fy) : 1.f;
        const float gm = f * nt, g2 = gm * gm;
        const int uo = u - du[d], vo = v - dv[d];
        float dop = 0.f;
        if (uo >= 0 && uo < W && vo >= 0 && vo < H && mask[vo * W + uo]) {
          const float e = z[vo * W + uo] - z[a];
          dop = e * e;
        }
        const float e2 = (z[b] - z[a]) * (z[b] - z[a]);
        o[d] = 1.f / (1.f + expf(-k * g2 * (dop - e2)));
      }
    }
    reinterpret_cast<float4*>(out)[a] = make_float4(o[0], o[1], o[2], o[3]);
  }
}

__global__ void k_make_tiles(const float4* __restrict__ nrm, const uint8_t* __restrict__ mask, int H, int W, int T,
                             int ntx, int nt, float4* __restrict__ out) {
  const int S = T + 2 * HALO;
  const long long total = (long long)nt * S * S;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % S), y = (int)((i / S) % S), t = (int)(i / ((long long)S * S));
    const int u = (t % ntx) * T + x - HALO, v = (t / ntx) * T + y - HALO;
    float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
    if (u >= 0 && u < W && v >= 0 && v < H) {
      const int a = v * W + u;
      if (mask[a]) {
        val = nrm[a];
        val.w = 1.f;
      }
    }
    out[i] = val;
  }
}

int grid_of(long long n, int threads, int cap = 4096) {
  long long b = (n + threads - 1) / threads;
  return (int)std::max(1LL, std::min(b, (long long)cap));
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

}  // namespace

struct ni_cnn {
  int maxB = 0, T = 0, S = 0;
  int np = 0;
  float* p = nullptr;   // FP32 master parameters
  float* g = nullptr;   // gradients
  float* m = nullptr;
  float* v = nullptr;
  bf16* wf[NL] = {};    // forward weights
  bf16* wdg[NL] = {};   // dgrad weights (layers 2..6)
  bf16* act[NL] = {};   // act[0] packed input; act[l] output of layer l (1..5)
  float* out = nullptr; // layer-6 output [B][T][T][8]
  bf16* gbuf[2] = {};   // gradient activations (ping-pong)
  bf16* pad = nullptr;  // padded gradient
  unsigned long long* cnt = nullptr;
  double* loss = nullptr;
  int* err = nullptr;   // NI_DEV_ERR_* bits of the tensor-core kernels
  int num_sms = 1;
  long long step = 0;
};

static int side(const ni_cnn* n, int l) { return n->S - 2 * l; }   // spatial side of act[l]

extern "C" int ni_cnn_num_params(void) { return num_params(); }

template <class T>
static cudaError_t alloc(T** p, size_t n) {
  return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
}

static void repack(ni_cnn* net, cudaStream_t s) {
  for (int l = 0; l < NL; ++l) {
    const int off = param_offset(l);
    // dgrad of layer l maps COUTP-ish gradient (16 for the last layer) to CINP
    const int dg_ci = (l == NL - 1) ? 16 : COUTP[l];
    k_repack<<<64, 256, 0, s>>>(net->p + off, CIN[l], COUT[l], CINP[l], COUTP[l], net->wf[l], dg_ci, CINP[l],
                                 l > 0 ? net->wdg[l] : nullptr);
  }
}

extern "C" ni_status ni_cnn_create(int max_batch, int tile, uint64_t seed, ni_cnn** out) {
  if (!out) return NI_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_batch < 1 || tile < 16 || tile % 16) return NI_ERR_INVALID_ARG;
  ni_cnn* net = new ni_cnn();
  net->maxB = max_batch;
  net->T = tile;
  net->S = tile + 2 * HALO;
  net->np = num_params();
  cudaError_t e = cudaSuccess;
  const size_t np = net->np;
  if (e == cudaSuccess) e = alloc(&net->p, np);
  if (e == cudaSuccess) e = alloc(&net->g, np);
  if (e == cudaSuccess) e = alloc(&net->m, np);
  if (e == cudaSuccess) e = alloc(&net->v, np);
  for (int l = 0; l < NL && e == cudaSuccess; ++l) {
    e = alloc(&net->wf[l], (size_t)9 * COUTP[l] * CINP[l]);
    if (e == cudaSuccess && l > 0) e = alloc(&net->wdg[l], (size_t)9 * CINP[l] * (l == NL - 1 ? 16 : COUTP[l]));
    const size_t sd = (size_t)side(net, l);
    if (e == cudaSuccess) e = alloc(&net->act[l], (size_t)max_batch * sd * sd * (l == 0 ? 16 : 32));
  }
  const size_t T = (size_t)tile, S = (size_t)net->S;
  if (e == cudaSuccess) e = alloc(&net->out, (size_t)max_batch * T * T * 8);
  if (e == cudaSuccess) e = alloc(&net->gbuf[0], (size_t)max_batch * S * S * 32);
  if (e == cudaSuccess) e = alloc(&net->gbuf[1], (size_t)max_batch * S * S * 32);
  if (e == cudaSuccess) e = alloc(&net->pad, (size_t)max_batch * (S + 4) * (S + 4) * 32);
  if (e == cudaSuccess) e = alloc(&net->cnt, 2);
  if (e == cudaSuccess) e = alloc(&net->loss, 2);
  if (e == cudaSuccess) e = alloc(&net->err, 1);
  if (e == cudaSuccess) e = cudaMemset(net->err, 0, sizeof(int));
  if (e == cudaSuccess) {
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&net->num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (e != cudaSuccess) {
    ni_cnn_destroy(net);
    return e == cudaErrorMemoryAllocation ? NI_ERR_OOM : NI_ERR_CUDA;
  }
  // He-normal initial weights from a counter-based generator (splitmix64 +
  // Box-Muller), zero biases
  std::vector<float> h(np, 0.f);
  uint64_t st = seed * 0x2545f4914f6cdd1dull + 1;
  for (int l = 0; l < NL; ++l) {
    const int off = param_offset(l);
    const float sd = sqrtf(2.f / (9.f * CIN[l]));
    for (int i = 0; i < w_size(l); ++i) {
      const double u1 = ((splitmix(st) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
      const double u2 = (splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
      h[off + i] = (float)(sd * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
    }
  }
  ni_status rc = ni_cnn_set_params(net, h.data());
  if (rc != NI_OK) {
    ni_cnn_destroy(net);
    return rc;
  }
  *out = net;
  return NI_OK;
}

extern "C" ni_status ni_cnn_destroy(ni_cnn* net) {
  if (!net) return NI_OK;
  cudaFree(net->p); cudaFree(net->g); cudaFree(net->m); cudaFree(net->v);
  for (int l = 0; l < NL; ++l) { cudaFree(net->wf[l]); cudaFree(net->wdg[l]); cudaFree(net->act[l]); }
  cudaFree(net->out); cudaFree(net->gbuf[0]); cudaFree(net->gbuf[1]); cudaFree(net->pad);
  cudaFree(net->cnt); cudaFree(net->loss); cudaFree(net->err);
  delete net;
  return NI_OK;
}

extern "C" ni_status ni_cnn_get_params(ni_cnn* net, float* host) {
  if (!net || !host) return NI_ERR_INVALID_ARG;
  return cudaMemcpy(host, net->p, sizeof(float) * net->np, cudaMemcpyDeviceToHost) == cudaSuccess ? NI_OK
                                                                                                  : NI_ERR_CUDA;
}

extern "C" ni_status ni_cnn_set_params(ni_cnn* net, const float* host) {
  if (!net || !host) return NI_ERR_INVALID_ARG;
  if (cudaMemcpy(net->p, host, sizeof(float) * net->np, cudaMemcpyHostToDevice) != cudaSuccess) return NI_ERR_CUDA;
  cudaMemset(net->m, 0, sizeof(float) * net->np);
  cudaMemset(net->v, 0, sizeof(float) * net->np);
  net->step = 0;
  repack(net, 0);
  return cudaDeviceSynchronize() == cudaSuccess ? NI_OK : NI_ERR_CUDA;
}

static void forward(ni_cnn* net, const float* in, int B, cudaStream_t s) {
  const long long npx0 = (long long)B * net->S * net->S;
  k_pack_input<<<grid_of(npx0, 256), 256, 0, s>>>(in, npx0, net->act[0]);
  for (int l = 0; l < NL; ++l) {
    const int Hi = side(net, l);
    const float* bias = net->p + param_offset(l) + w_size(l);
    if (l < NL - 1)
      conv3x3_tc(net->act[l], B, Hi, CINP[l], 32, 32, 0, net->wf[l], bias, COUT[l], net->act[l + 1], nullptr,
                 net->err, net->num_sms, s);
    else   // the 8 stored output channels padded to 16 for the MMA's N
      conv3x3_tc(net->act[l], B, Hi, 32, 16, 8, 1, net->wf[l], bias, COUT[l], net->out, nullptr, net->err,
                 net->num_sms, s);
  }
}

extern "C" ni_status ni_cnn_forward(ni_cnn* net, const float* in, int B, float* out, ni_stream_t stream) {
  if (!net || !in || !out || B < 1 || B > net->maxB) return NI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  forward(net, in, B, s);
  // copy channels 0..4 of the padded 8-channel output
  const size_t T = net->T;
  cudaMemcpy2DAsync(out, 5 * sizeof(float), net->out, 8 * sizeof(float), 5 * sizeof(float), (size_t)B * T * T,
                    cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError() == cudaSuccess ? NI_OK : NI_ERR_CUDA;
}

static ni_status backward(ni_cnn* net, const float* in, const float* tz, const int32_t* tl, const float* tw, int B,
                          float w_weight, double* loss_host, cudaStream_t s) {
  forward(net, in, B, s);
  const int T = net->T;
  const long long npx = (long long)B * T * T;
  cudaMemsetAsync(net->cnt, 0, 2 * sizeof(unsigned long long), s);
  cudaMemsetAsync(net->loss, 0, 2 * sizeof(double), s);
  cudaMemsetAsync(net->g, 0, sizeof(float) * net->np, s);
  k_loss_count<<<grid_of(npx, 256), 256, 0, s>>>(tl, B, T, net->cnt);
  bf16* gcur = net->gbuf[0];
  k_loss_grad<<<grid_of(npx, 256), 256, 0, s>>>(net->out, tz, tl, tw, B, T, w_weight, net->cnt, net->loss, gcur);
  for (int l = NL - 1; l >= 0; --l) {
    const int Ho = side(net, l) - 2;   // output side of layer l
    float* dW = net->g + param_offset(l);
    float* db = dW + w_size(l);
    const long long items = (long long)B * Ho * ((Ho + 15) / 16);
    const int gw = grid_of(items, 4, 512);
    const long long opx = (long long)B * Ho * Ho;
    if (l == NL - 1) {
      k_wgrad<32, 16, 5, 32><<<dim3(gw, 9), 128, 0, s>>>(gcur, net->act[l], B, Ho, Ho, dW);
      k_bias_grad<16, 5><<<grid_of(opx, 256, 1024), 256, 0, s>>>(gcur, opx, db);
    } else if (l > 0) {
      k_wgrad<32, 32, 32, 32><<<dim3(gw, 9), 128, 0, s>>>(gcur, net->act[l], B, Ho, Ho, dW);
      k_bias_grad<32, 32><<<grid_of(opx, 256, 1024), 256, 0, s>>>(gcur, opx, db);
    } else {
      k_wgrad<16, 32, 32, 4><<<dim3(gw, 9), 128, 0, s>>>(gcur, net->act[0], B, Ho, Ho, dW);
      k_bias_grad<32, 32><<<grid_of(opx, 256, 1024), 256, 0, s>>>(gcur, opx, db);
    }
    if (l == 0) break;
    // gradient w.r.t. act[l] (side Ho + 2) masked by its ReLU: conv of pad2(g)
    const int gc = (l == NL - 1) ? 16 : 32;
    const int Hp = Ho + 4;
    k_pad2<<<grid_of((long long)B * Hp * Hp * gc / 2, 256), 256, 0, s>>>(gcur, B, Ho, Ho, gc, net->pad);
    bf16* gnext = (gcur == net->gbuf[0]) ? net->gbuf[1] : net->gbuf[0];
    conv3x3_tc(net->pad, B, Hp, gc, 32, 32, 2, net->wdg[l], nullptr, 0, gnext, net->act[l], net->err, net->num_sms, s);
    gcur = gnext;
  }
  double lh[2];
  unsigned long long ch[2];
  cudaMemcpyAsync(lh, net->loss, sizeof(lh), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(ch, net->cnt, sizeof(ch), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return NI_ERR_CUDA;
  const double ld = ch[0] ? lh[0] / ch[0] : 0.0, lw = ch[1] ? lh[1] / ch[1] : 0.0;
  if (loss_host) {
    loss_host[0] = ld + w_weight * lw;
    loss_host[1] = ld;
    loss_host[2] = lw;
  }
  return cudaGetLastError() == cudaSuccess ? NI_OK : NI_ERR_CUDA;
}

extern "C" ni_status ni_cnn_loss_grad(ni_cnn* net, const float* in, const float* tz, const int32_t* tl, const float* tw,
                                      int B, float w_weight, double* loss_host, float* grad_host, ni_stream_t stream) {
  if (!net || !in || !tz || !tl || !tw || B < 1 || B > net->maxB) return NI_ERR_INVALID_ARG;
  ni_status rc = backward(net, in, tz, tl, tw, B, w_weight, loss_host, (cudaStream_t)stream);
  if (rc != NI_OK) return rc;
  if (grad_host && cudaMemcpy(grad_host, net->g, sizeof(float) * net->np, cudaMemcpyDeviceToHost) != cudaSuccess)
    return NI_ERR_CUDA;
  return NI_OK;
}

extern "C" ni_status ni_cnn_train_step(ni_cnn* net, const float* in, const float* tz, const int32_t* tl,
                                       const float* tw, int B, float w_weight, float lr, double* loss_host,
                                       ni_stream_t stream) {
  if (!net || !in || !tz || !tl || !tw || B < 1 || B > net->maxB || !(lr > 0)) return NI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  ni_status rc = backward(net, in, tz, tl, tw, B, w_weight, loss_host, s);
  if (rc != NI_OK) return rc;
  net->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)net->step), c2 = 1.f - powf(b2, (float)net->step);
  k_adam<<<grid_of(net->np, 256), 256, 0, s>>>(net->p, net->g, net->m, net->v, net->np, lr, b1, b2, 1e-8f, c1, c2);
  repack(net, s);
  return cudaGetLastError() == cudaSuccess ? NI_OK : NI_ERR_CUDA;
}

extern "C" ni_status ni_cnn_edge_targets(const float* normals, const uint8_t* mask, const float* logdepth, int H,
                                         int W, const ni_camera* cam, double k, float* out, ni_stream_t stream) {
  if (!normals || !mask || !logdepth || !out || !cam || H < 1 || W < 1) return NI_ERR_INVALID_ARG;
  const bool persp = cam->camera == 1;
  k_edge_targets<<<grid_of((long long)H * W, 256), 256, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const float4*>(normals), mask, logdepth, H, W, persp ? 1 : 0, persp ? (float)cam->fx : 1.f,
      persp ? (float)cam->fy : 1.f, persp ? (float)cam->cx : 0.f, persp ? (float)cam->cy : 0.f, (float)k, out);
  return cudaGetLastError() == cudaSuccess ? NI_OK : NI_ERR_CUDA;
}

extern "C" ni_status ni_cnn_make_tiles(const float* normals, const uint8_t* mask, int H, int W, int tile, float* out,
                                       ni_stream_t stream) {
  if (!normals || !mask || !out || H < 1 || W < 1 || tile < 16) return NI_ERR_INVALID_ARG;
  const int ntx = (W + tile - 1) / tile, nty = (H + tile - 1) / tile;
  const long long total = (long long)ntx * nty * (tile + 2 * HALO) * (tile + 2 * HALO);
  k_make_tiles<<<grid_of(total, 256), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const float4*>(normals), mask,
                                                                      H, W, tile, ntx, ntx * nty,
                                                                      reinterpret_cast<float4*>(out));
  return cudaGetLastError() == cudaSuccess ? NI_OK : NI_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// warm start inside the fill: x0 = network log-depth, tile by tile
// ---------------------------------------------------------------------------
// x0 = channel 0; with lw, also the continuity of the right, down, left and up
// edge (sigmoids of channels 1..4: the network's estimate of w^BiNI)
__global__ void k_scatter_x0(const float* __restrict__ pred, int H, int W, int T, int ntx, const int* __restrict__ labels,
                             float* __restrict__ x, float4* __restrict__ lw) {
  const int N = H * W;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    const int u = a % W, v = a / W;
    const int t = (v / T) * ntx + (u / T);
    const long long o = (((long long)t * T + (v % T)) * T + (u % T)) * 5;
    const bool ok = labels[a] >= 0;
    x[a] = ok ? pred[o] : 0.f;
    if (lw) {
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (ok) {
        q.x = 1.f / (1.f + __expf(-pred[o + 1]));
        q.y = 1.f / (1.f + __expf(-pred[o + 2]));
        q.z = 1.f / (1.f + __expf(-pred[o + 3]));
        q.w = 1.f / (1.f + __expf(-pred[o + 4]));
      }
      lw[a] = q;
    }
  }
}

ni_status warm_start_launch(ni_handle* h, cudaStream_t s) {
  ni_cnn* net = h->net;
  if (!net) return ni_fail(h, NI_ERR_NO_NET, "warm start requested but no network is loaded");
  const int T = net->T, S = net->S;
  const int ntx = (h->W + T - 1) / T, nty = (h->H + T - 1) / T, nt = ntx * nty;
  if (!h->tile_in) {
    cudaError_t e = cudaMalloc((void**)&h->tile_in, sizeof(float) * 4 * (size_t)nt * S * S);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->tile_out, sizeof(float) * 5 * (size_t)nt * T * T);
    if (e != cudaSuccess) return ni_cuda_check(h, e, "warm-start buffers");
  }
  ni_status rc = ni_cnn_make_tiles(reinterpret_cast<const float*>(h->normals), h->mask, h->H, h->W, T, h->tile_in, s);
  NI_COUNT(h);
  if (rc != NI_OK) return ni_fail(h, rc, "warm-start tiles");
  for (int b0 = 0; b0 < nt; b0 += net->maxB) {
    const int B = std::min(net->maxB, nt - b0);
    rc = ni_cnn_forward(net, h->tile_in + (size_t)b0 * S * S * 4, B, h->tile_out + (size_t)b0 * T * T * 5, s);
    h->launches += 1 + NL;
    if (rc != NI_OK) return ni_fail(h, rc, "warm-start forward");
  }
  if (h->cfg.learned_weights && !h->lw) {
    cudaError_t e = cudaMalloc((void**)&h->lw, sizeof(float4) * (size_t)h->N);
    if (e != cudaSuccess) return ni_cuda_check(h, e, "learned edge weights");
  }
  k_scatter_x0<<<grid_of(h->N, 256), 256, 0, s>>>(h->tile_out, h->H, h->W, T, ntx, h->labels, h->x,
                                                   h->cfg.learned_weights ? h->lw : nullptr); NI_COUNT(h);
  return ni_cuda_check(h, cudaGetLastError(), "warm start");
}

extern "C" ni_status ni_load_net(ni_handle* h, const char* path) {
  if (!h) return NI_ERR_INVALID_ARG;
  if (!path) return ni_fail(h, NI_ERR_INVALID_ARG, "path is required");
  FILE* f = fopen(path, "rb");
  if (!f) return ni_fail(h, NI_ERR_INVALID_ARG, std::string("cannot open ") + path);
  char magic[8] = {0};
  int hdr[2] = {0, 0};
  const int np = num_params();
  std::vector<float> buf(np);
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "NICNN001", 8) == 0 && fread(hdr, sizeof(int), 2, f) == 2 &&
            hdr[0] == np && hdr[1] >= 16 && hdr[1] % 16 == 0 && fread(buf.data(), sizeof(float), np, f) == (size_t)np;
  fclose(f);
  if (!ok) return ni_fail(h, NI_ERR_INVALID_ARG, std::string("malformed network file ") + path);
  if (h->net) ni_cnn_destroy(h->net);
  h->net = nullptr;
  // tiles per forward launch: the whole map up to 64 tiles (fewer, longer launches)
  const int nt = ((h->W + hdr[1] - 1) / hdr[1]) * ((h->H + hdr[1] - 1) / hdr[1]);
  ni_status rc = ni_cnn_create(std::max(1, std::min(nt, 64)), hdr[1], 0, &h->net);
  if (rc != NI_OK) return ni_fail(h, rc, "network allocation");
  rc = ni_cnn_set_params(h->net, buf.data());
  if (rc != NI_OK) return ni_fail(h, rc, "network upload");
  return NI_OK;
}
