// 3x3 valid convolutions of the learned warm start on the 5th-generation
// tensor cores (tcgen05.mma, BF16 operands, FP32 accumulator in tensor memory).
// Not in the paper: the network is an extension beyond it.
//
// Output pixels are numbered with the input's row pitch, p = y Wi + x (the two
// columns x >= Wo of every row are computed and dropped), so that the input
// pixel of tap (dy, dx) is p + dy Wi + dx for every p: linear in p across rows.
// Implicit GEMM per work item = 128 consecutive p of one image:
//   D[m][co] = sum_{dy, dx, ci} in[p0 + m + dy Wi + dx][ci] * w[dy, dx][co][ci]
// M = 128 pixels (the TMEM lanes), N = CO output channels, K = 9 taps x CI.
//   * A (pixels x channels, K-major) is staged in shared memory once per dy:
//     the 130 input pixels p0 + dy Wi .. p0 + dy Wi + 129, stored as the
//     no-swizzle canonical layout with 8-row groups 128 B apart (SBO) and the
//     16-byte channel chunks of all 130 rows 130 x 16 B apart (LBO).  The
//     views for dx = 0, 1, 2 are the same bytes with the descriptor's start
//     advanced by dx rows (16 B), so one load of 3 x 130 pixels feeds all 9 taps.
//   * B (channels x taps, K-major per output channel) lives in shared memory
//     for the whole launch.
//   * One thread issues the 9 x CI/16 MMAs of an item into a TMEM accumulator
//     of CO columns and commits them to an mbarrier; the four warps then read
//     their 32 TMEM lanes (pixels) with tcgen05.ld and run the epilogue (bias
//     and ReLU, the linear last layer, or the ReLU mask of the gradient).
//   * Two staging buffers and two accumulators: while the epilogue of item j
//     runs, the MMAs of item j + 1 and the cp.async loads of item j + 2 are
//     in flight.
// Every wait on the mbarrier is bounded; on a timeout the CTA flags
// NI_DEV_ERR_TIMEOUT, stops issuing, waits (bounded) for what it issued, frees
// its tensor memory and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "ni_internal.cuh"

typedef __nv_bfloat16 bf16;

namespace {

constexpr int TC_M = 128;          // output pixels per item (TMEM lanes)
constexpr int TC_ROWS = TC_M + 2;  // input pixels staged per row
constexpr int TC_THREADS = 128;
constexpr long long TC_SPIN = 1ll << 26;   // bounded mbarrier wait (polls)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle (layout type 0), version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3fff);
  d |= (uint64_t)((lbo >> 4) & 0x3fff) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3fff) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, int accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      :: "r"(tmem_d), "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}

// bounded wait for the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < TC_SPIN; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

template <int NC>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[NC]) {
  static_assert(NC == 16 || NC == 32, "columns");
  uint32_t r[NC];
  if constexpr (NC == 32) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < NC; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// CI input channels, CO output channels of the MMA (N), WCO output channels
// stored in the weights (WCO <= CO: the rest are zero), MODE as k_conv:
//   0: bf16 out = relu(acc + b); 1: float out [.][WCO] = acc + b; 2: bf16 out = acc * [act_mask > 0]
template <int CI, int CO, int WCO, int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tc(const bf16* __restrict__ in, int B, int Hi,
                                                        const bf16* __restrict__ w,
                                                        const float* __restrict__ bias, int nbias,
                                                        void* __restrict__ out, const bf16* __restrict__ act_mask,
                                                        int* err) {
  static_assert(CI % 16 == 0 && CO % 16 == 0 && WCO <= CO, "channels");
  constexpr int KC = CI / 8;                       // 16-byte channel chunks per pixel
  constexpr uint32_t LBO_A = TC_ROWS * 16;         // between channel chunks of the staged rows
  constexpr uint32_t ROW_BYTES = KC * LBO_A;       // one staged input row (130 px, all channels)
  constexpr uint32_t STAGE_BYTES = 3 * ROW_BYTES;  // rows y, y + 1, y + 2
  constexpr uint32_t LBO_B = CO * 16;              // between channel chunks of one tap's weights
  constexpr uint32_t TAP_B = KC * LBO_B;
  constexpr uint32_t idesc = idesc_bf16(TC_M, CO);
  constexpr uint32_t TCOLS = 2 * CO < 32 ? 32 : 2 * CO;   // two accumulators of CO columns
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* bsm = smem;                                  // weights: 9 taps
  unsigned char* asm0 = smem + ((9 * TAP_B + 1023) & ~1023u); // two staging buffers
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Ho = Hi - 2, Wi = Hi, Wo = Ho;
  const int per_img = (Ho * Wi + TC_M - 1) / TC_M;   // items of one image
  const long long items = (long long)B * per_img;
  const long long img_in = (long long)Hi * Wi;

  // weights -> shared memory, chunk k of tap t, output channel n at t * TAP_B + k * LBO_B + n * 16
  for (int i = tid; i < 9 * CO * KC; i += TC_THREADS) {
    const int k = i % KC, n = (i / KC) % CO, t = i / (KC * CO);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (n < WCO) v = *reinterpret_cast<const uint4*>(w + ((long long)t * WCO + n) * CI + k * 8);
    *reinterpret_cast<uint4*>(bsm + t * TAP_B + k * LBO_B + n * 16) = v;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(TCOLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  // stage the 3 x 130 input pixels of an item into buffer sb (zeros past the image)
  auto stage = [&](long long item, int sb) {
    const long long n = item / per_img;
    const int p0 = (int)(item % per_img) * TC_M;
    const uint32_t base = smem_u32(asm0 + sb * STAGE_BYTES);
    for (int i = tid; i < 3 * TC_ROWS * KC; i += TC_THREADS) {
      const int k = i % KC, m = (i / KC) % TC_ROWS, dy = i / (KC * TC_ROWS);
      const int q = p0 + dy * Wi + m;
      const bool ok = q < img_in;
      const bf16* src = in + (n * img_in + (ok ? q : 0)) * CI + k * 8;
      cp16(base + dy * ROW_BYTES + k * LBO_A + m * 16, src, ok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  // thread 0: the 9 x CI/16 MMAs of the item staged in buffer sb, into accumulator ab
  auto issue = [&](int sb, int ab) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t a0 = smem_u32(asm0 + sb * STAGE_BYTES), b0 = smem_u32(bsm);
    int acc = 0;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int dy = t / 3, dx = t % 3;
#pragma unroll
      for (int ks = 0; ks < CI / 16; ++ks) {
        const uint64_t ad = sdesc(a0 + dy * ROW_BYTES + dx * 16 + ks * 2 * LBO_A, LBO_A, 128);
        const uint64_t bd = sdesc(b0 + t * TAP_B + ks * 2 * LBO_B, LBO_B, 128);
        mma_issue(tmem + ab * CO, ad, bd, idesc, acc);
        acc = 1;
      }
    }
    mma_commit(&bar[ab]);
  };

  // Pipeline: item j lives in staging buffer j & 1 and accumulator j & 1.  While
  // the epilogue of item j runs, the MMAs of item j + 1 and the loads of item
  // j + 2 are in flight.
  const long long step = gridDim.x;
  uint32_t ph0 = 0u, ph1 = 0u;   // phase parity of bar[0], bar[1]
  long long item = blockIdx.x;
  if (item < items) {
    stage(item, 0);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // cp.async writes -> the MMA's reads
    __syncthreads();
    if (tid == 0) issue(0, 0);
    if (item + step < items) stage(item + step, 1);
  }
  for (int j = 0; item < items; item += step, ++j) {
    const int b = j & 1;
    const long long nxt = item + step;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (nxt < items && tid == 0) issue(b ^ 1, b ^ 1);
    const uint32_t pb = b ? ph1 : ph0;
    const bool ok = mbar_wait(&bar[b], pb);
    if (!ok) {
      if (tid == 0) atomicOr(err, NI_DEV_ERR_TIMEOUT);
      s_fail = 1;
    }
    __syncthreads();
    if (s_fail) {   // once more, bounded, for the MMAs in flight
      mbar_wait(&bar[b], pb);
      if (nxt < items) mbar_wait(&bar[b ^ 1], b ? ph0 : ph1);
      break;
    }
    if (b) ph1 ^= 1u; else ph0 ^= 1u;
    // item j's staging buffer is free: load item j + 2 into it
    if (nxt + step < items) stage(nxt + step, b);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: warp w owns TMEM lanes (pixels) 32 w .. 32 w + 31
    float v[CO];
    tmem_ld<CO>(tmem + ((uint32_t)(warp * 32) << 16) + b * CO, v);
    {
      const long long n = item / per_img;
      const int p = (int)(item % per_img) * TC_M + warp * 32 + lane;
      const int y = p / Wi, x = p % Wi;
      if (y < Ho && x < Wo) {
        const long long px = (n * Ho + y) * Wo + x;
        if constexpr (MODE == 0) {
          uint32_t pk[CO / 2];
#pragma unroll
          for (int c = 0; c < CO; c += 2)
            pk[c / 2] = pack2(fmaxf(v[c] + (c < nbias ? bias[c] : 0.f), 0.f),
                              fmaxf(v[c + 1] + (c + 1 < nbias ? bias[c + 1] : 0.f), 0.f));
          uint4* o = reinterpret_cast<uint4*>(static_cast<bf16*>(out) + px * CO);
#pragma unroll
          for (int q = 0; q < CO / 8; ++q) o[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
        } else if constexpr (MODE == 1) {
          float* o = static_cast<float*>(out) + px * WCO;
#pragma unroll
          for (int c = 0; c < WCO; ++c) o[c] = v[c] + (c < nbias ? bias[c] : 0.f);
        } else {
          const bf16* am = act_mask + px * CO;
          uint32_t pk[CO / 2];
#pragma unroll
          for (int c = 0; c < CO; c += 2) {
            const float m0 = __bfloat162float(am[c]) > 0.f ? 1.f : 0.f;
            const float m1 = __bfloat162float(am[c + 1]) > 0.f ? 1.f : 0.f;
            pk[c / 2] = pack2(v[c] * m0, v[c + 1] * m1);
          }
          uint4* o = reinterpret_cast<uint4*>(static_cast<bf16*>(out) + px * CO);
#pragma unroll
          for (int q = 0; q < CO / 8; ++q) o[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
        }
      }
    }
    // accumulator b is rewritten by the MMAs of item j + 2
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TCOLS)
                 : "memory");
}

template <int CI, int CO, int WCO, int MODE>
cudaError_t launch(const bf16* in, int B, int Hi, const bf16* w, const float* bias, int nbias, void* out,
                   const bf16* act_mask, int* err, int num_sms, cudaStream_t s) {
  constexpr int KC = CI / 8;
  constexpr uint32_t tapb = KC * CO * 16;
  constexpr uint32_t stage = 3 * KC * TC_ROWS * 16;
  constexpr size_t smem = ((9 * tapb + 1023) & ~1023u) + 2 * (size_t)stage;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv_tc<CI, CO, WCO, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const int Ho = Hi - 2;
  const long long items = (long long)B * ((Ho * Hi + TC_M - 1) / TC_M);
  // persistent CTAs: as many as shared memory lets one SM hold (CTAs beyond the
  // resident ones simply wait for a slot)
  const int per_sm = std::max(1, std::min(4, (int)((227 * 1024) / (smem + 2048))));
  const long long cap = (long long)num_sms * per_sm;
  const int grid = (int)std::max(1LL, std::min(items, cap));
  k_conv_tc<CI, CO, WCO, MODE><<<grid, TC_THREADS, smem, s>>>(in, B, Hi, w, bias, nbias, out, act_mask, err);
  return cudaGetLastError();
}

}  // namespace

// Valid 3x3 convolution of NHWC bf16 input [B][Hi][Hi][ci] with weights
// [9][wco][ci] on the tensor cores.  mode 0: bf16 relu(acc + b) with co
// channels; mode 1: float acc + b with wco channels; mode 2: bf16 acc masked
// by act_mask > 0.  bias holds nbias values (missing ones count as 0).
// Supported (ci, co, wco, mode): (16, 32, 32, 0), (32, 32, 32, 0),
// (32, 16, 8, 1), (16, 32, 32, 2), (32, 32, 32, 2).
cudaError_t conv3x3_tc(const bf16* in, int B, int Hi, int ci, int co, int wco, int mode, const bf16* w,
                       const float* bias, int nbias, void* out, const bf16* act_mask, int* err, int num_sms,
                       cudaStream_t s) {
  if (ci == 16 && co == 32 && wco == 32 && mode == 0)
    return launch<16, 32, 32, 0>(in, B, Hi, w, bias, nbias, out, act_mask, err, num_sms, s);
  if (ci == 32 && co == 32 && wco == 32 && mode == 0)
    return launch<32, 32, 32, 0>(in, B, Hi, w, bias, nbias, out, act_mask, err, num_sms, s);
  if (ci == 32 && co == 16 && wco == 8 && mode == 1)
    return launch<32, 16, 8, 1>(in, B, Hi, w, bias, nbias, out, act_mask, err, num_sms, s);
  if (ci == 16 && co == 32 && wco == 32 && mode == 2)
    return launch<16, 32, 32, 2>(in, B, Hi, w, bias, nbias, out, act_mask, err, num_sms, s);
  if (ci == 32 && co == 32 && wco == 32 && mode == 2)
    return launch<32, 32, 32, 2>(in, B, Hi, w, bias, nbias, out, act_mask, err, num_sms, s);
  return cudaErrorInvalidValue;
}
