// Allocation-free seeding entry point.
//
// Some callers of this library are not allowed to allocate device memory once
// they are running: a real-time pipeline that reserves all of its memory at
// start-up, a host framework whose own allocator owns the device and forbids
// other allocations, or code that runs where cudaMalloc would synchronise the
// device or fail under a fixed memory-pool limit.  ni_seed_components needs a
// handle, and ni_create allocates.  This entry point performs the same seeding
// (same kernels, same labels) with its scratch in a fixed, file-scope device
// array instead, so the caller supplies only the input and output buffers.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "ni_internal.cuh"

// kernels of ni_seed.cu (launched here with scratch pointers into g_scratch)
__global__ void k_seed_local(const float4* nrm, const uint8_t* mask, int H, int W, double cth, float fx,
                             float fy, float cx, float cy, int persp, int validate, int* parent,
                             DevState* st);
__global__ void k_seed_border(const float4* nrm, const uint8_t* mask, int H, int W, double cth, int nbx,
                              int nby, int* parent);
__global__ void k_compress(int* parent, int n);
__global__ void k_count_roots(const int* parent, const int* n_ptr, int n_const, int* blk);
__global__ void k_scan_blocks(int* blk, int nblocks, int* total_out);
__global__ void k_rank_roots(const int* parent, const int* n_ptr, int n_const, const int* blk, int* out);
__global__ void k_gather_labels(const int* parent, int n, int* labels);

// Layout of the static scratch: DevState, then the scan partials and a count,
// then the union-find parent array of NI_NOALLOC_MAX_PIXELS entries.
#define NI_NOALLOC_MAX_PIXELS (1 << 22)
#define NI_NOALLOC_HEAD_BYTES 16384
#define NI_NOALLOC_BYTES (NI_NOALLOC_HEAD_BYTES + 4 * (size_t)NI_NOALLOC_MAX_PIXELS)

// DevState, rounded up to 256 bytes, then NI_SCAN_BLOCKS + 1 partial sums and the count
static_assert(((sizeof(DevState) + 255) / 256) * 256 + 4 * (NI_SCAN_BLOCKS + 2) <= NI_NOALLOC_HEAD_BYTES,
              "scratch head too small");

static __device__ __align__(256) unsigned char g_scratch[NI_NOALLOC_BYTES];

namespace {
std::mutex g_mu;
unsigned char* g_ptr[64] = {};   // device address of g_scratch, per device ordinal
int g_sms[64] = {};
}  // namespace

// One-time set-up per device, with that device current: the host-side name
// g_scratch is only a stand-in, so the kernels get the device address.
static cudaError_t scratch_for_current_device(unsigned char** ptr, int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = static_cast<unsigned char*>(p);
    g_sms[dev] = n;
  }
  *ptr = g_ptr[dev];
  *sms = g_sms[dev];
  return cudaSuccess;
}

extern "C" ni_status ni_seed_components_noalloc(const float* normals, const uint8_t* mask, int H, int W,
                                                const ni_camera* cam, double theta_c_deg, int32_t* labels_out,
                                                int32_t* K_out_device, ni_stream_t stream) {
  if (!normals || !mask || !labels_out || !K_out_device || !cam) return NI_ERR_INVALID_ARG;
  if (H < 1 || W < 1) return NI_ERR_INVALID_ARG;
  if ((long long)H * W > NI_NOALLOC_MAX_PIXELS) return NI_ERR_INVALID_ARG;   // beyond the static scratch
  if (((uintptr_t)normals) & 15) return NI_ERR_INVALID_ARG;
  if (cam->camera != 0 && cam->camera != 1) return NI_ERR_INVALID_ARG;
  unsigned char* base = nullptr;
  int sms = 0;
  cudaError_t e = scratch_for_current_device(&base, &sms);
  if (e != cudaSuccess) return NI_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  DevState* st = reinterpret_cast<DevState*>(base);
  int* blk = reinterpret_cast<int*>(base + ((sizeof(DevState) + 255) / 256) * 256);
  int* count = blk + NI_SCAN_BLOCKS + 1;
  int* parent = reinterpret_cast<int*>(base + NI_NOALLOC_HEAD_BYTES);
  const int N = H * W;
  const bool persp = cam->camera == 1;
  const float fx = persp ? (float)cam->fx : 1.f, fy = persp ? (float)cam->fy : 1.f;
  const float cx = persp ? (float)cam->cx : 0.f, cy = persp ? (float)cam->cy : 0.f;
  const double cth = theta_c_deg < 0 ? 2.0 : cos(theta_c_deg * (M_PI / 180.0));
  // the counters a previous call left behind must start at zero
  e = cudaMemsetAsync(st, 0, sizeof(DevState), s);
  if (e != cudaSuccess) return NI_ERR_CUDA;
  const int nbx = (W + NI_SEED_TSW - 1) / NI_SEED_TSW, nby = (H + NI_SEED_TSH - 1) / NI_SEED_TSH;
  k_seed_local<<<dim3(nbx, nby), NI_SEED_TSW * NI_SEED_TSH, 0, s>>>(reinterpret_cast<const float4*>(normals), mask, H, W, cth, fx, fy,
                                              cx, cy, persp ? 1 : 0, 0, parent, st);
  const long long nb = (long long)nbx * H + (long long)nby * W;
  const int cap = sms * 8;
  const int gb = (int)std::max(1LL, std::min((nb + 255) / 256, (long long)cap));
  const int gp = (int)std::max(1LL, std::min(((long long)N + 255) / 256, (long long)cap));
  k_seed_border<<<gb, 256, 0, s>>>(reinterpret_cast<const float4*>(normals), mask, H, W, cth, nbx, nby, parent);
  k_compress<<<gp, 256, 0, s>>>(parent, N);
  k_count_roots<<<NI_SCAN_BLOCKS, NI_SCAN_THREADS, 0, s>>>(parent, nullptr, N, blk);
  k_scan_blocks<<<1, 1024, 0, s>>>(blk, NI_SCAN_BLOCKS, count);
  k_rank_roots<<<NI_SCAN_BLOCKS, NI_SCAN_THREADS, 0, s>>>(parent, nullptr, N, blk, labels_out);
  k_gather_labels<<<gp, 256, 0, s>>>(parent, N, labels_out);
  e = cudaMemcpyAsync(K_out_device, count, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return NI_ERR_CUDA;
  e = cudaGetLastError();
  return e == cudaSuccess ? NI_OK : NI_ERR_CUDA;
}
