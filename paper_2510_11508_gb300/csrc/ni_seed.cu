// Seeding of continuous components (Sec. 3.3, first paragraph; rows a1-a2).
//
// Edge predicate: an edge (a, b) of the 4-neighbour pixel graph (with
// 8-connectivity also the diagonal edges) is kept iff
// both pixels are valid and n_a . n_b > cos(theta_c), the dot product of the
// float32 inputs evaluated in float64 (products are exact, sums rounded in the
// order x, y, z), so the decision is bit-identical to any IEEE-754 evaluation
// of the same expression.
//
// Labelling: union-find in which a root always links under the smaller root,
// so every component's root is its smallest raster index.
//   k_seed_local   one CTA per 32 x 16 tile: normals into shared memory, the
//                  tile's internal edges united with shared-memory atomics,
//                  tile roots written to the global parent array;
//   k_seed_border  the edges that cross tile borders, united in global memory;
//   k_seed_diag    8-connectivity only: every diagonal edge, in global memory;
//   k_compress     parent[i] <- root(i);
//   k_count_roots / scan / k_rank_roots / k_gather_labels
//                  canonical labels = rank of each root among all roots in
//                  raster order, K = number of roots.
#include "ni_internal.cuh"

#define TSW NI_SEED_TSW
#define TSH NI_SEED_TSH

__device__ __forceinline__ bool seed_keep(const float4 a, const float4 b, double cth) {
  double d = __dadd_rn(__dmul_rn((double)a.x, (double)b.x), __dmul_rn((double)a.y, (double)b.y));
  d = __dadd_rn(d, __dmul_rn((double)a.z, (double)b.z));
  return d > cth;
}

__global__ void __launch_bounds__(TSW * TSH)
k_seed_local(const float4* __restrict__ nrm, const uint8_t* __restrict__ mask, int H, int W,
             double cth, float fx, float fy, float cx, float cy, int persp, int validate,
             int* __restrict__ parent, DevState* st) {
  __shared__ int sp[TSW * TSH];
  __shared__ float4 sn[TSW * TSH];
  __shared__ unsigned char sv[TSW * TSH];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int gx = blockIdx.x * TSW + tx, gy = blockIdx.y * TSH + ty;
  const int l = threadIdx.x;
  const bool in = (gx < W) && (gy < H);
  const int gi = in ? gy * W + gx : 0;
  const bool valid = in && mask[gi] != 0;
  float4 n = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid) n = ldg4(&nrm[gi]);
  sn[l] = n;
  sv[l] = valid ? 1 : 0;
  sp[l] = valid ? l : -1;
  int bad = 0;
  if (validate && valid) {
    float len = sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
    float nt = persp ? (n.x * ((gx - cx) / fx) + n.y * ((gy - cy) / fy) + n.z) : n.z;
    bad = !(fabsf(len - 1.0f) <= 1e-3f) || !(fabsf(nt) > 1e-6f);
  }
  int nbad = __syncthreads_count(bad);
  int nval = __syncthreads_count(valid);
  if (threadIdx.x == 0) {
    if (nval) atomicAdd(&st->n_valid, nval);
    if (nbad) {
      atomicAdd(&st->n_bad_normals, nbad);
      atomicOr(&st->err, NI_DEV_ERR_BAD_NORMAL);
    }
  }
  if (valid) {
    if (tx + 1 < TSW && gx + 1 < W && sv[l + 1] && seed_keep(n, sn[l + 1], cth)) uf_unite(sp, l, l + 1);
    if (ty + 1 < TSH && gy + 1 < H && sv[l + TSW] && seed_keep(n, sn[l + TSW], cth))
      uf_unite(sp, l, l + TSW);
  }
  __syncthreads();
  if (in) {
    int g = -1;
    if (valid) {
      int rl = uf_find(sp, l);
      g = (blockIdx.y * TSH + (rl / TSW)) * W + blockIdx.x * TSW + (rl % TSW);
    }
    parent[gi] = g;
  }
}

// Edges crossing tile borders: thread i < nbx * H handles the right edge of
// pixel (32 c + 31, y); the rest the down edge of pixel (x, 16 r + 15).
__global__ void k_seed_border(const float4* __restrict__ nrm, const uint8_t* __restrict__ mask,
                              int H, int W, double cth, int nbx, int nby, int* __restrict__ parent) {
  const long long nr = (long long)nbx * H;
  const long long total = nr + (long long)nby * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int a, b;
    if (i < nr) {
      int c = (int)(i / H), y = (int)(i % H);
      int x = c * TSW + TSW - 1;
      if (x + 1 >= W) continue;
      a = y * W + x;
      b = a + 1;
    } else {
      long long j = i - nr;
      int r = (int)(j / W), x = (int)(j % W);
      int y = r * TSH + TSH - 1;
      if (y + 1 >= H) continue;
      a = y * W + x;
      b = a + W;
    }
    if (!mask[a] || !mask[b]) continue;
    if (seed_keep(ldg4(&nrm[a]), ldg4(&nrm[b]), cth)) uf_unite(parent, a, b);
  }
}

// 8-connectivity: the two diagonal edges of each pixel, to the lower-right and
// lower-left neighbour, united in global memory after the 4-connected phases.
__global__ void k_seed_diag(const float4* __restrict__ nrm, const uint8_t* __restrict__ mask, int H, int W,
                            double cth, int* __restrict__ parent) {
  const long long n = (long long)(H - 1) * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int a = (int)i, x = a % W;
    if (!mask[a]) continue;
    const float4 na = ldg4(&nrm[a]);
    if (x + 1 < W && mask[a + W + 1] && seed_keep(na, ldg4(&nrm[a + W + 1]), cth)) uf_unite(parent, a, a + W + 1);
    if (x >= 1 && mask[a + W - 1] && seed_keep(na, ldg4(&nrm[a + W - 1]), cth)) uf_unite(parent, a, a + W - 1);
  }
}

__global__ void k_compress(int* __restrict__ parent, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int p = parent[i];
    if (p >= 0 && p != i) parent[i] = uf_find(parent, i);
  }
}

// ---------------------------------------------------------------------------
// chunked exclusive scan helpers: block b of the fixed grid owns elements
// [b * chunk, (b + 1) * chunk) with chunk = ceil(n / gridDim.x).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void chunk_range(int n, int& beg, int& end) {
  int chunk = (n + gridDim.x - 1) / gridDim.x;
  beg = min(n, blockIdx.x * chunk);
  end = min(n, beg + chunk);
}

__global__ void k_count_roots(const int* __restrict__ parent, const int* n_ptr, int n_const,
                              int* __restrict__ blk) {
  __shared__ int sh[40];
  int n = n_ptr ? *n_ptr : n_const;
  int beg, end;
  chunk_range(n, beg, end);
  int c = 0;
  for (int i = beg + threadIdx.x; i < end; i += blockDim.x) c += (parent[i] == i);
  c = block_sum_i(c, sh);
  if (threadIdx.x == 0) blk[blockIdx.x] = c;
}

// Single-block exclusive scan of nblocks (<= 1024) ints in place; total stored.
__global__ void k_scan_blocks(int* __restrict__ blk, int nblocks, int* __restrict__ total_out) {
  __shared__ int sh[40];
  int v = (threadIdx.x < nblocks) ? blk[threadIdx.x] : 0;
  int tot;
  int ex = block_excl_scan_i(v, sh, &tot);
  if (threadIdx.x < nblocks) blk[threadIdx.x] = ex;
  if (threadIdx.x == 0) *total_out = tot;
}

void scan_blocks_launch(int* blk, int nblocks, int* total_out, cudaStream_t s) {
  k_scan_blocks<<<1, 1024, 0, s>>>(blk, nblocks, total_out);
}

__global__ void k_rank_roots(const int* __restrict__ parent, const int* n_ptr, int n_const,
                             const int* __restrict__ blk, int* __restrict__ out) {
  __shared__ int sh[40];
  int n = n_ptr ? *n_ptr : n_const;
  int beg, end;
  chunk_range(n, beg, end);
  int base = blk[blockIdx.x];
  for (int t0 = beg; t0 < end; t0 += blockDim.x) {
    int i = t0 + threadIdx.x;
    int f = (i < end) && (parent[i] == i);
    int tot;
    int ex = block_excl_scan_i(f, sh, &tot);
    if (f) out[i] = base + ex;
    base += tot;
  }
}

__global__ void k_gather_labels(const int* __restrict__ parent, int n, int* __restrict__ labels) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int p = parent[i];
    if (p < 0) labels[i] = -1;
    else if (p != i) labels[i] = labels[p];
  }
}

__global__ void k_seed_finish(DevState* st, const int* count) {
  st->K = *count;
  st->K0 = *count;
}

static int grid_for(ni_handle* h, long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  long long cap = (long long)h->num_sms * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

ni_status seed_launch(ni_handle* h, cudaStream_t s) {
  const int H = h->H, W = h->W, N = h->N;
  const int nbx = (W + TSW - 1) / TSW, nby = (H + TSH - 1) / TSH;
  dim3 g(nbx, nby);
  k_seed_local<<<g, TSW * TSH, 0, s>>>(h->normals, h->mask, H, W, h->cos_theta, h->fx, h->fy, h->cx,
                                        h->cy, h->persp, h->cfg.validate, h->parent, h->st); NI_COUNT(h);
  long long nb = (long long)nbx * H + (long long)nby * W;
  k_seed_border<<<grid_for(h, nb, 256), 256, 0, s>>>(h->normals, h->mask, H, W, h->cos_theta, nbx, nby,
                                                       h->parent); NI_COUNT(h);
  if (h->cfg.connectivity == 8 && H > 1) {
    k_seed_diag<<<grid_for(h, (long long)(H - 1) * W, 256), 256, 0, s>>>(h->normals, h->mask, H, W, h->cos_theta,
                                                                        h->parent); NI_COUNT(h);
  }
  k_compress<<<grid_for(h, N, 256), 256, 0, s>>>(h->parent, N); NI_COUNT(h);
  k_count_roots<<<NI_SCAN_BLOCKS, NI_SCAN_THREADS, 0, s>>>(h->parent, nullptr, N, h->blk); NI_COUNT(h);
  scan_blocks_launch(h->blk, NI_SCAN_BLOCKS, h->d_count, s); NI_COUNT(h);
  k_rank_roots<<<NI_SCAN_BLOCKS, NI_SCAN_THREADS, 0, s>>>(h->parent, nullptr, N, h->blk, h->labels); NI_COUNT(h);
  k_gather_labels<<<grid_for(h, N, 256), 256, 0, s>>>(h->parent, N, h->labels); NI_COUNT(h);
  k_seed_finish<<<1, 1, 0, s>>>(h->st, h->d_count); NI_COUNT(h);
  return ni_cuda_check(h, cudaGetLastError(), "seeding kernels");
}
