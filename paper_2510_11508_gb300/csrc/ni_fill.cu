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
// Weights are two planes, wr[a] (edge a - a+1) and wd[a] (edge a - a+W); the
// left and upper weights of a are wr[a-1] and wd[a-W].  Because wr is 0 in the
// last column, raster-linear indexing needs no row tests: wr[a-1] is 0 when a
// starts a row.
//
// Solve: Jacobi-preconditioned CG on the block-diagonal weighted Laplacian,
//   matrix-free 5-point stencil in float32, reductions in float64 (or float32
//   warp/CTA trees, precision = 1):
//   plain   (batched = 0): one global CG; three kernels per iteration,
//           iteration chunks replayed from a CUDA graph;
//   batched (batched = 1): k_pcg_tiles, one cooperative persistent launch with
//           a step length, direction update and convergence mask per component,
//           working on a list of 1024-pixel tiles that still hold an active
//           component.
// Both start from x0 = 0, the batched one also from the warm start, which it
// first scales per component by the minimiser of the energy along x0; both
// project the right-hand side and the result to zero mean per component.
#include <algorithm>
#include <vector>

#include "ni_internal.cuh"
#include "ni_tile.cuh"

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
                             float* __restrict__ ntau, float* __restrict__ wr, float* __restrict__ wd) {
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
    wr[a] = w.x;
    wd[a] = w.y;
  }
}

// Jacobi inverse diagonal and right-hand side b_a = sum_b w_ab omega~_{b->a}.
__global__ void k_diag_rhs(const float* __restrict__ wr, const float* __restrict__ wd,
                           const float2* __restrict__ omega, int H, int W, float* __restrict__ invd,
                           float* __restrict__ rhs) {
  const int N = H * W;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    const int v = a / W;
    const float2 om = omega[a];
    const float wra = wr[a], wda = wd[a];
    float wl = 0.f, wu = 0.f, ol = 0.f, ou = 0.f;
    if (a > 0) { wl = wr[a - 1]; ol = omega[a - 1].x; }
    if (v > 0) { wu = wd[a - W]; ou = omega[a - W].y; }
    const float d = wra + wda + wl + wu;
    invd[a] = d > 0.f ? 1.0f / d : 0.f;
    // omega~_{l->a} = -omega~_{a->l} (antisymmetry of Eq. 3)
    rhs[a] = wra * om.x + wda * om.y - wl * ol - wu * ou;
  }
}

// BiNI reweighting sweep of the fill (n_fill_irls > 1): the weight of an edge
// (a, b) is W_{b->a} + W_{a->b} at the current z~ (Eq. 5), the opposite
// neighbours oa = a - (b - a) and ob = b + (b - a) counted only inside the
// component.  om_ab = omega~_{b->a}; om_oa = omega~ stored for the edge (oa, a),
// which is omega~_{a->oa}; om_ob = omega~ stored for the edge (b, ob), which is
// omega~_{ob->b}.  res: the two sides compared through their residuals
// chi_{c->p} = z~_p - z~_c - omega~_{c->p} instead of the raw differences.
__device__ __forceinline__ float bini_pair(float ga, float gb, float xa, float xb, float xoa, float xob, bool hoa,
                                           bool hob, float om_ab, float om_oa, float om_ob, int res, float k) {
  float main2, da, db;
  if (res) {
    const float c = xa - xb - om_ab;
    main2 = c * c;
    const float ca = xa - xoa + om_oa, cb = xb - xob - om_ob;
    da = hoa ? ca * ca : 0.f;
    db = hob ? cb * cb : 0.f;
  } else {
    main2 = (xb - xa) * (xb - xa);
    da = hoa ? (xoa - xa) * (xoa - xa) : 0.f;
    db = hob ? (xob - xb) * (xob - xb) : 0.f;
  }
  const float g2a = ga * ga, g2b = gb * gb;
  return g2a / (1.f + expf(-k * g2a * (da - main2))) + g2b / (1.f + expf(-k * g2b * (db - main2)));
}

__global__ void k_fill_reweight(const float* __restrict__ ntau, const int* __restrict__ labels,
                                const float* __restrict__ x, const float2* __restrict__ omega, int H, int W,
                                int persp, float fx, float fy, float k, int res, float* __restrict__ wr,
                                float* __restrict__ wd) {
  const int N = H * W;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    const int la = labels[a];
    const int u = a % W, v = a / W;
    if (la >= 0 && wr[a] > 0.f) {
      const int b = a + 1;
      const float f = persp ? fx : 1.f;
      const bool ho_a = (u > 0) && labels[a - 1] == la;
      const bool ho_b = (u + 2 < W) && labels[b + 1] == la;
      wr[a] = bini_pair(f * ntau[a], f * ntau[b], x[a], x[b], ho_a ? x[a - 1] : 0.f, ho_b ? x[b + 1] : 0.f, ho_a,
                        ho_b, omega[a].x, ho_a ? omega[a - 1].x : 0.f, ho_b ? omega[b].x : 0.f, res, k);
    }
    if (la >= 0 && wd[a] > 0.f) {
      const int b = a + W;
      const float f = persp ? fy : 1.f;
      const bool ho_a = (v > 0) && labels[a - W] == la;
      const bool ho_b = (v + 2 < H) && labels[b + W] == la;
      wd[a] = bini_pair(f * ntau[a], f * ntau[b], x[a], x[b], ho_a ? x[a - W] : 0.f, ho_b ? x[b + W] : 0.f, ho_a,
                        ho_b, omega[a].y, ho_a ? omega[a - W].y : 0.f, ho_b ? omega[b].y : 0.f, res, k);
    }
  }
}

// 8-connectivity: omega~ (Eq. 3, the same midpoint form as the axis edges with
// tau_b - tau_a = (du / f_x, dv / f_y, 0)) and the fill weight at z~ = 0 of the
// lower-right (du, dv) = (1, 1) and lower-left (-1, 1) edge of every valid
// pixel; gamma uses f = sqrt(f_x f_y) on diagonals.  Orthographic: the sum of
// the two axis terms, signed by the step.
__device__ __forceinline__ void diag_edge(const float4 na, const float4 nb, float A, float B, int du, int persp,
                                          float fx, float fy, float& om, float& w2) {
  if (persp) {
    const float da = du * na.x / fx + na.y / fy, db = du * nb.x / fx + nb.y / fy;
    const float qv = (da * B + A * db) / (A * (2.f * B - db));
    om = (qv > -1.f) ? log1pf(qv) : logf(fabsf(1.f + qv));
    w2 = 0.5f * (fx * fy) * (A * A + B * B);
  } else {
    om = 0.5f * (du * (na.x / na.z + nb.x / nb.z) + (na.y / na.z + nb.y / nb.z));
    w2 = 0.5f * (A * A + B * B);
  }
}

__global__ void k_edge_setup_diag(const float4* __restrict__ nrm, const uint8_t* __restrict__ mask,
                                  const int* __restrict__ labels, int H, int W, int persp, float fx, float fy,
                                  float cx, float cy, float2* __restrict__ omega_d, float* __restrict__ wdr,
                                  float* __restrict__ wdl) {
  const int N = H * W;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    float2 om = make_float2(0.f, 0.f), w = make_float2(0.f, 0.f);
    const int u = a % W, v = a / W;
    if (mask[a] && v + 1 < H) {
      const float4 na = ldg4(&nrm[a]);
      const float tax = persp ? (u - cx) / fx : 0.f, tay = persp ? (v - cy) / fy : 0.f;
      const float A = persp ? (na.x * tax + na.y * tay + na.z) : na.z;
      const float tby = persp ? (v + 1 - cy) / fy : 0.f;
      const int la = labels[a];
      if (u + 1 < W && mask[a + W + 1]) {
        const float4 nb = ldg4(&nrm[a + W + 1]);
        const float B = persp ? (nb.x * ((u + 1 - cx) / fx) + nb.y * tby + nb.z) : nb.z;
        float w2;
        diag_edge(na, nb, A, B, 1, persp, fx, fy, om.x, w2);
        if (labels[a + W + 1] == la) w.x = w2;
      }
      if (u >= 1 && mask[a + W - 1]) {
        const float4 nb = ldg4(&nrm[a + W - 1]);
        const float B = persp ? (nb.x * ((u - 1 - cx) / fx) + nb.y * tby + nb.z) : nb.z;
        float w2;
        diag_edge(na, nb, A, B, -1, persp, fx, fy, om.y, w2);
        if (labels[a + W - 1] == la) w.y = w2;
      }
    }
    omega_d[a] = om;
    wdr[a] = w.x;
    wdl[a] = w.y;
  }
}

// k_diag_rhs over the 8 neighbours: the upper-left neighbour's lower-right
// edge is wdr[a - W - 1], the upper-right neighbour's lower-left edge
// wdl[a - W + 1] (0 where the edge does not exist, so raster-linear indexing
// needs no column tests).
__global__ void k_diag_rhs8(const float* __restrict__ wr, const float* __restrict__ wd,
                            const float2* __restrict__ omega, const float* __restrict__ wdr,
                            const float* __restrict__ wdl, const float2* __restrict__ omega_d, int H, int W,
                            float* __restrict__ invd, float* __restrict__ rhs) {
  const int N = H * W;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    const int v = a / W;
    const float2 om = omega[a], od = omega_d[a];
    const float wra = wr[a], wda = wd[a], wdra = wdr[a], wdla = wdl[a];
    float wl = 0.f, wu = 0.f, ol = 0.f, ou = 0.f, wul = 0.f, wur = 0.f, oul = 0.f, our = 0.f;
    if (a > 0) { wl = wr[a - 1]; ol = omega[a - 1].x; }
    if (v > 0) { wu = wd[a - W]; ou = omega[a - W].y; }
    if (a - W - 1 >= 0) { wul = wdr[a - W - 1]; oul = omega_d[a - W - 1].x; }
    if (v > 0) { wur = wdl[a - W + 1]; our = omega_d[a - W + 1].y; }
    const float d = wra + wda + wl + wu + wdra + wdla + wul + wur;
    invd[a] = d > 0.f ? 1.0f / d : 0.f;
    rhs[a] = wra * om.x + wda * om.y - wl * ol - wu * ou + wdra * od.x + wdla * od.y - wul * oul - wur * our;
  }
}

// BiNI reweighting of the diagonal edges (n_fill_irls > 1); the opposite
// neighbour of a is a - (b - a), restricted to the component (bini_pair).
__global__ void k_fill_reweight_diag(const float* __restrict__ ntau, const int* __restrict__ labels,
                                     const float* __restrict__ x, const float2* __restrict__ omega_d, int H, int W,
                                     int persp, float fx, float fy, float k, int res, float* __restrict__ wdr,
                                     float* __restrict__ wdl) {
  const int N = H * W;
  const float f = persp ? sqrtf(fx * fy) : 1.f;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    const int la = labels[a];
    const int u = a % W, v = a / W;
    if (la >= 0 && wdr[a] > 0.f) {
      const int b = a + W + 1;
      const bool ho_a = (u > 0) && (v > 0) && labels[a - W - 1] == la;
      const bool ho_b = (u + 2 < W) && (v + 2 < H) && labels[b + W + 1] == la;
      wdr[a] = bini_pair(f * ntau[a], f * ntau[b], x[a], x[b], ho_a ? x[a - W - 1] : 0.f,
                         ho_b ? x[b + W + 1] : 0.f, ho_a, ho_b, omega_d[a].x, ho_a ? omega_d[a - W - 1].x : 0.f,
                         ho_b ? omega_d[b].x : 0.f, res, k);
    }
    if (la >= 0 && wdl[a] > 0.f) {
      const int b = a + W - 1;
      const bool ho_a = (u + 1 < W) && (v > 0) && labels[a - W + 1] == la;
      const bool ho_b = (u >= 2) && (v + 2 < H) && labels[b + W - 1] == la;
      wdl[a] = bini_pair(f * ntau[a], f * ntau[b], x[a], x[b], ho_a ? x[a - W + 1] : 0.f,
                         ho_b ? x[b + W - 1] : 0.f, ho_a, ho_b, omega_d[a].y, ho_a ? omega_d[a - W + 1].y : 0.f,
                         ho_b ? omega_d[b].y : 0.f, res, k);
    }
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

// Tiles are 32 x 32 pixel blocks (the last row / column of tiles may be cut by
// the image border).  Thread t of a 256-thread CTA owns the 4 pixels of tile row
// t / 8 starting at tile column 4 (t % 8).

// Label shared by every valid pixel of a tile (-1 when several labels meet,
// -2 when the tile holds no valid pixel).
__global__ void k_tile_labels(const int* __restrict__ labels, int ntiles, int ntx, int H, int W,
                              int* __restrict__ tile_lab) {
  __shared__ int smin, smax;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    if (threadIdx.x == 0) { smin = 0x7fffffff; smax = -1; }
    __syncthreads();
    const G4 g = group_of(t, ntx, H, W);
    int mn = 0x7fffffff, mx = -1;
    for (int j = 0; j < g.nval; ++j) {
      const int l = labels[g.a + j];
      if (l >= 0) { mn = min(mn, l); mx = max(mx, l); }
    }
    atomicMin(&smin, mn);
    atomicMax(&smax, mx);
    __syncthreads();
    if (threadIdx.x == 0) tile_lab[t] = smax < 0 ? -2 : (smin == smax ? smin : -1);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// plain Jacobi-PCG (global step lengths)
// ---------------------------------------------------------------------------
struct Stencil {
  float wr, wd, wl, wu;
};

__device__ __forceinline__ Stencil load_stencil(const float* __restrict__ wr, const float* __restrict__ wd,
                                                int a, int W) {
  Stencil s;
  s.wr = wr[a];
  s.wd = wd[a];
  s.wl = (a > 0) ? wr[a - 1] : 0.f;
  s.wu = (a >= W) ? wd[a - W] : 0.f;
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

// The diagonal part of (A p)_a with 8-connectivity: the lower-right and
// lower-left edges of a and the same edges of its upper-left and upper-right
// neighbours (weights 0 where an edge does not exist).
__device__ __forceinline__ float apply_diag(const float* __restrict__ wdr, const float* __restrict__ wdl,
                                            const float* __restrict__ p, int a, int W, float pa) {
  float acc = 0.f;
  const float w0 = wdr[a], w1 = wdl[a];
  const float w2 = (a - W - 1 >= 0) ? wdr[a - W - 1] : 0.f;
  const float w3 = (a - W + 1 >= 0) ? wdl[a - W + 1] : 0.f;
  if (w0 != 0.f) acc += w0 * (pa - p[a + W + 1]);
  if (w1 != 0.f) acc += w1 * (pa - p[a + W - 1]);
  if (w2 != 0.f) acc += w2 * (pa - p[a - W - 1]);
  if (w3 != 0.f) acc += w3 * (pa - p[a - W + 1]);
  return acc;
}

template <typename Acc>
__device__ __forceinline__ void block_atomic_add(double* dst, Acc v, double* sh) {
  double t = block_sum_d((double)v, sh);
  if (threadIdx.x == 0 && t != 0.0) atomicAdd(dst, t);
}

template <typename Acc, int CONN = 4>
__global__ void k_cg_init(const float* __restrict__ wr, const float* __restrict__ wd,
                          const float* __restrict__ invd, const float* __restrict__ rhs,
                          const float* __restrict__ x, float* __restrict__ r, float* __restrict__ p, int H,
                          int W, DevState* st, const float* __restrict__ wdr = nullptr,
                          const float* __restrict__ wdl = nullptr) {
  __shared__ double sh[33];
  const int N = H * W;
  Acc rz = 0, rr = 0, bb = 0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    Stencil s = load_stencil(wr, wd, a, W);
    float ax = apply_stencil(s, x, a, W, x[a]);
    if constexpr (CONN == 8) ax += apply_diag(wdr, wdl, x, a, W, x[a]);
    float ra = rhs[a] - ax;
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

template <typename Acc, int CONN = 4>
__global__ void k_cg_spmv(const float* __restrict__ wr, const float* __restrict__ wd,
                          const float* __restrict__ p, float* __restrict__ q, int H, int W, DevState* st,
                          const float* __restrict__ wdr = nullptr, const float* __restrict__ wdl = nullptr) {
  __shared__ double sh[33];
  if (*(volatile int*)&st->cg_done) return;
  const int N = H * W;
  Acc pap = 0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    Stencil s = load_stencil(wr, wd, a, W);
    const float pa = p[a];
    float qa = apply_stencil(s, p, a, W, pa);
    if constexpr (CONN == 8) qa += apply_diag(wdr, wdl, p, a, W, pa);
    q[a] = qa;
    // p^T A p as the sum over edges of w (p_a - p_b)^2 (no cancellation)
    if (s.wr != 0.f) { float d = pa - p[a + 1]; pap += (Acc)(s.wr * d * d); }
    if (s.wd != 0.f) { float d = pa - p[a + W]; pap += (Acc)(s.wd * d * d); }
    if constexpr (CONN == 8) {
      const float w0 = wdr[a], w1 = wdl[a];
      if (w0 != 0.f) { float d = pa - p[a + W + 1]; pap += (Acc)(w0 * d * d); }
      if (w1 != 0.f) { float d = pa - p[a + W - 1]; pap += (Acc)(w1 * d * d); }
    }
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
// batched persistent Jacobi-PCG over active tiles
// ---------------------------------------------------------------------------
// Per-component state (doubles, Kc each): 0,1 rz of iteration parity; 2,3 p^T A p;
// 4,5 rz_new; 6,7 r^T r; 8 b^T b; 9 sum x; 10 count; with a warm start also
// 11 x0^T b, 12 x0^T A x0, 13 the component's scale of x0.
// Per-component ints: [0, 2 Kc) active flag per parity; [2 Kc, 3 Kc) iterations.
// Iteration k (parity P = k & 1, Q = P ^ 1), on the tiles of list Q (active at k-1):
//  phase 1: deferred update x += alpha_{k-1} p_{k-1}; for components still active
//           p_k = D^-1 r + beta_k p_{k-1} (own pixels and stencil neighbours; a
//           neighbour joined by a nonzero weight is in the same component, so it
//           shares beta), q = A p_k, p_k^T A p_k; tiles with an active pixel go to
//           list P.  One thread per component moves rz_new_{k-1} into rz_k, sets
//           the flag of iteration k and clears the accumulators of parity P.
//  phase 2: alpha_k = rz_k / p^T A p; r -= alpha_k q; r^T D^-1 r and r^T r.
// A bounded grid barrier separates the phases.  Per-component sums: a tile whose
// valid pixels share one label is reduced by the CTA (one atomic per value);
// otherwise runs of equal labels across a warp are summed, the run totals are
// gathered per label in a shared-memory table, and the table is flushed with
// one atomic per label and value.
struct PcgArgs {
  const float* wr;
  const float* wd;
  const float* invd;
  const float* rhs;
  const int* labels;
  const int* tile_lab;
  float* x;
  float* r;
  float* pb0;
  float* pb1;
  float* q;
  double* cs;
  int* ci;
  int2* tiles;     // [2][ntiles] (tile, uniform label)
  int* ntl;        // [2] list lengths
  DevState* st;
  int N, H, W, K, Kc, ntiles, ntx, maxit;
  int warm;        // x0 comes from the warm start: scale it per component (energy-optimal)
  double tol2;
};


template <bool COMP, bool ALIGNED>
#ifndef NI_PCG_MIN_BLOCKS
#define NI_PCG_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(NI_TILE_THREADS, NI_PCG_MIN_BLOCKS) k_pcg_tiles(PcgArgs A) {
  __shared__ double sh[8 * 3 + 8];
  __shared__ int s_key[TAB_SLOTS];
  __shared__ double s_val[TAB_SLOTS * 3];
  __shared__ int s_lab[TAB_SLOTS];
  __shared__ float s_f[TAB_SLOTS * 4];
  const int Kc = A.Kc, K = A.K, W = A.W, H = A.H, N = A.N;
  double* rz = A.cs;
  double* pap = A.cs + 2 * (size_t)Kc;
  double* rzn = A.cs + 4 * (size_t)Kc;
  double* rr = A.cs + 6 * (size_t)Kc;
  double* bb = A.cs + 8 * (size_t)Kc;
  double* sx = A.cs + 9 * (size_t)Kc;
  double* xb = A.cs + 11 * (size_t)Kc;
  double* xax = A.cs + 12 * (size_t)Kc;
  double* alpha = A.cs + 13 * (size_t)Kc;
  int* act = A.ci;
  int* iters = A.ci + 2 * (size_t)Kc;
  int* err = &A.st->err;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthr = gridDim.x * blockDim.x;
  const int l8 = threadIdx.x & 7;
  const double tol2 = A.tol2;
  if (threadIdx.x < TAB_SLOTS) {
    s_key[threadIdx.x] = -1;
    s_val[threadIdx.x * 3] = s_val[threadIdx.x * 3 + 1] = s_val[threadIdx.x * 3 + 2] = 0.0;
  }
  __syncthreads();

  // ---- prologue: r = b - A x0 on every tile with a valid pixel; rz_{-1}, r^T r, b^T b
  for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
    const int ul = A.tile_lab[t];
    if (ul == -2) continue;   // no valid pixel (uniform across the CTA)
    const G4 g = group_of(t, A.ntx, H, W);
    int lab[4];
    ldlab<ALIGNED>(A.labels, g.a, g.nval, lab);
    const float4 x4 = ldg<ALIGNED>(A.x, g.a, g.nval), b4 = ldg<ALIGNED>(A.rhs, g.a, g.nval);
    const float4 id4 = ldg<ALIGNED>(A.invd, g.a, g.nval);
    const float4 wr4 = ldg<ALIGNED>(A.wr, g.a, g.nval), wd4 = ldg<ALIGNED>(A.wd, g.a, g.nval);
    float xl = __shfl_up_sync(NI_FULL, x4.w, 1), xr = __shfl_down_sync(NI_FULL, x4.x, 1);
    float wl0 = __shfl_up_sync(NI_FULL, wr4.w, 1);
    if (l8 == 0) {
      xl = (g.nval > 0 && g.col > 0) ? A.x[g.a - 1] : 0.f;
      wl0 = (g.nval > 0 && g.col > 0) ? A.wr[g.a - 1] : 0.f;
    }
    if (l8 == 7) xr = (g.nval == 4 && g.col + 4 < W) ? A.x[g.a + 4] : 0.f;
    const bool up = g.row > 0, dn = g.row + 1 < H;
    const float4 xu = up ? ldg<ALIGNED>(A.x, g.a - W, g.nval) : make_float4(0, 0, 0, 0);
    const float4 wu4 = up ? ldg<ALIGNED>(A.wd, g.a - W, g.nval) : make_float4(0, 0, 0, 0);
    const float4 xd = dn ? ldg<ALIGNED>(A.x, g.a + W, g.nval) : make_float4(0, 0, 0, 0);
    float4 r4, p0 = make_float4(0, 0, 0, 0);
    float pv[3][4];
    bool on[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float xa = f4get(x4, j);
      const float xR = j < 3 ? f4get(x4, j + 1) : xr, xL = j > 0 ? f4get(x4, j - 1) : xl;
      const float wl = j > 0 ? f4get(wr4, j - 1) : wl0;
      const float ax = f4get(wr4, j) * (xa - xR) + f4get(wd4, j) * (xa - f4get(xd, j)) + wl * (xa - xL) +
                       f4get(wu4, j) * (xa - f4get(xu, j));
      on[j] = lab[j] >= 0;
      float ra = f4get(b4, j) - ax;
      if (f4get(id4, j) == 0.f || !on[j]) ra = 0.f;
      f4set(r4, j, ra);
      if (A.warm) {   // x0^T b and x0^T A x0 of the warm start
        pv[0][j] = on[j] ? xa * f4get(b4, j) : 0.f;
        pv[1][j] = on[j] ? xa * ax : 0.f;
      } else {
        pv[0][j] = ra * ra * f4get(id4, j);
        pv[1][j] = ra * ra;
      }
      pv[2][j] = on[j] ? f4get(b4, j) * f4get(b4, j) : 0.f;
    }
    stg<ALIGNED>(A.r, g.a, g.nval, r4);
    stg<ALIGNED>(A.pb1, g.a, g.nval, p0);
    double* const dst[3] = {A.warm ? xb : rzn + Kc, A.warm ? xax : rr + Kc, bb};
    const int key = ul >= 0 ? ul : group_key(lab, on);
    float v[3];
    group_values<3>(key, lab, on, pv, dst, v);
    tile_accum<COMP, 3>(ul, key == -2 ? -1 : key, v, dst, s_key, s_val, sh);
    if (threadIdx.x == 0) {
      const int pos = atomicAdd(&A.ntl[1], 1);
      A.tiles[(size_t)A.ntiles + pos] = make_int2(t, ul);
    }
  }
  if (!grid_barrier(&A.st->bar, err)) return;
  if (A.warm) {
    // Warm start: scale the start vector per component by the minimiser of the
    // energy of alpha * x0, alpha = x0^T b / x0^T A x0, so that the start's
    // A-norm error never exceeds that of x0 = 0 (alpha = 0 is the cold start).
    for (int c = gtid; c < K; c += gthr) {
      const double al = (xax[c] > 0.0 && xb[c] > 0.0) ? xb[c] / xax[c] : 0.0;
      alpha[c] = al;
      if (al == 0.0 && bb[c] > 0.0) atomicAdd(&A.st->warm_fallbacks, 1);
    }
    if (!grid_barrier(&A.st->bar, err)) return;
    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
      const int ul = A.tile_lab[t];
      if (ul == -2) continue;
      const G4 g = group_of(t, A.ntx, H, W);
      int lab[4];
      ldlab<ALIGNED>(A.labels, g.a, g.nval, lab);
      float4 x4 = ldg<ALIGNED>(A.x, g.a, g.nval), r4 = ldg<ALIGNED>(A.r, g.a, g.nval);
      const float4 b4 = ldg<ALIGNED>(A.rhs, g.a, g.nval), id4 = ldg<ALIGNED>(A.invd, g.a, g.nval);
      float pv[2][4];
      bool on[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        on[j] = lab[j] >= 0;
        const float al = on[j] ? (float)alpha[lab[j]] : 0.f;
        f4set(x4, j, al * f4get(x4, j));
        // r = b - A (al x0) = (1 - al) b + al (b - A x0)
        float ra = (1.f - al) * f4get(b4, j) + al * f4get(r4, j);
        if (f4get(id4, j) == 0.f || !on[j]) ra = 0.f;
        f4set(r4, j, ra);
        pv[0][j] = ra * ra * f4get(id4, j);
        pv[1][j] = ra * ra;
      }
      stg<ALIGNED>(A.x, g.a, g.nval, x4);
      stg<ALIGNED>(A.r, g.a, g.nval, r4);
      double* const dst[2] = {rzn + Kc, rr + Kc};
      const int key = ul >= 0 ? ul : group_key(lab, on);
      float v[2];
      group_values<2>(key, lab, on, pv, dst, v);
      tile_accum<COMP, 2>(ul, key == -2 ? -1 : key, v, dst, s_key, s_val, sh);
    }
    if (!grid_barrier(&A.st->bar, err)) return;
  }

  for (int k = 0;; ++k) {
    const int P = k & 1, Q = P ^ 1;
    const bool last = k >= A.maxit;
    // ---- phase 1: per-component bookkeeping
    for (int c = gtid; c < K; c += gthr) {
      const int wasc = (k > 0) && act[(size_t)Q * Kc + c];
      const int nowc = (k == 0 || wasc) && bb[c] > 0.0 && rr[(size_t)Q * Kc + c] > tol2 * bb[c];
      if (last) {
        if (nowc) {
          atomicAdd(&A.st->fill_unconv, 1);
          atomicOr(err, NI_DEV_ERR_FILL_NOCONV);
        }
        act[(size_t)P * Kc + c] = 0;
      } else {
        act[(size_t)P * Kc + c] = nowc;
        if (nowc) {
          iters[c] += 1;
          rz[(size_t)P * Kc + c] = rzn[(size_t)Q * Kc + c];
        }
      }
      rzn[(size_t)P * Kc + c] = 0.0;
      rr[(size_t)P * Kc + c] = 0.0;
    }
    // ---- phase 1: tiles active at k-1
    const int nq = *(volatile int*)&A.ntl[Q];
    const float* pold = Q ? A.pb1 : A.pb0;
    float* pnew = P ? A.pb1 : A.pb0;
    for (int i = blockIdx.x; i < nq; i += gridDim.x) {
      const int2 te = A.tiles[(size_t)Q * A.ntiles + i];
      const int t = te.x, ul = te.y;
      const G4 g = group_of(t, A.ntx, H, W);
      int lab[4];
      if (ul >= 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) lab[j] = j < g.nval ? ul : -1;
      } else {
        ldlab<ALIGNED>(A.labels, g.a, g.nval, lab);
      }
      // per-component scalars once per label of the tile: alpha_{k-1} (deferred
      // x update), beta_k, active at k, active at k-1
      auto scalars1 = [&](int c, float* o) {
        const bool was = (k > 0) && act[(size_t)Q * Kc + c];
        const bool nw = !last && (k == 0 || was) && bb[c] > 0.0 && rr[(size_t)Q * Kc + c] > tol2 * bb[c];
        const double pp = pap[(size_t)Q * Kc + c], rzo = rz[(size_t)Q * Kc + c];
        o[0] = (was && pp > 0.0) ? (float)(rzo / pp) : 0.f;
        o[1] = (nw && k > 0 && rzo > 0.0) ? (float)(rzn[(size_t)Q * Kc + c] / rzo) : 0.f;
        o[2] = nw ? 1.f : 0.f;
        o[3] = was ? 1.f : 0.f;
      };
      // own-pixel operands, issued before the scalar cache so their latency overlaps it
      const float4 po4 = ldg<ALIGNED>(pold, g.a, g.nval);
      float4 x4 = ldg<ALIGNED>(A.x, g.a, g.nval);
      const float4 r4 = ldg<ALIGNED>(A.r, g.a, g.nval), id4 = ldg<ALIGNED>(A.invd, g.a, g.nval);
      const float4 wr4 = ldg<ALIGNED>(A.wr, g.a, g.nval), wd4 = ldg<ALIGNED>(A.wd, g.a, g.nval);
      int sl[4];
      tile_slots(ul, lab, sl, s_lab);
      if (threadIdx.x < TAB_SLOTS && s_lab[threadIdx.x] >= 0) scalars1(s_lab[threadIdx.x], &s_f[threadIdx.x * 4]);
      __syncthreads();
      float alpha[4], beta[4];
      bool now[4];
      int any_was = 0, any_now = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float o[4] = {0.f, 0.f, 0.f, 0.f};
        if (sl[j] >= 0) {
          o[0] = s_f[sl[j] * 4]; o[1] = s_f[sl[j] * 4 + 1]; o[2] = s_f[sl[j] * 4 + 2]; o[3] = s_f[sl[j] * 4 + 3];
        } else if (sl[j] == -2) {
          scalars1(lab[j], o);
        }
        alpha[j] = o[0];
        beta[j] = o[1];
        now[j] = o[2] != 0.f;
        any_was |= o[3] != 0.f;
        any_now |= now[j];
      }
      if (any_was) {
        x4.x += alpha[0] * po4.x;
        x4.y += alpha[1] * po4.y;
        x4.z += alpha[2] * po4.z;
        x4.w += alpha[3] * po4.w;
        stg<ALIGNED>(A.x, g.a, g.nval, x4);
      }
      if (!__syncthreads_or(any_now)) continue;
      // p_k at own pixels
      float4 pn;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        f4set(pn, j, now[j] ? f4get(r4, j) * f4get(id4, j) + beta[j] * f4get(po4, j) : 0.f);
      // neighbours: left/right through the 8 lanes of a tile row, row ends from memory
      float pl = __shfl_up_sync(NI_FULL, pn.w, 1), pr = __shfl_down_sync(NI_FULL, pn.x, 1);
      float wl0 = __shfl_up_sync(NI_FULL, wr4.w, 1);
      if (l8 == 0) {
        const int a = g.a - 1;
        wl0 = (g.nval > 0 && g.col > 0) ? A.wr[a] : 0.f;
        pl = (wl0 != 0.f && now[0]) ? A.r[a] * A.invd[a] + beta[0] * pold[a] : 0.f;
      }
      if (l8 == 7) {
        const int a = g.a + 4;
        pr = (g.nval == 4 && g.col + 4 < W && wr4.w != 0.f && now[3]) ? A.r[a] * A.invd[a] + beta[3] * pold[a]
                                                                      : 0.f;
      }
      float4 pu = make_float4(0, 0, 0, 0), pd = make_float4(0, 0, 0, 0), wu4 = make_float4(0, 0, 0, 0);
      if (g.row > 0) {
        wu4 = ldg<ALIGNED>(A.wd, g.a - W, g.nval);
        const float4 ru = ldg<ALIGNED>(A.r, g.a - W, g.nval), iu = ldg<ALIGNED>(A.invd, g.a - W, g.nval);
        const float4 pu0 = ldg<ALIGNED>(pold, g.a - W, g.nval);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          f4set(pu, j, (now[j] && f4get(wu4, j) != 0.f) ? f4get(ru, j) * f4get(iu, j) + beta[j] * f4get(pu0, j)
                                                          : 0.f);
      }
      if (g.row + 1 < H) {
        const float4 rd = ldg<ALIGNED>(A.r, g.a + W, g.nval), idd = ldg<ALIGNED>(A.invd, g.a + W, g.nval);
        const float4 pd0 = ldg<ALIGNED>(pold, g.a + W, g.nval);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          f4set(pd, j, (now[j] && f4get(wd4, j) != 0.f) ? f4get(rd, j) * f4get(idd, j) + beta[j] * f4get(pd0, j)
                                                          : 0.f);
      }
      float4 q4;
      float pv[1][4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float pa = f4get(pn, j);
        const float pR = j < 3 ? f4get(pn, j + 1) : pr, pL = j > 0 ? f4get(pn, j - 1) : pl;
        const float wl = j > 0 ? f4get(wr4, j - 1) : wl0;
        const float dR = pa - pR, dD = pa - f4get(pd, j);
        const float qa = f4get(wr4, j) * dR + f4get(wd4, j) * dD + wl * (pa - pL) + f4get(wu4, j) * (pa - f4get(pu, j));
        f4set(q4, j, now[j] ? qa : 0.f);
        pv[0][j] = now[j] ? f4get(wr4, j) * dR * dR + f4get(wd4, j) * dD * dD : 0.f;
      }
      stg<ALIGNED>(pnew, g.a, g.nval, pn);
      stg<ALIGNED>(A.q, g.a, g.nval, q4);
      double* const dst[1] = {pap + (size_t)P * Kc};
      const int key = ul >= 0 ? ul : group_key(lab, now);
      float v[1];
      group_values<1>(key, lab, now, pv, dst, v);
      tile_accum<COMP, 1>(ul, key == -2 ? -1 : key, v, dst, s_key, s_val, sh);
      if (threadIdx.x == 0) {
        const int pos = atomicAdd(&A.ntl[P], 1);
        A.tiles[(size_t)P * A.ntiles + pos] = make_int2(t, ul);
      }
    }
    if (!grid_barrier(&A.st->bar, err)) return;
    if (*(volatile int*)&A.ntl[P] == 0) break;
    // ---- phase 2: alpha_k, residual update, per-component r^T D^-1 r and r^T r
    for (int c = gtid; c < K; c += gthr) pap[(size_t)Q * Kc + c] = 0.0;
    if (gtid == 0) A.ntl[Q] = 0;
    const int np = *(volatile int*)&A.ntl[P];
    for (int i = blockIdx.x; i < np; i += gridDim.x) {
      const int2 te = A.tiles[(size_t)P * A.ntiles + i];
      const int t = te.x, ul = te.y;
      const G4 g = group_of(t, A.ntx, H, W);
      int lab[4];
      if (ul >= 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) lab[j] = j < g.nval ? ul : -1;
      } else {
        ldlab<ALIGNED>(A.labels, g.a, g.nval, lab);
      }
      float4 r4 = ldg<ALIGNED>(A.r, g.a, g.nval);
      const float4 q4 = ldg<ALIGNED>(A.q, g.a, g.nval), id4 = ldg<ALIGNED>(A.invd, g.a, g.nval);
      auto scalars2 = [&](int c, float* o) {
        const bool on = act[(size_t)P * Kc + c];
        const double pp = pap[(size_t)P * Kc + c];
        o[0] = (on && pp > 0.0) ? (float)(rz[(size_t)P * Kc + c] / pp) : 0.f;
        o[1] = on ? 1.f : 0.f;
      };
      int sl[4];
      tile_slots(ul, lab, sl, s_lab);
      if (threadIdx.x < TAB_SLOTS && s_lab[threadIdx.x] >= 0) scalars2(s_lab[threadIdx.x], &s_f[threadIdx.x * 4]);
      __syncthreads();
      float alpha[4];
      bool on[4];
      int any = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float o[2] = {0.f, 0.f};
        if (sl[j] >= 0) {
          o[0] = s_f[sl[j] * 4]; o[1] = s_f[sl[j] * 4 + 1];
        } else if (sl[j] == -2) {
          scalars2(lab[j], o);
        }
        alpha[j] = o[0];
        on[j] = o[1] != 0.f;
        any |= on[j];
      }
      float pv[2][4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float ra = f4get(r4, j);
        if (on[j]) ra -= alpha[j] * f4get(q4, j);
        f4set(r4, j, ra);
        pv[0][j] = on[j] ? ra * ra * f4get(id4, j) : 0.f;
        pv[1][j] = on[j] ? ra * ra : 0.f;
      }
      if (any) stg<ALIGNED>(A.r, g.a, g.nval, r4);
      double* const dst[2] = {rzn + (size_t)P * Kc, rr + (size_t)P * Kc};
      const int key = ul >= 0 ? ul : group_key(lab, on);
      float v[2];
      group_values<2>(key, lab, on, pv, dst, v);
      tile_accum<COMP, 2>(ul, key == -2 ? -1 : key, v, dst, s_key, s_val, sh);
    }
    if (!grid_barrier(&A.st->bar, err)) return;
  }
  // ---- epilogue: zero mean per component (the gauge of CG from 0), statistics
  for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
    const int ul = A.tile_lab[t];
    if (ul == -2) continue;
    const G4 g = group_of(t, A.ntx, H, W);
    int lab[4];
    ldlab<ALIGNED>(A.labels, g.a, g.nval, lab);
    const float4 x4 = ldg<ALIGNED>(A.x, g.a, g.nval);
    float pv[2][4];
    bool on[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      on[j] = lab[j] >= 0;
      pv[0][j] = on[j] ? f4get(x4, j) : 0.f;
      pv[1][j] = on[j] ? 1.f : 0.f;
    }
    double* const dst[2] = {sx, sx + Kc};
    const int key = ul >= 0 ? ul : group_key(lab, on);
    float v[2];
    group_values<2>(key, lab, on, pv, dst, v);
    tile_accum<true, 2>(ul, key == -2 ? -1 : key, v, dst, s_key, s_val, sh);
  }
  if (!grid_barrier(&A.st->bar, err)) return;
  for (int a = gtid; a < N; a += gthr) {
    const int c = A.labels[a];
    if (c >= 0) {
      const double cnt = sx[(size_t)Kc + c];
      if (cnt > 0) A.x[a] = (float)((double)A.x[a] - sx[c] / cnt);
    }
  }
  for (int c = gtid; c < K; c += gthr) {
    atomicMax(&A.st->fill_iters, iters[c]);
    if (iters[c] > 0)
      atomicAdd(&A.st->fill_px_iters, (unsigned long long)iters[c] * (unsigned long long)sx[(size_t)Kc + c]);
  }
}

ni_status fill_setup_launch(ni_handle* h, cudaStream_t s) {
  const int N = h->N;
  k_edge_setup<<<grid_px(h, N), 256, 0, s>>>(h->normals, h->mask, h->labels, h->H, h->W, h->persp, h->fx, h->fy,
                                               h->cx, h->cy, h->omega, h->ntau, h->wr, h->wd); NI_COUNT(h);
  if (h->cfg.connectivity == 8) {
    k_edge_setup_diag<<<grid_px(h, N), 256, 0, s>>>(h->normals, h->mask, h->labels, h->H, h->W, h->persp, h->fx,
                                                      h->fy, h->cx, h->cy, h->omega_d, h->wdr, h->wdl); NI_COUNT(h);
    k_diag_rhs8<<<grid_px(h, N), 256, 0, s>>>(h->wr, h->wd, h->omega, h->wdr, h->wdl, h->omega_d, h->H, h->W,
                                                h->invd, h->b); NI_COUNT(h);
  } else {
    k_diag_rhs<<<grid_px(h, N), 256, 0, s>>>(h->wr, h->wd, h->omega, h->H, h->W, h->invd, h->b); NI_COUNT(h);
  }
  k_tile_labels<<<grid_px(h, (long long)h->ntiles * 256), 256, 0, s>>>(h->labels, h->ntiles, h->ntx, h->H, h->W,
                                                                        h->tile_lab); NI_COUNT(h);
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
  const bool c8 = h->cfg.connectivity == 8;
  const float *wdr = h->wdr, *wdl = h->wdl;
  if (c8) {
    if (f64) k_cg_init<double, 8><<<g, 256, 0, s>>>(h->wr, h->wd, h->invd, h->b, h->x, h->r, h->p, H, W, h->st, wdr, wdl);
    else k_cg_init<float, 8><<<g, 256, 0, s>>>(h->wr, h->wd, h->invd, h->b, h->x, h->r, h->p, H, W, h->st, wdr, wdl);
  } else {
    if (f64) k_cg_init<double><<<g, 256, 0, s>>>(h->wr, h->wd, h->invd, h->b, h->x, h->r, h->p, H, W, h->st);
    else k_cg_init<float><<<g, 256, 0, s>>>(h->wr, h->wd, h->invd, h->b, h->x, h->r, h->p, H, W, h->st);
  }
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
    if (c8) {
      if (f64) k_cg_spmv<double, 8><<<g, 256, 0, cs>>>(h->wr, h->wd, h->p, h->q, H, W, h->st, wdr, wdl);
      else k_cg_spmv<float, 8><<<g, 256, 0, cs>>>(h->wr, h->wd, h->p, h->q, H, W, h->st, wdr, wdl);
    } else {
      if (f64) k_cg_spmv<double><<<g, 256, 0, cs>>>(h->wr, h->wd, h->p, h->q, H, W, h->st);
      else k_cg_spmv<float><<<g, 256, 0, cs>>>(h->wr, h->wd, h->p, h->q, H, W, h->st);
    }
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

template <bool FP64, bool AL>
static void* pcg_fn() {
  return (void*)k_pcg_tiles<FP64, AL>;
}

__global__ void k_clear_fill_flags(DevState* st) {
  st->fill_unconv = 0;
  st->err &= ~NI_DEV_ERR_FILL_NOCONV;
}

static ni_status batched_solve(ni_handle* h, cudaStream_t s, bool allow_warm = true) {
  const bool f64 = h->cfg.precision == 0;
  const bool al = (h->W % 4) == 0;
  void* fn = f64 ? (al ? pcg_fn<true, true>() : pcg_fn<true, false>())
                 : (al ? pcg_fn<false, true>() : pcg_fn<false, false>());
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NI_TILE_THREADS, 0);
  if (per_sm < 1) return ni_fail(h, NI_ERR_CUDA, "batched PCG: kernel cannot be resident");
  const int want = h->cfg.ctas_per_sm > 0 ? h->cfg.ctas_per_sm : 4;   // CTAs per SM (tuned)
  int grid = h->num_sms * std::min(per_sm, want);
  grid = std::max(1, std::min(grid, h->ntiles));
  cudaMemsetAsync(h->cacc, 0, sizeof(double) * 14 * (size_t)h->Kcap, s);
  cudaMemsetAsync(h->cflag, 0, sizeof(int) * 3 * (size_t)h->Kcap, s);
  cudaMemsetAsync(&h->st->bar, 0, sizeof(GridBar), s);
  int* ntl = reinterpret_cast<int*>(&h->st->bar2);
  cudaMemsetAsync(ntl, 0, sizeof(GridBar), s);
  PcgArgs a;
  a.wr = h->wr; a.wd = h->wd; a.invd = h->invd; a.rhs = h->b; a.labels = h->labels; a.tile_lab = h->tile_lab;
  a.x = h->x; a.r = h->r; a.pb0 = h->p; a.pb1 = h->p2; a.q = h->q;
  a.cs = h->cacc; a.ci = h->cflag; a.tiles = reinterpret_cast<int2*>(h->tiles); a.ntl = ntl; a.st = h->st;
  a.N = h->N; a.H = h->H; a.W = h->W; a.K = h->K_host; a.Kc = h->Kcap; a.ntiles = h->ntiles; a.ntx = h->ntx;
  a.maxit = h->cfg.cg_maxit; a.tol2 = h->cfg.cg_rtol * h->cfg.cg_rtol;
  a.warm = (allow_warm && h->cfg.warm_start) ? 1 : 0;
  void* args[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(NI_TILE_THREADS), args, 0, s);
  NI_COUNT(h);
  return ni_cuda_check(h, e, "batched PCG launch");
}

ni_status fill_solve_launch(ni_handle* h, cudaStream_t s) {
  ni_status rc = project_rhs(h, h->b, s);
  if (rc != NI_OK) return rc;
  for (int sweep = 0; sweep < std::max(1, h->cfg.n_fill_irls); ++sweep) {
    if (sweep > 0) {
      k_fill_reweight<<<grid_px(h, h->N), 256, 0, s>>>(h->ntau, h->labels, h->x, h->omega, h->H, h->W, h->persp,
                                                        h->fx, h->fy, (float)h->cfg.k, h->cfg.bini_residual, h->wr,
                                                        h->wd); NI_COUNT(h);
      if (h->cfg.connectivity == 8) {
        k_fill_reweight_diag<<<grid_px(h, h->N), 256, 0, s>>>(h->ntau, h->labels, h->x, h->omega_d, h->H, h->W,
                                                                h->persp, h->fx, h->fy, (float)h->cfg.k,
                                                                h->cfg.bini_residual, h->wdr, h->wdl);
        NI_COUNT(h);
        k_diag_rhs8<<<grid_px(h, h->N), 256, 0, s>>>(h->wr, h->wd, h->omega, h->wdr, h->wdl, h->omega_d, h->H,
                                                       h->W, h->invd, h->b); NI_COUNT(h);
      } else {
        k_diag_rhs<<<grid_px(h, h->N), 256, 0, s>>>(h->wr, h->wd, h->omega, h->H, h->W, h->invd, h->b); NI_COUNT(h);
      }
      rc = project_rhs(h, h->b, s);
      if (rc != NI_OK) return rc;
    }
    cudaMemsetAsync(&h->st->fill_iters, 0, 2 * sizeof(int), s);
    cudaMemsetAsync(&h->st->fill_px_iters, 0, sizeof(unsigned long long), s);
    cudaEventRecord(h->ev[5], s);
    if (h->cfg.batched && h->cfg.precond == 1) {
      rc = mg_solve_launch(h, s);
      if (rc == NI_OK) {
        // components the multigrid PCG left above the tolerance (float32 can stall
        // it on rare components): Jacobi PCG continues them from where they are
        cudaMemcpyAsync(&h->st_host->fill_unconv, &h->st->fill_unconv, sizeof(int), cudaMemcpyDeviceToHost, s);
        rc = ni_cuda_check(h, cudaStreamSynchronize(s), "multigrid PCG");
        if (rc == NI_OK && h->st_host->fill_unconv > 0) {
          h->fill_fallbacks += h->st_host->fill_unconv;
          k_clear_fill_flags<<<1, 1, 0, s>>>(h->st); NI_COUNT(h);
          rc = batched_solve(h, s, false);
        }
      }
      cudaEventRecord(h->ev[6], s);
    } else if (h->cfg.batched) {
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
