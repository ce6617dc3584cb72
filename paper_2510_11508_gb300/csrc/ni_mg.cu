// Fill solve with a multigrid-preconditioned CG (row a4, precond = 1).
//
// The fill systems of Eq. 10 are weighted graph Laplacians of the pixel grid,
// one block per component.  Jacobi-PCG needs a number of iterations that grows
// with the component's diameter (thousands on the large maps).  Here the
// preconditioner is one symmetric V-cycle of an aggregation multigrid built on
// the grid itself:
//
//   * level l+1 aggregates 2x2 cells of level l.  The coarse cell takes the
//     label of the first valid cell of its block (raster order); block cells of
//     another label are not aggregated (zero row of the prolongation), so every
//     coarse cell, and every coarse edge, stays inside one component and the
//     preconditioner is block-diagonal per component like the system;
//   * the coarse operator is the Galerkin product P^T A P of the piecewise-
//     constant prolongation: a 5-point stencil again, with edge weights summed
//     over the fine edges between two aggregates and the diagonal d_I = the
//     weights of all edges leaving the aggregate plus its cells' own diagonal
//     excess (sums of non-negative terms only);
//   * smoothing: one damped Jacobi step (weight om, default 0.9) before and
//     after the coarse correction, the coarse correction scaled by sc (default
//     1; over-correction sc > 1 cut the iterations on some maps but left single
//     components converging at a crawl in float32 on others); the coarsest level
//     (<= 4 cells) takes a few Jacobi steps.  The cycle is a fixed symmetric positive definite
//     operator, so CG with it converges like CG on a well-conditioned system.
//
// One cooperative persistent launch runs the whole solve.  Per iteration k:
//   V-cycle on r_k (restriction of level 0 by all CTAs, of the coarse levels
//   by as many CTAs as their size calls for, with barriers among those only;
//   the last levels, at most 512 cells, in CTA 0's shared memory), z_k and
//   r_k^T z_k;
//   phase A: p_k = z_k + beta_k p_{k-1}, q = A p_k, p^T A p per component;
//   phase B: x += alpha p, r -= alpha q, r^T r per component.
// Step lengths, convergence masks and iteration counts are per component, as
// in the Jacobi kernel; level-0 passes walk the list of 32x32 tiles that hold
// a valid pixel and skip tiles of converged components.
#include <algorithm>

#include "ni_internal.cuh"
#include "ni_tile.cuh"

struct MgArgs {
  const float* wr;
  const float* wd;
  const float* invd;
  const float* rhs;
  const int* labels;
  const int* tile_lab;
  const uint8_t* inc0;     // level-0 cell aggregated into its level-1 cell
  float* x;
  float* r;
  float* pb0;
  float* pb1;
  float* q;
  float* z;
  // coarse levels 1..L in pools; level l starts at loff[l]
  int* clab;
  float* cwr;
  float* cwd;
  float* cinvd;
  float* cb;
  float* ce;
  const uint8_t* cinc;
  int L, Lc;               // levels Lc..L live in CTA 0's shared memory
  int lh[NI_MG_MAX_LEVELS + 1], lw[NI_MG_MAX_LEVELS + 1];
  long long loff[NI_MG_MAX_LEVELS + 1];
  int smo[NI_MG_MAX_LEVELS + 1];   // offset of level l >= Lc in the shared arrays
  int pd[NI_MG_MAX_LEVELS + 1];    // CTAs of the restriction from level l (l < Lc)
  int pu[NI_MG_MAX_LEVELS + 1];    // CTAs of the prolongation to level l (l < Lc)
  GridBar* mbar;                   // [0..L]: after restrictions, [NI_MG_MAX_LEVELS+1+l]: before prolongations
  double* cs;
  int* ci;
  int2* tiles;             // list of tiles with a valid pixel (tile, uniform label)
  int2* tact;              // [2][ntiles]: tiles with an active pixel at iteration k, by parity of k
  int* ntl;                // [0] list length, [2..3] active components, [4..5] active tiles, by parity
  int per;                 // coarse cells per CTA of a coarse pass
  DevState* st;
  int N, H, W, K, Kc, ntiles, ntx, maxit, warm, ncs, project;
  float om, sc;
  double tol2;
};

// view of one coarse level
struct Lv {
  const int* lab;
  const float* wr;
  const float* wd;
  const float* invd;
  float* b;
  float* e;
  const uint8_t* inc;
  int H, W;
};

__device__ __forceinline__ Lv coarse_level(const MgArgs& A, int l) {
  Lv v;
  const long long o = A.loff[l];
  v.lab = A.clab + o; v.wr = A.cwr + o; v.wd = A.cwd + o; v.invd = A.cinvd + o;
  v.b = A.cb + o; v.e = A.ce + o; v.inc = A.cinc + o;
  v.H = A.lh[l]; v.W = A.lw[l];
  return v;
}

#define MG_SMEM_CELLS 512
#define NI_MG_MAXIT 2000

// the small levels, held in shared memory by CTA 0
struct MgSmem {
  int lab[MG_SMEM_CELLS];
  float wr[MG_SMEM_CELLS], wd[MG_SMEM_CELLS], invd[MG_SMEM_CELLS], b[MG_SMEM_CELLS], e[MG_SMEM_CELLS];
  uint8_t inc[MG_SMEM_CELLS];
};

__device__ __forceinline__ Lv smem_level(const MgArgs& A, MgSmem& S, int l) {
  Lv v;
  const int o = A.smo[l];
  v.lab = S.lab + o; v.wr = S.wr + o; v.wd = S.wd + o; v.invd = S.invd + o;
  v.b = S.b + o; v.e = S.e + o; v.inc = S.inc + o;
  v.H = A.lh[l]; v.W = A.lw[l];
  return v;
}

// pre-smoothed value plus the scaled coarse correction at cell (y, x)
// (all four loads issued together; (y, x) must lie inside the level)
__device__ __forceinline__ float zc_at(const float* __restrict__ b, const float* __restrict__ invd,
                                       const uint8_t* __restrict__ inc, const float* __restrict__ ec, int W,
                                       int Wc, int y, int x, float om, float sc, float mu) {
  const int a = y * W + x;
  const float bb = b[a], id = invd[a], e = ec[(y >> 1) * Wc + (x >> 1)];
  const bool ic = inc[a] != 0;
  return om * id * (bb - mu) + (ic ? sc * e : 0.f);
}

// Restriction of the 2x2 block (cy, cx) of a level: the sum over its aggregated
// cells of the residual after one damped Jacobi step from zero,
// (b_a - mu) - sum_n w_an (y_a - y_n), y = om D^-1 (b - mu).  Every load of the
// 4x4 window (b, 1/d), the 2x3 right and 3x2 down weights and the flags is
// issued before any arithmetic (one round trip instead of a chain); terms of
// absent edges are selected away, so unwritten values never propagate.
__device__ __forceinline__ float restrict_block(const float* __restrict__ b, const float* __restrict__ invd,
                                                const float* __restrict__ wr, const float* __restrict__ wd,
                                                const uint8_t* __restrict__ inc, int H, int W, int cy, int cx,
                                                float om, float mu) {
  const int y0 = 2 * cy, x0 = 2 * cx;
  float yv[4][4], bv[2][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      yv[i][j] = 0.f;
      if ((i == 0 || i == 3) && (j == 0 || j == 3)) continue;
      const int y = y0 - 1 + i, x = x0 - 1 + j;
      const bool in = y >= 0 && y < H && x >= 0 && x < W;
      const int a = in ? y * W + x : 0;
      const float bb = in ? b[a] : 0.f, id = in ? invd[a] : 0.f;
      yv[i][j] = om * id * (bb - mu);
      if (i >= 1 && i <= 2 && j >= 1 && j <= 2) bv[i - 1][j - 1] = bb - mu;
    }
  float wrv[2][3], wdv[3][2];
  bool incv[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int y = y0 + i, x = x0 - 1 + j;
      wrv[i][j] = (y < H && x >= 0 && x < W) ? wr[y * W + x] : 0.f;
    }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int y = y0 - 1 + i, x = x0 + j;
      wdv[i][j] = (y >= 0 && y < H && x < W) ? wd[y * W + x] : 0.f;
    }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int y = y0 + i, x = x0 + j;
      incv[i][j] = (y < H && x < W) ? inc[y * W + x] != 0 : false;
    }
  float s = 0.f;
#pragma unroll
  for (int di = 0; di < 2; ++di)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj) {
      const int i = di + 1, j = dj + 1;
      const float ya = yv[i][j];
      const float wR = wrv[di][dj + 1], wL = wrv[di][dj], wD = wdv[di + 1][dj], wU = wdv[di][dj];
      float t = 0.f;
      t += wR != 0.f ? wR * (ya - yv[i][j + 1]) : 0.f;
      t += wL != 0.f ? wL * (ya - yv[i][j - 1]) : 0.f;
      t += wD != 0.f ? wD * (ya - yv[i + 1][j]) : 0.f;
      t += wU != 0.f ? wU * (ya - yv[i - 1][j]) : 0.f;
      s += incv[di][dj] ? bv[di][dj] - t : 0.f;
    }
  return s;
}

// restriction of level f (>= 1) to level c over cells i0, i0 + stride, ...;
// cells of converged components (act) get 0 without reading their window
__device__ void mg_down(const Lv& f, const Lv& c, float om, int i0, int stride, const int* act) {
  const int nc = c.H * c.W;
  for (int I = i0; I < nc; I += stride) {
    const int cy = I / c.W, cx = I - cy * c.W;
    const int lc = c.lab[I];
    const bool on = lc >= 0 && (act == nullptr || act[lc]);
    c.b[I] = on ? restrict_block(f.b, f.invd, f.wr, f.wd, f.inc, f.H, f.W, cy, cx, om, 0.f) : 0.f;
  }
}

// prolongation and post-smoothing of cell (y, x) of level f: with
// zc = om D^-1 b + sc P e_c, e_f = zc + om D^-1 (b - A zc); all loads first
__device__ __forceinline__ float prolong_cell(const float* __restrict__ b, const float* __restrict__ invd,
                                              const float* __restrict__ wr, const float* __restrict__ wd,
                                              const uint8_t* __restrict__ inc, const float* __restrict__ ec,
                                              int H, int W, int Wc, int y, int x, float om, float sc,
                                              float mu) {
  const int dy[5] = {0, 0, 0, -1, 1}, dx[5] = {0, 1, -1, 0, 0};
  float zc[5], ba = 0.f, ida = 0.f;
#pragma unroll
  for (int n = 0; n < 5; ++n) {
    const int yy = y + dy[n], xx = x + dx[n];
    const bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
    const int a = in ? yy * W + xx : 0;
    const float bb = in ? b[a] - mu : 0.f, id = in ? invd[a] : 0.f;
    const bool ic = in && inc[a] != 0;
    const float e = in ? ec[(yy >> 1) * Wc + (xx >> 1)] : 0.f;
    zc[n] = om * id * bb + (ic ? sc * e : 0.f);
    if (n == 0) { ba = bb; ida = id; }
  }
  const int a = y * W + x;
  const float w0 = wr[a], w1 = x > 0 ? wr[a - 1] : 0.f, w2 = wd[a], w3 = y > 0 ? wd[a - W] : 0.f;
  float t = 0.f;
  t += w0 != 0.f ? w0 * (zc[0] - zc[1]) : 0.f;
  t += w1 != 0.f ? w1 * (zc[0] - zc[2]) : 0.f;
  t += w3 != 0.f ? w3 * (zc[0] - zc[3]) : 0.f;
  t += w2 != 0.f ? w2 * (zc[0] - zc[4]) : 0.f;
  return zc[0] + om * ida * (ba - t);
}

// prolongation and post-smoothing on level f (>= 1): e_f from b_f and e_c;
// cells of converged components (act) get 0 without reading their stencil
// (no active cell reads them: coarse edges never join two components)
__device__ void mg_up(const Lv& f, const Lv& c, float om, float sc, int i0, int stride, const int* act) {
  const int n = f.H * f.W;
  for (int a = i0; a < n; a += stride) {
    const int y = a / f.W, x = a - y * f.W;
    const int la = f.lab[a];
    const bool on = la >= 0 && (act == nullptr || act[la]);
    f.e[a] = on ? prolong_cell(f.b, f.invd, f.wr, f.wd, f.inc, c.e, f.H, f.W, c.W, y, x, om, sc, 0.f) : 0.f;
  }
}

// Levels 1..NI_MG_TILE_LEVELS have cells that lie inside one 32 x 32 tile of
// the pixel grid (a level-l cell covers 2^l x 2^l pixels), so the persistent
// kernel restricts to and prolongates on them over the list of active tiles
// only: (32 >> l)^2 cells of level l per tile, one cell per thread, consecutive
// threads on consecutive cells of a tile.  A listed tile with one label (te.y
// >= 0) holds an active component, so its cells need no activity check; in a
// mixed tile each cell checks its label.  The window or stencil loads do not
// wait for that check (values of cells left out are never read through a
// nonzero weight: coarse edges never join two components).
#define NI_MG_TILE_LEVELS 5
// the tile-local levels that the persistent kernel walks by the tile list:
// levels 1 and 2 (256 and 64 cells per tile), where skipping the converged
// tiles saves the most; the smaller levels run over all their cells, on fewer
// CTAs (measured: 374 -> 346 ms fill on the 8192^2 map, unchanged on 2048^2;
// the list on levels 3 to 5 as well cost 2 ms on 2048^2)
#define NI_MG_LIST_LEVELS 2
static_assert(NI_MG_LIST_LEVELS <= NI_MG_TILE_LEVELS, "list-driven levels must be tile-local");
static_assert(NI_TILE_W == 32 && NI_TILE_H == 32, "tile-local coarse levels assume 32 x 32 tiles");

// restriction from level l into level l + 1 (<= NI_MG_TILE_LEVELS) over the n
// listed tiles, items i0, i0 + stride, ...
__device__ void mg_down_tiles(const MgArgs& A, int l, const int2* __restrict__ list, int n, const int* act,
                              int i0, int stride) {
  const Lv f = coarse_level(A, l), c = coarse_level(A, l + 1);
  const int sh = NI_MG_TILE_LEVELS - (l + 1);   // log2 of the cells per tile side
  const int side = 1 << sh;
  const long long items = (long long)n << (2 * sh);
  for (long long i = i0; i < items; i += stride) {
    const int2 te = list[i >> (2 * sh)];
    const int j = (int)(i & ((1 << (2 * sh)) - 1));
    const int ty = te.x / A.ntx, tx = te.x - ty * A.ntx;
    const int cy = (ty << sh) + (j >> sh), cx = (tx << sh) + (j & (side - 1));
    if (cy >= c.H || cx >= c.W) continue;
    const int I = cy * c.W + cx;
    const int lc = c.lab[I];
    const float v = restrict_block(f.b, f.invd, f.wr, f.wd, f.inc, f.H, f.W, cy, cx, A.om, 0.f);
    const bool on = lc >= 0 && (te.y >= 0 || act[lc]);
    c.b[I] = on ? v : 0.f;
  }
}

// CTAs of the tile-local pass on level `level`: one per A.per of its cells in
// the na active tiles, and never fewer than `floor_n`, the CTAs of the first
// pass beyond the list-driven levels, so that the CTAs of a coarser pass are
// always among those of a finer one (each partial barrier then covers every
// writer of what the next pass reads)
__device__ __forceinline__ int mg_tile_ctas(const MgArgs& A, int na, int level, int floor_n) {
  const long long items = (long long)na << (2 * (NI_MG_TILE_LEVELS - level));
  const long long n = (items + A.per - 1) / A.per;
  return (int)max((long long)floor_n, min((long long)gridDim.x, max(1LL, n)));
}

// prolongation and post-smoothing on level l (<= NI_MG_TILE_LEVELS) from l + 1
// over the n listed tiles, items i0, i0 + stride, ...
__device__ void mg_up_tiles(const MgArgs& A, int l, const int2* __restrict__ list, int n, const int* act,
                            int i0, int stride) {
  const Lv f = coarse_level(A, l), c = coarse_level(A, l + 1);
  const int sh = NI_MG_TILE_LEVELS - l;
  const int side = 1 << sh;
  const long long items = (long long)n << (2 * sh);
  for (long long i = i0; i < items; i += stride) {
    const int2 te = list[i >> (2 * sh)];
    const int j = (int)(i & ((1 << (2 * sh)) - 1));
    const int ty = te.x / A.ntx, tx = te.x - ty * A.ntx;
    const int y = (ty << sh) + (j >> sh), x = (tx << sh) + (j & (side - 1));
    if (y >= f.H || x >= f.W) continue;
    const int a = y * f.W + x;
    const int la = f.lab[a];
    const float v = prolong_cell(f.b, f.invd, f.wr, f.wd, f.inc, c.e, f.H, f.W, c.W, y, x, A.om, A.sc, 0.f);
    const bool on = la >= 0 && (te.y >= 0 || act[la]);
    f.e[a] = on ? v : 0.f;
  }
}

// CTA 0, once per launch: the constant data of levels Lc..L into shared memory
__device__ void mg_smem_load(const MgArgs& A, MgSmem& S) {
  for (int l = A.Lc; l <= A.L; ++l) {
    const Lv g = coarse_level(A, l);
    const int o = A.smo[l], n = g.H * g.W;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      S.lab[o + i] = g.lab[i];
      S.wr[o + i] = g.wr[i];
      S.wd[o + i] = g.wd[i];
      S.invd[o + i] = g.invd[i];
      S.inc[o + i] = l < A.L ? g.inc[i] : 0;
    }
  }
  __syncthreads();
}

// CTA 0, every iteration: restriction from level Lc down to L, damped Jacobi
// steps on level L (<= 4 cells), prolongation and smoothing back up to Lc, all
// in shared memory; b_Lc comes from and e_Lc goes to global memory
__device__ void mg_cta_levels(const MgArgs& A, MgSmem& S, const int* act) {
  const Lv g = coarse_level(A, A.Lc);
  const Lv t = smem_level(A, S, A.Lc);
  const int n = g.H * g.W;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t.b[i] = g.b[i];
  __syncthreads();
  for (int l = A.Lc; l < A.L; ++l) {
    mg_down(smem_level(A, S, l), smem_level(A, S, l + 1), A.om, threadIdx.x, blockDim.x, act);
    __syncthreads();
  }
  const Lv c = smem_level(A, S, A.L);
  if (threadIdx.x == 0) {
    float e[4] = {0.f, 0.f, 0.f, 0.f}, en[4];
    const int nL = c.H * c.W;   // <= 4
    for (int it = 0; it < A.ncs; ++it) {
      for (int a = 0; a < nL; ++a) {
        if (c.lab[a] < 0) { en[a] = 0.f; continue; }
        const int y = a / c.W, x = a - y * c.W;
        float s = 0.f;
        if (x + 1 < c.W) s += c.wr[a] * (e[a] - e[a + 1]);
        if (x > 0) s += c.wr[a - 1] * (e[a] - e[a - 1]);
        if (y + 1 < c.H) s += c.wd[a] * (e[a] - e[a + c.W]);
        if (y > 0) s += c.wd[a - c.W] * (e[a] - e[a - c.W]);
        en[a] = e[a] + A.om * c.invd[a] * (c.b[a] - s);
      }
      for (int a = 0; a < nL; ++a) e[a] = en[a];
    }
    for (int a = 0; a < nL; ++a) c.e[a] = e[a];
  }
  __syncthreads();
  for (int l = A.L - 1; l >= A.Lc; --l) {
    mg_up(smem_level(A, S, l), smem_level(A, S, l + 1), A.om, A.sc, threadIdx.x, blockDim.x, act);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) g.e[i] = t.e[i];
}

// active at iteration k (pure function of the state left by iteration k-1)
__device__ __forceinline__ bool comp_now(const MgArgs& A, int c, int k) {
  const double* rr = A.cs + (size_t)(3 + (k & 1)) * A.Kc;
  const double* bb = A.cs + 5 * (size_t)A.Kc;
  const int* act = A.ci;
  const bool was = (k == 0) || act[(size_t)((k - 1) & 1) * A.Kc + c];
  return was && k < A.maxit && bb[c] > 0.0 && rr[c] > A.tol2 * bb[c];
}

// mean of the residual of component c at iteration k: projected out of r
// before the V-cycle (the float32 updates of r let a constant, which no
// operator step can remove, creep into each component's residual)
__device__ __forceinline__ float comp_mean(const MgArgs& A, int c, int k) {
  if (!A.project) return 0.f;
  const double n = A.cs[11 * (size_t)A.Kc + c];
  return n > 0.0 ? (float)(A.cs[(size_t)(12 + (k & 1)) * A.Kc + c] / n) : 0.f;
}

// level-0 restriction for the tile t: each of the 256 threads owns one level-1
// cell of the tile (16 x 16 cells)
template <bool CHECK>
__device__ __forceinline__ void down0_tile(const MgArgs& A, int t, int k, bool uon = true) {
  const int cy = (t / A.ntx) * (NI_TILE_H / 2) + (threadIdx.x >> 4);
  const int cx = (t % A.ntx) * (NI_TILE_W / 2) + (threadIdx.x & 15);
  const int H1 = A.lh[1], W1 = A.lw[1];
  if (cy >= H1 || cx >= W1) return;
  const int I = cy * W1 + cx;
  const int lc = A.clab[A.loff[1] + I];
  const float mu = (A.project && lc >= 0) ? comp_mean(A, lc, k) : 0.f;
  const float s = restrict_block(A.r, A.invd, A.wr, A.wd, A.inc0, A.H, A.W, cy, cx, A.om, mu);
  const bool on = lc >= 0 && (CHECK ? comp_now(A, lc, k) : uon);
  A.cb[A.loff[1] + I] = on ? s : 0.f;
}

template <bool ALIGNED>
__device__ __forceinline__ uchar4 ldinc(const uint8_t* p, int a, int nval) {
  if (ALIGNED && nval == 4) return *reinterpret_cast<const uchar4*>(p + a);
  return make_uchar4(nval > 0 ? p[a] : 0, nval > 1 ? p[a + 1] : 0, nval > 2 ? p[a + 2] : 0, nval > 3 ? p[a + 3] : 0);
}

__device__ __forceinline__ uint8_t u4get(const uchar4& v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

// ---------------------------------------------------------------------------
// per-tile bodies of the solve, shared by the persistent kernel and the
// per-phase kernels; every thread of the CTA calls them for the same tile
// ---------------------------------------------------------------------------
struct TileSmem {
  double sh[8 * 3 + 8];
  int key[TAB_SLOTS];
  double val[TAB_SLOTS * 3];
  int lab[TAB_SLOTS];
  float f[TAB_SLOTS * 4];
};

__device__ __forceinline__ void tile_smem_init(TileSmem& S) {
  if (threadIdx.x < TAB_SLOTS) {
    S.key[threadIdx.x] = -1;
    S.val[threadIdx.x * 3] = S.val[threadIdx.x * 3 + 1] = S.val[threadIdx.x * 3 + 2] = 0.0;
  }
  __syncthreads();
}

// per-component slots (doubles, Kc each)
#define MG_RZ 0    // [2] r^T z by iteration parity
#define MG_PQ 2    // p^T A p
#define MG_RR 3    // [2] r^T r by parity
#define MG_BB 5    // b^T b
#define MG_SX 6    // [2] sum x, pixel count (epilogue)
#define MG_XB 8    // warm start: x0^T b
#define MG_XAX 9   // warm start: x0^T A x0
#define MG_ALPH 10 // warm start: scale of x0
#define MG_CNT 11  // pixel count
#define MG_SR 12   // [2] sum of r by parity
__device__ __forceinline__ double* slot(const MgArgs& A, int s) { return A.cs + (size_t)s * A.Kc; }

__device__ __forceinline__ void load_labels_tile(const MgArgs& A, const G4& g, int ul, int (&lab)[4]) {
  if (ul >= 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) lab[j] = j < g.nval ? ul : -1;
  }
}

// prologue: r_0 = b - A x0; r^T r, sum r (or, warm, x0^T b and x0^T A x0), b^T b, count
template <bool COMP, bool ALIGNED>
__device__ void tile_prologue(const MgArgs& A, TileSmem& S, int t, int ul) {
  const int W = A.W, H = A.H, l8 = threadIdx.x & 7;
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
  float4 r4;
  float pv[3][4], pc[1][4];
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
    if (A.warm) {
      pv[0][j] = on[j] ? xa * f4get(b4, j) : 0.f;
      pv[1][j] = on[j] ? xa * ax : 0.f;
    } else {
      pv[0][j] = ra;
      pv[1][j] = ra * ra;
    }
    pv[2][j] = on[j] ? f4get(b4, j) * f4get(b4, j) : 0.f;
    pc[0][j] = on[j] ? 1.f : 0.f;
  }
  stg<ALIGNED>(A.r, g.a, g.nval, r4);
  stg<ALIGNED>(A.pb1, g.a, g.nval, make_float4(0, 0, 0, 0));
  double* const dst[3] = {slot(A, A.warm ? MG_XB : MG_SR), slot(A, A.warm ? MG_XAX : MG_RR), slot(A, MG_BB)};
  const int key = ul >= 0 ? ul : group_key(lab, on);
  float v[3];
  group_values<3>(key, lab, on, pv, dst, v);
  tile_accum<COMP, 3>(ul, key == -2 ? -1 : key, v, dst, S.key, S.val, S.sh);
  double* const dc[1] = {slot(A, MG_CNT)};
  float vc[1];
  group_values<1>(key, lab, on, pc, dc, vc);
  tile_accum<true, 1>(ul, key == -2 ? -1 : key, vc, dc, S.key, S.val, S.sh);
}

// warm start: x0 <- alpha_c x0, r <- (1 - alpha_c) b + alpha_c r (alpha from slot MG_ALPH)
template <bool COMP, bool ALIGNED>
__device__ void tile_warm(const MgArgs& A, TileSmem& S, int t, int ul) {
  const G4 g = group_of(t, A.ntx, A.H, A.W);
  int lab[4];
  ldlab<ALIGNED>(A.labels, g.a, g.nval, lab);
  float4 x4 = ldg<ALIGNED>(A.x, g.a, g.nval), r4 = ldg<ALIGNED>(A.r, g.a, g.nval);
  const float4 b4 = ldg<ALIGNED>(A.rhs, g.a, g.nval), id4 = ldg<ALIGNED>(A.invd, g.a, g.nval);
  const double* alph = slot(A, MG_ALPH);
  float pv[2][4];
  bool on[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    on[j] = lab[j] >= 0;
    const float al = on[j] ? (float)alph[lab[j]] : 0.f;
    f4set(x4, j, al * f4get(x4, j));
    float ra = (1.f - al) * f4get(b4, j) + al * f4get(r4, j);
    if (f4get(id4, j) == 0.f || !on[j]) ra = 0.f;
    f4set(r4, j, ra);
    pv[0][j] = ra * ra;
    pv[1][j] = ra;
  }
  stg<ALIGNED>(A.x, g.a, g.nval, x4);
  stg<ALIGNED>(A.r, g.a, g.nval, r4);
  double* const dst[2] = {slot(A, MG_RR), slot(A, MG_SR)};
  const int key = ul >= 0 ? ul : group_key(lab, on);
  float v[2];
  group_values<2>(key, lab, on, pv, dst, v);
  tile_accum<COMP, 2>(ul, key == -2 ? -1 : key, v, dst, S.key, S.val, S.sh);
}

// energy-optimal warm-start scale per component (grid-stride over c)
__device__ void comp_warm_alpha(const MgArgs& A, int i0, int stride) {
  const double* xb = slot(A, MG_XB);
  const double* xax = slot(A, MG_XAX);
  const double* bb = slot(A, MG_BB);
  double* alph = slot(A, MG_ALPH);
  for (int c = i0; c < A.K; c += stride) {
    const double al = (xax[c] > 0.0 && xb[c] > 0.0) ? xb[c] / xax[c] : 0.0;
    alph[c] = al;
    if (al == 0.0 && bb[c] > 0.0) atomicAdd(&A.st->warm_fallbacks, 1);
  }
}

// bookkeeping of iteration k (grid-stride over c): activity, iteration counts,
// unconverged flags, active count; p^T A p cleared for this iteration
__device__ void comp_book(const MgArgs& A, int k, int i0, int stride) {
  const int Kc = A.Kc, P = k & 1, Q = P ^ 1;
  const double* rrs = slot(A, MG_RR);
  const double* bb = slot(A, MG_BB);
  double* pq = slot(A, MG_PQ);
  int* act = A.ci;
  int* iters = A.ci + 2 * (size_t)Kc;
  for (int c = i0; c < A.K; c += stride) {
    const bool was = (k == 0) || act[(size_t)Q * Kc + c];
    const bool conv = !(bb[c] > 0.0 && rrs[(size_t)P * Kc + c] > A.tol2 * bb[c]);
    const bool nw = comp_now(A, c, k);
    if (was && !conv && k >= A.maxit) {
      atomicAdd(&A.st->fill_unconv, 1);
      atomicOr(&A.st->err, NI_DEV_ERR_FILL_NOCONV);
    }
    act[(size_t)P * Kc + c] = nw ? 1 : 0;
    if (nw) {
      iters[c] += 1;
      atomicAdd(&A.ntl[2 + P], 1);
    }
    pq[c] = 0.0;
  }
}

// level-0 restriction of tile t (one level-1 cell per thread)
__device__ __forceinline__ void tile_down0(const MgArgs& A, int t, int ul, int k);

// tile_down0 for the persistent kernel, which keeps a list of the tiles still
// active: returns (the same in every thread of the CTA) whether a pixel of the
// tile belongs to a component active at iteration k.  A tile that is not is
// visited once more (its level-1 cells get 0, as in tile_down0) and then left
// out of every later pass; the active set only shrinks.
__device__ __forceinline__ bool tile_down0_active(const MgArgs& A, int t, int ul, int k) {
  if (ul >= 0) {
    tile_down0(A, t, ul, k);
    return comp_now(A, ul, k);
  }
  down0_tile<true>(A, t, k);
  // mixed tile: the thread of level-1 cell (cy, cx) checks its 2 x 2 pixels
  const int cy = (t / A.ntx) * (NI_TILE_H / 2) + (threadIdx.x >> 4);
  const int cx = (t % A.ntx) * (NI_TILE_W / 2) + (threadIdx.x & 15);
  bool on = false;
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const int y = 2 * cy + dy, x = 2 * cx + dx;
      if (y < A.H && x < A.W) {
        const int lb = A.labels[y * A.W + x];
        on |= lb >= 0 && comp_now(A, lb, k);
      }
    }
  return __syncthreads_or(on) != 0;
}

__device__ __forceinline__ void tile_down0(const MgArgs& A, int t, int ul, int k) {
  if (ul >= 0) {
    // the window loads go out with those of the activity test; the level-1
    // cells of a converged component get 0
    down0_tile<false>(A, t, k, comp_now(A, ul, k));
  } else {
    down0_tile<true>(A, t, k);
  }
}

// level-0 prolongation and smoothing: z_k and r^T z per component
// LIST: t comes from the list of tiles active at k, so a tile with one label
// holds an active component and needs no activity load
template <bool COMP, bool ALIGNED, bool LIST = false>
__device__ void tile_up0(const MgArgs& A, TileSmem& S, int t, int ul, int k, const int* actk,
                         int par = -1) {
  if (!LIST && ul >= 0 && !actk[ul]) return;   // uniform across the CTA
  const int W = A.W, H = A.H, l8 = threadIdx.x & 7, W1 = A.lw[1];
  const float om = A.om, sc = A.sc;
  const float* e1 = A.ce + A.loff[1];
  double* rz = slot(A, MG_RZ + (k & 1));
  const G4 g = group_of(t, A.ntx, H, W);
  int lab[4];
  if (ul >= 0) load_labels_tile(A, g, ul, lab);
  else ldlab<ALIGNED>(A.labels, g.a, g.nval, lab);
  bool now[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) now[j] = lab[j] >= 0 && ((LIST && ul >= 0) || actk[lab[j]]);
  const float4 r4 = ldg<ALIGNED>(A.r, g.a, g.nval);
  const float4 id4 = ldg<ALIGNED>(A.invd, g.a, g.nval);
  float mu[4] = {0.f, 0.f, 0.f, 0.f};
  if (A.project) {
    int sl[4];
    tile_slots(ul, lab, sl, S.lab);
    if (threadIdx.x < TAB_SLOTS && S.lab[threadIdx.x] >= 0) S.f[threadIdx.x * 4] = comp_mean(A, S.lab[threadIdx.x], k);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j)
      mu[j] = sl[j] >= 0 ? S.f[sl[j] * 4] : (sl[j] == -2 ? comp_mean(A, lab[j], k) : 0.f);
  }
  const float4 wr4 = ldg<ALIGNED>(A.wr, g.a, g.nval), wd4 = ldg<ALIGNED>(A.wd, g.a, g.nval);
  const uchar4 in4 = ldinc<ALIGNED>(A.inc0, g.a, g.nval);
  float ec[4];
  {
    const float* er = e1 + (size_t)(g.row >> 1) * W1;
    float e0 = 0.f, e2 = 0.f;
    if (g.nval > 0) e0 = er[g.col >> 1];
    if (g.nval > 2) e2 = er[(g.col + 2) >> 1];
#pragma unroll
    for (int j = 0; j < 4; ++j) ec[j] = (j < g.nval && u4get(in4, j)) ? (j < 2 ? e0 : e2) : 0.f;
  }
  float4 zc;
#pragma unroll
  for (int j = 0; j < 4; ++j) f4set(zc, j, om * f4get(id4, j) * (f4get(r4, j) - mu[j]) + sc * ec[j]);
  float zl = __shfl_up_sync(NI_FULL, zc.w, 1), zr = __shfl_down_sync(NI_FULL, zc.x, 1);
  float wl0 = __shfl_up_sync(NI_FULL, wr4.w, 1);
  if (l8 == 0) {
    const bool ok = g.nval > 0 && g.col > 0;
    wl0 = ok ? A.wr[g.a - 1] : 0.f;
    const float zz = ok ? zc_at(A.r, A.invd, A.inc0, e1, W, W1, g.row, g.col - 1, om, sc, mu[0]) : 0.f;
    zl = wl0 != 0.f ? zz : 0.f;
  }
  if (l8 == 7) {
    const bool ok = g.nval == 4 && g.col + 4 < W;
    const float zz = ok ? zc_at(A.r, A.invd, A.inc0, e1, W, W1, g.row, g.col + 4, om, sc, mu[3]) : 0.f;
    zr = (ok && wr4.w != 0.f) ? zz : 0.f;
  }
  float4 zu = make_float4(0, 0, 0, 0), zd = make_float4(0, 0, 0, 0), wu4 = make_float4(0, 0, 0, 0);
  if (g.row > 0) {
    wu4 = ldg<ALIGNED>(A.wd, g.a - W, g.nval);
    const float4 ru = ldg<ALIGNED>(A.r, g.a - W, g.nval), iu = ldg<ALIGNED>(A.invd, g.a - W, g.nval);
    const uchar4 cu = ldinc<ALIGNED>(A.inc0, g.a - W, g.nval);
    const float* er = e1 + (size_t)((g.row - 1) >> 1) * W1;
    const float e0 = g.nval > 0 ? er[g.col >> 1] : 0.f, e2 = g.nval > 2 ? er[(g.col + 2) >> 1] : 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float zz = om * f4get(iu, j) * (f4get(ru, j) - mu[j]) + (u4get(cu, j) ? sc * (j < 2 ? e0 : e2) : 0.f);
      f4set(zu, j, (j < g.nval && f4get(wu4, j) != 0.f) ? zz : 0.f);
    }
  }
  if (g.row + 1 < H) {
    const float4 rd = ldg<ALIGNED>(A.r, g.a + W, g.nval), idd = ldg<ALIGNED>(A.invd, g.a + W, g.nval);
    const uchar4 cd = ldinc<ALIGNED>(A.inc0, g.a + W, g.nval);
    const float* er = e1 + (size_t)((g.row + 1) >> 1) * W1;
    const float e0 = g.nval > 0 ? er[g.col >> 1] : 0.f, e2 = g.nval > 2 ? er[(g.col + 2) >> 1] : 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float zz = om * f4get(idd, j) * (f4get(rd, j) - mu[j]) + (u4get(cd, j) ? sc * (j < 2 ? e0 : e2) : 0.f);
      f4set(zd, j, (j < g.nval && f4get(wd4, j) != 0.f) ? zz : 0.f);
    }
  }
  float4 z4;
  float pv[1][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float za = f4get(zc, j);
    const float zR = j < 3 ? f4get(zc, j + 1) : zr, zL = j > 0 ? f4get(zc, j - 1) : zl;
    const float wl = j > 0 ? f4get(wr4, j - 1) : wl0;
    const float az = f4get(wr4, j) * (za - zR) + f4get(wd4, j) * (za - f4get(zd, j)) + wl * (za - zL) +
                     f4get(wu4, j) * (za - f4get(zu, j));
    const float rp = now[j] ? f4get(r4, j) - mu[j] : f4get(r4, j);
    const float zf = now[j] ? za + om * f4get(id4, j) * (rp - az) : 0.f;
    f4set(z4, j, zf);
    pv[0][j] = zf * rp;
  }
  stg<ALIGNED>(A.z, g.a, g.nval, z4);
  double* const dst[1] = {rz};
  const int key = ul >= 0 ? ul : group_key(lab, now);
  float v[1];
  group_values<1>(key, lab, now, pv, dst, v);
  tile_accum<COMP, 1>(ul, key == -2 ? -1 : key, v, dst, S.key, S.val, S.sh, par);
}

// direction: p_k = z_k + beta_k p_{k-1}; q = A p_k; p^T A p per component
template <bool COMP, bool ALIGNED, bool LIST = false>
__device__ void tile_dir(const MgArgs& A, TileSmem& S, int t, int ul, int k, const int* actk,
                         int par = -1) {
  if (!LIST && ul >= 0 && !actk[ul]) return;
  const int W = A.W, H = A.H, l8 = threadIdx.x & 7, Kc = A.Kc;
  const int P = k & 1, Q = P ^ 1;
  const float* pold = Q ? A.pb1 : A.pb0;
  float* pnew = P ? A.pb1 : A.pb0;
  const double* rz = slot(A, MG_RZ + P);
  const double* rzo = slot(A, MG_RZ + Q);
  (void)Kc;
  const G4 g = group_of(t, A.ntx, H, W);
  int lab[4];
  if (ul >= 0) load_labels_tile(A, g, ul, lab);
  else ldlab<ALIGNED>(A.labels, g.a, g.nval, lab);
  auto betaf = [&](int c) -> float {
    const double ro = rzo[c];
    return (k > 0 && ro > 0.0) ? (float)(rz[c] / ro) : 0.f;
  };
  const float4 z4 = ldg<ALIGNED>(A.z, g.a, g.nval), po4 = ldg<ALIGNED>(pold, g.a, g.nval);
  const float4 wr4 = ldg<ALIGNED>(A.wr, g.a, g.nval), wd4 = ldg<ALIGNED>(A.wd, g.a, g.nval);
  // row ends: the neighbours' z, p and weight, loaded with the rest
  const bool okl = l8 == 0 && g.nval > 0 && g.col > 0, okr = l8 == 7 && g.nval == 4 && g.col + 4 < W;
  const float wle = okl ? A.wr[g.a - 1] : 0.f;
  const float zle = okl ? A.z[g.a - 1] : 0.f, ple = okl ? pold[g.a - 1] : 0.f;
  const float zre = okr ? A.z[g.a + 4] : 0.f, pre = okr ? pold[g.a + 4] : 0.f;
  float beta[4];
  bool now[4];
  if (ul >= 0) {   // one component: lane 0 of each warp computes beta, no CTA barrier
    float bt = (threadIdx.x & 31) == 0 ? betaf(ul) : 0.f;
    bt = __shfl_sync(NI_FULL, bt, 0);
    const bool on = LIST || actk[ul] != 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      now[j] = lab[j] >= 0 && on;
      beta[j] = bt;
    }
  } else {
    int sl[4];
    tile_slots(ul, lab, sl, S.lab);
    if (threadIdx.x < TAB_SLOTS && S.lab[threadIdx.x] >= 0) S.f[threadIdx.x * 4] = betaf(S.lab[threadIdx.x]);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      now[j] = lab[j] >= 0 && actk[lab[j]];
      beta[j] = sl[j] >= 0 ? S.f[sl[j] * 4] : (sl[j] == -2 ? betaf(lab[j]) : 0.f);
    }
  }
  float4 pn;
#pragma unroll
  for (int j = 0; j < 4; ++j) f4set(pn, j, now[j] ? f4get(z4, j) + beta[j] * f4get(po4, j) : 0.f);
  float pl = __shfl_up_sync(NI_FULL, pn.w, 1), pr = __shfl_down_sync(NI_FULL, pn.x, 1);
  float wl0 = __shfl_up_sync(NI_FULL, wr4.w, 1);
  if (l8 == 0) {
    wl0 = wle;
    pl = (wl0 != 0.f && now[0]) ? zle + beta[0] * ple : 0.f;
  }
  if (l8 == 7) pr = (okr && wr4.w != 0.f && now[3]) ? zre + beta[3] * pre : 0.f;
  float4 pu = make_float4(0, 0, 0, 0), pd = make_float4(0, 0, 0, 0), wu4 = make_float4(0, 0, 0, 0);
  if (g.row > 0) {
    wu4 = ldg<ALIGNED>(A.wd, g.a - W, g.nval);
    const float4 zu = ldg<ALIGNED>(A.z, g.a - W, g.nval), pu0 = ldg<ALIGNED>(pold, g.a - W, g.nval);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      f4set(pu, j, (now[j] && f4get(wu4, j) != 0.f) ? f4get(zu, j) + beta[j] * f4get(pu0, j) : 0.f);
  }
  if (g.row + 1 < H) {
    const float4 zd = ldg<ALIGNED>(A.z, g.a + W, g.nval), pd0 = ldg<ALIGNED>(pold, g.a + W, g.nval);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      f4set(pd, j, (now[j] && f4get(wd4, j) != 0.f) ? f4get(zd, j) + beta[j] * f4get(pd0, j) : 0.f);
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
  double* const dst[1] = {slot(A, MG_PQ)};
  const int key = ul >= 0 ? ul : group_key(lab, now);
  float v[1];
  group_values<1>(key, lab, now, pv, dst, v);
  tile_accum<COMP, 1>(ul, key == -2 ? -1 : key, v, dst, S.key, S.val, S.sh, par);
}

// update: alpha_k; x += alpha p; r = (r - mean) - alpha q; r^T r, sum r per component
template <bool COMP, bool ALIGNED, bool LIST = false>
__device__ void tile_upd(const MgArgs& A, TileSmem& S, int t, int ul, int k, const int* actk,
                         int par = -1) {
  if (!LIST && ul >= 0 && !actk[ul]) return;
  const int P = k & 1, Q = P ^ 1;
  const float* pnew = P ? A.pb1 : A.pb0;
  const double* rz = slot(A, MG_RZ + P);
  const double* pq = slot(A, MG_PQ);
  const G4 g = group_of(t, A.ntx, A.H, A.W);
  int lab[4];
  if (ul >= 0) load_labels_tile(A, g, ul, lab);
  else ldlab<ALIGNED>(A.labels, g.a, g.nval, lab);
  auto alphaf = [&](int c) -> float {
    const double pp = pq[c];
    return pp > 0.0 ? (float)(rz[c] / pp) : 0.f;
  };
  float4 x4 = ldg<ALIGNED>(A.x, g.a, g.nval), r4 = ldg<ALIGNED>(A.r, g.a, g.nval);
  const float4 p4 = ldg<ALIGNED>(pnew, g.a, g.nval), q4 = ldg<ALIGNED>(A.q, g.a, g.nval);
  int sl[4] = {-1, -1, -1, -1};
  float ual = 0.f, umu = 0.f;
  if (ul >= 0) {   // one component: lane 0 of each warp computes the scalars
    if ((threadIdx.x & 31) == 0) {
      ual = alphaf(ul);
      umu = comp_mean(A, ul, k);
    }
    ual = __shfl_sync(NI_FULL, ual, 0);
    umu = __shfl_sync(NI_FULL, umu, 0);
  } else {
    tile_slots(ul, lab, sl, S.lab);
    if (threadIdx.x < TAB_SLOTS && S.lab[threadIdx.x] >= 0) {
      S.f[threadIdx.x * 4] = alphaf(S.lab[threadIdx.x]);
      S.f[threadIdx.x * 4 + 1] = comp_mean(A, S.lab[threadIdx.x], k);
    }
    __syncthreads();
  }
  float pv[2][4];
  bool now[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    now[j] = lab[j] >= 0 && ((LIST && ul >= 0) || actk[lab[j]]);
    float al = 0.f, mu = 0.f;
    if (now[j]) {
      if (ul >= 0) {
        al = ual;
        mu = umu;
      } else if (sl[j] >= 0) {
        al = S.f[sl[j] * 4];
        mu = S.f[sl[j] * 4 + 1];
      } else if (sl[j] == -2) {
        al = alphaf(lab[j]);
        mu = comp_mean(A, lab[j], k);
      }
    }
    f4set(x4, j, f4get(x4, j) + al * f4get(p4, j));
    // r_{k+1} = (r_k - its component mean) - alpha q: the residual the V-cycle
    // of this iteration saw
    const float ra = (f4get(r4, j) - mu) - al * f4get(q4, j);
    f4set(r4, j, ra);
    pv[0][j] = now[j] ? ra * ra : 0.f;
    pv[1][j] = now[j] ? ra : 0.f;
  }
  stg<ALIGNED>(A.x, g.a, g.nval, x4);
  stg<ALIGNED>(A.r, g.a, g.nval, r4);
  double* const dst[2] = {slot(A, MG_RR + Q), slot(A, MG_SR + Q)};
  const int key = ul >= 0 ? ul : group_key(lab, now);
  float v[2];
  group_values<2>(key, lab, now, pv, dst, v);
  tile_accum<COMP, 2>(ul, key == -2 ? -1 : key, v, dst, S.key, S.val, S.sh, par);
}

// epilogue, first part: sum of x and pixel count per component
__device__ void tile_epi_sums(const MgArgs& A, TileSmem& S, int t, int ul) {
  const G4 g = group_of(t, A.ntx, A.H, A.W);
  int lab[4];
  ldlab<false>(A.labels, g.a, g.nval, lab);
  const float4 x4 = ldg<false>(A.x, g.a, g.nval);
  float pv[2][4];
  bool on[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    on[j] = lab[j] >= 0;
    pv[0][j] = on[j] ? f4get(x4, j) : 0.f;
    pv[1][j] = on[j] ? 1.f : 0.f;
  }
  double* const dst[2] = {slot(A, MG_SX), slot(A, MG_SX + 1)};
  const int key = ul >= 0 ? ul : group_key(lab, on);
  float v[2];
  group_values<2>(key, lab, on, pv, dst, v);
  tile_accum<true, 2>(ul, key == -2 ? -1 : key, v, dst, S.key, S.val, S.sh);
}

// epilogue, second part: zero mean per component; iteration statistics
__device__ void mg_epi_apply(const MgArgs& A, int i0, int stride) {
  const double* sx = slot(A, MG_SX);
  const double* cnt = slot(A, MG_SX + 1);
  const int* iters = A.ci + 2 * (size_t)A.Kc;
  for (int a = i0; a < A.N; a += stride) {
    const int c = A.labels[a];
    if (c >= 0 && cnt[c] > 0) A.x[a] = (float)((double)A.x[a] - sx[c] / cnt[c]);
  }
  for (int c = i0; c < A.K; c += stride) {
    atomicMax(&A.st->fill_iters, iters[c]);
    if (iters[c] > 0)
      atomicAdd(&A.st->fill_px_iters, (unsigned long long)iters[c] * (unsigned long long)cnt[c]);
  }
}

// ---------------------------------------------------------------------------
// persistent variant: one cooperative launch, grid barriers between phases
// ---------------------------------------------------------------------------
// the CTA's tiles of a list of n tiles (i = blockIdx.x, + gridDim.x, ...); the
// next entry is loaded before the current tile is processed, so its latency
// hides behind the tile's work
#define MG_LIST_LOOP(LIST, N, BODY)                                              \
  {                                                                              \
    int2 nx = blockIdx.x < (N) ? (LIST)[blockIdx.x] : make_int2(0, -2);          \
    int tpar = 0;   /* parity of the CTA's tile step */                          \
    for (int i = blockIdx.x; i < (N); i += gridDim.x, tpar ^= 1) {               \
      const int2 te = nx;                                                        \
      if (i + (int)gridDim.x < (N)) nx = (LIST)[i + gridDim.x];                  \
      BODY;                                                                      \
    }                                                                            \
    (void)tpar;                                                                  \
  }
template <bool COMP, bool ALIGNED>
__global__ void __launch_bounds__(NI_TILE_THREADS, 4) k_pcg_mg(MgArgs A) {
  __shared__ TileSmem S;
  __shared__ MgSmem s_mg;
  int* err = &A.st->err;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthr = gridDim.x * blockDim.x;
  tile_smem_init(S);
  if (blockIdx.x == 0) mg_smem_load(A, s_mg);
  for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
    const int ul = A.tile_lab[t];
    if (ul == -2) continue;
    tile_prologue<COMP, ALIGNED>(A, S, t, ul);
    if (threadIdx.x == 0) {
      const int pos = atomicAdd(&A.ntl[0], 1);
      A.tiles[pos] = make_int2(t, ul);
    }
  }
  if (!grid_barrier(&A.st->bar, err)) return;
  const int nt = *(volatile int*)&A.ntl[0];
  if (A.warm) {
    comp_warm_alpha(A, gtid, gthr);
    if (!grid_barrier(&A.st->bar, err)) return;
    MG_LIST_LOOP(A.tiles, nt, (tile_warm<COMP, ALIGNED>(A, S, te.x, te.y)));
    if (!grid_barrier(&A.st->bar, err)) return;
  }
  for (int k = 0;; ++k) {
    const int P = k & 1, Q = P ^ 1;
    comp_book(A, k, gtid, gthr);
    // restriction over the tiles active at k - 1 (all at k = 0); those still
    // active at k form the list of parity P that the later passes walk
    int2* const cur = A.tact + (size_t)P * A.ntiles;
    {
      const int2* prev = k == 0 ? A.tiles : A.tact + (size_t)Q * A.ntiles;
      const int np = k == 0 ? nt : *(volatile int*)&A.ntl[4 + Q];
      MG_LIST_LOOP(prev, np, {
        if (tile_down0_active(A, te.x, te.y, k) && threadIdx.x == 0) cur[atomicAdd(&A.ntl[4 + P], 1)] = te;
      });
    }
    if (!grid_barrier(&A.st->bar, err)) return;
    if (*(volatile int*)&A.ntl[2 + P] == 0) break;
    const int na = *(volatile int*)&A.ntl[4 + P];
    const int* actk = A.ci + (size_t)P * A.Kc;
    // coarse levels: a pass on level l runs on the first n CTAs and ends with a
    // barrier among them; n does not grow towards coarser levels
    const int tail_d = NI_MG_LIST_LEVELS < A.Lc ? A.pd[NI_MG_LIST_LEVELS] : 1;
    for (int l = 1; l < A.Lc; ++l) {
      const bool tl = l + 1 <= NI_MG_LIST_LEVELS;
      const int n = tl ? mg_tile_ctas(A, na, l + 1, tail_d) : A.pd[l];
      if (blockIdx.x >= n) break;
      if (tl) mg_down_tiles(A, l, cur, na, actk, gtid, n * blockDim.x);
      else mg_down(coarse_level(A, l), coarse_level(A, l + 1), A.om, gtid, n * blockDim.x, actk);
      if (!grid_barrier_n(&A.mbar[l], n, err)) return;
    }
    if (blockIdx.x == 0) mg_cta_levels(A, s_mg, actk);
    const int tail_u = NI_MG_LIST_LEVELS + 1 < A.Lc ? A.pu[NI_MG_LIST_LEVELS + 1] : 1;
    for (int l = A.Lc - 1; l >= 1; --l) {
      const bool tl = l <= NI_MG_LIST_LEVELS;
      const int n = tl ? mg_tile_ctas(A, na, l, tail_u) : A.pu[l];
      if (blockIdx.x >= n) continue;
      if (!grid_barrier_n(&A.mbar[NI_MG_MAX_LEVELS + 1 + l], n, err)) return;
      if (tl) mg_up_tiles(A, l, cur, na, actk, gtid, n * blockDim.x);
      else mg_up(coarse_level(A, l), coarse_level(A, l + 1), A.om, A.sc, gtid, n * blockDim.x, actk);
    }
    if (!grid_barrier(&A.st->bar, err)) return;
    if (gtid == 0) {
      A.ntl[2 + Q] = 0;
      A.ntl[4 + Q] = 0;   // the list of k - 1 is read no more: it takes the tiles of k + 1
    }
    for (int c = gtid; c < A.K; c += gthr) {
      slot(A, MG_RR + Q)[c] = 0.0;
      slot(A, MG_SR + Q)[c] = 0.0;
    }
    MG_LIST_LOOP(cur, na, (tile_up0<COMP, ALIGNED, true>(A, S, te.x, te.y, k, actk, tpar)));
    if (!grid_barrier(&A.st->bar, err)) return;
    MG_LIST_LOOP(cur, na, (tile_dir<COMP, ALIGNED, true>(A, S, te.x, te.y, k, actk, tpar)));
    if (!grid_barrier(&A.st->bar, err)) return;
    for (int c = gtid; c < A.K; c += gthr) slot(A, MG_RZ + Q)[c] = 0.0;
    MG_LIST_LOOP(cur, na, (tile_upd<COMP, ALIGNED, true>(A, S, te.x, te.y, k, actk, tpar)));
    if (!grid_barrier(&A.st->bar, err)) return;
  }
  MG_LIST_LOOP(A.tiles, nt, (tile_epi_sums(A, S, te.x, te.y)));
  if (!grid_barrier(&A.st->bar, err)) return;
  mg_epi_apply(A, gtid, gthr);
}

// ---------------------------------------------------------------------------
// per-phase variant: one kernel per pass, one tile (or cell) per CTA (thread),
// replayed from a CUDA graph in chunks of iterations; the iteration index and
// the done flag live on the device
// ---------------------------------------------------------------------------
struct MgIter {
  int k;      // current iteration
  int done;   // no component active any more
};

template <bool COMP, bool ALIGNED>
__global__ void __launch_bounds__(NI_TILE_THREADS) k_mgx_prologue(MgArgs A) {
  __shared__ TileSmem S;
  const int t = blockIdx.x;
  const int ul = A.tile_lab[t];
  if (ul == -2) return;
  tile_smem_init(S);
  tile_prologue<COMP, ALIGNED>(A, S, t, ul);
}

__global__ void k_mgx_warm_alpha(MgArgs A) { comp_warm_alpha(A, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x); }

template <bool COMP, bool ALIGNED>
__global__ void __launch_bounds__(NI_TILE_THREADS) k_mgx_warm(MgArgs A) {
  __shared__ TileSmem S;
  const int t = blockIdx.x;
  const int ul = A.tile_lab[t];
  if (ul == -2) return;
  tile_smem_init(S);
  tile_warm<COMP, ALIGNED>(A, S, t, ul);
}

// bookkeeping of iteration k (components) and the level-0 restriction (tiles)
__global__ void __launch_bounds__(NI_TILE_THREADS) k_mgx_book_down0(MgArgs A, MgIter* it) {
  if (*(volatile int*)&it->done) return;
  const int k = it->k;
  comp_book(A, k, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  if (blockIdx.x < A.ntiles) {
    const int ul = A.tile_lab[blockIdx.x];
    if (ul != -2) tile_down0(A, blockIdx.x, ul, k);
  }
}

__device__ __forceinline__ bool mgx_skip(const MgArgs& A, const MgIter* it) {
  return *(volatile int*)&it->done || *(volatile int*)&A.ntl[2 + (it->k & 1)] == 0;
}

__global__ void k_mgx_down(MgArgs A, MgIter* it, int l) {
  if (mgx_skip(A, it)) return;
  mg_down(coarse_level(A, l), coarse_level(A, l + 1), A.om, blockIdx.x * blockDim.x + threadIdx.x,
          gridDim.x * blockDim.x, A.ci + (size_t)(it->k & 1) * A.Kc);
}

__global__ void __launch_bounds__(NI_TILE_THREADS) k_mgx_cta(MgArgs A, MgIter* it) {
  __shared__ MgSmem s_mg;
  if (mgx_skip(A, it)) return;
  mg_smem_load(A, s_mg);
  mg_cta_levels(A, s_mg, A.ci + (size_t)(it->k & 1) * A.Kc);
}

__global__ void k_mgx_up(MgArgs A, MgIter* it, int l) {
  if (mgx_skip(A, it)) return;
  mg_up(coarse_level(A, l), coarse_level(A, l + 1), A.om, A.sc, blockIdx.x * blockDim.x + threadIdx.x,
        gridDim.x * blockDim.x, A.ci + (size_t)(it->k & 1) * A.Kc);
}

template <bool COMP, bool ALIGNED>
__global__ void __launch_bounds__(NI_TILE_THREADS) k_mgx_up0(MgArgs A, MgIter* it) {
  __shared__ TileSmem S;
  if (mgx_skip(A, it)) return;
  const int k = it->k, Q = (k & 1) ^ 1;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthr = gridDim.x * blockDim.x;
  if (gtid == 0) A.ntl[2 + Q] = 0;
  for (int c = gtid; c < A.K; c += gthr) {
    slot(A, MG_RR + Q)[c] = 0.0;
    slot(A, MG_SR + Q)[c] = 0.0;
  }
  const int ul = A.tile_lab[blockIdx.x];
  if (ul == -2) return;
  tile_smem_init(S);
  tile_up0<COMP, ALIGNED>(A, S, blockIdx.x, ul, k, A.ci + (size_t)(k & 1) * A.Kc);
}

template <bool COMP, bool ALIGNED>
__global__ void __launch_bounds__(NI_TILE_THREADS) k_mgx_dir(MgArgs A, MgIter* it) {
  __shared__ TileSmem S;
  if (mgx_skip(A, it)) return;
  const int ul = A.tile_lab[blockIdx.x];
  if (ul == -2) return;
  tile_smem_init(S);
  tile_dir<COMP, ALIGNED>(A, S, blockIdx.x, ul, it->k, A.ci + (size_t)(it->k & 1) * A.Kc);
}

template <bool COMP, bool ALIGNED>
__global__ void __launch_bounds__(NI_TILE_THREADS) k_mgx_upd(MgArgs A, MgIter* it) {
  __shared__ TileSmem S;
  if (mgx_skip(A, it)) return;
  const int k = it->k, Q = (k & 1) ^ 1;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthr = gridDim.x * blockDim.x;
  for (int c = gtid; c < A.K; c += gthr) slot(A, MG_RZ + Q)[c] = 0.0;
  const int ul = A.tile_lab[blockIdx.x];
  if (ul == -2) return;
  tile_smem_init(S);
  tile_upd<COMP, ALIGNED>(A, S, blockIdx.x, ul, k, A.ci + (size_t)(k & 1) * A.Kc);
}

// end of an iteration: the next index, or done once nothing was active
__global__ void k_mgx_next(MgArgs A, MgIter* it) {
  if (it->done) return;
  if (A.ntl[2 + (it->k & 1)] == 0) it->done = 1;
  else it->k += 1;
}

__global__ void __launch_bounds__(NI_TILE_THREADS) k_mgx_epi_sums(MgArgs A) {
  __shared__ TileSmem S;
  const int ul = A.tile_lab[blockIdx.x];
  if (ul == -2) return;
  tile_smem_init(S);
  tile_epi_sums(A, S, blockIdx.x, ul);
}

__global__ void k_mgx_epi_apply(MgArgs A) { mg_epi_apply(A, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x); }

// ---------------------------------------------------------------------------
// hierarchy setup: level l+1 from level l (Galerkin product of the 2x2
// piecewise-constant aggregation restricted to same-label cells)
// ---------------------------------------------------------------------------
struct LvIn {
  const int* lab;
  const float* wr;
  const float* wd;
  const float* s;      // leak of each cell (diagonal minus its edge weights); nullptr: 0 (level 0)
  uint8_t* inc;        // written: cell aggregated into its parent
  int H, W;
};

__device__ __forceinline__ int first_label(const LvIn& f, int cy, int cx) {
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const int y = 2 * cy + dy, x = 2 * cx + dx;
      if (y < f.H && x < f.W) {
        const int l = f.lab[y * f.W + x];
        if (l >= 0) return l;
      }
    }
  return -1;
}

// Every sum is over non-negative terms (no cancellation): the diagonal of an
// aggregate is its cells' leaks plus the weights of all edges that leave the
// block; its leak is the part of that which no coarse edge carries (leaks of
// its cells and edges to cells that are not aggregated into their own parent).
__global__ void k_mg_coarsen(LvIn f, int Hc, int Wc, int* __restrict__ clab, float* __restrict__ cwr,
                             float* __restrict__ cwd, float* __restrict__ cs, float* __restrict__ cinvd) {
  const int nc = Hc * Wc;
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
    const int cy = I / Wc, cx = I - cy * Wc;
    const int lc = first_label(f, cy, cx);
    float wrc = 0.f, wdc = 0.f, dc = 0.f, sc = 0.f;
    const int flR = (lc >= 0 && cx + 1 < Wc) ? first_label(f, cy, cx + 1) : -1;
    const int flL = (lc >= 0 && cx > 0) ? first_label(f, cy, cx - 1) : -1;
    const int flD = (lc >= 0 && cy + 1 < Hc) ? first_label(f, cy + 1, cx) : -1;
    const int flU = (lc >= 0 && cy > 0) ? first_label(f, cy - 1, cx) : -1;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int y = 2 * cy + dy, x = 2 * cx + dx;
        if (y >= f.H || x >= f.W) continue;
        const int a = y * f.W + x;
        const bool in = lc >= 0 && f.lab[a] == lc;
        f.inc[a] = in ? 1 : 0;
        if (!in) continue;
        const float sa = f.s ? f.s[a] : 0.f;
        dc += sa;
        sc += sa;
        if (dx == 1) {                      // edge to the block on the right
          const float w = f.wr[a];
          dc += w;
          if (flR == lc) wrc += w; else sc += w;
        } else if (x > 0) {                 // edge to the block on the left
          const float w = f.wr[a - 1];
          dc += w;
          if (flL != lc) sc += w;
        }
        if (dy == 1) {                      // edge to the block below
          const float w = f.wd[a];
          dc += w;
          if (flD == lc) wdc += w; else sc += w;
        } else if (y > 0) {                 // edge to the block above
          const float w = f.wd[a - f.W];
          dc += w;
          if (flU != lc) sc += w;
        }
      }
    clab[I] = lc;
    cwr[I] = wrc;
    cwd[I] = wdc;
    cs[I] = sc;
    cinvd[I] = dc > 0.f ? 1.0f / dc : 0.f;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int grid_cells(ni_handle* h, long long n) {
  long long b = (n + 255) / 256;
  return (int)std::max(1LL, std::min(b, (long long)h->num_sms * 8));
}

static ni_status ensure_mg(ni_handle* h, cudaStream_t s) {
  if (h->mg_cells > 0) return NI_OK;
  // level dimensions: halve until a level holds at most 4 cells
  long long total = 0;
  int L = 0, hh = h->H, ww = h->W;
  h->mg_h[0] = hh; h->mg_w[0] = ww; h->mg_off[0] = 0;
  do {
    hh = (hh + 1) / 2; ww = (ww + 1) / 2;
    ++L;
    if (L > NI_MG_MAX_LEVELS) return ni_fail(h, NI_ERR_INVALID_ARG, "multigrid: too many levels");
    h->mg_h[L] = hh; h->mg_w[L] = ww;
    h->mg_off[L] = total;
    total += ((long long)hh * ww + 63) / 64 * 64;
  } while ((long long)hh * ww > 4);
  h->mg_L = L;
  cudaError_t e = cudaSuccess;
  auto al = [&](auto** p, size_t n) {
    if (e == cudaSuccess) e = cudaMalloc((void**)p, n * sizeof(**p));
  };
  al(&h->mg_lab, total); al(&h->mg_wr, total); al(&h->mg_wd, total); al(&h->mg_d, total);
  al(&h->mg_invd, total); al(&h->mg_b, total); al(&h->mg_e, total); al(&h->mg_inc, total);
  al(&h->inc0, (size_t)h->Npad); al(&h->z, (size_t)h->Npad);
  al(&h->mg_bar, (size_t)2 * (NI_MG_MAX_LEVELS + 1));
  al(&h->mg_iter, (size_t)4);
  al(&h->mg_tact, (size_t)2 * h->ntiles);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ni_fail(h, NI_ERR_OOM, "multigrid hierarchy allocation failed");
  }
  h->mg_cells = total;
  cudaMemsetAsync(h->mg_b, 0, total * sizeof(float), s);
  cudaMemsetAsync(h->mg_e, 0, total * sizeof(float), s);
  cudaMemsetAsync(h->mg_inc, 0, total, s);
  cudaMemsetAsync(h->inc0, 0, (size_t)h->Npad, s);
  cudaMemsetAsync(h->z, 0, sizeof(float) * (size_t)h->Npad, s);
  return ni_cuda_check(h, cudaGetLastError(), "multigrid allocation");
}

void free_mg(ni_handle* h) {
  cudaFree(h->mg_lab); cudaFree(h->mg_wr); cudaFree(h->mg_wd); cudaFree(h->mg_d); cudaFree(h->mg_invd);
  cudaFree(h->mg_b); cudaFree(h->mg_e); cudaFree(h->mg_inc); cudaFree(h->inc0); cudaFree(h->z);
  cudaFree(h->mg_bar);
  cudaFree(h->mg_iter);
  cudaFree(h->mg_tact);
  h->mg_tact = nullptr;
  h->mg_bar = nullptr;
  h->mg_iter = nullptr;
  h->mg_lab = nullptr; h->mg_wr = h->mg_wd = h->mg_d = h->mg_invd = h->mg_b = h->mg_e = nullptr;
  h->mg_inc = h->inc0 = nullptr; h->z = nullptr;
  h->mg_cells = 0;
}

// per-phase variant: prologue, then chunks of MGX_CHUNK iterations replayed from
// a CUDA graph until the device says done, then the epilogue
#define MGX_CHUNK 8
template <bool COMP, bool AL>
static ni_status mgx_run(ni_handle* h, const MgArgs& a, cudaStream_t s) {
  const int nt = h->ntiles;
  auto blocks = [&](long long n) { return (int)std::max(1LL, (n + 255) / 256); };
  MgIter* itp = reinterpret_cast<MgIter*>(h->mg_iter);
  cudaMemsetAsync(itp, 0, sizeof(MgIter), s);
  k_mgx_prologue<COMP, AL><<<nt, NI_TILE_THREADS, 0, s>>>(a); NI_COUNT(h);
  if (a.warm) {
    k_mgx_warm_alpha<<<blocks(a.K), 256, 0, s>>>(a); NI_COUNT(h);
    k_mgx_warm<COMP, AL><<<nt, NI_TILE_THREADS, 0, s>>>(a); NI_COUNT(h);
  }
  ni_status rc = ni_cuda_check(h, cudaGetLastError(), "multigrid PCG prologue");
  if (rc != NI_OK) return rc;
  auto cells = [&](int l) { return (long long)a.lh[l] * a.lw[l]; };
  cudaStream_t cs;
  cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  const long long launches_before = h->launches;
  for (int i = 0; i < MGX_CHUNK; ++i) {
    k_mgx_book_down0<<<nt, NI_TILE_THREADS, 0, cs>>>(a, itp); NI_COUNT(h);
    for (int l = 1; l < a.Lc; ++l) { k_mgx_down<<<blocks(cells(l + 1)), 256, 0, cs>>>(a, itp, l); NI_COUNT(h); }
    k_mgx_cta<<<1, NI_TILE_THREADS, 0, cs>>>(a, itp); NI_COUNT(h);
    for (int l = a.Lc - 1; l >= 1; --l) { k_mgx_up<<<blocks(cells(l)), 256, 0, cs>>>(a, itp, l); NI_COUNT(h); }
    k_mgx_up0<COMP, AL><<<nt, NI_TILE_THREADS, 0, cs>>>(a, itp); NI_COUNT(h);
    k_mgx_dir<COMP, AL><<<nt, NI_TILE_THREADS, 0, cs>>>(a, itp); NI_COUNT(h);
    k_mgx_upd<COMP, AL><<<nt, NI_TILE_THREADS, 0, cs>>>(a, itp); NI_COUNT(h);
    k_mgx_next<<<1, 1, 0, cs>>>(a, itp); NI_COUNT(h);
  }
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  const long long per_chunk = h->launches - launches_before;
  h->launches = launches_before;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  rc = ni_cuda_check(h, e, "multigrid PCG graph");
  if (rc == NI_OK) {
    for (int done_it = 0; done_it <= a.maxit; done_it += MGX_CHUNK) {
      cudaGraphLaunch(exec, s);
      h->launches += per_chunk;
      cudaMemcpyAsync(&h->st_host->cg_done, &itp->done, sizeof(int), cudaMemcpyDeviceToHost, s);
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) break;
      if (h->st_host->cg_done) break;
    }
    rc = ni_cuda_check(h, e, "multigrid PCG");
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (rc != NI_OK) return rc;
  k_mgx_epi_sums<<<nt, NI_TILE_THREADS, 0, s>>>(a); NI_COUNT(h);
  k_mgx_epi_apply<<<grid_cells(h, a.N), 256, 0, s>>>(a); NI_COUNT(h);
  return ni_cuda_check(h, cudaGetLastError(), "multigrid PCG epilogue");
}

ni_status mg_solve_launch(ni_handle* h, cudaStream_t s) {
  ni_status rc = ensure_mg(h, s);
  if (rc != NI_OK) return rc;
  const int L = h->mg_L;
  // hierarchy for the current weights
  for (int l = 0; l < L; ++l) {
    LvIn f;
    if (l == 0) {
      f.lab = h->labels; f.wr = h->wr; f.wd = h->wd; f.s = nullptr; f.inc = h->inc0;
    } else {
      const long long o = h->mg_off[l];
      f.lab = h->mg_lab + o; f.wr = h->mg_wr + o; f.wd = h->mg_wd + o; f.s = h->mg_d + o; f.inc = h->mg_inc + o;
    }
    f.H = h->mg_h[l]; f.W = h->mg_w[l];
    const long long oc = h->mg_off[l + 1];
    const int Hc = h->mg_h[l + 1], Wc = h->mg_w[l + 1];
    k_mg_coarsen<<<grid_cells(h, (long long)Hc * Wc), 256, 0, s>>>(f, Hc, Wc, h->mg_lab + oc, h->mg_wr + oc,
                                                                   h->mg_wd + oc, h->mg_d + oc, h->mg_invd + oc);
    NI_COUNT(h);
  }
  const bool f64 = h->cfg.precision == 0;
  const bool aligned = (h->W % 4) == 0;
  void* fn = f64 ? (aligned ? (void*)k_pcg_mg<true, true> : (void*)k_pcg_mg<true, false>)
                 : (aligned ? (void*)k_pcg_mg<false, true> : (void*)k_pcg_mg<false, false>);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NI_TILE_THREADS, 0);
  if (per_sm < 1) return ni_fail(h, NI_ERR_CUDA, "multigrid PCG: kernel cannot be resident");
  const int want = h->cfg.ctas_per_sm > 0 ? h->cfg.ctas_per_sm : 4;
  int grid = h->num_sms * std::min(per_sm, want);
  grid = std::max(1, std::min(grid, h->ntiles));
  cudaMemsetAsync(h->cacc, 0, sizeof(double) * 14 * (size_t)h->Kcap, s);
  cudaMemsetAsync(h->cflag, 0, sizeof(int) * 3 * (size_t)h->Kcap, s);
  cudaMemsetAsync(&h->st->bar, 0, sizeof(GridBar), s);
  int* ntl = h->blk;   // scan scratch is free during the fill: [0] tiles, [2..5] active counts
  cudaMemsetAsync(ntl, 0, 8 * sizeof(int), s);
  MgArgs a;
  a.wr = h->wr; a.wd = h->wd; a.invd = h->invd; a.rhs = h->b; a.labels = h->labels; a.tile_lab = h->tile_lab;
  a.inc0 = h->inc0;
  a.x = h->x; a.r = h->r; a.pb0 = h->p; a.pb1 = h->p2; a.q = h->q; a.z = h->z;
  a.clab = h->mg_lab; a.cwr = h->mg_wr; a.cwd = h->mg_wd; a.cinvd = h->mg_invd; a.cb = h->mg_b; a.ce = h->mg_e;
  a.cinc = h->mg_inc;
  a.L = L;
  // levels Lc..L: the coarsest levels whose cells fit CTA 0's shared arrays
  auto cells = [&](int l) { return (long long)h->mg_h[l] * h->mg_w[l]; };
  int Lc = L;
  long long tail = cells(L);
  while (Lc > 1 && tail + cells(Lc - 1) <= MG_SMEM_CELLS) tail += cells(--Lc);
  a.Lc = Lc;
  const long long per_cta = h->cfg.mg_cta_cells > 0 ? h->cfg.mg_cta_cells : 256;
  int so = 0;
  for (int l = 0; l <= NI_MG_MAX_LEVELS; ++l) {
    a.lh[l] = l <= L ? h->mg_h[l] : 0;
    a.lw[l] = l <= L ? h->mg_w[l] : 0;
    a.loff[l] = l <= L ? h->mg_off[l] : 0;
    a.smo[l] = 0;
    if (l >= Lc && l <= L) { a.smo[l] = so; so += (int)cells(l); }
    a.pd[l] = a.pu[l] = grid;
    if (l >= 1 && l < Lc) {   // the tile-local levels size their passes on the device
      a.pd[l] = (int)std::max(1LL, std::min((long long)grid, (cells(l + 1) + per_cta - 1) / per_cta));
      a.pu[l] = (int)std::max(1LL, std::min((long long)grid, (cells(l) + per_cta - 1) / per_cta));
    }
  }
  a.mbar = h->mg_bar;
  cudaMemsetAsync(h->mg_bar, 0, sizeof(GridBar) * 2 * (NI_MG_MAX_LEVELS + 1), s);
  a.cs = h->cacc; a.ci = h->cflag; a.tiles = reinterpret_cast<int2*>(h->tiles); a.ntl = ntl; a.st = h->st;
  a.tact = h->mg_tact;
  a.per = (int)per_cta;
  a.N = h->N; a.H = h->H; a.W = h->W; a.K = h->K_host; a.Kc = h->Kcap; a.ntiles = h->ntiles; a.ntx = h->ntx;
  // the multigrid PCG converges in tens to hundreds of iterations; a component
  // still above the tolerance after NI_MG_MAXIT goes to the Jacobi fallback
  a.maxit = std::min(h->cfg.cg_maxit, NI_MG_MAXIT); a.warm = h->cfg.warm_start ? 1 : 0;
  a.ncs = h->cfg.mg_coarse_sweeps > 0 ? h->cfg.mg_coarse_sweeps : 4;
  a.project = (h->cfg.mg_flags & 1) ? 1 : 0;
  a.om = h->cfg.mg_omega > 0 ? (float)h->cfg.mg_omega : 0.9f;
  a.sc = h->cfg.mg_correction > 0 ? (float)h->cfg.mg_correction : 1.0f;
  a.tol2 = h->cfg.cg_rtol * h->cfg.cg_rtol;
  if (h->cfg.fill_kernels == 0) {
    if (f64) return aligned ? mgx_run<true, true>(h, a, s) : mgx_run<true, false>(h, a, s);
    return aligned ? mgx_run<false, true>(h, a, s) : mgx_run<false, false>(h, a, s);
  }
  void* args[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(NI_TILE_THREADS), args, 0, s);
  NI_COUNT(h);
  return ni_cuda_check(h, e, "multigrid PCG launch");
}
