// C ABI of libni: handle life cycle, Algorithm 1 orchestration, CUDA graph of
// the relative-scale loop, statistics.  All arithmetic runs in the kernels of
// ni_seed.cu, ni_fill.cu and ni_scale.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "../../include/ni_cnn.h"
#include "ni_internal.cuh"

ni_status ni_fail(ni_handle* h, ni_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

ni_status ni_cuda_check(ni_handle* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return NI_OK;
  (void)cudaGetLastError();
  return ni_fail(h, e == cudaErrorMemoryAllocation ? NI_ERR_OOM : NI_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

template <class T>
static cudaError_t dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMalloc((void**)p, n * sizeof(T));
}

template <class T>
static void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

extern "C" void ni_config_default(ni_config* c, int H, int W) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->H = H;
  c->W = W;
  c->cam.camera = 1;
  c->cam.fx = c->cam.fy = 1.5 * (W > 0 ? W : 1);
  c->cam.cx = W / 2.0;
  c->cam.cy = H / 2.0;
  c->theta_c_deg = 3.5;
  c->connectivity = 4;
  c->k = 2.0;
  c->L = 1e-5;
  c->U = 1e-3;
  c->T = 15;
  c->dE_max = 1e-3;
  c->can_merge = 0;
  c->freq_merging = 5;
  c->n_fill_irls = 1;
  c->cg_rtol = 1e-6;
  c->cg_maxit = 20000;
  c->scale_rtol = 1e-12;
  c->scale_maxit = 0;
  c->precision = 0;
  c->batched = 1;
  c->use_graph = 1;
  c->warm_start = 0;
  c->precond = 1;
  c->mg_omega = 0;
  c->mg_correction = 0;
  c->mg_cta_cells = 0;
  c->mg_flags = 0;
  c->fill_kernels = 1;
  c->hard_outliers = 0;
  c->validate = 1;
}

static ni_status check_config(const ni_config* c, std::string& why) {
  if (c->H < 1 || c->W < 1) { why = "H and W must be >= 1"; return NI_ERR_INVALID_ARG; }
  if ((long long)c->H * c->W >= (1LL << 30)) { why = "H * W must be < 2^30"; return NI_ERR_INVALID_ARG; }
  if (c->connectivity != 4 && c->connectivity != 8) { why = "connectivity must be 4 or 8"; return NI_ERR_INVALID_ARG; }
  if (c->connectivity == 8 && (long long)c->H * c->W >= (1LL << 29)) {
    why = "8-connectivity needs H * W < 2^29 (edge ids 4 a + dir)"; return NI_ERR_INVALID_ARG;
  }
  if (c->connectivity == 8 && c->batched) {
    why = "8-connectivity runs the plain fill PCG: set batched = 0"; return NI_ERR_INVALID_ARG;
  }
  if (c->cam.camera != 0 && c->cam.camera != 1) { why = "camera must be 0 or 1"; return NI_ERR_INVALID_ARG; }
  if (c->cam.camera == 1 && !(c->cam.fx > 0 && c->cam.fy > 0)) {
    why = "focal lengths must be > 0"; return NI_ERR_INVALID_ARG;
  }
  if (c->T < 1 || c->T > NI_MAX_T) { why = "T must be in [1, 256]"; return NI_ERR_INVALID_ARG; }
  if (c->freq_merging < 1) { why = "freq_merging must be >= 1"; return NI_ERR_INVALID_ARG; }
  if (!(c->L > 0 && c->U > c->L)) { why = "need 0 < L < U"; return NI_ERR_INVALID_ARG; }
  if (!(c->cg_rtol > 0) || c->cg_maxit < 1) { why = "bad fill CG tolerance"; return NI_ERR_INVALID_ARG; }
  if (!(c->scale_rtol > 0)) { why = "bad scale CG tolerance"; return NI_ERR_INVALID_ARG; }
  if (c->n_fill_irls < 1 || c->n_fill_irls > 16) { why = "n_fill_irls in [1, 16]"; return NI_ERR_INVALID_ARG; }
  if (c->precision != 0 && c->precision != 1) { why = "precision must be 0 or 1"; return NI_ERR_INVALID_ARG; }
  if (!(c->dE_max >= 0)) { why = "dE_max must be >= 0"; return NI_ERR_INVALID_ARG; }
  if (c->precond != 0 && c->precond != 1) { why = "precond must be 0 or 1"; return NI_ERR_INVALID_ARG; }
  if (!(c->mg_omega >= 0 && c->mg_omega < 1)) { why = "mg_omega must be in [0, 1)"; return NI_ERR_INVALID_ARG; }
  if (!(c->mg_correction >= 0 && c->mg_correction <= 3)) { why = "mg_correction must be in [0, 3]"; return NI_ERR_INVALID_ARG; }
  if (c->ctas_per_sm < 0 || c->ctas_per_sm > 8) { why = "ctas_per_sm in [0, 8]"; return NI_ERR_INVALID_ARG; }
  if (c->mg_coarse_sweeps < 0 || c->mg_coarse_sweeps > 64) { why = "mg_coarse_sweeps in [0, 64]"; return NI_ERR_INVALID_ARG; }
  if (c->fill_kernels != 0 && c->fill_kernels != 1) { why = "fill_kernels must be 0 or 1"; return NI_ERR_INVALID_ARG; }
  if (c->scale_solver < 0 || c->scale_solver > 2) { why = "scale_solver must be 0, 1 or 2"; return NI_ERR_INVALID_ARG; }
  if (c->bini_residual != 0 && c->bini_residual != 1) { why = "bini_residual must be 0 or 1"; return NI_ERR_INVALID_ARG; }
  if (c->learned_weights != 0 && c->learned_weights != 1) { why = "learned_weights must be 0 or 1"; return NI_ERR_INVALID_ARG; }
  if (c->learned_weights && !c->warm_start) { why = "learned_weights needs warm_start = 1"; return NI_ERR_INVALID_ARG; }
  if (c->mg_cta_cells < 0) { why = "mg_cta_cells must be >= 0"; return NI_ERR_INVALID_ARG; }
  if (c->warm_start && !c->batched) { why = "warm_start needs the batched fill (batched = 1)"; return NI_ERR_INVALID_ARG; }
  return NI_OK;
}

static void release_components(ni_handle* h) {
  dfree(h->soff); dfree(h->soff2); dfree(h->cacc); dfree(h->cflag); dfree(h->kparent);
  dfree(h->kmap); dfree(h->kkey); dfree(h->sv); dfree(h->sd); dfree(h->row_ptr);
  h->Kcap = 0;
}

static void release_edges(ni_handle* h) {
  dfree(h->e_id); dfree(h->e_id2); dfree(h->e_key); dfree(h->e_key2); dfree(h->e_val);
  dfree(h->e_val2); dfree(h->e_pair); dfree(h->p_lo); dfree(h->p_hi); dfree(h->p_acc);
  dfree(h->c_key); dfree(h->c_val); dfree(h->csr_col); dfree(h->csr_pair); dfree(h->csr_w);
  h->Ecap = 0;
}

ni_status ensure_component_capacity(ni_handle* h, int K) {
  int need = std::max(K, 16);
  if (need <= h->Kcap) return NI_OK;
  release_components(h);
  cudaError_t e = cudaSuccess;
  size_t k = (size_t)need;
  if (e == cudaSuccess) e = dalloc(&h->soff, k);
  if (e == cudaSuccess) e = dalloc(&h->soff2, k);
  if (e == cudaSuccess) e = dalloc(&h->cacc, 14 * k + 16);
  if (e == cudaSuccess) e = dalloc(&h->cflag, 3 * k);
  if (e == cudaSuccess) e = dalloc(&h->kparent, k);
  if (e == cudaSuccess) e = dalloc(&h->kmap, k);
  if (e == cudaSuccess) e = dalloc(&h->kkey, k);
  if (e == cudaSuccess) e = dalloc(&h->sv, 11 * k);
  if (e == cudaSuccess) e = dalloc(&h->sd, k);
  if (e == cudaSuccess) e = dalloc(&h->row_ptr, k + 1);
  if (e != cudaSuccess) {
    release_components(h);
    return ni_cuda_check(h, e, "component buffers");
  }
  h->Kcap = need;
  // radix passes for keys lo * K + hi < Kcap^2
  double bits = 2.0 * log2((double)std::max(need, 2));
  h->sort_passes = std::max(1, (int)ceil(bits / 8.0));
  return NI_OK;
}

ni_status ensure_edge_capacity(ni_handle* h, int nE) {
  int need = std::max(nE, 16);
  if (need <= h->Ecap) return NI_OK;
  release_edges(h);
  size_t n = (size_t)need;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = dalloc(&h->e_id, n);
  if (e == cudaSuccess) e = dalloc(&h->e_id2, n);
  if (e == cudaSuccess) e = dalloc(&h->e_key, 2 * n);
  if (e == cudaSuccess) e = dalloc(&h->e_key2, 2 * n);
  if (e == cudaSuccess) e = dalloc(&h->e_val, 2 * n);
  if (e == cudaSuccess) e = dalloc(&h->e_val2, 2 * n);
  if (e == cudaSuccess) e = dalloc(&h->e_pair, n);
  if (e == cudaSuccess) e = dalloc(&h->p_lo, n);
  if (e == cudaSuccess) e = dalloc(&h->p_hi, n);
  if (e == cudaSuccess) e = dalloc(&h->p_acc, 3 * n);
  if (e == cudaSuccess) e = dalloc(&h->c_key, 2 * n);
  if (e == cudaSuccess) e = dalloc(&h->c_val, 2 * n);
  if (e == cudaSuccess) e = dalloc(&h->csr_col, 2 * n);
  if (e == cudaSuccess) e = dalloc(&h->csr_pair, 2 * n);
  if (e == cudaSuccess) e = dalloc(&h->csr_w, 2 * n);
  if (e != cudaSuccess) {
    release_edges(h);
    return ni_cuda_check(h, e, "edge buffers");
  }
  h->Ecap = need;
  return NI_OK;
}

static void destroy_graph(ni_handle* h) {
  if (h->scale_graph) cudaGraphExecDestroy(h->scale_graph);
  h->scale_graph = nullptr;
  for (int i = 0; i < 6; ++i) h->graph_key[i] = -1;
}

extern "C" ni_status ni_create(const ni_config* cfg, ni_handle** out) {
  if (!out) return NI_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg) return NI_ERR_INVALID_ARG;
  std::string why;
  if (check_config(cfg, why) != NI_OK) return NI_ERR_INVALID_ARG;
  ni_handle* h = new ni_handle();
  h->cfg = *cfg;
  h->cfg_user = *cfg;
  h->H = cfg->H;
  h->W = cfg->W;
  h->N = cfg->H * cfg->W;
  h->persp = cfg->cam.camera == 1;
  h->fx = (float)cfg->cam.fx; h->fy = (float)cfg->cam.fy;
  h->cx = (float)cfg->cam.cx; h->cy = (float)cfg->cam.cy;
  if (!h->persp) { h->fx = h->fy = 1.f; h->cx = h->cy = 0.f; }
  h->cos_theta = cfg->theta_c_deg < 0 ? 2.0 : cos(cfg->theta_c_deg * (M_PI / 180.0));
  cudaError_t e = cudaGetDevice(&h->dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->dev);
  h->ntx = (h->W + NI_TILE_W - 1) / NI_TILE_W;
  h->ntiles = h->ntx * ((h->H + NI_TILE_H - 1) / NI_TILE_H);
  h->Npad = (h->N + NI_TILE_PX - 1) / NI_TILE_PX * NI_TILE_PX;
  const size_t N = (size_t)h->N, NP = (size_t)h->Npad;
  if (e == cudaSuccess) e = dalloc(&h->labels, NP);
  if (e == cudaSuccess) e = dalloc(&h->parent, N);
  if (e == cudaSuccess) e = dalloc(&h->omega, N);
  if (e == cudaSuccess) e = dalloc(&h->ntau, N);
  if (e == cudaSuccess) e = dalloc(&h->wr, NP);
  if (e == cudaSuccess) e = dalloc(&h->wd, NP);
  if (e == cudaSuccess) e = dalloc(&h->invd, NP);
  if (e == cudaSuccess) e = dalloc(&h->x, NP);
  if (e == cudaSuccess) e = dalloc(&h->r, NP);
  if (e == cudaSuccess) e = dalloc(&h->p, NP);
  if (e == cudaSuccess) e = dalloc(&h->p2, NP);
  if (e == cudaSuccess) e = dalloc(&h->q, NP);
  if (e == cudaSuccess) e = dalloc(&h->b, NP);
  if (cfg->connectivity == 8) {
    if (e == cudaSuccess) e = dalloc(&h->omega_d, N);
    if (e == cudaSuccess) e = dalloc(&h->wdr, NP);
    if (e == cudaSuccess) e = dalloc(&h->wdl, NP);
    if (e == cudaSuccess) e = cudaMemset(h->wdr, 0, NP * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(h->wdl, 0, NP * sizeof(float));
  }
  if (e == cudaSuccess) e = dalloc(&h->tile_lab, (size_t)h->ntiles);
  if (e == cudaSuccess) e = dalloc(&h->tiles, 4 * (size_t)h->ntiles);
  // padding pixels beyond N: label -1, weights and vectors 0 (never written later)
  if (e == cudaSuccess) e = cudaMemset(h->labels, 0xff, NP * sizeof(int32_t));
  float* zero_planes[] = {h->wr, h->wd, h->invd, h->x, h->r, h->p, h->p2, h->q, h->b};
  for (float* zp : zero_planes)
    if (e == cudaSuccess) e = cudaMemset(zp, 0, NP * sizeof(float));
  if (e == cudaSuccess) e = dalloc(&h->blk, NI_SCAN_BLOCKS + 1);
  if (e == cudaSuccess) e = dalloc(&h->d_count, 16);
  if (e == cudaSuccess) e = dalloc(&h->radix_hist, 256 * NI_SORT_BLOCKS);
  if (e == cudaSuccess) e = dalloc(&h->st, 1);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->st_host, sizeof(DevState));
  for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreate(&h->ev[i]);
  if (e != cudaSuccess) {
    ni_destroy(h);
    return e == cudaErrorMemoryAllocation ? NI_ERR_OOM : NI_ERR_CUDA;
  }
  *out = h;
  return NI_OK;
}

extern "C" ni_status ni_destroy(ni_handle* h) {
  if (!h) return NI_OK;
  destroy_graph(h);
  release_components(h);
  release_edges(h);
  dfree(h->labels); dfree(h->parent); dfree(h->omega); dfree(h->ntau); dfree(h->wr); dfree(h->wd);
  dfree(h->omega_d); dfree(h->wdr); dfree(h->wdl);
  dfree(h->tile_lab); dfree(h->tiles);
  dfree(h->invd); dfree(h->x); dfree(h->r); dfree(h->p); dfree(h->p2); dfree(h->q); dfree(h->b);
  dfree(h->blk); dfree(h->d_count); dfree(h->radix_hist); dfree(h->st);
  dfree(h->in_normals); dfree(h->in_mask); dfree(h->out_depth);
  dfree(h->tile_in); dfree(h->tile_out); dfree(h->lw);
  free_mg(h);
  free_made(h);
  if (h->net) ni_cnn_destroy(h->net);
  if (h->st_host) cudaFreeHost(h->st_host);
  for (int i = 0; i < 8; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  delete h;
  return NI_OK;
}

extern "C" const char* ni_last_error(const ni_handle* h) { return h ? h->err.c_str() : ""; }

extern "C" const char* ni_status_string(ni_status s) {
  switch (s) {
    case NI_OK: return "NI_OK";
    case NI_ERR_INVALID_ARG: return "NI_ERR_INVALID_ARG";
    case NI_ERR_CUDA: return "NI_ERR_CUDA";
    case NI_ERR_OOM: return "NI_ERR_OOM";
    case NI_ERR_NOT_CONVERGED: return "NI_ERR_NOT_CONVERGED";
    case NI_ERR_TIMEOUT: return "NI_ERR_TIMEOUT";
    case NI_ERR_STATE: return "NI_ERR_STATE";
    case NI_ERR_NO_NET: return "NI_ERR_NO_NET";
  }
  return "NI_ERR_UNKNOWN";
}

static ni_status pull_state(ni_handle* h, cudaStream_t s) {
  cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
  return ni_cuda_check(h, cudaStreamSynchronize(s), "device state");
}

static ni_status dev_errors(ni_handle* h) {
  const int err = h->st_host->err;
  if (err & NI_DEV_ERR_TIMEOUT) return ni_fail(h, NI_ERR_TIMEOUT, "a bounded device-side wait timed out");
  return NI_OK;
}

// ---------------------------------------------------------------------------
// stages
// ---------------------------------------------------------------------------
extern "C" ni_status ni_seed_components(ni_handle* h, const float* normals, const uint8_t* mask,
                                        int32_t* labels_out, int32_t* K_out, ni_stream_t stream) {
  if (!h) return NI_ERR_INVALID_ARG;
  if (!normals || !mask) return ni_fail(h, NI_ERR_INVALID_ARG, "normals and mask are required");
  if (((uintptr_t)normals) & 15) return ni_fail(h, NI_ERR_INVALID_ARG, "normals must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  h->err.clear();
  h->normals = reinterpret_cast<const float4*>(normals);
  h->mask = mask;
  cudaMemsetAsync(h->st, 0, sizeof(DevState), s);
  ni_status rc = seed_launch(h, s);
  if (rc != NI_OK) return rc;
  rc = pull_state(h, s);
  if (rc != NI_OK) return rc;
  if (h->st_host->err & NI_DEV_ERR_BAD_NORMAL)
    return ni_fail(h, NI_ERR_INVALID_ARG,
                   std::to_string(h->st_host->n_bad_normals) +
                       " valid pixels have normals that are not unit length within 1e-3 or have n.tau = 0");
  h->K_host = h->st_host->K;
  rc = ensure_component_capacity(h, h->K_host);
  if (rc != NI_OK) return rc;
  if (labels_out) cudaMemcpyAsync(labels_out, h->labels, sizeof(int32_t) * h->N, cudaMemcpyDeviceToDevice, s);
  if (K_out) *K_out = h->K_host;
  h->stage = 1;
  h->t_host = 0;
  destroy_graph(h);
  return ni_cuda_check(h, cudaStreamSynchronize(s), "seeding");
}

// The knobs the caller left at 0 (auto) take the first tuning-table row that
// covers this map's grid pixels and its number of components after seeding.
static void apply_tuning(ni_handle* h) {
  if (h->tune.empty()) return;
  const TuneRow* r = nullptr;
  for (const TuneRow& t : h->tune)
    if ((long long)h->N <= t.max_px && (long long)h->K_host <= t.max_k0) { r = &t; break; }
  const ni_config& u = h->cfg_user;
  h->cfg.ctas_per_sm = (r && u.ctas_per_sm == 0) ? r->ctas_per_sm : u.ctas_per_sm;
  h->cfg.mg_cta_cells = (r && u.mg_cta_cells == 0) ? r->mg_cta_cells : u.mg_cta_cells;
  h->cfg.mg_omega = (r && u.mg_omega == 0) ? r->mg_omega : u.mg_omega;
  h->cfg.scale_solver = (r && u.scale_solver == 0) ? r->scale_solver : u.scale_solver;
}

extern "C" ni_status ni_load_tuning(ni_handle* h, const char* path) {
  if (!h) return NI_ERR_INVALID_ARG;
  if (!path) return ni_fail(h, NI_ERR_INVALID_ARG, "path is required");
  FILE* f = fopen(path, "r");
  if (!f) return ni_fail(h, NI_ERR_INVALID_ARG, std::string("cannot open ") + path);
  std::vector<TuneRow> rows;
  char line[512];
  bool ok = true;
  while (fgets(line, sizeof line, f)) {
    const char* p = line;
    while (*p == ' ' || *p == '\t') ++p;
    if (*p == '#' || *p == '\n' || *p == '\0') continue;
    TuneRow t;
    if (sscanf(p, "%lld %lld %d %d %lf %d", &t.max_px, &t.max_k0, &t.ctas_per_sm, &t.mg_cta_cells, &t.mg_omega,
               &t.scale_solver) != 6 ||
        t.max_px < 1 || t.max_k0 < 1 || t.ctas_per_sm < 0 || t.ctas_per_sm > 8 || t.mg_cta_cells < 0 ||
        !(t.mg_omega >= 0 && t.mg_omega < 1) || t.scale_solver < 0 || t.scale_solver > 2) {
      ok = false;
      break;
    }
    rows.push_back(t);
  }
  fclose(f);
  if (!ok || rows.empty()) return ni_fail(h, NI_ERR_INVALID_ARG, std::string("malformed tuning table ") + path);
  h->tune = rows;
  return NI_OK;
}

extern "C" ni_status ni_solve_components(ni_handle* h, float* logdepth_out, ni_stream_t stream) {
  if (!h) return NI_ERR_INVALID_ARG;
  if (h->stage < 1) return ni_fail(h, NI_ERR_STATE, "ni_solve_components before ni_seed_components");
  apply_tuning(h);
  if (h->cfg.warm_start && !h->net)
    return ni_fail(h, NI_ERR_NO_NET, "warm start requested but no network is loaded");
  cudaStream_t s = (cudaStream_t)stream;
  h->err.clear();
  h->fill_fallbacks = 0;
  ni_status rc = fill_setup_launch(h, s);
  if (rc != NI_OK) return rc;
  cudaMemsetAsync(h->x, 0, sizeof(float) * h->N, s);
  if (h->cfg.warm_start) {
    rc = warm_start_launch(h, s);
    if (rc != NI_OK) return rc;
  }
  cudaMemsetAsync(h->soff, 0, sizeof(double) * h->Kcap, s);
  rc = fill_solve_launch(h, s);
  if (rc != NI_OK) return rc;
  rc = partition_build_launch(h, 1, s);
  if (rc != NI_OK) return rc;
  if (logdepth_out) export_logdepth_launch(h, logdepth_out, s);
  rc = pull_state(h, s);
  if (rc != NI_OK) return rc;
  h->ms_fill_solve = 0.f;
  cudaEventElapsedTime(&h->ms_fill_solve, h->ev[5], h->ev[6]);
  rc = dev_errors(h);
  if (rc != NI_OK) return rc;
  h->stage = 2;
  h->t_host = 0;
  if (h->st_host->err & NI_DEV_ERR_FILL_NOCONV)
    return ni_fail(h, NI_ERR_NOT_CONVERGED,
                   std::to_string(h->st_host->fill_unconv) + " component fills reached cg_maxit");
  return NI_OK;
}

static ni_status enqueue_scale_loop(ni_handle* h, int iters, int t0, cudaStream_t s) {
  for (int i = 0; i < iters; ++i) {
    const int tp = t0 + i + 1;
    ni_status rc = scale_iteration_launch(h, s);
    if (rc != NI_OK) return rc;
    if (h->cfg.can_merge && tp % h->cfg.freq_merging == 0) {
      merge_gate_launch(h, tp, 0, s);
      rc = merge_launch(h, nullptr, s);
      if (rc != NI_OK) return rc;
    }
  }
  return NI_OK;
}

static ni_status run_scale_loop(ni_handle* h, int iters, cudaStream_t s) {
  const int t0 = h->t_host;
  if (!h->cfg.use_graph) return enqueue_scale_loop(h, iters, t0, s);
  long long key[6] = {h->Kcap, h->Ecap, iters, t0, h->cfg.can_merge, h->cfg.freq_merging};
  bool same = h->scale_graph != nullptr;
  for (int i = 0; i < 6; ++i) same = same && key[i] == h->graph_key[i];
  if (!same) {
    destroy_graph(h);
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return ni_cuda_check(h, e, "capture stream");
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    ni_status rc = NI_OK;
    const long long before = h->launches;
    if (e == cudaSuccess) rc = enqueue_scale_loop(h, iters, t0, cs);
    const long long captured = h->launches - before;
    h->launches = before;
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess && rc == NI_OK) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (rc != NI_OK || e != cudaSuccess || !ex) {
      (void)cudaGetLastError();
      if (ex) cudaGraphExecDestroy(ex);
      // capture is an optimisation: run the same work directly
      return enqueue_scale_loop(h, iters, t0, s);
    }
    h->scale_graph = ex;
    h->scale_graph_count = captured;
    for (int i = 0; i < 6; ++i) h->graph_key[i] = key[i];
  }
  h->launches += h->scale_graph_count;
  return ni_cuda_check(h, cudaGraphLaunch(h->scale_graph, s), "scale loop graph");
}

extern "C" ni_status ni_solve_scales(ni_handle* h, int max_iters, float* logdepth_inout, double* energy_out,
                                     int* iters_done, ni_stream_t stream) {
  if (!h) return NI_ERR_INVALID_ARG;
  if (h->stage < 2) return ni_fail(h, NI_ERR_STATE, "ni_solve_scales before ni_solve_components");
  if (max_iters < 0) return ni_fail(h, NI_ERR_INVALID_ARG, "max_iters < 0");
  cudaStream_t s = (cudaStream_t)stream;
  h->err.clear();
  if (logdepth_inout) import_logdepth_launch(h, logdepth_inout, s);
  const int t_before = h->t_host;
  max_iters = std::min(max_iters, h->cfg.T - t_before);
  ni_status rc = NI_OK;
  if (max_iters > 0) rc = run_scale_loop(h, max_iters, s);
  if (rc != NI_OK) return rc;
  if (logdepth_inout) export_logdepth_launch(h, logdepth_inout, s);
  rc = pull_state(h, s);
  if (rc != NI_OK) return rc;
  const int t_after = h->st_host->t;
  h->t_host = t_after;
  h->K_host = h->st_host->K;
  if (iters_done) *iters_done = t_after - t_before;
  if (energy_out)
    for (int t = t_before + 1; t <= t_after && t <= NI_MAX_T; ++t) energy_out[t - t_before - 1] = h->st_host->E[t];
  // later calls continue the same schedule; the graph key includes t_before
  return dev_errors(h);
}

static ni_status merge_common(ni_handle* h, const float* chi_abs, int32_t* labels_out, int32_t* K_out,
                              cudaStream_t s) {
  if (h->stage < 2) return ni_fail(h, NI_ERR_STATE, "ni_merge before ni_solve_components");
  h->err.clear();
  merge_gate_launch(h, 0, 1, s);
  ni_status rc = merge_launch(h, chi_abs, s);
  if (rc != NI_OK) return rc;
  if (labels_out) cudaMemcpyAsync(labels_out, h->labels, sizeof(int32_t) * h->N, cudaMemcpyDeviceToDevice, s);
  rc = pull_state(h, s);
  if (rc != NI_OK) return rc;
  h->K_host = h->st_host->K;
  if (K_out) *K_out = h->K_host;
  destroy_graph(h);
  return dev_errors(h);
}

extern "C" ni_status ni_merge(ni_handle* h, int32_t* labels_out, int32_t* K_out, ni_stream_t stream) {
  if (!h) return NI_ERR_INVALID_ARG;
  return merge_common(h, nullptr, labels_out, K_out, (cudaStream_t)stream);
}

extern "C" ni_status ni_merge_residuals(ni_handle* h, const float* chi_abs, int32_t* labels_out, int32_t* K_out,
                                        ni_stream_t stream) {
  if (!h) return NI_ERR_INVALID_ARG;
  if (!chi_abs) return ni_fail(h, NI_ERR_INVALID_ARG, "chi_abs is required");
  return merge_common(h, chi_abs, labels_out, K_out, (cudaStream_t)stream);
}

extern "C" ni_status ni_integrate(ni_handle* h, const float* normals, const uint8_t* mask, float* depth_out,
                                  int32_t* labels_out, ni_stats* stats, ni_stream_t stream) {
  if (!h) return NI_ERR_INVALID_ARG;
  if (!depth_out) return ni_fail(h, NI_ERR_INVALID_ARG, "depth_out is required");
  cudaStream_t s = (cudaStream_t)stream;
  const long long launches0 = h->launches;
  cudaEventRecord(h->ev[0], s);
  ni_status rc = ni_seed_components(h, normals, mask, nullptr, nullptr, stream);
  if (rc != NI_OK) return rc;
  cudaEventRecord(h->ev[1], s);
  rc = ni_solve_components(h, nullptr, stream);
  if (rc != NI_OK && rc != NI_ERR_NOT_CONVERGED) return rc;
  ni_status fill_rc = rc;
  std::string fill_msg = h->err;
  cudaEventRecord(h->ev[2], s);
  rc = ni_solve_scales(h, h->cfg.T, nullptr, nullptr, nullptr, stream);
  if (rc != NI_OK) return rc;
  cudaEventRecord(h->ev[3], s);
  output_depth_launch(h, depth_out, s);
  NI_COUNT(h);
  if (labels_out) cudaMemcpyAsync(labels_out, h->labels, sizeof(int32_t) * h->N, cudaMemcpyDeviceToDevice, s);
  cudaEventRecord(h->ev[4], s);
  rc = pull_state(h, s);
  if (rc != NI_OK) return rc;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]); stats->ms_seed = ms;
    cudaEventElapsedTime(&ms, h->ev[1], h->ev[2]); stats->ms_fill = ms;
    cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]); stats->ms_scale = ms;
    cudaEventElapsedTime(&ms, h->ev[3], h->ev[4]); stats->ms_output = ms;
    cudaEventElapsedTime(&ms, h->ev[0], h->ev[4]); stats->ms_total = ms;
    const DevState* d = h->st_host;
    stats->n_valid = d->n_valid;
    stats->K0 = d->K0;
    stats->K_final = d->K;
    stats->merges = d->merges;
    stats->scale_iters = d->t;
    stats->fill_iters = d->fill_iters;
    stats->fill_unconverged = d->fill_unconv;
    stats->scale_cg_iters = d->scale_cg_iters;
    stats->n_energy = std::min(d->t, 64);
    for (int t = 1; t <= stats->n_energy; ++t) stats->energy[t - 1] = d->E[t];
    stats->ms_fill_solve = h->ms_fill_solve;
    stats->fill_px_iters = (int64_t)d->fill_px_iters;
    stats->kernel_launches = h->launches - launches0;
    stats->warm_fallbacks = d->warm_fallbacks;
    stats->fill_fallbacks = h->fill_fallbacks;
    stats->scale_cg_total = (int64_t)d->scale_cg_total;
  }
  if (fill_rc != NI_OK) return ni_fail(h, fill_rc, fill_msg);
  return NI_OK;
}

extern "C" ni_status ni_integrate_host(ni_handle* h, const float* normals_host, const uint8_t* mask_host,
                                       float* depth_host, ni_stats* stats, ni_stream_t stream) {
  if (!h) return NI_ERR_INVALID_ARG;
  if (!normals_host || !mask_host || !depth_host) return ni_fail(h, NI_ERR_INVALID_ARG, "null host buffer");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)h->N;
  cudaError_t e = cudaSuccess;
  if (!h->in_normals) e = dalloc(&h->in_normals, N);
  if (e == cudaSuccess && !h->in_mask) e = dalloc(&h->in_mask, N);
  if (e == cudaSuccess && !h->out_depth) e = dalloc(&h->out_depth, N);
  if (e != cudaSuccess) return ni_cuda_check(h, e, "host-path buffers");
  cudaMemcpyAsync(h->in_normals, normals_host, N * sizeof(float4), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->in_mask, mask_host, N, cudaMemcpyHostToDevice, s);
  ni_status rc = ni_integrate(h, reinterpret_cast<const float*>(h->in_normals), h->in_mask, h->out_depth,
                              nullptr, stats, stream);
  if (rc != NI_OK && rc != NI_ERR_NOT_CONVERGED) return rc;
  cudaMemcpyAsync(depth_host, h->out_depth, N * sizeof(float), cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ni_cuda_check(h, e, "host-path copy");
  return rc;
}

extern "C" ni_status ni_get_logdepth(ni_handle* h, float* out, ni_stream_t stream) {
  if (!h) return NI_ERR_INVALID_ARG;
  if (!out) return ni_fail(h, NI_ERR_INVALID_ARG, "logdepth_out is required");
  if (h->stage < 2) return ni_fail(h, NI_ERR_STATE, "no log-depth before ni_solve_components");
  cudaStream_t s = (cudaStream_t)stream;
  export_logdepth_launch(h, out, s);
  return ni_cuda_check(h, cudaStreamSynchronize(s), "log-depth export");
}

