/*
 * ni.h - C ABI of the GB300 (sm_103a) continuous-component normal integration
 * library (arXiv 2510.11508, "Towards Fast and Scalable Normal Integration
 * using Continuous Components").
 *
 * Problem (Sec. 3.1): reconstruct a depth map from a surface normal map and a
 * validity mask, given pinhole intrinsics (f_x, f_y, c_x, c_y).  The method
 * (Algorithm 1 of the supplementary pseudocode) is
 *   (a) seeding: connected components of the pixel graph after dropping every
 *       edge whose normals differ by theta_c or more (Sec. 3.3);
 *   (b) filling: per-component weighted least squares of the log-depth model
 *       of continuity (Eqs. 3, 9, 10), solved by preconditioned CG;
 *   (c) relative scales: one log-scale per component from the inter-component
 *       edges with BiNI and outlier weights (Eqs. 12-14, 11);
 *   (d) merging: every component joins the neighbour across its smallest
 *       residual edge (Sec. 3.5).
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller unless the name
 *    says `host`.  Layout is row-major [H][W] (pixel (u, v) = column u, row v
 *    at index v * W + u).  Normals are float[H][W][4] = (n_x, n_y, n_z, unused)
 *    and must be 16-byte aligned; the mask is uint8[H][W], nonzero = valid.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    queued on it asynchronously; calls that return a host scalar (K_out,
 *    iters_done, stats) synchronise that stream before returning.
 *  - Errors are returned as ni_status, never by aborting.  ni_last_error()
 *    gives a message.  A CUDA error is reported as NI_ERR_CUDA.
 *  - The handle owns all scratch memory (allocated by ni_create and, for
 *    component- and edge-sized buffers, on first use) and any CUDA graphs.
 *    A handle must not be used from two host threads at once.
 *  - Stage calls must follow Algorithm 1's order (seed, solve_components,
 *    solve_scales, with ni_merge allowed after solve_components); otherwise
 *    NI_ERR_STATE.
 */
#ifndef NI_H_
#define NI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ni_stream_t; /* same type as cudaStream_t */
typedef struct ni_handle ni_handle;

typedef enum {
  NI_OK = 0,
  NI_ERR_INVALID_ARG = 1,   /* bad size, pointer, alignment, parameter or normal */
  NI_ERR_CUDA = 2,          /* a CUDA runtime call or kernel failed */
  NI_ERR_OOM = 3,           /* device allocation failed */
  NI_ERR_NOT_CONVERGED = 4, /* a CG hit its iteration limit (result still written) */
  NI_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up (result invalid) */
  NI_ERR_STATE = 6,         /* stage call out of Algorithm 1's order */
  NI_ERR_NO_NET = 7         /* warm start requested without a loaded network */
} ni_status;

/* Pinhole camera (Sec. 3.1, Eq. 2): camera = 1 perspective with focal lengths
 * fx, fy and principal point (cx, cy); camera = 0 orthographic (unit pixel
 * pitch, depth is linear instead of logarithmic; fx..cy are ignored). */
typedef struct {
  int camera;
  double fx, fy, cx, cy;
} ni_camera;

typedef struct {
  int H, W;                 /* grid size; 1 <= H, W and H * W < 2^30 */
  ni_camera cam;
  double theta_c_deg;       /* seeding threshold theta_c (Sec. 3.3); < 0 = None (one
                               component per pixel, the paper's pixel-level limit) */
  int connectivity;         /* 4 (default) or 8 (H * W < 2^29, batched = 0): pixel
                               graph of every stage (8 adds the lower-right and
                               lower-left edges; the fill then runs the plain
                               PCG with a 9-point stencil) */
  double k;                 /* sigmoid sharpness of the BiNI weight (Sec. 3.1), default 2 */
  double L, U;              /* outlier thresholds of Eq. 11, default 1e-5, 1e-3 */
  int T;                    /* maximum relative-scale iterations, default 15 */
  double dE_max;            /* relative energy change that stops the loop, default 1e-3;
                               0 runs exactly T iterations */
  int can_merge;            /* merge every freq_merging iterations (Sec. 3.5) */
  int freq_merging;         /* default 5 */
  int n_fill_irls;          /* BiNI reweighting sweeps of the fill, default 1 */
  double cg_rtol;           /* fill PCG: stop a component when ||r_c|| <= rtol ||b_c|| */
  int cg_maxit;             /* fill PCG iteration limit */
  double scale_rtol;        /* scale PCG relative residual, default 1e-10 */
  int scale_maxit;          /* scale PCG iteration limit (0 = 4 K + 100) */
  int precision;            /* 0: FP64 reductions (products in FP32, sums in FP64);
                               1: FP32 warp/CTA tree sums, FP64 across CTAs */
  int batched;              /* 0: plain global Jacobi-PCG on the block-diagonal system;
                               1: one persistent launch, per-component step lengths and
                                  convergence masks */
  int use_graph;            /* capture the relative-scale loop in a CUDA graph */
  int warm_start;           /* 1: x0 of the fill from the loaded CNN (ni_load_net), scaled per
                               component by its energy-optimal factor; needs batched = 1 */
  int hard_outliers;        /* 1: hard W^out variant (supplementary, outlier ablation) */
  int validate;             /* 1: check normals (unit length within 1e-3, n.tau != 0) */
  int ctas_per_sm;          /* CTAs per SM of the persistent fill kernels (0: 4) */
  int mg_coarse_sweeps;     /* damped-Jacobi steps on the coarsest multigrid level (0: 4) */
  int precond;              /* preconditioner of the batched fill: 0 Jacobi, 1 (default) one
                               symmetric V-cycle of aggregation multigrid on the pixel grid */
  double mg_omega;          /* damped-Jacobi smoothing weight of the V-cycle (0: 0.9) */
  double mg_correction;     /* scale of the coarse-grid correction (0: 1) */
  int mg_cta_cells;         /* coarse-level cells per CTA of a restriction/prolongation pass; the
                               pass syncs only its CTAs (0: 256, one cell per thread) */
  int mg_flags;             /* bit 0: project each component's mean out of the residual
                               before the V-cycle */
  int fill_kernels;         /* multigrid fill: 0 one kernel per pass, chunks of iterations
                               replayed from a CUDA graph; 1 (default) one persistent
                               cooperative kernel with software grid barriers */
  int scale_solver;         /* relative-scale PCG launch: 0 (default) and 1: one thread-block
                               cluster of up to 16 CTAs (hardware cluster barriers, reductions
                               through distributed shared memory) where the device can schedule
                               it; 2: one CTA or a cooperative grid over all SMs with software
                               barriers (measured slower on every map here, kept for devices
                               without clusters) */
  int bini_residual;        /* 1: the BiNI weights (Eqs. 4-5) compare the residuals chi of the
                               two sides instead of their raw log-depth differences, in the
                               fill sweeps after the first and in the scale loop (t >= 2);
                               0 (default): as the paper writes them */
  int learned_weights;      /* 1 (needs warm_start): the two alignment iterations (t <= 1) of the
                               relative-scale loop weight each inter-edge row by the network's
                               predicted continuity of the edge (its estimate of w^BiNI, Eq. 4,
                               floored at 1e-3) instead of 1; 0 (default): uniform, as the
                               paper's alignment */
} ni_config;

/* Per-run statistics (host struct filled by ni_integrate / ni_integrate_host). */
typedef struct {
  double ms_seed, ms_setup, ms_fill, ms_scale, ms_output, ms_total;
  int64_t n_valid;          /* valid pixels */
  int32_t K0;               /* components after seeding */
  int32_t K_final;          /* components after the last merge */
  int32_t n_inter0;         /* inter-component edges of the initial partition */
  int32_t merges;           /* merges performed */
  int32_t scale_iters;      /* relative-scale iterations run */
  int32_t fill_iters;       /* fill PCG iterations (max over components when batched) */
  int32_t fill_unconverged; /* components that reached cg_maxit */
  int32_t scale_cg_iters;   /* largest scale-PCG iteration count over the loop */
  int32_t n_energy;
  double energy[64];        /* E_1 .. E_n of the relative-scale loop */
  double ms_fill_solve;     /* device time of the fill PCG launch(es) alone */
  int64_t fill_px_iters;    /* sum over components of pixels x PCG iterations */
  int64_t kernel_launches;  /* kernels this call launched (graph nodes included) */
  int32_t warm_fallbacks;   /* components whose energy-optimal warm-start scale was 0 (cold start) */
  int32_t fill_fallbacks;   /* components the multigrid PCG left above the tolerance after 2000
                               iterations, finished by the Jacobi PCG */
  int64_t scale_cg_total;   /* scale-PCG iterations summed over the loop's solves */
} ni_stats;

/* Default configuration for an H x W map (Algorithm 1's defaults of the paper's
 * experiments: T = 15, dE_max = 1e-3, freq_merging = 5, L = 1e-5, U = 1e-3). */
void ni_config_default(ni_config* cfg, int H, int W);

/* Create a handle for maps of cfg->H x cfg->W; allocates the per-pixel
 * workspace on the current device.  NI_ERR_INVALID_ARG for bad sizes or
 * parameters, NI_ERR_OOM if allocation fails.  *out is NULL on failure. */
ni_status ni_create(const ni_config* cfg, ni_handle** out);

/* Release the handle and every buffer and graph it owns.  NULL is accepted. */
ni_status ni_destroy(ni_handle* h);

/* Sec. 3.3 seeding (rows a1-a2): for each 4-neighbour edge (a, b) (with
 * connectivity 8 also each diagonal edge) with both pixels valid, keep it iff n_a . n_b > cos(theta_c) (the dot product of the
 * float32 inputs evaluated in float64, x then y then z; theta_c in degrees,
 * cos(theta_c_deg * (pi / 180))).  The components of the kept edges are
 * labelled canonically: label = rank of the component's smallest raster index;
 * invalid pixels get -1.  labels_out: device int32[H][W]; K_out: host.
 * The handle keeps `normals` and `mask` (not copied): they must stay valid and
 * unchanged until ni_solve_components has returned.  Synchronises `stream`. */
ni_status ni_seed_components(ni_handle* h, const float* normals, const uint8_t* mask,
                             int32_t* labels_out, int32_t* K_out, ni_stream_t stream);

/* Sec. 3.3 filling (rows a3-a4): per intra-component edge the coefficient
 * omega~_{b->a} of Eq. 3 and the BiNI weights W = gamma^2 w^BiNI (Eqs. 4-6),
 * then for every component z~_c = cg(A_c^T W_c A_c, A_c^T W_c b_c) (Eq. 10)
 * from z~ = 0 (or the CNN warm start), returned with zero mean per component.
 * logdepth_out: device float[H][W] (log-depth; linear depth for the
 * orthographic camera; 0 at invalid pixels), may be NULL.
 * NI_ERR_NOT_CONVERGED if some component reached cg_maxit. */
ni_status ni_solve_components(ni_handle* h, float* logdepth_out, ni_stream_t stream);

/* Sec. 3.4-3.5 relative-scale loop (row a5, and a6 when cfg.can_merge): up to
 * max_iters iterations of Algorithm 1's while loop (weights, Eq. 14 solve in
 * FP64, update of Eqs. 7-8, energy, stop test, scheduled merges), continuing
 * the iteration count of earlier calls.  logdepth_inout (device float[H][W],
 * may be NULL): if given, the log-depth is first loaded from it and the result
 * written back.  energy_out (host double[max_iters], may be NULL) receives
 * E_t of each iteration run; iters_done (host, may be NULL) the number run.
 * Synchronises `stream`. */
ni_status ni_solve_scales(ni_handle* h, int max_iters, float* logdepth_inout,
                          double* energy_out, int* iters_done, ni_stream_t stream);

/* Sec. 3.5 merging (row a6), now: each component selects its incident
 * inter-component edge of smallest |chi| = |z~_a - z~_b - omega~_{b->a}| at
 * the current log-depth (float32 |chi|, ties broken by the smaller edge id
 * 2 * a + dir, dir 0 = right, 1 = down; with connectivity 8 the id 4 * a + dir,
 * dir 2 = lower-right, 3 = lower-left); the connected components of the
 * selected edges form the new partition, labelled by the rank of their
 * smallest old label.  The log-depth is unchanged.  labels_out (device
 * int32[H][W], may be NULL), K_out (host, may be NULL).  Synchronises. */
ni_status ni_merge(ni_handle* h, int32_t* labels_out, int32_t* K_out, ni_stream_t stream);

/* The merge of ni_merge with caller-given residual magnitudes instead of the
 * handle's: chi_abs is device float[H][W][2] holding |chi| of the right
 * (index 0) and down (index 1) edge of each pixel (entries of edges that are
 * not inter-component are ignored); with connectivity 8 float[H][W][4], adding
 * the lower-right (2) and lower-left (3) edge.  Used to test the merge on
 * identical inputs. */
ni_status ni_merge_residuals(ni_handle* h, const float* chi_abs, int32_t* labels_out,
                             int32_t* K_out, ni_stream_t stream);

/* Algorithm 1 end to end (rows a1-a6, a8): seeding, fill, relative-scale
 * loop with scheduled merges, output.  depth_out: device float[H][W], depth
 * exp(z~) for the perspective camera, z~ for the orthographic one, NaN at
 * invalid pixels.  labels_out (device int32[H][W], may be NULL) receives the
 * final partition.  stats_out (host, may be NULL).  Synchronises. */
ni_status ni_integrate(ni_handle* h, const float* normals, const uint8_t* mask,
                       float* depth_out, int32_t* labels_out, ni_stats* stats_out,
                       ni_stream_t stream);

/* ni_integrate with HOST buffers: normals_host float[H][W][4], mask_host
 * uint8[H][W], depth_host float[H][W] (pinned memory gives full copy speed).
 * The host->device and device->host copies are part of the call. */
ni_status ni_integrate_host(ni_handle* h, const float* normals_host, const uint8_t* mask_host,
                            float* depth_host, ni_stats* stats_out, ni_stream_t stream);

/* Current log-depth z~ (the output of the last stage call): device
 * float[H][W], log-depth (linear depth for the orthographic camera), 0 at
 * invalid pixels.  NI_ERR_STATE before ni_solve_components. */
ni_status ni_get_logdepth(ni_handle* h, float* logdepth_out, ni_stream_t stream);

/* Quality diagnostic (supplementary material, the section on the components
 * found for different theta_c): the minimum mean absolute depth error that one
 * scale per component can reach against a ground-truth depth map,
 *   E_c = min_s sum_{i in c} |s d_i - g_i|    (perspective camera)
 *   E_c = min_s sum_{i in c} |d_i + s - g_i|  (orthographic camera)
 *   *made_out = sum_c E_c / (number of counted pixels),
 * i.e. the per-component minimal MADEs weighted by their pixel counts.  With
 * labels = NULL all pixels form one component: the MADE after the best global
 * scale (offset), the error report of a finished reconstruction.
 *   z: device float[H][W]: log-depth if z_is_log (d = exp(z), perspective
 *      only; the orthographic z is linear depth either way), else depth (the
 *      output of ni_integrate);
 *   labels: device int32[H][W] with values in [-1, K) (-1 = excluded), or NULL;
 *   K: number of components (ignored, taken as 1, when labels is NULL);
 *   depth_gt: device float[H][W] ground-truth depth;
 *   made_out: host; NaN if no pixel counts;
 *   comp_made_out: device double[K], E_c / n_c (0 for an empty component), may be NULL;
 *   comp_scale_out: device double[K], a minimising s per component (NaN for an
 *      empty one), may be NULL.
 * A pixel counts if its label is >= 0 and d, g are finite (and positive for
 * the perspective camera).  Computed in FP64 by bisection of each
 * component's weighted median; the per-component error is exact up to the
 * order of the FP64 sums.  NI_ERR_INVALID_ARG if K is outside [1, H * W] or
 * a label is >= K (then nothing is written).  Independent of the stage calls;
 * scratch (20 bytes per pixel, 60 per component) is owned by the handle from
 * the first call on.  Synchronises `stream`. */
ni_status ni_min_made(ni_handle* h, const float* z, int z_is_log, const int32_t* labels, int32_t K,
                      const float* depth_gt, double* made_out, double* comp_made_out,
                      double* comp_scale_out, ni_stream_t stream);

/* Learned warm start (not in the paper; an extension beyond it): load the
 * 6-layer 3x3 conv net's weights from a file written by the training code.
 * NI_ERR_INVALID_ARG if the file is missing or malformed. */
ni_status ni_load_net(ni_handle* h, const char* path);

/* Tuning table (not in the paper: launch shapes and preconditioner knobs of
 * this implementation).  A text file written by the package's tuner
 * (paper_2510_11508_gb300/tune.py): one row per line,
 *     max_px  max_k0  ctas_per_sm  mg_cta_cells  mg_omega  scale_solver
 * ('#' starts a comment).  From then on, every ni_solve_components (and
 * ni_integrate*) gives each of those four knobs that the handle's ni_config
 * left at 0 the value of the first row with H * W <= max_px and K0 (the
 * components after seeding) <= max_k0; with no such row, or for knobs set in
 * the config, nothing changes.  The knobs change speed, not the answer: the
 * tuner keeps only values whose result equals the default configuration's.
 * NI_ERR_INVALID_ARG if the file is missing or malformed (the previous table,
 * if any, stays).  Host only. */
ni_status ni_load_tuning(ni_handle* h, const char* path);

/* Seeding without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory while they
 * run -- for example a real-time pipeline that reserves all memory at start-up,
 * a host framework whose allocator owns the device, or code where cudaMalloc
 * would synchronise the device or fail under a fixed memory-pool limit.  It
 * always seeds with 4-connectivity (it takes no connectivity argument) and
 * then computes exactly what ni_seed_components computes for a handle created
 * with connectivity = 4 (same kernels, same canonical labels); a handle with
 * connectivity = 8 also unites diagonal edges and gives other labels.  It
 * needs no handle: the union-find parent array, the scan
 * partials and the counters live in one file-scope device array of
 * 16 MiB + 16 KiB that every GPU which loads this library keeps until the
 * process exits.
 *   normals, mask: device, as for ni_seed_components (normals 16-byte aligned);
 *   cam, theta_c_deg: as in ni_config (theta_c_deg < 0 = None); normals are
 *     not validated;
 *   labels_out: device int32[H][W]; K_out_device: device int32[1] receiving K.
 * Limit: H * W <= 4,194,304 (2^22) pixels; larger maps (and bad sizes or
 * pointers) return NI_ERR_INVALID_ARG without touching the GPU.
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it for the life of the process; after a
 * cudaDeviceReset (or any teardown of the device's primary context) that
 * cached address is stale, so do not call this entry point again in such a
 * process.  Make the first call before any stream capture.  All calls
 * share the one array, so calls that overlap on the GPU (other streams, other
 * host threads) race and must be serialised by the caller.  Asynchronous on
 * `stream`; calls no cudaMalloc, cudaFree or allocating library routine. */
ni_status ni_seed_components_noalloc(const float* normals, const uint8_t* mask, int H, int W,
                                     const ni_camera* cam, double theta_c_deg, int32_t* labels_out,
                                     int32_t* K_out_device, ni_stream_t stream);

/* Message of the last error on this handle ("" if none); never NULL. */
const char* ni_last_error(const ni_handle* h);

/* Static name of a status code. */
const char* ni_status_string(ni_status s);

#ifdef __cplusplus
}
#endif
#endif /* NI_H_ */
