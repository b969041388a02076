/*
 * chimera.h - C ABI of the B300 (sm_103a) hierarchical standard-siren
 * likelihood of arXiv 2504.02034 (CHIMERA 2.0).
 *
 * One hyperparameter point Lambda = (H0, Om, Xi0, n, alpha, mu_g, sigma_g,
 * m_min, m_max, gamma, kappa, z_p) maps to
 *
 *     ln L(Lambda) = sum_i ln I_i(Lambda) - N_obs ln xi(Lambda)     (Eq. hyperlike)
 *
 * with I_i the per-event integral over sky pixels and a redshift grid of the
 * GW kernel times the galaxy prior (Eqs. like-integrals, gw-kernel-many1d /
 * gw-kernel-single1d, p-cat) and xi the injection estimate of the selection
 * term (Eq. bias and the Monte Carlo sum under it).
 *
 * Conventions for every call below:
 *  - Return value: 0 on success, a negative CHIMERA_ERR_* code otherwise;
 *    chimera_strerror() names it and chimera_last_error() gives the detail
 *    of the most recent failure on the calling thread.
 *  - "host" pointers are ordinary CPU memory owned by the caller; the
 *    library copies what it needs during the call and keeps no reference.
 *  - "device" pointers are CUDA device memory on the context's GPU, owned by
 *    the caller; the library reads/writes them on the stream it is given.
 *  - All floating-point inputs and outputs are IEEE double.
 *  - A context is bound to one GPU; calls on one context are serialised by
 *    an internal lock and may come from any host thread.
 *  - No call falls back to the CPU.  Without a usable GPU chimera_create
 *    fails with CHIMERA_ERR_CUDA.
 */
#ifndef CHIMERA_H
#define CHIMERA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes (return values) ---- */
#define CHIMERA_OK 0
#define CHIMERA_ERR_INVALID_ARG (-1) /* a pointer, size or value is out of range */
#define CHIMERA_ERR_NOT_FOUND (-2)   /* unknown catalog id or serve ticket */
#define CHIMERA_ERR_ADMISSION (-3)   /* device footprint exceeds the HBM budget */
#define CHIMERA_ERR_CUDA (-4)        /* a CUDA runtime call failed */
#define CHIMERA_ERR_TIMEOUT (-5)     /* serve poll: result not ready yet */
#define CHIMERA_ERR_CANCELLED (-6)   /* serve request was cancelled */
#define CHIMERA_ERR_UNSUPPORTED (-7) /* a size exceeds a compiled-in limit */

/* ---- per-hyperpoint status bits (status[] outputs) ---- */
#define CHIMERA_PT_OK 0
#define CHIMERA_PT_OUT_OF_SUPPORT 1 /* ln L = -inf: some I_i = 0, xi = 0, or Lambda inadmissible */
#define CHIMERA_PT_NONMONOTONE 2    /* ln L = -inf: d d_L^gw/dz <= 0 on z in [0, 10] */
#define CHIMERA_PT_NEFF_LOW 4       /* warning: N_eff < 5 N_obs (Sec. 2.2); value still returned */

/* ---- precision of a likelihood call ---- */
#define CHIMERA_FP64 0  /* every stage in IEEE double */
#define CHIMERA_MIXED 1 /* FP64 tables, FP32 KDE/galaxy sums, FP64 logs and final sums */
/* CHIMERA_MIXED with the binned KDE (Sec. 2.3: the weighted PE samples of
 * each pixel, or of the event in single-1D, are binned).  Reading: each
 * weighted sample is split between the two nodes of the redshift grid's
 * lattice z_n = n dz that bracket it (linear binning: weights w (1 - f) and
 * w f, f = z/dz - floor(z/dz)), and the KDE is that of the nodes, with the
 * samples' bandwidth, windows and support.  An approximation of the
 * CHIMERA_MIXED result: linear binning keeps the weight and mean of every
 * sample and adds at most dz^2/4 to its kernel variance, so
 * |ln I_binned - ln I| stays below (dz/b)^2 / 8 per event (observed
 * <= 0.014 (dz/b)^2).  Pays where segments hold many more samples than grid
 * points under them (single-1D).  ln L and chimera_terms only: chimera_grad
 * and serving reject it (INVALID_ARG). */
#define CHIMERA_MIXED_BINNED 2
/* Kernel-shape flag, OR'ed into the precision of chimera_loglike,
 * chimera_loglike_device and chimera_terms (Sec. 2.3: the 1-D KDEs take a
 * Gaussian or an Epanechnikov kernel).  Reading: the Epanechnikov kernel
 * (3/4)(1 - u^2) on |u| <= 1, u = (z - z_j)/h, h = sqrt(5) b, the width whose
 * variance equals the Gaussian's b^2 (b by the same Scott rule); windows
 * are the kernel's own support |z - z_j| <= h.  Works with CHIMERA_FP64,
 * CHIMERA_MIXED (one evaluation per sample and grid point in FP32) and
 * CHIMERA_MIXED_BINNED; chimera_grad and serving reject it (INVALID_ARG). */
#define CHIMERA_KERNEL_EPANECHNIKOV 0x10
/* Jacobian-placement flag, OR'ed into the precision of chimera_loglike,
 * chimera_loglike_device and chimera_terms (Eq. jacobian inside Eq.
 * like-integrals).  Without it the Jacobian (1+z)^3 |d d_L^gw/dz| divides
 * the integrand on the redshift grid (the paper's form); with it, it divides
 * each PE sample's KDE weight at the sample's own redshift,
 * w_j / [(1+z_j)^3 |d d_L^gw/dz (z_j)|], the bandwidth keeping Scott's rule
 * of the weights w_j and the grid factor keeping psi(z) alone.  The two
 * placements differ to first order in the bandwidth.  Works with every
 * precision and with CHIMERA_KERNEL_EPANECHNIKOV; chimera_grad and serving
 * reject it (INVALID_ARG). */
#define CHIMERA_JACOBIAN_PER_SAMPLE 0x20

/* ---- KDE variant, fixed per catalog (Sec. 2.3) ---- */
#define CHIMERA_KDE_SINGLE_1D 0 /* one redshift KDE per event, Eq. gw-kernel-single1d */
#define CHIMERA_KDE_MANY_1D 1   /* one redshift KDE per pixel, Eq. gw-kernel-many1d */
/* The "3D" kernel, a cross-check variant: one weighted Gaussian KDE per event
 * over (z, x, y), (x, y) the event's flat sky chart (descriptor sky_xy,
 * pix_xy), with the bandwidth matrix of Scott's rule in three dimensions
 * (n_eff^(-2/7) times the weighted sample covariance, unbiased weighting;
 * the plain covariance of the valid samples if the weighted one is
 * degenerate), evaluated at (z_a, pixel centre) on the grid portion holding
 * the samples (their range +- 6 sqrt(H_zz)); it replaces K_k(z) S_k, so
 * sky_S is not used.  CHIMERA_FP64 only (with or without
 * CHIMERA_JACOBIAN_PER_SAMPLE); other precisions, the Epanechnikov flag,
 * chimera_grad and serving reject it (INVALID_ARG).  An event whose sample
 * covariance is degenerate in both forms has ln I = -inf. */
#define CHIMERA_KDE_3D 2

/* ---- device storage of galaxy redshifts and widths ---- */
#define CHIMERA_GAL_F32 0  /* z and sigma as float */
#define CHIMERA_GAL_F16 1  /* z as a half offset from the pixel's first galaxy, sigma as half */
#define CHIMERA_GAL_BF16 2 /* same with bfloat16 */

/* Number of hyperparameters and their order in every theta array. */
#define CHIMERA_NPARAM 12

typedef struct chimera_ctx chimera_ctx;

/*
 * Catalog description (all host pointers, caller-owned, copied by
 * chimera_load_catalog; the caller may free them once it returns).
 *
 *  n_events        N_obs, > 0.
 *  sample_off      [n_events+1] int64 CSR offsets into the PE-sample arrays.
 *  dL_Mpc, m1_det, m2_det
 *                  [sample_off[n_events]] detector-frame luminosity distance
 *                  (Mpc) and masses (Msun) of the PE samples (Sec. 2.2), > 0.
 *  pix_of_sample   [samples] int32 index of the sample's sky pixel within its
 *                  event's pixel list (0 .. n_pix_i - 1).
 *  pix_off         [n_events+1] int64 CSR offsets into the flat pixel list.
 *  sky_S           [pix_off[n_events]] sky factor S_ik of each pixel, a
 *                  density per steradian (the 2-D sky KDE of Eq.
 *                  gw-kernel-many1d evaluated at the pixel centre), >= 0.
 *  gal_off         [n_pix_total+1] int64 CSR offsets of galaxies per pixel.
 *  gal_z, gal_sigma
 *                  [gal_off[n_pix_total]] measured galaxy redshift and its
 *                  Gaussian width (Eq. p-cat), sigma > 0.
 *  n_gal_total     N_gal,tot, the prefactor 1/N_gal,tot of p_cat.
 *  z_max, n_z      redshift grid z_a = a z_max/(n_z-1), a = 0..n_z-1, with
 *                  trapezoid weights (Sec. 2.3 item b); n_z >= 2.
 *  n_inj_total     N_inj, all injections drawn (detected or not), >= n_det.
 *  n_det           number of detected injections stored below (may be 0).
 *  inj_dL, inj_m1d, inj_m2d, inj_log_pi
 *                  [n_det] detected injections: detector-frame d_L, masses
 *                  and the natural log of their draw density pi_inj in
 *                  (d_L, m1_det, m2_det).
 *  lambda_g, beta  fixed mass-model constants (Sec. 3.1, Table 1).
 *  kde_mode        CHIMERA_KDE_SINGLE_1D or CHIMERA_KDE_MANY_1D.
 *  gal_storage     CHIMERA_GAL_F32 / F16 / BF16 (mixed path only; the FP64
 *                  path always uses the double values).
 *  f_R, pix_area, completeness
 *                  incomplete catalog (Eqs. p-gal, p-miss, f-R), or
 *                  completeness = NULL for a complete one.  completeness
 *                  [pix_off[n_events] x n_z] is P_compl of each pixel on the
 *                  grid, in [0, 1]; pix_area [pix_off[n_events]] each pixel's
 *                  solid angle [sr], > 0; f_R in [0, 1] the catalog's
 *                  full-sky completeness fraction (Eq. f-R is an integral over
 *                  the whole sky, which the events' pixels do not cover).
 *                  Reading: p_gal = f_R p_cat + (1 - f_R) p_miss with the
 *                  missing galaxies homogeneous in comoving volume (Eq.
 *                  p-miss), so a pixel's galaxy term is
 *                  f_R G_cat(z) + (pix_area/4 pi)(1 - P_compl(z)) dV_c/dz / V_c(z_max).
 *  sky_xy, pix_xy  CHIMERA_KDE_3D catalogs only (NULL otherwise): each PE
 *                  sample's sky position [n_samples x 2] and each pixel's
 *                  centre [pix_off[n_events] x 2] in a flat local chart of
 *                  the event's sky (x, y) [rad], finite.
 */
typedef struct {
    int32_t n_events;
    const int64_t *sample_off;
    const double *dL_Mpc, *m1_det, *m2_det;
    const int32_t *pix_of_sample;
    const int64_t *pix_off;
    const double *sky_S;
    const int64_t *gal_off;
    const double *gal_z, *gal_sigma;
    double n_gal_total;
    double z_max;
    int32_t n_z;
    int64_t n_inj_total;
    int64_t n_det;
    const double *inj_dL, *inj_m1d, *inj_m2d, *inj_log_pi;
    double lambda_g, beta;
    int32_t kde_mode;
    int32_t gal_storage;
    double f_R;
    const double *pix_area;
    const double *completeness;
    const double *sky_xy;
    const double *pix_xy;
} chimera_catalog_desc;

/* Footprint and sizes of a resident catalog (chimera_catalog_info_t). */
typedef struct {
    int32_t n_events;
    int32_t n_z;
    int64_t n_samples;
    int64_t n_pixels;
    int64_t n_galaxies;
    int64_t n_det;
    int64_t device_bytes;   /* resident bytes of the catalog itself */
    int32_t max_samples_per_event;
    int32_t max_pixels_per_event;
    /* how the mixed-precision galaxy profiles of Eq. p-cat are built:
     * CHIMERA_PROFILE_CUDA_CORES (FP32 kernels) or CHIMERA_PROFILE_TENSOR_CORES
     * (photometric catalogs: every galaxy's sigma >= 0.02 and >= 8 grid
     * steps, complete, at least 4096 galaxies; FP16 Gaussians contracted
     * with split-FP16 columns on tcgen05 MMAs, FP32 accumulation).  Setting
     * CHIMERA_PROFILE_FP32=1 in the environment before a load keeps that
     * catalog on the FP32 kernels. */
    int32_t profile_path;
    /* warps per block of the mixed event kernel for this catalog: at load,
     * 10 (three blocks per SM) when the largest event's samples leave room
     * for three blocks in shared memory, else 16 (two per SM); the catalog's
     * first mixed call times both on its first tile and keeps the faster.
     * Both give the same results bit for bit; this is for performance
     * reports only. */
    int32_t event_kernel_warps;
} chimera_catalog_info_t;

#define CHIMERA_PROFILE_CUDA_CORES 0
#define CHIMERA_PROFILE_TENSOR_CORES 1

/* Compiled-in limits (CHIMERA_ERR_UNSUPPORTED beyond them). */
#define CHIMERA_MAX_SAMPLES_PER_EVENT 12288
#define CHIMERA_MAX_PIXELS_PER_EVENT 1024
#define CHIMERA_MAX_NZ 8192

/*
 * chimera_create: open a context on CUDA device `device`.  hbm_budget_bytes
 * bounds everything the context allocates (catalogs, caches, workspaces);
 * 0 means 90 % of the device's free memory at creation.  The per-Om caches
 * (distance tables, galaxy profiles of every resident catalog) fill what the
 * budget leaves free; an allocation that would exceed the budget first frees
 * cache entries that the running call does not use, least recently used
 * first, and fails with ADMISSION only when that is not enough.  *out receives the
 * context.  Errors: INVALID_ARG (out == NULL, bad device), CUDA.
 */
int chimera_create(chimera_ctx **out, int device, size_t hbm_budget_bytes);

/* chimera_destroy: stop the serving loop, free all device memory. NULL is a no-op. */
void chimera_destroy(chimera_ctx *ctx);

/*
 * chimera_load_catalog: validate `desc`, sort each event's samples by
 * (pixel, d_L) for many-1D or by d_L for single-1D, pack them for the
 * kernels and copy everything to device memory, where it stays resident
 * until chimera_unload_catalog or chimera_destroy.  *catalog_id receives a
 * non-negative id.  Errors: INVALID_ARG (malformed CSR, non-positive
 * distance or mass, bad enum), UNSUPPORTED (an event beyond the compiled
 * limits), ADMISSION (footprint over budget), CUDA.
 */
int chimera_load_catalog(chimera_ctx *ctx, const chimera_catalog_desc *desc, int32_t *catalog_id);
int chimera_unload_catalog(chimera_ctx *ctx, int32_t catalog_id);
int chimera_catalog_info(chimera_ctx *ctx, int32_t catalog_id, chimera_catalog_info_t *info);

/*
 * chimera_loglike: ln L for a batch of n_points hyperparameter points
 * (Eq. hyperlike), the effective injection count N_eff of each (Sec. 2.2)
 * and a status word per point (CHIMERA_PT_* bits).
 *   theta   host [n_points x 12] row-major, order as CHIMERA_NPARAM above.
 *   lnL     host [n_points] out;  neff  host [n_points] out (may be NULL);
 *   status  host [n_points] out (may be NULL).
 * Every stage runs on the GPU; the call returns when the results are in
 * host memory.  Results do not depend on which other points share the
 * batch.  Errors: INVALID_ARG, NOT_FOUND, ADMISSION (workspace), CUDA.
 */
int chimera_loglike(chimera_ctx *ctx, int32_t catalog_id, int32_t n_points, const double *theta,
                    int32_t precision, double *lnL, double *neff, int32_t *status);

/*
 * chimera_loglike_device: as chimera_loglike with device pointers, enqueued
 * on `stream` (a cudaStream_t; NULL = the context's own stream) and
 * returning before completion.  theta_dev [n_points x 12], lnL_dev,
 * neff_dev [n_points] double, status_dev [n_points] int32 (neff_dev and
 * status_dev may be NULL).  The hyperpoints are also read back to the host
 * once per call to group them by Om (that copy is synchronous).
 */
int chimera_loglike_device(chimera_ctx *ctx, int32_t catalog_id, int32_t n_points,
                           const double *theta_dev, int32_t precision, double *lnL_dev,
                           double *neff_dev, int32_t *status_dev, void *stream);

/*
 * chimera_terms: the stages of ln L for inspection and testing.
 *   lnI   host [n_points x n_events] ln I_i (Eq. like-integrals), or NULL;
 *   bw    host [n_points x n_events] KDE bandwidth b_i per event, or NULL;
 *   xi    host [n_points] selection term xi (Eq. bias), or NULL;
 *   neff  host [n_points] N_eff, or NULL.
 */
int chimera_terms(chimera_ctx *ctx, int32_t catalog_id, int32_t n_points, const double *theta,
                  int32_t precision, double *lnI, double *bw, double *xi, double *neff);

/*
 * chimera_grad: ln L and its gradient with respect to all 12
 * hyperparameters for each point, by a hand-written adjoint that recomputes
 * the KDE instead of storing it.
 *   dlnL  host [n_points x 12] out, same parameter order as theta.
 * The derivative with respect to m_min and m_max is the almost-everywhere
 * derivative (the jump of samples across the mass edges is not included).
 * Errors as chimera_loglike.
 */
int chimera_grad(chimera_ctx *ctx, int32_t catalog_id, int32_t n_points, const double *theta,
                 int32_t precision, double *lnL, double *dlnL, int32_t *status);

/*
 * Serving (continuous batching).  A request carries n_points hyperpoints
 * for one resident catalog; requests for the same catalog that are queued
 * together are evaluated in one batched launch, different catalogs run on
 * their own CUDA streams concurrently, and a request is admitted only while
 * the workspace it needs fits the HBM budget.
 *   flags   bit 0: CHIMERA_SERVE_GRAD (also compute dlnL),
 *           bit 1: CHIMERA_SERVE_MIXED (mixed precision, else FP64).
 *   theta   host [n_points x 12], copied during submit.
 *   ticket  out: identifies the request for poll/cancel.
 * chimera_serve_poll waits up to timeout_us microseconds (0 = do not wait,
 * < 0 = wait indefinitely) and copies the results into the host buffers
 * lnL [n], dlnL [n x 12] (grad requests, may be NULL), status [n] (may be
 * NULL); it returns CHIMERA_ERR_TIMEOUT while the request is pending and
 * forgets the ticket after the first successful poll.  chimera_serve_stats
 * reports latency quantiles (ms) over completed requests.
 */
#define CHIMERA_SERVE_GRAD 1
#define CHIMERA_SERVE_MIXED 2
int chimera_serve_submit(chimera_ctx *ctx, int32_t catalog_id, int32_t n_points, const double *theta,
                         int32_t flags, uint64_t *ticket);
int chimera_serve_poll(chimera_ctx *ctx, uint64_t ticket, int64_t timeout_us, double *lnL,
                       double *dlnL, int32_t *status);
int chimera_serve_cancel(chimera_ctx *ctx, uint64_t ticket);
typedef struct {
    int64_t completed;
    int64_t batches;
    int64_t points;
    double p50_ms, p99_ms, mean_ms;
    int64_t admitted_bytes_peak;
} chimera_serve_stats_t;
int chimera_serve_stats(chimera_ctx *ctx, chimera_serve_stats_t *out);
/* chimera_serve_reset_stats: forget the latencies and counters gathered so
 * far (e.g. after warm-up requests); requests in flight are still counted
 * when they complete.  Errors: INVALID_ARG for a NULL ctx. */
int chimera_serve_reset_stats(chimera_ctx *ctx);

/*
 * Tracing.  chimera_set_trace(ctx, 1) makes the synchronous likelihood
 * calls record CUDA events around each stage on the context's stream;
 * chimera_stage_ms then returns the last call's stage times in
 * milliseconds (ms holds 7 doubles): ms[0] cosmology tables (K1), ms[1]
 * galaxy profile (K3, 0 when cached), ms[2] event integrals (K4; with the
 * reweighting for FP64, where K2 is fused into it), ms[3] selection (K5,
 * which runs on a second stream beside K2/K4, so the stages overlap),
 * ms[4] combine (K6), ms[5] adjoint (K7, gradient calls only), ms[6]
 * reweighting (K2, mixed path).
 */
/*
 * chimera_memory: the context's device-memory accounting (no counterpart in
 * the paper; for operators sizing a budget).  out: host int64[5] receives
 * out[0] the budget, out[1] the bytes held against it, and of those out[2]
 * the resident catalogs, out[3] the per-Om caches (distance tables, galaxy
 * profiles and their Om derivatives) and out[4] the workspaces (the
 * context's and the serving lanes').  Errors: INVALID_ARG.
 */
int chimera_memory(chimera_ctx *ctx, int64_t *out);

int chimera_set_trace(chimera_ctx *ctx, int enable);
int chimera_stage_ms(chimera_ctx *ctx, double *ms);

/*
 * chimera_kde_pairs: algorithmic work of the mixed-precision event kernel,
 * for the roofline: for each of the n_points hyperpoints, the number of
 * (PE sample, grid point) pairs with w_j > 0 and |z_a - z_j| <= 5.5 b_i,
 * summed over all events.  pairs: host [n_points] int64 out.
 */
int chimera_kde_pairs(chimera_ctx *ctx, int32_t catalog_id, int32_t n_points, const double *theta,
                      int64_t *pairs);

/*
 * chimera_selection_static: the selection term xi and N_eff (the FP64
 * arithmetic of the catalog path, with the inverse distance table spanning
 * the injections alone, so the results agree with the catalog path to
 * ~1e-10 relative rather than bit for bit) for callers that cannot allocate device
 * memory, e.g. code whose memory pool owns the whole device, code that must
 * stay inside another framework's allocator, or loops that must not let
 * cudaMalloc / cudaFree synchronise the device.  The paper has no
 * counterpart; this is an interface convenience.
 *
 * It allocates nothing: every intermediate lives in one fixed device array
 * of about 14 MB compiled into the library, which every GPU that loads the
 * library holds until exit.  It runs on the calling thread's current CUDA
 * device and on `stream` (a cudaStream_t; NULL = the legacy default stream).
 *   theta        host [n_points x 12], n_points <= 64 (else UNSUPPORTED).
 *   n_det        detected injections, 1 .. 8388608 (else UNSUPPORTED);
 *   n_inj_total  all injections drawn, >= n_det.
 *   inj_dL, inj_m1d, inj_m2d, inj_log_pi
 *                device [n_det] double, as in chimera_catalog_desc.
 *   lambda_g, beta, z_max  as in chimera_catalog_desc.
 *   xi, neff     device [n_points] double out (0 for an inadmissible point).
 * The first call on a device looks up the array's device address; every
 * call reads the largest d_L back to the host, so it synchronises `stream`
 * once.  Calls share the
 * array: calls that overlap on the GPU race and must be serialised by the
 * caller.  Errors: INVALID_ARG (also when inj_dL holds no positive finite
 * distance), UNSUPPORTED, CUDA.
 */
int chimera_selection_static(int32_t n_points, const double *theta, int64_t n_det,
                             int64_t n_inj_total, const double *inj_dL, const double *inj_m1d,
                             const double *inj_m2d, const double *inj_log_pi, double lambda_g,
                             double beta, double z_max, double *xi, double *neff, void *stream);

/* Name of an error code; never NULL. */
const char *chimera_strerror(int code);
/* Detail of the last failure on the calling thread ("" if none). */
const char *chimera_last_error(void);

/*
 * chimera_peaks: microbenchmarks that give roofline denominators on this
 * GPU: out[0] = FP32 Horner-step rate (one FFMA per pair, pairs/s),
 * out[1] = MUFU ex2 rate (evaluations/s), out[2] = FP64 DFMA rate (DFMA/s),
 * out[3] = device-to-device copy bandwidth (bytes/s, read + write).
 * `out` is host [4].  Not part of the method; used by the benchmark.
 */
int chimera_peaks(chimera_ctx *ctx, double *out);

#ifdef __cplusplus
}
#endif
#endif
