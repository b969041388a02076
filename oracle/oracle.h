/*
 * Plain FP64 CPU oracle for the hierarchical standard-siren likelihood of
 * arXiv 2504.02034 (CHIMERA 2.0).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; it is used by tests/, by __graft_entry__.smoke() and by
 * the cpu_baseline / reference legs of bench.py.  It shares no code with the
 * CUDA path.
 *
 * Every quantity is evaluated the slow, direct way: adaptive quadrature for
 * the comoving distance at every redshift that is needed, bracketed root
 * finding for every d_L -> z inversion, the full redshift grid for every KDE
 * and every galaxy Gaussian (no truncation windows), IEEE double throughout.
 *
 * Hyperparameter vector theta (12 doubles), in this order:
 *   H0 [km/s/Mpc], Om, Xi0, n, alpha, mu_g, sigma_g, m_min, m_max,
 *   gamma, kappa, z_p
 * lambda_g and beta are fixed per catalog.
 */
#ifndef CHIMERA_ORACLE_H
#define CHIMERA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_C_KMS 299792.458
#define ORC_Z_TABLE_MAX 10.0    /* redshift search range [0, 10] */
#define ORC_MONO_NODES 4096     /* J is checked at z_k = 10 k / 4096 */
#define ORC_KDE_MARGIN 6.0      /* KDE support: sample range +- 6 bandwidths */

enum { ORC_OK = 0, ORC_OUT_OF_SUPPORT = 1, ORC_NONMONOTONE = 2, ORC_NEFF_LOW = 4 };
enum { ORC_KDE_SINGLE_1D = 0, ORC_KDE_MANY_1D = 1, ORC_KDE_3D = 2 };
/* KDE kernel shape (Sec. 2.3 offers Gaussian and Epanechnikov).  Reading:
 * the Epanechnikov kernel (3/4)(1 - u^2) on |u| <= 1, u = (z - z_j)/h, with
 * h = sqrt(5) b, the width whose variance equals the Gaussian's b^2. */
enum { ORC_KERNEL_GAUSSIAN = 0, ORC_KERNEL_EPANECHNIKOV = 1 };
/* Jacobian placement variant.  Reading: per sample, the KDE weight of
 * sample j becomes w_j / [(1+z_j)^3 |J(z_j)|] while the bandwidth keeps
 * Scott's rule of the weights w_j of Eq. gw-kernel, and the grid factor
 * keeps psi(z) alone; the two placements differ to first order in b. */
enum { ORC_JACOBIAN_GRID = 0, ORC_JACOBIAN_PER_SAMPLE = 1 };

/* Test hooks.  Defaults (psi_scale = mass_scale = 1, flags = 0) give the
 * paper's likelihood; the others exist so that tests can check invariants and
 * closed forms.  flags bit 0: grid factor F(z) := 1; bit 1: dV_c/dz := 1 in
 * the galaxy prior. */
typedef struct {
    double psi_scale;
    double mass_scale;
    int32_t flags;
} orc_hooks;

typedef struct {
    int64_t n_events;
    const int64_t *sample_off;      /* [n_events+1] */
    const double *dL, *m1d, *m2d;   /* per PE sample, detector frame */
    const int32_t *pix_of_sample;   /* index within the event's pixel list */
    const int64_t *pix_off;         /* [n_events+1] into the flat pixel list */
    const double *sky_S;            /* per flat pixel, sr^-1 */
    const int64_t *gal_off;         /* [n_pix_total+1] */
    const double *gal_z, *gal_sigma;
    double n_gal_total;
    double z_max;
    int64_t n_z;
    int64_t n_inj_total;
    int64_t n_det;
    const double *inj_dL, *inj_m1d, *inj_m2d, *inj_log_pi;
    double lambda_g, beta;
    int32_t kde_mode;
    int32_t kernel;                 /* ORC_KERNEL_GAUSSIAN or ORC_KERNEL_EPANECHNIKOV */
    /* incomplete catalog (Eqs. p-gal, p-miss, f-R), or completeness = NULL
     * for a complete one: f_R, the solid angle of each flat pixel [sr] and
     * the completeness P_compl of each pixel on the grid [n_pix_total x n_z] */
    double f_R;
    const double *pix_area;
    const double *completeness;
    /* placement of the Jacobian (1+z)^3 |d d_L^gw/dz| of Eq. jacobian in
     * Eq. like-integrals: ORC_JACOBIAN_GRID (on the grid, the paper's form)
     * or ORC_JACOBIAN_PER_SAMPLE (on each PE sample's KDE weight) */
    int32_t jacobian;
    /* the "3D" kernel (kde_mode ORC_KDE_3D): each sample's sky position and
     * each flat pixel's centre in a flat local chart of the event's sky
     * (x, y) [rad], [n_samples x 2] and [n_pix_total x 2] */
    const double *sky_xy;
    const double *pix_xy;
} orc_catalog;

/* ---- cosmology (Eqs. dL-em, dL-mg, jacobian) ---- */
double orc_E(double z, double Om);
double orc_Dc(double z, double H0, double Om);
double orc_Xi(double z, double Xi0, double n);
double orc_dL_em(double z, double H0, double Om);
double orc_dL_gw(double z, const double *th);
double orc_J(double z, const double *th);          /* d d_L^gw / dz */
double orc_dVc_dz(double z, double H0, double Om); /* full sky, Mpc^3 */
double orc_Vc(double z, double H0, double Om);
int orc_z_of_dL(double d, const double *th, double *z); /* 0 ok, 1 none */

/* ---- population (Sec. 3.1) ---- */
double orc_p_m1(double m1, const double *th, double lambda_g);
double orc_p_m2(double m2, double m1, const double *th, double beta);
double orc_psi(double z, const double *th);

int orc_check_theta(const double *th);   /* 0 = admissible */
int orc_monotone(const double *th);      /* 1 = J > 0 on the check nodes */

/* ---- per-event stages (Eqs. gw-kernel, gw-kernel-many1d/single1d) ---- */
int orc_event_samples(const orc_catalog *c, const double *th, int64_t ev,
                      double *z, double *w, int32_t *valid);
int orc_event_bandwidth(const orc_catalog *c, const double *th, int64_t ev,
                        double *b);
int orc_event_kde(const orc_catalog *c, const double *th, int64_t ev,
                  int32_t pixel, double *K);
int orc_galaxy_profile(const orc_catalog *c, const double *th, int64_t ev,
                       int32_t pixel, const orc_hooks *hk, double *G);
int orc_grid_factor(const orc_catalog *c, const double *th,
                    const orc_hooks *hk, double *F);
int orc_event_lnI(const orc_catalog *c, const double *th, int64_t ev,
                  const orc_hooks *hk, double *lnI);

/* ---- binned KDE option (Sec. 2.3: the weighted samples are binned) ----
 * Reading: linear binning onto the grid lattice z_b = b dz; the KDE of the
 * bins keeps the bandwidth, normalisation and support of the samples' KDE.
 * orc_linear_bins returns the number of sample parts outside [b0, b0+nb). */
int64_t orc_linear_bins(int64_t n, const double *z, const double *w, double dz,
                        int64_t b0, int64_t nb, double *cb);
int orc_kde_arrays(int64_t n, const double *z, const double *w, double b, int64_t nz,
                   double z_max, int32_t binned, int32_t kernel, double *K);
/* The "3D" kernel (Sec. 2.3, kde_mode ORC_KDE_3D): the bandwidth matrix H
 * (row-major 3 x 3 over (z, x, y); returns 1 when the sample covariance is
 * degenerate) and the KDE at the grid points of one pixel's centre. */
int orc_event_kde3_bandwidth(const orc_catalog *c, const double *th, int64_t ev, double *H);
int orc_event_kde3(const orc_catalog *c, const double *th, int64_t ev, int32_t pixel, double *K);
int orc_event_kde_binned(const orc_catalog *c, const double *th, int64_t ev,
                         int32_t pixel, double *K);
int orc_event_lnI_binned(const orc_catalog *c, const double *th, int64_t ev,
                         const orc_hooks *hk, double *lnI);

/* ---- selection (Eq. bias, injection sum and N_eff) ---- */
int orc_selection(const orc_catalog *c, const double *th, const orc_hooks *hk,
                  int nthreads, double *xi, double *neff, double *s_out);

/* ---- full ln L (Eq. hyperlike) ---- */
int orc_loglike(const orc_catalog *c, const double *th, const orc_hooks *hk,
                int nthreads, double *lnL, double *lnI, double *xi,
                double *neff, int32_t *status);
int orc_loglike_binned(const orc_catalog *c, const double *th, const orc_hooks *hk,
                       int nthreads, double *lnL, double *lnI, double *xi,
                       double *neff, int32_t *status);

/* ---- analytic gradient (Gaussian kernel, Jacobian on the grid) ----
 * ln L and d ln L / d theta (12) by the chain rule written out in FP64:
 * the distance relation and its inversion, the mass model, Scott's rule,
 * the KDE, the galaxy term, the grid factor and the selection term.  The
 * almost-everywhere derivative (mass-edge, z_max and KDE-support jumps are
 * not contained).  orc_dDc_dOm: d D_c / d Om by adaptive quadrature. */
double orc_dDc_dOm(double z, double H0, double Om);
int orc_grad(const orc_catalog *c, const double *th, int nthreads, double *lnL, double *grad,
             int32_t *status);

#ifdef __cplusplus
}
#endif
#endif
