/*
 * Plain FP64 CPU oracle for the hierarchical standard-siren likelihood of
 * arXiv 2504.02034 (CHIMERA 2.0).  TEST INFRASTRUCTURE ONLY: the product
 * library never links or calls this file; see oracle.h.
 *
 * Readings of the paper that this file fixes:
 *  - KDE normalisation: mean-weight estimator c * sum_j w_j phi_b, with
 *    c = 1/N_s (single-1D) or 1/N_k (many-1D)            (Eqs. gw-kernel-*)
 *  - bandwidth: Scott's rule with the weighted n_eff, one b per event and
 *    hyperpoint, shared by the event's pixels; fallback to the unweighted
 *    rule, then to the grid spacing
 *  - redshift grid: uniform on [0, z_max], trapezoid weights    (Sec. 2.3)
 *  - each KDE is zero outside the grid segment that holds its samples,
 *    widened by ORC_KDE_MARGIN bandwidths                         (Sec. 2.3)
 *  - galaxy Gaussians normalised on the same grid (discrete Z_g), w_g = 1,
 *    prefactor 1/N_gal,tot; complete catalog (f_R = 1)        (Eq. p-cat)
 *  - incomplete catalog (Eqs. p-gal, p-miss, f-R) when a completeness is
 *    given: the completeness P_compl of each pixel on the grid, the pixel's
 *    solid angle and f_R are inputs (the paper leaves the completeness model
 *    to the analysis; f_R is a full-sky integral); the pixel's galaxy mass is
 *    f_R G_cat + (dOmega/4 pi)(1 - P_compl) dV_c/dz / V_c(z_max)
 *  - sky factor S_ik is an input density per steradian  (Eq. gw-kernel-many1d)
 *  - the "3D" kernel (Sec. 2.3) as a cross-check variant: a weighted Gaussian
 *    KDE over (z, x, y), (x, y) a flat local sky chart of the event, with the
 *    bandwidth matrix of Scott's rule in three dimensions, n_eff^(-2/7) times
 *    the weighted sample covariance (unbiased weighting, as in the usual
 *    weighted gaussian_kde), evaluated at (z_a, pixel centre) on the grid
 *    portion that holds the samples (their range +- ORC_KDE_MARGIN sqrt(H_zz));
 *    it replaces K_k(z) S_k in Eq. like-integrals
 *  - the Jacobian (1+z)^3 |J| on the grid (Eq. like-integrals), or, as a
 *    variant, on each sample's KDE weight w_j / [(1+z_j)^3 |J(z_j)|] with the
 *    bandwidth of the weights w_j and psi alone on the grid      (Eq. jacobian)
 *  - PE priors uniform: pi_PE = 1                                (Sec. 3.2)
 *  - mass model without low-edge smoothing; lambda_g, beta fixed (Sec. 3.1)
 *  - selection: s_j carries the injection draw density and the homogeneous
 *    redshift prior dV_c/dz / V_c(z_max)                 (Eqs. bias, p-miss)
 *  - samples whose d_L lies beyond d_L^gw(z = 10) get weight 0.
 *  - binned-KDE option (Sec. 2.3 bins the weighted samples): linear binning
 *    onto the grid lattice z_n = n dz, then the KDE of the nodes with the
 *    samples' bandwidth, normalisation and support
 *  - Epanechnikov kernel option (Sec. 2.3): (3/4)(1 - u^2) on |u| <= 1 with
 *    width h = sqrt(5) b (the Gaussian's variance b^2)
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Gauss-Legendre rule (10 points), nodes found by Newton iteration on */
/* the Legendre polynomial; used by an adaptive bisection integrator.  */
/* ------------------------------------------------------------------ */
#define GL_N 10
static double gl_x[GL_N], gl_w[GL_N];

static void legendre(int n, double x, double *pn, double *dpn) {
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; k++) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *dpn = n * (x * p1 - p0) / (x * x - 1.0);
}

__attribute__((constructor)) static void gl_init(void) {
    for (int i = 0; i < GL_N; i++) {
        double x = cos(M_PI * (i + 0.75) / (GL_N + 0.5)), p, dp;
        for (int it = 0; it < 100; it++) {
            legendre(GL_N, x, &p, &dp);
            double dx = p / dp;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        legendre(GL_N, x, &p, &dp);
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

double orc_E(double z, double Om) {
    double a = 1.0 + z;
    return sqrt(Om * a * a * a + 1.0 - Om);
}

static double gl_seg(double a, double b, double Om) {
    double m = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < GL_N; i++) s += gl_w[i] / orc_E(m + h * gl_x[i], Om);
    return s * h;
}

static double gl_adapt(double a, double b, double whole, double Om, int depth) {
    double m = 0.5 * (a + b);
    double l = gl_seg(a, m, Om), r = gl_seg(m, b, Om);
    if (depth >= 40 || fabs(l + r - whole) <= 2e-15 * fabs(l + r)) return l + r;
    return gl_adapt(a, m, l, Om, depth + 1) + gl_adapt(m, b, r, Om, depth + 1);
}

/* Comoving distance, flat geometry: D_c = (c/H0) int_0^z dz'/E(z')
 * (Eq. dL-em divided by 1+z), E^2 = Om (1+z)^3 + 1 - Om.               */
double orc_Dc(double z, double H0, double Om) {
    if (!(z > 0.0)) return 0.0;
    double I = gl_adapt(0.0, z, gl_seg(0.0, z, Om), Om, 0);
    return ORC_C_KMS / H0 * I;
}

/* Xi(z) = Xi0 + (1 - Xi0) / (1+z)^n                          (Eq. dL-mg) */
double orc_Xi(double z, double Xi0, double n) {
    return Xi0 + (1.0 - Xi0) * pow(1.0 + z, -n);
}

double orc_dL_em(double z, double H0, double Om) {
    return (1.0 + z) * orc_Dc(z, H0, Om);
}

double orc_dL_gw(double z, const double *th) {
    return orc_dL_em(z, th[0], th[1]) * orc_Xi(z, th[2], th[3]);
}

/* d d_L^gw/dz by the product rule on Eq. dL-mg:
 *   [D_c + (1+z) c/(H0 E)] Xi + d_L^em dXi/dz,
 *   dXi/dz = -n (1 - Xi0) (1+z)^(-n-1).                                  */
static double J_from_Dc(double z, double Dc, const double *th) {
    double H0 = th[0], Om = th[1], Xi0 = th[2], n = th[3];
    double a = 1.0 + z;
    double ddem = Dc + a * ORC_C_KMS / (H0 * orc_E(z, Om));
    double xi = Xi0 + (1.0 - Xi0) * pow(a, -n);
    double dxi = -n * (1.0 - Xi0) * pow(a, -n - 1.0);
    return ddem * xi + a * Dc * dxi;
}

double orc_J(double z, const double *th) {
    return J_from_Dc(z, orc_Dc(z, th[0], th[1]), th);
}

/* Full-sky comoving volume element and volume, flat geometry.            */
double orc_dVc_dz(double z, double H0, double Om) {
    double Dc = orc_Dc(z, H0, Om);
    return 4.0 * M_PI * (ORC_C_KMS / H0) * Dc * Dc / orc_E(z, Om);
}

double orc_Vc(double z, double H0, double Om) {
    double Dc = orc_Dc(z, H0, Om);
    return 4.0 / 3.0 * M_PI * Dc * Dc * Dc;
}

/* d_L -> z (Sec. 2.1): safeguarded Newton inside the bracket [0, 10].
 * Returns 1 when d is not positive or lies beyond d_L^gw(10).            */
int orc_z_of_dL(double d, const double *th, double *zout) {
    if (!(d > 0.0) || !isfinite(d)) return 1;
    double lo = 0.0, hi = ORC_Z_TABLE_MAX;
    double dhi = orc_dL_gw(hi, th);
    if (!(d <= dhi)) return 1;
    double z = hi * d / dhi;
    for (int it = 0; it < 300; it++) {
        double Dc = orc_Dc(z, th[0], th[1]);
        double f = (1.0 + z) * Dc * orc_Xi(z, th[2], th[3]) - d;
        if (f == 0.0) break;
        if (f > 0.0) hi = z; else lo = z;
        double zn = z - f / J_from_Dc(z, Dc, th);
        if (!(zn > lo && zn < hi)) zn = 0.5 * (lo + hi);
        double step = fabs(zn - z);
        z = zn;
        if (step <= 1e-15 * (1.0 + z) || hi - lo <= 1e-15 * (1.0 + z)) break;
    }
    *zout = z;
    return 0;
}

/* ---- mass model: power law + Gaussian peak for m1, power law for m2 ---- */
/* int_lo^hi m^(-a) dm                                                     */
static double pl_integral(double a, double lo, double hi) {
    if (fabs(1.0 - a) < 1e-12) return log(hi / lo);
    return (pow(hi, 1.0 - a) - pow(lo, 1.0 - a)) / (1.0 - a);
}

static double std_normal_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* p(m1): (1 - lambda_g) PL(m1; alpha) + lambda_g N(m1; mu_g, sigma_g),
 * both components normalised on [m_min, m_max], zero outside (Sec. 3.1). */
double orc_p_m1(double m1, const double *th, double lambda_g) {
    double alpha = th[4], mu = th[5], sg = th[6], mmin = th[7], mmax = th[8];
    if (!(m1 >= mmin && m1 <= mmax)) return 0.0;
    double pl = pow(m1, -alpha) / pl_integral(alpha, mmin, mmax);
    double den = std_normal_cdf((mmax - mu) / sg) - std_normal_cdf((mmin - mu) / sg);
    double g = 0.0;
    if (den > 0.0) {
        double u = (m1 - mu) / sg;
        g = exp(-0.5 * u * u) / (sg * sqrt(2.0 * M_PI)) / den;
    }
    return (1.0 - lambda_g) * pl + lambda_g * g;
}

/* p(m2 | m1) proportional to m2^beta on [m_min, m1]                       */
double orc_p_m2(double m2, double m1, const double *th, double beta) {
    double mmin = th[7];
    if (!(m1 > mmin) || !(m2 >= mmin && m2 <= m1)) return 0.0;
    return pow(m2, beta) / pl_integral(-beta, mmin, m1);
}

/* Madau-Dickinson shape, left unnormalised as in the paper (Sec. 3.1)    */
double orc_psi(double z, const double *th) {
    double gam = th[9], kap = th[10], zp = th[11];
    double a = 1.0 + z;
    return pow(a, gam) / (1.0 + pow(a / (1.0 + zp), gam + kap));
}

int orc_check_theta(const double *th) {
    for (int k = 0; k < 12; k++)
        if (!isfinite(th[k])) return 1;
    if (!(th[0] > 0.0)) return 1;                 /* H0 */
    if (!(th[1] >= 0.0 && th[1] <= 1.0)) return 1; /* Om */
    if (!(th[2] > 0.0)) return 1;                 /* Xi0 */
    if (!(th[6] > 0.0)) return 1;                 /* sigma_g */
    if (!(th[7] > 0.0 && th[8] > th[7])) return 1; /* m_min < m_max */
    if (!(th[11] > -1.0)) return 1;               /* z_p */
    return 0;
}

int orc_monotone(const double *th) {
    for (int k = 0; k <= ORC_MONO_NODES; k++) {
        double z = ORC_Z_TABLE_MAX * k / ORC_MONO_NODES;
        if (!(orc_J(z, th) > 0.0)) return 0;
    }
    return 1;
}

static const orc_hooks default_hooks = {1.0, 1.0, 0};

static double grid_dz(const orc_catalog *c) { return c->z_max / (double)(c->n_z - 1); }
static double grid_z(const orc_catalog *c, int64_t a) { return c->z_max * (double)a / (double)(c->n_z - 1); }
static double grid_w(const orc_catalog *c, int64_t a) {
    double dz = grid_dz(c);
    return (a == 0 || a == c->n_z - 1) ? 0.5 * dz : dz;
}

/* Per-sample redshift and KDE weight w_j = p(m1, m2) / pi_PE with
 * m = m_det / (1+z) (Sec. 2.1, Eq. gw-kernel), pi_PE = 1.                 */
static void samples_h(const orc_catalog *c, const double *th, int64_t ev,
                      const orc_hooks *hk, double *z, double *w, int32_t *valid) {
    int64_t j0 = c->sample_off[ev], j1 = c->sample_off[ev + 1];
    for (int64_t j = j0; j < j1; j++) {
        double zj = 0.0;
        int ok = orc_z_of_dL(c->dL[j], th, &zj) == 0;
        valid[j - j0] = ok;
        z[j - j0] = ok ? zj : 0.0;
        if (!ok) { w[j - j0] = 0.0; continue; }
        double m1 = c->m1d[j] / (1.0 + zj), m2 = c->m2d[j] / (1.0 + zj);
        w[j - j0] = hk->mass_scale * orc_p_m1(m1, th, c->lambda_g) * orc_p_m2(m2, m1, th, c->beta);
    }
}

int orc_event_samples(const orc_catalog *c, const double *th, int64_t ev,
                      double *z, double *w, int32_t *valid) {
    samples_h(c, th, ev, &default_hooks, z, w, valid);
    return 0;
}

/* Scott's rule with the weighted effective sample size (two-pass moments). */
static double bandwidth_of(int64_t n, const double *z, const double *w,
                           const int32_t *valid, double fallback) {
    double W1 = 0.0, W2 = 0.0, Wz = 0.0;
    for (int64_t j = 0; j < n; j++) {
        if (!valid[j]) continue;
        W1 += w[j];
        W2 += w[j] * w[j];
        Wz += w[j] * z[j];
    }
    if (W1 > 0.0) {
        double mean = Wz / W1, var = 0.0;
        for (int64_t j = 0; j < n; j++)
            if (valid[j]) var += w[j] * (z[j] - mean) * (z[j] - mean);
        var /= W1;
        double neff = W1 * W1 / W2;
        if (neff >= 2.0 && var > 0.0) return sqrt(var) * pow(neff, -0.2);
    }
    int64_t nv = 0;
    double s = 0.0;
    for (int64_t j = 0; j < n; j++)
        if (valid[j]) { nv++; s += z[j]; }
    if (nv >= 2) {
        double mean = s / nv, var = 0.0;
        for (int64_t j = 0; j < n; j++)
            if (valid[j]) var += (z[j] - mean) * (z[j] - mean);
        var /= nv;
        if (var > 0.0) return sqrt(var) * pow((double)nv, -0.2);
    }
    return fallback;
}

/* The per-sample Jacobian variant: after the bandwidth, each valid sample's
 * KDE weight is divided by (1+z_j)^3 |J(z_j)|                 (Eq. jacobian) */
static void jacobian_per_sample(const orc_catalog *c, const double *th, int64_t n, const double *z,
                                double *w, const int32_t *valid) {
    if (c->jacobian != ORC_JACOBIAN_PER_SAMPLE) return;
    for (int64_t j = 0; j < n; j++) {
        if (!valid[j] || w[j] == 0.0) continue;
        double ap = 1.0 + z[j];
        w[j] /= ap * ap * ap * fabs(orc_J(z[j], th));
    }
}

int orc_event_bandwidth(const orc_catalog *c, const double *th, int64_t ev, double *b) {
    int64_t n = c->sample_off[ev + 1] - c->sample_off[ev];
    double *z = malloc(sizeof(double) * (n + 1)), *w = malloc(sizeof(double) * (n + 1));
    int32_t *v = malloc(sizeof(int32_t) * (n + 1));
    samples_h(c, th, ev, &default_hooks, z, w, v);
    *b = bandwidth_of(n, z, w, v, grid_dz(c));
    free(z); free(w); free(v);
    return 0;
}

/* Linear binning of weighted samples onto the lattice z_b = b dz (the
 * binned-KDE option: the paper bins the weighted samples of each pixel or
 * event, Sec. 2.3; reading: each sample is split between the two lattice
 * nodes that bracket it, in proportion to its distance from the other one).
 * A sample at z with t = z / dz, b = floor(t), f = t - b adds w (1 - f) to
 * node b and w f to node b + 1.  Nodes [b0, b0 + nb) are kept in cb; the
 * return value counts sample parts that fell outside that range.          */
int64_t orc_linear_bins(int64_t n, const double *z, const double *w, double dz,
                        int64_t b0, int64_t nb, double *cb) {
    int64_t lost = 0;
    for (int64_t b = 0; b < nb; b++) cb[b] = 0.0;
    for (int64_t j = 0; j < n; j++) {
        if (w[j] == 0.0 || !isfinite(z[j])) continue;
        double t = z[j] / dz, fb = floor(t), f = t - fb;
        int64_t b = (int64_t)fb - b0;
        if (b >= 0 && b < nb) cb[b] += w[j] * (1.0 - f); else lost++;
        if (b + 1 >= 0 && b + 1 < nb) cb[b + 1] += w[j] * f; else lost++;
    }
    return lost;
}

/* Weighted KDE of one sample set on the grid (Eqs.
 * gw-kernel-many1d/single1d), Gaussian:
 * K(z_a) = (1/N) sum_{j in set} w_j exp(-(z_a - z_j)^2 / 2b^2) / (sqrt(2 pi) b),
 * or Epanechnikov: (1/N) sum w_j (3/4h) max(0, 1 - ((z_a - z_j)/h)^2),
 * h = sqrt(5) b; N the set's size (all its samples, valid or not).  The KDE
 * is evaluated only on the part of the grid that holds the set's samples and
 * is zero elsewhere (Sec. 2.3): z_a in [min z_j - ORC_KDE_MARGIN b,
 * max z_j + ORC_KDE_MARGIN b] over the samples with a redshift; every sample
 * term inside is kept in full.  binned != 0: the samples are replaced by
 * their linear bins (orc_linear_bins) before the same sum; the support stays
 * that of the samples.                                                    */
static void kde_set(int64_t n, const double *z, const double *w, const int32_t *valid,
                    int64_t N, double b, int64_t nz, double z_max, int binned, int kernel, double *K) {
    const double dz = z_max / (double)(nz - 1);
    const int epan = kernel == ORC_KERNEL_EPANECHNIKOV;
    const double hw = epan ? sqrt(5.0) * b : b;  /* the kernel's width */
    double zlo = INFINITY, zhi = -INFINITY;
    for (int64_t j = 0; j < n; j++)
        if (valid[j]) {
            if (z[j] < zlo) zlo = z[j];
            if (z[j] > zhi) zhi = z[j];
        }
    double norm = epan ? 0.75 / hw : 1.0 / (sqrt(2.0 * M_PI) * b);
    double *zb = NULL, *cb = NULL, *wv = NULL;
    int64_t m = 0;
    if (binned && zlo <= zhi) {
        int64_t b0 = (int64_t)floor(zlo / dz), nb = (int64_t)floor(zhi / dz) - b0 + 2;
        cb = malloc(sizeof(double) * nb);
        zb = malloc(sizeof(double) * nb);
        wv = malloc(sizeof(double) * (n + 1));
        for (int64_t j = 0; j < n; j++) wv[j] = valid[j] ? w[j] : 0.0;
        orc_linear_bins(n, z, wv, dz, b0, nb, cb);
        for (int64_t k = 0; k < nb; k++) zb[k] = z_max * (double)(b0 + k) / (double)(nz - 1);
        m = nb;
    }
    zlo -= ORC_KDE_MARGIN * b;
    zhi += ORC_KDE_MARGIN * b;
    for (int64_t a = 0; a < nz; a++) {
        double za = z_max * (double)a / (double)(nz - 1), s = 0.0;
        if (!(za >= zlo && za <= zhi)) { K[a] = 0.0; continue; }
        if (binned) {
            for (int64_t k = 0; k < m; k++) {
                if (cb[k] == 0.0) continue;
                double u = (za - zb[k]) / hw;
                s += cb[k] * (epan ? (fabs(u) <= 1.0 ? 1.0 - u * u : 0.0) : exp(-0.5 * u * u));
            }
        } else {
            for (int64_t j = 0; j < n; j++) {
                if (!valid[j] || w[j] == 0.0) continue;
                double u = (za - z[j]) / hw;
                s += w[j] * (epan ? (fabs(u) <= 1.0 ? 1.0 - u * u : 0.0) : exp(-0.5 * u * u));
            }
        }
        K[a] = N > 0 ? s * norm / (double)N : 0.0;
    }
    free(zb); free(cb); free(wv);
}

int orc_kde_arrays(int64_t n, const double *z, const double *w, double b, int64_t nz,
                   double z_max, int32_t binned, int32_t kernel, double *K) {
    int32_t *v = malloc(sizeof(int32_t) * (n + 1));
    for (int64_t j = 0; j < n; j++) v[j] = isfinite(z[j]) ? 1 : 0;
    kde_set(n, z, w, v, n, b, nz, z_max, binned, kernel, K);
    free(v);
    return 0;
}

/* The KDE of one pixel's samples (pixel >= 0) or of all the event's samples
 * (pixel = -1) on the grid. */
static void kde_grid(const orc_catalog *c, int64_t ev, int32_t pixel,
                     const double *z, const double *w, const int32_t *valid,
                     double b, int binned, double *K) {
    int64_t j0 = c->sample_off[ev], n = c->sample_off[ev + 1] - j0;
    double *zs = malloc(sizeof(double) * (n + 1)), *ws = malloc(sizeof(double) * (n + 1));
    int32_t *vs = malloc(sizeof(int32_t) * (n + 1));
    int64_t cnt = 0;
    for (int64_t j = 0; j < n; j++) {
        if (pixel >= 0 && c->pix_of_sample[j0 + j] != pixel) continue;
        zs[cnt] = z[j];
        ws[cnt] = w[j];
        vs[cnt] = valid[j];
        cnt++;
    }
    kde_set(cnt, zs, ws, vs, cnt, b, c->n_z, c->z_max, binned, c->kernel, K);
    free(zs); free(ws); free(vs);
}

static int event_kde_impl(const orc_catalog *c, const double *th, int64_t ev,
                          int32_t pixel, int binned, double *K) {
    int64_t n = c->sample_off[ev + 1] - c->sample_off[ev];
    double *z = malloc(sizeof(double) * (n + 1)), *w = malloc(sizeof(double) * (n + 1));
    int32_t *v = malloc(sizeof(int32_t) * (n + 1));
    samples_h(c, th, ev, &default_hooks, z, w, v);
    double b = bandwidth_of(n, z, w, v, grid_dz(c));
    jacobian_per_sample(c, th, n, z, w, v);
    kde_grid(c, ev, pixel, z, w, v, b, binned, K);
    free(z); free(w); free(v);
    return 0;
}

int orc_event_kde(const orc_catalog *c, const double *th, int64_t ev,
                  int32_t pixel, double *K) {
    return event_kde_impl(c, th, ev, pixel, 0, K);
}

int orc_event_kde_binned(const orc_catalog *c, const double *th, int64_t ev,
                         int32_t pixel, double *K) {
    return event_kde_impl(c, th, ev, pixel, 1, K);
}

/* ---- the "3D" kernel ---------------------------------------------------- */

static double det3(const double *A) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* Covariance of the valid samples' (z, x, y): weighted (weights w, unbiased
 * normalisation sum w - sum w^2 / sum w) or, with w = NULL, plain (n - 1).  */
static void cov3(int64_t n, const double *z, const double *xy, const double *w, const int32_t *valid,
                 double *C) {
    double V1 = 0.0, V2 = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; j++) {
        if (!valid[j]) continue;
        double wj = w ? w[j] : 1.0, v[3] = {z[j], xy[2 * j], xy[2 * j + 1]};
        V1 += wj;
        V2 += wj * wj;
        for (int r = 0; r < 3; r++) m[r] += wj * v[r];
    }
    for (int r = 0; r < 9; r++) C[r] = 0.0;
    if (!(V1 > 0.0)) return;
    for (int r = 0; r < 3; r++) m[r] /= V1;
    for (int64_t j = 0; j < n; j++) {
        if (!valid[j]) continue;
        double wj = w ? w[j] : 1.0, v[3] = {z[j] - m[0], xy[2 * j] - m[1], xy[2 * j + 1] - m[2]};
        for (int r = 0; r < 3; r++)
            for (int s = 0; s < 3; s++) C[3 * r + s] += wj * v[r] * v[s];
    }
    double fact = V1 - V2 / V1;
    for (int r = 0; r < 9; r++) C[r] = fact > 0.0 ? C[r] / fact : 0.0;
}

/* H = Scott factor^2 x covariance, Scott factor n_eff^(-1/7) (d = 3): the
 * weighted covariance with n_eff = (sum w)^2 / sum w^2, else the plain one
 * with n = the valid samples; 1 if both are degenerate.                   */
static int kde3_bandwidth(int64_t n, const double *z, const double *xy, const double *w,
                          const int32_t *valid, double *H) {
    double W1 = 0.0, W2 = 0.0;
    int64_t nv = 0;
    for (int64_t j = 0; j < n; j++)
        if (valid[j]) { W1 += w[j]; W2 += w[j] * w[j]; nv++; }
    double C[9];
    if (W1 > 0.0 && W1 * W1 / W2 >= 2.0) {
        cov3(n, z, xy, w, valid, C);
        if (det3(C) > 0.0) {
            double f2 = pow(W1 * W1 / W2, -2.0 / 7.0);
            for (int r = 0; r < 9; r++) H[r] = f2 * C[r];
            return 0;
        }
    }
    if (nv >= 4) {
        cov3(n, z, xy, NULL, valid, C);
        if (det3(C) > 0.0) {
            double f2 = pow((double)nv, -2.0 / 7.0);
            for (int r = 0; r < 9; r++) H[r] = f2 * C[r];
            return 0;
        }
    }
    return 1;
}

/* K(z_a) = (1/N) sum_j w_j N3((z_a, X_k, Y_k) - (z_j, x_j, y_j); H) on the
 * support, N the event's sample count.                                    */
static void kde3_pixel(const orc_catalog *c, int64_t ev, int32_t pixel, const double *z,
                       const double *w, const int32_t *valid, const double *H, double *K) {
    int64_t j0 = c->sample_off[ev], n = c->sample_off[ev + 1] - j0;
    const double *xy = c->sky_xy + 2 * j0, *P = c->pix_xy + 2 * (c->pix_off[ev] + pixel);
    double d = det3(H), Hi[9];
    Hi[0] = (H[4] * H[8] - H[5] * H[7]) / d; Hi[1] = (H[2] * H[7] - H[1] * H[8]) / d;
    Hi[2] = (H[1] * H[5] - H[2] * H[4]) / d; Hi[3] = (H[5] * H[6] - H[3] * H[8]) / d;
    Hi[4] = (H[0] * H[8] - H[2] * H[6]) / d; Hi[5] = (H[2] * H[3] - H[0] * H[5]) / d;
    Hi[6] = (H[3] * H[7] - H[4] * H[6]) / d; Hi[7] = (H[1] * H[6] - H[0] * H[7]) / d;
    Hi[8] = (H[0] * H[4] - H[1] * H[3]) / d;
    double zlo = INFINITY, zhi = -INFINITY;
    for (int64_t j = 0; j < n; j++)
        if (valid[j]) { if (z[j] < zlo) zlo = z[j]; if (z[j] > zhi) zhi = z[j]; }
    zlo -= ORC_KDE_MARGIN * sqrt(H[0]);
    zhi += ORC_KDE_MARGIN * sqrt(H[0]);
    double norm = 1.0 / (pow(2.0 * M_PI, 1.5) * sqrt(d) * (double)n);
    for (int64_t a = 0; a < c->n_z; a++) {
        double za = grid_z(c, a), s = 0.0;
        K[a] = 0.0;
        if (!(za >= zlo && za <= zhi)) continue;
        for (int64_t j = 0; j < n; j++) {
            if (!valid[j] || w[j] == 0.0) continue;
            double v[3] = {za - z[j], P[0] - xy[2 * j], P[1] - xy[2 * j + 1]}, q = 0.0;
            for (int r = 0; r < 3; r++)
                for (int t = 0; t < 3; t++) q += v[r] * Hi[3 * r + t] * v[t];
            s += w[j] * exp(-0.5 * q);
        }
        K[a] = s * norm;
    }
}

int orc_event_kde3_bandwidth(const orc_catalog *c, const double *th, int64_t ev, double *H) {
    int64_t j0 = c->sample_off[ev], n = c->sample_off[ev + 1] - j0;
    double *z = malloc(sizeof(double) * (n + 1)), *w = malloc(sizeof(double) * (n + 1));
    int32_t *v = malloc(sizeof(int32_t) * (n + 1));
    samples_h(c, th, ev, &default_hooks, z, w, v);
    int rc = kde3_bandwidth(n, z, c->sky_xy + 2 * j0, w, v, H);
    free(z); free(w); free(v);
    return rc;
}

int orc_event_kde3(const orc_catalog *c, const double *th, int64_t ev, int32_t pixel, double *K) {
    int64_t j0 = c->sample_off[ev], n = c->sample_off[ev + 1] - j0;
    double *z = malloc(sizeof(double) * (n + 1)), *w = malloc(sizeof(double) * (n + 1)), H[9];
    int32_t *v = malloc(sizeof(int32_t) * (n + 1));
    samples_h(c, th, ev, &default_hooks, z, w, v);
    int rc = kde3_bandwidth(n, z, c->sky_xy + 2 * j0, w, v, H);
    jacobian_per_sample(c, th, n, z, w, v);
    if (rc == 0) kde3_pixel(c, ev, pixel, z, w, v, H, K);
    else for (int64_t a = 0; a < c->n_z; a++) K[a] = 0.0;
    free(z); free(w); free(v);
    return rc;
}

/* Galaxy prior of one pixel on the grid (Eq. p-cat, complete catalog):
 * G(z_a) = (1/N_gal,tot) dV_c/dz(z_a) sum_g N(z_a; z_g, s_g) / Z_g,
 * Z_g = sum_a w_a N(z_a; z_g, s_g) dV_c/dz(z_a); galaxies with Z_g = 0
 * are dropped.                                                            */
static void galaxy_profile_dv(const orc_catalog *c, int64_t ev, int32_t pixel,
                              const double *dv, double vmax, double *G) {
    int64_t p = c->pix_off[ev] + pixel;
    for (int64_t a = 0; a < c->n_z; a++) G[a] = 0.0;
    for (int64_t g = c->gal_off[p]; g < c->gal_off[p + 1]; g++) {
        double zg = c->gal_z[g], sg = c->gal_sigma[g];
        double norm = 1.0 / (sqrt(2.0 * M_PI) * sg);
        double Z = 0.0;
        for (int64_t a = 0; a < c->n_z; a++) {
            double u = (grid_z(c, a) - zg) / sg;
            Z += grid_w(c, a) * norm * exp(-0.5 * u * u) * dv[a];
        }
        if (!(Z > 0.0)) continue;
        for (int64_t a = 0; a < c->n_z; a++) {
            double u = (grid_z(c, a) - zg) / sg;
            G[a] += norm * exp(-0.5 * u * u) / Z;
        }
    }
    for (int64_t a = 0; a < c->n_z; a++) G[a] *= dv[a] / c->n_gal_total;
    if (c->completeness) {
        /* incomplete catalog: the pixel's mass of p_gal = f_R p_cat +
         * (1 - f_R) p_miss, the missing galaxies homogeneous in comoving
         * volume (Eq. p-miss): (dOmega_k / 4 pi) (1 - P_compl) dV_c/dz / V_c(z_max) */
        const double area = c->pix_area[p] / (4.0 * M_PI);
        const double *P = c->completeness + p * c->n_z;
        for (int64_t a = 0; a < c->n_z; a++)
            G[a] = c->f_R * G[a] + area * (1.0 - P[a]) * dv[a] / vmax;
    }
}

static void grid_dvdz(const orc_catalog *c, const double *th, const orc_hooks *hk, double *dv) {
    for (int64_t a = 0; a < c->n_z; a++)
        dv[a] = (hk->flags & 2) ? 1.0 : orc_dVc_dz(grid_z(c, a), th[0], th[1]);
}

/* V_c(z_max), the normalisation of the homogeneous missing-galaxy prior
 * (Eq. p-miss); z_max under the dV_c/dz := 1 test hook. */
static double grid_vmax(const orc_catalog *c, const double *th, const orc_hooks *hk) {
    return (hk->flags & 2) ? c->z_max : orc_Vc(c->z_max, th[0], th[1]);
}

int orc_galaxy_profile(const orc_catalog *c, const double *th, int64_t ev,
                       int32_t pixel, const orc_hooks *hk, double *G) {
    if (!hk) hk = &default_hooks;
    double *dv = malloc(sizeof(double) * c->n_z);
    grid_dvdz(c, th, hk, dv);
    galaxy_profile_dv(c, ev, pixel, dv, grid_vmax(c, th, hk), G);
    free(dv);
    return 0;
}

/* Redshift part of the integrand of Eq. like-integrals:
 * F(z) = psi(z) / [(1+z)^3 |d d_L^gw / dz|]                  (Eq. jacobian),
 * or psi(z) alone when the Jacobian sits on the samples.                  */
int orc_grid_factor(const orc_catalog *c, const double *th,
                    const orc_hooks *hk, double *F) {
    if (!hk) hk = &default_hooks;
    for (int64_t a = 0; a < c->n_z; a++) {
        if (hk->flags & 1) { F[a] = 1.0; continue; }
        double z = grid_z(c, a), ap = 1.0 + z;
        F[a] = hk->psi_scale * orc_psi(z, th);
        if (c->jacobian != ORC_JACOBIAN_PER_SAMPLE) F[a] /= ap * ap * ap * fabs(orc_J(z, th));
    }
    return 0;
}

/* ln I_i: Eq. like-integrals on the pixel x redshift grid.
 * many-1D : I = sum_k S_k sum_a w_a K_k(z_a) F(z_a) G_k(z_a)
 * single-1D: I = sum_a w_a K(z_a) F(z_a) sum_k S_k G_k(z_a)              */
static double event_lnI_impl(const orc_catalog *c, const double *th, int64_t ev,
                             const orc_hooks *hk, const double *F, const double *dv, int binned) {
    const double vmax = c->completeness ? grid_vmax(c, th, hk) : 1.0;
    int64_t n = c->sample_off[ev + 1] - c->sample_off[ev];
    int64_t nz = c->n_z;
    int32_t npix = (int32_t)(c->pix_off[ev + 1] - c->pix_off[ev]);
    double *z = malloc(sizeof(double) * (n + 1)), *w = malloc(sizeof(double) * (n + 1));
    int32_t *v = malloc(sizeof(int32_t) * (n + 1));
    double *K = malloc(sizeof(double) * nz), *G = malloc(sizeof(double) * nz);
    double *Gs = calloc((size_t)nz, sizeof(double));
    samples_h(c, th, ev, hk, z, w, v);
    double b = bandwidth_of(n, z, w, v, grid_dz(c)), H[9];
    int degenerate3 = c->kde_mode == ORC_KDE_3D &&
                      kde3_bandwidth(n, z, c->sky_xy + 2 * c->sample_off[ev], w, v, H);
    jacobian_per_sample(c, th, n, z, w, v);
    double I = 0.0;
    if (c->kde_mode == ORC_KDE_3D) {
        /* I = sum_k sum_a w_a K3(z_a, pixel centre k) F(z_a) G_k(z_a) */
        for (int32_t k = 0; k < npix && !degenerate3; k++) {
            kde3_pixel(c, ev, k, z, w, v, H, K);
            galaxy_profile_dv(c, ev, k, dv, vmax, G);
            for (int64_t a = 0; a < nz; a++) I += grid_w(c, a) * K[a] * F[a] * G[a];
        }
    } else if (c->kde_mode == ORC_KDE_MANY_1D) {
        for (int32_t k = 0; k < npix; k++) {
            double S = c->sky_S[c->pix_off[ev] + k];
            kde_grid(c, ev, k, z, w, v, b, binned, K);
            galaxy_profile_dv(c, ev, k, dv, vmax, G);
            double s = 0.0;
            for (int64_t a = 0; a < nz; a++) s += grid_w(c, a) * K[a] * F[a] * G[a];
            I += S * s;
        }
    } else {
        kde_grid(c, ev, -1, z, w, v, b, binned, K);
        for (int32_t k = 0; k < npix; k++) {
            double S = c->sky_S[c->pix_off[ev] + k];
            galaxy_profile_dv(c, ev, k, dv, vmax, G);
            for (int64_t a = 0; a < nz; a++) Gs[a] += S * G[a];
        }
        for (int64_t a = 0; a < nz; a++) I += grid_w(c, a) * K[a] * F[a] * Gs[a];
    }
    free(z); free(w); free(v); free(K); free(G); free(Gs);
    return (I > 0.0 && isfinite(I)) ? log(I) : -INFINITY;
}

static int event_lnI_entry(const orc_catalog *c, const double *th, int64_t ev,
                           const orc_hooks *hk, int binned, double *lnI) {
    if (!hk) hk = &default_hooks;
    double *F = malloc(sizeof(double) * c->n_z), *dv = malloc(sizeof(double) * c->n_z);
    orc_grid_factor(c, th, hk, F);
    grid_dvdz(c, th, hk, dv);
    *lnI = event_lnI_impl(c, th, ev, hk, F, dv, binned);
    free(F); free(dv);
    return isfinite(*lnI) ? 0 : 1;
}

int orc_event_lnI(const orc_catalog *c, const double *th, int64_t ev,
                  const orc_hooks *hk, double *lnI) {
    return event_lnI_entry(c, th, ev, hk, 0, lnI);
}

int orc_event_lnI_binned(const orc_catalog *c, const double *th, int64_t ev,
                         const orc_hooks *hk, double *lnI) {
    return event_lnI_entry(c, th, ev, hk, 1, lnI);
}

/* Neumaier compensated sum                                                */
static double neumaier(const double *x, int64_t n) {
    double s = 0.0, comp = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double t = s + x[i];
        if (fabs(s) >= fabs(x[i])) comp += (s - t) + x[i];
        else comp += (x[i] - t) + s;
        s = t;
    }
    return s + comp;
}

/* Selection term from detected injections (Eq. bias as an MC sum):
 * s_j = p(m1,m2) psi(z_j) p_z(z_j) / [(1+z_j)^3 |J(z_j)| pi_inj,j],
 * p_z = dV_c/dz / V_c(z_max) on [0, z_max], 0 beyond;
 * xi = sum s / N_inj; N_eff = (sum s)^2 / (sum s^2 - (sum s)^2 / N_inj).    */
int orc_selection(const orc_catalog *c, const double *th, const orc_hooks *hk,
                  int nthreads, double *xi, double *neff, double *s_out) {
    if (!hk) hk = &default_hooks;
    int64_t n = c->n_det;
    double *s = malloc(sizeof(double) * (n + 1)), *s2 = malloc(sizeof(double) * (n + 1));
    double vmax = orc_Vc(c->z_max, th[0], th[1]);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
    for (int64_t j = 0; j < n; j++) {
        double z = 0.0, val = 0.0;
        if (orc_z_of_dL(c->inj_dL[j], th, &z) == 0 && z <= c->z_max) {
            double m1 = c->inj_m1d[j] / (1.0 + z), m2 = c->inj_m2d[j] / (1.0 + z);
            double pm = hk->mass_scale * orc_p_m1(m1, th, c->lambda_g) * orc_p_m2(m2, m1, th, c->beta);
            if (pm > 0.0) {
                double a = 1.0 + z;
                double pz = orc_dVc_dz(z, th[0], th[1]) / vmax;
                val = pm * hk->psi_scale * orc_psi(z, th) * pz /
                      (a * a * a * fabs(orc_J(z, th)) * exp(c->inj_log_pi[j]));
            }
        }
        s[j] = val;
        s2[j] = val * val;
    }
    double S1 = neumaier(s, n), S2 = neumaier(s2, n);
    double N = (double)c->n_inj_total;
    *xi = S1 / N;
    *neff = S1 > 0.0 ? S1 * S1 / (S2 - S1 * S1 / N) : 0.0;
    if (s_out) memcpy(s_out, s, sizeof(double) * n);
    free(s); free(s2);
    return 0;
}

/* ln L = sum_i ln I_i - N_obs ln xi                          (Eq. hyperlike) */
static int loglike_impl(const orc_catalog *c, const double *th, const orc_hooks *hk,
                        int nthreads, int binned, double *lnL, double *lnI_out, double *xi_out,
                        double *neff_out, int32_t *status) {
    if (!hk) hk = &default_hooks;
    int64_t ne = c->n_events;
    *status = ORC_OK;
    if (xi_out) *xi_out = 0.0;
    if (neff_out) *neff_out = 0.0;
    if (orc_check_theta(th)) { *lnL = -INFINITY; *status = ORC_OUT_OF_SUPPORT; return 0; }
    if (!orc_monotone(th)) { *lnL = -INFINITY; *status = ORC_NONMONOTONE; return 0; }
    double *lnI = malloc(sizeof(double) * (ne + 1));
    double *F = malloc(sizeof(double) * c->n_z), *dv = malloc(sizeof(double) * c->n_z);
    orc_grid_factor(c, th, hk, F);
    grid_dvdz(c, th, hk, dv);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < ne; i++) lnI[i] = event_lnI_impl(c, th, i, hk, F, dv, binned);
    double xi, neff;
    orc_selection(c, th, hk, nthreads, &xi, &neff, NULL);
    int bad = !(xi > 0.0);
    for (int64_t i = 0; i < ne; i++) bad |= !isfinite(lnI[i]);
    if (bad) { *lnL = -INFINITY; *status = ORC_OUT_OF_SUPPORT; }
    else *lnL = neumaier(lnI, ne) - (double)ne * log(xi);
    if (!(neff >= 5.0 * (double)ne)) *status |= ORC_NEFF_LOW;
    if (lnI_out) memcpy(lnI_out, lnI, sizeof(double) * ne);
    if (xi_out) *xi_out = xi;
    if (neff_out) *neff_out = neff;
    free(lnI); free(F); free(dv);
    return 0;
}

int orc_loglike(const orc_catalog *c, const double *th, const orc_hooks *hk,
                int nthreads, double *lnL, double *lnI_out, double *xi_out,
                double *neff_out, int32_t *status) {
    return loglike_impl(c, th, hk, nthreads, 0, lnL, lnI_out, xi_out, neff_out, status);
}

int orc_loglike_binned(const orc_catalog *c, const double *th, const orc_hooks *hk,
                       int nthreads, double *lnL, double *lnI_out, double *xi_out,
                       double *neff_out, int32_t *status) {
    return loglike_impl(c, th, hk, nthreads, 1, lnL, lnI_out, xi_out, neff_out, status);
}

/* ====================================================================== */
/* Analytic gradient of ln L (the chain rule through Eqs. hyperlike,      */
/* like-integrals, gw-kernel-many1d/single1d, p-cat, jacobian, bias and   */
/* the Sec. 3.1 population), FP64, Gaussian kernel, Jacobian on the grid. */
/* The almost-everywhere derivative: samples or injections crossing a     */
/* mass edge or z_max, and grid points crossing a KDE support edge, make  */
/* jumps that it does not contain.                                        */
/* ====================================================================== */

enum { P_H0 = 0, P_OM, P_XI0, P_N, P_ALPHA, P_MU, P_SG, P_MMIN, P_MMAX, P_GAM, P_KAP, P_ZP, NP = 12 };

/* d D_c / d Om = (c/H0) int_0^z d(1/E)/dOm dz', d(1/E)/dOm = -((1+z)^3 - 1) / (2 E^3),
 * with (1+z)^3 - 1 = z (3 + 3z + z^2) written without cancellation (the
 * adaptive rule's relative tolerance would otherwise chase rounding noise) */
static double dinvE_dOm(double z, double Om) {
    double E = orc_E(z, Om);
    return -0.5 * z * (3.0 + z * (3.0 + z)) / (E * E * E);
}

static double gl_seg_om(double a, double b, double Om) {
    double m = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < GL_N; i++) s += gl_w[i] * dinvE_dOm(m + h * gl_x[i], Om);
    return s * h;
}

static double gl_adapt_om(double a, double b, double whole, double Om, int depth) {
    double m = 0.5 * (a + b);
    double l = gl_seg_om(a, m, Om), r = gl_seg_om(m, b, Om);
    if (depth >= 30 || fabs(l + r - whole) <= 4e-15 * fabs(l + r) + 1e-300) return l + r;
    return gl_adapt_om(a, m, l, Om, depth + 1) + gl_adapt_om(m, b, r, Om, depth + 1);
}

double orc_dDc_dOm(double z, double H0, double Om) {
    if (!(z > 0.0)) return 0.0;
    return ORC_C_KMS / H0 * gl_adapt_om(0.0, z, gl_seg_om(0.0, z, Om), Om, 0);
}

/* The distance relation and its derivatives at redshift z (Eqs. dL-em,
 * dL-mg, jacobian): d = d_L^gw, J = dd/dz, Jz = d^2 d / dz^2, and at fixed
 * z the derivatives dd[k], dJ[k] with respect to (H0, Om, Xi0, n).        */
typedef struct {
    double a, E, Dc, dDc_Om, xi, d, J, Jz;
    double dd[4], dJ[4];
    double dv, dv_Om, dlndv_dz;   /* full-sky dV_c/dz, its Om derivative, d ln dV_c/dz / dz */
} cosmo_d;

static void cosmo_at(double z, const double *th, cosmo_d *o) {
    const double H0 = th[P_H0], Om = th[P_OM], X0 = th[P_XI0], n = th[P_N];
    const double cH = ORC_C_KMS / H0;
    const double a = 1.0 + z, E = orc_E(z, Om);
    const double Dc = orc_Dc(z, H0, Om), dDc = orc_dDc_dOm(z, H0, Om);
    const double an = pow(a, -n);                       /* (1+z)^-n */
    const double xi = X0 + (1.0 - X0) * an;
    const double xi1 = -n * (1.0 - X0) * an / a;        /* dXi/dz */
    const double xi2 = n * (n + 1.0) * (1.0 - X0) * an / (a * a);
    const double Dc1 = cH / E;                           /* dD_c/dz */
    const double E1 = 1.5 * Om * a * a / E;              /* dE/dz */
    const double Dc2 = -cH * E1 / (E * E);
    const double dinvE = dinvE_dOm(z, Om);               /* d(1/E)/dOm */
    o->a = a; o->E = E; o->Dc = Dc; o->dDc_Om = dDc; o->xi = xi;
    o->d = a * Dc * xi;
    o->J = (Dc + a * Dc1) * xi + a * Dc * xi1;
    o->Jz = 2.0 * Dc1 * xi + 2.0 * Dc * xi1 + a * Dc2 * xi + 2.0 * a * Dc1 * xi1 + a * Dc * xi2;
    /* at fixed z: d_gw = a Dc Xi */
    o->dd[P_H0] = -o->d / H0;
    o->dd[P_OM] = a * dDc * xi;
    o->dd[P_XI0] = a * Dc * (1.0 - an);
    o->dd[P_N] = -a * Dc * (1.0 - X0) * an * log(a);
    /* J = (Dc + a cH / E) Xi + a Dc Xi' */
    o->dJ[P_H0] = -o->J / H0;
    o->dJ[P_OM] = (dDc + a * cH * dinvE) * xi + a * dDc * xi1;
    o->dJ[P_XI0] = (Dc + a * Dc1) * (1.0 - an) + a * Dc * n * an / a;
    {
        const double dxi_dn = -(1.0 - X0) * an * log(a);
        const double dxi1_dn = (1.0 - X0) * an / a * (n * log(a) - 1.0);
        o->dJ[P_N] = (Dc + a * Dc1) * dxi_dn + a * Dc * dxi1_dn;
    }
    o->dv = 4.0 * M_PI * cH * Dc * Dc / E;
    o->dv_Om = 4.0 * M_PI * cH * (2.0 * Dc * dDc / E + Dc * Dc * dinvE);
    o->dlndv_dz = Dc > 0.0 ? 2.0 * Dc1 / Dc - E1 / E : 0.0;
}

/* Mass model (Sec. 3.1) with derivatives: returns w = p(m1) p(m2|m1) (0
 * outside the support), dlw[k] = d ln w / d theta_k at fixed source-frame
 * masses, and *dlna = d ln w / d ln(1+z) at fixed detector-frame masses
 * (m = m_det / (1+z)).                                                    */
static double mass_dlog(double m1, double m2, const double *th, double lambda_g, double beta,
                        double *dlw, double *dlna) {
    for (int k = 0; k < NP; k++) dlw[k] = 0.0;
    *dlna = 0.0;
    const double alpha = th[P_ALPHA], mu = th[P_MU], sg = th[P_SG], mmin = th[P_MMIN], mmax = th[P_MMAX];
    if (!(m1 >= mmin && m1 <= mmax && m2 >= mmin && m2 <= m1) || !(m1 > mmin)) return 0.0;
    /* power law: m1^-alpha / Z_PL */
    double Zpl, dZpl_da;
    if (fabs(1.0 - alpha) < 1e-12) {
        Zpl = log(mmax / mmin);
        dZpl_da = -0.5 * (log(mmax) * log(mmax) - log(mmin) * log(mmin));
    } else {
        const double num = pow(mmax, 1.0 - alpha) - pow(mmin, 1.0 - alpha);
        Zpl = num / (1.0 - alpha);
        const double dnum = -log(mmax) * pow(mmax, 1.0 - alpha) + log(mmin) * pow(mmin, 1.0 - alpha);
        dZpl_da = dnum / (1.0 - alpha) + Zpl / (1.0 - alpha);
    }
    const double PL = pow(m1, -alpha) / Zpl;
    /* truncated Gaussian: N(m1; mu, sg) / [Phi(b) - Phi(a)] */
    const double ua = (mmin - mu) / sg, ub = (mmax - mu) / sg;
    const double phia = exp(-0.5 * ua * ua) / sqrt(2.0 * M_PI), phib = exp(-0.5 * ub * ub) / sqrt(2.0 * M_PI);
    const double ZG = std_normal_cdf(ub) - std_normal_cdf(ua);
    const double x = (m1 - mu) / sg;
    const double G = ZG > 0.0 ? exp(-0.5 * x * x) / (sg * sqrt(2.0 * M_PI)) / ZG : 0.0;
    const double p1 = (1.0 - lambda_g) * PL + lambda_g * G;
    if (!(p1 > 0.0)) return 0.0;
    const double cpl = (1.0 - lambda_g) / p1, cg = lambda_g / p1;  /* d p1 = cpl dPL + cg dG, over p1 */
    /* p(m2|m1) = m2^beta / Z2, Z2 = int_{m_min}^{m1} m^beta dm */
    double Z2;
    if (fabs(1.0 + beta) < 1e-12) Z2 = log(m1 / mmin);
    else Z2 = (pow(m1, 1.0 + beta) - pow(mmin, 1.0 + beta)) / (1.0 + beta);
    const double p2 = pow(m2, beta) / Z2;
    /* explicit parameter derivatives of ln w */
    dlw[P_ALPHA] = cpl * PL * (-log(m1) - dZpl_da / Zpl);
    dlw[P_MU] = cg * G * (x / sg - (phia - phib) / (sg * ZG));
    dlw[P_SG] = cg * G * (-1.0 / sg + x * x / sg - (ua * phia - ub * phib) / (sg * ZG));
    dlw[P_MMIN] = cpl * PL * pow(mmin, -alpha) / Zpl + cg * G * phia / (sg * ZG) + pow(mmin, beta) / Z2;
    dlw[P_MMAX] = -cpl * PL * pow(mmax, -alpha) / Zpl - cg * G * phib / (sg * ZG);
    /* mass derivatives: d ln w / d m1, d ln w / d m2 */
    const double dl_dm1 = (cpl * PL * (-alpha / m1) + cg * G * (-x / sg)) - pow(m1, beta) / Z2;
    const double dl_dm2 = beta / m2;
    /* m = m_det / (1+z): d m / d ln(1+z) = -m */
    *dlna = -(m1 * dl_dm1 + m2 * dl_dm2);
    return p1 * p2;
}

/* ln psi and its derivatives (Sec. 3.1): dl[0..2] with respect to
 * (gamma, kappa, z_p) at fixed z, *dz = d ln psi / dz.                    */
static double psi_dlog(double z, const double *th, double *dl, double *dz) {
    const double gam = th[P_GAM], kap = th[P_KAP], zp = th[P_ZP];
    const double a = 1.0 + z, r = a / (1.0 + zp), rk = pow(r, gam + kap), q = rk / (1.0 + rk);
    dl[0] = log(a) - q * log(r);
    dl[1] = -q * log(r);
    dl[2] = (gam + kap) * q / (1.0 + zp);
    *dz = gam / a - (gam + kap) * q / a;
    return pow(a, gam) / (1.0 + rk);
}

/* The Scott bandwidth of Eq. gw-kernel's reading and its derivative from
 * the samples' dz[j][k] and dw[j][k] = d w_j / d theta_k (the same rule
 * and fallbacks as bandwidth_of). */
static double bandwidth_grad(int64_t n, const double *z, const double *w, const int32_t *valid,
                             const double *dz, const double *dw, double fallback, double *dlnb) {
    for (int k = 0; k < NP; k++) dlnb[k] = 0.0;
    double W1 = 0.0, W2 = 0.0, Wz = 0.0;
    for (int64_t j = 0; j < n; j++) {
        if (!valid[j]) continue;
        W1 += w[j]; W2 += w[j] * w[j]; Wz += w[j] * z[j];
    }
    if (W1 > 0.0) {
        double mean = Wz / W1, var = 0.0;
        for (int64_t j = 0; j < n; j++)
            if (valid[j]) var += w[j] * (z[j] - mean) * (z[j] - mean);
        var /= W1;
        double neff = W1 * W1 / W2;
        if (neff >= 2.0 && var > 0.0) {
            for (int k = 0; k < NP; k++) {
                double dW1 = 0.0, dW2 = 0.0, dV = 0.0;
                for (int64_t j = 0; j < n; j++) {
                    if (!valid[j]) continue;
                    const double dwj = dw[j * NP + k], dzj = k < 4 ? dz[j * 4 + k] : 0.0, u = z[j] - mean;
                    dW1 += dwj;
                    dW2 += 2.0 * w[j] * dwj;
                    dV += dwj * u * u + 2.0 * w[j] * u * dzj;
                }
                const double dvar = dV / W1 - var * dW1 / W1;
                dlnb[k] = 0.5 * dvar / var - 0.2 * (2.0 * dW1 / W1 - dW2 / W2);
            }
            return sqrt(var) * pow(neff, -0.2);
        }
    }
    int64_t nv = 0;
    double s = 0.0;
    for (int64_t j = 0; j < n; j++)
        if (valid[j]) { nv++; s += z[j]; }
    if (nv >= 2) {
        double mean = s / nv, var = 0.0;
        for (int64_t j = 0; j < n; j++)
            if (valid[j]) var += (z[j] - mean) * (z[j] - mean);
        var /= nv;
        if (var > 0.0) {
            for (int k = 0; k < 4; k++) {
                double dV = 0.0;
                for (int64_t j = 0; j < n; j++)
                    if (valid[j]) dV += 2.0 * (z[j] - mean) * dz[j * 4 + k];
                dlnb[k] = 0.5 * (dV / nv) / var;
            }
            return sqrt(var) * pow((double)nv, -0.2);
        }
    }
    return fallback;
}

/* KDE of one sample set on the grid with its derivatives (the same sum,
 * normalisation and support as kde_set, Gaussian kernel):
 * dK[a*NP + k] = d K(z_a) / d theta_k.  idx: the set's sample indices.   */
static void kde_set_grad(int64_t m, const int64_t *idx, const double *z, const double *w,
                         const int32_t *valid, const double *dz, const double *dw, double b,
                         const double *dlnb, int64_t nz, double z_max, double *K, double *dK) {
    double zlo = INFINITY, zhi = -INFINITY;
    for (int64_t q = 0; q < m; q++) {
        int64_t j = idx[q];
        if (valid[j]) { if (z[j] < zlo) zlo = z[j]; if (z[j] > zhi) zhi = z[j]; }
    }
    zlo -= ORC_KDE_MARGIN * b;
    zhi += ORC_KDE_MARGIN * b;
    const double norm = m > 0 ? 1.0 / (sqrt(2.0 * M_PI) * b * (double)m) : 0.0;
    for (int64_t a = 0; a < nz; a++) {
        double za = z_max * (double)a / (double)(nz - 1), s = 0.0, ds[NP];
        for (int k = 0; k < NP; k++) ds[k] = 0.0;
        if (za >= zlo && za <= zhi) {
            for (int64_t q = 0; q < m; q++) {
                int64_t j = idx[q];
                if (!valid[j] || w[j] == 0.0) continue;
                const double u = za - z[j], e = exp(-0.5 * u * u / (b * b));
                s += w[j] * e;
                for (int k = 0; k < NP; k++) {
                    double t = dw[j * NP + k] + w[j] * (u * u / (b * b) - 1.0) * dlnb[k];
                    if (k < 4) t += w[j] * u / (b * b) * dz[j * 4 + k];
                    ds[k] += e * t;
                }
            }
        }
        K[a] = s * norm;
        for (int k = 0; k < NP; k++) dK[a * NP + k] = ds[k] * norm;
    }
}

/* Galaxy term of one pixel and its Om derivative (Eq. p-cat as
 * galaxy_profile_dv; H0 cancels between dV_c/dz and Z_g). */
static void galaxy_profile_grad(const orc_catalog *c, int64_t ev, int32_t pixel, const double *dv,
                                const double *dv_Om, double vmax, double dlnvmax, double *G, double *dG) {
    int64_t p = c->pix_off[ev] + pixel;
    for (int64_t a = 0; a < c->n_z; a++) { G[a] = 0.0; dG[a] = 0.0; }
    for (int64_t g = c->gal_off[p]; g < c->gal_off[p + 1]; g++) {
        double zg = c->gal_z[g], sg = c->gal_sigma[g];
        double norm = 1.0 / (sqrt(2.0 * M_PI) * sg);
        double Z = 0.0, Zp = 0.0;
        for (int64_t a = 0; a < c->n_z; a++) {
            double u = (grid_z(c, a) - zg) / sg, Na = norm * exp(-0.5 * u * u);
            Z += grid_w(c, a) * Na * dv[a];
            Zp += grid_w(c, a) * Na * dv_Om[a];
        }
        if (!(Z > 0.0)) continue;
        for (int64_t a = 0; a < c->n_z; a++) {
            double u = (grid_z(c, a) - zg) / sg, Na = norm * exp(-0.5 * u * u);
            G[a] += Na / Z;
            dG[a] -= Na * Zp / (Z * Z);
        }
    }
    for (int64_t a = 0; a < c->n_z; a++) {
        const double S = G[a], dS = dG[a];
        G[a] = dv[a] * S / c->n_gal_total;
        dG[a] = (dv_Om[a] * S + dv[a] * dS) / c->n_gal_total;
    }
    if (c->completeness) {
        const double area = c->pix_area[p] / (4.0 * M_PI);
        const double *P = c->completeness + p * c->n_z;
        for (int64_t a = 0; a < c->n_z; a++) {
            const double miss = area * (1.0 - P[a]) * dv[a] / vmax;
            const double dmiss = area * (1.0 - P[a]) * (dv_Om[a] / vmax - dv[a] / vmax * dlnvmax);
            G[a] = c->f_R * G[a] + miss;
            dG[a] = c->f_R * dG[a] + dmiss;
        }
    }
}

/* ln I_i and d ln I_i / d theta (Eq. like-integrals). */
static double event_grad(const orc_catalog *c, const double *th, int64_t ev, const double *F,
                         const double *dlnF, const double *dv, const double *dv_Om, double vmax,
                         double dlnvmax, double *dlnI) {
    const int64_t j0 = c->sample_off[ev], n = c->sample_off[ev + 1] - j0, nz = c->n_z;
    const int32_t npix = (int32_t)(c->pix_off[ev + 1] - c->pix_off[ev]);
    double *z = malloc(sizeof(double) * (n + 1)), *w = malloc(sizeof(double) * (n + 1));
    int32_t *v = malloc(sizeof(int32_t) * (n + 1));
    double *dz = calloc((size_t)(n + 1) * 4, sizeof(double)), *dw = calloc((size_t)(n + 1) * NP, sizeof(double));
    int64_t *idx = malloc(sizeof(int64_t) * (n + 1));
    double *K = malloc(sizeof(double) * nz), *dK = malloc(sizeof(double) * nz * NP);
    double *G = malloc(sizeof(double) * nz), *dG = malloc(sizeof(double) * nz);
    double *Gs = calloc((size_t)nz, sizeof(double)), *dGs = calloc((size_t)nz, sizeof(double));
    for (int64_t j = 0; j < n; j++) {
        double zj = 0.0;
        v[j] = orc_z_of_dL(c->dL[j0 + j], th, &zj) == 0;
        z[j] = v[j] ? zj : 0.0;
        w[j] = 0.0;
        if (!v[j]) continue;
        cosmo_d cd;
        cosmo_at(zj, th, &cd);
        for (int k = 0; k < 4; k++) dz[j * 4 + k] = -cd.dd[k] / cd.J;   /* d_gw(z_j) = d_L,j */
        double dlw[NP], dlna;
        const double a = 1.0 + zj;
        w[j] = mass_dlog(c->m1d[j0 + j] / a, c->m2d[j0 + j] / a, th, c->lambda_g, c->beta, dlw, &dlna);
        for (int k = 0; k < NP; k++) {
            double t = dlw[k];
            if (k < 4) t += dlna / a * dz[j * 4 + k];
            dw[j * NP + k] = w[j] * t;
        }
    }
    double dlnb[NP];
    const double b = bandwidth_grad(n, z, w, v, dz, dw, grid_dz(c), dlnb);
    double I = 0.0, dI[NP];
    for (int k = 0; k < NP; k++) dI[k] = 0.0;
    if (c->kde_mode == ORC_KDE_MANY_1D) {
        for (int32_t k = 0; k < npix; k++) {
            int64_t m = 0;
            for (int64_t j = 0; j < n; j++)
                if (c->pix_of_sample[j0 + j] == k) idx[m++] = j;
            const double S = c->sky_S[c->pix_off[ev] + k];
            kde_set_grad(m, idx, z, w, v, dz, dw, b, dlnb, nz, c->z_max, K, dK);
            galaxy_profile_grad(c, ev, k, dv, dv_Om, vmax, dlnvmax, G, dG);
            for (int64_t a = 0; a < nz; a++) {
                const double wa = grid_w(c, a) * S;
                I += wa * K[a] * F[a] * G[a];
                for (int q = 0; q < NP; q++) {
                    double t = dK[a * NP + q] * F[a] * G[a] + K[a] * F[a] * dlnF[a * NP + q] * G[a];
                    if (q == P_OM) t += K[a] * F[a] * dG[a];
                    dI[q] += wa * t;
                }
            }
        }
    } else {
        for (int64_t j = 0; j < n; j++) idx[j] = j;
        kde_set_grad(n, idx, z, w, v, dz, dw, b, dlnb, nz, c->z_max, K, dK);
        for (int32_t k = 0; k < npix; k++) {
            const double S = c->sky_S[c->pix_off[ev] + k];
            galaxy_profile_grad(c, ev, k, dv, dv_Om, vmax, dlnvmax, G, dG);
            for (int64_t a = 0; a < nz; a++) { Gs[a] += S * G[a]; dGs[a] += S * dG[a]; }
        }
        for (int64_t a = 0; a < nz; a++) {
            const double wa = grid_w(c, a);
            I += wa * K[a] * F[a] * Gs[a];
            for (int q = 0; q < NP; q++) {
                double t = dK[a * NP + q] * F[a] * Gs[a] + K[a] * F[a] * dlnF[a * NP + q] * Gs[a];
                if (q == P_OM) t += K[a] * F[a] * dGs[a];
                dI[q] += wa * t;
            }
        }
    }
    for (int q = 0; q < NP; q++) dlnI[q] = I > 0.0 ? dI[q] / I : 0.0;
    free(z); free(w); free(v); free(dz); free(dw); free(idx); free(K); free(dK); free(G); free(dG);
    free(Gs); free(dGs);
    return (I > 0.0 && isfinite(I)) ? log(I) : -INFINITY;
}

/* xi (Eq. bias, Monte Carlo sum) and d ln xi / d theta. */
static double selection_grad(const orc_catalog *c, const double *th, double vmax, double dlnvmax,
                             int nthreads, double *dlnxi) {
    const int64_t n = c->n_det;
    double *s = malloc(sizeof(double) * (n + 1)), *ds = calloc((size_t)(n + 1) * NP, sizeof(double));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
    for (int64_t j = 0; j < n; j++) {
        s[j] = 0.0;
        double z = 0.0;
        if (orc_z_of_dL(c->inj_dL[j], th, &z) != 0 || !(z <= c->z_max)) continue;
        const double a = 1.0 + z;
        double dlw[NP], dlna, dpsi[3], dpsi_z;
        const double w = mass_dlog(c->inj_m1d[j] / a, c->inj_m2d[j] / a, th, c->lambda_g, c->beta, dlw, &dlna);
        if (!(w > 0.0)) continue;
        cosmo_d cd;
        cosmo_at(z, th, &cd);
        const double psi = psi_dlog(z, th, dpsi, &dpsi_z);
        const double pz = cd.dv / vmax;
        s[j] = w * psi * pz / (a * a * a * fabs(cd.J) * exp(c->inj_log_pi[j]));
        /* d ln s / dz at fixed theta and detector-frame masses */
        const double dls_dz = dlna / a + dpsi_z + cd.dlndv_dz - 3.0 / a - cd.Jz / cd.J;
        double g[NP];
        for (int k = 0; k < NP; k++) g[k] = dlw[k];
        g[P_GAM] += dpsi[0];
        g[P_KAP] += dpsi[1];
        g[P_ZP] += dpsi[2];
        g[P_OM] += (cd.Dc > 0.0 ? cd.dv_Om / cd.dv : 0.0) - dlnvmax;  /* p_z at fixed z */
        for (int k = 0; k < 4; k++) {
            const double dzk = -cd.dd[k] / cd.J;
            g[k] += -cd.dJ[k] / cd.J + dls_dz * dzk;
        }
        for (int k = 0; k < NP; k++) ds[j * NP + k] = s[j] * g[k];
    }
    double S1 = neumaier(s, n);
    for (int k = 0; k < NP; k++) {
        double acc = 0.0, comp = 0.0;
        for (int64_t j = 0; j < n; j++) {  /* Neumaier over the column */
            double x = ds[j * NP + k], t = acc + x;
            if (fabs(acc) >= fabs(x)) comp += (acc - t) + x; else comp += (x - t) + acc;
            acc = t;
        }
        dlnxi[k] = S1 > 0.0 ? (acc + comp) / S1 : 0.0;
    }
    free(s); free(ds);
    return S1 / (double)c->n_inj_total;
}

/* ln L (Eq. hyperlike) and its gradient with respect to the 12 parameters.
 * Gaussian kernel with the Jacobian on the grid, many-1D or single-1D,
 * complete or incomplete catalog; an inadmissible or non-monotone point has
 * ln L = -inf and gradient 0. */
int orc_grad(const orc_catalog *c, const double *th, int nthreads, double *lnL, double *grad,
             int32_t *status) {
    for (int k = 0; k < NP; k++) grad[k] = 0.0;
    *status = ORC_OK;
    if (orc_check_theta(th)) { *lnL = -INFINITY; *status = ORC_OUT_OF_SUPPORT; return 0; }
    if (!orc_monotone(th)) { *lnL = -INFINITY; *status = ORC_NONMONOTONE; return 0; }
    const int64_t ne = c->n_events, nz = c->n_z;
    double *F = malloc(sizeof(double) * nz), *dlnF = calloc((size_t)nz * NP, sizeof(double));
    double *dv = malloc(sizeof(double) * nz), *dv_Om = malloc(sizeof(double) * nz);
    for (int64_t a = 0; a < nz; a++) {
        const double za = grid_z(c, a);
        cosmo_d cd;
        cosmo_at(za, th, &cd);
        double dpsi[3], dpsi_z;
        const double psi = psi_dlog(za, th, dpsi, &dpsi_z), ap = 1.0 + za;
        F[a] = psi / (ap * ap * ap * fabs(cd.J));
        for (int k = 0; k < 4; k++) dlnF[a * NP + k] = -cd.dJ[k] / cd.J;
        dlnF[a * NP + P_GAM] = dpsi[0];
        dlnF[a * NP + P_KAP] = dpsi[1];
        dlnF[a * NP + P_ZP] = dpsi[2];
        dv[a] = cd.dv;
        dv_Om[a] = cd.dv_Om;
    }
    const double Dm = orc_Dc(c->z_max, th[P_H0], th[P_OM]);
    const double vmax = orc_Vc(c->z_max, th[P_H0], th[P_OM]);
    const double dlnvmax = 3.0 * orc_dDc_dOm(c->z_max, th[P_H0], th[P_OM]) / Dm;
    double *lnI = malloc(sizeof(double) * (ne + 1)), *dlnI = malloc(sizeof(double) * (ne + 1) * NP);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < ne; i++)
        lnI[i] = event_grad(c, th, i, F, dlnF, dv, dv_Om, vmax, dlnvmax, dlnI + i * NP);
    double dlnxi[NP];
    const double xi = selection_grad(c, th, vmax, dlnvmax, nthreads, dlnxi);
    int bad = !(xi > 0.0);
    for (int64_t i = 0; i < ne; i++) bad |= !isfinite(lnI[i]);
    if (bad) {
        *lnL = -INFINITY;
        *status = ORC_OUT_OF_SUPPORT;
    } else {
        *lnL = neumaier(lnI, ne) - (double)ne * log(xi);
        for (int k = 0; k < NP; k++) {
            double acc = 0.0;
            for (int64_t i = 0; i < ne; i++) acc += dlnI[i * NP + k];
            grad[k] = acc - (double)ne * dlnxi[k];
        }
    }
    free(F); free(dlnF); free(dv); free(dv_Om); free(lnI); free(dlnI);
    return 0;
}
