// K7: hand-written adjoint of ln L with respect to the 12 hyperparameters
// (H0, Om, Xi0, n, alpha, mu_g, sigma_g, m_min, m_max, gamma, kappa, z_p).
//
// ln L = sum_i ln I_i - N_obs ln xi                            (Eq. hyperlike)
//
// Event term.  In grid units I_i' = sum_k pf_k sum_{j in k} w_j S0_j with
//   S0_j = sum_a e_ja H_k(a), e_ja = exp(-u_ja^2/2), u_ja = (z_a - z_j)/b,
//   H_k(a) = w'_a F(z_a) G_k(z_a),  and ln I_i = ln I_i' - ln b + const.
// Differentiating (the KDE is recomputed, nothing per pair is stored):
//   dI'/dtheta = sum pf w [ S0 dln w/dtheta + (S1 / b) dz/dtheta ]
//              + S2tot dln b/dtheta + sum_a M(a) dln F(z_a)/dtheta
//              + [Om only] sum_k pf_k sum_a w'_a F K_k(a) dG_k(a)/dOm,
//   S1_j = sum_a e H u, S2_j = sum_a e H u^2, S2tot = sum pf w S2,
//   K_k(a) = sum_{j in k} w_j e_ja (the pixel KDE on the grid, recomputed
//   grid-point by grid-point), M(a) = sum_k pf_k H_k(a) K_k(a).
// z_j depends on (H0, Om, Xi0, n) through d_L^gw(z_j) = d_j (Eq. dL-mg),
// dz/dtheta = -(d d_L^gw/dtheta)/J; w_j on the mass parameters and on z_j
// through m = m_det/(1+z) (Sec. 2.1); b on every sample through Scott's rule
// (weighted mean/variance and n_eff).  The edges of the mass ranges and of
// the KDE windows are not differentiated (the almost-everywhere derivative).
//
// Selection term (Eq. bias as the injection sum):
//   dxi/dtheta = (1/N_inj) sum_j s_j dln s_j/dtheta,
//   ln s = ln p(m1,m2) + ln psi(z) + ln p_z(z) - 3 ln(1+z) - ln J(z) - ln pi_inj,
// with the chain through z_j for the cosmological parameters.
#include <algorithm>
#include <type_traits>
#include <map>

#include <cuda_fp16.h>
#include <math_constants.h>

#include "mass.cuh"
#include "runtime.cuh"

namespace chim {

// Per-hyperpoint constants of the adjoint (FP64).
struct HPd {
    double dlc_pl[3];  // d ln c_pl / d(alpha, m_min, m_max)
    double dlc_g[4];   // d ln c_g / d(mu_g, sigma_g, m_min, m_max)
    double dlpz_zmax;  // d ln [1 / V_c(z_max)] / dOm
    float dlc_pl32[3], dlc_g32[4], dlpz_zmax32;  // FP32 copies (mixed adjoint)
};

// Device views of the adjoint's inputs and scratch.
struct AdjPtrs {
    const double *const *fwdO;   // [H] dDhat/dOm table of h's Om
    const double *const *dprof;  // [H] dG/dOm profile of h's Om (rows as the forward profile; FP32 values on the mixed path)
    HPd *hpd;                    // [H]
    double *dznode;              // [H x (NU+1) x 4] dz/d(H0, Om, Xi0, n) at the inverse-table nodes
    float4 *dznode32;            // [H x (NU+1)] FP32 copy
    double *Q;                   // [H x n_z x 7] d ln F / d(H0, Om, Xi0, n, gamma, kappa, z_p)
    float *QT;                   // [H x n_z x AM_QT] FP32 (Q_k, dQ_k/dz, d2Q_k/dz2 / 2), k = Om .. z_p
    double *dlnI;                // [H x n_events x 12]
    double *selg;                // [H x n_chunk x 13] sum s dln s / dtheta (12), sum s
    double *grad;                // [H x 12]
};

namespace {

using chimd::dcO_hermite;
constexpr int ADJ_THREADS = 256;

// Transcendentals of the derivative helpers below: libm in FP64, the SFU
// intrinsics in FP32.  The mixed gradient is held to 2e-3 of the FP64 one,
// far above the intrinsics' ~1e-6 relative error, and they cost a few
// instructions instead of tens.
__device__ __forceinline__ double ax_exp(double x) { return exp(x); }
__device__ __forceinline__ float ax_exp(float x) { return __expf(x); }
__device__ __forceinline__ double ax_log(double x) { return log(x); }
__device__ __forceinline__ float ax_log(float x) { return __logf(x); }
__device__ __forceinline__ double ax_pow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float ax_pow(float x, float y) { return __powf(x, y); }

// Derivatives of the distance relation at redshift z for one hyperpoint
// (Eq. dL-mg and its z-derivative J), given Dh = D_c / (c/H0) and
// DhO = dDh/dOm at z.
template <typename T>
struct ZDerT {
    T dz[4];      // dz/d(H0, Om, Xi0, n) at fixed d_L
    T dlnJ[4];    // d ln J / d(H0, Om, Xi0, n) at fixed z
    T dlnJ_dz;    // d ln J / dz
    T dlnpz_dOm;  // d ln p_z / dOm at fixed z (p_z = dV/dz / V(z_max))
    T dlnpz_dz;
};
using ZDer = ZDerT<double>;

template <typename T>
__device__ ZDerT<T> zder_t(T z, T H0, T Om, T Xi0, T n, T Dh, T DhO, T dlpz_zmax) {
    ZDerT<T> r;
    const T one = T(1), cH = T(C_KMS) / H0, a = one + z;
    const T E = sqrt(Om * a * a * a + one - Om), iE = one / E;
    const T D = cH * Dh, DO = cH * DhO;
    const T la = ax_log(a), pw = ax_exp(-n * la);
    const T xi = Xi0 + (one - Xi0) * pw, dxi = -n * (one - Xi0) * pw / a;
    const T P = D + a * cH * iE;  // d d_L^em / dz
    const T J = P * xi + a * D * dxi;
    const T d = a * D * xi;
    const T dd[4] = {-d / H0, a * DO * xi, a * D * (one - pw), -a * D * (one - Xi0) * la * pw};
    for (int k = 0; k < 4; k++) r.dz[k] = -dd[k] / J;
    const T diE_dOm = -(a * a * a - one) * T(0.5) * iE * iE * iE;
    const T dxi_dn = -(one - Xi0) * la * pw, ddxi_dn = (one - Xi0) * (pw / a) * (n * la - one);
    const T dJ[4] = {-J / H0, (DO + a * cH * diE_dOm) * xi + a * DO * dxi, P * (one - pw) + D * n * pw,
                     P * dxi_dn + a * D * ddxi_dn};
    for (int k = 0; k < 4; k++) r.dlnJ[k] = dJ[k] / J;
    const T Ep = T(1.5) * Om * a * a * iE;  // dE/dz
    const T d2xi = n * (n + one) * (one - Xi0) * pw / (a * a);
    const T dJdz = (T(2) * cH * iE - a * cH * Ep * iE * iE) * xi + T(2) * P * dxi + a * D * d2xi;
    r.dlnJ_dz = dJdz / J;
    r.dlnpz_dOm = T(2) * DhO / Dh - (a * a * a - one) * T(0.5) * iE * iE + dlpz_zmax;
    r.dlnpz_dz = T(2) * iE / Dh - Ep * iE;
    return r;
}

__device__ ZDer zder(double z, const double *th, const double *fwd, const double *fwdO, double dlpz_zmax) {
    return zder_t<double>(z, th[0], th[1], th[2], th[3], chimd::dc_hermite(fwd, z, th[1]),
                          dcO_hermite(fwdO, z, th[1]), dlpz_zmax);
}

// d ln psi / d(gamma, kappa, z_p) and d ln psi / dz (Sec. 3.1)
template <typename T>
__device__ void dlnpsi_t(T z, T gam, T kap, T zp, T *g3, T *dz) {
    const T one = T(1), a = one + z;
    const T L = ax_log(a / (one + zp));
    const T x = ax_exp((gam + kap) * L);
    const T r = x / (one + x);
    g3[0] = ax_log(a) - r * L;
    g3[1] = -r * L;
    g3[2] = r * (gam + kap) / (one + zp);
    *dz = gam / a - r * (gam + kap) / a;
}
__device__ void dlnpsi(double z, const double *th, double *g3, double *dz) {
    dlnpsi_t<double>(z, th[9], th[10], th[11], g3, dz);
}

// Mass-model log-derivatives for source masses (m1, m2): direct derivatives
// d ln p / d(alpha, mu, sigma, m_min, m_max) and d ln p / dz through
// m = m_det / (1+z).  Zero when the weight is zero.
template <typename T>
struct MassDer {
    T alpha, mu, sg, mmin, mmax, c_pl, c_g, b1, mmin_b1, beta;
    T dlc_pl[3], dlc_g[4];
};

template <typename T>
__device__ void dlnpm_t(const MassDer<T> &md, T m1, T m2, T a, T *d5, T *ddz) {
    for (int k = 0; k < 5; k++) d5[k] = T(0);
    *ddz = T(0);
    const T one = T(1);
    if (!(m1 >= md.mmin && m1 <= md.mmax && m2 >= md.mmin && m2 <= m1) || !(m1 > md.mmin)) return;
    const T isg = one / md.sg, x = (m1 - md.mu) * isg;
    const T PL = md.c_pl * ax_pow(m1, -md.alpha), GG = md.c_g * ax_exp(T(-0.5) * x * x);
    const T p1 = PL + GG;
    if (!(p1 > T(0))) return;
    const T ip1 = one / p1;
    d5[0] = PL * (md.dlc_pl[0] - ax_log(m1)) * ip1;
    d5[1] = GG * (md.dlc_g[0] + x * isg) * ip1;
    d5[2] = GG * (md.dlc_g[1] + x * x * isg) * ip1;
    d5[3] = (PL * md.dlc_pl[1] + GG * md.dlc_g[2]) * ip1;
    d5[4] = (PL * md.dlc_pl[2] + GG * md.dlc_g[3]) * ip1;
    const T dp1_dm1 = (-md.alpha * PL / m1 - GG * x * isg) * ip1;
    T dp2_dm1, dp2_dm2, dp2_dmin;
    if (fabs(md.b1) < T(1e-6)) {
        const T L = ax_log(m1 / md.mmin);
        dp2_dm1 = -one / (m1 * L);
        dp2_dm2 = -one / m2;
        dp2_dmin = one / (md.mmin * L);
    } else {
        const T q = ax_pow(m1, md.b1) - md.mmin_b1;
        dp2_dm1 = -md.b1 * ax_pow(m1, md.beta) / q;
        dp2_dm2 = md.beta / m2;
        dp2_dmin = md.b1 * ax_pow(md.mmin, md.beta) / q;
    }
    d5[3] += dp2_dmin;
    *ddz = -(m1 * (dp1_dm1 + dp2_dm1) + m2 * dp2_dm2) / a;
}

__device__ MassDer<double> mass_der64(const HP &hp, const HPd &hd, double beta) {
    MassDer<double> md;
    md.alpha = hp.th[4]; md.mu = hp.th[5]; md.sg = hp.th[6]; md.mmin = hp.th[7]; md.mmax = hp.th[8];
    md.c_pl = hp.c_pl; md.c_g = hp.c_g; md.b1 = hp.b1; md.mmin_b1 = hp.mmin_b1; md.beta = beta;
    for (int k = 0; k < 3; k++) md.dlc_pl[k] = hd.dlc_pl[k];
    for (int k = 0; k < 4; k++) md.dlc_g[k] = hd.dlc_g[k];
    return md;
}

__device__ MassDer<float> mass_der32(const HP &hp, const HPd &hd) {
    MassDer<float> md;
    md.alpha = hp.alpha32; md.mu = hp.mu32; md.sg = (float)hp.th[6]; md.mmin = hp.mmin32; md.mmax = hp.mmax32;
    md.c_pl = hp.c_pl32; md.c_g = hp.c_g32; md.b1 = hp.b1_32; md.mmin_b1 = hp.mmin_b1_32; md.beta = hp.beta32;
    for (int k = 0; k < 3; k++) md.dlc_pl[k] = hd.dlc_pl32[k];
    for (int k = 0; k < 4; k++) md.dlc_g[k] = hd.dlc_g32[k];
    return md;
}

__device__ double std_normal_pdf(double x) { return 0.39894228040143267794 * exp(-0.5 * x * x); }

// ---- per-hyperpoint derivative tables (blockIdx.y splits the nodes and
// grid points of one hyperpoint over several blocks) ----
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_tables(DevCatalog c, CallPtrs p, AdjPtrs q) {
    const int h = blockIdx.x;
    const int t = blockIdx.y * ADJ_THREADS + threadIdx.x, nt = gridDim.y * ADJ_THREADS;
    const HP &hp = p.hp[h];
    const double *th = hp.th;
    const double *fwd = p.fwd[h], *fwdO = q.fwdO[h];
    if (t == 0) {
        HPd hd;
        const double alpha = th[4], mu = th[5], sg = th[6], mmin = th[7], mmax = th[8];
        const double s1 = 1.0 - alpha;
        double PL, dPLds;
        const double la = log(mmax), lb = log(mmin);
        if (fabs(s1) < 1e-12) {
            PL = la - lb;
            dPLds = 0.5 * (la * la - lb * lb);
        } else {
            const double A = pow(mmax, s1), B = pow(mmin, s1);
            PL = (A - B) / s1;
            dPLds = ((la * A - lb * B) * s1 - (A - B)) / (s1 * s1);
        }
        hd.dlc_pl[0] = dPLds / PL;  // d ln c_pl / d alpha = -(dPL/dalpha)/PL, dPL/dalpha = -dPL/ds
        hd.dlc_pl[1] = pow(mmin, -alpha) / PL;
        hd.dlc_pl[2] = -pow(mmax, -alpha) / PL;
        const double A = (mmin - mu) / sg, B = (mmax - mu) / sg;
        const double den = 0.5 * erfc(-B * 0.70710678118654752440) - 0.5 * erfc(-A * 0.70710678118654752440);
        const double pA = std_normal_pdf(A), pB = std_normal_pdf(B);
        if (den > 0.0) {
            hd.dlc_g[0] = -((pA - pB) / sg) / den;
            hd.dlc_g[1] = -1.0 / sg - ((A * pA - B * pB) / sg) / den;
            hd.dlc_g[2] = pA / (sg * den);
            hd.dlc_g[3] = -pB / (sg * den);
        } else {
            hd.dlc_g[0] = hd.dlc_g[1] = hd.dlc_g[2] = hd.dlc_g[3] = 0.0;
        }
        const double zm = c.z_max;
        hd.dlpz_zmax = -3.0 * dcO_hermite(fwdO, zm, th[1]) / chimd::dc_hermite(fwd, zm, th[1]);
        for (int k = 0; k < 3; k++) hd.dlc_pl32[k] = (float)hd.dlc_pl[k];
        for (int k = 0; k < 4; k++) hd.dlc_g32[k] = (float)hd.dlc_g[k];
        hd.dlpz_zmax32 = (float)hd.dlpz_zmax;
        q.hpd[h] = hd;
    }
    // dz/dtheta at the inverse-table nodes
    const double2 *nd = p.inv64 + (size_t)h * (NU + 1);
    for (int k = t; k <= NU; k += nt) {
        double z = nd[k].x;
        double *o = q.dznode + ((size_t)h * (NU + 1) + k) * 4;
        if (k == 0 || !isfinite(z)) {
            for (int j = 0; j < 4; j++) o[j] = 0.0;
            q.dznode32[(size_t)h * (NU + 1) + k] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        ZDer r = zder(z, th, fwd, fwdO, 0.0);
        for (int j = 0; j < 4; j++) o[j] = r.dz[j];
        q.dznode32[(size_t)h * (NU + 1) + k] = make_float4((float)r.dz[0], (float)r.dz[1], (float)r.dz[2], (float)r.dz[3]);
    }
    // d ln F / dtheta on the grid, F = psi / ((1+z)^3 J)
    for (int a = t; a < c.n_z; a += nt) {
        double z = a * c.dz;
        ZDer r = zder(z, th, fwd, fwdO, 0.0);
        double g3[3], dz;
        dlnpsi(z, th, g3, &dz);
        double *o = q.Q + ((size_t)h * c.n_z + a) * 7;
        for (int j = 0; j < 4; j++) o[j] = -r.dlnJ[j];
        o[4] = g3[0];
        o[5] = g3[1];
        o[6] = g3[2];
    }
}

// The FP32 second-order Taylor table of d ln F / dtheta on the grid for the
// mixed adjoint: per grid point and k = Om, Xi0, n, gamma, kappa, z_p the
// value, first derivative and half the second derivative in z, by central
// differences of the FP64 table (one-sided at the grid ends).
constexpr int AM_QT = 20;  // 18 used, padded to five float4
__global__ void k_q_taylor(DevCatalog c, AdjPtrs q, int H) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int nz = c.n_z;
    if (i >= (int64_t)H * nz) return;
    const int h = (int)(i / nz), a = (int)(i % nz);
    float *o = q.QT + (size_t)i * AM_QT;
    if (nz < 3) {  // no stencil: the value alone
        const double *Qa = q.Q + ((size_t)h * nz + a) * 7;
        for (int k = 1; k < 7; k++) {
            o[3 * (k - 1)] = (float)Qa[k];
            o[3 * (k - 1) + 1] = 0.f;
            o[3 * (k - 1) + 2] = 0.f;
        }
        o[18] = o[19] = 0.f;
        return;
    }
    const int am = a == 0 ? 0 : (a == nz - 1 ? nz - 3 : a - 1);  // three consecutive points
    const double *Q = q.Q + ((size_t)h * nz + am) * 7;
    const double idz = 1.0 / c.dz, t = (double)(a - am - 1);  // a relative to the middle point
    for (int k = 1; k < 7; k++) {
        const double q0 = Q[k], q1 = Q[7 + k], q2 = Q[14 + k];
        const double d1 = 0.5 * (q2 - q0) * idz, d2 = (q2 - 2.0 * q1 + q0) * idz * idz;
        // value and slope at a from the parabola through the three points
        o[3 * (k - 1)] = (float)(q1 + d1 * t * c.dz + 0.5 * d2 * t * t * c.dz * c.dz);
        o[3 * (k - 1) + 1] = (float)(d1 + d2 * t * c.dz);
        o[3 * (k - 1) + 2] = (float)(0.5 * d2);
    }
    o[18] = 0.f;
    o[19] = 0.f;
}

// dz/dtheta of a sample by linear interpolation between inverse-table nodes
__device__ __forceinline__ void dz_interp(const AdjPtrs &q, int h, int k, double f, double *dz) {
    const double *a = q.dznode + ((size_t)h * (NU + 1) + k) * 4;
    for (int j = 0; j < 4; j++) dz[j] = a[j] + f * (a[4 + j] - a[j]);
}

template <int NV>
__device__ void bsum(double (&v)[NV], double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double s = v[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[wid * NV + k] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < ADJ_THREADS / 32; w++) s += red[w * NV + threadIdx.x];
        red[(ADJ_THREADS / 32) * NV + threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = red[(ADJ_THREADS / 32) * NV + k];
    __syncthreads();
}

// Per (event, hyperpoint) on the FP64 path: d ln I_i / d theta (12),
// following the FP64 forward kernel (inversion with Newton polish, +-9 b
// windows, FP64 profile) in double, so that the gradient is that of the
// computed ln L.
__global__ void __launch_bounds__(ADJ_THREADS) k_event_adj(DevCatalog c, CallPtrs p, AdjPtrs q, int H) {
    extern __shared__ double sh[];
    double *zs = sh;
    double *ws = zs + c.max_ns;
    const int segn = (c.max_seg + 2) & ~1;
    int *segv = reinterpret_cast<int *>(ws + c.max_ns);
    int *sA0 = segv + segn;   // first grid point of each segment's KDE support
    int *scum = sA0 + segn;   // exclusive prefix of the support lengths
    double *red = reinterpret_cast<double *>(scum + segn);
    const int h = blockIdx.x % H;
    const int ev = c.ev_order[blockIdx.x / H];
    const int tid = threadIdx.x;
    const HP &hp = p.hp[h];
    const HPd &hd = q.hpd[h];
    double *out = q.dlnI + ((size_t)h * c.n_events + ev) * 12;
    if (hp.status & (CHIMERA_PT_OUT_OF_SUPPORT | CHIMERA_PT_NONMONOTONE)) {
        if (tid < 12) out[tid] = 0.0;
        return;
    }
    // grid factor x trapezoid weight
    auto Fw = [&](int a) -> double {
        return ((a == 0 || a == c.n_z - 1) ? 0.5 : 1.0) * p.F64[(size_t)h * c.n_z + a];
    };
    const int64_t s0 = c.ev_soff[ev];
    const int ns = (int)(c.ev_soff[ev + 1] - s0);
    const double KW = KW64;
    // ---- z_j, w_j exactly as the FP64 forward kernel
    for (int j = tid; j < ns; j += ADJ_THREADS) {
        double z = CUDART_INF, w = 0.0, zz;
        if (invert64(c, p, h, hp, c.sd64[s0 + j], &zz)) {
            z = zz;
            w = mass_weight64(hp, c.beta, c.sm1_64[s0 + j] / (1.0 + zz), c.sm2_64[s0 + j] / (1.0 + zz));
        }
        zs[j] = z;
        ws[j] = w;
    }
    __syncthreads();
    // ---- moments (two-pass) and Scott's rule
    double m5[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // W1, Wz, W2, n_valid, Sz
    for (int j = tid; j < ns; j += ADJ_THREADS)
        if (zs[j] < CUDART_INF) {
            const double z = zs[j], w = ws[j];
            m5[0] += w; m5[1] += w * z; m5[2] += w * w; m5[3] += 1.0; m5[4] += z;
        }
    bsum<5>(m5, red);
    const double W1 = m5[0], W2 = m5[2], nv = m5[3];
    const double Mw = W1 > 0.0 ? m5[1] / W1 : 0.0, Mu = nv > 0.0 ? m5[4] / nv : 0.0;
    double m2v[2] = {0.0, 0.0};
    for (int j = tid; j < ns; j += ADJ_THREADS)
        if (zs[j] < CUDART_INF) {
            const double z = zs[j], w = ws[j];
            m2v[0] += w * (z - Mw) * (z - Mw);
            m2v[1] += (z - Mu) * (z - Mu);
        }
    bsum<2>(m2v, red);
    const double varw = W1 > 0.0 ? m2v[0] / W1 : 0.0, neffw = W1 > 0.0 ? W1 * W1 / W2 : 0.0;
    const double varu = nv > 0.0 ? m2v[1] / nv : 0.0;
    int rule;  // 0 weighted, 1 unweighted, 2 grid spacing
    double b;
    if (W1 > 0.0 && neffw >= 2.0 && varw > 0.0) {
        rule = 0;
        b = sqrt(varw) * pow(neffw, -0.2);
    } else if (nv >= 2.0 && varu > 0.0) {
        rule = 1;
        b = sqrt(varu) * pow(nv, -0.2);
    } else {
        rule = 2;
        b = c.dz;
    }

    // segment valid counts
    const int sg0 = c.ev_segoff[ev], nseg = c.ev_segoff[ev + 1] - sg0;
    for (int k = tid; k < nseg; k += ADJ_THREADS) {
        int lo = (int)(c.seg_soff[sg0 + k] - s0), hi = (int)(c.seg_soff[sg0 + k + 1] - s0);
        int l = lo, r = hi;
        while (l < r) {
            int m = (l + r) >> 1;
            if (zs[m] < CUDART_INF) l = m + 1; else r = m;
        }
        segv[k] = l - lo;
    }
    __syncthreads();

    // ---- per-sample derivatives: bandwidth gradient and the sample sums
    const int nz = c.n_z;
    const double dz = c.dz, ib = 1.0 / b;
    const double cw0 = W1 > 0.0 ? 1.0 / (W1 * varw) : 0.0, cw1 = W1 > 0.0 ? 2.0 / W1 : 0.0;
    const double cw2 = W2 > 0.0 ? 2.0 / W2 : 0.0, cu = nv > 0.0 && varu > 0.0 ? 1.0 / (nv * varu) : 0.0;
    const double *prof = reinterpret_cast<const double *>(p.prof[h]);
    auto Gv = [&](int64_t row, int a) -> double { return prof[row * nz + a]; };
    const MassDer<double> md64 = mass_der64(hp, hd, c.beta);
    double A9[9], B4[4], db9[9], S2t = 0.0, I0 = 0.0;
    for (int k = 0; k < 9; k++) { A9[k] = 0.0; db9[k] = 0.0; }
    for (int k = 0; k < 4; k++) B4[k] = 0.0;
    for (int j = tid; j < ns; j += ADJ_THREADS) {
        int l = 0, r = nseg;  // segment of j
        while (r - l > 1) {
            int m = (l + r) >> 1;
            if ((int)(c.seg_soff[sg0 + m] - s0) <= j) l = m; else r = m;
        }
        const int lo = (int)(c.seg_soff[sg0 + l] - s0);
        if (j - lo >= segv[l]) continue;
        const double z = zs[j], w = ws[j], a1 = 1.0 + z;
        // dz/dtheta (linear between inverse-table nodes) and d ln w/dtheta
        double dd[4], d5[5], dwz;
        {
            const double t = sqrt(c.sd64[s0 + j] / c.d_top) * NU;
            const int kk = min((int)t, NU - 1);
            dz_interp(q, h, kk, t - kk, dd);
        }
        dlnpm_t<double>(md64, c.sm1_64[s0 + j] / a1, c.sm2_64[s0 + j] / a1, a1, d5, &dwz);
        double dlw[9];
        for (int k = 0; k < 4; k++) dlw[k] = dwz * dd[k];
        for (int k = 0; k < 5; k++) dlw[4 + k] = d5[k];
        // Scott's rule: d ln b = sum_j (dlnb/dw_j) w_j dln w_j + (dlnb/dz_j) dz_j
        if (rule == 0) {
            const double cw = 0.5 * ((z - Mw) * (z - Mw) - varw) * cw0 - 0.2 * (cw1 - w * cw2);
            const double cz = w * (z - Mw) * cw0;
            for (int k = 0; k < 9; k++) db9[k] += cw * w * dlw[k] + (k < 4 ? cz * dd[k] : 0.0);
        } else if (rule == 1) {
            const double cz = (z - Mu) * cu;
            for (int k = 0; k < 4; k++) db9[k] += cz * dd[k];
        }
        if (w == 0.0) continue;
        // window sums S0, S1, S2 of e = exp(-u^2/2) H, u = (z_a - z)/b
        const double pf = c.seg_pf[sg0 + l];
        const int64_t row = c.kde_mode == CHIMERA_KDE_MANY_1D ? (int64_t)(sg0 + l) : (int64_t)ev;
        const double smin = zs[lo] - KDE_MARGIN * b, smax = zs[lo + segv[l] - 1] + KDE_MARGIN * b;
        const double a0 = fmax(ceil((z - KW * b) / dz), ceil(smin / dz));
        const double aa1 = fmin(floor((z + KW * b) / dz), floor(smax / dz));
        const int ia0 = a0 < 0.0 ? 0 : (a0 > nz ? nz : (int)a0);
        const int ia1 = aa1 > nz - 1 ? nz - 1 : (aa1 < -1.0 ? -1 : (int)aa1);
        double S0 = 0.0, S1 = 0.0, S2 = 0.0;
        if (ia0 <= ia1) {
            // exp(-u^2/2) along the window by the Gaussian recurrence
            // g_{a+1} = g_a r_a, r_{a+1} = r_a e^{-delta^2}, delta = dz / b
            // (two exponentials per sample; relative drift ~1e-14)
            const double dlt = dz * ib, u0 = (ia0 * dz - z) * ib;
            double g = exp(-0.5 * u0 * u0), r = exp(-u0 * dlt - 0.5 * dlt * dlt);
            const double qq = exp(-dlt * dlt);
            for (int a = ia0; a <= ia1; a++) {
                const double Hh = Fw(a) * Gv(row, a);
                const double u = (a * dz - z) * ib;
                const double e = g * Hh;
                S0 += e;
                S1 += e * u;
                S2 += e * u * u;
                g *= r;
                r *= qq;
            }
        }
        const double pw = pf * w;
        I0 += pw * S0;
        S2t += pw * S2;
        for (int k = 0; k < 9; k++) A9[k] += pw * S0 * dlw[k];
        for (int k = 0; k < 4; k++) B4[k] += pw * S1 * ib * dd[k];
    }
    // ---- grid term: the KDE K_k(a) at every grid point of every segment's
    // support; the (segment, grid point) items are spread over all threads
    for (int l = tid; l < nseg; l += ADJ_THREADS) {
        const int lo = (int)(c.seg_soff[sg0 + l] - s0), cnt = segv[l];
        int alo = 0, len = 0;
        if (cnt > 0) {
            const double smin = zs[lo] - KDE_MARGIN * b, smax = zs[lo + cnt - 1] + KDE_MARGIN * b;
            alo = max(0, (int)ceil(smin / dz));
            len = max(0, min(nz - 1, (int)floor(smax / dz)) - alo + 1);
        }
        sA0[l] = alo;
        scum[l + 1] = len;
    }
    __syncthreads();
    if (tid < 32) {  // in-place inclusive scan of scum[1 .. nseg] by warp 0
        int carry = 0;
        for (int b0 = 1; b0 <= nseg; b0 += 32) {
            const int i = b0 + tid;
            int v = i <= nseg ? scum[i] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, v, o);
                if (tid >= o) v += y;
            }
            if (i <= nseg) scum[i] = v + carry;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
        if (tid == 0) scum[0] = 0;
    }
    __syncthreads();
    double C8[8];  // 7 d ln F terms + the galaxy Om term
    for (int k = 0; k < 8; k++) C8[k] = 0.0;
    const int nitems = scum[nseg];
    for (int it = tid; it < nitems; it += ADJ_THREADS) {
        int l = 0, r = nseg;  // the segment: last l with scum[l] <= it
        while (r - l > 1) {
            const int m = (l + r) >> 1;
            if (scum[m] <= it) l = m; else r = m;
        }
        const int lo = (int)(c.seg_soff[sg0 + l] - s0), cnt = segv[l];
        const int a = sA0[l] + (it - scum[l]);
        const double pf = c.seg_pf[sg0 + l];
        const int64_t row = c.kde_mode == CHIMERA_KDE_MANY_1D ? (int64_t)(sg0 + l) : (int64_t)ev;
        const double za = a * dz;
        // samples whose window covers a: |z - za| <= KW b
        int jl = lo, jr = lo + cnt;
        while (jl < jr) {
            const int m = (jl + jr) >> 1;
            if (zs[m] < za - KW * b) jl = m + 1; else jr = m;
        }
        double K = 0.0;
        for (int j = jl; j < lo + cnt && zs[j] <= za + KW * b; j++) {
            const double u = (za - zs[j]) * ib;
            K += ws[j] * exp(-0.5 * u * u);
        }
        if (K == 0.0) continue;
        const double FK = pf * Fw(a) * K;
        const double M = FK * Gv(row, a);
        const double *Qa = q.Q + ((size_t)h * nz + a) * 7;
        for (int k = 0; k < 7; k++) C8[k] += M * Qa[k];
        C8[7] += FK * q.dprof[h][row * nz + a];
    }
    // ---- block sums (double) and the 12 derivatives
    double v[28];
    for (int k = 0; k < 9; k++) v[k] = A9[k];
    for (int k = 0; k < 4; k++) v[9 + k] = B4[k];
    v[13] = S2t;
    v[14] = I0;
    for (int k = 0; k < 8; k++) v[15 + k] = C8[k];
    for (int k = 0; k < 5; k++) v[23 + k] = 0.0;
    double vb[9];
    for (int k = 0; k < 9; k++) vb[k] = db9[k];
    bsum<28>(v, red);
    bsum<9>(vb, red);
    if (tid == 0) {
        const double I = v[14];
        double g[12];
        for (int k = 0; k < 12; k++) g[k] = 0.0;
        if (I > 0.0) {
            // cosmology (H0, Om, Xi0, n): w through z, z directly, b, grid factor
            for (int k = 0; k < 4; k++)
                g[k] = (v[k] + v[9 + k] + v[13] * vb[k] + v[15 + k]) / I - vb[k];
            g[1] += v[22] / I;  // galaxy prior through dV_c/dz and the Z_g
            // mass parameters: w directly and b
            for (int k = 0; k < 5; k++) g[4 + k] = (v[4 + k] + v[13] * vb[4 + k]) / I - vb[4 + k];
            // rate (gamma, kappa, z_p): grid factor only
            for (int k = 0; k < 3; k++) g[9 + k] = v[19 + k] / I;
        }
        for (int k = 0; k < 12; k++) out[k] = g[k];
    }
}

// ---- MIXED event adjoint on the factorised Gaussian ----
//
// The per-sample sums of the adjoint are sums over grid offsets of the same
// Gaussian as the forward kernel's: with an origin t_o per run of samples,
// u = (z_j - z_o)/(sqrt2 b), ds = dz/(sqrt2 b), B = exp(2 u ds),
//   e_ja = exp(-u^2) B^tau C_tau,  tau = a - t_o,  C_tau = exp(-(ds tau)^2),
//   u_ja = (z_a - z_j)/b = sqrt2 (ds tau - u),
// so that with P_X(B) = sum_tau X_tau C_tau H(a) B^tau
//   S0 = e^{-u^2} P_1,  S1 = sqrt2 e^{-u^2} (ds P_tau - u P_1),
//   S2 = 2 e^{-u^2} (ds^2 P_tau2 - 2 ds u P_tau + u^2 P_1),
// and the galaxy term sum_a e_ja w'_a F dG/dOm is a fourth polynomial.  The
// four are evaluated together by Horner's rule (one FMA per polynomial,
// sample and grid point) from a table of 4 floats per offset, staged by the
// warp in chunks of AM_CH offsets per side, the +m and -m rows side by side.
//
// The grid term, sum_a M(a) Q_k(a) = sum_j pf w_j sum_a e_ja H(a) Q_k(a),
// needs per sample sum_a e_ja H(a) Q_k(a).  Q_k = d ln F / dtheta_k is a
// smooth function of z (Q for H0 is exactly 1/H0); over a window of +-KW32 b
// it is replaced by its second-order Taylor polynomial about the sample's
// grid point a_j, so that
//   sum_a e H Q_k = Q_k S0 + Q_k' m1 + (Q_k''/2) m2,
//   m1 = b S1 + d S0,  m2 = b^2 S2 + 2 d b S1 + d^2 S0,  d = z_j - z_aj,
// with (Q, Q', Q''/2) from a per-grid-point FP32 table (central differences
// of the FP64 table).  The truncation is third order in the window, ~1e-5
// of the term at the benchmark's bandwidths, below the mixed path's FP32
// error budget for the gradient.
//
// Runs hold up to 64 neighbouring samples of one group (one or two per lane)
// whose spread is at most 16 b; beyond 8 b the table is scaled by e^20
// (undone in e^{-u^2}), which keeps every coefficient and intermediate in the
// normal float range.  Kernels narrower than ~0.7 grid steps (ds > 0.5) use
// direct exponentials.  Each lane then takes its samples' own derivative
// terms (dz/dtheta, d ln w/dtheta and Scott's rule) from the run's sums, left
// in the warp's table space.
constexpr int AM_THREADS = ADJ_THREADS, AM_WARPS = AM_THREADS / 32;
constexpr int AM_CH = 64;
constexpr int AM_NP = 4;               // polynomials (table floats per offset)
constexpr int AM_SLOT = 2 * AM_NP / 4;  // float4 per slot: the +m and -m rows
constexpr int AM_SLOTS = AM_CH + 1;     // per warp; slot AM_CH holds tau = 0
constexpr int AM_RUN = 64;              // samples per run
static_assert(AM_NP * AM_RUN <= 4 * AM_SLOT * AM_SLOTS, "run sums fit in the table space");
constexpr int AM_RED = 32;              // floats per warp in the block sums

// Fixed-order FP32 block sum of NV values (NV <= AM_RED); every thread gets
// the totals.  FP32 keeps the reduction off B300's narrow FP64 pipe.
template <int NV>
__device__ void bsumf(float (&v)[NV], float *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        float s = v[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[wid * NV + k] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        float s = 0.f;
        for (int w = 0; w < AM_WARPS; w++) s += red[w * NV + threadIdx.x];
        red[AM_WARPS * NV + threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = red[AM_WARPS * NV + k];
    __syncthreads();
}

// Per-block constants of the sample terms, kept in shared memory (the
// Horner chains need the registers).
struct AdjMixConst {
    MassDer<float> md;
    float cw0, cw1, cw2, cu, Mw, Mu, varw, ib;
    int rule;
};

struct AdjMixLayout {
    int ns_pad, nz_pad, seg_pad;
    __host__ __device__ AdjMixLayout(int max_ns, int nz, int max_seg)
        : ns_pad((max_ns + 3) & ~3), nz_pad((nz + 3) & ~3), seg_pad((max_seg + 4) & ~3) {}
    // float4: table rows; float: block sums, zs, ws, F', segment
    // prefactors; int: segment valid counts, starts and KDE supports
    __host__ __device__ size_t bytes() const {
        return sizeof(float4) * AM_SLOT * (size_t)AM_WARPS * AM_SLOTS +
               sizeof(float) * ((AM_WARPS + 1) * AM_RED + 2 * (size_t)ns_pad + nz_pad + seg_pad) +
               sizeof(int) * 4 * (size_t)seg_pad;
    }
};

__global__ void __launch_bounds__(AM_THREADS, 2) k_event_adj_mixed(DevCatalog c, CallPtrs p, AdjPtrs q, int H) {
    extern __shared__ float4 am4[];
    __shared__ AdjMixConst kc;
    const AdjMixLayout L(c.max_ns, c.n_z, c.max_seg);
    float4 *rows = am4;
    float *red = reinterpret_cast<float *>(rows + AM_SLOT * AM_WARPS * AM_SLOTS);
    float *zs = red + (AM_WARPS + 1) * AM_RED;
    float *ws = zs + L.ns_pad;
    float *Fs = ws + L.ns_pad;  // F' = trapezoid weight x F / F_scale
    float *segpf = Fs + L.nz_pad;
    int *segv = reinterpret_cast<int *>(segpf + L.seg_pad);
    int *seglo = segv + L.seg_pad;
    int *segA0 = seglo + L.seg_pad;
    int *segA1 = segA0 + L.seg_pad;

    const int h = blockIdx.x % H;
    const int4 ei = __ldg(c.ev_info + 2 * (blockIdx.x / H));      // (ev, s0, ns, zoff)
    const int4 ej = __ldg(c.ev_info + 2 * (blockIdx.x / H) + 1);  // (g0, ngroups, sg0, nseg)
    const int ev = ei.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const HP &hp = p.hp[h];
    const HPd &hd = q.hpd[h];
    double *out = q.dlnI + ((size_t)h * c.n_events + ev) * 12;
    if (hp.status & (CHIMERA_PT_OUT_OF_SUPPORT | CHIMERA_PT_NONMONOTONE)) {
        if (tid < 12) out[tid] = 0.0;
        return;
    }
    const int64_t s0 = ei.y;
    const int ns = ei.z;
    const int g0 = ej.x, ngroups = ej.y, sg0 = ej.z, nseg = ej.w;
    const int nz = c.n_z;
    const MixParams mp = mix_params(hp);
    const float4 *inv = p.inv32 + (size_t)h * NU;
    for (int a = tid; a < nz; a += AM_THREADS)
        Fs[a] = ((a == 0 || a == nz - 1) ? 0.5f : 1.f) * p.F32[(size_t)h * nz + a];
    for (int k = tid; k <= nseg; k += AM_THREADS) {
        seglo[k] = (int)(c.seg_soff[sg0 + k] - s0);
        if (k < nseg) segpf[k] = (float)c.seg_pf[sg0 + k];
    }
    // ---- z_j, w_j exactly as the mixed reweighting kernel
    for (int j = tid; j < ns; j += AM_THREADS) {
        float z = CUDART_INF_F, w = 0.f;
        const float4 sv = __ldg(c.s32 + s0 + j);
        const int k = __float_as_int(sv.x);
        if ((k < mp.kv) || (k == mp.kv && sv.y <= mp.fv)) {
            const float zz = chimd::hermite4(__ldg(inv + k), sv.y);
            if (zz < CUDART_INF_F) {
                z = zz;
                const float lz = __log2f(1.f + zz);
                w = mass_weight32(mp, sv.z - lz, sv.w - lz);
            }
        }
        zs[j] = z;
        ws[j] = w;
    }
    __syncthreads();
    // ---- moments (two-pass) for the derivative of Scott's rule
    float m5[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // W1, Wz, W2, n_valid, Sz
    for (int j = tid; j < ns; j += AM_THREADS)
        if (zs[j] < CUDART_INF_F) {
            const float z = zs[j], w = ws[j];
            m5[0] += w; m5[1] += w * z; m5[2] += w * w; m5[3] += 1.f; m5[4] += z;
        }
    bsumf<5>(m5, red);
    const float W1 = m5[0], W2 = m5[2], nv = m5[3];
    const float Mw = W1 > 0.f ? m5[1] / W1 : 0.f, Mu = nv > 0.f ? m5[4] / nv : 0.f;
    float m2v[2] = {0.f, 0.f};
    for (int j = tid; j < ns; j += AM_THREADS)
        if (zs[j] < CUDART_INF_F) {
            const float z = zs[j], w = ws[j];
            m2v[0] += w * (z - Mw) * (z - Mw);
            m2v[1] += (z - Mu) * (z - Mu);
        }
    bsumf<2>(m2v, red);
    const float varw = W1 > 0.f ? m2v[0] / W1 : 0.f, neffw = W1 > 0.f ? W1 * W1 / W2 : 0.f;
    const float varu = nv > 0.f ? m2v[1] / nv : 0.f;
    // 0 weighted, 1 unweighted, 2 grid spacing; the bandwidth itself is the
    // reweighting kernel's FP32 one
    const int rule = (W1 > 0.f && neffw >= 2.f && varw > 0.f) ? 0 : ((nv >= 2.f && varu > 0.f) ? 1 : 2);
    const float b = (float)p.bw[(size_t)h * c.n_events + ev];
    const float dz = c.dz32, inv_dz = 1.f / dz, ib = 1.f / b;
    const float inv_s2b = 0.70710678f / b, ds = dz * inv_s2b, halfk = KW32 * b;
    // ---- segment valid counts and KDE supports (as the forward kernel)
    for (int k = tid; k < nseg; k += AM_THREADS) {
        const int lo = seglo[k], hi = seglo[k + 1];
        int l = lo, r = hi;
        while (l < r) {
            const int m = (l + r) >> 1;
            if (zs[m] < CUDART_INF_F) l = m + 1; else r = m;
        }
        segv[k] = l - lo;
        if (l > lo) {
            segA0[k] = max(0, (int)ceilf((zs[lo] - (float)KDE_MARGIN * b) * inv_dz));
            segA1[k] = min(nz - 1, (int)floorf((zs[l - 1] + (float)KDE_MARGIN * b) * inv_dz));
        } else {
            segA0[k] = 0;
            segA1[k] = -1;
        }
    }
    __syncthreads();

    if (tid == 0) {
        kc.md = mass_der32(hp, hd);
        kc.cw0 = rule == 0 ? 1.f / (W1 * varw) : 0.f;
        kc.cw1 = W1 > 0.f ? 2.f / W1 : 0.f;
        kc.cw2 = W2 > 0.f ? 2.f / W2 : 0.f;
        kc.cu = nv > 0.f && varu > 0.f ? 1.f / (nv * varu) : 0.f;
        kc.Mw = Mw;
        kc.Mu = Mu;
        kc.varw = varw;
        kc.ib = ib;
        kc.rule = rule;
    }
    __syncthreads();
    const float4 *dzn = q.dznode32 + (size_t)h * (NU + 1);
    float A9[9], B4[4], C8[8], db9[9], S2t = 0.f, I0 = 0.f;
    for (int k = 0; k < 9; k++) { A9[k] = 0.f; db9[k] = 0.f; }
    for (int k = 0; k < 4; k++) B4[k] = 0.f;
    for (int k = 0; k < 8; k++) C8[k] = 0.f;
    // one valid sample with its sums Sv = (S0, S1, S2, sum over dG/dOm), H
    // without the segment prefactor; the grid-term sums over Q_k come from
    // S0, S1, S2 and the sample's Taylor row (see the kernel's comment)
    const float iH0 = 1.f / hp.h0_32;
    const float4 *QT4 = reinterpret_cast<const float4 *>(q.QT + (size_t)h * nz * AM_QT);
    auto sample_terms = [&](int j, float pf, const float (&Sv)[AM_NP]) {
        const float S0 = Sv[0], S1 = Sv[1], S2 = Sv[2];
        const float z = zs[j], w = ws[j], a1 = 1.f + z;
        const float4 sv = __ldg(c.s32 + s0 + j);
        float dd[4];
        {
            const int kk = __float_as_int(sv.x);
            const float f = sv.y;
            const float4 n0 = __ldg(dzn + kk), n1 = __ldg(dzn + kk + 1);
            dd[0] = n0.x + f * (n1.x - n0.x);
            dd[1] = n0.y + f * (n1.y - n0.y);
            dd[2] = n0.z + f * (n1.z - n0.z);
            dd[3] = n0.w + f * (n1.w - n0.w);
        }
        float dlw[9];
        {
            const float lz = __log2f(a1);
            float e5[5], ez;
            dlnpm_t<float>(kc.md, ex2(sv.z - lz), ex2(sv.w - lz), a1, e5, &ez);
            for (int k = 0; k < 4; k++) dlw[k] = ez * dd[k];
            for (int k = 0; k < 5; k++) dlw[4 + k] = e5[k];
        }
        if (kc.rule == 0) {
            const float zm = z - kc.Mw;
            const float cw = 0.5f * (zm * zm - kc.varw) * kc.cw0 - 0.2f * (kc.cw1 - w * kc.cw2);
            const float cz = w * zm * kc.cw0;
            for (int k = 0; k < 9; k++) db9[k] += cw * w * dlw[k] + (k < 4 ? cz * dd[k] : 0.f);
        } else if (kc.rule == 1) {
            const float cz = (z - kc.Mu) * kc.cu;
            for (int k = 0; k < 4; k++) db9[k] += cz * dd[k];
        }
        if (w == 0.f) return;
        const float pw = pf * w, pwb = pw * S1 * kc.ib;
        I0 += pw * S0;
        S2t += pw * S2;
        for (int k = 0; k < 9; k++) A9[k] += pw * S0 * dlw[k];
        for (int k = 0; k < 4; k++) B4[k] += pwb * dd[k];
        C8[0] += pw * S0 * iH0;
        {
            // moments of e H about the sample's grid point a_j:
            // m1 = sum e H (z_a - z_aj), m2 = sum e H (z_a - z_aj)^2
            const int aj = min(nz - 1, max(0, (int)rintf(z * inv_dz)));
            const float dl = z - aj * dz, bS1 = b * S1;
            const float m1 = fmaf(dl, S0, bS1), m2 = fmaf(b * b, S2, dl * fmaf(dl, S0, 2.f * bS1));
            const float4 *row = QT4 + (size_t)aj * (AM_QT / 4);
            const float4 r0 = __ldg(row), r1 = __ldg(row + 1), r2 = __ldg(row + 2), r3 = __ldg(row + 3),
                         r4 = __ldg(row + 4);
            const float t[18] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x,
                                 r2.y, r2.z, r2.w, r3.x, r3.y, r3.z, r3.w, r4.x, r4.y};
#pragma unroll
            for (int k = 0; k < 6; k++) C8[1 + k] += pw * fmaf(t[3 * k + 2], m2, fmaf(t[3 * k + 1], m1, t[3 * k] * S0));
        }
        C8[7] += pw * Sv[3];
    };

    float4 *tw = rows + AM_SLOT * wid * AM_SLOTS;  // this warp's table
    float *twf = reinterpret_cast<float *>(tw);
    float *buf = twf;  // a run's per-sample sums [k][idx], after its chains
    const float *prof = reinterpret_cast<const float *>(p.prof[h]);
    const float *dprof = reinterpret_cast<const float *>(q.dprof[h]);  // FP32 on this path
    // groups in a fixed warp assignment (the sums do not depend on timing)
    for (int g = wid; g < ngroups; g += AM_WARPS) {
        const int4 gi = __ldg(c.groups + g0 + g);
        const int sk = gi.z, lo = gi.x;
        const int cnt = min(gi.y, segv[sk] - (lo - seglo[sk]));  // valid samples only
        if (cnt <= 0) continue;
        const float pf = segpf[sk];
        const int64_t row = c.kde_mode == CHIMERA_KDE_MANY_1D ? (int64_t)(sg0 + sk) : (int64_t)ev;
        const float *G = prof + row * nz;
        const float *dG = dprof + row * nz;
        const int s_lo = segA0[sk], s_hi = segA1[sk];
        // narrow kernel: direct exponentials on each sample's window
        auto direct = [&](int st, int n) {
            for (int idx = lane; idx < n; idx += 32) {
                const int j = lo + st + idx;
                const float z = zs[j];
                float Sv[AM_NP];
                for (int k = 0; k < AM_NP; k++) Sv[k] = 0.f;
                if (ws[j] != 0.f) {
                    const int a0 = max(s_lo, (int)ceilf((z - halfk) * inv_dz));
                    const int a1 = min(s_hi, (int)floorf((z + halfk) * inv_dz));
                    for (int a = a0; a <= a1; a++) {
                        const float x = (a * dz - z) * inv_s2b;
                        const float e = __expf(-x * x) * Fs[a];
                        const float eh = e * __ldg(G + a), U = 1.41421356f * x;
                        Sv[0] += eh;
                        Sv[1] += eh * U;
                        Sv[2] += eh * U * U;
                        Sv[3] += e * __ldg(dG + a);
                    }
                }
                for (int k = 0; k < AM_NP; k++) buf[k * AM_RUN + idx] = Sv[k];
            }
        };
        // one run of n samples from st on, R per lane (n <= 32 R)
        auto run = [&](auto Rc, int st, int n) {
            constexpr int R = decltype(Rc)::value;
            const float zlo = zs[lo + st], zhi = zs[lo + st + n - 1];
            const float fA0 = floorf((zlo - halfk) * inv_dz), fA1 = ceilf((zhi + halfk) * inv_dz);
            const int A0 = fA0 < (float)s_lo ? s_lo : (int)fA0;
            const int A1 = fA1 > (float)s_hi ? s_hi : (int)fA1;
            const int t_o = (int)rintf(0.5f * (zlo + zhi) * inv_dz);
            const int T = max(0, max(A1 - t_o, t_o - A0));
            const float lnscale = zhi - zlo > 8.f * b ? 20.f : 0.f;
            const float zo = t_o * dz;
            float u[R], Bf[R], Bb[R];
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int idx = lane + 32 * r;
                u[r] = idx < n ? (zs[lo + st + idx] - zo) * inv_s2b : 0.f;
                Bf[r] = __expf(2.f * u[r] * ds);
                Bb[r] = __expf(-2.f * u[r] * ds);
            }
            // the forward (powers of B) and backward (powers of 1/B) chains of
            // each polynomial run side by side as one float2: one paired
            // FFMA2 per step of both, each element rounded as a scalar fmaf
            float2 m2[R], s2[R][AM_NP];
#pragma unroll
            for (int r = 0; r < R; r++) {
                m2[r] = make_float2(Bf[r], Bb[r]);
#pragma unroll
                for (int k = 0; k < AM_NP; k++) s2[r][k] = make_float2(0.f, 0.f);
            }
            // Horner from the outermost offsets in, AM_CH offsets per side at
            // a time (slot i: the rows of +m and -m, m = mhi - i); the last
            // chunk also stages tau = 0, which closes the forward chain
            for (int mhi = T;; mhi -= AM_CH) {
                const int mlo = max(1, mhi - AM_CH + 1), nr = max(0, mhi - mlo + 1);
                const bool last = mlo <= 1;
                const int nst = 2 * nr + (last ? 1 : 0);
                __syncwarp();
                for (int i = lane; i < nst; i += 32) {
                    int tau;
                    float *dst;
                    if (i < nr) { tau = mhi - i; dst = twf + 4 * AM_SLOT * i; }
                    else if (i < 2 * nr) { tau = -(mhi - (i - nr)); dst = twf + 4 * AM_SLOT * (i - nr) + 1; }
                    else { tau = 0; dst = twf + 4 * AM_SLOT * AM_CH; }
                    const int a = t_o + tau;
                    float2 r0 = make_float2(0.f, 0.f), r1 = r0;
                    if (a >= A0 && a <= A1) {
                        const float x = ds * (float)tau;
                        const float cf = __expf(lnscale - x * x) * Fs[a];
                        const float hh = cf * __ldg(G + a);
                        const float tt = (float)tau;
                        r0 = make_float2(hh, tt * hh);
                        r1 = make_float2(tt * tt * hh, cf * __ldg(dG + a));
                    }
                    if (i < 2 * nr) {
                        // forward and backward coefficients of a polynomial
                        // side by side (the paired chains read them as one float2)
                        dst[0] = r0.x;
                        dst[2] = r0.y;
                        dst[4] = r1.x;
                        dst[6] = r1.y;
                    } else {
                        float2 *d2 = reinterpret_cast<float2 *>(dst);
                        d2[0] = r0;
                        d2[1] = r1;
                    }
                }
                __syncwarp();
#pragma unroll 2
                for (int i = 0; i < nr; i++) {
                    const float4 *sl = tw + AM_SLOT * i;
                    const float4 v0 = sl[0], v1 = sl[1];  // (f0, b0, f1, b1), (f2, b2, f3, b3)
                    const float2 c_[AM_NP] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w),
                                              make_float2(v1.x, v1.y), make_float2(v1.z, v1.w)};
#pragma unroll
                    for (int r = 0; r < R; r++)
#pragma unroll
                        for (int k = 0; k < AM_NP; k++) s2[r][k] = __ffma2_rn(s2[r][k], m2[r], c_[k]);
                }
                if (last) {
                    const float4 v0 = tw[AM_SLOT * AM_CH];
                    const float c0_[AM_NP] = {v0.x, v0.y, v0.z, v0.w};
#pragma unroll
                    for (int r = 0; r < R; r++)
#pragma unroll
                        for (int k = 0; k < AM_NP; k++) s2[r][k].x = fmaf(s2[r][k].x, Bf[r], c0_[k]);
                    break;
                }
            }
            __syncwarp();  // the table space now takes the run's sums
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int idx = lane + 32 * r;
                if (idx >= n) continue;
                const float uu = u[r], E = __expf(-uu * uu - lnscale);
                float P[AM_NP];
#pragma unroll
                for (int k = 0; k < AM_NP; k++) P[k] = E * fmaf(Bb[r], s2[r][k].y, s2[r][k].x);
                buf[idx] = P[0];
                buf[AM_RUN + idx] = 1.41421356f * (ds * P[1] - uu * P[0]);
                buf[2 * AM_RUN + idx] = 2.f * (ds * ds * P[2] - 2.f * ds * uu * P[1] + uu * uu * P[0]);
                buf[3 * AM_RUN + idx] = P[3];
            }
        };
        for (int st = 0; st < cnt;) {
            int n;
            if (ds > 0.5f) {
                n = min(AM_RUN, cnt - st);
                direct(st, n);
            } else {
                // a run: the longest prefix of up to 64 samples spanning <= 16 b
                const float zf = zs[lo + st], lim = 16.f * b;
                const bool p0 = st + lane < cnt && zs[lo + st + lane] - zf <= lim;
                const bool p1 = st + 32 + lane < cnt && zs[lo + st + 32 + lane] - zf <= lim;
                const unsigned b0 = __ballot_sync(0xffffffffu, p0), b1 = __ballot_sync(0xffffffffu, p1);
                n = b0 != 0xffffffffu ? __ffs(~b0) - 1 : 32 + (b1 != 0xffffffffu ? __ffs(~b1) - 1 : 32);
                if (n <= 32) run(std::integral_constant<int, 1>{}, st, n);
                else run(std::integral_constant<int, 2>{}, st, n);
            }
            // each lane reads back the sums it wrote
            for (int idx = lane; idx < n; idx += 32) {
                float Sv[AM_NP];
#pragma unroll
                for (int k = 0; k < AM_NP; k++) Sv[k] = buf[k * AM_RUN + idx];
                sample_terms(lo + st + idx, pf, Sv);
            }
            __syncwarp();
            st += n;
        }
    }
    // ---- block sums (FP32, fixed order) and the 12 derivatives
    float v[32];
    for (int k = 0; k < 9; k++) v[k] = A9[k];
    for (int k = 0; k < 4; k++) v[9 + k] = B4[k];
    v[13] = S2t;
    v[14] = I0;
    for (int k = 0; k < 8; k++) v[15 + k] = C8[k];
    for (int k = 0; k < 9; k++) v[23 + k] = db9[k];  // d ln b / dtheta
    bsumf<32>(v, red);
    if (tid == 0) {
        const double I = v[14];
        const float *vb = v + 23;
        double gr[12];
        for (int k = 0; k < 12; k++) gr[k] = 0.0;
        if (I > 0.0) {
            const double iI = 1.0 / I;
            for (int k = 0; k < 4; k++)
                gr[k] = ((double)v[k] + v[9 + k] + (double)v[13] * vb[k] + v[15 + k]) * iI - vb[k];
            gr[1] += v[22] * iI;
            for (int k = 0; k < 5; k++) gr[4 + k] = ((double)v[4 + k] + (double)v[13] * vb[4 + k]) * iI - vb[4 + k];
            for (int k = 0; k < 3; k++) gr[9 + k] = v[19 + k] * iI;
        }
        for (int k = 0; k < 12; k++) out[k] = gr[k];
    }
}

// Hermite interpolation of dDhat/dOm in FP32 (table values rounded).
__device__ __forceinline__ float dcO_hermite32(const double *fwdO, float z, float Om) {
    const float t = z * float(1.0 / HT);
    int k = (int)floorf(t);
    k = max(0, min(k, NT_FWD - 2));
    const float f = t - k;
    auto g = [Om](float zz) {
        const float a = 1.f + zz, E = sqrtf(Om * a * a * a + 1.f - Om);
        return -0.5f * (a * a * a - 1.f) / (E * E * E);
    };
    const float ht = float(HT);
    const float m0 = ht * g(k * ht), m1 = ht * g((k + 1) * ht);
    const float f2 = f * f, f3 = f2 * f;
    return (2.f * f3 - 3.f * f2 + 1.f) * float(fwdO[k]) + (f3 - 2.f * f2 + f) * m0 +
           (-2.f * f3 + 3.f * f2) * float(fwdO[k + 1]) + (f3 - f2) * m1;
}

// Selection adjoint: per block, sum_j s_j dln s_j / dtheta (12) and sum_j s_j,
// with dln s/dz chained through z_j for the cosmological parameters.  FP64
// recomputes s_j as the FP64 selection kernel does; MIXED in float from the
// mixed kernel's z_j (D_c from the measured distance, D_c = d_L/((1+z) Xi)).
template <bool F64>
__global__ void __launch_bounds__(ADJ_THREADS, F64 ? 1 : 4) k_select_adj(DevCatalog c, CallPtrs p, AdjPtrs q, int H) {
    using T = typename std::conditional<F64, double, float>::type;
    __shared__ double red[(ADJ_THREADS / 32 + 1) * 13];
    const int h = blockIdx.y, chunk = blockIdx.x;
    const HP &hp = p.hp[h];
    const HPd &hd = q.hpd[h];
    const double *th = hp.th;
    T acc[13];
    for (int k = 0; k < 13; k++) acc[k] = T(0);
    const MixParams mp = mix_params(hp);
    const MassDer<double> md64 = mass_der64(hp, hd, c.beta);
    const MassDer<float> md32 = mass_der32(hp, hd);
    const int64_t base = (int64_t)chunk * SEL_CHUNK;
    const T one = T(1);
    for (int qq = 0; qq < SEL_PER_THREAD; qq++) {
        int64_t j = base + qq * ADJ_THREADS + threadIdx.x;
        if (j >= c.n_det) break;
        T z, m1, m2, s;
        ZDerT<T> r;
        T d5[5], dwz;
        if constexpr (F64) {
            double zz;
            if (!invert64(c, p, h, hp, c.id64[j], &zz)) continue;
            if (!(zz <= c.z_max)) continue;
            const double a1 = 1.0 + zz;
            const double dm1 = c.im1_64[j] / a1, dm2 = c.im2_64[j] / a1;
            const double mmin = th[7], mmax = th[8];
            if (!(dm1 >= mmin && dm1 <= mmax && dm2 >= mmin && dm2 <= dm1) || !(dm1 > mmin)) continue;
            const double x = (dm1 - th[5]) / th[6];
            const double p1 = hp.c_pl * pow(dm1, -th[4]) + hp.c_g * exp(-0.5 * x * x);
            const double p2 = fabs(hp.b1) < 1e-12 ? 1.0 / (dm2 * log(dm1 / mmin))
                                                  : hp.b1 * pow(dm2, c.beta) / (pow(dm1, hp.b1) - hp.mmin_b1);
            const double Dc = hp.cH * chimd::dc_hermite(p.fwd[h], zz, th[1]);
            double dd, J;
            chimd::dgw_J(zz, Dc, th, hp.cH, &dd, &J);
            const double E = chimd::E_of(zz, th[1]);
            const double pz = 3.0 * hp.cH * Dc * Dc / E / (hp.dc_zmax * hp.dc_zmax * hp.dc_zmax);
            s = T(p1 * p2 * chimd::psi_of(zz, th) * pz / (a1 * a1 * a1 * fabs(J) * exp(c.ilp64[j])));
            const ZDer r64 = zder(zz, th, p.fwd[h], q.fwdO[h], hd.dlpz_zmax);
            r = r64;
            double e5[5], ez;
            dlnpm_t<double>(md64, dm1, dm2, a1, e5, &ez);
            for (int k = 0; k < 5; k++) d5[k] = T(e5[k]);
            dwz = T(ez);
            z = T(zz); m1 = T(dm1); m2 = T(dm2);
        } else {
            const float4 a4 = c.i32a[j];
            const int k = __float_as_int(a4.x);
            if (!((k < mp.kv) || (k == mp.kv && a4.y <= mp.fv))) continue;
            const float zz = chimd::hermite4(p.inv32[(size_t)h * NU + k], a4.y);
            if (!(zz <= c.z_max32)) continue;
            const float a1 = 1.f + zz, lz = __logf(a1);
            const float lz2 = lz * 1.44269504088896340736f;
            const float l1 = a4.z - lz2, l2 = a4.w - lz2;  // log2 of the source masses
            const float fm1 = ex2(l1), fm2 = ex2(l2);
            const float mmin = hp.mmin32, mmax = hp.mmax32;
            if (!(fm1 >= mmin && fm1 <= mmax && fm2 >= mmin && fm2 <= fm1) || !(fm1 > mmin)) continue;
            const float x = (fm1 - hp.mu32) * hp.inv_sg32;
            const float p1 = hp.c_pl32 * ex2(-hp.alpha32 * l1) + hp.c_g32 * __expf(-0.5f * x * x);
            const float p2 = fabsf(hp.b1_32) < 1e-6f ? __fdividef(1.f, fm2 * __logf(fm1 / mmin))
                                                    : __fdividef(hp.b1_32 * ex2(hp.beta32 * l2), ex2(hp.b1_32 * l1) - hp.mmin_b1_32);
            const float fn = hp.n32, fxi0 = hp.xi0_32, pwz = ex2(-fn * lz2);
            const float xi = fxi0 + (1.f - fxi0) * pwz, dxi = -fn * (1.f - fxi0) * pwz / a1;
            const float Dc = c.i32b[j].x / (a1 * xi);
            const float fom = hp.om32, E = sqrtf(fom * a1 * a1 * a1 + 1.f - fom);
            const float fcH = hp.cH32;
            const float J = (Dc + a1 * fcH / E) * xi + a1 * Dc * dxi;
            const float pz = 3.f * fcH * Dc * Dc / E * hp.inv_dc3_32;
            const float psi = __fdividef(__expf(hp.gam32 * lz), 1.f + __expf((hp.gam32 + hp.kap32) * (lz - hp.l1zp32)));
            s = T(__fdividef(p1 * p2 * psi * pz, a1 * a1 * a1 * fabsf(J) * __expf(c.i32b[j].y)));
            const float DhO = dcO_hermite32(q.fwdO[h], zz, fom);
            const ZDerT<float> r32 = zder_t<float>(zz, hp.h0_32, fom, fxi0, fn, Dc / fcH, DhO, hd.dlpz_zmax32);
            r = r32;
            float e5[5], ez;
            dlnpm_t<float>(md32, fm1, fm2, a1, e5, &ez);
            for (int kk = 0; kk < 5; kk++) d5[kk] = T(e5[kk]);
            dwz = T(ez);
            z = T(zz); m1 = T(fm1); m2 = T(fm2);
        }
        (void)m1; (void)m2;
        T g3[3], dpsiz;
        if constexpr (F64) dlnpsi_t<T>(z, th[9], th[10], th[11], g3, &dpsiz);
        else dlnpsi_t<T>(z, hp.gam32, hp.kap32, hp.zp32, g3, &dpsiz);
        const T dls_dz = dwz + dpsiz + r.dlnpz_dz - T(3) / (one + z) - r.dlnJ_dz;
        T g[12];
        g[0] = -r.dlnJ[0];
        g[1] = r.dlnpz_dOm - r.dlnJ[1];
        g[2] = -r.dlnJ[2];
        g[3] = -r.dlnJ[3];
        for (int k = 0; k < 4; k++) g[k] += dls_dz * r.dz[k];
        for (int k = 0; k < 5; k++) g[4 + k] = d5[k];
        for (int k = 0; k < 3; k++) g[9 + k] = g3[k];
        for (int k = 0; k < 12; k++) acc[k] += s * g[k];
        acc[12] += s;
    }
    // block partial sums: FP64 on the FP64 path, a fixed-order FP32 tree on
    // the mixed path (off the narrow FP64 pipe); the chunks are added in
    // FP64 by the combine kernel
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T *redT = reinterpret_cast<T *>(red);
    for (int k = 0; k < 13; k++) {
        T v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) redT[wid * 13 + k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 13) {
        T v = T(0);
        for (int w = 0; w < ADJ_THREADS / 32; w++) v += redT[w * 13 + threadIdx.x];
        q.selg[((size_t)h * p.n_chunk + chunk) * 13 + threadIdx.x] = double(v);
    }
}

// grad[h] = sum_i d ln I_i - N_obs (sum_j s_j dln s_j) / (sum_j s_j); zero
// for a point whose ln L is -inf.  Fixed-order sums (deterministic).
__global__ void __launch_bounds__(ADJ_THREADS) k_combine_adj(DevCatalog c, CallPtrs p, AdjPtrs q, int H) {
    __shared__ double red[(ADJ_THREADS / 32 + 1) * 25];
    const int h = blockIdx.x;
    double v[25];
    for (int k = 0; k < 25; k++) v[k] = 0.0;
    for (int i = threadIdx.x; i < c.n_events; i += ADJ_THREADS) {
        const double *d = q.dlnI + ((size_t)h * c.n_events + i) * 12;
        for (int k = 0; k < 12; k++) v[k] += d[k];
    }
    for (int ch = threadIdx.x; ch < p.n_chunk; ch += ADJ_THREADS) {
        const double *d = q.selg + ((size_t)h * p.n_chunk + ch) * 13;
        for (int k = 0; k < 13; k++) v[12 + k] += d[k];
    }
    bsum<25>(v, red);
    if (threadIdx.x < 12) {
        const int k = threadIdx.x;
        const double S = v[24];
        const bool bad = !isfinite(p.lnL[h]) || !(S > 0.0);
        q.grad[(size_t)h * 12 + k] = bad ? 0.0 : v[k] - (double)c.n_events * v[12 + k] / S;
    }
}

// dV_c/dz (as D^2/E) and its Om derivative on the grid, for one Om.
__global__ void k_dv_pair(const double *fwd, const double *fwdO, double Om, double dz, int nz, double *dv,
                          double *dvO, float *dv32, float *dvO32) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nz) return;
    chimd::dv_pair(fwd, fwdO, a * dz, Om, dv[a], dvO[a]);
    dv32[a] = (float)dv[a];
    dvO32[a] = (float)dvO[a];
}

// Single-1D, mixed: sum_k S_k dG_k/dOm per event in FP32.
__global__ void k_dprofile_sum32(DevCatalog c, const float *G, float *outh) {
    const int ev = blockIdx.x, nz = c.n_z;
    const int64_t p0 = c.ev_poff[ev], p1 = c.ev_poff[ev + 1];
    for (int a = threadIdx.x; a < nz; a += blockDim.x) {
        float s = 0.f;
        for (int64_t p = p0; p < p1; p++) s += (float)c.pix_S[p] * G[p * nz + a];
        outh[(int64_t)ev * nz + a] = s;
    }
}

// Single-1D: sum_k S_k dG_k/dOm per event.
__global__ void k_dprofile_sum(DevCatalog c, const double *G, double *outh) {
    const int ev = blockIdx.x, nz = c.n_z;
    const int64_t p0 = c.ev_poff[ev], p1 = c.ev_poff[ev + 1];
    for (int a = threadIdx.x; a < nz; a += blockDim.x) {
        double s = 0.0;
        for (int64_t p = p0; p < p1; p++) s += c.pix_S[p] * G[p * nz + a];
        outh[(int64_t)ev * nz + a] = s;
    }
}

}  // namespace

size_t adjoint_event_smem(const DevCatalog &c, bool fp64) {
    if (!fp64) return AdjMixLayout(c.max_ns, c.n_z, c.max_seg).bytes();
    return sizeof(double) * 2 * (size_t)c.max_ns + sizeof(int) * 3 * (size_t)((c.max_seg + 2) & ~1) +
           sizeof(double) * (ADJ_THREADS / 32 + 1) * 28;
}

void launch_adjoint(const DevCatalog &c, const CallPtrs &p, const AdjPtrs &q, int H, bool fp64, cudaStream_t st) {
    k_adj_tables<<<dim3(H, 8), ADJ_THREADS, 0, st>>>(c, p, q);
    if (!fp64) {
        const int64_t n = (int64_t)H * c.n_z;
        k_q_taylor<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c, q, H);
    }
    const size_t smem = adjoint_event_smem(c, fp64);
    const unsigned nb = (unsigned)((int64_t)c.n_events * H);
    if (fp64) {
        cudaFuncSetAttribute(k_event_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (nb) k_event_adj<<<nb, ADJ_THREADS, smem, st>>>(c, p, q, H);
        if (p.n_chunk) k_select_adj<true><<<dim3(p.n_chunk, H), ADJ_THREADS, 0, st>>>(c, p, q, H);
    } else {
        cudaFuncSetAttribute(k_event_adj_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (nb) k_event_adj_mixed<<<nb, AM_THREADS, smem, st>>>(c, p, q, H);
        if (p.n_chunk) k_select_adj<false><<<dim3(p.n_chunk, H), ADJ_THREADS, 0, st>>>(c, p, q, H);
    }
    k_combine_adj<<<H, ADJ_THREADS, 0, st>>>(c, p, q, H);
}

#define CK(call)                                               \
    do {                                                       \
        int rc_ = cuda_check((call), #call);                   \
        if (rc_) return rc_;                                   \
    } while (0)
#define RC(call)                                               \
    do {                                                       \
        int rc_ = (call);                                      \
        if (rc_) return rc_;                                   \
    } while (0)

namespace {

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Layout of the adjoint scratch for H points of catalog c.
struct AdjLayout {
    size_t o_ptrs, o_hpd, o_dzn, o_dzn32, o_Q, o_QT, o_dlnI, o_selg, total;
    AdjLayout(const DevCatalog &c, int H, int nchunk) {
        size_t o = 0;
        auto take = [&](size_t b) { size_t r = o; o += al256(b); return r; };
        o_ptrs = take(2 * sizeof(void *) * (size_t)H);
        o_hpd = take(sizeof(HPd) * (size_t)H);
        o_dzn = take(sizeof(double) * 4 * (size_t)H * (NU + 1));
        o_dzn32 = take(sizeof(float4) * (size_t)H * (NU + 1));
        o_Q = take(sizeof(double) * 7 * (size_t)H * c.n_z);
        o_QT = take(sizeof(float) * AM_QT * (size_t)H * c.n_z);
        o_dlnI = take(sizeof(double) * 12 * (size_t)H * c.n_events);
        o_selg = take(sizeof(double) * 13 * (size_t)H * std::max(nchunk, 1));
        total = o;
    }
};

// A mixed dG/dOm profile allocated but still to be computed (batched).
struct PendingDprof {
    double Om;
    const double *fwd, *fwdO;
    std::pair<uint64_t, int> key;
};

// The one-Om dG/dOm kernels into entry e.
// (v: the context's profile scratch, acquired by the caller)
int dprofile_one(Workspace &ws, const ProfView &v, const DevCatalog &c, double Om, bool f64, const double *fwd,
                 const double *fwdO, ProfEntry &e) {
    double *dv = v.adv, *dvO = v.advO, *invZ = v.ainvZ, *ZO = v.aZO;
    float *dv32 = reinterpret_cast<float *>(dv + c.n_z), *dvO32 = reinterpret_cast<float *>(dvO + c.n_z);
    k_dv_pair<<<(c.n_z + 63) / 64, 64, 0, ws.st>>>(fwd, fwdO, Om, c.dz, c.n_z, dv, dvO, dv32, dvO32);
    launch_galaxy_dOm(c, fwd, fwdO, Om, dv, dvO, dv32, dvO32, f64, invZ, ZO, e.G, ws.st);
    return CHIMERA_OK;
}

// Sky sums (single-1D) and the ready event of a computed entry.
int dprofile_finish(Workspace &ws, const DevCatalog &c, bool f64, ProfEntry &e) {
    if (e.Gh) {
        if (f64) k_dprofile_sum<<<c.n_events, 256, 0, ws.st>>>(c, (const double *)e.G, (double *)e.Gh);
        else k_dprofile_sum32<<<c.n_events, 256, 0, ws.st>>>(c, (const float *)e.G, (float *)e.Gh);
    }
    CK(cudaGetLastError());
    CK(cudaEventRecord(e.ready, ws.st));
    return CHIMERA_OK;
}

// dG/dOm profile for (Om, precision), cached with the forward profiles
// (FP64 rows for FP64 calls, FP32 rows for mixed ones).  With `defer`, a new
// mixed profile is only allocated and queued for flush_dprofiles.
int dprofile(Ctx &ctx, Catalog &cat, Workspace &ws, double Om, bool f64, const double *fwd,
             const double *fwdO, const double **out, std::vector<PendingDprof> *defer) {
    const int kind = f64 ? 2 : 3;
    auto key = std::make_pair(bits_of(Om), kind);
    auto it = cat.prof.find(key);
    const DevCatalog &c = cat.d;
    if (it == cat.prof.end()) {
        ProfEntry e;
        const size_t per = f64 ? sizeof(double) : sizeof(float);
        e.bytes = per * (size_t)c.n_pix * c.n_z;
        const size_t hb = c.kde_mode == CHIMERA_KDE_SINGLE_1D ? per * (size_t)c.n_events * c.n_z : 0;
        evict_profiles(ctx, cat, e.bytes + hb);
        RC(cache_alloc(ctx, &e.G, e.bytes, ws.st));
        if (hb) {
            int rc = cache_alloc(ctx, &e.Gh, hb, ws.st);
            if (rc) { cache_free(ctx, e.G, e.bytes); return rc; }
            e.hbytes = hb;
        }
        if (cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming) != cudaSuccess) {
            free_prof_entry(ctx, e);
            return cuda_check(cudaGetLastError(), "cudaEventCreate");
        }
        if (defer && !f64) {
            it = cat.prof.emplace(key, e).first;
            defer->push_back({Om, fwd, fwdO, key});
        } else {
            ProfView v;
            if (int rc = prof_scratch_acquire(ctx, c, ws.st, &v)) {
                free_prof_entry(ctx, e);
                return rc;
            }
            RC(dprofile_one(ws, v, c, Om, f64, fwd, fwdO, e));
            RC(dprofile_finish(ws, c, f64, e));
            RC(prof_scratch_release(ctx, ws.st));
            it = cat.prof.emplace(key, e).first;
        }
    } else {
        CK(cudaStreamWaitEvent(ws.st, it->second.ready, 0));
    }
    it->second.last_use = ctx.tick;
    // FP32 rows on the mixed path (the pointer table is typed double*)
    *out = reinterpret_cast<const double *>(c.kde_mode == CHIMERA_KDE_SINGLE_1D ? it->second.Gh : it->second.G);
    return CHIMERA_OK;
}

// Launch the pending mixed dG/dOm profiles, PROF_MB Om values per batched
// pass (one alone takes the one-Om kernels; both give the same values).
int flush_dprofiles(Ctx &ctx, Catalog &cat, Workspace &ws, std::vector<PendingDprof> &pend) {
    const DevCatalog &c = cat.d;
    if (pend.empty()) return CHIMERA_OK;
    ProfView v;
    RC(prof_scratch_acquire(ctx, c, ws.st, &v));
    for (size_t b = 0; b < pend.size(); b += PROF_MB) {
        const int n = (int)std::min<size_t>(PROF_MB, pend.size() - b);
        if (n == 1) {
            const PendingDprof &q = pend[b];
            RC(dprofile_one(ws, v, c, q.Om, false, q.fwd, q.fwdO, cat.prof.at(q.key)));
        } else {
            MultiOm m{};
            m.n = n;
            for (int j = 0; j < PROF_MB; j++) {
                const PendingDprof &q = pend[b + (j < n ? j : 0)];
                m.fwd[j] = q.fwd;
                m.fwdO[j] = q.fwdO;
                m.Om[j] = q.Om;
                m.out[j] = j < n ? (float *)cat.prof.at(q.key).G : nullptr;
            }
            launch_galaxy_profile_multi(c, m, true, v.dvm, v.invZm, ws.st);
        }
        for (int j = 0; j < n; j++) RC(dprofile_finish(ws, c, false, cat.prof.at(pend[b + j].key)));
    }
    pend.clear();
    return prof_scratch_release(ctx, ws.st);
}

void drop_dpending(Ctx &ctx, Catalog &cat, Workspace &ws, std::vector<PendingDprof> &pend) {
    cudaStreamSynchronize(ws.st);  // nothing may still write the entries freed below
    for (auto &q : pend) {
        auto it = cat.prof.find(q.key);
        if (it == cat.prof.end()) continue;
        free_prof_entry(ctx, it->second);
        cat.prof.erase(it);
    }
    pend.clear();
}

}  // namespace

void adjoint_release(Ctx &ctx, Workspace &ws) {
    if (ws.gscr) dev_free(ctx, ws.gscr, ws.gscr_bytes);
    ws.gscr = nullptr;
    ws.gscr_bytes = 0;
    if (ws.ahstage) cudaFreeHost(ws.ahstage);
    ws.ahstage = nullptr;
    ws.ahstage_bytes = 0;
}

int backward(Ctx &ctx, Catalog &cat, Workspace &ws, int H, int precision) {
    const DevCatalog &c = cat.d;
    const bool f64 = precision == CHIMERA_FP64;
    const int nchunk = selection_chunks(c);
    AdjLayout L(c, H, nchunk);
    if (ws.gscr_bytes < L.total) {
        if (ws.st) CK(cudaStreamSynchronize(ws.st));
        if (ws.gscr) dev_free(ctx, ws.gscr, ws.gscr_bytes);
        ws.gscr = nullptr;
        ws.gscr_bytes = 0;
        RC(dev_alloc(ctx, (void **)&ws.gscr, L.total));
        ws.gscr_bytes = L.total;
    }
    const size_t hb = 2 * sizeof(void *) * (size_t)H;
    if (ws.ahstage_bytes < hb) {
        if (ws.st) CK(cudaStreamSynchronize(ws.st));
        if (ws.ahstage) cudaFreeHost(ws.ahstage);
        ws.ahstage = nullptr;
        ws.ahstage_bytes = 0;
        if (cudaMallocHost(&ws.ahstage, hb) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMallocHost failed for the adjoint staging buffer");
            return CHIMERA_ERR_CUDA;
        }
        ws.ahstage_bytes = hb;
    }
    if (ws.trace) CK(cudaEventRecord(ws.tev[6], ws.st));
    // the sanitised theta and the forward-table pointers forward() staged
    const double *th = reinterpret_cast<const double *>(ws.hstage);
    const double *const *fw =
        reinterpret_cast<const double *const *>(ws.hstage + sizeof(double) * 12 * H + 8 * (size_t)H);
    const double **hO = reinterpret_cast<const double **>(ws.ahstage);
    const double **hP = hO + H;
    // distinct Om values: their dD/dOm tables (batched), then their dG/dOm
    // profiles (new mixed ones batched)
    std::map<uint64_t, int> slot;
    std::vector<double> oms;
    std::vector<const double *> fws;
    for (int h = 0; h < H; h++) {
        const double Om = th[12 * h + 1];
        if (slot.emplace(bits_of(Om), (int)oms.size()).second) {
            oms.push_back(Om);
            fws.push_back(fw[h]);
        }
    }
    std::vector<const double *> fOs(oms.size()), dGs(oms.size());
    RC(fwd_tables(ctx, oms.data(), (int)oms.size(), ws.st, fOs.data(), true));
    std::vector<PendingDprof> pend;
    for (size_t i = 0; i < oms.size(); i++) {
        int rc = dprofile(ctx, cat, ws, oms[i], f64, fws[i], fOs[i], &dGs[i], &pend);
        if (rc != CHIMERA_OK) {
            drop_dpending(ctx, cat, ws, pend);
            return rc;
        }
    }
    if (int rc = flush_dprofiles(ctx, cat, ws, pend)) {
        drop_dpending(ctx, cat, ws, pend);
        return rc;
    }
    for (int h = 0; h < H; h++) {
        const int i = slot.at(bits_of(th[12 * h + 1]));
        hO[h] = fOs[i];
        hP[h] = dGs[i];
    }
    CK(cudaMemcpyAsync(ws.gscr + L.o_ptrs, ws.ahstage, hb, cudaMemcpyHostToDevice, ws.st));
    AdjPtrs q;
    q.fwdO = reinterpret_cast<const double *const *>(ws.gscr + L.o_ptrs);
    q.dprof = q.fwdO + H;
    q.hpd = reinterpret_cast<HPd *>(ws.gscr + L.o_hpd);
    q.dznode = reinterpret_cast<double *>(ws.gscr + L.o_dzn);
    q.dznode32 = reinterpret_cast<float4 *>(ws.gscr + L.o_dzn32);
    q.Q = reinterpret_cast<double *>(ws.gscr + L.o_Q);
    q.QT = reinterpret_cast<float *>(ws.gscr + L.o_QT);
    q.dlnI = reinterpret_cast<double *>(ws.gscr + L.o_dlnI);
    q.selg = reinterpret_cast<double *>(ws.gscr + L.o_selg);
    q.grad = ws.grad;
    CallPtrs p = ws.ptrs(H, c);
    launch_adjoint(c, p, q, H, f64, ws.st);
    CK(cudaGetLastError());
    if (ws.trace) {
        CK(cudaEventRecord(ws.tev[7], ws.st));
        ws.traced_adjoint = true;
    }
    return CHIMERA_OK;
}

}  // namespace chim
