// Per-sample reweighting helpers shared by the forward and adjoint kernels:
// the mass-model weight p(m1) p(m2 | m1) (Sec. 3.1) in FP32 and FP64, and the
// FP64 d_L -> z inversion.  Internal to libchimera.
#pragma once

#include <math_constants.h>

#include "internal.cuh"

namespace chim {

// 2^x by the SFU (PTX ex2.approx.ftz: relative error ~2^-22, 0 for very
// negative x).
inline __device__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// FP32 mass-model constants of one hyperpoint, in the log2 domain: the
// weight is built from exp2 / log2 of the SFU (relative error ~1e-6 per
// sample, independent between samples).
struct MixParams {
    float c_pl, c_g, mu, inv_sg, mmin_b1, b1;
    float na2;     // -alpha             (m1^-alpha   = 2^(na2 l1))
    float gk;      // -log2(e)/2 / sg^2 folded with (m1 - mu): 2^(gk x^2), x = m1 - mu
    float beta;    //                     (m2^beta    = 2^(beta l2))
    float l2min, l2max;
    float inv_lmin_ln2;  // beta = -1 form: 1 / ln 2
    bool logp2;    // beta == -1: p(m2|m1) = 1 / (m2 ln(m1 / m_min))
    int kv;
    float fv;
};

inline __device__ MixParams mix_params(const HP &hp) {
    MixParams q;
    q.c_pl = hp.c_pl32;
    q.c_g = hp.c_g32;
    q.mu = hp.mu32;
    q.inv_sg = hp.inv_sg32;
    q.mmin_b1 = hp.mmin_b1_32;
    q.b1 = hp.b1_32;
    q.na2 = -hp.alpha32;
    q.gk = -0.72134752044448170368f * hp.inv_sg32 * hp.inv_sg32;
    q.beta = hp.beta32;
    q.l2min = hp.l2min32;
    q.l2max = hp.l2max32;
    q.inv_lmin_ln2 = 1.44269504088896340736f;
    q.logp2 = fabsf(hp.b1_32) < 1e-6f;
    q.kv = hp.k_valid;
    q.fv = hp.f_valid;
    return q;
}

// Mass-model weight p(m1) p(m2|m1) (Sec. 3.1) from log2 source-frame masses
// l1 = log2 m1, l2 = log2 m2; zero outside m_min <= m2 <= m1 <= m_max.
// Branch-free apart from the hyperpoint-uniform beta = -1 form.
inline __device__ float mass_weight32(const MixParams &q, float l1, float l2) {
    const float m1 = ex2(l1);
    const float x = m1 - q.mu;
    const float p1 = q.c_pl * ex2(q.na2 * l1) + q.c_g * ex2(q.gk * x * x);
    float p2;
    if (q.logp2) {
        const float m2 = ex2(l2);
        const float l = l1 - q.l2min;
        p2 = l > 0.f ? __fdividef(q.inv_lmin_ln2, m2 * l) : 0.f;
    } else {
        const float den = ex2(q.b1 * l1) - q.mmin_b1;
        p2 = den > 0.f ? __fdividef(q.b1 * ex2(q.beta * l2), den) : 0.f;
    }
    const bool in = (l2 >= q.l2min) & (l2 <= l1) & (l1 <= q.l2max);
    return in ? p1 * p2 : 0.f;
}

inline __device__ double mass_weight64(const HP &hp, double beta, double m1, double m2) {
    const double mmin = hp.th[7], mmax = hp.th[8];
    if (!(m1 >= mmin && m1 <= mmax && m2 >= mmin && m2 <= m1) || !(m1 > mmin)) return 0.0;
    double x = (m1 - hp.th[5]) / hp.th[6];
    double p1 = hp.c_pl * pow(m1, -hp.th[4]) + hp.c_g * exp(-0.5 * x * x);
    double p2;
    if (fabs(hp.b1) < 1e-12) p2 = 1.0 / (m2 * log(m1 / mmin));
    else p2 = hp.b1 * pow(m2, beta) / (pow(m1, hp.b1) - hp.mmin_b1);
    return p1 * p2;
}

// d_L -> z in FP64: Hermite in u on the inverse table, then Newton on the
// forward relation.  Returns false when d is beyond d_L^gw(10).
inline __device__ bool invert64(const DevCatalog &c, const CallPtrs &p, int h, const HP &hp, double d,
                         double *zout) {
    if (!(d > 0.0) || !(d <= hp.d_valid)) return false;
    double t = sqrt(d / c.d_top) * NU;
    int k = (int)t;
    if (k > NU - 1) k = NU - 1;
    double f = t - k;
    const double2 *nd = p.inv64 + (size_t)h * (NU + 1);
    double2 a = nd[k], b = nd[k + 1];
    double f2 = f * f, f3 = f2 * f;
    double z = (2 * f3 - 3 * f2 + 1) * a.x + (f3 - 2 * f2 + f) * a.y / NU + (-2 * f3 + 3 * f2) * b.x +
               (f3 - f2) * b.y / NU;
    if (!isfinite(z)) return false;
    // one Newton step: the Hermite seed on the FP64 node pairs is already
    // good to ~1e-14, and the step brings it to the forward relation's root
    const double *fwd = p.fwd[h];
    double dd, J;
    chimd::dgw_J(z, hp.cH * chimd::dc_hermite(fwd, z, hp.th[1]), hp.th, hp.cH, &dd, &J);
    const double step = (dd - d) / J;
    if (isfinite(step)) z -= step;
    *zout = z;
    return true;
}


}  // namespace chim
