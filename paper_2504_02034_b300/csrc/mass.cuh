// Per-sample reweighting helpers shared by the forward and adjoint kernels:
// the mass-model weight p(m1) p(m2 | m1) (Sec. 3.1) in FP32 and FP64, and the
// FP64 d_L -> z inversion.  Internal to libchimera.
#pragma once

#include <math_constants.h>

#include "internal.cuh"

namespace chim {

struct MixParams {
    float c_pl, c_g, alpha, mu, inv_sg, mmin, mmax, beta, b1, mmin_b1, lmmin;
    int kv;
    float fv;
};

// Mass-model weight p(m1) p(m2|m1) from log source-frame masses, with the
// SFU exponential (relative error ~1e-6, independent between samples).
inline __device__ float mass_weight32(const MixParams &q, float lm1, float lm2) {
    float m1 = __expf(lm1), m2 = __expf(lm2);
    if (!(m1 >= q.mmin && m1 <= q.mmax && m2 >= q.mmin && m2 <= m1)) return 0.f;
    float x = (m1 - q.mu) * q.inv_sg;
    float p1 = q.c_pl * __expf(-q.alpha * lm1) + q.c_g * __expf(-0.5f * x * x);
    float p2;
    if (fabsf(q.b1) < 1e-6f) {
        float l = lm1 - q.lmmin;
        p2 = l > 0.f ? __fdividef(1.f, m2 * l) : 0.f;
    } else {
        float den = m1 * __expf(q.beta * lm1) - q.mmin_b1;
        p2 = den > 0.f ? __fdividef(q.b1 * __expf(q.beta * lm2), den) : 0.f;
    }
    return p1 * p2;
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
    const double *fwd = p.fwd[h];
    for (int it = 0; it < 2; it++) {
        double dd, J;
        chimd::dgw_J(z, hp.cH * chimd::dc_hermite(fwd, z, hp.th[1]), hp.th, hp.cH, &dd, &J);
        double step = (dd - d) / J;
        if (isfinite(step)) z -= step;
    }
    *zout = z;
    return true;
}


}  // namespace chim
