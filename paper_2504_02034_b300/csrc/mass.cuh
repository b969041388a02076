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

// ---- FP32 arithmetic without a shared error ------------------------------
// The mixed path adds millions of FP32 terms.  Rounding errors that differ
// from term to term average out in such a sum; an error that every term
// shares (a constant rounded to float, an SFU approximation with a non-zero
// mean error over its inputs) does not, and it shifts every event integral
// and the selection term by the same relative amount.  These helpers keep
// the shared part far below the FP32 resolution.

// c x, with c carried to ~48 bits (a single rounding of the result).
inline __device__ float mul_f2(F2 c, float x) { return fmaf(c.hi, x, c.lo * x); }
// log2(e) as a float pair: the FP32 rounding of log2(e) alone would give
// e^x a relative error of 1.3e-8 |x| of one sign.
constexpr float L2E_HI = 1.44269502162933349609375f;
constexpr float L2E_LO = 1.925963033500011e-8f;

// 2^(t + r), |r| << 1: the integer part of t is split off exactly and the
// SFU ex2 sees only the fraction in [-0.5, 0.5]; the integer part goes into
// the exponent field.  Measured on B300, ex2.approx has a mean relative
// error of -5.1e-8 for every negative argument interval [n, n+1) and +3.3e-8
// for every positive one, so an argument of fixed sign (a power law) would
// give all terms the same error, while fractions of both signs bring it to
// about -8e-9.  ex2_pair_n assumes |t| < 120 (no range test), ex2_pair
// handles any t.
// The integer part comes from adding 1.5 * 2^23 (round to nearest into the
// low mantissa bits) rather than a float-to-int conversion, which measured
// as a large share of the FP64 pipe's time on B300.
constexpr float RND_MAGIC = 12582912.f;  // 1.5 * 2^23
constexpr int RND_MAGIC_BITS = 0x4B400000;
inline __device__ float ex2_pair_n(float t, float r) {
    const float big = t + RND_MAGIC;
    const float n = big - RND_MAGIC;  // rint(t)
    const float y = ex2((t - n) + r);  // t - n is exact
    return __int_as_float(__float_as_int(y) + ((__float_as_int(big) - RND_MAGIC_BITS) << 23));
}
inline __device__ float ex2_pair(float t, float r) {
    return fabsf(t) < 120.f ? ex2_pair_n(t, r) : ex2(t + r);
}
inline __device__ float ex2c(float x) { return ex2_pair(x, 0.f); }
// 2^(c x) for a constant c: the product's rounding error is kept (an FMA
// gives it exactly) and the constant's low part is added; _n: |c x| < 120.
inline __device__ float ex2_mul_n(F2 c, float x) {
    const float t = c.hi * x;
    return ex2_pair_n(t, fmaf(c.hi, x, -t) + c.lo * x);
}
inline __device__ float ex2_mul(F2 c, float x) {
    const float t = c.hi * x;
    return ex2_pair(t, fmaf(c.hi, x, -t) + c.lo * x);
}
// e^x through ex2_mul with log2(e) as a pair.
inline __device__ float expc(float x) {
    const F2 l2e{L2E_HI, L2E_LO};
    return ex2_mul(l2e, x);
}

// Guard band in log2 m around the mass edges: within it the FP32 decision
// whether a sample's source-frame masses lie in [m_min, m_max] (the log2
// masses below carry errors of ~1e-7, from the FP32 redshift) is taken again
// in FP64, weight included, as the FP64 path and the oracle take it.
constexpr float EDGE_GUARD = 1e-6f;
// Corner band above m_min: p(m2|m1) ~ 1 / (m1 - m_min), so the FP32
// d1 = log2(m1/m_min) (absolute error ~1e-7) would give the weight a
// relative error ~1e-7 / d1.  Below W_FP64 (m1 < 1.0014 m_min) d1 is taken
// from the FP64 redshift instead, with an error relative to d1 itself
// (corner_d1: about thirty FP64 operations, a few samples in a thousand).
constexpr float W_FP64 = 2e-3f;
// Same for an injection's redshift against z_max.
constexpr float ZMAX_GUARD = 4e-6f;
// Below this distance of m1 above m_min (log2 m) the normalisation of
// p(m2|m1), 2^(b1 d1) - 1, is taken from its power series.
constexpr float W_SERIES = 0.0625f;

// Mixed-path mass model relative to the point's shared normalisation
// w_scale (carried in FP64, hp.ln_wscale, and added to the log of the event
// integral and of the selection term), in terms of the log2 mass ratios
// d1 = log2(m1/m_min), d2 = log2(m2/m_min), which the sample's log2 masses
// (stored as float pairs) give without cancellation near m_min:
//   p(m1)          = C1 m_min^-alpha [r_pl 2^(-alpha d1) + r_g exp(-(m1 - mu)^2 / 2 sigma^2)],
//   p(m2|m1) |b1|^-1 = m_min^-1 sgn(b1) 2^(beta d2) / (2^(b1 d1) - 1),   b1 = 1 + beta,
//   (beta = -1:   p(m2|m1) = log2(e) m_min^-1 / (2^d2 d1)),
// w_scale = C1 m_min^-alpha m_min^-1 (|b1| or log2 e), C1 = c_pl (c_g when
// c_pl = 0); r_g carries m_min^alpha.
struct WParams {
    float r_pl, r_g;  // c_pl / C1, m_min^alpha c_g / C1
    float mu;
    F2 gk;            // -log2(e) / (2 sigma^2)
    F2 na;            // -alpha
    F2 beta, b1;
    F2 b1ln2;         // b1 ln 2
    F2 l2min, l2max;  // log2 m_min, log2 m_max
    float sgn_b1;
    bool logp2;
    int kv;
    float fv;
};

inline __device__ WParams w_params(const HP &hp) {
    WParams q;
    q.r_pl = hp.r_pl32;
    q.r_g = hp.r_g32;
    q.mu = hp.mu32;
    q.gk = hp.gk2;
    q.na = hp.na2;
    q.beta = hp.beta2;
    q.b1 = hp.b1_2;
    q.b1ln2 = hp.b1ln2_2;
    q.l2min = hp.l2min2;
    q.l2max = hp.l2max2;
    q.sgn_b1 = hp.b1 < 0.0 ? -1.f : 1.f;
    q.logp2 = fabs(hp.b1) < 1e-12;
    q.kv = hp.k_valid;
    q.fv = hp.f_valid;
    return q;
}

// Source-frame log2 masses of a sample from its stored log2 detector-frame
// masses (float hi parts h1, h2 and their low parts lo) and lz = log2(1+z).
struct LogMass {
    float l1, l2;  // log2 m1, log2 m2
    float d1, d2;  // log2(m1 / m_min), log2(m2 / m_min)
    float e1;      // log2(m1 / m_max)
    bool ord;      // m2 <= m1 (redshift-independent)
};
inline __device__ LogMass log_mass(const WParams &q, float h1, float h2, float2 lo, float lz) {
    LogMass m;
    m.l1 = h1 - lz;
    m.l2 = h2 - lz;
    // h - log2 m_min is exact when the two are close (Sterbenz), so the
    // differences keep the low parts
    m.d1 = (h1 - q.l2min.hi) + ((lo.x - q.l2min.lo) - lz);
    m.d2 = (h2 - q.l2min.hi) + ((lo.y - q.l2min.lo) - lz);
    m.e1 = (h1 - q.l2max.hi) + ((lo.x - q.l2max.lo) - lz);
    m.ord = (h2 - h1) + (lo.y - lo.x) <= 0.f;
    return m;
}
// m_min <= m2 <= m1 <= m_max, m1 > m_min.
inline __device__ bool w_in_range(const LogMass &m) {
    return (m.d2 >= 0.f) & (m.e1 <= 0.f) & m.ord & (m.d1 > 0.f);
}
// Whether the sample needs the FP64 weight (see EDGE_GUARD).
inline __device__ bool w_needs64(const LogMass &m) {
    return (fabsf(m.d2) < EDGE_GUARD) | (fabsf(m.e1) < EDGE_GUARD) | ((m.d1 < EDGE_GUARD) & (m.d2 > -EDGE_GUARD));
}
// The weight of an in-range sample, relative to w_scale, as a quotient
// num / den, so that the caller can fold the division into its own one:
//   num = sgn(b1) 2^(-alpha d1 + beta d2) [r_pl + r_g 2^(gk x^2 + alpha d1)],
//   den = 2^(b1 d1) - 1  (its power series near m_min),
// with x = m1 - mu.  Exponents stay far inside +-120 for any admissible
// population; the Gaussian's is clamped at -100 (its term is then ~1e-30
// of the peak and irrelevant beside the power law).
struct WQuot {
    float num, den;
};
inline __device__ WQuot mass_weight_rel(const WParams &q, const LogMass &m) {
    const float x = ex2_pair_n(m.l1, 0.f) - q.mu, x2 = x * x;
    // -alpha d1 and, for the peak, gk x^2 + alpha d1, each with its rounding residual
    const float ta = q.na.hi * m.d1, ra = fmaf(q.na.hi, m.d1, -ta) + q.na.lo * m.d1;
    const float tg = fmaf(q.gk.hi, x2, -ta);
    const float rg = fmaf(q.gk.hi, x2, -(tg + ta)) + q.gk.lo * x2 - ra;
    const float g = ex2_pair_n(fmaxf(tg, -100.f), rg);
    WQuot r;
    if (q.logp2) {
        r.num = ex2_pair_n(ta - m.d2, ra) * fmaf(q.r_g, g, q.r_pl);
        r.den = m.d1;
    } else {
        const float tb = q.beta.hi * m.d2, rb = fmaf(q.beta.hi, m.d2, -tb) + q.beta.lo * m.d2;
        r.num = q.sgn_b1 * ex2_pair_n(ta + tb, ra + rb) * fmaf(q.r_g, g, q.r_pl);
        if (m.d1 < W_SERIES) {
            // 2^(b1 d1) - 1 = expm1(t), t = b1 ln2 d1, |t| < 0.1: Taylor to t^7
            const float t = mul_f2(q.b1ln2, m.d1);
            r.den = t * (1.f + t * (0.5f + t * (1.f / 6.f + t * (1.f / 24.f + t * (1.f / 120.f +
                                                                                  t * (1.f / 720.f + t * (1.f / 5040.f)))))));
        } else {
            r.den = ex2_mul_n(q.b1, m.d1) - 1.f;
        }
    }
    return r;
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



// The FP64 redshift of a sample or injection with an FP32 one z32 (which
// only says whether it has one): cubic Hermite in u = sqrt(d / d_top) on the
// FP64 inverse-table node pairs.  Its interpolation error is ~1e-11 of z at
// z = 0.2 and ~1e-9 at z = 0.002 (measured against a 30-digit inversion),
// far below what the guard bands (1e-6 in log2 m) and the corner band need,
// in about thirty FP64 operations; a Newton step on the forward relation,
// with its power of (1+z), takes some two hundred on B300's narrow FP64
// pipe.  False when d lies beyond d_L^gw(10).
static __device__ bool refine64(const CallPtrs &p, int h, const HP &hp, double inv_dtop, float z32, double d,
                                double *zout) {
    if (!(d > 0.0) || !(d <= hp.d_valid) || !(z32 < CUDART_INF_F)) return false;
    const double x = d * inv_dtop;
    const double t = x * chimd::rsqrt64(x) * NU;  // sqrt(d / d_top) NU
    int k = (int)t;
    if (k > NU - 1) k = NU - 1;
    const double f = t - k;
    const double2 *nd = p.inv64 + (size_t)h * (NU + 1);
    const double2 na = nd[k], nb = nd[k + 1];
    const double f2 = f * f, f3 = f2 * f;
    const double z = (2 * f3 - 3 * f2 + 1) * na.x + (f3 - 2 * f2 + f) * na.y * (1.0 / NU) +
                     (-2 * f3 + 3 * f2) * nb.x + (f3 - f2) * nb.y * (1.0 / NU);
    if (!isfinite(z)) return false;
    *zout = z;
    return true;
}

// d1 = log2(m1 / m_min) of a sample in the corner band (W_FP64) from its
// FP64 redshift: x = m1_det / (m_min (1+z)) - 1 in FP64 (small here, exact to
// ~1e-16 absolute), then log2(1 + x) = log1p(x) log2(e) in FP32, whose error
// is relative to d1 itself.  Not inlined: as straight-line code in the caller
// it could be predicated for every sample.
static __noinline__ __device__ float corner_d1(const CallPtrs &p, int h, const HP &hp, double inv_dtop, float z32,
                                               double d, double m1d, float d1_32) {
    double z;
    if (!refine64(p, h, hp, inv_dtop, z32, d, &z)) return d1_32;
    const double x = m1d / (hp.th[7] * (1.0 + z)) - 1.0;
    const F2 l2e{L2E_HI, L2E_LO};
    return mul_f2(l2e, log1pf((float)x));
}

// The mixed weight of one PE sample or injection in FP64, relative to the
// point's shared normalisation (as mass_weight_rel), with the range test of
// the oracle; 0 when the distance has no redshift or the masses are outside.
static __noinline__ __device__ float mass_weight_rel64(const CallPtrs &p, int h, const HP &hp, double inv_dtop,
                                                       double beta, float z32, double d, double m1d, double m2d) {
    double z;
    if (!refine64(p, h, hp, inv_dtop, z32, d, &z)) return 0.f;
    const double a = 1.0 + z;
    return (float)(mass_weight64(hp, beta, m1d / a, m2d / a) * hp.inv_wscale);
}

}  // namespace chim
