// K2 + K4: per-event integral I_i for every (event, hyperpoint).
//
// Phase A (reweighting, Sec. 2.1 and Eq. gw-kernel): every PE sample's d_L is
// inverted to z through the hyperpoint's inverse table, the detector-frame
// masses become source-frame masses m = m_det / (1+z), and the KDE weight is
// w = p(m1) p(m2 | m1) (pi_PE = 1).  The weighted moments give the
// bandwidth b = sigma_w n_eff^(-1/5) (Scott's rule with the weighted n_eff,
// shared by the event's pixels).
//
// Phase B (Eqs. like-integrals, gw-kernel-many1d / gw-kernel-single1d):
//   I = sum_k pf_k sum_{j in k} w_j sum_a w_a phi_b(z_a - z_j) F(z_a) G_k(z_a)
// with pf_k = S_k / N_k (many-1D) or 1 / N_s (single-1D, G summed over
// pixels).  Samples are stored sorted by d_L inside each segment, hence by z
// for every hyperpoint, and processed in warp groups of up to 64 neighbours.
//
// Mixed kernel, fast path: for a group with origin grid index t_o the
// Gaussian factorises on the uniform grid,
//   exp(-(u - ds tau)^2) = exp(-u^2) * exp(2 u ds)^tau * exp(-ds^2 tau^2),
// u = (z_j - z_o)/(sqrt2 b), ds = dz/(sqrt2 b), tau = a - t_o, so with the
// per-group table D_tau = exp(-ds^2 tau^2) w'_a F(z_a) G(z_a) in shared
// memory the inner loop is one multiply (P *= B) and one FMA (acc += P D)
// per grid point and sample, with D read as a broadcast float4.  Two chains
// per sample run outwards from the group centre.  Groups whose spread
// exceeds 8 b, whose kernel is narrower than 1.4 grid steps, or whose table
// would not fit, use a direct per-sample window with one exp per point.
//
// FP64 kernel: the plain form, one exp per grid point and sample within
// +-9 b, every quantity in double.
#include <math_constants.h>

#include "internal.cuh"

namespace chim {

namespace {

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sumd(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of NV floats per thread, accumulated across warps in double.
// Result left in red[0..NV-1]; all threads see it after the call.
template <int NV, int NT>
__device__ void block_sum(float (&v)[NV], double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; q++) {
        float s = warp_sum(v[q]);
        if (lane == 0) red[8 + wid * NV + q] = (double)s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; w++) s += red[8 + w * NV + threadIdx.x];
        red[threadIdx.x] = s;
    }
    __syncthreads();
}

template <int NV, int NT>
__device__ void block_sumd(double (&v)[NV], double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; q++) {
        double s = warp_sumd(v[q]);
        if (lane == 0) red[8 + wid * NV + q] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; w++) s += red[8 + w * NV + threadIdx.x];
        red[threadIdx.x] = s;
    }
    __syncthreads();
}

// Scott bandwidth from the moment sums (same rule as the paper reading:
// weighted, then unweighted, then the grid spacing).
__device__ __forceinline__ double bandwidth_rule(double W1, double W2, double Vw, double nv,
                                                 double Vu, double dz) {
    if (W1 > 0.0) {
        double var = Vw / W1, neff = W1 * W1 / W2;
        if (neff >= 2.0 && var > 0.0) return sqrt(var) * pow(neff, -0.2);
    }
    if (nv >= 2.0 && Vu > 0.0) return sqrt(Vu / nv) * pow(nv, -0.2);
    return dz;
}

// Shared layout of the mixed kernel (floats unless noted).
struct MixLayout {
    int ns_pad, nz_pad, seg_pad;
    __host__ __device__ static int pad4(int x) { return (x + 3) & ~3; }
    __host__ __device__ MixLayout(int max_ns, int nz, int max_seg) {
        ns_pad = pad4(max_ns);
        nz_pad = pad4(nz);
        seg_pad = pad4(max_seg + 1);
    }
    __host__ __device__ size_t bytes() const {
        return sizeof(float) * (2 * (size_t)ns_pad + nz_pad + (size_t)EV_WARPS * DCAP) +
               sizeof(int) * 2 * (size_t)seg_pad + sizeof(double) * (8 + EV_WARPS * 8);
    }
};

struct MixParams {
    float c_pl, c_g, alpha, mu, inv_sg, mmin, mmax, beta, b1, mmin_b1, lmmin;
    int kv;
    float fv;
};

__device__ __forceinline__ float mass_weight32(const MixParams &q, float lm1, float lm2) {
    float m1 = expf(lm1), m2 = expf(lm2);
    if (!(m1 >= q.mmin && m1 <= q.mmax && m2 >= q.mmin && m2 <= m1)) return 0.f;
    float x = (m1 - q.mu) * q.inv_sg;
    float p1 = q.c_pl * expf(-q.alpha * lm1) + q.c_g * expf(-0.5f * x * x);
    float p2;
    if (fabsf(q.b1) < 1e-6f) {
        float l = lm1 - q.lmmin;
        p2 = l > 0.f ? 1.f / (m2 * l) : 0.f;
    } else {
        float den = m1 * expf(q.beta * lm1) - q.mmin_b1;
        p2 = den > 0.f ? q.b1 * expf(q.beta * lm2) / den : 0.f;
    }
    return p1 * p2;
}

template <int R>
__device__ __forceinline__ void chains(const float *D, int T4, const float (&u)[R], float ds,
                                       float (&acc)[R]) {
    float Pf[R], Pb[R], B[R], Bi[R], af[R], ab[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        float A = expf(-u[r] * u[r]);
        B[r] = expf(2.f * u[r] * ds);
        Bi[r] = expf(-2.f * u[r] * ds);
        Pf[r] = A;
        Pb[r] = A * Bi[r];
        af[r] = 0.f;
        ab[r] = 0.f;
    }
    const float4 *Df = reinterpret_cast<const float4 *>(D + T4 + 4);
    const int nq = (T4 + 4) >> 2;
#pragma unroll 2
    for (int q = 0; q < nq; q++) {
        float4 d = Df[q];
        float4 e = Df[-q - 1];
#pragma unroll
        for (int r = 0; r < R; r++) {
            af[r] = fmaf(Pf[r], d.x, af[r]); Pf[r] *= B[r];
            af[r] = fmaf(Pf[r], d.y, af[r]); Pf[r] *= B[r];
            af[r] = fmaf(Pf[r], d.z, af[r]); Pf[r] *= B[r];
            af[r] = fmaf(Pf[r], d.w, af[r]); Pf[r] *= B[r];
            ab[r] = fmaf(Pb[r], e.w, ab[r]); Pb[r] *= Bi[r];
            ab[r] = fmaf(Pb[r], e.z, ab[r]); Pb[r] *= Bi[r];
            ab[r] = fmaf(Pb[r], e.y, ab[r]); Pb[r] *= Bi[r];
            ab[r] = fmaf(Pb[r], e.x, ab[r]); Pb[r] *= Bi[r];
        }
    }
#pragma unroll
    for (int r = 0; r < R; r++) acc[r] = af[r] + ab[r];
}

__global__ void __launch_bounds__(EV_THREADS, 2) k_event_mixed(DevCatalog c, CallPtrs p, int H) {
    extern __shared__ float4 smem4[];
    const MixLayout L(c.max_ns, c.n_z, c.max_seg);
    float *zs = reinterpret_cast<float *>(smem4);
    float *ws = zs + L.ns_pad;
    float *Fs = ws + L.ns_pad;
    float *Dt = Fs + L.nz_pad;
    int *segv = reinterpret_cast<int *>(Dt + EV_WARPS * DCAP);
    int *gpre = segv + L.seg_pad;
    double *red = reinterpret_cast<double *>(gpre + L.seg_pad);
    __shared__ int s_gctr;

    const int h = blockIdx.x % H;
    const int ev = c.ev_order[blockIdx.x / H];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const size_t out = (size_t)h * c.n_events + ev;
    const HP &hp = p.hp[h];
    if (hp.status & (CHIMERA_PT_OUT_OF_SUPPORT | CHIMERA_PT_NONMONOTONE)) {
        if (tid == 0) { p.lnI[out] = 0.0; p.bw[out] = 0.0; }
        return;
    }
    MixParams q;
    q.c_pl = (float)hp.c_pl; q.c_g = (float)hp.c_g; q.alpha = (float)hp.th[4];
    q.mu = (float)hp.th[5]; q.inv_sg = (float)(1.0 / hp.th[6]); q.mmin = (float)hp.th[7];
    q.mmax = (float)hp.th[8]; q.beta = (float)c.beta; q.b1 = (float)hp.b1;
    q.mmin_b1 = (float)hp.mmin_b1; q.lmmin = (float)hp.lmmin; q.kv = hp.k_valid; q.fv = hp.f_valid;

    const int nz = c.n_z;
    const float dz = (float)c.dz;
    for (int a = tid; a < nz; a += EV_THREADS) Fs[a] = p.F32[(size_t)h * nz + a];

    // ---- phase A: z_j, w_j and the moment sums
    const int64_t s0 = c.ev_soff[ev];
    const int ns = (int)(c.ev_soff[ev + 1] - s0);
    const float4 *inv = p.inv32 + (size_t)h * NU;
    float acc1[4] = {0.f, 0.f, 0.f, 0.f};  // W1, Wz, W2, n_valid
    float accz = 0.f;
    for (int j = tid; j < ns; j += EV_THREADS) {
        float4 s = c.s32[s0 + j];
        int k = __float_as_int(s.x);
        float f = s.y;
        float z = CUDART_INF_F, w = 0.f;
        bool valid = (k < q.kv) || (k == q.kv && f <= q.fv);
        if (valid) {
            float zz = chimd::hermite4(inv[k], f);
            if (isfinite(zz)) {
                z = zz;
                float lz = log1pf(z);
                w = mass_weight32(q, s.z - lz, s.w - lz);
            }
        }
        zs[j] = z;
        ws[j] = w;
        if (z < CUDART_INF_F) {
            acc1[0] += w; acc1[1] += w * z; acc1[2] += w * w; acc1[3] += 1.f;
            accz += z;
        }
    }
    {
        float v[5] = {acc1[0], acc1[1], acc1[2], acc1[3], accz};
        block_sum<5, EV_THREADS>(v, red);
    }
    const double W1 = red[0], Wz = red[1], W2 = red[2], nv = red[3], Sz = red[4];
    __syncthreads();
    const float mw = W1 > 0.0 ? (float)(Wz / W1) : 0.f;
    const float mu_ = nv > 0.0 ? (float)(Sz / nv) : 0.f;
    {
        float v[2] = {0.f, 0.f};
        for (int j = tid; j < ns; j += EV_THREADS) {
            float z = zs[j];
            if (z < CUDART_INF_F) {
                float dw = z - mw, du = z - mu_;
                v[0] += ws[j] * dw * dw;
                v[1] += du * du;
            }
        }
        block_sum<2, EV_THREADS>(v, red);
    }
    const double bd = bandwidth_rule(W1, W2, red[0], nv, red[1], c.dz);
    const float b = (float)bd;

    // ---- segments: valid prefix (sorted d_L => z ascending, invalid at the end)
    const int sg0 = c.ev_segoff[ev], nseg = c.ev_segoff[ev + 1] - sg0;
    for (int k = tid; k < nseg; k += EV_THREADS) {
        int lo = (int)(c.seg_soff[sg0 + k] - s0), hi = (int)(c.seg_soff[sg0 + k + 1] - s0);
        int l = lo, r = hi;
        while (l < r) {
            int m = (l + r) >> 1;
            if (zs[m] < CUDART_INF_F) l = m + 1; else r = m;
        }
        segv[k] = l - lo;
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int k = 0; k < nseg; k++) {
            gpre[k] = acc;
            acc += (segv[k] + GROUP_MAX - 1) / GROUP_MAX;
        }
        gpre[nseg] = acc;
        s_gctr = 0;
    }
    __syncthreads();
    const int ngroups = gpre[nseg];

    // ---- phase B: warp groups
    const float inv_s2b = 0.70710678f / b;
    const float ds = dz * inv_s2b;
    const float halfk = KW32 * b;
    float *D = Dt + wid * DCAP;
    const float *prof = reinterpret_cast<const float *>(p.prof[h]);
    float lsum = 0.f, lcomp = 0.f;  // Kahan
    unsigned long long npairs = 0;  // algorithmic pair count (roofline only)
    while (true) {
        int g = 0;
        if (lane == 0) g = atomicAdd(&s_gctr, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ngroups) break;
        int l = 0, r = nseg;  // gpre[l] <= g < gpre[l+1]
        while (r - l > 1) {
            int m = (l + r) >> 1;
            if (gpre[m] <= g) l = m; else r = m;
        }
        const int sk = l;
        const int gi = g - gpre[sk];
        const int lo = (int)(c.seg_soff[sg0 + sk] - s0) + gi * GROUP_MAX;
        const int cnt = min(GROUP_MAX, segv[sk] - gi * GROUP_MAX);
        const float pf = (float)c.seg_pf[sg0 + sk];
        const int64_t row = c.kde_mode == CHIMERA_KDE_MANY_1D ? (int64_t)(sg0 + sk) : (int64_t)ev;
        const float *G = prof + row * nz;
        const float zlo = zs[lo], zhi = zs[lo + cnt - 1];
        const float spread = zhi - zlo;
        const float halfw = 0.5f * spread + halfk;
        const float Tf = ceilf(halfw / dz) + 1.f;
        const int T = Tf < (float)DCAP ? (int)Tf : DCAP;  // beyond DCAP the fast path is off anyway
        const int T4 = (T + 3) & ~3;
        const int t_o = (int)rintf(0.5f * (zlo + zhi) / dz);
        if (p.pairs) {
            for (int j = lane; j < cnt; j += 32) {
                float z = zs[lo + j];
                if (ws[lo + j] == 0.f) continue;
                int a0 = max(0, (int)ceilf((z - halfk) / dz));
                int a1 = min(nz - 1, (int)floorf((z + halfk) / dz));
                if (a1 >= a0) npairs += (unsigned long long)(a1 - a0 + 1);
            }
        }
        if (t_o - T > nz - 1 || t_o + T < 0) continue;  // group entirely off the grid
        const bool fast = spread <= 8.f * b && ds <= 0.5f && 2 * T4 + 8 <= DCAP;
        float v = 0.f;
        if (fast) {
            __syncwarp();
            for (int idx = lane; idx < 2 * T4 + 8; idx += 32) {
                int tau = idx - (T4 + 4);
                int a = t_o + tau;
                float val = 0.f;
                if (tau >= -T && tau <= T && a >= 0 && a < nz) {
                    float x = ds * (float)tau;
                    float wa = (a == 0 || a == nz - 1) ? 0.5f : 1.f;
                    val = expf(-x * x) * wa * Fs[a] * G[a];
                }
                D[idx] = val;
            }
            __syncwarp();
            const float zo = t_o * dz;
            if (cnt > 32) {
                float u[2], w2[2], acc[2];
#pragma unroll
                for (int rr = 0; rr < 2; rr++) {
                    int j = lane + 32 * rr;
                    bool in = j < cnt;
                    u[rr] = in ? (zs[lo + j] - zo) * inv_s2b : 0.f;
                    w2[rr] = in ? ws[lo + j] : 0.f;
                }
                chains<2>(D, T4, u, ds, acc);
                v = w2[0] * acc[0] + w2[1] * acc[1];
            } else {
                float u[1], acc[1];
                bool in = lane < cnt;
                u[0] = in ? (zs[lo + lane] - zo) * inv_s2b : 0.f;
                float w1 = in ? ws[lo + lane] : 0.f;
                chains<1>(D, T4, u, ds, acc);
                v = w1 * acc[0];
            }
        } else {
            for (int j = lane; j < cnt; j += 32) {
                float z = zs[lo + j], w = ws[lo + j];
                if (w == 0.f) continue;
                int a0 = max(0, (int)ceilf((z - halfk) / dz));
                int a1 = min(nz - 1, (int)floorf((z + halfk) / dz));
                float s = 0.f;
                for (int a = a0; a <= a1; a++) {
                    float x = (a * dz - z) * inv_s2b;
                    float wa = (a == 0 || a == nz - 1) ? 0.5f : 1.f;
                    s += expf(-x * x) * wa * Fs[a] * G[a];
                }
                v += w * s;
            }
        }
        float y = pf * v - lcomp;
        float t = lsum + y;
        lcomp = (t - lsum) - y;
        lsum = t;
    }
    {
        float vv[1] = {lsum};
        __syncthreads();
        block_sum<1, EV_THREADS>(vv, red);
    }
    if (p.pairs) {
        for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
        if (lane == 0 && npairs) atomicAdd(p.pairs + h, npairs);
    }
    if (tid == 0) {
        double I = red[0];
        double pref = c.dz * hp.F_scale / (c.n_gal_total * 2.50662827463100050242 * bd);
        p.lnI[out] = I > 0.0 ? log(I) + log(pref) : -CUDART_INF;
        p.bw[out] = bd;
    }
}

// ---------------------------------------------------------------- FP64 ---
__device__ double mass_weight64(const HP &hp, double beta, double m1, double m2) {
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
__device__ bool invert64(const DevCatalog &c, const CallPtrs &p, int h, const HP &hp, double d,
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

__global__ void __launch_bounds__(EV64_THREADS) k_event_fp64(DevCatalog c, CallPtrs p, int H) {
    extern __shared__ double sd[];
    double *zs = sd;
    double *ws = zs + c.max_ns;
    int *segv = reinterpret_cast<int *>(ws + c.max_ns);
    double *red = reinterpret_cast<double *>(segv + ((c.max_seg + 2) & ~1));
    const int h = blockIdx.x % H;
    const int ev = c.ev_order[blockIdx.x / H];
    const int tid = threadIdx.x;
    const size_t out = (size_t)h * c.n_events + ev;
    const HP &hp = p.hp[h];
    if (hp.status & (CHIMERA_PT_OUT_OF_SUPPORT | CHIMERA_PT_NONMONOTONE)) {
        if (tid == 0) { p.lnI[out] = 0.0; p.bw[out] = 0.0; }
        return;
    }
    const int64_t s0 = c.ev_soff[ev];
    const int ns = (int)(c.ev_soff[ev + 1] - s0);
    double a4[5] = {0, 0, 0, 0, 0};
    for (int j = tid; j < ns; j += EV64_THREADS) {
        double z = 0.0, w = 0.0;
        bool ok = invert64(c, p, h, hp, c.sd64[s0 + j], &z);
        if (ok) {
            double m1 = c.sm1_64[s0 + j] / (1.0 + z), m2 = c.sm2_64[s0 + j] / (1.0 + z);
            w = mass_weight64(hp, c.beta, m1, m2);
            a4[0] += w; a4[1] += w * z; a4[2] += w * w; a4[3] += 1.0; a4[4] += z;
        } else {
            z = CUDART_INF;
        }
        zs[j] = z;
        ws[j] = w;
    }
    block_sumd<5, EV64_THREADS>(a4, red);
    const double W1 = red[0], Wz = red[1], W2 = red[2], nv = red[3], Sz = red[4];
    __syncthreads();
    const double mw = W1 > 0.0 ? Wz / W1 : 0.0, mu_ = nv > 0.0 ? Sz / nv : 0.0;
    {
        double v[2] = {0.0, 0.0};
        for (int j = tid; j < ns; j += EV64_THREADS) {
            double z = zs[j];
            if (z < CUDART_INF) {
                v[0] += ws[j] * (z - mw) * (z - mw);
                v[1] += (z - mu_) * (z - mu_);
            }
        }
        block_sumd<2, EV64_THREADS>(v, red);
    }
    const double b = bandwidth_rule(W1, W2, red[0], nv, red[1], c.dz);
    const int sg0 = c.ev_segoff[ev], nseg = c.ev_segoff[ev + 1] - sg0;
    for (int k = tid; k < nseg; k += EV64_THREADS) {
        int lo = (int)(c.seg_soff[sg0 + k] - s0), hi = (int)(c.seg_soff[sg0 + k + 1] - s0);
        int l = lo, r = hi;
        while (l < r) {
            int m = (l + r) >> 1;
            if (zs[m] < CUDART_INF) l = m + 1; else r = m;
        }
        segv[k] = l - lo;
    }
    __syncthreads();
    const int nz = c.n_z;
    const double dz = c.dz;
    const double *F = p.F64 + (size_t)h * nz;
    const double *prof = reinterpret_cast<const double *>(p.prof[h]);
    double tsum = 0.0;
    for (int j = tid; j < ns; j += EV64_THREADS) {
        // segment of sample j: last k with seg_soff[sg0 + k] - s0 <= j
        int l = 0, r = nseg;
        while (r - l > 1) {
            int m = (l + r) >> 1;
            if ((int)(c.seg_soff[sg0 + m] - s0) <= j) l = m; else r = m;
        }
        const int lo = (int)(c.seg_soff[sg0 + l] - s0);
        if (j - lo >= segv[l]) continue;  // beyond d_L^gw(10)
        double z = zs[j], w = ws[j];
        if (w == 0.0) continue;
        const int64_t row = c.kde_mode == CHIMERA_KDE_MANY_1D ? (int64_t)(sg0 + l) : (int64_t)ev;
        const double *G = prof + row * nz;
        double a0 = ceil((z - KW64 * b) / dz), a1 = floor((z + KW64 * b) / dz);
        int ia0 = a0 < 0.0 ? 0 : (a0 > nz ? nz : (int)a0);
        int ia1 = a1 > nz - 1 ? nz - 1 : (a1 < -1.0 ? -1 : (int)a1);
        double s = 0.0;
        for (int a = ia0; a <= ia1; a++) {
            double x = (a * dz - z) / b;
            double wa = (a == 0 || a == nz - 1) ? 0.5 : 1.0;
            s += exp(-0.5 * x * x) * wa * F[a] * G[a];
        }
        tsum += c.seg_pf[sg0 + l] * w * s;
    }
    {
        double v[1] = {tsum};
        __syncthreads();
        block_sumd<1, EV64_THREADS>(v, red);
    }
    if (tid == 0) {
        double I = red[0] * dz / (c.n_gal_total * 2.50662827463100050242 * b);
        p.lnI[out] = I > 0.0 ? log(I) : -CUDART_INF;
        p.bw[out] = b;
    }
}

}  // namespace

size_t event_mixed_smem(const DevCatalog &c) { return MixLayout(c.max_ns, c.n_z, c.max_seg).bytes(); }

size_t event_fp64_smem(const DevCatalog &c) {
    return sizeof(double) * 2 * (size_t)c.max_ns + sizeof(int) * (size_t)((c.max_seg + 2) & ~1) +
           sizeof(double) * (8 + (EV64_THREADS / 32) * 8);
}

void launch_event_mixed(const DevCatalog &c, const CallPtrs &p, int H, cudaStream_t st) {
    size_t smem = event_mixed_smem(c);
    cudaFuncSetAttribute(k_event_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_event_mixed<<<(unsigned)(c.n_events * H), EV_THREADS, smem, st>>>(c, p, H);
}

void launch_event_fp64(const DevCatalog &c, const CallPtrs &p, int H, cudaStream_t st) {
    size_t smem = event_fp64_smem(c);
    cudaFuncSetAttribute(k_event_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_event_fp64<<<(unsigned)(c.n_events * H), EV64_THREADS, smem, st>>>(c, p, H);
}

}  // namespace chim
