// K5: selection term from the detected injections (Eq. bias and its Monte
// Carlo estimate, Sec. 2.2):
//   s_j = p(m1,m2) psi(z_j) p_z(z_j) / [(1+z_j)^3 |J(z_j)| pi_inj,j],
//   p_z = dV_c/dz / V_c(z_max) on [0, z_max] and 0 beyond,
//   xi = sum_j s_j / N_inj,  N_eff = (sum s)^2 / (sum s^2 - (sum s)^2 / N_inj).
// Each block reduces SEL_CHUNK injections for one hyperpoint into a pair of
// FP64 partial sums (sum s, sum s^2); K6 adds the partials in a fixed order.
// Given z_j, D_c follows exactly from the measured distance,
// D_c = d_L / ((1+z) Xi(z)), so no forward table lookup is needed.
//
// K6: ln L = sum_i ln I_i - N_obs ln xi (Eq. hyperlike), FP64, fixed order.
#include <math_constants.h>

#include "internal.cuh"

namespace chim {

namespace {

__device__ __forceinline__ double warp_sumd(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// mixed: FP32 per term with full-accuracy libm, FP64 across warps
__global__ void __launch_bounds__(SEL_THREADS) k_select_mixed(DevCatalog c, CallPtrs p, int H) {
    __shared__ double red[2 * (SEL_THREADS / 32)];
    const int h = blockIdx.y, chunk = blockIdx.x;
    const HP &hp = p.hp[h];
    const float4 *inv = p.inv32 + (size_t)h * NU;
    const int kv = hp.k_valid;
    const float fv = hp.f_valid;
    const float xi0 = hp.xi0_32, n = hp.n32, om = hp.om32;
    const float gam = hp.gam32, kap = hp.kap32, l1zp = hp.l1zp32;
    const float cH = hp.cH32, zmax = c.z_max32;
    const float inv_dc3 = hp.inv_dc3_32;
    const float mmin = hp.mmin32, mmax = hp.mmax32, mu = hp.mu32;
    const float inv_sg = hp.inv_sg32, alpha = hp.alpha32;
    const float c_pl = hp.c_pl32, c_g = hp.c_g32, beta = hp.beta32;
    const float b1 = hp.b1_32, mmin_b1 = hp.mmin_b1_32, lmmin = hp.lmmin32;
    float s1 = 0.f, s2 = 0.f;
    const int64_t base = (int64_t)chunk * SEL_CHUNK;
    for (int q = 0; q < SEL_PER_THREAD; q++) {
        int64_t j = base + q * SEL_THREADS + threadIdx.x;
        if (j >= c.n_det) break;
        float4 a = c.i32a[j];
        float2 bq = c.i32b[j];
        int k = __float_as_int(a.x);
        float f = a.y;
        if (!((k < kv) || (k == kv && f <= fv))) continue;
        float z = chimd::hermite4(inv[k], f);
        if (!(z <= zmax)) continue;
        float lz = log1pf(z), ap = 1.f + z;
        float lm1 = a.z - lz, lm2 = a.w - lz;
        float m1 = expf(lm1), m2 = expf(lm2);
        if (!(m1 >= mmin && m1 <= mmax && m2 >= mmin && m2 <= m1)) continue;
        float x = (m1 - mu) * inv_sg;
        float p1 = c_pl * expf(-alpha * lm1) + c_g * expf(-0.5f * x * x);
        float p2;
        if (fabsf(b1) < 1e-6f) {
            float l = lm1 - lmmin;
            p2 = l > 0.f ? 1.f / (m2 * l) : 0.f;
        } else {
            float den = m1 * expf(beta * lm1) - mmin_b1;
            p2 = den > 0.f ? b1 * expf(beta * lm2) / den : 0.f;
        }
        float pw = expf(-n * lz);
        float xi = xi0 + (1.f - xi0) * pw;
        float dxi = -n * (1.f - xi0) * pw / ap;
        float Dc = bq.x / (ap * xi);
        float E = sqrtf(om * ap * ap * ap + 1.f - om);
        float J = (Dc + ap * cH / E) * xi + ap * Dc * dxi;
        float psi = expf(gam * lz) / (1.f + expf((gam + kap) * (lz - l1zp)));
        float pz = 3.f * cH * Dc * Dc / E * inv_dc3;
        float s = p1 * p2 * psi * pz / (ap * ap * ap * fabsf(J)) * expf(-bq.y);
        s1 += s;
        s2 += s * s;
    }
    s1 = warp_sumf(s1);
    s2 = warp_sumf(s2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[2 * wid] = s1;
        red[2 * wid + 1] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < SEL_THREADS / 32; w++) {
            a1 += red[2 * w];
            a2 += red[2 * w + 1];
        }
        double *o = p.selp + ((size_t)h * p.n_chunk + chunk) * 2;
        o[0] = a1;
        o[1] = a2;
    }
}

__device__ bool invert64_sel(const DevCatalog &c, const CallPtrs &p, int h, const HP &hp, double d,
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

__global__ void __launch_bounds__(SEL_THREADS) k_select_fp64(DevCatalog c, CallPtrs p, int H) {
    __shared__ double red[2 * (SEL_THREADS / 32)];
    const int h = blockIdx.y, chunk = blockIdx.x;
    const HP &hp = p.hp[h];
    const double *th = hp.th;
    const double cH = hp.cH, inv_dc3 = 1.0 / (hp.dc_zmax * hp.dc_zmax * hp.dc_zmax);
    double s1 = 0.0, s2 = 0.0;
    const int64_t base = (int64_t)chunk * SEL_CHUNK;
    for (int q = 0; q < SEL_PER_THREAD; q++) {
        int64_t j = base + q * SEL_THREADS + threadIdx.x;
        if (j >= c.n_det) break;
        double d = c.id64[j], z;
        if (!invert64_sel(c, p, h, hp, d, &z) || !(z <= c.z_max)) continue;
        double ap = 1.0 + z;
        double m1 = c.im1_64[j] / ap, m2 = c.im2_64[j] / ap;
        const double mmin = th[7], mmax = th[8];
        if (!(m1 >= mmin && m1 <= mmax && m2 >= mmin && m2 <= m1) || !(m1 > mmin)) continue;
        double x = (m1 - th[5]) / th[6];
        double p1 = hp.c_pl * pow(m1, -th[4]) + hp.c_g * exp(-0.5 * x * x);
        double p2 = fabs(hp.b1) < 1e-12 ? 1.0 / (m2 * log(m1 / mmin))
                                         : hp.b1 * pow(m2, c.beta) / (pow(m1, hp.b1) - hp.mmin_b1);
        double dd, J;
        double Dc = cH * chimd::dc_hermite(p.fwd[h], z, th[1]);
        chimd::dgw_J(z, Dc, th, cH, &dd, &J);
        double E = chimd::E_of(z, th[1]);
        double pz = 3.0 * cH * Dc * Dc / E * inv_dc3;
        double s = p1 * p2 * chimd::psi_of(z, th) * pz / (ap * ap * ap * fabs(J) * exp(c.ilp64[j]));
        s1 += s;
        s2 += s * s;
    }
    s1 = warp_sumd(s1);
    s2 = warp_sumd(s2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[2 * wid] = s1;
        red[2 * wid + 1] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < SEL_THREADS / 32; w++) {
            a1 += red[2 * w];
            a2 += red[2 * w + 1];
        }
        double *o = p.selp + ((size_t)h * p.n_chunk + chunk) * 2;
        o[0] = a1;
        o[1] = a2;
    }
}

constexpr int CMB_THREADS = 256;

// Block sum in a fixed order: thread t adds elements t, t+256, ... in
// sequence, then a pairwise tree over the 256 partial sums.
__device__ double fixed_order_sum(const double *x, int64_t n, int64_t stride, double *sh) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += CMB_THREADS) s += x[i * stride];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = CMB_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(CMB_THREADS) k_combine(DevCatalog c, CallPtrs p, int H) {
    __shared__ double sh[2 * CMB_THREADS];
    __shared__ int s_bad;
    const int h = blockIdx.x;
    const HP &hp = p.hp[h];
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    const double *lnI = p.lnI + (size_t)h * c.n_events;
    for (int i = threadIdx.x; i < c.n_events; i += CMB_THREADS)
        if (!isfinite(lnI[i])) s_bad = 1;
    double sI = fixed_order_sum(lnI, c.n_events, 1, sh);
    double S1 = fixed_order_sum(p.selp + (size_t)h * p.n_chunk * 2, p.n_chunk, 2, sh);
    double S2 = fixed_order_sum(p.selp + (size_t)h * p.n_chunk * 2 + 1, p.n_chunk, 2, sh);
    if (threadIdx.x == 0) {
        int st = hp.status;
        double N = (double)c.n_inj_total;
        double xi = S1 / N;
        double neff = S1 > 0.0 ? S1 * S1 / (S2 - S1 * S1 / N) : 0.0;
        if (st & (CHIMERA_PT_OUT_OF_SUPPORT | CHIMERA_PT_NONMONOTONE)) {
            xi = 0.0;
            neff = 0.0;
        }
        double lnL;
        if (st & (CHIMERA_PT_OUT_OF_SUPPORT | CHIMERA_PT_NONMONOTONE)) {
            lnL = -CUDART_INF;
        } else if (s_bad || !(xi > 0.0)) {
            lnL = -CUDART_INF;
            st |= CHIMERA_PT_OUT_OF_SUPPORT;
        } else {
            lnL = sI - (double)c.n_events * log(xi);
        }
        // the effective-count warning is only meaningful for an admissible point
        if (!(hp.status & (CHIMERA_PT_OUT_OF_SUPPORT | CHIMERA_PT_NONMONOTONE)) &&
            !(neff >= 5.0 * c.n_events))
            st |= CHIMERA_PT_NEFF_LOW;
        p.lnL[h] = lnL;
        p.neff[h] = neff;
        p.xi[h] = xi;
        p.status[h] = st;
    }
}

}  // namespace

int selection_chunks(const DevCatalog &c) {
    int64_t n = (c.n_det + SEL_CHUNK - 1) / SEL_CHUNK;
    return (int)(n > 0 ? n : 1);
}

void launch_selection(const DevCatalog &c, const CallPtrs &p, int H, bool fp64, cudaStream_t st) {
    dim3 grid(p.n_chunk, H);
    if (fp64) k_select_fp64<<<grid, SEL_THREADS, 0, st>>>(c, p, H);
    else k_select_mixed<<<grid, SEL_THREADS, 0, st>>>(c, p, H);
}

void launch_combine(const DevCatalog &c, const CallPtrs &p, int H, cudaStream_t st) {
    k_combine<<<H, CMB_THREADS, 0, st>>>(c, p, H);
}

}  // namespace chim
