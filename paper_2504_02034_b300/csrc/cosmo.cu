// K1: cosmology tables (Eqs. dL-em, dL-mg, jacobian; Sec. 2.1).
//
// k_fwd_panels + k_fwd_offsets - per distinct Om: cumulative D_c(z_k)/(c/H0)
//                on the forward grid z_k = k*HT by 5-point Gauss-Legendre
//                panels, one panel per thread over FWD_BLOCKS blocks (the FP64
//                evaluations spread over that many SMs), block prefix sums and
//                a one-block pass that adds the preceding blocks' totals, all
//                in FP64.  The same pair gives the Om derivative of the table
//                for the adjoint.
// k_nodes_grid, k_inv_nodes, k_hyper_final - per hyperpoint, each spread over
//                (nodes x hyperpoints) so that the work uses every SM: d_L^gw
//                and J on the forward nodes (monotonicity check on z <= 10),
//                the inverse table z(u), u = sqrt(d_L/d_top), by Newton on the
//                Hermite-interpolated forward relation, the grid factor
//                F(z_a) = psi(z_a) / [(1+z_a)^3 |J(z_a)|] of Eq. like-integrals,
//                and the mass-model normalisations.
#include <math_constants.h>

#include "internal.cuh"
#include "mass.cuh"

namespace chim {

namespace {

constexpr int FWD_THREADS = 128;
constexpr int FWD_BLOCKS = (NT_FWD - 1 + FWD_THREADS - 1) / FWD_THREADS;

// Integrand of the table: 1/E (KIND 0) or d(1/E)/dOm = -((1+z)^3 - 1)/(2 E^3)
// (KIND 1, the Om derivative used by the adjoint).
template <int KIND>
__device__ __forceinline__ double fwd_integrand(double z, double Om) {
    const double E = chimd::E_of(z, Om);
    if (KIND == 0) return 1.0 / E;
    const double a = 1.0 + z;
    return -0.5 * (a * a * a - 1.0) / (E * E * E);
}

// One panel [z_k, z_k+1] per thread, 5-point Gauss-Legendre (nodes and
// weights in closed form); out[k+1] = the block's inclusive prefix.  The
// tables of a batch of Om values are built side by side (blockIdx.y).
template <int KIND>
__global__ void __launch_bounds__(FWD_THREADS) k_fwd_panels(FwdBatch b) {
    __shared__ double warp_tot[FWD_THREADS / 32];
    const double Om = b.Om[blockIdx.y];
    double *out = b.out[blockIdx.y];
    const int t = threadIdx.x, k = blockIdx.x * FWD_THREADS + t;
    const double x1 = sqrt(5.0 - 2.0 * sqrt(10.0 / 7.0)) / 3.0;
    const double x2 = sqrt(5.0 + 2.0 * sqrt(10.0 / 7.0)) / 3.0;
    const double w0 = 128.0 / 225.0;
    const double w1 = (322.0 + 13.0 * sqrt(70.0)) / 900.0;
    const double w2 = (322.0 - 13.0 * sqrt(70.0)) / 900.0;
    double s = 0.0;
    if (k < NT_FWD - 1) {
        const double m = (k + 0.5) * HT, hh = 0.5 * HT;
        s = hh * (w0 * fwd_integrand<KIND>(m, Om) +
                  w1 * (fwd_integrand<KIND>(m - hh * x1, Om) + fwd_integrand<KIND>(m + hh * x1, Om)) +
                  w2 * (fwd_integrand<KIND>(m - hh * x2, Om) + fwd_integrand<KIND>(m + hh * x2, Om)));
    }
    const int lane = t & 31, wid = t >> 5;
    double v = s;
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    double off = 0.0;
    for (int w = 0; w < wid; w++) off += warp_tot[w];
    if (k < NT_FWD - 1) out[k + 1] = off + v;
    if (k == 0) out[0] = 0.0;
}

// Adds to every block's entries the totals of the blocks before it (the
// totals are read in parallel, then added in block order).
__global__ void __launch_bounds__(1024) k_fwd_offsets(FwdBatch b) {
    __shared__ double tot[FWD_BLOCKS], off[FWD_BLOCKS];
    double *out = b.out[blockIdx.x];
    if (threadIdx.x + 1 < FWD_BLOCKS) tot[threadIdx.x] = out[(threadIdx.x + 1) * FWD_THREADS];  // block's total
    __syncthreads();
    if (threadIdx.x == 0) {
        double run = 0.0;
        for (int b = 0; b < FWD_BLOCKS; b++) {
            off[b] = run;
            if (b + 1 < FWD_BLOCKS) run += tot[b];
        }
    }
    __syncthreads();
    for (int k = FWD_THREADS + threadIdx.x; k < NT_FWD - 1; k += 1024) out[k + 1] += off[k / FWD_THREADS];
}

constexpr int HYP_THREADS = 256;


__device__ double std_normal_cdf(double x) { return 0.5 * erfc(-x * 0.70710678118654752440); }

// FP32 forward relation at z from D = D_c [Mpc]: d_L^gw and its z-derivative J.
__device__ __forceinline__ void dgw_J32(float z, float D, float cH, float om, float xi0, float n, float &d,
                                       float &J) {
    const float a = 1.f + z;
    const float pw = exp2f(-n * log2f(a));  // (1+z)^-n
    const float xi = xi0 + (1.f - xi0) * pw;
    const float dxi = -n * (1.f - xi0) * pw / a;
    const float E = sqrtf(om * a * a * a + 1.f - om);
    d = a * D * xi;
    J = (D + a * cH / E) * xi + a * D * dxi;
}

// The mixed path's FP32 forward relation for the grid factor: the
// hyperpoint's constants as float pairs (built once per block in FP64), so
// that F carries only errors that differ from point to point of the grid (a
// constant rounded to float would scale every event integral of the
// hyperpoint alike).
struct FwdC32 {
    F2 cH;              // c / H0 [Mpc]
    F2 xi0, omx;        // Xi0, 1 - Xi0
    F2 nn, nomx;        // -n, n (1 - Xi0)
    F2 om, omc;         // Om, 1 - Om
    F2 gam, gkp, l2zp;  // gamma, gamma + kappa, log2(1 + z_p)
};
__device__ FwdC32 fwd_consts32(const double *th) {
    FwdC32 k;
    k.cH = split_f2(C_KMS / th[0]);
    k.xi0 = split_f2(th[2]);
    k.omx = split_f2(1.0 - th[2]);
    k.nn = split_f2(-th[3]);
    k.nomx = split_f2(th[3] * (1.0 - th[2]));
    k.om = split_f2(th[1]);
    k.omc = split_f2(1.0 - th[1]);
    k.gam = split_f2(th[9]);
    k.gkp = split_f2(th[9] + th[10]);
    k.l2zp = split_f2(log1p(th[11]) * 1.4426950408889634074);
    return k;
}
__device__ __forceinline__ float E32p(const FwdC32 &k, float a) {
    const float a3 = a * a * a;
    return sqrtf(fmaf(k.om.hi, a3, k.omc.hi) + fmaf(k.om.lo, a3, k.omc.lo));
}
// Dhat = D_c H0 / c by cubic Hermite on the FP64 forward table (node values
// rounded to float, slopes 1/E with the pair constants).
__device__ __forceinline__ float dc_hermite32p(const double *fwd, float z, const FwdC32 &kc) {
    const float ht = (float)HT;
    const float t = z * (1.f / (float)HT);  // HT is a power of two: exact
    const int k = min(max((int)floorf(t), 0), NT_FWD - 2);
    const float f = t - k, f2 = f * f, f3 = f2 * f;
    return (2.f * f3 - 3.f * f2 + 1.f) * (float)fwd[k] + (f3 - 2.f * f2 + f) * (ht / E32p(kc, 1.f + k * ht)) +
           (-2.f * f3 + 3.f * f2) * (float)fwd[k + 1] + (f3 - f2) * (ht / E32p(kc, 1.f + (k + 1) * ht));
}
// At z (lz = log2(1+z)) from Dhat: pw = (1+z)^-n, Xi, and Jh = J H0 / c =
// (Dhat + (1+z)/E) Xi - n (1 - Xi0) (1+z)^-n Dhat.
__device__ __forceinline__ void fwd32p(const FwdC32 &k, float z, float lz, float Dh, float &xi, float &Jh) {
    const float a = 1.f + z;
    const float pw = ex2_mul_n(k.nn, lz);
    xi = fmaf(k.omx.hi, pw, k.xi0.hi) + fmaf(k.omx.lo, pw, k.xi0.lo);
    Jh = (Dh + a / E32p(k, a)) * xi - mul_f2(k.nomx, pw) * Dh;
}

// K1b.1, one launch for two independent parts per hyperpoint (blockIdx.y):
//  * blocks x < nbn: d_L^gw and J at the forward nodes, in FP32 (they seed
//    the FP64 inversion and carry the monotonicity check: J <= 0 on z <= 10
//    sets the NONMONOTONE bit);
//  * blocks x >= nbn: the grid factor F(z_a) = psi / ((1+z)^3 |J|) (psi alone
//    when the Jacobian sits on the samples, p.jac_ps) and its
//    maximum, in FP64 for FP64 calls (F64), in FP32 for mixed ones (F32, not
//    yet normalised).
__global__ void __launch_bounds__(HYP_THREADS) k_nodes_grid(DevCatalog c, CallPtrs p, float2 *djall,
                                                           unsigned long long *fmax_bits, int nbn, bool f64) {
    const int h = blockIdx.y;
    const double *th = p.theta + 12 * h;
    const double cH = C_KMS / th[0];
    const double *fwd = p.fwd[h];
    if ((int)blockIdx.x < nbn) {
        const int k = blockIdx.x * HYP_THREADS + threadIdx.x;
        if (k >= NT_FWD) return;
        float d, J;
        dgw_J32(k * (float)HT, (float)(cH * fwd[k]), (float)cH, (float)th[1], (float)th[2], (float)th[3], d, J);
        djall[(size_t)h * NT_FWD + k] = make_float2(d, J);
        if (k <= K_Z10 && !(J > 0.f)) atomicOr(p.status + h, CHIMERA_PT_NONMONOTONE);
        return;
    }
    __shared__ FwdC32 kc;
    if (!f64 && threadIdx.x == 0) kc = fwd_consts32(th);
    __syncthreads();
    const int a = (blockIdx.x - nbn) * HYP_THREADS + threadIdx.x;
    unsigned long long bits = 0;
    if (a < c.n_z) {
        if (f64) {
            double z = a * c.dz, d, J;
            chimd::dgw_J(z, cH * chimd::dc_hermite(fwd, z, th[1]), th, cH, &d, &J);
            const double ap = 1.0 + z;
            double F = p.jac_ps ? chimd::psi_of(z, th) : chimd::psi_of(z, th) / (ap * ap * ap * fabs(J));
            if (!isfinite(F)) F = 0.0;
            p.F64[(size_t)h * c.n_z + a] = F;
            bits = (unsigned long long)__double_as_longlong(F);
        } else {
            // mixed: F' = F c / H0 = psi / ((1+z)^3 |J H0/c|) in FP32 with the
            // pair constants (H0 / c goes into the FP64 log offset ln_k0);
            // psi alone with the Jacobian on the samples
            const float z = (float)(a * c.dz), ap = 1.f + z;
            const F2 l2e{L2E_HI, L2E_LO};
            const float lz = mul_f2(l2e, log1pf(z));
            const float psi = ex2_mul_n(kc.gam, lz) / (1.f + ex2_mul(kc.gkp, (lz - kc.l2zp.hi) - kc.l2zp.lo));
            float F = psi;
            if (!p.jac_ps) {
                float xi, Jh;
                fwd32p(kc, z, lz, dc_hermite32p(fwd, z, kc), xi, Jh);
                F = psi / (ap * ap * ap * fabsf(Jh));
            }
            if (!isfinite(F)) F = 0.f;
            p.F32[(size_t)h * c.n_z + a] = F;
            bits = (unsigned long long)__float_as_uint(F);
        }
    }
    // F >= 0, so the ordering of the bit patterns is the ordering of the values
    for (int o = 16; o > 0; o >>= 1) bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, o));
    if ((threadIdx.x & 31) == 0 && bits > 0) atomicMax(fmax_bits + h, bits);
}

// K1b.2: inverse nodes z(u_k), d = d_top u_k^2: bracketing on the forward
// nodes (staged in shared memory), cubic Hermite of z(d) between the two
// bracketing nodes (slopes 1/J), then one FP64 Newton step on the Hermite-
// interpolated forward relation.  The FP64 nodes (inv64) serve the FP64
// path and the adjoint; the FP32 node pairs that the mixed kernels
// interpolate (inv32) are those nodes rounded, and beside them go the pairs
// of log2(1+z) (linv32), which the mixed kernels interpolate in place of a
// log per sample.  (Measured on the benchmark catalogs: FP32 Newton nodes,
// even with the hyperpoint's constants as float pairs, shift every event of
// a hyperpoint by up to 1e-7 in ln I alike; the rounded FP64 nodes do not.)
// A block computes the nodes base .. base+INV_THREADS (one more than it
// owns) so that it also writes the FP32 pairs of its intervals.
constexpr int INV_THREADS = 128;  // 2049 nodes x H spread over every SM
__global__ void __launch_bounds__(INV_THREADS) k_inv_nodes(DevCatalog c, CallPtrs p, const float2 *djall) {
    __shared__ float sdk[NT_FWD];
    __shared__ float4 snd32[INV_THREADS + 1];  // z, dz/du, lz, dlz/du
    const int h = blockIdx.y;
    const int base = blockIdx.x * INV_THREADS;
    const float2 *dj = djall + (size_t)h * NT_FWD;
    for (int i = threadIdx.x; i < NT_FWD; i += INV_THREADS) sdk[i] = dj[i].x;
    __syncthreads();
    const double *th = p.theta + 12 * h;
    const double *fwd = p.fwd[h];
    const double cH = C_KMS / th[0], Om = th[1];
    const double dtop = c.d_top;
    const F2 l2e{L2E_HI, L2E_LO};
    for (int t = threadIdx.x; t <= INV_THREADS; t += INV_THREADS) {
        const int k = base + t;
        if (k > NU) break;
        const double u = (double)k / NU, d = dtop * u * u;
        double z = 0.0, dzdu = 0.0;
        if (k > 0) {
            if (!(d <= (double)sdk[NT_FWD - 1])) {
                z = CUDART_NAN;
                dzdu = CUDART_NAN;
            } else {
                // the bracket compares floats with fd, the largest float <= d
                // (x <= d holds for a float x exactly when x <= fd), so the
                // search needs no FP64 conversion per step
                float fd = (float)d;
                if ((double)fd > d) fd = __int_as_float(__float_as_int(fd) - 1);
                int lo = 0, hi = NT_FWD - 1;  // sdk[lo] <= d < sdk[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (sdk[mid] <= fd) lo = mid; else hi = mid;
                }
                // Hermite seed of z(d) between the bracketing nodes in FP32: the
                // node values are FP32, so the seed carries their ~1e-7 error
                // in any precision, and the FP64 Newton step below squares it
                const float dl = sdk[lo], dh = sdk[hi], den = dh - dl;
                const float tt = den > 0.f ? (float)(d - (double)dl) / den : 0.f;
                const float t2 = tt * tt, t3 = t2 * tt;
                const float HTf = (float)HT;  // 10 / 4096, exact in FP32
                z = (double)((2.f * t3 - 3.f * t2 + 1.f) * ((float)lo * HTf) + (t3 - 2.f * t2 + tt) * den / dj[lo].y +
                             (-2.f * t3 + 3.f * t2) * ((float)hi * HTf) + (t3 - t2) * den / dj[hi].y);
                double dd, J;
                chimd::dgw_J_r(z, cH * chimd::dc_hermite_r(fwd, z, Om), th, cH, &dd, &J);
                const double rJ = 1.0 / J;
                const double step = (dd - d) * rJ;
                if (isfinite(step)) z -= step;
                dzdu = 2.0 * u * dtop * rJ;
            }
        }
        const float z32 = (float)z, dzdu32 = (float)dzdu;
        // log2(1+z) and its u-derivative at the node
        const float lzn = mul_f2(l2e, log1pf(z32));
        const float dlz = dzdu32 * L2E_HI / (1.f + z32);
        snd32[t] = make_float4(z32, dzdu32, lzn, dlz);
        if (t < INV_THREADS || k == NU) p.inv64[(size_t)h * (NU + 1) + k] = make_double2(z, dzdu);
    }
    __syncthreads();
    const int k = base + threadIdx.x;
    if (k < NU) {
        const float inv_nu = 1.f / NU;  // exact: NU is a power of two
        const float4 a = snd32[threadIdx.x], b = snd32[threadIdx.x + 1];
        p.inv32[(size_t)h * NU + k] = make_float4(a.x, a.y * inv_nu, b.x, b.y * inv_nu);
        if (p.linv32) p.linv32[(size_t)h * NU + k] = make_float4(a.z, a.w * inv_nu, b.z, b.w * inv_nu);
    }
}

// K1b.3: per-hyperpoint constants (block x = 0, the independent FP64 scalars
// one per lane) and, for mixed calls, F normalised by its maximum.
__global__ void __launch_bounds__(HYP_THREADS) k_hyper_final(DevCatalog c, CallPtrs p,
                                                            const unsigned long long *fmax_bits, bool f64) {
    const int h = blockIdx.y, t = threadIdx.x;
    const double Fm = f64 ? __longlong_as_double((long long)fmax_bits[h])
                          : (double)__uint_as_float((unsigned)fmax_bits[h]);
    // F_scale: the power of two just above the maximum, so that F / F_scale
    // in FP32 is exact (no rounded scale shared by every grid point)
    int fe = 0;
    if (Fm > 0.0) frexp(Fm, &fe);
    const double Fs = Fm > 0.0 ? ldexp(1.0, fe) : 1.0;
    if (!f64) {
        const float iFs = (float)(1.0 / Fs);
        const int a = blockIdx.x * HYP_THREADS + t;
        if (a < c.n_z) p.F32[(size_t)h * c.n_z + a] *= iFs;
    }
    if (blockIdx.x != 0) return;
    // the FP64 scalars, one warp each (lane 0), so that their transcendental
    // chains run side by side instead of serialised by divergence
    __shared__ double sc[20];
    const double *th = p.theta + 12 * h;
    const double alpha = th[4], mu = th[5], sg = th[6], mmin = th[7], mmax = th[8];
    const double lam = c.lambda_g, beta = c.beta;
    const double cH = C_KMS / th[0];
    const int w = t >> 5;
    if ((t & 31) == 0) {
        double v = 0.0;
        switch (w) {
            case 0:
                v = fabs(1.0 - alpha) < 1e-12 ? log(mmax / mmin)
                                              : (pow(mmax, 1.0 - alpha) - pow(mmin, 1.0 - alpha)) / (1.0 - alpha);
                sc[12] = log(v);  // ln of the power law's normalisation integral
                break;
            case 1:
                v = std_normal_cdf((mmax - mu) / sg) - std_normal_cdf((mmin - mu) / sg);
                sc[13] = v > 0.0 ? log(v) : 0.0;
                break;
            case 2:
                v = pow(mmin, 1.0 + beta);
                sc[14] = log(fabs(1.0 + beta) < 1e-12 ? 1.4426950408889634074 : fabs(1.0 + beta));
                break;
            case 3:
                v = chimd::dc_hermite(p.fwd[h], c.z_max, th[1]);
                sc[15] = log(3.0 / (v * v * v));
                break;
            case 4: {  // d_L^gw at the end of the redshift range, z = 10, in FP64
                double J;
                chimd::dgw_J(K_Z10 * HT, cH * p.fwd[h][K_Z10], th, cH, &v, &J);
                sc[8] = sqrt(v / c.d_top) * NU;  // its inverse-table coordinate
                break;
            }
            case 5:
                v = log(mmin);
                sc[9] = log1p(th[11]);
                sc[16] = log(th[0] / C_KMS);
                break;
            case 6:
                v = log2(mmin);
                sc[10] = 1.0 / sg;
                sc[17] = pow(mmin, alpha);
                sc[18] = log(sg);
                break;
            default:
                v = log2(mmax);
                // ln of the constant factor of the mixed path's raw event
                // integral: dz F_scale / (N_gal,tot sqrt(2 pi)), times 1/b per event
                // (the mixed F32 holds F c / H0 unless the Jacobian sits on the samples)
                sc[11] = log(c.dz * Fs / (c.n_gal_total * 2.50662827463100050242)) +
                         (p.jac_ps ? 0.0 : log(th[0] / C_KMS));
                break;
        }
        sc[w] = v;
    }
    __syncthreads();
    if (t == 0) {
        HP hp;
        for (int k = 0; k < 12; k++) hp.th[k] = th[k];
        hp.cH = cH;
        const double plint = sc[0], den = sc[1];
        hp.c_pl = (1.0 - lam) / plint;
        hp.c_g = den > 0.0 ? lam / (sg * 2.50662827463100050242 * den) : 0.0;
        hp.b1 = 1.0 + beta;
        hp.mmin_b1 = sc[2];
        hp.lmmin = sc[5];
        hp.dc_zmax = cH * sc[3];
        hp.d_valid = sc[4];
        hp.F_scale = Fs;
        const double tv = sc[8];
        hp.t_valid = tv;
        if (!(tv < NU)) {
            hp.k_valid = NU;
            hp.f_valid = 0.f;
        } else {
            hp.k_valid = (int)floor(tv);
            hp.f_valid = (float)(tv - hp.k_valid);
        }
        // the mixed path's mass model relative to its shared normalisation
        // (the logs come from the warps above; only sums and products here)
        const bool logp2 = fabs(hp.b1) < 1e-12;
        const bool use_pl = hp.c_pl > 0.0;
        double C1 = use_pl ? hp.c_pl : hp.c_g;
        double lnC1 = use_pl ? c.ln1m_lambda - sc[12]
                             : c.ln_lambda - sc[18] - 0.91893853320467274178 - sc[13];  // ln(lam / (sg sqrt(2 pi) den))
        if (!(C1 > 0.0)) { C1 = 1.0; lnC1 = 0.0; }
        const double mmin_a = sc[17];  // m_min^alpha
        const double wscale = C1 / (mmin_a * mmin) * (logp2 ? 1.4426950408889634074 : fabs(hp.b1));
        hp.ln_wscale = lnC1 - alpha * sc[5] - sc[5] + sc[14];
        hp.inv_wscale = 1.0 / wscale;
        hp.ln_k0 = sc[11] + hp.ln_wscale;
        // s_j = w_scale (3 / Dhat(z_max)^3) (H0 / c) x the mixed selection
        // kernel's relative term (Dhat = D_c H0 / c)
        hp.ln_sel = hp.ln_wscale + sc[15] + sc[16];
        hp.sel_cfac = exp(hp.ln_sel + c.ln_ipi_shift);
        hp.r_pl32 = (float)(hp.c_pl / C1);
        hp.r_g32 = (float)(hp.c_g / C1 * mmin_a);
        hp.na2 = split_f2(-alpha);
        hp.gk2 = split_f2(-0.72134752044448170368 / (sg * sg));
        hp.beta2 = split_f2(beta);
        hp.b1_2 = split_f2(hp.b1);
        hp.l2min2 = split_f2(sc[6]);
        hp.l2max2 = split_f2(sc[7]);
        hp.b1ln2_2 = split_f2(hp.b1 * 0.69314718055994530942);
        hp.kH2 = split_f2(th[0] / C_KMS);
        hp.xi0_2 = split_f2(th[2]);
        hp.omx2 = split_f2(1.0 - th[2]);
        hp.nn2 = split_f2(-th[3]);
        hp.nomx2 = split_f2(th[3] * (1.0 - th[2]));
        hp.om2 = split_f2(th[1]);
        hp.omc2 = split_f2(1.0 - th[1]);
        hp.gam2 = split_f2(th[9]);
        hp.gk_psi2 = split_f2(th[9] + th[10]);
        hp.l2zp2 = split_f2(sc[9] * 1.4426950408889634074);
        hp.status = p.status[h];
        hp.c_pl32 = (float)hp.c_pl;
        hp.c_g32 = (float)hp.c_g;
        hp.alpha32 = (float)alpha;
        hp.mu32 = (float)mu;
        hp.inv_sg32 = (float)sc[10];
        hp.mmin32 = (float)mmin;
        hp.mmax32 = (float)mmax;
        hp.beta32 = (float)beta;
        hp.b1_32 = (float)hp.b1;
        hp.mmin_b1_32 = (float)hp.mmin_b1;
        hp.lmmin32 = (float)hp.lmmin;
        hp.xi0_32 = (float)th[2];
        hp.n32 = (float)th[3];
        hp.om32 = (float)th[1];
        hp.gam32 = (float)th[9];
        hp.kap32 = (float)th[10];
        hp.l1zp32 = (float)sc[9];
        hp.cH32 = (float)cH;
        hp.inv_dc3_32 = (float)(1.0 / (hp.dc_zmax * hp.dc_zmax * hp.dc_zmax));
        hp.l2min32 = (float)sc[6];
        hp.l2max32 = (float)sc[7];
        hp.h0_32 = (float)th[0];
        hp.zp32 = (float)th[11];
        p.hp[h] = hp;
    }
}

}  // namespace

void launch_fwd_tables(const FwdBatch &b, bool dOm, cudaStream_t st) {
    if (b.n <= 0) return;
    if (dOm) k_fwd_panels<1><<<dim3(FWD_BLOCKS, b.n), FWD_THREADS, 0, st>>>(b);
    else k_fwd_panels<0><<<dim3(FWD_BLOCKS, b.n), FWD_THREADS, 0, st>>>(b);
    k_fwd_offsets<<<b.n, 1024, 0, st>>>(b);
}

void launch_fwd_table(double Om, double *out, cudaStream_t st) {
    FwdBatch b{};
    b.n = 1;
    b.Om[0] = Om;
    b.out[0] = out;
    launch_fwd_tables(b, false, st);
}

cudaError_t launch_hyper_tables(const DevCatalog &c, const CallPtrs &p, int H, bool fp64, double *dk,
                                unsigned long long *fmax_bits, cudaStream_t st, cudaStream_t side,
                                cudaEvent_t ev_fork, cudaEvent_t ev_join) {
    float2 *dj = reinterpret_cast<float2 *>(dk);  // (d, J) of the forward nodes, FP32
    cudaError_t e = cudaMemsetAsync(fmax_bits, 0, sizeof(unsigned long long) * H, st);
    if (e != cudaSuccess) return e;
    const int nbn = (NT_FWD + HYP_THREADS - 1) / HYP_THREADS;
    const int nbg = (c.n_z + HYP_THREADS - 1) / HYP_THREADS;
    k_nodes_grid<<<dim3(nbn + nbg, H), HYP_THREADS, 0, st>>>(c, p, dj, fmax_bits, nbn, fp64);
    const dim3 gi((NU + INV_THREADS - 1) / INV_THREADS, H);
    const dim3 gf(fp64 ? 1 : nbg, H);
    if (side) {
        // k_hyper_final needs only the grid factor's maximum and the
        // forward tables, not the inverse nodes: its per-point FP64 chains
        // (a few threads each, latency-bound on B300's FP64 pipe) run on the
        // side stream beside k_inv_nodes
        if ((e = cudaEventRecord(ev_fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side, ev_fork, 0)) != cudaSuccess) return e;
        k_hyper_final<<<gf, HYP_THREADS, 0, side>>>(c, p, fmax_bits, fp64);
        if ((e = cudaEventRecord(ev_join, side)) != cudaSuccess) return e;
        k_inv_nodes<<<gi, INV_THREADS, 0, st>>>(c, p, dj);
        return cudaStreamWaitEvent(st, ev_join, 0);
    }
    k_inv_nodes<<<gi, INV_THREADS, 0, st>>>(c, p, dj);
    k_hyper_final<<<gf, HYP_THREADS, 0, st>>>(c, p, fmax_bits, fp64);
    return cudaSuccess;
}

void launch_hyper_tables(const DevCatalog &c, const CallPtrs &p, int H, bool fp64, double *dk,
                         unsigned long long *fmax_bits, cudaStream_t st) {
    launch_hyper_tables(c, p, H, fp64, dk, fmax_bits, st, nullptr, nullptr, nullptr);
}

}  // namespace chim
