// K1: cosmology tables (Eqs. dL-em, dL-mg, jacobian; Sec. 2.1).
//
// k_fwd_table  - per distinct Om: cumulative D_c(z_k)/(c/H0) on the forward
//                grid z_k = k*HT by 5-point Gauss-Legendre panels and a block
//                prefix sum, all in FP64.
// k_hyper      - per hyperpoint: mass-model normalisations, d_L^gw and J on
//                the forward nodes (monotonicity check on z <= 10), the
//                inverse table z(u), u = sqrt(d_L / d_top), by Newton on the
//                Hermite-interpolated forward relation, and the grid factor
//                F(z_a) = psi(z_a) / [(1+z_a)^3 |J(z_a)|] of Eq. like-integrals.
#include <math_constants.h>

#include "internal.cuh"

namespace chim {

namespace {

constexpr int FWD_THREADS = 512;
constexpr int FWD_PER_THREAD = 10;
static_assert(FWD_THREADS * FWD_PER_THREAD >= NT_FWD - 1, "forward table coverage");

__global__ void __launch_bounds__(FWD_THREADS) k_fwd_table(double Om, double *out) {
    __shared__ double warp_tot[FWD_THREADS / 32];
    const int t = threadIdx.x;
    // 5-point Gauss-Legendre nodes and weights in closed form.
    const double x1 = sqrt(5.0 - 2.0 * sqrt(10.0 / 7.0)) / 3.0;
    const double x2 = sqrt(5.0 + 2.0 * sqrt(10.0 / 7.0)) / 3.0;
    const double w0 = 128.0 / 225.0;
    const double w1 = (322.0 + 13.0 * sqrt(70.0)) / 900.0;
    const double w2 = (322.0 - 13.0 * sqrt(70.0)) / 900.0;
    double loc[FWD_PER_THREAD];
    double run = 0.0;
#pragma unroll
    for (int c = 0; c < FWD_PER_THREAD; c++) {
        int k = t * FWD_PER_THREAD + c;
        if (k < NT_FWD - 1) {
            double m = (k + 0.5) * HT, hh = 0.5 * HT;
            double s = w0 / chimd::E_of(m, Om) +
                       w1 * (1.0 / chimd::E_of(m - hh * x1, Om) + 1.0 / chimd::E_of(m + hh * x1, Om)) +
                       w2 * (1.0 / chimd::E_of(m - hh * x2, Om) + 1.0 / chimd::E_of(m + hh * x2, Om));
            run += s * hh;
        }
        loc[c] = run;
    }
    // block exclusive scan of the per-thread totals
    const int lane = t & 31, wid = t >> 5;
    double v = run;
    for (int o = 1; o < 32; o <<= 1) {
        double y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double x = lane < FWD_THREADS / 32 ? warp_tot[lane] : 0.0;
        for (int o = 1; o < 32; o <<= 1) {
            double y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < FWD_THREADS / 32) warp_tot[lane] = x;
    }
    __syncthreads();
    double offset = (v - run) + (wid > 0 ? warp_tot[wid - 1] : 0.0);
#pragma unroll
    for (int c = 0; c < FWD_PER_THREAD; c++) {
        int k = t * FWD_PER_THREAD + c;
        if (k < NT_FWD - 1) out[k + 1] = offset + loc[c];
    }
    if (t == 0) out[0] = 0.0;
}

constexpr int HYP_THREADS = 512;

__device__ double std_normal_cdf(double x) { return 0.5 * erfc(-x * 0.70710678118654752440); }

__global__ void __launch_bounds__(HYP_THREADS) k_hyper(DevCatalog c, CallPtrs p, int H) {
    extern __shared__ double sh[];
    double *dk = sh;                  // [NT_FWD] d_L^gw at the forward nodes
    double *Jk = dk + NT_FWD;         // [NT_FWD] its derivative
    double2 *nodes = (double2 *)(Jk + NT_FWD);  // [NU+1]
    __shared__ double th[12];
    __shared__ int s_nonmono;
    __shared__ double s_fmax[HYP_THREADS / 32];
    const int h = blockIdx.x, t = threadIdx.x;
    if (t < 12) th[t] = p.theta[h * 12 + t];
    if (t == 0) s_nonmono = 0;
    __syncthreads();
    const double *fwd = p.fwd[h];
    const double H0 = th[0], Om = th[1];
    const double cH = C_KMS / H0;

    // forward relation at the nodes; J <= 0 on z <= 10 flags non-monotonicity
    for (int k = t; k < NT_FWD; k += HYP_THREADS) {
        double z = k * HT, d, J;
        chimd::dgw_J(z, cH * fwd[k], th, cH, &d, &J);
        dk[k] = d;
        Jk[k] = J;
        if (k <= K_Z10 && !(J > 0.0)) s_nonmono = 1;
    }
    __syncthreads();

    // inverse nodes z(u_k), d = d_top u_k^2
    const double dtop = c.d_top;
    for (int k = t; k <= NU; k += HYP_THREADS) {
        double u = (double)k / NU, d = dtop * u * u;
        double z = 0.0, dzdu = 0.0;
        if (k > 0) {
            if (!(d <= dk[NT_FWD - 1])) {
                z = CUDART_NAN;
                dzdu = CUDART_NAN;
            } else {
                int lo = 0, hi = NT_FWD - 1;  // dk[lo] <= d < dk[hi]
                while (hi - lo > 1) {
                    int mid = (lo + hi) >> 1;
                    if (dk[mid] <= d) lo = mid; else hi = mid;
                }
                double den = dk[hi] - dk[lo];
                double fr = den > 0.0 ? (d - dk[lo]) / den : 0.0;
                z = (lo + fr) * HT;
                double dd, J;
                for (int it = 0; it < 3; it++) {
                    chimd::dgw_J(z, cH * chimd::dc_hermite(fwd, z, Om), th, cH, &dd, &J);
                    double step = (dd - d) / J;
                    if (isfinite(step)) z -= step;
                }
                chimd::dgw_J(z, cH * chimd::dc_hermite(fwd, z, Om), th, cH, &dd, &J);
                dzdu = 2.0 * u * dtop / J;
            }
        }
        nodes[k] = make_double2(z, dzdu);
        p.inv64[(size_t)h * (NU + 1) + k] = make_double2(z, dzdu);
    }
    __syncthreads();
    for (int k = t; k < NU; k += HYP_THREADS) {
        double2 a = nodes[k], b = nodes[k + 1];
        p.inv32[(size_t)h * NU + k] =
            make_float4((float)a.x, (float)(a.y / NU), (float)b.x, (float)(b.y / NU));
    }

    // grid factor F(z_a) = psi / ((1+z)^3 |J|)
    double fm = 0.0;
    const int nz = c.n_z;
    for (int a = t; a < nz; a += HYP_THREADS) {
        double z = a * c.dz, d, J;
        chimd::dgw_J(z, cH * chimd::dc_hermite(fwd, z, Om), th, cH, &d, &J);
        double ap = 1.0 + z;
        double F = chimd::psi_of(z, th) / (ap * ap * ap * fabs(J));
        if (!isfinite(F)) F = 0.0;
        p.F64[(size_t)h * nz + a] = F;
        fm = fm > F ? fm : F;
    }
    for (int o = 16; o > 0; o >>= 1) fm = fmax(fm, __shfl_xor_sync(0xffffffffu, fm, o));
    if ((t & 31) == 0) s_fmax[t >> 5] = fm;
    __syncthreads();
    if (t < 32) {
        double x = t < HYP_THREADS / 32 ? s_fmax[t] : 0.0;
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
        if (t == 0) s_fmax[0] = x;
    }
    __syncthreads();
    const double Fs = s_fmax[0] > 0.0 ? s_fmax[0] : 1.0;
    for (int a = t; a < nz; a += HYP_THREADS)
        p.F32[(size_t)h * nz + a] = (float)(p.F64[(size_t)h * nz + a] / Fs);

    if (t == 0) {
        HP hp;
        for (int k = 0; k < 12; k++) hp.th[k] = th[k];
        hp.cH = cH;
        const double alpha = th[4], mu = th[5], sg = th[6], mmin = th[7], mmax = th[8];
        const double lam = c.lambda_g, beta = c.beta;
        double plint = fabs(1.0 - alpha) < 1e-12
                           ? log(mmax / mmin)
                           : (pow(mmax, 1.0 - alpha) - pow(mmin, 1.0 - alpha)) / (1.0 - alpha);
        double den = std_normal_cdf((mmax - mu) / sg) - std_normal_cdf((mmin - mu) / sg);
        hp.c_pl = (1.0 - lam) / plint;
        hp.c_g = den > 0.0 ? lam / (sg * 2.50662827463100050242 * den) : 0.0;
        hp.b1 = 1.0 + beta;
        hp.mmin_b1 = pow(mmin, 1.0 + beta);
        hp.lmmin = log(mmin);
        hp.dc_zmax = cH * chimd::dc_hermite(fwd, c.z_max, Om);
        hp.d_valid = dk[K_Z10];
        hp.F_scale = Fs;
        double tv = sqrt(hp.d_valid / dtop) * NU;
        hp.t_valid = tv;
        if (!(tv < NU)) {
            hp.k_valid = NU;
            hp.f_valid = 0.f;
        } else {
            hp.k_valid = (int)floor(tv);
            hp.f_valid = (float)(tv - hp.k_valid);
        }
        int st = p.status[h];
        if (s_nonmono) st |= CHIMERA_PT_NONMONOTONE;
        hp.status = st;
        hp.pad = 0.f;
        p.hp[h] = hp;
    }
}

}  // namespace

void launch_fwd_table(double Om, double *out, cudaStream_t st) {
    k_fwd_table<<<1, FWD_THREADS, 0, st>>>(Om, out);
}

void launch_hyper_tables(const DevCatalog &c, const CallPtrs &p, int H, cudaStream_t st) {
    size_t smem = sizeof(double) * 2 * NT_FWD + sizeof(double2) * (NU + 1);
    cudaFuncSetAttribute(k_hyper, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_hyper<<<H, HYP_THREADS, smem, st>>>(c, p, H);
}

}  // namespace chim
