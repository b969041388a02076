// K1: cosmology tables (Eqs. dL-em, dL-mg, jacobian; Sec. 2.1).
//
// k_fwd_table  - per distinct Om: cumulative D_c(z_k)/(c/H0) on the forward
//                grid z_k = k*HT by 5-point Gauss-Legendre panels and a block
//                prefix sum, all in FP64.
// k_fwd_nodes, k_inv_nodes, k_grid, k_hyper_final - per hyperpoint, each
//                spread over (nodes x hyperpoints) so that the FP64 work uses
//                every SM: d_L^gw and J on the forward nodes (monotonicity
//                check on z <= 10), the inverse table z(u), u = sqrt(d_L/d_top),
//                by Newton on the Hermite-interpolated forward relation, the
//                grid factor F(z_a) = psi(z_a) / [(1+z_a)^3 |J(z_a)|] of
//                Eq. like-integrals, and the mass-model normalisations.
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

constexpr int HYP_THREADS = 256;

__device__ double std_normal_cdf(double x) { return 0.5 * erfc(-x * 0.70710678118654752440); }

// K1b.1: d_L^gw and J at the forward nodes of every hyperpoint; J <= 0 on
// z <= 10 sets the NONMONOTONE bit.
__global__ void __launch_bounds__(HYP_THREADS) k_fwd_nodes(CallPtrs p, double *dk, double *jk) {
    const int h = blockIdx.y;
    const int k = blockIdx.x * HYP_THREADS + threadIdx.x;
    if (k >= NT_FWD) return;
    const double *th = p.theta + 12 * h;
    const double cH = C_KMS / th[0];
    double d, J;
    chimd::dgw_J(k * HT, cH * p.fwd[h][k], th, cH, &d, &J);
    dk[(size_t)h * NT_FWD + k] = d;
    jk[(size_t)h * NT_FWD + k] = J;
    if (k <= K_Z10 && !(J > 0.0)) atomicOr(p.status + h, CHIMERA_PT_NONMONOTONE);
}

// K1b.2: inverse nodes z(u_k), d = d_top u_k^2: bracketing on the forward
// nodes (staged in shared memory), cubic Hermite of z(d) between the two
// bracketing nodes (slopes 1/J), then one Newton step on the
// Hermite-interpolated forward relation.
__global__ void __launch_bounds__(HYP_THREADS) k_inv_nodes(DevCatalog c, CallPtrs p, const double *dkall,
                                                          const double *jkall) {
    __shared__ double sdk[NT_FWD];
    const int h = blockIdx.y;
    const int k = blockIdx.x * HYP_THREADS + threadIdx.x;
    const double *dk = dkall + (size_t)h * NT_FWD;
    const double *jk = jkall + (size_t)h * NT_FWD;
    for (int i = threadIdx.x; i < NT_FWD; i += HYP_THREADS) sdk[i] = dk[i];
    __syncthreads();
    if (k > NU) return;
    const double *th = p.theta + 12 * h;
    const double *fwd = p.fwd[h];
    const double cH = C_KMS / th[0], Om = th[1];
    const double dtop = c.d_top;
    double u = (double)k / NU, d = dtop * u * u;
    double z = 0.0, dzdu = 0.0;
    if (k > 0) {
        if (!(d <= sdk[NT_FWD - 1])) {
            z = CUDART_NAN;
            dzdu = CUDART_NAN;
        } else {
            int lo = 0, hi = NT_FWD - 1;  // sdk[lo] <= d < sdk[hi]
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (sdk[mid] <= d) lo = mid; else hi = mid;
            }
            const double dl = sdk[lo], dh = sdk[hi], den = dh - dl;
            const double t = den > 0.0 ? (d - dl) / den : 0.0;
            const double t2 = t * t, t3 = t2 * t;
            z = (2 * t3 - 3 * t2 + 1) * (lo * HT) + (t3 - 2 * t2 + t) * den / jk[lo] +
                (-2 * t3 + 3 * t2) * (hi * HT) + (t3 - t2) * den / jk[hi];
            double dd, J;
            chimd::dgw_J(z, cH * chimd::dc_hermite(fwd, z, Om), th, cH, &dd, &J);
            const double step = (dd - d) / J;
            if (isfinite(step)) z -= step;
            dzdu = 2.0 * u * dtop / J;
        }
    }
    p.inv64[(size_t)h * (NU + 1) + k] = make_double2(z, dzdu);
}

// K1b.3: grid factor F(z_a) = psi / ((1+z)^3 |J|) and its maximum.
__global__ void __launch_bounds__(HYP_THREADS) k_grid(DevCatalog c, CallPtrs p, unsigned long long *fmax_bits) {
    const int h = blockIdx.y;
    const int a = blockIdx.x * HYP_THREADS + threadIdx.x;
    double F = 0.0;
    if (a < c.n_z) {
        const double *th = p.theta + 12 * h;
        const double cH = C_KMS / th[0];
        double z = a * c.dz, d, J;
        chimd::dgw_J(z, cH * chimd::dc_hermite(p.fwd[h], z, th[1]), th, cH, &d, &J);
        double ap = 1.0 + z;
        F = chimd::psi_of(z, th) / (ap * ap * ap * fabs(J));
        if (!isfinite(F)) F = 0.0;
        p.F64[(size_t)h * c.n_z + a] = F;
    }
    for (int o = 16; o > 0; o >>= 1) F = fmax(F, __shfl_xor_sync(0xffffffffu, F, o));
    // F >= 0, so the ordering of the bit patterns is the ordering of the values
    if ((threadIdx.x & 31) == 0 && F > 0.0) atomicMax(fmax_bits + h, (unsigned long long)__double_as_longlong(F));
}

// K1b.4: per-hyperpoint constants, FP32 inverse intervals, normalised F.
__global__ void __launch_bounds__(HYP_THREADS) k_hyper_final(DevCatalog c, CallPtrs p,
                                                            const double *dkall,
                                                            const unsigned long long *fmax_bits) {
    const int h = blockIdx.x, t = threadIdx.x;
    const double Fm = __longlong_as_double((long long)fmax_bits[h]);
    const double Fs = Fm > 0.0 ? Fm : 1.0;
    const double2 *nd = p.inv64 + (size_t)h * (NU + 1);
    __shared__ double sc[8];
    const double inv_nu = 1.0 / NU;  // exact: NU is a power of two
    for (int k = t; k < NU; k += HYP_THREADS) {
        double2 a = nd[k], b = nd[k + 1];
        p.inv32[(size_t)h * NU + k] =
            make_float4((float)a.x, (float)(a.y * inv_nu), (float)b.x, (float)(b.y * inv_nu));
    }
    const double iFs = 1.0 / Fs;
    for (int a = t; a < c.n_z; a += HYP_THREADS)
        p.F32[(size_t)h * c.n_z + a] = (float)(p.F64[(size_t)h * c.n_z + a] * iFs);
    const double *th = p.theta + 12 * h;
    const double alpha = th[4], mu = th[5], sg = th[6], mmin = th[7], mmax = th[8];
    const double lam = c.lambda_g, beta = c.beta;
    // the independent FP64 scalars, one per lane of warp 0
    if (t < 4) {
        double v = 0.0;
        if (t == 0)
            v = fabs(1.0 - alpha) < 1e-12 ? log(mmax / mmin)
                                          : (pow(mmax, 1.0 - alpha) - pow(mmin, 1.0 - alpha)) / (1.0 - alpha);
        else if (t == 1)
            v = std_normal_cdf((mmax - mu) / sg) - std_normal_cdf((mmin - mu) / sg);
        else if (t == 2)
            v = pow(mmin, 1.0 + beta);
        else
            v = chimd::dc_hermite(p.fwd[h], c.z_max, th[1]);
        sc[t] = v;
    }
    __syncthreads();
    if (t == 0) {
        HP hp;
        for (int k = 0; k < 12; k++) hp.th[k] = th[k];
        const double cH = C_KMS / th[0];
        hp.cH = cH;
        const double plint = sc[0], den = sc[1];
        hp.c_pl = (1.0 - lam) / plint;
        hp.c_g = den > 0.0 ? lam / (sg * 2.50662827463100050242 * den) : 0.0;
        hp.b1 = 1.0 + beta;
        hp.mmin_b1 = sc[2];
        hp.lmmin = log(mmin);
        hp.dc_zmax = cH * sc[3];
        hp.d_valid = dkall[(size_t)h * NT_FWD + K_Z10];
        hp.F_scale = Fs;
        double tv = sqrt(hp.d_valid / c.d_top) * NU;
        hp.t_valid = tv;
        if (!(tv < NU)) {
            hp.k_valid = NU;
            hp.f_valid = 0.f;
        } else {
            hp.k_valid = (int)floor(tv);
            hp.f_valid = (float)(tv - hp.k_valid);
        }
        hp.status = p.status[h];
        hp.c_pl32 = (float)hp.c_pl;
        hp.c_g32 = (float)hp.c_g;
        hp.alpha32 = (float)alpha;
        hp.mu32 = (float)mu;
        hp.inv_sg32 = (float)(1.0 / sg);
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
        hp.l1zp32 = (float)log1p(th[11]);
        hp.cH32 = (float)cH;
        hp.inv_dc3_32 = (float)(1.0 / (hp.dc_zmax * hp.dc_zmax * hp.dc_zmax));
        hp.l2min32 = (float)log2(mmin);
        hp.l2max32 = (float)log2(mmax);
        p.hp[h] = hp;
    }
}

}  // namespace

void launch_fwd_table(double Om, double *out, cudaStream_t st) {
    k_fwd_table<<<1, FWD_THREADS, 0, st>>>(Om, out);
}

void launch_hyper_tables(const DevCatalog &c, const CallPtrs &p, int H, double *dk,
                         unsigned long long *fmax_bits, cudaStream_t st) {
    cudaMemsetAsync(fmax_bits, 0, sizeof(unsigned long long) * H, st);
    double *jk = dk + (size_t)H * NT_FWD;  // J at the forward nodes
    k_fwd_nodes<<<dim3((NT_FWD + HYP_THREADS - 1) / HYP_THREADS, H), HYP_THREADS, 0, st>>>(p, dk, jk);
    k_inv_nodes<<<dim3((NU + 1 + HYP_THREADS - 1) / HYP_THREADS, H), HYP_THREADS, 0, st>>>(c, p, dk, jk);
    k_grid<<<dim3((c.n_z + HYP_THREADS - 1) / HYP_THREADS, H), HYP_THREADS, 0, st>>>(c, p, fmax_bits);
    k_hyper_final<<<H, HYP_THREADS, 0, st>>>(c, p, dk, fmax_bits);
}

}  // namespace chim
