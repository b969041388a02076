// K4, the "3D" kernel (Sec. 2.3), FP64: see k_event_3d.
#include <math_constants.h>

#include "internal.cuh"
#include "mass.cuh"

namespace chim {

namespace {

__device__ __forceinline__ double warp_sumd3(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of NV doubles per thread in a fixed order; result in
// red[0..NV-1] (red holds 8 + warps x NV doubles), seen by all threads.
template <int NV, int NT>
__device__ void block_sumd(double (&v)[NV], double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; q++) {
        double s = warp_sumd3(v[q]);
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

// The "3D" kernel (Sec. 2.3, catalogs of kde_mode CHIMERA_KDE_3D), FP64, a
// cross-check variant: a weighted Gaussian KDE over (z, x, y) ((x, y) the
// event's flat sky chart) with the bandwidth matrix H = n_eff^(-2/7) x the
// weighted covariance (unbiased weighting; the plain covariance with
// n = valid samples if that one is degenerate), evaluated at (z_a, pixel
// centre).  Here the Gaussian is split into a sky factor and a conditional
// Gaussian in z,
//   N3 = N2(ds; H_ss) N1(z_a; z_j + c.ds, b_c^2),
//   c = H_zs H_ss^-1, b_c^2 = H_zz - c H_sz, ds = pixel centre - (x_j, y_j),
// so that each (pixel, sample) pair is a 1-D kernel of width b_c on a window
// of +-KW64 b_c (and sky factors below exp(-KW64^2) are skipped), the
// Gaussian along the window by a two-multiplication recurrence.  One block
// per (event, point); the samples are in d_L order, so the valid ones (z
// exists) are a prefix.
__global__ void __launch_bounds__(EV64_THREADS) k_event_3d(DevCatalog c, CallPtrs p, int H) {
    extern __shared__ double sd[];
    double *zs = sd;
    double *ws = zs + c.max_ns;
    double *red = ws + c.max_ns;
    __shared__ double kc[10];  // Hss^-1 (3), c (2), b_c, norm, zlo, zhi, ok
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
    const double2 *xy = c.sky_xy + s0;
    // pass 1: z, w and first moments (weighted and plain)
    double m1[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // W1, W2, Wz, Wx, Wy, n, Sz, Sx (Sy below)
    double sy = 0.0;
    for (int j = tid; j < ns; j += EV64_THREADS) {
        double z = 0.0, w = 0.0;
        if (invert64(c, p, h, hp, c.sd64[s0 + j], &z)) {
            const double m1s = c.sm1_64[s0 + j] / (1.0 + z), m2s = c.sm2_64[s0 + j] / (1.0 + z);
            w = mass_weight64(hp, c.beta, m1s, m2s);
            const double2 v = xy[j];
            m1[0] += w; m1[1] += w * w; m1[2] += w * z; m1[3] += w * v.x; m1[4] += w * v.y;
            m1[5] += 1.0; m1[6] += z; m1[7] += v.x; sy += v.y;
        } else {
            z = CUDART_INF;
        }
        zs[j] = z;
        ws[j] = w;
    }
    block_sumd<8, EV64_THREADS>(m1, red);
    const double W1 = red[0], W2 = red[1], nv = red[5];
    const double mw[3] = {W1 > 0.0 ? red[2] / W1 : 0.0, W1 > 0.0 ? red[3] / W1 : 0.0, W1 > 0.0 ? red[4] / W1 : 0.0};
    const double mzu = nv > 0.0 ? red[6] / nv : 0.0, mxu = nv > 0.0 ? red[7] / nv : 0.0;
    __syncthreads();
    {
        double t[1] = {sy};
        block_sumd<1, EV64_THREADS>(t, red);
    }
    const double myu = nv > 0.0 ? red[0] / nv : 0.0;
    __syncthreads();
    // pass 2: centred second moments, weighted (6) and plain (6)
    double m2[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = tid; j < ns; j += EV64_THREADS) {
        const double z = zs[j];
        if (!(z < CUDART_INF)) continue;
        const double w = ws[j];
        const double2 v = xy[j];
        const double a[3] = {z - mw[0], v.x - mw[1], v.y - mw[2]};
        const double u[3] = {z - mzu, v.x - mxu, v.y - myu};
        m2[0] += w * a[0] * a[0]; m2[1] += w * a[0] * a[1]; m2[2] += w * a[0] * a[2];
        m2[3] += w * a[1] * a[1]; m2[4] += w * a[1] * a[2]; m2[5] += w * a[2] * a[2];
        m2[6] += u[0] * u[0]; m2[7] += u[0] * u[1]; m2[8] += u[0] * u[2];
        m2[9] += u[1] * u[1]; m2[10] += u[1] * u[2]; m2[11] += u[2] * u[2];
    }
    block_sumd<12, EV64_THREADS>(m2, red);
    if (tid == 0) {
        // H = Scott factor^2 x covariance (entries zz, zx, zy, xx, xy, yy)
        double Hm[6];
        bool ok = false;
        auto det3 = [](const double *C) {
            return C[0] * (C[3] * C[5] - C[4] * C[4]) - C[1] * (C[1] * C[5] - C[4] * C[2]) +
                   C[2] * (C[1] * C[4] - C[3] * C[2]);
        };
        if (W1 > 0.0 && W1 * W1 / W2 >= 2.0) {
            const double fact = W1 - W2 / W1;
            double C[6];
            for (int r = 0; r < 6; r++) C[r] = fact > 0.0 ? red[r] / fact : 0.0;
            if (det3(C) > 0.0) {
                const double f2 = pow(W1 * W1 / W2, -2.0 / 7.0);
                for (int r = 0; r < 6; r++) Hm[r] = f2 * C[r];
                ok = true;
            }
        }
        if (!ok && nv >= 4.0) {
            double C[6];
            for (int r = 0; r < 6; r++) C[r] = red[6 + r] / (nv - 1.0);
            if (det3(C) > 0.0) {
                const double f2 = pow(nv, -2.0 / 7.0);
                for (int r = 0; r < 6; r++) Hm[r] = f2 * C[r];
                ok = true;
            }
        }
        kc[9] = ok ? 1.0 : 0.0;
        if (ok) {
            const double dets = Hm[3] * Hm[5] - Hm[4] * Hm[4];
            const double i00 = Hm[5] / dets, i01 = -Hm[4] / dets, i11 = Hm[3] / dets;
            const double cx = Hm[1] * i00 + Hm[2] * i01, cy = Hm[1] * i01 + Hm[2] * i11;
            const double bc2 = Hm[0] - (cx * Hm[1] + cy * Hm[2]);
            const int nvi = (int)nv;
            kc[0] = i00; kc[1] = i01; kc[2] = i11; kc[3] = cx; kc[4] = cy;
            kc[5] = bc2 > 0.0 ? sqrt(bc2) : 0.0;
            // (2 pi)^(-3/2) / (sqrt(det H_ss) b_c N)
            kc[6] = 0.063493635934240969785 / (sqrt(dets) * kc[5] * (double)ns);
            kc[7] = zs[0] - KDE_MARGIN * sqrt(Hm[0]);
            kc[8] = zs[nvi - 1] + KDE_MARGIN * sqrt(Hm[0]);
            if (!(kc[5] > 0.0)) kc[9] = 0.0;
            p.bw[out] = sqrt(Hm[0]);
        } else {
            p.bw[out] = 0.0;
        }
    }
    __syncthreads();
    if (kc[9] == 0.0) {  // degenerate sample covariance: no 3D kernel
        if (tid == 0) p.lnI[out] = -CUDART_INF;
        return;
    }
    const double i00 = kc[0], i01 = kc[1], i11 = kc[2], cx = kc[3], cy = kc[4], bc = kc[5];
    const double zlo = kc[7], zhi = kc[8];
    const double dlt = c.dz / bc, qq = exp(-dlt * dlt);
    const int nz = c.n_z, nvi = (int)nv;
    const double dz = c.dz;
    const double *F = p.F64 + (size_t)h * nz;
    const double *prof = reinterpret_cast<const double *>(p.prof[h]);
    const int64_t p0 = c.ev_poff[ev], np = c.ev_poff[ev + 1] - p0;
    const bool jac = p.jac_ps != 0;
    double tsum = 0.0;
    for (int64_t k = 0; k < np; k++) {
        const double2 P = c.pix_xy[p0 + k];
        const double *G = prof + (p0 + k) * nz;
        for (int j = tid; j < nvi; j += EV64_THREADS) {
            double w = ws[j];
            if (w == 0.0) continue;
            const double2 v = xy[j];
            const double dx = P.x - v.x, dy = P.y - v.y;
            const double q = dx * (i00 * dx + i01 * dy) + dy * (i01 * dx + i11 * dy);
            if (q > 2.0 * KW64 * KW64) continue;
            const double z = zs[j];
            if (jac) {  // the Jacobian on the sample (Eq. jacobian), after the bandwidth
                double dd, J;
                chimd::dgw_J(z, hp.cH * chimd::dc_hermite(p.fwd[h], z, hp.th[1]), hp.th, hp.cH, &dd, &J);
                const double ap = 1.0 + z;
                w /= ap * ap * ap * fabs(J);
            }
            const double mu = z + cx * dx + cy * dy;
            const double a0 = fmax(ceil((mu - KW64 * bc) / dz), ceil(zlo / dz));
            const double a1 = fmin(floor((mu + KW64 * bc) / dz), floor(zhi / dz));
            const int ia0 = a0 < 0.0 ? 0 : (a0 > nz ? nz : (int)a0);
            const int ia1 = a1 > nz - 1 ? nz - 1 : (a1 < -1.0 ? -1 : (int)a1);
            // exp(-x^2/2) along the window by the Gaussian recurrence
            // g_{a+1} = g_a r_a, r_{a+1} = r_a e^{-delta^2} (x steps by
            // delta = dz / b_c; relative drift ~1e-14 over a window)
            double s = 0.0;
            if (ia0 <= ia1) {
                const double x0 = (ia0 * dz - mu) / bc;
                double g = exp(-0.5 * x0 * x0), r = exp(-x0 * dlt - 0.5 * dlt * dlt);
                for (int a = ia0; a <= ia1; a++) {
                    const double wa = (a == 0 || a == nz - 1) ? 0.5 : 1.0;
                    s += g * wa * F[a] * G[a];
                    g *= r;
                    r *= qq;
                }
            }
            tsum += w * exp(-0.5 * q) * s;
        }
    }
    {
        double v[1] = {tsum};
        __syncthreads();
        block_sumd<1, EV64_THREADS>(v, red);
    }
    if (tid == 0) {
        const double I = red[0] * dz * kc[6] / c.n_gal_total;
        p.lnI[out] = I > 0.0 ? log(I) : -CUDART_INF;
    }
}


}  // namespace

size_t event_3d_smem(const DevCatalog &c) {
    return sizeof(double) * 2 * (size_t)c.max_ns + sizeof(double) * (8 + (EV64_THREADS / 32) * 12);
}

void launch_event_3d(const DevCatalog &c, const CallPtrs &p, int H, cudaStream_t st) {
    size_t smem = event_3d_smem(c);
    cudaFuncSetAttribute(k_event_3d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_event_3d<<<(unsigned)(c.n_events * H), EV64_THREADS, smem, st>>>(c, p, H);
}

}  // namespace chim
