// K3: pixelised galaxy redshift prior on the grid (Eq. p-cat, complete
// catalog), for one Om:
//
//   G_k(z_a) = dV_c/dz(z_a) sum_{g in k} N(z_a; z_g, s_g) / Z_g,
//   Z_g      = sum_a w_a N(z_a; z_g, s_g) dV_c/dz(z_a),
//
// stored as N_gal,tot times the paper's p_cat (the 1/N_gal,tot prefactor is
// applied in the final FP64 log).  The normalisation makes the constant
// factors of dV_c/dz cancel, so dV_c/dz is evaluated as D_c^2 / E.  Each
// galaxy contributes on the grid points within KWG sigma of its redshift,
// in both Z_g and G, so every galaxy keeps unit weight on the grid.
//
// One block per pixel: phase 1 computes 1/Z_g for the pixel's galaxies,
// phase 2 gathers, for each grid point, the galaxies whose window covers it
// (galaxies are sorted by z inside a pixel at load time), so the sums are
// formed in a fixed order without atomics.
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "internal.cuh"

namespace chim {

namespace {

constexpr int GAL_THREADS = 256;

__global__ void k_dvdz(const double *fwd, double Om, double dz, int nz, double *dv) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < nz) {
        double z = a * dz;
        double D = chimd::dc_hermite(fwd, z, Om);
        dv[a] = D * D / chimd::E_of(z, Om);
    }
}

__device__ __forceinline__ float bf16_bits_to_float(uint16_t b) {
    return __uint_as_float(((uint32_t)b) << 16);
}

// Galaxy (z, sigma) as the device stores it for the mixed path.
__device__ __forceinline__ void gal32(const DevCatalog &c, int64_t p, int64_t g, float &z, float &s) {
    if (c.gal_storage == CHIMERA_GAL_F32) {
        z = c.gz32[g];
        s = c.gs32[g];
    } else if (c.gal_storage == CHIMERA_GAL_F16) {
        z = c.pix_zref[p] + __half2float(__ushort_as_half(c.gzq[g]));
        s = __half2float(__ushort_as_half(c.gsq[g]));
    } else {
        z = c.pix_zref[p] + bf16_bits_to_float(c.gzq[g]);
        s = bf16_bits_to_float(c.gsq[g]);
    }
}

__device__ __forceinline__ void window(double zg, double kw, double dz, int nz, int &lo, int &hi) {
    double a0 = ceil((zg - kw) / dz), a1 = floor((zg + kw) / dz);
    lo = a0 < 0.0 ? 0 : (a0 > nz ? nz : (int)a0);
    hi = a1 > nz - 1 ? nz - 1 : (a1 < -1.0 ? -1 : (int)a1);
}

// FP64 profile from the double galaxy values.
__global__ void __launch_bounds__(GAL_THREADS) k_profile64(DevCatalog c, const double *dv,
                                                          double *invZ, double *G) {
    const int64_t p = blockIdx.x;
    const int64_t g0 = c.gal_off[p], g1 = c.gal_off[p + 1];
    const int nz = c.n_z;
    const double dz = c.dz, norm = 0.39894228040143267794;
    for (int64_t g = g0 + threadIdx.x; g < g1; g += GAL_THREADS) {
        double zg = c.gz64[g], sg = c.gs64[g];
        int lo, hi;
        window(zg, KWG64 * sg, dz, nz, lo, hi);
        double Z = 0.0;
        for (int a = lo; a <= hi; a++) {
            double u = (a * dz - zg) / sg;
            double wa = (a == 0 || a == nz - 1) ? 0.5 * dz : dz;
            Z += wa * norm / sg * exp(-0.5 * u * u) * dv[a];
        }
        invZ[g] = Z > 0.0 ? 1.0 / Z : 0.0;
    }
    __syncthreads();
    const double smax = c.pix_sigmax[p] * KWG64;
    for (int a = threadIdx.x; a < nz; a += GAL_THREADS) {
        double za = a * dz, acc = 0.0;
        // first galaxy with z >= za - smax, first with z > za + smax
        int64_t l = g0, r = g1;
        while (l < r) {
            int64_t m = (l + r) >> 1;
            if (c.gz64[m] < za - smax) l = m + 1; else r = m;
        }
        for (int64_t g = l; g < g1; g++) {
            double zg = c.gz64[g];
            if (zg > za + smax) break;
            double sg = c.gs64[g];
            int lo, hi;
            window(zg, KWG64 * sg, dz, nz, lo, hi);
            if (a < lo || a > hi) continue;
            double u = (za - zg) / sg;
            acc += norm / sg * exp(-0.5 * u * u) * invZ[g];
        }
        G[p * nz + a] = acc * dv[a];
    }
}

// Mixed-path profile (FP32 arithmetic) from the stored galaxy values.
__global__ void __launch_bounds__(GAL_THREADS) k_profile32(DevCatalog c, const double *dv,
                                                          float *invZ, float *G) {
    const int64_t p = blockIdx.x;
    const int64_t g0 = c.gal_off[p], g1 = c.gal_off[p + 1];
    const int nz = c.n_z;
    const float dz = (float)c.dz, norm = 0.3989422804f;
    for (int64_t g = g0 + threadIdx.x; g < g1; g += GAL_THREADS) {
        float zg, sg;
        gal32(c, p, g, zg, sg);
        int lo, hi;
        window(zg, (double)(KWG32 * sg), c.dz, nz, lo, hi);
        float Z = 0.f;
        for (int a = lo; a <= hi; a++) {
            float u = (a * dz - zg) / sg;
            float wa = (a == 0 || a == nz - 1) ? 0.5f * dz : dz;
            Z += wa * norm / sg * expf(-0.5f * u * u) * (float)dv[a];
        }
        invZ[g] = Z > 0.f ? 1.f / Z : 0.f;
    }
    __syncthreads();
    const float smax = c.pix_sigmax32[p] * KWG32;
    for (int a = threadIdx.x; a < nz; a += GAL_THREADS) {
        float za = a * dz, acc = 0.f;
        int64_t l = g0, r = g1;
        while (l < r) {
            int64_t m = (l + r) >> 1;
            float zm, sm;
            gal32(c, p, m, zm, sm);
            if (zm < za - smax) l = m + 1; else r = m;
        }
        for (int64_t g = l; g < g1; g++) {
            float zg, sg;
            gal32(c, p, g, zg, sg);
            if (zg > za + smax) break;
            int lo, hi;
            window(zg, (double)(KWG32 * sg), c.dz, nz, lo, hi);
            if (a < lo || a > hi) continue;
            float u = (za - zg) / sg;
            acc += norm / sg * expf(-0.5f * u * u) * invZ[g];
        }
        G[p * nz + a] = acc * (float)dv[a];
    }
}

// Single-1D: sum_k S_k G_k(z_a) per event.
__global__ void k_profile_sum(DevCatalog c, const double *G64, const float *G32, double *out64,
                              float *out32) {
    const int ev = blockIdx.x, nz = c.n_z;
    const int64_t p0 = c.ev_poff[ev], p1 = c.ev_poff[ev + 1];
    for (int a = threadIdx.x; a < nz; a += blockDim.x) {
        if (G64) {
            double s = 0.0;
            for (int64_t p = p0; p < p1; p++) s += c.pix_S[p] * G64[p * nz + a];
            out64[(int64_t)ev * nz + a] = s;
        }
        if (G32) {
            float s = 0.f;
            for (int64_t p = p0; p < p1; p++) s += (float)c.pix_S[p] * G32[p * nz + a];
            out32[(int64_t)ev * nz + a] = s;
        }
    }
}

}  // namespace

void launch_galaxy_profile(const DevCatalog &c, const double *fwd, double Om, double *dv,
                           double *invZ64, float *invZ32, double *out64, float *out32,
                           cudaStream_t st) {
    k_dvdz<<<(c.n_z + 255) / 256, 256, 0, st>>>(fwd, Om, c.dz, c.n_z, dv);
    if (c.n_pix == 0) return;
    if (out64) k_profile64<<<(unsigned)c.n_pix, GAL_THREADS, 0, st>>>(c, dv, invZ64, out64);
    if (out32) k_profile32<<<(unsigned)c.n_pix, GAL_THREADS, 0, st>>>(c, dv, invZ32, out32);
}

void launch_profile_sum(const DevCatalog &c, const double *G64, const float *G32, double *outh64,
                        float *outh32, cudaStream_t st) {
    k_profile_sum<<<c.n_events, 256, 0, st>>>(c, G64, G32, outh64, outh32);
}

}  // namespace chim
