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
// The Om derivative used by the adjoint has the same structure:
//   dG/dOm = dv' sum_g N_g / Z_g - dv sum_g N_g Z_g' / Z_g^2,
//   Z_g'   = sum_a w_a N_g(z_a) dv'(z_a),   dv = dV_c/dz, dv' = d dv / dOm.
//
// Three launches per profile, balanced whatever the pixel occupancy (a
// pixel can hold tens of thousands of galaxies while most hold a few
// hundred):
//   norm:   1 / Z_g (and Z_g') for every galaxy, over load-time chunks of
//           GAL_CHUNK galaxies of one pixel, one galaxy per thread;
//   gather: one block per pixel of at most GAL_DENSE galaxies, one grid
//           point per thread, the galaxies whose window covers it (sorted by
//           z inside the pixel at load time, found by binary search);
//   dense:  per (dense pixel, grid point) with galaxies in reach (load-time
//           lists), a block (more than GAL_HEAVY candidates) or a warp, the
//           candidates spread over its threads and added by a fixed tree.
// Every sum has a fixed order, so a profile is reproducible bit for bit.
//
// Incomplete catalogs (Eqs. p-gal, p-miss, f-R) add, after the gathers, the
// missing galaxies, homogeneous in comoving volume: in the same N_gal,tot
// units, G_k <- f_R G_k + N_gal,tot m_k(z_a) dV_c/dz(z_a) / V_c(z_max), with
// m_k = (1 - P_compl) dOmega_k / 4 pi from the load and
// dV_c/dz / V_c(z_max) = 3 dv / D_max^3 (dv = D^2/E, D in units of c/H0).
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "internal.cuh"

namespace chim {

namespace {

constexpr int GAL_THREADS = 256;

// dV_c/dz (up to constants) on the grid, FP64 and its FP32 copy.
__global__ void k_dvdz(const double *fwd, double Om, double dz, int nz, double *dv, float *dv32) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < nz) {
        dv[a] = chimd::dv_of(fwd, a * dz, Om);
        dv32[a] = (float)dv[a];
    }
}

__device__ __forceinline__ void window(double zg, double kw, double dz, int nz, int &lo, int &hi) {
    double a0 = ceil((zg - kw) / dz), a1 = floor((zg + kw) / dz);
    lo = a0 < 0.0 ? 0 : (a0 > nz ? nz : (int)a0);
    hi = a1 > nz - 1 ? nz - 1 : (a1 < -1.0 ? -1 : (int)a1);
}

// Galaxy access by precision: FP64 values and windows of KWG64 sigma, or the
// stored values of the mixed path and its windows of KWG32 sigma.
template <bool F64>
struct Gal;
template <>
struct Gal<true> {
    using T = double;
    __device__ static void read(const DevCatalog &c, int64_t, int64_t g, double &z, double &s) {
        z = c.gz64[g];
        s = c.gs64[g];
    }
    __device__ static void win(const DevCatalog &c, double zg, double sg, int &lo, int &hi) {
        window(zg, KWG64 * sg, c.dz, c.n_z, lo, hi);
    }
    __device__ static double reach(const DevCatalog &c, int64_t p) { return c.pix_sigmax[p] * KWG64; }
    __device__ static double step(const DevCatalog &c) { return c.dz; }
    __device__ static double gauss(double u) { return exp(-0.5 * u * u); }
};
template <>
struct Gal<false> {
    using T = float;
    __device__ static void read(const DevCatalog &c, int64_t p, int64_t g, float &z, float &s) {
        chimd::gal32(c, p, g, z, s);
    }
    __device__ static void win(const DevCatalog &c, float zg, float sg, int &lo, int &hi) {
        chimd::gal_window32(zg, sg, 1.f / c.dz32, c.n_z, lo, hi);
    }
    __device__ static float reach(const DevCatalog &c, int64_t p) { return c.pix_sigmax32[p] * KWG32; }
    __device__ static float step(const DevCatalog &c) { return c.dz32; }
    __device__ static float gauss(float u) { return __expf(-0.5f * u * u); }
};

// 1 / Z_g (and Z_g' with WITH_O) for the galaxies of one load-time chunk.
template <bool F64, bool WITH_O>
__global__ void __launch_bounds__(GAL_CHUNK) k_gal_norm(DevCatalog c, const typename Gal<F64>::T *dv,
                                                       const typename Gal<F64>::T *dvO,
                                                       typename Gal<F64>::T *invZ, typename Gal<F64>::T *ZO) {
    using G = Gal<F64>;
    using T = typename G::T;
    const int p = c.gw_pix[blockIdx.x];
    const int64_t g = c.gw_g0[blockIdx.x] + threadIdx.x;
    if (g >= c.gal_off[p + 1]) return;
    const int nz = c.n_z;
    const T dz = G::step(c), norm = T(0.39894228040143267794);
    T zg, sg;
    G::read(c, p, g, zg, sg);
    int lo, hi;
    G::win(c, zg, sg, lo, hi);
    const T isg = T(1) / sg;
    T Z = T(0), Zp = T(0);
    for (int a = lo; a <= hi; a++) {
        const T u = (a * dz - zg) * isg;
        const T Nv = ((a == 0 || a == nz - 1) ? T(0.5) * dz : dz) * G::gauss(u);
        Z += Nv * dv[a];
        if (WITH_O) Zp += Nv * dvO[a];
    }
    Z *= norm * isg;
    invZ[g] = Z > T(0) ? T(1) / Z : T(0);
    if (WITH_O) ZO[g] = Zp * norm * isg;
}

// The sums of one grid point over galaxies [l, r) of pixel p, strided by
// `step` from `first`: s1 = sum N/Z, s2 = sum N Z'/Z^2 (WITH_O).
template <bool F64, bool WITH_O>
__device__ __forceinline__ void gather_range(const DevCatalog &c, int64_t p, int a, int64_t first, int64_t r,
                                             int stride, const typename Gal<F64>::T *invZ,
                                             const typename Gal<F64>::T *ZO, typename Gal<F64>::T &s1,
                                             typename Gal<F64>::T &s2) {
    using G = Gal<F64>;
    using T = typename G::T;
    const T za = a * G::step(c);
    for (int64_t g = first; g < r; g += stride) {
        T zg, sg;
        G::read(c, p, g, zg, sg);
        int lo, hi;
        G::win(c, zg, sg, lo, hi);
        const T iz = invZ[g];
        if (a < lo || a > hi || iz == T(0)) continue;
        const T isg = T(1) / sg, u = (za - zg) * isg;
        const T Nv = isg * G::gauss(u);
        s1 += Nv * iz;
        if (WITH_O) s2 += Nv * ZO[g] * iz * iz;
    }
}

// First galaxy of pixel p (galaxies [g0, g1), sorted by z) with z >= x, or
// with z > x when `after`.
template <bool F64>
__device__ __forceinline__ int64_t gal_bound(const DevCatalog &c, int64_t p, int64_t g0, int64_t g1,
                                             typename Gal<F64>::T x, bool after) {
    using G = Gal<F64>;
    using T = typename G::T;
    int64_t l = g0, r = g1;
    while (l < r) {
        const int64_t m = (l + r) >> 1;
        T zm, sm;
        G::read(c, p, m, zm, sm);
        if (after ? zm <= x : zm < x) l = m + 1; else r = m;
    }
    return l;
}

template <bool F64, bool WITH_O>
__device__ __forceinline__ typename Gal<F64>::T gather_out(const typename Gal<F64>::T *dv,
                                                           const typename Gal<F64>::T *dvO, int a,
                                                           typename Gal<F64>::T s1, typename Gal<F64>::T s2) {
    using T = typename Gal<F64>::T;
    const T norm = T(0.39894228040143267794);
    return WITH_O ? norm * (dvO[a] * s1 - dv[a] * s2) : norm * s1 * dv[a];
}

// One block per pixel of at most GAL_DENSE galaxies, one grid point per
// thread; the pixel's galaxies (z, sigma, 1/Z, Z') are staged in shared
// memory first, so the two binary searches and the gather of every grid
// point read shared memory.
template <bool F64, bool WITH_O>
__global__ void __launch_bounds__(GAL_THREADS) k_gal_gather(DevCatalog c, const typename Gal<F64>::T *dv,
                                                           const typename Gal<F64>::T *dvO,
                                                           const typename Gal<F64>::T *invZ,
                                                           const typename Gal<F64>::T *ZO,
                                                           typename Gal<F64>::T *out) {
    using G = Gal<F64>;
    using T = typename G::T;
    __shared__ T sz[GAL_DENSE], ss[GAL_DENSE], siz[GAL_DENSE], szo[WITH_O ? GAL_DENSE : 1];
    const int64_t p = blockIdx.x;
    const int64_t g0 = c.gal_off[p], g1 = c.gal_off[p + 1];
    const int ng = (int)(g1 - g0);
    if (ng > GAL_DENSE) {  // the dense kernel's pixel: zero its row, the dense kernel fills it
        for (int a = threadIdx.x; a < c.n_z; a += GAL_THREADS) out[p * c.n_z + a] = T(0);
        return;
    }
    for (int i = threadIdx.x; i < ng; i += GAL_THREADS) {
        G::read(c, p, g0 + i, sz[i], ss[i]);
        siz[i] = invZ[g0 + i];
        if (WITH_O) szo[i] = ZO[g0 + i];
    }
    __syncthreads();
    const int nz = c.n_z;
    const T dz = G::step(c), reach = G::reach(c, p);
    for (int a = threadIdx.x; a < nz; a += GAL_THREADS) {
        const T za = a * dz;
        int l = 0, r = ng;  // first galaxy with z >= za - reach
        while (l < r) {
            const int m = (l + r) >> 1;
            if (sz[m] < za - reach) l = m + 1; else r = m;
        }
        T s1 = T(0), s2 = T(0);
        for (int i = l; i < ng && sz[i] <= za + reach; i++) {
            int lo, hi;
            G::win(c, sz[i], ss[i], lo, hi);
            const T iz = siz[i];
            if (a < lo || a > hi || iz == T(0)) continue;
            const T isg = T(1) / ss[i], u = (za - sz[i]) * isg;
            const T Nv = isg * G::gauss(u);
            s1 += Nv * iz;
            if (WITH_O) s2 += Nv * szo[i] * iz * iz;
        }
        out[p * nz + a] = gather_out<F64, WITH_O>(dv, dvO, a, s1, s2);
    }
}

// Candidate ranges of the dense pixels: one thread per (dense pixel, grid
// point), the same bounds as the gather kernel's.
template <bool F64>
__global__ void k_dense_ranges(DevCatalog c, int2 *lr) {
    using G = Gal<F64>;
    using T = typename G::T;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)c.n_dense * c.n_z) return;
    const int64_t p = c.dense_pix[i / c.n_z];
    const int a = (int)(i % c.n_z);
    const int64_t g0 = c.gal_off[p], g1 = c.gal_off[p + 1];
    const T za = a * G::step(c), reach = G::reach(c, p);
    const int64_t l = gal_bound<F64>(c, p, g0, g1, za - reach, false);
    const int64_t r = gal_bound<F64>(c, p, l, g1, za + reach, true);
    lr[i] = make_int2((int)(l - g0), (int)(r - g0));
}

// Dense pixels, over the load-time lists of (dense pixel, grid point) pairs
// whose candidate range is not empty (the other points of a dense row are
// zeroed by the gather kernel).  HEAVY: one block per pair (ranges above
// GAL_HEAVY galaxies), the range spread over the block and added by a fixed
// tree; otherwise one warp per pair, added by a fixed xor tree.
template <bool F64, bool WITH_O, bool HEAVY>
__global__ void __launch_bounds__(GAL_THREADS) k_gal_gather_dense(DevCatalog c, const typename Gal<F64>::T *dv,
                                                                 const typename Gal<F64>::T *dvO,
                                                                 const typename Gal<F64>::T *invZ,
                                                                 const typename Gal<F64>::T *ZO,
                                                                 typename Gal<F64>::T *out) {
    using T = typename Gal<F64>::T;
    __shared__ T red[2][GAL_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t n_heavy = F64 ? c.n_dheavy64 : c.n_dheavy32;
    const int64_t n_all = F64 ? c.n_ditems64 : c.n_ditems32;
    const int64_t idx = HEAVY ? (int64_t)blockIdx.x
                              : n_heavy + (int64_t)blockIdx.x * (GAL_THREADS / 32) + wid;
    if (!HEAVY && idx >= n_all) return;  // whole warps leave together
    const int2 item = (F64 ? c.dense_items64 : c.dense_items32)[idx];  // (dense index, grid point)
    const int64_t p = c.dense_pix[item.x];
    const int a = item.y;
    const int64_t g0 = c.gal_off[p];
    const int2 lr = (F64 ? c.dense_lr64 : c.dense_lr32)[(int64_t)item.x * c.n_z + a];
    T s1 = T(0), s2 = T(0);
    if (HEAVY) gather_range<F64, WITH_O>(c, p, a, g0 + lr.x + threadIdx.x, g0 + lr.y, GAL_THREADS, invZ, ZO, s1, s2);
    else gather_range<F64, WITH_O>(c, p, a, g0 + lr.x + lane, g0 + lr.y, 32, invZ, ZO, s1, s2);
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        if (WITH_O) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (!HEAVY) {
        if (lane == 0) out[p * c.n_z + a] = gather_out<F64, WITH_O>(dv, dvO, a, s1, s2);
        return;
    }
    if (lane == 0) {
        red[0][wid] = s1;
        red[1][wid] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T t1 = T(0), t2 = T(0);
        for (int w = 0; w < GAL_THREADS / 32; w++) {
            t1 += red[0][w];
            t2 += red[1][w];
        }
        out[p * c.n_z + a] = gather_out<F64, WITH_O>(dv, dvO, a, t1, t2);
    }
}

template <bool F64, bool WITH_O>
void launch_profile_t(const DevCatalog &c, const typename Gal<F64>::T *dv, const typename Gal<F64>::T *dvO,
                      typename Gal<F64>::T *invZ, typename Gal<F64>::T *ZO, typename Gal<F64>::T *out,
                      cudaStream_t st) {
    if (c.n_pix == 0) return;
    if (c.n_gw > 0) k_gal_norm<F64, WITH_O><<<(unsigned)c.n_gw, GAL_CHUNK, 0, st>>>(c, dv, dvO, invZ, ZO);
    k_gal_gather<F64, WITH_O><<<(unsigned)c.n_pix, GAL_THREADS, 0, st>>>(c, dv, dvO, invZ, ZO, out);
    {
        const int64_t nh = F64 ? c.n_dheavy64 : c.n_dheavy32;
        const int64_t nl = (F64 ? c.n_ditems64 : c.n_ditems32) - nh;
        const int wpb = GAL_THREADS / 32;
        if (nh > 0)
            k_gal_gather_dense<F64, WITH_O, true><<<(unsigned)nh, GAL_THREADS, 0, st>>>(c, dv, dvO, invZ, ZO, out);
        if (nl > 0)
            k_gal_gather_dense<F64, WITH_O, false>
                <<<(unsigned)((nl + wpb - 1) / wpb), GAL_THREADS, 0, st>>>(c, dv, dvO, invZ, ZO, out);
    }
}

// f_R G + (m c) dv with every rounding explicit (no contraction), so the
// one-Om and batched launches agree bit for bit.
__device__ __forceinline__ float miss_update(float fR, float G, float m, float c, float dv) {
    return __fadd_rn(__fmul_rn(fR, G), __fmul_rn(__fmul_rn(m, c), dv));
}
__device__ __forceinline__ double miss_update(double fR, double G, double m, double c, double dv) {
    return __dadd_rn(__dmul_rn(fR, G), __dmul_rn(__dmul_rn(m, c), dv));
}
// Its Om derivative form: f_R dG + m (c1 dv' + c2 dv).
__device__ __forceinline__ float miss_update_O(float fR, float G, float m, float c1, float dvO, float c2, float dv) {
    return __fadd_rn(__fmul_rn(fR, G), __fmul_rn(m, __fadd_rn(__fmul_rn(c1, dvO), __fmul_rn(c2, dv))));
}
__device__ __forceinline__ double miss_update_O(double fR, double G, double m, double c1, double dvO, double c2,
                                                double dv) {
    return __dadd_rn(__dmul_rn(fR, G), __dmul_rn(m, __dadd_rn(__dmul_rn(c1, dvO), __dmul_rn(c2, dv))));
}

// The missing-galaxy term of an incomplete catalog, over the whole profile
// (grid-stride); WITH_O writes its Om derivative, f_R dG + 3 N m (dv' -
// 3 dv D_max'/D_max) / D_max^3, into the dG/dOm rows.  Thread 0 of each
// block evaluates D_max (and D_max') once.
template <bool F64, bool WITH_O>
__global__ void __launch_bounds__(GAL_THREADS) k_gal_missing(DevCatalog c, const double *fwd, const double *fwdO,
                                                            double Om, const typename Gal<F64>::T *dv,
                                                            const typename Gal<F64>::T *dvO,
                                                            typename Gal<F64>::T *out) {
    using T = typename Gal<F64>::T;
    __shared__ T s_c[2];
    if (threadIdx.x == 0) {
        double c1, c2;
        chimd::miss_scales(fwd, WITH_O ? fwdO : nullptr, c.z_max, Om, c.n_gal_total, c1, c2);
        s_c[0] = T(c1);
        s_c[1] = T(c2);
    }
    __syncthreads();
    const T c1 = s_c[0], c2 = s_c[1], fR = T(c.f_R);
    const T *m = F64 ? (const T *)c.miss64 : (const T *)c.miss32;
    const int nz = c.n_z;
    const int64_t n = c.n_pix * nz;
    for (int64_t i = blockIdx.x * (int64_t)GAL_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * GAL_THREADS) {
        const int a = (int)(i % nz);
        if (WITH_O) out[i] = miss_update_O(fR, out[i], m[i], c1, dvO[a], c2, dv[a]);
        else out[i] = miss_update(fR, out[i], m[i], c1, dv[a]);
    }
}

template <bool F64, bool WITH_O>
void launch_missing_t(const DevCatalog &c, const double *fwd, const double *fwdO, double Om,
                      const typename Gal<F64>::T *dv, const typename Gal<F64>::T *dvO,
                      typename Gal<F64>::T *out, cudaStream_t st) {
    if (!c.incomplete || c.n_pix == 0) return;
    const int64_t n = c.n_pix * c.n_z;
    const int64_t nb = std::min<int64_t>((n + GAL_THREADS - 1) / GAL_THREADS, 148 * 8);
    k_gal_missing<F64, WITH_O><<<(unsigned)nb, GAL_THREADS, 0, st>>>(c, fwd, fwdO, Om, dv, dvO, out);
}

// ---- batched profiles of PROF_MB Om values (mixed path).  The same
// arithmetic as the kernels above, per column j, in the same order, so the
// results equal the one-Om launches bit for bit; only the Gaussian of each
// (galaxy, grid point) pair is shared by the columns.  WITH_O: the dG/dOm
// rows (two sums per column, as in the one-Om WITH_O kernels).

// dV_c/dz of every column, [(n_z + 1) x PROF_MB] (the columns of a grid
// point side by side, two float4), row n_z the missing-galaxy scale c1;
// WITH_O also dV_c/dz' into dvOm (row n_z: c2).
template <bool WITH_O>
__global__ void k_dvdz_multi(MultiOm m, DevCatalog c, float *dvm, float *dvOm) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, nz = c.n_z;
    const int64_t o = (int64_t)a * PROF_MB + j;
    if (a < nz) {
        if (WITH_O) {
            double dv, dvO;
            chimd::dv_pair(m.fwd[j], m.fwdO[j], a * c.dz, m.Om[j], dv, dvO);
            dvm[o] = (float)dv;
            dvOm[o] = (float)dvO;
        } else {
            dvm[o] = (float)chimd::dv_of(m.fwd[j], a * c.dz, m.Om[j]);
        }
    } else if (a == nz) {
        double c1, c2;
        chimd::miss_scales(m.fwd[j], WITH_O ? m.fwdO[j] : nullptr, c.z_max, m.Om[j], c.n_gal_total, c1, c2);
        dvm[o] = (float)c1;
        if (WITH_O) dvOm[o] = (float)c2;
    }
}

__device__ __forceinline__ void load8(const float *src, float *v) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int q = 0; q < PROF_MB / 4; q++) {
        const float4 x = s4[q];
        v[4 * q] = x.x;
        v[4 * q + 1] = x.y;
        v[4 * q + 2] = x.z;
        v[4 * q + 3] = x.w;
    }
}

__device__ __forceinline__ void store8(float *dst, const float *v) {
    float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int q = 0; q < PROF_MB / 4; q++) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

template <bool WITH_O>
__global__ void __launch_bounds__(GAL_CHUNK) k_gal_norm_multi(DevCatalog c, const float *dvm, const float *dvOm,
                                                             float *invZm, float *ZOm) {
    using G = Gal<false>;
    const int p = c.gw_pix[blockIdx.x];
    const int64_t g = c.gw_g0[blockIdx.x] + threadIdx.x;
    if (g >= c.gal_off[p + 1]) return;
    const int nz = c.n_z;
    const float dz = G::step(c), norm = 0.39894228040143267794f;
    float zg, sg;
    G::read(c, p, g, zg, sg);
    int lo, hi;
    G::win(c, zg, sg, lo, hi);
    const float isg = 1.f / sg;
    float Z[PROF_MB], Zp[PROF_MB];
#pragma unroll
    for (int j = 0; j < PROF_MB; j++) Z[j] = Zp[j] = 0.f;
    for (int a = lo; a <= hi; a++) {
        const float u = (a * dz - zg) * isg;
        const float Nv = ((a == 0 || a == nz - 1) ? 0.5f * dz : dz) * G::gauss(u);
        float d[PROF_MB];
        load8(dvm + (int64_t)a * PROF_MB, d);
#pragma unroll
        for (int j = 0; j < PROF_MB; j++) Z[j] += Nv * d[j];
        if (WITH_O) {
            load8(dvOm + (int64_t)a * PROF_MB, d);
#pragma unroll
            for (int j = 0; j < PROF_MB; j++) Zp[j] += Nv * d[j];
        }
    }
    float v[PROF_MB];
#pragma unroll
    for (int j = 0; j < PROF_MB; j++) {
        const float Zj = Z[j] * (norm * isg);
        v[j] = Zj > 0.f ? 1.f / Zj : 0.f;
    }
    store8(invZm + g * PROF_MB, v);
    if (WITH_O) {
#pragma unroll
        for (int j = 0; j < PROF_MB; j++) v[j] = Zp[j] * norm * isg;
        store8(ZOm + g * PROF_MB, v);
    }
}

// Adds one galaxy's terms to the column sums (skipping columns with 1/Z = 0,
// as the one-Om kernels skip the galaxy).
template <bool WITH_O>
__device__ __forceinline__ void add_multi(float Nv, const float *iz, const float *zo, float *s1, float *s2) {
#pragma unroll
    for (int j = 0; j < PROF_MB; j++)
        if (iz[j] != 0.f) {
            s1[j] += Nv * iz[j];
            if (WITH_O) s2[j] += Nv * zo[j] * iz[j] * iz[j];
        }
}

template <bool WITH_O>
__device__ __forceinline__ void store_multi(const MultiOm &m, const float *dvm, const float *dvOm, int64_t p, int nz,
                                            int a, const float *s1, const float *s2) {
    const float norm = 0.39894228040143267794f;
    float d[PROF_MB], dO[PROF_MB];
    load8(dvm + (int64_t)a * PROF_MB, d);
    if (WITH_O) load8(dvOm + (int64_t)a * PROF_MB, dO);
#pragma unroll
    for (int j = 0; j < PROF_MB; j++)
        if (m.out[j]) m.out[j][p * nz + a] = WITH_O ? norm * (dO[j] * s1[j] - d[j] * s2[j]) : norm * s1[j] * d[j];
}

// Pixels of at most GAL_DENSE galaxies: block per pixel, point per thread,
// galaxies staged in (dynamic) shared memory (dense pixels' rows are zeroed).
template <bool WITH_O>
__global__ void __launch_bounds__(GAL_THREADS) k_gal_gather_multi(DevCatalog c, MultiOm m, const float *dvm,
                                                                 const float *dvOm, const float *invZm,
                                                                 const float *ZOm) {
    using G = Gal<false>;
    extern __shared__ float4 gm_smem[];
    float4 *siz = gm_smem;                              // [GAL_DENSE x PROF_MB]
    float4 *szo = siz + GAL_DENSE * PROF_MB / 4;        // WITH_O
    float *sz = reinterpret_cast<float *>(siz + (WITH_O ? 2 : 1) * GAL_DENSE * PROF_MB / 4);
    float *ss = sz + GAL_DENSE;
    const int64_t p = blockIdx.x;
    const int64_t g0 = c.gal_off[p], g1 = c.gal_off[p + 1];
    const int ng = (int)(g1 - g0), nz = c.n_z;
    if (ng > GAL_DENSE) {
        for (int a = threadIdx.x; a < nz; a += GAL_THREADS)
#pragma unroll
            for (int j = 0; j < PROF_MB; j++)
                if (m.out[j]) m.out[j][p * nz + a] = 0.f;
        return;
    }
    for (int i = threadIdx.x; i < ng; i += GAL_THREADS) G::read(c, p, g0 + i, sz[i], ss[i]);
    const float4 *src = reinterpret_cast<const float4 *>(invZm + g0 * PROF_MB);
    for (int i = threadIdx.x; i < ng * (PROF_MB / 4); i += GAL_THREADS) siz[i] = src[i];
    if (WITH_O) {
        const float4 *so = reinterpret_cast<const float4 *>(ZOm + g0 * PROF_MB);
        for (int i = threadIdx.x; i < ng * (PROF_MB / 4); i += GAL_THREADS) szo[i] = so[i];
    }
    __syncthreads();
    const float *sizf = reinterpret_cast<const float *>(siz), *szof = reinterpret_cast<const float *>(szo);
    const float dz = G::step(c), reach = G::reach(c, p);
    for (int a = threadIdx.x; a < nz; a += GAL_THREADS) {
        const float za = a * dz;
        int l = 0, r = ng;
        while (l < r) {
            const int mid = (l + r) >> 1;
            if (sz[mid] < za - reach) l = mid + 1; else r = mid;
        }
        float s1[PROF_MB], s2[PROF_MB];
#pragma unroll
        for (int j = 0; j < PROF_MB; j++) s1[j] = s2[j] = 0.f;
        for (int i = l; i < ng && sz[i] <= za + reach; i++) {
            int lo, hi;
            G::win(c, sz[i], ss[i], lo, hi);
            if (a < lo || a > hi) continue;
            const float isg = 1.f / ss[i], u = (za - sz[i]) * isg;
            const float Nv = isg * G::gauss(u);
            float iz[PROF_MB], zo[PROF_MB];
            load8(sizf + i * PROF_MB, iz);
            if (WITH_O) load8(szof + i * PROF_MB, zo);
            add_multi<WITH_O>(Nv, iz, zo, s1, s2);
        }
        store_multi<WITH_O>(m, dvm, dvOm, p, nz, a, s1, s2);
    }
}

constexpr size_t gather_multi_smem(bool with_o) {
    return (with_o ? 2 : 1) * sizeof(float) * GAL_DENSE * PROF_MB + 2 * sizeof(float) * GAL_DENSE;
}

// Dense pixels over the load-time item lists (HEAVY: block per item).
template <bool WITH_O, bool HEAVY>
__global__ void __launch_bounds__(GAL_THREADS) k_gal_gather_dense_multi(DevCatalog c, MultiOm m, const float *dvm,
                                                                       const float *dvOm, const float *invZm,
                                                                       const float *ZOm) {
    using G = Gal<false>;
    __shared__ float red[2][PROF_MB][GAL_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t idx = HEAVY ? (int64_t)blockIdx.x
                              : c.n_dheavy32 + (int64_t)blockIdx.x * (GAL_THREADS / 32) + wid;
    if (!HEAVY && idx >= c.n_ditems32) return;
    const int2 item = c.dense_items32[idx];
    const int64_t p = c.dense_pix[item.x];
    const int a = item.y, nz = c.n_z;
    const int64_t g0 = c.gal_off[p];
    const int2 lr = c.dense_lr32[(int64_t)item.x * nz + a];
    float s1[PROF_MB], s2[PROF_MB];
#pragma unroll
    for (int j = 0; j < PROF_MB; j++) s1[j] = s2[j] = 0.f;
    const float za = a * G::step(c);
    const int stride = HEAVY ? GAL_THREADS : 32;
    for (int64_t g = g0 + lr.x + (HEAVY ? threadIdx.x : lane); g < g0 + lr.y; g += stride) {
        float zg, sg;
        G::read(c, p, g, zg, sg);
        int lo, hi;
        G::win(c, zg, sg, lo, hi);
        if (a < lo || a > hi) continue;
        const float isg = 1.f / sg, u = (za - zg) * isg;
        const float Nv = isg * G::gauss(u);
        float iz[PROF_MB], zo[PROF_MB];
        load8(invZm + g * PROF_MB, iz);
        if (WITH_O) load8(ZOm + g * PROF_MB, zo);
        add_multi<WITH_O>(Nv, iz, zo, s1, s2);
    }
#pragma unroll
    for (int j = 0; j < PROF_MB; j++)
        for (int o = 16; o > 0; o >>= 1) {
            s1[j] += __shfl_xor_sync(0xffffffffu, s1[j], o);
            if (WITH_O) s2[j] += __shfl_xor_sync(0xffffffffu, s2[j], o);
        }
    if (!HEAVY) {
        if (lane == 0) store_multi<WITH_O>(m, dvm, dvOm, p, nz, a, s1, s2);
        return;
    }
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < PROF_MB; j++) {
            red[0][j][wid] = s1[j];
            red[1][j][wid] = s2[j];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        float t1[PROF_MB], t2[PROF_MB];
#pragma unroll
        for (int j = 0; j < PROF_MB; j++) {
            t1[j] = t2[j] = 0.f;
            for (int w = 0; w < GAL_THREADS / 32; w++) {
                t1[j] += red[0][j][w];
                t2[j] += red[1][j][w];
            }
        }
        store_multi<WITH_O>(m, dvm, dvOm, p, nz, a, t1, t2);
    }
}

// The missing-galaxy term of an incomplete catalog for every column.
template <bool WITH_O>
__global__ void __launch_bounds__(GAL_THREADS) k_gal_missing_multi(DevCatalog c, MultiOm m, const float *dvm,
                                                                  const float *dvOm) {
    const float fR = (float)c.f_R;
    const int nz = c.n_z;
    const int64_t n = c.n_pix * nz;
    for (int64_t i = blockIdx.x * (int64_t)GAL_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * GAL_THREADS) {
        const int a = (int)(i % nz);
        const float mi = c.miss32[i];
        const int64_t oa = (int64_t)a * PROF_MB, oz = (int64_t)nz * PROF_MB;
#pragma unroll
        for (int j = 0; j < PROF_MB; j++) {
            if (!m.out[j]) continue;
            m.out[j][i] = WITH_O ? miss_update_O(fR, m.out[j][i], mi, dvm[oz + j], dvOm[oa + j], dvOm[oz + j], dvm[oa + j])
                                 : miss_update(fR, m.out[j][i], mi, dvm[oz + j], dvm[oa + j]);
        }
    }
}

template <bool WITH_O>
void launch_multi_t(const DevCatalog &c, const MultiOm &m, float *dvm, float *invZm, cudaStream_t st) {
    float *dvOm = WITH_O ? dvm + (size_t)(c.n_z + 1) * PROF_MB : nullptr;
    float *ZOm = WITH_O ? invZm + (size_t)std::max<int64_t>(c.n_gal, 1) * PROF_MB : nullptr;
    k_dvdz_multi<WITH_O><<<dim3((unsigned)((c.n_z + 1 + 63) / 64), PROF_MB), 64, 0, st>>>(m, c, dvm, dvOm);
    if (c.n_gw > 0) k_gal_norm_multi<WITH_O><<<(unsigned)c.n_gw, GAL_CHUNK, 0, st>>>(c, dvm, dvOm, invZm, ZOm);
    constexpr size_t smem = gather_multi_smem(WITH_O);
    // the opt-in to more than 48 KB of dynamic shared memory is per device:
    // set it on every launch (the current device may change between calls)
    cudaFuncSetAttribute(k_gal_gather_multi<WITH_O>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gal_gather_multi<WITH_O><<<(unsigned)c.n_pix, GAL_THREADS, smem, st>>>(c, m, dvm, dvOm, invZm, ZOm);
    const int64_t nh = c.n_dheavy32, nl = c.n_ditems32 - nh;
    const int wpb = GAL_THREADS / 32;
    if (nh > 0)
        k_gal_gather_dense_multi<WITH_O, true><<<(unsigned)nh, GAL_THREADS, 0, st>>>(c, m, dvm, dvOm, invZm, ZOm);
    if (nl > 0)
        k_gal_gather_dense_multi<WITH_O, false>
            <<<(unsigned)((nl + wpb - 1) / wpb), GAL_THREADS, 0, st>>>(c, m, dvm, dvOm, invZm, ZOm);
    if (c.incomplete) {
        const int64_t n = c.n_pix * c.n_z;
        const int64_t nb = std::min<int64_t>((n + GAL_THREADS - 1) / GAL_THREADS, 148 * 8);
        k_gal_missing_multi<WITH_O><<<(unsigned)nb, GAL_THREADS, 0, st>>>(c, m, dvm, dvOm);
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
    float *dv32 = reinterpret_cast<float *>(dv + c.n_z);
    k_dvdz<<<(c.n_z + 63) / 64, 64, 0, st>>>(fwd, Om, c.dz, c.n_z, dv, dv32);  // FP64: spread over SMs
    if (out64) {
        launch_profile_t<true, false>(c, dv, nullptr, invZ64, nullptr, out64, st);
        launch_missing_t<true, false>(c, fwd, nullptr, Om, dv, nullptr, out64, st);
    }
    if (out32) {
        launch_profile_t<false, false>(c, dv32, nullptr, invZ32, nullptr, out32, st);
        launch_missing_t<false, false>(c, fwd, nullptr, Om, dv32, nullptr, out32, st);
    }
}

void launch_galaxy_profile_multi(const DevCatalog &c, const MultiOm &m, bool dOm, float *dvm, float *invZm,
                                 cudaStream_t st) {
    if (c.n_pix == 0) return;
    if (dOm) launch_multi_t<true>(c, m, dvm, invZm, st);
    else launch_multi_t<false>(c, m, dvm, invZm, st);
}

void launch_dense_ranges(const DevCatalog &c, cudaStream_t st) {
    const int64_t n = (int64_t)c.n_dense * c.n_z;
    if (n == 0) return;
    const unsigned nb = (unsigned)((n + 255) / 256);
    k_dense_ranges<true><<<nb, 256, 0, st>>>(c, c.dense_lr64);
    k_dense_ranges<false><<<nb, 256, 0, st>>>(c, c.dense_lr32);
}

void launch_galaxy_dOm(const DevCatalog &c, const double *fwd, const double *fwdO, double Om, const double *dv,
                       const double *dvO, const float *dv32, const float *dvO32, bool f64, void *invZ, void *ZO,
                       void *out, cudaStream_t st) {
    if (f64) {
        launch_profile_t<true, true>(c, dv, dvO, (double *)invZ, (double *)ZO, (double *)out, st);
        launch_missing_t<true, true>(c, fwd, fwdO, Om, dv, dvO, (double *)out, st);
    } else {
        launch_profile_t<false, true>(c, dv32, dvO32, (float *)invZ, (float *)ZO, (float *)out, st);
        launch_missing_t<false, true>(c, fwd, fwdO, Om, dv32, dvO32, (float *)out, st);
    }
}

void launch_profile_sum(const DevCatalog &c, const double *G64, const float *G32, double *outh64,
                        float *outh32, cudaStream_t st) {
    k_profile_sum<<<c.n_events, 256, 0, st>>>(c, G64, G32, outh64, outh32);
}

}  // namespace chim
