// f2 on the tensor cores: the galaxy term of Eq. p-cat for a batch of up to
// TC_COLS Om values at once, for catalogs of wide (photometric) galaxies,
// where the Om-independent Gaussians N(z_a; z_g, s_g) form a dense
// (grid point x galaxy) matrix and the profile is two contractions with it:
//
//   Z_g(j)    = sum_a N_ga w_a dv_j(z_a)                  (norm pass)
//   G_k(a, j) = dv_j(z_a) sum_{g in k} N_ga / Z_g(j)      (gather pass)
//
// with dv_j = dV_c/dz at the j-th Om (up to constants, which cancel) and w_a
// the trapezoid weights.  Both run as tcgen05 MMAs (M = 128 Om columns,
// N = 256 galaxies or grid points per tile, K = 64 per stage):
//   * the Gaussians are evaluated by the CTA's threads (FP32, __expf, the
//     mixed path's +-6 sigma windows), rounded to FP16 and written into
//     shared memory in the 128-byte-swizzled K-major layout; the same values
//     enter both passes, so every galaxy keeps unit weight on the grid;
//   * the Om-dependent operands (w_a dv_j, scaled by 2^12, and 1/Z_g, scaled
//     by a power of two chosen at load) are split into two FP16 terms,
//     x = hi + lo, each its own MMA, which leaves them about 22 bits; they are
//     laid out in global memory as the exact shared-memory image of a stage
//     and fetched by one bulk copy per stage;
//   * the tensor cores' FP32 accumulation rounds toward zero, so a long sum
//     drifts low (measured: ~2e-5 relative over 1000 accumulations); the
//     partial sums are therefore accumulated in tensor memory for TC_PROMO
//     stages at a time only and added, on the CUDA cores and rounded to
//     nearest, into a running FP32 sum kept in a second tensor-memory region.
// Rounding: every Gaussian carries one FP16 rounding (relative 2^-11, in a
// different direction for every (galaxy, grid point) pair, so the sums
// average it down); the split operands carry ~2^-22.
//
// Work: the norm pass takes 256 consecutive galaxy slots per CTA (a slot
// space padded to 64 per pixel); the gather pass is a persistent kernel over
// (pixel, 256-point grid tile, range of <= TC_KSPLIT 64-galaxy blocks) items,
// heaviest first; items of a pixel split along K write partial sums that a
// third kernel adds in a fixed order.  Items and blocks are fixed at load.
// Each CTA holds two stages of shared memory (~131 KB) and all 512
// tensor-memory columns (the partial and the running sum), so one CTA runs
// per SM.
//
// Waits on mbarriers are bounded: a wait that runs out records an error
// flag, the CTA stops issuing work, waits (bounded) for what it issued and
// frees its tensor memory; later CTAs of the pass see the flag and return.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "tc.cuh"

namespace chim {

int cuda_check(cudaError_t e, const char *what);

namespace {

constexpr int TC_THREADS = 512;
constexpr int TC_CG = TC_THREADS / 128;     // column groups: warps sharing one TMEM lane quarter
constexpr int TC_IMG = TC_M * TC_K * 2;     // one 128 x 64 FP16 operand image (16 KB)
constexpr int TC_BIMG = TC_N * TC_K * 2;    // the generated 256 x 64 FP16 operand (32 KB)
constexpr int TC_AST = 2 * TC_IMG;          // A operands of a stage: (hi, lo)
constexpr int TC_STAGE = TC_AST + TC_BIMG;  // 64 KB
constexpr int TC_TROW = TC_N + 4;           // row pitch (floats) of the epilogue's staging tile
constexpr int TC_TBYTES = TC_M * TC_TROW * 4;  // the staging tile (aliases the stages)
constexpr int TC_SMEM_MAIN = ((2 * TC_STAGE > TC_TBYTES ? 2 * TC_STAGE : TC_TBYTES) + 1023) / 1024 * 1024;
constexpr int TC_SMEM = TC_SMEM_MAIN + 2048 + 256 + 1024;  // + per-stage galaxy parameters, barriers, alignment
constexpr float TC_SV = 4096.f;             // scale of w_a dv_j in the norm pass
constexpr uint32_t TC_IDESC = tc::idesc_f16_f32(TC_M, TC_N);
constexpr uint32_t TC_TCOLS = 2 * TC_N;     // tensor-memory columns: partial [0, 256), running sum [256, 512)
constexpr uint32_t TC_SUM = TC_N;           // column of the running sum
// one CTA per SM: a second could not allocate its tensor memory anyway
static_assert(2 * TC_SMEM > 232448, "two CTAs would fit in shared memory");

// The Gaussian of grid point a and a galaxy, as both passes evaluate it:
// exp(-(a dz - z_g)^2 / (2 sigma_g^2)) = 2^-(a c_g - d_g)^2 with
// c_g = dz / sigma_g * sqrt(log2(e) / 2) and d_g = z_g / sigma_g * sqrt(log2(e) / 2),
// one FMA, one multiply and one SFU exponential per element.  No window test:
// beyond 5.88 sigma the value is below half the smallest FP16 subnormal and
// rounds to zero, so the FP16 operand holds the mixed path's +-6 sigma
// window by itself (the mass between 5.88 and 6 sigma is ~1e-9 of a
// galaxy's).  A slot without a galaxy takes c = 0, d = -1e4 (value 0).
constexpr float TC_S2L = 0.84932180028801904272f;  // sqrt(log2(e) / 2)
__device__ __forceinline__ float tc_gauss(float af, float2 cd) {
    const float t = __fmaf_rn(af, cd.x, -cd.y);
    return tc::ex2(-__fmul_rn(t, t));
}

struct TcSmem {
    char *st[2];   // stage: A operands (hi, lo images) then the generated B operand (1024-aligned)
    float2 *gp;    // [2][64] galaxy (c_g, d_g) of the gather stage
    uint64_t *full, *mma;  // [2] each
    uint32_t *tmem_holder;
    int *flag;
};

__device__ __forceinline__ TcSmem tc_smem(char *raw) {
    TcSmem s;
    char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
    s.st[0] = base;
    s.st[1] = base + TC_STAGE;
    char *tail = base + TC_SMEM_MAIN;
    s.gp = reinterpret_cast<float2 *>(tail);  // 1 KB
    s.full = reinterpret_cast<uint64_t *>(tail + 2048);
    s.mma = s.full + 2;
    s.tmem_holder = reinterpret_cast<uint32_t *>(s.mma + 2);
    s.flag = reinterpret_cast<int *>(s.tmem_holder + 1);
    return s;
}

// Barriers and tensor memory of a CTA (warp 0 allocates).  *s.flag (read
// by every thread after the call) is set when an earlier CTA of the pass
// recorded a timeout in err: the CTA then does no work.
__device__ __forceinline__ uint32_t tc_setup(TcSmem &s, const int *err) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; i++) {
            tc::mbar_init(s.full + i, 1);
            tc::mbar_init(s.mma + i, 1);
        }
        *s.flag = *reinterpret_cast<const volatile int *>(err);
        tc::fence_mbar_init();
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(s.tmem_holder, TC_TCOLS);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    return *s.tmem_holder;
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem) {
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(tmem, TC_TCOLS);
}

// One stage of MMAs into the partial sum: K = 64 in four steps, each the hi
// and the lo operand.  Thread 0 only.
__device__ __forceinline__ void tc_issue(uint32_t tmem, const char *stage, bool first) {
    const uint32_t a0 = tc::smem_u32(stage), b0 = a0 + TC_AST;
#pragma unroll
    for (int ks = 0; ks < TC_K / 16; ks++) {
        const uint64_t bd = tc::desc_sw128(b0 + 32 * ks);
#pragma unroll
        for (int hl = 0; hl < 2; hl++) {
            const uint64_t ad = tc::desc_sw128(a0 + (uint32_t)(hl * TC_IMG) + 32 * ks);
            tc::mma_f16(tmem, ad, bd, TC_IDESC, (first && ks == 0 && hl == 0) ? 0u : 1u);
        }
    }
}

// Columns of the accumulator a thread handles outside the MMAs: warp w
// reads TMEM lanes 32 (w & 3) + lane (row r of the tile) and columns
// [64 (w >> 2), 64 (w >> 2) + 64).
__device__ __forceinline__ uint32_t tc_lane_base() { return (uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16; }
__device__ __forceinline__ int tc_col0() { return (threadIdx.x >> 7) * (TC_N / TC_CG); }

// Promotion: running sum (+)= partial, on the CUDA cores (the MMAs that wrote
// the partial have completed and are fenced): per 32 columns two loads, one
// wait, the FP32 additions (round to nearest) and a store; one store wait.
__device__ __forceinline__ void tc_promote(uint32_t tmem, bool first) {
    const uint32_t lb = tc_lane_base();
    const int c0 = tc_col0();
#pragma unroll
    for (int n0 = c0; n0 < c0 + TC_N / TC_CG; n0 += 32) {
        uint32_t pv[32], sv[32];
        tc::tmem_ld32_nowait(tmem + lb + (uint32_t)n0, pv);
        if (!first) tc::tmem_ld32_nowait(tmem + lb + TC_SUM + (uint32_t)n0, sv);
        tc::tmem_wait_ld();
        if (!first)
#pragma unroll
            for (int i = 0; i < 32; i++) pv[i] = __float_as_uint(__uint_as_float(pv[i]) + __uint_as_float(sv[i]));
        tc::tmem_st32_nowait(tmem + lb + TC_SUM + (uint32_t)n0, pv);
    }
    tc::tmem_wait_st();
}

// The epilogue's transpose: the running sum's 128 rows x 256 columns staged in
// shared memory (rows padded to 260 floats), so that a warp then writes
// 1 KB of one row with 16-byte stores.
__device__ __forceinline__ void tc_stage_rows(uint32_t tmem, bool have, float *T) {
    const int r = threadIdx.x & 127, c0 = tc_col0();
    const uint32_t lb = tc_lane_base();
    float *row = T + (size_t)r * TC_TROW;
    for (int n0 = c0; n0 < c0 + TC_N / TC_CG; n0 += 16) {
        float d[16];
        if (have) tc::tmem_ld16(tmem + lb + TC_SUM + (uint32_t)n0, d);
        else
#pragma unroll
            for (int i = 0; i < 16; i++) d[i] = 0.f;
#pragma unroll
        for (int i = 0; i < 4; i++)
            *reinterpret_cast<float4 *>(row + n0 + 4 * i) = make_float4(d[4 * i], d[4 * i + 1], d[4 * i + 2], d[4 * i + 3]);
    }
}

// Bounded wait (thread 0) for what a CTA issued before it stops (error path).
__device__ __forceinline__ void tc_drain(TcSmem &s, const bool *copy_out, const uint32_t *fill,
                                         const bool *mma_out, const uint32_t *use) {
    if (threadIdx.x == 0)
        for (int st = 0; st < 2; st++) {
            if (copy_out[st]) tc::mbar_wait(s.full + st, fill[st] & 1u);
            if (mma_out[st]) tc::mbar_wait(s.mma + st, use[st] & 1u);
        }
    __syncthreads();
}

// The K loop shared by both passes, software-pipelined over two stage
// buffers.  Stage i's operand copy is issued as soon as its buffer is free
// (two stages ahead: right after the MMAs of stage i-2 have completed), so
// its latency hides behind a whole stage; while the MMAs of stage i run, the
// CTA generates stage i+1; then the partial of stage i is promoted into the
// running sum and stage i+1's MMAs are issued.  `copy(st, i)` (thread 0)
// issues the bulk copies of stage i into buffer st and arms its barrier;
// `gen(st, i)` writes the generated operand.  GEN_READS_COPY: the generator
// reads data the copy brings (the gather pass's galaxy coefficients), so
// every thread waits for the copy before generating; otherwise only thread
// 0 waits, before the MMAs.  Returns false on a timeout (uniform).
static_assert(TC_PROMO == 1, "the pipeline promotes after every stage");
template <bool GEN_READS_COPY, class Copy, class Gen>
__device__ __forceinline__ bool tc_kloop(TcSmem &s, uint32_t tmem, int nst, const int *err, bool *copy_out,
                                         uint32_t *fill, bool *mma_out, uint32_t *use, Copy copy, Gen gen) {
    const int t = threadIdx.x;
    bool bad = false;
    auto arm = [&](int st, int i) {
        if (t == 0) copy(st, i);
        copy_out[st] = true;
    };
    auto wait_copy = [&](int st) {
        if (GEN_READS_COPY || t == 0) bad |= !tc::mbar_wait(s.full + st, fill[st] & 1u);
        fill[st]++;
        copy_out[st] = false;
    };
    auto issue = [&](int st, int i) {  // after a barrier that follows gen(st, i)
        if (!GEN_READS_COPY) wait_copy(st);
        if (t == 0 && !bad) {
            tc::tc_fence_after();
            tc_issue(tmem, s.st[st], true);
            tc::mma_commit(s.mma + st);
        }
        mma_out[st] = true;
    };
    if (nst <= 0) return true;
    if (t == 0 && *reinterpret_cast<const volatile int *>(err)) bad = true;
    if (__syncthreads_or(bad)) return false;
    arm(0, 0);
    if (nst > 1) arm(1, 1);
    if (GEN_READS_COPY) wait_copy(0);
    gen(0, 0);
    tc::fence_async_smem();
    if (__syncthreads_or(bad)) return false;
    issue(0, 0);
    for (int i = 0; i < nst; i++) {
        const int st = i & 1, sn = st ^ 1;
        const bool more = i + 1 < nst;
        if (more) {
            if (GEN_READS_COPY) wait_copy(sn);
            gen(sn, i + 1);
            tc::fence_async_smem();
        }
        // the MMAs of stage i (and all before) have completed
        bad |= !tc::mbar_wait(s.mma + st, use[st] & 1u);
        use[st]++;
        mma_out[st] = false;
        if (t == 0 && *reinterpret_cast<const volatile int *>(err)) bad = true;
        if (__syncthreads_or(bad)) return false;
        tc::tc_fence_after();
        tc_promote(tmem, i == 0);
        tc::tc_fence_before();
        __syncthreads();
        if (i + 2 < nst) arm(st, i + 2);  // buffer st is free again
        if (more) issue(sn, i + 1);
    }
    return !__syncthreads_or(bad);
}

// ---- the Om-dependent operand of the norm pass: w'_a dv_j(z_a) 2^12 as
// (hi, lo) images per 64-point chunk, and dv_j(z_a) in FP32 for the gather
// epilogue.  w'_a = 1/2 at the two end points, 1 inside, 0 beyond the grid.
__global__ void k_tc_prep(DevCatalog c, TcBatch b, TcCols m) {
    const int j = blockIdx.y;                             // column, < TC_M
    const int a = blockIdx.x * blockDim.x + threadIdx.x;  // < nkc * 64
    if (a >= b.nkc * TC_K) return;
    const int nz = c.n_z;
    double v = 0.0, dvv = 0.0;
    if (j < m.n && a < nz) {
        dvv = chimd::dv_of(m.fwd[j], a * c.dz, m.Om[j]);
        v = (double)TC_SV * ((a == 0 || a == nz - 1) ? 0.5 : 1.0) * dvv;
        b.dvT[(size_t)j * nz + a] = (float)dvv;
    }
    const __half hi = __double2half(v);
    const __half lo = __double2half(v - (double)__half2float(hi));
    const int kc = a / TC_K, k = a % TC_K;
    char *img = reinterpret_cast<char *>(b.vimg) + (size_t)kc * 2 * TC_IMG;
    const uint32_t off = tc::sw128_offset((uint32_t)j, (uint32_t)k);
    *reinterpret_cast<__half *>(img + off) = hi;
    *reinterpret_cast<__half *>(img + TC_IMG + off) = lo;
}

// ---- norm pass: 1/Z_g(j) of 256 galaxy slots (four 64-blocks) per CTA.
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_norm(DevCatalog c, TcBatch b, int64_t blk0, int64_t nblk) {
    extern __shared__ char tc_raw[];
    TcSmem s = tc_smem(tc_raw);
    __shared__ int s_lo, s_hi;
    const int t = threadIdx.x, slot = t & (TC_N - 1), half = t / TC_N;  // two threads per galaxy slot
    const int64_t kb_rel = 4 * (int64_t)blockIdx.x + slot / 64;  // block of this slot, relative to the group
    // this slot's Gaussian coefficients (load time; c = 0 for no galaxy)
    const float2 cd = kb_rel < nblk ? c.tc_coef[(blk0 + kb_rel) * 64 + (slot & 63)] : make_float2(0.f, -1e4f);
    // grid points within 6 sigma, where its FP16 Gaussian can be nonzero
    int lo = 0, hi = -1;
    if (cd.x > 0.f) {
        const float k6 = 6.f * TC_S2L;
        lo = max(0, (int)floorf((cd.y - k6) / cd.x) - 1);
        hi = min(c.n_z - 1, (int)ceilf((cd.y + k6) / cd.x) + 1);
    }
    const bool valid = hi >= lo;
    if (t == 0) {
        s_lo = 1 << 30;
        s_hi = -1;
    }
    const uint32_t tmem = tc_setup(s, b.err);
    if (*s.flag) {
        tc_teardown(tmem);
        return;
    }
    if (valid) {
        atomicMin(&s_lo, lo);
        atomicMax(&s_hi, hi);
    }
    __syncthreads();
    const int kc0 = s_hi >= 0 ? s_lo / TC_K : 0, kc1 = s_hi >= 0 ? s_hi / TC_K : -1;
    const int nst = kc1 - kc0 + 1;  // stages (0 when no slot has a galaxy on the grid)
    bool copy_out[2] = {false, false}, mma_out[2] = {false, false};
    uint32_t fill[2] = {0u, 0u}, use[2] = {0u, 0u};
    auto copy = [&](int st, int i) {
        tc::mbar_expect_tx(s.full + st, TC_AST);
        tc::bulk_g2s(s.st[st], reinterpret_cast<const char *>(b.vimg) + (size_t)(kc0 + i) * TC_AST, TC_AST,
                     s.full + st);
    };
    auto gen = [&](int st, int i) {
        // row `slot`: this slot's Gaussian at 32 of the stage's 64 grid points
        char *brow = s.st[st] + TC_AST;
        const int kc = kc0 + i;
#pragma unroll
        for (int q = 4 * half; q < 4 * half + 4; q++) {
            float v[8];
            const float a0f = (float)(kc * TC_K + 8 * q);
#pragma unroll
            for (int e = 0; e < 8; e++) v[e] = tc_gauss(a0f + (float)e, cd);
            const uint4 pk = make_uint4(tc::pack_half2(v[0], v[1]), tc::pack_half2(v[2], v[3]),
                                        tc::pack_half2(v[4], v[5]), tc::pack_half2(v[6], v[7]));
            *reinterpret_cast<uint4 *>(brow + tc::sw128_offset((uint32_t)slot, (uint32_t)(8 * q))) = pk;
        }
    };
    const bool ok = tc_kloop<false>(s, tmem, nst, b.err, copy_out, fill, mma_out, use, copy, gen);
    if (!ok) {
        if (t == 0) atomicOr(b.err, 1);
        tc_drain(s, copy_out, fill, mma_out, use);
        tc_teardown(tmem);
        return;
    }
    // epilogue: stage the running sum's rows in shared memory, then the two
    // threads of a galaxy slot write 1/Z of 64 columns each as (hi, lo) FP16
    // into the gather pass's swizzled operand images (64 threads cover a
    // 128-byte row)
    float *T = reinterpret_cast<float *>(s.st[0]);
    tc::tc_fence_after();
    tc_stage_rows(tmem, nst > 0, T);
    __syncthreads();
    const int64_t kbg = 4 * (int64_t)blockIdx.x + slot / 64;
    if (kbg < nblk) {
        const int k = slot & 63;
        char *img = reinterpret_cast<char *>(b.cimg) + (size_t)kbg * 2 * TC_IMG;
        for (int r = half * (TC_M / 2); r < (half + 1) * (TC_M / 2); r++) {
            const float Zp = T[(size_t)r * TC_TROW + slot];
            // slots without a galaxy have Z = 0 exactly (zero Gaussians)
            const float cv = Zp > 0.f ? fminf(__fdividef(b.sc, Zp), 65504.f) : 0.f;
            const __half hh = __float2half_rn(cv);
            const __half ll = __float2half_rn(cv - __half2float(hh));
            const uint32_t off = tc::sw128_offset((uint32_t)r, (uint32_t)k);
            *reinterpret_cast<__half *>(img + off) = hh;
            *reinterpret_cast<__half *>(img + TC_IMG + off) = ll;
        }
    }
    tc_teardown(tmem);
}

// ---- gather pass: persistent over the group's items.
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_gather(DevCatalog c, TcBatch b, int64_t blk0, int64_t item0,
                                                             int64_t n_items, int *counter) {
    extern __shared__ char tc_raw[];
    TcSmem s = tc_smem(tc_raw);
    __shared__ int s_item;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int row = t & (TC_N - 1), half = t / TC_N;  // two threads per grid point
    const uint32_t tmem = tc_setup(s, b.err);
    if (*s.flag) {
        tc_teardown(tmem);
        return;
    }
    const int nz = c.n_z;
    const bool vec = (nz & 3) == 0;
    bool copy_out[2] = {false, false}, mma_out[2] = {false, false};
    uint32_t fill[2] = {0u, 0u}, use[2] = {0u, 0u};
    bool ok = true;
    while (true) {
        if (t == 0) s_item = *reinterpret_cast<const volatile int *>(b.err) ? INT32_MAX : atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int4 item = c.tc_items[item0 + it];
        const int slot = c.tc_islot[item0 + it];
        const int p = item.x, a0 = item.y * TC_N;
        const int kb_a = item.z;
        const int nst = item.w - item.z;
        const float af = (float)(a0 + row);  // this thread's grid point (row of the generated operand)
        auto copy = [&](int st, int i) {
            const int64_t kb = (int64_t)kb_a + i;  // relative to the group
            tc::mbar_expect_tx(s.full + st, TC_AST + 64 * sizeof(float2));
            tc::bulk_g2s(s.st[st], reinterpret_cast<const char *>(b.cimg) + (size_t)kb * TC_AST, TC_AST, s.full + st);
            tc::bulk_g2s(s.gp + st * 64, c.tc_coef + (blk0 + kb) * 64, 64 * sizeof(float2), s.full + st);
        };
        auto gen = [&](int st, int) {
            char *brow = s.st[st] + TC_AST;
            const float4 *gp = reinterpret_cast<const float4 *>(s.gp + st * 64);  // two galaxies per load
#pragma unroll 2
            for (int q = 4 * half; q < 4 * half + 4; q++) {
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    const float4 g2 = gp[(8 * q + e) / 2];
                    v[e] = tc_gauss(af, make_float2(g2.x, g2.y));
                    v[e + 1] = tc_gauss(af, make_float2(g2.z, g2.w));
                }
                const uint4 pk = make_uint4(tc::pack_half2(v[0], v[1]), tc::pack_half2(v[2], v[3]),
                                            tc::pack_half2(v[4], v[5]), tc::pack_half2(v[6], v[7]));
                *reinterpret_cast<uint4 *>(brow + tc::sw128_offset((uint32_t)row, (uint32_t)(8 * q))) = pk;
            }
        };
        ok = tc_kloop<true>(s, tmem, nst, b.err, copy_out, fill, mma_out, use, copy, gen);
        if (!ok) break;
        // epilogue: rows staged in shared memory, then each warp writes 8
        // rows: G = dv_j(z_a) gfac S into the profile of column j, or the raw
        // sums into the item's partial slot
        float *T = reinterpret_cast<float *>(s.st[0]);
        tc::tc_fence_after();
        tc_stage_rows(tmem, nst > 0, T);
        __syncthreads();
        for (int rr = 0; rr < TC_M / (TC_THREADS / 32); rr++) {
            const int j = w * (TC_M / (TC_THREADS / 32)) + rr;
            const float *row = T + (size_t)j * TC_TROW;
            if (slot >= 0) {
                float *dst = b.part + ((size_t)slot * TC_M + j) * TC_N;
                reinterpret_cast<float4 *>(dst)[lane] = reinterpret_cast<const float4 *>(row)[lane];
                reinterpret_cast<float4 *>(dst)[lane + 32] = reinterpret_cast<const float4 *>(row)[lane + 32];
            } else if (j < b.n_cols && b.out[j]) {
                float *o = b.out[j] + (size_t)p * nz;
                const float *dv = b.dvT + (size_t)j * nz;
                for (int h2 = 0; h2 < 2; h2++) {
                    const int aa = a0 + 4 * (lane + 32 * h2);
                    const float4 x = reinterpret_cast<const float4 *>(row)[lane + 32 * h2];
                    if (vec && aa + 3 < nz) {
                        const float4 d4 = *reinterpret_cast<const float4 *>(dv + aa);
                        *reinterpret_cast<float4 *>(o + aa) = make_float4(
                            d4.x * b.gfac * x.x, d4.y * b.gfac * x.y, d4.z * b.gfac * x.z, d4.w * b.gfac * x.w);
                    } else {
                        const float xs[4] = {x.x, x.y, x.z, x.w};
                        for (int e = 0; e < 4; e++)
                            if (aa + e < nz) o[aa + e] = dv[aa + e] * b.gfac * xs[e];
                    }
                }
            }
        }
        tc::tc_fence_before();
        __syncthreads();
    }
    if (!ok) {
        if (t == 0) atomicOr(b.err, 1);
        tc_drain(s, copy_out, fill, mma_out, use);
    }
    tc_teardown(tmem);
}

// ---- partial sums of split items, added in slot order: block (reduction,
// group of 8 columns), thread = grid point of the tile.
constexpr int TC_RED_COLS = 8;
__global__ void k_tc_reduce(DevCatalog c, TcBatch b, int64_t red0) {
    const int4 r = c.tc_reds[red0 + blockIdx.x];  // (pixel, grid tile, first slot, slots)
    const int n = threadIdx.x, nz = c.n_z;
    const int aa = r.y * TC_N + n;
    const int j0 = blockIdx.y * TC_RED_COLS;
#pragma unroll
    for (int jj = 0; jj < TC_RED_COLS; jj++) {
        const int j = j0 + jj;
        if (j >= b.n_cols) break;
        float sacc = 0.f;
        for (int q = 0; q < r.w; q++) sacc += b.part[((size_t)(r.z + q) * TC_M + j) * TC_N + n];
        float *o = b.out[j];
        if (o && aa < nz) o[(size_t)r.x * nz + aa] = b.dvT[(size_t)j * nz + aa] * b.gfac * sacc;
    }
}

}  // namespace

size_t tc_scratch_bytes(const DevCatalog &c, const TcHost &h) {
    if (!c.tc_ok) return 0;
    const size_t nkc = (size_t)(c.n_z + TC_K - 1) / TC_K;
    auto up = [&](size_t x) { return (std::max<size_t>(x, 16) + 255) & ~(size_t)255; };
    return up(nkc * TC_AST) + up(sizeof(float) * TC_COLS * (size_t)c.n_z) + up((size_t)h.max_gblk * TC_AST) +
           up(sizeof(float) * (size_t)h.max_slots * TC_M * TC_N) + up(16 * sizeof(int));
}

int launch_galaxy_profile_tc(const DevCatalog &c, const TcHost &h, const TcCols &m, float *const *out, char *scratch,
                             cudaStream_t st) {
    if (!c.tc_ok || m.n < 1 || m.n > TC_COLS) return CHIMERA_ERR_INVALID_ARG;
    const size_t nkc = (size_t)(c.n_z + TC_K - 1) / TC_K;
    auto up = [&](size_t x) { return (std::max<size_t>(x, 16) + 255) & ~(size_t)255; };
    TcBatch b{};
    b.n_cols = m.n;
    b.nkc = (int)nkc;
    b.sc = c.tc_sc;
    b.gfac = (float)((double)TC_SV / (c.dz * (double)c.tc_sc));
    char *q = scratch;
    b.vimg = reinterpret_cast<uint4 *>(q);
    q += up(nkc * TC_AST);
    b.dvT = reinterpret_cast<float *>(q);
    q += up(sizeof(float) * TC_COLS * (size_t)c.n_z);
    b.cimg = reinterpret_cast<uint4 *>(q);
    q += up((size_t)h.max_gblk * TC_AST);
    b.part = reinterpret_cast<float *>(q);
    q += up(sizeof(float) * (size_t)h.max_slots * TC_M * TC_N);
    b.err = reinterpret_cast<int *>(q);
    for (int j = 0; j < TC_COLS; j++) b.out[j] = j < m.n ? out[j] : nullptr;
    cudaMemsetAsync(b.err, 0, 16 * sizeof(int), st);
    k_tc_prep<<<dim3((unsigned)((nkc * TC_K + 127) / 128), (unsigned)TC_M), 128, 0, st>>>(c, b, m);
    // the opt-in to more than 48 KB of dynamic shared memory is per device
    cudaFuncSetAttribute(k_tc_norm, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    cudaFuncSetAttribute(k_tc_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    int nsm = 148;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    const int ng = (int)h.gblk.size() - 1;
    for (int gi = 0; gi < ng; gi++) {
        const int64_t blk0 = h.gblk[gi], nblk = h.gblk[gi + 1] - h.gblk[gi];
        const int64_t it0 = h.gitem[gi], nit = h.gitem[gi + 1] - h.gitem[gi];
        const int64_t rd0 = h.gred[gi], nrd = h.gred[gi + 1] - h.gred[gi];
        if (nblk > 0) k_tc_norm<<<(unsigned)((nblk + 3) / 4), TC_THREADS, TC_SMEM, st>>>(c, b, blk0, nblk);
        int *counter = b.err + 4 + (gi & 3);
        cudaMemsetAsync(counter, 0, sizeof(int), st);
        if (nit > 0) {
            const unsigned grid = (unsigned)std::min<int64_t>(nit, nsm);
            k_tc_gather<<<grid, TC_THREADS, TC_SMEM, st>>>(c, b, blk0, it0, nit, counter);
        }
        if (nrd > 0)
            k_tc_reduce<<<dim3((unsigned)nrd, (unsigned)((m.n + TC_RED_COLS - 1) / TC_RED_COLS)), TC_N, 0, st>>>(c, b,
                                                                                                          rd0);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CHIMERA_OK : cuda_check(e, "tensor-core galaxy profile");
}

// Load-time plan: eligibility, the padded block list, groups of pixels whose
// operand images fit the scratch, and the gather items.  zs, ss: the galaxies'
// stored (z, sigma) as the kernels decode them, sorted by z inside a pixel;
// smax: the widest stored sigma of each pixel.
void tc_plan(int64_t np, const int64_t *goff, const float *zs, const float *ss, const float *smax, int n_z,
             double dz, bool incomplete, int kde_mode, DevCatalog &c, TcHost &h, std::vector<int2> &blk,
             std::vector<float2> &coef, std::vector<int4> &items, std::vector<int32_t> &islot,
             std::vector<int4> &reds) {
    c.tc_ok = 0;
    blk.clear();
    coef.clear();
    items.clear();
    islot.clear();
    reds.clear();
    const int64_t ng = goff[np];
    if (ng < TC_MIN_GAL || incomplete || kde_mode == CHIMERA_KDE_3D) return;
    double smin = 1e300;
    for (int64_t g = 0; g < ng; g++) smin = std::min(smin, (double)ss[g]);
    if (!(smin >= TC_SIGMA_MIN) || !(smin >= 8.0 * dz)) return;
    std::vector<int64_t> pblk(np + 1, 0);  // blocks of each pixel
    for (int64_t p = 0; p < np; p++) {
        const int64_t nb = (goff[p + 1] - goff[p] + 63) / 64;
        if (nb > TC_GRP_BLK) return;  // a pixel larger than a group: FP32 kernels
        pblk[p + 1] = pblk[p] + nb;
    }
    if (pblk[np] > (int64_t)INT32_MAX / 2) return;
    // scale of 1/Z': Z'' = dz sum_a w'_a N dv >= ~0.05 sigma_min^3 (a galaxy at
    // z = 0: dv ~ z^2 over [0, sigma]), Z' = 2^12 Z'' / dz; c = sc / Z' <= 2^15
    const double zmin = (double)TC_SV / dz * 0.05 * smin * smin * smin;
    c.tc_sc = (float)std::exp2(std::floor(std::log2(32768.0 * zmin)));
    const int ntile = (n_z + TC_N - 1) / TC_N;
    const float dz32 = (float)dz;
    h.gblk.assign(1, 0);
    h.gitem.assign(1, 0);
    h.gred.assign(1, 0);
    h.max_gblk = 0;
    h.max_slots = 0;
    int64_t gb = 0;      // blocks in the current group
    int32_t gslots = 0;  // partial slots in the current group
    struct It {
        int4 v;
        int32_t slot;
        int64_t work;
    };
    std::vector<It> git;
    std::vector<int4> gred;
    auto close_group = [&]() {
        // heaviest first; a pixel's grid tiles stay together (they read the
        // same operand images)
        std::stable_sort(git.begin(), git.end(), [](const It &x, const It &y) { return x.work > y.work; });
        for (auto &x : git) {
            items.push_back(x.v);
            islot.push_back(x.slot);
        }
        for (auto &r : gred) reds.push_back(r);
        h.max_gblk = std::max(h.max_gblk, gb);
        h.max_slots = std::max(h.max_slots, gslots);
        h.gblk.push_back((int64_t)blk.size());
        h.gitem.push_back((int64_t)items.size());
        h.gred.push_back((int64_t)reds.size());
        git.clear();
        gred.clear();
        gb = 0;
        gslots = 0;
    };
    for (int64_t p = 0; p < np; p++) {
        const int64_t nb = pblk[p + 1] - pblk[p];
        if (gb + nb > TC_GRP_BLK) close_group();
        const int64_t b0 = gb;  // the pixel's first block, relative to the group
        for (int64_t i = 0; i < nb; i++) {
            blk.push_back(make_int2((int)p, (int)(goff[p] + 64 * i)));
            // the Gaussian coefficients of the block's 64 slots: a galaxy
            // with no grid point within 6 sigma (mixed-path window) drops out
            for (int k = 0; k < 64; k++) {
                const int64_t g = goff[p] + 64 * i + k;
                float2 cd = make_float2(0.f, -1e4f);
                if (g < goff[p + 1]) {
                    const float zg = zs[g], sg = ss[g], kw = KWG32 * sg;
                    const float a0 = std::ceil((zg - kw) * (1.f / dz32)), a1 = std::floor((zg + kw) * (1.f / dz32));
                    if (a1 >= 0.f && a0 <= (float)(n_z - 1) && a1 >= a0) {
                        const float isg = 1.f / sg;
                        cd = make_float2(dz32 * isg * TC_S2L, zg * isg * TC_S2L);
                    }
                }
                coef.push_back(cd);
            }
        }
        gb += nb;
        // a galaxy's window is within KWG32 sigma of its z; two grid steps of
        // margin cover the rounding of the window's end points
        const float reach = KWG32 * smax[p] * 1.001f + 2.f * dz32;
        const float *zb = zs + goff[p], *ze = zs + goff[p + 1];
        for (int t = 0; t < ntile; t++) {
            const float zlo = (float)(t * TC_N) * dz32 - reach, zhi = (float)(t * TC_N + TC_N - 1) * dz32 + reach;
            const int64_t gl = std::lower_bound(zb, ze, zlo) - zb;
            const int64_t gr = std::upper_bound(zb, ze, zhi) - zb;
            const int64_t ka = gl / 64, kbe = gr > gl ? (gr + 63) / 64 : ka;
            const int64_t nk = kbe - ka;
            if (nk <= TC_KSPLIT) {
                git.push_back({make_int4((int)p, t, (int)(b0 + ka), (int)(b0 + kbe)), -1, nk});
            } else {
                const int ns = (int)((nk + TC_KSPLIT - 1) / TC_KSPLIT);
                for (int q = 0; q < ns; q++) {
                    const int64_t x0 = ka + (int64_t)q * TC_KSPLIT, x1 = std::min(kbe, x0 + TC_KSPLIT);
                    git.push_back({make_int4((int)p, t, (int)(b0 + x0), (int)(b0 + x1)), gslots + q, x1 - x0});
                }
                gred.push_back(make_int4((int)p, t, gslots, ns));
                gslots += ns;
            }
        }
    }
    close_group();
    c.tc_nblk = (int64_t)blk.size();
    c.tc_ok = 1;
}

}  // namespace chim
