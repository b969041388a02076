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
// for every hyperpoint, and processed in warp groups of up to 128 neighbours
// (fixed at load time).
//
// Mixed kernel: for a group with origin grid index t_o the Gaussian
// factorises on the uniform grid,
//   exp(-(u - ds tau)^2) = exp(-u^2) * B^tau * C_tau,  B = exp(2 u ds),
//   C_tau = exp(-ds^2 tau^2), u = (z_j - z_o)/(sqrt2 b), ds = dz/(sqrt2 b),
// tau = a - t_o, so with the per-group table D_tau = C_tau w_a F(z_a) G(z_a)
// in shared memory the sum over the grid is a polynomial in B (and one in
// 1/B for tau < 0), evaluated by Horner's rule: one FFMA per (sample, grid
// point), with D read as a broadcast float4 and up to four samples per lane.
// Groups wider than 16 b use a per-lane Horner chain on their own windows;
// kernels narrower than ~0.7 grid steps (ds > 2) use direct exponentials.
//
// FP64 kernel: the plain form, one exp per grid point and sample within
// +-9 b, every quantity in double.
//
// Both kernels keep each KDE on its support, the grid segment between its
// first and last sample widened by KDE_MARGIN bandwidths (Sec. 2.3).
#include <math_constants.h>

#include "internal.cuh"
#include "mass.cuh"

namespace chim {

namespace {

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Compensated sums (per-event Kahan-style summation of the mixed path):
// TwoSum gives the exact rounding error e of s = a + b (s + e = a + b
// exactly, whatever the order of a and b), so the butterfly below carries
// each partial sum with its error and every lane ends with the same value.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}
__device__ __forceinline__ float warp_sum_c(float v) {
    float c = 0.f;
    for (int o = 16; o > 0; o >>= 1) {
        const float vo = __shfl_xor_sync(0xffffffffu, v, o), co = __shfl_xor_sync(0xffffffffu, c, o);
        float sm, e;
        two_sum(v, vo, sm, e);
        v = sm;
        c = __fadd_rn(__fadd_rn(c, co), e);
    }
    return __fadd_rn(v, c);
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

// ln I of a mixed event kernel from its raw FP32 integral I' (grid factor in
// units of F_scale, without the 1/b and catalog constants):
//   ln I = ln I' - ln b + ln(dz F_scale / (N_gal,tot sqrt(2 pi))),
// the last term per point in FP64 (hp.ln_k0); ln I' and ln b are split as
// m 2^e so that the FP32 logs only see m in [0.5, 1) (absolute error
// ~1e-7, the order of the FP32 sums themselves).
// ln_k0 carries the Gaussian's 1/sqrt(2 pi); the Epanechnikov kernel's
// normalisation 3/(4 sqrt5 b) adds ln(3 sqrt(2 pi) / (4 sqrt5)).
__device__ __forceinline__ double ln_mixed(float I, float b, double ln_k0, bool epan = false) {
    if (!(I > 0.f)) return -CUDART_INF;
    int eI, eb;
    const float mI = frexpf(I, &eI), mb = frexpf(b, &eb);
    return ln_k0 + (epan ? -0.17346249546415843 : 0.0) + (double)(logf(mI) - logf(mb)) +
           (double)(eI - eb) * 0.69314718055994530942;
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

// Shared layout of the mixed kernel (nw warps per block).
struct MixLayout {
    int ns_pad, nz_pad, seg_pad, gmax_pad, nw;
    __host__ __device__ static int pad4(int x) { return (x + 3) & ~3; }
    __host__ __device__ MixLayout(int max_ns, int nz, int max_seg, int max_groups, int nw_) {
        ns_pad = pad4(max_ns);
        nz_pad = pad4(nz);
        seg_pad = pad4(max_seg + 1);
        gmax_pad = pad4(max_groups);
        nw = nw_;
    }
    // int4: group metadata and descriptors (two per group); floats: zs, ws,
    // Fs, D tables, C table (both signs of tau), group prefactors / results;
    // staged segment offsets and prefactors; the reduction scratch
    __host__ __device__ size_t bytes() const {
        return sizeof(int4) * 2 * (size_t)gmax_pad +
               sizeof(float) * (2 * (size_t)ns_pad + nz_pad + (size_t)nw * DCAP + 2 * CCAP + gmax_pad) +
               sizeof(double) * 2 * (size_t)seg_pad + sizeof(double) * (8 + nw * 8);
    }
};

// The per-sample sums are polynomials in B = exp(2 u ds):
// The per-sample sums are polynomials in B = exp(2 u ds):
//   sum_{tau >= 0} D_tau B^tau      and      sum_{tau >= 1} D_-tau B^-tau,
// evaluated by Horner's rule from the highest power down: one FMA per
// (sample, grid point).  The intermediates are partial sums divided by
// exp(-u^2) B^tau, so they stay within the float range for |u| <= 3.1.
// The two chains of a sample run side by side as one float2 (the forward
// and backward partial sums, multipliers B and 1/B), one paired FFMA2 of
// sm_100+ per step of both, on a table that stores the coefficients of a
// step in pairs: P_k = (D_k, D_-k-1), k in [0, 4 nq), read as float4 from
// the top down.  Each element rounds as a scalar fmaf would, so the sums
// are those of two scalar chains.
// R samples per lane (lane, lane+32, ...) of a group share one table; each
// sample's weight and its factor exp(-u^2) are folded into one coefficient
// before the chains.
template <int R>
__device__ __forceinline__ float union_samples(const float *D, int nq, const float *z, const float *w, int cnt,
                                               int lane, float zo, float inv_s2b, float ds, float iscale) {
    float cw[R];
    float2 m[R], s[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int j = lane + 32 * r;
        const bool in = j < cnt;
        const float u = in ? (z[j] - zo) * inv_s2b : 0.f;
        // iscale: 1 or 2^-29, exact (it undoes the table's power-of-two scale)
        // SFU exponentials here: measured on the benchmark catalogs, the
        // accurate expc gave no smaller shared error at this spot (the per-
        // sample factors' errors differ between samples) and cost 6 % of K4
        cw[r] = in ? w[j] * (__expf(-u * u) * iscale) : 0.f;
        m[r] = make_float2(__expf(2.f * u * ds), __expf(-2.f * u * ds));
        s[r] = make_float2(0.f, 0.f);
    }
    const float4 *P4 = reinterpret_cast<const float4 *>(D);
#pragma unroll 4
    for (int it = nq - 1; it >= 0; it--) {
        const float4 q1 = P4[2 * it + 1], q0 = P4[2 * it];  // k = 4 it + 2, +3 and k = 4 it, +1
#pragma unroll
        for (int r = 0; r < R; r++) s[r] = __ffma2_rn(s[r], m[r], make_float2(q1.z, q1.w));
#pragma unroll
        for (int r = 0; r < R; r++) s[r] = __ffma2_rn(s[r], m[r], make_float2(q1.x, q1.y));
#pragma unroll
        for (int r = 0; r < R; r++) s[r] = __ffma2_rn(s[r], m[r], make_float2(q0.z, q0.w));
#pragma unroll
        for (int r = 0; r < R; r++) s[r] = __ffma2_rn(s[r], m[r], make_float2(q0.x, q0.y));
    }
    float v = 0.f;
#pragma unroll
    for (int r = 0; r < R; r++) v = fmaf(cw[r], fmaf(m[r].y, s[r].y, s[r].x), v);
    return v;
}

// The paired table of union_samples for a group with origin t_o (a multiple
// of 4; G and Fs 16-byte aligned): D_tau = C_|tau| scale F'(z_a) G(z_a) at
// a = t_o + tau, zero outside [A0, A1].  Each lane builds four forward
// (tau = 4i .. 4i+3) and four backward (tau = -4i-4 .. -4i-1) entries from
// one 128-bit load of each operand and interleaves them into P.
__device__ __forceinline__ void stage_table4(float *D, int nq, int t_o, int A0, int A1, const float *G,
                                             const float *Fs, const float *CT, float scale, int lane) {
    float4 *D4 = reinterpret_cast<float4 *>(D);
    auto quad = [&](int a4, const float *cq) {
        float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a4 + 3 >= A0 && a4 <= A1) {
            // a4 >= A0 - 3 >= -3 and a4 is a multiple of 4, so a4 >= 0; a4 <= A1 < nz
            float4 g = __ldg(reinterpret_cast<const float4 *>(G + a4));
            const float4 f = *reinterpret_cast<const float4 *>(Fs + a4);
            const float4 cc = *reinterpret_cast<const float4 *>(cq);
            val = make_float4(cc.x * scale * f.x * g.x, cc.y * scale * f.y * g.y, cc.z * scale * f.z * g.z,
                              cc.w * scale * f.w * g.w);
            if (a4 < A0 || a4 + 3 > A1) {
                if (a4 < A0 || a4 > A1) val.x = 0.f;
                if (a4 + 1 < A0 || a4 + 1 > A1) val.y = 0.f;
                if (a4 + 2 < A0 || a4 + 2 > A1) val.z = 0.f;
                if (a4 + 3 < A0 || a4 + 3 > A1) val.w = 0.f;
            }
        }
        return val;
    };
#pragma unroll 2
    for (int i = lane; i < nq; i += 32) {
        const float4 hf = quad(t_o + 4 * i, CT + 4 * i);          // tau = 4i .. 4i+3
        const float4 hb = quad(t_o - 4 * i - 4, CT - 4 * i - 4);  // tau = -4i-4 .. -4i-1
        D4[2 * i] = make_float4(hf.x, hb.w, hf.y, hb.z);
        D4[2 * i + 1] = make_float4(hf.z, hb.y, hf.w, hb.x);
    }
}

// The same table without the 16-byte alignment (n_z not a multiple of 4):
// element 2k holds D_k and element 2k+1 holds D_-k-1; the profile loads of
// up to eight entries per lane are issued before any of them is used.
__device__ __forceinline__ void stage_table_p(float *D, int nq, int t_o, int A0, int A1, const float *G,
                                              const float *Fs, const float *CT, float scale, int lane) {
    const int len = 8 * nq;
    for (int i0 = 0; i0 < len; i0 += 8 * 32) {
        float gv[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int idx = i0 + u * 32 + lane;
            const int k = idx >> 1, tau = (idx & 1) ? -k - 1 : k;
            const int a = t_o + tau;
            gv[u] = (idx < len && a >= A0 && a <= A1) ? __ldg(G + a) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int idx = i0 + u * 32 + lane;
            if (idx < len) {
                const int k = idx >> 1, tau = (idx & 1) ? -k - 1 : k;
                const int a = t_o + tau;
                const float f = (a >= A0 && a <= A1) ? Fs[a] : 0.f;
                D[idx] = f * gv[u] * (CT[tau < 0 ? -tau : tau] * scale);
            }
        }
    }
}
// group's range, each sums the samples whose window holds it (one SFU
// exponential per pair); cheaper than a table for so few samples.
constexpr int SMALL_CNT = 6;  // measured with the paired Horner chains: 0 and 6 equal, 12 slower by 1.6 %
__device__ __forceinline__ float small_group(const float *z, const float *w, int cnt, int A0, int A1,
                                             const float *G, const float *Fs, float dz, float dz_lo,
                                             float inv_s2b, float halfk, int lane) {
    float acc = 0.f;
#pragma unroll 2
    for (int a = A0 + lane; a <= A1; a += 32) {
        const float za = fmaf((float)a, dz, (float)a * dz_lo);
        const float h = Fs[a] * __ldg(G + a);
        float k = 0.f;
        for (int j = 0; j < cnt; j++) {
            const float d = za - z[j];
            const float x = d * inv_s2b, x2 = x * x;
            // SFU ex2 with log2 e as a pair (these groups hold ~0.5 % of the
            // pairs: the SFU's own mean error is immaterial here)
            const float e = ex2(fmaf(-x2, L2E_HI, -x2 * L2E_LO));
            k = fabsf(d) <= halfk ? fmaf(w[j], e, k) : k;
        }
        acc = fmaf(k, h, acc);
    }
    return acc;
}

// Asynchronous 16-byte global -> shared copies (cp.async, completion per
// thread by commit groups).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}


// Warp-cooperative staging of the profile product of the per-lane path:
// for idx < len and grid point a = a_first + idx, D[idx] = F'(z_a) G(z_a)
// (F' carrying the trapezoid weight), zero outside [A0, A1].  The profile
// loads of up to eight entries per lane are issued before any of them is
// used, so a table costs about one memory latency per 256 entries instead
// of one per 32.
__device__ __forceinline__ void stage_table(float *D, int len, int a_first, int A0, int A1, const float *G,
                                            const float *Fs, int lane) {
    for (int i0 = 0; i0 < len; i0 += 8 * 32) {
        float gv[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int idx = i0 + u * 32 + lane;
            const int a = a_first + idx;
            gv[u] = (idx < len && a >= A0 && a <= A1) ? __ldg(G + a) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int idx = i0 + u * 32 + lane;
            if (idx < len) {
                const int a = a_first + idx;
                const float f = (a >= A0 && a <= A1) ? Fs[a] : 0.f;
                D[idx] = f * gv[u];
            }
        }
    }
}

// Per-lane path for a sparse group: every lane runs its own window around
// the grid point ts nearest to its sample, exp(-(u - ds t)^2) =
// exp(-u^2) B^t C_t with |u| <= ds/2, as two Horner chains in B and 1/B
// over the group's H' (staged with zero padding, so no bounds tests).
__device__ __forceinline__ float lane_chain(const float *Hc, const float *CT, int Tw, float z,
                                            int ts, float dz, float dz_lo, float inv_s2b, float ds) {
    const float u = (z - fmaf((float)ts, dz, (float)ts * dz_lo)) * inv_s2b;
    const float A = __expf(-u * u), B = __expf(2.f * u * ds), Bi = __expf(-2.f * u * ds);
    float af = CT[Tw] * Hc[Tw], ab = CT[Tw + 1] * Hc[-Tw - 1];
#pragma unroll 2
    for (int t = Tw - 1; t >= 0; t--) {
        const float c = CT[t], c1 = CT[t + 1];
        af = fmaf(af, B, c * Hc[t]);
        ab = fmaf(ab, Bi, c1 * Hc[-1 - t]);
    }
    return A * fmaf(Bi, ab, af);
}

// K2 (mixed): reweighting of every PE sample for hyperpoints h0 .. h0+nh-1,
// one block per (event, point): z_j and w_j go to the tile buffer (FP32,
// 16-byte aligned per event), the one-pass moments about the redshift of
// the event's median d_L give the FP32 Scott bandwidth.  Many small blocks
// keep the SMs full while the loads of the inverse-table nodes are in flight
// (measured on the 300-event catalog: 128 threads with eight blocks per SM
// 0.177 ms, 256 with four 0.190, 96 with ten 0.196, 64 with sixteen 0.244).
// Each thread has three samples' loads in flight (0.161 ms against 0.171 ms
// with two, whose register allocation at the 64-register cap spilled a few
// bytes; four spill more).
constexpr int RW_THREADS = 128;
#ifndef CHIM_RW_INFLIGHT
#define CHIM_RW_INFLIGHT 3
#endif
#ifndef CHIM_RW_MINB
#define CHIM_RW_MINB 8
#endif
#ifndef CHIM_RW_SMEMQ
#define CHIM_RW_SMEMQ 0
#endif
constexpr int RW_INFLIGHT = CHIM_RW_INFLIGHT;  // samples per thread in flight
constexpr int RW_SPEC_CAP = 256;               // deferred (FP64-weight) samples listed per block
constexpr int RW_CHUNKS = CHIMERA_MAX_SAMPLES_PER_EVENT / 32;  // 32-sample chunks of the largest event
static_assert(RW_CHUNKS % RW_THREADS == 0, "chunks spread evenly over the threads");
constexpr int RW_MINB = CHIM_RW_MINB;          // resident blocks per SM asked of the compiler
// 1 / [(1+z)^3 |d d_L^gw/dz|] at a sample (Eq. jacobian), FP32, from its
// d_L (D_c = d_L / ((1+z) Xi)) and lz = log2(1+z).
__device__ __forceinline__ float jac_inv32(const HP &hp, float z, float lz, float d) {
    const float ap = 1.f + z, rap = __fdividef(1.f, ap);
    const float pw = ex2(-hp.n32 * lz);  // (1+z)^-n
    const float xi = hp.xi0_32 + (1.f - hp.xi0_32) * pw;
    const float dxi = -hp.n32 * (1.f - hp.xi0_32) * pw * rap;
    const float Dc = __fdividef(d * rap, xi);
    const float rE = rsqrtf(hp.om32 * ap * ap * ap + 1.f - hp.om32);
    const float J = (Dc + ap * hp.cH32 * rE) * xi + ap * Dc * dxi;
    return __fdividef(rap * rap * rap, fabsf(J));
}

// JAC: the per-sample Jacobian option (a template parameter so that the
// default kernel keeps its registers and occupancy).
// The event's slice of the inverse tables (its samples' intervals
// kmin .. kmax, z and log2(1+z) node pairs) is staged in shared memory when
// it fits RW_STAGE_MAX intervals, so that each sample's table lookup is a
// shared-memory read instead of a global gather that waits on the sample's
// own load.
constexpr int RW_STAGE_MAX = 768;  // 24 KB of node pairs per block
template <bool JAC, bool STAGE>
__global__ void __launch_bounds__(RW_THREADS, RW_MINB) k_reweight(DevCatalog c, CallPtrs p, int h0, int nh) {
    __shared__ double red[8 + (RW_THREADS / 32) * 8];
    extern __shared__ float4 rw_nodes[];  // STAGE: [2 x nk] node pairs of z, then of log2(1+z)
    const int hl = blockIdx.x % nh, h = h0 + hl;
    const int ev = blockIdx.x / nh;  // natural order: consecutive blocks stream neighbouring samples
    const int tid = threadIdx.x;
    const HP &hp = p.hp[h];
    if (hp.status & (CHIMERA_PT_OUT_OF_SUPPORT | CHIMERA_PT_NONMONOTONE)) return;
#if CHIM_RW_SMEMQ
    __shared__ WParams sq;
    if (tid == 0) sq = w_params(hp);
    __syncthreads();
    const WParams &q = sq;
#else
    const WParams q = w_params(hp);
#endif
    const int64_t s0 = c.ev_soff[ev];
    const int ns = (int)(c.ev_soff[ev + 1] - s0);
    float *zd = p.zw + (size_t)hl * 2 * c.n_zpad + c.ev_zoff[ev];
    float *wd = zd + c.n_zpad;
    const float4 *inv = p.inv32 + (size_t)h * NU;
    const float4 *linv = p.linv32 + (size_t)h * NU;
    int koff = 0;
    if (STAGE) {
        const int2 kr = c.ev_krange[ev];
        const int nk = kr.y - kr.x + 1;
        for (int i = tid; i < nk; i += RW_THREADS) {
            rw_nodes[i] = __ldg(inv + kr.x + i);
            rw_nodes[nk + i] = __ldg(linv + kr.x + i);
        }
        __syncthreads();
        inv = rw_nodes;
        linv = rw_nodes + nk;
        koff = kr.x;
    }
    const float4 *sp = c.s32 + s0;
    float zref;
    {
        const float2 zr = c.ev_ref[ev];
        const int k = __float_as_int(zr.x);
        const bool ok = (k < q.kv) || (k == q.kv && zr.y <= q.fv);
        zref = ok ? chimd::hermite4(inv[k - koff], zr.y) : 0.f;
        if (!isfinite(zref)) zref = 0.f;
    }
    float m[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // W1, Wd, Wd2, W2, n, Sd, Sd2
    const float dtop = (float)c.d_top;
    // one sample: table coordinate -> z (Hermite on the node pair), log2
    // source masses, weight relative to the point's shared normalisation
    // (mass.cuh), moments; invalid samples (beyond d_L^gw(10)) get z = inf
    // and w = 0 and stay out of the moments.  Near a mass edge the in-range
    // test is taken in FP64 from the sample's FP64 distance and masses.
    // Samples whose weight needs FP64 (guard bands at the mass edges, the
    // corner band above m_min; a few in a thousand at most) are deferred to
    // a list and taken after the loop, so that the loop itself carries no
    // FP64 call (whose register saves would cost every sample).
    // Each deferred sample sets its bit in the mask of its 32-sample chunk
    // (an atomic OR: the result does not depend on the order); after the
    // loop the masks give the list of deferred samples in index order.
    __shared__ unsigned s_smask[RW_CHUNKS];
    __shared__ int s_spec[RW_SPEC_CAP];
    __shared__ int s_wtot[RW_THREADS / 32];
    for (int cc = tid; cc < RW_CHUNKS; cc += RW_THREADS) s_smask[cc] = 0u;
    __syncthreads();
    auto jac = [&](float w, float z, float lz, const float4 &sv) {
        if (JAC) {  // the Jacobian on the sample (the moments keep w)
            const float t = (float)__float_as_int(sv.x) + sv.y, u = t * (1.f / NU);
            w *= jac_inv32(hp, z, lz, dtop * u * u);
        }
        return w;
    };
    auto sample = [&](const float4 &sv, const float4 &nd, const float4 &ndl, const float2 &slo, int j) {
        const float z = chimd::hermite4(nd, sv.y);
        const bool ok = z < CUDART_INF_F;  // false for inf and NaN
        const float lz = chimd::hermite4(ndl, sv.y);  // log2(1+z) from its own node pairs
        const LogMass lm = log_mass(q, sv.z, sv.w, slo, lz);
        const bool inr = w_in_range(lm);
        float w = 0.f;
        if (ok && (w_needs64(lm) || (inr && lm.d1 < W_FP64))) {
            atomicOr(&s_smask[j >> 5], 1u << (j & 31));
        } else if (ok && inr) {
            // rcp.approx: mean relative error +4e-9 on B300 (measured), no shared bias to speak of
            const WQuot wq = mass_weight_rel(q, lm);
            w = __fdividef(wq.num, wq.den);
            w = w > 0.f ? w : 0.f;
        }
        const float d = ok ? z - zref : 0.f;
        const float wd_ = w * d;
        m[0] += w; m[1] += wd_; m[2] = fmaf(wd_, d, m[2]); m[3] = fmaf(w, w, m[3]);
        m[4] += ok ? 1.f : 0.f; m[5] += d; m[6] = fmaf(d, d, m[6]);
        zd[j] = ok ? z : CUDART_INF_F;
        wd[j] = ok ? jac(w, z, lz, sv) : 0.f;
    };
    auto node = [&](const float4 &sv, float4 &nl) {
        const int k = __float_as_int(sv.x);
        const bool valid = (k < q.kv) || (k == q.kv && sv.y <= q.fv);
        nl = valid ? linv[k - koff] : make_float4(0.f, 0.f, 0.f, 0.f);
        return valid ? inv[k - koff] : make_float4(CUDART_INF_F, 0.f, 0.f, 0.f);
    };
    // the deferred weight of sample j (in FP64 where needed) and its moments
    auto special = [&](int j) {
        const float4 sv = __ldg(sp + j);
        float4 nl;
        const float4 nd = node(sv, nl);
        const float z = chimd::hermite4(nd, sv.y), lz = chimd::hermite4(nl, sv.y);
        LogMass lm = log_mass(q, sv.z, sv.w, __ldg(c.s32lo + s0 + j), lz);
        float w = 0.f;
        if (w_needs64(lm)) {
            w = mass_weight_rel64(p, h, hp, c.inv_d_top, c.beta, z, c.sd64[s0 + j], c.sm1_64[s0 + j], c.sm2_64[s0 + j]);
        } else {
            lm.d1 = corner_d1(p, h, hp, c.inv_d_top, z, c.sd64[s0 + j], c.sm1_64[s0 + j], lm.d1);
            const WQuot wq = mass_weight_rel(q, lm);
            w = __fdividef(wq.num, wq.den);
            w = w > 0.f ? w : 0.f;
        }
        const float d = z - zref, wd_ = w * d;
        m[0] += w; m[1] += wd_; m[2] = fmaf(wd_, d, m[2]); m[3] = fmaf(w, w, m[3]);
        wd[j] = jac(w, z, lz, sv);
    };
    int j = tid;
    // RW_INFLIGHT samples per thread in flight: loads first, then the arithmetic
    for (; j + (RW_INFLIGHT - 1) * RW_THREADS < ns; j += RW_INFLIGHT * RW_THREADS) {
        float4 sv[RW_INFLIGHT], nd[RW_INFLIGHT], nl[RW_INFLIGHT];
        float2 lo2[RW_INFLIGHT];
#pragma unroll
        for (int uu = 0; uu < RW_INFLIGHT; uu++) sv[uu] = __ldg(sp + j + uu * RW_THREADS);
#pragma unroll
        for (int uu = 0; uu < RW_INFLIGHT; uu++) lo2[uu] = __ldg(c.s32lo + s0 + j + uu * RW_THREADS);
#pragma unroll
        for (int uu = 0; uu < RW_INFLIGHT; uu++) nd[uu] = node(sv[uu], nl[uu]);
#pragma unroll
        for (int uu = 0; uu < RW_INFLIGHT; uu++) sample(sv[uu], nd[uu], nl[uu], lo2[uu], j + uu * RW_THREADS);
    }
    for (; j < ns; j += RW_THREADS) {
        const float4 sv = __ldg(sp + j);
        const float2 lo2 = __ldg(c.s32lo + s0 + j);
        float4 nl;
        const float4 nd = node(sv, nl);
        sample(sv, nd, nl, lo2, j);
    }
    __syncthreads();
    // the deferred samples in index order: thread t counts the chunks
    // 3t .. 3t+2, an exclusive scan over the threads gives its offset, and it
    // writes its chunks' samples there; the list is then shared out over the
    // threads, so the same thread adds the same sample's moments on every run
    // (the order of the atomic updates varies from run to run)
    const int lane = tid & 31, wid = tid >> 5;
    constexpr int CPT = RW_CHUNKS / RW_THREADS;
    int cnt = 0;
#pragma unroll
    for (int u = 0; u < CPT; u++) cnt += __popc(s_smask[CPT * tid + u]);
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_wtot[wid] = incl;
    __syncthreads();
    int pos = incl - cnt, nspec = 0;
    for (int w = 0; w < RW_THREADS / 32; w++) {
        if (w < wid) pos += s_wtot[w];
        nspec += s_wtot[w];
    }
    if (nspec <= RW_SPEC_CAP) {
#pragma unroll
        for (int u = 0; u < CPT; u++) {
            const int cc = CPT * tid + u;
            for (unsigned m = s_smask[cc]; m; m &= m - 1) s_spec[pos++] = 32 * cc + __ffs(m) - 1;
        }
        __syncthreads();
        for (int i = tid; i < nspec; i += RW_THREADS) special(s_spec[i]);
    } else {
        // more deferred samples than the list holds: find them all again
        for (int jj = tid; jj < ns; jj += RW_THREADS) {
            const float4 sv = __ldg(sp + jj);
            float4 nl;
            const float4 nd = node(sv, nl);
            const float z = chimd::hermite4(nd, sv.y);
            if (!(z < CUDART_INF_F)) continue;
            const LogMass lm = log_mass(q, sv.z, sv.w, __ldg(c.s32lo + s0 + jj), chimd::hermite4(nl, sv.y));
            if (w_needs64(lm) || (w_in_range(lm) && lm.d1 < W_FP64)) special(jj);
        }
    }
    block_sum<7, RW_THREADS>(m, red);
    if (tid == 0) {
        // Scott's rule from the FP64 block sums: the moments' difference
        // E[d^2] - E[d]^2 in FP64 (no cancellation in FP32), the rest in FP32
        // (errors that differ between events; B300's FP64 pipe would make a
        // double pow this block's longest step): weighted, then unweighted,
        // then the grid spacing
        float bl = c.dz32;
        const double W1 = red[0], n = red[4];
        bool done = false;
        if (W1 > 0.0) {
            const double mw = red[1] / W1, var = red[2] / W1 - mw * mw;
            const double neff = W1 * W1 / red[3];
            if (neff >= 2.0 && var > 0.0) {
                bl = sqrtf((float)var) * exp2f(-0.2f * log2f((float)neff));
                done = true;
            }
        }
        if (!done && n >= 2.0) {
            const double mu = red[5] / n, var = red[6] / n - mu * mu;
            if (var > 0.0) bl = sqrtf((float)var) * exp2f(-0.2f * log2f((float)n));
        }
        p.bw[(size_t)h * c.n_events + ev] = (double)bl;
    }
}

// K4 (mixed): the event integral for hyperpoints h0 .. h0+nh-1 from the
// reweighted samples of the tile buffer, one block per (event, point).
// The block first describes every warp group once, one thread per group
// (valid count, grid range, origin, table length and evaluation path), so
// that the warps of phase B do not each repeat that bookkeeping on all of
// their lanes.
enum : int { GP_NONE = 0, GP_SMALL = 1, GP_UNION = 2, GP_LANE = 3, GP_DIRECT = 4, GP_BIG = 16 };
template <int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) k_event_mixed(DevCatalog c, CallPtrs p, int h0, int nh) {
    constexpr int NT = NW * 32;
    extern __shared__ float4 smem4[];
    const MixLayout L(c.max_ns, c.n_z, c.max_seg, c.max_groups, NW);
    int4 *grp = reinterpret_cast<int4 *>(smem4);  // group metadata, then (lo, cnt, A0, A1)
    int4 *gd1 = grp + L.gmax_pad;                   // (t_o, nq, path | GP_BIG, profile row)
    float *zs = reinterpret_cast<float *>(gd1 + L.gmax_pad);
    float *ws = zs + L.ns_pad;
    float *Fs = ws + L.ns_pad;
    float *Dt = Fs + L.nz_pad;
    float *CT2 = Dt + NW * DCAP;        // C at tau = t - CCAP, t in [0, 2 CCAP)
    float *CT = CT2 + CCAP;             // C at tau, tau in [-CCAP, CCAP)
    float *gres = CT2 + 2 * CCAP;       // per group: its prefactor, then its value
    long long *seg64 = reinterpret_cast<long long *>(gres + L.gmax_pad);  // staged segment offsets
    double *spf64 = reinterpret_cast<double *>(seg64 + L.seg_pad);        // staged prefactors
    double *red = spf64 + L.seg_pad;
    __shared__ int s_gctr;

    const int hl = blockIdx.x % nh, h = h0 + hl;
    const int4 ei = __ldg(c.ev_info + 2 * (blockIdx.x / nh));      // (ev, s0, ns, zoff)
    const int4 ej = __ldg(c.ev_info + 2 * (blockIdx.x / nh) + 1);  // (g0, ngroups, sg0, nseg)
    const int ev = ei.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const size_t out = (size_t)h * c.n_events + ev;
    const HP &hp = p.hp[h];
    const double bd = p.bw[out];  // the reweighting kernel's FP32 bandwidth (in flight with the status)
    if (hp.status & (CHIMERA_PT_OUT_OF_SUPPORT | CHIMERA_PT_NONMONOTONE)) {
        if (tid == 0) { p.lnI[out] = 0.0; p.bw[out] = 0.0; }
        return;
    }
    const int nz = c.n_z;
    const float dz = c.dz32;
    const float inv_dz = 1.f / dz;
    if (tid == 0) s_gctr = 0;
    // ---- prologue: the event's reweighted samples, its group and segment
    // metadata and F, all requested at once with cp.async
    const int64_t s0 = ei.y;
    const int ns = ei.z;
    const int g0 = ej.x, ngroups = ej.y;
    const int sg0 = ej.z, nseg = ej.w;
    {
        const float *zsrc = p.zw + (size_t)hl * 2 * c.n_zpad + ei.w;
        const float *wsrc = zsrc + c.n_zpad;
        for (int i = tid; i < (ns + 3) >> 2; i += NT) {
            cp_async16(zs + 4 * i, zsrc + 4 * i);
            cp_async16(ws + 4 * i, wsrc + 4 * i);
        }
    }
    for (int g = tid; g < ngroups; g += NT) cp_async16(grp + g, c.groups + g0 + g);
    for (int k = tid; k <= nseg; k += NT) {
        cp_async8(seg64 + k, c.seg_soff + sg0 + k);
        if (k < nseg) cp_async8(spf64 + k, c.seg_pf + sg0 + k);
    }
    // F(z_a) (the trapezoid weight of the two end points is applied below)
    for (int a = tid; a < nz; a += NT) cp_async4(Fs + a, p.F32 + (size_t)h * nz + a);
    cp_async_commit();
    // per-point constants while the copies are in flight:
    // 1/(sqrt2 b) and dz/(sqrt2 b) with 1/sqrt2 and dz as float pairs, so
    // that no constant rounded to float scales every Gaussian of the event
    // alike (FP32 only: an FP64 division in every thread would cost B300's
    // FP64 pipe more than the rest of the prologue)
    const float b = (float)bd;
    const float ib = 1.f / b;
    const float inv_s2b = fmaf(0.707106769084930419921875f, ib, 1.2101617042e-8f * ib);
    const float dz_lo = c.dz_lo32;
    const float ds = fmaf(dz, inv_s2b, dz_lo * inv_s2b);
    const float halfk = KW32 * b;
    const int Tw = (int)ceilf(halfk * inv_dz + 0.5f);
    const bool vec4 = (nz & 3) == 0;  // profile rows 16-byte aligned
    cp_async_wait<0>();
    __syncthreads();

    // ---- the Gaussian factor table C_t = exp(-(ds t)^2), the trapezoid
    // end weights and one descriptor per warp group
    for (int t = tid; t < 2 * CCAP; t += NT) {
        float x = ds * (float)(t - CCAP);
        CT2[t] = expc(-x * x);
    }
    if (tid == 0) Fs[0] *= 0.5f;
    if (tid == 1 && nz > 1) Fs[nz - 1] *= 0.5f;
    for (int g = tid; g < ngroups; g += NT) {
        const int4 gi = grp[g];  // (first sample, samples, segment, -)
        const int sk = gi.z;
        const int seg_lo = (int)(seg64[sk] - s0), seg_hi = (int)(seg64[sk + 1] - s0);
        // the segment's valid samples are a prefix (redshifts beyond the
        // table are +inf and sort last)
        int nv = seg_hi - seg_lo;
        if (nv > 0 && !(zs[seg_hi - 1] < CUDART_INF_F)) {
            int l = seg_lo, r = seg_hi;
            while (l < r) {
                const int mm = (l + r) >> 1;
                if (zs[mm] < CUDART_INF_F) l = mm + 1; else r = mm;
            }
            nv = l - seg_lo;
        }
        const int lo = gi.x;
        const int cnt = min(gi.y, nv - (lo - seg_lo));  // valid samples only
        int A0 = 0, A1 = -1, t_o = 0, nq = 0, path = GP_NONE;
        if (cnt > 0) {
            // KDE support of the segment: its samples' range +- KDE_MARGIN b
            const int s_lo = max(0, (int)ceilf((zs[seg_lo] - (float)KDE_MARGIN * b) * inv_dz));
            const int s_hi = min(nz - 1, (int)floorf((zs[seg_lo + nv - 1] + (float)KDE_MARGIN * b) * inv_dz));
            const float zlo = zs[lo], zhi = zs[lo + cnt - 1];
            const float spread = zhi - zlo;
            // grid range the group can touch
            const float fA0 = floorf((zlo - halfk) * inv_dz), fA1 = ceilf((zhi + halfk) * inv_dz);
            A0 = fA0 < (float)s_lo ? s_lo : (int)fA0;
            A1 = fA1 > (float)s_hi ? s_hi : (int)fA1;
            if (A0 <= A1) {
                if (cnt <= SMALL_CNT) {
                    path = GP_SMALL;
                } else {
                    // group origin; a multiple of 4 when the profile rows are
                    // 16-byte aligned, so that the table is staged as float4
                    const float tof = vec4 ? 4.f * rintf(0.125f * (zlo + zhi) * inv_dz)
                                           : rintf(0.5f * (zlo + zhi) * inv_dz);
                    t_o = tof > 1e8f ? 100000000 : (int)tof;
                    const int thi = A1 - t_o, tlo = t_o - A0;  // tau in [-tlo, thi]
                    const int nqf = thi >= 0 ? (thi + 4) >> 2 : 0;
                    const int nqb = tlo >= 1 ? (tlo + 3) >> 2 : 0;
                    nq = max(nqf, nqb);  // symmetric table, zero-padded
                    // shared origin for spreads up to 16 b; beyond 8 b the table is
                    // scaled by 2^29 (undone in A, exactly) to keep every relevant
                    // coefficient and Horner intermediate in the normal float range
                    if (ds <= 0.5f && spread <= 16.f * b && thi >= -1 && tlo >= 0 && 8 * nq <= DCAP &&
                        4 * nq < CCAP)
                        path = GP_UNION | (spread > 8.f * b ? GP_BIG : 0);
                    else if (ds <= 2.f && Tw + 2 < CCAP && (A1 - A0 + 1) + 2 * Tw + 4 <= DCAP)
                        path = GP_LANE;
                    else
                        path = GP_DIRECT;
                }
            }
        }
        const int row = c.kde_mode == CHIMERA_KDE_MANY_1D ? sg0 + sk : ev;
        grp[g] = make_int4(lo, cnt, A0, A1);
        gd1[g] = make_int4(t_o, nq, path, row);
        gres[g] = (float)spf64[sk];
    }
    __syncthreads();

    // ---- phase B: groups taken dynamically by warps; each group's value is
    // computed by a fixed lane assignment and stored in its own slot, and the
    // slots are added in group order, so the result does not depend on timing.
    float *D = Dt + wid * DCAP;
    const float *prof = reinterpret_cast<const float *>(p.prof[h]);
    unsigned long long npairs = 0;  // algorithmic pair count (roofline only)
    // a warp claims its next group as it starts the current one, so that the
    // shared-memory atomic's round trip is hidden behind the group's work
    int gnext = 0;
    if (lane == 0) gnext = atomicAdd(&s_gctr, 1);
    gnext = __shfl_sync(0xffffffffu, gnext, 0);
    while (true) {
        const int g = gnext;
        if (g >= ngroups) break;
        int gclaim = 0;
        if (lane == 0) gclaim = atomicAdd(&s_gctr, 1);
        const int4 d0 = grp[g], d1 = gd1[g];
        const int lo = d0.x, cnt = d0.y, A0 = d0.z, A1 = d0.w;
        const int path = d1.z & 15;
        float v = 0.f;
        if (path != GP_NONE) {
            const float pf = gres[g];
            const float *G = prof + (int64_t)d1.w * nz;
            if (p.pairs) {
                for (int j = lane; j < cnt; j += 32) {
                    float z = zs[lo + j];
                    if (ws[lo + j] == 0.f) continue;
                    int a0 = max(A0, (int)ceilf((z - halfk) * inv_dz));
                    int a1 = min(A1, (int)floorf((z + halfk) * inv_dz));
                    if (a1 >= a0) npairs += (unsigned long long)(a1 - a0 + 1);
                }
            }
            if (path == GP_SMALL) {
                // a few samples: lanes over the grid points, direct exponentials
                v = small_group(zs + lo, ws + lo, cnt, A0, A1, G, Fs, dz, dz_lo, inv_s2b, halfk, lane);
            } else if (path == GP_UNION) {
                const int t_o = d1.x, nq = d1.y;
                const bool big = (d1.z & GP_BIG) != 0;
                const float iscale = big ? 1.862645149230957e-9f : 1.f;  // 2^-29
                const float scale = big ? 536870912.f : 1.f;             // 2^29
                __syncwarp();
                if (vec4) stage_table4(D, nq, t_o, A0, A1, G, Fs, CT, scale, lane);
                else stage_table_p(D, nq, t_o, A0, A1, G, Fs, CT, scale, lane);
                __syncwarp();
                const float zo = fmaf((float)t_o, dz, (float)t_o * dz_lo);  // t_o dz without dz's rounding
#define CHIM_UNION(R) v = union_samples<R>(D, nq, zs + lo, ws + lo, cnt, lane, zo, inv_s2b, ds, iscale)
                switch ((cnt + 31) >> 5) {
                    case 1: CHIM_UNION(1); break;
                    case 2: CHIM_UNION(2); break;
                    case 3: CHIM_UNION(3); break;
                    default: CHIM_UNION(4); break;
                }
#undef CHIM_UNION
            } else if (path == GP_LANE) {
                // stage H' on [base, base + span) with zeros outside [A0, A1]
                const int base = A0 - Tw - 2, span = (A1 - A0 + 1) + 2 * Tw + 4;
                __syncwarp();
                stage_table(D, span, base, A0, A1, G, Fs, lane);
                __syncwarp();
                for (int j = lane; j < cnt; j += 32) {
                    float w = ws[lo + j];
                    if (w == 0.f) continue;
                    float z = zs[lo + j];
                    int ts = (int)rintf(fminf(z * inv_dz, 1e8f));
                    ts = min(max(ts, A0 - 1), A1 + 1);
                    // a sample further than its window from [A0, A1] adds nothing
                    // (and would push exp(2 u ds) out of range)
                    if (fabsf(z - ts * dz) > halfk + dz) continue;
                    v += w * lane_chain(D + (ts - base), CT, Tw, z, ts, dz, dz_lo, inv_s2b, ds);
                }
            } else {
                for (int j = lane; j < cnt; j += 32) {
                    float z = zs[lo + j], w = ws[lo + j];
                    if (w == 0.f) continue;
                    int a0 = max(A0, (int)ceilf((z - halfk) * inv_dz));
                    int a1 = min(A1, (int)floorf((z + halfk) * inv_dz));
                    float sacc = 0.f;
                    for (int a = a0; a <= a1; a++) {
                        float x = (fmaf((float)a, dz, (float)a * dz_lo) - z) * inv_s2b;
                        sacc += expf(-x * x) * Fs[a] * G[a];
                    }
                    v += w * sacc;
                }
            }
            // within a group a plain tree (32 lanes; compensating it too was
            // measured at +2.3 % of this kernel for at most 2.4e-7 in ln I)
            v = warp_sum(v) * pf;
        }
        if (lane == 0) gres[g] = v;
        gnext = __shfl_sync(0xffffffffu, gclaim, 0);
    }
    __syncthreads();
    // the event's sum of the group values in a fixed order, compensated at
    // every step (FP32 with the rounding errors carried: a double reduction
    // would be the block's longest step at B300's FP64 rate), then ln I
    // (ln_mixed); the first EV_RED threads take the groups, whatever the
    // block size, so both geometries add them in the same order
    {
        float sacc = 0.f, cacc = 0.f;
        for (int g = tid; tid < EV_RED && g < ngroups; g += EV_RED) {
            float sm, e;
            two_sum(sacc, gres[g], sm, e);
            sacc = sm;
            cacc = __fadd_rn(cacc, e);
        }
        sacc = warp_sum_c(__fadd_rn(sacc, cacc));
        float *redf = reinterpret_cast<float *>(red);
        if (lane == 0) redf[wid] = sacc;
        __syncthreads();
        if (tid == 0) {
            float I = 0.f, cI = 0.f;
            for (int w = 0; w < EV_RED / 32; w++) {
                float sm, e;
                two_sum(I, redf[w], sm, e);
                I = sm;
                cI = __fadd_rn(cI, e);
            }
            I = __fadd_rn(I, cI);
            p.lnI[out] = ln_mixed(I, (float)bd, p.hp[h].ln_k0);
            p.bw[out] = bd;
        }
    }
    if (p.pairs) {
        for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
        if (lane == 0 && npairs) atomicAdd(p.pairs + h, npairs);
    }
}

// ------------------------------------------------------------ binned ---
// K4 (mixed, binned-KDE option; Sec. 2.3: the weighted samples of each
// pixel, or of the whole event in single-1D, are binned).  Reading: linear
// binning onto the grid lattice z_n = n dz, then the Gaussian KDE of the
// nodes with the samples' bandwidth, windows (+-KW32 b) and support:
//   I = sum_k pf_k sum_n c_kn sum_a C_{|a-n|} F'(z_a) G_k(z_a),
//   c_kn = sum_{j in k} w_j max(0, 1 - |z_j / dz - n|),  C_m = exp(-(m dz)^2 / 2b^2),
// in the mixed kernel's units (ln_mixed gives ln I).  The work per segment is
// (nodes) x (window) instead of (samples) x (window), which pays where a
// segment holds many more samples than grid points under its samples
// (single-1D).  One thread per node gathers the node's weight from the
// segment's samples in sample order (sorted by z), so the sums are
// deterministic, then runs the node's window over the segment's staged
// H = F' G (consecutive nodes across a warp read consecutive H entries;
// the C entry is a broadcast).
constexpr int BN_THREADS = 256;
constexpr int BN_HPAD = 4;  // zero entries staged on each side of a segment's support

struct BinLayout {
    int ns_pad, nz_pad, seg_pad;
    __host__ __device__ BinLayout(int max_ns, int nz, int max_seg)
        : ns_pad((max_ns + 3) & ~3), nz_pad((nz + 2 * BN_HPAD + 3) & ~3), seg_pad((max_seg + 4) & ~3) {}
    // floats: zs, ws, F', H (padded), C table (2 n_z entries), segment
    // prefactors, block sums; ints: segment starts, valid counts
    __host__ __device__ size_t bytes() const {
        return sizeof(float) * (2 * (size_t)ns_pad + 4 * (size_t)nz_pad + seg_pad + BN_THREADS / 32) +
               sizeof(int) * 2 * (size_t)seg_pad;
    }
};

// BINNED = false: the same block structure with one thread per sample and a
// direct evaluation of the kernel per (sample, grid point); the mixed path's
// Epanechnikov form (the Horner factorisation of the main kernel is specific
// to the Gaussian).  The kernel shape (p.kshape) sets the weight table and
// window: exp(-x^2/2), |x| <= KW32, or 1 - x^2/5, |x| <= sqrt5, x = dz m / b.
template <bool BINNED>
__global__ void __launch_bounds__(BN_THREADS) k_event_binned(DevCatalog c, CallPtrs p, int h0, int nh) {
    extern __shared__ float4 bsm4[];
    const BinLayout L(c.max_ns, c.n_z, c.max_seg);
    float *zs = reinterpret_cast<float *>(bsm4);
    float *ws = zs + L.ns_pad;
    float *Fs = ws + L.ns_pad;
    float *Hs = Fs + L.nz_pad;      // H[a] at Hs[a + BN_HPAD]
    float *Ct = Hs + L.nz_pad;      // C_m, m < 2 nz_pad
    float *segpf = Ct + 2 * L.nz_pad;
    float *redf = segpf + L.seg_pad;
    int *seglo = reinterpret_cast<int *>(redf + BN_THREADS / 32);
    int *segv = seglo + L.seg_pad;

    const int hl = blockIdx.x % nh, h = h0 + hl;
    const int4 ei = __ldg(c.ev_info + 2 * (blockIdx.x / nh));      // (ev, s0, ns, zoff)
    const int4 ej = __ldg(c.ev_info + 2 * (blockIdx.x / nh) + 1);  // (g0, ngroups, sg0, nseg)
    const int ev = ei.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const size_t out = (size_t)h * c.n_events + ev;
    const HP &hp = p.hp[h];
    if (hp.status & (CHIMERA_PT_OUT_OF_SUPPORT | CHIMERA_PT_NONMONOTONE)) {
        if (tid == 0) { p.lnI[out] = 0.0; p.bw[out] = 0.0; }
        return;
    }
    const int nz = c.n_z;
    const float dz = c.dz32, inv_dz = 1.f / dz;
    const int ns = ei.z, sg0 = ej.z, nseg = ej.w;
    const int64_t s0 = ei.y;
    {
        const float *zsrc = p.zw + (size_t)hl * 2 * c.n_zpad + ei.w;
        const float *wsrc = zsrc + c.n_zpad;
        for (int i = tid; i < ns; i += BN_THREADS) {
            zs[i] = __ldg(zsrc + i);
            ws[i] = __ldg(wsrc + i);
        }
    }
    for (int a = tid; a < nz; a += BN_THREADS)
        Fs[a] = ((a == 0 || a == nz - 1) ? 0.5f : 1.f) * p.F32[(size_t)h * nz + a];
    for (int k = tid; k <= nseg; k += BN_THREADS) {
        seglo[k] = (int)(c.seg_soff[sg0 + k] - s0);
        if (k < nseg) segpf[k] = (float)c.seg_pf[sg0 + k];
    }
    const double bd = p.bw[out];  // the reweighting kernel's FP32 bandwidth
    const float b = (float)bd;
    const bool epan = p.kshape == 1;
    const float ib = 1.f / b;
    const float half = epan ? 2.23606798f * b : KW32 * b;  // the kernel's window
    auto kern = [&](float x) {  // x = (z_a - z) / b
        return epan ? fmaxf(0.f, fmaf(-0.2f * x, x, 1.f)) : __expf(-0.5f * x * x);
    };
    const int W = (int)fminf(half * inv_dz, 1e8f);  // window half-width in nodes
    const int nct = min(W + 1, 2 * L.nz_pad);
    if (BINNED)
        for (int m = tid; m < nct; m += BN_THREADS) Ct[m] = kern(m * dz * ib);
    __syncthreads();
    for (int k = tid; k < nseg; k += BN_THREADS) {
        int l = seglo[k], r = seglo[k + 1];
        const int lo = l;
        while (l < r) {
            const int m = (l + r) >> 1;
            if (zs[m] < CUDART_INF_F) l = m + 1; else r = m;
        }
        segv[k] = l - lo;
    }
    __syncthreads();
    const float *prof = reinterpret_cast<const float *>(p.prof[h]);
    float acc = 0.f;
    for (int k = 0; k < nseg; k++) {
        const int lo = seglo[k], cnt = segv[k];
        if (cnt == 0) continue;
        // the segment's KDE support (as the unbinned kernel) and its nodes
        const int A0 = max(0, (int)ceilf((zs[lo] - (float)KDE_MARGIN * b) * inv_dz));
        const int A1 = min(nz - 1, (int)floorf((zs[lo + cnt - 1] + (float)KDE_MARGIN * b) * inv_dz));
        if (A0 > A1) continue;
        const int N0 = (int)floorf(zs[lo] * inv_dz);
        const int N1 = (int)fminf(floorf(zs[lo + cnt - 1] * inv_dz) + 1.f, (float)A1 + (float)W);
        const int64_t row = c.kde_mode == CHIMERA_KDE_MANY_1D ? (int64_t)(sg0 + k) : (int64_t)ev;
        const float *G = prof + row * nz;
        for (int a = A0 - BN_HPAD + tid; a <= A1 + BN_HPAD; a += BN_THREADS)
            Hs[a + BN_HPAD] = (a >= A0 && a <= A1) ? Fs[a] * __ldg(G + a) : 0.f;
        __syncthreads();
        const float pf = segpf[k];
        if (BINNED) {
            for (int n = N0 + tid; n <= N1; n += BN_THREADS) {
                // the node's weight: samples with floor(z / dz) in {n - 1, n}
                int l = lo, r = lo + cnt;
                while (l < r) {
                    const int m = (l + r) >> 1;
                    if (floorf(zs[m] * inv_dz) < (float)(n - 1)) l = m + 1; else r = m;
                }
                float cw = 0.f;
                for (int j = l; j < lo + cnt; j++) {
                    const float t = zs[j] * inv_dz, fb = floorf(t);
                    if (fb > (float)n) break;
                    const float f = t - fb;
                    cw += fb == (float)n ? ws[j] * (1.f - f) : ws[j] * f;
                }
                if (cw == 0.f) continue;
                const int a0 = max(A0, n - W), a1 = min(A1, n + W);
                float sacc = 0.f;
                for (int a = a0; a <= a1; a++) {
                    const int m = abs(a - n);
                    const float cm = m < nct ? Ct[m] : kern(m * dz * ib);
                    sacc = fmaf(cm, Hs[a + BN_HPAD], sacc);
                }
                acc = fmaf(pf * cw, sacc, acc);
            }
        } else {
            for (int j = lo + tid; j < lo + cnt; j += BN_THREADS) {
                const float z = zs[j], w = ws[j];
                if (w == 0.f) continue;
                const int a0 = max(A0, (int)ceilf((z - half) * inv_dz));
                const int a1 = min(A1, (int)floorf((z + half) * inv_dz));
                float sacc = 0.f;
                for (int a = a0; a <= a1; a++) sacc = fmaf(kern((a * dz - z) * ib), Hs[a + BN_HPAD], sacc);
                acc = fmaf(pf * w, sacc, acc);
            }
        }
        __syncthreads();  // Hs is restaged for the next segment
    }
    // fixed-order FP32 tree sum, then ln I (ln_mixed)
    acc = warp_sum(acc);
    if (lane == 0) redf[wid] = acc;
    __syncthreads();
    if (tid == 0) {
        float I = 0.f;
        for (int w = 0; w < BN_THREADS / 32; w++) I += redf[w];
        p.lnI[out] = ln_mixed(I, b, hp.ln_k0, epan);
        p.bw[out] = bd;
    }
}

// ---------------------------------------------------------------- FP64 ---
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
    const bool epan = p.kshape == 1;
    const double *F = p.F64 + (size_t)h * nz;
    const double *prof = reinterpret_cast<const double *>(p.prof[h]);
    const double dlt = dz / b, qq = exp(-dlt * dlt);
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
        if (p.jac_ps) {  // the Jacobian on the sample, after the bandwidth (Eq. jacobian)
            double dd, J;
            chimd::dgw_J(z, hp.cH * chimd::dc_hermite(p.fwd[h], z, hp.th[1]), hp.th, hp.cH, &dd, &J);
            const double ap = 1.0 + z;
            w /= ap * ap * ap * fabs(J);
        }
        const int64_t row = c.kde_mode == CHIMERA_KDE_MANY_1D ? (int64_t)(sg0 + l) : (int64_t)ev;
        const double *G = prof + row * nz;
        // window +-KW64 b (Gaussian) or +-h = sqrt(5) b (Epanechnikov),
        // clipped to the segment's KDE support
        const double smin = zs[lo] - KDE_MARGIN * b, smax = zs[lo + segv[l] - 1] + KDE_MARGIN * b;
        const double half = epan ? 2.23606797749978969641 * b : KW64 * b;
        double a0 = fmax(ceil((z - half) / dz), ceil(smin / dz));
        double a1 = fmin(floor((z + half) / dz), floor(smax / dz));
        int ia0 = a0 < 0.0 ? 0 : (a0 > nz ? nz : (int)a0);
        int ia1 = a1 > nz - 1 ? nz - 1 : (a1 < -1.0 ? -1 : (int)a1);
        double s = 0.0;
        if (epan) {
            for (int a = ia0; a <= ia1; a++) {
                const double x = (a * dz - z) / b;
                const double wa = (a == 0 || a == nz - 1) ? 0.5 : 1.0;
                s += fmax(0.0, 1.0 - 0.2 * x * x) * wa * F[a] * G[a];
            }
        } else if (ia0 <= ia1) {
            // exp(-x^2/2) along the window by the Gaussian recurrence
            // g_{a+1} = g_a r_a, r_{a+1} = r_a e^{-delta^2}, delta = dz / b
            // (two exponentials per sample; relative drift ~1e-14)
            const double x0 = (ia0 * dz - z) / b;
            double g = exp(-0.5 * x0 * x0), r = exp(-x0 * dlt - 0.5 * dlt * dlt);
            for (int a = ia0; a <= ia1; a++) {
                const double wa = (a == 0 || a == nz - 1) ? 0.5 : 1.0;
                s += g * wa * F[a] * G[a];
                g *= r;
                r *= qq;
            }
        }
        tsum += c.seg_pf[sg0 + l] * w * s;
    }
    {
        double v[1] = {tsum};
        __syncthreads();
        block_sumd<1, EV64_THREADS>(v, red);
    }
    if (tid == 0) {
        // kernel normalisation: 1/(sqrt(2 pi) b), or 3/(4 h) = 3/(4 sqrt5 b)
        const double kn = epan ? 0.33541019662496845446 : 0.39894228040143267794;
        double I = red[0] * dz * kn / (c.n_gal_total * b);
        p.lnI[out] = I > 0.0 ? log(I) : -CUDART_INF;
        p.bw[out] = b;
    }
}


}  // namespace

size_t event_mixed_smem(const DevCatalog &c, int geom) {
    return MixLayout(c.max_ns, c.n_z, c.max_seg, c.max_groups, geom == 1 ? EV_WARPS_3 : EV_WARPS_2).bytes();
}

// Three resident blocks of 10 warps when they fit the SM's shared memory and
// registers, else two of 16 (10 again if a 16-warp block would not fit the
// device's shared memory per block at all).
int event_mixed_pick(const DevCatalog &c) {
    int dev = 0, maxsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
        event_mixed_smem(c, 0) > (size_t)maxsm)
        return 1;
    cudaGetLastError();
    const size_t smem = event_mixed_smem(c, 1);
    if (cudaFuncSetAttribute(k_event_mixed<EV_WARPS_3, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_event_mixed<EV_WARPS_3, 3>, EV_WARPS_3 * 32, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb >= 3 ? 1 : 0;
}

size_t event_fp64_smem(const DevCatalog &c) {
    return sizeof(double) * 2 * (size_t)c.max_ns + sizeof(int) * (size_t)((c.max_seg + 2) & ~1) +
           sizeof(double) * (8 + (EV64_THREADS / 32) * 8);
}

void launch_reweight(const DevCatalog &c, const CallPtrs &p, int h0, int nh, cudaStream_t st) {
    const unsigned nb = (unsigned)((int64_t)c.n_events * nh);
    const bool stage = c.max_krange <= RW_STAGE_MAX;
    const size_t smem = stage ? 2 * sizeof(float4) * (size_t)c.max_krange : 0;
    if (!nb) return;
    if (p.jac_ps) {
        if (stage) k_reweight<true, true><<<nb, RW_THREADS, smem, st>>>(c, p, h0, nh);
        else k_reweight<true, false><<<nb, RW_THREADS, 0, st>>>(c, p, h0, nh);
    } else {
        if (stage) k_reweight<false, true><<<nb, RW_THREADS, smem, st>>>(c, p, h0, nh);
        else k_reweight<false, false><<<nb, RW_THREADS, 0, st>>>(c, p, h0, nh);
    }
}

void launch_event_mixed(const DevCatalog &c, const CallPtrs &p, int h0, int nh, cudaStream_t st) {
    const size_t smem = event_mixed_smem(c, c.ev_geom);
    const unsigned nb = (unsigned)((int64_t)c.n_events * nh);
    if (c.ev_geom == 1) {
        cudaFuncSetAttribute(k_event_mixed<EV_WARPS_3, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (nb) k_event_mixed<EV_WARPS_3, 3><<<nb, EV_WARPS_3 * 32, smem, st>>>(c, p, h0, nh);
    } else {
        cudaFuncSetAttribute(k_event_mixed<EV_WARPS_2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (nb) k_event_mixed<EV_WARPS_2, 2><<<nb, EV_WARPS_2 * 32, smem, st>>>(c, p, h0, nh);
    }
}

size_t event_binned_smem(const DevCatalog &c) { return BinLayout(c.max_ns, c.n_z, c.max_seg).bytes(); }

void launch_event_binned(const DevCatalog &c, const CallPtrs &p, int h0, int nh, bool binned,
                         cudaStream_t st) {
    size_t smem = event_binned_smem(c);
    const unsigned nb = (unsigned)((int64_t)c.n_events * nh);
    if (binned) {
        cudaFuncSetAttribute(k_event_binned<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (nb) k_event_binned<true><<<nb, BN_THREADS, smem, st>>>(c, p, h0, nh);
    } else {
        cudaFuncSetAttribute(k_event_binned<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (nb) k_event_binned<false><<<nb, BN_THREADS, smem, st>>>(c, p, h0, nh);
    }
}

void launch_event_fp64(const DevCatalog &c, const CallPtrs &p, int H, cudaStream_t st) {
    size_t smem = event_fp64_smem(c);
    cudaFuncSetAttribute(k_event_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_event_fp64<<<(unsigned)(c.n_events * H), EV64_THREADS, smem, st>>>(c, p, H);
}

}  // namespace chim
