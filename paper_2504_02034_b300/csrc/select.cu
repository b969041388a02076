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
#include "mass.cuh"

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

// mixed: each term in FP32 with the injection's own rounding errors only
// (they differ between injections and average out in the sum): the
// hyperpoint's constants enter as float pairs or through the FP64 factor
// hp.ln_sel, 1/pi_inj comes rounded from FP64, logs are the accurate log2f,
// exponentials split off their integer part before the SFU (mass.cuh), and
// the test whether an injection lies inside the mass range and below z_max is
// taken again in FP64 where the FP32 one could differ (as the FP64 path and
// the oracle take it).  Partial sums in FP64 across warps.  A block takes one
// chunk of injections for SEL_HB hyperpoints: every injection is read once
// and evaluated for all of them.
constexpr int SEL_HB = 2;

struct SelConst {
    WParams q;
    const float4 *inv, *linv;
    F2 kH, xi0, omx, nn, nomx, om, omc, gam, gkp, l2zp;
    double cfac;  // exp(hp.ln_sel + K ln 2): the shared factor of every term
};

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
    // one Newton step from the Hermite seed (see invert64)
    const double *fwd = p.fwd[h];
    double dd, J;
    chimd::dgw_J(z, hp.cH * chimd::dc_hermite(fwd, z, hp.th[1]), hp.th, hp.cH, &dd, &J);
    const double step = (dd - d) / J;
    if (isfinite(step)) z -= step;
    *zout = z;
    return true;
}

// Injections are stored sorted by d_L, so a chunk spans a narrow slice of
// the inverse tables: up to SEL_STAGE intervals of it (z and log2(1+z) node
// pairs of each hyperpoint) are staged in shared memory.
constexpr int SEL_STAGE = 128;
constexpr int SEL_DEF_CAP = 512;  // deferred FP64 pairs listed per block (more: taken by their words' threads)

__global__ void __launch_bounds__(SEL_THREADS) k_select_mixed(DevCatalog c, CallPtrs p, int H) {
    __shared__ double red[2 * SEL_HB * (SEL_THREADS / 32)];
    __shared__ SelConst scs[SEL_HB];
    __shared__ float4 snode[SEL_HB][2][SEL_STAGE];
    __shared__ unsigned s_dm[SEL_HB][SEL_CHUNK / 32];  // deferred (point, injection) pairs of the chunk
    __shared__ int s_dl[SEL_DEF_CAP];                  // their list, in (point, injection) order
    __shared__ int s_dwt[SEL_THREADS / 32];
    const int chunk = blockIdx.x, h0 = blockIdx.y * SEL_HB;
    const int nh = min(SEL_HB, H - h0);
    const int64_t base = (int64_t)chunk * SEL_CHUNK;
    const int64_t last = min(base + SEL_CHUNK, c.n_det) - 1;
    if (threadIdx.x < nh) {
        const HP &hp = p.hp[h0 + threadIdx.x];
        SelConst k;
        k.q = w_params(hp);
        k.inv = p.inv32 + (size_t)(h0 + threadIdx.x) * NU;
        k.linv = p.linv32 + (size_t)(h0 + threadIdx.x) * NU;
        k.kH = hp.kH2; k.xi0 = hp.xi0_2; k.omx = hp.omx2; k.nn = hp.nn2; k.nomx = hp.nomx2;
        k.om = hp.om2; k.omc = hp.omc2; k.gam = hp.gam2; k.gkp = hp.gk_psi2; k.l2zp = hp.l2zp2;
        k.cfac = hp.sel_cfac;
        scs[threadIdx.x] = k;
    }
    // the chunk's interval range (sorted by d_L; the last valid interval is NU - 1)
    int klo = 0, nk = 0;
    if (base <= last) {
        int k0, k1;
        const float a0 = __ldg(&c.i32a[base].x), a1 = __ldg(&c.i32a[last].x);
        k0 = __float_as_int(a0);
        k1 = __float_as_int(a1);
        if (k1 - k0 + 1 <= SEL_STAGE) {
            klo = k0;
            nk = k1 - k0 + 1;
        }
    }
    for (int i = threadIdx.x; i < SEL_HB * (SEL_CHUNK / 32); i += SEL_THREADS) (&s_dm[0][0])[i] = 0u;
    for (int i = threadIdx.x; i < nh * nk; i += SEL_THREADS) {
        const int hb = i / nk, r = i - hb * nk;
        snode[hb][0][r] = __ldg(p.inv32 + (size_t)(h0 + hb) * NU + klo + r);
        snode[hb][1][r] = __ldg(p.linv32 + (size_t)(h0 + hb) * NU + klo + r);
    }
    __syncthreads();
    if (nk > 0 && threadIdx.x < nh) {  // the kernel reads the staged pairs at k - klo
        scs[threadIdx.x].inv = snode[threadIdx.x][0] - klo;
        scs[threadIdx.x].linv = snode[threadIdx.x][1] - klo;
    }
    __syncthreads();
    const float zmax = c.z_max32;
    float s1[SEL_HB], s2[SEL_HB];
#pragma unroll
    for (int hb = 0; hb < SEL_HB; hb++) s1[hb] = s2[hb] = 0.f;
    // The few (injection, point) pairs that need FP64 (guard bands at the
    // mass edges and z_max, the corner band above m_min) are deferred: a bit
    // per pair in the chunk's masks (atomic OR, order-free), then after the
    // loop the list in (point, injection) order shared out over the threads,
    // so that their FP64 chains, long on B300's narrow FP64 pipe, run side by
    // side instead of stalling a warp each inside the loop, and every pair
    // goes to the same thread on every run.
    auto sel_term = [&](int hb, int64_t j, bool deferred) -> float {
        const float4 a = __ldg(c.i32a + j);
        const float dL = __ldg(&c.i32b[j].x);
        const float ipi = __ldg(c.iipi32 + j);
        const float2 lo = __ldg(c.i32lo + j);
        const int k = __float_as_int(a.x);
        const SelConst &K = scs[hb];
        if (!((k < K.q.kv) || (k == K.q.kv && a.y <= K.q.fv))) return 0.f;
        const float z = chimd::hermite4(K.inv[k], a.y);
        if (!(z < CUDART_INF_F)) return 0.f;
        const float ap = 1.f + z, lz = chimd::hermite4(K.linv[k], a.y);  // log2(1+z)
        LogMass lm = log_mass(K.q, a.z, a.w, lo, lz);
        float wn, wd;  // the weight as a quotient
        const bool f64 = w_needs64(lm) || fabsf(z - zmax) < ZMAX_GUARD;
        if (!f64 && !(w_in_range(lm) && z <= zmax)) return 0.f;
        if (!deferred && (f64 || lm.d1 < W_FP64)) {
            const int li = (int)(j - base);
            atomicOr(&s_dm[hb][li >> 5], 1u << (li & 31));
            return 0.f;
        }
        if (f64) {
            // FP64: range and z_max tests as the oracle takes them, and
            // the weight itself
            const int h = h0 + hb;
            const HP &hp = p.hp[h];
            double z64;
            if (!refine64(p, h, hp, c.inv_d_top, z, c.id64[j], &z64) || !(z64 <= c.z_max)) return 0.f;
            const double a64 = 1.0 + z64;
            wn = (float)(mass_weight64(hp, c.beta, c.im1_64[j] / a64, c.im2_64[j] / a64) * hp.inv_wscale);
            wd = 1.f;
        } else {
            if (lm.d1 < W_FP64) lm.d1 = corner_d1(p, h0 + hb, p.hp[h0 + hb], c.inv_d_top, z, c.id64[j], c.im1_64[j], lm.d1);
            const WQuot wq = mass_weight_rel(K.q, lm);
            wn = wq.num;
            wd = wq.den;
        }
        const float pw = ex2_mul_n(K.nn, lz);  // (1+z)^-n
        const float xi = fmaf(K.omx.hi, pw, K.xi0.hi) + fmaf(K.omx.lo, pw, K.xi0.lo);
        const float N = mul_f2(K.kH, dL);  // d_L H0 / c
        const float axi = ap * xi;       // Dhat = D_c H0 / c = N / ((1+z) Xi)
        const float a3 = ap * ap * ap;
        const float E = sqrtf(fmaf(K.om.hi, a3, K.omc.hi) + fmaf(K.om.lo, a3, K.omc.lo));
        // J H0 / c = (Dhat + (1+z)/E) Xi - n (1 - Xi0) (1+z)^-n Dhat; times E (1+z) Xi:
        const float JE = fmaf(N, E, ap * axi) * xi - mul_f2(K.nomx, pw) * N * E;
        const float r = ex2_mul_n(K.gkp, (lz - K.l2zp.hi) - K.l2zp.lo);  // ((1+z)/(1+z_p))^(gamma+kappa)
        // s / cfac = w' psi Dhat^2 / (E (1+z)^3 |J H0/c|) 2^-K / pi_inj
        //          = w' (1+z)^gamma N^2 2^-K / pi_inj / ((1+z) Xi (1 + r) (1+z)^3 |JE|)
        const float sv = __fdividef(wn * ex2_mul_n(K.gam, lz) * N * N * ipi, wd * axi * (1.f + r) * a3 * fabsf(JE));
        return sv > 0.f ? sv : 0.f;
    };
    for (int qq = 0; qq < SEL_PER_THREAD; qq++) {
        const int64_t j = base + qq * SEL_THREADS + threadIdx.x;
        if (j >= c.n_det) break;
#pragma unroll
        for (int hb = 0; hb < SEL_HB; hb++) {
            if (hb >= nh) break;
            const float sv = sel_term(hb, j, false);
            s1[hb] += sv;
            s2[hb] = fmaf(sv, sv, s2[hb]);
        }
    }
    __syncthreads();
    {
        // the deferred pairs: word w of the masks (point w / (SEL_CHUNK/32))
        // counted by thread w, an exclusive scan, the list written in order
        constexpr int NWD = SEL_HB * (SEL_CHUNK / 32);
        static_assert(NWD <= SEL_THREADS, "one mask word per thread");
        const unsigned *dmf = &s_dm[0][0];
        const int ln = threadIdx.x & 31, wi = threadIdx.x >> 5;
        const unsigned mw = threadIdx.x < NWD ? dmf[threadIdx.x] : 0u;
        const int cnt = __popc(mw);
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (ln >= o) incl += v;
        }
        if (ln == 31) s_dwt[wi] = incl;
        __syncthreads();
        int pos = incl - cnt, nd = 0;
        for (int w = 0; w < SEL_THREADS / 32; w++) {
            if (w < wi) pos += s_dwt[w];
            nd += s_dwt[w];
        }
        auto take = [&](int e) {  // e = word * 32 + bit
            const int hb = e / SEL_CHUNK, li = e - hb * SEL_CHUNK;
            const float sv = sel_term(hb, base + li, true);
#pragma unroll
            for (int q = 0; q < SEL_HB; q++)
                if (q == hb) {
                    s1[q] += sv;
                    s2[q] = fmaf(sv, sv, s2[q]);
                }
        };
        if (nd <= SEL_DEF_CAP) {
            for (unsigned m = mw; m; m &= m - 1) s_dl[pos++] = 32 * threadIdx.x + __ffs(m) - 1;
            __syncthreads();
            for (int i = threadIdx.x; i < nd; i += SEL_THREADS) take(s_dl[i]);
        } else {
            // more than the list holds: each thread takes the pairs of its own word
            for (unsigned m = mw; m; m &= m - 1) take(32 * threadIdx.x + __ffs(m) - 1);
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int hb = 0; hb < SEL_HB; hb++) {
        const float a1 = warp_sumf(s1[hb]), a2 = warp_sumf(s2[hb]);
        if (lane == 0) {
            red[(2 * hb) * (SEL_THREADS / 32) + wid] = a1;
            red[(2 * hb + 1) * (SEL_THREADS / 32) + wid] = a2;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * nh) {
        double acc = 0.0;
        for (int w = 0; w < SEL_THREADS / 32; w++) acc += red[threadIdx.x * (SEL_THREADS / 32) + w];
        const int hb = threadIdx.x >> 1;
        const double cf = scs[hb].cfac;
        acc *= (threadIdx.x & 1) ? cf * cf : cf;
        p.selp[((size_t)(h0 + hb) * p.n_chunk + chunk) * 2 + (threadIdx.x & 1)] = acc;
    }
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

// K6, one block per hyperpoint: the three sums (ln I over the events, and
// the selection partials sum s and sum s^2 over the chunks) in one pass and
// a fixed order - thread t adds elements t, t+256, ... in sequence, a warp
// butterfly adds its 32 lanes, then the 8 warp values are added in warp
// order - so the result does not depend on timing.  The last steps (xi,
// N_eff, ln xi) run on two warps side by side: every FP64 operation waits on
// B300's narrow FP64 pipe, so the block's time is its longest FP64 chain.
__global__ void __launch_bounds__(CMB_THREADS) k_combine(DevCatalog c, CallPtrs p, int H) {
    __shared__ double sh[3][CMB_THREADS / 32];
    __shared__ double s_lnxi, s_xi, s_neff;
    __shared__ int s_bad;
    const int h = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0) s_bad = 0;
    __syncthreads();
    const double *lnI = p.lnI + (size_t)h * c.n_events;
    const double *sp = p.selp + (size_t)h * p.n_chunk * 2;
    double a = 0.0, b1 = 0.0, b2 = 0.0;
    bool bad = false;
    for (int i = t; i < c.n_events; i += CMB_THREADS) {
        const double v = lnI[i];
        bad |= !isfinite(v);
        a += v;
    }
    for (int i = t; i < p.n_chunk; i += CMB_THREADS) {
        b1 += sp[2 * i];
        b2 += sp[2 * i + 1];
    }
    if (bad) s_bad = 1;
    a = warp_sumd(a);
    b1 = warp_sumd(b1);
    b2 = warp_sumd(b2);
    if (lane == 0) {
        sh[0][wid] = a;
        sh[1][wid] = b1;
        sh[2][wid] = b2;
    }
    __syncthreads();
    const int st0 = p.hp[h].status;
    const bool dead = (st0 & (CHIMERA_PT_OUT_OF_SUPPORT | CHIMERA_PT_NONMONOTONE)) != 0;
    const double N = (double)c.n_inj_total;
    if (t == 0) {  // xi and its log
        double S1 = 0.0;
        for (int w = 0; w < CMB_THREADS / 32; w++) S1 += sh[1][w];
        const double xi = dead ? 0.0 : S1 / N;
        s_xi = xi;
        s_lnxi = xi > 0.0 ? log(xi) : 0.0;
    } else if (t == 32) {  // N_eff beside it
        double S1 = 0.0, S2 = 0.0;
        for (int w = 0; w < CMB_THREADS / 32; w++) {
            S1 += sh[1][w];
            S2 += sh[2][w];
        }
        s_neff = dead ? 0.0 : (S1 > 0.0 ? S1 * S1 / (S2 - S1 * S1 / N) : 0.0);
    }
    __syncthreads();
    if (t == 0) {
        double sI = 0.0;
        for (int w = 0; w < CMB_THREADS / 32; w++) sI += sh[0][w];
        int st = st0;
        const double xi = s_xi, neff = s_neff;
        double lnL;
        if (dead) {
            lnL = -CUDART_INF;
        } else if (s_bad || !(xi > 0.0)) {
            lnL = -CUDART_INF;
            st |= CHIMERA_PT_OUT_OF_SUPPORT;
        } else {
            lnL = sI - (double)c.n_events * s_lnxi;
        }
        // the effective-count warning is only meaningful for an admissible point
        if (!dead && !(neff >= 5.0 * c.n_events)) st |= CHIMERA_PT_NEFF_LOW;
        p.lnL[h] = lnL;
        p.neff[h] = neff;
        p.xi[h] = xi;
        p.status[h] = st;
        if (p.out_lnL) p.out_lnL[h] = lnL;
        if (p.out_neff) p.out_neff[h] = neff;
        if (p.out_status) p.out_status[h] = st;
    }
}

}  // namespace

int selection_chunks(const DevCatalog &c) {
    int64_t n = (c.n_det + SEL_CHUNK - 1) / SEL_CHUNK;
    return (int)(n > 0 ? n : 1);
}

void launch_selection(const DevCatalog &c, const CallPtrs &p, int H, bool fp64, cudaStream_t st) {
    if (fp64) k_select_fp64<<<dim3(p.n_chunk, H), SEL_THREADS, 0, st>>>(c, p, H);
    else k_select_mixed<<<dim3(p.n_chunk, (H + SEL_HB - 1) / SEL_HB), SEL_THREADS, 0, st>>>(c, p, H);
}

void launch_combine(const DevCatalog &c, const CallPtrs &p, int H, cudaStream_t st) {
    k_combine<<<H, CMB_THREADS, 0, st>>>(c, p, H);
}

}  // namespace chim
