// Internal declarations shared by the CUDA translation units of libchimera.
// Device data layout, per-hyperpoint parameter block and the host-side
// launch wrappers of every kernel.  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <vector>

#include "chimera.h"

namespace chim {

constexpr double C_KMS = 299792.458;
// Forward comoving-distance table: nodes z_k = k * HT, k = 0 .. NT_FWD-1.
// HT = 10/4096 is exact in binary; node 4096 is z = 10, the end of the
// redshift search range; the table runs a little past z = 12.
constexpr double HT = 10.0 / 4096.0;
constexpr int K_Z10 = 4096;
constexpr int NT_FWD = 4918;
// Inverse table: NU intervals uniform in u = sqrt(d_L / d_top).
constexpr int NU = 2048;
// KDE window half-widths in bandwidths (mixed / FP64) and galaxy window in sigmas.
constexpr float KW32 = 5.5f;
constexpr double KW64 = 9.0;
constexpr float KWG32 = 6.0f;
constexpr int GAL_CHUNK = 256;   // galaxies per normalisation block
constexpr int GAL_DENSE = 1024;  // pixels above this gather per grid point by blocks
constexpr int GAL_HEAVY = 256;   // dense-pixel points with more candidates: a block each
constexpr int PROF_MB = 16;      // Om values per batched (mixed) profile pass
// Each KDE is zero outside the grid segment holding its samples, widened by
// KDE_MARGIN bandwidths (Sec. 2.3: evaluated only where the samples are).
constexpr double KDE_MARGIN = 6.0;
constexpr double KWG64 = 9.0;
// Mixed event kernel geometry: two instantiations, chosen per catalog at
// load time (DevCatalog::ev_geom): 10 warps with three blocks per SM when the
// catalog's largest event leaves room for three in shared memory (measured
// on the 300-event catalog: 3.7 % faster than 16 warps with two, the extra
// resident block covering the prologue and tail of the other two), else 16
// warps with two.  Both use the same table capacity and the same partition
// of the event sum, so they give the same results bit for bit.
constexpr int EV_WARPS_3 = 10, EV_WARPS_2 = 16;
constexpr int EV_RED = 256;           // threads of the event's fixed-order group sum
constexpr int DCAP = 512;             // D-table floats per warp
constexpr int GROUP_MAX = 128;        // samples per warp group (up to 4 per lane)
constexpr int CCAP = DCAP / 2 + 8;    // entries of the Gaussian factor table exp(-(ds t)^2)
// FP64 event kernel.
constexpr int EV64_THREADS = 256;
// Selection kernel: injections per block per hyperpoint.
constexpr int SEL_THREADS = 256;
constexpr int SEL_PER_THREAD = 8;
constexpr int SEL_CHUNK = SEL_THREADS * SEL_PER_THREAD;

// A double constant as an unevaluated pair of floats, x = hi + lo (the
// mixed kernels multiply by it without the float rounding of the constant).
struct F2 {
    float hi, lo;
};
inline __host__ __device__ F2 split_f2(double x) {
    F2 r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}

// Per-hyperpoint parameters, written by the cosmology kernel (FP64).
struct HP {
    double th[12];
    double cH;        // c / H0 [Mpc]
    double c_pl;      // (1 - lambda_g) / int m^-alpha over [m_min, m_max]
    double c_g;       // lambda_g / (sigma_g sqrt(2 pi) [Phi(b) - Phi(a)])
    double b1;        // 1 + beta
    double mmin_b1;   // m_min^(1+beta)
    double lmmin;     // ln m_min
    double dc_zmax;   // D_c(z_max) [Mpc]
    double d_valid;   // d_L^gw(z = 10) [Mpc]
    double F_scale;   // max over the grid of F(z_a)
    double t_valid;   // inverse-table coordinate of d_valid
    double ln_k0;     // ln(dz F_scale / (N_gal,tot sqrt(2 pi))): the mixed event kernels' log offset
    int32_t status;   // CHIMERA_PT_* bits known after the table stage
    int32_t k_valid;  // floor(t_valid), clamped
    float f_valid;    // t_valid - k_valid
    // FP32 copies for the mixed-precision kernels (converted once here, so
    // that no kernel thread runs FP64 conversions or divisions)
    float c_pl32, c_g32, alpha32, mu32, inv_sg32, mmin32, mmax32, beta32, b1_32, mmin_b1_32,
        lmmin32, xi0_32, n32, om32, gam32, kap32, l1zp32, cH32, inv_dc3_32;
    float l2min32, l2max32;  // log2 m_min, log2 m_max
    float h0_32, zp32;
    // mixed forward path (K2, K5): the mass model relative to its shared
    // normalisation w_scale = C1 m_min^-(alpha+1) |1 + beta| (log2 e in
    // place of |1 + beta| when beta = -1), C1 = c_pl (c_g when c_pl = 0),
    // and the constants of the weight and of the selection term as float pairs
    double ln_wscale;        // ln w_scale
    double inv_wscale;       // 1 / w_scale
    double ln_sel;           // ln(w_scale (3 / Dhat(z_max)^3) H0 / c): the selection terms' shared factor
    double sel_cfac;         // exp(ln_sel + the catalog's 1/pi_inj scale K ln 2)
    float r_pl32, r_g32;     // c_pl / C1, m_min^alpha c_g / C1
    F2 na2, gk2, beta2, b1_2, l2min2;  // -alpha, -log2 e / (2 sigma^2), beta, 1 + beta, log2 m_min
    F2 l2max2, b1ln2_2;                // log2 m_max, (1 + beta) ln 2
    F2 kH2;                  // H0 / c [1/Mpc]
    F2 xi0_2, omx2, nn2, nomx2;  // Xi0, 1 - Xi0, -n, n (1 - Xi0)
    F2 om2, omc2;            // Om, 1 - Om
    F2 gam2, gk_psi2, l2zp2; // gamma, gamma + kappa, log2(1 + z_p)
};

// Resident catalog (device pointers unless noted).
struct DevCatalog {
    int32_t n_events, n_z, kde_mode, gal_storage;
    int64_t n_samples, n_pix, n_gal, n_det, n_inj_total;
    double z_max, dz, n_gal_total, lambda_g, beta, d_top;
    double inv_d_top;  // 1 / d_top
    double ln_lambda, ln1m_lambda;  // ln lambda_g, ln(1 - lambda_g) (0 when the argument is 0)
    float z_max32, dz32;  // float copies for the mixed kernels
    float dz_lo32;        // dz - dz32: grid positions a dz in FP32 as fmaf(a, dz32, a dz_lo32)
    int32_t max_ns, max_seg, max_npix;
    int32_t ev_geom;      // mixed event kernel: 1 = 10 warps x 3 blocks per SM, 0 = 16 warps x 2
    // events
    int64_t *ev_soff;     // [n_events+1] sample offsets (sorted storage)
    int64_t *ev_poff;     // [n_events+1] flat pixel offsets
    int32_t *ev_order;    // [n_events] heavy-first launch order
    // per launch position (heavy-first order): the event's index and offsets,
    // read by one 32-byte load: (ev, s0, ns, zoff) and (g0, ngroups, sg0, nseg)
    int4 *ev_info;
    // KDE segments: many-1D = pixels, single-1D = events
    int64_t n_seg;
    int64_t *seg_soff;    // [n_seg+1] sample offsets of each segment
    double *seg_pf;       // [n_seg] S_ik / N_k (many-1D) or 1 / N_s (single-1D)
    int32_t *ev_segoff;   // [n_events+1] segment offsets per event
    // warp groups of the mixed event kernel, fixed at load: up to 64
    // neighbouring samples of one segment (split in two when their spread in
    // ln d_L is wide); (start relative to the event, count, segment relative
    // to the event, 0)
    int4 *groups;
    int32_t *ev_goff;     // [n_events+1] group offsets per event
    int32_t max_groups;   // most groups of any event
    float2 *ev_ref;       // [n_events] inverse-table (k bits, f) of the event's median d_L
    int2 *ev_krange;      // [n_events] smallest and largest inverse-table interval of the event's samples
    int32_t max_krange;   // most intervals any event spans (kmax - kmin + 1)
    int64_t *ev_zoff;     // [n_events+1] offsets of the events in a reweighted-sample row
                          // (each a multiple of 4 floats)
    int64_t n_zpad;       // length of a reweighted-sample row
    // pixels
    double *pix_S;        // [n_pix]
    int64_t *gal_off;     // [n_pix+1], galaxies sorted by z inside a pixel
    double *pix_sigmax;   // [n_pix] widest galaxy of the pixel (FP64 values)
    float *pix_sigmax32;  // [n_pix] widest galaxy (stored values)
    float *pix_zref;      // [n_pix] F16/BF16 offset reference
    // galaxy-profile work lists, fixed at load: every chunk of up to
    // GAL_CHUNK galaxies of one pixel (pixel, first galaxy), and the pixels
    // with more than GAL_DENSE galaxies
    int64_t n_gw;
    int32_t *gw_pix;
    int64_t *gw_g0;
    int32_t n_dense;
    int32_t *dense_pix;
    // [n_dense x n_z] per dense pixel and grid point, the galaxies whose
    // window can cover the point, [x, y) relative to the pixel's first
    // galaxy (FP64 values and reach; stored values and the mixed reach);
    // filled on the device at load
    int2 *dense_lr64, *dense_lr32;
    // the (dense pixel index, grid point) pairs whose range is not empty,
    // per precision (built at load from the ranges): the first n_dheavy hold
    // more than GAL_THREADS galaxies (a block each), the rest a warp each
    int64_t n_ditems64, n_ditems32, n_dheavy64, n_dheavy32;
    int2 *dense_items64, *dense_items32;
    // incomplete catalog: f_R and, per pixel and grid point, the missing-
    // galaxy weight (1 - P_compl) pix_area / 4 pi (nullptr when complete)
    // the "3D" kernel: samples' sky positions (device order) and pixel
    // centres in the event's flat sky chart [rad] (nullptr otherwise)
    double2 *sky_xy, *pix_xy;
    int32_t incomplete;
    double f_R;
    double *miss64;
    float *miss32;
    // galaxies
    double *gz64, *gs64;  // FP64 values
    float *gz32, *gs32;   // F32 storage
    uint16_t *gzq, *gsq;  // F16/BF16 storage (z as offset from pix_zref)
    // PE samples
    float4 *s32;          // (inverse-table interval k as int bits, fraction f, log2 m1_det, log2 m2_det)
    float2 *s32lo;        // low parts of log2 m1_det, log2 m2_det (value - the float above)
    double *sd64, *sm1_64, *sm2_64;
    // detected injections
    float4 *i32a;         // (k bits, f, log2 m1_det, log2 m2_det)
    float2 *i32lo;        // low parts of log2 m1_det, log2 m2_det
    float2 *i32b;         // (d_L, ln pi_inj)
    float *iipi32;        // 2^-K / pi_inj, computed in FP64 and rounded (mixed selection)
    double ln_ipi_shift;  // K ln 2
    double *id64, *im1_64, *im2_64, *ilp64;
    // tensor-core galaxy profiles (photometric catalogs; tc_ok = 0 when the
    // catalog takes the FP32 kernels): the padded 64-galaxy blocks (pixel,
    // first galaxy), the gather items (pixel, grid tile, first and end block
    // relative to the item's group) with their partial slot (or -1), and the
    // reductions of split items (pixel, grid tile, first slot, slots)
    int32_t tc_ok;
    float tc_sc;  // scale of the 1/Z operand (a power of two)
    int64_t tc_nblk;
    int2 *tc_blk;
    float2 *tc_coef;  // [tc_nblk x 64] each slot's Gaussian coefficients (c_g, d_g); (0, -1e4) for no galaxy
    int4 *tc_items;
    int32_t *tc_islot;
    int4 *tc_reds;
};

// Per-call views the kernels need for hyperpoint h.
struct CallPtrs {
    const double *theta;      // [H x 12]
    HP *hp;                   // [H]
    const double *const *fwd; // [H] forward table of h's Om (device pointer array)
    double2 *inv64;           // [H x (NU+1)] (z_k, dz/du_k)
    float4 *inv32;            // [H x NU] (z_k, dz/du_k / NU, z_k+1, dz/du_k+1 / NU)
    float4 *linv32;           // [H x NU] the same for log2(1 + z), or nullptr
    double *F64;              // [H x n_z]
    float *F32;               // [H x n_z], F / F_scale
    const void *const *prof;  // [H] galaxy profile base (double* or float*) of h's Om
    double *lnI;              // [H x n_events]
    double *bw;               // [H x n_events]
    double *selp;             // [H x n_chunk x 2] selection partial sums (scratch)
    float *zw;                // [tile x 2 x n_zpad] reweighted samples (z row, then w row) of a
                              // tile of hyperpoints (mixed path)
    int32_t n_chunk;
    int32_t kshape;           // KDE kernel: 0 Gaussian, 1 Epanechnikov
    int32_t jac_ps;           // 1: the Jacobian of Eq. jacobian on each sample's weight, not on the grid
    double *lnL, *neff, *xi;  // [H]
    int32_t *status;          // [H]
    unsigned long long *pairs;  // [H] windowed-pair counter, or nullptr
    // caller buffers [H] that the combine kernel also fills (device entry
    // point), or nullptr
    double *out_lnL, *out_neff;
    int32_t *out_status;
};

// ---- launch wrappers (host) ----
// K1a: forward table D_c(z_k) / (c/H0) for one Om into `out` [NT_FWD].
void launch_fwd_table(double Om, double *out, cudaStream_t st);
// The tables (or, dOm, their Om derivatives d/dOm of D_c(z_k)/(c/H0), for
// the adjoint) of up to FWD_MB Om values in one launch pair; each equals the
// one-Om launch's.
constexpr int FWD_MB = 32;
struct FwdBatch {
    int n;
    double Om[FWD_MB];
    double *out[FWD_MB];
};
void launch_fwd_tables(const FwdBatch &b, bool dOm, cudaStream_t st);
// K1b: per-hyperpoint parameters, inverse tables, grid factors (F64 for
// fp64, normalised F32 otherwise), status.  dk: scratch of at least
// H x NT_FWD x 8 bytes (FP32 d_L^gw and J at the forward nodes),
// fmax_bits: [H] scratch.
// Every call gets the FP64 inverse nodes (inv64) and their rounded FP32
// pairs (inv32, and linv32 for log2(1+z) when given).
void launch_hyper_tables(const DevCatalog &c, const CallPtrs &p, int H, bool fp64, double *dk,
                         unsigned long long *fmax_bits, cudaStream_t st);
// The same with k_hyper_final on a side stream beside k_inv_nodes (forked
// after the forward nodes with ev_fork, joined back into st with ev_join).
cudaError_t launch_hyper_tables(const DevCatalog &c, const CallPtrs &p, int H, bool fp64, double *dk,
                                unsigned long long *fmax_bits, cudaStream_t st, cudaStream_t side,
                                cudaEvent_t ev_fork, cudaEvent_t ev_join);
// K3: galaxy redshift prior on the grid for one Om.  dv: scratch of n_z
// doubles followed by n_z floats, invZ: [n_gal] scratch; out64 (FP64
// values) or out32 (stored values).
void launch_galaxy_profile(const DevCatalog &c, const double *fwd, double Om, double *dv,
                           double *invZ64, float *invZ32, double *out64, float *out32,
                           cudaStream_t st);
// The mixed-path profiles of up to PROF_MB Om values in one pass: the
// galaxies' Gaussians (Om-independent) are evaluated once and contracted with
// the PROF_MB columns of dV_c/dz and 1/Z_g.  Unused slots repeat slot 0 and
// have out = nullptr.  dvm: [(n_z + 1) x PROF_MB] floats scratch, invZm:
// [n_gal x PROF_MB] floats scratch; each out[j] [n_pix x n_z].  Every value
// equals the one-Om launch's bit for bit (same operations in the same order).
// With fwdO set (dOm), the dG/dOm rows instead (invZm then [2 x n_gal x
// PROF_MB], dvm [2 x (n_z + 1) x PROF_MB]).
struct MultiOm {
    int n;
    const double *fwd[PROF_MB];
    const double *fwdO[PROF_MB];
    double Om[PROF_MB];
    float *out[PROF_MB];
};
void launch_galaxy_profile_multi(const DevCatalog &c, const MultiOm &m, bool dOm, float *dvm, float *invZm,
                                 cudaStream_t st);
// The mixed-path profiles of up to TC_COLS Om values on the tensor cores
// (galaxy_tc.cu), for catalogs whose galaxies are all wide (photometric):
// two tcgen05 contractions of the FP16 Gaussians with the Om-dependent
// columns split in two FP16 terms, FP32 accumulation with the tensor-memory
// partial sums promoted into an FP32 running sum every TC_PROMO stages.
constexpr int TC_M = 128;               // Om columns per batch (the MMA's M)
constexpr int TC_N = 256;               // galaxies (norm pass) or grid points (gather pass) per tile
constexpr int TC_K = 64;                // K per stage (one 128-byte row of FP16)
constexpr int TC_COLS = TC_M;           // Om columns per batch
constexpr int TC_PROMO = 1;             // stages accumulated in tensor memory before each promotion
constexpr int64_t TC_MIN_GAL = 4096;    // smaller catalogs take the FP32 kernels
constexpr double TC_SIGMA_MIN = 0.02;   // narrowest galaxy of a tensor-core catalog
constexpr int64_t TC_GRP_BLK = 16384;   // 64-galaxy blocks per group of pixels (operand images: 512 MiB)
constexpr int TC_KSPLIT = 128;          // blocks per gather item; longer ranges are split
struct TcBatch {
    int n_cols, nkc;
    float sc, gfac;     // 1/Z scale; 2^12 / (dz sc)
    uint4 *vimg;        // [nkc][hi, lo] 16 KB images of the norm pass's column operand
    float *dvT;         // [TC_COLS][n_z] dv_j(z_a)
    uint4 *cimg;        // [group blocks][hi, lo] 16 KB images of 1/Z
    float *part;        // [slots][TC_M][TC_N] partial sums of split items
    int *err;           // [16]: [0] timeout flag, [4..7] item counters
    float *out[TC_COLS];
};
struct TcCols {
    int n;
    const double *fwd[TC_COLS];
    double Om[TC_COLS];
};
struct TcHost {
    std::vector<int64_t> gblk, gitem, gred;  // [groups + 1] offsets of blocks, items, reductions
    int64_t max_gblk = 0;
    int32_t max_slots = 0;
};
size_t tc_scratch_bytes(const DevCatalog &c, const TcHost &h);
int launch_galaxy_profile_tc(const DevCatalog &c, const TcHost &h, const TcCols &m, float *const *out, char *scratch,
                             cudaStream_t st);
// Load-time plan from the galaxies' stored (z, sigma) as the kernels decode
// them (sorted by z inside a pixel) and each pixel's widest stored sigma;
// sets c.tc_ok, c.tc_sc, c.tc_nblk and fills the lists.
void tc_plan(int64_t np, const int64_t *goff, const float *zs, const float *ss, const float *smax, int n_z,
             double dz, bool incomplete, int kde_mode, DevCatalog &c, TcHost &h, std::vector<int2> &blk,
             std::vector<float2> &coef, std::vector<int4> &items, std::vector<int32_t> &islot,
             std::vector<int4> &reds);
// dG/dOm of the galaxy profile (FP64 from dv, dvO, or FP32 from their FP32
// copies); invZ, ZO: [n_gal] scratch of the precision's type; out [n_pix x n_z].
// fwd, fwdO: the D_c table and its Om derivative (the missing-galaxy term of
// an incomplete catalog needs D_c(z_max) and its derivative).
void launch_galaxy_dOm(const DevCatalog &c, const double *fwd, const double *fwdO, double Om, const double *dv,
                       const double *dvO, const float *dv32, const float *dvO32, bool f64, void *invZ, void *ZO,
                       void *out, cudaStream_t st);
// Candidate galaxy ranges of the dense pixels (Om-independent), into
// c.dense_lr64 / c.dense_lr32.
void launch_dense_ranges(const DevCatalog &c, cudaStream_t st);
// Single-1D sky-summed profile: outh[event][a] = sum_k S_k G[k][a].
void launch_profile_sum(const DevCatalog &c, const double *G64, const float *G32, double *outh64,
                        float *outh32, cudaStream_t st);
// K2+K4: per-event ln I for every (event, h).
// Mixed: reweighting (K2) into p.zw, then the event integral (K4) from it,
// for the hyperpoints h0 .. h0+nh-1 (nh at most the tile the buffer holds).
void launch_reweight(const DevCatalog &c, const CallPtrs &p, int h0, int nh, cudaStream_t st);
void launch_event_mixed(const DevCatalog &c, const CallPtrs &p, int h0, int nh, cudaStream_t st);
void launch_event_fp64(const DevCatalog &c, const CallPtrs &p, int H, cudaStream_t st);
// K4 with the binned KDE (CHIMERA_MIXED_BINNED), or (binned = false) the
// direct one-evaluation-per-pair form used for the Epanechnikov kernel, from
// the same tile buffer as launch_event_mixed.
void launch_event_binned(const DevCatalog &c, const CallPtrs &p, int h0, int nh, bool binned,
                         cudaStream_t st);
size_t event_binned_smem(const DevCatalog &c);
size_t event_mixed_smem(const DevCatalog &c, int geom);
// The mixed event kernel's geometry for a catalog (DevCatalog::ev_geom).
int event_mixed_pick(const DevCatalog &c);
size_t event_fp64_smem(const DevCatalog &c);
// The "3D" kernel of CHIMERA_KDE_3D catalogs (FP64 only).
size_t event_3d_smem(const DevCatalog &c);
void launch_event_3d(const DevCatalog &c, const CallPtrs &p, int H, cudaStream_t st);
// K5: selection partial sums; K6: combine into ln L.
void launch_selection(const DevCatalog &c, const CallPtrs &p, int H, bool fp64, cudaStream_t st);
// raw: the mixed event kernel left raw integrals in lnI (K6 takes the log).
void launch_combine(const DevCatalog &c, const CallPtrs &p, int H, cudaStream_t st);
int selection_chunks(const DevCatalog &c);
// K8 microbenchmarks.
int run_peaks(double *out, cudaStream_t st);

}  // namespace chim

// ---- device helpers shared by the kernels ----
namespace chimd {

__device__ __forceinline__ double E_of(double z, double Om) {
    double a = 1.0 + z;
    return sqrt(Om * a * a * a + 1.0 - Om);
}

// Cubic Hermite interpolation of D_c/(c/H0) on the forward table; the node
// derivatives are 1/E(z_k) exactly.
__device__ __forceinline__ double dc_hermite(const double *fwd, double z, double Om) {
    double t = z / chim::HT;
    int k = (int)floor(t);
    if (k < 0) k = 0;
    if (k > chim::NT_FWD - 2) k = chim::NT_FWD - 2;
    double f = t - k;
    double z0 = k * chim::HT, z1 = (k + 1) * chim::HT;
    double p0 = fwd[k], p1 = fwd[k + 1];
    double m0 = chim::HT / E_of(z0, Om), m1 = chim::HT / E_of(z1, Om);
    double f2 = f * f, f3 = f2 * f;
    return (2 * f3 - 3 * f2 + 1) * p0 + (f3 - 2 * f2 + f) * m0 + (-2 * f3 + 3 * f2) * p1 +
           (f3 - f2) * m1;
}

// Hermite interpolation of dDhat/dOm (node derivatives known in closed form).
__device__ __forceinline__ double dcO_hermite(const double *fwdO, double z, double Om) {
    double t = z / chim::HT;
    int k = (int)floor(t);
    if (k < 0) k = 0;
    if (k > chim::NT_FWD - 2) k = chim::NT_FWD - 2;
    double f = t - k;
    auto g = [Om](double zz) {
        double a = 1.0 + zz, E = chimd::E_of(zz, Om);
        return -0.5 * (a * a * a - 1.0) / (E * E * E);
    };
    double m0 = chim::HT * g(k * chim::HT), m1 = chim::HT * g((k + 1) * chim::HT);
    double f2 = f * f, f3 = f2 * f;
    return (2 * f3 - 3 * f2 + 1) * fwdO[k] + (f3 - 2 * f2 + f) * m0 + (-2 * f3 + 3 * f2) * fwdO[k + 1] +
           (f3 - f2) * m1;
}

// dV_c/dz up to constants, D^2/E (D = D_c/(c/H0)), and with fwdO its Om
// derivative.  Shared by every kernel that builds a galaxy profile so that
// they agree bit for bit.
__device__ __forceinline__ double dv_of(const double *fwd, double z, double Om) {
    const double D = dc_hermite(fwd, z, Om);
    return D * D / E_of(z, Om);
}
__device__ __forceinline__ void dv_pair(const double *fwd, const double *fwdO, double z, double Om, double &dv,
                                        double &dvO) {
    const double ap = 1.0 + z;
    const double D = dc_hermite(fwd, z, Om), DO = dcO_hermite(fwdO, z, Om), E = E_of(z, Om);
    dv = D * D / E;
    dvO = 2.0 * D * DO / E - D * D * (ap * ap * ap - 1.0) * 0.5 / (E * E * E);
}
// Scales of the missing-galaxy term of an incomplete catalog:
// c1 = 3 N_gal,tot / D_max^3 (so that c1 dv = N_gal,tot dV_c/dz / V_c(z_max))
// and, with fwdO, c2 = -3 c1 D_max'/D_max (d/dOm of c1 dv = c1 dv' + c2 dv).
__device__ __forceinline__ void miss_scales(const double *fwd, const double *fwdO, double zmax, double Om, double N,
                                            double &c1, double &c2) {
    const double D = dc_hermite(fwd, zmax, Om), D3 = D * D * D;
    c1 = 3.0 * N / D3;
    c2 = fwdO ? -3.0 * c1 * dcO_hermite(fwdO, zmax, Om) / D : 0.0;
}

__device__ __forceinline__ double xi_of(double z, double xi0, double n) {
    return xi0 + (1.0 - xi0) * pow(1.0 + z, -n);
}

// d_L^gw and its z-derivative J from D_c (Mpc) at z, Eq. dL-mg and its
// product-rule derivative.
// 1 / sqrt(x) in FP64 for x of order one to a few hundred: the SFU's FP32
// estimate (rsqrtf, relative error ~2^-22) refined by two Newton-Raphson
// steps on f(y) = y^-2 - x, y <- y (3 - x y^2) / 2, each of which squares
// the relative error (2^-43, then below FP64 rounding): a handful of FP64
// operations in place of a square root and a division, which matter on
// B300's narrow FP64 pipe.
__device__ __forceinline__ double rsqrt64(double x) {
    double y = (double)rsqrtf((float)x);
    y = y * (1.5 - 0.5 * x * y * y);
    return y * (1.5 - 0.5 * x * y * y);
}
// The FP64 forward relation (as dc_hermite and dgw_J) with 1/E from
// rsqrt64, for the inverse nodes and the Newton steps of the FP64 redshifts:
// D_c by cubic Hermite on the forward table (slopes HT / E at the nodes),
// d_L^gw and J = d d_L^gw / dz (Eqs. dL-em, dL-mg).
__device__ __forceinline__ double dc_hermite_r(const double *fwd, double z, double Om) {
    const double t = z * (4096.0 / 10.0);  // z / HT (a product: no FP64 division)
    int k = (int)floor(t);
    if (k < 0) k = 0;
    if (k > chim::NT_FWD - 2) k = chim::NT_FWD - 2;
    const double f = t - k, a0 = 1.0 + k * chim::HT, a1 = 1.0 + (k + 1) * chim::HT;
    const double m0 = chim::HT * rsqrt64(Om * a0 * a0 * a0 + 1.0 - Om), m1 = chim::HT * rsqrt64(Om * a1 * a1 * a1 + 1.0 - Om);
    const double f2 = f * f, f3 = f2 * f;
    return (2 * f3 - 3 * f2 + 1) * fwd[k] + (f3 - 2 * f2 + f) * m0 + (-2 * f3 + 3 * f2) * fwd[k + 1] + (f3 - f2) * m1;
}
__device__ __forceinline__ void dgw_J_r(double z, double Dc, const double *th, double cH, double *d, double *J) {
    const double a = 1.0 + z;
    const double p = exp(-th[3] * log(a));  // (1+z)^-n
    const double xi = th[2] + (1.0 - th[2]) * p;
    const double dxi = -th[3] * (1.0 - th[2]) * p / a;
    const double rE = rsqrt64(th[1] * a * a * a + 1.0 - th[1]);
    *d = a * Dc * xi;
    *J = (Dc + a * cH * rE) * xi + a * Dc * dxi;
}

__device__ __forceinline__ void dgw_J(double z, double Dc, const double *th, double cH, double *d,
                                      double *J) {
    double a = 1.0 + z;
    double p = exp(-th[3] * log(a));  // (1+z)^-n
    double xi = th[2] + (1.0 - th[2]) * p;
    double dxi = -th[3] * (1.0 - th[2]) * p / a;
    double E = E_of(z, th[1]);
    *d = a * Dc * xi;
    *J = (Dc + a * cH / E) * xi + a * Dc * dxi;
}

// Madau-Dickinson shape (Sec. 3.1), unnormalised.
__device__ __forceinline__ double psi_of(double z, const double *th) {
    const double la = log(1.0 + z);
    return exp(th[9] * la) / (1.0 + exp((th[9] + th[10]) * (la - log1p(th[11]))));
}

// Galaxy (z, sigma) as the device stores it for the mixed path: F32, or
// F16/BF16 with z as an offset from the pixel's reference redshift.
__device__ __forceinline__ void gal32(const chim::DevCatalog &c, int64_t p, int64_t g, float &z, float &s) {
    if (c.gal_storage == CHIMERA_GAL_F32) {
        z = c.gz32[g];
        s = c.gs32[g];
    } else if (c.gal_storage == CHIMERA_GAL_F16) {
        z = c.pix_zref[p] + __half2float(__ushort_as_half(c.gzq[g]));
        s = __half2float(__ushort_as_half(c.gsq[g]));
    } else {
        z = c.pix_zref[p] + __uint_as_float(((uint32_t)c.gzq[g]) << 16);
        s = __uint_as_float(((uint32_t)c.gsq[g]) << 16);
    }
}

// Grid window of a galaxy on the mixed path: the points within KWG32 sigma
// of its redshift, [lo, hi] (empty when hi < lo).  The forward profile and
// its Om derivative take their windows from here, so that every galaxy
// keeps unit weight on the same grid points in both.
__device__ __forceinline__ void gal_window32(float zg, float sg, float inv_dz, int nz, int &lo, int &hi) {
    const float kw = chim::KWG32 * sg;
    const float a0 = ceilf((zg - kw) * inv_dz), a1 = floorf((zg + kw) * inv_dz);
    lo = a0 < 0.f ? 0 : (a0 > (float)nz ? nz : (int)a0);
    hi = a1 > (float)(nz - 1) ? nz - 1 : (a1 < -1.f ? -1 : (int)a1);
}

__device__ __forceinline__ float hermite4(float4 nd, float f) {
    float f2 = f * f, f3 = f2 * f;
    return (2.f * f3 - 3.f * f2 + 1.f) * nd.x + (f3 - 2.f * f2 + f) * nd.y +
           (-2.f * f3 + 3.f * f2) * nd.z + (f3 - f2) * nd.w;
}

}  // namespace chimd
