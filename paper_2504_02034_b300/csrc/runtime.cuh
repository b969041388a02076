// Host runtime of libchimera: context, budgeted device allocator, resident
// catalogs, per-Om caches and per-stream workspaces.  Internal only.
#pragma once

#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace chim {

void set_error(const std::string &msg);

// Admissibility of a hyperparameter point (every component finite, H0 > 0,
// Om in [0, 1], Xi0 > 0, sigma_g > 0, 0 < m_min < m_max, z_p > -1); an
// inadmissible point is evaluated at kSafeTheta instead and reported as
// OUT_OF_SUPPORT with ln L = -inf.
inline bool theta_admissible(const double *t) {
    for (int k = 0; k < 12; k++)
        if (!std::isfinite(t[k])) return false;
    return t[0] > 0.0 && t[1] >= 0.0 && t[1] <= 1.0 && t[2] > 0.0 && t[6] > 0.0 && t[7] > 0.0 &&
           t[8] > t[7] && t[11] > -1.0;
}
inline constexpr double kSafeTheta[12] = {70.0, 0.3, 1.0, 1.91, 3.4, 34.0, 3.6, 5.0, 100.0, 2.7, 3.0, 2.0};

struct Ctx;

// Forward table cache entry (one per distinct Om).
struct FwdEntry {
    double *table = nullptr;
    cudaEvent_t ready = nullptr;
    uint64_t last_use = 0;  // Ctx::tick of the last call that read it
};

// Galaxy profile cache entry for one (Om, kind) of one catalog.  Kinds:
// 0 FP64 profile, 1 FP32 profile of the stored galaxy values, 2 FP64 dG/dOm,
// 3 FP32 dG/dOm of the stored galaxy values.
struct ProfEntry {
    void *G = nullptr;   // [n_pix x n_z] double (kind 0) or float (kind 1)
    void *Gh = nullptr;  // single-1D: [n_events x n_z]
    size_t bytes = 0;    // bytes of G
    size_t hbytes = 0;   // bytes of Gh
    cudaEvent_t ready = nullptr;
    uint64_t last_use = 0;
};

struct Catalog {
    DevCatalog d{};
    std::vector<void *> allocs;
    size_t bytes = 0;
    chimera_catalog_info_t info{};
    std::map<std::pair<uint64_t, int>, ProfEntry> prof;
    std::atomic<int> in_use{0};
    TcHost tc;  // tensor-core profile plan (used when d.tc_ok)
    bool ev_tuned = false;  // the mixed event kernel's geometry timed on a first call
};

// Device and pinned buffers for one stream of likelihood calls.
struct Workspace {
    cudaStream_t st = nullptr;
    int Hcap = 0;
    int64_t nev_cap = 0;
    int nz_cap = 0;
    int nchunk_cap = 0;
    size_t bytes = 0;
    // device
    char *param = nullptr;  // theta | status | fwd ptrs | prof ptrs
    HP *hp = nullptr;
    double2 *inv64 = nullptr;
    float4 *inv32 = nullptr;
    float4 *linv32 = nullptr;
    double *F64 = nullptr;
    float *F32 = nullptr;
    double *lnI = nullptr, *bw = nullptr, *selp = nullptr;
    double *lnL = nullptr, *neff = nullptr, *xi = nullptr;
    double *dk = nullptr;                  // [H x NT_FWD] forward-node scratch (FP32 d, J)
    float *zw = nullptr;                   // [tile x 2 x n_zpad] reweighted samples (mixed)
    size_t zw_bytes = 0;                   // its size; a call's tile is zw_bytes / (8 n_zpad) points
    unsigned long long *fmax_bits = nullptr;  // [H]
    // adjoint buffers
    double *grad = nullptr;       // [H x 12]
    char *gscr = nullptr;         // adjoint scratch (allocated on the first gradient call)
    size_t gscr_bytes = 0;
    char *ahstage = nullptr;      // pinned staging of the adjoint's pointer arrays
    size_t ahstage_bytes = 0;
    // windowed-pair counters (roofline accounting), used when count_pairs
    unsigned long long *pairs = nullptr;
    bool count_pairs = false;
    // second stream for the selection term, which runs beside the event
    // kernels (fork after the per-point tables, join before the combine)
    cudaStream_t st2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_tab_fork = nullptr, ev_tab_join = nullptr;  // per-point tables: k_hyper_final on st2
    // stage tracing (CUDA events around K1, K3, K4, K5, K6, K7)
    bool trace = false;
    cudaEvent_t tev[10] = {};
    bool traced_adjoint = false;
    std::vector<cudaEvent_t> tile_ev;  // mixed: after the reweighting and after K4 of each tile
    int traced_tiles = 0;
    // host pinned staging
    char *hstage = nullptr;
    size_t hstage_bytes = 0;
    std::vector<void *> allocs;
    CallPtrs ptrs(int H, const DevCatalog &c) const;
    size_t param_bytes(int H) const { return (size_t)H * (12 * 8 + 8 + 8 + 8); }
};

struct Server;

// Scratch of the galaxy-profile kernels: the dV_c/dz column(s) and the
// per-galaxy normalisations 1/Z_g of one Om, or of PROF_MB Om values at a
// time on the batched path, and for the adjoint Z_g' and dV_c/dz'.  One per
// context, shared by its workspace and the serving lanes': profiles are
// computed only on a cache miss, and the batched part alone takes
// 2 x 4 x PROF_MB = 128 bytes per galaxy.  Uses are enqueued under the
// context's mutex; each waits on `done` of the previous use and records it
// after its own kernels.
struct ProfScratch {
    char *base = nullptr;
    size_t bytes = 0;
    cudaEvent_t done = nullptr;
    bool recorded = false;
    uint64_t last_use = 0;
};
// The scratch's regions for one catalog (they alias: the one-Om, batched
// and adjoint kernels of a call run one after another on one stream).
struct ProfView {
    double *dv;           // [n_z] FP64, then [n_z] FP32
    double *invZ64;       // [n_gal]
    float *invZ32;        // [n_gal]
    float *dvm, *invZm;   // [2 x (n_z+1) x PROF_MB], [2 x n_gal x PROF_MB]
    double *adv, *advO;   // adjoint: [n_z] FP64 then [n_z] FP32, each
    double *ainvZ, *aZO;  // adjoint: [n_gal] each
    char *tc;             // tensor-core profiles: tc_scratch_bytes
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t dev_done = nullptr;  // device entry point: the caller's stream waits on it
    double *dev_theta_h = nullptr;   // device entry point: pinned host copy of theta
    size_t dev_theta_cap = 0;        // its capacity in doubles
    cudaMemPool_t pool = nullptr;    // cache entries (cache_alloc)
    size_t budget = 0;
    std::atomic<size_t> used{0};
    std::recursive_mutex mu;
    std::map<int32_t, std::shared_ptr<Catalog>> cats;
    int32_t next_id = 0;
    std::unordered_map<uint64_t, FwdEntry> fwd;
    std::unordered_map<uint64_t, FwdEntry> fwdO;  // dDhat/dOm tables (adjoint)
    Workspace ws;
    uint64_t tick = 0;
    Server *server = nullptr;
    ProfScratch ps;
};

// Budgeted allocation; returns a CHIMERA_ERR_* code.
int dev_alloc(Ctx &ctx, void **p, size_t bytes);
void dev_free(Ctx &ctx, void *p, size_t bytes);
// Cache entries (distance tables, galaxy profiles and their Om derivatives)
// come from the context's stream-ordered memory pool, which keeps freed
// memory for reuse: a call with many new Om values allocates without a
// cudaMalloc each.  The allocation is ordered on `st`; other streams use the
// entry after waiting on its ready event.  cache_free is called only with
// the device idle (eviction, unload, destroy).
int cache_alloc(Ctx &ctx, void **p, size_t bytes, cudaStream_t st);
void cache_free(Ctx &ctx, void *p, size_t bytes);
void trim_cache_pool(Ctx &ctx);

int ws_ensure(Ctx &ctx, Workspace &ws, int H, const Catalog &cat);
void ws_release(Ctx &ctx, Workspace &ws);
// Destroys the workspace's side stream and fork/join events.
void ws_destroy_streams(Workspace &ws);

// Forward pass for H points on workspace `ws` (enqueued on ws.st).
// theta: host [H x 12].  Leaves lnL / neff / xi / status / lnI / bw on the
// device in `ws`.  Returns a CHIMERA_ERR_* code.
// The forward pass; out_* (device, may be nullptr) also receive ln L, N_eff
// and the status words from the combine kernel.
// PREC_WITH_GRAD, OR'ed into the precision by the gradient entry points only:
// the forward pass of a gradient call (keeps the FP64 inverse nodes the
// adjoint reads).
constexpr int PREC_WITH_GRAD = 0x1000;
int forward(Ctx &ctx, Catalog &cat, Workspace &ws, int H, const double *theta, int precision,
            double *out_lnL = nullptr, double *out_neff = nullptr, int32_t *out_status = nullptr);
// Adjoint after forward() on the same workspace (reads the sanitised theta
// and the forward tables forward() left there); leaves grad [H x 12].
int backward(Ctx &ctx, Catalog &cat, Workspace &ws, int H, int precision);
// Releases the adjoint's scratch of a workspace.
void adjoint_release(Ctx &ctx, Workspace &ws);

// Cache helpers shared by the forward and adjoint orchestration.
uint64_t bits_of(double x);
int fwd_table(Ctx &ctx, double Om, cudaStream_t st, const double **out);
int fwd_tables(Ctx &ctx, const double *Om, int n, cudaStream_t st, const double **out, bool dOm);
void evict_profiles(Ctx &ctx, Catalog &cat, size_t need);
bool make_room(Ctx &ctx, size_t need);
// The profile scratch sized for catalog c, after the previous use on any
// stream (st waits on it); release records the end of this use on st.
int prof_scratch_acquire(Ctx &ctx, const DevCatalog &c, cudaStream_t st, ProfView *v, const TcHost *tc = nullptr);
int prof_scratch_release(Ctx &ctx, cudaStream_t st);
void prof_scratch_free(Ctx &ctx);
void free_prof_entry(Ctx &ctx, ProfEntry &e);

std::shared_ptr<Catalog> find_catalog(Ctx &ctx, int32_t id);

int cuda_check(cudaError_t e, const char *what);

// serving
int serve_submit(Ctx &ctx, int32_t cat, int32_t n, const double *theta, int32_t flags,
                 uint64_t *ticket);
int serve_poll(Ctx &ctx, uint64_t ticket, int64_t timeout_us, double *lnL, double *dlnL,
               int32_t *status);
int serve_cancel(Ctx &ctx, uint64_t ticket);
int serve_stats(Ctx &ctx, chimera_serve_stats_t *out);
int serve_reset_stats(Ctx &ctx);
void serve_shutdown(Ctx &ctx);
// Bytes held by the serving lanes' workspaces (called under ctx.mu).
size_t serve_ws_bytes(Ctx &ctx);

}  // namespace chim
