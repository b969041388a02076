// C ABI of libchimera (include/chimera.h) and the host runtime behind it:
// budgeted device allocation, catalog packing and residency, per-Om caches
// of the forward distance table and of the galaxy profile, and the
// orchestration of the kernels K1 -> K3 -> K2/K4 -> K5 -> K6 on a stream.
#include <algorithm>
#include <cmath>
#include <functional>
#include <cstdio>
#include <cstdlib>
#include <numeric>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "runtime.cuh"

namespace chim {

// ------------------------------------------------------------ errors ----
static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

int cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return CHIMERA_OK;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return CHIMERA_ERR_CUDA;
}

#define CK(call)                                               \
    do {                                                       \
        int rc_ = cuda_check((call), #call);                   \
        if (rc_) return rc_;                                   \
    } while (0)
#define RC(call)                                               \
    do {                                                       \
        int rc_ = (call);                                      \
        if (rc_) return rc_;                                   \
    } while (0)

// ------------------------------------------------------- allocation ----
// CHIMERA_FAULT_ALLOC=N makes the N-th device allocation fail, counted from
// the moment the variable took its current value (host-side fault injection
// for tests: a test sets it to 1 and the next budgeted allocation fails).
static std::mutex g_fault_mu;
static std::string g_fault_val;
static long g_alloc_count = 0;

static bool injected_alloc_failure() {
    const char *f = getenv("CHIMERA_FAULT_ALLOC");
    std::lock_guard<std::mutex> lk(g_fault_mu);
    const std::string v = f ? f : "";
    if (v != g_fault_val) {
        g_fault_val = v;
        g_alloc_count = 0;
    }
    const long n = ++g_alloc_count;
    return f && atol(f) == n;
}

int dev_alloc(Ctx &ctx, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (injected_alloc_failure()) {
        set_error("injected allocation failure (CHIMERA_FAULT_ALLOC)");
        return CHIMERA_ERR_CUDA;
    }
    if (ctx.used.load() + bytes > ctx.budget && !make_room(ctx, bytes)) {
        set_error("allocation of " + std::to_string(bytes) + " bytes exceeds the HBM budget");
        return CHIMERA_ERR_ADMISSION;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return cuda_check(e, "cudaMalloc");
    }
    ctx.used += bytes;
    return CHIMERA_OK;
}

void dev_free(Ctx &ctx, void *p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    cudaFree(p);
    ctx.used -= bytes;
}

int cache_alloc(Ctx &ctx, void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    long n = ++g_alloc_count;
    if (const char *f = getenv("CHIMERA_FAULT_ALLOC")) {
        if (atol(f) == n) {
            set_error("injected allocation failure (CHIMERA_FAULT_ALLOC)");
            return CHIMERA_ERR_CUDA;
        }
    }
    if (ctx.used.load() + bytes > ctx.budget && !make_room(ctx, bytes)) {
        set_error("allocation of " + std::to_string(bytes) + " bytes exceeds the HBM budget");
        return CHIMERA_ERR_ADMISSION;
    }
    if (!ctx.pool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = ctx.device;
        cudaError_t e = cudaMemPoolCreate(&ctx.pool, &props);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx.pool = nullptr;
            return cuda_check(e, "cudaMemPoolCreate");
        }
        uint64_t keep = UINT64_MAX;  // freed memory stays in the pool
        cudaMemPoolSetAttribute(ctx.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx.pool, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return cuda_check(e, "cudaMallocFromPoolAsync");
    }
    ctx.used += bytes;
    return CHIMERA_OK;
}

void cache_free(Ctx &ctx, void *p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    cudaFreeAsync(p, ctx.stream);
    ctx.used -= bytes;
}

// Returns the pool's unused memory to the device (after evictions and
// unloads), so that the budget accounting stays a bound on what is held.
void trim_cache_pool(Ctx &ctx) {
    if (!ctx.pool) return;
    cudaStreamSynchronize(ctx.stream);
    cudaMemPoolTrimTo(ctx.pool, 0);
}

// ------------------------------------------------------- workspace ----
CallPtrs Workspace::ptrs(int H, const DevCatalog &c) const {
    CallPtrs p{};
    char *q = param;
    p.theta = reinterpret_cast<const double *>(q);
    q += sizeof(double) * 12 * H;
    p.status = reinterpret_cast<int32_t *>(q);
    q += sizeof(int64_t) * H;  // int32 status padded to 8 bytes
    p.fwd = reinterpret_cast<const double *const *>(q);
    q += sizeof(void *) * H;
    p.prof = reinterpret_cast<const void *const *>(q);
    p.hp = hp;
    p.inv64 = inv64;
    p.inv32 = inv32;
    p.linv32 = linv32;
    p.F64 = F64;
    p.F32 = F32;
    p.lnI = lnI;
    p.bw = bw;
    p.selp = selp;
    p.zw = zw;
    p.n_chunk = selection_chunks(c);
    p.lnL = lnL;
    p.neff = neff;
    p.xi = xi;
    p.pairs = count_pairs ? pairs : nullptr;
    return p;
}

void ws_destroy_streams(Workspace &ws) {
    if (ws.st2) cudaStreamSynchronize(ws.st2);
    if (ws.ev_fork) cudaEventDestroy(ws.ev_fork);
    if (ws.ev_join) cudaEventDestroy(ws.ev_join);
    if (ws.ev_tab_fork) cudaEventDestroy(ws.ev_tab_fork);
    if (ws.ev_tab_join) cudaEventDestroy(ws.ev_tab_join);
    if (ws.st2) cudaStreamDestroy(ws.st2);
    ws.st2 = nullptr;
    ws.ev_fork = ws.ev_join = ws.ev_tab_fork = ws.ev_tab_join = nullptr;
}

void ws_release(Ctx &ctx, Workspace &ws) {
    adjoint_release(ctx, ws);
    for (void *a : ws.allocs) cudaFree(a);
    ws.allocs.clear();
    ctx.used -= ws.bytes;
    ws.bytes = 0;
    if (ws.hstage) cudaFreeHost(ws.hstage);
    ws.hstage = nullptr;
    ws.hstage_bytes = 0;
    ws.Hcap = 0;
    ws.nev_cap = 0;
    ws.nz_cap = 0;
    ws.nchunk_cap = 0;
    ws.zw_bytes = 0;
}

// Bytes of the reweighting tile buffer for H points of a catalog: z and w of
// every sample for as many points as fit the cap (at least one point).  The
// cap is 1/32 of the context's HBM budget, within [1 GiB, 8 GiB]: measured on
// the photometric 300-event catalog at 512 points per launch, caps of 256 MiB,
// 1, 4 and 16 GiB gave 21.0, 20.5, 19.9 and 19.2 ms per launch (fewer, larger
// reweighting launches fill the GPU better), so the cap grows with the memory
// a context may hold.
static size_t zw_cap(const Ctx &ctx) {
    const size_t lo = (size_t)1 << 30, hi = (size_t)8 << 30;
    return std::min(hi, std::max(lo, ctx.budget / 32));
}
static size_t zw_bytes_for(int H, int64_t n_zpad, size_t cap) {
    const int64_t per = 8 * std::max<int64_t>(n_zpad, 1);
    const int64_t t = std::max<int64_t>(1, std::min<int64_t>(H, (int64_t)(cap / (size_t)per)));
    return (size_t)(t * per);
}

int ws_ensure(Ctx &ctx, Workspace &ws, int H, const Catalog &cat) {
    const DevCatalog &c = cat.d;
    int nch = selection_chunks(c);
    const size_t zwb = zw_bytes_for(H, c.n_zpad, zw_cap(ctx));
    if (H <= ws.Hcap && c.n_events <= ws.nev_cap && c.n_z <= ws.nz_cap && nch <= ws.nchunk_cap &&
        zwb <= ws.zw_bytes)
        return CHIMERA_OK;
    // grow (with some headroom) and re-allocate everything
    int Hn = std::max(H, ws.Hcap);
    int64_t nev = std::max<int64_t>(c.n_events, ws.nev_cap);
    int nz = std::max(c.n_z, ws.nz_cap);
    int nc = std::max(nch, ws.nchunk_cap);
    const size_t zw_bytes = std::max(zwb, ws.zw_bytes);
    if (ws.st) cudaStreamSynchronize(ws.st);
    ws_release(ctx, ws);
    struct Item { void **p; size_t b; };
    std::vector<Item> items = {
        {(void **)&ws.param, ws.param_bytes(Hn)},
        {(void **)&ws.hp, sizeof(HP) * Hn},
        {(void **)&ws.inv64, sizeof(double2) * (size_t)Hn * (NU + 1)},
        {(void **)&ws.inv32, sizeof(float4) * (size_t)Hn * NU},
        {(void **)&ws.linv32, sizeof(float4) * (size_t)Hn * NU},
        {(void **)&ws.F64, sizeof(double) * (size_t)Hn * nz},
        {(void **)&ws.F32, sizeof(float) * (size_t)Hn * nz},
        {(void **)&ws.lnI, sizeof(double) * (size_t)Hn * nev},
        {(void **)&ws.bw, sizeof(double) * (size_t)Hn * nev},
        {(void **)&ws.selp, sizeof(double) * 2 * (size_t)Hn * nc},
        {(void **)&ws.lnL, sizeof(double) * Hn},
        {(void **)&ws.neff, sizeof(double) * Hn},
        {(void **)&ws.xi, sizeof(double) * Hn},
        {(void **)&ws.grad, sizeof(double) * 12 * (size_t)Hn},
        {(void **)&ws.pairs, sizeof(unsigned long long) * (size_t)Hn},
        {(void **)&ws.dk, sizeof(float) * 2 * (size_t)Hn * NT_FWD},
        {(void **)&ws.fmax_bits, sizeof(unsigned long long) * (size_t)Hn},
        {(void **)&ws.zw, zw_bytes},
    };
    // ws_release freed the old buffers: forget their addresses, so that a
    // failure below frees only what this attempt allocated
    for (auto &it : items) *it.p = nullptr;
    for (auto &it : items) {
        int rc = dev_alloc(ctx, it.p, it.b);
        if (rc) {
            for (auto &jt : items)
                if (*jt.p) { cudaFree(*jt.p); *jt.p = nullptr; }
            ctx.used -= ws.bytes;
            ws.bytes = 0;
            ws.allocs.clear();
            return rc;
        }
        size_t rb = (it.b + 255) & ~(size_t)255;
        ws.bytes += rb;
        ws.allocs.push_back(*it.p);
    }
    ws.hstage_bytes = ws.param_bytes(Hn);
    if (cudaMallocHost(&ws.hstage, ws.hstage_bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMallocHost failed for the staging buffer");
        return CHIMERA_ERR_CUDA;
    }
    ws.Hcap = Hn;
    ws.nev_cap = nev;
    ws.nz_cap = nz;
    ws.nchunk_cap = nc;
    ws.zw_bytes = zw_bytes;
    return CHIMERA_OK;
}

// ------------------------------------------------------------ caches ----
uint64_t bits_of(double x) {
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
}

// The distance tables (dOm: their Om derivatives) of n distinct Om values:
// cached ones are waited for, new ones built FWD_MB at a time (one launch
// pair per batch).
int fwd_tables(Ctx &ctx, const double *Om, int n, cudaStream_t st, const double **out, bool dOm) {
    FwdBatch b{};
    std::vector<FwdEntry *> fresh;
    auto flush = [&]() -> int {
        if (b.n == 0) return CHIMERA_OK;
        launch_fwd_tables(b, dOm, st);
        CK(cudaGetLastError());
        for (FwdEntry *e : fresh) CK(cudaEventRecord(e->ready, st));
        b.n = 0;
        fresh.clear();
        return CHIMERA_OK;
    };
    for (int i = 0; i < n; i++) {
        const uint64_t key = bits_of(Om[i]);
        auto &cache = dOm ? ctx.fwdO : ctx.fwd;
        auto it = cache.find(key);
        if (it == cache.end()) {
            FwdEntry e;
            int rc = cache_alloc(ctx, (void **)&e.table, sizeof(double) * NT_FWD, st);
            if (rc == CHIMERA_OK && cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming) != cudaSuccess) {
                cache_free(ctx, e.table, sizeof(double) * NT_FWD);
                rc = cuda_check(cudaGetLastError(), "cudaEventCreate");
            }
            if (rc != CHIMERA_OK) {
                flush();  // the entries already made get their tables
                return rc;
            }
            e.last_use = ctx.tick;
            it = cache.emplace(key, e).first;
            b.Om[b.n] = Om[i];
            b.out[b.n++] = it->second.table;
            fresh.push_back(&it->second);
            if (b.n == FWD_MB) RC(flush());
        } else {
            it->second.last_use = ctx.tick;
            CK(cudaStreamWaitEvent(st, it->second.ready, 0));
        }
        out[i] = it->second.table;
    }
    return flush();
}

int fwd_table(Ctx &ctx, double Om, cudaStream_t st, const double **out) {
    return fwd_tables(ctx, &Om, 1, st, out, false);
}

void free_prof_entry(Ctx &ctx, ProfEntry &e) {
    cache_free(ctx, e.G, e.bytes);
    if (e.Gh) cache_free(ctx, e.Gh, e.hbytes);
    if (e.ready) cudaEventDestroy(e.ready);
    e.G = e.Gh = nullptr;
    e.ready = nullptr;
}

// Frees cache entries that the running call has not touched, least recently
// used first (the galaxy profiles of every resident catalog, then the
// distance tables), until `need` more bytes fit the budget.  Every call of
// the context runs under its mutex, and the device is idled before the first
// entry is freed, so no kernel still reads a freed entry.  Returns whether
// the bytes fit.
bool make_room(Ctx &ctx, size_t need) {
    bool synced = false, freed = false;
    while (ctx.used.load() + need > ctx.budget) {
        Catalog *vc = nullptr;
        std::map<std::pair<uint64_t, int>, ProfEntry>::iterator victim;
        for (auto &kv : ctx.cats) {
            Catalog &cat = *kv.second;
            for (auto it = cat.prof.begin(); it != cat.prof.end(); ++it)
                if (it->second.last_use < ctx.tick && (!vc || it->second.last_use < victim->second.last_use)) {
                    vc = &cat;
                    victim = it;
                }
        }
        std::unordered_map<uint64_t, FwdEntry> *fc = nullptr;
        std::unordered_map<uint64_t, FwdEntry>::iterator fvictim;
        if (!vc)
            for (auto *cache : {&ctx.fwd, &ctx.fwdO})
                for (auto it = cache->begin(); it != cache->end(); ++it)
                    if (it->second.last_use < ctx.tick && (!fc || it->second.last_use < fvictim->second.last_use)) {
                        fc = cache;
                        fvictim = it;
                    }
        if (!vc && !fc) {
            // last, the profile scratch, when this call has not used it
            if (ctx.ps.base && ctx.ps.last_use < ctx.tick) {
                cudaDeviceSynchronize();
                synced = true;
                prof_scratch_free(ctx);
                continue;
            }
            break;
        }
        if (!synced) {
            cudaDeviceSynchronize();
            synced = true;
        }
        if (vc) {
            free_prof_entry(ctx, victim->second);
            vc->prof.erase(victim);
        } else {
            cache_free(ctx, fvictim->second.table, sizeof(double) * NT_FWD);
            if (fvictim->second.ready) cudaEventDestroy(fvictim->second.ready);
            fc->erase(fvictim);
        }
        freed = true;
    }
    if (freed) trim_cache_pool(ctx);
    return ctx.used.load() + need <= ctx.budget;
}

void evict_profiles(Ctx &ctx, Catalog &, size_t need) { make_room(ctx, need); }

static size_t ps_al(size_t b) { return (std::max<size_t>(b, 16) + 255) & ~(size_t)255; }

int prof_scratch_acquire(Ctx &ctx, const DevCatalog &c, cudaStream_t st, ProfView *v, const TcHost *tc) {
    const size_t nz = (size_t)c.n_z, ng = (size_t)std::max<int64_t>(c.n_gal, 1);
    const size_t s_one = ps_al(12 * nz) + ps_al(8 * ng) + ps_al(4 * ng);
    const size_t s_multi = ps_al(2 * sizeof(float) * PROF_MB * (nz + 1)) + ps_al(2 * sizeof(float) * PROF_MB * ng);
    const size_t s_adj = 2 * ps_al(12 * nz) + 2 * ps_al(8 * ng);
    const size_t s_tc = tc ? tc_scratch_bytes(c, *tc) : 0;
    const size_t need = std::max(std::max(s_one, s_tc), std::max(s_multi, s_adj));
    ProfScratch &ps = ctx.ps;
    ps.last_use = ctx.tick;
    if (!ps.done) CK(cudaEventCreateWithFlags(&ps.done, cudaEventDisableTiming));
    if (need > ps.bytes) {
        if (ps.recorded) CK(cudaEventSynchronize(ps.done));  // the last use has ended
        if (ps.base) dev_free(ctx, ps.base, ps.bytes);
        ps.base = nullptr;
        ps.bytes = 0;
        RC(dev_alloc(ctx, (void **)&ps.base, need));
        ps.bytes = need;
        ps.last_use = ctx.tick;
    }
    if (ps.recorded) CK(cudaStreamWaitEvent(st, ps.done, 0));
    char *b = ps.base;
    v->dv = reinterpret_cast<double *>(b);
    v->invZ64 = reinterpret_cast<double *>(b + ps_al(12 * nz));
    v->invZ32 = reinterpret_cast<float *>(b + ps_al(12 * nz) + ps_al(8 * ng));
    v->dvm = reinterpret_cast<float *>(b);
    v->invZm = reinterpret_cast<float *>(b + ps_al(2 * sizeof(float) * PROF_MB * (nz + 1)));
    v->adv = reinterpret_cast<double *>(b);
    v->advO = reinterpret_cast<double *>(b + ps_al(12 * nz));
    v->ainvZ = reinterpret_cast<double *>(b + 2 * ps_al(12 * nz));
    v->aZO = reinterpret_cast<double *>(b + 2 * ps_al(12 * nz) + ps_al(8 * ng));
    v->tc = b;
    return CHIMERA_OK;
}

int prof_scratch_release(Ctx &ctx, cudaStream_t st) {
    CK(cudaEventRecord(ctx.ps.done, st));
    ctx.ps.recorded = true;
    return CHIMERA_OK;
}

// Frees the profile scratch; the device must be idle.
void prof_scratch_free(Ctx &ctx) {
    ProfScratch &ps = ctx.ps;
    if (ps.base) dev_free(ctx, ps.base, ps.bytes);
    ps.base = nullptr;
    ps.bytes = 0;
    ps.recorded = false;
}

// A mixed profile whose entry exists but whose kernels are still to be
// launched (batched by flush_profiles).
struct PendingProf {
    double Om;
    const double *fwd;
    std::pair<uint64_t, int> key;
};

// Launch the pending mixed profiles: PROF_MB Om values per batched pass (one
// Om alone takes the one-Om kernels; both give the same values).
static int flush_profiles(Ctx &ctx, Catalog &cat, Workspace &ws, std::vector<PendingProf> &pend) {
    const DevCatalog &c = cat.d;
    if (pend.empty()) return CHIMERA_OK;
    ProfView v;
    RC(prof_scratch_acquire(ctx, c, ws.st, &v, c.tc_ok ? &cat.tc : nullptr));
    if (c.tc_ok) {
        // photometric catalog: every mixed profile on the tensor cores, up to
        // TC_COLS Om values per batch (a profile is a function of its Om
        // alone, whatever the batch)
        for (size_t b = 0; b < pend.size(); b += TC_COLS) {
            const int n = (int)std::min<size_t>(TC_COLS, pend.size() - b);
            TcCols m{};
            m.n = n;
            for (int j = 0; j < n; j++) {
                m.fwd[j] = pend[b + j].fwd;
                m.Om[j] = pend[b + j].Om;
            }
            // the launcher takes the outputs through the columns' entries
            std::vector<float *> outs(n);
            for (int j = 0; j < n; j++) outs[j] = (float *)cat.prof.at(pend[b + j].key).G;
            RC(launch_galaxy_profile_tc(c, cat.tc, m, outs.data(), v.tc, ws.st));
            for (int j = 0; j < n; j++) {
                ProfEntry &e = cat.prof.at(pend[b + j].key);
                if (e.Gh) launch_profile_sum(c, nullptr, (float *)e.G, nullptr, (float *)e.Gh, ws.st);
                CK(cudaGetLastError());
                CK(cudaEventRecord(e.ready, ws.st));
            }
        }
        pend.clear();
        return prof_scratch_release(ctx, ws.st);
    }
    for (size_t b = 0; b < pend.size(); b += PROF_MB) {
        const int n = (int)std::min<size_t>(PROF_MB, pend.size() - b);
        if (n == 1) {
            ProfEntry &e = cat.prof.at(pend[b].key);
            launch_galaxy_profile(c, pend[b].fwd, pend[b].Om, v.dv, v.invZ64, v.invZ32, nullptr, (float *)e.G,
                                  ws.st);
        } else {
            MultiOm m{};
            m.n = n;
            for (int j = 0; j < PROF_MB; j++) {
                const PendingProf &q = pend[b + (j < n ? j : 0)];
                m.fwd[j] = q.fwd;
                m.fwdO[j] = nullptr;
                m.Om[j] = q.Om;
                m.out[j] = j < n ? (float *)cat.prof.at(q.key).G : nullptr;
            }
            launch_galaxy_profile_multi(c, m, false, v.dvm, v.invZm, ws.st);
        }
        for (int j = 0; j < n; j++) {
            ProfEntry &e = cat.prof.at(pend[b + j].key);
            if (e.Gh) launch_profile_sum(c, nullptr, (float *)e.G, nullptr, (float *)e.Gh, ws.st);
            CK(cudaGetLastError());
            CK(cudaEventRecord(e.ready, ws.st));
        }
    }
    pend.clear();
    return prof_scratch_release(ctx, ws.st);
}

// Drop pending entries (after an error: their kernels never ran).
static void drop_pending(Ctx &ctx, Catalog &cat, Workspace &ws, std::vector<PendingProf> &pend) {
    cudaStreamSynchronize(ws.st);  // nothing may still write the entries freed below
    for (auto &q : pend) {
        auto it = cat.prof.find(q.key);
        if (it == cat.prof.end()) continue;
        free_prof_entry(ctx, it->second);
        cat.prof.erase(it);
    }
    pend.clear();
}

// The profile of (Om, kind), from the cache or computed; with `defer`, a new
// mixed profile is only allocated and queued for flush_profiles.
static int profile(Ctx &ctx, Catalog &cat, Workspace &ws, double Om, int kind, const double *fwd,
                   const void **out, std::vector<PendingProf> *defer) {
    auto key = std::make_pair(bits_of(Om), kind);
    auto it = cat.prof.find(key);
    const DevCatalog &c = cat.d;
    if (it == cat.prof.end() && defer && kind == 1) {
        ProfEntry e;
        e.bytes = sizeof(float) * (size_t)c.n_pix * c.n_z;
        const size_t hb = c.kde_mode == CHIMERA_KDE_SINGLE_1D ? sizeof(float) * (size_t)c.n_events * c.n_z : 0;
        evict_profiles(ctx, cat, e.bytes + hb);
        RC(cache_alloc(ctx, &e.G, e.bytes, ws.st));
        if (hb) {
            int rc = cache_alloc(ctx, &e.Gh, hb, ws.st);
            if (rc) { cache_free(ctx, e.G, e.bytes); return rc; }
            e.hbytes = hb;
        }
        if (cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming) != cudaSuccess) {
            free_prof_entry(ctx, e);
            return cuda_check(cudaGetLastError(), "cudaEventCreate");
        }
        it = cat.prof.emplace(key, e).first;
        defer->push_back({Om, fwd, key});
    } else if (it == cat.prof.end()) {
        ProfEntry e;
        size_t esz = kind == 0 ? sizeof(double) : sizeof(float);
        e.bytes = esz * (size_t)c.n_pix * c.n_z;
        size_t hb = c.kde_mode == CHIMERA_KDE_SINGLE_1D ? esz * (size_t)c.n_events * c.n_z : 0;
        evict_profiles(ctx, cat, e.bytes + hb);
        RC(cache_alloc(ctx, &e.G, e.bytes, ws.st));
        if (hb) {
            int rc = cache_alloc(ctx, &e.Gh, hb, ws.st);
            if (rc) { cache_free(ctx, e.G, e.bytes); return rc; }
            e.hbytes = hb;
        }
        CK(cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming));
        ProfView v;
        if (int rc = prof_scratch_acquire(ctx, c, ws.st, &v)) {
            free_prof_entry(ctx, e);
            return rc;
        }
        if (kind == 0)
            launch_galaxy_profile(c, fwd, Om, v.dv, v.invZ64, v.invZ32, (double *)e.G, nullptr, ws.st);
        else
            launch_galaxy_profile(c, fwd, Om, v.dv, v.invZ64, v.invZ32, nullptr, (float *)e.G, ws.st);
        if (hb) {
            if (kind == 0) launch_profile_sum(c, (double *)e.G, nullptr, (double *)e.Gh, nullptr, ws.st);
            else launch_profile_sum(c, nullptr, (float *)e.G, nullptr, (float *)e.Gh, ws.st);
        }
        CK(cudaGetLastError());
        CK(cudaEventRecord(e.ready, ws.st));
        RC(prof_scratch_release(ctx, ws.st));
        it = cat.prof.emplace(key, e).first;
    } else {
        CK(cudaStreamWaitEvent(ws.st, it->second.ready, 0));
    }
    it->second.last_use = ctx.tick;
    *out = c.kde_mode == CHIMERA_KDE_SINGLE_1D ? it->second.Gh : it->second.G;
    return CHIMERA_OK;
}

// The mixed event kernel's block geometry, timed once per catalog: on the
// catalog's first mixed call, once the selection term on the side stream has
// finished, both instantiations (10 warps, three blocks per SM; 16 warps,
// two) run on the call's first tile, twice each in alternation, and the
// faster is kept for the catalog.  They write the same
// values (the event kernel reads the reweighting kernel's bandwidth and
// writes ln I and the same bandwidth back), so the call's results do not
// depend on the choice.  The load-time choice by occupancy stands when the
// 16-warp form does not fit, and while windowed pairs are being counted.
static int tune_event_geometry(Catalog &cat, const CallPtrs &p, int h0, int nh, Workspace &ws) {
    cat.ev_tuned = true;
    int dev = 0, maxsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if ((int)event_mixed_smem(cat.d, 0) > maxsm) return CHIMERA_OK;
    cudaEvent_t e[5] = {};
    for (auto &x : e)
        if (cudaEventCreate(&x) != cudaSuccess) {
            cudaGetLastError();
            for (auto &y : e)
                if (y) cudaEventDestroy(y);
            return CHIMERA_OK;  // timing unavailable: keep the load-time choice
        }
    DevCatalog cg = cat.d;
    // the selection term on the side stream would run beside the timed
    // launches and load them unevenly: wait for it first
    cudaError_t err = ws.ev_join ? cudaStreamWaitEvent(ws.st, ws.ev_join, 0) : cudaSuccess;
    if (err == cudaSuccess) err = cudaEventRecord(e[0], ws.st);
    for (int k = 0; k < 4 && err == cudaSuccess; k++) {
        cg.ev_geom = k & 1;
        launch_event_mixed(cg, p, h0, nh, ws.st);
        err = cudaEventRecord(e[k + 1], ws.st);
    }
    if (err == cudaSuccess) err = cudaEventSynchronize(e[4]);
    float t[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < 4 && err == cudaSuccess; k++) err = cudaEventElapsedTime(&t[k], e[k], e[k + 1]);
    for (auto &x : e) cudaEventDestroy(x);
    if (err != cudaSuccess) return cuda_check(err, "event kernel geometry timing");
    const float t16 = std::min(t[0], t[2]), t10 = std::min(t[1], t[3]);
    cat.d.ev_geom = t10 <= t16 ? 1 : 0;
    cat.info.event_kernel_warps = cat.d.ev_geom == 1 ? EV_WARPS_3 : EV_WARPS_2;
    return CHIMERA_OK;
}

// ----------------------------------------------------------- forward ----
int forward(Ctx &ctx, Catalog &cat, Workspace &ws, int H, const double *theta, int precision,
            double *out_lnL, double *out_neff, int32_t *out_status) {
    const bool epan = (precision & CHIMERA_KERNEL_EPANECHNIKOV) != 0;
    const bool jac_ps = (precision & CHIMERA_JACOBIAN_PER_SAMPLE) != 0;
    const bool for_grad = (precision & PREC_WITH_GRAD) != 0;
    precision &= ~(CHIMERA_KERNEL_EPANECHNIKOV | CHIMERA_JACOBIAN_PER_SAMPLE | PREC_WITH_GRAD);  // the base precision
    if (cat.d.kde_mode == CHIMERA_KDE_3D && (precision != CHIMERA_FP64 || epan)) {
        set_error("CHIMERA_KDE_3D catalogs take CHIMERA_FP64 with the Gaussian kernel");
        return CHIMERA_ERR_INVALID_ARG;
    }
    ctx.tick++;  // before the workspace grows: the previous call's cache entries may go
    RC(ws_ensure(ctx, ws, H, cat));
    const DevCatalog &c = cat.d;
    // stage: theta (admissible copy) | status | fwd ptrs | prof ptrs
    char *q = ws.hstage;
    double *th = reinterpret_cast<double *>(q);
    int32_t *st = reinterpret_cast<int32_t *>(q + sizeof(double) * 12 * H);
    const double **fw = reinterpret_cast<const double **>(q + sizeof(double) * 12 * H + 8 * H);
    const void **pr = reinterpret_cast<const void **>(q + sizeof(double) * 12 * H + 8 * H + 8 * H);
    const int kind = precision == CHIMERA_FP64 ? 0 : 1;
    if (ws.trace) {
        for (auto &e : ws.tev)
            if (!e) CK(cudaEventCreate(&e));
        ws.traced_adjoint = false;
        ws.traced_tiles = 0;
        CK(cudaEventRecord(ws.tev[0], ws.st));
    }
    memset(st, 0, 8 * (size_t)H);
    for (int h = 0; h < H; h++) {
        const double *t = theta + 12 * h;
        bool ok = theta_admissible(t);
        memcpy(th + 12 * h, ok ? t : kSafeTheta, sizeof(double) * 12);
        st[h] = ok ? 0 : CHIMERA_PT_OUT_OF_SUPPORT;
    }
    // distinct Om values in order of first appearance: their distance tables
    // (batched), then their profiles (new mixed ones batched)
    std::map<uint64_t, int> slot;
    std::vector<double> oms;
    for (int h = 0; h < H; h++) {
        const double Om = th[12 * h + 1];
        if (slot.emplace(bits_of(Om), (int)oms.size()).second) oms.push_back(Om);
    }
    std::vector<const double *> fws(oms.size());
    std::vector<const void *> prs(oms.size());
    RC(fwd_tables(ctx, oms.data(), (int)oms.size(), ws.st, fws.data(), false));
    std::vector<PendingProf> pend;
    for (size_t i = 0; i < oms.size(); i++) {
        int rc = profile(ctx, cat, ws, oms[i], kind, fws[i], &prs[i], &pend);
        if (rc != CHIMERA_OK) {
            drop_pending(ctx, cat, ws, pend);
            return rc;
        }
    }
    for (int h = 0; h < H; h++) {
        const int i = slot.at(bits_of(th[12 * h + 1]));
        fw[h] = fws[i];
        pr[h] = prs[i];
    }
    if (int rc = flush_profiles(ctx, cat, ws, pend)) {
        drop_pending(ctx, cat, ws, pend);
        return rc;
    }
    if (ws.trace) CK(cudaEventRecord(ws.tev[1], ws.st));
    CK(cudaMemcpyAsync(ws.param, ws.hstage, ws.param_bytes(H), cudaMemcpyHostToDevice, ws.st));
    CallPtrs p = ws.ptrs(H, c);
    p.kshape = epan ? 1 : 0;
    p.jac_ps = jac_ps ? 1 : 0;
    if (p.pairs) CK(cudaMemsetAsync(p.pairs, 0, sizeof(unsigned long long) * H, ws.st));
    // the side stream, of the lowest priority: the per-point FP64 scalars
    // beside the inverse nodes, then the selection term beside the event
    // kernels, whose blocks are dispatched first (the library streams have
    // the highest priority)
    if (!ws.st2) {
        int lo = 0, hi = 0;
        CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CK(cudaStreamCreateWithPriority(&ws.st2, cudaStreamNonBlocking, lo));
        CK(cudaEventCreateWithFlags(&ws.ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ws.ev_join, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ws.ev_tab_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ws.ev_tab_join, cudaEventDisableTiming));
    }
    CK(launch_hyper_tables(c, p, H, precision == CHIMERA_FP64, ws.dk, ws.fmax_bits, ws.st, ws.st2,
                           ws.ev_tab_fork, ws.ev_tab_join));
    if (ws.trace) CK(cudaEventRecord(ws.tev[2], ws.st));
    // the selection term needs only the per-point tables
    CK(cudaEventRecord(ws.ev_fork, ws.st));
    CK(cudaStreamWaitEvent(ws.st2, ws.ev_fork, 0));
    if (ws.trace) CK(cudaEventRecord(ws.tev[8], ws.st2));
    launch_selection(c, p, H, precision == CHIMERA_FP64, ws.st2);
    if (ws.trace) CK(cudaEventRecord(ws.tev[9], ws.st2));
    CK(cudaEventRecord(ws.ev_join, ws.st2));
    if (precision == CHIMERA_FP64) {
        if (c.kde_mode == CHIMERA_KDE_3D) launch_event_3d(c, p, H, ws.st);
        else launch_event_fp64(c, p, H, ws.st);
    } else {
        // reweighting and event integrals by tiles of hyperpoints
        const int64_t fit = (int64_t)(ws.zw_bytes / (8 * (size_t)std::max<int64_t>(c.n_zpad, 1)));
        const int tile = (int)std::max<int64_t>(1, std::min<int64_t>(H, fit));
        const int ntiles = (H + tile - 1) / tile;
        if (ws.trace) {
            while ((int)ws.tile_ev.size() < 2 * ntiles) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                ws.tile_ev.push_back(e);
            }
            ws.traced_tiles = ntiles;
        }
        for (int t = 0; t < ntiles; t++) {
            const int h0 = t * tile, nh = std::min(tile, H - h0);
            launch_reweight(c, p, h0, nh, ws.st);
            if (ws.trace) CK(cudaEventRecord(ws.tile_ev[2 * t], ws.st));
            if (precision == CHIMERA_MIXED_BINNED || epan) {
                launch_event_binned(c, p, h0, nh, precision == CHIMERA_MIXED_BINNED, ws.st);
            } else {
                if (!cat.ev_tuned && !p.pairs) RC(tune_event_geometry(cat, p, h0, nh, ws));
                launch_event_mixed(c, p, h0, nh, ws.st);
            }
            if (ws.trace) CK(cudaEventRecord(ws.tile_ev[2 * t + 1], ws.st));
        }
    }
    if (ws.trace) CK(cudaEventRecord(ws.tev[3], ws.st));
    CK(cudaStreamWaitEvent(ws.st, ws.ev_join, 0));
    if (ws.trace) CK(cudaEventRecord(ws.tev[4], ws.st));
    p.out_lnL = out_lnL;
    p.out_neff = out_neff;
    p.out_status = out_status;
    launch_combine(c, p, H, ws.st);
    if (ws.trace) CK(cudaEventRecord(ws.tev[5], ws.st));
    CK(cudaGetLastError());
    return CHIMERA_OK;
}

std::shared_ptr<Catalog> find_catalog(Ctx &ctx, int32_t id) {
    auto it = ctx.cats.find(id);
    if (it == ctx.cats.end()) return nullptr;
    return it->second;
}

// ----------------------------------------------------- catalog load ----
static uint16_t f32_to_half_bits(float x) { return __half_as_ushort(__float2half_rn(x)); }
static uint16_t f32_to_bf16_bits(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;  // NaN
    uint32_t r = u + 0x7fffu + ((u >> 16) & 1u);         // round to nearest even
    return (uint16_t)(r >> 16);
}
static float half_bits_to_f32(uint16_t b) { return __half2float(__ushort_as_half(b)); }
static float bf16_bits_to_f32(uint16_t b) {
    uint32_t u = ((uint32_t)b) << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

static bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

static int load_catalog(Ctx &ctx, const chimera_catalog_desc *d, int32_t *out_id) {
    if (!d || !out_id) { set_error("null descriptor or id pointer"); return CHIMERA_ERR_INVALID_ARG; }
    const int ne = d->n_events;
    auto bad = [](const std::string &m) { set_error(m); return CHIMERA_ERR_INVALID_ARG; };
    if (ne <= 0) return bad("n_events must be positive");
    if (!d->sample_off || !d->dL_Mpc || !d->m1_det || !d->m2_det || !d->pix_of_sample ||
        !d->pix_off || !d->sky_S || !d->gal_off)
        return bad("null array in catalog descriptor");
    if (d->n_z < 2) return bad("n_z must be >= 2");
    if (d->n_z > CHIMERA_MAX_NZ) { set_error("n_z above CHIMERA_MAX_NZ"); return CHIMERA_ERR_UNSUPPORTED; }
    if (!finite_pos(d->z_max)) return bad("z_max must be positive");
    if (!finite_pos(d->n_gal_total)) return bad("n_gal_total must be positive");
    if (d->n_det < 0 || d->n_inj_total < 1 || d->n_inj_total < d->n_det) return bad("bad injection counts");
    if (d->n_det > 0 && (!d->inj_dL || !d->inj_m1d || !d->inj_m2d || !d->inj_log_pi))
        return bad("null injection array");
    if (!(d->lambda_g >= 0.0 && d->lambda_g <= 1.0) || !std::isfinite(d->beta))
        return bad("lambda_g must lie in [0, 1] and beta be finite");
    if (d->kde_mode != CHIMERA_KDE_SINGLE_1D && d->kde_mode != CHIMERA_KDE_MANY_1D && d->kde_mode != CHIMERA_KDE_3D)
        return bad("bad kde_mode");
    if (d->kde_mode == CHIMERA_KDE_3D && (!d->sky_xy || !d->pix_xy))
        return bad("a CHIMERA_KDE_3D catalog needs sky_xy and pix_xy");
    if (d->gal_storage < 0 || d->gal_storage > 2) return bad("bad gal_storage");
    if (d->completeness) {
        if (!d->pix_area) return bad("an incomplete catalog needs pix_area");
        if (!(d->f_R >= 0.0 && d->f_R <= 1.0)) return bad("f_R must lie in [0, 1]");
    }
    if (d->sample_off[0] != 0 || d->pix_off[0] != 0) return bad("CSR offsets must start at 0");
    int max_ns = 0, max_np = 0;
    for (int i = 0; i < ne; i++) {
        int64_t a = d->sample_off[i + 1] - d->sample_off[i];
        int64_t b = d->pix_off[i + 1] - d->pix_off[i];
        if (a < 1 || b < 1) return bad("every event needs >= 1 sample and >= 1 pixel");
        if (a > CHIMERA_MAX_SAMPLES_PER_EVENT || b > CHIMERA_MAX_PIXELS_PER_EVENT) {
            set_error("event " + std::to_string(i) + " exceeds the per-event sample or pixel limit");
            return CHIMERA_ERR_UNSUPPORTED;
        }
        max_ns = std::max<int>(max_ns, (int)a);
        max_np = std::max<int>(max_np, (int)b);
    }
    const int64_t ns = d->sample_off[ne], np = d->pix_off[ne];
    // sample offsets (padded to 4 per event) are 32-bit on the device
    if (ns + 3 * (int64_t)ne >= ((int64_t)1 << 31)) {
        set_error("more than 2^31 PE samples in one catalog");
        return CHIMERA_ERR_UNSUPPORTED;
    }
    if (d->gal_off[0] != 0) return bad("gal_off must start at 0");
    for (int64_t p = 0; p < np; p++) {
        if (d->gal_off[p + 1] < d->gal_off[p]) return bad("gal_off not monotone");
        if (!(std::isfinite(d->sky_S[p]) && d->sky_S[p] >= 0.0)) return bad("sky_S must be finite and >= 0");
    }
    const int64_t ng = d->gal_off[np];
    if (ng > 0 && (!d->gal_z || !d->gal_sigma)) return bad("null galaxy array");
    for (int64_t j = 0; j < ns; j++) {
        if (!finite_pos(d->dL_Mpc[j]) || !finite_pos(d->m1_det[j]) || !finite_pos(d->m2_det[j]))
            return bad("PE sample distances and masses must be finite and positive");
    }
    for (int i = 0; i < ne; i++)
        for (int64_t j = d->sample_off[i]; j < d->sample_off[i + 1]; j++)
            if (d->pix_of_sample[j] < 0 || d->pix_of_sample[j] >= d->pix_off[i + 1] - d->pix_off[i])
                return bad("pix_of_sample out of range");
    for (int64_t g = 0; g < ng; g++)
        if (!std::isfinite(d->gal_z[g]) || !finite_pos(d->gal_sigma[g])) return bad("bad galaxy z or sigma");
    for (int64_t j = 0; j < d->n_det; j++)
        if (!finite_pos(d->inj_dL[j]) || !finite_pos(d->inj_m1d[j]) || !finite_pos(d->inj_m2d[j]) ||
            !std::isfinite(d->inj_log_pi[j]))
            return bad("bad injection values");

    auto cat = std::make_shared<Catalog>();
    DevCatalog &c = cat->d;
    c.n_events = ne;
    c.n_z = d->n_z;
    c.kde_mode = d->kde_mode;
    c.gal_storage = d->gal_storage;
    c.n_samples = ns;
    c.n_pix = np;
    c.n_gal = ng;
    c.n_det = d->n_det;
    c.n_inj_total = d->n_inj_total;
    c.z_max = d->z_max;
    c.dz = d->z_max / (d->n_z - 1);
    c.z_max32 = (float)c.z_max;
    c.dz32 = (float)c.dz;
    c.dz_lo32 = (float)(c.dz - (double)c.dz32);
    c.n_gal_total = d->n_gal_total;
    c.lambda_g = d->lambda_g;
    c.ln_lambda = d->lambda_g > 0.0 ? std::log(d->lambda_g) : 0.0;
    c.ln1m_lambda = d->lambda_g < 1.0 ? std::log1p(-d->lambda_g) : 0.0;
    c.beta = d->beta;
    c.max_ns = max_ns;
    c.max_npix = max_np;
    double dmax = 0.0;
    for (int64_t j = 0; j < ns; j++) dmax = std::max(dmax, d->dL_Mpc[j]);
    for (int64_t j = 0; j < d->n_det; j++) dmax = std::max(dmax, d->inj_dL[j]);
    c.d_top = dmax * (1.0 + 1e-9);
    c.inv_d_top = 1.0 / c.d_top;

    // ---- samples: sort inside each event
    std::vector<int64_t> order(ns);
    std::iota(order.begin(), order.end(), 0);
    const bool many = d->kde_mode == CHIMERA_KDE_MANY_1D;
    for (int i = 0; i < ne; i++) {
        auto b = order.begin() + d->sample_off[i], e = order.begin() + d->sample_off[i + 1];
        std::stable_sort(b, e, [&](int64_t x, int64_t y) {
            if (many && d->pix_of_sample[x] != d->pix_of_sample[y])
                return d->pix_of_sample[x] < d->pix_of_sample[y];
            return d->dL_Mpc[x] < d->dL_Mpc[y];
        });
    }
    std::vector<float4> s32(ns);
    std::vector<float2> s32lo(ns);
    std::vector<double> sd(ns), sm1(ns), sm2(ns);
    auto tcoord = [&](double dl, int &k, float &f) {
        double t = std::sqrt(dl / c.d_top) * NU;
        k = std::min((int)t, NU - 1);
        double fr = t - k;
        f = (float)std::min(fr, 1.0);
    };
    for (int64_t j = 0; j < ns; j++) {
        int64_t o = order[j];
        int k;
        float f;
        tcoord(d->dL_Mpc[o], k, f);
        float kb;
        memcpy(&kb, &k, 4);
        const double l1 = std::log2(d->m1_det[o]), l2 = std::log2(d->m2_det[o]);
        s32[j] = make_float4(kb, f, (float)l1, (float)l2);
        s32lo[j] = make_float2((float)(l1 - (double)(float)l1), (float)(l2 - (double)(float)l2));
        sd[j] = d->dL_Mpc[o];
        sm1[j] = d->m1_det[o];
        sm2[j] = d->m2_det[o];
    }
    // ---- segments
    std::vector<int64_t> seg_soff;
    std::vector<double> seg_pf;
    std::vector<int32_t> ev_segoff(ne + 1);
    int max_seg = 1;
    if (many) {
        seg_soff.resize(np + 1);
        seg_pf.resize(np);
        for (int i = 0; i < ne; i++) {
            ev_segoff[i] = (int32_t)d->pix_off[i];
            int npi = (int)(d->pix_off[i + 1] - d->pix_off[i]);
            std::vector<int64_t> cnt(npi, 0);
            for (int64_t j = d->sample_off[i]; j < d->sample_off[i + 1]; j++) cnt[d->pix_of_sample[j]]++;
            int64_t run = d->sample_off[i];
            for (int k = 0; k < npi; k++) {
                int64_t p = d->pix_off[i] + k;
                seg_soff[p] = run;
                run += cnt[k];
                seg_pf[p] = cnt[k] > 0 ? d->sky_S[p] / (double)cnt[k] : 0.0;
            }
            max_seg = std::max(max_seg, npi);
        }
        seg_soff[np] = ns;
        ev_segoff[ne] = (int32_t)np;
    } else {
        seg_soff.assign(d->sample_off, d->sample_off + ne + 1);
        seg_pf.resize(ne);
        for (int i = 0; i < ne; i++) {
            ev_segoff[i] = i;
            seg_pf[i] = 1.0 / (double)(d->sample_off[i + 1] - d->sample_off[i]);
        }
        ev_segoff[ne] = ne;
    }
    c.n_seg = (int64_t)seg_pf.size();
    c.max_seg = max_seg;
    // ---- warp groups, the per-event redshift reference and inverse-table
    // range (mixed kernels)
    std::vector<int4> groups;
    std::vector<int32_t> ev_goff(ne + 1, 0);
    std::vector<float2> ev_ref(ne);
    std::vector<int2> ev_krange(ne);
    std::vector<int64_t> ev_zoff(ne + 1, 0);
    int max_groups = 1, max_krange = 1;
    for (int i = 0; i < ne; i++) {
        const int64_t a = d->sample_off[i], n = d->sample_off[i + 1] - a;
        {
            int kmin = NU, kmax = 0;
            for (int64_t j = a; j < a + n; j++) {
                int k;
                memcpy(&k, &s32[j].x, 4);
                kmin = std::min(kmin, k);
                kmax = std::max(kmax, k);
            }
            if (kmin > kmax) kmin = kmax = 0;
            ev_krange[i] = make_int2(kmin, kmax);
            max_krange = std::max(max_krange, kmax - kmin + 1);
        }
        double m = 0, m2 = 0;
        for (int64_t j = a; j < a + n; j++) {
            double l = std::log(sd[j]);
            m += l;
            m2 += l * l;
        }
        m /= n;
        const double sl = std::sqrt(std::max(m2 / n - m * m, 0.0)) * std::pow((double)n, -0.2);
        // reference: the median d_L of the event
        std::vector<double> dd(sd.begin() + a, sd.begin() + a + n);
        std::nth_element(dd.begin(), dd.begin() + n / 2, dd.end());
        {
            int k;
            float f;
            tcoord(dd[n / 2], k, f);
            float kb;
            memcpy(&kb, &k, 4);
            ev_ref[i] = make_float2(kb, f);
        }
        ev_goff[i] = (int32_t)groups.size();
        for (int32_t sgi = ev_segoff[i]; sgi < ev_segoff[i + 1]; sgi++) {
            const int64_t s0 = seg_soff[sgi], s1 = seg_soff[sgi + 1];
            const int sr = sgi - ev_segoff[i];
            // a chunk of up to 128 neighbours is halved (in multiples of 32)
            // while its spread in ln d_L exceeds 16 bandwidth-equivalents (wider groups are
            // still evaluated, by the per-lane path; the threshold was tuned on the
            // 300-event catalog)
            std::function<void(int64_t, int)> emit = [&](int64_t st, int cnt) {
                double spread = std::log(sd[st + cnt - 1]) - std::log(sd[st]);
                if (cnt > 32 && spread > 16.0 * sl) {
                    int first = 32 * ((cnt + 63) / 64);
                    emit(st, first);
                    emit(st + first, cnt - first);
                } else {
                    groups.push_back(make_int4((int)(st - a), cnt, sr, 0));
                }
            };
            for (int64_t g0 = s0; g0 < s1; g0 += GROUP_MAX)
                emit(g0, (int)std::min<int64_t>(GROUP_MAX, s1 - g0));
        }
        // costliest groups first (samples x (ln d_L spread + window)), so that
        // the warps of a block finish their last groups close together
        {
            auto cost_of = [&](const int4 &g) {
                const int64_t st = a + g.x;
                const double spread = std::log(sd[st + g.y - 1]) - std::log(sd[st]);
                return (double)((g.y + 31) / 32) * (spread + 12.0 * sl);
            };
            std::stable_sort(groups.begin() + ev_goff[i], groups.end(),
                             [&](const int4 &x, const int4 &y) { return cost_of(x) > cost_of(y); });
        }
        max_groups = std::max<int>(max_groups, (int)groups.size() - ev_goff[i]);
    }
    ev_goff[ne] = (int32_t)groups.size();
    for (int i = 0; i < ne; i++)
        ev_zoff[i + 1] = ev_zoff[i] + ((d->sample_off[i + 1] - d->sample_off[i] + 3) & ~(int64_t)3);
    c.n_zpad = std::max<int64_t>(ev_zoff[ne], 4);
    c.max_groups = max_groups;
    c.max_krange = max_krange;
    // ---- heavy-first event order: cost ~ N_s x spread of ln d_L
    std::vector<double> cost(ne);
    for (int i = 0; i < ne; i++) {
        double m = 0, m2 = 0;
        int64_t n = d->sample_off[i + 1] - d->sample_off[i];
        for (int64_t j = d->sample_off[i]; j < d->sample_off[i + 1]; j++) {
            double l = std::log(d->dL_Mpc[j]);
            m += l;
            m2 += l * l;
        }
        m /= n;
        cost[i] = n * std::sqrt(std::max(m2 / n - m * m, 0.0) + 1e-6);
    }
    std::vector<int32_t> ev_order(ne);
    std::iota(ev_order.begin(), ev_order.end(), 0);
    std::stable_sort(ev_order.begin(), ev_order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<int4> ev_info(2 * (size_t)ne);
    for (int pos = 0; pos < ne; pos++) {
        const int e = ev_order[pos];
        ev_info[2 * pos] = make_int4(e, (int)d->sample_off[e], (int)(d->sample_off[e + 1] - d->sample_off[e]),
                                     (int)ev_zoff[e]);
        ev_info[2 * pos + 1] = make_int4(ev_goff[e], ev_goff[e + 1] - ev_goff[e], ev_segoff[e],
                                         ev_segoff[e + 1] - ev_segoff[e]);
    }
    // ---- galaxies: sorted by z inside each pixel
    std::vector<int64_t> gorder(ng);
    std::iota(gorder.begin(), gorder.end(), 0);
    for (int64_t p = 0; p < np; p++)
        std::stable_sort(gorder.begin() + d->gal_off[p], gorder.begin() + d->gal_off[p + 1],
                         [&](int64_t x, int64_t y) { return d->gal_z[x] < d->gal_z[y]; });
    std::vector<double> gz(ng), gs(ng), sigmax(np, 0.0);
    std::vector<float> gz32, gs32, zref(np, 0.f), sigmax32(np, 0.f);
    std::vector<uint16_t> gzq, gsq;
    std::vector<float> zdec_all(ng), sdec_all(ng);  // the stored values as the kernels decode them
    if (d->gal_storage == CHIMERA_GAL_F32) { gz32.resize(ng); gs32.resize(ng); }
    else { gzq.resize(ng); gsq.resize(ng); }
    for (int64_t p = 0; p < np; p++) {
        int64_t a = d->gal_off[p], b = d->gal_off[p + 1];
        if (b > a) zref[p] = (float)d->gal_z[gorder[a]];
        for (int64_t g = a; g < b; g++) {
            int64_t o = gorder[g];
            gz[g] = d->gal_z[o];
            gs[g] = d->gal_sigma[o];
            sigmax[p] = std::max(sigmax[p], gs[g]);
            float sdec;
            if (d->gal_storage == CHIMERA_GAL_F32) {
                gz32[g] = (float)gz[g];
                gs32[g] = (float)gs[g];
                sdec = gs32[g];
                zdec_all[g] = gz32[g];
            } else {
                float off = (float)gz[g] - zref[p];
                bool h16 = d->gal_storage == CHIMERA_GAL_F16;
                gzq[g] = h16 ? f32_to_half_bits(off) : f32_to_bf16_bits(off);
                gsq[g] = h16 ? f32_to_half_bits((float)gs[g]) : f32_to_bf16_bits((float)gs[g]);
                sdec = h16 ? half_bits_to_f32(gsq[g]) : bf16_bits_to_f32(gsq[g]);
                float zdec = zref[p] + (h16 ? half_bits_to_f32(gzq[g]) : bf16_bits_to_f32(gzq[g]));
                if (!std::isfinite(zdec)) return bad("galaxy z offset not representable in 16-bit storage");
                zdec_all[g] = zdec;
            }
            sdec_all[g] = sdec;
            if (!(sdec > 0.f) || !std::isfinite(sdec)) return bad("galaxy sigma not representable in the storage type");
            sigmax32[p] = std::max(sigmax32[p], sdec);
        }
    }
    // ---- tensor-core profile plan (photometric catalogs)
    std::vector<int2> tc_blk;
    std::vector<float2> tc_coef;
    std::vector<int4> tc_items, tc_reds;
    std::vector<int32_t> tc_islot;
    {
        const char *f32 = getenv("CHIMERA_PROFILE_FP32");
        if (!(f32 && f32[0] == '1'))
            tc_plan(np, d->gal_off, zdec_all.data(), sdec_all.data(), sigmax32.data(), d->n_z, c.dz,
                    d->completeness != nullptr, d->kde_mode, c, cat->tc, tc_blk, tc_coef, tc_items, tc_islot, tc_reds);
    }
    // ---- injections, stored sorted by d_L: the selection kernel's chunks of
    // consecutive injections then read a few neighbouring inverse-table
    // intervals (the sum does not depend on the order beyond rounding)
    const int64_t nd = d->n_det;
    std::vector<int64_t> iord(nd);
    std::iota(iord.begin(), iord.end(), 0);
    std::stable_sort(iord.begin(), iord.end(), [&](int64_t x, int64_t y) { return d->inj_dL[x] < d->inj_dL[y]; });
    std::vector<double> idL(nd), im1(nd), im2(nd), ilp(nd);
    for (int64_t j = 0; j < nd; j++) {
        idL[j] = d->inj_dL[iord[j]];
        im1[j] = d->inj_m1d[iord[j]];
        im2[j] = d->inj_m2d[iord[j]];
        ilp[j] = d->inj_log_pi[iord[j]];
    }
    std::vector<float4> i32a(nd);
    std::vector<float2> i32lo(nd);
    std::vector<float2> i32b(nd);
    std::vector<float> iipi(nd);
    // 1 / pi_inj for the mixed selection, in FP64 and rounded once, scaled
    // by 2^-K with K the middle of the catalog's range of -log2 pi_inj so
    // that every value fits the float range; K ln 2 is carried in FP64
    {
        double lo = 0.0, hi = 0.0;
        for (int64_t j = 0; j < nd; j++) {
            const double l2 = -ilp[j] * 1.4426950408889634074;
            lo = j ? std::min(lo, l2) : l2;
            hi = j ? std::max(hi, l2) : l2;
        }
        const double K = std::floor(0.5 * (lo + hi));
        c.ln_ipi_shift = K * 0.69314718055994530942;
        for (int64_t j = 0; j < nd; j++) iipi[j] = (float)std::exp2(-ilp[j] * 1.4426950408889634074 - K);
    }
    for (int64_t j = 0; j < nd; j++) {
        int k;
        float f;
        tcoord(idL[j], k, f);
        float kb;
        memcpy(&kb, &k, 4);
        const double l1 = std::log2(im1[j]), l2 = std::log2(im2[j]);
        i32a[j] = make_float4(kb, f, (float)l1, (float)l2);
        i32lo[j] = make_float2((float)(l1 - (double)(float)l1), (float)(l2 - (double)(float)l2));
        i32b[j] = make_float2((float)idL[j], (float)ilp[j]);
    }
    std::vector<int64_t> ev_soff(d->sample_off, d->sample_off + ne + 1);
    std::vector<int64_t> ev_poff(d->pix_off, d->pix_off + ne + 1);
    std::vector<int64_t> goff(d->gal_off, d->gal_off + np + 1);
    std::vector<double> pixS(d->sky_S, d->sky_S + np);
    // the "3D" kernel's sky chart: samples in device order, pixels as given
    std::vector<double2> sxy, pxy;
    if (d->kde_mode == CHIMERA_KDE_3D) {
        sxy.resize(ns);
        pxy.resize(np);
        for (int64_t j = 0; j < ns; j++) {
            const int64_t o = order[j];
            sxy[j] = make_double2(d->sky_xy[2 * o], d->sky_xy[2 * o + 1]);
            if (!std::isfinite(sxy[j].x) || !std::isfinite(sxy[j].y)) return bad("sky_xy must be finite");
        }
        for (int64_t q = 0; q < np; q++) {
            pxy[q] = make_double2(d->pix_xy[2 * q], d->pix_xy[2 * q + 1]);
            if (!std::isfinite(pxy[q].x) || !std::isfinite(pxy[q].y)) return bad("pix_xy must be finite");
        }
    }
    // incomplete catalog: the missing-galaxy weight (1 - P_compl) pix_area / 4 pi
    std::vector<double> miss64;
    std::vector<float> miss32;
    c.incomplete = d->completeness != nullptr;
    c.f_R = d->completeness ? d->f_R : 1.0;
    if (c.incomplete) {
        const size_t nm = (size_t)np * (size_t)d->n_z;
        miss64.resize(nm);
        miss32.resize(nm);
        for (int64_t p = 0; p < np; p++) {
            const double ar = d->pix_area[p];
            if (!(ar > 0.0) || !std::isfinite(ar)) return bad("pix_area must be positive");
            for (int a = 0; a < d->n_z; a++) {
                const double P = d->completeness[p * d->n_z + a];
                if (!(P >= 0.0 && P <= 1.0)) return bad("completeness must lie in [0, 1]");
                miss64[p * d->n_z + a] = (1.0 - P) * ar / (4.0 * M_PI);
                miss32[p * d->n_z + a] = (float)miss64[p * d->n_z + a];
            }
        }
    }
    // galaxy-profile work lists
    std::vector<int32_t> gw_pix, dense_pix;
    std::vector<int64_t> gw_g0;
    for (int64_t p = 0; p < np; p++) {
        for (int64_t g = goff[p]; g < goff[p + 1]; g += GAL_CHUNK) {
            gw_pix.push_back((int32_t)p);
            gw_g0.push_back(g);
        }
        if (goff[p + 1] - goff[p] > GAL_DENSE) dense_pix.push_back((int32_t)p);
    }
    c.n_gw = (int64_t)gw_pix.size();
    c.n_dense = (int32_t)dense_pix.size();

    // ---- upload
    struct Up { void **dst; const void *src; size_t bytes; };
    std::vector<Up> ups = {
        {(void **)&c.ev_soff, ev_soff.data(), 8 * ev_soff.size()},
        {(void **)&c.ev_poff, ev_poff.data(), 8 * ev_poff.size()},
        {(void **)&c.ev_order, ev_order.data(), 4 * ev_order.size()},
        {(void **)&c.ev_info, ev_info.data(), 16 * ev_info.size()},
        {(void **)&c.seg_soff, seg_soff.data(), 8 * seg_soff.size()},
        {(void **)&c.seg_pf, seg_pf.data(), 8 * seg_pf.size()},
        {(void **)&c.ev_segoff, ev_segoff.data(), 4 * ev_segoff.size()},
        {(void **)&c.groups, groups.data(), 16 * groups.size()},
        {(void **)&c.ev_goff, ev_goff.data(), 4 * ev_goff.size()},
        {(void **)&c.ev_ref, ev_ref.data(), 8 * ev_ref.size()},
        {(void **)&c.ev_krange, ev_krange.data(), 8 * ev_krange.size()},
        {(void **)&c.ev_zoff, ev_zoff.data(), 8 * ev_zoff.size()},
        {(void **)&c.pix_S, pixS.data(), 8 * pixS.size()},
        {(void **)&c.gal_off, goff.data(), 8 * goff.size()},
        {(void **)&c.pix_sigmax, sigmax.data(), 8 * sigmax.size()},
        {(void **)&c.pix_sigmax32, sigmax32.data(), 4 * sigmax32.size()},
        {(void **)&c.pix_zref, zref.data(), 4 * zref.size()},
        {(void **)&c.gw_pix, gw_pix.data(), 4 * gw_pix.size()},
        {(void **)&c.miss64, miss64.data(), 8 * miss64.size()},
        {(void **)&c.miss32, miss32.data(), 4 * miss32.size()},
        {(void **)&c.sky_xy, sxy.data(), 16 * sxy.size()},
        {(void **)&c.pix_xy, pxy.data(), 16 * pxy.size()},
        {(void **)&c.gw_g0, gw_g0.data(), 8 * gw_g0.size()},
        {(void **)&c.dense_pix, dense_pix.data(), 4 * dense_pix.size()},
        {(void **)&c.gz64, gz.data(), 8 * gz.size()},
        {(void **)&c.gs64, gs.data(), 8 * gs.size()},
        {(void **)&c.s32, s32.data(), 16 * s32.size()},
        {(void **)&c.s32lo, s32lo.data(), 8 * s32lo.size()},
        {(void **)&c.sd64, sd.data(), 8 * sd.size()},
        {(void **)&c.sm1_64, sm1.data(), 8 * sm1.size()},
        {(void **)&c.sm2_64, sm2.data(), 8 * sm2.size()},
    };
    if (nd > 0) {
        ups.push_back({(void **)&c.i32a, i32a.data(), 16 * (size_t)nd});
        ups.push_back({(void **)&c.i32lo, i32lo.data(), 8 * (size_t)nd});
        ups.push_back({(void **)&c.i32b, i32b.data(), 8 * (size_t)nd});
        ups.push_back({(void **)&c.iipi32, iipi.data(), 4 * (size_t)nd});
        ups.push_back({(void **)&c.id64, idL.data(), 8 * (size_t)nd});
        ups.push_back({(void **)&c.im1_64, im1.data(), 8 * (size_t)nd});
        ups.push_back({(void **)&c.im2_64, im2.data(), 8 * (size_t)nd});
        ups.push_back({(void **)&c.ilp64, ilp.data(), 8 * (size_t)nd});
    }
    if (c.tc_ok) {
        ups.push_back({(void **)&c.tc_blk, tc_blk.data(), 8 * tc_blk.size()});
        ups.push_back({(void **)&c.tc_coef, tc_coef.data(), 8 * tc_coef.size()});
        ups.push_back({(void **)&c.tc_items, tc_items.data(), 16 * tc_items.size()});
        ups.push_back({(void **)&c.tc_islot, tc_islot.data(), 4 * tc_islot.size()});
        ups.push_back({(void **)&c.tc_reds, tc_reds.data(), 16 * tc_reds.size()});
    }
    if (d->gal_storage == CHIMERA_GAL_F32) {
        ups.push_back({(void **)&c.gz32, gz32.data(), 4 * gz32.size()});
        ups.push_back({(void **)&c.gs32, gs32.data(), 4 * gs32.size()});
    } else {
        ups.push_back({(void **)&c.gzq, gzq.data(), 2 * gzq.size()});
        ups.push_back({(void **)&c.gsq, gsq.data(), 2 * gsq.size()});
    }
    // the dense pixels' candidate ranges: allocated here, filled on the device
    if (c.n_dense > 0) {
        const size_t lb = sizeof(int2) * (size_t)c.n_dense * c.n_z;
        ups.push_back({(void **)&c.dense_lr64, nullptr, lb});
        ups.push_back({(void **)&c.dense_lr32, nullptr, lb});
    }
    size_t total = 0;
    for (auto &u : ups) total += (std::max<size_t>(u.bytes, 16) + 255) & ~(size_t)255;
    ctx.tick++;  // a load reads no cache entry: every one may make room
    if (ctx.used.load() + total > ctx.budget && !make_room(ctx, total)) {
        set_error("catalog footprint " + std::to_string(total) + " bytes exceeds the HBM budget");
        return CHIMERA_ERR_ADMISSION;
    }
    for (auto &u : ups) {
        int rc = dev_alloc(ctx, u.dst, u.bytes);
        if (rc) {
            for (void *a : cat->allocs) cudaFree(a);
            ctx.used -= cat->bytes;
            return rc;
        }
        cat->allocs.push_back(*u.dst);
        cat->bytes += (std::max<size_t>(u.bytes, 16) + 255) & ~(size_t)255;
        if (u.bytes && u.src) {
            cudaError_t e = cudaMemcpy(*u.dst, u.src, u.bytes, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                for (void *a : cat->allocs) cudaFree(a);
                ctx.used -= cat->bytes;
                return cuda_check(e, "cudaMemcpy catalog upload");
            }
        }
    }
    if (c.n_dense > 0) {
        launch_dense_ranges(c, 0);
        cudaError_t e = cudaStreamSynchronize(0);
        if (e == cudaSuccess) e = cudaGetLastError();
        // the work lists of the dense gather: points with galaxies in reach
        const size_t nl = (size_t)c.n_dense * c.n_z;
        std::vector<int2> lr(nl), items;
        for (int prec = 0; prec < 2 && e == cudaSuccess; prec++) {
            e = cudaMemcpy(lr.data(), prec ? c.dense_lr32 : c.dense_lr64, sizeof(int2) * nl, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) break;
            items.clear();
            for (int pass = 0; pass < 2; pass++)  // heavy ranges first, then light ones
                for (size_t i = 0; i < nl; i++) {
                    const int len = lr[i].y - lr[i].x;
                    if (len > 0 && (len > GAL_HEAVY) == (pass == 0))
                        items.push_back(make_int2((int)(i / c.n_z), (int)(i % c.n_z)));
                    if (pass == 0 && i + 1 == nl) (prec ? c.n_dheavy32 : c.n_dheavy64) = (int64_t)items.size();
                }
            int2 **dst = prec ? &c.dense_items32 : &c.dense_items64;
            (prec ? c.n_ditems32 : c.n_ditems64) = (int64_t)items.size();
            const size_t ib = sizeof(int2) * std::max<size_t>(items.size(), 1);
            int rc = dev_alloc(ctx, (void **)dst, ib);
            if (rc) {
                for (void *a : cat->allocs) cudaFree(a);
                ctx.used -= cat->bytes;
                return rc;
            }
            cat->allocs.push_back(*dst);
            cat->bytes += (ib + 255) & ~(size_t)255;
            if (!items.empty())
                e = cudaMemcpy(*dst, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            for (void *a : cat->allocs) cudaFree(a);
            ctx.used -= cat->bytes;
            return cuda_check(e, "dense galaxy ranges");
        }
    }
    // event kernels need their shared memory
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx.device);
    if ((int)event_mixed_smem(c, 1) > maxsm || (int)event_fp64_smem(c) > maxsm ||
        (int)event_binned_smem(c) > maxsm || (int)event_3d_smem(c) > maxsm) {
        for (void *a : cat->allocs) cudaFree(a);
        ctx.used -= cat->bytes;
        set_error("catalog needs more shared memory per block than the device offers");
        return CHIMERA_ERR_UNSUPPORTED;
    }
    c.ev_geom = event_mixed_pick(c);  // the mixed event kernel's block geometry
    cat->info.n_events = ne;
    cat->info.n_z = c.n_z;
    cat->info.n_samples = ns;
    cat->info.n_pixels = np;
    cat->info.n_galaxies = ng;
    cat->info.n_det = nd;
    cat->info.device_bytes = (int64_t)cat->bytes;
    cat->info.max_samples_per_event = max_ns;
    cat->info.max_pixels_per_event = max_np;
    cat->info.profile_path = c.tc_ok ? CHIMERA_PROFILE_TENSOR_CORES : CHIMERA_PROFILE_CUDA_CORES;
    cat->info.event_kernel_warps = c.ev_geom == 1 ? EV_WARPS_3 : EV_WARPS_2;
    int32_t id_ = ctx.next_id++;
    ctx.cats[id_] = cat;
    *out_id = id_;
    return CHIMERA_OK;
}

static void free_catalog(Ctx &ctx, Catalog &cat) {
    for (auto &kv : cat.prof) free_prof_entry(ctx, kv.second);
    cat.prof.clear();
    trim_cache_pool(ctx);
    for (void *a : cat.allocs) cudaFree(a);
    cat.allocs.clear();
    ctx.used -= cat.bytes;
    cat.bytes = 0;
}

}  // namespace chim

using namespace chim;

struct chimera_ctx {
    Ctx c;
};

// ================================================================ C ABI ====
extern "C" {

const char *chimera_strerror(int code) {
    switch (code) {
        case CHIMERA_OK: return "ok";
        case CHIMERA_ERR_INVALID_ARG: return "invalid argument";
        case CHIMERA_ERR_NOT_FOUND: return "not found";
        case CHIMERA_ERR_ADMISSION: return "HBM budget exceeded";
        case CHIMERA_ERR_CUDA: return "CUDA error";
        case CHIMERA_ERR_TIMEOUT: return "timeout (result pending)";
        case CHIMERA_ERR_CANCELLED: return "cancelled";
        case CHIMERA_ERR_UNSUPPORTED: return "unsupported size";
        default: return "unknown error";
    }
}

const char *chimera_last_error(void) { return g_last_error.c_str(); }

int chimera_create(chimera_ctx **out, int device, size_t budget) {
    if (!out) { set_error("out is NULL"); return CHIMERA_ERR_INVALID_ARG; }
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        set_error("no CUDA device available");
        return CHIMERA_ERR_CUDA;
    }
    if (device < 0 || device >= n) { set_error("device index out of range"); return CHIMERA_ERR_INVALID_ARG; }
    CK(cudaSetDevice(device));
    auto *h = new chimera_ctx();
    h->c.device = device;
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (cudaStreamCreateWithPriority(&h->c.stream, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
        delete h;
        set_error("cudaStreamCreate failed");
        return CHIMERA_ERR_CUDA;
    }
    h->c.ws.st = h->c.stream;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    h->c.budget = budget ? budget : (size_t)(0.9 * fr);
    *out = h;
    return CHIMERA_OK;
}

void chimera_destroy(chimera_ctx *h) {
    if (!h) return;
    Ctx &ctx = h->c;
    serve_shutdown(ctx);
    cudaSetDevice(ctx.device);
    cudaDeviceSynchronize();
    for (auto &kv : ctx.cats) free_catalog(ctx, *kv.second);
    ctx.cats.clear();
    for (auto &kv : ctx.fwd) {
        cache_free(ctx, kv.second.table, sizeof(double) * NT_FWD);
        cudaEventDestroy(kv.second.ready);
    }
    ctx.fwd.clear();
    for (auto &kv : ctx.fwdO) {
        cache_free(ctx, kv.second.table, sizeof(double) * NT_FWD);
        cudaEventDestroy(kv.second.ready);
    }
    ctx.fwdO.clear();
    ws_release(ctx, ctx.ws);
    prof_scratch_free(ctx);
    if (ctx.ps.done) cudaEventDestroy(ctx.ps.done);
    ws_destroy_streams(ctx.ws);
    for (auto &e : ctx.ws.tev)
        if (e) cudaEventDestroy(e);
    for (auto &e : ctx.ws.tile_ev) cudaEventDestroy(e);
    ctx.ws.tile_ev.clear();
    if (ctx.dev_done) cudaEventDestroy(ctx.dev_done);
    if (ctx.dev_theta_h) cudaFreeHost(ctx.dev_theta_h);
    cudaStreamSynchronize(ctx.stream);  // the pool's frees are ordered on it
    if (ctx.pool) cudaMemPoolDestroy(ctx.pool);
    cudaStreamDestroy(ctx.stream);
    delete h;
}

int chimera_load_catalog(chimera_ctx *h, const chimera_catalog_desc *desc, int32_t *id) {
    if (!h) { set_error("ctx is NULL"); return CHIMERA_ERR_INVALID_ARG; }
    std::lock_guard<std::recursive_mutex> lk(h->c.mu);
    CK(cudaSetDevice(h->c.device));
    return load_catalog(h->c, desc, id);
}

int chimera_unload_catalog(chimera_ctx *h, int32_t id) {
    if (!h) { set_error("ctx is NULL"); return CHIMERA_ERR_INVALID_ARG; }
    std::lock_guard<std::recursive_mutex> lk(h->c.mu);
    auto cat = find_catalog(h->c, id);
    if (!cat) { set_error("unknown catalog id"); return CHIMERA_ERR_NOT_FOUND; }
    CK(cudaSetDevice(h->c.device));
    cudaDeviceSynchronize();
    free_catalog(h->c, *cat);
    h->c.cats.erase(id);
    return CHIMERA_OK;
}

int chimera_catalog_info(chimera_ctx *h, int32_t id, chimera_catalog_info_t *info) {
    if (!h || !info) { set_error("null argument"); return CHIMERA_ERR_INVALID_ARG; }
    std::lock_guard<std::recursive_mutex> lk(h->c.mu);
    auto cat = find_catalog(h->c, id);
    if (!cat) { set_error("unknown catalog id"); return CHIMERA_ERR_NOT_FOUND; }
    *info = cat->info;
    return CHIMERA_OK;
}

static int check_call(chimera_ctx *h, int32_t n, const void *theta, int32_t prec, const void *out) {
    if (!h || !theta || !out) { set_error("null argument"); return CHIMERA_ERR_INVALID_ARG; }
    if (n <= 0) { set_error("n_points must be positive"); return CHIMERA_ERR_INVALID_ARG; }
    const int base = prec & ~(CHIMERA_KERNEL_EPANECHNIKOV | CHIMERA_JACOBIAN_PER_SAMPLE);
    if (base != CHIMERA_FP64 && base != CHIMERA_MIXED && base != CHIMERA_MIXED_BINNED) {
        set_error("bad precision");
        return CHIMERA_ERR_INVALID_ARG;
    }
    return CHIMERA_OK;
}

int chimera_loglike(chimera_ctx *h, int32_t id, int32_t n, const double *theta, int32_t prec,
                    double *lnL, double *neff, int32_t *status) {
    RC(check_call(h, n, theta, prec, lnL));
    Ctx &ctx = h->c;
    std::lock_guard<std::recursive_mutex> lk(ctx.mu);
    auto cat = find_catalog(ctx, id);
    if (!cat) { set_error("unknown catalog id"); return CHIMERA_ERR_NOT_FOUND; }
    CK(cudaSetDevice(ctx.device));
    RC(forward(ctx, *cat, ctx.ws, n, theta, prec));
    cudaStream_t st = ctx.ws.st;
    CK(cudaMemcpyAsync(lnL, ctx.ws.lnL, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    if (neff) CK(cudaMemcpyAsync(neff, ctx.ws.neff, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    if (status) {
        CallPtrs p = ctx.ws.ptrs(n, cat->d);
        CK(cudaMemcpyAsync(status, p.status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    return CHIMERA_OK;
}

int chimera_loglike_device(chimera_ctx *h, int32_t id, int32_t n, const double *theta_dev,
                           int32_t prec, double *lnL_dev, double *neff_dev, int32_t *status_dev,
                           void *stream) {
    RC(check_call(h, n, theta_dev, prec, lnL_dev));
    Ctx &ctx = h->c;
    std::lock_guard<std::recursive_mutex> lk(ctx.mu);
    auto cat = find_catalog(ctx, id);
    if (!cat) { set_error("unknown catalog id"); return CHIMERA_ERR_NOT_FOUND; }
    CK(cudaSetDevice(ctx.device));
    cudaStream_t us = stream ? (cudaStream_t)stream : ctx.stream;
    // theta comes back to the host (the Om caches are looked up there) through
    // a pinned buffer, a direct DMA instead of a staged pageable copy
    const size_t nth = 12 * (size_t)n;
    if (ctx.dev_theta_cap < nth) {
        if (ctx.dev_theta_h) cudaFreeHost(ctx.dev_theta_h);
        ctx.dev_theta_h = nullptr;
        ctx.dev_theta_cap = 0;
        if (cudaMallocHost((void **)&ctx.dev_theta_h, sizeof(double) * nth) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMallocHost failed for the theta staging buffer");
            return CHIMERA_ERR_CUDA;
        }
        ctx.dev_theta_cap = nth;
    }
    CK(cudaMemcpyAsync(ctx.dev_theta_h, theta_dev, sizeof(double) * nth, cudaMemcpyDeviceToHost, us));
    CK(cudaStreamSynchronize(us));
    // the combine kernel writes the caller's buffers directly
    RC(forward(ctx, *cat, ctx.ws, n, ctx.dev_theta_h, prec, lnL_dev, neff_dev, status_dev));
    if (!ctx.dev_done) CK(cudaEventCreateWithFlags(&ctx.dev_done, cudaEventDisableTiming));
    CK(cudaEventRecord(ctx.dev_done, ctx.ws.st));
    CK(cudaStreamWaitEvent(us, ctx.dev_done, 0));
    return CHIMERA_OK;
}

int chimera_terms(chimera_ctx *h, int32_t id, int32_t n, const double *theta, int32_t prec,
                  double *lnI, double *bw, double *xi, double *neff) {
    RC(check_call(h, n, theta, prec, theta));
    Ctx &ctx = h->c;
    std::lock_guard<std::recursive_mutex> lk(ctx.mu);
    auto cat = find_catalog(ctx, id);
    if (!cat) { set_error("unknown catalog id"); return CHIMERA_ERR_NOT_FOUND; }
    CK(cudaSetDevice(ctx.device));
    RC(forward(ctx, *cat, ctx.ws, n, theta, prec));
    cudaStream_t st = ctx.ws.st;
    size_t ne = (size_t)cat->d.n_events;
    if (lnI) CK(cudaMemcpyAsync(lnI, ctx.ws.lnI, sizeof(double) * n * ne, cudaMemcpyDeviceToHost, st));
    if (bw) CK(cudaMemcpyAsync(bw, ctx.ws.bw, sizeof(double) * n * ne, cudaMemcpyDeviceToHost, st));
    if (xi) CK(cudaMemcpyAsync(xi, ctx.ws.xi, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    if (neff) CK(cudaMemcpyAsync(neff, ctx.ws.neff, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return CHIMERA_OK;
}

int chimera_grad(chimera_ctx *h, int32_t id, int32_t n, const double *theta, int32_t prec,
                 double *lnL, double *dlnL, int32_t *status) {
    RC(check_call(h, n, theta, prec, lnL));
    if (prec != CHIMERA_FP64 && prec != CHIMERA_MIXED) {
        set_error("the adjoint follows the unbinned Gaussian KDE: use CHIMERA_FP64 or CHIMERA_MIXED");
        return CHIMERA_ERR_INVALID_ARG;
    }
    if (!dlnL) { set_error("dlnL is NULL"); return CHIMERA_ERR_INVALID_ARG; }
    Ctx &ctx = h->c;
    std::lock_guard<std::recursive_mutex> lk(ctx.mu);
    auto cat = find_catalog(ctx, id);
    if (!cat) { set_error("unknown catalog id"); return CHIMERA_ERR_NOT_FOUND; }
    if (cat->d.kde_mode == CHIMERA_KDE_3D) {
        set_error("the adjoint covers the 1-D kernels: CHIMERA_KDE_3D catalogs have no gradient");
        return CHIMERA_ERR_INVALID_ARG;
    }
    CK(cudaSetDevice(ctx.device));
    RC(forward(ctx, *cat, ctx.ws, n, theta, prec | PREC_WITH_GRAD));
    RC(backward(ctx, *cat, ctx.ws, n, prec));
    cudaStream_t st = ctx.ws.st;
    CK(cudaMemcpyAsync(lnL, ctx.ws.lnL, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(dlnL, ctx.ws.grad, sizeof(double) * 12 * n, cudaMemcpyDeviceToHost, st));
    if (status) {
        CallPtrs p = ctx.ws.ptrs(n, cat->d);
        CK(cudaMemcpyAsync(status, p.status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    return CHIMERA_OK;
}

int chimera_serve_submit(chimera_ctx *h, int32_t id, int32_t n, const double *theta, int32_t flags,
                         uint64_t *ticket) {
    if (!h || !theta || !ticket || n <= 0) { set_error("bad argument"); return CHIMERA_ERR_INVALID_ARG; }
    {
        std::lock_guard<std::recursive_mutex> lk(h->c.mu);
        auto cat = find_catalog(h->c, id);
        if (cat && cat->d.kde_mode == CHIMERA_KDE_3D) {
            set_error("serving runs the mixed 1-D kernels: CHIMERA_KDE_3D catalogs are not served");
            return CHIMERA_ERR_INVALID_ARG;
        }
    }
    return serve_submit(h->c, id, n, theta, flags, ticket);
}

int chimera_serve_poll(chimera_ctx *h, uint64_t ticket, int64_t timeout_us, double *lnL, double *dlnL,
                       int32_t *status) {
    if (!h || !lnL) { set_error("bad argument"); return CHIMERA_ERR_INVALID_ARG; }
    return serve_poll(h->c, ticket, timeout_us, lnL, dlnL, status);
}

int chimera_serve_cancel(chimera_ctx *h, uint64_t ticket) {
    if (!h) { set_error("bad argument"); return CHIMERA_ERR_INVALID_ARG; }
    return serve_cancel(h->c, ticket);
}

int chimera_serve_reset_stats(chimera_ctx *h) {
    if (!h) { set_error("bad argument"); return CHIMERA_ERR_INVALID_ARG; }
    return serve_reset_stats(h->c);
}

int chimera_serve_stats(chimera_ctx *h, chimera_serve_stats_t *out) {
    if (!h || !out) { set_error("bad argument"); return CHIMERA_ERR_INVALID_ARG; }
    return serve_stats(h->c, out);
}

int chimera_set_trace(chimera_ctx *h, int enable) {
    if (!h) { set_error("ctx is NULL"); return CHIMERA_ERR_INVALID_ARG; }
    std::lock_guard<std::recursive_mutex> lk(h->c.mu);
    h->c.ws.trace = enable != 0;
    return CHIMERA_OK;
}

int chimera_stage_ms(chimera_ctx *h, double *ms) {
    if (!h || !ms) { set_error("null argument"); return CHIMERA_ERR_INVALID_ARG; }
    std::lock_guard<std::recursive_mutex> lk(h->c.mu);
    Workspace &ws = h->c.ws;
    for (int i = 0; i < 7; i++) ms[i] = 0.0;
    if (!ws.trace || !ws.tev[5]) { set_error("tracing is off or no traced call yet"); return CHIMERA_ERR_INVALID_ARG; }
    CK(cudaEventSynchronize(ws.tev[5]));
    float t;
    // events: 0 start | 1 after K1a/K3 | 2 after K1b | 3 after K4 | 4 after K5 | 5 after K6
    CK(cudaEventElapsedTime(&t, ws.tev[1], ws.tev[2])); ms[0] = t;
    CK(cudaEventElapsedTime(&t, ws.tev[0], ws.tev[1])); ms[1] = t;
    CK(cudaEventElapsedTime(&t, ws.tev[2], ws.tev[3])); ms[2] = t;
    if (ws.traced_tiles > 0) {  // mixed: split K2 and K4 per tile
        double rw = 0.0, ev = 0.0;
        for (int i = 0; i < ws.traced_tiles; i++) {
            CK(cudaEventElapsedTime(&t, i == 0 ? ws.tev[2] : ws.tile_ev[2 * i - 1], ws.tile_ev[2 * i]));
            rw += t;
            CK(cudaEventElapsedTime(&t, ws.tile_ev[2 * i], ws.tile_ev[2 * i + 1]));
            ev += t;
        }
        ms[2] = ev;
        ms[6] = rw;
    }
    CK(cudaEventElapsedTime(&t, ws.tev[8], ws.tev[9])); ms[3] = t;  // side stream
    CK(cudaEventElapsedTime(&t, ws.tev[4], ws.tev[5])); ms[4] = t;
    if (ws.traced_adjoint && ws.tev[6] && ws.tev[7]) {
        CK(cudaEventSynchronize(ws.tev[7]));
        CK(cudaEventElapsedTime(&t, ws.tev[6], ws.tev[7])); ms[5] = t;
    }
    return CHIMERA_OK;
}

int chimera_kde_pairs(chimera_ctx *h, int32_t id, int32_t n, const double *theta, int64_t *pairs) {
    RC(check_call(h, n, theta, CHIMERA_MIXED, pairs));
    Ctx &ctx = h->c;
    std::lock_guard<std::recursive_mutex> lk(ctx.mu);
    auto cat = find_catalog(ctx, id);
    if (!cat) { set_error("unknown catalog id"); return CHIMERA_ERR_NOT_FOUND; }
    CK(cudaSetDevice(ctx.device));
    ctx.ws.count_pairs = true;
    int rc = forward(ctx, *cat, ctx.ws, n, theta, CHIMERA_MIXED);
    ctx.ws.count_pairs = false;
    RC(rc);
    std::vector<unsigned long long> v(n);
    CK(cudaMemcpyAsync(v.data(), ctx.ws.pairs, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, ctx.ws.st));
    CK(cudaStreamSynchronize(ctx.ws.st));
    for (int i = 0; i < n; i++) pairs[i] = (int64_t)v[i];
    return CHIMERA_OK;
}

int chimera_memory(chimera_ctx *h, int64_t *out) {
    if (!h || !out) { set_error("bad argument"); return CHIMERA_ERR_INVALID_ARG; }
    Ctx &ctx = h->c;
    std::lock_guard<std::recursive_mutex> lk(ctx.mu);
    auto r = [](size_t b) { return (std::max<size_t>(b, 16) + 255) & ~(size_t)255; };
    size_t cats = 0, cache = 0;
    for (auto &kv : ctx.cats) {
        cats += kv.second->bytes;
        for (auto &pe : kv.second->prof) cache += r(pe.second.bytes) + (pe.second.Gh ? r(pe.second.hbytes) : 0);
    }
    cache += (ctx.fwd.size() + ctx.fwdO.size()) * r(sizeof(double) * NT_FWD);
    out[0] = (int64_t)ctx.budget;
    out[1] = (int64_t)ctx.used.load();
    out[2] = (int64_t)cats;
    out[3] = (int64_t)cache;
    out[4] = (int64_t)(ctx.ws.bytes + ctx.ws.gscr_bytes + serve_ws_bytes(ctx) + ctx.ps.bytes);
    return CHIMERA_OK;
}

int chimera_peaks(chimera_ctx *h, double *out) {
    if (!h || !out) { set_error("bad argument"); return CHIMERA_ERR_INVALID_ARG; }
    std::lock_guard<std::recursive_mutex> lk(h->c.mu);
    CK(cudaSetDevice(h->c.device));
    if (run_peaks(out, h->c.stream)) { set_error("peak microbenchmark failed"); return CHIMERA_ERR_CUDA; }
    return CHIMERA_OK;
}

}  // extern "C"
