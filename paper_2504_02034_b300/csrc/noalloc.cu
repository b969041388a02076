// chimera_selection_static: the selection term xi and its effective
// injection count for callers that cannot allocate device memory.
//
// Some callers run where a device allocation is not allowed: code that has
// handed the whole device memory to its own pool (and so fails or stalls on
// cudaMalloc), code running inside another framework's allocator discipline,
// or embedded / real-time loops that must not synchronise the device, which
// cudaMalloc and cudaFree can do.  This entry point computes the same FP64
// selection term as the catalog path (cosmology tables, injection sum and
// its fixed-order reduction) but keeps every intermediate in one file-scope
// device array of fixed size, so it calls no cudaMalloc, cudaFree or other
// allocating routine.  The caller passes its own device buffers for the
// injections and for the outputs.  Its inverse distance table spans the
// injections' own largest d_L (the catalog path's spans the PE samples too),
// so the nodes differ and xi, N_eff agree with the catalog path to ~1e-10
// relative, not bit for bit.
//
// Host code never dereferences the array's symbol: the first call on a
// device asks the runtime for its device address (cudaGetSymbolAddress) and
// remembers it for that device.  Every call also reads the largest injection
// distance back to the host, which synchronises `stream` once per call.  All calls share
// the array and it keeps the previous call's contents, so everything that
// must start at zero is cleared on the call's stream, and calls whose work
// overlaps on the GPU (different streams or threads at the same time) race
// on it.
#include <mutex>

#include "runtime.cuh"

namespace chim {

namespace {

constexpr int ST_HMAX = 64;          // hyperpoints per call
constexpr int ST_CHUNK_MAX = 4096;   // injection chunks: n_det <= 4096 * SEL_CHUNK
constexpr int ST_NZ = 2;             // grid factor is not used by the selection term
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets of the regions inside the array
constexpr size_t OFF_PARAM = 0;  // theta | status | fwd ptrs | prof ptrs (Workspace layout)
constexpr size_t SZ_PARAM = (size_t)ST_HMAX * (12 * 8 + 8 + 8 + 8);
constexpr size_t OFF_HP = al(OFF_PARAM + SZ_PARAM);
constexpr size_t OFF_INV64 = al(OFF_HP + sizeof(HP) * ST_HMAX);
constexpr size_t OFF_INV32 = al(OFF_INV64 + sizeof(double2) * ST_HMAX * (NU + 1));
constexpr size_t OFF_F64 = al(OFF_INV32 + sizeof(float4) * ST_HMAX * NU);
constexpr size_t OFF_F32 = al(OFF_F64 + sizeof(double) * ST_HMAX * ST_NZ);
constexpr size_t OFF_DK = al(OFF_F32 + sizeof(float) * ST_HMAX * ST_NZ);
constexpr size_t OFF_FMAX = al(OFF_DK + sizeof(float) * 2 * ST_HMAX * NT_FWD);  // FP32 d and J per node
constexpr size_t OFF_FWD = al(OFF_FMAX + sizeof(unsigned long long) * ST_HMAX);
constexpr size_t OFF_SELP = al(OFF_FWD + sizeof(double) * ST_HMAX * NT_FWD);
constexpr size_t OFF_DTOP = al(OFF_SELP + sizeof(double) * 2 * ST_HMAX * ST_CHUNK_MAX);
constexpr size_t SCRATCH_BYTES = al(OFF_DTOP + 8);

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

std::mutex g_mu;
void *g_addr[256] = {};  // device address of g_scratch per device ordinal

__global__ void k_dmax(const double *x, int64_t n, unsigned long long *out) {
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, x[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// fixed-order reduction of the per-chunk partial sums into xi and N_eff
__global__ void k_static_reduce(const double *selp, int n_chunk, double n_inj, const HP *hp,
                                double *xi, double *neff) {
    __shared__ double s1[256], s2[256];
    const int h = blockIdx.x, t = threadIdx.x;
    double a = 0.0, b = 0.0;
    for (int i = t; i < n_chunk; i += 256) {
        a += selp[((size_t)h * n_chunk + i) * 2];
        b += selp[((size_t)h * n_chunk + i) * 2 + 1];
    }
    s1[t] = a;
    s2[t] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) {
            s1[t] += s1[t + w];
            s2[t] += s2[t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        double S1 = s1[0], S2 = s2[0];
        bool bad = hp[h].status & (CHIMERA_PT_OUT_OF_SUPPORT | CHIMERA_PT_NONMONOTONE);
        xi[h] = bad ? 0.0 : S1 / n_inj;
        neff[h] = (bad || !(S1 > 0.0)) ? 0.0 : S1 * S1 / (S2 - S1 * S1 / n_inj);
    }
}

int scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
    if (dev < 0 || dev >= 256) {
        set_error("device ordinal out of range");
        return CHIMERA_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return cuda_check(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return CHIMERA_OK;
}

}  // namespace

}  // namespace chim

using namespace chim;

extern "C" int chimera_selection_static(int32_t n_points, const double *theta, int64_t n_det,
                                        int64_t n_inj_total, const double *inj_dL,
                                        const double *inj_m1d, const double *inj_m2d,
                                        const double *inj_log_pi, double lambda_g, double beta,
                                        double z_max, double *xi, double *neff, void *stream) {
    if (!theta || !xi || !neff || n_points <= 0) {
        set_error("null theta/output or n_points <= 0");
        return CHIMERA_ERR_INVALID_ARG;
    }
    if (n_points > ST_HMAX) {
        set_error("chimera_selection_static: at most 64 hyperpoints per call");
        return CHIMERA_ERR_UNSUPPORTED;
    }
    if (n_det < 1 || n_inj_total < n_det || !inj_dL || !inj_m1d || !inj_m2d || !inj_log_pi) {
        set_error("need n_det >= 1 detected injections, n_inj_total >= n_det and four device arrays");
        return CHIMERA_ERR_INVALID_ARG;
    }
    if (n_det > (int64_t)ST_CHUNK_MAX * SEL_CHUNK) {
        set_error("chimera_selection_static: at most 8388608 detected injections per call");
        return CHIMERA_ERR_UNSUPPORTED;
    }
    if (!(z_max > 0.0) || !(lambda_g >= 0.0 && lambda_g <= 1.0) || !(beta == beta)) {
        set_error("bad z_max, lambda_g or beta");
        return CHIMERA_ERR_INVALID_ARG;
    }
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    char *S = static_cast<char *>(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int H = n_points;

    // largest injection distance: the inverse-table range
    unsigned long long *dtop_bits = reinterpret_cast<unsigned long long *>(S + OFF_DTOP);
    cudaMemsetAsync(dtop_bits, 0, 8, st);
    k_dmax<<<148, 256, 0, st>>>(inj_dL, n_det, dtop_bits);
    unsigned long long bits = 0;
    cudaError_t e = cudaMemcpyAsync(&bits, dtop_bits, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(e, "chimera_selection_static: d_top");
    double dmax;
    memcpy(&dmax, &bits, 8);
    if (!(dmax > 0.0) || !std::isfinite(dmax)) {
        // no positive finite distance: the inverse table u = sqrt(d / d_top)
        // would have no range
        set_error("chimera_selection_static: inj_dL holds no positive finite distance");
        return CHIMERA_ERR_INVALID_ARG;
    }

    DevCatalog c{};
    c.n_z = ST_NZ;
    c.z_max = z_max;
    c.dz = z_max / (ST_NZ - 1);
    c.z_max32 = (float)z_max;
    c.dz32 = (float)c.dz;
    c.lambda_g = lambda_g;
    c.ln_lambda = lambda_g > 0.0 ? std::log(lambda_g) : 0.0;
    c.ln1m_lambda = lambda_g < 1.0 ? std::log1p(-lambda_g) : 0.0;
    c.beta = beta;
    c.d_top = dmax * (1.0 + 1e-9);
    c.n_det = n_det;
    c.n_inj_total = n_inj_total;
    c.id64 = const_cast<double *>(inj_dL);
    c.im1_64 = const_cast<double *>(inj_m1d);
    c.im2_64 = const_cast<double *>(inj_m2d);
    c.ilp64 = const_cast<double *>(inj_log_pi);

    // parameters staged on the host stack, copied into the array
    unsigned char stage[SZ_PARAM];
    double *th = reinterpret_cast<double *>(stage);
    int32_t *status = reinterpret_cast<int32_t *>(stage + sizeof(double) * 12 * H);
    const double **fw = reinterpret_cast<const double **>(stage + sizeof(double) * 12 * H + 8 * H);
    const void **pr = reinterpret_cast<const void **>(stage + sizeof(double) * 12 * H + 16 * H);
    memset(status, 0, 8 * (size_t)H);
    double *fwd_base = reinterpret_cast<double *>(S + OFF_FWD);
    double oms[ST_HMAX];
    int nom = 0;
    for (int h = 0; h < H; h++) {
        bool ok = theta_admissible(theta + 12 * h);
        memcpy(th + 12 * h, ok ? theta + 12 * h : kSafeTheta, sizeof(double) * 12);
        status[h] = ok ? 0 : CHIMERA_PT_OUT_OF_SUPPORT;
        double Om = th[12 * h + 1];
        int slot = -1;
        for (int k = 0; k < nom; k++)
            if (memcmp(&oms[k], &Om, 8) == 0) slot = k;
        if (slot < 0) {
            slot = nom;
            oms[nom++] = Om;
            launch_fwd_table(Om, fwd_base + (size_t)slot * NT_FWD, st);
        }
        fw[h] = fwd_base + (size_t)slot * NT_FWD;
        pr[h] = nullptr;
    }
    e = cudaMemcpyAsync(S + OFF_PARAM, stage, (size_t)H * (12 * 8 + 8 + 8 + 8), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_check(e, "chimera_selection_static: parameters");

    CallPtrs p{};
    p.theta = reinterpret_cast<const double *>(S + OFF_PARAM);
    p.status = reinterpret_cast<int32_t *>(S + OFF_PARAM + sizeof(double) * 12 * H);
    p.fwd = reinterpret_cast<const double *const *>(S + OFF_PARAM + sizeof(double) * 12 * H + 8 * H);
    p.prof = reinterpret_cast<const void *const *>(S + OFF_PARAM + sizeof(double) * 12 * H + 16 * H);
    p.hp = reinterpret_cast<HP *>(S + OFF_HP);
    p.inv64 = reinterpret_cast<double2 *>(S + OFF_INV64);
    p.inv32 = reinterpret_cast<float4 *>(S + OFF_INV32);
    p.F64 = reinterpret_cast<double *>(S + OFF_F64);
    p.F32 = reinterpret_cast<float *>(S + OFF_F32);
    p.selp = reinterpret_cast<double *>(S + OFF_SELP);
    p.n_chunk = selection_chunks(c);
    launch_hyper_tables(c, p, H, true, reinterpret_cast<double *>(S + OFF_DK),
                        reinterpret_cast<unsigned long long *>(S + OFF_FMAX), st);
    launch_selection(c, p, H, true, st);
    k_static_reduce<<<H, 256, 0, st>>>(p.selp, p.n_chunk, (double)n_inj_total, p.hp, xi, neff);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(e, "chimera_selection_static: launch");
    return CHIMERA_OK;
}
