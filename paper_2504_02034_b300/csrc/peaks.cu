// K8: microbenchmarks for the roofline denominators of this GPU.
//  - FP32 "pair" rate: the KDE inner-loop step, one FFMA (Horner: acc = acc *
//    B + D) per pair, eight independent chains per thread;
//  - MUFU ex2 rate (ex2.approx.f32 in independent chains);
//  - FP64 DFMA rate;
//  - device-to-device copy bandwidth (read + write bytes).
// Each rate is the best of a few timed launches with CUDA events.
#include "internal.cuh"

namespace chim {

namespace {

constexpr int PK_THREADS = 256;

__global__ void k_pairs(float *out, int iters, float seed) {
    float P[8], B[8], A[8];
#pragma unroll
    for (int r = 0; r < 8; r++) {
        P[r] = seed + r * 1e-3f + threadIdx.x * 1e-7f;
        B[r] = 1.0f - 1e-7f * r;
        A[r] = 0.f;
    }
    const float D = 0.5f + seed * 1e-3f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < 8; r++) A[r] = fmaf(A[r], B[r], D);  // Horner step
    }
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < 8; r++) s += A[r] + P[r];
    if (s == 12345.678f) out[threadIdx.x] = s;
}

__global__ void k_ex2(float *out, int iters, float seed) {
    float x[8];
#pragma unroll
    for (int r = 0; r < 8; r++) x[r] = -1e-3f * (r + 1) + seed * 1e-9f * threadIdx.x;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < 8; r++) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[r]));
            x[r] = y - 1.0f;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < 8; r++) s += x[r];
    if (s == 12345.678f) out[threadIdx.x] = s;
}

__global__ void k_dfma(double *out, int iters, double seed) {
    double a[8];
#pragma unroll
    for (int r = 0; r < 8; r++) a[r] = seed + r;
    const double m = 0.999999, c = 1e-9;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < 8; r++) a[r] = fma(a[r], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < 8; r++) s += a[r];
    if (s == 12345.678) out[threadIdx.x] = s;
}

template <typename F>
double best_ms(F launch, cudaStream_t st, int reps) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();  // warm-up
    double best = 1e30;
    for (int i = 0; i < reps; i++) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

}  // namespace

int run_peaks(double *out, cudaStream_t st) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    float *fb = nullptr;
    if (cudaMalloc(&fb, 4096) != cudaSuccess) return -1;
    const int blocks = nsm * 8;
    const int it = 4096;
    double ms = best_ms([&] { k_pairs<<<blocks, PK_THREADS, 0, st>>>(fb, it, 0.3f); }, st, 5);
    out[0] = (double)blocks * PK_THREADS * it * 8 / (ms * 1e-3);
    ms = best_ms([&] { k_ex2<<<blocks, PK_THREADS, 0, st>>>(fb, it / 4, 0.3f); }, st, 5);
    out[1] = (double)blocks * PK_THREADS * (it / 4) * 8 / (ms * 1e-3);
    ms = best_ms([&] { k_dfma<<<blocks, PK_THREADS, 0, st>>>((double *)fb, it / 16, 0.3); }, st, 5);
    out[2] = (double)blocks * PK_THREADS * (it / 16) * 8 / (ms * 1e-3);
    cudaFree(fb);
    const size_t bytes = (size_t)1 << 29;
    void *a = nullptr, *b = nullptr;
    if (cudaMalloc(&a, bytes) != cudaSuccess) return -1;
    if (cudaMalloc(&b, bytes) != cudaSuccess) { cudaFree(a); return -1; }
    cudaMemsetAsync(a, 0, bytes, st);
    ms = best_ms([&] { cudaMemcpyAsync(b, a, bytes, cudaMemcpyDeviceToDevice, st); }, st, 5);
    out[3] = 2.0 * bytes / (ms * 1e-3);
    cudaFree(a);
    cudaFree(b);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace chim
