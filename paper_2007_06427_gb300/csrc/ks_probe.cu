// ks_probe.cu - measured arithmetic peaks of the current GPU (FP64 and FP32 fused multiply-add).
//
// The hot path of the tau-descent is bound by the FP64 (double descent) or FP32 (float bulk)
// pipes, not by HBM; the roofline fractions the benchmark reports are taken against the nominal
// rates, and this probe measures what the pipes deliver on the part at hand.  Every thread of a
// grid of (SMs x blocks_per_sm) blocks runs `iters` rounds of kAcc independent FMA chains (no
// memory traffic inside the loop); the result is written so the compiler keeps the chains.
#include <cuda_runtime.h>

#include "ks_loop.h"

namespace {

constexpr int kAcc = 8;         // independent accumulators per thread (hides the FMA latency)
constexpr int kThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kThreads) k_fma_probe(R* out, int iters, R a, R b) {
    R acc[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i) acc[i] = (R)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kAcc; ++i) acc[i] = acc[i] * a + b;
    }
    R s = 0;
#pragma unroll
    for (int i = 0; i < kAcc; ++i) s += acc[i];
    // the chains stay positive for the a, b below, so nothing is written; the store keeps them live
    if (out && s == (R)-1.2345) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

void ks_internal_set_error(const char* msg);

namespace {
int probe_fail(int code, const char* msg) {
    ks_internal_set_error(msg);
    return code;
}
}  // namespace

extern "C" int ks_probe_peak(int precision, int iters, double* tflops, void* stream) {
    ks_internal_set_error("");
    if (!tflops || (precision != KS_FP64 && precision != KS_FP32) || iters < 1)
        return probe_fail(KS_ERR_ARG, "ks_probe_peak: precision must be KS_FP64 or KS_FP32, iters >= 1, tflops non-null");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return probe_fail(KS_ERR_CUDA, "no usable CUDA device");
    }
    cudaError_t e = precision == KS_FP64
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<double>, kThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<float>, kThreads, 0);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return probe_fail(KS_ERR_CUDA, "occupancy query failed");
    }
    const int grid = sms * per_sm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return probe_fail(KS_ERR_CUDA, "event creation failed");
    }
    float ms = 0.f;
    // warm-up launch (clocks up, code loaded), then the timed one
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, s);
        if (precision == KS_FP64)
            k_fma_probe<double><<<grid, kThreads, 0, s>>>(nullptr, iters, 0.999999, 1e-9);
        else
            k_fma_probe<float><<<grid, kThreads, 0, s>>>(nullptr, iters, 0.9999f, 1e-6f);
        cudaEventRecord(e1, s);
    }
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0.f) {
        cudaGetLastError();
        return probe_fail(KS_ERR_CUDA, "probe launch failed");
    }
    const double flops = 2.0 * kAcc * (double)iters * (double)grid * kThreads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return KS_OK;
}
