// Fused multiply-add throughput of the GPU, FP32 or FP64: the denominator of
// the arithmetic rooflines the benchmark reports (no counterpart in the paper).
//
// Every thread runs kChains independent FMA chains x <- x a + b (a just below 1,
// so the values stay near b / (1 - a) and never overflow or go subnormal);
// kChains independent chains per thread and 32 warps per SM keep every FMA
// pipe busy despite its latency.  The sum of the chains is stored, so that the
// work cannot be removed.  The device time comes from CUDA events around a
// launch sized to take about target_ms, after one warm-up launch.  Nothing
// here reads or changes clocks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ffsat.h"
#include "ffsat_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

template <typename R>
__global__ void __launch_bounds__(kThreads) fma_chains(R *out, int iters, R a, R b) {
    R x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = R(threadIdx.x + k) * R(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    R s = R(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename R>
int measure(double target_ms, double *tflops, double *ms_out, cudaStream_t s) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ffsat::set_error(FFSAT_ERR_CUDA, "cudaGetDevice / multiProcessorCount failed");
    const int grid = sms * kBlocksPerSm;
    R *out = nullptr;
    if (cudaMalloc(&out, (size_t)grid * kThreads * sizeof(R)) != cudaSuccess)
        return ffsat::set_error(FFSAT_ERR_CUDA, "cudaMalloc of the peak benchmark's output failed");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = FFSAT_OK;
    auto timed = [&](int iters, float &ms) -> bool {
        if (cudaEventRecord(e0, s) != cudaSuccess) return false;
        fma_chains<R><<<grid, kThreads, 0, s>>>(out, iters, R(0.999999), R(1e-6));
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess)
            return false;
        return cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    };
    float ms = 0.0f;
    int iters = 64;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess || !timed(iters, ms)) {
        rc = ffsat::set_error(FFSAT_ERR_CUDA, "peak benchmark launch failed");
    } else {
        // grow the launch until it takes about target_ms: at most 16x per step (a
        // first launch dominated by its overhead must not size a seconds-long one)
        // and at most 2^24 iterations
        for (int k = 0; k < 20 && ms < 0.5 * target_ms && iters < (1 << 24); ++k) {
            const double grow = std::min(16.0, std::max(2.0, target_ms / std::max((double)ms, 1e-3)));
            iters = (int)std::min<double>((double)(1 << 24), iters * grow);
            if (!timed(iters, ms)) {
                rc = ffsat::set_error(FFSAT_ERR_CUDA, "peak benchmark launch failed");
                break;
            }
        }
        if (rc == FFSAT_OK && !timed(iters, ms)) rc = ffsat::set_error(FFSAT_ERR_CUDA, "peak benchmark launch failed");
    }
    if (rc == FFSAT_OK) {
        const double flops = 2.0 * kChains * kUnroll * (double)iters * (double)grid * kThreads;
        *tflops = flops / (ms * 1e-3) / 1e12;
        if (ms_out) *ms_out = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}

}  // namespace

extern "C" int ffsat_alu_peak(int32_t dtype, double target_ms, double *tflops, double *ms, void *stream) {
    if (!tflops) return ffsat::set_error(FFSAT_ERR_ARG, "tflops is NULL");
    if (dtype != FFSAT_F32 && dtype != FFSAT_F64) return ffsat::set_error(FFSAT_ERR_ARG, "dtype must be FFSAT_F32 or FFSAT_F64");
    if (!(target_ms > 0.0 && target_ms <= 10000.0)) return ffsat::set_error(FFSAT_ERR_ARG, "target_ms must be in (0, 10000]");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return dtype == FFSAT_F32 ? measure<float>(target_ms, tflops, ms, s) : measure<double>(target_ms, tflops, ms, s);
}
