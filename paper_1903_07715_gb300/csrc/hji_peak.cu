// hji_peak_fma: the measured fused-multiply-add rate of this GPU in FP32 or
// FP64, the denominator of the arithmetic roofline the stage kernels are
// reported against (a measurement aid; the paper has no counterpart).
//
// Every thread runs kChains independent multiply-add chains a <- a*b + c,
// enough to cover the FMA latency with a few warps per scheduler; the grid
// fills every SM with kBlocksPerSM CTAs of 256 threads.  One FMA counts as
// two floating-point operations.  The host calibrates the loop count to the
// requested duration, then times several launches with CUDA events on the
// caller's stream and reports the fastest.
#include <cmath>
#include <cstdio>

#include "hji_common.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kBlocksPerSM = 8;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(long long iters, T b, T c, T* sink) {
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = T(threadIdx.x + i) * T(1e-3);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
        }
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    // The chains converge to c / (1 - b) > 0: this store never happens, but
    // the compiler cannot know it, so every FMA stays.
    if (s < T(0) && sink != nullptr) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

thread_local char g_err[256] = "";

}  // namespace

extern "C" const char* hji_peak_last_error(void) { return g_err; }

extern "C" hji_status hji_peak_fma(hji_precision prec, double target_ms, void* cuda_stream,
                                   double* tflops, double* ms_per_launch) {
    if (prec != HJI_F64 && prec != HJI_F32) {
        std::snprintf(g_err, sizeof(g_err), "unknown precision");
        return HJI_E_INVALID;
    }
    if (!tflops || !(target_ms >= 1.0 && target_ms <= 1000.0)) {
        std::snprintf(g_err, sizeof(g_err), "tflops must be non-NULL and target_ms in [1, 1000]");
        return HJI_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = sms * kBlocksPerSM;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    auto run = [&](long long iters, float* ms) {
        cudaError_t r = cudaEventRecord(ev[0], s);
        if (r != cudaSuccess) return r;
        if (prec == HJI_F32)
            fma_peak_kernel<float><<<grid, kPeakThreads, 0, s>>>(iters, 0.999999f, 1e-7f, nullptr);
        else
            fma_peak_kernel<double><<<grid, kPeakThreads, 0, s>>>(iters, 0.999999, 1e-7, nullptr);
        r = cudaGetLastError();
        if (r == cudaSuccess) r = cudaEventRecord(ev[1], s);
        if (r == cudaSuccess) r = cudaEventSynchronize(ev[1]);
        if (r == cudaSuccess) r = cudaEventElapsedTime(ms, ev[0], ev[1]);
        return r;
    };
    double best = 0.0, best_ms = 0.0;
    if (e == cudaSuccess) {
        // Calibrate: grow the loop count until a launch takes a tenth of the
        // target, then scale to the target.
        long long iters = 64;
        float ms = 0.0f;
        for (int k = 0; k < 24 && e == cudaSuccess; ++k) {
            e = run(iters, &ms);
            if (e != cudaSuccess || ms >= 0.1 * target_ms) break;
            iters *= 4;
        }
        if (e == cudaSuccess && ms > 0.0f)
            iters = (long long)std::ceil(iters * (target_ms / ms));
        for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
            e = run(iters, &ms);
            const double flops = 2.0 * kChains * 16.0 * (double)iters * grid * kPeakThreads;
            const double tf = flops / (ms * 1e-3) / 1e12;
            if (e == cudaSuccess && tf > best) {
                best = tf;
                best_ms = ms;
            }
        }
    }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) {
        std::snprintf(g_err, sizeof(g_err), "FMA peak: %s", cudaGetErrorString(e));
        return HJI_E_CUDA;
    }
    *tflops = best;
    if (ms_per_launch) *ms_per_launch = best_ms;
    return HJI_OK;
}
