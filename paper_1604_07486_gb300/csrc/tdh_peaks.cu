// Arithmetic-rate probes: the FP32 (FFMA) and FP64 (DFMA) throughput of the current device,
// the denominators of the execute kernels' rooflines (the execute path is bound by the
// floating-point pipe, not by HBM).  Plain kernels timed with CUDA events; they change no
// clock or other device setting.
#include <cuda_runtime.h>

#include <algorithm>

#include "tdh_internal.cuh"

namespace tdh {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;   // independent FMA chains per thread (hides the pipe latency)
constexpr int kUnroll = 16;  // FMAs per chain per loop iteration

// Every thread runs kChains dependent chains x <- x * a + b, kUnroll * iters FMAs each.  The
// result is stored only if it equals an impossible value, so nothing is optimised away and
// nothing is written.
template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_rate(T* out, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == T(-12345.0)) out[blockIdx.x] = s;
}

template <typename T>
int measure(int iters, double* tflops, cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    TDH_CUDA(cudaGetDevice(&dev));
    TDH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TDH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate<T>,
                                                           kProbeThreads, 0));
    const int blocks = sms * std::max(per_sm, 1);
    T* sink = nullptr;
    TDH_TRY(scratch_alloc(reinterpret_cast<void**>(&sink), sizeof(T) * (size_t)blocks, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {  // one warm-up, three timed
        e = cudaEventRecord(e0, s);
        if (e != cudaSuccess) break;
        k_fma_rate<T><<<blocks, kProbeThreads, 0, s>>>(sink, iters, T(0.999999), T(1e-6));
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    scratch_free(sink, s);
    if (e != cudaSuccess) {
        set_error("fma rate probe: %s", cudaGetErrorString(e));
        return TDH_ERR_CUDA;
    }
    const double flops =
        2.0 * kChains * kUnroll * (double)iters * (double)blocks * (double)kProbeThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return TDH_OK;
}

}  // namespace
}  // namespace tdh

extern "C" int tdh_measure_fma_rate(int prec, double* tflops, void* stream) {
    tdh::clear_error();
    if (!tflops || (prec != TDH_FP32 && prec != TDH_FP64)) {
        tdh::set_error("tdh_measure_fma_rate: need prec TDH_FP32 or TDH_FP64 and non-NULL tflops");
        return TDH_ERR_INVALID_ARG;
    }
    cudaStream_t s = tdh::as_stream(stream);
    // about 30-60 ms per launch at the nominal rates (FP32 ~80, FP64 ~1.3 TFLOP/s)
    return prec == TDH_FP32 ? tdh::measure<float>(12000, tflops, s)
                            : tdh::measure<double>(200, tflops, s);
}
