// Rate probes: the FP32 (FFMA) and FP64 (DFMA) throughput of the current device, the
// denominators of the execute kernels' rooflines (the execute path is bound by the
// floating-point pipe, not by HBM), and the distributed-shared-memory throughput that bounds
// the cluster kernel's cross stage.  Plain kernels timed with CUDA events or clock64; they
// change no clock or other device setting.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

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

// Distributed shared memory: the access pattern of the float32 cluster kernel's cross stage
// in a 4-CTA cluster with one 512-thread CTA per SM.  CTA k owns a quarter of a 128 KB
// buffer's positions; for its quarter it moves 16-byte pairs from (mode 0: loads), to
// (mode 1: stores) or from and back to (mode 2: both, the cross stage without its
// arithmetic) the three other CTAs' buffers, `rounds` times (no barrier between rounds: each
// CTA touches only its own quarter of every buffer; one cluster barrier ends the timed part).
// Each CTA records its clock64 cycles; the probe reports remote bytes per cycle per SM, with
// every cluster that fits resident at once and (loads) with one cluster alone on the GPU.
constexpr int kDsmC = 4, kDsmThreads = 512;
constexpr int kDsmBuf = 128 * 1024;          // bytes of buffer per CTA
constexpr int kDsmOwn = kDsmBuf / kDsmC / 16;  // 16-byte pairs owned per CTA

// One round of the probe's mode 2 (H: the half of the thread's positions it loads).
template <int H, int PER>
__device__ __forceinline__ void dsmem_half_round(float4 (&v)[PER][kDsmC],
                                                 float4* const (&rb)[kDsmC], int k, int tid,
                                                 bool store) {
#pragma unroll
    for (int q = 0; q < PER / 2; ++q) {
        constexpr int kHalf = PER / 2;
        const int pl = kHalf * H + q, ps = kHalf * (1 - H) + q;
        const int al = k * kDsmOwn + tid + pl * kDsmThreads;
        const int as = k * kDsmOwn + tid + ps * kDsmThreads;
#pragma unroll
        for (int j = 0; j < kDsmC; ++j) {
            v[pl][j] = rb[j][al];
            if (j != k && store)
                rb[j][as] = make_float4(v[ps][j].x + 1.f, v[ps][j].y, v[ps][j].z, v[ps][j].w);
        }
    }
}

__global__ void __launch_bounds__(kDsmThreads, 1)
    k_dsmem_rate(int mode, int rounds, long long* cycles, float* sink) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) float4 dbuf[];
    cg::cluster_group cl = cg::this_cluster();
    const int k = (int)cl.block_rank(), tid = threadIdx.x;
    for (int i = tid; i < kDsmBuf / 16; i += kDsmThreads)
        dbuf[i] = make_float4((float)i, (float)k, 1.f, 2.f);
    cl.sync();
    float4* rb[kDsmC];
#pragma unroll
    for (int j = 0; j < kDsmC; ++j) rb[j] = cl.map_shared_rank(dbuf, j);
    float acc = 0.f;
    constexpr int kPer = kDsmOwn / kDsmThreads;  // positions per thread and round
    static_assert(kDsmOwn % kDsmThreads == 0, "whole positions per thread");
    float4 v[kPer][kDsmC];
#pragma unroll
    for (int p = 0; p < kPer; ++p)
#pragma unroll
        for (int j = 0; j < kDsmC; ++j) v[p][j] = make_float4(0.f, 0.f, 0.f, 0.f);
    const long long t0 = clock64();
#pragma unroll 1
    for (int r = 0; r < rounds; ++r) {
        // every access of the round is issued before any is used (as many in flight as the
        // thread can have); stored values differ from the loaded ones, so no store is elided.
        // Mode 2 keeps both directions busy at once, on different places: in round r the
        // thread loads the positions of half r % 2 and stores, to the other half, the values
        // it loaded there in the previous round.
        if (mode == 2) {
            if (r & 1)
                dsmem_half_round<1, kPer>(v, rb, k, tid, r > 0);
            else
                dsmem_half_round<0, kPer>(v, rb, k, tid, r > 0);
        } else {
#pragma unroll
            for (int p = 0; p < kPer; ++p) {
                const int at = k * kDsmOwn + tid + p * kDsmThreads;
#pragma unroll
                for (int j = 0; j < kDsmC; ++j)
                    v[p][j] = (mode == 0) ? rb[j][at] : make_float4(acc + p, (float)j, 1.f, 2.f);
            }
        }
        if (mode == 0) {
#pragma unroll
            for (int p = 0; p < kPer; ++p)
#pragma unroll
                for (int j = 0; j < kDsmC; ++j) acc += v[p][j].x + v[p][j].w;
        } else if (mode == 1) {
#pragma unroll
            for (int p = 0; p < kPer; ++p) {
                const int at = k * kDsmOwn + tid + p * kDsmThreads;
#pragma unroll
                for (int j = 0; j < kDsmC; ++j) {
                    if (j == k) continue;
                    float4 w = v[p][j];
                    w.x += 1.f;
                    rb[j][at] = w;
                }
            }
        }
        asm volatile("" ::: "memory");  // the next round loads again (no caching in registers)
    }
    cl.sync();  // every access of every CTA complete
    const long long t1 = clock64();
    if (tid == 0) cycles[blockIdx.x] = t1 - t0;
    if (acc == -12345.f) sink[blockIdx.x] = acc;  // keeps the loads; never true
}

int measure_dsmem(double* bytes_per_cycle, cudaStream_t s) {
    constexpr int kRounds = 200;
    TDH_CUDA(cudaFuncSetAttribute(k_dsmem_rate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kDsmBuf));
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kDsmThreads, 1, 1);
    cfg.dynamicSmemBytes = kDsmBuf;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kDsmC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(kDsmC, 1, 1);
    int clusters = 0;
    TDH_CUDA(cudaOccupancyMaxActiveClusters(&clusters, k_dsmem_rate, &cfg));
    clusters = std::max(clusters, 1);  // all resident at once: the network fully loaded
    const int grid = clusters * kDsmC;
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    char* mem = nullptr;
    TDH_TRY(scratch_alloc(reinterpret_cast<void**>(&mem),
                          (sizeof(long long) + sizeof(float)) * (size_t)grid, s));
    long long* cyc = reinterpret_cast<long long*>(mem);
    float* sink = reinterpret_cast<float*>(cyc + grid);
    std::vector<long long> h((size_t)grid);
    cudaError_t e = cudaSuccess;
    // runs 0-2: modes 0-2 with every cluster resident; run 3: mode 0 with one cluster alone
    for (int run = 0; e == cudaSuccess && run < 4; ++run) {
        const int mode = run < 3 ? run : 0;
        const int g = run < 3 ? grid : kDsmC;
        cfg.gridDim = dim3((unsigned)g, 1, 1);
        long long best = 0;
        for (int rep = 0; e == cudaSuccess && rep < 3; ++rep) {  // one warm-up, two timed
            e = cudaLaunchKernelEx(&cfg, k_dsmem_rate, mode, kRounds, cyc, sink);
            if (e == cudaSuccess) note_launches(1);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h.data(), cyc, sizeof(long long) * (size_t)g,
                                    cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess || rep == 0) continue;
            const long long worst = *std::max_element(h.begin(), h.begin() + g);
            if (best == 0 || worst < best) best = worst;
        }
        // remote bytes of one CTA: three other CTAs' quarters, one way (loads or stores) per
        // round; mode 2 moves half a quarter each way per round (its first round only loads)
        const double bytes = (mode == 2 ? (2.0 * kRounds - 1.0) / 2.0 : (double)kRounds) *
                             (kDsmC - 1) * kDsmOwn * 16.0;
        if (e == cudaSuccess) bytes_per_cycle[run] = bytes / (double)std::max(best, 1LL);
    }
    scratch_free(mem, s);
    if (e != cudaSuccess) {
        set_error("distributed shared memory probe: %s", cudaGetErrorString(e));
        return TDH_ERR_CUDA;
    }
    return TDH_OK;
}

}  // namespace
}  // namespace tdh

extern "C" int tdh_measure_dsmem_rate(double* bytes_per_cycle, void* stream) {
    tdh::clear_error();
    if (!bytes_per_cycle) {
        tdh::set_error("tdh_measure_dsmem_rate: NULL bytes_per_cycle");
        return TDH_ERR_INVALID_ARG;
    }
    return tdh::measure_dsmem(bytes_per_cycle, tdh::as_stream(stream));
}

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
