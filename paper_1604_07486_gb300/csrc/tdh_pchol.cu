// Step a2: pivoted Cholesky of a positive semidefinite Hankel block, O(K^2 N), in float64
// (Sec. 2.1, Fig. 2).
//
// Only the diagonal d and the K selected columns are ever formed.  Step r:
//   p_r = argmax_j d_j                      (lowest index on ties)
//   c   = H[:, p_r] - sum_{i<r} u_i u_i[p_r]   (earlier steps applied to column p_r)
//   a_r = c[p_r];  u_r = c / sqrt(a_r);  d <- d - u_r^2
// and the factorisation stops before any step whose pivot (max d, or a_r) is
// <= tol * max(diag H).  u_r = l_r / sqrt(a_r) in the paper's notation, so
// H ~ sum_r l_r l_r^T / a_r = sum_r u_r u_r^T.
//
// One launch per step over a grid of blocks; each block owns a fixed slice of indices and
// also publishes the argmax of its slice of the updated d, which every block of the next
// step reduces (a few hundred entries) to find the next pivot.  Every block takes the same
// stop decision from the same data, so no grid-wide wait is needed.  The host reads the
// "done" flag every few steps and stops launching.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tdh_internal.cuh"

namespace tdh {
namespace {

constexpr int kThreads = 256;
constexpr int kKmaxShared = 1024;  // u_i[p] for i < r staged in shared memory

struct ArgMax {
    double v;
    int64_t i;
};

struct State {
    double thresh;  // tol * d0
    int64_t K;      // steps taken so far
    int done;
};

__device__ __forceinline__ ArgMax amax(ArgMax a, ArgMax b) {
    return (b.v > a.v || (b.v == a.v && b.i < a.i)) ? b : a;
}

__device__ ArgMax block_argmax(ArgMax x) {
    __shared__ double sv[kThreads / 32];
    __shared__ int64_t si[kThreads / 32];
    for (int off = 16; off > 0; off >>= 1) {
        ArgMax o;
        o.v = __shfl_down_sync(0xffffffffu, x.v, off);
        o.i = __shfl_down_sync(0xffffffffu, x.i, off);
        x = amax(x, o);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sv[w] = x.v;
        si[w] = x.i;
    }
    __syncthreads();
    if (w == 0) {
        x.v = (l < kThreads / 32) ? sv[l] : -INFINITY;
        x.i = (l < kThreads / 32) ? si[l] : INT64_MAX;
        for (int off = 16; off > 0; off >>= 1) {
            ArgMax o;
            o.v = __shfl_down_sync(0xffffffffu, x.v, off);
            o.i = __shfl_down_sync(0xffffffffu, x.i, off);
            x = amax(x, o);
        }
        if (l == 0) {
            sv[0] = x.v;
            si[0] = x.i;
        }
    }
    __syncthreads();
    ArgMax r{sv[0], si[0]};
    __syncthreads();
    return r;
}

// d_j = H_jj = h[2j] for j >= j0 (excluded indices get -inf); publish block argmax.
__global__ void __launch_bounds__(kThreads) pchol_init(const double* __restrict__ h, int64_t n,
                                                       int64_t j0, const double* __restrict__ w,
                                                       double* __restrict__ d,
                                                       ArgMax* __restrict__ part) {
    ArgMax best{-INFINITY, INT64_MAX};
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * kThreads) {
        double v = (j >= j0) ? h[2 * j] * (w ? w[j] * w[j] : 1.0) : -INFINITY;
        d[j] = v;
        best = amax(best, ArgMax{v, j});
    }
    best = block_argmax(best);
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

__global__ void __launch_bounds__(kThreads) pchol_step(
    const double* __restrict__ h, int64_t n, int64_t j0, const double* __restrict__ w, double tol,
    int r, double* __restrict__ u, int64_t* __restrict__ piv, double* __restrict__ d,
    const ArgMax* __restrict__ part_in, ArgMax* __restrict__ part_out, int nparts,
    State* __restrict__ st) {
    __shared__ double s_up[kKmaxShared];
    __shared__ double s_a;
    if (st->done) return;
    // every block reduces the same partials: identical pivot and decision everywhere
    ArgMax best{-INFINITY, INT64_MAX};
    for (int i = threadIdx.x; i < nparts; i += kThreads) best = amax(best, part_in[i]);
    best = block_argmax(best);
    double thresh = (r == 0) ? tol * best.v : st->thresh;
    if (r == 0 && blockIdx.x == 0 && threadIdx.x == 0) st->thresh = thresh;
    const int64_t p = best.i;
    if (!(best.v > thresh) || p < j0 || p >= n) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->K = r;
            st->done = 1;
        }
        return;
    }
    for (int i = threadIdx.x; i < r; i += kThreads) s_up[i] = u[(int64_t)i * n + p];
    __syncthreads();
    const double wp = w ? w[p] : 1.0;
    if (threadIdx.x == 0) {
        double a = h[2 * p] * wp * wp;
        for (int i = 0; i < r; ++i) a -= s_up[i] * s_up[i];
        s_a = a;
    }
    __syncthreads();
    const double a = s_a;
    if (!(a > thresh)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->K = r;
            st->done = 1;
        }
        return;
    }
    const double inv = 1.0 / sqrt(a);
    ArgMax nb{-INFINITY, INT64_MAX};
    double* ur = u + (int64_t)r * n;
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * kThreads) {
        double val = 0.0;
        double dj = -INFINITY;
        if (j >= j0) {
            double c = h[j + p] * (w ? w[j] * wp : 1.0);
            for (int i = 0; i < r; ++i) c -= u[(int64_t)i * n + j] * s_up[i];
            val = c * inv;
            dj = d[j] - val * val;
            d[j] = dj;
        }
        ur[j] = val;
        nb = amax(nb, ArgMax{dj, j});
    }
    nb = block_argmax(nb);
    if (threadIdx.x == 0) part_out[blockIdx.x] = nb;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        piv[r] = p;
        st->K = r + 1;
    }
}

}  // namespace

int pchol_run(const double* h, const double* w, int64_t n, int64_t j0, double tol, int64_t kmax,
              double* u, int64_t* pivots, int64_t* K, cudaStream_t s) {
    if (kmax > kKmaxShared) kmax = kKmaxShared;
    if (kmax > n - j0) kmax = n - j0;
    int nblk = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 4 * (int64_t)sm_count());
    if (nblk < 1) nblk = 1;
    double* d = nullptr;
    ArgMax* part = nullptr;
    State* st = nullptr;
    int rc = TDH_OK;
    State host{0.0, 0, 0};
    if ((rc = dev_alloc_t(&d, (size_t)n)) != TDH_OK) goto done;
    if ((rc = dev_alloc_t(&part, (size_t)2 * nblk)) != TDH_OK) goto done;
    if ((rc = dev_alloc_t(&st, 1)) != TDH_OK) goto done;
    {
        cudaError_t e = cudaMemsetAsync(st, 0, sizeof(State), s);
        if (e == cudaSuccess) {
            pchol_init<<<nblk, kThreads, 0, s>>>(h, n, j0, w, d, part);
            e = cudaGetLastError();
        }
        for (int64_t r = 0; e == cudaSuccess && r < kmax; ++r) {
            pchol_step<<<nblk, kThreads, 0, s>>>(h, n, j0, w, tol, (int)r, u, pivots, d,
                                                 part + (r & 1) * nblk,
                                                 part + ((r + 1) & 1) * nblk, nblk, st);
            e = cudaGetLastError();
            if (e == cudaSuccess && ((r & 7) == 7 || r + 1 == kmax)) {
                e = cudaMemcpyAsync(&host, st, sizeof(State), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e == cudaSuccess && host.done) break;
            }
        }
        if (e == cudaSuccess) {
            e = cudaMemcpyAsync(&host, st, sizeof(State), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        if (e != cudaSuccess) {
            set_error("pivoted Cholesky: %s", cudaGetErrorString(e));
            rc = TDH_ERR_CUDA;
        }
    }
    if (rc == TDH_OK) *K = host.K;
done:
    if (d || part || st) cudaStreamSynchronize(s);
    dev_free(d);
    dev_free(part);
    dev_free(st);
    return rc;
}

// ----------------------------------------------------------------------------------------
// Accuracy-targeted truncation.  The residual R = H - sum_{r<K} u_r u_r^T of a pivoted
// Cholesky of a positive semidefinite H is positive semidefinite (a Schur complement), so each
// 2 x 2 principal minor gives |R_jk| <= sqrt(d_j d_k) with d = diag(R).  In A = D1 (T o H) D2
// the truncation error is then |(A - A_K)_jk| <= max|t| |D1_j| sqrt(d_j) |D2_k| sqrt(d_k), and
// max |beta_K - beta| <= B(K) ||alpha||_1 with B(K) = max|t| max_j |D1_j| sqrt(d_j)
// max_k |D2_k| sqrt(d_k).  One pass over j evaluates B for every prefix K' <= K.
namespace {

// Non-negative doubles order like their bit patterns: atomicMax on the bits.
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* m, double v) {
    atomicMax(m, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v) {
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// m[0] = max|t|; m[1 + k] = max_j |D1_j| sqrt(d_j^(k)), m[2 + K + k] = max_j |D2_j| sqrt(d_j^(k))
// for k = 0..K (d^(k): residual diagonal after k steps, indices j >= j0).
__global__ void __launch_bounds__(kThreads) k_trunc_bound(
    const double* __restrict__ h, const double* __restrict__ u, int64_t n, int64_t j0, int K,
    const double* __restrict__ t, const double* __restrict__ d1, const double* __restrict__ d2,
    const double* __restrict__ so, const double* __restrict__ si, const double* __restrict__ w,
    unsigned long long* __restrict__ m) {
    const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool in = j < n;
    const bool blk = in && j >= j0;
    const int lane = threadIdx.x & 31;
    const double tm = warp_max(in ? fabs(t[j]) : 0.0);
    if (lane == 0) atomic_max_nonneg(&m[0], tm);
    const double wj = (blk && w) ? w[j] : 1.0;
    const double a1 = blk ? fabs(d1[j] * (so ? so[j] : 1.0)) / wj : 0.0;
    const double a2 = blk ? fabs(d2[j] * (si ? si[j] : 1.0)) / wj : 0.0;
    double dj = blk ? h[2 * j] * wj * wj : 0.0;
    for (int k = 0; k <= K; ++k) {
        const double sq = sqrt(fmax(dj, 0.0));
        const double v1 = warp_max(a1 * sq), v2 = warp_max(a2 * sq);
        if (lane == 0) {
            atomic_max_nonneg(&m[1 + k], v1);
            atomic_max_nonneg(&m[2 + K + k], v2);
        }
        if (k < K && blk) {
            const double x = u[(int64_t)k * n + j];
            dj -= x * x;
        }
    }
}

// w_j = sqrt(|D1_j D2_j|) (with the step's scalings), 1 where that is 0 or not finite.
__global__ void k_pivot_weights(const double* __restrict__ d1, const double* __restrict__ d2,
                                const double* __restrict__ so, const double* __restrict__ si,
                                int64_t n, double* __restrict__ w) {
    const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (j >= n) return;
    const double v = sqrt(fabs(d1[j] * (so ? so[j] : 1.0) * d2[j] * (si ? si[j] : 1.0)));
    w[j] = (v > 0.0 && isfinite(v)) ? v : 1.0;
}

// u[r][j] /= w_j: factors of W H W -> factors of H
__global__ void k_unweight(double* __restrict__ u, const double* __restrict__ w, int64_t K,
                           int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i < K * n) u[i] /= w[i % n];
}

}  // namespace

int pchol_weights(const double* d1, const double* d2, const double* so, const double* si,
                  int64_t n, double* w, cudaStream_t s) {
    k_pivot_weights<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(d1, d2, so, si,
                                                                                  n, w);
    TDH_CUDA(cudaGetLastError());
    return TDH_OK;
}

int pchol_unweight(double* u, const double* w, int64_t K, int64_t n, cudaStream_t s) {
    if (K <= 0) return TDH_OK;
    k_unweight<<<(unsigned)((K * n + kThreads - 1) / kThreads), kThreads, 0, s>>>(u, w, K, n);
    TDH_CUDA(cudaGetLastError());
    return TDH_OK;
}

int pchol_truncate(const double* h, const double* w, const double* u, int64_t n, int64_t j0,
                   int64_t K, const double* t, const double* d1, const double* d2,
                   const double* so, const double* si, double target, int64_t* Kout,
                   double* bound, cudaStream_t s) {
    *Kout = K;
    if (K <= 0) return TDH_OK;
    const size_t words = 2 * (size_t)K + 3;
    unsigned long long* m = nullptr;
    TDH_TRY(dev_alloc_t(&m, words));
    std::vector<unsigned long long> host(words);
    cudaError_t e = cudaMemsetAsync(m, 0, sizeof(unsigned long long) * words, s);
    if (e == cudaSuccess) {
        const unsigned blocks = (unsigned)((n + kThreads - 1) / kThreads);
        k_trunc_bound<<<blocks, kThreads, 0, s>>>(h, u, n, j0, (int)K, t, d1, d2, so, si, w, m);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host.data(), m, sizeof(unsigned long long) * words,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(m);
    if (e != cudaSuccess) {
        set_error("truncation bound: %s", cudaGetErrorString(e));
        return TDH_ERR_CUDA;
    }
    auto as_d = [&](size_t i) {
        double v;
        std::memcpy(&v, &host[i], sizeof(double));
        return v;
    };
    const double tmax = as_d(0);
    for (int64_t k = 0; k <= K; ++k) {
        const double b = tmax * as_d(1 + (size_t)k) * as_d(2 + (size_t)K + (size_t)k);
        if (bound) *bound = b;
        if (b <= target) {
            *Kout = k;
            return TDH_OK;
        }
    }
    return TDH_OK;
}

}  // namespace tdh

extern "C" int tdh_pchol(const double* h, int64_t n, int64_t j0, double tol, int64_t kmax,
                         double* u, int64_t* pivots, int64_t* K, void* stream) {
    tdh::clear_error();
    if (n < 1 || (j0 != 0 && j0 != 1) || j0 >= n || !(tol > 0.0) || kmax < 1 || !h || !u ||
        !pivots || !K) {
        tdh::set_error("tdh_pchol: need n >= 1, j0 in {0,1} < n, tol > 0, kmax >= 1, non-NULL");
        return TDH_ERR_INVALID_ARG;
    }
    return tdh::pchol_run(h, nullptr, n, j0, tol, kmax, u, pivots, K, tdh::as_stream(stream));
}

// ----------------------------------------------------------------------------------------
// Allocation-free pivoted Cholesky.
//
// Some callers cannot call cudaMalloc at all: code that runs while a caching allocator owns
// the device memory and forbids outside allocations, or inside allocation-free real-time
// sections.  This variant runs the same kernels as tdh_pchol but takes its scratch (the
// residual diagonal, the per-block argmax partials and the stop state) from one statically
// sized device array that lives in this file.  The array is part of the library image: every
// GPU that loads the library holds it until the process exits.
//
// Every call looks up the array's device address for the current device with
// cudaGetSymbolAddress (a lookup, not an allocation) and passes it to the kernels, so the
// address is always the one of the current context.  All calls on a device share the one
// array and it keeps the contents of the last call: the state words that must start at zero
// are cleared by every call, the rest is fully rewritten.  Two calls whose work overlaps on
// the GPU (different streams, or different host threads) race on the array; serialise them.
// Each call synchronises `stream` (it reads the stop state back every few steps).
namespace tdh {
namespace {

constexpr int64_t kNoAllocMaxN = 65536;
constexpr int kNoAllocMaxParts = (int)((kNoAllocMaxN + kThreads - 1) / kThreads);
constexpr size_t kNoAllocDBytes = sizeof(double) * (size_t)kNoAllocMaxN;
constexpr size_t kNoAllocPartBytes = sizeof(ArgMax) * 2 * (size_t)kNoAllocMaxParts;
constexpr size_t kNoAllocBytes = kNoAllocDBytes + kNoAllocPartBytes + 256;

static __device__ __align__(256) unsigned char g_pchol_scratch[kNoAllocBytes];

int noalloc_scratch(unsigned char** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_pchol_scratch);
    if (e != cudaSuccess || !p) {
        set_error("tdh_pchol_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return TDH_ERR_CUDA;
    }
    *out = static_cast<unsigned char*>(p);
    return TDH_OK;
}

}  // namespace
}  // namespace tdh

extern "C" int tdh_pchol_noalloc(const double* h, int64_t n, int64_t j0, double tol,
                                 int64_t kmax, double* u, int64_t* pivots, int64_t* K,
                                 void* stream) {
    using namespace tdh;
    clear_error();
    if (n < 1 || (j0 != 0 && j0 != 1) || j0 >= n || !(tol > 0.0) || kmax < 1 || !h || !u ||
        !pivots || !K) {
        set_error("tdh_pchol_noalloc: need n >= 1, j0 in {0,1} < n, tol > 0, kmax >= 1, non-NULL");
        return TDH_ERR_INVALID_ARG;
    }
    if (n > kNoAllocMaxN) {
        set_error("tdh_pchol_noalloc: n = %lld exceeds the static scratch limit of %lld "
                  "coefficients; use tdh_pchol", (long long)n, (long long)kNoAllocMaxN);
        return TDH_ERR_INVALID_ARG;
    }
    unsigned char* base = nullptr;
    TDH_TRY(noalloc_scratch(&base));
    cudaStream_t s = as_stream(stream);
    double* d = reinterpret_cast<double*>(base);
    ArgMax* part = reinterpret_cast<ArgMax*>(base + kNoAllocDBytes);
    State* st = reinterpret_cast<State*>(base + kNoAllocDBytes + kNoAllocPartBytes);
    if (kmax > kKmaxShared) kmax = kKmaxShared;
    if (kmax > n - j0) kmax = n - j0;
    // the same grid as tdh_pchol (at most 4 blocks per SM), within the array's partials
    int nblk = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 4 * (int64_t)sm_count());
    if (nblk < 1) nblk = 1;
    State host{0.0, 0, 0};
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(State), s);
    if (e == cudaSuccess) {
        pchol_init<<<nblk, kThreads, 0, s>>>(h, n, j0, nullptr, d, part);
        e = cudaGetLastError();
    }
    for (int64_t r = 0; e == cudaSuccess && r < kmax; ++r) {
        pchol_step<<<nblk, kThreads, 0, s>>>(h, n, j0, nullptr, tol, (int)r, u, pivots, d,
                                             part + (r & 1) * nblk, part + ((r + 1) & 1) * nblk,
                                             nblk, st);
        e = cudaGetLastError();
        if (e == cudaSuccess && ((r & 7) == 7 || r + 1 == kmax)) {
            e = cudaMemcpyAsync(&host, st, sizeof(State), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e == cudaSuccess && host.done) break;
        }
    }
    if (e == cudaSuccess) {
        e = cudaMemcpyAsync(&host, st, sizeof(State), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        set_error("tdh_pchol_noalloc: %s", cudaGetErrorString(e));
        return TDH_ERR_CUDA;
    }
    *K = host.K;
    return TDH_OK;
}
