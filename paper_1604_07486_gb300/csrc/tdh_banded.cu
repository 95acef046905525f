// Case 1 of the ultraspherical conversion (Sec. 5.2): when l2 - l1 = M is a positive integer,
// A = P_N S_{l2-1} ... S_{l1+1} S_{l1} P_N^T (eq. (sparseFactorization)) with
//   (S_l c)_j = a_j c_j - a_{j+2} c_{j+2},   a_j = l/(l+j),
// an O(n) product: no plan factors, no FFT.  The coefficients a_j of every factor are a plan
// table (float64 arithmetic, rounded once), so the kernels do no division.  The transpose
// (for reverse-mode use) is (S_l^T g)_k = a_k (g_k - g_{k-2}), applied in the opposite
// factor order.
//
// One factor, float32, rows of a multiple of 4: a streaming kernel, one float4 of a vector per
// thread (its neighbour's float4 supplies c_{j+2} from cache).  Otherwise each block stages a
// tile plus a halo of 2M coefficients in shared memory and applies the M factors in turn.
// Either way the work is ~3 flops per 8 bytes moved: bound by HBM.
#include "tdh_internal.cuh"

namespace tdh {
namespace {

constexpr int kBandThreads = 256;
constexpr int kBandTile = 2048;
constexpr int kBandMaxM = 16;

template <typename T>
__global__ void __launch_bounds__(kBandThreads) banded_kernel(const T* __restrict__ in,
                                                              T* __restrict__ out, int64_t n,
                                                              const T* __restrict__ coef, int M,
                                                              int adjoint) {
    __shared__ T buf[2][kBandTile + 2 * kBandMaxM];
    const int64_t vec = blockIdx.y;
    const int64_t j0 = (int64_t)blockIdx.x * kBandTile;
    const T* x = in + vec * n;
    T* y = out + vec * n;
    const int W = kBandTile + 2 * M;  // staged width
    // forward: stage [j0, j0 + W); adjoint: stage [j0 - 2M, j0 + T)
    const int64_t base = adjoint ? j0 - 2 * M : j0;
    for (int i = threadIdx.x; i < W; i += kBandThreads) {
        const int64_t j = base + i;
        buf[0][i] = (j >= 0 && j < n) ? x[j] : T(0);
    }
    __syncthreads();
    int cur = 0;
    for (int f = 0; f < M; ++f) {
        // forward applies S_{l0}, S_{l0+1}, ...; the adjoint applies the transposes in reverse
        const T* a = coef + (int64_t)(adjoint ? M - 1 - f : f) * (n + 2);
        for (int i = threadIdx.x; i < W; i += kBandThreads) {
            const int64_t j = base + i;
            T v = T(0);
            if (j >= 0 && j < n) {
                if (!adjoint) {
                    const T c2 = (i + 2 < W && j + 2 < n) ? buf[cur][i + 2] : T(0);
                    v = a[j] * buf[cur][i] - a[j + 2] * c2;
                } else {
                    const T g2 = (i >= 2 && j >= 2) ? buf[cur][i - 2] : T(0);
                    v = a[j] * (buf[cur][i] - g2);
                }
            }
            buf[cur ^ 1][i] = v;
        }
        __syncthreads();
        cur ^= 1;
    }
    const int off = adjoint ? 2 * M : 0;
    for (int i = threadIdx.x; i < kBandTile; i += kBandThreads) {
        const int64_t j = j0 + i;
        if (j < n) y[j] = buf[cur][i + off];
    }
}

// One factor, float32, n % 4 == 0, 16-byte aligned rows: chunk c = 4 coefficients.
__global__ void __launch_bounds__(kBandThreads) banded1_f4(const float4* __restrict__ in,
                                                           float4* __restrict__ out, int64_t nq,
                                                           int64_t total, const float4* __restrict__ a4,
                                                           int adjoint) {
    const int64_t c = (int64_t)blockIdx.x * kBandThreads + threadIdx.x;
    if (c >= total) return;
    const int64_t q = c % nq;  // chunk within its vector
    const float4 x = in[c];
    const float4 a = a4[q];
    float4 r;
    if (!adjoint) {
        const bool last = q + 1 == nq;
        const float4 xn = last ? make_float4(0.f, 0.f, 0.f, 0.f) : in[c + 1];
        const float4 an = last ? make_float4(0.f, 0.f, 0.f, 0.f) : a4[q + 1];
        r.x = a.x * x.x - a.z * x.z;
        r.y = a.y * x.y - a.w * x.w;
        r.z = a.z * x.z - an.x * xn.x;
        r.w = a.w * x.w - an.y * xn.y;
    } else {
        const float4 xp = q == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : in[c - 1];
        r.x = a.x * (x.x - xp.z);
        r.y = a.y * (x.y - xp.w);
        r.z = a.z * (x.z - x.x);
        r.w = a.w * (x.w - x.y);
    }
    out[c] = r;
}

// coef[f][j] = l_f / (l_f + j), l_f = lam0 + f, j < n + 2 (float64, rounded once)
template <typename T>
__global__ void banded_coef(T* __restrict__ coef, int64_t n2, double lam0, int M) {
    const int64_t i = (int64_t)blockIdx.x * kBandThreads + threadIdx.x;
    if (i >= n2 * M) return;
    const int f = (int)(i / n2);
    const int64_t j = i % n2;
    const double l = lam0 + f;
    coef[i] = (T)(l / (l + (double)j));
}

}  // namespace

int banded_prepare(int prec, int64_t n, double lam0, int M, void** coef, cudaStream_t s) {
    if (M < 1 || M > kBandMaxM) {
        set_error("banded conversion supports 1..%d factors (got %d)", kBandMaxM, M);
        return TDH_ERR_UNSUPPORTED;
    }
    const size_t esz = prec == TDH_FP32 ? 4 : 8;
    const int64_t n2 = n + 2;
    // float4 rows of the table need 16-byte alignment: pad each factor's row
    TDH_TRY(dev_alloc(coef, esz * (size_t)n2 * M + 16));
    const unsigned blocks = (unsigned)((n2 * M + kBandThreads - 1) / kBandThreads);
    if (prec == TDH_FP32)
        banded_coef<float><<<blocks, kBandThreads, 0, s>>>(static_cast<float*>(*coef), n2, lam0, M);
    else
        banded_coef<double><<<blocks, kBandThreads, 0, s>>>(static_cast<double*>(*coef), n2, lam0, M);
    TDH_CUDA(cudaGetLastError());
    return TDH_OK;
}

int banded_launch(int prec, const void* in, void* out, int64_t n, int64_t batch, const void* coef,
                  int M, int adjoint, cudaStream_t s) {
    if (M < 1 || M > kBandMaxM) {
        set_error("banded conversion supports 1..%d factors (got %d)", kBandMaxM, M);
        return TDH_ERR_UNSUPPORTED;
    }
    const bool f4 = prec == TDH_FP32 && M == 1 && n % 4 == 0 &&
                    (reinterpret_cast<uintptr_t>(in) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    if (f4) {
        const int64_t total = batch * (n / 4);
        const unsigned blocks = (unsigned)((total + kBandThreads - 1) / kBandThreads);
        banded1_f4<<<blocks, kBandThreads, 0, s>>>(static_cast<const float4*>(in),
                                                   static_cast<float4*>(out), n / 4, total,
                                                   static_cast<const float4*>(coef), adjoint);
        TDH_CUDA(cudaGetLastError());
        return TDH_OK;
    }
    if (batch > 65535) {
        set_error("banded conversion: batch above 65535 per launch");
        return TDH_ERR_UNSUPPORTED;
    }
    dim3 grid((unsigned)((n + kBandTile - 1) / kBandTile), (unsigned)batch);
    if (prec == TDH_FP32)
        banded_kernel<float><<<grid, kBandThreads, 0, s>>>(static_cast<const float*>(in),
                                                            static_cast<float*>(out), n,
                                                            static_cast<const float*>(coef), M,
                                                            adjoint);
    else
        banded_kernel<double><<<grid, kBandThreads, 0, s>>>(static_cast<const double*>(in),
                                                             static_cast<double*>(out), n,
                                                             static_cast<const double*>(coef), M,
                                                             adjoint);
    TDH_CUDA(cudaGetLastError());
    return TDH_OK;
}

}  // namespace tdh
