// Case 1 of the ultraspherical conversion (Sec. 5.2): when l2 - l1 = M is a positive integer,
// A = P_N S_{l2-1} ... S_{l1+1} S_{l1} P_N^T (eq. (sparseFactorization)) with
//   (S_l c)_j = l/(l+j) c_j - l/(l+j+2) c_{j+2},
// an O(n) product: no plan factors, no FFT.  Each block converts one tile of one vector: it
// stages the tile plus a halo of 2M coefficients in shared memory and applies the M factors
// in turn.  The transpose (for reverse-mode use) is (S_l^T g)_k = l/(l+k) (g_k - g_{k-2}),
// applied in the opposite factor order with the halo below the tile.
//
// The work is 2 loads/stores and ~3 flops per coefficient per factor: bound by HBM.
#include "tdh_internal.cuh"

namespace tdh {
namespace {

constexpr int kBandThreads = 256;
constexpr int kBandTile = 2048;
constexpr int kBandMaxM = 16;

template <typename T>
__global__ void __launch_bounds__(kBandThreads) banded_kernel(const T* __restrict__ in,
                                                              T* __restrict__ out, int64_t n,
                                                              double lam0, int M, int adjoint) {
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
        const T lam = (T)(adjoint ? lam0 + (M - 1 - f) : lam0 + f);
        for (int i = threadIdx.x; i < W; i += kBandThreads) {
            const int64_t j = base + i;
            T v = T(0);
            if (j >= 0 && j < n) {
                if (!adjoint) {
                    const T c2 = (i + 2 < W && j + 2 < n) ? buf[cur][i + 2] : T(0);
                    v = lam / (lam + (T)j) * buf[cur][i] - lam / (lam + (T)(j + 2)) * c2;
                } else {
                    const T g2 = (i >= 2 && j >= 2) ? buf[cur][i - 2] : T(0);
                    v = lam / (lam + (T)j) * (buf[cur][i] - g2);
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

}  // namespace

int banded_launch(int prec, const void* in, void* out, int64_t n, int64_t batch, double lam0,
                  int M, int adjoint, cudaStream_t s) {
    if (M < 1 || M > kBandMaxM) {
        set_error("banded conversion supports 1..%d factors (got %d)", kBandMaxM, M);
        return TDH_ERR_UNSUPPORTED;
    }
    if (batch > 65535) {
        set_error("banded conversion: batch above 65535 per launch");
        return TDH_ERR_UNSUPPORTED;
    }
    dim3 grid((unsigned)((n + kBandTile - 1) / kBandTile), (unsigned)batch);
    if (prec == TDH_FP32)
        banded_kernel<float><<<grid, kBandThreads, 0, s>>>(static_cast<const float*>(in),
                                                            static_cast<float*>(out), n, lam0, M,
                                                            adjoint);
    else
        banded_kernel<double><<<grid, kBandThreads, 0, s>>>(static_cast<const double*>(in),
                                                             static_cast<double*>(out), n, lam0,
                                                             M, adjoint);
    TDH_CUDA(cudaGetLastError());
    return TDH_OK;
}

}  // namespace tdh
