// Case 1 of the ultraspherical (Sec. 5.2) and Jacobi (Sec. 5.3) conversions: when the two
// parameters differ by an integer, A is a product of sparse upper-triangular factors, each
// applied in O(n) (Eq. (12) and its Jacobi analogue).  A factor is
//   (S c)_j = p_j c_j + q_j c_{j+off}
// with
//   ultraspherical S_l (C^(l) -> C^(l+1)), off = 2:  p_j = l/(l+j),  q_j = -l/(l+j+2);
//   Jacobi S_(a,b) ((a,b) -> (a+1,b)), off = 1:
//       p_0 = 1,  p_j = (j+a+b+1)/(2j+a+b+1),  q_j = -(j+b+1)/(2j+a+b+3)
// (the superdiagonal numerator is j+b+1: that is what the exact conversion gives; the form
// with j+a+1 is the factor for raising b, up to sign).  Inside a reflected part of a Jacobi
// chain each factor is conjugated by diag((-1)^k), which negates q.  A step to a smaller
// parameter applies the inverses: S x = c is solved by back-substitution (Sec. 5.2, 5.3:
// "backward substitution"),
//   x_j = rho_j c_j + mu_j x_{j+off},   rho_j = 1/p_j,  mu_j = -q_j/p_j,
// a first-order linear recurrence.  On the GPU it is a scan of affine maps x -> m x + b
// (the multipliers kept as logs, so long products do not drift):
// each block reduces a tile of coefficients to one map per chain, a second kernel
// scans the tile maps of each vector, a third replays each tile from its carried-in value.
// The transposes (reverse mode) are (S^T g)_k = p_k g_k + q_{k-off} g_{k-off} and, for the
// inverse, the same recurrence run upward with mu'_k = -q_{k-off}/p_k.
//
// Diagonal scalings out = diag(s) A diag(sigma) (the Chebyshev normalisation of jac2cheb /
// cheb2jac) fold into the tables of the last / first factor.  Tables are float64 closed
// forms rounded once to the execute precision, so the kernels do no division.  All of this
// is ~3 flops per 8 bytes moved: bound by HBM.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "tdh_internal.cuh"

namespace tdh {
namespace {

constexpr int kThreads = 256;
constexpr int kTile = 2048;     // forward factors: coefficients per block
constexpr int kMaxM = 16;       // factors per step
constexpr int kInvRows = 5;     // table rows of an inverse factor
// back-substitution: E coefficients per thread (a tile of 4096 floats or 2048 doubles; the
// three staged arrays take 50 KB of dynamic shared memory), one padding slot per 128 bytes
template <typename T>
struct Scan {
    static constexpr int E = 64 / (int)sizeof(T);
    static constexpr int tile = kThreads * E;
    static constexpr int per_pad = 128 / (int)sizeof(T);
    static constexpr int smem = tile + tile / per_pad;
};

struct FactorSpec {
    int family;    // SP_ULTRA, SP_JACOBI, SP_IDENTITY
    int off;
    int M;
    int inverse;
    int flip;
    double par0, dir, b;
    int64_t n, ld;
};

__device__ void factor_pq(const FactorSpec& F, double par, int64_t j, double* p, double* q) {
    const double x = (double)j;
    if (F.family == SP_ULTRA) {
        *p = par / (par + x);
        *q = -par / (par + x + 2.0);
    } else if (F.family == SP_JACOBI) {
        const double s = par + F.b;
        *p = j == 0 ? 1.0 : (x + s + 1.0) / (2.0 * x + s + 1.0);
        *q = -(x + F.b + 1.0) / (2.0 * x + s + 3.0);
        if (F.flip) *q = -*q;
    } else {
        *p = 1.0;
        *q = 0.0;
    }
}

// 1 - mu_j for the downward recurrence (mu_j = -q_j/p_j) and 1 - mu'_k for the upward one
// (mu'_k = -q_{k-off}/p_k) of an unflipped, unscaled factor, in closed form (no cancellation
// near 1):  ultraspherical  1 - mu_j = 2/(l+j+2),  mu'_k = 1;
//           Jacobi          1 - mu_j = (2j(a+1) + (a+b+1)(a+2)) / ((2j+a+b+3)(j+a+b+1)),
//                           1 - mu_0 = (a+2)/(a+b+3),  1 - mu'_k = (a+1)/(k+a+b+1).
__device__ double delta_down(const FactorSpec& F, double par, int64_t j) {
    const double x = (double)j;
    if (F.family == SP_ULTRA) return 2.0 / (par + x + 2.0);
    if (F.family == SP_JACOBI) {
        const double a = par, s = par + F.b;
        if (j == 0) return (a + 2.0) / (s + 3.0);
        return (2.0 * x * (a + 1.0) + (s + 1.0) * (a + 2.0)) / ((2.0 * x + s + 3.0) * (x + s + 1.0));
    }
    return 1.0;
}

__device__ double delta_up(const FactorSpec& F, double par, int64_t k) {
    if (F.family == SP_ULTRA) return 0.0;
    if (F.family == SP_JACOBI) return (par + 1.0) / ((double)k + par + F.b + 1.0);
    return 1.0;
}

// forward: tab[f][0][j] = s_j p_j sigma_j, tab[f][1][j] = s_j q_j sigma_{j+off};
// inverse (tables of the unflipped factor; a flip is applied as signs by the kernels):
//   tab[f][0][j] = rho_j = s_j sigma_j / p_j,
//   tab[f][1][j] = delta_j = 1 - mu_j s_j / s_{j+off}  (downward recurrence, 1 past the end),
//   tab[f][2][j] = log(1 - delta_j)                       (-inf where the multiplier is 0),
//   tab[f][3][k] = 1 - mu'_k sigma_k / sigma_{k-off}    (upward recurrence, 1 for k < off),
//   tab[f][4][k] = its log;
// with a scale ratio r, 1 - mu r = (1 - r) + (1 - mu) r.  Every multiplier is positive.
// s = sout on the last factor, sigma = sin on the first, 1 elsewhere; zero for j >= n.
template <typename T>
__global__ void k_sparse_tables(FactorSpec F, const double* __restrict__ sout,
                                const double* __restrict__ sin, T* __restrict__ tab) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= F.ld * F.M) return;
    const int f = (int)(i / F.ld);
    const int64_t j = i % F.ld;
    const int rows = F.inverse ? kInvRows : 2;
    T* t = tab + (int64_t)f * rows * F.ld;
    if (j >= F.n) {
        for (int r = 0; r < rows; ++r) t[r * F.ld + j] = T(0);
        return;
    }
    const double par = F.par0 + F.dir * (double)f;
    const double* so = (f == F.M - 1) ? sout : nullptr;
    const double* si = (f == 0) ? sin : nullptr;
    auto S = [&](int64_t k) { return so ? so[k] : 1.0; };
    auto G = [&](int64_t k) { return si ? si[k] : 1.0; };
    double p, q;
    if (!F.inverse) {
        factor_pq(F, par, j, &p, &q);
        const bool up = j + F.off < F.n;
        t[j] = (T)(S(j) * p * G(j));
        t[F.ld + j] = up ? (T)(S(j) * q * G(j + F.off)) : T(0);
        return;
    }
    FactorSpec U = F;
    U.flip = 0;
    factor_pq(U, par, j, &p, &q);
    t[j] = (T)(S(j) * G(j) / p);
    double dn = 1.0, du = 1.0;
    if (j + F.off < F.n) {
        dn = delta_down(U, par, j);
        if (so) {
            const double r = S(j) / S(j + F.off);
            dn = (1.0 - r) + dn * r;
        }
    }
    if (j >= F.off) {
        du = delta_up(U, par, j);
        if (si) {
            const double r = G(j) / G(j - F.off);
            du = (1.0 - r) + du * r;
        }
    }
    t[F.ld + j] = (T)dn;
    t[2 * F.ld + j] = (T)log1p(-dn);
    t[3 * F.ld + j] = (T)du;
    t[4 * F.ld + j] = (T)log1p(-du);
}

// ---------------------------------------------------------------- forward factors

// Halo of each tile for an in-place step: the OFF*M coefficients after the tile (forward) or
// before it (transpose), saved before any block overwrites them.
template <typename T>
__global__ void k_halo_save(const T* __restrict__ x, T* __restrict__ halo, int64_t n,
                            int64_t ntiles, int H, int adjoint, int64_t total) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= total) return;
    const int64_t vt = i / H;
    const int e = (int)(i % H);
    const int64_t v = vt / ntiles, t = vt % ntiles;
    const int64_t j = adjoint ? t * kTile - H + e : (t + 1) * kTile + e;
    halo[i] = (j >= 0 && j < n) ? x[v * n + j] : T(0);
}

// Each block stages a tile plus a halo of OFF*M coefficients in shared memory and applies
// the M factors in turn (the halo shrinks by OFF per factor, so the tile stays exact).
template <typename T, int OFF>
__global__ void __launch_bounds__(kThreads) k_fwd_tile(const T* in, T* out, int64_t n,
                                                       int64_t ntiles, const T* __restrict__ tab,
                                                       int64_t ld, int M, int adjoint,
                                                       const T* __restrict__ halo) {
    __shared__ T buf[2][kTile + OFF * kMaxM];
    const int64_t vec = blockIdx.x / ntiles;
    const int64_t tile = blockIdx.x % ntiles;
    const int64_t j0 = tile * kTile;
    const T* x = in + vec * n;
    const int H = OFF * M;
    const int W = kTile + H;
    const int64_t base = adjoint ? j0 - H : j0;
    const T* hv = halo ? halo + (vec * ntiles + tile) * H : nullptr;
    for (int i = threadIdx.x; i < W; i += kThreads) {
        const int64_t j = base + i;
        T v = T(0);
        if (j >= 0 && j < n) {
            const bool in_halo = adjoint ? i < H : i >= kTile;
            v = (hv && in_halo) ? hv[adjoint ? i : i - kTile] : x[j];
        }
        buf[0][i] = v;
    }
    __syncthreads();
    int cur = 0;
    for (int f = 0; f < M; ++f) {
        const int ff = adjoint ? M - 1 - f : f;
        const T* P = tab + (int64_t)(2 * ff) * ld;
        const T* Q = P + ld;
        for (int i = threadIdx.x; i < W; i += kThreads) {
            const int64_t j = base + i;
            T v = T(0);
            if (j >= 0 && j < n) {
                if (!adjoint) {
                    const T c2 = (i + OFF < W) ? buf[cur][i + OFF] : T(0);
                    v = P[j] * buf[cur][i] + Q[j] * c2;
                } else {
                    const T g2 = (i >= OFF && j >= OFF) ? buf[cur][i - OFF] * Q[j - OFF] : T(0);
                    v = P[j] * buf[cur][i] + g2;
                }
            }
            buf[cur ^ 1][i] = v;
        }
        __syncthreads();
        cur ^= 1;
    }
    const int o = adjoint ? H : 0;
    T* y = out + vec * n;
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        const int64_t j = j0 + i;
        if (j < n) y[j] = buf[cur][i + o];
    }
}

// One factor, float32, n % 4 == 0, out of place: one float4 of a vector per thread, the
// neighbouring float4 supplies c_{j+off} (or g_{k-off}) from cache.
template <int OFF>
__global__ void __launch_bounds__(kThreads) k_fwd_f4(const float4* __restrict__ in,
                                                     float4* __restrict__ out, int64_t nq,
                                                     int64_t total, const float4* __restrict__ P4,
                                                     const float4* __restrict__ Q4, int adjoint) {
    const int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (c >= total) return;
    const int64_t q = c % nq;
    const float4 x = in[c];
    const float4 p = P4[q];
    float4 r;
    if (!adjoint) {
        const float4 qq = Q4[q];  // zero where j + off >= n
        const bool last = q + 1 == nq;
        const float4 xn = last ? make_float4(0.f, 0.f, 0.f, 0.f) : in[c + 1];
        if (OFF == 2) {
            r.x = p.x * x.x + qq.x * x.z;
            r.y = p.y * x.y + qq.y * x.w;
            r.z = p.z * x.z + qq.z * xn.x;
            r.w = p.w * x.w + qq.w * xn.y;
        } else {
            r.x = p.x * x.x + qq.x * x.y;
            r.y = p.y * x.y + qq.y * x.z;
            r.z = p.z * x.z + qq.z * x.w;
            r.w = p.w * x.w + qq.w * xn.x;
        }
    } else {
        const float4 qq = Q4[q];
        const bool first = q == 0;
        const float4 xp = first ? make_float4(0.f, 0.f, 0.f, 0.f) : in[c - 1];
        const float4 qp = first ? make_float4(0.f, 0.f, 0.f, 0.f) : Q4[q - 1];
        if (OFF == 2) {
            r.x = p.x * x.x + qp.z * xp.z;
            r.y = p.y * x.y + qp.w * xp.w;
            r.z = p.z * x.z + qq.x * x.x;
            r.w = p.w * x.w + qq.y * x.y;
        } else {
            r.x = p.x * x.x + qp.w * xp.w;
            r.y = p.y * x.y + qq.x * x.x;
            r.z = p.z * x.z + qq.y * x.y;
            r.w = p.w * x.w + qq.z * x.z;
        }
    }
    out[c] = r;
}

// ---------------------------------------------------------------- back-substitution

// Affine map x -> m x + b on each of the OFF interleaved chains, with the multiplier (always
// positive) kept as L = log m: composites add their logs, so a product over N positions
// carries O(log N) roundings.  Multiplying the rounded factors 1 - delta instead drifts by
// up to N ulp when the rounding errors are correlated, as they are for slowly varying
// multipliers near 1 (measured 5e-5 relative at n = 2^20 in float32).  Single positions use
// x - delta x, exact to the rounding of delta.
template <typename T, int OFF>
struct Aff {
    T L[OFF], b[OFF];
};

template <typename T, int OFF>
__device__ __forceinline__ Aff<T, OFF> aff_id() {
    Aff<T, OFF> r;
#pragma unroll
    for (int c = 0; c < OFF; ++c) {
        r.L[c] = T(0);
        r.b[c] = T(0);
    }
    return r;
}

// expm1(L) for |L| <= 1/2 by its Taylor series (float: degree 9, remainder below 2^-26 of
// the result); double uses the library function.
__device__ __forceinline__ float expm1_small(float L) {
    float t = 1.0f + L * (1.0f / 9.0f);
    t = 1.0f + L * (1.0f / 8.0f) * t;
    t = 1.0f + L * (1.0f / 7.0f) * t;
    t = 1.0f + L * (1.0f / 6.0f) * t;
    t = 1.0f + L * (1.0f / 5.0f) * t;
    t = 1.0f + L * (1.0f / 4.0f) * t;
    t = 1.0f + L * (1.0f / 3.0f) * t;
    t = 1.0f + L * 0.5f * t;
    return L * t;
}
__device__ __forceinline__ double expm1_small(double L) { return expm1(L); }

// exp(L) x: near m = 1 as x + expm1(L) x (relative accuracy of m - 1 kept)
template <typename T>
__device__ __forceinline__ T mul_m(T L, T x) {
    return L > T(-0.5) ? fma(expm1_small(L), x, x) : exp(L) * x;
}

// x first, then y
template <typename T, int OFF>
__device__ __forceinline__ Aff<T, OFF> aff_then(const Aff<T, OFF>& x, const Aff<T, OFF>& y) {
    Aff<T, OFF> r;
#pragma unroll
    for (int c = 0; c < OFF; ++c) {
        r.L[c] = x.L[c] + y.L[c];
        r.b[c] = mul_m(y.L[c], x.b[c]) + y.b[c];
    }
    return r;
}

template <typename T, int OFF>
__device__ __forceinline__ Aff<T, OFF> aff_shfl_up(const Aff<T, OFF>& v, int k) {
    Aff<T, OFF> r;
#pragma unroll
    for (int c = 0; c < OFF; ++c) {
        r.L[c] = __shfl_up_sync(0xffffffffu, v.L[c], k);
        r.b[c] = __shfl_up_sync(0xffffffffu, v.b[c], k);
    }
    return r;
}

// padded shared-memory slot: thread t reads slots E*t .. E*t+E-1 without bank conflicts
template <typename T>
__device__ __forceinline__ int spad(int i) { return i + i / Scan<T>::per_pad; }

// Exclusive block scan of the threads' maps (thread order); *total = all threads' map.
// warp_tot: [kThreads / 32 + 1] shared scratch.
template <typename T, int OFF>
__device__ Aff<T, OFF> block_exclusive(const Aff<T, OFF>& mine, Aff<T, OFF>* warp_tot,
                                       Aff<T, OFF>* total) {
    constexpr int NW = kThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Aff<T, OFF> inc = mine;
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const Aff<T, OFF> o = aff_shfl_up(inc, k);
        if (lane >= k) inc = aff_then(o, inc);
    }
    Aff<T, OFF> exl = aff_shfl_up(inc, 1);
    if (lane == 0) exl = aff_id<T, OFF>();
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        // exclusive scan of the warp totals by the first warp; the total goes to slot NW
        Aff<T, OFF> v = lane < NW ? warp_tot[lane] : aff_id<T, OFF>();
#pragma unroll
        for (int k = 1; k < NW; k <<= 1) {
            const Aff<T, OFF> o = aff_shfl_up(v, k);
            if (lane >= k) v = aff_then(o, v);
        }
        Aff<T, OFF> ex = aff_shfl_up(v, 1);
        if (lane == 0) ex = aff_id<T, OFF>();
        __syncwarp();
        if (lane < NW) warp_tot[lane] = ex;
        if (lane == NW - 1) warp_tot[NW] = v;
    }
    __syncthreads();
    if (total) *total = warp_tot[NW];
    return aff_then(warp_tot[warp], exl);
}

// Logical position l runs in recurrence order: physical index l (REV = 0, x_k depends on
// x_{k-off}) or n-1-l (REV = 1, x_j depends on x_{j+off}).  Stages b = rho * c (times
// (-1)^j for a factor conjugated by diag((-1)^k)), delta = 1 - multiplier and log(multiplier)
// of each position of the tile; positions past the end are identity maps.
template <typename T, int REV>
__device__ void scan_load(const T* x, int64_t n, int64_t l0, const T* __restrict__ rho,
                          const T* __restrict__ delta, const T* __restrict__ logm, int flip,
                          T* sb, T* sd, T* sl) {
    constexpr int IT = Scan<T>::tile / kThreads, BATCH = 8;
    static_assert(IT % BATCH == 0, "load batches");
#pragma unroll
    for (int i0 = 0; i0 < IT; i0 += BATCH) {
        // all loads of a batch first (independent, in flight together), then the stores
        T bv[BATCH], dv[BATCH], lv[BATCH];
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int i = threadIdx.x + (i0 + u) * kThreads;
            const int64_t l = l0 + i;
            bv[u] = T(0);
            dv[u] = T(0);
            lv[u] = T(0);
            if (l < n) {
                const int64_t j = REV ? n - 1 - l : l;
                bv[u] = rho[j] * x[j];
                if (flip && (j & 1)) bv[u] = -bv[u];
                dv[u] = delta[j];
                lv[u] = logm[j];
            }
        }
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int i = threadIdx.x + (i0 + u) * kThreads;
            sb[spad<T>(i)] = bv[u];
            sd[spad<T>(i)] = dv[u];
            sl[spad<T>(i)] = lv[u];
        }
    }
}

template <typename T, int OFF>
__device__ Aff<T, OFF> thread_map(const T* sb, const T* sd, const T* sl) {
    Aff<T, OFF> r = aff_id<T, OFF>();
#pragma unroll
    for (int e = 0; e < Scan<T>::E; ++e) {
        const int i = spad<T>(threadIdx.x * Scan<T>::E + e);
        const int c = e % OFF;
        r.L[c] += sl[i];
        r.b[c] = fma(-sd[i], r.b[c], r.b[c]) + sb[i];
    }
    return r;
}

// Kernel 1: the map of every tile (its chains' values at the tile end as functions of the
// values entering it).  sum: [batch * ntiles] maps.
template <typename T, int OFF, int REV>
__global__ void __launch_bounds__(kThreads) k_scan_tiles(const T* __restrict__ in, int64_t n,
                                                         int64_t ntiles, const T* __restrict__ rho,
                                                         const T* __restrict__ delta,
                                                         const T* __restrict__ logm, int flip,
                                                         Aff<T, OFF>* __restrict__ sum) {
    extern __shared__ __align__(16) unsigned char scan_smem[];
    T* sb = reinterpret_cast<T*>(scan_smem);
    T* sd = sb + Scan<T>::smem;
    T* sl = sd + Scan<T>::smem;
    __shared__ Aff<T, OFF> wt[kThreads / 32 + 1];
    const int64_t vec = blockIdx.x / ntiles, tile = blockIdx.x % ntiles;
    scan_load<T, REV>(in + vec * n, n, tile * Scan<T>::tile, rho, delta, logm, flip, sb, sd, sl);
    __syncthreads();
    const Aff<T, OFF> mine = thread_map<T, OFF>(sb, sd, sl);
    Aff<T, OFF> tot;
    block_exclusive<T, OFF>(mine, wt, &tot);
    if (threadIdx.x == 0) sum[blockIdx.x] = tot;
}

// Kernel 2: per vector, the values entering each tile (x = 0 before the first position).
template <typename T, int OFF>
__global__ void __launch_bounds__(kThreads) k_scan_carry(const Aff<T, OFF>* __restrict__ sum,
                                                         int64_t ntiles,
                                                         Aff<T, OFF>* __restrict__ carry) {
    __shared__ Aff<T, OFF> wt[kThreads / 32 + 1];
    const Aff<T, OFF>* s = sum + (int64_t)blockIdx.x * ntiles;
    Aff<T, OFF>* cr = carry + (int64_t)blockIdx.x * ntiles;
    const int64_t per = (ntiles + kThreads - 1) / kThreads;
    const int64_t t0 = std::min<int64_t>(ntiles, per * threadIdx.x);
    const int64_t t1 = std::min<int64_t>(ntiles, t0 + per);
    Aff<T, OFF> mine = aff_id<T, OFF>();
    for (int64_t t = t0; t < t1; ++t) mine = aff_then(mine, s[t]);
    Aff<T, OFF> run = block_exclusive<T, OFF>(mine, wt, nullptr);
    for (int64_t t = t0; t < t1; ++t) {
        cr[t] = run;  // entering values = run.b (run applied to 0)
        run = aff_then(run, s[t]);
    }
}

// Kernel 3: replay each tile from its entering values and write x (in place allowed: a
// block reads its whole tile before writing it).
template <typename T, int OFF, int REV>
__global__ void __launch_bounds__(kThreads) k_scan_solve(const T* in, T* out, int64_t n,
                                                         int64_t ntiles, const T* __restrict__ rho,
                                                         const T* __restrict__ delta,
                                                         const T* __restrict__ logm, int flip,
                                                         const Aff<T, OFF>* __restrict__ carry) {
    extern __shared__ __align__(16) unsigned char scan_smem[];
    T* sb = reinterpret_cast<T*>(scan_smem);
    T* sd = sb + Scan<T>::smem;
    T* sl = sd + Scan<T>::smem;
    __shared__ Aff<T, OFF> wt[kThreads / 32 + 1];
    const int64_t vec = blockIdx.x / ntiles, tile = blockIdx.x % ntiles;
    const int64_t l0 = tile * Scan<T>::tile;
    scan_load<T, REV>(in + vec * n, n, l0, rho, delta, logm, flip, sb, sd, sl);
    __syncthreads();
    const Aff<T, OFF> mine = thread_map<T, OFF>(sb, sd, sl);
    const Aff<T, OFF> ex = block_exclusive<T, OFF>(mine, wt, nullptr);
    const Aff<T, OFF> cin = carry[blockIdx.x];
    T st[OFF];
#pragma unroll
    for (int c = 0; c < OFF; ++c) st[c] = mul_m(ex.L[c], cin.b[c]) + ex.b[c];
#pragma unroll
    for (int e = 0; e < Scan<T>::E; ++e) {
        const int i = spad<T>(threadIdx.x * Scan<T>::E + e);
        const int c = e % OFF;
        st[c] = fma(-sd[i], st[c], st[c]) + sb[i];
        sb[i] = st[c];
    }
    __syncthreads();
    T* y = out + vec * n;
    for (int i = threadIdx.x; i < Scan<T>::tile; i += kThreads) {
        const int64_t l = l0 + i;
        if (l < n) {
            const int64_t j = REV ? n - 1 - l : l;
            const T v = sb[spad<T>(i)];
            y[j] = (flip && (j & 1)) ? -v : v;
        }
    }
}

unsigned blocks_for(int64_t count) { return (unsigned)((count + kThreads - 1) / kThreads); }

template <typename T, int OFF>
int forward_typed(const Step& st, const void* in, void* out, int64_t batch, int adjoint,
                  cudaStream_t s) {
    const int64_t n = st.n;
    const T* tab = static_cast<const T*>(st.sp_tab);
    const bool inplace = in == out;
    if (std::is_same<T, float>::value && st.sp_M == 1 && n % 4 == 0 && !inplace) {
        const int64_t total = batch * (n / 4);
        k_fwd_f4<OFF><<<blocks_for(total), kThreads, 0, s>>>(
            static_cast<const float4*>(in), static_cast<float4*>(out), n / 4, total,
            reinterpret_cast<const float4*>(tab), reinterpret_cast<const float4*>(tab + st.sp_ld),
            adjoint);
        TDH_CUDA(cudaGetLastError());
        note_launches(1);
        return TDH_OK;
    }
    const int64_t ntiles = (n + kTile - 1) / kTile;
    if (batch * ntiles > INT32_MAX) {
        set_error("sparse factors: batch * tiles above 2^31");
        return TDH_ERR_UNSUPPORTED;
    }
    const int H = OFF * st.sp_M;
    T* halo = nullptr;
    if (inplace) {
        const int64_t total = batch * ntiles * H;
        TDH_TRY(scratch_alloc(reinterpret_cast<void**>(&halo), sizeof(T) * total, s));
        k_halo_save<T><<<blocks_for(total), kThreads, 0, s>>>(static_cast<const T*>(in), halo, n,
                                                               ntiles, H, adjoint, total);
        note_launches(1);
    }
    k_fwd_tile<T, OFF><<<(unsigned)(batch * ntiles), kThreads, 0, s>>>(
        static_cast<const T*>(in), static_cast<T*>(out), n, ntiles, tab, st.sp_ld, st.sp_M,
        adjoint, halo);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) note_launches(1);
    if (halo) scratch_free(halo, s);
    TDH_CUDA(e);
    return TDH_OK;
}

template <typename T, int OFF>
int inverse_typed(const Step& st, const void* in, void* out, int64_t batch, int adjoint,
                  cudaStream_t s) {
    const int64_t n = st.n;
    const int64_t ntiles = (n + Scan<T>::tile - 1) / Scan<T>::tile;
    if (batch * ntiles > INT32_MAX || batch > INT32_MAX) {
        set_error("back-substitution: batch * tiles above 2^31");
        return TDH_ERR_UNSUPPORTED;
    }
    using A = Aff<T, OFF>;
    constexpr size_t smem = 3 * sizeof(T) * (size_t)Scan<T>::smem;
    static PerDevice attr_once;
    const cudaError_t attr = per_device(attr_once, [](int*) {
        const void* ks[4] = {(const void*)k_scan_tiles<T, OFF, 0>, (const void*)k_scan_tiles<T, OFF, 1>,
                             (const void*)k_scan_solve<T, OFF, 0>, (const void*)k_scan_solve<T, OFF, 1>};
        cudaError_t e = cudaSuccess;
        for (const void* k : ks)
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return e;
    });
    if (attr != cudaSuccess) {
        set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(attr));
        return TDH_ERR_CUDA;
    }
    A *sum = nullptr, *carry = nullptr;
    TDH_TRY(scratch_alloc(reinterpret_cast<void**>(&sum), sizeof(A) * batch * ntiles * 2, s));
    carry = sum + batch * ntiles;
    const unsigned grid = (unsigned)(batch * ntiles);
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < st.sp_M && e == cudaSuccess; ++f) {
        // A^{-1} applies the factors' inverses in order; its transpose in reverse order
        const int ff = adjoint ? st.sp_M - 1 - f : f;
        const T* tab = static_cast<const T*>(st.sp_tab) + (int64_t)ff * kInvRows * st.sp_ld;
        const T* rho = tab;
        const T* src = static_cast<const T*>(f == 0 ? in : out);
        const int flip = st.sp_flip;
        if (!adjoint) {
            const T* dl = tab + st.sp_ld;
            const T* lg = tab + 2 * st.sp_ld;
            k_scan_tiles<T, OFF, 1><<<grid, kThreads, smem, s>>>(src, n, ntiles, rho, dl, lg, flip, sum);
            k_scan_carry<T, OFF><<<(unsigned)batch, kThreads, 0, s>>>(sum, ntiles, carry);
            k_scan_solve<T, OFF, 1><<<grid, kThreads, smem, s>>>(src, static_cast<T*>(out), n, ntiles,
                                                              rho, dl, lg, flip, carry);
        } else {
            const T* dl = tab + 3 * st.sp_ld;
            const T* lg = tab + 4 * st.sp_ld;
            k_scan_tiles<T, OFF, 0><<<grid, kThreads, smem, s>>>(src, n, ntiles, rho, dl, lg, flip, sum);
            k_scan_carry<T, OFF><<<(unsigned)batch, kThreads, 0, s>>>(sum, ntiles, carry);
            k_scan_solve<T, OFF, 0><<<grid, kThreads, smem, s>>>(src, static_cast<T*>(out), n, ntiles,
                                                              rho, dl, lg, flip, carry);
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) note_launches(3);
    }
    scratch_free(sum, s);
    TDH_CUDA(e);
    return TDH_OK;
}

template <typename T>
int launch_typed(const Step& st, const void* in, void* out, int64_t batch, int adjoint,
                 cudaStream_t s) {
    if (st.sp_inverse)
        return st.sp_off == 2 ? inverse_typed<T, 2>(st, in, out, batch, adjoint, s)
                              : inverse_typed<T, 1>(st, in, out, batch, adjoint, s);
    return st.sp_off == 2 ? forward_typed<T, 2>(st, in, out, batch, adjoint, s)
                          : forward_typed<T, 1>(st, in, out, batch, adjoint, s);
}

}  // namespace

int sparse_prepare(Step& st, int prec, cudaStream_t s) {
    if (st.sp_M < 1 || st.sp_M > kMaxM) {
        set_error("sparse-factor steps support 1..%d factors (got %d)", kMaxM, st.sp_M);
        return TDH_ERR_UNSUPPORTED;
    }
    if (st.sp_off != 1 && st.sp_off != 2) {
        set_error("sparse-factor band offset must be 1 or 2");
        return TDH_ERR_INVALID_ARG;
    }
    FactorSpec F{};
    F.family = st.sp_family;
    F.off = st.sp_off;
    F.M = st.sp_M;
    F.inverse = st.sp_inverse;
    F.flip = st.sp_flip;
    F.par0 = st.sp_par0;
    F.dir = st.sp_dir;
    F.b = st.sp_b;
    F.n = st.n;
    F.ld = (st.n + 2 + 3) / 4 * 4;  // float4 rows stay 16-byte aligned
    st.sp_ld = F.ld;
    const int rows = st.sp_inverse ? kInvRows : 2;
    const size_t esz = prec != TDH_FP64 ? 4 : 8;
    TDH_TRY(dev_alloc(&st.sp_tab, esz * (size_t)F.ld * rows * st.sp_M));
    const unsigned blocks = blocks_for(F.ld * F.M);
    if (prec != TDH_FP64)
        k_sparse_tables<float><<<blocks, kThreads, 0, s>>>(F, st.scale_out, st.scale_in,
                                                           static_cast<float*>(st.sp_tab));
    else
        k_sparse_tables<double><<<blocks, kThreads, 0, s>>>(F, st.scale_out, st.scale_in,
                                                            static_cast<double*>(st.sp_tab));
    TDH_CUDA(cudaGetLastError());
    return TDH_OK;
}

int sparse_launch(const Step& st, int prec, const void* in, void* out, int64_t batch, int adjoint,
                  cudaStream_t s) {
    if (prec != TDH_FP64) return launch_typed<float>(st, in, out, batch, adjoint, s);
    return launch_typed<double>(st, in, out, batch, adjoint, s);
}

}  // namespace tdh
