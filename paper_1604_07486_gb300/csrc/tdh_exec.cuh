// Steps a4-a7: the fused execute kernel, beta = D1 sum_r u_r o T (u_r o D2 alpha)
// (Fig. 1 steps 3-5, Eq. (5)), and its adjoint.
//
// Layout.  T has the parity structure of the Legendre/Chebyshev/ultraspherical cases
// (T_jk = 0 for k - j odd), so even and odd indices never mix: with z_a = x_{2a} + i x_{2a+1}
// both halves are upper-triangular Toeplitz products with the same generator s_m = t_{2m},
// and one complex correlation y_a = sum_{b>=a} s_{b-a} z_b does both.  The float pairs of a
// coefficient vector are exactly that complex array, so no shuffle is needed.  Each
// correlation is a circular one of length L >= 2m - 1 (m = ceil(n/2)): zero-padded FFT,
// multiply by conj(DFT(s)), inverse FFT (Sec. 1, citing Ng Sec. 3.4).
//
// One vector is handled by a cluster of C CTAs (C = 1 when the FFT fits one CTA's shared
// memory).  CTA k1 of the cluster owns the decimated sequence z[k1 + C k2], k2 < LC = L / C,
// keeps it and the scaled input in shared memory, and runs all K rank terms:
//   forward local DIF passes (radix R, natural order in, digit-reversed out)
//   -> cross-CTA stage through distributed shared memory (twiddle, C-point DFT, symbol
//      multiply, inverse C-point DFT, conjugate twiddle; fused into one exchange)
//   -> inverse local DIT passes (digit-reversed in, natural out)
// accumulating w += u_r o y in registers.  alpha is read once and beta written once.
#pragma once

#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "tdh_fft.cuh"
#include "tdh_internal.cuh"
#include "tdh_tc.cuh"

namespace tdh {

namespace cg = cooperative_groups;

// Pass geometry of a local FFT of length 2^LOGLC with radix-R passes and a trailing
// smaller radix when log2(R) does not divide LOGLC.
struct PassGeom {
    int logLC, R;
    __host__ __device__ constexpr int LC() const { return 1 << logLC; }
    __host__ __device__ constexpr int logR() const { return ilog2(R); }
    __host__ __device__ constexpr int npr() const { return logLC / logR(); }
    __host__ __device__ constexpr int r0() const { return 1 << (logLC - npr() * logR()); }
    __host__ __device__ constexpr int np() const { return npr() + (r0() > 1 ? 1 : 0); }
    __host__ __device__ constexpr int rad(int i) const { return i < npr() ? R : r0(); }
    __host__ __device__ constexpr int M(int i) const {
        int m = LC();
        for (int j = 0; j < i; ++j) m /= rad(j);
        return m;
    }
    __host__ __device__ constexpr int S(int i) const { return M(i) / rad(i); }
    // offset of middle pass i (1 <= i <= np()-2) in the concatenated [p][o] tables
    __host__ __device__ constexpr int twoff(int i) const {
        int off = 0;
        for (int j = 1; j < i; ++j) off += M(j);
        return off;
    }
    __host__ __device__ constexpr int twp_len() const { return twoff(np() - 1); }
};

// Natural frequency of local position pos after the DIF passes (digit reversal).
__host__ __device__ inline int local_freq(const PassGeom& G, int pos) {
    int rem = pos, f = 0, mult = 1;
    for (int i = 0; i < G.np(); ++i) {
        const int s = G.S(i);
        const int p = rem / s;
        rem %= s;
        f += p * mult;
        mult *= G.rad(i);
    }
    return f;
}

// Radix of the local passes: 16 where the float32 FFT has room for it, else 8.
__host__ __device__ constexpr int radix_for(bool f32, int logLC) {
    return f32 && logLC > 9 ? 16 : 8;
}

// Compiled execute schedules: local FFT length 2^logLC, cluster size C, threads per CTA NT,
// the occupancy the registers are capped for (MINB CTAs per SM: 65536 / (NT MINB) registers
// per thread) and the radix of the local passes (0: radix_for's).  The first schedule of each
// (logLC, C) is the default one; the others trade threads per CTA for CTAs per SM, local
// length for cluster size, or four radix-16 passes for three of radix 32, 32 and 16.
struct Sched {
    int logLC, C, NT, MINB, R = 0;
};
__host__ __device__ constexpr int sched_radix(const Sched& e, bool f32) {
    return e.R ? e.R : radix_for(f32, e.logLC);
}
constexpr Sched kSchedF32[] = {
    {8, 1, 32, 1},    {8, 1, 32, 16},   {9, 1, 64, 1},    {9, 1, 64, 8},    {10, 1, 64, 1},
    {10, 1, 64, 8},   {10, 1, 32, 16},  {11, 1, 128, 1},  {11, 1, 128, 4},  {11, 1, 64, 8},
    {12, 1, 256, 1},  {12, 1, 256, 2},  {12, 1, 128, 4},  {13, 1, 512, 1},  {13, 1, 256, 2},
    {14, 1, 512, 1},  {14, 2, 512, 1},  {14, 4, 512, 1},  {14, 8, 512, 1},  {13, 2, 256, 2},
    {13, 4, 256, 2},  {13, 8, 256, 2},  {9, 2, 64, 1},    {8, 4, 32, 1},    {10, 2, 64, 1},
    {11, 2, 128, 1},  {12, 2, 256, 2},  {14, 2, 512, 1, 32}, {14, 4, 512, 1, 32},
    {14, 8, 512, 1, 32}, {14, 1, 512, 1, 32}, {13, 1, 256, 2, 32},
};
constexpr Sched kSchedF64[] = {
    {8, 1, 32, 1},    {8, 1, 32, 16},   {9, 1, 64, 1},    {9, 1, 64, 8},    {10, 1, 128, 1},
    {10, 1, 128, 4},  {11, 1, 256, 1},  {11, 1, 256, 2},  {11, 1, 128, 4},  {12, 1, 512, 1},
    {12, 1, 256, 2},  {13, 1, 512, 1},  {13, 2, 512, 1},  {13, 4, 512, 1},  {13, 8, 512, 1},
    {12, 2, 256, 2},  {12, 4, 256, 2},  {12, 8, 256, 2},  {9, 2, 64, 1},    {8, 4, 32, 1},
    {10, 2, 128, 1},  {9, 4, 64, 1},    {11, 2, 256, 1},  {10, 4, 128, 1},
};
template <bool F32>
struct SchedTable {
    static constexpr int size = (int)(sizeof(kSchedF32) / sizeof(Sched));
    static constexpr Sched at(int i) { return kSchedF32[i]; }
};
template <>
struct SchedTable<false> {
    static constexpr int size = (int)(sizeof(kSchedF64) / sizeof(Sched));
    static constexpr Sched at(int i) { return kSchedF64[i]; }
};
// Split-bfloat16 tensor-core schedules (TDH_BF16X3): the float32 geometries with one CTA per
// SM's worth of registers, and the two-CTA variants of the 8192-point slices.
constexpr Sched kSchedTC[] = {
    {8, 1, 32, 1},   {9, 1, 64, 1},   {10, 1, 64, 1},  {11, 1, 128, 1}, {12, 1, 256, 1},
    {13, 1, 512, 1}, {14, 1, 512, 1}, {14, 2, 512, 1}, {14, 4, 512, 1}, {14, 8, 512, 1},
    {13, 2, 256, 2}, {13, 4, 256, 2}, {13, 8, 256, 2}, {9, 2, 64, 1},   {8, 4, 32, 1},
    {10, 2, 64, 1},  {11, 2, 128, 1}, {12, 2, 256, 2},
};
struct SchedTableTC {
    static constexpr int size = (int)(sizeof(kSchedTC) / sizeof(Sched));
    static constexpr Sched at(int i) { return kSchedTC[i]; }
};

// Tensor-core passes: TMEM columns a CTA allocates for local length 2^LOGLC, radix R and NT
// threads.  A middle pass of LC / R groups runs as tiles of RT = min(NT, 128) groups (one
// group per TMEM lane); a tile holds its A operand as split-bfloat16 hi and lo rows (R
// columns each) and its float32 result D (2R columns).
__host__ __device__ constexpr int tc_rows(int NT) { return NT < 128 ? NT : 128; }
__host__ __device__ constexpr int tc_cols(int LOGLC, int R, int NT) {
    const int need = ((1 << LOGLC) / R / tc_rows(NT)) * 4 * R;
    int c = 32;
    while (c < need) c *= 2;
    return c;
}

// Float32 kernels whose local FFT has 32 points per thread (2^14 points on 512 threads, or
// single-CTA FFTs of 2^13 points on 256 threads, two CTAs per SM) keep in tensor memory,
// which they do not otherwise use: the spectrum values their threads multiply by -- the same
// for every rank term and every vector -- instead of reading them from L2 for every rank
// term, and the output accumulators w, which otherwise hold 32 registers across the whole
// rank loop (the room radix-32 passes need).  Each thread owns one TMEM lane (thread t of
// warp w: lane 32 (w % 4) + t); the four warps that share a lane set take 128 columns each.
//   cluster kernels (C = 2, 4, 8; 512 threads): per cross-stage iteration the first `head` of
//     its 4 + 4C words (two twiddles, the spectrum of two positions) at columns [0, 64), the
//     last 4 at [64, 96);
//   single-CTA kernels: the spectrum of each of the thread's last-pass groups, in the order
//     the group multiplies by it, at columns [0, 64);
//   both: the 32 accumulator words at [96, 128).
// A CTA allocates 128 columns per 128 threads; single-CTA 2^13 kernels take more than a third
// of an SM's shared memory, so at most two share an SM's 512 columns.
template <typename T, int LOGLC, int C, int NT, int MINB, bool TC>
struct SpecTmem {
    static constexpr bool f32 = !TC && std::is_same<T, float>::value;
    static constexpr bool cluster = f32 && C > 1 && C <= 8 && LOGLC == 14 && NT == 512 &&
                                    MINB == 1;
    static constexpr bool single = f32 && C == 1 && ((LOGLC == 14 && NT == 512 && MINB == 1) ||
                                                     (LOGLC == 13 && NT == 256 && MINB == 2));
    static constexpr bool on = cluster || single;
    static constexpr int cols = NT;                            // columns allocated
    static constexpr int iters = (1 << LOGLC) / C / (2 * NT);  // cross-stage iterations
    static constexpr int words = 4 + 4 * C;                    // per iteration
    static constexpr int head = words >= 32 ? 32 : (words >= 16 ? 16 : 8);  // first load width
    static constexpr int tail_col = 64;                        // columns of the last 4 words
    static constexpr int acc_col = 96;                         // the accumulators' 32 words
    static_assert(!cluster || (words - head == 4 && iters * head == 64 && iters * 4 <= 32),
                  "slot layout");
    static_assert(!single || 2 * (1 << LOGLC) / NT == 64, "single-CTA spectrum: 64 words");
};

template <typename T>
struct ExecParams {
    using V = typename cx<T>::t;
    const T* in;
    T* out;
    int64_t n;
    int64_t K;
    const V* u;     // [K][C][LC/2]
    const V* spec;  // [LC][C]
    const V* twx;   // [LC]
    const V* tw0;   // [LC/R]
    const V* twp;   // [twp_len]
    const T* din;   // D2 (forward) or D1 (adjoint), [n]
    const T* dout;  // D1 (forward) or D2 (adjoint), [n]
    const T* row0;  // row 0 applied directly (Chebyshev-to-Legendre), [n], or null
    int adjoint;
    int full;       // 0: parity packing (x_2a, x_2a+1); 1: rank pairs (u_r, u_r+1) per index
    int sign_in;    // multiply input coefficient k by (-1)^k (Jacobi reflection)
    int sign_out;   // multiply output coefficient k by (-1)^k
    int64_t u_stride;  // complex entries between consecutive (rank, k1) rows of u
    // dense batches, balanced split: the launch's G clusters share the batch's U = batch * Ku
    // (vector, rank term) units equally (Ku = max(K, 1)); cluster c applies units
    // [U c / G, U (c+1) / G) and writes a vector split between clusters as partial sums:
    // slot 2c+1 for its piece holding rank 0, slot 2c for a later piece (partial: [2G][n])
    int64_t batch;
    T* partial;
    // ragged batches: vector v occupies [offs[v], offs[v+1]); this launch converts the
    // vectors list[0 .. *count) of one FFT-length class, taking them from the *next counter
    int ragged;
    const int64_t* offs;
    const int* list;
    const int* count;
    int* next;
    // device status word (TDH_STATUS_* bits, may be null): a tensor-core pass whose MMA wait
    // ran out of time sets TDH_STATUS_TIMEOUT
    int* status;
    // test hook (tdh_test_tc_stall): tensor-core passes issue no products, so their bounded
    // waits run out
    int tc_stall;
    // rank-pair packing: output factor of each pair's second term (1 / its input scale^2)
    const T* pair_c;
};

#ifndef TDH_SMEM_PAD
#define TDH_SMEM_PAD 0
#endif
#if TDH_SMEM_PAD
// Shared-memory index of FFT element i: one padding element after every 128-byte row.
template <typename V>
__device__ __forceinline__ int sidx(int i) {
    constexpr int epr = 128 / (int)sizeof(V);
    return i + i / epr;
}
template <typename V>
__host__ __device__ constexpr int padded_len(int n) {
    return n + n / (128 / (int)sizeof(V));
}
// element pair (2k, 2k+1) -> (first address, swapped?)
template <typename V>
__device__ __forceinline__ bool pair_swapped(int) { return false; }
#else
// Shared-memory index of FFT element i: XOR swizzle within 128-byte rows (column ^= row),
// free of bank conflicts for every pass's access pattern.
template <typename V>
__device__ __forceinline__ int sidx(int i) {
    constexpr int epr = 128 / (int)sizeof(V);
    return i ^ ((i / epr) & (epr - 1));
}
template <typename V>
__host__ __device__ constexpr int padded_len(int n) {
    return n;
}
// The aligned pair (2k, 2k+1) stays an aligned pair under the swizzle, swapped when bit 0 of
// its row index is set.
template <typename V>
__device__ __forceinline__ bool pair_swapped(int i) {
    constexpr int epr = 128 / (int)sizeof(V);
    return ((i / epr) & 1) != 0;
}
#endif

// Two consecutive complex values as one 16-byte (float) or two 16-byte (double) accesses.
__device__ __forceinline__ void pair_load(const float2* p, float2& a, float2& b) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void pair_store(float2* p, float2 a, float2 b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void pair_load(const double2* p, double2& a, double2& b) {
    a = p[0];
    b = p[1];
}
__device__ __forceinline__ void pair_store(double2* p, double2 a, double2 b) {
    p[0] = a;
    p[1] = b;
}

// powers w^p, p in [0, R), from w^1 by a binary tree of products (error ~ log2(p) ulp)
template <int R, typename V>
__device__ __forceinline__ void powers(V w1, V (&wp)[R]) {
    wp[0] = mk<V>(1, 0);
    if constexpr (R > 1) wp[1] = w1;
#pragma unroll
    for (int p = 2; p < R; ++p) {
        int hi = 1;
        while (hi * 2 <= p) hi *= 2;
        wp[p] = (hi == p) ? cmul(wp[p / 2], wp[p / 2]) : cmul(wp[hi], wp[p - hi]);
    }
}

// The twiddles w^p, p in [0, R), of one radix-R group.  Up to R = 16 every power is held in
// registers; for R = 32 (64 registers of data already) only w^0..w^7 and (w^8)^0..(w^8)^3 are,
// and w^p = (w^8)^(p/8) w^(p%8) costs one product where both factors differ from 1 -- about as
// many products as the full table, in 24 registers instead of 64.
template <int R, typename V>
struct TwPow {
    static constexpr bool split = R > 16;
    static constexpr int NL = split ? 8 : R;
    static constexpr int NH = split ? R / 8 : 1;
    V lo[NL];
    V hi[NH];
    __device__ __forceinline__ explicit TwPow(V w1) {
        powers<NL>(w1, lo);
        if constexpr (split) {
            hi[0] = mk<V>(1, 0);
            hi[1] = cmul(lo[4], lo[4]);
#pragma unroll
            for (int h = 2; h < NH; ++h) hi[h] = (h % 2 == 0) ? cmul(hi[h / 2], hi[h / 2])
                                                              : cmul(hi[h - 1], hi[1]);
        }
    }
    // x w^p (p a constant after unrolling)
    __device__ __forceinline__ V mul(V x, int p) const {
        if constexpr (!split) {
            return p == 0 ? x : cmul(x, lo[p]);
        } else {
            if (p == 0) return x;
            if (p % 8 == 0) return cmul(x, hi[p / 8]);
            if (p < 8) return cmul(x, lo[p]);
            return cmul(x, cmul(hi[p / 8], lo[p % 8]));
        }
    }
    // x conj(w^p)
    __device__ __forceinline__ V mulc(V x, int p) const {
        if constexpr (!split) {
            return p == 0 ? x : cmulc(x, lo[p]);
        } else {
            if (p == 0) return x;
            if (p % 8 == 0) return cmulc(x, hi[p / 8]);
            if (p < 8) return cmulc(x, lo[p]);
            return cmulc(x, cmul(hi[p / 8], lo[p % 8]));
        }
    }
};

// Middle forward pass i: radix RAD, sub-length M, stride S, twiddles from the [p][o] table.
// Every group g = tid + i NT of a thread has the same offset o = g % S (NT is a multiple of
// S), so its twiddles omega_M^{p o} are powers of one table entry, formed once per pass in
// registers instead of read per group from shared memory.
template <int RAD, int M, int S, int LC, int NT, typename V>
__device__ __forceinline__ void pass_fwd(V* buf, const V* tw) {
    static_assert(NT % S == 0, "thread count must be a multiple of the pass stride");
    const TwPow<RAD, V> wp(tw[S + (int)threadIdx.x % S]);
#pragma unroll 1
    for (int g = threadIdx.x; g < LC / RAD; g += NT) {
        const int b = g / S, o = g % S;
        const int base = b * M + o;
        V x[RAD];
#pragma unroll
        for (int q = 0; q < RAD; ++q) x[q] = buf[sidx<V>(base + q * S)];
        dif<RAD>(x);
#pragma unroll
        for (int jj = 0; jj < RAD; ++jj) {
            const int p = bitrev(jj, RAD);
            buf[sidx<V>(base + p * S)] = wp.mul(x[jj], p);
        }
    }
}

template <int RAD, int M, int S, int LC, int NT, typename V>
__device__ __forceinline__ void pass_inv(V* buf, const V* tw) {
    static_assert(NT % S == 0, "thread count must be a multiple of the pass stride");
    const TwPow<RAD, V> wp(tw[S + (int)threadIdx.x % S]);
#pragma unroll 1
    for (int g = threadIdx.x; g < LC / RAD; g += NT) {
        const int b = g / S, o = g % S;
        const int base = b * M + o;
        V x[RAD];
#pragma unroll
        for (int p = 0; p < RAD; ++p) x[bitrev(p, RAD)] = wp.mulc(buf[sidx<V>(base + p * S)], p);
        dit<RAD>(x);
#pragma unroll
        for (int q = 0; q < RAD; ++q) buf[sidx<V>(base + q * S)] = x[q];
    }
}

// ------------------------------------------------------------ split-bfloat16 DFT-GEMM passes
//
// A middle pass as a matrix product on the tensor cores (TDH_BF16X3).  Group g (offset o,
// block b) holds the RAD points x_q = buf[b M + o + q S]; as a row of 2 RAD reals (re, im
// interleaved) its radix-RAD DFT is one row of A W, W the 2 RAD x 2 RAD real form of the DFT
// matrix.  Both factors are split, A = Ah + Al and W = Wh + Wl (bfloat16 hi and lo parts), and
// the three products Ah Wh + Al Wh + Ah Wl accumulate in float32 in tensor memory (the
// dropped Al Wl is below 2^-17 of the product).  Forward: D = A W, then the twiddles
// omega_M^{p o} in float32; inverse: the conjugate twiddles first, then the product with the
// conjugate DFT matrix.  Same values as pass_fwd / pass_inv up to the split's rounding.
//
// Per-CTA state: TMEM base address, the four B matrices in shared memory (forward hi, lo,
// inverse hi, lo; K-major core-matrix layout), the MMA-completion mbarriers (one per
// warpgroup and tile) and their common phase.
struct TcState {
    uint32_t spec_tmem;  // SpecTmem: base of the cross stage's spectrum and twiddles
    uint32_t tmem;
    uint32_t bsm;
    uint32_t mbar;
    uint32_t phase;
    int* fail;    // shared: set once a wait ran out (later passes do not wait)
    int* status;  // global status word or null
    int stall;    // test hook: issue no products (every wait runs out)
};

// Limit of one wait for the MMAs of a pass (they take microseconds).
constexpr uint64_t kTcWaitNs = 1000000000ull;

// W (forward: sign +1; inverse: -1) in bfloat16 hi/lo parts, K-major core matrices: element
// (n, k) at byte (k/8 (N/8) + n/8) 128 + (n%8) 16 + (k%8) 2, N = 2 RAD.
template <int RAD, int NT>
__device__ __forceinline__ void tc_build_dft(unsigned char* bsm) {
    constexpr int N = 2 * RAD;
    constexpr int BM = N * N * 2;
    for (int i = threadIdx.x; i < 2 * N * N; i += NT) {
        const int inv = i / (N * N), e = i % (N * N);
        const int n = e / N, k = e % N;
        const int a = n >> 1, b = k >> 1;
        const int r = (a * b) % RAD;
        double sn, cs;
        sincospi(2.0 * (double)r / (double)RAD, &sn, &cs);
        const double sig = inv ? -1.0 : 1.0;
        // out_re = c x_re + sig s x_im ; out_im = -sig s x_re + c x_im
        const double w = ((n & 1) == (k & 1)) ? cs : ((n & 1) == 0 ? sig * sn : -sig * sn);
        const __nv_bfloat16 hi = __double2bfloat16(w);
        const __nv_bfloat16 lo = __double2bfloat16(w - (double)__bfloat162float(hi));
        const int off = ((k >> 3) * (N / 8) + (n >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2;
        *reinterpret_cast<__nv_bfloat16*>(bsm + inv * 2 * BM + off) = hi;
        *reinterpret_cast<__nv_bfloat16*>(bsm + inv * 2 * BM + BM + off) = lo;
    }
}

// Warpgroups of a tensor-core pass: RT = min(NT, 128) threads own the RT lanes of their tiles;
// warpgroup w of the CTA takes tiles w, w + NWG, ... (one per group index i of its threads).
// Each warpgroup stages, issues and drains its own tiles, with its own mbarriers (one per
// tile index i) and a named barrier, so the tensor core works on one warpgroup's products
// while others stage or drain theirs, and the products of a warpgroup's tile i overlap the
// staging of its tile i + 1.
constexpr int kTcMaxTilesPerGroup = 4;
constexpr int kTcMaxGroups = 4;

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(nthreads) : "memory");
}

template <int RAD, int M, int S, int LC, int NT, bool FWD>
__device__ __forceinline__ void tc_pass(float2* buf, const float2* tw, TcState& ts) {
    static_assert(NT % S == 0, "thread count must be a multiple of the pass stride");
    static_assert(RAD == 8 || RAD == 16, "tensor-core passes are radix 8 or 16");
    using V = float2;
    constexpr int G = LC / RAD;            // groups: one TMEM lane (row of A and D) each
    constexpr int J = G / NT;              // groups (tiles) per thread
    constexpr int RT = tc_rows(NT);        // rows per tile = threads per warpgroup
    constexpr int NWG = NT / RT;           // warpgroups
    constexpr int CT = 4 * RAD;            // TMEM columns per tile: hi, lo (RAD each), D (2 RAD)
    constexpr int N = 2 * RAD;             // MMA N (and K of one operand part)
    constexpr int NCH = N / 16;            // K = 16 chunks per part
    constexpr uint32_t KST = (N / 8) * 128;   // bytes between K-adjacent core matrices of W
    constexpr uint32_t BM = N * N * 2;
    static_assert(J >= 1 && G % NT == 0 && NT % RT == 0, "groups must divide over threads");
    static_assert(J <= kTcMaxTilesPerGroup && NWG <= kTcMaxGroups, "mbarrier slots");
    const int tid = threadIdx.x;
    const int wg = tid / RT;
    const bool leader = (tid % RT) == 0;
    const uint32_t lane_base = (uint32_t)(32 * ((tid >> 5) & 3)) << 16;
    V wp[RAD];  // twiddle powers: used before the products (inverse) or after (forward)
    if constexpr (!FWD) powers<RAD>(tw[S + tid % S], wp);
    // 1. per tile: split rows into TMEM (inverse: conjugate twiddles first), then the
    //    warpgroup's leader issues the three split products and commits to the tile's mbarrier
#pragma unroll 1
    for (int i = 0; i < J; ++i) {
        const int g = tid + i * NT;
        const int t = g / RT;
        const int base = (g / S) * M + (g % S);
        const uint32_t col = ts.tmem + lane_base + (uint32_t)(t * CT);
        // eight points at a time (hi to columns [q0, q0 + 8), lo to [RAD + q0, ...))
#pragma unroll
        for (int q0 = 0; q0 < RAD; q0 += 8) {
            uint32_t hi[8], lo[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                V x = buf[sidx<V>(base + (q0 + q) * S)];
                if (!FWD && q0 + q > 0) x = cmulc(x, wp[q0 + q]);
                tc::split2(x.x, x.y, hi[q], lo[q]);
            }
            tc::tmem_st8(col + q0, hi);
            tc::tmem_st8(col + RAD + q0, lo);
        }
        tc::tmem_wait_st();
        tc::fence_before_sync();
        named_barrier(1 + wg, RT);
        if (leader && !ts.stall) {
            tc::fence_after_sync();
            constexpr uint32_t idesc = tc::idesc_bf16(128, N);
            const uint32_t wh = ts.bsm + (FWD ? 0u : 2u * BM), wl = wh + BM;
            const uint32_t a = ts.tmem + (uint32_t)(t * CT);
            const uint32_t d = a + 2 * RAD;
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                tc::mma_ts(d, a + 8 * c, tc::smem_desc(wh + c * 2 * KST, KST, 128), idesc,
                           c > 0 ? 1u : 0u);
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                tc::mma_ts(d, a + RAD + 8 * c, tc::smem_desc(wh + c * 2 * KST, KST, 128), idesc, 1u);
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                tc::mma_ts(d, a + 8 * c, tc::smem_desc(wl + c * 2 * KST, KST, 128), idesc, 1u);
            tc::mma_commit(ts.mbar + 8u * (uint32_t)(wg * kTcMaxTilesPerGroup + i));
        }
    }
    // 2. per tile: wait for its products (bounded), read D, twiddle (forward), store
    if constexpr (FWD) powers<RAD>(tw[S + tid % S], wp);
#pragma unroll 1
    for (int i = 0; i < J; ++i) {
        const uint32_t mb = ts.mbar + 8u * (uint32_t)(wg * kTcMaxTilesPerGroup + i);
        if (!*ts.fail && !tc::mbar_wait_bounded(mb, ts.phase, kTcWaitNs)) {
            *ts.fail = 1;
            if (ts.status) atomicOr(ts.status, TDH_STATUS_TIMEOUT);
        }
        __syncwarp();
        tc::fence_after_sync();
        const int g = tid + i * NT;
        const int t = g / RT;
        const int base = (g / S) * M + (g % S);
        const uint32_t col = ts.tmem + lane_base + (uint32_t)(t * CT + 2 * RAD);
        uint32_t dv[N];
        if constexpr (RAD == 16)
            tc::tmem_ld32(col, dv);
        else
            tc::tmem_ld16(col, dv);
#pragma unroll
        for (int p = 0; p < RAD; ++p) {
            V y = mk<V>(__uint_as_float(dv[2 * p]), __uint_as_float(dv[2 * p + 1]));
            if (FWD && p > 0) y = cmul(y, wp[p]);
            buf[sidx<V>(base + p * S)] = y;
        }
    }
    ts.phase ^= 1u;
    tc::fence_before_sync();
}

template <int I, int LOGLC, int R, int NT, bool TC, typename V>
__device__ __forceinline__ void middle_fwd(V* buf, const V* twt, TcState* ts) {
    constexpr PassGeom G{LOGLC, R};
    if constexpr (I <= G.np() - 2) {
        if constexpr (TC)
            tc_pass<G.rad(I), G.M(I), G.S(I), G.LC(), NT, true>(buf, twt + G.twoff(I), *ts);
        else
            pass_fwd<G.rad(I), G.M(I), G.S(I), G.LC(), NT>(buf, twt + G.twoff(I));
        __syncthreads();
        middle_fwd<I + 1, LOGLC, R, NT, TC>(buf, twt, ts);
    }
}

template <int I, int LOGLC, int R, int NT, bool TC, typename V>
__device__ __forceinline__ void middle_inv(V* buf, const V* twt, TcState* ts) {
    constexpr PassGeom G{LOGLC, R};
    if constexpr (I >= 1) {
        if constexpr (TC)
            tc_pass<G.rad(I), G.M(I), G.S(I), G.LC(), NT, false>(buf, twt + G.twoff(I), *ts);
        else
            pass_inv<G.rad(I), G.M(I), G.S(I), G.LC(), NT>(buf, twt + G.twoff(I));
        __syncthreads();
        middle_inv<I - 1, LOGLC, R, NT, TC>(buf, twt, ts);
    }
}

// Cross stage, float32: the values at the pair of positions (pos, pos+1), pos even, in each of
// the C CTAs' buffers (one 16-byte access per CTA); a[u][j] = position pos + u of CTA j.
template <int C, typename V>
__device__ __forceinline__ void cross_pair_load(V* const (&rbuf)[C], int pos, V (&a)[2][C]) {
    const bool swp = pair_swapped<V>(pos);
    const int sp = sidx<V>(pos) & ~1;
#pragma unroll
    for (int j = 0; j < C; ++j) {
        V e0, e1;
        pair_load(rbuf[j] + sp, e0, e1);
        a[0][j] = swp ? e1 : e0;
        a[1][j] = swp ? e0 : e1;
    }
}

// The inverse middle passes np-2 ... 1 with a barrier between passes but none after the last:
// the caller issues loads that do not touch the FFT buffer before that barrier.
template <int I, int LOGLC, int R, int NT, bool TC, typename V>
__device__ __forceinline__ void middle_inv_open(V* buf, const V* twt, TcState* ts) {
    constexpr PassGeom G{LOGLC, R};
    if constexpr (I >= 1) {
        if constexpr (TC)
            tc_pass<G.rad(I), G.M(I), G.S(I), G.LC(), NT, false>(buf, twt + G.twoff(I), *ts);
        else
            pass_inv<G.rad(I), G.M(I), G.S(I), G.LC(), NT>(buf, twt + G.twoff(I));
        if constexpr (I > 1) {
            __syncthreads();
            middle_inv_open<I - 1, LOGLC, R, NT, TC>(buf, twt, ts);
        }
    }
}

// One vector: v = D alpha -> all K rank terms -> beta (the whole of Fig. 1 steps 3-5).
template <typename T, int LOGLC, int R, int C, int NT, bool TC, bool STM>
__device__ __forceinline__ void convert_vector(const ExecParams<T>& P, const T* in, T* out,
                                               const int64_t n, const int k1,
                                               typename cx<T>::t* buf, typename cx<T>::t* vbuf,
                                               const typename cx<T>::t* twt, T* red,
                                               const int64_t r_begin, const int64_t r_end,
                                               const bool lead, TcState* ts) {
    using V = typename cx<T>::t;
    constexpr PassGeom G{LOGLC, R};
    constexpr int LC = G.LC();
    constexpr int S0 = LC / R;
    constexpr int J0 = S0 / NT;
    constexpr int RL = G.rad(G.np() - 1);  // radix of the last pass (stride 1)
    static_assert(R <= 16 || STM, "radix-32 passes need the accumulators in tensor memory");
    const int tid = threadIdx.x;
    T r0acc = T(0);
    for (int k2 = tid; k2 < LC / 2; k2 += NT) {
        const int64_t a = (int64_t)k1 + (int64_t)C * k2;
        V v = mk<V>(0, 0);
        if (P.full) {
            // one coefficient per complex slot, duplicated for the two packed rank terms
            if (a < n) {
                T x = in[a];
                if (P.sign_in && (a & 1)) x = -x;
                if (P.row0 && !P.adjoint) r0acc += P.row0[a] * x;
                const T xv = x * P.din[a];
                v = mk<V>(xv, xv);
            }
        } else {
            const int64_t i0 = 2 * a;
            if (i0 < n) {
                const T x0 = in[i0];
                T x1 = (i0 + 1 < n) ? in[i0 + 1] : T(0);
                if (P.sign_in) x1 = -x1;
                const T s1 = (i0 + 1 < n) ? P.din[i0 + 1] : T(0);
                if (P.row0 && !P.adjoint)
                    r0acc += P.row0[i0] * x0 + ((i0 + 1 < n) ? P.row0[i0 + 1] * x1 : T(0));
                v = mk<V>(x0 * P.din[i0], x1 * s1);
            }
        }
        vbuf[k2] = v;
    }
    V w0[J0];
#pragma unroll
    for (int j = 0; j < J0; ++j) w0[j] = P.tw0[tid + j * NT];
    // w accumulators: registers, or (STM) this thread's 32 words of tensor memory, loaded only
    // around the inverse pass 0 of each rank term and in the epilogue
    V acc[J0][R / 2];
    constexpr int ACCW = J0 * R;  // float words of the accumulators
    uint32_t acc_col = 0;
    if constexpr (STM) {
        static_assert(ACCW == 32, "tensor-memory accumulators: 32 words per thread");
        using ST = SpecTmem<T, LOGLC, C, NT, 1, false>;
        acc_col = ts->spec_tmem + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) +
                  (uint32_t)((tid >> 7) * 128 + ST::acc_col);
        uint32_t z[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) z[i] = 0u;
        tc::tmem_st<32>(acc_col, z);
        tc::tmem_wait_st();
    } else {
#pragma unroll
        for (int j = 0; j < J0; ++j)
#pragma unroll
            for (int q = 0; q < R / 2; ++q) acc[j][q] = mk<V>(0, 0);
    }
    // The factor values of both passes 0 are read from L2 once per rank term.  In the float32
    // kernels they are loaded ahead, before the barrier that precedes their use, so their
    // latency overlaps the wait: ul0 (forward pass 0, every group) at the end of the previous
    // rank term, ulp (inverse pass 0, the first group) before the last inverse middle pass's
    // barrier.  (Measured: 0.5 % faster there; float64 and tensor-core kernels, which have no
    // registers to spare, load them at the start of the pass.)
    constexpr bool kAhead = !TC && sizeof(T) == 4;
    V ul0[J0][R / 2], ulp[R / 2];
    auto load_ul0 = [&](int64_t r) {
        const V* u = P.u + ((int64_t)r * C + k1) * P.u_stride;
#pragma unroll
        for (int j = 0; j < J0; ++j)
#pragma unroll
            for (int q = 0; q < R / 2; ++q) ul0[j][q] = u[tid + j * NT + q * S0];
    };
    if (kAhead && r_begin < r_end) load_ul0(r_begin);
    __syncthreads();

    V* rbuf[C];
    if constexpr (C > 1) {
        cg::cluster_group cl = cg::this_cluster();
#pragma unroll
        for (int j = 0; j < C; ++j) rbuf[j] = cl.map_shared_rank(buf, j);
    } else {
        rbuf[0] = buf;
    }

#pragma unroll 1
    for (int64_t r = r_begin; r < r_end; ++r) {
        const V* ur = P.u + ((int64_t)r * C + k1) * P.u_stride;
        const T cpair = (P.full && P.pair_c) ? P.pair_c[r] : T(1);
        // ---- forward pass 0: inputs u_r o v (upper half zero), radix R, stride S0
        if constexpr (!kAhead) load_ul0(r);
#pragma unroll
        for (int j = 0; j < J0; ++j) {
            const int o = tid + j * NT;
            V x[R];
#pragma unroll
            for (int q = 0; q < R / 2; ++q) x[q] = cwmul(vbuf[o + q * S0], ul0[j][q]);
            dif_halfzero<R>(x);
            const TwPow<R, V> wp(w0[j]);
#pragma unroll
            for (int jj = 0; jj < R; ++jj) {
                const int p = bitrev(jj, R);
                buf[sidx<V>(o + p * S0)] = wp.mul(x[jj], p);
            }
        }
        __syncthreads();
        middle_fwd<1, LOGLC, R, NT, TC>(buf, twt, ts);
        // ---- last pass (stride 1), spectrum, first inverse pass
        if constexpr (C == 1) {
#pragma unroll 1
            for (int g = tid, i = 0; g < LC / RL; g += NT, ++i) {
                V x[RL];
#pragma unroll
                for (int q = 0; q < RL; ++q) x[q] = buf[sidx<V>(g * RL + q)];
                dif<RL>(x);
                V sp[RL];
                if constexpr (STM) {  // this group's spectrum from the thread's TMEM lane
                    uint32_t sw[2 * RL];
                    tc::tmem_ld<2 * RL>(ts->spec_tmem + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) +
                                            (uint32_t)((tid >> 7) * 128 + i * 2 * RL),
                                        sw);
#pragma unroll
                    for (int jj = 0; jj < RL; ++jj)
                        sp[jj] = mk<V>(__uint_as_float(sw[2 * jj]), __uint_as_float(sw[2 * jj + 1]));
                } else {
#pragma unroll
                    for (int jj = 0; jj < RL; ++jj) sp[jj] = P.spec[g * RL + bitrev(jj, RL)];
                }
#pragma unroll
                for (int jj = 0; jj < RL; ++jj)
                    x[jj] = P.adjoint ? cmulc(x[jj], sp[jj]) : cmul(x[jj], sp[jj]);
                dit<RL>(x);
#pragma unroll
                for (int q = 0; q < RL; ++q) buf[sidx<V>(g * RL + q)] = x[q];
            }
        } else {
            // Last local pass (radix RL, stride 1), then the cross-CTA stage, then the first
            // inverse local pass.  In the cross stage each thread takes two consecutive
            // positions, so every access to another CTA's shared memory moves 16 bytes.
            // CTA k1 owns positions [k1 LC/C, (k1+1) LC/C).
            constexpr int PPC = LC / C;
            static_assert(PPC % (2 * NT) == 0, "two positions per thread");
            // float64: one complex value is already a 16-byte access, so a thread takes one
            // position at a time (half the registers of a pair)
            constexpr bool kPairs = sizeof(T) == 4;
            cg::cluster_group cl = cg::this_cluster();
#pragma unroll 1
            for (int g = tid; g < LC / RL; g += NT) {
                V x[RL];
#pragma unroll
                for (int q = 0; q < RL; ++q) x[q] = buf[sidx<V>(g * RL + q)];
                dif<RL>(x);
#pragma unroll
                for (int jj = 0; jj < RL; ++jj) buf[sidx<V>(g * RL + bitrev(jj, RL))] = x[jj];
            }
            cl.sync();
            if constexpr (!kPairs) {
#pragma unroll 1
                for (int pi = tid; pi < PPC; pi += NT) {
                    const int pos = k1 * PPC + pi;
                    const int sp = sidx<V>(pos);
                    V a[C], sc[C], twj[C];
#pragma unroll
                    for (int j = 0; j < C; ++j) a[j] = rbuf[j][sp];
                    const V tw = P.twx[pos];
#pragma unroll
                    for (int f = 0; f < C; ++f) sc[f] = P.spec[(int64_t)pos * C + f];
                    twj[0] = mk<V>(1, 0);
#pragma unroll
                    for (int j = 1; j < C; ++j) twj[j] = cmul(twj[j - 1], tw);
#pragma unroll
                    for (int j = 0; j < C; ++j) a[j] = cmul(a[j], twj[j]);
                    dif<C>(a);
#pragma unroll
                    for (int ff = 0; ff < C; ++ff) {
                        const V sv = sc[bitrev(ff, C)];
                        a[ff] = P.adjoint ? cmulc(a[ff], sv) : cmul(a[ff], sv);
                    }
                    dit<C>(a);
#pragma unroll
                    for (int j = 0; j < C; ++j) rbuf[j][sp] = cmulc(a[j], twj[j]);
                }
            }
            // float32: the pair (pos, pos+1) per thread and iteration.  Up to C = 4 the next
            // iteration's remote values are loaded before this iteration's results are stored
            // (other positions, so the early load reads final values): one remote round trip
            // overlaps the arithmetic.  (C = 8 has two iterations and no registers to spare.)
            constexpr bool kAhead = kPairs && C <= 4;
            V an[2][C];
            if constexpr (kAhead) cross_pair_load<C>(rbuf, k1 * PPC + 2 * tid, an);
#pragma unroll 1
            for (int pi = 2 * tid, it = 0; kPairs && pi < PPC; pi += 2 * NT, ++it) {
                const int pos = k1 * PPC + pi;  // even: the pair (pos, pos+1) is contiguous
                const bool swp = pair_swapped<V>(pos);
                const int sp = sidx<V>(pos) & ~1;
                V a[2][C], sc[2][C], tw[2];
                if constexpr (kAhead) {
#pragma unroll
                    for (int j = 0; j < C; ++j) {
                        a[0][j] = an[0][j];
                        a[1][j] = an[1][j];
                    }
                    if (pi + 2 * NT < PPC) cross_pair_load<C>(rbuf, pos + 2 * NT, an);
                } else {
                    cross_pair_load<C>(rbuf, pos, a);
                }
                using ST = SpecTmem<T, LOGLC, C, NT, 1, false>;
                if constexpr (STM) {
                    // twiddles and spectrum from this thread's tensor-memory slot
                    const uint32_t col = ts->spec_tmem +
                                         ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) +
                                         (uint32_t)((tid >> 7) * 128);
                    uint32_t wh[ST::head], wt[4];
                    tc::tmem_ld<ST::head>(col + it * ST::head, wh);
                    tc::tmem_ld<4>(col + ST::tail_col + it * 4, wt);
                    float fw[ST::words];
#pragma unroll
                    for (int i = 0; i < ST::words; ++i)
                        fw[i] = __uint_as_float(i < ST::head ? wh[i] : wt[i - ST::head]);
                    tw[0] = mk<V>(fw[0], fw[1]);
                    tw[1] = mk<V>(fw[2], fw[3]);
#pragma unroll
                    for (int u = 0; u < 2; ++u)
#pragma unroll
                        for (int f = 0; f < C; ++f)
                            sc[u][f] = mk<V>(fw[4 + 2 * (u * C + f)], fw[5 + 2 * (u * C + f)]);
                } else {
                    pair_load(P.twx + pos, tw[0], tw[1]);
#pragma unroll
                    for (int f = 0; f < C; f += 2) {
                        pair_load(P.spec + (int64_t)pos * C + f, sc[0][f], sc[0][f + 1]);
                        pair_load(P.spec + (int64_t)(pos + 1) * C + f, sc[1][f], sc[1][f + 1]);
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    V twj[C];
                    twj[0] = mk<V>(1, 0);
#pragma unroll
                    for (int j = 1; j < C; ++j) twj[j] = cmul(twj[j - 1], tw[u]);
#pragma unroll
                    for (int j = 0; j < C; ++j) a[u][j] = cmul(a[u][j], twj[j]);
                    dif<C>(a[u]);
#pragma unroll
                    for (int ff = 0; ff < C; ++ff) {
                        const V sv = sc[u][bitrev(ff, C)];
                        a[u][ff] = P.adjoint ? cmulc(a[u][ff], sv) : cmul(a[u][ff], sv);
                    }
                    dit<C>(a[u]);
#pragma unroll
                    for (int j = 0; j < C; ++j) a[u][j] = cmulc(a[u][j], twj[j]);
                }
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    if (swp)
                        pair_store(rbuf[j] + sp, a[1][j], a[0][j]);
                    else
                        pair_store(rbuf[j] + sp, a[0][j], a[1][j]);
                }
            }
            cl.sync();
#pragma unroll 1
            for (int g = tid; g < LC / RL; g += NT) {
                V x[RL];
#pragma unroll
                for (int p = 0; p < RL; ++p) x[bitrev(p, RL)] = buf[sidx<V>(g * RL + p)];
                dit<RL>(x);
#pragma unroll
                for (int q = 0; q < RL; ++q) buf[sidx<V>(g * RL + q)] = x[q];
            }
        }
        if constexpr (G.np() >= 3) {
            __syncthreads();
            middle_inv_open<G.np() - 2, LOGLC, R, NT, TC>(buf, twt, ts);
        }
        if constexpr (kAhead) {
#pragma unroll
            for (int q = 0; q < R / 2; ++q) ulp[q] = ur[tid + q * S0];
        }
        __syncthreads();
        // ---- inverse pass 0: outputs [0, LC/2) only, accumulate u_r o y
#pragma unroll
        for (int j = 0; j < J0; ++j) {
            const int o = tid + j * NT;
            V ul[R / 2];  // factor values before the pass: their L2 latency overlaps it
#pragma unroll
            for (int q = 0; q < R / 2; ++q) ul[q] = (kAhead && j == 0) ? ulp[q] : ur[o + q * S0];
            V x[R];
            {
                const TwPow<R, V> wp(w0[j]);
#pragma unroll
                for (int p = 0; p < R; ++p) x[bitrev(p, R)] = wp.mulc(buf[sidx<V>(o + p * S0)], p);
            }
            dit_halfout<R>(x);
            if constexpr (STM) {  // this group's R accumulator words, after the butterflies
                uint32_t aw[R];
                tc::tmem_ld<R>(acc_col + j * R, aw);
#pragma unroll
                for (int q = 0; q < R / 2; ++q)
                    acc[j][q] = mk<V>(__uint_as_float(aw[2 * q]), __uint_as_float(aw[2 * q + 1]));
            }
#pragma unroll
            for (int q = 0; q < R / 2; ++q) {
                const V uu = ul[q];
                if (P.full) {
                    acc[j][q].x = fma(uu.y * cpair, x[q].y, fma(uu.x, x[q].x, acc[j][q].x));
                } else {
                    acc[j][q].x = fma(uu.x, x[q].x, acc[j][q].x);
                    acc[j][q].y = fma(uu.y, x[q].y, acc[j][q].y);
                }
            }
            if constexpr (STM) {
                uint32_t aw[R];
#pragma unroll
                for (int q = 0; q < R / 2; ++q) {
                    aw[2 * q] = __float_as_uint(acc[j][q].x);
                    aw[2 * q + 1] = __float_as_uint(acc[j][q].y);
                }
                tc::tmem_st<R>(acc_col + j * R, aw);
            }
        }
        if constexpr (STM) tc::tmem_wait_st();
        // unconditional (the last rank term reloads its own values): a conditional load would
        // keep ul0 live across the whole loop body
        if constexpr (kAhead) load_ul0(r + 1 < r_end ? r + 1 : r);
        __syncthreads();
    }

    // ---- epilogue: beta = D1 w (forward) / D2 w (adjoint), row 0, write once
    if constexpr (STM) {
        uint32_t aw[32];
        tc::tmem_ld<32>(acc_col, aw);
#pragma unroll
        for (int j = 0; j < J0; ++j)
#pragma unroll
            for (int q = 0; q < R / 2; ++q)
                acc[j][q] = mk<V>(__uint_as_float(aw[2 * (j * (R / 2) + q)]),
                                  __uint_as_float(aw[2 * (j * (R / 2) + q) + 1]));
    }
    T g0 = T(0);
    if (P.row0 && P.adjoint && lead) g0 = in[0];
#pragma unroll
    for (int j = 0; j < J0; ++j) {
        const int o = tid + j * NT;
#pragma unroll
        for (int q = 0; q < R / 2; ++q) {
            const int64_t a = (int64_t)k1 + (int64_t)C * (o + q * S0);
            if (P.full) {
                if (a < n) {
                    T b = acc[j][q].x * P.dout[a];
                    if (P.row0 && P.adjoint) b += P.row0[a] * g0;
                    if (P.sign_out && (a & 1)) b = -b;
                    out[a] = b;
                }
                continue;
            }
            const int64_t i0 = 2 * a;
            if (i0 < n) {
                T b0 = acc[j][q].x * P.dout[i0];
                if (P.row0 && P.adjoint) b0 += P.row0[i0] * g0;
                out[i0] = b0;
                if (i0 + 1 < n) {
                    T b1 = acc[j][q].y * P.dout[i0 + 1];
                    if (P.row0 && P.adjoint) b1 += P.row0[i0 + 1] * g0;
                    if (P.sign_out) b1 = -b1;
                    out[i0 + 1] = b1;
                }
            }
        }
    }
    if (P.row0 && !P.adjoint && lead) {
        // beta_0 = sum_k A_0k alpha_k: block reduction, then across the cluster
        for (int off = 16; off > 0; off >>= 1) r0acc += __shfl_down_sync(0xffffffffu, r0acc, off);
        if ((tid & 31) == 0) red[tid >> 5] = r0acc;
        __syncthreads();
        if (tid == 0) {
            T s = T(0);
            for (int w = 0; w < NT / 32; ++w) s += red[w];
            red[0] = s;
        }
        if constexpr (C > 1) {
            cg::cluster_group cl = cg::this_cluster();
            cl.sync();
            if (k1 == 0 && tid == 0) {
                T s = T(0);
                for (int j = 0; j < C; ++j) s += *cl.map_shared_rank(&red[0], j);
                out[0] = s;
            }
            cl.sync();
        } else {
            __syncthreads();
            if (tid == 0) out[0] = red[0];
        }
    }
}

// Dense batches: cluster blockIdx.x / C converts vector blockIdx.x / C.  Ragged batches
// (RAGGED): persistent clusters take vectors of one FFT-length class from a work counter.
// Two kernels so that each inlines the per-vector body once (register pressure).
// Bytes of dynamic shared memory before the tensor-core passes' DFT matrices (FFT buffer,
// input pairs, twiddles), rounded up to 128, and the matrices' size (four 2R x 2R bfloat16).
template <typename V>
__host__ __device__ constexpr size_t exec_smem_base(int LOGLC, int R) {
    return ((size_t)(padded_len<V>(1 << LOGLC) + (1 << LOGLC) / 2 +
                     PassGeom{LOGLC, R}.twp_len()) * sizeof(V) + 127) / 128 * 128;
}
__host__ __device__ constexpr size_t tc_dft_bytes(int R) { return (size_t)4 * (2 * R) * (2 * R) * 2; }

template <typename V, int LOGLC, int R, int NT, bool TC>
constexpr size_t exec_smem();

template <typename T, int LOGLC, int R, int C, int NT, int MINB, bool RAGGED, bool TC>
__global__ void __launch_bounds__(NT, MINB) exec_kernel(const ExecParams<T> P) {
    using V = typename cx<T>::t;
    constexpr PassGeom G{LOGLC, R};
    constexpr int LC = G.LC();
    constexpr int S0 = LC / R;
    constexpr int J0 = S0 / NT;
    constexpr int TWP = G.twp_len();
    static_assert(G.np() >= 2, "local FFT needs at least two passes");
    static_assert(J0 >= 1 && S0 % NT == 0, "pass-0 groups must divide over threads");
    static_assert(!TC || std::is_same<T, float>::value, "tensor-core passes are float32");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    V* buf = reinterpret_cast<V*>(smem_raw);  // [LC] FFT buffer, padded rows
    V* vbuf = buf + padded_len<V>(LC);        // [LC/2] scaled input pairs
    V* twt = vbuf + LC / 2;                   // [TWP] middle-pass twiddles
    __shared__ T red[NT / 32];

    const int tid = threadIdx.x;
    int k1 = 0;
    if constexpr (C > 1) k1 = (int)cg::this_cluster().block_rank();
    for (int i = tid; i < TWP; i += NT) twt[i] = P.twp[i];

    // tensor-core passes: DFT matrices in shared memory, TMEM for A and D, one mbarrier
    constexpr int TCOLS = tc_cols(LOGLC, R, NT);
    __shared__ uint32_t tc_slot;
    __shared__ __align__(8) uint64_t tc_mbar[TC ? kTcMaxGroups * kTcMaxTilesPerGroup : 1];
    __shared__ int tc_fail;
    TcState tcs{};
    if constexpr (TC) {
        unsigned char* bsm = smem_raw + exec_smem_base<V>(LOGLC, R);
        tc_build_dft<R, NT>(bsm);
        tc::fence_proxy_async_smem();
        if (tid < 32) {
            tc::tmem_alloc(tc::smem_u32(&tc_slot), TCOLS);
            tc::tmem_relinquish();
        }
        if (tid < kTcMaxGroups * kTcMaxTilesPerGroup) tc::mbar_init(tc::smem_u32(&tc_mbar[tid]), 1);
        if (tid == 0) {
            tc::mbar_fence_init();
            tc_fail = 0;
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        tcs.tmem = tc_slot;
        tcs.bsm = tc::smem_u32(bsm);
        tcs.mbar = tc::smem_u32(&tc_mbar[0]);
        tcs.phase = 0;
        tcs.fail = &tc_fail;
        tcs.status = P.status;
        tcs.stall = P.tc_stall;
    }
    // float32 kernels with 32 points per thread: the spectrum values (and the cross stage's
    // twiddles) into tensor memory, once
    constexpr bool STM = SpecTmem<T, LOGLC, C, NT, MINB, TC>::on;
    __shared__ uint32_t stm_slot;
    if constexpr (STM) {
        using ST = SpecTmem<T, LOGLC, C, NT, MINB, TC>;
        static_assert(ST::cols == 512 || 3 * (exec_smem<V, LOGLC, R, NT, TC>() + 1024) > 233472,
                      "at most two CTAs of 256 columns per SM");
        constexpr int PPC = LC / C;
        if (tid < 32) {
            tc::tmem_alloc(tc::smem_u32(&stm_slot), ST::cols);
            tc::tmem_relinquish();
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        tcs.spec_tmem = stm_slot;
        const uint32_t col = tcs.spec_tmem + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) +
                             (uint32_t)((tid >> 7) * 128);
        if constexpr (ST::single) {
            // group i of the thread (g = tid + i NT) multiplies its point jj by
            // spec[g RL + bitrev(jj)]: words [2 (i RL + jj), +1]
            constexpr int RL = PassGeom{LOGLC, R}.rad(PassGeom{LOGLC, R}.np() - 1);
            constexpr int NG = LC / RL / NT;
            static_assert(NG * RL * 2 == 64, "64 spectrum words per thread");
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {  // two halves of 32 words
                uint32_t w[32];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int e = h * 16 + k;  // entry i RL + jj of the thread
                    const int i = e / RL, jj = e % RL;
                    const V v = P.spec[(tid + i * NT) * RL + bitrev(jj, RL)];
                    w[2 * k] = __float_as_uint(v.x);
                    w[2 * k + 1] = __float_as_uint(v.y);
                }
                tc::tmem_st<32>(col + h * 32, w);
            }
        }
#pragma unroll 1
        for (int it = 0; ST::cluster && it < ST::iters; ++it) {
            const int pos = k1 * PPC + 2 * tid + it * 2 * NT;
            // slot words: twiddles of the two positions, then their spectra [u][f]
            const float* tf = reinterpret_cast<const float*>(P.twx + pos);
            const float* sf = reinterpret_cast<const float*>(P.spec + (int64_t)pos * C);
            uint32_t wh[ST::head], wt[4];
#pragma unroll
            for (int i = 0; i < ST::words; ++i) {
                const uint32_t v = __float_as_uint(i < 4 ? tf[i] : sf[i - 4]);
                if (i < ST::head)
                    wh[i] = v;
                else
                    wt[i - ST::head] = v;
            }
            tc::tmem_st<ST::head>(col + it * ST::head, wh);
            tc::tmem_st<4>(col + ST::tail_col + it * 4, wt);
        }
        tc::tmem_wait_st();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if constexpr (!RAGGED) {
        const int64_t G = gridDim.x / C;
        const int64_t cid = blockIdx.x / C;
        const int64_t Ku = P.K > 0 ? P.K : 1;
        const int64_t U = P.batch * Ku;
        int64_t u = U * cid / G;
        const int64_t u1 = U * (cid + 1) / G;
        for (int it = 0; u < u1; ++it) {
            if (it > 0) __syncthreads();
            const int64_t vec = u / Ku, r0 = u % Ku;
            const int64_t r1 = r0 + u1 - u < Ku ? r0 + u1 - u : Ku;
            T* outp = (r0 == 0 && r1 == Ku) ? P.out + vec * P.n
                                            : P.partial + (2 * cid + (r0 == 0 ? 1 : 0)) * P.n;
            convert_vector<T, LOGLC, R, C, NT, TC, STM>(P, P.in + vec * P.n, outp, P.n, k1, buf, vbuf,
                                                   twt, red, r0, r1 < P.K ? r1 : P.K, r0 == 0,
                                                   &tcs);
            u += r1 - r0;
        }
    } else {
        __shared__ int slot[2];
        const int count = *P.count;
        for (int it = 0;; ++it) {
            if (k1 == 0 && tid == 0) slot[it & 1] = atomicAdd(P.next, 1);
            int sidx;
            if constexpr (C > 1) {
                cg::cluster_group cl = cg::this_cluster();
                cl.sync();
                sidx = *cl.map_shared_rank(&slot[it & 1], 0);
            } else {
                __syncthreads();
                sidx = slot[it & 1];
            }
            if (sidx >= count) break;
            const int64_t vec = P.list[sidx];
            const int64_t off = P.offs[vec];
            const int64_t n = P.offs[vec + 1] - off;
            convert_vector<T, LOGLC, R, C, NT, TC, STM>(P, P.in + off, P.out + off, n, k1, buf, vbuf,
                                                   twt, red, 0, P.K, true, &tcs);
        }
        if constexpr (C > 1) cg::this_cluster().sync();  // no CTA leaves while its slot is read
    }
    if constexpr (TC) {  // every tensor-memory access of the CTA is complete: free it
        tc::fence_before_sync();
        __syncthreads();
        if (tid < 32) {
            tc::fence_after_sync();
            tc::tmem_dealloc(tcs.tmem, TCOLS);
        }
    }
    if constexpr (STM) {
        tc::fence_before_sync();
        __syncthreads();
        if (tid < 32) {
            tc::fence_after_sync();
            tc::tmem_dealloc(tcs.spec_tmem, SpecTmem<T, LOGLC, C, NT, MINB, TC>::cols);
        }
    }
}

// Balanced split, second pass: each vector split between clusters is the sum of its pieces
// in cluster order (deterministic).  blockIdx.y + 1 = c indexes the boundary between clusters
// c-1 and c; the first boundary inside a vector owns it.
template <typename T>
__global__ void k_balance_fixup(const T* __restrict__ partial, T* __restrict__ out, int64_t n,
                                int64_t U, int64_t Ku, int64_t G) {
    const int64_t c = (int64_t)blockIdx.y + 1;
    const int64_t b = U * c / G;
    if (b % Ku == 0) return;
    const int64_t v = b / Ku;
    if (U * (c - 1) / G > v * Ku) return;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    T acc = partial[(2 * (c - 1) + 1) * n + k];
    for (int64_t cc = c; cc < G && U * cc / G < (v + 1) * Ku; ++cc) acc += partial[2 * cc * n + k];
    out[v * n + k] = acc;
}

// Dynamic shared memory of a launch.  Tensor-core kernels also hold the DFT matrices, and at
// least enough shared memory that the CTAs resident on one SM can never ask for more than the
// SM's 512 TMEM columns together (tcgen05.alloc would otherwise wait for another CTA's columns,
// and CTAs of a cluster waiting on each other could then never proceed): with at most
// k = 512 / TCOLS CTAs allowed, each takes more than 1/(k+1) of the SM's 228 KB.
template <typename V, int LOGLC, int R, int NT, bool TC>
constexpr size_t exec_smem() {
    if constexpr (!TC) {
        return (size_t)(padded_len<V>(1 << LOGLC) + (1 << LOGLC) / 2 +
                        PassGeom{LOGLC, R}.twp_len()) * sizeof(V);
    } else {
        const size_t need = exec_smem_base<V>(LOGLC, R) + tc_dft_bytes(R);
        const size_t k = (size_t)(512 / tc_cols(LOGLC, R, NT));
        const size_t floor_bytes = (size_t)233472 / (k + 1) - 1024 + 128;
        return need > floor_bytes ? need : floor_bytes;
    }
}

template <typename T, int LOGLC, int R, int C, int NT, int MINB, bool RAGGED, bool TC>
int launch_inst(const ExecParams<T>& P0, int64_t batch, cudaStream_t s) {
    using V = typename cx<T>::t;
    constexpr size_t smem = exec_smem<V, LOGLC, R, NT, TC>();
    static_assert(smem <= 232448, "shared memory budget");
    static_assert(!TC || tc_cols(LOGLC, R, NT) <= 512, "tensor memory budget");
    auto kern = exec_kernel<T, LOGLC, R, C, NT, MINB, RAGGED, TC>;
    static PerDevice attr_once;
    const cudaError_t attr_err = per_device(attr_once, [&](int*) {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (attr_err != cudaSuccess) {
        set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(attr_err));
        return TDH_ERR_CUDA;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(batch * C), 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (C > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    // persistent: as many clusters as can be resident (queried once per kernel and device)
    static PerDevice res_once;
    int resident = 0;
    const cudaError_t res_err = per_device(res_once, [&](int* out) {
        if (C > 1) return cudaOccupancyMaxActiveClusters(out, kern, &cfg);
        int per_sm = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
        *out = per_sm * sm_count();
        return e;
    }, &resident);
    if (res_err != cudaSuccess) {
        set_error("occupancy query: %s", cudaGetErrorString(res_err));
        return TDH_ERR_CUDA;
    }
    ExecParams<T> P = P0;
    if constexpr (RAGGED) {
        // at most one cluster per vector; vectors come from the class's work counter
        const int64_t nclusters = std::max<int64_t>(1, std::min<int64_t>(batch, resident));
        cfg.gridDim = dim3((unsigned)(nclusters * C), 1, 1);
        TDH_CUDA(cudaLaunchKernelEx(&cfg, kern, P));
        note_launches(1);
        return TDH_OK;
    } else {
        // balanced split: one wave of G clusters, at most one per (vector, rank term) unit
        const int64_t Ku = P.K > 0 ? P.K : 1;
        const int64_t U = batch * Ku;
        const int64_t G = std::max<int64_t>(1, std::min<int64_t>(U, resident));
        bool split = false;
        for (int64_t c = 1; c < G && !split; ++c) split = (U * c / G) % Ku != 0;
        P.batch = batch;
        P.partial = nullptr;
        if (split) {
            if (G - 1 > 65535) {
                set_error("balanced split: too many clusters");
                return TDH_ERR_UNSUPPORTED;
            }
            TDH_TRY(scratch_alloc(reinterpret_cast<void**>(&P.partial),
                                  sizeof(T) * (size_t)(2 * G) * (size_t)P.n, s));
        }
        cfg.gridDim = dim3((unsigned)(G * C), 1, 1);
        cudaError_t e = cudaLaunchKernelEx(&cfg, kern, P);
        if (e == cudaSuccess) note_launches(1);
        if (e == cudaSuccess && split) {
            dim3 fg((unsigned)((P.n + 255) / 256), (unsigned)(G - 1), 1);
            k_balance_fixup<T><<<fg, 256, 0, s>>>(P.partial, P.out, P.n, U, Ku, G);
            e = cudaGetLastError();
            if (e == cudaSuccess) note_launches(1);
        }
        if (P.partial) scratch_free(P.partial, s);
        TDH_CUDA(e);
        return TDH_OK;
    }
}

// Kernel instantiation for a geometry (switch over the built configurations).
// Table-driven dispatch: the kernel instantiation whose schedule equals g's.
template <typename T, bool RAGGED, int I = 0>
int dispatch_geom(const Geometry& g, const ExecParams<T>& P, int64_t batch, cudaStream_t s) {
    constexpr bool f32 = std::is_same<T, float>::value;
    if constexpr (I < SchedTable<f32>::size) {
        constexpr Sched e = SchedTable<f32>::at(I);
        if (g.logLC == e.logLC && g.C == e.C && g.NT == e.NT && g.MINB == e.MINB &&
            g.R == sched_radix(e, f32))
            return launch_inst<T, e.logLC, sched_radix(e, f32), e.C, e.NT, e.MINB, RAGGED,
                               false>(P, batch, s);
        return dispatch_geom<T, RAGGED, I + 1>(g, P, batch, s);
    } else {
        set_error("no %s kernel for local length 2^%d, cluster %d, %d threads, %d CTAs per SM",
                  f32 ? "float32" : "float64", g.logLC, g.C, g.NT, g.MINB);
        return TDH_ERR_UNSUPPORTED;
    }
}

// The same over the split-bfloat16 tensor-core instantiations.
template <bool RAGGED, int I = 0>
int dispatch_geom_tc(const Geometry& g, const ExecParams<float>& P, int64_t batch,
                     cudaStream_t s) {
    if constexpr (I < SchedTableTC::size) {
        constexpr Sched e = SchedTableTC::at(I);
        if (g.logLC == e.logLC && g.C == e.C && g.NT == e.NT && g.MINB == e.MINB &&
            g.R == sched_radix(e, true))
            return launch_inst<float, e.logLC, sched_radix(e, true), e.C, e.NT, e.MINB,
                               RAGGED, true>(P, batch, s);
        return dispatch_geom_tc<RAGGED, I + 1>(g, P, batch, s);
    } else {
        set_error("no split-bfloat16 kernel for local length 2^%d, cluster %d, %d threads, "
                  "%d CTAs per SM", g.logLC, g.C, g.NT, g.MINB);
        return TDH_ERR_UNSUPPORTED;
    }
}

// Defined in tdh_dense_f32/f64.cu and tdh_ragged_f32/f64.cu, one instantiation set each.
int dispatch_dense(const Geometry& g, const ExecParams<float>& P, int64_t batch, cudaStream_t s);
int dispatch_dense(const Geometry& g, const ExecParams<double>& P, int64_t batch, cudaStream_t s);
int dispatch_ragged(const Geometry& g, const ExecParams<float>& P, int64_t batch, cudaStream_t s);
int dispatch_ragged(const Geometry& g, const ExecParams<double>& P, int64_t batch, cudaStream_t s);
// Defined in tdh_dense_tc.cu and tdh_ragged_tc.cu (split-bfloat16 tensor-core passes).
int dispatch_dense_tc(const Geometry& g, const ExecParams<float>& P, int64_t batch, cudaStream_t s);
int dispatch_ragged_tc(const Geometry& g, const ExecParams<float>& P, int64_t batch, cudaStream_t s);

}  // namespace tdh
