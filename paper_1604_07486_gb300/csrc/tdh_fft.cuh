// Register-level FFT building blocks for the execute kernels (float and double).
//
// A radix-R pass works on R complex values held in registers.  dif<R> is the
// decimation-in-frequency butterfly network: natural order in, bit-reversed order out,
// forward sign (omega = exp(-2 pi i / R)).  dit<R> is its exact inverse up to the factor R:
// bit-reversed order in, natural order out, conjugate twiddles.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace tdh {

template <typename T>
struct cx;
template <>
struct cx<float> {
    using t = float2;
};
template <>
struct cx<double> {
    using t = double2;
};

template <typename V>
__device__ __forceinline__ V mk(decltype(V::x) x, decltype(V::x) y) {
    V v;
    v.x = x;
    v.y = y;
    return v;
}
template <typename V>
__device__ __forceinline__ V cadd(V a, V b) {
    return mk<V>(a.x + b.x, a.y + b.y);
}
template <typename V>
__device__ __forceinline__ V csub(V a, V b) {
    return mk<V>(a.x - b.x, a.y - b.y);
}
// a * b
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
    return mk<V>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename V>
__device__ __forceinline__ V cmulc(V a, V b) {
    return mk<V>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
template <typename V>
__device__ __forceinline__ V conjv(V a) {
    return mk<V>(a.x, -a.y);
}
// componentwise product (used for the packed real pairs)
template <typename V>
__device__ __forceinline__ V cwmul(V a, V b) {
    return mk<V>(a.x * b.x, a.y * b.y);
}

// x * omega_{N}^{i} (FWD) or x * omega_{N}^{-i}, omega_N = exp(-2 pi i / N), N <= 32.
template <int N, int I, bool FWD, typename V>
__device__ __forceinline__ V rot(V x);

// Odd multiples of 2 pi / 32 (N = 32 only): cos and sin of pi/16 and 3 pi/16, then the
// symmetries of the circle.
template <int K32, bool FWD, typename V>
__device__ __forceinline__ V rot32_odd(V x) {
    using S = decltype(V::x);
    constexpr S ca = S(0.98078528040323044913);  // cos(pi/16)
    constexpr S sa = S(0.19509032201612826785);  // sin(pi/16)
    constexpr S cb = S(0.83146961230254523708);  // cos(3 pi/16)
    constexpr S sb = S(0.55557023301960222474);  // sin(3 pi/16)
    // angle t = 2 pi kk / 32, kk odd; forward multiplies by (cos t, -sin t)
    constexpr int kk = FWD ? K32 : (32 - K32) % 32;
    constexpr S cs[32] = {S(1), ca, S(0), cb, S(0), sb, S(0), sa, S(0), -sa, S(0), -sb, S(0), -cb,
                          S(0), -ca, S(0), -ca, S(0), -cb, S(0), -sb, S(0), -sa, S(0), sa, S(0),
                          sb, S(0), cb, S(0), ca};
    constexpr S sn[32] = {S(0), sa, S(0), sb, S(0), cb, S(0), ca, S(0), ca, S(0), cb, S(0), sb,
                          S(0), sa, S(0), -sa, S(0), -sb, S(0), -cb, S(0), -ca, S(0), -ca, S(0),
                          -cb, S(0), -sb, S(0), -sa};
    return mk<V>(fma(x.x, cs[kk], x.y * sn[kk]), fma(x.y, cs[kk], -x.x * sn[kk]));
}

template <int N, int I, bool FWD, typename V>
__device__ __forceinline__ V rot(V x) {
    using S = decltype(V::x);
    static_assert(N <= 32, "rotations up to omega_32");
    if constexpr ((I * 32 / N) % 2 == 1) return rot32_odd<(I * 32 / N) % 32, FWD>(x);
    constexpr int k = (I * 16 / N) % 16;  // angle in units of 2 pi / 16
    constexpr S c8 = S(0.70710678118654752440);
    constexpr S c1 = S(0.92387953251128675613);
    constexpr S s1 = S(0.38268343236508977173);
    // forward: multiply by exp(-2 pi i k / 16) = (cos, -sin)
    constexpr int kk = FWD ? k : (16 - k) % 16;
    if constexpr (kk == 0) {
        return x;
    } else if constexpr (kk == 4) {
        return mk<V>(x.y, -x.x);  // * (-i)
    } else if constexpr (kk == 8) {
        return mk<V>(-x.x, -x.y);
    } else if constexpr (kk == 12) {
        return mk<V>(-x.y, x.x);  // * (+i)
    } else if constexpr (kk == 2) {
        return mk<V>(c8 * (x.x + x.y), c8 * (x.y - x.x));
    } else if constexpr (kk == 6) {
        return mk<V>(c8 * (x.y - x.x), -c8 * (x.x + x.y));
    } else if constexpr (kk == 10) {
        return mk<V>(-c8 * (x.x + x.y), c8 * (x.x - x.y));
    } else if constexpr (kk == 14) {
        return mk<V>(c8 * (x.x - x.y), c8 * (x.x + x.y));
    } else {
        // odd multiples of pi/8: (cos t, -sin t) with t = 2 pi kk / 16
        constexpr S cs[16] = {S(1), c1, c8, s1, S(0), -s1, -c8, -c1, S(-1), -c1, -c8, -s1, S(0), s1, c8, c1};
        constexpr S sn[16] = {S(0), s1, c8, c1, S(1), c1, c8, s1, S(0), -s1, -c8, -c1, S(-1), -c1, -c8, -s1};
        return mk<V>(fma(x.x, cs[kk], x.y * sn[kk]), fma(x.y, cs[kk], -x.x * sn[kk]));
    }
}

template <int R, int H, int BLK, int I, typename V>
__device__ __forceinline__ void dif_bfly(V (&x)[R]) {
    V a = x[BLK + I], b = x[BLK + I + H];
    x[BLK + I] = cadd(a, b);
    x[BLK + I + H] = rot<2 * H, I, true>(csub(a, b));
}

template <int R, int H, int BLK, int I, typename V>
__device__ __forceinline__ void dit_bfly(V (&x)[R]) {
    V a = x[BLK + I];
    V b = rot<2 * H, I, false>(x[BLK + I + H]);
    x[BLK + I] = cadd(a, b);
    x[BLK + I + H] = csub(a, b);
}

template <int R, int H, int BLK, typename V, int... I>
__device__ __forceinline__ void dif_blk(V (&x)[R], std::integer_sequence<int, I...>) {
    (dif_bfly<R, H, BLK, I>(x), ...);
}
template <int R, int H, int BLK, typename V, int... I>
__device__ __forceinline__ void dit_blk(V (&x)[R], std::integer_sequence<int, I...>) {
    (dit_bfly<R, H, BLK, I>(x), ...);
}
template <int R, int H, typename V, int... B>
__device__ __forceinline__ void dif_stage(V (&x)[R], std::integer_sequence<int, B...>) {
    (dif_blk<R, H, B * 2 * H>(x, std::make_integer_sequence<int, H>{}), ...);
}
template <int R, int H, typename V, int... B>
__device__ __forceinline__ void dit_stage(V (&x)[R], std::integer_sequence<int, B...>) {
    (dit_blk<R, H, B * 2 * H>(x, std::make_integer_sequence<int, H>{}), ...);
}

template <int R, int H, typename V>
__device__ __forceinline__ void dif_from(V (&x)[R]) {
    if constexpr (H >= 1) {
        dif_stage<R, H>(x, std::make_integer_sequence<int, R / (2 * H)>{});
        dif_from<R, H / 2>(x);
    }
}
template <int R, int H, int HMAX, typename V>
__device__ __forceinline__ void dit_range(V (&x)[R]) {
    if constexpr (H <= HMAX) {
        dit_stage<R, H>(x, std::make_integer_sequence<int, R / (2 * H)>{});
        dit_range<R, H * 2, HMAX>(x);
    }
}

// Full networks.
template <int R, typename V>
__device__ __forceinline__ void dif(V (&x)[R]) {
    dif_from<R, R / 2>(x);
}
template <int R, typename V>
__device__ __forceinline__ void dit(V (&x)[R]) {
    dit_range<R, 1, R / 2>(x);
}
// dif with x[R/2..R) known to be zero: the first stage reduces to x[i+R/2] = w^i x[i].
template <int R, typename V, int... I>
__device__ __forceinline__ void dif_half_first(V (&x)[R], std::integer_sequence<int, I...>) {
    ((x[I + R / 2] = rot<R, I, true>(x[I])), ...);
}
template <int R, typename V>
__device__ __forceinline__ void dif_halfzero(V (&x)[R]) {
    if constexpr (R == 1) {
        return;
    } else {
        dif_half_first<R>(x, std::make_integer_sequence<int, R / 2>{});
        dif_from<R, R / 4>(x);
    }
}
// dit producing only outputs [0, R/2): the last stage keeps the sums.
template <int R, typename V, int... I>
__device__ __forceinline__ void dit_half_last(V (&x)[R], std::integer_sequence<int, I...>) {
    ((x[I] = cadd(x[I], rot<R, I, false>(x[I + R / 2]))), ...);
}
template <int R, typename V>
__device__ __forceinline__ void dit_halfout(V (&x)[R]) {
    if constexpr (R == 1) {
        return;
    } else {
        dit_range<R, 1, R / 4>(x);
        dit_half_last<R>(x, std::make_integer_sequence<int, R / 2>{});
    }
}

__host__ __device__ constexpr int bitrev(int j, int R) {
    int r = 0;
    for (int b = 1; b < R; b <<= 1) {
        r = (r << 1) | (j & 1);
        j >>= 1;
    }
    return r;
}

__host__ __device__ constexpr int ilog2(int x) {
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

}  // namespace tdh
