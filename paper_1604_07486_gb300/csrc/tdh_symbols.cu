// Step a1: the split A = D1 (T o H) D2 of each conversion, from its closed form, in float64.
//
// Every generator entry is a scaled Gamma ratio Gamma(z + a) / Gamma(z + b) at z on a
// uniform grid.  Differences of log-gamma values lose about log10(z) digits at large z
// (the absolute error of lgamma(z) is ~ z log z ulp), so instead the pair is centred,
// Gamma(z+a)/Gamma(z+b) = Gamma(w+h)/Gamma(w-h) with w = z + (a+b)/2, h = (a-b)/2, and
//   w >= Zt:  Gamma(w+h)/Gamma(w-h) = w^(2h) exp(S(1/w)), with S the difference of the two
//             Stirling series, S = sum_k (-1)^(k+1) [B_{k+1}(h) - B_{k+1}(-h)] / (k(k+1) w^k)
//             (B_k the Bernoulli polynomials; the asymptotic ratio expansion the paper cites
//             from Tricomi & Erdelyi, used in the proof of Thm 3.2);
//   w <  Zt:  shift up with Gamma(x + 1) = x Gamma(x) until w >= Zt.
// The series terms behave like (h/w)^k and k!/(2 pi w)^k: with Zt = 16 + 4|a-b| and 16 terms
// the truncation error is below 1e-19 relative for any a, b (centring keeps large parameters,
// e.g. l = 17 in an ultraspherical symbol, out of the series).  The result carries the
// rounding of pow and exp, a few ulp.  The same routine runs on the host for the constant
// factors Gamma(x)/Gamma(y) (no overflow of Gamma itself for large x, y).
#include <cmath>
#include <cstdarg>
#include <vector>

#include "tdh_internal.cuh"

namespace tdh {
namespace {

constexpr int kTerms = 16;
constexpr double kZ0 = 16.0;

struct TableSpec {
    double a, b;         // ratio Gamma(z + a) / Gamma(z + b); ignored when no_ratio
    double cen, h, zt;   // centre (a+b)/2, half difference (a-b)/2, series threshold
    double z0, dz;       // z = z0 + dz * i
    double scale;        // overall factor
    double lin0, lin1;   // extra factor (lin0 + lin1 * i) when use_lin
    double special_v;    // value at index special_i (if special_i >= 0)
    int64_t special_i;
    int even_only;       // odd i -> 0
    int no_ratio;
    int use_lin;
    double c[kTerms];    // series coefficients of the (a, b) pair
};

// Bernoulli numbers B_0..B_{n} from sum_{j<=m} C(m+1, j) B_j = 0 (host, float64).
void bernoulli(double* B, int n) {
    B[0] = 1.0;
    for (int m = 1; m <= n; ++m) {
        double acc = 0.0, binom = 1.0;  // C(m+1, j)
        for (int j = 0; j < m; ++j) {
            acc += binom * B[j];
            binom = binom * (double)(m + 1 - j) / (double)(j + 1);
        }
        B[m] = -acc / (double)(m + 1);
    }
}

double bernoulli_poly(int n, double x, const double* B) {
    // B_n(x) = sum_j C(n, j) B_j x^(n-j)
    double acc = 0.0, binom = 1.0;
    for (int j = 0; j <= n; ++j) {
        acc += binom * B[j] * std::pow(x, (double)(n - j));
        binom = binom * (double)(n - j) / (double)(j + 1);
    }
    return acc;
}

void series_coeffs(double a, double b, double* c) {
    double B[kTerms + 2];
    bernoulli(B, kTerms + 1);
    for (int k = 1; k <= kTerms; ++k) {
        double sgn = (k % 2 == 1) ? 1.0 : -1.0;  // (-1)^(k+1)
        c[k - 1] = sgn * (bernoulli_poly(k + 1, a, B) - bernoulli_poly(k + 1, b, B)) /
                   ((double)k * (double)(k + 1));
    }
}

TableSpec ratio_spec(double a, double b, double z0, double dz, double scale) {
    TableSpec s{};
    s.a = a;
    s.b = b;
    s.cen = 0.5 * (a + b);
    s.h = 0.5 * (a - b);
    s.zt = kZ0 + 4.0 * std::fabs(a - b);
    s.z0 = z0;
    s.dz = dz;
    s.scale = scale;
    s.special_i = -1;
    series_coeffs(s.h, -s.h, s.c);
    return s;
}

TableSpec linear_spec(double scale, double lin0, double lin1) {
    TableSpec s{};
    s.scale = scale;
    s.no_ratio = 1;
    s.use_lin = 1;
    s.lin0 = lin0;
    s.lin1 = lin1;
    s.special_i = -1;
    return s;
}

__host__ __device__ double gamma_ratio(double z, const TableSpec& s) {
    double w = z + s.cen;
    double f = 1.0;
    if (w < s.zt) {
        const int N = (int)ceil(s.zt - w);
        double num = 1.0, den = 1.0;
        for (int i = 0; i < N; ++i) {
            num *= (w - s.h + (double)i);  // = z + b + i
            den *= (w + s.h + (double)i);  // = z + a + i
        }
        f = num / den;
        w += (double)N;
    }
    const double iw = 1.0 / w;
    double S = 0.0;
#pragma unroll
    for (int k = kTerms; k >= 1; --k) S = (S + s.c[k - 1]) * iw;
    return f * pow(w, 2.0 * s.h) * exp(S);
}

// Gamma(x) / Gamma(y) on the host (x, y not at poles).
double gratio(double x, double y) { return gamma_ratio(0.0, ratio_spec(x, y, 0.0, 1.0, 1.0)); }

__global__ void table_kernel(TableSpec s, int64_t count, double* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double v;
    if (i == s.special_i) {
        v = s.special_v;
    } else if (s.even_only && (i & 1)) {
        v = 0.0;
    } else {
        v = s.scale;
        if (!s.no_ratio) v *= gamma_ratio(s.z0 + s.dz * (double)i, s);
        if (s.use_lin) v *= (s.lin0 + s.lin1 * (double)i);
    }
    out[i] = v;
}

int launch_table(const TableSpec& s, int64_t count, double* out, cudaStream_t st) {
    if (count <= 0) return TDH_OK;
    int threads = 256;
    int64_t blocks = (count + threads - 1) / threads;
    table_kernel<<<(unsigned)blocks, threads, 0, st>>>(s, count, out);
    TDH_CUDA(cudaGetLastError());
    return TDH_OK;
}

bool is_nonpos_integer(double x) { return x <= 0.0 && std::floor(x) == x; }

}  // namespace

int chebyshev_scale_launch(int64_t n, int inverse, double* out, cudaStream_t st) {
    // Gamma(k + 1/2) / (Gamma(1/2) Gamma(k + 1)), or its reciprocal
    const double sqrtpi = 1.7724538509055160273;
    const TableSpec ts = inverse ? ratio_spec(1.0, 0.5, 0.0, 1.0, sqrtpi)
                                 : ratio_spec(0.5, 1.0, 0.0, 1.0, 1.0 / sqrtpi);
    return launch_table(ts, n, out, st);
}

int symbols_launch(int kind, int64_t n, const double* p, double* t, double* h, double* d1,
                   double* d2, cudaStream_t st) {
    const double pi = 3.14159265358979323846;
    int64_t nh = 2 * n - 1;
    switch (kind) {
    case TDH_LEG2CHEB: {
        // Eq. (7): T = Lambda((k-j)/2) for k-j even, H = Lambda((j+k)/2),
        // D1 = 2/pi diag(1/2, 1, ..., 1), D2 = I; Lambda(z) = Gamma(z+1/2)/Gamma(z+1).
        TableSpec ts = ratio_spec(0.5, 1.0, 0.0, 0.5, 1.0);
        ts.even_only = 1;
        TDH_TRY(launch_table(ts, n, t, st));
        TDH_TRY(launch_table(ratio_spec(0.5, 1.0, 0.0, 0.5, 1.0), nh, h, st));
        TableSpec s1 = linear_spec(2.0 / pi, 1.0, 0.0);
        s1.special_i = 0;
        s1.special_v = 1.0 / pi;
        TDH_TRY(launch_table(s1, n, d1, st));
        TDH_TRY(launch_table(linear_spec(1.0, 1.0, 0.0), n, d2, st));
        return TDH_OK;
    }
    case TDH_CHEB2LEG: {
        // Sec. 5.1: T = Gamma((m-1)/2)/Gamma((m+2)/2) (m = k-j even),
        // H = Gamma((j+k)/2)/Gamma((j+k+3)/2) with H_00 = 1,
        // D1 = diag(j + 1/2), D2 = -1/4 diag(4/sqrt(pi), 1, 2, ..., N).
        TableSpec ts = ratio_spec(-0.5, 1.0, 0.0, 0.5, 1.0);
        ts.even_only = 1;
        TDH_TRY(launch_table(ts, n, t, st));
        TableSpec hs = ratio_spec(0.0, 1.5, 0.0, 0.5, 1.0);
        hs.special_i = 0;
        hs.special_v = 1.0;
        TDH_TRY(launch_table(hs, nh, h, st));
        TDH_TRY(launch_table(linear_spec(1.0, 0.5, 1.0), n, d1, st));
        TableSpec s2 = linear_spec(-0.25, 0.0, 1.0);
        s2.special_i = 0;
        s2.special_v = -1.0 / std::sqrt(pi);
        TDH_TRY(launch_table(s2, n, d2, st));
        return TDH_OK;
    }
    case TDH_ULTRA2ULTRA: {
        // Sec. 5.2, Case 2 (|l1 - l2| < 1): T = Gamma(m/2 + d)/(Gamma(d) Gamma(m/2 + 1)),
        // d = l1 - l2 (reading: Gamma(d) divides); H = Gamma(l2) Gamma(s/2 + l1) /
        // (Gamma(l1) Gamma(s/2 + l2 + 1)); D1 = diag(j + l2), D2 = I.
        double l1 = p[0], l2 = p[1], d = l1 - l2;
        if (!(l1 > 0.0) || !(l2 > 0.0)) {
            set_error("ultraspherical parameters must be > 0 (got %g, %g)", l1, l2);
            return TDH_ERR_INVALID_ARG;
        }
        if (is_nonpos_integer(d) || !(std::fabs(d) < 1.0)) {
            set_error("tdh_symbols: ultraspherical split needs |l1 - l2| < 1, non-integer");
            return TDH_ERR_UNSUPPORTED;
        }
        TableSpec ts = ratio_spec(d, 1.0, 0.0, 0.5, 1.0 / std::tgamma(d));
        ts.even_only = 1;
        TDH_TRY(launch_table(ts, n, t, st));
        TDH_TRY(launch_table(ratio_spec(l1, l2 + 1.0, 0.0, 0.5, gratio(l2, l1)),
                             nh, h, st));
        TDH_TRY(launch_table(linear_spec(1.0, l2, 1.0), n, d1, st));
        TDH_TRY(launch_table(linear_spec(1.0, 1.0, 0.0), n, d2, st));
        return TDH_OK;
    }
    case TDH_JAC2JAC: {
        // Sec. 5.3, Case 2 with b == d: A_jk = E1(j) E2(k) T(k-j) G(k+j), each factor a Gamma
        // ratio normalised to 1 at index 0 (their product there is 1):
        //   E1(j) = (2j + s) Gamma(j+s)/Gamma(j+b+1) * Gamma(b+1)/Gamma(s+1),  s = g + b + 1
        //   E2(k) = Gamma(k+b+1)/Gamma(k+a+b+1) * Gamma(a+b+1)/Gamma(b+1)
        //   T(m)  = Gamma(m + a - g)/(Gamma(a - g) Gamma(m + 1))
        //   G(q)  = Gamma(q+a+b+1)/Gamma(q+s+1) * Gamma(s+1)/Gamma(a+b+1)
        double a = p[0], b = p[1], g = p[2];
        double s = g + b + 1.0;
        if (!(a > -1.0) || !(b > -1.0) || !(g > -1.0)) {
            set_error("Jacobi parameters must be > -1");
            return TDH_ERR_INVALID_ARG;
        }
        if (!(std::fabs(a - g) < 1.0) || is_nonpos_integer(a - g)) {
            set_error("tdh_symbols: Jacobi split needs |a - g| < 1, a != g (Cases 2 and 3)");
            return TDH_ERR_UNSUPPORTED;
        }
        TDH_TRY(launch_table(ratio_spec(a - g, 1.0, 0.0, 1.0, 1.0 / std::tgamma(a - g)), n, t, st));
        if (!(a + b > -1.0)) {
            // Case 3 (a + b <= -1): E2 and G touch Gamma(a+b+1) at index 0, where the two cancel
            // (A_00 = 1, applied directly).  Normalise both at index 1; their product there is
            // Gamma(s+1)/Gamma(b+1) * Gamma(b+2)/Gamma(s+2) = (b+1)/(s+1), carried by D1.
            // Index-0 entries of h and d2 are unused and set to 0.
            TableSpec hs = ratio_spec(a + b + 1.0, s + 1.0, 0.0, 1.0,
                                      gratio(s + 2.0, a + b + 2.0));
            hs.special_i = 0;
            hs.special_v = 0.0;
            TDH_TRY(launch_table(hs, nh, h, st));
            TableSpec e1 = ratio_spec(s, b + 1.0, 0.0, 1.0,
                                      (b + 1.0) / (s + 1.0) * gratio(b + 1.0, s + 1.0));
            e1.use_lin = 1;
            e1.lin0 = s;
            e1.lin1 = 2.0;
            e1.special_i = 0;
            e1.special_v = (b + 1.0) / (s + 1.0);
            TDH_TRY(launch_table(e1, n, d1, st));
            TableSpec e2 = ratio_spec(b + 1.0, a + b + 1.0, 0.0, 1.0,
                                      gratio(a + b + 2.0, b + 2.0));
            e2.special_i = 0;
            e2.special_v = 0.0;
            TDH_TRY(launch_table(e2, n, d2, st));
            return TDH_OK;
        }
        TDH_TRY(launch_table(ratio_spec(a + b + 1.0, s + 1.0, 0.0, 1.0,
                                        gratio(s + 1.0, a + b + 1.0)),
                             nh, h, st));
        TableSpec e1 = ratio_spec(s, b + 1.0, 0.0, 1.0, gratio(b + 1.0, s + 1.0));
        e1.use_lin = 1;
        e1.lin0 = s;
        e1.lin1 = 2.0;
        e1.special_i = 0;
        e1.special_v = 1.0;
        TDH_TRY(launch_table(e1, n, d1, st));
        TDH_TRY(launch_table(ratio_spec(b + 1.0, a + b + 1.0, 0.0, 1.0,
                                        gratio(a + b + 1.0, b + 1.0)),
                             n, d2, st));
        return TDH_OK;
    }
    case TDH_LAG2LAG: {
        // Sec. 5.4: A_jk = Gamma(k-j+d)/(Gamma(d) Gamma(k-j+1)), d = a1 - a2: a Toeplitz matrix,
        // i.e. T o H with H the matrix of all ones; D1 = D2 = I.
        const double d = p[0] - p[1];
        if (!(p[0] > -1.0) || !(p[1] > -1.0)) {
            set_error("Laguerre parameters must be > -1");
            return TDH_ERR_INVALID_ARG;
        }
        if (is_nonpos_integer(d)) {
            // 1/Gamma(d) = 0 with poles in the numerator: t_m = (-1)^m C(-d, m), m <= -d
            const int M = (int)(-d);
            std::vector<double> tm((size_t)std::min<int64_t>(n, M + 1));
            double c = 1.0;
            for (int m = 0; m < (int)tm.size(); ++m) {
                tm[m] = (m % 2 ? -c : c);
                c = c * (double)(M - m) / (double)(m + 1);
            }
            TDH_CUDA(cudaMemsetAsync(t, 0, sizeof(double) * n, st));
            TDH_CUDA(cudaMemcpyAsync(t, tm.data(), sizeof(double) * tm.size(), cudaMemcpyHostToDevice, st));
            TDH_CUDA(cudaStreamSynchronize(st));
        } else {
            TDH_TRY(launch_table(ratio_spec(d, 1.0, 0.0, 1.0, 1.0 / std::tgamma(d)), n, t, st));
        }
        TDH_TRY(launch_table(linear_spec(1.0, 1.0, 0.0), nh, h, st));
        TDH_TRY(launch_table(linear_spec(1.0, 1.0, 0.0), n, d1, st));
        TDH_TRY(launch_table(linear_spec(1.0, 1.0, 0.0), n, d2, st));
        return TDH_OK;
    }
    default:
        set_error("unknown kind %d", kind);
        return TDH_ERR_INVALID_ARG;
    }
}

}  // namespace tdh

extern "C" int tdh_symbols(int kind, int64_t n, const double* p, double* t, double* h,
                           double* d1, double* d2, void* stream) {
    tdh::clear_error();
    if (n < 1 || !t || !h || !d1 || !d2) {
        tdh::set_error("tdh_symbols: n >= 1 and non-NULL outputs required");
        return TDH_ERR_INVALID_ARG;
    }
    double zero[4] = {0, 0, 0, 0};
    return tdh::symbols_launch(kind, n, p ? p : zero, t, h, d1, d2, tdh::as_stream(stream));
}
