/*
 * Dense CPU oracle for polynomial basis conversion beta = A alpha.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct reference that
 * the CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline legs of bench.py may load it.  It shares no code, header, table or constant
 * generator with the CUDA library, and the CUDA library never calls it.
 *
 * Source: Townsend, Webb & Olver, "Fast polynomial transforms based on Toeplitz and
 * Hankel matrices" (arXiv:1604.07486).  The oracle is the paper's "Direct" algorithm
 * (Sec. 4): every entry A_jk is generated from its closed form and dotted with alpha,
 * O(n^2) work and O(n) memory.  The closed forms are
 *   LEG2CHEB   Eq. (2)            M_jk
 *   CHEB2LEG   Eq. (11)     L_jk
 *   ULTRA      Eq. (13), Sec. 5.2
 *   JAC        the Jacobi formula of Sec. 5.3 (beta = delta), Cases 2 and 3
 *   LAG        the Laguerre formula of Sec. 5.4
 * together with the paper's diagonal/Toeplitz/Hankel split of each (Eq. (7),
 * Sec. 5.1, 5.2, 5.3), exported separately so that tests can check the split identity.
 *
 * Precision.  Every Gamma ratio the formulas need is produced by its first-order
 * recurrence Gamma(z+1) = z Gamma(z), started from an exact value, in double-double
 * arithmetic (about 106 bits); entries and the row sums are also formed in double-double
 * and rounded once at the end.  Double-double follows Dekker (1971) and Knuth (TAOCP
 * vol. 2, Sec. 4.2.2): two-sum, Veltkamp splitting and Dekker's exact product.  No
 * fused multiply-add is used, so results are identical on x86-64 and aarch64 when built
 * with -ffp-contract=off.
 *
 * Reading where the paper is garbled: Eq. (2) states the j = 0 row for "j even"; the
 * row is nonzero for k even (j = 0 is always even), which is what exact conversion
 * gives.  The ultraspherical T of Sec. 5.2 prints Gamma(lambda1-lambda2) in the
 * numerator; the reading that matches Eq. (13) divides by it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ double-double */

typedef struct { double hi, lo; } dd;

/* Knuth's two-sum: s + e == a + b exactly. */
static inline dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    dd r = {s, e};
    return r;
}

/* Dekker's fast two-sum, valid when |a| >= |b| (or a == 0). */
static inline dd fast_two_sum(double a, double b) {
    double s = a + b;
    double e = b - (s - a);
    dd r = {s, e};
    return r;
}

/* Veltkamp split of a double into two 26-bit halves. */
static inline void split(double a, double* h, double* l) {
    const double c = 134217729.0; /* 2^27 + 1 */
    double t = c * a;
    *h = t - (t - a);
    *l = a - *h;
}

/* Dekker's exact product: p + e == a * b exactly (barring overflow). */
static inline dd two_prod(double a, double b) {
    double p = a * b;
    double ah, al, bh, bl;
    split(a, &ah, &al);
    split(b, &bh, &bl);
    double e = ((ah * bh - p) + ah * bl + al * bh) + al * bl;
    dd r = {p, e};
    return r;
}

static inline dd dd_from(double a) { dd r = {a, 0.0}; return r; }

static inline dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

static inline dd dd_neg(dd a) { dd r = {-a.hi, -a.lo}; return r; }
static inline dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

static inline dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p.hi, p.lo);
}

static inline dd dd_mul_d(dd a, double b) {
    dd p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return fast_two_sum(p.hi, p.lo);
}

/* Long division: three quotient digits, each corrected against the remainder. */
static inline dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul_d(b, q1));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul_d(b, q2));
    double q3 = r.hi / b.hi;
    dd q = fast_two_sum(q1, q2);
    return dd_add(q, dd_from(q3));
}

/* Square root by one Newton correction of the double estimate, in double-double. */
static inline dd dd_sqrt(dd a) {
    if (a.hi <= 0.0) return dd_from(0.0);
    double x = sqrt(a.hi);
    dd xx = two_prod(x, x);
    dd r = dd_sub(a, xx);
    double corr = r.hi / (2.0 * x);
    return fast_two_sum(x, corr);
}

static inline double dd_round(dd a) { return a.hi + a.lo; }

/* pi to double-double precision (pi = 3.14159265358979323846264338327950288...). */
static dd dd_pi(void) { dd r = {3.141592653589793116, 1.2246467991473532072e-16}; return r; }

/* ------------------------------------------------------------------ kinds */

enum { K_LEG2CHEB = 0, K_CHEB2LEG = 1, K_ULTRA = 2, K_JAC = 3, K_LAG = 4 };

typedef struct {
    int kind;
    int64_t n;
    double prm[4];
    /* tables, all double-double */
    dd* lam;      /* LEG2CHEB/CHEB2LEG: lam[i] = Lambda(i/2), i in [0, 2n+2) */
    dd* P;        /* ULTRA: P'(m) = Gamma(m+d)/(Gamma(d) Gamma(m+1)), m in [0, n]
                     JAC/LAG: T(m) = Gamma(m+a-g)/(Gamma(a-g) Gamma(m+1)), m in [0, n]   */
    dd* Q;        /* ULTRA: Q'(m) = Gamma(l2) Gamma(m+l1) / (Gamma(l1) Gamma(m+l2+1)), m in [0, n] */
    dd* E1;       /* JAC: normalised row factor, j in [0, n)     */
    dd* E2;       /* JAC: normalised column factor, k in [0, n)  */
    dd* G;        /* JAC: normalised Hankel factor, q in [0, 2n) */
    dd c_row0, c_rest; /* LEG2CHEB constants 1/pi and 2/pi; JAC: constant factor */
    int case3;         /* JAC with a + b <= -1 (factors normalised at index 1) */
    dd sqrtpi;
} tables;

/*
 * Lambda(z) = Gamma(z + 1/2) / Gamma(z + 1) at z = i/2 (Eq. (2)).
 * Integer z: Lambda(0) = sqrt(pi); half-integer z: Lambda(1/2) = Gamma(1)/Gamma(3/2) = 2/sqrt(pi).
 * Both chains advance by Lambda(z+1) = Lambda(z) (z + 1/2) / (z + 1).
 */
static void build_lambda(dd* lam, int64_t count, dd sqrtpi) {
    if (count > 0) lam[0] = sqrtpi;
    if (count > 1) lam[1] = dd_div(dd_from(2.0), sqrtpi);
    for (int64_t i = 2; i < count; ++i) {
        double z = 0.5 * (double)(i - 2); /* lam[i] = Lambda(z + 1), lam[i-2] = Lambda(z) */
        dd num = dd_from(z + 0.5);
        dd den = dd_from(z + 1.0);
        lam[i] = dd_div(dd_mul(lam[i - 2], num), den);
    }
}

static int build_tables(tables* tb, int kind, const double* prm, int64_t n) {
    memset(tb, 0, sizeof(*tb));
    tb->kind = kind;
    tb->n = n;
    if (prm) memcpy(tb->prm, prm, sizeof(tb->prm));
    dd pi = dd_pi();
    tb->sqrtpi = dd_sqrt(pi);
    if (kind == K_LEG2CHEB || kind == K_CHEB2LEG) {
        int64_t cnt = 2 * n + 2;
        tb->lam = (dd*)malloc(sizeof(dd) * (size_t)cnt);
        if (!tb->lam) return -1;
        build_lambda(tb->lam, cnt, tb->sqrtpi);
        tb->c_row0 = dd_div(dd_from(1.0), pi);
        tb->c_rest = dd_div(dd_from(2.0), pi);
        return 0;
    }
    if (kind == K_ULTRA) {
        double l1 = prm[0], l2 = prm[1], d = l1 - l2;
        tb->P = (dd*)malloc(sizeof(dd) * (size_t)(n + 1));
        tb->Q = (dd*)malloc(sizeof(dd) * (size_t)(n + 1));
        if (!tb->P || !tb->Q) return -1;
        /* P'(0) = 1, P'(m+1) = P'(m) (m + d) / (m + 1) */
        tb->P[0] = dd_from(1.0);
        for (int64_t m = 0; m < n; ++m)
            tb->P[m + 1] = dd_div(dd_mul(tb->P[m], dd_add(dd_from((double)m), dd_from(d))),
                                  dd_from((double)(m + 1)));
        /* Q'(0) = Gamma(l2)/Gamma(l2+1) = 1/l2, Q'(m+1) = Q'(m) (m + l1) / (m + l2 + 1) */
        tb->Q[0] = dd_div(dd_from(1.0), dd_from(l2));
        for (int64_t m = 0; m < n; ++m)
            tb->Q[m + 1] = dd_div(dd_mul(tb->Q[m], dd_add(dd_from((double)m), dd_from(l1))),
                                  dd_add(dd_from((double)m + 1.0), dd_from(l2)));
        return 0;
    }
    if (kind == K_JAC) {
        double a = prm[0], b = prm[1], g = prm[2];
        double s = g + b + 1.0;
        tb->P = (dd*)malloc(sizeof(dd) * (size_t)(n + 1));
        tb->E1 = (dd*)malloc(sizeof(dd) * (size_t)n);
        tb->E2 = (dd*)malloc(sizeof(dd) * (size_t)n);
        tb->G = (dd*)malloc(sizeof(dd) * (size_t)(2 * n));
        if (!tb->P || !tb->E1 || !tb->E2 || !tb->G) return -1;
        /* T(m) = Gamma(m + a - g) / (Gamma(a - g) Gamma(m + 1)) */
        tb->P[0] = dd_from(1.0);
        for (int64_t m = 0; m < n; ++m)
            tb->P[m + 1] = dd_div(dd_mul(tb->P[m], dd_add(dd_from((double)m), dd_from(a - g))),
                                  dd_from((double)(m + 1)));
        /*
         * Row factor (2j+s) Gamma(j+s)/Gamma(j+b+1), normalised by its j = 0 value
         * Gamma(s+1)/Gamma(b+1):
         *   E1(0) = 1,  E1(j) = (2j + s) F(j) for j >= 1, where
         *   F(j) = prod_{i=1}^{j-1} (s + i) / prod_{i=0}^{j-1} (b + 1 + i).
         * Written this way it stays finite at s = 0 (the Chebyshev target).
         */
        if (n > 0) tb->E1[0] = dd_from(1.0);
        dd F = dd_div(dd_from(1.0), dd_from(b + 1.0));
        for (int64_t j = 1; j < n; ++j) {
            if (j > 1) {
                F = dd_mul(F, dd_add(dd_from(s), dd_from((double)(j - 1))));
                F = dd_div(F, dd_add(dd_from(b + 1.0), dd_from((double)(j - 1))));
            }
            tb->E1[j] = dd_mul(F, dd_add(dd_from(2.0 * (double)j), dd_from(s)));
        }
        if (a + b + 1.0 > 0.0) {
            /* Column factor Gamma(k+b+1)/Gamma(k+a+b+1), normalised by its k = 0 value. */
            if (n > 0) tb->E2[0] = dd_from(1.0);
            for (int64_t k = 0; k + 1 < n; ++k)
                tb->E2[k + 1] = dd_div(dd_mul(tb->E2[k], dd_add(dd_from((double)k), dd_from(b + 1.0))),
                                       dd_add(dd_from((double)k), dd_from(a + b + 1.0)));
            /* Hankel factor Gamma(q+a+b+1)/Gamma(q+s+1), normalised by its q = 0 value. */
            tb->G[0] = dd_from(1.0);
            for (int64_t q = 0; q + 1 < 2 * n; ++q)
                tb->G[q + 1] = dd_div(dd_mul(tb->G[q], dd_add(dd_from((double)q), dd_from(a + b + 1.0))),
                                      dd_add(dd_from((double)q), dd_from(s + 1.0)));
            tb->c_rest = dd_from(1.0);
            tb->case3 = 0;
        } else {
            /* Case 3 (a + b <= -1): the column and Hankel factors touch Gamma(a+b+1) at index
               0, where they cancel (A_00 = 1).  Normalise them at index 1 instead; their values
               there multiply to Gamma(s+1)/Gamma(b+1) * Gamma(b+2)/Gamma(s+2) = (b+1)/(s+1),
               kept as a separate constant.  Entries with index 0 of these factors are unused. */
            tb->E2[0] = dd_from(0.0);
            if (n > 1) tb->E2[1] = dd_from(1.0);
            for (int64_t k = 1; k + 1 < n; ++k)
                tb->E2[k + 1] = dd_div(dd_mul(tb->E2[k], dd_add(dd_from((double)k), dd_from(b + 1.0))),
                                       dd_add(dd_from((double)k), dd_from(a + b + 1.0)));
            tb->G[0] = dd_from(0.0);
            if (2 * n > 1) tb->G[1] = dd_from(1.0);
            for (int64_t q = 1; q + 1 < 2 * n; ++q)
                tb->G[q + 1] = dd_div(dd_mul(tb->G[q], dd_add(dd_from((double)q), dd_from(a + b + 1.0))),
                                      dd_add(dd_from((double)q), dd_from(s + 1.0)));
            tb->c_rest = dd_div(dd_from(b + 1.0), dd_from(s + 1.0));
            tb->case3 = 1;
        }
        return 0;
    }
    if (kind == K_LAG) {
        double d = prm[0] - prm[1];
        tb->P = (dd*)malloc(sizeof(dd) * (size_t)(n + 1));
        if (!tb->P) return -1;
        tb->P[0] = dd_from(1.0);
        for (int64_t m = 0; m < n; ++m)
            tb->P[m + 1] = dd_div(dd_mul(tb->P[m], dd_add(dd_from((double)m), dd_from(d))),
                                  dd_from((double)(m + 1)));
        return 0;
    }
    return -2;
}

static void free_tables(tables* tb) {
    free(tb->lam);
    free(tb->P);
    free(tb->Q);
    free(tb->E1);
    free(tb->E2);
    free(tb->G);
    memset(tb, 0, sizeof(*tb));
}

/*
 * A_jk from the closed forms.  Returns zero outside the upper triangle and, for the
 * parity-structured kinds, where k - j is odd.
 */
static inline dd entry(const tables* tb, int64_t j, int64_t k) {
    dd zero = dd_from(0.0);
    if (k < j) return zero;
    switch (tb->kind) {
    case K_LEG2CHEB: {
        /* Eq. (2): M_0k = Lambda(k/2)^2 / pi (k even); M_jk = 2/pi Lambda((k-j)/2) Lambda((k+j)/2). */
        if ((k - j) & 1) return zero;
        if (j == 0) return dd_mul(tb->c_row0, dd_mul(tb->lam[k], tb->lam[k]));
        return dd_mul(tb->c_rest, dd_mul(tb->lam[k - j], tb->lam[k + j]));
    }
    case K_CHEB2LEG: {
        /* Eq. (11). */
        if ((k - j) & 1) return zero;
        if (j == k) {
            if (j == 0) return dd_from(1.0);
            return dd_div(tb->sqrtpi, dd_mul_d(tb->lam[2 * j], 2.0));
        }
        /* -k (j + 1/2) Lambda((k-j-2)/2)/(k-j) * Lambda((j+k-1)/2)/(j+k+1) */
        dd f1 = dd_div(tb->lam[k - j - 2], dd_from((double)(k - j)));
        dd f2 = dd_div(tb->lam[j + k - 1], dd_from((double)(j + k + 1)));
        dd c = dd_mul(dd_from(-(double)k), dd_add(dd_from((double)j), dd_from(0.5)));
        return dd_mul(c, dd_mul(f1, f2));
    }
    case K_ULTRA: {
        /* Eq. (13): (j + l2) P'((k-j)/2) Q'((k+j)/2), k - j even. */
        if ((k - j) & 1) return zero;
        dd c = dd_add(dd_from((double)j), dd_from(tb->prm[1]));
        return dd_mul(c, dd_mul(tb->P[(k - j) / 2], tb->Q[(k + j) / 2]));
    }
    case K_JAC: {
        /* Sec. 5.3, normalised factors: c E1(j) E2(k) T(k-j) G(k+j); A_00 = 1. */
        if (tb->case3 && k == 0) return dd_from(1.0);
        dd v = dd_mul(dd_mul(tb->E1[j], tb->E2[k]), dd_mul(tb->P[k - j], tb->G[k + j]));
        return tb->case3 ? dd_mul(v, tb->c_rest) : v;
    }
    case K_LAG: {
        /* Sec. 5.4: Gamma(k-j+d) / (Gamma(d) Gamma(k-j+1)). */
        return tb->P[k - j];
    }
    }
    return zero;
}

/* --------------------------------------------------------------- exported API */

static int set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) return nthreads;
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/*
 * y[b][r] = sum_k A_{row_r, k} x[b][k]        (transpose == 0)
 * y[b][r] = sum_j A_{j, row_r} x[b][j]        (transpose == 1, the adjoint A^T)
 * rows == NULL means every index 0..n-1 (then nrows must equal n).
 * x has leading dimension ldx, y has leading dimension ldy.  Returns 0 or a negative code.
 */
int tdho_matvec(int kind, const double* prm, int64_t n, const double* x, int64_t batch,
                int64_t ldx, const int64_t* rows, int64_t nrows, double* y, int64_t ldy,
                int transpose, int nthreads) {
    if (n < 1 || batch < 0 || nrows < 0) return -1;
    tables tb;
    int rc = build_tables(&tb, kind, prm, n);
    if (rc) { free_tables(&tb); return rc; }
    int nt = set_threads(nthreads);
    int64_t total = batch * nrows;
    int64_t it;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (it = 0; it < total; ++it) {
        int64_t b = it / nrows, r = it % nrows;
        int64_t i = rows ? rows[r] : r;
        const double* xb = x + b * ldx;
        dd acc = dd_from(0.0);
        if (i >= 0 && i < n) {
            if (!transpose) {
                for (int64_t k = i; k < n; ++k) {
                    double xv = xb[k];
                    if (xv == 0.0) continue;
                    acc = dd_add(acc, dd_mul_d(entry(&tb, i, k), xv));
                }
            } else {
                for (int64_t j = 0; j <= i; ++j) {
                    double xv = xb[j];
                    if (xv == 0.0) continue;
                    acc = dd_add(acc, dd_mul_d(entry(&tb, j, i), xv));
                }
            }
        }
        y[b * ldy + r] = dd_round(acc);
    }
    free_tables(&tb);
    return 0;
}

/* Dense block out[(j - j0) * (k1 - k0) + (k - k0)] = A_jk, rounded once to double. */
int tdho_entries(int kind, const double* prm, int64_t n, int64_t j0, int64_t j1, int64_t k0,
                 int64_t k1, double* out) {
    if (n < 1 || j0 < 0 || k0 < 0 || j1 > n || k1 > n || j1 < j0 || k1 < k0) return -1;
    tables tb;
    int rc = build_tables(&tb, kind, prm, n);
    if (rc) { free_tables(&tb); return rc; }
    for (int64_t j = j0; j < j1; ++j)
        for (int64_t k = k0; k < k1; ++k)
            out[(j - j0) * (k1 - k0) + (k - k0)] = dd_round(entry(&tb, j, k));
    free_tables(&tb);
    return 0;
}

/*
 * The paper's split A = D1 (T o H) D2 (Fig. 1 step 1), as generator sequences:
 *   t[m]  = T_{j, j+m}, m in [0, n)          (upper-triangular Toeplitz)
 *   h[s]  = H_{jk} with j + k = s, s in [0, 2n-1)
 *   d1[j], d2[k], j, k in [0, n)
 * LEG2CHEB   Eq. (7): D1 = 2/pi diag(1/2, 1, ...), D2 = I,
 *            t_m = Lambda(m/2) (m even, else 0), h_s = Lambda(s/2).
 * CHEB2LEG   Sec. 5.1: D1 = diag(j + 1/2), D2 = -1/4 diag(4/sqrt(pi), 1, 2, ..., N),
 *            t_m = Gamma((m-1)/2)/Gamma((m+2)/2) (m even), h_s = Gamma(s/2)/Gamma((s+3)/2), h_0 = 1.
 * ULTRA      Sec. 5.2: D1 = diag(j + l2), D2 = I, t_m = P'(m/2) (m even),
 *            h_s = Q'(s/2); at odd s, Q'(s/2) starts from Gamma values computed in double.
 * JAC        Sec. 5.3: D1 = E1, D2 = E2, t = T, h = G (Case 3: normalised at index 1, index-0
 *            entries of D2 and h unused and set to 0, the constant (b+1)/(s+1) in D1).
 * LAG        Sec. 5.4: D1 = D2 = I, t = T, h = 1.
 */
int tdho_split(int kind, const double* prm, int64_t n, double* t, double* h, double* d1,
               double* d2) {
    if (n < 1) return -1;
    tables tb;
    int rc = build_tables(&tb, kind, prm, n);
    if (rc) { free_tables(&tb); return rc; }
    int64_t nh = 2 * n - 1;
    switch (kind) {
    case K_LEG2CHEB: {
        for (int64_t m = 0; m < n; ++m) t[m] = (m & 1) ? 0.0 : dd_round(tb.lam[m]);
        for (int64_t s = 0; s < nh; ++s) h[s] = dd_round(tb.lam[s]);
        for (int64_t j = 0; j < n; ++j) {
            d1[j] = dd_round(j == 0 ? tb.c_row0 : tb.c_rest);
            d2[j] = 1.0;
        }
        break;
    }
    case K_CHEB2LEG: {
        /* t at m = 2i: tau(i) = Gamma(i - 1/2)/Gamma(i + 1); tau(0) = Gamma(-1/2) = -2 sqrt(pi). */
        dd tau = dd_mul_d(tb.sqrtpi, -2.0);
        for (int64_t m = 0; m < n; ++m) {
            if (m & 1) { t[m] = 0.0; continue; }
            int64_t i = m / 2;
            t[m] = dd_round(tau);
            tau = dd_div(dd_mul(tau, dd_from((double)i - 0.5)), dd_from((double)i + 1.0));
        }
        /* h at s = 2i (i >= 1): Gamma(i)/Gamma(i + 3/2), start 1/Gamma(5/2) = 4/(3 sqrt(pi)).
           h at s = 2i+1:        Gamma(i + 1/2)/Gamma(i + 2), start Gamma(1/2) = sqrt(pi). */
        dd he = dd_div(dd_from(4.0), dd_mul_d(tb.sqrtpi, 3.0));
        dd ho = tb.sqrtpi;
        for (int64_t s = 0; s < nh; ++s) {
            if (s == 0) { h[s] = 1.0; continue; }
            if (s & 1) {
                int64_t i = (s - 1) / 2;
                h[s] = dd_round(ho);
                ho = dd_div(dd_mul(ho, dd_from((double)i + 0.5)), dd_from((double)i + 2.0));
            } else {
                int64_t i = s / 2;
                h[s] = dd_round(he);
                he = dd_div(dd_mul(he, dd_from((double)i)), dd_from((double)i + 1.5));
            }
        }
        for (int64_t j = 0; j < n; ++j) {
            d1[j] = (double)j + 0.5;
            d2[j] = (j == 0) ? dd_round(dd_div(dd_from(-1.0), tb.sqrtpi)) : -0.25 * (double)j;
        }
        break;
    }
    case K_ULTRA: {
        double l1 = prm[0], l2 = prm[1];
        for (int64_t m = 0; m < n; ++m) t[m] = (m & 1) ? 0.0 : dd_round(tb.P[m / 2]);
        /* odd s: Q'(i + 1/2) = Gamma(l2) Gamma(i + 1/2 + l1) / (Gamma(l1) Gamma(i + l2 + 3/2)) */
        double q0 = exp(lgamma(l2) + lgamma(l1 + 0.5) - lgamma(l1) - lgamma(l2 + 1.5));
        dd qo = dd_from(q0);
        for (int64_t s = 0; s < nh; ++s) {
            if (!(s & 1)) { h[s] = dd_round(tb.Q[s / 2]); continue; }
            int64_t i = (s - 1) / 2;
            h[s] = dd_round(qo);
            qo = dd_div(dd_mul(qo, dd_from((double)i + 0.5 + l1)), dd_from((double)i + l2 + 1.5));
        }
        for (int64_t j = 0; j < n; ++j) { d1[j] = (double)j + l2; d2[j] = 1.0; }
        break;
    }
    case K_JAC: {
        /* Case 3: row and column 0 are applied directly (A_00 = 1); the constant goes to D1. */
        for (int64_t m = 0; m < n; ++m) t[m] = dd_round(tb.P[m]);
        for (int64_t s = 0; s < nh; ++s) h[s] = dd_round(tb.G[s]);
        for (int64_t j = 0; j < n; ++j) {
            d1[j] = dd_round(tb.case3 ? dd_mul(tb.E1[j], tb.c_rest) : tb.E1[j]);
            d2[j] = dd_round(tb.E2[j]);
        }
        break;
    }
    case K_LAG: {
        for (int64_t m = 0; m < n; ++m) t[m] = dd_round(tb.P[m]);
        for (int64_t s = 0; s < nh; ++s) h[s] = 1.0;
        for (int64_t j = 0; j < n; ++j) { d1[j] = 1.0; d2[j] = 1.0; }
        break;
    }
    default:
        free_tables(&tb);
        return -2;
    }
    free_tables(&tb);
    return 0;
}

/* Lambda(i/2) for i in [0, count) as double-double pairs (for pins against mpmath). */
int tdho_lambda(int64_t count, double* hi, double* lo) {
    if (count < 0) return -1;
    dd* lam = (dd*)malloc(sizeof(dd) * (size_t)(count > 0 ? count : 1));
    if (!lam) return -1;
    build_lambda(lam, count, dd_sqrt(dd_pi()));
    for (int64_t i = 0; i < count; ++i) { hi[i] = lam[i].hi; lo[i] = lam[i].lo; }
    free(lam);
    return 0;
}

/* Number of threads the oracle uses by default (for reporting). */
int tdho_threads(void) { return set_threads(0); }
