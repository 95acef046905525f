// Host side of the execute path: per-plan tables (step a3 and the kernel's twiddles and
// factor layout) and the launch dispatch over the kernel instantiations.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "tdh_exec.cuh"

namespace tdh {
namespace {

// Threads and occupancy of the multi-pass kernels for local length 2^logLC: slices one below
// the shared-memory cap run 256 threads, two CTAs per SM; full slices 512 threads, one CTA.
void mp_threads(int prec, int logLC, int* NT, int* MINB) {
    const int cap = (prec != TDH_FP64) ? 14 : 13;
    *NT = logLC == cap ? 512 : 256;
    *MINB = logLC == cap ? 1 : 2;
}

// Default FFT geometry for a transform of 2^logL points in precision `prec`.  Split-bfloat16
// plans take the float32 geometry, with tensor-core passes within one cluster (the multi-pass
// FFTs beyond it run the float32 kernels).
bool choose_geometry(int prec, int logL, Geometry* g) {
    g->prec = prec;
    g->logL = logL;
    g->tc = 0;
    g->tma = 0;
    const int cap = (prec != TDH_FP64) ? 14 : 13;  // largest local FFT held in shared memory
    if (logL <= cap) {
        g->logLC = logL;
        g->C = 1;
    } else {
        g->logLC = cap;
        g->C = 1 << (logL - cap);
        if (g->C > 8 && g->C <= 128) {
            // multi-pass: slices of half the size, two CTAs per SM (up to 256 slices, the
            // register-DFT cross stage's limit)
            g->logLC = cap - 1;
            g->C = 1 << (logL - cap + 1);
        }
    }
    if (g->C > 512) return false;  // C > 8: multi-pass through global memory
    g->R = radix_for(prec != TDH_FP64, g->logLC);
    // float32 2^14-point slices, one CTA or 2-8-CTA clusters: radix 32, 32, 16 (three
    // shared-memory passes instead of four; their accumulators are in tensor memory)
    if (prec == TDH_FP32 && g->logLC == 14 && g->C <= 8) g->R = 32;
    // the float32 multi-pass kernels (also under split-bfloat16 plans): radix 32 as well
    if (prec != TDH_FP64 && g->C > 8) g->R = 32;
    g->NT = std::min(512, (1 << g->logLC) / g->R);
    g->MINB = 1;
    if (g->C > 8) mp_threads(prec, g->logLC, &g->NT, &g->MINB);
    g->tc = (prec == TDH_BF16X3 && g->C <= 8) ? 1 : 0;
    return true;
}

bool same_schedule(const Geometry& a, const Geometry& b) {
    return a.logLC == b.logLC && a.C == b.C && a.NT == b.NT && a.MINB == b.MINB && a.tc == b.tc &&
           a.tma == b.tma && a.R == b.R;
}

// Every schedule with a compiled kernel for 2^logL points, the default first: the cluster
// schedules of the table whose LC * C = L, and for C > 8 (not in ragged batches, which stay
// within one cluster) the multi-pass kernels on full and on half-size slices.
std::vector<Geometry> schedule_candidates(int prec, int logL, bool ragged) {
    std::vector<Geometry> out;
    Geometry d{};
    if (!choose_geometry(prec, logL, &d)) return out;
    out.push_back(d);
    auto add = [&](int logLC, int C, int NT, int MINB, int tma = 0, int R = 0) {
        Geometry g = d;
        g.logLC = logLC;
        g.C = C;
        g.R = R ? R : radix_for(prec != TDH_FP64, logLC);
        g.NT = NT;
        g.MINB = MINB;
        g.tc = (prec == TDH_BF16X3 && C <= 8) ? 1 : 0;
        g.tma = tma;
        for (const Geometry& o : out)
            if (same_schedule(o, g)) return;
        out.push_back(g);
    };
    const bool f32 = prec != TDH_FP64;
    const int n = prec == TDH_BF16X3 ? SchedTableTC::size
                  : f32             ? SchedTable<true>::size
                                    : SchedTable<false>::size;
    for (int i = 0; i < n; ++i) {
        const Sched e = prec == TDH_BF16X3 ? SchedTableTC::at(i)
                        : f32              ? SchedTable<true>::at(i)
                                           : SchedTable<false>::at(i);
        if (e.logLC + ilog2(e.C) == logL) add(e.logLC, e.C, e.NT, e.MINB, 0, e.R);
    }
    if (!ragged) {
        const int cap = f32 ? 14 : 13;  // (multi-pass kernels: float32 arithmetic for BF16X3)
        for (int lc = cap; lc >= cap - 1; --lc) {
            if (logL - lc < 4 || logL - lc > 9) continue;  // 16 ... 512 slices
            int NT, MINB;
            mp_threads(prec, lc, &NT, &MINB);
            add(lc, 1 << (logL - lc), NT, MINB);
        }
        // the same multi-pass kernels with the cross stage's block moved by TMA copies
        for (int lc = cap; lc >= cap - 1; --lc) {
            if (logL - lc < 4 || logL - lc > 8) continue;  // 16 ... 256 slices
            int NT, MINB;
            mp_threads(prec, lc, &NT, &MINB);
            add(lc, 1 << (logL - lc), NT, MINB, 1);
        }
        // float32: the multi-pass kernels with radix-32 local passes
        for (int lc = cap; f32 && lc >= cap - 1; --lc) {
            if (logL - lc < 4 || logL - lc > 9) continue;
            int NT, MINB;
            mp_threads(prec, lc, &NT, &MINB);
            add(lc, 1 << (logL - lc), NT, MINB, 0, 32);
        }
    }
    if (ragged) {
        std::vector<Geometry> in;
        in.swap(out);
        for (const Geometry& g : in)
            if (g.C <= 8) out.push_back(g);
    }
    return out;
}

constexpr int kThreads = 256;
inline unsigned blocks_for(int64_t count) { return (unsigned)((count + kThreads - 1) / kThreads); }

__device__ __forceinline__ double2 omega(int64_t e, int64_t den) {
    // exp(-2 pi i e / den), argument reduced exactly before sincospi
    const int64_t r = ((e % den) + den) % den;
    double s, c;
    sincospi(2.0 * (double)r / (double)den, &s, &c);
    return make_double2(c, -s);
}

template <typename V>
__device__ __forceinline__ V from_d2(double2 z);
template <>
__device__ __forceinline__ float2 from_d2<float2>(double2 z) {
    return make_float2((float)z.x, (float)z.y);
}
template <>
__device__ __forceinline__ double2 from_d2<double2>(double2 z) {
    return z;
}

// symbol of the packed correlation: s_i = t_{stride i} for i < m, zero-padded to L
// (stride 2 for parity packing, 1 for rank-pair packing)
__global__ void k_fill_symbol(const double* __restrict__ t, int64_t m, int64_t L, int stride,
                              double2* __restrict__ x) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i < L) x[i] = make_double2(i < m ? t[stride * i] : 0.0, 0.0);
}

// one radix-2 Stockham stage (natural order in and out), float64
__global__ void k_stockham(const double2* __restrict__ x, double2* __restrict__ y, int64_t L,
                           int64_t m) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= L / 2) return;
    const int64_t j = i / m, k = i % m;
    const double2 w = omega(k, 2 * m);
    const double2 a = x[j * m + k];
    const double2 b0 = x[j * m + k + L / 2];
    const double2 b = make_double2(w.x * b0.x - w.y * b0.y, w.x * b0.y + w.y * b0.x);
    y[2 * j * m + k] = make_double2(a.x + b.x, a.y + b.y);
    y[2 * j * m + k + m] = make_double2(a.x - b.x, a.y - b.y);
}

// conj(S[f1(pos) + LC f2]) / L at spec[pos][f2] (cluster kernels) or spec[f2][pos]
// (multi-pass cross stage, `by_f2`)
template <typename V>
__global__ void k_spec(const double2* __restrict__ S, const int* __restrict__ perm, int LC, int C,
                       int64_t L, int by_f2, V* __restrict__ spec) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= (int64_t)LC * C) return;
    const int pos = (int)(i / C), f2 = (int)(i % C);
    const double2 z = S[perm[pos] + (int64_t)LC * f2];
    const double inv = 1.0 / (double)L;
    spec[by_f2 ? (int64_t)f2 * LC + pos : i] = from_d2<V>(make_double2(z.x * inv, -z.y * inv));
}

// twx[pos] = omega_L^{f1(pos)}
template <typename V>
__global__ void k_twx(const int* __restrict__ perm, int LC, int64_t L, V* __restrict__ twx) {
    int i = blockIdx.x * kThreads + threadIdx.x;
    if (i < LC) twx[i] = from_d2<V>(omega(perm[i], L));
}

// out[i] = omega_den^{(i / S) * (i % S)} for i < count (S = count: plain omega_den^i)
template <typename V>
__global__ void k_omega_table(V* __restrict__ out, int64_t count, int64_t S, int64_t den) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i < count) out[i] = from_d2<V>(omega((i / S) * (i % S), den));
}

template <typename V>
__global__ void k_omega_lin(V* __restrict__ out, int64_t count, int64_t den) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i < count) out[i] = from_d2<V>(omega(i, den));
}

// out[i] = omega_den^{i * mult}
template <typename V>
__global__ void k_omega_scaled(V* __restrict__ out, int64_t count, int64_t mult, int64_t den) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i < count) out[i] = from_d2<V>(omega(i * mult, den));
}

// u_dec[r][k1][k2] = (u[r][2a], u[r][2a+1]), a = k1 + C k2 (zero beyond n)
template <typename T>
__global__ void k_u_gather(const double* __restrict__ u, int64_t n, int64_t K, int C, int half,
                           typename cx<T>::t* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int64_t total = K * C * (int64_t)half;
    if (i >= total) return;
    const int64_t k2 = i % half;
    const int64_t k1 = (i / half) % C;
    const int64_t r = i / ((int64_t)half * C);
    const int64_t a = k1 + (int64_t)C * k2;
    const int64_t i0 = 2 * a;
    const double* ur = u + r * n;
    T x0 = (i0 < n) ? (T)ur[i0] : T(0);
    T x1 = (i0 + 1 < n) ? (T)ur[i0 + 1] : T(0);
    typename cx<T>::t v;
    v.x = x0;
    v.y = x1;
    out[i] = v;
}

// rank-pair packing: out[rp][k1][k2] = (u[i0][a], s_rp u[i1][a]), a = k1 + C k2, with
// (i0, i1) = (idx[2rp], idx[2rp+1]) and s_rp = scale[rp] (the step's pairing)
template <typename T>
__global__ void k_u_gather_pairs(const double* __restrict__ u, int64_t n, int64_t K, int C,
                                 int half, const int* __restrict__ idx,
                                 const double* __restrict__ scale,
                                 typename cx<T>::t* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int64_t KP = (K + 1) / 2;
    const int64_t total = KP * C * (int64_t)half;
    if (i >= total) return;
    const int64_t k2 = i % half;
    const int64_t k1 = (i / half) % C;
    const int64_t rp = i / ((int64_t)half * C);
    const int64_t a = k1 + (int64_t)C * k2;
    T x0 = (a < n) ? (T)u[(int64_t)idx[2 * rp] * n + a] : T(0);
    T x1 = (a < n && 2 * rp + 1 < K) ? (T)(scale[rp] * u[(int64_t)idx[2 * rp + 1] * n + a]) : T(0);
    typename cx<T>::t v;
    v.x = x0;
    v.y = x1;
    out[i] = v;
}

template <typename T>
__global__ void k_cast(const double* __restrict__ in, T* __restrict__ out, int64_t count) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i < count) out[i] = (T)in[i];
}

// row 0 of A = D1 (T o H) D2 (valid for k >= 1), with A_00 = 1 (Sec. 5.1, Sec. 5.3 Case 3);
// with the step's scalings A_00 becomes so_0 si_0 (d1, d2 already carry them)
template <typename T>
__global__ void k_row0(const double* __restrict__ t, const double* __restrict__ h,
                       const double* __restrict__ d1, const double* __restrict__ d2, int64_t n,
                       const double* __restrict__ so, const double* __restrict__ si,
                       T* __restrict__ out) {
    int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (k >= n) return;
    const double a00 = (so ? so[0] : 1.0) * (si ? si[0] : 1.0);
    out[k] = (k == 0) ? (T)a00 : (T)(d1[0] * t[k] * h[k] * d2[k]);
}

// d[i] *= s[i]
__global__ void k_scale(double* __restrict__ d, const double* __restrict__ s, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i < n) d[i] *= s[i];
}

template <typename T>
int prepare_typed(Step& st, ExecData& ex, const Geometry& g, const void* shared_u,
                  int64_t shared_stride, cudaStream_t s) {
    using V = typename cx<T>::t;
    const PassGeom G{g.logLC, g.R};
    const int LC = G.LC(), C = g.C;
    const int64_t L = (int64_t)1 << g.logL;
    // symbol entries the correlation can touch: below m, and below L/2 so nothing wraps
    const int64_t m = std::min<int64_t>(ex.m, L / 2);
    int rc = TDH_OK;
    double2 *x = nullptr, *y = nullptr;
    int* perm_d = nullptr;
    std::vector<int> perm(LC);
    for (int pos = 0; pos < LC; ++pos) perm[pos] = local_freq(G, pos);

    if ((rc = dev_alloc_t(&x, L)) || (rc = dev_alloc_t(&y, L)) || (rc = dev_alloc_t(&perm_d, LC)))
        goto out;
    if ((rc = dev_alloc(&ex.spec, sizeof(V) * (size_t)LC * C)) ||
        (rc = dev_alloc(&ex.tw0, sizeof(V) * (size_t)(LC / g.R))))
        goto out;
    if (shared_u) {
        ex.u = const_cast<void*>(shared_u);
        ex.u_owned = false;
        ex.u_stride = shared_stride;
    } else {
        ex.u_stride = LC / 2;
        if ((rc = dev_alloc(&ex.u, sizeof(V) * (size_t)std::max<int64_t>(st.K, 1) * C * (LC / 2))))
            goto out;
    }
    ex.twp_len = G.twp_len();
    if (ex.twp_len > 0 && (rc = dev_alloc(&ex.twp, sizeof(V) * (size_t)ex.twp_len))) goto out;
    ex.multipass = C > 8;
    if (C > 1 && !ex.multipass && (rc = dev_alloc(&ex.twx, sizeof(V) * (size_t)LC))) goto out;
    if (ex.multipass) {
        ex.twl_shift = (g.logL + 1) / 2;
        if ((rc = dev_alloc(&ex.twl_hi, sizeof(V) * (size_t)(L >> ex.twl_shift))) ||
            (rc = dev_alloc(&ex.twl_lo, sizeof(V) * ((size_t)1 << ex.twl_shift))))
            goto out;
    }
    {
        cudaError_t e = cudaMemcpyAsync(perm_d, perm.data(), sizeof(int) * LC,
                                        cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            set_error("table upload: %s", cudaGetErrorString(e));
            rc = TDH_ERR_CUDA;
            goto out;
        }
        // a3: S = DFT_L(s) in float64, natural order, by log2 L Stockham stages
        k_fill_symbol<<<blocks_for(L), kThreads, 0, s>>>(st.t, m, L, st.full ? 1 : 2, x);
        for (int64_t mm = 1; mm < L; mm *= 2) {
            k_stockham<<<blocks_for(L / 2), kThreads, 0, s>>>(x, y, L, mm);
            std::swap(x, y);
        }
        k_spec<V><<<blocks_for((int64_t)LC * C), kThreads, 0, s>>>(x, perm_d, LC, C, L,
                                                                   ex.multipass, (V*)ex.spec);
        if (C > 1 && !ex.multipass)
            k_twx<V><<<blocks_for(LC), kThreads, 0, s>>>(perm_d, LC, L, (V*)ex.twx);
        if (ex.multipass) {
            const int64_t nhi = L >> ex.twl_shift, nlo = (int64_t)1 << ex.twl_shift;
            k_omega_scaled<V><<<blocks_for(nhi), kThreads, 0, s>>>((V*)ex.twl_hi, nhi, nlo, L);
            k_omega_scaled<V><<<blocks_for(nlo), kThreads, 0, s>>>((V*)ex.twl_lo, nlo, 1, L);
        }
        k_omega_lin<V><<<blocks_for(LC / g.R), kThreads, 0, s>>>((V*)ex.tw0, LC / g.R, LC);
        for (int i = 1; i <= G.np() - 2; ++i)
            k_omega_table<V><<<blocks_for(G.M(i)), kThreads, 0, s>>>(
                (V*)ex.twp + G.twoff(i), G.M(i), G.S(i), G.M(i));
        if (st.K > 0 && !st.full && !shared_u)
            k_u_gather<T><<<blocks_for(st.K * C * (int64_t)(LC / 2)), kThreads, 0, s>>>(
                st.u64, st.n, st.K, C, LC / 2, (V*)ex.u);
        if (st.K > 0 && st.full && !shared_u)
            k_u_gather_pairs<T><<<blocks_for((st.K + 1) / 2 * C * (int64_t)(LC / 2)), kThreads, 0,
                                  s>>>(st.u64, st.n, st.K, C, LC / 2, st.pair_idx, st.pair_s,
                                       (V*)ex.u);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("execute tables: %s", cudaGetErrorString(e));
            rc = TDH_ERR_CUDA;
        }
    }
out:
    if (x || y || perm_d) cudaStreamSynchronize(s);
    dev_free(x);
    dev_free(y);
    if (rc == TDH_OK && ex.multipass)
        ex.perm = perm_d;  // the multi-pass exchange kernel maps positions to frequencies
    else
        dev_free(perm_d);
    return rc;
}

// max_k |u_r[k] d2[k]| for rank term r = blockIdx.x (the size of term r's FFT input per unit
// of ||alpha||_inf)
__global__ void __launch_bounds__(kThreads) k_factor_size(const double* __restrict__ u,
                                                          const double* __restrict__ d2, int64_t n,
                                                          double* __restrict__ out) {
    __shared__ double red[kThreads];
    const double* ur = u + (int64_t)blockIdx.x * n;
    double m = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += kThreads) m = fmax(m, fabs(ur[k] * d2[k]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// Rank-pair packing puts two rank terms in the real and imaginary parts of one complex FFT,
// whose rounding is relative to the larger of the two: a term much smaller than its partner
// would lose its accuracy.  The terms are sorted by size (max_k |u_r[k] D2_k|), paired with
// their neighbour, and the smaller one is scaled up to its partner's size on the way in
// (scale s <= 1e6) and back down by 1 / s^2 on the way out (the same table serves both).
template <typename T>
int prepare_pairs(Step& st, cudaStream_t s) {
    const int64_t K = st.K, KP = (K + 1) / 2;
    std::vector<double> size(K);
    double* dsize = nullptr;
    TDH_TRY(dev_alloc_t(&dsize, (size_t)K));
    k_factor_size<<<(unsigned)K, kThreads, 0, s>>>(st.u64, st.d2, st.n, dsize);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(size.data(), dsize, sizeof(double) * K, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(dsize);
    if (e != cudaSuccess) {
        set_error("rank pairing: %s", cudaGetErrorString(e));
        return TDH_ERR_CUDA;
    }
    std::vector<int> idx(K);
    for (int64_t r = 0; r < K; ++r) idx[r] = (int)r;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return size[a] > size[b]; });
    std::vector<double> sc(KP, 1.0);
    std::vector<T> cc(KP, T(1));
    for (int64_t p = 0; p < KP; ++p) {
        if (2 * p + 1 >= K) {
            cc[p] = T(0);
            continue;
        }
        const double big = size[idx[2 * p]], small = size[idx[2 * p + 1]];
        double f = (small > 0.0 && big > small) ? big / small : 1.0;
        f = std::min(f, 1e6);
        sc[p] = f;
        cc[p] = (T)(1.0 / (f * f));
    }
    TDH_TRY(dev_alloc_t(&st.pair_idx, (size_t)K));
    TDH_TRY(dev_alloc_t(&st.pair_s, (size_t)KP));
    TDH_TRY(dev_alloc(&st.pair_c, sizeof(T) * (size_t)KP));
    TDH_CUDA(cudaMemcpyAsync(st.pair_idx, idx.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
    TDH_CUDA(cudaMemcpyAsync(st.pair_s, sc.data(), sizeof(double) * KP, cudaMemcpyHostToDevice, s));
    TDH_CUDA(cudaMemcpyAsync(st.pair_c, cc.data(), sizeof(T) * KP, cudaMemcpyHostToDevice, s));
    TDH_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
    return TDH_OK;
}

template <typename T>
int prepare_diagonals(Step& st, cudaStream_t s) {
    const int64_t n = st.n;
    // diag(scale_out) D1 (T o H) D2 diag(scale_in)
    if (st.scale_out) k_scale<<<blocks_for(n), kThreads, 0, s>>>(st.d1, st.scale_out, n);
    if (st.scale_in) k_scale<<<blocks_for(n), kThreads, 0, s>>>(st.d2, st.scale_in, n);
    TDH_TRY(dev_alloc(&st.d1x, sizeof(T) * n));
    TDH_TRY(dev_alloc(&st.d2x, sizeof(T) * n));
    k_cast<T><<<blocks_for(n), kThreads, 0, s>>>(st.d1, (T*)st.d1x, n);
    k_cast<T><<<blocks_for(n), kThreads, 0, s>>>(st.d2, (T*)st.d2x, n);
    if (st.j0 == 1) {
        TDH_TRY(dev_alloc(&st.row0, sizeof(T) * n));
        k_row0<T><<<blocks_for(n), kThreads, 0, s>>>(st.t, st.h, st.d1, st.d2, n, st.scale_out,
                                                     st.scale_in, (T*)st.row0);
    }
    TDH_CUDA(cudaGetLastError());
    return TDH_OK;
}

// ----------------------------------------------------------------------------- launch

template <typename T>
int dispatch(const Geometry& g, const ExecParams<T>& P, int64_t batch, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        if (g.tc)
            return P.ragged ? dispatch_ragged_tc(g, P, batch, s) : dispatch_dense_tc(g, P, batch, s);
    }
    return P.ragged ? dispatch_ragged(g, P, batch, s) : dispatch_dense(g, P, batch, s);
}

template <typename T>
int launch_typed(const Step& st, const void* in, void* out, int64_t batch, int adjoint,
                 cudaStream_t s) {
    using V = typename cx<T>::t;
    const ExecData& ex = st.ex;
    ExecParams<T> P;
    P.in = static_cast<const T*>(in);
    P.out = static_cast<T*>(out);
    P.n = st.n;
    P.K = st.K;
    P.u = static_cast<const V*>(ex.u);
    P.spec = static_cast<const V*>(ex.spec);
    P.twx = static_cast<const V*>(ex.twx);
    P.tw0 = static_cast<const V*>(ex.tw0);
    P.twp = static_cast<const V*>(ex.twp);
    P.din = static_cast<const T*>(adjoint ? st.d1x : st.d2x);
    P.dout = static_cast<const T*>(adjoint ? st.d2x : st.d1x);
    P.row0 = static_cast<const T*>(st.row0);
    P.adjoint = adjoint;
    P.full = st.full;
    P.sign_in = st.sign_in;
    P.sign_out = st.sign_out;
    if (st.full) P.K = (st.K + 1) / 2;
    P.u_stride = ((int64_t)1 << ex.g.logLC) / 2;
    P.ragged = 0;
    P.offs = nullptr;
    P.list = nullptr;
    P.count = nullptr;
    P.next = nullptr;
    P.batch = batch;
    P.partial = nullptr;
    P.status = st.status;
    P.tc_stall = tc_stall_enabled();
    P.pair_c = static_cast<const T*>(st.pair_c);
    return dispatch<T>(ex.g, P, batch, s);
}

}  // namespace

int exec_prepare(Step& st, int prec, cudaStream_t s) {
    ExecData& ex = st.ex;
    ex.m = st.full ? st.n : (st.n + 1) / 2;
    int logL = 8;
    while (((int64_t)1 << logL) < 2 * ex.m - 1) ++logL;
    if (!choose_geometry(prec, logL, &ex.g)) {
        set_error("length %lld needs an FFT of 2^%d points, beyond the library's cluster limit",
                  (long long)st.n, logL);
        return TDH_ERR_UNSUPPORTED;
    }
    if (prec != TDH_FP64) {
        TDH_TRY(prepare_diagonals<float>(st, s));
        if (st.full && st.K > 0) TDH_TRY(prepare_pairs<float>(st, s));
        return prepare_typed<float>(st, ex, ex.g, nullptr, 0, s);
    }
    TDH_TRY(prepare_diagonals<double>(st, s));
    if (st.full && st.K > 0) TDH_TRY(prepare_pairs<double>(st, s));
    return prepare_typed<double>(st, ex, ex.g, nullptr, 0, s);
}

namespace {
template <typename T>
int prepare_ragged_typed(Step& st, int prec, cudaStream_t s) {
    using V = typename cx<T>::t;
    const int64_t half = (st.n + 1) / 2;
    TDH_TRY(dev_alloc(&st.u_nat, sizeof(V) * (size_t)std::max<int64_t>(st.K, 1) * half));
    if (st.K > 0)
        k_u_gather<T><<<blocks_for(st.K * half), kThreads, 0, s>>>(st.u64, st.n, st.K, 1,
                                                                   (int)half, (V*)st.u_nat);
    TDH_CUDA(cudaGetLastError());
    for (int logL = 8; logL <= st.ex.g.logL; ++logL) {
        st.rcls.emplace_back();
        ExecData& ex = st.rcls.back();
        ex.m = st.ex.m;
        if (!choose_geometry(prec, logL, &ex.g) || ex.g.C > 8) {
            set_error("ragged batches are built for FFT lengths within one cluster");
            return TDH_ERR_UNSUPPORTED;
        }
        const bool nat = ex.g.C == 1;
        TDH_TRY(prepare_typed<T>(st, ex, ex.g, nat ? st.u_nat : nullptr, nat ? half : 0, s));
    }
    return TDH_OK;
}
}  // namespace

int exec_prepare_ragged(Step& st, int prec, cudaStream_t s) {
    if (st.full || st.sp_M > 0) {
        set_error("ragged batches are built for the parity-packed kinds");
        return TDH_ERR_UNSUPPORTED;
    }
    if (prec != TDH_FP64) return prepare_ragged_typed<float>(st, prec, s);
    return prepare_ragged_typed<double>(st, prec, s);
}

void exec_release(ExecData& ex) {
    if (!ex.u_owned) ex.u = nullptr;
    dev_free(ex.perm);
    dev_free(ex.twl_hi);
    dev_free(ex.twl_lo);
    dev_free(ex.spec);
    dev_free(ex.twx);
    dev_free(ex.tw0);
    dev_free(ex.twp);
    dev_free(ex.u);
    ex = ExecData{};
}

namespace {

// Group the vectors of a ragged batch by FFT length class (device side, any order).  Checks
// recorded in the plan's status word: the whole output range [offs[0], offs[batch]) of `out`
// overlapping that of `in` (nothing is converted), and vectors longer than n_max or with
// decreasing offsets (those are left unwritten).
__global__ void k_classify(const int64_t* __restrict__ offs, int64_t batch, int64_t n_max,
                           int ncls, int* __restrict__ count, int* __restrict__ list,
                           const char* in, const char* out, int esz, int* status) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= batch) return;
    const int64_t span = (offs[batch] - offs[0]) * esz;
    const int64_t gap = in > out ? (int64_t)(in - out) : (int64_t)(out - in);
    if (span > 0 && gap < span) {
        if (i == 0 && status) atomicOr(status, TDH_STATUS_ALIAS);
        return;
    }
    const int64_t n = offs[i + 1] - offs[i];
    if ((n < 0 || n > n_max) && status) atomicOr(status, TDH_STATUS_LENGTH);
    if (n <= 0 || n > n_max) return;  // nothing to do / outside the plan (documented)
    const int64_t m = (n + 1) / 2;
    int logL = 8;
    while (((int64_t)1 << logL) < 2 * m - 1) ++logL;
    const int c = logL - 8;
    if (c >= ncls) return;
    const int idx = atomicAdd(&count[c], 1);
    list[(int64_t)c * batch + idx] = (int)i;
}

template <typename T>
ExecParams<T> ragged_params(const Step& st, const ExecData& ex, const void* in, void* out,
                            const int64_t* offs, int* list, int* count, int* next, int64_t batch) {
    using V = typename cx<T>::t;
    ExecParams<T> P;
    P.in = static_cast<const T*>(in);
    P.out = static_cast<T*>(out);
    P.n = st.n;
    P.K = st.K;
    P.u = static_cast<const V*>(ex.u);
    P.spec = static_cast<const V*>(ex.spec);
    P.twx = static_cast<const V*>(ex.twx);
    P.tw0 = static_cast<const V*>(ex.tw0);
    P.twp = static_cast<const V*>(ex.twp);
    P.din = static_cast<const T*>(st.d2x);
    P.dout = static_cast<const T*>(st.d1x);
    P.row0 = static_cast<const T*>(st.row0);
    P.adjoint = 0;
    P.full = 0;
    P.sign_in = 0;
    P.sign_out = 0;
    P.u_stride = ex.u_stride;
    P.batch = batch;
    P.partial = nullptr;
    P.ragged = 1;
    P.offs = offs;
    P.list = list;
    P.count = count;
    P.next = next;
    P.status = st.status;
    P.tc_stall = tc_stall_enabled();
    P.pair_c = nullptr;  // ragged plans are parity-packed
    return P;
}

template <typename T>
int launch_ragged_typed(const Step& st, const void* in, void* out, const int64_t* offs,
                        int64_t batch, cudaStream_t s, const std::vector<cudaStream_t>& side,
                        const std::vector<cudaEvent_t>& ev) {
    const int ncls = (int)st.rcls.size();
    if ((int)side.size() < ncls || (int)ev.size() < ncls + 1) {
        set_error("ragged execute: plan streams missing");
        return TDH_ERR_INVALID_ARG;
    }
    int* scratch = nullptr;
    const size_t words = 2 * (size_t)ncls + (size_t)ncls * batch;
    TDH_TRY(scratch_alloc(reinterpret_cast<void**>(&scratch), sizeof(int) * words, s));
    int* count = scratch;
    int* next = scratch + ncls;
    int* list = scratch + 2 * ncls;
    int rc = TDH_OK;
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int) * 2 * ncls, s);
    if (e == cudaSuccess) {
        k_classify<<<blocks_for(batch), kThreads, 0, s>>>(
            offs, batch, st.n, ncls, count, list, static_cast<const char*>(in),
            static_cast<const char*>(out), (int)sizeof(T), st.status);
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    // longest class first; each class on its own stream
    for (int c = ncls - 1; e == cudaSuccess && rc == TDH_OK && c >= 0; --c) {
        const ExecData& ex = st.rcls[c];
        cudaStream_t sc = side[c];
        e = cudaStreamWaitEvent(sc, ev[0], 0);
        if (e != cudaSuccess) break;
        ExecParams<T> P = ragged_params<T>(st, ex, in, out, offs, list + (int64_t)c * batch,
                                           count + c, next + c, batch);
        rc = dispatch<T>(ex.g, P, batch, sc);
        if (rc == TDH_OK) e = cudaEventRecord(ev[1 + c], sc);
        if (e == cudaSuccess && rc == TDH_OK) e = cudaStreamWaitEvent(s, ev[1 + c], 0);
    }
    if (e != cudaSuccess && rc == TDH_OK) {
        set_error("ragged execute: %s", cudaGetErrorString(e));
        rc = TDH_ERR_CUDA;
    }
    scratch_free(scratch, s);
    return rc;
}

}  // namespace

int exec_launch_ragged(const Step& st, int prec, const void* in, void* out, const int64_t* offs,
                       int64_t batch, cudaStream_t s, const std::vector<cudaStream_t>& side,
                       const std::vector<cudaEvent_t>& ev) {
    if (prec != TDH_FP64) return launch_ragged_typed<float>(st, in, out, offs, batch, s, side, ev);
    return launch_ragged_typed<double>(st, in, out, offs, batch, s, side, ev);
}

int exec_launch(const Step& st, int prec, const void* in, void* out, int64_t batch, int adjoint,
                cudaStream_t s) {
    if (st.ex.multipass) return mp_launch(st, prec, in, out, batch, adjoint, s);
    if (prec != TDH_FP64) return launch_typed<float>(st, in, out, batch, adjoint, s);
    return launch_typed<double>(st, in, out, batch, adjoint, s);
}

// ----------------------------------------------------------------------------- schedules

namespace {

struct ConfigRef {
    Step* st;
    int cls;  // -1: the step's dense configuration, else its ragged length class
};

std::vector<ConfigRef> plan_configs(tdh_plan_s& plan) {
    std::vector<ConfigRef> out;
    for (auto& st : plan.steps) {
        if (st.sp_M > 0) continue;
        out.push_back({&st, -1});
        for (int c = 0; c < (int)st.rcls.size(); ++c) out.push_back({&st, c});
    }
    return out;
}

ExecData& config_data(const ConfigRef& r) { return r.cls < 0 ? r.st->ex : r.st->rcls[r.cls]; }

// Rebuild configuration r's tables for schedule g (nothing to do if it already runs g).
int rebuild_config(const ConfigRef& r, int prec, const Geometry& g, cudaStream_t s) {
    ExecData& cur = config_data(r);
    if (same_schedule(cur.g, g)) return TDH_OK;
    ExecData nx;
    nx.m = cur.m;
    nx.g = g;
    const bool nat = r.cls >= 0 && g.C == 1;  // ragged single-CTA classes share u_nat
    const void* su = nat ? r.st->u_nat : nullptr;
    const int64_t ss = nat ? (r.st->n + 1) / 2 : 0;
    const int rc = prec != TDH_FP64 ? prepare_typed<float>(*r.st, nx, g, su, ss, s)
                                    : prepare_typed<double>(*r.st, nx, g, su, ss, s);
    if (rc != TDH_OK) {
        exec_release(nx);
        return rc;
    }
    exec_release(cur);
    cur = nx;
    return TDH_OK;
}

// Deterministic test values in [-1, 1) (an integer hash of the index, then scaled).
template <typename T>
__global__ void k_fill_test(T* __restrict__ x, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= count) return;
    uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;
    z ^= z >> 29;
    x[i] = (T)((double)(z >> 11) * 0x1.0p-52 - 1.0);
}

// Uniform ragged batch for timing one length class: b vectors of length len.
__global__ void k_ragged_uniform(int64_t* __restrict__ offs, int* __restrict__ list,
                                 int* __restrict__ ctr, int64_t b, int64_t len) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i < b) list[i] = (int)i;
    if (i <= b) offs[i] = i * len;
    if (i == 0) {
        ctr[0] = (int)b;
        ctr[1] = 0;
    }
}

struct TuneBuffers {
    void* in = nullptr;
    void* out = nullptr;
    int64_t* offs = nullptr;
    int* list = nullptr;
    int* ctr = nullptr;
    cudaEvent_t ev[4] = {};
};

// Vectors and length each timing of configuration r uses.
void tune_shape(const ConfigRef& r, int64_t batch, int64_t* b, int64_t* len) {
    if (r.cls < 0) {
        *b = batch;
        *len = r.st->n;
        return;
    }
    const int64_t ncls = (int64_t)r.st->rcls.size();
    *b = std::max<int64_t>(1, batch / ncls);
    *len = std::min<int64_t>(r.st->n, (int64_t)1 << r.st->rcls[r.cls].g.logL);
}

// Shortest of three timed launches of configuration r (after one untimed).
template <typename T>
int time_config(const ConfigRef& r, int64_t batch, const TuneBuffers& tb, cudaStream_t s,
                float* ms) {
    int64_t b, len;
    tune_shape(r, batch, &b, &len);
    const Step& st = *r.st;
    if (r.cls >= 0) {
        k_ragged_uniform<<<blocks_for(b + 1), kThreads, 0, s>>>(tb.offs, tb.list, tb.ctr, b, len);
        TDH_CUDA(cudaGetLastError());
    }
    auto launch = [&]() -> int {
        if (r.cls < 0) return exec_launch(st, std::is_same<T, float>::value ? TDH_FP32 : TDH_FP64,
                                          tb.in, tb.out, b, 0, s);
        TDH_CUDA(cudaMemsetAsync(tb.ctr + 1, 0, sizeof(int), s));
        const ExecData& ex = st.rcls[r.cls];
        ExecParams<T> P = ragged_params<T>(st, ex, tb.in, tb.out, tb.offs, tb.list, tb.ctr,
                                           tb.ctr + 1, b);
        return dispatch<T>(ex.g, P, b, s);
    };
    TDH_TRY(launch());
    for (int i = 0; i < 4; ++i) {
        TDH_CUDA(cudaEventRecord(tb.ev[i], s));
        if (i < 3) TDH_TRY(launch());
    }
    TDH_CUDA(cudaEventSynchronize(tb.ev[3]));
    float best = 0;
    for (int i = 0; i < 3; ++i) {
        float t = 0;
        TDH_CUDA(cudaEventElapsedTime(&t, tb.ev[i], tb.ev[i + 1]));
        if (i == 0 || t < best) best = t;
    }
    *ms = best;
    return TDH_OK;
}

template <typename T>
int autotune_typed(tdh_plan_s& plan, int64_t batch, cudaStream_t s) {
    const int prec = plan.params.prec;
    std::vector<ConfigRef> cfgs;
    for (const ConfigRef& r : plan_configs(plan))  // only what has a choice to make
        if (schedule_candidates(prec, config_data(r).g.logL, r.cls >= 0).size() > 1)
            cfgs.push_back(r);
    if (cfgs.empty()) return TDH_OK;
    int64_t elems = 0, bmax = 0;
    for (const ConfigRef& r : cfgs) {
        int64_t b, len;
        tune_shape(r, batch, &b, &len);
        elems = std::max(elems, b * len);
        bmax = std::max(bmax, b);
    }
    TuneBuffers tb;
    int rc = TDH_OK;
    auto cleanup = [&] {
        cudaStreamSynchronize(s);
        for (cudaEvent_t e : tb.ev)
            if (e) cudaEventDestroy(e);
        dev_free(tb.in);
        dev_free(tb.out);
        dev_free(tb.offs);
        dev_free(tb.list);
        dev_free(tb.ctr);
    };
    if ((rc = dev_alloc(&tb.in, sizeof(T) * (size_t)elems)) ||
        (rc = dev_alloc(&tb.out, sizeof(T) * (size_t)elems)) ||
        (rc = dev_alloc_t(&tb.offs, (size_t)bmax + 1)) ||
        (rc = dev_alloc_t(&tb.list, (size_t)bmax)) || (rc = dev_alloc_t(&tb.ctr, 2))) {
        cleanup();
        return rc;
    }
    for (cudaEvent_t& e : tb.ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            set_error("autotune: event creation failed");
            cleanup();
            return TDH_ERR_CUDA;
        }
    k_fill_test<T><<<blocks_for(elems), kThreads, 0, s>>>(static_cast<T*>(tb.in), elems);
    if (cudaGetLastError() != cudaSuccess) {
        set_error("autotune: input fill launch failed");
        cleanup();
        return TDH_ERR_CUDA;
    }
    for (const ConfigRef& r : cfgs) {
        const std::vector<Geometry> cands =
            schedule_candidates(prec, config_data(r).g.logL, r.cls >= 0);
        if (cands.size() < 2) continue;
        int best = -1;
        float best_ms = 0;
        for (size_t i = 0; rc == TDH_OK && i < cands.size(); ++i) {
            float ms = 0;
            rc = rebuild_config(r, prec, cands[i], s);
            if (rc == TDH_OK) rc = time_config<T>(r, batch, tb, s, &ms);
            if (rc == TDH_OK && (best < 0 || ms < best_ms)) {
                best = (int)i;
                best_ms = ms;
            }
        }
        if (rc == TDH_OK) rc = rebuild_config(r, prec, cands[best], s);
        if (rc != TDH_OK) break;
    }
    cleanup();
    return rc;
}

}  // namespace

int exec_schedules(int prec, int logL, int ragged, int* out, int cap, int* count) {
    const std::vector<Geometry> c = schedule_candidates(prec, logL, ragged != 0);
    *count = (int)c.size();
    for (int i = 0; i < (int)c.size() && i < cap; ++i) {
        const int v[6] = {c[i].logLC, c[i].C, c[i].R, c[i].NT, c[i].MINB,
                          c[i].C > 8 ? (c[i].tma ? 2 : 1) : 0};
        for (int k = 0; k < 6; ++k) out[6 * i + k] = v[k];
    }
    return TDH_OK;
}

int exec_schedule_count(const tdh_plan_s& plan) {
    return (int)plan_configs(const_cast<tdh_plan_s&>(plan)).size();
}

int exec_schedule_info(const tdh_plan_s& plan, int config, int* info) {
    std::vector<ConfigRef> cfgs = plan_configs(const_cast<tdh_plan_s&>(plan));
    if (config < 0 || config >= (int)cfgs.size()) {
        set_error("configuration %d out of range (%d)", config, (int)cfgs.size());
        return TDH_ERR_INVALID_ARG;
    }
    const ConfigRef& r = cfgs[config];
    const Geometry& g = config_data(r).g;
    const std::vector<Geometry> cands = schedule_candidates(plan.params.prec, g.logL, r.cls >= 0);
    int idx = -1;
    for (size_t i = 0; i < cands.size(); ++i)
        if (same_schedule(cands[i], g)) idx = (int)i;
    const int v[8] = {g.logL, g.logLC, g.C, g.R, g.NT, g.MINB, idx, (int)cands.size()};
    for (int i = 0; i < 8; ++i) info[i] = v[i];
    return TDH_OK;
}

int exec_set_schedule(tdh_plan_s& plan, int index, cudaStream_t s) {
    if (index < 0) {
        set_error("schedule index must be >= 0");
        return TDH_ERR_INVALID_ARG;
    }
    for (const ConfigRef& r : plan_configs(plan)) {
        const std::vector<Geometry> cands =
            schedule_candidates(plan.params.prec, config_data(r).g.logL, r.cls >= 0);
        if (cands.empty()) continue;
        TDH_TRY(rebuild_config(r, plan.params.prec, cands[std::min<size_t>(index, cands.size() - 1)],
                               s));
    }
    return TDH_OK;
}

int exec_autotune(tdh_plan_s& plan, int64_t batch, cudaStream_t s) {
    if (batch < 1) {
        set_error("autotune batch must be >= 1");
        return TDH_ERR_INVALID_ARG;
    }
    if (plan.params.prec != TDH_FP64) return autotune_typed<float>(plan, batch, s);
    return autotune_typed<double>(plan, batch, s);
}

}  // namespace tdh
