// Multi-pass execute for FFT lengths beyond one thread-block cluster (L = C * LC, C > 8):
// the same decomposition as the cluster kernel, with the cross-CTA stage done through
// global memory between kernel launches instead of distributed shared memory.
//
// Per vector b and local slice k1 (z[k1 + C k2], k2 < LC), per rank term r:
//   mp_fwd   : u_r o v (v staged once in global memory), forward local DIF passes in
//              shared memory, local spectrum -> Y[b][k1][pos]
//   cross    : for every local position pos, the C values Y[b][*][pos]: twiddle
//              omega_L^{k1 f1(pos)}, C-point DFT, multiply by conj(S)/L, inverse C-point
//              DFT, conjugate twiddle (radix 16 x C/16 in registers for 16 <= C <= 256)
//   mp_inv   : inverse local DIT passes, W[b][k1][k2] += u_r o y
// then beta = D1 W (D2 for the adjoint).  Scratch (v, Y, W) is stream-ordered
// (the library's stream-ordered pool) and vectors are processed in chunks that bound it.
#include <cuda.h>
#include <algorithm>
#include <mutex>

#include "tdh_exec.cuh"

namespace tdh {
namespace {

template <typename T>
struct MPParams {
    using V = typename cx<T>::t;
    const T* in;
    T* out;
    int64_t n, L, K;
    int C, logC, shift, adjoint, full, sign_in, sign_out;
    const V* u;
    const V* spec;
    const int* perm;
    const V* thi;
    const V* tlo;
    const V* tw0;
    const V* twp;
    const T* din;
    const T* dout;
    const T* row0;
    V* vdec;  // [B][C][LC/2]
    V* Y;     // [B][C][LC]
    V* W;     // [B][C][LC/2]
    T* r0;    // [B] row-0 sum (forward) or g_0 (adjoint)
    const T* pair_c;  // rank-pair packing: output factor of each pair's second term
    int* status;      // the plan's device status word (a TMA wait that ran out)
};

constexpr int kEw = 256;

// Programmatic dependent launch between the kernels of one multi-pass execute: each kernel
// lets the next one be scheduled as soon as all of its own CTAs are running, and does only
// read-only set-up (twiddle tables, plan factors) before it waits for the previous kernel to
// complete and its writes to be visible.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute a[1];
    a[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    a[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = a;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename V>
__device__ __forceinline__ V omega_L(const V* thi, const V* tlo, int64_t e, int64_t L, int shift) {
    e &= (L - 1);
    return cmul(thi[e >> shift], tlo[e & (((int64_t)1 << shift) - 1)]);
}

// v in the decimated packed layout; W = 0; row-0 data
template <typename T, int LC>
__global__ void mp_load(const MPParams<T> P, int64_t b0, int64_t nb) {
    using V = typename cx<T>::t;
    const int64_t per = (int64_t)P.C * (LC / 2);
    const int64_t total = nb * per;
    for (int64_t i = (int64_t)blockIdx.x * kEw + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * kEw) {
        const int64_t bl = i / per, rem = i % per;
        const int64_t k1 = rem / (LC / 2), k2 = rem % (LC / 2);
        const int64_t a = k1 + (int64_t)P.C * k2;
        const T* in = P.in + (b0 + bl) * P.n;
        V v = mk<V>(0, 0);
        if (P.full) {
            if (a < P.n) {
                T x = in[a];
                if (P.sign_in && (a & 1)) x = -x;
                v = mk<V>(x * P.din[a], x * P.din[a]);
            }
        } else {
            const int64_t i0 = 2 * a;
            if (i0 < P.n) {
                T x1 = (i0 + 1 < P.n) ? in[i0 + 1] : T(0);
                if (P.sign_in) x1 = -x1;
                v = mk<V>(in[i0] * P.din[i0], (i0 + 1 < P.n) ? x1 * P.din[i0 + 1] : T(0));
            }
        }
        P.vdec[i] = v;
        P.W[i] = mk<V>(0, 0);
    }
}

// forward: r0[b] = sum_k row0[k] alpha_k; adjoint: r0[b] = g_0
template <typename T>
__global__ void mp_row0(const MPParams<T> P, int64_t b0) {
    __shared__ T red[kEw / 32];
    const T* in = P.in + (b0 + blockIdx.x) * P.n;
    if (P.adjoint) {
        if (threadIdx.x == 0) P.r0[blockIdx.x] = in[0];
        return;
    }
    T acc = T(0);
    for (int64_t k = threadIdx.x; k < P.n; k += kEw) {
        T x = in[k];
        if (P.sign_in && (k & 1)) x = -x;
        acc += P.row0[k] * x;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        T s = T(0);
        for (int w = 0; w < kEw / 32; ++w) s += red[w];
        P.r0[blockIdx.x] = s;
    }
}

template <typename T, int LOGLC, int R, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1) mp_fwd(const MPParams<T> P, int64_t r) {
    using V = typename cx<T>::t;
    constexpr PassGeom G{LOGLC, R};
    constexpr int LC = G.LC(), S0 = LC / R, J0 = S0 / NT, RL = G.rad(G.np() - 1);
    constexpr int TWP = G.twp_len();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* buf = reinterpret_cast<V*>(smem_raw);
    V* twt = buf + padded_len<V>(LC);
    const int tid = threadIdx.x;
    const int64_t bl = blockIdx.x / P.C;
    const int k1 = blockIdx.x % P.C;
    pdl_trigger();
    const V* vs = P.vdec + (bl * P.C + k1) * (LC / 2);
    const V* ur = P.u + (r * P.C + k1) * (LC / 2);
    V zl[J0][R / 2];  // every global load of the pass first: one latency for all groups
#pragma unroll
    for (int j = 0; j < J0; ++j)
#pragma unroll
        for (int q = 0; q < R / 2; ++q) zl[j][q] = ur[tid + j * NT + q * S0];
    for (int i = tid; i < TWP; i += NT) twt[i] = P.twp[i];  // overlaps the loads above
    pdl_wait();  // v was written by an earlier kernel
#pragma unroll
    for (int j = 0; j < J0; ++j)
#pragma unroll
        for (int q = 0; q < R / 2; ++q) zl[j][q] = cwmul(vs[tid + j * NT + q * S0], zl[j][q]);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < J0; ++j) {
        const int o = tid + j * NT;
        V x[R];
#pragma unroll
        for (int q = 0; q < R / 2; ++q) x[q] = zl[j][q];
        dif_halfzero<R>(x);
        const TwPow<R, V> wp(P.tw0[o]);
#pragma unroll
        for (int jj = 0; jj < R; ++jj) {
            const int p = bitrev(jj, R);
            buf[sidx<V>(o + p * S0)] = wp.mul(x[jj], p);
        }
    }
    __syncthreads();
    middle_fwd<1, LOGLC, R, NT, false>(buf, twt, (TcState*)nullptr);
#pragma unroll 1
    for (int g = tid; g < LC / RL; g += NT) {
        V x[RL];
#pragma unroll
        for (int q = 0; q < RL; ++q) x[q] = buf[sidx<V>(g * RL + q)];
        dif<RL>(x);
#pragma unroll
        for (int jj = 0; jj < RL; ++jj) buf[sidx<V>(g * RL + bitrev(jj, RL))] = x[jj];
    }
    __syncthreads();
    V* y = P.Y + (bl * P.C + k1) * LC;
    for (int pos = tid; pos < LC; pos += NT) y[pos] = buf[sidx<V>(pos)];
}

// Bring `bytes` (a multiple of 16, 16-byte aligned address) into L2 without waiting: one bulk
// prefetch per 16 KB piece, issued by the first threads of the block.
__device__ __forceinline__ void prefetch_l2(const void* p, int bytes) {
    constexpr int kPiece = 16384;
    const int pieces = (bytes + kPiece - 1) / kPiece;
    for (int i = threadIdx.x; i < pieces; i += blockDim.x) {
        const int sz = min(kPiece, bytes - i * kPiece);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                     :: "l"(static_cast<const char*>(p) + (size_t)i * kPiece), "r"(sz)
                     : "memory");
    }
}

template <typename T, int LOGLC, int R, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1) mp_inv(const MPParams<T> P, int64_t r) {
    using V = typename cx<T>::t;
    constexpr PassGeom G{LOGLC, R};
    constexpr int LC = G.LC(), S0 = LC / R, J0 = S0 / NT, RL = G.rad(G.np() - 1);
    constexpr int TWP = G.twp_len();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* buf = reinterpret_cast<V*>(smem_raw);
    V* twt = buf + padded_len<V>(LC);
    const int tid = threadIdx.x;
    const int64_t bl = blockIdx.x / P.C;
    const int k1 = blockIdx.x % P.C;
    pdl_trigger();
    const V* ur = P.u + (r * P.C + k1) * (LC / 2);
    const T cpair = (P.full && P.pair_c) ? P.pair_c[r] : T(1);
    V* w = P.W + (bl * P.C + k1) * (LC / 2);
    // the factor and accumulator slices of the last pass, on their way to L2 meanwhile
    prefetch_l2(ur, (int)sizeof(V) * (LC / 2));
    pdl_wait();  // Y and W were written by earlier kernels
    prefetch_l2(w, (int)sizeof(V) * (LC / 2));
    const V* y = P.Y + (bl * P.C + k1) * LC;
    constexpr int NY = LC / NT;  // the whole slice in one batch of loads
    static_assert(LC % NT == 0 && NY <= 32, "load batch");
    {
        V v[NY];
#pragma unroll
        for (int i = 0; i < NY; ++i) v[i] = y[tid + i * NT];
        for (int i = tid; i < TWP; i += NT) twt[i] = P.twp[i];  // overlaps the loads above
#pragma unroll
        for (int i = 0; i < NY; ++i) buf[sidx<V>(tid + i * NT)] = v[i];
    }
    __syncthreads();
#pragma unroll 1
    for (int g = tid; g < LC / RL; g += NT) {
        V x[RL];
#pragma unroll
        for (int p = 0; p < RL; ++p) x[bitrev(p, RL)] = buf[sidx<V>(g * RL + p)];
        dit<RL>(x);
#pragma unroll
        for (int q = 0; q < RL; ++q) buf[sidx<V>(g * RL + q)] = x[q];
    }
    __syncthreads();
    middle_inv<G.np() - 2, LOGLC, R, NT, false>(buf, twt, (TcState*)nullptr);
#pragma unroll
    for (int j = 0; j < J0; ++j) {
        const int o = tid + j * NT;
        // global loads first: their latency overlaps the pass (radix 32, whose 64 registers
        // of data leave no room for both, loads the accumulators after the butterflies)
        constexpr bool kEarlyW = R <= 16;
        V ul[R / 2], wl[R / 2];
#pragma unroll
        for (int q = 0; q < R / 2; ++q) {
            ul[q] = ur[o + q * S0];
            if (kEarlyW) wl[q] = w[o + q * S0];
        }
        V x[R];
        {
            const TwPow<R, V> wp(P.tw0[o]);
#pragma unroll
            for (int p = 0; p < R; ++p) x[bitrev(p, R)] = wp.mulc(buf[sidx<V>(o + p * S0)], p);
        }
        dit_halfout<R>(x);
        if constexpr (!kEarlyW) {
#pragma unroll
            for (int q = 0; q < R / 2; ++q) wl[q] = w[o + q * S0];
        }
#pragma unroll
        for (int q = 0; q < R / 2; ++q) {
            const V uu = ul[q];
            V acc = wl[q];
            if (P.full) {
                acc.x = fma(uu.y * cpair, x[q].y, fma(uu.x, x[q].x, acc.x));
            } else {
                acc.x = fma(uu.x, x[q].x, acc.x);
                acc.y = fma(uu.y, x[q].y, acc.y);
            }
            w[o + q * S0] = acc;
        }
    }
}

// Cross stage for C outside [16, 256]: one warp per local position, C values in shared memory
// (padded rows), radix 2.
template <typename T, int LC>
__global__ void __launch_bounds__(256) mp_cross(const MPParams<T> P) {
    using V = typename cx<T>::t;
    constexpr int PPB = 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = P.C, ld = C + 1;
    V* tile = reinterpret_cast<V*>(smem_raw);  // [PPB][C + 1]
    V* twc = tile + PPB * ld;                  // omega_C^k, k < C/2
    const int64_t bl = blockIdx.y;
    const int pos0 = blockIdx.x * PPB;
    pdl_trigger();
    for (int k = threadIdx.x; k < C / 2; k += blockDim.x)
        twc[k] = omega_L(P.thi, P.tlo, (int64_t)k * (P.L / C), P.L, P.shift);
    pdl_wait();  // Y was written by the previous kernel
    const V* Yb = P.Y + bl * (int64_t)C * LC;
    V* Yw = P.Y + bl * (int64_t)C * LC;
    for (int idx = threadIdx.x; idx < PPB * C; idx += blockDim.x) {
        const int k1 = idx / PPB, p = idx % PPB;
        const int pos = pos0 + p;
        const V w = omega_L(P.thi, P.tlo, (int64_t)k1 * P.perm[pos], P.L, P.shift);
        tile[p * ld + k1] = cmul(Yb[(int64_t)k1 * LC + pos], w);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int p = warp; p < PPB; p += nw) {
        V* x = tile + p * ld;
        for (int h = C / 2; h >= 1; h >>= 1) {
            for (int i = lane; i < C / 2; i += 32) {
                const int j = i % h, i0 = (i / h) * 2 * h + j, i1 = i0 + h;
                const V a = x[i0], c = x[i1];
                x[i0] = cadd(a, c);
                x[i1] = cmul(csub(a, c), twc[j * (C / (2 * h))]);
            }
            __syncwarp();
        }
        const int64_t pos = pos0 + p;
        for (int i = lane; i < C; i += 32) {
            const int f2 = (int)(__brev((unsigned)i) >> (32 - P.logC));
            const V s = P.spec[(int64_t)f2 * LC + pos];
            x[i] = P.adjoint ? cmulc(x[i], s) : cmul(x[i], s);
        }
        __syncwarp();
        for (int h = 1; h <= C / 2; h <<= 1) {
            for (int i = lane; i < C / 2; i += 32) {
                const int j = i % h, i0 = (i / h) * 2 * h + j, i1 = i0 + h;
                const V a = x[i0], c = cmulc(x[i1], twc[j * (C / (2 * h))]);
                x[i0] = cadd(a, c);
                x[i1] = csub(a, c);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < PPB * C; idx += blockDim.x) {
        const int k1 = idx / PPB, p = idx % PPB;
        const int pos = pos0 + p;
        const V w = omega_L(P.thi, P.tlo, (int64_t)k1 * P.perm[pos], P.L, P.shift);
        Yw[(int64_t)k1 * LC + pos] = cmulc(tile[p * ld + k1], w);
    }
}

// Cross stage for 16 <= C <= 256 slices: the C-point DFT of each local position split as
// C = 16 C2 (Cooley-Tukey: k1 = a + C2 b, f = c + 16 d,
//   X[c + 16 d] = sum_a omega_C2^{a d} omega_C^{a c} sum_b omega_16^{b c} x[a + C2 b]),
// each short DFT in registers, PP = 4096 / C positions of a block in shared memory
// ([PP][C + 1]: every phase reads with consecutive positions on consecutive lanes, so the
// padded rows give conflict-free banks and the global accesses are coalesced).  Then the
// spectrum (stored [f][pos]) and the inverse in the reverse order.
template <typename T, int LC, int C>
__global__ void __launch_bounds__(256) mp_cross16(const MPParams<T> P) {
    using V = typename cx<T>::t;
    constexpr int NTH = 256, PP = 4096 / C, C2 = C / 16, LD = C + 1;
    static_assert(C >= 16 && C <= 256 && LC % PP == 0 && PP * C2 == NTH, "cross-stage shape");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tile = reinterpret_cast<V*>(smem_raw);  // [PP][LD]
    V* twc = tile + PP * LD;                   // omega_C^k, k < C
    // float64: the phase-A twiddles kept for phase E ([PP][LD]); float32 recomputes them
    // (measured: keeping them costs float32 more in occupancy than the table loads it saves)
    constexpr bool kKeepW = sizeof(T) == 8;
    V* wt = twc + C;
    const int tid = threadIdx.x;
    const int64_t bl = blockIdx.y;
    const int pos0 = blockIdx.x * PP;
    pdl_trigger();
    for (int k = tid; k < C; k += NTH)
        twc[k] = omega_L(P.thi, P.tlo, (int64_t)k * (P.L / C), P.L, P.shift);
    pdl_wait();  // Y was written by the previous kernel
    V* Yb = P.Y + bl * (int64_t)C * LC;
    // phases A and E: thread (p, k0) moves slices k1 = k0 + C2 i, i < 16, of position p (all
    // loads of a thread independent, so they are in flight together)
    const int pB = tid % PP, aB = tid / PP;
    const int64_t fpos = P.perm[pos0 + pB];
    {
        // omega_L^{k1 fpos} for k1 = aB + C2 i.  float32: omega_L^{aB fpos} times the powers
        // of omega_L^{C2 fpos} (two table products and a depth-4 power tree per thread
        // instead of sixteen table products: far fewer loads queued on the load/store unit);
        // float64, where the multiplies cost more than the loads, one table product each.
        V y[16], w[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) y[i] = Yb[(int64_t)(aB + C2 * i) * LC + pos0 + pB];
        if constexpr (sizeof(T) == 4) {
            const V wb = omega_L(P.thi, P.tlo, (int64_t)aB * fpos, P.L, P.shift);
            powers<16>(omega_L(P.thi, P.tlo, (int64_t)C2 * fpos, P.L, P.shift), w);
#pragma unroll
            for (int i = 0; i < 16; ++i) w[i] = cmul(wb, w[i]);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                w[i] = omega_L(P.thi, P.tlo, (int64_t)(aB + C2 * i) * fpos, P.L, P.shift);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            tile[pB * LD + aB + C2 * i] = cmul(y[i], w[i]);
            if constexpr (kKeepW) wt[pB * LD + aB + C2 * i] = w[i];
        }
    }
    __syncthreads();
    // phases B and D: one (position, a) per thread
    {
        V x[16];
#pragma unroll
        for (int b = 0; b < 16; ++b) x[b] = tile[pB * LD + aB + C2 * b];
        dif<16>(x);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
            const int c = bitrev(jj, 16);
            tile[pB * LD + aB + C2 * c] = (aB * c == 0) ? x[jj] : cmul(x[jj], twc[aB * c]);
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int g = tid; g < PP * 16; g += NTH) {
        const int p = g % PP, c = g / PP;
        const int64_t pos = pos0 + p;
        V x[C2];
#pragma unroll
        for (int a = 0; a < C2; ++a) x[a] = tile[p * LD + a + C2 * c];
        dif<C2>(x);
#pragma unroll
        for (int jj = 0; jj < C2; ++jj) {
            const V sv = P.spec[(int64_t)(c + 16 * bitrev(jj, C2)) * LC + pos];
            x[jj] = P.adjoint ? cmulc(x[jj], sv) : cmul(x[jj], sv);
        }
        dit<C2>(x);
#pragma unroll
        for (int a = 0; a < C2; ++a)
            tile[p * LD + a + C2 * c] = (a * c == 0) ? x[a] : cmulc(x[a], twc[a * c]);
    }
    __syncthreads();
    {
        V x[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) x[jj] = tile[pB * LD + aB + C2 * bitrev(jj, 16)];
        dit<16>(x);
#pragma unroll
        for (int b = 0; b < 16; ++b) tile[pB * LD + aB + C2 * b] = x[b];
    }
    __syncthreads();
    if constexpr (kKeepW) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int k1 = aB + C2 * i;
            Yb[(int64_t)k1 * LC + pos0 + pB] = cmulc(tile[pB * LD + k1], wt[pB * LD + k1]);
        }
    } else {
        V w[16];
        const V wb = omega_L(P.thi, P.tlo, (int64_t)aB * fpos, P.L, P.shift);
        powers<16>(omega_L(P.thi, P.tlo, (int64_t)C2 * fpos, P.L, P.shift), w);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int k1 = aB + C2 * i;
            Yb[(int64_t)k1 * LC + pos0 + pB] = cmulc(tile[pB * LD + k1], cmul(wb, w[i]));
        }
    }
}

// The same cross stage with the block of Y it works on (C slices x PP positions) moved by the
// tensor memory accelerator: one bulk tensor copy in, issued by one thread once the previous
// kernel's writes are visible, while the others form their twiddles; one bulk copy out.  The
// block stays in shared memory in the copy's own layout, slice-major ([C][PP], or
// [NX][C][PP / NX] when a row exceeds the 256-element box limit): every phase reads
// consecutive positions on consecutive lanes, so no padding is needed.
constexpr uint64_t kTmaWaitNs = 1000000000ull;

template <typename T, int LC, int C>
__global__ void __launch_bounds__(256) mp_cross16_tma(const MPParams<T> P,
                                                      const __grid_constant__ CUtensorMap tmap) {
    using V = typename cx<T>::t;
    constexpr int NTH = 256, PP = 4096 / C, C2 = C / 16;
    constexpr int XE = PP * (int)sizeof(V) / 8;  // 8-byte elements per row of the block
    constexpr int NX = XE > 256 ? XE / 256 : 1;  // copies along x (box rows <= 256 elements)
    constexpr int PX = PP / NX;                  // positions per copy
    static_assert(C >= 16 && C <= 256 && LC % PP == 0 && PP * C2 == NTH, "cross-stage shape");
    static_assert(PX * NX == PP && PX * (int)sizeof(V) % 16 == 0, "TMA box rows");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // bulk tensor copies need a 128-byte aligned shared address; the dynamic region is only
    // guaranteed 16 (static shared variables come first), so the block starts at the next
    // 128-byte boundary (the launch reserves 128 bytes for this)
    const uint32_t pad = (128u - (tc::smem_u32(smem_raw) & 127u)) & 127u;
    V* tile = reinterpret_cast<V*>(smem_raw + pad);  // the block: (k1, p) at tix(k1, p)
    V* twc = tile + C * PP;                          // omega_C^k, k < C
    constexpr bool kKeepW = sizeof(T) == 8;    // float64 keeps the phase-A twiddles (see above)
    V* wt = twc + C;
    auto tix = [](int k1, int p) { return (p / PX) * (C * PX) + k1 * PX + (p % PX); };
    __shared__ __align__(8) uint64_t mbar;
    const int tid = threadIdx.x;
    const int64_t bl = blockIdx.y;
    const int pos0 = blockIdx.x * PP;
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&mbar), 1);
        tc::mbar_fence_init();
    }
    pdl_trigger();
    for (int k = tid; k < C; k += NTH)
        twc[k] = omega_L(P.thi, P.tlo, (int64_t)k * (P.L / C), P.L, P.shift);
    __syncthreads();  // the mbarrier is initialised
    pdl_wait();       // Y was written by the previous kernel
    // the copies' alignment rules, checked before any copy is issued (a violation would be
    // a device fault): 128-byte shared addresses, x offsets in multiples of 16 bytes
    const bool aligned = (tc::smem_u32(tile) & 127u) == 0 &&
                         ((pos0 * (int)sizeof(V)) & 15) == 0;
    if (tid == 0) {
        if (aligned) {
            tc::mbar_arrive_expect_tx(tc::smem_u32(&mbar), (uint32_t)(C * PP * sizeof(V)));
            for (int i = 0; i < NX; ++i)
                tc::tma_load_3d(tc::smem_u32(tile + i * C * PX), &tmap,
                                (pos0 + i * PX) * (int)sizeof(V) / 8, 0, (int)bl,
                                tc::smem_u32(&mbar));
        } else {
            if (P.status) atomicOr(P.status, TDH_STATUS_FAULT);
            tc::mbar_arrive(tc::smem_u32(&mbar));  // no copy: complete the phase at once
        }
    }
    const int pB = tid % PP, aB = tid / PP;
    const int64_t fpos = P.perm[pos0 + pB];
    V w[16];  // omega_L^{k1 fpos}, k1 = aB + C2 i, formed while the copy is in flight
    if constexpr (sizeof(T) == 4) {
        const V wb = omega_L(P.thi, P.tlo, (int64_t)aB * fpos, P.L, P.shift);
        powers<16>(omega_L(P.thi, P.tlo, (int64_t)C2 * fpos, P.L, P.shift), w);
#pragma unroll
        for (int i = 0; i < 16; ++i) w[i] = cmul(wb, w[i]);
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i)
            w[i] = omega_L(P.thi, P.tlo, (int64_t)(aB + C2 * i) * fpos, P.L, P.shift);
    }
    if (!tc::mbar_wait_bounded(tc::smem_u32(&mbar), 0, kTmaWaitNs) && P.status)
        atomicOr(P.status, TDH_STATUS_TIMEOUT);
    // phase A: twiddles in place
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int e = tix(aB + C2 * i, pB);
        tile[e] = cmul(tile[e], w[i]);
        if constexpr (kKeepW) wt[e] = w[i];
    }
    __syncthreads();
    // phases B and D: one (position, a) per thread
    {
        V x[16];
#pragma unroll
        for (int b = 0; b < 16; ++b) x[b] = tile[tix(aB + C2 * b, pB)];
        dif<16>(x);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
            const int c = bitrev(jj, 16);
            tile[tix(aB + C2 * c, pB)] = (aB * c == 0) ? x[jj] : cmul(x[jj], twc[aB * c]);
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int g = tid; g < PP * 16; g += NTH) {
        const int p = g % PP, c = g / PP;
        const int64_t pos = pos0 + p;
        V x[C2];
#pragma unroll
        for (int a = 0; a < C2; ++a) x[a] = tile[tix(a + C2 * c, p)];
        dif<C2>(x);
#pragma unroll
        for (int jj = 0; jj < C2; ++jj) {
            const V sv = P.spec[(int64_t)(c + 16 * bitrev(jj, C2)) * LC + pos];
            x[jj] = P.adjoint ? cmulc(x[jj], sv) : cmul(x[jj], sv);
        }
        dit<C2>(x);
#pragma unroll
        for (int a = 0; a < C2; ++a)
            tile[tix(a + C2 * c, p)] = (a * c == 0) ? x[a] : cmulc(x[a], twc[a * c]);
    }
    __syncthreads();
    {
        V x[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) x[jj] = tile[tix(aB + C2 * bitrev(jj, 16), pB)];
        dit<16>(x);
#pragma unroll
        for (int b = 0; b < 16; ++b) tile[tix(aB + C2 * b, pB)] = x[b];
    }
    __syncthreads();
    // phase E: conjugate twiddles in place, then the block back to Y
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int e = tix(aB + C2 * i, pB);
        tile[e] = cmulc(tile[e], kKeepW ? wt[e] : w[i]);
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && aligned) {
        for (int i = 0; i < NX; ++i)
            tc::tma_store_3d(&tmap, (pos0 + i * PX) * (int)sizeof(V) / 8, 0, (int)bl,
                             tc::smem_u32(tile + i * C * PX));
        tc::bulk_commit_group();
        tc::bulk_wait_read();  // shared memory stays valid until the copy has read it
    }
}

// cuTensorMapEncodeTiled from the driver (through the runtime; the library links no driver
// library), looked up once.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    });
    return fn;
}

// Tensor map of a chunk's Y, [nb][C][LC] complex values, as 8-byte elements: x = position
// (times sizeof(V) / 8), y = slice, z = vector; box = (PX positions, C slices, 1 vector).
template <typename T>
int cross_tensor_map(const MPParams<T>& Q, int LC, int64_t nb, CUtensorMap* tm) {
    using V = typename cx<T>::t;
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return TDH_ERR_UNSUPPORTED;
    }
    const int PP = 4096 / Q.C;
    const int XE = PP * (int)sizeof(V) / 8;
    const int NX = XE > 256 ? XE / 256 : 1;
    const cuuint64_t dims[3] = {(cuuint64_t)LC * sizeof(V) / 8, (cuuint64_t)Q.C, (cuuint64_t)nb};
    const cuuint64_t strides[2] = {(cuuint64_t)LC * sizeof(V), (cuuint64_t)Q.C * LC * sizeof(V)};
    const cuuint32_t box[3] = {(cuuint32_t)(XE / NX), (cuuint32_t)Q.C, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, Q.Y, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return TDH_ERR_CUDA;
    }
    return TDH_OK;
}

template <typename T, int LC, int C>
int cross16_tma_launch(const MPParams<T>& Q, int64_t nb, const CUtensorMap& tm, cudaStream_t s) {
    using V = typename cx<T>::t;
    constexpr int PP = 4096 / C;
    constexpr size_t smem = (size_t)((sizeof(T) == 8 ? 2 : 1) * PP * C + C) * sizeof(V) + 128;
    static PerDevice attr_once;
    const cudaError_t err = per_device(attr_once, [&](int*) {
        return cudaFuncSetAttribute(mp_cross16_tma<T, LC, C>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    cudaError_t e = err;
    if (e == cudaSuccess)
        e = launch_pdl(mp_cross16_tma<T, LC, C>, dim3(LC / PP, (unsigned)nb), dim3(256), smem, s,
                       Q, tm);
    if (e != cudaSuccess) {
        set_error("multi-pass cross stage (TMA): %s", cudaGetErrorString(e));
        return TDH_ERR_CUDA;
    }
    note_launches(1);
    return TDH_OK;
}

template <typename T, int LC, int C>
int cross16_launch(const MPParams<T>& Q, int64_t nb, cudaStream_t s) {
    using V = typename cx<T>::t;
    constexpr int PP = 4096 / C;
    constexpr size_t smem = (size_t)((sizeof(T) == 8 ? 2 : 1) * PP * (C + 1) + C) * sizeof(V);
    static PerDevice attr_once;
    const cudaError_t err = per_device(attr_once, [&](int*) {
        return cudaFuncSetAttribute(mp_cross16<T, LC, C>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (err != cudaSuccess) {
        set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(err));
        return TDH_ERR_CUDA;
    }
    const cudaError_t e =
        launch_pdl(mp_cross16<T, LC, C>, dim3(LC / PP, (unsigned)nb), dim3(256), smem, s, Q);
    if (e != cudaSuccess) {
        set_error("multi-pass cross stage: %s", cudaGetErrorString(e));
        return TDH_ERR_CUDA;
    }
    note_launches(1);
    return TDH_OK;
}

// The cross stage for one rank term of a chunk of nb vectors (tm: the chunk's tensor map
// when the schedule moves the block by TMA, else null).
template <typename T, int LC>
int cross_launch(const MPParams<T>& Q, int64_t nb, size_t smem_cross, const CUtensorMap* tm,
                 cudaStream_t s) {
    if (tm) {
        switch (Q.C) {
        case 16: return cross16_tma_launch<T, LC, 16>(Q, nb, *tm, s);
        case 32: return cross16_tma_launch<T, LC, 32>(Q, nb, *tm, s);
        case 64: return cross16_tma_launch<T, LC, 64>(Q, nb, *tm, s);
        case 128: return cross16_tma_launch<T, LC, 128>(Q, nb, *tm, s);
        case 256: return cross16_tma_launch<T, LC, 256>(Q, nb, *tm, s);
        default: break;
        }
    }
    switch (Q.C) {
    case 16: return cross16_launch<T, LC, 16>(Q, nb, s);
    case 32: return cross16_launch<T, LC, 32>(Q, nb, s);
    case 64: return cross16_launch<T, LC, 64>(Q, nb, s);
    case 128: return cross16_launch<T, LC, 128>(Q, nb, s);
    case 256: return cross16_launch<T, LC, 256>(Q, nb, s);
    default: {
        const cudaError_t e =
            launch_pdl(mp_cross<T, LC>, dim3(LC / 16, (unsigned)nb), dim3(256), smem_cross, s, Q);
        if (e != cudaSuccess) {
            set_error("multi-pass cross stage: %s", cudaGetErrorString(e));
            return TDH_ERR_CUDA;
        }
        note_launches(1);
        return TDH_OK;
    }
    }
}

template <typename T, int LC>
__global__ void mp_store(const MPParams<T> P, int64_t b0, int64_t nb) {
    using V = typename cx<T>::t;
    pdl_wait();  // W (and the row-0 sums) were written by earlier kernels
    const int64_t per_out = P.n;
    const int64_t total = nb * per_out;
    for (int64_t i = (int64_t)blockIdx.x * kEw + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * kEw) {
        const int64_t bl = i / per_out, k = i % per_out;
        const int64_t a = P.full ? k : k / 2;
        const int64_t k1 = a % P.C, k2 = a / P.C;
        const V w = P.W[(bl * P.C + k1) * (LC / 2) + k2];
        T v = (P.full || !(k & 1)) ? w.x : w.y;
        v *= P.dout[k];
        if (P.row0 && P.adjoint) v += P.row0[k] * P.r0[bl];
        if (P.row0 && !P.adjoint && k == 0) v = P.r0[bl];
        if (P.sign_out && (k & 1)) v = -v;
        P.out[(b0 + bl) * P.n + k] = v;
    }
}

template <typename T, int LOGLC, int R, int NT>
int run_typed(const Step& st, const void* in, void* out, int64_t batch, int adjoint,
              cudaStream_t s) {
    using V = typename cx<T>::t;
    constexpr PassGeom G{LOGLC, R};
    constexpr int LC = G.LC();
    const ExecData& ex = st.ex;
    if (ex.g.logLC != LOGLC || ex.g.R != R) {
        set_error("multi-pass geometry mismatch");
        return TDH_ERR_UNSUPPORTED;
    }
    MPParams<T> P{};
    P.in = static_cast<const T*>(in);
    P.out = static_cast<T*>(out);
    P.n = st.n;
    P.C = ex.g.C;
    P.logC = ilog2(P.C);
    P.L = (int64_t)1 << ex.g.logL;
    P.K = st.full ? (st.K + 1) / 2 : st.K;
    P.shift = ex.twl_shift;
    P.adjoint = adjoint;
    P.full = st.full;
    P.sign_in = st.sign_in;
    P.sign_out = st.sign_out;
    P.u = static_cast<const V*>(ex.u);
    P.spec = static_cast<const V*>(ex.spec);
    P.perm = ex.perm;
    P.thi = static_cast<const V*>(ex.twl_hi);
    P.tlo = static_cast<const V*>(ex.twl_lo);
    P.tw0 = static_cast<const V*>(ex.tw0);
    P.twp = static_cast<const V*>(ex.twp);
    P.din = static_cast<const T*>(adjoint ? st.d1x : st.d2x);
    P.dout = static_cast<const T*>(adjoint ? st.d2x : st.d1x);
    P.row0 = static_cast<const T*>(st.row0);
    P.pair_c = static_cast<const T*>(st.pair_c);
    P.status = st.status;

    // chunk the batch so the scratch stays below ~2 GB
    const size_t per_vec = sizeof(V) * (size_t)P.L * 2 + sizeof(T);
    int64_t chunk = std::max<int64_t>(1, (int64_t)((size_t)2 << 30) / (int64_t)per_vec);
    chunk = std::min(chunk, batch);
    char* scratch = nullptr;
    const size_t bytes = per_vec * (size_t)chunk + 256;
    TDH_TRY(scratch_alloc(reinterpret_cast<void**>(&scratch), bytes, s));
    P.vdec = reinterpret_cast<V*>(scratch);
    P.W = P.vdec + (size_t)chunk * P.L / 2;
    P.Y = P.W + (size_t)chunk * P.L / 2;
    P.r0 = reinterpret_cast<T*>(P.Y + (size_t)chunk * P.L);

    constexpr size_t smem_pass = (size_t)(padded_len<V>(LC) + G.twp_len()) * sizeof(V);
    const size_t smem_cross = (size_t)(16 * (P.C + 1) + P.C / 2) * sizeof(V);
    static PerDevice attr_once;
    const cudaError_t attr_err = per_device(attr_once, [&](int*) {
        cudaError_t e = cudaFuncSetAttribute(mp_fwd<T, LOGLC, R, NT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_pass);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(mp_inv<T, LOGLC, R, NT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_pass);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(mp_cross<T, LC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(V) * (16 * 513 + 256)));
        return e;
    });
    int rc = TDH_OK;
    if (attr_err != cudaSuccess) {
        set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(attr_err));
        rc = TDH_ERR_CUDA;
    }
    for (int64_t b0 = 0; rc == TDH_OK && b0 < batch; b0 += chunk) {
        const int64_t nb = std::min(chunk, batch - b0);
        MPParams<T> Q = P;
        Q.in = P.in + b0 * P.n;
        const unsigned ew = (unsigned)std::min<int64_t>((nb * P.L / 2 + kEw - 1) / kEw, 4096);
        mp_load<T, LC><<<ew, kEw, 0, s>>>(Q, 0, nb);
        if (P.row0) mp_row0<T><<<(unsigned)nb, kEw, 0, s>>>(Q, 0);
        note_launches(P.row0 ? 2 : 1);
        cudaError_t e = cudaSuccess;
        const dim3 gp((unsigned)(nb * P.C)), bp(NT);
        CUtensorMap tm;
        const bool use_tma = ex.g.tma && P.C >= 16 && P.C <= 256;
        if (use_tma) rc = cross_tensor_map<T>(Q, LC, nb, &tm);
        for (int64_t r = 0; rc == TDH_OK && e == cudaSuccess && r < P.K; ++r) {
            e = launch_pdl(mp_fwd<T, LOGLC, R, NT>, gp, bp, smem_pass, s, Q, r);
            if (e != cudaSuccess) break;
            rc = cross_launch<T, LC>(Q, nb, smem_cross, use_tma ? &tm : nullptr, s);
            if (rc != TDH_OK) break;
            e = launch_pdl(mp_inv<T, LOGLC, R, NT>, gp, bp, smem_pass, s, Q, r);
            if (e == cudaSuccess) note_launches(2);
        }
        if (rc != TDH_OK) break;
        Q.in = P.in;
        const unsigned eo = (unsigned)std::min<int64_t>((nb * P.n + kEw - 1) / kEw, 4096);
        if (e == cudaSuccess) e = launch_pdl(mp_store<T, LC>, dim3(eo), dim3(kEw), 0, s, Q, b0, nb);
        if (e == cudaSuccess) note_launches(1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("multi-pass launch: %s", cudaGetErrorString(e));
            rc = TDH_ERR_CUDA;
        }
    }
    scratch_free(scratch, s);
    return rc;
}

}  // namespace

int mp_launch(const Step& st, int prec, const void* in, void* out, int64_t batch, int adjoint,
              cudaStream_t s) {
    if (st.ex.g.C > 512) {
        set_error("multi-pass cross stage supports at most 512 slices");
        return TDH_ERR_UNSUPPORTED;
    }
    // slices one below the shared-memory cap run two CTAs per SM; longer FFTs keep full slices
    if (prec != TDH_FP64) {
        const bool r32 = st.ex.g.R == 32;
        if (st.ex.g.logLC == 13)
            return r32 ? run_typed<float, 13, 32, 256>(st, in, out, batch, adjoint, s)
                       : run_typed<float, 13, 16, 256>(st, in, out, batch, adjoint, s);
        return r32 ? run_typed<float, 14, 32, 512>(st, in, out, batch, adjoint, s)
                   : run_typed<float, 14, 16, 512>(st, in, out, batch, adjoint, s);
    }
    return st.ex.g.logLC == 12 ? run_typed<double, 12, 8, 256>(st, in, out, batch, adjoint, s)
                               : run_typed<double, 13, 8, 512>(st, in, out, batch, adjoint, s);
}

}  // namespace tdh
