// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "tdh.h"

namespace tdh {

void set_error(const char* fmt, ...);
void clear_error();

#define TDH_CUDA(expr)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            ::tdh::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),     \
                             __FILE__, __LINE__);                                        \
            return TDH_ERR_CUDA;                                                         \
        }                                                                                \
    } while (0)

#define TDH_TRY(expr)                                                                    \
    do {                                                                                 \
        int rc_ = (expr);                                                                \
        if (rc_ != TDH_OK) return rc_;                                                   \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Device allocation that records failures as TDH_ERR_NOMEM.
int dev_alloc(void** p, size_t bytes);
template <typename T>
int dev_alloc_t(T** p, size_t count) {
    return dev_alloc(reinterpret_cast<void**>(p), count * sizeof(T));
}
void dev_free(void* p);
// Stream-ordered execute scratch from the library's per-device pool (kept mapped).
int scratch_alloc(void** p, size_t bytes, cudaStream_t s);
void scratch_free(void* p, cudaStream_t s);

int sm_count();
// Allocation bookkeeping: {allocations made, plan blocks live, scratch blocks live}; and the
// test hook that makes the k-th allocation from now fail (k = 0: none).
void alloc_stats(int64_t* out);
void fail_alloc_after(int64_t k);
// Test hook: while set, tensor-core passes issue no products (their bounded waits run out).
int tc_stall_enabled();
void set_tc_stall(int on);

// One-time set-up per device (kernel attributes, occupancy queries): `f(int* val)` returns a
// cudaError_t and runs once for each device that is current when it is needed; its result
// code and *val are kept per device.
constexpr int kDeviceSlots = 64;
struct PerDevice {
    std::once_flag flag[kDeviceSlots];
    cudaError_t err[kDeviceSlots] = {};
    int val[kDeviceSlots] = {};
};
template <typename F>
cudaError_t per_device(PerDevice& pd, F&& f, int* val = nullptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kDeviceSlots) return cudaErrorInvalidDevice;
    std::call_once(pd.flag[dev], [&] { pd.err[dev] = f(&pd.val[dev]); });
    if (val) *val = pd.val[dev];
    return pd.err[dev];
}

// Count kernel launches made by execute calls (reported by tdh_launch_count).
void note_launches(int64_t k);

// ----------------------------------------------------------------------------- a1
// Fill t[n], h[2n-1], d1[n], d2[n] (device, float64) for `kind`; p = kind parameters.
int symbols_launch(int kind, int64_t n, const double* p, double* t, double* h, double* d1,
                   double* d2, cudaStream_t s);

// ----------------------------------------------------------------------------- a2
// Pivoted Cholesky of H[j,k] = h[j+k] (w null) or of the congruent W H W, entries
// w_j h[j+k] w_k (w: n positive weights), j,k in [j0,n); u: [kmax][n]; pivots: [kmax].
// *K receives the rank (synchronises `s`).
int pchol_run(const double* h, const double* w, int64_t n, int64_t j0, double tol, int64_t kmax,
              double* u, int64_t* pivots, int64_t* K, cudaStream_t s);
// Weights w_j = sqrt(|D1_j D2_j|) of the accuracy-targeted factorisation (1 where zero), and
// the conversion of factors of W H W back to factors of H (u[r][j] /= w_j).
int pchol_weights(const double* d1, const double* d2, const double* so, const double* si,
                  int64_t n, double* w, cudaStream_t s);
int pchol_unweight(double* u, const double* w, int64_t K, int64_t n, cudaStream_t s);

// Accuracy-targeted truncation of the rank-K factors u [K][n] of W H W (w null: of H; block
// j, k >= j0): *Kout = the fewest terms K' <= K whose bound B(K') = max|t| max_j |D1_j / w_j|
// sqrt(d_j) max_k |D2_k / w_k| sqrt(d_k) <= target (d: residual diagonal of W H W after K'
// steps; D1, D2 times the optional scalings so, si), else K.  *bound (may be null) receives
// B(*Kout).  Synchronises s.
int pchol_truncate(const double* h, const double* w, const double* u, int64_t n, int64_t j0,
                   int64_t K, const double* t, const double* d1, const double* d2,
                   const double* so, const double* si, double target, int64_t* Kout,
                   double* bound, cudaStream_t s);

// ----------------------------------------------------------------------------- a3-a7
// FFT geometry of one execute configuration: L = C * LC points, local radix R.
struct Geometry {
    int prec;   // TDH_FP32 / TDH_FP64
    int logL;   // L = 2^logL complex points
    int logLC;  // per-CTA local length
    int C;      // cluster size (CTAs per vector)
    int R;      // radix of the local passes
    int NT;     // threads per CTA
    int MINB;   // CTAs per SM the kernel's registers are capped for (launch bounds)
    int tc;     // 1: middle passes as split-bfloat16 tensor-core DFT products (TDH_BF16X3)
    int tma;    // multi-pass, 16 <= C <= 256: the cross stage's block moved by TMA copies
};

// Device data of one execute configuration.
struct ExecData {
    Geometry g{};
    int64_t m = 0;        // complex length of the packed vector (ceil(n/2))
    void* spec = nullptr; // [LC][C] complex: conj(DFT(symbol)) / L in the kernel's order
    void* twx = nullptr;  // [LC] complex: omega_L^{f1(pos)} (C > 1)
    void* tw0 = nullptr;  // [LC/R] complex: omega_LC^o, pass-0 twiddle bases
    void* twp = nullptr;  // later-pass twiddle tables, concatenated [p][o] blocks
    int64_t twp_len = 0;  // complex entries in twp
    void* u = nullptr;    // [K][C][u_stride] complex: factors decimated by C (packed pairs)
    int64_t u_stride = 0;
    bool u_owned = true;
    // multi-pass execution (C above the cluster limit: exchange through global memory)
    int multipass = 0;
    int* perm = nullptr;     // [LC] natural frequency of each local position
    void* twl_hi = nullptr;  // omega_L^{i << twl_shift}
    void* twl_lo = nullptr;  // omega_L^{i}, i < 2^twl_shift
    int twl_shift = 0;
};

// One T o H conversion step of a plan.
struct Step {
    int kind = 0;
    double p[4] = {0, 0, 0, 0};
    int64_t n = 0;
    int64_t K = 0;
    int64_t j0 = 0;
    int full = 0;          // Toeplitz part without parity structure (Jacobi): rank-pair packing
    int sign_in = 0;       // (-1)^k on the input (reflection step of a Jacobi chain)
    int sign_out = 0;      // (-1)^k on the output
    int* status = nullptr;  // the plan's device status word (TDH_STATUS_* bits)
    // Case-1 step (Sec. 5.2, 5.3): sp_M > 0 sparse factors instead of T o H
    int sp_M = 0;
    int sp_family = 0;     // SP_ULTRA (offset 2), SP_JACOBI (offset 1), SP_IDENTITY
    int sp_off = 0;        // band offset of the factors
    int sp_inverse = 0;    // apply the factors' inverses (step to a smaller parameter)
    int sp_flip = 0;       // Jacobi: factors conjugated by diag((-1)^k) (reflected frame)
    double sp_par0 = 0;    // parameter of the first factor (l, or a of S_(a,b))
    double sp_dir = 1;     // parameter change from one factor to the next (+1 or -1)
    double sp_b = 0;       // Jacobi: the fixed parameter b
    void* sp_tab = nullptr;  // [M][2 or 3][sp_ld] factor tables in execute precision
    int64_t sp_ld = 0;
    // diagonal scalings folded into this step: the step computes diag(scale_out) A_step
    // diag(scale_in) (float64 device arrays of n entries, owned by the step, may be null)
    double* scale_out = nullptr;
    double* scale_in = nullptr;
    double* t = nullptr;   // [n]
    double* h = nullptr;   // [2n-1]
    double* d1 = nullptr;  // [n]
    double* d2 = nullptr;  // [n]
    double* u64 = nullptr; // [K][n]
    int64_t* piv = nullptr;
    void* d1x = nullptr;   // diagonals in execute precision
    void* d2x = nullptr;
    void* row0 = nullptr;  // CHEB2LEG: row 0 of A in execute precision, else null
    ExecData ex;
    // rank-pair packing (full): the terms of pair p are pair_idx[2p] and pair_idx[2p+1] (sorted
    // by max_k |u_r[k] D2_k|), the second scaled by pair_s[p] on the way in and its output by
    // pair_c[p] = 1 / pair_s[p]^2 (execute precision), so both halves of the packed complex FFT
    // carry comparable magnitudes and neither's rounding swamps the other
    int* pair_idx = nullptr;
    double* pair_s = nullptr;
    void* pair_c = nullptr;
    // ragged batches: one execute configuration per FFT length 2^(8+i), sharing u_nat
    std::vector<ExecData> rcls;
    void* u_nat = nullptr;  // [K][ceil(n/2)] packed factor pairs in execute precision
};

}  // namespace tdh

struct tdh_plan_s {
    int kind = 0;
    int64_t n_max = 0;
    tdh_params params{};
    double tol = 0;
    int device = 0;
    std::vector<tdh::Step> steps;
    int* status = nullptr;  // device: TDH_STATUS_* bits recorded by kernels (tdh_plan_status)
    std::vector<cudaStream_t> side;  // ragged batches: one stream per length class
    std::vector<cudaEvent_t> ev;     // fork/join events (ev[0] fork, ev[1+i] joins)
    // host-buffer execution: copy-in and copy-out streams and their events
    // (hev[0] start, hev[1+s] copied in, hev[3+s] computed, hev[5+s] copied out, slot s < 2)
    cudaStream_t hs[2] = {nullptr, nullptr};
    cudaEvent_t hev[7] = {};
    std::mutex host_mu;
    // serialises the enqueue of ragged calls: their fork/join events are the plan's own, so
    // each call's records and waits must not interleave with another call's
    std::mutex ragged_mu;
};

namespace tdh {
// Case-1 sparse factors: tables of st's factors (scalings folded in), then out = product of
// the factors (or of their inverses) applied to in, or its transpose; in == out allowed.
enum { SP_ULTRA = 0, SP_JACOBI = 1, SP_IDENTITY = 2 };
int sparse_prepare(Step& st, int prec, cudaStream_t s);
int sparse_launch(const Step& st, int prec, const void* in, void* out, int64_t batch, int adjoint,
                  cudaStream_t s);
// P_k^(-1/2,-1/2)(1) = Gamma(k+1/2)/(Gamma(1/2) Gamma(k+1)), k < n (its reciprocal if
// `inverse`), float64 device array: T_k = P_k^(-1/2,-1/2) / P_k^(-1/2,-1/2)(1).
int chebyshev_scale_launch(int64_t n, int inverse, double* out, cudaStream_t s);
// Build the execute configuration of `st` for precision `prec` (spectrum, twiddles, factors).
int exec_prepare(Step& st, int prec, cudaStream_t s);
void exec_release(ExecData& ex);
// Configurations for every FFT length a ragged batch of vectors up to st.n can need.
int exec_prepare_ragged(Step& st, int prec, cudaStream_t s);
// Ragged batch: vector v = in[offs[v] .. offs[v+1]), length <= st.n.
int exec_launch_ragged(const Step& st, int prec, const void* in, void* out, const int64_t* offs,
                       int64_t batch, cudaStream_t s, const std::vector<cudaStream_t>& side,
                       const std::vector<cudaEvent_t>& ev);
// Execute schedules (FFT geometries with a compiled kernel) of the plan's T o H steps.
// Configurations in order: each T o H step's dense configuration, then (ragged plans) one per
// FFT length class.  info = {log2 L, log2 LC, C, R, NT, MINB, index, count}.
int exec_schedules(int prec, int logL, int ragged, int* out, int cap, int* count);
int exec_schedule_count(const tdh_plan_s& plan);
int exec_schedule_info(const tdh_plan_s& plan, int config, int* info);
// Every configuration takes its schedule min(index, count - 1) (tables rebuilt as needed).
int exec_set_schedule(tdh_plan_s& plan, int index, cudaStream_t s);
// Time every schedule of every configuration on synthetic input and keep the fastest.
int exec_autotune(tdh_plan_s& plan, int64_t batch, cudaStream_t s);
// Multi-pass execute of one step (FFT longer than one cluster's shared memory).
int mp_launch(const Step& st, int prec, const void* in, void* out, int64_t batch, int adjoint,
              cudaStream_t s);
// beta = A alpha (adjoint = 0) or A^T g (adjoint = 1) for one step.
int exec_launch(const Step& st, int prec, const void* in, void* out, int64_t batch, int adjoint,
                cudaStream_t s);
}  // namespace tdh
