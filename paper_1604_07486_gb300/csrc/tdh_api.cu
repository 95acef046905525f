// C ABI: plan construction (Fig. 1 steps 1-2), execution (steps 3-5), queries, errors.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "tdh_internal.cuh"

namespace tdh {

namespace {
thread_local char g_err[1024];
std::atomic<int64_t> g_launches{0};
// allocation bookkeeping (tdh_alloc_stats) and the test hook that makes one fail
std::atomic<int64_t> g_allocs{0};         // device allocations made (plan + scratch)
std::atomic<int64_t> g_dev_live{0};       // plan blocks (dev_alloc) not yet freed
std::atomic<int64_t> g_scratch_live{0};   // scratch blocks (scratch_alloc) not yet freed
std::atomic<int64_t> g_fail_countdown{0}; // > 0: the allocation that brings it to 0 fails

// True when the test hook says this allocation is the one to fail.
bool injected_failure() {
    int64_t k = g_fail_countdown.load();
    while (k > 0) {
        if (g_fail_countdown.compare_exchange_weak(k, k - 1)) return k == 1;
    }
    return false;
}
}  // namespace

void note_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

int dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (injected_failure()) {
        set_error("cudaMalloc(%zu bytes): out of memory (failure injected by "
                  "tdh_test_fail_alloc)", bytes);
        return TDH_ERR_NOMEM;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error("cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TDH_ERR_NOMEM : TDH_ERR_CUDA;
    }
    g_allocs.fetch_add(1);
    g_dev_live.fetch_add(1);
    return TDH_OK;
}

void dev_free(void* p) {
    if (!p) return;
    cudaFree(p);
    g_dev_live.fetch_sub(1);
}

// Execute-time scratch comes from one library-owned memory pool per device whose release
// threshold is unlimited: freed blocks stay mapped for the next call instead of returning to
// the driver at every synchronisation (the default pool's behaviour), which would make each
// execute map its scratch again.
int scratch_alloc(void** p, size_t bytes, cudaStream_t s) {
    static std::mutex mu;
    static cudaMemPool_t pools[128] = {};
    *p = nullptr;
    int dev = 0;
    TDH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) {
        set_error("device index %d out of range", dev);
        return TDH_ERR_UNSUPPORTED;
    }
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t created = nullptr;
            TDH_CUDA(cudaMemPoolCreate(&created, &props));
            uint64_t keep = UINT64_MAX;
            TDH_CUDA(cudaMemPoolSetAttribute(created, cudaMemPoolAttrReleaseThreshold, &keep));
            pools[dev] = created;
        }
        pool = pools[dev];
    }
    if (injected_failure()) {
        set_error("scratch allocation of %zu bytes: out of memory (failure injected by "
                  "tdh_test_fail_alloc)", bytes);
        return TDH_ERR_NOMEM;
    }
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error("scratch allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TDH_ERR_NOMEM : TDH_ERR_CUDA;
    }
    g_allocs.fetch_add(1);
    g_scratch_live.fetch_add(1);
    return TDH_OK;
}

void scratch_free(void* p, cudaStream_t s) {
    if (!p) return;
    cudaFreeAsync(p, s);
    g_scratch_live.fetch_sub(1);
}

void alloc_stats(int64_t* out) {
    out[0] = g_allocs.load();
    out[1] = g_dev_live.load();
    out[2] = g_scratch_live.load();
}

void fail_alloc_after(int64_t k) { g_fail_countdown.store(k > 0 ? k : 0); }

namespace {
std::atomic<int> g_tc_stall{0};
}
int tc_stall_enabled() { return g_tc_stall.load(); }
void set_tc_stall(int on) { g_tc_stall.store(on ? 1 : 0); }

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

namespace {

void release_step(Step& st) {
    for (auto& ex : st.rcls) exec_release(ex);
    st.rcls.clear();
    dev_free(st.u_nat);
    dev_free(st.sp_tab);
    dev_free(st.scale_out);
    dev_free(st.scale_in);
    dev_free(st.t);
    dev_free(st.h);
    dev_free(st.d1);
    dev_free(st.d2);
    dev_free(st.u64);
    dev_free(st.piv);
    dev_free(st.d1x);
    dev_free(st.d2x);
    dev_free(st.row0);
    dev_free(st.pair_idx);
    dev_free(st.pair_s);
    dev_free(st.pair_c);
    exec_release(st.ex);
    st = Step{};
}

// Build one conversion step: symbols (a1), pivoted Cholesky (a2), execute tables (a3).
// Relative stop threshold of the Cholesky of an accuracy-targeted plan: run to the rounding
// floor, then keep the prefix the truncation bound asks for.
constexpr double kTargetRelTol = 1e-18;

int build_step(Step& st, double tol, int target, int64_t kmax, int prec, cudaStream_t s) {
    const int64_t n = st.n;
    if (st.sp_M > 0)  // sparse factors: only their tables
        return sparse_prepare(st, prec, s);
    TDH_TRY(dev_alloc_t(&st.t, n));
    TDH_TRY(dev_alloc_t(&st.h, 2 * n - 1));
    TDH_TRY(dev_alloc_t(&st.d1, n));
    TDH_TRY(dev_alloc_t(&st.d2, n));
    TDH_TRY(symbols_launch(st.kind, n, st.p, st.t, st.h, st.d1, st.d2, s));
    // row 0 applied directly, Hankel block on indices >= 1: Chebyshev-to-Legendre (Sec. 5.1)
    // and Jacobi Case 3, a + b <= -1 (Sec. 5.3)
    st.j0 = (st.kind == TDH_CHEB2LEG || (st.kind == TDH_JAC2JAC && !(st.p[0] + st.p[1] > -1.0)))
                ? 1 : 0;
    st.K = 0;
    if (st.j0 < n) {
        int64_t kcap = std::min<int64_t>(kmax, n - st.j0);
        double* ubig = nullptr;
        TDH_TRY(dev_alloc_t(&st.piv, (size_t)kcap));
        TDH_TRY(dev_alloc_t(&ubig, (size_t)kcap * n));
        int64_t K = 0;
        // accuracy-targeted plans pivot on the congruent W H W, w_j = sqrt(|D1_j D2_j|): the
        // same A (D1 W^-1 (T o W H W) W^-1 D2), with the greedy step chasing the residual the
        // output error weighs; the factors are converted back to factors of H (u_r / w)
        double* w = nullptr;
        int rc = TDH_OK;
        if (target) {
            rc = dev_alloc_t(&w, (size_t)n);
            if (rc == TDH_OK)
                rc = pchol_weights(st.d1, st.d2, st.scale_out, st.scale_in, n, w, s);
        }
        if (rc == TDH_OK)
            rc = pchol_run(st.h, w, n, st.j0, target ? kTargetRelTol : tol, kcap, ubig, st.piv,
                           &K, s);
        if (rc == TDH_OK && target && K > 0)
            rc = pchol_truncate(st.h, w, ubig, n, st.j0, K, st.t, st.d1, st.d2, st.scale_out,
                                st.scale_in, tol, &K, nullptr, s);
        if (rc == TDH_OK && target && K > 0) rc = pchol_unweight(ubig, w, K, n, s);
        if (w) {
            cudaStreamSynchronize(s);
            dev_free(w);
        }
        if (rc == TDH_OK && K > 0) {
            rc = dev_alloc_t(&st.u64, (size_t)K * n);
            if (rc == TDH_OK) {
                cudaError_t e = cudaMemcpyAsync(st.u64, ubig, sizeof(double) * K * n,
                                                cudaMemcpyDeviceToDevice, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) {
                    set_error("factor copy: %s", cudaGetErrorString(e));
                    rc = TDH_ERR_CUDA;
                }
            }
        }
        dev_free(ubig);
        TDH_TRY(rc);
        st.K = K;
    }
    return exec_prepare(st, prec, s);
}

void destroy_plan_streams(tdh_plan_s* plan) {
    for (auto ss : plan->side) cudaStreamDestroy(ss);
    for (auto ev : plan->ev) cudaEventDestroy(ev);
    for (auto ss : plan->hs)
        if (ss) cudaStreamDestroy(ss);
    for (auto ev : plan->hev)
        if (ev) cudaEventDestroy(ev);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool overlaps(const void* a, const void* b, size_t bytes) {
    auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + bytes && y < x + bytes;
}

int run(tdh_plan_t plan, const void* in, void* out, int64_t batch, void* stream, int adjoint) {
    clear_error();
    if (!plan) {
        set_error("NULL plan");
        return TDH_ERR_INVALID_ARG;
    }
    if (batch < 0) {
        set_error("batch must be >= 0");
        return TDH_ERR_INVALID_ARG;
    }
    if (batch == 0) return TDH_OK;
    if (!in || !out) {
        set_error("NULL in/out");
        return TDH_ERR_INVALID_ARG;
    }
    if (!aligned16(in) || !aligned16(out)) {
        set_error("in/out must be 16-byte aligned");
        return TDH_ERR_ALIGN;
    }
    const size_t esz = plan->params.prec == TDH_FP64 ? 8 : 4;
    const size_t bytes = (size_t)batch * (size_t)plan->n_max * esz;
    if (overlaps(in, out, bytes)) {
        set_error("out overlaps in");
        return TDH_ERR_ALIAS;
    }
    cudaStream_t s = as_stream(stream);
    const size_t nsteps = plan->steps.size();
    if (nsteps == 0) {  // identity conversion (same basis)
        TDH_CUDA(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s));
        return TDH_OK;
    }
    // A = A_m ... A_1: the first step reads `in`, later steps work in place on `out` (each
    // cluster reads its whole vector before writing it; sparse factors save their tiles'
    // halos first); A^T runs the steps in reverse.
    for (size_t i = 0; i < nsteps; ++i) {
        const Step& st = plan->steps[adjoint ? nsteps - 1 - i : i];
        const void* src = i == 0 ? in : out;
        if (st.sp_M > 0)
            TDH_TRY(sparse_launch(st, plan->params.prec, src, out, batch, adjoint, s));
        else
            TDH_TRY(exec_launch(st, plan->params.prec, src, out, batch, adjoint, s));
    }
    return TDH_OK;
}

// Host buffers: the batch goes through the device in chunks, two device slots each way, so
// the copy of chunk i+1 in, the conversion of chunk i and the copy of chunk i-1 out overlap
// (copy-in stream, the caller's stream, copy-out stream).  Chunks hold at least 8 MB or a
// quarter of the batch, whichever is larger.
int run_host(tdh_plan_t plan, const void* h_in, void* h_out, int64_t batch, void* stream,
             int adjoint) {
    clear_error();
    if (!plan) {
        set_error("NULL plan");
        return TDH_ERR_INVALID_ARG;
    }
    if (batch < 0) {
        set_error("batch must be >= 0");
        return TDH_ERR_INVALID_ARG;
    }
    if (batch == 0) return TDH_OK;
    if (!h_in || !h_out) {
        set_error("NULL in/out");
        return TDH_ERR_INVALID_ARG;
    }
    const size_t esz = plan->params.prec == TDH_FP64 ? 8 : 4;
    const size_t vec_bytes = esz * (size_t)plan->n_max;
    if (overlaps(h_in, h_out, vec_bytes * (size_t)batch)) {
        set_error("out overlaps in");
        return TDH_ERR_ALIAS;
    }
    int64_t chunk = std::max<int64_t>((int64_t)((8u << 20) / vec_bytes), (batch + 3) / 4);
    chunk = std::max<int64_t>(1, std::min(chunk, batch));
    // Chunk sizes.  Each chunk's conversion has a fixed cost (a launch, its prologue and tail),
    // so chunks stay few; from three chunks' worth of vectors on, the first and the last are a
    // quarter chunk (a short copy in before the first conversion, a short copy out after the
    // last) around two equal middle chunks of up to two chunks each.
    std::vector<int64_t> sizes;
    if (batch >= 3 * chunk) {
        const int64_t e = std::max<int64_t>(1, chunk / 4), rem = batch - 2 * e;
        const int64_t nmid = (rem + 2 * chunk - 1) / (2 * chunk);
        sizes.push_back(e);
        for (int64_t j = 0; j < nmid; ++j) sizes.push_back(rem * (j + 1) / nmid - rem * j / nmid);
        sizes.push_back(e);
    } else {
        for (int64_t rem = batch; rem > 0; rem -= std::min(chunk, rem))
            sizes.push_back(std::min(chunk, rem));
    }
    const int64_t slot_vecs = *std::max_element(sizes.begin(), sizes.end());
    const int64_t nchunks = (int64_t)sizes.size();
    const int nslots = nchunks > 1 ? 2 : 1;
    const size_t slot_bytes = (vec_bytes * (size_t)slot_vecs + 255) / 256 * 256;  // aligned
    std::lock_guard<std::mutex> lock(plan->host_mu);
    cudaStream_t s = as_stream(stream);
    cudaStream_t cin = plan->hs[0], cout = plan->hs[1];
    cudaEvent_t* hev = plan->hev;
    char* dev = nullptr;  // [slot][in, out]
    TDH_TRY(scratch_alloc(reinterpret_cast<void**>(&dev), 2 * slot_bytes * nslots, s));
    auto din = [&](int64_t i) { return dev + 2 * slot_bytes * (i % nslots); };
    auto dout = [&](int64_t i) { return din(i) + slot_bytes; };
    const char* hi = static_cast<const char*>(h_in);
    char* ho = static_cast<char*>(h_out);
    int rc = TDH_OK;
    cudaError_t e = cudaEventRecord(hev[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cin, hev[0], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cout, hev[0], 0);
    int64_t first = 0;  // index of the chunk's first vector
    for (int64_t i = 0; e == cudaSuccess && rc == TDH_OK && i < nchunks; first += sizes[i++]) {
        const int sl = (int)(i % nslots);
        const int64_t nb = sizes[i];
        const size_t bytes = vec_bytes * (size_t)nb;
        // copy in once the conversion of the chunk that last used this slot has read it
        if (i >= nslots) e = cudaStreamWaitEvent(cin, hev[3 + sl], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(din(i), hi + vec_bytes * (size_t)first, bytes,
                                cudaMemcpyHostToDevice, cin);
        if (e == cudaSuccess) e = cudaEventRecord(hev[1 + sl], cin);
        // convert once the chunk is in and the slot's previous result has been copied out
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, hev[1 + sl], 0);
        if (e == cudaSuccess && i >= nslots) e = cudaStreamWaitEvent(s, hev[5 + sl], 0);
        if (e != cudaSuccess) break;
        rc = run(plan, din(i), dout(i), nb, s, adjoint);
        if (rc != TDH_OK) break;
        e = cudaEventRecord(hev[3 + sl], s);
        // copy out once converted
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cout, hev[3 + sl], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ho + vec_bytes * (size_t)first, dout(i), bytes,
                                cudaMemcpyDeviceToHost, cout);
        if (e == cudaSuccess) e = cudaEventRecord(hev[5 + sl], cout);
    }
    // join: the caller's stream waits for the last copy out; the slots are freed after it
    cudaError_t ej = cudaEventRecord(hev[0], cout);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s, hev[0], 0);
    scratch_free(dev, s);
    if (rc != TDH_OK) return rc;
    if (e == cudaSuccess) e = ej;
    if (e != cudaSuccess) {
        set_error("host-buffer execute: %s", cudaGetErrorString(e));
        return TDH_ERR_CUDA;
    }
    return TDH_OK;
}

// Parameters are usually given in decimal: differences within 1e-14 (relative) of an integer
// count as integers (Case 1), so e.g. 0.1 -> 1.1 takes one sparse factor.
bool near_integer(double x) {
    return std::fabs(x - std::round(x)) <= 1e-14 * std::max(1.0, std::fabs(x));
}

// Whole steps x -> x +- M with sparse factors, at most kMaxSparse factors per step; returns
// the parameter reached.
constexpr int kMaxSparse = 16;
double sparse_steps(std::vector<Step>& steps, int kind, int64_t n, int family, double x, int M,
                    int up, double b, int flip) {
    while (M > 0) {
        const int m = std::min(M, kMaxSparse);
        Step st;
        st.kind = kind;
        st.n = n;
        st.sp_M = m;
        st.sp_family = family;
        st.sp_off = family == SP_ULTRA ? 2 : 1;
        st.sp_b = b;
        st.sp_flip = flip;
        st.sp_inverse = up ? 0 : 1;
        // up: S_x, S_{x+1}, ...; down: inverses of S_{x-1}, S_{x-2}, ...
        st.sp_par0 = up ? x : x - 1.0;
        st.sp_dir = up ? 1.0 : -1.0;
        steps.push_back(st);
        x += up ? m : -m;
        M -= m;
    }
    return x;
}

// Whole steps while |y - x| >= 1 (Case 1, or the reduction of Case 3 / Case 4), returning the
// parameter reached; *rest is set when a fractional difference is left for a T o H step.
double whole_steps(std::vector<Step>& steps, int kind, int64_t n, int family, double x, double y,
                   double b, int flip, bool* rest) {
    const double d = y - x;
    const bool integer = near_integer(d);
    const int M = integer ? (int)std::lround(std::fabs(d)) : (int)std::floor(std::fabs(d));
    *rest = !integer;
    return sparse_steps(steps, kind, n, family, x, M, d > 0, b, flip);
}

// Whole steps and fractional rest of one parameter's change x -> y.
struct ParamPath {
    int M;         // whole steps (Case 1 / Case 4)
    bool integer;  // no fractional rest (Case 1)
    bool up;
};

ParamPath param_path(double x, double y) {
    const double d = y - x;
    ParamPath p;
    p.integer = near_integer(d);
    p.M = p.integer ? (int)std::lround(std::fabs(d)) : (int)std::floor(std::fabs(d));
    p.up = d > 0;
    return p;
}

// One Case 2 / Case 3 step x -> y of the first Jacobi parameter at fixed second parameter o
// (reflected: in the frame P_k^(a,b)(x) = (-1)^k P_k^(b,a)(-x), i.e. conjugated by
// diag((-1)^k)).
void jacobi_toh(std::vector<Step>& steps, int64_t n, double x, double y, double o, int reflected) {
    Step st;
    st.kind = TDH_JAC2JAC;
    st.n = n;
    st.full = 1;
    st.sign_in = st.sign_out = reflected;
    st.p[0] = x;
    st.p[1] = o;
    st.p[2] = y;
    steps.push_back(st);
}

// Jacobi (a, b) -> (g, d), Sec. 5.3: a changes at fixed b directly, b at fixed a through the
// reflection.  Each change splits into whole steps with the bidiagonal factors (Case 1 /
// Case 4; their inverses, by back-substitution, when lowering) and one Toeplitz-dot-Hankel
// step for a fractional rest (Case 2, or Case 3 when its source parameters sum to <= -1).
// All conversion matrices compose, so the chain is free to choose the order, and it picks
// the one with the least error: every downward whole step first, then the T o H steps at
// the lower end of each range, then every upward whole step.  The paper raises the parameter
// before the T o H step; at the higher end D1 grows like j^(g+1) and D2 like k^(-a), which
// amplifies the Hankel factorisation's rounding (measured at n = 5001, (0.25, 0) ->
// (1.75, 0): 2e-13 relative in the paper's order, 5e-16 in this one), and downward whole
// steps after a T o H step would sum its rounding errors over the whole tail (measured 1e-2
// in float32 for Jacobi (1.5, 0.25) -> (-1/2, -1/2)).
void jacobi_chain(std::vector<Step>& steps, int64_t n, double a, double b, double g, double d) {
    const ParamPath pa = param_path(a, g), pb = param_path(b, d);
    // downward whole steps
    if (!pa.up && pa.M > 0) {
        a = sparse_steps(steps, TDH_JAC2JAC, n, SP_JACOBI, a, pa.M, 0, b, 0);
        if (pa.integer) a = g;
    }
    if (!pb.up && pb.M > 0) {
        b = sparse_steps(steps, TDH_JAC2JAC, n, SP_JACOBI, b, pb.M, 0, a, 1);
        if (pb.integer) b = d;
    }
    // fractional rests
    if (!pb.integer) {
        const double to = pb.up ? d - pb.M : d;
        jacobi_toh(steps, n, b, to, a, 1);
        b = to;
    }
    if (!pa.integer) {
        const double to = pa.up ? g - pa.M : g;
        jacobi_toh(steps, n, a, to, b, 0);
        a = to;
    }
    // upward whole steps
    if (pb.up && pb.M > 0) sparse_steps(steps, TDH_JAC2JAC, n, SP_JACOBI, b, pb.M, 1, a, 1);
    b = d;
    if (pa.up && pa.M > 0) sparse_steps(steps, TDH_JAC2JAC, n, SP_JACOBI, a, pa.M, 1, b, 0);
}

}  // namespace
}  // namespace tdh

using namespace tdh;

extern "C" {

const char* tdh_last_error(void) { return g_err; }

int tdh_launch_count(int64_t* count) {
    clear_error();
    if (!count) {
        set_error("NULL count");
        return TDH_ERR_INVALID_ARG;
    }
    *count = g_launches.load(std::memory_order_relaxed);
    return TDH_OK;
}

int tdh_alloc_stats(int64_t* stats) {
    tdh::clear_error();
    if (!stats) {
        tdh::set_error("tdh_alloc_stats: NULL stats");
        return TDH_ERR_INVALID_ARG;
    }
    tdh::alloc_stats(stats);
    return TDH_OK;
}

int tdh_test_tc_stall(int on) {
    tdh::clear_error();
    tdh::set_tc_stall(on);
    return TDH_OK;
}

int tdh_test_fail_alloc(int64_t k) {
    tdh::clear_error();
    if (k < 0) {
        tdh::set_error("tdh_test_fail_alloc: k must be >= 0");
        return TDH_ERR_INVALID_ARG;
    }
    tdh::fail_alloc_after(k);
    return TDH_OK;
}

int tdh_plan_create(int kind, int64_t n_max, const tdh_params* params, double tol,
                    tdh_plan_t* out) {
    clear_error();
    if (!out || !params) {
        set_error("NULL params/out");
        return TDH_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (kind < TDH_LEG2CHEB || kind > TDH_CHEB2JAC) {
        set_error("unknown kind %d", kind);
        return TDH_ERR_INVALID_ARG;
    }
    if (n_max < 1 || !(tol > 0.0) || !std::isfinite(tol)) {
        set_error("need n_max >= 1 and finite tol > 0");
        return TDH_ERR_INVALID_ARG;
    }
    if (params->prec != TDH_FP32 && params->prec != TDH_FP64 && params->prec != TDH_BF16X3) {
        set_error("unknown precision %d", params->prec);
        return TDH_ERR_INVALID_ARG;
    }
    if (params->kmax < 0) {
        set_error("kmax must be >= 0");
        return TDH_ERR_INVALID_ARG;
    }
    const double* p = params->p;
    const int njac = kind == TDH_JAC2JAC ? 4 : (kind == TDH_JAC2CHEB || kind == TDH_CHEB2JAC) ? 2 : 0;
    for (int i = 0; i < njac; ++i) {
        if (!(p[i] > -1.0) || !std::isfinite(p[i])) {
            set_error("Jacobi parameters must be finite and > -1");
            return TDH_ERR_INVALID_ARG;
        }
    }
    if (kind == TDH_ULTRA2ULTRA && (!(p[0] > 0.0) || !(p[1] > 0.0) || !std::isfinite(p[0]) ||
                                    !std::isfinite(p[1]))) {
        set_error("ultraspherical parameters must be finite and > 0");
        return TDH_ERR_INVALID_ARG;
    }
    if (kind == TDH_LAG2LAG && (!(p[0] > -1.0) || !(p[1] > -1.0))) {
        set_error("Laguerre parameters must be > -1");
        return TDH_ERR_INVALID_ARG;
    }
    if ((kind == TDH_ULTRA2ULTRA && std::fabs(p[1] - p[0]) > 4096.0) ||
        (kind == TDH_JAC2JAC && (std::fabs(p[2] - p[0]) > 4096.0 || std::fabs(p[3] - p[1]) > 4096.0)) ||
        ((kind == TDH_JAC2CHEB || kind == TDH_CHEB2JAC) && (p[0] > 4096.0 || p[1] > 4096.0))) {
        set_error("parameter differences above 4096 are not supported");
        return TDH_ERR_UNSUPPORTED;
    }
    tdh_plan_s* plan = new (std::nothrow) tdh_plan_s;
    if (!plan) {
        set_error("host allocation failed");
        return TDH_ERR_NOMEM;
    }
    plan->kind = kind;
    plan->n_max = n_max;
    plan->params = *params;
    plan->tol = tol;
    cudaGetDevice(&plan->device);
    const int64_t kmax = params->kmax > 0 ? params->kmax : 128;
    cudaStream_t s = nullptr;
    int rc = TDH_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        set_error("cudaStreamCreate: %s", cudaGetErrorString(e));
        delete plan;
        return TDH_ERR_CUDA;
    }
    std::vector<Step>& steps = plan->steps;
    if (kind == TDH_JAC2JAC) {
        // Sec. 5.3: Cases 1-4, with the reflection when b != d
        jacobi_chain(steps, n_max, p[0], p[1], p[2], p[3]);
    } else if (kind == TDH_JAC2CHEB || kind == TDH_CHEB2JAC) {
        // T_k = P_k^(-1/2,-1/2) / P_k^(-1/2,-1/2)(1) (Sec. 5.3, end): a Jacobi conversion to or
        // from (-1/2, -1/2) with the normalisation folded into its last or first step
        const bool to_cheb = kind == TDH_JAC2CHEB;
        if (to_cheb)
            jacobi_chain(steps, n_max, p[0], p[1], -0.5, -0.5);
        else
            jacobi_chain(steps, n_max, -0.5, -0.5, p[0], p[1]);
        if (steps.empty()) {  // (a, b) = (-1/2, -1/2): the normalisation alone
            Step st;
            st.kind = TDH_JAC2JAC;
            st.n = n_max;
            st.sp_M = 1;
            st.sp_family = SP_IDENTITY;
            st.sp_off = 1;
            steps.push_back(st);
        }
        Step& target = to_cheb ? steps.back() : steps.front();
        double** slot = to_cheb ? &target.scale_out : &target.scale_in;
        rc = dev_alloc_t(slot, (size_t)n_max);
        if (rc == TDH_OK) rc = chebyshev_scale_launch(n_max, to_cheb ? 0 : 1, *slot, s);
    } else if (kind == TDH_ULTRA2ULTRA) {
        // Sec. 5.2: Case 1 (integer difference): sparse factors only; Case 3 (difference above
        // one, not an integer): whole steps with the sparse factors, then Case 2 (|l1 - l2| < 1)
        // with the Toeplitz-dot-Hankel product.  Downward steps apply the factors' inverses.
        bool rest = false;
        const double l1 = whole_steps(steps, kind, n_max, SP_ULTRA, p[0], p[1], 0.0, 0, &rest);
        if (rest) {
            Step st;
            st.kind = kind;
            st.n = n_max;
            st.p[0] = l1;
            st.p[1] = p[1];
            steps.push_back(st);
        }
    } else if (kind == TDH_LAG2LAG) {
        // Sec. 5.4: Toeplitz only (H = all ones, rank 1); no parity structure
        if (p[0] != p[1]) {
            Step st;
            st.kind = kind;
            st.n = n_max;
            st.full = 1;
            std::memcpy(st.p, p, sizeof(st.p));
            steps.push_back(st);
        }
    } else {
        Step st;
        st.kind = kind;
        st.n = n_max;
        std::memcpy(st.p, p, sizeof(st.p));
        steps.push_back(st);
    }
    if (rc == TDH_OK) {
        rc = dev_alloc_t(&plan->status, 4);
        if (rc == TDH_OK && cudaMemsetAsync(plan->status, 0, 4 * sizeof(int), s) != cudaSuccess) {
            set_error("status word: cudaMemsetAsync failed");
            rc = TDH_ERR_CUDA;
        }
    }
    for (auto& st : plan->steps) {
        if (rc != TDH_OK) break;
        st.status = plan->status;
        rc = build_step(st, tol, (params->flags & TDH_FLAG_TARGET) ? 1 : 0, kmax, params->prec, s);
        if (rc != TDH_OK) break;
    }
    if (rc == TDH_OK && (params->flags & TDH_FLAG_RAGGED)) {
        if (plan->steps.size() != 1) {
            set_error("ragged batches need a single-step conversion");
            rc = TDH_ERR_UNSUPPORTED;
        } else {
            rc = exec_prepare_ragged(plan->steps[0], params->prec, s);
        }
        const size_t ncls = plan->steps.empty() ? 0 : plan->steps[0].rcls.size();
        for (size_t i = 0; rc == TDH_OK && i < ncls; ++i) {
            cudaStream_t ss = nullptr;
            cudaError_t ee = cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking);
            if (ee == cudaSuccess) plan->side.push_back(ss);
            else rc = TDH_ERR_CUDA;
        }
        for (size_t i = 0; rc == TDH_OK && i < ncls + 1; ++i) {
            cudaEvent_t ev = nullptr;
            cudaError_t ee = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (ee == cudaSuccess) plan->ev.push_back(ev);
            else rc = TDH_ERR_CUDA;
        }
        if (rc == TDH_ERR_CUDA && !tdh_last_error()[0]) set_error("stream/event creation failed");
    }
    for (int i = 0; rc == TDH_OK && i < 2; ++i)
        if (cudaStreamCreateWithFlags(&plan->hs[i], cudaStreamNonBlocking) != cudaSuccess) {
            set_error("stream creation failed");
            rc = TDH_ERR_CUDA;
        }
    for (int i = 0; rc == TDH_OK && i < 7; ++i)
        if (cudaEventCreateWithFlags(&plan->hev[i], cudaEventDisableTiming) != cudaSuccess) {
            set_error("event creation failed");
            rc = TDH_ERR_CUDA;
        }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (rc != TDH_OK) {
        for (auto& x : plan->steps) release_step(x);
        dev_free(plan->status);
        destroy_plan_streams(plan);
        delete plan;
        return rc;
    }
    *out = plan;
    return TDH_OK;
}

int tdh_plan_execute_ragged(tdh_plan_t plan, const void* in, void* out, const int64_t* offsets,
                            int64_t batch, void* stream) {
    clear_error();
    if (!plan) {
        set_error("NULL plan");
        return TDH_ERR_INVALID_ARG;
    }
    if (batch < 0) {
        set_error("batch must be >= 0");
        return TDH_ERR_INVALID_ARG;
    }
    if (batch == 0) return TDH_OK;
    if (!in || !out || !offsets) {
        set_error("NULL in/out/offsets");
        return TDH_ERR_INVALID_ARG;
    }
    if (in == out) {
        set_error("out overlaps in");
        return TDH_ERR_ALIAS;
    }
    if (!(plan->params.flags & TDH_FLAG_RAGGED) || plan->steps.size() != 1 ||
        plan->steps[0].rcls.empty()) {
        set_error("plan was not created with TDH_FLAG_RAGGED");
        return TDH_ERR_INVALID_ARG;
    }
    if (batch > (int64_t)1 << 31) {
        set_error("ragged batch above 2^31 vectors");
        return TDH_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(plan->ragged_mu);
    return exec_launch_ragged(plan->steps[0], plan->params.prec, in, out, offsets, batch,
                              as_stream(stream), plan->side, plan->ev);
}

// Ragged batch in host memory: chunks of whole vectors move through the device like
// run_host's (a sixteenth of the coefficients first and last, the rest in two halves), each
// chunk converted by the device ragged path with offsets relative to its own staging slot.
int tdh_plan_execute_ragged_host(tdh_plan_t plan, const void* h_in, void* h_out,
                                 const int64_t* offsets, int64_t batch, void* stream) {
    clear_error();
    if (!plan) {
        set_error("NULL plan");
        return TDH_ERR_INVALID_ARG;
    }
    if (batch < 0) {
        set_error("batch must be >= 0");
        return TDH_ERR_INVALID_ARG;
    }
    if (batch == 0) return TDH_OK;
    if (!h_in || !h_out || !offsets) {
        set_error("NULL in/out/offsets");
        return TDH_ERR_INVALID_ARG;
    }
    if (!(plan->params.flags & TDH_FLAG_RAGGED) || plan->steps.size() != 1 ||
        plan->steps[0].rcls.empty()) {
        set_error("plan was not created with TDH_FLAG_RAGGED");
        return TDH_ERR_INVALID_ARG;
    }
    if (batch > (int64_t)1 << 31) {
        set_error("ragged batch above 2^31 vectors");
        return TDH_ERR_UNSUPPORTED;
    }
    // the offsets are on the host here, so every length is checked before anything runs
    if (offsets[0] < 0) {
        set_error("offsets[0] < 0");
        return TDH_ERR_INVALID_ARG;
    }
    for (int64_t v = 0; v < batch; ++v) {
        const int64_t len = offsets[v + 1] - offsets[v];
        if (len < 0 || len > plan->n_max) {
            set_error("vector %lld: length %lld outside [0, n_max = %lld]", (long long)v,
                      (long long)len, (long long)plan->n_max);
            return TDH_ERR_INVALID_ARG;
        }
    }
    const int64_t c0 = offsets[0], total = offsets[batch] - offsets[0];
    if (total == 0) return TDH_OK;
    const size_t esz = plan->params.prec == TDH_FP64 ? 8 : 4;
    const char* hi = static_cast<const char*>(h_in) + esz * (size_t)c0;
    char* ho = static_cast<char*>(h_out) + esz * (size_t)c0;
    if (overlaps(hi, ho, esz * (size_t)total)) {
        set_error("out overlaps in");
        return TDH_ERR_ALIAS;
    }
    // chunk boundaries (vector indices) at coefficient targets: 1/16, 1/2, 15/16 of the total
    // from 24 MB on, else one chunk; empty chunks dropped
    std::vector<int64_t> cut{0};
    if (esz * (size_t)total >= ((size_t)24 << 20)) {
        for (const int64_t t : {total / 16, total / 2, total - total / 16}) {
            const int64_t v = std::lower_bound(offsets, offsets + batch + 1, c0 + t) - offsets;
            if (v > cut.back() && v < batch) cut.push_back(v);
        }
    }
    cut.push_back(batch);
    const int64_t nchunks = (int64_t)cut.size() - 1;
    int64_t max_c = 0, max_v = 0;
    for (int64_t i = 0; i < nchunks; ++i) {
        max_c = std::max(max_c, offsets[cut[i + 1]] - offsets[cut[i]]);
        max_v = std::max(max_v, cut[i + 1] - cut[i]);
    }
    // chunk-relative offsets of every chunk, uploaded once before the chunks (the host array
    // may be pageable; an event tells when that copy has read it)
    std::vector<int64_t> rel((size_t)(batch + nchunks));
    std::vector<int64_t> first(nchunks);  // index of each chunk's offsets in rel
    for (int64_t i = 0, k = 0; i < nchunks; ++i) {
        first[i] = k;
        for (int64_t v = cut[i]; v <= cut[i + 1]; ++v) rel[(size_t)k++] = offsets[v] - offsets[cut[i]];
    }
    const int nslots = nchunks > 1 ? 2 : 1;
    const size_t data_bytes = (esz * (size_t)max_c + 255) / 256 * 256;
    const size_t slot_bytes = 2 * data_bytes;  // [in, out]
    std::lock_guard<std::mutex> lock(plan->host_mu);
    std::lock_guard<std::mutex> rlock(plan->ragged_mu);
    cudaStream_t s = as_stream(stream);
    cudaStream_t cin = plan->hs[0], cout = plan->hs[1];
    cudaEvent_t* hev = plan->hev;
    char* dev = nullptr;
    TDH_TRY(scratch_alloc(reinterpret_cast<void**>(&dev),
                          slot_bytes * nslots + sizeof(int64_t) * rel.size(), s));
    auto din = [&](int64_t i) { return dev + slot_bytes * (i % nslots); };
    auto dout = [&](int64_t i) { return din(i) + data_bytes; };
    int64_t* doffs = reinterpret_cast<int64_t*>(dev + slot_bytes * nslots);
    int rc = TDH_OK;
    cudaEvent_t ev_off = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev_off, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(hev[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cin, hev[0], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cout, hev[0], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(doffs, rel.data(), sizeof(int64_t) * rel.size(), cudaMemcpyHostToDevice,
                            cin);
    if (e == cudaSuccess) e = cudaEventRecord(ev_off, cin);
    for (int64_t i = 0; e == cudaSuccess && rc == TDH_OK && i < nchunks; ++i) {
        const int sl = (int)(i % nslots);
        const int64_t v0 = cut[i], nv = cut[i + 1] - v0;
        const size_t off = esz * (size_t)(offsets[v0] - c0);
        const size_t bytes = esz * (size_t)(offsets[cut[i + 1]] - offsets[v0]);
        // copy in once the conversion of the chunk that last used this slot has read it
        if (i >= nslots) e = cudaStreamWaitEvent(cin, hev[3 + sl], 0);
        if (e == cudaSuccess && bytes)
            e = cudaMemcpyAsync(din(i), hi + off, bytes, cudaMemcpyHostToDevice, cin);
        if (e == cudaSuccess) e = cudaEventRecord(hev[1 + sl], cin);
        // convert once the chunk is in and the slot's previous result has been copied out
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, hev[1 + sl], 0);
        if (e == cudaSuccess && i >= nslots) e = cudaStreamWaitEvent(s, hev[5 + sl], 0);
        if (e != cudaSuccess) break;
        rc = exec_launch_ragged(plan->steps[0], plan->params.prec, din(i), dout(i),
                                doffs + first[i], nv, s, plan->side, plan->ev);
        if (rc != TDH_OK) break;
        e = cudaEventRecord(hev[3 + sl], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cout, hev[3 + sl], 0);
        if (e == cudaSuccess && bytes)
            e = cudaMemcpyAsync(ho + off, dout(i), bytes, cudaMemcpyDeviceToHost, cout);
        if (e == cudaSuccess) e = cudaEventRecord(hev[5 + sl], cout);
    }
    // join: the caller's stream waits for the last copy out; the slots are freed after it
    cudaError_t ej = cudaEventRecord(hev[0], cout);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s, hev[0], 0);
    scratch_free(dev, s);
    // `rel` must outlive the copy that reads it (issued first; normally long complete)
    if (ev_off) {
        const cudaError_t es = cudaEventSynchronize(ev_off);
        if (ej == cudaSuccess) ej = es;
        cudaEventDestroy(ev_off);
    }
    if (rc != TDH_OK) return rc;
    if (e == cudaSuccess) e = ej;
    if (e != cudaSuccess) {
        set_error("ragged host-buffer execute: %s", cudaGetErrorString(e));
        return TDH_ERR_CUDA;
    }
    return TDH_OK;
}

int tdh_plan_execute(tdh_plan_t plan, const void* in, void* out, int64_t batch, void* stream) {
    return run(plan, in, out, batch, stream, 0);
}

int tdh_plan_execute_adjoint(tdh_plan_t plan, const void* in, void* out, int64_t batch,
                             void* stream) {
    return run(plan, in, out, batch, stream, 1);
}

int tdh_plan_execute_host(tdh_plan_t plan, const void* in, void* out, int64_t batch, int adjoint,
                          void* stream) {
    return run_host(plan, in, out, batch, stream, adjoint ? 1 : 0);
}

int tdh_plan_query(tdh_plan_t plan, int64_t* K, int64_t* n_max) {
    clear_error();
    if (!plan) {
        set_error("NULL plan");
        return TDH_ERR_INVALID_ARG;
    }
    int64_t kk = 0;
    for (const auto& st : plan->steps) kk = std::max(kk, st.K);
    if (K) *K = kk;
    if (n_max) *n_max = plan->n_max;
    return TDH_OK;
}

int tdh_schedules(int prec, int logL, int ragged, int* out, int cap, int* count) {
    clear_error();
    if ((prec != TDH_FP32 && prec != TDH_FP64 && prec != TDH_BF16X3) || logL < 1 || logL > 62 ||
        cap < 0 || !count ||
        (cap > 0 && !out)) {
        set_error("tdh_schedules: need a known precision, 1 <= logL <= 62, cap >= 0, non-NULL");
        return TDH_ERR_INVALID_ARG;
    }
    return exec_schedules(prec, logL, ragged, out, cap, count);
}

int tdh_plan_schedule_count(tdh_plan_t plan, int* count) {
    clear_error();
    if (!plan || !count) {
        set_error("NULL plan or count");
        return TDH_ERR_INVALID_ARG;
    }
    *count = exec_schedule_count(*plan);
    return TDH_OK;
}

int tdh_plan_schedule_info(tdh_plan_t plan, int config, int* info) {
    clear_error();
    if (!plan || !info) {
        set_error("NULL plan or info");
        return TDH_ERR_INVALID_ARG;
    }
    return exec_schedule_info(*plan, config, info);
}

int tdh_plan_set_schedule(tdh_plan_t plan, int index, void* stream) {
    clear_error();
    if (!plan) {
        set_error("NULL plan");
        return TDH_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(plan->host_mu);
    cudaStream_t s = as_stream(stream);
    const int rc = exec_set_schedule(*plan, index, s);
    TDH_CUDA(cudaStreamSynchronize(s));
    return rc;
}

int tdh_plan_autotune(tdh_plan_t plan, int64_t batch, void* stream) {
    clear_error();
    if (!plan) {
        set_error("NULL plan");
        return TDH_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(plan->host_mu);
    cudaStream_t s = as_stream(stream);
    const int rc = exec_autotune(*plan, batch, s);
    TDH_CUDA(cudaStreamSynchronize(s));
    return rc;
}

int tdh_plan_destroy(tdh_plan_t plan) {
    clear_error();
    if (!plan) return TDH_OK;
    for (auto& st : plan->steps) release_step(st);
    dev_free(plan->status);
    destroy_plan_streams(plan);
    delete plan;
    return TDH_OK;
}

int tdh_plan_status(tdh_plan_t plan, int* status, void* stream) {
    clear_error();
    if (!plan || !status) {
        set_error("tdh_plan_status: NULL plan or status");
        return TDH_ERR_INVALID_ARG;
    }
    cudaStream_t s = as_stream(stream);
    int v = 0;
    TDH_CUDA(cudaMemcpyAsync(&v, plan->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    TDH_CUDA(cudaMemsetAsync(plan->status, 0, sizeof(int), s));
    TDH_CUDA(cudaStreamSynchronize(s));
    *status = v;
    return TDH_OK;
}

}  // extern "C"
