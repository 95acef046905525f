// C ABI: plan construction (Fig. 1 steps 1-2), execution (steps 3-5), queries, errors.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "tdh_internal.cuh"

namespace tdh {

namespace {
thread_local char g_err[1024];
}

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
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error("cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TDH_ERR_NOMEM : TDH_ERR_CUDA;
    }
    return TDH_OK;
}

void dev_free(void* p) {
    if (p) cudaFree(p);
}

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
    dev_free(st.band_coef);
    dev_free(st.t);
    dev_free(st.h);
    dev_free(st.d1);
    dev_free(st.d2);
    dev_free(st.u64);
    dev_free(st.piv);
    dev_free(st.d1x);
    dev_free(st.d2x);
    dev_free(st.row0);
    exec_release(st.ex);
    st = Step{};
}

// Build one conversion step: symbols (a1), pivoted Cholesky (a2), execute tables (a3).
int build_step(Step& st, double tol, int64_t kmax, int prec, cudaStream_t s) {
    const int64_t n = st.n;
    if (st.banded_M > 0)  // sparse factors: only their coefficient table
        return banded_prepare(prec, n, st.banded_lam0, st.banded_M, &st.band_coef, s);
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
        int rc = pchol_run(st.h, n, st.j0, tol, kcap, ubig, st.piv, &K, s);
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
    const size_t esz = plan->params.prec == TDH_FP32 ? 4 : 8;
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
    // cluster reads its whole vector before writing it); A^T runs the steps in reverse.
    for (size_t i = 0; i < nsteps; ++i) {
        const Step& st = plan->steps[adjoint ? nsteps - 1 - i : i];
        if (st.banded_M > 0) {
            // the tiled sparse-factor kernel reads a halo from neighbouring tiles: out of place
            if (i != 0) {
                set_error("this chain's transpose would apply sparse factors in place "
                          "(not built)");
                return TDH_ERR_UNSUPPORTED;
            }
            TDH_TRY(banded_launch(plan->params.prec, in, out, st.n, batch, st.band_coef,
                                  st.banded_M, adjoint, s));
            continue;
        }
        TDH_TRY(exec_launch(st, plan->params.prec, i == 0 ? in : out, out, batch, adjoint, s));
    }
    return TDH_OK;
}

bool case2(double a, double b, double g) {
    // Sec. 5.3 Case 2 (|a - g| < 1, a != g, a + b > -1) or Case 3 (the same with a + b <= -1)
    (void)b;
    return std::fabs(a - g) < 1.0 && a != g;
}

}  // namespace
}  // namespace tdh

using namespace tdh;

extern "C" {

const char* tdh_last_error(void) { return g_err; }

int tdh_plan_create(int kind, int64_t n_max, const tdh_params* params, double tol,
                    tdh_plan_t* out) {
    clear_error();
    if (!out || !params) {
        set_error("NULL params/out");
        return TDH_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (kind < TDH_LEG2CHEB || kind > TDH_LAG2LAG) {
        set_error("unknown kind %d", kind);
        return TDH_ERR_INVALID_ARG;
    }
    if (n_max < 1 || !(tol > 0.0) || !std::isfinite(tol)) {
        set_error("need n_max >= 1 and finite tol > 0");
        return TDH_ERR_INVALID_ARG;
    }
    if (params->prec != TDH_FP32 && params->prec != TDH_FP64) {
        set_error("unknown precision %d", params->prec);
        return TDH_ERR_INVALID_ARG;
    }
    if (params->kmax < 0) {
        set_error("kmax must be >= 0");
        return TDH_ERR_INVALID_ARG;
    }
    if (kind == TDH_JAC2JAC) {
        const double a = params->p[0], b = params->p[1], g = params->p[2], d = params->p[3];
        if (!(a > -1.0) || !(b > -1.0) || !(g > -1.0) || !(d > -1.0)) {
            set_error("Jacobi parameters must be > -1");
            return TDH_ERR_INVALID_ARG;
        }
        if ((b != d && !case2(b, a, d)) || (a != g && !case2(a, d, g))) {
            set_error("Jacobi conversion is built for chains of Case-2/3 steps "
                      "(|b-d| < 1 and |a-g| < 1); Case 4 (integer shifts) is not built");
            return TDH_ERR_UNSUPPORTED;
        }
    }
    if (kind == TDH_ULTRA2ULTRA) {
        double l1 = params->p[0], l2 = params->p[1];
        if (!(l1 > 0.0) || !(l2 > 0.0)) {
            set_error("ultraspherical parameters must be > 0");
            return TDH_ERR_INVALID_ARG;
        }
        if (l1 - l2 >= 1.0) {
            set_error("ultraspherical conversion to a smaller parameter by 1 or more needs "
                      "back-substitution (not built)");
            return TDH_ERR_UNSUPPORTED;
        }
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
    if (kind == TDH_JAC2JAC) {
        // Sec. 5.3: with b != d, reflect (P_k^(a,b)(x) = (-1)^k P_k^(b,a)(-x)), convert the
        // first parameter b -> d, reflect back; then convert a -> g at fixed d.
        const double a = params->p[0], b = params->p[1], g = params->p[2], d = params->p[3];
        if (b != d) {
            Step st;
            st.kind = kind;
            st.n = n_max;
            st.full = 1;
            st.sign_in = st.sign_out = 1;
            st.p[0] = b;
            st.p[1] = a;
            st.p[2] = d;
            plan->steps.push_back(st);
        }
        if (a != g) {
            Step st;
            st.kind = kind;
            st.n = n_max;
            st.full = 1;
            st.p[0] = a;
            st.p[1] = d;
            st.p[2] = g;
            plan->steps.push_back(st);
        }
    } else if (kind == TDH_ULTRA2ULTRA) {
        // Sec. 5.2: Case 1 (l2 - l1 a positive integer): sparse factors only; Case 3
        // (l2 - l1 > 1, not an integer): raise l1 by whole steps with the sparse factors,
        // then Case 2 (|l1 - l2| < 1) with the Toeplitz-dot-Hankel product.
        double l1 = params->p[0], l2 = params->p[1];
        const double up = std::floor(l2 - l1);
        if (up >= 1.0) {
            Step st;
            st.kind = kind;
            st.n = n_max;
            st.banded_M = (int)up;
            st.banded_lam0 = l1;
            plan->steps.push_back(st);
            l1 += up;
        }
        if (l1 != l2) {
            Step st;
            st.kind = kind;
            st.n = n_max;
            st.p[0] = l1;
            st.p[1] = l2;
            plan->steps.push_back(st);
        }
    } else if (kind == TDH_LAG2LAG) {
        // Sec. 5.4: Toeplitz only (H = all ones, rank 1); no parity structure
        if (!(params->p[0] > -1.0) || !(params->p[1] > -1.0)) {
            rc = TDH_ERR_INVALID_ARG;
            set_error("Laguerre parameters must be > -1");
        } else if (params->p[0] != params->p[1]) {
            Step st;
            st.kind = kind;
            st.n = n_max;
            st.full = 1;
            std::memcpy(st.p, params->p, sizeof(st.p));
            plan->steps.push_back(st);
        }
    } else {
        Step st;
        st.kind = kind;
        st.n = n_max;
        std::memcpy(st.p, params->p, sizeof(st.p));
        plan->steps.push_back(st);
    }
    for (auto& st : plan->steps) {
        if (rc != TDH_OK) break;
        rc = build_step(st, tol, kmax, params->prec, s);
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
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (rc != TDH_OK) {
        for (auto& x : plan->steps) release_step(x);
        for (auto ss : plan->side) cudaStreamDestroy(ss);
        for (auto ev : plan->ev) cudaEventDestroy(ev);
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
    if (!(plan->params.flags & TDH_FLAG_RAGGED) || plan->steps.size() != 1 ||
        plan->steps[0].rcls.empty()) {
        set_error("plan was not created with TDH_FLAG_RAGGED");
        return TDH_ERR_INVALID_ARG;
    }
    if (batch > (int64_t)1 << 31) {
        set_error("ragged batch above 2^31 vectors");
        return TDH_ERR_UNSUPPORTED;
    }
    return exec_launch_ragged(plan->steps[0], plan->params.prec, in, out, offsets, batch,
                              as_stream(stream), plan->side, plan->ev);
}

int tdh_plan_execute(tdh_plan_t plan, const void* in, void* out, int64_t batch, void* stream) {
    return run(plan, in, out, batch, stream, 0);
}

int tdh_plan_execute_adjoint(tdh_plan_t plan, const void* in, void* out, int64_t batch,
                             void* stream) {
    return run(plan, in, out, batch, stream, 1);
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

int tdh_plan_destroy(tdh_plan_t plan) {
    clear_error();
    if (!plan) return TDH_OK;
    for (auto& st : plan->steps) release_step(st);
    for (auto ss : plan->side) cudaStreamDestroy(ss);
    for (auto ev : plan->ev) cudaEventDestroy(ev);
    delete plan;
    return TDH_OK;
}

}  // extern "C"
