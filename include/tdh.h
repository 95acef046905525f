/*
 * tdh.h -- C ABI of the GB300 Toeplitz-dot-Hankel polynomial basis conversion library.
 *
 * Method: Townsend, Webb & Olver, "Fast polynomial transforms based on Toeplitz and Hankel
 * matrices" (arXiv:1604.07486).  A conversion matrix is split as A = D1 (T o H) D2 (Fig. 1
 * step 1, Eq. (3)); the Hankel part H is compressed by pivoted Cholesky,
 * H ~ sum_r l_r l_r^T / a_r (Sec. 2.1, Fig. 2); and beta = A alpha is computed as
 * D1 sum_r D_{u_r} T D_{u_r} D2 alpha with u_r = l_r / sqrt(a_r) (Eq. (5)),
 * each Toeplitz product by zero-padded FFTs of length about 2N (Sec. 1).
 *
 * Conventions for every entry point
 *   - Pointers named d_* or documented as "device" are CUDA device pointers on the current
 *     device; pointers documented as "host" are ordinary host memory.  The library never
 *     takes ownership of caller memory.
 *   - Vectors are dense, row-major: vector b of a batch occupies in[b * n .. b * n + n).
 *     Element k is the coefficient of the degree-k basis polynomial.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Work is
 *     enqueued asynchronously on it unless stated otherwise.
 *   - Every function returns TDH_OK (0) or a negative TDH_ERR_* code; on error a message is
 *     available from tdh_last_error() (thread-local) and no output is written unless stated.
 *   - The library is single-GPU: a plan belongs to the device that was current at creation
 *     and must be used with that device current.
 *   - Scratch: execute calls take temporary device memory stream-ordered from one memory
 *     pool per device owned by the library (cudaMallocFromPoolAsync), whose freed blocks stay
 *     mapped for later calls (release threshold unlimited).  The first execute on a device
 *     creates the pool, so make it outside stream capture.
 */
#ifndef TDH_H
#define TDH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- kinds (basis pairs) */
#define TDH_LEG2CHEB    0 /* Legendre -> Chebyshev, Eq. (2), split Eq. (7)       */
#define TDH_CHEB2LEG    1 /* Chebyshev -> Legendre, Eq. (11), split Sec. 5.1           */
#define TDH_ULTRA2ULTRA 2 /* ultraspherical C^(l1) -> C^(l2), Sec. 5.2, p = {l1, l2}          */
#define TDH_JAC2JAC     3 /* Jacobi P^(a,b) -> P^(g,d), Sec. 5.3, p = {a, b, g, d}           */
#define TDH_LAG2LAG     4 /* generalised Laguerre L^(a1) -> L^(a2), Sec. 5.4, p = {a1, a2}   */
#define TDH_JAC2CHEB    5 /* Jacobi P^(a,b) -> Chebyshev T, Sec. 5.3 (end), p = {a, b}      */
#define TDH_CHEB2JAC    6 /* Chebyshev T -> Jacobi P^(a,b), Sec. 5.3 (end), p = {a, b}      */

/* ---------------------------------------------------------------- execute precisions */
#define TDH_FP64  0 /* float64 in/out, float64 FFT                                             */
#define TDH_FP32  1 /* float32 in/out, float32 FFT (plan factors rounded once from float64)    */
/* float32 in/out; within one thread-block cluster (FFTs of up to 2^17 points) the radix-16
 * (radix-8 for short FFTs) middle passes of every FFT run on the tensor cores as DFT matrix
 * products in split bfloat16: each operand x = hi + lo (bfloat16 parts) and the three products
 * hi*hi + lo*hi + hi*lo accumulate in float32 (tcgen05, tensor memory); every other pass and
 * the multi-pass FFTs beyond one cluster are float32.  The split keeps about 16 bits of each
 * operand, so errors are larger than TDH_FP32's.                                              */
#define TDH_BF16X3 2

/* ---------------------------------------------------------------- plan flags */
#define TDH_FLAG_NONE   0
#define TDH_FLAG_RAGGED 1 /* also prepare every shorter FFT length (tdh_plan_execute_ragged)  */
#define TDH_FLAG_TARGET 2 /* tol is the target accuracy of the truncation (tdh_plan_create)   */

/* ---------------------------------------------------------------- error codes */
#define TDH_OK               0
#define TDH_ERR_INVALID_ARG (-1) /* bad kind, n < 1, parameter out of range, tol <= 0, NULL  */
#define TDH_ERR_UNSUPPORTED (-2) /* valid request the library does not implement          */
#define TDH_ERR_NOMEM       (-3) /* device or host allocation failed                       */
#define TDH_ERR_ALIGN       (-4) /* pointer not aligned to 16 bytes                         */
#define TDH_ERR_TIMEOUT     (-5) /* reserved (device-side waits report through tdh_plan_status) */
#define TDH_ERR_CUDA        (-6) /* a CUDA runtime call failed (message has the detail)     */
#define TDH_ERR_ALIAS       (-7) /* out overlaps in where the operation forbids it          */

/* ---------------------------------------------------------------- device status bits */
#define TDH_STATUS_TIMEOUT 1 /* a tensor-core pass's bounded wait for its products ran out  */
#define TDH_STATUS_LENGTH  2 /* a ragged vector was longer than n_max (or offsets decreased) */
#define TDH_STATUS_ALIAS   4 /* a ragged call's out range overlapped its in range          */
#define TDH_STATUS_FAULT   8 /* a kernel skipped a bulk copy whose alignment it found wrong  */

/* opaque; after creation only tdh_plan_set_schedule and tdh_plan_autotune change it */
typedef struct tdh_plan_s* tdh_plan_t;

typedef struct {
    double p[4];  /* kind parameters: ULTRA {l1, l2}; JAC {a, b, g, d}; LAG {a1, a2};
                     JAC2CHEB / CHEB2JAC {a, b}                                              */
    int prec;     /* TDH_FP64, TDH_FP32 or TDH_BF16X3: execute in/out type, FFT arithmetic  */
    int flags;    /* TDH_FLAG_NONE, or TDH_FLAG_RAGGED and/or TDH_FLAG_TARGET (bitwise or)    */
    int64_t kmax; /* cap on the rank of each Hankel factorisation; 0 selects 128            */
} tdh_params;

/*
 * tdh_plan_create -- build everything beta = A alpha needs for vectors of n_max coefficients
 * (degree n_max - 1), on the current device, in float64 (Fig. 1 steps 1-2):
 *   a1  the split's generator sequences t, h and diagonals D1, D2 from their closed forms
 *       (Gamma ratios by an asymptotic series at large argument, Tricomi-Erdelyi);
 *   a2  pivoted Cholesky of H (Sec. 2.1, Fig. 2), stopping before the first pivot a_r with
 *       a_r <= tol * max(diag H) (a negligible pivot ends it, Sec. 2.1), at most kmax steps;
 *   a3  the spectrum of the Toeplitz symbol for each FFT length in use.
 * For TDH_CHEB2LEG the factorisation covers indices 1..n_max-1 and row 0 is applied directly
 * (Sec. 5.1).  tol > 0 is relative to the largest diagonal entry of H; Sec. 2.1 sets it
 * near the unit roundoff of the arithmetic used.
 * With TDH_FLAG_TARGET, tol is instead the accuracy asked of each T o H step's truncation:
 * the factorisation pivots on the congruent W H W, w_j = sqrt(|D1_j D2_j|) (1 where zero;
 * the same A = D1 W^-1 (T o W H W) W^-1 D2, so the greedy pivot chases the residual that the
 * output error weighs; its factors are returned divided by w), runs to its rounding floor
 * (relative threshold 1e-18, at most kmax steps), and the step keeps the fewest K' terms with
 *   B(K') = max_m |t_m| * max_j |D1_j| sqrt(d_j) * max_k |D2_k| sqrt(d_k) <= tol,
 * d the diagonal of the residual R = H - sum_{r<K'} u_r u_r^T (indices of the Hankel block;
 * D1, D2 including the step's Chebyshev scalings).  R is positive semidefinite (a Schur
 * complement), so |R_jk| <= sqrt(d_j d_k), every entry of A - A_K' is at most B(K') and
 * max |beta_K' - beta| <= B(K') ||alpha||_1 in exact arithmetic; the execute precision's
 * rounding comes on top.  If no prefix meets tol, every computed term is kept.
 * Case dispatch (a plan is a chain of steps applied in order):
 *   ULTRA (l1, l2 > 0): integer l2 - l1 (Case 1): sparse factors S_l of
 *     Eq. (12), or their inverses by back-substitution when l2 < l1;
 *     |l2 - l1| > 1 not an integer (Case 3): whole steps with those factors until the
 *     difference is below one, then Case 2 (T o H).  Differences within 1e-14 (relative) of
 *     an integer count as integers.
 *   JAC (a, b, g, d > -1): a -> g at fixed b directly, b -> d at fixed a in the reflected
 *     frame P_k^(a,b)(x) = (-1)^k P_k^(b,a)(-x).  Each change takes Case 1 / 4 whole steps
 *     with the bidiagonal factors S_(a,b) (their inverses when lowering) and one Case 2
 *     (T o H) step for a fractional rest, or Case 3 (row 0 direct) when that step's source
 *     parameters sum to <= -1.  Order: every downward whole step first, then the T o H steps
 *     at the lower end of each range (where the diagonal scalings amplify the Hankel
 *     factorisation's rounding least), then every upward whole step.
 *   JAC2CHEB / CHEB2JAC: the Jacobi chain to / from (-1/2, -1/2) with the normalisation
 *     T_k = P_k^(-1/2,-1/2) / P_k^(-1/2,-1/2)(1) folded into its last / first step.
 *   LAG (a1, a2 > -1): one Toeplitz step (H = all ones).
 * Parameter differences above 4096 return UNSUPPORTED.
 * Synchronous: returns after the plan is complete.  *out receives the handle.
 * Errors: INVALID_ARG (kind, n_max < 1, tol <= 0, NULL out/params, parameters outside the
 * supported case), UNSUPPORTED (a case the library lacks), NOMEM, CUDA.
 */
int tdh_plan_create(int kind, int64_t n_max, const tdh_params* params, double tol,
                    tdh_plan_t* out);

/*
 * tdh_plan_execute -- beta = A alpha for `batch` vectors of n_max coefficients (Fig. 1 steps
 * 3-5): v = D2 alpha, w = sum_r u_r o T (u_r o v), beta = D1 w (+ row 0 for Cheb->Leg).
 * in:  device, batch * n_max values of the plan's precision (float64 or float32).
 * out: device, same shape and type; must not overlap `in` (TDH_ERR_ALIAS).
 * Both pointers 16-byte aligned (TDH_ERR_ALIGN).  batch == 0 is a no-op.
 * Asynchronous on `stream`; the plan may be used from several streams at once.
 */
int tdh_plan_execute(tdh_plan_t plan, const void* in, void* out, int64_t batch, void* stream);

/*
 * tdh_plan_execute_ragged -- beta = A alpha for `batch` vectors of different lengths in one
 * call.  Vector v occupies in[offsets[v] .. offsets[v+1]) and its result the same range of
 * out; its length n_v = offsets[v+1] - offsets[v] must be <= n_max (longer vectors are left
 * unwritten and TDH_STATUS_LENGTH is recorded, see tdh_plan_status; n_v = 0 is allowed).  One plan serves every length: H and T depend only on j+k
 * and k-j, so the n_v-prefix of the n_max factors approximates the n_v problem within the same
 * tolerance (the residual of a principal submatrix is a principal submatrix of the residual).
 * in, out: device arrays of offsets[batch] values of the plan's precision; out must not
 * overlap in.  The offsets live on the device, so that check runs there: if the ranges
 * [offsets[0], offsets[batch]) of in and out overlap, nothing is converted and
 * TDH_STATUS_ALIAS is recorded (tdh_plan_status); in == out is rejected on the host
 * (TDH_ERR_ALIAS).  offsets: device, batch + 1 int64, non-decreasing, offsets[0] >= 0.
 * The plan must have been created with TDH_FLAG_RAGGED (else TDH_ERR_INVALID_ARG) and have a
 * single T o H conversion step (Legendre/Chebyshev/ultraspherical Case 2; plan creation with
 * the flag returns UNSUPPORTED for other chains) with FFT lengths within
 * one thread-block cluster.  Vectors are grouped by FFT length on the device; each length
 * class is converted by one persistent launch that takes vectors from a work counter, and the
 * classes run concurrently on plan-owned streams forked from `stream` (capturable in a CUDA
 * graph).  Calls from several host threads are serialised while they enqueue (the fork and
 * join events are the plan's).  Asynchronous; scratch is stream-ordered (see Scratch above).
 */
int tdh_plan_execute_ragged(tdh_plan_t plan, const void* in, void* out, const int64_t* offsets,
                            int64_t batch, void* stream);

/*
 * tdh_plan_execute_adjoint -- grad = A^T g for `batch` vectors (the transpose product used
 * by reverse-mode differentiation): A^T = D2 (T^T o H) D1 with H symmetric, so the same
 * factors serve and T^T is applied with the conjugate (reversed) symbol.
 * Same layout, alignment, aliasing and stream rules as tdh_plan_execute.
 */
int tdh_plan_execute_adjoint(tdh_plan_t plan, const void* in, void* out, int64_t batch,
                             void* stream);

/*
 * tdh_plan_execute_host -- beta = A alpha (adjoint = 0) or A^T g (adjoint != 0) for `batch`
 * vectors in HOST memory: in and out are host pointers (batch * n_max values of the plan's
 * precision; page-locked memory lets the copies run asynchronously and overlap the work).
 * The batch moves through the device in chunks of at least 8 MB or a quarter of the batch:
 * the copy of one chunk in, the conversion of the previous one and the copy of the one
 * before out overlap on the plan's two copy streams and `stream`.  Device staging comes from
 * the library's scratch pool.  Asynchronous on `stream`: out is complete, and in may be
 * reused, once `stream` has been synchronised.  Host-buffer calls on one plan are serialised
 * by the library (it holds per-plan events); out must not overlap in (TDH_ERR_ALIAS).
 */
int tdh_plan_execute_host(tdh_plan_t plan, const void* in, void* out, int64_t batch, int adjoint,
                          void* stream);

/*
 * tdh_plan_execute_ragged_host -- tdh_plan_execute_ragged for vectors in HOST memory: vector v
 * occupies in[offsets[v] .. offsets[v+1]) and its result the same range of out.  in, out:
 * host arrays of the plan's precision (page-locked memory lets the copies overlap the work);
 * offsets: HOST, batch + 1 int64.  Because the offsets are on the host, every length is checked
 * before anything is enqueued: offsets[0] < 0, a decreasing offset or a vector longer than
 * n_max is TDH_ERR_INVALID_ARG; overlapping in and out ranges are TDH_ERR_ALIAS.  From 24 MB
 * of coefficients on, the batch moves through the device in chunks of whole vectors (about
 * a sixteenth of the coefficients first and last, the rest in two halves): the copy of one
 * chunk in, the conversion of the previous one (the device ragged path) and the copy of the
 * one before out overlap on the plan's copy streams and `stream`.  Results equal those of
 * tdh_plan_execute_ragged bit for bit (each vector is converted the same way in any chunk).
 * The plan requirements are those of tdh_plan_execute_ragged.  Device staging comes from the
 * library's scratch pool.  Asynchronous on `stream` (the call returns once the chunk offsets,
 * copied first, have been read): out is complete, and in may be reused, once `stream` has
 * been synchronised.  Host-buffer calls on one plan are serialised by the library.
 */
int tdh_plan_execute_ragged_host(tdh_plan_t plan, const void* in, void* out,
                                 const int64_t* offsets, int64_t batch, void* stream);

/*
 * tdh_plan_query -- report the plan's rank and size.  K (host, may be NULL) receives the
 * largest rank over the plan's conversion steps; n_max (host, may be NULL) its length.
 */
int tdh_plan_query(tdh_plan_t plan, int64_t* K, int64_t* n_max);

/*
 * Execute schedules (no counterpart in the paper, which fixes no GPU geometry).  Each FFT of
 * the execute path (Eq. (5): K zero-padded FFT pairs of length about 2N, Sec. 1) runs on one of
 * several compiled schedules: local FFT length LC = 2^log2LC per CTA, C CTAs per vector (a
 * thread-block cluster for C <= 8, a multi-pass exchange through global memory above), local
 * radix R, NT threads per CTA, and MINB, the CTAs per SM its registers are capped for.  A
 * plan's "configurations" are, in order: the dense configuration of each T o H step of its
 * chain, then (TDH_FLAG_RAGGED plans) one per FFT length class 2^8, 2^9, ... .  At creation
 * every configuration takes its default schedule (schedule 0).  Schedules differ only in
 * the order of floating-point operations.
 *
 * tdh_plan_schedule_count -- *count (host) receives the number of configurations.
 * tdh_plan_schedule_info -- info (host, 8 ints) receives, for configuration `config`:
 *   {log2 L, log2 LC, C, R, NT, MINB, index of the schedule in use, number of schedules}.
 *   Errors: INVALID_ARG (NULL plan/info, config out of range).
 * tdh_plan_set_schedule -- every configuration takes its schedule min(index, count - 1) (the
 *   execute tables are rebuilt where the schedule changes).  Synchronises `stream`.
 * tdh_plan_autotune -- times every schedule of every configuration on synthetic input (the
 *   dense configurations on `batch` vectors of n_max coefficients, each ragged length class on
 *   max(1, batch / classes) vectors of the class's longest length), shortest of three
 *   launches after one untimed, and keeps the fastest.  Uses about 2 * batch * n_max values of
 *   device memory while it runs; synchronises `stream`.  Errors: INVALID_ARG (batch < 1),
 *   NOMEM, CUDA.
 * Both calls that change schedules are synchronous, must not run while executes of the plan
 * are in flight or being captured, and free the tables the old schedule used: CUDA graphs
 * captured from the plan before the change must not be replayed after it.
 */
int tdh_plan_schedule_count(tdh_plan_t plan, int* count);
/*
 * tdh_schedules -- host only (no device call): the compiled schedules for an FFT of 2^logL
 * points in precision prec, the default first (ragged != 0: only those usable by ragged
 * batches, i.e. within one cluster).  out (host, 6 ints per schedule: log2 LC, C, R, NT,
 * MINB, and 0 within one cluster, 1 multi-pass, 2 multi-pass whose cross stage moves its
 * blocks by bulk tensor copies (TMA)) receives at most cap schedules; *count the number there
 * are (0 when no kernel covers that length).  Errors: INVALID_ARG.
 */
int tdh_schedules(int prec, int logL, int ragged, int* out, int cap, int* count);
int tdh_plan_schedule_info(tdh_plan_t plan, int config, int* info);
int tdh_plan_set_schedule(tdh_plan_t plan, int index, void* stream);
int tdh_plan_autotune(tdh_plan_t plan, int64_t batch, void* stream);

/* tdh_plan_destroy -- free the plan's device and host memory.  NULL is a no-op.  Waits for
 * nothing: the caller must not destroy a plan with launches still in flight. */
int tdh_plan_destroy(tdh_plan_t plan);

/*
 * tdh_plan_status -- conditions the plan's kernels found on the device: *status (host)
 * receives the TDH_STATUS_* bits recorded by the plan's executes so far (any stream), which
 * are then cleared.  TIMEOUT: a split-bfloat16 kernel gave up waiting (after about one
 * second) for its tensor-core products, and the outputs of that execute are not valid.
 * FAULT: a multi-pass cross stage found a bulk tensor copy misaligned and skipped it (outputs
 * not valid; never expected).  LENGTH, ALIAS: see tdh_plan_execute_ragged.  Synchronises `stream`; executes of interest
 * must be complete before it (e.g. enqueued on the same stream).
 * Errors: INVALID_ARG (NULL plan or status), CUDA.
 */
int tdh_plan_status(tdh_plan_t plan, int* status, void* stream);

/* tdh_last_error -- message of the last failing call on this thread ("" if none). */
const char* tdh_last_error(void);

/*
 * tdh_launch_count -- instrumentation (the paper has no counterpart): *count (host) receives
 * the number of kernel launches the library has enqueued for execute calls
 * (tdh_plan_execute, _ragged, _adjoint, _host, and the timed launches of tdh_plan_autotune)
 * in this process since it was loaded, all devices and threads together.  Plan creation and
 * the step entry points are not counted.
 * Errors: INVALID_ARG (NULL count).
 */
int tdh_launch_count(int64_t* count);

/*
 * tdh_alloc_stats -- instrumentation (the paper has no counterpart): stats (host, 3 int64)
 * receives, for this process, all devices and threads together:
 *   stats[0]  device allocations the library has made (plan memory and execute scratch);
 *   stats[1]  plan-memory blocks currently held (freed by tdh_plan_destroy);
 *   stats[2]  execute-scratch blocks currently held (returned to the pool stream-ordered).
 * Errors: INVALID_ARG (NULL stats).
 */
int tdh_alloc_stats(int64_t* stats);

/*
 * tdh_measure_fma_rate -- instrumentation (the paper has no counterpart): the fused
 * multiply-add throughput of the current device in precision prec (TDH_FP32: FFMA,
 * TDH_FP64: DFMA), counted as two flops per FMA, in TFLOP/s, written to *tflops (host).
 * A kernel of independent FMA chains fills every SM; the best of three timed launches (CUDA
 * events on `stream`, after one untimed) is reported.  These rates bound the execute
 * kernels, whose FFTs are arithmetic-bound.  Synchronous; changes no device setting.
 * Errors: INVALID_ARG, NOMEM, CUDA.
 */
int tdh_measure_fma_rate(int prec, double* tflops, void* stream);

/*
 * tdh_measure_dsmem_rate -- instrumentation (the paper has no counterpart): the throughput of
 * distributed shared memory in the access pattern of the float32 cluster kernel's cross stage
 * (4-CTA clusters, one 512-thread CTA per SM, as many clusters as can be resident, 16-byte
 * accesses to the other CTAs' shared memory).  bytes_per_cycle (host, 4 doubles) receives
 * the remote bytes per SM clock cycle per SM for { loads only, stores only, loads and stores
 * to other places at once (both directions counted) } with every cluster that fits resident,
 * and { loads only } with a single cluster on the whole device, from each CTA's clock64
 * cycles (the slowest CTA, best of two timed launches after one untimed).  The cross stage
 * moves 96 KB in and 96 KB out per rank term and CTA at C = 4, while other clusters are in
 * other phases.  Synchronous; changes no device setting.
 * Errors: INVALID_ARG, NOMEM, CUDA.
 */
int tdh_measure_dsmem_rate(double* bytes_per_cycle, void* stream);

/*
 * tdh_test_fail_alloc -- failure injection for tests (the paper has no counterpart): the k-th
 * device allocation the library attempts from now on (k >= 1, counting plan memory and
 * execute scratch, all threads) fails on the host as if the device were out of memory: the
 * calling entry point returns TDH_ERR_NOMEM with a message, frees what it had allocated, and
 * no CUDA allocation is attempted for it.  k = 0 cancels a pending failure.  Only the one
 * allocation fails; later ones proceed normally.  Errors: INVALID_ARG (k < 0).
 */
int tdh_test_fail_alloc(int64_t k);

/*
 * tdh_test_tc_stall -- failure injection for tests (the paper has no counterpart): while on
 * (on != 0), executes enqueued from then on with TDH_BF16X3 plans issue none of their
 * tensor-core products, so the first bounded wait of every CTA runs out after about one
 * second; the kernels then skip their remaining waits, finish, free their tensor memory and
 * record TDH_STATUS_TIMEOUT (tdh_plan_status).  Their outputs are not valid.  The setting is
 * process-wide and read when an execute is enqueued (a captured CUDA graph keeps the value it
 * was captured with).  Returns TDH_OK.
 */
int tdh_test_tc_stall(int on);

/*
 * tdh_symbols -- step a1 on its own: the split A = D1 (T o H) D2 of `kind` for n
 * coefficients, in float64, written to device arrays
 *   t[n]       T_{j, j+m} = t[m]           (upper-triangular Toeplitz generator)
 *   h[2n-1]    H_{jk} = h[j + k]           (Hankel generator)
 *   d1[n], d2[n]                            (the diagonals)
 * following Eq. (7) (LEG2CHEB), Sec. 5.1 (CHEB2LEG; h[0] = 1), Sec. 5.2 (ULTRA,
 * Case 2, |l1 - l2| < 1) and Sec. 5.3 (JAC with b == d, Case 2).  p as in tdh_params.p.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, UNSUPPORTED, CUDA.
 */
int tdh_symbols(int kind, int64_t n, const double* p, double* t, double* h, double* d1,
                double* d2, void* stream);

/*
 * tdh_pchol -- step a2 on its own: pivoted Cholesky (Sec. 2.1, Fig. 2) of the positive
 * semidefinite Hankel block H[j, k] = h[j + k], j, k in [j0, n), in float64.
 *   h       device, 2n - 1 values.
 *   u       device, kmax * n values (row-major [kmax][n]); row r receives
 *           u_r = l_r / sqrt(a_r) (zero below j0), so that H ~ sum_r u_r u_r^T.
 *   pivots  device, kmax int64 values; pivot index p_r (in [j0, n)) of step r.
 *   K       host; receives the number of steps taken.
 * Step r picks p_r = argmax d (lowest index on ties), forms column p_r of H minus the
 * earlier steps applied to it, and stops before any pivot a_r <= tol * max(diag H).
 * Synchronous (reads K back).  Errors: INVALID_ARG (n < 1, j0 not 0/1, tol <= 0,
 * kmax < 1), NOMEM, CUDA.
 */
int tdh_pchol(const double* h, int64_t n, int64_t j0, double tol, int64_t kmax, double* u,
              int64_t* pivots, int64_t* K, void* stream);

/*
 * tdh_pchol_noalloc -- tdh_pchol without any device allocation.  The paper has no
 * counterpart; this entry point exists for callers that may not call cudaMalloc (for
 * example code running where a caching allocator owns all device memory, or inside an
 * allocation-free section).  Same arguments, results and errors as tdh_pchol, with:
 *   - scratch from one static device array inside the library, sized for n <= 65536
 *     (about 0.5 MB, held by every GPU that loads the library until the process exits);
 *     n > 65536 returns TDH_ERR_INVALID_ARG with a message;
 *   - no cudaMalloc / cudaFree or allocating library call;
 *   - every call looks up the array's address for the current device
 *     (cudaGetSymbolAddress, which allocates nothing) and synchronises `stream`;
 *   - all calls on a device share the array: calls whose GPU work overlaps (other streams or
 *     host threads) race and must be serialised by the caller.
 */
int tdh_pchol_noalloc(const double* h, int64_t n, int64_t j0, double tol, int64_t kmax,
                      double* u, int64_t* pivots, int64_t* K, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TDH_H */
