/*
 * dvqls.h - C-ABI of the GB300 (sm_103a) D-VQLS hot path.
 *
 * Two parts of the Distributed Variational Quantum Linear Solver:
 *   1. the FWHT-based Pauli decomposition of A with tau pruning / top-L
 *      selection that produces the L weighted Pauli strings (Sec. 2.2,
 *      Eq. 3, Eq. 5; Algorithm 1, Steps 1-2), and
 *   2. the ideal state-vector evaluation of every Hadamard-test term of the
 *      global cost (Eq. 1 with A = sum_l c_l A_l):
 *          beta_lm  = <psi(alpha)| A_l^dag A_m |psi(alpha)>
 *          delta_l  = <b| A_l |psi(alpha)>
 *          C        = 1 - |sum_l c_l delta_l|^2 / sum_lm c_l^* c_m beta_lm
 *      and of the parameter-shift gradient (2P+1 shifted evaluations),
 *      i.e. Stages I-III of Sec. 2.3 (Algorithm 1, Steps 4a-4c) collapsed
 *      into one device pass.
 *
 * Conventions used by every entry point:
 *   - Basis index i = sum_k i_k 2^k; qubit k is bit k.  N = 2^n.
 *   - Pauli string from two bitmasks: sigma(x,z) = i^popc(x&z) X^x Z^z
 *     (Y where both bits are set), so sigma|i> = i^popc(x&z) (-1)^popc(z&i)
 *     |i XOR x>.  It is Hermitian, hence A_l^dag = A_l.
 *   - Complex numbers are interleaved (re, im) doubles.
 *   - Ansatz DVQLS_ANSATZ_RY_CZRING (the hardware-efficient ansatz of Sec.
 *     2.3 / Sec. 3 in its Ry + CZ form): an Ry layer with angles alpha[0..n),
 *     then `depth` times { CZ ring ; Ry layer alpha[l*n .. l*n+n) }, so
 *     P = n (depth+1) angles.  Ry(t) = [[cos t/2, -sin t/2], [sin t/2,
 *     cos t/2]]; the CZ ring is CZ(q,q+1) for q < n-1 plus CZ(n-1,0) when
 *     n >= 3.
 *   - Gradient: the parameter-shift rule, exact for both the numerator and
 *     the denominator of Eq. 1 because every angle enters one
 *     exp(-i a Y / 2) gate: f' = [f(a + pi/2) - f(a - pi/2)] / 2.
 *
 * Memory: every pointer argument may be host memory or device memory of the
 * context's device (told apart with cudaPointerGetAttributes; a context
 * remembers the addresses it found to be host memory and does not ask
 * again; host addresses lie outside the range the driver reserves for device
 * allocations).  Every array argument is dense: its elements follow each
 * other in memory in the order the function names them (only the address
 * crosses the ABI).  The caller owns all buffers; the library never frees caller
 * memory and never dereferences a caller pointer after the call returns.  The
 * context owns its workspace, staging buffers and CUDA graphs.  Work is
 * ordered on the context's stream.
 * Unless a function says otherwise it returns after its results are in the
 * caller's buffers.
 *
 * Errors: every function returns a dvqls_status.  No exception crosses the
 * ABI.  dvqls_last_error() gives a one-line description of the last failure
 * on the context.
 *
 * Tracing: the main calls, and inside a cost pass the autotuning and the
 * pass kernels, are NVTX ranges on a profiler's timeline (nothing happens
 * without a profiler attached); dvqls_profile_* times the kernels of a pass.
 */
#ifndef DVQLS_H
#define DVQLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DVQLS_OK = 0,
    DVQLS_ERR_INVALID_ARG = 1, /* bad size, mask, pointer or non-finite input */
    DVQLS_ERR_UNSUPPORTED = 2, /* valid request this build does not serve    */
    DVQLS_ERR_CUDA = 3,        /* a CUDA runtime call failed                  */
    DVQLS_ERR_TIMEOUT = 4,     /* a bounded device wait gave up               */
    DVQLS_ERR_NUMERIC = 5,     /* D <= 0 or a non-finite result               */
    DVQLS_ERR_ALLOC = 6        /* device or pinned allocation failed          */
} dvqls_status;

/* Arithmetic of the state build and the term reductions.  The FP32 paths
 * keep the coefficient-weighted L^2 sum, the cost ratio and the gradient
 * combine in FP64.
 *   DVQLS_FP32:    FP32 states, FP32 term reductions on the CUDA cores.
 *   DVQLS_FP32_TC: FP32 states; the term Gram on the tensor cores
 *                  (tcgen05 kind::f16: every amplitude, scaled by 2^12,
 *                  split into FP16 hi + lo; the products hi hi + hi lo +
 *                  lo hi with FP32 accumulation and periodic round-to-nearest
 *                  folding), 64-term tiles and pairs of tiles for any L,
 *                  which keeps FP32-level accuracy (the FP32 bounds of the
 *                  parity tests hold).  Weighted sums in float-float (~2^-44
 *                  relative), combined in FP64.  Served for the global
 *                  and the local cost (flavour j of the local cost as the
 *                  Gram of a tile against its strings with x ^ e_j).
 *   DVQLS_FP32_WHT: an exact reformulation of the same terms (not the
 *                  paper's per-term evaluation): the pairs (l, m) are
 *                  grouped by x_l ^ x_m and one FP32
 *                  Walsh-Hadamard transform of psi[i] psi[i ^ x] gives every
 *                  beta of a group (likewise delta by x_l); cost for
 *                  structured LCUs is (groups) x N log N instead of L^2 N.
 *                  The local cost's flavour j reads the transform at
 *                  x ^ e_j (X_j between the two terms).  Served for the
 *                  global and the local cost when every instance has
 *                  L <= 64 and n <= 10; other global-cost calls run as
 *                  DVQLS_FP32_TC, other local-cost calls as DVQLS_FP32. */
typedef enum { DVQLS_FP64 = 0, DVQLS_FP32 = 1, DVQLS_FP32_TC = 2, DVQLS_FP32_WHT = 3 } dvqls_precision;

typedef enum { DVQLS_ANSATZ_RY_CZRING = 0 } dvqls_ansatz_kind;

/* Largest n served with the state resident in shared memory; above it (up to
 * DVQLS_MAX_QUBITS) the cost passes build every shifted state in HBM
 * (S x 2^n amplitudes of workspace) and stream it through L2. */
#define DVQLS_MAX_SMEM_QUBITS 12
#define DVQLS_MAX_QUBITS 20
/* Largest n for a dense decomposition input (N x N doubles). */
#define DVQLS_MAX_DENSE_QUBITS 12

typedef struct dvqls_ctx dvqls_ctx;

/* A context is not thread-safe: its workspace, staging buffers, graph cache
 * and autotuning table are shared by its calls, so one thread at a time may
 * use it (one context per host thread for concurrent work). */

/* Create a context on CUDA device `device`.  `stream` is the cudaStream_t
 * every call of this context is ordered on (passed as void* so this header
 * needs no CUDA include); NULL is the default stream.  The context never
 * destroys the caller's stream; it creates one private stream of its own,
 * used only to record CUDA graphs of the cost pass.  *out receives the
 * context.
 * Errors: INVALID_ARG (out == NULL or no such device), CUDA, ALLOC. */
int dvqls_create(dvqls_ctx** out, int device, void* stream);

/* Synchronise the context's stream and release everything the context owns.
 * NULL is accepted and ignored. */
void dvqls_destroy(dvqls_ctx* ctx);

/* One-line description of the last failure on `ctx` ("" if none).  The
 * string lives until the next call on the context. */
const char* dvqls_last_error(const dvqls_ctx* ctx);

/* Wait for all work enqueued on the context's stream and return the first
 * deferred error of an asynchronous call (see dvqls_cost_grad_batched). */
int dvqls_sync(dvqls_ctx* ctx);

/* Kernel timing for measurement.  While enabled, each kernel launch of the
 * batched cost pass is bracketed by CUDA events recorded on the context's
 * stream.  Enabling (enable = 1) resets the counters; disabling keeps them.
 * dvqls_profile_read synchronises the stream and returns, for `phase`
 * (0: prepare, 1: term tiles, 2: combine, 3: state passes in HBM for n > 12,
 * 4: the on-chip state build of the tensor-core pass), the number of
 * launches and their total duration in milliseconds since the last reset.
 * Errors: INVALID_ARG (phase out of range), CUDA. */
int dvqls_profile_enable(dvqls_ctx* ctx, int enable);
int dvqls_profile_read(dvqls_ctx* ctx, int phase, long long* launches, double* ms);

/* Failure detection: the timeout budget of the device waits.  The warp roles
 * of the tensor-core term kernel (DVQLS_FP32_TC) hand work to each other
 * through shared-memory barriers; every wait on one gives up after
 * `microseconds` of the GPU's global timer (<= 0 restores the default of one
 * second; at most an hour).  A wait that gives up stops the kernel cleanly --
 * each role leaves at its next check and waits no more, the tensor memory is
 * freed only after every issued MMA has completed -- and the call (or the
 * next dvqls_sync) returns DVQLS_ERR_TIMEOUT; the context stays usable.  A
 * budget far below the time the work takes makes calls time out; a healthy
 * kernel's waits last microseconds.  The paper has no counterpart: there
 * every circuit is its own asynchronous job (Sec. 2.3), here one kernel holds
 * the whole pass, so a stuck hand-over must end in an error instead of a wait
 * without end.
 * Errors: INVALID_ARG (ctx NULL). */
int dvqls_set_wait_budget(dvqls_ctx* ctx, long long microseconds);

/* ------------------------------------------------------------------------
 * Pauli decomposition (Sec. 2.2, Eq. 5; Algorithm 1, Steps 1-2).
 *
 * c(x,z) = Tr(sigma(x,z)^dag A) / N, computed by grouping the entries of A by
 * X-mask x = row XOR column, a Walsh-Hadamard transform of each diagonal
 * d_x(i) = A[i XOR x, i] (radix-2, strides 1, 2, ..., N/2), the phase
 * (-i)^popc(x&z) and the 1/N scale.  Pruning (one scan): with
 * key = re*re + im*im (no fused multiply-add) and thr = (tau*tau) * max key
 * (thr = 0 when tau <= 0), keep the coefficients with key > thr, i.e.
 * |c| > tau * max|c| -- the largest coefficient normalised to one, as in
 * Sec. 2.5.1.  Order: key descending, ties by (x << n) | z ascending.  At
 * most L_max rows are written.
 *
 * A:      dense real N x N, row-major, FP64; 1 <= n <= DVQLS_MAX_DENSE_QUBITS.
 * coef:   L_max complex128 (2 L_max doubles), xmask, zmask: L_max uint32.
 * L_out:  rows written = min(L_post, L_max).       (host int)
 * L_pre:  number of nonzero coefficients.          (host int)
 * L_post: number passing the tau filter (before the L_max cap). (host int)
 * Errors: INVALID_ARG (n out of range, L_max < 1, tau NaN or negative
 * infinity, NULL output), ALLOC, CUDA. */
int dvqls_pauli_decompose(dvqls_ctx* ctx, const double* A, int n, double tau, int L_max,
                          double* coef, uint32_t* xmask, uint32_t* zmask,
                          int* L_out, int* L_pre, int* L_post);

/* Same for a banded real matrix, for sizes whose dense form does not fit
 * (up to n = DVQLS_MAX_QUBITS).  offsets[k] is the diagonal offset (column -
 * row) of band k; band_values is nbands x N, band_values[k*N + r] =
 * A[r, r + offsets[k]] (entries that fall outside the matrix are ignored).
 * Offsets must be distinct with |offset| < N.  offsets is a host array. */
int dvqls_pauli_decompose_banded(dvqls_ctx* ctx, int n, int nbands, const int* offsets,
                                 const double* band_values, double tau, int L_max,
                                 double* coef, uint32_t* xmask, uint32_t* zmask,
                                 int* L_out, int* L_pre, int* L_post);

/* ------------------------------------------------------------------------
 * Cost and gradient (Eq. 1, Eq. 3; Sec. 2.3 Stages I-III).
 */
typedef struct {
    int n;     /* system qubits, 1 <= n <= DVQLS_MAX_QUBITS               */
    int depth; /* ansatz layers d >= 0; P = n (d + 1) angles              */
    int kind;  /* dvqls_ansatz_kind                                       */
} dvqls_ansatz;

typedef struct {
    int L;                 /* number of terms, >= 1                       */
    const double* coef;    /* L complex128 c_l                            */
    const uint32_t* xmask; /* L X-masks, each < 2^n                       */
    const uint32_t* zmask; /* L Z-masks, each < 2^n                       */
} dvqls_lcu;

/* Cost C(alpha) of Eq. 1 for one instance.
 * alpha: P doubles.  b: N complex128 right-hand side; the library uses
 * b / ||b|| (||b|| = 0 is an INVALID_ARG).
 * Outputs (any may be NULL except cost): cost (1 double), beta (L x L
 * complex128, row l, column m), delta (L complex128), both at alpha.
 * Errors: INVALID_ARG, UNSUPPORTED, NUMERIC (D <= 0 or non-finite), ALLOC,
 * CUDA. */
int dvqls_cost(dvqls_ctx* ctx, const dvqls_ansatz* ansatz, const double* alpha,
               const dvqls_lcu* lcu, const double* b, int precision,
               double* cost, double* beta, double* delta);

/* Cost and parameter-shift gradient for one instance: the 2P+1 angle
 * vectors alpha, alpha + (pi/2) e_k, alpha - (pi/2) e_k each take all
 * L^2 + L terms; then C = 1 - N0/D0 and
 * dC/dalpha_k = -(N'_k D0 - N0 D'_k) / D0^2 with N'_k, D'_k half the
 * difference of the shifted values.  grad: P doubles.  Other arguments as
 * dvqls_cost. */
int dvqls_cost_grad(dvqls_ctx* ctx, const dvqls_ansatz* ansatz, const double* alpha,
                    const dvqls_lcu* lcu, const double* b, int precision,
                    double* cost, double* grad, double* beta, double* delta);

/* One problem of a batch. */
typedef struct {
    dvqls_ansatz ansatz;
    dvqls_lcu lcu;
    const double* alpha; /* P doubles      */
    const double* b;     /* N complex128    */
} dvqls_instance;

/* Cost and gradient of `count` independent instances (mixed n, depth, L)
 * in one device pass: all S_i (L_i^2 + L_i) terms of every instance are
 * work items of one persistent launch, ordered longest-first.
 * costs: count doubles; grads: sum_i P_i doubles, instance i at offset
 * sum_{j<i} P_j.  Either may be NULL.
 * When costs and grads are both device memory (or NULL) and every input is
 * device memory, the call only enqueues work and returns; numeric errors are
 * then reported by the next dvqls_sync().  Otherwise it returns after the
 * results are in place.
 * Launch: the first call of a problem signature (precision and every
 * instance's n, depth, L) times each split of the amplitude range among the
 * candidates 1, 2, 4, 8 -- for the tensor-core kernel each with the layouts
 * of the on-chip states (split hi / lo arrays, for every size or only from
 * 2^9 amplitudes, or packed copies) where they fit -- on the real inputs (the
 * fastest of three passes per candidate) and keeps the fastest for the
 * context (an autotuner; that call is synchronous), unless dvqls_set_tuning
 * fixed the choices.  The kernel sequence of a
 * pass is captured once as a CUDA graph and replayed while the instance
 * table (shapes and pointers) is unchanged; with profiling enabled, or when
 * the caller is capturing the stream, kernels are launched directly.
 * Errors: as dvqls_cost_grad, for any instance; INVALID_ARG for count < 1
 * (an empty batch) or inst NULL. */
int dvqls_cost_grad_batched(dvqls_ctx* ctx, int count, const dvqls_instance* inst,
                            int precision, double* costs, double* grads);

/* Fixes the autotuner's choices for this context's later batched and single
 * calls instead of timing candidates (A9; the paper has no autotuner): the
 * amplitude split `split` (1, 2, 4 or 8; 0 = tune again) and, for the
 * tensor-core kernel, the state layout `layout` (0: split hi / lo arrays for
 * states of 2^4 .. 2^10 amplitudes, 1: split arrays only from 2^9, 2: packed
 * copies; -1 = tuned, or 0 when the split is fixed).  A layout that does not
 * fit the CTA's shared memory falls back as the tuner would.  For callers
 * that cannot afford the synchronous tuning call, and for comparing layouts:
 * the layouts give bit-identical results (the same operand values reach the
 * tensor cores), the splits differ only in summation order.
 * Errors: INVALID_ARG (ctx NULL, split not 0, 1, 2, 4, 8, layout not -1..2). */
int dvqls_set_tuning(dvqls_ctx* ctx, int split, int layout);

/* One instance split across ranks (Sec. 2.3 Stage III; Algorithm 1, Step
 * 4c).  A rank evaluates the shifts s_begin .. s_end - 1 of the 2P + 1
 * parameter-shift evaluations (0 <= s_begin < s_end <= 2P + 1; shift 0 is
 * alpha, 2k + 1 is alpha + (pi/2) e_k, 2k + 2 is alpha - (pi/2) e_k) and
 * writes, for every shift g of the instance, the four doubles
 *     partials[4 g .. 4 g + 3] = (Re T_g, Im T_g, Re D_g, Im D_g),
 *     T_g = sum_l c_l delta_l (b normalised), D_g = sum_lm c_l^* c_m beta_lm,
 * with zeros for the shifts outside its range.  The arrays of ranks whose
 * ranges cover 0 .. 2P without overlap add up, element by element (one SUM
 * allreduce of (2P + 1) x 4 doubles, the paper's exchange of two scalars per
 * evaluated cost), to the whole instance's; N_g = |T_g|^2 is formed only
 * after that sum, by dvqls_combine_partials.  partials: (2P + 1) x 4
 * doubles, host or device.  Other arguments as dvqls_cost_grad.
 * Errors: as dvqls_cost_grad; INVALID_ARG for an empty or out-of-range shift
 * range. */
int dvqls_cost_grad_partials(dvqls_ctx* ctx, const dvqls_ansatz* ansatz, const double* alpha,
                             const dvqls_lcu* lcu, const double* b, int precision, int s_begin, int s_end,
                             double* partials);

/* Cost and parameter-shift gradient of one instance from its complete
 * per-shift sums (the layout dvqls_cost_grad_partials writes, summed over
 * the ranks): N_g = |T_g|^2, C = 1 - N_0 / D_0 and dC/dalpha_k =
 * -(N'_k D_0 - N_0 D'_k) / D_0^2 with N'_k, D'_k half the difference of the
 * shifted values (Eq. 1; the shift rule), in FP64 on the GPU.  n, depth give
 * P = n (depth + 1); partials: (2P + 1) x 4 doubles; cost: 1 double; grad:
 * P doubles; host or device.
 * Errors: INVALID_ARG, UNSUPPORTED (P > 1024), NUMERIC (D_0 <= 0 or not
 * finite), ALLOC, CUDA. */
int dvqls_combine_partials(dvqls_ctx* ctx, int n, int depth, const double* partials, double* cost, double* grad);

/* Local cost (Eq. 2, expanded in Eq. 4; closed form of Sec. 2.3 Stage III):
 *   C_L = 1 - (1/n) sum_j <x|A^dag U_b P_j U_b^dag A|x> / <x|A^dag A|x>,
 *   P_j = (I + Z_j)/2, which is C_L = 1/2 - E / (2 n D) with
 *   D = sum_lm c_l^* c_m beta_lm and E = sum_j sum_lm c_l^* c_m gamma^j_lm,
 *   gamma^j_lm = <x| A_l^dag U_b Z_j U_b^dag A_m |x>
 * -- the paper's (n+1) L^2 expectation values per evaluation.  Served for
 * b = |+>^n (U_b = H^(x)n, so U_b Z_j U_b^dag = X_j and every gamma^j_lm is a
 * Pauli-string overlap); b is not an argument.  grad may be NULL (cost only);
 * with grad, the 2P+1 shifted evaluations give the exact parameter-shift
 * gradient of E and D.  Same arithmetic split as dvqls_cost_grad (FP32 or
 * FP64 terms, FP64 sums). */
int dvqls_local_cost_grad(dvqls_ctx* ctx, const dvqls_ansatz* ansatz, const double* alpha,
                          const dvqls_lcu* lcu, int precision, double* cost, double* grad);

/* Local cost of `count` instances in one pass (inst[i].b is ignored); costs,
 * grads, the asynchronous behaviour and the errors as dvqls_cost_grad_batched;
 * grads NULL evaluates the cost only. */
int dvqls_local_cost_grad_batched(dvqls_ctx* ctx, int count, const dvqls_instance* inst,
                                  int precision, double* costs, double* grads);

/* Per-circuit FP64 path (Sec. 2.3 execution model; Sec. 2.2 after Eq. 4):
 * each Hadamard-test circuit -- S (L^2 + L) expectation values, real and
 * imaginary part each from its own circuit, 2 S (L^2 + L) circuits -- is
 * simulated on its own (n+1)-qubit complex128 state vector gate by gate
 * (H, Ry / controlled Ry, CZ / CCZ, controlled X / Y / Z per Pauli factor,
 * controlled U_b^dag, S^dag) and measured as <Z_ancilla>; then the same FP64
 * combine as dvqls_cost_grad.  U_b is H^(x)n when b = |+>^n, else the phased
 * Householder reflection mapping |0> to b/||b||.  Same arguments and outputs
 * as dvqls_cost_grad (FP64 only); n + 1 <= 13.  It is the comparison path of
 * the batched evaluation and a second FP64 check of it. */
int dvqls_circuit_cost_grad_fp64(dvqls_ctx* ctx, const dvqls_ansatz* ansatz, const double* alpha,
                                 const dvqls_lcu* lcu, const double* b,
                                 double* cost, double* grad, double* beta, double* delta);

/* ------------------------------------------------------------------------
 * Fidelity, classical solve and the optimizer loop (Sec. 3.1; Algorithm 1).
 */

/* F = |<xhat|psi(alpha)>|^2 / ||xhat||^2 with psi(alpha) = V(alpha)|0> built
 * in FP64 (Sec. 3.1: fidelity against the classical solution).  xhat: N
 * complex128, any nonzero norm.  n <= DVQLS_MAX_QUBITS: above
 * DVQLS_MAX_SMEM_QUBITS the state is built in HBM (N doubles of workspace) and
 * the overlap is summed over the GPU in a fixed block order.
 * Errors: INVALID_ARG (n, depth, NULL, a non-finite angle, xhat = 0),
 * UNSUPPORTED (another ansatz), ALLOC, CUDA. */
int dvqls_fidelity(dvqls_ctx* ctx, const dvqls_ansatz* ansatz, const double* alpha,
                   const double* xhat, double* F);

/* Classical solution x = A~^{-1} b of the system the LCU encodes,
 * A~ = sum_l c_l A_l applied as a Pauli-string matvec in FP64: conjugate
 * gradients (A~ Hermitian positive definite), falling back to CG on the
 * normal equations when CG breaks down (p^dag A~ p <= 0).  Stops when
 * ||r|| / ||rhs|| <= tol or after max_iter iterations.  N < 4096: one CTA;
 * larger: the same iteration spread over the whole GPU (grid kernels, the dot
 * products added in a fixed block order).  x: N complex128
 * (not normalised).  iters, rel_resid may be NULL.  Returns NUMERIC when tol
 * was not reached (x then holds the last iterate). */
int dvqls_lcu_solve(dvqls_ctx* ctx, int n, const dvqls_lcu* lcu, const double* b, double tol,
                    int max_iter, double* x, int* iters, double* rel_resid);

/* The same solve for nrhs >= 1 right-hand sides of one LCU in one launch (one
 * CTA each).  b and x: nrhs x N complex128, right-hand side k at offset k N.
 * iters, rel_resid: NULL or nrhs entries (host memory).  Every solve runs to
 * tol or max_iter; returns NUMERIC when any did not reach tol (x, iters and
 * rel_resid are still written for all). */
int dvqls_lcu_solve_batched(dvqls_ctx* ctx, int n, const dvqls_lcu* lcu, int nrhs, const double* b,
                            double tol, int max_iter, double* x, int* iters, double* rel_resid);

typedef struct {
    double lr, beta1, beta2, eps; /* Adam step size and moment decay rates   */
    int max_iter;                 /* updates at most                          */
    double target_fidelity;       /* stop an instance once F >= this          */
    int precision;                /* dvqls_precision of the cost pass         */
    const double* targets;        /* NULL, or one target per instance (host
                                     memory) used instead of target_fidelity */
} dvqls_adam;

typedef struct {
    int iters;       /* Adam updates made before the stop                */
    int converged;   /* 1 when F >= target_fidelity was reached          */
    double cost;     /* C at the final angles                            */
    double fidelity; /* F at the final angles                            */
} dvqls_opt_result;

/* Adam on the angles of `count` instances in lock step (Algorithm 1's loop
 * with Adam as the optimizer): each iteration evaluates, for every instance
 * still running, F(alpha) against xhat and the batched cost and parameter-
 * shift gradient, stops the instances with F >= target_fidelity, and updates
 * the others.  Starts from inst[i].alpha; inst[i].alpha is not written.
 * xhat: packed N_i complex128 per instance (the classical solution).
 * alpha_out: packed P_i doubles per instance (final angles).  results: count
 * entries (host memory).  The optimizer allocates its own state for the
 * call and frees it before returning.
 * Errors: INVALID_ARG for count < 1 or a NULL argument, else as
 * dvqls_cost_grad_batched and dvqls_fidelity. */
int dvqls_optimize(dvqls_ctx* ctx, int count, const dvqls_instance* inst, const double* xhat,
                   const dvqls_adam* opt, double* alpha_out, dvqls_opt_result* results);

/* Checkpoint and resume of the optimizer loop.  The Adam state of `count`
 * instances: the first and second moments (packed P_i doubles per instance,
 * like the angles) and the number of updates each instance has had (its bias
 * corrections are 1 - beta^steps).  Host or device memory, read and written
 * by dvqls_optimize_resume. */
typedef struct {
    double* m;        /* sum_i P_i doubles                     */
    double* v;        /* sum_i P_i doubles                     */
    long long* steps; /* count updates made so far             */
} dvqls_adam_state;

/* dvqls_optimize from a checkpoint: starts from inst[i].alpha with the given
 * Adam state (m = v = 0, steps = 0 is a fresh start, identical to
 * dvqls_optimize), runs at most opt->max_iter updates, and writes the final
 * angles to alpha_out and the final state back to *state.  Saving alpha_out
 * and the state after K updates and resuming from them gives, bit for bit,
 * the angles and state of one run of K + K' updates (the bias-correction
 * products are formed in the same order).
 * Errors: as dvqls_optimize; INVALID_ARG for a NULL state array or a
 * negative update count. */
int dvqls_optimize_resume(dvqls_ctx* ctx, int count, const dvqls_instance* inst, const double* xhat,
                          const dvqls_adam* opt, dvqls_adam_state* state, double* alpha_out,
                          dvqls_opt_result* results);

/* ------------------------------------------------------------------------
 * Learned warm start.  Algorithm 1, Step 3 initialises theta randomly; this
 * replaces that step with a prediction (the paper has no learned
 * initialisation; random or fixed initialisation stays the fallback).  A
 * small MLP maps a problem description (features) to initial angles:
 *   h1 = GELU(W1 x + b1), h2 = GELU(W2 h1 + b2), y = W3 h2 + b3,
 *   GELU(z) = z (1 + erf(z / sqrt 2)) / 2,
 * trained on the GPU by these kernels (FP32) on the masked mean squared
 * error sum M (y - t)^2 / sum M with Adam (beta 0.9, 0.999, eps 1e-8).
 * Parameters are one flat FP32 vector: W1 [H x I], b1 [H], W2 [H x H],
 * b2 [H], W3 [O x H], b3 [O] (row-major), dvqls_ws_param_count() floats.
 * Batch arrays are row-major: feats [batch x I], target and mask
 * [batch x O] (mask 1 where the target entry counts, else 0).  Pointers may
 * be host or device memory.
 */
typedef struct dvqls_ws dvqls_ws;

/* Number of parameters, or -1 for a dimension < 1. */
long long dvqls_ws_param_count(int in_dim, int hidden, int out_dim);

/* New network on ctx's device with the given initial parameters (the
 * caller draws them); Adam moments start at zero. */
int dvqls_ws_create(dvqls_ctx* ctx, int in_dim, int hidden, int out_dim, const float* params,
                    dvqls_ws** out);
void dvqls_ws_destroy(dvqls_ws* ws);

/* out [batch x O] = y(feats). */
int dvqls_ws_infer(dvqls_ws* ws, int batch, const float* feats, float* out);

/* Loss (may be NULL) and its gradient with respect to the parameters
 * (param_count floats), without updating anything. */
int dvqls_ws_grad(dvqls_ws* ws, int batch, const float* feats, const float* target,
                  const float* mask, float* loss, float* grad);

/* One Adam step on the batch with step size lr.  loss (may be NULL) is the
 * batch loss before the step; passing NULL avoids a synchronisation. */
int dvqls_ws_train_step(dvqls_ws* ws, int batch, const float* feats, const float* target,
                        const float* mask, float lr, float* loss);

int dvqls_ws_get_params(dvqls_ws* ws, float* params);

/* Checkpoint: "DVQLSWS1", int32 I, H, O, int64 Adam step, then the
 * parameters and both Adam moments (FP32).  Loading restores training
 * state exactly. */
int dvqls_ws_save(dvqls_ws* ws, const char* path);
int dvqls_ws_load(dvqls_ctx* ctx, const char* path, dvqls_ws** out);

/* ------------------------------------------------------------------------
 * Allocation-free cost and gradient.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate GPU memory, such as
 * code running inside a memory pool or allocator that owns the whole device,
 * a real-time loop whose allocation pattern is fixed, or a plugin host that
 * forbids cudaMalloc.  It computes what dvqls_cost_grad computes in
 * DVQLS_FP64 or DVQLS_FP32 (the same kernels; no beta / delta output)
 * without a context: it calls no cudaMalloc, cudaFree, cudaMallocHost or
 * other allocating routine.
 *
 * Its scratch is one fixed device array of DVQLS_NOALLOC_SCRATCH_BYTES
 * inside this library; every GPU that loads the library holds it until the
 * process exits.  A request whose scratch exceeds it is rejected with
 * INVALID_ARG.  The scratch it needs is, in bytes (each term rounded up to
 * 256): sizeof record + 256 + 16 L + 16 L^2 + 48 P + 8 + 16 S T^2 k
 * + 16 S T k + 24 S, with S = 2P+1, T = ceil(L/64) and k <= 8 the split of
 * the amplitude range, plus 16 L^2 + 16 L in DVQLS_FP32 (the weights as
 * float pairs).  With the largest split (k = 8), n = 10, depth 4 (P = 50)
 * fits up to L = 160 in FP32 and L = 200 in FP64 on any GPU.
 *
 * The call runs on the current CUDA device, ordered on `stream` (a
 * cudaStream_t, NULL = default stream); it waits for that stream before it
 * returns, so cost and grad are written when it returns.  alpha, b, the lcu
 * arrays, cost and grad must all be device memory of the current device
 * (nothing is staged): a host pointer is INVALID_ARG.
 * Every call looks up the array's device address (cudaGetSymbolAddress,
 * with the current device) instead of keeping one from an earlier call, so a
 * device reset by the host program between calls leaves no stale address.
 * Every call shares the one array and finds the previous call's contents
 * there: two calls that overlap on the GPU (other streams, other threads)
 * race and give wrong results, so keep calls ordered on one stream or
 * serialise them.
 * Errors: INVALID_ARG; UNSUPPORTED (n > DVQLS_MAX_SMEM_QUBITS, another
 * ansatz, or precision DVQLS_FP32_TC / DVQLS_FP32_WHT); NUMERIC; CUDA, also
 * returned without any work when the caller's thread already has a CUDA
 * error pending (that error is left in place).  No error text is kept
 * (there is no context). */
#define DVQLS_NOALLOC_SCRATCH_BYTES (1u << 20)
int dvqls_cost_grad_noalloc(void* stream, const dvqls_ansatz* ansatz, const double* alpha,
                            const dvqls_lcu* lcu, const double* b, int precision,
                            double* cost, double* grad);

#ifdef __cplusplus
}
#endif

#endif /* DVQLS_H */
