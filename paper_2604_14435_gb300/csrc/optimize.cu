// Fidelity, classical solve and the optimizer loop (Algorithm 1, Step 3 and
// the while-loop; Sec. 3.1 fidelity).
//
//   dvqls_fidelity      F = |<xhat|psi(alpha)>|^2 / ||xhat||^2, psi built in
//                       FP64 in shared memory.
//   dvqls_lcu_solve(_batched)  xhat = A~^{-1} b for A~ = sum_l c_l A_l applied as a
//                       Pauli-string matvec, by conjugate gradients (A~
//                       Hermitian positive definite), falling back to CG on
//                       the normal equations A~^dag A~ x = A~^dag b when CG
//                       breaks down; FP64, bounded iteration count.
//   dvqls_optimize      Adam on alpha with the batched cost and parameter-
//                       shift gradient each iteration, many instances in
//                       lock step; an instance stops when F >= target.
#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "state.cuh"

namespace dvqls {


namespace {

constexpr int FT = 256;
constexpr int CGT = 1024;

struct FidInst {
    int n, d, P;
    const double* alpha;
    const double2* xhat;
    double2* cs;  // P (cos, sin) scratch
    double* F;
};

__device__ double2 block_sum2_all(double2 v, double2* red) {
    for (int o = 16; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        s.x += red[k].x;
        s.y += red[k].y;
    }
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(FT) k_fidelity(const FidInst* __restrict__ insts, int* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double2 red[FT / 32];
    const FidInst I = insts[blockIdx.x];
    const int N = 1 << I.n;
    double2* psi = reinterpret_cast<double2*>(smem);
    double2* scs = psi + N;
    for (int a = threadIdx.x; a < I.P; a += FT) {
        const double al = I.alpha[a];
        if (!isfinite(al)) atomicCAS(status, 0, DEV_NONFINITE_INPUT);
        double s, c;
        sincos(0.5 * al, &s, &c);
        I.cs[a] = make_double2(c, s);
    }
    __syncthreads();
    build_state<double>(psi, scs, I.n, I.d, I.P, I.cs, 0);
    double2 ov = make_double2(0.0, 0.0), nx = make_double2(0.0, 0.0);
    for (int j = threadIdx.x; j < N; j += FT) {
        const double2 x = I.xhat[j], p = psi[j];
        ov.x += x.x * p.x + x.y * p.y;  // conj(x) p
        ov.y += x.x * p.y - x.y * p.x;
        nx.x += x.x * x.x + x.y * x.y;
    }
    ov = block_sum2_all(ov, red);
    nx = block_sum2_all(nx, red);
    if (threadIdx.x == 0) {
        if (!(nx.x > 0.0) || !isfinite(nx.x)) atomicCAS(status, 0, DEV_BAD_NORM);
        *I.F = (ov.x * ov.x + ov.y * ov.y) / nx.x;
    }
}

// y = A~ v (conj_coef = 0) or A~^dag v (conj_coef = 1); all threads of the CTA.
__device__ void lcu_matvec(int n, int L, const double2* coef, const uint32_t* xm, const uint32_t* zm,
                           const double2* v, double2* y, int conj_coef) {
    const int N = 1 << n;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double yr = 0.0, yi = 0.0;
        for (int l = 0; l < L; ++l) {
            const uint32_t x = xm[l] & (N - 1), z = zm[l] & (N - 1);
            double2 c = coef[l];
            if (conj_coef) c.y = -c.y;  // (c_l sigma_l)^dag = conj(c_l) sigma_l (sigma_l is Hermitian)
            double2 ph;  // i^popc(x&z)
            switch (__popc(x & z) & 3) {
                case 0: ph = make_double2(1, 0); break;
                case 1: ph = make_double2(0, 1); break;
                case 2: ph = make_double2(-1, 0); break;
                default: ph = make_double2(0, -1); break;
            }
            const uint32_t src = uint32_t(j) ^ x;
            const double sg = (__popc(z & src) & 1) ? -1.0 : 1.0;
            const double2 a = v[src];
            const double cr = c.x * ph.x - c.y * ph.y, ci = c.x * ph.y + c.y * ph.x;
            yr += sg * (cr * a.x - ci * a.y);
            yi += sg * (cr * a.y + ci * a.x);
        }
        y[j] = make_double2(yr, yi);
    }
    __syncthreads();
}

__device__ double2 dotc(int N, const double2* a, const double2* b, double2* red) {  // a^dag b
    double2 s = make_double2(0.0, 0.0);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double2 x = a[j], y = b[j];
        s.x += x.x * y.x + x.y * y.y;
        s.y += x.x * y.y - x.y * y.x;
    }
    return block_sum2_all(s, red);
}

// Single CTA conjugate gradients; vectors in global memory (L2-resident).
// out: [0] iterations, [1] relative residual, [2] 1 if converged, [3] 1 if
// the normal equations were used.
__global__ void __launch_bounds__(CGT) k_cg(int n, int L, const double2* coef, const uint32_t* xm, const uint32_t* zm,
                                           const double2* b, double2* x, double2* r, double2* p, double2* Ap,
                                           double2* tmp, double tol, int max_iter, double* out) {
    __shared__ double2 red[CGT / 32];
    const int N = 1 << n;
    {  // one CTA per right-hand side: vectors of N entries each, four result words
        const long long o = (long long)blockIdx.x * N;
        b += o;
        x += o;
        r += o;
        p += o;
        Ap += o;
        tmp += o;
        out += 4 * blockIdx.x;
    }
    for (int normal = 0; normal < 2; ++normal) {
        // r = rhs (b, or A~^dag b), x = 0, p = r
        if (normal) lcu_matvec(n, L, coef, xm, zm, b, r, 1);
        else
            for (int j = threadIdx.x; j < N; j += blockDim.x) r[j] = b[j];
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            x[j] = make_double2(0.0, 0.0);
            p[j] = r[j];
        }
        __syncthreads();
        double rr = dotc(N, r, r, red).x;
        const double rhs = sqrt(rr);
        bool broke = false;
        int it = 0;
        double rel = rhs > 0.0 ? 1.0 : 0.0;
        while (it < max_iter && rel > tol) {
            if (normal) {
                lcu_matvec(n, L, coef, xm, zm, p, tmp, 0);
                lcu_matvec(n, L, coef, xm, zm, tmp, Ap, 1);
            } else {
                lcu_matvec(n, L, coef, xm, zm, p, Ap, 0);
            }
            const double pAp = dotc(N, p, Ap, red).x;
            if (!(pAp > 0.0)) {
                broke = true;
                break;
            }
            const double a = rr / pAp;
            for (int j = threadIdx.x; j < N; j += blockDim.x) {
                x[j].x += a * p[j].x;
                x[j].y += a * p[j].y;
                r[j].x -= a * Ap[j].x;
                r[j].y -= a * Ap[j].y;
            }
            __syncthreads();
            const double rr2 = dotc(N, r, r, red).x;
            const double bet = rr2 / rr;
            for (int j = threadIdx.x; j < N; j += blockDim.x) {
                p[j].x = r[j].x + bet * p[j].x;
                p[j].y = r[j].y + bet * p[j].y;
            }
            __syncthreads();
            rr = rr2;
            rel = rhs > 0.0 ? sqrt(rr) / rhs : 0.0;
            ++it;
        }
        if (!broke) {
            if (threadIdx.x == 0) {
                out[0] = it;
                out[1] = rel;
                out[2] = rel <= tol ? 1.0 : 0.0;
                out[3] = normal;
            }
            return;
        }
    }
    if (threadIdx.x == 0) {
        out[0] = max_iter;
        out[1] = INFINITY;
        out[2] = 0.0;
        out[3] = 1.0;
    }
}

// One Adam update of the active angles: element i is angle gmap[i], whose
// instance has the bias corrections c1[i] = 1 - beta1^t and c2[i] = 1 - beta2^t.
__global__ void k_adam(int count, const int* __restrict__ gmap, const double* __restrict__ g, double* alpha,
                       double* m, double* v, double lr, double b1, double b2, double eps, const double* __restrict__ c1,
                       const double* __restrict__ c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int k = gmap[i];
    const double gi = g[i];
    const double mi = b1 * m[k] + (1.0 - b1) * gi;
    const double vi = b2 * v[k] + (1.0 - b2) * gi * gi;
    m[k] = mi;
    v[k] = vi;
    alpha[k] -= lr * (mi / c1[i]) / (sqrt(vi / c2[i]) + eps);
}

// cudaMalloc'd block owned by one optimizer call.
struct DevBlock {
    char* p = nullptr;
    ~DevBlock() {
        if (p) cudaFree(p);
    }
};

}  // namespace

}  // namespace dvqls

using namespace dvqls;

extern "C" int dvqls_fidelity(dvqls_ctx* ctx, const dvqls_ansatz* an, const double* alpha, const double* xhat,
                              double* F) {
    DVQLS_NVTX("dvqls_fidelity");
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!an || !alpha || !xhat || !F) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "NULL argument");
    const int n = an->n, d = an->depth;
    if (n < 1 || n > DVQLS_MAX_QUBITS || d < 0) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "n = %d", n);
    if (an->kind != DVQLS_ANSATZ_RY_CZRING) return set_error(ctx, DVQLS_ERR_UNSUPPORTED, "ansatz kind");
    if (n > DVQLS_MAX_SMEM_QUBITS) {  // the state in HBM
        cudaSetDevice(ctx->device);
        return fidelity_hbm(ctx, n, d, alpha, xhat, F);
    }
    const int P = n * (d + 1);
    const long long N = 1LL << n;
    cudaSetDevice(ctx->device);
    Arena ar, pin;
    const size_t o_al = ar.reserve(size_t(P) * 8), p_al = pin.reserve(size_t(P) * 8);
    const size_t o_x = ar.reserve(size_t(N) * 16), p_x = pin.reserve(size_t(N) * 16);
    const size_t o_cs = ar.reserve(size_t(P) * 16);
    const size_t o_F = ar.reserve(8), p_F = pin.reserve(8);
    const size_t o_t = ar.reserve(sizeof(FidInst)), p_t = pin.reserve(sizeof(FidInst));
    int rc = ensure_workspace(ctx, ar.total());
    if (!rc) rc = ensure_pinned(ctx, pin.total());
    if (!rc) rc = pin_acquire(ctx);
    if (rc) return rc;
    FidInst I{};
    I.n = n;
    I.d = d;
    I.P = P;
    I.alpha = (const double*)stage_in(ctx, alpha, size_t(P) * 8, p_al, o_al);
    I.xhat = (const double2*)stage_in(ctx, xhat, size_t(N) * 16, p_x, o_x);
    I.cs = (double2*)(ctx->ws + o_cs);
    I.F = (double*)(ctx->ws + o_F);
    memcpy(ctx->pin + p_t, &I, sizeof I);
    DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ws + o_t, ctx->pin + p_t, sizeof I, cudaMemcpyHostToDevice, ctx->stream));
    const size_t smem = size_t(N + P) * 16;
    DVQLS_CUDA_TRY(ctx, allow_dynamic_smem((const void*)k_fidelity));
    k_fidelity<<<1, FT, smem, ctx->stream>>>((const FidInst*)(ctx->ws + o_t), ctx->d_status);
    DVQLS_CUDA_TRY(ctx, cudaGetLastError());
    rc = pin_release(ctx);
    std::vector<PendingOut> pend;
    if (!rc) rc = enqueue_out(ctx, F, I.F, 8, p_F, pend);
    if (!rc) rc = sync_and_check(ctx);
    if (rc) return rc;
    finish_out(ctx, pend);
    return DVQLS_OK;
}

// ------------------------------------------------ grid-wide CG (large N)
// The same conjugate gradients for one right-hand side of N >= CGM_MIN_N
// amplitudes, spread over the whole GPU: each step is a grid kernel (the
// matvec, the vector updates with per-block partial dot products) followed by
// a one-CTA kernel that adds the partials in block order (deterministic) and
// forms the CG scalars in device memory.  The host issues CGM_CHUNK
// iterations at a time and reads the scalars between chunks; every kernel
// returns at once after the stop flag is set.  Scalars: [0] r.r, [1] ||rhs||,
// [2] alpha, [3] beta, [4] stop, [5] iterations, [6] relative residual,
// [7] breakdown (p.Ap <= 0).
constexpr long long CGM_MIN_N = 4096;
constexpr int CGM_T = 256, CGM_CHUNK = 8;

__device__ double cgm_block_sum(double v, double* red) {  // valid in thread 0
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < CGM_T / 32; ++k) s += red[k];
    return s;
}

__global__ void __launch_bounds__(CGM_T) k_cgm_matvec(int n, int L, const double2* coef, const uint32_t* xm,
                                                      const uint32_t* zm, const double2* v, double2* y, int conj_coef,
                                                      const double* sc) {
    if (sc[4] != 0.0) return;
    const int N = 1 << n;
    for (int j = blockIdx.x * CGM_T + threadIdx.x; j < N; j += gridDim.x * CGM_T) {
        double yr = 0.0, yi = 0.0;
        for (int l = 0; l < L; ++l) {
            const uint32_t x = xm[l] & (N - 1), z = zm[l] & (N - 1);
            double2 c = coef[l];
            if (conj_coef) c.y = -c.y;
            double2 ph;
            switch (__popc(x & z) & 3) {
                case 0: ph = make_double2(1, 0); break;
                case 1: ph = make_double2(0, 1); break;
                case 2: ph = make_double2(-1, 0); break;
                default: ph = make_double2(0, -1); break;
            }
            const uint32_t src = uint32_t(j) ^ x;
            const double sg = (__popc(z & src) & 1) ? -1.0 : 1.0;
            const double2 a = v[src];
            const double cr = c.x * ph.x - c.y * ph.y, ci = c.x * ph.y + c.y * ph.x;
            yr += sg * (cr * a.x - ci * a.y);
            yi += sg * (cr * a.y + ci * a.x);
        }
        y[j] = make_double2(yr, yi);
    }
}

// r = b (copy_b) then x = 0, p = r, partial r.r; clears the flags.
__global__ void __launch_bounds__(CGM_T) k_cgm_start(int N, const double2* b, int copy_b, double2* x, double2* r,
                                                     double2* p, double* part) {
    __shared__ double red[CGM_T / 32];
    double s = 0.0;
    for (int j = blockIdx.x * CGM_T + threadIdx.x; j < N; j += gridDim.x * CGM_T) {
        const double2 v = copy_b ? b[j] : r[j];
        if (copy_b) r[j] = v;
        x[j] = make_double2(0.0, 0.0);
        p[j] = v;
        s += v.x * v.x + v.y * v.y;
    }
    s = cgm_block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_cgm_reset(double* sc) {
    for (int k = 0; k < 8; ++k) sc[k] = 0.0;
}

__global__ void __launch_bounds__(CGM_T) k_cgm_scalar_start(int G, const double* part, double* sc, double tol) {
    if (threadIdx.x != 0) return;
    double rr = 0.0;
    for (int k = 0; k < G; ++k) rr += part[k];
    sc[0] = rr;
    sc[1] = sqrt(rr);
    sc[5] = 0.0;
    sc[6] = sc[1] > 0.0 ? 1.0 : 0.0;
    sc[7] = 0.0;
    sc[4] = sc[6] <= tol ? 1.0 : 0.0;
}

__global__ void __launch_bounds__(CGM_T) k_cgm_dot(int N, const double2* a, const double2* b, double* part,
                                                   const double* sc) {  // partial Re(a^dag b)
    if (sc[4] != 0.0) return;
    __shared__ double red[CGM_T / 32];
    double s = 0.0;
    for (int j = blockIdx.x * CGM_T + threadIdx.x; j < N; j += gridDim.x * CGM_T) {
        const double2 x = a[j], y = b[j];
        s += x.x * y.x + x.y * y.y;
    }
    s = cgm_block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_cgm_alpha(int G, const double* part, double* sc) {
    if (sc[4] != 0.0) return;
    double pAp = 0.0;
    for (int k = 0; k < G; ++k) pAp += part[k];
    if (!(pAp > 0.0)) {
        sc[7] = 1.0;
        sc[4] = 1.0;
    } else {
        sc[2] = sc[0] / pAp;
    }
}

// x += alpha p, r -= alpha Ap, partial r.r
__global__ void __launch_bounds__(CGM_T) k_cgm_update(int N, double2* x, double2* r, const double2* p,
                                                      const double2* Ap, double* part, const double* sc) {
    if (sc[4] != 0.0) return;
    __shared__ double red[CGM_T / 32];
    const double a = sc[2];
    double s = 0.0;
    for (int j = blockIdx.x * CGM_T + threadIdx.x; j < N; j += gridDim.x * CGM_T) {
        double2 xv = x[j], rv = r[j];
        const double2 pv = p[j], av = Ap[j];
        xv.x += a * pv.x;
        xv.y += a * pv.y;
        rv.x -= a * av.x;
        rv.y -= a * av.y;
        x[j] = xv;
        r[j] = rv;
        s += rv.x * rv.x + rv.y * rv.y;
    }
    s = cgm_block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_cgm_beta(int G, const double* part, double* sc, double tol, int max_iter) {
    if (sc[4] != 0.0) return;
    double rr2 = 0.0;
    for (int k = 0; k < G; ++k) rr2 += part[k];
    sc[3] = rr2 / sc[0];
    sc[0] = rr2;
    sc[5] += 1.0;
    sc[6] = sc[1] > 0.0 ? sqrt(rr2) / sc[1] : 0.0;
    if (sc[6] <= tol || sc[5] >= max_iter) sc[4] = 1.0;
}

__global__ void __launch_bounds__(CGM_T) k_cgm_p(int N, const double2* r, double2* p, const double* sc) {
    if (sc[4] != 0.0) return;
    const double bet = sc[3];
    for (int j = blockIdx.x * CGM_T + threadIdx.x; j < N; j += gridDim.x * CGM_T) {
        const double2 rv = r[j], pv = p[j];
        p[j] = make_double2(rv.x + bet * pv.x, rv.y + bet * pv.y);
    }
}

// out as k_cg: iterations, relative residual, converged, normal equations used.
__global__ void k_cgm_finish(const double* sc, double* out, double tol, int normal, int max_iter) {
    const bool broke = sc[7] != 0.0;
    out[0] = broke ? max_iter : sc[5];
    out[1] = broke ? INFINITY : sc[6];
    out[2] = (!broke && sc[6] <= tol) ? 1.0 : 0.0;
    out[3] = normal;
}

static int cg_multi(dvqls_ctx* ctx, int n, int L, const double2* coef, const uint32_t* xm, const uint32_t* zm,
                    const double2* b, double2* x, double2* r, double2* p, double2* Ap, double2* tmp, double tol,
                    int max_iter, double* out, double* sc, double* part, int G) {
    const int N = 1 << n;
    cudaStream_t st = ctx->stream;
    for (int normal = 0; normal < 2; ++normal) {
        k_cgm_reset<<<1, 1, 0, st>>>(sc);
        if (normal) k_cgm_matvec<<<G, CGM_T, 0, st>>>(n, L, coef, xm, zm, b, r, 1, sc);  // r = A~^dag b
        k_cgm_start<<<G, CGM_T, 0, st>>>(N, b, normal ? 0 : 1, x, r, p, part);
        k_cgm_scalar_start<<<1, CGM_T, 0, st>>>(G, part, sc, tol);
        DVQLS_CUDA_TRY(ctx, cudaGetLastError());
        double h[8];
        for (;;) {
            for (int k = 0; k < CGM_CHUNK; ++k) {
                if (normal) {
                    k_cgm_matvec<<<G, CGM_T, 0, st>>>(n, L, coef, xm, zm, p, tmp, 0, sc);
                    k_cgm_matvec<<<G, CGM_T, 0, st>>>(n, L, coef, xm, zm, tmp, Ap, 1, sc);
                } else {
                    k_cgm_matvec<<<G, CGM_T, 0, st>>>(n, L, coef, xm, zm, p, Ap, 0, sc);
                }
                k_cgm_dot<<<G, CGM_T, 0, st>>>(N, p, Ap, part, sc);
                k_cgm_alpha<<<1, 1, 0, st>>>(G, part, sc);
                k_cgm_update<<<G, CGM_T, 0, st>>>(N, x, r, p, Ap, part, sc);
                k_cgm_beta<<<1, 1, 0, st>>>(G, part, sc, tol, max_iter);
                k_cgm_p<<<G, CGM_T, 0, st>>>(N, r, p, sc);
            }
            DVQLS_CUDA_TRY(ctx, cudaGetLastError());
            DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(h, sc, sizeof h, cudaMemcpyDeviceToHost, st));
            DVQLS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
            if (h[4] != 0.0) break;
        }
        if (h[7] == 0.0 || normal) {  // converged or out of iterations, or the normal equations broke down too
            k_cgm_finish<<<1, 1, 0, st>>>(sc, out, tol, normal, max_iter);
            DVQLS_CUDA_TRY(ctx, cudaGetLastError());
            return DVQLS_OK;
        }
    }
    return DVQLS_OK;
}

extern "C" int dvqls_lcu_solve_batched(dvqls_ctx* ctx, int n, const dvqls_lcu* lcu, int nrhs, const double* b,
                                       double tol, int max_iter, double* x, int* iters, double* rel_resid) {
    DVQLS_NVTX("dvqls_lcu_solve_batched");
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!lcu || !b || !x || lcu->L < 1 || !lcu->coef || !lcu->xmask || !lcu->zmask)
        return set_error(ctx, DVQLS_ERR_INVALID_ARG, "NULL argument or empty LCU");
    if (n < 1 || n > DVQLS_MAX_QUBITS) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "n = %d", n);
    if (nrhs < 1) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "nrhs = %d", nrhs);
    if (!(tol > 0.0) || max_iter < 1) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "tol > 0 and max_iter >= 1 needed");
    const int L = lcu->L;
    const long long N = 1LL << n;
    const size_t vec = size_t(nrhs) * size_t(N) * 16;  // one complex128 vector per right-hand side
    cudaSetDevice(ctx->device);
    Arena ar, pin;
    const size_t o_c = ar.reserve(size_t(L) * 16), p_c = pin.reserve(size_t(L) * 16);
    const size_t o_xm = ar.reserve(size_t(L) * 4), p_xm = pin.reserve(size_t(L) * 4);
    const size_t o_zm = ar.reserve(size_t(L) * 4), p_zm = pin.reserve(size_t(L) * 4);
    const size_t o_b = ar.reserve(vec), p_b = pin.reserve(vec);
    const size_t o_x = ar.reserve(vec), p_xo = pin.reserve(vec);
    const size_t o_r = ar.reserve(vec);
    const size_t o_p = ar.reserve(vec);
    const size_t o_ap = ar.reserve(vec);
    const size_t o_tmp = ar.reserve(vec);
    const size_t o_out = ar.reserve(size_t(nrhs) * 32);
    const bool multi = nrhs == 1 && N >= CGM_MIN_N;  // one large system: the grid-wide CG
    const int G = multi ? (int)std::min<long long>(N / CGM_T, (long long)ctx->num_sms * 8) : 0;
    const size_t o_sc = ar.reserve(64), o_part = ar.reserve(size_t(std::max(G, 1)) * 8);
    int rc = ensure_workspace(ctx, ar.total());
    if (!rc) rc = ensure_pinned(ctx, pin.total());
    if (!rc) rc = pin_acquire(ctx);
    if (rc) return rc;
    char* ws = ctx->ws;
    auto coef = (const double2*)stage_in(ctx, lcu->coef, size_t(L) * 16, p_c, o_c);
    auto xm = (const uint32_t*)stage_in(ctx, lcu->xmask, size_t(L) * 4, p_xm, o_xm);
    auto zm = (const uint32_t*)stage_in(ctx, lcu->zmask, size_t(L) * 4, p_zm, o_zm);
    auto bd = (const double2*)stage_in(ctx, b, vec, p_b, o_b);
    double* out = (double*)(ws + o_out);
    if (multi) {
        rc = cg_multi(ctx, n, L, coef, xm, zm, bd, (double2*)(ws + o_x), (double2*)(ws + o_r), (double2*)(ws + o_p),
                      (double2*)(ws + o_ap), (double2*)(ws + o_tmp), tol, max_iter, out, (double*)(ws + o_sc),
                      (double*)(ws + o_part), G);
        if (rc) return rc;
    } else {
        k_cg<<<nrhs, CGT, 0, ctx->stream>>>(n, L, coef, xm, zm, bd, (double2*)(ws + o_x), (double2*)(ws + o_r),
                                            (double2*)(ws + o_p), (double2*)(ws + o_ap), (double2*)(ws + o_tmp), tol,
                                            max_iter, out);
    }
    DVQLS_CUDA_TRY(ctx, cudaGetLastError());
    rc = pin_release(ctx);
    std::vector<PendingOut> pend;
    if (!rc) rc = enqueue_out(ctx, x, ws + o_x, vec, p_xo, pend);
    std::vector<double> res(size_t(nrhs) * 4, 0.0);
    if (!rc)
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(res.data(), out, res.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (!rc) rc = sync_and_check(ctx);
    if (rc) return rc;
    finish_out(ctx, pend);
    int failed = -1;
    for (int k = 0; k < nrhs; ++k) {
        if (iters) iters[k] = int(res[4 * k]);
        if (rel_resid) rel_resid[k] = res[4 * k + 1];
        if (res[4 * k + 2] != 1.0 && failed < 0) failed = k;
    }
    if (failed >= 0)
        return set_error(ctx, DVQLS_ERR_NUMERIC,
                         "solve %d did not reach tol (relative residual %.3g after %d iterations)", failed,
                         res[4 * failed + 1], int(res[4 * failed]));
    return DVQLS_OK;
}

extern "C" int dvqls_lcu_solve(dvqls_ctx* ctx, int n, const dvqls_lcu* lcu, const double* b, double tol, int max_iter,
                               double* x, int* iters, double* rel_resid) {
    DVQLS_NVTX("dvqls_lcu_solve");
    return dvqls_lcu_solve_batched(ctx, n, lcu, 1, b, tol, max_iter, x, iters, rel_resid);
}

// The optimizer loop; `state` (may be NULL: a fresh start) carries the Adam
// moments and update counts in and out.
static int optimize(dvqls_ctx* ctx, int count, const dvqls_instance* inst, const double* xhat, const dvqls_adam* opt,
                    dvqls_adam_state* state, double* alpha_out, dvqls_opt_result* results) {
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (count < 1 || !inst || !xhat || !opt || !alpha_out || !results)
        return set_error(ctx, DVQLS_ERR_INVALID_ARG, "NULL argument or count < 1");
    if (state && (!state->m || !state->v || !state->steps))
        return set_error(ctx, DVQLS_ERR_INVALID_ARG, "NULL moment or step array");
    if (!(opt->lr > 0.0) || opt->max_iter < 0 || !(opt->beta1 >= 0.0 && opt->beta1 < 1.0) ||
        !(opt->beta2 >= 0.0 && opt->beta2 < 1.0) || !(opt->eps > 0.0))
        return set_error(ctx, DVQLS_ERR_INVALID_ARG, "bad Adam settings");
    cudaSetDevice(ctx->device);
    std::vector<int> P(count), N(count), L(count);
    std::vector<long long> aoff(count + 1, 0), xoff(count + 1, 0), loff(count + 1, 0), boff(count + 1, 0);
    int nmax = 1;
    for (int i = 0; i < count; ++i) {
        const dvqls_instance& q = inst[i];
        if (q.ansatz.n < 1 || q.ansatz.n > DVQLS_MAX_SMEM_QUBITS || q.ansatz.depth < 0 || q.lcu.L < 1 || !q.alpha ||
            !q.b || !q.lcu.coef || !q.lcu.xmask || !q.lcu.zmask)
            return set_error(ctx, DVQLS_ERR_INVALID_ARG, "instance %d", i);
        P[i] = q.ansatz.n * (q.ansatz.depth + 1);
        N[i] = 1 << q.ansatz.n;
        L[i] = q.lcu.L;
        nmax = std::max(nmax, q.ansatz.n);
        aoff[i + 1] = aoff[i] + P[i];
        xoff[i + 1] = xoff[i] + N[i];
        loff[i + 1] = loff[i] + L[i];
    }
    const long long Pt = aoff[count], Nt = xoff[count], Lt = loff[count];
    // Optimizer-owned device memory (the context workspace is reused by the
    // cost pass and may move).
    Arena ar;
    const size_t o_al = ar.reserve(size_t(Pt) * 8), o_m = ar.reserve(size_t(Pt) * 8), o_v = ar.reserve(size_t(Pt) * 8);
    const size_t o_g = ar.reserve(size_t(Pt) * 8), o_gm = ar.reserve(size_t(Pt) * 4);
    const size_t o_c1 = ar.reserve(size_t(Pt) * 8), o_c2 = ar.reserve(size_t(Pt) * 8);
    const size_t o_x = ar.reserve(size_t(Nt) * 16), o_b = ar.reserve(size_t(Nt) * 16);
    const size_t o_c = ar.reserve(size_t(Lt) * 16), o_xm = ar.reserve(size_t(Lt) * 4), o_zm = ar.reserve(size_t(Lt) * 4);
    const size_t o_cost = ar.reserve(size_t(count) * 8), o_F = ar.reserve(size_t(count) * 8);
    const size_t o_cs = ar.reserve(size_t(Pt) * 16), o_ft = ar.reserve(sizeof(FidInst) * count);
    DevBlock blk;
    if (cudaMalloc(&blk.p, ar.total()) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, DVQLS_ERR_ALLOC, "optimizer state of %zu bytes", ar.total());
    }
    char* base = blk.p;
    double* alpha = (double*)(base + o_al);
    double* m = (double*)(base + o_m);
    double* v = (double*)(base + o_v);
    double* g = (double*)(base + o_g);
    int* gmap = (int*)(base + o_gm);
    double* costs = (double*)(base + o_cost);
    double* F = (double*)(base + o_F);
    double* c1d = (double*)(base + o_c1);
    double* c2d = (double*)(base + o_c2);
    // Adam state: zero moments and no updates, or the caller's checkpoint.  The
    // bias corrections 1 - beta^t are kept as products formed on the host in
    // the same order as a run that never stopped, so a resumed run continues
    // bit for bit.
    std::vector<long long> steps(count, 0);
    std::vector<double> p1(count, 1.0), p2(count, 1.0);  // beta1^t, beta2^t per instance
    if (state) {
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(m, state->m, size_t(Pt) * 8, cudaMemcpyDefault, ctx->stream));
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(v, state->v, size_t(Pt) * 8, cudaMemcpyDefault, ctx->stream));
        DVQLS_CUDA_TRY(ctx, cudaMemcpy(steps.data(), state->steps, size_t(count) * 8, cudaMemcpyDefault));
        for (int i = 0; i < count; ++i) {
            if (steps[i] < 0) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "instance %d: negative update count", i);
            for (long long t = 0; t < steps[i]; ++t) {
                p1[i] *= opt->beta1;
                p2[i] *= opt->beta2;
            }
        }
    } else {
        DVQLS_CUDA_TRY(ctx, cudaMemsetAsync(m, 0, size_t(Pt) * 8, ctx->stream));
        DVQLS_CUDA_TRY(ctx, cudaMemsetAsync(v, 0, size_t(Pt) * 8, ctx->stream));
    }
    std::vector<dvqls_instance> dinst(count);
    std::vector<FidInst> fid(count);
    for (int i = 0; i < count; ++i) {
        const dvqls_instance& q = inst[i];
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(alpha + aoff[i], q.alpha, size_t(P[i]) * 8, cudaMemcpyDefault, ctx->stream));
        double2* xd = (double2*)(base + o_x) + xoff[i];
        double2* bd = (double2*)(base + o_b) + xoff[i];
        double2* cd = (double2*)(base + o_c) + loff[i];
        uint32_t* xmd = (uint32_t*)(base + o_xm) + loff[i];
        uint32_t* zmd = (uint32_t*)(base + o_zm) + loff[i];
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(xd, xhat + 2 * xoff[i], size_t(N[i]) * 16, cudaMemcpyDefault, ctx->stream));
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(bd, q.b, size_t(N[i]) * 16, cudaMemcpyDefault, ctx->stream));
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(cd, q.lcu.coef, size_t(L[i]) * 16, cudaMemcpyDefault, ctx->stream));
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(xmd, q.lcu.xmask, size_t(L[i]) * 4, cudaMemcpyDefault, ctx->stream));
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(zmd, q.lcu.zmask, size_t(L[i]) * 4, cudaMemcpyDefault, ctx->stream));
        dinst[i] = q;
        dinst[i].alpha = alpha + aoff[i];
        dinst[i].b = (const double*)bd;
        dinst[i].lcu.coef = (const double*)cd;
        dinst[i].lcu.xmask = xmd;
        dinst[i].lcu.zmask = zmd;
        FidInst f{};
        f.n = q.ansatz.n;
        f.d = q.ansatz.depth;
        f.P = P[i];
        f.alpha = alpha + aoff[i];
        f.xhat = xd;
        f.cs = (double2*)(base + o_cs) + aoff[i];
        f.F = F + i;
        fid[i] = f;
        results[i].iters = 0;
        results[i].converged = 0;
        results[i].cost = NAN;
        results[i].fidelity = NAN;
    }
    const size_t fsmem = (size_t(1) << nmax) * 16 + size_t(*std::max_element(P.begin(), P.end())) * 16;
    DVQLS_CUDA_TRY(ctx, allow_dynamic_smem((const void*)k_fidelity));
    std::vector<int> active(count);
    for (int i = 0; i < count; ++i) active[i] = i;
    std::vector<double> hF(count), hC(count);
    std::vector<int> hmap;
    std::vector<dvqls_instance> ainst;
    std::vector<FidInst> afid;
    bool dirty = true;
    long long Pa = 0;
    std::vector<double> hc1, hc2;
    int rc = DVQLS_OK;
    for (int it = 0; it <= opt->max_iter && !active.empty(); ++it) {
        if (dirty) {
            ainst.clear();
            afid.clear();
            hmap.clear();
            for (int i : active) {
                ainst.push_back(dinst[i]);
                afid.push_back(fid[i]);
                for (int k = 0; k < P[i]; ++k) hmap.push_back(int(aoff[i] + k));
            }
            Pa = (long long)hmap.size();
            DVQLS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            DVQLS_CUDA_TRY(ctx, cudaMemcpy(gmap, hmap.data(), hmap.size() * 4, cudaMemcpyHostToDevice));
            DVQLS_CUDA_TRY(ctx, cudaMemcpy(base + o_ft, afid.data(), afid.size() * sizeof(FidInst), cudaMemcpyHostToDevice));
            dirty = false;
        }
        const int na = int(active.size());
        k_fidelity<<<na, FT, fsmem, ctx->stream>>>((const FidInst*)(base + o_ft), ctx->d_status);
        rc = run_batch(ctx, na, ainst.data(), opt->precision, true, costs, g, nullptr, nullptr, false);
        if (rc) return rc;
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(hF.data(), F, size_t(count) * 8, cudaMemcpyDeviceToHost, ctx->stream));
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(hC.data(), costs, size_t(na) * 8, cudaMemcpyDeviceToHost, ctx->stream));
        rc = sync_and_check(ctx);
        if (rc) return rc;
        std::vector<int> still;
        for (int a = 0; a < na; ++a) {
            const int i = active[a];
            results[i].iters = it;
            results[i].cost = hC[a];
            results[i].fidelity = hF[i];
            const double target = opt->targets ? opt->targets[i] : opt->target_fidelity;
            if (hF[i] >= target) results[i].converged = 1;
            else if (it < opt->max_iter) still.push_back(i);
        }
        if (still.size() != active.size()) {
            // Compact the gradient of the instances that go on: they are the
            // ones to update; rebuild the map to match run_batch's packing.
            std::vector<int> keep_map;
            std::vector<long long> goff(na + 1, 0);
            for (int a = 0; a < na; ++a) goff[a + 1] = goff[a] + P[active[a]];
            std::vector<double> hg(static_cast<size_t>(goff[na]));
            DVQLS_CUDA_TRY(ctx, cudaMemcpy(hg.data(), g, hg.size() * 8, cudaMemcpyDeviceToHost));
            std::vector<double> ng;
            for (int a = 0; a < na; ++a) {
                const int i = active[a];
                if (std::find(still.begin(), still.end(), i) == still.end()) continue;
                for (int k = 0; k < P[i]; ++k) {
                    ng.push_back(hg[size_t(goff[a] + k)]);
                    keep_map.push_back(int(aoff[i] + k));
                }
            }
            if (!ng.empty()) {
                DVQLS_CUDA_TRY(ctx, cudaMemcpy(g, ng.data(), ng.size() * 8, cudaMemcpyHostToDevice));
                DVQLS_CUDA_TRY(ctx, cudaMemcpy(gmap, keep_map.data(), keep_map.size() * 4, cudaMemcpyHostToDevice));
            }
            Pa = (long long)keep_map.size();
            active = still;
            dirty = true;
        }
        if (active.empty() || Pa == 0) break;
        hc1.clear();
        hc2.clear();
        for (int i : active) {  // the update of instance i is its (steps[i] + 1)-th
            p1[i] *= opt->beta1;
            p2[i] *= opt->beta2;
            ++steps[i];
            hc1.insert(hc1.end(), size_t(P[i]), 1.0 - p1[i]);
            hc2.insert(hc2.end(), size_t(P[i]), 1.0 - p2[i]);
        }
        DVQLS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        DVQLS_CUDA_TRY(ctx, cudaMemcpy(c1d, hc1.data(), hc1.size() * 8, cudaMemcpyHostToDevice));
        DVQLS_CUDA_TRY(ctx, cudaMemcpy(c2d, hc2.data(), hc2.size() * 8, cudaMemcpyHostToDevice));
        k_adam<<<ceil_div(Pa, 256), 256, 0, ctx->stream>>>(int(Pa), gmap, g, alpha, m, v, opt->lr, opt->beta1,
                                                          opt->beta2, opt->eps, c1d, c2d);
        DVQLS_CUDA_TRY(ctx, cudaGetLastError());
    }
    DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(alpha_out, alpha, size_t(Pt) * 8, cudaMemcpyDefault, ctx->stream));
    if (state) {
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(state->m, m, size_t(Pt) * 8, cudaMemcpyDefault, ctx->stream));
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(state->v, v, size_t(Pt) * 8, cudaMemcpyDefault, ctx->stream));
    }
    DVQLS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (state) DVQLS_CUDA_TRY(ctx, cudaMemcpy(state->steps, steps.data(), size_t(count) * 8, cudaMemcpyDefault));
    return DVQLS_OK;
}

extern "C" int dvqls_optimize(dvqls_ctx* ctx, int count, const dvqls_instance* inst, const double* xhat,
                              const dvqls_adam* opt, double* alpha_out, dvqls_opt_result* results) {
    DVQLS_NVTX("dvqls_optimize");
    return optimize(ctx, count, inst, xhat, opt, nullptr, alpha_out, results);
}

extern "C" int dvqls_optimize_resume(dvqls_ctx* ctx, int count, const dvqls_instance* inst, const double* xhat,
                                     const dvqls_adam* opt, dvqls_adam_state* state, double* alpha_out,
                                     dvqls_opt_result* results) {
    DVQLS_NVTX("dvqls_optimize_resume");
    if (ctx && !state) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "NULL optimizer state");
    return optimize(ctx, count, inst, xhat, opt, state, alpha_out, results);
}
