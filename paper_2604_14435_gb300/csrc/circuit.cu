// Per-circuit FP64 path: every Hadamard-test circuit of the global cost and
// its parameter-shift gradient is simulated on its own (n+1)-qubit state
// vector in complex128, gate by gate, and measured on the ancilla -- the
// execution model of Sec. 2.3 (one circuit per expectation value, real and
// imaginary parts from separate circuits, Sec. 2.2 after Eq. 4).  It is the
// comparison path for the batched term evaluation and its FP64 check.
//
// Circuits (ancilla = qubit n, system qubits 0..n-1):
//   beta_lm, part p:  H(anc); V(alpha_s); C-A_m; C-A_l; [S^dag(anc) if p];
//                     H(anc); <Z_anc> = Re / Im <psi|A_l A_m|psi>
//   delta_l, part p:  H(anc); C-V(alpha_s) (CRy, CCZ); C-A_l; C-U_b^dag;
//                     [S^dag(anc)]; H(anc); <Z_anc> = Re / Im <b|A_l|psi>
// C-A is one controlled X / Y / Z per qubit of the Pauli string.  U_b is
// H^(x)n when b = |+>^n and otherwise the phased Householder reflection
// e^{i phi}(I - 2 w w^dag / w^dag w), w = e^{i phi}|0> - b/||b||, which maps
// |0> to b/||b||.  One CTA runs one circuit with the state in shared memory.
#include <algorithm>

#include "internal.cuh"

namespace dvqls {

namespace {

constexpr int CT = 256;

struct CircInst {
    int n, d, L, P, S;
    long long circuits;  // S * (L*L + L) * 2
    const double2* coef;
    const uint32_t* xm;
    const uint32_t* zm;
    const double* alpha;
    const double2* b;
    double2* cs;    // 3P (cos, sin) of half angles: base, +pi/2, -pi/2
    double2* bhat;  // N: b / ||b||
    double2* w;     // N: Householder vector
    double* scal;   // [0] ||b||^2, [1] w^dag w, [2] re e^{i phi}, [3] im e^{i phi}, [4] b == |+>^n
    double* z;      // circuits results <Z_anc>, index (s * (L*L+L) + term) * 2 + part
    double* NsDs;   // 3S
    double* cost;
    double* grad;
    double2* beta;
    double2* delta;
};

__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, 0, code); }

__global__ void __launch_bounds__(CT) k_circ_prepare(CircInst I, int* status) {
    const int t = threadIdx.x;
    const long long N = 1LL << I.n;
    __shared__ double red[CT / 32];
    __shared__ int notplus;
    if (t == 0) notplus = 0;
    double acc = 0.0;
    for (long long j = t; j < N; j += CT) {
        const double2 v = I.b[j];
        if (!isfinite(v.x) || !isfinite(v.y)) set_status(status, DEV_NONFINITE_INPUT);
        acc += v.x * v.x + v.y * v.y;
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((t & 31) == 0) red[t >> 5] = acc;
    for (int l = t; l < I.L; l += CT)
        if (I.xm[l] >= N || I.zm[l] >= N) set_status(status, DEV_BAD_MASK);
    for (int a = t; a < I.P; a += CT) {
        const double al = I.alpha[a];
        if (!isfinite(al)) set_status(status, DEV_NONFINITE_INPUT);
        double s0, c0, s1, c1, s2, c2;
        sincos(0.5 * al, &s0, &c0);
        sincos(0.5 * (al + 0.5 * M_PI), &s1, &c1);
        sincos(0.5 * (al - 0.5 * M_PI), &s2, &c2);
        I.cs[a] = make_double2(c0, s0);
        I.cs[I.P + a] = make_double2(c1, s1);
        I.cs[2 * I.P + a] = make_double2(c2, s2);
    }
    __syncthreads();
    double bn2 = 0.0;
    for (int k = 0; k < CT / 32; ++k) bn2 += red[k];
    if (!(bn2 > 0.0) || !isfinite(bn2)) {
        if (t == 0) set_status(status, DEV_BAD_NORM);
        bn2 = 1.0;
    }
    const double inv = 1.0 / sqrt(bn2);
    const double2 b0 = I.b[0];
    const double a0 = sqrt(b0.x * b0.x + b0.y * b0.y);
    const double2 ph = a0 > 0.0 ? make_double2(b0.x / a0, b0.y / a0) : make_double2(1.0, 0.0);
    __syncthreads();
    double ww = 0.0;
    for (long long j = t; j < N; j += CT) {
        const double2 v = I.b[j];
        const double2 bh = make_double2(v.x * inv, v.y * inv);
        I.bhat[j] = bh;
        if (!(v.x == b0.x && v.y == 0.0 && b0.x > 0.0)) atomicOr(&notplus, 1);
        const double2 wj = make_double2((j == 0 ? ph.x : 0.0) - bh.x, (j == 0 ? ph.y : 0.0) - bh.y);
        I.w[j] = wj;
        ww += wj.x * wj.x + wj.y * wj.y;
    }
    for (int o = 16; o; o >>= 1) ww += __shfl_xor_sync(0xffffffffu, ww, o);
    __syncthreads();
    if ((t & 31) == 0) red[t >> 5] = ww;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int k = 0; k < CT / 32; ++k) s += red[k];
        I.scal[0] = bn2;
        I.scal[1] = s;
        I.scal[2] = ph.x;
        I.scal[3] = ph.y;
        I.scal[4] = notplus ? 0.0 : 1.0;
    }
}

// ------------------------------------------------------------- gates
struct Sim {
    double2* psi;
    int nq;  // n + 1
    int dim;
};

__device__ __forceinline__ int insert0(int p, int q) { return ((p >> q) << (q + 1)) | (p & ((1 << q) - 1)); }

__device__ void g_ry(const Sim& s, int q, double c, double sn, int cmask) {
    for (int p = threadIdx.x; p < s.dim / 2; p += CT) {
        const int i0 = insert0(p, q), i1 = i0 | (1 << q);
        if ((i0 & cmask) != cmask) continue;
        const double2 a = s.psi[i0], b = s.psi[i1];
        s.psi[i0] = make_double2(c * a.x - sn * b.x, c * a.y - sn * b.y);
        s.psi[i1] = make_double2(sn * a.x + c * b.x, sn * a.y + c * b.y);
    }
    __syncthreads();
}

__device__ void g_h(const Sim& s, int q, int cmask) {
    const double r = 0.70710678118654752440;
    for (int p = threadIdx.x; p < s.dim / 2; p += CT) {
        const int i0 = insert0(p, q), i1 = i0 | (1 << q);
        if ((i0 & cmask) != cmask) continue;
        const double2 a = s.psi[i0], b = s.psi[i1];
        s.psi[i0] = make_double2(r * (a.x + b.x), r * (a.y + b.y));
        s.psi[i1] = make_double2(r * (a.x - b.x), r * (a.y - b.y));
    }
    __syncthreads();
}

__device__ void g_flip(const Sim& s, int when) {  // Z, CZ, CCZ: sign flip where all bits of `when` are set
    for (int i = threadIdx.x; i < s.dim; i += CT)
        if ((i & when) == when) s.psi[i] = make_double2(-s.psi[i].x, -s.psi[i].y);
    __syncthreads();
}

__device__ void g_cx(const Sim& s, int ctrl, int q) {
    for (int p = threadIdx.x; p < s.dim / 2; p += CT) {
        const int i0 = insert0(p, q), i1 = i0 | (1 << q);
        if (!((i0 >> ctrl) & 1)) continue;
        const double2 a = s.psi[i0];
        s.psi[i0] = s.psi[i1];
        s.psi[i1] = a;
    }
    __syncthreads();
}

__device__ void g_cy(const Sim& s, int ctrl, int q) {  // Y: new0 = -i old1, new1 = i old0
    for (int p = threadIdx.x; p < s.dim / 2; p += CT) {
        const int i0 = insert0(p, q), i1 = i0 | (1 << q);
        if (!((i0 >> ctrl) & 1)) continue;
        const double2 a = s.psi[i0], b = s.psi[i1];
        s.psi[i0] = make_double2(b.y, -b.x);
        s.psi[i1] = make_double2(-a.y, a.x);
    }
    __syncthreads();
}

__device__ void g_sdg(const Sim& s, int q) {  // S^dag: amplitudes with bit q set times -i
    for (int i = threadIdx.x; i < s.dim; i += CT)
        if ((i >> q) & 1) s.psi[i] = make_double2(s.psi[i].y, -s.psi[i].x);
    __syncthreads();
}

__device__ void ansatz(const Sim& s, int n, int d, const double2* scs, int cmask) {
    for (int q = 0; q < n; ++q) g_ry(s, q, scs[q].x, scs[q].y, cmask);
    for (int layer = 1; layer <= d; ++layer) {
        for (int q = 0; q + 1 < n; ++q) g_flip(s, cmask | (1 << q) | (1 << (q + 1)));
        if (n >= 3) g_flip(s, cmask | (1 << (n - 1)) | 1);
        for (int q = 0; q < n; ++q) g_ry(s, q, scs[layer * n + q].x, scs[layer * n + q].y, cmask);
    }
}

__device__ void c_pauli(const Sim& s, int n, int anc, uint32_t x, uint32_t z) {
    for (int q = 0; q < n; ++q) {
        const int xb = (x >> q) & 1, zb = (z >> q) & 1;
        if (xb && zb) g_cy(s, anc, q);
        else if (xb) g_cx(s, anc, q);
        else if (zb) g_flip(s, (1 << anc) | (1 << q));
    }
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < CT / 32; ++k) s += red[k];
    __syncthreads();
    return s;  // every thread
}

// Controlled U_b^dag on the ancilla = 1 half (anc is the top bit).
__device__ void c_ub_dag(const Sim& s, const CircInst& I, int n, double* red) {
    const int N = 1 << n;
    double2* v = s.psi + N;
    if (I.scal[4] != 0.0) {
        for (int q = 0; q < n; ++q) g_h(s, q, 1 << n);
        return;
    }
    const double ww = I.scal[1];
    const double2 ph = make_double2(I.scal[2], I.scal[3]);
    if (ww > 0.0) {
        double ar = 0.0, ai = 0.0;  // w^dag v
        for (int j = threadIdx.x; j < N; j += CT) {
            const double2 wj = I.w[j], vj = v[j];
            ar += wj.x * vj.x + wj.y * vj.y;
            ai += wj.x * vj.y - wj.y * vj.x;
        }
        ar = block_sum(ar, red);
        ai = block_sum(ai, red);
        const double fr = 2.0 * ar / ww, fi = 2.0 * ai / ww;
        for (int j = threadIdx.x; j < N; j += CT) {
            const double2 wj = I.w[j];
            v[j].x -= fr * wj.x - fi * wj.y;
            v[j].y -= fr * wj.y + fi * wj.x;
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < N; j += CT) {  // times e^{-i phi}
        const double2 a = v[j];
        v[j] = make_double2(ph.x * a.x + ph.y * a.y, ph.x * a.y - ph.y * a.x);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(CT) k_circuits(CircInst I) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[CT / 32];
    const int n = I.n, anc = n;
    double2* scs = reinterpret_cast<double2*>(smem);  // P
    Sim sim{scs + I.P, n + 1, 1 << (n + 1)};
    const long long per_shift = ((long long)I.L * I.L + I.L) * 2;
    for (long long c = blockIdx.x; c < I.circuits; c += gridDim.x) {
        const int s = int(c / per_shift);
        const long long r = c % per_shift;
        const long long term = r >> 1;
        const int part = int(r & 1);
        int k = -1, which = 0;
        if (s > 0) {
            k = (s - 1) >> 1;
            which = ((s - 1) & 1) ? 2 : 1;
        }
        for (int a = threadIdx.x; a < I.P; a += CT) scs[a] = I.cs[(a == k ? which : 0) * I.P + a];
        for (int i = threadIdx.x; i < sim.dim; i += CT) sim.psi[i] = make_double2(i == 0 ? 1.0 : 0.0, 0.0);
        __syncthreads();
        g_h(sim, anc, 0);
        if (term < (long long)I.L * I.L) {
            const int l = int(term / I.L), m = int(term % I.L);
            ansatz(sim, n, I.d, scs, 0);
            c_pauli(sim, n, anc, I.xm[m] & ((1u << n) - 1), I.zm[m] & ((1u << n) - 1));
            c_pauli(sim, n, anc, I.xm[l] & ((1u << n) - 1), I.zm[l] & ((1u << n) - 1));
        } else {
            const int l = int(term - (long long)I.L * I.L);
            ansatz(sim, n, I.d, scs, 1 << anc);
            c_pauli(sim, n, anc, I.xm[l] & ((1u << n) - 1), I.zm[l] & ((1u << n) - 1));
            c_ub_dag(sim, I, n, red);
        }
        if (part) g_sdg(sim, anc);
        g_h(sim, anc, 0);
        double p = 0.0;
        for (int i = threadIdx.x; i < sim.dim; i += CT) {
            const double2 a = sim.psi[i];
            const double pr = a.x * a.x + a.y * a.y;
            p += (i >> anc) & 1 ? -pr : pr;
        }
        p = block_sum(p, red);
        if (threadIdx.x == 0) I.z[c] = p;
    }
}

__global__ void __launch_bounds__(CT) k_circ_combine(CircInst I, int* status) {
    const int t = threadIdx.x, L = I.L;
    const long long LL = (long long)L * L, per = LL + L;
    for (int s = t; s < I.S; s += CT) {
        const double* zs = I.z + (long long)s * per * 2;
        double Dr = 0.0, Di = 0.0, Tr = 0.0, Ti = 0.0;
        for (long long e = 0; e < LL; ++e) {
            const int l = int(e / L), m = int(e % L);
            const double br = zs[2 * e], bi = zs[2 * e + 1];
            const double2 cl = I.coef[l], cm = I.coef[m];
            const double wr = cl.x * cm.x + cl.y * cm.y, wi = cl.x * cm.y - cl.y * cm.x;  // conj(c_l) c_m
            Dr += wr * br - wi * bi;
            Di += wr * bi + wi * br;
        }
        for (int l = 0; l < L; ++l) {
            const double dr = zs[2 * (LL + l)], di = zs[2 * (LL + l) + 1];
            const double2 c = I.coef[l];
            Tr += c.x * dr - c.y * di;
            Ti += c.x * di + c.y * dr;
        }
        I.NsDs[3 * s] = Tr * Tr + Ti * Ti;
        I.NsDs[3 * s + 1] = Dr;
        I.NsDs[3 * s + 2] = Di;
    }
    __syncthreads();
    const double N0 = I.NsDs[0], D0 = I.NsDs[1];
    if (t == 0) {
        if (!(D0 > 0.0) || !isfinite(D0) || !isfinite(N0)) set_status(status, DEV_BAD_DENOMINATOR);
        *I.cost = 1.0 - N0 / D0;
    }
    if (I.grad)
        for (int k = t; k < I.P; k += CT) {
            const double dN = 0.5 * (I.NsDs[3 * (2 * k + 1)] - I.NsDs[3 * (2 * k + 2)]);
            const double dD = 0.5 * (I.NsDs[3 * (2 * k + 1) + 1] - I.NsDs[3 * (2 * k + 2) + 1]);
            I.grad[k] = -(dN * D0 - N0 * dD) / (D0 * D0);
        }
    if (I.beta)
        for (long long e = t; e < LL; e += CT) I.beta[e] = make_double2(I.z[2 * e], I.z[2 * e + 1]);
    if (I.delta)
        for (int l = t; l < L; l += CT) I.delta[l] = make_double2(I.z[2 * (LL + l)], I.z[2 * (LL + l) + 1]);
}

}  // namespace

int run_circuits(dvqls_ctx* ctx, const dvqls_ansatz* an, const double* alpha, const dvqls_lcu* lcu,
                 const double* b, bool want_grad, double* cost, double* grad, double* beta_out,
                 double* delta_out) {
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!an || !lcu || !cost) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "NULL ansatz, lcu or cost");
    const int n = an->n, d = an->depth, L = lcu->L;
    if (n < 1 || n > DVQLS_MAX_QUBITS || d < 0) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "n = %d, depth = %d", n, d);
    if (n + 1 > 13) return set_error(ctx, DVQLS_ERR_UNSUPPORTED, "circuit path keeps n+1 <= 13 qubits in shared memory");
    if (an->kind != DVQLS_ANSATZ_RY_CZRING) return set_error(ctx, DVQLS_ERR_UNSUPPORTED, "ansatz kind %d", an->kind);
    if (L < 1 || !lcu->coef || !lcu->xmask || !lcu->zmask || !alpha || !b)
        return set_error(ctx, DVQLS_ERR_INVALID_ARG, "empty LCU or NULL input");
    if (want_grad && !grad) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "grad is NULL");
    const int P = n * (d + 1);
    if (P > 1024) return set_error(ctx, DVQLS_ERR_UNSUPPORTED, "%d angles", P);
    const int S = want_grad ? 2 * P + 1 : 1;
    const long long N = 1LL << n, LL = (long long)L * L;
    cudaSetDevice(ctx->device);

    Arena ar, pin;
    const size_t o_coef = ar.reserve(size_t(L) * 16), p_coef = pin.reserve(size_t(L) * 16);
    const size_t o_xm = ar.reserve(size_t(L) * 4), p_xm = pin.reserve(size_t(L) * 4);
    const size_t o_zm = ar.reserve(size_t(L) * 4), p_zm = pin.reserve(size_t(L) * 4);
    const size_t o_al = ar.reserve(size_t(P) * 8), p_al = pin.reserve(size_t(P) * 8);
    const size_t o_b = ar.reserve(size_t(N) * 16), p_b = pin.reserve(size_t(N) * 16);
    const size_t o_cs = ar.reserve(size_t(3) * P * 16);
    const size_t o_bh = ar.reserve(size_t(N) * 16);
    const size_t o_w = ar.reserve(size_t(N) * 16);
    const size_t o_sc = ar.reserve(64);
    const size_t o_z = ar.reserve(size_t(S) * (LL + L) * 2 * 8);
    const size_t o_ns = ar.reserve(size_t(S) * 24);
    const size_t o_cost = ar.reserve(8), p_cost = pin.reserve(8);
    const size_t o_grad = ar.reserve(size_t(P) * 8), p_grad = pin.reserve(size_t(P) * 8);
    const size_t o_beta = ar.reserve(size_t(LL) * 16), p_beta = pin.reserve(size_t(LL) * 16);
    const size_t o_delta = ar.reserve(size_t(L) * 16), p_delta = pin.reserve(size_t(L) * 16);
    int rc = ensure_workspace(ctx, ar.total());
    if (!rc) rc = ensure_pinned(ctx, pin.total());
    if (!rc) rc = pin_acquire(ctx);
    if (rc) return rc;
    char* ws = ctx->ws;
    CircInst I{};
    I.n = n;
    I.d = d;
    I.L = L;
    I.P = P;
    I.S = S;
    I.circuits = (long long)S * (LL + L) * 2;
    I.coef = (const double2*)stage_in(ctx, lcu->coef, size_t(L) * 16, p_coef, o_coef);
    I.xm = (const uint32_t*)stage_in(ctx, lcu->xmask, size_t(L) * 4, p_xm, o_xm);
    I.zm = (const uint32_t*)stage_in(ctx, lcu->zmask, size_t(L) * 4, p_zm, o_zm);
    I.alpha = (const double*)stage_in(ctx, alpha, size_t(P) * 8, p_al, o_al);
    I.b = (const double2*)stage_in(ctx, b, size_t(N) * 16, p_b, o_b);
    I.cs = (double2*)(ws + o_cs);
    I.bhat = (double2*)(ws + o_bh);
    I.w = (double2*)(ws + o_w);
    I.scal = (double*)(ws + o_sc);
    I.z = (double*)(ws + o_z);
    I.NsDs = (double*)(ws + o_ns);
    I.cost = (double*)(ws + o_cost);
    I.grad = want_grad ? (double*)(ws + o_grad) : nullptr;
    I.beta = beta_out ? (double2*)(ws + o_beta) : nullptr;
    I.delta = delta_out ? (double2*)(ws + o_delta) : nullptr;
    // Householder data use b / ||b||; keep the normalised copy for the circuits.
    k_circ_prepare<<<1, CT, 0, ctx->stream>>>(I, ctx->d_status);
    I.b = I.bhat;
    const size_t smem = size_t(P) * 16 + (size_t(2) << n) * 16;
    DVQLS_CUDA_TRY(ctx, allow_dynamic_smem((const void*)k_circuits));
    int bps = 0;
    DVQLS_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_circuits, CT, smem));
    if (bps < 1) return set_error(ctx, DVQLS_ERR_UNSUPPORTED, "circuit kernel does not fit");
    const long long grid = std::min<long long>(I.circuits, (long long)ctx->num_sms * bps);
    prof_begin(ctx, 1);
    k_circuits<<<int(grid), CT, smem, ctx->stream>>>(I);
    prof_end(ctx);
    prof_begin(ctx, 2);
    k_circ_combine<<<1, CT, 0, ctx->stream>>>(I, ctx->d_status);
    prof_end(ctx);
    DVQLS_CUDA_TRY(ctx, cudaGetLastError());
    rc = pin_release(ctx);
    if (rc) return rc;
    std::vector<PendingOut> pend;
    rc = enqueue_out(ctx, cost, I.cost, 8, p_cost, pend);
    if (!rc && want_grad) rc = enqueue_out(ctx, grad, I.grad, size_t(P) * 8, p_grad, pend);
    if (!rc && beta_out) rc = enqueue_out(ctx, beta_out, I.beta, size_t(LL) * 16, p_beta, pend);
    if (!rc && delta_out) rc = enqueue_out(ctx, delta_out, I.delta, size_t(L) * 16, p_delta, pend);
    if (rc) return rc;
    rc = sync_and_check(ctx);
    if (rc) return rc;
    finish_out(ctx, pend);
    return DVQLS_OK;
}

}  // namespace dvqls

extern "C" int dvqls_circuit_cost_grad_fp64(dvqls_ctx* ctx, const dvqls_ansatz* ansatz, const double* alpha,
                                            const dvqls_lcu* lcu, const double* b, double* cost, double* grad,
                                            double* beta, double* delta) {
    DVQLS_NVTX("dvqls_circuit_cost_grad_fp64");
    return dvqls::run_circuits(ctx, ansatz, alpha, lcu, b, true, cost, grad, beta, delta);
}
