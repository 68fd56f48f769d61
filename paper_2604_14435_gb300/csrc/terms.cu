// Batched Hadamard-test term evaluation: cost and parameter-shift gradient
// of the VQLS global cost (Eq. 1 with A = sum_l c_l A_l, Eq. 3), i.e. the
// work of Stages I-III of Sec. 2.3 done as one persistent device pass.
//
// Work items.  For instance i with P angles there are S = 2P+1 shifted angle
// vectors (s = 0: alpha; s = 2k+1: alpha + pi/2 e_k; s = 2k+2: alpha - pi/2
// e_k).  With T = ceil(L/64) term tiles, item (s, tl, tm, ks) is one CTA's
// share: the 64 x 64 block (tl, tm) of
//     G~_lm = sum_j conj(phi_l[j]) phi_m[j],  phi_l[j] = (-1)^popc(z_l & (j^x_l)) psi_s[j ^ x_l]
// over the amplitude range ks of K-split `ks`, where psi_s = V(alpha_s)|0>.
// This is beta_lm = <psi|A_l^dag A_m|psi> up to the exact phase
// conj(i^popc(x_l&z_l)) i^popc(x_m&z_m) (the masked permute-and-sign
// reduction).  Diagonal tiles also reduce delta~_l = sum_j conj(b_j) phi_l[j].
//
// Each CTA builds psi_s in shared memory (n <= 12), then streams chunks of
// 32 amplitudes: it materialises phi_l / phi_m for the chunk in shared memory
// and every thread accumulates a 4 x 4 block of complex products in
// registers (4 FMA per complex product).  The tile's contribution to
// D_s = sum_lm conj(c_l) c_m beta_lm and T_s = sum_l c_l delta_l is formed in
// FP64 from the FP32 (or FP64) tile and written to a per-item slot; the
// combine kernel adds the slots in a fixed order, so results do not depend
// on scheduling.  C = 1 - N_0/D_0 with N_s = |T_s|^2/||b||^2 and
// dC/dalpha_k = -(N'_k D_0 - N_0 D'_k)/D_0^2 (parameter-shift rule).
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "internal.cuh"
#include "state.cuh"

namespace dvqls {

constexpr int TT = 64;    // term tile edge (l and m)
constexpr int KG = 2;     // K-groups per CTA (each sums half of every chunk)
constexpr int KSLOT = 144; // task slots per K-group (136 used on diagonal tiles, 128 off-diagonal)
constexpr int NT = KG * KSLOT;  // threads per CTA (9 warps)
constexpr int JC = 64;    // amplitudes per chunk (a power of two)
constexpr int MAX_ANGLES = 1024;

struct Inst {
    int n, d, L, P, S, T, ks;
    int F;      // term flavors per shift: 1 (global cost) or n + 1 (local cost)
    int s0;     // first shift of the pass: its shift s selects the angles of shift s0 + s (0 unless split)
    int local;  // 1: local cost C_L (b = |+>^n), 0: global cost
    int items;
    long long item_base;
    const double2* coef;
    const uint32_t* xm;
    const uint32_t* zm;
    const double* alpha;
    const double2* b;
    double2* ctil;   // L: c_l i^popc(x_l & z_l)
    double2* w;      // L*L: conj(ctil_l) ctil_m
    float4* wf;      // L*L or null: w as float pairs (Re hi, Re lo, Im hi, Im lo)
    float4* cf;      // L or null: ctil as float pairs
    void* bop;       // tensor-core tiles: the b rows of the B operand, TC_BOP_STAGE bytes per stage, or null
    void* wht;       // Walsh-Hadamard classes: the class table (WHT_TABLE_BYTES), or null
    float2* bf;      // Walsh-Hadamard classes: b in FP32, or null
    double2* cs;     // 3P: (cos, sin) of half angles: base, +pi/2, -pi/2
    double* bn2;     // ||b||^2
    double2* Dpart;  // S*T*T*ks
    double2* Tpart;  // S*T*ks
    void* Gpart;     // ks*L*L (shift 0 only; null when beta is not requested)
    void* dpart;     // ks*L   (shift 0 only; null when delta is not requested)
    double* NsDs;    // 3S: N_s, Re D_s, Im D_s
    void* states;    // n > 12: the S shifted states in HBM (S x N), else null
    void* tcst;      // tensor-core pass, n <= 12: the S shifted states as packed FP16 pairs (S x N words), else null
    double* cost;
    double* grad;    // P or null
    double2* beta;   // L*L or null
    double2* delta;  // L or null
};

struct GraphCacheEntry {
    cudaGraphExec_t exec = nullptr;
    std::vector<char> key;  // byte image of the launch plan it was captured for
};

void release_graph_cache(dvqls_ctx* ctx) {
    if (ctx->graph) {
        if (ctx->graph->exec) cudaGraphExecDestroy(ctx->graph->exec);
        delete ctx->graph;
        ctx->graph = nullptr;
    }
}

__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, 0, code); }

// ---------------------------------------------------------------- prepare
// A complex FP64 value as two float pairs: x = hi + lo with hi = RN_f32(x).
__device__ __forceinline__ float4 split_ff(double2 v) {
    const float xh = (float)v.x, yh = (float)v.y;
    return make_float4(xh, (float)(v.x - (double)xh), yh, (float)(v.y - (double)yh));
}

// c~_l = c_l i^popc(x_l & z_l): the phase of sigma(x, z) as an exact swap / sign.
__device__ __forceinline__ double2 ctil_of(const Inst& I, int l) {
    const double2 c = I.coef[l];
    switch (__popc(I.xm[l] & I.zm[l]) & 3) {
        case 0: return c;
        case 1: return make_double2(-c.y, c.x);
        case 2: return make_double2(-c.x, -c.y);
        default: return make_double2(c.y, -c.x);
    }
}

// Per-instance tables of a pass (Sec. 2.3 Stage I inputs).  Grid (instances,
// parts): part 0 checks the inputs, forms ||b||^2 and c~; every part takes its
// share of the shift angle tables and of the L^2 weights w_lm = conj(c~_l) c~_m.
// Programmatic dependent launch: the kernels of a pass after the first are
// launched so that their CTAs may start while the previous kernel finishes;
// each waits for the previous grid's completion (and its memory) before its
// first dependent access, and lets the next kernel start once all its CTAs
// are running.  Launched without the attribute, both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }


// ------------------------------------------------------------ term tiles
template <typename R>
__device__ __forceinline__ void load4(const typename V2<R>::t* p, typename V2<R>::t (&v)[4]);
template <>
__device__ __forceinline__ void load4<float>(const float2* p, float2 (&v)[4]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0];
    const float4 b = reinterpret_cast<const float4*>(p)[1];
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y);
    v[3] = make_float2(b.z, b.w);
}
template <>
__device__ __forceinline__ void load4<double>(const double2* p, double2 (&v)[4]) {
    v[0] = p[0];
    v[1] = p[1];
    v[2] = p[2];
    v[3] = p[3];
}

__device__ __forceinline__ double2 block_sum2(double2 v, double2* red) {
    for (int o = 16; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double2 s = make_double2(0.0, 0.0);
    if (threadIdx.x == 0)
        for (int k = 0; k < NT / 32; ++k) {
            s.x += red[k].x;
            s.y += red[k].y;
        }
    return s;  // valid in thread 0
}

// One work item (see the file comment).  Item u of a shift: u < T is the
// diagonal tile (u, u); u >= T is half h of the off-diagonal tile pair
// (tl < tm) number (u - T) / 2.  Only blocks with l <= m are computed:
// beta_ml = conj(beta_lm) exactly, so the pair contributes 2 Re(w_lm G~_lm) to
// D_s and nothing to its imaginary part.  Threads: two K-groups of KSLOT task
// slots; each active slot owns one 4 x 4 block of complex products and
// accumulates it over its K-group's half of every chunk, in registers.
__device__ __forceinline__ double2 block_sum2_n(double2 v, double2* red, int nthreads) {
    for (int o = 16; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double2 s = make_double2(0.0, 0.0);
    if (threadIdx.x == 0)
        for (int k = 0; k < nthreads / 32; ++k) {
            s.x += red[k].x;
            s.y += red[k].y;
        }
    return s;  // valid in thread 0
}

// Float-float accumulation: (S, E) += p exactly (two-sum), and
// (S, E) += (wh + wl) g with wh g exact by FMA (two-product).
__device__ __forceinline__ void ff_add(float& S, float& E, float p) {
    const float s = S + p, bv = s - S;
    E += (S - (s - bv)) + (p - bv);
    S = s;
}
__device__ __forceinline__ void ff_mac(float& S, float& E, float wh, float wl, float g) {
    const float p = wh * g;
    const float err = fmaf(wl, g, fmaf(wh, g, -p));
    ff_add(S, E, p);
    E += err;
}
__device__ __forceinline__ void ff_warp_sum(float& S, float& E) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, S, o), e2 = __shfl_xor_sync(0xffffffffu, E, o);
        ff_add(S, E, s2);
        E += e2;
    }
}

// Sum over the block of a float-float pair per thread: exact pairs within
// warps, FP64 across the warps.  Valid in thread 0.
__device__ __forceinline__ double block_sum_ff(float S, float E, double* red) {
    ff_warp_sum(S, E);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)S + (double)E;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += red[k];
    return r;
}

template <typename R>
__device__ __forceinline__ void load4r(const R* p, R (&v)[4]);
template <>
__device__ __forceinline__ void load4r<float>(const float* p, float (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
}
template <>
__device__ __forceinline__ void load4r<double>(const double* p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}
template <typename R>
__device__ __forceinline__ void store4r(R* p, const R (&v)[4]);
template <>
__device__ __forceinline__ void store4r<float>(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void store4r<double>(double* p, const double (&v)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// The Ry + CZ-ring state is real, so with the phase i^popc(x & z) in c~_l
// every phi_l[j] = (-1)^popc(z_l & (j ^ x_l)) psi[j ^ x_l] is real and the
// Gram G~ is real symmetric: one FMA per product, and delta_l = sum_j
// conj(b_j) phi_l[j] takes Re b and Im b separately.
template <typename R>
__device__ void process_item(const Inst& I, int local, unsigned char* smem, uint32_t* smask, double2* red) {
    using R2 = typename V2<R>::t;
    const int n = I.n, N = 1 << n, L = I.L, T = I.T, ks = I.ks, t = threadIdx.x;
    const int ksi = local % ks;
    const int rest = local / ks;
    const int u = rest % (T * T), rest2 = rest / (T * T);
    const int f = rest2 % I.F, s = rest2 / I.F;  // flavor 0: beta; j + 1: gamma^j (X_j on the m side)
    int tl, tm, half = 0;
    const bool diag = u < T;
    if (diag) {
        tl = tm = u;
    } else {
        const int v = u - T, pr = v >> 1;
        half = v & 1;
        int a = 0, rem = pr;
        while (rem >= T - 1 - a) {
            rem -= T - 1 - a;
            ++a;
        }
        tl = a;
        tm = a + 1 + rem;
    }
    const int kper = N / ks, kbeg = ksi * kper, kend = kbeg + kper;

    // n <= 12: psi_s is built in shared memory; n > 12: it was built in HBM
    // by the state passes (real) and is read from there (L2-resident while in
    // use).
    R* psi_smem = reinterpret_cast<R*>(smem);
    const R* psi_g = I.states ? reinterpret_cast<const R*>(I.states) + (size_t)s * N : nullptr;
    R* Phl = psi_smem + (I.states ? 0 : ((N + 3) & ~3));  // 16-byte aligned for the vector loads
    R* Phm = Phl + JC * TT;
    R2* bch = reinterpret_cast<R2*>(Phm + JC * TT);
    R2* scs = bch + JC;  // P entries (only used during the state build)
    uint32_t* sxl = smask;
    uint32_t* szl = smask + TT;
    uint32_t* sxm = smask + 2 * TT;
    uint32_t* szm = smask + 3 * TT;
    const int mofs = diag ? 0 : half * (TT / 2);  // first m column of this item within tile tm
    const int mcols = diag ? TT : TT / 2;
    const bool same = diag && f == 0;                     // phi_m is phi_l
    const bool want_delta = diag && f == 0 && !I.local;   // delta~ rows (global cost only)
    const uint32_t xflip = f > 0 ? (1u << (f - 1)) : 0u;  // X_j A_m = sigma(x_m ^ e_j, z_m)
    if (t < TT) {
        const int l = tl * TT + t;
        sxl[t] = l < L ? I.xm[l] : 0u;
        szl[t] = l < L ? I.zm[l] : 0u;
        const int m = tm * TT + t;
        sxm[t] = m < L ? (I.xm[m] ^ xflip) : 0u;
        szm[t] = m < L ? I.zm[m] : 0u;
    }
    if (I.states) __syncthreads();
    else build_state_real<R>(psi_smem, scs, I.n, I.d, I.P, I.cs, s + I.s0, t, NT, 0, (R)1);

    // Task of this thread: block (a, b) = rows 4a.., columns 4b.. of the tile.
    const int g = t / KSLOT, slot = t % KSLOT;
    const int ntask = diag ? 136 : 128;
    const bool active = slot < ntask;
    int ba = 0, bb = 0;
    if (active) {
        if (diag) {  // upper-triangle blocks (a <= b) of the 16 x 16 block grid, row-major
            int rem = slot;
            while (rem >= 16 - ba) {
                rem -= 16 - ba;
                ++ba;
            }
            bb = ba + rem;
        } else {
            ba = slot >> 3;
            bb = half * 8 + (slot & 7);
        }
    }
    const R* Pm = same ? Phl : Phm;
    R acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (R)0;
    R2 dacc;
    dacc.x = dacc.y = (R)0;
    const int lcount = min(TT, L - tl * TT), mcount = min(TT, L - tm * TT);

    for (int j0 = kbeg; j0 < kend; j0 += JC) {
        // phi chunk rows jj = 0..JC-1, stored with the 4-term groups
        // XOR-swizzled by the row index (group q of row jj at 4 (q ^ (jj & 15))).
        // A thread fills one group of one row; a warp takes 32 consecutive
        // rows of one group, so each of its four gathers reads one aligned
        // 32-amplitude block of psi (permuted by the low bits of the term's
        // x), and its 16-byte stores fall in distinct bank groups.
        for (int e = t; e < JC * (TT / 4); e += NT) {
            const int jj = e & (JC - 1), q = e / JC, j = j0 + jj;
            R v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int l = 4 * q + k;
                v[k] = (R)0;
                if (j < kend && l < lcount) {
                    const int src = (j ^ int(sxl[l])) & (N - 1);  // masks >= 2^n are reported, never followed
                    v[k] = psi_g ? psi_g[src] : psi_smem[src];
                    if (__popc(szl[l] & uint32_t(src)) & 1) v[k] = -v[k];
                }
            }
            store4r<R>(Phl + jj * TT + ((4 * q) ^ ((jj & 15) << 2)), v);
        }
        if (!same) {
            for (int e = t; e < JC * (mcols / 4); e += NT) {
                const int jj = e & (JC - 1), q = mofs / 4 + e / JC, j = j0 + jj;
                R v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int m = 4 * q + k;
                    v[k] = (R)0;
                    if (j < kend && m < mcount) {
                        const int src = (j ^ int(sxm[m])) & (N - 1);
                        v[k] = psi_g ? psi_g[src] : psi_smem[src];
                        if (__popc(szm[m] & uint32_t(src)) & 1) v[k] = -v[k];
                    }
                }
                store4r<R>(Phm + jj * TT + ((4 * q) ^ ((jj & 15) << 2)), v);
            }
        }
        if (want_delta && t < JC) {
            R2 v;
            v.x = v.y = (R)0;
            if (j0 + t < kend) {
                const double2 b2 = I.b[j0 + t];
                v.x = (R)b2.x;
                v.y = (R)b2.y;
            }
            bch[t] = v;
        }
        __syncthreads();
        if (active) {
            const int r0 = g * (JC / KG);
#pragma unroll 4
            for (int jj = r0; jj < r0 + JC / KG; ++jj) {
                R lv[4], mv[4];
                const int sw = (jj & 15) << 2;
                load4r<R>(Phl + jj * TT + ((ba * 4) ^ sw), lv);
                load4r<R>(Pm + jj * TT + ((bb * 4) ^ sw), mv);
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fma(lv[a], mv[b], acc[a][b]);
            }
        }
        if (want_delta && t < 4 * TT) {  // delta~_l partial: thread t owns l = t % 64, a quarter of the chunk rows
            const int l = t % TT, q = t / TT;
#pragma unroll
            for (int jj = q * (JC / 4); jj < (q + 1) * (JC / 4); ++jj) {
                const R v = Phl[jj * TT + (l ^ ((jj & 15) << 2))];
                const R2 b2 = bch[jj];
                dacc.x = fma(b2.x, v, dacc.x);  // conj(b) phi with phi real
                dacc.y = fma(-b2.y, v, dacc.y);
            }
        }
        __syncthreads();
    }

    // Add the second K-group's block into the first (through shared memory).
    R* kred = Phl;  // chunk buffer is free now
    if (g == 1 && active) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) kred[(a * 4 + b) * KSLOT + slot] = acc[a][b];
    }
    __syncthreads();
    double2 dsum = make_double2(0.0, 0.0);
    float dS = 0.f, dE = 0.f;  // FP32 path: float-float weighting (FP64 issues at 1/64 rate on this part)
    if (g == 0 && active) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += kred[(a * 4 + b) * KSLOT + slot];
        // Weighting: contribution of this block (and its mirror) to D_s.
        // G~ is real symmetric: Re(w_lm) G~_lm, doubled for the mirror; in
        // FP64 the imaginary part is kept as a residual on self-mirrored blocks.
        const bool mirror = !(diag && ba == bb);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int l = tl * TT + ba * 4 + a, m = tm * TT + bb * 4 + b;
                if (l < L && m < L) {
                    if constexpr (sizeof(R) == 4) {
                        const float4 wv = I.wf[(long long)l * L + m];  // (Re hi, Re lo, Im hi, Im lo)
                        ff_mac(dS, dE, wv.x, wv.y, mirror ? 2.f * (float)acc[a][b] : (float)acc[a][b]);
                    } else {
                        const double2 w = I.w[(long long)l * L + m];
                        const double gr = (double)acc[a][b];
                        if (mirror) {
                            dsum.x += 2.0 * (w.x * gr);
                        } else {
                            dsum.x += w.x * gr;
                            dsum.y += w.y * gr;
                        }
                    }
                }
            }
        if (s == 0 && f == 0 && I.Gpart) {
            R2* G = reinterpret_cast<R2*>(I.Gpart) + (long long)ksi * L * L;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int l = tl * TT + ba * 4 + a, m = tm * TT + bb * 4 + b;
                    if (l < L && m < L) {
                        R2 v;
                        v.x = acc[a][b];
                        v.y = (R)0;
                        G[(long long)l * L + m] = v;
                        if (mirror) G[(long long)m * L + l] = v;
                    }
                }
        }
    }
    const long long slotD = (((long long)s * I.F + f) * T * T + u) * ks + ksi;
    if constexpr (sizeof(R) == 4) {
        const double dtot = block_sum_ff(dS, dE, reinterpret_cast<double*>(red));
        if (t == 0) I.Dpart[slotD] = make_double2(dtot, 0.0);
    } else {
        const double2 dtot = block_sum2(dsum, red);
        if (t == 0) I.Dpart[slotD] = dtot;
    }
    if (want_delta) {
        // Reduce the four row-quarter partials of each l, then weight by ctil in FP64.
        R2* dred = reinterpret_cast<R2*>(Phm);  // free (diagonal items do not use it)
        if (t < 4 * TT) dred[t] = dacc;
        __syncthreads();
        double2 tsum = make_double2(0.0, 0.0);
        float trS = 0.f, trE = 0.f, tiS = 0.f, tiE = 0.f;
        if (t < TT) {
            const int l = tl * TT + t;
            R2 v = dred[t];
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                v.x += dred[q * TT + t].x;
                v.y += dred[q * TT + t].y;
            }
            if (l < L) {
                if constexpr (sizeof(R) == 4) {
                    const float4 cv = I.cf[l];  // c~_l as (Re hi, Re lo, Im hi, Im lo)
                    ff_mac(trS, trE, cv.x, cv.y, (float)v.x);
                    ff_mac(trS, trE, -cv.z, -cv.w, (float)v.y);
                    ff_mac(tiS, tiE, cv.x, cv.y, (float)v.y);
                    ff_mac(tiS, tiE, cv.z, cv.w, (float)v.x);
                } else {
                    const double2 c = I.ctil[l];
                    const double vr = (double)v.x, vi = (double)v.y;
                    tsum = make_double2(c.x * vr - c.y * vi, c.x * vi + c.y * vr);
                }
                if (s == 0 && I.dpart) reinterpret_cast<R2*>(I.dpart)[(long long)ksi * L + l] = v;
            }
        }
        if constexpr (sizeof(R) == 4) {
            const double tr = block_sum_ff(trS, trE, reinterpret_cast<double*>(red));
            const double ti = block_sum_ff(tiS, tiE, reinterpret_cast<double*>(red));
            if (t == 0) I.Tpart[((long long)s * T + tl) * ks + ksi] = make_double2(tr, ti);
        } else {
            const double2 ttot = block_sum2(tsum, red);
            if (t == 0) I.Tpart[((long long)s * T + tl) * ks + ksi] = ttot;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int find_instance(const Inst* insts, int count, long long g) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (insts[mid].item_base <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename R>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 3 : 1) k_terms_smem(const Inst* __restrict__ insts, int count, long long total,
                                                  unsigned long long* queue) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t smask[4 * TT];
    __shared__ double2 red[NT / 32];
    __shared__ long long s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(queue, 1ull);
        __syncthreads();
        const long long g = s_item;
        __syncthreads();
        if (g >= total) break;
        const int idx = find_instance(insts, count, g);
        const Inst& I = insts[idx];
        process_item<R>(I, int(g - I.item_base), smem, smask, red);
    }
}

// ------------------------------------------------- states in HBM (n > 12)
// The S shifted states of one instance, S x N real amplitudes (the ansatz is
// real), built by passes over HBM: the initial Ry layer on |0> is a product
// state written directly; each further layer is one pass over 4096-amplitude
// chunks (CZ ring signs and the Ry rotations of qubits 0..11 in shared memory)
// and one pass over column tiles of HC consecutive low indices x all high
// indices (Ry of qubits 12..; a warp reads whole 128-byte rows).
constexpr int LOQ = 12, LOC = 1 << LOQ, HC = 32;

template <typename R>
__device__ __forceinline__ void shift_angle(const Inst& I, int s, int a, R& c, R& sn) {
    int k = -1, which = 0;
    const int sg = s + I.s0;  // the shift's index in the instance
    if (sg > 0) {
        k = (sg - 1) >> 1;
        which = ((sg - 1) & 1) ? 2 : 1;
    }
    const double2 v = I.cs[(a == k ? which : 0) * I.P + a];
    c = (R)v.x;
    sn = (R)v.y;
}

template <typename R>
__global__ void __launch_bounds__(256) k_hbm_init(const Inst* __restrict__ insts, int idx) {
    // The product state factorises over bit groups: amplitude i of this chunk
    // is t0[i & 63] t1[(i >> 6) & 63] h, the factors of qubits 0..5, 6..11 and
    // of the chunk's high bits (two multiplies per amplitude).
    const Inst& I = insts[idx];
    __shared__ R cq[32], sq[32], t0[64], t1[64], hc;
    const int s = blockIdx.y, n = I.n, t = threadIdx.x;
    const size_t N = size_t(1) << n;
    if (t < n) shift_angle<R>(I, s, t, cq[t], sq[t]);
    __syncthreads();
    if (t < 128) {
        const int g = t >> 6, k = t & 63;
        R v = (R)1;
        for (int q = 0; q < 6; ++q) v *= ((k >> q) & 1) ? sq[6 * g + q] : cq[6 * g + q];
        (g ? t1 : t0)[k] = v;
    } else if (t == 128) {
        R v = (R)1;
        for (int q = LOQ; q < n; ++q) v *= ((blockIdx.x >> (q - LOQ)) & 1) ? sq[q] : cq[q];
        hc = v;
    }
    __syncthreads();
    R* st = reinterpret_cast<R*>(I.states) + s * N + ((size_t)blockIdx.x << LOQ);
    constexpr int VE = 16 / sizeof(R);
#pragma unroll 4
    for (int e4 = t; e4 < LOC / VE; e4 += 256) {
        R v[VE];
#pragma unroll
        for (int k = 0; k < VE; ++k) {
            const int e = e4 * VE + k;
            v[k] = t0[e & 63] * t1[(e >> 6) & 63] * hc;
        }
        uint4 u;
        memcpy(&u, v, 16);
        reinterpret_cast<uint4*>(st)[e4] = u;
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_hbm_lo(const Inst* __restrict__ insts, int idx, int layer) {
    extern __shared__ __align__(16) unsigned char sm[];
    R* w = reinterpret_cast<R*>(sm);
    const Inst& I = insts[idx];
    __shared__ R cq[LOQ], sq[LOQ];
    const int s = blockIdx.y, n = I.n, base = blockIdx.x << LOQ;
    const size_t N = size_t(1) << n;
    if (threadIdx.x < LOQ) shift_angle<R>(I, s, layer * n + threadIdx.x, cq[threadIdx.x], sq[threadIdx.x]);
    R* st = reinterpret_cast<R*>(I.states) + s * N + base;
    constexpr int VE = 16 / sizeof(R);  // amplitudes per 16-byte vector: all of a thread's loads in flight
#pragma unroll
    for (int e4 = threadIdx.x; e4 < LOC / VE; e4 += 256) {
        const uint4 u = reinterpret_cast<const uint4*>(st)[e4];
        R v[VE];
        memcpy(v, &u, 16);
#pragma unroll
        for (int k = 0; k < VE; ++k) {
            const int e = e4 * VE + k;
            w[e] = czring_parity(base + e, n) ? -v[k] : v[k];
        }
    }
    __syncthreads();
    for (int q = 0; q < LOQ; ++q) {
        const R c = cq[q], sn = sq[q];
        for (int p = threadIdx.x; p < LOC / 2; p += blockDim.x) {
            const int i0 = ((p >> q) << (q + 1)) | (p & ((1 << q) - 1)), i1 = i0 | (1 << q);
            const R a = w[i0], b = w[i1];
            w[i0] = c * a - sn * b;
            w[i1] = sn * a + c * b;
        }
        __syncthreads();
    }
#pragma unroll
    for (int e4 = threadIdx.x; e4 < LOC / VE; e4 += 256)
        reinterpret_cast<uint4*>(st)[e4] = reinterpret_cast<const uint4*>(w)[e4];
}

// The same low-qubit pass for FP32 states with the chunk in registers, 16
// amplitudes per thread, every Ry on register bits (no shuffles): the chunk is
// read with each thread holding 16 consecutive amplitudes (qubits 0..3 on its
// register bits, four 16-byte loads), then two transposes through shared
// memory put qubits 4..7 and then 8..11 on the register bits; the last layout
// stores 128 contiguous bytes per warp and register.  The CZ-ring signs come
// from the thread's part of the index and the register's (the ring's pairs
// split into those within each part, the pair across bits 3 and 4 and the
// wrap-around pair).  Amplitude e sits at word e + 4 (e >> 5) + 16 (e >> 8), so
// both transposes read and write without bank conflicts (the 16-byte stores of
// eight consecutive threads, 64 bytes apart, fall in eight different bank
// groups; the two half-warps of a 256-strided read sit 16 banks apart).
__device__ __forceinline__ int lo_pad(int e) { return e + ((e >> 5) << 2) + ((e >> 8) << 4); }
__global__ void __launch_bounds__(256) k_hbm_lo_regs(const Inst* __restrict__ insts, int idx, int layer) {
    constexpr int PADW = LOC + (LOC >> 5) * 4 + (LOC >> 8) * 16;
    __shared__ __align__(16) float scr[2][PADW];
    __shared__ float rq[LOQ], fq[LOQ];
    __shared__ int sfq[LOQ];
    const Inst& I = insts[idx];
    const int s = blockIdx.y, n = I.n, base = blockIdx.x << LOQ, t = threadIdx.x;
    const size_t N = size_t(1) << n;
    if (t < LOQ) {  // the rotations in scaled form; their factors are applied at the store
        float c, sn;
        shift_angle<float>(I, s, layer * n + t, c, sn);
        const RyScaled q = ry_scaled(c, sn);
        rq[t] = q.r;
        fq[t] = q.fac;
        sfq[t] = q.sform;
    }
    float* st = reinterpret_cast<float*>(I.states) + s * N + base;
    float v[16];
    // layout A: amplitude 16 t + r
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float4 x = reinterpret_cast<const float4*>(st)[4 * t + c];
        v[4 * c + 0] = x.x;
        v[4 * c + 1] = x.y;
        v[4 * c + 2] = x.z;
        v[4 * c + 3] = x.w;
    }
    {
        // CZ ring: parity of popc(i & (i >> 1)) over bits 0..n-2, plus bit n-1 times bit 0, for
        // i = base | 16 t | r: the thread's part, the pairs inside r, the pair (3, 4) and the wrap.
        const int pt = czring_parity(base | (t << 4), n);
        const int t0 = t & 1, bn1 = (base >> (n - 1)) & 1;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            int p = pt ^ (__popc(r & (r >> 1)) & 1);
            if (r & 8) p ^= t0;
            if (r & 1) p ^= bn1;
            v[r] = __int_as_float(__float_as_int(v[r]) ^ (p << 31));
        }
    }
    __syncthreads();  // the angles
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) ry_regs_scaled<16>(v, kb, rq[kb], sfq[kb]);  // qubits 0..3
#pragma unroll
    for (int c = 0; c < 4; ++c)
        *reinterpret_cast<float4*>(&scr[0][lo_pad(16 * t + 4 * c)]) = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    __syncthreads();
    // layout B: amplitude (t & 15) | 16 r | 256 (t >> 4)
    const int eb = (t & 15) | ((t >> 4) << 8);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = scr[0][lo_pad(eb | (r << 4))];
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) ry_regs_scaled<16>(v, kb, rq[4 + kb], sfq[4 + kb]);  // qubits 4..7
#pragma unroll
    for (int r = 0; r < 16; ++r) scr[1][lo_pad(eb | (r << 4))] = v[r];
    __syncthreads();
    // layout C: amplitude t | 256 r
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = scr[1][lo_pad(t | (r << 8))];
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) ry_regs_scaled<16>(v, kb, rq[8 + kb], sfq[8 + kb]);  // qubits 8..11
    float fac = 1.f;
#pragma unroll
    for (int q = 0; q < LOQ; ++q) fac *= fq[q];
#pragma unroll
    for (int r = 0; r < 16; ++r) st[t | (r << 8)] = v[r] * fac;
}

template <typename R>
__global__ void __launch_bounds__(256) k_hbm_hi(const Inst* __restrict__ insts, int idx, int layer) {
    extern __shared__ __align__(16) unsigned char sm[];
    R* w = reinterpret_cast<R*>(sm);  // [H][HC]
    const Inst& I = insts[idx];
    __shared__ R cq[32], sq[32];
    const int s = blockIdx.y, n = I.n, H = 1 << (n - LOQ), lo0 = blockIdx.x * HC;
    const size_t N = size_t(1) << n;
    if (threadIdx.x < n - LOQ)
        shift_angle<R>(I, s, layer * n + LOQ + threadIdx.x, cq[threadIdx.x], sq[threadIdx.x]);
    R* st = reinterpret_cast<R*>(I.states) + s * N;
    constexpr int VE = 16 / sizeof(R);  // 16-byte vectors of a row's HC columns
#pragma unroll 8
    for (int e4 = threadIdx.x; e4 < H * HC / VE; e4 += 256) {
        const int e = e4 * VE;
        reinterpret_cast<uint4*>(w)[e4] = *reinterpret_cast<const uint4*>(st + ((size_t)(e / HC) << LOQ) + lo0 + e % HC);
    }
    __syncthreads();
    for (int q = 0; q < n - LOQ; ++q) {
        const R c = cq[q], sn = sq[q];
        for (int p = threadIdx.x; p < (H / 2) * HC; p += blockDim.x) {
            const int hp = p / HC, lo = p % HC;
            const int h0 = ((hp >> q) << (q + 1)) | (hp & ((1 << q) - 1)), h1 = h0 | (1 << q);
            const R a = w[h0 * HC + lo], b = w[h1 * HC + lo];
            w[h0 * HC + lo] = c * a - sn * b;
            w[h1 * HC + lo] = sn * a + c * b;
        }
        __syncthreads();
    }
#pragma unroll 8
    for (int e4 = threadIdx.x; e4 < H * HC / VE; e4 += 256) {
        const int e = e4 * VE;
        *reinterpret_cast<uint4*>(st + ((size_t)(e / HC) << LOQ) + lo0 + e % HC) = reinterpret_cast<const uint4*>(w)[e4];
    }
}

// The high-qubit pass for FP32 states of 2^(12 + LOGH) amplitudes, LOGH >= 6
// (n >= 18), in registers: a CTA takes the 2^LOGH rows x 32 columns of its
// tile, lane = column.  Loaded with row h = (r << 3) | w (r: H/8 registers),
// the qubits on h bits 3.. rotate in place; one padded, conflict-free transpose
// to h = (w << (LOGH - 3)) | r puts h bits 0..2 (qubits 12..14) on registers,
// and the tile is stored from there (a warp writes one 128-byte row segment per
// register).  One barrier per tile instead of one per qubit.
template <int LOGH>
__global__ void __launch_bounds__(256) k_hbm_hi_regs(const Inst* __restrict__ insts, int idx, int layer) {
    constexpr int H = 1 << LOGH, RG = H / 8;
    __shared__ float scr[H * 33];
    __shared__ float rq[LOGH], fq[LOGH];
    __shared__ int sfq[LOGH];
    const Inst& I = insts[idx];
    const int s = blockIdx.y, n = I.n, lo0 = blockIdx.x * 32, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const size_t N = size_t(1) << n;
    if (t < LOGH) {  // the rotations in scaled form; their factors are applied at the store
        float c, sn;
        shift_angle<float>(I, s, layer * n + LOQ + t, c, sn);
        const RyScaled q = ry_scaled(c, sn);
        rq[t] = q.r;
        fq[t] = q.fac;
        sfq[t] = q.sform;
    }
    float* st = reinterpret_cast<float*>(I.states) + s * N + lo0 + lane;
    float v[RG];
#pragma unroll
    for (int r = 0; r < RG; ++r) v[r] = st[(size_t)((r << 3) | w) << LOQ];
    __syncthreads();
#pragma unroll
    for (int kb = 0; kb < LOGH - 3; ++kb)  // h bit 3 + kb: qubit 15 + kb, register bit kb
        ry_regs_scaled<RG>(v, kb, rq[3 + kb], sfq[3 + kb]);
#pragma unroll
    for (int r = 0; r < RG; ++r) scr[((r << 3) | w) * 33 + lane] = v[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RG; ++r) v[r] = scr[((w << (LOGH - 3)) | r) * 33 + lane];
#pragma unroll
    for (int kb = 0; kb < 3; ++kb)  // h bit kb: qubit 12 + kb, register bit kb
        ry_regs_scaled<RG>(v, kb, rq[kb], sfq[kb]);
    float fac = 1.f;
#pragma unroll
    for (int q = 0; q < LOGH; ++q) fac *= fq[q];
#pragma unroll
    for (int r = 0; r < RG; ++r) st[(size_t)((w << (LOGH - 3)) | r) << LOQ] = v[r] * fac;
}

template <typename R>
int build_hbm_states(dvqls_ctx* ctx, const Inst* dtable, int idx, int n, int d, int S, bool marks) {
    const int chunks = 1 << (n - LOQ), tiles = LOC / HC;
    const size_t lo_smem = sizeof(R) * LOC, hi_smem = sizeof(R) * ((size_t)chunks * HC);
    DVQLS_CUDA_TRY(ctx, allow_dynamic_smem((const void*)k_hbm_lo<R>));
    DVQLS_CUDA_TRY(ctx, allow_dynamic_smem((const void*)k_hbm_hi<R>));
    if (marks) prof_begin(ctx, 3);  // one profiling mark per kernel
    k_hbm_init<R><<<dim3(chunks, S), 256, 0, ctx->stream>>>(dtable, idx);
    if (marks) prof_end(ctx);
    for (int layer = 1; layer <= d; ++layer) {
        if (marks) prof_begin(ctx, 3);
        if constexpr (sizeof(R) == 4)
            k_hbm_lo_regs<<<dim3(chunks, S), 256, 0, ctx->stream>>>(dtable, idx, layer);
        else
            k_hbm_lo<R><<<dim3(chunks, S), 256, lo_smem, ctx->stream>>>(dtable, idx, layer);
        if (marks) prof_end(ctx);
        if (marks) prof_begin(ctx, 3);
        if (sizeof(R) == 4 && n == 20)
            k_hbm_hi_regs<8><<<dim3(LOC / 32, S), 256, 0, ctx->stream>>>(dtable, idx, layer);
        else if (sizeof(R) == 4 && n == 19)
            k_hbm_hi_regs<7><<<dim3(LOC / 32, S), 256, 0, ctx->stream>>>(dtable, idx, layer);
        else if (sizeof(R) == 4 && n == 18)
            k_hbm_hi_regs<6><<<dim3(LOC / 32, S), 256, 0, ctx->stream>>>(dtable, idx, layer);
        else
            k_hbm_hi<R><<<dim3(tiles, S), 256, hi_smem, ctx->stream>>>(dtable, idx, layer);
        if (marks) prof_end(ctx);
    }
    DVQLS_CUDA_TRY(ctx, cudaGetLastError());
    return DVQLS_OK;
}

// Amplitudes per work item for states in HBM (each FP32 sum runs over half
// of them; items are added in FP64), and its log2.
constexpr long long HBM_K = 2048;
constexpr int HBM_KQ = 11;

// ------------------------------------------------- tensor-core term tiles
// Precision DVQLS_FP32_TC: the Gram of a 64-term tile on the tensor cores.
// The Ry + CZ-ring ansatz state is real, so with the phase i^popc(x & z) in
// c~_l every phi_l[j] = (-1)^popc(z_l & (j ^ x_l)) psi[j ^ x_l] is real and
// G~ is a real symmetric 64 x 64 Gram: G~ = Z Z^T for the 64 x N matrix Z of
// the tile's phi_l.
//
// Split.  Every entry of 2^12 Z (and of 2^e b, e from ||b||) is split
// x = hi + lo into FP16 (round to nearest; the scale keeps lo clear of FP16
// subnormals for amplitudes above ~3e-5, and below that lo's absolute error
// stays under 2^-37), and Z Z^T ~ hi hi^T + hi lo^T + lo hi^T (lo lo^T, ~2^-22
// relative, dropped).  Only sum_lm Re(w_lm) G~_lm is formed and Re(w) is
// symmetric, so hi lo^T + lo hi^T may be replaced by (2 lo) hi^T: the sum
// G' = hi hi^T + (2 lo) hi^T has the symmetric part G~.  One tcgen05.mma
// kind::f16 per k-step of 16 amplitudes gives both terms: A = [2 lo; hi]
// (128 rows: the tile's 64 terms twice) against B = [hi; b] (80 rows: the
// same 64 hi rows, then hi and lo of Re b and Im b and 12 zero rows), so
// accumulator lanes 0..63 hold (2 lo) hi^T and lanes 64..127 hi hi^T (columns
// 0..63), with columns 64..67 the products with b that give
// delta_l = sum_j conj(b_j) phi_l[j] (hi hi(b) + hi lo(b) + lo hi(b)).  Every
// accumulator entry is a wanted one.  FP16 carries the 11-bit significand of
// TF32 at twice its tensor rate and half its operand bytes.
//
// Work split.  The shifted states are built before the term kernel
// (k_tc_states; packed pairs hi | (2 lo) << 16 of 2^12 psi, L2-resident), so
// the term kernel only streams.  One CTA per SM (it allocates tensor memory)
// with three warp roles:
//   - 16 builder warps take items from the queue, load an item's state into
//     shared memory in four copies (copy t holds psi[k ^ t], so a term's 16
//     amplitudes of a block are four aligned 16-byte loads: the low two bits
//     of x_l pick the copy, the next two permute the loads), and write the
//     operands of each stage (K-major, no swizzle: core matrices of 8 rows x
//     16 bytes; LBO 128 B between the two halves of a k-step, SBO 256 B between
//     8-row groups, 18 row groups per k-step: 2 lo rows in groups 0..7, hi
//     rows in 8..15, the b rows in 16, zeros in 17) into a ring of TC_NSTG
//     stages, one term's 16 amplitudes at two places of the stage per thread;
//   - one MMA warp issues each stage into the accumulator of its block and
//     commits the stage's buffer back to the builders;
//   - 4 epilogue warps (one per quarter of the tensor-memory lanes) fold each
//     finished accumulator block, read out an item's Gram and delta and weight
//     them, while the builders and the MMA warp go on with the next items.
// The tensor core adds each MMA's sum into the accumulator with a rounding
// that is not to nearest (measured: a one-sided drift of ~2^-24 |acc| per
// MMA), so an accumulator block covers TC_FLUSH stages and the epilogue folds
// its used parts (the Gram columns and two delta columns per lane)
// into FP32 running sums in tensor memory with round-to-nearest adds.  Two
// accumulators alternate between blocks, so the MMAs of a block never wait for
// the fold of the previous one.  The weighting runs in float-float arithmetic
// (two-product by FMA, two-sum; ~2^-44 relative) -- FP64 instructions issue at
// 1/64 of the FP32 rate on this part -- and only the final partial sums are
// formed in FP64.
// Every wait is bounded (a time budget, set per context); a role whose wait
// gives up raises the abort flag, every role stops at its next check, the MMA
// warp waits for its issued MMAs before the tensor memory is freed, and the
// host gets DVQLS_ERR_TIMEOUT.
// Served for tiles with L <= 64 (T = 1) of the global cost.
constexpr int TCK = 128;            // amplitudes per stage of a diagonal tile: 8 MMA k-steps of 16
constexpr int TC_BW = 16;           // builder warps
constexpr int TC_BT = 32 * TC_BW;   // builder threads: one 16-amplitude half-row of one term per stage each
constexpr int TC_EW = 8;            // epilogue warps, two per quarter of the tensor-memory lanes
constexpr int TC_ET = 32 * TC_EW;
constexpr int TCT = TC_BT + 32 + TC_ET;  // builders, the MMA warp, the epilogue warps
constexpr int TC_NSTG = 4;          // operand stages in flight
constexpr int TC_NIT = 4;           // item records in flight from the builders to the epilogue
constexpr int TC_FLUSH = 4;         // stages per accumulator block (8 MMAs of each Gram entry per stage)
constexpr int TC_NB = 144;          // row groups per k-step x 8: 2 lo and hi of 64 terms, b rows, zero rows
constexpr uint32_t TC_ACC1 = 256;   // tensor-memory columns of builder half h: 256 h ..
constexpr uint32_t TC_SLOT = 80;    // its two accumulator slots at 0 and 80 (blocks alternate between them) ..
constexpr int TC_SUM = 160;         // .. then the running sums of the Gram quadrants (64 columns) ..
constexpr int TC_DSUM = 224;        // .. and of the two delta columns of a lane
constexpr int TC_COLS = 512;        // tensor-memory columns allocated
// kind::f16 instruction descriptor: F32 accumulator (bits 4-5 = 1), A and B
// FP16 (bits 7-9, 10-12 = 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t tc_idesc(uint32_t nn) { return (1u << 4) | ((nn >> 3) << 17) | ((128u >> 4) << 24); }
constexpr long long TC_DRAIN_NS = 1000000000LL;  // 1 s for issued MMAs to complete (they take microseconds)
constexpr float TC_SCALE = 4096.f;                     // 2^12 on the state
constexpr float TC_UNSCALE = 1.f / (4096.f * 4096.f);  // 2^-24 on the Gram
constexpr int TC_KSTEP_BYTES = (TC_NB / 8) * 2 * 128;       // 18 row groups x 2 halves x 128 B
constexpr int TC_OPND_BYTES = (TCK / 32) * TC_KSTEP_BYTES;  // a pair stage's operand array (first or second tile)
constexpr int TC_STAGE_BYTES = 2 * TC_OPND_BYTES;           // = TCK / 16 k-steps of a diagonal stage
constexpr int TC_BROW = 16 * 256;   // offset of row group 16 (the b rows) inside a k-step
constexpr int TC_OFF_HALF = (TCK / 2 / 16) * TC_KSTEP_BYTES;  // 64 amplitudes further along k in a stage
constexpr int TC_HIROW = 64;        // first hi row of a diagonal k-step (rows 0..63: 2 lo)
constexpr int TC_ND = 80;           // B rows of a diagonal k-step: 64 hi rows, 4 b rows, 12 zero rows
constexpr int TC_X = 64 * 65;       // readout floats of one Gram quadrant ([64][65])
constexpr int TC_EPI_BYTES = 2 * TC_X * 4 + 2 * 64 * 8;  // both quadrants and their delta sums
constexpr int TC_BOP_STAGE = 1024;  // bytes of the b rows of one stage (4 rows x 128 amplitudes)
// Tile item u of a shift for T = ceil(L/64) tiles: u < T is the diagonal tile
// (u, u); u >= T the off-diagonal pair number u - T, pairs (tl < tm) in
// row-major order.
__host__ __device__ inline void tc_tile_pair(int u, int T, int& tl, int& tm) {
    if (u < T) {
        tl = tm = u;
        return;
    }
    int a = 0, rem = u - T;
    while (rem >= T - 1 - a) {
        rem -= T - 1 - a;
        ++a;
    }
    tl = a;
    tm = a + 1 + rem;
}

constexpr uint32_t TC_EXIT = 0xFFFFFFFFu;  // stage record of builders that have no more items
static_assert(TC_STAGE_BYTES % 1024 == 0, "stages keep the 1024-byte alignment of the ring");

// States in shared memory of 2^4 .. 2^copy_nmax amplitudes are kept in four
// copies, copy t holding psi[k ^ t] at word t (N + 8) + k; the copies start 32
// bytes apart in the banks.  copy_nmax <= TC_COPY_NMAX is chosen per batch so
// that the CTA's shared memory fits.
constexpr int TC_COPY_NMAX = 11;
__host__ __device__ inline size_t tc_psi_bytes(int n, bool copies) {
    const size_t N = size_t(1) << n;
    return copies ? 4 * (4 * N + 32) : ((N * 4 + 15) & ~size_t(15));
}
__host__ __device__ inline bool tc_copies(int n, int copy_nmax) { return n >= 4 && n <= copy_nmax; }
// States of 2^4 .. 2^split_nmax amplitudes (split_nmax <= TC_SPLIT_NMAX, chosen
// per batch like copy_nmax, and taking precedence) are instead kept as separate
// FP16 arrays of the hi and the 2 lo parts, eight copies of each: copy t holds
// element k ^ t (t < 8) at half t S + k, S = 2^n + 8 halves (the pad puts the
// copies 16 bytes apart in the banks); hi copy t starts at byte 2 t S, lo copy
// t at byte 2 (8 + t) S.  A term's 16 amplitudes of a block are then two
// 16-byte loads of hi and two of lo, already in order (the low three bits of
// x_l pick the copy, bit 3 the order of the loads): no byte permutes.
constexpr int TC_SPLIT_NMAX = 10;
__host__ __device__ inline bool tc_split(int n, int split_nmax) { return n >= 4 && n <= split_nmax; }
__host__ __device__ inline int tc_split_stride(int n) { return 2 * (1 << n) + 16; }  // bytes of one array
__host__ __device__ inline size_t tc_split_bytes(int n) { return 16 * (size_t)tc_split_stride(n); }
// Shared bytes of the term kernel for states of up to 2^nmax amplitudes in
// shared memory (0: every state in HBM), split arrays up to 2^split_nmax and
// packed copies up to 2^copy_nmax.
inline size_t tc_psi_region(int nmax_smem, int copy_nmax, int split_nmax) {
    size_t psi = 0;
    if (nmax_smem > 0) {
        auto one = [&](int n) {
            return tc_split(n, split_nmax) ? tc_split_bytes(n) : tc_psi_bytes(n, tc_copies(n, copy_nmax));
        };
        psi = std::max(one(nmax_smem), std::max(one(std::min(nmax_smem, copy_nmax)), one(std::min(nmax_smem, split_nmax))));
    }
    return (psi + 1023) & ~size_t(1023);
}
// A state region for each builder half; the shared-memory readout of the
// epilogue only for passes that return beta or delta (no other item touches it).
inline size_t tc_smem_bytes(int nmax_smem, int copy_nmax, int split_nmax, bool readout) {
    return 1024 + (size_t)TC_NSTG * TC_STAGE_BYTES + 2 * tc_psi_region(nmax_smem, copy_nmax, split_nmax) +
           (readout ? TC_EPI_BYTES : 0);
}
// Stages of the b rows of an instance with 2^n amplitudes.
__host__ __device__ inline long long tc_bop_stages(long long N) { return (N + TCK - 1) / TCK; }

// Power of two 2^e with |b_j| 2^e <= 2^12 for every j (from ||b||^2).
__device__ __forceinline__ float tc_bscale(double bn2) {
    int ex;
    frexp(sqrt(bn2), &ex);  // ||b|| <= 2^ex
    return ldexpf(1.f, 12 - ex);
}

// The b rows of the diagonal tiles' B operand for stages blk, blk + nblk,
// ..., in the shared-memory order of row group 16: [k-step 0..7][k half
// 0..1][row 0..3][8 FP16 values], rows 0..3 being hi of Re b, hi of Im b, lo
// of Re b and lo of Im b.  b is scaled by tc_bscale(||b||^2).
__device__ __forceinline__ void tc_fill_bop(const Inst& I, double bn2, int blk, int nblk) {
    const long long N = 1LL << I.n, chunks = tc_bop_stages(N) * (TC_BOP_STAGE / 16);
    const float sb = tc_bscale(bn2);
    for (long long c = (long long)blk * 256 + threadIdx.x; c < chunks; c += 256LL * nblk) {
        const long long stage = c >> 6;
        const int u = int(c & 63), ks = u >> 3, kh = (u >> 2) & 1, row = u & 3;
        const int part = row >> 1, im = row & 1;  // part 0: hi, 1: lo
        uint32_t wv[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            uint16_t hv[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const long long j = stage * TCK + ks * 16 + kh * 8 + e + q;
                const double v = j < N ? (im ? I.b[j].y : I.b[j].x) : 0.0;
                const float x = (float)(v * (double)sb);
                const __half h = __float2half_rn(x);
                const __half o = part == 0 ? h : __float2half_rn(x - __half2float(h));
                hv[q] = __half_as_ushort(o);
            }
            wv[e >> 1] = (uint32_t)hv[0] | ((uint32_t)hv[1] << 16);
        }
        reinterpret_cast<uint4*>(I.bop)[c] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
}
// States of up to this many amplitudes get their b rows from the prepare
// kernel; larger ones from k_prep_bop.
constexpr long long TC_BOP_FUSED_N = 4096;

__global__ void __launch_bounds__(256) k_prep_bop(const Inst* __restrict__ insts) {
    pdl_wait();
    pdl_trigger();
    const Inst I = insts[blockIdx.x];
    if (!I.bop || !I.b) return;
    tc_fill_bop(I, *I.bn2, blockIdx.y, gridDim.y);
}

// ||b||^2 of an instance (1 for the local cost, whose b = |+>^n is implied),
// valid in thread 0.  One compiled copy serves every caller, so each CTA that
// needs it gets the same bits.
__device__ __noinline__ double b_norm2(const Inst& I, double* red) {
    const int t = threadIdx.x;
    const long long N = 1LL << I.n;
    double acc = 0.0;
    if (I.b) {
#pragma unroll 4
        for (long long j = t; j < N; j += NT) {
            const double2 v = I.b[j];
            acc += v.x * v.x + v.y * v.y;
        }
    } else if (t == 0) {
        acc = 1.0;
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((t & 31) == 0) red[t >> 5] = acc;
    __syncthreads();
    double sum = 0.0;
    if (t == 0)
        for (int k = 0; k < NT / 32; ++k) sum += red[k];
    return sum;
}

// Per instance: CTAs 0 .. prep_parts - 1 form ||b||^2 and c~ (part 0), the
// half-angle tables (part 1, or 0 when alone) and the pair weights (all
// parts); CTAs from prep_parts on, when launched, build the tensor-core b rows
// (states of up to TC_BOP_FUSED_N amplitudes) from their own ||b||^2.
__global__ void __launch_bounds__(NT) k_prepare(const Inst* __restrict__ insts, int* status,
                                                unsigned long long* queue, int prep_parts) {
    pdl_trigger();
    if (queue && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *queue = 0ull;  // the term kernel's work queue
    const Inst I = insts[blockIdx.x];
    const int t = threadIdx.x, part = blockIdx.y, parts = prep_parts;
    const long long N = 1LL << I.n;
    __shared__ double red[NT / 32];
    if (part >= parts) {
        if (!I.bop || !I.b || N > TC_BOP_FUSED_N) return;
        __shared__ double s_bn2;
        const double bn2 = b_norm2(I, red);
        if (t == 0) s_bn2 = bn2;
        __syncthreads();
        tc_fill_bop(I, s_bn2, part - parts, int(gridDim.y) - parts);
        return;
    }
    if (part == 0) {
        const double sum = b_norm2(I, red);
        for (int l = t; l < I.L; l += NT) {
            const uint32_t x = I.xm[l], z = I.zm[l];
            if (x >= N || z >= N) set_status(status, DEV_BAD_MASK);
            const double2 c = I.coef[l];
            if (!isfinite(c.x) || !isfinite(c.y)) set_status(status, DEV_NONFINITE_INPUT);
            const double2 r = ctil_of(I, l);
            I.ctil[l] = r;
            if (I.cf) I.cf[l] = split_ff(r);
        }
        if (t == 0) {
            *I.bn2 = sum;
            if (!(sum > 0.0) || !isfinite(sum)) set_status(status, DEV_BAD_NORM);
        }
    }
    if (part == (parts > 1 ? 1 : 0))
        for (int a = t; a < I.P; a += NT) {
            const double al = I.alpha[a];
            if (!isfinite(al)) set_status(status, DEV_NONFINITE_INPUT);
            double s0, c0;
            sincos(0.5 * al, &s0, &c0);
            // Half angles of alpha +- pi/2 are alpha/2 +- pi/4: sin = (s0 +- c0) / sqrt 2,
            // cos = (c0 -+ s0) / sqrt 2.
            const double s1 = (s0 + c0) * M_SQRT1_2, c1 = (c0 - s0) * M_SQRT1_2;
            const double s2 = (s0 - c0) * M_SQRT1_2, c2 = (c0 + s0) * M_SQRT1_2;
            I.cs[a] = make_double2(c0, s0);
            I.cs[I.P + a] = make_double2(c1, s1);
            I.cs[2 * I.P + a] = make_double2(c2, s2);
        }
    const long long LL = I.w ? (long long)I.L * I.L : 0;  // no pair weights for the tensor-core tiles
    const long long per = (LL + parts - 1) / parts, e0 = part * per, e1 = min(LL, e0 + per);
    for (long long e = e0 + t; e < e1; e += NT) {
        const double2 a = ctil_of(I, int(e / I.L)), b = ctil_of(I, int(e % I.L));
        const double2 wv = make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
        I.w[e] = wv;
        if (I.wf) I.wf[e] = split_ff(wv);
    }
}

// Shifted states of the on-chip instances of a tensor-core pass (Stage I):
// 2^12 psi_s as packed pairs (split_h2l), S x N words per instance in
// workspace (I.tcst), built once per (instance, shift) before the term kernel.
// Grid (jobs, instances) of 256 threads: n <= 10 builds eight states per CTA,
// one per warp, in registers (qubits on lane bits by shuffles, the others in
// place) with no barrier; n = 11, 12 build one state per CTA with the
// 256-thread builder and copy it out.
constexpr int TCS_WARP_NMAX = 10;
__host__ __device__ inline int tcs_jobs(int n, int S) { return n <= TCS_WARP_NMAX ? (S + 7) / 8 : S; }
__host__ __device__ inline size_t tcs_smem(int n, int P) {
    const size_t N = size_t(1) << n;
    return n <= TCS_WARP_NMAX ? 8 * (size_t)P * sizeof(float2)
                              : N * 4 + 2 * (N + N / 32) * 4 + (size_t)P * sizeof(float2);
}

__global__ void __launch_bounds__(256) k_tc_states(const Inst* __restrict__ insts) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem[];
    const Inst& I = insts[blockIdx.y];
    if (!I.tcst) return;
    const int n = I.n, N = 1 << n, P = I.P, t = threadIdx.x, w = t >> 5, lane = t & 31;
    uint32_t* out = reinterpret_cast<uint32_t*>(I.tcst);
    if (n <= TCS_WARP_NMAX) {
        const int s = blockIdx.x * 8 + w;
        if (s >= I.S) return;  // this warp only: nothing below waits on other warps
        float2* scs = reinterpret_cast<float2*>(smem) + (size_t)w * P;
        int k = -1, which = 0;
        const int sg = s + I.s0;  // the shift's index in the instance
        if (sg > 0) {
            k = (sg - 1) >> 1;
            which = ((sg - 1) & 1) ? 2 : 1;
        }
        for (int a = lane; a < P; a += 32) {
            const double2 v = I.cs[(a == k ? which : 0) * P + a];
            scs[a] = make_float2((float)v.x, (float)v.y);
        }
        __syncwarp();
        void* psi = out + (size_t)s * N;
        switch (n) {
            case 6: state_regs_warp<2, 1, true>(psi, scs, n, I.d, lane, TC_SCALE); break;
            case 7: state_regs_warp<4, 2, true>(psi, scs, n, I.d, lane, TC_SCALE); break;
            case 8: state_regs_warp<8, 3, true>(psi, scs, n, I.d, lane, TC_SCALE); break;
            case 9: state_regs_warp<16, 4, true>(psi, scs, n, I.d, lane, TC_SCALE); break;
            case 10: state_regs_warp<32, 5, true>(psi, scs, n, I.d, lane, TC_SCALE); break;
            default: state_regs_warp<1, 0, true>(psi, scs, n, I.d, lane, TC_SCALE); break;  // n <= 5
        }
        return;
    }
    const int s = blockIdx.x;
    if (s >= I.S) return;  // the whole CTA
    uint32_t* psi = reinterpret_cast<uint32_t*>(smem);
    float* scratch = reinterpret_cast<float*>(smem + (size_t)N * 4);
    float2* scs = reinterpret_cast<float2*>(smem + (size_t)N * 4 + 2 * (size_t)(N + N / 32) * 4);
    build_state_regs<true>(psi, scratch, scs, n, I.d, P, I.cs, s + I.s0, t, 0, TC_SCALE);  // ends with a barrier
    uint4* dst = reinterpret_cast<uint4*>(out + (size_t)s * N);
    for (int c = t; c < N / 4; c += 256) dst[c] = reinterpret_cast<const uint4*>(psi)[c];
}

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128u >> 4) << 16;  // LBO: next 16-byte half along K
    d |= (uint64_t)(256u >> 4) << 32;  // SBO: next 8-row group
    d |= (uint64_t)1 << 46;            // descriptor version
    return d;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t phase) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    return done != 0;
}
// Non-blocking test of an mbarrier phase: for loops that poll several
// barriers, where a blocking try_wait on one could hold up work on another.
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t phase) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long gtimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for phase `phase` of an mbarrier for at most budget_ns nanoseconds of
// the global timer (and at most 2^32 tries, should the timer not advance).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, long long budget_ns) {
    if (mbar_try(bar, phase)) return true;
    const unsigned long long t0 = gtimer_ns();
    for (long long it = 0; it < (1LL << 32); ++it) {
        if (mbar_try(bar, phase)) return true;
        if ((long long)(gtimer_ns() - t0) > budget_ns) return false;
    }
    return false;
}
// The abort flag as other roles may have just written it.
__device__ __forceinline__ bool aborted(const int* f) { return *reinterpret_cast<const volatile int*>(f) != 0; }

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(bar) : "memory");
}

// Instance of work item g, from the cached bases of the first TC_MAXC
// instances (shared memory) or from the table.
constexpr int TC_MAXC = 128;
__device__ __forceinline__ int find_instance_cached(const Inst* insts, const long long* sbase, int count,
                                                    long long g) {
    if (count > TC_MAXC) return find_instance(insts, count, g);
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sbase[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Named barrier of `nthreads` threads that also returns the OR of a predicate
// over them: every thread gets the same answer, so a group decides to stop
// together.
__device__ __forceinline__ bool bar_or(int id, int nthreads, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void bar_n(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Byte offset of Z[row][kk .. kk+7] (FP16, kk a multiple of 8 below TCK/2)
// inside one operand array of a stage.
__device__ __forceinline__ int tc_off16(int row, int kk) {
    return (((kk >> 4) * (TC_NB / 8) + (row >> 3)) * 2 + ((kk >> 3) & 1)) * 128 + (row & 7) * 16;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
        "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
        "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}

__device__ __forceinline__ float2 tmem_ld2(uint32_t taddr) {
    uint32_t a, b;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(a), "=r"(b) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return make_float2(__uint_as_float(a), __uint_as_float(b));
}

__device__ __forceinline__ void tmem_st2(uint32_t taddr, float2 v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(taddr), "r"(__float_as_uint(v.x)),
                 "r"(__float_as_uint(v.y))
                 : "memory");
}

// One finished accumulator block (slot columns hb + slot ..) folded by an
// epilogue warp whose tensor-memory lanes are 32 q .. 32 q + 31 (Gram columns
// 32 ch .. 32 ch + 31; the delta columns when ch = 0).  Off-diagonal pair
// (`off`): lanes 0..63 are the first tile's hi rows and lanes 64..127 its lo
// rows, each against hi + lo of the second tile (two MMAs into the same 64
// columns; lo lo, ~2^-22 of the product, rides along).  Diagonal tile: lanes
// 0..63 are the 2 lo rows (delta: 2 lo hi(b) in columns 64, 65, halved here;
// 2 lo lo(b) in 66, 67 is dropped), lanes 64..127 the hi rows (delta: columns
// 64 + 66, 65 + 67), Gram columns 0..63 in both.  The first block of an item
// starts the half's running sums (columns hb + TC_SUM.., hb + TC_DSUM..), later
// ones add to them with round-to-nearest adds.  The last block (plus the running
// sums) is either stored to X[part][row][col] and XD[part][row] in shared
// memory (`toX`: shift-0 items whose beta / delta are returned; part: lane
// half) or weighted here: each entry meets its column weight c~_m (cB, float4
// (Re hi, Re lo, Im hi, Im lo) per column) in the sums (SA, EA) =
// sum_m Re c~_m g_am and (SB, EB) = sum_m Im c~_m g_am of this thread's row a --
// float-float for the main quadrant, FP32 for the correction quadrant (2 lo hi^T,
// or a pair's lo rows), SB skipped when every Im c~_m is zero (`imz`) -- and the
// delta columns are returned in dr.
__device__ __forceinline__ void tc_fold(uint32_t tmem, uint32_t hb, uint32_t slot, int q, int ch, int lane, bool first,
                                        bool last, bool off, bool toX, float* X, float2* XD, const float4* cB,
                                        float& SA, float& EA, float& SB, float& EB, float2& dr, bool imz) {
    const uint32_t base = tmem + ((32u * uint32_t(q)) << 16), acc = hb + slot * TC_SLOT;
    const int xr = (q & 1) * 32 + lane;  // row within the lane half
    float* Xq = X + (q >> 1) * TC_X;
#pragma unroll 1
    for (int g = 2 * ch; g < 2 * ch + 2; ++g) {  // this warp's 32 of the quadrant's 64 columns
        float v[16];
        tmem_ld16(base + acc + 16 * g, v);
        if (!first) {
            float u[16];
            tmem_ld16(base + hb + TC_SUM + 16 * g, u);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] += u[j];
        }
        if (last && toX) {
#pragma unroll
            for (int j = 0; j < 16; ++j) Xq[xr * 65 + 16 * g + j] = v[j];
        } else if (last && (off ? q >= 2 : q < 2)) {
            // the correction quadrant (2 lo hi^T of a diagonal tile, or the lo rows of a pair's
            // first tile) is ~2^-10 of the main one: FP32 products and sums leave its rounding
            // near 2^-34 of the weighted sum
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float4 cm = cB[16 * g + j];  // one address per warp: a broadcast
                SA = fmaf(cm.x, v[j], SA);
                if (!imz) SB = fmaf(cm.z, v[j], SB);
            }
        } else if (last && imz) {  // every Im c~_m of the columns is zero: the second form is zero
#pragma unroll
            for (int j = 0; j < 16; ++j) ff_mac(SA, EA, cB[16 * g + j].x, cB[16 * g + j].y, v[j]);
        } else if (last) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float4 cm = cB[16 * g + j];  // one address per warp: a broadcast
                ff_mac(SA, EA, cm.x, cm.y, v[j]);
                ff_mac(SB, EB, cm.z, cm.w, v[j]);
            }
        } else {
            tmem_st16(base + hb + TC_SUM + 16 * g, v);
        }
    }
    if (ch == 0 && !off) {  // the delta columns
        const float2 d0 = tmem_ld2(base + acc + 64);
        float2 dv;
        if (q < 2) {
            dv = make_float2(0.5f * d0.x, 0.5f * d0.y);  // exact
        } else {
            const float2 d1 = tmem_ld2(base + acc + 66);
            dv = make_float2(d0.x + d1.x, d0.y + d1.y);
        }
        if (!first) {
            const float2 du = tmem_ld2(base + hb + TC_DSUM);
            dv.x += du.x;
            dv.y += du.y;
        }
        if (last && toX) XD[(q >> 1) * 64 + xr] = dv;
        else if (last) dr = dv;
        else tmem_st2(base + hb + TC_DSUM, dv);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// A builder thread's share of a stage: the 16 amplitudes jb .. jb + 15 of one
// term at k = kk0 .. kk0 + 15, hi into row rhi of dhi and the low part into
// row rlo of dlo (doubled as stored, or halved back when HALVE).  psi_hl holds
// the Na amplitudes of the state's block that contains the sources (Na = N for
// states in shared memory).  With jb a multiple of 16, the sources j ^ x_l of the
// block are rb | (i ^ xlo) with rb = (jb ^ x_l) & ~15: a permutation of 16
// consecutive amplitudes, whose signs are the parity of z_l & rb times the
// per-term 16-bit pattern sgn (bit i: parity of z_l & (i ^ xlo)).  psi_hl holds
// the state in shared memory -- the split hi / lo arrays (`split`), four
// packed copies (`copies`) or one packed copy -- and psi_g the FP32 state in
// HBM (HBM).
// Two packed FP16 values times 1/2 (the low parts of an off-diagonal tile
// pair, stored doubled): exact, but for values that fall below the normal
// range (|lo| < 2^-14 of the scaled state, an error under 2^-25).
__device__ __forceinline__ uint32_t halve2(uint32_t v) {
    __half2 h = *reinterpret_cast<__half2*>(&v);
    h = __hmul2(h, __float2half2_rn(0.5f));
    return *reinterpret_cast<uint32_t*>(&h);
}

// oh, ol: byte offsets tc_off16(rhi, kk0), tc_off16(rlo, kk0) of the two rows
// (kk0 a multiple of 16, so the second 8 amplitudes sit 128 bytes further).
// The split arrays' stride is recomputed here from Na rather than passed in:
// one argument fewer live across the stage loop keeps the kernel's spills
// at a few bytes under its 72-register cap.
template <bool HBM, bool HALVE>
__device__ __forceinline__ void tc_build_half(const uint32_t* psi_hl, const float* psi_g, int N, int Na, int jb, int kend,
                                              bool act, uint32_t xl, uint32_t zl, const uint32_t (&sgn)[8],
                                              unsigned char* dhi, int oh, unsigned char* dlo, int ol, bool copies,
                                              bool split) {
    const uint32_t xhi = xl & ~15u, xlo = xl & 15u & uint32_t(N - 1);
    const int nval = act ? min(16, max(0, kend - jb)) : 0;
    const uint32_t rb = (uint32_t(jb) ^ xhi) & uint32_t(N - 1) & ~15u;
    const uint32_t flip = (__popc(zl & rb) & 1) ? 0x80008000u : 0u;  // the block's common sign
    const uint32_t ra = rb & uint32_t(Na - 1);  // the sources' offset in psi_hl (a block of Na amplitudes)
    const uint32_t sst = 2u * uint32_t(Na) + 16u;  // bytes of one split array (tc_split_stride)
    uint32_t hw[8], lw[8];  // word j: elements 2j, 2j + 1 of the hi and of the (2) lo row
    if (!HBM && split) {
        // target elements 8c .. 8c + 7 = copy (x_l & 7) at ra + 8 (c ^ bit 3 of x_l): one 16-byte load each
        const unsigned char* hb = reinterpret_cast<const unsigned char*>(psi_hl) + (xlo & 7u) * sst + 2u * ra;
        const uint32_t o0 = (xlo & 8u) ? 16u : 0u;
        const uint4 h0 = *reinterpret_cast<const uint4*>(hb + o0), h1 = *reinterpret_cast<const uint4*>(hb + (o0 ^ 16u));
        const unsigned char* lb = hb + 8u * sst;
        const uint4 l0 = *reinterpret_cast<const uint4*>(lb + o0), l1 = *reinterpret_cast<const uint4*>(lb + (o0 ^ 16u));
        hw[0] = h0.x; hw[1] = h0.y; hw[2] = h0.z; hw[3] = h0.w; hw[4] = h1.x; hw[5] = h1.y; hw[6] = h1.z; hw[7] = h1.w;
        lw[0] = l0.x; lw[1] = l0.y; lw[2] = l0.z; lw[3] = l0.w; lw[4] = l1.x; lw[5] = l1.y; lw[6] = l1.z; lw[7] = l1.w;
        if (nval < 16) {  // elements past the range (or of an inactive term) are zero
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t m = (2 * j < nval ? 0x0000FFFFu : 0u) | (2 * j + 1 < nval ? 0xFFFF0000u : 0u);
                hw[j] &= m;
                lw[j] &= m;
            }
        }
    } else {
    uint32_t w[16];
    if (!HBM && copies && nval == 16) {
        // w[4c + r] = psi[rb + 4 (c ^ xc) + (r ^ (x_l & 3))] = cpy[ra + 4 (c ^ xc) + r]
        const uint32_t* cpy = psi_hl + (xlo & 3u) * uint32_t(Na + 8);  // copy holding psi[k ^ (x_l & 3)]
        const uint32_t xc = xlo >> 2;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint4 v = *reinterpret_cast<const uint4*>(cpy + ra + 4u * (uint32_t(c) ^ xc));
            w[4 * c + 0] = v.x;
            w[4 * c + 1] = v.y;
            w[4 * c + 2] = v.z;
            w[4 * c + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            uint32_t x = 0u;
            if (i < nval) x = HBM ? split_h2l(psi_g[rb | (uint32_t(i) ^ xlo)] * TC_SCALE) : psi_hl[ra | (uint32_t(i) ^ xlo)];
            w[i] = x;
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // packed words to hi and lo words
        hw[j] = __byte_perm(w[2 * j], w[2 * j + 1], 0x5410);
        lw[j] = __byte_perm(w[2 * j], w[2 * j + 1], 0x7632);
    }
    }
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        // Sign bits of packed pairs sit at bits 15 and 31 of a hi (or 2 lo)
        // word: one three-input XOR applies the term's and the block's sign.
        uint4 hi, lo;
        hi.x = hw[4 * g + 0] ^ sgn[4 * g + 0] ^ flip;
        hi.y = hw[4 * g + 1] ^ sgn[4 * g + 1] ^ flip;
        hi.z = hw[4 * g + 2] ^ sgn[4 * g + 2] ^ flip;
        hi.w = hw[4 * g + 3] ^ sgn[4 * g + 3] ^ flip;
        lo.x = lw[4 * g + 0] ^ sgn[4 * g + 0] ^ flip;
        lo.y = lw[4 * g + 1] ^ sgn[4 * g + 1] ^ flip;
        lo.z = lw[4 * g + 2] ^ sgn[4 * g + 2] ^ flip;
        lo.w = lw[4 * g + 3] ^ sgn[4 * g + 3] ^ flip;
        if (HALVE) {
            lo.x = halve2(lo.x);
            lo.y = halve2(lo.y);
            lo.z = halve2(lo.z);
            lo.w = halve2(lo.w);
        }
        *reinterpret_cast<uint4*>(dhi + oh + 128 * g) = hi;
        *reinterpret_cast<uint4*>(dlo + ol + 128 * g) = lo;
    }
}

// Warp roles: two builder halves of 8 warps (warps 0..7 and 8..15), each
// running its own items -- its own queue fetches, state layout, masks, two of
// the ring's stages (slots 2h, 2h + 1), item records and two accumulator slots
// (TMEM columns 256 h .., its blocks alternating between them) -- so one
// half's item set-up (fetch, state load, masks) overlaps the other half's
// stages; warp 16 issues the MMAs of both halves, taking whichever half has a
// stage ready; warps 17..24 run the epilogue of both, taking whichever
// accumulator block has finished (both poll with non-blocking test_wait, so a
// barrier of one half never holds up the other).  Hand-overs, per half h: a
// stage by its `full` mbarrier (the half's 256 builder threads arrive after a
// proxy fence; the stage record -- address of the hi array, first / last stage
// of an accumulator block, pair flag -- is written first) and back by `empty`
// (the MMA warp's commit); an accumulator block by accf[h][slot] (commit after
// its last stage) and back by acce[h][slot] (every epilogue thread, after its
// tensor-memory loads); an item record (instance, shift, amplitude part, tile
// item, stages, flavour) by itf[h][r] and back by ite[h][r].  Every wait
// gives up after budget_ns nanoseconds; a thread that has seen the abort flag
// waits no more.
constexpr int TC_HT = TC_BT / 2;  // threads of a builder half
__global__ void __launch_bounds__(TCT, 1) k_terms_tc(const Inst* __restrict__ insts, int count, long long total,
                                                     unsigned long long* queue, int* status, int copy_nmax,
                                                     int split_range, int psi_half, long long budget_ns) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long fullb[TC_NSTG], emptyb[TC_NSTG], accf[2][2], acce[2][2],
        itf[2][TC_NIT], ite[2][TC_NIT], drainb;
    __shared__ uint32_t srec[TC_NSTG][2];
    __shared__ int4 irec[2][TC_NIT];
    __shared__ int4 s_cur[2];  // epilogue: the item record each half is on
    __shared__ uint32_t s_tmem;
    __shared__ long long s_item[2];
    __shared__ int s_abort, s_pick;
    __shared__ uint32_t sxl[2][128], szl[2][128];  // per half: masks of the item's tile (and of a pair's second)
    __shared__ float sred[3][2][TC_EW];
    __shared__ __align__(16) float4 scf[2][128];  // per half: c~ of the item's two tiles (zero past L)
    __shared__ long long s_ibase[TC_MAXC];  // item bases of the first TC_MAXC instances
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    unsigned char* base;
    {
        const uint32_t a = su32(smem_raw);
        base = smem_raw + ((1024u - (a & 1023u)) & 1023u);
    }
    // The readout (X, XD) is allocated only when the pass returns beta or delta; only
    // shift-0 items of such a pass touch it.
    float* X = reinterpret_cast<float*>(base + TC_NSTG * TC_STAGE_BYTES + 2 * psi_half);
    float2* XD = reinterpret_cast<float2*>(X + 2 * TC_X);
    if (t == 0) {
        for (int k = 0; k < TC_NSTG; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&fullb[k])), "r"(TC_HT));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&emptyb[k])), "r"(1));
        }
        for (int k = 0; k < 2; ++k) {
            for (int sl = 0; sl < 2; ++sl) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&accf[k][sl])), "r"(1));
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&acce[k][sl])), "r"(TC_ET));
            }
            for (int r = 0; r < TC_NIT; ++r) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&itf[k][r])), "r"(1));
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&ite[k][r])), "r"(1));
            }
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&drainb)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_abort = 0;
    }
    // Rows 4..7 of row group 16 and row group 17 of every k-step of every stage
    // stay zero (a diagonal stage's MMA reads them as B rows 68..79; the pair
    // stages use row groups 0..15 only, and only rows 0..3 of group 16 take b).
    for (int c = t; c < TC_NSTG * (TC_STAGE_BYTES / TC_KSTEP_BYTES) * 24; c += TCT) {
        const int blk = c / 24, u = c % 24;  // 16-byte chunk u of the zero area of k-step block blk
        const int off16 = u < 8 ? TC_BROW + (u >> 2) * 128 + 64 + (u & 3) * 16 : TC_BROW + 256 + (u - 8) * 16;
        *reinterpret_cast<uint4*>(base + blk * TC_KSTEP_BYTES + off16) = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int i = t; i < min(count, TC_MAXC); i += TCT) s_ibase[i] = insts[i].item_base;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                     "r"(TC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (w < TC_BW) {  // ------------------------------------------------------------ builder halves
        const int h = w >> 3, wl = w & 7, tt = t & (TC_HT - 1), bar = 1 + h;
        uint32_t* psi_hl = reinterpret_cast<uint32_t*>(base + TC_NSTG * TC_STAGE_BYTES + h * psi_half);
        uint32_t* xs = sxl[h];
        uint32_t* zs = szl[h];
        // Tasks of a thread in a stage: a diagonal tile's term l = lane % 8 + 8 wl,
        // block `sub` = (lane / 8) % 4 of 16 amplitudes, in both halves of the
        // stage; a pair's term l of side `side` (lane bit 3), blocks 2 sp and
        // 2 sp + 1 (sp: lane bit 4) of the stage's 64 amplitudes.  Either way
        // both tasks share the term's masks.
        const int l = (lane & 7) | (wl << 3), sub = (lane >> 3) & 3;
        const int pside = (lane >> 3) & 1, psp = (lane >> 4) & 1;
        // Byte offsets of this thread's rows at its first k in a stage: diagonal (hi row
        // TC_HIROW + l, 2 lo row l, k = 16 sub; the second half of the stage TC_OFF_HALF
        // further) and pair (hi row l, lo row 64 + l, k = 32 psp; the next 16 one k-step further).
        const int ohd = tc_off16(TC_HIROW + l, sub * 16), old = tc_off16(l, sub * 16);
        const int ohp = tc_off16(l, 32 * psp), olp = tc_off16(64 + l, 32 * psp);
        uint32_t eph = 0u, pend = 0u;   // bit q: parity of empty[2h + q] to wait for; stage in flight
        uint32_t iph = 0u, iused = 0u;  // item ring (thread 0 of the half): parity of ite[h][r]; slot used
        int ir = 0;
        uint32_t gc = 0u;  // stages the half has handed over
        bool ab = false;
        long long cur = total, nxt = total;  // thread 0 of the half: this item and the next from the queue
        if (tt == 0) {
            cur = (long long)atomicAdd(queue, 1ull);
            nxt = cur < total ? (long long)atomicAdd(queue, 1ull) : total;
        }
        for (;;) {
            if (tt == 0) s_item[h] = (aborted(&s_abort) || ab) ? total : cur;
            ab = bar_or(bar, TC_HT, ab);
            const long long gi = s_item[h];
            ab = bar_or(bar, TC_HT, ab);
            if (ab || gi >= total) break;
            if (tt == 0) {  // the next queue position, fetched while this item runs
                cur = nxt;
                nxt = cur < total && !aborted(&s_abort) ? (long long)atomicAdd(queue, 1ull) : total;
            }
            const int ii = find_instance_cached(insts, s_ibase, count, gi);
            const Inst& I = insts[ii];
            const int local = int(gi - I.item_base);
            const int n = I.n, N = 1 << n, L = I.L, ks = I.ks, T = I.T, NU = T * (T + 1) / 2;
            const int ksi = local % ks, u = (local / ks) % NU, f = (local / ks / NU) % I.F, s = (local / ks / NU) / I.F;
            int tl, tm;
            tc_tile_pair(u, T, tl, tm);
            // a pair of different tiles, or a local-cost flavour f > 0 (the second side's
            // strings X_j A_m = sigma(x_m ^ e_j, z_m), j = f - 1): stages of 64 amplitudes,
            // [hi; lo] rows on both sides
            const bool off = tl != tm || f > 0;
            const uint32_t xflip = f > 0 ? (1u << (f - 1)) : 0u;
            const int kper = N / ks, kbeg = ksi * kper, kend = kbeg + kper;
            const int step = off ? TCK / 2 : TCK;
            const int nch = (kend - kbeg + step - 1) / step;
            if (tt == 0) {  // the item's record for the epilogue
                if ((iused >> ir) & 1u) {
                    if (!ab && (aborted(&s_abort) || !mbar_wait(su32(&ite[h][ir]), (iph >> ir) & 1u, budget_ns)))
                        ab = true;
                    iph ^= 1u << ir;
                }
                iused |= 1u << ir;
                irec[h][ir] = make_int4(ii, s, ksi | (u << 16), nch | (f << 16));  // ksi < 2^16
                mbar_arrive(su32(&itf[h][ir]));
            }
            ir = (ir + 1) % TC_NIT;
            if (tt < 128) {
                const int gt = (tt < 64 ? tl : tm) * TT + (tt & 63);
                xs[tt] = gt < L ? I.xm[gt] ^ (tt < 64 ? 0u : xflip) : 0u;
                zs[tt] = gt < L ? I.zm[gt] : 0u;
            }
            const float* psi_g = I.states ? reinterpret_cast<const float*>(I.states) + (size_t)s * N : nullptr;
            // A state in HBM whose item reads only its own block of HBM_K amplitudes
            // (every X-mask of the item's tiles below HBM_K) is staged once in shared
            // memory and gathered from there like an on-chip state.
            bool blk = false;
            if (I.states) {
                const int gt = (tt < 64 ? tl : tm) * TT + (tt & 63);
                const bool far = tt < 128 && gt < L && xs[tt] >= uint32_t(HBM_K);
                blk = kper == HBM_K && !bar_or(bar, TC_HT, far);
            }
            const int Na = blk ? int(HBM_K) : N;  // amplitudes in shared memory
            // split_range: the largest n of the split arrays in bits 0..7, the smallest (at least 4) in 8..15
            const int sn = blk ? HBM_KQ : n;
            const bool split = (!I.states || blk) && tc_split(sn, split_range & 255) && sn >= (split_range >> 8);
            const bool copies = !split && (!I.states || blk) && tc_copies(blk ? HBM_KQ : n, copy_nmax);
            const int sst = tc_split_stride(blk ? HBM_KQ : n);  // bytes of one split array
            if (blk) {  // the item's block of the FP32 state in HBM, split into packed pairs here
                // the FP32 block lands in the last copy's room (with copies) or in place
                float* stage = reinterpret_cast<float*>(psi_hl + (copies ? 3 * (Na + 8) : 0));
                for (int k = 4 * tt; k < Na; k += 4 * TC_HT)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(stage + k)),
                                 "l"(__cvta_generic_to_global(psi_g + kbeg + k))
                                 : "memory");
                asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
                bar_n(bar, TC_HT);
                float vb[HBM_K / TC_HT];
#pragma unroll
                for (int e = 0; e < HBM_K / TC_HT; ++e) vb[e] = stage[tt * (HBM_K / TC_HT) + e];
                bar_n(bar, TC_HT);
                const int ncp = copies ? 4 : 1;
#pragma unroll
                for (int e = 0; e < HBM_K / TC_HT; ++e) {
                    const int k = tt * (HBM_K / TC_HT) + e;
                    const uint32_t v = split_h2l(vb[e] * TC_SCALE);
                    for (int t3 = 0; t3 < ncp; ++t3) psi_hl[t3 * (Na + 8) + (k ^ t3)] = v;
                }
            } else if (!I.states) {  // the packed state of shift s (built by k_tc_states)
                const uint32_t* src = reinterpret_cast<const uint32_t*>(I.tcst) + (size_t)s * N;
                // split arrays: the packed words land in the room of the last two lo copies
                uint32_t* dst = split ? reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(psi_hl) + 14 * sst)
                                      : psi_hl;
                if (N >= 4) {
                    for (int k = 4 * tt; k < N; k += 4 * TC_HT)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(dst + k)),
                                     "l"(__cvta_generic_to_global(src + k))
                                     : "memory");
                    asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
                } else if (tt < N) {
                    dst[tt] = src[tt];
                }
            }
            ab = bar_or(bar, TC_HT, ab);
            if (split) {
                // Group gi of 8 amplitudes (one per thread: N / 8 <= 128 groups): its packed words
                // p_i = hi_i | (2 lo)_i << 16 go to the hi and lo copies t = 0..7, whose words j hold
                // elements (2j) ^ t, (2j + 1) ^ t of the group: word j ^ (t >> 1) of the pairs in order
                // (t even) or swapped (t odd).
                unsigned char* pb = reinterpret_cast<unsigned char*>(psi_hl);
                const int gi = tt;
                uint4 p0 = make_uint4(0u, 0u, 0u, 0u), p1 = p0;
                if (gi < N / 8) {
                    const uint4* stg = reinterpret_cast<const uint4*>(pb + 14 * sst);
                    p0 = stg[2 * gi];
                    p1 = stg[2 * gi + 1];
                }
                bar_n(bar, TC_HT);  // every staged word is read before the copies overwrite them
                if (gi < N / 8) {
                    const uint32_t pw[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
                    uint32_t HP[4], HS[4], LP[4], LS[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        HP[k] = __byte_perm(pw[2 * k], pw[2 * k + 1], 0x5410);
                        HS[k] = __byte_perm(pw[2 * k], pw[2 * k + 1], 0x1054);
                        LP[k] = __byte_perm(pw[2 * k], pw[2 * k + 1], 0x7632);
                        LS[k] = __byte_perm(pw[2 * k], pw[2 * k + 1], 0x3276);
                    }
#pragma unroll
                    for (int t8 = 0; t8 < 8; ++t8) {
                        const int u = t8 >> 1;
                        const uint32_t* H = (t8 & 1) ? HS : HP;
                        const uint32_t* Lw = (t8 & 1) ? LS : LP;
                        *reinterpret_cast<uint4*>(pb + t8 * sst + 16 * gi) = make_uint4(H[0 ^ u], H[1 ^ u], H[2 ^ u], H[3 ^ u]);
                        *reinterpret_cast<uint4*>(pb + (8 + t8) * sst + 16 * gi) =
                            make_uint4(Lw[0 ^ u], Lw[1 ^ u], Lw[2 ^ u], Lw[3 ^ u]);
                    }
                }
                bar_n(bar, TC_HT);
            }
            if (copies && !blk) {  // copy t: psi[k ^ t] at word t (N + 8) + k
                for (int k = tt; k < N; k += TC_HT) {
                    const uint32_t v = psi_hl[k];
#pragma unroll
                    for (int t3 = 1; t3 < 4; ++t3) psi_hl[t3 * (N + 8) + (k ^ t3)] = v;
                }
                bar_n(bar, TC_HT);
            }
            const int side = off ? pside : 0;
            const bool act = (side ? tm : tl) * TT + l < L;
            const uint32_t xl = xs[side * 64 + l], zl = zs[side * 64 + l];
            uint32_t sgn[8];  // word g: sign bits of elements 2g (bit 15) and 2g + 1 (bit 31) of a 16-block
            {
                const uint32_t xlo = xl & 15u & uint32_t(N - 1);
#pragma unroll
                for (int g = 0; g < 8; ++g)
                    sgn[g] = ((__popc(zl & 15u & (uint32_t(2 * g) ^ xlo)) & 1) ? 0x8000u : 0u) |
                             ((__popc(zl & 15u & (uint32_t(2 * g + 1) ^ xlo)) & 1) ? 0x80000000u : 0u);
            }
            const bool gl = I.states && !blk;  // gather from the state in HBM
            for (int c = 0; c < nch; ++c, ++gc) {
                const int q = int(gc & 1u), st = 2 * h + q;
                if ((pend >> q) & 1u) {  // the MMAs that read this buffer last time must be done
                    if (!ab && (aborted(&s_abort) || !mbar_wait(su32(&emptyb[st]), (eph >> q) & 1u, budget_ns)))
                        ab = true;
                    eph ^= 1u << q;
                    pend &= ~(1u << q);
                }
                unsigned char* zhi = base + st * TC_STAGE_BYTES;
                unsigned char* zlo = zhi + TC_OPND_BYTES;
                const int j0 = kbeg + c * step;
                const bool brow = !off && I.bop && tt < TC_BOP_STAGE / 16;
                if (brow) {  // the stage's b rows (j0 is a multiple of TCK), copied while the terms are built
                    const uint4* srcb = reinterpret_cast<const uint4*>(I.bop) + (long long)(j0 / TCK) * (TC_BOP_STAGE / 16) + tt;
                    const int ks8 = tt >> 3, kh = (tt >> 2) & 1, br = tt & 3;
                    const uint32_t dst = su32(zhi + ks8 * TC_KSTEP_BYTES + TC_BROW + kh * 128 + br * 16);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n\tcp.async.commit_group;" ::"r"(dst),
                                 "l"(__cvta_generic_to_global(srcb))
                                 : "memory");
                }
                if (!off) {
                    // diagonal: amplitudes kk = 64 hf + 16 sub .. of the stage, hi to row
                    // TC_HIROW + l and 2 lo to row l of the same k-steps
#pragma unroll 1
                    for (int hf = 0; hf < 2; ++hf) {
                        const int jb = j0 + hf * (TCK / 2) + sub * 16, dk = hf * TC_OFF_HALF;
                        if (gl)
                            tc_build_half<true, false>(nullptr, psi_g, N, Na, jb, kend, act, xl, zl, sgn, zhi,
                                                       ohd + dk, zhi, old + dk, false, false);
                        else
                            tc_build_half<false, false>(psi_hl, nullptr, N, Na, jb, kend, act, xl, zl, sgn, zhi,
                                                        ohd + dk, zhi, old + dk, copies, split);
                    }
                } else {
                    // pair: the side's array (hi array: first tile, 2 lo array: second),
                    // hi to row l and lo (halved back) to row 64 + l
                    unsigned char* dst = pside ? zlo : zhi;
#pragma unroll 1
                    for (int qb = 0; qb < 2; ++qb) {
                        const int jb = j0 + (2 * psp + qb) * 16, dk = qb * TC_KSTEP_BYTES;
                        if (gl)
                            tc_build_half<true, true>(nullptr, psi_g, N, Na, jb, kend, act, xl, zl, sgn, dst, ohp + dk,
                                                      dst, olp + dk, false, false);
                        else
                            tc_build_half<false, true>(psi_hl, nullptr, N, Na, jb, kend, act, xl, zl, sgn, dst, ohp + dk,
                                                       dst, olp + dk, copies, split);
                    }
                }
                if (brow) asm volatile("cp.async.wait_all;" ::: "memory");
                if (tt == 0) {
                    srec[st][0] = su32(zhi);
                    srec[st][1] = (c % TC_FLUSH == 0 ? 1u : 0u) | ((c % TC_FLUSH == TC_FLUSH - 1 || c + 1 == nch) ? 2u : 0u) |
                                  (off ? 4u : 0u);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(su32(&fullb[st]));
                pend |= 1u << q;
            }
        }
        // No more items: an exit stage for the MMA warp and an exit record for
        // the epilogue (their waits are bounded whatever happens here).
        {
            const int q = int(gc & 1u), st = 2 * h + q;
            if (((pend >> q) & 1u) && !ab && !aborted(&s_abort)) mbar_wait(su32(&emptyb[st]), (eph >> q) & 1u, budget_ns);
            if (tt == 0) srec[st][0] = TC_EXIT;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(su32(&fullb[st]));
            if (tt == 0) {
                if (((iused >> ir) & 1u) && !ab && !aborted(&s_abort))
                    mbar_wait(su32(&ite[h][ir]), (iph >> ir) & 1u, budget_ns);
                irec[h][ir] = make_int4(-1, 0, 0, 0);
                mbar_arrive(su32(&itf[h][ir]));
            }
        }
        if (ab) s_abort = 1;
    } else if (w == TC_BW) {  // ------------------------------------------------------------- MMA warp
        if (lane == 0) {
            // per half h: next ring slot (bit h), parity of full[2h + q] (bit 2h + q), accumulator slot
            // of the block in progress (bit h) and of the next block (bit h); per accumulator slot sl of
            // half h (bit 2h + sl): parity of acce[h][sl], slot used before; done (bit h)
            uint32_t nq = 0u, fph = 0u, csl = 0u, nsl = 0u, aph = 0u, aused = 0u, done = 0u;
            unsigned long long idle0 = gtimer_ns();
            while (done != 3u) {
                bool progressed = false;
                for (int h = 0; h < 2; ++h) {
                    if ((done >> h) & 1u) continue;
                    const int q = (nq >> h) & 1, st = 2 * h + q;
                    if (!mbar_test(su32(&fullb[st]), (fph >> st) & 1u)) continue;
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t hb = srec[st][0], fl = srec[st][1];
                    if (hb != TC_EXIT && (fl & 1u)) {
                        // first stage of a block: its slot must have been read out by the epilogue
                        // (the block before last of this half); the other half meanwhile
                        const uint32_t sl = (nsl >> h) & 1u, sb = 2u * h + sl;
                        if ((aused >> sb) & 1u) {
                            if (!mbar_test(su32(&acce[h][sl]), (aph >> sb) & 1u)) continue;
                            aph ^= 1u << sb;
                            asm volatile("tcgen05.fence::after_thread_sync;");
                        }
                        aused |= 1u << sb;
                        csl = (csl & ~(1u << h)) | (sl << h);
                        nsl ^= 1u << h;
                    }
                    fph ^= 1u << st;
                    nq ^= 1u << h;
                    progressed = true;
                    if (hb == TC_EXIT) {
                        done |= 1u << h;
                        continue;
                    }
                    const uint32_t sl = (csl >> h) & 1u;
                    const uint32_t lb = hb + TC_OPND_BYTES, tm = s_tmem + uint32_t(h) * TC_ACC1 + sl * TC_SLOT;
                    if (fl & 4u) {  // pair: [hi; lo] of the first tile against hi, then lo, of the second
                        const uint64_t dA = tc_desc(hb), dB = tc_desc(lb);
                        const uint32_t aLo = uint32_t(dA), aHi = uint32_t(dA >> 32), bLo = uint32_t(dB), bHi = uint32_t(dB >> 32);
                        const uint32_t acc0 = (fl & 1u) ? 0u : 1u;
#pragma unroll
                        for (int ksx = 0; ksx < TCK / 32; ++ksx) {
                            const uint32_t kofs = uint32_t(ksx * (TC_KSTEP_BYTES >> 4));
                            asm volatile(
                                "{\n\t.reg .pred p;\n\t.reg .b64 da, db;\n\tsetp.ne.b32 p, %6, 0;\n\t"
                                "mov.b64 da, {%1, %2};\n\tmov.b64 db, {%3, %4};\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n\t}\n" ::"r"(tm),
                                "r"(aLo + kofs), "r"(aHi), "r"(bLo + kofs), "r"(bHi), "r"(tc_idesc(64)),
                                "r"(ksx == 0 ? acc0 : 1u));
                            asm volatile(
                                "{\n\t.reg .b64 da, db;\n\t"
                                "mov.b64 da, {%1, %2};\n\tmov.b64 db, {%3, %4};\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, 1;\n\t}\n" ::"r"(tm),
                                "r"(aLo + kofs), "r"(aHi), "r"(bLo + kofs + uint32_t((8 * 256) >> 4)), "r"(bHi),
                                "r"(tc_idesc(64)));
                        }
                    } else {  // diagonal: A = [2 lo; hi] (row groups 0..15), B = [hi; b] (8..17)
                        const uint64_t dA = tc_desc(hb), dB = tc_desc(hb + (TC_HIROW / 8) * 256);
                        const uint32_t aLo = uint32_t(dA), aHi = uint32_t(dA >> 32), bLo = uint32_t(dB), bHi = uint32_t(dB >> 32);
                        const uint32_t acc0 = (fl & 1u) ? 0u : 1u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\t.reg .b64 da, db;\n\tsetp.ne.b32 p, %6, 0;\n\t"
                            "mov.b64 da, {%1, %2};\n\tmov.b64 db, {%3, %4};\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n\t}\n" ::"r"(tm),
                            "r"(aLo), "r"(aHi), "r"(bLo), "r"(bHi), "r"(tc_idesc(TC_ND)), "r"(acc0));
#pragma unroll
                        for (int ksx = 1; ksx < TCK / 16; ++ksx) {
                            asm volatile(
                                "{\n\t.reg .b64 da, db;\n\t"
                                "mov.b64 da, {%1, %2};\n\tmov.b64 db, {%3, %4};\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, 1;\n\t}\n" ::"r"(tm),
                                "r"(aLo + uint32_t(ksx * (TC_KSTEP_BYTES >> 4))), "r"(aHi),
                                "r"(bLo + uint32_t(ksx * (TC_KSTEP_BYTES >> 4))), "r"(bHi), "r"(tc_idesc(TC_ND)));
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        su32(&emptyb[st])));
                    if (fl & 2u)
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            su32(&accf[h][sl])));
                }
                if (progressed) {
                    idle0 = gtimer_ns();
                } else if (aborted(&s_abort) || (long long)(gtimer_ns() - idle0) > budget_ns) {
                    s_abort = 1;
                    break;
                }
            }
            // Every MMA issued has completed before the tensor memory is freed.
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                su32(&drainb)));
            if (!mbar_wait(su32(&drainb), 0u, TC_DRAIN_NS)) s_abort = 1;
        }
        __syncwarp();
    } else {  // ----------------------------------------------------------------------------- epilogue
        const int et = t - (TC_BT + 32), ew = et >> 5, q = w & 3, ch = ew >> 2;  // q: this warp's TMEM lane quarter
        // Thread 0 keeps, per half, the item-ring position, the ring's parities and
        // whether it holds the current record, and the accumulator slot of the
        // half's next block with the parities of accf; every thread keeps the
        // block count.
        uint32_t fph = 0u, aph = 0u, esl = 0u, have = 0u, done = 0u;
        int r[2] = {0, 0}, blkc[2] = {0, 0}, last_pick = 1;
        bool ab = false;
        for (;;) {
            if (et == 0) {  // the half whose accumulator block is ready next
                int pick = -1, pslot = 0;
                const unsigned long long t0 = gtimer_ns();
                for (;;) {
                    for (int k = 1; k <= 2 && pick < 0; ++k) {
                        const int hh = (last_pick + k) & 1;
                        if ((done >> hh) & 1u) continue;
                        if (!((have >> hh) & 1u)) {
                            const uint32_t pb = hh * TC_NIT + r[hh];
                            if (!mbar_test(su32(&itf[hh][r[hh]]), (fph >> pb) & 1u)) continue;
                            fph ^= 1u << pb;
                            const int4 rc = irec[hh][r[hh]];
                            s_cur[hh] = rc;
                            if (rc.x < 0) {
                                done |= 1u << hh;
                                continue;
                            }
                            have |= 1u << hh;
                        }
                        const uint32_t sl = (esl >> hh) & 1u, sb = 2u * hh + sl;
                        if (mbar_test(su32(&accf[hh][sl]), (aph >> sb) & 1u)) {
                            aph ^= 1u << sb;
                            esl ^= 1u << hh;
                            pick = hh;
                            pslot = int(sl);
                        }
                    }
                    if (pick >= 0 || done == 3u) break;
                    if (aborted(&s_abort) || (long long)(gtimer_ns() - t0) > budget_ns) {
                        pick = -2;
                        break;
                    }
                }
                if (pick >= 0) last_pick = pick;
                s_pick = pick | (pslot << 4);
            }
            bar_n(3, TC_ET);
            const int pick = s_pick < 0 ? s_pick : (s_pick & 15), slot = s_pick < 0 ? 0 : (s_pick >> 4);
            if (pick == -2) ab = true;
            if (pick < 0) break;
            const int4 rc = s_cur[pick];
            const Inst& I = insts[rc.x];
            const int s = rc.y, ksi = rc.z & 0xFFFF, u = rc.z >> 16, nch = rc.w & 0xFFFF, f = rc.w >> 16;
            const int L = I.L, ks = I.ks, T = I.T;
            int tl, tm;
            tc_tile_pair(u, T, tl, tm);
            const bool off = tl != tm || f > 0;
            const int nblk = (nch + TC_FLUSH - 1) / TC_FLUSH, b = blkc[pick];
            const bool lastb = b + 1 == nblk;
            float4* cfh = scf[pick];
            if (b == 0 && et < 128) {  // c~ of the item's two tiles, fetched while its blocks run
                const int gl = ((et >> 6) ? tm : tl) * TT + (et & 63);
                if (gl < L)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n\tcp.async.commit_group;" ::"r"(
                                     su32(cfh + et)),
                                 "l"(__cvta_generic_to_global(I.cf + gl))
                                 : "memory");
                else
                    cfh[et] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            // The beta / delta outputs of shift 0 need the two quadrants added entry by entry:
            // that item's last block goes through shared memory (X, XD); every other item's last
            // block is weighted in the fold, straight from the tensor-memory loads.
            const bool toX = s == 0 && (I.Gpart || I.dpart);
            bool imz = false;  // the column weights c~_m of the item are all real (a real A gives real c~)
            if (lastb && !toX) {
                asm volatile("cp.async.wait_all;" ::: "memory");
                bar_n(3, TC_ET);  // c~ of the item's tiles is in cfh
                const float4 c0 = cfh[(off ? 64 : 0) + lane], c1 = cfh[(off ? 64 : 0) + 32 + lane];
                imz = __all_sync(0xffffffffu, c0.z == 0.f && c0.w == 0.f && c1.z == 0.f && c1.w == 0.f);
            }
            float SA = 0.f, EA = 0.f, SB = 0.f, EB = 0.f;
            float2 dr = make_float2(0.f, 0.f);
            asm volatile("tcgen05.fence::after_thread_sync;");
            tc_fold(s_tmem, uint32_t(pick) * TC_ACC1, uint32_t(slot), q, ch, lane, b == 0, lastb, off, toX, X, XD,
                    cfh + (off ? 64 : 0), SA, EA, SB, EB, dr, imz);
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(su32(&acce[pick][slot]));
            blkc[pick] = lastb ? 0 : b + 1;
            if (!lastb) {
                bar_n(3, TC_ET);  // s_pick and s_cur are read before thread 0 writes them again
                continue;
            }
            if (toX) {
                asm volatile("cp.async.wait_all;" ::: "memory");
                bar_n(3, TC_ET);  // the readout is in X (and XD), c~ in cfh
            }
            const int nl = min(TT, L - tl * TT);  // terms in the first tile
            const float* Xu = X;
            const float* Xl = X + TC_X;
            float S = 0.f, E = 0.f, TrS = 0.f, TrE = 0.f, TiS = 0.f, TiE = 0.f;
            float2* Gp = (s == 0 && I.Gpart) ? reinterpret_cast<float2*>(I.Gpart) + (long long)ksi * L * L : nullptr;
            if (!toX) {
                // Row a of this thread's quadrant (2 lo or hi rows of a diagonal tile, hi or lo rows
                // of a pair's first tile): the two quadrants of a row hold two parts of the same
                // entries, so each adds its own share of sum_am Re w_am g_am, with
                // Re w_am = Re c~_a Re c~_m + Im c~_a Im c~_m (terms past L: c~ = 0, zero rows).
                const int a = (q & 1) * 32 + lane;
                const float4 cl = cfh[a];
                const float fac = tl != tm ? 2.f : 1.f;
                ff_mac(S, E, fac * cl.x, fac * cl.y, SA);
                E += fac * cl.x * EA;
                ff_mac(S, E, fac * cl.z, fac * cl.w, SB);
                E += fac * cl.z * EB;
                if (!off && ch == 0 && a < nl && !I.local) {  // this quadrant's part of delta~_a
                    const float dsc = 1.f / (TC_SCALE * tc_bscale(*I.bn2));  // exact: a power of two
                    const float2 dacc = make_float2(dr.x * dsc, -dr.y * dsc);  // conj(b) phi
                    ff_mac(TrS, TrE, cl.x, cl.y, dacc.x);
                    ff_mac(TrS, TrE, -cl.z, -cl.w, dacc.y);
                    ff_mac(TiS, TiE, cl.x, cl.y, dacc.y);
                    ff_mac(TiS, TiE, cl.z, cl.w, dacc.x);
                }
            } else {
                // Re w_lm = Re c~_l Re c~_m + Im c~_l Im c~_m, so the weighted sum is the
                // pair of bilinear forms sum_lm (Re c~_l Re c~_m + Im c~_l Im c~_m) g_lm
                // over the readout g = Xu + Xl.  On a diagonal tile g = G' = hi hi^T +
                // (2 lo) hi^T, whose symmetric part is G~ (scaled by 2^24): a form with
                // symmetric weights sees only that part.  On a pair g = G~_ab for term a
                // of the first tile and b of the second (for flavour f > 0, gamma^j_ab);
                // different tiles stand for both orders of the pair (the Gram, gamma^j
                // and Re w are symmetric), so those count twice (exact doubling).  Thread
                // et takes row a = et / 4 and columns 8 (et % 4) + j, 32 + 8 (et % 4) + j
                // (j < 8: one bank per lane); terms past L have c~ = 0 and zero rows.
                const float4* cB = cfh + (off ? 64 : 0);
                const int a = et >> 2, cq = et & 3;
                float SA = 0.f, EA = 0.f, SB = 0.f, EB = 0.f;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int bc = ((k >> 3) << 5) | (cq << 3) | (k & 7);
                    const float g = Xu[a * 65 + bc] + Xl[a * 65 + bc];
                    const float4 cm = cB[bc];
                    ff_mac(SA, EA, cm.x, cm.y, g);
                    ff_mac(SB, EB, cm.z, cm.w, g);
                    if (Gp && (off ? f == 0 : true)) {
                        const long long ga = tl * TT + a, gb = tm * TT + bc;
                        if (ga < L && gb < L) {
                            if (off) {
                                const float2 gv = make_float2(g * TC_UNSCALE, 0.f);
                                Gp[ga * L + gb] = gv;
                                Gp[gb * L + ga] = gv;
                            } else {  // the symmetric part, each ordered entry from its own thread
                                const float gt = Xu[bc * 65 + a] + Xl[bc * 65 + a];
                                Gp[ga * L + gb] = make_float2(0.5f * (g + gt) * TC_UNSCALE, 0.f);
                            }
                        }
                    }
                }
                const float4 cl = cfh[a];
                const float fac = tl != tm ? 2.f : 1.f;
                ff_mac(S, E, fac * cl.x, fac * cl.y, SA);
                E += fac * cl.x * EA;
                ff_mac(S, E, fac * cl.z, fac * cl.w, SB);
                E += fac * cl.z * EB;
            }
            if (toX && !off && et < 64 && et < nl && !I.local) {  // delta~_l and its product with c~_l
                const int gl = tl * TT + et;
                const float2 du = XD[et], dl = XD[64 + et];
                const float dsc = 1.f / (TC_SCALE * tc_bscale(*I.bn2));  // exact: a power of two
                const float2 dacc = make_float2((du.x + dl.x) * dsc, -(du.y + dl.y) * dsc);  // conj(b) phi
                const float4 cv = cfh[et];  // c~_l as (Re hi, Re lo, Im hi, Im lo)
                ff_mac(TrS, TrE, cv.x, cv.y, dacc.x);
                ff_mac(TrS, TrE, -cv.z, -cv.w, dacc.y);
                ff_mac(TiS, TiE, cv.x, cv.y, dacc.y);
                ff_mac(TiS, TiE, cv.z, cv.w, dacc.x);
                if (s == 0 && I.dpart) reinterpret_cast<float2*>(I.dpart)[(long long)ksi * L + gl] = dacc;
            }
            ff_warp_sum(S, E);
            ff_warp_sum(TrS, TrE);
            ff_warp_sum(TiS, TiE);
            if (lane == 0) {
                sred[0][0][ew] = S;
                sred[0][1][ew] = E;
                sred[1][0][ew] = TrS;
                sred[1][1][ew] = TrE;
                sred[2][0][ew] = TiS;
                sred[2][1][ew] = TiE;
            }
            bar_n(3, TC_ET);
            if (et == 0) {  // FP64 only for the final pairs, added in a fixed order
                double qv[3];
                for (int k = 0; k < 3; ++k) {
                    float S2 = 0.f, E2 = 0.f;
                    for (int v = 0; v < TC_EW; ++v) {
                        ff_add(S2, E2, sred[k][0][v]);
                        E2 += sred[k][1][v];
                    }
                    qv[k] = (double)S2 + (double)E2;
                }
                // slots as the CUDA-core tiles use them: diagonal tile u at u, pair p at
                // T + 2p (and T + 2p + 1, which the tiles use for the pair's second half);
                // per flavour f of the local cost: slots (s F + f) T^2 ..
                const long long slot2 = ((long long)s * I.F + f) * T * T + (tl != tm ? T + 2 * (u - T) : u);
                I.Dpart[slot2 * ks + ksi] = make_double2(qv[0] * (double)TC_UNSCALE, 0.0);
                if (tl != tm) I.Dpart[(slot2 + 1) * ks + ksi] = make_double2(0.0, 0.0);
                else if (f == 0 && !I.local) I.Tpart[((long long)s * T + tl) * ks + ksi] = make_double2(qv[1], qv[2]);
                // the half's item record is free again
                mbar_arrive(su32(&ite[pick][r[pick]]));
                r[pick] = (r[pick] + 1) % TC_NIT;
                have &= ~(1u << pick);
            }
            bar_n(3, TC_ET);  // X, sred and s_cur are free again
        }
        asm volatile("cp.async.wait_all;" ::: "memory");  // no copy into shared memory outlives the CTA
        if (ab) s_abort = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (t == 0 && s_abort) atomicCAS(status, 0, DEV_TIMEOUT);
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(TC_COLS));
}

// ------------------------------------------- Walsh-Hadamard term classes
// Precision DVQLS_FP32_WHT, an exact reformulation of the term reductions
// (the same terms of Sec. 2.2, evaluated by class with fewer operations).  With
// the real state and the phases in c~ (as in the tile kernels),
//   G~_lm = (-1)^popc(z_l & x) W_x(z_l ^ z_m),  x = x_l ^ x_m,
//   W_x(z) = sum_i (-1)^popc(z & i) psi[i] psi[i ^ x],
// so one Walsh-Hadamard transform of g_x(i) = psi[i] psi[i ^ x] gives the
// terms of every pair (l, m) in the class of x; likewise
//   delta_l = sum_i (-1)^popc(z_l & i) conj(b[i ^ x_l]) psi[i]
// is entry z_l of the transform of h(i) = conj(b[i ^ x_l]) psi[i], one per
// distinct x_l.  A banded Toeplitz LCU has few classes (n = 10, top 64:
// 22 pair classes, 7 term classes), against 2,080 pair reductions.
// One CTA of 8 warps per item (instance, shift); a warp transforms one class
// at a time with the vector in registers (n <= 10: 2^n / 32 values per lane;
// register bits butterfly in place, lane bits by shuffles or, at n = 10,
// through the warp's padded shared-memory row), leaves it in that row and
// looks up the class's terms.  Weighted sums in
// float-float, FP64 across warps.  Served for the global cost when every
// instance has L <= 64 and n <= 10.
constexpr int WHT_MAXP = 64 * 65 / 2;  // pairs l <= m of a 64-term LCU
constexpr int WHT_NT = 256;
constexpr int WHT_MAXN = 10;
constexpr int WHT_CT = 1024;  // threads of the class-table kernel
// Per-instance class table, built on the device by k_wht_classes (bytes):
constexpr size_t WHT_OFF_CX = 16;                                   // uint32 class masks [WHT_MAXP]
constexpr size_t WHT_OFF_CO = WHT_OFF_CX + 4 * WHT_MAXP;            // int class offsets [WHT_MAXP + 1]
constexpr size_t WHT_OFF_PR = WHT_OFF_CO + 4 * (WHT_MAXP + 1);      // uint16 pairs l | m << 8 by class
constexpr size_t WHT_OFF_DX = (WHT_OFF_PR + 2 * WHT_MAXP + 15) & ~size_t(15);  // uint32 term-class masks [64]
constexpr size_t WHT_OFF_DO = WHT_OFF_DX + 4 * 64;                  // int term-class offsets [65]
constexpr size_t WHT_OFF_DT = WHT_OFF_DO + 4 * 65;                  // uint16 terms by class [64]
constexpr size_t WHT_OFF_EZ = (WHT_OFF_DT + 2 * 64 + 15) & ~size_t(15);  // uint16 z_l ^ z_m by class
constexpr size_t WHT_OFF_EK = (WHT_OFF_EZ + 2 * WHT_MAXP + 15) & ~size_t(15);  // float2 signed weights by class
constexpr size_t WHT_OFF_KEY = WHT_OFF_EK + 8 * WHT_MAXP;  // the inputs the table was built from: int L,
                                                              // uint32 x[64], z[64], double2 coef[64]
constexpr size_t WHT_OFF_SUM = WHT_OFF_KEY + 16 + 8 * 64 + 16 * 64;  // uint64 checksum of bytes [0, WHT_OFF_SUM)
constexpr size_t WHT_OFF_BIM = WHT_OFF_SUM + 8;  // int: b has a nonzero imaginary part (rewritten every call)
constexpr size_t WHT_TABLE_BYTES = WHT_OFF_SUM + 16;                   // header: int pair classes, term classes

// 64-bit checksum of a table (sum of mixed, position-tagged 32-bit words;
// valid in every thread of the block).
__device__ inline unsigned long long wht_checksum(const unsigned char* tb, unsigned long long* red) {
    const uint32_t* wds = reinterpret_cast<const uint32_t*>(tb);
    unsigned long long h = 0;
    for (int i = threadIdx.x; i < int(WHT_OFF_SUM / 4); i += blockDim.x) {
        unsigned long long z = ((unsigned long long)wds[i] | ((unsigned long long)i << 32)) + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        h += z ^ (z >> 31);
    }
    for (int o = 16; o; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = h;
    __syncthreads();
    unsigned long long s = 0;
    for (int k = 0; k < int(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

// Class tables of one instance (one CTA of 256 per instance): pairs (l <= m)
// sorted by x_l ^ x_m (bitonic sort of (mask, pair) keys), each with its
// transform index z_l ^ z_m and its weight (-1)^popc(z_l & x) Re(w_lm),
// doubled for l < m, as a float pair; terms by x_l; and b as float2.  Runs
// after k_prepare (which forms the weights).
__global__ void __launch_bounds__(WHT_CT) k_wht_classes(const Inst* __restrict__ insts) {
    pdl_wait();
    pdl_trigger();
    const Inst I = insts[blockIdx.x];
    if (!I.wht) return;
    __shared__ unsigned long long key[4096];
    __shared__ uint32_t sx[64], sz[64];
    unsigned char* tb = reinterpret_cast<unsigned char*>(I.wht);
    const int L = I.L, t = threadIdx.x, np = L * (L + 1) / 2;
    const long long N = 1LL << I.n;
    bool im = false;
    for (long long j = t; I.b && j < N; j += WHT_CT) {  // the local cost has no b here (|+>^n is implied)
        const double2 v = I.b[j];
        I.bf[j] = make_float2((float)v.x, (float)v.y);
        im |= (float)v.y != 0.f;
    }
    if (__syncthreads_or(im) != 0) {
        if (t == 0) *reinterpret_cast<int*>(tb + WHT_OFF_BIM) = 1;
    } else if (t == 0) {
        *reinterpret_cast<int*>(tb + WHT_OFF_BIM) = 0;
    }
    if (t < 64) {
        sx[t] = t < L ? I.xm[t] : 0u;
        sz[t] = t < L ? I.zm[t] : 0u;
    }
    // The table is a function of L, the masks and the coefficients alone: when
    // the copy kept with it matches them exactly, it is still valid.
    int* kL = reinterpret_cast<int*>(tb + WHT_OFF_KEY);
    uint32_t* kx = reinterpret_cast<uint32_t*>(tb + WHT_OFF_KEY + 16);
    uint32_t* kz = kx + 64;
    double2* kc = reinterpret_cast<double2*>(tb + WHT_OFF_KEY + 16 + 8 * 64);
    bool differs = false;
    if (t < L) {
        const double2 c = I.coef[t], k = kc[t];
        differs = kx[t] != I.xm[t] || kz[t] != I.zm[t] || __double_as_longlong(c.x) != __double_as_longlong(k.x) ||
                  __double_as_longlong(c.y) != __double_as_longlong(k.y);
    }
    if (t == 0 && *kL != L) differs = true;
    __shared__ unsigned long long red[WHT_CT / 32];
    unsigned long long* ksum = reinterpret_cast<unsigned long long*>(tb + WHT_OFF_SUM);
    if (!__syncthreads_or(differs) && wht_checksum(tb, red) == *ksum) return;  // still valid, untouched
    for (int e = np + t; e < 4096; e += WHT_CT) key[e] = ~0ull;
    __syncthreads();
    for (int q = t; q < L * L; q += WHT_CT) {  // pair (l, m), l <= m, at e = l L - l (l - 1) / 2 + m - l
        const int l = q / L, m = q % L;
        if (l <= m)
            key[l * L - l * (l - 1) / 2 + (m - l)] =
                ((unsigned long long)(sx[l] ^ sx[m]) << 16) | (unsigned long long)(l | (m << 8));
    }
    __syncthreads();
    for (int k = 2; k <= 4096; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int e = t; e < 4096; e += WHT_CT) {
                const int p = e ^ j;
                if (p > e) {
                    const unsigned long long a = key[e], b = key[p];
                    if (((e & k) == 0) == (a > b)) {
                        key[e] = b;
                        key[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    // Class numbers: a class starts where the mask changes; its number is the
    // count of starts up to it (block prefix sum over 4096 / WHT_CT keys per
    // thread).
    constexpr int PER = 4096 / WHT_CT, LANE_N = WHT_CT / 32;
    __shared__ int tsum[WHT_CT];
    uint32_t* cx = reinterpret_cast<uint32_t*>(tb + WHT_OFF_CX);
    int* co = reinterpret_cast<int*>(tb + WHT_OFF_CO);
    uint16_t* pr = reinterpret_cast<uint16_t*>(tb + WHT_OFF_PR);
    const int e0 = t * PER;
    int cnt = 0;
    for (int e = e0; e < e0 + PER; ++e)
        if (e < np && (e == 0 || uint32_t(key[e] >> 16) != uint32_t(key[e - 1] >> 16))) ++cnt;
    tsum[t] = cnt;
    __syncthreads();
    if (t < 32) {  // exclusive scan of the per-thread counts by one warp (LANE_N per lane)
        int v[LANE_N], run = 0;
        for (int q = 0; q < LANE_N; ++q) {
            v[q] = run;
            run += tsum[t * LANE_N + q];
        }
        int incl = run;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (t >= o) incl += y;
        }
        const int base = incl - run;
        for (int q = 0; q < LANE_N; ++q) tsum[t * LANE_N + q] = base + v[q];
        if (t == 31) reinterpret_cast<int*>(tb)[0] = incl;  // number of pair classes
    }
    __syncthreads();
    int cid = tsum[t];
    for (int e = e0; e < e0 + PER && e < np; ++e) {
        const uint32_t x = uint32_t(key[e] >> 16);
        if (e == 0 || x != uint32_t(key[e - 1] >> 16)) {
            cx[cid] = x;
            co[cid] = e;
            ++cid;
        }
        const int p = int(key[e] & 0xFFFFu), l = p & 0xFF, m = p >> 8;
        pr[e] = uint16_t(p);
        const uint32_t zl = sz[l], zm = sz[m];
        reinterpret_cast<uint16_t*>(tb + WHT_OFF_EZ)[e] = uint16_t((zl ^ zm) & uint32_t(N - 1));
        const float4 wv = I.wf[l * L + m];
        const float sg = ((__popc(zl & x) & 1) ? -1.f : 1.f) * (l < m ? 2.f : 1.f);  // exact scaling
        reinterpret_cast<float2*>(tb + WHT_OFF_EK)[e] = make_float2(sg * wv.x, sg * wv.y);
    }
    if (t == WHT_CT - 1) co[tsum[WHT_CT - 1] + cnt] = np;  // the end of the last class
    __shared__ int sfirst[64];  // term k is the first with its mask
    if (t < L) {
        bool f = true;
        for (int q = 0; q < t && f; ++q) f = sx[q] != sx[t];
        sfirst[t] = f ? 1 : 0;
    }
    __syncthreads();
    if (t < L) {  // term classes by x_l: rank and class number of term l from counts
        uint32_t* dx = reinterpret_cast<uint32_t*>(tb + WHT_OFF_DX);
        int* dof = reinterpret_cast<int*>(tb + WHT_OFF_DO);
        uint16_t* dt = reinterpret_cast<uint16_t*>(tb + WHT_OFF_DT);
        const uint32_t xl = sx[t];
        int below = 0, rank = 0, cls = 0, nd = 0;
        bool first = true;
        for (int k = 0; k < L; ++k) {
            const uint32_t xk = sx[k];
            const bool kfirst = sfirst[k] != 0;
            if (xk < xl) {
                ++below;
                if (kfirst) ++cls;
            }
            if (xk < xl || (xk == xl && k < t)) ++rank;
            if (xk == xl && k < t) first = false;
            if (kfirst) ++nd;
        }
        dt[rank] = uint16_t(t);
        if (first) {
            dx[cls] = xl;
            dof[cls] = below;
        }
        if (t == 0) {
            dof[nd] = L;
            reinterpret_cast<int*>(tb)[1] = nd;
        }
    }
    __syncthreads();  // the table is complete: record what it was built from
    if (t < L) {
        kx[t] = I.xm[t];
        kz[t] = I.zm[t];
        kc[t] = I.coef[t];
    }
    if (t == 0) *kL = L;
    __syncthreads();  // every word of the table is written
    const unsigned long long sum = wht_checksum(tb, red);
    if (t == 0) *ksum = sum;
}

// Unnormalised Walsh-Hadamard transform of a warp's vector, v[r] at index
// (r << 5) | lane (n >= 5), or lane mod 2^n (n < 5, lanes repeat it):
// butterflies (a, b) -> (a + b, a - b) on every index bit.
template <int A, int LOGA>
__device__ __forceinline__ void wht_warp(float (&v)[A], int lane, int nl) {
#pragma unroll
    for (int kb = 0; kb < LOGA; ++kb)
#pragma unroll
        for (int r = 0; r < A; ++r)
            if (!((r >> kb) & 1)) {
                const float a = v[r], b = v[r | (1 << kb)];
                v[r] = a + b;
                v[r | (1 << kb)] = a - b;
            }
    for (int b = 0; b < nl; ++b)
#pragma unroll
        for (int r = 0; r < A; ++r) {
            const float p = __shfl_xor_sync(0xffffffffu, v[r], 1 << b);
            v[r] = ((lane >> b) & 1) ? p - v[r] : v[r] + p;
        }
}

// The same transform for 2^10 values (32 per lane) without shuffles: the
// register bits butterfly in place, the vector goes through the warp's row
// (stride 33, conflict-free both ways) so that lane L holds the 32 values whose
// index has high bits L, and the other five bits butterfly in place too.  The
// result is left in the row at the padded position i + (i >> 5).
__device__ __forceinline__ void wht_warp_1024(float (&v)[32], int lane, float* row) {
#pragma unroll
    for (int kb = 0; kb < 5; ++kb)
#pragma unroll
        for (int r = 0; r < 32; ++r)
            if (!((r >> kb) & 1)) {
                const float a = v[r], b = v[r | (1 << kb)];
                v[r] = a + b;
                v[r | (1 << kb)] = a - b;
            }
#pragma unroll
    for (int r = 0; r < 32; ++r) row[r * 33 + lane] = v[r];  // index (r << 5) | lane
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = row[lane * 33 + j];  // index (lane << 5) | j
    __syncwarp();
#pragma unroll
    for (int kb = 0; kb < 5; ++kb)
#pragma unroll
        for (int r = 0; r < 32; ++r)
            if (!((r >> kb) & 1)) {
                const float a = v[r], b = v[r | (1 << kb)];
                v[r] = a + b;
                v[r | (1 << kb)] = a - b;
            }
#pragma unroll
    for (int j = 0; j < 32; ++j) row[lane * 33 + j] = v[j];  // index (lane << 5) | j at i + (i >> 5)
}

// One item: every pair class, then every term class, of one shifted state.
// The transform of g_x(i) = psi[i] psi[i ^ x] into the warp's row (at
// i + (i >> 5) for 2^10 values, else at i).
template <int A, int LOGA>
__device__ __forceinline__ void wht_row(const float* psi, uint32_t x, float* wb, int N, int lane) {
    const int lm = N < 32 ? N - 1 : 31, nl = N < 32 ? __ffs(N) - 1 : 5;
    float v[A];
#pragma unroll
    for (int r = 0; r < A; ++r) {
        const int i = (r << 5) | (lane & lm);
        v[r] = psi[i] * psi[(i ^ int(x)) & (N - 1)];
    }
    if constexpr (A == 32) {
        wht_warp_1024(*reinterpret_cast<float(*)[32]>(v), lane, wb);
    } else {
        wht_warp<A, LOGA>(v, lane, nl);
        if (lane < N || N >= 32) {
#pragma unroll
            for (int r = 0; r < A; ++r) wb[(r << 5) | lane] = v[r];
        }
    }
    __syncwarp();
}

// Local cost (Eq. 2/4, b = |+>^n): with X_j inserted between the two terms,
//   gamma~^j_lm = sum_i phi_l[i] phi_m[i ^ e_j] = (-1)^popc(z_l & X) W_X(z_l ^ z_m),
//   X = x_l ^ x_m ^ e_j,
// so the pairs of the class of x serve flavour j through the transform at
// x ^ e_j, with the sign of the class's weight flipped where bit j of z_l is
// set.  Jobs are (flavour, class): flavour 0 forms D (the global terms),
// flavours 1..n form E.
template <int A, int LOGA>
__device__ void wht_item_local(const Inst& I, const float* psi, float* wb, const uint32_t* szl, float& S, float& E,
                               float& SL, float& EL, int lane) {
    constexpr bool PAD = A == 32;
    const int n = I.n, N = 1 << n, w = threadIdx.x >> 5;
    const unsigned char* tb = reinterpret_cast<const unsigned char*>(I.wht);
    const int ncls = reinterpret_cast<const int*>(tb)[0];
    const uint32_t* cx = reinterpret_cast<const uint32_t*>(tb + WHT_OFF_CX);
    const int* co = reinterpret_cast<const int*>(tb + WHT_OFF_CO);
    const uint16_t* pr = reinterpret_cast<const uint16_t*>(tb + WHT_OFF_PR);
    const uint16_t* ez = reinterpret_cast<const uint16_t*>(tb + WHT_OFF_EZ);
    const float2* ek = reinterpret_cast<const float2*>(tb + WHT_OFF_EK);
    const int jobs = ncls * (n + 1);
#pragma unroll 1
    for (int job = w; job < jobs; job += WHT_NT / 32) {
        const int f = job / ncls, c = job - f * ncls;
        const uint32_t x = cx[c] ^ (f ? 1u << (f - 1) : 0u);
        wht_row<A, LOGA>(psi, x, wb, N, lane);
        const int e0 = co[c], e1 = co[c + 1];
        if (f == 0) {
            for (int e = e0 + lane; e < e1; e += 32) {
                const uint32_t z = ez[e];
                const float2 k = ek[e];
                ff_mac(S, E, k.x, k.y, wb[PAD ? z + (z >> 5) : z]);
            }
        } else {
            for (int e = e0 + lane; e < e1; e += 32) {
                const uint32_t z = ez[e];
                float2 k = ek[e];
                if ((szl[pr[e] & 0xFF] >> (f - 1)) & 1u) k = make_float2(-k.x, -k.y);
                ff_mac(SL, EL, k.x, k.y, wb[PAD ? z + (z >> 5) : z]);
            }
        }
        __syncwarp();
    }
}

template <int A, int LOGA>
__device__ void wht_item(const Inst& I, int s, const float* psi, const float2* sb, float* wb, float* dre, float* dim,
                         const uint32_t* szl, float& S, float& E, int lane) {
    constexpr bool PAD = A == 32;  // the 2^10 transform leaves its result at i + (i >> 5)
    const int n = I.n, N = 1 << n, L = I.L, w = threadIdx.x >> 5, nl = n < 5 ? n : 5;
    const int lm = N < 32 ? N - 1 : 31;
    const unsigned char* tb = reinterpret_cast<const unsigned char*>(I.wht);
    const int ncls = reinterpret_cast<const int*>(tb)[0], nd = reinterpret_cast<const int*>(tb)[1];
    const uint32_t* cx = reinterpret_cast<const uint32_t*>(tb + WHT_OFF_CX);
    const int* co = reinterpret_cast<const int*>(tb + WHT_OFF_CO);
    const uint16_t* pr = reinterpret_cast<const uint16_t*>(tb + WHT_OFF_PR);
    const uint16_t* ez = reinterpret_cast<const uint16_t*>(tb + WHT_OFF_EZ);
    const float2* ek = reinterpret_cast<const float2*>(tb + WHT_OFF_EK);
    float2* Gp = (s == 0 && I.Gpart) ? reinterpret_cast<float2*>(I.Gpart) : nullptr;
    const uint32_t* dx = reinterpret_cast<const uint32_t*>(tb + WHT_OFF_DX);
    const int* dof = reinterpret_cast<const int*>(tb + WHT_OFF_DO);
    const uint16_t* dt = reinterpret_cast<const uint16_t*>(tb + WHT_OFF_DT);
    // One list of transforms for the warps: the pair classes, then the term
    // classes (Re, and Im when b has an imaginary part: dim stays zero else).
    const int parts = 1 + *reinterpret_cast<const int*>(tb + WHT_OFF_BIM);
    const int jobs = ncls + nd * parts;
#pragma unroll 1
    for (int j = w; j < jobs; j += WHT_NT / 32) {
        if (j >= ncls) {
            const int c = (j - ncls) / parts, part = (j - ncls) - c * parts, x = int(dx[c]);
            float v[A];  // h(i) = conj(b[i ^ x]) psi[i], its real or imaginary part
#pragma unroll
            for (int r = 0; r < A; ++r) {
                const int i = (r << 5) | (lane & lm);
                const float2 bb = sb[(i ^ x) & (N - 1)];
                v[r] = (part ? -bb.y : bb.x) * psi[i];
            }
            if constexpr (A == 32) {
                wht_warp_1024(*reinterpret_cast<float(*)[32]>(v), lane, wb);
            } else {
                wht_warp<A, LOGA>(v, lane, nl);
                if (lane < N || N >= 32) {
#pragma unroll
                    for (int r = 0; r < A; ++r) wb[(r << 5) | lane] = v[r];
                }
            }
            __syncwarp();
            for (int e = dof[c] + lane; e < dof[c + 1]; e += 32) {
                const int l = dt[e];
                const uint32_t zz = szl[l] & uint32_t(N - 1);
                (part ? dim : dre)[l] = wb[PAD ? zz + (zz >> 5) : zz];
            }
            __syncwarp();
            continue;
        }
        const int c = j;
        const uint32_t x = cx[c];
        float v[A];
#pragma unroll
        for (int r = 0; r < A; ++r) {
            const int i = (r << 5) | (lane & lm);
            v[r] = psi[i] * psi[(i ^ int(x)) & (N - 1)];  // masks >= 2^n are reported, never followed
        }
        if constexpr (A == 32) {
            wht_warp_1024(*reinterpret_cast<float(*)[32]>(v), lane, wb);
        } else {
            wht_warp<A, LOGA>(v, lane, nl);
            if (lane < N || N >= 32) {
#pragma unroll
                for (int r = 0; r < A; ++r) wb[(r << 5) | lane] = v[r];
            }
        }
        __syncwarp();
        const int e0 = co[c], e1 = co[c + 1];
        for (int e = e0 + lane; e < e1; e += 4 * 32) {  // four independent lookups per lane in flight
            uint32_t z[4];
            float2 k[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int eq = e + 32 * q;
                z[q] = eq < e1 ? ez[eq] : 0u;
                k[q] = eq < e1 ? ek[eq] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) ff_mac(S, E, k[q].x, k[q].y, wb[PAD ? z[q] + (z[q] >> 5) : z[q]]);
        }
        if (Gp)  // the beta output of the unshifted state
            for (int e = e0 + lane; e < e1; e += 32) {
                const int p = pr[e], l = p & 0xFF, m = p >> 8;
                const uint32_t ze = ez[e];
                float beta = wb[PAD ? ze + (ze >> 5) : ze];
                if (__popc(szl[l] & x) & 1) beta = -beta;
                Gp[(long long)l * L + m] = make_float2(beta, 0.f);
                Gp[(long long)m * L + l] = make_float2(beta, 0.f);
            }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(WHT_NT, 4) k_terms_wht(const Inst* __restrict__ insts, int count, long long total,
                                                      unsigned long long* queue) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t szl[TT];
    __shared__ float dre[TT], dim[TT];
    __shared__ double red[WHT_NT / 32];
    __shared__ long long s_item;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    constexpr int ROW = (1 << WHT_MAXN) + (1 << WHT_MAXN) / 32;      // a transform row, padded
    float* psi = reinterpret_cast<float*>(smem);                       // 2^WHT_MAXN
    float* wb = psi + (1 << WHT_MAXN) + w * ROW;                       // this warp's transform row
    float* scratch = psi + (1 << WHT_MAXN) + 8 * ROW;                  // state transposes
    float2* sb = reinterpret_cast<float2*>(scratch + 2 * ((1 << WHT_MAXN) + (1 << WHT_MAXN) / 32));  // b, FP32
    float2* scs = sb + (1 << WHT_MAXN);
    for (;;) {
        if (t == 0) s_item = (long long)atomicAdd(queue, 1ull);
        __syncthreads();
        const long long gi = s_item;
        __syncthreads();
        if (gi >= total) break;
        const Inst& I = insts[find_instance(insts, count, gi)];
        const int s = int(gi - I.item_base), L = I.L;
        if (t < TT) {
            szl[t] = t < L ? I.zm[t] : 0u;
            dre[t] = dim[t] = 0.f;
        }
        for (int j = t; !I.local && j < (1 << I.n); j += WHT_NT) sb[j] = I.bf[j];
        build_state_regs<false>(psi, scratch, scs, I.n, I.d, I.P, I.cs, s + I.s0, t, 0, 1.f);  // ends with a barrier
        float S = 0.f, E = 0.f;
        if (I.local) {
            float SL = 0.f, EL = 0.f;
            switch (I.n) {
                case 10: wht_item_local<32, 5>(I, psi, wb, szl, S, E, SL, EL, lane); break;
                case 9: wht_item_local<16, 4>(I, psi, wb, szl, S, E, SL, EL, lane); break;
                case 8: wht_item_local<8, 3>(I, psi, wb, szl, S, E, SL, EL, lane); break;
                case 7: wht_item_local<4, 2>(I, psi, wb, szl, S, E, SL, EL, lane); break;
                case 6: wht_item_local<2, 1>(I, psi, wb, szl, S, E, SL, EL, lane); break;
                default: wht_item_local<1, 0>(I, psi, wb, szl, S, E, SL, EL, lane); break;  // n <= 5
            }
            // Slot 0 of a shift holds D, slot 1 E (summed over the flavours), the rest zero.
            const double D = block_sum_ff(S, E, red);
            const double El = block_sum_ff(SL, EL, red);
            if (t == 0) {  // the sums are valid in thread 0
                I.Dpart[(long long)s * I.F] = make_double2(D, 0.0);
                I.Dpart[(long long)s * I.F + 1] = make_double2(El, 0.0);
            } else if (t >= 2 && t < I.F) {
                I.Dpart[(long long)s * I.F + t] = make_double2(0.0, 0.0);
            }
            __syncthreads();
            continue;
        }
        switch (I.n) {
            case 10: wht_item<32, 5>(I, s, psi, sb, wb, dre, dim, szl, S, E, lane); break;
            case 9: wht_item<16, 4>(I, s, psi, sb, wb, dre, dim, szl, S, E, lane); break;
            case 8: wht_item<8, 3>(I, s, psi, sb, wb, dre, dim, szl, S, E, lane); break;
            case 7: wht_item<4, 2>(I, s, psi, sb, wb, dre, dim, szl, S, E, lane); break;
            case 6: wht_item<2, 1>(I, s, psi, sb, wb, dre, dim, szl, S, E, lane); break;
            default: wht_item<1, 0>(I, s, psi, sb, wb, dre, dim, szl, S, E, lane); break;  // n <= 5
        }
        __syncthreads();
        float TrS = 0.f, TrE = 0.f, TiS = 0.f, TiE = 0.f;
        if (t < L) {
            const float4 cv = I.cf[t];  // c~_l as (Re hi, Re lo, Im hi, Im lo)
            const float dr = dre[t], di = dim[t];
            ff_mac(TrS, TrE, cv.x, cv.y, dr);
            ff_mac(TrS, TrE, -cv.z, -cv.w, di);
            ff_mac(TiS, TiE, cv.x, cv.y, di);
            ff_mac(TiS, TiE, cv.z, cv.w, dr);
            if (s == 0 && I.dpart) reinterpret_cast<float2*>(I.dpart)[t] = make_float2(dr, di);
        }
        const double D = block_sum_ff(S, E, red);
        const double tr = block_sum_ff(TrS, TrE, red);
        const double ti = block_sum_ff(TiS, TiE, red);
        if (t == 0) {
            I.Dpart[s] = make_double2(D, 0.0);
            I.Tpart[s] = make_double2(tr, ti);
        }
        __syncthreads();
    }
}

// Shared bytes of the Walsh-Hadamard term kernel (states up to 2^10, Pmax angles).
inline size_t wht_smem_bytes(int Pmax) {
    const size_t N = size_t(1) << WHT_MAXN;
    return 4 * (N + 8 * (N + N / 32) + 2 * (N + N / 32)) + 8 * N + 8 * (size_t)Pmax;
}

// ---------------------------------------------------------------- combine
template <typename R>
__global__ void __launch_bounds__(NT) k_combine(const Inst* __restrict__ insts, int* status) {
    pdl_wait();
    using R2 = typename V2<R>::t;
    const Inst I = insts[blockIdx.x];
    const int t = threadIdx.x, T = I.T, ks = I.ks, L = I.L;
    const double bn2 = *I.bn2;
    for (int s = t; s < I.S; s += NT) {
        double2 D = make_double2(0.0, 0.0), Tv = make_double2(0.0, 0.0);
        const double2* dp = I.Dpart + (long long)s * I.F * T * T * ks;
        for (int e = 0; e < T * T * ks; ++e) {
            D.x += dp[e].x;
            D.y += dp[e].y;
        }
        if (I.local) {  // E_s = sum over the gamma flavors (real parts)
            double E = 0.0;
            for (int e = T * T * ks; e < I.F * T * T * ks; ++e) E += dp[e].x;
            I.NsDs[3 * s] = E;
            I.NsDs[3 * s + 1] = D.x;
            I.NsDs[3 * s + 2] = D.y;
            continue;
        }
        const double2* tp = I.Tpart + (long long)s * T * ks;
        for (int e = 0; e < T * ks; ++e) {
            Tv.x += tp[e].x;
            Tv.y += tp[e].y;
        }
        I.NsDs[3 * s] = (Tv.x * Tv.x + Tv.y * Tv.y) / bn2;
        I.NsDs[3 * s + 1] = D.x;
        I.NsDs[3 * s + 2] = D.y;
    }
    __syncthreads();
    const double N0 = I.NsDs[0], D0 = I.NsDs[1];
    // Global cost: C = 1 - N/D.  Local cost: C_L = 1/2 - E / (2 n D) (N holds E).
    const double scale = I.local ? 0.5 / I.n : 1.0;
    if (t == 0) {
        if (!(D0 > 0.0) || !isfinite(D0) || !isfinite(N0)) set_status(status, DEV_BAD_DENOMINATOR);
        *I.cost = (I.local ? 0.5 : 1.0) - scale * N0 / D0;
    }
    if (I.grad && I.S > 1)
        for (int k = t; k < I.P; k += NT) {
            const double dN = 0.5 * (I.NsDs[3 * (2 * k + 1)] - I.NsDs[3 * (2 * k + 2)]);
            const double dD = 0.5 * (I.NsDs[3 * (2 * k + 1) + 1] - I.NsDs[3 * (2 * k + 2) + 1]);
            I.grad[k] = -scale * (dN * D0 - N0 * dD) / (D0 * D0);
        }
    if (I.beta) {
        const R2* G = reinterpret_cast<const R2*>(I.Gpart);
        const long long LL = (long long)L * L;
        for (long long e = t; e < LL; e += NT) {
            double gr = 0.0, gi = 0.0;
            for (int k = 0; k < ks; ++k) {
                gr += (double)G[k * LL + e].x;
                gi += (double)G[k * LL + e].y;
            }
            const int l = int(e / L), m = int(e % L);
            const int r = ((__popc(I.xm[m] & I.zm[m]) - __popc(I.xm[l] & I.zm[l])) % 4 + 4) % 4;
            double2 v;
            if (r == 0) v = make_double2(gr, gi);
            else if (r == 1) v = make_double2(-gi, gr);
            else if (r == 2) v = make_double2(-gr, -gi);
            else v = make_double2(gi, -gr);
            I.beta[e] = v;
        }
    }
    if (I.delta) {
        const R2* dpp = reinterpret_cast<const R2*>(I.dpart);
        const double inv = 1.0 / sqrt(bn2);
        for (int l = t; l < L; l += NT) {
            double vr = 0.0, vi = 0.0;
            for (int k = 0; k < ks; ++k) {
                vr += (double)dpp[(long long)k * L + l].x;
                vi += (double)dpp[(long long)k * L + l].y;
            }
            double2 v;
            switch (__popc(I.xm[l] & I.zm[l]) & 3) {
                case 0: v = make_double2(vr, vi); break;
                case 1: v = make_double2(-vi, vr); break;
                case 2: v = make_double2(-vr, -vi); break;
                default: v = make_double2(vi, -vr); break;
            }
            I.delta[l] = make_double2(v.x * inv, v.y * inv);
        }
    }
}

// Stage III of Sec. 2.3 across ranks (Algorithm 1, Step 4c): the per-shift
// partial sums of a pass over the shift range s0 .. s0 + S - 1 of one
// instance.  out[4 g .. 4 g + 3] = (Re T, Im T, Re D, Im D) of the instance's
// shift g, with T = sum_l c_l delta_l for the normalised b and
// D = sum_lm conj(c_l) c_m beta_lm; zeros for the shifts outside the range,
// so the arrays of ranks that cover disjoint ranges add up (one SUM
// allreduce) to the whole instance's.
__global__ void __launch_bounds__(NT) k_partials(const Inst* __restrict__ insts, int S_full, double* out) {
    pdl_wait();
    const Inst& I = insts[0];
    const int T = I.T, ks = I.ks;
    const double inv = 1.0 / sqrt(*I.bn2);
    for (int g = threadIdx.x; g < S_full; g += NT) {
        const int s = g - I.s0;
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        if (s >= 0 && s < I.S) {
            const double2* dp = I.Dpart + (long long)s * T * T * ks;
            for (int e = 0; e < T * T * ks; ++e) {
                v[2] += dp[e].x;
                v[3] += dp[e].y;
            }
            const double2* tp = I.Tpart + (long long)s * T * ks;
            for (int e = 0; e < T * ks; ++e) {
                v[0] += tp[e].x;
                v[1] += tp[e].y;
            }
            v[0] *= inv;
            v[1] *= inv;
        }
        for (int k = 0; k < 4; ++k) out[4 * g + k] = v[k];
    }
}

// Cost and parameter-shift gradient from the reduced per-shift sums of
// k_partials (all 2P + 1 shifts): N_s = |T_s|^2, C = 1 - N_0 / D_0 and
// dC/dalpha_k = -(N'_k D_0 - N_0 D'_k) / D_0^2 (Eq. 1; the shift rule).
__global__ void __launch_bounds__(NT) k_combine_partials(const double* __restrict__ part, int P, int* status,
                                                         double* cost, double* grad) {
    const int t = threadIdx.x;
    const double N0 = part[0] * part[0] + part[1] * part[1], D0 = part[2];
    if (t == 0) {
        if (!(D0 > 0.0) || !isfinite(D0) || !isfinite(N0)) set_status(status, DEV_BAD_DENOMINATOR);
        *cost = 1.0 - N0 / D0;
    }
    for (int k = t; k < P; k += NT) {
        const double* a = part + 4 * (2 * k + 1);
        const double* b = part + 4 * (2 * k + 2);
        const double dN = 0.5 * ((a[0] * a[0] + a[1] * a[1]) - (b[0] * b[0] + b[1] * b[1]));
        const double dD = 0.5 * (a[2] - b[2]);
        grad[k] = -(dN * D0 - N0 * dD) / (D0 * D0);
    }
}

// ------------------------------------------------------------------- host
struct HostInst {
    int n, d, L, P, S, T, ks, F;
    long long N;
    int order;  // position in the caller's array
    bool hbm;   // n > 12: states built in HBM
};



template <typename R>
size_t smem_bytes(int nmax, int Pmax) {  // real state (padded to 4 values), two real chunks, b chunk, angles
    using R2 = typename V2<R>::t;
    return sizeof(R) * (((size_t(1) << nmax) + 3) & ~size_t(3)) + sizeof(R) * (2 * JC * TT) + sizeof(R2) * JC +
           sizeof(R2) * Pmax;
}

// Launch parameters of one cost pass (everything but the table contents).
struct PassShape {
    int fp32, tc, wht, count, grid;
    long long total;
    size_t smem;
    int copy_nmax;   // tensor-core kernel: states of 2^4 .. 2^copy_nmax amplitudes kept in four copies (0: none)
    int split_nmax;  // tensor-core kernel: states of 2^split_nmin .. 2^split_nmax amplitudes kept as split
    int split_nmin;  // hi / lo arrays (split_nmax 0: none)
    int psi_region;  // tensor-core kernel: shared bytes of a builder half's state copies
    int st_grid;     // tensor-core pass: CTAs per instance of k_tc_states (0: no state in shared memory)
    int st_smem;     // and its dynamic shared bytes
    long long budget_ns;  // tensor-core kernel: time limit of each bounded wait
    double* partials;     // shift-range pass (one instance): per-shift sums here instead of the combine
    int S_full;           // and the instance's 2P + 1 shifts
    int prep_parts;  // CTAs per instance of k_prepare (weights split ~256 per CTA)
    int bop_parts;   // CTAs per instance building the tensor-core b rows
    int bop_fused;   // 1: those CTAs are part of k_prepare (every state has <= TC_BOP_FUSED_N amplitudes)
};

// Launch with programmatic stream serialization (the kernel starts with
// pdl_wait, so it observes everything its predecessor wrote).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// The kernel sequence of one cost pass on stream `st`: queue reset, prepare,
// state passes of the instances with states in HBM, term tiles, combine.
static int launch_pass(dvqls_ctx* ctx, cudaStream_t st, const Inst* dtable, const PassShape& ps,
                       const std::vector<const HostInst*>& tab, bool marks) {
    // One profiling mark per kernel, so the launch counts are exact.  The
    // prepare kernel also resets the work queue.
    if (marks) prof_begin(ctx, 0);
    k_prepare<<<dim3(ps.count, ps.prep_parts + (ps.tc && ps.bop_fused ? ps.bop_parts : 0)), NT, 0, st>>>(
        dtable, ctx->d_status, ctx->d_queue, ps.prep_parts);
    if (marks) prof_end(ctx);
    if (ps.tc && !ps.bop_fused) {
        if (marks) prof_begin(ctx, 0);
        DVQLS_CUDA_TRY(ctx, launch_pdl(k_prep_bop, dim3(ps.count, ps.bop_parts), dim3(256), 0, st, dtable));
        if (marks) prof_end(ctx);
    }
    if (ps.wht) {
        if (marks) prof_begin(ctx, 0);
        DVQLS_CUDA_TRY(ctx, launch_pdl(k_wht_classes, dim3(ps.count), dim3(WHT_CT), 0, st, dtable));
        if (marks) prof_end(ctx);
    }
    if (ps.tc && ps.st_grid > 0) {  // shifted states of the on-chip instances, packed for the term kernel
        if (marks) prof_begin(ctx, 4);
        DVQLS_CUDA_TRY(ctx, launch_pdl(k_tc_states, dim3(ps.st_grid, ps.count), dim3(256), size_t(ps.st_smem), st,
                                       dtable));
        if (marks) prof_end(ctx);
    }
    for (int oi = 0; oi < ps.count; ++oi) {
        const HostInst& h = *tab[oi];
        if (!h.hbm) continue;
        cudaStream_t keep = ctx->stream;
        ctx->stream = st;
        const int rc = ps.fp32 ? build_hbm_states<float>(ctx, dtable, oi, h.n, h.d, h.S, marks)
                               : build_hbm_states<double>(ctx, dtable, oi, h.n, h.d, h.S, marks);
        ctx->stream = keep;
        if (rc) return rc;
    }
    if (marks) prof_begin(ctx, 1);
    if (ps.wht)
        DVQLS_CUDA_TRY(ctx, launch_pdl(k_terms_wht, dim3(ps.grid), dim3(WHT_NT), ps.smem, st, dtable, ps.count,
                                       ps.total, ctx->d_queue));
    else if (ps.tc)
        DVQLS_CUDA_TRY(ctx, launch_pdl(k_terms_tc, dim3(ps.grid), dim3(TCT), ps.smem, st, dtable, ps.count, ps.total,
                                       ctx->d_queue, ctx->d_status, ps.copy_nmax, ps.split_nmax | (ps.split_nmin << 8), ps.psi_region,
                                       ps.budget_ns));
    else if (ps.fp32)
        DVQLS_CUDA_TRY(ctx, launch_pdl(k_terms_smem<float>, dim3(ps.grid), dim3(NT), ps.smem, st, dtable, ps.count,
                                       ps.total, ctx->d_queue));
    else
        DVQLS_CUDA_TRY(ctx, launch_pdl(k_terms_smem<double>, dim3(ps.grid), dim3(NT), ps.smem, st, dtable, ps.count,
                                       ps.total, ctx->d_queue));
    if (marks) prof_end(ctx);
    if (marks) prof_begin(ctx, 2);
    if (ps.partials)
        DVQLS_CUDA_TRY(ctx, launch_pdl(k_partials, dim3(1), dim3(NT), 0, st, dtable, ps.S_full, ps.partials));
    else if (ps.fp32)
        DVQLS_CUDA_TRY(ctx, launch_pdl(k_combine<float>, dim3(ps.count), dim3(NT), 0, st, dtable, ctx->d_status));
    else DVQLS_CUDA_TRY(ctx, launch_pdl(k_combine<double>, dim3(ps.count), dim3(NT), 0, st, dtable, ctx->d_status));
    if (marks) prof_end(ctx);
    DVQLS_CUDA_TRY(ctx, cudaGetLastError());
    return DVQLS_OK;
}

// Replays a captured graph of the pass when the launch (table bytes and
// shape) is the one captured last; otherwise captures it on the context's
// private capture stream first.  Profiling and callers that are capturing
// the stream themselves get direct launches.
static int run_pass(dvqls_ctx* ctx, const Inst* dtable, const PassShape& ps, const std::vector<const HostInst*>& tab,
                    const std::vector<char>& table_bytes) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;
    }
    if (ctx->profiling || cap != cudaStreamCaptureStatusNone)
        return launch_pass(ctx, ctx->stream, dtable, ps, tab, ctx->profiling);
    std::vector<char> key(table_bytes);
    const char* pk = reinterpret_cast<const char*>(&ps);
    key.insert(key.end(), pk, pk + sizeof ps);
    if (!ctx->graph || ctx->graph->key != key) {
        release_graph_cache(ctx);
        if (!ctx->cap_stream) DVQLS_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        DVQLS_CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = launch_pass(ctx, ctx->cap_stream, dtable, ps, tab, false);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, DVQLS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        }
        GraphCacheEntry* ge = new GraphCacheEntry();
        const cudaError_t ei = cudaGraphInstantiate(&ge->exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            cudaGetLastError();
            delete ge;
            return set_error(ctx, DVQLS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ei));
        }
        ge->key.swap(key);
        ctx->graph = ge;
    }
    DVQLS_CUDA_TRY(ctx, cudaGraphLaunch(ctx->graph->exec, ctx->stream));
    return DVQLS_OK;
}

int run_batch(dvqls_ctx* ctx, int count, const dvqls_instance* inst, int precision, bool want_grad,
              double* costs, double* grads, double* beta_out, double* delta_out, bool local,
              const ShiftRange* range) {
    DVQLS_NVTX(range ? "dvqls cost pass (shift range)" : local ? "dvqls local cost pass" : "dvqls cost pass");
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    if (range && (count != 1 || local || !want_grad || beta_out || delta_out || costs || grads || !range->partials))
        return set_error(ctx, DVQLS_ERR_INVALID_ARG, "a shift-range pass takes one global-cost instance");
    if (local && (beta_out || delta_out))
        return set_error(ctx, DVQLS_ERR_UNSUPPORTED, "the local cost has no beta / delta output");
    ctx->err.clear();
    if (count < 1 || !inst) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "count must be >= 1");
    if (precision != DVQLS_FP32 && precision != DVQLS_FP64 && precision != DVQLS_FP32_TC &&
        precision != DVQLS_FP32_WHT)
        return set_error(ctx, DVQLS_ERR_INVALID_ARG, "unknown precision %d", precision);
    std::vector<HostInst> hi(count);
    int nmax = 1, Pmax = 1;
    long long LLmax = 1, Nmax = 1;
    bool any_smem = false;
    for (int i = 0; i < count; ++i) {
        const dvqls_instance& q = inst[i];
        const int n = q.ansatz.n, d = q.ansatz.depth;
        if (n < 1 || n > DVQLS_MAX_QUBITS) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "instance %d: n = %d", i, n);
        if (d < 0) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "instance %d: depth < 0", i);
        if (q.ansatz.kind != DVQLS_ANSATZ_RY_CZRING)
            return set_error(ctx, DVQLS_ERR_UNSUPPORTED, "instance %d: ansatz kind %d", i, q.ansatz.kind);
        const int L = q.lcu.L;
        if (L < 1 || !q.lcu.coef || !q.lcu.xmask || !q.lcu.zmask || !q.alpha || (!q.b && !local))
            return set_error(ctx, DVQLS_ERR_INVALID_ARG, "instance %d: empty LCU or NULL input", i);
        const long long P = (long long)n * (d + 1);
        if (P > MAX_ANGLES) return set_error(ctx, DVQLS_ERR_UNSUPPORTED, "instance %d: %lld angles", i, P);
        HostInst& h = hi[i];
        h.F = local ? n + 1 : 1;
        h.n = n;
        h.d = d;
        h.L = L;
        h.P = int(P);
        h.S = want_grad ? 2 * h.P + 1 : 1;
        if (range) {
            if (range->s0 < 0 || range->s1 > h.S || range->s0 >= range->s1)
                return set_error(ctx, DVQLS_ERR_INVALID_ARG, "shift range [%d, %d) outside [0, %d)", range->s0,
                                 range->s1, h.S);
            h.S = range->s1 - range->s0;
        }
        h.T = ceil_div(L, TT);
        h.N = 1LL << n;
        h.order = i;
        h.hbm = n > DVQLS_MAX_SMEM_QUBITS;
        if (!h.hbm) {
            nmax = std::max(nmax, n);
            any_smem = true;
        }
        Pmax = std::max(Pmax, h.P);
        LLmax = std::max(LLmax, (long long)L * L);
        Nmax = std::max(Nmax, h.N);
    }
    cudaSetDevice(ctx->device);
    const bool fp32 = precision != DVQLS_FP64;
    // Walsh-Hadamard classes serve the global cost when every LCU fits one
    // 64-term tile and every state n <= 10 qubits; tensor-core tiles when
    // every LCU fits one tile (asked for directly, or as the fallback of the
    // classes); anything else runs the FP32 CUDA-core tiles.
    bool wht = precision == DVQLS_FP32_WHT;
    for (const auto& h : hi) wht = wht && h.T == 1 && h.n <= WHT_MAXN;
    bool tc = !wht && (precision == DVQLS_FP32_TC || (precision == DVQLS_FP32_WHT && !local));
    int copy_nmax = 0, split_nmax = 0;
    const bool readout = beta_out || delta_out;
    // the tensor-core kernel's shared state region: the largest on-chip state, and
    // a staged block of HBM_K amplitudes when some state lives in HBM
    bool any_hbm = false;
    for (const auto& h : hi) any_hbm = any_hbm || h.hbm;
    const int tc_nsm = std::max(any_smem ? nmax : 0, any_hbm ? HBM_KQ : 0);
    if (tc) {  // and when the kernel's shared memory fits one CTA
        int optin = 0;
        cudaFuncAttributes fa;
        DVQLS_CUDA_TRY(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
        DVQLS_CUDA_TRY(ctx, cudaFuncGetAttributes(&fa, (const void*)k_terms_tc));
        tc = tc_smem_bytes(tc_nsm, 0, 0, readout) + fa.sharedSizeBytes <= (size_t)optin;
        for (int c = TC_COPY_NMAX; tc && tc_nsm > 0 && c >= 4 && !copy_nmax; --c)
            if (tc_smem_bytes(tc_nsm, c, 0, readout) + fa.sharedSizeBytes <= (size_t)optin) copy_nmax = c;
        for (int c = std::min(TC_SPLIT_NMAX, tc_nsm); tc && c >= 4 && !split_nmax; --c)
            if (tc_smem_bytes(tc_nsm, copy_nmax, c, readout) + fa.sharedSizeBytes <= (size_t)optin) split_nmax = c;
    }
    // The tensor-core pass builds the on-chip states in a kernel of its own.
    int st_grid = 0;
    size_t st_smem = 0;
    if (tc)
        for (const auto& h : hi)
            if (!h.hbm) {
                st_grid = std::max(st_grid, tcs_jobs(h.n, h.S));
                st_smem = std::max(st_smem, tcs_smem(h.n, h.P));
            }
    if (st_grid > 0) DVQLS_CUDA_TRY(ctx, allow_dynamic_smem((const void*)k_tc_states));
    const size_t smem = wht  ? wht_smem_bytes(Pmax)
                        : tc ? tc_smem_bytes(tc_nsm, copy_nmax, split_nmax, readout)
                        : fp32 ? smem_bytes<float>(nmax, Pmax) : smem_bytes<double>(nmax, Pmax);
    const size_t r2 = fp32 ? 8 : 16;
    auto kfun = wht ? (const void*)k_terms_wht
                : tc ? (const void*)k_terms_tc
                : fp32 ? (const void*)k_terms_smem<float> : (const void*)k_terms_smem<double>;
    DVQLS_CUDA_TRY(ctx, allow_dynamic_smem(kfun));
    int bps = 0;
    DVQLS_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kfun, wht ? WHT_NT : tc ? TCT : NT, smem));
    if (tc) bps = std::min(bps, 1);  // one CTA per SM (it allocates tensor memory)
    if (bps < 1) return set_error(ctx, DVQLS_ERR_UNSUPPORTED, "term kernel does not fit (%zu B shared)", smem);
    const long long slots = (long long)ctx->num_sms * bps;

    // Amplitude split of the shared-memory instances: autotuned per problem
    // signature (first call times each candidate); states in HBM take a fixed
    // HBM_K amplitudes per item.
    std::string sig = std::to_string(precision) + (want_grad ? "g" : "c") + (beta_out ? "b" : "") +
                      (delta_out ? "d" : "") + (local ? "L" : "") +
                      (range ? "R" + std::to_string(range->s1 - range->s0) : std::string());
    for (const auto& h : hi) sig += "|" + std::to_string(h.n) + "," + std::to_string(h.d) + "," + std::to_string(h.L);
    if (ctx->fixed_layout >= 0) sig += "|F" + std::to_string(ctx->fixed_layout);  // tuned under a fixed layout
    const int cands[] = {1, 2, 4, 8};
    auto tuned = ctx->tune.find(sig);
    const bool fixed = ctx->fixed_split > 0;  // dvqls_set_tuning
    const bool tuning = any_smem && !wht && tuned == ctx->tune.end() && !fixed;
    auto ks_for = [&](const HostInst& h, int ks) {  // tensor-core items start on whole 128-amplitude stages
        if (wht) return 1;                            // a class item covers a whole state
        return h.hbm ? (int)std::max<long long>(1, h.N / HBM_K)
                     : (int)std::min<long long>(ks, std::max<long long>(1, h.N / (tc ? TCK : JC)));
    };

    // Plan the workspace (caller order; sized for the largest split tried).
    Arena ar;
    Arena pin;
    struct Off {
        size_t coef, xm, zm, alpha, b;       // staged inputs (ws) ...
        size_t pcoef, pxm, pzm, palpha, pb;  // ... and their pinned slots
        size_t ctil, w, wf, cf, bop, wht, bf, cs, bn2, Dp, Tp, Gp, dp, NsDs, cost, grad, beta, delta, states, tcst;
        size_t pcost, pgrad, pbeta, pdelta;
    };
    std::vector<Off> off(count);
    const size_t o_table = ar.reserve(sizeof(Inst) * count);
    const size_t p_table = pin.reserve(sizeof(Inst) * count);
    const int S_full = range ? 2 * hi[0].P + 1 : 0;
    const bool dev_part = range && is_device_ptr(ctx, range->partials);
    const size_t o_part = range && !dev_part ? ar.reserve(size_t(S_full) * 32) : 0;
    const size_t p_part = range && !dev_part ? pin.reserve(size_t(S_full) * 32) : 0;
    // A tuned choice: amplitude split in bits 0..7, the state layout (see the tuning loop) in bits 8..9.
    const int ks_plan_smem = fixed ? ctx->fixed_split : tuning ? 8 : (tuned != ctx->tune.end() ? (tuned->second & 255) : 1);
    int split_use = split_nmax, split_min = 4;
    // Staged inputs of all instances first, then the results, each reserved
    // in both arenas in the same order, so that the copies of a call merge
    // into one host-to-device and one device-to-host transfer.
    for (int i = 0; i < count; ++i) {
        const HostInst& h = hi[i];
        Off& o = off[i];
        const size_t L = h.L;
        o.coef = ar.reserve(L * 16);
        o.pcoef = pin.reserve(L * 16);
        o.xm = ar.reserve(L * 4);
        o.pxm = pin.reserve(L * 4);
        o.zm = ar.reserve(L * 4);
        o.pzm = pin.reserve(L * 4);
        o.alpha = ar.reserve(size_t(h.P) * 8);
        o.palpha = pin.reserve(size_t(h.P) * 8);
        o.b = local ? 0 : ar.reserve(size_t(h.N) * 16);
        o.pb = local ? 0 : pin.reserve(size_t(h.N) * 16);
    }
    for (int i = 0; i < count; ++i) {
        const HostInst& h = hi[i];
        Off& o = off[i];
        const size_t L = h.L;
        o.cost = ar.reserve(8);
        o.pcost = pin.reserve(8);
        o.grad = ar.reserve(size_t(h.P) * 8);
        o.pgrad = pin.reserve(size_t(h.P) * 8);
        o.beta = beta_out ? ar.reserve(L * L * 16) : 0;
        o.pbeta = beta_out ? pin.reserve(L * L * 16) : 0;
        o.delta = delta_out ? ar.reserve(L * 16) : 0;
        o.pdelta = delta_out ? pin.reserve(L * 16) : 0;
    }
    for (int i = 0; i < count; ++i) {
        HostInst& h = hi[i];
        const int kp = ks_for(h, ks_plan_smem);
        Off& o = off[i];
        const size_t L = h.L;
        o.ctil = ar.reserve(L * 16);
        // pair weights w_lm for the CUDA-core and Walsh-Hadamard kernels (the
        // tensor-core epilogue forms its weights from c~ alone)
        o.w = tc ? 0 : ar.reserve(L * L * 16);
        o.wf = fp32 && !tc ? ar.reserve(L * L * 16) : 0;  // float-float weights of the FP32 term kernels
        o.cf = fp32 ? ar.reserve(L * 16) : 0;
        o.bop = tc && !local ? ar.reserve(size_t(tc_bop_stages(h.N)) * TC_BOP_STAGE) : 0;
        o.wht = wht ? ar.reserve(WHT_TABLE_BYTES) : 0;
        o.bf = wht ? ar.reserve(size_t(h.N) * 8) : 0;
        o.cs = ar.reserve(size_t(3) * h.P * 16);
        o.bn2 = ar.reserve(8);
        o.Dp = ar.reserve(size_t(h.S) * h.F * h.T * h.T * kp * 16);
        o.Tp = ar.reserve(size_t(h.S) * h.T * kp * 16);
        o.Gp = beta_out ? ar.reserve(size_t(kp) * L * L * r2) : 0;
        o.dp = delta_out ? ar.reserve(size_t(kp) * L * r2) : 0;
        o.NsDs = ar.reserve(size_t(h.S) * 24);
        o.states = h.hbm ? ar.reserve(size_t(h.S) * size_t(h.N) * (r2 / 2)) : 0;  // real amplitudes
        o.tcst = tc && !h.hbm ? ar.reserve(size_t(h.S) * size_t(h.N) * 4) : 0;     // packed FP16 pairs
    }
    int rc = ensure_workspace(ctx, ar.total());
    if (!rc) rc = ensure_pinned(ctx, pin.total());
    if (rc) return rc;
    char* ws = ctx->ws;

    // Host inputs are staged through pinned memory: wait until the previous
    // call's copies out of it are done before writing it again.
    bool all_device = true;
    for (int i = 0; i < count && all_device; ++i) {
        const dvqls_instance& q = inst[i];
        all_device = is_device_ptr(ctx, q.lcu.coef) && is_device_ptr(ctx, q.lcu.xmask) &&
                     is_device_ptr(ctx, q.lcu.zmask) && is_device_ptr(ctx, q.alpha) &&
                     (local || is_device_ptr(ctx, q.b));
    }
    if (!all_device) {
        rc = pin_acquire(ctx);
        if (rc) return rc;
    }
    std::vector<long long> grad_off(count, 0);
    {
        long long g = 0;
        for (int i = 0; i < count; ++i) {
            grad_off[i] = g;
            g += hi[i].P;
        }
    }
    // Per-instance records in caller order (staging happens once here).
    struct StagingScope {
        dvqls_ctx* c;
        ~StagingScope() { end_staging(c); }
    } staging{ctx};
    begin_staging(ctx);
    std::vector<Inst> rec(count);
    const bool dev_cost = costs && is_device_ptr(ctx, costs);
    const bool dev_grad = grads && is_device_ptr(ctx, grads);
    for (int i = 0; i < count; ++i) {
        const HostInst& h = hi[i];
        const Off& o = off[i];
        const dvqls_instance& q = inst[i];
        Inst& I = rec[i];
        memset(&I, 0, sizeof I);
        I.n = h.n;
        I.d = h.d;
        I.L = h.L;
        I.P = h.P;
        I.S = h.S;
        I.T = h.T;
        I.coef = (const double2*)stage_in(ctx, q.lcu.coef, size_t(h.L) * 16, o.pcoef, o.coef);
        I.xm = (const uint32_t*)stage_in(ctx, q.lcu.xmask, size_t(h.L) * 4, o.pxm, o.xm);
        I.zm = (const uint32_t*)stage_in(ctx, q.lcu.zmask, size_t(h.L) * 4, o.pzm, o.zm);
        I.alpha = (const double*)stage_in(ctx, q.alpha, size_t(h.P) * 8, o.palpha, o.alpha);
        I.b = local ? nullptr : (const double2*)stage_in(ctx, q.b, size_t(h.N) * 16, o.pb, o.b);
        I.F = h.F;
        I.s0 = range ? range->s0 : 0;
        I.local = local ? 1 : 0;
        I.ctil = (double2*)(ws + o.ctil);
        I.w = tc ? nullptr : (double2*)(ws + o.w);
        I.wf = fp32 && !tc ? (float4*)(ws + o.wf) : nullptr;
        I.cf = fp32 ? (float4*)(ws + o.cf) : nullptr;
        I.bop = tc && !local ? (void*)(ws + o.bop) : nullptr;
        I.wht = wht ? (void*)(ws + o.wht) : nullptr;
        I.bf = wht ? (float2*)(ws + o.bf) : nullptr;
        I.cs = (double2*)(ws + o.cs);
        I.bn2 = (double*)(ws + o.bn2);
        I.Dpart = (double2*)(ws + o.Dp);
        I.Tpart = (double2*)(ws + o.Tp);
        I.Gpart = beta_out ? (void*)(ws + o.Gp) : nullptr;
        I.dpart = delta_out ? (void*)(ws + o.dp) : nullptr;
        I.NsDs = (double*)(ws + o.NsDs);
        I.states = h.hbm ? (void*)(ws + o.states) : nullptr;
        I.tcst = tc && !h.hbm ? (void*)(ws + o.tcst) : nullptr;
        // Device outputs are written in place by the combine kernel.
        I.cost = dev_cost ? costs + i : (double*)(ws + o.cost);
        I.grad = !want_grad ? nullptr : dev_grad ? grads + grad_off[i] : (double*)(ws + o.grad);
        I.beta = beta_out ? (double2*)(ws + o.beta) : nullptr;
        I.delta = delta_out ? (double2*)(ws + o.delta) : nullptr;
    }
    const Inst* dtable = (const Inst*)(ws + o_table);
    const size_t tbytes = sizeof(Inst) * count;

    rc = flush_in(ctx);
    if (rc) return rc;

    // Table for split `ks`: instances ordered longest item first (LPT),
    // item ranges assigned in that order.
    std::vector<Inst> table(count);
    std::vector<const HostInst*> tab(count);
    auto build_table = [&](int ks, PassShape& ps) {
        std::vector<int> ord(count);
        for (int i = 0; i < count; ++i) ord[i] = i;
        std::vector<int> kk(count);
        for (int i = 0; i < count; ++i) kk[i] = ks_for(hi[i], ks);
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int a, int b) { return hi[a].N / kk[a] > hi[b].N / kk[b]; });
        long long base = 0;
        for (int oi = 0; oi < count; ++oi) {
            const int i = ord[oi];
            Inst I = rec[i];
            I.ks = kk[i];
            // a Walsh-Hadamard item covers every flavour; the tensor-core tiles take
            // each pair of tiles once (T (T + 1) / 2 per shift), the CUDA-core tiles T^2
            I.items = wht ? I.S : tc ? I.S * I.F * (I.T * (I.T + 1) / 2) * I.ks : I.S * I.F * I.T * I.T * I.ks;
            I.item_base = base;
            base += I.items;
            table[oi] = I;
            tab[oi] = &hi[i];
        }
        ps.fp32 = fp32;
        ps.tc = tc;
        ps.wht = wht;
        ps.count = count;
        ps.total = base;
        ps.grid = (int)std::min<long long>(base, slots);
        ps.smem = smem;
        ps.copy_nmax = copy_nmax;
        ps.split_nmax = split_use;
        ps.split_nmin = split_min;
        ps.psi_region = tc ? (int)tc_psi_region(tc_nsm, copy_nmax, split_nmax) : 0;
        ps.st_grid = st_grid;
        ps.st_smem = (int)st_smem;
        ps.budget_ns = ctx->wait_budget_us * 1000;
        ps.partials = !range ? nullptr : dev_part ? range->partials : (double*)(ws + o_part);
        ps.S_full = S_full;
        ps.prep_parts = (int)std::min<long long>(16, std::max<long long>(1, LLmax / NT));
        ps.bop_parts = (int)std::min<long long>(64, std::max<long long>(1, tc_bop_stages(Nmax) * (TC_BOP_STAGE / 16) / 256));
        ps.bop_fused = Nmax <= TC_BOP_FUSED_N;
    };
    auto upload = [&]() -> int {
        const char* tb = reinterpret_cast<const char*>(table.data());
        if (ctx->last_table.size() == tbytes && memcmp(ctx->last_table.data(), tb, tbytes) == 0) return DVQLS_OK;
        if (all_device) {
            int r = pin_acquire(ctx);
            if (r) return r;
        }
        memcpy(ctx->pin + p_table, tb, tbytes);
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync((void*)dtable, ctx->pin + p_table, tbytes, cudaMemcpyHostToDevice,
                                            ctx->stream));
        ctx->last_table.assign(tb, tb + tbytes);
        return pin_release(ctx);
    };

    PassShape ps{};
    int ks_use = fixed ? ctx->fixed_split : tuned != ctx->tune.end() ? (tuned->second & 255) : 1;
    int lay_use = fixed ? std::max(0, ctx->fixed_layout) : tuned != ctx->tune.end() ? (tuned->second >> 8) & 3 : 0;
    if (tuning) {
        DVQLS_NVTX("dvqls autotune");
        // Time full passes per candidate -- the amplitude split, and the state layout of the
        // tensor-core builders (split hi / lo arrays or packed copies) where both fit -- and
        // keep the fastest.
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        DVQLS_CUDA_TRY(ctx, cudaEventCreate(&e0));
        DVQLS_CUDA_TRY(ctx, cudaEventCreate(&e1));
        float best = 0.f;
        // Each candidate runs TUNE_REPS passes back to back and keeps the fastest: the
        // first pass of a candidate (and of the whole call) also pays one-time costs
        // (cold caches, first launches) that a single timing would charge to it.
        constexpr int TUNE_REPS = 3;
        bool first = true;
        // layouts: 0 split arrays for 2^4 .. 2^split_nmax amplitudes, 1 only from 2^9 (small items keep
        // the packed copies, whose set-up has one barrier less), 2 packed copies only
        bool small = false;
        for (const auto& h : hi) small = small || (!h.hbm && h.n >= 4 && h.n < 9);
        for (int lay = 0; lay < (split_nmax > 0 ? 3 : 1); ++lay) {
        if (lay == 1 && ctx->fixed_layout != 1 && (!small || split_nmax < 9)) continue;
        if (ctx->fixed_layout >= 0 && lay != ctx->fixed_layout) continue;  // dvqls_set_tuning
        for (int c : cands) {
            split_use = lay == 2 ? 0 : split_nmax;
            split_min = lay == 1 ? 9 : 4;
            build_table(c, ps);
            rc = upload();
            float cbest = 0.f;
            for (int rep = 0; rep < TUNE_REPS && !rc; ++rep) {
                rc = (cudaEventRecord(e0, ctx->stream) == cudaSuccess) ? DVQLS_OK : DVQLS_ERR_CUDA;
                if (!rc) rc = launch_pass(ctx, ctx->stream, dtable, ps, tab, false);
                if (!rc) rc = (cudaEventRecord(e1, ctx->stream) == cudaSuccess) ? DVQLS_OK : DVQLS_ERR_CUDA;
                if (!rc) rc = (cudaEventSynchronize(e1) == cudaSuccess) ? DVQLS_OK : DVQLS_ERR_CUDA;
                float ms = 0.f;
                if (!rc) rc = (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) ? DVQLS_OK : DVQLS_ERR_CUDA;
                if (!rc && (rep == 0 || ms < cbest)) cbest = ms;
            }
            if (rc) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                cudaGetLastError();
                return rc == DVQLS_ERR_CUDA ? set_error(ctx, rc, "autotune pass failed") : rc;
            }
            if (first || cbest < best) {
                best = cbest;
                ks_use = c;
                lay_use = lay;
            }
            first = false;
        }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        // A pass that reported an error (a bounded wait that gave up, bad input)
        // timed nothing meaningful: report it and keep no choice.
        rc = sync_and_check(ctx);
        if (rc) return rc;
        ctx->tune[sig] = ks_use | (lay_use << 8);
    }
    split_use = lay_use == 2 ? 0 : split_nmax;
    split_min = lay_use == 1 ? 9 : 4;
    build_table(ks_use, ps);
    rc = upload();
    if (!rc && !all_device) rc = pin_release(ctx);
    if (rc) return rc;
    {
        DVQLS_NVTX("dvqls pass kernels");
        rc = run_pass(ctx, dtable, ps, tab, ctx->last_table);
    }
    if (rc) return rc;

    // Results.
    std::vector<PendingOut> pend;
    if (range && !dev_part) {
        rc = enqueue_out(ctx, range->partials, ws + o_part, size_t(S_full) * 32, p_part, pend);
        if (rc) return rc;
    }
    for (int i = 0; i < count; ++i) {
        const Off& o = off[i];
        const HostInst& h = hi[i];
        if (costs && !dev_cost) {
            rc = enqueue_out(ctx, costs + i, ws + o.cost, 8, o.pcost, pend);
            if (rc) return rc;
        }
        if (want_grad && grads && !dev_grad) {
            rc = enqueue_out(ctx, grads + grad_off[i], ws + o.grad, size_t(h.P) * 8, o.pgrad, pend);
            if (rc) return rc;
        }
        if (beta_out) {
            rc = enqueue_out(ctx, beta_out, ws + o.beta, size_t(h.L) * h.L * 16, o.pbeta, pend);
            if (rc) return rc;
        }
        if (delta_out) {
            rc = enqueue_out(ctx, delta_out, ws + o.delta, size_t(h.L) * 16, o.pdelta, pend);
            if (rc) return rc;
        }
    }
    rc = flush_out(ctx);
    if (rc) return rc;
    const bool async_ok = all_device && pend.empty() && !beta_out && !delta_out && !range;
    if (async_ok) return DVQLS_OK;
    rc = sync_and_check(ctx);
    if (rc) return rc;
    finish_out(ctx, pend);
    return DVQLS_OK;
}

// ------------------------------------------------ fidelity of a state in HBM
// F = |<xhat|psi(alpha)>|^2 / ||xhat||^2 (Sec. 3.1) for states above the
// shared-memory size: psi in FP64 by the HBM state passes (one shift), then a
// reduction whose block partials are added in a fixed order.
constexpr int FIDH_T = 256;

__global__ void __launch_bounds__(FIDH_T) k_fid_angles(const Inst* __restrict__ insts, int* status) {
    const Inst& I = insts[0];
    for (int a = threadIdx.x; a < I.P; a += FIDH_T) {
        const double al = I.alpha[a];
        if (!isfinite(al)) set_status(status, DEV_NONFINITE_INPUT);
        double sn, c;
        sincos(0.5 * al, &sn, &c);
        I.cs[a] = make_double2(c, sn);
    }
}

// Block b: sum over its share of j of conj(xhat_j) psi_j (psi real) and |xhat_j|^2.
__global__ void __launch_bounds__(FIDH_T) k_fid_partial(const Inst* __restrict__ insts, const double2* __restrict__ xh,
                                                        double* part) {
    const Inst& I = insts[0];
    const long long N = 1LL << I.n;
    const double* psi = reinterpret_cast<const double*>(I.states);
    double re = 0.0, im = 0.0, nr = 0.0;
    for (long long j = (long long)blockIdx.x * FIDH_T + threadIdx.x; j < N; j += (long long)gridDim.x * FIDH_T) {
        const double2 x = xh[j];
        const double p = psi[j];
        re += x.x * p;
        im -= x.y * p;
        nr += x.x * x.x + x.y * x.y;
    }
    __shared__ double red[3][FIDH_T / 32];
    for (int o = 16; o; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
        nr += __shfl_xor_sync(0xffffffffu, nr, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = re;
        red[1][w] = im;
        red[2][w] = nr;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int k = 0; k < FIDH_T / 32; ++k) v += red[threadIdx.x][k];
        part[3 * blockIdx.x + threadIdx.x] = v;
    }
}

__global__ void k_fid_final(const double* __restrict__ part, int nb, int* status, double* F) {
    if (threadIdx.x != 0) return;
    double re = 0.0, im = 0.0, nr = 0.0;
    for (int b = 0; b < nb; ++b) {
        re += part[3 * b];
        im += part[3 * b + 1];
        nr += part[3 * b + 2];
    }
    if (!(nr > 0.0) || !isfinite(nr)) set_status(status, DEV_BAD_NORM);
    *F = (re * re + im * im) / nr;
}

int fidelity_hbm(dvqls_ctx* ctx, int n, int d, const double* alpha, const double* xhat, double* F) {
    const int P = n * (d + 1);
    const long long N = 1LL << n;
    const int nb = (int)std::min<long long>(4LL * ctx->num_sms, (N + FIDH_T - 1) / FIDH_T);
    Arena ar, pin;
    const size_t o_t = ar.reserve(sizeof(Inst)), p_t = pin.reserve(sizeof(Inst));
    const size_t o_al = ar.reserve(size_t(P) * 8), p_al = pin.reserve(size_t(P) * 8);
    const size_t o_x = ar.reserve(size_t(N) * 16), p_x = pin.reserve(size_t(N) * 16);
    const size_t o_cs = ar.reserve(size_t(P) * 16);
    const size_t o_st = ar.reserve(size_t(N) * 8);
    const size_t o_pt = ar.reserve(size_t(nb) * 24);
    const size_t o_F = ar.reserve(8), p_F = pin.reserve(8);
    int rc = ensure_workspace(ctx, ar.total());
    if (!rc) rc = ensure_pinned(ctx, pin.total());
    if (!rc) rc = pin_acquire(ctx);
    if (rc) return rc;
    Inst I;
    memset(&I, 0, sizeof I);
    I.n = n;
    I.d = d;
    I.P = P;
    I.S = 1;
    I.alpha = (const double*)stage_in(ctx, alpha, size_t(P) * 8, p_al, o_al);
    const double2* xd = (const double2*)stage_in(ctx, xhat, size_t(N) * 16, p_x, o_x);
    I.cs = (double2*)(ctx->ws + o_cs);
    I.states = ctx->ws + o_st;
    Inst* dt = (Inst*)(ctx->ws + o_t);
    memcpy(ctx->pin + p_t, &I, sizeof I);
    DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(dt, ctx->pin + p_t, sizeof I, cudaMemcpyHostToDevice, ctx->stream));
    rc = pin_release(ctx);
    if (rc) return rc;
    k_fid_angles<<<1, FIDH_T, 0, ctx->stream>>>(dt, ctx->d_status);
    rc = build_hbm_states<double>(ctx, dt, 0, n, d, 1, false);
    if (rc) return rc;
    k_fid_partial<<<nb, FIDH_T, 0, ctx->stream>>>(dt, xd, (double*)(ctx->ws + o_pt));
    k_fid_final<<<1, 32, 0, ctx->stream>>>((const double*)(ctx->ws + o_pt), nb, ctx->d_status,
                                           (double*)(ctx->ws + o_F));
    DVQLS_CUDA_TRY(ctx, cudaGetLastError());
    std::vector<PendingOut> pend;
    rc = enqueue_out(ctx, F, ctx->ws + o_F, 8, p_F, pend);
    if (!rc) rc = sync_and_check(ctx);
    if (rc) return rc;
    return finish_out(ctx, pend);
}

}  // namespace dvqls

using namespace dvqls;

static int single(dvqls_ctx* ctx, const dvqls_ansatz* ansatz, const double* alpha, const dvqls_lcu* lcu,
                  const double* b, int precision, bool grad, double* cost, double* g, double* beta, double* delta) {
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    if (!ansatz || !lcu || !cost) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "NULL ansatz, lcu or cost");
    dvqls_instance in;
    in.ansatz = *ansatz;
    in.lcu = *lcu;
    in.alpha = alpha;
    in.b = b;
    int rc = run_batch(ctx, 1, &in, precision, grad, cost, g, beta, delta, false);
    if (rc == DVQLS_OK && is_device_ptr(ctx, cost)) rc = sync_and_check(ctx);
    return rc;
}

extern "C" int dvqls_cost(dvqls_ctx* ctx, const dvqls_ansatz* ansatz, const double* alpha, const dvqls_lcu* lcu,
                          const double* b, int precision, double* cost, double* beta, double* delta) {
    return single(ctx, ansatz, alpha, lcu, b, precision, false, cost, nullptr, beta, delta);
}

extern "C" int dvqls_cost_grad(dvqls_ctx* ctx, const dvqls_ansatz* ansatz, const double* alpha,
                               const dvqls_lcu* lcu, const double* b, int precision, double* cost, double* grad,
                               double* beta, double* delta) {
    if (ctx && !grad) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "grad is NULL");
    return single(ctx, ansatz, alpha, lcu, b, precision, true, cost, grad, beta, delta);
}

extern "C" int dvqls_cost_grad_batched(dvqls_ctx* ctx, int count, const dvqls_instance* inst, int precision,
                                       double* costs, double* grads) {
    return run_batch(ctx, count, inst, precision, true, costs, grads, nullptr, nullptr, false);
}

extern "C" int dvqls_local_cost_grad_batched(dvqls_ctx* ctx, int count, const dvqls_instance* inst, int precision,
                                             double* costs, double* grads) {
    return run_batch(ctx, count, inst, precision, grads != nullptr, costs, grads, nullptr, nullptr, true);
}

extern "C" int dvqls_local_cost_grad(dvqls_ctx* ctx, const dvqls_ansatz* ansatz, const double* alpha,
                                     const dvqls_lcu* lcu, int precision, double* cost, double* grad) {
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    if (!ansatz || !lcu || !cost) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "NULL ansatz, lcu or cost");
    dvqls_instance in;
    in.ansatz = *ansatz;
    in.lcu = *lcu;
    in.alpha = alpha;
    in.b = nullptr;
    int rc = run_batch(ctx, 1, &in, precision, grad != nullptr, cost, grad, nullptr, nullptr, true);
    if (rc == DVQLS_OK && is_device_ptr(ctx, cost)) rc = sync_and_check(ctx);
    return rc;
}

extern "C" int dvqls_cost_grad_partials(dvqls_ctx* ctx, const dvqls_ansatz* ansatz, const double* alpha,
                                        const dvqls_lcu* lcu, const double* b, int precision, int s_begin,
                                        int s_end, double* partials) {
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    if (!ansatz || !lcu || !partials) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "NULL ansatz, lcu or partials");
    dvqls_instance in;
    in.ansatz = *ansatz;
    in.lcu = *lcu;
    in.alpha = alpha;
    in.b = b;
    const ShiftRange range{s_begin, s_end, partials};
    return run_batch(ctx, 1, &in, precision, true, nullptr, nullptr, nullptr, nullptr, false, &range);
}

extern "C" int dvqls_combine_partials(dvqls_ctx* ctx, int n, int depth, const double* partials, double* cost,
                                      double* grad) {
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n < 1 || n > DVQLS_MAX_QUBITS || depth < 0 || !partials || !cost || !grad)
        return set_error(ctx, DVQLS_ERR_INVALID_ARG, "n, depth or a pointer out of range");
    const long long Pl = (long long)n * (depth + 1);
    if (Pl > MAX_ANGLES) return set_error(ctx, DVQLS_ERR_UNSUPPORTED, "%lld angles", Pl);
    const int P = int(Pl), S = 2 * P + 1;
    cudaSetDevice(ctx->device);
    Arena ar, pin;
    const size_t o_in = ar.reserve(size_t(S) * 32), p_in = pin.reserve(size_t(S) * 32);
    const size_t o_cost = ar.reserve(8), p_cost = pin.reserve(8);
    const size_t o_grad = ar.reserve(size_t(P) * 8), p_grad = pin.reserve(size_t(P) * 8);
    int rc = ensure_workspace(ctx, ar.total());
    if (!rc) rc = ensure_pinned(ctx, pin.total());
    if (!rc) rc = pin_acquire(ctx);
    if (rc) return rc;
    const double* dpart = (const double*)stage_in(ctx, partials, size_t(S) * 32, p_in, o_in);
    rc = pin_release(ctx);
    if (rc) return rc;
    const bool dcost = is_device_ptr(ctx, cost), dgrad = is_device_ptr(ctx, grad);
    double* c_out = dcost ? cost : (double*)(ctx->ws + o_cost);
    double* g_out = dgrad ? grad : (double*)(ctx->ws + o_grad);
    k_combine_partials<<<1, NT, 0, ctx->stream>>>(dpart, P, ctx->d_status, c_out, g_out);
    DVQLS_CUDA_TRY(ctx, cudaGetLastError());
    std::vector<PendingOut> pend;
    if (!dcost) rc = enqueue_out(ctx, cost, c_out, 8, p_cost, pend);
    if (!rc && !dgrad) rc = enqueue_out(ctx, grad, g_out, size_t(P) * 8, p_grad, pend);
    if (!rc) rc = sync_and_check(ctx);
    if (rc) return rc;
    return finish_out(ctx, pend);
}

// ------------------------------------------------- allocation-free variant
// dvqls_cost_grad_noalloc runs the same three kernels as dvqls_cost_grad for
// one instance, but takes its scratch (instance record, weights, per-item
// partial sums, queue counter, status word) from the file-scope device array
// below instead of a context workspace, so it needs no cudaMalloc, no pinned
// staging and no context.  Every GPU that loads the library holds the array
// until the process exits.
namespace dvqls {

constexpr size_t NOALLOC_BYTES = size_t(DVQLS_NOALLOC_SCRATCH_BYTES);
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

__global__ void k_noalloc_store(Inst I, Inst* dst) { *dst = I; }

constexpr int NOALLOC_MAX_DEVICES = 64;

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol's name is only a host-side stand-in; the address comes from
// cudaGetSymbolAddress with the device current.  It is looked up on every
// call rather than cached: a device reset by the host program gives the
// array a new address, and a cached one would then point at freed memory.
static int noalloc_scratch_address(char** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return DVQLS_ERR_CUDA;
    }
    *out = static_cast<char*>(p);
    return DVQLS_OK;
}

static bool noalloc_dev_ptr(const void* p, int dev) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

}  // namespace dvqls

extern "C" int dvqls_cost_grad_noalloc(void* stream_arg, const dvqls_ansatz* ansatz, const double* alpha,
                                       const dvqls_lcu* lcu, const double* b, int precision, double* cost,
                                       double* grad) {
    using namespace dvqls;
    cudaStream_t stream = (cudaStream_t)stream_arg;
    // An error the caller's own CUDA work left pending is not this call's to
    // clear: report it and leave it in place.
    if (cudaPeekAtLastError() != cudaSuccess) return DVQLS_ERR_CUDA;
    if (!ansatz || !lcu || !cost || !grad) return DVQLS_ERR_INVALID_ARG;
    if (precision == DVQLS_FP32_TC || precision == DVQLS_FP32_WHT) return DVQLS_ERR_UNSUPPORTED;
    if (precision != DVQLS_FP32 && precision != DVQLS_FP64) return DVQLS_ERR_INVALID_ARG;
    const int n = ansatz->n, d = ansatz->depth, L = lcu->L;
    if (n < 1 || n > DVQLS_MAX_QUBITS || d < 0 || L < 1) return DVQLS_ERR_INVALID_ARG;
    if (n > DVQLS_MAX_SMEM_QUBITS || ansatz->kind != DVQLS_ANSATZ_RY_CZRING) return DVQLS_ERR_UNSUPPORTED;
    const long long Pl = (long long)n * (d + 1);
    if (Pl > MAX_ANGLES) return DVQLS_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return DVQLS_ERR_CUDA;
    }
    const void* ptrs[] = {alpha, b, lcu->coef, lcu->xmask, lcu->zmask, cost, grad};
    for (const void* p : ptrs)
        if (!noalloc_dev_ptr(p, dev)) return DVQLS_ERR_INVALID_ARG;  // device memory only: nothing is staged

    const bool fp32 = precision == DVQLS_FP32;
    const int P = int(Pl), S = 2 * P + 1, T = ceil_div(L, TT);
    const long long N = 1LL << n;
    const size_t smem = fp32 ? smem_bytes<float>(n, P) : smem_bytes<double>(n, P);
    auto kfun = fp32 ? (const void*)k_terms_smem<float> : (const void*)k_terms_smem<double>;
    if (allow_dynamic_smem(kfun) != cudaSuccess) {
        cudaGetLastError();
        return DVQLS_ERR_CUDA;
    }
    int bps = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kfun, NT, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return DVQLS_ERR_CUDA;
    }
    if (bps < 1) return DVQLS_ERR_UNSUPPORTED;
    const long long slots = (long long)sms * bps, base_items = (long long)S * T * T;
    int ks = 1;
    while (ks < 8 && base_items * ks < 2 * slots) ks *= 2;
    ks = (int)std::min<long long>(ks, std::max<long long>(1, N / JC));

    // Scratch layout (offsets 256-byte aligned).
    Arena ar;
    const size_t o_table = ar.reserve(sizeof(Inst));
    const size_t o_words = ar.reserve(256);  // status word, queue counter
    const size_t o_ctil = ar.reserve(size_t(L) * 16);
    const size_t o_w = ar.reserve(size_t(L) * L * 16);
    const size_t o_wf = fp32 ? ar.reserve(size_t(L) * L * 16) : 0;  // float-float weights (FP32 kernel)
    const size_t o_cf = fp32 ? ar.reserve(size_t(L) * 16) : 0;
    const size_t o_cs = ar.reserve(size_t(3) * P * 16);
    const size_t o_bn2 = ar.reserve(8);
    const size_t o_Dp = ar.reserve(size_t(S) * T * T * ks * 16);
    const size_t o_Tp = ar.reserve(size_t(S) * T * ks * 16);
    const size_t o_NsDs = ar.reserve(size_t(S) * 24);
    if (ar.total() > NOALLOC_BYTES) return DVQLS_ERR_INVALID_ARG;  // beyond the fixed scratch
    char* base = nullptr;
    int rc = noalloc_scratch_address(&base);
    if (rc) return rc;

    Inst I;
    memset(&I, 0, sizeof I);
    I.n = n;
    I.d = d;
    I.L = L;
    I.P = P;
    I.S = S;
    I.T = T;
    I.ks = ks;
    I.F = 1;
    I.items = S * T * T * ks;
    I.item_base = 0;
    I.coef = (const double2*)lcu->coef;
    I.xm = lcu->xmask;
    I.zm = lcu->zmask;
    I.alpha = alpha;
    I.b = (const double2*)b;
    I.ctil = (double2*)(base + o_ctil);
    I.w = (double2*)(base + o_w);
    I.wf = fp32 ? (float4*)(base + o_wf) : nullptr;
    I.cf = fp32 ? (float4*)(base + o_cf) : nullptr;
    I.cs = (double2*)(base + o_cs);
    I.bn2 = (double*)(base + o_bn2);
    I.Dpart = (double2*)(base + o_Dp);
    I.Tpart = (double2*)(base + o_Tp);
    I.NsDs = (double*)(base + o_NsDs);
    I.cost = cost;
    I.grad = grad;
    Inst* table = (Inst*)(base + o_table);
    int* status = (int*)(base + o_words);
    unsigned long long* queue = (unsigned long long*)(base + o_words + 64);

    // The array keeps the previous call's contents: the status word and the
    // work-queue counter must start at zero; everything else is overwritten.
    if (cudaMemsetAsync(base + o_words, 0, 256, stream) != cudaSuccess) {
        cudaGetLastError();
        return DVQLS_ERR_CUDA;
    }
    k_noalloc_store<<<1, 1, 0, stream>>>(I, table);
    k_prepare<<<1, NT, 0, stream>>>(table, status, nullptr, 1);
    const long long total = I.items;
    const int grid = (int)std::min<long long>(total, slots);
    if (fp32) k_terms_smem<float><<<grid, NT, smem, stream>>>(table, 1, total, queue);
    else k_terms_smem<double><<<grid, NT, smem, stream>>>(table, 1, total, queue);
    if (fp32) k_combine<float><<<1, NT, 0, stream>>>(table, status);
    else k_combine<double><<<1, NT, 0, stream>>>(table, status);
    int st = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        return DVQLS_ERR_CUDA;
    }
    switch (st) {
        case DEV_OK: return DVQLS_OK;
        case DEV_BAD_MASK:
        case DEV_NONFINITE_INPUT:
        case DEV_BAD_NORM: return DVQLS_ERR_INVALID_ARG;
        default: return DVQLS_ERR_NUMERIC;
    }
}
