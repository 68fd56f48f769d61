// Shared-memory state vector of the Ry + CZ-ring ansatz, used by the term
// kernels, the fidelity and the optimizer.  Ansatz (Sec. 2.3 / Sec. 3, Ry + CZ
// form): Ry layer alpha[0..n), then d times { CZ ring ; Ry layer
// alpha[l*n .. l*n+n) }, with Ry(t) = [[cos t/2, -sin t/2], [sin t/2, cos t/2]]
// and the CZ ring CZ(q,q+1), q < n-1, plus CZ(n-1,0) when n >= 3.
#pragma once

#include <cuda_fp16.h>

#include <cuda_runtime.h>

namespace dvqls {

template <typename R>
struct V2;
template <>
struct V2<float> {
    using t = float2;
};
template <>
struct V2<double> {
    using t = double2;
};

template <typename R2>
__device__ __forceinline__ R2 neg2(R2 v) {
    v.x = -v.x;
    v.y = -v.y;
    return v;
}

__device__ __forceinline__ int czring_parity(int i, int n) {
    int p = __popc(i & (i >> 1) & ((1 << (n - 1)) - 1));
    if (n >= 3) p += (i >> (n - 1)) & i & 1;
    return p & 1;
}

// psi = V(alpha_s)|0> in shared memory, all threads of the CTA (blockDim.x
// of them) taking part; ends with a barrier.  cs holds (cos, sin) of the half
// angles: [0, P) at alpha, [P, 2P) at alpha + pi/2, [2P, 3P) at alpha - pi/2;
// shift s selects alpha (s = 0), alpha + pi/2 e_k (s = 2k+1) or
// alpha - pi/2 e_k (s = 2k+2).  scs receives the P (cos, sin) pairs used.
// Barrier over the threads that build a state: the whole block (bar = 0) or
// the NTH threads that share named barrier `bar`.
__device__ __forceinline__ void group_sync(int bar, int NTH) {
    if (bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(NTH) : "memory");
}

// Builds shifted state s with threads t = 0 .. NTH-1 of a group.
template <typename R>
__device__ void build_state_group(typename V2<R>::t* psi, typename V2<R>::t* scs, int n, int d, int P,
                                  const double2* cs, int s, int t, int NTH, int bar) {
    using R2 = typename V2<R>::t;
    const int N = 1 << n;
    int k = -1, which = 0;
    if (s > 0) {
        k = (s - 1) >> 1;
        which = ((s - 1) & 1) ? 2 : 1;
    }
    for (int a = t; a < P; a += NTH) {
        const double2 v = cs[(a == k ? which : 0) * P + a];
        R2 r;
        r.x = (R)v.x;
        r.y = (R)v.y;
        scs[a] = r;
    }
    group_sync(bar, NTH);
    for (int i = t; i < N; i += NTH) {  // initial Ry layer on |0>: a product state
        R v = (R)1;
        for (int q = 0; q < n; ++q) v *= ((i >> q) & 1) ? scs[q].y : scs[q].x;
        R2 r;
        r.x = v;
        r.y = (R)0;
        psi[i] = r;
    }
    group_sync(bar, NTH);
    // Layers: the CZ ring (diagonal) is applied while loading the first pass;
    // the Ry rotations of qubits q and q+1 are fused into one pass over groups
    // of four amplitudes (bits q, q+1 = 00, 01, 10, 11), so a layer takes
    // ceil(n/2) passes and barriers.
    for (int layer = 1; layer <= d; ++layer) {
        for (int q = 0; q < n; q += 2) {
            const R c0 = scs[layer * n + q].x, s0 = scs[layer * n + q].y;
            if (q + 1 < n) {
                const R c1 = scs[layer * n + q + 1].x, s1 = scs[layer * n + q + 1].y;
                for (int p = t; p < N / 4; p += NTH) {
                    const int i00 = ((p >> q) << (q + 2)) | (p & ((1 << q) - 1));
                    const int i01 = i00 | (1 << q), i10 = i00 | (2 << q), i11 = i00 | (3 << q);
                    R2 a = psi[i00], b = psi[i01], c = psi[i10], e = psi[i11];
                    if (q == 0) {
                        if (czring_parity(i00, n)) a = neg2(a);
                        if (czring_parity(i01, n)) b = neg2(b);
                        if (czring_parity(i10, n)) c = neg2(c);
                        if (czring_parity(i11, n)) e = neg2(e);
                    }
                    R2 a1, b1, c1r, e1;  // Ry on qubit q: pairs (a, b) and (c, e)
                    a1.x = c0 * a.x - s0 * b.x;
                    a1.y = c0 * a.y - s0 * b.y;
                    b1.x = s0 * a.x + c0 * b.x;
                    b1.y = s0 * a.y + c0 * b.y;
                    c1r.x = c0 * c.x - s0 * e.x;
                    c1r.y = c0 * c.y - s0 * e.y;
                    e1.x = s0 * c.x + c0 * e.x;
                    e1.y = s0 * c.y + c0 * e.y;
                    R2 u;  // Ry on qubit q+1: pairs (a1, c1r) and (b1, e1)
                    u.x = c1 * a1.x - s1 * c1r.x;
                    u.y = c1 * a1.y - s1 * c1r.y;
                    psi[i00] = u;
                    u.x = s1 * a1.x + c1 * c1r.x;
                    u.y = s1 * a1.y + c1 * c1r.y;
                    psi[i10] = u;
                    u.x = c1 * b1.x - s1 * e1.x;
                    u.y = c1 * b1.y - s1 * e1.y;
                    psi[i01] = u;
                    u.x = s1 * b1.x + c1 * e1.x;
                    u.y = s1 * b1.y + c1 * e1.y;
                    psi[i11] = u;
                }
            } else {
                for (int p = t; p < N / 2; p += NTH) {
                    const int i0 = ((p >> q) << (q + 1)) | (p & ((1 << q) - 1)), i1 = i0 | (1 << q);
                    R2 a = psi[i0], b = psi[i1];
                    if (q == 0) {
                        if (czring_parity(i0, n)) a = neg2(a);
                        if (czring_parity(i1, n)) b = neg2(b);
                    }
                    R2 u, v;
                    u.x = c0 * a.x - s0 * b.x;
                    u.y = c0 * a.y - s0 * b.y;
                    v.x = s0 * a.x + c0 * b.x;
                    v.y = s0 * a.y + c0 * b.y;
                    psi[i0] = u;
                    psi[i1] = v;
                }
            }
            group_sync(bar, NTH);
        }
    }
}

// The same state with real amplitudes (every gate of the ansatz is real),
// multiplied by `scale`, in precision R: psi[0 .. 2^n), scs[0 .. P) as
// (cos, sin).
template <typename R>
__device__ inline void build_state_real(R* psi, typename V2<R>::t* scs, int n, int d, int P, const double2* cs, int s,
                                        int t, int NTH, int bar, R scale) {
    using R2 = typename V2<R>::t;
    const int N = 1 << n;
    int k = -1, which = 0;
    if (s > 0) {
        k = (s - 1) >> 1;
        which = ((s - 1) & 1) ? 2 : 1;
    }
    for (int a = t; a < P; a += NTH) {
        const double2 v = cs[(a == k ? which : 0) * P + a];
        R2 r;
        r.x = (R)v.x;
        r.y = (R)v.y;
        scs[a] = r;
    }
    group_sync(bar, NTH);
    for (int i = t; i < N; i += NTH) {  // initial Ry layer on |0>: a product state
        R v = scale;
        for (int q = 0; q < n; ++q) v *= ((i >> q) & 1) ? scs[q].y : scs[q].x;
        psi[i] = v;
    }
    group_sync(bar, NTH);
    for (int layer = 1; layer <= d; ++layer) {
        for (int q = 0; q < n; q += 2) {
            const R c0 = scs[layer * n + q].x, s0 = scs[layer * n + q].y;
            if (q + 1 < n) {
                const R c1 = scs[layer * n + q + 1].x, s1 = scs[layer * n + q + 1].y;
                for (int p = t; p < N / 4; p += NTH) {
                    const int i00 = ((p >> q) << (q + 2)) | (p & ((1 << q) - 1));
                    const int i01 = i00 | (1 << q), i10 = i00 | (2 << q), i11 = i00 | (3 << q);
                    R a = psi[i00], b = psi[i01], c = psi[i10], e = psi[i11];
                    if (q == 0) {  // the CZ ring, applied while loading the layer's first pass
                        if (czring_parity(i00, n)) a = -a;
                        if (czring_parity(i01, n)) b = -b;
                        if (czring_parity(i10, n)) c = -c;
                        if (czring_parity(i11, n)) e = -e;
                    }
                    const R a1 = c0 * a - s0 * b, b1 = s0 * a + c0 * b;  // Ry on qubit q
                    const R c2 = c0 * c - s0 * e, e1 = s0 * c + c0 * e;
                    psi[i00] = c1 * a1 - s1 * c2;  // Ry on qubit q + 1
                    psi[i10] = s1 * a1 + c1 * c2;
                    psi[i01] = c1 * b1 - s1 * e1;
                    psi[i11] = s1 * b1 + c1 * e1;
                }
            } else {
                for (int p = t; p < N / 2; p += NTH) {
                    const int i0 = ((p >> q) << (q + 1)) | (p & ((1 << q) - 1)), i1 = i0 | (1 << q);
                    R a = psi[i0], b = psi[i1];
                    if (q == 0) {
                        if (czring_parity(i0, n)) a = -a;
                        if (czring_parity(i1, n)) b = -b;
                    }
                    psi[i0] = c0 * a - s0 * b;
                    psi[i1] = s0 * a + c0 * b;
                }
            }
            group_sync(bar, NTH);
        }
    }
}

// ---- Register-resident real state build for a group of 256 threads.
//
// The group holds 2^n = 256 A amplitudes with A per thread.  Mapping M1:
// i = (r << 8) | (warp << 5) | lane (qubits 0-4 on lanes, 5-7 on warps, 8+ on
// registers); mapping M2: i = (r << 8) | (lane << 3) | warp (qubits 3-7 on
// lanes, 0-2 on warps).  A qubit on a lane bit rotates with one shuffle, on a
// register bit in place; the warp-bit qubits of a layer are reached by one
// transpose through shared memory (padded by one word per 32, conflict-free),
// alternating M1 and M2 from layer to layer.  Ry gates of a layer commute, so
// the layer splits across the transpose; the CZ ring is a sign per amplitude.

// The tensor-core operand pair of x: hi = RN_fp16(x) in the low half-word and
// RN_fp16(2 (x - hi)) -- the low part, doubled -- in the high one (x - hi is
// exact in FP32).  x ~ hi + (high half) / 2.
__device__ __forceinline__ uint32_t split_h2l(float x) {
    const __half h = __float2half_rn(x);
    const __half l = __float2half_rn(2.f * (x - __half2float(h)));
    return (uint32_t)__half_as_ushort(h) | ((uint32_t)__half_as_ushort(l) << 16);
}

__device__ __forceinline__ int st_index(int M, int r, int w, int lane) {
    return M == 0 ? (r << 8) | (w << 5) | lane : (r << 8) | (lane << 3) | w;
}
__device__ __forceinline__ int st_pad(int i) { return i + (i >> 5); }

// Ry(theta) on a register bit in scaled form.  With c = cos(theta/2) and
// s = sin(theta/2), Ry = c [[1, -t], [t, 1]] (t = s/c) when |c| >= |s|, else
// s [[u, -1], [1, u]] (u = c/s): the bracketed matrix takes one FMA per
// amplitude (two per pair instead of four), and the factor (c or s) is
// applied once for all the rotations of a pass.  |t|, |u| <= 1 keeps every
// step as well conditioned as the plain rotation.
struct RyScaled {
    float r, fac;
    int sform;
};
__device__ __forceinline__ RyScaled ry_scaled(float c, float s) {
    RyScaled q;
    if (fabsf(c) >= fabsf(s)) {
        q.r = s / c;
        q.fac = c;
        q.sform = 0;
    } else {
        q.r = c / s;
        q.fac = s;
        q.sform = 1;
    }
    return q;
}
// The bracketed matrix on register bit kb (a compile-time constant in the
// unrolled callers) of the A amplitudes v.
template <int A>
__device__ __forceinline__ void ry_regs_scaled(float (&v)[A], int kb, float r, int sform) {
    if (sform) {
#pragma unroll
        for (int i = 0; i < A; ++i)
            if (!((i >> kb) & 1)) {
                const float a0 = v[i], a1 = v[i | (1 << kb)];
                v[i] = fmaf(r, a0, -a1);
                v[i | (1 << kb)] = fmaf(r, a1, a0);
            }
    } else {
#pragma unroll
        for (int i = 0; i < A; ++i)
            if (!((i >> kb) & 1)) {
                const float a0 = v[i], a1 = v[i | (1 << kb)];
                v[i] = fmaf(-r, a1, a0);
                v[i | (1 << kb)] = fmaf(r, a0, a1);
            }
    }
}

// Ry(theta) on the qubit of lane bit b: v' = c v -+ s v_partner.
__device__ __forceinline__ float ry_lane(float v, int lane, int b, float c, float s) {
    const float p = __shfl_xor_sync(0xffffffffu, v, 1 << b);
    return fmaf(c, v, ((lane >> b) & 1) ? s * p : -s * p);
}

// Final store of an amplitude: packed FP16 (hi, 2 lo) (PACK) or FP32.
template <bool PACK>
__device__ __forceinline__ void st_out(void* psi, int i, float v) {
    if (PACK) reinterpret_cast<uint32_t*>(psi)[i] = split_h2l(v);
    else reinterpret_cast<float*>(psi)[i] = v;
}

template <int A, int LOGA, bool PACK>
__device__ void state_regs_multiwarp(void* psi, float* scr0, float* scr1, const float2* scs, int n, int d, int t,
                                     int bar, float scale) {
    const int lane = t & 31, w = t >> 5;
    float v[A];
#pragma unroll
    for (int r = 0; r < A; ++r) {  // initial Ry layer on |0>: a product state
        const int i = st_index(0, r, w, lane);
        float x = scale;
        for (int q = 0; q < n; ++q) x *= ((i >> q) & 1) ? scs[q].y : scs[q].x;
        v[r] = x;
    }
    int M = 0, k = 0;
    for (int layer = 1; layer <= d; ++layer) {
        const float2* ang = scs + layer * n;
#pragma unroll
        for (int r = 0; r < A; ++r)
            if (czring_parity(st_index(M, r, w, lane), n)) v[r] = -v[r];
        const int qlane = M == 0 ? 0 : 3;  // qubit of lane bit 0
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            const float c = ang[qlane + b].x, sn = ang[qlane + b].y;
#pragma unroll
            for (int r = 0; r < A; ++r) v[r] = ry_lane(v[r], lane, b, c, sn);
        }
#pragma unroll
        for (int kb = 0; kb < LOGA; ++kb) {  // register-bit qubits 8 + kb
            const float c = ang[8 + kb].x, sn = ang[8 + kb].y;
#pragma unroll
            for (int r = 0; r < A; ++r)
                if (!((r >> kb) & 1)) {
                    const float a0 = v[r], a1 = v[r | (1 << kb)];
                    v[r] = c * a0 - sn * a1;
                    v[r | (1 << kb)] = sn * a0 + c * a1;
                }
        }
        // transpose to the other mapping through scratch buffer k
        float* scr = k ? scr1 : scr0;
#pragma unroll
        for (int r = 0; r < A; ++r) scr[st_pad(st_index(M, r, w, lane))] = v[r];
        group_sync(bar, 256);
        M ^= 1;
        k ^= 1;
#pragma unroll
        for (int r = 0; r < A; ++r) v[r] = scr[st_pad(st_index(M, r, w, lane))];
        // the qubits that were on warp bits are now on lanes: M1 lanes 0-2 = qubits 0-2,
        // M2 lanes 2-4 = qubits 5-7
        const int b0 = M == 0 ? 0 : 2, q0 = M == 0 ? 0 : 5;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float c = ang[q0 + j].x, sn = ang[q0 + j].y;
#pragma unroll
            for (int r = 0; r < A; ++r) v[r] = ry_lane(v[r], lane, b0 + j, c, sn);
        }
    }
#pragma unroll
    for (int r = 0; r < A; ++r) st_out<PACK>(psi, st_index(M, r, w, lane), v[r]);
    group_sync(bar, 256);
}

// n <= 10: one warp holds the whole state (i = (r << 5) | lane; for n < 5 lane
// i is lane mod 2^n), no barrier inside.  The initial Ry layer on |0> is a
// product state: a lane factor (qubits on lane bits) times register factors
// built by doubling (qubits on register bits).  The CZ-ring signs depend only
// on the amplitude index, so they are one bit mask per lane for every layer.
template <int A, int LOGA, bool PACK>
__device__ void state_regs_warp(void* psi, const float2* scs, int n, int d, int lane, float scale) {
    const int N = 1 << n, lmask = N < 32 ? N - 1 : 31, nl = n < 5 ? n : 5, li = lane & lmask;
    float v[A];
    {
        float f = scale;  // qubits 0 .. nl - 1 on the lane bits
        for (int q = 0; q < nl; ++q) f *= ((li >> q) & 1) ? scs[q].y : scs[q].x;
        v[0] = f;
#pragma unroll
        for (int kb = 0; kb < LOGA; ++kb) {  // qubit 5 + kb on register bit kb
            const float c = scs[5 + kb].x, sn = scs[5 + kb].y;
#pragma unroll
            for (int r = 0; r < (1 << kb); ++r) {
                v[r + (1 << kb)] = v[r] * sn;
                v[r] *= c;
            }
        }
    }
    uint32_t czm = 0u;  // bit r: the CZ ring flips the sign of amplitude (r << 5) | lane
#pragma unroll
    for (int r = 0; r < A; ++r) czm |= uint32_t(czring_parity((r << 5) | li, n)) << r;
    for (int layer = 1; layer <= d; ++layer) {
        const float2* ang = scs + layer * n;
#pragma unroll
        for (int r = 0; r < A; ++r)
            v[r] = __uint_as_float(__float_as_uint(v[r]) ^ (((czm >> r) & 1u) << 31));
        for (int b = 0; b < nl; ++b) {
            const float c = ang[b].x, sb = ((lane >> b) & 1) ? ang[b].y : -ang[b].y;
#pragma unroll
            for (int r = 0; r < A; ++r) v[r] = fmaf(c, v[r], sb * __shfl_xor_sync(0xffffffffu, v[r], 1 << b));
        }
#pragma unroll
        for (int kb = 0; kb < LOGA; ++kb) {  // register-bit qubits 5 + kb
            const float c = ang[5 + kb].x, sn = ang[5 + kb].y;
#pragma unroll
            for (int r = 0; r < A; ++r)
                if (!((r >> kb) & 1)) {
                    const float a0 = v[r], a1 = v[r | (1 << kb)];
                    v[r] = c * a0 - sn * a1;
                    v[r | (1 << kb)] = sn * a0 + c * a1;
                }
        }
    }
    if (lane < N || N >= 32) {
#pragma unroll
        for (int r = 0; r < A; ++r) st_out<PACK>(psi, (r << 5) | lane, v[r]);
    }
}

// The real state of shift s, times `scale`, for a group of 256 threads (ids t,
// named barrier `bar`) into psi[0 .. 2^n), as packed FP16 (hi, 2 lo) pairs
// (split_h2l; PACK) or as FP32; n <= 12.  scratch: 2 x (2^n + 2^n / 32) floats
// of shared memory that nothing else uses meanwhile.
template <bool PACK>
__device__ inline void build_state_regs(void* psi, float* scratch, float2* scs, int n, int d, int P,
                                        const double2* cs, int s, int t, int bar, float scale) {
    int k = -1, which = 0;
    if (s > 0) {
        k = (s - 1) >> 1;
        which = ((s - 1) & 1) ? 2 : 1;
    }
    for (int a = t; a < P; a += 256) {
        const double2 v = cs[(a == k ? which : 0) * P + a];
        scs[a] = make_float2((float)v.x, (float)v.y);
    }
    group_sync(bar, 256);
    const int N = 1 << n;
    float* scr1 = scratch + N + N / 32;
    switch (n) {
        case 9: state_regs_multiwarp<2, 1, PACK>(psi, scratch, scr1, scs, n, d, t, bar, scale); return;
        case 10: state_regs_multiwarp<4, 2, PACK>(psi, scratch, scr1, scs, n, d, t, bar, scale); return;
        case 11: state_regs_multiwarp<8, 3, PACK>(psi, scratch, scr1, scs, n, d, t, bar, scale); return;
        case 12: {  // 16 amplitudes per thread would crowd the registers: gate passes in shared memory
            float* f = reinterpret_cast<float*>(psi);
            build_state_real<float>(f, scs, n, d, P, cs, s, t, 256, bar, scale);  // ends with a barrier
            if (PACK) {
                for (int i = t; i < N; i += 256) st_out<true>(psi, i, f[i]);  // in place, one word each
                group_sync(bar, 256);
            }
            return;
        }
        default: break;
    }
    if ((t >> 5) == 0) {
        const int lane = t & 31;
        switch (n) {
            case 6: state_regs_warp<2, 1, PACK>(psi, scs, n, d, lane, scale); break;
            case 7: state_regs_warp<4, 2, PACK>(psi, scs, n, d, lane, scale); break;
            case 8: state_regs_warp<8, 3, PACK>(psi, scs, n, d, lane, scale); break;
            default: state_regs_warp<1, 0, PACK>(psi, scs, n, d, lane, scale); break;  // n <= 5
        }
    }
    group_sync(bar, 256);
}

template <typename R>
__device__ void build_state(typename V2<R>::t* psi, typename V2<R>::t* scs, int n, int d, int P,
                            const double2* cs, int s) {
    build_state_group<R>(psi, scs, n, d, P, cs, s, threadIdx.x, blockDim.x, 0);
}

}  // namespace dvqls
