// Shared-memory state vector of the Ry + CZ-ring ansatz, used by the term
// kernels, the fidelity and the optimizer.  Ansatz (Sec. 2.3 / Sec. 3, Ry + CZ
// form): Ry layer alpha[0..n), then d times { CZ ring ; Ry layer
// alpha[l*n .. l*n+n) }, with Ry(t) = [[cos t/2, -sin t/2], [sin t/2, cos t/2]]
// and the CZ ring CZ(q,q+1), q < n-1, plus CZ(n-1,0) when n >= 3.
#pragma once

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
template <typename R>
__device__ void build_state(typename V2<R>::t* psi, typename V2<R>::t* scs, int n, int d, int P,
                            const double2* cs, int s) {
    using R2 = typename V2<R>::t;
    const int N = 1 << n, t = threadIdx.x, NTH = blockDim.x;
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
    __syncthreads();
    for (int i = t; i < N; i += NTH) {  // initial Ry layer on |0>: a product state
        R v = (R)1;
        for (int q = 0; q < n; ++q) v *= ((i >> q) & 1) ? scs[q].y : scs[q].x;
        R2 r;
        r.x = v;
        r.y = (R)0;
        psi[i] = r;
    }
    __syncthreads();
    for (int layer = 1; layer <= d; ++layer) {
        for (int q = 0; q < n; ++q) {
            const R c = scs[layer * n + q].x, sn = scs[layer * n + q].y;
            for (int p = t; p < N / 2; p += NTH) {
                const int i0 = ((p >> q) << (q + 1)) | (p & ((1 << q) - 1)), i1 = i0 | (1 << q);
                R2 a = psi[i0], b = psi[i1];
                if (q == 0) {  // the CZ ring (diagonal) precedes the layer's rotations
                    if (czring_parity(i0, n)) a = neg2(a);
                    if (czring_parity(i1, n)) b = neg2(b);
                }
                R2 u, v;
                u.x = c * a.x - sn * b.x;
                u.y = c * a.y - sn * b.y;
                v.x = sn * a.x + c * b.x;
                v.y = sn * a.y + c * b.y;
                psi[i0] = u;
                psi[i1] = v;
            }
            __syncthreads();
        }
    }
}

}  // namespace dvqls
