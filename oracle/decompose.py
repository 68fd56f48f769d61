"""FWHT-based Pauli decomposition with tau pruning: the plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
library.

What it follows (D-VQLS, Sec. 2.2):
  - Eq. 5: c_l = Tr(sigma_l^dag A) / N with Tr(sigma_l^dag sigma_l') = N delta.
  - The FWHT-based decomposition (Georges et al., cited in Sec. 2.2) in
    O(N^2 log N): group the entries of A by the X-mask x = row XOR column, take
    the Walsh-Hadamard transform of each diagonal d_x(i) = A[i XOR x, i], then
    apply the phase (-i)^popc(x&z) and the 1/N scale.
  - Absolute-magnitude pruning, one scan (Sec. 2.2 after Eq. 5; Algorithm 1,
    Step 2): keep |c_l| > tau.  Sec. 2.5.1 normalises the largest coefficient
    to one, so the threshold is applied relative to max |c|.
  - The exact top-L Frobenius error quoted in Sec. 1 and Sec. 3.2, by
    Parseval: ||A - A_L||_F^2 = N * sum_discarded |c|^2.

Conventions: qubit k is bit k of the basis index; sigma(x,z) = i^popc(x&z) X^x
Z^z, so sigma|i> = i^popc(x&z) (-1)^popc(z&i) |i XOR x>.  Selection order:
key |c|^2 = re*re + im*im (two products, one sum; no fused multiply-add)
descending, ties by the packed index (x << n) | z ascending.  The threshold is
thr = (tau*tau) * max_key and a coefficient passes when key > thr.
"""
import numpy as np


def popcount(a):
    """Bit count of each element of a non-negative integer array (<= 40 bits)."""
    a = np.asarray(a, dtype=np.int64)
    out = np.zeros(a.shape, dtype=np.int64)
    for k in range(40):
        out += (a >> k) & 1
    return out


def xmask_diagonals(A):
    """X-masks present in A and their diagonals d_x(i) = A[i XOR x, i].

    Returns (masks uint32 ascending, d float64 [len(masks), N])."""
    A = np.asarray(A, dtype=np.float64)
    N = A.shape[0]
    i = np.arange(N)
    masks, rows = [], []
    for x in range(N):
        dx = A[i ^ x, i]
        if np.any(dx != 0.0):
            masks.append(x)
            rows.append(dx.copy())
    if not masks:
        return np.zeros(0, np.uint32), np.zeros((0, N))
    return np.array(masks, dtype=np.uint32), np.stack(rows)


def banded_xmask_diagonals(n, offsets, band_values):
    """Same as xmask_diagonals for a banded matrix given by its diagonals.

    band_values[k][r] = A[r, r + offsets[k]] (entries outside the matrix are
    ignored).  Used where the dense matrix would not fit (n = 20)."""
    N = 1 << n
    rows, cols, vals = [], [], []
    for off, v in zip(offsets, band_values):
        r = np.arange(N)
        c = r + int(off)
        ok = (c >= 0) & (c < N)
        v = np.asarray(v, dtype=np.float64)
        ok &= v != 0.0
        rows.append(r[ok])
        cols.append(c[ok])
        vals.append(v[ok])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    x = r ^ c
    masks = np.unique(x).astype(np.uint32)
    d = np.zeros((masks.size, N))
    d[np.searchsorted(masks, x), c] = v  # d_x(i) = A[i ^ x, i]: column i = c
    return masks, d


def fwht_rows(d):
    """Walsh-Hadamard transform W(z) = sum_i (-1)^popc(z&i) d(i) of each row.

    Radix-2 order: stride h = 1, 2, 4, ..., N/2; at each stride the pair
    (u, v) = (d[j], d[j+h]) becomes (u + v, u - v)."""
    W = np.array(d, dtype=np.float64, copy=True)
    M, N = W.shape
    h = 1
    while h < N:
        V = W.reshape(M, N // (2 * h), 2, h)
        u = V[:, :, 0, :].copy()
        v = V[:, :, 1, :].copy()
        V[:, :, 0, :] = u + v
        V[:, :, 1, :] = u - v
        W = V.reshape(M, N)
        h *= 2
    return W


def pauli_coefficients(masks, d, n):
    """All coefficients c(x, z) for the given X-masks (Eq. 5 via the FWHT).

    Returns complex128 [len(masks), N]: c(x,z) = (-i)^popc(x&z) W_x(z) / N."""
    N = 1 << n
    W = fwht_rows(d) / float(N)
    z = np.arange(N)
    coef = np.zeros(W.shape, dtype=np.complex128)
    for r, x in enumerate(masks):
        k = popcount(int(x) & z) % 4
        re = np.where(k == 0, W[r], np.where(k == 2, -W[r], 0.0))
        im = np.where(k == 1, -W[r], np.where(k == 3, W[r], 0.0))
        coef[r] = re + 1j * im
    return coef


def select_terms(coef, masks, n, tau, L_max):
    """tau filter and top-L selection (Algorithm 1, Step 2).

    Returns dict with keys coef (complex128 [L]), x, z (uint32 [L]),
    L_out, L_pre (nonzero count) and L_post (count passing the filter)."""
    N = 1 << n
    re = coef.real.ravel()
    im = coef.imag.ravel()
    key = re * re + im * im
    xs = np.repeat(np.asarray(masks, dtype=np.int64), N)
    zs = np.tile(np.arange(N, dtype=np.int64), len(masks))
    packed = (xs << n) | zs
    smax = key.max() if key.size else 0.0
    thr = (tau * tau) * smax if tau > 0 else 0.0
    L_pre = int(np.count_nonzero(key > 0.0))
    keep = np.nonzero(key > thr)[0]
    L_post = int(keep.size)
    order = keep[np.lexsort((packed[keep], -key[keep]))]
    take = order[: L_max] if L_max > 0 else order
    return {
        "coef": coef.ravel()[take].copy(),
        "x": xs[take].astype(np.uint32),
        "z": zs[take].astype(np.uint32),
        "L_out": int(take.size),
        "L_pre": L_pre,
        "L_post": L_post,
    }


def decompose(A, tau=0.0, L_max=0):
    """Dense A (N x N, N = 2^n, real) -> selected LCU (see select_terms)."""
    A = np.asarray(A, dtype=np.float64)
    n = int(round(np.log2(A.shape[0])))
    masks, d = xmask_diagonals(A)
    coef = pauli_coefficients(masks, d, n)
    out = select_terms(coef, masks, n, tau, L_max)
    out["all_coef"] = coef
    out["masks"] = masks
    return out


def decompose_banded(n, offsets, band_values, tau=0.0, L_max=0):
    masks, d = banded_xmask_diagonals(n, offsets, band_values)
    coef = pauli_coefficients(masks, d, n)
    out = select_terms(coef, masks, n, tau, L_max)
    out["all_coef"] = coef
    out["masks"] = masks
    return out


def frobenius_error(all_coef, kept_coef):
    """Relative Frobenius error of the pruned matrix, by Parseval:
    eps_F = sqrt(sum_discarded |c|^2 / sum_all |c|^2)."""
    tot = float(np.sum(np.abs(all_coef) ** 2))
    kept = float(np.sum(np.abs(kept_coef) ** 2))
    return np.sqrt(max(tot - kept, 0.0) / tot)


def circuits_per_iteration(n, L):
    """Hadamard-test circuits per iteration of the local cost: (n+1) L^2
    overlaps, real and imaginary circuits each (Sec. 2.2 after Eq. 4)."""
    return 2 * (n + 1) * L * L
