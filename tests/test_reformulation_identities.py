"""The identities the fast kernels rest on, checked in plain numpy on small
random cases (CPU): the Walsh-Hadamard form of the real Gram terms (global
cost, and the local cost's X_j flavours), the index algebra of the
four-copy and the split state layouts of the tensor-core tiles, and the
rotation form, CZ-ring sign and transpose layouts of the HBM state passes."""
import numpy as np
import pytest


def popc(a):
    return bin(int(a)).count("1")


def phi(psi, x, z):
    """X^x Z^z psi as a real vector: phi[j] = (-1)^popc(z & (j ^ x)) psi[j ^ x]."""
    N = psi.size
    j = np.arange(N)
    src = j ^ x
    sign = np.array([1.0 - 2.0 * (popc(z & s) & 1) for s in src])
    return sign * psi[src]


def wht(v):
    """Unnormalised Walsh-Hadamard transform: W(z) = sum_i (-1)^popc(z & i) v[i]."""
    N = v.size
    i = np.arange(N)
    return np.array([np.sum(v * (1.0 - 2.0 * (np.vectorize(popc)(z & i) & 1))) for z in range(N)])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gram_terms_by_walsh_hadamard_classes(seed):
    rng = np.random.default_rng(seed)
    n = 5
    N = 1 << n
    psi = rng.normal(size=N)
    masks = rng.integers(0, N, size=(6, 2))
    for xl, zl in masks:
        for xm, zm in masks:
            g = np.dot(phi(psi, xl, zl), phi(psi, xm, zm))
            x = xl ^ xm
            W = wht(psi * psi[np.arange(N) ^ x])
            assert abs(g - (1 - 2 * (popc(zl & x) & 1)) * W[zl ^ zm]) < 1e-12
            for j in range(n):  # local-cost flavour: X_j between the terms
                gj = np.dot(phi(psi, xl, zl), phi(psi, xm, zm)[np.arange(N) ^ (1 << j)])
                X = x ^ (1 << j)
                WX = wht(psi * psi[np.arange(N) ^ X])
                assert abs(gj - (1 - 2 * (popc(zl & X) & 1)) * WX[zl ^ zm]) < 1e-12
                # the sign of flavour j is the class sign flipped by bit j of z_l
                assert (popc(zl & X) & 1) == ((popc(zl & x) & 1) ^ ((zl >> j) & 1))


def test_delta_by_walsh_hadamard_of_term_classes():
    rng = np.random.default_rng(5)
    n, N = 4, 16
    psi = rng.normal(size=N)
    b = rng.normal(size=N) + 1j * rng.normal(size=N)
    for x, z in rng.integers(0, N, size=(8, 2)):
        d = np.vdot(b, phi(psi, x, z))  # sum_j conj(b_j) phi_l[j]
        h = np.conj(b[np.arange(N) ^ x]) * psi
        assert abs(d - (wht(h.real) + 1j * wht(h.imag))[z]) < 1e-12


def test_four_copy_layout_index_algebra():
    """Term value i of a 16-block: psi[rb | (i ^ xlo)] = copy_t[rb + 4 (c ^ xc) + r] with
    i = 4c + r, t = xlo & 3, xc = xlo >> 2 and copy_t[k] = psi[k ^ t]."""
    N = 256
    psi = np.arange(N) * 1.0 + 0.5
    copies = [psi[np.arange(N) ^ t] for t in range(4)]
    for xl in range(N):
        xlo = xl & 15
        for rb in range(0, N, 16):
            for i in range(16):
                c, r = i >> 2, i & 3
                assert psi[rb | (i ^ xlo)] == copies[xlo & 3][rb + 4 * (c ^ (xlo >> 2)) + r]


def prmt(a, b, sel):
    """Byte permute of the eight bytes of (a, b): byte i of the result is
    byte (nibble i of sel) & 7 of b:a."""
    src = [(a >> (8 * k)) & 0xFF for k in range(4)] + [(b >> (8 * k)) & 0xFF for k in range(4)]
    return sum(src[(sel >> (4 * i)) & 7] << (8 * i) for i in range(4))


def test_split_copy_layout_index_algebra():
    """The split state layout: from the packed words p_k = hi_k | lo_k << 16,
    group g of eight amplitudes of hi copy t (t < 8) is the words
    W[j ^ (t >> 1)], j = 0..3, with W = byte permutes 0x5410 (t even) or 0x1054
    (t odd) of the word pairs (p_{8g+2k}, p_{8g+2k+1}); lo the same with 0x7632 /
    0x3276.  Copy t then holds hi_{k ^ t}, and target elements 8c .. 8c + 7 of a
    term's 16-block are copy (x & 7) at rb + 8 (c ^ bit 3 of x)."""
    N = 64
    rng = np.random.default_rng(3)
    hi = rng.integers(0, 1 << 16, N)
    lo = rng.integers(0, 1 << 16, N)
    packed = [int(h) | (int(l) << 16) for h, l in zip(hi, lo)]
    H = np.zeros((8, N), dtype=np.int64)
    Lo = np.zeros((8, N), dtype=np.int64)
    for g in range(N // 8):
        pw = packed[8 * g:8 * g + 8]
        HP = [prmt(pw[2 * k], pw[2 * k + 1], 0x5410) for k in range(4)]
        HS = [prmt(pw[2 * k], pw[2 * k + 1], 0x1054) for k in range(4)]
        LP = [prmt(pw[2 * k], pw[2 * k + 1], 0x7632) for k in range(4)]
        LS = [prmt(pw[2 * k], pw[2 * k + 1], 0x3276) for k in range(4)]
        for t in range(8):
            u = t >> 1
            Wh, Wl = (HS, LS) if t & 1 else (HP, LP)
            for j in range(4):
                for half in range(2):
                    H[t, 8 * g + 2 * j + half] = (Wh[j ^ u] >> (16 * half)) & 0xFFFF
                    Lo[t, 8 * g + 2 * j + half] = (Wl[j ^ u] >> (16 * half)) & 0xFFFF
    for t in range(8):
        assert np.array_equal(H[t], hi[np.arange(N) ^ t])
        assert np.array_equal(Lo[t], lo[np.arange(N) ^ t])
    for xl in range(N):
        xlo = xl & 15
        for rb in range(0, N, 16):
            for i in range(16):
                c, e = i >> 3, i & 7
                src = rb + 8 * (c ^ (xlo >> 3)) + e
                assert hi[rb | (i ^ xlo)] == H[xlo & 7, src]
                assert lo[rb | (i ^ xlo)] == Lo[xlo & 7, src]


def test_scaled_rotation_form():
    """Ry(theta) = c [[1, -t], [t, 1]] (t = s / c) when |c| >= |s|, else
    s [[u, -1], [1, u]] (u = c / s): the HBM passes apply the bracketed
    matrices (one FMA per amplitude) and the product of the factors at the end;
    |t|, |u| <= 1 always."""
    rng = np.random.default_rng(7)
    for theta in np.concatenate([rng.uniform(-4 * np.pi, 4 * np.pi, 200), [0.0, np.pi, -np.pi, np.pi / 2, 3 * np.pi]]):
        c, s = np.cos(theta / 2), np.sin(theta / 2)
        ry = np.array([[c, -s], [s, c]])
        if abs(c) >= abs(s):
            r, fac, m = s / c, c, np.array([[1.0, -s / c], [s / c, 1.0]])
        else:
            r, fac, m = c / s, s, np.array([[c / s, -1.0], [1.0, c / s]])
        assert abs(r) <= 1.0
        assert np.allclose(fac * m, ry, atol=1e-15)
    # twelve rotations with the factors deferred to the end
    v = rng.normal(size=(2,))
    w = v.copy()
    fac = 1.0
    for theta in rng.uniform(-np.pi, np.pi, 12):
        c, s = np.cos(theta / 2), np.sin(theta / 2)
        v = np.array([[c, -s], [s, c]]) @ v
        if abs(c) >= abs(s):
            t = s / c
            w = np.array([w[0] - t * w[1], w[1] + t * w[0]])
            fac *= c
        else:
            u = c / s
            w = np.array([u * w[0] - w[1], u * w[1] + w[0]])
            fac *= s
    assert np.allclose(fac * w, v, atol=1e-13)


def czring_parity(i, n):
    """Sign bit of the CZ ring on amplitude i: pairs (k, k + 1), k < n - 1, and (n - 1, 0)."""
    p = popc(i & (i >> 1) & ((1 << (n - 1)) - 1))
    if n >= 3:
        p += (i >> (n - 1)) & i & 1
    return p & 1


def test_czring_sign_from_index_parts():
    """The low-qubit HBM pass forms the CZ-ring sign of i = base | 16 t | r
    (base: bits 12.., t: bits 4..11, r: bits 0..3) from its parts: the thread's
    part czring(base | 16 t), the pairs inside r, the pair (3, 4) and the
    wrap-around pair (n - 1, 0)."""
    rng = np.random.default_rng(11)
    for n in (13, 16, 20):
        for _ in range(3000):
            base = int(rng.integers(0, 1 << (n - 12))) << 12
            t, r = int(rng.integers(0, 256)), int(rng.integers(0, 16))
            p = czring_parity(base | (t << 4), n) ^ (popc(r & (r >> 1)) & 1)
            if r & 8:
                p ^= t & 1
            if r & 1:
                p ^= (base >> (n - 1)) & 1
            assert p == czring_parity(base | (t << 4) | r, n)


def test_low_pass_transpose_layouts():
    """The low-qubit HBM pass's chunk of 4096 amplitudes: the three thread
    layouts (16 consecutive amplitudes per thread; bits 4..7 on the registers;
    bits 8..11 on the registers) each cover the chunk once, and the padded word
    e + 4 (e >> 5) + 16 (e >> 8) is one-to-one, keeps 16-byte groups whole, puts
    the 16-byte stores of eight consecutive threads in eight bank groups, and
    the 256-strided half-warps of the second layout 16 banks apart."""
    LOC = 4096
    pad = lambda e: e + ((e >> 5) << 2) + ((e >> 8) << 4)
    words = [pad(e) for e in range(LOC)]
    assert len(set(words)) == LOC
    A = sorted(16 * t + r for t in range(256) for r in range(16))
    B = sorted(((t & 15) | ((t >> 4) << 8)) | (r << 4) for t in range(256) for r in range(16))
    C = sorted(t | (r << 8) for t in range(256) for r in range(16))
    assert A == B == C == list(range(LOC))
    for t in range(256):
        for c in range(4):
            e = 16 * t + 4 * c
            assert pad(e) % 4 == 0 and all(pad(e + k) == pad(e) + k for k in range(4))
    for t0 in range(0, 256, 8):
        for c in range(4):
            groups = {(pad(16 * t + 4 * c) // 4) % 8 for t in range(t0, t0 + 8)}
            assert len(groups) == 8
    for w in range(8):
        for r in range(16):
            lanes = range(32 * w, 32 * w + 32)
            for layout in (lambda t: ((t & 15) | ((t >> 4) << 8)) | (r << 4), lambda t: t | (r << 8)):
                banks = [pad(layout(t)) % 32 for t in lanes]
                assert len(set(banks)) == 32
