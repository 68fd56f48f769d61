"""The identities the fast kernels rest on, checked in plain numpy on small
random cases (CPU): the Walsh-Hadamard form of the real Gram terms (global
cost, and the local cost's X_j flavours), and the index algebra of the
four-copy state layout of the tensor-core tiles."""
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
