"""Pins of the local-cost oracle (Eq. 2, expanded in Eq. 4; closed form of
Sec. 2.3 Stage III) against dense projector matrices, the circuits with a
general U_b, a planted solution and finite differences."""
from functools import reduce

import numpy as np
import pytest

from oracle import circuit, terms
from paper_2604_14435_gb300 import workloads as wl

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
H1 = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)


def embed(ops, n):
    return reduce(np.kron, [ops.get(q, I2) for q in reversed(range(n))])


def pauli_dense(x, z, n):
    return embed({q: (PY if (x >> q) & (z >> q) & 1 else PX if (x >> q) & 1 else PZ if (z >> q) & 1 else I2)
                  for q in range(n)}, n)


def dense_local_cost(n, psi, coef, xs, zs, Ub):
    """1 - (1/n) sum_j <x|A^dag U_b P_j U_b^dag A|x> / <x|A^dag A|x>, P_j = |0><0|_j."""
    A = sum(c * pauli_dense(int(x), int(z), n) for c, x, z in zip(coef, xs, zs))
    Ax = A @ psi
    den = np.vdot(Ax, Ax).real
    num = 0.0
    for j in range(n):
        Pj = embed({j: np.diag([1.0, 0.0]).astype(complex)}, n)
        num += np.vdot(Ax, Ub @ Pj @ Ub.conj().T @ Ax).real
    return 1.0 - num / (n * den)


def random_lcu(rng, n, L):
    N = 1 << n
    return (rng.normal(size=L) + 1j * rng.normal(size=L), rng.integers(0, N, L).astype(np.uint32),
            rng.integers(0, N, L).astype(np.uint32))


@pytest.mark.parametrize("n,d,L", [(1, 1, 2), (2, 2, 3), (3, 2, 5), (4, 1, 6)])
def test_local_cost_matches_dense_projectors(n, d, L):
    rng = np.random.default_rng(30 + n)
    coef, xs, zs = random_lcu(rng, n, L)
    alpha = wl.random_angles(n * (d + 1), 31 + n)
    psi = terms.ansatz_state(n, d, alpha)
    beta, gamma = terms.local_terms(psi, xs, zs, n)
    C, E, D = terms.local_combine(coef, beta, gamma)
    assert abs(C - dense_local_cost(n, psi, coef, xs, zs, embed({q: H1 for q in range(n)}, n))) < 1e-13
    assert -1e-14 <= C <= 1.0 + 1e-14


@pytest.mark.parametrize("n,d,L", [(1, 1, 2), (3, 2, 4), (5, 1, 3)])
def test_gamma_circuits_match_definition(n, d, L):
    rng = np.random.default_rng(40 + n)
    _, xs, zs = random_lcu(rng, n, L)
    alpha = wl.random_angles(n * (d + 1), 41 + n)
    _, gamma = terms.local_terms(terms.ansatz_state(n, d, alpha), xs, zs, n)
    cg, _ = circuit.circuit_local_terms(n, d, alpha, wl.plus_state(n), xs, zs)
    assert np.abs(cg - gamma).max() < 1e-13


def test_gamma_circuits_general_b():
    """With a general b the circuits use the Householder U_b: compare with the
    dense operator A_l^dag U_b Z_j U_b^dag A_m."""
    n, d, L = 3, 2, 3
    rng = np.random.default_rng(5)
    coef, xs, zs = random_lcu(rng, n, L)
    b = rng.normal(size=8) + 1j * rng.normal(size=8)
    b /= np.linalg.norm(b)
    alpha = wl.random_angles(9, 6)
    psi = terms.ansatz_state(n, d, alpha)
    ph = b[0] / abs(b[0])
    w = ph * np.eye(8)[0] - b
    Ub = ph * (np.eye(8) - 2 * np.outer(w, w.conj()) / np.vdot(w, w).real)
    assert np.allclose(Ub @ np.eye(8)[0], b)
    cg, _ = circuit.circuit_local_terms(n, d, alpha, b, xs, zs, b_plus=False)
    for j in range(n):
        Zj = embed({j: PZ}, n)
        for l in range(L):
            for m in range(L):
                ref = np.vdot(psi, pauli_dense(int(xs[l]), int(zs[l]), n).conj().T @ Ub @ Zj @ Ub.conj().T
                              @ pauli_dense(int(xs[m]), int(zs[m]), n) @ psi)
                assert abs(cg[j, l, m] - ref) < 1e-13


def test_local_cost_zero_at_planted_solution():
    """A x proportional to |+>^n gives C_L = 0 (and a zero gradient)."""
    n, d = 3, 2
    rng = np.random.default_rng(8)
    alpha = wl.random_angles(9, 9)
    psi = terms.ansatz_state(n, d, alpha)
    # A = |+><psi| + small terms orthogonal in the Pauli basis would not stay an LCU of few terms;
    # use A = sum over all Pauli strings of Tr(sigma^dag M)/N with M = |+><psi| + (I - |psi><psi|)
    plus = wl.plus_state(n)
    M = np.outer(plus, psi.conj()) + (np.eye(8) - np.outer(psi, psi.conj()))
    xs, zs, coef = [], [], []
    for x in range(8):
        for z in range(8):
            c = np.trace(pauli_dense(x, z, n).conj().T @ M) / 8
            if abs(c) > 1e-15:
                xs.append(x)
                zs.append(z)
                coef.append(c)
    r = terms.local_cost_grad(n, d, alpha, np.array(coef), np.array(xs, np.uint32), np.array(zs, np.uint32))
    assert abs(r["cost"]) < 1e-13 and np.abs(r["grad"]).max() < 1e-12


def test_local_shift_rule_and_circuits():
    n, d, L = 3, 1, 4
    rng = np.random.default_rng(12)
    coef, xs, zs = random_lcu(rng, n, L)
    alpha = wl.random_angles(6, 13)
    r = terms.local_cost_grad(n, d, alpha, coef, xs, zs)
    h = 1e-5

    def C(a):
        beta, gamma = terms.local_terms(terms.ansatz_state(n, d, a), xs, zs, n)
        return terms.local_combine(coef, beta, gamma)[0]

    for k in range(alpha.size):
        e = np.zeros_like(alpha)
        e[k] = h
        assert abs((C(alpha + e) - C(alpha - e)) / (2 * h) - r["grad"][k]) < 1e-8
    rc = circuit.circuit_local_cost_grad(n, d, alpha, wl.plus_state(n), coef, xs, zs)
    assert abs(rc["cost"] - r["cost"]) < 1e-13 and np.abs(rc["grad"] - r["grad"]).max() < 1e-13
