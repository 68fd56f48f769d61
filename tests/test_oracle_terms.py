"""Pins of the state / term / cost / gradient oracles.

Independent references: dense Kronecker-built gates and Pauli strings
(n <= 5), the n = 1 closed form, Gram-matrix invariants, a planted exact
solution, central finite differences, and agreement between the two
oracles (definition level vs the gate-by-gate Hadamard-test circuits)."""
from functools import reduce

import numpy as np
import pytest

from oracle import circuit, terms
from oracle import decompose as dec
from paper_2604_14435_gb300 import workloads as wl

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.diag([1.0, 0.0]).astype(complex)
P1 = np.diag([0.0, 1.0]).astype(complex)


def embed(ops, n):
    """Kronecker product with ops[q] on qubit q (identity elsewhere); qubit n-1 leftmost."""
    return reduce(np.kron, [ops.get(q, I2) for q in reversed(range(n))])


def ry(t):
    return np.array([[np.cos(t / 2), -np.sin(t / 2)], [np.sin(t / 2), np.cos(t / 2)]], dtype=complex)


def cz_dense(q1, q2, n):
    return embed({q1: P0}, n) + embed({q1: P1, q2: PZ}, n)


def ansatz_dense(n, d, alpha):
    V = embed({q: ry(alpha[q]) for q in range(n)}, n)
    for layer in range(1, d + 1):
        ring = np.eye(1 << n, dtype=complex)
        pairs = [(q, q + 1) for q in range(n - 1)] + ([(n - 1, 0)] if n >= 3 else [])
        for q1, q2 in pairs:
            ring = cz_dense(q1, q2, n) @ ring
        V = embed({q: ry(alpha[layer * n + q]) for q in range(n)}, n) @ ring @ V
    return V


def pauli_dense(x, z, n):
    return embed({q: (PY if (x >> q) & (z >> q) & 1 else PX if (x >> q) & 1 else PZ if (z >> q) & 1 else I2)
                  for q in range(n)}, n)


def random_lcu(rng, n, L, real=False):
    N = 1 << n
    xs = rng.integers(0, N, L).astype(np.uint32)
    zs = rng.integers(0, N, L).astype(np.uint32)
    c = rng.normal(size=L) + (0 if real else 1j * rng.normal(size=L))
    return c, xs, zs


@pytest.mark.parametrize("n,d", [(1, 0), (1, 3), (2, 1), (3, 2), (4, 2), (5, 3)])
def test_state_matches_dense_circuit(n, d):
    alpha = wl.random_angles(n * (d + 1), 5 + n)
    psi = terms.ansatz_state(n, d, alpha)
    e0 = np.zeros(1 << n, dtype=complex)
    e0[0] = 1
    assert np.abs(psi - ansatz_dense(n, d, alpha) @ e0).max() < 1e-14
    assert np.abs(circuit.ansatz_state(n, d, alpha) - psi).max() < 1e-14
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-14


def test_single_qubit_closed_form():
    """n = 1: psi = (cos s/2, sin s/2) with s the sum of the angles; <X> = sin s, <Z> = cos s."""
    alpha = np.array([0.3, -1.1, 2.0])
    s = alpha.sum()
    psi = terms.ansatz_state(1, 2, alpha)
    assert np.allclose(psi, [np.cos(s / 2), np.sin(s / 2)], atol=1e-15)
    beta, _ = terms.beta_delta(psi, wl.plus_state(1), [0, 1], [1, 0])
    # beta[0,1] = <Z X> = i <Y> = 0 for a real state; beta via sigma products
    assert abs(np.vdot(psi, pauli_dense(1, 0, 1) @ psi) - np.sin(s)) < 1e-15
    assert abs(beta[0, 0] - 1.0) < 1e-15
    assert abs(circuit.hadamard_beta(1, 2, alpha, 0, 0, 1, 0) - np.sin(s)) < 1e-14
    assert abs(circuit.hadamard_beta(1, 2, alpha, 0, 0, 0, 1) - np.cos(s)) < 1e-14


def test_zero_angles_give_basis_state():
    psi = terms.ansatz_state(4, 3, np.zeros(16))
    assert psi[0] == 1.0 and np.count_nonzero(psi) == 1


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_terms_match_dense_brute_force(n):
    rng = np.random.default_rng(40 + n)
    d = 2
    alpha = wl.random_angles(n * (d + 1), 60 + n)
    c, xs, zs = random_lcu(rng, n, 6)
    b = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    b /= np.linalg.norm(b)
    psi = ansatz_dense(n, d, alpha)[:, 0]
    beta, delta = terms.beta_delta(terms.ansatz_state(n, d, alpha), b, xs, zs)
    for l in range(6):
        Sl = pauli_dense(int(xs[l]), int(zs[l]), n)
        assert abs(delta[l] - np.vdot(b, Sl @ psi)) < 1e-14
        for m in range(6):
            Sm = pauli_dense(int(xs[m]), int(zs[m]), n)
            assert abs(beta[l, m] - np.vdot(psi, Sl.conj().T @ Sm @ psi)) < 1e-14
    A = sum(ci * pauli_dense(int(x), int(z), n) for ci, x, z in zip(c, xs, zs))
    C, N, D = terms.combine(c, beta, delta)
    assert abs(N - abs(np.vdot(b, A @ psi)) ** 2) < 1e-13
    assert abs(D - np.vdot(psi, A.conj().T @ A @ psi)) < 1e-13
    assert abs(C - (1 - abs(np.vdot(b, A @ psi)) ** 2 / np.vdot(psi, A.conj().T @ A @ psi).real)) < 1e-13


@pytest.mark.parametrize("n,d,L", [(1, 1, 3), (2, 2, 5), (3, 2, 8), (5, 2, 6), (6, 3, 5)])
@pytest.mark.parametrize("bkind", ["plus", "complex"])
def test_circuits_match_definition(n, d, L, bkind):
    """Hadamard-test circuits on n+1 qubits reproduce the definition-level terms."""
    rng = np.random.default_rng(1000 * n + L)
    alpha = wl.random_angles(n * (d + 1), 70 + n)
    _, xs, zs = random_lcu(rng, n, L)
    if bkind == "plus":
        b = wl.plus_state(n)
    else:
        b = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
        b /= np.linalg.norm(b)
    beta, delta = terms.beta_delta(terms.ansatz_state(n, d, alpha), b, xs, zs)
    cb, cd, _ = circuit.circuit_terms(n, d, alpha, b, xs, zs)
    assert np.abs(cb - beta).max() < 1e-13
    assert np.abs(cd - delta).max() < 1e-13
    if bkind == "plus":  # U_b as H^n and as the Householder reflection agree
        for l in range(L):
            v = circuit.hadamard_delta(n, d, alpha, b, int(xs[l]), int(zs[l]), b_plus=False)
            assert abs(v - delta[l]) < 1e-13


def test_gram_invariants():
    """beta_ll = 1, Hermitian, PSD, |beta| <= 1; real for a real state, real b
    and strings with an even number of Y."""
    n, d = 6, 3
    out = dec.decompose(wl.toeplitz_dense(n, 2.2, -0.8))
    psi = terms.ansatz_state(n, d, wl.random_angles(n * (d + 1), 3))
    beta, delta = terms.beta_delta(psi, wl.plus_state(n), out["x"], out["z"])
    assert np.abs(np.diag(beta) - 1).max() < 1e-14
    assert np.abs(beta - beta.conj().T).max() < 1e-15
    assert np.linalg.eigvalsh(beta).min() > -1e-12
    assert np.abs(beta).max() <= 1 + 1e-14 and np.abs(delta).max() <= 1 + 1e-14
    assert np.abs(beta.imag).max() < 1e-15 and np.abs(delta.imag).max() < 1e-15


def test_planted_solution_gives_zero_cost_and_gradient():
    n, d = 4, 2
    rng = np.random.default_rng(9)
    c, xs, zs = random_lcu(rng, n, 7)
    alpha_star = wl.random_angles(n * (d + 1), 19)
    psi = terms.ansatz_state(n, d, alpha_star)
    A = terms.lcu_matrix(c, xs, zs, n)
    b = A @ psi
    b /= np.linalg.norm(b)
    r = terms.cost_grad(n, d, alpha_star, b, c, xs, zs)
    assert abs(r["cost"]) < 1e-14
    assert np.abs(r["grad"]).max() < 1e-13
    xhat = terms.classical_solution(A, b)
    assert abs(terms.fidelity(psi, xhat) - 1.0) < 1e-12
    assert np.linalg.norm(A @ (xhat * (np.vdot(xhat, psi))) - A @ psi) < 1e-12


def test_identity_system_cost():
    """L = 1, A = I: C = 1 - |<b|psi>|^2, and 0 <= C <= 1."""
    n, d = 3, 2
    b = np.random.default_rng(4).normal(size=8) + 0j
    b /= np.linalg.norm(b)
    for seed in range(5):
        alpha = wl.random_angles(9, seed)
        psi = terms.ansatz_state(n, d, alpha)
        C = terms.cost_only(n, d, alpha, b, [1.0], [0], [0])
        assert abs(C - (1 - abs(np.vdot(b, psi)) ** 2)) < 1e-15
        assert 0.0 <= C <= 1.0


@pytest.mark.parametrize("n,d", [(2, 1), (3, 2), (4, 2)])
def test_shift_rule_matches_finite_differences(n, d):
    rng = np.random.default_rng(50 + n)
    c, xs, zs = random_lcu(rng, n, 5)
    b = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    b /= np.linalg.norm(b)
    alpha = wl.random_angles(n * (d + 1), 80 + n)
    r = terms.cost_grad(n, d, alpha, b, c, xs, zs)
    h = 1e-5
    for k in range(alpha.size):
        e = np.zeros_like(alpha)
        e[k] = h
        fd = (terms.cost_only(n, d, alpha + e, b, c, xs, zs) - terms.cost_only(n, d, alpha - e, b, c, xs, zs)) / (2 * h)
        assert abs(fd - r["grad"][k]) < 1e-8


def test_circuit_cost_grad_matches_definition():
    n, d = 3, 2
    sysd = wl.validation_system()
    out = dec.decompose(sysd["A"])
    alpha = sysd["alphas"][0]
    r1 = terms.cost_grad(n, d, alpha, sysd["b"], out["coef"], out["x"], out["z"])
    r2 = circuit.circuit_cost_grad(n, d, alpha, sysd["b"], out["coef"], out["x"], out["z"])
    assert abs(r1["cost"] - r2["cost"]) < 1e-13
    assert np.abs(r1["grad"] - r2["grad"]).max() < 1e-13
    assert out["L_out"] == 8
