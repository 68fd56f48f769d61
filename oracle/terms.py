"""Definition-level FP64 CPU oracle for the VQLS global cost and its gradient.

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
library.

What it computes, each quantity straight from its definition:
  - psi(alpha) = V(alpha)|0> (Sec. 2.1), gate by gate, for the Ry + CZ-ring
    hardware-efficient ansatz: an Ry layer alpha[0..n), then d times
    { CZ ring ; Ry layer alpha[l*n .. l*n+n) }.
  - beta_lm = <psi| A_l^dag A_m |psi> and delta_l = <b| A_l |psi> for Pauli
    strings A_l (Eq. 3, Eq. 4 denominator; Eq. 1 numerator), as
    beta = Phi^H Phi and delta = Phi^T conj(b) with Phi[:, l] = A_l psi.
  - Eq. 1 with A = sum_l c_l A_l: N = |sum_l c_l delta_l|^2,
    D = sum_lm conj(c_l) c_m beta_lm, C = 1 - N / D.
  - The gradient by the parameter-shift rule: each angle enters one
    exp(-i a Y / 2) gate and N, D are expectation values, so
    f'(a) = [f(a + pi/2) - f(a - pi/2)] / 2 holds exactly for both;
    dC = -(N' D - N D') / D^2.  Shift s = 0 is alpha, s = 2k+1 is
    alpha + (pi/2) e_k and s = 2k+2 is alpha - (pi/2) e_k.
  - Fidelity F = |<xhat|psi>|^2 (Sec. 3.1).
  - The local cost (Eq. 2, expanded in Eq. 4) for b = |+>^n, where
    U_b Z_j U_b^dag = X_j: with P_j = (I + Z_j)/2,
    C_L = 1 - (1/n) sum_j sum_lm conj(c_l) c_m (beta_lm + gamma^j_lm) / (2 D)
        = 1/2 - Re[E / (n D)] / 2,  E = sum_j sum_lm conj(c_l) c_m gamma^j_lm,
    gamma^j_lm = <psi| A_l^dag X_j A_m |psi> (the closed form of Sec. 2.3,
    Stage III), and its parameter-shift gradient from E and D.

Conventions: qubit k is bit k of the basis index; Ry(t) = [[cos t/2,
-sin t/2], [sin t/2, cos t/2]]; CZ ring = CZ(q, q+1) for q < n-1 plus
CZ(n-1, 0) when n >= 3; sigma(x,z) = i^popc(x&z) X^x Z^z.
"""
import numpy as np

from .decompose import popcount


def num_angles(n, d):
    return n * (d + 1)


def apply_ry(psi, n, q, theta):
    c, s = np.cos(0.5 * theta), np.sin(0.5 * theta)
    v = psi.reshape(-1, 2, 1 << q)
    a = v[:, 0, :].copy()
    b = v[:, 1, :].copy()
    v[:, 0, :] = c * a - s * b
    v[:, 1, :] = s * a + c * b
    return v.reshape(-1)


def apply_cz(psi, q1, q2):
    i = np.arange(psi.size)
    both = ((i >> q1) & 1) & ((i >> q2) & 1)
    return np.where(both == 1, -psi, psi)


def ansatz_state(n, d, alpha):
    """psi = V(alpha)|0>, complex128 of length 2^n."""
    alpha = np.asarray(alpha, dtype=np.float64)
    assert alpha.size == num_angles(n, d)
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    for q in range(n):
        psi = apply_ry(psi, n, q, alpha[q])
    for layer in range(1, d + 1):
        for q in range(n - 1):
            psi = apply_cz(psi, q, q + 1)
        if n >= 3:
            psi = apply_cz(psi, n - 1, 0)
        for q in range(n):
            psi = apply_ry(psi, n, q, alpha[layer * n + q])
    return psi


def apply_pauli(x, z, v):
    """sigma(x,z) v with sigma|i> = i^popc(x&z) (-1)^popc(z&i) |i XOR x>."""
    N = v.size
    i = np.arange(N)
    phase = 1j ** (int(popcount(int(x) & int(z))) % 4)
    sign = 1.0 - 2.0 * (popcount(int(z) & i) % 2)
    out = np.zeros(N, dtype=np.complex128)
    out[i ^ int(x)] = phase * sign * v
    return out


def beta_delta(psi, b, xs, zs):
    """beta (L x L) and delta (L) by their definitions."""
    Phi = np.stack([apply_pauli(x, z, psi) for x, z in zip(xs, zs)], axis=1)
    beta = Phi.conj().T @ Phi
    delta = Phi.T @ np.conj(np.asarray(b, dtype=np.complex128))
    return beta, delta


def combine(coef, beta, delta):
    """(C, N, D) from the terms: Eq. 1 with A = sum_l c_l A_l."""
    coef = np.asarray(coef, dtype=np.complex128)
    T = np.sum(coef * delta)
    Nv = float(np.abs(T) ** 2)
    Dc = np.conj(coef) @ beta @ coef
    return 1.0 - Nv / Dc.real, Nv, Dc


def shifted_angles(alpha):
    """The 2P+1 angle vectors of the parameter-shift rule, rows s = 0..2P."""
    alpha = np.asarray(alpha, dtype=np.float64)
    P = alpha.size
    out = np.tile(alpha, (2 * P + 1, 1))
    for k in range(P):
        out[2 * k + 1, k] += 0.5 * np.pi
        out[2 * k + 2, k] -= 0.5 * np.pi
    return out


def cost_grad(n, d, alpha, b, coef, xs, zs):
    """Cost, gradient and the unshifted terms.

    Returns dict: cost, grad (P), beta (L x L), delta (L), N_s, D_s (per shift,
    D_s complex so its imaginary residual is visible)."""
    shifts = shifted_angles(alpha)
    S = shifts.shape[0]
    Ns = np.zeros(S)
    Ds = np.zeros(S, dtype=np.complex128)
    beta0 = delta0 = None
    for s in range(S):
        psi = ansatz_state(n, d, shifts[s])
        beta, delta = beta_delta(psi, b, xs, zs)
        _, Ns[s], Ds[s] = combine(coef, beta, delta)
        if s == 0:
            beta0, delta0 = beta, delta
    D = Ds.real
    P = len(alpha)
    dN = 0.5 * (Ns[1::2] - Ns[2::2])
    dD = 0.5 * (D[1::2] - D[2::2])
    grad = -(dN * D[0] - Ns[0] * dD) / (D[0] ** 2)
    assert grad.size == P
    return {"cost": 1.0 - Ns[0] / D[0], "grad": grad, "beta": beta0, "delta": delta0,
            "N_s": Ns, "D_s": Ds}


def cost_only(n, d, alpha, b, coef, xs, zs):
    psi = ansatz_state(n, d, alpha)
    beta, delta = beta_delta(psi, b, xs, zs)
    return combine(coef, beta, delta)[0]


def lcu_matrix(coef, xs, zs, n):
    """Dense A~ = sum_l c_l sigma_l (for the classical solve at small n):
    entry [i XOR x, i] of sigma(x,z) is i^popc(x&z) (-1)^popc(z&i)."""
    N = 1 << n
    M = np.zeros((N, N), dtype=np.complex128)
    i = np.arange(N)
    for c, x, z in zip(coef, xs, zs):
        phase = 1j ** (int(popcount(int(x) & int(z))) % 4)
        sign = 1.0 - 2.0 * (popcount(int(z) & i) % 2)
        M[i ^ int(x), i] += c * phase * sign
    return M


def classical_solution(M, b):
    """xhat = M^{-1} b normalised (the direct solve the fidelity is measured against)."""
    x = np.linalg.solve(M, np.asarray(b, dtype=np.complex128))
    return x / np.linalg.norm(x)


def fidelity(psi, xhat):
    return float(np.abs(np.vdot(xhat, psi)) ** 2)


def apply_x(j, v):
    """X on qubit j: amplitude i takes the value at i XOR 2^j."""
    i = np.arange(v.size)
    return v[i ^ (1 << j)]


def local_terms(psi, xs, zs, n):
    """beta (L x L) and gamma (n x L x L) for b = |+>^n by their definitions."""
    Phi = np.stack([apply_pauli(x, z, psi) for x, z in zip(xs, zs)], axis=1)
    beta = Phi.conj().T @ Phi
    gamma = np.stack([Phi.conj().T @ np.stack([apply_x(j, Phi[:, m]) for m in range(Phi.shape[1])], axis=1)
                      for j in range(n)])
    return beta, gamma


def local_combine(coef, beta, gamma):
    """(C_L, E, D): E = sum_j conj(c)^T gamma^j c, D = conj(c)^T beta c."""
    coef = np.asarray(coef, dtype=np.complex128)
    D = (np.conj(coef) @ beta @ coef).real
    E = sum((np.conj(coef) @ g @ coef).real for g in gamma)
    n = len(gamma)
    return 0.5 - 0.5 * E / (n * D), E, D


def local_cost_grad(n, d, alpha, coef, xs, zs):
    """Local cost (b = |+>^n) and its parameter-shift gradient."""
    shifts = shifted_angles(alpha)
    S = shifts.shape[0]
    E = np.zeros(S)
    D = np.zeros(S)
    for s in range(S):
        beta, gamma = local_terms(ansatz_state(n, d, shifts[s]), xs, zs, n)
        _, E[s], D[s] = local_combine(coef, beta, gamma)
    dE = 0.5 * (E[1::2] - E[2::2])
    dD = 0.5 * (D[1::2] - D[2::2])
    return {"cost": 0.5 - 0.5 * E[0] / (n * D[0]), "grad": -0.5 * (dE * D[0] - E[0] * dD) / (n * D[0] ** 2),
            "E_s": E, "D_s": D}
