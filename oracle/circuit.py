"""ctypes wrapper of the circuit-level oracle (hadamard_sim.c).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every Hadamard-test
circuit of the global cost is simulated gate by gate on n+1 qubits in FP64;
the combine of Eq. 1 and the parameter-shift gradient are then taken from the
simulated terms."""
import ctypes
import os

import numpy as np

from . import build_csim
from .terms import shifted_angles, combine

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_csim.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        up = ctypes.POINTER(ctypes.c_uint32)
        L.oracle_ansatz_state.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        L.oracle_hadamard_beta.argtypes = [ctypes.c_int, ctypes.c_int, dp] + [ctypes.c_uint32] * 4 + [dp, dp]
        L.oracle_hadamard_delta.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                            ctypes.c_uint32, ctypes.c_uint32, dp, dp]
        L.oracle_circuit_terms.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int,
                                           up, up, dp, dp, ctypes.c_int]
        L.oracle_circuit_local_terms.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int,
                                                 up, up, dp, ctypes.c_int]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _up(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _cvec(b):
    return np.ascontiguousarray(np.asarray(b, dtype=np.complex128))


def ansatz_state(n, d, alpha):
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    out = np.zeros(1 << n, dtype=np.complex128)
    assert lib().oracle_ansatz_state(n, d, _dp(a), _dp(out.view(np.float64))) == 0
    return out


def is_plus_state(b):
    b = np.asarray(b, dtype=np.complex128)
    return bool(np.all(b == b[0]) and b[0] == 1.0 / np.sqrt(b.size))


def hadamard_beta(n, d, alpha, xl, zl, xm, zm):
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    re, im = ctypes.c_double(), ctypes.c_double()
    assert lib().oracle_hadamard_beta(n, d, _dp(a), xl, zl, xm, zm, ctypes.byref(re), ctypes.byref(im)) == 0
    return complex(re.value, im.value)


def hadamard_delta(n, d, alpha, b, xl, zl, b_plus=None):
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    bv = _cvec(b)
    if b_plus is None:
        b_plus = is_plus_state(bv)
    re, im = ctypes.c_double(), ctypes.c_double()
    assert lib().oracle_hadamard_delta(n, d, _dp(a), _dp(bv.view(np.float64)), int(b_plus), xl, zl,
                                       ctypes.byref(re), ctypes.byref(im)) == 0
    return complex(re.value, im.value)


def circuit_terms(n, d, alpha, b, xs, zs, nthreads=0, b_plus=None):
    """All beta (L x L) and delta (L) from 2 (L^2 + L) simulated circuits.
    Returns (beta, delta, threads used)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    bv = _cvec(b)
    if b_plus is None:
        b_plus = is_plus_state(bv)
    x = np.ascontiguousarray(xs, dtype=np.uint32)
    z = np.ascontiguousarray(zs, dtype=np.uint32)
    L = x.size
    beta = np.zeros((L, L), dtype=np.complex128)
    delta = np.zeros(L, dtype=np.complex128)
    used = lib().oracle_circuit_terms(n, d, _dp(a), _dp(bv.view(np.float64)), int(b_plus), L, _up(x), _up(z),
                                      _dp(beta.view(np.float64)), _dp(delta.view(np.float64)), int(nthreads))
    assert used > 0
    return beta, delta, used


def circuit_cost_grad(n, d, alpha, b, coef, xs, zs, nthreads=0, shifts=None):
    """Cost and parameter-shift gradient with every term from its circuits.

    shifts: optional list of shift indices to evaluate (a bounded sample);
    then only N_s, D_s of those shifts are returned."""
    A = shifted_angles(alpha)
    idx = range(A.shape[0]) if shifts is None else shifts
    Ns, Ds = {}, {}
    beta0 = delta0 = None
    for s in idx:
        beta, delta, _ = circuit_terms(n, d, A[s], b, xs, zs, nthreads)
        _, Ns[s], Ds[s] = combine(coef, beta, delta)
        if s == 0:
            beta0, delta0 = beta, delta
    out = {"N_s": Ns, "D_s": Ds, "beta": beta0, "delta": delta0}
    if shifts is None:
        S = A.shape[0]
        N = np.array([Ns[s] for s in range(S)])
        D = np.array([Ds[s].real for s in range(S)])
        dN = 0.5 * (N[1::2] - N[2::2])
        dD = 0.5 * (D[1::2] - D[2::2])
        out["cost"] = 1.0 - N[0] / D[0]
        out["grad"] = -(dN * D[0] - N[0] * dD) / D[0] ** 2
    return out


def circuit_local_terms(n, d, alpha, b, xs, zs, nthreads=0, b_plus=None):
    """gamma[j, l, m] = <psi| A_l^dag U_b Z_j U_b^dag A_m |psi> from 2 n L^2
    simulated circuits.  Returns (gamma, threads used)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    bv = _cvec(b)
    if b_plus is None:
        b_plus = is_plus_state(bv)
    x = np.ascontiguousarray(xs, dtype=np.uint32)
    z = np.ascontiguousarray(zs, dtype=np.uint32)
    L = x.size
    gamma = np.zeros((n, L, L), dtype=np.complex128)
    used = lib().oracle_circuit_local_terms(n, d, _dp(a), _dp(bv.view(np.float64)), int(b_plus), L, _up(x),
                                            _up(z), _dp(gamma.view(np.float64)), int(nthreads))
    assert used > 0
    return gamma, used


def circuit_local_cost_grad(n, d, alpha, b, coef, xs, zs, nthreads=0):
    """Local cost C_L and its parameter-shift gradient with every overlap from
    its Hadamard-test circuits (2 (n+1) L^2 per angle vector)."""
    from .terms import local_combine
    A = shifted_angles(alpha)
    E = np.zeros(A.shape[0])
    D = np.zeros(A.shape[0])
    for s in range(A.shape[0]):
        beta, _, _ = circuit_terms(n, d, A[s], b, xs, zs, nthreads)
        gamma, _ = circuit_local_terms(n, d, A[s], b, xs, zs, nthreads)
        _, E[s], D[s] = local_combine(coef, beta, gamma)
    n_ = float(n)
    dE = 0.5 * (E[1::2] - E[2::2])
    dD = 0.5 * (D[1::2] - D[2::2])
    return {"cost": 0.5 - 0.5 * E[0] / (n_ * D[0]),
            "grad": -0.5 * (dE * D[0] - E[0] * dD) / (n_ * D[0] ** 2)}
