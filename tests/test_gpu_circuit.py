"""Per-circuit FP64 GPU path vs the oracle (1e-12): every Hadamard-test
circuit simulated gate by gate on n+1 qubits, real and imaginary parts from
separate circuits."""
import numpy as np
import pytest
import torch

from oracle import circuit as ocirc
from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = 1e-12


def run(dv, ctx, n, d, alpha, b, coef, xs, zs):
    L = len(xs)
    c_ = np.ascontiguousarray(np.asarray(coef, np.complex128)).view(np.float64)
    x_ = np.ascontiguousarray(xs, np.uint32)
    z_ = np.ascontiguousarray(zs, np.uint32)
    b_ = np.ascontiguousarray(np.asarray(b, np.complex128)).view(np.float64)
    cost, grad = np.zeros(1), np.zeros(n * (d + 1))
    beta, delta = np.zeros(2 * L * L), np.zeros(2 * L)
    dv.dvqls_circuit_cost_grad_fp64(ctx, dv.make_ansatz(n, d), np.ascontiguousarray(alpha, np.float64),
                                    dv.make_lcu(L, c_, x_, z_), b_, cost, grad, beta, delta)
    return cost[0], grad, beta.view(np.complex128).reshape(L, L), delta.view(np.complex128)


def close(a, b):
    return np.all(np.abs(np.asarray(a) - np.asarray(b)) <= TOL * np.maximum(1.0, np.abs(b)))


@pytest.mark.parametrize("n,d,L", [(1, 1, 2), (2, 2, 4), (3, 2, 8), (5, 1, 6), (7, 2, 5)])
@pytest.mark.parametrize("bkind", ["plus", "complex"])
def test_circuits_match_oracles(dv, ctx, n, d, L, bkind):
    rng = np.random.default_rng(60 + n + L)
    N = 1 << n
    xs = rng.integers(0, N, L).astype(np.uint32)
    zs = rng.integers(0, N, L).astype(np.uint32)
    coef = rng.normal(size=L) + 1j * rng.normal(size=L)
    b = wl.plus_state(n) if bkind == "plus" else rng.normal(size=N) + 1j * rng.normal(size=N)
    alpha = wl.random_angles(n * (d + 1), 7 + n)
    cost, grad, beta, delta = run(dv, ctx, n, d, alpha, b, coef, xs, zs)
    bn = b / np.linalg.norm(b)
    cb, cd, _ = ocirc.circuit_terms(n, d, alpha, bn, xs, zs)
    assert close(beta, cb) and close(delta, cd)
    ref = oterms.cost_grad(n, d, alpha, bn, coef, xs, zs)
    assert close(cost, ref["cost"]) and close(grad, ref["grad"])


def test_circuits_full_size_throughput_system(dv, ctx):
    """n = 10, L = 64: 840,320 circuits; cost, gradient and terms at 1e-12."""
    inst = wl.throughput_instance(3)
    n, d = inst["n"], inst["d"]
    dec = odec.decompose_banded(n, inst["offsets"], inst["bands"], 0.0, 64)
    cost, grad, beta, delta = run(dv, ctx, n, d, inst["alpha"], inst["b"], dec["coef"], dec["x"], dec["z"])
    ref = oterms.cost_grad(n, d, inst["alpha"], inst["b"], dec["coef"], dec["x"], dec["z"])
    assert close(cost, ref["cost"]) and close(grad, ref["grad"])
    assert close(beta, ref["beta"]) and close(delta, ref["delta"])


def test_circuit_path_rejects_too_many_qubits(dv, ctx):
    with pytest.raises(dv.DvqlsError) as e:
        run(dv, ctx, 13, 1, np.zeros(26), wl.plus_state(13), [1.0], [0], [0])
    assert e.value.code == dv.DVQLS_ERR_UNSUPPORTED
