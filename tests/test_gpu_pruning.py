"""Pruning sweep of Sec. 3.2 on the GPU (decompositions, matrix error, batched
classical solves) against the paper's printed table and dense solves of the
oracle's matrices; the batched multi-right-hand-side solve; the L-BFGS-B loop
of Algorithm 1 over the GPU cost and gradient."""
import json
import os

import numpy as np
import pytest

from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "toeplitz_pruning_n10.json")


@pytest.mark.parametrize("shift", [2.0, 0.5])
def test_batched_solve_equals_single_solves(dv, ctx, shift):
    """One CTA per right-hand side runs the single-solve arithmetic: bit-exact.
    A~ = shift I + Z_0 + 0.3 X_1 is positive definite at shift 2 and
    indefinite at 0.5 (CG breaks down and the normal equations take over)."""
    rng = np.random.default_rng(5)
    n, N, nrhs = 4, 16, 3
    coef = np.array([shift, 1.0, 0.3], np.complex128)
    xs = np.array([0, 0, 2], np.uint32)
    zs = np.array([0, 1, 0], np.uint32)
    cpk = np.ascontiguousarray(coef).view(np.float64)
    lcu = dv.make_lcu(len(coef), cpk, xs, zs)
    B = rng.normal(size=(nrhs, N)) + 1j * rng.normal(size=(nrhs, N))
    bp = np.ascontiguousarray(B).view(np.float64).reshape(-1)
    x = np.zeros(2 * nrhs * N)
    it, rr = dv.dvqls_lcu_solve_batched(ctx, n, lcu, nrhs, bp, 1e-13, 20000, x)
    X = x.view(np.complex128).reshape(nrhs, N)
    M = oterms.lcu_matrix(coef, xs, zs, n)
    for k in range(nrhs):
        xk = np.zeros(2 * N)
        itk, rrk = dv.dvqls_lcu_solve(ctx, n, lcu, np.ascontiguousarray(B[k]).view(np.float64), 1e-13, 20000, xk)
        assert np.array_equal(xk, x.reshape(nrhs, 2 * N)[k]) and itk == it[k] and rrk == rr[k]
        ref = np.linalg.solve(M, B[k])
        assert np.linalg.norm(X[k] - ref) <= 1e-10 * np.linalg.norm(ref)


def test_paper_pruning_sweep(dv, ctx):
    """tau -> L and eps_F as printed (Sec. 3.2); solution errors equal those of
    dense solves of the oracle's pruned and full matrices."""
    from paper_2604_14435_gb300.pruning import pruning_sweep
    g = json.load(open(GOLDEN))
    n = 10
    offsets, bands = wl.toeplitz_bands(n, [1.0, -1.0 / 3.0])
    B = wl.gaussian_rhs(1 << n, 8, seed=0)
    out = pruning_sweep(ctx, n, offsets, bands, taus=g["tau"], rhs=B)
    assert out["L_full"] == 1 << n and out["circuits_full"] == g["circuits_per_iteration"]["1024"]
    A = wl.toeplitz_dense(n, 1.0, -1.0 / 3.0)
    X = np.linalg.solve(A, B.T)
    for row, tau, L in zip(out["rows"], g["tau"], g["L"]):
        assert row["tau"] == tau and row["L"] == L
        if str(L) in g["frobenius_error_percent"]:
            assert round(100.0 * row["frobenius_error"], g["frobenius_error_decimals"]) == \
                g["frobenius_error_percent"][str(L)]
            assert row["circuits_per_iteration"] == g["circuits_per_iteration"][str(L)]
        dec = odec.decompose_banded(n, offsets, bands, tau, 0)
        AL = oterms.lcu_matrix(dec["coef"], dec["x"], dec["z"], n)
        err = np.linalg.norm(np.linalg.solve(AL, B.T) - X, axis=0) / np.linalg.norm(X, axis=0)
        assert abs(row["solution_error_median"] - np.median(err)) <= 1e-8 * np.median(err)
        assert abs(row["solution_error_q25"] - np.percentile(err, 25)) <= 1e-8 * np.median(err)
        assert abs(row["solution_error_q75"] - np.percentile(err, 75)) <= 1e-8 * np.median(err)
    assert out["rows"][4]["circuit_reduction"] == g["circuit_reduction_at_L64"]


@pytest.mark.parametrize("prec,local,eps,fid", [(0, False, 1e-10, 0.9999), (1, False, 1e-6, 0.999),
                                                (0, True, 1e-10, 0.9999)])
def test_lbfgsb_on_the_gpu(dv, ctx, prec, local, eps, fid):
    pytest.importorskip("scipy")
    from paper_2604_14435_gb300.lbfgs import solve
    v = wl.validation_system()
    n, d = v["n"], v["d"]
    dec = odec.decompose(v["A"], tau=0.0, L_max=v["L_max"])
    coef, xs, zs = dec["coef"], dec["x"], dec["z"]
    cpk = np.ascontiguousarray(coef.astype(np.complex128)).view(np.float64)
    xm, zm = np.ascontiguousarray(xs, np.uint32), np.ascontiguousarray(zs, np.uint32)
    lcu = dv.make_lcu(len(coef), cpk, xm, zm)
    b = np.ascontiguousarray(v["b"].astype(np.complex128)).view(np.float64)
    r = solve(ctx, n, d, lcu, b, v["alphas"][2], precision=prec, eps=eps, max_iter=500, local=local)
    assert r["converged"]
    xhat = oterms.classical_solution(oterms.lcu_matrix(coef, xs, zs, n), v["b"])
    assert oterms.fidelity(oterms.ansatz_state(n, d, r["alpha"]), xhat) >= fid
    if local:
        ref = oterms.local_cost_grad(n, d, r["alpha"], coef, xs, zs)["cost"]
    else:
        ref = oterms.cost_grad(n, d, r["alpha"], v["b"], coef, xs, zs)["cost"]
    # In FP32 the loop minimises the rounded cost, so it ends where the rounding
    # error is most negative: a few times the 1e-6 of a random point.
    assert abs(ref - r["cost"]) <= (1e-12 if prec == 0 else 5e-6)
