"""Host logic of the pruning sweep (Sec. 3.2) on the CPU: the library calls
are replaced by oracle-backed stand-ins, so the test checks what the sweep
forms on the host (Parseval error, quantiles, circuit counts, the order of
calls) against the printed table and direct formulas."""
import json
import os

import numpy as np

from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import pruning
from paper_2604_14435_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "toeplitz_pruning_n10.json")


class FakeLib:
    """dvqls_pauli_decompose_banded and dvqls_lcu_solve_batched by the oracle
    (dense solves); same argument conventions as the binding."""

    def __init__(self):
        self.solves = 0

    def dvqls_pauli_decompose_banded(self, ctx, n, offsets, bands, tau, L_max, coef, xm, zm):
        full = odec.decompose_banded(n, offsets, bands, 0.0, 0)
        out = odec.decompose_banded(n, offsets, bands, tau, 0)
        L = min(out["L_post"], L_max)
        c = np.ascontiguousarray(out["coef"][:L].astype(np.complex128)).view(np.float64)
        coef[: 2 * L] = c
        xm[:L] = out["x"][:L]
        zm[:L] = out["z"][:L]
        return L, full["L_pre"], out["L_post"]

    def make_lcu(self, L, coef, xm, zm):
        return (L, coef.view(np.complex128)[:L].copy(), xm[:L].copy(), zm[:L].copy())

    def dvqls_lcu_solve_batched(self, ctx, n, lcu, nrhs, b, tol, max_iter, x):
        L, c, xs, zs = lcu
        M = oterms.lcu_matrix(c, xs, zs, n)
        B = b.view(np.complex128).reshape(nrhs, 1 << n)
        X = np.linalg.solve(M, B.T).T
        x.view(np.complex128).reshape(nrhs, 1 << n)[:] = X
        self.solves += 1
        return np.full(nrhs, 7, np.int32), np.zeros(nrhs)


def test_sweep_host_summaries(monkeypatch):
    g = json.load(open(GOLDEN))
    fake = FakeLib()
    for name in ("dvqls_pauli_decompose_banded", "make_lcu", "dvqls_lcu_solve_batched"):
        monkeypatch.setattr(pruning.D, name, getattr(fake, name))
    n = 8  # small enough for dense solves; the tau -> L rule of Sec. 2.4 gives min(2^n, 64) at tau = 0.01
    offsets, bands = wl.toeplitz_bands(n, [1.0, -1.0 / 3.0])
    B = wl.gaussian_rhs(1 << n, 6, seed=1)
    taus = (0.1, 0.03, 0.01)
    out = pruning.pruning_sweep(None, n, offsets, bands, taus=taus, rhs=B)
    assert fake.solves == 1 + len(taus)
    full = odec.decompose_banded(n, offsets, bands, 0.0, 0)
    assert out["L_full"] == full["L_pre"] and out["circuits_full"] == 2 * (n + 1) * full["L_pre"] ** 2
    A = wl.toeplitz_dense(n, 1.0, -1.0 / 3.0)
    X = np.linalg.solve(A, B.T).T
    for row, tau in zip(out["rows"], taus):
        dec = odec.decompose_banded(n, offsets, bands, tau, 0)
        assert row["L"] == dec["L_post"]
        assert abs(row["frobenius_error"] - odec.frobenius_error(full["all_coef"], dec["coef"])) < 1e-13
        AL = oterms.lcu_matrix(dec["coef"], dec["x"], dec["z"], n)
        err = np.linalg.norm(np.linalg.solve(AL, B.T).T - X, axis=1) / np.linalg.norm(X, axis=1)
        assert abs(row["solution_error_median"] - np.median(err)) < 1e-10
        assert abs(row["solution_error_q25"] - np.percentile(err, 25)) < 1e-10
        assert abs(row["solution_error_q75"] - np.percentile(err, 75)) < 1e-10
        assert row["circuits_per_iteration"] == odec.circuits_per_iteration(n, row["L"])
        assert row["cg_iterations_max"] == 7
    assert out["rows"][-1]["L"] == min(1 << n, 64)
    # the circuit counts of the printed table follow from the same formula
    for L, count in g["circuits_per_iteration"].items():
        assert pruning.circuits_per_iteration(10, int(L)) == count
