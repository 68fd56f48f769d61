"""L-BFGS-B host loop (Algorithm 1 with the paper's optimizer, Sec. 3) driven
by the oracle's cost and gradient on the CPU: the loop logic (stop at the
first iteration with C <= eps, bounds, iteration cap, best point kept)."""
import numpy as np
import pytest

pytest.importorskip("scipy")

from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl
from paper_2604_14435_gb300.lbfgs import lbfgsb_loop


def _validation():
    v = wl.validation_system()
    n, d = v["n"], v["d"]
    dec = odec.decompose(v["A"], tau=0.0, L_max=v["L_max"])
    coef, xs, zs = dec["coef"], dec["x"], dec["z"]
    xhat = oterms.classical_solution(oterms.lcu_matrix(coef, xs, zs, n), v["b"])
    calls = []

    def fun_grad(a):
        calls.append(np.array(a))
        r = oterms.cost_grad(n, d, a, v["b"], coef, xs, zs)
        return r["cost"], r["grad"]

    return v, n, d, xhat, fun_grad, calls


@pytest.mark.parametrize("start", [0, 3])
def test_reaches_eps_and_the_classical_solution(start):
    v, n, d, xhat, fun_grad, calls = _validation()
    r = lbfgsb_loop(fun_grad, v["alphas"][start], eps=1e-10, max_iter=500)
    assert r["converged"] and r["cost"] <= 1e-10
    assert r["history"][-1] <= 1e-10 and all(c > 1e-10 for c in r["history"][:-1])  # stops at the first
    assert r["evals"] == len(calls)
    assert oterms.fidelity(oterms.ansatz_state(n, d, r["alpha"]), xhat) >= 0.9999
    # the returned cost is the oracle's cost at the returned angles
    assert abs(oterms.cost_grad(n, d, r["alpha"], v["b"], *_lcu(v))["cost"] - r["cost"]) < 1e-15


def _lcu(v):
    dec = odec.decompose(v["A"], tau=0.0, L_max=v["L_max"])
    return dec["coef"], dec["x"], dec["z"]


def test_iteration_cap_and_bounds():
    v, n, d, xhat, fun_grad, calls = _validation()
    r = lbfgsb_loop(fun_grad, v["alphas"][1], eps=1e-14, max_iter=3, bounds=(-1.0, 1.0))
    assert not r["converged"] and r["iters"] <= 3
    assert np.all(np.abs(r["alpha"]) <= 1.0)
    assert all(np.all(np.abs(a) <= 1.0 + 1e-12) for a in calls[1:])  # every evaluated point inside the box
    assert r["cost"] == min(oterms.cost_grad(n, d, a, v["b"], *_lcu(v))["cost"] for a in calls)


def test_quadratic_closed_form():
    """A separable quadratic with its minimum at a known point inside the box."""
    target = np.array([0.5, -1.25, 2.0])

    def fg(a):
        return float(np.sum((a - target) ** 2)), 2.0 * (a - target)

    r = lbfgsb_loop(fg, np.zeros(3), eps=1e-20, max_iter=100)
    assert np.allclose(r["alpha"], target, atol=1e-9)
    r = lbfgsb_loop(fg, np.zeros(3), eps=1e-20, max_iter=100, bounds=(-1.0, 1.0))
    assert np.allclose(r["alpha"], np.clip(target, -1.0, 1.0), atol=1e-9)


def test_solve_routes_to_the_library_calls(monkeypatch):
    """lbfgs.solve evaluates through dvqls_cost_grad (global) or
    dvqls_local_cost_grad (local) with the given precision; stand-ins driven
    by the oracle take the place of the library here."""
    from paper_2604_14435_gb300 import dvqls as D
    from paper_2604_14435_gb300 import lbfgs

    v, n, d, xhat, fun_grad, calls = _validation()
    coef, xs, zs = _lcu(v)
    seen = []

    def fake_global(ctx, an, a, lcu, b, prec, cost, grad, beta=None, delta=None):
        seen.append(("global", prec, an.n, an.depth))
        r = oterms.cost_grad(n, d, np.asarray(a), v["b"], coef, xs, zs)
        cost[0], grad[:] = r["cost"], r["grad"]

    def fake_local(ctx, an, a, lcu, prec, cost, grad=None):
        seen.append(("local", prec, an.n, an.depth))
        r = oterms.local_cost_grad(n, d, np.asarray(a), coef, xs, zs)
        cost[0], grad[:] = r["cost"], r["grad"]

    monkeypatch.setattr(D, "dvqls_cost_grad", fake_global)
    monkeypatch.setattr(D, "dvqls_local_cost_grad", fake_local)
    r = lbfgs.solve(None, n, d, None, None, v["alphas"][0], precision=D.DVQLS_FP64, eps=1e-10, max_iter=200)
    assert r["converged"] and {s[0] for s in seen} == {"global"} and {s[1:] for s in seen} == {(0, n, d)}
    seen.clear()
    r = lbfgs.solve(None, n, d, None, None, v["alphas"][0], precision=D.DVQLS_FP32, eps=1e-10, max_iter=200,
                    local=True)
    assert r["converged"] and {s[0] for s in seen} == {"local"} and {s[1] for s in seen} == {1}
    assert oterms.local_cost_grad(n, d, r["alpha"], coef, xs, zs)["cost"] <= 1e-10
