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
