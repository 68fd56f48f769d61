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


def test_stopping_tests_and_final_gradient():
    """gtol / ftol end the run by L-BFGS-B's own tests; the returned gradient
    is the one evaluated at the returned angles."""
    v, n, d, xhat, fun_grad, calls = _validation()
    r = lbfgsb_loop(fun_grad, v["alphas"][2], eps=-1.0, max_iter=2000, gtol=1e-7, ftol=1e-14)
    assert r["stopped"] == "gtol/ftol" and not r["converged"]
    ref = oterms.cost_grad(n, d, r["alpha"], v["b"], *_lcu(v))
    assert r["cost"] == ref["cost"] and np.array_equal(r["grad"], ref["grad"])
    assert np.abs(r["grad"]).max() <= 1e-5
    r = lbfgsb_loop(fun_grad, v["alphas"][2], eps=-1.0, max_iter=4)
    assert r["stopped"] == "max_iter" and r["iters"] == 4


def _oracle_batched():
    v, n, d, xhat, fun_grad, calls = _validation()
    coef, xs, zs = _lcu(v)
    batches = []

    def fgb(idx, alphas):
        batches.append(list(idx))
        rs = [oterms.cost_grad(n, d, np.asarray(a), v["b"], coef, xs, zs) for a in alphas]
        return [r["cost"] for r in rs], [r["grad"] for r in rs]

    return v, n, d, xhat, fgb, batches


def test_lockstep_quadratic_and_rosenbrock():
    """Problems of different sizes in one run: a separable quadratic (minimum
    at a known point) and the Rosenbrock function (minimum at (1, 1))."""
    from paper_2604_14435_gb300.lbfgs import lbfgs_lockstep

    target = np.array([0.5, -1.25, 2.0])

    def fgb(idx, alphas):
        out_f, out_g = [], []
        for k, a in zip(idx, alphas):
            if k == 0:
                out_f.append(float(np.sum((a - target) ** 2)))
                out_g.append(2.0 * (a - target))
            else:
                x, y = a
                out_f.append((1 - x) ** 2 + 100 * (y - x * x) ** 2)
                out_g.append(np.array([-2 * (1 - x) - 400 * x * (y - x * x), 200 * (y - x * x)]))
        return out_f, out_g

    r = lbfgs_lockstep(fgb, [np.zeros(3), np.array([-1.2, 1.0])], gtol=1e-9, ftol=0.0, max_iter=500, first_step=1.0)
    assert r[0]["stopped"] == "gtol" and np.allclose(r[0]["alpha"], target, atol=1e-9)
    assert r[1]["stopped"] == "gtol" and np.allclose(r[1]["alpha"], [1.0, 1.0], atol=1e-7)
    assert r[0]["iters"] < r[1]["iters"] < 200
    assert all(np.all(np.diff(x["history"]) <= 0) for x in r)  # Armijo: the cost never rises


def test_lockstep_reaches_the_solution_and_batches_rounds():
    """On the n = 3 validation system (oracle cost and gradient) every start
    converges to C ~ 0 and F >= 0.9999; each round evaluates the running
    problems together, and a problem's result does not depend on the others
    it ran with."""
    from paper_2604_14435_gb300.lbfgs import lbfgs_lockstep

    v, n, d, xhat, fgb, batches = _oracle_batched()
    starts = [np.asarray(a) for a in v["alphas"][:4]]
    res = lbfgs_lockstep(fgb, starts, gtol=1e-8, ftol=0.0, max_iter=300)
    for r in res:
        # at C ~ 1e-15 the FP64 cost is rounding noise: a run may end there on a failed line search
        assert r["stopped"] in ("gtol", "ls") and r["cost"] <= 1e-10 and np.abs(r["grad"]).max() <= 1e-7
        assert oterms.fidelity(oterms.ansatz_state(n, d, r["alpha"]), xhat) >= 0.9999
        assert r["evals"] >= r["iters"] + 1 and len(r["history"]) == r["iters"]
    assert batches[0] == [0, 1, 2, 3] and sum(len(b) for b in batches) == sum(r["evals"] for r in res)
    alone = lbfgs_lockstep(fgb, starts[2:3], gtol=1e-8, ftol=0.0, max_iter=300)[0]
    assert alone["iters"] == res[2]["iters"] and alone["stopped"] == res[2]["stopped"]
    assert np.allclose(alone["alpha"], res[2]["alpha"], atol=1e-12, rtol=0)


def test_lockstep_stopping_tests():
    """ftol ends a run on a small relative decrease; max_iter caps it; a
    stationary start (zero gradient) ends at once; evaluation errors reach
    the caller."""
    from paper_2604_14435_gb300.lbfgs import lbfgs_lockstep

    v, n, d, xhat, fgb, batches = _oracle_batched()
    a0 = np.asarray(v["alphas"][1])
    r = lbfgs_lockstep(fgb, [a0], gtol=0.0, ftol=1e-6, max_iter=1000)[0]
    assert r["stopped"] == "ftol"
    h = [fgb([0], [a0])[0][0]] + r["history"]
    assert h[-2] - h[-1] <= 1e-6 * max(abs(h[-2]), abs(h[-1]), 1.0)
    assert all(h[k] - h[k + 1] > 1e-6 * max(abs(h[k]), abs(h[k + 1]), 1.0) for k in range(len(h) - 2))
    r = lbfgs_lockstep(fgb, [a0], gtol=0.0, ftol=0.0, max_iter=3)[0]
    assert r["stopped"] == "max_iter" and r["iters"] == 3
    flat = lbfgs_lockstep(lambda idx, al: ([1.0] * len(idx), [np.zeros_like(a) for a in al]), [np.ones(4)])[0]
    assert flat["stopped"] == "gtol" and flat["iters"] == 0 and flat["evals"] == 1

    def boom(idx, alphas):
        raise RuntimeError("device failure")

    with pytest.raises(RuntimeError, match="device failure"):
        lbfgs_lockstep(boom, [np.zeros(3)])
