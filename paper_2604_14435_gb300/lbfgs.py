"""L-BFGS-B host loop of Algorithm 1 around the GPU cost and gradient.

The paper drives the angles with SciPy's L-BFGS-B (Sec. 3) while the cost is
above the tolerance epsilon (Algorithm 1, the while loop over Steps 4a-4c).
Here SciPy holds the optimizer state on the host and every function value
and gradient comes from one `dvqls_cost_grad` (global cost, Eq. 1) or
`dvqls_local_cost_grad` (local cost, Eq. 2/4, b = |+>^n) call: the
parameter-shift gradient of all P angles in one device pass.

The paper states neither the gradient method nor the bounds: the gradient is
the exact parameter-shift one, and the default box is [-2 pi, 2 pi] per
angle (the cost is 2 pi-periodic in each angle, so the box holds a copy of
every minimum away from its faces).  The loop stops after the first
iteration whose cost is <= eps, when L-BFGS-B itself converges, or after
max_iter iterations.
"""
import numpy as np

from . import dvqls as D


class _Reached(Exception):
    pass


def lbfgsb_loop(fun_grad, alpha0, eps=1e-10, max_iter=1000, bounds=(-2.0 * np.pi, 2.0 * np.pi), maxcor=10):
    """Minimise C(alpha) with L-BFGS-B until C <= eps (Algorithm 1).

    fun_grad(alpha) -> (C, dC/dalpha) for a float64 array alpha.  bounds: one
    (low, high) pair for every angle, or None.  Returns a dict: alpha, cost,
    iters (L-BFGS-B iterations), evals (cost + gradient evaluations),
    converged (C <= eps reached), history (cost after each iteration)."""
    from scipy.optimize import minimize
    alpha0 = np.array(alpha0, dtype=np.float64)
    P = alpha0.size
    state = {"evals": 0, "last": None, "best": (np.inf, alpha0.copy())}
    history = []

    def f(a):
        a = np.array(a, dtype=np.float64)
        c, g = fun_grad(a)
        c = float(c)
        state["evals"] += 1
        state["last"] = (a, c)
        if c < state["best"][0]:
            state["best"] = (c, a.copy())
        return c, np.array(g, dtype=np.float64)

    def cost_at(xk):
        last = state["last"]
        if last is not None and np.array_equal(last[0], xk):
            return last[1]
        return f(xk)[0]

    def callback(xk):
        c = cost_at(np.asarray(xk, dtype=np.float64))
        history.append(c)
        if c <= eps:
            raise _Reached

    try:
        res = minimize(f, alpha0, jac=True, method="L-BFGS-B", callback=callback,
                       bounds=None if bounds is None else [tuple(bounds)] * P,
                       options={"maxiter": int(max_iter), "maxcor": int(maxcor), "ftol": 0.0, "gtol": 0.0})
        alpha = np.array(res.x, dtype=np.float64)
        cost = cost_at(alpha)
    except _Reached:
        cost, alpha = state["last"][1], state["last"][0]
    if state["best"][0] < cost:  # a line search may end above the best point it evaluated
        cost, alpha = state["best"]
    return {"alpha": alpha, "cost": cost, "iters": len(history), "evals": state["evals"],
            "converged": bool(cost <= eps), "history": history}


def solve(ctx, n, depth, lcu, b, alpha0, precision=D.DVQLS_FP64, eps=1e-10, max_iter=1000, local=False,
          bounds=(-2.0 * np.pi, 2.0 * np.pi)):
    """Algorithm 1's loop on the GPU: L-BFGS-B over `dvqls_cost_grad` (or
    `dvqls_local_cost_grad` with local=True; b is then |+>^n and ignored).
    lcu: a dvqls_lcu (its arrays kept alive by the caller); b: 2^n complex128
    as 2^(n+1) float64.  Returns the dict of `lbfgsb_loop`."""
    an = D.make_ansatz(n, depth)
    P = n * (depth + 1)
    cost = np.zeros(1)
    grad = np.zeros(P)

    def fun_grad(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if local:
            D.dvqls_local_cost_grad(ctx, an, a, lcu, precision, cost, grad)
        else:
            D.dvqls_cost_grad(ctx, an, a, lcu, b, precision, cost, grad)
        return float(cost[0]), grad.copy()

    return lbfgsb_loop(fun_grad, alpha0, eps=eps, max_iter=max_iter, bounds=bounds)
