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


def lbfgsb_loop(fun_grad, alpha0, eps=1e-10, max_iter=1000, bounds=(-2.0 * np.pi, 2.0 * np.pi), maxcor=10,
                gtol=0.0, ftol=0.0):
    """Minimise C(alpha) with L-BFGS-B until C <= eps (Algorithm 1).

    fun_grad(alpha) -> (C, dC/dalpha) for a float64 array alpha.  bounds: one
    (low, high) pair for every angle, or None.  gtol, ftol: L-BFGS-B's own
    stopping tests (projected-gradient max-norm <= gtol; relative decrease
    (C_k - C_k+1) / max(|C_k|, |C_k+1|, 1) <= ftol), off at 0.  Returns a
    dict: alpha, cost, grad (the gradient at alpha), iters (L-BFGS-B
    iterations), evals (cost + gradient evaluations), converged (C <= eps
    reached), stopped ("eps", "gtol/ftol" when L-BFGS-B's own test ended it,
    "max_iter" or "other"), history (cost after each iteration)."""
    from scipy.optimize import minimize
    alpha0 = np.array(alpha0, dtype=np.float64)
    P = alpha0.size
    state = {"evals": 0, "last": None, "best": (np.inf, alpha0.copy(), None)}
    history = []

    def f(a):
        a = np.array(a, dtype=np.float64)
        c, g = fun_grad(a)
        c = float(c)
        g = np.array(g, dtype=np.float64)
        state["evals"] += 1
        state["last"] = (a, c, g)
        if c < state["best"][0]:
            state["best"] = (c, a.copy(), g.copy())
        return c, g

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

    stopped = "eps"
    try:
        res = minimize(f, alpha0, jac=True, method="L-BFGS-B", callback=callback,
                       bounds=None if bounds is None else [tuple(bounds)] * P,
                       options={"maxiter": int(max_iter), "maxcor": int(maxcor), "ftol": float(ftol),
                                "gtol": float(gtol)})
        cost_at(np.array(res.x, dtype=np.float64))
        stopped = "max_iter" if len(history) >= max_iter else "gtol/ftol" if res.success else "other"
    except _Reached:
        pass
    alpha, cost, grad = state["last"]  # the point the loop ended on (cost_at evaluated it if needed)
    if state["best"][0] < cost:  # a line search may end above the best point it evaluated
        cost, alpha, grad = state["best"]
    return {"alpha": alpha, "cost": cost, "grad": grad, "iters": len(history), "evals": state["evals"],
            "converged": bool(cost <= eps), "stopped": stopped, "history": history}


def lbfgs_lockstep(fun_grad_batched, alpha0s, m=10, gtol=1e-5, ftol=2.2e-9, max_iter=5000, max_ls=30, c1=1e-4,
                   first_step=0.1):
    """Limited-memory BFGS for many problems in lock step (no bounds: the
    cost is 2 pi-periodic in every angle), each round one batched evaluation
    of all the problems still running.

    fun_grad_batched(indices, alphas) -> (costs, grads) evaluates the listed
    problems at the given points.  Per problem: the direction from the
    two-loop recursion over the last m pairs (s, y) (a pair is kept when
    s.y > 1e-10 |s| |y|; the initial matrix is (s.y / y.y) I, and the first
    step is scaled so that no angle moves by more than `first_step`), a
    backtracking line search to the Armijo condition C(a + t d) <= C(a) +
    c1 t g.d (t = 1, 1/2, ...; the history is cleared and d = -g when d is no
    descent direction), and the stopping tests of L-BFGS-B: max |g| <= gtol
    ("gtol"), relative decrease (C_k - C_k+1) / max(|C_k|, |C_k+1|, 1) <=
    ftol ("ftol"), no Armijo point after max_ls halvings ("ls"), or max_iter
    iterations ("max_iter").  The defaults are L-BFGS-B's (pgtol 1e-5, factr
    1e7).  Returns one dict per problem: alpha, cost, grad, iters, evals,
    stopped, history (cost after each iteration)."""
    K = len(alpha0s)
    sizes = np.array([np.asarray(a).size for a in alpha0s])
    PM = int(sizes.max()) if K else 0
    X = np.zeros((K, PM))
    for k, a in enumerate(alpha0s):
        X[k, :sizes[k]] = np.asarray(a, dtype=np.float64)
    G = np.zeros((K, PM))
    F = np.zeros(K)
    S = np.zeros((K, m, PM))
    Y = np.zeros((K, m, PM))
    RHO = np.zeros((K, m))
    iters = np.zeros(K, int)
    evals = np.zeros(K, int)
    stopped = [None] * K
    hist = [[] for _ in range(K)]

    def evaluate(idx, pts):
        costs, grads = fun_grad_batched([int(k) for k in idx], [pts[j, :sizes[k]].copy() for j, k in enumerate(idx)])
        g = np.zeros((len(idx), PM))
        for j, k in enumerate(idx):
            g[j, :sizes[k]] = np.asarray(grads[j], dtype=np.float64)
        evals[idx] += 1
        return np.asarray(costs, dtype=np.float64), g

    allk = np.arange(K)
    if K:
        F[:], G[:] = evaluate(allk, X)
    active = np.ones(K, bool)
    for k in allk[np.abs(G).max(axis=1) <= gtol] if K else []:
        stopped[k] = "gtol"
        active[k] = False
    if max_iter <= 0:
        for k in allk[active]:
            stopped[k] = "max_iter"
        active[:] = False
    while active.any():
        idx = allk[active]
        g = G[idx]
        # two-loop recursion (empty history slots have rho = 0 and drop out)
        q = g.copy()
        a = np.zeros((idx.size, m))
        for i in range(m - 1, -1, -1):
            a[:, i] = RHO[idx, i] * np.einsum("kp,kp->k", S[idx, i], q)
            q -= a[:, i, None] * Y[idx, i]
        sy = np.einsum("kp,kp->k", S[idx, m - 1], Y[idx, m - 1])
        yy = np.einsum("kp,kp->k", Y[idx, m - 1], Y[idx, m - 1])
        has = RHO[idx, m - 1] > 0
        gamma = np.where(has, sy / np.where(yy > 0, yy, 1.0), 1.0)
        r = gamma[:, None] * q
        for i in range(m):
            bta = RHO[idx, i] * np.einsum("kp,kp->k", Y[idx, i], r)
            r += S[idx, i] * (a[:, i] - bta)[:, None]
        d = -r
        gd = np.einsum("kp,kp->k", g, d)
        bad = ~(gd < 0)
        if bad.any():  # not a descent direction: restart from steepest descent
            RHO[idx[bad]] = 0.0
            d[bad] = -g[bad]
            gd[bad] = -np.einsum("kp,kp->k", g[bad], g[bad])
            has[bad] = False
        dmax = np.abs(d).max(axis=1)
        t = np.where(has, 1.0, np.minimum(1.0, first_step / np.where(dmax > 0, dmax, 1.0)))
        todo = np.arange(idx.size)
        newF = np.zeros(idx.size)
        newG = np.zeros((idx.size, PM))
        ok = np.zeros(idx.size, bool)
        for _ in range(max_ls + 1):
            if todo.size == 0:
                break
            pts = X[idx[todo]] + t[todo, None] * d[todo]
            fc, gc = evaluate(idx[todo], pts)
            acc = fc <= F[idx[todo]] + c1 * t[todo] * gd[todo]
            newF[todo[acc]] = fc[acc]
            newG[todo[acc]] = gc[acc]
            ok[todo[acc]] = True
            todo = todo[~acc]
            t[todo] *= 0.5
        for j in np.flatnonzero(~ok):
            k = idx[j]
            stopped[k] = "ls"
            active[k] = False
        j = np.flatnonzero(ok)
        k = idx[j]
        s_ = t[j, None] * d[j]
        y_ = newG[j] - G[k]
        f_old = F[k].copy()
        X[k] += s_
        F[k] = newF[j]
        G[k] = newG[j]
        iters[k] += 1
        for kk, c in zip(k, F[k]):
            hist[kk].append(float(c))
        syv = np.einsum("kp,kp->k", s_, y_)
        keep = syv > 1e-10 * np.linalg.norm(s_, axis=1) * np.linalg.norm(y_, axis=1)
        kp = k[keep]
        S[kp, :-1] = S[kp, 1:]
        Y[kp, :-1] = Y[kp, 1:]
        RHO[kp, :-1] = RHO[kp, 1:]
        S[kp, -1] = s_[keep]
        Y[kp, -1] = y_[keep]
        RHO[kp, -1] = 1.0 / syv[keep]
        for kk, fo in zip(k, f_old):
            if np.abs(G[kk]).max() <= gtol:
                stopped[kk] = "gtol"
            elif fo - F[kk] <= ftol * max(abs(fo), abs(F[kk]), 1.0):
                stopped[kk] = "ftol"
            elif iters[kk] >= max_iter:
                stopped[kk] = "max_iter"
            if stopped[kk] is not None:
                active[kk] = False
    return [{"alpha": X[k, :sizes[k]].copy(), "cost": float(F[k]), "grad": G[k, :sizes[k]].copy(),
             "iters": int(iters[k]), "evals": int(evals[k]), "stopped": stopped[k], "history": hist[k]}
            for k in range(K)]


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


def solve_batched(ctx, specs, alpha0s, precision=D.DVQLS_FP64, **kw):
    """Many systems at once: lbfgs_lockstep over `dvqls_cost_grad_batched`
    (global cost), one batched device pass per round of all running systems.
    specs: one (n, depth, lcu, b) per system, as for `solve` (arrays kept
    alive by the caller).  Returns the list of `lbfgs_lockstep` results."""
    ans = [D.make_ansatz(n, depth) for n, depth, _, _ in specs]
    if len(alpha0s) != len(specs) or any(np.asarray(a).size != n * (depth + 1)
                                         for a, (n, depth, _, _) in zip(alpha0s, specs)):
        raise ValueError("one start of n (depth + 1) angles per system is required")

    def fgb(idx, alphas):
        keep = [np.ascontiguousarray(a, dtype=np.float64) for a in alphas]
        inst = D.make_instances([(ans[k], specs[k][2], a, specs[k][3]) for k, a in zip(idx, keep)])
        costs = np.zeros(len(idx))
        grads = np.zeros(sum(a.size for a in keep))
        D.dvqls_cost_grad_batched(ctx, inst, precision, costs, grads)
        out, off = [], 0
        for a in keep:
            out.append(grads[off:off + a.size])
            off += a.size
        return costs, out

    return lbfgs_lockstep(fgb, alpha0s, **kw)
