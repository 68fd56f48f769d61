"""Learned warm start for D-VQLS (replaces the random initialisation of
Algorithm 1, Step 3 with a prediction; random / fixed initialisation stays
the fallback, and the exact cost and the fidelity measure the result).

Every numeric step of the method runs in the CUDA library: decomposition
(dvqls_pauli_decompose_banded), classical solve (dvqls_lcu_solve), cost and
parameter-shift gradient (dvqls_cost_grad_batched, FP64 for the training
targets), Adam runs (dvqls_optimize, FP64 fidelity), network training and
inference (dvqls_ws_*).  The training targets come from the paper's
optimizer family, limited-memory BFGS (Sec. 3), carried to convergence: the
L-BFGS steps of all systems run in lock step on the host (a few hundred
flops per system and iteration, lbfgs.lbfgs_lockstep), each round one
batched FP64 device pass of all running systems, until L-BFGS-B's
projected-gradient or relative-decrease test holds.  This module
orchestrates the calls and builds the feature / target arrays.

Problem family (tridiagonal Toeplitz, Sec. 2.5.1): n in 6..10, a ~ U(2,4),
c ~ U(-1.5,-0.5) with a > 2|c|, b = |+>^n, top-64 Pauli terms, depth-4
Ry + CZ-ring ansatz (P = 5n <= 50 angles).  Features: [a/4, c/1.5,
one-hot(n - 6) (5)].  Targets: the converged angles of FP64 runs started from
the |+> initialisation (first-layer angles pi/2, the rest 0: with an even depth
the CZ rings cancel and V|0> = |+>^n) moved off its saddle (plus_start),
zero-padded to 50 with a mask.
"""
import time

import numpy as np

from . import dvqls as D
from . import lbfgs
from . import workloads as wl

DEPTH = 4
N_MIN, N_MAX = 6, 10
P_MAX = N_MAX * (DEPTH + 1)
FEATURES = 2 + (N_MAX - N_MIN + 1)
L_TERMS = 64


def features(a, c, n):
    f = np.zeros(FEATURES, dtype=np.float32)
    f[0] = a / 4.0
    f[1] = c / 1.5
    f[2 + n - N_MIN] = 1.0
    return f


def plus_init(n, d=DEPTH):
    alpha = np.zeros(n * (d + 1))
    alpha[:n] = 0.5 * np.pi
    return alpha


def plus_start(n, d=DEPTH, scale=1e-2):
    """The |+> start moved off the stationary point it is for this family:
    with J = X^(x)n, a persymmetric A (J A J = A; its Pauli terms all have an
    even number of Z / Y factors, so a pruned LCU keeps it) and b = |+>^n
    (J b = b), V(alpha)|0> = |+>^n at the |+> angles, and the derivative of
    the state along any angle is J-odd there (J Y_k J = -Y_k, J CZ-ring J =
    +-CZ-ring for n >= 3, and an even depth), so <b|A|dpsi> = <psi|A^T A|dpsi>
    = 0 and the gradient of the cost vanishes.  A fixed seeded perturbation of
    `scale` rad per angle, the same for every system of a given n (so the
    runs leave the saddle the same way), is added."""
    return plus_init(n, d) + scale * np.random.default_rng(7_000 + 100 * d + n).normal(size=n * (d + 1))


class Problem:
    """One system prepared on the GPU: LCU (host copies), b, xhat, features."""

    def __init__(self, ctx, seed, n):
        inst = wl.throughput_instance(seed, n=n, d=DEPTH, L_max=L_TERMS)
        self.seed, self.n, self.a, self.c = seed, n, inst["a"], inst["c"]
        self.P = n * (DEPTH + 1)
        coef = np.zeros(2 * L_TERMS)
        xm = np.zeros(L_TERMS, np.uint32)
        zm = np.zeros(L_TERMS, np.uint32)
        bands = np.ascontiguousarray(inst["bands"], dtype=np.float64)
        L, _, _ = D.dvqls_pauli_decompose_banded(ctx, n, inst["offsets"], bands, 0.0, L_TERMS, coef, xm, zm)
        self.L = L
        self.coef, self.xm, self.zm = coef[: 2 * L].copy(), xm[:L].copy(), zm[:L].copy()
        self.b = np.ascontiguousarray(inst["b"]).view(np.float64).copy()
        self.lcu = D.make_lcu(L, self.coef, self.xm, self.zm)
        x = np.zeros(2 << n)
        D.dvqls_lcu_solve(ctx, n, self.lcu, self.b, 1e-12, 20000, x)
        self.xhat = x
        self.feat = features(self.a, self.c, n)


def prepare(ctx, seeds_and_n):
    return [Problem(ctx, s, n) for s, n in seeds_and_n]


def optimize(ctx, problems, inits, precision=D.DVQLS_FP32, lr=0.02, max_iter=3000, target=0.9999, depth=DEPTH):
    """Adam runs of all problems in lock step; `target` is one fidelity for all
    or an array with one per problem.  Returns (results, final angles, seconds)."""
    keep = [np.ascontiguousarray(a, dtype=np.float64) for a in inits]
    sizes = [p.n * (depth + 1) for p in problems]
    if len(keep) != len(problems) or any(a.size != P for a, P in zip(keep, sizes)):
        raise ValueError("one start of n (depth + 1) angles per problem is required")
    items = [(D.make_ansatz(p.n, depth), p.lcu, a, p.b) for p, a in zip(problems, keep)]
    inst = D.make_instances(items)
    xhat = np.concatenate([p.xhat for p in problems])
    out = np.zeros(sum(sizes))
    targets = None
    if np.ndim(target) == 1:
        targets = np.ascontiguousarray(target, dtype=np.float64)
        target = 1.0
    opt = D.make_adam(lr=lr, max_iter=max_iter, target_fidelity=target, precision=precision, targets=targets)
    t0 = time.perf_counter()
    res = D.dvqls_optimize(ctx, inst, xhat, opt, out)
    secs = time.perf_counter() - t0
    alphas, off = [], 0
    for P in sizes:
        alphas.append(out[off:off + P].copy())
        off += P
    return res, alphas, secs


def fidelities(ctx, problems, alphas, depth=DEPTH):
    """F(alpha) against the classical solution (FP64, on the GPU)."""
    res, _, _ = optimize(ctx, problems, alphas, max_iter=0, target=2.0, depth=depth)
    return np.array([r.fidelity for r in res])


def converged(ctx, problems, inits, depth=DEPTH, precision=D.DVQLS_FP64, gtol=1e-5, ftol=2.2e-9, max_iter=5000):
    """L-BFGS (the paper's optimizer family) from `inits` to convergence on
    the FP64 cost and gradient, all problems in lock step: each run ends on
    L-BFGS-B's stopping tests with its default tolerances (max |grad| <= gtol,
    relative decrease <= ftol), on a failed line search at the rounding floor,
    or after max_iter iterations.  Returns (results, fidelities, seconds)."""
    specs = [(p.n, depth, p.lcu, p.b) for p in problems]
    t0 = time.perf_counter()
    res = lbfgs.solve_batched(ctx, specs, [np.asarray(a, dtype=np.float64) for a in inits], precision=precision,
                              max_iter=max_iter, gtol=gtol, ftol=ftol)
    secs = time.perf_counter() - t0
    return res, fidelities(ctx, problems, [r["alpha"] for r in res], depth), secs


def lbfgs_summary(res, F, secs):
    it = np.array([r["iters"] for r in res])
    ev = np.array([r["evals"] for r in res])
    gmax = np.array([np.abs(r["grad"]).max() for r in res])
    stops = {}
    for r in res:
        stops[r["stopped"]] = stops.get(r["stopped"], 0) + 1
    return {"runs": len(res), "seconds": secs, "iters_median": float(np.median(it)), "iters_max": int(it.max()),
            "evals_median": float(np.median(ev)), "evals_total": int(ev.sum()), "stopped": stops,
            "grad_maxnorm_median": float(np.median(gmax)), "grad_maxnorm_max": float(gmax.max()),
            "cost_median": float(np.median([r["cost"] for r in res])),
            "fidelity_median": float(np.median(F)), "fidelity_min": float(F.min()), "fidelity_max": float(F.max()),
            "reach_0.9999": int((F >= 0.9999).sum())}


def training_arrays(problems, alphas):
    X = np.stack([p.feat for p in problems]).astype(np.float32)
    Y = np.zeros((len(problems), P_MAX), np.float32)
    M = np.zeros((len(problems), P_MAX), np.float32)
    for k, (p, a) in enumerate(zip(problems, alphas)):
        Y[k, : p.P] = a
        M[k, : p.P] = 1.0
    return X, Y, M


def init_params(hidden, seed):
    """Seeded uniform(+-sqrt(6/(fan_in+fan_out))) weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((FEATURES, hidden), (hidden, hidden), (hidden, P_MAX)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def train(ctx, X, Y, M, hidden=256, steps=3000, lr=2e-3, seed=0, batch=None, log_every=0):
    ws = D.dvqls_ws_create(ctx, FEATURES, hidden, P_MAX, init_params(hidden, seed))
    rng = np.random.default_rng(seed + 1)
    losses = []
    B = len(X) if batch is None else min(batch, len(X))
    for step in range(steps):
        if B < len(X):
            idx = rng.choice(len(X), B, replace=False)
            xb, yb, mb = X[idx], Y[idx], M[idx]
        else:
            xb, yb, mb = X, Y, M
        want = log_every and (step % log_every == 0 or step == steps - 1)
        loss = D.dvqls_ws_train_step(ws, B, np.ascontiguousarray(xb), np.ascontiguousarray(yb),
                                     np.ascontiguousarray(mb), lr, want_loss=bool(want))
        if want:
            losses.append((step, loss))
    return ws, losses


def predict(ws, problems):
    X = np.stack([p.feat for p in problems]).astype(np.float32)
    out = np.zeros((len(problems), P_MAX), np.float32)
    D.dvqls_ws_infer(ws, len(problems), X, out)
    return [out[k, : p.P].astype(np.float64) for k, p in enumerate(problems)]


def summarize(res, secs, cap):
    it = np.array([r.iters if r.converged else cap for r in res])
    conv = np.array([r.converged for r in res], bool)
    return {"reached": int(conv.sum()), "count": len(res), "iters_median": float(np.median(it)),
            "iters_mean": float(it.mean()), "seconds": secs,
            "final_fidelity_median": float(np.median([r.fidelity for r in res]))}


def attainable(ctx, problems, iters):
    """Fidelity each problem reaches after `iters` Adam updates from the |+>
    start with an unreachable target."""
    res, alphas, secs = optimize(ctx, problems, [plus_init(p.n) for p in problems], max_iter=iters, target=2.0)
    return np.array([r.fidelity for r in res]), alphas, secs


def run(ctx, n_train=2000, n_eval=200, max_iter=3000, train_steps=3000, gap=1e-4, seed=0, gtol=1e-5, ftol=2.2e-9,
        lbfgs_max_iter=5000, n_deep=50, deep_depth=6, log=print):
    """The full pipeline: converged FP64 training targets, training, and the
    held-out comparison of initialisations.  Returns a summary dict.

    Training targets: the angles where FP64 L-BFGS from the (perturbed) |+>
    start converges (gtol, ftol).  Evaluation on the held-out systems, for each
    start (learned, zero, random, |+>):
    - Adam (FP32 cost pass, FP64 fidelity): iterations and wall time to reach
      F >= F_ref - gap, F_ref being the fidelity of the converged FP64
      L-BFGS run from |+> on that system, and to F >= 0.99 and 0.9999;
    - FP64 L-BFGS to convergence: iterations, evaluations, wall time and
      the fidelity it ends at.
    The |+> start is plus_start (|+> itself is a stationary point).
    A depth-`deep_depth` converged run on the first `n_deep` held-out
    systems shows what a deeper ansatz of the same family attains."""
    rng = np.random.default_rng(seed)
    train_specs = [(10_000 + k, int(rng.integers(N_MIN, N_MAX + 1))) for k in range(n_train)]
    eval_specs = [(90_000 + k, N_MAX) for k in range(n_eval)]
    conv = dict(gtol=gtol, ftol=ftol, max_iter=lbfgs_max_iter)
    t0 = time.perf_counter()
    tr = prepare(ctx, train_specs)
    ev = prepare(ctx, eval_specs)
    log("prepared %d + %d problems in %.1f s" % (len(tr), len(ev), time.perf_counter() - t0))
    res_tr, F_tr, secs = converged(ctx, tr, [plus_start(p.n) for p in tr], **conv)
    targets = lbfgs_summary(res_tr, F_tr, secs)
    log("training targets: %s" % targets)
    X, Y, M = training_arrays(tr, [r["alpha"] for r in res_tr])
    t1 = time.perf_counter()
    ws, losses = train(ctx, X, Y, M, steps=train_steps, log_every=max(1, train_steps // 10))
    train_s = time.perf_counter() - t1
    log("trained in %.1f s, loss %s" % (train_s, losses[-1] if losses else None))
    inits = {
        "mlp": predict(ws, ev),
        "zero": [np.zeros(p.P) for p in ev],
        "random": [np.random.default_rng(p.seed).uniform(-np.pi, np.pi, p.P) for p in ev],
        "plus": [plus_start(p.n) for p in ev],
    }
    D.dvqls_ws_destroy(ws)
    out = {"train": {"targets": targets, "gtol": gtol, "ftol": ftol, "train_seconds": train_s,
                     "loss_curve": losses},
           "eval": {"problems": len(ev), "n": N_MAX, "gap": gap}, "inits": {}}
    lb = {}
    for name, a0 in inits.items():
        r, F, s_ = converged(ctx, ev, a0, **conv)
        lb[name] = (r, F)
        out["inits"][name] = {"lbfgs_fp64": lbfgs_summary(r, F, s_)}
        log("eval %-6s L-BFGS %s" % (name, out["inits"][name]["lbfgs_fp64"]))
    F_ref = lb["plus"][1]
    out["eval"].update({"reference": "FP64 L-BFGS from |+> (plus_start) to convergence",
                        "reference_fidelity_median": float(np.median(F_ref)),
                        "reference_fidelity_min": float(F_ref.min()), "reference_fidelity_max": float(F_ref.max())})
    for name, a0 in inits.items():
        row = out["inits"][name]
        r, _, s_ = optimize(ctx, ev, a0, max_iter=max_iter, target=F_ref - gap)
        row["adam_to_reference"] = summarize(r, s_, max_iter)
        for level in (0.99, 0.9999):
            r, _, s_ = optimize(ctx, ev, a0, max_iter=max_iter, target=level)
            row["adam_to_%g" % level] = summarize(r, s_, max_iter)
        row["initial_fidelity_median"] = float(np.median(fidelities(ctx, ev, a0)))
        log("eval %-6s Adam %s" % (name, {k: v for k, v in row.items() if k != "lbfgs_fp64"}))
    if n_deep > 0:
        deep = ev[:n_deep]
        r, F, s_ = converged(ctx, deep, [plus_start(p.n, deep_depth) for p in deep], depth=deep_depth, **conv)
        F4 = F_ref[:n_deep]
        out["deep"] = {"depth": deep_depth, "angles": N_MAX * (deep_depth + 1), **lbfgs_summary(r, F, s_),
                       "depth4_fidelity_median_same_systems": float(np.median(F4)),
                       "improved_over_depth4": int((F > F4).sum())}
        log("depth %d: %s" % (deep_depth, out["deep"]))
    return out


def main():
    import argparse
    import json

    import torch

    ap = argparse.ArgumentParser(description="learned warm start: train and evaluate")
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--max-iter", type=int, default=3000, help="Adam updates at most in the evaluation")
    ap.add_argument("--steps", type=int, default=3000, help="network training steps")
    ap.add_argument("--gtol", type=float, default=1e-5)
    ap.add_argument("--ftol", type=float, default=2.2e-9)
    ap.add_argument("--lbfgs-max-iter", type=int, default=5000)
    ap.add_argument("--deep", type=int, default=50, help="held-out systems of the deeper-ansatz run")
    ap.add_argument("--deep-depth", type=int, default=6)
    args = ap.parse_args()
    assert torch.cuda.is_available()
    ctx = D.dvqls_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        out = run(ctx, args.train, args.eval, args.max_iter, args.steps, gtol=args.gtol, ftol=args.ftol,
                  lbfgs_max_iter=args.lbfgs_max_iter, n_deep=args.deep, deep_depth=args.deep_depth)
    finally:
        D.dvqls_destroy(ctx)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
