"""Pauli-pruning accuracy and cost sweep on the GPU (Sec. 3.2, Fig. 5).

For a real banded matrix A and a list of pruning thresholds tau, every step
that touches the system runs through the C-ABI on the device:

- the full and the pruned Pauli decompositions (Sec. 2.2, Eq. 5;
  `dvqls_pauli_decompose_banded`);
- the matrix error of the pruned matrix, by Parseval (the Pauli strings are
  orthogonal under the trace inner product):
  eps_F = ||A - A_L||_F / ||A||_F = sqrt(sum_dropped |c|^2 / sum_all |c|^2);
- the classical solutions of the full and of every pruned system for a batch
  of right-hand sides b_j (`dvqls_lcu_solve_batched`, one CTA per b_j), and
  the relative solution errors e_j(L) = ||A_L^-1 b_j - A^-1 b_j|| / ||A^-1 b_j||,
  reported as the median and the 25th / 75th percentiles (Sec. 3.2);
- the Hadamard-test circuits of one optimizer iteration of the local cost,
  2 (n + 1) L^2 (Sec. 2.4), and, on request, the measured seconds of one cost
  + gradient evaluation at each L through the C-ABI with host buffers (global
  cost of Eq. 1 and local cost of Eq. 2/4, b = |+>^n).

Only the summaries (sums of the returned coefficients, norms of solution
differences, quantiles) are formed on the host.

Command line: ``python -m paper_2604_14435_gb300.pruning`` runs the paper's
n = 10 tridiagonal Toeplitz system (diagonal 1, off-diagonals -1/3) over
tau = 0.1, 0.05, 0.03, 0.02, 0.01, 0.005 with 64 seeded Gaussian right-hand
sides and prints one JSON object.
"""
import json
import math
import time

import numpy as np

from . import dvqls as D
from . import workloads as wl

PAPER_TAUS = (0.1, 0.05, 0.03, 0.02, 0.01, 0.005)


def circuits_per_iteration(n, L):
    """Hadamard-test circuits of one local-cost optimizer iteration: (n + 1) L^2
    overlaps, each as a real and an imaginary circuit (Sec. 2.4)."""
    return 2 * (n + 1) * L * L


def _decompose(ctx, n, offsets, bands, tau, L_max):
    coef = np.zeros(2 * L_max)
    xm = np.zeros(L_max, np.uint32)
    zm = np.zeros(L_max, np.uint32)
    L, L_pre, L_post = D.dvqls_pauli_decompose_banded(ctx, n, offsets, bands, tau, L_max, coef, xm, zm)
    return {"L": L, "L_pre": L_pre, "L_post": L_post, "coef": coef[: 2 * L].copy(), "x": xm[:L].copy(),
            "z": zm[:L].copy()}


def _sum_sq(coef):
    return math.fsum(float(v) * float(v) for v in coef)


def _solve(ctx, n, dec, B, tol, max_iter):
    """Solutions of A_L x = b_j for the rows b_j of the real matrix B."""
    nrhs, N = B.shape
    b = np.zeros((nrhs, N), np.complex128)
    b.real = B
    b = np.ascontiguousarray(b).view(np.float64).reshape(-1)
    x = np.zeros(2 * nrhs * N)
    lcu = D.make_lcu(dec["L"], dec["coef"], dec["x"], dec["z"])
    iters, _ = D.dvqls_lcu_solve_batched(ctx, n, lcu, nrhs, b, tol, max_iter, x)
    return x.view(np.complex128).reshape(nrhs, N), iters


def _time_eval(ctx, n, depth, dec, precision, reps, local):
    P = n * (depth + 1)
    an = D.make_ansatz(n, depth)
    lcu = D.make_lcu(dec["L"], dec["coef"], dec["x"], dec["z"])
    alpha = wl.random_angles(P, 2026)
    b = np.ascontiguousarray(wl.plus_state(n)).view(np.float64).copy()
    cost, grad = np.zeros(1), np.zeros(P)

    def once():
        if local:
            D.dvqls_local_cost_grad(ctx, an, alpha, lcu, precision, cost, grad)
        else:
            D.dvqls_cost_grad(ctx, an, alpha, lcu, b, precision, cost, grad)

    for _ in range(3):
        once()
    t0 = time.perf_counter()
    for _ in range(reps):
        once()
    return (time.perf_counter() - t0) / reps


def pruning_sweep(ctx, n, offsets, bands, taus=PAPER_TAUS, rhs=None, tol=1e-12, max_iter=20000,
                  time_depth=None, time_reps=20, precision=None):
    """Accuracy (and optionally cost) of the pruned LCU for each tau.

    offsets, bands: the banded description of A (as for
    `dvqls_pauli_decompose_banded`).  rhs: real (count x 2^n) right-hand
    sides, or None for none.  time_depth: ansatz depth of the timed
    evaluations, or None to skip timing.  precision: of the timed global-cost
    pass (default: DVQLS_FP32_TC for L <= 64, DVQLS_FP32 above).
    Returns a dict with the full decomposition size and one row per tau."""
    bands = np.ascontiguousarray(bands, dtype=np.float64)
    probe = _decompose(ctx, n, offsets, bands, 0.0, 1)
    if probe["L_pre"] < 1:
        raise ValueError("A has no nonzero Pauli coefficient")
    full = _decompose(ctx, n, offsets, bands, 0.0, probe["L_pre"])
    total = _sum_sq(full["coef"])
    X = None
    if rhs is not None:
        X, _ = _solve(ctx, n, full, np.asarray(rhs, dtype=np.float64), tol, max_iter)
        xnorm = np.linalg.norm(X, axis=1)
    rows = []
    for tau in taus:
        dec = _decompose(ctx, n, offsets, bands, float(tau), full["L"])
        L = dec["L"]
        kept = _sum_sq(dec["coef"])
        row = {"tau": float(tau), "L": L, "frobenius_error": math.sqrt(max(total - kept, 0.0) / total),
               "circuits_per_iteration": circuits_per_iteration(n, L),
               "circuit_reduction": circuits_per_iteration(n, full["L"]) / circuits_per_iteration(n, L)}
        if X is not None:
            XL, iters = _solve(ctx, n, dec, np.asarray(rhs, dtype=np.float64), tol, max_iter)
            err = np.linalg.norm(XL - X, axis=1) / xnorm
            row.update({"solution_error_median": float(np.median(err)),
                        "solution_error_q25": float(np.percentile(err, 25)),
                        "solution_error_q75": float(np.percentile(err, 75)),
                        "cg_iterations_max": int(np.max(iters))})
        if time_depth is not None:
            prec = precision if precision is not None else (D.DVQLS_FP32_TC if L <= 64 else D.DVQLS_FP32)
            row["global_cost_grad_s"] = _time_eval(ctx, n, time_depth, dec, prec, time_reps, False)
            row["local_cost_grad_s"] = _time_eval(ctx, n, time_depth, dec, D.DVQLS_FP32, max(time_reps // 4, 2),
                                                  True)
            row["timed_precision"] = {0: "fp64", 1: "fp32", 2: "fp32_tc", 3: "fp32_wht"}[prec]
        rows.append(row)
    return {"n": n, "L_full": full["L"], "circuits_full": circuits_per_iteration(n, full["L"]), "rows": rows}


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="Pauli-pruning accuracy and cost sweep (Sec. 3.2) on the GPU")
    ap.add_argument("--n", type=int, default=10)
    ap.add_argument("--rhs", type=int, default=64, help="seeded Gaussian right-hand sides")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--depth", type=int, default=4, help="ansatz depth of the timed evaluations")
    ap.add_argument("--no-time", action="store_true")
    ap.add_argument("--device", type=int, default=0)
    args = ap.parse_args(argv)
    offsets, bands = wl.toeplitz_bands(args.n, [1.0, -1.0 / 3.0])
    ctx = D.dvqls_create(args.device)
    try:
        out = pruning_sweep(ctx, args.n, offsets, bands, rhs=wl.gaussian_rhs(1 << args.n, args.rhs, args.seed),
                            time_depth=None if args.no_time else args.depth)
    finally:
        D.dvqls_destroy(ctx)
    out["system"] = "tridiagonal Toeplitz, diagonal 1, off-diagonals -1/3"
    out["rhs"] = {"count": args.rhs, "seed": args.seed, "kind": "normalised Gaussian"}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
