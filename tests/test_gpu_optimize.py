"""Fidelity (Sec. 3.1), the classical solve it is measured against, and the
Adam optimizer loop (Algorithm 1) vs the oracle."""
import numpy as np
import pytest
import torch

from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def cv(a):
    return np.ascontiguousarray(np.asarray(a, np.complex128)).view(np.float64)


def lcu_of(dv, coef, xs, zs):
    keep = (cv(coef), np.ascontiguousarray(xs, np.uint32), np.ascontiguousarray(zs, np.uint32))
    return dv.make_lcu(len(xs), *keep), keep


@pytest.mark.parametrize("n,d", [(1, 0), (3, 2), (6, 3), (10, 4), (12, 1)])
def test_fidelity_matches_oracle(dv, ctx, n, d):
    rng = np.random.default_rng(n)
    alpha = wl.random_angles(n * (d + 1), 3 + n)
    xhat = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    F = np.zeros(1)
    dv.dvqls_fidelity(ctx, dv.make_ansatz(n, d), alpha, cv(xhat), F)
    ref = oterms.fidelity(oterms.ansatz_state(n, d, alpha), xhat / np.linalg.norm(xhat))
    assert abs(F[0] - ref) <= 1e-12


@pytest.mark.parametrize("n,d", [(13, 1), (16, 2), (20, 3)])
def test_fidelity_states_in_hbm(dv, ctx, n, d):
    """n > 12: the FP64 state is built in HBM; xhat near psi keeps F of order one."""
    rng = np.random.default_rng(70 + n)
    alpha = wl.random_angles(n * (d + 1), 71 + n)
    psi = oterms.ansatz_state(n, d, alpha)
    noise = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    xhat = psi + 0.7 * noise / np.linalg.norm(noise)
    F = np.zeros(1)
    dv.dvqls_fidelity(ctx, dv.make_ansatz(n, d), alpha, cv(xhat), F)
    ref = oterms.fidelity(psi, xhat / np.linalg.norm(xhat))
    assert 0.3 < ref < 0.9
    assert abs(F[0] - ref) <= 1e-12


def test_fidelity_of_planted_state_is_one(dv, ctx):
    n, d = 5, 2
    alpha = wl.random_angles(n * (d + 1), 1)
    psi = oterms.ansatz_state(n, d, alpha)
    F = np.zeros(1)
    dv.dvqls_fidelity(ctx, dv.make_ansatz(n, d), alpha, cv(3.0 * psi), F)
    assert abs(F[0] - 1.0) <= 1e-13


@pytest.mark.parametrize("case", ["validation", "toeplitz10", "indefinite"])
def test_lcu_solve_matches_dense_solve(dv, ctx, case):
    if case == "validation":
        s = wl.validation_system()
        n, b = s["n"], s["b"]
        dec = odec.decompose(s["A"], 0.0, 64)
    elif case == "toeplitz10":
        inst = wl.throughput_instance(2)
        n, b = inst["n"], inst["b"]
        dec = odec.decompose_banded(n, inst["offsets"], inst["bands"], 0.0, 64)
    else:  # Hermitian, indefinite: 0.5 I + Z_0 + 0.3 X_1
        n = 4
        dec = {"coef": np.array([0.5, 1.0, 0.3]), "x": np.array([0, 0, 2], np.uint32), "z": np.array([0, 1, 0], np.uint32)}
        b = np.random.default_rng(0).normal(size=16) + 0j
    lcu, keep = lcu_of(dv, dec["coef"], dec["x"], dec["z"])
    x = np.zeros(2 << n)
    it, rr = dv.dvqls_lcu_solve(ctx, n, lcu, cv(b), 1e-13, 20000, x)
    x = x.view(np.complex128)
    M = oterms.lcu_matrix(dec["coef"], dec["x"], dec["z"], n)
    ref = np.linalg.solve(M, b)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    assert rr <= 1e-13


def adam_reference(n, d, alpha0, b, coef, xs, zs, xhat, lr, max_iter, target):
    """Adam driven by the oracle's exact gradient (same order of operations
    as the optimizer's contract: evaluate, stop on F, else update)."""
    a = np.array(alpha0, dtype=np.float64)
    m = np.zeros_like(a)
    v = np.zeros_like(a)
    b1, b2, eps = 0.9, 0.999, 1e-8
    c1 = c2 = 1.0
    for it in range(max_iter + 1):
        F = oterms.fidelity(oterms.ansatz_state(n, d, a), xhat)
        r = oterms.cost_grad(n, d, a, b, coef, xs, zs)
        if F >= target or it == max_iter:
            return it, a, F, r["cost"], F >= target
        g = r["grad"]
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        c1 *= b1
        c2 *= b2
        a = a - lr * (m / (1 - c1)) / (np.sqrt(v / (1 - c2)) + eps)


def test_validation_system_adam_run_reaches_target(dv, ctx):
    """n = 3 Toeplitz, full decomposition, one Adam run from seed 0 to
    F >= 0.9999 against the classical solve (Sec. 3.1)."""
    s = wl.validation_system()
    n, d, b = s["n"], s["d"], s["b"]
    dec = odec.decompose(s["A"], 0.0, 64)
    xhat = oterms.classical_solution(oterms.lcu_matrix(dec["coef"], dec["x"], dec["z"], n), b)
    alpha0 = wl.random_angles(n * (d + 1), 0)
    lcu, keep = lcu_of(dv, dec["coef"], dec["x"], dec["z"])
    inst = dv.make_instances([(dv.make_ansatz(n, d), lcu, alpha0, cv(b))])
    out = np.zeros(alpha0.size)
    opt = dv.make_adam(lr=0.02, max_iter=3000, target_fidelity=0.9999, precision=dv.DVQLS_FP64)
    res = dv.dvqls_optimize(ctx, inst, cv(xhat), opt, out)[0]
    it, a_ref, F_ref, C_ref, conv = adam_reference(n, d, alpha0, b, dec["coef"], dec["x"], dec["z"], xhat, 0.02, 3000,
                                                   0.9999)
    assert conv and res.converged == 1
    assert res.fidelity >= 0.9999
    assert abs(res.iters - it) <= 1
    if res.iters == it:
        assert np.abs(out - a_ref).max() <= 1e-8
    assert abs(oterms.fidelity(oterms.ansatz_state(n, d, out), xhat) - res.fidelity) <= 1e-12
    assert abs(oterms.cost_only(n, d, out, b, dec["coef"], dec["x"], dec["z"]) - res.cost) <= 1e-12


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_optimizer_runs_each_instance(dv, ctx, prec):
    """Several instances in lock step: each stops on its own fidelity."""
    items, keeps, xh, a0s, refs = [], [], [], [], []
    for k, n in enumerate([3, 4, 5, 4]):
        d = 2
        A = wl.toeplitz_dense(n, 2.0 + 0.3 * k, -0.6 - 0.1 * k)
        dec = odec.decompose(A, 0.0, 64)
        b = wl.plus_state(n)
        xhat = oterms.classical_solution(oterms.lcu_matrix(dec["coef"], dec["x"], dec["z"], n), b)
        alpha0 = wl.random_angles(n * (d + 1), 100 + k)
        lcu, keep = lcu_of(dv, dec["coef"], dec["x"], dec["z"])
        keeps.append((keep, cv(b), alpha0))
        items.append((dv.make_ansatz(n, d), lcu, alpha0, keeps[-1][1]))
        xh.append(xhat)
        a0s.append(alpha0)
        refs.append((n, d, b, dec, xhat))
    inst = dv.make_instances(items)
    P = sum(a.size for a in a0s)
    out = np.zeros(P)
    opt = dv.make_adam(lr=0.03, max_iter=80, target_fidelity=0.99, precision=prec)
    res = dv.dvqls_optimize(ctx, inst, cv(np.concatenate(xh)), opt, out)
    off = 0
    for r, (n, d, b, dec, xhat), a0 in zip(res, refs, a0s):
        a = out[off:off + a0.size]
        off += a0.size
        F = oterms.fidelity(oterms.ansatz_state(n, d, a), xhat)
        assert abs(F - r.fidelity) <= (1e-12 if prec == 0 else 1e-6)
        assert r.converged == (1 if F >= 0.99 else 0) or abs(F - 0.99) < 1e-6
        if prec == 0:
            it_ref, a_ref = adam_reference(n, d, a0, b, dec["coef"], dec["x"], dec["z"], xhat, 0.03, 80, 0.99)[:2]
            assert abs(r.iters - it_ref) <= 1
            if r.iters == it_ref:
                assert np.abs(a - a_ref).max() <= 1e-8


@pytest.mark.parametrize("case", ["toeplitz12", "indefinite12", "toeplitz20"])
def test_grid_cg_large_systems(dv, ctx, case):
    """One system of N >= 4096 runs the grid-wide CG: the residual of the
    returned x, formed on the CPU with the oracle's Pauli action, meets the
    tolerance (indefinite A~ through the normal equations)."""
    if case == "indefinite12":  # 0.5 I + Z_0 + 0.3 X_1: CG breaks down, the normal equations converge
        n = 12
        dec = {"coef": np.array([0.5, 1.0, 0.3]), "x": np.array([0, 0, 2], np.uint32),
               "z": np.array([0, 1, 0], np.uint32)}
        b = np.random.default_rng(4).normal(size=1 << n) + 0j
        tol = 1e-11
    else:
        n = 12 if case == "toeplitz12" else 20
        inst = wl.throughput_instance(3, n=n)
        dec = odec.decompose_banded(n, inst["offsets"], inst["bands"], 0.0, 64)
        b = inst["b"].astype(np.complex128)
        tol = 1e-12
    lcu, keep = lcu_of(dv, dec["coef"], dec["x"], dec["z"])
    x = np.zeros(2 << n)
    it, rr = dv.dvqls_lcu_solve(ctx, n, lcu, cv(b), tol, 20000, x)
    x = x.view(np.complex128)
    Ax = np.zeros_like(x)
    for c, xm, zm in zip(dec["coef"], dec["x"], dec["z"]):
        Ax += c * oterms.apply_pauli(xm, zm, x)
    if case == "indefinite12":  # the normal equations' residual is ||A^dag (A x - b)||
        res = np.zeros_like(x)
        for c, xm, zm in zip(dec["coef"], dec["x"], dec["z"]):
            res += np.conj(c) * oterms.apply_pauli(xm, zm, Ax - b)
        rhs = np.zeros_like(x)
        for c, xm, zm in zip(dec["coef"], dec["x"], dec["z"]):
            rhs += np.conj(c) * oterms.apply_pauli(xm, zm, b)
        assert np.linalg.norm(res) <= 10 * tol * np.linalg.norm(rhs)
        assert np.linalg.norm(Ax - b) <= 1e-8 * np.linalg.norm(b)
    else:
        assert np.linalg.norm(Ax - b) <= 10 * tol * np.linalg.norm(b)
    assert rr <= tol and it > 0


@pytest.mark.parametrize("prec", [0, 2])
def test_optimizer_checkpoint_resume_is_bit_exact(dv, ctx, prec):
    """K1 updates, a checkpoint of (angles, Adam moments, update counts), then K2
    more updates from it give, bit for bit, the angles and state of one run of
    K1 + K2 updates; a fresh state reproduces dvqls_optimize."""
    items, keeps, xh, P = [], [], [], []
    for k, n in enumerate([3, 5]):
        d = 2
        A = wl.toeplitz_dense(n, 2.2 + 0.3 * k, -0.7)
        dec = odec.decompose(A, 0.0, 64)
        b = wl.plus_state(n)
        xh.append(oterms.classical_solution(oterms.lcu_matrix(dec["coef"], dec["x"], dec["z"], n), b))
        alpha0 = wl.random_angles(n * (d + 1), 300 + k)
        lcu, keep = lcu_of(dv, dec["coef"], dec["x"], dec["z"])
        keeps.append((keep, cv(b), alpha0))
        items.append((dv.make_ansatz(n, d), lcu, alpha0, keeps[-1][1]))
        P.append(n * (d + 1))
    inst = dv.make_instances(items)
    xhat = np.concatenate([cv(x) for x in xh])
    Pt = sum(P)

    def opt(iters):  # an unreachable target: every instance runs all its updates
        return dv.make_adam(lr=0.03, max_iter=iters, target_fidelity=2.0, precision=prec)

    # one run of 20 updates
    m, v, steps = np.zeros(Pt), np.zeros(Pt), np.zeros(2, np.int64)
    a_full = np.zeros(Pt)
    dv.dvqls_optimize_resume(ctx, inst, xhat, opt(20), m, v, steps, a_full)
    assert list(steps) == [20, 20]
    plain = np.zeros(Pt)
    dv.dvqls_optimize(ctx, inst, xhat, opt(20), plain)
    assert np.array_equal(plain.view(np.uint64), a_full.view(np.uint64))
    # 8 updates, checkpoint, 12 more
    m2, v2, st2 = np.zeros(Pt), np.zeros(Pt), np.zeros(2, np.int64)
    a8 = np.zeros(Pt)
    dv.dvqls_optimize_resume(ctx, inst, xhat, opt(8), m2, v2, st2, a8)
    assert list(st2) == [8, 8]
    items2, off = [], 0
    for (an, lcu, _, b), p in zip(items, P):
        items2.append((an, lcu, a8[off:off + p].copy(), b))
        off += p
    keep_a = [it[2] for it in items2]
    inst2 = dv.make_instances(items2)
    a20 = np.zeros(Pt)
    dv.dvqls_optimize_resume(ctx, inst2, xhat, opt(12), m2, v2, st2, a20)
    assert list(st2) == [20, 20]
    for x, y in ((a20, a_full), (m2, m), (v2, v)):
        assert np.array_equal(x.view(np.uint64), y.view(np.uint64))
    assert len(keep_a) == 2
