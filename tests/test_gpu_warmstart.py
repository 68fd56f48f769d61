"""Learned warm start: GPU MLP kernels vs the FP64 oracle, checkpointing, and
what the trained network gains over the fallback initialisation."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2604_14435_gb300 import warmstart as W

pytestmark = pytest.mark.gpu


def random_net(I, H, O, B, seed):
    rng = np.random.default_rng(seed)
    p = (rng.normal(size=omlp.param_count(I, H, O)) * 0.3).astype(np.float32)
    X = rng.normal(size=(B, I)).astype(np.float32)
    T = rng.normal(size=(B, O)).astype(np.float32)
    M = (rng.random((B, O)) < 0.6).astype(np.float32)
    return p, X, T, M


@pytest.mark.parametrize("I,H,O,B", [(7, 33, 11, 37), (7, 256, 50, 64)])
def test_forward_and_gradient_match_oracle(dv, ctx, I, H, O, B):
    p, X, T, M = random_net(I, H, O, B, I + H)
    assert dv.dvqls_ws_param_count(I, H, O) == p.size
    ws = dv.dvqls_ws_create(ctx, I, H, O, p)
    try:
        y = np.zeros((B, O), np.float32)
        dv.dvqls_ws_infer(ws, B, X, y)
        y_ref, _ = omlp.forward(p.astype(np.float64), X, I, H, O)
        assert np.abs(y - y_ref).max() <= 1e-4 * max(1.0, np.abs(y_ref).max())
        g = np.zeros(p.size, np.float32)
        loss = dv.dvqls_ws_grad(ws, B, X, T, M, g)
        l_ref = omlp.loss(p.astype(np.float64), X, T, M, I, H, O)
        g_ref = omlp.grad(p.astype(np.float64), X, T, M, I, H, O)
        assert abs(loss - l_ref) <= 1e-4 * max(1.0, abs(l_ref))
        assert np.abs(g - g_ref).max() <= 1e-4 * max(1.0, np.abs(g_ref).max())
    finally:
        dv.dvqls_ws_destroy(ws)


def test_train_step_is_adam_on_the_gradient(dv, ctx):
    I, H, O, B = 7, 16, 9, 20
    p, X, T, M = random_net(I, H, O, B, 5)
    ws = dv.dvqls_ws_create(ctx, I, H, O, p)
    try:
        lr = 1e-2
        q = p.astype(np.float64).copy()
        m = np.zeros_like(q)
        v = np.zeros_like(q)
        for step in range(1, 4):
            loss = dv.dvqls_ws_train_step(ws, B, X, T, M, lr)
            assert abs(loss - omlp.loss(q, X, T, M, I, H, O)) <= 1e-4 * max(1.0, loss)
            g = omlp.grad(q, X, T, M, I, H, O)
            m = 0.9 * m + 0.1 * g
            v = 0.999 * v + 0.001 * g * g
            q = q - lr * (m / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
        got = np.zeros(p.size, np.float32)
        dv.dvqls_ws_get_params(ws, got)
        assert np.abs(got - q).max() <= 1e-4
    finally:
        dv.dvqls_ws_destroy(ws)


def test_checkpoint_round_trip(dv, ctx, tmp_path):
    I, H, O, B = 7, 12, 6, 10
    p, X, T, M = random_net(I, H, O, B, 9)
    a = dv.dvqls_ws_create(ctx, I, H, O, p)
    try:
        for _ in range(3):
            dv.dvqls_ws_train_step(a, B, X, T, M, 5e-3)
        path = tmp_path / "ws.bin"
        dv.dvqls_ws_save(a, path)
        b = dv.dvqls_ws_load(ctx, path)
        try:
            la = dv.dvqls_ws_train_step(a, B, X, T, M, 5e-3)
            lb = dv.dvqls_ws_train_step(b, B, X, T, M, 5e-3)
            assert la == lb
            pa = np.zeros(p.size, np.float32)
            pb = np.zeros(p.size, np.float32)
            dv.dvqls_ws_get_params(a, pa)
            dv.dvqls_ws_get_params(b, pb)
            assert np.array_equal(pa, pb)
        finally:
            dv.dvqls_ws_destroy(b)
    finally:
        dv.dvqls_ws_destroy(a)
    with pytest.raises(dv.DvqlsError):
        bad = tmp_path / "bad.bin"
        bad.write_bytes(b"not a checkpoint")
        dv.dvqls_ws_load(ctx, bad)


def test_learned_start_beats_fallback(dv, ctx):
    """The warm-start pipeline at reduced size (200 training systems of n =
    6..10, 20 held-out systems of n = 10).  Training targets: FP64 L-BFGS runs
    from the perturbed |+> start carried to convergence (L-BFGS-B's default
    stopping tests).  Held out, the network's angles start closer than the zero
    start; Adam from them reaches F_ref - 1e-4 (F_ref: the converged FP64 run
    from |+>) in at least three runs of four and in fewer iterations (median)
    than from the zero start; FP64 L-BFGS from them converges in fewer
    iterations (median) than from |+>."""
    out = W.run(ctx, n_train=200, n_eval=20, max_iter=2000, train_steps=1500, n_deep=0, log=lambda *a: None)
    tg = out["train"]["targets"]
    assert sum(tg["stopped"].get(k, 0) for k in ("gtol", "ftol", "ls")) == tg["runs"] == 200
    assert tg["grad_maxnorm_median"] <= 1e-2
    loss = out["train"]["loss_curve"]
    assert loss[-1][1] < loss[0][1]
    mlp, zero, plus = (out["inits"][k] for k in ("mlp", "zero", "plus"))
    assert mlp["initial_fidelity_median"] > zero["initial_fidelity_median"]
    assert mlp["adam_to_reference"]["reached"] >= (3 * 20) // 4
    assert mlp["adam_to_reference"]["iters_median"] < zero["adam_to_reference"]["iters_median"]
    assert mlp["lbfgs_fp64"]["iters_median"] < plus["lbfgs_fp64"]["iters_median"]
