"""GPU cost / gradient / beta / delta vs the oracle.

Tolerances: FP64 path
|gpu - cpu| <= 1e-12 * max(1, |cpu|) for beta, delta, cost and gradient; FP32
path <= 1e-5 absolute on beta and delta, <= 1e-6 on the cost, <= 1e-5 on the
gradient."""
import numpy as np
import pytest
import torch

from oracle import circuit as ocirc
from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = {"beta": 1e-5, "delta": 1e-5, "cost": 1e-6, "grad": 1e-5}


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype)


def cvec(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64)


def gpu_cost_grad(dv, ctx, n, d, alpha, b, coef, xs, zs, prec, grad=True, on_device=True):
    L = len(xs)
    if on_device:
        c_ = dev(cvec(coef))
        x_ = dev(np.asarray(xs, np.uint32).view(np.int32), torch.int32)
        z_ = dev(np.asarray(zs, np.uint32).view(np.int32), torch.int32)
        a_ = dev(alpha)
        b_ = dev(cvec(b))
    else:
        c_, x_, z_ = cvec(coef), np.ascontiguousarray(xs, np.uint32), np.ascontiguousarray(zs, np.uint32)
        a_, b_ = np.ascontiguousarray(alpha, np.float64), cvec(b)
    an = dv.make_ansatz(n, d)
    lcu = dv.make_lcu(L, c_, x_, z_)
    cost = np.zeros(1)
    beta = np.zeros(2 * L * L)
    delta = np.zeros(2 * L)
    out = {}
    if grad:
        g = np.zeros(n * (d + 1))
        dv.dvqls_cost_grad(ctx, an, a_, lcu, b_, prec, cost, g, beta, delta)
        out["grad"] = g
    else:
        dv.dvqls_cost(ctx, an, a_, lcu, b_, prec, cost, beta, delta)
    out["cost"] = cost[0]
    out["beta"] = beta.view(np.complex128).reshape(L, L)
    out["delta"] = delta.view(np.complex128)
    return out


def check(got, ref, prec):
    if prec == 0:
        for k in ("beta", "delta"):
            assert np.all(np.abs(got[k] - ref[k]) <= TOL64 * np.maximum(1.0, np.abs(ref[k]))), k
        assert abs(got["cost"] - ref["cost"]) <= TOL64 * max(1.0, abs(ref["cost"]))
        if "grad" in got:
            assert np.all(np.abs(got["grad"] - ref["grad"]) <= TOL64 * np.maximum(1.0, np.abs(ref["grad"])))
    else:
        for k in ("beta", "delta"):
            assert np.abs(got[k] - ref[k]).max() <= TOL32[k], (k, np.abs(got[k] - ref[k]).max())
        assert abs(got["cost"] - ref["cost"]) <= TOL32["cost"], abs(got["cost"] - ref["cost"])
        if "grad" in got:
            assert np.abs(got["grad"] - ref["grad"]).max() <= TOL32["grad"]


def random_problem(rng, n, L, complex_b=True):
    N = 1 << n
    xs = rng.integers(0, N, L).astype(np.uint32)
    zs = rng.integers(0, N, L).astype(np.uint32)
    coef = rng.normal(size=L) + 1j * rng.normal(size=L)
    b = rng.normal(size=N) + (1j * rng.normal(size=N) if complex_b else 0)
    return coef, xs, zs, b / np.linalg.norm(b)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("n,d,L", [(1, 0, 1), (1, 2, 3), (2, 1, 5), (3, 2, 8), (4, 3, 17), (5, 2, 64),
                                   (6, 2, 65), (7, 1, 130), (8, 2, 40)])
def test_random_lcu_against_definition(dv, ctx, prec, n, d, L):
    """Several tiles, ragged tails, complex b and coefficients, Y strings."""
    rng = np.random.default_rng(500 + 31 * n + L)
    coef, xs, zs, b = random_problem(rng, n, L)
    alpha = wl.random_angles(n * (d + 1), 900 + n)
    ref = oterms.cost_grad(n, d, alpha, b, coef, xs, zs)
    check(gpu_cost_grad(dv, ctx, n, d, alpha, b, coef, xs, zs, prec), ref, prec)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n,d,L", [(11, 1, 24), (12, 1, 20)])
def test_largest_on_chip_states(dv, ctx, prec, n, d, L):
    """n = 11 (four state copies per pipeline, the largest that fit) and n = 12
    (one copy; shared-memory gate passes) on the tensor-core and CUDA-core tiles."""
    rng = np.random.default_rng(600 + n)
    coef, xs, zs, b = random_problem(rng, n, L)
    alpha = wl.random_angles(n * (d + 1), 610 + n)
    ref = oterms.cost_grad(n, d, alpha, b, coef, xs, zs)
    check(gpu_cost_grad(dv, ctx, n, d, alpha, b, coef, xs, zs, prec), ref, prec)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_cost_only_and_host_pointers(dv, ctx, prec):
    rng = np.random.default_rng(77)
    n, d, L = 5, 3, 20
    coef, xs, zs, b = random_problem(rng, n, L)
    alpha = wl.random_angles(n * (d + 1), 78)
    ref = oterms.cost_grad(n, d, alpha, b, coef, xs, zs)
    got = gpu_cost_grad(dv, ctx, n, d, alpha, b, coef, xs, zs, prec, grad=False, on_device=False)
    check(got, ref, prec)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_validation_system_32_angles(dv, ctx, prec):
    """n = 3 Toeplitz, full decomposition (L = 8), 32 seeded angle vectors."""
    s = wl.validation_system()
    dec = odec.decompose(s["A"], 0.0, 64)
    for alpha in s["alphas"]:
        ref = oterms.cost_grad(3, 2, alpha, s["b"], dec["coef"], dec["x"], dec["z"])
        check(gpu_cost_grad(dv, ctx, 3, 2, alpha, s["b"], dec["coef"], dec["x"], dec["z"], prec), ref, prec)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("seed", [0, 1])
def test_throughput_system_full_size(dv, ctx, prec, seed):
    """n = 10, top-64 terms, depth 4: all 101 x 4160 terms against the
    definition-level oracle, and sampled terms against the circuit oracle."""
    inst = wl.throughput_instance(seed)
    n, d = inst["n"], inst["d"]
    dec = odec.decompose_banded(n, inst["offsets"], inst["bands"], 0.0, 64)
    ref = oterms.cost_grad(n, d, inst["alpha"], inst["b"], dec["coef"], dec["x"], dec["z"])
    got = gpu_cost_grad(dv, ctx, n, d, inst["alpha"], inst["b"], dec["coef"], dec["x"], dec["z"], prec)
    check(got, ref, prec)
    rng = np.random.default_rng(seed)
    for _ in range(6):
        l, m = rng.integers(0, 64, 2)
        v = ocirc.hadamard_beta(n, d, inst["alpha"], int(dec["x"][l]), int(dec["z"][l]), int(dec["x"][m]),
                                int(dec["z"][m]))
        assert abs(got["beta"][l, m] - v) <= (1e-12 if prec == 0 else TOL32["beta"])
    v = ocirc.hadamard_delta(n, d, inst["alpha"], inst["b"], int(dec["x"][5]), int(dec["z"][5]))
    assert abs(got["delta"][5] - v) <= (1e-12 if prec == 0 else TOL32["delta"])


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_batched_matches_single(dv, ctx, prec):
    """Mixed n, depth and L in one persistent launch == one call each."""
    rng = np.random.default_rng(5)
    probs = []
    for n, d, L in [(3, 1, 4), (10, 4, 64), (6, 3, 70), (12, 1, 9), (1, 0, 2), (8, 2, 33)]:
        coef, xs, zs, b = random_problem(rng, n, L)
        probs.append((n, d, L, wl.random_angles(n * (d + 1), int(rng.integers(1 << 30))), coef, xs, zs, b))
    keep = []
    items = []
    for n, d, L, alpha, coef, xs, zs, b in probs:
        t = (dev(cvec(coef)), dev(np.asarray(xs, np.uint32).view(np.int32), torch.int32),
             dev(np.asarray(zs, np.uint32).view(np.int32), torch.int32), dev(alpha), dev(cvec(b)))
        keep.append(t)
        items.append((dv.make_ansatz(n, d), dv.make_lcu(L, t[0], t[1], t[2]), t[3], t[4]))
    arr = dv.make_instances(items)
    P = sum(p[0] * (p[1] + 1) for p in probs)
    costs = torch.zeros(len(probs), device="cuda", dtype=torch.float64)
    grads = torch.zeros(P, device="cuda", dtype=torch.float64)
    for _ in range(2):  # second call reuses the uploaded table
        dv.dvqls_cost_grad_batched(ctx, arr, prec, costs, grads)
        dv.dvqls_sync(ctx)
        off = 0
        for k, (n, d, L, alpha, coef, xs, zs, b) in enumerate(probs):
            ref = oterms.cost_grad(n, d, alpha, b, coef, xs, zs)
            P_k = n * (d + 1)
            tol_c = TOL64 if prec == 0 else TOL32["cost"]
            tol_g = TOL64 if prec == 0 else TOL32["grad"]
            assert abs(costs[k].item() - ref["cost"]) <= tol_c * max(1, abs(ref["cost"]))
            g = grads[off:off + P_k].cpu().numpy()
            assert np.all(np.abs(g - ref["grad"]) <= tol_g * np.maximum(1, np.abs(ref["grad"])))
            off += P_k


def test_invalid_inputs_report_status(dv, ctx):
    rng = np.random.default_rng(1)
    coef, xs, zs, b = random_problem(rng, 3, 4)
    bad = xs.copy()
    bad[2] = 8  # >= 2^n
    with pytest.raises(dv.DvqlsError) as e:
        gpu_cost_grad(dv, ctx, 3, 1, np.zeros(6), b, coef, bad, zs, 1)
    assert e.value.code == dv.DVQLS_ERR_INVALID_ARG
    with pytest.raises(dv.DvqlsError) as e:
        gpu_cost_grad(dv, ctx, 3, 1, np.zeros(6), np.zeros(8), coef, xs, zs, 1)
    assert e.value.code == dv.DVQLS_ERR_INVALID_ARG
    a = np.zeros(6)
    a[3] = np.nan
    with pytest.raises(dv.DvqlsError) as e:
        gpu_cost_grad(dv, ctx, 3, 1, a, b, coef, xs, zs, 0)
    assert e.value.code == dv.DVQLS_ERR_INVALID_ARG
    with pytest.raises(dv.DvqlsError) as e:  # zero operator: D = 0
        gpu_cost_grad(dv, ctx, 3, 1, np.zeros(6), b, np.zeros(4, complex), xs, zs, 0)
    assert e.value.code == dv.DVQLS_ERR_NUMERIC
    with pytest.raises(dv.DvqlsError) as e:
        gpu_cost_grad(dv, ctx, 0, 1, np.zeros(1), b, coef, xs, zs, 0)
    assert e.value.code == dv.DVQLS_ERR_INVALID_ARG
    # still usable
    ref = oterms.cost_grad(3, 1, np.zeros(6), b, coef, xs, zs)
    check(gpu_cost_grad(dv, ctx, 3, 1, np.zeros(6), b, coef, xs, zs, 0), ref, 0)


def test_empty_batch_is_rejected(dv, ctx):
    """An empty batch is INVALID_ARG for the batched global and local calls and the
    optimizer; the context stays usable."""
    empty = dv.make_instances([])
    costs = torch.zeros(1, device="cuda", dtype=torch.float64)
    for call in (dv.dvqls_cost_grad_batched, dv.dvqls_local_cost_grad_batched):
        with pytest.raises(dv.DvqlsError) as e:
            call(ctx, empty, dv.DVQLS_FP32, costs, None)
        assert e.value.code == dv.DVQLS_ERR_INVALID_ARG
    with pytest.raises(dv.DvqlsError) as e:
        dv.dvqls_optimize(ctx, empty, np.zeros(2), dv.make_adam(max_iter=1), np.zeros(1))
    assert e.value.code == dv.DVQLS_ERR_INVALID_ARG
    rng = np.random.default_rng(2)
    coef, xs, zs, b = random_problem(rng, 3, 4)
    ref = oterms.cost_grad(3, 1, np.zeros(6), b, coef, xs, zs)
    check(gpu_cost_grad(dv, ctx, 3, 1, np.zeros(6), b, coef, xs, zs, 0), ref, 0)
