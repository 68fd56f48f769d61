"""One instance split into shift ranges on one GPU, then combined (Sec. 2.3
Stage III; Algorithm 1, Step 4c): the per-shift sums of the ranges add up
to the whole instance's, and dvqls_combine_partials then gives the cost and
gradient of dvqls_cost_grad and of the FP64 oracle (tolerances as in the
other GPU tests)."""
import numpy as np
import pytest
import torch

from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl

from test_gpu_terms import TOL32, TOL64, cvec, dev, random_problem

pytestmark = pytest.mark.gpu


def device_args(dv, n, d, alpha, b, coef, xs, zs):
    t = (dev(cvec(coef)), dev(np.asarray(xs, np.uint32).view(np.int32), torch.int32),
         dev(np.asarray(zs, np.uint32).view(np.int32), torch.int32), dev(alpha), dev(cvec(b)))
    return t, dv.make_ansatz(n, d), dv.make_lcu(len(xs), t[0], t[1], t[2])


def split_cost_grad(dv, ctx, an, lcu, alpha_d, b_d, prec, cuts, host=False):
    P = an.n * (an.depth + 1)
    S = 2 * P + 1
    edges = [0] + list(cuts) + [S]
    total = np.zeros(S * 4)
    for s0, s1 in zip(edges, edges[1:]):
        part = np.full(S * 4, np.nan) if host else torch.full((S * 4,), np.nan, device="cuda", dtype=torch.float64)
        dv.dvqls_cost_grad_partials(ctx, an, alpha_d, lcu, b_d, prec, s0, s1, part)
        p = part if host else part.cpu().numpy()
        outside = np.ones(S, bool)
        outside[s0:s1] = False
        assert np.all(p.reshape(S, 4)[outside] == 0.0)  # zeros outside the rank's range
        assert np.all(np.isfinite(p))
        total += p
    cost = torch.zeros(1, device="cuda", dtype=torch.float64)
    grad = torch.zeros(P, device="cuda", dtype=torch.float64)
    dv.dvqls_combine_partials(ctx, an.n, an.depth, dev(total), cost, grad)
    return cost.item(), grad.cpu().numpy()


def compare(prec, cost, grad, ref):
    if prec == 0:
        assert abs(cost - ref["cost"]) <= TOL64 * max(1.0, abs(ref["cost"]))
        assert np.all(np.abs(grad - ref["grad"]) <= TOL64 * np.maximum(1.0, np.abs(ref["grad"])))
    else:
        assert abs(cost - ref["cost"]) <= TOL32["cost"]
        assert np.abs(grad - ref["grad"]).max() <= TOL32["grad"]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_split_throughput_instance_matches_whole(dv, ctx, prec):
    inst = wl.throughput_instance(1)
    n, d = inst["n"], inst["d"]
    dec = odec.decompose_banded(n, inst["offsets"], inst["bands"], 0.0, 64)
    args = (n, d, inst["alpha"], inst["b"], dec["coef"], dec["x"], dec["z"])
    ref = oterms.cost_grad(*args)
    t, an, lcu = device_args(dv, *args)
    whole_c = np.zeros(1)
    whole_g = np.zeros(50)
    dv.dvqls_cost_grad(ctx, an, t[3], lcu, t[4], prec, whole_c, whole_g)
    for cuts in ((40,), (1, 50, 77)):
        cost, grad = split_cost_grad(dv, ctx, an, lcu, t[3], t[4], prec, cuts, host=(len(cuts) == 3))
        compare(prec, cost, grad, ref)
        tol = TOL64 if prec == 0 else TOL32["cost"]
        assert abs(cost - whole_c[0]) <= tol * max(1.0, abs(whole_c[0]))


@pytest.mark.parametrize("prec", [1, 2])
def test_split_hbm_instance(dv, ctx, prec):
    """States in HBM (n = 14): each range builds only its own shifted states."""
    rng = np.random.default_rng(41)
    n, d, L = 14, 1, 20
    coef, xs, zs, b = random_problem(rng, n, L)
    alpha = wl.random_angles(n * (d + 1), 42)
    ref = oterms.cost_grad(n, d, alpha, b, coef, xs, zs)
    t, an, lcu = device_args(dv, n, d, alpha, b, coef, xs, zs)
    cost, grad = split_cost_grad(dv, ctx, an, lcu, t[3], t[4], prec, (28,))
    compare(prec, cost, grad, ref)


def test_split_rejects_bad_ranges(dv, ctx):
    rng = np.random.default_rng(3)
    n, d, L = 4, 1, 5
    coef, xs, zs, b = random_problem(rng, n, L)
    alpha = wl.random_angles(n * (d + 1), 4)
    t, an, lcu = device_args(dv, n, d, alpha, b, coef, xs, zs)
    S = 2 * n * (d + 1) + 1
    part = torch.zeros(S * 4, device="cuda", dtype=torch.float64)
    for s0, s1 in ((3, 3), (-1, 4), (0, S + 1), (5, 2)):
        with pytest.raises(dv.DvqlsError) as e:
            dv.dvqls_cost_grad_partials(ctx, an, t[3], lcu, t[4], 1, s0, s1, part)
        assert e.value.code == dv.DVQLS_ERR_INVALID_ARG
    zero = torch.zeros(S * 4, device="cuda", dtype=torch.float64)  # D_0 = 0
    with pytest.raises(dv.DvqlsError) as e:
        dv.dvqls_combine_partials(ctx, n, d, zero, torch.zeros(1, device="cuda", dtype=torch.float64),
                                  torch.zeros(n * (d + 1), device="cuda", dtype=torch.float64))
    assert e.value.code == dv.DVQLS_ERR_NUMERIC
