"""Local cost (Eq. 2/4, b = |+>^n) on the GPU vs the oracle."""
import numpy as np
import pytest
import torch

from oracle import circuit as ocirc
from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# 2: the tensor-core tiles (flavour j as a Gram of the tile against its strings with x ^ e_j);
# 3: the Walsh-Hadamard classes (served for L <= 64, n <= 10; FP32 otherwise); both held to the FP32 bounds
TOL = {0: (1e-12, 1e-12), 1: (1e-6, 1e-5), 2: (1e-6, 1e-5), 3: (1e-6, 1e-5)}


def cv(a):
    return np.ascontiguousarray(np.asarray(a, np.complex128)).view(np.float64)


def run(dv, ctx, n, d, alpha, coef, xs, zs, prec, grad=True):
    lcu = dv.make_lcu(len(xs), cv(coef), np.ascontiguousarray(xs, np.uint32), np.ascontiguousarray(zs, np.uint32))
    cost = np.zeros(1)
    g = np.zeros(n * (d + 1)) if grad else None
    dv.dvqls_local_cost_grad(ctx, dv.make_ansatz(n, d), np.ascontiguousarray(alpha, np.float64), lcu, prec, cost, g)
    return cost[0], g


def ok(got, ref, tol):
    return np.all(np.abs(np.asarray(got) - np.asarray(ref)) <= tol * np.maximum(1.0, np.abs(ref)))


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("n,d,L", [(1, 1, 2), (2, 1, 5), (3, 2, 8), (5, 2, 33), (6, 1, 70), (8, 1, 20)])
def test_local_cost_matches_oracle(dv, ctx, prec, n, d, L):
    rng = np.random.default_rng(900 + n + L)
    N = 1 << n
    coef = rng.normal(size=L) + 1j * rng.normal(size=L)
    xs = rng.integers(0, N, L).astype(np.uint32)
    zs = rng.integers(0, N, L).astype(np.uint32)
    alpha = wl.random_angles(n * (d + 1), 901 + n)
    ref = oterms.local_cost_grad(n, d, alpha, coef, xs, zs)
    cost, g = run(dv, ctx, n, d, alpha, coef, xs, zs, prec)
    tc, tg = TOL[prec]
    assert ok(cost, ref["cost"], tc) and ok(g, ref["grad"], tg)
    c_only, _ = run(dv, ctx, n, d, alpha, coef, xs, zs, prec, grad=False)
    assert ok(c_only, ref["cost"], tc)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_local_cost_throughput_system(dv, ctx, prec):
    """n = 10 Toeplitz, top-64: the paper's 90,112-circuit evaluation, with
    sampled gamma overlaps checked against their Hadamard-test circuits."""
    inst = wl.throughput_instance(7)
    n, d = 10, 4
    dec = odec.decompose_banded(n, inst["offsets"], inst["bands"], 0.0, 64)
    ref = oterms.local_cost_grad(n, d, inst["alpha"], dec["coef"], dec["x"], dec["z"])
    cost, g = run(dv, ctx, n, d, inst["alpha"], dec["coef"], dec["x"], dec["z"], prec)
    tc, tg = TOL[prec]
    assert ok(cost, ref["cost"], tc) and ok(g, ref["grad"], tg)
    # the oracle's definition-level gamma against its own circuits on a sample
    _, gamma = oterms.local_terms(oterms.ansatz_state(n, d, inst["alpha"]), dec["x"][:3], dec["z"][:3], n)
    cg, _ = ocirc.circuit_local_terms(n, d, inst["alpha"], inst["b"], dec["x"][:3], dec["z"][:3])
    assert np.abs(cg - gamma).max() < 1e-13


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_local_cost_batched_and_hbm(dv, ctx, prec):
    rng = np.random.default_rng(3)
    probs = []
    for n, d, L in [(4, 1, 6), (13, 1, 5), (7, 2, 9)]:
        N = 1 << n
        probs.append((n, d, rng.normal(size=L) + 1j * rng.normal(size=L), rng.integers(0, N, L).astype(np.uint32),
                      rng.integers(0, N, L).astype(np.uint32), wl.random_angles(n * (d + 1), n)))
    keep, items = [], []
    for n, d, coef, xs, zs, alpha in probs:
        t = (cv(coef), xs, zs, np.ascontiguousarray(alpha))
        keep.append(t)
        items.append((dv.make_ansatz(n, d), dv.make_lcu(len(xs), t[0], t[1], t[2]), t[3], None))
    arr = dv.make_instances(items)
    P = sum(p[0] * (p[1] + 1) for p in probs)
    costs = torch.zeros(len(probs), device="cuda", dtype=torch.float64)
    grads = torch.zeros(P, device="cuda", dtype=torch.float64)
    dv.dvqls_local_cost_grad_batched(ctx, arr, prec, costs, grads)
    dv.dvqls_sync(ctx)
    tc, tg = TOL[prec]
    off = 0
    for k, (n, d, coef, xs, zs, alpha) in enumerate(probs):
        ref = oterms.local_cost_grad(n, d, alpha, coef, xs, zs)
        assert ok(costs[k].item(), ref["cost"], tc)
        assert ok(grads[off:off + n * (d + 1)].cpu().numpy(), ref["grad"], tg)
        off += n * (d + 1)


def test_local_cost_batched_wht(dv, ctx):
    """A batch the Walsh-Hadamard classes serve (every n <= 10, L <= 64), twice:
    the second call reuses the class tables."""
    rng = np.random.default_rng(31)
    probs = []
    for n, d, L in [(4, 1, 6), (7, 2, 9), (10, 1, 64), (1, 2, 2)]:
        N = 1 << n
        probs.append((n, d, rng.normal(size=L) + 1j * rng.normal(size=L), rng.integers(0, N, L).astype(np.uint32),
                      rng.integers(0, N, L).astype(np.uint32), wl.random_angles(n * (d + 1), 40 + n)))
    keep, items = [], []
    for n, d, coef, xs, zs, alpha in probs:
        t = (cv(coef), xs, zs, np.ascontiguousarray(alpha))
        keep.append(t)
        items.append((dv.make_ansatz(n, d), dv.make_lcu(len(xs), t[0], t[1], t[2]), t[3], None))
    arr = dv.make_instances(items)
    P = sum(p[0] * (p[1] + 1) for p in probs)
    tc, tg = TOL[3]
    for _ in range(2):
        costs = torch.zeros(len(probs), device="cuda", dtype=torch.float64)
        grads = torch.zeros(P, device="cuda", dtype=torch.float64)
        dv.dvqls_local_cost_grad_batched(ctx, arr, 3, costs, grads)
        dv.dvqls_sync(ctx)
        off = 0
        for k, (n, d, coef, xs, zs, alpha) in enumerate(probs):
            ref = oterms.local_cost_grad(n, d, alpha, coef, xs, zs)
            assert ok(costs[k].item(), ref["cost"], tc)
            assert ok(grads[off:off + n * (d + 1)].cpu().numpy(), ref["grad"], tg)
            off += n * (d + 1)
