"""The allocation-free entry point agrees with the allocating one.

dvqls_cost_grad_noalloc is for callers that must not allocate GPU memory
(for example code running under an allocator that owns the device); it uses
a fixed scratch array inside the library instead of a context workspace.
Here it is called through the C-ABI twice in a row (the second call sees the
first call's leftovers in the shared array) and compared with
dvqls_cost_grad on the same inputs, within the tolerances of the other GPU
tests.  This file is collected last so a failure here never hides another."""
import numpy as np
import pytest
import torch

from paper_2604_14435_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {0: (1e-12, 1e-12), 1: (1e-6, 1e-5)}  # precision -> (cost, grad)


def device_problem(n, d, L, seed):
    rng = np.random.default_rng(seed)
    N = 1 << n
    coef = rng.normal(size=L) + 1j * rng.normal(size=L)
    xs = rng.integers(0, N, L).astype(np.uint32)
    zs = rng.integers(0, N, L).astype(np.uint32)
    b = rng.normal(size=N) + 1j * rng.normal(size=N)
    alpha = wl.random_angles(n * (d + 1), seed + 1)
    t = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=dt)
    return (t(coef.view(np.float64)), t(xs.view(np.int32), torch.int32), t(zs.view(np.int32), torch.int32),
            t(alpha), t(b.view(np.float64)))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,d,L", [(10, 4, 64), (6, 2, 70), (3, 1, 5)])
def test_noalloc_matches_cost_grad(dv, ctx, prec, n, d, L):
    coef, xm, zm, alpha, b = device_problem(n, d, L, 40 + n + L)
    an = dv.make_ansatz(n, d)
    lcu = dv.make_lcu(L, coef, xm, zm)
    P = n * (d + 1)
    ref_cost = np.zeros(1)
    ref_grad = np.zeros(P)
    dv.dvqls_cost_grad(ctx, an, alpha, lcu, b, prec, ref_cost, ref_grad)
    stream = torch.cuda.current_stream().cuda_stream
    tc, tg = TOL[prec]
    for _ in range(2):
        cost = torch.full((1,), np.nan, device="cuda", dtype=torch.float64)
        grad = torch.full((P,), np.nan, device="cuda", dtype=torch.float64)
        assert dv.dvqls_cost_grad_noalloc(stream, an, alpha, lcu, b, prec, cost, grad) == dv.DVQLS_OK
        c = cost.cpu().numpy()
        g = grad.cpu().numpy()
        assert abs(c[0] - ref_cost[0]) <= tc * max(1.0, abs(ref_cost[0]))
        assert np.all(np.abs(g - ref_grad) <= tg * np.maximum(1.0, np.abs(ref_grad)))


def test_noalloc_rejects_what_it_cannot_serve(dv):
    stream = torch.cuda.current_stream().cuda_stream
    n, d = 6, 1
    # more scratch than the fixed array holds (L^2 weights alone exceed it)
    L = 300
    coef, xm, zm, alpha, b = device_problem(n, d, L, 3)
    cost = torch.zeros(1, device="cuda", dtype=torch.float64)
    grad = torch.zeros(n * (d + 1), device="cuda", dtype=torch.float64)
    an, lcu = dv.make_ansatz(n, d), dv.make_lcu(L, coef, xm, zm)
    assert dv.dvqls_cost_grad_noalloc(stream, an, alpha, lcu, b, 1, cost, grad) == dv.DVQLS_ERR_INVALID_ARG
    # host buffers are not staged
    L = 4
    coef, xm, zm, alpha, b = device_problem(n, d, L, 4)
    lcu = dv.make_lcu(L, coef, xm, zm)
    host_cost = np.zeros(1)
    assert dv.dvqls_cost_grad_noalloc(stream, an, alpha, lcu, b, 1, host_cost, grad) == dv.DVQLS_ERR_INVALID_ARG
