"""The allocation-free entry point against the oracle and the allocating one.

dvqls_cost_grad_noalloc is for callers that must not allocate GPU memory
(for example code running under an allocator or memory pool that owns the
whole device, or a plugin host that forbids cudaMalloc); it uses a fixed
scratch array inside the library instead of a context workspace.  Here it is
called through the C-ABI twice in a row (the second call finds the first
call's leftovers in the shared array) and compared with the definition-level
FP64 oracle and with dvqls_cost_grad on the same inputs, within the
tolerances of the other GPU tests.  The largest sizes the header promises to
fit (n = 10, depth 4: L = 160 in FP32, L = 200 in FP64) are among the cases.
This file is collected last so a failure here never hides another."""
import numpy as np
import pytest
import torch

from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# precision -> (cost, grad) bounds: FP64 relative 1e-12; FP32 absolute 1e-6 / 1e-5
TOL = {0: (1e-12, 1e-12), 1: (1e-6, 1e-5)}
SCRATCH = 1 << 20  # DVQLS_NOALLOC_SCRATCH_BYTES


def host_problem(n, d, L, seed):
    rng = np.random.default_rng(seed)
    N = 1 << n
    coef = rng.normal(size=L) + 1j * rng.normal(size=L)
    xs = rng.integers(0, N, L).astype(np.uint32)
    zs = rng.integers(0, N, L).astype(np.uint32)
    b = rng.normal(size=N) + 1j * rng.normal(size=N)
    b /= np.linalg.norm(b)
    alpha = wl.random_angles(n * (d + 1), seed + 1)
    return coef, xs, zs, alpha, b


def to_device(coef, xs, zs, alpha, b):
    t = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=dt)
    return (t(coef.view(np.float64)), t(xs.view(np.int32), torch.int32), t(zs.view(np.int32), torch.int32),
            t(alpha), t(b.view(np.float64)))


def scratch_bytes(n, d, L, fp32, ks=8):
    """The header's scratch formula with the largest amplitude split."""
    r = lambda x: (x + 255) & ~255
    P = n * (d + 1)
    S, T = 2 * P + 1, (L + 63) // 64
    total = r(512) + 256 + r(16 * L) + r(16 * L * L) + r(48 * P) + r(8) + r(16 * S * T * T * ks) \
        + r(16 * S * T * ks) + r(24 * S)
    if fp32:
        total += r(16 * L * L) + r(16 * L)
    return total


_oracle_cache = {}


def oracle(n, d, L, seed):
    key = (n, d, L, seed)
    if key not in _oracle_cache:
        coef, xs, zs, alpha, b = host_problem(n, d, L, seed)
        _oracle_cache[key] = oterms.cost_grad(n, d, alpha, b, coef, xs, zs)
    return _oracle_cache[key]


@pytest.mark.parametrize("prec,n,d,L", [(0, 10, 4, 64), (1, 10, 4, 64), (0, 6, 2, 70), (1, 6, 2, 70),
                                        (0, 3, 1, 5), (1, 3, 1, 5), (1, 10, 4, 160), (0, 10, 4, 200)])
def test_noalloc_matches_oracle_and_cost_grad(dv, ctx, prec, n, d, L):
    assert scratch_bytes(n, d, L, prec == 1) <= SCRATCH  # fits whatever split the GPU picks
    seed = 40 + n + L
    host = host_problem(n, d, L, seed)
    coef, xm, zm, alpha, b = to_device(*host)
    an = dv.make_ansatz(n, d)
    lcu = dv.make_lcu(L, coef, xm, zm)
    P = n * (d + 1)
    ref_cost = np.zeros(1)
    ref_grad = np.zeros(P)
    dv.dvqls_cost_grad(ctx, an, alpha, lcu, b, prec, ref_cost, ref_grad)
    orc = oracle(n, d, L, seed)
    stream = torch.cuda.current_stream().cuda_stream
    tc, tg = TOL[prec]
    for _ in range(2):
        cost = torch.full((1,), np.nan, device="cuda", dtype=torch.float64)
        grad = torch.full((P,), np.nan, device="cuda", dtype=torch.float64)
        assert dv.dvqls_cost_grad_noalloc(stream, an, alpha, lcu, b, prec, cost, grad) == dv.DVQLS_OK
        c = cost.cpu().numpy()[0]
        g = grad.cpu().numpy()
        # against the FP64 oracle
        if prec == 0:
            assert abs(c - orc["cost"]) <= tc * max(1.0, abs(orc["cost"]))
            assert np.all(np.abs(g - orc["grad"]) <= tg * np.maximum(1.0, np.abs(orc["grad"])))
        else:
            assert abs(c - orc["cost"]) <= tc, abs(c - orc["cost"])
            assert np.abs(g - orc["grad"]).max() <= tg, np.abs(g - orc["grad"]).max()
        # against the allocating entry point
        assert abs(c - ref_cost[0]) <= tc * max(1.0, abs(ref_cost[0]))
        assert np.all(np.abs(g - ref_grad) <= tg * np.maximum(1.0, np.abs(ref_grad)))


def test_noalloc_rejects_what_it_cannot_serve(dv):
    stream = torch.cuda.current_stream().cuda_stream
    n, d = 6, 1
    # more scratch than the fixed array holds (L^2 weights alone exceed it)
    L = 300
    coef, xm, zm, alpha, b = to_device(*host_problem(n, d, L, 3))
    cost = torch.zeros(1, device="cuda", dtype=torch.float64)
    grad = torch.zeros(n * (d + 1), device="cuda", dtype=torch.float64)
    an, lcu = dv.make_ansatz(n, d), dv.make_lcu(L, coef, xm, zm)
    assert dv.dvqls_cost_grad_noalloc(stream, an, alpha, lcu, b, 1, cost, grad) == dv.DVQLS_ERR_INVALID_ARG
    # host buffers are not staged
    L = 4
    coef, xm, zm, alpha, b = to_device(*host_problem(n, d, L, 4))
    lcu = dv.make_lcu(L, coef, xm, zm)
    host_cost = np.zeros(1)
    assert dv.dvqls_cost_grad_noalloc(stream, an, alpha, lcu, b, 1, host_cost, grad) == dv.DVQLS_ERR_INVALID_ARG
    # the tensor-core and Walsh-Hadamard precisions are valid but not served here
    for prec in (dv.DVQLS_FP32_TC, dv.DVQLS_FP32_WHT):
        assert dv.dvqls_cost_grad_noalloc(stream, an, alpha, lcu, b, prec, cost, grad) == dv.DVQLS_ERR_UNSUPPORTED
    assert dv.dvqls_cost_grad_noalloc(stream, an, alpha, lcu, b, 7, cost, grad) == dv.DVQLS_ERR_INVALID_ARG
    # and the entry point still works after the rejections
    assert dv.dvqls_cost_grad_noalloc(stream, an, alpha, lcu, b, 0, cost, grad) == dv.DVQLS_OK
