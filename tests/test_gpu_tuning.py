"""The autotuner's choices pinned with dvqls_set_tuning, against the oracle.

A mixed batch on the tensor-core tiles (n = 4 .. 11, one to two 64-term tiles)
runs with every state layout of the builders -- split hi / lo arrays for every
size, split arrays only from 2^9 amplitudes, packed copies -- and every
amplitude split.  The layouts put the same operand values into the same MMAs,
so their results agree bit for bit; the splits change only the order of the
partial sums.  Every run is checked against the FP64 oracle within the FP32
bounds of the other parity tests.  Each test owns its context, since the
setting stays with a context."""
import numpy as np
import pytest
import torch

from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl

from test_gpu_terms import TOL32, cvec, dev, random_problem

pytestmark = pytest.mark.gpu

SHAPES = [(4, 1, 6), (6, 2, 20), (8, 1, 33), (10, 2, 64), (11, 1, 40), (9, 1, 70)]


@pytest.fixture(scope="module")
def batch():
    rng = np.random.default_rng(21)
    probs = []
    for n, d, L in SHAPES:
        coef, xs, zs, b = random_problem(rng, n, L)
        probs.append((n, d, L, wl.random_angles(n * (d + 1), int(rng.integers(1 << 30))), coef, xs, zs, b))
    refs = [oterms.cost_grad(n, d, a, b, c, x, z) for n, d, L, a, c, x, z, b in probs]
    return probs, refs


def run(dv, probs, split, layout):
    ctx = dv.dvqls_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        dv.dvqls_set_tuning(ctx, split, layout)
        keep, items = [], []
        for n, d, L, alpha, coef, xs, zs, b in probs:
            t = (dev(cvec(coef)), dev(np.asarray(xs, np.uint32).view(np.int32), torch.int32),
                 dev(np.asarray(zs, np.uint32).view(np.int32), torch.int32), dev(alpha), dev(cvec(b)))
            keep.append(t)
            items.append((dv.make_ansatz(n, d), dv.make_lcu(L, t[0], t[1], t[2]), t[3], t[4]))
        arr = dv.make_instances(items)
        P = sum(p[0] * (p[1] + 1) for p in probs)
        costs = torch.zeros(len(probs), device="cuda", dtype=torch.float64)
        grads = torch.zeros(P, device="cuda", dtype=torch.float64)
        dv.dvqls_cost_grad_batched(ctx, arr, dv.DVQLS_FP32_TC, costs, grads)
        dv.dvqls_sync(ctx)
        return costs.cpu().numpy(), grads.cpu().numpy()
    finally:
        dv.dvqls_destroy(ctx)


def check(probs, refs, costs, grads):
    off = 0
    for k, (n, d, L, *_rest) in enumerate(probs):
        P_k = n * (d + 1)
        assert abs(costs[k] - refs[k]["cost"]) <= TOL32["cost"], (k, costs[k], refs[k]["cost"])
        assert np.abs(grads[off:off + P_k] - refs[k]["grad"]).max() <= TOL32["grad"]
        off += P_k


def test_layouts_agree_bit_for_bit_and_with_the_oracle(dv, batch):
    probs, refs = batch
    out = [run(dv, probs, 1, layout) for layout in (0, 1, 2)]
    for costs, grads in out:
        check(probs, refs, costs, grads)
    for costs, grads in out[1:]:
        assert np.array_equal(costs, out[0][0])
        assert np.array_equal(grads, out[0][1])


@pytest.mark.parametrize("split", [2, 4, 8])
def test_amplitude_splits_match_the_oracle(dv, batch, split):
    probs, refs = batch
    check(probs, refs, *run(dv, probs, split, 0))


def test_tuned_layout_with_a_fixed_split_and_reset(dv, batch):
    probs, refs = batch
    check(probs, refs, *run(dv, probs, 0, 2))   # layout fixed, split tuned
    check(probs, refs, *run(dv, probs, 4, -1))  # split fixed, default layout
    check(probs, refs, *run(dv, probs, 0, -1))  # both tuned


def test_set_tuning_rejects_bad_values(dv):
    ctx = dv.dvqls_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        for split, layout in ((3, 0), (16, 0), (-1, 0), (1, 3), (1, -2)):
            with pytest.raises(dv.DvqlsError) as e:
                dv.dvqls_set_tuning(ctx, split, layout)
            assert e.value.code == dv.DVQLS_ERR_INVALID_ARG
    finally:
        dv.dvqls_destroy(ctx)
