"""One instance split across two `gloo` ranks on CPU (Sec. 2.3 Stage III;
Algorithm 1, Step 4c).

The library calls are replaced by oracle-backed stand-ins with the same
conventions: a rank's per-shift sums (T_g, D_g) come from the definition-
level oracle for its shifts, zeros elsewhere.  The test checks the host
logic of the split -- disjoint ranges that cover every shift, one SUM
allreduce, N_g = |T_g|^2 formed after it -- by comparing the reduced cost
and gradient on every rank with the oracle's whole evaluation."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import terms as oterms
from paper_2604_14435_gb300 import stage3
from paper_2604_14435_gb300 import workloads as wl


class Ansatz:
    def __init__(self, n, depth):
        self.n, self.depth = n, depth


def problem(seed=7, n=4, d=2, L=9):
    rng = np.random.default_rng(seed)
    N = 1 << n
    coef = rng.normal(size=L) + 1j * rng.normal(size=L)
    xs = rng.integers(0, N, L).astype(np.uint32)
    zs = rng.integers(0, N, L).astype(np.uint32)
    b = rng.normal(size=N) + 1j * rng.normal(size=N)
    b /= np.linalg.norm(b)  # the library normalises b; the oracle takes it as given
    alpha = wl.random_angles(n * (d + 1), seed + 1)
    return n, d, alpha, b, coef, xs, zs


class OracleLib:
    """dvqls_cost_grad_partials and dvqls_combine_partials by the oracle."""

    def __init__(self, prob):
        self.prob = prob
        self.calls = []

    def dvqls_cost_grad_partials(self, ctx, ansatz, alpha, lcu, b, precision, s0, s1, part):
        n, d, alpha, b, coef, xs, zs = self.prob
        self.calls.append((s0, s1))
        shifts = oterms.shifted_angles(alpha)
        bn = b / np.linalg.norm(b)
        out = np.zeros((shifts.shape[0], 4))
        for g in range(s0, s1):
            beta, delta = oterms.beta_delta(oterms.ansatz_state(n, d, shifts[g]), bn, xs, zs)
            T = np.sum(coef * delta)
            D = np.conj(coef) @ beta @ coef
            out[g] = (T.real, T.imag, D.real, D.imag)
        part.copy_(torch.from_numpy(out.ravel()))

    def dvqls_combine_partials(self, ctx, n, depth, part, cost, grad):
        p = part.numpy().reshape(-1, 4)
        Ns = p[:, 0] ** 2 + p[:, 1] ** 2
        Ds = p[:, 2]
        cost[0] = 1.0 - Ns[0] / Ds[0]
        dN = 0.5 * (Ns[1::2] - Ns[2::2])
        dD = 0.5 * (Ds[1::2] - Ds[2::2])
        grad.copy_(torch.from_numpy(-(dN * Ds[0] - Ns[0] * dD) / Ds[0] ** 2))


def test_shift_ranges_cover_disjoint_and_balanced():
    for S in (1, 2, 19, 101, 441):
        for ws in (1, 2, 3, 4, 8, 500):
            rs = stage3.shift_ranges(S, ws)
            assert len(rs) == ws
            assert rs[0][0] == 0 and rs[-1][1] == S
            for (a0, a1), (b0, b1) in zip(rs, rs[1:]):
                assert a1 == b0 and a0 <= a1
            sizes = [r[1] - r[0] for r in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        stage3.shift_ranges(0, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = problem()
        lib = OracleLib(prob)
        n, d = prob[0], prob[1]
        cost, grad = stage3.cost_grad_split(lib, None, Ansatz(n, d), None, None, None, 0, dist, torch, "cpu")
        out.put((rank, lib.calls, float(cost[0]), grad.numpy().copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_split_one_instance(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted([q.get(timeout=180) for _ in range(world)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n, d, alpha, b, coef, xs, zs = problem()
    ref = oterms.cost_grad(n, d, alpha, b, coef, xs, zs)
    S = 2 * n * (d + 1) + 1
    covered = sorted(c for r in results for c in r[1])
    assert covered == stage3.shift_ranges(S, world)  # each rank evaluated exactly its own range
    for _, _, cost, grad in results:  # every rank holds the whole instance's result
        assert abs(cost - ref["cost"]) <= 1e-12 * max(1.0, abs(ref["cost"]))
        assert np.all(np.abs(grad - ref["grad"]) <= 1e-12 * np.maximum(1.0, np.abs(ref["grad"])))
