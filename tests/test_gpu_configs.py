"""The two larger workloads at their own sizes, against the FP64 oracle.

Hele-Shaw-type pressure system: a 32 x 32 variable-permeability 5-point
Laplacian (n = 10), top-256 Pauli terms, depth-6 ansatz (P = 70, S = 141
shifted states): every beta, delta, the cost and every gradient component
element by element, in FP64, FP32 and the tensor-core precision.

Uneven batch: 62 Toeplitz instances with n in {4, 6, 8, 10, 12} (tri- and
pentadiagonal, tau = 0.01, L <= 64, depth n/2) plus two tridiagonal n = 20
instances whose states live in HBM, all 64 in one dvqls_cost_grad_batched
call.  The 62 on-chip instances are compared with the oracle's cost and
whole gradient; each n = 20 instance with the size-independent identity
C = 1 - |<b|A~ psi>|^2 / ||A~ psi||^2 on oracle states and two gradient
components by the shift rule on oracle states (Eq. 1, Eq. 3; Sec. 2.3).

Tolerances: FP64 |gpu - oracle| <= 1e-12 max(1, |oracle|); FP32 paths
<= 1e-5 absolute on beta and delta, <= 1e-6 on the cost, <= 1e-5 on the
gradient."""
import numpy as np
import pytest
import torch

from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl

from test_gpu_terms import TOL32, TOL64, check, cvec, dev, gpu_cost_grad

pytestmark = pytest.mark.gpu

_CACHE = {}


def hele_shaw_case():
    if "hs" not in _CACHE:
        hs = wl.hele_shaw_pressure(0)
        dec = odec.decompose(hs["A"], 0.0, 256)
        ref = oterms.cost_grad(hs["n"], hs["d"], hs["alpha"], hs["b"], dec["coef"], dec["x"], dec["z"])
        _CACHE["hs"] = (hs, dec, ref)
    return _CACHE["hs"]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_hele_shaw_L256_depth6_all_shifts(dv, ctx, prec):
    hs, dec, ref = hele_shaw_case()
    n, d = hs["n"], hs["d"]
    assert (n, d, dec["L_out"]) == (10, 6, 256)
    got = gpu_cost_grad(dv, ctx, n, d, hs["alpha"], hs["b"], dec["coef"], dec["x"], dec["z"], prec)
    assert got["grad"].size == 70
    check(got, ref, prec)


def uneven_grad_angles(k, n, d):
    """The two gradient components checked on an n = 20 instance: one angle of
    the first layers and one of the last."""
    return (7 + k % 5, n * (d + 1) - 3)


def uneven_case():
    """Oracle values of the uneven batch, computed in a spawn pool (the 62
    on-chip evaluations and the ten n = 20 states take minutes serially)."""
    if "uneven" not in _CACHE:
        import multiprocessing as mp
        import os

        import oracle_workers as ow
        insts = wl.uneven_batch(seed=0)
        decs = [ow.uneven_decomposition(k)[1] for k in range(len(insts))]
        chip = [k for k, i in enumerate(insts) if i["n"] <= 12]
        big = [k for k, i in enumerate(insts) if i["n"] > 12]
        nd_jobs = [(k, 0, 0) for k in big]
        for k in big:
            for j in uneven_grad_angles(k, insts[k]["n"], insts[k]["d"]):
                nd_jobs += [(k, j, 1), (k, j, -1)]
        # one BLAS thread per worker process (the children read these when they import numpy)
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for v in saved:
            os.environ[v] = "1"
        try:
            pool = mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))
        finally:
            for v, x in saved.items():
                if x is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = x
        with pool:
            nd_async = pool.starmap_async(ow.uneven_n_d, nd_jobs, chunksize=1)
            # largest instances first so the pool's tail is short
            chip_sorted = sorted(chip, key=lambda k: -(insts[k]["n"] * 100 + insts[k]["d"]))
            chip_res = dict(zip(chip_sorted, pool.map(ow.uneven_cost_grad, chip_sorted, chunksize=1)))
            nd = dict(zip(nd_jobs, nd_async.get()))
        refs = []
        for k, inst in enumerate(insts):
            if k in chip_res:
                refs.append(chip_res[k])
                continue
            n, d = inst["n"], inst["d"]
            N0, D0 = nd[(k, 0, 0)]
            comps = {}
            for j in uneven_grad_angles(k, n, d):
                Np, Dp = nd[(k, j, 1)]
                Nm, Dm = nd[(k, j, -1)]
                comps[j] = -(0.5 * (Np - Nm) * D0 - N0 * 0.5 * (Dp - Dm)) / D0 ** 2
            refs.append({"cost": 1.0 - N0 / D0, "grad_at": comps})
        _CACHE["uneven"] = (insts, decs, refs)
    return _CACHE["uneven"]


@pytest.mark.parametrize("prec", [1, 2])
def test_uneven_batch_64_instances_one_call(dv, ctx, prec):
    insts, decs, refs = uneven_case()
    assert len(insts) == 64 and sum(i["n"] == 20 for i in insts) == 2
    keep, items = [], []
    for inst, dec in zip(insts, decs):
        L = dec["L_out"]
        t = (dev(cvec(dec["coef"])), dev(np.asarray(dec["x"], np.uint32).view(np.int32), torch.int32),
             dev(np.asarray(dec["z"], np.uint32).view(np.int32), torch.int32), dev(inst["alpha"]),
             dev(cvec(inst["b"])))
        keep.append(t)
        items.append((dv.make_ansatz(inst["n"], inst["d"]), dv.make_lcu(L, t[0], t[1], t[2]), t[3], t[4]))
    arr = dv.make_instances(items)
    P = sum(i["n"] * (i["d"] + 1) for i in insts)
    costs = torch.zeros(len(insts), device="cuda", dtype=torch.float64)
    grads = torch.zeros(P, device="cuda", dtype=torch.float64)
    dv.dvqls_cost_grad_batched(ctx, arr, prec, costs, grads)
    dv.dvqls_sync(ctx)
    c = costs.cpu().numpy()
    g = grads.cpu().numpy()
    off = 0
    for k, (inst, ref) in enumerate(zip(insts, refs)):
        Pk = inst["n"] * (inst["d"] + 1)
        assert abs(c[k] - ref["cost"]) <= TOL32["cost"], (k, inst["n"], c[k], ref["cost"])
        if "grad" in ref:
            assert np.abs(g[off:off + Pk] - ref["grad"]).max() <= TOL32["grad"], (k, inst["n"])
        else:
            for j, v in ref["grad_at"].items():
                assert abs(g[off + j] - v) <= TOL32["grad"], (k, j, g[off + j], v)
                # these gradients are ~1e-6 (random angles leave psi nearly orthogonal to |+>^20),
                # so the absolute bound alone would not see a wrong value: relative agreement too
                assert abs(g[off + j] - v) <= 0.05 * abs(v) + 1e-9, (k, j, g[off + j], v)
        off += Pk
