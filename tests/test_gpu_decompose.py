"""GPU decomposition vs the oracle: masks, order, L counts and coefficients
bit-exact (Sec. 2.2, Eq. 5; Algorithm 1 Steps 1-2)."""
import numpy as np
import pytest
import torch

from oracle import decompose as odec
from paper_2604_14435_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def run_dense(dv, ctx, A, tau, L_max, device=True):
    n = int(round(np.log2(A.shape[0])))
    if device:
        Ad = torch.tensor(A, device="cuda", dtype=torch.float64)
        coef = torch.zeros(2 * L_max, device="cuda", dtype=torch.float64)
        xm = torch.zeros(L_max, device="cuda", dtype=torch.int32)
        zm = torch.zeros(L_max, device="cuda", dtype=torch.int32)
    else:
        Ad = np.ascontiguousarray(A, dtype=np.float64)
        coef = np.zeros(2 * L_max)
        xm = np.zeros(L_max, np.uint32)
        zm = np.zeros(L_max, np.uint32)
    L, Lpre, Lpost = dv.dvqls_pauli_decompose(ctx, Ad, n, tau, L_max, coef, xm, zm)
    c = (coef.cpu().numpy() if device else coef).view(np.complex128)[:L]
    x = (xm.cpu().numpy() if device else xm)[:L].astype(np.uint32)
    z = (zm.cpu().numpy() if device else zm)[:L].astype(np.uint32)
    return {"coef": c, "x": x, "z": z, "L_out": L, "L_pre": Lpre, "L_post": Lpost}


def run_banded(dv, ctx, n, offsets, bands, tau, L_max):
    coef = torch.zeros(2 * L_max, device="cuda", dtype=torch.float64)
    xm = torch.zeros(L_max, device="cuda", dtype=torch.int32)
    zm = torch.zeros(L_max, device="cuda", dtype=torch.int32)
    bv = torch.tensor(np.ascontiguousarray(bands), device="cuda", dtype=torch.float64)
    L, Lpre, Lpost = dv.dvqls_pauli_decompose_banded(ctx, n, offsets, bv, tau, L_max, coef, xm, zm)
    return {"coef": coef.cpu().numpy().view(np.complex128)[:L], "x": xm.cpu().numpy()[:L].astype(np.uint32),
            "z": zm.cpu().numpy()[:L].astype(np.uint32), "L_out": L, "L_pre": Lpre, "L_post": Lpost}


def same(got, ref):
    assert (got["L_out"], got["L_pre"], got["L_post"]) == (ref["L_out"], ref["L_pre"], ref["L_post"])
    assert np.array_equal(got["x"], ref["x"])
    assert np.array_equal(got["z"], ref["z"])
    # bit-exact: the float64 words themselves (a complex == would accept -0.0 for +0.0)
    g = np.ascontiguousarray(got["coef"]).view(np.uint64)
    r = np.ascontiguousarray(ref["coef"]).view(np.uint64)
    assert g.shape == r.shape and np.array_equal(g, r)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 9])
@pytest.mark.parametrize("sym", [True, False])
def test_dense_random(dv, ctx, n, sym):
    rng = np.random.default_rng(300 + n)
    A = rng.normal(size=(1 << n, 1 << n))
    if sym:
        A = A + A.T
    A[rng.random(A.shape) < 0.5] = 0.0
    L_max = min(1 << (2 * n), 2048)
    for tau in (0.0, 0.05, 0.3):
        same(run_dense(dv, ctx, A, tau, L_max), odec.decompose(A, tau, L_max))


def test_dense_host_pointers(dv, ctx):
    A = wl.validation_system()["A"]
    same(run_dense(dv, ctx, A, 0.0, 64, device=False), odec.decompose(A, 0.0, 64))


@pytest.mark.parametrize("n", [4, 10, 12])
def test_dense_toeplitz_ties(dv, ctx, n):
    """Equal magnitudes within each level: ties broken by (x << n) | z."""
    A = wl.toeplitz_dense(n, 1.0, -1.0 / 3.0)
    for tau, L_max in ((0.01, 64), (0.0, 100), (0.0, 1)):
        same(run_dense(dv, ctx, A, tau, L_max), odec.decompose(A, tau, L_max))


@pytest.mark.parametrize("n", [10, 13, 16, 20])
def test_banded_toeplitz(dv, ctx, n):
    for seed in range(2):
        inst = wl.throughput_instance(seed, n=n)
        g = run_banded(dv, ctx, n, inst["offsets"], inst["bands"], 0.01, 64)
        same(g, odec.decompose_banded(n, inst["offsets"], inst["bands"], 0.01, 64))


def test_banded_pentadiagonal_and_laplacian(dv, ctx):
    n = 12
    offsets, bands = wl.toeplitz_bands(n, [3.3, -0.9, 0.45])
    same(run_banded(dv, ctx, n, offsets, bands, 0.001, 512),
         odec.decompose_banded(n, offsets, bands, 0.001, 512))
    hs = wl.hele_shaw_pressure(0)
    same(run_dense(dv, ctx, hs["A"], 0.0, 256), odec.decompose(hs["A"], 0.0, 256))


def test_paper_pruning_levels(dv, ctx):
    """tau -> L of Sec. 3.2 on the GPU."""
    n = 10
    offsets, bands = wl.toeplitz_bands(n, [1.0, -1.0 / 3.0])
    for tau, L in zip([0.1, 0.05, 0.03, 0.02, 0.01, 0.005], [4, 8, 16, 32, 64, 128]):
        g = run_banded(dv, ctx, n, offsets, bands, tau, 2048)
        assert g["L_post"] == L and g["L_out"] == L and g["L_pre"] == 1024


def test_zero_matrix_and_errors(dv, ctx):
    g = run_dense(dv, ctx, np.zeros((8, 8)), 0.0, 8)
    assert (g["L_out"], g["L_pre"], g["L_post"]) == (0, 0, 0)
    with pytest.raises(dv.DvqlsError) as e:
        run_dense(dv, ctx, np.eye(8), 0.0, 0)
    assert e.value.code == dv.DVQLS_ERR_INVALID_ARG
    A = np.eye(8)
    A[1, 2] = np.nan
    with pytest.raises(dv.DvqlsError) as e:
        run_dense(dv, ctx, A, 0.0, 8)
    assert e.value.code == dv.DVQLS_ERR_INVALID_ARG
    # the context stays usable after an error
    same(run_dense(dv, ctx, np.eye(8), 0.0, 8), odec.decompose(np.eye(8), 0.0, 8))
