"""States streamed through HBM (n > 12) vs the oracle: full parity at
n = 13..16, 18 and 19, and sampled outputs / size-independent identities at
n = 20."""
import numpy as np
import pytest
import torch

from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl

from test_gpu_terms import TOL32, TOL64, check, gpu_cost_grad, random_problem, cvec, dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("n,d,L", [(13, 1, 9), (14, 1, 66), (16, 0, 5)])
def test_hbm_states_match_definition(dv, ctx, prec, n, d, L):
    rng = np.random.default_rng(700 + n + L)
    coef, xs, zs, b = random_problem(rng, n, L)
    alpha = wl.random_angles(n * (d + 1), 800 + n)
    ref = oterms.cost_grad(n, d, alpha, b, coef, xs, zs)
    check(gpu_cost_grad(dv, ctx, n, d, alpha, b, coef, xs, zs, prec), ref, prec)


_REG_CASES = {}


@pytest.mark.parametrize("n", [18, 19])
@pytest.mark.parametrize("prec", [1, 2])
def test_hbm_states_register_passes(dv, ctx, prec, n):
    """n = 18, 19: the FP32 high-qubit pass keeps its tiles in registers (as at
    n = 20); full parity against the oracle with one ansatz layer."""
    if n not in _REG_CASES:  # the oracle takes tens of seconds here: once per size
        rng = np.random.default_rng(710 + n)
        coef, xs, zs, b = random_problem(rng, n, 5)
        alpha = wl.random_angles(n * 2, 810 + n)
        _REG_CASES[n] = (coef, xs, zs, b, alpha, oterms.cost_grad(n, 1, alpha, b, coef, xs, zs))
    coef, xs, zs, b, alpha, ref = _REG_CASES[n]
    check(gpu_cost_grad(dv, ctx, n, 1, alpha, b, coef, xs, zs, prec), ref, prec)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_mixed_batch_smem_and_hbm(dv, ctx, prec):
    rng = np.random.default_rng(11)
    probs = []
    for n, d, L in [(14, 1, 12), (6, 2, 20), (13, 2, 7), (10, 1, 64)]:
        coef, xs, zs, b = random_problem(rng, n, L)
        probs.append((n, d, L, wl.random_angles(n * (d + 1), int(rng.integers(1 << 30))), coef, xs, zs, b))
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
    dv.dvqls_cost_grad_batched(ctx, arr, prec, costs, grads)
    dv.dvqls_sync(ctx)
    off = 0
    tc = TOL64 if prec == 0 else TOL32["cost"]
    tg = TOL64 if prec == 0 else TOL32["grad"]
    for k, (n, d, L, alpha, coef, xs, zs, b) in enumerate(probs):
        ref = oterms.cost_grad(n, d, alpha, b, coef, xs, zs)
        assert abs(costs[k].item() - ref["cost"]) <= tc * max(1, abs(ref["cost"]))
        g = grads[off:off + n * (d + 1)].cpu().numpy()
        assert np.all(np.abs(g - ref["grad"]) <= tg * np.maximum(1, np.abs(ref["grad"])))
        off += n * (d + 1)


@pytest.mark.parametrize("prec", [1, 2])
def test_n20_sampled_terms_and_cost_identity(dv, ctx, prec):
    """n = 20 tridiagonal Toeplitz, top-64 terms, depth 2, FP32 (CUDA cores and
    tensor cores): sampled beta and delta against the oracle state, and
    C = 1 - |<b|A~psi>|^2 / ||A~psi||^2 (exact for any size)."""
    n, d = 20, 2
    inst = wl.throughput_instance(4, n=n, d=d)
    dec = odec.decompose_banded(n, inst["offsets"], inst["bands"], 0.0, 64)
    alpha = inst["alpha"]
    got = gpu_cost_grad(dv, ctx, n, d, alpha, inst["b"], dec["coef"], dec["x"], dec["z"], prec, grad=False)
    psi = oterms.ansatz_state(n, d, alpha)
    rng = np.random.default_rng(0)
    phis = {}

    def phi(l):
        if l not in phis:
            phis[l] = oterms.apply_pauli(dec["x"][l], dec["z"][l], psi)
        return phis[l]

    for l, m in rng.integers(0, 64, (6, 2)):
        assert abs(got["beta"][l, m] - np.vdot(phi(l), phi(m))) <= TOL32["beta"]
    for l in rng.integers(0, 64, 3):
        assert abs(got["delta"][l] - np.vdot(inst["b"], phi(l))) <= TOL32["delta"]
    Apsi = np.zeros_like(psi)
    for l in range(64):
        Apsi += dec["coef"][l] * oterms.apply_pauli(dec["x"][l], dec["z"][l], psi)
    cost = 1.0 - abs(np.vdot(inst["b"], Apsi)) ** 2 / np.vdot(Apsi, Apsi).real
    assert abs(got["cost"] - cost) <= TOL32["cost"]


@pytest.mark.parametrize("prec", [1, 2])
def test_n20_gradient_components(dv, ctx, prec):
    """Two gradient components at n = 20 against the shift rule evaluated on
    oracle states (the identity above gives each shifted cost)."""
    n, d = 20, 1
    inst = wl.throughput_instance(5, n=n, d=d)
    dec = odec.decompose_banded(n, inst["offsets"], inst["bands"], 0.0, 16)
    got = gpu_cost_grad(dv, ctx, n, d, inst["alpha"], inst["b"], dec["coef"], dec["x"], dec["z"], prec)

    def N_D(alpha):
        psi = oterms.ansatz_state(n, d, alpha)
        Apsi = np.zeros_like(psi)
        for c, x, z in zip(dec["coef"], dec["x"], dec["z"]):
            Apsi += c * oterms.apply_pauli(x, z, psi)
        return abs(np.vdot(inst["b"], Apsi)) ** 2, np.vdot(Apsi, Apsi).real

    N0, D0 = N_D(inst["alpha"])
    for k in (3, 27):
        e = np.zeros_like(inst["alpha"])
        e[k] = 0.5 * np.pi
        Np, Dp = N_D(inst["alpha"] + e)
        Nm, Dm = N_D(inst["alpha"] - e)
        g = -(0.5 * (Np - Nm) * D0 - N0 * 0.5 * (Dp - Dm)) / D0 ** 2
        assert abs(got["grad"][k] - g) <= TOL32["grad"]
