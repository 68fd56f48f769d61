"""Host-side facts the warm-start pipeline rests on, checked with the oracle
on the CPU: the |+> angles are a stationary point of the global cost (Eq. 1)
for a persymmetric system with b = |+>^n (so the FP64 runs start from a
perturbed |+>), and the perturbation moves them off it."""
import numpy as np
import pytest

from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import warmstart as W
from paper_2604_14435_gb300 import workloads as wl


@pytest.mark.parametrize("n,seed", [(3, 1), (4, 2), (5, 3)])
def test_plus_angles_are_stationary_and_plus_start_is_not(n, seed):
    inst = wl.throughput_instance(seed, n=n, d=W.DEPTH, L_max=64)
    dec = odec.decompose_banded(n, inst["offsets"], inst["bands"], 0.0, 64)
    args = (inst["b"], dec["coef"], dec["x"], dec["z"])
    assert all(bin(int(z)).count("1") % 2 == 0 for z in dec["z"])  # J sigma J = sigma: even Z/Y count
    at_plus = oterms.cost_grad(n, W.DEPTH, W.plus_init(n), *args)
    assert np.abs(at_plus["grad"]).max() <= 1e-13
    psi = oterms.ansatz_state(n, W.DEPTH, W.plus_init(n))
    assert np.allclose(psi, np.full(1 << n, 2.0 ** (-n / 2)), atol=1e-14)
    a0 = W.plus_start(n)
    assert np.abs(a0 - W.plus_init(n)).max() <= 0.05
    assert np.array_equal(a0, W.plus_start(n))  # the same perturbation every time
    assert np.abs(oterms.cost_grad(n, W.DEPTH, a0, *args)["grad"]).max() >= 1e-5
