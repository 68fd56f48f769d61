"""Oracle jobs for the GPU tests of the larger workloads, run in a process
pool (spawn) so that their CPU time overlaps.  Imports only numpy, the
oracle and the input generators."""
import numpy as np

from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl


def uneven_decomposition(k, seed=0):
    inst = wl.uneven_batch(seed=seed)[k]
    return inst, odec.decompose_banded(inst["n"], inst["offsets"], inst["bands"], inst["tau"], inst["L_max"])


def uneven_cost_grad(k):
    """Cost and whole gradient of on-chip instance k of the uneven batch."""
    inst, dec = uneven_decomposition(k)
    return oterms.cost_grad(inst["n"], inst["d"], inst["alpha"], inst["b"], dec["coef"], dec["x"], dec["z"])


def uneven_n_d(k, j, sign):
    """N = |<b|A~ psi>|^2 and D = ||A~ psi||^2 on the oracle state of instance k,
    with angle j shifted by sign * pi/2 (sign 0: unshifted)."""
    inst, dec = uneven_decomposition(k)
    alpha = inst["alpha"].copy()
    if sign:
        alpha[j] += sign * 0.5 * np.pi
    psi = oterms.ansatz_state(inst["n"], inst["d"], alpha)
    Apsi = np.zeros_like(psi)
    for c, x, z in zip(dec["coef"], dec["x"], dec["z"]):
        Apsi += c * oterms.apply_pauli(x, z, psi)
    return abs(np.vdot(inst["b"], Apsi)) ** 2, np.vdot(Apsi, Apsi).real
