"""Walsh-Hadamard term classes (DVQLS_FP32_WHT): the per-instance class table
is kept between calls while its inputs (L, masks, coefficients) and its
checksum are unchanged.  Every reuse path is checked against the oracle."""
import numpy as np
import pytest
import torch

from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl

from test_gpu_terms import check, gpu_cost_grad, random_problem

pytestmark = pytest.mark.gpu


def run(dv, ctx, prob, prec=3):
    n, d, alpha, b, coef, xs, zs = prob
    ref = oterms.cost_grad(n, d, alpha, b, coef, xs, zs)
    check(gpu_cost_grad(dv, ctx, n, d, alpha, b, coef, xs, zs, prec), ref, prec)


def test_class_table_reuse_and_invalidation(dv, ctx):
    rng = np.random.default_rng(2024)
    n, d, L = 8, 2, 40
    coef, xs, zs, b = random_problem(rng, n, L)
    alpha = wl.random_angles(n * (d + 1), 31)
    p1 = (n, d, alpha, b, coef, xs, zs)
    run(dv, ctx, p1)  # builds the table
    run(dv, ctx, p1)  # reuses it
    # a call with another plan writes over the workspace in between
    big = random_problem(rng, 10, 70)
    run(dv, ctx, (10, 1, wl.random_angles(20, 5), big[3], big[0], big[1], big[2]), prec=1)
    run(dv, ctx, p1)  # the checksum catches any overwritten word
    # same masks, new coefficients: the table (signed weights) must be rebuilt
    coef2 = coef * (1.0 + 0.5j) + 0.25
    run(dv, ctx, (n, d, alpha, b, coef2, xs, zs))
    # one mask changed
    xs3 = xs.copy()
    xs3[7] ^= 5
    run(dv, ctx, (n, d, alpha, b, coef2, xs3, zs))
    # the unshifted beta and delta outputs on a reused table
    run(dv, ctx, (n, d, alpha, b, coef2, xs3, zs))


@pytest.mark.parametrize("n,L", [(1, 1), (3, 8), (5, 33), (10, 64)])
def test_toeplitz_and_small_systems(dv, ctx, n, L):
    """Banded (few classes) and tiny systems (n < 5: lanes repeat the vector)."""
    rng = np.random.default_rng(77 + n)
    if n >= 3:
        inst = wl.throughput_instance(3, n=n, d=2, L_max=L)
        dec = odec.decompose_banded(n, inst["offsets"], inst["bands"], 0.0, L)
        p = (n, 2, inst["alpha"], inst["b"], dec["coef"], dec["x"], dec["z"])
    else:
        coef, xs, zs, b = random_problem(rng, n, L)
        p = (n, 2, wl.random_angles(3 * n, 9), b, coef, xs, zs)
    run(dv, ctx, p)
