"""Failure detection on the GPU without a fault: the bounded waits of the
tensor-core term kernel.

The kernel's warp roles hand work to each other through shared-memory
barriers, and every wait gives up after the context's time budget.  With a
budget of one microsecond the waits run out (nothing the kernel waits for
can be ready that soon), the kernel stops cleanly and the call returns
DVQLS_ERR_TIMEOUT; with the default budget restored, the same context then
passes the parity check against the oracle.  Nothing here traps, faults or
hangs the GPU: a wait that runs out is an ordinary branch of the kernel."""
import numpy as np
import pytest

from oracle import decompose as odec
from oracle import terms as oterms
from paper_2604_14435_gb300 import workloads as wl

from test_gpu_terms import check, gpu_cost_grad

pytestmark = pytest.mark.gpu


def test_wait_budget_times_out_then_context_recovers(dv, ctx):
    inst = wl.throughput_instance(3)
    n, d = inst["n"], inst["d"]
    dec = odec.decompose_banded(n, inst["offsets"], inst["bands"], 0.0, 64)
    args = (n, d, inst["alpha"], inst["b"], dec["coef"], dec["x"], dec["z"])
    dv.dvqls_set_wait_budget(ctx, 1)
    try:
        for _ in range(2):  # the context's graph and status word survive repeated timeouts
            with pytest.raises(dv.DvqlsError) as e:
                gpu_cost_grad(dv, ctx, *args, dv.DVQLS_FP32_TC)
            assert e.value.code == dv.DVQLS_ERR_TIMEOUT, e.value
    finally:
        dv.dvqls_set_wait_budget(ctx, 0)
    ref = oterms.cost_grad(*args)
    check(gpu_cost_grad(dv, ctx, *args, dv.DVQLS_FP32_TC), ref, dv.DVQLS_FP32_TC)
    # the other precisions do not use the budget and are unaffected
    check(gpu_cost_grad(dv, ctx, *args, dv.DVQLS_FP32), ref, dv.DVQLS_FP32)


def test_wait_budget_rejects_null_context(dv):
    assert dv.lib().dvqls_set_wait_budget(None, 5) == dv.DVQLS_ERR_INVALID_ARG
