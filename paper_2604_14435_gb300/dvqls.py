"""Thin ctypes binding of libdvqls.so (include/dvqls.h): argument marshalling only.

Every function keeps the C name and order of arguments; array arguments may
be numpy arrays (host memory) or torch tensors (host or CUDA memory of the
context's device).  Nothing here computes any part of the method: a missing
library is an error, never a fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdvqls.so")

DVQLS_OK = 0
DVQLS_ERR_INVALID_ARG = 1
DVQLS_ERR_UNSUPPORTED = 2
DVQLS_ERR_CUDA = 3
DVQLS_ERR_TIMEOUT = 4
DVQLS_ERR_NUMERIC = 5
DVQLS_ERR_ALLOC = 6
DVQLS_FP64 = 0
DVQLS_FP32 = 1
DVQLS_FP32_TC = 2
DVQLS_FP32_WHT = 3
DVQLS_ANSATZ_RY_CZRING = 0
DVQLS_MAX_SMEM_QUBITS = 12
DVQLS_MAX_QUBITS = 20
DVQLS_MAX_DENSE_QUBITS = 12

EXPORTED = [
    "dvqls_create", "dvqls_destroy", "dvqls_last_error", "dvqls_sync",
    "dvqls_pauli_decompose", "dvqls_pauli_decompose_banded",
    "dvqls_cost", "dvqls_cost_grad", "dvqls_cost_grad_batched",
    "dvqls_profile_enable", "dvqls_profile_read", "dvqls_set_wait_budget", "dvqls_set_tuning",
    "dvqls_cost_grad_noalloc",
    "dvqls_circuit_cost_grad_fp64", "dvqls_fidelity", "dvqls_lcu_solve", "dvqls_lcu_solve_batched",
    "dvqls_optimize", "dvqls_optimize_resume",
    "dvqls_ws_param_count", "dvqls_ws_create", "dvqls_ws_destroy", "dvqls_ws_infer", "dvqls_ws_grad",
    "dvqls_ws_train_step", "dvqls_ws_get_params", "dvqls_ws_save", "dvqls_ws_load",
    "dvqls_local_cost_grad", "dvqls_local_cost_grad_batched",
    "dvqls_cost_grad_partials", "dvqls_combine_partials",
]


class DvqlsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("dvqls status %d: %s" % (code, msg))
        self.code = code


class dvqls_ansatz(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("depth", ctypes.c_int), ("kind", ctypes.c_int)]


class dvqls_lcu(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("coef", ctypes.c_void_p), ("xmask", ctypes.c_void_p),
                ("zmask", ctypes.c_void_p)]


class dvqls_instance(ctypes.Structure):
    _fields_ = [("ansatz", dvqls_ansatz), ("lcu", dvqls_lcu), ("alpha", ctypes.c_void_p),
                ("b", ctypes.c_void_p)]


class dvqls_adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("max_iter", ctypes.c_int), ("target_fidelity", ctypes.c_double),
                ("precision", ctypes.c_int), ("targets", ctypes.c_void_p)]


class dvqls_adam_state(ctypes.Structure):
    _fields_ = [("m", ctypes.c_void_p), ("v", ctypes.c_void_p), ("steps", ctypes.c_void_p)]


class dvqls_opt_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("cost", ctypes.c_double),
                ("fidelity", ctypes.c_double)]


_lib = None


def lib():
    """Open libdvqls.so (built by paper_2604_14435_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libdvqls.so is not built (run __graft_entry__.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p
        L.dvqls_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, vp]
        L.dvqls_destroy.argtypes = [vp]
        L.dvqls_destroy.restype = None
        L.dvqls_last_error.argtypes = [vp]
        L.dvqls_last_error.restype = ctypes.c_char_p
        L.dvqls_sync.argtypes = [vp]
        L.dvqls_pauli_decompose.argtypes = [vp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                            dp, vp, vp, ip, ip, ip]
        L.dvqls_pauli_decompose_banded.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, dp, ctypes.c_double,
                                                   ctypes.c_int, dp, vp, vp, ip, ip, ip]
        L.dvqls_cost.argtypes = [vp, ctypes.POINTER(dvqls_ansatz), dp, ctypes.POINTER(dvqls_lcu), dp,
                                 ctypes.c_int, dp, dp, dp]
        L.dvqls_cost_grad.argtypes = [vp, ctypes.POINTER(dvqls_ansatz), dp, ctypes.POINTER(dvqls_lcu), dp,
                                      ctypes.c_int, dp, dp, dp, dp]
        L.dvqls_cost_grad_batched.argtypes = [vp, ctypes.c_int, ctypes.POINTER(dvqls_instance), ctypes.c_int,
                                              dp, dp]
        L.dvqls_profile_enable.argtypes = [vp, ctypes.c_int]
        L.dvqls_set_wait_budget.argtypes = [vp, ctypes.c_longlong]
        L.dvqls_set_tuning.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.dvqls_profile_read.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(ctypes.c_double)]
        L.dvqls_cost_grad_noalloc.argtypes = [vp, ctypes.POINTER(dvqls_ansatz), dp, ctypes.POINTER(dvqls_lcu), dp,
                                              ctypes.c_int, dp, dp]
        L.dvqls_circuit_cost_grad_fp64.argtypes = [vp, ctypes.POINTER(dvqls_ansatz), dp, ctypes.POINTER(dvqls_lcu),
                                                   dp, dp, dp, dp, dp]
        L.dvqls_fidelity.argtypes = [vp, ctypes.POINTER(dvqls_ansatz), dp, dp, dp]
        L.dvqls_lcu_solve.argtypes = [vp, ctypes.c_int, ctypes.POINTER(dvqls_lcu), dp, ctypes.c_double, ctypes.c_int,
                                      dp, ip, ctypes.POINTER(ctypes.c_double)]
        L.dvqls_lcu_solve_batched.argtypes = [vp, ctypes.c_int, ctypes.POINTER(dvqls_lcu), ctypes.c_int, dp,
                                              ctypes.c_double, ctypes.c_int, dp, vp, dp]
        L.dvqls_optimize.argtypes = [vp, ctypes.c_int, ctypes.POINTER(dvqls_instance), dp, ctypes.POINTER(dvqls_adam),
                                     dp, ctypes.POINTER(dvqls_opt_result)]
        L.dvqls_optimize_resume.argtypes = [vp, ctypes.c_int, ctypes.POINTER(dvqls_instance), dp,
                                            ctypes.POINTER(dvqls_adam), ctypes.POINTER(dvqls_adam_state), dp,
                                            ctypes.POINTER(dvqls_opt_result)]
        L.dvqls_ws_param_count.argtypes = [ctypes.c_int] * 3
        L.dvqls_ws_param_count.restype = ctypes.c_longlong
        L.dvqls_ws_create.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_void_p)]
        L.dvqls_ws_destroy.argtypes = [vp]
        L.dvqls_ws_destroy.restype = None
        L.dvqls_ws_infer.argtypes = [vp, ctypes.c_int, vp, vp]
        L.dvqls_ws_grad.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.POINTER(ctypes.c_float), vp]
        L.dvqls_ws_train_step.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]
        L.dvqls_ws_get_params.argtypes = [vp, vp]
        L.dvqls_ws_save.argtypes = [vp, ctypes.c_char_p]
        L.dvqls_ws_load.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
        L.dvqls_local_cost_grad.argtypes = [vp, ctypes.POINTER(dvqls_ansatz), dp, ctypes.POINTER(dvqls_lcu),
                                            ctypes.c_int, dp, dp]
        L.dvqls_local_cost_grad_batched.argtypes = [vp, ctypes.c_int, ctypes.POINTER(dvqls_instance), ctypes.c_int,
                                                    dp, dp]
        L.dvqls_cost_grad_partials.argtypes = [vp, ctypes.POINTER(dvqls_ansatz), dp, ctypes.POINTER(dvqls_lcu), dp,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.dvqls_combine_partials.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        _lib = L
    return _lib


def ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL).  Only the
    address crosses the ABI, so the array must be dense (C-contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr() or None
    if isinstance(a, np.ndarray):
        return a.ctypes.data or None
    raise TypeError("expected a numpy array or a torch tensor, got %r" % type(a))


def _check(ctx, code):
    if code != DVQLS_OK:
        msg = lib().dvqls_last_error(ctx).decode() if ctx else ""
        raise DvqlsError(code, msg)


def dvqls_create(device=0, stream=None):
    """Returns the context handle.  stream: a cudaStream_t as int (or None)."""
    h = ctypes.c_void_p()
    _check(None, lib().dvqls_create(ctypes.byref(h), int(device), stream))
    return h


def dvqls_destroy(ctx):
    lib().dvqls_destroy(ctx)


def dvqls_last_error(ctx):
    return lib().dvqls_last_error(ctx).decode()


def dvqls_sync(ctx):
    _check(ctx, lib().dvqls_sync(ctx))


def _ints():
    return ctypes.c_int(), ctypes.c_int(), ctypes.c_int()


def dvqls_pauli_decompose(ctx, A, n, tau, L_max, coef, xmask, zmask):
    """Returns (L_out, L_pre, L_post); coef/xmask/zmask are filled in place."""
    a, b, c = _ints()
    _check(ctx, lib().dvqls_pauli_decompose(ctx, ptr(A), int(n), float(tau), int(L_max), ptr(coef), ptr(xmask),
                                            ptr(zmask), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def dvqls_pauli_decompose_banded(ctx, n, offsets, band_values, tau, L_max, coef, xmask, zmask):
    offs = np.ascontiguousarray(offsets, dtype=np.int32)
    a, b, c = _ints()
    _check(ctx, lib().dvqls_pauli_decompose_banded(ctx, int(n), offs.size, ptr(offs), ptr(band_values),
                                                   float(tau), int(L_max), ptr(coef), ptr(xmask), ptr(zmask),
                                                   ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def make_ansatz(n, depth, kind=DVQLS_ANSATZ_RY_CZRING):
    return dvqls_ansatz(int(n), int(depth), int(kind))


def make_lcu(L, coef, xmask, zmask):
    return dvqls_lcu(int(L), ptr(coef), ptr(xmask), ptr(zmask))


def dvqls_cost(ctx, ansatz, alpha, lcu, b, precision, cost, beta=None, delta=None):
    _check(ctx, lib().dvqls_cost(ctx, ctypes.byref(ansatz), ptr(alpha), ctypes.byref(lcu), ptr(b), int(precision),
                                 ptr(cost), ptr(beta), ptr(delta)))


def dvqls_cost_grad(ctx, ansatz, alpha, lcu, b, precision, cost, grad, beta=None, delta=None):
    _check(ctx, lib().dvqls_cost_grad(ctx, ctypes.byref(ansatz), ptr(alpha), ctypes.byref(lcu), ptr(b),
                                      int(precision), ptr(cost), ptr(grad), ptr(beta), ptr(delta)))


def make_instances(items):
    """items: sequence of (ansatz, lcu, alpha, b) -> ctypes array of dvqls_instance."""
    arr = (dvqls_instance * len(items))()
    for k, (an, lc, al, bb) in enumerate(items):
        arr[k].ansatz = an
        arr[k].lcu = lc
        arr[k].alpha = ptr(al)
        arr[k].b = ptr(bb)
    return arr


def dvqls_cost_grad_batched(ctx, instances, precision, costs, grads):
    _check(ctx, lib().dvqls_cost_grad_batched(ctx, len(instances), instances, int(precision), ptr(costs),
                                              ptr(grads)))


def dvqls_profile_enable(ctx, enable):
    _check(ctx, lib().dvqls_profile_enable(ctx, int(enable)))


def dvqls_set_wait_budget(ctx, microseconds):
    """Time limit of each bounded device wait of the tensor-core term kernel."""
    _check(ctx, lib().dvqls_set_wait_budget(ctx, int(microseconds)))


def dvqls_set_tuning(ctx, split, layout=-1):
    """Fix the amplitude split (0: tune) and the tensor-core state layout (-1: tune)."""
    _check(ctx, lib().dvqls_set_tuning(ctx, int(split), int(layout)))


def dvqls_profile_read(ctx, phase):
    """Returns (launches, total milliseconds) of one kernel phase."""
    n, ms = ctypes.c_longlong(), ctypes.c_double()
    _check(ctx, lib().dvqls_profile_read(ctx, int(phase), ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def dvqls_cost_grad_noalloc(stream, ansatz, alpha, lcu, b, precision, cost, grad):
    """Allocation-free cost + gradient (device buffers only).  Returns the
    status code instead of raising, since there is no context to describe it."""
    return lib().dvqls_cost_grad_noalloc(stream, ctypes.byref(ansatz), ptr(alpha), ctypes.byref(lcu), ptr(b),
                                         int(precision), ptr(cost), ptr(grad))


def dvqls_circuit_cost_grad_fp64(ctx, ansatz, alpha, lcu, b, cost, grad, beta=None, delta=None):
    _check(ctx, lib().dvqls_circuit_cost_grad_fp64(ctx, ctypes.byref(ansatz), ptr(alpha), ctypes.byref(lcu), ptr(b),
                                                   ptr(cost), ptr(grad), ptr(beta), ptr(delta)))


def dvqls_fidelity(ctx, ansatz, alpha, xhat, F):
    _check(ctx, lib().dvqls_fidelity(ctx, ctypes.byref(ansatz), ptr(alpha), ptr(xhat), ptr(F)))


def dvqls_lcu_solve(ctx, n, lcu, b, tol, max_iter, x):
    """Returns (iterations, relative residual)."""
    it, rr = ctypes.c_int(), ctypes.c_double()
    _check(ctx, lib().dvqls_lcu_solve(ctx, int(n), ctypes.byref(lcu), ptr(b), float(tol), int(max_iter), ptr(x),
                                      ctypes.byref(it), ctypes.byref(rr)))
    return it.value, rr.value


def dvqls_lcu_solve_batched(ctx, n, lcu, nrhs, b, tol, max_iter, x):
    """b, x: nrhs x 2^n complex128 as float64 (packed).  Returns (iterations,
    relative residuals), one per right-hand side."""
    it = np.zeros(int(nrhs), np.int32)
    rr = np.zeros(int(nrhs), np.float64)
    _check(ctx, lib().dvqls_lcu_solve_batched(ctx, int(n), ctypes.byref(lcu), int(nrhs), ptr(b), float(tol),
                                              int(max_iter), ptr(x), ptr(it), ptr(rr)))
    return it, rr


def make_adam(lr=0.02, beta1=0.9, beta2=0.999, eps=1e-8, max_iter=5000, target_fidelity=0.9999,
              precision=DVQLS_FP64, targets=None):
    """targets: optional float64 numpy array, one fidelity target per instance
    (keep it alive for the call)."""
    return dvqls_adam(lr, beta1, beta2, eps, int(max_iter), target_fidelity, int(precision), ptr(targets))


def dvqls_optimize(ctx, instances, xhat, opt, alpha_out):
    """Returns a list of dvqls_opt_result, one per instance."""
    res = (dvqls_opt_result * len(instances))()
    _check(ctx, lib().dvqls_optimize(ctx, len(instances), instances, ptr(xhat), ctypes.byref(opt), ptr(alpha_out),
                                     res))
    return list(res)


def dvqls_optimize_resume(ctx, instances, xhat, opt, m, v, steps, alpha_out):
    """dvqls_optimize from the Adam state (m, v: packed angle-sized arrays;
    steps: int64 per instance), which is updated in place.  Returns the
    per-instance results."""
    res = (dvqls_opt_result * len(instances))()
    st = dvqls_adam_state(ptr(m), ptr(v), ptr(steps))
    _check(ctx, lib().dvqls_optimize_resume(ctx, len(instances), instances, ptr(xhat), ctypes.byref(opt),
                                            ctypes.byref(st), ptr(alpha_out), res))
    return list(res)


# -------------------------------------------------------------- warm start
# A dvqls_ws handle is paired with its context so errors can be described.


class WarmStart:
    """Handle of a dvqls_ws network (ctx, ws pointer, dimensions)."""

    def __init__(self, ctx, handle, I, H, O):
        self.ctx, self.handle, self.I, self.H, self.O = ctx, handle, I, H, O


def dvqls_ws_param_count(I, H, O):
    return lib().dvqls_ws_param_count(int(I), int(H), int(O))


def dvqls_ws_create(ctx, I, H, O, params):
    h = ctypes.c_void_p()
    _check(ctx, lib().dvqls_ws_create(ctx, int(I), int(H), int(O), ptr(params), ctypes.byref(h)))
    return WarmStart(ctx, h, I, H, O)


def dvqls_ws_destroy(ws):
    lib().dvqls_ws_destroy(ws.handle)


def dvqls_ws_infer(ws, batch, feats, out):
    _check(ws.ctx, lib().dvqls_ws_infer(ws.handle, int(batch), ptr(feats), ptr(out)))


def dvqls_ws_grad(ws, batch, feats, target, mask, grad):
    loss = ctypes.c_float()
    _check(ws.ctx, lib().dvqls_ws_grad(ws.handle, int(batch), ptr(feats), ptr(target), ptr(mask), ctypes.byref(loss),
                                       ptr(grad)))
    return loss.value


def dvqls_ws_train_step(ws, batch, feats, target, mask, lr, want_loss=True):
    loss = ctypes.c_float()
    _check(ws.ctx, lib().dvqls_ws_train_step(ws.handle, int(batch), ptr(feats), ptr(target), ptr(mask), float(lr),
                                             ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def dvqls_ws_get_params(ws, params):
    _check(ws.ctx, lib().dvqls_ws_get_params(ws.handle, ptr(params)))


def dvqls_ws_save(ws, path):
    _check(ws.ctx, lib().dvqls_ws_save(ws.handle, str(path).encode()))


def dvqls_ws_load(ctx, path):
    h = ctypes.c_void_p()
    _check(ctx, lib().dvqls_ws_load(ctx, str(path).encode(), ctypes.byref(h)))
    with open(path, "rb") as f:
        f.read(8)
        I, H, O = np.frombuffer(f.read(12), dtype=np.int32)
    return WarmStart(ctx, h, int(I), int(H), int(O))


def dvqls_local_cost_grad(ctx, ansatz, alpha, lcu, precision, cost, grad=None):
    _check(ctx, lib().dvqls_local_cost_grad(ctx, ctypes.byref(ansatz), ptr(alpha), ctypes.byref(lcu),
                                            int(precision), ptr(cost), ptr(grad)))


def dvqls_local_cost_grad_batched(ctx, instances, precision, costs, grads):
    _check(ctx, lib().dvqls_local_cost_grad_batched(ctx, len(instances), instances, int(precision), ptr(costs),
                                                    ptr(grads)))


def dvqls_cost_grad_partials(ctx, ansatz, alpha, lcu, b, precision, s_begin, s_end, partials):
    """Per-shift sums (Re T, Im T, Re D, Im D) of the shifts s_begin .. s_end - 1
    of one instance into partials ((2P+1) x 4 doubles; zeros elsewhere)."""
    _check(ctx, lib().dvqls_cost_grad_partials(ctx, ctypes.byref(ansatz), ptr(alpha), ctypes.byref(lcu), ptr(b),
                                               int(precision), int(s_begin), int(s_end), ptr(partials)))


def dvqls_combine_partials(ctx, n, depth, partials, cost, grad):
    """Cost and gradient of one instance from its summed per-shift sums."""
    _check(ctx, lib().dvqls_combine_partials(ctx, int(n), int(depth), ptr(partials), ptr(cost), ptr(grad)))
