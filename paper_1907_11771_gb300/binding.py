"""ctypes binding of libgbs.so: the C ABI of include/gbs.h under the same names.

Argument marshalling only -- every step of the computation runs in the CUDA
library.  Tensors are passed by ``data_ptr()``; the caller keeps them alive.
If the library has not been built (``__graft_entry__.build()`` or
``python -m paper_1907_11771_gb300.build``), every call raises: there is no CPU
fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbs.so")

GBS_OK = 0
STATUS_NAMES = {0: "GBS_OK", 1: "GBS_ERR_INVALID", 2: "GBS_ERR_ORDER", 3: "GBS_ERR_UNSTABLE",
                4: "GBS_ERR_CUDA", 5: "GBS_ERR_NOMEM", 6: "GBS_ERR_TIMEOUT", 7: "GBS_ERR_NONFINITE",
                8: "GBS_ERR_STATE"}
GBS_WAVE1D, GBS_ACOUSTIC, GBS_ONEWAY_SPECTRAL = 1, 2, 3
GBS_F32_STATE_F64_COMBINE, GBS_F64, GBS_F32X2 = 0, 1, 2
GBS_KERNEL_AUTO, GBS_KERNEL_PLAIN, GBS_KERNEL_FUSED = 0, 1, 2
GBS_MAX_SLOTS, GBS_MAX_SEQ, GBS_MAX_STEPS = 8, 16, 64


class GbsError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class gbs_problem(ctypes.Structure):
    _fields_ = [("system", ctypes.c_int), ("ndim", ctypes.c_int), ("fd_order", ctypes.c_int),
                ("precision", ctypes.c_int), ("batch", ctypes.c_int), ("enable_adjoint", ctypes.c_int),
                ("shape", ctypes.POINTER(ctypes.c_int64)), ("dx", ctypes.POINTER(ctypes.c_double))]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_I64 = ctypes.c_int64

_SIGS = {
    "gbs_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(gbs_problem), _I]),
    "gbs_state_elems": (ctypes.c_size_t, [ctypes.POINTER(gbs_problem)]),
    "gbs_create": (_I, [ctypes.POINTER(gbs_problem), _P, _P, _P, ctypes.POINTER(_P)]),
    "gbs_set_media": (_I, [_P, _P, _P]),
    "gbs_set_weights": (_I, [_P, _I, _I, _I, ctypes.POINTER(_I), _I, ctypes.POINTER(_I),
                             ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "gbs_get_weights": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D),
                             ctypes.POINTER(_D)]),
    "gbs_assign_slots": (_I, [_P, ctypes.POINTER(_I)]),
    "gbs_stability_limit": (_I, [_P, ctypes.POINTER(_D)]),
    "gbs_step": (_I, [_P, _P, _P, _D, _I]),
    "gbs_step_batch": (_I, [_P, _P, _P, ctypes.POINTER(_D), _I]),
    "gbs_step_partial": (_I, [_P, _P, _P, _D, ctypes.c_uint32]),
    "gbs_combine_partial": (_I, [_P, _P, _P, _P]),
    "gbs_step_host": (_I, [_P, _P, _P, _D, _I]),
    "gbs_step_host_stream": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _D, _I]),
    "gbs_adjoint_step": (_I, [_P, _P, _P, _P, _P, _D, _P, _I, _P]),
    "gbs_misfit": (_I, [_P, _P, _P, _I, _P, _P, _P]),
    "gbs_norms": (_I, [_P, _P, _P, ctypes.POINTER(_D)]),
    "gbs_inject": (_I, [_P, _P, _P, _I, _P]),
    "gbs_set_option": (_I, [_P, ctypes.c_char_p, _I64]),
    "gbs_get_option": (_I, [_P, ctypes.c_char_p, ctypes.POINTER(_I64)]),
    "gbs_kernel_time": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "gbs_sync": (_I, [_P]),
    "gbs_destroy": (_I, [_P]),
    "gbs_last_error": (ctypes.c_char_p, [_P]),
    "gbs_kernel_launches": (_I64, [_P]),
    "gbs_selftest_f32_to_f64": (_I, [ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    "gbs_step_noalloc": (_I, [ctypes.POINTER(gbs_problem), _P, _P, _I, _I, ctypes.POINTER(_I), _I,
                              ctypes.POINTER(_I), ctypes.POINTER(_D), _P, _P, _D, _I, _P]),
    "gbs_noalloc_last_error": (ctypes.c_char_p, []),
}


def lib():
    """Load libgbs.so (raises if it is missing: the CUDA library is required)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -m paper_1907_11771_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(x):
    """Device/host address of a tensor, numpy array or integer (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to the GBS library must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(h, status):
    if status != GBS_OK:
        msg = lib().gbs_last_error(h)
        raise GbsError(status, msg.decode() if msg else "")


def _arr(ctype, vals):
    vals = list(vals)
    return (ctype * max(1, len(vals)))(*vals)


def make_problem(system, ndim, fd_order, precision, shapes, dx, enable_adjoint=False):
    """Build a gbs_problem; shapes/dx are per-problem (nx, ny, nz) triples."""
    shapes = [tuple(int(v) for v in s) + (1,) * (3 - len(s)) for s in shapes]
    dx = [tuple(float(v) for v in d) + (1.0,) * (3 - len(d)) for d in dx]
    sh = _arr(ctypes.c_int64, [v for s in shapes for v in s])
    dd = _arr(ctypes.c_double, [v for d in dx for v in d])
    pb = gbs_problem(system, ndim, fd_order, precision, len(shapes), int(bool(enable_adjoint)),
                     ctypes.cast(sh, ctypes.POINTER(ctypes.c_int64)), ctypes.cast(dd, ctypes.POINTER(ctypes.c_double)))
    pb._keep = (sh, dd)
    return pb


# ---------------------------------------------------------------------------
# Entry points, same names as the C ABI
# ---------------------------------------------------------------------------

def gbs_workspace_bytes(pb, max_steps):
    return lib().gbs_workspace_bytes(ctypes.byref(pb), int(max_steps))


def gbs_state_elems(pb):
    return lib().gbs_state_elems(ctypes.byref(pb))


def gbs_create(pb, kappa=None, rho=None, stream=None):
    h = _P()
    st = lib().gbs_create(ctypes.byref(pb), _ptr(kappa), _ptr(rho), _ptr(stream), ctypes.byref(h))
    _check(None, st)
    return h.value


def gbs_set_media(h, kappa, rho):
    _check(h, lib().gbs_set_media(h, _ptr(kappa), _ptr(rho)))


def gbs_set_weights(h, slot, order, steps_dep, steps_free=(), c_free=(), c_full=None):
    sd, sf = list(steps_dep), list(steps_free)
    cf = _arr(_D, [float(v) for v in c_free]) if len(sf) else None
    cfull = _arr(_D, [float(v) for v in c_full]) if c_full is not None else None
    _check(h, lib().gbs_set_weights(h, int(slot), int(order), len(sd), _arr(_I, sd), len(sf),
                                    _arr(_I, sf) if sf else None, cf, cfull))


def gbs_get_weights(h, slot):
    m = _I()
    steps = (_I * GBS_MAX_SEQ)()
    c = (_D * GBS_MAX_SEQ)()
    isb = _D()
    _check(h, lib().gbs_get_weights(h, int(slot), ctypes.byref(m), steps, c, ctypes.byref(isb)))
    return list(steps[:m.value]), list(c[:m.value]), isb.value


def gbs_assign_slots(h, slots):
    _check(h, lib().gbs_assign_slots(h, _arr(_I, [int(s) for s in slots])))


def gbs_stability_limit(h, batch):
    out = (_D * batch)()
    _check(h, lib().gbs_stability_limit(h, out))
    return list(out)


def gbs_step(h, y_in, y_out, H, n_macro):
    _check(h, lib().gbs_step(h, _ptr(y_in), _ptr(y_out), float(H), int(n_macro)))


def gbs_step_batch(h, y_in, y_out, H, n_macro):
    _check(h, lib().gbs_step_batch(h, _ptr(y_in), _ptr(y_out), _arr(_D, [float(v) for v in H]), int(n_macro)))


def gbs_step_partial(h, y_in, partial, H, seq_mask):
    _check(h, lib().gbs_step_partial(h, _ptr(y_in), _ptr(partial), float(H), int(seq_mask) & 0xFFFFFFFF))


def gbs_combine_partial(h, y_in, total, y_out):
    _check(h, lib().gbs_combine_partial(h, _ptr(y_in), _ptr(total), _ptr(y_out)))


def gbs_step_host(h, y_in_host, y_out_host, H, n_macro):
    _check(h, lib().gbs_step_host(h, _ptr(y_in_host), _ptr(y_out_host), float(H), int(n_macro)))


def gbs_step_host_stream(h, y_in_hosts, y_out_hosts, H, n_macro):
    n = len(y_in_hosts)
    if len(y_out_hosts) != n:
        raise ValueError("as many output buffers as inputs are needed")
    ins = (_P * max(n, 1))(*[_ptr(t) for t in y_in_hosts])
    outs = (_P * max(n, 1))(*[_ptr(t) for t in y_out_hosts])
    _check(h, lib().gbs_step_host_stream(h, ins, outs, n, float(H), int(n_macro)))


def gbs_adjoint_step(h, y_in, lam_out, lam_in, grad_kappa, H, rcv_idx=None, rcv_resid=None):
    n_rcv = 0 if rcv_idx is None else int(rcv_idx.numel() if hasattr(rcv_idx, "numel") else len(rcv_idx))
    _check(h, lib().gbs_adjoint_step(h, _ptr(y_in), _ptr(lam_out), _ptr(lam_in), _ptr(grad_kappa), float(H),
                                     _ptr(rcv_idx), n_rcv, _ptr(rcv_resid)))


def gbs_misfit(h, y, rcv_idx, data, resid=None, J=None):
    n = int(rcv_idx.numel())
    _check(h, lib().gbs_misfit(h, _ptr(y), _ptr(rcv_idx), n, _ptr(data), _ptr(resid), _ptr(J)))


def gbs_inject(h, lam, rcv_idx, values):
    _check(h, lib().gbs_inject(h, _ptr(lam), _ptr(rcv_idx), int(rcv_idx.numel()), _ptr(values)))


def gbs_norms(h, a, b=None):
    out = (_D * 4)()
    _check(h, lib().gbs_norms(h, _ptr(a), _ptr(b), out))
    return tuple(out)


def gbs_set_option(h, name, value):
    _check(h, lib().gbs_set_option(h, name.encode(), int(value)))


def gbs_get_option(h, name):
    v = _I64()
    _check(h, lib().gbs_get_option(h, name.encode(), ctypes.byref(v)))
    return v.value


def gbs_kernel_time(h):
    """(launches, total_ms, algorithmic_bytes) of the dominant kernel since the last call."""
    n, ms, by = _I64(), _D(), _D()
    _check(h, lib().gbs_kernel_time(h, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)))
    return n.value, ms.value, by.value


def gbs_sync(h):
    _check(h, lib().gbs_sync(h))


def gbs_destroy(h):
    _check(h, lib().gbs_destroy(h))


def gbs_last_error(h):
    m = lib().gbs_last_error(h)
    return m.decode() if m else ""


def gbs_kernel_launches(h):
    return lib().gbs_kernel_launches(h)


def gbs_step_noalloc(pb, kappa, rho, order, steps_dep, steps_free, c_free, y_in, y_out, H, n_macro, stream=None):
    """Allocation-free stepping (see include/gbs.h); raises GbsError on failure."""
    sd, sf = list(steps_dep), list(steps_free)
    cf = _arr(_D, [float(v) for v in c_free]) if sf else None
    st = lib().gbs_step_noalloc(ctypes.byref(pb), _ptr(kappa), _ptr(rho), int(order), len(sd), _arr(_I, sd),
                                len(sf), _arr(_I, sf) if sf else None, cf, _ptr(y_in), _ptr(y_out), float(H),
                                int(n_macro), _ptr(stream))
    if st != GBS_OK:
        msg = lib().gbs_noalloc_last_error()
        raise GbsError(st, msg.decode() if msg else "")


def gbs_selftest_f32_to_f64(first, count):
    """(non-NaN differences, NaN differences beyond the quiet bit, NaN differences in the quiet
    bit alone) of the exact FP32 -> FP64 promotion against the conversion instruction over the
    float bit patterns [first, first + count)."""
    out = (ctypes.c_uint64 * 3)()
    st = lib().gbs_selftest_f32_to_f64(int(first), int(count), out)
    if st != GBS_OK:
        raise GbsError(st, "self-test of the FP32 -> FP64 promotion failed")
    return int(out[0]), int(out[1]), int(out[2])


def gbs_noalloc_last_error():
    m = lib().gbs_noalloc_last_error()
    return m.decode() if m else ""
