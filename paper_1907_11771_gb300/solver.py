"""A small object wrapper over the C ABI (marshalling only).

``GBSSolver`` owns one library handle and remembers the problem description so
that callers can pass torch tensors and Python lists.  Memory and streams come
from PyTorch; every computation happens in libgbs.so.
"""
import torch

from . import binding as B
from .schemes import Scheme

_DTYPES = {B.GBS_F32_STATE_F64_COMBINE: torch.float32, B.GBS_F64: torch.float64, B.GBS_F32X2: torch.float64}


class GBSSolver:
    def __init__(self, system, shapes, dx, fd_order=4, precision=B.GBS_F32_STATE_F64_COMBINE,
                 kappa=None, rho=None, enable_adjoint=False, stream=None):
        """shapes, dx: per problem (nx, ny, nz) triples (x fastest).  kappa, rho:
        concatenated media tensors on the GPU (None for the 1D wave system)."""
        self.system = system
        self.shapes = [tuple(s) + (1,) * (3 - len(s)) for s in shapes]
        self.ndim = 1 if system != B.GBS_ACOUSTIC else max(1, len(shapes[0]))
        self.batch = len(self.shapes)
        self.precision = precision
        self.fd_order = fd_order
        self.slots = [0] * len(shapes)
        self.dtype = _DTYPES[precision]
        self.F = 2 if system == B.GBS_WAVE1D else 1 if system == B.GBS_ONEWAY_SPECTRAL else 1 + self.ndim
        self.pb = B.make_problem(system, self.ndim, fd_order, precision, self.shapes, dx, enable_adjoint)
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        self._media = (kappa, rho)
        self.h = B.gbs_create(self.pb, kappa, rho, stream)

    def close(self):
        if self.h:
            B.gbs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_media(self, kappa, rho):
        """Point the solver at new media tensors (kept alive here; b = 1/rho recomputed)."""
        B.gbs_set_media(self.h, kappa, rho)
        self._media = (kappa, rho)

    # -- scheme set-up -------------------------------------------------------
    def set_scheme(self, scheme: Scheme, slot=0):
        B.gbs_set_weights(self.h, slot, scheme.order, scheme.steps_dep, scheme.steps_free, scheme.c_free)

    def weights(self, slot=0):
        return B.gbs_get_weights(self.h, slot)

    def assign_slots(self, slots):
        B.gbs_assign_slots(self.h, slots)
        self.slots = [int(v) for v in slots]

    def stability_limit(self):
        return B.gbs_stability_limit(self.h, self.batch)

    # -- state helpers ------------------------------------------------------------
    @property
    def state_elems(self):
        return B.gbs_state_elems(self.pb)

    def empty_state(self, device="cuda"):
        return torch.empty(self.state_elems, dtype=self.dtype, device=device)

    # -- stepping -----------------------------------------------------------------
    def step(self, y_in, y_out, H, n_macro=1):
        if isinstance(H, (list, tuple)):
            B.gbs_step_batch(self.h, y_in, y_out, H, n_macro)
        else:
            B.gbs_step(self.h, y_in, y_out, H, n_macro)

    def step_partial(self, y_in, partial, H, seq_mask):
        B.gbs_step_partial(self.h, y_in, partial, H, seq_mask)

    def combine_partial(self, y_in, total, y_out):
        B.gbs_combine_partial(self.h, y_in, total, y_out)

    def step_host(self, y_in_host, y_out_host, H, n_macro=1):
        B.gbs_step_host(self.h, y_in_host, y_out_host, H, n_macro)

    def step_host_stream(self, y_in_hosts, y_out_hosts, H, n_macro=1):
        """Independent host inputs through the device with copies overlapping the steps."""
        B.gbs_step_host_stream(self.h, y_in_hosts, y_out_hosts, H, n_macro)

    def adjoint_step(self, y_in, lam_out, lam_in, grad_kappa, H, rcv_idx=None, rcv_resid=None):
        B.gbs_adjoint_step(self.h, y_in, lam_out, lam_in, grad_kappa, H, rcv_idx, rcv_resid)

    def misfit(self, y, rcv_idx, data, resid=None, J=None):
        B.gbs_misfit(self.h, y, rcv_idx, data, resid, J)

    def inject(self, lam, rcv_idx, values):
        B.gbs_inject(self.h, lam, rcv_idx, values)

    def norms(self, a, b=None):
        return B.gbs_norms(self.h, a, b)

    def set_option(self, name, value):
        B.gbs_set_option(self.h, name, value)

    def get_option(self, name):
        return B.gbs_get_option(self.h, name)

    def uses_fused(self):
        return B.gbs_get_option(self.h, "kernel_in_use") == B.GBS_KERNEL_FUSED

    def kernel_time(self):
        return B.gbs_kernel_time(self.h)

    def sync(self):
        B.gbs_sync(self.h)

    @property
    def kernel_launches(self):
        return B.gbs_kernel_launches(self.h)
