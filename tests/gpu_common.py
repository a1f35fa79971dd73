"""Shared helpers for the GPU parity tests: run the same seeded inputs through the
CUDA library (via the C ABI binding) and through the FP64 CPU oracle."""
from fractions import Fraction

import numpy as np
import torch

from oracle import gbs as OG
from oracle import mol as OM
from oracle import weights as OW
from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import inputs
from paper_1907_11771_gb300.solver import GBSSolver
from tests.conftest import load_golden

GOLD = load_golden("paper_schemes.txt")
GOLD_OF = {"GBS_8,6": "gbs_8_6", "GBS_8,8": "gbs_8_8", "GBS_12,8": "gbs_12_8",
           "SQ8{2,16,18,20}": "table1_order8", "SQ12{2,8,12,14,16,20}": "table1_order12",
           "SQ16{2,8,...,22}": "table1_order16"}


def oracle_scheme(scheme):
    """Step counts and FP64-rounded exact weights, from the paper's printed values."""
    if scheme.name in GOLD_OF:
        g = GOLD[GOLD_OF[scheme.name]]
        dep = [int(t) for t in g["dep"].split()]
        free = [int(t) for t in g.get("free", "").split()]
        cf = [Fraction(t) for t in g.get("cfree", "").split()]
        steps, c = OW.scheme_weights(int(g["order"]), dep, free, cf)
    elif scheme.steps_free:  # schemes optimised here: their recorded rationals are the data
        steps, c = OW.scheme_weights(scheme.order, list(scheme.steps_dep), list(scheme.steps_free),
                                     [Fraction(t) for t in scheme.c_free_text])
    else:  # textbook square schemes
        steps = list(scheme.steps_dep)
        c = OW.square_weights(steps, scheme.order)
    return steps, OW.to_fp64(c)


def fp32_floor(scheme, n_macro):
    """4 x 2^-24 x sqrt(sum_k c_k^2 (N_k + 1)) x sqrt(M): the FP32 rounding floor of M macro-steps
    (four roundings of 2^-24 per leap-frog update, independent across the N_k + 1 updates of a
    sequence and across macro-steps, amplified by the weights c_k)."""
    import math
    steps, c = oracle_scheme(scheme)
    amp = math.sqrt(sum(float(ck) ** 2 * (n + 1) for n, ck in zip(steps, c)))
    return 4 * 2.0 ** -24 * amp * math.sqrt(n_macro)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class AcousticCase:
    """A seeded acoustic problem on a (z,) y, x grid, run on GPU and oracle."""

    def __init__(self, shape_zyx, order, precision, seed=0, n_gauss=3, sigma=None, const_rho=False):
        self.shape = tuple(shape_zyx)
        self.ndim = len(self.shape)
        self.order = order
        self.precision = precision
        self.np_dtype = np.float32 if precision == B.GBS_F32_STATE_F64_COMBINE else np.float64
        sigma = sigma if sigma is not None else max(2.0, min(self.shape) / 8.0)
        y0, kappa, rho = inputs.acoustic_problem(self.shape, seed, n_gauss, sigma, const_rho=const_rho)
        # smooth non-zero velocities (seeded Gaussian bumps) exercise every term of the operator
        rng = np.random.default_rng(seed + 99)
        for f in range(1, y0.shape[0]):
            c = [[rng.uniform(0, n) for n in self.shape]]
            y0[f] = 0.3 * rng.uniform(-1, 1) * inputs.gaussian_pulses(self.shape, sigma, c)
        # both sides see the same (rounded) inputs
        self.y0 = y0.astype(self.np_dtype).astype(np.float64)
        self.kappa = kappa.astype(self.np_dtype).astype(np.float64)
        self.rho = rho.astype(self.np_dtype).astype(np.float64)
        self.dx = [1.0] * self.ndim
        self.shape_xyz = tuple(reversed(self.shape))

    def solver(self, enable_adjoint=False):
        dt = torch.float32 if self.precision == B.GBS_F32_STATE_F64_COMBINE else torch.float64
        self.t_kappa = torch.tensor(self.kappa.ravel(), dtype=dt, device="cuda")
        self.t_rho = torch.tensor(self.rho.ravel(), dtype=dt, device="cuda")
        return GBSSolver(B.GBS_ACOUSTIC, [self.shape_xyz], [tuple(self.dx)], fd_order=self.order,
                         precision=self.precision, kappa=self.t_kappa, rho=self.t_rho,
                         enable_adjoint=enable_adjoint)

    def f(self, y):
        return OM.rhs_acoustic(y, self.kappa, 1.0 / self.rho, self.dx, self.order)

    def fT(self, y):
        return OM.rhs_acoustic_T(y, self.kappa, 1.0 / self.rho, self.dx, self.order)

    def pair(self, mu, y):
        return OM.dA_dkappa_pairing(mu, y, self.dx, self.order)

    def oracle_run(self, steps, c, H, n_macro):
        return OG.gbs_run(self.f, self.y0, H, steps, c, n_macro)

    def gpu_run(self, solver, H, n_macro):
        dt = torch.float32 if self.precision == B.GBS_F32_STATE_F64_COMBINE else torch.float64
        y = torch.tensor(self.y0.ravel(), dtype=dt, device="cuda")
        out = torch.empty_like(y)
        solver.step(y, out, H, n_macro)
        solver.sync()
        return out.double().cpu().numpy().reshape(self.y0.shape)
