"""Sequence-parallel macro-steps on one GPU: the ranks of a partition run one after another
(gbs_step_partial with each rank's mask), their FP64 shares are summed, gbs_combine_partial
completes the step, and the result matches the whole macro-step (gbs_step) of the same handle
-- so an all-reduce across GPUs computes exactly what one GPU does (Sec. 3.6's distribution
of the sequences over cores).  Every precision, both the plain and the time-blocked kernels,
several macro-steps; a whole step after partial ones still uses the full schedule.

Tolerances: FP64 and FP32 pairs, the same FP64 terms c_k y*_k summed in another order: at most
(m + ranks) roundings of 2^-53 of sum_k |c_k| |y| per macro-step, n_macro (m + ranks) 2^-53
sum_k |c_k| (1.8e-13 for three GBS_8,6 macro-steps on six ranks); FP32 states 1e-7 (the same
FP64 sum rounded once to FP32).
"""
import numpy as np
import pytest
import torch

from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import inputs
from paper_1907_11771_gb300 import schemes as S
from paper_1907_11771_gb300 import seqpar
from paper_1907_11771_gb300.solver import GBSSolver

pytestmark = pytest.mark.gpu
F32, F64, X2 = B.GBS_F32_STATE_F64_COMBINE, B.GBS_F64, B.GBS_F32X2


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case(shape, prec, kernel):
    y0, kappa, rho = inputs.acoustic_problem(shape, 17, 3, max(2.0, min(shape) / 8))
    dt = torch.float32 if prec == F32 else torch.float64
    npdt = np.float32 if prec == F32 else np.float64
    t = lambda a: torch.tensor(a.astype(npdt).ravel(), dtype=dt, device="cuda")
    y, k, r = t(y0), t(kappa), t(rho)
    sol = GBSSolver(B.GBS_ACOUSTIC, [shape[::-1]], [(1.0,) * len(shape)], fd_order=6 if len(shape) == 2 else 4,
                    precision=prec, kappa=k, rho=r)
    sol._keep = (k, r)
    sol.set_scheme(S.GBS_8_6)
    sol.set_option("kernel", kernel)
    return sol, y


def _emulated(sol, y, H, masks, n_macro):
    """n_macro sequence-parallel macro-steps with the ranks of `masks` run one after another."""
    cur = y.clone()
    part = torch.empty(y.numel(), dtype=torch.float64, device="cuda")
    total = torch.empty_like(part)
    for _ in range(n_macro):
        total.zero_()
        for m in masks:
            if m:
                sol.step_partial(cur, part, H, m)
                total += part
        sol.combine_partial(cur, total, cur)
    sol.sync()
    return cur


@pytest.mark.parametrize("prec,kernel", [(F32, B.GBS_KERNEL_FUSED), (F32, B.GBS_KERNEL_PLAIN),
                                         (F64, B.GBS_KERNEL_PLAIN), (X2, B.GBS_KERNEL_PLAIN)])
@pytest.mark.parametrize("ranks", [2, 3, 6])
def test_partial_steps_summed_over_ranks_equal_the_whole_step(prec, kernel, ranks):
    sol, y = _case((72, 100), prec, kernel)
    H = 0.8 * sol.stability_limit()[0]
    masks, _ = seqpar.partition(S.GBS_8_6.steps, ranks)
    got = _emulated(sol, y, H, masks, 3)
    ref = torch.empty_like(y)
    sol.step(y, ref, H, 3)
    sol.sync()
    assert sol.uses_fused() == (kernel == B.GBS_KERNEL_FUSED)
    err = (torch.linalg.vector_norm((got - ref).double()) / torch.linalg.vector_norm(ref.double())).item()
    sum_c = sum(abs(c) for c in sol.weights()[1])
    bound = 1e-7 if prec == F32 else 3 * (S.GBS_8_6.m + ranks) * 2.0 ** -53 * sum_c
    assert err <= bound, (err, bound)
    sol.close()


def test_partial_steps_3d_and_whole_step_after_them():
    sol, y = _case((12, 20, 24), F32, B.GBS_KERNEL_AUTO)
    H = 0.8 * sol.stability_limit()[0]
    ref = torch.empty_like(y)
    sol.step(y, ref, H, 2)
    got = _emulated(sol, y, H, seqpar.partition(S.GBS_8_6.steps, 4)[0], 2)
    again = torch.empty_like(y)
    sol.step(y, again, H, 2)                       # the whole step after partial ones
    sol.sync()
    rel = lambda a: (torch.linalg.vector_norm((a - ref).double()) / torch.linalg.vector_norm(ref.double())).item()
    assert rel(got) <= 1e-7
    assert torch.equal(again, ref)
    sol.close()


def test_partial_step_refuses_an_empty_mask():
    sol, y = _case((32, 32), F32, B.GBS_KERNEL_PLAIN)
    part = torch.empty(y.numel(), dtype=torch.float64, device="cuda")
    with pytest.raises(B.GbsError) as e:
        sol.step_partial(y, part, 0.1, 0)
    assert e.value.status == 1
    sol.close()
