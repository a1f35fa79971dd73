"""The sequence-fused one-level step (FP32 2D/3D acoustics on the one-level kernels): one launch
per leap-frog level advances every sequence that has that level (Sec. 2.1 eq. "GBS", the
sequences of Sec. 3.6 run side by side), each from its own pair of level buffers.  On by default
in 2D; set explicitly here in 3D.

Each update is the one-sequence-per-launch kernel's, so with step counts in increasing order
(the combine then adds the sequences' terms in the same order) the two agree bit for bit: 2D
and 3D, ragged tiles, tensor-copy and load staging, batches with mixed sizes and slots of
different sequence counts, partial steps.  With step counts out of order (GBS_12,8) only the
FP64 combine's summation order differs: the results agree to the FP32 rounding of the sum, and
both meet the oracle.
"""
import numpy as np
import pytest
import torch

from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import schemes as S
from paper_1907_11771_gb300 import seqpar
from paper_1907_11771_gb300.solver import GBSSolver
from tests.gpu_common import AcousticCase, fp32_floor, oracle_scheme, rel_l2

pytestmark = pytest.mark.gpu
F32 = B.GBS_F32_STATE_F64_COMBINE


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _solver(case, scheme, seqfuse, tma=-1):
    sol = case.solver()
    sol.set_scheme(scheme)
    sol.set_option("kernel", B.GBS_KERNEL_PLAIN)
    sol.set_option("seqfuse", seqfuse)
    sol.set_option("tma", tma)
    assert sol.get_option("seqfuse") == seqfuse
    return sol


def _run(sol, y0, H, n_macro):
    y = torch.tensor(np.asarray(y0).ravel(), dtype=torch.float32, device="cuda")
    out = torch.empty_like(y)
    sol.step(y, out, H, n_macro)
    sol.sync()
    return out


@pytest.mark.parametrize("scheme", [S.GBS_8_6, S.SQ8_2468])
@pytest.mark.parametrize("shape,order,tma", [((45, 70), 6, 0), ((64, 96), 6, 1), ((40, 37), 4, 0),
                                             ((13, 21, 30), 4, -1), ((9, 40, 36), 4, 0), ((7, 33, 20), 6, -1)])
def test_fused_sequences_are_bit_identical_to_one_sequence_per_launch(scheme, shape, order, tma):
    case = AcousticCase(shape, order, F32, seed=17)
    a_sol, b_sol = _solver(case, scheme, 1, tma), _solver(case, scheme, 0, tma)
    H = 0.8 * a_sol.stability_limit()[0]
    a, b = _run(a_sol, case.y0, H, 3), _run(b_sol, case.y0, H, 3)
    assert torch.isfinite(a).all()
    assert torch.equal(a, b), (a - b).abs().max().item()
    a_sol.close()
    b_sol.close()


def test_fused_sequences_out_of_order_steps_meet_the_oracle():
    case = AcousticCase((11, 18, 25), 4, F32, seed=4)
    a_sol, b_sol = _solver(case, S.GBS_12_8, 1), _solver(case, S.GBS_12_8, 0)
    H = 0.5 * a_sol.stability_limit()[0]
    a, b = _run(a_sol, case.y0, H, 2), _run(b_sol, case.y0, H, 2)
    ref = torch.linalg.vector_norm(b.double())
    assert (torch.linalg.vector_norm((a - b).double()) / ref).item() <= 2e-7
    steps, c = oracle_scheme(S.GBS_12_8)
    o = case.oracle_run(steps, c, H, 2)
    # GBS_12,8's large weights amplify FP32 rounding: its floor, not the order-8 schemes' 1e-5
    assert rel_l2(a.double().cpu().numpy().reshape(o.shape), o) <= fp32_floor(S.GBS_12_8, 2)
    a_sol.close()
    b_sol.close()


def test_fused_sequences_batch_mixed_slots():
    cases = [AcousticCase(s, 6, F32, seed=50 + i) for i, s in enumerate([(30, 44), (17, 29), (52, 40), (8, 9)])]
    kappa = torch.tensor(np.concatenate([c.kappa.ravel() for c in cases]), dtype=torch.float32, device="cuda")
    rho = torch.tensor(np.concatenate([c.rho.ravel() for c in cases]), dtype=torch.float32, device="cuda")
    y0 = np.concatenate([c.y0.ravel() for c in cases])
    outs = []
    for fuse in (1, 0):
        sol = GBSSolver(B.GBS_ACOUSTIC, [c.shape_xyz for c in cases], [(1.0, 1.0)] * 4, fd_order=6,
                        precision=F32, kappa=kappa, rho=rho)
        sol.set_scheme(S.GBS_8_6, slot=0)
        sol.set_scheme(S.SQ8_2468, slot=1)
        sol.assign_slots([0, 1, 1, 0])
        sol.set_option("kernel", B.GBS_KERNEL_PLAIN)
        sol.set_option("seqfuse", fuse)
        assert sol.get_option("seqfuse") == fuse
        H = 0.8 * min(sol.stability_limit())
        outs.append(_run(sol, y0, H, 2))
        sol.close()
    assert torch.equal(outs[0], outs[1])


def test_fused_sequences_partial_steps():
    case = AcousticCase((10, 26, 33), 4, F32, seed=41)
    a_sol, b_sol = _solver(case, S.GBS_8_6, 1), _solver(case, S.GBS_8_6, 0)
    H = 0.8 * a_sol.stability_limit()[0]
    y = torch.tensor(case.y0.ravel(), dtype=torch.float32, device="cuda")
    for m in seqpar.partition(S.GBS_8_6.steps, 3)[0]:
        a = torch.empty(y.numel(), dtype=torch.float64, device="cuda")
        b = torch.empty_like(a)
        a_sol.step_partial(y, a, H, m)
        b_sol.step_partial(y, b, H, m)
        a_sol.sync()
        b_sol.sync()
        assert torch.equal(a, b)
    a_sol.close()
    b_sol.close()


def test_fused_sequences_where_they_apply():
    # the default for the one-level kernels in 2D; in 3D only when asked for (measured slower
    # there); never with the time-blocked kernel, nor for FP64 states
    c3 = AcousticCase((8, 20, 24), 4, F32)
    s3 = c3.solver()
    s3.set_scheme(S.GBS_8_6)
    assert not s3.uses_fused() and s3.get_option("seqfuse") == 0
    s3.set_option("seqfuse", 1)
    assert s3.get_option("seqfuse") == 1
    s3.close()
    c2 = AcousticCase((40, 48), 6, F32)
    s2 = c2.solver()
    s2.set_scheme(S.GBS_8_6)
    assert s2.uses_fused() and s2.get_option("seqfuse") == 0
    s2.set_option("kernel", B.GBS_KERNEL_PLAIN)
    assert s2.get_option("seqfuse") == 1
    s2.close()
    c64 = AcousticCase((8, 20, 24), 4, B.GBS_F64)
    s64 = c64.solver()
    s64.set_scheme(S.GBS_8_6)
    assert s64.get_option("seqfuse") == 0
    s64.close()
