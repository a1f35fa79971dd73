"""The 3D time-blocked pass kernel (two leap-frog levels per pass, z-sweep with register
windows; Sec. 2.1 eq. "GBS") against the one-level kernel and the CPU oracle.

Its updates carry the one-level kernel's arithmetic in the same order, so the two must agree
bit for bit: grids with several tiles and ragged edges in x and y (24 x 16 output columns per
tile at 4th order, 20 x 12 at 6th), z-segments with a ragged last one, grids smaller than a
tile or than the z-skew (every coordinate wraps), batches with mixed sizes and weight slots,
and sequence-parallel partial steps.  Against the FP64 oracle it meets the FP32 parity
tolerance of the other FP32 paths.  It runs when GBS_KERNEL_FUSED is set; the default choice in
3D is the one-level kernel.
"""
import numpy as np
import pytest
import torch

from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import schemes as S
from paper_1907_11771_gb300 import seqpar
from paper_1907_11771_gb300.solver import GBSSolver
from tests.gpu_common import AcousticCase, oracle_scheme, rel_l2

pytestmark = pytest.mark.gpu
F32 = B.GBS_F32_STATE_F64_COMBINE


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _both(case, scheme, zseg=None):
    """(time-blocked, one-level) solvers of the same case."""
    out = []
    for kernel in (B.GBS_KERNEL_FUSED, B.GBS_KERNEL_PLAIN):
        sol = case.solver()
        sol.set_scheme(scheme)
        sol.set_option("kernel", kernel)
        if zseg is not None:
            sol.set_option("zseg", zseg)
        out.append(sol)
    assert out[0].uses_fused() and not out[1].uses_fused()
    return out


def _run(sol, y0, H, n_macro):
    y = torch.tensor(y0.ravel(), dtype=torch.float32, device="cuda")
    out = torch.empty_like(y)
    sol.step(y, out, H, n_macro)
    sol.sync()
    return out


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("scheme", [S.GBS_8_6, S.SQ8_2468])
@pytest.mark.parametrize("shape,zseg", [((37, 45, 70), None), ((19, 20, 25), 7), ((5, 7, 9), 3), ((3, 40, 52), 128)])
def test_time_blocked_3d_is_bit_identical_to_the_one_level_kernel(order, scheme, shape, zseg):
    case = AcousticCase(shape, order, F32, seed=13)
    tb, plain = _both(case, scheme, zseg)
    H = 0.8 * tb.stability_limit()[0]
    a = _run(tb, case.y0, H, 3)
    b = _run(plain, case.y0, H, 3)
    assert torch.isfinite(a).all()
    assert torch.equal(a, b), (a - b).abs().max().item()
    tb.close()
    plain.close()


@pytest.mark.parametrize("order", [4, 6])
def test_time_blocked_3d_matches_the_oracle(order):
    case = AcousticCase((13, 21, 30), order, F32, seed=21)
    sol = case.solver()
    sol.set_scheme(S.GBS_8_6)
    assert not sol.uses_fused()        # the default choice in 3D: the one-level kernel
    sol.set_option("kernel", B.GBS_KERNEL_FUSED)
    sol.set_option("zseg", 5)
    assert sol.uses_fused()
    H = 0.8 * sol.stability_limit()[0]
    steps, c = oracle_scheme(S.GBS_8_6)
    err = rel_l2(case.gpu_run(sol, H, 2), case.oracle_run(steps, c, H, 2))
    assert err <= 1e-5, err
    sol.close()


def test_time_blocked_3d_batch_mixed_sizes_and_slots():
    cases = [AcousticCase(s, 4, F32, seed=30 + i) for i, s in enumerate([(9, 30, 26), (14, 17, 40), (4, 5, 6)])]
    kappa = torch.tensor(np.concatenate([c.kappa.ravel() for c in cases]), dtype=torch.float32, device="cuda")
    rho = torch.tensor(np.concatenate([c.rho.ravel() for c in cases]), dtype=torch.float32, device="cuda")
    y0 = np.concatenate([c.y0.ravel() for c in cases])
    outs = []
    for kernel in (B.GBS_KERNEL_FUSED, B.GBS_KERNEL_PLAIN):
        sol = GBSSolver(B.GBS_ACOUSTIC, [c.shape_xyz for c in cases], [(1.0, 1.0, 1.0)] * 3, fd_order=4,
                        precision=F32, kappa=kappa, rho=rho)
        sol.set_scheme(S.GBS_8_6, slot=0)
        sol.set_scheme(S.SQ8_2468, slot=1)
        sol.assign_slots([0, 1, 0])
        sol.set_option("kernel", kernel)
        sol.set_option("zseg", 6)
        assert sol.uses_fused() == (kernel == B.GBS_KERNEL_FUSED)
        H = 0.8 * min(sol.stability_limit())
        outs.append(_run(sol, y0, H, 2))
        sol.close()
    assert torch.equal(outs[0], outs[1])


def test_time_blocked_3d_partial_steps_match_the_one_level_kernel():
    case = AcousticCase((10, 26, 33), 4, F32, seed=41)
    tb, plain = _both(case, S.GBS_8_6, zseg=4)
    H = 0.8 * tb.stability_limit()[0]
    y = torch.tensor(case.y0.ravel(), dtype=torch.float32, device="cuda")
    for m in seqpar.partition(S.GBS_8_6.steps, 3)[0]:
        a = torch.empty(y.numel(), dtype=torch.float64, device="cuda")
        b = torch.empty_like(a)
        tb.step_partial(y, a, H, m)
        plain.step_partial(y, b, H, m)
        tb.sync()
        plain.sync()
        assert torch.equal(a, b)
    tb.close()
    plain.close()


def test_zseg_option_range_and_kernel_timing():
    case = AcousticCase((8, 20, 20), 4, F32, seed=2)
    sol = case.solver()
    sol.set_scheme(S.SQ8_2468)
    sol.set_option("kernel", B.GBS_KERNEL_FUSED)
    assert sol.get_option("zseg") == 128
    with pytest.raises(B.GbsError):
        sol.set_option("zseg", 0)
    sol.set_option("time_kernels", 1)
    H = 0.5 * sol.stability_limit()[0]
    _run(sol, case.y0, H, 1)
    launches, ms, nbytes = sol.kernel_time()
    # SQ8{2,4,6,8}: 1 + 2 + 3 + 4 passes of two levels
    assert launches == 10 and ms > 0 and nbytes > 0
    sol.close()
