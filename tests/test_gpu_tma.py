"""GPU parity of the tensor-memory-access (TMA) staging of the FP32 tiled leap-frog step.

For one 2D or 3D acoustic problem with nx a multiple of 4, the one-step-per-launch kernel
stages the tiles whose box lies inside the grid with one tensor copy each (edge tiles with
loads; by default in 3D only, where it measured faster).  The copy moves the same values as
the loads, so the results with it on and off are
identical bit for bit, and both match the FP64 oracle within the FP32 tolerance of the other
tests.  The shapes give several interior tiles, edge tiles on both sides, and a partial last
tile; the option reports 0 where the copies do not apply (a batch, nx not a multiple of 4, FP64).
"""
import numpy as np
import pytest
import torch

from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import schemes as S
from tests.gpu_common import AcousticCase, oracle_scheme, rel_l2

pytestmark = pytest.mark.gpu
F32, F64 = B.GBS_F32_STATE_F64_COMBINE, B.GBS_F64


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("shape,order", [((136, 160), 6), ((136, 160), 4), ((6, 76, 72), 4), ((5, 70, 104), 6)])
def test_tma_staging_is_bit_identical_and_matches_oracle(shape, order):
    case = AcousticCase(shape, order, F32, seed=11)
    sol = case.solver()
    sol.set_scheme(S.GBS_8_6)
    sol.set_option("kernel", B.GBS_KERNEL_PLAIN)
    assert sol.get_option("tma") == (1 if len(shape) == 3 else 0)   # default: 3D only
    sol.set_option("tma", 1)
    assert sol.get_option("tma") == 1
    H = 0.7 * sol.stability_limit()[0]
    with_tma = case.gpu_run(sol, H, 2)
    sol.set_option("tma", 0)
    assert sol.get_option("tma") == 0
    without = case.gpu_run(sol, H, 2)
    assert np.array_equal(with_tma, without)
    steps, c = oracle_scheme(S.GBS_8_6)
    ref = case.oracle_run(steps, c, H, 2)
    assert rel_l2(with_tma, ref) <= 1e-5
    sol.close()


def test_tma_not_used_where_it_does_not_apply():
    odd = AcousticCase((64, 70), 4, F32, seed=2)          # nx = 70: not a multiple of 4
    sol = odd.solver()
    sol.set_option("tma", 1)
    assert sol.get_option("tma") == 0
    sol.close()
    f64 = AcousticCase((64, 72), 4, F64, seed=2)
    sol = f64.solver()
    sol.set_option("tma", 1)
    assert sol.get_option("tma") == 0
    sol.close()
