"""GPU check of gbs_step_host_stream: a stream of independent host inputs, copies overlapping the
macro-steps through two alternating device staging states.

Each result must equal, bit for bit, gbs_step on the same input held on the device (the same
kernels run on the same values; only the copies move), for the time-blocked 2D path and the
plain 3D path, with outputs that alias one another and an empty stream.
"""
import numpy as np
import pytest
import torch

from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import schemes as S
from tests.gpu_common import AcousticCase

pytestmark = pytest.mark.gpu
F32 = B.GBS_F32_STATE_F64_COMBINE


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("shape,order", [((96, 128), 6), ((6, 40, 44), 4)])
def test_host_stream_equals_device_steps(shape, order):
    case = AcousticCase(shape, order, F32, seed=4)
    sol = case.solver()
    sol.set_scheme(S.GBS_8_6)
    H = 0.7 * sol.stability_limit()[0]
    rng = np.random.default_rng(8)
    ins = [torch.tensor((case.y0 * (1 + 0.1 * i) + 0.01 * rng.standard_normal(case.y0.shape)).astype(np.float32).ravel())
           .pin_memory() for i in range(5)]
    outs = [torch.empty_like(t).pin_memory() for t in ins]
    sol.step_host_stream(ins, outs, H, 2)
    for t, o in zip(ins, outs):
        d = t.cuda()
        ref = torch.empty_like(d)
        sol.step(d, ref, H, 2)
        sol.sync()
        assert torch.equal(o, ref.cpu())
    # every result into one host buffer (aliased outputs, written in order): the last one stays
    last = torch.empty_like(ins[0]).pin_memory()
    sol.step_host_stream(ins, [last] * len(ins), H, 2)
    assert torch.equal(last, outs[-1])
    sol.step_host_stream([], [], H, 2)
    sol.close()
