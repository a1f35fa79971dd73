"""GPU parity of the time-blocked FP32 path (2D acoustics): against the FP64 oracle
(relative L2 <= 1e-5) and against the point-parallel path on the same inputs.

Grids span several strips and row segments with ragged edges, both pass lengths of the
default build occur (T = 4, and T = 2 for the first pass of every N = 2 mod 4: GBS_{8,6} has
N = 2..22, GBS_{8,8} N = 2..30), and a batch mixes problem sizes and schemes.
"""
import numpy as np
import pytest
import torch

from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import schemes as S
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


def _run(case, sol, H, n, kernel, hseg=None):
    sol.set_option("kernel", kernel)
    if hseg:
        sol.set_option("hseg", hseg)
    return case.gpu_run(sol, H, n)


@pytest.mark.parametrize("shape,order,scheme,hseg", [
    ((37, 53), 6, S.GBS_8_6, None),          # one tile
    ((300, 290), 6, S.GBS_8_6, 96),          # 3 strips (97, 97, 96 columns) x 4 segments
    ((256, 384), 4, S.GBS_8_8, 64),          # 3 strips x 4 segments, N up to 30
    ((130, 260), 6, S.SQ8_TABLE1, 48),       # ragged both ways
])
def test_fused_vs_oracle_and_plain(shape, order, scheme, hseg):
    case = AcousticCase(shape, order, F32, seed=11)
    sol = case.solver()
    sol.set_scheme(scheme)
    H = 0.8 * sol.stability_limit()[0]
    g_fused = _run(case, sol, H, 2, B.GBS_KERNEL_FUSED, hseg)
    assert sol.uses_fused()
    g_plain = _run(case, sol, H, 2, B.GBS_KERNEL_PLAIN)
    steps, c = oracle_scheme(scheme)
    o = case.oracle_run(steps, c, H, 2)
    assert rel_l2(g_fused, o) <= 1e-5
    assert rel_l2(g_fused, g_plain) <= 1e-5
    sol.close()


def test_fused_batch_mixed_sizes_and_slots():
    shapes_yx = [(128, 128), (256, 128), (96, 200), (64, 64)]
    cases = [AcousticCase(s, 6, F32, seed=40 + i) for i, s in enumerate(shapes_yx)]
    kappa = torch.tensor(np.concatenate([c.kappa.ravel() for c in cases]), dtype=torch.float32, device="cuda")
    rho = torch.tensor(np.concatenate([c.rho.ravel() for c in cases]), dtype=torch.float32, device="cuda")
    sol = GBSSolver(B.GBS_ACOUSTIC, [c.shape_xyz for c in cases], [(1.0, 1.0)] * len(cases), fd_order=6,
                    precision=F32, kappa=kappa, rho=rho)
    sol.set_scheme(S.GBS_8_6, slot=0)
    sol.set_scheme(S.SQ8_TABLE1, slot=1)
    slots = [0, 1, 1, 0]
    sol.assign_slots(slots)
    sol.set_option("kernel", B.GBS_KERNEL_FUSED)
    sol.set_option("hseg", 64)
    assert sol.uses_fused()
    Hs = [0.8 * h for h in sol.stability_limit()]
    y = torch.tensor(np.concatenate([c.y0.ravel() for c in cases]), dtype=torch.float32, device="cuda")
    out = torch.empty_like(y)
    sol.step(y, out, Hs, 2)
    sol.sync()
    g = out.double().cpu().numpy()
    off = 0
    for i, c in enumerate(cases):
        n = c.y0.size
        steps, cw = oracle_scheme(S.GBS_8_6 if slots[i] == 0 else S.SQ8_TABLE1)
        assert rel_l2(g[off:off + n], c.oracle_run(steps, cw, Hs[i], 2)) <= 1e-5, i
        off += n
    sol.close()


def test_fused_in_place_graph_and_repeatability():
    case = AcousticCase((200, 256), 6, F32, seed=12)
    sol = case.solver()
    sol.set_scheme(S.GBS_8_6)
    sol.set_option("kernel", B.GBS_KERNEL_FUSED)
    sol.set_option("hseg", 64)
    H = 0.8 * sol.stability_limit()[0]
    y = torch.tensor(case.y0.ravel(), dtype=torch.float32, device="cuda")
    a = torch.empty_like(y)
    sol.step(y, a, H, 3)
    b = y.clone()
    sol.step(b, b, H, 3)                  # in place, graph replay
    sol.set_option("graph", 0)
    c = torch.empty_like(y)
    sol.step(y, c, H, 3)                  # direct launches
    sol.sync()
    assert torch.equal(a, b) and torch.equal(a, c)   # the dataflow schedule is deterministic
    sol.close()


def test_fused_unaligned_output_buffer():
    """The combine writes float4 groups only into 16-byte aligned output; an output view at a
    4-byte offset takes the element-wise path and gives the same bits."""
    case = AcousticCase((128, 160), 6, F32, seed=13)
    sol = case.solver()
    sol.set_scheme(S.GBS_8_6)
    sol.set_option("kernel", B.GBS_KERNEL_FUSED)
    H = 0.8 * sol.stability_limit()[0]
    y = torch.tensor(case.y0.ravel(), dtype=torch.float32, device="cuda")
    a = torch.empty_like(y)
    sol.step(y, a, H, 1)
    big = torch.zeros(y.numel() + 1, dtype=torch.float32, device="cuda")
    b = big[1:]
    assert b.data_ptr() % 16 != 0
    sol.step(y, b, H, 1)
    sol.sync()
    assert torch.equal(a, b)
    sol.close()


def test_fused_not_used_where_unsupported():
    case = AcousticCase((10, 16), 6, F32, seed=1)    # fewer rows than the 12-row halo
    sol = case.solver()
    sol.set_scheme(S.GBS_8_6)
    assert not sol.uses_fused()
    with pytest.raises(B.GbsError):
        sol.set_option("kernel", B.GBS_KERNEL_FUSED)
    sol.close()


def test_dependency_wait_timeout_is_reported_and_recoverable():
    """Failure detection without a fault: the first work item is made to wait on a flag
    that nothing sets; its bounded wait runs out, the kernel latches GBS_ERR_TIMEOUT
    (reported by gbs_sync) and the handle keeps working once the hook is off."""
    case = AcousticCase((64, 96), 6, F32, seed=13)
    sol = case.solver()
    sol.set_scheme(S.GBS_8_6)
    sol.set_option("kernel", B.GBS_KERNEL_FUSED)
    H = 0.8 * sol.stability_limit()[0]
    ref = case.gpu_run(sol, H, 1)
    sol.set_option("spin_limit", 2000)
    sol.set_option("inject_unsatisfiable_wait", 1)
    y = torch.tensor(case.y0.ravel(), dtype=torch.float32, device="cuda")
    out = torch.empty_like(y)
    sol.step(y, out, H, 1)
    with pytest.raises(B.GbsError) as e:
        sol.sync()
    assert e.value.status == 6   # GBS_ERR_TIMEOUT
    sol.set_option("inject_unsatisfiable_wait", 0)
    sol.set_option("spin_limit", 1 << 20)
    again = case.gpu_run(sol, H, 1)
    assert np.array_equal(again, ref)
    sol.close()
