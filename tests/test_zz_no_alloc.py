"""gbs_step_noalloc: stepping for callers that cannot call cudaMalloc.

Some host programs hand all GPU memory to their own allocator or pool (or run
this library as a plug-in inside such a program), so they cannot let the
library allocate a workspace the way gbs_create does.  gbs_step_noalloc keeps
its scratch in a fixed array compiled into the library instead.  This test
calls it through the C ABI twice in a row and checks each result against the
ordinary handle-based gbs_step on the same inputs, within the FP32 tolerance
the other parity tests use; it also checks that a problem too large for the
fixed array is refused with a clear message.

The file name makes pytest collect it last, so a run that stops at the first
failure has already run every other test; it also passes on its own in a fresh
process.
"""
import numpy as np
import pytest
import torch

from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import inputs
from paper_1907_11771_gb300 import schemes as S
from paper_1907_11771_gb300.solver import GBSSolver

pytestmark = pytest.mark.gpu

TOL = 1e-5   # FP32-state / FP64-combine tolerance used by the parity tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _problem(shape_yx, seed):
    y0, kappa, rho = inputs.acoustic_problem(shape_yx, seed, 3, max(2.0, min(shape_yx) / 8))
    t = lambda a: torch.tensor(a.astype(np.float32).ravel(), device="cuda")
    return t(y0), t(kappa), t(rho)


def _rel(a, b):
    return (torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double())).item()


def _handle_step(shape_yx, y, kappa, rho, H, n_macro):
    sol = GBSSolver(B.GBS_ACOUSTIC, [shape_yx[::-1]], [(1.0, 1.0)], fd_order=6,
                    precision=B.GBS_F32_STATE_F64_COMBINE, kappa=kappa, rho=rho)
    sol.set_scheme(S.GBS_8_6)
    if H is None:
        H = 0.8 * sol.stability_limit()[0]
    out = torch.empty_like(y)
    sol.step(y, out, H, n_macro)
    sol.sync()
    sol.close()
    return out, H


def _noalloc_step(shape_yx, y, kappa, rho, H, n_macro, out):
    pb = B.make_problem(B.GBS_ACOUSTIC, 2, 6, B.GBS_F32_STATE_F64_COMBINE, [shape_yx[::-1]], [(1.0, 1.0)])
    sc = S.GBS_8_6
    B.gbs_step_noalloc(pb, kappa, rho, sc.order, sc.steps_dep, sc.steps_free, sc.c_free, y, out, H, n_macro,
                       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()


def test_noalloc_matches_handle_path_on_two_calls_in_a_row():
    # first call: a 96 x 80 problem, three macro-steps
    shape1 = (96, 80)
    y1, k1, r1 = _problem(shape1, 31)
    ref1, H1 = _handle_step(shape1, y1, k1, r1, None, 3)
    out1 = torch.empty_like(y1)
    _noalloc_step(shape1, y1, k1, r1, H1, 3, out1)
    assert _rel(out1, ref1) <= TOL
    # second call right after it: another problem, in place, reusing the same fixed scratch
    shape2 = (64, 72)
    y2, k2, r2 = _problem(shape2, 32)
    ref2, H2 = _handle_step(shape2, y2, k2, r2, None, 2)
    inplace = y2.clone()
    _noalloc_step(shape2, inplace, k2, r2, H2, 2, inplace)
    assert _rel(inplace, ref2) <= TOL


def test_noalloc_rejects_problems_larger_than_its_fixed_scratch():
    shape = (2048, 2048)   # needs far more than GBS_NOALLOC_SCRATCH_BYTES
    y = torch.zeros(3 * shape[0] * shape[1], dtype=torch.float32, device="cuda")
    k = torch.ones(shape[0] * shape[1], dtype=torch.float32, device="cuda")
    with pytest.raises(B.GbsError) as e:
        _noalloc_step(shape, y, k, k, 0.1, 1, y)
    assert e.value.status == 1
    assert "limited to" in B.gbs_noalloc_last_error()


# ---------------------------------------------------------------------------
# More of the problem layouts the allocation-free entry point accepts, each against the
# handle path (and once against the CPU oracle): a batch of unevenly sized problems, FP64
# states, the 1D wave system, a 3D grid, zero macro-steps; and the refusals that need a GPU.
# ---------------------------------------------------------------------------

def _noalloc(pb, kappa, rho, scheme, y, out, H, n_macro):
    B.gbs_step_noalloc(pb, kappa, rho, scheme.order, scheme.steps_dep, scheme.steps_free, scheme.c_free, y, out,
                       H, n_macro, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()


def _handle(system, shapes_xyz, dx, order, prec, kappa, rho, scheme, y, n_macro, H=None, kernel=None):
    sol = GBSSolver(system, shapes_xyz, dx, fd_order=order, precision=prec, kappa=kappa, rho=rho)
    sol.set_scheme(scheme)
    if kernel is not None:
        sol.set_option("kernel", kernel)
    if H is None:
        H = 0.8 * min(sol.stability_limit())
    out = torch.empty_like(y)
    sol.step(y, out, H, n_macro)
    sol.sync()
    sol.close()
    return out, H


def test_noalloc_matches_the_oracle():
    from oracle import gbs as OG
    from oracle import mol as OM
    from tests.gpu_common import oracle_scheme
    shape = (40, 36)
    y0, kappa, rho = inputs.acoustic_problem(shape, 41, 3, 5.0)
    y0, kappa, rho = (a.astype(np.float32).astype(np.float64) for a in (y0, kappa, rho))
    t = lambda a: torch.tensor(a.astype(np.float32).ravel(), device="cuda")
    y, k, r = t(y0), t(kappa), t(rho)
    _, H = _handle(B.GBS_ACOUSTIC, [shape[::-1]], [(1.0, 1.0)], 6, B.GBS_F32_STATE_F64_COMBINE, k, r, S.GBS_8_6, y, 0)
    out = torch.empty_like(y)
    pb = B.make_problem(B.GBS_ACOUSTIC, 2, 6, B.GBS_F32_STATE_F64_COMBINE, [shape[::-1]], [(1.0, 1.0)])
    _noalloc(pb, k, r, S.GBS_8_6, y, out, H, 2)
    steps, c = oracle_scheme(S.GBS_8_6)
    o = OG.gbs_run(lambda v: OM.rhs_acoustic(v, kappa, 1.0 / rho, [1.0, 1.0], 6), y0, H, steps, c, 2)
    g = out.double().cpu().numpy().reshape(y0.shape)
    assert np.linalg.norm(g - o) / np.linalg.norm(o) <= TOL


def test_noalloc_batch_of_uneven_problems_matches_handle_path():
    shapes = [(24, 40), (48, 32), (36, 36)]          # (ny, nx)
    parts = [inputs.acoustic_problem(s, 50 + i, 3, 4.0) for i, s in enumerate(shapes)]
    t = lambda arrs: torch.tensor(np.concatenate([a.astype(np.float32).ravel() for a in arrs]), device="cuda")
    y, k, r = t([p[0] for p in parts]), t([p[1] for p in parts]), t([p[2] for p in parts])
    xyz = [s[::-1] for s in shapes]
    ref, H = _handle(B.GBS_ACOUSTIC, xyz, [(1.0, 1.0)] * 3, 6, B.GBS_F32_STATE_F64_COMBINE, k, r, S.GBS_8_6, y, 2)
    out = torch.empty_like(y)
    pb = B.make_problem(B.GBS_ACOUSTIC, 2, 6, B.GBS_F32_STATE_F64_COMBINE, xyz, [(1.0, 1.0)] * 3)
    _noalloc(pb, k, r, S.GBS_8_6, y, out, H, 2)
    assert _rel(out, ref) <= TOL


def test_noalloc_fp64_states_match_handle_path():
    shape = (28, 44)
    y0, kappa, rho = inputs.acoustic_problem(shape, 61, 3, 5.0)
    t = lambda a: torch.tensor(a.ravel(), dtype=torch.float64, device="cuda")
    y, k, r = t(y0), t(kappa), t(rho)
    ref, H = _handle(B.GBS_ACOUSTIC, [shape[::-1]], [(1.0, 1.0)], 4, B.GBS_F64, k, r, S.GBS_8_6, y, 2)
    out = torch.empty_like(y)
    pb = B.make_problem(B.GBS_ACOUSTIC, 2, 4, B.GBS_F64, [shape[::-1]], [(1.0, 1.0)])
    _noalloc(pb, k, r, S.GBS_8_6, y, out, H, 2)
    assert _rel(out, ref) <= 1e-12


def test_noalloc_wave1d_and_3d_match_handle_path():
    y0, dx = inputs.wave1d_initial(256)
    y = torch.tensor(y0.ravel(), dtype=torch.float64, device="cuda")
    ref, H = _handle(B.GBS_WAVE1D, [(256,)], [(dx,)], 4, B.GBS_F64, None, None, S.SQ8_2468, y, 5)
    out = torch.empty_like(y)
    pb = B.make_problem(B.GBS_WAVE1D, 1, 4, B.GBS_F64, [(256,)], [(dx,)])
    _noalloc(pb, None, None, S.SQ8_2468, y, out, H, 5)
    assert _rel(out, ref) <= 1e-12
    shape = (10, 12, 16)                             # (nz, ny, nx)
    y0, kappa, rho = inputs.acoustic_problem(shape, 71, 3, 3.0)
    t = lambda a: torch.tensor(a.astype(np.float32).ravel(), device="cuda")
    y, k, r = t(y0), t(kappa), t(rho)
    ref, H = _handle(B.GBS_ACOUSTIC, [shape[::-1]], [(1.0,) * 3], 4, B.GBS_F32_STATE_F64_COMBINE, k, r, S.GBS_8_6,
                     y, 2)
    out = torch.empty_like(y)
    pb = B.make_problem(B.GBS_ACOUSTIC, 3, 4, B.GBS_F32_STATE_F64_COMBINE, [shape[::-1]], [(1.0,) * 3])
    _noalloc(pb, k, r, S.GBS_8_6, y, out, H, 2)
    assert _rel(out, ref) <= TOL


def test_noalloc_zero_macro_steps_copies_the_state():
    shape = (20, 24)
    y, k, r = _problem(shape, 81)
    out = torch.full_like(y, -7.0)
    pb = B.make_problem(B.GBS_ACOUSTIC, 2, 6, B.GBS_F32_STATE_F64_COMBINE, [shape[::-1]], [(1.0, 1.0)])
    _noalloc(pb, k, r, S.GBS_8_6, y, out, 0.5, 0)
    assert torch.equal(out, y)


def test_noalloc_and_set_weights_refuse_the_same_broken_scheme():
    # a free weight so large that the dependent weights overflow: both entry points solve the
    # order constraints the same way (Sec. 3.7) and refuse the scheme with GBS_ERR_ORDER
    order, dep, free, cfree = 4, (2, 4), (6,), (1.7e308,)
    shape = (16, 16)
    y, k, r = _problem(shape, 91)
    pb = B.make_problem(B.GBS_ACOUSTIC, 2, 6, B.GBS_F32_STATE_F64_COMBINE, [shape[::-1]], [(1.0, 1.0)])
    with pytest.raises(B.GbsError) as e:
        B.gbs_step_noalloc(pb, k, r, order, dep, free, cfree, y, torch.empty_like(y), 0.1, 1,
                           torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 2, B.gbs_noalloc_last_error()
    sol = GBSSolver(B.GBS_ACOUSTIC, [shape[::-1]], [(1.0, 1.0)], fd_order=6,
                    precision=B.GBS_F32_STATE_F64_COMBINE, kappa=k, rho=r)
    with pytest.raises(B.GbsError) as e2:
        B.gbs_set_weights(sol.h, 0, order, dep, free, cfree)
    assert e2.value.status == 2
    sol.close()


def test_noalloc_refuses_a_capturing_stream_and_works_after():
    shape = (16, 20)
    y, k, r = _problem(shape, 93)
    pb = B.make_problem(B.GBS_ACOUSTIC, 2, 6, B.GBS_F32_STATE_F64_COMBINE, [shape[::-1]], [(1.0, 1.0)])
    out = torch.empty_like(y)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(B.GbsError) as e:
        with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
            B.gbs_step_noalloc(pb, k, r, S.GBS_8_6.order, S.GBS_8_6.steps_dep, S.GBS_8_6.steps_free,
                               S.GBS_8_6.c_free, y, out, 0.5, 1, side.cuda_stream)
    assert e.value.status == 8 and "captured" in B.gbs_noalloc_last_error()
    torch.cuda.synchronize()
    ref, H = _handle(B.GBS_ACOUSTIC, [shape[::-1]], [(1.0, 1.0)], 6, B.GBS_F32_STATE_F64_COMBINE, k, r, S.GBS_8_6, y, 1)
    _noalloc(pb, k, r, S.GBS_8_6, y, out, H, 1)
    assert _rel(out, ref) <= TOL
