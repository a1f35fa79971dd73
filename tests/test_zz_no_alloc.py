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
