"""GBS_F32X2: FP64 states, FP32-pair arithmetic on the FP32 units.

Tolerance (relative L2 over the state): 1e-10.  The FP64 path is held to 1e-12; pair
arithmetic has a unit roundoff near 2^-47 (hi + lo carry about 48 significant bits; the sums
and products are error-free transformations renormalised once), 64 times FP64's 2^-53, so the
same bar scaled by 64 is 6.4e-11, rounded up to 1e-10.  The FP32-state path, by contrast,
floors near 1e-5 (its stencil is FP32 arithmetic), which the accuracy test shows directly.
"""
import numpy as np
import pytest
import torch

from oracle import gbs as OG
from oracle import mol as OM
from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import inputs
from paper_1907_11771_gb300 import schemes as S
from paper_1907_11771_gb300.solver import GBSSolver
from tests.gpu_common import AcousticCase, oracle_scheme, rel_l2

pytestmark = pytest.mark.gpu
X2, F64, F32 = B.GBS_F32X2, B.GBS_F64, B.GBS_F32_STATE_F64_COMBINE
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("scheme", [S.GBS_8_6, S.SQ8_2468])
@pytest.mark.parametrize("shape", [(37, 53), (40, 68)])   # point-by-point and vector staging
def test_acoustic2d_parity(order, scheme, shape):
    case = AcousticCase(shape, order, X2, seed=3)
    sol = case.solver()
    sol.set_scheme(scheme)
    assert sol.uses_fused()                      # the default for 2D pairs: the time-blocked kernel
    sol.set_option("kernel", B.GBS_KERNEL_PLAIN)
    assert not sol.uses_fused()
    H = 0.8 * sol.stability_limit()[0]
    steps, c = oracle_scheme(scheme)
    err = rel_l2(case.gpu_run(sol, H, 3), case.oracle_run(steps, c, H, 3))
    assert err <= TOL, err
    sol.close()


def test_acoustic3d_and_1d_parity():
    for shape, order, scheme, n in (((11, 14, 19), 4, S.GBS_8_6, 2), ((11, 14, 20), 4, S.GBS_8_6, 2),
                                    ((45,), 6, S.GBS_12_8, 4)):
        case = AcousticCase(shape, order, X2, seed=5)
        sol = case.solver()
        sol.set_scheme(scheme)
        H = (0.8 if len(shape) > 1 else 0.5) * sol.stability_limit()[0]
        steps, c = oracle_scheme(scheme)
        err = rel_l2(case.gpu_run(sol, H, n), case.oracle_run(steps, c, H, n))
        assert err <= TOL, (shape, err)
        sol.close()


def test_wave1d_parity():
    n = 256
    y0, dx = inputs.wave1d_initial(n)
    sol = GBSSolver(B.GBS_WAVE1D, [(n,)], [(dx,)], fd_order=4, precision=X2)
    sol.set_scheme(S.SQ8_2468)
    H, M = 2 * np.pi / 114, 20
    y = torch.tensor(y0.ravel(), dtype=torch.float64, device="cuda")
    out = torch.empty_like(y)
    sol.step(y, out, H, M)
    sol.sync()
    steps, c = oracle_scheme(S.SQ8_2468)
    o = OG.gbs_run(lambda v: OM.rhs_wave1d(v, dx, 4), y0, H, steps, c, M)
    assert rel_l2(out.cpu().numpy().reshape(2, n), o) <= TOL
    sol.close()


def test_batch_mixed_slots():
    cases = [AcousticCase(s, 6, X2, seed=20 + i) for i, s in enumerate([(24, 40), (33, 17), (16, 16)])]
    kappa = torch.tensor(np.concatenate([c.kappa.ravel() for c in cases]), dtype=torch.float64, device="cuda")
    rho = torch.tensor(np.concatenate([c.rho.ravel() for c in cases]), dtype=torch.float64, device="cuda")
    sol = GBSSolver(B.GBS_ACOUSTIC, [c.shape_xyz for c in cases], [(1.0, 1.0)] * 3, fd_order=6, precision=X2,
                    kappa=kappa, rho=rho)
    sol.set_scheme(S.GBS_8_6, slot=0)
    sol.set_scheme(S.SQ8_2468, slot=1)
    sol.assign_slots([0, 1, 0])
    Hs = [0.7 * h for h in sol.stability_limit()]
    y0 = np.concatenate([c.y0.ravel() for c in cases])
    y = torch.tensor(y0, dtype=torch.float64, device="cuda")
    out = torch.empty_like(y)
    sol.step(y, out, Hs, 2)
    sol.sync()
    g = out.cpu().numpy()
    off = 0
    for i, c in enumerate(cases):
        n = c.y0.size
        steps, cw = oracle_scheme(S.GBS_8_6 if i != 1 else S.SQ8_2468)
        o = c.oracle_run(steps, cw, Hs[i], 2)
        assert rel_l2(g[off:off + n].reshape(c.y0.shape), o) <= TOL, i
        off += n
    sol.close()


def test_pairs_remove_the_fp32_floor():
    """Many macro-steps of the same problem: the FP32-pair state stays within a few 1e-13 of
    the FP64 path while the FP32 state drifts to about 1e-6 and beyond."""
    res = {}
    for prec in (F64, X2, F32):
        case = AcousticCase((64, 64), 6, prec, seed=11)
        sol = case.solver()
        sol.set_scheme(S.GBS_8_6)
        H = 0.8 * sol.stability_limit()[0]
        res[prec] = case.gpu_run(sol, H, 40)
        sol.close()
    e_x2 = rel_l2(res[X2], res[F64])
    e_32 = rel_l2(res[F32], res[F64])
    assert e_x2 <= TOL, e_x2
    assert e_32 > 1e3 * e_x2, (e_32, e_x2)


def test_adjoint_of_a_pair_handle_matches_the_fp64_adjoint():
    # the pair handle's adjoint runs in FP32-pair arithmetic (about 2^-44 per operation): one
    # adjoint macro-step agrees with the FP64 handle's to that rounding level
    res = []
    for prec in (F64, X2):
        case = AcousticCase((20, 24), 4, prec, seed=12, const_rho=True)
        sol = case.solver(enable_adjoint=True)
        sol.set_scheme(S.GBS_8_6)
        H = 0.8 * sol.stability_limit()[0]
        y = torch.tensor(case.y0.ravel(), dtype=torch.float64, device="cuda")
        lam = torch.tensor(np.random.default_rng(1).standard_normal(case.y0.size), device="cuda")
        li = torch.empty_like(lam)
        g = torch.zeros(case.y0[0].size, dtype=torch.float64, device="cuda")
        sol.adjoint_step(y, lam, li, g, H)
        sol.sync()
        res.append((li.cpu().numpy(), g.cpu().numpy()))
        sol.close()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(res[1][0], res[0][0]) <= 1e-10
    assert rel(res[1][1], res[0][1]) <= 1e-9


def test_time_blocked_kernel_refused_for_fp64_states_and_3d_pairs():
    for shape, prec in (((64, 64), F64), ((8, 40, 40), X2)):
        case = AcousticCase(shape, 6, prec)
        sol = case.solver()
        sol.set_scheme(S.GBS_8_6)
        with pytest.raises(B.GbsError):
            sol.set_option("kernel", B.GBS_KERNEL_FUSED)
        sol.close()


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("scheme", [S.GBS_8_6, S.SQ8_2468])
@pytest.mark.parametrize("shape,hseg", [((60, 520), 32), ((45, 251), 256)])
def test_time_blocked_pairs_parity(order, scheme, shape, hseg):
    """The time-blocked kernel in FP32-pair arithmetic (passes of two levels) against the FP64
    oracle at the pair tolerance: several strips and row segments, ragged edges, odd nx."""
    case = AcousticCase(shape, order, X2, seed=7)
    sol = case.solver()
    sol.set_scheme(scheme)
    sol.set_option("kernel", B.GBS_KERNEL_FUSED)
    sol.set_option("hseg", hseg)
    assert sol.uses_fused()
    H = 0.8 * sol.stability_limit()[0]
    steps, c = oracle_scheme(scheme)
    fused = case.gpu_run(sol, H, 3)
    err = rel_l2(fused, case.oracle_run(steps, c, H, 3))
    assert err <= TOL, err
    sol.set_option("kernel", B.GBS_KERNEL_PLAIN)
    plain = case.gpu_run(sol, H, 3)
    assert rel_l2(fused, plain) <= TOL
    sol.close()
