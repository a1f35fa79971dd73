"""GPU parity: the CUDA library (through the C ABI) against the FP64 CPU oracle.

Tolerances (relative L2 over the whole state): <= 1e-12 for the FP64 path and
<= 1e-5 for the FP32-state / FP64-combine path, the bounds the workloads are
specified with.  Grids are ragged (not multiples of any tile) and span many
thread blocks.
"""
import math

import numpy as np
import pytest
import torch

from oracle import gbs as OG
from oracle import mol as OM
from oracle import weights as OW
from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import inputs
from paper_1907_11771_gb300 import schemes as S
from paper_1907_11771_gb300.solver import GBSSolver
from tests.gpu_common import AcousticCase, oracle_scheme, rel_l2

pytestmark = pytest.mark.gpu

TOL = {B.GBS_F64: 1e-12, B.GBS_F32_STATE_F64_COMBINE: 1e-5}
F32, F64 = B.GBS_F32_STATE_F64_COMBINE, B.GBS_F64


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _ulps(a, b):
    return abs(a - b) / math.ulp(max(abs(a), abs(b)))


@pytest.mark.parametrize("scheme", [S.GBS_8_6, S.GBS_8_8, S.GBS_12_8, S.SQ8_TABLE1, S.SQ12_TABLE1,
                                    S.SQ16_TABLE1, S.SQ8_2468])
def test_weights_and_isb_match_oracle(scheme):
    """Dependent weights: the library solves them in double-double from the FP64-rounded free
    weights, so they must equal the exact rational solve of those same binary inputs to within
    2 ulp; against the paper's exact rationals they differ only by the rounding of c_free."""
    from fractions import Fraction
    from tests.gpu_common import GOLD, GOLD_OF
    case = AcousticCase((16, 16), 4, F64)
    sol = case.solver()
    sol.set_scheme(scheme)
    steps, c, isb = sol.weights()
    o_steps, o_c = oracle_scheme(scheme)
    assert steps == list(o_steps)
    n_dep = len(scheme.steps_dep)
    # same binary inputs, exact solve
    _, c_same = OW.scheme_weights(scheme.order, list(scheme.steps_dep), list(scheme.steps_free),
                                  [Fraction(v) for v in scheme.c_free])
    for a, b in zip(c, OW.to_fp64(c_same)):
        assert _ulps(a, b) <= 2, (a, b)
    # paper rationals: free weights identical, dependent ones within the propagated rounding
    scale = sum(abs(v) for v in o_c)
    for k, (a, b) in enumerate(zip(c, o_c)):
        if k >= n_dep:
            assert a == b
        else:
            assert abs(a - b) <= 4e-16 * scale, (k, a, b)
    if scheme.name in GOLD_OF:
        g = GOLD[GOLD_OF[scheme.name]]
        _, c_e = OW.scheme_weights(int(g["order"]), [int(t) for t in g["dep"].split()],
                                   [int(t) for t in g.get("free", "").split()],
                                   [Fraction(t) for t in g.get("cfree", "").split()])
    else:
        c_e = OW.square_weights(list(o_steps), scheme.order)
    isb_exact = OW.isb_exact(OW.stability_poly(o_steps, c_e))
    assert isb == pytest.approx(isb_exact, rel=1e-9)
    sol.close()


def test_wave1d_config1_fp64_parity_and_dalembert():
    n = 256
    y0, dx = inputs.wave1d_initial(n)
    steps, c = oracle_scheme(S.SQ8_2468)
    H, M = 2 * np.pi / 200, 200
    sol = GBSSolver(B.GBS_WAVE1D, [(n,)], [(dx,)], fd_order=4, precision=F64)
    sol.set_scheme(S.SQ8_2468)
    y = torch.tensor(y0.ravel(), dtype=torch.float64, device="cuda")
    out = torch.empty_like(y)
    sol.step(y, out, H, M)
    sol.sync()
    g = out.cpu().numpy().reshape(y0.shape)
    o = OG.gbs_run(lambda v: OM.rhs_wave1d(v, dx, 4), y0, H, steps, c, M)
    assert rel_l2(g, o) <= TOL[F64]
    # d'Alembert: the periodic solution at t = 2 pi equals the initial state; the error is
    # the 4th-order spatial error, identical for both implementations
    assert rel_l2(g, y0) == pytest.approx(rel_l2(o, y0), rel=1e-9)
    assert 3e-3 < rel_l2(g, y0) < 6e-3
    sol.close()


@pytest.mark.parametrize("precision", [F64, F32])
@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("scheme", [S.GBS_8_6, S.SQ8_2468])
@pytest.mark.parametrize("shape", [(37, 53), (40, 68)])   # nx odd: point-by-point staging; nx % 4 == 0: vectors
def test_acoustic2d_parity(precision, order, scheme, shape):
    case = AcousticCase(shape, order, precision, seed=3)
    sol = case.solver()
    sol.set_scheme(scheme)
    H = 0.8 * sol.stability_limit()[0]
    steps, c = oracle_scheme(scheme)
    g = case.gpu_run(sol, H, 3)
    o = case.oracle_run(steps, c, H, 3)
    err = rel_l2(g, o)
    assert err <= TOL[precision], err
    sol.close()


@pytest.mark.parametrize("precision", [F64, F32])
@pytest.mark.parametrize("shape", [(11, 14, 19), (11, 14, 20)])
def test_acoustic3d_parity(precision, shape):
    case = AcousticCase(shape, 4, precision, seed=5)
    sol = case.solver()
    sol.set_scheme(S.GBS_8_6)
    H = 0.8 * sol.stability_limit()[0]
    steps, c = oracle_scheme(S.GBS_8_6)
    err = rel_l2(case.gpu_run(sol, H, 2), case.oracle_run(steps, c, H, 2))
    assert err <= TOL[precision], err
    sol.close()


def test_acoustic1d_parity():
    case = AcousticCase((45,), 6, F64, seed=8)
    sol = case.solver()
    sol.set_scheme(S.GBS_12_8)
    H = 0.5 * sol.stability_limit()[0]
    steps, c = oracle_scheme(S.GBS_12_8)
    assert rel_l2(case.gpu_run(sol, H, 4), case.oracle_run(steps, c, H, 4)) <= TOL[F64]
    sol.close()


@pytest.mark.parametrize("precision", [F64, F32])
def test_batch_mixed_slots(precision):
    shapes_yx = [(24, 24), (40, 32), (17, 29), (8, 9)]
    cases = [AcousticCase(s, 6, precision, seed=20 + i) for i, s in enumerate(shapes_yx)]
    dt = torch.float64 if precision == F64 else torch.float32
    kappa = torch.tensor(np.concatenate([c.kappa.ravel() for c in cases]), dtype=dt, device="cuda")
    rho = torch.tensor(np.concatenate([c.rho.ravel() for c in cases]), dtype=dt, device="cuda")
    sol = GBSSolver(B.GBS_ACOUSTIC, [c.shape_xyz for c in cases], [(1.0, 1.0)] * len(cases), fd_order=6,
                    precision=precision, kappa=kappa, rho=rho)
    sol.set_scheme(S.GBS_8_6, slot=0)
    sol.set_scheme(S.SQ8_TABLE1, slot=1)
    slots = [0, 1, 0, 1]
    sol.assign_slots(slots)
    Hs = [0.7 * h for h in sol.stability_limit()]
    y = torch.tensor(np.concatenate([c.y0.ravel() for c in cases]), dtype=dt, device="cuda")
    out = torch.empty_like(y)
    sol.step(y, out, Hs, 2)
    sol.sync()
    g = out.double().cpu().numpy()
    off = 0
    for i, c in enumerate(cases):
        n = c.y0.size
        steps, cw = oracle_scheme(S.GBS_8_6 if slots[i] == 0 else S.SQ8_TABLE1)
        o = c.oracle_run(steps, cw, Hs[i], 2)
        assert rel_l2(g[off:off + n], o) <= TOL[precision], i
        off += n
    sol.close()


def test_in_place_zero_steps_graph_and_host_paths():
    case = AcousticCase((33, 30), 4, F32, seed=4)
    sol = case.solver()
    sol.set_scheme(S.GBS_8_6)
    H = 0.8 * sol.stability_limit()[0]
    y = torch.tensor(case.y0.ravel(), dtype=torch.float32, device="cuda")
    out = torch.empty_like(y)
    sol.step(y, out, H, 3)
    # in place
    z = y.clone()
    sol.step(z, z, H, 3)
    # without graph replay
    sol.set_option("graph", 0)
    w = torch.empty_like(y)
    sol.step(y, w, H, 3)
    sol.set_option("graph", 1)
    # zero steps copy
    c0 = torch.empty_like(y)
    sol.step(y, c0, H, 0)
    # host buffers (end-to-end entry point)
    hin = y.cpu().numpy().copy()
    hout = np.empty_like(hin)
    sol.step_host(hin, hout, H, 3)
    sol.sync()
    assert torch.equal(out, z)
    assert torch.equal(out, w)
    assert torch.equal(c0, y)
    assert np.array_equal(hout, out.cpu().numpy())
    assert sol.kernel_launches > 0
    sol.close()


def test_error_reporting():
    case = AcousticCase((16, 16), 4, F64)
    sol = case.solver()
    y = torch.zeros(sol.state_elems, dtype=torch.float64, device="cuda")
    with pytest.raises(B.GbsError) as e:
        sol.step(y, y, 0.1, 1)             # no weights yet
    assert e.value.status == 8
    with pytest.raises(B.GbsError) as e:
        B.gbs_set_weights(sol.h, 0, 8, [2, 4, 6, 7])   # odd step count
    assert e.value.status == 1
    with pytest.raises(B.GbsError) as e:
        B.gbs_set_weights(sol.h, 0, 8, [2, 4, 6, 8], c_full=[-1 / 360, 16 / 45, -729 / 280, 1024 / 315 + 1e-9])
    assert e.value.status == 2
    with pytest.raises(B.GbsError) as e:
        B.gbs_set_weights(sol.h, 0, 8, [2, 4, 6, 6])
    assert e.value.status == 1
    sol.set_scheme(S.SQ8_2468)
    with pytest.raises(B.GbsError):
        sol.step(y, y, -1.0, 1)
    with pytest.raises(B.GbsError):
        sol.step(y, y[1:], 0.1, 1)          # partial overlap
    sol.set_option("check_stability", 1)
    with pytest.raises(B.GbsError) as e:
        sol.step(y, y, 1.01 * sol.stability_limit()[0], 1)
    assert e.value.status == 3
    sol.close()


def test_stability_limit_bounds_spectral_radius():
    case = AcousticCase((24, 20), 6, F64, seed=2)
    sol = case.solver()
    sol.set_scheme(S.GBS_8_6)
    Hmax = sol.stability_limit()[0]
    _, _, isb = sol.weights()
    rho_hat = isb / Hmax
    rho = OM.power_iteration_rho(case.f, case.y0.shape, iters=400)
    assert rho <= rho_hat * (1 + 1e-9)
    assert rho >= 0.5 * rho_hat
    sol.close()


@pytest.mark.parametrize("precision", [F64, F32])
@pytest.mark.parametrize("shape,order", [((20, 23), 4), ((45, 70), 6), ((9, 10, 11), 4), ((20, 24), 4),
                                         ((40, 68), 6), ((9, 10, 12), 4)])
def test_adjoint_parity(precision, shape, order):
    # one tile; several 32 x 32 tiles with ragged edges; 3D (z-stencils through the cache); each
    # with an odd nx and with nx % 4 == 0 (vector staging of the forward recompute)
    case = AcousticCase(shape, order, precision, seed=6)
    sol = case.solver(enable_adjoint=True)
    sol.set_scheme(S.GBS_8_6)
    H = 0.8 * sol.stability_limit()[0]
    steps, c = oracle_scheme(S.GBS_8_6)
    rng = np.random.default_rng(1)
    lam = rng.standard_normal(case.y0.shape).astype(case.np_dtype).astype(np.float64)
    rcv = np.array([5, 77, 300, 301], dtype=np.int64) % case.y0[0].size
    resid = rng.standard_normal(4).astype(case.np_dtype).astype(np.float64)
    o_lam, o_g = OG.gbs_macro_step_adjoint(case.f, case.fT, case.pair, case.y0, lam, H, steps, c)
    o_lam = o_lam + OG.inject_receivers(case.y0.shape, rcv, resid)
    dt = torch.float64 if precision == F64 else torch.float32
    ty = torch.tensor(case.y0.ravel(), dtype=dt, device="cuda")
    tl = torch.tensor(lam.ravel(), dtype=dt, device="cuda")
    out = torch.empty_like(tl)
    g = torch.zeros(case.y0[0].size, dtype=torch.float64, device="cuda")
    ridx = torch.tensor(rcv, device="cuda")
    rres = torch.tensor(resid, dtype=dt, device="cuda")
    sol.adjoint_step(ty, tl, out, g, H, ridx, rres)
    sol.sync()
    assert rel_l2(out.double().cpu().numpy(), o_lam) <= TOL[precision]
    gtol = 1e-11 if precision == F64 else 2e-5
    assert rel_l2(g.cpu().numpy(), o_g.ravel()) <= gtol
    # in place (lam_in aliases lam_out), gradient accumulates
    sol.adjoint_step(ty, tl, tl, g, H, ridx, rres)
    sol.sync()
    assert rel_l2(tl.double().cpu().numpy(), o_lam) <= TOL[precision]
    assert rel_l2(g.cpu().numpy(), 2 * o_g.ravel()) <= gtol
    sol.close()


def test_norms_and_misfit():
    case = AcousticCase((31, 17), 4, F64, seed=9)
    sol = case.solver()
    rng = np.random.default_rng(3)
    a = rng.standard_normal(case.y0.size)
    b = rng.standard_normal(case.y0.size)
    ta = torch.tensor(a, device="cuda")
    tb = torch.tensor(b, device="cuda")
    s2, b2, mx, nf = sol.norms(ta, tb)
    assert s2 == pytest.approx(np.sum((a - b) ** 2), rel=1e-13)
    assert b2 == pytest.approx(np.sum(b ** 2), rel=1e-13)
    assert mx == np.max(np.abs(a - b))
    assert nf == 0
    ta[7] = float("nan")
    assert sol.norms(ta, tb)[3] == 1
    idx = torch.tensor([0, 5, 99, 400], device="cuda")
    data = torch.tensor(rng.standard_normal(4), device="cuda")
    resid = torch.empty(4, dtype=torch.float64, device="cuda")
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    sol.misfit(tb, idx, data, resid, J)
    sol.sync()
    r = b[[0, 5, 99, 400]] - data.cpu().numpy()
    np.testing.assert_allclose(resid.cpu().numpy(), r, rtol=0, atol=0)
    assert J.item() == pytest.approx(0.5 * np.sum(r ** 2), rel=1e-14)
    sol.close()


def test_full_size_2048_sampled_points():
    """2D acoustics 2048^2, 6th order, GBS_{8,6}, FP32 state: one macro-step in the
    launch configuration the benchmark uses, checked at sampled points against the
    oracle run on periodic patches that contain each point's domain of dependence
    (radius 3 x 23 = 69 cells for the longest sequence)."""
    n = 2048
    y0, kappa, rho = inputs.acoustic_problem((n, n), 0, 16, 20.0)
    y0 = y0.astype(np.float32)
    kappa = kappa.astype(np.float32)
    rho = rho.astype(np.float32)
    tk = torch.tensor(kappa.ravel(), device="cuda")
    tr = torch.tensor(rho.ravel(), device="cuda")
    sol = GBSSolver(B.GBS_ACOUSTIC, [(n, n)], [(1.0, 1.0)], fd_order=6, precision=F32, kappa=tk, rho=tr)
    sol.set_scheme(S.GBS_8_6)
    H = 0.8 * sol.stability_limit()[0]
    y = torch.tensor(y0.ravel(), device="cuda")
    out = torch.empty_like(y)
    sol.step(y, out, H, 1)
    sol.sync()
    g = out.cpu().numpy().reshape(y0.shape)
    steps, c = oracle_scheme(S.GBS_8_6)
    half = 80
    rng = np.random.default_rng(0)
    pts = [(n // 2, n // 2), (0, 0), (n - 1, 5), (17, n - 2)] + [tuple(rng.integers(0, n, 2)) for _ in range(4)]
    scale = np.abs(g).max()
    for (py, px) in pts:
        iy = (np.arange(py - half, py + half) % n)
        ix = (np.arange(px - half, px + half) % n)
        sub = lambda a: a[np.ix_(iy, ix)].astype(np.float64)
        ky, kk, kr = sub(y0[0]), sub(kappa), sub(rho)
        yy = np.stack([sub(y0[f]) for f in range(3)])
        f = lambda v: OM.rhs_acoustic(v, kk, 1.0 / kr, [1.0, 1.0], 6)
        o = OG.gbs_macro_step(f, yy, H, steps, c)
        err = np.max(np.abs(o[:, half, half] - g[:, py, px]))
        assert err <= 1e-5 * scale, (py, px, err)
    sol.close()


def test_workspace_allocation_failure_is_reported():
    """A batch far larger than the device: gbs_create's cudaMalloc fails and the call
    returns GBS_ERR_NOMEM with a message instead of aborting."""
    n = 40000
    pb = B.make_problem(B.GBS_ACOUSTIC, 2, 4, F64, [(n, n)] * 40, [(1.0, 1.0)] * 40)
    k = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(B.GbsError) as e:
        B.gbs_create(pb, k, k)
    assert e.value.status == 5
    assert "cudaMalloc" in B.gbs_last_error(None)


@pytest.mark.parametrize("kernel", ["plain", "fused"])
@pytest.mark.parametrize("steps", [(2,), (4,), (2, 4)])
def test_degenerate_schemes(kernel, steps):
    """One sequence with c = 1 (order 2: plain GBS, no extrapolation) and the smallest square
    scheme {2, 4} (order 4, Richardson weights -1/3, 4/3), on the FP64 plain kernels and on the
    FP32 time-blocked kernel (whose first pass is then also its last)."""
    prec = F64 if kernel == "plain" else F32
    case = AcousticCase((64, 72), 6, prec, seed=21)
    sol = case.solver()
    order = 2 * len(steps)
    B.gbs_set_weights(sol.h, 0, order, list(steps), [], [])
    if kernel == "fused":
        sol.set_option("kernel", B.GBS_KERNEL_FUSED)
        assert sol.uses_fused()
    H = 0.5 * sol.stability_limit()[0] if sol.weights()[2] > 0 else 0.05
    c = OW.to_fp64(OW.square_weights(list(steps), order))
    err = rel_l2(case.gpu_run(sol, H, 3), case.oracle_run(list(steps), c, H, 3))
    assert err <= TOL[prec], err
    sol.close()
