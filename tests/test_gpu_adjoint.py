"""GPU parity of the discrete adjoint and of the autograd / checkpointing layer.

* receiver misfit J and dJ/dkappa over several macro-steps with two-level
  checkpointing (segments of C macro-steps, the last one partial) and with
  binomial checkpointing (s stored states) against the oracle's FP64
  misfit_and_gradient;
* dJ/dkappa against central finite differences of the GPU forward on 16 seeded
  directions (FP64 states);
* GBSStepFn / GBSMisfitFn through torch.autograd.
"""
import numpy as np
import pytest
import torch

from oracle import gbs as OG
from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import schemes as S
from paper_1907_11771_gb300.autograd import GBSMisfitFn, GBSStepFn, gbs_misfit_and_grad
from tests.gpu_common import AcousticCase, oracle_scheme, rel_l2

pytestmark = pytest.mark.gpu
F32, F64, X2 = B.GBS_F32_STATE_F64_COMBINE, B.GBS_F64, B.GBS_F32X2


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _setup(precision, shape=(24, 28), n_macro=7, seed=5):
    case = AcousticCase(shape, 4, precision, seed=seed, const_rho=True)
    sol = case.solver(enable_adjoint=True)
    sol.set_scheme(S.GBS_8_6)
    H = 0.7 * sol.stability_limit()[0]
    n = shape[0] * shape[1]
    rcv = np.array([3, 40, 41, 200, n - 5, 333], dtype=np.int64)
    rng = np.random.default_rng(seed)
    data = (0.05 * rng.standard_normal((n_macro, rcv.size))).astype(case.np_dtype).astype(np.float64)
    dt = torch.float32 if precision == F32 else torch.float64
    t = dict(y0=torch.tensor(case.y0.ravel(), dtype=dt, device="cuda"),
             rcv=torch.tensor(rcv, device="cuda"),
             data=torch.tensor(data, dtype=dt, device="cuda"))
    return case, sol, H, rcv, data, t


@pytest.mark.parametrize("precision,ckpt,snaps", [(F64, 3, None), (F64, 100, None), (F32, 3, None),
                                                 (F64, None, 2), (F64, None, 3), (F32, None, 2)])
def test_misfit_gradient_with_checkpointing_matches_oracle(precision, ckpt, snaps):
    n_macro = 7
    case, sol, H, rcv, data, t = _setup(precision, n_macro=n_macro)
    J, g = gbs_misfit_and_grad(sol, t["y0"], H, n_macro, t["rcv"], t["data"], checkpoint_every=ckpt or 1,
                               snapshots=snaps)
    steps, c = oracle_scheme(S.GBS_8_6)
    oJ, og = OG.misfit_and_gradient(case.f, case.fT, case.pair, case.y0, H, steps, c, n_macro, rcv, data)
    tol = 1e-10 if precision == F64 else 2e-5
    assert J == pytest.approx(oJ, rel=tol)
    assert rel_l2(g.cpu().numpy(), og.ravel()) <= (1e-10 if precision == F64 else 1e-4)
    sol.close()


@pytest.mark.parametrize("ckpt,snaps", [(3, None), (None, 2)])
def test_pair_adjoint_matches_the_oracle_and_the_fp64_adjoint(ckpt, snaps):
    # FP64 states in FP32 pairs: the adjoint kernels run in pair arithmetic (about 2^-44 per
    # operation against FP64's 2^-53): the gradient agrees with the oracle's FP64 gradient and
    # with the FP64 handle's to the pair rounding level
    n_macro = 7
    case, sol, H, rcv, data, t = _setup(X2, n_macro=n_macro)
    J, g = gbs_misfit_and_grad(sol, t["y0"], H, n_macro, t["rcv"], t["data"], checkpoint_every=ckpt or 1,
                               snapshots=snaps)
    steps, c = oracle_scheme(S.GBS_8_6)
    oJ, og = OG.misfit_and_gradient(case.f, case.fT, case.pair, case.y0, H, steps, c, n_macro, rcv, data)
    assert J == pytest.approx(oJ, rel=1e-10)
    assert rel_l2(g.cpu().numpy(), og.ravel()) <= 1e-9
    case64, sol64, H64, _, _, t64 = _setup(F64, n_macro=n_macro)
    _, g64 = gbs_misfit_and_grad(sol64, t64["y0"], H64, n_macro, t64["rcv"], t64["data"],
                                 checkpoint_every=ckpt or 1, snapshots=snaps)
    assert rel_l2(g.cpu().numpy(), g64.cpu().numpy()) <= 1e-9
    sol.close()
    sol64.close()


def test_pair_adjoint_step_in_place_and_receivers():
    # lam_in written over lam_out, receiver residuals injected into the FP64 result
    case, sol, H, rcv, data, t = _setup(X2, n_macro=1)
    rng = np.random.default_rng(7)
    lam = torch.tensor(rng.standard_normal(case.y0.size), device="cuda")
    y = t["y0"]
    ref_in = torch.empty_like(lam)
    g1 = torch.zeros(case.kappa.size, dtype=torch.float64, device="cuda")
    g2 = torch.zeros_like(g1)
    resid = torch.tensor(rng.standard_normal(rcv.size), device="cuda")
    B.gbs_adjoint_step(sol.h, y, lam, ref_in, g1, H, t["rcv"], resid)
    lam2 = lam.clone()
    B.gbs_adjoint_step(sol.h, y, lam2, lam2, g2, H, t["rcv"], resid)
    sol.sync()
    assert torch.equal(lam2, ref_in) and torch.equal(g1, g2)
    steps, c = oracle_scheme(S.GBS_8_6)
    olam, og = OG.gbs_macro_step_adjoint(case.f, case.fT, case.pair, case.y0, lam.cpu().numpy().reshape(case.y0.shape),
                                         H, steps, c)
    olam = olam.ravel().copy()
    olam[rcv] += resid.cpu().numpy()
    assert rel_l2(ref_in.cpu().numpy(), olam) <= 1e-10
    assert rel_l2(g1.cpu().numpy(), og.ravel()) <= 1e-9
    sol.close()


@pytest.mark.parametrize("precision", [F64])
def test_misfit_gradient_central_differences_on_16_directions(precision):
    # the adjoint workload's check: dJ/dkappa against central differences on 16 seeded
    # directions to 1e-6 relative (FP64 states)
    n_macro = 4
    case, sol, H, rcv, data, t = _setup(precision, n_macro=n_macro)
    J, g = gbs_misfit_and_grad(sol, t["y0"], H, n_macro, t["rcv"], t["data"], checkpoint_every=2)
    g = g.cpu().numpy()
    rng = np.random.default_rng(3)
    base = case.kappa.ravel()
    for _ in range(16):
        d = rng.standard_normal(base.size)
        eps = 1e-6
        Js = []
        for sgn in (1, -1):
            k = torch.tensor(base + sgn * eps * d, dtype=torch.float64, device="cuda")
            sol.set_media(k, case.t_rho)
            Js.append(gbs_misfit_and_grad(sol, t["y0"], H, n_macro, t["rcv"], t["data"], 2)[0])
        fd = (Js[0] - Js[1]) / (2 * eps)
        assert np.dot(g, d) == pytest.approx(fd, rel=1e-6)
    sol.set_media(case.t_kappa, case.t_rho)
    sol.close()


@pytest.mark.parametrize("snaps", [1, 2, 3])
def test_autograd_step_with_binomial_checkpointing_equals_all_states(snaps):
    # the same adjoint macro-steps on the same (recomputed) states: identical gradients
    case, sol, H, rcv, data, t = _setup(F64, n_macro=3)
    kappa = case.t_kappa
    rng = np.random.default_rng(9)
    w = None
    grads = []
    for s in (None, snaps):
        y = t["y0"].clone().requires_grad_(True)
        kappa.grad = None
        kappa.requires_grad_(True)
        out = GBSStepFn.apply(y, kappa, sol, H, 6, s)
        if w is None:
            w = torch.tensor(rng.standard_normal(out.numel()), device="cuda")
        (out * w).sum().backward()
        grads.append((y.grad.clone(), kappa.grad.clone()))
    assert torch.equal(grads[0][0], grads[1][0]) and torch.equal(grads[0][1], grads[1][1])
    sol.close()


def test_autograd_step_and_misfit_functions():
    case, sol, H, rcv, data, t = _setup(F64, n_macro=3)
    # GBSStepFn: d<w, y_out>/dy_in and d/dkappa against the oracle adjoint of 2 macro-steps
    y = t["y0"].clone().requires_grad_(True)
    kappa = case.t_kappa
    kappa.requires_grad_(True)
    out = GBSStepFn.apply(y, kappa, sol, H, 2)
    rng = np.random.default_rng(0)
    w = torch.tensor(rng.standard_normal(out.numel()), device="cuda")
    (out * w).sum().backward()
    steps, c = oracle_scheme(S.GBS_8_6)
    y1 = OG.gbs_macro_step(case.f, case.y0, H, steps, c)
    lam1, g1 = OG.gbs_macro_step_adjoint(case.f, case.fT, case.pair, y1, w.cpu().numpy().reshape(case.y0.shape),
                                         H, steps, c)
    lam0, g0 = OG.gbs_macro_step_adjoint(case.f, case.fT, case.pair, case.y0, lam1, H, steps, c)
    assert rel_l2(y.grad.cpu().numpy(), lam0) <= 1e-11
    assert rel_l2(kappa.grad.cpu().numpy(), (g0 + g1).ravel()) <= 1e-10
    # GBSMisfitFn
    kappa.grad = None
    J = GBSMisfitFn.apply(kappa, sol, t["y0"], H, 3, t["rcv"], t["data"], 2)
    J.backward()
    _, og = OG.misfit_and_gradient(case.f, case.fT, case.pair, case.y0, H, steps, c, 3, rcv, data)
    assert rel_l2(kappa.grad.cpu().numpy(), og.ravel()) <= 1e-10
    sol.close()
