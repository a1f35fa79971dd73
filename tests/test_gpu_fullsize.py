"""Full-size parity on sampled outputs.

One macro-step (or adjoint macro-step) of each workload at its full size runs on
the GPU; the oracle then recomputes sampled output points exactly on periodic
patches around them that contain each point's whole domain of dependence
(radius R x (N_max + 1) cells: every right-hand side evaluation widens it by
R), so the patch's own wrap-around never reaches the sample.

* 3D acoustics 512^3, 4th order, 64-Gaussian media, 3 pulses (FP32 state)
* 256 independent 2D problems, sides drawn from {128, ..., 1024}, the optimised order-8
  GBS_{8,6} and order-6 GBS_{6,6} schemes alternating
* adjoint: 2D 1024^2, 4th order, constant rho (FP32 state), lambda_in and
  dJ/dkappa at sampled points
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
from tests.gpu_common import oracle_scheme

pytestmark = pytest.mark.gpu
F32 = B.GBS_F32_STATE_F64_COMBINE


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _patch(a, center, half):
    """Periodic patch of array a (grid axes last) of width 2*half around center (grid order)."""
    idx = [(np.arange(c - half, c + half) % n) for c, n in zip(center, a.shape[-len(center):])]
    return a[(Ellipsis,) + np.ix_(*idx)]


def test_3d_512_one_macro_step_sampled():
    n = 512
    y0, kappa, rho = inputs.acoustic_problem((n, n, n), 0, 64, 4.0, n_pulses=3, centred=False, dtype=np.float32)
    tk = torch.from_numpy(kappa.ravel()).cuda()
    tr = torch.from_numpy(rho.ravel()).cuda()
    sol = GBSSolver(B.GBS_ACOUSTIC, [(n, n, n)], [(1.0, 1.0, 1.0)], fd_order=4, precision=F32, kappa=tk, rho=tr)
    checks = []
    for scheme, half, npts in ((S.SQ8_2468, 20, 4), (S.GBS_8_6, 48, 1)):
        sol.set_scheme(scheme)
        H = 0.8 * sol.stability_limit()[0]
        y = torch.from_numpy(y0.ravel()).cuda()
        out = torch.empty_like(y)
        sol.step(y, out, H, 1)
        sol.sync()
        g = out.cpu().numpy().reshape(y0.shape)
        steps, c = oracle_scheme(scheme)
        rng = np.random.default_rng(1)
        pts = [(0, 0, 0)] + [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(npts - 1)]
        scale = np.abs(g).max()
        for p in pts:
            yy = _patch(y0, p, half).astype(np.float64)
            kk = _patch(kappa, p, half).astype(np.float64)
            rr = _patch(rho, p, half).astype(np.float64)
            o = OG.gbs_macro_step(lambda v: OM.rhs_acoustic(v, kk, 1.0 / rr, [1.0] * 3, 4), yy, H, steps, c)
            err = np.max(np.abs(o[:, half, half, half] - g[(slice(None),) + p]))
            checks.append(err / scale)
            assert err <= 1e-5 * scale, (scheme.name, p, err)
        del y, out
    sol.close()


def test_batch_256_problems_one_macro_step_sampled():
    sides = inputs.batch_sides(256, 0)
    probs = [inputs.acoustic_problem((s, s), 1000 + i, 16, 20.0 * s / 2048, dtype=np.float32)
             for i, s in enumerate(sides)]
    kappa = torch.from_numpy(np.concatenate([p[1].ravel() for p in probs])).cuda()
    rho = torch.from_numpy(np.concatenate([p[2].ravel() for p in probs])).cuda()
    sol = GBSSolver(B.GBS_ACOUSTIC, [(s, s) for s in sides], [(1.0, 1.0)] * len(sides), fd_order=6,
                    precision=F32, kappa=kappa, rho=rho)
    sol.set_scheme(S.GBS_8_6, slot=0)
    sol.set_scheme(S.GBS_6_6, slot=1)
    slots = [i % 2 for i in range(len(sides))]
    sol.assign_slots(slots)
    assert sol.uses_fused()
    Hs = [0.8 * h for h in sol.stability_limit()]
    y = torch.from_numpy(np.concatenate([p[0].ravel() for p in probs])).cuda()
    out = torch.empty_like(y)
    sol.step(y, out, Hs, 1)
    sol.sync()
    g = out.cpu().numpy()
    offs = np.cumsum([0] + [3 * s * s for s in sides])
    rng = np.random.default_rng(2)
    half = 72
    for i in (0, 1, 100, 255):
        s = sides[i]
        gi = g[offs[i]:offs[i + 1]].reshape(3, s, s)
        y0, kap, rh = (a.astype(np.float64) for a in probs[i])
        steps, c = oracle_scheme(S.GBS_8_6 if slots[i] == 0 else S.GBS_6_6)
        scale = np.abs(gi).max()
        for _ in range(2):
            p = tuple(int(v) for v in rng.integers(0, s, 2))
            yy, kk, rr = _patch(y0, p, half), _patch(kap, p, half), _patch(rh, p, half)
            o = OG.gbs_macro_step(lambda v: OM.rhs_acoustic(v, kk, 1.0 / rr, [1.0, 1.0], 6), yy, Hs[i], steps, c)
            err = np.max(np.abs(o[:, half, half] - gi[(slice(None),) + p]))
            assert err <= 1e-5 * scale, (i, p, err)
    sol.close()


def test_adjoint_1024_sampled():
    n = 1024
    y0, kappa, rho = inputs.acoustic_problem((n, n), 0, 16, 8.0, const_rho=True, dtype=np.float32)
    rng = np.random.default_rng(4)
    lam = np.zeros_like(y0)
    lam[0] = inputs.gaussian_pulses((n, n), 30.0, [[n / 3, n / 2]]).astype(np.float32)
    lam[1] = 0.5 * inputs.gaussian_pulses((n, n), 30.0, [[n / 2, n / 3]]).astype(np.float32)
    tk = torch.from_numpy(kappa.ravel()).cuda()
    tr = torch.from_numpy(rho.ravel()).cuda()
    sol = GBSSolver(B.GBS_ACOUSTIC, [(n, n)], [(1.0, 1.0)], fd_order=4, precision=F32, kappa=tk, rho=tr,
                    enable_adjoint=True)
    sol.set_scheme(S.GBS_8_6)
    H = 0.8 * sol.stability_limit()[0]
    ty = torch.from_numpy(y0.ravel()).cuda()
    tl = torch.from_numpy(lam.ravel()).cuda()
    li = torch.empty_like(tl)
    g = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    sol.adjoint_step(ty, tl, li, g, H)
    sol.sync()
    li = li.cpu().numpy().reshape(y0.shape)
    g = g.cpu().numpy().reshape(n, n)
    steps, c = oracle_scheme(S.GBS_8_6)
    half = 100
    lscale, gscale = np.abs(li).max(), np.abs(g).max()
    for p in [(n // 3, n // 2), (n // 2, n // 3), tuple(int(v) for v in rng.integers(0, n, 2))]:
        yy = _patch(y0, p, half).astype(np.float64)
        ll = _patch(lam, p, half).astype(np.float64)
        kk = _patch(kappa, p, half).astype(np.float64)
        b = np.ones_like(kk)
        f = lambda v: OM.rhs_acoustic(v, kk, b, [1.0, 1.0], 4)
        fT = lambda v: OM.rhs_acoustic_T(v, kk, b, [1.0, 1.0], 4)
        pair = lambda mu, v: OM.dA_dkappa_pairing(mu, v, [1.0, 1.0], 4)
        ol, og = OG.gbs_macro_step_adjoint(f, fT, pair, yy, ll, H, steps, c)
        assert np.max(np.abs(ol[:, half, half] - li[(slice(None),) + p])) <= 1e-5 * lscale, p
        assert abs(og[half, half] - g[p]) <= 1e-5 * gscale, p
    sol.close()
