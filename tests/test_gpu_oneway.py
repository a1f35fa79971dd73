"""The one-way wave with spectral derivatives (Sec. 4) on the GPU: parity with the FP64 oracle,
the stability bound, a batch of sizes and schemes, and Sec. 4's run (lambda = dt/dx =
0.99 ISB / pi, once around the interval) against the oracle's error at every refinement level.

Tolerances: relative L2 1e-11 for parity.  Both sides are FP64, but every evaluation passes
through two FFTs that round differently from numpy's (about log2(n) u each), and the
extrapolation amplifies rounding by sum|c_k| (31 for GBS_8,6) over the 143 evaluations of a
macro-step: a few 1e-12 per macro-step at n = 64, against 1e-12 for the stencil paths.  For the
errors of Sec. 4's run: 1% of the error or the FP64 rounding floor of the run, about
1e-16 sum|c_k| per macro-step."""
import numpy as np
import pytest
import torch

from oracle import gbs as OG
from oracle import mol as OM
from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import schemes as S
from paper_1907_11771_gb300.solver import GBSSolver
from tests.gpu_common import oracle_scheme, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _u0(n):
    x = np.arange(n) / n
    return 0.5 * (1 - np.cos(2 * np.pi * x))


def _solver(ns, schemes=None):
    sol = GBSSolver(B.GBS_ONEWAY_SPECTRAL, [(n,) for n in ns], [(1.0 / n,) for n in ns], fd_order=0,
                    precision=B.GBS_F64)
    return sol


def test_parity_and_stability_bound():
    n = 64
    sol = _solver([n])
    sol.set_scheme(S.GBS_8_6)
    Hlim = sol.stability_limit()[0]
    steps, c = oracle_scheme(S.GBS_8_6)
    isb = sol.weights()[2]
    assert Hlim == pytest.approx(isb / (np.pi * n), rel=1e-12)
    rng = np.random.default_rng(3)
    y0 = rng.standard_normal(n)                   # every mode, not only the paper's one
    H = 0.9 * Hlim
    y = torch.tensor(y0, dtype=torch.float64, device="cuda")
    out = torch.empty_like(y)
    sol.step(y, out, H, 5)
    sol.sync()
    o = OG.gbs_run(lambda v: OM.rhs_oneway_spectral(v, 1.0 / n), y0[None, :], H, steps, c, 5)[0]
    assert rel_l2(out.cpu().numpy(), o) <= 1e-11
    sol.close()


def test_batch_of_sizes_and_schemes_in_place():
    ns = [16, 64, 256, 2048]
    sol = _solver(ns)
    sol.set_scheme(S.GBS_8_6, slot=0)
    sol.set_scheme(S.GBS_12_8, slot=1)
    slots = [0, 1, 1, 0]
    sol.assign_slots(slots)
    Hs = [0.8 * h for h in sol.stability_limit()]
    rng = np.random.default_rng(4)
    y0s = [rng.standard_normal(n) for n in ns]
    y = torch.tensor(np.concatenate(y0s), dtype=torch.float64, device="cuda")
    sol.step(y, y, Hs, 3)
    sol.sync()
    g = y.cpu().numpy()
    off = 0
    for n, y0, sl, H in zip(ns, y0s, slots, Hs):
        steps, c = oracle_scheme(S.GBS_8_6 if sl == 0 else S.GBS_12_8)
        o = OG.gbs_run(lambda v: OM.rhs_oneway_spectral(v, 1.0 / n), y0[None, :], H, steps, c, 3)[0]
        assert rel_l2(g[off:off + n], o) <= 1e-11, n
        off += n
    sol.close()


@pytest.mark.parametrize("scheme", [S.GBS_8_6, S.GBS_12_8])
def test_section4_errors_match_the_oracle(scheme):
    steps, c = oracle_scheme(scheme)
    sumc = float(np.sum(np.abs(c)))
    errs = []
    for n in (16, 32, 64, 128, 256, 512, 1024):
        sol = _solver([n])
        sol.set_scheme(scheme)
        isb = sol.weights()[2]
        M = int(np.ceil(1.0 / (0.99 / np.pi * isb / n)))
        dt = 1.0 / M
        u0 = _u0(n)
        y = torch.tensor(u0, dtype=torch.float64, device="cuda")
        sol.step(y, y, dt, M)
        sol.sync()
        err = float(np.max(np.abs(y.cpu().numpy() - u0)))
        o = OG.gbs_run(lambda v: OM.rhs_oneway_spectral(v, 1.0 / n), u0[None, :], dt, steps, c, M)[0]
        oerr = float(np.max(np.abs(o - u0)))
        assert abs(err - oerr) <= max(1e-2 * oerr, 1e-16 * sumc * M), (n, err, oerr)
        errs.append(err)
        sol.close()
    if scheme.order == 8:
        assert abs(np.log2(errs[0] / errs[1]) - 8) < 0.6
    assert errs[-1] < 1e-11          # the FP64 floor, reached by both schemes
