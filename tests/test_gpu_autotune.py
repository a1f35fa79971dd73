"""Autotuning the time-blocked schedule on a real problem: every candidate runs, the chosen
options are applied and cached, and the tuned kernel still matches the oracle."""
import pytest
import torch

from paper_1907_11771_gb300 import autotune as A
from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import schemes as S
from tests.gpu_common import AcousticCase, oracle_scheme, rel_l2

pytestmark = pytest.mark.gpu
F32 = B.GBS_F32_STATE_F64_COMBINE


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_autotune_applies_caches_and_keeps_parity(tmp_path):
    case = AcousticCase((300, 290), 6, F32, seed=14)
    sol = case.solver()
    sol.set_scheme(S.GBS_8_6)
    H = 0.8 * sol.stability_limit()[0]
    y = torch.tensor(case.y0.ravel(), dtype=torch.float32, device="cuda")
    cache = str(tmp_path / "tune.json")
    space = {"hseg": [48, 96, 512], "tmax": [4, 2], "schedule": [0, 1]}
    r = A.autotune(sol, y, H, space=space, cache=cache)
    assert not r["cached"] and len(r["table"]) == 12 + 1          # the schedules and the plain kernels
    assert all(row["seconds"] > 0 for row in r["table"])
    for k in A.KNOBS + ("kernel",):
        assert sol.get_option(k) == r["options"][k]
    steps, c = oracle_scheme(S.GBS_8_6)
    o = case.oracle_run(steps, c, H, 2)
    assert rel_l2(case.gpu_run(sol, H, 2), o) <= 1e-5
    # every candidate is a valid schedule: spot-check the slowest one against the oracle too
    worst = max(r["table"], key=lambda row: row["seconds"])["options"]
    for k, v in worst.items():
        sol.set_option(k, v)
    assert rel_l2(case.gpu_run(sol, H, 2), o) <= 1e-5
    r2 = A.autotune(sol, y, H, space=space, cache=cache)
    assert r2["cached"] and r2["options"] == r["options"]
    sol.close()
