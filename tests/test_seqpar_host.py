"""Sequence parallelism's host logic (no GPU): the partition of a scheme's sequences over ranks
(Sec. 3.6's pair folding) and one macro-step completed by an FP64 all-reduce of the ranks'
combine shares, on two gloo ranks on 127.0.0.1.

The ranks' shares come from a stand-in for the CUDA library's gbs_step_partial /
gbs_combine_partial written here with the CPU oracle's GBS sequences; the test checks
seqpar.step's dispatch (a rank's mask, zero for a rank without sequences, the all-reduce, the
completion) against the oracle's whole macro-step.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1907_11771_gb300 import schemes as S
from paper_1907_11771_gb300 import seqpar


def test_pair_folding_follows_the_papers_example():
    # N_max = 10 on three cores: {10}, {8, 2}, {6, 4} (Sec. 3.6)
    steps = [2, 4, 6, 8, 10]
    groups = sorted(sorted(steps[k] for k in g) for g in seqpar.fold_pairs(steps))
    assert groups == [[2, 8], [4, 6], [10]]
    masks, loads = seqpar.partition(steps, 3)
    assert sorted(loads) == [11, 12, 12]          # N_max + 1 = 11 per core, plus one FE per extra sequence


@pytest.mark.parametrize("scheme,ranks", [(S.GBS_8_6, 6), (S.GBS_8_8, 8)])
def test_schemes_on_4g_minus_2_balance_on_g_ranks(scheme, ranks):
    # N_max = 4 g - 2: the folded pairs load g ranks evenly (within the extra FE level of a pair)
    masks, loads = seqpar.partition(scheme.steps, ranks)
    assert max(loads) - min(loads) <= 1
    assert max(loads) <= max(scheme.steps) + 2


@pytest.mark.parametrize("scheme", [S.GBS_8_6, S.GBS_8_8, S.SQ8_2468, S.GBS_12_8])
@pytest.mark.parametrize("ranks", [1, 2, 3, 4, 5, 8, 13])
def test_partition_is_a_disjoint_cover_with_its_stated_loads(scheme, ranks):
    steps = scheme.steps
    masks, loads = seqpar.partition(steps, ranks)
    assert len(masks) == ranks
    union = 0
    for m, l in zip(masks, loads):
        assert union & m == 0
        union |= m
        assert l == sum(steps[k] + 1 for k in range(len(steps)) if (m >> k) & 1)
    assert union == (1 << len(steps)) - 1
    # never worse than the ideal by more than one sequence's work
    assert max(loads) <= sum(loads) / ranks + max(steps) + 1


class OracleShares:
    """Stand-in for the library's partial steps on the 1D wave system, from the CPU oracle."""

    def __init__(self, scheme, dx):
        from oracle import mol as OM
        from tests.gpu_common import oracle_scheme
        self.steps, self.c = oracle_scheme(scheme)
        self.f = lambda v: OM.rhs_wave1d(v, dx, 4)
        self.calls = []

    def step_partial(self, y_in, partial, H, mask):
        from oracle import gbs as OG
        self.calls.append(mask)
        y0 = y_in.numpy().reshape(2, -1)
        f0 = self.f(y0)
        acc = np.zeros_like(y0)
        for k, (N, ck) in enumerate(zip(self.steps, self.c)):
            if (mask >> k) & 1:
                acc += float(ck) * (OG.gbs_sequence(self.f, y0, H, N, f0) - y0)
        partial.copy_(torch.from_numpy(acc.ravel()))

    def combine_partial(self, y_in, total, y_out):
        y_out.copy_(y_in + total)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, ranks_masks, out):
    import torch.distributed as dist
    from paper_1907_11771_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    y0, dx = inputs.wave1d_initial(64)
    sol = OracleShares(S.SQ8_2468, dx)
    y = torch.from_numpy(y0.ravel().copy())
    H = 0.05
    for _ in range(3):          # three macro-steps, each completed on both ranks
        seqpar.step(sol, y, y, H, ranks_masks[rank])
    out[rank] = (y.numpy().copy(), sol.calls)
    dist.destroy_process_group()


@pytest.mark.parametrize("split", ["balanced", "one_rank_idle"])
def test_two_gloo_ranks_complete_the_macro_step(split):
    from oracle import gbs as OG
    from oracle import mol as OM
    from paper_1907_11771_gb300 import inputs
    from tests.gpu_common import oracle_scheme
    masks = seqpar.partition(S.SQ8_2468.steps, 2)[0] if split == "balanced" else [0b1111, 0]
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(port, masks, out), nprocs=2, join=True)
        res = dict(out)
    y0, dx = inputs.wave1d_initial(64)
    steps, c = oracle_scheme(S.SQ8_2468)
    ref = OG.gbs_run(lambda v: OM.rhs_wave1d(v, dx, 4), y0, 0.05, steps, c, 3).ravel()
    for rank in (0, 1):
        y, calls = res[rank]
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-14
        assert calls == ([masks[rank]] * 3 if masks[rank] else [])
    assert np.array_equal(res[0][0], res[1][0])      # every rank holds the same completed state


def test_min_ranks_reproduces_the_papers_core_counts():
    from paper_1907_11771_gb300.seqpar import min_ranks
    # Table 1: the fully determined schemes on three, four and five cores
    assert min_ranks((2, 16, 18, 20)) == 3
    assert min_ranks((2, 8, 12, 14, 16, 20)) == 4
    assert min_ranks((2, 8, 10, 12, 14, 16, 18, 22)) == 5
    # Table 2: all even counts up to N_opt on 8, 11, 10 and 9 cores
    for n_opt, cores in ((28, 8), (40, 11), (36, 10), (32, 9)):
        assert min_ranks(range(2, n_opt + 1, 2)) == cores, n_opt
    # Sec. 3.6: the even counts up to 4g - 2 fill g cores; Sec. 3.8's six- and eight-core schemes
    for g in range(1, 9):
        assert min_ranks(range(2, 4 * g - 1, 2)) == g
    assert min_ranks(S.GBS_8_6.steps) == 6
    assert min_ranks(S.GBS_8_8.steps) == 8
    assert min_ranks(S.GBS_12_8.steps) == 8
    assert min_ranks((2, 4, 6, 8)) == 3 and min_ranks(()) == 0     # 8 | 6 + 2 | 4
