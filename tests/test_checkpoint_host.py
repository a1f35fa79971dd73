"""Host logic of the checkpointed misfit gradient (no GPU).

* The binomial schedule's closed-form cost r l - beta(c + 1, r - 1) equals the
  brute-force minimum over every recursive split (dynamic programming on small
  chains), and the split rule attains it.
* Running a schedule on integer "states" hands every adjoint macro-step the
  state at its own start, in reverse order, exactly once, with at most s
  stored states.
* ``gbs_misfit_and_grad`` with a fake solver (a small linear map on CPU
  tensors whose adjoint and kappa-derivative are exact) gives the same J and
  gradient with two-level and binomial checkpointing, and both match central
  finite differences of J; ``GBSStepFn``'s backward, with every state or a
  binomial schedule, matches torch's autograd through the same map.
"""
from functools import lru_cache

import numpy as np
import pytest
import torch

from paper_1907_11771_gb300.autograd import gbs_misfit_and_grad
from paper_1907_11771_gb300.checkpoint import WORK, beta, min_advances, revolve_plan, split_length


@lru_cache(maxsize=None)
def brute_cost(l, c):
    """Least advances over every recursive split of a chain of l steps with c states."""
    if l == 1:
        return 0
    if c == 1:
        return l * (l - 1) // 2
    return min(l1 + brute_cost(l - l1, c - 1) + brute_cost(l1, c) for l1 in range(1, l))


def test_beta_is_pascal():
    for r in range(0, 8):
        assert beta(1, r) == r + 1   # one state: restart from the chain's start for every step
        for c in range(2, 8):
            assert beta(c, r) == beta(c, r - 1) + beta(c - 1, r)


@pytest.mark.parametrize("c", [1, 2, 3, 4, 5, 6])
def test_closed_form_equals_brute_force(c):
    for l in range(1, 70):
        assert min_advances(l, c) == brute_cost(l, c), (l, c)


def test_split_rule_attains_the_minimum():
    for c in range(2, 7):
        for l in range(2, 70):
            l1 = split_length(l, c)
            assert 1 <= l1 < l
            assert l1 + brute_cost(l - l1, c - 1) + brute_cost(l1, c) == brute_cost(l, c), (l, c)


def _simulate(plan, n, s):
    """Run a plan on integer states; return the adjoint order and the advances counted."""
    slots = {0: 0}
    for m, k in plan.forward_stores:
        assert 0 < k < s and k not in slots
        slots[k] = m
    order, advanced = [], 0
    for act in plan.actions:
        if act[0] == "advance":
            _, src, dst, a, m = act
            assert slots[src] == a and m > a and dst != src
            advanced += m - a
            slots[dst] = m
            assert len([k for k in slots if k != WORK]) <= s
        else:
            _, k, m = act
            assert slots[k] == m, "adjoint given the wrong state"
            order.append(m)
    return order, advanced


@pytest.mark.parametrize("n,s", [(1, 1), (1, 4), (2, 1), (7, 1), (7, 2), (10, 3), (33, 3), (64, 4),
                                 (100, 2), (100, 6), (200, 10), (12, 12), (12, 40)])
def test_plan_reverses_every_step_once_with_the_right_state(n, s):
    plan = revolve_plan(n, s)
    order, advanced = _simulate(plan, n, s)
    assert order == list(range(n - 1, -1, -1))
    assert advanced == plan.advances
    assert plan.max_slots <= s
    # the first descent is paid by the forward sweep: the rest is the binomial minimum
    descent = plan.forward_stores[-1][0] if plan.forward_stores else 0
    assert plan.advances + descent == min_advances(n, s)


def test_revolve_needs_fewer_states_than_two_level():
    # 2000 macro-steps: two-level checkpointing every 50 holds 40 + 50 states; 10 binomial
    # states reverse the chain advancing each step at most r = 5 times
    plan = revolve_plan(2000, 10)
    assert plan.max_slots == 10
    assert plan.advances + plan.forward_stores[-1][0] == 5 * 2000 - beta(11, 4)


class FakeLinearSolver:
    """y_(m+1) = (A0 + diag(kappa) B) y_m on CPU tensors, with the exact adjoint and kappa-derivative,
    behind the solver methods the checkpointing code calls."""

    F = 1

    def __init__(self, P, seed=0):
        rng = np.random.default_rng(seed)
        self.A0 = torch.tensor(0.3 * rng.standard_normal((P, P)) / np.sqrt(P) + 0.9 * np.eye(P))
        self.B = torch.tensor(0.2 * rng.standard_normal((P, P)) / np.sqrt(P))
        self.kappa = torch.tensor(rng.uniform(0.5, 1.5, P))
        self.state_elems = P
        self.steps = 0

    def A(self):
        return self.A0 + torch.diag(self.kappa) @ self.B

    def step(self, y_in, y_out, H, n_macro=1):
        y = y_in.clone()
        for _ in range(n_macro):
            y = self.A() @ y
        self.steps += n_macro
        y_out.copy_(y)

    def misfit(self, y, rcv, data, resid, J):
        resid.copy_(y[rcv] - data)
        J += 0.5 * (resid.double() ** 2).sum()

    def inject(self, lam, rcv, values):
        lam.index_add_(0, rcv, values)

    def adjoint_step(self, y_in, lam_out, lam_in, grad, H, rcv=None, resid=None):
        grad += (self.B @ y_in) * lam_out          # d(A y)/dkappa_i = e_i (B y)_i
        new = self.A().T @ lam_out
        if rcv is not None:
            new.index_add_(0, rcv, resid)
        lam_in.copy_(new)

    def sync(self):
        pass


def _fake_problem(n_macro, seed=1):
    sol = FakeLinearSolver(24, seed)
    rng = np.random.default_rng(seed + 7)
    y0 = torch.tensor(rng.standard_normal(24))
    rcv = torch.tensor([1, 5, 11, 20])
    data = torch.tensor(0.3 * rng.standard_normal((n_macro, 4)))
    return sol, y0, rcv, data


@pytest.mark.parametrize("n_macro", [1, 2, 9, 17])
def test_misfit_gradient_revolve_equals_two_level_and_finite_differences(n_macro):
    sol, y0, rcv, data = _fake_problem(n_macro)
    J2, g2 = gbs_misfit_and_grad(sol, y0, 0.1, n_macro, rcv, data, checkpoint_every=4)
    for s in (1, 2, 3, n_macro + 2):
        Jr, gr = gbs_misfit_and_grad(sol, y0, 0.1, n_macro, rcv, data, snapshots=s)
        assert Jr == pytest.approx(J2, rel=1e-14)
        assert torch.allclose(gr, g2, rtol=1e-12, atol=1e-14)
    base = sol.kappa.clone()
    rng = np.random.default_rng(5)
    for _ in range(3):
        d = torch.tensor(rng.standard_normal(base.numel()))
        eps = 1e-6
        Js = []
        for sgn in (1, -1):
            sol.kappa = base + sgn * eps * d
            Js.append(gbs_misfit_and_grad(sol, y0, 0.1, n_macro, rcv, data, snapshots=2)[0])
        sol.kappa = base
        fd = (Js[0] - Js[1]) / (2 * eps)
        assert float(g2 @ d) == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_revolve_recomputes_no_more_than_the_schedule_says():
    n, s = 30, 3
    sol, y0, rcv, data = _fake_problem(n)
    sol.steps = 0
    gbs_misfit_and_grad(sol, y0, 0.1, n, rcv, data, snapshots=s)
    assert sol.steps == n + revolve_plan(n, s).advances


@pytest.mark.parametrize("n,s", [(1, 1), (5, 1), (9, 2), (17, 3), (6, 10)])
def test_step_function_backward_with_and_without_checkpoints(n, s):
    # GBSStepFn's backward on the fake solver: every state (None) and a binomial schedule of s
    # states give the gradients of torch's own autograd through the dense map A(kappa)^n
    from paper_1907_11771_gb300.autograd import GBSStepFn
    sol = FakeLinearSolver(16, seed=3)
    sol.kappa.requires_grad_(True)
    sol._media = (sol.kappa,)
    rng = np.random.default_rng(11)
    y0 = torch.tensor(rng.standard_normal(16))
    w = torch.tensor(rng.standard_normal(16))
    yr = y0.clone().requires_grad_(True)
    kr = sol.kappa.detach().clone().requires_grad_(True)
    out = yr
    for _ in range(n):
        out = (sol.A0 + torch.diag(kr) @ sol.B) @ out
    (w * out).sum().backward()
    for snaps in (None, s):
        y = y0.clone().requires_grad_(True)
        sol.kappa.grad = None
        res = GBSStepFn.apply(y, sol.kappa, sol, 0.1, n, snaps)
        (w * res).sum().backward()
        assert torch.allclose(y.grad, yr.grad, rtol=1e-12, atol=1e-13)
        assert torch.allclose(sol.kappa.grad, kr.grad, rtol=1e-12, atol=1e-13)
