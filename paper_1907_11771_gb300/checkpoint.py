"""Binomial ("revolve") checkpointing schedules for reversing a chain of macro-steps.

The misfit gradient runs the adjoint macro-steps in reverse order, and the
adjoint of macro-step m needs the forward state y_m at its start.  With room
for only ``s`` stored states, the states are recomputed from stored ones.
Binomial checkpointing (Griewank, Optim. Methods Softw. 1 (1992); Griewank &
Walther, ACM TOMS 26 (2000)) places the stored states so that the number of
recomputed macro-steps is the least possible:

* beta(c, r) = C(c + r, c) is the longest chain that c stored states (the one
  at the chain's start included) reverse when no step is advanced more than r
  times; beta(c, r) = beta(c, r - 1) + beta(c - 1, r).
* For a chain of l steps with c states, the repetition number r is the least
  r with beta(c, r) >= l, and the least number of advanced steps is
  r l - beta(c + 1, r - 1).
* A split of the chain into [a, a + l1) and [a + l1, b) attains it when
  beta(c, r - 2) <= l1 <= beta(c, r - 1) and l - l1 <= beta(c - 1, r): the
  right part is reversed first with one state fewer (the left part's start is
  still held) and r repetitions, then the left part with all c states and one
  repetition fewer (its steps were advanced once to reach the split).

``revolve_plan`` turns this recursion into an explicit action list over
numbered state slots, so the host code that runs it (``autograd.py``) only
follows the list.  Host logic only: no GPU work happens here.
"""
from dataclasses import dataclass, field
from math import comb

WORK = -1   # slot id of the scratch state (the running state of the forward sweep)


def beta(c: int, r: int) -> int:
    """Longest chain c stored states reverse with at most r advances per step (0 for r < 0)."""
    return comb(c + r, c) if r >= 0 else 0


def repetition_number(l: int, c: int) -> int:
    """Least r >= 0 with beta(c, r) >= l, for l >= 1 steps and c >= 1 stored states."""
    if l < 1 or c < 1:
        raise ValueError("need at least one step and one stored state")
    r = 0
    while beta(c, r) < l:
        r += 1
    return r


def min_advances(l: int, c: int) -> int:
    """Least number of macro-steps advanced to reverse l steps holding at most c states."""
    r = repetition_number(l, c)
    return r * l - beta(c + 1, r - 1)


def split_length(l: int, c: int) -> int:
    """Length l1 of the left part of an optimal split of l >= 2 steps with c >= 2 states."""
    r = repetition_number(l, c)
    return max(1, beta(c, r - 2), l - beta(c - 1, r))


@dataclass
class RevolvePlan:
    """Actions that reverse n steps with at most s stored states.

    forward_stores: (position m, slot) pairs stored while the forward sweep passes
        y_m (slot 0 holds y_0 before the sweep).
    actions: in order, one of
        ("advance", src, dst, a, m)  slot dst <- y_m, computed from y_a in slot src
                                     (m - a macro-steps; dst may be WORK)
        ("adjoint", slot, m)         adjoint of macro-step m with y_m read from slot
    advances: macro-steps advanced by the actions (the forward sweep not counted).
    max_slots: most stored slots live at once (WORK not counted).
    """
    n: int
    s: int
    forward_stores: list = field(default_factory=list)
    actions: list = field(default_factory=list)
    advances: int = 0
    max_slots: int = 1


def revolve_plan(n: int, s: int) -> RevolvePlan:
    """Binomial checkpointing schedule for n >= 1 macro-steps and s >= 1 stored states.

    The first descent of the recursion (the split points on the way to the
    chain's last step) lies on the forward sweep, so those states are stored as
    the sweep passes them instead of being advanced again."""
    if n < 1 or s < 1:
        raise ValueError("revolve_plan needs n >= 1 macro-steps and s >= 1 stored states")
    plan = RevolvePlan(n=n, s=s)
    a, c, slot = 0, s, 0
    while c >= 2 and n - a >= 2:
        m = a + split_length(n - a, c)
        slot += 1
        plan.forward_stores.append((m, slot))
        a, c = m, c - 1
    prestored = set(plan.forward_stores)
    held = {0}
    # explicit stack (a chain of n steps with s >= n states nests n deep): ("rev", a, b, c, base)
    # reverses steps [a, b) from y_a in slot base with c states; ("free", slot) releases a slot
    todo = [("rev", 0, n, s, 0)]
    while todo:
        task = todo.pop()
        if task[0] == "free":
            held.discard(task[1])
            continue
        _, a, b, c, base = task
        l = b - a
        if l == 1:
            plan.actions.append(("adjoint", base, a))
            continue
        if c == 1:
            for i in range(b - 1, a, -1):
                plan.actions.append(("advance", base, WORK, a, i))
                plan.advances += i - a
                plan.actions.append(("adjoint", WORK, i))
            plan.actions.append(("adjoint", base, a))
            continue
        m = a + split_length(l, c)
        new = min(set(range(s)) - held)
        held.add(new)
        plan.max_slots = max(plan.max_slots, len(held))
        if (m, new) in prestored:
            prestored.discard((m, new))
        else:
            plan.actions.append(("advance", base, new, a, m))
            plan.advances += m - a
        # the right part first, then release its start, then the left part
        todo += [("rev", a, m, c, base), ("free", new), ("rev", m, b, c - 1, new)]
    return plan
