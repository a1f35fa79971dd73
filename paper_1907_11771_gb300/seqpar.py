"""Sequence parallelism across GPUs: the sequences of one macro-step split over ranks.

Sec. 3.6 observes that the sequences of an extrapolated macro-step are independent and
spreads them over cores; with N_max = 4 n_cores - 2 the even step counts 2 .. N_max balance
exactly when pairs whose counts add up to N_max share a core ({10}, {8, 2}, {6, 4} for
N_max = 10).  Here a rank is a GPU.  Every rank holds the state y_0 and the media, runs its
sequences (gbs_step_partial), and one FP64 all-reduce of the combine shares per macro-step
completes the step (gbs_combine_partial) on every rank.

The work of sequence k is N_k leap-frog levels plus its Forward-Euler level (the first
right-hand side is evaluated once per rank).  partition() folds the pairs as Sec. 3.6 does
and assigns the groups to ranks longest-first onto the least loaded rank, so any rank count
and any scheme (not only the even counts up to 4 g - 2) get a balanced, disjoint cover.
min_ranks() gives the fewest ranks that keep every rank within the longest sequence's time,
the core counts that Tables 1 and 2 print.
This module holds host logic only: the arithmetic runs in the CUDA library, the exchange in
torch.distributed (NCCL between GPUs; gloo in the CPU tests).
"""
import torch


def fold_pairs(steps):
    """Sec. 3.6's folding: sequence indices grouped so that paired step counts add up to the
    largest one (a count whose partner is absent, or the largest itself, stays alone).
    Returns lists of indices into ``steps``."""
    order = sorted(range(len(steps)), key=lambda k: steps[k])
    n_max = steps[order[-1]]
    left = set(order)
    groups = []
    for k in sorted(order, key=lambda k: -steps[k]):
        if k not in left:
            continue
        left.discard(k)
        partner = [j for j in left if steps[j] + steps[k] == n_max]
        if partner:
            left.discard(partner[0])
            groups.append([k, partner[0]])
        else:
            groups.append([k])
    return groups


def min_ranks(steps):
    """The fewest ranks (cores, in Sec. 3.6) that run the sequences in the time of the longest
    one: each rank evaluates the first right-hand side and then the leap-frog levels of its
    sequences, at most N_max + 1 evaluations, so the counts N_k are packed into bins of
    capacity N_max.  Exact (backtracking over the sequences, longest first, for the at most
    16 sequences of a scheme).  For the even counts 2 .. 4g - 2 it is g (Sec. 3.6's folded
    pairs)."""
    items = sorted((int(n) for n in steps), reverse=True)
    if not items:
        return 0
    cap = items[0]

    def fits(k):
        bins = [0] * k

        def place(i):
            if i == len(items):
                return True
            seen = set()
            for b in range(k):
                if bins[b] + items[i] <= cap and bins[b] not in seen:
                    seen.add(bins[b])          # bins with equal loads are interchangeable
                    bins[b] += items[i]
                    if place(i + 1):
                        return True
                    bins[b] -= items[i]
            return False
        return place(0)

    k = -(-sum(items) // cap)
    while not fits(k):
        k += 1
    return k


def _place(groups, steps, n_ranks):
    work = lambda g: sum(steps[k] + 1 for k in g)
    loads, masks = [0] * n_ranks, [0] * n_ranks
    for g in sorted(groups, key=work, reverse=True):
        r = min(range(n_ranks), key=lambda i: (loads[i], i))
        loads[r] += work(g)
        for k in g:
            masks[r] |= 1 << k
    return masks, loads


def partition(steps, n_ranks):
    """Disjoint sequence sets, one per rank, covering every sequence (load of a sequence:
    N_k + 1 levels).  Sec. 3.6's folded pairs placed longest first on the least loaded rank,
    or the single sequences placed so, whichever leaves the smaller largest load (pairs are
    indivisible, so with ranks that do not divide the number of pairs, or more ranks than
    pairs, single sequences balance better).  Returns (masks, loads): masks[r] has bit k set
    for the sequences of rank r; a rank may get none when there are more ranks than
    sequences."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    steps = list(steps)
    folded = _place(fold_pairs(steps), steps, n_ranks)
    single = _place([[k] for k in range(len(steps))], steps, n_ranks)
    return folded if max(folded[1]) <= max(single[1]) else single


def step(solver, y_in, y_out, H, mask, group=None, partial=None):
    """One sequence-parallel macro-step on this rank: its share of the combine (zero for a rank
    without sequences), an FP64 SUM all-reduce over ``group`` (torch.distributed; skipped when
    no process group is initialised), and the completion into y_out (y_out may be y_in).
    ``partial``: optional FP64 work buffer of the state's length; returned."""
    import torch.distributed as dist
    if partial is None:
        partial = torch.empty(y_in.numel(), dtype=torch.float64, device=y_in.device)
    if mask:
        solver.step_partial(y_in, partial, H, mask)
    else:
        partial.zero_()
    if dist.is_available() and dist.is_initialized():
        if partial.is_cuda and dist.get_backend(group) != "nccl":
            torch.cuda.current_stream().synchronize()   # other backends do not order on the stream
        dist.all_reduce(partial, op=dist.ReduceOp.SUM, group=group)
    solver.combine_partial(y_in, partial, y_out)
    return partial
