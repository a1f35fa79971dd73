"""Autotuner for the time-blocked schedule.

The 2D time-blocked kernel's work decomposition has three knobs that change its speed but not
its results beyond rounding order: the row-segment height of a tile ("hseg"), the most leap-frog
levels per pass ("tmax"; deeper passes move fewer bytes but widen the halo) and the order of
the work queue ("schedule").  The 3D pass kernel has one, the z-planes per block ("zseg": longer
segments repeat fewer warm-up planes, shorter ones give more blocks to fill the GPU).  The plain one-step-per-launch kernels are one more candidate: with
few sequences on a small grid the time-blocked kernel has too few independent items and waits on
its dependencies, and the plain kernels are faster.  ``autotune`` times every candidate on the
caller's own problem
(whole macro-steps, CUDA events on the current stream, a buffer larger than L2 written before
each timed step), applies the fastest and caches the choice in a JSON file keyed by the
workload and the GPU, so a later run with the same key applies it without timing.
"""
import hashlib
import itertools
import json
import os

import torch

DEFAULT_SPACE = {"hseg": [96, 128, 192, 256, 384], "tmax": [4, 2], "schedule": [0, 1]}
KNOBS = ("hseg", "tmax", "schedule")
DEFAULT_SPACE_3D = {"zseg": [32, 64, 128, 256, 512]}
KNOBS_3D = ("zseg",)


def _knobs(solver):
    return KNOBS_3D if getattr(solver, "ndim", 2) == 3 else KNOBS


def default_cache_path():
    return os.environ.get("GBS_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "gbs_gb300_tune.json"))


def library_id():
    """Content hash of the loaded kernel library: a rebuilt kernel is tuned afresh."""
    from . import binding as B
    h = hashlib.sha1()
    with open(B.LIB_PATH, "rb") as f:
        for chunk in iter(lambda: f.read(1 << 20), b""):
            h.update(chunk)
    return h.hexdigest()[:16]


def workload_key(solver, device_name=None):
    """Shapes, system, order, precision, the step counts of the slots in use, the GPU and the
    kernel library."""
    from . import binding as B
    slots = sorted(set(solver.slots))
    steps = {str(s): B.gbs_get_weights(solver.h, s)[0] for s in slots}
    if device_name is None:
        device_name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return json.dumps({"system": solver.system, "fd_order": solver.fd_order, "precision": solver.precision,
                       "shapes": [list(s) for s in solver.shapes], "slots": solver.slots, "steps": steps,
                       "device": device_name, "library": library_id()}, sort_keys=True)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, table):
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def event_timer(solver, y, H, reps=3, warmup=1, flush_bytes=256 << 20):
    """A timer(config) -> seconds of one macro-step (best of `reps`) for the current options."""
    out = torch.empty_like(y)
    flush = torch.empty(flush_bytes // 4, dtype=torch.float32, device=y.device)

    def timer():
        for _ in range(warmup):
            solver.step(y, out, H, 1)
        best = float("inf")
        for i in range(reps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            solver.step(y, out, H, 1)
            b.record()
            b.synchronize()
            best = min(best, a.elapsed_time(b) / 1e3)
        return best

    return timer


def _apply(solver, options):
    from . import binding as B
    for k in _knobs(solver):
        solver.set_option(k, options[k])
    solver.set_option("kernel", options.get("kernel", B.GBS_KERNEL_FUSED))


def autotune(solver, y=None, H=None, space=None, cache=None, timer=None, key=None, retune=False, plain=True):
    """Pick the fastest time-blocked schedule for `solver`'s problem -- or the plain kernels, if
    `plain` and they are faster -- and apply it.

    y, H: a representative state and step size (used by the default event timer).  space: dict
    knob -> candidate values (default DEFAULT_SPACE).  cache: JSON path (default
    default_cache_path(); False disables caching).  timer: callable() -> seconds for the options
    currently set (default: CUDA-event timing of one macro-step).  Returns a dict with the chosen
    options ("kernel" plus the schedule knobs), their time and the whole table; None when the
    problem does not use the time-blocked kernel (nothing to tune)."""
    from . import binding as B
    if not solver.uses_fused():
        return None
    knobs = _knobs(solver)
    space = dict((DEFAULT_SPACE_3D if knobs == KNOBS_3D else DEFAULT_SPACE) if space is None else space)
    if cache is None:
        cache = default_cache_path()
    key = key or workload_key(solver)
    table = _load(cache) if cache else {}
    if cache and not retune and key in table:
        best = table[key]
        _apply(solver, best["options"])
        return dict(best, cached=True)
    if timer is None:
        timer = event_timer(solver, y, H)
    rows = []
    solver.set_option("kernel", B.GBS_KERNEL_FUSED)
    for values in itertools.product(*(space[k] for k in knobs)):
        opts = dict(zip(knobs, values))
        for k, v in opts.items():
            solver.set_option(k, v)
        rows.append({"options": dict(opts, kernel=B.GBS_KERNEL_FUSED), "seconds": float(timer())})
    if plain:   # the plain kernels, keeping the best schedule for a later switch back
        fused_best = min(rows, key=lambda r: r["seconds"])["options"]
        solver.set_option("kernel", B.GBS_KERNEL_PLAIN)
        rows.append({"options": dict(fused_best, kernel=B.GBS_KERNEL_PLAIN), "seconds": float(timer())})
    best = min(rows, key=lambda r: r["seconds"])
    _apply(solver, best["options"])
    result = {"options": best["options"], "seconds": best["seconds"], "table": rows}
    if cache:
        table = _load(cache)
        table[key] = result
        _store(cache, table)
    return dict(result, cached=False)
