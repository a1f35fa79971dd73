"""Seeded synthetic inputs for the wave workloads (shared by tests, bench and smoke).

This module only generates data -- initial states, media, receiver positions,
problem-size mixes.  It contains none of the time-stepping method's arithmetic,
so the CUDA path and the CPU oracle can both be fed from it.

Recipes (all grids periodic, cell units dx = 1 unless stated):

* ``wave1d_initial``: 1D wave on [0, 2 pi) with n points, u0 = exp(-20 (x - pi)^2),
  v0 = 0.
* ``smooth_media``: 1 + sum of ``n_gauss`` periodic Gaussians, amplitudes
  U[0, 0.5], widths U[N/32, N/8] cells (N = smallest side), centres U[0, N)^d,
  numpy ``default_rng(seed)``.
* ``gaussian_pulses``: pressure = sum of periodic Gaussians exp(-r^2 / (2 sigma^2)),
  velocities zero.
* ``acoustic_problem``: kappa from ``seed``, rho from ``seed + 1``, pulse centres
  from ``seed + 2`` (or the grid centre for a single centred pulse).
* ``batch_sides``: 256 grid sides drawn uniformly from {128,...,1024} (seed 0);
  problem i then uses seed 1000 + i.
* ``line_receivers``: n_rcv receivers on the row y = 3N/4 at x = round((j + 1/2) N / n_rcv).
"""
import numpy as np


def wave1d_initial(n=256):
    x = 2.0 * np.pi * np.arange(n) / n
    u0 = np.exp(-20.0 * (x - np.pi) ** 2)
    return np.stack([u0, np.zeros_like(u0)]), 2.0 * np.pi / n


def _periodic_sq_dist_1d(n, c):
    d = np.abs(np.arange(n, dtype=np.float64) - c)
    d = np.minimum(d, n - d)
    return d * d


def _gaussian(shape, center, width, dtype):
    """exp(-|x - c|^2_periodic / (2 w^2)) on a grid of shape (z,) (y,) x, built separably."""
    nd = len(shape)
    out = None
    for ax in range(nd):
        n = shape[ax]
        g1 = np.exp(-_periodic_sq_dist_1d(n, center[ax]) / (2.0 * width * width)).astype(dtype)
        sh = [1] * nd
        sh[ax] = n
        g1 = g1.reshape(sh)
        out = g1 if out is None else out * g1
    return out


def smooth_media(shape, n_gauss, seed, amp_max=0.5, dtype=np.float64):
    rng = np.random.default_rng(seed)
    N = min(shape)
    m = np.ones(shape, dtype=dtype)
    for _ in range(n_gauss):
        a = rng.uniform(0.0, amp_max)
        w = rng.uniform(N / 32.0, N / 8.0)
        c = [rng.uniform(0.0, n) for n in shape]
        m += a * _gaussian(shape, c, w, dtype)
    return m


def gaussian_pulses(shape, sigma, centers, dtype=np.float64):
    p = np.zeros(shape, dtype=dtype)
    for c in centers:
        p += _gaussian(shape, c, sigma, dtype)
    return p


def acoustic_problem(shape, seed, n_gauss, sigma, n_pulses=1, centred=True, const_rho=False,
                     dtype=np.float64):
    """Initial state y0[field, (z,) (y,) x] = (p0, 0, ...), kappa and rho arrays.

    ``shape`` is given in array order ((z,) (y,) x)."""
    shape = tuple(int(s) for s in shape)
    kappa = smooth_media(shape, n_gauss, seed, dtype=dtype)
    rho = np.ones(shape, dtype=dtype) if const_rho else smooth_media(shape, n_gauss, seed + 1, dtype=dtype)
    if centred and n_pulses == 1:
        centers = [[n / 2.0 for n in shape]]
    else:
        rng = np.random.default_rng(seed + 2)
        centers = [[rng.uniform(0.0, n) for n in shape] for _ in range(n_pulses)]
    y0 = np.zeros((1 + len(shape),) + shape, dtype=dtype)
    y0[0] = gaussian_pulses(shape, sigma, centers, dtype)
    return y0, kappa, rho


def batch_sides(n_problems=256, seed=0, choices=(128, 256, 384, 512, 768, 1024)):
    rng = np.random.default_rng(seed)
    return [int(choices[i]) for i in rng.integers(0, len(choices), size=n_problems)]


def line_receivers(n, n_rcv=64):
    """Flat indices (row-major y, x) of receivers on the row y = 3n/4 of an n x n grid."""
    row = (3 * n) // 4
    xs = [int(round((j + 0.5) * n / n_rcv)) % n for j in range(n_rcv)]
    return np.array([row * n + x for x in xs], dtype=np.int64)
