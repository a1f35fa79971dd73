"""One extrapolated GBS macro-step and its discrete adjoint (oracle side).

Paper passages followed:

* Sec. 2.1 eq. "GBS": one sequence with N steps of h = H/N is
      y_1 = y_0 + h f(y_0)                       (Forward Euler)
      y_(n+1) = y_(n-1) + 2 h f(y_n), n = 1..N   (leap-frog)
      y*_N = (y_(N-1) + 2 y_N + y_(N+1)) / 4     (averaging)
* Sec. 3.6: the first function evaluation f(y_0) has the same argument for
  every sequence and is computed once and shared.
* Sec. 2.1 / Sec. 3.2: the extrapolated result is sum_k c_k y*_k.  The sum is
  taken in FP64 in the order the sequences are given.

Precision: the whole computation runs in the dtype of ``y`` (FP64; complex128
for the spectral test problem's modes).

The adjoint is the exact transpose of these steps, derived by hand (reverse
accumulation through the recurrences); the gradient with respect to kappa
collects <mu, (dA/dkappa) y> from every application of A.
"""
import numpy as np


def gbs_sequence(f, y0, H, N, f0=None):
    """y*_N of one GBS sequence (Sec. 2.1 eq. "GBS").  ``f0`` = f(y0) if shared."""
    dt = y0.dtype.type
    h = dt(H / N)
    if f0 is None:
        f0 = f(y0)
    ys = [y0, y0 + h * f0]                         # FE
    for n in range(1, N + 1):                      # LF, n = 1..N
        ys.append(ys[n - 1] + dt(2) * h * f(ys[n]))
    return (ys[N - 1] + dt(2) * ys[N] + ys[N + 1]) / dt(4)   # averaging


def gbs_macro_step(f, y, H, steps, c):
    """sum_k c_k y*_k for the sequences ``steps`` with weights ``c``, summed in ascending k.
    Sec. 2.1 eq. "GBS" per sequence, combined as in Sec. 3.2."""
    f0 = f(y)                                      # shared first evaluation
    acc = np.zeros_like(y)
    for N, ck in zip(steps, c):
        acc = acc + float(ck) * gbs_sequence(f, y, H, N, f0)
    return acc


def gbs_run(f, y, H, steps, c, n_macro):
    """n_macro consecutive macro-steps (the time interval split into sections, Sec. 2.1)."""
    for _ in range(n_macro):
        y = gbs_macro_step(f, y, H, steps, c)
    return y


# --------------------------------------------------------------------------
# Discrete adjoint of one macro-step (transpose of the steps above)
# --------------------------------------------------------------------------

def gbs_macro_step_adjoint(f, fT, pair, y0, lam_out, H, steps, c):
    """Not in the paper: the exact transpose of the Sec. 2.1 macro-step.
    Return (lam_in, g) with lam_in = M^T lam_out for the linear macro-step
    y_out = M y0 = sum_k c_k S_k y0, and g = d<lam_out, M(kappa) y0>/dkappa
    pointwise (``pair(mu, y)`` returns <mu, dA/dkappa_i y> for every i).

    Reverse accumulation, sequence by sequence (mu_n is the adjoint of y_n):
      averaging:   mu_(N+1) += w/4, mu_N += w/2, mu_(N-1) += w/4   (w = c_k lam_out)
      LF n=N..1:   y_(n+1) = y_(n-1) + 2h A y_n  gives
                   mu_(n-1) += mu_(n+1);  mu_n += 2h A^T mu_(n+1);  g += 2h pair(mu_(n+1), y_n)
      FE:          y_1 = y_0 + h f0 gives mu_0 += mu_1 and, through the shared
                   f0 = A y_0, the term A^T (sum_k h_k mu_1^k) plus
                   g += pair(sum_k h_k mu_1^k, y_0).
    """
    f0 = f(y0)
    lam_in = np.zeros_like(y0)
    shared = np.zeros_like(y0)      # sum_k h_k mu_1^(k), fed through A^T once
    g = np.zeros(y0.shape[1:], dtype=y0.dtype)
    for N, ck in zip(steps, c):
        h = H / N
        ys = [y0, y0 + h * f0]
        for n in range(1, N + 1):
            ys.append(ys[n - 1] + 2 * h * f(ys[n]))
        w = float(ck) * lam_out
        mu = [np.zeros_like(y0) for _ in range(N + 2)]
        mu[N + 1] = mu[N + 1] + w / 4
        mu[N] = mu[N] + w / 2
        mu[N - 1] = mu[N - 1] + w / 4
        for n in range(N, 0, -1):
            mu[n - 1] = mu[n - 1] + mu[n + 1]
            mu[n] = mu[n] + 2 * h * fT(mu[n + 1])
            g = g + 2 * h * pair(mu[n + 1], ys[n])
        lam_in = lam_in + mu[0] + mu[1]
        shared = shared + h * mu[1]
    lam_in = lam_in + fT(shared)
    g = g + pair(shared, y0)
    return lam_in, g


# --------------------------------------------------------------------------
# Receiver misfit and its gradient over many macro-steps
# --------------------------------------------------------------------------

def sample_receivers(y, rcv_flat):
    """Pressure (field 0) at flat grid indices ``rcv_flat`` (receiver sampling; not in the paper)."""
    return y[0].reshape(-1)[rcv_flat]


def inject_receivers(shape, rcv_flat, values, dtype=np.float64):
    """Not in the paper: the transpose of ``sample_receivers``.
    A state-shaped array that is zero except field 0 at the receivers (adds duplicates)."""
    out = np.zeros(shape, dtype=dtype)
    flat = out[0].reshape(-1)
    np.add.at(flat, rcv_flat, values)
    out[0] = flat.reshape(shape[1:])
    return out


def misfit_and_gradient(f, fT, pair, y0, H, steps, c, n_macro, rcv_flat, data):
    """Not in the paper (receiver misfit and its gradient by the adjoint).
    J = 1/2 sum_m sum_r (p(x_r, t_m) - d_r(t_m))^2 over macro-step ends m = 1..n_macro
    and dJ/dkappa by the discrete adjoint.  ``data`` has shape (n_macro, n_rcv)."""
    states = [y0]
    for _ in range(n_macro):
        states.append(gbs_macro_step(f, states[-1], H, steps, c))
    resid = np.stack([sample_receivers(states[m + 1], rcv_flat) - data[m] for m in range(n_macro)])
    J = 0.5 * float(np.sum(resid ** 2))
    lam = inject_receivers(y0.shape, rcv_flat, resid[n_macro - 1])
    g = np.zeros(y0.shape[1:], dtype=np.float64)
    for m in range(n_macro - 1, -1, -1):
        lam, gm = gbs_macro_step_adjoint(f, fT, pair, states[m], lam, H, steps, c)
        g = g + gm
        if m > 0:
            lam = lam + inject_receivers(y0.shape, rcv_flat, resid[m - 1])
    return J, g
