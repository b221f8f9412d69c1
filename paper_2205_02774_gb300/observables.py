"""Post-processing of the channel statistics (Sec. V of the paper).

Host-side reductions of what the library accumulates on the device (the FP64
sums of u and u u over z and the sampled steps, per (x, y)) and of probe time
series; all in lattice units.  Node j sits at y = j + 1/2 from the lower wall
(half-way bounce-back), the upper wall at y = ny.

* mean_and_stress:    <u>(x, y) and <u'_a u'_b>(x, y) from the sums
* friction_velocity:  eq. (u_shear), first-order wall gradient
* wall_units:         eqs. (y_plus), (v_rms): y+, u+, u+_rms, v+_rms, w+_rms
* u_theory_force / u_theory_re: the reference friction velocity of the
  u_tau / u_theory comparison (force balance, or the target Re_tau)
* autocorrelation, integral_time: B_uu and eq. (time-integral)
"""
from __future__ import annotations

import numpy as np

# order of the second-moment sums: uu, vv, ww, uv, uw, vw
_PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def mean_and_stress(mean_sum, rey_sum, n_samples, nz):
    """Mean velocity U[3][ny][nx] and Reynolds stresses R[6][ny][nx]
    (uu, vv, ww, uv, uw, vw) about that mean, averaged over z and the
    sampled steps: R_ab = <u_a u_b> - <u_a><u_b>."""
    n = float(n_samples) * float(nz)
    if n <= 0:
        raise ValueError("no samples")
    U = np.asarray(mean_sum, dtype=np.float64) / n
    UU = np.asarray(rey_sum, dtype=np.float64) / n
    R = np.empty_like(UU)
    for k, (a, b) in enumerate(_PAIRS):
        R[k] = UU[k] - U[a] * U[b]
    return U, R


def friction_velocity(Ux, nu):
    """u_tau(x) of eq. (u_shear): sqrt(nu dU/dy) at the wall with the
    first-order difference between the wall (U = 0) and the first node half a
    spacing away, averaged over the two walls.  Ux: [ny][nx] (or [ny])."""
    Ux = np.asarray(Ux, dtype=np.float64)
    grad = (Ux[0] + Ux[-1]) / 2.0 / 0.5
    return np.sqrt(nu * np.maximum(grad, 0.0))


def wall_units(U, R, nu, x, half="lower"):
    """Profiles of column x in wall units, eqs. (y_plus), (v_rms): returns
    y+, u+, and the rms of the three velocity components over u_tau, for the
    lower half of the channel (or the upper half mirrored, half="upper", or
    the mean of the two halves, half="both")."""
    ny = U.shape[1]
    ut = float(friction_velocity(U[0][:, x], nu))
    y = np.arange(ny) + 0.5
    h = ny // 2
    u = U[0][:, x]
    rms = np.sqrt(np.maximum(R[:3, :, x], 0.0))
    lo = slice(0, h)
    up = slice(ny - 1, ny - 1 - h, -1)
    if half == "lower":
        uu, rr = u[lo], rms[:, lo]
    elif half == "upper":
        uu, rr = u[up], rms[:, up]
    else:
        uu, rr = 0.5 * (u[lo] + u[up]), 0.5 * (rms[:, lo] + rms[:, up])
    return y[:h] * ut / nu, uu / ut, rr / ut, ut


def u_theory_force(F, h):
    """Friction velocity of a channel of half-height h driven by the body
    force F per unit volume (density 1): the wall shear balances the force,
    tau_w = F h, so u_tau = sqrt(F h)."""
    return np.sqrt(F * h)


def u_theory_re(re_tau, nu, h):
    """Friction velocity that gives the target Re_tau = u_tau h / nu."""
    return re_tau * nu / h


def autocorrelation(series, max_lag=None):
    """Normalized auto-correlation B(k) = <u'(t) u'(t + k)> / <u'^2> of a
    time series (mean removed), lags 0 .. max_lag."""
    s = np.asarray(series, dtype=np.float64)
    s = s - s.mean()
    n = s.size
    max_lag = n - 1 if max_lag is None else min(max_lag, n - 1)
    var = float(np.dot(s, s)) / n
    if var <= 0:
        raise ValueError("constant series")
    return np.array([float(np.dot(s[: n - k], s[k:])) / (n - k) / var for k in range(max_lag + 1)])


def integral_time(B, dt=1.0):
    """Eq. (time-integral): the integral of B from 0 to its first zero
    (linear interpolation of the crossing, trapezoidal rule)."""
    B = np.asarray(B, dtype=np.float64)
    neg = np.nonzero(B <= 0.0)[0]
    if neg.size == 0:
        return float(np.trapezoid(B, dx=dt)) if hasattr(np, "trapezoid") else float(np.trapz(B, dx=dt))
    k = int(neg[0])
    total = 0.0
    for i in range(k - 1):
        total += 0.5 * (B[i] + B[i + 1]) * dt
    # partial interval up to the crossing between k-1 and k
    b0, b1 = B[k - 1], B[k]
    frac = b0 / (b0 - b1) if b0 != b1 else 0.0
    total += 0.5 * b0 * frac * dt
    return total
