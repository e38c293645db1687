"""Storage-precision emulation of the tracklet fit (test infrastructure).

Re-states, in numpy float64 arithmetic, the fit sequence the sector tracker
applies to a tracklet whose hits are known (chord seed from the start hit to
the chain end, forward pass over the rows from the start row to the last hit,
covariance reset to the seed at the last hit, backward pass down to the
innermost hit; helix transport with its exact Jacobian, Kalman update with
diagonal measurement variance).  After every transport and update the state
and/or chosen covariance entries can be rounded to binary32, which separates
the effect of binary32 *storage* from that of binary32 arithmetic.

Used to show that some binary64-vs-binary32 differences of the fitted q/pT
are a property of storing the covariance itself in binary32, and that
storing a square-root factor U (C = U U^T) instead, as the tracker's
backward pass does, removes them.  Shares no code with the CUDA path or the
oracle.
"""
import math

import numpy as np

KAPPA = 0.299792458e-2


def _transport_j(x0, x1, p, kB):
    dx = x1 - x0
    ck = -kB * p[4]
    s0 = p[2]
    s1 = s0 + ck * dx
    c0 = math.sqrt((1 - s0) * (1 + s0))
    c1 = math.sqrt((1 - s1) * (1 + s1))
    cc, ss = c0 + c1, s0 + s1
    dy = dx * ss / cc
    ch = math.hypot(dx, dy)
    h = 0.5 * abs(ck) * ch
    dS = ch * (math.asin(h) / h if h > 0 else 1.0) * (-1.0 if dx < 0 else 1.0)
    t = p[3]
    J = np.eye(5)
    J[0, 2] = dx * (2 * cc + ss * (s0 / c0 + s1 / c1)) / (cc * cc)
    J[0, 4] = -kB * dx * dx * (cc + ss * s1 / c1) / (cc * cc)
    J[1, 2] = t * dx * ss / (c0 * c1 * cc)
    J[1, 3] = dS
    dphi = ck * dS
    if abs(dphi) < 1e-6:
        sinc2, rest = 1.0, -dphi / 6.0
    else:
        hs = math.sin(0.5 * dphi) / (0.5 * dphi)
        sinc2, rest = hs * hs, (math.sin(dphi) - dphi) / (dphi * dphi)
    J[1, 4] = -kB * t * dS * dS * (0.5 * s1 / c1 * sinc2 + rest)
    J[2, 4] = -kB * dx
    q = p.copy()
    q[0] += dy
    q[1] += t * dS
    q[2] = s1
    return q, J


def _transport(x0, x1, p, C, kB):
    q, J = _transport_j(x0, x1, p, kB)
    return q, J @ C @ J.T


def _update(p, C, my, mz, vy, vz):
    S = C[:2, :2] + np.diag([vy, vz])
    K = C[:, :2] @ np.linalg.inv(S)
    r = np.array([my - p[0], mz - p[1]])
    return p + K @ r, C - K @ C[:2, :]


def _seed_cov(s, vy, vz, var_s, var_t, var_q):
    c2 = (1 - s) * (1 + s)
    return np.diag([vy, vz, var_s * c2 ** 3, var_t * c2, var_q])


def _factor_update(p, U, i, m, v):
    """Scalar measurement of component i in Potter's square-root form:
    a = U^T e_i, alpha = a.a + v, p += U a r / alpha,
    U <- U - U a a^T / (alpha + sqrt(alpha v))."""
    a = U[i].copy()
    alpha = a @ a + v
    w = U @ a
    r = m - p[i]
    return p + w * (r / alpha), U - np.outer(w, a) / (alpha + math.sqrt(alpha * v))


def fit_known_hits(row_x, hy, hz, rowhit, r0, rk, *, bz=0.5, sigma=0.1, seed_var=(1.0, 1.0, 100.0),
                   round_state=False, round_cov=None, backward_factor=False):
    """State at the innermost hit of a tracklet with hit rowhit[r] (cluster
    index or -1) on row r, start row r0 and chain end row rk.  round_cov is a
    5x5 boolean mask of covariance entries rounded to binary32 after every
    step (None: none); round_state rounds the 5-vector likewise.  With
    backward_factor the backward pass carries a square-root factor U of the
    covariance (C = U U^T) instead, and round_cov rounds entries of U."""
    kB = KAPPA * bz
    vy = vz = sigma * sigma
    xr = np.asarray(row_x, np.float64)
    Y = np.asarray(hy, np.float64)
    Z = np.asarray(hz, np.float64)
    f32 = lambda v: v.astype(np.float32).astype(np.float64)
    rp = f32 if round_state else (lambda v: v)
    rc = (lambda C: np.where(round_cov, f32(C), C)) if round_cov is not None else (lambda C: C)
    rows = np.nonzero(rowhit >= 0)[0]
    last, first = int(rows.max()), int(rows.min())
    h0, hk = rowhit[r0], rowhit[rk]
    tphi = (Y[hk] - Y[h0]) / (xr[rk] - xr[r0])
    dzdx = (Z[hk] - Z[h0]) / (xr[rk] - xr[r0])
    cphi = 1.0 / math.sqrt(1.0 + tphi * tphi)
    yref, zref = Y[h0], Z[h0]  # y and z relative to the start hit
    p = rp(np.array([0.0, 0.0, tphi * cphi, dzdx * cphi, 0.0]))
    C = rc(_seed_cov(p[2], vy, vz, *seed_var))
    p, C = _update(p, C, 0.0, 0.0, vy, vz)
    p, C = rp(p), rc(C)
    x = xr[r0]
    for r in range(r0 + 1, last + 1):
        p, C = _transport(x, xr[r], p, C, kB)
        p, C, x = rp(p), rc(C), xr[r]
        if rowhit[r] >= 0:
            p, C = _update(p, C, Y[rowhit[r]] - yref, Z[rowhit[r]] - zref, vy, vz)
            p, C = rp(p), rc(C)
    if backward_factor:
        U = rc(np.sqrt(_seed_cov(p[2], vy, vz, *seed_var)))
        x = xr[last]
        for r in range(last, first - 1, -1):
            if r != last:
                p, J = _transport_j(x, xr[r], p, kB)
                p, U, x = rp(p), rc(J @ U), xr[r]
            if rowhit[r] >= 0:
                p, U = _factor_update(p, U, 0, Y[rowhit[r]] - yref, vy)
                p, U = _factor_update(p, U, 1, Z[rowhit[r]] - zref, vz)
                p, U = rp(p), rc(U)
        out = p.copy()
        out[0] += yref
        out[1] += zref
        return out
    C = rc(_seed_cov(p[2], vy, vz, *seed_var))
    p, C = _update(p, C, Y[rowhit[last]] - yref, Z[rowhit[last]] - zref, vy, vz)
    p, C, x = rp(p), rc(C), xr[last]
    for r in range(last - 1, first - 1, -1):
        p, C = _transport(x, xr[r], p, C, kB)
        p, C, x = rp(p), rc(C), xr[r]
        if rowhit[r] >= 0:
            p, C = _update(p, C, Y[rowhit[r]] - yref, Z[rowhit[r]] - zref, vy, vz)
            p, C = rp(p), rc(C)
    out = p.copy()
    out[0] += yref
    out[1] += zref
    return out
