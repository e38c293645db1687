"""Pins of the oracle's tracklet fit (C7 passes and the C9 iteration).

* At zero field a noiseless straight line is fitted exactly, and the final
  covariance equals the batch least-squares covariance of the same linear
  model with the same prior (the seed covariance at the outermost hit).
* Noiseless helices from the generator: the iterated fit returns the
  generator's truth at the innermost hit to 1e-9.
"""
import math

import numpy as np
import pytest

from paper_1712_09416_b300 import synth


def _rows_and_hits(ev):
    sec = np.bincount(ev.sector).argmax()
    m = np.nonzero(ev.sector == sec)[0]
    o = m[np.argsort(ev.row[m])]
    return ev.row[o].astype(np.int32), ev.y[o], ev.z[o], ev.true_sinphi[o]


@pytest.mark.parametrize("s0,t", [(0.0, 0.0), (0.25, 0.5), (-0.4, -0.9), (0.6, 0.1)])
def test_zero_field_line_equals_batch_least_squares(orc, s0, t):
    xr = synth.default_row_x().astype(np.float64)
    rows = np.arange(10, 140, dtype=np.int32)
    c0 = math.sqrt(1 - s0 * s0)
    x0 = xr[rows[0]]
    y0, z0 = 1.5, -20.0
    dx = xr[rows] - x0
    hy = y0 + dx * s0 / c0
    hz = z0 + t * dx / c0
    params = orc.Params()
    rc, p, Ct, chi2, ndf = orc.fit_fixed(xr, rows, hy, hz, n_iter=0, bz=0.0, params=params)
    assert rc == 0
    np.testing.assert_allclose(p[:4], [y0, z0, s0, t], rtol=0, atol=1e-12)
    assert p[4] == 0.0
    assert chi2 < 1e-20 and ndf == 2 * len(rows) - 5
    # batch: state q0 at the innermost hit; the i-th measurement sees
    # y = y0 + dx_i s/c, z = z0 + t dx_i / c; the prior sits on the state at
    # the outermost hit, q_L = F q0.
    def jac_meas(d):
        return np.array([[1, 0, d / c0 ** 3, 0, 0],
                         [0, 1, t * d * s0 / c0 ** 3, d / c0, 0]])
    dL = dx[-1]
    F = np.eye(5)
    F[0, 2] = dL / c0 ** 3
    F[1, 2] = t * dL * s0 / c0 ** 3
    F[1, 3] = dL / c0
    # seed covariance: slope variances carried to sin(phi), tan(lambda) at s0
    P0 = np.diag([params.sigma_y ** 2, params.sigma_z ** 2, params.seed_var_s * c0 ** 6,
                  params.seed_var_t * c0 ** 2, params.seed_var_q])
    Vi = np.diag([1 / params.sigma_y ** 2, 1 / params.sigma_z ** 2])
    info = F.T @ np.linalg.inv(P0) @ F
    for d in dx:
        H = jac_meas(d)
        info += H.T @ Vi @ H
    np.testing.assert_allclose(orc.unpack_cov(Ct), np.linalg.inv(info), rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("q,pt,tanl,phi0", [
    (1.0, 1.5, 0.3, math.radians(14.0)),
    (-1.0, 1.5, -0.6, math.radians(6.0)),
    (1.0, 6.0, 0.8, math.radians(10.0)),
    (-1.0, 0.6, 0.1, math.radians(15.0)),
])
def test_noiseless_helix_iterated_fit_gives_truth(orc, q, pt, tanl, phi0):
    ev = synth.noiseless_track(q, pt, tanl, phi0, n_sectors_phi=18)
    rows, hy, hz, hs = _rows_and_hits(ev)
    assert len(rows) >= 30
    xr = ev.row_x.astype(np.float64)
    rc, p, Ct, chi2, ndf = orc.fit_fixed(xr, rows, hy, hz, n_iter=6, bz=0.5)
    assert rc == 0
    truth = np.array([hy[0], hz[0], hs[0], tanl, q / pt])
    err = np.abs(p - truth)
    assert err[0] < 1e-9 and err[1] < 1e-9, err
    assert err[2] < 1e-9 and err[3] < 1e-9 and err[4] < 1e-9 * max(1.0, abs(q / pt)), err
    assert chi2 < 1e-12


def test_single_pass_noiseless_helix_is_close(orc):
    """The plain C7 passes (no iteration) are already near truth on a noiseless helix."""
    ev = synth.noiseless_track(-1.0, 1.0, 0.4, math.radians(12.0), n_sectors_phi=18)
    rows, hy, hz, hs = _rows_and_hits(ev)
    rc, p, _, _, _ = orc.fit_fixed(ev.row_x.astype(np.float64), rows, hy, hz, n_iter=0, bz=0.5)
    assert rc == 0
    assert abs(p[4] - (-1.0)) < 1e-3
    assert abs(p[0] - hy[0]) < 1e-3 and abs(p[1] - hz[0]) < 1e-3


@pytest.mark.parametrize("s0,t", [(0.0, 0.3), (0.3, 0.5), (-0.5, -0.8)])
def test_seed_of_a_straight_line_is_its_exact_state(orc, s0, t):
    c0 = math.sqrt(1 - s0 * s0)
    x0, x1, y0, z0 = 90.0, 97.0, 2.0, 10.0
    y1 = y0 + (x1 - x0) * s0 / c0
    z1 = z0 + t * (x1 - x0) / c0
    p = orc.seed(x0, y0, z0, x1, y1, z1)
    np.testing.assert_allclose(p, [y0, z0, s0, t, 0.0], rtol=0, atol=1e-14)
