"""Pins for the oracle's hysteresis loop (Sec. 4.1, standard problem 2
driver): a single cubic tile is a Stoner-Wohlfarth particle (its own demag
field is -Ms m / 3, parallel to m, so it exerts no torque), whose descending
branch has closed forms.  With the field at angle psi to the easy axis and
h = H / H_K, H_K = 2 K / (mu0 Ms):

* it jumps at h_sw = -1 / (cos^(2/3) psi + sin^(2/3) psi)^(3/2);
* the projection of m on the field direction is zero at h_sw for
  psi < 45 deg, and on the continuous branch at h = -sin psi cos psi for
  psi > 45 deg;
* at h = 0 it lies along the easy axis (remanence cos psi along the field).
"""
import math

import numpy as np
import pytest

import oracle

MU0 = 4e-7 * math.pi
MS = 8.0e5
K = 5.0e4
HK = 2 * K / (MU0 * MS)


def cube_model():
    return oracle.Model(np.zeros((1, 3)), np.full((1, 3), 10e-9), MS, 0.0, K, (0.0, 0.0, 1.0))


def sw_field(psi):
    return -1.0 / (math.cos(psi) ** (2 / 3) + math.sin(psi) ** (2 / 3)) ** 1.5


def run_loop(psi, dh=0.01):
    md = cube_model()
    d = np.array([math.sin(psi), 0.0, math.cos(psi)])
    h = np.arange(1.2, -1.2 - 1e-9, -dh)
    opts = oracle.ode_opts(rtol=1e-9, atol=1e-9, h0=1e-14, hmax=1e-9)
    st, mavg, m = oracle.hysteresis(md, d[None, :], h * HK, d, opts, 20e-9)
    assert st == oracle.OK
    return h, mavg, d


@pytest.mark.parametrize("psi_deg", [30.0, 60.0])
def test_stoner_wohlfarth_loop(psi_deg):
    psi = math.radians(psi_deg)
    h, mavg, d = run_loop(psi)
    dh = h[0] - h[1]
    hc, mr = oracle.loop_summary(h * HK, mavg, d)
    # remanence: along the easy axis (up to what 20 ns of relaxation at the
    # rate alpha H_K ~ 4e8 /s leaves of the previous value's tilt, ~2e-6)
    np.testing.assert_allclose(mr, [0.0, 0.0, 1.0], atol=1e-5)
    assert abs(mr @ d - math.cos(psi)) < 1e-5
    # the jump: the first field value after which m has a negative z component
    s_jump = int(np.argmax(mavg[:, 2] < 0))
    assert h[s_jump] <= sw_field(psi) + 1e-12
    assert h[s_jump] > sw_field(psi) - 3 * dh  # critical slowing may delay it by a step or two
    if psi_deg < 45:
        assert abs(hc / HK - sw_field(psi)) < 3 * dh
    else:
        assert abs(hc / HK + math.sin(psi) * math.cos(psi)) < 2e-3
    # the upper branch, value by value, against the energy minimum tracked
    # by Newton's method on the torque sin t cos t + h sin(t - psi) = 0
    # (dtheta/dt = -alpha H_K f(theta) with f the torque above, so a value
    # held for t_step leaves at most the change from the previous value times
    # exp(-alpha H_K f'(theta) t_step): the lag grows towards the jump)
    theta = np.arctan2(mavg[:, 0], mavg[:, 2])
    t = psi
    for s in range(s_jump - 2):
        t_prev = t
        for _ in range(50):
            f = math.sin(t) * math.cos(t) + h[s] * math.sin(t - psi)
            t -= f / (math.cos(2 * t) + h[s] * math.cos(t - psi))
        fp = math.cos(2 * t) + h[s] * math.cos(t - psi)
        lag = 2 * abs(t - t_prev) * math.exp(-4000.0 * HK * fp * 20e-9) + 1e-7
        assert abs(theta[s] - t) < lag, (s, h[s], theta[s], t, lag)
    assert np.abs(np.linalg.norm(mavg, axis=1) - 1).max() < 1e-9


def test_loop_summary_on_a_line():
    # a straight descending line crossing zero at h = -0.25
    H = np.linspace(1, -1, 9)
    mavg = np.zeros((9, 3))
    mavg[:, 0] = H + 0.25
    hc, mr = oracle.loop_summary(H, mavg, (1, 0, 0))
    assert abs(hc + 0.25) < 1e-12
    np.testing.assert_allclose(mr, [0.25, 0, 0], atol=1e-12)
