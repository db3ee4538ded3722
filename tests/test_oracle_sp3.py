"""Pins for the oracle's standard-problem-3 pieces (Sec. 4.2): the crossing
search on lines with a known crossing, and the energy density of a small
cube, where exchange forces a uniform state whose energy has a plain form."""
import math

import numpy as np

import oracle
from paper_2107_05364_gb300 import workloads as wl

MU0 = 4e-7 * math.pi
KM = 0.5 * MU0 * 8e5 ** 2


def test_first_crossing_on_lines():
    x = np.linspace(7, 10, 7)
    a = 0.2 - 0.01 * (x - 8.3)
    b = 0.2 - 0.03 * (x - 8.3)
    assert abs(oracle.first_crossing(x, a, b) - 8.3) < 1e-12
    assert math.isnan(oracle.first_crossing(x, a, a + 1))
    # the first of two crossings
    c = 0.2 + 0.001 * np.cos(3 * x)
    xs = oracle.first_crossing(x, c, np.full_like(x, 0.2))
    assert x[0] < xs < x[2]


def test_small_cube_approaches_the_uniform_state():
    # for a small cube exchange dominates: both seeds relax to the same
    # flower, close to m = z, whose energy density lies below the uniform
    # state's  K_m / 3 - K_u  (the tile tensor of a cube averages to I/3 by
    # symmetry) by a gain that vanishes as L^2 (perturbation about uniform)
    t = wl.cube(4, 1.0)
    N = oracle.demag_tensor(t.centre, t.edge)
    assert abs(N[:, :, 5].sum() / t.n - 1 / 3) < 1e-13
    e_uniform = KM / 3 - t.Ku[0]
    md = oracle.Model.from_tiles(t)
    p = oracle.llg_params(alpha=4000.0, form=1, precess=0)
    eu = oracle.energy(md, np.tile([0.0, 0.0, 1.0], (t.n, 1)), p)["total"] / md.volume.sum()
    assert abs(eu - e_uniform) < 1e-12 * KM
    opts = oracle.ode_opts(rtol=1e-8, atol=1e-8, h0=1e-14, hmax=1e-10)
    lam = [0.25, 0.5]
    eA, eB, lc, states = oracle.crossover(t.centre, t.edge, t.Ms, t.Aex, t.Ku, t.axis, t.nbr, lam,
                                          wl.m_flower(t), wl.m_vortex(t), p, opts, 1e-7, 50e-9)
    gain = e_uniform - eA
    assert np.all(gain > 0)
    np.testing.assert_allclose(eB, eA, rtol=1e-10)
    assert 3.9 < gain[1] / gain[0] < 4.05
    assert math.isnan(lc)
    for m in states:
        assert np.abs(m.mean(0) - [0, 0, 1]).max() < 2e-6
