"""Pins for the oracle's local fields, equation of motion and integrator.

Exchange (Eq. 12 with the Neumann condition of Eq. 3), anisotropy (Eq. 16),
energy (Eqs. 4-15), the Landau-Lifshitz right-hand side (Eq. 1, and its
Gilbert form) and the Runge-Kutta (4,5) driver of Sec. 3.1 are checked
against closed forms (discrete Laplacian of a spiral, macrospin precession
and damped switching), invariants (|m| conservation, energy decay, flux
conservation, Eq. 5 as the energy gradient), Butcher's order conditions and
an independent library ODE solver (scipy).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2107_05364_gb300 import workloads as wl

MU0 = 4e-7 * math.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=", 1)
                vals[k.strip()] = [float(x) for x in v.split()]
    return vals


# ---------------------------------------------------------------------------
# exchange, anisotropy, energy
# ---------------------------------------------------------------------------
def test_exchange_uniform_and_linear_give_zero():
    t = wl.graded_film(12, 6, 3, size=(90e-9, 40e-9, 9e-9), seed=2)
    md = oracle.Model.from_tiles(t)
    m = np.tile([0.6, 0.0, 0.8], (t.n, 1))
    assert np.abs(oracle.exchange_field(md, m)).max() == 0.0
    # m linear in x: the finite-volume Laplacian is exact -> 0 on interior tiles
    x = t.centre[:, 0]
    ml = np.stack([x / x.max(), 0.2 + 0 * x, 0.1 + 0 * x], 1)
    H = oracle.exchange_field(md, ml)
    interior = (t.nbr[:, 0] >= 0) & (t.nbr[:, 1] >= 0)
    scale = 2 * t.Aex[0] / (MU0 * t.Ms[0]) / t.edge[:, 0].min() ** 2
    assert np.abs(H[interior]).max() < 1e-9 * scale


def test_exchange_spiral_closed_form():
    # m_i = (cos k x_i, sin k x_i, 0) on a uniform chain: the 3-point stencil
    # gives exactly (2A/(mu0 Ms)) (2 cos(kh) - 2)/h^2 m_i in the interior,
    # -> -k^2 (2A/(mu0 Ms)) m as h -> 0 (Eq. 12)
    L = 200e-9
    for nx in (50, 100, 200):
        t = wl.grid_tiles(np.linspace(0, L, nx + 1), [0, 5e-9], [0, 5e-9], 8e5, 1.3e-11, 0.0)
        md = oracle.Model.from_tiles(t)
        k = 2 * math.pi * 3 / L
        x = t.centre[:, 0]
        m = np.stack([np.cos(k * x), np.sin(k * x), 0 * x], 1)
        H = oracle.exchange_field(md, m)
        h = L / nx
        pref = 2 * 1.3e-11 / (MU0 * 8e5)
        exact = pref * (2 * math.cos(k * h) - 2) / h ** 2 * m
        np.testing.assert_allclose(H[1:-1], exact[1:-1], rtol=1e-9, atol=1e-6 * abs(pref) / h ** 2)
        cont = -k * k * pref * m
        rel = np.abs(H[1:-1] - cont[1:-1]).max() / np.abs(cont).max()
        assert rel < (k * h) ** 2 / 12 * 1.01 + 1e-12


def test_exchange_flux_conservation_graded():
    # Neumann boundary: no flux leaves the body, so sum_i V_i H_ex,i = 0
    t = wl.graded_film(10, 5, 3, size=(80e-9, 40e-9, 9e-9), seed=9)
    md = oracle.Model.from_tiles(t)
    m = wl.m_random(t.n, seed=3)
    H = oracle.exchange_field(md, m)
    s = (t.volume[:, None] * H).sum(0)
    assert np.abs(s).max() < 1e-10 * np.abs(t.volume[:, None] * H).sum()


def test_effective_field_is_energy_gradient():
    # Eq. 5: H_eff,i = -(1/(mu0 Ms_i V_i)) dG/dm_i.  Uniform mesh (so that
    # V_i N_ij = V_j N_ji) with every interaction switched on.
    t = wl.grid_tiles(np.linspace(0, 30e-9, 6), np.linspace(0, 15e-9, 4), [0, 4e-9, 8e-9],
                      8e5, 1.3e-11, 3e5, (0.3, 0.4, 0.866))
    md = oracle.Model.from_tiles(t)
    p = oracle.llg_params(Ha=(1e4, -2e4, 5e3))
    m = wl.m_random(t.n, seed=11)
    H = oracle.effective_field(md, m, p)
    eps = 1e-6
    for i in (0, 7, t.n - 1):
        for c in range(3):
            mp_, mm_ = m.copy(), m.copy()
            mp_[i, c] += eps
            mm_[i, c] -= eps
            g = (oracle.energy(md, mp_, p)["total"] - oracle.energy(md, mm_, p)["total"]) / (2 * eps)
            hfd = -g / (MU0 * t.Ms[i] * t.volume[i])
            assert abs(hfd - H[i, c]) < 1e-6 * np.abs(H).max(), (i, c, hfd, H[i, c])


def test_single_cube_demag_energy_closed_form():
    # one uniformly magnetised cube: E_demag = (mu0 Ms^2 / 2) V / 3
    h = 5e-9
    t = wl.grid_tiles([0, h], [0, h], [0, h], 8e5, 1.3e-11, 0.0)
    md = oracle.Model.from_tiles(t)
    E = oracle.energy(md, [[0.0, 0.6, 0.8]], oracle.llg_params())
    assert abs(E["demag"] - 0.5 * MU0 * 8e5 ** 2 * h ** 3 / 3) < 1e-12 * E["demag"]
    assert E["exchange"] == 0.0


def test_anisotropy_field_closed_form():
    t = wl.grid_tiles([0, 5e-9], [0, 5e-9], [0, 5e-9], 6e5, 1e-11, 4e4, (0, 0.6, 0.8))
    md = oracle.Model.from_tiles(t)
    m = np.array([[0.0, 1.0, 0.0]])
    H = oracle.anisotropy_field(md, m)
    # (2K/(mu0 Ms)) (m.e) e with m.e = 0.6
    np.testing.assert_allclose(H[0], 2 * 4e4 / (MU0 * 6e5) * 0.6 * np.array([0, 0.6, 0.8]), rtol=1e-14)


# ---------------------------------------------------------------------------
# equation of motion
# ---------------------------------------------------------------------------
def test_rhs_preserves_norm_and_forms():
    t = wl.film(8, 4, 1)
    md = oracle.Model.from_tiles(t)
    m = wl.m_random(t.n, seed=5)
    for form, alpha in ((0, 0.02), (0, 0.5), (1, 4420.0)):
        k, tau = oracle.llg_rhs(md, m, oracle.llg_params(alpha=alpha, form=form, Ha=(1e4, 0, 0)))
        # m . dm/dt = 0 (Sec. 2.1: the equation preserves |m|)
        assert np.abs((k * m).sum(1)).max() < 1e-12 * np.abs(k).max()
        assert tau > 0
    # Gilbert with alpha_G equals LL with gamma' = gamma/(1+a^2), alpha_LL = gamma' a
    g, a = 2.211e5, 0.3
    kg, _ = oracle.llg_rhs(md, m, oracle.llg_params(gamma=g, alpha=a, form=0))
    kl, _ = oracle.llg_rhs(md, m, oracle.llg_params(gamma=g / (1 + a * a), alpha=g * a / (1 + a * a), form=1))
    np.testing.assert_allclose(kg, kl, rtol=1e-12, atol=1e-12 * np.abs(kg).max())


def _macrospin(Ha_z=4e4, Ms=8e5):
    h = 5e-9
    t = wl.grid_tiles([0, h], [0, h], [0, h], Ms, 1.3e-11, 0.0)
    return oracle.Model.from_tiles(t)


@pytest.mark.parametrize("form,alpha", [(0, 0.0), (0, 0.1), (1, 0.1 * 2.211e5)])
def test_macrospin_closed_form(form, alpha):
    # one cube, no anisotropy: H_d = -Ms m/3 is parallel to m and drops out of
    # m x H.  With H = H zhat:  phi(t) = phi0 + w t,  tan(theta/2) =
    # tan(theta0/2) exp(-d t); Gilbert: w = gamma' H, d = alpha gamma' H with
    # gamma' = gamma/(1+alpha^2); LL (Eq. 1): w = gamma H, d = alpha H.
    md = _macrospin()
    gamma, H = 2.211e5, 4e4
    th0, ph0 = 1.2, 0.3
    m0 = np.array([[math.sin(th0) * math.cos(ph0), math.sin(th0) * math.sin(ph0), math.cos(th0)]])
    p = oracle.llg_params(gamma=gamma, alpha=alpha, Ha=(0, 0, H), form=form)
    if form == 0:
        w = gamma / (1 + alpha ** 2) * H
        d = alpha * w
    else:
        w = gamma * H
        d = alpha * H
    T = 2e-9
    n_out = 20
    st, m, mavg, stats = oracle.integrate(md, m0, p, oracle.ode_opts(rtol=1e-10, atol=1e-10, h0=1e-15),
                                          0.0, T, n_out)
    assert st == oracle.OK
    ts = T * np.arange(1, n_out + 1) / n_out
    th = 2 * np.arctan(math.tan(th0 / 2) * np.exp(-d * ts))
    ph = ph0 + w * ts
    exp = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    assert np.abs(mavg - exp).max() < 1e-7
    assert abs(np.linalg.norm(m[0]) - 1) < 1e-14


def test_damping_only_keeps_azimuth():
    md = _macrospin()
    m0 = np.array([[0.6, 0.0, 0.8]])
    p = oracle.llg_params(alpha=0.5, Ha=(0, 0, 4e4), precess=0)
    st, m, mavg, _ = oracle.integrate(md, m0, p, oracle.ode_opts(rtol=1e-9, atol=1e-9), 0, 1e-9, 5)
    assert st == oracle.OK
    assert np.abs(mavg[:, 1]).max() < 1e-12
    assert mavg[-1, 2] > 0.8


def test_energy_decays_with_damping():
    # dG/dt = -mu0 sum V Ms (dm/dt . H) <= 0 for alpha > 0 (uniform mesh)
    t = wl.film(12, 4, 1, size=(60e-9, 20e-9, 3e-9))
    md = oracle.Model.from_tiles(t)
    p = oracle.llg_params(alpha=0.1, Ha=(-1.5e4, 4e3, 0))
    m = wl.m_noisy(t.n, (1, 1, 1), 0.05, seed=0)
    E_prev = oracle.energy(md, m, p)["total"]
    for _ in range(6):
        st, m, _, _ = oracle.integrate(md, m, p, oracle.ode_opts(rtol=1e-8, atol=1e-8), 0, 5e-11, 1)
        assert st == oracle.OK
        E = oracle.energy(md, m, p)["total"]
        assert E <= E_prev + 1e-12 * abs(E_prev)
        E_prev = E


# ---------------------------------------------------------------------------
# Runge-Kutta (4,5)
# ---------------------------------------------------------------------------
def test_dp45_order_conditions():
    # Butcher's conditions: b is 5th order, bhat 4th order but not 5th
    c, A, b, bh = oracle.dp45_tableau()
    Af = np.zeros((7, 7))
    Af[:, :6] = A
    np.testing.assert_allclose(Af.sum(1), c, atol=1e-15)  # row sums = nodes

    def conds(w):
        return [w.sum() - 1, w @ c - 1 / 2, w @ c ** 2 - 1 / 3, w @ (Af @ c) - 1 / 6,
                w @ c ** 3 - 1 / 4, w @ (c * (Af @ c)) - 1 / 8, w @ (Af @ c ** 2) - 1 / 12,
                w @ (Af @ Af @ c) - 1 / 24,
                w @ c ** 4 - 1 / 5, w @ (c ** 2 * (Af @ c)) - 1 / 10, w @ ((Af @ c) ** 2) - 1 / 20,
                w @ (c * (Af @ c ** 2)) - 1 / 15, w @ (Af @ c ** 3) - 1 / 20,
                w @ (c * (Af @ Af @ c)) - 1 / 30, w @ (Af @ (c * (Af @ c))) - 1 / 40,
                w @ (Af @ Af @ c ** 2) - 1 / 60, w @ (Af @ Af @ Af @ c) - 1 / 120]
    assert np.abs(conds(b)).max() < 1e-14
    assert np.abs(conds(bh)[:8]).max() < 1e-14
    assert np.abs(conds(bh)[8:]).max() > 1e-4
    # first same as last: last row of A equals b
    np.testing.assert_allclose(A[6], b[:6], atol=0)


def test_dp45_linear_problem():
    lam = np.array([-1.0, 0.5, -20.0, 2.0])
    y0 = np.array([1.0, -2.0, 0.5, 0.1])
    st, y, yout, stats = oracle.integrate_linear(lam, y0, oracle.ode_opts(rtol=1e-10, atol=1e-12, h0=1e-3,
                                                                          hmax=1.0), 0.0, 2.0, 8)
    assert st == oracle.OK
    ts = 2.0 * np.arange(1, 9) / 8
    np.testing.assert_allclose(yout, y0[None, :] * np.exp(lam[None, :] * ts[:, None]), rtol=2e-9, atol=1e-12)
    assert stats["n_reject"] >= 0 and stats["n_accept"] > 8


def test_dp45_fixed_step_fifth_order():
    lam = np.array([-1.3, 0.7])
    y0 = np.array([1.0, 1.0])
    errs = []
    for h in (0.1, 0.05, 0.025):
        st, y, _, _ = oracle.integrate_linear(lam, y0, oracle.ode_opts(fixed_h=h), 0.0, 1.0, 1)
        assert st == oracle.OK
        errs.append(np.abs(y - np.exp(lam)).max())
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(r > 26) and np.all(r < 40), r


def test_against_scipy_nonlinear():
    # one tile with anisotropy at an angle and an oblique applied field: a
    # nonlinear ODE; compare with scipy's DOP853 at tight tolerance
    scipy_int = pytest.importorskip("scipy.integrate")
    h = 4e-9
    t = wl.grid_tiles([0, h], [0, h * 1.5], [0, h * 0.7], 8e5, 1.3e-11, 2e5, (0.2, 0.5, 0.84))
    md = oracle.Model.from_tiles(t)
    p = oracle.llg_params(alpha=0.05, Ha=(2e4, -3e4, 1e4))
    m0 = np.array([[0.1, 0.7, -0.7]])
    m0 /= np.linalg.norm(m0)

    def f(_, y):
        k, _ = oracle.llg_rhs(md, y, p)
        return k.ravel()

    T = 0.3e-9
    ref = scipy_int.solve_ivp(f, (0, T), m0.ravel(), method="DOP853", rtol=1e-12, atol=1e-12,
                              t_eval=T * np.arange(1, 7) / 6)
    st, m, mavg, _ = oracle.integrate(md, m0, p, oracle.ode_opts(rtol=1e-10, atol=1e-10, h0=1e-15), 0, T, 6)
    assert st == oracle.OK
    assert np.abs(mavg - ref.y.T).max() < 2e-8


# ---------------------------------------------------------------------------
# relaxation (Brown's equation, Eq. 2)
# ---------------------------------------------------------------------------
def test_mean_m_is_volume_weighted():
    # <m> of the traces is the volume average (1/V) sum_i V_i m_i.  Two tiles
    # of volumes V and 3V magnetised along x and y: <m> = (1/4, 3/4, 0) (an
    # unweighted mean would give (1/2, 1/2, 0)).  With gamma = 0 the equation
    # of motion is dm/dt = 0, so the integrator's recorded <m> is that of m0.
    h = 2e-9
    centre = np.array([[0.0, 0.0, 0.0], [3.0 * h, 0.0, 0.0]])
    edge = np.array([[h, h, h], [3.0 * h, h, h]])
    md = oracle.Model(centre, edge, wl.SP4_MS, wl.SP4_AEX, 0.0, (0, 0, 1))
    m0 = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    p = oracle.llg_params(gamma=0.0, alpha=0.0)
    st, m, mavg, _ = oracle.integrate(md, m0, p, oracle.ode_opts(fixed_h=1e-13), 0.0, 3e-13, 3)
    assert st == oracle.OK
    np.testing.assert_array_equal(m, m0)
    np.testing.assert_allclose(mavg, np.tile([0.25, 0.75, 0.0], (3, 1)), rtol=0, atol=1e-15)
    np.testing.assert_allclose(md.mean_m(m0), [0.25, 0.75, 0.0], rtol=0, atol=1e-15)
    # a graded film: the same against a sum written out tile by tile
    t = wl.graded_film(9, 5, 3, size=(60e-9, 30e-9, 9e-9), seed=6)
    mr = wl.m_random(t.n, seed=4)
    num, den = np.zeros(3), 0.0
    for i in range(t.n):
        V = t.edge[i, 0] * t.edge[i, 1] * t.edge[i, 2]
        num += V * mr[i]
        den += V
    mdg = oracle.Model.from_tiles(t)
    st, _, mavg, _ = oracle.integrate(mdg, mr, p, oracle.ode_opts(fixed_h=1e-13), 0.0, 1e-13, 1)
    assert st == oracle.OK
    np.testing.assert_allclose(mavg[0], num / den, rtol=0, atol=1e-14)
    assert np.abs(mavg[0] - mr.mean(0)).max() > 1e-3  # the grading matters here


def test_relax_reaches_equilibrium():
    t = wl.film(10, 3, 1, size=(100e-9, 30e-9, 3e-9))
    md = oracle.Model.from_tiles(t)
    p = oracle.llg_params(alpha=0.5)
    m0 = wl.m_noisy(t.n, (1, 1, 1), 1e-3, seed=0)
    E0 = oracle.energy(md, m0, p)["total"]
    st, m, stats = oracle.relax(md, m0, p, oracle.ode_opts(rtol=1e-6, atol=1e-6), 1e-6, 20e-9)
    assert st == oracle.OK, stats
    _, tau = oracle.llg_rhs(md, m, p)
    assert tau < 2e-6
    assert oracle.energy(md, m, p)["total"] < E0
    np.testing.assert_allclose(np.linalg.norm(m, axis=1), 1.0, atol=1e-14)


def test_relax_reports_no_convergence_at_cap():
    t = wl.film(6, 2, 1, size=(60e-9, 20e-9, 3e-9))
    md = oracle.Model.from_tiles(t)
    st, _, stats = oracle.relax(md, wl.m_noisy(t.n), oracle.llg_params(alpha=0.02),
                                oracle.ode_opts(), 1e-9, 1e-12)
    assert st == oracle.ENOCONV


# ---------------------------------------------------------------------------
# values printed in the paper
# ---------------------------------------------------------------------------
def test_sp4_parameters_golden():
    g = _read_golden("sp4_parameters.txt")
    t = wl.film(40, 10, 1)
    assert t.Ms[0] == g["Ms"][0] and t.Aex[0] == g["A_exch"][0]
    lo = t.centre - t.edge / 2
    hi = t.centre + t.edge / 2
    np.testing.assert_allclose(hi.max(0) - lo.min(0), np.array(g["size_nm"]) * 1e-9, rtol=1e-14)
    # reading of the damping value: the paper's alpha is the LL-form rate
    # alpha_LL = gamma * alpha_G with alpha_G = 0.02 (the muMAG SP4 value)
    assert abs(g["gamma"][0] * 0.02 - g["alpha"][0]) < 1e-9 * g["alpha"][0]
    # field 1 in A/m
    assert abs(g["field1_mT"][0] * 1e-3 / MU0 - (-24.6e-3 / MU0)) < 1e-9
