"""Hysteresis driver (Sec. 4.1, standard problem 2) on the GPU: the
per-simulation exchange factor against the oracle on geometries that are
really scaled, a Stoner-Wohlfarth particle against its closed forms, and a
batched standard-problem-2 loop over several d / l_ex against the oracle's
loop on each scaled film."""
import math

import numpy as np
import pytest

import oracle
from paper_2107_05364_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
MU0 = 4e-7 * math.pi


@pytest.fixture(scope="module")
def mt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2107_05364_gb300 import build
    build.build()
    from paper_2107_05364_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(mt):
    return mt.mt_ctx_create(0)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def scaled(t, lam):
    return oracle.Model(lam * t.centre, lam * t.edge, t.Ms, t.Aex, t.Ku, t.axis, t.nbr)


def test_exch_scale_is_a_scaled_geometry(mt, ctx):
    import torch
    t = wl.sp2_film(20, 4, 3, d_lex=10.0)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    lams = np.array([1.0, 0.5, 2.0, 3.0])
    B = len(lams)
    m = np.stack([wl.m_random(t.n, seed=20 + b) for b in range(B)]).astype(np.float32)
    Ha = np.array([3e4, -1e4, 2e4])
    p, keep = mt.llg_params(B, alpha=4000.0, Ha=Ha, form=mt.MT_FORM_LL, precess=0, exch_scale=1 / lams ** 2)
    mg = torch.tensor(m.ravel(), device="cuda")
    dm = torch.empty_like(mg)
    mt.mt_llg_rhs(T, p, mg, dm, B=B)
    E = mt.mt_energy(T, p, mg, B=B)
    torch.cuda.synchronize()
    dm = dm.cpu().numpy().reshape(B, -1, 3)
    for b, lam in enumerate(lams):
        md = scaled(t, lam)
        pr = oracle.llg_params(alpha=4000.0, Ha=Ha, form=1, precess=0)
        ref, _ = oracle.llg_rhs(md, m[b].astype(np.float64), pr)
        assert _rel(dm[b], ref) < 1e-5, (lam, _rel(dm[b], ref))
        # energies: every density is intensive, so the scaled geometry's
        # energy is lam^3 times the reference tiles' with A / lam^2
        eo = oracle.energy(md, m[b].astype(np.float64), pr)
        assert abs(E[b][0] * lam ** 3 - eo["total"]) <= 1e-5 * abs(eo["total"])


def sw_cube():
    return wl.grid_tiles([0, 10e-9], [0, 10e-9], [0, 10e-9], 8.0e5, 0.0, 5.0e4, (0, 0, 1))


def test_stoner_wohlfarth_batch(mt, ctx):
    t = sw_cube()
    HK = 2 * 5.0e4 / (MU0 * 8.0e5)
    psis = np.radians([30.0, 60.0])
    dirs = np.stack([np.sin(psis), np.zeros(2), np.cos(psis)], axis=1)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    p, keep = mt.llg_params(2, alpha=4000.0, form=mt.MT_FORM_LL, precess=0)
    I = mt.Integrator(T, p, mt.ode_opts(rtol=1e-6, atol=1e-6, h0=1e-14, hmax=1e-9), B=2)
    I.set_state(dirs.astype(np.float32).ravel())
    dh = 0.01
    h = np.arange(1.2, -1.2 - 1e-9, -dh)
    mavg, tau, hc, mr, st = I.hysteresis(dirs, h * HK, 20e-9)
    md = oracle.Model.from_tiles(t)
    for b, psi in enumerate(psis):
        sw = -1.0 / (math.cos(psi) ** (2 / 3) + math.sin(psi) ** (2 / 3)) ** 1.5
        s_jump = int(np.argmax(mavg[:, b, 2] < 0))
        assert sw - 3 * dh < h[s_jump] <= sw + 1e-12
        if psi < math.pi / 4:
            assert abs(hc[b] / HK - sw) < 3 * dh
        else:
            assert abs(hc[b] / HK + math.sin(psi) * math.cos(psi)) < 2e-3
        np.testing.assert_allclose(mr[b], [0, 0, 1], atol=1e-4)
        # the oracle's loop, value by value, away from the jump
        opts = oracle.ode_opts(rtol=1e-9, atol=1e-9, h0=1e-14, hmax=1e-9)
        sto, mo, _ = oracle.hysteresis(md, dirs[b][None, :], h * HK, dirs[b], opts, 20e-9)
        assert sto == oracle.OK
        far = np.abs(np.arange(len(h)) - s_jump) > 2
        assert np.abs(mavg[far, b] - mo[far]).max() < 1e-4


def test_sp2_loop_batched_over_d_lex(mt, ctx):
    # reference tiles at d / l_ex = 10; the batch covers 10, 20, 30 with
    # exchange factors (10 / d_lex)^2, the oracle runs each film really scaled
    t = wl.sp2_film(20, 4, 1, d_lex=10.0)
    d_lex = np.array([10.0, 20.0, 30.0])
    lams = d_lex / 10.0
    B = len(d_lex)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    H = wl.sp2_fields(9)
    t_step = 10e-9
    p, keep = mt.llg_params(B, alpha=4000.0, form=mt.MT_FORM_LL, precess=0, exch_scale=1 / lams ** 2)
    opts = dict(rtol=1e-6, atol=1e-6, h0=1e-14, hmax=1e-10)
    I = mt.Integrator(T, p, mt.ode_opts(**opts), B=B)
    m0 = wl.m_noisy(t.n, wl.SP2_DIR, 1e-3, seed=0).astype(np.float32)
    I.set_state(np.tile(m0.ravel(), B))
    mavg, tau, hc, mr, st = I.hysteresis(wl.SP2_DIR, H, t_step)
    for b, lam in enumerate(lams):
        md = scaled(t, lam)
        sto, mo, _ = oracle.hysteresis(md, m0.astype(np.float64), H, wl.SP2_DIR, oracle.ode_opts(**opts), t_step)
        assert sto == oracle.OK
        dev = np.abs(mavg[:, b] - mo).max()
        print("d/l_ex %g: max |d<m>| %.2e, hc/Ms %.4f" % (d_lex[b], dev, hc[b] / wl.SP4_MS))
        assert dev < 1e-4, (d_lex[b], dev)
        hco, mro = oracle.loop_summary(H, mo, wl.SP2_DIR)
        assert (np.isnan(hc[b]) and np.isnan(hco)) or abs(hc[b] - hco) < 1e-3 * wl.SP4_MS
        np.testing.assert_allclose(mr[b], mro, atol=1e-4)


def test_sp2_loop_relaxed_to_torque_matches_oracle(mt, ctx):
    # the coarse-loop mode: each value relaxed until max |m x H| / Ms < 5e-3
    # (cap 10 ns; the first values stop early, the ones near the switch run
    # to the cap); two runs that stop below the same torque agree to about
    # that torque over the stiffness of the softest mode
    t = wl.sp2_film(20, 4, 1, d_lex=20.0)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    H = wl.sp2_fields(7)
    p, keep = mt.llg_params(1, alpha=4000.0, form=mt.MT_FORM_LL, precess=0)
    opts = dict(rtol=1e-7, atol=1e-7, h0=1e-14, hmax=1e-10)
    I = mt.Integrator(T, p, mt.ode_opts(**opts))
    m0 = wl.m_noisy(t.n, wl.SP2_DIR, 1e-3, seed=0).astype(np.float32)
    I.set_state(m0.ravel())
    mavg, tau, hc, mr, st = I.hysteresis(wl.SP2_DIR, H, 10e-9, tol=5e-3)
    md = oracle.Model.from_tiles(t)
    sto, mo, _ = oracle.hysteresis(md, m0.astype(np.float64), H, wl.SP2_DIR, oracle.ode_opts(**opts), 10e-9,
                                   tol=5e-3)
    assert sto == oracle.OK
    dev = np.abs(mavg[:, 0] - mo).max()
    print("relax-to-torque loop: max |d<m>| %.2e, torque at the ends %s" % (dev, np.round(tau[:, 0], 6)))
    assert dev < 2e-3
    assert np.any(tau[:, 0] < 5e-3) and np.any(tau[:, 0] >= 5e-3)  # both endings occurred
