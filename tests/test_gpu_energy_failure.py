"""GPU energy (Eqs. 4, 6, 8, 11, 15) against the FP64 oracle, the SP3 cube
flower/vortex relaxations, and the failure-detection path of the device
waits (a wait that can never complete gives up, reports MT_ETIMEOUT and the
context stays usable) -- no GPU fault is provoked."""
import time

import numpy as np
import pytest

import oracle
from paper_2107_05364_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


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


def test_energy_matches_oracle(mt, ctx):
    import torch
    t = wl.graded_film(22, 9, 2, (220e-9, 90e-9, 6e-9), seed=3)
    t.Ku[:] = 6e4
    t.axis[:] = np.array([0.0, 0.6, 0.8])
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    md = oracle.Model.from_tiles(t)
    B = 2
    Ha = np.array([[1.5e4, -2e4, 3e3], [0, 0, 4e4]])
    m = np.stack([wl.m_random(t.n, seed=30 + b) for b in range(B)]).astype(np.float32)
    p, keep = mt.llg_params(B, Ha=Ha)
    E = mt.mt_energy(T, p, torch.tensor(m.ravel(), device="cuda"), B=B)
    for b in range(B):
        ref = oracle.energy(md, m[b].astype(np.float64), oracle.llg_params(Ha=Ha[b]))
        got = dict(zip(("total", "zeeman", "demag", "exchange", "anisotropy"), E[b]))
        for k in ref:
            assert abs(got[k] - ref[k]) <= 1e-5 * max(abs(ref[k]), 1e-3 * abs(ref["demag"])), (b, k, got[k], ref[k])


def test_sp3_cube_flower_and_vortex(mt, ctx):
    # 20 l_ex cube as 20^3 tiles (n = 8,000), K_u = 0.1 K_m along z: both
    # seeds lower their energy under damping; the vortex (the low-energy state
    # this far above the crossover) keeps its circulation
    import torch
    t = wl.cube(20, 20.0)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    p, keep = mt.llg_params(1, alpha=0.5)
    for name, m0 in (("flower", wl.m_flower(t)), ("vortex", wl.m_vortex(t))):
        m0 = m0.astype(np.float32)
        E0 = mt.mt_energy(T, p, torch.tensor(m0.ravel(), device="cuda"))[0, 0]
        I = mt.Integrator(T, p, mt.ode_opts(rtol=1e-6, atol=1e-6))
        I.set_state(m0.ravel())
        I.run(2e-9, 1)
        m = I.get_state()[0]
        E = mt.mt_energy(T, p, torch.tensor(m.ravel(), device="cuda"))[0, 0]
        assert E < E0, name
        mean = m.mean(0)
        np.testing.assert_allclose(np.linalg.norm(m, axis=1), 1.0, atol=1e-5)
        print("SP3 cube %s: E %.4e -> %.4e J, <m> = %s" % (name, E0, E, np.round(mean, 4)))
        if name == "vortex":
            c = t.centre - t.centre.mean(0)
            circ = (c[:, 0] * m[:, 1] - c[:, 1] * m[:, 0]).mean() / np.abs(c[:, :2]).mean()
            assert circ > 0.3 and abs(mean[0]) < 0.2 and abs(mean[1]) < 0.2, (circ, mean)


def test_bounded_wait_gives_up_and_context_survives(mt, ctx):
    import torch
    t0 = time.time()
    st = mt.mt_selftest_wait_timeout(ctx, 0.2)
    dt = time.time() - t0
    assert st == mt.MT_ETIMEOUT
    assert 0.15 < dt < 5.0
    # the context still computes
    t = wl.film(8, 2, 1)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    mg = torch.tensor(wl.m_random(t.n).astype(np.float32).ravel(), device="cuda")
    H = torch.empty_like(mg)
    mt.mt_demag_field(T, mg, H)
    torch.cuda.synchronize()
    assert torch.isfinite(H).all()


def test_grid_barrier_gives_up_and_context_survives(mt, ctx):
    # one CTA of a cooperative launch never arrives at the barrier the
    # one-kernel integrator uses between its stages: the others give up
    # after their bounded wait and report it; the context keeps working,
    # including the one-kernel path itself
    t0 = time.time()
    st = mt.mt_selftest_grid_barrier_timeout(ctx)
    dt = time.time() - t0
    assert st == mt.MT_ETIMEOUT
    assert 1.5 < dt < 10.0
    t = wl.film(20, 5, 1)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    p, keep = mt.llg_params(1, alpha=0.1)
    I = mt.Integrator(T, p, mt.ode_opts(fixed_h=1e-13))
    assert I.path() == mt.MT_PATH_PERSISTENT
    I.set_state(wl.m_noisy(t.n, (1, 1, 1), 1e-2, seed=0).astype(np.float32).ravel())
    I.step(5)
    s = I.stats()[0]
    assert s["status"] == 0 and s["n_accept"] == 5
    assert np.isfinite(I.get_state()).all()
