"""Served jobs against the FP64 oracle, through the C ABI.

A mix of relax jobs (Sec. 4.1, Brown's criterion Eq. 2) and field-sweep jobs
(the Sec. 4.1 field loop as one request) on three small geometries is served
by FP32 streaming engines under an HBM budget that holds two engines at a
time, so engines are evicted and re-assembled while jobs run.  Every served
result is compared element by element with the oracle run on the same
inputs: a relax job's final state with oracle.relax, a sweep job's <m> at
the end of every field value and its final state with oracle.hysteresis (the
same schedule, tolerance and cap per value).  Bound: max |dm| <= 1e-4 (the
relaxed-state tolerance); both sides relax to a torque of 1e-5 with
rtol = atol = 1e-7, so that the stopping points agree well inside it.
"""
import numpy as np
import pytest

import oracle
from _observe import observe
from paper_2107_05364_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
MU0 = 4e-7 * np.pi
GAMMA = 2.211e5
TOL, T_CAP, RTOL = 1e-5, 20e-9, 1e-7


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


def _geoms():
    return [wl.film(12, 4, 1, size=(60e-9, 20e-9, 3e-9)),
            wl.grid_tiles(np.linspace(0, 20e-9, 5), np.linspace(0, 20e-9, 5), np.linspace(0, 15e-9, 4),
                          6e5, 1.3e-11, 0.0),
            wl.film(20, 5, 1, size=(100e-9, 25e-9, 3e-9), Ms=1.0e6)]


def _jobs(geoms):
    """Nine jobs in arrival order: relax and sweep, on every geometry."""
    u = wl.unit01(11, 600, 27)
    jobs = []
    for k in range(9):
        g = k % 3
        a = u[3 * k:3 * k + 3]
        d = np.array([np.cos(6.283 * a[0]), np.sin(6.283 * a[0]), 0.2])
        d /= np.linalg.norm(d)
        m0 = wl.m_noisy(geoms[g].n, d + np.array([0.0, 0.0, 0.3]), 0.2, seed=700 + k)
        alpha = (0.5, 1.0, 0.3)[k % 3]
        if k % 2 == 0:
            Ha = (20e-3 + 40e-3 * a[1]) / MU0 * d
            jobs.append(dict(kind="relax", geometry=g, m0=m0, alpha=alpha, Ha=Ha))
        else:
            # descending field values along one direction, away from switching
            H = np.array([60e-3, 35e-3, 15e-3]) / MU0
            jobs.append(dict(kind="sweep", geometry=g, m0=m0, alpha=alpha, H=H, d=d))
    return jobs


def test_served_relax_and_sweep_jobs_match_oracle(mt, ctx):
    geoms = _geoms()
    jobs = _jobs(geoms)
    opts = dict(rtol=RTOL, atol=RTOL, h0=1e-14, hmax=1e-11)
    # room for two engines: a third geometry evicts the least recently used
    S = mt.Server(ctx, max_batch=2, prec="f32", hbm_budget_bytes=11 << 20, opts=mt.ode_opts(**opts))
    gids = [S.add_geometry(t) for t in geoms]
    ids = []
    for j in jobs:
        if j["kind"] == "relax":
            ids.append(S.submit(gids[j["geometry"]], j["m0"], alpha=j["alpha"], Ha=j["Ha"], tol=TOL, t_max=T_CAP))
        else:
            ids.append(S.submit(gids[j["geometry"]], j["m0"], alpha=j["alpha"], tol=TOL, t_max=T_CAP,
                                fields=j["H"][:, None] * j["d"][None, :]))
    out = [S.wait(i, 300.0, geometry=gids[j["geometry"]]) for i, j in zip(ids, jobs)]
    st = S.stats()
    S.close()
    assert st["evictions"] >= 1 and st["assemblies"] >= 3, st
    assert st["completed"] == len(jobs) and st["failed"] == 0, st
    models = [oracle.Model.from_tiles(t) for t in geoms]
    worst = 0.0
    for (s, r, m), j in zip(out, jobs):
        assert s == 0 and r["status"] == 0, (j["kind"], r)
        md = models[j["geometry"]]
        m0 = j["m0"].astype(np.float32).astype(np.float64)  # what the server was given
        if j["kind"] == "relax":
            so, mo, sto = oracle.relax(md, m0, oracle.llg_params(gamma=GAMMA, alpha=j["alpha"], Ha=j["Ha"]),
                                       oracle.ode_opts(**opts), TOL, T_CAP)
            assert so == oracle.OK and r["tau"] < TOL and r["values_done"] == 1 and r["values_converged"] == 1
            dm = np.abs(m - mo).max()
        else:
            so, mavg, mo = oracle.hysteresis(md, m0, j["H"], j["d"], oracle.ode_opts(**opts), T_CAP,
                                             gamma=GAMMA, alpha=j["alpha"], form=0, precess=1, tol=TOL)
            assert so == oracle.OK
            assert r["values_done"] == len(j["H"])
            sw = r["sweep"]
            assert np.all(sw[:, 3] < TOL), sw
            dm = max(np.abs(m - mo).max(), np.abs(sw[:, :3] - mavg).max())
        worst = max(worst, dm)
        assert dm <= 1e-4, (j["kind"], dm)
        np.testing.assert_allclose(np.linalg.norm(m, axis=1), 1.0, atol=1e-5)
    observe("serving_vs_oracle_max_dm", worst, 1e-4)


def test_invalid_geometry_fails_its_jobs(mt, ctx):
    # a geometry whose tiles cannot be created (a non-positive edge) or whose
    # tiles overlap fails its jobs with that status; the server keeps serving
    good = wl.film(8, 2, 1)
    bad_edge = wl.film(8, 2, 1)
    bad_edge.edge[3, 0] = -1e-9
    overlap = wl.film(8, 2, 1)
    overlap.centre[1] = overlap.centre[0] + np.array([0.3, 0, 0]) * overlap.edge[0]
    overlap.nbr = None
    S = mt.Server(ctx, max_batch=2, prec="f32", opts=mt.ode_opts(rtol=1e-5, atol=1e-5))
    gg, ge, go = S.add_geometry(good), S.add_geometry(bad_edge), S.add_geometry(overlap)
    je = S.submit(ge, wl.m_noisy(bad_edge.n), tol=1e-4, t_max=1e-9)
    jo = S.submit(go, wl.m_noisy(overlap.n), tol=1e-4, t_max=1e-9)
    jg = S.submit(gg, wl.m_noisy(good.n), tol=1e-4, t_max=1e-9)
    s, r, _ = S.wait(je, 60.0)
    assert s == 0 and r["status"] == mt.MT_EINVAL
    s, r, _ = S.wait(jo, 60.0)
    assert s == 0 and r["status"] == mt.MT_EOVERLAP
    s, r, _ = S.wait(jg, 60.0)
    assert s == 0 and r["status"] in (mt.MT_OK, mt.MT_ENOCONV)
    S.close()


def test_sweep_rejects_bad_schedules(mt, ctx):
    t = wl.film(8, 2, 1)
    S = mt.Server(ctx, max_batch=2, prec="f32")
    g = S.add_geometry(t)
    with pytest.raises(mt.MtError) as e:
        S.submit(g, wl.m_noisy(t.n), fields=np.array([[1.0, np.nan, 0.0]]))
    assert e.value.status == mt.MT_EINVAL
    with pytest.raises(mt.MtError) as e:
        S.submit(g, wl.m_noisy(t.n), fields=np.zeros((0, 3)))
    assert e.value.status == mt.MT_EINVAL
    S.close()
