"""Standard problem 3 energy crossover (Sec. 4.2) on the GPU against the
oracle: a 6^3-tile cube, flower and vortex seeds (the vortex core along x,
across the easy axis z) relaxed at six sizes in one batch (the sizes enter as exchange factors on one tensor), against the
oracle's relaxations of really scaled cubes.  Energy densities within 1e-5
of the oracle's (relative to K_m), the crossing within 5e-3 l_ex."""
import math

import numpy as np
import pytest

import oracle
from paper_2107_05364_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
KM = 0.5 * 4e-7 * math.pi * 8e5 ** 2


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


LAM = np.array([7.0, 7.5, 8.0, 8.5, 9.0, 9.5])
OPTS = dict(rtol=1e-6, atol=1e-6, h0=1e-14, hmax=1e-10)


@pytest.fixture(scope="module")
def reference():
    t = wl.cube(6, 1.0)
    p = oracle.llg_params(alpha=4000.0, form=1, precess=0)
    eA, eB, lc, _ = oracle.crossover(t.centre, t.edge, t.Ms, t.Aex, t.Ku, t.axis, t.nbr, LAM, wl.m_flower(t),
                                     wl.m_vortex(t, axis=0), p, oracle.ode_opts(**OPTS), 1e-4, 20e-9)
    return t, eA, eB, lc


@pytest.mark.parametrize("prec,layout", [("f32", 0), ("split", 1)])
def test_crossover_matches_oracle(mt, ctx, reference, prec, layout):
    t, eA, eB, lc = reference
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble_ex(tiles, prec, layout)
    K = len(LAM)
    p, keep = mt.llg_params(2 * K, alpha=4000.0, form=mt.MT_FORM_LL, precess=0)
    I = mt.Integrator(T, p, mt.ode_opts(**OPTS), B=2 * K)
    gA, gB, glc, states, st = I.crossover(LAM, wl.m_flower(t), wl.m_vortex(t, axis=0), 1e-4, 20e-9,
                                         states=True)
    print("%s: crossing %.4f (oracle %.4f); max energy difference %.2e K_m" %
          (prec, glc, lc, max(np.abs(gA - eA).max(), np.abs(gB - eB).max()) / KM))
    assert np.abs(gA - eA).max() < 1e-5 * KM
    assert np.abs(gB - eB).max() < 1e-5 * KM
    assert abs(glc - lc) < 5e-3
    assert np.abs(np.linalg.norm(states, axis=2) - 1).max() < 1e-5
