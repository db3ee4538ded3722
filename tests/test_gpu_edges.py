"""Edge cases of every storage path against the oracle: one and two tiles,
a ragged tile count (129: one tile past a 128-wide chunk), batches of 1, 5
and 300 simulations, and the thresholded layout with several simulations
(field and integrator)."""
import numpy as np
import pytest

import oracle
from paper_2107_05364_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "f32": 1e-6, "bf16": 5e-3, "split": 1e-6}


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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def geom(n):
    if n == 1:
        return wl.film(1, 1, 1, size=(5e-9, 4e-9, 3e-9))
    if n == 2:
        return wl.film(2, 1, 1, size=(10e-9, 4e-9, 3e-9))
    return wl.graded_film(43, 3, 1, (215e-9, 15e-9, 3e-9), seed=11)  # 129 tiles, no lattice


def field(mt, T, m, B, f64=False):
    import torch
    if f64:
        mg = torch.tensor(m.astype(np.float64).ravel(), device="cuda")
        H = torch.full_like(mg, float("nan"))
        mt.mt_demag_field_f64(T, mg, H, B=B)
    else:
        mg = torch.tensor(m.astype(np.float32).ravel(), device="cuda")
        H = torch.full_like(mg, float("nan"))
        mt.mt_demag_field(T, mg, H, B=B)
    torch.cuda.synchronize()
    return H.cpu().numpy().reshape(B, -1, 3)


@pytest.mark.parametrize("n", [1, 2, 129])
@pytest.mark.parametrize("prec,layout", [("f64", 0), ("f32", 0), ("bf16", 0), ("split", 0), ("bf16", 1),
                                         ("split", 1)])
@pytest.mark.parametrize("B", [1, 5])
def test_field_small_and_ragged(mt, ctx, n, prec, layout, B):
    t = geom(n)
    assert t.n == n
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble_ex(tiles, prec, layout)
    m = np.stack([wl.m_random(n, seed=40 + b) for b in range(B)])
    Hg = field(mt, T, m, B, f64=(prec == "f64"))
    assert np.isfinite(Hg).all()
    md = oracle.Model.from_tiles(t)
    for b in range(B):
        ref = oracle.demag_field(md, m[b].astype(np.float64) if prec == "f64" else
                                 m[b].astype(np.float32).astype(np.float64))
        assert _rel(Hg[b], ref) <= TOL[prec], (n, prec, layout, B, b, _rel(Hg[b], ref))


def test_stream_field_wide_batch(mt, ctx):
    # 300 simulations through the streaming FP32 product
    t = geom(129)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    B = 300
    m = np.stack([wl.m_random(t.n, seed=500 + b) for b in range(B)])
    Hg = field(mt, T, m, B)
    md = oracle.Model.from_tiles(t)
    for b in (0, 1, 150, 298, 299):
        ref = oracle.demag_field(md, m[b].astype(np.float32).astype(np.float64))
        assert _rel(Hg[b], ref) <= 1e-6, b


def test_sparse_field_and_steps_with_several_simulations(mt, ctx):
    t = geom(129)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    S, thr, kept = mt.mt_tensor_threshold(T, 0.3)
    Nt = mt.mt_tensor_read_rows(S, 0, t.n)
    md = oracle.Model.from_tiles(t, N=Nt)
    B = 5
    m = np.stack([wl.m_random(t.n, seed=60 + b) for b in range(B)]).astype(np.float32)
    Hg = field(mt, S, m, B)
    for b in range(B):
        assert _rel(Hg[b], oracle.demag_field(md, m[b].astype(np.float64))) <= 1e-6, b
    # fixed Runge-Kutta steps of 3 simulations with different damping
    h = 1e-13
    alphas = [0.02, 0.1, 0.5]
    p, keep = mt.llg_params(3, alpha=alphas)
    I = mt.Integrator(S, p, mt.ode_opts(fixed_h=h), B=3)
    m0 = np.stack([wl.m_noisy(t.n, (1, 1, 1), 1e-2, seed=70 + b) for b in range(3)]).astype(np.float32)
    I.set_state(m0.ravel())
    I.step(15)
    got = I.get_state()
    for b in range(3):
        st, mo, _, _ = oracle.integrate(md, m0[b].astype(np.float64), oracle.llg_params(alpha=alphas[b]),
                                        oracle.ode_opts(fixed_h=h), 0.0, 15 * h, 1)
        assert st == oracle.OK
        assert np.abs(got[b] - mo).max() < 2e-5, b
