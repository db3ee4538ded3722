"""Half storage of the tensor of a tile set of one shape (Sec. 3.2: the
tensor is symmetric), through the C ABI.

For cuboids of equal edges the point tensor of tile j at the centre of tile
i is a function of c_i - c_j that is even in it, so N_ij = N_ji.  An FP32
streaming tensor of such tiles stores only the upper triangle of column
chunks (by default from 4,096 tiles on; at any size with
MT_LAYOUT_STREAM_HALF, used here to keep the oracle's tensors small); the
product applies each off-diagonal chunk to its rows and, transposed, to its
columns.  Checked here against the FP64
oracle (fields at the FP32 tolerance 1e-6, relative L2; stored entries at
FP32 rounding), against the same tensor stored in full, for batches that
exercise every group width of the product (1, 2, 3, 5 simulations), on a
single-layer film (4 entry planes) and a prism (6 planes) whose tile counts
leave ragged panels and chunks; and in the integrator (fixed steps).
"""
import numpy as np
import pytest

import oracle
from _observe import observe
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


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


GEOMS = {
    # n = 2,800: 175 panels of 16 rows, 22 chunks of 128 columns (the last ragged)
    "film70x40": lambda: wl.film(70, 40, 1, size=(350e-9, 200e-9, 3e-9)),
    # n = 2,520: 157.5 panels (ragged), 6 entry planes
    "prism15x14x12": lambda: wl.grid_tiles(np.linspace(0, 75e-9, 16), np.linspace(0, 70e-9, 15),
                                           np.linspace(0, 60e-9, 13), 8e5, 1.3e-11, 0.0),
}


@pytest.fixture(scope="module", params=list(GEOMS))
def case(mt, ctx, request):
    t = GEOMS[request.param]()
    tiles = mt.mt_tiles_create(ctx, t)
    Th = mt.mt_demag_assemble_ex(tiles, "f32", mt.MT_LAYOUT_STREAM_HALF)
    Tf = mt.mt_demag_assemble_ex(tiles, "f32", mt.MT_LAYOUT_STREAM_FULL)
    return request.param, t, tiles, Th, Tf, oracle.Model.from_tiles(t)


def test_half_storage_is_chosen_and_smaller(mt, case):
    name, t, tiles, Th, Tf, md = case
    ih, ifu = Th.info(), Tf.info()
    assert ih["half"] == 1 and ifu["half"] == 0
    # stored half, zz is left to the trace: a single-layer film keeps xx, xy,
    # yy, the prism xx, xy, xz, yy, yz
    film = name.startswith("film")
    assert ifu["planes"] == (4 if film else 6) and ih["planes"] == (3 if film else 5)
    # the upper triangle of chunks: a bit more than half of the full tensor,
    # times 3/4 (film) or 5/6 (prism) for the planes
    lo, hi = (0.375, 0.42) if film else (0.416, 0.467)
    assert lo < ih["bytes"] / ifu["bytes"] < hi


def test_half_stored_rows_are_the_tensor(mt, case):
    # rows read from the half storage (lower blocks taken from their upper
    # partners; zz = delta_ij - xx - yy) against the oracle's FP64 blocks, at
    # FP32 rounding
    name, t, tiles, Th, Tf, md = case
    rows = [0, 15, 16, 127, 128, t.n // 2, t.n - 1]
    for i in rows:
        h = mt.mt_tensor_read_rows(Th, i, i + 1)[0]
        ref = md.N[i]
        assert np.abs(h - ref).max() <= 2e-7 * np.abs(ref).max(), i
        f = mt.mt_tensor_read_rows(Tf, i, i + 1)[0]
        assert np.abs(h - f).max() <= 2e-7 * np.abs(ref).max(), i


@pytest.mark.parametrize("B", [1, 2, 3, 5])
def test_half_field_matches_oracle_and_full(mt, case, B):
    import torch
    name, t, tiles, Th, Tf, md = case
    m = np.stack([wl.m_random(t.n, seed=60 + b) for b in range(B)]).astype(np.float32)
    mg = torch.tensor(m.ravel(), device="cuda")
    Hh = torch.full_like(mg, float("nan"))
    Hf = torch.full_like(mg, float("nan"))
    mt.mt_demag_field(Th, mg, Hh, B=B)
    mt.mt_demag_field(Tf, mg, Hf, B=B)
    torch.cuda.synchronize()
    hh = Hh.cpu().numpy().reshape(B, t.n, 3)
    hf = Hf.cpu().numpy().reshape(B, t.n, 3)
    assert np.isfinite(hh).all()
    for b in range(B):
        ref = oracle.demag_field(md, m[b].astype(np.float64))
        assert _rel(hh[b], ref) <= 1e-6, (name, B, b, _rel(hh[b], ref))
        assert _rel(hh[b], hf[b]) <= 1e-6, (name, B, b)
    # deterministic: the same bits on a second call
    H2 = torch.full_like(mg, float("nan"))
    mt.mt_demag_field(Th, mg, H2, B=B)
    torch.cuda.synchronize()
    assert torch.equal(Hh, H2)


def test_half_integrator_steps_match_oracle(mt, case):
    name, t, tiles, Th, Tf, md = case
    h = 1e-13
    m0 = wl.m_noisy(t.n, (1, 1, 1), 1e-2, seed=3).astype(np.float32)
    p, keep = mt.llg_params(1, alpha=0.05, Ha=(1e4, -2e4, 5e3))
    out = {}
    for key, T in (("half", Th), ("full", Tf)):
        I = mt.Integrator(T, p, mt.ode_opts(fixed_h=h))
        assert I.path() == mt.MT_PATH_GRAPH
        I.set_state(m0.ravel())
        I.step(8)
        out[key] = I.get_state()[0].copy()
        I.close()
    so, mo, _, _ = oracle.integrate(md, m0.astype(np.float64), oracle.llg_params(alpha=0.05, Ha=(1e4, -2e4, 5e3)),
                                    oracle.ode_opts(fixed_h=h), 0.0, 8 * h, 1)
    assert so == oracle.OK
    assert np.abs(out["half"] - mo).max() <= 3e-6
    assert np.abs(out["half"] - out["full"]).max() <= 3e-6


def test_half_relax_of_two_simulations_with_active_masks(mt, case):
    # two simulations relaxed together at different damping: the faster one
    # stops first and leaves the slot inactive while the other runs on (the
    # product then skips the finished simulation's field).  Relaxed to a
    # torque of 1e-5 (rtol = atol = 1e-7 keeps the integrator's torque floor
    # below that), the states of the half and the full storage -- the same
    # sums in another rounding order, so other stopping points -- agree to
    # 1e-4 (at a torque of 1e-4 they differed by 1.1e-4)
    name, t, tiles, Th, Tf, md = case
    m0 = np.stack([wl.m_noisy(t.n, (1, 0.2, 0), 0.2, seed=11), wl.m_noisy(t.n, (0, 1, 0.1), 0.2, seed=12)])
    # fields of 0.1 and 0.075 T: relaxation times (1 + a^2) / (a gamma H) of
    # 0.1 and 0.4 ns, so both reach the torque well inside the 10 ns cap
    p, keep = mt.llg_params(2, alpha=np.array([0.8, 0.3]), Ha=np.array([[8e4, 0, 0], [0, -6e4, 0]]))
    out = {}
    for key, T in (("half", Th), ("full", Tf)):
        I = mt.Integrator(T, p, mt.ode_opts(rtol=1e-7, atol=1e-7), B=2)
        I.set_state(m0.astype(np.float32).ravel())
        st, stats = I.relax(1e-5, 1e-8, check=False)
        assert st == mt.MT_OK, (key, stats)
        out[key] = (I.get_state().reshape(2, t.n, 3).copy(), [x["t"] for x in stats], [x["tau"] for x in stats])
        I.close()
    (mh, th, tauh), (mf, tf, tauf) = out["half"], out["full"]
    assert max(tauh) < 1e-5 and max(tauf) < 1e-5
    assert th[0] != th[1]  # the two simulations stopped at different times
    observe("half_vs_full_relaxed_two_sims_" + name, float(np.abs(mh - mf).max()), 1e-4)
    assert np.abs(mh - mf).max() <= 1e-4
    np.testing.assert_allclose(np.linalg.norm(mh, axis=2), 1.0, atol=1e-5)


def test_half_storage_limits(mt, ctx, case):
    import torch
    name, t, tiles, Th, Tf, md = case
    # thresholding and the allocation-free product need every block
    with pytest.raises(mt.MtError) as e:
        mt.mt_tensor_threshold(Th, 0.3)
    assert e.value.status == mt.MT_EINVAL
    mg = torch.zeros(3 * t.n, device="cuda")
    with pytest.raises(mt.MtError) as e:
        mt.mt_demag_field_noalloc(Th, mg, torch.zeros_like(mg))
    assert e.value.status == mt.MT_EINVAL
    # tiles of different shapes keep every block; the explicit half layout
    # refuses them and other precisions
    g = mt.mt_tiles_create(ctx, wl.graded_film(60, 40, 1, (300e-9, 200e-9, 3e-9), seed=8))  # n = 2,400
    assert mt.mt_demag_assemble(g, "f32").info()["half"] == 0
    for tl, prec in ((g, "f32"), (tiles, "split"), (tiles, "bf16"), (tiles, "f64")):
        with pytest.raises(mt.MtError) as e:
            mt.mt_demag_assemble_ex(tl, prec, mt.MT_LAYOUT_STREAM_HALF)
        assert e.value.status == mt.MT_EINVAL
    # the default layout: full storage up to 4,096 tiles of one shape, half above
    assert mt.mt_demag_assemble(tiles, "f32").info()["half"] == 0
    big = mt.mt_tiles_create(ctx, wl.film(80, 52, 1, size=(400e-9, 260e-9, 3e-9)))  # n = 4,160
    assert mt.mt_demag_assemble(big, "f32").info()["half"] == 1
    assert mt.mt_demag_assemble_ex(big, "f32", mt.MT_LAYOUT_STREAM_FULL).info()["half"] == 0


@pytest.mark.parametrize("nx,ny", [(1, 1), (17, 1), (16, 8), (43, 3), (30, 10)])
def test_half_edge_shapes_match_oracle(mt, ctx, nx, ny):
    # forced half storage on tile counts at the layout's edges: one tile,
    # one ragged chunk (17), exactly one super-row (128), one tile into the
    # second super-row (129) and a ragged 300; fields at the FP32 tolerance
    import torch
    t = wl.film(nx, ny, 1, size=(5e-9 * nx, 4e-9 * ny, 3e-9))
    tiles = mt.mt_tiles_create(ctx, t)
    Th = mt.mt_demag_assemble_ex(tiles, "f32", mt.MT_LAYOUT_STREAM_HALF)
    assert Th.info()["half"] == 1
    md = oracle.Model.from_tiles(t)
    for B in (1, 2):
        m = np.stack([wl.m_random(t.n, seed=70 + b) for b in range(B)]).astype(np.float32)
        mg = torch.tensor(m.ravel(), device="cuda")
        H = torch.full_like(mg, float("nan"))
        mt.mt_demag_field(Th, mg, H, B=B)
        torch.cuda.synchronize()
        h = H.cpu().numpy().reshape(B, t.n, 3)
        for b in range(B):
            ref = oracle.demag_field(md, m[b].astype(np.float64))
            assert _rel(h[b], ref) <= 1e-6, (t.n, B, b, _rel(h[b], ref))


def test_default_half_above_the_threshold(mt, ctx):
    # 4,160 tiles of one shape: stored half by default; the field equals the
    # full storage's and the oracle's matrix-free rows on sampled rows
    import torch
    t = wl.film(80, 52, 1, size=(400e-9, 260e-9, 3e-9))
    tiles = mt.mt_tiles_create(ctx, t)
    Th = mt.mt_demag_assemble(tiles, "f32")
    Tf = mt.mt_demag_assemble_ex(tiles, "f32", mt.MT_LAYOUT_STREAM_FULL)
    assert Th.info()["half"] == 1 and Tf.info()["half"] == 0
    for B in (1, 2, 3):
        m = np.stack([wl.m_random(t.n, seed=80 + b) for b in range(B)]).astype(np.float32)
        mg = torch.tensor(m.ravel(), device="cuda")
        Hh, Hf = torch.empty_like(mg), torch.empty_like(mg)
        mt.mt_demag_field(Th, mg, Hh, B=B)
        mt.mt_demag_field(Tf, mg, Hf, B=B)
        torch.cuda.synchronize()
        hh = Hh.cpu().numpy().reshape(B, t.n, 3)
        hf = Hf.cpu().numpy().reshape(B, t.n, 3)
        assert _rel(hh, hf) <= 1e-6, B
    rows = np.unique(np.concatenate([[0, 127, 128, 4095, t.n - 1],
                                     np.random.default_rng(5).integers(0, t.n, 40)]))
    ref = oracle.demag_field_rows(t.centre, t.edge, t.Ms, m[0].astype(np.float64), rows)
    assert _rel(hh[0][rows], ref) <= 1e-6
