"""Thresholded tensor (Sec. 4.3.1) on the GPU against the oracle's
thresholding: the same cut value and kept elements (the decision is taken on
FP32 values on both sides), the sparse product within the FP32 field
tolerance (1e-6) of the oracle's FP64 product with the same kept values,
close to the oracle's thresholding of its own FP64 tensor, and the integrator
running on it."""
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


@pytest.mark.parametrize("geom", ["film", "graded"])
@pytest.mark.parametrize("fraction", [0.0, 0.2, 0.4, 0.7])
def test_threshold_matches_oracle(mt, ctx, geom, fraction):
    import torch
    t = wl.film(40, 10, 1) if geom == "film" else wl.graded_film(21, 8, 3, (210e-9, 80e-9, 9e-9), seed=6)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    S, thr, kept = mt.mt_tensor_threshold(T, fraction)
    # the selection, on identical inputs (the stored FP32 values): the same
    # cut, the same kept elements.  (The FP64 far-field values of the two
    # assemblies differ by ~1e-12 relative through the corner-sum
    # cancellation, enough to move a few hundred of them across an FP32
    # rounding boundary, so the inputs are taken from the GPU tensor here.)
    N32 = mt.mt_tensor_read_rows(T, 0, t.n)
    Nt32, thr_o, kept_o = oracle.threshold_tensor(N32, fraction)
    assert np.float32(thr) == np.float32(thr_o)
    assert kept == kept_o
    rows = mt.mt_tensor_read_rows(S, 0, t.n)
    np.testing.assert_array_equal(rows, Nt32)
    assert S.info()["layout"] == mt.MT_LAYOUT_SPARSE
    # the product against the oracle's own thresholding of its FP64 tensor
    N = oracle.demag_tensor(t.centre, t.edge)
    Nt, _, kept_f64 = oracle.threshold_tensor(N, fraction)
    assert abs(kept_f64 - kept) <= 1e-3 * kept
    md32 = oracle.Model.from_tiles(t, N=Nt32.astype(np.float64))
    md = oracle.Model.from_tiles(t, N=Nt)
    # a random state, and a uniform one (long sums of one sign that cancel
    # against the self term: the case where FP32 summation order shows)
    for m in (wl.m_random(t.n, seed=9), np.tile(np.array([[0.6, 0.48, 0.64]]), (t.n, 1))):
        m = m.astype(np.float32)
        mg = torch.tensor(m.ravel(), device="cuda")
        H = torch.full_like(mg, float("nan"))
        mt.mt_demag_field(S, mg, H)
        torch.cuda.synchronize()
        Hg = H.cpu().numpy().reshape(-1, 3)
        # the sparse product itself: FP64 product of the same kept FP32 values
        assert _rel(Hg, oracle.demag_field(md32, m.astype(np.float64))) <= 1e-6
        # and the oracle's own thresholding of its FP64 tensor: the few
        # elements within one FP32 rounding of the cut may fall on the other
        # side, each worth about t relative to fields of order max|N|
        assert _rel(Hg, oracle.demag_field(md, m.astype(np.float64))) <= 1e-4


def test_integrator_on_thresholded_tensor(mt, ctx):
    t = wl.film(40, 10, 1)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    S, thr, kept = mt.mt_tensor_threshold(T, 0.4)
    N = oracle.demag_tensor(t.centre, t.edge)
    Nt, _, _ = oracle.threshold_tensor(N, 0.4)
    md = oracle.Model.from_tiles(t, N=Nt)
    m0 = wl.m_noisy(t.n, (1, 1, 1), 1e-3, seed=0).astype(np.float32)
    Ha = np.array([-24.6e-3, 4.3e-3, 0.0]) / MU0
    h = 1e-13
    p, keep = mt.llg_params(1, alpha=0.02, Ha=Ha)
    I = mt.Integrator(S, p, mt.ode_opts(fixed_h=h))
    I.set_state(m0.ravel())
    I.step(20)
    mg = I.get_state()[0]
    st, mo, _, _ = oracle.integrate(md, m0.astype(np.float64), oracle.llg_params(alpha=0.02, Ha=Ha),
                                    oracle.ode_opts(fixed_h=h), 0.0, 20 * h, 1)
    assert st == oracle.OK
    assert np.abs(mg - mo).max() <= 2e-5


def test_threshold_full_size_sampled_rows(mt, ctx):
    # the time-vs-error workload (standard-problem-4 film at 160 x 40 x 1,
    # n = 6,400) at 40 %: properties that hold at any size, on sampled rows
    import torch
    t = wl.film(160, 40, 1)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble_ex(tiles, "f32", mt.MT_LAYOUT_STREAM_FULL)  # thresholding reads every block
    _, _, nz = mt.mt_tensor_threshold(T, 0.0)
    S, thr, kept = mt.mt_tensor_threshold(T, 0.4)
    k = int(0.4 * nz)
    assert nz - kept in (k, k - 1)  # exactly k, or k - 1 when the cut splits an entry's two copies
    rows = np.unique(np.concatenate([[0, t.n - 1, 3200], np.random.default_rng(2).integers(0, t.n, 12)]))
    t32 = np.float32(thr)
    for i in rows:
        full = mt.mt_tensor_read_rows(T, int(i), int(i) + 1)[0]
        kept_row = mt.mt_tensor_read_rows(S, int(i), int(i) + 1)[0]
        a = np.abs(full.astype(np.float32))
        on = kept_row != 0
        np.testing.assert_array_equal(kept_row[on], full[on])  # kept values untouched
        assert np.all(a[on] >= t32)                            # kept: at or above the cut
        assert np.all(a[(~on) & (a > 0)] <= t32)               # dropped: at or below it
        assert np.all(a[a > t32] > 0) and np.all(on[a > t32])  # everything above the cut kept
    # the sparse field on the sampled rows: FP64 product of the kept values
    m = wl.m_random(t.n, seed=4).astype(np.float32)
    mg = torch.tensor(m.ravel(), device="cuda")
    H = torch.full_like(mg, float("nan"))
    mt.mt_demag_field(S, mg, H)
    torch.cuda.synchronize()
    Hg = H.cpu().numpy().reshape(-1, 3)[rows]
    x = (t.Ms[:, None] * m.astype(np.float64))
    ref = []
    for i in rows:
        blk = mt.mt_tensor_read_rows(S, int(i), int(i) + 1)[0]
        full = oracle.six_to_full(blk[None])[0]  # (n, 3, 3)
        ref.append(-np.einsum("jab,jb->a", full, x))
    assert _rel(Hg, np.array(ref)) < 1e-6


def test_single_layer_sparse_stores_four_planes(mt, ctx):
    # a thresholded single-layer tensor keeps the source's 4 value planes
    # (20 bytes per kept block) and gives the 6-plane sparse tensor's field
    import torch
    t = wl.film(40, 10, 1)
    tiles = mt.mt_tiles_create(ctx, t)
    S4, thr4, kept4 = mt.mt_tensor_threshold(mt.mt_demag_assemble(tiles, "f32"), 0.4)
    S6, thr6, kept6 = mt.mt_tensor_threshold(mt.mt_demag_assemble_ex(tiles, "f32", mt.MT_LAYOUT_STREAM6), 0.4)
    assert S4.info()["planes"] == 4 and S6.info()["planes"] == 6
    assert np.float32(thr4) == np.float32(thr6) and kept4 == kept6
    assert S4.info()["bytes"] < 0.8 * S6.info()["bytes"]
    np.testing.assert_array_equal(mt.mt_tensor_read_rows(S4, 0, t.n), mt.mt_tensor_read_rows(S6, 0, t.n))
    m = wl.m_random(t.n, seed=5).astype(np.float32)
    mg = torch.tensor(m.ravel(), device="cuda")
    H4, H6 = torch.full_like(mg, float("nan")), torch.full_like(mg, float("nan"))
    mt.mt_demag_field(S4, mg, H4)
    mt.mt_demag_field(S6, mg, H6)
    torch.cuda.synchronize()
    assert torch.equal(H4, H6)


@pytest.mark.parametrize("nx,ny,fraction,warps", [(64, 32, 0.3, 2), (80, 40, 0.0, 4)])
def test_rows_split_among_warps(mt, ctx, nx, ny, fraction, warps):
    # rows of ~14 and 25 steps of 128 blocks: the product gives each row to 2
    # and 4 warps, each starting from the run that holds its first block
    import torch
    t = wl.film(nx, ny, 1)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble_ex(tiles, "f32", mt.MT_LAYOUT_STREAM_FULL)
    S, thr, kept = mt.mt_tensor_threshold(T, fraction)
    assert S.info()["row_warps"] == warps and T.info()["row_warps"] == 0
    N = oracle.demag_tensor(t.centre, t.edge)
    if fraction == 0.0:
        # nothing dropped: the oracle's tensor rounded to FP32 is the stored one
        # to an ulp here and there
        md32 = oracle.Model.from_tiles(t, N=N.astype(np.float32).astype(np.float64))
    else:
        # the selection on the stored FP32 values (see test_threshold_matches_oracle)
        N32 = mt.mt_tensor_read_rows(T, 0, t.n)
        Nt32, thr_o, kept_o = oracle.threshold_tensor(N32, fraction)
        assert np.float32(thr) == np.float32(thr_o) and kept == kept_o
        md32 = oracle.Model.from_tiles(t, N=Nt32.astype(np.float64))
    Nt, _, _ = oracle.threshold_tensor(N, fraction)
    md = oracle.Model.from_tiles(t, N=Nt)
    ms = [wl.m_random(t.n, seed=11), np.tile(np.array([[0.6, 0.48, 0.64]]), (t.n, 1))]
    mg = torch.tensor(np.concatenate([m.astype(np.float32).ravel() for m in ms]), device="cuda")
    H = torch.full_like(mg, float("nan"))
    mt.mt_demag_field(S, mg, H, B=2)
    torch.cuda.synchronize()
    for b, m in enumerate(ms):
        Hg = H[b * 3 * t.n:(b + 1) * 3 * t.n].cpu().numpy().reshape(-1, 3)
        m64 = m.astype(np.float32).astype(np.float64)
        assert _rel(Hg, oracle.demag_field(md32, m64)) <= 1e-6
        assert _rel(Hg, oracle.demag_field(md, m64)) <= 1e-4
        # a simulation's field does not depend on the batch it is computed in
        H1 = torch.full((3 * t.n,), float("nan"), device="cuda")
        mt.mt_demag_field(S, mg[b * 3 * t.n:(b + 1) * 3 * t.n].contiguous(), H1)
        torch.cuda.synchronize()
        assert torch.equal(H1, H[b * 3 * t.n:(b + 1) * 3 * t.n])
