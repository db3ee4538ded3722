"""GPU parity of the batched tensor-core product (dense BF16 / split BF16
tensor, tcgen05) and of the integrator running on it, against the FP64 oracle
through the C ABI.

Tolerances (relative L2): BF16 field 5e-3; split BF16 field 1e-6; the far
field carries the storage error, the touching blocks are FP64.
"""
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


TOL = {"bf16": 5e-3, "split": 1e-6}


@pytest.mark.parametrize("prec", ["bf16", "split"])
def test_dense_tensor_entries(mt, ctx, prec):
    t = wl.graded_film(23, 7, 3, (230e-9, 70e-9, 9e-9), seed=4)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble_ex(tiles, prec, mt.MT_LAYOUT_DENSE)
    assert T.info()["layout"] == mt.MT_LAYOUT_DENSE and T.info()["near_blocks"] > 0
    N = mt.mt_tensor_read_rows(T, 0, t.n)
    ref = oracle.demag_tensor(t.centre, t.edge)
    # per-entry storage error: 2^-9 (BF16) / 2^-17 (hi + lo)
    bound = 2.0 ** -8 if prec == "bf16" else 2.0 ** -16
    assert np.abs(N - ref).max() <= bound * np.abs(ref).max()
    assert _rel(N, ref) <= (3e-3 if prec == "bf16" else 2e-5)


@pytest.mark.parametrize("prec", ["bf16", "split"])
@pytest.mark.parametrize("B", [1, 3, 17, 64, 100, 128])  # padded 16, 16, 32, 64, 128, 128
def test_dense_field_parity(mt, ctx, prec, B):
    import torch
    t = wl.graded_film(29, 9, 2, (290e-9, 90e-9, 6e-9), seed=6)   # 3n = 1566: ragged 128-row tiles
    t.Ms[:] = np.linspace(5e5, 1.1e6, t.n)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble_ex(tiles, prec, mt.MT_LAYOUT_DENSE)
    md = oracle.Model.from_tiles(t)
    m = np.stack([wl.m_random(t.n, seed=100 + b) for b in range(B)]).astype(np.float32)
    mg = torch.tensor(m.ravel(), device="cuda")
    H = torch.full_like(mg, float("nan"))
    mt.mt_demag_field(T, mg, H, B=B)
    torch.cuda.synchronize()
    Hg = H.cpu().numpy().reshape(B, t.n, 3)
    assert np.isfinite(Hg).all()
    for b in sorted({0, B // 2, B - 1}):
        ref = oracle.demag_field(md, m[b].astype(np.float64))
        assert _rel(Hg[b], ref) <= TOL[prec], (prec, B, b, _rel(Hg[b], ref))


def test_dense_field_config4_shape_sampled(mt, ctx):
    # the batched workload: film 200 x 50 x 2 (n = 20,000), B = 64, sampled rows
    import torch
    t = wl.film(200, 50, 2)
    tiles = mt.mt_tiles_create(ctx, t)
    B = 64
    rows = np.unique(np.concatenate([[0, 1, t.n - 1, 9999, 10000], np.random.default_rng(2).integers(0, t.n, 40)]))
    m = np.stack([wl.m_noisy(t.n, (1, 1, 1), 0.3, seed=b) for b in range(B)]).astype(np.float32)
    mg = torch.tensor(m.ravel(), device="cuda")
    for prec in ("bf16", "split"):
        T = mt.mt_demag_assemble_ex(tiles, prec, mt.MT_LAYOUT_DENSE)
        H = torch.full_like(mg, float("nan"))
        mt.mt_demag_field(T, mg, H, B=B)
        torch.cuda.synchronize()
        Hg = H.cpu().numpy().reshape(B, t.n, 3)
        for b in (0, 37, 63):
            ref = oracle.demag_field_rows(t.centre, t.edge, t.Ms, m[b].astype(np.float64), rows)
            assert _rel(Hg[b][rows], ref) <= TOL[prec], (prec, b)
        T.close()


def test_batched_integrator_on_tensor_cores(mt, ctx):
    # B = 8 simulations, split BF16 dense tensor on tcgen05, against the FP32
    # streaming integrator run per simulation: <m>(t) over 20 ps
    t = wl.film(40, 10, 1)
    tiles = mt.mt_tiles_create(ctx, t)
    Td = mt.mt_demag_assemble_ex(tiles, "split", mt.MT_LAYOUT_DENSE)
    Ts = mt.mt_demag_assemble(tiles, "f32")
    B = 8
    Ha, _ = wl.sweep_fields(B, 50.0, seed=0)
    alphas = wl.sweep_alphas(B)
    m0 = np.stack([wl.m_noisy(t.n, (1, 1, 1), 1e-3, seed=b) for b in range(B)]).astype(np.float32)
    opts = mt.ode_opts(rtol=1e-6, atol=1e-6, h0=1e-14, hmax=1e-11)
    p, keep = mt.llg_params(B, alpha=alphas, Ha=Ha)
    I = mt.Integrator(Td, p, opts, B=B)
    I.set_state(m0.ravel())
    _, mavg, st = I.run(2e-11, 4)
    assert all(s["status"] == 0 for s in st)
    for b in (0, 3, 7):
        p1, k1 = mt.llg_params(1, alpha=alphas[b], Ha=Ha[b])
        I1 = mt.Integrator(Ts, p1, opts, B=1)
        I1.set_state(m0[b].ravel())
        _, mavg1, _ = I1.run(2e-11, 4)
        assert np.abs(mavg1[:, 0] - mavg[:, b]).max() <= 1e-4, b


def test_dense_rejects_unsupported(mt, ctx):
    t = wl.film(4, 2, 1)
    tiles = mt.mt_tiles_create(ctx, t)
    with pytest.raises(mt.MtError) as e:
        mt.mt_demag_assemble_ex(tiles, "f32", mt.MT_LAYOUT_DENSE)
    assert e.value.status == mt.MT_EINVAL
