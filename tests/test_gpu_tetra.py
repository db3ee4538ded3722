"""Tetrahedral tiles (Sec. 3) on the GPU against the oracle: the FP64
tensor of an irregular mesh, FP32 and split-BF16 fields (small and at a
full 24,000-tile mesh on sampled rows), the right-hand side with the
two-point-flux exchange, fixed Runge-Kutta steps, a box's union tensor for
uniform m, and overlap detection."""
import math

import numpy as np
import pytest

import oracle
from paper_2107_05364_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
MS, AEX = 8.0e5, 1.3e-11


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


@pytest.fixture(scope="module")
def mesh():
    verts, tets = wl.tetra_box(5, 4, 3, size=(50e-9, 40e-9, 15e-9), jitter=0.25, seed=7)
    return verts, tets


def tiles_of(mt, ctx, verts, tets, Ku=0.0):
    return mt.mt_tiles_create_tetra(ctx, verts, tets, MS, AEX, Ku, (0.0, 0.0, 1.0))


def test_tensor_fp64_matches_oracle(mt, ctx, mesh):
    verts, tets = mesh
    tiles = tiles_of(mt, ctx, verts, tets)
    T = mt.mt_demag_assemble(tiles, "f64")
    got = mt.mt_tensor_read_rows(T, 0, len(tets))
    ref = oracle.tetra_demag_tensor(verts[tets])
    assert _rel(got, ref) < 1e-12


@pytest.mark.parametrize("prec,layout,tol", [("f32", 0, 1e-6), ("split", 1, 1e-6), ("bf16", 1, 5e-3)])
def test_field_matches_oracle(mt, ctx, mesh, prec, layout, tol):
    import torch
    verts, tets = mesh
    tiles = tiles_of(mt, ctx, verts, tets)
    T = mt.mt_demag_assemble_ex(tiles, prec, layout)
    N = oracle.tetra_demag_tensor(verts[tets])
    for m in (wl.m_random(len(tets), seed=3), np.tile([[0.6, 0.48, 0.64]], (len(tets), 1))):
        m = m.astype(np.float32)
        mg = torch.tensor(m.ravel(), device="cuda")
        H = torch.full_like(mg, float("nan"))
        mt.mt_demag_field(T, mg, H)
        torch.cuda.synchronize()
        ref = oracle.demag_field_dense(N, np.full(len(tets), MS), m.astype(np.float64))
        assert _rel(H.cpu().numpy().reshape(-1, 3), ref) < tol


def test_full_size_mesh_sampled_rows(mt, ctx):
    # 20 x 20 x 10 cells x 6 = 24,000 jittered tetrahedra, FP32 tensor
    import torch
    verts, tets = wl.tetra_box(20, 20, 10, size=(200e-9, 200e-9, 50e-9), jitter=0.2, seed=9)
    n = len(tets)
    tiles = tiles_of(mt, ctx, verts, tets)
    T = mt.mt_demag_assemble(tiles, "f32")
    m = wl.m_random(n, seed=5).astype(np.float32)
    mg = torch.tensor(m.ravel(), device="cuda")
    H = torch.full_like(mg, float("nan"))
    mt.mt_demag_field(T, mg, H)
    torch.cuda.synchronize()
    rows = np.unique(np.concatenate([[0, n - 1, n // 2], np.random.default_rng(1).integers(0, n, 29)]))
    ref = oracle.tetra_field_rows(verts[tets], np.full(n, MS), m.astype(np.float64), rows)
    assert _rel(H.cpu().numpy().reshape(-1, 3)[rows], ref) < 1e-6


def test_union_box_for_uniform_m(mt, ctx):
    # the Kuhn tetrahedra of a box add up to the box: the field at every
    # centroid for uniform m is that of the whole box (cuboid closed form)
    import torch
    verts, tets = wl.tetra_box(4, 3, 2, size=(40e-9, 30e-9, 10e-9), jitter=0.0)
    tiles = tiles_of(mt, ctx, verts, tets)
    T = mt.mt_demag_assemble(tiles, "f32")
    n = len(tets)
    mu = np.array([0.6, 0.0, 0.8])
    mg = torch.tensor(np.tile(mu, n).astype(np.float32), device="cuda")
    H = torch.empty_like(mg)
    mt.mt_demag_field(T, mg, H)
    torch.cuda.synchronize()
    cen = verts[tets].mean(1)
    ref = np.array([-oracle.point_tensor(c, [20e-9, 15e-9, 5e-9], [40e-9, 30e-9, 10e-9]) @ (MS * mu) for c in cen])
    assert _rel(H.cpu().numpy().reshape(-1, 3), ref) < 1e-6


def test_rhs_and_steps_with_exchange(mt, ctx):
    # a milder jitter than the tensor tests: slivers make the two-point flux
    # stiff beyond any explicit step (see the next test)
    import torch
    verts, tets = wl.tetra_box(5, 4, 3, size=(50e-9, 40e-9, 15e-9), jitter=0.1, seed=7)
    n = len(tets)
    tiles = tiles_of(mt, ctx, verts, tets, Ku=5e4)
    T = mt.mt_demag_assemble(tiles, "f32")
    md = oracle.tetra_model(verts, tets, MS, AEX, 5e4, (0.0, 0.0, 1.0))
    Ha = np.array([1e4, -2e4, 3e3])
    m = wl.m_random(n, seed=8).astype(np.float32)
    p, keep = mt.llg_params(1, alpha=0.1, Ha=Ha)
    mg = torch.tensor(m.ravel(), device="cuda")
    dm = torch.empty_like(mg)
    mt.mt_llg_rhs(T, p, mg, dm)
    torch.cuda.synchronize()
    pr = oracle.llg_params(alpha=0.1, Ha=Ha)
    ref, _ = oracle.llg_rhs(md, m.astype(np.float64), pr)
    assert _rel(dm.cpu().numpy().reshape(-1, 3), ref) < 1e-5
    E = mt.mt_energy(T, p, mg)[0]
    eo = oracle.energy(md, m.astype(np.float64), pr)
    for k, name in enumerate(("total", "zeeman", "demag", "exchange", "anisotropy")):
        assert abs(E[k] - eo[name]) <= 1e-5 * max(abs(eo[name]), 1e-3 * abs(eo["demag"])), name
    h = 2e-14
    I = mt.Integrator(T, p, mt.ode_opts(fixed_h=h))
    m0 = wl.m_noisy(n, (1, 1, 1), 1e-2, seed=1).astype(np.float32)
    I.set_state(m0.ravel())
    I.step(20)
    st, mo, _, _ = oracle.integrate(md, m0.astype(np.float64), pr, oracle.ode_opts(fixed_h=h), 0.0, 20 * h, 1)
    assert st == oracle.OK
    assert np.abs(I.get_state()[0] - mo).max() < 2e-5


def test_sliver_stiffness_is_reported_on_both_sides(mt, ctx, mesh):
    # the 0.25-jitter mesh holds slivers whose two-point exchange coefficient
    # (~1.6e10 A/m) needs steps below ~1e-15 s: a fixed step of 2e-14 s
    # leaves the finite numbers, and both sides say so
    verts, tets = mesh
    n = len(tets)
    tiles = tiles_of(mt, ctx, verts, tets)
    T = mt.mt_demag_assemble(tiles, "f32")
    md = oracle.tetra_model(verts, tets, MS, AEX, 0.0, (0.0, 0.0, 1.0))
    p, keep = mt.llg_params(1, alpha=0.1)
    I = mt.Integrator(T, p, mt.ode_opts(fixed_h=2e-14))
    m0 = wl.m_noisy(n, (1, 1, 1), 1e-2, seed=1).astype(np.float32)
    I.set_state(m0.ravel())
    I.step(40)
    st = I.stats()[0]
    so, _, _, _ = oracle.integrate(md, m0.astype(np.float64), oracle.llg_params(alpha=0.1),
                                   oracle.ode_opts(fixed_h=2e-14), 0.0, 40 * 2e-14, 1)
    assert so == oracle.ENONFINITE
    assert st["status"] == mt.MT_ENONFINITE
    assert np.isfinite(I.get_state()).all()  # the last finite state is kept


def test_overlap_is_reported(mt, ctx):
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0.1, 0.1, 0.1], [1.1, 0.1, 0.1],
                      [0.1, 1.1, 0.1], [0.1, 0.1, 1.1]]) * 1e-8
    tets = np.array([[0, 1, 2, 3], [4, 5, 6, 7]])
    tiles = tiles_of(mt, ctx, verts, tets)
    with pytest.raises(mt.MtError) as e:
        mt.mt_demag_assemble(tiles, "f32")
    assert e.value.status == mt.MT_EOVERLAP


def test_bad_meshes_are_rejected(mt, ctx):
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]]) * 1e-8
    for tets in (np.array([[0, 1, 2, 2]]), np.array([[0, 1, 2, 9]]), np.array([[0, 1, 4, 4]])):
        with pytest.raises(mt.MtError) as e:
            tiles_of(mt, ctx, verts, tets)
        assert e.value.status == mt.MT_EINVAL
    flat = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]]) * 1e-8
    with pytest.raises(mt.MtError):
        tiles_of(mt, ctx, flat, np.array([[0, 1, 2, 3]]))
