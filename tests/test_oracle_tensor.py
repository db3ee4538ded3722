"""Pins for the oracle's cuboid demagnetization tensor and demag field.

The paper (Sec. 3) evaluates the field of each uniformly magnetised cuboid
tile at the centre of every other tile from a closed-form tensor that it does
not print.  These tests pin the oracle's closed form against facts that do
not depend on it: textbook self terms, Laplace's equation, the dipole limit,
exact superposition of tiles into a larger prism, arbitrary-precision
evaluation, and an independent surface-charge quadrature of the field.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

import oracle
from paper_2107_05364_gb300 import workloads as wl


def test_cube_self_term_is_one_third():
    # uniformly magnetised cube, field at its centre: N = I/3 (textbook)
    for h in (1.0, 2.5e-9, 7.0):
        N = oracle.point_tensor([0.3, -0.2, 0.1], [0.3, -0.2, 0.1], [h, h, h])
        np.testing.assert_allclose(N, np.eye(3) / 3.0, atol=1e-15)


def test_cuboid_self_term_closed_form_and_unit_trace():
    # at the centre of a box with half-edges a, b, c every corner contributes
    # equally: N_xx = (2/pi) atan(b c / (a sqrt(a^2+b^2+c^2))), trace = 1
    rng = np.random.default_rng(5)
    for _ in range(20):
        e = rng.uniform(0.1, 5.0, 3)
        a, b, c = e / 2
        R = math.sqrt(a * a + b * b + c * c)
        N = oracle.point_tensor([0, 0, 0], [0, 0, 0], e)
        exp = np.diag([2 / math.pi * math.atan(b * c / (a * R)),
                       2 / math.pi * math.atan(a * c / (b * R)),
                       2 / math.pi * math.atan(a * b / (c * R))])
        np.testing.assert_allclose(N, exp, atol=1e-15)
        assert abs(np.trace(N) - 1.0) < 1e-14


def test_trace_zero_outside_and_symmetric():
    # Laplace: the potential of the box is harmonic outside it -> trace N = 0
    rng = np.random.default_rng(6)
    for _ in range(50):
        e = rng.uniform(0.5, 2.0, 3)
        r = rng.uniform(-6, 6, 3)
        if np.all(np.abs(r) < e / 2 + 1e-3):
            continue
        N = oracle.point_tensor(r, [0, 0, 0], e)
        scale = np.abs(N).max()
        assert abs(np.trace(N)) < 1e-12 * max(scale, 1e-3)
        np.testing.assert_array_equal(N, N.T)


def test_reciprocity_equal_tiles():
    # N_ij = N_ji for two equal tiles (point symmetry of the box)
    t = wl.film(8, 4, 2, size=(80e-9, 40e-9, 6e-9))
    N = oracle.demag_tensor(t.centre, t.edge)
    np.testing.assert_allclose(N, N.transpose(1, 0, 2), rtol=1e-11, atol=5e-15)


def test_dipole_limit():
    # far from the tile: N -> -(V / 4 pi r^3) (3 rr - I); error O((h/r)^2)
    e = np.array([1.0, 2.0, 0.7])
    V = np.prod(e)
    d = np.array([0.6, -0.3, 0.74])
    d /= np.linalg.norm(d)
    errs = []
    for dist in (20.0, 40.0, 80.0, 160.0):
        r = dist * d
        N = oracle.point_tensor(r, [0, 0, 0], e)
        D = -(V / (4 * math.pi * dist ** 3)) * (3 * np.outer(d, d) - np.eye(3))
        errs.append(np.abs(N - D).max() / np.abs(D).max())
    errs = np.array(errs)
    assert errs[0] < 5e-3
    # second-order convergence towards the dipole (ratio ~4 per doubling)
    ratios = errs[:-1] / errs[1:]
    assert np.all(ratios > 3.0) and np.all(ratios < 5.0), ratios


def _mp_point_tensor(r, c, e, dps=60):
    """The closed form evaluated in arbitrary precision, written straight from
    N = -(1/4pi) grad grad Phi without the stable rewrites."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = dps
    r = [mp.mpf(float(x)) for x in r]
    lo = [mp.mpf(float(c[a])) - mp.mpf(float(e[a])) / 2 for a in range(3)]
    hi = [mp.mpf(float(c[a])) + mp.mpf(float(e[a])) / 2 for a in range(3)]
    faces = [lo, hi]
    S = {k: mp.mpf(0) for k in ("xx", "yy", "zz", "xy", "xz", "yz")}
    for i in range(2):
        for j in range(2):
            for k in range(2):
                s = (-1) ** (i + j + k + 3)  # (-1)^(i+j+k) with faces numbered 1, 2
                U = r[0] - faces[i][0]
                V = r[1] - faces[j][1]
                W = r[2] - faces[k][2]
                R = mp.sqrt(U * U + V * V + W * W)
                S["xx"] += s * (mp.atan(V * W / (U * R)) if U != 0 else 0)
                S["yy"] += s * (mp.atan(U * W / (V * R)) if V != 0 else 0)
                S["zz"] += s * (mp.atan(U * V / (W * R)) if W != 0 else 0)
                S["xy"] += s * mp.log(W + R)
                S["xz"] += s * mp.log(V + R)
                S["yz"] += s * mp.log(U + R)
    c4 = 1 / (4 * mp.pi)
    return np.array([[float(-c4 * S["xx"]), float(c4 * S["xy"]), float(c4 * S["xz"])],
                     [float(c4 * S["xy"]), float(-c4 * S["yy"]), float(c4 * S["yz"])],
                     [float(c4 * S["xz"]), float(c4 * S["yz"]), float(-c4 * S["zz"])]])


def test_far_field_against_arbitrary_precision():
    # points far from the tile in every direction, including far below it
    # (where ln(W+R) cancels): the FP64 oracle keeps relative accuracy
    # ~ eps (r/h)^3 of the 60-digit value
    e = np.array([2.5e-9, 2.5e-9, 3e-9])
    rng = np.random.default_rng(7)
    for dist in (5e-9, 40e-9, 200e-9):
        for _ in range(6):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            r = dist * d
            N = oracle.point_tensor(r, [0, 0, 0], e)
            M = _mp_point_tensor(r, [0, 0, 0], e)
            rel = np.abs(N - M).max() / np.abs(M).max()
            bound = 2e-16 * 50 * (dist / 2.5e-9) ** 3 + 1e-15
            assert rel < bound, (dist, rel, bound)
    # straight below/above/beside the tile on the axes (U = V = 0 lines)
    for r in ([0, 0, -60e-9], [0, 0, 60e-9], [0, -60e-9, 0], [-60e-9, 0, 0]):
        N = oracle.point_tensor(r, [0, 0, 0], e)
        M = _mp_point_tensor(r, [0, 0, 0], e)
        assert np.abs(N - M).max() / np.abs(M).max() < 1e-9


def _quadrature_tensor(r, c, e, nq=48):
    """N from the surface charge of M = e_k: H = (1/4pi) sum over faces of
    sigma (r - r') / |r - r'|^3 dS', sigma = M.n; N[:, k] = -H.
    Gauss-Legendre on each face, split into 4x4 panels."""
    g, w = leggauss(nq)
    r = np.asarray(r, float)
    c = np.asarray(c, float)
    a = np.asarray(e, float) / 2
    N = np.zeros((3, 3))
    for k in range(3):
        H = np.zeros(3)
        o = [q for q in range(3) if q != k]
        for sgn in (-1.0, 1.0):
            for pu in range(4):
                for pv in range(4):
                    u0 = c[o[0]] - a[o[0]] + pu * a[o[0]] / 2
                    v0 = c[o[1]] - a[o[1]] + pv * a[o[1]] / 2
                    hu, hv = a[o[0]] / 4, a[o[1]] / 4
                    U = u0 + hu + hu * g
                    V = v0 + hv + hv * g
                    UU, VV = np.meshgrid(U, V, indexing="ij")
                    P = np.zeros(UU.shape + (3,))
                    P[..., k] = c[k] + sgn * a[k]
                    P[..., o[0]] = UU
                    P[..., o[1]] = VV
                    d = r - P
                    dn = np.linalg.norm(d, axis=-1)
                    W = np.outer(w, w) * hu * hv
                    H += sgn * (W[..., None] * d / dn[..., None] ** 3).sum((0, 1)) / (4 * math.pi)
        N[:, k] = -H
    return N


def test_against_surface_charge_quadrature():
    # independent numerics: field of the equivalent surface charges
    rng = np.random.default_rng(8)
    cases = [([0, 0, 0], [1.0, 2.0, 3.0]),       # self term, elongated box
             ([1.6, 0.2, -0.3], [1.0, 2.0, 3.0]),  # beside, close
             ([0.0, 0.0, 2.0], [1.0, 1.0, 1.0]),   # face neighbour of a cube (centre)
             ([1.0, 1.0, 1.0], [1.0, 1.0, 1.0]),   # corner neighbour
             ([4.0, -3.0, 2.0], [2.0, 0.5, 1.0])]
    for _ in range(5):
        e = rng.uniform(0.3, 2.0, 3)
        r = rng.uniform(-3, 3, 3)
        if np.any(np.abs(r) > e / 2 + 0.4):
            cases.append((list(r), list(e)))
    for r, e in cases:
        N = oracle.point_tensor(r, [0, 0, 0], e)
        Q = _quadrature_tensor(r, [0, 0, 0], e)
        assert np.abs(N - Q).max() < 1e-9 * max(1.0, np.abs(Q).max()), (r, e, N, Q)


def test_field_point_in_face_plane_is_the_limit():
    # reading: atan term := 0 where U == 0 (point in a face plane, outside the
    # face).  The value must equal the limit from either side.
    e = [1.0, 1.0, 1.0]
    r0 = np.array([0.5, 2.0, 0.3])  # x = +a plane, outside the face in y
    N0 = oracle.point_tensor(r0, [0, 0, 0], e)
    for dx in (1e-7, -1e-7):
        N1 = oracle.point_tensor(r0 + [dx, 0, 0], [0, 0, 0], e)
        assert np.abs(N1 - N0).max() < 1e-6
    Q = _quadrature_tensor(r0, [0, 0, 0], e)
    assert np.abs(N0 - Q).max() < 1e-9


def test_superposition_into_union_prism():
    # the tiles of a tensor-product grid add up to the prism they fill:
    # sum_j N_ij = N_prism(c_i), exactly (same potential), for a uniform and
    # a graded grid.  Pins the field of a uniform magnetisation too.
    for t in (wl.film(10, 4, 2, size=(100e-9, 40e-9, 6e-9)),
              wl.graded_film(9, 5, 3, size=(120e-9, 50e-9, 9e-9), seed=3)):
        N = oracle.demag_tensor(t.centre, t.edge)
        lo = t.centre - t.edge / 2
        hi = t.centre + t.edge / 2
        pc = (lo.min(0) + hi.max(0)) / 2
        pe = hi.max(0) - lo.min(0)
        Ssum = oracle.six_to_full(N.sum(axis=1))
        for i in range(t.n):
            Nb = oracle.point_tensor(t.centre[i], pc, pe)
            assert np.abs(Ssum[i] - Nb).max() < 1e-12
        # uniform m, uniform Ms: H_d,i = -N_prism(c_i) Ms m
        m = np.tile(np.array([0.3, -0.5, 0.81]) / np.linalg.norm([0.3, -0.5, 0.81]), (t.n, 1))
        H = oracle.demag_field_dense(N, t.Ms, m)
        for i in range(0, t.n, 7):
            Nb = oracle.point_tensor(t.centre[i], pc, pe)
            np.testing.assert_allclose(H[i], -Nb @ (t.Ms[i] * m[i]), rtol=1e-11, atol=1e-6)


def test_dense_field_equals_rows_and_brute_force():
    t = wl.graded_film(7, 4, 2, size=(60e-9, 30e-9, 4e-9), seed=1)
    t.Ms[:] = np.linspace(4e5, 1.2e6, t.n)
    N = oracle.demag_tensor(t.centre, t.edge)
    m = wl.m_random(t.n, seed=4)
    H = oracle.demag_field_dense(N, t.Ms, m)
    # brute force with the full 3x3 blocks
    F = oracle.six_to_full(N)
    Hb = -np.einsum("ijab,jb->ia", F, t.Ms[:, None] * m)
    np.testing.assert_allclose(H, Hb, rtol=1e-12, atol=1e-9)
    rows = np.array([0, 5, t.n - 1, 17])
    Hr = oracle.demag_field_rows(t.centre, t.edge, t.Ms, m, rows)
    np.testing.assert_allclose(Hr, H[rows], rtol=1e-13, atol=1e-9)


def test_blocks_match_full_tensor():
    t = wl.film(6, 3, 1)
    N = oracle.demag_tensor(t.centre, t.edge)
    pairs = np.array([[0, 0], [1, 5], [17, 2], [10, 10]])
    B = oracle.demag_blocks(t.centre, t.edge, pairs)
    np.testing.assert_array_equal(B, N[pairs[:, 0], pairs[:, 1]])


def test_overlap_detection():
    t = wl.film(4, 2, 1)
    assert oracle.check_tiles(t.centre, t.edge) == oracle.OK
    c = t.centre.copy()
    c[1] = c[0] + np.array([0.3, 0, 0]) * t.edge[0]  # tile 1 overlaps tile 0
    assert oracle.check_tiles(c, t.edge) == oracle.EOVERLAP


def test_centre_on_another_tile_surface_is_rejected():
    # The closed form is singular where a field point lies on a source tile's
    # surface (ln(W + R) with R = |W| on a face, and atan(./0) on its edges),
    # so a tile centre in or on another tile is invalid even where the two
    # volumes do not overlap measurably.  A tile too thin to overlap within
    # the relative tolerance 1e-12 (edge 1e-22 m against 1e-8 m), whose
    # centre lies on the +x face, on an edge, or at a corner of a 10 nm cube,
    # tests that rule alone; the same thin tile just outside the face is valid.
    h, eps = 10e-9, 1e-22
    edge = np.array([[h, h, h], [eps, eps, eps]])
    for where in ([0.5 * h, 0.0, 0.0], [0.5 * h, 0.5 * h, 0.0], [0.5 * h, -0.5 * h, 0.5 * h],
                  [0.5 * h, 0.2 * h, -0.3 * h]):
        c = np.array([[0.0, 0.0, 0.0], where])
        assert oracle.check_tiles(c, edge) == oracle.EOVERLAP, where
    c = np.array([[0.0, 0.0, 0.0], [0.5 * h * (1 + 1e-6), 0.0, 0.0]])
    assert oracle.check_tiles(c, edge) == oracle.OK
    # face-adjacent tiles of a grid touch without either centre on the other
    t = wl.graded_film(5, 4, 2, size=(40e-9, 30e-9, 6e-9), seed=4)
    assert oracle.check_tiles(t.centre, t.edge) == oracle.OK


def test_threshold_drops_the_smallest_fraction():
    # Sec. 4.3.1: a threshold f sets the fraction f of the nonzero tensor
    # elements with the smallest magnitude to zero -- checked on the explicit
    # 3n x 3n matrix, built block by block
    t = wl.graded_film(7, 5, 2, size=(70e-9, 50e-9, 6e-9), seed=3)
    N = oracle.demag_tensor(t.centre, t.edge)
    full = oracle.six_to_full(N).transpose(0, 2, 1, 3).reshape(3 * t.n, 3 * t.n)
    nz_before = np.count_nonzero(full.astype(np.float32))
    for f in (0.2, 0.4, 0.7):
        Nt, thr, kept = oracle.threshold_tensor(N, f)
        ft = oracle.six_to_full(Nt).transpose(0, 2, 1, 3).reshape(3 * t.n, 3 * t.n)
        nz_after = np.count_nonzero(ft)
        dropped = nz_before - nz_after
        # exactly k, or k - 1 when the cut splits the two copies of an entry
        assert dropped in (int(f * nz_before), int(f * nz_before) - 1)
        assert kept == nz_after
        # every dropped element is no larger than every kept one
        a = np.abs(full.astype(np.float32))
        d_max = a[(ft == 0) & (a > 0)].max()
        k_min = np.abs(ft.astype(np.float32))[ft != 0].min()
        assert d_max <= k_min
        np.testing.assert_array_equal(oracle.six_to_full(Nt), oracle.six_to_full(Nt).transpose(0, 1, 3, 2))
    Nt, thr, kept = oracle.threshold_tensor(N, 0.0)
    np.testing.assert_array_equal(Nt, N)


def test_threshold_ties_brute_force():
    # a uniform grid: the tensor depends only on the offset between tiles, so
    # each value appears many times and the cut falls inside a run of ties.
    # Brute force: every element of the full matrix as (FP32 magnitude,
    # position), a stable sort, the first k marked; an entry (both copies of
    # an off-diagonal one) is dropped iff all its copies are marked.
    t = wl.film(6, 4, 1)
    N = oracle.demag_tensor(t.centre, t.edge)
    n = t.n
    elems = []
    for i in range(n):
        for j in range(n):
            for e in range(6):
                v = abs(float(np.float32(N[i, j, e])))
                if v > 0:
                    for c in range(int(oracle._MULT[e])):
                        elems.append((v, len(elems), (i, j, e)))
    order = sorted(elems, key=lambda x: (x[0], x[1]))
    ties_at_cut = 0
    for f in (0.1, 0.25, 0.5, 0.7):
        k = int(f * len(elems))
        marked = {}
        for rank, (v, _, ent) in enumerate(order):
            marked.setdefault(ent, []).append(rank < k)
        ties_at_cut += sum(1 for x in order if x[0] == order[k][0])
        Nt, thr, kept = oracle.threshold_tensor(N, f)
        assert thr == order[k][0]
        for (i, j, e), flags in marked.items():
            assert (Nt[i, j, e] == 0) == all(flags), (f, i, j, e, flags)
            if not all(flags):
                assert Nt[i, j, e] == N[i, j, e]
        assert kept == sum(len(fl) for fl in marked.values() if not all(fl))
    assert ties_at_cut > 8  # the case does exercise ties


def test_scaled_geometry_tensor_and_exchange():
    # the point tensor depends only on shape ratios: scaling every centre and
    # edge by lam leaves N unchanged, while the exchange field scales as
    # lam^-2 (a size sweep, e.g. the d/l_ex axis of standard problem 2,
    # keeps one tensor and changes the exchange stiffness by lam^-2)
    t = wl.graded_film(6, 4, 2, size=(60e-9, 40e-9, 6e-9), seed=5)
    lam = 3.7
    N1 = oracle.demag_tensor(t.centre, t.edge)
    N2 = oracle.demag_tensor(lam * t.centre, lam * t.edge)
    assert np.abs(N1 - N2).max() <= 1e-12 * np.abs(N1).max()
    m = wl.m_random(t.n, seed=3)
    md1 = oracle.Model.from_tiles(t)
    md2 = oracle.Model(lam * t.centre, lam * t.edge, t.Ms, t.Aex, t.Ku, t.axis, t.nbr, N=N1)
    H1 = oracle.exchange_field(md1, m)
    H2 = oracle.exchange_field(md2, m)
    np.testing.assert_allclose(H2, H1 / lam ** 2, rtol=1e-12, atol=1e-12 * np.abs(H1).max())


def test_single_layer_xz_yz_vanish_by_mirror_symmetry():
    # every tile in one layer (same centre z and z edge): the field point lies
    # in each source's mid-plane and N_xz, N_yz (odd in the z offset) vanish;
    # on a graded in-plane grid at an arbitrary height they are FP64
    # round-off (<= 1e-12), while a second layer makes them O(1e-2)
    rng = np.random.default_rng(7)
    xf = np.concatenate([[0.0], np.cumsum(rng.uniform(2e-9, 8e-9, 9))])
    yf = np.concatenate([[0.0], np.cumsum(rng.uniform(2e-9, 8e-9, 5))])
    for z0 in (0.0, 17.3e-9):
        t = wl.grid_tiles(xf, yf, np.array([z0, z0 + 3e-9]), wl.SP4_MS, wl.SP4_AEX, 0.0)
        N = oracle.demag_tensor(t.centre, t.edge)
        assert np.abs(N[..., [2, 4]]).max() <= 1e-12
        assert np.abs(N[..., [0, 1, 3, 5]]).max() > 0.1  # the in-plane part is not small
    two = wl.grid_tiles(xf, yf, np.array([0.0, 3e-9, 6e-9]), wl.SP4_MS, wl.SP4_AEX, 0.0)
    N2 = oracle.demag_tensor(two.centre, two.edge)
    assert np.abs(N2[..., [2, 4]]).max() > 1e-3
