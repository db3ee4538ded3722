"""Pins for the oracle's tetrahedron tile (Sec. 3: the tensor of a uniformly
magnetised tetrahedron, cited by the paper but not printed; written in the
oracle from the face charges) and for its tile-set model.

* superposition: the 6 tetrahedra of a cube's Kuhn triangulation add up to
  the cuboid tensor (pinned on its own in test_oracle_tensor.py), at points
  outside and inside the cube;
* trace 1 inside a tetrahedron, 0 outside; symmetric 3x3 blocks;
* the dipole limit with second-order convergence;
* Gauss-Legendre quadrature of the face charges (independent numerics);
* a mesh of tetrahedra filling a box gives the union body's tensor, and its
  two-point-flux exchange field vanishes for uniform m.
"""
import itertools
import math

import numpy as np
from numpy.polynomial.legendre import leggauss

import oracle
from paper_2107_05364_gb300 import workloads as wl


def kuhn_tets(lo, hi):
    """The 6 tetrahedra (0, e_a, e_a + e_b, 1) of the box [lo, hi]."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    out = []
    for perm in itertools.permutations(range(3)):
        p = np.zeros(3)
        vs = [p.copy()]
        for a in perm:
            p[a] = 1.0
            vs.append(p.copy())
        out.append(lo + np.array(vs) * (hi - lo))
    return np.array(out)


def test_kuhn_cube_sums_to_the_cuboid():
    lo, hi = np.array([-0.5, -1.0, -0.35]), np.array([0.5, 1.0, 0.35])
    tets = kuhn_tets(lo, hi)
    assert abs(sum(abs(np.linalg.det(t[1:] - t[0])) / 6 for t in tets) - np.prod(hi - lo)) < 1e-12
    rng = np.random.default_rng(3)
    pts = [np.array([1.7, 0.3, -0.2]), np.array([0.1, 0.2, 3.0]), np.array([4.0, -5.0, 6.0]),
           np.array([0.11, 0.23, 0.05]), np.array([-0.3, 0.7, -0.2])]
    pts += list(rng.uniform(-3, 3, (6, 3)))
    for r in pts:
        S = sum(oracle.tetra_point_tensor(r, t, full=True) for t in tets)
        C = oracle.point_tensor(r, (lo + hi) / 2, hi - lo)
        assert np.abs(S - C).max() < 1e-12 * max(1.0, np.abs(C).max()), (r, S, C)


def random_tet(rng):
    while True:
        v = rng.uniform(-1, 1, (4, 3))
        if abs(np.linalg.det(v[1:] - v[0])) > 0.3:
            return v


def test_trace_and_symmetry():
    rng = np.random.default_rng(5)
    for _ in range(10):
        v = random_tet(rng)
        w = rng.dirichlet(np.ones(4))
        inside = w @ v
        N = oracle.tetra_point_tensor(inside, v, full=True)
        assert abs(np.trace(N) - 1) < 1e-12
        assert np.abs(N - N.T).max() < 1e-12
        out = v.mean(0) + rng.uniform(2.5, 4, 3) * rng.choice([-1, 1], 3)
        N = oracle.tetra_point_tensor(out, v, full=True)
        assert abs(np.trace(N)) < 1e-13 * max(1, np.abs(N).max()) + 1e-15
        assert np.abs(N - N.T).max() < 1e-13


def test_dipole_limit():
    v = np.array([[0, 0, 0], [1.0, 0.1, 0], [0.2, 1.3, 0.1], [0.3, 0.2, 0.9]])
    c = v.mean(0)
    V = abs(np.linalg.det(v[1:] - v[0])) / 6
    d = np.array([0.5, -0.7, 0.3])
    d /= np.linalg.norm(d)
    errs = []
    for dist in (20.0, 40.0, 80.0, 160.0):
        N = oracle.tetra_point_tensor(c + dist * d, v, full=True)
        D = -(V / (4 * math.pi * dist ** 3)) * (3 * np.outer(d, d) - np.eye(3))
        errs.append(np.abs(N - D).max() / np.abs(D).max())
    errs = np.array(errs)
    assert errs[0] < 1e-2
    ratios = errs[:-1] / errs[1:]
    assert np.all(ratios > 3.0) and np.all(ratios < 5.0), ratios


def quadrature_tensor(r, v, nq=40):
    """N[:, k] = -H for M = e_k, H the field of the face charges M.n:
    (1/4pi) sum_f (M.n_f) int_f (r - r')/|r - r'|^3 dS', each face mapped
    from the unit square (collapsed at one vertex) with Gauss-Legendre."""
    g, w = leggauss(nq)
    s = 0.5 * (g + 1)
    ws = 0.5 * w
    U, Vv = np.meshgrid(s, s, indexing="ij")
    W = np.outer(ws, ws)
    N = np.zeros((3, 3))
    cen = v.mean(0)
    for f in range(4):
        a, b, c = [v[k] for k in range(4) if k != f]
        nrm = np.cross(b - a, c - a)
        area2 = np.linalg.norm(nrm)
        nrm /= area2
        if np.dot(nrm, a - cen) < 0:
            nrm = -nrm
        # x(u, t) = a + u (b - a) + u t (c - b), Jacobian u * |(b - a) x (c - b)|
        P = a + U[..., None] * (b - a) + (U * Vv)[..., None] * (c - b)
        J = U * np.linalg.norm(np.cross(b - a, c - b))
        d = r - P
        dn = np.linalg.norm(d, axis=-1)
        G = ((W * J)[..., None] * d / dn[..., None] ** 3).sum((0, 1)) / (4 * math.pi)
        for k in range(3):
            N[:, k] -= nrm[k] * G
    return N


def test_against_face_charge_quadrature():
    rng = np.random.default_rng(11)
    for _ in range(6):
        v = random_tet(rng)
        r = v.mean(0) + rng.uniform(1.8, 3.0, 3) * rng.choice([-1, 1], 3)
        N = oracle.tetra_point_tensor(r, v, full=True)
        Q = quadrature_tensor(r, v)
        assert np.abs(N - Q).max() < 1e-10 * max(1.0, np.abs(Q).max()), (N, Q)


def test_tetra_mesh_of_a_box():
    # a box meshed with 6 tetrahedra per cell: the tensors of the tiles add up
    # to the union box's tensor at every centroid (uniform m), and exchange
    # vanishes for uniform m and for m linear in x (interior tiles)
    verts, tets = wl.tetra_box(3, 2, 2, size=(30e-9, 20e-9, 10e-9), jitter=0.0)
    md = oracle.tetra_model(verts, tets, 8e5, 1.3e-11, 0.0, (0, 0, 1))
    big = oracle.point_tensor
    for i in range(0, md.n, 7):
        S = md.N[i].sum(0)
        C = big(md.centre[i], [15e-9, 10e-9, 5e-9], [30e-9, 20e-9, 10e-9])
        full = np.array([[S[0], S[1], S[2]], [S[1], S[3], S[4]], [S[2], S[4], S[5]]])
        assert np.abs(full - C).max() < 1e-11
    H = oracle.exchange_field(md, np.tile([0.6, 0.0, 0.8], (md.n, 1)))
    assert np.abs(H).max() < 1e-6
    assert np.all(md.vol > 0) and abs(md.vol.sum() - 6e-24) < 1e-36
    # every interior face has two owners: each tile has at most 4 neighbours
    assert np.all((md.nbr >= 0).sum(1) <= 4)


def test_field_rows_match_dense_product():
    verts, tets = wl.tetra_box(3, 2, 2, size=(30e-9, 20e-9, 10e-9), jitter=0.2, seed=4)
    P = verts[tets]
    N = oracle.tetra_demag_tensor(P)
    m = wl.m_random(len(tets), seed=2)
    Ms = np.full(len(tets), 8e5)
    Hd = oracle.demag_field_dense(N, Ms, m)
    rows = np.array([0, 5, 17, len(tets) - 1])
    np.testing.assert_allclose(oracle.tetra_field_rows(P, Ms, m, rows), Hd[rows], rtol=1e-13, atol=1e-9)
