"""FP64 CPU oracle for the tile-based micromagnetic method (arXiv 2107.05364).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, double-precision
statement of what the GPU path computes.  Only the test-suite, the smoke
check and the CPU-baseline leg of ``bench.py`` may import it; the product
path (the CUDA library and its binding) never does, and shares no code with
it.  The arithmetic lives in ``oracle.c``; this module only marshals numpy
arrays into it (``ctypes``).

Functions and the passage each follows (see ``oracle.c`` for the formulas):

* :func:`point_tensor`, :func:`demag_tensor`, :func:`demag_blocks` --
  Sec. 3, cuboid tile tensor evaluated at tile centres (closed form of the
  Newtonian potential; Eq. 9 read as ``H_d = -N (Ms m)``).
* :func:`demag_field_dense`, :func:`demag_field_rows` -- Eq. 9 / Eq. 17.
* :func:`exchange_field` -- Eq. 12 with the Neumann condition of Eq. 3.
* :func:`anisotropy_field` -- Eq. 16.  Zeeman -- Eq. 7.
* :func:`llg_rhs` -- Eq. 1 (Landau-Lifshitz) or its Gilbert form.
* :func:`integrate`, :func:`relax`, :func:`integrate_linear` -- Sec. 3.1,
  Dormand-Prince RK(4,5).
* :func:`energy` -- Eqs. 4, 6, 8, 11, 15.
* :func:`threshold_tensor` -- Sec. 4.3.1, dropping the smallest fraction of
  the nonzero tensor elements.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

MU0 = 4e-7 * np.pi

OK, EINVAL, EOVERLAP, ENOCONV, ENONFINITE = 0, 1, 3, 4, 6


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (gcc, OpenMP, -O2,
    strict IEEE arithmetic: no fast-math, no host-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Model(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64),
                ("centre", ctypes.c_void_p), ("edge", ctypes.c_void_p),
                ("Ms", ctypes.c_void_p), ("Aex", ctypes.c_void_p),
                ("Ku", ctypes.c_void_p), ("axis", ctypes.c_void_p),
                ("nbr", ctypes.c_void_p), ("N", ctypes.c_void_p),
                ("xw", ctypes.c_void_p), ("vol", ctypes.c_void_p)]


class _Llg(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("alpha", ctypes.c_double),
                ("Ha", ctypes.c_double * 3), ("form", ctypes.c_int),
                ("precess", ctypes.c_int)]


class _Ode(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("h0", ctypes.c_double), ("hmax", ctypes.c_double),
                ("max_steps", ctypes.c_int64), ("fixed_h", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("n_accept", ctypes.c_int64), ("n_reject", ctypes.c_int64),
                ("n_rhs", ctypes.c_int64), ("t", ctypes.c_double),
                ("h", ctypes.c_double), ("tau", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_SO)
    return _lib


def num_threads() -> int:
    return int(lib().or_num_threads())


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


# ---------------------------------------------------------------------------
# tensor and field
# ---------------------------------------------------------------------------
def point_tensor(r, centre, edge) -> np.ndarray:
    """3x3 point tensor of the cuboid (``centre``, full ``edge``) at ``r``."""
    r = np.ascontiguousarray(r, np.float64)
    c = np.ascontiguousarray(centre, np.float64)
    e = np.ascontiguousarray(edge, np.float64)
    out = np.zeros(6)
    lib().or_point_tensor(_p(r), _p(c), _p(e), _p(out))
    return six_to_full(out)


def six_to_full(n6: np.ndarray) -> np.ndarray:
    """{xx,xy,xz,yy,yz,zz} (last axis) -> symmetric 3x3 (last two axes)."""
    n6 = np.asarray(n6)
    idx = np.array([[0, 1, 2], [1, 3, 4], [2, 4, 5]])
    return n6[..., idx]


def check_tiles(centre, edge) -> int:
    c = np.ascontiguousarray(centre, np.float64).reshape(-1)
    e = np.ascontiguousarray(edge, np.float64).reshape(-1)
    return int(lib().or_check_tiles(ctypes.c_int64(c.size // 3), _p(c), _p(e)))


def demag_tensor(centre, edge) -> np.ndarray:
    """All blocks; returns (n, n, 6): [i, j] = tile j at the centre of tile i."""
    c = np.ascontiguousarray(centre, np.float64).reshape(-1)
    e = np.ascontiguousarray(edge, np.float64).reshape(-1)
    n = c.size // 3
    out = np.empty((n, n, 6))
    lib().or_demag_tensor(ctypes.c_int64(n), _p(c), _p(e), _p(out))
    return out


def tetra_point_tensor(r, verts, full=False) -> np.ndarray:
    """Tensor of the uniformly magnetised tetrahedron verts (4, 3) at r:
    (3, 3) if full, else the 6 entries of its symmetric part."""
    r = np.ascontiguousarray(r, np.float64)
    v = np.ascontiguousarray(verts, np.float64).reshape(12)
    if full:
        out = np.empty(9)
        lib().or_tetra_point_tensor_full(_p(r), _p(v), _p(out))
        return out.reshape(3, 3)
    out = np.empty(6)
    lib().or_tetra_point_tensor(_p(r), _p(v), _p(out))
    return out


def tetra_demag_tensor(verts) -> np.ndarray:
    """(n, n, 6) tensor of tetrahedral tiles verts (n, 4, 3) at their centroids."""
    v = np.ascontiguousarray(verts, np.float64).reshape(-1, 12)
    n = v.shape[0]
    N = np.empty((n, n, 6))
    lib().or_tetra_demag_tensor(ctypes.c_int64(n), _p(v), _p(N))
    return N


def tetra_field_rows(verts, Ms, m, rows) -> np.ndarray:
    """H_d at the centroids of tetrahedral tiles `rows` (verts (n, 4, 3)),
    row by row without storing the tensor."""
    v = np.ascontiguousarray(verts, np.float64).reshape(-1)
    n = v.size // 12
    Ms = np.ascontiguousarray(np.broadcast_to(Ms, (n,)), np.float64)
    m = np.ascontiguousarray(m, np.float64).reshape(-1)
    rows = np.ascontiguousarray(rows, np.int64)
    H = np.empty(3 * rows.size)
    lib().or_tetra_field_rows(ctypes.c_int64(n), _p(v), _p(Ms), _p(m), ctypes.c_int64(rows.size), _p(rows),
                              _p(H))
    return H.reshape(-1, 3)


def tetra_model(verts, tets, Ms, Aex, Ku, axis, N=None):
    """Oracle model of tetrahedral tiles: vertices (nv, 3), tets (n, 4)
    vertex indices.  Centroids, volumes, the tensor (Sec. 3) and the
    two-point-flux exchange coefficients area / (V_i d_ip) over shared faces
    (d_ip the centroid distance along the face normal; a face on the
    boundary carries no flux)."""
    verts = np.asarray(verts, np.float64)
    tets = np.asarray(tets, np.int64)
    n = tets.shape[0]
    P = verts[tets]  # (n, 4, 3)
    cen = P.mean(axis=1)
    vol = np.abs(np.einsum("ij,ij->i", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))) / 6
    faces = {}
    for i in range(n):
        for f in range(4):
            key = tuple(sorted(int(tets[i, k]) for k in range(4) if k != f))
            faces.setdefault(key, []).append((i, f))
    nbr = -np.ones((n, 6), np.int32)
    xw = np.zeros((n, 6))
    for key, owners in faces.items():
        if len(owners) != 2:
            continue
        a, b, c = verts[list(key)]
        nrm = np.cross(b - a, c - a)
        area = 0.5 * np.linalg.norm(nrm)
        nrm = nrm / np.linalg.norm(nrm)
        (i, fi), (j, fj) = owners
        d = abs(np.dot(cen[j] - cen[i], nrm))
        nbr[i, fi], nbr[j, fj] = j, i
        xw[i, fi] = area / (vol[i] * d)
        xw[j, fj] = area / (vol[j] * d)
    if N is None:
        N = tetra_demag_tensor(P)
    return Model(cen, None, Ms, Aex, Ku, axis, nbr, N=N, xw=xw, vol=vol)


def demag_blocks(centre, edge, pairs) -> np.ndarray:
    c = np.ascontiguousarray(centre, np.float64).reshape(-1)
    e = np.ascontiguousarray(edge, np.float64).reshape(-1)
    pr = np.ascontiguousarray(pairs, np.int64).reshape(-1, 2)
    out = np.empty((pr.shape[0], 6))
    lib().or_demag_blocks(_p(c), _p(e), ctypes.c_int64(pr.shape[0]), _p(pr), _p(out))
    return out


def demag_field_dense(N, Ms, m) -> np.ndarray:
    N = np.ascontiguousarray(N, np.float64)
    n = N.shape[0]
    Ms = np.ascontiguousarray(Ms, np.float64)
    m = np.ascontiguousarray(m, np.float64).reshape(-1)
    H = np.empty(3 * n)
    lib().or_demag_field_dense(ctypes.c_int64(n), _p(N), _p(Ms), _p(m), _p(H))
    return H.reshape(n, 3)


def demag_field_rows(centre, edge, Ms, m, rows) -> np.ndarray:
    c = np.ascontiguousarray(centre, np.float64).reshape(-1)
    e = np.ascontiguousarray(edge, np.float64).reshape(-1)
    n = c.size // 3
    Ms = np.ascontiguousarray(Ms, np.float64)
    m = np.ascontiguousarray(m, np.float64).reshape(-1)
    rows = np.ascontiguousarray(rows, np.int64)
    H = np.empty(3 * rows.size)
    lib().or_demag_field_rows(ctypes.c_int64(n), _p(c), _p(e), _p(Ms), _p(m),
                              ctypes.c_int64(rows.size), _p(rows), _p(H))
    return H.reshape(-1, 3)


# ---------------------------------------------------------------------------
# model-level functions
# ---------------------------------------------------------------------------
class Model:
    """Tiles + stored FP64 tensor.  Arrays are kept alive by this object."""

    def __init__(self, centre, edge, Ms, Aex, Ku, axis, nbr=None, N=None, xw=None, vol=None):
        """Cuboid tiles (centre, edge), or any tiles with their tensor N,
        volumes vol and exchange face coefficients xw (6 per tile, 1/m^2)."""
        self.centre = np.ascontiguousarray(centre, np.float64).reshape(-1, 3)
        self.n = self.centre.shape[0]
        self.edge = np.ascontiguousarray(edge if edge is not None else np.ones((self.n, 3)),
                                         np.float64).reshape(-1, 3)
        self.xw = None if xw is None else np.ascontiguousarray(xw, np.float64).reshape(-1, 6)
        self.vol = None if vol is None else np.ascontiguousarray(vol, np.float64).reshape(-1)
        self.Ms = np.ascontiguousarray(np.broadcast_to(Ms, (self.n,)), np.float64)
        self.Aex = np.ascontiguousarray(np.broadcast_to(Aex, (self.n,)), np.float64)
        self.Ku = np.ascontiguousarray(np.broadcast_to(Ku, (self.n,)), np.float64)
        self.axis = np.ascontiguousarray(
            np.broadcast_to(np.asarray(axis, np.float64).reshape(-1, 3), (self.n, 3)))
        self.nbr = None if nbr is None else np.ascontiguousarray(nbr, np.int32).reshape(-1, 6)
        self.N = demag_tensor(self.centre, self.edge) if N is None else np.ascontiguousarray(N, np.float64)
        self._s = _Model(self.n, _p(self.centre), _p(self.edge), _p(self.Ms), _p(self.Aex),
                         _p(self.Ku), _p(self.axis), _p(self.nbr) if self.nbr is not None else None,
                         _p(self.N), _p(self.xw) if self.xw is not None else None,
                         _p(self.vol) if self.vol is not None else None)

    @classmethod
    def from_tiles(cls, tiles, N=None):
        """Build from a workload tile-set object (fields centre, edge, Ms,
        Aex, Ku, axis, nbr)."""
        return cls(tiles.centre, tiles.edge, tiles.Ms, tiles.Aex, tiles.Ku, tiles.axis,
                   tiles.nbr, N)

    @property
    def volume(self):
        return self.vol if self.vol is not None else np.prod(self.edge, axis=1)

    def mean_m(self, m):
        m = np.asarray(m, np.float64).reshape(-1, 3)
        V = self.volume
        return (V[:, None] * m).sum(0) / V.sum()


def llg_params(gamma=2.211e5, alpha=0.02, Ha=(0.0, 0.0, 0.0), form=0, precess=1):
    return _Llg(float(gamma), float(alpha), (ctypes.c_double * 3)(*[float(x) for x in Ha]),
                int(form), int(precess))


def ode_opts(rtol=1e-6, atol=1e-6, h0=1e-14, hmax=1e-11, max_steps=10_000_000, fixed_h=0.0):
    return _Ode(float(rtol), float(atol), float(h0), float(hmax), int(max_steps), float(fixed_h))


def demag_field(model: Model, m) -> np.ndarray:
    return demag_field_dense(model.N, model.Ms, m)


def exchange_field(model: Model, m) -> np.ndarray:
    m = np.ascontiguousarray(m, np.float64).reshape(-1)
    H = np.empty(3 * model.n)
    lib().or_exchange_field(ctypes.byref(model._s), _p(m), _p(H))
    return H.reshape(-1, 3)


def anisotropy_field(model: Model, m) -> np.ndarray:
    m = np.ascontiguousarray(m, np.float64).reshape(-1)
    H = np.empty(3 * model.n)
    lib().or_anisotropy_field(ctypes.byref(model._s), _p(m), _p(H))
    return H.reshape(-1, 3)


def effective_field(model: Model, m, params) -> np.ndarray:
    m = np.ascontiguousarray(m, np.float64).reshape(-1)
    H = np.empty(3 * model.n)
    lib().or_effective_field(ctypes.byref(model._s), ctypes.byref(params), _p(m), _p(H), None)
    return H.reshape(-1, 3)


def llg_rhs(model: Model, m, params):
    """Returns (dm/dt (n,3), tau = max_i |m_i x H_i|/Ms_i)."""
    m = np.ascontiguousarray(m, np.float64).reshape(-1)
    k = np.empty(3 * model.n)
    tau = ctypes.c_double(0.0)
    lib().or_llg_rhs(ctypes.byref(model._s), ctypes.byref(params), _p(m), _p(k), ctypes.byref(tau))
    return k.reshape(-1, 3), tau.value


def energy(model: Model, m, params) -> dict:
    m = np.ascontiguousarray(m, np.float64).reshape(-1)
    out = np.empty(5)
    lib().or_energy(ctypes.byref(model._s), ctypes.byref(params), _p(m), _p(out))
    return dict(total=out[0], zeeman=out[1], demag=out[2], exchange=out[3], anisotropy=out[4])


def _stats(st: _Stats) -> dict:
    return dict(n_accept=st.n_accept, n_reject=st.n_reject, n_rhs=st.n_rhs, t=st.t, h=st.h,
                tau=st.tau)


def integrate(model: Model, m0, params, opts, t0: float, t1: float, n_out: int):
    """Integrate Eq. 1 from t0 to t1.  Returns (status, m_final (n,3),
    <m> at t0 + (k+1)(t1-t0)/n_out (n_out,3), stats)."""
    m = np.ascontiguousarray(m0, np.float64).reshape(-1).copy()
    mavg = np.zeros((n_out, 3))
    st = _Stats()
    s = lib().or_integrate(ctypes.byref(model._s), ctypes.byref(params), ctypes.byref(opts), _p(m),
                           ctypes.c_double(t0), ctypes.c_double(t1), ctypes.c_int64(n_out), _p(mavg),
                           ctypes.byref(st))
    return int(s), m.reshape(-1, 3), mavg, _stats(st)


def relax(model: Model, m0, params, opts, tol: float, t_max: float):
    """Relax until max torque < tol.  Returns (status, m (n,3), stats)."""
    m = np.ascontiguousarray(m0, np.float64).reshape(-1).copy()
    st = _Stats()
    s = lib().or_relax(ctypes.byref(model._s), ctypes.byref(params), ctypes.byref(opts), _p(m),
                       ctypes.c_double(tol), ctypes.c_double(t_max), ctypes.byref(st))
    return int(s), m.reshape(-1, 3), _stats(st)


def integrate_linear(lam, y0, opts, t0, t1, n_out):
    """y' = lam * y (component-wise) with the same RK(4,5) driver."""
    lam = np.ascontiguousarray(lam, np.float64)
    y = np.ascontiguousarray(y0, np.float64).copy()
    yout = np.zeros((n_out, y.size))
    st = _Stats()
    s = lib().or_integrate_linear(ctypes.c_int64(y.size), _p(lam), ctypes.byref(opts), _p(y),
                                  ctypes.c_double(t0), ctypes.c_double(t1), ctypes.c_int64(n_out),
                                  _p(yout), ctypes.byref(st))
    return int(s), y, yout, _stats(st)


def dp45_tableau():
    c = np.zeros(7)
    a = np.zeros(42)
    b = np.zeros(7)
    bh = np.zeros(7)
    lib().or_dp45_tableau(_p(c), _p(a), _p(b), _p(bh))
    return c, a.reshape(7, 6), b, bh


# ---------------------------------------------------------------------------
# Sec. 4.3.1: thresholding
# ---------------------------------------------------------------------------
_MULT = np.array([1, 2, 2, 1, 2, 1])  # copies of each stored entry in the full 3x3 block


def threshold_tensor(N, fraction):
    """Sec. 4.3.1: the fraction `fraction` of the nonzero elements of the full
    3n x 3n tensor with the smallest magnitude is set to zero.

    Readings: the elements are those of the full matrix (an off-diagonal
    entry of a symmetric block stands for two elements); they are ranked by
    magnitude rounded to FP32 (the storage precision the product uses), ties
    in (row tile i, column tile j, entry xx, xy, xz, yy, yz, zz) order with an
    off-diagonal entry's two copies adjacent; the first k = floor(fraction *
    nonzeros) of that order are dropped, except that an entry whose two
    copies are split by the cut stays (every 3x3 block stays symmetric).
    Returns (thresholded FP64 tensor (n, n, 6), t = magnitude of the element
    of rank k, kept nonzero elements)."""
    N = np.asarray(N, np.float64)
    a32 = np.abs(N.astype(np.float32)).astype(np.float64)
    flat = a32.ravel()  # (i, j, entry) order
    mult = np.tile(_MULT, flat.size // 6)
    nzm = flat > 0
    nz = np.sort(np.repeat(flat[nzm], mult[nzm]))
    k = int(fraction * nz.size)
    if k == 0 or nz.size == 0:
        return N.copy(), 0.0, int(nz.size)
    t = nz[k]
    less = nzm & (flat < t)
    r = k - int(mult[less].sum())  # elements equal to t still to drop
    tie = flat == t
    cum = np.cumsum(np.where(tie, mult, 0))  # copies of t up to and including this entry
    drop = less | (tie & (cum <= r))
    keep = (nzm & ~drop).reshape(N.shape)
    out = np.where(keep, N, 0.0)
    kept = int((keep.reshape(-1, 6) * _MULT).sum())
    return out, float(t), kept


def hysteresis(model: Model, m0, H, direction, opts, t_step, gamma=2.211e5, alpha=4000.0, form=1, precess=0,
               tol=0.0):
    """Sec. 4.1 (standard problem 2): the applied field takes the values
    H[s] * direction (A/m) in turn; at each value the state, carried over
    from the previous one, is evolved for t_step seconds (tol = 0: the paper
    holds every field value for a fixed time), or relaxed until the torque is
    below tol with t_step as the cap (reaching the cap is not an error).  LL
    form with the precession term dropped and a large damping, as the paper.
    Returns (status, <m> at the end of each value (S, 3), final state)."""
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    m = np.asarray(m0, np.float64).reshape(-1, 3).copy()
    out = np.zeros((len(H), 3))
    t = 0.0
    for s, h in enumerate(H):
        p = llg_params(gamma=gamma, alpha=alpha, Ha=h * d, form=form, precess=precess)
        if tol > 0:
            st, m, _ = relax(model, m, p, opts, tol, t_step)
            if st == ENOCONV:
                st = OK
        else:
            st, m, mav, _ = integrate(model, m, p, opts, t, t + t_step, 1)
        if st != OK:
            return st, out, m
        out[s] = model.mean_m(m)
        t += t_step
    return OK, out, m


def loop_summary(H, mavg, direction):
    """Coercivity and remanence of a descending branch (Sec. 4.1): the field
    at which the projection of <m> on the field direction first changes
    sign, linearly interpolated between the two field values around it (nan
    if it never does), and <m> at H = 0, interpolated likewise (nan if the
    schedule does not cross zero)."""
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    H = np.asarray(H, np.float64)
    mavg = np.asarray(mavg, np.float64).reshape(-1, 3)
    proj = mavg @ d
    hc = float("nan")
    for s in range(1, len(H)):
        if proj[s - 1] > 0 >= proj[s]:
            hc = H[s - 1] + (H[s] - H[s - 1]) * proj[s - 1] / (proj[s - 1] - proj[s])
            break
    mr = np.full(3, np.nan)
    for s in range(1, len(H)):
        if H[s - 1] >= 0 >= H[s] and H[s - 1] != H[s]:
            w = H[s - 1] / (H[s - 1] - H[s])
            mr = (1 - w) * mavg[s - 1] + w * mavg[s]
            break
    return float(hc), mr


def crossover(centre, edge, Ms, Aex, Ku, axis, nbr, lam, mA, mB, params, opts, tol, t_max):
    """Sec. 4.2 (standard problem 3): for each size lam[k] the body is
    really scaled (centres and edges times lam[k], its tensor recomputed),
    states A and B are relaxed (torque below tol or t_max, which counts as
    done), and their energy densities E / V (J/m^3) compared.  Returns
    (eA, eB, lam at which eA - eB first changes sign, linear between the two
    sizes around it (nan if none), relaxed states)."""
    K = len(lam)
    eA, eB = np.zeros(K), np.zeros(K)
    states = []
    for k, lk in enumerate(lam):
        md = Model(lk * np.asarray(centre), lk * np.asarray(edge), Ms, Aex, Ku, axis, nbr)
        V = md.volume.sum()
        for m0, out in ((mA, eA), (mB, eB)):
            st, m, _ = relax(md, m0, params, opts, tol, t_max)
            if st not in (OK, ENOCONV):
                raise RuntimeError("oracle relax failed with status %d" % st)
            out[k] = energy(md, m, params)["total"] / V
            states.append(m)
    return eA, eB, first_crossing(lam, eA, eB), states


def first_crossing(x, a, b):
    """The x at which a - b first changes sign, linear between the two
    samples around it (nan if it never does)."""
    for k in range(1, len(x)):
        d0, d1 = a[k - 1] - b[k - 1], a[k] - b[k]
        if (d0 < 0) != (d1 < 0):
            return float(x[k - 1] + (x[k] - x[k - 1]) * d0 / (d0 - d1))
    return float("nan")
