"""Seeded synthetic inputs shaped like the paper's workloads.

This module generates *data only*: tile geometries and materials, face
neighbour tables of tensor-product meshes, initial magnetisations, applied
field sets and request streams.  It holds none of the method's arithmetic
(no tensor, no field, no dynamics), so both the CUDA path and the CPU oracle
may consume what it produces.  It imports numpy only.

Random numbers come from splitmix64 (Steele, Lea & Flood 2014; Vigna's
published constants) used as a counter-based generator: value k of stream
``(seed, stream)`` is ``mix(key + (k+1) * golden)`` with
``key = mix(seed * golden ^ stream)``, mapped to [-1, 1) from its top 53 bits.

Workloads (sizes follow the paper's micromagnetic standard problems):

* ``film``          -- muMAG standard problem 4 film 500 x 125 x 3 nm (Sec. 4.3)
                       as a uniform nx x ny x nz grid.
* ``cube``          -- standard problem 3 cube (Sec. 4.2), edge in exchange
                       lengths, uniaxial anisotropy along z.
* ``graded_film``   -- non-uniform tensor-product grid of a 1000 x 250 x 5 nm
                       film, column/row/layer widths h0 * 2^u, u ~ U(-1, 1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MU0 = 4e-7 * math.pi
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# standard problem 4 material (Sec. 4.3)
SP4_MS = 8.0e5
SP4_AEX = 1.3e-11
GAMMA = 2.211e5


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` numbers uniform in [-1, 1) from stream ``(seed, stream)``."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([(np.uint64(seed) * _GOLDEN) ^ np.uint64(stream)], np.uint64))[0]
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = _mix(key + k * _GOLDEN)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


def unit01(seed: int, stream: int, count: int) -> np.ndarray:
    """Uniform in [0, 1)."""
    return 0.5 * (uniform(seed, stream, count) + 1.0)


@dataclasses.dataclass
class Tiles:
    """A set of cuboid tiles.  Arrays are tile-major (row i = tile i)."""
    centre: np.ndarray   # (n, 3) m
    edge: np.ndarray     # (n, 3) full edge lengths, m
    Ms: np.ndarray       # (n,) A/m
    Aex: np.ndarray      # (n,) J/m
    Ku: np.ndarray       # (n,) J/m^3
    axis: np.ndarray     # (n, 3) unit easy axis
    nbr: np.ndarray      # (n, 6) int32 face neighbours (-x,+x,-y,+y,-z,+z), -1 none
    shape: tuple         # (nx, ny, nz) of the tensor-product grid
    name: str = ""

    @property
    def n(self) -> int:
        return self.centre.shape[0]

    @property
    def volume(self) -> np.ndarray:
        return np.prod(self.edge, axis=1)


def grid_tiles(xf, yf, zf, Ms, Aex, Ku, axis=(0.0, 0.0, 1.0), name="") -> Tiles:
    """Tensor-product grid from the face coordinates along each axis
    (``xf`` has nx+1 increasing entries, ...).  Tile (ix, iy, iz) has index
    ix + nx (iy + ny iz) (x fastest)."""
    xf, yf, zf = (np.asarray(a, np.float64) for a in (xf, yf, zf))
    nx, ny, nz = len(xf) - 1, len(yf) - 1, len(zf) - 1
    cx, cy, cz = 0.5 * (xf[1:] + xf[:-1]), 0.5 * (yf[1:] + yf[:-1]), 0.5 * (zf[1:] + zf[:-1])
    ex, ey, ez = np.diff(xf), np.diff(yf), np.diff(zf)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    n = nx * ny * nz
    centre = np.stack([cx[ix], cy[iy], cz[iz]], axis=1)
    edge = np.stack([ex[ix], ey[iy], ez[iz]], axis=1)
    idx = ix + nx * (iy + ny * iz)
    nbr = np.full((n, 6), -1, np.int32)
    nbr[:, 0] = np.where(ix > 0, idx - 1, -1)
    nbr[:, 1] = np.where(ix < nx - 1, idx + 1, -1)
    nbr[:, 2] = np.where(iy > 0, idx - nx, -1)
    nbr[:, 3] = np.where(iy < ny - 1, idx + nx, -1)
    nbr[:, 4] = np.where(iz > 0, idx - nx * ny, -1)
    nbr[:, 5] = np.where(iz < nz - 1, idx + nx * ny, -1)
    ax = np.asarray(axis, np.float64).reshape(-1, 3)
    ax = ax / np.linalg.norm(ax, axis=1, keepdims=True)
    return Tiles(centre=centre, edge=edge,
                 Ms=np.broadcast_to(np.asarray(Ms, np.float64), (n,)).copy(),
                 Aex=np.broadcast_to(np.asarray(Aex, np.float64), (n,)).copy(),
                 Ku=np.broadcast_to(np.asarray(Ku, np.float64), (n,)).copy(),
                 axis=np.broadcast_to(ax, (n, 3)).copy(), nbr=nbr, shape=(nx, ny, nz), name=name)


def film(nx=40, ny=10, nz=1, size=(500e-9, 125e-9, 3e-9), Ms=SP4_MS, Aex=SP4_AEX, Ku=0.0) -> Tiles:
    """Uniform grid of the standard-problem-4 film (Sec. 4.3)."""
    return grid_tiles(np.linspace(0, size[0], nx + 1), np.linspace(0, size[1], ny + 1),
                      np.linspace(0, size[2], nz + 1), Ms, Aex, Ku,
                      name="film_%dx%dx%d" % (nx, ny, nz))


def exchange_length(Ms=SP4_MS, Aex=SP4_AEX) -> float:
    """l_ex = sqrt(A / K_m) with K_m = mu0 Ms^2 / 2 (SI reading of Sec. 4.1)."""
    return math.sqrt(Aex / (0.5 * MU0 * Ms * Ms))


def tetra_box(nx, ny, nz, size=(30e-9, 20e-9, 10e-9), jitter=0.0, seed=0):
    """Tetrahedral tiles filling a box: an nx x ny x nz grid of cells, each
    cut into the 6 tetrahedra of its Kuhn triangulation (all sharing the
    cell diagonal, so the mesh is conforming); interior vertices moved by up
    to `jitter` times the cell size (seeded) for an irregular mesh.  Returns
    (vertices (nv, 3), tets (6 nx ny nz, 4) vertex indices)."""
    gx, gy, gz = (np.linspace(0, L, k + 1) for L, k in zip(size, (nx, ny, nz)))
    Z, Y, X = np.meshgrid(gz, gy, gx, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    if jitter > 0:
        h = np.array([size[0] / nx, size[1] / ny, size[2] / nz])
        u = uniform(seed, 11, verts.size).reshape(-1, 3)
        interior = np.all((verts > 1e-12 * np.array(size)) & (verts < (1 - 1e-12) * np.array(size)), axis=1)
        verts = verts + (interior[:, None] * jitter * h) * u
    idx = lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)
    tets = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
                    p = [0, 0, 0]
                    vs = [idx(i, j, k)]
                    for a in perm:
                        p[a] = 1
                        vs.append(idx(i + p[0], j + p[1], k + p[2]))
                    tets.append(vs)
    return verts, np.array(tets, np.int32)


def sp2_film(nx=100, ny=20, nz=3, d_lex=10.0, Ms=SP4_MS, Aex=SP4_AEX) -> Tiles:
    """Standard problem 2 film (Sec. 4.1): length L, width d = L / 5,
    thickness t = d / 10, with d = d_lex exchange lengths; no anisotropy."""
    d = d_lex * exchange_length(Ms, Aex)
    return film(nx, ny, nz, size=(5.0 * d, d, 0.1 * d), Ms=Ms, Aex=Aex, Ku=0.0)


def sp2_fields(S=4001, h_max=0.08, Ms=SP4_MS) -> np.ndarray:
    """Descending field values of standard problem 2 (Sec. 4.1): from
    +h_max Ms to -h_max Ms in S - 1 equal steps, A/m."""
    return np.linspace(h_max, -h_max, S) * Ms


SP2_DIR = (1.0, 1.0, 1.0)  # the field direction of standard problem 2


def cube(nside=20, L_lex=20.0, Ms=SP4_MS, Aex=SP4_AEX, ku_frac=0.1) -> Tiles:
    """Standard problem 3 cube (Sec. 4.2): edge L_lex exchange lengths,
    K_u = ku_frac * K_m along z."""
    L = L_lex * exchange_length(Ms, Aex)
    f = np.linspace(0, L, nside + 1)
    Km = 0.5 * MU0 * Ms * Ms
    return grid_tiles(f, f, f, Ms, Aex, ku_frac * Km, (0, 0, 1), name="cube_%d" % nside)


def graded_faces(count: int, length: float, seed: int, stream: int) -> np.ndarray:
    """Face coordinates of ``count`` cells with widths h0 * 2^u, u ~ U(-1, 1),
    rescaled to span exactly ``length``."""
    u = uniform(seed, stream, count)
    w = np.power(2.0, u)
    w *= length / w.sum()
    f = np.concatenate([[0.0], np.cumsum(w)])
    f[-1] = length
    return f


def graded_film(nx=200, ny=50, nz=3, size=(1000e-9, 250e-9, 5e-9), seed=0, Ms=SP4_MS,
                Aex=SP4_AEX) -> Tiles:
    """Graded (non-uniform) tensor-product film: no translation invariance."""
    return grid_tiles(graded_faces(nx, size[0], seed, 101), graded_faces(ny, size[1], seed, 102),
                      graded_faces(nz, size[2], seed, 103), Ms, Aex, 0.0,
                      name="graded_%dx%dx%d" % (nx, ny, nz))


# ---------------------------------------------------------------------------
# initial magnetisations
# ---------------------------------------------------------------------------
def _normalise(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def m_noisy(n: int, direction=(1.0, 1.0, 1.0), noise=1e-3, seed=0, stream=1) -> np.ndarray:
    """normalise(d/|d| + noise * xi), xi uniform in [-1,1)^3 per tile."""
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    xi = uniform(seed, stream, 3 * n).reshape(n, 3)
    return _normalise(d[None, :] + noise * xi)


def m_random(n: int, seed=1, stream=2) -> np.ndarray:
    """Random unit vectors (normalised cube samples, tiles uniform in [-1,1)^3)."""
    xi = uniform(seed, stream, 3 * n).reshape(n, 3)
    xi[np.linalg.norm(xi, axis=1) < 1e-3] += 0.5
    return _normalise(xi)


def m_flower(t: Tiles, seed=0) -> np.ndarray:
    return m_noisy(t.n, (0, 0, 1), 0.1, seed, 3)


def m_vortex(t: Tiles, core_lex=1.0, axis=2) -> np.ndarray:
    """Vortex seed: m circulates about the line through the body's centre
    along coordinate `axis` (0, 1, 2 = x, y, z), with a core of radius
    core_lex exchange lengths pointing along +axis."""
    c = t.centre - t.centre.mean(0)
    u, v = (axis + 1) % 3, (axis + 2) % 3
    rc = core_lex * exchange_length(float(t.Ms[0]), float(t.Aex[0]))
    rho2 = c[:, u] ** 2 + c[:, v] ** 2
    m = np.zeros_like(c)
    m[:, u] = -c[:, v]
    m[:, v] = c[:, u]
    m[:, axis] = rc * np.exp(-rho2 / (rc * rc))
    return _normalise(m)


# ---------------------------------------------------------------------------
# batched field sweep (hysteresis points) and serving streams
# ---------------------------------------------------------------------------
def sweep_fields(B=64, h_max_mT=50.0, seed=0):
    """B applied fields mu0 H_b = (h_max - 2 h_max b/(B-1)) mT along one
    seeded in-plane direction; returns (Ha (B,3) in A/m, unit direction)."""
    theta = math.pi * (uniform(seed, 7, 1)[0] + 1.0)
    d = np.array([math.cos(theta), math.sin(theta), 0.0])
    b = np.arange(B, dtype=np.float64)
    mu0h = (h_max_mT - 2.0 * h_max_mT * b / max(B - 1, 1)) * 1e-3
    return (mu0h[:, None] * d[None, :]) / MU0, d


def sweep_alphas(B=64, values=(0.02, 0.1, 0.5)):
    return np.array([values[b % len(values)] for b in range(B)], np.float64)


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    geometry: int
    Ha: np.ndarray       # (3,) A/m
    m0_seed: int


def serving_geometries(count=12, n_min=500, n_max=40000, seed=0):
    """Film and prism geometries with n log-uniform in [n_min, n_max]."""
    out = []
    for g in range(count):
        u = unit01(seed, 200 + g, 4)
        n_target = math.exp(math.log(n_min) + u[0] * (math.log(n_max) - math.log(n_min)))
        Ms = 4e5 + u[1] * 8e5
        if g % 2 == 0:
            # film: thickness 3 nm (one layer), aspect 4:1 in plane, ~cubic-ish tiles
            ny = max(1, int(round(math.sqrt(n_target / 4.0))))
            nx = max(1, int(round(n_target / ny)))
            h = 2.5e-9 + 2.5e-9 * u[2]
            t = grid_tiles(np.linspace(0, nx * h, nx + 1), np.linspace(0, ny * h, ny + 1),
                           np.linspace(0, 3e-9, 2), Ms, SP4_AEX, 0.0, name="film%d" % g)
        else:
            a = 1.0 + u[3]  # aspect <= 2
            nz = max(1, int(round((n_target / a) ** (1.0 / 3.0))))
            ny = nz
            nx = max(1, int(round(n_target / (ny * nz))))
            h = 3e-9 + 2e-9 * u[2]
            t = grid_tiles(np.linspace(0, nx * h, nx + 1), np.linspace(0, ny * h, ny + 1),
                           np.linspace(0, nz * h, nz + 1), Ms, SP4_AEX, 0.0, name="prism%d" % g)
        out.append(t)
    return out


def serving_requests(count=2000, rate_hz=200.0, n_geom=12, seed=0, h_max_mT=100.0):
    """Poisson arrivals; geometry uniform over n_geom; mu0 H uniform in the
    ball |mu0 H| <= h_max_mT; each request seeds its own random m0."""
    u = unit01(seed, 300, 6 * count)
    reqs = []
    t = 0.0
    for r in range(count):
        a = u[6 * r:6 * r + 6]
        t += -math.log(max(1.0 - a[0], 1e-300)) / rate_hz
        g = min(int(a[1] * n_geom), n_geom - 1)
        # uniform in the ball: direction from two uniforms, radius ~ cbrt(u)
        cz = 2.0 * a[2] - 1.0
        ph = 2.0 * math.pi * a[3]
        s = math.sqrt(max(0.0, 1.0 - cz * cz))
        rad = h_max_mT * 1e-3 * a[4] ** (1.0 / 3.0)
        Ha = rad * np.array([s * math.cos(ph), s * math.sin(ph), cz]) / MU0
        reqs.append(Request(r, t, g, Ha, 1000 + r))
    return reqs
