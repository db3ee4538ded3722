// Tensor assembly (FP64) and packing into the tile-blocked storage.
//
// Sec. 3 of the paper: the field of every uniformly magnetised cuboid or
// tetrahedral tile is evaluated analytically at the centre of every other tile; the tensor is
// computed once, at the start (Sec. 3.1), and stored in a reduced precision
// (FP32 in the paper, Sec. 3.2).  One thread evaluates one 3x3 block in FP64
// and stores its 6 unique entries directly in the requested precision.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "mt_internal.cuh"

namespace {

// Tensor of the cuboid (centre c, full edges e) at the point r, from the
// Newtonian potential Phi of the box:  N = -(1/4 pi) grad grad Phi, so that
// H = -N M.  Faces are numbered low (0) / high (1) on each axis; a corner's
// sign is s = -(-1)^(f_x + f_y + f_z): +1 when an odd number of its faces are
// high faces.
//   N_xx = -(1/4 pi) sum_corners s atan(dy dz / (dx R))
//   N_xy = +(1/4 pi) sum_corners s log(dz + R)         (xz: dy, yz: dx)
// dx == 0 (point in a face plane, outside the face): the arctan term is 0,
// its +-pi/2 limits cancel between corners.  A log pair whose two offsets
// are both negative is rewritten with log(R - d), exact and free of the
// cancellation of d + R when the point lies far on the negative side.
struct Corners {
  double d[3][2];  // offsets r - face, [axis][face]
  double R[8];     // corner distance, index fx | fy << 1 | fz << 2
};

__device__ __forceinline__ double atan_ratio(double num_a, double num_b, double den, double R) {
  return den == 0.0 ? 0.0 : atan((num_a * num_b) / (den * R));
}

// log(dp + Rp) - log(dm + Rm) for the two faces (m = low face, p = high face)
// of one axis, with the fixed other two corner coordinates.
__device__ __forceinline__ double log_diff(double dm, double Rm, double dp, double Rp) {
  if (dm < 0.0 && dp < 0.0) return log(Rm - dm) - log(Rp - dp);
  return log(dp + Rp) - log(dm + Rm);
}

__device__ void cuboid_tensor(const double *r, const double *c, const double *e, double out[6]) {
  Corners K;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    K.d[a][0] = r[a] - (c[a] - 0.5 * e[a]);
    K.d[a][1] = r[a] - (c[a] + 0.5 * e[a]);
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double x = K.d[0][q & 1], y = K.d[1][(q >> 1) & 1], z = K.d[2][(q >> 2) & 1];
    K.R[q] = sqrt(x * x + y * y + z * z);
  }
  double txx = 0.0, tyy = 0.0, tzz = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double s = (__popc(q) & 1) ? 1.0 : -1.0;
    const double x = K.d[0][q & 1], y = K.d[1][(q >> 1) & 1], z = K.d[2][(q >> 2) & 1];
    txx += s * atan_ratio(y, z, x, K.R[q]);
    tyy += s * atan_ratio(x, z, y, K.R[q]);
    tzz += s * atan_ratio(x, y, z, K.R[q]);
  }
  // Off-diagonal entries: pair the two faces of the log's axis.  For a pair
  // with the other two faces (f1, f2) fixed, the corner with the low face
  // has sign s_lo = -(-1)^(f1+f2) and the high-face corner -s_lo, so the pair
  // contributes s_lo (log(d_lo + R_lo) - log(d_hi + R_hi)) = -s_lo log_diff.
  double txy = 0.0, txz = 0.0, tyz = 0.0;
#pragma unroll
  for (int f1 = 0; f1 < 2; ++f1) {
#pragma unroll
    for (int f2 = 0; f2 < 2; ++f2) {
      const double s_lo = ((f1 + f2) & 1) ? 1.0 : -1.0;
      // xy: log axis z, fixed (fx = f1, fy = f2)
      txy -= s_lo * log_diff(K.d[2][0], K.R[f1 | (f2 << 1)], K.d[2][1], K.R[f1 | (f2 << 1) | 4]);
      // xz: log axis y, fixed (fx = f1, fz = f2)
      txz -= s_lo * log_diff(K.d[1][0], K.R[f1 | (f2 << 2)], K.d[1][1], K.R[f1 | 2 | (f2 << 2)]);
      // yz: log axis x, fixed (fy = f1, fz = f2)
      tyz -= s_lo * log_diff(K.d[0][0], K.R[(f1 << 1) | (f2 << 2)], K.d[0][1], K.R[1 | (f1 << 1) | (f2 << 2)]);
    }
  }
  const double k = 0.25 / MT_PI;
  out[0] = -k * txx;
  out[1] = k * txy;
  out[2] = k * txz;
  out[3] = -k * tyy;
  out[4] = k * tyz;
  out[5] = -k * tzz;
}

// Tensor of a uniformly magnetised tetrahedron (vertices v[4][3]) at r.
// The body's field is that of its face charges sigma_f = M.n_f, so with
// H = -N M,  N = (1/4 pi) sum_f g_f n_f^T,  g_f = grad_r int_f dS / |r - r'|.
// For a plane triangle the gradient splits into a part along n_f, -n_f times
// the solid angle under which the face is seen (signed like the height of r
// above the face), and an in-plane part from the 2-D divergence theorem:
// minus the sum over the edges of the edge's outward in-plane normal times
// int_edge dl / |r - r'|.  Solid angle: atan2 form of Van Oosterom and
// Strackee (1983); edge integral: log((R_b + s_b) / (R_a + s_a)) with s the
// projections on the edge direction, or the equal log((R_a - s_a) /
// (R_b - s_b)) where the first would cancel.  FP64 throughout.
__device__ __forceinline__ void sub3(const double *a, const double *b, double *c) {
  c[0] = a[0] - b[0];
  c[1] = a[1] - b[1];
  c[2] = a[2] - b[2];
}
__device__ __forceinline__ double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ void crs3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ void tetra_tensor(const double *r, const double *v, double out[6]) {
  double N[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll 1
  for (int f = 0; f < 4; ++f) {
    // face (a, b, c) opposite vertex f, made counter-clockwise about its
    // outward normal
    const int ia = f == 0 ? 1 : 0;
    const int ib = f <= 1 ? 2 : 1;
    const int ic = f <= 2 ? 3 : 2;
    const double *A = v + 3 * ia, *Bv = v + 3 * ib, *C = v + 3 * ic;
    double ab[3], ac[3], nf[3], to_f[3];
    sub3(Bv, A, ab);
    sub3(C, A, ac);
    crs3(ab, ac, nf);
    sub3(v + 3 * f, A, to_f);
    if (dot3(nf, to_f) > 0.0) {
      const double *t = Bv;
      Bv = C;
      C = t;
      nf[0] = -nf[0];
      nf[1] = -nf[1];
      nf[2] = -nf[2];
    }
    const double inv = 1.0 / sqrt(dot3(nf, nf));
    nf[0] *= inv;
    nf[1] *= inv;
    nf[2] *= inv;
    double ra[3], rb[3], rc[3], bxc[3];
    sub3(A, r, ra);
    sub3(Bv, r, rb);
    sub3(C, r, rc);
    crs3(rb, rc, bxc);
    const double la = sqrt(dot3(ra, ra)), lb = sqrt(dot3(rb, rb)), lc = sqrt(dot3(rc, rc));
    const double omega = -2.0 * atan2(dot3(ra, bxc), la * lb * lc + dot3(ra, rb) * lc + dot3(ra, rc) * lb +
                                                         dot3(rb, rc) * la);
    double g[3] = {-omega * nf[0], -omega * nf[1], -omega * nf[2]};
    const double *P[3] = {A, Bv, C};
    const double *Rv[3] = {ra, rb, rc};
    const double L[3] = {la, lb, lc};
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int e2 = (e + 1) % 3;
      double t[3], u[3];
      sub3(P[e2], P[e], t);
      const double len = sqrt(dot3(t, t));
      t[0] /= len;
      t[1] /= len;
      t[2] /= len;
      crs3(t, nf, u);  // in-plane, out of the face
      const double s1 = dot3(Rv[e], t), s2 = dot3(Rv[e2], t);
      const double li = (s1 + s2 >= 0.0) ? log((L[e2] + s2) / (L[e] + s1)) : log((L[e] - s1) / (L[e2] - s2));
      g[0] -= u[0] * li;
      g[1] -= u[1] * li;
      g[2] -= u[2] * li;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) N[a][b] += g[a] * nf[b];
  }
  const double k = 0.25 / MT_PI;
  out[0] = k * N[0][0];
  out[1] = 0.5 * k * (N[0][1] + N[1][0]);
  out[2] = 0.5 * k * (N[0][2] + N[2][0]);
  out[3] = k * N[1][1];
  out[4] = 0.5 * k * (N[1][2] + N[2][1]);
  out[5] = k * N[2][2];
}

// One block per lattice offset (dx, dy, dz): the tensor of the tile at the
// origin seen from (dx ex, dy ey, dz ez).  Index ((dx + Lx - 1)(2Ly - 1) +
// dy + Ly - 1)(2Lz - 1) + dz + Lz - 1.
__global__ void k_offset_table(int Lx, int Ly, int Lz, double ex, double ey, double ez, double *table) {
  const int64_t Ny = 2 * Ly - 1, Nz = 2 * Lz - 1;
  const int64_t tot = (int64_t)(2 * Lx - 1) * Ny * Nz;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= tot) return;
  const int dz = (int)(t % Nz) - (Lz - 1);
  const int dy = (int)((t / Nz) % Ny) - (Ly - 1);
  const int dx = (int)(t / (Ny * Nz)) - (Lx - 1);
  const double r[3] = {dx * ex, dy * ey, dz * ez};
  const double c[3] = {0.0, 0.0, 0.0};
  const double e[3] = {ex, ey, ez};
  cuboid_tensor(r, c, e, table + 6 * t);
}

// Relations of tetrahedra i and j (i != j), as pair_relation: bit 0 = the
// centroid of i lies in or on tetrahedron j (barycentric coordinates all
// >= -eps), bit 1 = they share a vertex (a "near" pair).
__device__ int tetra_relation(const double *ci, const double *vi, const double *vj) {
  bool touch = false;
#pragma unroll 1
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      touch = touch || (vi[3 * a] == vj[3 * b] && vi[3 * a + 1] == vj[3 * b + 1] && vi[3 * a + 2] == vj[3 * b + 2]);
  // barycentric coordinates of ci in j: solve [v1-v0, v2-v0, v3-v0] x = ci - v0
  double e1[3], e2[3], e3[3], d[3], c23[3], c31[3], c12[3];
  sub3(vj + 3, vj, e1);
  sub3(vj + 6, vj, e2);
  sub3(vj + 9, vj, e3);
  sub3(ci, vj, d);
  crs3(e2, e3, c23);
  crs3(e3, e1, c31);
  crs3(e1, e2, c12);
  const double det = dot3(e1, c23);
  const double x = dot3(d, c23) / det, y = dot3(d, c31) / det, z = dot3(d, c12) / det;
  const double eps = 1e-12;
  const bool in = x >= -eps && y >= -eps && z >= -eps && (1.0 - x - y - z) >= -eps;
  return (in ? 1 : 0) | (touch ? 2 : 0);
}

// Geometry relations of tiles i and j (i != j): bit 0 = volumes overlap or
// the centre of i lies in/on tile j (invalid), bit 1 = the closed boxes touch
// (a "near" pair, kept in FP64 for the BF16 precisions).
__device__ __forceinline__ int pair_relation(const double *ci, const double *ei, const double *cj,
                                             const double *ej) {
  bool vol = true, pt = true, touch = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double d = fabs(ci[a] - cj[a]);
    const double half = 0.5 * (ei[a] + ej[a]);
    const double tol = 1e-12 * (ei[a] + ej[a]);
    vol = vol && (d < half - tol);
    pt = pt && (d <= 0.5 * ej[a] + tol);
    touch = touch && (d <= half * (1.0 + 1e-9));
  }
  return ((vol || pt) ? 1 : 0) | (touch ? 2 : 0);
}

__device__ __forceinline__ int64_t scale_index(int64_t i, int64_t j, int TR, int TC, int64_t Q) {
  const int64_t p = i / TR, q = j / TC;
  const int r = (int)(i - p * TR), c = (int)(j - q * TC);
  return ((p * Q + q) * TR + r) * (int64_t)TC + c;
}

struct AsmArgs {
  const double *centre, *edge;
  const double *vert;  // 12n, tetrahedral tiles
  int kind;            // MT_TILE_CUBOID / MT_TILE_TETRA
  // uniform lattice: block (i, j) = table[offset lat_i - lat_j] (nullptr: evaluate)
  const double *table;
  const int32_t *lat;
  int Lx, Ly, Lz;
  int64_t n;
  int TR, TC, nplane;
  int64_t Q;
  int prec;
  void *data;
  int8_t *scale;
  int *bad;           // set to 1 on overlap
  int *planar_bad;    // set to 1 if a 4- or 3-plane (single-layer) tensor meets |N_xz| or |N_yz| >
                      // kPlanarTol, or (3 or 5 planes) a block's trace off delta_ij by more than kTraceTol
  int dense;          // 1: 9-entry row-major matrix (Kp x Kp), else tile-blocked
  int half;           // 1: streaming FP32 tensor of one tile shape, upper triangle of chunks only
  int64_t Kp;
  int *near_fill;     // per-row fill counter (BF16 precisions)
  const int32_t *near_ptr;
  int32_t *near_col;
  double *near_val;
  int count_only;     // 1: only count near blocks per row into near_fill
};

// grid (Q, P); TC threads; thread = column j of the chunk, loop over the
// panel's TR rows i.
__global__ void k_assemble(AsmArgs A) {
  const int64_t q = blockIdx.x, p = blockIdx.y;
  const int64_t j = q * A.TC + threadIdx.x;
  if (j >= A.n) return;
  const bool tet = A.kind == MT_TILE_TETRA;
  double cj[3], ej[3], vj[12];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cj[a] = A.centre[3 * j + a];
    ej[a] = A.edge[3 * j + a];
  }
  if (tet)
#pragma unroll
    for (int a = 0; a < 12; ++a) vj[a] = A.vert[12 * j + a];
  for (int r = 0; r < A.TR; ++r) {
    const int64_t i = p * A.TR + r;
    if (i >= A.n) break;
    double ci[3], ei[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ci[a] = A.centre[3 * i + a];
      ei[a] = A.edge[3 * i + a];
    }
    int rel;
    int64_t toff = 0;
    if (A.table) {
      // lattice: the offset decides everything (a repeated index = overlap,
      // touching = at most one step on every axis)
      const int dx = A.lat[3 * i] - A.lat[3 * j], dy = A.lat[3 * i + 1] - A.lat[3 * j + 1];
      const int dz = A.lat[3 * i + 2] - A.lat[3 * j + 2];
      const bool same = dx == 0 && dy == 0 && dz == 0;
      const bool touch = dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1;
      rel = (i == j) ? 2 : ((same ? 1 : 0) | (touch ? 2 : 0));
      toff = ((int64_t)(dx + A.Lx - 1) * (2 * A.Ly - 1) + (dy + A.Ly - 1)) * (2 * A.Lz - 1) + (dz + A.Lz - 1);
    } else {
      rel = (i == j) ? 2 : tet ? tetra_relation(ci, A.vert + 12 * i, vj) : pair_relation(ci, ei, cj, ej);
    }
    if (rel & 1) atomicExch(A.bad, 1);
    // half storage: block (i, j) of an omitted chunk is block (j, i), which
    // its own chunk stores (the relation above is still checked for all pairs)
    if (A.half && half_q0(p, A.TC / A.TR) > q) continue;
    const bool near = (rel & 2) && (A.prec == MT_BF16_SCALED || A.prec == MT_BF16_SPLIT);
    if (A.count_only) {
      if (near) atomicAdd(&A.near_fill[i], 1);
      continue;
    }
    double N6[6];
    if (A.table) {
#pragma unroll
      for (int e = 0; e < 6; ++e) N6[e] = A.table[6 * toff + e];
    } else if (tet) {
      tetra_tensor(ci, vj, N6);
    } else {
      cuboid_tensor(ci, cj, ej, N6);
    }
    if (near) {
      const int slot = atomicAdd(&A.near_fill[i], 1);
      const int64_t at = A.near_ptr[i] + slot;
      A.near_col[at] = (int32_t)j;
#pragma unroll
      for (int e = 0; e < 6; ++e) A.near_val[6 * at + e] = N6[e];
      continue;  // dense store keeps zeros there
    }
    if (A.dense) {
      // all 9 entries: row 3i + a, column 3j + b (scales fixed to 1)
      __nv_bfloat16 *D = (__nv_bfloat16 *)A.data;
      const size_t plane = (size_t)A.Kp * A.Kp;
      const int e_of[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const double v = N6[e_of[a][b]];
          const size_t at = dense_a_index(3 * i + a, 3 * j + b, A.Kp / 64);
          const __nv_bfloat16 hi = __double2bfloat16(v);
          D[at] = hi;
          if (A.prec == MT_BF16_SPLIT) D[plane + at] = __double2bfloat16(v - (double)__bfloat162float(hi));
        }
      continue;
    }
    switch (A.prec) {
      case MT_F64: {
        double *D = (double *)A.data;
#pragma unroll
        for (int e = 0; e < 6; ++e) D[layout_index(i, j, e, A.TR, A.TC, 6, A.Q)] = N6[e];
      } break;
      case MT_F32: {
        float *D = (float *)A.data;
#pragma unroll
        for (int e = 0; e < 6; ++e) {
          const int pl = stream_plane(e, A.nplane);
          if (pl >= 0) D[layout_index_h(i, j, pl, A.TR, A.TC, A.nplane, A.Q, A.half)] = (float)N6[e];
          else if (traceless(A.nplane) && e == 5) {
            // zz is not stored: the identity that gives it must hold here
            const double tr = N6[0] + N6[3] + N6[5] - (i == j ? 1.0 : 0.0);
            if (!(fabs(tr) <= kTraceTol * (fabs(N6[0]) + fabs(N6[3]) + fabs(N6[5])) + kPlanarTol))
              *A.planar_bad = 1;
          } else if (!(fabs(N6[e]) <= kPlanarTol)) *A.planar_bad = 1;
        }
      } break;
      case MT_BF16_SCALED: {
        // power-of-two scale of the block: 2^s with s = exponent of max |N|
        double mx = 0.0;
#pragma unroll
        for (int e = 0; e < 6; ++e) mx = fmax(mx, fabs(N6[e]));
        int s = 0;
        if (mx > 0.0) {
          frexp(mx, &s);
          s = max(-126, min(126, s));
        }
        __nv_bfloat16 *D = (__nv_bfloat16 *)A.data;
#pragma unroll
        for (int e = 0; e < 6; ++e) {
          const int pl = stream_plane(e, A.nplane);
          if (pl >= 0) D[layout_index(i, j, pl, A.TR, A.TC, A.nplane, A.Q)] = __double2bfloat16(ldexp(N6[e], -s));
          else if (!(fabs(N6[e]) <= kPlanarTol)) *A.planar_bad = 1;
        }
        A.scale[scale_index(i, j, A.TR, A.TC, A.Q)] = (int8_t)s;
      } break;
      case MT_BF16_SPLIT: {
        __nv_bfloat16 *D = (__nv_bfloat16 *)A.data;
#pragma unroll
        const int half = A.nplane / 2;  // hi planes, then as many lo planes
        for (int e = 0; e < 6; ++e) {
          const int pl = stream_plane(e, half);
          if (pl < 0) {
            if (!(fabs(N6[e]) <= kPlanarTol)) *A.planar_bad = 1;
            continue;
          }
          const __nv_bfloat16 hi = __double2bfloat16(N6[e]);
          const __nv_bfloat16 lo = __double2bfloat16(N6[e] - (double)__bfloat162float(hi));
          D[layout_index(i, j, pl, A.TR, A.TC, A.nplane, A.Q)] = hi;
          D[layout_index(i, j, half + pl, A.TR, A.TC, A.nplane, A.Q)] = lo;
        }
      } break;
    }
  }
}

// sort each row's near blocks by column so that the FP64 near sum has a
// fixed order (one thread per row; rows hold at most 27 entries for cuboid
// grids, a few dozen for tetrahedral meshes)
__global__ void k_sort_near(int64_t n, const int32_t *ptr, int32_t *col, double *val) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t b = ptr[i], e = ptr[i + 1];
  for (int32_t a = b + 1; a < e; ++a) {
    const int32_t cj = col[a];
    double v[6];
    for (int q = 0; q < 6; ++q) v[q] = val[6 * a + q];
    int32_t z = a - 1;
    while (z >= b && col[z] > cj) {
      col[z + 1] = col[z];
      for (int q = 0; q < 6; ++q) val[6 * (z + 1) + q] = val[6 * z + q];
      --z;
    }
    col[z + 1] = cj;
    for (int q = 0; q < 6; ++q) val[6 * (z + 1) + q] = v[q];
  }
}

// near blocks times the source tile's Ms as FP32 hi + lo pairs
// (N_ij Ms_j = hi + lo to ~2^-48 relative; Ms_j as the FP32 value every
// product uses), so that the near product multiplies plain m
__global__ void k_near_split(int64_t count6, const double *val, const int32_t *col, const float *Ms, float2 *hl) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count6) return;
  const double v = val[t] * (double)Ms[col[t / 6]];
  const float hi = (float)v;
  hl[t] = make_float2(hi, (float)(v - (double)hi));
}

__global__ void k_blocks(const double *centre, const double *edge, const double *vert, int kind, int64_t count,
                         const int64_t *pairs, double *out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= count) return;
  const int64_t i = pairs[2 * p], j = pairs[2 * p + 1];
  if (kind == MT_TILE_TETRA)
    tetra_tensor(&centre[3 * i], &vert[12 * j], &out[6 * p]);
  else
    cuboid_tensor(&centre[3 * i], &centre[3 * j], &edge[3 * j], &out[6 * p]);
}

// stored value -> double, rows [i0, i1), all columns; out[((i-i0)*n + j)*6 + e]
__global__ void k_read_rows(const void *data, const int8_t *scale, int prec, int64_t n, int TR, int TC,
                            int nplane, int64_t Q, bool hs, int64_t i0, int64_t i1, double *out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t rows = i1 - i0;
  if (t >= rows * n) return;
  const int64_t i = i0 + t / n, j = t % n;
  for (int e = 0; e < 6; ++e) {
    double v = 0.0;
    switch (prec) {
      case MT_F64: v = ((const double *)data)[layout_index(i, j, e, TR, TC, 6, Q)]; break;
      case MT_F32: {
        auto stored = [&](int ee) {
          const int pl = stream_plane(ee, nplane);
          int64_t at = pl < 0 ? -1 : layout_index_h(i, j, pl, TR, TC, nplane, Q, hs);
          if (pl >= 0 && at < 0) at = layout_index_h(j, i, pl, TR, TC, nplane, Q, hs);  // N_ij = N_ji
          return pl < 0 ? 0.0 : (double)((const float *)data)[at];
        };
        if (traceless(nplane) && e == 5)  // zz from the trace: delta_ij - xx - yy of the stored values, in FP32
          v = (double)((i == j ? 1.0f : 0.0f) - ((float)stored(0) + (float)stored(3)));
        else
          v = stored(e);
      } break;
      case MT_BF16_SCALED: {
        const int pl = stream_plane(e, nplane);
        v = pl < 0 ? 0.0
                   : ldexp((double)__bfloat162float(
                               ((const __nv_bfloat16 *)data)[layout_index(i, j, pl, TR, TC, nplane, Q)]),
                           (int)scale[scale_index(i, j, TR, TC, Q)]);
      } break;
      case MT_BF16_SPLIT: {
        const int half = nplane / 2, pl = stream_plane(e, half);
        const __nv_bfloat16 *d = (const __nv_bfloat16 *)data;
        v = pl < 0 ? 0.0
                   : (double)__bfloat162float(d[layout_index(i, j, pl, TR, TC, nplane, Q)]) +
                         (double)__bfloat162float(d[layout_index(i, j, half + pl, TR, TC, nplane, Q)]);
      } break;
    }
    out[t * 6 + e] = v;
  }
}

// dense layout -> double, rows [i0, i1)
__global__ void k_read_rows_dense(const __nv_bfloat16 *D, int split, int64_t n, int64_t Kp, int64_t i0, int64_t i1,
                                  double *out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t rows = i1 - i0;
  if (t >= rows * n) return;
  const int64_t i = i0 + t / n, j = t % n;
  const int ra[6] = {0, 0, 0, 1, 1, 2}, cb[6] = {0, 1, 2, 1, 2, 2};
  const size_t plane = (size_t)Kp * Kp;
  for (int e = 0; e < 6; ++e) {
    const size_t at = dense_a_index(3 * i + ra[e], 3 * j + cb[e], Kp / 64);
    double v = (double)__bfloat162float(D[at]);
    if (split) v += (double)__bfloat162float(D[plane + at]);
    out[t * 6 + e] = v;
  }
}

// merge the FP64 near blocks of rows [i0, i1) into out
__global__ void k_merge_near(int64_t n, int64_t i0, int64_t i1, const int32_t *ptr, const int32_t *col,
                             const double *val, double *out) {
  const int64_t i = i0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= i1) return;
  for (int32_t a = ptr[i]; a < ptr[i + 1]; ++a) {
    const int64_t j = col[a];
    for (int e = 0; e < 6; ++e) out[((i - i0) * n + j) * 6 + e] = val[6 * a + e];
  }
}

}  // namespace

namespace mt {

mt_status assemble(mt_tensor *T) {
  mt_tiles *t = T->tiles;
  const int64_t n = T->n;
  const mt_layout &L = T->L;
  DevTemp<int> bad_flag;
  MT_CUDA(bad_flag.alloc(2));
  int *d_bad = bad_flag.p;
  MT_CUDA(cudaMemset(d_bad, 0, 2 * sizeof(int)));
  AsmArgs A{};
  A.centre = t->d_centre;
  A.edge = t->d_edge;
  A.vert = t->d_vert;
  A.kind = t->kind;
  A.n = n;
  A.TR = L.TR;
  A.TC = L.TC;
  A.nplane = L.nplane;
  A.Q = L.Q;
  A.prec = T->prec;
  A.data = T->d_data;
  A.scale = T->d_scale;
  A.bad = d_bad;
  A.planar_bad = d_bad + 1;
  A.dense = T->layout == MT_LAYOUT_DENSE;
  A.half = T->L.half ? 1 : 0;
  A.Kp = T->Kp;
  DevTemp<double> table;
  double *d_table = nullptr;
  if (t->lattice && t->kind == MT_TILE_CUBOID) {
    const int64_t cnt = (int64_t)(2 * t->Lx - 1) * (2 * t->Ly - 1) * (2 * t->Lz - 1);
    MT_CUDA(table.alloc(6 * cnt));
    d_table = table.p;
    k_offset_table<<<(unsigned)((cnt + 127) / 128), 128>>>(t->Lx, t->Ly, t->Lz, t->lat_edge[0], t->lat_edge[1],
                                                          t->lat_edge[2], d_table);
    MT_CUDA(cudaGetLastError());
    A.table = d_table;
    A.lat = t->d_lat;
    A.Lx = t->Lx;
    A.Ly = t->Ly;
    A.Lz = t->Lz;
  }
  const bool has_near = (T->prec == MT_BF16_SCALED || T->prec == MT_BF16_SPLIT);
  dim3 grid((unsigned)L.Q, (unsigned)L.P);
  if (has_near) {
    DevTemp<int> fill;
    MT_CUDA(fill.alloc(n));
    int *d_fill = fill.p;
    MT_CUDA(cudaMemset(d_fill, 0, sizeof(int) * n));
    A.near_fill = d_fill;
    A.count_only = 1;
    k_assemble<<<grid, L.TC>>>(A);
    MT_CUDA(cudaGetLastError());
    std::vector<int> cnt(n);
    MT_CUDA(cudaMemcpy(cnt.data(), d_fill, sizeof(int) * n, cudaMemcpyDeviceToHost));
    std::vector<int32_t> ptr(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) ptr[i + 1] = ptr[i] + cnt[i];
    T->near_count = ptr[n];
    MT_CUDA(cudaMalloc(&T->d_near_ptr, sizeof(int32_t) * (n + 1)));
    MT_CUDA(cudaMalloc(&T->d_near_col, sizeof(int32_t) * std::max<int64_t>(1, T->near_count)));
    MT_CUDA(cudaMalloc(&T->d_near_val, sizeof(double) * 6 * std::max<int64_t>(1, T->near_count)));
    MT_CUDA(cudaMemcpy(T->d_near_ptr, ptr.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice));
    MT_CUDA(cudaMemset(d_fill, 0, sizeof(int) * n));
    A.near_ptr = T->d_near_ptr;
    A.near_col = T->d_near_col;
    A.near_val = T->d_near_val;
    A.count_only = 0;
    k_assemble<<<grid, L.TC>>>(A);
    MT_CUDA(cudaGetLastError());
    k_sort_near<<<(unsigned)((n + 127) / 128), 128>>>(n, T->d_near_ptr, T->d_near_col, T->d_near_val);
    MT_CUDA(cudaGetLastError());
    const int64_t c6 = 6 * std::max<int64_t>(1, T->near_count);
    MT_CUDA(cudaMalloc(&T->d_near_hl, sizeof(float2) * c6));
    if (T->near_count > 0) {
      k_near_split<<<(unsigned)((6 * T->near_count + 255) / 256), 256>>>(6 * T->near_count, T->d_near_val,
                                                                        T->d_near_col, t->d_Ms, T->d_near_hl);
      MT_CUDA(cudaGetLastError());
    }
    MT_CUDA(cudaDeviceSynchronize());
  } else {
    k_assemble<<<grid, L.TC>>>(A);
    MT_CUDA(cudaGetLastError());
    MT_CUDA(cudaDeviceSynchronize());
  }
  int bad[2] = {0, 0};
  MT_CUDA(cudaMemcpy(bad, d_bad, 2 * sizeof(int), cudaMemcpyDeviceToHost));
  MT_CHECK(!bad[0], MT_EOVERLAP, "mt_demag_assemble: tiles overlap or a tile centre lies on another tile");
  if (bad[1] && (T->L.nplane == 4 || traceless(T->L.nplane))) {
    // an xz or yz entry of the single-layer set is not round-off, or (3
    // planes) a block's trace is off its identity: store all 6 planes after
    // all (within the budget reserved for them)
    mt_ctx *ctx = t->ctx;
    const bool half = T->L.half;
    layout_for(T->prec, &T->L);
    T->L.P = (n + T->L.TR - 1) / T->L.TR;
    T->L.Q = (n + T->L.TC - 1) / T->L.TC;
    T->L.half = half;
    T->L.CH = half ? half_chunks(T->L.P, T->L.Q, T->L.TC / T->L.TR) : T->L.P * T->L.Q;
    const size_t bytes = (size_t)T->L.CH * (T->L.chunk_bytes() + T->L.scale_bytes_per_chunk);
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      MT_CHECK(ctx->in_use - T->bytes + bytes <= ctx->budget, MT_ENOMEM,
               "mt_demag_assemble: %zu bytes exceed the context budget", bytes);
      ctx->in_use += bytes - T->bytes;
      T->bytes = bytes;
    }
    const size_t data_bytes = (size_t)T->L.CH * T->L.chunk_bytes();
    MT_CUDA(cudaFree(T->d_data));
    T->d_data = nullptr;
    MT_CUDA(cudaMalloc(&T->d_data, data_bytes));
    MT_CUDA(cudaMemset(T->d_data, 0, data_bytes));
    A.data = T->d_data;
    A.TR = T->L.TR;
    A.TC = T->L.TC;
    A.nplane = T->L.nplane;
    A.Q = T->L.Q;
    k_assemble<<<dim3((unsigned)T->L.Q, (unsigned)T->L.P), T->L.TC>>>(A);
    MT_CUDA(cudaGetLastError());
    MT_CUDA(cudaDeviceSynchronize());
  }
  return MT_OK;
}

mt_status blocks_fp64(mt_tiles *t, int64_t count, const int64_t *pairs, double *out) {
  if (count == 0) return MT_OK;
  for (int64_t p = 0; p < 2 * count; ++p)
    MT_CHECK(pairs[p] >= 0 && pairs[p] < t->n, MT_EINVAL, "mt_demag_blocks: pair index out of range");
  int64_t *d_pairs = nullptr;
  double *d_out = nullptr;
  MT_CUDA(cudaMalloc(&d_pairs, sizeof(int64_t) * 2 * count));
  MT_CUDA(cudaMalloc(&d_out, sizeof(double) * 6 * count));
  MT_CUDA(cudaMemcpy(d_pairs, pairs, sizeof(int64_t) * 2 * count, cudaMemcpyHostToDevice));
  k_blocks<<<(unsigned)((count + 127) / 128), 128>>>(t->d_centre, t->d_edge, t->d_vert, t->kind, count, d_pairs,
                                                     d_out);
  MT_CUDA(cudaGetLastError());
  MT_CUDA(cudaMemcpy(out, d_out, sizeof(double) * 6 * count, cudaMemcpyDeviceToHost));
  cudaFree(d_pairs);
  cudaFree(d_out);
  return MT_OK;
}

mt_status read_rows(const mt_tensor *T, int64_t i0, int64_t i1, double *out) {
  const int64_t n = T->n;
  const int64_t rows = i1 - i0;
  if (rows <= 0) return MT_OK;
  double *d_out = nullptr;
  MT_CUDA(cudaMalloc(&d_out, sizeof(double) * 6 * rows * n));
  const int64_t tot = rows * n;
  if (T->layout == MT_LAYOUT_DENSE)
    k_read_rows_dense<<<(unsigned)((tot + 255) / 256), 256>>>((const __nv_bfloat16 *)T->d_data,
                                                              T->prec == MT_BF16_SPLIT, n, T->Kp, i0, i1, d_out);
  else
    k_read_rows<<<(unsigned)((tot + 255) / 256), 256>>>(T->d_data, T->d_scale, T->prec, n, T->L.TR, T->L.TC,
                                                         T->L.nplane, T->L.Q, T->L.half, i0, i1, d_out);
  MT_CUDA(cudaGetLastError());
  if (T->near_count > 0) {
    k_merge_near<<<(unsigned)((rows + 127) / 128), 128>>>(n, i0, i1, T->d_near_ptr, T->d_near_col,
                                                          T->d_near_val, d_out);
    MT_CUDA(cudaGetLastError());
  }
  MT_CUDA(cudaMemcpy(out, d_out, sizeof(double) * 6 * rows * n, cudaMemcpyDeviceToHost));
  cudaFree(d_out);
  return MT_OK;
}

}  // namespace mt
