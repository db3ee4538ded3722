/*
 * FP64 CPU oracle for the tile-based micromagnetic method of Bjork et al.,
 * "MagTense: a micromagnetic framework using the analytical demagnetization
 * tensor" (arXiv 2107.05364).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * reference that the CUDA path is checked against.  Nothing in the product
 * path may link, import or call it; only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark do.  It shares no code, header, table
 * or constant with the CUDA library: every formula below is written out again
 * from the paper's equations and from the closed form of the cuboid tensor.
 *
 * Everything is double precision, SI units (H in A/m, lengths in m,
 * Ms in A/m, A_ex in J/m, K in J/m^3, gamma in m/(A s)).
 *
 * Parts and the passage each follows:
 *   - cuboid point tensor ........ Sec. 3 (tiles, Smith et al. closed form),
 *                                   Eq. 9 read as H_d = -N (Ms m)
 *   - tetrahedron point tensor ... Sec. 3 (tetrahedron tiles), from the
 *                                   surface charges of a uniform body
 *   - demag field ................ Eq. 9/10, Sec. 3.1 Eq. 17 (dense product)
 *   - exchange field ............. Eq. 12, Neumann boundary from Eq. 3,
 *                                   3-point stencil of Sec. 4.1
 *   - anisotropy field ........... Eq. 16
 *   - Zeeman field ............... Eq. 7
 *   - Landau-Lifshitz RHS ........ Eq. 1 (and its Gilbert-form equivalent)
 *   - RK(4,5) integration ........ Sec. 3.1 (an explicit Runge-Kutta 4(5) pair),
 *                                   Dormand & Prince 1980 coefficients
 *   - relaxation ................. Sec. 4.1 (damping-only relaxation), Eq. 2
 *   - energy ..................... Eqs. 4, 6, 8, 11, 15
 *
 * Parity status: every function here is pinned by the tests in
 * tests/test_oracle_*.py (closed forms, invariants, quadrature, library
 * ODE solvers).  No function is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
/* vacuum permeability, classical value 4 pi 1e-7 H/m */
#define OR_MU0 (4.0e-7 * OR_PI)

/* status codes, same meaning as the library's */
#define OR_OK 0
#define OR_EINVAL 1
#define OR_EOVERLAP 3
#define OR_ENOCONV 4
#define OR_ENONFINITE 6

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Demagnetization tensor of one uniformly magnetised rectangular cuboid     */
/* ------------------------------------------------------------------------ */
/*
 * Sec. 3: the field of each tile is evaluated at the centre of every other
 * tile, assuming the tile is uniformly magnetised.  The closed form for the
 * cuboid (cited by the paper to Smith et al. 2010, not printed there) is
 * written out here from the Newtonian potential of the box,
 *     Phi(r) = int_box dV' / |r - r'|,   N = -(1/4 pi) grad grad Phi,
 * so that H = -N M and the self term of a cube is I/3.
 *
 * With corner offsets U = x - x_c, V = y - y_c, W = z - z_c (x_c, y_c, z_c
 * the coordinates of the box's faces), R = sqrt(U^2+V^2+W^2) and the sign
 * s = (-1)^(i+j+k), i,j,k in {1,2} numbering the low (1) and high (2) face
 * of each axis:
 *     N_xx = -(1/4pi) sum s atan(V W / (U R))      (yy, zz cyclic)
 *     N_xy = +(1/4pi) sum s ln(W + R)               (xz: ln(V+R), yz: ln(U+R))
 *
 * Readings of degenerate points:
 *  - U == 0 (field point in the plane of a face, outside the face): the atan
 *    term is taken as 0; the +-pi/2 limits cancel over the other two axes.
 *  - ln(W+R) with both W of a pair negative loses all digits when the point
 *    lies far below the box; there ln(W+R) = ln(U^2+V^2) - ln(R-W) and the
 *    first part cancels exactly inside the pair, so the pair is evaluated as
 *    -(ln(R2-W2) - ln(R1-W1)).  Same for the V and U logarithms.
 */

/* pair sum over the two faces of one axis:  ln(w2+R2) - ln(w1+R1),
 * written without cancellation when both offsets are negative */
static double or_log_pair(double w1, double r1, double w2, double r2) {
  if (w1 < 0.0 && w2 < 0.0) return -(log(r2 - w2) - log(r1 - w1));
  return log(w2 + r2) - log(w1 + r1);
}

static double or_atan_term(double u, double v, double w, double r) {
  if (u == 0.0) return 0.0;
  return atan((v * w) / (u * r));
}

/* N6 = {xx, xy, xz, yy, yz, zz} of the tile (centre cs, full edges e)
 * at the field point r */
void or_point_tensor(const double *r, const double *cs, const double *e, double *N6) {
  double U[2], V[2], W[2];
  /* index 0 = low face (coordinate c - e/2), 1 = high face */
  U[0] = r[0] - (cs[0] - 0.5 * e[0]);
  U[1] = r[0] - (cs[0] + 0.5 * e[0]);
  V[0] = r[1] - (cs[1] - 0.5 * e[1]);
  V[1] = r[1] - (cs[1] + 0.5 * e[1]);
  W[0] = r[2] - (cs[2] - 0.5 * e[2]);
  W[1] = r[2] - (cs[2] + 0.5 * e[2]);

  double sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
  double R[2][2][2];
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++)
      for (int k = 0; k < 2; k++)
        R[i][j][k] = sqrt(U[i] * U[i] + V[j] * V[j] + W[k] * W[k]);

  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++)
      for (int k = 0; k < 2; k++) {
        /* s = (-1)^(i+j+k) with 1-based face numbers = -(-1)^(i+j+k) 0-based */
        double s = ((i + j + k) % 2 == 0) ? -1.0 : 1.0;
        double rr = R[i][j][k];
        sxx += s * or_atan_term(U[i], V[j], W[k], rr);
        syy += s * or_atan_term(V[j], U[i], W[k], rr);
        szz += s * or_atan_term(W[k], U[i], V[j], rr);
      }
  /* log entries: sum over the third axis as a pair, then signs of the other two.
   * For fixed (i,j): sum_k s ln(W_k + R) = s(i,j,0) [ln(W0+R0) - ln(W1+R1)]
   * since s flips with k; s(i,j,0) = -(-1)^(i+j). */
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) {
      double s0 = ((i + j) % 2 == 0) ? -1.0 : 1.0; /* s at k = 0 */
      /* ln(W0+R0) - ln(W1+R1) = -(ln(W1+R1) - ln(W0+R0)) */
      sxy += -s0 * or_log_pair(W[0], R[i][j][0], W[1], R[i][j][1]);
    }
  for (int i = 0; i < 2; i++)
    for (int k = 0; k < 2; k++) {
      double s0 = ((i + k) % 2 == 0) ? -1.0 : 1.0; /* s at j = 0 */
      sxz += -s0 * or_log_pair(V[0], R[i][0][k], V[1], R[i][1][k]);
    }
  for (int j = 0; j < 2; j++)
    for (int k = 0; k < 2; k++) {
      double s0 = ((j + k) % 2 == 0) ? -1.0 : 1.0; /* s at i = 0 */
      syz += -s0 * or_log_pair(U[0], R[0][j][k], U[1], R[1][j][k]);
    }
  const double c = 1.0 / (4.0 * OR_PI);
  N6[0] = -c * sxx;
  N6[1] = c * sxy;
  N6[2] = c * sxz;
  N6[3] = -c * syy;
  N6[4] = c * syz;
  N6[5] = -c * szz;
}

/*
 * Geometry check (Sec. 3: tiles are adjacent and do not overlap).
 * Returns OR_EOVERLAP if two tiles share volume, or if a tile centre lies
 * inside or on the surface of another tile (the field point would sit on a
 * source's surface, where the point tensor is undefined).
 */
int or_check_tiles(int64_t n, const double *centre, const double *edge) {
  for (int64_t i = 0; i < n; i++)
    for (int64_t j = 0; j < n; j++) {
      if (i == j) continue;
      int vol = 1, pt = 1;
      for (int a = 0; a < 3; a++) {
        double d = fabs(centre[3 * i + a] - centre[3 * j + a]);
        double tol = 1e-12 * (edge[3 * i + a] + edge[3 * j + a]);
        if (!(d < 0.5 * (edge[3 * i + a] + edge[3 * j + a]) - tol)) vol = 0;
        if (!(d <= 0.5 * edge[3 * j + a] + tol)) pt = 0;
      }
      if (vol || pt) return OR_EOVERLAP;
    }
  return OR_OK;
}

/* Full tensor, block (i, j) = tile j evaluated at the centre of tile i,
 * stored row-major as N[(i*n + j)*6 + e]. */
void or_demag_tensor(int64_t n, const double *centre, const double *edge, double *N) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; i++)
    for (int64_t j = 0; j < n; j++)
      or_point_tensor(&centre[3 * i], &centre[3 * j], &edge[3 * j], &N[(i * n + j) * 6]);
}

/* Selected blocks (i = pairs[2p], j = pairs[2p+1]) */
void or_demag_blocks(const double *centre, const double *edge, int64_t np, const int64_t *pairs,
                     double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < np; p++) {
    int64_t i = pairs[2 * p], j = pairs[2 * p + 1];
    or_point_tensor(&centre[3 * i], &centre[3 * j], &edge[3 * j], &out[6 * p]);
  }
}

/* H = -N x for one symmetric block, x = Ms_j m_j */
static void or_block_apply(const double *N6, const double *x, double *acc) {
  acc[0] += N6[0] * x[0] + N6[1] * x[1] + N6[2] * x[2];
  acc[1] += N6[1] * x[0] + N6[3] * x[1] + N6[4] * x[2];
  acc[2] += N6[2] * x[0] + N6[4] * x[1] + N6[5] * x[2];
}

/*
 * Demag field from the stored tensor (Eq. 9 as a sum over tiles, Eq. 17):
 *   H_d,i = - sum_j N_ij (Ms_j m_j),  all j including j = i.
 * m is tile-major (m[3j + c]).
 */
/* ------------------------------------------------------------------------ */
/* Tetrahedron tile (Sec. 3: the tensor of a uniformly magnetised            */
/* tetrahedron is known in closed form; the paper cites it, not prints it)  */
/* ------------------------------------------------------------------------ */
/*
 * Written here from the surface-charge form of the field.  A body of uniform
 * magnetisation M carries the charge density M.n_f on each plane face f
 * (outward unit normal n_f), so
 *     H(r) = -(1/4 pi) sum_f (M . n_f) G_f(r),   G_f(r) = grad_r int_f dS'/|r - r'|,
 * and with H = -N M:   N_ab(r) = (1/4 pi) sum_f G_f,a(r) n_f,b.
 * Splitting r - r' into the height h = (r - r').n_f and in-plane parts, the
 * normal part of G_f is -n_f int_f h/R^3 dS' = -n_f Omega_f(r) (the solid
 * angle of the face seen from r, signed like h), and by the 2-D gradient
 * theorem the in-plane part is -sum_e u_e int_e dl'/R, u_e the in-plane unit
 * normal pointing out of the face across edge e.  For the edge p1 -> p2 with
 * unit tangent t and s_k = (p_k - r).t, R_k = |p_k - r|:
 *     int_e dl'/R = ln((R2 + s2)/(R1 + s1)) = ln((R1 - s1)/(R2 - s2)),
 * the second form used when the first would cancel (s1 + s2 < 0).
 * The solid angle of a triangle is taken from the formula of Van Oosterom
 * and Strackee (1983):
 *     tan(Omega/2) = a.(b x c) / (|a||b||c| + (a.b)|c| + (a.c)|b| + (b.c)|a|),
 * a, b, c the vertices relative to r; with the vertices counter-clockwise
 * about n_f the triple product is -h times a positive quantity, hence the sign.
 * Outside the body the solid angles cancel and tr N = 0; inside they add up
 * to -4 pi and tr N = 1.
 */
static double or_dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void or_cross3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

static double or_edge_integral(const double *r, const double *p1, const double *p2) {
  double t[3], d1[3], d2[3];
  for (int c = 0; c < 3; c++) {
    t[c] = p2[c] - p1[c];
    d1[c] = p1[c] - r[c];
    d2[c] = p2[c] - r[c];
  }
  double len = sqrt(or_dot3(t, t));
  for (int c = 0; c < 3; c++) t[c] /= len;
  double s1 = or_dot3(d1, t), s2 = or_dot3(d2, t);
  double R1 = sqrt(or_dot3(d1, d1)), R2 = sqrt(or_dot3(d2, d2));
  if (s1 + s2 >= 0) return log((R2 + s2) / (R1 + s1));
  return log((R1 - s1) / (R2 - s2));
}

/* int over the triangle (v0, v1, v2) of h/R^3, vertices counter-clockwise
   about the face normal, h = (r - v0).n */
static double or_triangle_solid_angle(const double *r, const double *v0, const double *v1, const double *v2) {
  double a[3], b[3], c[3], bc[3];
  for (int k = 0; k < 3; k++) {
    a[k] = v0[k] - r[k];
    b[k] = v1[k] - r[k];
    c[k] = v2[k] - r[k];
  }
  or_cross3(b, c, bc);
  double num = or_dot3(a, bc);
  double la = sqrt(or_dot3(a, a)), lb = sqrt(or_dot3(b, b)), lc = sqrt(or_dot3(c, c));
  double den = la * lb * lc + or_dot3(a, b) * lc + or_dot3(a, c) * lb + or_dot3(b, c) * la;
  return -2.0 * atan2(num, den);
}

/* full 3x3 point tensor (row-major) of the tetrahedron v[0..11] at r */
void or_tetra_point_tensor_full(const double *r, const double *v, double *N9) {
  for (int k = 0; k < 9; k++) N9[k] = 0.0;
  for (int f = 0; f < 4; f++) {
    /* face opposite vertex f, oriented so that its normal points away from it */
    const double *p[3];
    int q = 0;
    for (int k = 0; k < 4; k++)
      if (k != f) p[q++] = &v[3 * k];
    double e1[3], e2[3], nrm[3], w[3];
    for (int c = 0; c < 3; c++) {
      e1[c] = p[1][c] - p[0][c];
      e2[c] = p[2][c] - p[0][c];
      w[c] = v[3 * f + c] - p[0][c];
    }
    or_cross3(e1, e2, nrm);
    if (or_dot3(nrm, w) > 0) { /* reverse the order: counter-clockwise about the outward normal */
      const double *tmp = p[1];
      p[1] = p[2];
      p[2] = tmp;
      for (int c = 0; c < 3; c++) nrm[c] = -nrm[c];
    }
    double ln = sqrt(or_dot3(nrm, nrm));
    for (int c = 0; c < 3; c++) nrm[c] /= ln;
    double G[3];
    double om = or_triangle_solid_angle(r, p[0], p[1], p[2]);
    for (int c = 0; c < 3; c++) G[c] = -nrm[c] * om;
    for (int e = 0; e < 3; e++) {
      const double *a = p[e], *b = p[(e + 1) % 3];
      double t[3], u[3];
      for (int c = 0; c < 3; c++) t[c] = b[c] - a[c];
      or_cross3(t, nrm, u); /* in-plane, pointing out of the face for counter-clockwise edges */
      double lu = sqrt(or_dot3(u, u));
      double L = or_edge_integral(r, a, b);
      for (int c = 0; c < 3; c++) G[c] -= u[c] / lu * L;
    }
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) N9[3 * a + b] += G[a] * nrm[b] / (4.0 * OR_PI);
  }
}

/* the 6 unique entries (xx, xy, xz, yy, yz, zz) of the symmetrised tensor */
void or_tetra_point_tensor(const double *r, const double *v, double *N6) {
  double N9[9];
  or_tetra_point_tensor_full(r, v, N9);
  N6[0] = N9[0];
  N6[1] = 0.5 * (N9[1] + N9[3]);
  N6[2] = 0.5 * (N9[2] + N9[6]);
  N6[3] = N9[4];
  N6[4] = 0.5 * (N9[5] + N9[7]);
  N6[5] = N9[8];
}

/* full tensor of a tetrahedral tile set, evaluated at the centroids */
void or_tetra_demag_tensor(int64_t n, const double *v, double *N) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; i++) {
    double r[3];
    for (int c = 0; c < 3; c++)
      r[c] = 0.25 * (v[12 * i + c] + v[12 * i + 3 + c] + v[12 * i + 6 + c] + v[12 * i + 9 + c]);
    for (int64_t j = 0; j < n; j++) or_tetra_point_tensor(r, &v[12 * j], &N[(i * n + j) * 6]);
  }
}

void or_demag_field_dense(int64_t n, const double *N, const double *Ms, const double *m, double *H) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) {
    double acc[3] = {0, 0, 0};
    for (int64_t j = 0; j < n; j++) {
      double x[3] = {Ms[j] * m[3 * j], Ms[j] * m[3 * j + 1], Ms[j] * m[3 * j + 2]};
      or_block_apply(&N[(i * n + j) * 6], x, acc);
    }
    H[3 * i] = -acc[0];
    H[3 * i + 1] = -acc[1];
    H[3 * i + 2] = -acc[2];
  }
}

/* Same field for selected rows, tensor blocks evaluated on the fly. */
void or_demag_field_rows(int64_t n, const double *centre, const double *edge, const double *Ms,
                         const double *m, int64_t nrows, const int64_t *rows, double *H) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; r++) {
    int64_t i = rows[r];
    double acc[3] = {0, 0, 0};
    for (int64_t j = 0; j < n; j++) {
      double N6[6];
      or_point_tensor(&centre[3 * i], &centre[3 * j], &edge[3 * j], N6);
      double x[3] = {Ms[j] * m[3 * j], Ms[j] * m[3 * j + 1], Ms[j] * m[3 * j + 2]};
      or_block_apply(N6, x, acc);
    }
    H[3 * r] = -acc[0];
    H[3 * r + 1] = -acc[1];
    H[3 * r + 2] = -acc[2];
  }
}

/* H_d at the centroids of the tetrahedral tiles `rows`, row by row (matrix-free) */
void or_tetra_field_rows(int64_t n, const double *v, const double *Ms, const double *m, int64_t nrows,
                         const int64_t *rows, double *H) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; r++) {
    int64_t i = rows[r];
    double c[3];
    for (int a = 0; a < 3; a++)
      c[a] = 0.25 * (v[12 * i + a] + v[12 * i + 3 + a] + v[12 * i + 6 + a] + v[12 * i + 9 + a]);
    double acc[3] = {0, 0, 0};
    for (int64_t j = 0; j < n; j++) {
      double N6[6];
      or_tetra_point_tensor(c, &v[12 * j], N6);
      double x[3] = {Ms[j] * m[3 * j], Ms[j] * m[3 * j + 1], Ms[j] * m[3 * j + 2]};
      or_block_apply(N6, x, acc);
    }
    H[3 * r] = -acc[0];
    H[3 * r + 1] = -acc[1];
    H[3 * r + 2] = -acc[2];
  }
}

/* ------------------------------------------------------------------------ */
/* Local fields                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t n;
  const double *centre; /* 3n, m */
  const double *edge;   /* 3n, full edge lengths, m */
  const double *Ms;     /* n, A/m */
  const double *Aex;    /* n, J/m */
  const double *Ku;     /* n, J/m^3 */
  const double *axis;   /* 3n, unit easy axis */
  const int32_t *nbr;   /* 6n: -x,+x,-y,+y,-z,+z face neighbour, -1 = none; may be NULL */
  const double *N;      /* n*n*6 stored tensor */
  const double *xw;     /* 6n face coefficients area/(V_i d_ip), 1/m^2, replacing the
                           Cartesian 1/(h_i d_ip) (unstructured tiles); may be NULL */
  const double *vol;    /* n tile volumes replacing the edge products; may be NULL */
} or_model;

typedef struct {
  double gamma;  /* m/(A s) */
  double alpha;  /* Gilbert form: dimensionless; LL form: m/(A s) as in Eq. 1 */
  double Ha[3];  /* applied field, A/m */
  int form;      /* 0 = Gilbert (LLG) form, 1 = Landau-Lifshitz form of Eq. 1 */
  int precess;   /* 1 = keep the precession term, 0 = drop it (damping only) */
} or_llg;

/*
 * Exchange field, Eq. 12, H_ex = (2 A / (mu0 Ms)) laplacian(m), discretised
 * by finite volumes on the Cartesian tile mesh: the flux through the face
 * shared with neighbour p is (m_p - m_i) / d_ip, d_ip the centre distance
 * along the face normal; dividing the face sum by the tile volume gives
 *     H_ex,i = (2 A_i/(mu0 Ms_i)) sum_p (m_p - m_i) / (h_i d_ip),
 * h_i the tile's edge along that axis.  On a uniform grid this is the
 * 3-point stencil of Sec. 4.1.  A missing neighbour contributes no flux,
 * which is the Neumann condition dm/dn = 0 of Eq. 3.  For unstructured
 * tiles (tetrahedra) the same two-point flux is used with the face
 * coefficient area_f / (V_i d_ip) given per face (d_ip the centre distance
 * along the face normal); the paper leaves that operator to later work.
 */
void or_exchange_field(const or_model *md, const double *m, double *H) {
  int64_t n = md->n;
  for (int64_t i = 0; i < n; i++) {
    H[3 * i] = H[3 * i + 1] = H[3 * i + 2] = 0.0;
    if (!md->nbr) continue;
    double pref = 2.0 * md->Aex[i] / (OR_MU0 * md->Ms[i]);
    for (int f = 0; f < 6; f++) {
      int32_t p = md->nbr[6 * i + f];
      if (p < 0) continue;
      double w;
      if (md->xw) {
        w = md->xw[6 * i + f];
      } else {
        int ax = f / 2;
        double d = fabs(md->centre[3 * p + ax] - md->centre[3 * i + ax]);
        w = 1.0 / (md->edge[3 * i + ax] * d);
      }
      for (int c = 0; c < 3; c++) H[3 * i + c] += pref * w * (m[3 * p + c] - m[3 * i + c]);
    }
  }
}

/* Uniaxial anisotropy field, Eq. 16: (2K/(mu0 Ms)) (m . e) e */
void or_anisotropy_field(const or_model *md, const double *m, double *H) {
  for (int64_t i = 0; i < md->n; i++) {
    const double *e = &md->axis[3 * i];
    double me = m[3 * i] * e[0] + m[3 * i + 1] * e[1] + m[3 * i + 2] * e[2];
    double pref = 2.0 * md->Ku[i] / (OR_MU0 * md->Ms[i]);
    for (int c = 0; c < 3; c++) H[3 * i + c] = pref * me * e[c];
  }
}

/* Effective field Eq. 5 / Eq. 17: H_d + H_ex + H_an + H_a.
 * Hd (3n) receives the demag part alone if non-NULL. */
void or_effective_field(const or_model *md, const or_llg *p, const double *m, double *H, double *Hd) {
  int64_t n = md->n;
  double *hd = (double *)malloc(sizeof(double) * 3 * n);
  double *hx = (double *)malloc(sizeof(double) * 3 * n);
  double *ha = (double *)malloc(sizeof(double) * 3 * n);
  or_demag_field_dense(n, md->N, md->Ms, m, hd);
  or_exchange_field(md, m, hx);
  or_anisotropy_field(md, m, ha);
  for (int64_t k = 0; k < 3 * n; k++) H[k] = hd[k] + hx[k] + ha[k] + p->Ha[k % 3];
  if (Hd) memcpy(Hd, hd, sizeof(double) * 3 * n);
  free(hd);
  free(hx);
  free(ha);
}

static void or_cross(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/*
 * Right-hand side of the equation of motion.  Eq. 1 (Landau-Lifshitz):
 *     dm/dt = -gamma m x H - alpha m x (m x H)
 * Gilbert form (the LLG equation named in Sec. 4.1), written explicitly:
 *     dm/dt = -gamma/(1+alpha^2) [ m x H + alpha m x (m x H) ]
 * precess = 0 drops the m x H term (Sec. 4.1 uses gamma = 0 to relax).
 * tau (optional) receives max_i |m_i x H_i| / Ms_i.
 */
void or_llg_rhs(const or_model *md, const or_llg *p, const double *m, double *dmdt, double *tau) {
  int64_t n = md->n;
  double *H = (double *)malloc(sizeof(double) * 3 * n);
  or_effective_field(md, p, m, H, NULL);
  double g1, g2;
  if (p->form == 0) {
    g1 = p->gamma / (1.0 + p->alpha * p->alpha);
    g2 = g1 * p->alpha;
  } else {
    g1 = p->gamma;
    g2 = p->alpha;
  }
  if (!p->precess) g1 = 0.0;
  double tmax = 0.0;
  for (int64_t i = 0; i < n; i++) {
    double mxh[3], mxmxh[3];
    or_cross(&m[3 * i], &H[3 * i], mxh);
    or_cross(&m[3 * i], mxh, mxmxh);
    for (int c = 0; c < 3; c++) dmdt[3 * i + c] = -g1 * mxh[c] - g2 * mxmxh[c];
    double t = sqrt(mxh[0] * mxh[0] + mxh[1] * mxh[1] + mxh[2] * mxh[2]) / md->Ms[i];
    if (t > tmax) tmax = t;
  }
  if (tau) *tau = tmax;
  free(H);
}

/* ------------------------------------------------------------------------ */
/* Energy, Eqs. 4, 6, 8, 11, 15                                             */
/* ------------------------------------------------------------------------ */
/*
 * G = sum_i V_i g_i with the densities of Eqs. 6, 8, 11 and 15.  Each
 * quadratic density equals -(mu0 Ms/2) m . H_term (the field being the
 * first variation, Eq. 5), the Zeeman one -mu0 Ms m . H_a, so
 *     G = - mu0 sum_i V_i Ms_i m_i . (H_a + (H_d + H_ex + H_an)/2).
 * out[0..4] = total, Zeeman, demag, exchange, anisotropy (J).
 */
void or_energy(const or_model *md, const or_llg *p, const double *m, double *out) {
  int64_t n = md->n;
  double *hd = (double *)malloc(sizeof(double) * 3 * n);
  double *hx = (double *)malloc(sizeof(double) * 3 * n);
  double *ha = (double *)malloc(sizeof(double) * 3 * n);
  or_demag_field_dense(n, md->N, md->Ms, m, hd);
  or_exchange_field(md, m, hx);
  or_anisotropy_field(md, m, ha);
  double ez = 0, ed = 0, ex = 0, ea = 0;
  for (int64_t i = 0; i < n; i++) {
    double V = md->vol ? md->vol[i] : md->edge[3 * i] * md->edge[3 * i + 1] * md->edge[3 * i + 2];
    double w = OR_MU0 * md->Ms[i] * V;
    for (int c = 0; c < 3; c++) {
      double mc = m[3 * i + c];
      ez += -w * mc * p->Ha[c];
      ed += -0.5 * w * mc * hd[3 * i + c];
      ex += -0.5 * w * mc * hx[3 * i + c];
      ea += -0.5 * w * mc * ha[3 * i + c];
    }
  }
  out[0] = ez + ed + ex + ea;
  out[1] = ez;
  out[2] = ed;
  out[3] = ex;
  out[4] = ea;
  free(hd);
  free(hx);
  free(ha);
}

/* volume-weighted mean magnetisation */
static void or_mean_m(const or_model *md, const double *m, double *avg) {
  double s[3] = {0, 0, 0}, vt = 0;
  for (int64_t i = 0; i < md->n; i++) {
    double V = md->edge[3 * i] * md->edge[3 * i + 1] * md->edge[3 * i + 2];
    vt += V;
    for (int c = 0; c < 3; c++) s[c] += V * m[3 * i + c];
  }
  for (int c = 0; c < 3; c++) avg[c] = s[c] / vt;
}

/* ------------------------------------------------------------------------ */
/* Explicit Runge-Kutta (4,5): Dormand & Prince 1980                        */
/* ------------------------------------------------------------------------ */
/*
 * Sec. 3.1 integrates Eq. 1 with an explicit Runge-Kutta (4,5) formula
 * (Matlab's ode45, i.e. the Dormand-Prince pair).  The coefficients are the
 * published ones of Dormand & Prince (J. Comput. Appl. Math. 6, 1980).
 * Readings (the paper states no tolerances or controller):
 *   - error norm: RMS over all 3n components of e / (atol + rtol max(|y|,|y_new|)),
 *     e = h sum_j (b_j - bhat_j) k_j (Hairer, Norsett & Wanner II.4);
 *   - step accepted when the norm is <= 1;
 *   - new step h * clamp(0.9 err^(-1/5), 0.2, 5), capped at hmax;
 *   - first-same-as-last: the derivative at the 5th-order solution is reused
 *     as the first stage of the next step;
 *   - after acceptance every m_i is renormalised to |m_i| = 1 (Sec. 2.1:
 *     the equation preserves |m|, the discrete scheme does not exactly);
 *   - steps are shortened to land exactly on each output time.
 * Fixed-step mode (fixed_h > 0) takes steps of exactly fixed_h (shortened
 * only at output times), accepts all of them and still renormalises.
 */
static const double DP_C[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
/* 5th-order weights are the last row of A; 4th-order (embedded) weights: */
static const double DP_BHAT[7] = {5179.0 / 57600.0,    0.0,           7571.0 / 16695.0, 393.0 / 640.0,
                                  -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};

void or_dp45_tableau(double *c7, double *a76, double *b7, double *bhat7) {
  for (int s = 0; s < 7; s++) {
    c7[s] = DP_C[s];
    for (int j = 0; j < 6; j++) a76[s * 6 + j] = DP_A[s][j];
    b7[s] = (s < 6) ? DP_A[6][s] : 0.0;
    bhat7[s] = DP_BHAT[s];
  }
}

typedef struct {
  double rtol, atol;
  double h0;       /* first trial step, s */
  double hmax;     /* largest step, s */
  int64_t max_steps;  /* cap on attempted steps */
  double fixed_h;  /* > 0: fixed-step mode */
} or_ode;

typedef struct {
  int64_t n_accept, n_reject, n_rhs;
  double t, h, tau;
} or_stats;

/* Generic RHS used by the integrator: f(y) -> k, returns tau via *tau. */
typedef void (*or_rhs_fn)(void *ctx, const double *y, double *k, double *tau);

typedef struct {
  const or_model *md;
  const or_llg *p;
} or_llg_ctx;

static void or_llg_rhs_cb(void *ctx, const double *y, double *k, double *tau) {
  or_llg_ctx *c = (or_llg_ctx *)ctx;
  or_llg_rhs(c->md, c->p, y, k, tau);
}

/* Linear test problem y' = lambda y, component-wise lambda (for pins). */
typedef struct {
  int64_t dim;
  const double *lambda;
} or_lin_ctx;

static void or_lin_rhs_cb(void *ctx, const double *y, double *k, double *tau) {
  or_lin_ctx *c = (or_lin_ctx *)ctx;
  for (int64_t q = 0; q < c->dim; q++) k[q] = c->lambda[q] * y[q];
  if (tau) *tau = 0.0;
}

/*
 * Core driver.  dim state components; renorm != 0 renormalises consecutive
 * triples after acceptance; mode 0 = integrate to t1 with n_out outputs of
 * the (volume weighted, via the callback) mean; mode 1 = relax until
 * tau < tau_tol (or t1 reached -> OR_ENOCONV).
 * out_fn records an output row at each output time.
 */
typedef void (*or_out_fn)(void *octx, int64_t k, const double *y);

static int or_dp45_core(or_rhs_fn f, void *fctx, int64_t dim, int renorm, const or_ode *o, double *y,
                        double t0, double t1, int64_t n_out, or_out_fn out, void *octx, int relax,
                        double tau_tol, or_stats *st) {
  double *k[7], *ys, *ynew;
  for (int s = 0; s < 7; s++) k[s] = (double *)malloc(sizeof(double) * dim);
  ys = (double *)malloc(sizeof(double) * dim);
  ynew = (double *)malloc(sizeof(double) * dim);
  int status = OR_OK;
  double t = t0;
  double h = (o->fixed_h > 0) ? o->fixed_h : o->h0;
  double tau = 0.0;
  int64_t nacc = 0, nrej = 0, nrhs = 0;
  int64_t iout = 0;
  if (n_out < 1) n_out = 1;
  double dt_out = (t1 - t0) / (double)n_out;
  double t_next = relax ? t1 : t0 + dt_out;

  f(fctx, y, k[0], &tau);
  nrhs++;
  if (relax && tau < tau_tol) goto done;

  for (int64_t attempt = 0;; attempt++) {
    if (attempt >= o->max_steps) {
      status = OR_ENOCONV;
      break;
    }
    double hs = h;
    int clipped = 0;
    if (o->fixed_h <= 0 && o->hmax > 0 && hs > o->hmax) hs = o->hmax;
    if (t + hs >= t_next) {
      hs = t_next - t;
      clipped = 1;
    }
    /* stages 2..7 */
    for (int s = 1; s < 7; s++) {
      for (int64_t q = 0; q < dim; q++) {
        double acc = 0.0;
        for (int j = 0; j < s; j++) acc += DP_A[s][j] * k[j][q];
        ys[q] = y[q] + hs * acc;
      }
      if (s == 6) memcpy(ynew, ys, sizeof(double) * dim);
      f(fctx, ys, k[s], &tau);
      nrhs++;
    }
    /* embedded error */
    double err = 0.0;
    if (o->fixed_h <= 0) {
      double sum = 0.0;
      for (int64_t q = 0; q < dim; q++) {
        double eq = 0.0;
        for (int s = 0; s < 7; s++) {
          double bs = (s < 6) ? DP_A[6][s] : 0.0;
          eq += (bs - DP_BHAT[s]) * k[s][q];
        }
        eq *= hs;
        double sc = o->atol + o->rtol * fmax(fabs(y[q]), fabs(ynew[q]));
        sum += (eq / sc) * (eq / sc);
      }
      err = sqrt(sum / (double)dim);
      if (!isfinite(err)) {
        status = OR_ENONFINITE;
        break;
      }
    } else {
      /* no error norm to watch: a step that left the finite numbers ends the run */
      int finite = 1;
      for (int64_t q = 0; q < dim; q++) finite = finite && isfinite(ynew[q]);
      if (!finite) {
        status = OR_ENONFINITE;
        break;
      }
    }
    int accept = (o->fixed_h > 0) || (err <= 1.0);
    if (accept) {
      t = clipped ? t_next : t + hs;
      memcpy(y, ynew, sizeof(double) * dim);
      if (renorm)
        for (int64_t i = 0; i < dim / 3; i++) {
          double nr = sqrt(y[3 * i] * y[3 * i] + y[3 * i + 1] * y[3 * i + 1] + y[3 * i + 2] * y[3 * i + 2]);
          for (int c = 0; c < 3; c++) y[3 * i + c] /= nr;
        }
      memcpy(k[0], k[6], sizeof(double) * dim); /* first same as last */
      nacc++;
      if (!relax && clipped) {
        if (out) out(octx, iout, y);
        iout++;
        if (iout >= n_out) break;
        t_next = t0 + (double)(iout + 1) * dt_out;
        if (iout + 1 == n_out) t_next = t1;
      }
      if (relax) {
        if (tau < tau_tol) break;
        if (clipped) {
          status = OR_ENOCONV;
          break;
        }
      }
    } else {
      nrej++;
    }
    if (o->fixed_h > 0) {
      h = o->fixed_h;
    } else {
      double fac = (err > 0.0) ? 0.9 * pow(err, -0.2) : 5.0;
      if (fac < 0.2) fac = 0.2;
      if (fac > 5.0) fac = 5.0;
      h = hs * fac;
      if (o->hmax > 0 && h > o->hmax) h = o->hmax;
    }
  }
done:
  if (st) {
    st->n_accept = nacc;
    st->n_reject = nrej;
    st->n_rhs = nrhs;
    st->t = t;
    st->h = h;
    st->tau = tau;
  }
  for (int s = 0; s < 7; s++) free(k[s]);
  free(ys);
  free(ynew);
  return status;
}

typedef struct {
  const or_model *md;
  double *mavg; /* n_out * 3 */
} or_mavg_ctx;

static void or_mavg_out(void *octx, int64_t k, const double *y) {
  or_mavg_ctx *c = (or_mavg_ctx *)octx;
  or_mean_m(c->md, y, &c->mavg[3 * k]);
}

/* Integrate Eq. 1 from t0 to t1, recording <m> at t0 + (k+1)(t1-t0)/n_out. */
int or_integrate(const or_model *md, const or_llg *p, const or_ode *o, double *m, double t0, double t1,
                 int64_t n_out, double *mavg, or_stats *st) {
  or_llg_ctx c = {md, p};
  or_mavg_ctx oc = {md, mavg};
  return or_dp45_core(or_llg_rhs_cb, &c, 3 * md->n, 1, o, m, t0, t1, n_out, mavg ? or_mavg_out : NULL, &oc,
                      0, 0.0, st);
}

/* Relax (Sec. 4.1, Eq. 2): integrate until max_i |m_i x H_eff,i|/Ms_i < tol,
 * or give up at t_max with OR_ENOCONV. */
int or_relax(const or_model *md, const or_llg *p, const or_ode *o, double *m, double tol, double t_max,
             or_stats *st) {
  or_llg_ctx c = {md, p};
  return or_dp45_core(or_llg_rhs_cb, &c, 3 * md->n, 1, o, m, 0.0, t_max, 1, NULL, NULL, 1, tol, st);
}

/* y' = lambda y with the same driver (no renormalisation), output y at the
 * output times into yout (n_out * dim). */
typedef struct {
  int64_t dim;
  double *yout;
} or_lin_out_ctx;
static void or_lin_out(void *octx, int64_t k, const double *y) {
  or_lin_out_ctx *c = (or_lin_out_ctx *)octx;
  memcpy(&c->yout[k * c->dim], y, sizeof(double) * c->dim);
}
int or_integrate_linear(int64_t dim, const double *lambda, const or_ode *o, double *y, double t0, double t1,
                        int64_t n_out, double *yout, or_stats *st) {
  or_lin_ctx c = {dim, lambda};
  or_lin_out_ctx oc = {dim, yout};
  return or_dp45_core(or_lin_rhs_cb, &c, dim, 0, o, y, t0, t1, n_out, yout ? or_lin_out : NULL, &oc, 0, 0.0,
                      st);
}
