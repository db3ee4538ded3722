// C ABI of libmagtile: contexts, tile sets, tensors and the field / RHS
// entry points.  The integrator lives in llg.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "mt_internal.cuh"

namespace {
thread_local std::string g_err;
}

namespace mt {

void set_error(const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

mt_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
  return e == cudaErrorMemoryAllocation ? MT_ENOMEM : MT_ECUDA;
}

void ctx_release(mt_ctx *c) {
  if (c && --c->refs == 0) {
    cudaFree(c->d_status);
    if (c->small_ev) cudaEventDestroy(c->small_ev);
    delete c;
  }
}

}  // namespace mt

namespace {

template <typename P>
mt_status upload(P **dst, const P *src, size_t count) {
  MT_CUDA(cudaMalloc((void **)dst, sizeof(P) * std::max<size_t>(count, 1)));
  MT_CUDA(cudaMemcpy(*dst, src, sizeof(P) * count, cudaMemcpyHostToDevice));
  return MT_OK;
}

template <typename P>
mt_status copy_to(P *dst, const P *src, size_t count) {
  MT_CUDA(cudaMemcpy(dst, src, sizeof(P) * count, cudaMemcpyHostToDevice));
  return MT_OK;
}

void free_tiles(mt_tiles *t) {
  mt_ctx *ctx = t->ctx;
  cudaFree(t->d_centre);
  cudaFree(t->d_edge);
  cudaFree(t->d_Ms);
  cudaFree(t->d_wex);
  cudaFree(t->d_nbr);
  cudaFree(t->d_kan);
  cudaFree(t->d_axis);
  cudaFree(t->d_wvol);
  cudaFree(t->d_vert);
  cudaFree(t->d_lat);
  delete t;
  if (ctx) mt::ctx_release(ctx);
}

void free_tensor_mem(mt_tensor *T) {
  cudaFree(T->d_data);
  cudaFree(T->d_scale);
  cudaFree(T->d_near_ptr);
  cudaFree(T->d_near_col);
  cudaFree(T->d_near_val);
  cudaFree(T->d_near_hl);
  cudaFree(T->d_xs);
  cudaFree(T->d_part);
  cudaFree(T->d_count);
  cudaFree(T->d_Hd);
  cudaFree(T->d_colpart);
  cudaFree(T->d_sp_ptr);
  cudaFree(T->d_sp_rptr);
  cudaFree(T->d_sp_col);
  cudaFree(T->d_sp_val);
  cudaFree(T->d_sp_seg);
}

// workspace of the standalone field/rhs calls for B simulations
mt_status ensure_workspace(mt_tensor *T, int B) {
  const bool dense = T->layout == MT_LAYOUT_DENSE;
  if (dense && T->xs_B != B) {  // the padded batch is part of the operand's layout
    cudaFree(T->d_xs);
    T->d_xs = nullptr;
    T->xs_B = 0;
    cudaFree(T->d_part);
    T->d_part = nullptr;
  }
  if (T->xs_B < B) {
    cudaFree(T->d_xs);
    T->d_xs = nullptr;
    const size_t bytes = dense ? mt::dense_x_bytes(T, B) : sizeof(float) * mt::xs_floats(T) * B;
    MT_CUDA(cudaMalloc(&T->d_xs, bytes));
    MT_CUDA(cudaMemset(T->d_xs, 0, bytes));
    T->xs_B = B;
  }
  if (!T->d_part) {
    MT_CUDA(cudaMalloc(&T->d_part, dense ? mt::dense_part_bytes(T, B) : mt::matvec_part_bytes(T)));
  }
  if (T->L.half && T->colpart_B < B) {  // half storage: column work area (grows with B)
    cudaFree(T->d_colpart);
    T->d_colpart = nullptr;
    T->colpart_B = 0;
    MT_CUDA(cudaMalloc(&T->d_colpart, mt::matvec_colpart_bytes(T, B)));
    T->colpart_B = B;
  }
  if (T->count_B < B) {
    cudaFree(T->d_count);
    T->d_count = nullptr;
    const size_t bytes = dense ? mt::dense_count_bytes(T) : mt::matvec_count_bytes(T, B);
    MT_CUDA(cudaMalloc(&T->d_count, bytes));
    MT_CUDA(cudaMemset(T->d_count, 0, bytes));
    T->count_B = B;
  }
  if (T->Hd_B < B) {
    cudaFree(T->d_Hd);
    T->d_Hd = nullptr;
    MT_CUDA(cudaMalloc(&T->d_Hd, sizeof(float) * 3 * T->n * B));
    T->Hd_B = B;
  }
  return MT_OK;
}

// H = -N (Ms m) with the tensor's own workspace: streaming product or, for
// the dense layout, the batched tensor-core product; then the FP64 near blocks
mt_status demag_apply(mt_tensor *T, const float *m, int B, float *H, cudaStream_t s) {
  if (T->layout == MT_LAYOUT_SPARSE) {
    mt::launch_prep_xs(T, m, B, T->d_xs, s);
    mt::launch_spmv(T, T->d_xs, B, H, nullptr, s);
    return MT_OK;
  }
  if (T->layout == MT_LAYOUT_DENSE) {
    GemmPlan plan;
    mt_status st = mt::gemm_plan(T, B, T->d_xs, &plan);
    if (st != MT_OK) return st;
    st = mt::gemm_tune(T, &plan, H, T->d_part, T->d_count, T->tiles->ctx->d_status, s);
    if (st != MT_OK) return st;
    mt::launch_prep_dense_x(T, m, B, T->d_xs, s);
    mt::launch_gemm(T, plan, H, T->d_part, T->d_count, nullptr, T->tiles->ctx->d_status, s);
    mt::launch_near(T, mt::dense_mT(T, B, T->d_xs), 1, mt::dense_pad_batch(B), B, H, nullptr, s);
  } else {
    mt::launch_prep_xs(T, m, B, T->d_xs, s);
    mt::launch_matvec(T, T->d_xs, B, H, T->d_part, T->d_count, nullptr, T->tiles->ctx->d_status, s, T->d_colpart);
    mt::launch_near(T, m, 3 * T->n, 1, B, H, nullptr, s);
  }
  return MT_OK;
}

}  // namespace

extern "C" {

const char *mt_version(void) { return "magtile 0.1 (sm_103a)"; }

const char *mt_last_error(void) { return g_err.c_str(); }

mt_status mt_ctx_create(int device, size_t hbm_budget_bytes, mt_ctx **out) {
  MT_CHECK(out, MT_EINVAL, "mt_ctx_create: out is NULL");
  int ndev = 0;
  MT_CUDA(cudaGetDeviceCount(&ndev));
  MT_CHECK(device >= 0 && device < ndev, MT_EINVAL, "mt_ctx_create: device %d of %d", device, ndev);
  MT_CUDA(cudaSetDevice(device));
  cudaDeviceProp prop;
  MT_CUDA(cudaGetDeviceProperties(&prop, device));
  MT_CHECK(prop.major * 10 + prop.minor >= 100, MT_EINVAL,
           "mt_ctx_create: device %d is sm_%d%d; this library is built for sm_103a", device, prop.major,
           prop.minor);
  mt_ctx *c = new mt_ctx();
  c->device = device;
  c->num_sms = prop.multiProcessorCount;
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    delete c;
    return mt::cuda_fail(e, "cudaMemGetInfo", __FILE__, __LINE__);
  }
  c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)free_b);
  e = cudaMalloc(&c->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = mt::matvec_prepare();
  if (e == cudaSuccess) e = mt::gemm_prepare();
  if (e != cudaSuccess) {
    cudaFree(c->d_status);
    delete c;
    return mt::cuda_fail(e, "mt_ctx_create", __FILE__, __LINE__);
  }
  *out = c;
  return MT_OK;
}

void mt_ctx_destroy(mt_ctx *ctx) { mt::ctx_release(ctx); }

size_t mt_ctx_bytes_in_use(const mt_ctx *ctx) { return ctx ? ctx->in_use : 0; }

mt_status mt_tiles_create(mt_ctx *ctx, int64_t n, const double *centre, const double *edge, const double *Ms,
                          const double *Aex, const double *Ku, const double *axis, const int32_t *nbr,
                          mt_tiles **out) {
  MT_CHECK(ctx && out, MT_EINVAL, "mt_tiles_create: NULL handle");
  MT_CHECK(n >= 1 && n <= (int64_t)1 << 26, MT_EINVAL, "mt_tiles_create: n = %lld out of range", (long long)n);
  MT_CHECK(centre && edge && Ms && Aex && Ku && axis, MT_EINVAL, "mt_tiles_create: NULL array");
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      MT_CHECK(std::isfinite(centre[3 * i + a]) && std::isfinite(axis[3 * i + a]), MT_EINVAL,
               "mt_tiles_create: non-finite centre/axis at tile %lld", (long long)i);
      MT_CHECK(std::isfinite(edge[3 * i + a]) && edge[3 * i + a] > 0, MT_EINVAL,
               "mt_tiles_create: edge of tile %lld must be positive", (long long)i);
    }
    MT_CHECK(std::isfinite(Ms[i]) && Ms[i] > 0, MT_EINVAL, "mt_tiles_create: Ms of tile %lld must be positive",
             (long long)i);
    MT_CHECK(std::isfinite(Aex[i]) && std::isfinite(Ku[i]), MT_EINVAL,
             "mt_tiles_create: non-finite A_ex/K_u at tile %lld", (long long)i);
    if (nbr)
      for (int f = 0; f < 6; ++f) {
        const int32_t p = nbr[6 * i + f];
        MT_CHECK(p >= -1 && p < n && p != i, MT_EINVAL, "mt_tiles_create: bad neighbour %d of tile %lld", p,
                 (long long)i);
      }
  }
  MT_CUDA(cudaSetDevice(ctx->device));
  mt_tiles *t = new mt_tiles();
  t->ctx = ctx;
  ctx->refs++;
  t->n = n;
  t->centre.assign(centre, centre + 3 * n);
  t->edge.assign(edge, edge + 3 * n);
  t->Ms.assign(Ms, Ms + n);
  t->Aex.assign(Aex, Aex + n);
  t->Ku.assign(Ku, Ku + n);
  t->axis.resize(3 * n);
  std::vector<float> msf(n), kan(n), axf(3 * n), wex(6 * n, 0.0f);
  std::vector<double> wvol(n);
  double vt = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double *e = &axis[3 * i];
    double nr = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    for (int a = 0; a < 3; ++a) {
      const double v = nr > 0 ? e[a] / nr : (a == 2 ? 1.0 : 0.0);
      t->axis[3 * i + a] = v;
      axf[3 * i + a] = (float)v;
    }
    msf[i] = (float)Ms[i];
    kan[i] = (float)(2.0 * Ku[i] / (MT_MU0 * Ms[i]));
    wvol[i] = edge[3 * i] * edge[3 * i + 1] * edge[3 * i + 2];
    vt += wvol[i];
  }
  for (auto &v : wvol) v /= vt;
  t->vol_total = vt;
  if (nbr) {
    t->nbr.assign(nbr, nbr + 6 * n);
    t->has_exchange = true;
    // finite-volume exchange weights (Eq. 12): 2 A_i / (mu0 Ms_i h_i d_ip)
    for (int64_t i = 0; i < n; ++i)
      for (int f = 0; f < 6; ++f) {
        const int32_t p = nbr[6 * i + f];
        if (p < 0) continue;
        const int ax = f / 2;
        const double d = std::fabs(centre[3 * p + ax] - centre[3 * i + ax]);
        const double h = edge[3 * i + ax];
        if (!(d > 0)) {
          free_tiles(t);
          mt::set_error("mt_tiles_create: neighbour %d of tile %lld has the same centre", p, (long long)i);
          return MT_EINVAL;
        }
        wex[6 * i + f] = (float)(2.0 * Aex[i] / (MT_MU0 * Ms[i] * h * d));
      }
  }
  std::vector<int32_t> nb(6 * n, -1);
  if (nbr) std::copy(nbr, nbr + 6 * n, nb.begin());
  // uniform lattice?  equal edges and every centre within 1e-9 edges of
  // c_min + index * edge; the offset table must stay small
  std::vector<int32_t> lat;
  {
    bool ok = true;
    double cmin[3] = {centre[0], centre[1], centre[2]};
    for (int64_t i = 0; i < n && ok; ++i)
      for (int a = 0; a < 3; ++a) {
        ok = ok && std::fabs(edge[3 * i + a] - edge[a]) <= 1e-12 * edge[a];
        cmin[a] = std::min(cmin[a], centre[3 * i + a]);
      }
    int64_t L[3] = {1, 1, 1};
    if (ok) {
      lat.resize(3 * n);
      for (int64_t i = 0; i < n && ok; ++i)
        for (int a = 0; a < 3; ++a) {
          const double u = (centre[3 * i + a] - cmin[a]) / edge[a];
          const double r = std::nearbyint(u);
          ok = ok && std::fabs(u - r) <= 1e-9 && r < 1e6;
          lat[3 * i + a] = (int32_t)r;
          L[a] = std::max<int64_t>(L[a], (int64_t)r + 1);
        }
    }
    ok = ok && (2 * L[0] - 1) * (2 * L[1] - 1) * (2 * L[2] - 1) <= ((int64_t)1 << 22);
    if (ok) {
      t->lattice = true;
      t->Lx = (int)L[0];
      t->Ly = (int)L[1];
      t->Lz = (int)L[2];
      for (int a = 0; a < 3; ++a) t->lat_edge[a] = edge[a];
    }
  }
  mt_status st = MT_OK;
  if (t->lattice && (st = upload(&t->d_lat, lat.data(), 3 * n)) != MT_OK) {
    free_tiles(t);
    return st;
  }
  if ((st = upload(&t->d_centre, centre, 3 * n)) != MT_OK || (st = upload(&t->d_edge, edge, 3 * n)) != MT_OK ||
      (st = upload(&t->d_Ms, msf.data(), n)) != MT_OK || (st = upload(&t->d_wex, wex.data(), 6 * n)) != MT_OK ||
      (st = upload(&t->d_nbr, nb.data(), 6 * n)) != MT_OK || (st = upload(&t->d_kan, kan.data(), n)) != MT_OK ||
      (st = upload(&t->d_axis, axf.data(), 3 * n)) != MT_OK || (st = upload(&t->d_wvol, wvol.data(), n)) != MT_OK) {
    free_tiles(t);
    return st;
  }
  *out = t;
  return MT_OK;
}

mt_status mt_tiles_create_tetra(mt_ctx *ctx, int64_t nv, const double *vertices, int64_t n, const int32_t *tets,
                                const double *Ms, const double *Aex, const double *Ku, const double *axis,
                                mt_tiles **out) {
  MT_CHECK(ctx && out, MT_EINVAL, "mt_tiles_create_tetra: NULL handle");
  MT_CHECK(n >= 1 && n <= (int64_t)1 << 26, MT_EINVAL, "mt_tiles_create_tetra: n = %lld out of range", (long long)n);
  MT_CHECK(nv >= 4 && nv <= (int64_t)1 << 30, MT_EINVAL, "mt_tiles_create_tetra: nv = %lld out of range",
           (long long)nv);
  MT_CHECK(vertices && tets && Ms && Aex && Ku && axis, MT_EINVAL, "mt_tiles_create_tetra: NULL array");
  for (int64_t k = 0; k < 3 * nv; ++k)
    MT_CHECK(std::isfinite(vertices[k]), MT_EINVAL, "mt_tiles_create_tetra: non-finite vertex coordinate");
  std::vector<double> centre(3 * n), edge(3 * n), vert(12 * n), vol(n);
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 4; ++a) {
      const int32_t q = tets[4 * i + a];
      MT_CHECK(q >= 0 && q < nv, MT_EINVAL, "mt_tiles_create_tetra: vertex index %d of tile %lld out of range", q,
               (long long)i);
      for (int b = 0; b < a; ++b)
        MT_CHECK(tets[4 * i + b] != q, MT_EINVAL, "mt_tiles_create_tetra: repeated vertex in tile %lld",
                 (long long)i);
      for (int c = 0; c < 3; ++c) vert[12 * i + 3 * a + c] = vertices[3 * q + c];
    }
    const double *v = &vert[12 * i];
    double e1[3], e2[3], e3[3];
    for (int c = 0; c < 3; ++c) {
      e1[c] = v[3 + c] - v[c];
      e2[c] = v[6 + c] - v[c];
      e3[c] = v[9 + c] - v[c];
      centre[3 * i + c] = 0.25 * (v[c] + v[3 + c] + v[6 + c] + v[9 + c]);
    }
    const double det = e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
                       e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]);
    const double scale = std::max({std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]),
                                   std::sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]),
                                   std::sqrt(e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2])});
    vol[i] = std::fabs(det) / 6.0;
    MT_CHECK(vol[i] > 1e-12 * scale * scale * scale, MT_EINVAL, "mt_tiles_create_tetra: tile %lld is degenerate",
             (long long)i);
    const double h = std::cbrt(vol[i]);
    edge[3 * i] = edge[3 * i + 1] = edge[3 * i + 2] = h;
  }
  // tiles sharing a face: sort the faces by their vertex triples
  struct Face {
    int32_t a, b, c;
    int64_t tile;
    int slot;
  };
  std::vector<Face> faces(4 * n);
  for (int64_t i = 0; i < n; ++i)
    for (int f = 0; f < 4; ++f) {
      int32_t q[3], k = 0;
      for (int a = 0; a < 4; ++a)
        if (a != f) q[k++] = tets[4 * i + a];
      std::sort(q, q + 3);
      faces[4 * i + f] = {q[0], q[1], q[2], i, f};
    }
  std::sort(faces.begin(), faces.end(), [](const Face &x, const Face &y) {
    return x.a != y.a ? x.a < y.a : x.b != y.b ? x.b < y.b : x.c != y.c ? x.c < y.c : x.tile < y.tile;
  });
  std::vector<int32_t> nbr(6 * n, -1);
  std::vector<double> coef(6 * n, 0.0);  // area / (V_i d_ip)
  for (size_t k = 0; k < faces.size();) {
    size_t e = k + 1;
    while (e < faces.size() && faces[e].a == faces[k].a && faces[e].b == faces[k].b && faces[e].c == faces[k].c) ++e;
    MT_CHECK(e - k <= 2, MT_EINVAL, "mt_tiles_create_tetra: a face is shared by more than two tiles");
    if (e - k == 2) {
      const Face &F = faces[k], &G = faces[k + 1];
      const double *pa = &vertices[3 * F.a], *pb = &vertices[3 * F.b], *pc = &vertices[3 * F.c];
      double u[3], w[3], nr[3];
      for (int c = 0; c < 3; ++c) {
        u[c] = pb[c] - pa[c];
        w[c] = pc[c] - pa[c];
      }
      nr[0] = u[1] * w[2] - u[2] * w[1];
      nr[1] = u[2] * w[0] - u[0] * w[2];
      nr[2] = u[0] * w[1] - u[1] * w[0];
      const double l = std::sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
      const double area = 0.5 * l;
      double d = 0.0;
      for (int c = 0; c < 3; ++c) d += (centre[3 * G.tile + c] - centre[3 * F.tile + c]) * nr[c] / l;
      d = std::fabs(d);
      MT_CHECK(d > 0, MT_EINVAL, "mt_tiles_create_tetra: tiles %lld and %lld share a face but not its sides",
               (long long)F.tile, (long long)G.tile);
      nbr[6 * F.tile + F.slot] = (int32_t)G.tile;
      nbr[6 * G.tile + G.slot] = (int32_t)F.tile;
      coef[6 * F.tile + F.slot] = area / (vol[F.tile] * d);
      coef[6 * G.tile + G.slot] = area / (vol[G.tile] * d);
    }
    k = e;
  }
  // the cuboid path builds the tile set; then the tetrahedral parts replace
  // the geometry-dependent ones
  mt_tiles *t = nullptr;
  mt_status st = mt_tiles_create(ctx, n, centre.data(), edge.data(), Ms, Aex, Ku, axis, nullptr, &t);
  if (st != MT_OK) return st;
  t->kind = MT_TILE_TETRA;
  t->lattice = false;  // centroids may happen to sit on a lattice; the tiles are not cuboids
  std::vector<float> wex(6 * n, 0.0f);
  bool any = false;
  for (int64_t i = 0; i < n; ++i)
    for (int f = 0; f < 6; ++f)
      if (nbr[6 * i + f] >= 0) {
        wex[6 * i + f] = (float)(2.0 * Aex[i] / (MT_MU0 * Ms[i]) * coef[6 * i + f]);
        any = true;
      }
  double vt = 0.0;
  for (int64_t i = 0; i < n; ++i) vt += vol[i];
  std::vector<double> wvol(n);
  for (int64_t i = 0; i < n; ++i) wvol[i] = vol[i] / vt;
  t->vol_total = vt;
  t->has_exchange = any;
  t->nbr = nbr;
  if ((st = upload(&t->d_vert, vert.data(), 12 * n)) != MT_OK ||
      (st = copy_to(t->d_wex, wex.data(), 6 * n)) != MT_OK || (st = copy_to(t->d_nbr, nbr.data(), 6 * n)) != MT_OK ||
      (st = copy_to(t->d_wvol, wvol.data(), n)) != MT_OK) {
    mt::tiles_release(t);
    return st;
  }
  *out = t;
  return MT_OK;
}

void mt_tiles_destroy(mt_tiles *tiles) { mt::tiles_release(tiles); }

mt_status mt_demag_assemble(mt_tiles *tiles, mt_prec prec, mt_tensor **out) {
  return mt_demag_assemble_ex(tiles, prec, MT_LAYOUT_STREAM, out);
}

mt_status mt_demag_assemble_ex(mt_tiles *tiles, mt_prec prec, int layout, mt_tensor **out) {
  MT_CHECK(tiles && out, MT_EINVAL, "mt_demag_assemble: NULL argument");
  MT_CHECK(prec >= MT_F64 && prec <= MT_BF16_SPLIT, MT_EINVAL, "mt_demag_assemble: bad precision %d", (int)prec);
  MT_CHECK(layout == MT_LAYOUT_STREAM || layout == MT_LAYOUT_DENSE || layout == MT_LAYOUT_STREAM6 ||
               layout == MT_LAYOUT_STREAM_FULL || layout == MT_LAYOUT_STREAM_HALF,
           MT_EINVAL, "mt_demag_assemble: bad layout %d", layout);
  const bool allow_planar =
      layout == MT_LAYOUT_STREAM || layout == MT_LAYOUT_STREAM_FULL || layout == MT_LAYOUT_STREAM_HALF;
  const bool force_half = layout == MT_LAYOUT_STREAM_HALF;
  const bool allow_half = layout == MT_LAYOUT_STREAM || force_half;
  MT_CHECK(!force_half || (prec == MT_F32 && tiles->kind == MT_TILE_CUBOID), MT_EINVAL,
           "mt_demag_assemble: MT_LAYOUT_STREAM_HALF stores FP32 tensors of cuboid tiles only");
  if (layout != MT_LAYOUT_DENSE) layout = MT_LAYOUT_STREAM;
  MT_CHECK(layout == MT_LAYOUT_STREAM || prec == MT_BF16_SCALED || prec == MT_BF16_SPLIT, MT_EINVAL,
           "mt_demag_assemble: the dense layout stores BF16 or split BF16 only");
  mt_ctx *ctx = tiles->ctx;
  MT_CUDA(cudaSetDevice(ctx->device));
  mt_tensor *T = new mt_tensor();
  T->tiles = tiles;
  tiles->refs++;
  T->prec = prec;
  T->layout = layout;
  T->n = tiles->n;
  size_t data_bytes = 0, scale_bytes = 0;
  if (layout == MT_LAYOUT_DENSE) {
    // thread mapping of the assembly kernel: 16-row panels x 128-column chunks
    T->L.TR = 16;
    T->L.TC = 128;
    T->L.nplane = 9;
    T->L.elem_bytes = 2;
    T->L.P = (T->n + T->L.TR - 1) / T->L.TR;
    T->L.Q = (T->n + T->L.TC - 1) / T->L.TC;
    T->Kp = ((3 * T->n + 127) / 128) * 128;
    data_bytes = (size_t)T->Kp * T->Kp * 2 * (prec == MT_BF16_SPLIT ? 2 : 1);
  } else {
    mt::layout_for(prec, &T->L);
    // single-layer cuboid set (every tile: the same centre z and z edge): the
    // FP32 tensor's xz and yz entries vanish; 4 entry planes
    if (allow_planar && prec != MT_F64 && tiles->kind == MT_TILE_CUBOID) {
      bool planar = true;
      for (int64_t i = 1; i < tiles->n && planar; ++i)
        planar = tiles->centre[3 * i + 2] == tiles->centre[2] && tiles->edge[3 * i + 2] == tiles->edge[2];
      if (planar) mt::layout_for_planar(prec, &T->L);
    }
    T->L.P = (T->n + T->L.TR - 1) / T->L.TR;
    T->L.Q = (T->n + T->L.TC - 1) / T->L.TC;
    // FP32 tiles of one shape: the tensor is symmetric (N_ij = N_ji), so
    // only the upper triangle of chunks is stored (Sec. 3.2); by default
    // from kHalfMinTiles tiles on, where the half product is the faster one
    if (allow_half && prec == MT_F32 && tiles->kind == MT_TILE_CUBOID && (force_half || T->n > kHalfMinTiles)) {
      // one shape: equal edges to 1e-12 (as for the lattice test; the
      // tensor then differs from a symmetric one far below FP32 rounding)
      bool same = true;
      for (int64_t i = 1; i < tiles->n && same; ++i)
        for (int a = 0; a < 3; ++a)
          same = same && std::fabs(tiles->edge[3 * i + a] - tiles->edge[a]) <= 1e-12 * tiles->edge[a];
      T->L.half = same;
    }
    // an FP32 tensor stored half leaves out zz, which the trace gives
    // (traceless; checked on every block at assembly): 3 planes for a single
    // layer, 5 otherwise
    if (T->L.half && prec == MT_F32) mt::layout_for_traceless(&T->L, T->L.nplane == 4);
    if (force_half && !T->L.half) {
      delete T;
      mt::tiles_release(tiles);
      MT_CHECK(false, MT_EINVAL, "mt_demag_assemble: MT_LAYOUT_STREAM_HALF needs tiles of one shape");
    }
    T->L.CH = T->L.half ? half_chunks(T->L.P, T->L.Q, T->L.TC / T->L.TR) : T->L.P * T->L.Q;
    data_bytes = (size_t)T->L.CH * T->L.chunk_bytes();
    scale_bytes = (size_t)T->L.CH * T->L.scale_bytes_per_chunk;
  }
  T->bytes = data_bytes + scale_bytes;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->in_use + T->bytes > ctx->budget) {
      mt::set_error("mt_demag_assemble: %zu bytes exceed the context budget (%zu of %zu in use)", T->bytes,
                    ctx->in_use, ctx->budget);
      delete T;
      mt::tiles_release(tiles);
      return MT_ENOMEM;
    }
    ctx->in_use += T->bytes;
  }
  auto fail = [&](mt_status st) {
    free_tensor_mem(T);
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      ctx->in_use -= T->bytes;
    }
    delete T;
    mt::tiles_release(tiles);
    return st;
  };
  cudaError_t e = cudaMalloc(&T->d_data, data_bytes);
  if (e == cudaSuccess) e = cudaMemset(T->d_data, 0, data_bytes);
  if (e == cudaSuccess && scale_bytes) {
    e = cudaMalloc(&T->d_scale, scale_bytes);
    if (e == cudaSuccess) e = cudaMemset(T->d_scale, 0, scale_bytes);
  }
  if (e != cudaSuccess) return fail(mt::cuda_fail(e, "tensor allocation", __FILE__, __LINE__));
  mt_status st = mt::assemble(T);
  if (st != MT_OK) return fail(st);
  *out = T;
  return MT_OK;
}

void mt_tensor_destroy(mt_tensor *T) { mt::tensor_release(T); }

mt_status mt_tensor_get_info(const mt_tensor *T, mt_tensor_info *info) {
  MT_CHECK(T && info, MT_EINVAL, "mt_tensor_get_info: NULL argument");
  info->n = T->n;
  info->prec = T->prec;
  info->rows_per_panel = T->L.TR;
  info->cols_per_chunk = T->L.TC;
  info->layout = T->layout;
  info->planes = T->layout == MT_LAYOUT_DENSE ? 9 : T->L.nplane;  // sparse: as its source
  info->bytes = (int64_t)T->bytes;
  info->near_blocks = T->near_count;
  info->half = T->L.half ? 1 : 0;
  info->row_warps = T->layout == MT_LAYOUT_SPARSE ? T->sp_split : 0;
  return MT_OK;
}

mt_status mt_tensor_read_rows(const mt_tensor *T, int64_t i0, int64_t i1, double *out) {
  MT_CHECK(T && out, MT_EINVAL, "mt_tensor_read_rows: NULL argument");
  MT_CHECK(0 <= i0 && i0 <= i1 && i1 <= T->n, MT_EINVAL, "mt_tensor_read_rows: bad row range");
  if (T->layout == MT_LAYOUT_SPARSE) return mt::read_rows_sparse(T, i0, i1, out);
  return mt::read_rows(T, i0, i1, out);
}

mt_status mt_demag_blocks(mt_tiles *tiles, int64_t count, const int64_t *pairs, double *out) {
  MT_CHECK(tiles && count >= 0 && (count == 0 || (pairs && out)), MT_EINVAL, "mt_demag_blocks: bad argument");
  MT_CUDA(cudaSetDevice(tiles->ctx->device));
  return mt::blocks_fp64(tiles, count, pairs, out);
}

mt_status mt_demag_field(mt_tensor *T, const float *m, int B, float *H, void *stream) {
  MT_CHECK(T && m && H, MT_EINVAL, "mt_demag_field: NULL argument");
  MT_CHECK(B >= 1, MT_EINVAL, "mt_demag_field: B must be >= 1");
  MT_CHECK(T->prec != MT_F64, MT_EINVAL, "mt_demag_field: FP64 tensors use mt_demag_field_f64");
  mt_status st = ensure_workspace(T, B);
  if (st != MT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = demag_apply(T, m, B, H, s)) != MT_OK) return st;
  MT_CUDA(cudaGetLastError());
  return MT_OK;
}

mt_status mt_demag_field_f64(mt_tensor *T, const double *m, int B, double *H, void *stream) {
  MT_CHECK(T && m && H, MT_EINVAL, "mt_demag_field_f64: NULL argument");
  MT_CHECK(B >= 1, MT_EINVAL, "mt_demag_field_f64: B must be >= 1");
  MT_CHECK(T->prec == MT_F64, MT_EINVAL, "mt_demag_field_f64: needs an FP64 tensor");
  mt_status st = ensure_workspace(T, B);
  if (st != MT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  mt::launch_prep_xs_f64(T, m, B, reinterpret_cast<double *>(T->d_xs), s);
  mt::launch_matvec(T, T->d_xs, B, reinterpret_cast<float *>(H), T->d_part, T->d_count, nullptr,
                    T->tiles->ctx->d_status, s);
  MT_CUDA(cudaGetLastError());
  return MT_OK;
}

mt_status mt_llg_rhs(mt_tensor *T, const mt_llg_params *p, const float *m, int B, float *dmdt, float *tau,
                     void *stream) {
  MT_CHECK(T && p && m && dmdt && p->alpha && p->Ha, MT_EINVAL, "mt_llg_rhs: NULL argument");
  MT_CHECK(B >= 1, MT_EINVAL, "mt_llg_rhs: B must be >= 1");
  MT_CHECK(T->prec != MT_F64, MT_EINVAL, "mt_llg_rhs: the FP64 tensor serves field checks only");
  mt_status st = ensure_workspace(T, B);
  if (st != MT_OK) return st;
  std::vector<float> g1, g2, ha;
  std::vector<float> xsc;
  mt::llg_prefactors(p, B, g1, g2, ha, xsc);
  float *d_par = nullptr;
  MT_CUDA(cudaMalloc(&d_par, sizeof(float) * 6 * B));
  cudaStream_t s = (cudaStream_t)stream;
  MT_CUDA(cudaMemcpyAsync(d_par, g1.data(), sizeof(float) * B, cudaMemcpyHostToDevice, s));
  MT_CUDA(cudaMemcpyAsync(d_par + B, g2.data(), sizeof(float) * B, cudaMemcpyHostToDevice, s));
  MT_CUDA(cudaMemcpyAsync(d_par + 2 * B, ha.data(), sizeof(float) * 3 * B, cudaMemcpyHostToDevice, s));
  MT_CUDA(cudaMemcpyAsync(d_par + 5 * B, xsc.data(), sizeof(float) * B, cudaMemcpyHostToDevice, s));
  if ((st = demag_apply(T, m, B, T->d_Hd, s)) != MT_OK) return st;
  if (tau) MT_CUDA(cudaMemsetAsync(tau, 0, sizeof(float) * B, s));
  mt::launch_rhs_plain(T, m, T->d_Hd, B, d_par, d_par + B, d_par + 2 * B, d_par + 5 * B, dmdt, tau, s);
  MT_CUDA(cudaGetLastError());
  // the parameter block must outlive the kernels
  MT_CUDA(cudaStreamSynchronize(s));
  cudaFree(d_par);
  return MT_OK;
}

}  // extern "C"

namespace mt {

void tiles_release(mt_tiles *t) {
  if (t && --t->refs == 0) free_tiles(t);
}

void tensor_release(mt_tensor *T) {
  if (!T || --T->refs != 0) return;
  cudaDeviceSynchronize();
  free_tensor_mem(T);
  mt_tiles *tiles = T->tiles;
  {
    std::lock_guard<std::mutex> lk(tiles->ctx->mu);
    tiles->ctx->in_use -= T->bytes;
  }
  delete T;
  tiles_release(tiles);
}

}  // namespace mt

namespace mt {

// device bytes of a tensor of n tiles in a precision and layout (as allocated
// by mt_demag_assemble_ex)
size_t tensor_bytes_for(int64_t n, int prec, int layout) {
  if (layout == MT_LAYOUT_DENSE) {
    const size_t Kp = (size_t)((3 * n + 127) / 128) * 128;
    return Kp * Kp * 2 * (prec == MT_BF16_SPLIT ? 2 : 1);
  }
  mt_layout L;
  layout_for(prec, &L);
  L.P = (n + L.TR - 1) / L.TR;
  L.Q = (n + L.TC - 1) / L.TC;
  return (size_t)L.P * L.Q * (L.chunk_bytes() + L.scale_bytes_per_chunk);
}

}  // namespace mt

extern "C" mt_status mt_energy(mt_tensor *T, const mt_llg_params *p, const float *m, int B, double *E,
                               void *stream) {
  MT_CHECK(T && p && m && E && p->Ha, MT_EINVAL, "mt_energy: NULL argument");
  MT_CHECK(B >= 1, MT_EINVAL, "mt_energy: B must be >= 1");
  MT_CHECK(T->prec != MT_F64, MT_EINVAL, "mt_energy: the FP64 tensor serves field checks only");
  mt_status st = ensure_workspace(T, B);
  if (st != MT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<float> ha(4 * B);  // Ha, then the exchange factors
  for (int q = 0; q < 3 * B; ++q) ha[q] = (float)p->Ha[q];
  for (int b = 0; b < B; ++b) ha[3 * B + b] = p->exch_scale ? (float)p->exch_scale[b] : 1.0f;
  float *d_ha = nullptr;
  double *d_E = nullptr;
  MT_CUDA(cudaMalloc(&d_ha, sizeof(float) * 4 * B));
  MT_CUDA(cudaMalloc(&d_E, sizeof(double) * 4 * B));
  MT_CUDA(cudaMemcpyAsync(d_ha, ha.data(), sizeof(float) * 4 * B, cudaMemcpyHostToDevice, s));
  MT_CUDA(cudaMemsetAsync(d_E, 0, sizeof(double) * 4 * B, s));
  if ((st = demag_apply(T, m, B, T->d_Hd, s)) != MT_OK) return st;
  mt::launch_energy(T, m, T->d_Hd, B, d_ha, d_ha + 3 * B, d_E, s);
  MT_CUDA(cudaGetLastError());
  std::vector<double> e4(4 * B);
  MT_CUDA(cudaMemcpyAsync(e4.data(), d_E, sizeof(double) * 4 * B, cudaMemcpyDeviceToHost, s));
  MT_CUDA(cudaStreamSynchronize(s));
  cudaFree(d_ha);
  cudaFree(d_E);
  for (int b = 0; b < B; ++b) {
    E[5 * b + 1] = e4[4 * b];
    E[5 * b + 2] = e4[4 * b + 1];
    E[5 * b + 3] = e4[4 * b + 2];
    E[5 * b + 4] = e4[4 * b + 3];
    E[5 * b] = e4[4 * b] + e4[4 * b + 1] + e4[4 * b + 2] + e4[4 * b + 3];
  }
  return MT_OK;
}

namespace {
// A wait that can never complete (one expected arrival, none comes), bounded
// by limit_ns: exercises the give-up path every pipelined kernel relies on.
__global__ void k_wait_selftest(int *status, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mtd::mbar_init(&bar, 1);
    mtd::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mtd::mbar_wait_bounded(&bar, 0u, status, limit_ns);
}
}  // namespace

extern "C" mt_status mt_selftest_wait_timeout(mt_ctx *ctx, double limit_s) {
  MT_CHECK(ctx && limit_s > 0 && limit_s <= 10.0, MT_EINVAL, "mt_selftest_wait_timeout: limit in (0, 10] s");
  MT_CUDA(cudaSetDevice(ctx->device));
  int *d = nullptr;
  MT_CUDA(cudaMalloc(&d, sizeof(int)));
  MT_CUDA(cudaMemset(d, 0, sizeof(int)));
  k_wait_selftest<<<1, 32>>>(d, (uint64_t)(limit_s * 1e9));
  MT_CUDA(cudaGetLastError());
  int h = 0;
  MT_CUDA(cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost));
  cudaFree(d);
  if (h == MT_DEV_TIMEOUT) {
    mt::set_error("mt_selftest_wait_timeout: the bounded wait gave up as designed");
    return MT_ETIMEOUT;
  }
  mt::set_error("mt_selftest_wait_timeout: the wait did not report a timeout");
  return MT_ECUDA;
}
