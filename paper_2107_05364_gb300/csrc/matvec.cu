// Streaming demag product H_d = -N (Ms m) (Eq. 9, Eq. 17 of the paper).
//
// The product is bound by HBM: every stored tensor value is read once per
// right-hand side and used for 1.5 multiply-adds on average.  Design:
//   * one persistent CTA per SM; the (simulation group, panel, chunk) units
//     are split evenly over the CTAs in storage order ("stream-K"), so every
//     CTA streams one contiguous stretch of the tensor and the load is
//     balanced to within one chunk whatever n is; a group of up to 4
//     simulations shares each chunk read (a batch of B reads the tensor
//     ceil(B / 4) times, not B times);
//   * a producer warp moves each chunk (48 KB, all 6 planes of TR x TC blocks)
//     and the matching slice of the Ms-scaled magnetisation into a 4-stage
//     shared-memory ring with bulk TMA copies (cp.async.bulk + mbarrier
//     transaction counts); the tensor stream is marked evict-first in L2, the
//     small operand evict-last;
//   * consumer warps own TR/W rows each; a lane owns VEC adjacent columns and
//     keeps its operand values in registers while it walks the rows, so each
//     tensor value is read from shared memory once, as a 16-byte vector;
//   * a panel split between two CTAs is finished by whichever warp arrives
//     last (counter per panel and warp): it sums the partial rows in CTA
//     order, so the result does not depend on timing;
//   * before waiting on the kernel ahead of it (which writes the operand,
//     never the tensor), each CTA prefetches its first chunks into L2.
// A tensor of tiles of one shape is symmetric and stored as its upper
// triangle (Sec. 3.2); k_matvec_half and k_half_cols below apply it, each
// stored chunk above the diagonal also to its columns.
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "mt_internal.cuh"

namespace {

// FP32 / scaled-BF16 tensors of a single-layer tile set: the xz and yz
// planes are not stored (they vanish by mirror symmetry), planes xx, xy, yy,
// zz
constexpr int kF32Planar = 4;
constexpr int kBF16Planar = 5;
constexpr int kSplitPlanar = 6;  // hi planes xx, xy, yy, zz, then the lo planes
// FP32 tensor of a single-layer tile set stored half: planes xx, xy, yy
// (zz = delta_ij - xx - yy, the trace; see traceless in mt_internal.cuh)
constexpr int kF32Traceless = 7;
// FP32 tensor of a tile set of one shape stored half, not single-layer:
// planes xx, xy, xz, yy, yz (zz from the trace)
constexpr int kF32Traceless5 = 8;

template <int PREC>
struct MvCfg;
template <>
struct MvCfg<MT_F32> {
  using T = float;
  using Acc = float;
  static constexpr int TR = 16, TC = 128, NPLANE = 6, VEC = 4, W = 4, STAGES = 4;
  static constexpr bool SCALED = false, PLANAR = false;
};
template <>
struct MvCfg<kF32Planar> {
  using T = float;
  using Acc = float;
  // 16-row panels of 32 KB chunks, 6 in the ring.  32-row panels (64 KB
  // chunks) timed faster alone (0.234 against 0.248 ms at n = 10,000) but
  // slower inside the step graph (1.450 against 1.397 ms per attempt)
  static constexpr int TR = 16, TC = 128, NPLANE = 4, VEC = 4, W = 4, STAGES = 6;
  static constexpr bool SCALED = false, PLANAR = true;
};
template <>
struct MvCfg<kF32Traceless> {
  using T = float;
  using Acc = float;
  // 24 KB chunks: 8 in the ring
  static constexpr int TR = 16, TC = 128, NPLANE = 3, VEC = 4, W = 4, STAGES = 8;
  static constexpr bool SCALED = false, PLANAR = true;
};
template <>
struct MvCfg<kF32Traceless5> {
  using T = float;
  using Acc = float;
  // 40 KB chunks: 5 in the ring
  static constexpr int TR = 16, TC = 128, NPLANE = 5, VEC = 4, W = 4, STAGES = 5;
  static constexpr bool SCALED = false, PLANAR = false;
};
template <>
struct MvCfg<MT_F64> {
  using T = double;
  using Acc = double;
  static constexpr int TR = 16, TC = 64, NPLANE = 6, VEC = 2, W = 4, STAGES = 4;
  static constexpr bool SCALED = false, PLANAR = false;
};
template <>
struct MvCfg<MT_BF16_SCALED> {
  using T = __nv_bfloat16;
  using Acc = float;
  static constexpr int TR = 16, TC = 256, NPLANE = 6, VEC = 8, W = 4, STAGES = 4;
  static constexpr bool SCALED = true, PLANAR = false;
};
template <>
struct MvCfg<kBF16Planar> {
  using T = __nv_bfloat16;
  using Acc = float;
  static constexpr int TR = 16, TC = 256, NPLANE = 4, VEC = 8, W = 4, STAGES = 5;
  static constexpr bool SCALED = true, PLANAR = true;
};
template <>
struct MvCfg<kSplitPlanar> {
  using T = __nv_bfloat16;
  using Acc = float;
  static constexpr int TR = 8, TC = 256, NPLANE = 8, VEC = 8, W = 4, STAGES = 6;
  static constexpr bool SCALED = false, PLANAR = true;
};
template <>
struct MvCfg<MT_BF16_SPLIT> {
  using T = __nv_bfloat16;
  using Acc = float;
  static constexpr int TR = 8, TC = 256, NPLANE = 12, VEC = 8, W = 4, STAGES = 4;
  static constexpr bool SCALED = false, PLANAR = false;
};

template <int PREC, int SB>
struct MvShape {
  using C = MvCfg<PREC>;
  static constexpr int NCW = C::W;         // consumer warps
  static constexpr int RPW = C::TR / NCW;  // rows per consumer warp
  static constexpr int DATA_BYTES = C::NPLANE * C::TR * C::TC * (int)sizeof(typename C::T);
  static constexpr int SCALE_BYTES = C::SCALED ? C::TR * C::TC : 0;
  static constexpr int XS_BYTES = 3 * C::TC * (int)sizeof(typename C::Acc);  // one simulation's slice
  static constexpr int STAGE_BYTES = DATA_BYTES + SCALE_BYTES + SB * XS_BYTES;
  // ring depth: up to C::STAGES within 226 KB of shared memory (the
  // barriers and the abort flag fill the rest of the 227 KB a CTA may have)
  static constexpr int STAGES =
      (C::STAGES * STAGE_BYTES <= 226 * 1024) ? C::STAGES : (226 * 1024) / STAGE_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 2 * STAGES * 8 + 16;
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory of one CTA");
  static constexpr int THREADS = (NCW + 1) * 32;
  static_assert(STAGES >= 2, "at least a double-buffered ring");
  static_assert(C::TR % NCW == 0, "whole rows per warp");
  static_assert(C::TC == 32 * C::VEC, "a warp covers one chunk row");
  static_assert(3 * RPW <= 32, "one lane per (row, component) in the flush");
  static_assert(DATA_BYTES % 16 == 0 && SCALE_BYTES % 16 == 0 && XS_BYTES % 16 == 0, "bulk copy sizes");
};

// ---- per-precision load of VEC adjacent values of one plane row ----------
template <int PREC>
__device__ __forceinline__ void load_vals(const unsigned char *stage, int plane, int row, int lane,
                                          typename MvCfg<PREC>::Acc v[MvCfg<PREC>::VEC]) {
  using C = MvCfg<PREC>;
  if constexpr (PREC == MT_F32 || PREC == kF32Planar || PREC == kF32Traceless || PREC == kF32Traceless5) {
    const float4 a = reinterpret_cast<const float4 *>(stage)[(plane * C::TR + row) * (C::TC / 4) + lane];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else if constexpr (PREC == MT_F64) {
    const double2 a = reinterpret_cast<const double2 *>(stage)[(plane * C::TR + row) * (C::TC / 2) + lane];
    v[0] = a.x; v[1] = a.y;
  } else if constexpr (PREC == MT_BF16_SCALED || PREC == kBF16Planar) {
    const uint4 a = reinterpret_cast<const uint4 *>(stage)[(plane * C::TR + row) * (C::TC / 8) + lane];
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&a);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __bfloat1622float2(h[k]);
      v[2 * k] = f.x;
      v[2 * k + 1] = f.y;
    }
  } else {  // split: hi plane `plane`, lo plane `plane + NPLANE / 2`
    const uint4 a = reinterpret_cast<const uint4 *>(stage)[(plane * C::TR + row) * (C::TC / 8) + lane];
    const uint4 b =
        reinterpret_cast<const uint4 *>(stage)[((plane + C::NPLANE / 2) * C::TR + row) * (C::TC / 8) + lane];
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&a);
    const __nv_bfloat162 *l = reinterpret_cast<const __nv_bfloat162 *>(&b);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 fh = __bfloat1622float2(h[k]);
      const float2 fl = __bfloat1622float2(l[k]);
      v[2 * k] = fh.x + fl.x;
      v[2 * k + 1] = fh.y + fl.y;
    }
  }
}

template <int PREC>
__device__ __forceinline__ void load_xs(const unsigned char *xs, int comp, int lane,
                                        typename MvCfg<PREC>::Acc v[MvCfg<PREC>::VEC]) {
  using C = MvCfg<PREC>;
  if constexpr (PREC == MT_F64) {
    const double2 a = reinterpret_cast<const double2 *>(xs)[comp * (C::TC / 2) + lane];
    v[0] = a.x; v[1] = a.y;
  } else {
    const float4 *p = reinterpret_cast<const float4 *>(xs) + comp * (C::TC / 4) + lane * (C::VEC / 4);
#pragma unroll
    for (int k = 0; k < C::VEC / 4; ++k) {
      const float4 a = p[k];
      v[4 * k] = a.x; v[4 * k + 1] = a.y; v[4 * k + 2] = a.z; v[4 * k + 3] = a.w;
    }
  }
}

struct MvArgs {
  const void *tensor;
  const int8_t *scale;
  const void *xs;
  void *H;
  void *part;
  int *count;
  const int *active;
  int *status;
  int64_t n, P, Q;
  int64_t CH;  // stored chunks
  int B;
};


// Units in storage order: (group of simulations g, stored chunk c) with c
// the chunk (panel p, column chunk q) = p Q + q.
struct UnitCursor {
  int64_t g, p, q, c;
};
__device__ __forceinline__ void unit_decode(const MvArgs &A, int64_t u, UnitCursor &cu) {
  cu.g = u / A.CH;
  cu.c = u - cu.g * A.CH;
  cu.p = cu.c / A.Q;
  cu.q = cu.c - cu.p * A.Q;
}
__device__ __forceinline__ void unit_next(const MvArgs &A, UnitCursor &cu) {
  ++cu.c;
  if (++cu.q == A.Q) {
    ++cu.p;
    cu.q = 0;
  }
  if (cu.c == A.CH) {
    cu.c = 0;
    ++cu.g;
    cu.p = 0;
  }
}

// SB simulations share every chunk read: unit = (group of SB simulations,
// panel, chunk); the stage holds the chunk and the group's SB operand slices
// and each tensor value is used for all of them.  (Members of a last, partial
// group beyond B read simulation 0's slice and are not written.)
__device__ __forceinline__ bool group_live(const MvArgs &A, int64_t g, int SB) {
  if (!A.active) return true;
  for (int s = 0; s < SB; ++s) {
    const int64_t b = g * SB + s;
    if (b < A.B && A.active[b]) return true;
  }
  return false;
}

template <int PREC, int SB>
__global__ void __launch_bounds__(MvShape<PREC, SB>::THREADS, 1) k_matvec(MvArgs A) {
  using C = MvCfg<PREC>;
  using S = MvShape<PREC, SB>;
  using Acc = typename C::Acc;
  {
    // before waiting on the previous kernel (which writes the operand, not
    // the tensor): the CTA's first ring-full of tensor chunks into L2
    const int64_t G = gridDim.x, NG = (A.B + SB - 1) / SB, U = NG * A.CH;
    const int64_t u0 = mtd::sk_begin(blockIdx.x, U, G), u1 = mtd::sk_begin(blockIdx.x + 1, U, G);
    const int64_t c0 = u0 % A.CH;
    if (threadIdx.x < S::STAGES && u0 + threadIdx.x < u1 && c0 + threadIdx.x < A.CH)
      mtd::bulk_prefetch_l2(reinterpret_cast<const unsigned char *>(A.tensor) + (size_t)(c0 + threadIdx.x) * S::DATA_BYTES,
                            S::DATA_BYTES);
  }
  mtd::pdl_enter();
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + S::STAGES * S::STAGE_BYTES);
  uint64_t *empty = full + S::STAGES;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + S::STAGES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = gridDim.x, k = blockIdx.x;
  const int64_t NG = (A.B + SB - 1) / SB;
  const int64_t U = NG * A.CH;
  const int64_t u0 = mtd::sk_begin(k, U, G), u1 = mtd::sk_begin(k + 1, U, G);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S::STAGES; ++s) {
      mtd::mbar_init(&full[s], 1);
      mtd::mbar_init(&empty[s], S::NCW);
    }
    *abort_flag = 0;
    mtd::fence_mbar_init();
  }
  __syncthreads();

  if (warp == S::NCW) {
    // ---------------- producer ----------------
    if (lane == 0) {
      const uint64_t pol_stream = mtd::policy_evict_first();
      const uint64_t pol_keep = mtd::policy_evict_last();
      const unsigned char *tens = reinterpret_cast<const unsigned char *>(A.tensor);
      const unsigned char *xs = reinterpret_cast<const unsigned char *>(A.xs);
      int it = 0;
      UnitCursor cu;
      unit_decode(A, u0, cu);
      for (int64_t u = u0; u < u1; ++u, unit_next(A, cu)) {
        const int64_t g = cu.g, q = cu.q;
        if (!group_live(A, g, SB)) continue;
        const int s = it % S::STAGES;
        const uint32_t ph = (uint32_t)(it / S::STAGES) & 1u;
        if (it >= S::STAGES) {
          if (*abort_flag || !mtd::mbar_wait_bounded(&empty[s], ph ^ 1u, A.status)) {
            *abort_flag = 1;
            break;
          }
        }
        unsigned char *st = smem + (size_t)s * S::STAGE_BYTES;
        mtd::mbar_arrive_expect_tx(&full[s], S::STAGE_BYTES);
        mtd::bulk_g2s(st, tens + (size_t)cu.c * S::DATA_BYTES, S::DATA_BYTES, &full[s], pol_stream);
        if constexpr (C::SCALED)
          mtd::bulk_g2s(st + S::DATA_BYTES, A.scale + (size_t)cu.c * S::SCALE_BYTES, S::SCALE_BYTES, &full[s],
                        pol_stream);
#pragma unroll
        for (int m = 0; m < SB; ++m) {
          const int64_t b = g * SB + m < A.B ? g * SB + m : 0;
          mtd::bulk_g2s(st + S::DATA_BYTES + S::SCALE_BYTES + m * S::XS_BYTES,
                        xs + (size_t)(b * A.Q + q) * S::XS_BYTES, S::XS_BYTES, &full[s], pol_keep);
        }
        ++it;
      }
      // drain: every copy issued must have landed before the CTA may exit
      for (int s = 0; s < S::STAGES && s < it; ++s) {
        const int last = it - 1 - ((it - 1 - s) % S::STAGES);  // last issue on stage s
        mtd::mbar_wait_bounded(&full[s], (uint32_t)(last / S::STAGES) & 1u, A.status);
      }
    }
    return;
  }

  // ---------------- consumers ----------------
  Acc acc[SB][S::RPW][3];
  int64_t gp_cur = -1;
  int it = 0;
  bool aborted = false;

  auto flush = [&](int64_t gp) {
    // lane sums -> every lane holds the warp totals
#pragma unroll
    for (int m = 0; m < SB; ++m)
#pragma unroll
      for (int r = 0; r < S::RPW; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[m][r][c] = mtd::warp_sum(acc[m][r][c]);
    const int64_t g = gp / A.P, p = gp - g * A.P;
    const int64_t pu0 = g * A.CH + p * A.Q, pu1 = pu0 + A.Q;  // the panel's units
    const int64_t kf = mtd::sk_owner(pu0, U, G), kl = mtd::sk_owner(pu1 - 1, U, G);
    // this lane's (row, component)
    const int lr = lane / 3, lc = lane - 3 * (lane / 3);
    Acc mine[SB];
#pragma unroll
    for (int m = 0; m < SB; ++m) {
      mine[m] = 0;
#pragma unroll
      for (int r = 0; r < S::RPW; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (r == lr && c == lc) mine[m] = acc[m][r][c];
    }
    const int row_in_panel = warp * S::RPW + lr;
    const int64_t row = p * C::TR + row_in_panel;
    Acc *part = reinterpret_cast<Acc *>(A.part);
    const bool writer = lane < 3 * S::RPW;
    auto out = [&](int m) -> Acc * {
      const int64_t b = g * SB + m;
      return (b < A.B && (!A.active || A.active[b])) ? reinterpret_cast<Acc *>(A.H) + (size_t)b * 3 * A.n : nullptr;
    };
    if (kf == kl) {
      if (writer && row < A.n)
#pragma unroll
        for (int m = 0; m < SB; ++m)
          if (Acc *H = out(m)) H[3 * row + lc] = -mine[m];
      return;
    }
    const int64_t slot = (u0 >= pu0) ? 2 * k : 2 * k + 1;  // this CTA starts inside the panel: its first
    if (writer)
#pragma unroll
      for (int m = 0; m < SB; ++m) part[((slot * SB + m) * C::TR + row_in_panel) * 3 + lc] = mine[m];
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane == 0) {
      const int old = atomicAdd(&A.count[gp * S::NCW + warp], 1);
      last = (old == (int)(kl - kf));
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence();
      if (writer) {
        // the parts in CTA order, each CTA's simulations loaded together
        Acc tot[SB];
#pragma unroll
        for (int m = 0; m < SB; ++m) tot[m] = 0;
        for (int64_t kk = kf; kk <= kl; ++kk) {
          // slot of CTA kk: 2 kk if this panel is its first, else 2 kk + 1
          const int64_t sl = (mtd::sk_begin(kk, U, G) >= pu0) ? 2 * kk : 2 * kk + 1;
#pragma unroll
          for (int m = 0; m < SB; ++m) tot[m] += __ldcg(&part[((sl * SB + m) * C::TR + row_in_panel) * 3 + lc]);
        }
#pragma unroll
        for (int m = 0; m < SB; ++m) {
          Acc *H = out(m);
          if (H && row < A.n) H[3 * row + lc] = -tot[m];
        }
      }
      if (lane == 0) A.count[gp * S::NCW + warp] = 0;  // ready for the next launch
    }
  };

  UnitCursor cu;
  unit_decode(A, u0, cu);
  for (int64_t u = u0; u < u1; ++u, unit_next(A, cu)) {
    const int64_t g = cu.g, gp = g * A.P + cu.p;
    if (!group_live(A, g, SB)) continue;
    if (gp != gp_cur) {
      if (gp_cur >= 0) flush(gp_cur);
      gp_cur = gp;
#pragma unroll
      for (int m = 0; m < SB; ++m)
#pragma unroll
        for (int r = 0; r < S::RPW; ++r) acc[m][r][0] = acc[m][r][1] = acc[m][r][2] = 0;
    }
    const int s = it % S::STAGES;
    const uint32_t ph = (uint32_t)(it / S::STAGES) & 1u;
    ++it;
    if (!aborted) {
      if (*abort_flag || !mtd::mbar_wait_bounded(&full[s], ph, A.status)) {
        aborted = true;
        *abort_flag = 1;
      }
    }
    if (!aborted) {
      const unsigned char *st = smem + (size_t)s * S::STAGE_BYTES;
      Acc X[SB][C::VEC], Y[SB][C::VEC], Z[SB][C::VEC];
#pragma unroll
      for (int m = 0; m < SB; ++m) {
        const unsigned char *xsm = st + S::DATA_BYTES + S::SCALE_BYTES + m * S::XS_BYTES;
        load_xs<PREC>(xsm, 0, lane, X[m]);
        load_xs<PREC>(xsm, 1, lane, Y[m]);
        load_xs<PREC>(xsm, 2, lane, Z[m]);
      }
#pragma unroll
      for (int r = 0; r < S::RPW; ++r) {
        const int row = warp * S::RPW + r;
        if constexpr (C::PLANAR) {
          Acc nxx[C::VEC], nxy[C::VEC], nyy[C::VEC], nzz[C::VEC];
          load_vals<PREC>(st, 0, row, lane, nxx);
          load_vals<PREC>(st, 1, row, lane, nxy);
          load_vals<PREC>(st, 2, row, lane, nyy);
          load_vals<PREC>(st, 3, row, lane, nzz);
          if constexpr (C::SCALED) {
            // per-block power-of-two scale: value = stored * 2^s
            const uint2 sc = reinterpret_cast<const uint2 *>(st + S::DATA_BYTES)[row * (C::TC / 8) + lane];
            const int8_t *e8 = reinterpret_cast<const int8_t *>(&sc);
#pragma unroll
            for (int v = 0; v < C::VEC; ++v) {
              const float f = __int_as_float(((int)e8[v] + 127) << 23);
              nxx[v] *= f;
              nxy[v] *= f;
              nyy[v] *= f;
              nzz[v] *= f;
            }
          }
#pragma unroll
          for (int m = 0; m < SB; ++m) {
            Acc sx = 0, sy = 0, sz = 0;
#pragma unroll
            for (int v = 0; v < C::VEC; ++v) {
              sx = fma(nxx[v], X[m][v], fma(nxy[v], Y[m][v], sx));
              sy = fma(nxy[v], X[m][v], fma(nyy[v], Y[m][v], sy));
              sz = fma(nzz[v], Z[m][v], sz);
            }
            acc[m][r][0] += sx;
            acc[m][r][1] += sy;
            acc[m][r][2] += sz;
          }
          continue;
        }
        Acc nxx[C::VEC], nxy[C::VEC], nxz[C::VEC], nyy[C::VEC], nyz[C::VEC], nzz[C::VEC];
        load_vals<PREC>(st, 0, row, lane, nxx);
        load_vals<PREC>(st, 1, row, lane, nxy);
        load_vals<PREC>(st, 2, row, lane, nxz);
        load_vals<PREC>(st, 3, row, lane, nyy);
        load_vals<PREC>(st, 4, row, lane, nyz);
        load_vals<PREC>(st, 5, row, lane, nzz);
        if constexpr (C::SCALED) {
          // per-block power-of-two scale: value = stored * 2^s
          const uint2 sc = reinterpret_cast<const uint2 *>(st + S::DATA_BYTES)[row * (C::TC / 8) + lane];
          const int8_t *e8 = reinterpret_cast<const int8_t *>(&sc);
#pragma unroll
          for (int v = 0; v < C::VEC; ++v) {
            const float f = __int_as_float(((int)e8[v] + 127) << 23);
            nxx[v] *= f;
            nxy[v] *= f;
            nxz[v] *= f;
            nyy[v] *= f;
            nyz[v] *= f;
            nzz[v] *= f;
          }
        }
#pragma unroll
        for (int m = 0; m < SB; ++m) {
          Acc sx = 0, sy = 0, sz = 0;
#pragma unroll
          for (int v = 0; v < C::VEC; ++v) {
            sx = fma(nxx[v], X[m][v], fma(nxy[v], Y[m][v], fma(nxz[v], Z[m][v], sx)));
            sy = fma(nxy[v], X[m][v], fma(nyy[v], Y[m][v], fma(nyz[v], Z[m][v], sy)));
            sz = fma(nxz[v], X[m][v], fma(nyz[v], Y[m][v], fma(nzz[v], Z[m][v], sz)));
          }
          acc[m][r][0] += sx;
          acc[m][r][1] += sy;
          acc[m][r][2] += sz;
        }
      }
    }
    __syncwarp();
    if (lane == 0) mtd::mbar_arrive(&empty[s]);
  }
  if (gp_cur >= 0) flush(gp_cur);
}

// ===========================================================================
// Half-stored tensors (tiles of one shape, N_ij = N_ji; order: half_gbase).
// k_matvec_half streams the stored chunks in order, a group of K chunks at a
// time: the K panels of super-row R against column chunk q.  Each chunk is
// applied to its rows; a group above the diagonal (q > R) is applied,
// transposed, to its columns too.  Its K chunks arrive one after the other,
// so a thread keeps its columns' sums over the whole group in registers, and
// the consumer warps meet once per group (not per chunk) to add them.  A
// group's column sums go to the work area (a group split between two CTAs
// is finished by the last of them to arrive, adding the parts in CTA
// order); k_half_cols then adds, for each column chunk q, the sums of the
// groups (R, q), R < q, in order of R and subtracts them from H.  Up to 2
// simulations share a chunk read (more take several passes: their row
// sums would not fit the registers).
// chunks a half-product CTA prefetches into L2 before the PDL wait
constexpr int kHalfPrefetch = 18;

template <int PREC, int SB>
struct HalfShape {
  using C = MvCfg<PREC>;
  static constexpr int K = C::TC / C::TR;  // panels per super-row
  static constexpr int NCW = 2 * C::W;     // consumer warps
  static constexpr int RPW = C::TR / NCW;  // rows of each panel per warp
  static constexpr int DATA_BYTES = C::NPLANE * C::TR * C::TC * 4;
  static constexpr int XS_BYTES = 3 * C::TC * 4;
  static constexpr int STAGE_BYTES = DATA_BYTES + SB * XS_BYTES;
  static constexpr int CB_BYTES = NCW * SB * 3 * C::TC * 4;  // the warps' column sums of a group
  static constexpr int XI_BYTES = NCW * SB * K * RPW * 16;   // each warp's row operand (x, y, z, 0)
  static constexpr int STAGES = (C::STAGES * STAGE_BYTES + CB_BYTES + XI_BYTES <= 226 * 1024)
                                    ? C::STAGES
                                    : (226 * 1024 - CB_BYTES - XI_BYTES) / STAGE_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + CB_BYTES + XI_BYTES + 2 * STAGES * 8 + 16;
  static constexpr int THREADS = (NCW + 1) * 32;
  static constexpr int NV = K * RPW * 3;  // row values a warp holds per simulation
  static constexpr int NVAL = SB * RPW * 3;        // a warp's row values per chunk
  static constexpr int NSLOT = NVAL <= 8 ? 8 : 16;  // padded for the reduce-scatter
  static_assert(SB == 1 || SB == 2, "one or two simulations per chunk read");
  static_assert(C::VEC == 4 && C::TC == 32 * C::VEC && C::TR % NCW == 0, "float4 columns, whole rows per warp");
  static_assert((NCW * 32) % C::TC == 0 && NV <= 64 && 16 * SB <= 32, "flush and operand lanes");
  static_assert(STAGES >= 2 && SMEM_BYTES <= 227 * 1024, "ring within one CTA's shared memory");
};

// Sums over the warp's lanes of NS values (NS a power of two <= 32), scattered:
// lane l returns the total of value l / (32 / NS).  Recursive halving: at the
// step with offset o a lane keeps the upper half of its values if (l & o),
// else the lower half, and adds its partner's copy of them; once one value is
// left the remaining offsets add it whole.
template <int NS>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[NS], int lane) {
  static_assert(NS >= 1 && NS <= 32 && (NS & (NS - 1)) == 0, "a power of two up to 32");
  int o = 16;
#pragma unroll
  for (int cnt = NS / 2; cnt >= 1; cnt /= 2, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < cnt; ++i) {
      const float send = up ? v[i] : v[cnt + i];
      const float keep = up ? v[cnt + i] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  return v[0];
}

struct HalfArgs {
  const float *tensor;
  const float *xs;   // [b][q][3][TC], Ms m
  float *H;
  float *part;       // row partials of super-rows shared by CTAs [2 G][SB][K TR][3]
  int *count;        // arrival counters per (simulation group, super-row, warp)
  int *gcount;       // arrival counters per (simulation group, group)
  float *colpart;    // column sums of every group above the diagonal [NG][NGR][SB][3][TC]
  float *colsplit;   // parts of the groups shared by CTAs [2 G][SB][3][TC]
  const int *active;
  int *status;
  int64_t n, P, Q, CH, NGR;  // NGR = Q (Q + 1) / 2 groups
  int B;
};

__device__ __forceinline__ bool half_live(const HalfArgs &A, int64_t g, int SB) {
  if (!A.active) return true;
  for (int s = 0; s < SB; ++s) {
    const int64_t b = g * SB + s;
    if (b < A.B && A.active[b]) return true;
  }
  return false;
}

// (simulation group g, group gi = (super-row R, column chunk q)) in storage
// order; a group's first unit is g CH + K gi, its length K except for the
// last group (the last super-row's diagonal), CH - K (NGR - 1)
struct GroupCursor {
  int64_t g, R, q, gi;
};
template <int K>
__device__ __forceinline__ int64_t group_decode(const HalfArgs &A, int64_t u, GroupCursor &gc) {
  gc.g = u / A.CH;
  const int64_t c = u - gc.g * A.CH;
  gc.gi = c / K;
  int64_t lo = 0, hi = A.Q - 1;  // the last super-row whose first group is <= gi
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (half_gbase(mid, A.Q) <= gc.gi) lo = mid;
    else hi = mid - 1;
  }
  gc.R = lo;
  gc.q = lo + (gc.gi - half_gbase(lo, A.Q));
  return u - (c - K * gc.gi);  // the group's first unit
}
__device__ __forceinline__ void group_next(const HalfArgs &A, GroupCursor &gc) {
  ++gc.gi;
  if (++gc.q == A.Q) {
    ++gc.R;
    gc.q = gc.R;
  }
  if (gc.gi == A.NGR) {
    gc.gi = 0;
    ++gc.g;
    gc.R = 0;
    gc.q = 0;
  }
}
template <int K>
__device__ __forceinline__ int group_len(const HalfArgs &A, const GroupCursor &gc) {
  return gc.gi == A.NGR - 1 ? (int)(A.CH - (int64_t)K * (A.NGR - 1)) : K;
}

template <int PREC, int SB>
__global__ void __launch_bounds__(HalfShape<PREC, SB>::THREADS, 1) k_matvec_half(HalfArgs A) {
  using C = MvCfg<PREC>;
  using S = HalfShape<PREC, SB>;
  constexpr int K = S::K, TR = C::TR, TC = C::TC;
  {
    // before waiting on the previous kernel (which writes the operand, not
    // the tensor): the CTA's first ring-full of tensor chunks into L2
    const int64_t G = gridDim.x, NG = (A.B + SB - 1) / SB, U = NG * A.CH;
    const int64_t u0 = mtd::sk_begin(blockIdx.x, U, G), u1 = mtd::sk_begin(blockIdx.x + 1, U, G);
    const int64_t c0 = u0 % A.CH;
    if (threadIdx.x < kHalfPrefetch && u0 + threadIdx.x < u1 && c0 + threadIdx.x < A.CH)
      mtd::bulk_prefetch_l2(reinterpret_cast<const unsigned char *>(A.tensor) + (size_t)(c0 + threadIdx.x) * S::DATA_BYTES,
                            S::DATA_BYTES);
  }
  mtd::pdl_enter();
  extern __shared__ __align__(128) unsigned char smem[];
  float *cb = reinterpret_cast<float *>(smem + S::STAGES * S::STAGE_BYTES);
  float4 *xi_all = reinterpret_cast<float4 *>(smem + S::STAGES * S::STAGE_BYTES + S::CB_BYTES);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + S::STAGES * S::STAGE_BYTES + S::CB_BYTES + S::XI_BYTES);
  uint64_t *empty = full + S::STAGES;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + S::STAGES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = gridDim.x, kcta = blockIdx.x;
  const int64_t NG = (A.B + SB - 1) / SB;
  const int64_t U = NG * A.CH;
  const int64_t u0 = mtd::sk_begin(kcta, U, G), u1 = mtd::sk_begin(kcta + 1, U, G);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S::STAGES; ++s) {
      mtd::mbar_init(&full[s], 1);
      mtd::mbar_init(&empty[s], S::NCW);
    }
    *abort_flag = 0;
    mtd::fence_mbar_init();
  }
  __syncthreads();

  if (warp == S::NCW) {
    // ---------------- producer: the CTA's units in storage order ----------------
    if (lane == 0) {
      const uint64_t pol_stream = mtd::policy_evict_first();
      const uint64_t pol_keep = mtd::policy_evict_last();
      const unsigned char *tens = reinterpret_cast<const unsigned char *>(A.tensor);
      const unsigned char *xs = reinterpret_cast<const unsigned char *>(A.xs);
      int it = 0;
      GroupCursor gc;
      bool stop = false;
      for (int64_t gs = group_decode<K>(A, u0, gc); gs < u1 && !stop; gs += group_len<K>(A, gc), group_next(A, gc)) {
        if (!half_live(A, gc.g, SB)) continue;
        const int len = group_len<K>(A, gc);
        const int kb = (int)(u0 > gs ? u0 - gs : 0), ke = (int)(u1 - gs < len ? u1 - gs : len);
        for (int k = kb; k < ke; ++k) {
          const int s = it % S::STAGES;
          const uint32_t ph = (uint32_t)(it / S::STAGES) & 1u;
          if (it >= S::STAGES) {
            if (*abort_flag || !mtd::mbar_wait_bounded(&empty[s], ph ^ 1u, A.status)) {
              *abort_flag = 1;
              stop = true;
              break;
            }
          }
          unsigned char *st = smem + (size_t)s * S::STAGE_BYTES;
          const int64_t c = gs - gc.g * A.CH + k;  // stored chunk
          mtd::mbar_arrive_expect_tx(&full[s], S::STAGE_BYTES);
          mtd::bulk_g2s(st, tens + (size_t)c * S::DATA_BYTES, S::DATA_BYTES, &full[s], pol_stream);
#pragma unroll
          for (int m = 0; m < SB; ++m) {
            const int64_t b = gc.g * SB + m < A.B ? gc.g * SB + m : 0;
            mtd::bulk_g2s(st + S::DATA_BYTES + m * S::XS_BYTES, xs + (size_t)(b * A.Q + gc.q) * S::XS_BYTES,
                          S::XS_BYTES, &full[s], pol_keep);
          }
          ++it;
        }
      }
      // drain: every copy issued must have landed before the CTA may exit
      for (int s = 0; s < S::STAGES && s < it; ++s) {
        const int last = it - 1 - ((it - 1 - s) % S::STAGES);  // last issue on stage s
        mtd::mbar_wait_bounded(&full[s], (uint32_t)(last / S::STAGES) & 1u, A.status);
      }
    }
    return;
  }

  // ---------------- consumers ----------------
  // warp w holds rows w RPW + r (r < RPW) of each of the K panels of the
  // current super-row; lane l holds columns 4 l .. 4 l + 3.
  // - One simulation: lane l keeps the running sums of its part of every row
  //   value of every panel (acc, K RPW 3 registers) and the warp adds them
  //   over its lanes at the super-row's flush.
  // - Two (twice those sums spilled registers): after each chunk the warp's
  //   NVAL row values (value (m RPW + r) 3 + c: simulation m, row r,
  //   component c) are added over the lanes by a reduce-scatter that leaves
  //   value l / LPS in lane l, which keeps its running sum for the chunk's
  //   panel k in accs[k].  A simulation's sums then run in another order
  //   than alone (each chunk's warp total first): equal to rounding.
  constexpr bool SCATTER = SB == 2;
  constexpr int NVAL = S::NVAL, NSLOT = S::NSLOT, LPS = 32 / NSLOT;
  float acc[SCATTER ? 1 : SB][SCATTER ? 1 : K][S::RPW][3];
  float accs[SCATTER ? K : 1];
  const int my_val = lane / LPS;
  float4 *xi = xi_all + warp * SB * K * S::RPW;  // [m][k RPW + r]
  int64_t sr_cur = -1;  // current (simulation group, super-row) = g Q + R
  int it = 0;
  bool aborted = false;
  const int ct = threadIdx.x;  // consumer thread 0 .. 32 NCW - 1
  __shared__ int split_last;

  auto out = [&](int64_t b) -> float * {
    return (b < A.B && (!A.active || A.active[b])) ? A.H + (size_t)b * 3 * A.n : nullptr;
  };

  // rows of super-row sr: warp totals, then written (or, for a super-row
  // shared by CTAs, parked and added in CTA order by the last to arrive)
  auto flush_lane = [&](int64_t sr) {
    if constexpr (!SCATTER) {
#pragma unroll
      for (int m = 0; m < SB; ++m)
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
          for (int r = 0; r < S::RPW; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[m][k][r][c] = mtd::warp_sum(acc[m][k][r][c]);
      const int64_t g = sr / A.Q, R = sr - g * A.Q;
      const int64_t su0 = g * A.CH + (int64_t)K * half_gbase(R, A.Q);
      const int64_t su1 = (R == A.Q - 1) ? (g + 1) * A.CH : g * A.CH + (int64_t)K * half_gbase(R + 1, A.Q);
      const int64_t kf = mtd::sk_owner(su0, U, G), kl = mtd::sk_owner(su1 - 1, U, G);
      // lane l holds values v = l and l + 32 (v = (k RPW + r) 3 + c)
      float mine[SB][2];
#pragma unroll
      for (int m = 0; m < SB; ++m) {
        mine[m][0] = mine[m][1] = 0.0f;
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
          for (int r = 0; r < S::RPW; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const int v = (k * S::RPW + r) * 3 + c;
              if (v == lane) mine[m][0] = acc[m][k][r][c];
              if (v == lane + 32) mine[m][1] = acc[m][k][r][c];
            }
      }
      auto row_of = [&](int v) {  // row within the super-row
        const int k = v / (S::RPW * 3), r = (v / 3) % S::RPW;
        return k * TR + warp * S::RPW + r;
      };
      // traceless storage: the self block's N_zz is 1 - xx - yy, the stream
      // gave -(xx + yy), so the row's z sum lacks Ms_i m_i,z (its operand)
      auto self_z = [&](int m, int v) -> float {
        if constexpr (C::NPLANE == 3 || C::NPLANE == 5) {
          if (v % 3 != 2) return 0.0f;
          const int k = v / (S::RPW * 3), r = (v / 3) % S::RPW;
          return xi[m * K * S::RPW + k * S::RPW + r].z;
        } else {
          return 0.0f;
        }
      };
      const int64_t row0 = R * K * TR;
      if (kf == kl) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int v = lane + 32 * h;
          if (v >= S::NV) continue;
          const int64_t row = row0 + row_of(v);
          if (row >= A.n) continue;
#pragma unroll
          for (int m = 0; m < SB; ++m)
            if (float *H = out(g * SB + m)) H[3 * row + v % 3] = -(mine[m][h] + self_z(m, v));
        }
        return;
      }
      const int64_t slot = (u0 >= su0) ? 2 * kcta : 2 * kcta + 1;  // the super-row is this CTA's first or last
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int v = lane + 32 * h;
        if (v >= S::NV) continue;
#pragma unroll
        for (int m = 0; m < SB; ++m) A.part[((slot * SB + m) * K * TR + row_of(v)) * 3 + v % 3] = mine[m][h];
      }
      __threadfence();
      __syncwarp();
      int last = 0;
      if (lane == 0) last = (atomicAdd(&A.count[sr * S::NCW + warp], 1) == (int)(kl - kf));
      last = __shfl_sync(0xffffffffu, last, 0);
      if (!last) return;
      __threadfence();
      // the parts in CTA order, each CTA's values loaded together
      float tot[2][SB];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int m = 0; m < SB; ++m) tot[h][m] = 0.0f;
      for (int64_t kk = kf; kk <= kl; ++kk) {
        const int64_t sl = (mtd::sk_begin(kk, U, G) >= su0) ? 2 * kk : 2 * kk + 1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int v = lane + 32 * h;
          if (v >= S::NV) continue;
#pragma unroll
          for (int m = 0; m < SB; ++m)
            tot[h][m] += __ldcg(&A.part[((sl * SB + m) * K * TR + row_of(v)) * 3 + v % 3]);
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int v = lane + 32 * h;
        if (v >= S::NV) continue;
        const int64_t row = row0 + row_of(v);
#pragma unroll
        for (int m = 0; m < SB; ++m) {
          float *H = out(g * SB + m);
          if (H && row < A.n) H[3 * row + v % 3] = -(tot[h][m] + self_z(m, v));
        }
      }
      if (lane == 0) A.count[sr * S::NCW + warp] = 0;  // ready for the next launch
        }
  };

  // the same for SCATTER: lane l holds value j = l / LPS of every panel; the
  // LPS lanes of a value share the panels (lane l takes k = l % LPS,
  // l % LPS + LPS, ...)
  auto flush_scatter = [&](int64_t sr) {
    if constexpr (SCATTER) {
      const int64_t g = sr / A.Q, R = sr - g * A.Q;
      const int64_t su0 = g * A.CH + (int64_t)K * half_gbase(R, A.Q);
      const int64_t su1 = (R == A.Q - 1) ? (g + 1) * A.CH : g * A.CH + (int64_t)K * half_gbase(R + 1, A.Q);
      const int64_t kf = mtd::sk_owner(su0, U, G), kl = mtd::sk_owner(su1 - 1, U, G);
      const bool valid = my_val < NVAL;
      const int m = my_val / (S::RPW * 3), r = (my_val / 3) % S::RPW, c = my_val % 3;
      const int row_in = warp * S::RPW + r;  // row within each panel
      auto self_z = [&](int k) -> float {  // as in flush_lane
        if constexpr (C::NPLANE == 3 || C::NPLANE == 5) {
          return c == 2 ? xi[m * K * S::RPW + k * S::RPW + r].z : 0.0f;
        } else {
          return 0.0f;
        }
      };
      const int64_t row0 = R * K * TR;
      float *H = valid ? out(g * SB + m) : nullptr;
      if (kf == kl) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (!valid || k % LPS != lane % LPS) continue;
          const int64_t row = row0 + k * TR + row_in;
          if (H && row < A.n) H[3 * row + c] = -(accs[k] + self_z(k));
        }
        return;
      }
      const int64_t slot = (u0 >= su0) ? 2 * kcta : 2 * kcta + 1;  // the super-row is this CTA's first or last
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (!valid || k % LPS != lane % LPS) continue;
        A.part[((slot * SB + m) * K * TR + k * TR + row_in) * 3 + c] = accs[k];
      }
      __threadfence();
      __syncwarp();
      int last = 0;
      if (lane == 0) last = (atomicAdd(&A.count[sr * S::NCW + warp], 1) == (int)(kl - kf));
      last = __shfl_sync(0xffffffffu, last, 0);
      if (!last) return;
      __threadfence();
      // the parts in CTA order, each CTA's values loaded together
      float tot[K];
#pragma unroll
      for (int k = 0; k < K; ++k) tot[k] = 0.0f;
      for (int64_t kk = kf; kk <= kl; ++kk) {
        const int64_t sl = (mtd::sk_begin(kk, U, G) >= su0) ? 2 * kk : 2 * kk + 1;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (!valid || k % LPS != lane % LPS) continue;
          tot[k] += __ldcg(&A.part[((sl * SB + m) * K * TR + k * TR + row_in) * 3 + c]);
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (!valid || k % LPS != lane % LPS) continue;
        const int64_t row = row0 + k * TR + row_in;
        if (H && row < A.n) H[3 * row + c] = -(tot[k] + self_z(k));
      }
      if (lane == 0) A.count[sr * S::NCW + warp] = 0;  // ready for the next launch
        }
  };
  auto flush_rows = [&](int64_t sr) {
    if constexpr (SCATTER) flush_scatter(sr);
    else flush_lane(sr);
  };

  // the chunks kb .. ke - 1 of one group; STRICT: also its column sums
  auto run_group = [&](auto strict_c, const GroupCursor &gc, int kb, int ke, float colp[SB][4][3]) {
    constexpr bool STRICT = decltype(strict_c)::value;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (k < kb || k >= ke) continue;
      const int s = it % S::STAGES;
      const uint32_t ph = (uint32_t)(it / S::STAGES) & 1u;
      ++it;
      if (!aborted) {
        if (*abort_flag || !mtd::mbar_wait_bounded(&full[s], ph, A.status)) {
          aborted = true;
          *abort_flag = 1;
        }
      }
      float rv[SCATTER ? NSLOT : 1];  // SCATTER: this chunk's row values (zero if the wait gave up)
      if constexpr (SCATTER) {
#pragma unroll
        for (int j = 0; j < NSLOT; ++j) rv[j] = 0.0f;
      }
      if (!aborted) {
        const unsigned char *st = smem + (size_t)s * S::STAGE_BYTES;
        float X[SB][4], Y[SB][4], Z[SB][4];
#pragma unroll
        for (int m = 0; m < SB; ++m) {
          const unsigned char *xsm = st + S::DATA_BYTES + m * S::XS_BYTES;
          load_xs<PREC>(xsm, 0, lane, X[m]);
          load_xs<PREC>(xsm, 1, lane, Y[m]);
          load_xs<PREC>(xsm, 2, lane, Z[m]);
        }
#pragma unroll
        for (int r = 0; r < S::RPW; ++r) {
          const int row = warp * S::RPW + r;
          float4 xr[SB];
          if constexpr (STRICT) {
#pragma unroll
            for (int m = 0; m < SB; ++m) xr[m] = xi[m * K * S::RPW + k * S::RPW + r];
          }
          if constexpr (C::NPLANE == 3) {
            // zz = -(xx + yy) (trace 0; the self blocks' +1 is added in
            // flush_rows)
            float nxx[4], nxy[4], nyy[4];
            load_vals<PREC>(st, 0, row, lane, nxx);
            load_vals<PREC>(st, 1, row, lane, nxy);
            load_vals<PREC>(st, 2, row, lane, nyy);
#pragma unroll
            for (int m = 0; m < SB; ++m) {
              float sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                const float nzz = -(nxx[v] + nyy[v]);
                sx = fmaf(nxx[v], X[m][v], fmaf(nxy[v], Y[m][v], sx));
                sy = fmaf(nxy[v], X[m][v], fmaf(nyy[v], Y[m][v], sy));
                sz = fmaf(nzz, Z[m][v], sz);
                if constexpr (STRICT) {
                  colp[m][v][0] = fmaf(nxx[v], xr[m].x, fmaf(nxy[v], xr[m].y, colp[m][v][0]));
                  colp[m][v][1] = fmaf(nxy[v], xr[m].x, fmaf(nyy[v], xr[m].y, colp[m][v][1]));
                  colp[m][v][2] = fmaf(nzz, xr[m].z, colp[m][v][2]);
                }
              }
              if constexpr (SCATTER) {
                rv[(m * S::RPW + r) * 3 + 0] = sx;
                rv[(m * S::RPW + r) * 3 + 1] = sy;
                rv[(m * S::RPW + r) * 3 + 2] = sz;
              } else {
                acc[m][k][r][0] += sx;
                acc[m][k][r][1] += sy;
                acc[m][k][r][2] += sz;
              }
            }
          } else if constexpr (C::NPLANE == 5) {
            // zz = -(xx + yy) (trace 0; the self blocks' +1 is added in
            // flush_rows)
            float nxx[4], nxy[4], nxz[4], nyy[4], nyz[4];
            load_vals<PREC>(st, 0, row, lane, nxx);
            load_vals<PREC>(st, 1, row, lane, nxy);
            load_vals<PREC>(st, 2, row, lane, nxz);
            load_vals<PREC>(st, 3, row, lane, nyy);
            load_vals<PREC>(st, 4, row, lane, nyz);
#pragma unroll
            for (int m = 0; m < SB; ++m) {
              float sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                const float nzz = -(nxx[v] + nyy[v]);
                sx = fmaf(nxx[v], X[m][v], fmaf(nxy[v], Y[m][v], fmaf(nxz[v], Z[m][v], sx)));
                sy = fmaf(nxy[v], X[m][v], fmaf(nyy[v], Y[m][v], fmaf(nyz[v], Z[m][v], sy)));
                sz = fmaf(nxz[v], X[m][v], fmaf(nyz[v], Y[m][v], fmaf(nzz, Z[m][v], sz)));
                if constexpr (STRICT) {
                  colp[m][v][0] = fmaf(nxx[v], xr[m].x, fmaf(nxy[v], xr[m].y, fmaf(nxz[v], xr[m].z, colp[m][v][0])));
                  colp[m][v][1] = fmaf(nxy[v], xr[m].x, fmaf(nyy[v], xr[m].y, fmaf(nyz[v], xr[m].z, colp[m][v][1])));
                  colp[m][v][2] = fmaf(nxz[v], xr[m].x, fmaf(nyz[v], xr[m].y, fmaf(nzz, xr[m].z, colp[m][v][2])));
                }
              }
              if constexpr (SCATTER) {
                rv[(m * S::RPW + r) * 3 + 0] = sx;
                rv[(m * S::RPW + r) * 3 + 1] = sy;
                rv[(m * S::RPW + r) * 3 + 2] = sz;
              } else {
                acc[m][k][r][0] += sx;
                acc[m][k][r][1] += sy;
                acc[m][k][r][2] += sz;
              }
            }
          } else if constexpr (C::PLANAR) {
            float nxx[4], nxy[4], nyy[4], nzz[4];
            load_vals<PREC>(st, 0, row, lane, nxx);
            load_vals<PREC>(st, 1, row, lane, nxy);
            load_vals<PREC>(st, 2, row, lane, nyy);
            load_vals<PREC>(st, 3, row, lane, nzz);
#pragma unroll
            for (int m = 0; m < SB; ++m) {
              float sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                sx = fmaf(nxx[v], X[m][v], fmaf(nxy[v], Y[m][v], sx));
                sy = fmaf(nxy[v], X[m][v], fmaf(nyy[v], Y[m][v], sy));
                sz = fmaf(nzz[v], Z[m][v], sz);
                if constexpr (STRICT) {
                  colp[m][v][0] = fmaf(nxx[v], xr[m].x, fmaf(nxy[v], xr[m].y, colp[m][v][0]));
                  colp[m][v][1] = fmaf(nxy[v], xr[m].x, fmaf(nyy[v], xr[m].y, colp[m][v][1]));
                  colp[m][v][2] = fmaf(nzz[v], xr[m].z, colp[m][v][2]);
                }
              }
              if constexpr (SCATTER) {
                rv[(m * S::RPW + r) * 3 + 0] = sx;
                rv[(m * S::RPW + r) * 3 + 1] = sy;
                rv[(m * S::RPW + r) * 3 + 2] = sz;
              } else {
                acc[m][k][r][0] += sx;
                acc[m][k][r][1] += sy;
                acc[m][k][r][2] += sz;
              }
            }
          } else {
            float nxx[4], nxy[4], nxz[4], nyy[4], nyz[4], nzz[4];
            load_vals<PREC>(st, 0, row, lane, nxx);
            load_vals<PREC>(st, 1, row, lane, nxy);
            load_vals<PREC>(st, 2, row, lane, nxz);
            load_vals<PREC>(st, 3, row, lane, nyy);
            load_vals<PREC>(st, 4, row, lane, nyz);
            load_vals<PREC>(st, 5, row, lane, nzz);
#pragma unroll
            for (int m = 0; m < SB; ++m) {
              float sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                sx = fmaf(nxx[v], X[m][v], fmaf(nxy[v], Y[m][v], fmaf(nxz[v], Z[m][v], sx)));
                sy = fmaf(nxy[v], X[m][v], fmaf(nyy[v], Y[m][v], fmaf(nyz[v], Z[m][v], sy)));
                sz = fmaf(nxz[v], X[m][v], fmaf(nyz[v], Y[m][v], fmaf(nzz[v], Z[m][v], sz)));
                if constexpr (STRICT) {
                  colp[m][v][0] = fmaf(nxx[v], xr[m].x, fmaf(nxy[v], xr[m].y, fmaf(nxz[v], xr[m].z, colp[m][v][0])));
                  colp[m][v][1] = fmaf(nxy[v], xr[m].x, fmaf(nyy[v], xr[m].y, fmaf(nyz[v], xr[m].z, colp[m][v][1])));
                  colp[m][v][2] = fmaf(nxz[v], xr[m].x, fmaf(nyz[v], xr[m].y, fmaf(nzz[v], xr[m].z, colp[m][v][2])));
                }
              }
              if constexpr (SCATTER) {
                rv[(m * S::RPW + r) * 3 + 0] = sx;
                rv[(m * S::RPW + r) * 3 + 1] = sy;
                rv[(m * S::RPW + r) * 3 + 2] = sz;
              } else {
                acc[m][k][r][0] += sx;
                acc[m][k][r][1] += sy;
                acc[m][k][r][2] += sz;
              }
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mtd::mbar_arrive(&empty[s]);
      if constexpr (SCATTER) accs[k] += warp_reduce_scatter<NSLOT>(rv, lane);  // every lane, aborted or not
    }
  };

  GroupCursor gc;
  for (int64_t gs = group_decode<K>(A, u0, gc); gs < u1; gs += group_len<K>(A, gc), group_next(A, gc)) {
    if (!half_live(A, gc.g, SB)) continue;
    const int len = group_len<K>(A, gc);
    const int kb = (int)(u0 > gs ? u0 - gs : 0), ke = (int)(u1 - gs < len ? u1 - gs : len);
    const int64_t sr = gc.g * A.Q + gc.R;
    if (sr != sr_cur) {
      if (sr_cur >= 0) flush_rows(sr_cur);
      sr_cur = sr;
      if constexpr (SCATTER) {
#pragma unroll
        for (int k = 0; k < K; ++k) accs[k] = 0.0f;
      } else {
#pragma unroll
        for (int m = 0; m < SB; ++m)
#pragma unroll
          for (int k = 0; k < K; ++k)
#pragma unroll
            for (int r = 0; r < S::RPW; ++r) acc[m][k][r][0] = acc[m][k][r][1] = acc[m][k][r][2] = 0.0f;
      }
      // the operand of this warp's rows of the super-row (column chunk R of
      // the operand): lane l < 16 SB takes simulation l / 16, row slot l % 16
      __syncwarp();
      if (lane < SB * K * S::RPW) {
        const int m = lane / (K * S::RPW), kr = lane % (K * S::RPW);
        const int k = kr / S::RPW, r = kr % S::RPW;
        const int64_t b = gc.g * SB + m < A.B ? gc.g * SB + m : 0;
        const float *x = A.xs + (size_t)(b * A.Q + gc.R) * 3 * TC + k * TR + warp * S::RPW + r;
        xi[m * K * S::RPW + kr] = make_float4(__ldg(x), __ldg(x + TC), __ldg(x + 2 * TC), 0.0f);
      }
      __syncwarp();
    }
    if (gc.q == gc.R) {  // the diagonal group: rows only
      run_group(std::false_type{}, gc, kb, ke, nullptr);
      continue;
    }
    float colp[SB][4][3];
#pragma unroll
    for (int m = 0; m < SB; ++m)
#pragma unroll
      for (int v = 0; v < 4; ++v) colp[m][v][0] = colp[m][v][1] = colp[m][v][2] = 0.0f;
    run_group(std::true_type{}, gc, kb, ke, colp);
    // column sums of the group: each warp's (its rows) to shared memory,
    // then thread t adds column t % TC, components t / TC, t / TC + 2, ...,
    // over the warps in order
#pragma unroll
    for (int m = 0; m < SB; ++m)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        *reinterpret_cast<float4 *>(cb + ((warp * SB + m) * 3 + c) * TC + lane * 4) =
            make_float4(colp[m][0][c], colp[m][1][c], colp[m][2][c], colp[m][3][c]);
    asm volatile("bar.sync 1, %0;" ::"r"(S::NCW * 32) : "memory");
    constexpr int NT = S::NCW * 32 / TC;  // thread sets over the columns
    const int col = ct % TC;
    const bool whole = (kb == 0 && ke == len);
    const int64_t slot = (u0 >= gs) ? 2 * kcta : 2 * kcta + 1;  // a split group: this CTA's first or last
#pragma unroll
    for (int c0 = 0; c0 < 3; c0 += NT) {
      const int c = c0 + ct / TC;
      if (c >= 3) break;
#pragma unroll
      for (int m = 0; m < SB; ++m) {
        float tot = 0.0f;
#pragma unroll
        for (int w = 0; w < S::NCW; ++w) tot += cb[((w * SB + m) * 3 + c) * TC + col];
        if (whole) A.colpart[(((gc.g * A.NGR + gc.gi) * SB + m) * 3 + c) * TC + col] = tot;
        else A.colsplit[((slot * SB + m) * 3 + c) * TC + col] = tot;
      }
    }
    if (!whole) __threadfence();
    asm volatile("bar.sync 1, %0;" ::"r"(S::NCW * 32) : "memory");  // CB free; a split part is out
    if (whole) continue;
    // a group split between CTAs: the last to arrive adds the parts in CTA order
    const int64_t kf = mtd::sk_owner(gs, U, G), kl = mtd::sk_owner(gs + len - 1, U, G);
    int *gcount = &A.gcount[gc.g * A.NGR + gc.gi];
    if (ct == 0) split_last = (atomicAdd(gcount, 1) == (int)(kl - kf));
    asm volatile("bar.sync 1, %0;" ::"r"(S::NCW * 32) : "memory");
    if (!split_last) continue;
    __threadfence();
    constexpr int NC = (3 + NT - 1) / NT;  // components per thread
    float tot[NC][SB];
#pragma unroll
    for (int i = 0; i < NC; ++i)
#pragma unroll
      for (int m = 0; m < SB; ++m) tot[i][m] = 0.0f;
    for (int64_t kk = kf; kk <= kl; ++kk) {  // the parts in CTA order, each CTA's loaded together
      const int64_t sl = (mtd::sk_begin(kk, U, G) >= gs) ? 2 * kk : 2 * kk + 1;
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        const int c = i * NT + ct / TC;
        if (c >= 3) break;
#pragma unroll
        for (int m = 0; m < SB; ++m) tot[i][m] += __ldcg(&A.colsplit[((sl * SB + m) * 3 + c) * TC + col]);
      }
    }
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      const int c = i * NT + ct / TC;
      if (c >= 3) break;
#pragma unroll
      for (int m = 0; m < SB; ++m) A.colpart[(((gc.g * A.NGR + gc.gi) * SB + m) * 3 + c) * TC + col] = tot[i][m];
    }
    if (ct == 0) *gcount = 0;  // ready for the next launch
  }
  if (sr_cur >= 0) flush_rows(sr_cur);
}

// The transposed part of a half-stored product.  Column j of column chunk q
// gets the sum over the groups (R, q), R < q, of their column sums.  One CTA
// per (q, simulation), kHalfColLanes threads per column: thread (r, t) adds
// column t of the groups R = r, r + kHalfColLanes, ... in increasing R, and
// the lanes' sums are added in order of r (a fixed order: the result does
// not depend on timing) before H_j -= total.  Every load of a CTA is issued
// in one round (the group sums were just written and sit in L2), and no
// CTA waits on another.
constexpr int kHalfColLanes = 8;
template <int TC>
__global__ void __launch_bounds__(kHalfColLanes *TC) k_half_cols(HalfArgs A, int SB) {
  mtd::pdl_enter();
  const int64_t q = blockIdx.x;
  const int b = blockIdx.y;
  const int t = threadIdx.x % TC, r = threadIdx.x / TC;
  const int64_t g = b / SB, m = b - g * SB;
  // group (R, q) is number half_gbase(R) + q - R
  const float *base = A.colpart + ((g * A.NGR * SB + m) * 3) * TC + t;
  const int64_t gstride = (int64_t)SB * 3 * TC;
  constexpr int L = kHalfColLanes;
  float tot[3] = {0.0f, 0.0f, 0.0f};
  int64_t R = r;
  for (; R + 3 * L < q; R += 4 * L) {  // four groups' loads in flight
    float v[4][3];
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      const int64_t Rk = R + k2 * L;
      const float *cp = base + (half_gbase(Rk, A.Q) + q - Rk) * gstride;
      v[k2][0] = __ldcg(cp);
      v[k2][1] = __ldcg(cp + TC);
      v[k2][2] = __ldcg(cp + 2 * TC);
    }
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      tot[0] += v[k2][0];
      tot[1] += v[k2][1];
      tot[2] += v[k2][2];
    }
  }
  for (; R < q; R += L) {
    const float *cp = base + (half_gbase(R, A.Q) + q - R) * gstride;
    tot[0] += __ldcg(cp);
    tot[1] += __ldcg(cp + TC);
    tot[2] += __ldcg(cp + 2 * TC);
  }
  __shared__ float lane_sum[L][3][TC];
  lane_sum[r][0][t] = tot[0];
  lane_sum[r][1][t] = tot[1];
  lane_sum[r][2][t] = tot[2];
  __syncthreads();
  if (r != 0) return;
  const int64_t j = q * TC + t;
  if (j >= A.n || (A.active && !A.active[b])) return;
  float v[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float s = 0.0f;
#pragma unroll
    for (int k2 = 0; k2 < L; ++k2) s += lane_sum[k2][c][t];
    v[c] = s;
  }
  float *H = A.H + (size_t)b * 3 * A.n + 3 * j;
  H[0] -= v[0];
  H[1] -= v[1];
  H[2] -= v[2];
}

// xs[b][q][c][t] = Ms_j m_j[c] with j = q*TC + t (0 beyond n)
template <typename In, typename Out>
__global__ void k_prep_xs(const In *m, const float *Ms, int64_t n, int64_t Q, int TC, int B, Out *xs) {
  const int64_t tot = (int64_t)B * Q * TC;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / (Q * TC), rem = t - b * Q * TC;
    const int64_t q = rem / TC, c = rem - q * TC;
    const int64_t j = q * TC + c;
    Out x = 0, y = 0, z = 0;
    if (j < n) {
      const Out ms = (Out)Ms[j];
      const In *mj = m + (size_t)b * 3 * n + 3 * j;
      x = ms * (Out)mj[0];
      y = ms * (Out)mj[1];
      z = ms * (Out)mj[2];
    }
    Out *dst = xs + ((size_t)(b * Q + q) * 3) * TC + c;
    dst[0] = x;
    dst[TC] = y;
    dst[2 * TC] = z;
  }
}

// Near-field blocks (BF16 precisions of the streaming layout): double-FP32
// sums (mtd::ff) of N_ij Ms_j m_j over the touching tiles, added to the far
// field and rounded once.  Threads enumerate (tile, simulation) pairs with
// the simulation fastest, so a warp of a wide batch shares its tile's blocks
// (broadcast loads); m element (b, j, c) sits at m[b * sb + (3 j + c) * se]:
// se = 1 for the tile-major state, sb = 1 for a simulation-fastest copy.
using mtd::ff;
using mtd::ff_add;
using mtd::ff_fma_lazy;

// FF = false (the BF16 precision, whose far part carries ~1e-4 errors):
// plain FP32 sums of the high words, H = far - near in FP32
template <bool FF>
__global__ void k_near(int64_t n, int B, const int32_t *ptr, const int32_t *col, const float2 *val,
                       const float *m, int64_t sb, int64_t se, float *H, const int *active) {
  mtd::pdl_enter();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * B) return;
  const int64_t i = t / B;
  const int b = (int)(t - i * B);
  if (active && !active[b]) return;
  const float *mb = m + (size_t)b * sb;
  ff hx = {0, 0}, hy = {0, 0}, hz = {0, 0};
  for (int32_t a = ptr[i]; a < ptr[i + 1]; ++a) {
    const int64_t j = col[a];
    // val holds N_ij Ms_j: the operand is m itself, exact in FP32
    const float x0 = mb[(3 * j) * se], x1 = mb[(3 * j + 1) * se], x2 = mb[(3 * j + 2) * se];
    // 48 bytes per block, 16-byte aligned: three float4 requests
    const float4 *vp = reinterpret_cast<const float4 *>(val + 6 * (size_t)a);
    const float4 w0 = vp[0], w1 = vp[1], w2 = vp[2];
    const float2 v0 = make_float2(w0.x, w0.y), v1 = make_float2(w0.z, w0.w), v2 = make_float2(w1.x, w1.y);
    const float2 v3 = make_float2(w1.z, w1.w), v4 = make_float2(w2.x, w2.y), v5 = make_float2(w2.z, w2.w);
    if (!FF) {
      hx.hi = fmaf(v0.x, x0, fmaf(v1.x, x1, fmaf(v2.x, x2, hx.hi)));
      hy.hi = fmaf(v1.x, x0, fmaf(v3.x, x1, fmaf(v4.x, x2, hy.hi)));
      hz.hi = fmaf(v2.x, x0, fmaf(v4.x, x1, fmaf(v5.x, x2, hz.hi)));
      continue;
    }
    ff_fma_lazy(hx, v0, x0);
    ff_fma_lazy(hx, v1, x1);
    ff_fma_lazy(hx, v2, x2);
    ff_fma_lazy(hy, v1, x0);
    ff_fma_lazy(hy, v3, x1);
    ff_fma_lazy(hy, v4, x2);
    ff_fma_lazy(hz, v2, x0);
    ff_fma_lazy(hz, v4, x1);
    ff_fma_lazy(hz, v5, x2);
  }
  float *Hb = H + (size_t)b * 3 * n + 3 * i;
  // H = far - near, rounded once
  const ff rx = ff_add({Hb[0], 0.0f}, -hx.hi, -hx.lo);
  const ff ry = ff_add({Hb[1], 0.0f}, -hy.hi, -hy.lo);
  const ff rz = ff_add({Hb[2], 0.0f}, -hz.hi, -hz.lo);
  Hb[0] = rx.hi + rx.lo;
  Hb[1] = ry.hi + ry.lo;
  Hb[2] = rz.hi + rz.lo;
}

// The same for the simulation-fastest copy of a batch (element (b, j, c) at
// mT[(3 j + c) Bp + b]): a thread takes V adjacent simulations of one tile
// (one vector load per component), so a warp covers 32 V simulations and
// shares the tile's blocks; the column of the next block is fetched one step
// ahead.
template <int V>
struct VecF;
template <>
struct VecF<1> {
  using T = float;
  static __device__ __forceinline__ void get(T v, float *o) { o[0] = v; }
};
template <>
struct VecF<2> {
  using T = float2;
  static __device__ __forceinline__ void get(T v, float *o) {
    o[0] = v.x;
    o[1] = v.y;
  }
};
template <>
struct VecF<4> {
  using T = float4;
  static __device__ __forceinline__ void get(T v, float *o) {
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  }
};

template <bool FF, int V>
__global__ void k_near_v(int64_t n, int B, int Bp, const int32_t *ptr, const int32_t *col, const float2 *val,
                         const float *mT, float *H, const int *active) {
  mtd::pdl_enter();
  using VT = typename VecF<V>::T;
  const int Bv = (B + V - 1) / V;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * Bv) return;
  const int64_t i = t / Bv;
  const int b0 = (int)(t - i * Bv) * V;
  ff hx[V], hy[V], hz[V];
#pragma unroll
  for (int v = 0; v < V; ++v) hx[v] = hy[v] = hz[v] = ff{0.0f, 0.0f};
  const int32_t a0 = ptr[i], a1 = ptr[i + 1];
  int64_t jn = a0 < a1 ? col[a0] : 0;
  for (int32_t a = a0; a < a1; ++a) {
    const int64_t j = jn;
    if (a + 1 < a1) jn = col[a + 1];
    const float4 *vp = reinterpret_cast<const float4 *>(val + 6 * (size_t)a);
    const float4 w0 = vp[0], w1 = vp[1], w2 = vp[2];
    float x0[V], x1[V], x2[V];
    VecF<V>::get(*reinterpret_cast<const VT *>(mT + (size_t)(3 * j) * Bp + b0), x0);
    VecF<V>::get(*reinterpret_cast<const VT *>(mT + (size_t)(3 * j + 1) * Bp + b0), x1);
    VecF<V>::get(*reinterpret_cast<const VT *>(mT + (size_t)(3 * j + 2) * Bp + b0), x2);
    const float2 v0 = make_float2(w0.x, w0.y), v1 = make_float2(w0.z, w0.w), v2 = make_float2(w1.x, w1.y);
    const float2 v3 = make_float2(w1.z, w1.w), v4 = make_float2(w2.x, w2.y), v5 = make_float2(w2.z, w2.w);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if (!FF) {
        hx[v].hi = fmaf(v0.x, x0[v], fmaf(v1.x, x1[v], fmaf(v2.x, x2[v], hx[v].hi)));
        hy[v].hi = fmaf(v1.x, x0[v], fmaf(v3.x, x1[v], fmaf(v4.x, x2[v], hy[v].hi)));
        hz[v].hi = fmaf(v2.x, x0[v], fmaf(v4.x, x1[v], fmaf(v5.x, x2[v], hz[v].hi)));
      } else {
        ff_fma_lazy(hx[v], v0, x0[v]);
        ff_fma_lazy(hx[v], v1, x1[v]);
        ff_fma_lazy(hx[v], v2, x2[v]);
        ff_fma_lazy(hy[v], v1, x0[v]);
        ff_fma_lazy(hy[v], v3, x1[v]);
        ff_fma_lazy(hy[v], v4, x2[v]);
        ff_fma_lazy(hz[v], v2, x0[v]);
        ff_fma_lazy(hz[v], v4, x1[v]);
        ff_fma_lazy(hz[v], v5, x2[v]);
      }
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int b = b0 + v;
    if (b >= B || (active && !active[b])) continue;
    float *Hb = H + (size_t)b * 3 * n + 3 * i;
    // H = far - near, rounded once
    const ff rx = ff_add({Hb[0], 0.0f}, -hx[v].hi, -hx[v].lo);
    const ff ry = ff_add({Hb[1], 0.0f}, -hy[v].hi, -hy[v].lo);
    const ff rz = ff_add({Hb[2], 0.0f}, -hz[v].hi, -hz[v].lo);
    Hb[0] = rx.hi + rx.lo;
    Hb[1] = ry.hi + ry.lo;
    Hb[2] = rz.hi + rz.lo;
  }
}

// half storage is built for FP32 tensors only (6 or 4 planes)
template <int PREC>
constexpr bool has_half() {
  return PREC == MT_F32 || PREC == kF32Planar || PREC == kF32Traceless || PREC == kF32Traceless5;
}

template <int PREC, int SB>
cudaError_t prepare_mv_one() {
  cudaError_t e = cudaFuncSetAttribute(k_matvec<PREC, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       MvShape<PREC, SB>::SMEM_BYTES);
  if constexpr (has_half<PREC>() && SB <= 2) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_matvec_half<PREC, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               HalfShape<PREC, SB>::SMEM_BYTES);
  }
  return e;
}

template <int PREC>
cudaError_t prepare_mv() {
  cudaError_t e;
  if ((e = prepare_mv_one<PREC, 1>()) != cudaSuccess || (e = prepare_mv_one<PREC, 2>()) != cudaSuccess) return e;
  if constexpr (PREC == MT_BF16_SCALED || PREC == kBF16Planar) return cudaSuccess;
  else return prepare_mv_one<PREC, 4>();
}

// simulations per chunk read: 1, 2 or 4 (2 at most for the scaled BF16
// tensor, whose 8-wide rows with 4 operands spill registers: measured 0.56 ms
// for 4 simulations at n = 10,000 against 0.21 ms for one; 2 at most for a
// half-stored tensor, whose threads hold the sums of 16 rows per simulation)
inline int mv_group(int B, int prec, bool half) {
  const int cap = (half || prec == MT_BF16_SCALED || prec == kBF16Planar) ? 2 : 4;
  return B <= 1 ? 1 : (B == 2 || cap == 2) ? 2 : 4;
}

template <int PREC, int SB>
void launch_mv_sb(const MvArgs &A, int grid_cap, cudaStream_t s) {
  // never more CTAs than units: every CTA then owns at least one unit, which
  // the panel bookkeeping (owners of a panel's first and last unit bound its
  // contributors) relies on
  const int64_t U = (int64_t)((A.B + SB - 1) / SB) * A.CH;
  const int grid = (int)std::min<int64_t>(grid_cap, U);
  using S = MvShape<PREC, SB>;
  mt::launch_pdl(k_matvec<PREC, SB>, dim3(grid), dim3(S::THREADS), S::SMEM_BYTES, s, A);
}

// work area of a half-stored product over B simulations, SB per chunk read
// (floats): the column sums of every group [NG][NGR][SB][3][TC]; the parts of
// groups split between CTAs [2 grid_cap][SB][3][TC]
struct HalfArea {
  size_t colpart, colsplit, bytes;
};
inline HalfArea half_area(int64_t Q, int64_t B, int SB, int grid_cap, int TC) {
  const int64_t NG = (B + SB - 1) / SB, NGR = half_groups(Q);
  HalfArea h;
  h.colpart = 0;
  h.colsplit = h.colpart + (size_t)NG * NGR * SB * 3 * TC;
  h.bytes = (h.colsplit + (size_t)2 * grid_cap * SB * 3 * TC) * sizeof(float);
  return h;
}

template <int PREC, int SB>
void launch_half(const mt_tensor *T, const float *xs, int B, float *H, float *part, int *count, const int *active,
                 int *status, float *work, cudaStream_t s) {
  using S = HalfShape<PREC, SB>;
  constexpr int TC = MvCfg<PREC>::TC;
  const int cap = mt::matvec_grid(T);
  const HalfArea h = half_area(T->L.Q, B, SB, cap, TC);
  HalfArgs A;
  A.tensor = reinterpret_cast<const float *>(T->d_data);
  A.xs = xs;
  A.H = H;
  A.part = part;
  A.count = count;
  A.gcount = count + (size_t)B * T->L.P * 8;  // after the row counters (all counters rest at zero)
  A.colpart = work + h.colpart;
  A.colsplit = work + h.colsplit;
  A.active = active;
  A.status = status;
  A.n = T->n;
  A.P = T->L.P;
  A.Q = T->L.Q;
  A.CH = T->L.CH;
  A.NGR = half_groups(T->L.Q);
  A.B = B;
  const int64_t U = (int64_t)((B + SB - 1) / SB) * A.CH;
  const int grid = (int)std::min<int64_t>(cap, U);
  mt::launch_pdl(k_matvec_half<PREC, SB>, dim3(grid), dim3(S::THREADS), S::SMEM_BYTES, s, A);
  mt::launch_pdl(k_half_cols<TC>, dim3((unsigned)A.Q, (unsigned)B), dim3(kHalfColLanes * TC), 0, s, A, SB);
}

// a layout that exists only stored half (3 planes)
template <int PREC>
void launch_half_only(const mt_tensor *T, const void *xs, int B, void *H, void *part, int *count,
                      const int *active, int *status, float *colpart, cudaStream_t s) {
  if (mv_group(B, PREC, true) == 1)
    launch_half<PREC, 1>(T, (const float *)xs, B, (float *)H, (float *)part, count, active, status, colpart, s);
  else
    launch_half<PREC, 2>(T, (const float *)xs, B, (float *)H, (float *)part, count, active, status, colpart, s);
}

template <int PREC>
void launch_mv(const mt_tensor *T, const void *xs, int B, void *H, void *part, int *count, const int *active,
               int *status, float *colpart, cudaStream_t s) {
  if constexpr (has_half<PREC>()) {
    if (T->L.half) {
      if (mv_group(B, PREC, true) == 1)
        launch_half<PREC, 1>(T, (const float *)xs, B, (float *)H, (float *)part, count, active, status, colpart, s);
      else
        launch_half<PREC, 2>(T, (const float *)xs, B, (float *)H, (float *)part, count, active, status, colpart, s);
      return;
    }
  }
  MvArgs A;
  A.tensor = T->d_data;
  A.scale = T->d_scale;
  A.xs = xs;
  A.H = H;
  A.part = part;
  A.count = count;
  A.active = active;
  A.status = status;
  A.n = T->n;
  A.P = T->L.P;
  A.Q = T->L.Q;
  A.CH = T->L.CH;
  A.B = B;
  const int cap = mt::matvec_grid(T);
  switch (mv_group(B, PREC, false)) {
    case 1: launch_mv_sb<PREC, 1>(A, cap, s); break;
    case 2: launch_mv_sb<PREC, 2>(A, cap, s); break;
    default:
      if constexpr (PREC != MT_BF16_SCALED && PREC != kBF16Planar) launch_mv_sb<PREC, 4>(A, cap, s);
      break;
  }
}

}  // namespace

namespace mt {

int matvec_grid(const mt_tensor *T) { return T->tiles->ctx->num_sms; }

cudaError_t matvec_prepare() {
  cudaError_t e;
  if ((e = prepare_mv<MT_F32>()) != cudaSuccess) return e;
  if ((e = prepare_mv<kF32Planar>()) != cudaSuccess) return e;
  // the traceless layout is always stored half: its half kernels only
  if ((e = cudaFuncSetAttribute(k_matvec_half<kF32Traceless, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                HalfShape<kF32Traceless, 1>::SMEM_BYTES)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_matvec_half<kF32Traceless, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                HalfShape<kF32Traceless, 2>::SMEM_BYTES)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_matvec_half<kF32Traceless5, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                HalfShape<kF32Traceless5, 1>::SMEM_BYTES)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_matvec_half<kF32Traceless5, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                HalfShape<kF32Traceless5, 2>::SMEM_BYTES)) != cudaSuccess)
    return e;
  if ((e = prepare_mv<kBF16Planar>()) != cudaSuccess) return e;
  if ((e = prepare_mv<kSplitPlanar>()) != cudaSuccess) return e;
  if ((e = prepare_mv<MT_F64>()) != cudaSuccess) return e;
  if ((e = prepare_mv<MT_BF16_SCALED>()) != cudaSuccess) return e;
  return prepare_mv<MT_BF16_SPLIT>();
}

void layout_for_planar(int prec, mt_layout *L) {
  if (prec == MT_BF16_SPLIT) {
    L->TR = MvCfg<kSplitPlanar>::TR;
    L->TC = MvCfg<kSplitPlanar>::TC;
    L->nplane = MvCfg<kSplitPlanar>::NPLANE;
    L->elem_bytes = 2;
    L->scale_bytes_per_chunk = 0;
  } else if (prec == MT_BF16_SCALED) {
    L->TR = MvCfg<kBF16Planar>::TR;
    L->TC = MvCfg<kBF16Planar>::TC;
    L->nplane = MvCfg<kBF16Planar>::NPLANE;
    L->elem_bytes = 2;
    L->scale_bytes_per_chunk = (int64_t)L->TR * L->TC;
  } else {
    L->TR = MvCfg<kF32Planar>::TR;
    L->TC = MvCfg<kF32Planar>::TC;
    L->nplane = MvCfg<kF32Planar>::NPLANE;
    L->elem_bytes = 4;
    L->scale_bytes_per_chunk = 0;
  }
}

void layout_for_traceless(mt_layout *L, bool planar) {
  L->TR = MvCfg<kF32Traceless>::TR;
  L->TC = MvCfg<kF32Traceless>::TC;
  L->nplane = planar ? MvCfg<kF32Traceless>::NPLANE : MvCfg<kF32Traceless5>::NPLANE;
  L->elem_bytes = 4;
  L->scale_bytes_per_chunk = 0;
}

void layout_for(int prec, mt_layout *L) {
  switch (prec) {
    case MT_F32: L->TR = MvCfg<MT_F32>::TR; L->TC = MvCfg<MT_F32>::TC; L->nplane = 6; L->elem_bytes = 4; break;
    case MT_F64: L->TR = MvCfg<MT_F64>::TR; L->TC = MvCfg<MT_F64>::TC; L->nplane = 6; L->elem_bytes = 8; break;
    case MT_BF16_SCALED:
      L->TR = MvCfg<MT_BF16_SCALED>::TR; L->TC = MvCfg<MT_BF16_SCALED>::TC; L->nplane = 6; L->elem_bytes = 2; break;
    default:
      L->TR = MvCfg<MT_BF16_SPLIT>::TR; L->TC = MvCfg<MT_BF16_SPLIT>::TC; L->nplane = 12; L->elem_bytes = 2; break;
  }
  L->scale_bytes_per_chunk = (prec == MT_BF16_SCALED) ? (int64_t)L->TR * L->TC : 0;
}

int64_t xs_floats(const mt_tensor *T) {
  if (T->layout == MT_LAYOUT_SPARSE) return 4 * sparse_x_stride(T->n);  // float4 (Ms m, 0) per tile
  const int64_t per = T->L.Q * 3 * T->L.TC;
  return T->prec == MT_F64 ? 2 * per : per;  // doubles take two floats
}

size_t matvec_part_bytes(const mt_tensor *T) {
  const size_t el = T->prec == MT_F64 ? 8 : 4;
  if (T->L.half)  // super-rows of K panels, up to 2 simulations per chunk read
    return (size_t)2 * matvec_grid(T) * 2 * (T->L.TC / T->L.TR) * T->L.TR * 3 * el;
  return (size_t)2 * matvec_grid(T) * 4 /*simulations per chunk read, at most*/ * T->L.TR * 3 * el;
}

// per (simulation, panel) up to 8 warp counters; a half-stored tensor adds
// one counter per (simulation, group)
size_t matvec_count_bytes(const mt_tensor *T, int B) {
  const size_t rows = (size_t)B * T->L.P * 8;
  return (rows + (T->L.half ? (size_t)B * half_groups(T->L.Q) : 0)) * sizeof(int);
}

// half storage: the work area of the product over B simulations (a call
// with fewer simulations uses less of each part)
size_t matvec_colpart_bytes(const mt_tensor *T, int B) {
  if (!T->L.half) return 0;
  const int sb = mv_group(B, MT_F32, true);
  return half_area(T->L.Q, B, sb, matvec_grid(T), T->L.TC).bytes;
}

void launch_prep_xs(const mt_tensor *T, const float *m, int B, float *xs, cudaStream_t s) {
  if (T->layout == MT_LAYOUT_SPARSE) {
    launch_prep_sparse_x(T, m, B, xs, s);
    return;
  }
  const int64_t tot = (int64_t)B * T->L.Q * T->L.TC;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 4096);
  if (T->prec == MT_F64)
    k_prep_xs<float, double><<<blocks, 256, 0, s>>>(m, T->tiles->d_Ms, T->n, T->L.Q, T->L.TC, B,
                                                     reinterpret_cast<double *>(xs));
  else
    k_prep_xs<float, float><<<blocks, 256, 0, s>>>(m, T->tiles->d_Ms, T->n, T->L.Q, T->L.TC, B, xs);
}

void launch_prep_xs_f64(const mt_tensor *T, const double *m, int B, double *xs, cudaStream_t s) {
  const int64_t tot = (int64_t)B * T->L.Q * T->L.TC;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 4096);
  k_prep_xs<double, double><<<blocks, 256, 0, s>>>(m, T->tiles->d_Ms, T->n, T->L.Q, T->L.TC, B, xs);
}

void launch_matvec(const mt_tensor *T, const float *xs, int B, float *H, float *part, int *count,
                   const int *active, int *status, cudaStream_t s, float *colpart) {
  switch (T->prec) {
    case MT_F32:
      if (T->L.nplane == 3) launch_half_only<kF32Traceless>(T, xs, B, H, part, count, active, status, colpart, s);
      else if (T->L.nplane == 5)
        launch_half_only<kF32Traceless5>(T, xs, B, H, part, count, active, status, colpart, s);
      else if (T->L.nplane == 4) launch_mv<kF32Planar>(T, xs, B, H, part, count, active, status, colpart, s);
      else launch_mv<MT_F32>(T, xs, B, H, part, count, active, status, colpart, s);
      break;
    case MT_F64: launch_mv<MT_F64>(T, xs, B, H, part, count, active, status, nullptr, s); break;
    case MT_BF16_SCALED:
      if (T->L.nplane == 4) launch_mv<kBF16Planar>(T, xs, B, H, part, count, active, status, nullptr, s);
      else launch_mv<MT_BF16_SCALED>(T, xs, B, H, part, count, active, status, nullptr, s);
      break;
    case MT_BF16_SPLIT:
      if (T->L.nplane == 8) launch_mv<kSplitPlanar>(T, xs, B, H, part, count, active, status, nullptr, s);
      else launch_mv<MT_BF16_SPLIT>(T, xs, B, H, part, count, active, status, nullptr, s);
      break;
  }
}

void launch_near(const mt_tensor *T, const float *m, int64_t sb, int64_t se, int B, float *H, const int *active,
                 cudaStream_t s) {
  if (T->near_count == 0) return;
  const int64_t tot = T->n * (int64_t)B;
  const unsigned grid = (unsigned)((tot + 255) / 256);
  const int32_t *ptr = T->d_near_ptr, *col = T->d_near_col;
  const float2 *hl = T->d_near_hl;
  const int64_t n = T->n;
  if (sb == 1 && se >= B && se % 4 == 0) {  // simulation-fastest copy, rows of se >= B floats
    const int V = B >= 128 ? 4 : B >= 64 ? 2 : 1;
    const int64_t threads = n * ((B + V - 1) / V);
    const unsigned g = (unsigned)((threads + 255) / 256);
    const int Bp = (int)se;
    const bool split = T->prec == MT_BF16_SPLIT;
#define MT_NEAR_V(FF, VV) \
  mt::launch_pdl(k_near_v<FF, VV>, dim3(g), dim3(256), 0, s, n, B, Bp, ptr, col, hl, m, H, active)
    if (split) {
      if (V == 4) MT_NEAR_V(true, 4);
      else if (V == 2) MT_NEAR_V(true, 2);
      else MT_NEAR_V(true, 1);
    } else {
      if (V == 4) MT_NEAR_V(false, 4);
      else if (V == 2) MT_NEAR_V(false, 2);
      else MT_NEAR_V(false, 1);
    }
#undef MT_NEAR_V
    return;
  }
  if (T->prec == MT_BF16_SPLIT)
    mt::launch_pdl(k_near<true>, dim3(grid), dim3(256), 0, s, n, B, ptr, col, hl, m, sb, se, H, active);
  else
    mt::launch_pdl(k_near<false>, dim3(grid), dim3(256), 0, s, n, B, ptr, col, hl, m, sb, se, H, active);
}

}  // namespace mt
