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
//     order, so the result does not depend on timing.
#include <algorithm>
#include <cstdio>

#include "mt_internal.cuh"

namespace {

// FP32 / scaled-BF16 tensors of a single-layer tile set: the xz and yz
// planes are not stored (they vanish by mirror symmetry), planes xx, xy, yy,
// zz
constexpr int kF32Planar = 4;
constexpr int kBF16Planar = 5;
constexpr int kSplitPlanar = 6;  // hi planes xx, xy, yy, zz, then the lo planes

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

template <int PREC, int SB, bool HALF = false>
struct MvShape {
  using C = MvCfg<PREC>;
  // consumer warps: W, or 2 W for a half-stored tensor and up to two
  // simulations per chunk read (its chunks carry twice the arithmetic per
  // byte, the row and the column product, and one warp per SM sub-partition
  // left the issue slots idle on latency; with four simulations the halved
  // register budget spills)
  static constexpr int NCW = (HALF && SB <= 2) ? 2 * C::W : C::W;
  static constexpr int RPW = C::TR / NCW;  // rows per consumer warp
  static constexpr int DATA_BYTES = C::NPLANE * C::TR * C::TC * (int)sizeof(typename C::T);
  static constexpr int SCALE_BYTES = C::SCALED ? C::TR * C::TC : 0;
  static constexpr int XS_BYTES = 3 * C::TC * (int)sizeof(typename C::Acc);  // one simulation's slice
  static constexpr int STAGE_BYTES = DATA_BYTES + SCALE_BYTES + SB * XS_BYTES;
  // half storage: the consumer warps' column sums of a chunk, double buffered
  static constexpr int CB_BYTES = HALF ? 2 * NCW * SB * 3 * C::TC * (int)sizeof(typename C::Acc) : 0;
  // ring depth: up to C::STAGES within 226 KB of shared memory (the
  // barriers and the abort flag fill the rest of the 227 KB a CTA may have)
  static constexpr int STAGES = (C::STAGES * STAGE_BYTES + CB_BYTES <= 226 * 1024)
                                    ? C::STAGES
                                    : (226 * 1024 - CB_BYTES) / STAGE_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + CB_BYTES + 2 * STAGES * 8 + 16;
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory of one CTA");
  static constexpr int THREADS = (NCW + 1) * 32;
  static_assert(STAGES >= 2, "at least a double-buffered ring");
  static_assert(C::TR % NCW == 0 && (!HALF || (NCW * 32) % C::TC == 0), "whole rows per warp, whole column sets");
  static_assert(C::TC == 32 * C::VEC, "a warp covers one chunk row");
  static_assert(3 * RPW <= 32, "one lane per (row, component) in the flush");
  static_assert(DATA_BYTES % 16 == 0 && SCALE_BYTES % 16 == 0 && XS_BYTES % 16 == 0, "bulk copy sizes");
};

// ---- per-precision load of VEC adjacent values of one plane row ----------
template <int PREC>
__device__ __forceinline__ void load_vals(const unsigned char *stage, int plane, int row, int lane,
                                          typename MvCfg<PREC>::Acc v[MvCfg<PREC>::VEC]) {
  using C = MvCfg<PREC>;
  if constexpr (PREC == MT_F32 || PREC == kF32Planar) {
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
  int64_t CH;     // stored chunks per group of simulations
  float *colpart; // half storage: column sums [unit][SB][3][TC]
  int *arrive;    // half storage: k_half_cols arrival counters [B][Q], zeroed by k_matvec
  int B;
};

// slices of a column chunk's panel range in k_half_cols: about 32 panels each
inline int half_col_slices(int64_t P) { return (int)std::max<int64_t>(1, std::min<int64_t>(64, (P + 31) / 32)); }

// Units in storage order: (group of simulations g, stored chunk c) with c
// the chunk (panel p, column chunk q).  Without half storage c = p Q + q;
// with it panel p holds chunks q0(p) .. Q-1 (see half_cum).
struct UnitCursor {
  int64_t g, p, q, c;
};
template <int K, bool HALF>
__device__ __forceinline__ void unit_decode(const MvArgs &A, int64_t u, UnitCursor &cu) {
  cu.g = u / A.CH;
  cu.c = u - cu.g * A.CH;
  if (!HALF) {
    cu.p = cu.c / A.Q;
    cu.q = cu.c - cu.p * A.Q;
    return;
  }
  int64_t lo = 0, hi = A.P - 1;  // the last panel whose first chunk is <= c
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (half_cum(mid, A.Q, K) <= cu.c) lo = mid;
    else hi = mid - 1;
  }
  cu.p = lo;
  cu.q = half_q0(lo, K) + (cu.c - half_cum(lo, A.Q, K));
}
template <int K, bool HALF>
__device__ __forceinline__ void unit_next(const MvArgs &A, UnitCursor &cu) {
  ++cu.c;
  if (++cu.q == A.Q) {
    ++cu.p;
    cu.q = HALF ? half_q0(cu.p, K) : 0;
  }
  if (cu.c == A.CH) {
    cu.c = 0;
    ++cu.g;
    cu.p = 0;
    cu.q = 0;
  }
}
// first unit of panel p of group g
template <int K, bool HALF>
__device__ __forceinline__ int64_t panel_first_unit(const MvArgs &A, int64_t g, int64_t p) {
  return g * A.CH + (HALF ? half_cum(p, A.Q, K) : p * A.Q);
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

template <int PREC, int SB, bool HALF>
__global__ void __launch_bounds__(MvShape<PREC, SB, HALF>::THREADS, 1) k_matvec(MvArgs A) {
  mtd::pdl_enter();
  using C = MvCfg<PREC>;
  using S = MvShape<PREC, SB, HALF>;
  if constexpr (HALF) {  // the column pass that follows counts its arrivals from zero
    for (int64_t k = blockIdx.x * (int64_t)S::THREADS + threadIdx.x; k < (int64_t)A.B * A.Q;
         k += (int64_t)gridDim.x * S::THREADS)
      A.arrive[k] = 0;
  }
  using Acc = typename C::Acc;
  constexpr int K = C::TC / C::TR;  // panels per column chunk
  extern __shared__ __align__(128) unsigned char smem[];
  Acc *cb = reinterpret_cast<Acc *>(smem + S::STAGES * S::STAGE_BYTES);  // half: column sums
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + S::STAGES * S::STAGE_BYTES + S::CB_BYTES);
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
      unit_decode<K, HALF>(A, u0, cu);
      for (int64_t u = u0; u < u1; ++u, unit_next<K, HALF>(A, cu)) {
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
  Acc xi[HALF ? SB : 1][S::RPW][3];  // half: the operand of this warp's rows (the transposed product)
  int64_t gp_cur = -1;
  int it = 0, strict_it = 0;
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
    const int64_t pu0 = panel_first_unit<K, HALF>(A, g, p), pu1 = panel_first_unit<K, HALF>(A, g, p + 1);
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
      if (writer)
        for (int m = 0; m < SB; ++m) {
          Acc tot = 0;
          for (int64_t kk = kf; kk <= kl; ++kk) {
            // slot of CTA kk: 2 kk if this panel is its first, else 2 kk + 1
            const int64_t sl = (mtd::sk_begin(kk, U, G) >= pu0) ? 2 * kk : 2 * kk + 1;
            tot += __ldcg(&part[((sl * SB + m) * C::TR + row_in_panel) * 3 + lc]);
          }
          Acc *H = out(m);
          if (H && row < A.n) H[3 * row + lc] = -tot;
        }
      if (lane == 0) A.count[gp * S::NCW + warp] = 0;  // ready for the next launch
    }
  };

  UnitCursor cu;
  unit_decode<K, HALF>(A, u0, cu);
  for (int64_t u = u0; u < u1; ++u, unit_next<K, HALF>(A, cu)) {
    const int64_t g = cu.g, gp = g * A.P + cu.p;
    if (!group_live(A, g, SB)) continue;
    if (gp != gp_cur) {
      if (gp_cur >= 0) flush(gp_cur);
      gp_cur = gp;
#pragma unroll
      for (int m = 0; m < SB; ++m)
#pragma unroll
        for (int r = 0; r < S::RPW; ++r) acc[m][r][0] = acc[m][r][1] = acc[m][r][2] = 0;
      if constexpr (HALF) {
        // the operand of this warp's rows, for the transposed product
        const Acc *xsg = reinterpret_cast<const Acc *>(A.xs);
#pragma unroll
        for (int m = 0; m < SB; ++m) {
          const int64_t b = g * SB + m < A.B ? g * SB + m : 0;
#pragma unroll
          for (int r = 0; r < S::RPW; ++r) {
            const int64_t i = cu.p * C::TR + warp * S::RPW + r;
            const int64_t qi = i / C::TC, ti = i - qi * C::TC;
#pragma unroll
            for (int c = 0; c < 3; ++c) xi[m][r][c] = __ldg(&xsg[((b * A.Q + qi) * 3 + c) * C::TC + ti]);
          }
        }
      }
    }
    // an off-diagonal chunk of the half storage also serves its columns
    const bool strict = HALF && cu.q > half_q0(cu.p, K);
    Acc colp[HALF ? SB : 1][C::VEC][3];
    if constexpr (HALF) {
#pragma unroll
      for (int m = 0; m < SB; ++m)
#pragma unroll
        for (int v = 0; v < C::VEC; ++v) colp[m][v][0] = colp[m][v][1] = colp[m][v][2] = 0;
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
          if constexpr (HALF) {
            if (strict) {
              // block (row, v) transposed: the same symmetric block times this row's operand
#pragma unroll
              for (int m = 0; m < SB; ++m)
#pragma unroll
                for (int v = 0; v < C::VEC; ++v) {
                  colp[m][v][0] = fma(nxx[v], xi[m][r][0], fma(nxy[v], xi[m][r][1], colp[m][v][0]));
                  colp[m][v][1] = fma(nxy[v], xi[m][r][0], fma(nyy[v], xi[m][r][1], colp[m][v][1]));
                  colp[m][v][2] = fma(nzz[v], xi[m][r][2], colp[m][v][2]);
                }
            }
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
        if constexpr (HALF) {
          if (strict) {
#pragma unroll
            for (int m = 0; m < SB; ++m)
#pragma unroll
              for (int v = 0; v < C::VEC; ++v) {
                colp[m][v][0] =
                    fma(nxx[v], xi[m][r][0], fma(nxy[v], xi[m][r][1], fma(nxz[v], xi[m][r][2], colp[m][v][0])));
                colp[m][v][1] =
                    fma(nxy[v], xi[m][r][0], fma(nyy[v], xi[m][r][1], fma(nyz[v], xi[m][r][2], colp[m][v][1])));
                colp[m][v][2] =
                    fma(nxz[v], xi[m][r][0], fma(nyz[v], xi[m][r][1], fma(nzz[v], xi[m][r][2], colp[m][v][2])));
              }
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mtd::mbar_arrive(&empty[s]);
    if constexpr (HALF) {
      if (strict) {
        // column sums of the chunk: each warp's partial (its rows) to shared
        // memory, then thread t sums column t % TC, components t / TC,
        // t / TC + NCW 32 / TC, ..., over the warps in order, and writes them
        // to the chunk's slot of the work area
        const int buf = strict_it & 1;
        ++strict_it;
        Acc *mine = cb + (size_t)((buf * S::NCW + warp) * SB) * 3 * C::TC;
#pragma unroll
        for (int m = 0; m < SB; ++m)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            *reinterpret_cast<float4 *>(mine + (m * 3 + c) * C::TC + lane * C::VEC) =
                make_float4(colp[m][0][c], colp[m][1][c], colp[m][2][c], colp[m][3][c]);
        asm volatile("bar.sync 1, %0;" ::"r"(S::NCW * 32) : "memory");
        constexpr int NT = S::NCW * 32 / C::TC;  // thread sets over the columns
        const int t = warp * 32 + lane, col = t % C::TC;
        const int64_t uu = cu.g * A.CH + cu.c;
#pragma unroll
        for (int m = 0; m < SB; ++m) {
          if (g * SB + m >= A.B) continue;
#pragma unroll
          for (int c0 = 0; c0 < 3; c0 += NT) {
            const int c = c0 + t / C::TC;
            if (c >= 3) break;
            Acc tot = 0;
#pragma unroll
            for (int w = 0; w < S::NCW; ++w) tot += cb[((size_t)((buf * S::NCW + w) * SB + m) * 3 + c) * C::TC + col];
            A.colpart[((uu * SB + m) * 3 + c) * C::TC + col] = tot;
          }
        }
      }
    }
  }
  if (gp_cur >= 0) flush(gp_cur);
}

// Half storage: the transposed part of the product.  Column j of chunk q
// received, from every panel p whose chunk (p, q) lies above the diagonal
// (p < K q), the column sums that chunk left in the work area.  CTA (q, s, b)
// sums the panels of slice s of that range (NS slices, in increasing p) and
// parks its sums; the last CTA of (q, b) to arrive adds the NS slice sums in
// slice order (a fixed order: the result does not depend on timing) and
// does H_j -= total.  One thread per column of the chunk.
__global__ void __launch_bounds__(128) k_half_cols(MvArgs A, int SB, int TC, int K, int NS, float *slice_sum) {
  mtd::pdl_enter();
  const int64_t q = blockIdx.x;
  const int sl = blockIdx.y, b = blockIdx.z;
  const int t = threadIdx.x;
  const int64_t np = K * q;  // panels above the diagonal of chunk q
  const int64_t len = (np + NS - 1) / NS;
  const int64_t pa = sl * len, pb = np < pa + len ? np : pa + len;
  const int64_t g = b / SB, m = b - g * SB;
  float tot[3] = {0.0f, 0.0f, 0.0f};
  // walk the panels with the chunk (p, q)'s unit index kept up to date:
  // panel p holds chunks q0(p) .. Q-1, q0 growing by one every K panels
  int64_t q0 = pa / K, cum = g * A.CH + half_cum(pa, A.Q, K);
  int kk = (int)(pa - q0 * K);
  const float *base = A.colpart + m * 3 * TC + t;
  const int64_t ustride = (int64_t)SB * 3 * TC;
  auto next = [&] {
    cum += A.Q - q0;
    if (++kk == K) {
      kk = 0;
      ++q0;
    }
  };
  int64_t p = pa;
  for (; p + 4 <= pb; p += 4) {  // four panels' loads in flight
    float v[4][3];
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      const float *cp = base + (cum + (q - q0)) * ustride;
      v[k2][0] = __ldcg(cp);
      v[k2][1] = __ldcg(cp + TC);
      v[k2][2] = __ldcg(cp + 2 * TC);
      next();
    }
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      tot[0] += v[k2][0];
      tot[1] += v[k2][1];
      tot[2] += v[k2][2];
    }
  }
  for (; p < pb; ++p) {
    const float *cp = base + (cum + (q - q0)) * ustride;
    tot[0] += __ldcg(cp);
    tot[1] += __ldcg(cp + TC);
    tot[2] += __ldcg(cp + 2 * TC);
    next();
  }
  const int64_t qb = (int64_t)b * A.Q + q;
  float *mine = slice_sum + ((qb * NS + sl) * 3) * TC + t;
  mine[0] = tot[0];
  mine[TC] = tot[1];
  mine[2 * TC] = tot[2];
  __threadfence();
  __syncthreads();
  __shared__ int last;
  if (t == 0) last = (atomicAdd(&A.arrive[qb], 1) == NS - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int64_t j = q * TC + t;
  if (j >= A.n || (A.active && !A.active[b])) return;
  float v[3] = {0.0f, 0.0f, 0.0f};
  for (int k2 = 0; k2 < NS; ++k2) {
    const float *ss = slice_sum + ((qb * NS + k2) * 3) * TC + t;
    v[0] += __ldcg(ss);
    v[1] += __ldcg(ss + TC);
    v[2] += __ldcg(ss + 2 * TC);
  }
  float *H = reinterpret_cast<float *>(A.H) + (size_t)b * 3 * A.n + 3 * j;
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
  return PREC == MT_F32 || PREC == kF32Planar;
}

template <int PREC, int SB>
cudaError_t prepare_mv_one() {
  cudaError_t e = cudaFuncSetAttribute(k_matvec<PREC, SB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       MvShape<PREC, SB, false>::SMEM_BYTES);
  if constexpr (has_half<PREC>()) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_matvec<PREC, SB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               MvShape<PREC, SB, true>::SMEM_BYTES);
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
// for 4 simulations at n = 10,000 against 0.21 ms for one)
inline int mv_group(int B, int prec) {
  const int cap = (prec == MT_BF16_SCALED || prec == kBF16Planar) ? 2 : 4;
  return B <= 1 ? 1 : (B == 2 || cap == 2) ? 2 : 4;
}

template <int PREC, int SB>
void launch_mv_sb(const MvArgs &A, bool half, int grid_cap, cudaStream_t s) {
  // never more CTAs than units: every CTA then owns at least one unit, which
  // the panel bookkeeping (owners of a panel's first and last unit bound its
  // contributors) relies on
  const int64_t U = (int64_t)((A.B + SB - 1) / SB) * A.CH;
  const int grid = (int)std::min<int64_t>(grid_cap, U);
  if constexpr (has_half<PREC>()) {
    if (half) {
      using S = MvShape<PREC, SB, true>;
      static_assert(MvCfg<PREC>::TC % MvCfg<PREC>::TR == 0, "panels tile a chunk row");
      // the work area: chunk sums, then the slice sums and arrival counters
      // of the column pass
      constexpr int TC = MvCfg<PREC>::TC;
      const int ns = half_col_slices(A.P);
      const int64_t ng = (A.B + SB - 1) / SB;
      float *slice_sum = A.colpart + (size_t)ng * SB * A.CH * 3 * TC;
      MvArgs A2 = A;
      A2.arrive = reinterpret_cast<int *>(slice_sum + (size_t)A.B * A.Q * ns * 3 * TC);
      mt::launch_pdl(k_matvec<PREC, SB, true>, dim3(grid), dim3(S::THREADS), S::SMEM_BYTES, s, A2);
      // the transposed part, summed per column
      mt::launch_pdl(k_half_cols, dim3((unsigned)A.Q, (unsigned)ns, (unsigned)A.B), dim3(TC), 0, s, A2, SB, TC,
                     TC / MvCfg<PREC>::TR, ns, slice_sum);
      return;
    }
  }
  using S = MvShape<PREC, SB, false>;
  mt::launch_pdl(k_matvec<PREC, SB, false>, dim3(grid), dim3(S::THREADS), S::SMEM_BYTES, s, A);
}

template <int PREC>
void launch_mv(const mt_tensor *T, const void *xs, int B, void *H, void *part, int *count, const int *active,
               int *status, float *colpart, cudaStream_t s) {
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
  A.colpart = colpart;
  A.arrive = nullptr;
  A.B = B;
  const int cap = mt::matvec_grid(T);
  const bool half = T->L.half;
  switch (mv_group(B, PREC)) {
    case 1: launch_mv_sb<PREC, 1>(A, half, cap, s); break;
    case 2: launch_mv_sb<PREC, 2>(A, half, cap, s); break;
    default:
      if constexpr (PREC != MT_BF16_SCALED && PREC != kBF16Planar) launch_mv_sb<PREC, 4>(A, half, cap, s);
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
  return (size_t)2 * matvec_grid(T) * 4 /*simulations per chunk read, at most*/ * T->L.TR * 3 * el;
}

size_t matvec_count_bytes(const mt_tensor *T, int B) { return (size_t)B * T->L.P * 8 /*W<=8*/ * sizeof(int); }

// half storage: the column sums of every stored chunk for B simulations
// (groups of up to 4 share a chunk read; a partial group keeps its slots),
// then the slice sums of k_half_cols and its arrival counters (a call with
// fewer simulations uses a prefix of each part)
size_t matvec_colpart_bytes(const mt_tensor *T, int B) {
  if (!T->L.half) return 0;
  const int sb = mv_group(B, T->L.nplane == 4 ? kF32Planar : MT_F32);
  const int64_t ng = (B + sb - 1) / sb;
  const int ns = half_col_slices(T->L.P);
  return (size_t)ng * sb * T->L.CH * 3 * T->L.TC * sizeof(float) +
         (size_t)B * T->L.Q * ns * 3 * T->L.TC * sizeof(float) + (size_t)B * T->L.Q * sizeof(int);
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
      if (T->L.nplane == 4) launch_mv<kF32Planar>(T, xs, B, H, part, count, active, status, colpart, s);
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
