// Batched demag product on the 5th-generation tensor cores (tcgen05).
//
// B simulations on one geometry turn the product H_d = -N (Ms m) (Eq. 9,
// Eq. 17) into a GEMM: D[3n x B] = N[3n x 3n] X^T with X[b] = Ms m_b.  The
// tensor is stored dense (all 9 entries of each block, row r = 3i + a,
// column c = 3j + b) in BF16, or as a BF16 hi + lo pair ("split").  The
// split product carries the operand as three BF16 terms x0 + x1 + x2 (24
// significant bits: a relaxed, nearly uniform state would otherwise round
// every x the same way and leave a coherent error) and forms
// N_hi (x0 + x1 + x2) + N_lo (x0 + x1); the blocks of touching tiles are
// zero there and are applied with FP64-class accuracy by the near-field
// kernel.
//
// The GEMM is HBM-bound for B <= ~300 (64 flop per tensor byte at B = 64),
// so the design streams the tensor once per batched product:
//   * persistent CTAs, one per SM; the (row tile, K block) units are split
//     evenly over the CTAs in storage order (stream-K);
//   * warp 0 issues 2-D TMA loads (128-byte swizzle) of a 128 x 64 tensor
//     tile and the 64-wide slice of X^T into a shared-memory ring;
//   * warp 1 issues tcgen05.mma (M = 128, N = B, K = 16, BF16 -> FP32) into
//     a ring of four TMEM accumulators, each filled over a few K blocks (the
//     tensor cores' FP32 accumulation rounds with a bias, so chains stay
//     short), and releases ring slots with tcgen05.commit;
//   * warps 2-5 drain each finished accumulator with tcgen05.ld (one TMEM
//     lane = one row per thread) into FP32 register sums while the next ones
//     fill; rows split between two CTAs are summed by whichever warp arrives
//     last, in CTA order;
//   * the number of K blocks per accumulator and the ring depth are chosen
//     per tensor and batch width by timing candidates on first use.
// Every wait is bounded; on a timeout the kernel records MT_DEV_TIMEOUT,
// still frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "mt_internal.cuh"

namespace {

constexpr int GM = 128;  // rows per tile (MMA M)
constexpr int GK = 64;   // K per ring stage: one 128-byte swizzle row of BF16
constexpr int EPI_WARPS = 4;
constexpr int NACC = 4;  // TMEM accumulators in flight between the MMA warp and the epilogue

// The split product with a padded batch up to 64 "stacks" the three operand
// planes x0 | x1 | x2 into one N = 3 Bp operand: one MMA gives N_hi x0,
// N_hi x1, N_hi x2 side by side in TMEM and a second (N = 2 Bp) adds N_lo x0
// and N_lo x1 onto the first two groups; the epilogue adds the groups in
// FP32.  That reads each tensor tile from shared memory twice per K step
// instead of five times (the split product was bound by the shared-memory
// reads that feed the tensor cores).  N <= 256 limits it to Bp <= 64; wider
// batches issue the five MMAs.
template <bool SPLIT, int BP>
struct GemmShape {
  static constexpr bool STACK = SPLIT && BP <= 64;
  static constexpr int ACC_COLS = STACK ? 3 * BP : BP;  // TMEM columns of one accumulator
  // accumulators (<= 512 TMEM columns); the BF16 product at BP <= 64 keeps 8
  // in flight
  static constexpr int NA = STACK ? (BP == 64 ? 2 : 4) : (BP <= 64 ? 2 * NACC : NACC);
};
constexpr int GEMM_THREADS = 32 * (2 + EPI_WARPS);

// ---- tcgen05 / TMA wrappers -------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(mtd::smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (tmem) = A (smem) * B (smem) [+ D]; BF16 inputs, FP32 accumulate
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on `bar` once every tcgen05.mma issued so far by this thread is done
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   mtd::smem_u32(bar))
               : "memory");
}
// 32 lanes x 32 bit, 16 consecutive columns per thread; the registers are
// valid only after tmem_wait_ld()
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t r[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar,
                                       uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(mtd::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mtd::smem_u32(bar)), "l"(policy)
      : "memory");
}
// shared-memory matrix descriptor: K-major tile, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

struct GemmArgs {
  int64_t n3;    // valid rows (3n)
  int64_t MT;    // row tiles
  int64_t KB;    // K blocks
  int64_t KBU;   // units per row tile (a unit = KPS consecutive K blocks)
  int B, Bp;     // batch, padded batch (MMA N)
  int chunk;     // K blocks per TMEM accumulation before the FP32 promotion
  int stages;
  int stage_bytes;
  uint32_t tmem_cols;
  float *H;      // [B][n3]
  float *part;   // [2G][Bp][GM]
  int *count;    // [MT][EPI_WARPS]
  const int *n_active;
  int *status;
};

template <bool SPLIT, int BP, int KPS>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    k_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tAlo,
           const __grid_constant__ CUtensorMap tX, const __grid_constant__ CUtensorMap tX1,
           const __grid_constant__ CUtensorMap tX2, GemmArgs P) {
  mtd::pdl_enter();
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned base for the swizzled tiles
  const uint32_t raw = mtd::smem_u32(smem_raw);
  unsigned char *smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const int A_BYTES = GM * GK * 2;
  const int X_BYTES = P.Bp * GK * 2;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)P.stages * P.stage_bytes);
  uint64_t *empty = full + P.stages;
  uint64_t *accf = empty + P.stages;
  using SH = GemmShape<SPLIT, BP>;
  constexpr int NA = SH::NA;
  uint64_t *acce = accf + NA;
  uint64_t *mma_done = acce + NA;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = gridDim.x, k = blockIdx.x;
  // a unit is KPS consecutive K blocks of one row tile; a ring stage holds
  // one unit: KPS sub-blocks of [A (| x0 | A_lo | x1 | x2) | X]
  const int SB = SPLIT ? 2 * A_BYTES + 3 * X_BYTES : A_BYTES + X_BYTES;
  const int64_t U = P.MT * P.KBU;
  const int64_t u0 = mtd::sk_begin(k, U, G), u1 = mtd::sk_begin(k + 1, U, G);
  const bool idle = P.n_active && *P.n_active == 0;  // every simulation finished

  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) {
      mtd::mbar_init(&full[s], 1);
      mtd::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < NA; ++a) {
      mtd::mbar_init(&accf[a], 1);
      mtd::mbar_init(&acce[a], EPI_WARPS);
    }
    mtd::mbar_init(mma_done, 1);
    *abort_flag = 0;
    mtd::fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, P.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (!idle && warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    const uint64_t pol_stream = mtd::policy_evict_first();
    const uint64_t pol_keep = mtd::policy_evict_last();
    int it = 0;
    for (int64_t u = u0; u < u1; ++u, ++it) {
      const int64_t mt = u / P.KBU, kbu = u - mt * P.KBU;
      const int s = it % P.stages;
      const uint32_t ph = (uint32_t)(it / P.stages) & 1u;
      if (it >= P.stages && (*abort_flag || !mtd::mbar_wait_bounded(&empty[s], ph ^ 1u, P.status))) {
        *abort_flag = 1;
        break;
      }
      unsigned char *st = smem + (size_t)s * P.stage_bytes;
      mtd::mbar_arrive_expect_tx(&full[s], (uint32_t)(KPS * SB));
#pragma unroll
      for (int q = 0; q < KPS; ++q) {
        // tile (mt, kb) is one contiguous 16 KB block; X block kb likewise
        const int64_t kb = kbu * KPS + q;
        const int ya = (int)((mt * P.KB + kb) * GM), yx = (int)(kb * P.Bp);
        unsigned char *sb = st + q * SB;
        tma_2d(sb, &tA, 0, ya, &full[s], pol_stream);
        if (SPLIT) {
          // sub-block: A_hi | A_lo | x0 | x1 | x2 (the planes of x adjacent:
          // one 3 Bp-row operand)
          tma_2d(sb + A_BYTES, &tAlo, 0, ya, &full[s], pol_stream);
          tma_2d(sb + 2 * A_BYTES, &tX, 0, yx, &full[s], pol_keep);
          tma_2d(sb + 2 * A_BYTES + X_BYTES, &tX1, 0, yx, &full[s], pol_keep);
          tma_2d(sb + 2 * A_BYTES + 2 * X_BYTES, &tX2, 0, yx, &full[s], pol_keep);
        } else {
          tma_2d(sb + A_BYTES, &tX, 0, yx, &full[s], pol_keep);
        }
      }
    }
    // drain: every copy issued must have landed before the CTA may exit
    for (int s = 0; s < P.stages && s < it; ++s) {
      const int last = it - 1 - ((it - 1 - s) % P.stages);  // last issue on stage s
      mtd::mbar_wait_bounded(&full[s], (uint32_t)(last / P.stages) & 1u, P.status);
    }
  } else if (!idle && warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = (1u << 4)                       // D: FP32
                           | (1u << 7) | (1u << 10)        // A, B: BF16
                           | ((uint32_t)(P.Bp >> 3) << 17)  // N
                           | ((uint32_t)(GM >> 4) << 24);   // M
    // stacked split: N = 3 Bp (N_hi [x0 | x1 | x2]) and N = 2 Bp (N_lo [x0 | x1])
    const uint32_t idesc3 = (idesc & ~(0x3Fu << 17)) | ((uint32_t)((3 * BP) >> 3) << 17);
    const uint32_t idesc2 = (idesc & ~(0x3Fu << 17)) | ((uint32_t)((2 * BP) >> 3) << 17);
    // The tensor cores' FP32 accumulation rounds with a bias, so a product
    // is accumulated in TMEM over at most P.chunk K blocks and then handed to
    // the epilogue, which adds the chunks in FP32 (round to nearest).
    int it = 0, chunk = 0;
    bool issued = false;
    int64_t u = u0;
    while (u < u1 && !*abort_flag) {
      const int64_t mt = u / P.KBU;
      const int64_t seg_end = u1 < (mt + 1) * P.KBU ? u1 : (mt + 1) * P.KBU;
      while (u < seg_end && !*abort_flag) {
        const int64_t c_end = seg_end < u + P.chunk ? seg_end : u + P.chunk;
        const int a = chunk % NA;
        if (chunk >= NA && !mtd::mbar_wait_bounded(&acce[a], (uint32_t)(chunk / NA - 1) & 1u, P.status)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(a * SH::ACC_COLS);
        bool first = true;
        for (; u < c_end; ++u, ++it) {
          const int s = it % P.stages;
          const uint32_t ph = (uint32_t)(it / P.stages) & 1u;
          if (*abort_flag || !mtd::mbar_wait_bounded(&full[s], ph, P.status)) {
            *abort_flag = 1;
            break;
          }
          tc_fence_after();
          const uint32_t st = mtd::smem_u32(smem + (size_t)s * P.stage_bytes);
#pragma unroll
          for (int q = 0; q < KPS; ++q) {
            const uint32_t sa = st + q * SB;
#pragma unroll
            for (int kk = 0; kk < GK / 16; ++kk) {
              // K advance inside the 128-byte swizzle row: 16 BF16 = 32 bytes
              const uint64_t da = sw128_desc(sa + 32 * kk);
              if (!SPLIT) {
                umma_bf16(d_tmem, da, sw128_desc(sa + A_BYTES + 32 * kk), idesc, first ? 0u : 1u);
              } else if (SH::STACK) {
                const uint32_t salo = sa + A_BYTES, sx = salo + A_BYTES;
                const uint64_t dx = sw128_desc(sx + 32 * kk);
                umma_bf16(d_tmem, da, dx, idesc3, first ? 0u : 1u);                  // N_hi [x0 | x1 | x2]
                umma_bf16(d_tmem, sw128_desc(salo + 32 * kk), dx, idesc2, 1u);       // N_lo [x0 | x1]
              } else {
                const uint32_t salo = sa + A_BYTES, sx = salo + A_BYTES, sx1 = sx + X_BYTES, sx2 = sx1 + X_BYTES;
                const uint64_t dx = sw128_desc(sx + 32 * kk), d1 = sw128_desc(sx1 + 32 * kk);
                const uint64_t dlo = sw128_desc(salo + 32 * kk);
                umma_bf16(d_tmem, da, dx, idesc, first ? 0u : 1u);            // N_hi x0
                umma_bf16(d_tmem, da, d1, idesc, 1u);                         // N_hi x1
                umma_bf16(d_tmem, da, sw128_desc(sx2 + 32 * kk), idesc, 1u);  // N_hi x2
                umma_bf16(d_tmem, dlo, dx, idesc, 1u);                        // N_lo x0
                umma_bf16(d_tmem, dlo, d1, idesc, 1u);                        // N_lo x1
              }
              first = false;
            }
          }
          issued = true;
          umma_commit(&empty[s]);  // ring slot free once these MMAs are done
        }
        umma_commit(&accf[a]);  // accumulator a holds the chunk
        ++chunk;
      }
    }
    if (issued) umma_commit(mma_done);
    else mtd::mbar_arrive(mma_done);
  } else if (!idle && warp >= 2) {
    // ---------------- epilogue ----------------
    const int g = warp & 3;  // TMEM lane group accessible to this warp
    const int row = g * 32 + lane;
    const int64_t first_mt = u0 / P.KBU;
    int chunk = 0;
    int64_t u = u0;
    float run[BP];  // FP32 sum of the chunks of the current row tile
    while (u < u1) {
      const int64_t mt = u / P.KBU;
      const int64_t seg_end = u1 < (mt + 1) * P.KBU ? u1 : (mt + 1) * P.KBU;
      bool ok = true;
      bool first_chunk = true;
      while (u < seg_end) {
        u = seg_end < u + P.chunk ? seg_end : u + P.chunk;
        const int a = chunk % NA;
        const bool got = !*abort_flag && mtd::mbar_wait_bounded(&accf[a], (uint32_t)(chunk / NA) & 1u, P.status);
        if (!got) {
          *abort_flag = 1;
          ok = false;
        }
        tc_fence_after();
        const uint32_t acc = tmem_base + ((uint32_t)(g * 32) << 16) + (uint32_t)(a * SH::ACC_COLS);
        if (SH::STACK) {
          // the three column groups x0, x1, x2 of each 16-column piece, the
          // two small ones added first
#pragma unroll
          for (int c0 = 0; c0 < BP; c0 += 16) {
            uint32_t v0[16], v1[16], v2[16];
            tmem_ld16(acc + (uint32_t)c0, v0);
            tmem_ld16(acc + (uint32_t)(BP + c0), v1);
            tmem_ld16(acc + (uint32_t)(2 * BP + c0), v2);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float x = __uint_as_float(v0[j]) + (__uint_as_float(v1[j]) + __uint_as_float(v2[j]));
              run[c0 + j] = first_chunk ? x : run[c0 + j] + x;
            }
          }
        } else {
          // all loads of the accumulator in flight at once, one wait
          uint32_t v[BP];
#pragma unroll
          for (int c0 = 0; c0 < BP; c0 += 16) tmem_ld16(acc + (uint32_t)c0, &v[c0]);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < BP; ++j)
            run[j] = first_chunk ? __uint_as_float(v[j]) : run[j] + __uint_as_float(v[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mtd::mbar_arrive(&acce[a]);
        first_chunk = false;
        ++chunk;
      }
      if (!ok) continue;
      const int64_t kf = mtd::sk_owner(mt * P.KBU, U, G), kl = mtd::sk_owner(mt * P.KBU + P.KBU - 1, U, G);
      const int64_t r = mt * GM + row;
      if (kf == kl) {
#pragma unroll
        for (int b = 0; b < BP; ++b)
          if (b < P.B && r < P.n3) P.H[(size_t)b * P.n3 + r] = -run[b];
        continue;
      }
      const int64_t slot = (mt == first_mt) ? 2 * k : 2 * k + 1;
#pragma unroll
      for (int b = 0; b < BP; ++b) P.part[((size_t)slot * BP + b) * GM + row] = run[b];
      __threadfence();
      __syncwarp();
      int last = 0;
      if (lane == 0) {
        const int old = atomicAdd(&P.count[mt * EPI_WARPS + g], 1);
        last = (old == (int)(kl - kf));
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      if (last) {
        __threadfence();
        // 16 simulations at a time: all their parts loaded (in CTA order per
        // simulation) before their stores to H, which the compiler cannot
        // move loads across
        for (int b0 = 0; b0 < P.B; b0 += 16) {
          float tot[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) tot[j] = 0.0f;
          for (int64_t kk = kf; kk <= kl; ++kk) {
            const int64_t fm = mtd::sk_begin(kk, U, G) / P.KBU;
            const int64_t sl = (mt == fm) ? 2 * kk : 2 * kk + 1;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (b0 + j < P.B) tot[j] += __ldcg(&P.part[((size_t)sl * BP + b0 + j) * GM + row]);
          }
          if (r < P.n3)
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (b0 + j < P.B) P.H[(size_t)(b0 + j) * P.n3 + r] = -tot[j];
        }
        if (lane == 0) P.count[mt * EPI_WARPS + g] = 0;
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    if (!idle) mtd::mbar_wait_bounded(mma_done, 0u, P.status);
    tc_fence_after();
    tmem_dealloc(tmem_base, P.tmem_cols);
  }
}

// X[b][c] = BF16(Ms_j m_j[a]) for c = 3j + a (zero for padding), and the
// low part X_lo = BF16(x - X_hi) for the split product
__global__ void k_prep_dense_x(const float *m, const float *Ms, int64_t n, int64_t Kp, int B, int Bp,
                               __nv_bfloat16 *X, __nv_bfloat16 *X1, __nv_bfloat16 *X2, float *mT) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (t >= Kp) return;
  float x = 0.0f;
  if (t < 3 * n) {
    const float mv = m[(size_t)b * 3 * n + t];
    x = Ms[t / 3] * mv;
    mT[(size_t)t * Bp + b] = mv;
  }
  const __nv_bfloat16 hi = __float2bfloat16(x);
  const size_t at = dense_x_index(b, t, Bp);
  X[at] = hi;
  if (X1) {  // three-term split x = x0 + x1 + x2
    const float r = x - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16(r);
    X1[at] = mid;
    X2[at] = __float2bfloat16(r - __bfloat162float(mid));
  }
}

using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

// 2-D BF16 map over a row-major [rows][cols] array, box (64 cols, box_rows)
mt_status make_map(CUtensorMap *map, const void *base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
  EncodeFn fn = encode_fn();
  MT_CHECK(fn, MT_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)GK, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  MT_CHECK(r == CUDA_SUCCESS, MT_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return MT_OK;
}

// Tile shape along K: the K blocks (64 columns each) one ring stage holds,
// 1 or 2 (a stage of 16 or 32 KB of tensor per plane), chosen by the
// autotuner together with the ring depth; the split product at a padded
// batch of 128 holds one (two would need 160 KB a stage: no room for two).
constexpr int kps_max(bool split, int Bp) { return split && Bp > 64 ? 1 : 2; }

int stage_bytes_for(int Bp, bool split, int kps) {
  return kps * (split ? 2 * GM * GK * 2 + 3 * Bp * GK * 2 : GM * GK * 2 + Bp * GK * 2);
}

int stages_for(int Bp, bool split, int kps) {
  const int stage = stage_bytes_for(Bp, split, kps);
  const int budget = 224 * 1024;
  return std::max(2, std::min(8, budget / stage));  // >= 2 stages always fit (stage <= 112 KB)
}

}  // namespace

namespace mt {

// MMA N of a batch: 16, 32, 64 or 128 (one kernel instance each)
int dense_pad_batch(int B) {
  int bp = 16;
  while (bp < B && bp < 128) bp *= 2;
  return bp;
}

// operand planes: 1 (BF16) or 3 (split: x0, x1, x2)
size_t dense_x_bytes(const mt_tensor *T, int B) {
  const size_t x = (size_t)dense_pad_batch(B) * T->Kp * 2 * (T->prec == MT_BF16_SPLIT ? 3 : 1);
  return x + (size_t)3 * T->n * dense_pad_batch(B) * sizeof(float);  // + simulation-fastest copy of m
}

float *dense_mT(const mt_tensor *T, int B, void *X) {
  const size_t x = (size_t)dense_pad_batch(B) * T->Kp * 2 * (T->prec == MT_BF16_SPLIT ? 3 : 1);
  return reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(X) + x);
}
size_t dense_part_bytes(const mt_tensor *T, int B) {
  return (size_t)2 * matvec_grid(T) * dense_pad_batch(B) * GM * sizeof(float);
}
size_t dense_count_bytes(const mt_tensor *T) { return (size_t)(T->Kp / GM) * EPI_WARPS * sizeof(int); }

// (Measured when a stage first held two K blocks: the per-stage handshakes
// of the TMA, MMA and commit path cost a fixed few hundred cycles, so 16 KB
// tiles alone left the BF16 product at 0.70 of HBM and two per stage reached
// 0.87; the split product went from 0.73 to 0.83 with a 2-deep ring of
// 112 KB.  Both shapes stay candidates of the autotuner.)
template <bool SPLIT, int BP>
cudaError_t prep_one() {
  cudaError_t e = cudaFuncSetAttribute(k_gemm<SPLIT, BP, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024);
  if (e == cudaSuccess && kps_max(SPLIT, BP) == 2)
    e = cudaFuncSetAttribute(k_gemm<SPLIT, BP, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  return e;
}

cudaError_t gemm_prepare() {
  cudaError_t e;
  if ((e = prep_one<false, 16>()) != cudaSuccess || (e = prep_one<false, 32>()) != cudaSuccess ||
      (e = prep_one<false, 64>()) != cudaSuccess || (e = prep_one<false, 128>()) != cudaSuccess ||
      (e = prep_one<true, 16>()) != cudaSuccess || (e = prep_one<true, 32>()) != cudaSuccess ||
      (e = prep_one<true, 64>()) != cudaSuccess || (e = prep_one<true, 128>()) != cudaSuccess)
    return e;
  return cudaSuccess;
}

void launch_prep_dense_x(const mt_tensor *T, const float *m, int B, void *X, cudaStream_t s) {
  const int Bp = dense_pad_batch(B);
  __nv_bfloat16 *x = reinterpret_cast<__nv_bfloat16 *>(X);
  const bool split = T->prec == MT_BF16_SPLIT;
  __nv_bfloat16 *x1 = split ? x + (size_t)Bp * T->Kp : nullptr;
  __nv_bfloat16 *x2 = split ? x + (size_t)2 * Bp * T->Kp : nullptr;
  dim3 grid((unsigned)((T->Kp + 255) / 256), (unsigned)B);
  k_prep_dense_x<<<grid, 256, 0, s>>>(m, T->tiles->d_Ms, T->n, T->Kp, B, Bp, x, x1, x2, dense_mT(T, B, X));
}

mt_status gemm_plan(const mt_tensor *T, int B, const void *X, GemmPlan *plan) {
  const int Bp = dense_pad_batch(B);
  MT_CHECK(B >= 1 && B <= 128, MT_EINVAL, "batched product: B = %d outside 1..128 simulations per pass", B);
  // TMA row coordinates are 32-bit: (row tile * K blocks + K block) * 128
  MT_CHECK((T->Kp / GM) * (T->Kp / GK) * (int64_t)GM < ((int64_t)1 << 31), MT_EINVAL,
           "batched product: the dense tensor (3n = %lld) exceeds the 32-bit TMA coordinate range",
           (long long)(3 * T->n));
  const bool split = T->prec == MT_BF16_SPLIT;
  const __nv_bfloat16 *A = reinterpret_cast<const __nv_bfloat16 *>(T->d_data);
  const __nv_bfloat16 *x = reinterpret_cast<const __nv_bfloat16 *>(X);
  mt_status st;
  // blocked storage seen as a [tiles * 128][64] array (A) and [KB * Bp][64] (X)
  const uint64_t a_rows = (uint64_t)T->Kp * T->Kp / GK, x_rows = (uint64_t)(T->Kp / GK) * Bp;
  if ((st = make_map(&plan->tA, A, GK, a_rows, GM)) != MT_OK) return st;
  if ((st = make_map(&plan->tX, x, GK, x_rows, Bp)) != MT_OK) return st;
  if (split) {
    if ((st = make_map(&plan->tAlo, A + (size_t)T->Kp * T->Kp, GK, a_rows, GM)) != MT_OK) return st;
    if ((st = make_map(&plan->tX1, x + (size_t)Bp * T->Kp, GK, x_rows, Bp)) != MT_OK) return st;
    if ((st = make_map(&plan->tX2, x + (size_t)2 * Bp * T->Kp, GK, x_rows, Bp)) != MT_OK) return st;
  } else {
    plan->tAlo = plan->tA;
    plan->tX1 = plan->tX;
    plan->tX2 = plan->tX;
  }
  plan->B = B;
  plan->Bp = Bp;
  plan->split = split;
  plan->kps = kps_max(split, Bp);
  plan->stages = stages_for(Bp, split, plan->kps);
  plan->chunk = 4 / plan->kps;  // units per accumulator chunk: 4 K blocks either way
  return MT_OK;
}

// The autotuner: per tensor and padded batch width, time the product for
// each tile shape along K (1 or 2 K blocks per ring stage) and three ring
// depths (the deepest that fits in shared memory and one and two stages
// shallower) and keep the fastest; numerics do not depend on the choice.
mt_status gemm_tune(mt_tensor *T, GemmPlan *plan, float *H, float *part, int *count, int *status, cudaStream_t s) {
  int key = 0;
  while ((16 << key) < plan->Bp) ++key;
  if (T->gemm_stages[key] > 0) {
    plan->stages = T->gemm_stages[key];
    plan->kps = T->gemm_kps[key];
    plan->chunk = 4 / plan->kps;
    return MT_OK;
  }
  cudaEvent_t e0, e1;
  MT_CUDA(cudaEventCreate(&e0));
  MT_CUDA(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  int best = 0, best_kps = plan->kps;
  for (int kps = kps_max(plan->split, plan->Bp); kps >= 1; --kps) {
    const int smax = stages_for(plan->Bp, plan->split, kps);
    const int cand[3] = {smax, std::max(2, smax - 1), std::max(2, smax - 2)};
    for (int c = 0; c < 3; ++c) {
      if (c > 0 && cand[c] == cand[c - 1]) continue;
      plan->kps = kps;
      plan->chunk = 4 / kps;
      plan->stages = cand[c];
      launch_gemm(T, *plan, H, part, count, nullptr, status, s);  // warm
      MT_CUDA(cudaEventRecord(e0, s));
      for (int r = 0; r < 3; ++r) launch_gemm(T, *plan, H, part, count, nullptr, status, s);
      MT_CUDA(cudaEventRecord(e1, s));
      MT_CUDA(cudaEventSynchronize(e1));
      float ms = 0.0f;
      MT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        best = cand[c];
        best_kps = kps;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  MT_CUDA(cudaGetLastError());
  T->gemm_stages[key] = best;
  T->gemm_kps[key] = best_kps;
  plan->stages = best;
  plan->kps = best_kps;
  plan->chunk = 4 / best_kps;
  return MT_OK;
}

void launch_gemm(const mt_tensor *T, const GemmPlan &plan, float *H, float *part, int *count, const int *n_active,
                 int *status, cudaStream_t s) {
  GemmArgs P;
  P.n3 = 3 * T->n;
  P.MT = T->Kp / GM;
  P.KB = T->Kp / GK;
  P.KBU = P.KB / plan.kps;
  P.B = plan.B;
  P.Bp = plan.Bp;
  P.chunk = plan.chunk;
  P.stages = plan.stages;
  P.stage_bytes = stage_bytes_for(plan.Bp, plan.split, plan.kps);
  const bool stack = plan.split && plan.Bp <= 64;
  const int acc_cols = stack ? 3 * plan.Bp : plan.Bp;
  const int na = stack ? (plan.Bp == 64 ? 2 : 4) : (plan.Bp <= 64 ? 2 * NACC : NACC);  // as GemmShape
  uint32_t cols = 32;
  while (cols < (uint32_t)(na * acc_cols)) cols <<= 1;
  P.tmem_cols = cols;
  P.H = H;
  P.part = part;
  P.count = count;
  P.n_active = n_active;
  P.status = status;
  const int64_t U = P.MT * P.KBU;
  const int grid = (int)std::min<int64_t>(matvec_grid(T), U);
  const size_t smem = (size_t)P.stages * P.stage_bytes + 1024 + 512;  // + alignment slack, barriers
#define MT_GEMM_LAUNCH_K(SP, BPV, K)                                                                            \
  mt::launch_pdl(k_gemm<SP, BPV, K>, dim3(grid), dim3(GEMM_THREADS), smem, s, plan.tA, plan.tAlo, plan.tX, plan.tX1, \
                 plan.tX2, P)
#define MT_GEMM_LAUNCH(SP, BPV)                          \
  do {                                                   \
    if (plan.kps == 2 && kps_max(SP, BPV) == 2)          \
      MT_GEMM_LAUNCH_K(SP, BPV, kps_max(SP, BPV));       \
    else                                                 \
      MT_GEMM_LAUNCH_K(SP, BPV, 1);                      \
  } while (0)
  if (plan.split) {
    switch (plan.Bp) {
      case 16: MT_GEMM_LAUNCH(true, 16); break;
      case 32: MT_GEMM_LAUNCH(true, 32); break;
      case 64: MT_GEMM_LAUNCH(true, 64); break;
      default: MT_GEMM_LAUNCH(true, 128); break;
    }
  } else {
    switch (plan.Bp) {
      case 16: MT_GEMM_LAUNCH(false, 16); break;
      case 32: MT_GEMM_LAUNCH(false, 32); break;
      case 64: MT_GEMM_LAUNCH(false, 64); break;
      default: MT_GEMM_LAUNCH(false, 128); break;
    }
  }
#undef MT_GEMM_LAUNCH
#undef MT_GEMM_LAUNCH_K
}

}  // namespace mt
