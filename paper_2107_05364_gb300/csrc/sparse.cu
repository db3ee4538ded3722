// Thresholded (sparse) tensor, Sec. 4.3.1 of the paper: the smallest
// fraction f of the nonzero tensor elements (by absolute value) is set to
// zero and the rest is stored as a sparse matrix, so the product reads only
// what is kept.
//
// Reading of the rule (drop the smallest fraction f of the nonzero elements): the elements
// are those of the full 3n x 3n matrix (an off-diagonal entry of a symmetric
// 3x3 block stands for two), ranked by magnitude of the stored FP32 value,
// ties in (row tile i, column tile j, entry) order with an off-diagonal
// entry's two copies adjacent; the first k = floor(f * nonzeros) are dropped,
// except that an entry whose two copies the cut splits stays (blocks stay
// symmetric).  The magnitude t of the element of rank k is found exactly by
// a two-pass radix select on the FP32 bit patterns (non-negative floats order
// like their bits); every element below t goes, and of the elements equal
// to t the first r = k - #(below t) in that order.
//
// Storage: block-sparse rows of tiles; a 3x3 block is kept if any of its
// entries survives, with its 6 unique entries (dropped ones zero), in
// increasing column order.  The threshold drops the blocks of distant tiles,
// so the kept columns of a row form long runs of consecutive tiles (about
// one per line of tiles): columns are stored as runs, not one index per
// block.  A run starts at a kept column; later kept columns join it while
// they are at most 4 columns past the last one (the gap is stored as zero
// blocks); each run is padded with zero blocks to a multiple of 4.  Row i
// holds K4 = ptr[i+1] - ptr[i] blocks as np planes of K4 floats,
// val[np ptr[i] + e K4 + a] (np = 6, or 4 when the source is a single-layer
// tensor without the xz and yz planes), and its runs rptr[i] .. rptr[i+1]-1
// as pairs (first block a0 within the row, first column c0): block a of the
// run has column c0 + (a - a0).  Every row and run starts on a 16-byte
// boundary, so a lane reads 4 blocks with np vector loads and their 4
// operands as one contiguous 64-byte stretch.
//
// Product: one warp per (tile row, simulation); the operand is a float4
// (Ms m, 0) per tile (n + 4 per simulation, the last 4 zero for padding that
// runs past the last tile), read from L2 in whole runs.  Partial sums are
// compensated (each addition's rounding error is kept by an error-free
// two-sum and added back at the end, Ogita, Rump and Oishi's Sum2), so the
// result does not depend on the long per-lane summation order to more than
// the FP32 storage error.
#include <algorithm>
#include <cstring>
#include <vector>

#include "mt_internal.cuh"

namespace {

__device__ __forceinline__ uint32_t abs_bits(float v) { return __float_as_uint(v) & 0x7fffffffu; }
__device__ __forceinline__ float f4_at(const float4 &v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }

// entries of the streaming FP32 layout belonging to real tiles, with their
// multiplicity in the full matrix (diagonal 1, off-diagonal 2)
template <typename F>
__device__ __forceinline__ void for_each_entry(const float *D, int64_t n, int TR, int TC, int np, int64_t Q,
                                               int64_t blk, F &&f) {
  // blk enumerates (p, q, r, c) chunk positions; the 6 entries of the block
  // (np planes stored: 6, or 4 for a single-layer tensor without xz, yz)
  const int64_t per_chunk = (int64_t)TR * TC;
  const int64_t chunk = blk / per_chunk, rc = blk - chunk * per_chunk;
  const int64_t p = chunk / Q, q = chunk - p * Q;
  const int r = (int)(rc / TC), c = (int)(rc - (int64_t)(rc / TC) * TC);
  const int64_t i = p * TR + r, j = q * TC + c;
  if (i >= n || j >= n) return;
  const float *base = D + chunk * np * per_chunk + (int64_t)r * TC + c;
  const int mult[6] = {1, 2, 2, 1, 2, 1};
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const int pl = stream_plane(e, np);
    f(i, j, e, pl < 0 ? 0.0f : base[pl * per_chunk], mult[e]);
  }
}

__global__ void k_hist(const float *D, int64_t n, int TR, int TC, int np, int64_t Q, int64_t nblk, int pass,
                       uint32_t hi, unsigned long long *hist) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x)
    for_each_entry(D, n, TR, TC, np, Q, b, [&](int64_t, int64_t, int, float v, int mult) {
      const uint32_t bits = abs_bits(v);
      if (bits == 0) return;
      if (pass == 0) atomicAdd(&hist[bits >> 16], (unsigned long long)mult);
      else if ((bits >> 16) == hi) atomicAdd(&hist[bits & 0xffffu], (unsigned long long)mult);
    });
}

// copies of the cut value t in row tile i (counted for the tie order)
__global__ void k_row_ties(const float *D, int64_t n, int TR, int TC, int np, int64_t Q, uint32_t tbits,
                           unsigned long long *ties) {
  const int64_t i = blockIdx.x;
  const int64_t p = i / TR;
  const int r = (int)(i - p * TR);
  unsigned long long local = 0;
  const int mult[6] = {1, 2, 2, 1, 2, 1};
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const int64_t q = j / TC;
    const int c = (int)(j - q * TC);
    const float *base = D + (p * Q + q) * np * (int64_t)TR * TC + (int64_t)r * TC + c;
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const int pl = stream_plane(e, np);
      if (pl >= 0) local += abs_bits(base[pl * (int64_t)TR * TC]) == tbits ? mult[e] : 0;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
  __shared__ unsigned long long sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    ties[i] = s;
  }
}

// a later kept column joins the run when it lies at most this far past the
// run's last kept column (the columns between are stored as zero blocks)
constexpr int kRunJoin = 4;

// Row tile i in increasing column order, one warp per row, 32 columns per
// step.  An entry is kept if |v| > t, or if |v| == t and the copies of t up
// to and including it (counted from tie_start[i], in column and entry order)
// exceed r.  The kept columns are grouped into runs (see the storage note);
// every lane walks the step's kept columns in order, so the run state is
// the same in all lanes.  FILL = false: the row's stored blocks (runs padded
// to 4) into cnt[i] and its runs into nrun[i]; FILL = true: each kept block
// at its slot and each run's (first block, first column) pair (the value
// planes were zeroed before).  With t = 0 every nonzero entry is kept.
template <bool FILL>
__global__ void k_rows(const float *D, int64_t n, int TR, int TC, int np, int64_t Q, uint32_t tbits,
                       const unsigned long long *tie_start, unsigned long long r, int *cnt, int *nrun,
                       const int64_t *ptr, const int64_t *rptr, int32_t *run, float *val) {
  const int64_t i = blockIdx.x;
  const int lane = threadIdx.x;
  const int64_t p = i / TR;
  const int rr = (int)(i - p * TR);
  const int mult[6] = {1, 2, 2, 1, 2, 1};
  const int64_t o = FILL ? ptr[i] : 0, K4 = FILL ? ptr[i + 1] - o : 0;
  float *rv = FILL ? val + np * o : nullptr;  // np value planes, as the source
  int32_t *rd = FILL ? run + 2 * rptr[i] : nullptr;
  unsigned long long carry = tie_start ? tie_start[i] : 0;
  // run state: stored blocks before the open run, its first and last column
  int64_t ofs = 0, col0 = -1, last = -1;
  int64_t runs = 0;
  for (int64_t j0 = 0; j0 < n; j0 += 32) {
    const int64_t j = j0 + lane;
    float v[6] = {0, 0, 0, 0, 0, 0};
    uint32_t bits[6] = {0, 0, 0, 0, 0, 0};
    unsigned tm = 0;  // copies of t in this lane's block
    if (j < n) {
      const int64_t q = j / TC;
      const int c = (int)(j - q * TC);
      const float *base = D + (p * Q + q) * np * (int64_t)TR * TC + (int64_t)rr * TC + c;
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int pl = stream_plane(e, np);
        v[e] = pl < 0 ? 0.0f : base[pl * (int64_t)TR * TC];
        bits[e] = abs_bits(v[e]);
        tm += (bits[e] != 0 && bits[e] == tbits) ? mult[e] : 0;
      }
    }
    // inclusive scan of tm over the lanes (columns in order)
    unsigned incl = tm;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    unsigned long long cum = carry + (incl - tm);
    bool keep = false;
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      bool k = bits[e] != 0 && bits[e] > tbits;
      if (bits[e] != 0 && bits[e] == tbits) {
        cum += mult[e];
        k = cum > r;
      }
      if (!k) v[e] = 0.0f;
      keep = keep || k;
    }
    carry += __shfl_sync(0xffffffffu, incl, 31);
    // runs: the kept columns of this step in order (the mask is the same in
    // every lane, so is the walk)
    unsigned mk = __ballot_sync(0xffffffffu, keep);
    int64_t slot = -1;
    while (mk) {
      const int l = __ffs(mk) - 1;
      mk &= mk - 1;
      const int64_t jk = j0 + l;
      if (col0 < 0 || jk - last > kRunJoin) {  // a new run
        if (col0 >= 0) ofs += (last - col0 + 4) & ~(int64_t)3;  // close the open one, padded to 4
        col0 = jk;
        if (FILL && lane == 0) {
          rd[2 * runs] = (int32_t)ofs;
          rd[2 * runs + 1] = (int32_t)jk;
        }
        ++runs;
      }
      if (l == lane) slot = ofs + (jk - col0);
      last = jk;
    }
    if (FILL && keep) {
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int pl = stream_plane(e, np);
        if (pl >= 0) rv[pl * K4 + slot] = v[e];
      }
    }
  }
  if (col0 >= 0) ofs += (last - col0 + 4) & ~(int64_t)3;
  if (!FILL && lane == 0) {
    cnt[i] = (int)ofs;
    nrun[i] = (int)runs;
  }
}

// s + t = u + err exactly (Knuth's two-sum); the error goes to c
__device__ __forceinline__ void sum2_add(float &s, float &c, float t) {
  const float u = s + t;
  const float bp = u - s;
  c += (s - (u - bp)) + (t - bp);
  s = u;
}

// the warp's (sum, error) pairs combined into lane 0's (s, c) (and every
// lane's: butterfly), errors carried
__device__ __forceinline__ void warp_sum2_pair(float &s, float &c) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float so = __shfl_xor_sync(0xffffffffu, s, off);
    const float co = __shfl_xor_sync(0xffffffffu, c, off);
    c += co;
    sum2_add(s, c, so);
  }
}


// A row's blocks are taken 128 at a time (a step: 4 consecutive blocks of one
// run per lane).  The product may give a row to S = 1, 2, 4 or 8 warps, warp
// k taking steps floor(k st / S) .. floor((k + 1) st / S) - 1 of the row's
// st steps; seg[8 i + k'] holds the run (from the row's first) that contains
// the first block of eighth k', so a warp starts its cursor there.
constexpr int kSpSegMax = 8;

__global__ void k_seg_runs(int64_t n, const int64_t *__restrict__ ptr, const int64_t *__restrict__ rptr,
                           const int2 *__restrict__ run, int32_t *seg) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * kSpSegMax) return;
  const int64_t i = t / kSpSegMax;
  const int k = (int)(t - i * kSpSegMax);
  const int64_t st = (ptr[i + 1] - ptr[i] + 127) / 128;
  const int64_t a = 128 * ((k * st) / kSpSegMax);
  int64_t lo = rptr[i], hi = rptr[i + 1] - 1;  // the last run starting at or before block a
  if (hi < lo) {
    seg[t] = 0;
    return;
  }
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (run[mid].x <= a) lo = mid;
    else hi = mid - 1;
  }
  seg[t] = (int32_t)(lo - rptr[i]);
}

// H_i = -sum_kept N_ij Ms_j m_j, rows of one simulation consecutive; xs =
// float4 (Ms m, 0) per tile, n + 4 per simulation.  S = 1: one warp per
// (row, simulation), two per CTA.  S > 1: one CTA per (row, simulation), its
// S warps on consecutive step ranges, their compensated sums added in warp
// order in shared memory.  Each lane takes 4 consecutive blocks of one run
// per step (NP vector loads of the values and 4 contiguous operands) and
// follows the row's runs with a cursor of its own.  (Lanes on interleaved
// blocks, for wider contiguous loads, needed a cursor walk per block and
// measured 2.4x slower.)
template <int NP, int S>
__global__ void __launch_bounds__(S == 1 ? 64 : 32 * S) k_spmv(int64_t n, int B, const int64_t *__restrict__ ptr,
                                                               const int64_t *__restrict__ rptr,
                                                               const int2 *__restrict__ run,
                                                               const int32_t *__restrict__ seg,
                                                               const float *__restrict__ val,
                                                               const float4 *__restrict__ xs, float *H,
                                                               const int *active) {
  mtd::pdl_enter();
  const int lane = threadIdx.x & 31;
  int64_t rid;  // b n + i
  int k;        // this warp's part of the row
  if constexpr (S == 1) {
    rid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    k = 0;
    if (rid >= n * B) return;
  } else {
    rid = blockIdx.x;
    k = threadIdx.x >> 5;
  }
  const int64_t i = rid % n;
  const int b = (int)(rid / n);
  if (active && !active[b]) return;  // the whole CTA when S > 1
  const float4 *xb = xs + (size_t)b * sparse_x_stride(n);
  const int64_t o = ptr[i], K4 = ptr[i + 1] - o;
  const int64_t st = (K4 + 127) / 128;
  const int64_t a_lo = 128 * ((k * st) / S);
  const int64_t a_e = 128 * (((k + 1) * st) / S), a_hi = a_e < K4 ? a_e : K4;
  const float *rv = val + NP * o;
  const int64_t r1 = rptr[i + 1];
  int64_t rc = rptr[i] + (S == 1 ? 0 : seg[i * kSpSegMax + k * (kSpSegMax / S)]);  // this lane's run
  int2 cur = rc < r1 ? run[rc] : make_int2(0, 0);
  int64_t next = rc + 1 < r1 ? run[rc + 1].x : INT64_MAX;  // first block of the following run
  float sx = 0, cx = 0, sy = 0, cy = 0, sz = 0, cz = 0;
  for (int64_t a = a_lo + 4 * (int64_t)lane; a < a_hi; a += 128) {
    // the values stream past (read once: no L1 allocation); the operands,
    // read by every row, stay cached
    float4 v[NP];
#pragma unroll
    for (int e = 0; e < NP; ++e) v[e] = __ldcs(reinterpret_cast<const float4 *>(rv + e * K4 + a));
    while (a >= next) {
      ++rc;
      cur = run[rc];
      next = rc + 1 < r1 ? run[rc + 1].x : INT64_MAX;
    }
    const int64_t c = cur.y + (a - cur.x);  // column of block a
    float4 x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = xb[c + q];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if constexpr (NP == 6) {
        // per block: (v0 v1 v2; v1 v3 v4; v2 v4 v5) (x, y, z)
        const float n0 = f4_at(v[0], q), n1 = f4_at(v[1], q), n2 = f4_at(v[2], q);
        const float n3 = f4_at(v[3], q), n4 = f4_at(v[4], q), n5 = f4_at(v[5], q);
        sum2_add(sx, cx, fmaf(n0, x[q].x, fmaf(n1, x[q].y, n2 * x[q].z)));
        sum2_add(sy, cy, fmaf(n1, x[q].x, fmaf(n3, x[q].y, n4 * x[q].z)));
        sum2_add(sz, cz, fmaf(n2, x[q].x, fmaf(n4, x[q].y, n5 * x[q].z)));
      } else {
        // single-layer tensor: (v0 v1 0; v1 v2 0; 0 0 v3) (x, y, z)
        const float n0 = f4_at(v[0], q), n1 = f4_at(v[1], q);
        const float n3 = f4_at(v[2], q), n5 = f4_at(v[3], q);
        sum2_add(sx, cx, fmaf(n0, x[q].x, n1 * x[q].y));
        sum2_add(sy, cy, fmaf(n1, x[q].x, n3 * x[q].y));
        sum2_add(sz, cz, __fmul_rn(n5, x[q].z));  // a rounded product, as in the 6-plane form
      }
    }
  }
  warp_sum2_pair(sx, cx);
  warp_sum2_pair(sy, cy);
  warp_sum2_pair(sz, cz);
  float *Hb = H + (size_t)b * 3 * n + 3 * i;
  if constexpr (S == 1) {
    if (lane == 0) {
      Hb[0] = -(sx + cx);
      Hb[1] = -(sy + cy);
      Hb[2] = -(sz + cz);
    }
  } else {
    __shared__ float part[S][6];
    if (lane == 0) {
      part[k][0] = sx;
      part[k][1] = cx;
      part[k][2] = sy;
      part[k][3] = cy;
      part[k][4] = sz;
      part[k][5] = cz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < S; ++w) {
        cx += part[w][1];
        sum2_add(sx, cx, part[w][0]);
        cy += part[w][3];
        sum2_add(sy, cy, part[w][2]);
        cz += part[w][5];
        sum2_add(sz, cz, part[w][4]);
      }
      Hb[0] = -(sx + cx);
      Hb[1] = -(sy + cy);
      Hb[2] = -(sz + cz);
    }
  }
}

// xs[b][j] = (Ms_j m_j, 0) (the 4 padding entries per simulation stay zero)
__global__ void k_prep_sparse_x(const float *m, const float *Ms, int64_t n, int B, float4 *xs) {
  const int64_t tot = (int64_t)B * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / n, j = t - b * n;
    const float ms = Ms[j];
    const float *mj = m + 3 * t;
    xs[b * sparse_x_stride(n) + j] = make_float4(ms * mj[0], ms * mj[1], ms * mj[2], 0.0f);
  }
}

// Warps per row of the sparse product, a property of the tensor (so that a
// simulation's field does not depend on the batch it runs in): doubled while
// one simulation's rows give fewer than 4 waves of resident warps (32 per SM)
// and every warp keeps at least 6 steps of 128 blocks.  With one warp per row
// the last, partial wave runs a whole row's chain of dependent steps on
// mostly idle SMs.
int sparse_split(int64_t n, int64_t nnzb, int sms) {
  const double steps = n > 0 ? (double)nnzb / (double)n / 128.0 : 0.0;
  const int64_t resident = (int64_t)std::max(1, sms) * 32;
  int S = 1;
  while (S < kSpSegMax && n * S < 4 * resident && steps / (2 * S) >= 6.0) S *= 2;
  return S;
}

// position of rank k in a 65536-bin histogram: bin and rank within it
void select_bin(const std::vector<unsigned long long> &h, unsigned long long k, uint32_t *bin,
                unsigned long long *rest) {
  unsigned long long cum = 0;
  for (uint32_t b = 0; b < h.size(); ++b) {
    if (cum + h[b] > k) {
      *bin = b;
      *rest = k - cum;
      return;
    }
    cum += h[b];
  }
  *bin = (uint32_t)h.size() - 1;
  *rest = 0;
}

}  // namespace

namespace mt {

void launch_spmv(const mt_tensor *T, const float *xs, int B, float *H, const int *active, cudaStream_t s) {
  const int64_t rows = T->n * (int64_t)B;
  const int64_t *ptr = (const int64_t *)T->d_sp_ptr;
  const int64_t *rptr = (const int64_t *)T->d_sp_rptr;
  const int2 *run = reinterpret_cast<const int2 *>(T->d_sp_col);
  const int32_t *seg = T->d_sp_seg;
  const float *val = (const float *)T->d_sp_val;
  const float4 *x4 = reinterpret_cast<const float4 *>(xs);
  const int S = T->sp_split;
  const dim3 grid((unsigned)(S == 1 ? (rows + 1) / 2 : rows)), block(S == 1 ? 64 : 32 * S);
#define MT_SPMV(NP, SS) \
  mt::launch_pdl(k_spmv<NP, SS>, grid, block, 0, s, T->n, B, ptr, rptr, run, seg, val, x4, H, active)
  if (T->L.nplane == 4) {
    if (S == 8) MT_SPMV(4, 8);
    else if (S == 4) MT_SPMV(4, 4);
    else if (S == 2) MT_SPMV(4, 2);
    else MT_SPMV(4, 1);
  } else {
    if (S == 8) MT_SPMV(6, 8);
    else if (S == 4) MT_SPMV(6, 4);
    else if (S == 2) MT_SPMV(6, 2);
    else MT_SPMV(6, 1);
  }
#undef MT_SPMV
}

void launch_prep_sparse_x(const mt_tensor *T, const float *m, int B, float *xs, cudaStream_t s) {
  const int64_t tot = (int64_t)B * T->n;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 4096);
  k_prep_sparse_x<<<blocks, 256, 0, s>>>(m, T->tiles->d_Ms, T->n, B, reinterpret_cast<float4 *>(xs));
}

}  // namespace mt

extern "C" mt_status mt_tensor_threshold(mt_tensor *T, double fraction, mt_tensor **out, double *threshold,
                                         int64_t *kept_elements) {
  MT_CHECK(T && out, MT_EINVAL, "mt_tensor_threshold: NULL argument");
  MT_CHECK(T->prec == MT_F32 && T->layout == MT_LAYOUT_STREAM, MT_EINVAL,
           "mt_tensor_threshold: needs an FP32 tensor of the streaming layout");
  MT_CHECK(fraction >= 0.0 && fraction < 1.0, MT_EINVAL, "mt_tensor_threshold: fraction in [0, 1)");
  MT_CHECK(!T->L.half, MT_EINVAL,
           "mt_tensor_threshold: needs every block stored; assemble with MT_LAYOUT_STREAM_FULL");
  MT_CUDA(cudaSetDevice(T->tiles->ctx->device));
  const int64_t n = T->n;
  const mt_layout &L = T->L;
  const float *D = reinterpret_cast<const float *>(T->d_data);
  const int64_t nblk = L.P * L.Q * (int64_t)L.TR * L.TC;
  DevTemp<unsigned long long> hist;
  MT_CUDA(hist.alloc(65536));
  unsigned long long *d_hist = hist.p;
  std::vector<unsigned long long> h(65536);
  const int grid = 4 * T->tiles->ctx->num_sms;
  // pass 1: top 16 bits
  MT_CUDA(cudaMemset(d_hist, 0, sizeof(unsigned long long) * 65536));
  k_hist<<<grid, 256>>>(D, n, L.TR, L.TC, L.nplane, L.Q, nblk, 0, 0, d_hist);
  MT_CUDA(cudaGetLastError());
  MT_CUDA(cudaMemcpy(h.data(), d_hist, sizeof(unsigned long long) * 65536, cudaMemcpyDeviceToHost));
  unsigned long long nz = 0;
  for (auto x : h) nz += x;
  const unsigned long long k = (unsigned long long)(fraction * (double)nz);
  uint32_t tbits = 0;
  unsigned long long r = 0;  // copies of t to drop (the first r in tie order)
  if (k > 0 && nz > 0) {
    uint32_t b1 = 0;
    unsigned long long rest = 0;
    select_bin(h, k, &b1, &rest);
    // pass 2: low 16 bits inside bin b1
    MT_CUDA(cudaMemset(d_hist, 0, sizeof(unsigned long long) * 65536));
    k_hist<<<grid, 256>>>(D, n, L.TR, L.TC, L.nplane, L.Q, nblk, 1, b1, d_hist);
    MT_CUDA(cudaGetLastError());
    MT_CUDA(cudaMemcpy(h.data(), d_hist, sizeof(unsigned long long) * 65536, cudaMemcpyDeviceToHost));
    uint32_t b2 = 0;
    unsigned long long rest2 = 0;
    select_bin(h, rest, &b2, &rest2);
    tbits = (b1 << 16) | b2;
    r = rest2;
  }
  // tie order: copies of t before each row tile
  DevTemp<unsigned long long> tie_start;
  unsigned long long *d_tie = nullptr;
  if (r > 0) {
    MT_CUDA(tie_start.alloc(n));
    d_tie = tie_start.p;
    k_row_ties<<<(unsigned)n, 256>>>(D, n, L.TR, L.TC, L.nplane, L.Q, tbits, d_tie);
    MT_CUDA(cudaGetLastError());
    std::vector<unsigned long long> ties(n);
    MT_CUDA(cudaMemcpy(ties.data(), d_tie, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost));
    unsigned long long acc = 0;
    for (int64_t i = 0; i < n; ++i) {
      const unsigned long long c = ties[i];
      ties[i] = acc;
      acc += c;
    }
    MT_CUDA(cudaMemcpy(d_tie, ties.data(), sizeof(unsigned long long) * n, cudaMemcpyHostToDevice));
  }
  // stored blocks and runs per row
  DevTemp<int> cnt_rows, run_rows;
  MT_CUDA(cnt_rows.alloc(n));
  MT_CUDA(run_rows.alloc(n));
  int *d_cnt = cnt_rows.p, *d_nrun = run_rows.p;
  k_rows<false><<<(unsigned)n, 32>>>(D, n, L.TR, L.TC, L.nplane, L.Q, tbits, d_tie, r, d_cnt, d_nrun, nullptr,
                                     nullptr, nullptr, nullptr);
  MT_CUDA(cudaGetLastError());
  std::vector<int> cnt(n), nrun(n);
  MT_CUDA(cudaMemcpy(cnt.data(), d_cnt, sizeof(int) * n, cudaMemcpyDeviceToHost));
  MT_CUDA(cudaMemcpy(nrun.data(), d_nrun, sizeof(int) * n, cudaMemcpyDeviceToHost));
  std::vector<int64_t> ptr(n + 1, 0), rptr(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    ptr[i + 1] = ptr[i] + cnt[i];  // runs are padded to 4 blocks already
    rptr[i + 1] = rptr[i] + nrun[i];
  }
  const int64_t nnzb = ptr[n], nruns = rptr[n];
  mt_ctx *ctx = T->tiles->ctx;
  mt_tensor *S = new mt_tensor();
  S->tiles = T->tiles;
  T->tiles->refs++;
  S->prec = MT_F32;
  S->layout = MT_LAYOUT_SPARSE;
  S->n = n;
  S->L = T->L;
  S->sp_blocks = nnzb;
  S->sp_runs = nruns;
  S->sp_split = sparse_split(n, nnzb, ctx->num_sms);
  const int np = T->L.nplane;  // value planes: those the source stores (6, or 4 for a single layer)
  S->bytes = 2 * sizeof(int64_t) * (n + 1) + 2 * sizeof(int32_t) * (size_t)std::max<int64_t>(1, nruns) +
             np * sizeof(float) * (size_t)std::max<int64_t>(1, nnzb) + sizeof(int32_t) * kSpSegMax * (size_t)n;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->in_use + S->bytes > ctx->budget) {
      const size_t need = S->bytes;
      delete S;
      mt::tiles_release(T->tiles);
      mt::set_error("mt_tensor_threshold: %zu bytes exceed the context budget", need);
      return MT_ENOMEM;
    }
    ctx->in_use += S->bytes;
  }
  cudaError_t e = cudaMalloc(&S->d_sp_ptr, sizeof(int64_t) * (n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_sp_rptr, sizeof(int64_t) * (n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_sp_col, 2 * sizeof(int32_t) * std::max<int64_t>(1, nruns));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_sp_val, np * sizeof(float) * std::max<int64_t>(1, nnzb));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_sp_seg, sizeof(int32_t) * kSpSegMax * (size_t)n);
  if (e == cudaSuccess) e = cudaMemcpy(S->d_sp_ptr, ptr.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(S->d_sp_rptr, rptr.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice);
  // gap and padding blocks are zero
  if (e == cudaSuccess) e = cudaMemset(S->d_sp_val, 0, np * sizeof(float) * std::max<int64_t>(1, nnzb));
  if (e != cudaSuccess) {
    mt::tensor_release(S);
    return mt::cuda_fail(e, "mt_tensor_threshold allocation", __FILE__, __LINE__);
  }
  k_rows<true><<<(unsigned)n, 32>>>(D, n, L.TR, L.TC, L.nplane, L.Q, tbits, d_tie, r, nullptr, nullptr,
                                    S->d_sp_ptr, S->d_sp_rptr, S->d_sp_col, S->d_sp_val);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    k_seg_runs<<<(unsigned)((n * kSpSegMax + 255) / 256), 256>>>(
        n, S->d_sp_ptr, S->d_sp_rptr, reinterpret_cast<const int2 *>(S->d_sp_col), S->d_sp_seg);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    mt::tensor_release(S);
    return mt::cuda_fail(e, "mt_tensor_threshold fill", __FILE__, __LINE__);
  }
  if (threshold) {
    float tf;
    std::memcpy(&tf, &tbits, sizeof(tf));
    *threshold = (double)tf;
  }
  if (kept_elements) {
    // kept elements of the full matrix (off-diagonal entries count twice)
    std::vector<float> vals(np * (size_t)std::max<int64_t>(1, nnzb));
    MT_CUDA(cudaMemcpy(vals.data(), S->d_sp_val, np * sizeof(float) * nnzb, cudaMemcpyDeviceToHost));
    int64_t kept = 0;
    const int mult[6] = {1, 2, 2, 1, 2, 1};
    for (int64_t i = 0; i < n; ++i) {
      const int64_t o = ptr[i], K4 = ptr[i + 1] - o;
      for (int e = 0; e < 6; ++e)
        for (int64_t a = 0; a < K4; ++a) {
          const int pl = stream_plane(e, np);
          kept += (pl >= 0 && vals[np * o + pl * K4 + a] != 0.0f) ? mult[e] : 0;
        }
    }
    *kept_elements = kept;
  }
  *out = S;
  return MT_OK;
}

namespace mt {

// rows [i0, i1) of a thresholded tensor as dense FP64 blocks
mt_status read_rows_sparse(const mt_tensor *T, int64_t i0, int64_t i1, double *out) {
  const int64_t n = T->n;
  std::vector<int64_t> ptr(i1 - i0 + 1), rptr(i1 - i0 + 1);
  MT_CUDA(cudaMemcpy(ptr.data(), T->d_sp_ptr + i0, sizeof(int64_t) * (i1 - i0 + 1), cudaMemcpyDeviceToHost));
  MT_CUDA(cudaMemcpy(rptr.data(), T->d_sp_rptr + i0, sizeof(int64_t) * (i1 - i0 + 1), cudaMemcpyDeviceToHost));
  const int64_t a0 = ptr[0], a1 = ptr[i1 - i0], q0 = rptr[0], q1 = rptr[i1 - i0];
  std::vector<int32_t> run(2 * std::max<int64_t>(1, q1 - q0));
  const int np = T->L.nplane;
  std::vector<float> val(np * std::max<int64_t>(1, a1 - a0));
  if (a1 > a0) {
    MT_CUDA(cudaMemcpy(run.data(), T->d_sp_col + 2 * q0, 2 * sizeof(int32_t) * (q1 - q0), cudaMemcpyDeviceToHost));
    MT_CUDA(cudaMemcpy(val.data(), T->d_sp_val + np * a0, np * sizeof(float) * (a1 - a0), cudaMemcpyDeviceToHost));
  }
  std::memset(out, 0, sizeof(double) * 6 * (size_t)(i1 - i0) * n);
  for (int64_t i = i0; i < i1; ++i) {
    const int64_t o = ptr[i - i0], K4 = ptr[i - i0 + 1] - o;
    const float *rv = val.data() + np * (o - a0);
    const int64_t rb = rptr[i - i0] - q0, re = rptr[i - i0 + 1] - q0;
    for (int64_t q = rb; q < re; ++q) {
      const int64_t b0 = run[2 * q], c0 = run[2 * q + 1];
      const int64_t b1 = q + 1 < re ? run[2 * (q + 1)] : K4;
      for (int64_t a = b0; a < b1; ++a) {
        const int64_t j = c0 + (a - b0);
        if (j >= n) break;  // padding past the last tile (zero)
        for (int e = 0; e < 6; ++e) {
          const int pl = stream_plane(e, np);
          if (pl >= 0) out[((i - i0) * n + j) * 6 + e] += rv[pl * K4 + a];
        }
      }
    }
  }
  return MT_OK;
}

}  // namespace mt
