// Effective field, Landau-Lifshitz right-hand side and the Runge-Kutta (4,5)
// integrator (Sec. 2, Sec. 3.1 of the paper).
//
// One Dormand-Prince step of B simulations is a fixed sequence of kernels,
// captured once in a CUDA graph:
//   begin      commit the previous step if it was accepted (m <- |m_new|^-1
//              m_new, k1 <- k7), form the stage-2 input;
//   6 x [ streaming demag product ; stage kernel ]
//              a stage kernel adds exchange (Eq. 12), anisotropy (Eq. 16)
//              and applied field (Eq. 7) to H_d, evaluates Eq. 1 and forms
//              the next stage's input; the last one also reduces the
//              embedded error, the torque and the mean magnetisation, and its
//              last block decides accept/reject and the next step size on
//              the device.
// The host only replays the graph and polls a counter of unfinished
// simulations every few steps.
#include <algorithm>
#include <limits>
#include <cmath>
#include <cstring>
#include <vector>

#include "mt_internal.cuh"

namespace {

// Dormand & Prince (1980) RK5(4)7M: stage couplings, 5th-order weights
// (= last coupling row, first same as last) and the difference between the
// 5th- and the embedded 4th-order weights, which estimates the local error.
__constant__ double c_dp_a[7][7] = {
    {0, 0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0}};
__constant__ double c_dp_err[7] = {35.0 / 384 - 5179.0 / 57600,
                                   0.0,
                                   500.0 / 1113 - 7571.0 / 16695,
                                   125.0 / 192 - 393.0 / 640,
                                   -2187.0 / 6784 + 92097.0 / 339200,
                                   11.0 / 84 - 187.0 / 2100,
                                   -1.0 / 40};

// ---------------------------------------------------------------------------
// per-simulation control block (device memory)
// ---------------------------------------------------------------------------
struct SimCtl {
  double t, h, hs, t_next, t_out0, dt_out, t1, tol;
  double tau, err;
  double m_last[3];  // volume-averaged m of the last accepted (or starting) state
  int64_t iout, n_out;
  int64_t n_accept, n_reject, n_rhs, n_attempt, attempt_cap;
  int mode;      // 0 = fixed number of steps, 1 = integrate to t1, 2 = relax
  int accepted;  // last attempt accepted: begin/commit must adopt it
  int clipped;   // the current attempt ends exactly on t_next
  int status;
  int done;
  int fresh;  // admitted since the last k1 evaluation (serving slots)
};

enum { MODE_STEPS = 0, MODE_RUN = 1, MODE_RELAX = 2 };

struct StageArgs {
  int64_t n;
  int B;
  // geometry / material
  const int32_t *nbr;
  const float *wex, *kan, *axis, *Ms;
  const double *wvol;
  bool exch;
  // per-simulation equation parameters
  const float *g1, *g2, *Ha;
  const float *xsc;  // [B] factor on the exchange stiffness (nullptr: 1)
  // state
  float *y, *ys0, *ys1, *Hd, *xs;
  float *k[7];
  int64_t Q;
  int TC;
  // operand of the batched tensor-core product (dense layout): X[b][Kp] BF16
  // (+ low part for the split precision); xs_mode 0 = streaming layout
  int xs_mode;  // 0 streaming FP32 chunks, 1 dense BF16, 2 dense split BF16, 3 sparse float4
  int64_t Kp;
  int Bp;
  __nv_bfloat16 *X;
  float *mT;  // simulation-fastest copy of the stage input (near blocks)
  // control
  SimCtl *ctl;
  int *active;
  int *n_active;
  float *red;      // [B][nblk][5]
  int *red_count;  // [B]
  double *mavg;    // [n_out][B][3]
  double rtol, atol, hmax, fixed_h;
  int fresh_only;  // stage 1: evaluate k1 only for freshly admitted simulations
};

constexpr int kStageThreads = 256;

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Effective field of tile i (Eq. 5/17): H_d (from the demag product) + exchange
// (finite volumes, Eq. 12; absent neighbour = Neumann, Eq. 3) + uniaxial
// anisotropy (Eq. 16) + applied field (Eq. 7).
// H holds H_d on entry.  ha, xs: the simulation's applied field and exchange
// factor; nbr6, wex6: the tile's six face neighbours (-1: none) and their
// weights; ka, e: its anisotropy prefactor and axis; yb: the simulation's
// state of all tiles (the neighbours' m).
__device__ __forceinline__ void local_fields(const float *ha, float xs, bool exch, const int32_t *nbr6,
                                             const float *wex6, float ka, const float *e, const float *yb,
                                             const float mi[3], float H[3]) {
  H[0] = H[0] + ha[0];
  H[1] = H[1] + ha[1];
  H[2] = H[2] + ha[2];
  if (exch) {
    float he[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int32_t p = nbr6[f];
      if (p >= 0) {
        const float w = wex6[f];
        he[0] += w * (yb[3 * p] - mi[0]);
        he[1] += w * (yb[3 * p + 1] - mi[1]);
        he[2] += w * (yb[3 * p + 2] - mi[2]);
      }
    }
    H[0] += xs * he[0];
    H[1] += xs * he[1];
    H[2] += xs * he[2];
  }
  if (ka != 0.0f) {
    const float me = mi[0] * e[0] + mi[1] * e[1] + mi[2] * e[2];
    H[0] += ka * me * e[0];
    H[1] += ka * me * e[1];
    H[2] += ka * me * e[2];
  }
}

__device__ __forceinline__ void add_local_fields(const StageArgs &A, const float *yb, int64_t i, int b,
                                                 const float mi[3], float H[3]) {
  local_fields(A.Ha + 3 * b, A.xsc ? A.xsc[b] : 1.0f, A.exch, A.nbr + 6 * i, A.wex + 6 * i, A.kan[i],
               A.axis + 3 * i, yb, mi, H);
}

__device__ __forceinline__ void effective_field(const StageArgs &A, const float *yin, const float *Hd, int64_t i,
                                                int b, const float mi[3], float H[3]) {
  const float *hd = Hd + (size_t)b * 3 * A.n + 3 * i;
  H[0] = hd[0];
  H[1] = hd[1];
  H[2] = hd[2];
  add_local_fields(A, yin + (size_t)b * 3 * A.n, i, b, mi, H);
}

// Eq. 1 with prefactors g1 (precession) and g2 (damping):
// dm/dt = -g1 m x H - g2 m x (m x H); returns |m x H|.
__device__ __forceinline__ float llg(float g1, float g2, const float m[3], const float H[3], float k[3]) {
  float a[3], c[3];
  cross3(m, H, a);
  cross3(m, a, c);
  k[0] = -g1 * a[0] - g2 * c[0];
  k[1] = -g1 * a[1] - g2 * c[1];
  k[2] = -g1 * a[2] - g2 * c[2];
  return sqrtf(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
}

__device__ __forceinline__ void write_stage_input(const StageArgs &A, float *ysn, int64_t i, int b,
                                                  const float v[3]) {
  float *d = ysn + (size_t)b * 3 * A.n + 3 * i;
  d[0] = v[0];
  d[1] = v[1];
  d[2] = v[2];
  const float ms = A.Ms[i];
  if (A.xs_mode == 0) {
    const int64_t q = i / A.TC, t = i - q * A.TC;
    float *x = A.xs + ((size_t)(b * A.Q + q) * 3) * A.TC + t;
    x[0] = ms * v[0];
    x[A.TC] = ms * v[1];
    x[2 * A.TC] = ms * v[2];
  } else if (A.xs_mode == 3) {
    reinterpret_cast<float4 *>(A.xs)[(size_t)b * sparse_x_stride(A.n) + i] =
        make_float4(ms * v[0], ms * v[1], ms * v[2], 0.0f);
  } else {
    __nv_bfloat16 *x1 = A.X + (size_t)A.Bp * A.Kp;  // split: second and third operand terms
    __nv_bfloat16 *x2 = x1 + (size_t)A.Bp * A.Kp;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float f = ms * v[c];
      const __nv_bfloat16 hi = __float2bfloat16(f);
      const size_t at = dense_x_index(b, 3 * i + c, A.Bp);
      A.X[at] = hi;
      if (A.xs_mode == 2) {
        const float r = f - __bfloat162float(hi);
        const __nv_bfloat16 mid = __float2bfloat16(r);
        x1[at] = mid;
        x2[at] = __float2bfloat16(r - __bfloat162float(mid));
      }
      A.mT[(size_t)(3 * i + c) * A.Bp + b] = v[c];
    }
  }
}

// Block-reduce NV floats (sum for all but index `max_idx`, which is a
// NaN-propagating max) and return them in thread 0.
template <int NV>
__device__ __forceinline__ void block_reduce(float v[NV], int max_idx) {
  __shared__ float sh[kStageThreads / 32][NV];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = (q == max_idx) ? mtd::warp_max(v[q]) : mtd::warp_sum(v[q]);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[w][q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < NV; ++q) {
      float acc = sh[0][q];
      for (int ww = 1; ww < (int)(blockDim.x >> 5); ++ww)
        acc = (q == max_idx) ? mtd::nan_max(acc, sh[ww][q]) : acc + sh[ww][q];
      v[q] = acc;
    }
  }
  __syncthreads();
}

// Deterministic per-simulation reduction across blocks: every block writes
// its 5 values, the last block to arrive sums them in block order.  Returns
// true in thread 0 of the last block (with tot filled).  FP32 throughout:
// the sums (squared scaled errors, volume-weighted m) need no more, and FP64
// arithmetic on the one latency-critical thread is slow on this part.
__device__ bool reduce_across_blocks(const StageArgs &A, int b, float v[5], double tot[5]) {
  const int nblk = gridDim.x;
  __shared__ int s_last;
  block_reduce<5>(v, 1);
  if (threadIdx.x == 0) {
    float *dst = A.red + ((size_t)b * nblk + blockIdx.x) * 5;
    for (int q = 0; q < 5; ++q) dst[q] = v[q];
    __threadfence();
    const int old = atomicAdd(&A.red_count[b], 1);
    s_last = (old == nblk - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  float acc[5] = {0, 0, 0, 0, 0};
  for (int blk = threadIdx.x; blk < nblk; blk += blockDim.x) {
    const float *src = A.red + ((size_t)b * nblk + blk) * 5;
    acc[0] += __ldcg(&src[0]);
    acc[1] = mtd::nan_max(acc[1], __ldcg(&src[1]));
    acc[2] += __ldcg(&src[2]);
    acc[3] += __ldcg(&src[3]);
    acc[4] += __ldcg(&src[4]);
  }
  block_reduce<5>(acc, 1);
  if (threadIdx.x == 0) {
    A.red_count[b] = 0;
    for (int q = 0; q < 5; ++q) tot[q] = (double)acc[q];
  }
  return threadIdx.x == 0;
}

__device__ __forceinline__ void finish_sim(SimCtl &c, int status) {
  c.done = 1;
  c.status = status;
}

// Step size for the next attempt: the proposal h capped by hmax, shortened to
// land on the next output (or end) time.
__device__ __forceinline__ void plan_attempt(const StageArgs &A, SimCtl &c) {
  double hs = c.h;
  if (A.fixed_h <= 0.0 && A.hmax > 0.0 && hs > A.hmax) hs = A.hmax;
  c.clipped = 0;
  if (c.t + hs >= c.t_next) {
    hs = c.t_next - c.t;
    c.clipped = 1;
  }
  c.hs = hs;
}

// After the first derivative of a run: its torque, and a relaxation that is
// already below tolerance ends here.
__device__ __forceinline__ void close_first(SimCtl &c, double tau) {
  c.tau = tau;
  c.n_rhs += 1;
  c.fresh = 0;
  if (!isfinite(c.tau)) finish_sim(c, MT_ENONFINITE);
  else if (c.mode == MODE_RELAX && c.tau < c.tol) finish_sim(c, MT_OK);
}

// Step control after an attempt, from the simulation's reduced sums tot =
// (sum of squared scaled errors, max torque, volume-weighted <m>): accept or
// reject, advance the time, record an output (*out_row = its index, else
// -1), finish on the end time, on the torque tolerance or on the attempt
// cap, choose the next step size and plan the next attempt.
__device__ __forceinline__ void close_attempt(const StageArgs &A, SimCtl &c, const double tot[5], int64_t *out_row) {
  *out_row = -1;
  const bool fixed = A.fixed_h > 0.0;
  // the RMS of the scaled errors; its sum is an FP32 sum on both paths
  const double err = (double)sqrtf((float)tot[0] / (3.0f * (float)A.n));
  const double tau = tot[1];
  c.err = err;
  c.n_attempt += 1;
  c.n_rhs += 6;
  const bool finite = isfinite(err) && isfinite(tot[2]) && isfinite(tot[3]) && isfinite(tot[4]);
  const bool accept = finite && (fixed || err <= 1.0);
  if (!finite) {
    c.accepted = 0;
    finish_sim(c, MT_ENONFINITE);
    return;
  }
  if (accept) {
    c.n_accept += 1;
    c.t = c.clipped ? c.t_next : c.t + c.hs;
    c.tau = tau;
    c.m_last[0] = tot[2];
    c.m_last[1] = tot[3];
    c.m_last[2] = tot[4];
    if (c.mode == MODE_RUN && c.clipped) {
      *out_row = c.iout;
      c.iout += 1;
      if (c.iout >= c.n_out) {
        finish_sim(c, MT_OK);
      } else {
        c.t_next = (c.iout + 1 == c.n_out) ? c.t1 : c.t_out0 + (double)(c.iout + 1) * c.dt_out;
      }
    } else if (c.mode == MODE_RELAX) {
      if (tau < c.tol) finish_sim(c, MT_OK);
      else if (c.clipped) finish_sim(c, MT_ENOCONV);
    }
  } else {
    c.n_reject += 1;
  }
  c.accepted = accept ? 1 : 0;
  if (fixed) {
    c.h = A.fixed_h;
  } else {
    // 0.9 err^(-1/5) clamped to [0.2, 5], in FP32 (a relative 1e-7 on the
    // proposal is immaterial; FP64 transcendentals are slow on this part)
    const float ef = (float)err;
    double fac = ef > 0.0f ? (double)(0.9f * exp2f(-0.2f * log2f(ef))) : 5.0;
    fac = fmin(5.0, fmax(0.2, fac));
    c.h = c.hs * fac;
    if (A.hmax > 0.0 && c.h > A.hmax) c.h = A.hmax;
  }
  if (!c.done && c.mode != MODE_STEPS && c.n_attempt >= c.attempt_cap) finish_sim(c, MT_ENOCONV);
  plan_attempt(A, c);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__global__ void k_begin(StageArgs A) {
  mtd::pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= A.n) return;
  const SimCtl &c = A.ctl[b];
  const size_t o = (size_t)b * 3 * A.n + 3 * i;
  float m[3], k1[3];
  if (c.accepted) {
    const float *yn = A.ys1 + o;  // 5th-order solution of the previous attempt
    const float inv = rsqrtf(yn[0] * yn[0] + yn[1] * yn[1] + yn[2] * yn[2]);
    m[0] = yn[0] * inv;
    m[1] = yn[1] * inv;
    m[2] = yn[2] * inv;
    const float *k7 = A.k[6] + o;
    k1[0] = k7[0];
    k1[1] = k7[1];
    k1[2] = k7[2];
    A.y[o] = m[0];
    A.y[o + 1] = m[1];
    A.y[o + 2] = m[2];
    A.k[0][o] = k1[0];
    A.k[0][o + 1] = k1[1];
    A.k[0][o + 2] = k1[2];
  } else {
    m[0] = A.y[o];
    m[1] = A.y[o + 1];
    m[2] = A.y[o + 2];
    k1[0] = A.k[0][o];
    k1[1] = A.k[0][o + 1];
    k1[2] = A.k[0][o + 2];
  }
  if (!A.active[b]) return;
  const float h = (float)(c.hs * c_dp_a[1][0]);
  const float v[3] = {m[0] + h * k1[0], m[1] + h * k1[1], m[2] + h * k1[2]};
  write_stage_input(A, A.ys0, i, b, v);
}

// commit only (after the last replay)
__global__ void k_commit(StageArgs A) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= A.n || !A.ctl[b].accepted) return;
  const size_t o = (size_t)b * 3 * A.n + 3 * i;
  const float *yn = A.ys1 + o;
  const float inv = rsqrtf(yn[0] * yn[0] + yn[1] * yn[1] + yn[2] * yn[2]);
  A.y[o] = yn[0] * inv;
  A.y[o + 1] = yn[1] * inv;
  A.y[o + 2] = yn[2] * inv;
  A.k[0][o] = A.k[6][o];
  A.k[0][o + 1] = A.k[6][o + 1];
  A.k[0][o + 2] = A.k[6][o + 2];
}

// Stage S (1..7).  S == 1 evaluates k1 at the state (start of a run);
// S in 2..6 also forms the input of stage S+1; S == 7 closes the attempt.
template <int S>
__global__ void __launch_bounds__(kStageThreads) k_stage(StageArgs A) {
  mtd::pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (!A.active[b]) return;  // uniform per block
  if (S == 1 && A.fresh_only && !A.ctl[b].fresh) return;
  const bool live = i < A.n;
  const float *yin = (S == 1) ? A.y : ((S & 1) ? A.ys1 : A.ys0);
  const size_t o = (size_t)b * 3 * A.n + 3 * i;
  float tau_i = 0.0f;
  float mi[3] = {0, 0, 0}, kk[3] = {0, 0, 0};
  if (live) {
    mi[0] = yin[o];
    mi[1] = yin[o + 1];
    mi[2] = yin[o + 2];
    float H[3];
    effective_field(A, yin, A.Hd, i, b, mi, H);
    tau_i = llg(A.g1[b], A.g2[b], mi, H, kk) / A.Ms[i];
    float *ko = A.k[S - 1] + o;
    ko[0] = kk[0];
    ko[1] = kk[1];
    ko[2] = kk[2];
  }
  if constexpr (S >= 2 && S <= 6) {
    if (live) {
      const double hs = A.ctl[b].hs;
      float acc[3] = {0, 0, 0};
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const float a = (float)(hs * c_dp_a[S][j]);
        if (a != 0.0f) {
          const float *kj = (j == S - 1) ? kk : A.k[j] + o;
          acc[0] += a * kj[0];
          acc[1] += a * kj[1];
          acc[2] += a * kj[2];
        }
      }
      const float *y0 = A.y + o;
      const float v[3] = {y0[0] + acc[0], y0[1] + acc[1], y0[2] + acc[2]};
      write_stage_input(A, (S + 1) & 1 ? A.ys1 : A.ys0, i, b, v);
    }
    return;
  }
  if constexpr (S == 1) {
    // torque and <m> of the starting state (a relaxation that is already
    // converged ends here with its mean recorded)
    float v[5] = {0.0f, tau_i, 0.0f, 0.0f, 0.0f};
    if (live) {
      const float w = (float)A.wvol[i] / sqrtf(mi[0] * mi[0] + mi[1] * mi[1] + mi[2] * mi[2]);
      v[2] = w * mi[0];
      v[3] = w * mi[1];
      v[4] = w * mi[2];
    }
    double tot[5];
    if (reduce_across_blocks(A, b, v, tot)) {
      SimCtl c = A.ctl[b];
      c.m_last[0] = tot[2];
      c.m_last[1] = tot[3];
      c.m_last[2] = tot[4];
      close_first(c, tot[1]);
      if (c.done) {
        A.active[b] = 0;
        atomicSub(A.n_active, 1);
      }
      A.ctl[b] = c;
    }
    return;
  }
  if constexpr (S == 7) {
    // embedded error, torque and <m> at the 5th-order solution, in FP32
    float v[5] = {0.0f, tau_i, 0.0f, 0.0f, 0.0f};
    if (live) {
      const float hs = (float)A.ctl[b].hs;
      const float atol = (float)A.atol, rtol = (float)A.rtol;
      const float *y0 = A.y + o;
      float e2 = 0.0f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float e = 0.0f;
#pragma unroll
        for (int j = 0; j < 7; ++j)
          if (c_dp_err[j] != 0.0) e = fmaf((float)c_dp_err[j], (j == 6) ? kk[c] : A.k[j][o + c], e);
        const float r = e * hs / (atol + rtol * fmaxf(fabsf(y0[c]), fabsf(mi[c])));
        e2 = fmaf(r, r, e2);
      }
      v[0] = e2;
      const float w = (float)A.wvol[i] / sqrtf(mi[0] * mi[0] + mi[1] * mi[1] + mi[2] * mi[2]);
      v[2] = w * mi[0];
      v[3] = w * mi[1];
      v[4] = w * mi[2];
    }
    double tot[5];
    if (reduce_across_blocks(A, b, v, tot)) {
      SimCtl c = A.ctl[b];
      int64_t row = -1;
      close_attempt(A, c, tot, &row);
      if (row >= 0) {
        double *mo = A.mavg + ((size_t)row * A.B + b) * 3;
        mo[0] = tot[2];
        mo[1] = tot[3];
        mo[2] = tot[4];
      }
      if (c.done) {
        A.active[b] = 0;
        atomicSub(A.n_active, 1);
      }
      A.ctl[b] = c;
    }
  }
}

// ---------------------------------------------------------------------------
// Small tile sets: a whole run in one cooperative kernel
// ---------------------------------------------------------------------------
// Below about two thousand tiles the FP32 tensor is a few tens of MB, a
// right-hand side is a few microseconds of work, and the step graph's 13
// dependent launches per attempt are what the step costs.  Here one CTA per
// SM keeps its rows of the tensor in shared memory for the whole call (or,
// when they do not fit, reads them from the L2-resident tensor), the stage
// inputs of all tiles pass through L2 between grid-wide barriers, and every
// CTA takes the step-control decisions itself from the same per-CTA partial
// sums reduced in the same fixed order (so all CTAs agree bit for bit): per
// attempt one barrier before each of the right-hand sides 3..7 and one for
// the error norm (the stage-2 input every CTA forms for all tiles itself),
// no launches.  The stage arithmetic is the graph path's except that the
// error norm and <m> are summed over rows and CTAs in another order.
constexpr int kSmallThreads = 256;
constexpr int kSmallWarps = kSmallThreads / 32;

struct SmallArgs {
  StageArgs A;
  const float *N;  // stored FP32 tensor, streaming layout
  int TR, TC;
  int64_t Q;
  float *xg;                // 2 x B x 3n: stage inputs of all tiles (ping-pong)
  float *part;              // [G][B][5] per-CTA partial sums
  unsigned long long *bar;  // barrier words (kBarWords, zeroed before the launch)
  int *abort_flag;          // a bounded wait gave up: every CTA leaves
  int *status;              // device status word (MT_DEV_TIMEOUT)
  int64_t iters;            // attempts at most
  int init;                 // evaluate k1 and the torque at the state first
  int R;                    // rows per CTA at most
  int nsmem;                // 1: the CTA's tensor rows live in shared memory, 0: read from L2
  int nplane;               // stored entry planes: 6, or 4 (single layer: no xz, yz)
};

// byte offsets of the dynamic shared memory of k_small_run
struct SmallSmem {
  size_t ctl, red, hd, y, k, tau, coef, par, kc, nbr, wex, kan, axis, wv, Ms, M, N, total;
};
__host__ __device__ __forceinline__ size_t small_take(size_t &o, size_t bytes) {
  const size_t at = o;
  o += (bytes + 15) & ~(size_t)15;
  return at;
}
__host__ __device__ __forceinline__ SmallSmem small_smem(int64_t n, int B, int R, bool nsmem) {
  SmallSmem s;
  size_t o = 0;
  s.ctl = small_take(o, sizeof(SimCtl) * B);
  s.red = small_take(o, sizeof(float) * kSmallWarps * 3 * 8);
  s.hd = small_take(o, sizeof(float) * B * R * 3);
  s.y = small_take(o, sizeof(float) * B * R * 3);
  s.k = small_take(o, sizeof(float) * 7 * B * R * 3);
  s.tau = small_take(o, sizeof(float) * B * R);
  s.coef = small_take(o, sizeof(float) * B * 36);  // (float)(h a_sj), s = 1..6, j < s
  s.par = small_take(o, sizeof(float) * B * 6);    // g1, g2, Ha, exchange factor
  s.kc = small_take(o, sizeof(int) * B);           // buffer of the committed k1 (0: k[0], 1: k[6])
  s.nbr = small_take(o, sizeof(int32_t) * R * 6);  // the CTA's rows: neighbours,
  s.wex = small_take(o, sizeof(float) * R * 6);    // exchange weights,
  s.kan = small_take(o, sizeof(float) * R);        // anisotropy, axis,
  s.axis = small_take(o, sizeof(float) * R * 3);
  s.wv = small_take(o, sizeof(float) * R);         // volume weights
  s.Ms = small_take(o, sizeof(float) * n);
  s.M = small_take(o, sizeof(float) * B * 3 * n);
  s.N = small_take(o, nsmem ? sizeof(float) * 6 * R * n : 0);
  s.total = o;
  return s;
}

struct SmallSh {
  SimCtl *ctl;
  float *red, *hd, *y, *k, *tau, *coef, *par, *wex, *kan, *axis, *wv, *Ms, *M, *N;
  int32_t *nbr;
  int *kc;
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Barrier words: [0] the arrival counter, which only grows (zeroed before
// the launch): barrier k is complete when it reaches k x G.  The abort flag
// sits on the next 128-byte line.
constexpr int kBarLine = 16;  // 8-byte words per 128-byte line
constexpr size_t kBarWords = kBarLine;

// Grid-wide barrier of a cooperative launch (all CTAs co-resident): the
// CTA's writes are ordered before thread 0's release-add by the CTA barrier,
// and the other CTAs' writes before its acquire-load of the completed count
// (release/acquire at GPU scope, no full fences).  The wait is bounded:
// after ~2 s (or once another CTA gave up) the status word gets
// MT_DEV_TIMEOUT, the abort flag is raised and false is returned.
__device__ __forceinline__ bool small_grid_sync(const SmallArgs &S, unsigned long long &k) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    k += 1;
    const unsigned long long target = k * gridDim.x;
    red_release_add_u64(S.bar, 1ull);
    int ok = 1;
    if (ld_acquire_u64(S.bar) < target) {
      const uint64_t t0 = mtd::globaltimer_ns();
      for (uint32_t it = 1;; ++it) {
        if (ld_acquire_u64(S.bar) >= target) break;
        if ((it & 63u) == 0u) {
          if (*reinterpret_cast<volatile int *>(S.abort_flag)) {
            ok = 0;
            break;
          }
          if (mtd::globaltimer_ns() - t0 > 2000000000ull) {
            atomicExch(S.status, MT_DEV_TIMEOUT);
            atomicExch(S.abort_flag, 1);
            ok = 0;
            break;
          }
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Eq. 1 for the CTA's rows from H_d in sh.hd: the local fields and the
// right-hand side into kout, the torque |m x H|/Ms into sh.tau (the
// arithmetic of k_stage).
__device__ __forceinline__ void small_llg(const StageArgs &A, const SmallSh &sh, float *kout, int R, int nr,
                                          int64_t r0) {
  const int64_t n = A.n;
  for (int p = threadIdx.x; p < A.B * nr; p += kSmallThreads) {
    const int b = p / nr, q = p - (p / nr) * nr;
    if (sh.ctl[b].done) continue;
    const int64_t i = r0 + q;
    const float *yb = sh.M + (size_t)b * 3 * n;
    const float mi[3] = {yb[3 * i], yb[3 * i + 1], yb[3 * i + 2]};
    const float *hd = sh.hd + ((size_t)b * R + q) * 3;
    const float *pb = sh.par + 6 * b;
    float H[3] = {hd[0], hd[1], hd[2]}, k[3];
    local_fields(pb + 2, pb[5], A.exch, sh.nbr + 6 * q, sh.wex + 6 * q, sh.kan[q], sh.axis + 3 * q, yb, mi, H);
    const float t = llg(pb[0], pb[1], mi, H, k) / sh.Ms[i];
    float *ko = kout + ((size_t)b * R + q) * 3;
    ko[0] = k[0];
    ko[1] = k[1];
    ko[2] = k[2];
    sh.tau[(size_t)b * R + q] = t;
  }
  __syncthreads();
}

// k_S of the CTA's rows [r0, r0 + nr) for every running simulation, from
// the stage input of all tiles in sh.M: H_d = -N (Ms m) from the rows held
// in sh.N, then the local fields and Eq. 1 (the arithmetic of k_stage); the
// torque |m x H|/Ms into sh.tau.
template <int RMAX>
__device__ __forceinline__ void small_rhs(const StageArgs &A, const SmallSh &sh, float *kout, int R, int nr,
                                          int64_t r0) {
  const int64_t n = A.n;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const size_t pl = (size_t)R * n;  // entries of one plane of the CTA's rows
  for (int b = 0; b < A.B; ++b) {
    if (sh.ctl[b].done) continue;  // the same in every thread
    float acc[RMAX][3];
#pragma unroll
    for (int q = 0; q < RMAX; ++q) acc[q][0] = acc[q][1] = acc[q][2] = 0.0f;
    const float *mb = sh.M + (size_t)b * 3 * n;
    for (int64_t j = tid; j < n; j += kSmallThreads) {
      const float ms = sh.Ms[j];
      const float x0 = ms * mb[3 * j], x1 = ms * mb[3 * j + 1], x2 = ms * mb[3 * j + 2];
#pragma unroll
      for (int q = 0; q < RMAX; ++q) {
        if (q < nr) {
          const float *e = sh.N + (size_t)q * n + j;
          const float nxx = e[0], nxy = e[pl], nxz = e[2 * pl], nyy = e[3 * pl], nyz = e[4 * pl], nzz = e[5 * pl];
          acc[q][0] = fmaf(nxx, x0, fmaf(nxy, x1, fmaf(nxz, x2, acc[q][0])));
          acc[q][1] = fmaf(nxy, x0, fmaf(nyy, x1, fmaf(nyz, x2, acc[q][1])));
          acc[q][2] = fmaf(nxz, x0, fmaf(nyz, x1, fmaf(nzz, x2, acc[q][2])));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RMAX; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float v = mtd::warp_sum(acc[q][c]);
        if (lane == 0 && q < nr) sh.red[w * 3 * RMAX + 3 * q + c] = v;
      }
    __syncthreads();
    if (tid < 3 * nr) {
      float s = 0.0f;
      for (int ww = 0; ww < kSmallWarps; ++ww) s += sh.red[ww * 3 * RMAX + tid];
      sh.hd[(size_t)b * R * 3 + tid] = -s;
    }
    __syncthreads();
  }
  small_llg(A, sh, kout, R, nr, r0);
}

// The same for tile sets whose rows do not fit the shared memory but whose
// tensor stays in L2 (up to ~100 MB): each warp owns rows w and w + 8 of the
// CTA (at most 16) and reads them from the streaming layout, lanes over the
// columns (128 consecutive columns of an entry plane are contiguous, 16-byte
// aligned), so no cross-warp reduction is needed.
__device__ __forceinline__ void small_rhs_l2(const SmallArgs &S, const StageArgs &A, const SmallSh &sh,
                                             float *kout, int R, int nr, int64_t r0) {
  const int64_t n = A.n;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const size_t plane = (size_t)S.TR * S.TC, chunk = (size_t)S.nplane * plane;
  const float *rowp[2] = {nullptr, nullptr};
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int q = w + kSmallWarps * r;
    if (q < nr) {
      const int64_t i = r0 + q, p = i / S.TR;
      rowp[r] = S.N + (size_t)p * S.Q * chunk + (size_t)(i - p * S.TR) * S.TC;
    }
  }
  for (int b = 0; b < A.B; ++b) {
    if (sh.ctl[b].done) continue;  // the same in every thread
    float acc[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
    const float *mb = sh.M + (size_t)b * 3 * n;
    // a lane takes 4 adjacent columns (one 16-byte load per entry plane; the
    // padding of the last column chunk holds zeros), two such groups per
    // step so that 24 loads per lane are in flight
    for (int64_t j0 = 4 * lane; j0 < n; j0 += 256) {
      float4 ent[2][2][6];
      float x[2][4][3];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int64_t j = j0 + 128 * u;
        const int64_t cq = j / S.TC;
        const size_t off = (size_t)cq * chunk + (size_t)(j - cq * S.TC);
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int e = 0; e < 6; ++e) {
            const int pl = stream_plane(e, S.nplane);
            ent[u][r][e] = (rowp[r] && j < n && pl >= 0)
                               ? __ldg(reinterpret_cast<const float4 *>(rowp[r] + off + pl * plane))
                               : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const bool in = j + k < n;
          const float ms = in ? sh.Ms[j + k] : 0.0f;
#pragma unroll
          for (int c = 0; c < 3; ++c) x[u][k][c] = in ? ms * mb[3 * (j + k) + c] : 0.0f;
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float *ex = reinterpret_cast<const float *>(&ent[u][r][0]) + k;  // entry e at ex[4 e]
            const float nxx = ex[0], nxy = ex[4], nxz = ex[8], nyy = ex[12], nyz = ex[16], nzz = ex[20];
            const float x0 = x[u][k][0], x1 = x[u][k][1], x2 = x[u][k][2];
            acc[r][0] = fmaf(nxx, x0, fmaf(nxy, x1, fmaf(nxz, x2, acc[r][0])));
            acc[r][1] = fmaf(nxy, x0, fmaf(nyy, x1, fmaf(nyz, x2, acc[r][1])));
            acc[r][2] = fmaf(nxz, x0, fmaf(nyz, x1, fmaf(nzz, x2, acc[r][2])));
          }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (!rowp[r]) continue;  // the same in the whole warp
      const int q = w + kSmallWarps * r;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float v = mtd::warp_sum(acc[r][c]);
        if (lane == 0) sh.hd[((size_t)b * R + q) * 3 + c] = -v;
      }
    }
  }
  __syncthreads();
  small_llg(A, sh, kout, R, nr, r0);
}

// all tiles' stage input (B x 3n floats written by every CTA before the
// barrier) into shared memory, through L2
__device__ __forceinline__ void small_load_state(float *sM, const float *src, size_t count) {
  if ((count & 3) == 0) {  // src and sM are 16-byte aligned
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(sM);
    for (size_t q = threadIdx.x; q < count / 4; q += kSmallThreads) d4[q] = __ldcg(s4 + q);
  } else {
    for (size_t q = threadIdx.x; q < count; q += kSmallThreads) sM[q] = __ldcg(src + q);
  }
  __syncthreads();
}

// Warp 0: the sums of the CTA's 5 values per simulation (sum, max, sum,
// sum, sum over its rows, one lane per row) to part[g][b]; after the
// barrier, every CTA's warp 0 adds the G partials of b in the same fixed
// order (lane-strided, then a butterfly), so all CTAs hold the same totals.
__device__ __forceinline__ void small_warp_reduce(float v[5]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    v[1] = mtd::nan_max(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
    v[2] += __shfl_xor_sync(0xffffffffu, v[2], o);
    v[3] += __shfl_xor_sync(0xffffffffu, v[3], o);
    v[4] += __shfl_xor_sync(0xffffffffu, v[4], o);
  }
}
__device__ __forceinline__ void small_partial(const SmallArgs &S, int b, float v[5]) {
  small_warp_reduce(v);
  if ((threadIdx.x & 31) == 0) {
    float *dst = S.part + ((size_t)blockIdx.x * S.A.B + b) * 5;
    for (int q = 0; q < 5; ++q) dst[q] = v[q];
  }
}
__device__ __forceinline__ void small_total(const SmallArgs &S, int b, double tot[5]) {
  float acc[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  for (int g = threadIdx.x & 31; g < (int)gridDim.x; g += 32) {
    const float *src = S.part + ((size_t)g * S.A.B + b) * 5;
    acc[0] += __ldcg(&src[0]);
    acc[1] = mtd::nan_max(acc[1], __ldcg(&src[1]));
    acc[2] += __ldcg(&src[2]);
    acc[3] += __ldcg(&src[3]);
    acc[4] += __ldcg(&src[4]);
  }
  small_warp_reduce(acc);
  for (int q = 0; q < 5; ++q) tot[q] = (double)acc[q];
}

// m / |m| with every rounding pinned (no contraction freedom), so that the
// CTA committing a row and the CTAs forming the next stage input from it
// compute the same bits
__device__ __forceinline__ void small_unit(const float *v, float *out) {
  const float inv = rsqrtf(__fmaf_rn(v[2], v[2], __fmaf_rn(v[1], v[1], __fmul_rn(v[0], v[0]))));
  out[0] = __fmul_rn(v[0], inv);
  out[1] = __fmul_rn(v[1], inv);
  out[2] = __fmul_rn(v[2], inv);
}

// this CTA's rows [r0, r0 + nr) of a per-simulation plane (B x R x 3 in
// shared memory) into the tile-major global array dst (B x 3n)
__device__ __forceinline__ void small_publish_rows(float *dst, const float *src, int B, int R, int nr, int64_t r0,
                                                   int64_t n) {
  for (int p = threadIdx.x; p < B * nr * 3; p += kSmallThreads) {
    const int b = p / (nr * 3), qc = p - b * nr * 3;
    dst[(size_t)b * 3 * n + 3 * r0 + qc] = src[(size_t)b * R * 3 + qc];
  }
}

// (float)(h a_sj) of every stage-input row s = 1..6 (the inputs of stages
// 2..7) and j < s, per simulation: coef[36 b + 6 (s - 1) + j]
__device__ __forceinline__ void small_coefficients(const StageArgs &A, const SmallSh &sh) {
  for (int p = threadIdx.x; p < A.B * 36; p += kSmallThreads) {
    const int b = p / 36, rj = p - b * 36, r = rj / 6, j = rj - r * 6;
    if (j <= r) sh.coef[p] = (float)(sh.ctl[b].hs * c_dp_a[r + 1][j]);
  }
  __syncthreads();
}

template <int RMAX, bool NSMEM>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small_run(SmallArgs S) {
  extern __shared__ __align__(16) unsigned char smem[];
  const StageArgs &A = S.A;
  const int64_t n = A.n;
  const int B = A.B, R = S.R;
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)g * n / G, r1 = (int64_t)(g + 1) * n / G;
  const int nr = (int)(r1 - r0);
  const SmallSmem L = small_smem(n, B, R, NSMEM);
  SmallSh sh;
  sh.ctl = reinterpret_cast<SimCtl *>(smem + L.ctl);
  sh.red = reinterpret_cast<float *>(smem + L.red);
  sh.hd = reinterpret_cast<float *>(smem + L.hd);
  sh.y = reinterpret_cast<float *>(smem + L.y);
  sh.k = reinterpret_cast<float *>(smem + L.k);
  sh.tau = reinterpret_cast<float *>(smem + L.tau);
  sh.coef = reinterpret_cast<float *>(smem + L.coef);
  sh.par = reinterpret_cast<float *>(smem + L.par);
  sh.nbr = reinterpret_cast<int32_t *>(smem + L.nbr);
  sh.kc = reinterpret_cast<int *>(smem + L.kc);
  sh.wex = reinterpret_cast<float *>(smem + L.wex);
  sh.kan = reinterpret_cast<float *>(smem + L.kan);
  sh.axis = reinterpret_cast<float *>(smem + L.axis);
  sh.wv = reinterpret_cast<float *>(smem + L.wv);
  sh.Ms = reinterpret_cast<float *>(smem + L.Ms);
  sh.M = reinterpret_cast<float *>(smem + L.M);
  sh.N = reinterpret_cast<float *>(smem + L.N);
  const size_t kpl = (size_t)B * R * 3;  // floats of one derivative plane
  const size_t state = (size_t)B * 3 * n;
  unsigned long long nbar = 0;  // barriers passed
  bool ok = true;
  const float atol = (float)A.atol, rtol = (float)A.rtol;

  // control blocks and parameters, Ms, the CTA's rows of N (plane e, row q,
  // column j) and their tile constants, the rows of y and of the derivative
  // the next attempt starts from
  for (int b = tid; b < B; b += kSmallThreads) {
    sh.ctl[b] = A.ctl[b];
    float *pb = sh.par + 6 * b;
    pb[0] = A.g1[b];
    pb[1] = A.g2[b];
    pb[2] = A.Ha[3 * b];
    pb[3] = A.Ha[3 * b + 1];
    pb[4] = A.Ha[3 * b + 2];
    pb[5] = A.xsc ? A.xsc[b] : 1.0f;
    sh.kc[b] = 0;
  }
  for (int64_t j = tid; j < n; j += kSmallThreads) sh.Ms[j] = A.Ms[j];
  if (NSMEM)
    for (int64_t q = tid; q < (int64_t)6 * nr * n; q += kSmallThreads) {
      const int64_t j = q % n, eq = q / n;
      const int e = (int)(eq / nr), r = (int)(eq % nr);
      const int pl = stream_plane(e, S.nplane);
      sh.N[((size_t)e * R + r) * n + j] = pl < 0 ? 0.0f : S.N[layout_index(r0 + r, j, pl, S.TR, S.TC, S.nplane, S.Q)];
    }
  for (int q = tid; q < nr; q += kSmallThreads) {
    const int64_t i = r0 + q;
    for (int f = 0; f < 6; ++f) {
      sh.nbr[6 * q + f] = A.nbr[6 * i + f];
      sh.wex[6 * q + f] = A.wex[6 * i + f];
    }
    sh.kan[q] = A.kan[i];
    for (int c = 0; c < 3; ++c) sh.axis[3 * q + c] = A.axis[3 * i + c];
    sh.wv[q] = (float)A.wvol[i];
  }
  for (int p = tid; p < B * nr * 3; p += kSmallThreads) {
    const int b = p / (nr * 3), qc = p - b * nr * 3;
    const size_t o = (size_t)b * 3 * n + 3 * r0 + qc;
    sh.y[(size_t)b * R * 3 + qc] = A.y[o];
    sh.k[(size_t)b * R * 3 + qc] = A.k[0][o];
  }
  __syncthreads();

  if (S.init) {  // k1 and the torque at the state
    small_load_state(sh.M, A.y, state);
    if (NSMEM) small_rhs<RMAX>(A, sh, sh.k, R, nr, r0);
    else small_rhs_l2(S, A, sh, sh.k, R, nr, r0);
    small_publish_rows(A.k[0], sh.k, B, R, nr, r0, n);  // read by all CTAs after the barrier
    for (int b = warp; b < B; b += kSmallWarps) {
      if (sh.ctl[b].done) continue;
      float v[5] = {0.0f, lane < nr ? sh.tau[(size_t)b * R + lane] : 0.0f, 0.0f, 0.0f, 0.0f};
      small_partial(S, b, v);
    }
    ok = small_grid_sync(S, nbar);
    if (ok)
      for (int b = warp; b < B; b += kSmallWarps) {
        if (sh.ctl[b].done) continue;
        double tot[5];
        small_total(S, b, tot);
        if (lane == 0) close_first(sh.ctl[b], tot[1]);
        __syncwarp();
      }
    __syncthreads();
  }

  for (int64_t it = 0; ok && it < S.iters; ++it) {
    bool any = false;
    for (int b = 0; b < B; ++b) any = any || !sh.ctl[b].done;
    if (!any) break;
    small_coefficients(A, sh);
    // stage 2 needs no exchange between CTAs: every CTA forms the input of
    // all tiles, y + (h a_21) k1, from the committed state (after an accepted
    // attempt: the normalised 5th-order solution still in sh.M and the k7
    // every CTA published; else the committed y and k1 in global memory)
    for (int b = 0; b < B; ++b) {
      if (sh.ctl[b].done) continue;
      const bool adopt = it > 0 && sh.ctl[b].accepted;
      const float a21 = sh.coef[36 * b];
      const float *kb = (sh.kc[b] ? A.k[6] : A.k[0]) + (size_t)b * 3 * n;
      const float *yb = A.y + (size_t)b * 3 * n;
      float *mb = sh.M + (size_t)b * 3 * n;
      for (int64_t j = tid; j < n; j += kSmallThreads) {
        float y[3];
        if (adopt) {
          small_unit(mb + 3 * j, y);
        } else {
#pragma unroll
          for (int c = 0; c < 3; ++c) y[c] = __ldcg(yb + 3 * j + c);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) mb[3 * j + c] = __fadd_rn(y[c], __fmul_rn(a21, __ldcg(kb + 3 * j + c)));
      }
    }
    __syncthreads();
    if (NSMEM) small_rhs<RMAX>(A, sh, sh.k + kpl, R, nr, r0);
    else small_rhs_l2(S, A, sh, sh.k + kpl, R, nr, r0);
    for (int st = 3; st <= 7 && ok; ++st) {
      // this CTA's rows of the stage input y + sum_j (h a_sj) k_j
      float *xo = S.xg + (size_t)(st & 1) * state;
      for (int p = tid; p < B * nr; p += kSmallThreads) {
        const int b = p / nr, q = p - (p / nr) * nr;
        if (sh.ctl[b].done) continue;
        const float *cf = sh.coef + 36 * b + 6 * (st - 2);
        float acc[3] = {0.0f, 0.0f, 0.0f};
        for (int j = 0; j < st - 1; ++j) {
          const float a = cf[j];
          if (a != 0.0f) {
            const float *kj = sh.k + j * kpl + ((size_t)b * R + q) * 3;
            acc[0] += a * kj[0];
            acc[1] += a * kj[1];
            acc[2] += a * kj[2];
          }
        }
        const float *y0 = sh.y + ((size_t)b * R + q) * 3;
        float *d = xo + (size_t)b * 3 * n + 3 * (r0 + q);
        d[0] = y0[0] + acc[0];
        d[1] = y0[1] + acc[1];
        d[2] = y0[2] + acc[2];
      }
      ok = small_grid_sync(S, nbar);
      if (!ok) break;
      small_load_state(sh.M, xo, state);
      if (NSMEM) small_rhs<RMAX>(A, sh, sh.k + (st - 1) * kpl, R, nr, r0);
      else small_rhs_l2(S, A, sh, sh.k + (st - 1) * kpl, R, nr, r0);
    }
    if (!ok) break;
    // this CTA's k7 rows into the buffer not holding the committed k1: the
    // next attempt's k1 if this one is accepted
    for (int p = tid; p < B * nr * 3; p += kSmallThreads) {
      const int b = p / (nr * 3), qc = p - b * nr * 3;
      if (sh.ctl[b].done) continue;
      (sh.kc[b] ? A.k[0] : A.k[6])[(size_t)b * 3 * n + 3 * r0 + qc] = sh.k[6 * kpl + (size_t)b * R * 3 + qc];
    }
    // embedded error, torque and <m> at the 5th-order solution (the stage-7
    // input), in FP32 over the CTA's rows: one lane per row
    for (int b = warp; b < B; b += kSmallWarps) {
      if (sh.ctl[b].done) continue;
      float v[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      if (lane < nr) {
        const float hs = (float)sh.ctl[b].hs;
        const int64_t i = r0 + lane;
        const float *mi = sh.M + (size_t)b * 3 * n + 3 * i;
        const float *y0 = sh.y + ((size_t)b * R + lane) * 3;
        for (int c = 0; c < 3; ++c) {
          float e = 0.0f;
#pragma unroll
          for (int j = 0; j < 7; ++j)
            if (c_dp_err[j] != 0.0) e = fmaf((float)c_dp_err[j], sh.k[j * kpl + ((size_t)b * R + lane) * 3 + c], e);
          const float r = e * hs / (atol + rtol * fmaxf(fabsf(y0[c]), fabsf(mi[c])));
          v[0] = fmaf(r, r, v[0]);
        }
        v[1] = sh.tau[(size_t)b * R + lane];
        const float wv = sh.wv[lane] / sqrtf(mi[0] * mi[0] + mi[1] * mi[1] + mi[2] * mi[2]);
        v[2] = wv * mi[0];
        v[3] = wv * mi[1];
        v[4] = wv * mi[2];
      }
      small_partial(S, b, v);
    }
    ok = small_grid_sync(S, nbar);
    if (!ok) break;
    for (int b = warp; b < B; b += kSmallWarps) {
      if (sh.ctl[b].done) continue;
      double tot[5];
      small_total(S, b, tot);
      if (lane == 0) {
        int64_t row = -1;
        close_attempt(A, sh.ctl[b], tot, &row);
        if (g == 0 && row >= 0) {
          double *mo = A.mavg + ((size_t)row * B + b) * 3;
          mo[0] = tot[2];
          mo[1] = tot[3];
          mo[2] = tot[4];
        }
      }
      __syncwarp();
    }
    __syncthreads();
    // accepted: adopt the normalised 5th-order solution (this CTA's rows also
    // into the committed y in global memory, read after a later rejection);
    // k7 is the next k1
    for (int p = tid; p < B * nr; p += kSmallThreads) {
      const int b = p / nr, q = p - (p / nr) * nr;
      if (!sh.ctl[b].accepted) continue;
      const float *yn = sh.M + (size_t)b * 3 * n + 3 * (r0 + q);
      float *y0 = sh.y + ((size_t)b * R + q) * 3;
      float *k1 = sh.k + ((size_t)b * R + q) * 3;
      const float *k7 = sh.k + 6 * kpl + ((size_t)b * R + q) * 3;
      float *yg = A.y + (size_t)b * 3 * n + 3 * (r0 + q);
      small_unit(yn, y0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        yg[c] = y0[c];
        k1[c] = k7[c];
      }
    }
    __syncthreads();
    for (int b = tid; b < B; b += kSmallThreads)
      if (sh.ctl[b].accepted) sh.kc[b] ^= 1;
    __syncthreads();
  }
  if (!ok) return;  // timed out: the status word tells the host
  // write back: the state and the next derivative of this CTA's rows; CTA 0
  // the control blocks (nothing left to commit) and the active set
  for (int p = tid; p < B * nr * 3; p += kSmallThreads) {
    const int b = p / (nr * 3), qc = p - b * nr * 3;
    const size_t o = (size_t)b * 3 * n + 3 * r0 + qc;
    A.y[o] = sh.y[(size_t)b * R * 3 + qc];
    A.k[0][o] = sh.k[(size_t)b * R * 3 + qc];
  }
  if (g == 0 && tid == 0) {
    int na = 0;
    for (int b = 0; b < B; ++b) {
      SimCtl c = sh.ctl[b];
      c.accepted = 0;
      A.ctl[b] = c;
      A.active[b] = c.done ? 0 : 1;
      na += c.done ? 0 : 1;
    }
    *A.n_active = na;
  }
}

// failure-detection self-test: CTA 0 leaves without arriving, so the other
// CTAs' bounded barrier wait runs out
__global__ void k_barrier_selftest(SmallArgs S) {
  unsigned long long nbar = 0;
  if (blockIdx.x == 0) return;
  small_grid_sync(S, nbar);
}

// put a prepared control block into slot b and make it active
__global__ void k_admit(SimCtl *ctl, int *active, int *n_active, int b, SimCtl c) {
  ctl[b] = c;
  if (!active[b]) {
    active[b] = 1;
    atomicAdd(n_active, 1);
  }
}

// Energy (Eqs. 4, 6, 8, 11, 15): every quadratic density is -(mu0 Ms/2) m.H
// of its field and the Zeeman one -mu0 Ms m.Ha, so per tile
//   e_i = -mu0 Ms_i V_i m_i.(Ha + (H_d + H_ex + H_an)/2)  split by term.
__global__ void k_energy(int64_t n, const int32_t *nbr, const float *wex, const float *kan, const float *axis,
                         const float *Ms, const double *wvol, double vol_total, bool exch, const float *m,
                         const float *Hd, const float *Ha, const float *xsc, double *E) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  double e[4] = {0, 0, 0, 0};
  if (i < n) {
    const size_t o = (size_t)b * 3 * n + 3 * i;
    const float mi[3] = {m[o], m[o + 1], m[o + 2]};
    double hex[3] = {0, 0, 0}, han[3] = {0, 0, 0};
    if (exch) {
      const float *mb = m + (size_t)b * 3 * n;
      for (int f = 0; f < 6; ++f) {
        const int32_t p = nbr[6 * i + f];
        if (p < 0) continue;
        for (int c = 0; c < 3; ++c) hex[c] += (double)wex[6 * i + f] * ((double)mb[3 * p + c] - (double)mi[c]);
      }
      for (int c = 0; c < 3; ++c) hex[c] *= (double)xsc[b];
    }
    const double me = (double)mi[0] * axis[3 * i] + (double)mi[1] * axis[3 * i + 1] + (double)mi[2] * axis[3 * i + 2];
    for (int c = 0; c < 3; ++c) han[c] = (double)kan[i] * me * axis[3 * i + c];
    const double w = MT_MU0 * (double)Ms[i] * wvol[i] * vol_total;
    for (int c = 0; c < 3; ++c) {
      e[0] += -w * mi[c] * (double)Ha[3 * b + c];
      e[1] += -0.5 * w * mi[c] * (double)Hd[o + c];
      e[2] += -0.5 * w * mi[c] * hex[c];
      e[3] += -0.5 * w * mi[c] * han[c];
    }
  }
  __shared__ double sh[8][4];
  for (int q = 0; q < 4; ++q) e[q] = mtd::warp_sum(e[q]);
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  if (lane == 0)
    for (int q = 0; q < 4; ++q) sh[wq][q] = e[q];
  __syncthreads();
  if (threadIdx.x < 4) {
    double acc = 0;
    for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) acc += sh[ww][threadIdx.x];
    atomicAdd(&E[4 * b + threadIdx.x], acc);
  }
}

// standalone right-hand side: dmdt and per-simulation max torque
__global__ void k_rhs_plain(int64_t n, const int32_t *nbr, const float *wex, const float *kan, const float *axis,
                            const float *Ms, bool exch, const float *m, const float *Hd, const float *g1,
                            const float *g2, const float *Ha, const float *xsc, float *dmdt, float *tau) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= n) return;
  StageArgs A{};
  A.n = n;
  A.nbr = nbr;
  A.wex = wex;
  A.kan = kan;
  A.axis = axis;
  A.exch = exch;
  A.Ha = Ha;
  A.xsc = xsc;
  const size_t o = (size_t)b * 3 * n + 3 * i;
  const float mi[3] = {m[o], m[o + 1], m[o + 2]};
  float H[3], k[3];
  effective_field(A, m, Hd, i, b, mi, H);
  const float t = llg(g1[b], g2[b], mi, H, k) / Ms[i];
  dmdt[o] = k[0];
  dmdt[o + 1] = k[1];
  dmdt[o + 2] = k[2];
  if (tau) atomicMax(reinterpret_cast<int *>(tau + b), __float_as_int(t));
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace mt {

void launch_rhs_plain(const mt_tensor *T, const float *m, const float *Hd, int B, const float *g1,
                      const float *g2, const float *Ha, const float *xsc, float *dmdt, float *tau, cudaStream_t s) {
  const mt_tiles *t = T->tiles;
  dim3 grid((unsigned)((T->n + 255) / 256), (unsigned)B);
  k_rhs_plain<<<grid, 256, 0, s>>>(T->n, t->d_nbr, t->d_wex, t->d_kan, t->d_axis, t->d_Ms, t->has_exchange, m, Hd,
                                   g1, g2, Ha, xsc, dmdt, tau);
}

void launch_energy(const mt_tensor *T, const float *m, const float *Hd, int B, const float *Ha, const float *xsc,
                   double *E, cudaStream_t s) {
  const mt_tiles *t = T->tiles;
  dim3 grid((unsigned)((T->n + 255) / 256), (unsigned)B);
  k_energy<<<grid, 256, 0, s>>>(T->n, t->d_nbr, t->d_wex, t->d_kan, t->d_axis, t->d_Ms, t->d_wvol, t->vol_total,
                                t->has_exchange, m, Hd, Ha, xsc, E);
}

void llg_prefactors(const mt_llg_params *p, int B, std::vector<float> &g1, std::vector<float> &g2,
                    std::vector<float> &ha, std::vector<float> &xsc) {
  g1.resize(B);
  g2.resize(B);
  ha.resize(3 * B);
  xsc.resize(B);
  for (int b = 0; b < B; ++b) {
    const double a = p->alpha[b];
    double G1, G2;
    if (p->form == MT_FORM_GILBERT) {
      G1 = p->gamma / (1.0 + a * a);
      G2 = G1 * a;
    } else {
      G1 = p->gamma;
      G2 = a;
    }
    if (!p->precess) G1 = 0.0;
    g1[b] = (float)G1;
    g2[b] = (float)G2;
    for (int c = 0; c < 3; ++c) ha[3 * b + c] = (float)p->Ha[3 * b + c];
    xsc[b] = p->exch_scale ? (float)p->exch_scale[b] : 1.0f;
  }
}

}  // namespace mt

struct mt_integrator {
  mt_tensor *T = nullptr;
  int B = 0;
  cudaStream_t stream = nullptr;       // private non-blocking stream: capture and replay
  cudaStream_t user_stream = nullptr;  // the caller's stream, ordered against `stream` by events
  cudaEvent_t order_ev = nullptr;
  mt_ode_opts o{};
  int form = 0, precess = 1;
  double gamma = 0;
  // device state
  float *y = nullptr, *ys0 = nullptr, *ys1 = nullptr, *Hd = nullptr, *xs = nullptr;
  float *k[7] = {};
  float *g1 = nullptr, *g2 = nullptr, *Ha = nullptr, *xsc = nullptr;
  float *part = nullptr;
  float *colpart = nullptr;  // half-stored tensor: column work area of the product
  int *count = nullptr;
  SimCtl *ctl = nullptr;
  int *active = nullptr;
  int *n_active = nullptr;
  float *red = nullptr;
  int *red_count = nullptr;
  double *mavg = nullptr;
  int64_t mavg_cap = 0;
  int *h_poll = nullptr;  // pinned, 2 slots
  float *h_slot_par = nullptr;  // pinned staging of per-slot parameters (g1, g2, Ha) for admissions
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaGraphExec_t exec = nullptr;
  GemmPlan plan;  // dense layout: tensor maps of the batched product
  int nblk = 0;
  bool need_init = true;
  std::vector<void *> allocs;
  // small tile sets: the whole call in one cooperative kernel (k_small_run)
  int path = MT_PATH_GRAPH;  // the one in use
  bool small_ok = false;     // the tile set and batch fit it
  int small_G = 0, small_R = 0, small_rmax = 0;
  bool small_nsmem = true;  // tensor rows in shared memory (else read from L2)
  size_t small_smem_bytes = 0;
  float *sm_xg = nullptr;
  float *sm_part = nullptr;
  unsigned long long *sm_bar = nullptr;  // barrier words, then the abort flag
};

namespace {

StageArgs stage_args(mt_integrator *I) {
  const mt_tensor *T = I->T;
  const mt_tiles *t = T->tiles;
  StageArgs A{};
  A.n = T->n;
  A.B = I->B;
  A.nbr = t->d_nbr;
  A.wex = t->d_wex;
  A.kan = t->d_kan;
  A.axis = t->d_axis;
  A.Ms = t->d_Ms;
  A.wvol = t->d_wvol;
  A.exch = t->has_exchange;
  A.g1 = I->g1;
  A.g2 = I->g2;
  A.Ha = I->Ha;
  A.xsc = I->xsc;
  A.y = I->y;
  A.ys0 = I->ys0;
  A.ys1 = I->ys1;
  A.Hd = I->Hd;
  A.xs = I->xs;
  for (int s = 0; s < 7; ++s) A.k[s] = I->k[s];
  A.Q = T->L.Q;
  A.TC = T->L.TC;
  A.xs_mode = T->layout == MT_LAYOUT_DENSE ? (T->prec == MT_BF16_SPLIT ? 2 : 1) : T->layout == MT_LAYOUT_SPARSE ? 3 : 0;
  A.Kp = T->Kp;
  A.Bp = mt::dense_pad_batch(I->B);
  A.X = reinterpret_cast<__nv_bfloat16 *>(I->xs);
  A.mT = T->layout == MT_LAYOUT_DENSE ? mt::dense_mT(T, I->B, I->xs) : nullptr;
  A.ctl = I->ctl;
  A.active = I->active;
  A.n_active = I->n_active;
  A.red = I->red;
  A.red_count = I->red_count;
  A.mavg = I->mavg;
  A.rtol = I->o.rtol;
  A.atol = I->o.atol;
  A.hmax = I->o.hmax;
  A.fixed_h = I->o.fixed_h;
  return A;
}

constexpr size_t kSmallSmemMax = 225 * 1024;  // of the 227 KB a CTA may opt in to

template <int RMAX, bool NSMEM>
cudaError_t small_attr(size_t bytes, int *per_sm) {
  cudaError_t e =
      cudaFuncSetAttribute(k_small_run<RMAX, NSMEM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_small_run<RMAX, NSMEM>, kSmallThreads, bytes);
  return e;
}

// a tensor the one-kernel path reads from L2 every right-hand side must
// stay there (L2: 129 MB)
constexpr size_t kSmallL2Bytes = 96ull << 20;

// Does the one-kernel path fit this tile set and batch?  An FP32 streaming
// tensor; one CTA per SM (or per tile) and a co-resident grid; either at
// most 8 rows per CTA whose tensor rows and the state of all tiles fit the
// shared memory, or at most 16 rows per CTA read from an L2-resident tensor
// with the state in shared memory.
bool small_plan(mt_integrator *I) {
  const mt_tensor *T = I->T;
  if (T->prec != MT_F32 || T->layout != MT_LAYOUT_STREAM || T->L.half) return false;
  const int64_t n = T->n;
  const int sms = T->tiles->ctx->num_sms;
  if (n < 1 || sms < 1) return false;
  const int64_t r_sm = (n + sms - 1) / sms;
  for (int pass = 0; pass < 2; ++pass) {
    const bool nsmem = pass == 0;
    // rows per CTA: enough to cover the tiles with one CTA per SM (fewer
    // CTAs meeting at each barrier measured no faster)
    const int R = (int)r_sm;
    if (R > (nsmem ? 8 : 2 * kSmallWarps)) continue;
    if (!nsmem && (T->bytes > kSmallL2Bytes || T->L.TC % 4 != 0)) continue;
    const size_t bytes = small_smem(n, I->B, R, nsmem).total;
    if (bytes > kSmallSmemMax) continue;
    const int G = (int)((n + R - 1) / R);
    const int rmax = !nsmem ? 2 : R <= 2 ? 2 : R <= 4 ? 4 : 8;
    int per_sm = 0;
    const cudaError_t e = !nsmem     ? small_attr<2, false>(bytes, &per_sm)
                          : rmax == 2 ? small_attr<2, true>(bytes, &per_sm)
                          : rmax == 4 ? small_attr<4, true>(bytes, &per_sm)
                                      : small_attr<8, true>(bytes, &per_sm);
    if (e != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (per_sm < 1 || (int64_t)per_sm * sms < G) continue;
    I->small_G = G;
    I->small_R = R;
    I->small_rmax = rmax;
    I->small_nsmem = nsmem;
    I->small_smem_bytes = bytes;
    return true;
  }
  return false;
}

mt_status launch_small(mt_integrator *I, int init, int64_t iters) {
  const mt_tensor *T = I->T;
  SmallArgs S{};
  S.A = stage_args(I);
  S.N = static_cast<const float *>(T->d_data);
  S.TR = T->L.TR;
  S.TC = T->L.TC;
  S.Q = T->L.Q;
  S.xg = I->sm_xg;
  S.part = I->sm_part;
  S.bar = I->sm_bar;
  S.abort_flag = reinterpret_cast<int *>(I->sm_bar + kBarWords);
  S.status = T->tiles->ctx->d_status;
  S.iters = iters;
  S.init = init;
  S.R = I->small_R;
  S.nsmem = I->small_nsmem ? 1 : 0;
  S.nplane = T->L.nplane;
  MT_CUDA(cudaMemsetAsync(I->sm_bar, 0, (kBarWords + kBarLine) * sizeof(unsigned long long), I->stream));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)I->small_G);
  cfg.blockDim = dim3(kSmallThreads);
  cfg.dynamicSmemBytes = I->small_smem_bytes;
  cfg.stream = I->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // after the context's previous one-kernel launch, whatever its stream: two
  // such grids resident together could each hold SMs the other waits for
  mt_ctx *ctx = T->tiles->ctx;
  std::lock_guard<std::mutex> lock(ctx->small_mu);
  cudaError_t e = cudaSuccess;
  if (!ctx->small_ev) e = cudaEventCreateWithFlags(&ctx->small_ev, cudaEventDisableTiming);
  else e = cudaStreamWaitEvent(I->stream, ctx->small_ev, 0);
  if (e == cudaSuccess) {
    if (!I->small_nsmem) e = cudaLaunchKernelEx(&cfg, k_small_run<2, false>, S);
    else if (I->small_rmax == 2) e = cudaLaunchKernelEx(&cfg, k_small_run<2, true>, S);
    else if (I->small_rmax == 4) e = cudaLaunchKernelEx(&cfg, k_small_run<4, true>, S);
    else e = cudaLaunchKernelEx(&cfg, k_small_run<8, true>, S);
  }
  if (e == cudaSuccess) e = cudaEventRecord(ctx->small_ev, I->stream);
  if (e != cudaSuccess) return mt::cuda_fail(e, "k_small_run launch", __FILE__, __LINE__);
  I->need_init = false;
  return MT_OK;
}

template <int S>
void launch_stage(mt_integrator *I, const StageArgs &A) {
  dim3 grid((unsigned)I->nblk, (unsigned)I->B);
  mt::launch_pdl(k_stage<S>, grid, dim3(kStageThreads), 0, I->stream, A);
}

// demag product of the stage input `m` into I->Hd (xs already formed)
void demag(mt_integrator *I, const float *m) {
  if (I->T->layout == MT_LAYOUT_SPARSE) {
    mt::launch_spmv(I->T, I->xs, I->B, I->Hd, I->active, I->stream);
    return;
  }
  if (I->T->layout == MT_LAYOUT_DENSE) {
    mt::launch_gemm(I->T, I->plan, I->Hd, I->part, I->count, I->n_active, I->T->tiles->ctx->d_status, I->stream);
    mt::launch_near(I->T, mt::dense_mT(I->T, I->B, I->xs), 1, mt::dense_pad_batch(I->B), I->B, I->Hd, I->active,
                    I->stream);
  } else {
    mt::launch_matvec(I->T, I->xs, I->B, I->Hd, I->part, I->count, I->active, I->T->tiles->ctx->d_status,
                      I->stream, I->colpart);
    mt::launch_near(I->T, m, 3 * I->T->n, 1, I->B, I->Hd, I->active, I->stream);
  }
}

void enqueue_attempt(mt_integrator *I) {
  StageArgs A = stage_args(I);
  dim3 grid((unsigned)I->nblk, (unsigned)I->B);
  mt::launch_pdl(k_begin, grid, dim3(kStageThreads), 0, I->stream, A);
  demag(I, I->ys0);
  launch_stage<2>(I, A);
  demag(I, I->ys1);
  launch_stage<3>(I, A);
  demag(I, I->ys0);
  launch_stage<4>(I, A);
  demag(I, I->ys1);
  launch_stage<5>(I, A);
  demag(I, I->ys0);
  launch_stage<6>(I, A);
  demag(I, I->ys1);
  launch_stage<7>(I, A);
}

mt_status enqueue_init(mt_integrator *I, int fresh_only = 0) {
  StageArgs A = stage_args(I);
  A.fresh_only = fresh_only;
  if (I->T->layout == MT_LAYOUT_DENSE)
    mt::launch_prep_dense_x(I->T, I->y, I->B, I->xs, I->stream);
  else
    mt::launch_prep_xs(I->T, I->y, I->B, I->xs, I->stream);
  demag(I, I->y);
  launch_stage<1>(I, A);
  MT_CUDA(cudaGetLastError());
  I->need_init = false;
  return MT_OK;
}

mt_status enqueue_commit(mt_integrator *I) {
  StageArgs A = stage_args(I);
  dim3 grid((unsigned)I->nblk, (unsigned)I->B);
  k_commit<<<grid, kStageThreads, 0, I->stream>>>(A);
  MT_CUDA(cudaGetLastError());
  return MT_OK;
}

template <typename P>
mt_status dalloc(mt_integrator *I, P **p, size_t bytes) {
  MT_CUDA(cudaMalloc((void **)p, bytes));
  MT_CUDA(cudaMemsetAsync(*p, 0, bytes, I->stream));
  I->allocs.push_back((void *)*p);
  return MT_OK;
}

mt_status read_ctl(mt_integrator *I, std::vector<SimCtl> &c) {
  c.resize(I->B);
  MT_CUDA(cudaMemcpyAsync(c.data(), I->ctl, sizeof(SimCtl) * I->B, cudaMemcpyDeviceToHost, I->stream));
  MT_CUDA(cudaStreamSynchronize(I->stream));
  return MT_OK;
}

mt_status write_ctl(mt_integrator *I, const std::vector<SimCtl> &c) {
  std::vector<int> act(I->B);
  int na = 0;
  for (int b = 0; b < I->B; ++b) {
    act[b] = c[b].done ? 0 : 1;
    na += act[b];
  }
  MT_CUDA(cudaMemcpyAsync(I->ctl, c.data(), sizeof(SimCtl) * I->B, cudaMemcpyHostToDevice, I->stream));
  MT_CUDA(cudaMemcpyAsync(I->active, act.data(), sizeof(int) * I->B, cudaMemcpyHostToDevice, I->stream));
  MT_CUDA(cudaMemcpyAsync(I->n_active, &na, sizeof(int), cudaMemcpyHostToDevice, I->stream));
  MT_CUDA(cudaStreamSynchronize(I->stream));  // host vectors go out of scope
  return MT_OK;
}

void fill_stats(const std::vector<SimCtl> &c, mt_stats *st, int B) {
  if (!st) return;
  for (int b = 0; b < B; ++b) {
    st[b].n_accept = c[b].n_accept;
    st[b].n_reject = c[b].n_reject;
    st[b].n_rhs = c[b].n_rhs;
    st[b].t = c[b].t;
    st[b].h = c[b].h;
    st[b].tau = c[b].tau;
    st[b].status = c[b].status;
    st[b].pad = 0;
  }
}

void plan_host(const mt_integrator *I, SimCtl &c) {
  double hs = c.h;
  if (I->o.fixed_h <= 0.0 && I->o.hmax > 0.0 && hs > I->o.hmax) hs = I->o.hmax;
  c.clipped = 0;
  if (c.t + hs >= c.t_next) {
    hs = c.t_next - c.t;
    c.clipped = 1;
  }
  c.hs = hs;
}

// The one-kernel path in launches of at most kSmallChunk attempts, so that
// no launch runs for long; between them the host reads the number of
// unfinished simulations (and stops on a device timeout).
constexpr int64_t kSmallChunk = 4096;

mt_status small_steps(mt_integrator *I, int init, int64_t nsteps) {
  for (int64_t done = 0; done < nsteps || init;) {
    const int64_t todo = std::min<int64_t>(kSmallChunk, nsteps - done);
    mt_status st = launch_small(I, init, todo);
    if (st != MT_OK) return st;
    init = 0;
    done += todo;
  }
  return MT_OK;
}

mt_status small_until_done(mt_integrator *I, int64_t max_attempts) {
  int init = 1;
  for (int64_t done = 0;;) {
    const int64_t todo = std::min<int64_t>(kSmallChunk, max_attempts - done);
    mt_status st = launch_small(I, init, todo);
    if (st != MT_OK) return st;
    init = 0;
    done += todo;
    int h[2] = {0, 0};
    MT_CUDA(cudaMemcpyAsync(&h[0], I->n_active, sizeof(int), cudaMemcpyDeviceToHost, I->stream));
    MT_CUDA(cudaMemcpyAsync(&h[1], I->T->tiles->ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, I->stream));
    MT_CUDA(cudaStreamSynchronize(I->stream));
    if (h[0] == 0 || h[1] != 0 || done >= max_attempts) return MT_OK;
  }
}

// Replay the step graph until every simulation is finished (or a cap).
mt_status replay_until_done(mt_integrator *I, int64_t max_launches) {
  int64_t launched = 0;
  int chunk = 2;
  int slot = 0;
  bool pending[2] = {false, false};
  for (;;) {
    const int64_t todo = std::min<int64_t>(chunk, max_launches - launched);
    for (int64_t q = 0; q < todo; ++q) MT_CUDA(cudaGraphLaunch(I->exec, I->stream));
    launched += todo;
    MT_CUDA(cudaMemcpyAsync(&I->h_poll[slot], I->n_active, sizeof(int), cudaMemcpyDeviceToHost, I->stream));
    MT_CUDA(cudaEventRecord(I->ev[slot], I->stream));
    pending[slot] = true;
    const int prev = slot ^ 1;
    if (pending[prev]) {
      MT_CUDA(cudaEventSynchronize(I->ev[prev]));
      pending[prev] = false;
      if (I->h_poll[prev] == 0) break;
    }
    if (launched >= max_launches) {
      MT_CUDA(cudaEventSynchronize(I->ev[slot]));
      break;
    }
    slot = prev;
    if (chunk < 64) chunk *= 2;
  }
  MT_CUDA(cudaStreamSynchronize(I->stream));
  return MT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" {

mt_status mt_integrator_create(mt_tensor *T, const mt_llg_params *p, const mt_ode_opts *o, int B, void *stream,
                               mt_integrator **out) {
  MT_CHECK(T && p && o && out, MT_EINVAL, "mt_integrator_create: NULL argument");
  MT_CHECK(B >= 1 && B <= 4096, MT_EINVAL, "mt_integrator_create: B must be in [1, 4096]");
  MT_CHECK(T->prec != MT_F64, MT_EINVAL, "mt_integrator_create: the FP64 tensor serves field checks only");
  MT_CHECK(p->alpha && p->Ha, MT_EINVAL, "mt_integrator_create: alpha/Ha arrays required");
  MT_CHECK(o->fixed_h > 0.0 || (o->rtol > 0.0 && o->atol > 0.0 && o->h0 > 0.0), MT_EINVAL,
           "mt_integrator_create: rtol, atol and h0 must be positive");
  MT_CHECK(o->max_steps > 0, MT_EINVAL, "mt_integrator_create: max_steps must be positive");
  for (int b = 0; b < B; ++b)
    MT_CHECK(std::isfinite(p->alpha[b]) && std::isfinite(p->Ha[3 * b]) && std::isfinite(p->Ha[3 * b + 1]) &&
                 std::isfinite(p->Ha[3 * b + 2]),
             MT_EINVAL, "mt_integrator_create: non-finite parameter");
  MT_CUDA(cudaSetDevice(T->tiles->ctx->device));
  mt_integrator *I = new mt_integrator();
  I->T = T;
  T->refs++;
  I->B = B;
  I->user_stream = (cudaStream_t)stream;
  if (cudaStreamCreateWithFlags(&I->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&I->order_ev, cudaEventDisableTiming) != cudaSuccess) {
    mt_integrator_destroy(I);
    mt::set_error("mt_integrator_create: stream/event creation failed");
    return MT_ECUDA;
  }
  I->o = *o;
  I->form = p->form;
  I->precess = p->precess;
  I->gamma = p->gamma;
  const int64_t n = T->n;
  const size_t vec = sizeof(float) * 3 * n * B;
  I->nblk = (int)((n + kStageThreads - 1) / kStageThreads);
  mt_status st = MT_OK;
#define MT_TRY(x)              \
  do {                         \
    if ((st = (x)) != MT_OK) { \
      mt_integrator_destroy(I); \
      return st;               \
    }                          \
  } while (0)
  MT_TRY(dalloc(I, &I->y, vec));
  MT_TRY(dalloc(I, &I->ys0, vec));
  MT_TRY(dalloc(I, &I->ys1, vec));
  MT_TRY(dalloc(I, &I->Hd, vec));
  for (int s = 0; s < 7; ++s) MT_TRY(dalloc(I, &I->k[s], vec));
  const bool dense = T->layout == MT_LAYOUT_DENSE;
  if (dense) {
    MT_TRY(dalloc(I, (unsigned char **)&I->xs, mt::dense_x_bytes(T, B)));
    MT_TRY(mt::gemm_plan(T, B, I->xs, &I->plan));
  } else {
    MT_TRY(dalloc(I, &I->xs, sizeof(float) * mt::xs_floats(T) * B));
  }
  MT_TRY(dalloc(I, &I->g1, sizeof(float) * B));
  MT_TRY(dalloc(I, &I->g2, sizeof(float) * B));
  MT_TRY(dalloc(I, &I->Ha, sizeof(float) * 3 * B));
  MT_TRY(dalloc(I, &I->xsc, sizeof(float) * B));
  MT_TRY(dalloc(I, &I->part, dense ? mt::dense_part_bytes(T, B) : mt::matvec_part_bytes(T)));
  MT_TRY(dalloc(I, &I->count, dense ? mt::dense_count_bytes(T) : mt::matvec_count_bytes(T, B)));
  if (!dense && T->L.half) MT_TRY(dalloc(I, &I->colpart, mt::matvec_colpart_bytes(T, B)));
  MT_TRY(dalloc(I, &I->ctl, sizeof(SimCtl) * B));
  MT_TRY(dalloc(I, &I->active, sizeof(int) * B));
  MT_TRY(dalloc(I, &I->n_active, sizeof(int)));
  MT_TRY(dalloc(I, &I->red, sizeof(float) * 5 * I->nblk * B));
  MT_TRY(dalloc(I, &I->red_count, sizeof(int) * B));
  I->mavg_cap = 1;
  MT_TRY(dalloc(I, &I->mavg, sizeof(double) * 3 * B));
  I->small_ok = small_plan(I);
  if (I->small_ok) {
    MT_TRY(dalloc(I, &I->sm_xg, 2 * vec));
    MT_TRY(dalloc(I, &I->sm_part, sizeof(float) * 5 * I->small_G * B));
    MT_TRY(dalloc(I, &I->sm_bar, (kBarWords + kBarLine) * sizeof(unsigned long long)));
    I->path = MT_PATH_PERSISTENT;
  }
  if (cudaMallocHost(&I->h_poll, 2 * sizeof(int)) != cudaSuccess) {
    mt_integrator_destroy(I);
    mt::set_error("mt_integrator_create: pinned allocation failed");
    return MT_ENOMEM;
  }
  if (cudaEventCreateWithFlags(&I->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&I->ev[1], cudaEventDisableTiming) != cudaSuccess) {
    mt_integrator_destroy(I);
    mt::set_error("mt_integrator_create: event creation failed");
    return MT_ECUDA;
  }
  MT_TRY(mt_integrator_set_params(I, p));
  if (dense) MT_TRY(mt::gemm_tune(T, &I->plan, I->Hd, I->part, I->count, T->tiles->ctx->d_status, I->stream));
  // capture one attempt
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(I->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_attempt(I);
    e = cudaStreamEndCapture(I->stream, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&I->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    mt_integrator_destroy(I);
    return mt::cuda_fail(e, "graph capture", __FILE__, __LINE__);
  }
#undef MT_TRY
  *out = I;
  return MT_OK;
}

void mt_integrator_destroy(mt_integrator *I) {
  if (!I) return;
  if (I->stream) cudaStreamSynchronize(I->stream);
  if (I->exec) cudaGraphExecDestroy(I->exec);
  for (void *p : I->allocs) cudaFree(p);
  if (I->h_poll) cudaFreeHost(I->h_poll);
  if (I->h_slot_par) cudaFreeHost(I->h_slot_par);
  for (auto &e : I->ev)
    if (e) cudaEventDestroy(e);
  if (I->order_ev) cudaEventDestroy(I->order_ev);
  if (I->stream) cudaStreamDestroy(I->stream);
  mt::tensor_release(I->T);
  delete I;
}

mt_status mt_integrator_set_params(mt_integrator *I, const mt_llg_params *p) {
  MT_CHECK(I && p && p->alpha && p->Ha, MT_EINVAL, "mt_integrator_set_params: NULL argument");
  std::vector<float> g1, g2, ha, xsc;
  mt::llg_prefactors(p, I->B, g1, g2, ha, xsc);
  for (int b = 0; b < I->B; ++b)
    MT_CHECK(std::isfinite(xsc[b]) && xsc[b] >= 0.0f, MT_EINVAL, "mt_integrator_set_params: bad exch_scale");
  MT_CUDA(cudaMemcpyAsync(I->g1, g1.data(), sizeof(float) * I->B, cudaMemcpyHostToDevice, I->stream));
  MT_CUDA(cudaMemcpyAsync(I->g2, g2.data(), sizeof(float) * I->B, cudaMemcpyHostToDevice, I->stream));
  MT_CUDA(cudaMemcpyAsync(I->Ha, ha.data(), sizeof(float) * 3 * I->B, cudaMemcpyHostToDevice, I->stream));
  MT_CUDA(cudaMemcpyAsync(I->xsc, xsc.data(), sizeof(float) * I->B, cudaMemcpyHostToDevice, I->stream));
  MT_CUDA(cudaStreamSynchronize(I->stream));
  I->need_init = true;
  return MT_OK;
}

mt_status mt_integrator_set_state(mt_integrator *I, const float *m, int m_is_host, double t0) {
  MT_CHECK(I && m, MT_EINVAL, "mt_integrator_set_state: NULL argument");
  const size_t bytes = sizeof(float) * 3 * I->T->n * I->B;
  if (!m_is_host) {  // the caller's stream may still be writing m
    MT_CUDA(cudaEventRecord(I->order_ev, I->user_stream));
    MT_CUDA(cudaStreamWaitEvent(I->stream, I->order_ev, 0));
  }
  MT_CUDA(cudaMemcpyAsync(I->y, m, bytes, m_is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                          I->stream));
  std::vector<SimCtl> c(I->B);
  for (auto &x : c) {
    std::memset(&x, 0, sizeof(SimCtl));
    x.t = t0;
    x.h = I->o.fixed_h > 0 ? I->o.fixed_h : I->o.h0;
    x.t_next = 1e300;
    x.mode = MODE_STEPS;
    x.status = MT_OK;
    x.attempt_cap = INT64_MAX;
  }
  for (auto &x : c) plan_host(I, x);
  // write_ctl synchronises, which also orders the state copy
  mt_status st = write_ctl(I, c);
  if (st != MT_OK) return st;
  I->need_init = true;
  return MT_OK;
}

mt_status mt_integrator_get_state(mt_integrator *I, float *m, int m_is_host) {
  MT_CHECK(I && m, MT_EINVAL, "mt_integrator_get_state: NULL argument");
  const size_t bytes = sizeof(float) * 3 * I->T->n * I->B;
  MT_CUDA(cudaMemcpyAsync(m, I->y, bytes, m_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                          I->stream));
  if (m_is_host) {
    MT_CUDA(cudaStreamSynchronize(I->stream));
  } else {  // later work on the caller's stream sees the copy
    MT_CUDA(cudaEventRecord(I->order_ev, I->stream));
    MT_CUDA(cudaStreamWaitEvent(I->user_stream, I->order_ev, 0));
  }
  return MT_OK;
}

void *mt_integrator_stream(mt_integrator *I) { return I ? (void *)I->stream : nullptr; }

mt_status mt_integrator_set_path(mt_integrator *I, int path) {
  MT_CHECK(I, MT_EINVAL, "mt_integrator_set_path: NULL integrator");
  MT_CHECK(path == MT_PATH_GRAPH || path == MT_PATH_PERSISTENT, MT_EINVAL, "mt_integrator_set_path: unknown path %d",
           path);
  MT_CHECK(path == MT_PATH_GRAPH || I->small_ok, MT_EINVAL,
           "mt_integrator_set_path: the one-kernel path needs an FP32 streaming tensor of a small tile set");
  // both paths leave the state committed between calls (y and k1 current)
  MT_CUDA(cudaStreamSynchronize(I->stream));
  I->path = path;
  return MT_OK;
}

int mt_integrator_get_path(mt_integrator *I) { return I ? I->path : 0; }

mt_status mt_selftest_grid_barrier_timeout(mt_ctx *ctx) {
  MT_CHECK(ctx, MT_EINVAL, "mt_selftest_grid_barrier_timeout: NULL context");
  MT_CUDA(cudaSetDevice(ctx->device));
  unsigned long long *words = nullptr;
  const size_t bytes = (kBarWords + kBarLine) * sizeof(unsigned long long) + sizeof(int);
  MT_CUDA(cudaMalloc(&words, bytes));
  cudaError_t e = cudaMemset(words, 0, bytes);
  SmallArgs S{};
  S.bar = words;
  S.abort_flag = reinterpret_cast<int *>(words + kBarWords);
  S.status = reinterpret_cast<int *>(words + kBarWords + kBarLine);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(4);
    cfg.blockDim = dim3(32);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_barrier_selftest, S);
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, S.status, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(words);
  if (e != cudaSuccess) return mt::cuda_fail(e, "mt_selftest_grid_barrier_timeout", __FILE__, __LINE__);
  if (h == MT_DEV_TIMEOUT) {
    mt::set_error("mt_selftest_grid_barrier_timeout: the bounded barrier gave up as designed");
    return MT_ETIMEOUT;
  }
  mt::set_error("mt_selftest_grid_barrier_timeout: the barrier did not report a timeout");
  return MT_ECUDA;
}

mt_status mt_integrator_step(mt_integrator *I, int64_t nsteps) {
  MT_CHECK(I && nsteps >= 0, MT_EINVAL, "mt_integrator_step: bad argument");
  if (I->need_init) {
    // fixed number of attempts: no time target, every simulation active
    std::vector<SimCtl> c;
    mt_status st = read_ctl(I, c);
    if (st != MT_OK) return st;
    for (auto &x : c) {
      x.mode = MODE_STEPS;
      x.t_next = 1e300;
      x.done = 0;
      x.status = MT_OK;
      plan_host(I, x);
    }
    if ((st = write_ctl(I, c)) != MT_OK) return st;
    if (I->path == MT_PATH_PERSISTENT) return small_steps(I, 1, nsteps);
    if ((st = enqueue_init(I)) != MT_OK) return st;
  }
  if (I->path == MT_PATH_PERSISTENT) return small_steps(I, 0, nsteps);
  for (int64_t q = 0; q < nsteps; ++q) MT_CUDA(cudaGraphLaunch(I->exec, I->stream));
  return enqueue_commit(I);
}

// cap_ok: in relax mode a simulation that reached its time cap with the
// torque above tol counts as finished (hysteresis values)
static mt_status run_common(mt_integrator *I, int mode, double t1, int64_t n_out, double tol, double *mavg,
                            mt_stats *stats, bool cap_ok = false, std::vector<SimCtl> *out_ctl = nullptr) {
  std::vector<SimCtl> c;
  mt_status st = read_ctl(I, c);
  if (st != MT_OK) return st;
  if (mode == MODE_RUN && n_out > I->mavg_cap) {
    cudaFree(I->mavg);
    I->allocs.erase(std::remove(I->allocs.begin(), I->allocs.end(), (void *)I->mavg), I->allocs.end());
    I->mavg = nullptr;
    if ((st = dalloc(I, &I->mavg, sizeof(double) * 3 * I->B * n_out)) != MT_OK) return st;
    I->mavg_cap = n_out;
    // the graph bakes the output pointer in: recapture
    cudaGraphExecDestroy(I->exec);
    I->exec = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(I->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      enqueue_attempt(I);
      e = cudaStreamEndCapture(I->stream, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&I->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return mt::cuda_fail(e, "graph capture", __FILE__, __LINE__);
  }
  for (auto &x : c) {
    x.mode = mode;
    x.done = 0;
    x.status = MT_OK;
    x.accepted = 0;
    x.attempt_cap = x.n_attempt + I->o.max_steps;
    if (mode == MODE_RUN) {
      x.n_out = n_out;
      x.iout = 0;
      x.t1 = t1;
      x.t_out0 = x.t;
      x.dt_out = (t1 - x.t) / (double)n_out;
      x.t_next = (n_out == 1) ? t1 : x.t + x.dt_out;
    } else {
      x.tol = tol;
      x.t1 = x.t + t1;
      x.t_next = x.t1;
    }
    plan_host(I, x);
  }
  if ((st = write_ctl(I, c)) != MT_OK) return st;
  if (I->path == MT_PATH_PERSISTENT) {
    if ((st = small_until_done(I, I->o.max_steps + 2)) != MT_OK) return st;
  } else {
    if ((st = enqueue_init(I)) != MT_OK) return st;
    if ((st = replay_until_done(I, I->o.max_steps + 2)) != MT_OK) return st;
    if ((st = enqueue_commit(I)) != MT_OK) return st;
  }
  if ((st = read_ctl(I, c)) != MT_OK) return st;
  int dev_status = 0;
  MT_CUDA(cudaMemcpy(&dev_status, I->T->tiles->ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  MT_CHECK(dev_status == 0, MT_ETIMEOUT, "integrator: a bounded device wait ran out");
  if (mavg && mode == MODE_RUN) {
    MT_CUDA(cudaMemcpy(mavg, I->mavg, sizeof(double) * 3 * I->B * n_out, cudaMemcpyDeviceToHost));
  }
  fill_stats(c, stats, I->B);
  if (out_ctl) *out_ctl = c;
  for (int b = 0; b < I->B; ++b) {
    if (!c[b].done) {
      mt::set_error("integrator: simulation %d not finished", b);
      return MT_ENOCONV;
    }
    if (cap_ok && c[b].status == MT_ENOCONV && c[b].t >= c[b].t1) continue;
    if (c[b].status != MT_OK) {
      mt::set_error("integrator: simulation %d ended with status %d", b, c[b].status);
      return (mt_status)c[b].status;
    }
  }
  return MT_OK;
}

mt_status mt_integrator_run(mt_integrator *I, double t1, int64_t n_out, double *mavg, mt_stats *stats) {
  MT_CHECK(I && n_out >= 1, MT_EINVAL, "mt_integrator_run: bad argument");
  return run_common(I, MODE_RUN, t1, n_out, 0.0, mavg, stats);
}

mt_status mt_integrator_relax(mt_integrator *I, double tol, double t_max, mt_stats *stats) {
  MT_CHECK(I && tol > 0 && t_max > 0, MT_EINVAL, "mt_integrator_relax: bad argument");
  return run_common(I, MODE_RELAX, t_max, 1, tol, nullptr, stats);
}

mt_status mt_integrator_hysteresis(mt_integrator *I, const double *dir, const double *H, int64_t S, double t_step,
                                   double tol, double *mavg, double *tau, double *hc, double *mr, mt_stats *stats) {
  MT_CHECK(I && dir && H && S >= 1 && t_step > 0 && tol >= 0, MT_EINVAL, "mt_integrator_hysteresis: bad argument");
  const int B = I->B;
  std::vector<double> d(3 * B);
  for (int b = 0; b < B; ++b) {
    const double nrm = std::sqrt(dir[3 * b] * dir[3 * b] + dir[3 * b + 1] * dir[3 * b + 1] +
                                 dir[3 * b + 2] * dir[3 * b + 2]);
    MT_CHECK(std::isfinite(nrm) && nrm > 0, MT_EINVAL, "mt_integrator_hysteresis: direction %d is zero", b);
    for (int c = 0; c < 3; ++c) d[3 * b + c] = dir[3 * b + c] / nrm;
  }
  for (int64_t s = 0; s < S; ++s)
    MT_CHECK(std::isfinite(H[s]), MT_EINVAL, "mt_integrator_hysteresis: non-finite field value");
  std::vector<double> pm(3 * B * (size_t)S), pt(B * (size_t)S);
  std::vector<float> ha(3 * B);
  std::vector<SimCtl> c;
  mt_status st0 = read_ctl(I, c);
  if (st0 != MT_OK) return st0;
  double t_end = 0.0;  // fixed-time values: every simulation ends on the same times
  for (int b = 0; b < B; ++b) t_end = std::max(t_end, c[b].t);
  for (int64_t s = 0; s < S; ++s) {
    for (int q = 0; q < 3 * B; ++q) ha[q] = (float)(H[s] * d[q]);
    MT_CUDA(cudaMemcpyAsync(I->Ha, ha.data(), sizeof(float) * 3 * B, cudaMemcpyHostToDevice, I->stream));
    MT_CUDA(cudaStreamSynchronize(I->stream));
    I->need_init = true;  // k1 belongs to the previous field
    t_end += t_step;
    mt_status st = tol > 0 ? run_common(I, MODE_RELAX, t_step, 1, tol, nullptr, stats, true, &c)
                           : run_common(I, MODE_RUN, t_end, 1, 0.0, nullptr, stats, false, &c);
    if (st != MT_OK) return st;
    for (int b = 0; b < B; ++b) {
      for (int q = 0; q < 3; ++q) pm[((size_t)s * B + b) * 3 + q] = c[b].m_last[q];
      pt[(size_t)s * B + b] = c[b].tau;
    }
  }
  if (mavg) std::memcpy(mavg, pm.data(), sizeof(double) * pm.size());
  if (tau) std::memcpy(tau, pt.data(), sizeof(double) * pt.size());
  const double nan = std::numeric_limits<double>::quiet_NaN();
  for (int b = 0; b < B; ++b) {
    auto proj = [&](int64_t s) {
      const double *m = &pm[((size_t)s * B + b) * 3];
      return m[0] * d[3 * b] + m[1] * d[3 * b + 1] + m[2] * d[3 * b + 2];
    };
    if (hc) {
      hc[b] = nan;
      for (int64_t s = 1; s < S; ++s) {
        const double p0 = proj(s - 1), p1 = proj(s);
        if (p0 > 0 && p1 <= 0) {
          hc[b] = H[s - 1] + (H[s] - H[s - 1]) * p0 / (p0 - p1);
          break;
        }
      }
    }
    if (mr) {
      for (int q = 0; q < 3; ++q) mr[3 * b + q] = nan;
      for (int64_t s = 1; s < S; ++s) {
        if (H[s - 1] >= 0 && H[s] <= 0 && H[s - 1] != H[s]) {
          const double w = H[s - 1] / (H[s - 1] - H[s]);
          for (int q = 0; q < 3; ++q)
            mr[3 * b + q] = (1 - w) * pm[((size_t)(s - 1) * B + b) * 3 + q] + w * pm[((size_t)s * B + b) * 3 + q];
          break;
        }
      }
    }
  }
  return MT_OK;
}

mt_status mt_integrator_crossover(mt_integrator *I, const double *lam, int K, const float *mA, const float *mB,
                                  double tol, double t_max, double *eA, double *eB, double *lam_cross,
                                  float *m_out, mt_stats *stats) {
  MT_CHECK(I && lam && mA && mB && K >= 1 && tol > 0 && t_max > 0, MT_EINVAL,
           "mt_integrator_crossover: bad argument");
  MT_CHECK(I->B == 2 * K, MT_EINVAL, "mt_integrator_crossover: the integrator must hold 2K = %d simulations", 2 * K);
  for (int k = 0; k < K; ++k)
    MT_CHECK(std::isfinite(lam[k]) && lam[k] > 0, MT_EINVAL, "mt_integrator_crossover: sizes must be positive");
  const int64_t n = I->T->n;
  const int B = I->B;
  // sizes enter as exchange factors (the point tensor is scale-invariant)
  std::vector<float> xsc(B);
  for (int k = 0; k < K; ++k) xsc[k] = xsc[K + k] = (float)(1.0 / (lam[k] * lam[k]));
  MT_CUDA(cudaMemcpyAsync(I->xsc, xsc.data(), sizeof(float) * B, cudaMemcpyHostToDevice, I->stream));
  // state: family A at every size, then family B
  std::vector<float> m0((size_t)3 * n * B);
  for (int k = 0; k < K; ++k) {
    std::memcpy(&m0[(size_t)3 * n * k], mA, sizeof(float) * 3 * n);
    std::memcpy(&m0[(size_t)3 * n * (K + k)], mB, sizeof(float) * 3 * n);
  }
  mt_status st = mt_integrator_set_state(I, m0.data(), 1, 0.0);
  if (st != MT_OK) return st;
  if ((st = run_common(I, MODE_RELAX, t_max, 1, tol, nullptr, stats, true)) != MT_OK) return st;
  // energies of the relaxed states: demag product of y for every simulation
  // (finished ones are inactive after the relaxation), then the densities
  {
    std::vector<int> act(B, 1);
    MT_CUDA(cudaMemcpyAsync(I->active, act.data(), sizeof(int) * B, cudaMemcpyHostToDevice, I->stream));
    MT_CUDA(cudaMemcpyAsync(I->n_active, &B, sizeof(int), cudaMemcpyHostToDevice, I->stream));
    MT_CUDA(cudaStreamSynchronize(I->stream));
  }
  double *d_E = nullptr;
  MT_CUDA(cudaMalloc(&d_E, sizeof(double) * 4 * B));
  cudaError_t e = cudaMemsetAsync(d_E, 0, sizeof(double) * 4 * B, I->stream);
  if (e == cudaSuccess) {
    if (I->T->layout == MT_LAYOUT_DENSE)
      mt::launch_prep_dense_x(I->T, I->y, B, I->xs, I->stream);
    else
      mt::launch_prep_xs(I->T, I->y, B, I->xs, I->stream);
    demag(I, I->y);
    mt::launch_energy(I->T, I->y, I->Hd, B, I->Ha, I->xsc, d_E, I->stream);
    e = cudaGetLastError();
  }
  std::vector<double> e4(4 * B);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(e4.data(), d_E, sizeof(double) * 4 * B, cudaMemcpyDeviceToHost, I->stream);
  if (e == cudaSuccess && m_out)
    e = cudaMemcpyAsync(m_out, I->y, sizeof(float) * 3 * n * B, cudaMemcpyDeviceToHost, I->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(I->stream);
  cudaFree(d_E);
  if (e != cudaSuccess) return mt::cuda_fail(e, "mt_integrator_crossover", __FILE__, __LINE__);
  I->need_init = true;  // the workspace now holds the relaxed state's product
  const double vol = I->T->tiles->vol_total;
  std::vector<double> ea(K), eb(K);
  for (int k = 0; k < K; ++k) {
    ea[k] = (e4[4 * k] + e4[4 * k + 1] + e4[4 * k + 2] + e4[4 * k + 3]) / vol;
    eb[k] = (e4[4 * (K + k)] + e4[4 * (K + k) + 1] + e4[4 * (K + k) + 2] + e4[4 * (K + k) + 3]) / vol;
  }
  if (eA) std::memcpy(eA, ea.data(), sizeof(double) * K);
  if (eB) std::memcpy(eB, eb.data(), sizeof(double) * K);
  if (lam_cross) {
    *lam_cross = std::numeric_limits<double>::quiet_NaN();
    for (int k = 1; k < K; ++k) {
      const double d0 = ea[k - 1] - eb[k - 1], d1 = ea[k] - eb[k];
      if ((d0 < 0) != (d1 < 0)) {
        *lam_cross = lam[k - 1] + (lam[k] - lam[k - 1]) * d0 / (d0 - d1);
        break;
      }
    }
  }
  return MT_OK;
}

mt_status mt_integrator_stats(mt_integrator *I, mt_stats *stats) {
  MT_CHECK(I && stats, MT_EINVAL, "mt_integrator_stats: NULL argument");
  std::vector<SimCtl> c;
  mt_status st = read_ctl(I, c);
  if (st != MT_OK) return st;
  fill_stats(c, stats, I->B);
  return MT_OK;
}

// ---------------------------------------------------------------------------
// checkpoint / resume: header | SimCtl[B] | m[3nB] | k1[3nB] | FNV-1a 64
// ---------------------------------------------------------------------------
namespace {

struct CkptHeader {
  char magic[8];
  uint32_t version;
  uint32_t k1_valid;  // the saved derivative belongs to the saved m
  int64_t n;
  int32_t B;
  int32_t prec;
  int32_t layout;
  uint32_t ctl_bytes;  // sizeof(SimCtl) of the writer
};
constexpr char kCkptMagic[8] = {'M', 'T', 'C', 'K', 'P', 'T', '0', '1'};
constexpr uint32_t kCkptVersion = 1;

uint64_t fnv1a64(const unsigned char *p, size_t len) {
  uint64_t h = 1469598103934665603ull;
  for (size_t q = 0; q < len; ++q) {
    h ^= p[q];
    h *= 1099511628211ull;
  }
  return h;
}

size_t ckpt_bytes(const mt_integrator *I) {
  const size_t state = sizeof(float) * 3 * (size_t)I->T->n * I->B;
  return sizeof(CkptHeader) + sizeof(SimCtl) * I->B + 2 * state + sizeof(uint64_t);
}

}  // namespace

mt_status mt_integrator_checkpoint_bytes(mt_integrator *I, size_t *bytes) {
  MT_CHECK(I && bytes, MT_EINVAL, "mt_integrator_checkpoint_bytes: NULL argument");
  *bytes = ckpt_bytes(I);
  return MT_OK;
}

mt_status mt_integrator_checkpoint(mt_integrator *I, void *buf, size_t bytes) {
  MT_CHECK(I && buf, MT_EINVAL, "mt_integrator_checkpoint: NULL argument");
  const size_t need = ckpt_bytes(I);
  MT_CHECK(bytes >= need, MT_EINVAL, "mt_integrator_checkpoint: buffer of %zu bytes, %zu needed", bytes, need);
  unsigned char *p = static_cast<unsigned char *>(buf);
  CkptHeader h{};
  std::memcpy(h.magic, kCkptMagic, sizeof(h.magic));
  h.version = kCkptVersion;
  h.k1_valid = I->need_init ? 0u : 1u;
  h.n = I->T->n;
  h.B = I->B;
  h.prec = I->T->prec;
  h.layout = I->T->layout;
  h.ctl_bytes = (uint32_t)sizeof(SimCtl);
  std::memcpy(p, &h, sizeof(h));
  std::vector<SimCtl> c;
  mt_status st = read_ctl(I, c);  // also orders after every queued step
  if (st != MT_OK) return st;
  // every public call ends with the commit of the last accepted attempt
  // (m and k1 already hold it), so the flag that asks the next begin to
  // adopt it again is dropped: the next attempt starts from the same bits
  for (auto &x : c) x.accepted = 0;
  unsigned char *q = p + sizeof(h);
  std::memcpy(q, c.data(), sizeof(SimCtl) * I->B);
  q += sizeof(SimCtl) * I->B;
  const size_t state = sizeof(float) * 3 * (size_t)I->T->n * I->B;
  MT_CUDA(cudaMemcpyAsync(q, I->y, state, cudaMemcpyDeviceToHost, I->stream));
  MT_CUDA(cudaMemcpyAsync(q + state, I->k[0], state, cudaMemcpyDeviceToHost, I->stream));
  MT_CUDA(cudaStreamSynchronize(I->stream));
  q += 2 * state;
  const uint64_t sum = fnv1a64(p, (size_t)(q - p));
  std::memcpy(q, &sum, sizeof(sum));
  return MT_OK;
}

mt_status mt_integrator_restore(mt_integrator *I, const void *buf, size_t bytes) {
  MT_CHECK(I && buf, MT_EINVAL, "mt_integrator_restore: NULL argument");
  const unsigned char *p = static_cast<const unsigned char *>(buf);
  MT_CHECK(bytes >= sizeof(CkptHeader), MT_EINVAL, "mt_integrator_restore: %zu bytes is no checkpoint", bytes);
  CkptHeader h;
  std::memcpy(&h, p, sizeof(h));
  MT_CHECK(std::memcmp(h.magic, kCkptMagic, sizeof(h.magic)) == 0 && h.version == kCkptVersion &&
               h.ctl_bytes == sizeof(SimCtl),
           MT_EINVAL, "mt_integrator_restore: not a checkpoint of this format version");
  MT_CHECK(h.n == I->T->n && h.B == I->B, MT_EINVAL,
           "mt_integrator_restore: checkpoint of n = %lld, B = %d into an integrator of n = %lld, B = %d",
           (long long)h.n, h.B, (long long)I->T->n, I->B);
  const size_t need = ckpt_bytes(I);
  MT_CHECK(bytes >= need, MT_EINVAL, "mt_integrator_restore: %zu bytes, %zu expected", bytes, need);
  uint64_t sum;
  std::memcpy(&sum, p + need - sizeof(sum), sizeof(sum));
  MT_CHECK(sum == fnv1a64(p, need - sizeof(sum)), MT_EINVAL, "mt_integrator_restore: checksum mismatch");
  std::vector<SimCtl> c(I->B);
  const unsigned char *q = p + sizeof(h);
  std::memcpy(c.data(), q, sizeof(SimCtl) * I->B);
  q += sizeof(SimCtl) * I->B;
  const size_t state = sizeof(float) * 3 * (size_t)I->T->n * I->B;
  // the state of a finished simulation is restored with it; the derivative
  // only when it was evaluated with this kind of tensor
  const bool keep_k1 = h.k1_valid && h.prec == I->T->prec && h.layout == I->T->layout;
  MT_CUDA(cudaMemcpyAsync(I->y, q, state, cudaMemcpyHostToDevice, I->stream));
  if (keep_k1) MT_CUDA(cudaMemcpyAsync(I->k[0], q + state, state, cudaMemcpyHostToDevice, I->stream));
  mt_status st = write_ctl(I, c);  // synchronises: the host image may go after this
  if (st != MT_OK) return st;
  I->need_init = !keep_k1;
  return MT_OK;
}

mt_status mt_integrate(mt_tensor *T, const mt_llg_params *p, const mt_ode_opts *o, float *m, int B, double t0,
                       double t1, int64_t n_out, double *mavg, mt_stats *stats, void *stream) {
  mt_integrator *I = nullptr;
  mt_status st = mt_integrator_create(T, p, o, B, stream, &I);
  if (st != MT_OK) return st;
  st = mt_integrator_set_state(I, m, 0, t0);
  mt_status st2 = (st == MT_OK) ? mt_integrator_run(I, t1, n_out, mavg, stats) : st;
  if (st == MT_OK) st = mt_integrator_get_state(I, m, 0);
  if (st == MT_OK) {
    cudaError_t e = cudaStreamSynchronize(I->stream);
    if (e != cudaSuccess) st = mt::cuda_fail(e, "sync", __FILE__, __LINE__);
  }
  mt_integrator_destroy(I);
  return st2 != MT_OK ? st2 : st;
}

mt_status mt_relax(mt_tensor *T, const mt_llg_params *p, const mt_ode_opts *o, double tol, double t_max, float *m,
                   int B, mt_stats *stats, void *stream) {
  mt_integrator *I = nullptr;
  mt_status st = mt_integrator_create(T, p, o, B, stream, &I);
  if (st != MT_OK) return st;
  st = mt_integrator_set_state(I, m, 0, 0.0);
  mt_status st2 = (st == MT_OK) ? mt_integrator_relax(I, tol, t_max, stats) : st;
  if (st == MT_OK) st = mt_integrator_get_state(I, m, 0);
  if (st == MT_OK) {
    cudaError_t e = cudaStreamSynchronize(I->stream);
    if (e != cudaSuccess) st = mt::cuda_fail(e, "sync", __FILE__, __LINE__);
  }
  mt_integrator_destroy(I);
  return st2 != MT_OK ? st2 : st;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// slot-level control used by the serving loop (one simulation per slot,
// admitted and retired while the others keep running)
// ---------------------------------------------------------------------------
namespace mt {

size_t integ_ctl_bytes(const mt_integrator *I) { return sizeof(SimCtl) * I->B; }
int integ_batch(const mt_integrator *I) { return I->B; }
void *integ_stream(const mt_integrator *I) { return I->stream; }

// Enqueue the admission of one simulation into slot b: its state (host,
// 3n floats, must stay valid until the stream reaches the copy), its
// equation parameters, and a relax goal (torque < tol, time cap t_max).
mt_status integ_admit(mt_integrator *I, int b, const float *m0_host, double alpha, const double *Ha, double tol,
                      double t_max) {
  MT_CHECK(b >= 0 && b < I->B, MT_EINVAL, "slot %d out of range", b);
  const int64_t n = I->T->n;
  MT_CUDA(cudaMemcpyAsync(I->y + (size_t)b * 3 * n, m0_host, sizeof(float) * 3 * n, cudaMemcpyHostToDevice,
                          I->stream));
  const double a = alpha;
  double G1, G2;
  if (I->form == MT_FORM_GILBERT) {
    G1 = I->gamma / (1.0 + a * a);
    G2 = G1 * a;
  } else {
    G1 = I->gamma;
    G2 = a;
  }
  if (!I->precess) G1 = 0.0;
  // pinned staging: slot b's entries are reused only after its previous
  // simulation finished, i.e. after the stream consumed them
  float *par = I->h_slot_par + 5 * b;
  par[0] = (float)G1;
  par[1] = (float)G2;
  par[2] = (float)Ha[0];
  par[3] = (float)Ha[1];
  par[4] = (float)Ha[2];
  MT_CUDA(cudaMemcpyAsync(I->g1 + b, par, sizeof(float), cudaMemcpyHostToDevice, I->stream));
  MT_CUDA(cudaMemcpyAsync(I->g2 + b, par + 1, sizeof(float), cudaMemcpyHostToDevice, I->stream));
  MT_CUDA(cudaMemcpyAsync(I->Ha + 3 * b, par + 2, 3 * sizeof(float), cudaMemcpyHostToDevice, I->stream));
  SimCtl c;
  std::memset(&c, 0, sizeof(c));
  c.t = 0.0;
  c.h = I->o.fixed_h > 0 ? I->o.fixed_h : I->o.h0;
  c.mode = MODE_RELAX;
  c.tol = tol;
  c.t1 = t_max;
  c.t_next = t_max;
  c.attempt_cap = I->o.max_steps;
  c.status = MT_OK;
  c.fresh = 1;
  plan_host(I, c);
  k_admit<<<1, 1, 0, I->stream>>>(I->ctl, I->active, I->n_active, b, c);
  MT_CUDA(cudaGetLastError());
  return MT_OK;
}

// Enqueue the next leg of slot b's simulation from the state it holds (a
// field sweep moves to its next applied field): new applied field, a fresh
// relax goal (torque < tol, time cap t_max from t = 0) and the first trial
// step h0, as a new relaxation would start; k1 is re-evaluated by the next
// integ_init_fresh.  The damping stays.
mt_status integ_readmit(mt_integrator *I, int b, const double *Ha, double tol, double t_max) {
  MT_CHECK(b >= 0 && b < I->B, MT_EINVAL, "slot %d out of range", b);
  // pinned staging: slot b's entries were consumed at its admission, which
  // the stream completed before the poll that reported the slot done
  float *par = I->h_slot_par + 5 * b;
  par[2] = (float)Ha[0];
  par[3] = (float)Ha[1];
  par[4] = (float)Ha[2];
  MT_CUDA(cudaMemcpyAsync(I->Ha + 3 * b, par + 2, 3 * sizeof(float), cudaMemcpyHostToDevice, I->stream));
  SimCtl c;
  std::memset(&c, 0, sizeof(c));
  c.t = 0.0;
  c.h = I->o.fixed_h > 0 ? I->o.fixed_h : I->o.h0;
  c.mode = MODE_RELAX;
  c.tol = tol;
  c.t1 = t_max;
  c.t_next = t_max;
  c.attempt_cap = I->o.max_steps;
  c.status = MT_OK;
  c.fresh = 1;
  plan_host(I, c);
  k_admit<<<1, 1, 0, I->stream>>>(I->ctl, I->active, I->n_active, b, c);
  MT_CUDA(cudaGetLastError());
  return MT_OK;
}

// volume-averaged m of slot b after its last accepted step, from a polled
// control copy
void integ_slot_mavg(const void *ctl_host, int b, double m[3]) {
  const SimCtl &c = reinterpret_cast<const SimCtl *>(ctl_host)[b];
  for (int q = 0; q < 3; ++q) m[q] = c.m_last[q];
}

// k1 for the freshly admitted slots (one demag product for the batch)
mt_status integ_init_fresh(mt_integrator *I) { return enqueue_init(I, 1); }

mt_status integ_replay(mt_integrator *I, int k) {
  for (int q = 0; q < k; ++q) MT_CUDA(cudaGraphLaunch(I->exec, I->stream));
  return MT_OK;
}

// commit accepted states and copy every slot's control block to ctl_host
// (pinned); `ev` is recorded after the copy
mt_status integ_poll(mt_integrator *I, void *ctl_host, cudaEvent_t ev) {
  mt_status st = enqueue_commit(I);
  if (st != MT_OK) return st;
  MT_CUDA(cudaMemcpyAsync(ctl_host, I->ctl, sizeof(SimCtl) * I->B, cudaMemcpyDeviceToHost, I->stream));
  MT_CUDA(cudaEventRecord(ev, I->stream));
  return MT_OK;
}

// read slot b of a polled control copy
bool integ_slot_done(const void *ctl_host, int b, mt_stats *st) {
  const SimCtl &c = reinterpret_cast<const SimCtl *>(ctl_host)[b];
  if (st) {
    st->n_accept = c.n_accept;
    st->n_reject = c.n_reject;
    st->n_rhs = c.n_rhs;
    st->t = c.t;
    st->h = c.h;
    st->tau = c.tau;
    st->status = c.status;
    st->pad = 0;
  }
  return c.done != 0;
}

// enqueue the copy of slot b's committed state to host memory
mt_status integ_fetch_slot(mt_integrator *I, int b, float *m_host) {
  const int64_t n = I->T->n;
  MT_CUDA(cudaMemcpyAsync(m_host, I->y + (size_t)b * 3 * n, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost,
                          I->stream));
  return MT_OK;
}

// an integrator whose slots all start empty (no active simulation)
mt_status integ_create_idle(mt_tensor *T, const mt_llg_params *p, const mt_ode_opts *o, int B,
                            mt_integrator **out) {
  mt_integrator *I = nullptr;
  mt_status st = mt_integrator_create(T, p, o, B, nullptr, &I);
  if (st != MT_OK) return st;
  I->path = MT_PATH_GRAPH;  // slots are admitted between graph replays
  std::vector<SimCtl> c(B);
  for (auto &x : c) {
    std::memset(&x, 0, sizeof(SimCtl));
    x.done = 1;
    x.status = MT_OK;
    x.t_next = 1e300;
  }
  if ((st = write_ctl(I, c)) != MT_OK) {
    mt_integrator_destroy(I);
    return st;
  }
  if (cudaMallocHost(&I->h_slot_par, sizeof(float) * 5 * B) != cudaSuccess) {
    mt_integrator_destroy(I);
    mt::set_error("serving engine: pinned allocation failed");
    return MT_ENOMEM;
  }
  I->need_init = false;
  *out = I;
  return MT_OK;
}

}  // namespace mt
