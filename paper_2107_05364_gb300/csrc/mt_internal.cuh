// Internal declarations of libmagtile: handle structs, layout constants,
// device helpers (mbarrier, bulk TMA copies, bounded waits, reductions).
// Nothing here is part of the ABI; include/mt.h is.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "mt.h"

// ---------------------------------------------------------------------------
// error handling (host)
// ---------------------------------------------------------------------------
namespace mt {

void set_error(const char *fmt, ...);
mt_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);

}  // namespace mt

#define MT_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return mt::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define MT_CHECK(cond, code, ...)      \
  do {                                 \
    if (!(cond)) {                     \
      mt::set_error(__VA_ARGS__);      \
      return (code);                   \
    }                                  \
  } while (0)

// ---------------------------------------------------------------------------
// physical constants (SI)
// ---------------------------------------------------------------------------
#define MT_PI 3.14159265358979323846
#define MT_MU0 (4.0e-7 * MT_PI)  // vacuum permeability, classical value

// device-side error codes written to a status word by bounded waits
#define MT_DEV_TIMEOUT 1

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
// Handles are reference counted: a tile set keeps its context alive, a
// tensor its tile set, an integrator its tensor, so *_destroy may be called
// in any order (the memory goes when the last user lets go).
struct mt_ctx {
  std::atomic<int> refs{1};
  int device = 0;
  int num_sms = 0;
  size_t budget = 0;
  size_t in_use = 0;
  std::mutex mu;
  int *d_status = nullptr;  // device status word for bounded waits
  // one-kernel integrator launches (cooperative grids that wait on their own
  // CTAs) are chained through this event so that two never share the SMs
  std::mutex small_mu;
  cudaEvent_t small_ev = nullptr;
};

struct mt_tiles {
  std::atomic<int> refs{1};
  mt_ctx *ctx = nullptr;
  int64_t n = 0;
  // host copies (FP64, as given)
  std::vector<double> centre, edge, Ms, Aex, Ku, axis;
  std::vector<int32_t> nbr;  // empty = no exchange
  // device copies
  double *d_centre = nullptr;  // 3n
  double *d_edge = nullptr;    // 3n
  float *d_Ms = nullptr;       // n
  float *d_wex = nullptr;      // 6n: 2A_i/(mu0 Ms_i h_i d_ip) per face, 0 if none
  int32_t *d_nbr = nullptr;    // 6n
  float *d_kan = nullptr;      // n: 2K_i/(mu0 Ms_i)
  float *d_axis = nullptr;     // 3n unit easy axis
  double *d_wvol = nullptr;    // n: V_i / sum V
  double vol_total = 0.0;      // sum V, m^3
  bool has_exchange = false;
  int kind = 0;                // MT_TILE_CUBOID or MT_TILE_TETRA
  double *d_vert = nullptr;    // 12n: the 4 vertices of each tetrahedron (kind tetra)
  // uniform cuboid lattice (equal edges, centres on c0 + index * edge): a
  // block depends only on the index offset of its two tiles, so assembly
  // evaluates one block per offset and fills the tensor from that table
  bool lattice = false;
  int32_t *d_lat = nullptr;    // 3n lattice indices
  int Lx = 0, Ly = 0, Lz = 0;  // lattice extents
  double lat_edge[3] = {0, 0, 0};
};

enum { MT_TILE_CUBOID = 0, MT_TILE_TETRA = 1 };

namespace mt {
// launch with the programmatic-stream-serialisation attribute (the kernel
// must start with mtd::pdl_enter)
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
}  // namespace mt

// Device temporary of a host function, freed when the function returns (on
// the error paths of MT_CUDA / MT_CHECK too).
template <typename T>
struct DevTemp {
  T *p = nullptr;
  DevTemp() = default;
  DevTemp(const DevTemp &) = delete;
  DevTemp &operator=(const DevTemp &) = delete;
  ~DevTemp() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t count) { return cudaMalloc(reinterpret_cast<void **>(&p), sizeof(T) * count); }
};

// Tile-blocked storage: the n x n grid of 3x3 blocks is cut into row panels
// of TR tiles and column chunks of TC tiles.  Chunk (p, q) is contiguous and
// holds NPLANE planes of TR x TC values (plane-major, then row, then column),
// so a panel is one contiguous stream and a chunk one bulk TMA copy.
struct mt_layout {
  int TR = 16, TC = 128;
  int nplane = 6;           // 6 unique entries (12 for split hi/lo)
  int elem_bytes = 4;
  int64_t P = 0, Q = 0;     // panels, chunks per panel
  bool half = false;        // only the upper triangle of chunks (see half_gbase)
  int64_t CH = 0;           // stored chunks (P * Q, or half_chunks(P, Q) when half)
  int64_t chunk_elems() const { return (int64_t)nplane * TR * TC; }
  int64_t chunk_bytes() const { return chunk_elems() * elem_bytes; }
  int64_t scale_bytes_per_chunk = 0;  // BF16 scaled: TR x TC int8 exponents
};

// Half storage (Sec. 3.2: the tensor is symmetric).  For tiles of one shape
// the point tensor is even in the offset of the two centres, so N_ij = N_ji
// (and every block is symmetric).  With K = TC / TR panels per chunk row,
// super-row R (panels K R .. K R + K - 1: the rows of column chunk R; there
// are Q super-rows, as K TR = TC) keeps its chunks of column chunks q >= R.
// The diagonal group (q = R) is used as stored, for its rows; every higher
// chunk serves its rows and, transposed, its columns.  Stored order: super-row
// by super-row, in each the column chunks in turn, and for each column chunk
// its K panels one after the other (a "group" of K chunks): chunk (p, q) with
// R = p / K is number K (half_gbase(R) + q - R) + p - K R, half_gbase(R)
// counting the groups of the super-rows above R.  (A group's K chunks come
// one after the other, so the product keeps a column's sums over K panels.)
__host__ __device__ __forceinline__ int64_t half_q0(int64_t p, int K) { return p / K; }
__host__ __device__ __forceinline__ int64_t half_gbase(int64_t R, int64_t Q) { return R * Q - R * (R - 1) / 2; }
// groups and stored chunks of a half-stored P x Q chunk grid
__host__ __device__ __forceinline__ int64_t half_groups(int64_t Q) { return half_gbase(Q, Q); }
__host__ __device__ __forceinline__ int64_t half_chunks(int64_t P, int64_t Q, int K) {
  return (int64_t)K * half_gbase(Q - 1, Q) + (P - (int64_t)K * (Q - 1));  // the last super-row: one group
}
// stored chunk of (panel p, column chunk q), -1 if the half storage omits it
__host__ __device__ __forceinline__ int64_t stream_chunk(int64_t p, int64_t q, int64_t Q, int TR, int TC,
                                                         bool half) {
  if (!half) return p * Q + q;
  const int K = TC / TR;
  const int64_t R = p / K;
  return q < R ? -1 : (int64_t)K * (half_gbase(R, Q) + q - R) + (p - (int64_t)K * R);
}

struct mt_tensor {
  std::atomic<int> refs{1};
  mt_tiles *tiles = nullptr;
  int prec = MT_F32;
  int layout = MT_LAYOUT_STREAM;  // MT_LAYOUT_DENSE: 9-entry BF16 matrix for tensor cores
  int64_t n = 0;
  int64_t Kp = 0;                 // dense layout: rows = columns = 3n padded to 128
  mt_layout L;
  void *d_data = nullptr;
  size_t bytes = 0;
  int8_t *d_scale = nullptr;     // BF16 scaled: per-block exponent
  // near-field blocks held apart in FP64 (block sparse rows)
  int64_t near_count = 0;
  int32_t *d_near_ptr = nullptr;  // n+1
  int32_t *d_near_col = nullptr;  // near_count
  double *d_near_val = nullptr;   // near_count * 6 (FP64, as assembled)
  float2 *d_near_hl = nullptr;    // near_count * 6: the same values as FP32 hi + lo pairs
  // workspace of the standalone field / rhs calls
  float *d_xs = nullptr;
  int xs_B = 0;
  float *d_part = nullptr;
  int *d_count = nullptr;
  int count_B = 0;
  float *d_Hd = nullptr;
  int Hd_B = 0;
  float *d_colpart = nullptr;  // half storage: column work area of the standalone calls
  int colpart_B = 0;
  int gemm_stages[4] = {0, 0, 0, 0};  // tuned ring depth per padded batch 16/32/64/128
  int gemm_kps[4] = {0, 0, 0, 0};     // tuned K blocks per ring stage (tile shape along K)
  // thresholded layout: block-sparse rows (kept blocks, 6 FP32 entries each)
  int64_t sp_blocks = 0;         // stored blocks (runs padded to 4)
  int64_t sp_runs = 0;           // runs of consecutive columns
  int64_t *d_sp_ptr = nullptr;   // n + 1: first block of each row
  int64_t *d_sp_rptr = nullptr;  // n + 1: first run of each row
  int32_t *d_sp_col = nullptr;   // 2 per run: (first block within the row, first column)
  float *d_sp_val = nullptr;
  int32_t *d_sp_seg = nullptr;   // n x 8: the run holding each eighth of a row's steps
  int sp_split = 1;              // warps per row of the sparse product (1, 2, 4 or 8)
};

// Plane of entry e (xx, xy, xz, yy, yz, zz) in a streaming layout of
// nplane planes: the identity for 6, -1 for the xz and yz entries of a
// single-layer tensor (planes xx, xy, yy, zz), and with 3 planes (xx, xy,
// yy: a single-layer FP32 tensor stored half) -1 for zz as well, which the
// trace gives (see traceless).  The split precision holds two such sets (hi,
// then lo): call it with half its planes.
__host__ __device__ __forceinline__ int stream_plane(int e, int nplane) {
  if (nplane == 4) return e < 2 ? e : e == 3 ? 2 : e == 5 ? 3 : -1;
  if (nplane == 3) return e < 2 ? e : e == 3 ? 2 : -1;
  if (nplane == 5) return e < 5 ? e : -1;  // xx, xy, xz, yy, yz (zz from the trace)
  return e;
}
// zz is given by the trace (not stored) in a 3- or 5-plane layout
__host__ __device__ __forceinline__ bool traceless(int nplane) { return nplane == 3 || nplane == 5; }
// bound on |N_xz|, |N_yz| of a single-layer tile set (FP64 round-off of
// entries that vanish by mirror symmetry)
constexpr double kPlanarTol = 1e-12;
// Traceless storage.  The potential of a uniformly magnetised tile is
// harmonic outside it, so the point tensor of tile j at the centre of any
// other tile i has trace 0, and a self block trace 1: N_zz = delta_ij -
// N_xx - N_yy.  A 3-plane tensor stores xx, xy, yy only (a single layer,
// whose xz and yz vanish), a 5-plane one xx, xy, xz, yy, yz; assembly checks the
// identity on every block, |trace - delta_ij| <= kTraceTol (|N_xx| + |N_yy| +
// |N_zz|) + kPlanarTol (the FP64 round-off of the corner sums, which for
// distant tiles is absolute: their small entries are differences of O(1)
// terms); else all 6 planes are stored.
constexpr double kTraceTol = 1e-9;
// MT_LAYOUT_STREAM stores a tensor of tiles of one shape half from this many
// tiles on: measured on single-layer films, one simulation, per attempted
// integrator step, half against full storage 0.178 / 0.140 ms at 2,500 tiles,
// 0.255 / 0.253 at 3,600, 0.384 / 0.413 at 4,900, 0.516 / 0.646 at 6,400
// (the column pass costs a fixed ~15 us that a small tensor does not repay)
constexpr int64_t kHalfMinTiles = 4096;

// Index of entry e of block (i, j) in the tile-blocked streaming layout.
__host__ __device__ __forceinline__ int64_t layout_index(int64_t i, int64_t j, int e, int TR, int TC, int nplane,
                                                         int64_t Q) {
  const int64_t p = i / TR, q = j / TC;
  const int r = (int)(i - p * TR), c = (int)(j - q * TC);
  return (((p * Q + q) * nplane + e) * TR + r) * (int64_t)TC + c;
}
// The same for either storage; -1 where the half storage omits block (i, j)
// (it is block (j, i), stored: N_ij = N_ji for tiles of one shape).
__host__ __device__ __forceinline__ int64_t layout_index_h(int64_t i, int64_t j, int e, int TR, int TC, int nplane,
                                                           int64_t Q, bool half) {
  const int64_t p = i / TR, q = j / TC;
  const int64_t ch = stream_chunk(p, q, Q, TR, TC, half);
  if (ch < 0) return -1;
  const int r = (int)(i - p * TR), c = (int)(j - q * TC);
  return ((ch * nplane + e) * TR + r) * (int64_t)TC + c;
}

// Operand of the thresholded product: a float4 (Ms m, 0) per tile and
// simulation, n + 4 per simulation (the last 4 zero: a run's padding blocks
// may reach 3 columns past the last tile).
__host__ __device__ __forceinline__ int64_t sparse_x_stride(int64_t n) { return n + 4; }

// Dense layout, tile-blocked: the 3n x 3n matrix (padded to Kp = 128 k) is
// cut into 128-row x 64-column BF16 tiles, each stored contiguously (16 KB,
// rows of 128 bytes), tiles ordered by (row tile, K block); the low part of
// the split precision is a second such plane.  The operand X of a batch is
// cut the same way along K: block kb holds Bp rows of 64 values.
__host__ __device__ __forceinline__ size_t dense_a_index(int64_t r, int64_t c, int64_t KB) {
  return ((size_t)((r >> 7) * KB + (c >> 6)) * 128 + (size_t)(r & 127)) * 64 + (size_t)(c & 63);
}
__host__ __device__ __forceinline__ size_t dense_x_index(int64_t b, int64_t c, int64_t Bp) {
  return ((size_t)(c >> 6) * Bp + (size_t)b) * 64 + (size_t)(c & 63);
}

// Tensor maps and shape of one batched tensor-core product (dense layout).
struct GemmPlan {
  CUtensorMap tA, tAlo, tX, tX1, tX2;  // tensor hi/lo; operand terms (split: x0, x1, x2)
  const float *mT = nullptr;           // simulation-fastest copy of m (near blocks)
  int B = 0, Bp = 0, stages = 0;
  int kps = 1;    // K blocks per ring stage (one unit of work)
  int chunk = 4;  // units accumulated in TMEM before the FP32 promotion (4 K blocks)
  bool split = false;
};

// ---------------------------------------------------------------------------
// matvec workspace and launch
// ---------------------------------------------------------------------------
namespace mt {

// Number of CTAs of the streaming product (one per SM).
int matvec_grid(const mt_tensor *T);
// Set kernel attributes once, before any stream capture.
cudaError_t matvec_prepare();
// Panel/chunk shape of the storage for a precision (P, Q left to the caller).
void layout_for(int prec, mt_layout *L);
void layout_for_planar(int prec, mt_layout *L);  // single-layer tile set: 4 entry planes (split: 4 hi + 4 lo)
// FP32 tile set stored half: zz from the trace, 3 entry planes (xx, xy, yy)
// for a single layer (planar), else 5 (xx, xy, xz, yy, yz)
void layout_for_traceless(mt_layout *L, bool planar);
// floats of the padded, Ms-scaled operand of one simulation: Q * 3 * TC
int64_t xs_floats(const mt_tensor *T);
// bytes of the partial-sum workspace and of the panel counters for B sims
size_t matvec_part_bytes(const mt_tensor *T);
size_t matvec_count_bytes(const mt_tensor *T, int B);

// xs[b] = Ms * m[b] in the padded chunked layout ([Q][3][TC], zero padded)
void launch_prep_xs(const mt_tensor *T, const float *m, int B, float *xs, cudaStream_t s);
void launch_prep_xs_f64(const mt_tensor *T, const double *m, int B, double *xs, cudaStream_t s);
// bytes of the column work area of a half-stored tensor for B sims (0 if
// the tensor stores every block)
size_t matvec_colpart_bytes(const mt_tensor *T, int B);
// H[b] = -N xs[b]; active (may be null) skips finished simulations; colpart:
// the column work area (matvec_colpart_bytes) of a half-stored tensor
void launch_matvec(const mt_tensor *T, const float *xs, int B, float *H, float *part, int *count,
                   const int *active, int *status, cudaStream_t s, float *colpart = nullptr);
// H[b] -= near-field blocks applied to Ms m (BF16 precisions); element
// (b, j, c) of m at m[b * sb + (3 j + c) * se]
void launch_near(const mt_tensor *T, const float *m, int64_t sb, int64_t se, int B, float *H, const int *active,
                 cudaStream_t s);

// batched product on tcgen05 (dense layout)
cudaError_t gemm_prepare();
int dense_pad_batch(int B);
size_t dense_x_bytes(const mt_tensor *T, int B);
size_t dense_part_bytes(const mt_tensor *T, int B);
size_t dense_count_bytes(const mt_tensor *T);
void launch_prep_dense_x(const mt_tensor *T, const float *m, int B, void *X, cudaStream_t s);
mt_status gemm_plan(const mt_tensor *T, int B, const void *X, GemmPlan *plan);
// choose the ring depth of the batched product by timing (once per tensor
// and padded batch); writes scratch values into H, part
mt_status gemm_tune(mt_tensor *T, GemmPlan *plan, float *H, float *part, int *count, int *status, cudaStream_t s);
// the simulation-fastest copy of the state used by the near blocks of a
// dense-layout batch: mT[(3 j + c) * Bp + b], right after the operand X
float *dense_mT(const mt_tensor *T, int B, void *X);
void launch_gemm(const mt_tensor *T, const GemmPlan &plan, float *H, float *part, int *count, const int *n_active,
                 int *status, cudaStream_t s);

// thresholded tensor: product and inspection
// sparse product: xs = float4 (Ms m, 0) per tile and simulation (4 n B floats)
void launch_spmv(const mt_tensor *T, const float *xs, int B, float *H, const int *active, cudaStream_t s);
void launch_prep_sparse_x(const mt_tensor *T, const float *m, int B, float *xs, cudaStream_t s);
mt_status read_rows_sparse(const mt_tensor *T, int64_t i0, int64_t i1, double *out);

// reference counting of handles (see the handle structs)
void ctx_release(mt_ctx *c);
void tiles_release(mt_tiles *t);
void tensor_release(mt_tensor *T);

// assembly (FP64) and packing
mt_status assemble(mt_tensor *T);
mt_status blocks_fp64(mt_tiles *t, int64_t count, const int64_t *pairs, double *out);
mt_status read_rows(const mt_tensor *T, int64_t i0, int64_t i1, double *out);

// per-simulation prefactors of Eq. 1: g1 (precession), g2 (damping), Ha
void llg_prefactors(const mt_llg_params *p, int B, std::vector<float> &g1, std::vector<float> &g2,
                    std::vector<float> &ha, std::vector<float> &xsc);

// energy terms (Eqs. 4, 6, 8, 11, 15) per simulation, accumulated into
// E[b*4 + {0: Zeeman, 1: demag, 2: exchange, 3: anisotropy}] (device, zeroed)
void launch_energy(const mt_tensor *T, const float *m, const float *Hd, int B, const float *Ha, const float *xsc,
                   double *E, cudaStream_t s);

// standalone right-hand side
void launch_rhs_plain(const mt_tensor *T, const float *m, const float *Hd, int B, const float *g1,
                      const float *g2, const float *Ha, const float *xsc, float *dmdt, float *tau, cudaStream_t s);

}  // namespace mt

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
namespace mtd {

// Programmatic dependent launch (kernels of the step graph): wait until the
// preceding kernel of the stream has completed and its writes are visible
// (returns at once when the launch did not ask for it), then let the next
// kernel be scheduled, so that its launch and prologue overlap this kernel.
// Every kernel launched with mt::launch_pdl calls this before it touches
// global memory that its predecessor writes or reads.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of an mbarrier, giving up after ~limit_ns of wall
// time: then the status word gets MT_DEV_TIMEOUT and false is returned.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *status,
                                                  uint64_t limit_ns = 2000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0u) {
      if (globaltimer_ns() - t0 > limit_ns) {
        if (status) atomicExch(status, MT_DEV_TIMEOUT);
        return false;
      }
    }
  }
}

// 1-D bulk prefetch of global memory into L2 (no completion to wait for).
// src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared, completion signalled on `bar` (tx bytes).
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                         uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// max that propagates NaN (fmax would drop it and hide a non-finite state)
__device__ __forceinline__ double nan_max(double a, double b) { return (a > b || a != a) ? a : b; }
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nan_max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float nan_max(float a, float b) { return (a > b || a != a) ? a : b; }
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nan_max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Stream-K split of U work units over G CTAs: CTA k owns [begin(k), begin(k+1)).
__host__ __device__ __forceinline__ int64_t sk_begin(int64_t k, int64_t U, int64_t G) { return (k * U) / G; }
// CTA owning unit u: largest k with begin(k) <= u.
__host__ __device__ __forceinline__ int64_t sk_owner(int64_t u, int64_t U, int64_t G) {
  return ((u + 1) * G + U - 1) / U - 1;
}

// Double-FP32 sums for the near-field blocks (BF16 precisions): H_i -= sum
// over touching j of N_ij Ms_j m_j with FP64-class accuracy on the FP32
// pipes.  The blocks were assembled in FP64 and are held, times Ms_j, as FP32
// hi + lo pairs; products use the exact FMA product split (p = a b,
// e = fma(a, b, -p)) and the sum is carried as an unevaluated pair
// (hi + lo), Knuth's two-sum feeding every rounding error into lo, then
// added to the far field and rounded once.  (GB300 executes FP64 at a small
// fraction of its FP32 rate; this keeps ~2^-44 relative accuracy at FP32
// speed.)
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_add(ff acc, float p, float e) {
  ff s = ff_two_sum(acc.hi, p);
  s.lo += acc.lo + e;
  const float hi = s.hi + s.lo;
  return {hi, s.lo - (hi - s.hi)};
}
// acc += (v.hi + v.lo) * x with the error of the rounded product and of the
// addition collected in acc.lo (a cascaded sum: no renormalisation per term,
// acc.lo stays a few ulps of acc.hi over the <= 27 blocks of a row)
__device__ __forceinline__ void ff_fma_lazy(ff &acc, float2 v, float x) {
  const float p = v.x * x;
  const float e = fmaf(v.y, x, fmaf(v.x, x, -p));
  const float s = acc.hi + p;
  const float bp = s - acc.hi;
  acc.lo += ((acc.hi - (s - bp)) + (p - bp)) + e;
  acc.hi = s;
}

}  // namespace mtd
#endif
