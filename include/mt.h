/*
 * mt.h -- C ABI of the GB300 tile-micromagnetics library (libmagtile.so).
 *
 * The library implements the hot path of the tile-based micromagnetic
 * method of Bjork et al. (arXiv 2107.05364, "MagTense"): the magnet is
 * split into uniformly magnetised rectangular cuboid tiles (Sec. 3); the
 * demagnetization field of every tile is evaluated analytically at the
 * centre of every other tile, giving a dense 3n x 3n tensor N computed once
 * (Sec. 3.1); at every right-hand-side evaluation of the Landau-Lifshitz
 * equation (Eq. 1) the effective field H_eff = A m + b (Eq. 17) is formed
 * from the dense demag product H_d = -N (Ms m) (Eq. 9), the exchange field
 * (Eq. 12), the uniaxial anisotropy field (Eq. 16) and the applied field
 * (Eq. 7), and the equation is integrated with an explicit Runge-Kutta (4,5)
 * pair (Sec. 3.1).
 *
 * Conventions for every call:
 *   - SI units: lengths m, fields A/m, Ms A/m, A_ex J/m, K J/m^3,
 *     gamma m/(A s), time s.
 *   - Vectors of tiles are tile-major: m[3*i + c], c = x, y, z.  A batch of
 *     B simulations on one geometry is B such vectors back to back
 *     (m[b*3n + 3*i + c]).
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory on the context's device (e.g. from torch).  The caller
 *     owns every pointer it passes; the library never frees them and keeps
 *     none of them after the call returns, except where stated.
 *   - Handles (mt_ctx, mt_tiles, mt_tensor, mt_integrator, mt_server) are
 *     owned by the library and released with the matching *_destroy call.
 *   - Every call returns an mt_status.  On failure a message is available
 *     from mt_last_error() (thread-local) and outputs are unspecified.
 *     Nothing is thrown across the ABI.
 *   - Calls taking a `stream` (a cudaStream_t passed as void*, NULL = the
 *     legacy default stream) are asynchronous unless stated otherwise.
 */
#ifndef MT_H
#define MT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MT_API __attribute__((visibility("default")))
#else
#define MT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MT_OK = 0,
  MT_EINVAL = 1,      /* bad argument (size, pointer, non-finite parameter)   */
  MT_ENOMEM = 2,      /* device allocation failed or HBM budget exceeded      */
  MT_EOVERLAP = 3,    /* tiles overlap, or a centre lies on another tile      */
  MT_ENOCONV = 4,     /* step cap or time cap reached before the goal         */
  MT_ETIMEOUT = 5,    /* a bounded device wait or a host wait ran out         */
  MT_ENONFINITE = 6,  /* a NaN/Inf appeared in the state or the error norm    */
  MT_ECUDA = 7,       /* CUDA runtime error (message in mt_last_error)        */
  MT_EBUSY = 8        /* resource in use (e.g. server queue full)             */
} mt_status;

/* Storage precision of the assembled tensor.  Assembly itself is always
 * FP64 (the corner sums cancel catastrophically in the far field).  Every
 * product accumulates in FP32, except MT_F64 which accumulates in FP64. */
typedef enum {
  MT_F64 = 0,          /* 8 B per entry                                       */
  MT_F32 = 1,          /* 4 B per entry: the paper's storage (Sec. 3.2)        */
  MT_BF16_SCALED = 2,  /* 2 B per entry + a power-of-two scale per 3x3 block;  */
                       /* the tile and its touching neighbours are kept apart  */
                       /* (assembled FP64, applied in FP32)                    */
  MT_BF16_SPLIT = 3    /* hi + lo BF16 pair (4 B per entry); near blocks kept  */
                       /* apart, applied in double-FP32 (~FP64 accuracy)       */
} mt_prec;

/* Storage layout of the assembled tensor. */
typedef enum {
  MT_LAYOUT_STREAM = 0, /* 6 unique entries per block, tile-blocked panels for  */
                        /* the streaming product (one simulation per pass)      */
  MT_LAYOUT_DENSE = 1,  /* all 9 entries, row-major 3n x 3n BF16 (or hi + lo   */
                        /* pair) for the batched tensor-core product; only      */
                        /* MT_BF16_SCALED (scales fixed to 1) and MT_BF16_SPLIT */
  MT_LAYOUT_SPARSE = 2, /* thresholded FP32 tensor in block-sparse rows       */
                        /* (made by mt_tensor_threshold, Sec. 4.3.1)            */
  MT_LAYOUT_STREAM6 = 3, /* MT_LAYOUT_STREAM with all 6 entry planes and every  */
                        /* block stored (see mt_demag_assemble)                */
  MT_LAYOUT_STREAM_FULL = 4, /* MT_LAYOUT_STREAM with every block stored (no use */
                        /* of N_ij = N_ji; planes as for MT_LAYOUT_STREAM)      */
  MT_LAYOUT_STREAM_HALF = 5 /* MT_LAYOUT_STREAM with the half storage of tiles  */
                        /* of one shape at any size (FP32 cuboids of one shape */
                        /* only, else MT_EINVAL; see mt_demag_assemble)         */
} mt_layout_kind;

/* Equation-of-motion form. */
typedef enum {
  MT_FORM_GILBERT = 0, /* dm/dt = -gamma/(1+a^2) [m x H + a m x (m x H)]      */
  MT_FORM_LL = 1       /* Eq. 1: dm/dt = -gamma m x H - alpha m x (m x H)     */
} mt_form;

/* How an integrator executes its steps (mt_integrator_set_path). */
typedef enum {
  MT_PATH_GRAPH = 1,      /* one CUDA-graph replay per attempt: 6 demag       */
                          /* products + 7 stage kernels; every tensor kind    */
  MT_PATH_PERSISTENT = 2  /* a whole step/run/relax call as one cooperative    */
                          /* kernel: each SM holds its rows of the tensor in   */
                          /* shared memory, grid barriers between the stages; */
                          /* FP32 streaming tensors of small tile sets         */
} mt_path;

typedef struct mt_ctx mt_ctx;
typedef struct mt_tiles mt_tiles;
typedef struct mt_tensor mt_tensor;
typedef struct mt_integrator mt_integrator;

/* Per-simulation parameters of the equation of motion for a batch of B.
 * All arrays are HOST memory, copied by the call that receives them. */
typedef struct {
  double gamma;        /* gyromagnetic ratio, m/(A s) (2.211e5 for electrons) */
  const double *alpha; /* [B] damping: dimensionless (Gilbert) or m/(A s) (LL) */
  const double *Ha;    /* [3B] applied field per simulation, A/m (Eq. 7)      */
  int form;            /* mt_form                                             */
  int precess;         /* 1 = full equation, 0 = drop the m x H term           */
  const double *exch_scale; /* [B] factor on every tile's exchange stiffness A */
                       /* per simulation (NULL: 1).  The point tensor depends */
                       /* only on shape ratios, so the same tiles scaled by   */
                       /* lam behave as the originals with A / lam^2: a size  */
                       /* sweep (d / l_ex, Sec. 4.1) shares one tensor        */
} mt_llg_params;

/* Runge-Kutta (4,5) options (Dormand-Prince pair, Sec. 3.1). */
typedef struct {
  double rtol, atol;   /* error norm: RMS of e/(atol + rtol max(|y|,|y_new|)) */
  double h0;           /* first trial step, s                                 */
  double hmax;         /* largest step, s (<= 0: unlimited)                   */
  int64_t max_steps;   /* cap on attempted steps per call                     */
  double fixed_h;      /* > 0: fixed step of this size, no error control      */
} mt_ode_opts;

/* Per-simulation outcome of an integration. */
typedef struct {
  int64_t n_accept, n_reject, n_rhs;
  double t;            /* time reached, s                                     */
  double h;            /* next step proposal, s                               */
  double tau;          /* max_i |m_i x H_eff,i| / Ms_i at the last evaluation */
  int32_t status;      /* mt_status of this simulation                        */
  int32_t pad;
} mt_stats;

/* Description of an assembled tensor. */
typedef struct {
  int64_t n;           /* tiles                                               */
  int32_t prec;        /* mt_prec                                             */
  int32_t rows_per_panel, cols_per_chunk; /* tile-blocked layout (stream)     */
  int32_t layout;      /* mt_layout_kind                                      */
  int32_t planes;      /* stored values per 3x3 block: 6 (4 single-layer),    */
                       /* split 12 (8 single-layer), dense 9                  */
  int64_t bytes;       /* device bytes of the stored tensor                   */
  int64_t near_blocks; /* FP64 near-field blocks kept apart (0 if none)       */
  int32_t half;        /* 1: only the upper triangle of blocks is stored      */
                       /* (N_ij = N_ji, see mt_demag_assemble)                */
  int32_t row_warps;   /* sparse layout: warps that share a row of the        */
                       /* product (1, 2, 4 or 8; see mt_tensor_threshold);    */
                       /* 0 for the other layouts                             */
} mt_tensor_info;

/* ---------------------------------------------------------------------- */
/* library and context                                                     */
/* ---------------------------------------------------------------------- */

/* Version string; never fails. */
MT_API const char *mt_version(void);

/* Message of the last failed call on this thread ("" if none). */
MT_API const char *mt_last_error(void);

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * device memory of the tensors this context assembles (0 = 90 % of the
 * device's free memory at creation).  Errors: MT_EINVAL (bad device),
 * MT_ECUDA. */
MT_API mt_status mt_ctx_create(int device, size_t hbm_budget_bytes, mt_ctx **out);
MT_API void mt_ctx_destroy(mt_ctx *ctx);

/* Bytes of tensors currently held by the context. */
MT_API size_t mt_ctx_bytes_in_use(const mt_ctx *ctx);

/* ---------------------------------------------------------------------- */
/* tiles (Sec. 3: the magnet as N uniformly magnetised cuboid tiles)       */
/* ---------------------------------------------------------------------- */

/* Create a tile set of n >= 1 cuboids from HOST arrays (copied):
 *   centre[3n], edge[3n] (full edge lengths, > 0), Ms[n] (> 0), Aex[n],
 *   Ku[n], axis[3n] (easy axis, normalised by the call),
 *   nbr[6n] face neighbours (-x,+x,-y,+y,-z,+z; -1 = free surface) of a
 *   Cartesian (tensor-product) mesh, used by the finite-difference exchange
 *   of Sec. 3 with the Neumann boundary of Eq. 3; nbr == NULL disables
 *   exchange coupling.
 * Errors: MT_EINVAL (n < 1, NULL array, non-finite or non-positive value,
 * neighbour index out of range), MT_ECUDA. */
MT_API mt_status mt_tiles_create(mt_ctx *ctx, int64_t n, const double *centre, const double *edge,
                          const double *Ms, const double *Aex, const double *Ku, const double *axis,
                          const int32_t *nbr, mt_tiles **out);

/* Create a tile set of n >= 1 tetrahedra (Sec. 3: tetrahedral tiles, whose
 * tensor is known in closed form; evaluated here from the charges M.n of
 * the four faces) from HOST arrays (copied): vertices[3 nv], tets[4n] vertex
 * indices, Ms[n] (> 0), Aex[n], Ku[n], axis[3n].  The field point of a tile
 * is its centroid.  Exchange (which the paper leaves to later work for
 * unstructured tiles) is the two-point flux over shared faces:
 *   H_ex,i = (2 A_i / (mu0 Ms_i)) sum_faces area / (V_i d_ip) (m_p - m_i),
 * d_ip the centroid distance along the face normal; faces on the surface
 * carry no flux (Eq. 3).  It is exact for uniform m and first-order only
 * where the centroid line is normal to the face.  Two tiles sharing a vertex
 * count as touching (kept in FP64 for the BF16 precisions).
 * Errors: MT_EINVAL (index out of range, repeated vertex, degenerate tile,
 * a face shared by three tiles, non-finite value), MT_ECUDA; assembly
 * reports MT_EOVERLAP when a centroid lies in or on another tile. */
MT_API mt_status mt_tiles_create_tetra(mt_ctx *ctx, int64_t nv, const double *vertices, int64_t n,
                                       const int32_t *tets, const double *Ms, const double *Aex, const double *Ku,
                                       const double *axis, mt_tiles **out);
MT_API void mt_tiles_destroy(mt_tiles *tiles);

/* ---------------------------------------------------------------------- */
/* demagnetization tensor (Sec. 3, Sec. 3.1, Sec. 3.2)                     */
/* ---------------------------------------------------------------------- */

/* Assemble N on the device: one thread per 3x3 block (i, j) evaluates the
 * closed-form tensor of cuboid j at the centre of tile i in FP64 (all
 * 8-corner arctan/log sums), then stores the 6 unique entries of each
 * symmetric block in `prec` in a tile-blocked layout.  Synchronous.  The
 * tiles must outlive the tensor.
 * Errors: MT_EOVERLAP (two tiles overlap, or a centre lies inside/on
 * another tile), MT_ENOMEM (allocation failed or the context budget would
 * be exceeded), MT_EINVAL, MT_ECUDA. */
MT_API mt_status mt_demag_assemble(mt_tiles *tiles, mt_prec prec, mt_tensor **out);
/* Single-layer tile sets.  When every cuboid tile has the same centre z and
 * the same z edge, each tile's field point lies in the mid-plane of every
 * other tile, and the xz and yz entries of every block vanish by mirror
 * symmetry (they are odd in the z offset).  A streaming tensor of such a set
 * (FP32, scaled BF16 or split BF16) stores the 4 entry planes xx, xy, yy, zz
 * (FP32 and split: 16 bytes per block instead of 24; BF16: 8 + the scale
 * byte instead of 12 + 1),
 * provided that every assembled |N_xz|, |N_yz| is at most 1e-12
 * (their FP64 round-off; otherwise all 6 planes are stored).  Products,
 * row reads and thresholding treat the missing entries as zeros.
 * MT_LAYOUT_STREAM6 keeps the 6 planes.
 * Tiles of one shape.  When every cuboid has the same edges, the point
 * tensor of tile j at the centre of tile i depends only on c_i - c_j and is
 * even in it, so N_ij = N_ji and the whole tensor is symmetric (Sec. 3.2).
 * An FP32 streaming tensor of more than 4,096 such tiles (any number with
 * MT_LAYOUT_STREAM_HALF; below ~3,600 tiles the full storage's product is
 * the faster one, one simulation) then stores only the upper triangle: 16-row panel p keeps its 128-column chunks from the
 * one holding its own rows on (about n^2 / 2 blocks); the product applies
 * each off-diagonal chunk to its rows and, transposed, to its columns (a
 * column work area of 1.5 KB per stored chunk and simulation, held by the
 * tensor or the integrator).  Stored half, the tensor leaves out zz: a
 * tile's potential is harmonic outside it, so every block of two different
 * tiles has trace 0 (a self block trace 1), and the product forms N_zz =
 * delta_ij - N_xx - N_yy.  A single-layer set keeps 3 planes (xx, xy, yy),
 * others 5 (xx, xy, xz, yy, yz); assembly checks the identity on every block
 * and otherwise stores all 6 planes (mt_tensor_info.planes tells).
 * mt_tensor_info.half tells;
 * MT_LAYOUT_STREAM_FULL stores every block.  The half storage's product is
 * the faster one for products over 1 or 2 simulations (n = 10,000 film:
 * 0.11 against 0.25 ms for one, 0.15 against 0.26 ms for two); over 3 or
 * more simulations the full storage is (two passes, 0.31 against 0.24 ms
 * for four), so a caller that batches 3 or more should assemble
 * MT_LAYOUT_STREAM_FULL.  A pass over two simulations forms the row sums in
 * another order than a pass over one (each chunk's warp total first), so a
 * simulation's field from a half-stored tensor in a pair and alone agree to
 * rounding, not bit for bit.
 * Thresholding and the allocation-free product need every block stored. */
/* As mt_demag_assemble, with an explicit storage layout (mt_layout_kind).
 * MT_LAYOUT_DENSE turns every product over a batch of B simulations into a
 * GEMM on the tensor cores (tcgen05, BF16 in, FP32 accumulate); the rows and
 * columns of the 3n x 3n matrix are padded to a multiple of 128 (zeros) and
 * the blocks of touching tiles are kept apart in FP64 as for the streaming
 * layout.  Errors as mt_demag_assemble, plus MT_EINVAL for a precision the
 * layout does not support. */
MT_API mt_status mt_demag_assemble_ex(mt_tiles *tiles, mt_prec prec, int layout, mt_tensor **out);

/* Thresholded copy of an FP32 streaming-layout tensor (Sec. 4.3.1): the
 * smallest `fraction` (in [0, 1)) of the nonzero elements of the full 3n x 3n
 * matrix, ranked by absolute FP32 value (an off-diagonal block entry counts
 * twice), is set to zero and the rest stored in block-sparse rows (a block is
 * kept if any entry survives).  Exactly k = floor(fraction * nonzeros)
 * elements go: all below the magnitude t of the element of rank k, and of
 * those equal to t the first ones in (row tile, column tile, entry xx xy xz
 * yy yz zz) order; an off-diagonal entry whose two copies the cut would
 * split is kept whole (k - 1 go), so blocks stay symmetric.  The kept
 * columns of a row are stored as runs of consecutive tiles (gaps of up to 3
 * blocks filled with zeros, runs padded to 4 blocks), so the product reads
 * 24 B per stored block (6 FP32 entries; 16 B for a single-layer tile set)
 * plus 8 B per run, and sums in compensated FP32.  A row's blocks are split
 * among 1, 2, 4 or 8 warps (mt_tensor_info.row_warps), fixed per tensor from
 * its size and row lengths, so a simulation's field does not depend on the
 * batch it is computed in.  The
 * new tensor works with mt_demag_field, mt_llg_rhs, mt_energy and the
 * integrator; it keeps the tile set alive.  threshold (may be NULL) gets t,
 * kept_elements (may be NULL) the number of kept nonzero elements.
 * Synchronous.  Errors: MT_EINVAL (not FP32 streaming, bad fraction),
 * MT_ENOMEM, MT_ECUDA. */
MT_API mt_status mt_tensor_threshold(mt_tensor *T, double fraction, mt_tensor **out, double *threshold,
                                     int64_t *kept_elements);

MT_API void mt_tensor_destroy(mt_tensor *T);
MT_API mt_status mt_tensor_get_info(const mt_tensor *T, mt_tensor_info *info);

/* Copy the stored blocks of rows [i0, i1) back to HOST memory as FP64,
 * out[((i - i0) * n + j) * 6 + e], e = xx, xy, xz, yy, yz, zz.  For the
 * BF16 precisions the dequantised dense value is returned and near blocks
 * (held apart in FP64) are merged in.  Synchronous.  Errors: MT_EINVAL. */
MT_API mt_status mt_tensor_read_rows(const mt_tensor *T, int64_t i0, int64_t i1, double *out);

/* Evaluate selected blocks in FP64 on the device with the assembly kernel's
 * arithmetic: pairs[2p] = i (field point tile), pairs[2p+1] = j (source
 * tile), out[6p + e].  HOST arrays; synchronous.  Errors: MT_EINVAL. */
MT_API mt_status mt_demag_blocks(mt_tiles *tiles, int64_t count, const int64_t *pairs, double *out);

/* H_d = -N (Ms m) for B simulations (Eq. 9 / Eq. 17): m and H are DEVICE
 * arrays of B*3n floats (tile-major per simulation).  Streaming layout: the
 * stored tensor is streamed once per simulation.  Dense layout: one batched
 * tensor-core product per call (B <= 128); the first call for a batch width
 * times a few ring depths of the product (autotuning, a few extra launches,
 * results unaffected) and should precede any stream capture.
 * Errors: MT_EINVAL, MT_ECUDA. */
MT_API mt_status mt_demag_field(mt_tensor *T, const float *m, int B, float *H, void *stream);

/* The same product for an FP64 tensor, in FP64: m and H are DEVICE arrays
 * of B*3n doubles; accumulation in FP64.  Errors: MT_EINVAL (tensor not
 * MT_F64), MT_ECUDA. */
MT_API mt_status mt_demag_field_f64(mt_tensor *T, const double *m, int B, double *H, void *stream);

/* Size of the fixed device work area used by mt_demag_field_noalloc, per GPU
 * that loads the library (held until the process exits). */
#define MT_NOALLOC_SCRATCH_BYTES (4u << 20)

/* mt_demag_field for callers that must not let the library allocate device
 * memory: a loop that has given all free HBM to cached tensors, code next to
 * latency-critical streams that cannot take the device-wide synchronisation
 * cudaMalloc/cudaFree may cause, or an application whose own memory pool
 * forbids the CUDA allocator.  Same arguments, same result as mt_demag_field
 * for streaming-layout tensors (FP32, scaled BF16 and split BF16); this call
 * allocates nothing: its work areas (the scaled copy of m, partial panel
 * sums, panel counters) live in one fixed array of MT_NOALLOC_SCRATCH_BYTES
 * in the library's device image.  The paper has no counterpart; it is an
 * interface convenience.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress, which may load the library's device code);
 *     make that first call before any stream capture.
 *   - Every call on a device shares the one array and leaves its contents
 *     behind: calls that overlap on the GPU (different streams, or threads)
 *     race and corrupt each other's result.  Serialise them.
 *   - Scratch needed, each part rounded up to 256 bytes: the scaled operand,
 *     12 bytes per tile and simulation (tiles padded to whole column chunks);
 *     the panel counters, 32 / R bytes per tile and simulation (R = 16 tile
 *     rows per panel for FP32 and BF16, 8 for split: 2 or 4 bytes); the
 *     partial sums, 96 R bytes per SM (on a 152-SM GB300 about 233 KB for
 *     FP32 and BF16, 117 KB for split).  So B * n may reach about 282,000
 *     (FP32, BF16) or 254,000 (split) on a 152-SM GB300.
 *   - Errors: MT_EINVAL if B * n needs more scratch than
 *     MT_NOALLOC_SCRATCH_BYTES, for an FP64 tensor, for a dense-layout or
 *     thresholded (sparse) tensor, or a NULL pointer; MT_ECUDA. */
MT_API mt_status mt_demag_field_noalloc(mt_tensor *T, const float *m, int B, float *H, void *stream);

/* Landau-Lifshitz right-hand side (Eq. 1 or its Gilbert form) at m for B
 * simulations: dmdt (DEVICE, B*3n floats) = f(m, H_eff) with
 * H_eff = H_d + H_ex + H_an + H_a.  tau (DEVICE, B floats, may be NULL)
 * receives max_i |m_i x H_eff,i| / Ms_i per simulation.
 * Errors: MT_EINVAL, MT_ECUDA. */
MT_API mt_status mt_llg_rhs(mt_tensor *T, const mt_llg_params *p, const float *m, int B, float *dmdt,
                     float *tau, void *stream);

/* Micromagnetic energy (Eq. 4 with the densities of Eqs. 6, 8, 11, 15) of B
 * states m (DEVICE, B*3n floats), with the applied fields p->Ha and the
 * exchange factors p->exch_scale (nothing else is read).  E (HOST, 5 doubles per simulation, J): total, Zeeman, demag,
 * exchange, anisotropy; each quadratic term is -(mu0 Ms / 2) m.H of its
 * field, summed over tiles with their volumes.  Synchronous.
 * Errors: MT_EINVAL, MT_ECUDA. */
MT_API mt_status mt_energy(mt_tensor *T, const mt_llg_params *p, const float *m, int B, double *E, void *stream);

/* ---------------------------------------------------------------------- */
/* time integration (Sec. 3.1: explicit Runge-Kutta (4,5))                  */
/* ---------------------------------------------------------------------- */

/* An integrator holds the device state of B simulations on one tensor and
 * a CUDA graph of one Dormand-Prince step (6 right-hand sides, embedded
 * error, accept/reject, renormalisation |m_i| = 1, step-size control, all
 * decided on the device).  Parameters and options are copied.  `stream` is
 * the caller's stream (NULL = legacy default stream); see
 * mt_integrator_stream.
 * Errors: MT_EINVAL, MT_ENOMEM, MT_ECUDA. */
MT_API mt_status mt_integrator_create(mt_tensor *T, const mt_llg_params *p, const mt_ode_opts *o, int B,
                               void *stream, mt_integrator **out);
MT_API void mt_integrator_destroy(mt_integrator *I);

/* Load the state (B*3n floats; host or device pointer as flagged) and set
 * t = t0 for every simulation; resets step counters.  Asynchronous on the
 * integrator's stream (a host source must stay valid until the next
 * synchronising call). */
MT_API mt_status mt_integrator_set_state(mt_integrator *I, const float *m, int m_is_host, double t0);

/* Copy the state out (B*3n floats) to host or device memory.  Synchronous
 * when the destination is host memory. */
MT_API mt_status mt_integrator_get_state(mt_integrator *I, float *m, int m_is_host);

/* The CUDA stream (cudaStream_t as void*) on which the integrator launches
 * its kernels and graph replays.  It is private to the integrator and
 * non-blocking; set_state/get_state order it against the caller's stream
 * with events.  Use it to time or synchronise mt_integrator_step. */
MT_API void *mt_integrator_stream(mt_integrator *I);

/* Execution path (mt_path).  At creation an integrator takes
 * MT_PATH_PERSISTENT where it fits -- an FP32 streaming tensor with at most
 * 8 tiles per SM, whose rows and the B states of all tiles fit one SM's
 * shared memory (about 1,000 tiles for B = 1), or at most 16 tiles per SM
 * reading their rows from an L2-resident tensor of at most 96 MB (about
 * 2,000 tiles) -- and MT_PATH_GRAPH
 * otherwise.  Both compute the same stages with the same step control; they
 * differ in the summation order of the demag product (FP32 round-off).
 * The path may be switched between calls.  set: MT_EINVAL if the path is
 * unknown or does not fit.  get: the path in use (0 for a NULL handle). */
MT_API mt_status mt_integrator_set_path(mt_integrator *I, int path);
MT_API int mt_integrator_get_path(mt_integrator *I);

/* Change the applied field / damping of the batch (host arrays, copied). */
MT_API mt_status mt_integrator_set_params(mt_integrator *I, const mt_llg_params *p);

/* Take exactly `nsteps` attempted steps (accepted or rejected) for every
 * simulation, with no time limit.  Asynchronous. */
MT_API mt_status mt_integrator_step(mt_integrator *I, int64_t nsteps);

/* Integrate every simulation from its current time to t1, writing the
 * volume-weighted mean magnetisation at t_k = t + (k+1)(t1 - t)/n_out,
 * k < n_out, into mavg (HOST, n_out*B*3 doubles, may be NULL).
 * Synchronous; per-simulation outcome in stats (HOST, B entries, may be NULL).
 * Returns MT_OK if every simulation reached t1, else the first failing
 * simulation's status (MT_ENOCONV at the step cap, MT_ENONFINITE). */
MT_API mt_status mt_integrator_run(mt_integrator *I, double t1, int64_t n_out, double *mavg, mt_stats *stats);

/* Relax every simulation (Eq. 2): integrate until
 * max_i |m_i x H_eff,i| / Ms_i < tol, or report MT_ENOCONV once the time
 * t_max is spent.  Synchronous. */
MT_API mt_status mt_integrator_relax(mt_integrator *I, double tol, double t_max, mt_stats *stats);

/* Hysteresis loop (Sec. 4.1, micromagnetic standard problem 2).  For
 * s = 0 .. S-1 the applied field of simulation b is H[s] * dir_b (H: HOST,
 * S values in A/m; dir: HOST, 3B components, normalised here), replacing
 * the Ha of the parameters; then the batch is relaxed at that field, the
 * state carried over from the previous value: for t_step seconds of
 * simulated time when tol = 0 (the paper holds every value for a fixed
 * time), or until max_i |m_i x H_eff,i| / Ms_i < tol with t_step as the cap
 * when tol > 0 (reaching the cap is not an error; the torque is reported).
 * The rest of the equation is the integrator's (the paper: LL form, the
 * precession term dropped, a large damping).
 * Outputs (HOST, each may be NULL): mavg [S][B][3], the volume-averaged m at
 * the end of each value; tau [S][B], the torque there; hc [B], the field
 * (A/m, along dir) at which the projection of <m> on dir first changes sign
 * from positive, interpolated linearly between the two values around it
 * (NaN if it never does); mr [B][3], <m> at H = 0, interpolated between the
 * two values around the first crossing of zero (NaN if none); stats [B], the
 * counters at the end.  Synchronous.
 * Errors: MT_EINVAL, MT_ENONFINITE, MT_ENOCONV (the step cap of the options
 * ran out before a value was done), MT_ETIMEOUT, MT_ECUDA. */
MT_API mt_status mt_integrator_hysteresis(mt_integrator *I, const double *dir, const double *H, int64_t S,
                                          double t_step, double tol, double *mavg, double *tau, double *hc,
                                          double *mr, mt_stats *stats);

/* Energy crossover of two families of states over a size sweep (Sec. 4.2,
 * micromagnetic standard problem 3: the flower and the vortex state of a
 * cube).  The integrator must hold B = 2K simulations.  Size k is lam[k]
 * times the tiles' own size; since the point tensor depends only on shape
 * ratios it enters as the exchange factor 1 / lam[k]^2 (this replaces the
 * parameters' exch_scale).  Simulation k starts from mA and K + k from mB
 * (HOST, 3n floats each), the time is reset to 0, and all are relaxed until
 * max_i |m_i x H_eff,i| / Ms_i < tol or t_max (reaching t_max is not an
 * error; stats tells).  eA, eB (HOST, K each, may be NULL) get the energy
 * densities (total energy over the tiles' volume, J/m^3, which is the same
 * for the really scaled body); lam_cross (may be NULL) the size at which
 * eA - eB first changes sign, linear between the two sizes around it (NaN
 * if it never does; sizes in increasing order); m_out (HOST, 3nB floats,
 * may be NULL) the relaxed states.  Synchronous.
 * Errors: MT_EINVAL, MT_ENONFINITE, MT_ENOCONV (step cap), MT_ETIMEOUT,
 * MT_ECUDA. */
MT_API mt_status mt_integrator_crossover(mt_integrator *I, const double *lam, int K, const float *mA,
                                         const float *mB, double tol, double t_max, double *eA, double *eB,
                                         double *lam_cross, float *m_out, mt_stats *stats);

/* Per-simulation counters since the last set_state.  Synchronous. */
MT_API mt_status mt_integrator_stats(mt_integrator *I, mt_stats *stats);

/* Checkpoint / resume (no counterpart in the paper).  A checkpoint is a
 * self-describing HOST byte image of the integrator's dynamic state: for
 * every simulation its time, step size, step-control state and counters,
 * its m (3n floats) and the derivative the next step starts from (the
 * first-same-as-last stage of Dormand-Prince, 3n floats), plus a header
 * (format version, n, B, the tensor's precision and layout) and a 64-bit
 * FNV-1a checksum of everything before it.  Parameters (Ha, alpha, exchange
 * factors) and options are not part of it: they are the integrator's own.
 * mt_integrator_checkpoint_bytes gives the size (depends only on n and B).
 * mt_integrator_checkpoint writes the image into buf (HOST, at least that
 * many bytes).  mt_integrator_restore loads one into an integrator with the
 * same n and B (the same or another handle, in this or another process);
 * continuing from it takes bit for bit the steps the saved integrator would
 * have taken with the same tensor, parameters and options (every reduction
 * on the path runs in a fixed order, so this holds for adaptive steps too).
 * Restored onto a tensor of another precision or layout, the saved
 * derivative is dropped and re-evaluated on the new tensor.
 * All three are synchronous.
 * Errors: MT_EINVAL (NULL, buffer too small, wrong magic or version,
 * n or B mismatch, checksum mismatch; the integrator is then unchanged),
 * MT_ECUDA. */
MT_API mt_status mt_integrator_checkpoint_bytes(mt_integrator *I, size_t *bytes);
MT_API mt_status mt_integrator_checkpoint(mt_integrator *I, void *buf, size_t bytes);
MT_API mt_status mt_integrator_restore(mt_integrator *I, const void *buf, size_t bytes);

/* One-call forms of the above on DEVICE state m (B*3n floats, in/out). */
MT_API mt_status mt_integrate(mt_tensor *T, const mt_llg_params *p, const mt_ode_opts *o, float *m, int B,
                       double t0, double t1, int64_t n_out, double *mavg, mt_stats *stats, void *stream);
MT_API mt_status mt_relax(mt_tensor *T, const mt_llg_params *p, const mt_ode_opts *o, double tol, double t_max,
                   float *m, int B, mt_stats *stats, void *stream);

/* Self-test of failure detection: runs one kernel whose mbarrier wait can
 * never complete, bounded by limit_s seconds (0 < limit_s <= 10), as every
 * pipelined kernel's waits are (they record a timeout in a status word,
 * release their resources and return instead of hanging).  Returns
 * MT_ETIMEOUT when the wait gave up and reported it (the expected outcome),
 * MT_ECUDA otherwise.  The context stays usable.  Synchronous. */
MT_API mt_status mt_selftest_wait_timeout(mt_ctx *ctx, double limit_s);

/* Self-test of the grid-wide barrier of the one-kernel integrator path
 * (MT_PATH_PERSISTENT): a cooperative launch of 4 CTAs in which one CTA
 * leaves without arriving, so the others' bounded wait (about 2 s) runs
 * out; they record the timeout, raise the abort flag and return.  Returns
 * MT_ETIMEOUT when that was reported (the expected outcome), MT_ECUDA
 * otherwise.  The context stays usable.  Synchronous. */
MT_API mt_status mt_selftest_grid_barrier_timeout(mt_ctx *ctx);

/* ---------------------------------------------------------------------- */
/* request serving: relax and field-sweep jobs on many geometries,          */
/* continuously batched                                                    */
/* ---------------------------------------------------------------------- */
/* A server owns a worker thread that runs every job on the device.  For each
 * geometry with work it keeps the assembled tensor resident together with
 * an integrator of max_batch simulation slots (an "engine" on its own
 * stream); jobs queue per geometry in arrival order and take free slots
 * between graph replays, so work that arrives while other jobs run joins
 * the batch as slots free up.  Engines of different geometries overlap on
 * the device.  Residency is admitted by device footprint (tensor + batch
 * state) against hbm_budget_bytes; idle engines are evicted least recently
 * used.  A relax job integrates its own simulation until
 * max_i |m_i x H_eff,i| / Ms_i < tol (Eq. 2) or its time cap.  A sweep job
 * is the field loop of Sec. 4.1 as one request: its simulation is relaxed
 * at each applied field of its schedule in turn (tolerance tol, time cap
 * t_max per value; reaching the cap is not an error), the state carried
 * over; the job keeps <m> and the torque at the end of every value. */
typedef struct mt_server mt_server;

typedef enum {
  MT_JOB_RELAX = 0,  /* relax m0 at the applied field Ha                     */
  MT_JOB_SWEEP = 1   /* relax at fields[0], fields[1], ... in turn            */
} mt_job_kind;

typedef struct {
  size_t hbm_budget_bytes;  /* tensors + batch state (0: the context budget) */
  int32_t max_batch;        /* slots per resident geometry, 1..128          */
  int32_t prec;             /* mt_prec of cached tensors (not MT_F64)       */
  int32_t layout;           /* mt_layout_kind of cached tensors (not        */
                            /* MT_LAYOUT_SPARSE; MT_LAYOUT_STREAM_HALF      */
                            /* fails the jobs of geometries whose tiles     */
                            /* differ in shape); with MT_LAYOUT_STREAM and  */
                            /* max_batch >= 3 every block is stored         */
                            /* (MT_LAYOUT_STREAM_FULL): the half storage's  */
                            /* product is faster for one or two simulations */
                            /* per pass only                                */
  int32_t form;             /* mt_form of every job                         */
  double gamma;             /* m/(A s)                                      */
  mt_ode_opts ode;          /* integrator options; max_steps caps each job  */
  int32_t replays_per_poll; /* Runge-Kutta attempts between completion      */
                            /* checks (0: 16)                               */
  int32_t max_running;      /* jobs running at once over all geometries     */
                            /* (0: no limit beyond the slots); with a limit */
                            /* jobs start strictly in arrival order (1 and  */
                            /* max_batch 1: one job at a time, FIFO)        */
} mt_server_opts;

typedef struct {
  int32_t geometry;         /* id from mt_server_add_geometry               */
  int32_t kind;             /* mt_job_kind (0: MT_JOB_RELAX)                */
  double alpha;             /* damping of this job                          */
  double Ha[3];             /* relax: applied field, A/m (sweep: unused)    */
  const float *m0;          /* HOST, 3n floats, copied by mt_server_submit  */
  double tol;               /* torque tolerance (> 0)                       */
  double t_max;             /* simulated-time cap, s (> 0); sweep: per value */
  int64_t n_fields;         /* sweep: number of field values, >= 1          */
  const double *fields;     /* sweep: HOST [n_fields][3] applied fields,    */
                            /* A/m, copied by mt_server_submit              */
} mt_job;

typedef struct {
  int32_t status;           /* MT_OK, MT_ENOCONV (relax: time cap; both:    */
                            /* step cap), MT_ENONFINITE, MT_ENOMEM          */
                            /* (geometry exceeds the budget), or the status */
                            /* of a geometry that fails creation/assembly   */
  int32_t geometry;
  double t_submit, t_start, t_done; /* server clock, s since creation       */
  int64_t n_accept, n_reject, n_rhs; /* summed over a sweep's values        */
  double t_sim;             /* simulated time, s (summed over a sweep)      */
  double tau;               /* final torque                                 */
  int64_t values_done;      /* field values finished (relax: 1)             */
  int64_t values_converged; /* of those, values that met the tolerance      */
} mt_job_result;

typedef struct {
  int64_t submitted, completed, failed, evictions, assemblies, resident;
  size_t bytes_in_use, budget;
} mt_server_stats;

/* Errors: MT_EINVAL (bad options). */
MT_API mt_status mt_server_create(mt_ctx *ctx, const mt_server_opts *opts, mt_server **out);
/* Register a geometry (HOST arrays as for mt_tiles_create, copied); its
 * tensor is assembled when a job first needs it.  Returns its id. */
MT_API mt_status mt_server_add_geometry(mt_server *S, int64_t n, const double *centre, const double *edge,
                                        const double *Ms, const double *Aex, const double *Ku,
                                        const double *axis, const int32_t *nbr, int32_t *geometry_id);
/* Queue a job (copied); returns at once with its id. */
MT_API mt_status mt_server_submit(mt_server *S, const mt_job *job, uint64_t *job_id);
/* Wait up to timeout_s for a job; on MT_OK fills res, (if m_out is not
 * NULL) the final state (HOST, 3n floats) and, for a sweep job, (if
 * sweep_out is not NULL) sweep_out[4 s + q] = <m>_q (q < 3) and the torque
 * (q = 3) at the end of field value s (HOST, 4 n_fields doubles; NaN for
 * values not reached), and forgets the job.  Returns MT_ETIMEOUT if it is
 * not finished yet (it keeps running). */
MT_API mt_status mt_server_wait(mt_server *S, uint64_t job_id, double timeout_s, mt_job_result *res,
                                float *m_out, double *sweep_out);
MT_API mt_status mt_server_get_stats(mt_server *S, mt_server_stats *st);
/* Stops the worker after the device work in flight; unfinished jobs are
 * dropped. */
MT_API void mt_server_destroy(mt_server *S);

#ifdef __cplusplus
}
#endif
#endif /* MT_H */
