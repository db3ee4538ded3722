// Demag product with library-owned, statically allocated scratch.
//
// mt_demag_field needs three small work areas besides its inputs and
// outputs: the Ms-scaled, padded copy of m that the streaming kernel reads,
// the partial row sums of panels shared by two CTAs, and one arrival counter
// per panel.  It allocates them with cudaMalloc on first use.  Some callers
// cannot let a library allocate: a control or serving loop that has handed
// all free HBM to cached tensors and must not fail half-way through a step,
// code that runs next to latency-critical streams and cannot afford the
// device-wide synchronisation cudaMalloc/cudaFree may cause, or an
// application that owns all device memory through its own pool and forbids
// the CUDA allocator.  mt_demag_field_noalloc serves them: the work areas live
// in one fixed array in the library's device image (MT_NOALLOC_SCRATCH_BYTES
// per GPU that loads the library, held until the process exits), and the call
// performs no allocation of any kind.
#include <mutex>

#include "mt_internal.cuh"

namespace {

// The shared work area.  In host code this name is only a stand-in for the
// device object: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Resolve the scratch address once per device (that device must be current).
mt_status scratch_for_device(int dev, unsigned char **out) {
  MT_CHECK(dev >= 0 && dev < kMaxDevices, MT_EINVAL, "mt_demag_field_noalloc: device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return mt::cuda_fail(e, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
    MT_CHECK(p != nullptr, MT_ECUDA, "mt_demag_field_noalloc: scratch address unavailable");
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_scratch_ptr[dev]);
  return MT_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" mt_status mt_demag_field_noalloc(mt_tensor *T, const float *m, int B, float *H, void *stream) {
  MT_CHECK(T && m && H, MT_EINVAL, "mt_demag_field_noalloc: NULL argument");
  MT_CHECK(B >= 1, MT_EINVAL, "mt_demag_field_noalloc: B must be >= 1");
  MT_CHECK(T->prec != MT_F64, MT_EINVAL, "mt_demag_field_noalloc: FP64 tensors are not supported");
  MT_CHECK(T->layout == MT_LAYOUT_STREAM, MT_EINVAL,
           "mt_demag_field_noalloc: only streaming-layout tensors are supported");
  MT_CHECK(!T->L.half, MT_EINVAL,
           "mt_demag_field_noalloc: a half-stored tensor needs a column work area of 1.5 KB per stored chunk; "
           "assemble with MT_LAYOUT_STREAM_FULL or use mt_demag_field");
  const size_t count_bytes = align256(mt::matvec_count_bytes(T, B));
  const size_t part_bytes = align256(mt::matvec_part_bytes(T));
  const size_t xs_bytes = align256(sizeof(float) * (size_t)mt::xs_floats(T) * (size_t)B);
  const size_t need = count_bytes + part_bytes + xs_bytes;
  MT_CHECK(need <= (size_t)MT_NOALLOC_SCRATCH_BYTES, MT_EINVAL,
           "mt_demag_field_noalloc: n = %lld with B = %d needs %zu bytes of scratch, more than the fixed "
           "%zu (MT_NOALLOC_SCRATCH_BYTES); use mt_demag_field",
           (long long)T->n, B, need, (size_t)MT_NOALLOC_SCRATCH_BYTES);
  const int dev = T->tiles->ctx->device;
  MT_CUDA(cudaSetDevice(dev));
  unsigned char *base = nullptr;
  mt_status st = scratch_for_device(dev, &base);
  if (st != MT_OK) return st;
  int *count = reinterpret_cast<int *>(base);
  float *part = reinterpret_cast<float *>(base + count_bytes);
  float *xs = reinterpret_cast<float *>(base + count_bytes + part_bytes);
  cudaStream_t s = (cudaStream_t)stream;
  // the panel counters must start at zero; the previous call may have left
  // anything there.  xs is fully rewritten (padding included) and every
  // partial is written before it is read.
  MT_CUDA(cudaMemsetAsync(count, 0, count_bytes, s));
  mt::launch_prep_xs(T, m, B, xs, s);
  mt::launch_matvec(T, xs, B, H, part, count, nullptr, T->tiles->ctx->d_status, s);
  mt::launch_near(T, m, 3 * T->n, 1, B, H, nullptr, s);
  MT_CUDA(cudaGetLastError());
  return MT_OK;
}
