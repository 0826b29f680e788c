// zipnn_compress_into_static: compression that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they compress:
// a plugin that only receives device pointers from a host framework and has no
// handle on that framework's caching allocator (a cudaMalloc of its own would
// bypass the framework's memory accounting), a latency-critical loop where a
// cudaMalloc or cudaFree may synchronise the whole device at the wrong time, or
// a process whose device memory budget is fixed at start-up.  For them this
// entry point runs the same encoder kernels as zipnn_compress_into, but takes
// its scratch (histograms, code tables, map offsets) from a fixed array that
// lives in this file, instead of from a caller-provided workspace.
//
// Costs and rules of the fixed array:
//   - every GPU that loads the library holds kStaticScratchBytes (8 MiB) of it
//     until the process exits;
//   - one call may use at most that much scratch: 2,348 bytes per (chunk,
//     byte group) pair (1 KiB histogram, 1 KiB code table, 272 B table bytes,
//     16 B mode record, 8 B offset, 4 B zero count), each array rounded up to
//     256 B, plus 512 B -- at most 3,572 pairs, e.g. 446.5 MiB of BF16/FP16 or
//     223.25 MiB of FP32 at 256 KiB chunks; larger inputs are rejected with
//     ZIPNN_ENOMEM before anything is launched (the check calls the same
//     sizing function as the workspace entry point, so the figure cannot
//     drift from the layout);
//   - all calls on a device share the array and it keeps the last call's
//     contents.  Nothing in it has to start at zero: every scratch word a call
//     reads was written earlier by the same call (it runs the four-kernel
//     encoder).  Two calls whose kernels
//     overlap on the GPU (e.g. on two streams without ordering) race on the
//     array and produce garbage: order them on one stream or with events;
//   - the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (once per device, with that device current); make
//     that first call before any stream capture begins.
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "zipnn.h"
#include "host_internal.h"


using namespace zipnn;

namespace {

constexpr size_t kStaticScratchBytes = 8u << 20;
constexpr int kMaxStaticDevices = 64;

// The fixed scratch.  In host code this name is only a stand-in for the
// symbol; the kernels receive the device address looked up below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_ptr[kMaxStaticDevices];

// Device address of g_static_scratch on the current device (looked up once).
cudaError_t static_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxStaticDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" zipnn_status zipnn_compress_into_static(const void* d_src, const void* d_base_or_null,
                                                   size_t nbytes, int dtype, size_t chunk_bytes,
                                                   uint32_t lanes, void* d_out,
                                                   size_t out_capacity, uint64_t* d_out_nbytes,
                                                   void* cuda_stream) {
  if (dtype < ZIPNN_BF16 || dtype > ZIPNN_U8) return ZIPNN_EINVAL;
  if (lanes == 0) lanes = zipnn::default_lanes_for(dtype, chunk_bytes, d_base_or_null != nullptr);
  const int es = elem_size(dtype);
  if (nbytes % es || chunk_bytes < ZIPNN_MIN_CHUNK || chunk_bytes > ZIPNN_MAX_CHUNK ||
      chunk_bytes % 16 || lanes < 1 || lanes > ZIPNN_MAX_LANES || lanes > chunk_bytes / 16)
    return ZIPNN_EINVAL;
  if ((nbytes && !d_src) || !d_out || !aligned16(d_src) || !aligned16(d_out) ||
      !aligned16(d_base_or_null))
    return ZIPNN_EINVAL;
  if (out_capacity < zipnn_compress_bound(nbytes, dtype, chunk_bytes)) return ZIPNN_ENOMEM;
  const uint64_t nch = (nbytes + chunk_bytes - 1) / chunk_bytes;
  const uint64_t ngc = nch * (uint64_t)es;
  if (encode_scratch_bytes(nch, ngc, 1) > kStaticScratchBytes) return ZIPNN_ENOMEM;

  void* scratch = nullptr;
  cudaError_t e = static_scratch(&scratch);
  if (e != cudaSuccess) return ZIPNN_ECUDA;
  uint32_t* err = plan_err_word();
  if (!err) return ZIPNN_ECUDA;

  Job J;
  memset(&J, 0, sizeof(J));
  J.src = static_cast<const uint8_t*>(d_src);
  J.base = static_cast<const uint8_t*>(d_base_or_null);
  J.dst = static_cast<uint8_t*>(d_out);
  J.nbytes = nbytes;
  J.chunk_bytes = (uint32_t)chunk_bytes;
  J.lanes = lanes;
  J.n_chunks = (uint32_t)nch;
  J.dtype = dtype;
  J.flags = d_base_or_null ? ZIPNN_FLAG_DELTA : 0u;
  J.out_capacity = out_capacity;
  J.out_nbytes = d_out_nbytes;
  EncodeScratch s;
  encode_scratch_carve(scratch, nch, ngc, 1, &s);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  e = launch_encode(nullptr, &J, 1, nch, ngc, s, err, st, 0, (int)lanes, -1, false, 0);
  return e == cudaSuccess ? ZIPNN_OK : ZIPNN_ECUDA;
}
