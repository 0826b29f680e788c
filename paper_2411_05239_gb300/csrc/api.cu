// C ABI of libzipnn_gpu.so (declarations and contracts in include/zipnn.h).
// Host-side validation, job tables, stream-ordered allocation and launches of
// the encoder (encode.cu) and decoder (decode.cu) kernels.  No call falls back
// to the CPU: every byte of the codec is produced by the kernels.
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "zipnn.h"
#include "host_internal.h"


using namespace zipnn;

// Device error word: bit 0 corrupt container, bit 1 output too small,
// bit 2 a bounded wait gave up.  One per device.
__device__ uint32_t g_zipnn_err;

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_err_ptr[kMaxDevices];

// A caller-chosen error word for this thread's launches (the request server
// gives each batch its own), else the device's.
thread_local uint32_t* t_err_override = nullptr;

uint32_t* err_word() {
  if (t_err_override) return t_err_override;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_err_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_zipnn_err) != cudaSuccess) return nullptr;
    g_err_ptr[dev] = static_cast<uint32_t*>(p);
  }
  return g_err_ptr[dev];
}

// Pinned staging for job tables: the host copy lands in page-locked memory so
// the H2D copy is truly asynchronous (a pageable source would make the call
// wait for the stream to drain).  Regions are reused only after the event
// recorded behind their copy has completed.
class PinnedRing {
 public:
  cudaError_t h2d(void* dst, const void* src, size_t n, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(mu_);
    if (!buf_) {
      if (cudaHostAlloc(reinterpret_cast<void**>(&buf_), kCap, cudaHostAllocPortable) != cudaSuccess) {
        buf_ = nullptr;
        return cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice);
      }
    }
    if (n > kCap / 2) return cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice);
    const size_t need = (n + 255) / 256 * 256;
    if (head_ + need > kCap) {  // wrap: every earlier region must be consumed first
      for (cudaEvent_t ev : events_) {
        cudaEventSynchronize(ev);
        cudaEventDestroy(ev);
      }
      events_.clear();
      head_ = 0;
    }
    uint8_t* stage = buf_ + head_;
    memcpy(stage, src, n);
    head_ += need;
    cudaError_t e = cudaMemcpyAsync(dst, stage, n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev, st);
    events_.push_back(ev);
    return e;
  }

 private:
  static constexpr size_t kCap = 8u << 20;
  std::mutex mu_;
  uint8_t* buf_ = nullptr;
  size_t head_ = 0;
  std::vector<cudaEvent_t> events_;
};
PinnedRing g_ring;

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

zipnn_status check_params(int dtype, size_t nbytes, size_t chunk_bytes, uint32_t lanes) {
  if (dtype < ZIPNN_BF16 || dtype > ZIPNN_U8) return ZIPNN_EINVAL;
  const int es = elem_size(dtype);
  if (nbytes % es) return ZIPNN_EINVAL;
  if (chunk_bytes < ZIPNN_MIN_CHUNK || chunk_bytes > ZIPNN_MAX_CHUNK || chunk_bytes % 16)
    return ZIPNN_EINVAL;
  if (lanes < 1 || lanes > ZIPNN_MAX_LANES || lanes > chunk_bytes / 16) return ZIPNN_EINVAL;
  if ((nbytes + chunk_bytes - 1) / chunk_bytes > 0xFFFFFFFFull) return ZIPNN_EINVAL;
  return ZIPNN_OK;
}

zipnn_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return ZIPNN_OK;
  if (e == cudaErrorMemoryAllocation) return ZIPNN_ENOMEM;
  return ZIPNN_ECUDA;
}

Job make_job(const void* src, const void* base, void* dst, size_t nbytes, int dtype,
             size_t chunk_bytes, uint32_t lanes, uint32_t flags) {
  Job J;
  memset(&J, 0, sizeof(J));
  J.src = static_cast<const uint8_t*>(src);
  J.base = static_cast<const uint8_t*>(base);
  J.dst = static_cast<uint8_t*>(dst);
  J.nbytes = nbytes;
  J.chunk_bytes = (uint32_t)chunk_bytes;
  J.lanes = lanes;
  J.n_chunks = (uint32_t)((nbytes + chunk_bytes - 1) / chunk_bytes);
  J.dtype = dtype;
  J.flags = flags;
  return J;
}

zipnn_status read_header(const uint8_t* h, size_t nbytes, zipnn_stream* out) {
  if (h[0] != 'Z' || h[1] != 'N' || h[2] != 'N' || h[3] != '1') return ZIPNN_ECORRUPT;
  uint32_t ver = h[4] | (h[5] << 8);
  if (ver != 1) return ZIPNN_ECORRUPT;
  int dtype = h[6];
  uint32_t flags = h[7];
  uint64_t orig, P, total;
  uint32_t C, T, G, nch;
  memcpy(&orig, h + 8, 8);
  memcpy(&C, h + 16, 4);
  memcpy(&T, h + 20, 4);
  memcpy(&G, h + 24, 4);
  memcpy(&nch, h + 28, 4);
  memcpy(&P, h + 32, 8);
  memcpy(&total, h + 40, 8);
  if (dtype > ZIPNN_U8 || (flags & ~ZIPNN_FLAG_DELTA)) return ZIPNN_ECORRUPT;
  if (check_params(dtype, orig, C, T) != ZIPNN_OK) return ZIPNN_ECORRUPT;
  if (G != (uint32_t)elem_size(dtype)) return ZIPNN_ECORRUPT;
  if ((uint64_t)nch != (orig + C - 1) / C) return ZIPNN_ECORRUPT;
  if (P != kHdrBytes + (uint64_t)nch * G * kEntryBytes) return ZIPNN_ECORRUPT;
  if (total != nbytes || total < P) return ZIPNN_ECORRUPT;
  for (int k = 48; k < 64; k++)
    if (h[k]) return ZIPNN_ECORRUPT;
  out->nbytes = total;
  out->orig_nbytes = orig;
  out->dtype = dtype;
  out->flags = flags;
  out->chunk_bytes = C;
  out->lanes = T;
  out->n_chunks = nch;
  out->n_groups = G;
  return ZIPNN_OK;
}

zipnn_status check_stream(const zipnn_stream* s) {
  if (!s || !s->data || !aligned16(s->data)) return ZIPNN_EINVAL;
  if (check_params(s->dtype, s->orig_nbytes, s->chunk_bytes, s->lanes) != ZIPNN_OK)
    return ZIPNN_EINVAL;
  if (s->n_groups != (uint32_t)elem_size(s->dtype)) return ZIPNN_EINVAL;
  if ((uint64_t)s->n_chunks != (s->orig_nbytes + s->chunk_bytes - 1) / s->chunk_bytes)
    return ZIPNN_EINVAL;
  if (s->nbytes < kHdrBytes + (uint64_t)s->n_chunks * s->n_groups * kEntryBytes)
    return ZIPNN_EINVAL;
  return ZIPNN_OK;
}

Job decode_job(const zipnn_stream* s, const void* base, void* dst) {
  Job J = make_job(s->data, base, dst, s->orig_nbytes, s->dtype, s->chunk_bytes, s->lanes,
                   s->flags);
  J.stream_bytes = s->nbytes;
  return J;
}

}  // namespace

namespace zipnn {
uint32_t* plan_err_word() { return err_word(); }
void set_thread_err_word(uint32_t* d_err) { t_err_override = d_err; }

uint32_t default_lanes_for(int dtype, size_t chunk_bytes, bool delta) {
  const bool wide = !delta && (dtype == ZIPNN_BF16 || dtype == ZIPNN_FP16);
  uint64_t t = chunk_bytes / (wide ? 512u : 1024u);
  if (t < 1) t = 1;
  if (t > ZIPNN_MAX_LANES) t = ZIPNN_MAX_LANES;
  return (uint32_t)t;
}
}  // namespace zipnn

extern "C" {

int zipnn_version(void) { return 1; }

const char* zipnn_strerror(int status) {
  switch (status) {
    case ZIPNN_OK: return "ok";
    case ZIPNN_EINVAL: return "invalid argument";
    case ZIPNN_ENOMEM: return "out of device memory or buffer too small";
    case ZIPNN_ECORRUPT: return "corrupt container";
    case ZIPNN_ECUDA: return "CUDA runtime error";
    case ZIPNN_ETIMEOUT: return "bounded device wait gave up";
    case ZIPNN_EBUSY: return "memory budget exhausted";
    default: return "unknown status";
  }
}

uint32_t zipnn_default_lanes(int dtype, size_t chunk_bytes) {
  if (dtype < ZIPNN_BF16 || dtype > ZIPNN_U8) return 0;
  return default_lanes_for(dtype, chunk_bytes, false);
}

size_t zipnn_compress_bound(size_t nbytes, int dtype, size_t chunk_bytes) {
  if (dtype < ZIPNN_BF16 || dtype > ZIPNN_U8 || chunk_bytes == 0) return 0;
  const uint64_t G = elem_size(dtype);
  const uint64_t nch = (nbytes + chunk_bytes - 1) / chunk_bytes;
  return kHdrBytes + nch * G * kEntryBytes + nbytes + nch * G * 16;
}

size_t zipnn_compress_workspace_size(size_t nbytes, int dtype, size_t chunk_bytes) {
  if (dtype < ZIPNN_BF16 || dtype > ZIPNN_U8 || chunk_bytes == 0) return 0;
  const uint64_t G = elem_size(dtype);
  const uint64_t nch = (nbytes + chunk_bytes - 1) / chunk_bytes;
  return encode_scratch_bytes(nch, nch * G, 1);
}

zipnn_status zipnn_compress_into(const void* d_src, const void* d_base_or_null, size_t nbytes,
                                 int dtype, size_t chunk_bytes, uint32_t lanes, void* d_out,
                                 size_t out_capacity, void* d_workspace, size_t workspace_bytes,
                                 uint64_t* d_out_nbytes, void* cuda_stream) {
  if (lanes == 0 && dtype >= ZIPNN_BF16 && dtype <= ZIPNN_U8)
    lanes = default_lanes_for(dtype, chunk_bytes, d_base_or_null != nullptr);
  zipnn_status rc = check_params(dtype, nbytes, chunk_bytes, lanes);
  if (rc) return rc;
  if ((nbytes && !d_src) || !d_out || !aligned16(d_src) || !aligned16(d_out) ||
      !aligned16(d_base_or_null))
    return ZIPNN_EINVAL;
  if (out_capacity < zipnn_compress_bound(nbytes, dtype, chunk_bytes)) return ZIPNN_ENOMEM;
  if (!d_workspace || workspace_bytes < zipnn_compress_workspace_size(nbytes, dtype, chunk_bytes))
    return ZIPNN_ENOMEM;
  uint32_t* err = err_word();
  if (!err) return ZIPNN_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  Job J = make_job(d_src, d_base_or_null, d_out, nbytes, dtype, chunk_bytes, lanes,
                   d_base_or_null ? ZIPNN_FLAG_DELTA : 0u);
  J.out_capacity = out_capacity;
  J.out_nbytes = d_out_nbytes;
  const uint64_t ngc = (uint64_t)J.n_chunks * elem_size(dtype);
  EncodeScratch s;
  encode_scratch_carve(d_workspace, J.n_chunks, ngc, 1, &s);
  cudaError_t e = launch_encode(nullptr, &J, 1, J.n_chunks, ngc, s, err, st, 0, (int)lanes, -1,
                                false, 0);
  return cuda_status(e);
}

namespace {
struct BatchPlan {
  std::vector<Job> jobs;
  uint64_t nchunks = 0, ngc = 0;
  int max_lanes = 1;
  int max_groups = 1;
  int uniform = -2;  // common dtype of the batch, -1 if mixed
};

zipnn_status plan_batch_compress(const void* const* d_srcs, const void* const* d_bases,
                                 const size_t* nbytes, const int* dtypes, int count,
                                 size_t chunk_bytes, uint32_t lanes, void* const* d_outs,
                                 const size_t* caps, uint64_t* d_out_nbytes, BatchPlan* bp) {
  if (count <= 0 || !nbytes || !dtypes) return ZIPNN_EINVAL;
  bp->jobs.resize((size_t)count);
  for (int i = 0; i < count; i++) {
    const int dt = dtypes[i];
    const bool dl = d_bases && d_bases[i];
    const uint32_t ln = (lanes == 0 && dt >= ZIPNN_BF16 && dt <= ZIPNN_U8)
                            ? default_lanes_for(dt, chunk_bytes, dl)
                            : lanes;
    zipnn_status rc = check_params(dt, nbytes[i], chunk_bytes, ln);
    if (rc) return rc;
    const void* src = d_srcs ? d_srcs[i] : nullptr;
    const void* base = d_bases ? d_bases[i] : nullptr;
    void* out = d_outs ? d_outs[i] : nullptr;
    const bool query = (d_srcs == nullptr && d_outs == nullptr);  // workspace-size query
    if ((!query && nbytes[i] && !src) || !aligned16(src) || !aligned16(base) || !aligned16(out))
      return ZIPNN_EINVAL;
    if (d_outs) {
      if (!out) return ZIPNN_EINVAL;
      if (!caps || caps[i] < zipnn_compress_bound(nbytes[i], dt, chunk_bytes)) return ZIPNN_ENOMEM;
    }
    Job J = make_job(src, base, out, nbytes[i], dt, chunk_bytes, ln, base ? ZIPNN_FLAG_DELTA : 0u);
    J.out_capacity = caps ? caps[i] : 0;
    J.out_nbytes = d_out_nbytes ? d_out_nbytes + i : nullptr;
    J.chunk_begin = bp->nchunks;
    J.gc_begin = bp->ngc;
    bp->nchunks += J.n_chunks;
    bp->ngc += (uint64_t)J.n_chunks * elem_size(dt);
    if ((int)ln > bp->max_lanes) bp->max_lanes = (int)ln;
    if (elem_size(dt) > bp->max_groups) bp->max_groups = elem_size(dt);
    bp->uniform = (bp->uniform == -2 || bp->uniform == dt) ? dt : -1;
    bp->jobs[i] = J;
  }
  return ZIPNN_OK;
}

size_t batch_ws_bytes(const BatchPlan& bp) {
  return align_up(sizeof(Job) * bp.jobs.size(), 256) +
         encode_scratch_bytes(bp.nchunks, bp.ngc, (int)bp.jobs.size());
}
}  // namespace

extern "C" size_t zipnn_batch_compress_workspace_size(const size_t* nbytes, const int* dtypes,
                                                      int count, size_t chunk_bytes) {
  BatchPlan bp;
  if (plan_batch_compress(nullptr, nullptr, nbytes, dtypes, count, chunk_bytes, 0, nullptr,
                          nullptr, nullptr, &bp) != ZIPNN_OK)
    return 0;
  return batch_ws_bytes(bp);
}

extern "C" zipnn_status zipnn_batch_compress_into_ex(
    const void* const* d_srcs, const void* const* d_bases, const size_t* nbytes,
    const int* dtypes, int count, size_t chunk_bytes, const zipnn_encode_options* opts,
    void* const* d_outs, const size_t* out_capacities, void* d_workspace,
    size_t workspace_bytes, uint64_t* d_out_nbytes, void* cuda_stream) {
  if (!d_outs) return ZIPNN_EINVAL;
  const uint32_t lanes = opts ? opts->lanes : 0u;
  const uint32_t skip = opts ? opts->probe_skip : 0u;
  const uint32_t encoder = opts ? opts->encoder : 0u;
  const uint32_t dbg = opts ? opts->debug_flags : 0u;
  if (encoder > 1 || (dbg & ~1u)) return ZIPNN_EINVAL;
  BatchPlan bp;
  zipnn_status rc = plan_batch_compress(d_srcs, d_bases, nbytes, dtypes, count, chunk_bytes,
                                        lanes, d_outs, out_capacities, d_out_nbytes, &bp);
  if (rc) return rc;
  for (Job& J : bp.jobs) J.skip = skip;
  if (!d_workspace || workspace_bytes < batch_ws_bytes(bp)) return ZIPNN_ENOMEM;
  uint32_t* err = err_word();
  if (!err) return ZIPNN_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  uint8_t* ws = static_cast<uint8_t*>(d_workspace);
  Job* d_jobs = reinterpret_cast<Job*>(ws);
  ws += align_up(sizeof(Job) * bp.jobs.size(), 256);
  EncodeScratch s;
  encode_scratch_carve(ws, bp.nchunks, bp.ngc, count, &s);
  cudaError_t e = g_ring.h2d(d_jobs, bp.jobs.data(), sizeof(Job) * bp.jobs.size(), st);
  if (e == cudaSuccess)
    e = launch_encode(d_jobs, nullptr, count, bp.nchunks, bp.ngc, s, err, st, bp.max_groups,
                      bp.max_lanes, bp.uniform, skip != 0, (int)encoder, dbg,
                      any_base(d_bases, count));
  return cuda_status(e);
}

extern "C" zipnn_status zipnn_batch_compress_into(
    const void* const* d_srcs, const void* const* d_bases, const size_t* nbytes,
    const int* dtypes, int count, size_t chunk_bytes, uint32_t lanes, void* const* d_outs,
    const size_t* out_capacities, void* d_workspace, size_t workspace_bytes,
    uint64_t* d_out_nbytes, void* cuda_stream) {
  zipnn_encode_options o;
  memset(&o, 0, sizeof(o));
  o.lanes = lanes;
  return zipnn_batch_compress_into_ex(d_srcs, d_bases, nbytes, dtypes, count, chunk_bytes, &o,
                                      d_outs, out_capacities, d_workspace, workspace_bytes,
                                      d_out_nbytes, cuda_stream);
}

static zipnn_status compress_alloc(const void* d_src, const void* d_base, size_t nbytes, int dtype,
                                   size_t chunk_bytes, zipnn_stream* out, void* cuda_stream) {
  if (!out) return ZIPNN_EINVAL;
  memset(out, 0, sizeof(*out));
  const uint32_t lanes = (dtype >= ZIPNN_BF16 && dtype <= ZIPNN_U8)
                             ? default_lanes_for(dtype, chunk_bytes, d_base != nullptr)
                             : 0;
  zipnn_status rc = check_params(dtype, nbytes, chunk_bytes, lanes);
  if (rc) return rc;
  if ((nbytes && !d_src) || !aligned16(d_src) || !aligned16(d_base)) return ZIPNN_EINVAL;
  uint32_t* err = err_word();
  if (!err) return ZIPNN_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  Job J = make_job(d_src, d_base, nullptr, nbytes, dtype, chunk_bytes, lanes,
                   d_base ? ZIPNN_FLAG_DELTA : 0u);
  const uint64_t ngc = (uint64_t)J.n_chunks * elem_size(dtype);
  const size_t ws = encode_scratch_bytes(J.n_chunks, ngc, 1);
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, ws, st);
  if (e != cudaSuccess) return cuda_status(e);
  EncodeScratch s;
  encode_scratch_carve(scratch, J.n_chunks, ngc, 1, &s);
  e = launch_encode_analyse_ex(nullptr, &J, 1, J.n_chunks, ngc, s, err, st, 0, -1);
  uint64_t total = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, s.totals, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  void* buf = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(&buf, total ? total : 16, st);
  if (e == cudaSuccess) {
    J.dst = static_cast<uint8_t*>(buf);
    J.out_capacity = total;
    e = launch_encode_pack_ex(nullptr, &J, 1, J.n_chunks, (int)lanes, s, st, -1);
  }
  cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) {
    if (buf) cudaFreeAsync(buf, st);
    return cuda_status(e);
  }
  out->data = buf;
  out->nbytes = total;
  out->orig_nbytes = nbytes;
  out->dtype = dtype;
  out->flags = J.flags;
  out->chunk_bytes = (uint32_t)chunk_bytes;
  out->lanes = lanes;
  out->n_chunks = J.n_chunks;
  out->n_groups = (uint32_t)elem_size(dtype);
  out->owned = 1;
  return ZIPNN_OK;
}

zipnn_status zipnn_compress(const void* d_src, size_t nbytes, int dtype, size_t chunk_bytes,
                            zipnn_stream* out, void* cuda_stream) {
  return compress_alloc(d_src, nullptr, nbytes, dtype, chunk_bytes, out, cuda_stream);
}

zipnn_status zipnn_delta(const void* d_a, const void* d_b, size_t nbytes, int dtype,
                         size_t chunk_bytes, zipnn_stream* out, void* cuda_stream) {
  if (!d_b && nbytes) return ZIPNN_EINVAL;
  if (!d_b) {
    // empty delta: still a DELTA container
    zipnn_status rc = compress_alloc(d_a, nullptr, 0, dtype, chunk_bytes, out, cuda_stream);
    return rc;
  }
  return compress_alloc(d_a, d_b, nbytes, dtype, chunk_bytes, out, cuda_stream);
}

zipnn_status zipnn_stream_wrap(const void* d_data, size_t nbytes, zipnn_stream* out) {
  if (!out || !d_data || !aligned16(d_data) || nbytes < (size_t)kHdrBytes) return ZIPNN_EINVAL;
  memset(out, 0, sizeof(*out));
  uint8_t h[kHdrBytes];
  cudaError_t e = cudaMemcpy(h, d_data, kHdrBytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  zipnn_status rc = read_header(h, nbytes, out);
  if (rc) return rc;
  out->data = const_cast<void*>(d_data);
  out->owned = 0;
  return ZIPNN_OK;
}

zipnn_status zipnn_decompressed_size(const zipnn_stream* s, size_t* nbytes, int* dtype) {
  if (!s) return ZIPNN_EINVAL;
  if (nbytes) *nbytes = s->orig_nbytes;
  if (dtype) *dtype = s->dtype;
  return ZIPNN_OK;
}

zipnn_status zipnn_decompress(const zipnn_stream* s, const void* d_base_or_null, void* d_dst,
                              size_t dst_nbytes, void* cuda_stream) {
  zipnn_status rc = check_stream(s);
  if (rc) return rc;
  if (dst_nbytes != s->orig_nbytes) return ZIPNN_EINVAL;
  if (((s->flags & ZIPNN_FLAG_DELTA) != 0) != (d_base_or_null != nullptr)) return ZIPNN_EINVAL;
  if ((dst_nbytes && !d_dst) || !aligned16(d_dst) || !aligned16(d_base_or_null)) return ZIPNN_EINVAL;
  uint32_t* err = err_word();
  if (!err) return ZIPNN_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  Job J = decode_job(s, d_base_or_null, d_dst);
  cudaError_t e = launch_decode_ex(nullptr, &J, 1, J.n_chunks, (int)s->n_groups, nullptr, err,
                                   nullptr, st, s->dtype, s->chunk_bytes, s->lanes % 256 == 0,
                                   stage_frac64(s->dtype, s->flags),
                                   (s->flags & ZIPNN_FLAG_DELTA) != 0, false, 0u, s->lanes);
  return cuda_status(e);
}

zipnn_status zipnn_batch_decompress(const zipnn_stream* streams, const void* const* d_bases,
                                    void* const* d_dsts, int count, const zipnn_tuning* tuning,
                                    void* cuda_stream) {
  if (count < 0 || (count > 0 && (!streams || !d_dsts))) return ZIPNN_EINVAL;
  if (count == 0) return ZIPNN_OK;
  std::vector<Job> jobs((size_t)count);
  uint64_t chunk = 0, max_chunk = 0;
  int max_groups = 1;
  int uniform = streams[0].dtype;
  bool lanes256 = true, has_delta = false;
  int frac64 = 0;
  uint32_t common_lanes = streams[0].lanes;
  for (int i = 0; i < count; i++) {
    const zipnn_stream* s = &streams[i];
    if (s->lanes != common_lanes) common_lanes = 0;
    if (s->flags & ZIPNN_FLAG_DELTA) has_delta = true;
    if (s->dtype != uniform) uniform = -1;
    if (s->chunk_bytes > max_chunk) max_chunk = s->chunk_bytes;
    if (s->lanes % 256) lanes256 = false;
    if (stage_frac64(s->dtype, s->flags) > frac64) frac64 = stage_frac64(s->dtype, s->flags);
    zipnn_status rc = check_stream(s);
    if (rc) return rc;
    const void* base = d_bases ? d_bases[i] : nullptr;
    if (((s->flags & ZIPNN_FLAG_DELTA) != 0) != (base != nullptr)) return ZIPNN_EINVAL;
    if ((s->orig_nbytes && !d_dsts[i]) || !aligned16(d_dsts[i]) || !aligned16(base))
      return ZIPNN_EINVAL;
    jobs[i] = decode_job(s, base, d_dsts[i]);
    jobs[i].chunk_begin = chunk;
    chunk += jobs[i].n_chunks;
    if ((int)s->n_groups > max_groups) max_groups = (int)s->n_groups;
  }
  uint32_t* err = err_word();
  if (!err) return ZIPNN_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  void* dmem = nullptr;
  const size_t tbytes = sizeof(Job) * (size_t)count;
  cudaError_t e = cudaMallocAsync(&dmem, tbytes + 16, st);
  if (e != cudaSuccess) return cuda_status(e);
  Job* d_jobs = static_cast<Job*>(dmem);
  unsigned long long* d_ticket = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(dmem) + tbytes);
  // the job table and the two zeroed work-queue counters after it, in one copy
  std::vector<uint8_t> up(tbytes + 16, 0);
  memcpy(up.data(), jobs.data(), tbytes);
  e = g_ring.h2d(d_jobs, up.data(), up.size(), st);
  if (e == cudaSuccess)
    e = launch_decode_ex(d_jobs, nullptr, count, chunk, max_groups, tuning, err, d_ticket, st,
                         uniform, max_chunk, lanes256, frac64, has_delta, false, 0u,
                         common_lanes);
  cudaFreeAsync(dmem, st);
  return cuda_status(e);
}

zipnn_status zipnn_sync_status(void* cuda_stream) {
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ZIPNN_ECUDA;
  uint32_t* err = err_word();
  if (!err) return ZIPNN_ECUDA;
  uint32_t v = 0;
  e = cudaMemcpy(&v, err, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return ZIPNN_ECUDA;
  if (v) {
    uint32_t z = 0;
    cudaMemcpy(err, &z, 4, cudaMemcpyHostToDevice);
  }
  if (v & 1u) return ZIPNN_ECORRUPT;
  if (v & 2u) return ZIPNN_ENOMEM;
  if (v & 4u) return ZIPNN_ETIMEOUT;
  e = cudaGetLastError();
  return e == cudaSuccess ? ZIPNN_OK : ZIPNN_ECUDA;
}

void zipnn_stream_free(zipnn_stream* s) {
  if (!s) return;
  if (s->owned && s->data) cudaFree(s->data);
  memset(s, 0, sizeof(*s));
}

}  // extern "C"
