// Plans: a batch of tensors prepared once (device job table, scratch, work
// ticket) and captured as a CUDA graph, so that every later batched
// compression or persistent-kernel decompression of the same tensors costs one
// cudaGraphLaunch.  This is the batching form of the codec: many tensors of
// uneven sizes in one launch per kernel (ZipNN Sec. 5.1: chunks and byte groups
// are independent, so one grid serves them all).
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "zipnn.h"
#include "host_internal.h"


using namespace zipnn;

struct zipnn_plan {
  int kind = 0;                 // 1 = decompress, 2 = compress, 3 = load
  int device = 0;
  void* dmem = nullptr;         // job table + ticket + scratch
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t nchunks = 0;
  int count = 0;
};

namespace {

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// What a decode launch needs, read from its containers' chunk maps: per chunk
// the shared-memory stage that holds its coded (HUFF / SPARSE) payloads, 16-B
// padded, plus 32 B and the table of every coded group after the first (the
// decoder's staging rule), and whether a chunk takes the general fast loops
// (two coded groups, or a SPARSE first group).
struct MapNeed {
  uint64_t max_stage = 0;  // largest per-chunk need
  uint64_t chunks = 0;     // chunks seen
  uint64_t over = 0;       // chunks whose need exceeds the default stage
  bool general = false;
};

void add_map_need(const uint8_t* map, uint32_t n_chunks, uint32_t G, int w, uint64_t dflt,
                  MapNeed* nd) {
  for (uint32_t c = 0; c < n_chunks; c++) {
    uint64_t used = 0;
    uint32_t ncoded = 0;
    bool sparse0 = false;
    for (uint32_t g = 0; g < G; g++) {
      const uint8_t* e = map + ((uint64_t)c * G + g) * kEntryBytes;
      uint32_t size;
      memcpy(&size, e + 8, 4);
      const uint32_t mode = e[12];
      if (mode == kHuff || mode == kSparse) {
        used += align_up(size, 16);
        ncoded++;
        if (g == 0 && mode == kSparse) sparse0 = true;
      }
    }
    nd->chunks++;
    if (ncoded) {
      const uint64_t need = used + 32 + (uint64_t)(ncoded - 1) * (4u << w);
      if (need > nd->max_stage) nd->max_stage = need;
      if (need > dflt) nd->over++;
    }
    if (ncoded >= 2 || sparse0) nd->general = true;
  }
}

// The stage a plan asks for: 0 (the launcher's default rule) while the default
// stage holds the payloads of at least 99% of the chunks, else the largest
// need (which may leave one CTA per SM: the only way to stage such chunks).
uint32_t planned_stage(const MapNeed& nd) {
  if (nd.over * 100 <= nd.chunks) return 0;
  return (uint32_t)(nd.max_stage > 0xFFFFFFFFull ? 0xFFFFFFFFull : nd.max_stage);
}

int plan_lut_bits(const zipnn_tuning* tuning) {
  int w = (tuning && tuning->lut_bits) ? tuning->lut_bits : 12;
  return w < 10 ? 10 : (w > 12 ? 12 : w);
}

zipnn_status fail(zipnn_plan* p, cudaError_t e) {
  if (p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->dmem) cudaFree(p->dmem);
    delete p;
  }
  return e == cudaErrorMemoryAllocation ? ZIPNN_ENOMEM : ZIPNN_ECUDA;
}

// Capture `body` on a private stream into p->graph / p->exec.
template <class F>
cudaError_t capture(zipnn_plan* p, F body) {
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t eb = body(cs);
    e = cudaStreamEndCapture(cs, &p->graph);
    if (eb != cudaSuccess) e = eb;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  cudaStreamDestroy(cs);
  return e;
}

}  // namespace

extern "C" {

// Decode plan over the global chunk range [lo, hi) of the containers taken in
// order as one sequence (all of it for zipnn_plan_decompress; a rank's share
// for zipnn_plan_decompress_range).  A container whose chunks fall partly in
// the range becomes a job over those chunks only (Job.chunk0), and its
// destination (and base) pointer is shifted so that the kernel's
// dst + chunk * chunk_bytes lands in the caller's buffer of the range.
static zipnn_status plan_decode_range(const zipnn_stream* streams, const void* const* d_bases,
                                      void* const* d_dsts, int count, uint64_t lo, uint64_t hi,
                                      const zipnn_tuning* tuning, zipnn_plan** out) {
  if (!out || count <= 0 || !streams || !d_dsts || lo > hi) return ZIPNN_EINVAL;
  *out = nullptr;
  std::vector<Job> jobs;
  std::vector<const zipnn_stream*> used;
  uint64_t chunk = 0, max_chunk = 0, g = 0;
  int max_groups = 1;
  int uniform = -2;
  bool lanes256 = true, has_delta = false;
  int frac64 = 0;
  for (int i = 0; i < count; i++) {
    const zipnn_stream* s = &streams[i];
    if (s->n_groups != (uint32_t)elem_size(s->dtype) || s->dtype < 0 || s->dtype > ZIPNN_U8 ||
        s->lanes < 1 || s->lanes > ZIPNN_MAX_LANES || s->chunk_bytes < ZIPNN_MIN_CHUNK ||
        (uint64_t)s->n_chunks != (s->orig_nbytes + s->chunk_bytes - 1) / s->chunk_bytes)
      return ZIPNN_EINVAL;
    const uint64_t a = lo > g ? lo - g : 0;
    const uint64_t b = hi < g + s->n_chunks ? (hi > g ? hi - g : 0) : s->n_chunks;
    g += s->n_chunks;
    if (a >= b) continue;  // no chunk of this container in the range
    if (!s->data || !aligned16(s->data)) return ZIPNN_EINVAL;
    const void* base = d_bases ? d_bases[i] : nullptr;
    if (((s->flags & ZIPNN_FLAG_DELTA) != 0) != (base != nullptr)) return ZIPNN_EINVAL;
    if (!d_dsts[i] || !aligned16(d_dsts[i]) || !aligned16(base)) return ZIPNN_EINVAL;
    if (s->flags & ZIPNN_FLAG_DELTA) has_delta = true;
    uniform = (uniform == -2 || uniform == s->dtype) ? s->dtype : -1;
    if (s->chunk_bytes > max_chunk) max_chunk = s->chunk_bytes;
    if (s->lanes % 256) lanes256 = false;
    if (stage_frac64(s->dtype, s->flags) > frac64) frac64 = stage_frac64(s->dtype, s->flags);
    const uintptr_t shift = (uintptr_t)(a * s->chunk_bytes);
    Job J;
    memset(&J, 0, sizeof(J));
    J.src = static_cast<const uint8_t*>(s->data);
    J.base = base ? reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(base) - shift)
                  : nullptr;
    J.dst = reinterpret_cast<uint8_t*>(reinterpret_cast<uintptr_t>(d_dsts[i]) - shift);
    J.nbytes = s->orig_nbytes;
    J.chunk_bytes = s->chunk_bytes;
    J.lanes = s->lanes;
    J.n_chunks = s->n_chunks;
    J.dtype = s->dtype;
    J.flags = s->flags;
    J.stream_bytes = s->nbytes;
    J.chunk_begin = chunk;
    J.chunk0 = (uint32_t)a;
    chunk += b - a;
    if ((int)s->n_groups > max_groups) max_groups = (int)s->n_groups;
    jobs.push_back(J);
    used.push_back(s);
  }
  if (hi > g) return ZIPNN_EINVAL;
  if (jobs.empty()) return ZIPNN_EINVAL;  // nothing to decode in the range
  const int njobs = (int)jobs.size();
  // stage and kernel variant from the chunk maps present now
  MapNeed nd;
  {
    const int w = plan_lut_bits(tuning);
    const uint64_t dflt = max_chunk * (uint64_t)frac64 / 64 + 1024;
    std::vector<uint8_t> mb;
    for (int k = 0; k < njobs; k++) {
      const zipnn_stream* s = used[(size_t)k];
      const uint64_t mbytes = (uint64_t)s->n_chunks * s->n_groups * kEntryBytes;
      if (s->nbytes < kHdrBytes + mbytes) continue;  // malformed: the decoder reports it
      mb.resize((size_t)mbytes);
      if (mbytes && cudaMemcpy(mb.data(), static_cast<const uint8_t*>(s->data) + kHdrBytes,
                               (size_t)mbytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return ZIPNN_ECUDA;
      const Job& J = jobs[(size_t)k];
      const uint64_t n = k + 1 < njobs ? jobs[(size_t)k + 1].chunk_begin - J.chunk_begin
                                       : chunk - J.chunk_begin;
      add_map_need(mb.data() + (uint64_t)J.chunk0 * s->n_groups * kEntryBytes, (uint32_t)n,
                   s->n_groups, w, dflt, &nd);
    }
  }
  uint32_t* err = plan_err_word();
  if (!err) return ZIPNN_ECUDA;
  zipnn_plan* p = new zipnn_plan();
  p->kind = 1;
  p->count = njobs;
  p->nchunks = chunk;
  cudaGetDevice(&p->device);
  const size_t tbytes = align_up(sizeof(Job) * (size_t)njobs, 256);
  cudaError_t e = cudaMalloc(&p->dmem, tbytes + 256);
  if (e != cudaSuccess) return fail(p, e);
  Job* d_jobs = static_cast<Job*>(p->dmem);
  auto* ticket = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(p->dmem) + tbytes);
  e = cudaMemcpy(d_jobs, jobs.data(), sizeof(Job) * (size_t)njobs, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(ticket, 0, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) return fail(p, e);
  zipnn_tuning tu;
  memset(&tu, 0, sizeof(tu));
  if (tuning) tu = *tuning;
  const int uni = uniform < 0 ? -1 : uniform;
  uint32_t common_lanes = jobs[0].lanes;
  for (const Job& J : jobs)
    if (J.lanes != common_lanes) common_lanes = 0;
  e = capture(p, [&](cudaStream_t cs) {
    return launch_decode_ex(d_jobs, nullptr, njobs, chunk, max_groups, &tu, err, ticket, cs, uni,
                            max_chunk, lanes256, frac64, has_delta, nd.general,
                            planned_stage(nd), common_lanes);
  });
  if (e != cudaSuccess) return fail(p, e);
  *out = p;
  return ZIPNN_OK;
}

zipnn_status zipnn_plan_decompress(const zipnn_stream* streams, const void* const* d_bases,
                                   void* const* d_dsts, int count, const zipnn_tuning* tuning,
                                   zipnn_plan** out) {
  if (!out || count <= 0 || !streams || !d_dsts) return ZIPNN_EINVAL;
  uint64_t total = 0;
  for (int i = 0; i < count; i++) {
    total += streams[i].n_chunks;
    // every container decodes in full: its destination must be given (an
    // empty tensor has no chunks and needs none)
    if (streams[i].orig_nbytes && !d_dsts[i]) return ZIPNN_EINVAL;
  }
  if (total == 0) {
    // only empty containers: a plan whose launch does nothing
    zipnn_plan* p = new zipnn_plan();
    p->kind = 1;
    cudaGetDevice(&p->device);
    cudaError_t e = capture(p, [&](cudaStream_t) { return cudaSuccess; });
    if (e != cudaSuccess) return fail(p, e);
    *out = p;
    return ZIPNN_OK;
  }
  return plan_decode_range(streams, d_bases, d_dsts, count, 0, total, tuning, out);
}

zipnn_status zipnn_plan_decompress_range(const zipnn_stream* streams, const void* const* d_bases,
                                         void* const* d_dsts, int count, uint64_t chunk_lo,
                                         uint64_t chunk_hi, const zipnn_tuning* tuning,
                                         zipnn_plan** out) {
  return plan_decode_range(streams, d_bases, d_dsts, count, chunk_lo, chunk_hi, tuning, out);
}

zipnn_status zipnn_plan_compress(const void* const* d_srcs, const void* const* d_bases,
                                 const size_t* nbytes, const int* dtypes, int count,
                                 size_t chunk_bytes, uint32_t lanes, void* const* d_outs,
                                 const size_t* out_capacities, uint64_t* d_out_nbytes,
                                 zipnn_plan** out) {
  if (!out || count <= 0 || !nbytes || !dtypes || !d_outs || !out_capacities) return ZIPNN_EINVAL;
  *out = nullptr;
  std::vector<Job> jobs((size_t)count);
  uint64_t nch = 0, ngc = 0;
  int max_lanes = 1, max_groups = 1, uniform = dtypes[0];
  for (int i = 0; i < count; i++) {
    const int dt = dtypes[i];
    if (dt != uniform) uniform = -1;
    if (dt < ZIPNN_BF16 || dt > ZIPNN_U8) return ZIPNN_EINVAL;
    const uint32_t ln =
        lanes ? lanes : default_lanes_for(dt, chunk_bytes, d_bases && d_bases[i]);
    const int es = elem_size(dt);
    if (nbytes[i] % es || chunk_bytes < ZIPNN_MIN_CHUNK || chunk_bytes > ZIPNN_MAX_CHUNK ||
        chunk_bytes % 16 || ln < 1 || ln > ZIPNN_MAX_LANES || ln > chunk_bytes / 16)
      return ZIPNN_EINVAL;
    const void* src = d_srcs ? d_srcs[i] : nullptr;
    const void* base = d_bases ? d_bases[i] : nullptr;
    if ((nbytes[i] && !src) || !d_outs[i] || !aligned16(src) || !aligned16(base) ||
        !aligned16(d_outs[i]))
      return ZIPNN_EINVAL;
    if (out_capacities[i] < zipnn_compress_bound(nbytes[i], dt, chunk_bytes)) return ZIPNN_ENOMEM;
    Job J;
    memset(&J, 0, sizeof(J));
    J.src = static_cast<const uint8_t*>(src);
    J.base = static_cast<const uint8_t*>(base);
    J.dst = static_cast<uint8_t*>(d_outs[i]);
    J.nbytes = nbytes[i];
    J.chunk_bytes = (uint32_t)chunk_bytes;
    J.lanes = ln;
    J.n_chunks = (uint32_t)((nbytes[i] + chunk_bytes - 1) / chunk_bytes);
    J.dtype = dt;
    J.flags = base ? ZIPNN_FLAG_DELTA : 0u;
    J.out_capacity = out_capacities[i];
    J.out_nbytes = d_out_nbytes ? d_out_nbytes + i : nullptr;
    J.chunk_begin = nch;
    J.gc_begin = ngc;
    nch += J.n_chunks;
    ngc += (uint64_t)J.n_chunks * es;
    if ((int)ln > max_lanes) max_lanes = (int)ln;
    if (es > max_groups) max_groups = es;
    jobs[i] = J;
  }
  uint32_t* err = plan_err_word();
  if (!err) return ZIPNN_ECUDA;
  zipnn_plan* p = new zipnn_plan();
  p->kind = 2;
  p->count = count;
  p->nchunks = nch;
  cudaGetDevice(&p->device);
  const size_t tbytes = align_up(sizeof(Job) * (size_t)count, 256);
  const size_t sbytes = encode_scratch_bytes(nch, ngc, count);
  cudaError_t e = cudaMalloc(&p->dmem, tbytes + sbytes);
  if (e != cudaSuccess) return fail(p, e);
  Job* d_jobs = static_cast<Job*>(p->dmem);
  EncodeScratch s;
  encode_scratch_carve(static_cast<uint8_t*>(p->dmem) + tbytes, nch, ngc, count, &s);
  e = cudaMemcpy(d_jobs, jobs.data(), sizeof(Job) * (size_t)count, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(p, e);
  e = capture(p, [&](cudaStream_t cs) {
    return launch_encode(d_jobs, nullptr, count, nch, ngc, s, err, cs, max_groups, max_lanes,
                         uniform, false, 0, 0, any_base(d_bases, count));
  });
  if (e != cudaSuccess) return fail(p, e);
  *out = p;
  return ZIPNN_OK;
}

zipnn_status zipnn_plan_load(const zipnn_stream* streams, const void* const* h_containers,
                             const void* const* d_bases, void* const* d_dsts, int count,
                             size_t segment_bytes, const zipnn_tuning* tuning, zipnn_plan** out) {
  if (!out || count <= 0 || !streams || !h_containers || !d_dsts) return ZIPNN_EINVAL;
  *out = nullptr;
  if (segment_bytes == 0) segment_bytes = (size_t)512 << 20;
  // jobs as in zipnn_plan_decompress, grouped into segments of consecutive
  // containers holding about segment_bytes each
  std::vector<Job> jobs((size_t)count);
  std::vector<int> seg_first;
  size_t seg_fill = 0;
  for (int i = 0; i < count; i++) {
    const zipnn_stream* s = &streams[i];
    if (!s->data || !aligned16(s->data) || !h_containers[i]) return ZIPNN_EINVAL;
    const void* base = d_bases ? d_bases[i] : nullptr;
    if (((s->flags & ZIPNN_FLAG_DELTA) != 0) != (base != nullptr)) return ZIPNN_EINVAL;
    if ((s->orig_nbytes && !d_dsts[i]) || !aligned16(d_dsts[i]) || !aligned16(base))
      return ZIPNN_EINVAL;
    if (s->n_groups != (uint32_t)elem_size(s->dtype) || s->dtype < 0 || s->dtype > ZIPNN_U8 ||
        s->lanes < 1 || s->lanes > ZIPNN_MAX_LANES || s->chunk_bytes < ZIPNN_MIN_CHUNK ||
        (uint64_t)s->n_chunks != (s->orig_nbytes + s->chunk_bytes - 1) / s->chunk_bytes)
      return ZIPNN_EINVAL;
    if (i == 0 || seg_fill >= segment_bytes) {
      seg_first.push_back(i);
      seg_fill = 0;
    }
    seg_fill += s->nbytes;
    Job J;
    memset(&J, 0, sizeof(J));
    J.src = static_cast<const uint8_t*>(s->data);
    J.base = static_cast<const uint8_t*>(base);
    J.dst = static_cast<uint8_t*>(d_dsts[i]);
    J.nbytes = s->orig_nbytes;
    J.chunk_bytes = s->chunk_bytes;
    J.lanes = s->lanes;
    J.n_chunks = s->n_chunks;
    J.dtype = s->dtype;
    J.flags = s->flags;
    J.stream_bytes = s->nbytes;
    jobs[i] = J;
  }
  const int nseg = (int)seg_first.size();
  seg_first.push_back(count);
  // chunk numbering restarts in every segment (each has its own table and ticket)
  for (int k = 0; k < nseg; k++) {
    uint64_t ch = 0;
    for (int i = seg_first[k]; i < seg_first[k + 1]; i++) {
      jobs[i].chunk_begin = ch;
      ch += jobs[i].n_chunks;
    }
  }
  uint32_t* err = plan_err_word();
  if (!err) return ZIPNN_ECUDA;
  zipnn_plan* p = new zipnn_plan();
  p->kind = 3;
  p->count = count;
  cudaGetDevice(&p->device);
  const size_t tbytes = align_up(sizeof(Job) * (size_t)count, 256);
  const size_t kbytes = align_up(2 * sizeof(unsigned long long) * (size_t)nseg, 256);
  cudaError_t e = cudaMalloc(&p->dmem, tbytes + kbytes);
  if (e != cudaSuccess) return fail(p, e);
  Job* d_jobs = static_cast<Job*>(p->dmem);
  auto* tickets = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(p->dmem) + tbytes);
  e = cudaMemcpy(d_jobs, jobs.data(), sizeof(Job) * (size_t)count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(tickets, 0, kbytes);
  if (e != cudaSuccess) return fail(p, e);
  zipnn_tuning tu;
  memset(&tu, 0, sizeof(tu));
  if (tuning) tu = *tuning;
  // graph: the copy stream issues the H2D copies segment by segment and marks
  // each segment's end with an event; the capture stream decodes a segment as
  // soon as its copies have landed, while the copies of the next ones proceed
  cudaStream_t sc = nullptr;
  std::vector<cudaEvent_t> evs((size_t)nseg + 1, nullptr);
  e = cudaStreamCreateWithFlags(&sc, cudaStreamNonBlocking);
  for (int k = 0; k <= nseg && e == cudaSuccess; k++)
    e = cudaEventCreateWithFlags(&evs[(size_t)k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = capture(p, [&](cudaStream_t cs) {
    cudaError_t r = cudaEventRecord(evs[(size_t)nseg], cs);  // fork
    if (r == cudaSuccess) r = cudaStreamWaitEvent(sc, evs[(size_t)nseg], 0);
    for (int k = 0; k < nseg && r == cudaSuccess; k++) {
      const int a = seg_first[k], b = seg_first[k + 1];
      uint64_t nch = 0, max_chunk = 0;
      int max_groups = 1, uniform = jobs[a].dtype;
      bool lanes256 = true, has_delta = false;
      int frac64 = 0;
      for (int i = a; i < b; i++) {
        if (stage_frac64(jobs[i].dtype, jobs[i].flags) > frac64)
          frac64 = stage_frac64(jobs[i].dtype, jobs[i].flags);
        if (jobs[i].chunk_bytes > max_chunk) max_chunk = jobs[i].chunk_bytes;
      }
      // stage and kernel variant from the host copies' chunk maps
      MapNeed nd;
      const uint64_t dflt = max_chunk * (uint64_t)frac64 / 64 + 1024;
      for (int i = a; i < b; i++) {
        const zipnn_stream* s = &streams[i];
        const uint64_t mbytes = (uint64_t)s->n_chunks * s->n_groups * kEntryBytes;
        if (s->nbytes < kHdrBytes + mbytes) continue;
        add_map_need(static_cast<const uint8_t*>(h_containers[i]) + kHdrBytes, s->n_chunks,
                     s->n_groups, plan_lut_bits(&tu), dflt, &nd);
      }
      for (int i = a; i < b; i++) {
        if (jobs[i].flags & ZIPNN_FLAG_DELTA) has_delta = true;
        nch += jobs[i].n_chunks;
        if (jobs[i].dtype != uniform) uniform = -1;
        if ((int)streams[i].n_groups > max_groups) max_groups = (int)streams[i].n_groups;
        if (jobs[i].lanes % 256) lanes256 = false;
      }
      // one copy per run of containers that sit back to back in both host and
      // device memory (each copy costs the copy engine a few microseconds of
      // setup); exact adjacency only, so no byte outside a container is written
      for (int i = a; i < b && r == cudaSuccess; i++) {
        const uint8_t* hs = static_cast<const uint8_t*>(h_containers[i]);
        uint8_t* ds = static_cast<uint8_t*>(streams[i].data);
        size_t run = streams[i].nbytes;
        while (i + 1 < b && static_cast<const uint8_t*>(h_containers[i + 1]) == hs + run &&
               static_cast<uint8_t*>(streams[i + 1].data) == ds + run)
          run += streams[++i].nbytes;
        r = cudaMemcpyAsync(ds, hs, run, cudaMemcpyHostToDevice, sc);
      }
      if (r == cudaSuccess) r = cudaEventRecord(evs[(size_t)k], sc);
      if (r == cudaSuccess) r = cudaStreamWaitEvent(cs, evs[(size_t)k], 0);
      uint32_t common_lanes = jobs[a].lanes;
      for (int i = a; i < b; i++)
        if (jobs[i].lanes != common_lanes) common_lanes = 0;
      if (r == cudaSuccess)
        r = launch_decode_ex(d_jobs + a, nullptr, b - a, nch, max_groups, &tu, err,
                             tickets + 2 * k, cs, uniform, max_chunk, lanes256, frac64,
                             has_delta, nd.general, planned_stage(nd), common_lanes);
    }
    // the last wait above joined the copy stream back into the capture stream
    return r;
  });
  for (cudaEvent_t ev : evs)
    if (ev) cudaEventDestroy(ev);
  if (sc) cudaStreamDestroy(sc);
  if (e != cudaSuccess) return fail(p, e);
  *out = p;
  return ZIPNN_OK;
}

zipnn_status zipnn_plan_launch(zipnn_plan* p, void* cuda_stream) {
  if (!p || !p->exec) return ZIPNN_EINVAL;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) return ZIPNN_EINVAL;
  cudaError_t e = cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? ZIPNN_OK : ZIPNN_ECUDA;
}

void zipnn_plan_destroy(zipnn_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->dmem) cudaFree(p->dmem);
  delete p;
}

}  // extern "C"
