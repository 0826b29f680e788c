// Request server: continuous batching of compress / decompress requests with
// admission against a device-memory budget (the serving form of the codec).
//
// Requests arrive on any host thread (zipnn_server_submit).  A scheduler thread
// admits them in arrival order while (a) the budget covers the request's input
// (caller-owned, charged but not allocated), its output and its scratch
// (allocated from a device arena of exactly `budget` bytes), and (b) a slot --
// a CUDA stream -- is free.  Everything admitted in one scheduling pass forms a
// batch: its compress requests run as one batched compression (4 kernels for
// all of them) and its decompress requests as one persistent batched decode,
// on the slot's stream.  New requests keep being admitted into other slots
// while earlier batches run, so their work overlaps on the device.  A waiter
// thread per slot blocks on an event recorded after the batch and stamps the
// completion time; outputs stay resident (and charged) until the caller
// releases them.
#include <chrono>
#include <condition_variable>
#include <memory>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "zipnn.h"
#include "host_internal.h"

using namespace zipnn;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with 256-byte granularity.
class Arena {
 public:
  void reset(uint64_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = 0;
  }
  bool alloc(uint64_t n, uint64_t* off) {
    n = align_up(n ? n : 1, 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const uint64_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += n;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t n) {
    n = align_up(n ? n : 1, 256);
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  uint64_t used() const { return used_; }

 private:
  std::map<uint64_t, uint64_t> free_;
  uint64_t used_ = 0;
};

struct Req {
  uint64_t id = 0;
  zipnn_request r;
  uint64_t in_charge = 0;     // caller input bytes charged while in flight
  uint64_t out_off = 0, out_size = 0;
  uint64_t out_bytes = 0;     // result size
  int32_t status = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Batch;
constexpr int kMaxBatch = 4096;

struct Slot {
  cudaStream_t st = nullptr;
  Batch* batch = nullptr;
  uint64_t* h_sizes = nullptr;  // pinned, mapped: container sizes of the slot's batch
  uint32_t* d_err = nullptr;    // the device error word of the slot's batches
  uint32_t* h_err = nullptr;    // pinned: its value after each batch
  // completion: the scheduler records `ev` after the batch and hands the batch
  // to this slot's waiter thread, which blocks on the event (lower latency than
  // a stream host callback) and then queues the batch as finished
  cudaEvent_t ev = nullptr;
  Batch* launched = nullptr;
  bool quit = false;
  std::unique_ptr<std::condition_variable> wcv;
  std::thread waiter;
};

struct Batch {
  zipnn_server* srv = nullptr;
  int slot = -1;
  std::vector<Req*> reqs;
  uint64_t ws_off = 0, ws_size = 0;
  uint64_t* h_sizes = nullptr;  // the slot's pinned size array
  double t_done = 0;
  int32_t launch_status = 0;
  uint32_t dev_err = 0;  // the batch's device error word (decoder / encoder flags)
};

}  // namespace

struct zipnn_server {
  int device = 0;
  uint64_t budget = 0;
  uint8_t* arena_base = nullptr;
  Arena arena;
  uint64_t charged = 0;         // inputs in flight (outputs/scratch live in the arena)
  std::vector<Slot> slots;
  std::deque<Req*> pending;
  std::map<uint64_t, Req*> live;
  std::deque<Batch*> finished;  // pushed by the slot waiters
  std::deque<zipnn_completion> done;
  std::mutex mu;
  std::condition_variable cv;
  std::thread sched;
  bool stop = false;
  uint64_t next_id = 1;
  uint64_t inflight = 0;        // admitted, not finished
  zipnn_server_stats stats;
};

namespace {

uint64_t out_bytes_needed(const zipnn_request& r) {
  if (r.op == ZIPNN_OP_COMPRESS) {
    const uint64_t cb = r.chunk_bytes ? r.chunk_bytes : ZIPNN_DEFAULT_CHUNK;
    return zipnn_compress_bound(r.input_bytes, r.dtype, cb);
  }
  return r.container.orig_nbytes;
}

uint64_t ws_needed(const zipnn_request& r) {
  if (r.op != ZIPNN_OP_COMPRESS) return 0;
  const uint64_t cb = r.chunk_bytes ? r.chunk_bytes : ZIPNN_DEFAULT_CHUNK;
  return zipnn_compress_workspace_size(r.input_bytes, r.dtype, cb);
}

uint64_t in_bytes(const zipnn_request& r) {
  return r.op == ZIPNN_OP_COMPRESS ? r.input_bytes : r.container.nbytes;
}

// Waiter of slot si: waits for each batch launched on the slot to complete.
void slot_waiter(zipnn_server* s, int si) {
  cudaSetDevice(s->device);
  Slot& sl = s->slots[(size_t)si];
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    sl.wcv->wait(lk, [&] { return sl.launched != nullptr || sl.quit; });
    if (!sl.launched) break;  // quit with nothing in flight
    Batch* b = sl.launched;
    sl.launched = nullptr;
    lk.unlock();
    cudaEventSynchronize(sl.ev);
    b->t_done = now_s();
    b->dev_err = *sl.h_err;
    lk.lock();
    s->finished.push_back(b);
    s->cv.notify_all();
  }
}

// Launch one batch on slot `si` (called without the lock; the batch belongs to
// the scheduler until the slot's waiter has seen it complete).
void launch_batch(zipnn_server* s, int si, Batch* b) {
  Slot& slot = s->slots[(size_t)si];
  cudaStream_t st = slot.st;
  std::vector<const void*> csrc, cbase;
  std::vector<size_t> cnb, ccap;
  std::vector<int> cdt;
  std::vector<void*> cout;
  std::vector<zipnn_stream> dstr;
  std::vector<const void*> dbase;
  std::vector<void*> ddst;
  uint64_t chunk = ZIPNN_DEFAULT_CHUNK;  // all compress requests of a batch share it
  size_t ncomp = 0;
  for (Req* q : b->reqs) {
    if (q->r.op == ZIPNN_OP_COMPRESS) {
      chunk = q->r.chunk_bytes ? q->r.chunk_bytes : ZIPNN_DEFAULT_CHUNK;
      ncomp++;
      csrc.push_back(q->r.d_input);
      cbase.push_back(q->r.d_base);
      cnb.push_back(q->r.input_bytes);
      cdt.push_back(q->r.dtype);
      cout.push_back(s->arena_base + q->out_off);
      ccap.push_back(q->out_size);
    } else {
      dstr.push_back(q->r.container);
      dbase.push_back(q->r.d_base);
      ddst.push_back(s->arena_base + q->out_off);
    }
  }
  int32_t rc = ZIPNN_OK;
  // the batch's kernels report into the slot's own error word
  set_thread_err_word(slot.d_err);
  if (ncomp == 1 && dstr.empty()) {
    // a batch of one request (the idle server's common case) takes the direct
    // entry point: the job goes by value, no job table is uploaded
    rc = zipnn_compress_into(csrc[0], cbase[0], cnb[0], cdt[0], chunk, 0, cout[0], ccap[0],
                             s->arena_base + b->ws_off, b->ws_size, b->h_sizes, st);
  } else if (ncomp) {
    rc = zipnn_batch_compress_into(csrc.data(), cbase.data(), cnb.data(), cdt.data(), (int)ncomp,
                                   chunk, 0, cout.data(), ccap.data(), s->arena_base + b->ws_off,
                                   b->ws_size, b->h_sizes, st);
  }
  if (rc == ZIPNN_OK && dstr.size() == 1 && ncomp == 0)
    rc = zipnn_decompress(&dstr[0], dbase[0], ddst[0], dstr[0].orig_nbytes, st);
  else if (rc == ZIPNN_OK && !dstr.empty())
    rc = zipnn_batch_decompress(dstr.data(), dbase.data(), ddst.data(), (int)dstr.size(), nullptr,
                                st);
  set_thread_err_word(nullptr);
  b->launch_status = rc;
  // the word is read back after the batch; it is cleared (on the slot's
  // stream, before its next batch) only when it was set
  cudaMemcpyAsync(slot.h_err, slot.d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  cudaEventRecord(slot.ev, st);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    slot.launched = b;
  }
  slot.wcv->notify_one();
}

void finish_batch(zipnn_server* s, Batch* b) {
  size_t ci = 0;
  // a device-side error fails every request of its batch (the kernels share
  // one error word per batch)
  int32_t st = b->launch_status;
  if (b->dev_err) {
    if (st == ZIPNN_OK)
      st = (b->dev_err & 1u) ? ZIPNN_ECORRUPT : ((b->dev_err & 2u) ? ZIPNN_ENOMEM : ZIPNN_ETIMEOUT);
    Slot& sl = s->slots[(size_t)b->slot];
    cudaMemsetAsync(sl.d_err, 0, sizeof(uint32_t), sl.st);
  }
  for (Req* q : b->reqs) {
    q->t_done = b->t_done;
    q->status = st;
    if (q->r.op == ZIPNN_OP_COMPRESS) {
      q->out_bytes = b->h_sizes[ci++];
    } else {
      q->out_bytes = q->r.container.orig_nbytes;
    }
    s->charged -= q->in_charge;
    q->in_charge = 0;
    zipnn_completion c;
    memset(&c, 0, sizeof(c));
    c.id = q->id;
    c.tag = q->r.tag;
    c.status = q->status;
    c.op = q->r.op;
    c.d_output = s->arena_base + q->out_off;
    c.output_bytes = q->out_bytes;
    c.t_submit = q->t_submit;
    c.t_admit = q->t_admit;
    c.t_done = q->t_done;
    s->done.push_back(c);
    s->stats.completed++;
    s->stats.bytes_processed += q->r.op == ZIPNN_OP_COMPRESS ? q->r.input_bytes : q->out_bytes;
  }
  if (b->ws_size) s->arena.release(b->ws_off, b->ws_size);
  s->inflight -= b->reqs.size();
  s->slots[b->slot].batch = nullptr;
  delete b;
}

// Admission (the caller holds the lock): pending requests, in arrival order,
// into a batch on a free slot while the budget allows.  Returns the batch, its
// slot claimed and its requests counted in flight, ready for launch_batch
// without the lock; nullptr when no slot is free, nothing is pending or the
// head request does not fit now.  *never_fits: nothing is running or held and
// the head request still does not fit (it never will).
Batch* admit(zipnn_server* s, bool* never_fits) {
  *never_fits = false;
  int free_slot = -1;
  for (int i = 0; i < (int)s->slots.size(); i++)
    if (!s->slots[i].batch) { free_slot = i; break; }
  if (free_slot < 0 || s->pending.empty()) return nullptr;
  Batch* b = new Batch();
  b->srv = s;
  b->slot = free_slot;
  std::vector<size_t> nbs;
  std::vector<int> dts;
  uint64_t chunk = 0;
  while (!s->pending.empty() && b->reqs.size() < (size_t)kMaxBatch) {
    Req* q = s->pending.front();
    if (q->r.op == ZIPNN_OP_COMPRESS && chunk &&
        (q->r.chunk_bytes ? q->r.chunk_bytes : ZIPNN_DEFAULT_CHUNK) != chunk)
      break;  // a batch's compress requests share one chunk size
    const uint64_t in = in_bytes(q->r), outn = out_bytes_needed(q->r);
    if (s->charged + in + s->arena.used() + outn > s->budget) break;
    uint64_t oo;
    if (!s->arena.alloc(outn, &oo)) break;
    q->out_off = oo;
    q->out_size = outn;
    s->charged += in;
    q->in_charge = in;
    q->t_admit = now_s();
    s->pending.pop_front();
    b->reqs.push_back(q);
    if (q->r.op == ZIPNN_OP_COMPRESS) {
      nbs.push_back(q->r.input_bytes);
      dts.push_back(q->r.dtype);
      chunk = q->r.chunk_bytes ? q->r.chunk_bytes : ZIPNN_DEFAULT_CHUNK;
    }
  }
  // batch workspace for the compress requests.  Requests were admitted for
  // their input and output bytes alone; when the workspace of all the batch's
  // compress requests does not fit as well, requests go back to the front of
  // the queue from the tail of the batch (arrival order kept) until it fits
  // or a single compress request is left.  Only that one's own workspace can
  // then fail to fit, and only while other requests hold memory (the submit
  // check counts a request's workspace).
  auto hand_back = [&](Req* q) {
    s->arena.release(q->out_off, q->out_size);
    s->charged -= q->in_charge;
    q->in_charge = 0;
    s->pending.push_front(q);
  };
  bool ok = true;
  while (!nbs.empty()) {
    const uint64_t ws =
        zipnn_batch_compress_workspace_size(nbs.data(), dts.data(), (int)nbs.size(), chunk);
    uint64_t wo = 0;
    if (ws && s->charged + s->arena.used() + ws <= s->budget && s->arena.alloc(ws, &wo)) {
      b->ws_off = wo;
      b->ws_size = ws;
      break;
    }
    if (nbs.size() == 1) {
      ok = false;
      break;
    }
    Req* q = b->reqs.back();
    b->reqs.pop_back();
    if (q->r.op == ZIPNN_OP_COMPRESS) {
      nbs.pop_back();
      dts.pop_back();
    }
    hand_back(q);
  }
  if (!ok) {
    // not even one compress request's workspace fits now: hand the compress
    // requests back (the decompress requests of the batch still run)
    std::vector<Req*> keep;
    for (auto it = b->reqs.rbegin(); it != b->reqs.rend(); ++it) {
      Req* q = *it;
      if (q->r.op == ZIPNN_OP_COMPRESS) hand_back(q);
      else keep.push_back(q);
    }
    b->reqs.assign(keep.rbegin(), keep.rend());
  }
  if (b->reqs.empty()) {
    delete b;
    *never_fits = s->inflight == 0 && s->arena.used() == 0 && s->charged == 0;
    return nullptr;
  }
  b->h_sizes = s->slots[free_slot].h_sizes;
  s->slots[free_slot].batch = b;
  s->inflight += b->reqs.size();
  s->stats.batches++;
  if (b->reqs.size() > s->stats.max_batch) s->stats.max_batch = b->reqs.size();
  return b;
}

void scheduler(zipnn_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    while (!s->finished.empty()) {
      Batch* b = s->finished.front();
      s->finished.pop_front();
      finish_batch(s, b);
    }
    if (s->stop) {
      // shutting down: queued requests are cancelled, running batches finish
      while (!s->pending.empty()) {
        Req* q = s->pending.front();
        s->pending.pop_front();
        s->live.erase(q->id);
        delete q;
      }
      if (s->inflight == 0) break;
      s->cv.wait(lk);
      continue;
    }
    bool never_fits = false;
    Batch* b = admit(s, &never_fits);
    if (b) {
      // launch without the lock: submitters and the slot waiters stay free
      lk.unlock();
      launch_batch(s, b->slot, b);
      lk.lock();
      continue;
    }
    if (never_fits) {
      // nothing runs or holds memory and the head request still does not
      // fit: it never will (the submit check makes this unreachable for a
      // request whose input, output and workspace fit the budget); fail it
      Req* q = s->pending.front();
      s->pending.pop_front();
      zipnn_completion c;
      memset(&c, 0, sizeof(c));
      c.id = q->id;
      c.tag = q->r.tag;
      c.status = ZIPNN_EBUSY;
      c.op = q->r.op;
      c.t_submit = q->t_submit;
      c.t_done = now_s();
      s->done.push_back(c);
      s->live.erase(q->id);
      delete q;
      continue;
    }
    s->cv.wait(lk);
  }
}

}  // namespace

extern "C" {

zipnn_status zipnn_server_create(uint64_t budget_bytes, int slots, zipnn_server** out) {
  if (!out || slots < 1 || slots > 64 || budget_bytes < (1u << 20)) return ZIPNN_EINVAL;
  *out = nullptr;
  zipnn_server* s = new zipnn_server();
  memset(&s->stats, 0, sizeof(s->stats));
  cudaGetDevice(&s->device);
  s->budget = budget_bytes;
  void* base = nullptr;
  if (cudaMalloc(&base, budget_bytes) != cudaSuccess) {
    delete s;
    return ZIPNN_ENOMEM;
  }
  s->arena_base = static_cast<uint8_t*>(base);
  s->arena.reset(budget_bytes);
  s->slots.resize((size_t)slots);
  for (auto& sl : s->slots) {
    cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
    sl.wcv.reset(new std::condition_variable());
    if (!sl.ev ||
        cudaHostAlloc(reinterpret_cast<void**>(&sl.h_sizes), sizeof(uint64_t) * kMaxBatch,
                      cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&sl.h_err), sizeof(uint32_t),
                      cudaHostAllocPortable) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&sl.d_err), sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(sl.d_err, 0, sizeof(uint32_t)) != cudaSuccess) {
      for (auto& s2 : s->slots) {
        if (s2.h_sizes) cudaFreeHost(s2.h_sizes);
        if (s2.h_err) cudaFreeHost(s2.h_err);
        if (s2.d_err) cudaFree(s2.d_err);
        if (s2.ev) cudaEventDestroy(s2.ev);
        if (s2.st) cudaStreamDestroy(s2.st);
      }
      cudaFree(s->arena_base);
      delete s;
      return ZIPNN_ENOMEM;
    }
  }
  for (size_t i = 0; i < s->slots.size(); i++)
    s->slots[i].waiter = std::thread(slot_waiter, s, (int)i);
  s->sched = std::thread(scheduler, s);
  *out = s;
  return ZIPNN_OK;
}

zipnn_status zipnn_server_submit(zipnn_server* s, const zipnn_request* r, uint64_t* id) {
  if (!s || !r) return ZIPNN_EINVAL;
  if (r->op != ZIPNN_OP_COMPRESS && r->op != ZIPNN_OP_DECOMPRESS) return ZIPNN_EINVAL;
  if (r->op == ZIPNN_OP_COMPRESS) {
    if (r->dtype < ZIPNN_BF16 || r->dtype > ZIPNN_U8) return ZIPNN_EINVAL;
    if (r->input_bytes % (uint64_t)elem_size(r->dtype)) return ZIPNN_EINVAL;
    if ((r->input_bytes && !r->d_input) || (reinterpret_cast<uintptr_t>(r->d_input) & 15))
      return ZIPNN_EINVAL;
    const uint64_t cb = r->chunk_bytes ? r->chunk_bytes : ZIPNN_DEFAULT_CHUNK;
    if (cb < ZIPNN_MIN_CHUNK || cb > ZIPNN_MAX_CHUNK || cb % 16) return ZIPNN_EINVAL;
  } else {
    if (!r->container.data) return ZIPNN_EINVAL;
    if (((r->container.flags & ZIPNN_FLAG_DELTA) != 0) != (r->d_base != nullptr))
      return ZIPNN_EINVAL;
  }
  const uint64_t need = in_bytes(*r) + align_up(out_bytes_needed(*r), 256) + align_up(ws_needed(*r), 256);
  if (need > s->budget) return ZIPNN_EBUSY;  // could never be admitted
  Req* q = new Req();
  q->r = *r;
  q->t_submit = now_s();
  Batch* b = nullptr;
  uint64_t qid = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q->id = qid = s->next_id++;
    s->pending.push_back(q);
    s->live[q->id] = q;
    s->stats.submitted++;
    // nothing queued ahead and a slot free: admit and launch on this thread,
    // without waking the scheduler (its hand-off costs tens of microseconds)
    bool never_fits = false;
    if (!s->stop && s->pending.size() == 1) b = admit(s, &never_fits);
  }
  if (id) *id = qid;
  if (b) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    launch_batch(s, b->slot, b);
    if (prev != s->device && prev >= 0) cudaSetDevice(prev);
  } else {
    s->cv.notify_all();
  }
  return ZIPNN_OK;
}

int zipnn_server_poll(zipnn_server* s, zipnn_completion* out, int max) {
  if (!s || !out || max <= 0) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  int n = 0;
  while (n < max && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  return n;
}

zipnn_status zipnn_server_release(zipnn_server* s, uint64_t id) {
  if (!s) return ZIPNN_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->live.find(id);
    if (it == s->live.end()) return ZIPNN_EINVAL;
    Req* q = it->second;
    if (q->t_done == 0) return ZIPNN_EBUSY;  // still running
    s->arena.release(q->out_off, q->out_size);
    s->live.erase(it);
    delete q;
  }
  s->cv.notify_all();
  return ZIPNN_OK;
}

zipnn_status zipnn_server_drain(zipnn_server* s, double timeout_s) {
  if (!s) return ZIPNN_EINVAL;
  const double t_end = now_s() + timeout_s;
  std::unique_lock<std::mutex> lk(s->mu);
  while (!(s->pending.empty() && s->inflight == 0)) {
    if (now_s() > t_end) return ZIPNN_ETIMEOUT;
    s->cv.wait_for(lk, std::chrono::milliseconds(1));
  }
  return ZIPNN_OK;
}

zipnn_status zipnn_server_get_stats(zipnn_server* s, zipnn_server_stats* st) {
  if (!s || !st) return ZIPNN_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->stats;
  st->arena_used = s->arena.used();
  st->inputs_charged = s->charged;
  return ZIPNN_OK;
}

void zipnn_server_destroy(zipnn_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->sched.joinable()) s->sched.join();  // returns once no batch is in flight
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& sl : s->slots) sl.quit = true;
  }
  for (auto& sl : s->slots) {
    sl.wcv->notify_all();
    if (sl.waiter.joinable()) sl.waiter.join();
  }
  for (auto& sl : s->slots) {
    cudaStreamSynchronize(sl.st);
    cudaEventDestroy(sl.ev);
    cudaStreamDestroy(sl.st);
    cudaFreeHost(sl.h_sizes);
    cudaFreeHost(sl.h_err);
    cudaFree(sl.d_err);
  }
  for (auto& kv : s->live) delete kv.second;
  cudaFree(s->arena_base);
  delete s;
}

}  // extern "C"
