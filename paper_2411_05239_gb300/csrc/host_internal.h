// Host-side interfaces between the library's translation units: the launchers
// of the encoder and decoder kernels, the encoder's scratch layout, and the
// small helpers several entry points share.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "zipnn.h"
#include "zipnn_internal.cuh"

namespace zipnn {

struct EncodeScratch {
  uint32_t* hist;      // [ngc][256]
  uint32_t* codes;     // [ngc][256] (len << 16 | code)
  uint8_t* tabs;       // [ngc][kTabBytes]
  GcMeta* meta;        // [ngc]
  uint64_t* offs;      // [ngc] payload offsets
  uint64_t* totals;    // [njobs]
  uint32_t* zsyms;     // [ngc] symbols inside all-zero vectors (SPARSE candidate)
};
size_t encode_scratch_bytes(uint64_t nchunks_total, uint64_t ngc_total, int njobs);
void encode_scratch_carve(void* base, uint64_t nchunks_total, uint64_t ngc_total, int njobs,
                          EncodeScratch* s);

// Encoder (encode.cu): histogram + code build + offsets, then packing.  d_jobs
// is a device table of njobs jobs, unless njobs == 1 and h_one is given (the
// job is then passed by value); uniform_dtype is the dtype of every job or -1.
cudaError_t launch_encode_analyse_ex(const Job* d_jobs, const Job* h_one, int njobs,
                                     uint64_t nchunks_total, uint64_t ngc_total,
                                     const EncodeScratch& s, uint32_t* d_err, cudaStream_t st,
                                     int max_groups, int uniform_dtype);
// True when some of the count bases is given (a batch that holds deltas).
inline bool any_base(const void* const* d_bases, int count) {
  if (!d_bases) return false;
  for (int i = 0; i < count; i++)
    if (d_bases[i]) return true;
  return false;
}
// any_delta: some job has a base (its packer stages two coded groups per
// chunk in pass A); taken from the job itself when h_one is given.
cudaError_t launch_encode_pack_ex(const Job* d_jobs, const Job* h_one, int njobs,
                                  uint64_t nchunks_total, int max_lanes, const EncodeScratch& s,
                                  cudaStream_t st, int uniform_dtype, bool any_delta = false);
// The whole encoder: the four kernels above (encoder == 0), or the
// single-pass kernel (histogram, code build, offsets by look-back, packing:
// one launch after a memset of its look-back words) when encoder == 1 and
// every job is BF16, FP16 or U8 and none uses the skip-ahead probe.  Both
// write the same bytes.
cudaError_t launch_encode(const Job* d_jobs, const Job* h_one, int njobs, uint64_t nchunks_total,
                          uint64_t ngc_total, const EncodeScratch& s, uint32_t* d_err,
                          cudaStream_t st, int max_groups, int max_lanes, int uniform_dtype,
                          bool any_skip, int encoder, uint32_t debug_flags = 0,
                          bool any_delta = false);
bool fused_encoder_applies(int dtype, bool any_skip);

// Decoder (decode.cu): one persistent launch over all chunks of the jobs.
// d_ticket: the device work queue, two 64-bit counters that must be zero
// before the first launch on them (the kernel's last CTA zeroes them again),
// or nullptr for a static assignment of chunks to CTAs.  frac64: stage size as a fraction of
// the largest chunk (stage_frac64); has_delta: some job has a base; general:
// use the general fast loops (two coded groups, SPARSE first groups) even
// without a delta; stage_need: a stage size measured from the chunk maps (0 =
// use frac64); common_lanes: the lanes of every job, or 0 if they differ (a
// launch with few chunks may then split each chunk over several work items).
cudaError_t launch_decode_ex(const Job* d_jobs, const Job* h_one, int njobs,
                             uint64_t nchunks_total, int max_groups, const zipnn_tuning* tuning,
                             uint32_t* d_err, unsigned long long* d_ticket, cudaStream_t st,
                             int uniform_dtype, uint64_t max_chunk, bool lanes256, int frac64,
                             bool has_delta, bool general, uint32_t stage_need,
                             uint32_t common_lanes);

// Sub-streams per group-chunk when a call gives none: chunk_bytes / 512 for
// plain 16-bit containers (two sub-streams per thread of a 256-thread decoder
// CTA at 256 KiB), chunk_bytes / 1024 for FP32, U8 and deltas (whose payloads
// are small enough for the start-bit tables to show); clamped to [1, 1024].
uint32_t default_lanes_for(int dtype, size_t chunk_bytes, bool delta);
// The device error word of this host thread's launches (api.cu).
uint32_t* plan_err_word();
// Route the device error word of this host thread's launches to d_err (a
// 4-byte device word), or back to the device's own word (nullptr).
void set_thread_err_word(uint32_t* d_err);

}  // namespace zipnn
