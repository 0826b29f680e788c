// Host side of the decoder: shared-memory sizing and the launch entry point,
// which calls the translation unit of the requested table width
// (decode_w10/11/12.cu; the kernels are in decode_kernels.cuh).
#include "decode_kernels.cuh"
#include "host_internal.h"

namespace zipnn {

// Kernels of each (table width, CTA size) pair (decode_w<W>_<threads>.cu):
// the kernel for a launch's dtype (-1: mixed) and delta content.
const void* decode_kernel_w10_128(int dtype, bool gen);
const void* decode_kernel_w11_128(int dtype, bool gen);
const void* decode_kernel_w11_256(int dtype, bool gen);
const void* decode_kernel_w12_128(int dtype, bool gen);
const void* decode_kernel_w12_256(int dtype, bool gen);

namespace {

// Stage size.  Without a measured need (stage_need = 0): room for the payloads
// of the largest chunk (frac64 / 64 of it, see stage_frac64), at most what lets
// two CTAs share an SM.  With one (a plan that read its containers' chunk
// maps): exactly that many bytes, up to the whole SM when only one CTA per SM
// can stage the payloads.  Always room for the tables of every Huffman group
// after the first: in the stage for a 16-bit chunk's second group; in the
// stage and the raw-word rings behind it together for an FP32 chunk's
// groups 1-3 (such a chunk takes no fast loop, which leaves the rings free),
// so that the three spare tables do not cost FP32 launches a CTA per SM.
// Multiples of 128 B, as the decoder's table placement assumes.
uint32_t decode_stage_bytes(uint64_t max_chunk, int frac64, int max_groups, int w, uint32_t ring,
                            uint32_t stage_need) {
  const uint64_t fixed = (4u << w) + kStaticReserve + ring;
  uint64_t cap = (uint64_t)kStageCapPerSm / 2 - fixed;
  uint64_t want;
  if (stage_need) {
    want = ((uint64_t)stage_need + 127) & ~127ull;
    if (want > cap) cap = (uint64_t)kStageCapPerSm - fixed;
  } else {
    want = (max_chunk * (uint64_t)frac64 / 64 + 1024 + 127) & ~127ull;
  }
  uint32_t st = (uint32_t)(want < kStageMin ? kStageMin : (want > cap ? cap : want));
  const uint32_t lut = 4u << w;
  uint32_t tabs = max_groups > 1 ? lut + 256u : 0u;
  const uint32_t all = (uint32_t)(max_groups - 1) * lut + 256u;
  if (max_groups > 2 && all > tabs + ring) tabs = all - ring;
  return st > tabs ? st : tabs;
}

}  // namespace

cudaError_t launch_decode_ex(const Job* d_jobs, const Job* h_one, int njobs,
                             uint64_t nchunks_total, int max_groups, const zipnn_tuning* tuning,
                             uint32_t* d_err, unsigned long long* d_ticket, cudaStream_t st,
                             int uniform_dtype, uint64_t max_chunk, bool lanes256, int frac64,
                             bool has_delta, bool general, uint32_t stage_need,
                             uint32_t common_lanes) {
  if (nchunks_total == 0) return cudaSuccess;
  JobRef r;
  r.table = h_one ? nullptr : d_jobs;
  if (h_one) r.one = *h_one;
  else memset(&r.one, 0, sizeof(Job));
  r.n = njobs;
  if (h_one) {
    uniform_dtype = h_one->dtype;
    max_chunk = h_one->chunk_bytes;
    lanes256 = h_one->lanes % 256 == 0;
    frac64 = stage_frac64(h_one->dtype, h_one->flags);
    has_delta = (h_one->flags & ZIPNN_FLAG_DELTA) != 0;
    common_lanes = h_one->lanes;
  }
  int w = (tuning && tuning->lut_bits) ? tuning->lut_bits : 12;
  if (w < 10) w = 10;
  if (w > 12) w = 12;
  // CTA size: 256 threads (default) for single-dtype launches with W >= 11
  // whose lane counts are multiples of 256 (one or two sub-streams per
  // thread in the fast loop), else 128
  const int want = (tuning && tuning->threads) ? tuning->threads : 256;
  int threads =
      (want == 256 && w >= 11 && uniform_dtype >= 0 && lanes256) ? 256 : kDecThreads;
  // the GEN kernels for launches with deltas or, as a plan's chunk maps show,
  // chunks with two coded groups or a SPARSE first group; W = 10 has no fast
  // loops and no GEN kernels
  const bool gen = has_delta || general;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // Launches with few chunks (no more than half as many as SMs) split every
  // chunk of the model-weight layout over `parts` work items -- disjoint
  // sub-stream ranges, each a whole number of rounds of a 128-thread CTA --
  // so that more SMs work on them: the most parts (8, 4 or 2) that the lanes
  // allow and that keep the work items within two per SM (tuning->parts: 0 =
  // this rule, 1 = never, 2, 4 or 8 = whenever the lanes allow)
  uint32_t parts = 1;
  const int want_parts = tuning ? tuning->parts : 0;
  if (!gen && w >= 11 && uniform_dtype >= 0 && common_lanes && want_parts != 1) {
    for (uint32_t p = 8; p >= 2; p /= 2) {
      if (common_lanes % (p * (uint32_t)kDecThreads) != 0) continue;
      if (want_parts == 0 && nchunks_total * 2 > (uint64_t)sms) break;
      if (want_parts == 0 && nchunks_total * p > 2ull * (uint64_t)sms) continue;
      if (want_parts != 0 && (uint32_t)want_parts != p) continue;
      parts = p;
      threads = kDecThreads;
      break;
    }
  }
  const void* kern =
      w == 10   ? decode_kernel_w10_128(uniform_dtype, false)
      : w == 11 ? (threads == 256 ? decode_kernel_w11_256(uniform_dtype, gen)
                                  : decode_kernel_w11_128(uniform_dtype, gen))
                : (threads == 256 ? decode_kernel_w12_256(uniform_dtype, gen)
                                  : decode_kernel_w12_128(uniform_dtype, gen));
  int per_sm = 0;
  if (tuning && tuning->ctas_per_sm > 0) per_sm = tuning->ctas_per_sm;
  if (max_groups < 1 || max_groups > 4) max_groups = 4;
  // per-thread rings: launches that can hold FP32 chunks (raw words) or
  // deltas (base)
  const uint32_t ring =
      (uniform_dtype == ZIPNN_FP32 || uniform_dtype < 0 || has_delta)
          ? kRingBytes * (uint32_t)threads
          : 0u;
  uint32_t stage = decode_stage_bytes(max_chunk, frac64, max_groups, w, ring, stage_need);
  const int smem = (int)((4u << w) + stage + ring);  // one table slot | stage | rings
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  // all of the unified L1 / shared array as shared memory, so the CTAs per
  // SM that the occupancy query reports are the ones that become resident
  e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
  if (occ < 1) occ = 1;
  if (per_sm == 0 || per_sm > occ) per_sm = occ;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > nchunks_total * parts) grid = nchunks_total * parts;
  // a split launch runs as clusters of `parts` CTAs, one chunk per cluster
  // (its CTAs build the chunk's table together), items by stride: the grid
  // is a whole number of clusters
  bool clustered = false;
  if (parts > 1) {
    grid -= grid % parts;
    cudaLaunchConfig_t probe = {};
    probe.gridDim = dim3((unsigned)grid);
    probe.blockDim = dim3((unsigned)threads);
    probe.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute ca;
    ca.id = cudaLaunchAttributeClusterDimension;
    ca.val.clusterDim.x = parts;
    ca.val.clusterDim.y = 1;
    ca.val.clusterDim.z = 1;
    probe.attrs = &ca;
    probe.numAttrs = 1;
    int nclusters = 0;
    clustered = grid >= parts &&
                cudaOccupancyMaxActiveClusters(&nclusters, kern, &probe) == cudaSuccess &&
                nclusters > 0;
    if (!clustered) cudaGetLastError();  // clear a refused query; split without clusters
  }
  uint32_t dbg = tuning ? (uint32_t)tuning->debug_flags : 0u;
  // the fast loops' L2 prefetch budget, shared by the CTAs that run at once
  uint64_t pf64 = kPfBudget / grid;
  uint32_t pf = (uint32_t)(pf64 > (64u << 20) ? (64u << 20) : pf64);
  // the kernel's parameters, in the order of k_decode's signature
  unsigned long long* tk = clustered ? nullptr : d_ticket;  // clusters: items by stride
  void* args[] = {&r, &nchunks_total, &d_err, &tk, &dbg, &stage, &pf, &parts};
  if (!clustered)
    return cudaLaunchKernel(kern, dim3((unsigned)grid), dim3((unsigned)threads), args,
                            (size_t)smem, st);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute ca;
  ca.id = cudaLaunchAttributeClusterDimension;
  ca.val.clusterDim.x = parts;
  ca.val.clusterDim.y = 1;
  ca.val.clusterDim.z = 1;
  cfg.attrs = &ca;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, kern, args);
}

}  // namespace zipnn
