// Encoder kernels of the GB300 ZipNN codec (ZipNN Sec. 3.1, 3.2, 4.2, 5.1).
//
//   k_hist      one CTA per chunk: reads the chunk once with 16-B loads (XOR
//               with the delta base fused in), applies the exponent-extraction /
//               byte-grouping permutation in registers and builds one 256-bin
//               histogram per byte group (per-warp shared-memory copies).
//   k_build     one warp per group-chunk: mode decision (ZERO / CONST / RAW /
//               HUFF), length-limited code lengths by package-merge (limit 12),
//               canonical codes and the table bytes.  A Shannon lower bound
//               proves RAW without building a code for incompressible groups.
//   k_scan      one CTA per tensor: exclusive scan of the padded payload sizes
//               (the chunk map of Sec. 5.1) and the container size.
//   k_pack      one CTA per chunk: per-sub-stream bit counts, a CTA scan for
//               the sub-stream start bits, MSB-first bit packing, raw copies;
//               writes the map entries (and, in extra CTAs, the headers).
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "host_internal.h"

namespace zipnn {

namespace {

constexpr int kHistThreads = 256;
constexpr int kBuildWarps = 4;

struct JobRef {
  const Job* table;  // device table, or nullptr to use `one`
  Job one;
  int n;
};

__device__ __forceinline__ const Job& job_at(const JobRef& r, int j) {
  return r.table ? r.table[j] : r.one;
}

__device__ __forceinline__ int find_job_chunk(const JobRef& r, uint64_t chunk) {
  if (!r.table) return 0;
  return find_job(r.table, r.n, chunk);
}

__device__ __forceinline__ int find_job_gc(const JobRef& r, uint64_t gc) {
  if (!r.table) return 0;
  int lo = 0, hi = r.n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (r.table[mid].gc_begin <= gc) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Load original vector v (16 bytes) of a chunk, XOR-ed with the base when
// given; bytes past nb (a partial last vector) read as zero.
// Ask L2 for the 128-B line holding p, without a register or a wait: loads
// issued later find it in L2 instead of waiting for DRAM.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Shared-memory accesses through 32-bit shared-window addresses: the tables
// and slots below are reached through pointers the compiler cannot always
// place in shared memory, and would otherwise use generic loads and stores.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t lds32(uint32_t saddr) {  // read-only data (code tables)
  uint32_t v;
  asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(saddr));
  return v;
}
__device__ __forceinline__ uint32_t lds32v(uint32_t saddr) {  // data written in this kernel
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(saddr) : "memory");
  return v;
}
__device__ __forceinline__ void sts32(uint32_t saddr, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(saddr), "r"(v) : "memory");
}
// Code table entry (len << 16 | code) of byte k of w, table at shared address cb.
__device__ __forceinline__ uint32_t code_of(uint32_t cb, uint32_t w, int k) {
  return lds32(cb + 4u * __byte_perm(w, 0, 0x4440 + k));
}


__device__ __forceinline__ uint4 load_vec(const uint8_t* src, const uint8_t* base, uint64_t v,
                                          uint64_t nb) {
  uint4 a;
  if ((v + 1) * 16 <= nb) {
    a = __ldg(reinterpret_cast<const uint4*>(src) + v);
    if (base) {
      uint4 b = __ldg(reinterpret_cast<const uint4*>(base) + v);
      a.x ^= b.x; a.y ^= b.y; a.z ^= b.z; a.w ^= b.w;
    }
  } else {  // ragged last vector (static indices: the words stay in registers)
    uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 16; i++) {
      const uint64_t k = v * 16 + i;
      if (k < nb) w[i >> 2] |= (uint32_t)(src[k] ^ (base ? base[k] : 0u)) << (8 * (i & 3));
    }
    a = make_uint4(w[0], w[1], w[2], w[3]);
  }
  return a;
}

// Group bytes of one vector: out[g][q] holds 4 symbols each (q < V/4).
__device__ __forceinline__ void split_vec(int dtype, uint4 a, uint32_t out[4][4]) {
  if (dtype == ZIPNN_FP32) {
    uint32_t x[4] = {a.x, a.y, a.z, a.w}, g[4];
    split32(x, g);
    out[0][0] = g[0]; out[1][0] = g[1]; out[2][0] = g[2]; out[3][0] = g[3];
  } else if (dtype == ZIPNN_U8) {
    out[0][0] = a.x; out[0][1] = a.y; out[0][2] = a.z; out[0][3] = a.w;
  } else {
    split16(a.x, a.y, out[0][0], out[1][0]);
    split16(a.z, a.w, out[0][1], out[1][1]);
  }
}

// ---------------------------------------------------------------------------
// k_hist: shared-memory atomics into lane-indexed histograms.  Group g's
// counter for bin b and lane l sits at word (g * 256 + b) * 32 + l, shared by
// all warps of the CTA: the 32 lanes of one atomic instruction always address
// 32 different banks (one wavefront, whatever the symbols), which removes the
// bank conflicts that bound a plain per-warp histogram.

// Shared-memory add without a result, on a 32-bit shared-window address.
__device__ __forceinline__ void red_shared_inc(uint32_t saddr) {
  asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(saddr) : "memory");
}

// Histogram of a whole chunk of 16-bit elements (no ragged vector): the byte
// offsets of an element h's counters follow from its bits.  Exponent bin e =
// (h >> 7) & 0xFF sits at e * 128 = h & 0x7F80 (one mask per element).  The
// sign + low-fraction bins r = (h >> 8 & 0x80) | (h & 0x7F) of four elements
// (two words) are gathered into one word with two byte permutes and a bit
// select, as split16 does; bin r sits at 0x8000 + r * 128 (a byte permute
// and a shift-add per element).  hl is the shared-window address of lane 0's
// counter of exponent bin 0 plus 4 * lane.
__device__ __forceinline__ void hist16_words(uint32_t hl, uint32_t w0, uint32_t w1) {
  red_shared_inc(hl + (w0 & 0x7F80u));
  red_shared_inc(hl + ((w0 >> 16) & 0x7F80u));
  red_shared_inc(hl + (w1 & 0x7F80u));
  red_shared_inc(hl + ((w1 >> 16) & 0x7F80u));
  const uint32_t lo = __byte_perm(w0, w1, 0x6420), hi = __byte_perm(w0, w1, 0x7531);
  const uint32_t r = (hi & 0x80808080u) | (lo & 0x7F7F7F7Fu);
  const uint32_t hl8 = hl + 0x8000u;
#pragma unroll
  for (int k = 0; k < 4; k++) red_shared_inc(hl8 + (__byte_perm(r, 0, 0x4440 + k) << 7));
}

// Shared-memory add of v without a result, on a 32-bit shared-window address.
__device__ __forceinline__ void red_shared_add(uint32_t saddr, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(saddr), "r"(v) : "memory");
}

// Histogram of one FP32 element x with packed counters: group g's counter of
// bin b for this lane is the half b / 128 of the word at byte g * 16384 +
// (b % 128) * 128 from hl (the shared-window address of lane 0's word of
// group 0, bin 0, plus 4 * lane).  With g0 = x >> 23 & 0xFF, g1 = (x >> 24 &
// 0x80) | (x >> 16 & 0x7F), g2 = x >> 8 & 0xFF and g3 = x & 0xFF, each word
// offset is a shift and a mask of x and each half the bit 30, 31, 15 or 7
// of x: no byte is extracted.
__device__ __forceinline__ void hist32_elem(uint32_t hl, uint32_t x) {
  red_shared_add(hl + ((x >> 16) & 0x3F80u), (x & 0x40000000u) ? 0x10000u : 1u);
  red_shared_add(hl + 0x4000u + ((x >> 9) & 0x3F80u), (x & 0x80000000u) ? 0x10000u : 1u);
  red_shared_add(hl + 0x8000u + ((x >> 1) & 0x3F80u), (x & 0x8000u) ? 0x10000u : 1u);
  red_shared_add(hl + 0xC000u + ((x << 7) & 0x3F80u), (x & 0x80u) ? 0x10000u : 1u);
}

// Histograms of chunk c of job J by the NT threads of the CTA, with the
// lane-indexed counters in sh (hist_counter_words(DT) + G words); the bin
// totals go to hist_out[g * 256 + b] and the symbols inside all-zero vectors
// to zs_out[g] (global or shared memory).  Ends with every thread past a
// barrier.  FP32 keeps two 16-bit counters per word (bins b and b + 128 of a
// group and lane, low and high half): its four groups then take the 64 KiB
// that two 16-bit groups take, three CTAs per SM instead of one.  A word
// counts at most kPkRound / 8 symbols per half in a round of kPkRound vectors
// (lane l of every warp adds into it: NT / 32 threads of kPkRound / NT
// vectors each, 4 symbols per vector and group), so chunks of more than
// kPkRound vectors are counted in rounds, each round's halves added into
// per-thread totals before the next.
constexpr uint32_t kPkRound = 1u << 18;  // vectors (4 MiB) per round: <= 32768 per half
template <int DT>
__host__ __device__ constexpr int hist_counter_words() {
  return DT == ZIPNN_FP32 ? 4 * 128 * 32 : (DT == ZIPNN_U8 ? 1 : 2) * 256 * 32;
}
template <int DT, int NT = kHistThreads>
__device__ void hist_chunk(const Job& J, uint64_t c, uint32_t* sh, uint32_t* hist_out,
                           uint32_t* zs_out) {
  constexpr int G = DT == ZIPNN_FP32 ? 4 : (DT == ZIPNN_U8 ? 1 : 2);
  constexpr int V = 16 / (DT == ZIPNN_FP32 ? 4 : (DT == ZIPNN_U8 ? 1 : 2));
  constexpr int ES = 16 / V;
  constexpr bool PK = DT == ZIPNN_FP32;
  constexpr int CW = hist_counter_words<DT>();
  const int tid = threadIdx.x, lane = tid & 31;
  const uint64_t off = c * J.chunk_bytes;
  const uint64_t nb = min((uint64_t)J.chunk_bytes, J.nbytes - off);
  const uint8_t* src = J.src + off;
  const uint8_t* base = J.base ? J.base + off : nullptr;

  uint32_t* zcnt = sh + CW;  // per group: symbols inside all-zero vectors
  for (int i = tid; i < CW + G; i += NT) sh[i] = 0;
  __syncthreads();
  uint32_t zc[G];
#pragma unroll
  for (int g = 0; g < G; g++) zc[g] = 0;
  uint32_t* hl = sh + lane;
  const uint32_t hls = (uint32_t)__cvta_generic_to_shared(hl);
  const uint64_t nvec = (nb + 15) / 16;
  const uint64_t m = nb / ES;
  constexpr int U = 4;  // vectors in flight per thread
  uint64_t vstart = tid;
  if constexpr (DT == ZIPNN_BF16 || DT == ZIPNN_FP16) {
    // whole rounds of NT * U vectors of whole 16-bit elements
    const uint64_t nfast = nb % 16 ? 0 : nvec / ((uint64_t)NT * U) * (NT * U);
    // the second round, up to where the in-loop prefetches start
    for (uint64_t vp = tid + (uint64_t)NT * U; vp < nfast && vp < 2ull * NT * U;
         vp += NT) {
      prefetch_l2(reinterpret_cast<const uint4*>(src) + vp);
      if (base) prefetch_l2(reinterpret_cast<const uint4*>(base) + vp);
    }
    for (uint64_t v0 = tid; v0 < nfast; v0 += (uint64_t)NT * U) {
      uint4 a[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const uint64_t v = v0 + (uint64_t)u * NT;
        const uint64_t vp = v + 2ull * NT * U;  // two rounds ahead
        if (vp < nfast) {
          prefetch_l2(reinterpret_cast<const uint4*>(src) + vp);
          if (base) prefetch_l2(reinterpret_cast<const uint4*>(base) + vp);
        }
        a[u] = __ldg(reinterpret_cast<const uint4*>(src) + v);
        if (base) {
          const uint4 b = __ldg(reinterpret_cast<const uint4*>(base) + v);
          a[u].x ^= b.x; a[u].y ^= b.y; a[u].z ^= b.z; a[u].w ^= b.w;
        }
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        hist16_words(hls, a[u].x, a[u].y);
        hist16_words(hls, a[u].z, a[u].w);
        const uint32_t any = a[u].x | a[u].y | a[u].z | a[u].w;
        if (!(any & 0x7F807F80u)) zc[0] += 8;       // 8 zero exponent bytes
        if (!(any & 0x807F807Fu)) zc[1 % G] += 8;   // 8 zero sign + fraction bytes
      }
    }
    vstart = nfast + tid;
  }
  // packed counters: running totals of this thread's words (bins b, b + 128)
  constexpr int PKW = PK ? (G * 128 + NT - 1) / NT : 1;
  uint32_t tot_lo[PKW], tot_hi[PKW];
#pragma unroll
  for (int i = 0; i < PKW; i++) tot_lo[i] = tot_hi[i] = 0;
  auto add_packed = [&]() {
#pragma unroll
    for (int i = 0; i < PKW; i++) {
      const int bw = tid + i * NT;
      if (bw < G * 128) {
#pragma unroll 8
        for (int l = 0; l < 32; l++) {
          const uint32_t w = sh[bw * 32 + ((l + bw) & 31)];
          tot_lo[i] += w & 0xFFFFu;
          tot_hi[i] += w >> 16;
        }
      }
    }
  };
  // rounds of kPkRound vectors with packed counters, else one round; the
  // round bounds are the same in every thread, so all of them meet the
  // barriers between rounds
  const uint64_t vb = vstart - (uint64_t)tid;
  const uint64_t rlen = PK ? (uint64_t)kPkRound : (nvec > vb ? nvec - vb : 1u);
  for (uint64_t r0 = vb; r0 < nvec; r0 += rlen) {
    if (PK && r0 != vb) {
      // a round is complete: fold the halves into the totals, clear the words
      __syncthreads();
      add_packed();
      __syncthreads();
      for (int i = tid; i < CW; i += NT) sh[i] = 0;
      __syncthreads();
    }
    const uint64_t rend = min(nvec, r0 + rlen);
    for (uint64_t v0 = r0 + (uint64_t)tid; v0 < rend; v0 += (uint64_t)NT * U) {
      uint4 a[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const uint64_t v = v0 + (uint64_t)u * NT;
        a[u] = v < rend ? load_vec(src, base, v, nb) : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        const uint64_t v = v0 + (uint64_t)u * NT;
        if (v >= rend) break;
        const int valid = (v + 1) * V <= m ? V : (int)(m - v * V);
        if constexpr (PK) {
          if (valid == V) {  // four whole elements
            hist32_elem(hls, a[u].x);
            hist32_elem(hls, a[u].y);
            hist32_elem(hls, a[u].z);
            hist32_elem(hls, a[u].w);
            const uint32_t any = a[u].x | a[u].y | a[u].z | a[u].w;
            if (!(any & 0x7F800000u)) zc[0] += 4;
            if (!(any & 0x807F0000u)) zc[1 % G] += 4;
            if (!(any & 0x0000FF00u)) zc[2 % G] += 4;
            if (!(any & 0x000000FFu)) zc[3 % G] += 4;
            continue;
          }
        }
        uint32_t g[4][4];
        split_vec(DT, a[u], g);
#pragma unroll
        for (int gg = 0; gg < G; gg++) {
          uint32_t any = 0;
#pragma unroll
          for (int q = 0; q < V / 4; q++) any |= g[gg][q];
          if (!any) zc[gg] += (uint32_t)valid;   // bytes past the tail were loaded as zero
        }
        // symbol b of group gg: word (gg * 256 + b) * 32 + lane, or with packed
        // counters word (gg * 128 + b % 128) * 32 + lane, half b / 128
        auto count = [&](int gg, uint32_t b) {
          if constexpr (PK)
            atomicAdd(&hl[(gg * 128 + (b & 127u)) * 32], (b & 128u) ? 0x10000u : 1u);
          else
            atomicAdd(&hl[(gg * 256 + b) * 32], 1u);
        };
        if (valid == V) {
#pragma unroll
          for (int gg = 0; gg < G; gg++)
#pragma unroll
            for (int k = 0; k < V; k++)
              count(gg, __byte_perm(g[gg][k >> 2], 0, 0x4440 + (k & 3)));
        } else {
#pragma unroll
          for (int gg = 0; gg < G; gg++)
#pragma unroll
            for (int k = 0; k < V; k++)
              if (k < valid) count(gg, __byte_perm(g[gg][k >> 2], 0, 0x4440 + (k & 3)));
        }
      }
    }
  }
#pragma unroll
  for (int g = 0; g < G; g++) {
    uint32_t z = zc[g];
    for (int o = 16; o; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if (lane == 0 && z) atomicAdd(&zcnt[g], z);
  }
  __syncthreads();
  if (tid < G) zs_out[tid] = zcnt[tid];
  // bin totals: thread b sums the 32 lane counters of bin b (rotated start so
  // the 32 threads of a warp read 32 different banks)
  if constexpr (PK) {
    add_packed();
#pragma unroll
    for (int i = 0; i < PKW; i++) {
      const int bw = tid + i * NT;
      if (bw < G * 128) {
        hist_out[(bw >> 7) * 256 + (bw & 127)] = tot_lo[i];
        hist_out[(bw >> 7) * 256 + (bw & 127) + 128] = tot_hi[i];
      }
    }
  } else {
    for (int b = tid; b < G * 256; b += NT) {
      uint32_t s = 0;
#pragma unroll 8
      for (int i = 0; i < 32; i++) s += sh[b * 32 + ((i + b) & 31)];
      hist_out[b] = s;
    }
  }
  __syncthreads();
}

template <int DTS>
__global__ void __launch_bounds__(kHistThreads)
k_hist(JobRef jr, uint32_t* __restrict__ hist, uint32_t* __restrict__ zsyms) {
  extern __shared__ uint32_t hsm[];
  const uint64_t chunk = blockIdx.x;
  const int j = find_job_chunk(jr, chunk);
  const Job& J = job_at(jr, j);
  const uint64_t c = chunk - J.chunk_begin;
  const uint64_t gc0 = J.gc_begin + c * elem_size(J.dtype);
  uint32_t* ho = hist + gc0 * 256;
  uint32_t* zo = zsyms + gc0;
  if (DTS >= 0) {
    hist_chunk<(DTS < 0 ? 0 : DTS)>(J, c, hsm, ho, zo);
    return;
  }
  switch (J.dtype) {
    case ZIPNN_BF16: hist_chunk<ZIPNN_BF16>(J, c, hsm, ho, zo); break;
    case ZIPNN_FP16: hist_chunk<ZIPNN_FP16>(J, c, hsm, ho, zo); break;
    case ZIPNN_FP32: hist_chunk<ZIPNN_FP32>(J, c, hsm, ho, zo); break;
    default: hist_chunk<ZIPNN_U8>(J, c, hsm, ho, zo); break;
  }
}

// counters + zero-symbol words: a launch that may hold FP32 chunks (packed
// counters) needs as much as one of 16-bit chunks
static int hist_smem_bytes(int max_groups) {
  const int g = max_groups > 2 ? 2 : max_groups;
  return (g * 256 * 32 + max_groups) * 4;
}

// ---------------------------------------------------------------------------
// k_build: one warp per group-chunk.

struct BuildSmem {
  uint32_t leafw[256];    // leaf weights, sorted by (count asc, symbol desc)
  uint8_t leafsym[256];
  uint8_t lens[256];      // code length per symbol
  uint32_t lst[2][512];   // package-merge lists (double buffer)
  uint32_t pk[256];       // packages of the previous list
  uint32_t leafbits[kMaxLen][16];  // which positions of list i are leaves
  uint32_t keys[256];
};

__device__ __forceinline__ int upper_bound_u32(const uint32_t* a, int n, uint32_t x) {
  int lo = 0, hi = n;  // first index with a[i] > x
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int lower_bound_u32(const uint32_t* a, int n, uint32_t x) {
  int lo = 0, hi = n;  // first index with a[i] >= x
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Shannon bound: any prefix code spends >= sum c log2(n / c) bits on counts c
// summing to n.  True when even that many bits (plus `fixed` bytes) cannot
// qualify against the raw size m, or, with have_best, cannot beat `best`.
__device__ bool bound_rules_out(const uint32_t cnt[8], uint32_t n, uint64_t fixed, uint32_t m,
                                bool have_best, uint64_t best) {
  float part = 0.f;
  const float lm = log2f((float)n);
  for (int k = 0; k < 8; k++)
    if (cnt[k]) part += (float)cnt[k] * (lm - log2f((float)cnt[k]));
  for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  const float lower = part * (1.0f - 1e-4f) - 64.0f;
  if (!(lower > 0.f)) return false;
  const uint64_t lb_bits = (uint64_t)lower;
  const uint64_t lb_size = fixed + 4ull * ((lb_bits + 31) / 32);
  return lb_size + (m >> 6) >= m || (have_best && lb_size >= best);
}

// Code lengths limited to kMaxLen bits for the counts cnt[k] of symbols
// lane + 32 k (nz >= 2 of them non-zero), by package-merge; into S.lens.
__device__ void pm_lengths(BuildSmem& S, const uint32_t cnt[8], uint32_t nz, int lane) {
  // --- sort the leaves by key = count << 8 | (255 - symbol) (ascending):
  // compact the non-zero symbols (ballot prefix), then rank each key among
  // the nz compacted keys (keys are distinct: the symbol part differs)
  {
    uint32_t basek = 0;
    const uint32_t ltm = (1u << lane) - 1u;
    for (int k = 0; k < 8; k++) {
      const uint32_t b = __ballot_sync(0xffffffffu, cnt[k] > 0);
      if (cnt[k]) {
        const int s = lane + 32 * k;
        S.keys[basek + __popc(b & ltm)] = (cnt[k] << 8) | (uint32_t)(255 - s);
      }
      basek += __popc(b);
    }
  }
  __syncwarp();
  if (nz <= 96) {
    for (uint32_t i = lane; i < nz; i += 32) {
      const uint32_t key = S.keys[i];
      uint32_t r = 0;
      for (uint32_t q = 0; q < nz; q++) r += (S.keys[q] < key);
      S.leafw[r] = key >> 8;
      S.leafsym[r] = (uint8_t)(255 - (key & 0xFFu));
    }
  } else {
    // many leaves: a bitonic sort of the keys padded to 256 with the largest
    // key (element i = 8 * lane + r in register r of the lane; partners 8 or
    // more apart are exchanged by shuffles), instead of nz compares per key
    uint32_t v[8];
#pragma unroll
    for (int r = 0; r < 8; r++) {
      const uint32_t i = 8u * lane + r;
      v[r] = i < nz ? S.keys[i] : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int size = 2; size <= 256; size <<= 1) {
#pragma unroll
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        if (stride >= 8) {
          const int ls = stride >> 3;  // partner lane distance
#pragma unroll
          for (int r = 0; r < 8; r++) {
            const uint32_t i = 8u * lane + r;
            const uint32_t o = __shfl_xor_sync(0xffffffffu, v[r], ls);
            const bool up = (i & (uint32_t)size) == 0, lower = (lane & ls) == 0;
            v[r] = (lower == up) ? min(v[r], o) : max(v[r], o);
          }
        } else {
#pragma unroll
          for (int r = 0; r < 8; r++) {
            if (r & stride) continue;
            const int q = r | stride;
            const bool up = ((8u * lane + r) & (uint32_t)size) == 0;
            const uint32_t a = v[r], b = v[q];
            v[r] = up ? min(a, b) : max(a, b);
            v[q] = up ? max(a, b) : min(a, b);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 8; r++) {
      const uint32_t i = 8u * lane + r;
      if (i < nz) {
        S.leafw[i] = v[r] >> 8;
        S.leafsym[i] = (uint8_t)(255 - (v[r] & 0xFFu));
      }
    }
  }
  for (int i = lane; i < kMaxLen * 16; i += 32) (&S.leafbits[0][0])[i] = 0;
  __syncwarp();

  // --- package-merge: list 0 = leaves; list i = merge(leaves, packages(list i-1))
  const int n = (int)nz;
  int sp = n;
  uint32_t* prev = S.lst[0];
  for (int k = lane; k < n; k += 32) prev[k] = S.leafw[k];
  __syncwarp();
  int cur_buf = 1;
  for (int lvl = 1; lvl < kMaxLen; lvl++) {
    uint32_t* cur = S.lst[cur_buf];
    const int np = sp >> 1;
    for (int k = lane; k < np; k += 32) S.pk[k] = prev[2 * k] + prev[2 * k + 1];
    __syncwarp();
    // the merged list, a leaf before a package of equal weight.  Few leaves:
    // each package and leaf finds its position by a binary search in the
    // other list.  Many (more than 96): merge path, lane l writes outputs
    // [l * seg, (l + 1) * seg), one binary search finding how many leaves
    // precede its first output, then a sequential merge that marks its
    // leaves' positions (at most two bitmap words)
    const int total = n + np, seg = (total + 31) >> 5;
    const int d0 = min(total, lane * seg), d1 = min(total, d0 + seg);
    if (n <= 96) {
      for (int k = lane; k < np; k += 32) {
        uint32_t w = S.pk[k];
        cur[k + upper_bound_u32(S.leafw, n, w)] = w;      // after leaves of equal weight
      }
      for (int k = lane; k < n; k += 32) {
        uint32_t w = S.leafw[k];
        int pos = k + lower_bound_u32(S.pk, np, w);
        cur[pos] = w;
        atomicOr(&S.leafbits[lvl][pos >> 5], 1u << (pos & 31));
      }
    } else if (d0 < d1) {
      int lo = max(0, d0 - np), hi = min(d0, n);
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (S.leafw[mid] <= S.pk[d0 - mid - 1]) lo = mid + 1; else hi = mid;
      }
      int li = lo, pi = d0 - lo;
      uint64_t mask = 0;  // leaf positions from word d0 / 32
      const int off = d0 & 31;
      for (int d = d0; d < d1; d++) {
        const bool leaf = pi >= np || (li < n && S.leafw[li] <= S.pk[pi]);
        cur[d] = leaf ? S.leafw[li] : S.pk[pi];
        if (leaf) {
          mask |= 1ull << (off + d - d0);
          li++;
        } else {
          pi++;
        }
      }
      if ((uint32_t)mask) atomicOr(&S.leafbits[lvl][d0 >> 5], (uint32_t)mask);
      if (mask >> 32) atomicOr(&S.leafbits[lvl][(d0 >> 5) + 1], (uint32_t)(mask >> 32));
    }
    __syncwarp();
    sp = total;
    prev = cur;
    cur_buf ^= 1;
  }

  // --- selection, from the last list down: a[i] leaves and p packages among
  // the first c items; the packages select the first 2p items of list i-1.
  int a[kMaxLen];
  {
    int take = 2 * (n - 1);
    for (int lvl = kMaxLen - 1; lvl >= 1; lvl--) {
      int leaves = 0;
      for (int wv = 0; wv < 16; wv++) {
        int lo = wv * 32;
        if (lo >= take) break;
        uint32_t bits = S.leafbits[lvl][wv];
        int upto = take - lo;
        if (upto < 32) bits &= (1u << upto) - 1u;
        leaves += __popc(bits);
      }
      a[lvl] = leaves;
      take = 2 * (take - leaves);
    }
    a[0] = take;  // list 0 holds leaves only
  }
  for (int k = lane; k < n; k += 32) {
    int len = 0;
    for (int lvl = 0; lvl < kMaxLen; lvl++) len += (k < a[lvl]);
    S.lens[S.leafsym[k]] = (uint8_t)len;
  }
  for (int k = 0; k < 8; k++)
    if (!cnt[k]) S.lens[lane + 32 * k] = 0;
  __syncwarp();

}

// Mode decision, length-limited code and canonical table of one group-chunk
// by one warp: hist256 holds its 256 symbol counts (global or shared memory),
// zs the symbols inside all-zero vectors, m the symbol count, T the
// sub-streams and es the element size.  Writes the 256 (len << 16 | code)
// entries to mycodes (coded groups only), the table bytes to tab and the
// result to *meta_out.
__device__ void build_gc(const uint32_t* hist256, uint32_t zs, uint32_t m, uint32_t T, int es,
                         BuildSmem& S, uint32_t* mycodes, uint8_t* tab, GcMeta* meta_out) {
  const int lane = threadIdx.x & 31;
  // counts of symbols s = lane + 32 k
  uint32_t cnt[8];
  uint32_t nz = 0;
  for (int k = 0; k < 8; k++) {
    cnt[k] = hist256[lane + 32 * k];
    nz += __popc(__ballot_sync(0xffffffffu, cnt[k] > 0));
  }
  for (int k = 0; k < 8; k++) mycodes[lane + 32 * k] = 0;

  GcMeta res;
  res.nz = nz;
  res.value = 0;
  res.size = 0;
  if (nz <= 1) {
    uint32_t sym = 0;
    for (int k = 0; k < 8; k++) {
      uint32_t b = __ballot_sync(0xffffffffu, cnt[k] > 0);
      if (b) sym = 32 * k + (__ffs(b) - 1);
    }
    res.mode = (nz == 0 || sym == 0) ? kZero : kConst;
    res.value = (res.mode == kConst) ? sym : 0;
    if (lane == 0) *meta_out = res;
    return;
  }

  const uint32_t V = 16u / (uint32_t)es, nv = (m + V - 1) / V;

  // HUFF candidate: a code for all m symbols (skipped when the Shannon bound
  // already shows it cannot qualify)
  const uint32_t h = (uint32_t)align_up(12 + nz, 4);
  const uint64_t fixed = (uint64_t)h + 4ull * (T - 1);
  bool huff_ok = false;
  uint64_t hsize = 0;
  uint8_t lenH[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (!bound_rules_out(cnt, m, fixed, m, false, 0)) {
    pm_lengths(S, cnt, nz, lane);
    uint32_t bits = 0;
    for (int k = 0; k < 8; k++) {
      lenH[k] = S.lens[lane + 32 * k];
      bits += cnt[k] * lenH[k];
    }
    for (int o = 16; o; o >>= 1) bits += __shfl_xor_sync(0xffffffffu, bits, o);
    hsize = fixed + 4ull * ((bits + 31) / 32);
    huff_ok = hsize + (m >> 6) < m;
    __syncwarp();
  }

  // SPARSE candidate: a code for the symbols outside all-zero vectors (the
  // zeros of those vectors leave the histogram) plus a bitmap of the vectors
  bool sparse_ok = false;
  uint64_t ssize = 0;
  uint32_t nz2 = 0;
  uint8_t lenS[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (zs > 0) {
    uint32_t cnt2[8];
    for (int k = 0; k < 8; k++) cnt2[k] = cnt[k];
    if (lane == 0) cnt2[0] -= zs;                    // symbol 0 is lane 0, k = 0
    for (int k = 0; k < 8; k++) nz2 += __popc(__ballot_sync(0xffffffffu, cnt2[k] > 0));
    if (nz2 >= 2) {
      const uint64_t fixed2 = align_up(12 + nz2, 4) + 4ull * ((nv + 31) / 32) + 4ull * (T - 1);
      if (!bound_rules_out(cnt2, m - zs, fixed2, m, huff_ok, hsize)) {
        pm_lengths(S, cnt2, nz2, lane);
        uint32_t bits2 = 0;
        for (int k = 0; k < 8; k++) {
          lenS[k] = S.lens[lane + 32 * k];
          bits2 += cnt2[k] * lenS[k];
        }
        for (int o = 16; o; o >>= 1) bits2 += __shfl_xor_sync(0xffffffffu, bits2, o);
        ssize = fixed2 + 4ull * ((bits2 + 31) / 32);
        sparse_ok = ssize + (m >> 6) < m;
        __syncwarp();
      }
    }
  }

  // --- mode decision (SPARSE only when strictly smaller than a qualifying HUFF)
  uint8_t mylen[8];
  if (sparse_ok && (!huff_ok || ssize < hsize)) {
    res.mode = kSparse;
    res.size = (uint32_t)ssize;
    res.nz = nz2;
    for (int k = 0; k < 8; k++) mylen[k] = lenS[k];
  } else if (huff_ok) {
    res.mode = kHuff;
    res.size = (uint32_t)hsize;
    for (int k = 0; k < 8; k++) mylen[k] = lenH[k];
  } else {
    res.mode = kRaw;
    res.size = m;
    if (lane == 0) *meta_out = res;
    return;
  }

  // --- canonical codes (RFC 1951 Sec. 3.2.2) and the table bytes
  uint32_t count[kMaxLen + 1];
  for (int l = 0; l <= kMaxLen; l++) count[l] = 0;
  for (int l = 1; l <= kMaxLen; l++)
    for (int k = 0; k < 8; k++) count[l] += __popc(__ballot_sync(0xffffffffu, mylen[k] == l));
  if (lane < kMaxLen) tab[lane] = (uint8_t)count[lane + 1];
  uint32_t code0 = 0, first_idx = 0;
  const uint32_t ltmask = (1u << lane) - 1u;
  for (int l = 1; l <= kMaxLen; l++) {
    code0 = (code0 + count[l - 1]) << 1;
    uint32_t basek = 0;
    for (int k = 0; k < 8; k++) {
      uint32_t b = __ballot_sync(0xffffffffu, mylen[k] == l);
      if (mylen[k] == l) {
        uint32_t r = basek + __popc(b & ltmask);
        mycodes[lane + 32 * k] = ((uint32_t)l << 16) | (code0 + r);
        tab[12 + first_idx + r] = (uint8_t)(lane + 32 * k);
      }
      basek += __popc(b);
    }
    first_idx += count[l];
  }
  if (lane == 0) *meta_out = res;
}


__global__ void __launch_bounds__(kBuildWarps * 32)
k_build(JobRef jr, uint64_t ngc_total, const uint32_t* __restrict__ hist,
        const uint32_t* __restrict__ zsyms, uint32_t* __restrict__ codes,
        uint8_t* __restrict__ tabs, GcMeta* __restrict__ meta) {
  __shared__ BuildSmem smem[kBuildWarps];
  const int wid = threadIdx.x >> 5;
  const uint64_t gc = (uint64_t)blockIdx.x * kBuildWarps + wid;
  if (gc >= ngc_total) return;
  const int j = find_job_gc(jr, gc);
  const Job& J = job_at(jr, j);
  const int es = elem_size(J.dtype), G = es;
  const uint64_t c = (gc - J.gc_begin) / G;
  const uint64_t nb = min((uint64_t)J.chunk_bytes, J.nbytes - c * J.chunk_bytes);
  build_gc(hist + gc * 256, zsyms[gc], (uint32_t)(nb / es), J.lanes, es, smem[wid],
           codes + gc * 256, tabs + gc * kTabBytes, meta + gc);
}

// ---------------------------------------------------------------------------
// k_scan: one CTA per tensor, exclusive scan of padded payload sizes.  With
// the skip-ahead probe (J.skip > 0, ZipNN Sec. 3.2 "Identifying
// compressibility") thread g first walks the tensor's chunks in order for
// group g: after a group-chunk decided raw, the same group of the next J.skip
// chunks becomes raw (the builder's result for them is discarded), then
// decisions resume.

constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads)
k_scan(JobRef jr, GcMeta* __restrict__ meta, uint64_t* __restrict__ offs,
       uint64_t* __restrict__ totals, uint32_t* __restrict__ err) {
  __shared__ uint64_t warp_sums[kScanThreads / 32];
  const int j = blockIdx.x;
  const Job& J = job_at(jr, j);
  const int G = elem_size(J.dtype);
  const uint64_t ngc = (uint64_t)J.n_chunks * G;
  if (J.skip) {
    if ((int)threadIdx.x < G) {
      const int g = threadIdx.x;
      uint32_t left = 0;
      for (uint32_t c = 0; c < J.n_chunks; c++) {
        GcMeta& M = meta[J.gc_begin + (uint64_t)c * G + g];
        if (left) {
          left--;
          const uint64_t nb = min((uint64_t)J.chunk_bytes, J.nbytes - (uint64_t)c * J.chunk_bytes);
          M.mode = kRaw;
          M.value = 0;
          M.size = (uint32_t)(nb / G);
        } else if (M.mode == kRaw) {
          left = J.skip;
        }
      }
    }
    __syncthreads();
  }
  const uint64_t per = (ngc + kScanThreads - 1) / kScanThreads;
  const uint64_t b0 = min(ngc, per * threadIdx.x), b1 = min(ngc, b0 + per);
  uint64_t local = 0;
  for (uint64_t i = b0; i < b1; i++) local += align_up(meta[J.gc_begin + i].size, 16);
  // block exclusive scan of `local`
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t incl = local;
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint64_t w = warp_sums[lane];
    uint64_t wi = w;
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    warp_sums[lane] = wi - w;
  }
  __syncthreads();
  uint64_t run = warp_sums[wid] + incl - local;
  for (uint64_t i = b0; i < b1; i++) {
    offs[J.gc_begin + i] = run;
    run += align_up(meta[J.gc_begin + i].size, 16);
  }
  if (threadIdx.x == kScanThreads - 1) {
    const uint64_t P = kHdrBytes + ngc * kEntryBytes;
    const uint64_t total = P + run;
    totals[j] = total;
    if (J.out_nbytes) *J.out_nbytes = total;
    if (J.out_capacity && total > J.out_capacity) atomicOr(err, 2u);  // ENOMEM
  }
}

// ---------------------------------------------------------------------------
// k_pack: one CTA per chunk (extra CTAs write the headers).
//
// Each sub-stream t is split into R consecutive parts (R = threads / T), so a
// 512-thread CTA covers a 128-lane chunk with 4 threads per sub-stream.  The
// unit (t, k) of part k of sub-stream t runs on thread k*T + t: lanes of a warp
// hold consecutive t and touch consecutive 16-B vectors (coalesced).
//   pass A: bits of every unit for each Huffman group; raw groups are written
//           to their payloads in the same pass;
//   scan  : exclusive scan of the unit bits in (t, k) order -> bit offset of
//           every unit (the offset of (t, 0) is the sub-stream start);
//   pass B: codes emitted MSB-first from each unit's offset (the words a unit
//           shares with its neighbours are merged with atomicOr).
// With 2 CTAs per SM the chunks in flight (~78 MB) stay in L2 between the
// passes, so the input is read from DRAM once here.

constexpr int kPackThreads = 512;
constexpr int kPackMaxUnits = 1024;
constexpr uint32_t kPackSlotWords = 20480;  // 80 KiB of unit slots
constexpr uint32_t kPrefetchAhead = 8;  // pass-A vectors between an L2 prefetch and its load

__device__ __forceinline__ void put_u64(uint8_t* p, uint64_t v) {
  for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}
__device__ __forceinline__ void put_u32(uint8_t* p, uint32_t v) {
  for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}

// a / b and a % b for the sub-stream geometry: a shift and a mask when b is a
// power of two (the lane counts and unit counts in use), else the division.
__device__ __forceinline__ uint32_t gdiv(uint32_t a, uint32_t b) {
  return (b & (b - 1u)) == 0 ? a >> (__ffs(b) - 1) : a / b;
}
__device__ __forceinline__ uint32_t gmod(uint32_t a, uint32_t b) {
  return (b & (b - 1u)) == 0 ? a & (b - 1u) : a % b;
}

template <int DT> struct PTraits;
template <> struct PTraits<ZIPNN_BF16> { static constexpr int G = 2, V = 8; };
template <> struct PTraits<ZIPNN_FP16> { static constexpr int G = 2, V = 8; };
template <> struct PTraits<ZIPNN_FP32> { static constexpr int G = 4, V = 4; };
template <> struct PTraits<ZIPNN_U8> { static constexpr int G = 1, V = 16; };

struct PackSmem {
  uint32_t codes[4][256];
  uint32_t part[4][kPackMaxUnits + 1];  // unit bits, then exclusive offsets
  uint32_t wsum[kPackThreads / 32];
  GcMeta meta[4];
  uint64_t off[4];
  uint32_t capw[4];   // bitstream words available in the payload
  uint32_t hsz[4];    // table + start-offset bytes before the bitstream
  uint32_t sbits[kPackMaxUnits];  // bits of each unit of the slot-staged group
  uint32_t ptab[1024];  // pair table of the 16-bit pass A (pack_pair_a)
};

// Exclusive scan of a[0..n) in place (block-wide), the total into a[n];
// n <= kPackMaxUnits.
__device__ void block_exclusive_scan(uint32_t* a, uint32_t n, uint32_t* wsum) {
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t per = (n + nthr - 1) / nthr;
  const uint32_t b0 = min(n, per * tid), b1 = min(n, b0 + per);
  uint32_t local = 0;
  for (uint32_t i = b0; i < b1; i++) local += a[i];
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nw = nthr >> 5;
    uint32_t w = lane < nw ? wsum[lane] : 0u, wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) wsum[lane] = wi - w;
  }
  __syncthreads();
  uint32_t run = wsum[wid] + incl - local;
  for (uint32_t i = b0; i < b1; i++) {
    const uint32_t b = a[i];
    a[i] = run;
    run += b;
  }
  if (b0 < b1 && b1 == n) a[n] = run;  // the total, after the last offset
  __syncthreads();
}

// MSB-first writer of one unit's bits: acc holds nacc (< 32) pending bits;
// whole words go out with a plain store, except the unit's first word, which
// it shares with the previous unit (atomicOr into a zeroed word).
struct BitWriter {
  uint32_t* words;
  uint64_t acc;
  uint32_t nacc, wi, capw;
  bool first;
  __device__ __forceinline__ void put(uint32_t x, uint32_t n) {  // n <= 32, x < 2^n
    acc = (acc << n) | x;
    nacc += n;
    if (nacc >= 32) {
      nacc -= 32;
      const uint32_t word = (uint32_t)(acc >> nacc);
      if (wi < capw) {  // always true when the input did not change
        if (first) atomicOr(&words[wi], word);
        else words[wi] = word;
      }
      first = false;
      wi++;
      acc &= (1ull << nacc) - 1ull;
    }
  }
  __device__ __forceinline__ void put64(uint64_t x, uint32_t n) {  // n <= 64
    if (n > 32) {
      put((uint32_t)(x >> 32), n - 32);
      put((uint32_t)x, 32);
    } else {
      put((uint32_t)x, n);
    }
  }
  __device__ __forceinline__ void flush() {
    if (nacc > 0 && wi < capw) atomicOr(&words[wi], (uint32_t)(acc << (32 - nacc)));
  }
};

// MSB-first writer into a unit's private shared-memory slot of cap words.
// Counts every bit; words past the slot are dropped (the unit then takes the
// fallback path that re-reads its input).
struct SlotWriter {
  uint32_t slot;   // shared-window address of the unit's slot
  uint64_t acc;
  uint32_t nacc, wi, cap, bits;
  __device__ __forceinline__ void put(uint32_t x, uint32_t n) {  // n <= 32, x < 2^n
    acc = (acc << n) | x;
    nacc += n;
    bits += n;
    if (nacc >= 32) {
      nacc -= 32;
      if (wi < cap) sts32(slot + 4u * wi, (uint32_t)(acc >> nacc));
      wi++;
      acc &= (1ull << nacc) - 1ull;
    }
  }
  __device__ __forceinline__ void put64(uint64_t x, uint32_t n) {
    if (n > 32) {
      put((uint32_t)(x >> 32), n - 32);
      put((uint32_t)x, 32);
    } else {
      put((uint32_t)x, n);
    }
  }
  __device__ __forceinline__ void finish() {
    if (nacc > 0 && wi < cap) sts32(slot + 4u * wi, (uint32_t)(acc << (32 - nacc)));
  }
};

// Slot writer of the specialised pass A: the pending bits sit left-aligned
// in one 32-bit word; an append of n <= 32 bits places them with one 64-bit
// shift and stores a word when 32 bits are complete.  Same bits, counts and
// overflow rule as SlotWriter.
struct SlotWriter32 {
  uint32_t slot;   // shared-window address of the unit's slot
  uint32_t cur, nb, wi, cap, bits;
  __device__ __forceinline__ void put(uint32_t x, uint32_t n) {  // 1 <= n <= 32, x < 2^n
    const uint32_t total = nb + n;                                // <= 63
    const uint64_t X = (uint64_t)x << (64 - total);
    const uint32_t hi = cur | (uint32_t)(X >> 32);
    bits += n;
    if (total >= 32) {
      if (wi < cap) sts32(slot + 4u * wi, hi);
      wi++;
      cur = (uint32_t)X;
      nb = total - 32;
    } else {
      cur = hi;
      nb = total;
    }
  }
  __device__ __forceinline__ void put48(uint64_t x, uint32_t n) {  // n <= 48
    if (n > 32) {
      put((uint32_t)(x >> 32), n - 32);
      put((uint32_t)x, 32);
    } else {
      put((uint32_t)x, n);
    }
  }
  __device__ __forceinline__ void finish() {
    if (nb > 0 && wi < cap) sts32(slot + 4u * wi, cur);
  }
};

// Codes of 4 consecutive symbols (bytes of w) joined MSB-first: <= 48 bits.
__device__ __forceinline__ uint64_t join4(uint32_t cb, uint32_t w, uint32_t& len) {
  const uint32_t e0 = code_of(cb, w, 0), e1 = code_of(cb, w, 1);
  const uint32_t e2 = code_of(cb, w, 2), e3 = code_of(cb, w, 3);
  const uint32_t l1 = e1 >> 16, l3 = e3 >> 16;
  const uint32_t p0 = ((e0 & 0xFFFFu) << l1) | (e1 & 0xFFFFu);   // <= 24 bits
  const uint32_t p1 = ((e2 & 0xFFFFu) << l3) | (e3 & 0xFFFFu);
  const uint32_t lp0 = (e0 >> 16) + l1, lp1 = (e2 >> 16) + l3;
  len = lp0 + lp1;
  return ((uint64_t)p0 << lp1) | p1;
}

// Sum of the code lengths of the 4 bytes of w.
__device__ __forceinline__ uint32_t len4(uint32_t cb, uint32_t w) {
  return (code_of(cb, w, 0) >> 16) + (code_of(cb, w, 1) >> 16) + (code_of(cb, w, 2) >> 16) +
         (code_of(cb, w, 3) >> 16);
}

// Pass A for the dominant chunk layout: group 0 Huffman (slot-encoded), every
// other group raw, zero or constant (bit g of raw set for raw groups), a whole
// chunk whose vectors split evenly over the T sub-streams and R parts (per
// vectors per unit).  No tails: per vector one 16-B load (two in flight, the
// line requested from L2 eight vectors earlier), the
// split, V/4 joined code appends into the unit's slot and one store per raw
// group.
template <int DT>
__device__ __forceinline__ void pack_fast_a(const uint8_t* src, const uint8_t* base, uint32_t T,
                                            uint32_t R, uint32_t per, uint32_t* slots,
                                            uint32_t slot_cap, PackSmem& S, uint8_t* out,
                                            uint64_t P, uint32_t raw) {
  constexpr int G = PTraits<DT>::G, V = PTraits<DT>::V;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const uint32_t units = T * R;
  uint8_t* rawp[G];
#pragma unroll
  for (int g = 0; g < G; g++) rawp[g] = out + P + S.off[g];
  const uint32_t codes0 = smem_u32(S.codes[0]);
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  const uint4* b4 = reinterpret_cast<const uint4*>(base);
  auto ld = [&](uint32_t v) -> uint4 {
    uint4 a = __ldg(s4 + v);
    if (base) {
      const uint4 b = __ldg(b4 + v);
      a.x ^= b.x; a.y ^= b.y; a.z ^= b.z; a.w ^= b.w;
    }
    return a;
  };
  for (uint32_t u = tid; u < units; u += nthr) {
    const uint32_t t = gmod(u, T), k = gdiv(u, T), ui = t * R + k;
    SlotWriter32 sw;
    sw.slot = smem_u32(slots) + 4u * ui * slot_cap;
    sw.cur = 0;
    sw.nb = 0;
    sw.wi = 0;
    sw.cap = slot_cap;
    sw.bits = 0;
    uint32_t v = t + k * per * T;
    constexpr uint32_t D = 2;
    for (uint32_t i = D; i < kPrefetchAhead && i < per; i++) {
      prefetch_l2(s4 + v + i * T);
      if (base) prefetch_l2(b4 + v + i * T);
    }
    uint4 a0 = ld(v), a1 = per > 1 ? ld(v + T) : make_uint4(0, 0, 0, 0);
    auto one = [&](uint4& a, uint32_t i) {
      uint32_t g4[4][4];
      split_vec(DT, a, g4);
      if (i + D < per) a = ld(v + D * T);
      if (i + kPrefetchAhead < per) {
        prefetch_l2(s4 + v + kPrefetchAhead * T);
        if (base) prefetch_l2(b4 + v + kPrefetchAhead * T);
      }
      if constexpr (V / 4 == 1) {
        uint32_t len;
        const uint64_t x = join4(codes0, g4[0][0], len);
        sw.put48(x, len);
      } else {
#pragma unroll
        for (int q = 0; q < V / 4; q += 2) {
          uint32_t l0, l1;
          const uint64_t x0 = join4(codes0, g4[0][q], l0);
          const uint64_t x1 = join4(codes0, g4[0][q + 1], l1);
          if (l0 + l1 <= 32) {
            sw.put(((uint32_t)x0 << l1) | (uint32_t)x1, l0 + l1);
          } else {
            sw.put48(x0, l0);
            sw.put48(x1, l1);
          }
        }
      }
#pragma unroll
      for (int g = 1; g < G; g++) {
        if (!(raw >> g & 1u)) continue;
        if (V == 8) reinterpret_cast<uint2*>(rawp[g])[v] = make_uint2(g4[g][0], g4[g][1]);
        else reinterpret_cast<uint32_t*>(rawp[g])[v] = g4[g][0];
      }
      v += T;
    };
    for (uint32_t i = 0; i < per; i += D) {
      one(a0, i);
      if (i + 1 < per) one(a1, i + 1);
    }
    sw.finish();
    S.sbits[ui] = sw.bits;
    S.part[0][ui] = sw.bits;
  }
}

// Pass A for the same layout in 16-bit chunks whose exponent code gives its
// symbols distinct residues mod 32 (nearly every chunk of a model: the
// exponents of one chunk span fewer than 32 values).  Entry a + 32 b of the
// pair table holds the codes of the symbols with residues a and b joined
// MSB-first, as (joined code << 6) | joined length (<= 24 bits, <= 24).  An
// element pair x (one 32-bit word, first element in the low half) finds its
// entry without splitting bytes: the residues sit at bits 7-11 and 23-27, and
// (x & 0x0F800F80) * 0x801 places them side by side at bits 18-27, so the
// product's upper half is the entry's byte offset (plus the table's address,
// added in the same multiply-add).  Two entries (four symbols, <= 32 bits in
// all but rare cases) are joined in one register and appended to the unit's
// slot through a 64-bit accumulator that emits at most one word per append.
// Same slot words, bit counts and overflow rule as pack_fast_a.
constexpr uint32_t kNoSym = 0x100, kClash = 0x200;

// Builds S.ptab from S.codes[0] (all threads, S.codes[0] visible; no
// barrier: the caller's next one publishes the table); false when two
// symbols of the code share a residue (S.ptab unused).  Every warp finds the
// symbol of each residue itself (lane r: residue r), so the check needs no
// shared state.
__device__ bool build_pair_table(PackSmem& S) {
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  uint32_t sym = kNoSym;
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const uint32_t sy = (uint32_t)lane + 32u * k;
    if (S.codes[0][sy] >> 16) sym = sym == kNoSym ? sy : kClash;
  }
  if (__any_sync(0xffffffffu, sym == kClash)) return false;
  for (int i = tid; i < 1024; i += nthr) {  // warp-uniform trip count
    const uint32_t sa = __shfl_sync(0xffffffffu, sym, i & 31);
    const uint32_t sb = __shfl_sync(0xffffffffu, sym, i >> 5);
    uint32_t e = 0;
    if (sa < 256 && sb < 256) {
      const uint32_t ca = S.codes[0][sa], cb = S.codes[0][sb];
      const uint32_t lb = cb >> 16;
      e = ((((ca & 0xFFFFu) << lb) | (cb & 0xFFFFu)) << 6) | ((ca >> 16) + lb);
    }
    S.ptab[i] = e;
  }
  return true;
}

// One unit of pack_pair_a: vectors v, v + T, ... (per of them) from s4
// (XOR b4 when XB), its fraction bytes to rawp when RW; bits into the slot
// at shared address sa0 whose last word is at slast; returns the unit's bits.
// Branch-free appends: every append stores a word at the slot's next free
// word (the finished word when 32 bits are complete, else one that a later
// store overwrites or that lies past the unit's bits); a unit that runs past
// its slot is re-encoded from the input, so the clamped stores there are
// never read.
template <bool XB, bool RW>
__device__ __forceinline__ uint32_t pair_unit(const uint4* __restrict__ s4,
                                       const uint4* __restrict__ b4, uint2* rawp,
                                       uint32_t v, uint32_t T, uint32_t per, uint32_t pb16,
                                       uint32_t sa0, uint32_t slast) {
  uint32_t sa = sa0, lo = 0, hi = 0, nb = 0;  // pending bits: the low nb of hi:lo
  auto ld = [&](uint32_t w) -> uint4 {
    uint4 a = __ldg(s4 + w);
    if (XB) {
      const uint4 b = __ldg(b4 + w);
      a.x ^= b.x; a.y ^= b.y; a.z ^= b.z; a.w ^= b.w;
    }
    return a;
  };
  auto pf = [&](uint32_t w) {
    prefetch_l2(s4 + w);
    if (XB) prefetch_l2(b4 + w);
  };
  auto entry = [&](uint32_t x) -> uint32_t {
    return lds32(((x & 0x0F800F80u) * 0x801u + pb16) >> 16);
  };
  // sign + fraction bytes of the two elements of x at bytes 0 and 2
  auto frac2 = [](uint32_t x) -> uint32_t {
    return (x & 0x007F007Fu) | ((x >> 8) & 0x00800080u);
  };
  // append the L (0..32) bits of V
  auto put = [&](uint32_t V, uint32_t L) {
    hi = __funnelshift_lc(lo, hi, L);
    lo = __funnelshift_lc(0u, lo, L) | V;
    nb += L;
    sts32(min(sa, slast), __funnelshift_r(lo, hi, nb - 32u));  // the word if nb >= 32
    const bool full = nb >= 32;
    sa += full ? 4u : 0u;
    nb -= full ? 32u : 0u;
  };
  // four symbols: the entries of two element pairs
  auto quad = [&](uint32_t E0, uint32_t E1) {
    const uint32_t L = (E0 + E1) & 63u;
    if (L <= 32) {
      put(__funnelshift_l(0u, E0 >> 6, E1) | (E1 >> 6), L);
    } else {
      put(E0 >> 6, E0 & 63u);
      put(E1 >> 6, E1 & 63u);
    }
  };
  // one vector (a); then a <- the vector two ahead (LD) and an L2 prefetch of
  // the one kPrefetchAhead ahead (PF)
  auto one = [&](uint4& a, bool LD, bool PF) {
    const uint4 x = a;
    if (LD) a = ld(v + 2 * T);
    if (PF) pf(v + kPrefetchAhead * T);
    const uint32_t E0 = entry(x.x), E1 = entry(x.y), E2 = entry(x.z), E3 = entry(x.w);
    if (RW)
      rawp[v] = make_uint2(__byte_perm(frac2(x.x), frac2(x.y), 0x6420),
                           __byte_perm(frac2(x.z), frac2(x.w), 0x6420));
    quad(E0, E1);
    quad(E2, E3);
    v += T;
  };
  for (uint32_t i = 2; i < kPrefetchAhead && i < per; i++) pf(v + i * T);
  uint4 a0 = ld(v), a1 = per > 1 ? ld(v + T) : make_uint4(0, 0, 0, 0);
  uint32_t i = 0;
  for (; i + kPrefetchAhead + 1 < per; i += 2) {
    one(a0, true, true);
    one(a1, true, true);
  }
  for (; i < per; i += 2) {
    one(a0, i + 2 < per, i + kPrefetchAhead < per);
    if (i + 1 < per) one(a1, i + 3 < per, i + 1 + kPrefetchAhead < per);
  }
  if (nb) sts32(min(sa, slast), lo << (32 - nb));
  return (sa - sa0) * 8u + nb;
}

// The FP32 unit of pack_pair_a: a vector holds four elements, whose exponent
// bytes (bits 23-30) a byte permute gathers into the 16-bit pair layout (two
// entries, one four-symbol append per vector); the three other byte groups are
// stored through rawp[0..2] (groups 1-3; null: not raw).
template <bool XB>
__device__ __forceinline__ uint32_t pair_unit32(const uint4* __restrict__ s4,
                                                const uint4* __restrict__ b4,
                                                uint32_t* const (&rawp)[3], uint32_t v, uint32_t T,
                                                uint32_t per, uint32_t pb16, uint32_t sa0,
                                                uint32_t slast) {
  uint32_t sa = sa0, lo = 0, hi = 0, nb = 0;  // pending bits: the low nb of hi:lo
  auto ld = [&](uint32_t w) -> uint4 {
    uint4 a = __ldg(s4 + w);
    if (XB) {
      const uint4 b = __ldg(b4 + w);
      a.x ^= b.x; a.y ^= b.y; a.z ^= b.z; a.w ^= b.w;
    }
    return a;
  };
  auto pf = [&](uint32_t w) {
    prefetch_l2(s4 + w);
    if (XB) prefetch_l2(b4 + w);
  };
  auto entry = [&](uint32_t x) -> uint32_t {
    return lds32(((x & 0x0F800F80u) * 0x801u + pb16) >> 16);
  };
  auto put = [&](uint32_t V, uint32_t L) {
    hi = __funnelshift_lc(lo, hi, L);
    lo = __funnelshift_lc(0u, lo, L) | V;
    nb += L;
    sts32(min(sa, slast), __funnelshift_r(lo, hi, nb - 32u));  // the word if nb >= 32
    const bool full = nb >= 32;
    sa += full ? 4u : 0u;
    nb -= full ? 32u : 0u;
  };
  const bool anyraw = rawp[0] || rawp[1] || rawp[2];
  auto one = [&](uint4& a, bool LD, bool PF) {
    const uint4 x = a;
    if (LD) a = ld(v + 2 * T);
    if (PF) pf(v + kPrefetchAhead * T);
    // high halves of elements 0,1 and 2,3: exponents at bits 7-14 and 23-30
    const uint32_t E0 = entry(__byte_perm(x.x, x.y, 0x7632));
    const uint32_t E1 = entry(__byte_perm(x.z, x.w, 0x7632));
    if (anyraw) {
      const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
      uint32_t g[4];
      split32(xs, g);
#pragma unroll
      for (int q = 0; q < 3; q++)
        if (rawp[q]) rawp[q][v] = g[q + 1];
    }
    const uint32_t L = (E0 + E1) & 63u;
    if (L <= 32) {
      put(__funnelshift_l(0u, E0 >> 6, E1) | (E1 >> 6), L);
    } else {
      put(E0 >> 6, E0 & 63u);
      put(E1 >> 6, E1 & 63u);
    }
    v += T;
  };
  for (uint32_t i = 2; i < kPrefetchAhead && i < per; i++) pf(v + i * T);
  uint4 a0 = ld(v), a1 = per > 1 ? ld(v + T) : make_uint4(0, 0, 0, 0);
  uint32_t i = 0;
  for (; i + kPrefetchAhead + 1 < per; i += 2) {
    one(a0, true, true);
    one(a1, true, true);
  }
  for (; i < per; i += 2) {
    one(a0, i + 2 < per, i + kPrefetchAhead < per);
    if (i + 1 < per) one(a1, i + 3 < per, i + 1 + kPrefetchAhead < per);
  }
  if (nb) sts32(min(sa, slast), lo << (32 - nb));
  return (sa - sa0) * 8u + nb;
}

template <int DT>
__device__ __forceinline__ void pack_pair_a(const uint8_t* src, const uint8_t* base, uint32_t T,
                                            uint32_t R, uint32_t per, uint32_t* slots,
                                            uint32_t slot_cap, PackSmem& S, uint8_t* out,
                                            uint64_t P, uint32_t raw) {
  static_assert(DT == ZIPNN_BF16 || DT == ZIPNN_FP16 || DT == ZIPNN_FP32,
                "16-bit or FP32 chunks");
  const int tid = threadIdx.x, nthr = blockDim.x;
  const uint32_t units = T * R;
  if constexpr (DT == ZIPNN_FP32) {
    uint32_t* const rawp[3] = {
        (raw >> 1 & 1u) ? reinterpret_cast<uint32_t*>(out + P + S.off[1]) : nullptr,
        (raw >> 2 & 1u) ? reinterpret_cast<uint32_t*>(out + P + S.off[2]) : nullptr,
        (raw >> 3 & 1u) ? reinterpret_cast<uint32_t*>(out + P + S.off[3]) : nullptr};
    const uint32_t pb16 = smem_u32(S.ptab) << 16;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    const uint4* b4 = reinterpret_cast<const uint4*>(base);
    for (uint32_t u = tid; u < units; u += nthr) {
      const uint32_t t = gmod(u, T), k = gdiv(u, T), ui = t * R + k;
      const uint32_t sa0 = smem_u32(slots) + 4u * ui * slot_cap, slast = sa0 + 4u * (slot_cap - 1);
      const uint32_t v = t + k * per * T;
      const uint32_t bits = base ? pair_unit32<true>(s4, b4, rawp, v, T, per, pb16, sa0, slast)
                                 : pair_unit32<false>(s4, b4, rawp, v, T, per, pb16, sa0, slast);
      S.sbits[ui] = bits;
      S.part[0][ui] = bits;
    }
    return;
  }
  uint2* const rawp = reinterpret_cast<uint2*>(out + P + S.off[1]);
  const bool rw = (raw >> 1 & 1u) != 0;
  const uint32_t pb16 = smem_u32(S.ptab) << 16;  // table address < 61440 (checked by the caller)
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  const uint4* b4 = reinterpret_cast<const uint4*>(base);
  for (uint32_t u = tid; u < units; u += nthr) {
    const uint32_t t = gmod(u, T), k = gdiv(u, T), ui = t * R + k;
    const uint32_t sa0 = smem_u32(slots) + 4u * ui * slot_cap, slast = sa0 + 4u * (slot_cap - 1);
    const uint32_t v = t + k * per * T;
    uint32_t bits;
    if (base)
      bits = rw ? pair_unit<true, true>(s4, b4, rawp, v, T, per, pb16, sa0, slast)
                : pair_unit<true, false>(s4, b4, rawp, v, T, per, pb16, sa0, slast);
    else
      bits = rw ? pair_unit<false, true>(s4, b4, rawp, v, T, per, pb16, sa0, slast)
                : pair_unit<false, false>(s4, b4, rawp, v, T, per, pb16, sa0, slast);
    S.sbits[ui] = bits;
    S.part[0][ui] = bits;
  }
}

__device__ __forceinline__ bool coded_mode_pack(uint32_t m) { return m == kHuff || m == kSparse; }

// Map entries of chunk c (threads 0..G-1) from S.meta and S.off.
template <int G>
__device__ __forceinline__ void write_map_entries(const Job& J, uint64_t c, const PackSmem& S) {
  const int tid = threadIdx.x;
  if (tid < G) {
    uint8_t* e = J.dst + kHdrBytes + (c * G + tid) * kEntryBytes;
    put_u64(e, S.off[tid]);
    put_u32(e + 8, S.meta[tid].size);
    e[12] = (uint8_t)S.meta[tid].mode;
    e[13] = (uint8_t)S.meta[tid].value;
    e[14] = 0;
    e[15] = 0;
  }
}

// Packing of chunk c whose mode records (S.meta), payload offsets (S.off) and
// codes of its coded groups (S.codes) are in shared memory and whose map
// entries have been written; tabp[g] points to group g's table bytes.
template <int DT, bool S2 = false>
__device__ void pack_chunk_core(const Job& J, uint64_t c, PackSmem& S, uint32_t* slots,
                                const uint8_t* const* tabp);

template <int DT, bool S2 = false>
__device__ void pack_chunk(const Job& J, uint64_t c, PackSmem& S, uint32_t* slots,
                           const uint32_t* codes, const uint8_t* tabs, const GcMeta* meta,
                           const uint64_t* offs) {
  constexpr int G = PTraits<DT>::G;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const uint64_t gc0 = J.gc_begin + c * G;
  if (tid < G) {
    S.meta[tid] = meta[gc0 + tid];
    S.off[tid] = offs[gc0 + tid];
  }
  // group 0's code and table bytes (coded in nearly every chunk) in the same
  // round trip; the table bytes go out below, the rest of it zero
  for (int s = tid; s < 256; s += nthr) S.codes[0][s] = codes[gc0 * 256 + s];
  const uint32_t tw =
      tid < kTabBytes / 4 ? reinterpret_cast<const uint32_t*>(tabs + gc0 * kTabBytes)[tid] : 0u;
  __syncthreads();
  write_map_entries<G>(J, c, S);
#pragma unroll
  for (int g = 1; g < G; g++)
    if (S.meta[g].mode == kHuff || S.meta[g].mode == kSparse)
      for (int s = tid; s < 256; s += nthr) S.codes[g][s] = codes[(gc0 + g) * 256 + s];
  if (coded_mode_pack(S.meta[0].mode)) {
    const uint32_t n = 12 + S.meta[0].nz, b = 4u * (uint32_t)tid;
    if (b < n)
      *reinterpret_cast<uint32_t*>(J.dst + kHdrBytes + (uint64_t)J.n_chunks * G * kEntryBytes +
                                   S.off[0] + b) = n - b >= 4 ? tw : tw & ((1u << 8 * (n - b)) - 1u);
  }
  const uint8_t* tabp[4] = {nullptr, nullptr, nullptr, nullptr};  // null: written
#pragma unroll
  for (int g = 1; g < G; g++) tabp[g] = tabs + (gc0 + g) * kTabBytes;
  pack_chunk_core<DT, S2>(J, c, S, slots, tabp);
}

// Pass B of a chunk whose group 0 is its only coded group and whose units
// (offsets in S.part[0], bits in S.sbits) hold 32 to slot_cap * 32 bits
// each: word w (bits 32w .. 32w + 31 of the bitstream, tot bits, capw words
// of payload at words) belongs to the unit holding bit 32w, so each word is
// written whole (no zeroed words, no atomics) from at most two units' slots.
// Warp k writes the words of its share of the units, 32 consecutive words at
// a time (one 128-B store); each lane follows the unit of its word with a
// cursor that only moves forward (units are consecutive in the stream: the
// next one starts where the current one ends).  Then the padding words.
__device__ __forceinline__ void pass_b_whole(const PackSmem& S, const uint32_t* slots,
                                             uint32_t slot_cap, uint32_t units, uint32_t* words,
                                             uint32_t capw, uint32_t tot) {
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, nwarps = nthr >> 5;
  const uint32_t sl0 = smem_u32(slots);
  const uint32_t upw = (units + (uint32_t)nwarps - 1) / (uint32_t)nwarps;
  const uint32_t u0 = min(units, (uint32_t)(tid >> 5) * upw), u1 = min(units, u0 + upw);
  if (u0 < u1) {
    const uint32_t wend = u1 < units ? (S.part[0][u1] + 31) >> 5 : (tot + 31) >> 5;
    uint32_t cu = u0, o = S.part[0][u0], e = o + S.sbits[u0];
    for (uint32_t w = ((o + 31) >> 5) + (uint32_t)lane; w < wend; w += 32) {
      const uint32_t bit = 32u * w;
      while (bit >= e) {  // at most a few units per step (each holds >= 32 bits)
        cu++;
        o = e;
        e = o + S.sbits[cu];
      }
      const uint32_t k = bit - o, i = k >> 5, r = e - bit;
      const uint32_t sl = sl0 + 4u * cu * slot_cap;
      const uint32_t a = lds32v(sl + 4u * i);
      const uint32_t b = 32u * (i + 1) < e - o ? lds32v(sl + 4u * (i + 1)) : 0u;
      uint32_t x = __funnelshift_l(b, a, k & 31);
      if (r < 32 && cu + 1 < units) x |= lds32v(sl + 4u * slot_cap) >> r;
      words[w] = x;
    }
  }
  for (uint32_t w = ((tot + 31) >> 5) + tid; w < capw; w += nthr) words[w] = 0;
}

template <int DT, bool S2>
__device__ void pack_chunk_core(const Job& J, uint64_t c, PackSmem& S, uint32_t* slots,
                                const uint8_t* const* tabp) {
  constexpr int G = PTraits<DT>::G, V = PTraits<DT>::V, ES = 16 / V;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const uint64_t off0 = c * J.chunk_bytes;
  const uint64_t nb = min((uint64_t)J.chunk_bytes, J.nbytes - off0);
  const uint64_t m = nb / ES;
  const uint64_t nvec = (nb + 15) / 16;
  const uint32_t T = J.lanes;
  const uint32_t R = T <= (uint32_t)nthr ? gdiv((uint32_t)nthr, T) : 1u;  // parts per sub-stream
  const uint32_t units = T * R;                                        // <= max(nthr, T)
  // (32-bit divisions: a chunk holds fewer than 2^32 vectors)
  const uint64_t nvt = gdiv((uint32_t)nvec + T - 1, T);                // vectors of sub-stream 0
  const uint64_t per = gdiv((uint32_t)nvt + R - 1, R);                 // vectors per part
  const uint8_t* src = J.src + off0;
  const uint8_t* base = J.base ? J.base + off0 : nullptr;
  const uint64_t P = kHdrBytes + (uint64_t)J.n_chunks * G * kEntryBytes;
  uint8_t* out = J.dst;
  uint32_t huff = 0, raw = 0, sparse = 0;  // huff: every coded group (HUFF or SPARSE)
#pragma unroll
  for (int g = 0; g < G; g++) {
    if (S.meta[g].mode == kHuff || S.meta[g].mode == kSparse) huff |= 1u << g;
    if (S.meta[g].mode == kSparse) sparse |= 1u << g;
    if (S.meta[g].mode == kRaw) raw |= 1u << g;
  }
  // SPARSE groups: the vector bitmap (bit v % 32 of word v / 32) is built in
  // pass A from the vectors it loads anyway; start from zero
  const uint32_t bmw = (uint32_t)((nvec + 31) / 32);
  uint32_t* bmap[4] = {nullptr, nullptr, nullptr, nullptr};
#pragma unroll
  for (int g = 0; g < G; g++)
    if (sparse >> g & 1u) {
      bmap[g] = reinterpret_cast<uint32_t*>(out + P + S.off[g] +
                                            align_up(12 + S.meta[g].nz, 4));
      for (uint32_t w = tid; w < bmw; w += nthr) bmap[g][w] = 0;
    }
  // table bytes of the coded groups (counts per length, symbols), unless the
  // caller wrote them (null tabp)
#pragma unroll
  for (int g = 0; g < G; g++) {
    if (!(huff >> g & 1) || !tabp[g]) continue;
    uint8_t* p = out + P + S.off[g];
    const uint32_t nz = S.meta[g].nz, h = (uint32_t)align_up(12 + nz, 4);
    for (uint32_t i = tid; i < h; i += nthr) p[i] = (i < 12 + nz) ? tabp[g][i] : 0;
  }

  // The first Huffman group is encoded once, in pass A, into per-unit slots in
  // shared memory (slot_cap words each, odd so that neighbouring slots fall in
  // different banks); pass B only shifts the slot words into place.  With S2
  // (the packer of launches that hold deltas, whose chunks often code both
  // 16-bit groups) the second Huffman group is staged as well, into slots of
  // slot_cap1 words after the first group's, when the two groups' average
  // words per unit (from their payload sizes) leave at least 4 of a unit's
  // share of the slot area; the rest is split evenly between them.  Pass B
  // encodes from the input again only the groups not staged and the units
  // whose slot overflowed.
  int sg = -1, sg1 = -1;
#pragma unroll
  for (int g = 0; g < G; g++)
    if (huff >> g & 1) {
      if (sg < 0) sg = g;
      else if (S2 && sg1 < 0) sg1 = g;
    }
  uint32_t slot_cap = gdiv(kPackSlotWords, units), slot_cap1 = 0;
  if (S2 && sg1 >= 0) {
    const uint64_t uw = 32ull * units;
    const uint32_t n0 = (uint32_t)((8ull * S.meta[sg].size + uw - 1) / uw);
    const uint32_t n1 = (uint32_t)((8ull * S.meta[sg1].size + uw - 1) / uw);
    if (n0 + n1 + 4u <= slot_cap) {
      const uint32_t left = (slot_cap - n0 - n1) / 2u;
      slot_cap1 = n1 + left;
      slot_cap = n0 + left;
      if (!(slot_cap1 & 1u)) slot_cap1--;
    } else {
      sg1 = -1;  // encoded from the input in pass B, as a third group would be
    }
  }
  if (!(slot_cap & 1u)) slot_cap--;
  const uint32_t slots1 = smem_u32(slots) + 4u * units * slot_cap;  // second group's slots
  const bool fast_a = sg == 0 && huff == 1u && sparse == 0 && nb == J.chunk_bytes &&
                      gmod((uint32_t)nvec, T) == 0 && gmod((uint32_t)nvt, R) == 0 &&
                      T <= (uint32_t)nthr;
  bool pairs = false;
  if constexpr (DT == ZIPNN_BF16 || DT == ZIPNN_FP16 || DT == ZIPNN_FP32)
    pairs = fast_a && smem_u32(S.ptab) + 4096u <= 65536u && build_pair_table(S);
  __syncthreads();

  // pass A: unit bits (+ raw planes, + slot encoding of group sg)
  if (fast_a) {
    if constexpr (DT == ZIPNN_BF16 || DT == ZIPNN_FP16 || DT == ZIPNN_FP32) {
      if (pairs)
        pack_pair_a<DT>(src, base, T, R, gdiv((uint32_t)nvt, R), slots, slot_cap, S, out, P, raw);
    }
    if (!pairs)
      pack_fast_a<DT>(src, base, T, R, gdiv((uint32_t)nvt, R), slots, slot_cap, S, out, P, raw);
  }
  for (uint32_t u = fast_a ? units : tid; u < units; u += nthr) {
    const uint32_t t = gmod(u, T), k = gdiv(u, T);
    uint32_t bits[G];
#pragma unroll
    for (int g = 0; g < G; g++) bits[g] = 0;
    SlotWriter sw, sw1;
    sw.slot = smem_u32(slots) + 4u * (t * R + k) * slot_cap;
    sw1.slot = slots1 + 4u * (t * R + k) * slot_cap1;
    sw.acc = sw1.acc = 0;
    sw.nacc = sw1.nacc = 0;
    sw.wi = sw1.wi = 0;
    sw.cap = slot_cap;
    sw1.cap = slot_cap1;
    sw.bits = sw1.bits = 0;
    const uint64_t i1 = min(nvt, (uint64_t)(k + 1) * per);
    constexpr int U = 2;  // vectors in flight per thread
    for (uint64_t i0 = (uint64_t)k * per; i0 < i1; i0 += U) {
      uint4 a[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const uint64_t v = t + (i0 + u) * T;
        a[u] = (i0 + u < i1 && v < nvec) ? load_vec(src, base, v, nb) : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
      const uint64_t v = t + (i0 + u) * T;
      if (i0 + u >= i1 || v >= nvec) break;
      uint32_t g4[4][4];
      split_vec(DT, a[u], g4);
      const bool full = (v + 1) * V <= m;
      const int valid = full ? V : (int)(m - v * V);
#pragma unroll
      for (int g = 0; g < G; g++) {
        if (sparse >> g & 1u) {  // SPARSE: bitmap bit; all-zero vectors carry no codes
          uint32_t any = 0;
#pragma unroll
          for (int q = 0; q < V / 4; q++) any |= g4[g][q];
          if (T % 32 == 0) {
            // the active lanes hold consecutive vectors from a multiple of 32
            // (lane 0 first): one ballot is one bitmap word
            const uint32_t act = __activemask();
            const uint32_t word = __ballot_sync(act, any != 0);
            if ((threadIdx.x & 31) == (uint32_t)(__ffs(act) - 1)) bmap[g][v >> 5] = word;
          } else if (any) {
            atomicOr(&bmap[g][v >> 5], 1u << (v & 31));
          }
          if (!any) continue;
        }
        // this vector's symbols of group g into slot writer w
        auto stage = [&](SlotWriter& w) {
          if (full) {
#pragma unroll
            for (int q = 0; q < V / 4; q++) {
              uint32_t len;
              const uint64_t x = join4(smem_u32(S.codes[g]), g4[g][q], len);
              w.put64(x, len);
            }
          } else {
#pragma unroll
            for (int q = 0; q < V; q++)
              if (q < valid) {
                const uint32_t cl = code_of(smem_u32(S.codes[g]), g4[g][q >> 2], q & 3);
                w.put(cl & 0xFFFFu, cl >> 16);
              }
          }
        };
        if (g == sg) {
          stage(sw);
        } else if (S2 && g == sg1) {
          stage(sw1);
        } else if (huff >> g & 1) {
          if (full) {
#pragma unroll
            for (int q = 0; q < V / 4; q++) bits[g] += len4(smem_u32(S.codes[g]), g4[g][q]);
          } else {
#pragma unroll
            for (int q = 0; q < V; q++)
              if (q < valid) bits[g] += code_of(smem_u32(S.codes[g]), g4[g][q >> 2], q & 3) >> 16;
          }
        } else if (raw >> g & 1) {
          uint8_t* p = out + P + S.off[g] + v * V;
          if (full) {
            if (V == 8) *reinterpret_cast<uint2*>(p) = make_uint2(g4[g][0], g4[g][1]);
            else if (V == 4) *reinterpret_cast<uint32_t*>(p) = g4[g][0];
            else *reinterpret_cast<uint4*>(p) = make_uint4(g4[g][0], g4[g][1], g4[g][2], g4[g][3]);
          } else {
#pragma unroll
            for (int q = 0; q < V; q++)
              if (q < valid) p[q] = (uint8_t)__byte_perm(g4[g][q >> 2], 0, 0x4440 + (q & 3));
          }
        }
      }
      }
    }
    if (sg >= 0) {
      sw.finish();
#pragma unroll
      for (int g = 0; g < G; g++)
        if (g == sg) bits[g] = sw.bits;
      S.sbits[t * R + k] = sw.bits;
    }
    if (S2 && sg1 >= 0) {
      sw1.finish();
#pragma unroll
      for (int g = 0; g < G; g++)
        if (g == sg1) bits[g] = sw1.bits;
    }
#pragma unroll
    for (int g = 0; g < G; g++) S.part[g][t * R + k] = bits[g];
  }
  // raw padding
#pragma unroll
  for (int g = 0; g < G; g++) {
    if (!(raw >> g & 1)) continue;
    uint8_t* p = out + P + S.off[g];
    for (uint64_t q = m + tid; q < align_up(m, 16); q += nthr) p[q] = 0;
  }
  if (!huff) return;
  // Pass B writes each output word of the slot-staged group whole (no zeroed
  // words, no atomics) when that group is the only coded one and every unit
  // holds 32 to slot_cap * 32 bits (so a word spans at most two units)
  bool whole = sg == 0 && huff == 1u;
  // one unit per thread (unit tid): its exclusive bit offset from a warp scan
  // before this barrier and a scan of the warp totals after it
  const bool one = R == 1 && units == (uint32_t)nthr;
  const int lane = tid & 31, wid = tid >> 5;
  uint32_t ub = 0, uincl = 0;
  if (one) {
    ub = S.sbits[tid];
    whole = whole && ub >= 32u && ub <= slot_cap * 32u;
    uincl = ub;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, uincl, o);
      if (lane >= o) uincl += t;
    }
    if (lane == 31) S.wsum[wid] = uincl;
  } else {
    for (uint32_t u = tid; whole && u < units; u += nthr) {
      const uint32_t b = S.sbits[gmod(u, T) * R + gdiv(u, T)];
      whole = b >= 32u && b <= slot_cap * 32u;
    }
  }
  whole = __syncthreads_and(whole) != 0;
  if (whole && one) {
    const int nw = nthr >> 5;
    const uint32_t ws = lane < nw ? S.wsum[lane] : 0u;
    uint32_t wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    const uint32_t uoff = __shfl_sync(0xffffffffu, wi - ws, wid) + uincl - ub;
    const uint32_t tot = __shfl_sync(0xffffffffu, wi, nw - 1);
    S.part[0][tid] = uoff;
    uint8_t* p = out + P + S.off[0];
    const uint32_t h = (uint32_t)align_up(12 + S.meta[0].nz, 4);
    uint32_t* po = reinterpret_cast<uint32_t*>(p + h);
    if (tid > 0) po[tid - 1] = uoff;  // sub-stream starts (sub-stream tid = unit tid)
    uint32_t* words = po + (T - 1);
    const uint32_t capw = (uint32_t)(align_up(S.meta[0].size, 16) - h - 4ull * (T - 1)) / 4;
    __syncthreads();
    pass_b_whole(S, slots, slot_cap, units, words, capw, tot);
    return;
  }

  // scan unit bits -> unit offsets; table bytes, sub-stream starts, zeroed words
#pragma unroll
  for (int g = 0; g < G; g++) {
    if (!(huff >> g & 1)) continue;
    block_exclusive_scan(S.part[g], units, S.wsum);
    uint8_t* p = out + P + S.off[g];
    const uint32_t nz = S.meta[g].nz;
    const uint32_t h = (uint32_t)align_up(12 + nz, 4);
    const uint32_t nbm = (sparse >> g & 1u) ? bmw : 0u;  // bitmap words (written in pass A)
    uint32_t* po = reinterpret_cast<uint32_t*>(p + h + 4 * nbm);
    for (uint32_t t = 1 + tid; t < T; t += nthr) po[t - 1] = S.part[g][t * R];
    uint32_t* words = po + (T - 1);
    const uint32_t capw =
        (uint32_t)(align_up(S.meta[g].size, 16) - h - 4ull * nbm - 4ull * (T - 1)) / 4;
    if (!whole)
      for (uint32_t w = tid; w < capw; w += nthr) words[w] = 0;
    if (tid == 0) {
      S.capw[g] = capw;
      S.hsz[g] = h + 4 * nbm + 4 * (T - 1);
    }
  }
  __syncthreads();

  if (whole) {
    pass_b_whole(S, slots, slot_cap, units,
                 reinterpret_cast<uint32_t*>(out + P + S.off[0] + S.hsz[0]), S.capw[0],
                 S.part[0][units - 1] + S.sbits[units - 1]);
    return;
  }

  // pass B
  for (uint32_t u = tid; u < units; u += nthr) {
    const uint32_t t = gmod(u, T), k = gdiv(u, T);
    const uint32_t ui = t * R + k;
    // (1) slot-staged groups: shift the unit's slot words to its bit offset
    // (its bits: the staged count, or the next unit's offset minus its own)
    bool refill = false, refill1 = false;
#pragma unroll
    for (int s1 = 0; s1 < (S2 ? 2 : 1); s1++) {
      const int gs = s1 ? sg1 : sg;
      if (gs < 0) continue;
      const uint32_t o = S.part[gs][ui];
      const uint32_t nbits = s1 ? S.part[gs][ui + 1] - o : S.sbits[ui];
      const uint32_t cap = s1 ? slot_cap1 : slot_cap;
      if (nbits > cap * 32u) {
        (s1 ? refill1 : refill) = true;  // slot overflowed: re-encode below from the input
      } else if (nbits) {
        uint32_t* words = reinterpret_cast<uint32_t*>(out + P + S.off[gs] + S.hsz[gs]);
        const uint32_t sl = (s1 ? slots1 : smem_u32(slots)) + 4u * ui * cap;
        const uint32_t sh = o & 31, w0 = o >> 5;
        const uint32_t end = o + nbits, wl = (end - 1) >> 5;
        const uint32_t nsw = (nbits + 31) >> 5;
        uint32_t prev = 0;
        for (uint32_t w = w0; w <= wl; w++) {
          const uint32_t i = w - w0;
          const uint32_t cur = i < nsw ? lds32v(sl + 4u * i) : 0u;
          const uint32_t word = __funnelshift_r(cur, prev, sh);
          prev = cur;
          if (w >= S.capw[gs]) break;  // never taken for a consistent input
          if ((w == w0 && sh) || (w == wl && (end & 31))) atomicOr(&words[w], word);
          else words[w] = word;
        }
      }
    }
    // (2) other Huffman groups (and overflowed units): encode from the input
    bool any = refill || refill1;
#pragma unroll
    for (int g = 0; g < G; g++)
      if ((huff >> g & 1) && g != sg && g != sg1) any = true;
    if (!any) continue;
    BitWriter bw[G];
    bool emit[G];
#pragma unroll
    for (int g = 0; g < G; g++) {
      emit[g] = (huff >> g & 1) &&
                ((g != sg && g != sg1) || (g == sg && refill) || (g == sg1 && refill1));
      bw[g].words = reinterpret_cast<uint32_t*>(out + P + S.off[g] + S.hsz[g]);
      const uint32_t st = emit[g] ? S.part[g][ui] : 0u;
      bw[g].acc = 0;
      bw[g].nacc = st & 31;
      bw[g].wi = st >> 5;
      bw[g].first = (st & 31) != 0;
      bw[g].capw = S.capw[g];
    }
    const uint64_t i1 = min(nvt, (uint64_t)(k + 1) * per);
    for (uint64_t i = (uint64_t)k * per; i < i1; i++) {
      const uint64_t v = t + i * T;
      if (v >= nvec) break;
      uint32_t g4[4][4];
      split_vec(DT, load_vec(src, base, v, nb), g4);
      const bool full = (v + 1) * V <= m;
#pragma unroll
      for (int g = 0; g < G; g++) {
        if (!emit[g]) continue;
        if (sparse >> g & 1u) {  // SPARSE: all-zero vectors carry no codes
          uint32_t any = 0;
#pragma unroll
          for (int q = 0; q < V / 4; q++) any |= g4[g][q];
          if (!any) continue;
        }
        if (full) {
#pragma unroll
          for (int q = 0; q < V / 4; q++) {
            uint32_t len;
            const uint64_t x = join4(smem_u32(S.codes[g]), g4[g][q], len);
            bw[g].put64(x, len);
          }
        } else {
          const int valid = (int)(m - v * V);
#pragma unroll
          for (int q = 0; q < V; q++)
            if (q < valid) {
              const uint32_t cl = code_of(smem_u32(S.codes[g]), g4[g][q >> 2], q & 3);
              bw[g].put(cl & 0xFFFFu, cl >> 16);
            }
        }
      }
    }
#pragma unroll
    for (int g = 0; g < G; g++)
      if (emit[g]) bw[g].flush();
  }
}

// The 64-byte container header of job J (one thread).
__device__ void write_header(const Job& J, uint64_t total) {
  uint8_t* h = J.dst;
  const int G = elem_size(J.dtype);
  const uint64_t P = kHdrBytes + (uint64_t)J.n_chunks * G * kEntryBytes;
  h[0] = 'Z'; h[1] = 'N'; h[2] = 'N'; h[3] = '1';
  h[4] = 1; h[5] = 0;
  h[6] = (uint8_t)J.dtype;
  h[7] = (uint8_t)J.flags;
  put_u64(h + 8, J.nbytes);
  put_u32(h + 16, J.chunk_bytes);
  put_u32(h + 20, J.lanes);
  put_u32(h + 24, (uint32_t)G);
  put_u32(h + 28, J.n_chunks);
  put_u64(h + 32, P);
  put_u64(h + 40, total);
  for (int k = 48; k < 64; k++) h[k] = 0;
}

template <int DTS, bool S2>
__global__ void __launch_bounds__(kPackThreads, 2)
k_pack(JobRef jr, uint64_t nchunks_total, const uint32_t* __restrict__ codes,
       const uint8_t* __restrict__ tabs, const GcMeta* __restrict__ meta,
       const uint64_t* __restrict__ offs, const uint64_t* __restrict__ totals) {
  __shared__ PackSmem S;
  extern __shared__ uint32_t slots[];  // kPackSlotWords
  const int tid = threadIdx.x;
  if (blockIdx.x >= nchunks_total) {  // header CTAs
    const int j = (int)(blockIdx.x - nchunks_total);
    const Job& J = job_at(jr, j);
    if (totals[j] > J.out_capacity) return;
    if (tid == 0) write_header(J, totals[j]);
    return;
  }
  const uint64_t chunk = blockIdx.x;
  __shared__ int job;  // found by thread 0, read by all after the barrier
  if (tid == 0) job = find_job_chunk(jr, chunk);
  __syncthreads();
  const int j = job;
  const Job& J = job_at(jr, j);
  if (totals[j] > J.out_capacity) return;
  const uint64_t c = chunk - J.chunk_begin;
  if (DTS >= 0) {
    pack_chunk<(DTS < 0 ? 0 : DTS), S2>(J, c, S, slots, codes, tabs, meta, offs);
    return;
  }
  switch (J.dtype) {
    case ZIPNN_BF16: pack_chunk<ZIPNN_BF16, S2>(J, c, S, slots, codes, tabs, meta, offs); break;
    case ZIPNN_FP16: pack_chunk<ZIPNN_FP16, S2>(J, c, S, slots, codes, tabs, meta, offs); break;
    case ZIPNN_FP32: pack_chunk<ZIPNN_FP32, S2>(J, c, S, slots, codes, tabs, meta, offs); break;
    default: pack_chunk<ZIPNN_U8, S2>(J, c, S, slots, codes, tabs, meta, offs); break;
  }
}


// ---------------------------------------------------------------------------
// k_compress: the whole encoder in one persistent kernel, for launches of one
// dtype with at most two byte groups (BF16, FP16, U8).  Each CTA pulls chunks
// from a device ticket and, per chunk:
//   1. builds the histograms (the chunk's one read from DRAM);
//   2. builds each group's code (warp g: group g) in shared memory;
//   3. learns where its payloads go: the offset of a chunk within its
//      container is the sum of the padded payload sizes of the chunks before
//      it (the map of Sec. 5.1), found by a decoupled look-back over the
//      chunks of its tensor (Merrill & Garland, "Single-pass Parallel Prefix
//      Scan with Decoupled Look-back", 2016): the chunk publishes its own size
//      at once, then adds up its predecessors' published sizes until one
//      that has published its inclusive prefix;
//   4. packs, reading the chunk again while it is still in L2 (two 512-thread
//      CTAs per SM hold about 80 MB of chunks in flight).
// The last chunk of a tensor writes its header and size.  Chunks are taken in
// ticket order by running CTAs, so every chunk a look-back waits for belongs
// to a CTA that is running or finished and publishes its size right after its
// own code build: the wait always ends.  It is bounded all the same (%globaltimer,
// 2 s): past the limit the chunk is not written and the call reports
// ZIPNN_ETIMEOUT.  Work items past the chunks write the headers of empty tensors.

constexpr uint64_t kLbAgg = 1ull << 62;    // look-back word: own padded size only
constexpr uint64_t kLbIncl = 2ull << 62;   // look-back word: inclusive prefix
constexpr uint64_t kLbValue = (1ull << 62) - 1;
constexpr uint64_t kLbLimitNs = 2000000000ull;

__device__ __forceinline__ uint64_t enc_globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const unsigned long long* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive prefix, within its tensor, of the chunk with global index `gchunk`
// (index c within its tensor) whose payloads take `own` padded bytes.
// *timed_out is set if a predecessor's word did not appear within the limit.
// (Fault injection for tests, `hide`: the chunk publishes nothing, so the
// look-backs that need it run out their limit.)
__device__ uint64_t lookback(unsigned long long* lb, uint64_t gchunk, uint64_t c, uint64_t own,
                             uint64_t limit_ns, bool hide, bool* timed_out) {
  if (c == 0) {
    if (!hide) st_relaxed_u64(lb + gchunk, kLbIncl | own);
    return 0;
  }
  st_relaxed_u64(lb + gchunk, kLbAgg | own);
  const uint64_t first = gchunk - c;  // the tensor's first chunk publishes an inclusive prefix
  uint64_t prefix = 0, k = gchunk - 1;
  const uint64_t t0 = enc_globaltimer();
  for (;;) {
    const uint64_t v = ld_relaxed_u64(lb + k);
    if (!(v >> 62)) {
      if (enc_globaltimer() - t0 > limit_ns) {
        *timed_out = true;
        break;
      }
      __nanosleep(64);
      continue;
    }
    prefix += v & kLbValue;
    if ((v >> 62) == 2u) break;
    if (k == first) {  // cannot happen: the first chunk's word is always inclusive
      *timed_out = true;
      break;
    }
    k--;
  }
  st_relaxed_u64(lb + gchunk, kLbIncl | (prefix + own));
  return prefix;
}

struct FusedSmem {
  uint32_t hist[2][256];       // bin totals of the chunk
  uint32_t zs[2];              // symbols inside all-zero vectors
  uint8_t tab[2][kTabBytes];   // table bytes of the coded groups
  uint64_t chunk;              // the CTA's current work item
  int job;                     // its job
  uint32_t skip;               // 1: do not write the chunk (timed out / no room)
};

constexpr size_t kFusedDynBytes =
    (size_t)kPackSlotWords * 4 > (size_t)(2 * 256 * 32 + 2) * 4
        ? (size_t)kPackSlotWords * 4
        : (size_t)(2 * 256 * 32 + 2) * 4;
static_assert(2 * sizeof(BuildSmem) <= kFusedDynBytes, "build scratch must fit");

template <int DT>
__global__ void __launch_bounds__(kPackThreads, 2)
k_compress(JobRef jr, uint64_t nchunks_total, unsigned long long* lb,
           uint64_t* __restrict__ totals, uint32_t* __restrict__ err, uint32_t debug_flags) {
  constexpr int G = PTraits<DT>::G, ES = 16 / PTraits<DT>::V;
  static_assert(G <= 2, "the fused encoder handles at most two byte groups");
  // counters of the histograms, then the code builders' scratch, then the
  // packer's unit slots
  extern __shared__ __align__(16) uint32_t dyn[];
  __shared__ PackSmem S;
  __shared__ FusedSmem F;
  const int tid = threadIdx.x, wid = tid >> 5;
  unsigned long long* ticket = lb + nchunks_total;
  const uint64_t nitems = nchunks_total + (uint64_t)jr.n;
  if (tid == 0) F.job = 0;
  __syncthreads();
  for (;;) {
    // work item and its job (thread 0; items come in increasing order, so the
    // job is found scanning forward from the previous one)
    if (tid == 0) {
      const uint64_t it = atomicAdd(ticket, 1ull);
      int jj = 0;
      if (it >= nchunks_total) {
        jj = it < nitems ? (int)(it - nchunks_total) : 0;
      } else if (jr.table) {
        jj = F.job;
        int steps = 0;
        while (jj + 1 < jr.n && jr.table[jj + 1].chunk_begin <= it && steps < 8) {
          jj++;
          steps++;
        }
        if (steps == 8) jj += find_job(jr.table + jj, jr.n - jj, it);
      }
      F.chunk = it;
      F.job = jj;
    }
    __syncthreads();
    const uint64_t item = F.chunk;
    if (item >= nitems) break;
    const int j = F.job;
    const Job& J = job_at(jr, j);
    if (item >= nchunks_total) {
      // header of an empty tensor (its only content)
      if (tid == 0 && J.n_chunks == 0) {
        const uint64_t total = kHdrBytes;
        totals[j] = total;
        if (J.out_nbytes) *J.out_nbytes = total;
        if (total <= J.out_capacity) write_header(J, total);
        else atomicOr(err, 2u);
      }
      __syncthreads();
      continue;
    }
    const uint64_t c = item - J.chunk_begin;
    const uint64_t nb = min((uint64_t)J.chunk_bytes, J.nbytes - c * J.chunk_bytes);
    // 1. histograms (ends past a barrier)
    hist_chunk<DT, kPackThreads>(J, c, dyn, &F.hist[0][0], F.zs);
    // 2. codes: warp g builds group g's
    if (wid < G)
      build_gc(F.hist[wid], F.zs[wid], (uint32_t)(nb / ES), J.lanes, ES,
               reinterpret_cast<BuildSmem*>(dyn)[wid], S.codes[wid], F.tab[wid], &S.meta[wid]);
    __syncthreads();
    // 3. payload offsets (thread 0), header and size after the last chunk
    if (tid == 0) {
      uint64_t own = 0;
#pragma unroll
      for (int g = 0; g < G; g++) own += align_up(S.meta[g].size, 16);
      bool timed_out = false;
      // debug flag 1 (tests only): the first chunk of the launch hides its
      // offset and the limit is 100 ms -> ETIMEOUT
      const bool inject = (debug_flags & 1u) != 0;
      const uint64_t prefix = lookback(lb, item, c, own, inject ? 100000000ull : kLbLimitNs,
                                       inject && item == 0, &timed_out);
      uint64_t run = prefix;
#pragma unroll
      for (int g = 0; g < G; g++) {
        S.off[g] = run;
        run += align_up(S.meta[g].size, 16);
      }
      const uint64_t P = kHdrBytes + (uint64_t)J.n_chunks * G * kEntryBytes;
      F.skip = (timed_out || P + run > J.out_capacity) ? 1u : 0u;
      if (timed_out) atomicOr(err, 4u);
      if (c + 1 == J.n_chunks) {
        const uint64_t total = P + run;
        totals[j] = total;
        if (J.out_nbytes) *J.out_nbytes = total;
        if (total > J.out_capacity) atomicOr(err, 2u);
        else if (!timed_out) write_header(J, total);
      }
    }
    __syncthreads();
    // 4. map entries and packing (the chunk is read again, from L2)
    if (!F.skip) {
      write_map_entries<G>(J, c, S);
      const uint8_t* tabp[4] = {F.tab[0], G > 1 ? F.tab[1] : nullptr, nullptr, nullptr};
      pack_chunk_core<DT>(J, c, S, dyn, tabp);
    }
    __syncthreads();
  }
}

}  // namespace

size_t encode_scratch_bytes(uint64_t nchunks_total, uint64_t ngc_total, int njobs) {
  (void)nchunks_total;
  size_t b = 0;
  b += align_up(ngc_total * 256 * 4, 256);          // hist
  b += align_up(ngc_total * 256 * 4, 256);          // codes
  b += align_up(ngc_total * kTabBytes, 256);        // tabs
  b += align_up(ngc_total * sizeof(GcMeta), 256);   // meta
  b += align_up(ngc_total * 8, 256);                // offs
  b += align_up((uint64_t)njobs * 8, 256);          // totals
  b += align_up(ngc_total * 4, 256);                // zsyms
  return b + 256;
}

void encode_scratch_carve(void* base, uint64_t nchunks_total, uint64_t ngc_total, int njobs,
                          EncodeScratch* s) {
  (void)nchunks_total;
  uint8_t* p = reinterpret_cast<uint8_t*>(align_up(reinterpret_cast<uintptr_t>(base), 256));
  s->hist = reinterpret_cast<uint32_t*>(p); p += align_up(ngc_total * 256 * 4, 256);
  s->codes = reinterpret_cast<uint32_t*>(p); p += align_up(ngc_total * 256 * 4, 256);
  s->tabs = p; p += align_up(ngc_total * kTabBytes, 256);
  s->meta = reinterpret_cast<GcMeta*>(p); p += align_up(ngc_total * sizeof(GcMeta), 256);
  s->offs = reinterpret_cast<uint64_t*>(p); p += align_up(ngc_total * 8, 256);
  s->totals = reinterpret_cast<uint64_t*>(p); p += align_up((uint64_t)njobs * 8, 256);
  s->zsyms = reinterpret_cast<uint32_t*>(p);
}

static JobRef make_ref(const Job* d_jobs, int njobs, const Job* h_one) {
  JobRef r;
  r.table = h_one ? nullptr : d_jobs;
  if (h_one) r.one = *h_one;
  else memset(&r.one, 0, sizeof(Job));
  r.n = njobs;
  return r;
}

// Launch k_hist, k_build and k_scan.  d_jobs is a device table of njobs jobs,
// unless njobs == 1 and h_one is given (then the job is passed by value).
template <class K>
static K pick(int dt, K k0, K k1, K k2, K k3, K kmix) {
  switch (dt) {
    case ZIPNN_BF16: return k0;
    case ZIPNN_FP16: return k1;
    case ZIPNN_FP32: return k2;
    case ZIPNN_U8: return k3;
    default: return kmix;
  }
}

cudaError_t launch_encode_analyse_ex(const Job* d_jobs, const Job* h_one, int njobs,
                                     uint64_t nchunks_total, uint64_t ngc_total,
                                     const EncodeScratch& s, uint32_t* d_err, cudaStream_t st,
                                     int max_groups, int uniform_dtype) {
  JobRef r = make_ref(d_jobs, njobs, h_one);
  if (h_one) {
    max_groups = elem_size(h_one->dtype);
    uniform_dtype = h_one->dtype;
  }
  if (nchunks_total) {
    const int hs = hist_smem_bytes(max_groups < 1 ? 4 : (max_groups > 4 ? 4 : max_groups));
    auto kh = pick(uniform_dtype, k_hist<ZIPNN_BF16>, k_hist<ZIPNN_FP16>, k_hist<ZIPNN_FP32>,
                   k_hist<ZIPNN_U8>, k_hist<-1>);
    cudaError_t ea = cudaFuncSetAttribute(kh, cudaFuncAttributeMaxDynamicSharedMemorySize, hs);
    if (ea == cudaSuccess)
      ea = cudaFuncSetAttribute(kh, cudaFuncAttributePreferredSharedMemoryCarveout,
                                cudaSharedmemCarveoutMaxShared);
    if (ea != cudaSuccess) return ea;
    kh<<<(unsigned)nchunks_total, kHistThreads, hs, st>>>(r, s.hist, s.zsyms);
    unsigned nb = (unsigned)((ngc_total + kBuildWarps - 1) / kBuildWarps);
    k_build<<<nb, kBuildWarps * 32, 0, st>>>(r, ngc_total, s.hist, s.zsyms, s.codes, s.tabs,
                                             s.meta);
  }
  k_scan<<<njobs, kScanThreads, 0, st>>>(r, s.meta, s.offs, s.totals, d_err);
  return cudaGetLastError();
}

cudaError_t launch_encode_pack_ex(const Job* d_jobs, const Job* h_one, int njobs,
                                  uint64_t nchunks_total, int max_lanes, const EncodeScratch& s,
                                  cudaStream_t st, int uniform_dtype, bool any_delta) {
  JobRef r = make_ref(d_jobs, njobs, h_one);
  (void)max_lanes;
  if (h_one) {
    uniform_dtype = h_one->dtype;
    any_delta = h_one->base != nullptr;
  }
  // launches that hold deltas stage two coded groups in pass A (S2)
  auto kp = any_delta ? pick(uniform_dtype, k_pack<ZIPNN_BF16, true>, k_pack<ZIPNN_FP16, true>,
                             k_pack<ZIPNN_FP32, true>, k_pack<ZIPNN_U8, true>, k_pack<-1, true>)
                      : pick(uniform_dtype, k_pack<ZIPNN_BF16, false>, k_pack<ZIPNN_FP16, false>,
                             k_pack<ZIPNN_FP32, false>, k_pack<ZIPNN_U8, false>,
                             k_pack<-1, false>);
  const int ps = (int)(kPackSlotWords * 4);
  cudaError_t ea = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, ps);
  if (ea == cudaSuccess)
    ea = cudaFuncSetAttribute(kp, cudaFuncAttributePreferredSharedMemoryCarveout,
                              cudaSharedmemCarveoutMaxShared);
  if (ea != cudaSuccess) return ea;
  kp<<<(unsigned)(nchunks_total + njobs), kPackThreads, ps, st>>>(r, nchunks_total, s.codes, s.tabs,
                                                                s.meta, s.offs, s.totals);
  return cudaGetLastError();
}

bool fused_encoder_applies(int dtype, bool any_skip) {
  return !any_skip && (dtype == ZIPNN_BF16 || dtype == ZIPNN_FP16 || dtype == ZIPNN_U8);
}

// The single-pass encoder (k_compress) for jobs of one dtype with at most two
// groups and no skip-ahead probe.  Its look-back words (one per chunk) and
// work ticket live in the histogram area of the scratch, which this kernel
// does not otherwise use (it keeps its histograms in shared memory), and are
// cleared here, on the stream, before the launch.
cudaError_t launch_encode_fused(const Job* d_jobs, const Job* h_one, int njobs,
                                uint64_t nchunks_total, const EncodeScratch& s, uint32_t* d_err,
                                cudaStream_t st, int dtype, uint32_t debug_flags) {
  JobRef r = make_ref(d_jobs, njobs, h_one);
  unsigned long long* lb = reinterpret_cast<unsigned long long*>(s.hist);
  cudaError_t e =
      cudaMemsetAsync(lb, 0, (size_t)(nchunks_total + 2) * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const void* kern = dtype == ZIPNN_BF16   ? reinterpret_cast<const void*>(k_compress<ZIPNN_BF16>)
                     : dtype == ZIPNN_FP16 ? reinterpret_cast<const void*>(k_compress<ZIPNN_FP16>)
                                           : reinterpret_cast<const void*>(k_compress<ZIPNN_U8>);
  const int dynb = (int)kFusedDynBytes;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dynb);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kPackThreads, dynb);
  if (occ < 1) occ = 1;
  const uint64_t items = nchunks_total + (uint64_t)njobs;
  uint64_t grid = (uint64_t)sms * (uint64_t)occ;
  if (grid > items) grid = items;
  if (grid < 1) grid = 1;
  uint64_t* totals = s.totals;
  void* args[] = {&r, &nchunks_total, &lb, &totals, &d_err, &debug_flags};
  return cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(kPackThreads), args, (size_t)dynb, st);
}

cudaError_t launch_encode(const Job* d_jobs, const Job* h_one, int njobs, uint64_t nchunks_total,
                          uint64_t ngc_total, const EncodeScratch& s, uint32_t* d_err,
                          cudaStream_t st, int max_groups, int max_lanes, int uniform_dtype,
                          bool any_skip, int encoder, uint32_t debug_flags, bool any_delta) {
  const int dt = h_one ? h_one->dtype : uniform_dtype;
  const bool skip = h_one ? h_one->skip != 0 : any_skip;
  // (a launch of empty tensors only has no chunk, hence no histogram area to
  // hold the single-pass kernel's ticket: the four-kernel path writes its headers)
  if (encoder == 1 && nchunks_total > 0 && fused_encoder_applies(dt, skip))
    return launch_encode_fused(d_jobs, h_one, njobs, nchunks_total, s, d_err, st, dt,
                               debug_flags);
  cudaError_t e = launch_encode_analyse_ex(d_jobs, h_one, njobs, nchunks_total, ngc_total, s,
                                           d_err, st, max_groups, uniform_dtype);
  if (e == cudaSuccess)
    e = launch_encode_pack_ex(d_jobs, h_one, njobs, nchunks_total, max_lanes, s, st,
                              uniform_dtype, any_delta);
  return e;
}

}  // namespace zipnn
