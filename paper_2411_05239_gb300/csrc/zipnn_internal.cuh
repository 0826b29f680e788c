// Internal definitions of the GB300 ZipNN codec: container layout constants,
// the per-tensor job descriptor shared by the batched kernels, and small device
// helpers.  The container layout (ZipNN Sec. 5.1 "Metadata and parallelism"):
//   header 64 B | map: one 16-B entry per (chunk, group) | payloads, each
//   padded to 16 B, in (chunk, group) order.
// Map entry: u64 payload offset (relative to the payload area), u32 payload
// bytes, u8 mode, u8 value, u16 zero.
// HUFF payload: u8 count of codes per length 1..12, the symbols ordered by
// (length, symbol), zero pad to 4 B, u32 start bit of sub-streams 1..T-1, then
// the bitstream as u32 words whose most significant bit comes first.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "zipnn.h"

namespace zipnn {

constexpr int kMaxLen = 12;           // code length limit
constexpr int kLutSize = 1 << kMaxLen;
constexpr int kHdrBytes = 64;
constexpr int kEntryBytes = 16;
constexpr int kTabBytes = 272;        // 12 counts + up to 256 symbols, padded

enum Mode : uint32_t { kRaw = 0, kHuff = 1, kZero = 2, kConst = 3, kSparse = 4 };

__host__ __device__ inline int elem_size(int dtype) {
  return dtype == ZIPNN_FP32 ? 4 : (dtype == ZIPNN_U8 ? 1 : 2);
}
__host__ __device__ inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// Decoder stage sizing: the Huffman payload bytes of one chunk to provision
// for, in 64ths of the chunk.  Model weights: a BF16 exponent group codes to
// about a third of its half of the chunk (11/64 with margin), an FP16 one (5
// exponent + 3 fraction bits) to about 70% (24/64), an FP32 one to about a
// third of its quarter (8/64); U8 streams are unknown (32/64); a BF16 / FP32
// delta codes two groups, and the stage also holds the second group's table
// (20/64).  Chunks whose payloads exceed the stage are decoded from global
// memory instead.
inline int stage_frac64(int dtype, uint32_t flags) {
  const bool delta = (flags & 1u) != 0;
  switch (dtype) {
    case 0: return delta ? 20 : 11;
    case 1: return 24;
    case 2: return delta ? 20 : 8;
    default: return 32;
  }
}

// One tensor of a (possibly batched) call.
struct Job {
  const uint8_t* src;     // compress: input tensor; decompress: container
  const uint8_t* base;    // delta base or nullptr
  uint8_t* dst;           // compress: container; decompress: output tensor
  uint64_t nbytes;        // original bytes
  uint64_t chunk_begin;   // first global chunk index of this tensor in the batch
  uint64_t gc_begin;      // first global group-chunk index (scratch rows)
  uint64_t out_capacity;  // compress: bytes available at dst
  uint64_t* out_nbytes;   // compress: where to store the container size (may be null)
  uint64_t stream_bytes;  // decompress: container size
  uint32_t chunk_bytes;
  uint32_t lanes;
  uint32_t n_chunks;
  int32_t dtype;
  uint32_t flags;
  uint32_t skip;          // compress: skip-ahead probe window (0 = exact decisions)
  uint32_t chunk0;        // decompress: first chunk of the tensor this job decodes (a
                          // range job of a sharded decode; 0 otherwise).  Work item k of
                          // the job decodes chunk chunk0 + k; dst and base are then
                          // shifted on the host so that dst + chunk * chunk_bytes lands
                          // in the caller's buffer of the range
};

// Per group-chunk result of the code builder.
struct GcMeta {
  uint32_t size;    // payload bytes (unpadded)
  uint32_t mode;
  uint32_t value;
  uint32_t nz;
};

// Map a global chunk index to its job by binary search over chunk_begin.
__device__ inline int find_job(const Job* jobs, int njobs, uint64_t chunk) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].chunk_begin <= chunk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Split 16 bytes (one vector) into the group bytes of its elements.
// 16-bit types: 8 elements -> g0[8], g1[8] packed as 2x u32 each.
// FP32: 4 elements -> g0..g3, 4 bytes each (one u32 per group).
// U8: 16 bytes -> g0 as 4 x u32.
// Element x (u16): g0 = (x >> 7) & 0xFF, g1 = (x >> 8 & 0x80) | (x & 0x7F).
__device__ __forceinline__ void split16(uint32_t w0, uint32_t w1, uint32_t& e, uint32_t& r) {
  // w0 = elements 0,1 (lo, hi halves), w1 = elements 2,3
  // lo byte of element k: L_k, hi byte: H_k.  Gather L into one word, H into another.
  uint32_t lo = __byte_perm(w0, w1, 0x6420);   // L0 L1 L2 L3
  uint32_t hi = __byte_perm(w0, w1, 0x7531);   // H0 H1 H2 H3
  // g0 = (H << 1 | L >> 7) per byte; g1 = (H & 0x80) | (L & 0x7F)
  e = ((hi << 1) & 0xFEFEFEFEu) | ((lo >> 7) & 0x01010101u);
  r = (hi & 0x80808080u) | (lo & 0x7F7F7F7Fu);
}

// Inverse of split16 for 4 elements: bytes e (g0) and r (g1) -> two u32 words.
__device__ __forceinline__ void merge16(uint32_t e, uint32_t r, uint32_t& w0, uint32_t& w1) {
  uint32_t hi = (r & 0x80808080u) | ((e >> 1) & 0x7F7F7F7Fu);
  uint32_t lo = ((e << 7) & 0x80808080u) | (r & 0x7F7F7F7Fu);
  w0 = __byte_perm(lo, hi, 0x5140);  // L0 H0 L1 H1
  w1 = __byte_perm(lo, hi, 0x7362);  // L2 H2 L3 H3
}

// FP32 element x: g0 = x >> 23 & 0xFF, g1 = (x >> 24 & 0x80) | (x >> 16 & 0x7F),
// g2 = x >> 8 & 0xFF, g3 = x & 0xFF.  Four elements -> one u32 per group.
__device__ __forceinline__ void split32(const uint32_t x[4], uint32_t g[4]) {
  // 4x4 byte transpose: bK = byte K of elements 0..3
  uint32_t lo01 = __byte_perm(x[0], x[1], 0x5140), hi01 = __byte_perm(x[0], x[1], 0x7362);
  uint32_t lo23 = __byte_perm(x[2], x[3], 0x5140), hi23 = __byte_perm(x[2], x[3], 0x7362);
  uint32_t b0 = __byte_perm(lo01, lo23, 0x5410), b1 = __byte_perm(lo01, lo23, 0x7632);
  uint32_t b2 = __byte_perm(hi01, hi23, 0x5410), b3 = __byte_perm(hi01, hi23, 0x7632);
  g[0] = ((b3 << 1) & 0xFEFEFEFEu) | ((b2 >> 7) & 0x01010101u);
  g[1] = (b3 & 0x80808080u) | (b2 & 0x7F7F7F7Fu);
  g[2] = b1;
  g[3] = b0;
}

__device__ __forceinline__ void merge32(const uint32_t g[4], uint32_t x[4]) {
  uint32_t b3 = (g[1] & 0x80808080u) | ((g[0] >> 1) & 0x7F7F7F7Fu);
  uint32_t b2 = ((g[0] << 7) & 0x80808080u) | (g[1] & 0x7F7F7F7Fu);
  uint32_t b1 = g[2], b0 = g[3];
  // element k bytes (b0_k, b1_k, b2_k, b3_k) little-endian
  uint32_t lo01 = __byte_perm(b0, b1, 0x5140);  // b0_0 b1_0 b0_1 b1_1
  uint32_t hi01 = __byte_perm(b2, b3, 0x5140);  // b2_0 b3_0 b2_1 b3_1
  uint32_t lo23 = __byte_perm(b0, b1, 0x7362);
  uint32_t hi23 = __byte_perm(b2, b3, 0x7362);
  x[0] = __byte_perm(lo01, hi01, 0x5410);
  x[1] = __byte_perm(lo01, hi01, 0x7632);
  x[2] = __byte_perm(lo23, hi23, 0x5410);
  x[3] = __byte_perm(lo23, hi23, 0x7632);
}

}  // namespace zipnn
