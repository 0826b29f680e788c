// Decoder kernel of the GB300 ZipNN codec: table-driven Huffman decoding of
// every byte-group stream of a chunk and the merge back to the original dtype
// (ZipNN Sec. 3.1, 3.2 inverse; Sec. 4.2 XOR with the base; Sec. 5.1 map).
//
// Work unit = one chunk.  A persistent grid pulls chunks of all tensors of a
// batch from a device ticket (atomicAdd), so one launch decodes many tensors of
// uneven sizes.  Per chunk the CTA
//   1. loads and validates the chunk's map entries and Huffman tables with
//      16-byte / 4-byte cooperative loads into shared memory,
//   2. builds, per Huffman group, a 2^W-entry table (W = 10): the entry for a
//      W-bit window holds up to three whole codes that fit in it (symbols and
//      bits consumed); a window whose first code is longer than W bits points
//      to a slow path that resolves it with the canonical limits (< 0.3% of
//      exponent symbols),
//   3. decodes: thread t owns interleaved sub-stream t, i.e. the vectors
//      v = t, t+T, ... of the chunk, so each warp step touches 32 consecutive
//      16-byte vectors: raw-group loads (prefetched one vector ahead) and the
//      16-B output stores are fully coalesced; the inverse permutation and the
//      XOR with a delta base happen in registers.
// The decoder is total: symbol counts are fixed by the map, bit reads past a
// payload return zero bits, invalid codes and bad map entries set the error
// word, and every loop is bounded.
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "zipnn_internal.cuh"

namespace zipnn {

namespace {

constexpr int kDecThreads = 128;
constexpr int kW = 10;                 // primary table bits
constexpr int kLut = 1 << kW;
constexpr uint32_t kSlow = 0u;         // entry with n == 0: resolve on the slow path

template <int DT> struct Traits;
template <> struct Traits<ZIPNN_BF16> { static constexpr int G = 2, V = 8; };
template <> struct Traits<ZIPNN_FP16> { static constexpr int G = 2, V = 8; };
template <> struct Traits<ZIPNN_FP32> { static constexpr int G = 4, V = 4; };
template <> struct Traits<ZIPNN_U8> { static constexpr int G = 1, V = 16; };

struct JobRef {
  const Job* table;
  Job one;
  int n;
};

// Per-group canonical tables (shared memory).
struct GroupTab {
  uint32_t lim[kMaxLen + 2];    // left-justified (12-bit) end of the codes of length l
  uint32_t first[kMaxLen + 2];  // first code of length l
  uint32_t index[kMaxLen + 2];  // rank of that code in the symbol list
  uint32_t words[68];           // raw table bytes (counts + symbols), 272 B
};

struct ChunkInfo {
  uint32_t mode[4];
  uint32_t value[4];
  uint32_t size[4];
  uint32_t nwords[4];       // bitstream words (HUFF)
  uint64_t payload[4];      // byte offset of the payload within the container
  uint64_t bs[4];           // byte offset of the bitstream (HUFF)
  uint64_t offs[4];         // byte offset of the start-bit table (HUFF)
  uint32_t bad;
};

struct Smem {
  ChunkInfo ci;
  GroupTab tab[4];
  unsigned long long chunk;
};

__device__ __forceinline__ uint8_t tab_byte(const GroupTab& t, int i) {
  return (uint8_t)(t.words[i >> 2] >> (8 * (i & 3)));
}

__device__ __forceinline__ uint32_t ld_word(const uint32_t* w, uint32_t i, uint32_t n) {
  return i < n ? __ldg(w + i) : 0u;
}

// MSB-first reader over one sub-stream: w0:w1 hold the current 64 bits, w2
// the next word, loaded one word ahead so its latency overlaps decoding.
struct BitReader {
  const uint32_t* w;
  uint32_t n, idx, w0, w1, w2, pos;
  __device__ __forceinline__ void init(const uint32_t* words, uint32_t nwords, uint32_t start) {
    w = words;
    n = nwords;
    idx = start >> 5;
    pos = start & 31;
    w0 = ld_word(w, idx, n);
    w1 = ld_word(w, idx + 1, n);
    w2 = ld_word(w, idx + 2, n);
    idx += 3;
  }
  __device__ __forceinline__ uint32_t peek32() const { return __funnelshift_l(w1, w0, pos); }
  __device__ __forceinline__ void skip(uint32_t bits) {
    pos += bits;
    if (pos >= 32) {
      pos -= 32;
      w0 = w1;
      w1 = w2;
      w2 = ld_word(w, idx, n);
      idx++;
    }
  }
};

// Slow path: the first code of the 12-bit window is longer than kW bits.
// Returns a one-symbol entry (n = 1, consumed = length); flags invalid codes.
__device__ __noinline__ uint32_t slow_entry(const GroupTab& t, const uint8_t* syms,
                                            uint32_t win12, uint32_t& bad) {
  int l = kW + 1;
  while (l <= kMaxLen && win12 >= t.lim[l]) l++;
  if (l > kMaxLen) {
    bad = 1;
    return (1u << 24) | ((uint32_t)kMaxLen << 26);
  }
  const uint32_t r = t.index[l] + (win12 >> (kMaxLen - l)) - t.first[l];
  return (uint32_t)syms[r & 255] | (1u << 24) | ((uint32_t)l << 26);
}

// Decode the next V symbols of a sub-stream into acc (little-endian bytes).
// Entries: bits 0-23 up to three symbols, 24-25 count n, 26-29 bits consumed.
// lo:hi carry symbols decoded past the vector boundary to the next call.
template <int V>
struct SymQueue {
  uint64_t lo;
  uint32_t hi;
  uint32_t p;  // symbols held
};

template <int V>
__device__ __forceinline__ void decode_vec(BitReader& br, const uint32_t* lut, const GroupTab& t,
                                           const uint8_t* syms, SymQueue<V>& q, uint32_t out[4],
                                           uint32_t& bad) {
  if (V == 16) {
    // two halves of 8 symbols
#pragma unroll
    for (int half = 0; half < 2; half++) {
      while (q.p < 8) {
        uint32_t e = lut[br.peek32() >> (32 - kW)];
        if ((e >> 24 & 3u) == kSlow) e = slow_entry(t, syms, br.peek32() >> (32 - kMaxLen), bad);
        const uint32_t s24 = e & 0xFFFFFFu, sh = 8u * q.p;
        q.lo |= (uint64_t)s24 << sh;
        if (sh >= 48) q.hi |= s24 >> (64 - sh);
        q.p += e >> 24 & 3u;
        br.skip(e >> 26);
      }
      out[2 * half] = (uint32_t)q.lo;
      out[2 * half + 1] = (uint32_t)(q.lo >> 32);
      q.lo = q.hi;
      q.hi = 0;
      q.p -= 8;
    }
  } else {
    while (q.p < (uint32_t)V) {
      uint32_t e = lut[br.peek32() >> (32 - kW)];
      if ((e >> 24 & 3u) == kSlow) e = slow_entry(t, syms, br.peek32() >> (32 - kMaxLen), bad);
      const uint32_t s24 = e & 0xFFFFFFu, sh = 8u * q.p;
      q.lo |= (uint64_t)s24 << sh;
      if (sh >= 48) q.hi |= s24 >> (64 - sh);
      q.p += e >> 24 & 3u;
      br.skip(e >> 26);
    }
    if (V == 8) {
      out[0] = (uint32_t)q.lo;
      out[1] = (uint32_t)(q.lo >> 32);
      q.lo = q.hi;
      q.hi = 0;
      q.p -= 8;
    } else {  // V == 4
      out[0] = (uint32_t)q.lo;
      q.lo = (q.lo >> 32) | ((uint64_t)q.hi << 32);
      q.hi = 0;
      q.p -= 4;
    }
  }
}

__device__ __forceinline__ uint32_t rd_u32(const uint8_t* p) {
  return __ldg(reinterpret_cast<const uint32_t*>(p));
}

// Decode one chunk of a tensor of dtype DT.
template <int DT>
__device__ void decode_chunk(const Job& J, uint64_t c, Smem& S, uint32_t* lut_base,
                             uint32_t* err) {
  constexpr int G = Traits<DT>::G, V = Traits<DT>::V, ES = 16 / V;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const uint64_t off0 = c * J.chunk_bytes;
  const uint64_t nb = min((uint64_t)J.chunk_bytes, J.nbytes - off0);
  const uint64_t m = nb / ES;
  const uint64_t nvec = (nb + 15) / 16;
  const uint32_t T = J.lanes;
  const uint8_t* cont = J.src;
  const uint64_t P = kHdrBytes + (uint64_t)J.n_chunks * G * kEntryBytes;
  ChunkInfo& CI = S.ci;

  // 1a. map entries (one 16-B load per group)
  if (tid == 0) CI.bad = 0;
  __syncthreads();
  if (tid < G) {
    const uint4 e = __ldg(reinterpret_cast<const uint4*>(cont + kHdrBytes + (c * G + tid) * kEntryBytes));
    const uint64_t po = (uint64_t)e.x | ((uint64_t)e.y << 32);
    const uint32_t size = e.z, mode = e.w & 0xFFu, value = (e.w >> 8) & 0xFFu;
    uint32_t bad = (e.w >> 16) != 0;
    const uint64_t avail = J.stream_bytes > P ? J.stream_bytes - P : 0;
    if (mode > kConst || po > avail || align_up(size, 16) > avail - po || (po & 15)) bad = 1;
    if (mode == kRaw && size != m) bad = 1;
    if ((mode == kZero || mode == kConst) && size != 0) bad = 1;
    if (mode == kHuff && size < 12) bad = 1;
    CI.mode[tid] = bad ? kZero : mode;
    CI.value[tid] = value;
    CI.size[tid] = size;
    CI.payload[tid] = P + po;
    if (bad) atomicOr(&CI.bad, 1u);
  }
  __syncthreads();
  if (CI.bad) {
    if (tid == 0) atomicOr(err, 1u);
    return;
  }
  // 1b. table bytes of every Huffman group (word loads, clamped to the payload)
#pragma unroll
  for (int g = 0; g < G; g++) {
    if (CI.mode[g] != kHuff) continue;
    const uint8_t* p = cont + CI.payload[g];
    for (int i = tid; i < 68; i += nthr)
      S.tab[g].words[i] = (4u * i + 4u <= CI.size[g]) ? rd_u32(p + 4 * i) : 0u;
  }
  __syncthreads();
  // 1c. canonical limits (thread g), validation
  if (tid < G && CI.mode[tid] == kHuff) {
    GroupTab& t = S.tab[tid];
    uint32_t nz = 0, kraft = 0, code = 0, idx = 0, prevc = 0;
    t.lim[0] = 0;
    for (int l = 1; l <= kMaxLen; l++) {
      const uint32_t cl = tab_byte(t, l - 1);
      code = (code + prevc) << 1;
      t.first[l] = code;
      t.index[l] = idx;
      t.lim[l] = (code + cl) << (kMaxLen - l);
      idx += cl;
      prevc = cl;
      nz += cl;
      kraft += cl << (kMaxLen - l);
    }
    t.lim[kMaxLen + 1] = 0xFFFFFFFFu;
    const uint64_t h = align_up(12 + nz, 4);
    const uint64_t size = CI.size[tid];
    if (nz < 2 || nz > 256 || kraft > (uint32_t)kLutSize || size < h + 4ull * (T - 1) ||
        (size - h - 4ull * (T - 1)) % 4) {
      atomicOr(&CI.bad, 1u);
    } else {
      CI.offs[tid] = CI.payload[tid] + h;
      CI.bs[tid] = CI.payload[tid] + h + 4ull * (T - 1);
      CI.nwords[tid] = (uint32_t)((size - h - 4ull * (T - 1)) / 4);
    }
  }
  __syncthreads();
  if (CI.bad) {
    if (tid == 0) atomicOr(err, 1u);
    return;
  }

  // 2. multi-symbol tables.  Window w (kW bits): first code length
  // l1 = 1 + #{l <= kW : lim_W[l] <= w}; if l1 > kW, slow path.
#pragma unroll
  for (int g = 0; g < G; g++) {
    if (CI.mode[g] != kHuff) continue;
    const GroupTab& t = S.tab[g];
    const uint8_t* syms = reinterpret_cast<const uint8_t*>(t.words) + 12;
    uint32_t limw[kW + 1];
#pragma unroll
    for (int l = 1; l <= kW; l++) limw[l] = t.lim[l] >> (kMaxLen - kW);
    uint32_t* L = lut_base + g * kLut;
    for (int w = tid; w < kLut; w += nthr) {
      uint32_t ent = 0, n = 0, used = 0;
      uint32_t rest = (uint32_t)w;  // remaining window bits, left-aligned in kW bits
#pragma unroll
      for (int k = 0; k < 3; k++) {
        uint32_t l = 1;
#pragma unroll
        for (int q = 1; q <= kW; q++) l += (limw[q] <= rest);
        if (l > (uint32_t)(kW - used)) break;  // code not wholly inside the window
        const uint32_t r = t.index[l] + (rest >> (kW - l)) - t.first[l];
        ent |= (uint32_t)syms[r & 255] << (8 * k);
        n++;
        used += l;
        rest = (rest << l) & (kLut - 1);
      }
      L[w] = n ? (ent | (n << 24) | (used << 26)) : kSlow;
    }
  }
  __syncthreads();

  // 3. decode + merge
  uint8_t* dst = J.dst + off0;
  const uint8_t* base = J.base ? J.base + off0 : nullptr;
  uint32_t bad = 0;
  for (uint32_t t = tid; t < T; t += nthr) {
    BitReader br[G];
    SymQueue<V> sq[G];
#pragma unroll
    for (int g = 0; g < G; g++) {
      sq[g].lo = 0;
      sq[g].hi = 0;
      sq[g].p = 0;
      if (CI.mode[g] != kHuff) continue;
      uint32_t start = t ? rd_u32(cont + CI.offs[g] + 4ull * (t - 1)) : 0u;
      if (start > CI.nwords[g] * 32u) {
        bad = 1;
        start = CI.nwords[g] * 32u;
      }
      br[g].init(reinterpret_cast<const uint32_t*>(cont + CI.bs[g]), CI.nwords[g], start);
    }
    // raw group bytes of the next vector, prefetched
    uint32_t rawn[G][4] = {};
    auto load_raw = [&](uint64_t v, uint32_t (&r)[G][4]) {
#pragma unroll
      for (int g = 0; g < G; g++) {
        if (CI.mode[g] != kRaw || v >= nvec) continue;
        const uint8_t* p = cont + CI.payload[g] + v * V;
        if (V == 8) {
          const uint2 x = __ldg(reinterpret_cast<const uint2*>(p));
          r[g][0] = x.x; r[g][1] = x.y;
        } else if (V == 4) {
          r[g][0] = __ldg(reinterpret_cast<const uint32_t*>(p));
        } else {
          const uint4 x = __ldg(reinterpret_cast<const uint4*>(p));
          r[g][0] = x.x; r[g][1] = x.y; r[g][2] = x.z; r[g][3] = x.w;
        }
      }
    };
    load_raw(t, rawn);
    for (uint64_t v = t; v < nvec; v += T) {
      uint32_t gw[G][4];
#pragma unroll
      for (int g = 0; g < G; g++)
#pragma unroll
        for (int k = 0; k < 4; k++) gw[g][k] = rawn[g][k];
      load_raw(v + T, rawn);
      uint4 bv = make_uint4(0, 0, 0, 0);
      const bool full = (v + 1) * 16 <= nb;
      if (base && full) bv = __ldg(reinterpret_cast<const uint4*>(base) + v);
#pragma unroll
      for (int g = 0; g < G; g++) {
        const uint32_t mode = CI.mode[g];
        if (mode == kHuff) {
          const uint8_t* syms = reinterpret_cast<const uint8_t*>(S.tab[g].words) + 12;
          decode_vec<V>(br[g], lut_base + g * kLut, S.tab[g], syms, sq[g], gw[g], bad);
        } else if (mode != kRaw) {
          const uint32_t b = (mode == kConst) ? CI.value[g] * 0x01010101u : 0u;
          gw[g][0] = b; gw[g][1] = b; gw[g][2] = b; gw[g][3] = b;
        }
      }
      uint32_t x[4];
      if (DT == ZIPNN_FP32) {
        uint32_t g4[4] = {gw[0][0], gw[1 % G][0], gw[2 % G][0], gw[3 % G][0]};
        merge32(g4, x);
      } else if (DT == ZIPNN_U8) {
        x[0] = gw[0][0]; x[1] = gw[0][1]; x[2] = gw[0][2]; x[3] = gw[0][3];
      } else {
        merge16(gw[0][0], gw[1 % G][0], x[0], x[1]);
        merge16(gw[0][1], gw[1 % G][1], x[2], x[3]);
      }
      if (full) {
        x[0] ^= bv.x; x[1] ^= bv.y; x[2] ^= bv.z; x[3] ^= bv.w;
        reinterpret_cast<uint4*>(dst)[v] = make_uint4(x[0], x[1], x[2], x[3]);
      } else {
        for (uint64_t k = v * 16; k < nb; k++) {
          uint32_t byte = (x[(k - v * 16) >> 2] >> (8 * (k & 3))) & 0xFFu;
          if (base) byte ^= base[k];
          dst[k] = (uint8_t)byte;
        }
      }
    }
  }
  if (bad) atomicOr(err, 1u);
}

// DTS: the dtype of every job in the launch, or -1 for a mixed batch.
template <int DTS>
__global__ void __launch_bounds__(kDecThreads)
k_decode(JobRef jr, uint64_t nchunks_total, uint32_t* __restrict__ err,
         unsigned long long* __restrict__ ticket) {
  extern __shared__ uint32_t lut_smem[];  // [groups][kLut]
  __shared__ Smem S;
  const int tid = threadIdx.x;
  for (uint64_t iter = 0;; iter++) {
    // work item: from the device queue (batched form) or a static stride
    uint64_t chunk;
    if (ticket) {
      if (tid == 0) S.chunk = atomicAdd(ticket, 1ull);
      __syncthreads();
      chunk = S.chunk;
    } else {
      chunk = blockIdx.x + iter * gridDim.x;
    }
    if (chunk >= nchunks_total) break;
    const int j = jr.table ? find_job(jr.table, jr.n, chunk) : 0;
    const Job& J = jr.table ? jr.table[j] : jr.one;
    const uint64_t c = chunk - J.chunk_begin;
    if (DTS >= 0) {
      decode_chunk<(DTS < 0 ? 0 : DTS)>(J, c, S, lut_smem, err);
    } else {
      switch (J.dtype) {
        case ZIPNN_BF16: decode_chunk<ZIPNN_BF16>(J, c, S, lut_smem, err); break;
        case ZIPNN_FP16: decode_chunk<ZIPNN_FP16>(J, c, S, lut_smem, err); break;
        case ZIPNN_FP32: decode_chunk<ZIPNN_FP32>(J, c, S, lut_smem, err); break;
        default: decode_chunk<ZIPNN_U8>(J, c, S, lut_smem, err); break;
      }
    }
    __syncthreads();
  }
}

}  // namespace

int decode_smem_bytes(int max_groups) { return max_groups * kLut * 4; }

cudaError_t launch_decode_ex(const Job* d_jobs, const Job* h_one, int njobs,
                             uint64_t nchunks_total, int max_groups, const zipnn_tuning* tuning,
                             uint32_t* d_err, unsigned long long* d_ticket, cudaStream_t st,
                             int uniform_dtype) {
  if (nchunks_total == 0) return cudaSuccess;
  JobRef r;
  r.table = h_one ? nullptr : d_jobs;
  if (h_one) r.one = *h_one;
  else memset(&r.one, 0, sizeof(Job));
  r.n = njobs;
  if (h_one) uniform_dtype = h_one->dtype;
  void (*kern)(JobRef, uint64_t, uint32_t*, unsigned long long*);
  switch (uniform_dtype) {
    case ZIPNN_BF16: kern = k_decode<ZIPNN_BF16>; break;
    case ZIPNN_FP16: kern = k_decode<ZIPNN_FP16>; break;
    case ZIPNN_FP32: kern = k_decode<ZIPNN_FP32>; break;
    case ZIPNN_U8: kern = k_decode<ZIPNN_U8>; break;
    default: kern = k_decode<-1>; break;
  }
  const int threads = kDecThreads;
  int per_sm = 0;
  if (tuning && tuning->ctas_per_sm > 0) per_sm = tuning->ctas_per_sm;
  const int smem = decode_smem_bytes(max_groups);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (per_sm == 0) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    per_sm = occ > 0 ? occ : 1;
  }
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > nchunks_total) grid = nchunks_total;
  if (d_ticket) {
    cudaError_t e = cudaMemsetAsync(d_ticket, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  kern<<<(unsigned)grid, threads, smem, st>>>(r, nchunks_total, d_err, d_ticket);
  return cudaGetLastError();
}

}  // namespace zipnn
