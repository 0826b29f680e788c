// Decoder kernels of the GB300 ZipNN codec (device code, included by one
// translation unit per table width and CTA size, decode_w<W>_<threads>.cu, so
// that their kernels compile in parallel): table-driven Huffman decoding of
// every byte-group stream of a chunk and the merge back to the original dtype
// (ZipNN Sec. 3.1, 3.2 inverse; Sec. 4.2 XOR with the base; Sec. 5.1 map).
//
// Work unit = one chunk.  A persistent grid pulls chunks of all tensors of a
// batch from a device ticket (atomicAdd), so one launch decodes many tensors of
// uneven sizes.  Per chunk the CTA
//   1. loads and validates the chunk's map entries and Huffman tables with
//      16-byte / 4-byte cooperative loads into shared memory,
//   2. stages every Huffman payload that fits (table, start offsets,
//      bitstream) into shared memory with one TMA bulk copy per payload
//      (cp.async.bulk, completion on an mbarrier; payloads are 16-B aligned and
//      padded by the format), overlapped with step 3,
//   3. builds, per Huffman group, a 2^W-entry table (W = 10..12, chosen at
//      launch): the entry for a W-bit window holds its first two codes when
//      both fit in it (symbols and bits consumed), else its first code; with
//      W = 11 a 12-bit first code is resolved in the entry by its last bit,
//      with W = 10 longer first codes go through the canonical limits,
//   4. decodes: thread t owns interleaved sub-streams t (and t + nthr when
//      there are twice as many sub-streams as threads), i.e. the vectors
//      v = t, t+T, ... of the chunk, so each warp step touches 32 consecutive
//      16-byte vectors: raw-group loads and the 16-B output stores are fully
//      coalesced; the inverse permutation and the XOR with a delta base happen
//      in registers.  Chunks laid out as "exponent Huffman, every other group
//      raw, zero or constant" (nearly every chunk of a model) take a
//      specialised loop without per-group mode tests; its raw words arrive two
//      steps ahead in registers (16-bit) or through a per-thread ring of
//      asynchronous copies in shared memory (FP32), after a bulk L2 prefetch
//      of the chunk's first steps issued while the tables are built.  Kernels
//      for launches holding a delta (GEN) add the loops for a SPARSE exponent
//      group and for two coded 16-bit groups.
// The decoder is total: symbol counts are fixed by the map, bit reads past a
// payload return zero bits, invalid codes and bad map entries set the error
// word, and every loop is bounded; the wait for a bulk copy gives up after 2 s
// of %globaltimer (error ETIMEOUT, the CTA waits again, bounded, then exits).
#pragma once
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "zipnn_internal.cuh"

namespace zipnn {

namespace {

constexpr int kDecThreads = 128;  // CTA size of mixed-dtype and W = 10 launches; else 256
// Shared-memory staging for Huffman payloads: sized at launch from the largest
// chunk and the dtypes of the launch (decode_stage_bytes); payloads that do
// not fit are read from global memory instead.
constexpr uint32_t kStageMin = 4096;
constexpr uint32_t kStageCapPerSm = 227u * 1024u;  // shared memory an SM gives its CTAs
constexpr uint32_t kStaticReserve = 4096;          // static Smem + the per-CTA reservation
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kPfBudget = 16ull << 20;  // L2 bytes the fast loops' prefetches may hold

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// Loads and stores through 32-bit shared-window addresses, so that table
// lookups compile to shared-memory instructions even where the table's
// location is only known at run time.
__device__ __forceinline__ uint32_t lds32(uint32_t saddr) {
  uint32_t v;
  asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(saddr));
  return v;
}
__device__ __forceinline__ void sts32(uint32_t saddr, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(saddr), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
}
// 1-D TMA bulk copy global -> shared (16-B aligned addresses, size % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// Count `bytes` of the barrier's expected transaction bytes as arrived without
// a copy (cancels bytes that were expected but never requested).
__device__ __forceinline__ void mbar_complete_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity`; false if it gave up after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > limit_ns) return false;
  return true;
}

// Thread-block clusters (split work items of one chunk): the CTA's rank and
// the cluster's size, a shared address mapped into a peer CTA's shared
// memory, a store there, and the cluster-wide barrier (release / acquire).
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t n;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
  return n;
}
__device__ __forceinline__ uint32_t map_peer(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_peer(uint32_t caddr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(caddr), "r"(v) : "memory");
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

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
  uint64_t bs[4];           // bitstream offset within the payload (HUFF)
  uint64_t offs[4];         // start-bit table offset within the payload (HUFF)
  uint64_t bmo[4];          // vector bitmap offset within the payload (SPARSE)
  uint32_t staged[4];       // stage offset of the payload, or ~0 if read from global
  uint32_t stage_bytes;
  uint32_t bad;
};

struct Smem {
  ChunkInfo ci;
  GroupTab tab[4];
  uint32_t* lut_ptr[4];  // pair table of each Huffman group
  unsigned long long chunk;
  int job;               // job of the CTA's previous work item
  uint32_t part;         // part of the chunk (chunks split over several work items)
};

// Groups carried as Huffman sub-streams: HUFF, and SPARSE (the same after a
// bitmap of the vectors that hold a non-zero symbol).
__device__ __forceinline__ bool coded_mode(uint32_t m) { return m == kHuff || m == kSparse; }

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

// Reader over a bitstream staged in shared memory.  Word reads are clamped to
// index nwords + 1 (the staging leaves 32 bytes of slack after each payload),
// so a corrupt stream cannot walk the reader out of the stage.
struct SmemBitReader {
  const uint32_t* w;
  uint32_t idx, lim, w0, w1, pos;
  __device__ __forceinline__ void init(const uint32_t* words, uint32_t nwords, uint32_t start) {
    w = words;
    lim = nwords + 1;
    idx = start >> 5;
    pos = start & 31;
    w0 = w[min(idx, lim)];
    w1 = w[min(idx + 1, lim)];
    idx += 2;
  }
  __device__ __forceinline__ uint32_t peek32() const { return __funnelshift_l(w1, w0, pos); }
  __device__ __forceinline__ void skip(uint32_t bits) {
    pos += bits;
    if (pos >= 32) {
      pos -= 32;
      w0 = w1;
      w1 = w[min(idx, lim)];
      idx++;
    }
  }
};

__device__ __forceinline__ uint32_t rd_u32(const uint8_t* p) {
  return __ldg(reinterpret_cast<const uint32_t*>(p));
}

// Pair tables.  The entry for a W-bit window w describes the codes at its
// start:
//   bits 0-7    first symbol (or, for a long first code, its symbol when the
//               window's next bit is 0)
//   bits 8-15   second symbol (pair) or the long code's symbol for next bit 1
//   bits 16-19  length l1 of the first code (0: invalid window, or, for W = 10,
//               a first code longer than the window -> slow path)
//   bit 20      pair: both codes lie wholly inside the window
//   bit 21      long: the first code has W + 1 bits (W = 11 only)
//   bits 22-23  long code invalid for next bit 0 / 1
//   bits 27-31  bits consumed by the entry (pair: l1 + l2)
// Symbols are stored rotated right by one bit when the chunk takes the fast
// loop (the merge then needs only bit selects, see merge16r).
constexpr uint32_t kPair = 1u << 20;
constexpr uint32_t kLong = 1u << 21;
constexpr uint32_t kBadLong0 = 1u << 22;

// Slow path (W = 10): resolve the first code of a 12-bit window with the
// canonical limits.  Returns (symbol | length << 16); flags windows that start
// no code.
__device__ __noinline__ uint32_t slow_code(const GroupTab& t, const uint8_t* syms, uint32_t win12,
                                           uint32_t& bad) {
  int l = 1;
  while (l <= kMaxLen && win12 >= t.lim[l]) l++;
  if (l > kMaxLen) {
    bad = 1;
    return (uint32_t)kMaxLen << 16;
  }
  const uint32_t r = t.index[l] + (win12 >> (kMaxLen - l)) - t.first[l];
  return (uint32_t)syms[r & 255] | ((uint32_t)l << 16);
}

// First code of the 32-bit window `win` whose table entry is e:
// (symbol | length << 16).
template <int W>
__device__ __forceinline__ uint32_t first_code(uint32_t e, uint32_t win, const GroupTab& t,
                                               const uint8_t* syms, uint32_t& bad) {
  if (W == 11 && (e & kLong)) {
    const uint32_t nb = (win >> (31 - W)) & 1u;
    bad |= (e >> (22 + nb)) & 1u;
    return ((e >> (8 * nb)) & 0xFFu) | ((uint32_t)(W + 1) << 16);
  }
  const uint32_t l = (e >> 16) & 15u;
  if (l == 0) {
    if (W == 10) return slow_code(t, syms, win >> (32 - kMaxLen), bad);
    bad = 1;
    return (uint32_t)W << 16;
  }
  return (e & 0xFFu) | (l << 16);
}

// Entry for two symbols at the window: the table entry when it is a pair,
// otherwise the two first codes resolved one after the other (rare).  Bits
// 0-15 hold the symbols, 27-31 the bits consumed.
template <int W>
__device__ __forceinline__ uint32_t pair_at(uint32_t win, uint32_t lut, const GroupTab& t,
                                            const uint8_t* syms, uint32_t& bad) {
  uint32_t e = lds32(lut + ((win >> (32 - W)) << 2));
  if (!(e & kPair)) {
    const uint32_t c0 = first_code<W>(e, win, t, syms, bad);
    const uint32_t l0 = c0 >> 16;
    const uint32_t win2 = win << l0;
    const uint32_t c1 = first_code<W>(lds32(lut + ((win2 >> (32 - W)) << 2)), win2, t, syms, bad);
    e = (c0 & 0xFFu) | ((c1 & 0xFFu) << 8) | ((l0 + (c1 >> 16)) << 27);
  }
  return e;
}

// Two symbols (sym0 | sym1 << 8).
template <int W, class BR>
__device__ __forceinline__ uint32_t two_symbols(BR& br, uint32_t lut, const GroupTab& t,
                                                const uint8_t* syms, uint32_t& bad) {
  const uint32_t e = pair_at<W>(br.peek32(), lut, t, syms, bad);
  br.skip(e >> 27);
  return e & 0xFFFFu;
}

// merge16 / merge32 for exponent bytes stored rotated right by one bit
// (e' = e >> 1 | e << 7 per byte): each output byte is a bit select.
__device__ __forceinline__ void merge16r(uint32_t er, uint32_t r, uint32_t& w0, uint32_t& w1) {
  const uint32_t hi = (r & 0x80808080u) | (er & 0x7F7F7F7Fu);
  const uint32_t lo = (er & 0x80808080u) | (r & 0x7F7F7F7Fu);
  w0 = __byte_perm(lo, hi, 0x5140);
  w1 = __byte_perm(lo, hi, 0x7362);
}

struct Staging {
  uint8_t* base;       // shared-memory stage
  uint32_t cap;        // its size in bytes
  uint32_t pf_bytes;   // L2 prefetch window of the fast loops per CTA (bytes)
  uint32_t ring;       // shared-memory address of the raw-word rings (kRingBytes per thread)
  uint32_t ring_bytes; // their size (0: the launch has none); they follow the stage
  uint64_t* bar;       // its mbarrier
  uint32_t parity;     // phase to wait for next
  uint32_t extra_tx;   // fault injection: bytes expected but never sent (0 normally)
  uint64_t limit_ns;   // wait limit
};

// Decode loop of one chunk.  Each thread owns NS sub-streams (t, t + nthr,
// ...) and advances them in lockstep, one 16-byte vector each per step (V
// symbols per Huffman group = V/2 pair lookups, independent across the NS
// sub-streams, which gives the scheduler instruction-level parallelism); each
// vector is merged with the raw / constant groups and stored.
template <int DT, int W, class BR, bool STAGED, int NS>
__device__ __forceinline__ void decode_loop(const Job& J, uint64_t c, Smem& S, Staging& stg,
                                            uint32_t* err) {
  constexpr int G = Traits<DT>::G, V = Traits<DT>::V;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const uint64_t off0 = c * J.chunk_bytes;
  const uint32_t nb = (uint32_t)min((uint64_t)J.chunk_bytes, J.nbytes - off0);
  const uint32_t nvec = (nb + 15) / 16;
  const uint32_t T = J.lanes;
  const uint8_t* cont = J.src;
  ChunkInfo& CI = S.ci;
  uint8_t* dst = J.dst + off0;
  const uint8_t* base = J.base ? J.base + off0 : nullptr;
  uint32_t mode[G], cval[G], nwords[G], offs[G], bsoff[G];
  const uint8_t* rawp[G];
  const uint8_t* pay[G];
  const uint32_t* bmp[G];   // SPARSE: bitmap of the vectors holding a non-zero symbol
  uint32_t lut[G];  // shared-window addresses of the pair tables
#pragma unroll
  for (int g = 0; g < G; g++) {
    mode[g] = CI.mode[g];
    cval[g] = CI.value[g] * 0x01010101u;
    nwords[g] = CI.nwords[g];
    rawp[g] = cont + CI.payload[g];
    pay[g] = STAGED ? stg.base + CI.staged[g] : cont + CI.payload[g];
    offs[g] = (uint32_t)CI.offs[g];
    bsoff[g] = (uint32_t)CI.bs[g];
    lut[g] = smem_u32(S.lut_ptr[g]);
    bmp[g] = reinterpret_cast<const uint32_t*>(pay[g] + (uint32_t)CI.bmo[g]);
  }
  uint32_t bad = 0;
  for (uint32_t t0 = tid; t0 < T; t0 += NS * nthr) {
    BR br[NS][G];
    uint32_t tt[NS];
    bool act[NS];
#pragma unroll
    for (int j = 0; j < NS; j++) {
      tt[j] = t0 + j * nthr;
      act[j] = tt[j] < T;
      const uint32_t t = act[j] ? tt[j] : 0u;
#pragma unroll
      for (int g = 0; g < G; g++) {
        if (mode[g] != kHuff && mode[g] != kSparse) continue;
        uint32_t start = 0;
        if (t) start = STAGED ? *reinterpret_cast<const uint32_t*>(pay[g] + offs[g] + 4u * (t - 1))
                              : rd_u32(pay[g] + offs[g] + 4u * (t - 1));
        if (start > nwords[g] * 32u) {
          bad = 1;
          start = nwords[g] * 32u;
        }
        br[j][g].init(reinterpret_cast<const uint32_t*>(pay[g] + bsoff[g]), nwords[g], start);
      }
    }
    // raw group bytes, prefetched one vector ahead
    uint32_t rawn[NS][G][4] = {};
    auto load_raw = [&](int j, uint32_t v) {
#pragma unroll
      for (int g = 0; g < G; g++) {
        if (mode[g] != kRaw || v >= nvec) continue;
        const uint8_t* p = rawp[g] + (size_t)v * V;
        if (V == 8) {
          const uint2 x = __ldg(reinterpret_cast<const uint2*>(p));
          rawn[j][g][0] = x.x; rawn[j][g][1] = x.y;
        } else if (V == 4) {
          rawn[j][g][0] = __ldg(reinterpret_cast<const uint32_t*>(p));
        } else {
          const uint4 x = __ldg(reinterpret_cast<const uint4*>(p));
          rawn[j][g][0] = x.x; rawn[j][g][1] = x.y; rawn[j][g][2] = x.z; rawn[j][g][3] = x.w;
        }
      }
    };
#pragma unroll
    for (int j = 0; j < NS; j++)
      if (act[j]) load_raw(j, tt[j]);
    for (uint32_t ks = 0;; ks++) {
      uint32_t vv[NS];
      bool live[NS];
      bool any = false;
#pragma unroll
      for (int j = 0; j < NS; j++) {
        vv[j] = tt[j] + ks * T;
        live[j] = act[j] && vv[j] < nvec;
        any |= live[j];
      }
      if (!any) break;
      uint32_t gw[NS][G][4];
#pragma unroll
      for (int j = 0; j < NS; j++) {
#pragma unroll
        for (int g = 0; g < G; g++)
#pragma unroll
          for (int k = 0; k < 4; k++) gw[j][g][k] = rawn[j][g][k];
        if (live[j]) load_raw(j, vv[j] + T);
      }
#pragma unroll
      for (int g = 0; g < G; g++) {
        if (mode[g] == kHuff || mode[g] == kSparse) {
          const GroupTab& tb = S.tab[g];
          const uint8_t* syms = reinterpret_cast<const uint8_t*>(tb.words) + 12;
          // SPARSE: a vector whose bit is clear is all zero and has no codes
          bool coded[NS];
#pragma unroll
          for (int j = 0; j < NS; j++) {
            coded[j] = true;
            if (mode[g] == kSparse && live[j]) {
              const uint32_t wi = vv[j] >> 5;
              const uint32_t word = STAGED ? bmp[g][wi] : __ldg(bmp[g] + wi);
              coded[j] = (word >> (vv[j] & 31u)) & 1u;
            }
          }
#pragma unroll
          for (int q = 0; q < V / 4; q++) {
            uint32_t a[NS], b[NS];
#pragma unroll
            for (int j = 0; j < NS; j++)
              a[j] = coded[j] ? two_symbols<W>(br[j][g], lut[g], tb, syms, bad) : 0u;
#pragma unroll
            for (int j = 0; j < NS; j++)
              b[j] = coded[j] ? two_symbols<W>(br[j][g], lut[g], tb, syms, bad) : 0u;
#pragma unroll
            for (int j = 0; j < NS; j++) gw[j][g][q] = a[j] | (b[j] << 16);
          }
        } else if (mode[g] != kRaw) {
#pragma unroll
          for (int j = 0; j < NS; j++) {
            gw[j][g][0] = cval[g]; gw[j][g][1] = cval[g]; gw[j][g][2] = cval[g]; gw[j][g][3] = cval[g];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NS; j++) {
        if (!live[j]) continue;
        const uint32_t v = vv[j];
        uint32_t x[4];
        if (DT == ZIPNN_FP32) {
          uint32_t g4[4] = {gw[j][0][0], gw[j][1 % G][0], gw[j][2 % G][0], gw[j][3 % G][0]};
          merge32(g4, x);
        } else if (DT == ZIPNN_U8) {
          x[0] = gw[j][0][0]; x[1] = gw[j][0][1]; x[2] = gw[j][0][2]; x[3] = gw[j][0][3];
        } else {
          merge16(gw[j][0][0], gw[j][1 % G][0], x[0], x[1]);
          merge16(gw[j][0][1], gw[j][1 % G][1], x[2], x[3]);
        }
        if ((v + 1) * 16 <= nb) {
          if (base) {
            const uint4 bb = __ldg(reinterpret_cast<const uint4*>(base) + v);
            x[0] ^= bb.x; x[1] ^= bb.y; x[2] ^= bb.z; x[3] ^= bb.w;
          }
          reinterpret_cast<uint4*>(dst)[v] = make_uint4(x[0], x[1], x[2], x[3]);
        } else {
          for (uint32_t k = v * 16; k < nb; k++) {
            uint32_t byte = (x[(k - v * 16) >> 2] >> (8 * (k & 3))) & 0xFFu;
            if (base) byte ^= base[k];
            dst[k] = (uint8_t)byte;
          }
        }
      }
    }
  }
  if (bad) atomicOr(err, 1u);
}

// merge32 for a rotated exponent byte (see merge16r).
__device__ __forceinline__ void merge32r(uint32_t er, uint32_t g1, uint32_t g2, uint32_t g3,
                                         uint32_t x[4]) {
  const uint32_t b3 = (g1 & 0x80808080u) | (er & 0x7F7F7F7Fu);
  const uint32_t b2 = (er & 0x80808080u) | (g1 & 0x7F7F7F7Fu);
  const uint32_t lo01 = __byte_perm(g3, g2, 0x5140), hi01 = __byte_perm(b2, b3, 0x5140);
  const uint32_t lo23 = __byte_perm(g3, g2, 0x7362), hi23 = __byte_perm(b2, b3, 0x7362);
  x[0] = __byte_perm(lo01, hi01, 0x5410);
  x[1] = __byte_perm(lo01, hi01, 0x7632);
  x[2] = __byte_perm(lo23, hi23, 0x5410);
  x[3] = __byte_perm(lo23, hi23, 0x7632);
}

// Words of the groups 1..G-1 of one vector (V bytes per group): loaded from
// the raw payload when bit g of rawm is set, else the group's constant byte
// (ZERO / CONST) replicated in cw[g].
template <int DT>
__device__ __forceinline__ void load_raw_vec(const uint8_t* const* rawp, uint32_t rawm,
                                             const uint32_t* cw, uint32_t v, uint32_t* rw) {
  if constexpr (DT == ZIPNN_FP32) {
#pragma unroll
    for (int g = 1; g < 4; g++)
      rw[g - 1] = (rawm >> g & 1u) ? __ldg(reinterpret_cast<const uint32_t*>(rawp[g]) + v) : cw[g];
  } else if constexpr (DT != ZIPNN_U8) {
    if (rawm & 2u) {
      const uint2 x = __ldg(reinterpret_cast<const uint2*>(rawp[1]) + v);
      rw[0] = x.x;
      rw[1] = x.y;
    } else {
      rw[0] = cw[1];
      rw[1] = cw[1];
    }
  }
}

// Bulk prefetch into L2 (asynchronous, no registers, no completion to wait
// for), in pieces of at most 32 KiB; p 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const uint8_t* p, uint64_t bytes) {
  for (uint64_t o = 0; o < bytes; o += 32768u) {
    const uint32_t n = (uint32_t)(bytes - o < 32768u ? bytes - o : 32768u);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p + o), "r"(n) : "memory");
  }
}

// The fast loops read the raw groups (and a delta's base) straight from
// global memory, each thread a few vectors ahead: too few bytes in flight per
// SM to cover DRAM latency.  Step k of a fast loop consumes vectors
// [kT, (k+1)T) of the chunk, i.e. a contiguous slice of T * 16/G bytes of
// every raw group and T * 16 bytes of the base, so the slices of the first D
// steps are requested into L2 as bulk prefetches while the tables are built,
// and the FP32 and delta loops keep requesting D steps ahead of themselves.
// D = the CTA's share of an L2 budget (pf_bytes) over the bytes of one step,
// at least 2, at most the whole chunk.  Only when one pass over the
// sub-streams covers every lane (T == NS * nthr), so that all threads sweep
// the slices together.
template <int G>
__device__ __forceinline__ uint32_t pf_steps(uint32_t rawm, bool has_base, uint32_t T,
                                             uint32_t nper, uint32_t pf_bytes) {
  const uint32_t per_step = ((uint32_t)__popc(rawm) * (16u / G) + (has_base ? 16u : 0u)) * T;
  if (per_step == 0) return 0;
  const uint32_t d = pf_bytes / per_step;
  return d < 2u ? 2u : (d > nper ? nper : d);
}
template <int G>
__device__ __forceinline__ void prefetch_steps(const uint8_t* const (&rawp)[G], uint32_t rawm,
                                               const uint8_t* base, uint32_t T, uint32_t k0,
                                               uint32_t k1) {
  if (k1 <= k0) return;
  const uint64_t gb = (uint64_t)T * (16u / G);  // bytes of one raw group per step
#pragma unroll
  for (int g = 0; g < G; g++)
    if ((rawm >> g) & 1u) bulk_prefetch_l2(rawp[g] + k0 * gb, (k1 - k0) * gb);
  if (base) bulk_prefetch_l2(base + (uint64_t)k0 * T * 16u, (uint64_t)(k1 - k0) * T * 16u);
}

// Per-thread asynchronous copies global -> shared (no registers held while in
// flight); groups complete in the order they were committed.  The ring is
// touched only by these volatile statements, whose order the compiler keeps.
__device__ __forceinline__ void cp_async4(uint32_t saddr, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr), "l"(g));
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;");
}
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g));
}
__device__ __forceinline__ uint4 lds128(uint32_t saddr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(saddr));
  return v;
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N));
}
__device__ __forceinline__ uint32_t lds32v(uint32_t saddr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(saddr));
  return v;
}

// Raw-word ring of the FP32 fast loop: kRingBytes of shared memory per thread
// hold the three raw groups' words of the next RD steps of its NS sub-streams
// (4-B pieces), so that RD steps of loads are in flight per thread without
// holding registers.  The 16-bit loops keep their raw words in registers, two
// steps ahead: there the ring's shared memory costs a CTA per SM (W = 12) and
// the loop lost more than it gained.
constexpr uint32_t kRingBytes = 64;
template <int NS>
struct RawRing {
  static constexpr uint32_t per = kRingBytes / (NS * 3u * 4u);
  static constexpr uint32_t RD = per >= 8 ? 8u : (per >= 4 ? 4u : 2u);  // steps in the ring
};

// Fast loop for the dominant chunk layout: group 0 Huffman and staged, every
// other group raw, zero or constant, a whole chunk whose nvec vectors split evenly over the T
// sub-streams, and T a multiple of NS * nthr.  Thread t decodes sub-streams
// t, t + nthr, ... (NS in lockstep, interleaved for instruction-level
// parallelism); every vector is 16 B of output: V/2 pair lookups, the raw
// groups' words (16-bit: loaded two steps ahead into alternating register
// sets; FP32: from the thread's ring, copied RD steps ahead), bit-select merge
// with the rotated exponent symbols, a 16-B store.  No mode tests and no tails
// inside the loop.  Each sub-stream must end exactly where the next one starts
// (the last one within the bitstream); a mismatch flags the chunk as corrupt.
// The loop covers the sub-streams [t_lo, t_hi) of the chunk (all of them, or
// one part of a chunk split over several work items), t_hi - t_lo a multiple
// of NS * nthr.
template <int DT, int W, int NS, bool SPLIT>
__device__ __forceinline__ void decode_fast(const Job& J, uint64_t c, const Smem& S,
                                            const Staging& stg, uint32_t* err, uint32_t t_lo,
                                            uint32_t t_hi) {
  constexpr int G = Traits<DT>::G, V = Traits<DT>::V;
  constexpr int RW = DT == ZIPNN_FP32 ? 3 : (DT == ZIPNN_U8 ? 1 : 2);
  constexpr bool RING = DT == ZIPNN_FP32;
  constexpr uint32_t RD = RawRing<NS>::RD;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const ChunkInfo& CI = S.ci;
  const uint64_t off0 = c * J.chunk_bytes;
  const uint32_t T = J.lanes;
  const uint32_t nper = (J.chunk_bytes / 16u) / T;
  const uint8_t* pay = stg.base + CI.staged[0];
  const uint32_t* starts = reinterpret_cast<const uint32_t*>(pay + (uint32_t)CI.offs[0]);
  const uint32_t* words = reinterpret_cast<const uint32_t*>(pay + (uint32_t)CI.bs[0]);
  const uint32_t nwords = CI.nwords[0], nbits = nwords * 32u, wlim = nwords + 1u;
  const uint32_t lut = smem_u32(S.lut_ptr[0]);
  const GroupTab& tb = S.tab[0];
  const uint8_t* syms = reinterpret_cast<const uint8_t*>(tb.words) + 12;
  const uint8_t* rawp[G];
  uint32_t cw[G], rawm = 0;
#pragma unroll
  for (int g = 0; g < G; g++) {
    rawp[g] = J.src + CI.payload[g];
    cw[g] = CI.value[g] * 0x01010101u;  // ZERO groups carry value 0
    if (CI.mode[g] == kRaw) rawm |= 1u << g;
  }
  uint4* dst = reinterpret_cast<uint4*>(J.dst + off0);
  const uint4* base = J.base ? reinterpret_cast<const uint4*>(J.base + off0) : nullptr;
  const uint8_t* base8 = J.base ? J.base + off0 : nullptr;
  // FP32 ring: this thread's piece q of sub-stream j in slot sl is at
  // ring + ((sl * NS + j) * 3 + q) * rstride
  const uint32_t ring = stg.ring + (uint32_t)tid * 4u;
  const uint32_t rstride = (uint32_t)nthr * 4u;
  uint32_t bad = 0;
  // L2 prefetch window; steps [0, D) were requested when the chunk was set up.
  // Lane 0 of warp (k / 2) mod (warps) requests steps k + D and k + D + 1.
  // FP32 only: in the 16-bit kernels the extra live registers cost the loop
  // more than the later prefetches gain (the first window stays).
  const bool pfl = DT == ZIPNN_FP32 && (tid & 31) == 0 && T == (uint32_t)(NS * nthr);
  const uint32_t wid = (uint32_t)tid >> 5, wmask = ((uint32_t)nthr >> 5) - 1u;
  const uint32_t D = pfl ? pf_steps<G>(rawm, base8 != nullptr, T, nper, stg.pf_bytes) : 0u;
  const uint32_t t_begin = SPLIT ? t_lo : 0u, t_end = SPLIT ? t_hi : T;
  for (uint32_t t0 = t_begin + tid; t0 < t_end; t0 += NS * nthr) {
    // window w1:w0 (bit pos of w0 first); with PRE, wn is the word after it,
    // read one refill ahead so that a refill only moves registers: in the
    // 128-thread kernels, the FP16 ones (two 256-thread CTAs per SM) and FP32
    // (one sub-stream per thread); the BF16 256-thread kernel cannot spare the
    // registers at three CTAs per SM (2965 -> 2503 GB/s on the checkpoint,
    // from spills) and loses more than PRE gains at two (2541)
    constexpr bool PRE = SPLIT || DT == ZIPNN_FP16 || DT == ZIPNN_FP32;
    uint32_t w0[NS], w1[NS], wn[NS], pos[NS], idx[NS], vt[NS];
    uint32_t ra[NS][RW], rb[NS][RW];  // 16-bit: raw words of vectors k (even) and k + 1
    // FP32: raw words of step k into ring slot k mod RD (always one commit
    // group per step, empty past the end, so that step k has landed when at
    // most RD - 1 groups are pending)
    auto issue = [&](uint32_t k) {
      if (k < nper) {
        const uint32_t sl = (k & (RD - 1u)) * NS;
#pragma unroll
        for (int j = 0; j < NS; j++) {
          const uint32_t v = vt[j] + k * T;
#pragma unroll
          for (int q = 0; q < 3; q++)
            if ((rawm >> (q + 1)) & 1u)
              cp_async4(ring + ((sl + j) * 3u + q) * rstride, rawp[q + 1] + 4ull * v);
        }
      }
      cp_async_commit();
    };
#pragma unroll
    for (int j = 0; j < NS; j++) {
      const uint32_t t = t0 + j * nthr;
      vt[j] = t;
      uint32_t start = t ? starts[t - 1] : 0u;
      if (start > nbits) {
        bad = 1;
        start = nbits;
      }
      idx[j] = start >> 5;
      pos[j] = start & 31u;
      w0[j] = words[min(idx[j], wlim)];
      w1[j] = words[min(idx[j] + 1u, wlim)];
      if constexpr (PRE) wn[j] = words[min(idx[j] + 2u, wlim)];
      idx[j] += PRE ? 3 : 2;
      if constexpr (!RING) {
        load_raw_vec<DT>(rawp, rawm, cw, t, ra[j]);
        if (nper > 1) load_raw_vec<DT>(rawp, rawm, cw, t + T, rb[j]);
      }
    }
    if constexpr (RING) {
#pragma unroll
      for (uint32_t k = 0; k < RD; k++) issue(k);
    }
    // vector k of every sub-stream; 16-bit: rr holds its raw words and
    // receives those of vector k + 2
    auto vec = [&](uint32_t k, uint32_t (&rr)[NS][RW]) {
      uint32_t ex[NS][V / 4];
#pragma unroll
      for (int q = 0; q < V / 4; q++) {
        uint32_t h[2][NS];
#pragma unroll
        for (int p = 0; p < 2; p++) {
#pragma unroll
          for (int j = 0; j < NS; j++) {
            const uint32_t e = pair_at<W>(__funnelshift_l(w1[j], w0[j], pos[j]), lut, tb, syms, bad);
            pos[j] += e >> 27;
            if (pos[j] >= 32u) {
              pos[j] -= 32u;
              w0[j] = w1[j];
              if constexpr (PRE) {
                w1[j] = wn[j];
                wn[j] = words[min(idx[j], wlim)];
              } else {
                w1[j] = words[min(idx[j], wlim)];
              }
              idx[j]++;
            }
            h[p][j] = e;
          }
        }
#pragma unroll
        for (int j = 0; j < NS; j++) ex[j][q] = __byte_perm(h[0][j], h[1][j], 0x5410);
      }
      if constexpr (RING) {
        // this thread's copies of step k have landed
        cp_async_wait<RD - 1>();
        const uint32_t sl = (k & (RD - 1u)) * NS;
#pragma unroll
        for (int j = 0; j < NS; j++)
#pragma unroll
          for (int q = 0; q < 3; q++)
            rr[j][q] = ((rawm >> (q + 1)) & 1u) ? lds32v(ring + ((sl + j) * 3u + q) * rstride)
                                               : cw[q + 1];
      }
#pragma unroll
      for (int j = 0; j < NS; j++) {
        const uint32_t v = vt[j] + k * T;
        uint32_t x[4];
        if constexpr (DT == ZIPNN_FP32) {
          merge32r(ex[j][0], rr[j][0], rr[j][1], rr[j][2], x);
        } else if constexpr (DT == ZIPNN_U8) {
          x[0] = ex[j][0]; x[1] = ex[j][1]; x[2] = ex[j][2]; x[3] = ex[j][3];
        } else {
          merge16r(ex[j][0], rr[j][0], x[0], x[1]);
          merge16r(ex[j][1 % (V / 4)], rr[j][1 % RW], x[2], x[3]);
        }
        if constexpr (!RING)
          if (k + 2 < nper) load_raw_vec<DT>(rawp, rawm, cw, v + 2 * T, rr[j]);
        if (base) {
          const uint4 bb = __ldg(base + v);
          x[0] ^= bb.x; x[1] ^= bb.y; x[2] ^= bb.z; x[3] ^= bb.w;
        }
        dst[v] = make_uint4(x[0], x[1], x[2], x[3]);
      }
      // FP32: the slot is free again (its words were consumed above)
      if constexpr (RING) issue(k + RD);
    };
    for (uint32_t k = 0; k < nper; k += 2) {
      if (DT == ZIPNN_FP32 && pfl && ((k >> 1) & wmask) == wid && k + D < nper)
        prefetch_steps<G>(rawp, rawm, base8, T, k + D, min(k + D + 2u, nper));
      vec(k, ra);
      if (k + 1 < nper) vec(k + 1, rb);
    }
    if constexpr (RING) cp_async_wait<0>();
    // every sub-stream ends where the next begins
#pragma unroll
    for (int j = 0; j < NS; j++) {
      const uint32_t end = (idx[j] - (PRE ? 3u : 2u)) * 32u + pos[j];
      if (vt[j] + 1u < T) bad |= end != starts[vt[j]];
      else bad |= end > nbits;
    }
  }
  if (bad) atomicOr(err, 1u);
}

// A staged coded group (HUFF or SPARSE) and the reader of one of its
// sub-streams, as the fast loop sees them.
struct FastGroup {
  const uint32_t* words;   // bitstream (shared memory)
  const uint32_t* starts;  // start bits of sub-streams 1..T-1
  const uint32_t* bm;      // SPARSE: bitmap of the vectors holding a non-zero symbol
  uint32_t nbits, wlim, lut;
  bool sparse;
};
struct FastReader {
  uint32_t w0, w1, pos, idx;
};

// Two symbols of reader r (one pair lookup, refill clamped to the payload).
template <int W>
__device__ __forceinline__ uint32_t fast_pair(const FastGroup& F, FastReader& r, const GroupTab& tb,
                                              uint32_t& bad) {
  const uint8_t* syms = reinterpret_cast<const uint8_t*>(tb.words) + 12;
  const uint32_t e = pair_at<W>(__funnelshift_l(r.w1, r.w0, r.pos), F.lut, tb, syms, bad);
  r.pos += e >> 27;
  if (r.pos >= 32u) {
    r.pos -= 32u;
    r.w0 = r.w1;
    r.w1 = F.words[min(r.idx, F.wlim)];
    r.idx++;
  }
  return e;
}

// fast_pair for a SPARSE group without a branch on the vector's bitmap bit:
// every lane looks up the window at its position, and only lanes whose
// vector holds a non-zero symbol (live) advance, report invalid codes and
// keep the symbols (the warp's 32 vectors share one bitmap word, so a branch
// would make the warp run both sides whenever its vectors mix).
template <int W>
__device__ __forceinline__ uint32_t fast_pair_if(const FastGroup& F, FastReader& r,
                                                 const GroupTab& tb, uint32_t& bad, bool live) {
  const uint8_t* syms = reinterpret_cast<const uint8_t*>(tb.words) + 12;
  uint32_t b2 = 0;
  const uint32_t e = pair_at<W>(__funnelshift_l(r.w1, r.w0, r.pos), F.lut, tb, syms, b2);
  bad |= live ? b2 : 0u;
  r.pos += live ? (e >> 27) : 0u;
  if (r.pos >= 32u) {
    r.pos -= 32u;
    r.w0 = r.w1;
    r.w1 = F.words[min(r.idx, F.wlim)];
    r.idx++;
  }
  return live ? e : 0u;
}

// Fast loop for the other layouts of deltas, clean and pruned models: group 0
// coded (HUFF or SPARSE) and staged; with NC = 2 (16-bit dtypes)
// group 1 coded and staged too, else every group after the first raw, zero or
// constant; a whole chunk whose nvec vectors split evenly over the T
// sub-streams, and T a multiple of NS * nthr.  Thread t decodes sub-streams
// t, t + nthr, ... (NS in lockstep, interleaved for instruction-level
// parallelism); every vector is 16 B of output: V/2 pair lookups per coded
// group (none for an all-zero vector of a SPARSE group), one load per raw
// group (two vectors ahead), the base from a per-thread ring of asynchronous
// copies (RB steps ahead, and in L2 D steps ahead), bit-select merge with the
// rotated exponent
// symbols, a 16-B store.  No per-vector mode tests and no tails inside the
// loop.  Each sub-stream must end exactly where the next one starts (the last
// one within the bitstream); a mismatch flags the chunk as corrupt.
template <int DT, int W, int NS, int NC>
__device__ __forceinline__ void decode_fast_coded(const Job& J, uint64_t c, const Smem& S,
                                            const Staging& stg, uint32_t* err) {
  constexpr int G = Traits<DT>::G, V = Traits<DT>::V;
  constexpr int RW = DT == ZIPNN_FP32 ? 3 : (DT == ZIPNN_U8 ? 1 : 2);
  static_assert(NC == 1 || (NC == 2 && G == 2), "two coded groups: 16-bit dtypes only");
  const int tid = threadIdx.x, nthr = blockDim.x;
  const ChunkInfo& CI = S.ci;
  const uint64_t off0 = c * J.chunk_bytes;
  const uint32_t T = J.lanes;
  const uint32_t nper = (J.chunk_bytes / 16u) / T;
  FastGroup F[NC];
#pragma unroll
  for (int g = 0; g < NC; g++) {
    const uint8_t* pay = stg.base + CI.staged[g];
    F[g].words = reinterpret_cast<const uint32_t*>(pay + (uint32_t)CI.bs[g]);
    F[g].starts = reinterpret_cast<const uint32_t*>(pay + (uint32_t)CI.offs[g]);
    F[g].bm = reinterpret_cast<const uint32_t*>(pay + (uint32_t)CI.bmo[g]);
    F[g].sparse = CI.mode[g] == kSparse;
    F[g].nbits = CI.nwords[g] * 32u;
    F[g].wlim = CI.nwords[g] + 1u;
    F[g].lut = smem_u32(S.lut_ptr[g]);
  }
  const uint8_t* rawp[G];
  uint32_t cw[G], rawm = 0;
#pragma unroll
  for (int g = 0; g < G; g++) {
    rawp[g] = J.src + CI.payload[g];
    cw[g] = CI.value[g] * 0x01010101u;  // ZERO groups carry value 0
    if (g >= NC && CI.mode[g] == kRaw) rawm |= 1u << g;
  }
  uint4* dst = reinterpret_cast<uint4*>(J.dst + off0);
  const uint4* base = J.base ? reinterpret_cast<const uint4*>(J.base + off0) : nullptr;
  const uint8_t* base8 = J.base ? J.base + off0 : nullptr;
  uint32_t bad = 0;
  // delta base through a per-thread ring of 16-B asynchronous copies (RB steps
  // ahead; slot sl, sub-stream j at ring + ((sl * NS + j) * nthr + tid) * 16)
  constexpr uint32_t RB = kRingBytes / (NS * 16u) >= 4 ? 4u : 2u;
  const uint32_t bring = stg.ring + (uint32_t)tid * 16u;
  const uint32_t bstride = (uint32_t)nthr * 16u;
  // L2 prefetch window; steps [0, D) were requested when the chunk was set up.
  // Lane 0 of warp (k / 2) mod (warps) requests steps k + D and k + D + 1.
  const bool pfl = (tid & 31) == 0 && T == (uint32_t)(NS * nthr);
  const uint32_t wid = (uint32_t)tid >> 5, wmask = ((uint32_t)nthr >> 5) - 1u;
  const uint32_t D = pfl ? pf_steps<G>(rawm, base8 != nullptr, T, nper, stg.pf_bytes) : 0u;
  for (uint32_t t0 = tid; t0 < T; t0 += NS * nthr) {
    FastReader R[NC][NS];
    uint32_t vt[NS];
    uint32_t ra[NS][RW], rb[NS][RW];  // raw words of vectors k (even) and k + 1
#pragma unroll
    for (int j = 0; j < NS; j++) {
      const uint32_t t = t0 + j * nthr;
      vt[j] = t;
#pragma unroll
      for (int g = 0; g < NC; g++) {
        uint32_t start = t ? F[g].starts[t - 1] : 0u;
        if (start > F[g].nbits) {
          bad = 1;
          start = F[g].nbits;
        }
        FastReader& r = R[g][j];
        r.idx = start >> 5;
        r.pos = start & 31u;
        r.w0 = F[g].words[min(r.idx, F[g].wlim)];
        r.w1 = F[g].words[min(r.idx + 1u, F[g].wlim)];
        r.idx += 2;
      }
      if constexpr (NC == 1) {
        load_raw_vec<DT>(rawp, rawm, cw, t, ra[j]);
        if (nper > 1) load_raw_vec<DT>(rawp, rawm, cw, t + T, rb[j]);
      }
    }
    // base words of step k into ring slot k mod RB (one commit group per step)
    auto issue_base = [&](uint32_t k) {
      if (k < nper) {
        const uint32_t sl = (k & (RB - 1u)) * NS;
#pragma unroll
        for (int j = 0; j < NS; j++)
          cp_async16(bring + (sl + j) * bstride, base8 + 16ull * (vt[j] + k * T));
      }
      cp_async_commit();
    };
    if (base) {
#pragma unroll
      for (uint32_t k = 0; k < RB; k++) issue_base(k);
    }
    // vector k of every sub-stream; rr holds its raw words and receives those
    // of vector k + 2
    auto vec = [&](uint32_t k, uint32_t (&rr)[NS][RW]) {
      uint32_t ex[NC][NS][V / 4];
#pragma unroll
      for (int g = 0; g < NC; g++) {
        bool coded[NS];
#pragma unroll
        for (int j = 0; j < NS; j++) coded[j] = true;
        if (F[g].sparse) {  // uniform per chunk
#pragma unroll
          for (int j = 0; j < NS; j++) {
            const uint32_t v = vt[j] + k * T;
            coded[j] = (F[g].bm[v >> 5] >> (v & 31u)) & 1u;
          }
        }
#pragma unroll
        for (int q = 0; q < V / 4; q++) {
          uint32_t h[2][NS];
#pragma unroll
          for (int p = 0; p < 2; p++) {
#pragma unroll
            for (int j = 0; j < NS; j++) {
              if (F[g].sparse)
                h[p][j] = fast_pair_if<W>(F[g], R[g][j], S.tab[g], bad, coded[j]);
              else
                h[p][j] = fast_pair<W>(F[g], R[g][j], S.tab[g], bad);
            }
          }
#pragma unroll
          for (int j = 0; j < NS; j++) ex[g][j][q] = __byte_perm(h[0][j], h[1][j], 0x5410);
        }
      }
      // this thread's base copies of step k have landed
      if (base) cp_async_wait<RB - 1>();
#pragma unroll
      for (int j = 0; j < NS; j++) {
        const uint32_t v = vt[j] + k * T;
        uint32_t x[4];
        if constexpr (NC == 2) {
          merge16r(ex[0][j][0], ex[1][j][0], x[0], x[1]);
          merge16r(ex[0][j][1], ex[1][j][1], x[2], x[3]);
        } else if constexpr (DT == ZIPNN_FP32) {
          merge32r(ex[0][j][0], rr[j][0], rr[j][1], rr[j][2], x);
        } else if constexpr (DT == ZIPNN_U8) {
          x[0] = ex[0][j][0]; x[1] = ex[0][j][1]; x[2] = ex[0][j][2]; x[3] = ex[0][j][3];
        } else {
          merge16r(ex[0][j][0], rr[j][0], x[0], x[1]);
          merge16r(ex[0][j][1 % (V / 4)], rr[j][1 % RW], x[2], x[3]);
        }
        if constexpr (NC == 1)
          if (k + 2 < nper) load_raw_vec<DT>(rawp, rawm, cw, v + 2 * T, rr[j]);
        if (base) {
          const uint4 bb = lds128(bring + ((k & (RB - 1u)) * NS + j) * bstride);
          x[0] ^= bb.x; x[1] ^= bb.y; x[2] ^= bb.z; x[3] ^= bb.w;
        }
        dst[v] = make_uint4(x[0], x[1], x[2], x[3]);
      }
      // the base slot is free again: step k + RB
      if (base) issue_base(k + RB);
    };
    for (uint32_t k = 0; k < nper; k += 2) {
      if (pfl && ((k >> 1) & wmask) == wid && k + D < nper)
        prefetch_steps<G>(rawp, rawm, base8, T, k + D, min(k + D + 2u, nper));
      vec(k, ra);
      if (k + 1 < nper) vec(k + 1, rb);
    }
    if (base) cp_async_wait<0>();
    // every sub-stream ends where the next begins
#pragma unroll
    for (int g = 0; g < NC; g++)
#pragma unroll
      for (int j = 0; j < NS; j++) {
        const FastReader& r = R[g][j];
        const uint32_t end = (r.idx - 2u) * 32u + r.pos;
        if (vt[j] + 1u < T) bad |= end != F[g].starts[vt[j]];
        else bad |= end > F[g].nbits;
      }
  }
  if (bad) atomicOr(err, 1u);
}

// The generic loop out of line (kernels without the general fast loops).
template <int DT, int W, class BR, bool STAGED, int NS>
__device__ __noinline__ void decode_loop_ool(const Job& J, uint64_t c, Smem& S, Staging& stg,
                                             uint32_t* err) {
  decode_loop<DT, W, BR, STAGED, NS>(J, c, S, stg, err);
}

// Every layout but the Huffman loop of model weights, behind one out-of-line
// call (one call site keeps the register allocation of the kernel's hot path
// as it is): the general fast loop (SPARSE group 0, or two coded groups), else
// the generic loop over staged or global payloads.
template <int DT, int W>
__device__ __noinline__ void decode_other(const Job& J, uint64_t c, Smem& S, Staging& stg,
                                          uint32_t* err, int fast, int fast_nc) {
  constexpr int G = Traits<DT>::G;
  const uint32_t T = J.lanes;
  const int nthr = blockDim.x;
  if constexpr (W >= 11) {
    if (fast_nc == 2) {
      if constexpr (G == 2) {
        if (fast == 2) return decode_fast_coded<DT, W, 2, 2>(J, c, S, stg, err);
        if (fast == 1) return decode_fast_coded<DT, W, 1, 2>(J, c, S, stg, err);
      }
    } else {
      if (fast == 2) return decode_fast_coded<DT, W, 2, 1>(J, c, S, stg, err);
      if (fast == 1) return decode_fast_coded<DT, W, 1, 1>(J, c, S, stg, err);
    }
  }
  if (S.ci.stage_bytes) {
    if (T >= 2u * nthr) decode_loop<DT, W, SmemBitReader, true, 2>(J, c, S, stg, err);
    else decode_loop<DT, W, SmemBitReader, true, 1>(J, c, S, stg, err);
  } else {
    decode_loop<DT, W, BitReader, false, 1>(J, c, S, stg, err);
  }
}

// Decode one chunk of a tensor of dtype DT with W-bit pair tables.  Returns
// false if a bulk copy never completed (the caller must stop using the stage).
// Shared memory: one table slot (lut0) for the first Huffman group; tables of
// further Huffman groups and the staged payloads share the stage.
// With parts > 1 the chunk is one of `parts` work items (part = 0..parts-1):
// a chunk of the dominant layout (below) whose T sub-streams split into
// `parts` ranges that each fill whole rounds of the CTA's threads is decoded
// range by range, part p doing sub-streams [p T / parts, (p+1) T / parts)
// (each part stages the chunk's payload and builds its table); any other
// chunk is decoded whole by part 0, and the other parts leave after reading
// its map entries.
// (SPLIT: compiled into the 128-thread kernels only, the ones split launches
// use; the other kernels keep parts = 1 and their register allocation.)
template <int DT, int W, bool GEN, bool SPLIT>
__device__ bool decode_chunk(const Job& J, uint64_t c, Smem& S, uint32_t* lut0, Staging& stg,
                             uint32_t* err, uint32_t part, uint32_t parts) {
  if constexpr (!SPLIT) {
    part = 0;
    parts = 1;
  }
  constexpr int G = Traits<DT>::G, V = Traits<DT>::V, ES = 16 / V;
  constexpr int kLut = 1 << W;
  constexpr uint32_t kLutBytes = 4u << W;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const uint64_t off0 = c * J.chunk_bytes;
  const uint64_t nb = min((uint64_t)J.chunk_bytes, J.nbytes - off0);
  const uint64_t m = nb / ES;
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
    if (mode > kSparse || po > avail || align_up(size, 16) > avail - po || (po & 15)) bad = 1;
    if (mode == kRaw && size != m) bad = 1;
    if ((mode == kZero || mode == kConst) && size != 0) bad = 1;
    if ((mode == kHuff || mode == kSparse) && size < 12) bad = 1;
    CI.mode[tid] = bad ? kZero : mode;
    CI.value[tid] = value;
    CI.size[tid] = size;
    CI.payload[tid] = P + po;
    if (bad) atomicOr(&CI.bad, 1u);
  }
  __syncthreads();
  if (CI.bad) {
    if (tid == 0 && part == 0) atomicOr(err, 1u);
    return true;
  }
  // 1b. split over parts: only the dominant layout of model weights (group 0
  // HUFF and stageable, the others raw, zero or constant, a whole chunk, the
  // parts' sub-stream ranges whole rounds of the CTA's threads); this is
  // decided before any bulk copy is issued, so a part that leaves has none
  // in flight
  bool split = false;
  if (SPLIT && parts > 1) {
    if constexpr (SPLIT && W >= 11 && !GEN) {
      bool ok = CI.mode[0] == kHuff && nb == J.chunk_bytes && ((uint32_t)(nb / 16) % T) == 0 &&
                T % parts == 0 && ((T / parts) % (uint32_t)nthr) == 0 &&
                align_up(CI.size[0], 16) + 32 <= stg.cap;
#pragma unroll
      for (int g = 1; g < G; g++) ok = ok && !coded_mode(CI.mode[g]);
      split = ok;
    }
    if (!split && part != 0) return true;  // part 0 decodes the whole chunk
  }
  const uint32_t t_lo = SPLIT && split ? part * (T / parts) : 0u;
  const uint32_t t_hi = SPLIT && split ? t_lo + T / parts : T;
  const uint32_t Tp = t_hi - t_lo;
  // 2. placement of tables and payloads; thread 0 issues the bulk copies
  if (tid == 0) {
    uint32_t nhuff = 0, pay_total = 0;
    for (int g = 0; g < G; g++)
      if (coded_mode(CI.mode[g])) {
        nhuff++;
        pay_total += (uint32_t)align_up(CI.size[g], 16);
      }
    const uint32_t extra = nhuff > 1 ? (nhuff - 1) * kLutBytes : 0u;
    // an FP32 chunk with several coded groups takes no fast loop, so the
    // raw-word rings after the stage are free for its tables (the launch
    // sizes stage + rings for three more tables, the stage alone for one)
    const uint32_t tcap = stg.cap + ((G == 4 && nhuff > 1) ? stg.ring_bytes : 0u);
    // (the tables start at the first 128-B boundary after the payloads + 32 B)
    const bool stage_payloads = nhuff && ((pay_total + 32u + 127u) & ~127u) + extra <= tcap;
    uint32_t used = 0, k = 0;
    for (int g = 0; g < G; g++) {
      CI.staged[g] = 0xFFFFFFFFu;
      S.lut_ptr[g] = lut0;
      if (!coded_mode(CI.mode[g])) continue;
      if (stage_payloads) {
        CI.staged[g] = used;
        used += (uint32_t)align_up(CI.size[g], 16);
      }
      if (k++) S.lut_ptr[g] = nullptr;  // placed after the staged payloads below
    }
    CI.stage_bytes = used;
    uint32_t lo = (used + 32 + 127) & ~127u;
    for (int g = 0; g < G; g++)
      if (coded_mode(CI.mode[g]) && S.lut_ptr[g] == nullptr) {
        if (lo + kLutBytes > tcap) {  // cannot happen with the launch's sizing; fail closed
          CI.bad = 1;
          lo = 0;
        }
        S.lut_ptr[g] = reinterpret_cast<uint32_t*>(stg.base + lo);
        lo += kLutBytes;
      }
    if (used) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(stg.bar, used + stg.extra_tx);
      for (int g = 0; g < G; g++)
        if (CI.staged[g] != 0xFFFFFFFFu)
          bulk_g2s(stg.base + CI.staged[g], cont + CI.payload[g],
                   (uint32_t)align_up(CI.size[g], 16), stg.bar);
    }
  }
  // 3a. table bytes of every Huffman group (word loads, clamped to the payload)
#pragma unroll
  for (int g = 0; g < G; g++) {
    if (!coded_mode(CI.mode[g])) continue;
    const uint8_t* p = cont + CI.payload[g];
    for (int i = tid; i < 68; i += nthr)
      S.tab[g].words[i] = (4u * i + 4u <= CI.size[g]) ? rd_u32(p + 4 * i) : 0u;
  }
  __syncthreads();
  // 3b. canonical limits (thread g), validation
  if (tid < G && coded_mode(CI.mode[tid])) {
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
    // SPARSE: the vector bitmap (one bit per 16-byte vector of the chunk)
    // sits between the table and the start-bit table
    const uint64_t bmb = CI.mode[tid] == kSparse ? 4ull * ((nb + 511) / 512) : 0ull;
    const uint64_t size = CI.size[tid];
    const uint64_t hdr = h + bmb + 4ull * (T - 1);
    if (nz < 2 || nz > 256 || kraft > (uint32_t)kLutSize || size < hdr || (size - hdr) % 4) {
      atomicOr(&CI.bad, 1u);
    } else {
      CI.bmo[tid] = h;
      CI.offs[tid] = h + bmb;
      CI.bs[tid] = hdr;
      CI.nwords[tid] = (uint32_t)((size - hdr) / 4);
    }
  }
  __syncthreads();
  const bool bad_tab = CI.bad != 0;
  // fast loop (decode_fast) when the chunk has its layout; symbols are then
  // stored rotated in the table
  // fast = sub-streams per thread of a fast loop (0: generic loop), fast_nc =
  // coded groups in front (2: both groups of a 16-bit delta or clean model)
  int fast = 0, fast_nc = 1;
  if constexpr (W >= 11) {
    // without GEN only the Huffman loop of model weights is a fast loop
    bool ok = (GEN ? coded_mode(CI.mode[0]) : CI.mode[0] == kHuff) && CI.staged[0] != 0xFFFFFFFFu &&
              nb == J.chunk_bytes && ((uint32_t)(nb / 16) % T) == 0;
    if (GEN && G == 2 && coded_mode(CI.mode[1 % G])) {
      fast_nc = 2;
      ok = ok && CI.staged[1 % G] != 0xFFFFFFFFu;
    }
#pragma unroll
    for (int g = fast_nc; g < G; g++) ok = ok && !coded_mode(CI.mode[g]);
    // one sub-stream per thread for FP32 (its raw words come through the
    // shared-memory ring: 1787 -> 1853 GB/s on a 256 MiB tensor), two for the
    // 16-bit types (one: the checkpoint 2965 -> 2575 GB/s)
    if (ok)
      fast = (DT != ZIPNN_FP32 && Tp % (2u * nthr) == 0) ? 2 : ((Tp % (uint32_t)nthr == 0) ? 1 : 0);
  }
  // exponent symbols are stored rotated for the fast loops' merge
  const bool rot0 = fast != 0 && DT != ZIPNN_U8;
  // the fast loop's first L2 prefetch window, in flight while the tables are
  // built (same raw groups and window as the loop computes)
  if (fast != 0 && tid == 0 && Tp == (uint32_t)(fast * nthr)) {
    const uint8_t* rawp[G];
    uint32_t rawm = 0;
#pragma unroll
    for (int g = 0; g < G; g++) {
      rawp[g] = J.src + CI.payload[g];
      if (g >= fast_nc && CI.mode[g] == kRaw) rawm |= 1u << g;
    }
    const uint8_t* base8 = J.base ? J.base + c * J.chunk_bytes : nullptr;
    const uint32_t nper = (J.chunk_bytes / 16u) / T;
    // the window's steps cover every sub-stream of the chunk: a part of a
    // split chunk requests its share of the steps (the parts run together)
    const uint32_t D = pf_steps<G>(rawm, base8 != nullptr, T, nper, stg.pf_bytes);
    prefetch_steps<G>(rawp, rawm, base8, T, SPLIT && split ? part * D / parts : 0u,
                      SPLIT && split ? (part + 1) * D / parts : D);
  }
  // 3c. pair tables, in two passes.  Pass 1: for window w (W bits) the first
  // code has length l1 = the least l <= W with w < lim_W[l] (W + 1 if none);
  // with W = 11 a first code of 12 bits is resolved in the entry by its last
  // bit.  Each warp fills a contiguous block of the table, lane j the entries
  // j, j + 32, ... of it (conflict-free stores); along a lane w increases and
  // l1 with it, so l1 advances from the previous entry's, with its limit and
  // index[l1] - first[l1] held in registers.  Pass 2: the second code is the
  // first code of window (w << l1) & (2^W - 1) (the remaining W - l1 bits,
  // zero-filled), kept when it fits in them.  Pass 2 reads entries that other
  // threads are turning into pairs; a pair keeps the first code's symbol and
  // length where pass 2 reads them, so either value serves.
  // A chunk split over the CTAs of a cluster (one per part, launched as
  // such) builds its table together: CTA r fills windows [r, r + 1) * 2^W /
  // parts and stores every entry into all the cluster's tables (distributed
  // shared memory, the same offset in each CTA), with a cluster barrier
  // after each pass.  Every CTA of the cluster takes the same path here: the
  // chunk's map and table bytes decide it.
  uint32_t crank = 0, cn = 1;
  if constexpr (SPLIT) {
    if (split) {
      cn = cluster_size();
      crank = cluster_rank();
      if (cn != parts || crank != part) {  // not launched as a cluster of the parts
        cn = 1;
        crank = 0;
      }
    }
  }
  // every CTA of the cluster has started (and finished any earlier chunk's
  // loop, which reads its table) before the first store into a peer
  if (cn > 1) cluster_sync();
  if (!bad_tab) {
    const uint32_t span = (uint32_t)kLut / cn;  // windows of this CTA
    const uint32_t per_w = span / ((uint32_t)nthr >> 5);
    const uint32_t wb = crank * span + ((uint32_t)tid >> 5) * per_w;
    // store e at window w of group g's table in every CTA of the cluster
    auto put_all = [&](uint32_t L, uint32_t w, uint32_t e) {
      sts32(L + 4u * w, e);
      if constexpr (SPLIT) {
        for (uint32_t r = 1; r < cn; r++) st_peer(map_peer(L + 4u * w, (crank + r) % cn), e);
      }
    };
#pragma unroll
    for (int g = 0; g < G; g++) {
      if (!coded_mode(CI.mode[g])) continue;
      const GroupTab& t = S.tab[g];
      const uint8_t* syms = reinterpret_cast<const uint8_t*>(t.words) + 12;
      const bool rot = rot0 && g == 0;
      auto sym = [&](uint32_t r) -> uint32_t {
        const uint32_t v = syms[r & 255];
        return rot ? (((v >> 1) | (v << 7)) & 0xFFu) : v;
      };
      auto lim_of = [&](uint32_t l) -> uint32_t {
        return l <= (uint32_t)W ? (t.lim[l] >> (kMaxLen - W)) : 0xFFFFFFFFu;
      };
      const uint32_t L = smem_u32(S.lut_ptr[g]);
      uint32_t l1 = 1, lcur = lim_of(1), basel = t.index[1] - t.first[1];
      for (uint32_t w = wb + ((uint32_t)tid & 31u); w < wb + per_w; w += 32) {
        if (w >= lcur) {
          do {
            l1++;
            lcur = lim_of(l1);
          } while (w >= lcur);
          basel = l1 <= (uint32_t)W ? t.index[l1] - t.first[l1] : 0u;
        }
        uint32_t ent = 0;
        if (l1 <= (uint32_t)W) {
          const uint32_t r1 = basel + (w >> (W - l1));
          ent = sym(r1) | (l1 << 16) | (l1 << 27);
        } else if (W == 11) {
          // first code of 12 bits: w is its prefix, the next bit selects
          ent = kLong | (12u << 16) | (12u << 27);
#pragma unroll
          for (uint32_t nb = 0; nb < 2; nb++) {
            const uint32_t w12 = ((uint32_t)w << 1) | nb;
            if (w12 < t.lim[kMaxLen])
              ent |= sym(t.index[kMaxLen] + w12 - t.first[kMaxLen]) << (8 * nb);
            else
              ent |= kBadLong0 << nb;
          }
        }
        put_all(L, w, ent);
      }
    }
    if (cn > 1) cluster_sync();
    else __syncthreads();
#pragma unroll
    for (int g = 0; g < G; g++) {
      if (!coded_mode(CI.mode[g])) continue;
      const uint32_t L = smem_u32(S.lut_ptr[g]);
      for (uint32_t w = crank * span + (uint32_t)tid; w < (crank + 1) * span; w += (uint32_t)nthr) {
        const uint32_t e = lds32(L + 4u * w);
        const uint32_t l1 = (e >> 16) & 15u;
        if (l1 == 0 || l1 >= (uint32_t)W) continue;  // invalid, long, or no room left
        const uint32_t e2 = lds32(L + 4u * ((w << l1) & (kLut - 1)));
        const uint32_t l2 = (e2 >> 16) & 15u;
        if (l2 == 0 || l1 + l2 > (uint32_t)W) continue;
        put_all(L, w, (e & 0x000F00FFu) | ((e2 & 0xFFu) << 8) | ((l1 + l2) << 27) | kPair);
      }
    }
    if (cn > 1) cluster_sync();
  }
  // wait for the staged payloads (every thread; bounded)
  uint32_t timed_out = 0;
  if (CI.stage_bytes) {
    if (!mbar_wait(stg.bar, stg.parity, stg.limit_ns)) timed_out = 1;
    stg.parity ^= 1u;
  }
  if (timed_out) atomicOr(&CI.bad, 2u);
  __syncthreads();
  if (CI.bad & 2u) {
    // The wait gave up (ETIMEOUT).  Before the CTA leaves, drain the copies it
    // issued, so that none of them can still write into this shared memory:
    // thread 0 first cancels the bytes that were expected but never requested
    // (the test-only fault injection), so the phase completes exactly when the
    // real copies have landed; then every thread waits for it, again bounded.
    // Only copies that themselves never finish end this second wait by its
    // limit, and then the drain is best effort.
    if (tid == 0) {
      atomicOr(err, 4u);
      if (stg.extra_tx) mbar_complete_tx(stg.bar, stg.extra_tx);
    }
    __syncthreads();
    mbar_wait(stg.bar, stg.parity ^ 1u, stg.limit_ns);
    return false;
  }
  if (bad_tab) {
    if (tid == 0) atomicOr(err, 1u);
    return true;
  }
  // 4. decode + merge: the Huffman loop of model weights inline, the rest out
  // of line.  Kernels for launches with deltas (GEN) add the general fast
  // loops; merely linking them into a kernel costs the inline Huffman loop a
  // third of its speed (register allocation), so the other kernels keep the
  // generic loop alone behind their out-of-line calls.
  if constexpr (W >= 11) {
    if (fast_nc == 1 && CI.mode[0] == kHuff) {
      if (fast == 2) {
        decode_fast<DT, W, 2, SPLIT>(J, c, S, stg, err, t_lo, t_hi);
        return true;
      }
      if (fast == 1) {
        decode_fast<DT, W, 1, SPLIT>(J, c, S, stg, err, t_lo, t_hi);
        return true;
      }
    }
  }
  if constexpr (GEN) {
    decode_other<DT, W>(J, c, S, stg, err, fast, fast_nc);
  } else if (CI.stage_bytes) {
    if (T >= 2u * nthr) decode_loop_ool<DT, W, SmemBitReader, true, 2>(J, c, S, stg, err);
    else decode_loop_ool<DT, W, SmemBitReader, true, 1>(J, c, S, stg, err);
  } else {
    decode_loop_ool<DT, W, BitReader, false, 1>(J, c, S, stg, err);
  }
  return true;
}

// DTS: the dtype of every job in the launch, or -1 for a mixed batch.
// 256-thread CTAs: three per SM (80 registers) for the model-weight kernels;
// two (128 registers) for the GEN kernels, whose delta loops decode two coded
// groups and spill at 80, and for FP16, whose exponent codes are long (most
// lookups take the two-step path) and which gains from the refill preload
// (1408 -> 1523 GB/s on a 256 MiB tensor).
template <int DTS, int W, int NT, bool GEN>
__global__ void __launch_bounds__(NT, NT == 256 ? ((GEN || DTS == ZIPNN_FP16) ? 2 : 3) : 1)
k_decode(JobRef jr, uint64_t nchunks_total, uint32_t* __restrict__ err,
         unsigned long long* __restrict__ ticket, uint32_t debug_flags, uint32_t stage_cap,
         uint32_t pf_bytes, uint32_t parts) {
  extern __shared__ __align__(128) uint8_t dsm[];  // [table slot 0] | stage
  __shared__ Smem S;
  __shared__ uint64_t bar;
  uint32_t* lut0 = reinterpret_cast<uint32_t*>(dsm);
  Staging stg;
  stg.base = dsm + (4u << W);
  stg.cap = stage_cap;
  stg.pf_bytes = pf_bytes;
  stg.ring = smem_u32(dsm + (4u << W) + stage_cap);
  {
    uint32_t dyn;  // the launch's dynamic shared memory: table slot | stage | rings
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    stg.ring_bytes = dyn - (4u << W) - stage_cap;
  }
  stg.bar = &bar;
  stg.parity = 0;
  // debug flag 1 (tests only): expect 16 bytes more than the bulk copies send,
  // so the wait can only end by its (shortened) limit -> ETIMEOUT
  stg.extra_tx = (debug_flags & 1u) ? 16u : 0u;
  stg.limit_ns = (debug_flags & 1u) ? 100000000ull : kWaitLimitNs;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar);
    S.job = 0;
  }
  __syncthreads();
  for (uint64_t iter = 0;; iter++) {
    // work item, from the device queue (batched form) or a static stride, and
    // its job: thread 0 alone finds both and publishes them before the
    // barrier; S.chunk and S.job are read by the others only after it, and
    // written again only after the barrier that ends the iteration.  Work
    // items come in increasing order, so the job is found by scanning forward
    // from the previous item's job (a few steps; after eight, a search).
    if (tid == 0) {
      // work item -> chunk (and, below, the part of a chunk split over
      // `parts` items; parts = 1 but for launches with few chunks)
      const uint64_t itm = ticket ? atomicAdd(ticket, 1ull) : blockIdx.x + iter * gridDim.x;
      const uint32_t np = (NT == kDecThreads && DTS >= 0) ? parts : 1u;  // split: 128 threads, one dtype
      const uint64_t ch = np > 1 ? itm / np : itm;
      S.part = np > 1 ? (uint32_t)(itm - ch * np) : 0u;
      int jj = 0;
      if (jr.table && ch < nchunks_total) {
        jj = S.job;
        int steps = 0;
        while (jj + 1 < jr.n && jr.table[jj + 1].chunk_begin <= ch && steps < 8) {
          jj++;
          steps++;
        }
        if (steps == 8) jj += find_job(jr.table + jj, jr.n - jj, ch);
      }
      S.chunk = ch;
      S.job = jj;
    }
    __syncthreads();
    const uint64_t chunk = S.chunk;
    if (chunk >= nchunks_total) break;
    const int j = S.job;
    const Job& J = jr.table ? jr.table[j] : jr.one;
    const uint64_t c = chunk - J.chunk_begin + J.chunk0;
    const uint32_t part = S.part;
    // split work items (and the fast loops' deeper lookahead): 128-thread
    // kernels of one dtype (mixed launches are never split)
    constexpr bool SP = NT == kDecThreads && DTS >= 0;
    bool ok;
    if (DTS >= 0) {
      ok = decode_chunk<(DTS < 0 ? 0 : DTS), W, GEN, SP>(J, c, S, lut0, stg, err, part, parts);
    } else {
      switch (J.dtype) {
        case ZIPNN_BF16:
          ok = decode_chunk<ZIPNN_BF16, W, GEN, SP>(J, c, S, lut0, stg, err, part, parts);
          break;
        case ZIPNN_FP16:
          ok = decode_chunk<ZIPNN_FP16, W, GEN, SP>(J, c, S, lut0, stg, err, part, parts);
          break;
        case ZIPNN_FP32:
          ok = decode_chunk<ZIPNN_FP32, W, GEN, SP>(J, c, S, lut0, stg, err, part, parts);
          break;
        default: ok = decode_chunk<ZIPNN_U8, W, GEN, SP>(J, c, S, lut0, stg, err, part, parts); break;
      }
    }
    if (!ok) break;  // a bulk copy timed out: leave the stage alone
    __syncthreads();
  }
  // the last CTA to leave resets the work queue for the next launch on the
  // same buffer (ticket[0]: next work item, ticket[1]: CTAs done)
  if (ticket) {
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      if (atomicAdd(ticket + 1, 1ull) == (unsigned long long)gridDim.x - 1ull) {
        atomicExch(ticket, 0ull);
        atomicExch(ticket + 1, 0ull);
      }
    }
  }
}

using DecodeKernel = void (*)(JobRef, uint64_t, uint32_t*, unsigned long long*, uint32_t,
                             uint32_t, uint32_t, uint32_t);

// (Every translation unit instantiates the mixed-batch kernels its switch
// names: they share the dtype-specialised out-of-line decode functions with
// the other kernels of the unit, whose register allocation depends on them.)
template <int W, int NT>
DecodeKernel pick_kernel(int dt, bool gen) {
  // kernels with the general fast loops (deltas: two coded 16-bit groups)
  if constexpr (W >= 11) {
    if (gen) {
      switch (dt) {
        case ZIPNN_BF16: return k_decode<ZIPNN_BF16, W, NT, true>;
        case ZIPNN_FP16: return k_decode<ZIPNN_FP16, W, NT, true>;
        case ZIPNN_FP32: case ZIPNN_U8: break;
        default: return k_decode<-1, W, kDecThreads, true>;
      }
    }
  }
  switch (dt) {
    case ZIPNN_BF16: return k_decode<ZIPNN_BF16, W, NT, false>;
    case ZIPNN_FP16: return k_decode<ZIPNN_FP16, W, NT, false>;
    case ZIPNN_FP32: return k_decode<ZIPNN_FP32, W, NT, false>;
    case ZIPNN_U8: return k_decode<ZIPNN_U8, W, NT, false>;
    default: return k_decode<-1, W, kDecThreads, false>;  // mixed batches: 128 threads
  }
}


// Kernel of a (W, CTA size) pair for a launch's dtype and delta content, as
// the handle the runtime's launch and attribute calls take.
template <int W, int NT>
const void* kernel_handle(int dt, bool gen) {
  return reinterpret_cast<const void*>(pick_kernel<W, NT>(dt, gen));
}

}  // namespace
}  // namespace zipnn
