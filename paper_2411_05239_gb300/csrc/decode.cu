// Decoder kernel of the GB300 ZipNN codec: table-driven Huffman decoding of
// every byte-group stream of a chunk and the merge back to the original dtype
// (ZipNN Sec. 3.1, 3.2 inverse; Sec. 4.2 XOR with the base; Sec. 5.1 map).
//
// Work unit = one chunk.  A persistent grid pulls chunks of all tensors of a
// batch from a device ticket (atomicAdd), so one launch decodes many tensors of
// uneven sizes.  Per chunk the CTA
//   1. reads and validates the chunk's map entries and Huffman tables,
//   2. builds a 4096-entry {symbol, length} lookup table per Huffman group in
//      shared memory (12-bit windows: codes are limited to 12 bits),
//   3. decodes: thread t owns interleaved sub-stream t, i.e. the vectors
//      v = t, t+T, ... of the chunk, so every step of the warp touches 32
//      consecutive 16-byte vectors: raw-group loads and the 16-B output stores
//      are fully coalesced; the merge (inverse permutation, XOR base) happens
//      in registers.
// The decoder is total: symbol counts are fixed by the map, bit reads past a
// payload return zero bits, an invalid code or map entry sets the error word.
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "zipnn_internal.cuh"

namespace zipnn {

namespace {

constexpr int kDecThreads = 128;

struct JobRef {
  const Job* table;
  Job one;
  int n;
};

__device__ __forceinline__ const Job& job_at(const JobRef& r, int j) {
  return r.table ? r.table[j] : r.one;
}

struct ChunkInfo {
  uint32_t mode[4];
  uint32_t value[4];
  uint32_t nwords[4];       // bitstream words (HUFF)
  uint64_t payload[4];      // byte offset of the payload within the container
  uint64_t bs[4];           // byte offset of the bitstream (HUFF)
  uint64_t offs[4];         // byte offset of the start-bit table (HUFF)
  uint32_t bad;
};

__device__ __forceinline__ uint32_t ld_word(const uint32_t* w, uint32_t i, uint32_t n) {
  return i < n ? __ldg(w + i) : 0u;
}

struct BitReader {
  const uint32_t* w;
  uint32_t n, idx, w0, w1, pos;
  __device__ __forceinline__ void init(const uint32_t* words, uint32_t nwords, uint32_t start) {
    w = words;
    n = nwords;
    idx = start >> 5;
    pos = start & 31;
    w0 = ld_word(w, idx, n);
    w1 = ld_word(w, idx + 1, n);
    idx += 2;
  }
  // Decode one symbol with the 12-bit table; flags an invalid code.
  __device__ __forceinline__ uint32_t decode(const uint16_t* lut, uint32_t& bad) {
    uint32_t win = __funnelshift_l(w1, w0, pos) >> (32 - kMaxLen);
    uint32_t e = lut[win];
    uint32_t len = e >> 8;
    bad |= (len == 0);
    pos += len;
    if (pos >= 32) {
      pos -= 32;
      w0 = w1;
      w1 = ld_word(w, idx, n);
      idx++;
    }
    return e & 0xFFu;
  }
};

__device__ __forceinline__ uint32_t rd_u32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
__device__ __forceinline__ uint64_t rd_u64(const uint8_t* p) {
  return (uint64_t)rd_u32(p) | ((uint64_t)rd_u32(p + 4) << 32);
}

__global__ void __launch_bounds__(kDecThreads)
k_decode(JobRef jr, uint64_t nchunks_total, uint32_t* __restrict__ err,
         unsigned long long* __restrict__ ticket) {
  extern __shared__ uint16_t lut[];  // [4][kLutSize]
  __shared__ ChunkInfo CI;
  __shared__ unsigned long long s_chunk;
  __shared__ uint32_t s_cnt[4][kMaxLen + 1];
  __shared__ uint8_t s_sym[4][256];
  const int tid = threadIdx.x, nthr = blockDim.x;

  for (uint64_t iter = 0;; iter++) {
    // work item: from the device queue (batched form) or a static stride
    uint64_t chunk;
    if (ticket) {
      if (tid == 0) s_chunk = atomicAdd(ticket, 1ull);
      __syncthreads();
      chunk = s_chunk;
    } else {
      chunk = blockIdx.x + iter * gridDim.x;
    }
    if (chunk >= nchunks_total) break;
    const int j = jr.table ? find_job(jr.table, jr.n, chunk) : 0;
    const Job& J = job_at(jr, j);
    const int dtype = J.dtype;
    const int es = elem_size(dtype), G = es, V = 16 / es;
    const uint64_t c = chunk - J.chunk_begin;
    const uint64_t off0 = c * J.chunk_bytes;
    const uint64_t nb = min((uint64_t)J.chunk_bytes, J.nbytes - off0);
    const uint64_t m = nb / es;
    const uint64_t nvec = (nb + 15) / 16;
    const uint32_t T = J.lanes;
    const uint8_t* cont = J.src;
    const uint64_t P = kHdrBytes + (uint64_t)J.n_chunks * G * kEntryBytes;

    // 1. map entries + table validation (thread g handles group g)
    if (tid == 0) CI.bad = 0;
    __syncthreads();
    if (tid < G) {
      const uint8_t* e = cont + kHdrBytes + (c * G + tid) * kEntryBytes;
      const uint64_t po = rd_u64(e);
      const uint32_t size = rd_u32(e + 8);
      const uint32_t mode = e[12], value = e[13];
      uint32_t bad = 0;
      const uint64_t avail = J.stream_bytes > P ? J.stream_bytes - P : 0;
      if (mode > kConst || po > avail || align_up(size, 16) > avail - po) bad = 1;
      if (mode == kRaw && size != m) bad = 1;
      if ((mode == kZero || mode == kConst) && size != 0) bad = 1;
      CI.mode[tid] = mode;
      CI.value[tid] = value;
      CI.payload[tid] = P + po;
      if (!bad && mode == kHuff) {
        const uint8_t* p = cont + P + po;
        uint32_t nz = 0, kraft = 0;
        if (size < 12) bad = 1;
        else {
          for (int l = 1; l <= kMaxLen; l++) {
            uint32_t cl = p[l - 1];
            s_cnt[tid][l] = cl;
            nz += cl;
            kraft += cl << (kMaxLen - l);
          }
          const uint64_t h = align_up(12 + nz, 4);
          if (nz < 2 || nz > 256 || kraft > (uint32_t)kLutSize || size < h + 4ull * (T - 1) ||
              (size - h - 4ull * (T - 1)) % 4)
            bad = 1;
          else {
            CI.offs[tid] = P + po + h;
            CI.bs[tid] = P + po + h + 4ull * (T - 1);
            CI.nwords[tid] = (uint32_t)((size - h - 4ull * (T - 1)) / 4);
            for (uint32_t k = 0; k < nz; k++) s_sym[tid][k] = p[12 + k];
          }
        }
      }
      if (bad) atomicOr(&CI.bad, 1u);
    }
    __syncthreads();
    if (CI.bad) {
      if (tid == 0) atomicOr(err, 1u);
      __syncthreads();
      continue;
    }

    // 2. lookup tables: entry w (12-bit window) -> (length << 8) | symbol
    for (int g = 0; g < G; g++) {
      if (CI.mode[g] != kHuff) continue;
      uint32_t lim[kMaxLen + 1], first[kMaxLen + 1], index[kMaxLen + 1];
      uint32_t code = 0, idx = 0;
      uint32_t prevc = 0;
      for (int l = 1; l <= kMaxLen; l++) {
        code = (code + prevc) << 1;
        uint32_t cl = s_cnt[g][l];
        first[l] = code;
        index[l] = idx;
        lim[l] = (code + cl) << (kMaxLen - l);  // left-justified end of length-l codes
        idx += cl;
        prevc = cl;
      }
      uint16_t* L = lut + g * kLutSize;
      for (int w = tid; w < kLutSize; w += nthr) {
        int l = 1;
        while (l <= kMaxLen && (uint32_t)w >= lim[l]) l++;
        uint16_t ent = 0;
        if (l <= kMaxLen) {
          uint32_t r = index[l] + ((uint32_t)w >> (kMaxLen - l)) - first[l];
          ent = (uint16_t)((l << 8) | s_sym[g][r]);
        }
        L[w] = ent;
      }
    }
    __syncthreads();

    // 3. decode + merge
    uint8_t* dst = J.dst + off0;
    const uint8_t* base = J.base ? J.base + off0 : nullptr;
    uint32_t bad = 0;
    for (uint32_t t = tid; t < T; t += nthr) {
      BitReader br[4];
      for (int g = 0; g < G; g++) {
        if (CI.mode[g] != kHuff) continue;
        uint32_t start = t ? rd_u32(cont + CI.offs[g] + 4ull * (t - 1)) : 0u;
        if (start > CI.nwords[g] * 32u) { bad = 1; start = CI.nwords[g] * 32u; }
        br[g].init(reinterpret_cast<const uint32_t*>(cont + CI.bs[g]), CI.nwords[g], start);
      }
      for (uint64_t v = t; v < nvec; v += T) {
        const int valid = (int)min((uint64_t)V, m - v * V);
        uint32_t gw[4][4];
        for (int g = 0; g < G; g++) {
          const uint32_t mode = CI.mode[g];
          if (mode == kHuff) {
            const uint16_t* L = lut + g * kLutSize;
            uint32_t q[4] = {0, 0, 0, 0};
            if (valid == V) {
#pragma unroll
              for (int k = 0; k < 16; k++) {
                if (k < V) q[k >> 2] |= br[g].decode(L, bad) << (8 * (k & 3));
              }
            } else {
              for (int k = 0; k < valid; k++) q[k >> 2] |= br[g].decode(L, bad) << (8 * (k & 3));
            }
            gw[g][0] = q[0]; gw[g][1] = q[1]; gw[g][2] = q[2]; gw[g][3] = q[3];
          } else if (mode == kRaw) {
            const uint8_t* p = cont + CI.payload[g] + v * V;
            if (V == 8) {
              uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
              gw[g][0] = r.x; gw[g][1] = r.y;
            } else if (V == 4) {
              gw[g][0] = __ldg(reinterpret_cast<const uint32_t*>(p));
            } else {
              uint4 r = __ldg(reinterpret_cast<const uint4*>(p));
              gw[g][0] = r.x; gw[g][1] = r.y; gw[g][2] = r.z; gw[g][3] = r.w;
            }
          } else {
            uint32_t b = (mode == kConst) ? CI.value[g] * 0x01010101u : 0u;
            gw[g][0] = b; gw[g][1] = b; gw[g][2] = b; gw[g][3] = b;
          }
        }
        uint32_t x[4];
        if (dtype == ZIPNN_FP32) {
          uint32_t g4[4] = {gw[0][0], gw[1][0], gw[2][0], gw[3][0]};
          merge32(g4, x);
        } else if (dtype == ZIPNN_U8) {
          x[0] = gw[0][0]; x[1] = gw[0][1]; x[2] = gw[0][2]; x[3] = gw[0][3];
        } else {
          merge16(gw[0][0], gw[1][0], x[0], x[1]);
          merge16(gw[0][1], gw[1][1], x[2], x[3]);
        }
        if ((v + 1) * 16 <= nb) {
          if (base) {
            uint4 b = __ldg(reinterpret_cast<const uint4*>(base) + v);
            x[0] ^= b.x; x[1] ^= b.y; x[2] ^= b.z; x[3] ^= b.w;
          }
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
    __syncthreads();
  }
}

}  // namespace

int decode_smem_bytes(int max_groups) { return max_groups * kLutSize * 2; }

cudaError_t launch_decode_ex(const Job* d_jobs, const Job* h_one, int njobs,
                             uint64_t nchunks_total, int max_groups, const zipnn_tuning* tuning,
                             uint32_t* d_err, unsigned long long* d_ticket, cudaStream_t st) {
  if (nchunks_total == 0) return cudaSuccess;
  JobRef r;
  r.table = h_one ? nullptr : d_jobs;
  if (h_one) r.one = *h_one;
  else memset(&r.one, 0, sizeof(Job));
  r.n = njobs;
  int threads = kDecThreads;
  int per_sm = 0;
  if (tuning && tuning->ctas_per_sm > 0) per_sm = tuning->ctas_per_sm;
  const int smem = decode_smem_bytes(max_groups);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (per_sm == 0) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_decode, threads, smem);
    per_sm = occ > 0 ? occ : 1;
  }
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > nchunks_total) grid = nchunks_total;
  if (d_ticket) {
    cudaError_t e = cudaMemsetAsync(d_ticket, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  k_decode<<<(unsigned)grid, threads, smem, st>>>(r, nchunks_total, d_err, d_ticket);
  return cudaGetLastError();
}

}  // namespace zipnn
