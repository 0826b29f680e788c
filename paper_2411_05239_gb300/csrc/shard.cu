// Sharded decoding of one checkpoint over several GPUs: the split of the
// chunks (host code only; no CUDA call).
//
// ZipNN's chunks are independent and its map records every chunk and byte
// group (Sec. 5.1, "Chunking", "Metadata and parallelism"), so a set of
// containers taken in order is one sequence of (container, chunk) work items
// that any number of workers can split without exchanging anything.  This file
// cuts that sequence into `world` contiguous ranges of near-equal decode
// traffic, read from the maps: a chunk weighs its coded payload bytes (16-B
// padded, as stored) plus its original bytes, the bytes its decode reads and
// writes.  Rank r then decodes the chunks [bounds[r], bounds[r+1]) with
// zipnn_plan_decompress_range into its own memory.
#include <cstdint>
#include <cstring>
#include <vector>

#include "zipnn.h"
#include "host_internal.h"

using namespace zipnn;

extern "C" zipnn_status zipnn_partition_chunks(const zipnn_stream* streams,
                                               const void* const* h_maps, int count, int world,
                                               uint64_t* bounds) {
  if (!streams || !h_maps || count <= 0 || world < 1 || !bounds) return ZIPNN_EINVAL;
  // per-chunk weights of the whole sequence
  std::vector<uint64_t> pre;  // prefix sums, pre[k] = weight of chunks [0, k)
  pre.push_back(0);
  for (int i = 0; i < count; i++) {
    const zipnn_stream* s = &streams[i];
    if (s->dtype < ZIPNN_BF16 || s->dtype > ZIPNN_U8 ||
        s->n_groups != (uint32_t)elem_size(s->dtype) || s->chunk_bytes < ZIPNN_MIN_CHUNK ||
        (uint64_t)s->n_chunks != (s->orig_nbytes + s->chunk_bytes - 1) / s->chunk_bytes)
      return ZIPNN_EINVAL;
    if (!s->n_chunks) continue;  // an empty tensor has no work item
    if (!h_maps[i]) return ZIPNN_EINVAL;
    const uint8_t* map = static_cast<const uint8_t*>(h_maps[i]) + kHdrBytes;  // after the header
    for (uint32_t c = 0; c < s->n_chunks; c++) {
      uint64_t w = (uint64_t)s->chunk_bytes;
      if (c + 1 == s->n_chunks) w = s->orig_nbytes - (uint64_t)c * s->chunk_bytes;
      for (uint32_t g = 0; g < s->n_groups; g++) {
        const uint8_t* e = map + ((uint64_t)c * s->n_groups + g) * kEntryBytes;
        uint32_t size;
        memcpy(&size, e + 8, 4);
        const uint32_t mode = e[12];
        if (mode > kSparse) return ZIPNN_ECORRUPT;
        if (mode == kRaw || mode == kHuff || mode == kSparse) w += align_up(size, 16);
      }
      pre.push_back(pre.back() + w);
    }
  }
  // cut r lies at the first chunk boundary whose prefix reaches r/world of
  // the total; the heaviest range exceeds an equal share by less than one
  // chunk's weight
  const uint64_t n = pre.size() - 1, total = pre.back();
  bounds[0] = 0;
  uint64_t k = 0;
  for (int r = 1; r < world; r++) {
    const unsigned __int128 want = (unsigned __int128)total * (unsigned)r;
    while (k < n && (unsigned __int128)pre[k] * (unsigned)world < want) k++;
    bounds[r] = k;
  }
  bounds[world] = n;
  return ZIPNN_OK;
}
