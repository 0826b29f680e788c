/*
 * zipnn.h -- C ABI of libzipnn_gpu.so, a GB300 (sm_103a) implementation of the
 * lossless parameter codec of ZipNN (arXiv 2411.05239).
 *
 * What the codec computes (all of it in CUDA kernels on the device):
 *   - exponent extraction (Sec. 3.1): the 8 exponent bits of each BF16/FP32
 *     value form one byte stream; the sign moves to the top bit of the next
 *     byte.  FP16 uses the same 16-bit permutation (5 exponent bits + 3 high
 *     fraction bits form the first stream);
 *   - byte grouping (Sec. 3.2): every other byte position forms its own stream;
 *   - Huffman-only coding (Sec. 3.1) of every stream, in independent chunks
 *     (Sec. 5.1, 256 KiB by default), with all-zero and single-byte streams
 *     reduced to a header (Sec. 3.2) and incompressible streams stored raw
 *     (Sec. 3.2, "Identifying compressibility");
 *   - a map of every chunk and byte group so chunks decode in parallel
 *     (Sec. 5.1, "Metadata and parallelism");
 *   - XOR delta of two tensors (Sec. 4.2).
 * The container layout is specified in the project's design notes; streams are
 * byte-identical to those of the CPU oracle that implements that specification.
 *
 * Conventions for every call below:
 *   - "d_" pointers are CUDA device pointers owned by the caller unless stated
 *     otherwise; tensors and containers must start on a 16-byte boundary.
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue work on it and return without waiting, except
 *     where noted; results are valid once the stream has completed.
 *   - The return value reports host-side validation and launch errors.  Errors
 *     found by the kernels (a corrupt container, an exceeded wait) are recorded
 *     in a per-device error word and returned by zipnn_sync_status().
 *   - No call aborts, traps or falls back to the CPU.
 */
#ifndef ZIPNN_H
#define ZIPNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ZIPNN_BF16 = 0, /* 1 sign, 8 exponent, 7 fraction bits (Sec. 2.2) */
    ZIPNN_FP16 = 1, /* 1 sign, 5 exponent, 10 fraction bits */
    ZIPNN_FP32 = 2, /* 1 sign, 8 exponent, 23 fraction bits */
    ZIPNN_U8 = 3    /* plain bytes: one group, no permutation */
} zipnn_dtype;

typedef enum {
    ZIPNN_OK = 0,
    ZIPNN_EINVAL = -1,   /* bad argument: size, alignment, dtype, chunk size, base */
    ZIPNN_ENOMEM = -2,   /* device allocation failed or buffer too small */
    ZIPNN_ECORRUPT = -3, /* container failed validation */
    ZIPNN_ECUDA = -4,    /* a CUDA runtime call failed */
    ZIPNN_ETIMEOUT = -5, /* a bounded device-side wait gave up */
    ZIPNN_EBUSY = -6     /* admission refused: memory budget exhausted */
} zipnn_status;

#define ZIPNN_FLAG_DELTA 1u           /* container holds a XOR b (Sec. 4.2) */
#define ZIPNN_DEFAULT_CHUNK (256u << 10)  /* Sec. 5.1: 256 KB chunks */
#define ZIPNN_MIN_CHUNK 4096u
#define ZIPNN_MAX_CHUNK (16u << 20)
#define ZIPNN_MAX_LANES 1024u

/* A compressed container in device memory plus a host copy of its header
 * fields (so that decoding needs no device-to-host read). */
typedef struct zipnn_stream {
    void* data;           /* device pointer to the container (16-B aligned) */
    uint64_t nbytes;      /* container size in bytes */
    uint64_t orig_nbytes; /* size of the original tensor in bytes */
    int32_t dtype;        /* zipnn_dtype */
    uint32_t flags;       /* ZIPNN_FLAG_DELTA or 0 */
    uint32_t chunk_bytes; /* original bytes per chunk */
    uint32_t lanes;       /* interleaved sub-streams per Huffman group-chunk */
    uint32_t n_chunks;
    uint32_t n_groups;
    uint32_t owned;       /* 1: data was allocated by the library */
    uint32_t reserved;
} zipnn_stream;

/* Decoder launch parameters for batched decoding.  Zero fields take defaults;
 * the values change speed only, never the decoded bytes. */
typedef struct zipnn_tuning {
    int32_t threads;      /* decoder threads per CTA: 128 or 256 (0 = 256);
                             256 applies to batches of one dtype with W >= 11
                             whose lane counts are all multiples of 256;
                             otherwise, and for any other value, 128 */
    int32_t ctas_per_sm;  /* resident CTAs per SM for the persistent grid */
    int32_t lut_bits;     /* decode table width W in bits: 10, 11 or 12 (0 = 12);
                             W = 10 resolves codes longer than 10 bits through
                             the canonical limits, W = 11 resolves 12-bit codes
                             inside the table */
    int32_t debug_flags;  /* 0.  Bit 0 is fault injection for tests: the decoder
                             waits for 16 bytes that are never copied, so its
                             bounded wait gives up after 100 ms and the call
                             reports ZIPNN_ETIMEOUT via zipnn_sync_status */
    int32_t parts;        /* work items per chunk: 0 = automatic (launches whose
                             chunks would fill at most half the SMs split each
                             model-weight chunk's sub-streams over 2, 4 or 8
                             work items of 128-thread CTAs), 1 = never split,
                             2, 4 or 8 = split whenever the lanes allow */
} zipnn_tuning;

/* Library version (the container version is 1). */
int zipnn_version(void);

/* Text for a status code; never NULL. */
const char* zipnn_strerror(int status);

/* Sub-streams per Huffman group-chunk used when a call takes no lanes value,
 * for plain containers: chunk_bytes / 512 for BF16 and FP16 (512 at 256 KiB:
 * two sub-streams per thread of a 256-thread decoder CTA, whose fast loop runs
 * them in lockstep), chunk_bytes / 1024 for FP32 and U8; clamped to [1, 1024].
 * Deltas (a base given, no lanes value) take chunk_bytes / 1024 for every
 * dtype: their payloads are small, so the 4-byte start of every sub-stream
 * weighs on the ratio. */
uint32_t zipnn_default_lanes(int dtype, size_t chunk_bytes);

/* Upper bound on the container size for nbytes of the given dtype and chunk
 * size: header + map + raw data + 16-B padding per group-chunk. */
size_t zipnn_compress_bound(size_t nbytes, int dtype, size_t chunk_bytes);

/* Device scratch needed by zipnn_compress_into for this input. */
size_t zipnn_compress_workspace_size(size_t nbytes, int dtype, size_t chunk_bytes);

/* Compress nbytes of d_src (Sec. 3.1, 3.2, 5.1).  Allocates the container
 * (stream-ordered, on cuda_stream) and fills *out; free it with
 * zipnn_stream_free.  Synchronises cuda_stream once, to learn the exact
 * container size before allocating it.
 * Errors: EINVAL if dtype is unknown, nbytes is not a multiple of the element
 * size, chunk_bytes is not a multiple of 16 in [4 KiB, 16 MiB], or d_src is not
 * 16-B aligned; ENOMEM if allocation fails; ECUDA on a launch error. */
zipnn_status zipnn_compress(const void* d_src, size_t nbytes, int dtype, size_t chunk_bytes,
                            zipnn_stream* out, void* cuda_stream);

/* Delta (Sec. 4.2): compress d_a XOR d_b (both nbytes, caller-owned); the
 * container is flagged ZIPNN_FLAG_DELTA and decodes only with d_b as base. */
zipnn_status zipnn_delta(const void* d_a, const void* d_b, size_t nbytes, int dtype,
                         size_t chunk_bytes, zipnn_stream* out, void* cuda_stream);

/* Compress into caller-owned memory without allocating or synchronising.
 * d_base_or_null: NULL for a plain container, else the delta base (nbytes).
 * lanes: 0 = zipnn_default_lanes.  d_out must hold out_capacity >=
 * zipnn_compress_bound() bytes; d_workspace must hold workspace_bytes >=
 * zipnn_compress_workspace_size() bytes and must not be used by another call
 * until this one completes.  The container size is written, as a uint64, to
 * d_out_nbytes (a device or host-mapped pointer; may be NULL) -- it is also in
 * the container header at byte 40. */
zipnn_status zipnn_compress_into(const void* d_src, const void* d_base_or_null, size_t nbytes,
                                 int dtype, size_t chunk_bytes, uint32_t lanes, void* d_out,
                                 size_t out_capacity, void* d_workspace, size_t workspace_bytes,
                                 uint64_t* d_out_nbytes, void* cuda_stream);

/* No-allocation compression (the paper has no counterpart; this serves
 * callers that cannot allocate device memory when they compress: plugins that
 * only receive device pointers from a host framework whose caching allocator
 * they cannot reach, latency-critical loops where a cudaMalloc/cudaFree could
 * synchronise the device, processes with a device-memory budget fixed at
 * start-up).  Same arguments and output as zipnn_compress_into minus the
 * workspace: the scratch is a fixed 8 MiB device array inside the library
 * (held by every GPU that loads it until exit), so one call handles at most
 * 3,572 (chunk, byte group) pairs (2,348 bytes of scratch each) -- 446.5 MiB
 * of BF16/FP16 or 223.25 MiB of FP32 at 256 KiB chunks, 3,572 chunks of U8;
 * larger inputs return ZIPNN_ENOMEM before any launch.  It
 * calls no allocator.  All calls on a device share that array: calls whose
 * kernels overlap on the GPU (e.g. unordered streams) race and corrupt each
 * other's output, so order them.  The first call on a device looks up the
 * array's address (cudaGetSymbolAddress); make it before any stream capture. */
zipnn_status zipnn_compress_into_static(const void* d_src, const void* d_base_or_null,
                                        size_t nbytes, int dtype, size_t chunk_bytes,
                                        uint32_t lanes, void* d_out, size_t out_capacity,
                                        uint64_t* d_out_nbytes, void* cuda_stream);

/* Batched compression of `count` tensors in one set of launches (one
 * histogram, one code-build, one scan and one pack kernel for all of them).
 * d_srcs[i] holds nbytes[i] bytes of dtypes[i]; d_bases may be NULL or hold a
 * delta base (or NULL) per tensor; d_outs[i] must hold out_capacities[i] >=
 * zipnn_compress_bound() bytes; the container sizes are written to
 * d_out_nbytes[i] (device or host-mapped array, may be NULL).  The workspace
 * (>= zipnn_batch_compress_workspace_size) also holds the job table, copied
 * from host memory during the call.  Same errors as zipnn_compress_into. */
size_t zipnn_batch_compress_workspace_size(const size_t* nbytes, const int* dtypes, int count,
                                           size_t chunk_bytes);
zipnn_status zipnn_batch_compress_into(const void* const* d_srcs, const void* const* d_bases,
                                       const size_t* nbytes, const int* dtypes, int count,
                                       size_t chunk_bytes, uint32_t lanes, void* const* d_outs,
                                       const size_t* out_capacities, void* d_workspace,
                                       size_t workspace_bytes, uint64_t* d_out_nbytes,
                                       void* cuda_stream);

/* Encoder options (zipnn_batch_compress_into_ex).
 * lanes: sub-streams per Huffman group-chunk, 0 = zipnn_default_lanes.
 * probe_skip: the skip-ahead probe of ZipNN Sec. 3.2 ("Identifying
 *   compressibility"): after a group-chunk is decided raw, the same byte group
 *   of the next probe_skip chunks of the tensor is stored raw without its
 *   decision counting, then decisions resume; 0 = every group-chunk decided on
 *   its own (the default).  The containers stay valid version-1 containers.
 * encoder: 0 = four kernels (histograms, codes, offsets, packing; the
 *   default, and the faster on GB300).  1 = the single-pass encoder for
 *   batches whose tensors are all BF16, all FP16 or all U8, without
 *   probe_skip (one persistent kernel: each chunk's histograms, codes, offset
 *   -- by a bounded look-back over the chunks before it -- and packing, the
 *   chunk's second read coming from L2 when it is still there); the four
 *   kernels for other batches.  Both write the same bytes.  EINVAL for other
 *   values.
 * debug_flags: 0.  Bit 0 is fault injection for tests of the single-pass
 *   encoder: the launch's first chunk never publishes its payload size, so the
 *   look-backs that need it give up after 100 ms; those chunks are not
 *   written and zipnn_sync_status reports ZIPNN_ETIMEOUT.  Other bits: EINVAL. */
typedef struct zipnn_encode_options {
    uint32_t lanes;
    uint32_t probe_skip;
    uint32_t encoder;
    uint32_t debug_flags;
} zipnn_encode_options;

/* zipnn_batch_compress_into with encoder options (opts may be NULL: defaults);
 * arguments, workspace and errors otherwise as zipnn_batch_compress_into. */
zipnn_status zipnn_batch_compress_into_ex(
    const void* const* d_srcs, const void* const* d_bases, const size_t* nbytes,
    const int* dtypes, int count, size_t chunk_bytes, const zipnn_encode_options* opts,
    void* const* d_outs, const size_t* out_capacities, void* d_workspace,
    size_t workspace_bytes, uint64_t* d_out_nbytes, void* cuda_stream);

/* Wrap a container that is already in device memory (e.g. copied from a file)
 * as a zipnn_stream: reads and validates its 64-B header (synchronous copy of
 * 64 bytes).  The stream does not own d_data.  ECORRUPT if the header is bad. */
zipnn_status zipnn_stream_wrap(const void* d_data, size_t nbytes, zipnn_stream* out);

/* Original size and dtype of a container: the exact byte count that
 * decompression gives back (Sec. 2.3, "Lossless compression": compression
 * followed by decompression returns the input exactly), read from the header
 * fields that the map of Sec. 5.1 ("Metadata and parallelism") travels with.
 * Host-only; never touches the device.  EINVAL if s is NULL. */
zipnn_status zipnn_decompressed_size(const zipnn_stream* s, size_t* nbytes, int* dtype);

/* Decompress s into d_dst (caller-owned, exactly orig_nbytes bytes): the
 * inverse of compression, giving back the original bytes exactly (Sec. 2.3,
 * "Lossless compression").  The chunk map (Sec. 5.1, "Metadata and
 * parallelism") locates every chunk and byte group, so all chunks decode in
 * parallel in one launch; each group is Huffman-decoded, copied (raw) or
 * filled (zero, constant) and the groups are merged back into the dtype's
 * byte order (the inverse of Sec. 3.1 / 3.2); a delta container is XOR-ed
 * with its base (Sec. 4.2).
 * d_base_or_null must be the delta base (orig_nbytes) iff s is a delta
 * container, else NULL (EINVAL otherwise).  EINVAL also for a malformed
 * stream descriptor, a dst_nbytes other than orig_nbytes or an unaligned
 * pointer.  Chunks that fail validation on the device are skipped and
 * reported as ECORRUPT by zipnn_sync_status. */
zipnn_status zipnn_decompress(const zipnn_stream* s, const void* d_base_or_null, void* d_dst,
                              size_t dst_nbytes, void* cuda_stream);

/* Decompress count containers in ONE persistent kernel that pulls
 * (tensor, chunk) work items from a device queue (the batching form).  Each
 * container decodes to exactly its original bytes (Sec. 2.3), as with
 * zipnn_decompress; the chunk maps (Sec. 5.1, "Metadata and parallelism") make
 * every chunk of every container an independent work item, which is what
 * lets one grid serve tensors of uneven sizes (the paper's multi-worker
 * decompression of Sec. 5.3 is the CPU counterpart).
 * streams[i] decodes into d_dsts[i]; d_bases may be NULL (no deltas) or hold
 * one base pointer (or NULL) per container.  tuning may be NULL.  Errors as
 * zipnn_decompress, per container; ENOMEM if the job table cannot be
 * allocated (stream-ordered, freed after the launch). */
zipnn_status zipnn_batch_decompress(const zipnn_stream* streams, const void* const* d_bases,
                                    void* const* d_dsts, int count, const zipnn_tuning* tuning,
                                    void* cuda_stream);

/* Plans (batching form): a fixed set of tensors prepared once -- job table
 * uploaded to the device, scratch allocated, and the launches captured in a
 * CUDA graph -- so each later batched (de)compression of the same buffers is
 * one zipnn_plan_launch (one cudaGraphLaunch).  The pointers given at plan
 * creation must stay valid, and their contents may change between launches
 * (new weights in the same buffers); creation synchronises the device once.
 *
 * zipnn_plan_decompress: the persistent decoder over all containers (work
 *   items pulled from a device ticket), as zipnn_batch_decompress.  Creation
 *   reads the containers' chunk maps (a device-to-host copy) to size the
 *   decoder's shared-memory stage and pick its kernel variant; maps that
 *   change later change the speed, never the decoded bytes.
 * zipnn_plan_compress: the four encoder kernels over all tensors, as
 *   zipnn_batch_compress_into, with the scratch owned by the plan.
 * Errors: EINVAL for bad arguments (as the corresponding direct calls),
 * ENOMEM/ECUDA if allocation or capture fails.  zipnn_plan_launch returns
 * EINVAL when called with another device current than at creation. */
typedef struct zipnn_plan zipnn_plan;
zipnn_status zipnn_plan_decompress(const zipnn_stream* streams, const void* const* d_bases,
                                   void* const* d_dsts, int count, const zipnn_tuning* tuning,
                                   zipnn_plan** out);
zipnn_status zipnn_plan_compress(const void* const* d_srcs, const void* const* d_bases,
                                 const size_t* nbytes, const int* dtypes, int count,
                                 size_t chunk_bytes, uint32_t lanes, void* const* d_outs,
                                 const size_t* out_capacities, uint64_t* d_out_nbytes,
                                 zipnn_plan** out);
/* zipnn_plan_load (loading form, e.g. a checkpoint kept compressed in host
 *   memory): every launch copies container i from h_containers[i] (page-locked
 *   host memory, streams[i].nbytes bytes) into streams[i].data (device, 16-B
 *   aligned, at least streams[i].nbytes bytes; streams[i] describes the
 *   container, e.g. from zipnn_stream_wrap of an earlier copy) and decodes it
 *   into d_dsts[i] (XOR d_bases[i] for delta containers, as
 *   zipnn_batch_decompress).  Containers are taken in order in segments of
 *   about segment_bytes (0 = 512 MiB); each segment's persistent decode starts
 *   as soon as its copies have landed, while the copies of the next segments
 *   proceed on another stream: one graph, copies and decoding overlapped.
 *   Containers of a segment that sit back to back in both host and device
 *   memory (h_containers[i] + nbytes == h_containers[i+1] and likewise for
 *   data) travel in one copy; no byte outside a container is written.
 *   Pageable host memory cannot be captured and returns ECUDA.  Creation
 *   reads the host containers' chunk maps to size each segment's stage. */
zipnn_status zipnn_plan_load(const zipnn_stream* streams, const void* const* h_containers,
                             const void* const* d_bases, void* const* d_dsts, int count,
                             size_t segment_bytes, const zipnn_tuning* tuning, zipnn_plan** out);
/* Sharded decoding of one checkpoint over `world` GPUs (one process per GPU).
 * ZipNN's chunks are independent and the map records every chunk and byte
 * group (Sec. 5.1, "Chunking", "Metadata and parallelism"), so the chunks of
 * `count` containers taken in order form one sequence of work items that
 * ranks can split with no exchange.
 *
 * zipnn_partition_chunks (host only, calls no CUDA function): cuts that
 *   sequence into `world` contiguous ranges of near-equal decode traffic; a
 *   chunk weighs its stored payload bytes (16-B padded) plus its original
 *   bytes.  h_maps[i] is a host copy of container i's first 64 + 16 *
 *   n_chunks * n_groups bytes (header and map; a whole host container will
 *   do), streams[i] its descriptor.  Writes world + 1 global chunk indices to
 *   bounds: rank r owns chunks [bounds[r], bounds[r+1]); bounds[0] = 0 and
 *   bounds[world] = the total.  Each range's weight is within one chunk's
 *   weight of an equal share.  EINVAL for bad descriptors or world < 1,
 *   ECORRUPT for a map entry with an unknown mode.
 * zipnn_plan_decompress_range: as zipnn_plan_decompress, for the global
 *   chunks [chunk_lo, chunk_hi) only.  For a container whose chunks
 *   [a, b) (its own numbering) fall in the range, d_dsts[i] receives the
 *   original bytes [a * chunk_bytes, min(b * chunk_bytes, orig_nbytes)) --
 *   a buffer of just that extent, 16-B aligned -- and d_bases[i] (deltas)
 *   holds the base's bytes of the same extent.  Containers with no chunk in
 *   the range are ignored (their d_dsts entries may be NULL).  EINVAL if the
 *   range is empty or runs past the last chunk. */
zipnn_status zipnn_partition_chunks(const zipnn_stream* streams, const void* const* h_maps,
                                    int count, int world, uint64_t* bounds);
zipnn_status zipnn_plan_decompress_range(const zipnn_stream* streams, const void* const* d_bases,
                                         void* const* d_dsts, int count, uint64_t chunk_lo,
                                         uint64_t chunk_hi, const zipnn_tuning* tuning,
                                         zipnn_plan** out);
zipnn_status zipnn_plan_launch(zipnn_plan* plan, void* cuda_stream);
void zipnn_plan_destroy(zipnn_plan* plan);

/* Request server (serving form): continuous batching of compress and
 * decompress requests with admission against a device-memory budget.
 * zipnn_server_create allocates a device arena of budget_bytes (outputs and
 * scratch live there) and `slots` CUDA streams, and starts a scheduler thread
 * on the current device.  zipnn_server_submit (thread-safe, does not wait for
 * the device) queues a request; the scheduler admits requests in arrival order while their
 * input bytes (caller-owned, charged only), output and scratch fit the budget
 * and a slot is free, and launches everything admitted in one pass as one
 * batch (one batched compression + one persistent batched decode) on that
 * slot's stream, so batches on different slots overlap on the device.
 * zipnn_server_poll returns completions; each output stays in the arena (and
 * charged) until zipnn_server_release.  A request whose footprint exceeds the
 * whole budget is refused at submit with EBUSY.  The caller's inputs must stay
 * valid until the request completes.  A request that finds nothing queued and
 * a slot free is admitted and launched on the submitting thread (the call
 * then also returns after the launch, not only after queueing).  Completion
 * status: the launch's status, else the batch's device error word (a corrupt
 * container fails every request of its batch with ECORRUPT).  Times are
 * seconds on the host's steady clock (std::chrono::steady_clock). */
#define ZIPNN_OP_COMPRESS 0
#define ZIPNN_OP_DECOMPRESS 1
typedef struct zipnn_request {
    int32_t op;            /* ZIPNN_OP_COMPRESS or ZIPNN_OP_DECOMPRESS */
    int32_t dtype;         /* compress: zipnn_dtype of the input */
    const void* d_input;   /* compress: the tensor (16-B aligned) */
    uint64_t input_bytes;  /* compress: tensor bytes */
    zipnn_stream container;/* decompress: the container to decode */
    const void* d_base;    /* delta base (compress: makes a delta; decompress: required
                              for delta containers), else NULL */
    uint64_t chunk_bytes;  /* compress: 0 = 256 KiB */
    uint64_t tag;          /* caller's value, echoed in the completion */
} zipnn_request;
typedef struct zipnn_completion {
    uint64_t id;           /* server id returned by submit */
    uint64_t tag;
    int32_t status;        /* zipnn_status of the request's batch */
    int32_t op;
    void* d_output;        /* container (compress) or tensor (decompress) in the arena */
    uint64_t output_bytes;
    double t_submit, t_admit, t_done;
} zipnn_completion;
typedef struct zipnn_server_stats {
    uint64_t submitted, completed, batches, max_batch, bytes_processed;
    uint64_t arena_used, inputs_charged;
} zipnn_server_stats;
typedef struct zipnn_server zipnn_server;
zipnn_status zipnn_server_create(uint64_t budget_bytes, int slots, zipnn_server** out);
zipnn_status zipnn_server_submit(zipnn_server* s, const zipnn_request* r, uint64_t* id);
int zipnn_server_poll(zipnn_server* s, zipnn_completion* out, int max);
zipnn_status zipnn_server_release(zipnn_server* s, uint64_t id);
/* Wait until nothing is queued or running (ETIMEOUT after timeout_s).  Queued
 * requests are admitted only as budget frees up, so a caller that holds
 * unreleased outputs must keep releasing them while it waits. */
zipnn_status zipnn_server_drain(zipnn_server* s, double timeout_s);
zipnn_status zipnn_server_get_stats(zipnn_server* s, zipnn_server_stats* st);
/* Stop the scheduler: queued requests are cancelled (never run), running
 * batches complete, then the arena and streams are freed. */
void zipnn_server_destroy(zipnn_server* s);

/* Wait for cuda_stream and return (and clear) the device error word:
 * ECORRUPT for a container rejected by a kernel, ETIMEOUT for a bounded wait
 * that gave up, else the CUDA error state as ECUDA, else OK. */
zipnn_status zipnn_sync_status(void* cuda_stream);

/* Free a container allocated by the library (no-op for wrapped streams). */
void zipnn_stream_free(zipnn_stream* s);

#ifdef __cplusplus
}
#endif
#endif /* ZIPNN_H */
