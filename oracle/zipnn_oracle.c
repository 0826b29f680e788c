/*
 * ZipNN codec oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, single-threaded, deliberately slow CPU encoder/decoder of the
 * chunked, byte-grouped Huffman container.  It exists to define and check what
 * the CUDA path must produce: the GPU streams must be byte-identical to the
 * ones written here, and the bytes decoded here must equal the input.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm may load it; the product library never links or calls it.  It shares no
 * source with the CUDA path: it follows the written container specification.
 *
 * Method (ZipNN, arXiv 2411.05239):
 *   - exponent extraction: the 8 exponent bits of every float form one byte
 *     stream, the sign bit moves out of that byte (Sec. 3.1, Fig. "Exponent
 *     Extraction for BF16");
 *   - byte grouping: the remaining bytes of each parameter form one stream per
 *     byte position, compressed separately (Sec. 3.2, Fig. "Byte Grouping");
 *   - Huffman-only entropy coding of each stream (Sec. 3.1, "Huffman only
 *     Compression"); all-zero streams become a header only (Sec. 3.2);
 *     incompressible streams are stored raw (Sec. 3.2, "Identifying
 *     compressibility");
 *   - independent fixed-size chunks, 256 KB by default, with a metadata map of
 *     every chunk and byte group (Sec. 5.1, "Chunking", "Metadata and
 *     parallelism");
 *   - delta compression of two models by XOR (Sec. 4.2).
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   - sign bit goes to the MSB of the byte after the exponent (Table 2: the
 *     low FP32 mantissa bytes of clean models compress to 0.0%, so they hold
 *     no sign bit);
 *   - FP16 uses the same 16-bit permutation as BF16 (5 exponent bits + top 3
 *     mantissa bits form the first group; Table 2 FP16 rows);
 *   - code lengths: package-merge (Larmore & Hirschberg 1990) limited to 12
 *     bits, leaves ordered by (count ascending, symbol descending), leaves
 *     before packages on equal weight; canonical codes as in RFC 1951 3.2.2;
 *     table as code-length counts followed by the symbols (JPEG DHT layout).
 *     Two departures from the project's first plan for this step, both format
 *     choices that change no code cost: equal counts are ordered by symbol
 *     descending (the plan had ascending), and the selected lengths are used
 *     as they come out of package-merge, with no second pass that re-sorts
 *     symbols by count and re-deals the sorted lengths;
 *   - raw-vs-Huffman: exact per group-chunk decision with a 1/64 margin;
 *     the paper's skip-ahead probe (Sec. 3.2, "Identifying compressibility")
 *     is an option: after a group-chunk comes out raw, the same group of the
 *     next `skip` chunks is stored raw without being evaluated, then
 *     evaluation resumes ("the specific number varies": skip is a parameter);
 *   - symbols of a group-chunk are dealt to T interleaved sub-streams in
 *     vectors of V = 16/element_size symbols; each sub-stream's start bit is
 *     stored so sub-streams decode independently.
 *
 * Parity status: every function is pinned by tests/test_oracle_pins.py
 * (exhaustive split/merge, numeric exponent fields, Kraft equality, brute
 * force and DP optimality, textbook Huffman equality, dyadic closed forms,
 * hand-derived golden containers, round trips).
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

/* status codes (numeric values fixed by the container specification) */
#define OR_OK        0
#define OR_EINVAL   -1
#define OR_ENOMEM   -2
#define OR_ECORRUPT -3

/* dtypes */
#define OR_BF16 0
#define OR_FP16 1
#define OR_FP32 2
#define OR_U8   3

/* group modes */
#define OR_RAW   0
#define OR_HUFF  1
#define OR_ZERO  2
#define OR_CONST 3
#define OR_SPARSE 4

#define OR_MAXLEN     12      /* code length limit */
#define OR_HDR_BYTES  64
#define OR_ENTRY_BYTES 16
#define OR_FLAG_DELTA 1u
#define OR_MIN_CHUNK  4096u
#define OR_MAX_CHUNK  (16u << 20)
#define OR_MAX_LANES  1024u

/* ------------------------------------------------------------------------ */
/* little-endian field access                                               */

static void put_u16(uint8_t* p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void put_u32(uint8_t* p, uint32_t v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static void put_u64(uint8_t* p, uint64_t v) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static uint32_t get_u16(const uint8_t* p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static uint32_t get_u32(const uint8_t* p) {
    uint32_t v = 0;
    for (int i = 3; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}
static uint64_t get_u64(const uint8_t* p) {
    uint64_t v = 0;
    for (int i = 7; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}
static uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

/* ------------------------------------------------------------------------ */
/* dtype table (Sec. 2.2, Fig. "Representation of FP32, BF16, FP16")          */

int or_elem_size(int dtype) {
    switch (dtype) {
    case OR_BF16: case OR_FP16: return 2;
    case OR_FP32: return 4;
    case OR_U8: return 1;
    default: return 0;
    }
}
int or_n_groups(int dtype) { return or_elem_size(dtype); }

/* default interleave width (a container parameter, no arithmetic of the
 * method): plain 16-bit containers take one sub-stream per 512 bytes of
 * original data (32 vectors of 16 bytes), FP32, U8 and deltas one per 1 KiB;
 * clamped to [1, OR_MAX_LANES] */
static uint32_t default_lanes(int dtype, uint32_t chunk_bytes, int delta) {
    int es = or_elem_size(dtype);
    if (es == 0) return 0;
    uint32_t t = chunk_bytes / ((es == 2 && !delta) ? 512u : 1024u);
    if (t < 1) t = 1;
    if (t > OR_MAX_LANES) t = OR_MAX_LANES;
    return t;
}
uint32_t or_default_lanes(int dtype, uint32_t chunk_bytes) {
    return default_lanes(dtype, chunk_bytes, 0);
}
uint32_t or_default_lanes_delta(int dtype, uint32_t chunk_bytes) {
    return default_lanes(dtype, chunk_bytes, 1);
}

/* ------------------------------------------------------------------------ */
/* Exponent extraction + byte grouping of ONE element (Sec. 3.1, 3.2).
 * The element is read as an unsigned little-endian integer x.
 *   16-bit (BF16, FP16): g0 = bits 14..7 (BF16: the exponent);
 *                        g1 = sign bit (15) followed by bits 6..0.
 *   32-bit (FP32): g0 = bits 30..23 (the exponent);
 *                  g1 = sign bit (31) followed by bits 22..16;
 *                  g2 = bits 15..8; g3 = bits 7..0.
 *   U8: g0 = the byte.                                                       */
void or_split_elem(int dtype, const uint8_t* elem, uint8_t* g) {
    if (dtype == OR_BF16 || dtype == OR_FP16) {
        uint32_t x = get_u16(elem);
        uint32_t sign = (x >> 15) & 1u;
        g[0] = (uint8_t)((x >> 7) & 0xFFu);
        g[1] = (uint8_t)((sign << 7) | (x & 0x7Fu));
    } else if (dtype == OR_FP32) {
        uint32_t x = get_u32(elem);
        uint32_t sign = (x >> 31) & 1u;
        g[0] = (uint8_t)((x >> 23) & 0xFFu);
        g[1] = (uint8_t)((sign << 7) | ((x >> 16) & 0x7Fu));
        g[2] = (uint8_t)((x >> 8) & 0xFFu);
        g[3] = (uint8_t)(x & 0xFFu);
    } else {
        g[0] = elem[0];
    }
}

/* inverse of or_split_elem */
void or_merge_elem(int dtype, const uint8_t* g, uint8_t* elem) {
    if (dtype == OR_BF16 || dtype == OR_FP16) {
        uint32_t sign = (uint32_t)(g[1] >> 7) & 1u;
        uint32_t x = (sign << 15) | ((uint32_t)g[0] << 7) | ((uint32_t)g[1] & 0x7Fu);
        put_u16(elem, x);
    } else if (dtype == OR_FP32) {
        uint32_t sign = (uint32_t)(g[1] >> 7) & 1u;
        uint32_t x = (sign << 31) | ((uint32_t)g[0] << 23) | (((uint32_t)g[1] & 0x7Fu) << 16) |
                     ((uint32_t)g[2] << 8) | (uint32_t)g[3];
        put_u32(elem, x);
    } else {
        elem[0] = g[0];
    }
}

/* split n elements into planes[g * n + i] */
int or_split(int dtype, const uint8_t* src, size_t n, uint8_t* planes) {
    int es = or_elem_size(dtype);
    if (es == 0) return OR_EINVAL;
    int G = or_n_groups(dtype);
    for (size_t i = 0; i < n; i++) {
        uint8_t g[4];
        or_split_elem(dtype, src + i * (size_t)es, g);
        for (int k = 0; k < G; k++) planes[(size_t)k * n + i] = g[k];
    }
    return OR_OK;
}

int or_merge(int dtype, const uint8_t* planes, size_t n, uint8_t* dst) {
    int es = or_elem_size(dtype);
    if (es == 0) return OR_EINVAL;
    int G = or_n_groups(dtype);
    for (size_t i = 0; i < n; i++) {
        uint8_t g[4];
        for (int k = 0; k < G; k++) g[k] = planes[(size_t)k * n + i];
        or_merge_elem(dtype, g, dst + i * (size_t)es);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Length-limited code lengths by package-merge (Larmore & Hirschberg 1990),
 * the Huffman-only coder of Sec. 3.1 with the length limit of 12 bits.
 *
 * Leaves are the symbols with a non-zero count, ordered by (count ascending,
 * symbol descending).  list[0] is the leaves; list[i] is the stable merge of
 * the leaves with the packages of list[i-1] (each package joins two
 * consecutive items from the left; an odd last item is dropped), leaves placed
 * before packages of equal weight.  The first 2(n-1) items of the last list
 * are selected; a selected package selects both of its children in the list
 * below.  A symbol's length is the number of selected items that are its leaf.
 * Returns the number of symbols with a non-zero count (lengths stay 0 for
 * n < 2).                                                                   */
typedef struct { uint64_t w; int leaf; int a, b; } pm_item;

int or_code_lengths(const uint32_t* hist, uint8_t* len) {
    int sym[256];
    int n = 0;
    memset(len, 0, 256);
    for (int s = 255; s >= 0; s--)
        if (hist[s] > 0) sym[n++] = s;           /* symbol descending */
    /* stable insertion sort by count ascending keeps symbol descending on ties */
    for (int i = 1; i < n; i++) {
        int s = sym[i], j = i - 1;
        while (j >= 0 && hist[sym[j]] > hist[s]) { sym[j + 1] = sym[j]; j--; }
        sym[j + 1] = s;
    }
    if (n < 2) return n;

    pm_item list[OR_MAXLEN][512];
    uint8_t sel[OR_MAXLEN][512];
    int size[OR_MAXLEN];

    for (int k = 0; k < n; k++) {
        list[0][k].w = hist[sym[k]];
        list[0][k].leaf = k;
        list[0][k].a = list[0][k].b = -1;
    }
    size[0] = n;
    for (int i = 1; i < OR_MAXLEN; i++) {
        pm_item pkg[256];
        int np = size[i - 1] / 2;
        for (int k = 0; k < np; k++) {
            pkg[k].w = list[i - 1][2 * k].w + list[i - 1][2 * k + 1].w;
            pkg[k].leaf = -1;
            pkg[k].a = 2 * k;
            pkg[k].b = 2 * k + 1;
        }
        int ia = 0, ib = 0, o = 0;
        while (ia < n || ib < np) {
            int take_leaf;
            if (ia >= n) take_leaf = 0;
            else if (ib >= np) take_leaf = 1;
            else take_leaf = (list[0][ia].w <= pkg[ib].w);
            if (take_leaf) list[i][o++] = list[0][ia++];
            else list[i][o++] = pkg[ib++];
        }
        size[i] = o;
    }

    memset(sel, 0, sizeof(sel));
    for (int k = 0; k < 2 * (n - 1); k++) sel[OR_MAXLEN - 1][k] = 1;
    for (int i = OR_MAXLEN - 1; i >= 0; i--) {
        for (int k = 0; k < size[i]; k++) {
            if (!sel[i][k]) continue;
            const pm_item* it = &list[i][k];
            if (it->leaf >= 0) {
                len[sym[it->leaf]]++;
            } else {
                sel[i - 1][it->a] = 1;
                sel[i - 1][it->b] = 1;
            }
        }
    }
    return n;
}

/* Canonical codes from lengths (RFC 1951 Sec. 3.2.2): codes of equal length
 * are consecutive integers in symbol order, and the first code of length l
 * follows the last code of length l-1, shifted left by one.                 */
void or_canonical_codes(const uint8_t* len, uint32_t* code) {
    uint32_t bl_count[OR_MAXLEN + 1] = {0};
    uint32_t next_code[OR_MAXLEN + 2] = {0};
    for (int s = 0; s < 256; s++)
        if (len[s]) bl_count[len[s]]++;
    uint32_t c = 0;
    for (int l = 1; l <= OR_MAXLEN; l++) {
        c = (c + bl_count[l - 1]) << 1;
        next_code[l] = c;
    }
    for (int s = 0; s < 256; s++) {
        code[s] = 0;
        if (len[s]) code[s] = next_code[len[s]]++;
    }
}

/* ------------------------------------------------------------------------ */
/* MSB-first bit writer over 32-bit words (bit k of the stream is bit
 * 31 - (k mod 32) of word k / 32).                                          */
static void put_bits(uint32_t* words, uint64_t pos, uint32_t code, int nbits) {
    for (int k = 0; k < nbits; k++) {
        uint32_t bit = (code >> (nbits - 1 - k)) & 1u;
        uint64_t p = pos + (uint64_t)k;
        words[p >> 5] |= bit << (31 - (p & 31));
    }
}

static uint32_t get_bit(const uint8_t* bitstream, uint64_t p) {
    uint32_t w = get_u32(bitstream + 4 * (p >> 5));
    return (w >> (31 - (p & 31))) & 1u;
}

/* ------------------------------------------------------------------------ */
/* Validation of the user parameters.                                       */
static int check_params(int dtype, size_t nbytes, size_t chunk_bytes, uint32_t lanes) {
    int es = or_elem_size(dtype);
    if (es == 0) return OR_EINVAL;
    if (nbytes % (size_t)es) return OR_EINVAL;
    if (chunk_bytes < OR_MIN_CHUNK || chunk_bytes > OR_MAX_CHUNK || chunk_bytes % 16) return OR_EINVAL;
    if (lanes < 1 || lanes > OR_MAX_LANES || lanes > chunk_bytes / 16) return OR_EINVAL;
    return OR_OK;
}

/* Worst-case container size. */
size_t or_bound(size_t nbytes, int dtype, size_t chunk_bytes) {
    int G = or_n_groups(dtype);
    if (G == 0 || chunk_bytes == 0) return 0;
    size_t nch = (nbytes + chunk_bytes - 1) / chunk_bytes;
    return OR_HDR_BYTES + nch * (size_t)G * OR_ENTRY_BYTES + nbytes + nch * (size_t)G * 16;
}

/* ------------------------------------------------------------------------ */
/* Encoding of one group-chunk of m symbols (the plane of one byte group).
 * Mode rules (Sec. 3.2: zero streams truncated to a header; incompressible
 * streams stored raw):
 *   no symbol, or only the symbol 0x00   -> ZERO   (no payload)
 *   a single distinct non-zero symbol     -> CONST  (the byte in the entry)
 *   else two coded candidates:
 *     HUFF: a code for the histogram of all m symbols; size
 *           h = align4(12+nz) + 4(T-1) + 4*ceil(bits/32);
 *     SPARSE (only if some vector is all zero): a code for the histogram of
 *           the symbols outside all-zero vectors; size
 *           s = align4(12+nz') + 4*ceil(nv/32) + 4(T-1) + 4*ceil(bits'/32)
 *           (the second term is a bitmap of the vectors holding a non-zero
 *           symbol, bit v%32 of little-endian word v/32);
 *   a candidate qualifies when its size + floor(m/64) < m; SPARSE is taken
 *   when it qualifies and is smaller than a qualifying HUFF, HUFF when it
 *   qualifies, else RAW (payload = the m bytes).
 * SPARSE stands in for the paper's switch to Zstd on delta chunks that are
 * mostly zeros (Sec. 4.2, "Auto Detection"): Huffman alone cannot code a
 * symbol in less than one bit.
 * Sub-stream t (0 <= t < T) holds the vectors v = t, t+T, ... of V symbols
 * each (symbol i is in vector i / V; SPARSE leaves out the all-zero vectors);
 * its start bit is stored for t >= 1.
 * Returns the payload size written to out (capacity >= m + 1100 bytes).     */
typedef struct { int mode; int value; size_t size; } or_group_result;

/* table bytes: BITS[12] then the symbols ordered by (length, symbol) */
static size_t write_table(const uint8_t* len, uint8_t* out) {
    int k = 12;
    for (int l = 1; l <= OR_MAXLEN; l++) {
        int cnt = 0;
        for (int s = 0; s < 256; s++)
            if (len[s] == l) { out[k++] = (uint8_t)s; cnt++; }
        out[l - 1] = (uint8_t)cnt;
    }
    return (size_t)k;
}

/* is vector v (symbols v*V .. min(m, v*V+V)-1) all zero? */
static int vector_is_zero(const uint8_t* sym, size_t m, uint32_t V, size_t v) {
    for (size_t i = v * V; i < m && i < (v + 1) * V; i++)
        if (sym[i]) return 0;
    return 1;
}

/* sub-stream start table at offs and MSB-first words at bs; with skip_zero,
 * all-zero vectors contribute no codes */
static void write_streams(const uint8_t* sym, size_t m, uint32_t T, uint32_t V,
                          const uint32_t* code, const uint8_t* len, int skip_zero,
                          size_t nwords, uint8_t* offs, uint8_t* bs) {
    uint32_t* words = (uint32_t*)calloc(nwords + 1, sizeof(uint32_t));
    size_t nv = (m + V - 1) / V;
    uint64_t pos = 0;
    for (uint32_t t = 0; t < T; t++) {
        if (t > 0) put_u32(offs + 4u * (t - 1u), (uint32_t)pos);
        for (size_t v = t; v < nv; v += T) {
            if (skip_zero && vector_is_zero(sym, m, V, v)) continue;
            for (uint32_t j = 0; j < V; j++) {
                size_t i = v * V + j;
                if (i >= m) break;
                put_bits(words, pos, code[sym[i]], len[sym[i]]);
                pos += len[sym[i]];
            }
        }
    }
    for (size_t w = 0; w < nwords; w++) put_u32(bs + 4 * w, words[w]);
    free(words);
}

static or_group_result encode_group(const uint8_t* sym, size_t m, uint32_t T, uint32_t V,
                                   uint8_t* out) {
    or_group_result r = {OR_ZERO, 0, 0};
    uint32_t hist[256] = {0};
    for (size_t i = 0; i < m; i++) hist[sym[i]]++;
    int nz = 0, last = 0;
    for (int s = 0; s < 256; s++)
        if (hist[s]) { nz++; last = s; }
    if (nz == 0 || (nz == 1 && last == 0)) { r.mode = OR_ZERO; return r; }
    if (nz == 1) { r.mode = OR_CONST; r.value = last; return r; }

    /* HUFF candidate */
    uint8_t len[256];
    uint32_t code[256];
    or_code_lengths(hist, len);
    or_canonical_codes(len, code);
    uint64_t bits = 0;
    for (int s = 0; s < 256; s++) bits += (uint64_t)hist[s] * len[s];
    size_t h = (size_t)align_up(12u + (unsigned)nz, 4);
    size_t nwords = (size_t)((bits + 31) / 32);
    size_t s_huff = h + 4u * (T - 1u) + 4u * nwords;
    int huff_ok = s_huff + (m >> 6) < m;

    /* SPARSE candidate: the zeros of all-zero vectors leave the histogram */
    size_t nv = (m + V - 1) / V, zsyms = 0, zvec = 0;
    for (size_t v = 0; v < nv; v++)
        if (vector_is_zero(sym, m, V, v)) {
            zvec++;
            zsyms += (v * V + V <= m) ? V : m - v * V;
        }
    int sparse_ok = 0;
    uint32_t hist2[256];
    uint8_t len2[256];
    uint32_t code2[256];
    size_t h2 = 0, nbw = (nv + 31) / 32, nwords2 = 0, s_sparse = 0;
    if (zvec > 0) {
        memcpy(hist2, hist, sizeof(hist2));
        hist2[0] -= (uint32_t)zsyms;
        int nz2 = 0;
        for (int s = 0; s < 256; s++) nz2 += hist2[s] > 0;
        if (nz2 >= 2) {
            or_code_lengths(hist2, len2);
            or_canonical_codes(len2, code2);
            uint64_t bits2 = 0;
            for (int s = 0; s < 256; s++) bits2 += (uint64_t)hist2[s] * len2[s];
            h2 = (size_t)align_up(12u + (unsigned)nz2, 4);
            nwords2 = (size_t)((bits2 + 31) / 32);
            s_sparse = h2 + 4u * nbw + 4u * (T - 1u) + 4u * nwords2;
            sparse_ok = s_sparse + (m >> 6) < m;
        }
    }

    if (sparse_ok && (!huff_ok || s_sparse < s_huff)) {
        memset(out, 0, s_sparse);
        write_table(len2, out);
        uint8_t* bitmap = out + h2;
        for (size_t v = 0; v < nv; v++)
            if (!vector_is_zero(sym, m, V, v)) bitmap[v / 8] |= (uint8_t)(1u << (v % 8));
        write_streams(sym, m, T, V, code2, len2, 1, nwords2, out + h2 + 4u * nbw,
                      out + h2 + 4u * nbw + 4u * (T - 1u));
        r.mode = OR_SPARSE;
        r.size = s_sparse;
        return r;
    }
    if (!huff_ok) {
        r.mode = OR_RAW;
        r.size = m;
        memcpy(out, sym, m);
        return r;
    }
    memset(out, 0, s_huff);
    write_table(len, out);
    write_streams(sym, m, T, V, code, len, 0, nwords, out + h, out + h + 4u * (T - 1u));
    r.mode = OR_HUFF;
    r.size = s_huff;
    return r;
}

/* Encode the G group-chunks of one chunk (nb bytes of original data, nb a
 * multiple of the element size).  payload[g] receives up to nb/es + 1100
 * bytes.  Used by the container writer and, in tests, to compare single
 * chunks of a large stream.                                                 */
int or_compress_chunk(const uint8_t* src, size_t nb, int dtype, uint32_t lanes,
                      int32_t* modes, int32_t* values, uint64_t* sizes, uint8_t* payloads,
                      size_t payload_stride) {
    int es = or_elem_size(dtype);
    if (es == 0 || nb % (size_t)es || lanes < 1) return OR_EINVAL;
    int G = or_n_groups(dtype);
    size_t m = nb / (size_t)es;
    uint8_t* planes = (uint8_t*)malloc(m * (size_t)G + 1);
    if (!planes) return OR_ENOMEM;
    or_split(dtype, src, m, planes);
    uint32_t V = 16u / (uint32_t)es;
    for (int g = 0; g < G; g++) {
        or_group_result r = encode_group(planes + (size_t)g * m, m, lanes, V,
                                         payloads + (size_t)g * payload_stride);
        modes[g] = r.mode;
        values[g] = r.value;
        sizes[g] = r.size;
    }
    free(planes);
    return OR_OK;
}

/* Whole container (Sec. 5.1 metadata map):
 *   header 64 B: "ZNN1", u16 version 1, u8 dtype, u8 flags, u64 nbytes,
 *     u32 chunk_bytes, u32 lanes, u32 groups, u32 chunks, u64 payload offset,
 *     u64 total bytes, 16 reserved zero bytes;
 *   index: one 16 B entry per (chunk, group): u64 payload offset relative to
 *     the payload area, u32 payload size, u8 mode, u8 value, u16 zero;
 *   payloads in (chunk, group) order, each zero-padded to 16 B.            */
static int compress_impl(const uint8_t* src, size_t nbytes, int dtype, size_t chunk_bytes,
                         uint32_t lanes, uint32_t flags, uint32_t skip, uint8_t* out, size_t cap,
                         size_t* out_size) {
    int rc = check_params(dtype, nbytes, chunk_bytes, lanes);
    if (rc) return rc;
    int es = or_elem_size(dtype);
    int G = or_n_groups(dtype);
    size_t nch = (nbytes + chunk_bytes - 1) / chunk_bytes;
    size_t index_bytes = nch * (size_t)G * OR_ENTRY_BYTES;
    size_t P = OR_HDR_BYTES + index_bytes;
    if (cap < P) return OR_ENOMEM;
    memset(out, 0, P);

    size_t stride = chunk_bytes / (size_t)es + 1100;
    uint8_t* pay = (uint8_t*)malloc(stride * (size_t)G);
    uint8_t* planes = (uint8_t*)malloc(chunk_bytes + 16);
    if (!pay || !planes) { free(pay); free(planes); return OR_ENOMEM; }
    uint32_t skip_left[4] = {0, 0, 0, 0};
    uint64_t cursor = 0;
    for (size_t c = 0; c < nch; c++) {
        size_t off = c * chunk_bytes;
        size_t nb = nbytes - off < chunk_bytes ? nbytes - off : chunk_bytes;
        int32_t modes[4], values[4];
        uint64_t sizes[4];
        or_compress_chunk(src + off, nb, dtype, lanes, modes, values, sizes, pay, stride);
        if (skip) {
            /* skip-ahead probe: a group inside its skip window is stored raw
             * (its evaluation above is discarded); a group evaluated raw opens
             * a window over the next `skip` chunks */
            size_t m = nb / (size_t)es;
            or_split(dtype, src + off, m, planes);
            for (int g = 0; g < G; g++) {
                if (skip_left[g] > 0) {
                    skip_left[g]--;
                    modes[g] = OR_RAW;
                    values[g] = 0;
                    sizes[g] = m;
                    memcpy(pay + (size_t)g * stride, planes + (size_t)g * m, m);
                } else if (modes[g] == OR_RAW) {
                    skip_left[g] = skip;
                }
            }
        }
        for (int g = 0; g < G; g++) {
            uint8_t* e = out + OR_HDR_BYTES + (c * (size_t)G + (size_t)g) * OR_ENTRY_BYTES;
            put_u64(e, cursor);
            put_u32(e + 8, (uint32_t)sizes[g]);
            e[12] = (uint8_t)modes[g];
            e[13] = (uint8_t)values[g];
            size_t padded = (size_t)align_up(sizes[g], 16);
            if (P + cursor + padded > cap) { free(pay); free(planes); return OR_ENOMEM; }
            memset(out + P + cursor, 0, padded);
            memcpy(out + P + cursor, pay + (size_t)g * stride, sizes[g]);
            cursor += padded;
        }
    }
    free(pay);
    free(planes);
    uint8_t* h = out;
    h[0] = 'Z'; h[1] = 'N'; h[2] = 'N'; h[3] = '1';
    put_u16(h + 4, 1);
    h[6] = (uint8_t)dtype;
    h[7] = (uint8_t)flags;
    put_u64(h + 8, nbytes);
    put_u32(h + 16, (uint32_t)chunk_bytes);
    put_u32(h + 20, lanes);
    put_u32(h + 24, (uint32_t)G);
    put_u32(h + 28, (uint32_t)nch);
    put_u64(h + 32, P);
    put_u64(h + 40, P + cursor);
    *out_size = P + cursor;
    return OR_OK;
}

int or_compress(const uint8_t* src, size_t nbytes, int dtype, size_t chunk_bytes, uint32_t lanes,
                uint8_t* out, size_t cap, size_t* out_size) {
    return compress_impl(src, nbytes, dtype, chunk_bytes, lanes, 0, 0, out, cap, out_size);
}

/* Compression with the skip-ahead probe (Sec. 3.2, "Identifying
 * compressibility"): skip = chunks stored raw after a raw group-chunk. */
int or_compress_skip(const uint8_t* src, size_t nbytes, int dtype, size_t chunk_bytes,
                     uint32_t lanes, uint32_t skip, uint8_t* out, size_t cap, size_t* out_size) {
    return compress_impl(src, nbytes, dtype, chunk_bytes, lanes, 0, skip, out, cap, out_size);
}

/* Delta (Sec. 4.2): the container of a XOR b, flagged DELTA. */
int or_delta(const uint8_t* a, const uint8_t* b, size_t nbytes, int dtype, size_t chunk_bytes,
             uint32_t lanes, uint8_t* out, size_t cap, size_t* out_size) {
    uint8_t* x = (uint8_t*)malloc(nbytes + 1);
    if (!x) return OR_ENOMEM;
    for (size_t i = 0; i < nbytes; i++) x[i] = (uint8_t)(a[i] ^ b[i]);
    int rc = compress_impl(x, nbytes, dtype, chunk_bytes, lanes, OR_FLAG_DELTA, 0, out, cap,
                           out_size);
    free(x);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Decoding.  Each HUFF sub-stream is decoded bit by bit with the canonical
 * rule: after reading l bits the value c is a code of length l iff
 * first[l] <= c < first[l] + count[l].                                       */
static int decode_group(const uint8_t* p, size_t size, size_t m, uint32_t T, uint32_t V,
                        int sparse, uint8_t* sym) {
    if (size < 12) return OR_ECORRUPT;
    uint32_t count[OR_MAXLEN + 1] = {0};
    int nz = 0;
    for (int l = 1; l <= OR_MAXLEN; l++) { count[l] = p[l - 1]; nz += (int)count[l]; }
    if (nz < 2 || nz > 256) return OR_ECORRUPT;
    uint64_t kraft = 0;
    for (int l = 1; l <= OR_MAXLEN; l++) kraft += (uint64_t)count[l] << (OR_MAXLEN - l);
    if (kraft > (1u << OR_MAXLEN)) return OR_ECORRUPT;
    size_t h = (size_t)align_up(12u + (unsigned)nz, 4);
    size_t nv = (m + V - 1) / V;
    const uint8_t* bitmap = p + h;                 /* SPARSE: one bit per vector */
    if (sparse) h += 4u * ((nv + 31) / 32);
    if (size < h + 4u * (T - 1u) || (size - h - 4u * (T - 1u)) % 4) return OR_ECORRUPT;
    if (sparse)
        for (size_t v = nv; v < (nv + 31) / 32 * 32; v++)
            if (bitmap[v / 8] >> (v % 8) & 1u) return OR_ECORRUPT;   /* bits past nv */
    const uint8_t* symbols = p + 12;
    uint8_t seen[256] = {0};
    for (int k = 0; k < nz; k++) {
        if (seen[symbols[k]]) return OR_ECORRUPT;
        seen[symbols[k]] = 1;
    }
    uint32_t first[OR_MAXLEN + 2] = {0}, index[OR_MAXLEN + 2] = {0};
    uint32_t c = 0, idx = 0;
    for (int l = 1; l <= OR_MAXLEN; l++) {
        c = (c + count[l - 1]) << 1;
        first[l] = c;
        index[l] = idx;
        idx += count[l];
    }
    const uint8_t* offs = p + h;
    const uint8_t* bs = p + h + 4u * (T - 1u);
    uint64_t total_bits = (uint64_t)(size - h - 4u * (T - 1u)) * 8u;
    uint64_t pos = 0;
    for (uint32_t t = 0; t < T; t++) {
        uint64_t start = t ? get_u32(offs + 4u * (t - 1u)) : 0;
        if (start != pos) return OR_ECORRUPT;      /* sub-streams are contiguous */
        for (size_t v = t; v < nv; v += T) {
            if (sparse && !(bitmap[v / 8] >> (v % 8) & 1u)) {   /* all-zero vector */
                for (size_t i = v * V; i < m && i < (v + 1) * V; i++) sym[i] = 0;
                continue;
            }
            for (uint32_t j = 0; j < V; j++) {
                size_t i = v * V + j;
                if (i >= m) break;
                uint32_t code = 0;
                int found = 0;
                for (int l = 1; l <= OR_MAXLEN; l++) {
                    if (pos >= total_bits) return OR_ECORRUPT;
                    code = (code << 1) | get_bit(bs, pos);
                    pos++;
                    if (code - first[l] < count[l]) {
                        sym[i] = symbols[index[l] + (code - first[l])];
                        found = 1;
                        break;
                    }
                }
                if (!found) return OR_ECORRUPT;
            }
        }
    }
    if ((pos + 31) / 32 * 32 != total_bits) return OR_ECORRUPT;  /* no extra words */
    for (uint64_t q = pos; q < total_bits; q++)
        if (get_bit(bs, q)) return OR_ECORRUPT;                 /* zero padding */
    return OR_OK;
}

/* Parse the header; returns OR_OK and fills fields if valid. */
int or_parse_header(const uint8_t* s, size_t n, int32_t* dtype, uint32_t* flags, uint64_t* nbytes,
                    uint32_t* chunk_bytes, uint32_t* lanes, uint32_t* n_chunks) {
    if (n < OR_HDR_BYTES) return OR_ECORRUPT;
    if (s[0] != 'Z' || s[1] != 'N' || s[2] != 'N' || s[3] != '1') return OR_ECORRUPT;
    if (get_u16(s + 4) != 1) return OR_ECORRUPT;
    int dt = s[6];
    if (or_elem_size(dt) == 0) return OR_ECORRUPT;
    if (s[7] & ~OR_FLAG_DELTA) return OR_ECORRUPT;
    uint64_t nb = get_u64(s + 8);
    uint32_t C = get_u32(s + 16), T = get_u32(s + 20), G = get_u32(s + 24), nch = get_u32(s + 28);
    if (check_params(dt, nb, C, T)) return OR_ECORRUPT;
    if (G != (uint32_t)or_n_groups(dt)) return OR_ECORRUPT;
    if ((uint64_t)nch != (nb + C - 1) / C) return OR_ECORRUPT;
    uint64_t P = get_u64(s + 32), total = get_u64(s + 40);
    if (P != OR_HDR_BYTES + (uint64_t)nch * G * OR_ENTRY_BYTES) return OR_ECORRUPT;
    if (total != n || total < P) return OR_ECORRUPT;
    for (int k = 48; k < 64; k++)
        if (s[k]) return OR_ECORRUPT;
    *dtype = dt;
    *flags = s[7];
    *nbytes = nb;
    *chunk_bytes = C;
    *lanes = T;
    *n_chunks = nch;
    return OR_OK;
}

int or_decompress(const uint8_t* s, size_t n, const uint8_t* base, uint8_t* dst, size_t dst_n) {
    int32_t dtype;
    uint32_t flags, C, T, nch;
    uint64_t nbytes;
    int rc = or_parse_header(s, n, &dtype, &flags, &nbytes, &C, &T, &nch);
    if (rc) return rc;
    if (dst_n != nbytes) return OR_EINVAL;
    if (((flags & OR_FLAG_DELTA) != 0) != (base != NULL)) return OR_EINVAL;  /* base iff DELTA */
    int es = or_elem_size(dtype);
    int G = or_n_groups(dtype);
    uint32_t V = 16u / (uint32_t)es;
    uint64_t P = get_u64(s + 32);
    size_t mmax = C / (size_t)es;
    uint8_t* planes = (uint8_t*)malloc(mmax * (size_t)G + 1);
    if (!planes) return OR_ENOMEM;
    uint64_t cursor = 0;
    for (uint32_t c = 0; c < nch; c++) {
        size_t off = (size_t)c * C;
        size_t nb = nbytes - off < C ? nbytes - off : C;
        size_t m = nb / (size_t)es;
        for (int g = 0; g < G; g++) {
            const uint8_t* e = s + OR_HDR_BYTES + ((size_t)c * (size_t)G + (size_t)g) * OR_ENTRY_BYTES;
            uint64_t po = get_u64(e);
            uint32_t size = get_u32(e + 8);
            int mode = e[12], value = e[13];
            if (e[14] || e[15] || po != cursor) { free(planes); return OR_ECORRUPT; }
            uint64_t padded = align_up(size, 16);
            if (P + po + padded > n) { free(planes); return OR_ECORRUPT; }
            const uint8_t* p = s + P + po;
            for (uint64_t q = size; q < padded; q++)
                if (p[q]) { free(planes); return OR_ECORRUPT; }
            uint8_t* dstp = planes + (size_t)g * m;
            if (mode == OR_ZERO) {
                if (size || value) { free(planes); return OR_ECORRUPT; }
                memset(dstp, 0, m);
            } else if (mode == OR_CONST) {
                if (size || value == 0) { free(planes); return OR_ECORRUPT; }
                memset(dstp, value, m);
            } else if (mode == OR_RAW) {
                if (size != m || value) { free(planes); return OR_ECORRUPT; }
                memcpy(dstp, p, m);
            } else if (mode == OR_HUFF || mode == OR_SPARSE) {
                if (value) { free(planes); return OR_ECORRUPT; }
                rc = decode_group(p, size, m, T, V, mode == OR_SPARSE, dstp);
                if (rc) { free(planes); return rc; }
            } else {
                free(planes);
                return OR_ECORRUPT;
            }
            cursor += padded;
        }
        or_merge(dtype, planes, m, dst + off);
        if (flags & OR_FLAG_DELTA)
            for (size_t i = 0; i < nb; i++) dst[off + i] ^= base[off + i];
    }
    free(planes);
    if (P + cursor != n) return OR_ECORRUPT;
    return OR_OK;
}

int or_version(void) { return 1; }
