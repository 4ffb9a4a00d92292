/*
 * pc.h - C ABI of the GB300 particle position compressor.
 *
 * The library implements the hot path of the error-bounded, bit-adaptive
 * particle compressor of Ren, Di, Zhang, Zhao and Guo (arXiv 2404.02826):
 *   - per-particle quantization of xyz onto a lattice of step 2*eb' (Sec. 3,
 *     linear-scale quantization, Eq. 1), origin at the per-axis minimum;
 *   - a median k-d partition into subregions of at most r particles (Sec. 4.1,
 *     "initial particle partitioning"; axis = depth mod 3, the median on the
 *     larger-coordinate side);
 *   - one bit box per subregion: the particle closest to the AABB centre and
 *     the bits per axis m_d of Eq. 2 (Sec. 4.1, "bit box construction");
 *   - the codes of every particle packed at those widths into one stream
 *     (Sec. 4.2, Fig. 4 data layout), and the inverse unpack and dequantize.
 * Everything runs in hand-written CUDA kernels for sm_103a on one GPU.
 *
 * Conventions
 *   - All data pointers are DEVICE pointers unless the name starts with host_.
 *     The caller owns every buffer; no call allocates or frees device memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Positions are array-of-structs T[n][3] (x, y, z), T = float or double,
 *     naturally aligned (4 or 8 bytes); 16-byte alignment selects vector loads.
 *   - Every call returns a pc_status.  After an error no output is valid.
 *   - Calls are synchronous with respect to the host where stated: compress
 *     and decompress each read a few bytes back (the value range, then the
 *     final size or the error word) and so return with their work finished.
 *     Those bytes pass through page-locked host blocks of 4 KB that the
 *     library allocates on first use, sixteen at a time, and keeps for the
 *     life of the process (one block per call in flight; decompression also
 *     keeps one CUDA event per call in flight); pc_compress_noalloc allocates
 *     none (it uses blocks that exist, else plain copies).
 *
 * Stream format (little-endian), version 1:
 *   header, 96 bytes:
 *      0 char[4] "PCB1"   4 u16 version   6 u8 dtype   7 u8 eb_mode
 *      8 u64 n            16 f64 eb (as given)          24 f64 eps (absolute bound)
 *     32 f64 s (lattice step)                           40 f64 o[3] (origin)
 *     64 u64 num_leaves   72 u64 payload_words          80 u32 leaf_size
 *     84 u8 lossless-axis mask (bit d: axis d)              85..95 zero
 *   leaf table, 32 bytes per leaf (one sequence of Fig. 4 each), in k-d order:
 *      0 u64 index of the leaf's first decoded particle
 *      8 u64 index of the leaf's first payload word
 *     16 i32 q_ref[3] (lattice code of the bit-box centre; 0 on a lossless axis)
 *     28 u8 m[3] (bits per axis, 0..31; M = 32 or 64 on a lossless axis)   31 u8 zero
 *   payload: u32 words.  Each leaf starts on a word boundary; its non-centre
 *     particles follow in leaf order as c_x (m_x bits), c_y, c_z, packed least
 *     significant bit first, with c_d = (q_d - q_ref_d) + 2^(m_d-1) - 1.
 *   Lossless axes (Sec. 4.1: a dimension whose m_d would exceed M, M = 32 for
 *     float and 64 for double, is stored as the original coordinates).  Codes
 *     here have at most 30 bits (m_d <= 31); an axis whose code range reaches
 *     2^30, or every axis when eps is below the rounding margin of the type
 *     (no lattice keeps the bound through the rounding to T), is stored
 *     losslessly in every leaf.  Then every leaf's payload holds all its
 *     particles, the centre first, and a lossless field is the coordinate's
 *     M-bit pattern.  The tree splits such an axis on the key
 *     floor((p - min) / (max - min) * 2^29).  The bit-box reduction, the
 *     reordering and the leaf-size search need codes on every axis and return
 *     PC_ERR_EB_TOO_SMALL or PC_ERR_RANGE for such inputs.
 *   Stream size = 96 + 32 * num_leaves + 4 * payload_words bytes.
 *   Decoding emits, leaf by leaf, the centre and then the other particles;
 *   particle order is not preserved (the paper keeps positions only, Sec. 2).
 */
#ifndef PC_H
#define PC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PC_OK = 0,
    PC_ERR_ARG = 1,          /* null pointer, bad dtype/mode, eb <= 0 or not finite, n >= 2^31, bad leaf size, misalignment */
    PC_ERR_NONFINITE = 2,    /* NaN or Inf among the positions */
    PC_ERR_EB_TOO_SMALL = 3, /* eb' = eps - ulp_T(M2) - 4 ulp_f64(M2) <= 0, M2 = 2 max(max|p|, eps), with the
                                bit-box reduction, the reordering or the leaf-size search (the plain stream
                                stores such axes losslessly) */
    PC_ERR_RANGE = 4,        /* M2 above the largest finite T; or some code >= 2^30 with the reduction,
                                the reordering or the leaf-size search */
    PC_ERR_CAPACITY = 5,     /* output or workspace too small */
    PC_ERR_CORRUPT = 6,      /* stream fails validation (magic, version, sizes, widths, offsets) */
    PC_ERR_TIMEOUT = 7,      /* a bounded device wait expired; the output is invalid */
    PC_ERR_CUDA = 8          /* a CUDA runtime call failed */
} pc_status;

typedef enum { PC_F32 = 0, PC_F64 = 1 } pc_dtype;

/* Error-bound modes of Sec. 3: absolute |p - p_hat| <= eb per coordinate, or
 * value-range-relative eps = eb * Delta_max, Delta_max = max over axes of (max - min). */
typedef enum { PC_EB_ABS = 0, PC_EB_REL = 1 } pc_eb_mode;

/* Tuning knobs.  A NULL config means defaults. */
typedef struct {
    uint32_t leaf_size; /* r of Sec. 4.1: largest leaf; 0 = 4096; valid 1..PC_MAX_LEAF_SIZE.
                           With PC_FLAG_AUTOTUNE_LEAF: the largest candidate (0 = PC_MAX_LEAF_SIZE) */
    uint32_t flags;     /* 0, or any of PC_FLAG_AUTOTUNE_LEAF, PC_FLAG_BOX_REDUCTION, PC_FLAG_REORDER,
                           PC_FLAG_WIDEST_AXIS, PC_FLAG_AUTOTUNE_KNOBS */
    /* The two launch knobs below change how many threads work on one node or
     * one leaf, never a byte of the stream (no counterpart in the paper). */
    uint32_t warp_node_max; /* threads per node: in the k-d levels over HBM, nodes of at most this many
                               particles are split by one warp each (32 threads, one pass, no tiles), larger
                               ones by 512-thread blocks over tiles (count, tile scan, scatter passes);
                               0 = PC_DEFAULT_WARP_NODE_MAX; valid 1..PC_MAX_WARP_NODE_MAX */
    uint32_t warp_leaf_max; /* packing tile: when the leaves' bit boxes and packing run over HBM (the
                               leaf-size search, the reduction, the reordering, lossless axes), leaves of
                               at most this size (r) get one warp each, larger ones a 256-thread block each;
                               0 = PC_DEFAULT_WARP_LEAF_MAX; valid 1..PC_MAX_LEAF_SIZE */
} pc_config;

#define PC_DEFAULT_WARP_NODE_MAX 2048u
#define PC_MAX_WARP_NODE_MAX 65536u
#define PC_DEFAULT_WARP_LEAF_MAX 1024u

/* Leaf-size autotuning (no counterpart in the paper, which fixes r by hand,
 * Sec. 5): the leaves of the median tree for r = ceil(n / 2^d) are its nodes
 * at depth d, so the tree for a smaller leaf size extends the one for a larger
 * size.  With this flag compression builds the tree level by level from the
 * largest candidate depth on, computes the exact stream size of every
 * candidate depth d (leaf records + packed words) as it reaches it, and keeps
 * descending while the size shrinks; the stream uses the last depth before it
 * grows, r = ceil(n / 2^d), within [min(PC_AUTOTUNE_MIN_LEAF, max), max] with
 * max = leaf_size.  The header records that r, and a plain call with it
 * gives the same stream. */
#define PC_FLAG_AUTOTUNE_LEAF 1u

/* Bit-box reduction (Sec. 4.1, "bit box reduction and bit box intersection
 * update"; Alg. 1).  Starting from the leaves' bit boxes, boxes are emitted as
 * sequences in rounds: a round takes every alive box whose key (m_x + m_y +
 * m_z, then box index) is smaller than that of every other alive box its bit
 * box meets (such boxes are pairwise disjoint).  Each taken box becomes a
 * sequence holding its centre, its remaining particles, then the particles of
 * the other boxes it meets that lie inside its bit box (by source box, then
 * leaf order), coded with its widths.  Boxes that lost particles get the bit
 * box of what they keep (the leaf rules); empty boxes vanish.  Sequences are
 * written in round order, then box index, in place of the leaves: the stream
 * format and the decoder are unchanged, a sequence may hold more than r
 * particles, and there are at most as many sequences as leaves.  The paper
 * takes one box (the smallest key) at a time; taking all local minima per
 * round is this library's reading, which lets a round run in parallel.
 * Combined with PC_FLAG_AUTOTUNE_LEAF, the leaf size is chosen first (on the
 * plain stream size) and the reduction runs on those leaves. */
#define PC_FLAG_BOX_REDUCTION 2u

/* Reordering for an entropy coder (Sec. 4.2, after Fig. 4): the sequences
 * (leaves, or the reduction's sequences) are written in increasing order of
 * m_x + m_y + m_z, and the particles of each sequence, centre first, in
 * increasing order of their R-index: the particle's three codes joined, most
 * significant first, in the order of the axes' entropy levels (the entropy of
 * the distribution of m_d over all sequences, lowest first; entropies within
 * 1e-9 keep x, y, z order).  Equal keys keep their previous order.  The stream
 * format, its size and the decoder are unchanged (the decoded set is the
 * same, in another order; perm follows it).  The paper then entropy-codes the
 * stream (Huffman, ZSTD); that step is not part of this library. */
#define PC_FLAG_REORDER 4u

/* Split-axis variant of the k-d partition (Sec. 4.1 leaves the axis open;
 * the default is depth mod 3): every node splits on the axis along which its
 * cell is widest, the lowest axis of equal widths.  The root's cell spans the
 * codes [0, max code] per axis; a split at median code v gives the left child
 * the cell up to v and the right child the cell from v on, on that axis.  The
 * median rule, the leaves and the stream format are unchanged; the decoder
 * does not need to know the rule. */
#define PC_FLAG_WIDEST_AXIS 8u

/* Launch-knob autotuning (no counterpart in the paper): the autotuner's choice
 * of threads per node (warp_node_max) and packing tile (warp_leaf_max).  Calls
 * are grouped in classes by the bit length of n, dtype, the current CUDA
 * device, the other flags and leaf_size.  The first call of a class writes its
 * stream with the config's own knobs (the defaults for 0), then compresses
 * the same input again under each candidate that
 * changes the launches for that input (threads per node 512 .. 8192, then
 * packing tile 256 .. 4096 with the best threads per node; each timed on the
 * host clock, best of two) and keeps the fastest for the class; later calls of
 * the class run with it.  While one call of a class is tuning, other calls of
 * that class run with their config's own knobs.  The stream is the same under every
 * candidate (the tuner checks its size).  pc_tuned_config reports a class's
 * choice as a config for a plain call, which then makes the same launches and
 * writes the same stream.  The timing runs reuse the call's output, workspace
 * and perm, so a tuning call costs up to about twenty compressions. */
#define PC_FLAG_AUTOTUNE_KNOBS 16u
#define PC_AUTOTUNE_MIN_LEAF 64u

#define PC_DEFAULT_LEAF_SIZE 4096u
#define PC_MAX_LEAF_SIZE 12000u
#define PC_MAX_PARTICLES 2147483647ull /* n < 2^31 */
#define PC_HEADER_BYTES 96u
#define PC_LEAF_BYTES 32u

/* Decoded header (host structure). */
typedef struct {
    uint64_t n;
    uint32_t dtype;   /* pc_dtype */
    uint32_t eb_mode; /* pc_eb_mode */
    double eb;        /* bound as given to pc_compress */
    double eps;       /* absolute bound every coordinate honours */
    double s;         /* lattice step */
    double o[3];      /* lattice origin */
    uint64_t num_leaves;
    uint64_t payload_words;
    uint32_t leaf_size;
    uint64_t total_bytes; /* 96 + 32 num_leaves + 4 payload_words */
    uint32_t lossless_axes; /* bit d: axis d stored as the original coordinates (Sec. 4.1, m_d > M) */
} pc_info;

/* Worst-case stream size for n particles with this config, in bytes (host only). */
int pc_compress_bound(uint64_t n, int dtype, const pc_config *cfg, uint64_t *out_bytes);

/* Device scratch needed by pc_compress, in bytes (host only).  It always has
 * room for the input indices (the permutation output needs them, and so do
 * lossless axes, which only the value range reveals); with_perm is accepted
 * for compatibility and does not change the size. */
int pc_compress_workspace_size(uint64_t n, int dtype, const pc_config *cfg, int with_perm, uint64_t *out_bytes);

/* Compress n particles (Sec. 3, Sec. 4.1, Sec. 4.2).
 *   positions  device, T[n][3]
 *   out        device, at least pc_compress_bound bytes (16-byte aligned)
 *   out_size   host, receives the stream size in bytes
 *   workspace  device scratch of pc_compress_workspace_size bytes (256-byte aligned)
 *   perm       optional device u32[n]: perm[i] = input index of decoded particle i
 * Returns after the stream is complete on `stream`.  Every coordinate decodes
 * within eps of its input: eps = eb (PC_EB_ABS) or eb * Delta_max (PC_EB_REL). */
int pc_compress(const void *positions, uint64_t n, int dtype, int eb_mode, double eb, const pc_config *cfg,
                void *out, uint64_t out_capacity, uint64_t *out_size, void *workspace, uint64_t workspace_bytes,
                uint32_t *perm, void *stream);

/* The launch knobs PC_FLAG_AUTOTUNE_KNOBS uses for calls of the class of
 * (n, dtype, cfg) (no counterpart in the paper; host only, no device work):
 * *out = *cfg without that flag,
 * with warp_node_max and warp_leaf_max set to the class's tuned values, or to
 * cfg's own (defaults for 0) while the class is untuned.  *tuned = 1 when the
 * class has been tuned, else 0.  A pc_compress with *out makes the launches the
 * tuned calls make and writes the same stream.  cfg must carry the flag. */
int pc_tuned_config(uint64_t n, int dtype, const pc_config *cfg, pc_config *out, int *tuned);

/* Forget every class's tuned knobs (no counterpart in the paper; host only);
 * classes tune again on their next PC_FLAG_AUTOTUNE_KNOBS call. */
int pc_autotune_reset(void);

/* One tuned class of PC_FLAG_AUTOTUNE_KNOBS, as saved and restored (no
 * counterpart in the paper).  A later process can load the tuned classes
 * instead of timing them again. */
typedef struct {
    uint32_t n_bits;        /* bit length of n (0..31) */
    int32_t dtype;          /* pc_dtype */
    int32_t device;         /* CUDA device number (0..255) */
    uint32_t flags;         /* the class's flags, without PC_FLAG_AUTOTUNE_KNOBS */
    uint32_t leaf_size;     /* pc_config.leaf_size of the class */
    uint32_t warp_node_max; /* the tuned knobs */
    uint32_t warp_leaf_max;
    uint32_t reserved;      /* zero */
} pc_tuned_class;

/* Copy the tuned classes out (host only): up to `capacity` entries into
 * `out` (may be NULL when capacity is 0); *count receives the number of tuned
 * classes, which may exceed capacity.  Classes being tuned are not listed. */
int pc_autotune_export(pc_tuned_class *out, uint32_t capacity, uint32_t *count);

/* Enter classes as tuned (host only), replacing any entry of the same class;
 * later PC_FLAG_AUTOTUNE_KNOBS calls of those classes run with them.  Every
 * entry is checked first (n_bits <= 31, dtype, device 0..255, known flags
 * without PC_FLAG_AUTOTUNE_KNOBS, leaf_size and knobs within their ranges,
 * knobs nonzero, reserved zero): PC_ERR_ARG enters none.  PC_ERR_CAPACITY
 * when the table (256 classes) has no room for all new classes; none is
 * entered then either. */
int pc_autotune_import(const pc_tuned_class *classes, uint32_t count);

/* Compression for callers that may not allocate device memory (the paper has
 * no counterpart; this is a deployment convenience).  Examples are code running
 * inside another framework's memory pool that is only handed its input and
 * output buffers, and latency-critical paths where cudaMalloc / cudaFree could
 * synchronise the device.  It behaves like pc_compress without `perm`, but its
 * scratch is a library-owned static device array of PC_NOALLOC_SCRATCH_BYTES
 * (48 MiB) that each GPU using it keeps until the process exits:
 *   - problems whose scratch exceeds the array (above about 2^20 particles at
 *     the default leaf size; pc_compress_workspace_size tells) return
 *     PC_ERR_CAPACITY before any work;
 *   - the first call on a device looks up the array's device address and
 *     caches it: make that first call before any stream capture; a
 *     cudaDeviceReset of that device invalidates the cached address, so the
 *     entry point must not be called on it after such a reset;
 *   - all calls on a device share the array; what must start at zero is
 *     cleared by every call, but calls that overlap on the GPU race on it and
 *     must be serialised by the caller;
 *   - with PC_FLAG_AUTOTUNE_KNOBS it runs with a class's tuned launch knobs
 *     when that class has been tuned by another entry point, but never tunes;
 *   - no allocation happens while kernel tracing (pc_trace_enable) is off. */
#define PC_NOALLOC_SCRATCH_BYTES (48u << 20)
int pc_compress_noalloc(const void *positions, uint64_t n, int dtype, int eb_mode, double eb, const pc_config *cfg,
                        void *out, uint64_t out_capacity, uint64_t *out_size, void *stream);

/* Self-test of the library's bounded device waits (no counterpart in the
 * paper): one block waits on a shared-memory barrier that nothing completes,
 * through the same bounded wait the partition uses for its tile copies (with a
 * short poll limit).  The wait gives up, the kernel returns, and the call
 * returns PC_ERR_TIMEOUT with the context intact; any other status means the
 * mechanism failed.  Synchronous on `stream`. */
int pc_selftest_wait_timeout(void *stream);

/* Self-test of the partition's behaviour when a tile copy never lands (no
 * counterpart in the paper): one pc_compress of the given positions (value-
 * range-relative bound 1e-3, default configuration) in which the partition's
 * scatter issues no tile copy and waits at most 2^12 polls for each.  Every
 * scatter block gives up on its first tile and leaves; the kernels after it
 * see the error word and do nothing; the call returns PC_ERR_TIMEOUT and the
 * context stays usable.  Arguments and workspace as for pc_compress (device
 * pointers); the output holds nothing valid afterwards.  The copies are
 * dropped only for calls made from the calling host thread while this one
 * runs.  n must exceed 2^16, so that the first level runs the tiled scatter. */
int pc_selftest_scatter_timeout(const void *positions, uint64_t n, int dtype, void *out, uint64_t out_capacity,
                                void *workspace, uint64_t workspace_bytes, void *stream);

/* Parse a stream header held in host memory (the first 96 bytes suffice). */
int pc_stream_info(const void *host_header, uint64_t header_bytes, pc_info *info);

/* Device scratch needed by pc_decompress for a stream of n particles
 * (pc_info.n), in bytes (host only). */
int pc_decompress_workspace_size(uint64_t n, uint64_t *out_bytes);

/* Decompress a device stream into T[n][3] positions (Sec. 3 dequantization,
 * p_hat = (T)(o + s q) with one double multiply and one double add).
 *   stream_data     device, stream_bytes long (16-byte aligned)
 *   out_positions   device, out_capacity_bytes >= 3 * sizeof(T) * n
 *   workspace       device scratch of pc_decompress_workspace_size bytes
 * Validates the header and the leaf table; returns PC_ERR_CORRUPT on any
 * inconsistency without writing outside the given buffers. */
int pc_decompress(const void *stream_data, uint64_t stream_bytes, void *out_positions, uint64_t out_capacity_bytes,
                  void *workspace, uint64_t workspace_bytes, void *stream);

/* Host-buffer variants: the same operations on HOST positions and streams
 * (pinned memory gives the fastest copies).  The device workspace holds the
 * staged input and output as well as the scratch; size it with the
 * *_host_workspace_size calls.  Copies run on `stream` inside the call. */
int pc_compress_host_workspace_size(uint64_t n, int dtype, const pc_config *cfg, uint64_t *out_bytes);
int pc_compress_host(const void *host_positions, uint64_t n, int dtype, int eb_mode, double eb, const pc_config *cfg,
                     void *host_out, uint64_t out_capacity, uint64_t *out_size, void *workspace,
                     uint64_t workspace_bytes, void *stream);
int pc_decompress_host_workspace_size(uint64_t n, int dtype, uint64_t stream_bytes, uint64_t *out_bytes);
int pc_decompress_host(const void *host_stream, uint64_t stream_bytes, void *host_positions,
                       uint64_t out_capacity_bytes, void *workspace, uint64_t workspace_bytes, void *stream);

/* ---- Leaf-size sweep -----------------------------------------------------------
 * The stream size and its parts for every leaf size r = ceil(n / 2^d) in
 * [r_min, r_max] (16 <= r_min <= r_max <= PC_MAX_LEAF_SIZE), from one descent
 * of the median tree: the paper's study of the layout size against the leaf
 * fraction r / n (Sec. 4.2 storage cost, Sec. 5 parameter analysis), here
 * for this stream format.  Writes no stream.  points[i] for the i-th
 * candidate from the largest leaves down, at most `capacity`; *count is the
 * number of candidates. */
typedef struct {
    uint32_t leaf_size;      /* ceil(n / 2^depth) */
    uint32_t depth;
    uint64_t leaves;         /* 2^depth sequences */
    uint64_t header_bytes;   /* 96 */
    uint64_t table_bytes;    /* 32 per sequence: centre code, widths, offsets */
    uint64_t payload_bytes;  /* packed codes, each sequence rounded up to words */
    uint64_t total_bytes;
} pc_sweep_point;

int pc_leaf_size_sweep_workspace_size(uint64_t n, int dtype, uint32_t r_min, uint32_t r_max, uint64_t *out_bytes);
int pc_leaf_size_sweep(const void *positions, uint64_t n, int dtype, int eb_mode, double eb, uint32_t r_min,
                       uint32_t r_max, pc_sweep_point *points, uint32_t capacity, uint32_t *count, void *workspace,
                       uint64_t workspace_bytes, void *stream);

/* ---- Many snapshots --------------------------------------------------------
 * The paper compresses one snapshot at a time; nothing below has a
 * counterpart in it.
 * Compression runs many independent snapshots on one GPU through `lanes` CUDA
 * streams, each driven by its own host thread and owning one slice of the
 * workspace; items are taken largest first, so small snapshots overlap on the
 * device with each other and with large ones, and an item runs the plain
 * call's kernels in the plain call's order.
 * Decompression runs every item in one set of launches on `stream` (`lanes` is
 * not used): the headers are gathered and read back once, the leaves of all
 * streams are validated in one launch and their code tables built in one, and
 * the chunks of all streams of one kind (float32, float64) are decoded by one
 * persistent launch; streams with lossless axes decode one launch each.
 * Either way each item's stream (or positions) is byte-identical to a plain
 * pc_compress (or pc_decompress) of the same input.  Work queued on `stream`
 * before the call completes before any item starts; every item is complete
 * when the call returns.  The call returns PC_OK when every item succeeded,
 * else the status of the failed item with the lowest index; every item
 * carries its own status (a failed item's output holds nothing valid). */
typedef struct {
    const void *positions;  /* device, T[n][3] */
    uint64_t n;
    int32_t dtype;          /* pc_dtype */
    int32_t eb_mode;        /* pc_eb_mode */
    double eb;
    uint32_t leaf_size;     /* as pc_config.leaf_size */
    uint32_t flags;         /* as pc_config.flags; the launch knobs are the defaults, or with
                               PC_FLAG_AUTOTUNE_KNOBS those of the item's class */
    void *out;              /* device, out_capacity bytes (pc_compress_bound suffices) */
    uint64_t out_capacity;
    uint64_t out_size;      /* written: stream bytes */
    int32_t status;         /* written */
    int32_t reserved2;
} pc_compress_item;

typedef struct {
    const void *stream_data;  /* device, 16-byte aligned */
    uint64_t stream_bytes;
    uint64_t n;               /* particles of the stream (pc_info.n) */
    void *out_positions;      /* device */
    uint64_t out_capacity_bytes;
    int32_t status;           /* written */
    int32_t reserved;
} pc_decompress_item;

/* Device scratch for a batch: `lanes` slices, each the largest workspace any
 * item needs (host only).  lanes = 0 picks min(count, 8). */
int pc_compress_batch_workspace_size(const pc_compress_item *items, uint32_t count, uint32_t lanes,
                                     uint64_t *out_bytes);
int pc_compress_batch(pc_compress_item *items, uint32_t count, uint32_t lanes, void *workspace,
                      uint64_t workspace_bytes, void *stream);
/* Device scratch for a batched decompression (host only): per item a code
 * table and the chunk descriptors of pc_decompress_item.n particles, plus the
 * batch's headers and records; `lanes` is not used.  An item whose stream holds
 * more particles than its n fails with PC_ERR_CAPACITY. */
int pc_decompress_batch_workspace_size(const pc_decompress_item *items, uint32_t count, uint32_t lanes,
                                       uint64_t *out_bytes);
int pc_decompress_batch(pc_decompress_item *items, uint32_t count, uint32_t lanes, void *workspace,
                        uint64_t workspace_bytes, void *stream);

/* ---- Serving loop ------------------------------------------------------------
 * A server owns `lanes` worker threads, each with its own CUDA stream, and a
 * caller-provided device arena.  Submitted requests queue in arrival order;
 * a free lane admits the oldest request as soon as the arena has room for its
 * workspace and its output (first fit, 256-byte aligned), so requests that
 * arrive while others run overlap with them on the device.  A request that
 * can never fit completes with PC_ERR_CAPACITY.  Outputs stay in the arena
 * until pc_server_release.  Results are identical to plain calls on the same
 * inputs.  Inputs must stay valid and unchanged until their completion is
 * polled.  All server calls are thread-safe. */
typedef struct pc_server pc_server;

enum { PC_REQ_COMPRESS = 0, PC_REQ_DECOMPRESS = 1 };

typedef struct {
    int32_t kind;           /* PC_REQ_COMPRESS or PC_REQ_DECOMPRESS */
    int32_t dtype;          /* pc_dtype of the positions (decompress: as in the stream header) */
    int32_t eb_mode;        /* compress: pc_eb_mode */
    uint32_t leaf_size;     /* compress: as pc_config.leaf_size */
    uint32_t flags;         /* compress: as pc_config.flags */
    uint32_t reserved;      /* 0 */
    double eb;              /* compress */
    const void *input;      /* device: positions (compress) or stream (decompress) */
    uint64_t n;             /* particles */
    uint64_t input_bytes;   /* decompress: stream bytes */
    uint64_t tag;           /* caller's identifier, echoed in the completion */
} pc_request;

typedef struct {
    uint64_t tag;
    int32_t status;
    int32_t kind;
    void *output;           /* device, inside the arena: the stream or the positions */
    uint64_t output_bytes;
    double t_submit;        /* seconds on the host's steady clock */
    double t_start;         /* admitted to a lane */
    double t_done;          /* result complete on the device */
} pc_completion;

int pc_server_create(void *arena, uint64_t arena_bytes, uint32_t lanes, pc_server **out);
int pc_server_submit(pc_server *server, const pc_request *request);
/* Up to `max` completions in completion order; with wait != 0 blocks until at
 * least one is available or nothing is queued or running. */
int pc_server_poll(pc_server *server, pc_completion *out, uint32_t max, uint32_t *got, int wait);
/* Returns an output's arena space (the `output` pointer of a completion). */
int pc_server_release(pc_server *server, void *output);
/* Requests queued or running, and arena bytes in use. */
int pc_server_stats(pc_server *server, uint64_t *pending, uint64_t *arena_in_use);
/* Waits for running requests and admits queued ones while they fit; queued
 * requests that no longer can (outputs still held) complete with
 * PC_ERR_CAPACITY.  Then frees the server; unpolled completions are dropped. */
int pc_server_destroy(pc_server *server);
/* Host seconds on the clock the completions use. */
double pc_server_now(void);

/* Kernel tracing.  While enabled, every kernel launch of the library is
 * bracketed by CUDA events recorded on the launching stream; elapsed times are
 * accumulated per kernel name when a call synchronises (compress and
 * decompress do so before returning).  Tracing is off by default and costs two
 * event records per launch when on.  pc_trace_get reports entry i in
 * [0, pc_trace_count()): its static name, launches and total milliseconds. */
int pc_trace_enable(int on);
int pc_trace_reset(void);
int pc_trace_count(void);
int pc_trace_get(int i, const char **name, uint64_t *launches, double *total_ms);

/* Static text for a status code. */
const char *pc_error_string(int status);

/* Stream format version this library writes and reads. */
int pc_format_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PC_H */
