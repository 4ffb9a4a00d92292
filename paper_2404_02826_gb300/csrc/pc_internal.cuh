// Internal declarations shared by the translation units of the CUDA library.
// Nothing here is part of the public C ABI (include/pc.h).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "../../include/pc.h"

namespace pcx {

constexpr uint32_t kHeaderBytes = 96;
constexpr uint32_t kLeafBytes = 32;
constexpr int64_t kCodeLimit = int64_t(1) << 30;  // codes < 2^30, so m_d <= 31

// Polls of a tile copy's barrier before a wait gives up, and the short limit
// of the self-test that drops the copies.
constexpr uint32_t kBarSpinLimit = 1u << 22;
constexpr uint32_t kSelftestSpinLimit = 1u << 12;

// Bits of the device error word.
enum : uint32_t { kErrTimeout = 1u, kErrCorrupt = 2u, kErrInternal = 4u };

// Whether an earlier kernel of this call has set the error word (a wait that
// gave up, an inconsistency).  The partition's and the leaves' kernels then do
// nothing, so that no step reads data that was never written and a failed
// call ends promptly.  Block-uniform: every thread calls it at kernel entry.
__device__ __forceinline__ bool call_failed(const uint32_t *err) {
  return __syncthreads_or(threadIdx.x == 0 && *reinterpret_cast<const volatile uint32_t *>(err) != 0u) != 0;
}

// Radix digit of the warp-per-node median (levels of many small nodes).
constexpr uint32_t kMedD = 10;
// Largest node handled by one warp.
constexpr uint64_t kMedMaxNode = 1ull << 16;

// Result of the range reduction (Sec. 3: per-axis min / max, Delta_max).
struct RangeResult {
  double lo[3];
  double hi[3];
  uint32_t nonfinite;
  uint32_t pad;
};

// Lattice parameters handed to the quantize kernel.
struct QuantParams {
  double o[3];   // origin (per-axis minimum)
  double s;      // step 2 eb'
  float of[3];   // origin as float (exact for float input)
  float rh, rl;  // 1/s as an unevaluated float sum rh + rl
  double inv;    // fl(1/s)
  uint32_t raw;      // bit d: axis d stored losslessly; its code is the split key
  double lo[3];      //   floor((p - lo) / span * 2^29) (span = hi - lo; 0 when span is 0)
  double span[3];
};

// Per-node state of one global k-d level (Sec. 4.1 median split by radix select).
struct LevelNode {
  uint32_t lo, hi;   // code bounds of the node on its split axis
  uint32_t prefix;   // selected high digits of (code - lo)
  int32_t shift;     // low bit of the current digit
  uint32_t width;    // bits of the current digit; 0 once the split is known
  uint32_t below;    // particles in lower buckets of earlier digits
  uint32_t v;        // split code
  uint32_t less;     // particles with code < v
  uint32_t tleft;    // particles with code == v that go left (first in index order)
  uint32_t blo[3];   // code bounds on every axis, inherited from the ancestors' splits:
  uint32_t bhi[3];   //   the left child of a split at v has codes <= v, the right child >= v
  uint32_t axis;     // split axis of the node
};

// Per-leaf facts kept between the bit-box pass and the packing pass.
struct LeafRec {
  uint32_t off;       // first particle of the leaf (leaf-ordered arrays, = first decoded particle)
  uint32_t cnt;       // particles
  uint32_t centre;    // position of the bit-box centre inside the leaf
  uint32_t m;         // m_x | m_y << 8 | m_z << 16
  int32_t qref[3];    // centre code
  uint32_t words;     // payload words of the leaf
  uint64_t word_off;  // first payload word
  uint64_t pad;
};

// Offset and size of node j at depth `level` of the median tree over n
// particles: the left child takes floor(c/2), the right ceil(c/2) (Sec. 4.1).
__host__ __device__ inline void node_range(uint64_t n, int level, uint64_t j, uint64_t &off, uint64_t &cnt) {
  off = 0;
  cnt = n;
  for (int b = level - 1; b >= 0; --b) {
    uint64_t half = cnt >> 1;
    if ((j >> b) & 1ull) {
      off += half;
      cnt -= half;
    } else {
      cnt = half;
    }
  }
}

__host__ __device__ inline uint32_t bit_length(uint64_t x) {
  uint32_t b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

// Eq. 2 on the lattice: m = 0 for R = 0, else bit_length(R) + 1.
__host__ __device__ inline uint32_t bits_for_range(uint32_t R) { return R ? bit_length(R) + 1 : 0; }

// Brackets the launches issued during its lifetime with CUDA events when
// tracing is on (pc_trace_enable); results are collected by trace_flush().
class TraceScope {
 public:
  TraceScope(const char *name, cudaStream_t st);
  ~TraceScope();
  TraceScope(const TraceScope &) = delete;
  TraceScope &operator=(const TraceScope &) = delete;

 private:
  const char *name_;
  cudaStream_t st_;
  void *a_, *b_;
};
void trace_flush();
bool trace_enabled();  // whether kernel tracing is on (each launch then needs its own events)

// ---- launchers (defined in the kernel translation units) -------------------

struct RangeLaunch {
  const void *pos;
  uint64_t n;
  int dtype;
  bool vec;
  double *partial;  // [blocks][7]
  RangeResult *result;
  int blocks;
};
cudaError_t launch_range(const RangeLaunch &a, cudaStream_t st);

struct QuantLaunch {
  const void *pos;
  uint64_t n;
  int dtype;
  int code_bytes;  // 2 or 4
  bool vec;
  bool fast;
  QuantParams qp;
  void *q[3];
  uint32_t *idx;  // optional identity permutation
  int blocks;
};
cudaError_t launch_quantize(const QuantLaunch &a, cudaStream_t st);

struct LevelLaunch {
  struct RootHi {
    uint32_t v[3];
  };
  uint64_t n;
  int level;
  int code_bytes;
  bool with_idx;
  uint32_t leaf_size;     // nodes of at most this many particles are leaves (copied unchanged)
  uint32_t warp_node_max; // levels whose nodes hold at most this many particles: one warp per node
  uint32_t digit_bits;
  bool warp_median;       // one warp per node runs the whole radix select (k_median, kMedD-bit digits)
  uint32_t passes;
  uint32_t tiles_per_node;
  uint32_t root_hi[3];    // level 0: the codes of axis d lie in [0, root_hi[d]]
  bool widest;            // split every node on the axis of its widest cell (else depth mod 3)
  const void *src[3];
  void *dst[3];
  const uint32_t *src_idx;
  uint32_t *dst_idx;
  LevelNode *nodes;       // this level [2^level]
  const LevelNode *parents;  // previous level [2^(level-1)], null at level 0
  uint32_t *hist;         // [2^level][2^digit_bits], zero on entry, zero on exit
  unsigned long long *tile_state;
  void *groups;           // [tiles][scatter_groups()] group records of this level
  uint32_t *ticket;
  uint32_t *err;
  int hist_blocks;
  uint32_t wait_limit;    // polls of a tile copy's barrier before the scatter gives up
  bool drop_copies;       // self-test only: the scatter issues no tile copy, so its first wait gives up
};
cudaError_t launch_level(const LevelLaunch &a, cudaStream_t st);
cudaError_t launch_scatter(const LevelLaunch &a, cudaStream_t st);
uint32_t scatter_tile(int code_bytes, bool with_idx);    // largest tile of one scatter CTA
uint32_t scatter_groups(int code_bytes, bool with_idx);  // 16-byte group records per tile

struct LeafLaunch {
  uint64_t n;
  int split_level;          // last level that split nodes (-1: the root is the only leaf)
  int code_bytes;
  uint32_t leaf_size;
  uint32_t warp_leaf_max;   // leaf_size at most this: a warp per leaf for bit boxes and packing, else a block
  uint64_t num_leaves;
  const void *codes[3];     // leaf-ordered codes
  const uint32_t *idx;      // leaf-ordered input indices (optional)
  uint8_t *out;             // stream base
  uint32_t *perm;           // optional
  LeafRec *recs;            // [num_leaves]
  uint64_t *total_words;    // device slot: payload words of the stream
  uint64_t *slice_tot;      // [ceil(num_leaves / 8192)] scratch of the many-leaf word scan
  bool cost_only;           // bit boxes and payload words only (leaf-size autotuning)
  bool recs_ready;          // recs already hold off, cnt, centre, m, q_ref, words (the box reduction's sequences)
  bool box_only;            // leaf table and bit boxes only (the records are reordered before packing)
  uint64_t payload_cap;     // payload words the output holds after the header and the leaf table
  uint32_t *err;            // device error word: a record that would write past n or the payload is skipped
  uint32_t raw;             // lossless axes: m_d = M and q_ref_d = 0 in the record, every particle in the
                            // payload (centre first), the coordinate's M-bit pattern read through idx from pos
  const void *pos;          // input positions (lossless axes)
  int dtype;
};
cudaError_t launch_leaves(const LeafLaunch &a, cudaStream_t st);
// The leaf ranges alone (off, cnt of every leaf; the other fields zero).
cudaError_t launch_leaftable(uint64_t n, int split_level, uint32_t leaf_size, LeafRec *recs, uint64_t num_leaves,
                             cudaStream_t st);

// The deep levels, bit boxes and packing of every node at depth `depth` in
// one kernel (k_subtree.cu): a CTA per node, `levels` splits inside it.
struct SubtreeLaunch {
  uint64_t n;
  int depth;                  // depth of the CTAs' nodes; the levels above ran as global levels
  int levels;                 // splits inside a CTA (0: the nodes are the leaves)
  int code_bytes;
  uint32_t leaf_size;
  bool widest;                // widest-cell split axis (else depth mod 3)
  uint32_t root_hi[3];        // codes of axis d lie in [0, root_hi[d]]
  const LevelNode *parents;   // the records of depth - 1 (null at depth 0)
  const void *codes[3];       // arrangement at `depth`
  const uint32_t *idx;        // input indices in the same arrangement (optional)
  uint8_t *out;               // stream base
  uint32_t *perm;             // optional
  uint64_t num_leaves;
  uint64_t leaves_small, leaves_big;  // leaves under a node of n >> depth particles, and of one more
  unsigned long long *status; // [2^depth] look-back words, zero on entry
  uint32_t *ticket;           // zero on entry
  uint64_t *total_words;      // written by the last node
  uint64_t payload_cap;
  uint32_t *err;
  // the leaf-size search's pass (cost_words non-null): [levels + 1] payload words per in-CTA
  // depth (zero on entry), and where the deepest in-CTA arrangement goes (null: nowhere),
  // with the records of depth + levels - 1 (the nodes of that depth, in order)
  unsigned long long *cost_words;
  void *wb_codes[3];
  uint32_t *wb_idx;
  LevelNode *wb_nodes;
};
cudaError_t launch_subtree(const SubtreeLaunch &a, cudaStream_t st);
uint32_t subtree_capacity(int code_bytes, bool with_idx);  // largest node of one CTA

struct HeaderLaunch {
  uint8_t *out;
  uint64_t n;
  int dtype, eb_mode;
  double eb, eps, s, o[3];
  uint64_t num_leaves;
  uint32_t leaf_size;
  const uint64_t *total_words;  // null when there are no leaves
  uint64_t *total_bytes;        // device slot read back by the host
  uint32_t *err;
  uint32_t raw;                 // lossless-axis mask (header byte 84)
};
cudaError_t launch_header(const HeaderLaunch &a, cudaStream_t st);

struct DecodeLaunch {
  const uint8_t *stream;
  uint64_t n;
  int dtype;
  uint64_t num_leaves;
  uint64_t payload_words;
  double s, o[3];
  bool fast;       // float output with the float-pair fast path
  float of[3];     // origin as float
  float sh, sl;    // s as an unevaluated float sum
  void *out;
  bool vec;
  uint32_t *err;
  int32_t *qb;           // [6], zero on entry: per axis min(0, lowest code), then max(0, highest code)
  void *tab;             // [decode_table_bytes()]: dequantized value of every code, when they fit
  void *chunks;          // [decode_chunk_bytes(n)]: per decode chunk, its leaves and payload words
  uint32_t raw;          // lossless-axis mask: those axes hold M-bit patterns, every particle in the payload
  bool prologue_done;    // validation and tables already launched by launch_decode_prologue
  // optional, page-locked host memory: the error word as the decoder's last block reads it
  // once every block is done (the blocks count themselves in err[1], zero on entry); a
  // block that returns early leaves it untouched
  uint32_t *host_err;
};
cudaError_t launch_decode(const DecodeLaunch &a, cudaStream_t st);
// Validation and tables for a stream whose header is not yet on the host: both
// kernels read it from the stream (stream_bytes long) and check it as the host
// parser does; chunk_cap = the chunk facts the workspace holds.  err and qb
// zero on entry; launch_decode with prologue_done then launches the decoder.
cudaError_t launch_decode_prologue(const uint8_t *stream, uint64_t stream_bytes, uint64_t chunk_cap, uint32_t *err,
                                   int32_t *qb, void *tab, void *chunks, cudaStream_t st);
// The first launch of a decompression: clears the workspace's first 64 bytes (error
// word, block count, code bounds) and copies the stream's header into page-locked
// host memory (`host_header`, 16-byte aligned).
cudaError_t launch_decode_start(const uint8_t *stream, uint32_t *ws64, uint8_t *host_header, cudaStream_t st);

// Many streams decoded by one set of launches: each stream's plain launch
// fields, and where its leaves start in the batch's leaf space (a multiple of
// 32, so that no warp holds leaves of two streams) and its chunks in the chunk
// space of its kind (the streams one decode launch serves: float with the
// float-pair path, float, double).  A kind's chunk descriptors are one array,
// the streams' parts of it in the kind's order.
struct DecItem {
  DecodeLaunch a;
  uint64_t leaf0;
  uint64_t chunk0;
};
enum : int { kDecKindF32Fast = 0, kDecKindF32 = 1, kDecKindF64 = 2, kDecKinds = 3 };
// Copies the 96-byte header of `count` 16-byte aligned device streams into dst.
cudaError_t launch_gather_headers(const uint8_t *const *streams, uint32_t count, uint8_t *dst, cudaStream_t st);
// Validation and chunk descriptors of every stream (leaf_start: [count + 1], device).
cudaError_t launch_validate_batch(const DecItem *items, const uint64_t *leaf_start, uint32_t count, uint64_t leaves,
                                  cudaStream_t st);
// Code tables of every stream that decodes through them.
cudaError_t launch_dtable_batch(const DecItem *items, uint32_t count, cudaStream_t st);
// Every chunk of one kind's streams, one persistent launch (chunks: that kind's descriptors);
// berr: the batch's error word (a bounded wait that gave up).
cudaError_t launch_decode_batch(int kind, bool vec, const DecItem *items, const void *chunks,
                                uint64_t num_chunks, uint32_t *berr, cudaStream_t st);
// A stream with lossless axes, decoded on its own after the batch's validation.
cudaError_t launch_decode_lossless(const DecodeLaunch &a, cudaStream_t st);
uint64_t decode_chunks(uint64_t n);
uint64_t decode_table_bytes();
uint64_t decode_chunk_bytes(uint64_t n);

int device_sm_count();

// Small device-to-host read-backs (result words, a stream header), then one
// synchronisation of the stream.  The copies land in a page-locked staging
// block (one DMA each, no bounce through a driver buffer) and are copied out
// after the synchronisation; regions of more than 4 KB together go straight
// to their destinations.
struct ReadBack {
  void *dst;
  const void *src;
  size_t bytes;
};
cudaError_t read_back(const ReadBack *items, int count, cudaStream_t st);
inline cudaError_t read_back(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  const ReadBack r = {dst, src, bytes};
  return read_back(&r, 1, st);
}

// A stream header on its way to host memory: written into a page-locked block
// by launch_decode_start (which also clears the workspace's first 64 bytes) and
// waited for on an event (finish), so that what is queued on the stream after
// start runs meanwhile; the block's word after the header then receives the
// decoder's error word.  Without a block or an event, start clears and copies
// with plain calls and waits for them.
struct HeaderCopy {
  uint8_t h[kHeaderBytes];
  void *blk = nullptr;   // the staging block, host address
  void *dblk = nullptr;  // and device address
  cudaEvent_t ev = nullptr;
  int dev = 0;
  bool done = false;  // h holds the header (or the copy failed before it was queued)
  cudaError_t start(const void *src, uint32_t *ws64, cudaStream_t st);
  cudaError_t finish();
  // the word after the header in the staging block (null without one): host, device address
  volatile uint32_t *host_err() const {
    return blk ? reinterpret_cast<volatile uint32_t *>(static_cast<uint8_t *>(blk) + kHeaderBytes) : nullptr;
  }
  uint32_t *host_err_dev() const {
    return dblk ? reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(dblk) + kHeaderBytes) : nullptr;
  }
  ~HeaderCopy();
};

// Blocks of kernel F resident per SM with `smem` bytes of dynamic shared
// memory, after raising the kernel's dynamic shared-memory limit to `smem`.
// Both are done once per device and kernel (F itself is the template
// argument, so every kernel has its own cache); safe from several host threads.
template <auto F>
cudaError_t resident_blocks(int threads, size_t smem, int *per_sm) {
  static std::atomic<int> cache[64];  // per device: blocks per SM + 1, 0 = not yet known
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int slot = dev & 63;
  const int known = cache[slot].load(std::memory_order_acquire);
  if (known > 0) {
    *per_sm = known - 1;
    return cudaSuccess;
  }
  e = cudaFuncSetAttribute(F, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int v = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, F, threads, smem);
  if (e != cudaSuccess) return e;
  cache[slot].store(v + 1, std::memory_order_release);
  *per_sm = v;
  return cudaSuccess;
}

// Self-test switch of the calling host thread: its compress calls issue no
// tile copy in the partition's scatter (pc_selftest_scatter_timeout).
void set_drop_tile_copies(bool on);
// pc_compress without the optional permutation, on a caller-provided workspace.
int compress_device(const void *positions, uint64_t n, int dtype, int eb_mode, double eb, const pc_config *cfg,
                    void *out, uint64_t out_capacity, uint64_t *out_size, void *workspace, uint64_t workspace_bytes,
                    cudaStream_t st);

}  // namespace pcx
