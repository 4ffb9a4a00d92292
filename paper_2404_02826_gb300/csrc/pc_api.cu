// C ABI (include/pc.h): argument checks, the error-bound arithmetic of Sec. 3
// on the host, workspace layout, and the launch sequence of the hot path.
#include <cfloat>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/pc.h"
#include "pc_host.cuh"
#include "pc_internal.cuh"
#include "pc_reduce.cuh"
#include "pc_reorder.cuh"

namespace pcx {

namespace {
thread_local bool t_drop_tile_copies = false;
thread_local bool t_no_host_alloc = false;
}  // namespace

void set_drop_tile_copies(bool on) { t_drop_tile_copies = on; }
void set_no_host_alloc(bool on) { t_no_host_alloc = on; }
bool no_host_alloc() { return t_no_host_alloc; }

namespace {
constexpr size_t kPinnedBlock = 4096;
std::mutex g_pinned_mu;
std::vector<void *> g_pinned_free;  // staging blocks not in use, kept for the life of the process

constexpr int kPinnedBatch = 16;  // blocks page-locked together: concurrent callers rarely wait for one

void *pinned_take() {
  std::lock_guard<std::mutex> g(g_pinned_mu);
  if (g_pinned_free.empty()) {
    if (t_no_host_alloc) return nullptr;  // the copies go to their destinations
    void *p = nullptr;
    if (cudaHostAlloc(&p, kPinnedBlock * kPinnedBatch, cudaHostAllocPortable | cudaHostAllocMapped) != cudaSuccess) {
      cudaGetLastError();  // no staging block: the copies go to their destinations
      return nullptr;
    }
    for (int i = kPinnedBatch - 1; i >= 0; --i) g_pinned_free.push_back(static_cast<uint8_t *>(p) + kPinnedBlock * i);
  }
  void *p = g_pinned_free.back();
  g_pinned_free.pop_back();
  return p;
}

void pinned_give(void *p) {
  std::lock_guard<std::mutex> g(g_pinned_mu);
  g_pinned_free.push_back(p);
}

// Events without timing, per device, kept for the life of the process.
std::vector<cudaEvent_t> g_events[64];

cudaEvent_t event_take(int dev) {
  {
    std::lock_guard<std::mutex> g(g_pinned_mu);
    std::vector<cudaEvent_t> &v = g_events[dev & 63];
    if (!v.empty()) {
      cudaEvent_t e = v.back();
      v.pop_back();
      return e;
    }
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void event_give(int dev, cudaEvent_t e) {
  std::lock_guard<std::mutex> g(g_pinned_mu);
  g_events[dev & 63].push_back(e);
}
}  // namespace

HeaderCopy::~HeaderCopy() {
  if (!done) return;  // a copy that may still be in flight keeps its block and event
  if (blk) pinned_give(blk);
  if (ev) event_give(dev, ev);
}

cudaError_t HeaderCopy::start(const void *src, uint32_t *ws64, cudaStream_t st) {
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  blk = pinned_take();
  ev = blk ? event_take(dev) : nullptr;
  if (ev && cudaHostGetDevicePointer(&dblk, blk, 0) != cudaSuccess) {
    cudaGetLastError();
    dblk = nullptr;
  }
  if (!dblk) {  // no staging: plain calls, waited for here
    if (ev) event_give(dev, ev);
    if (blk) pinned_give(blk);
    ev = nullptr;
    blk = nullptr;
    dblk = nullptr;
    done = true;
    e = cudaMemsetAsync(ws64, 0, 64, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, src, kHeaderBytes, cudaMemcpyDefault, st);
    return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
  }
  e = launch_decode_start(static_cast<const uint8_t *>(src), ws64, static_cast<uint8_t *>(dblk), st);
  if (e == cudaSuccess) e = cudaEventRecord(ev, st);
  return e;
}

cudaError_t HeaderCopy::finish() {
  if (done) return cudaSuccess;
  const cudaError_t e = cudaEventSynchronize(ev);
  if (e != cudaSuccess) return e;
  std::memcpy(h, blk, kHeaderBytes);
  done = true;
  return cudaSuccess;
}

cudaError_t read_back(const ReadBack *items, int count, cudaStream_t st) {
  size_t total = 0;
  for (int i = 0; i < count; ++i) total += (items[i].bytes + 15) & ~size_t(15);
  void *blk = total <= kPinnedBlock ? pinned_take() : nullptr;
  cudaError_t e = cudaSuccess;
  size_t o = 0;
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    void *to = blk ? static_cast<uint8_t *>(blk) + o : items[i].dst;
    e = cudaMemcpyAsync(to, items[i].src, items[i].bytes, cudaMemcpyDefault, st);
    o += (items[i].bytes + 15) & ~size_t(15);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (blk && e == cudaSuccess) {
    o = 0;
    for (int i = 0; i < count; ++i) {
      std::memcpy(items[i].dst, static_cast<const uint8_t *>(blk) + o, items[i].bytes);
      o += (items[i].bytes + 15) & ~size_t(15);
    }
    pinned_give(blk);
  }
  // after a failure a copy may still be in flight into the block: it is not reused
  return e;
}

int device_sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  static std::atomic<int> cache[64];
  const int slot = dev & 63;
  const int known = cache[slot].load(std::memory_order_relaxed);
  if (known > 0) return known;
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
  cache[slot].store(v, std::memory_order_relaxed);
  return v;
}

}  // namespace pcx

namespace {

using namespace pcx;

constexpr uint64_t kAlign = 256;
inline uint64_t align_up(uint64_t x, uint64_t a = kAlign) { return (x + a - 1) / a * a; }

uint64_t leaves_for(uint64_t n, uint64_t r) {
  // Node sizes at one depth take at most two values, floor and floor + 1, so
  // count leaves per size class instead of walking the tree.
  if (n == 0) return 0;
  uint64_t total = 0;
  uint64_t a = n, ca = 1, cb = 0;  // ca nodes of size a, cb nodes of size a + 1
  for (;;) {
    if (a + 1 <= r) return total + ca + cb;
    if (a <= r) {  // size-a nodes are leaves, size-(a+1) nodes split once more into leaves
      if (a == 0) return total + 2 * cb;
      return total + ca + 2 * cb;
    }
    // every node splits
    const uint64_t h = a >> 1;
    uint64_t na = 0, nb = 0;  // counts of size h and h + 1 children
    if (a & 1) {  // a = 2h + 1 -> h, h+1 ; a + 1 = 2h + 2 -> h+1, h+1
      na += ca;
      nb += ca + 2 * cb;
    } else {  // a = 2h -> h, h ; a + 1 = 2h + 1 -> h, h+1
      na += 2 * ca + cb;
      nb += cb;
    }
    a = h;
    ca = na;
    cb = nb;
  }
}

struct Plan {
  uint64_t n = 0;
  int dtype = 0;
  uint32_t r = PC_DEFAULT_LEAF_SIZE;
  bool idx = false;
  uint64_t num_leaves = 0;
  int levels = 0;  // levels that split nodes: while the largest node exceeds r
  // workspace offsets
  uint64_t off_partial = 0, off_range = 0, off_codes_a = 0, off_codes_b = 0, off_idx_a = 0, off_idx_b = 0;
  uint64_t off_nodes = 0, off_leafrec = 0, off_words = 0;
  uint64_t off_zero = 0, zero_bytes = 0;  // zeroed at every call:
  uint64_t off_hist = 0, off_tiles = 0, off_tickets = 0, off_err = 0, off_total = 0;
  uint64_t off_status = 0;  // look-back words of the on-chip subtree kernel
  uint64_t off_groups = 0, off_slices = 0;
  uint64_t off_reduce = 0, off_seqrec = 0;  // bit-box reduction: its scratch and the sequence records
  uint64_t off_rorecs = 0, off_roscratch = 0;  // reordering: the records in the new order, its scratch
  bool reduce = false, reorder = false, widest = false;
  uint32_t warp_node_max = PC_DEFAULT_WARP_NODE_MAX;  // threads per node: a warp per node up to this size
  uint32_t warp_leaf_max = PC_DEFAULT_WARP_LEAF_MAX;  // packing tile: a warp per leaf up to this leaf size
  bool tune = false;  // leaf size chosen by descending from r_hi while the stream shrinks (sized for r)
  uint32_t r_hi = 0;
  int tune_first = 0, tune_last = 0;  // candidate depths
  uint64_t off_tunecost = 0;          // leaf-size search: payload words per in-CTA depth (zeroed)
  uint64_t total = 0;
  int range_blocks = 0;
};

// The on-chip subtree kernel (k_subtree.cu) takes the nodes of one depth D, a
// CTA each, and finishes their subtrees: the splits of D .. L - 1, the bit
// boxes and the packing.  D is the shallowest depth whose nodes fit one CTA and
// that leaves at most kSubMaxLevels splits to it, and at most L - 1 (so every
// CTA holds a node of the tree, split once more or a leaf); within that, deep
// enough to give every SM a node where the tree allows.  -1: not used.
constexpr int kSubMaxLevels = 6;
constexpr int kSubMaxDepth = 20;  // at most 2^20 CTAs (and look-back words)

uint64_t subtree_status_entries(int levels) {
  const int d = levels >= 1 ? (levels - 1 < kSubMaxDepth ? levels - 1 : kSubMaxDepth) : 0;
  return 1ull << d;
}

int subtree_depth(uint64_t n, uint32_t r, int levels, int code_bytes, bool idx, int sms) {
  if (n == 0) return -1;
  const uint64_t cap = subtree_capacity(code_bytes, idx);
  const int hi = levels >= 1 ? levels - 1 : 0;
  int lo = levels - kSubMaxLevels > 0 ? levels - kSubMaxLevels : 0;
  while (lo <= hi && ((n + (1ull << lo) - 1) >> lo) > cap) ++lo;
  if (lo > hi || lo > kSubMaxDepth || r > cap) return -1;
  int want = 0;
  while ((1 << want) < sms) ++want;
  int d = lo;
  if (d < want) d = want < hi ? want : hi;
  if (d > kSubMaxDepth) d = kSubMaxDepth;
  return d;
}

// Root depth of the leaf-size search's on-chip pass: the shallowest depth whose
// nodes fit a CTA (the pass is efficient on large nodes), below the deepest
// candidate, within the look-back room of the packing pass (2^(tune_last - 1)
// words), and reaching a candidate within kSubMaxLevels levels.  -1: the
// search stays on the levels over HBM.
int tune_subtree_depth(uint64_t n, int tune_first, int tune_last, int code_bytes, bool idx) {
  if (n == 0 || tune_last < 1) return -1;
  const uint64_t cap = subtree_capacity(code_bytes, idx);
  int d = 0;
  while (d < tune_last && ((n + (1ull << d) - 1) >> d) > cap) ++d;
  if (d >= tune_last || d > kSubMaxDepth || d + kSubMaxLevels < tune_first) return -1;
  return d;
}

// Levels of the median tree that split nodes: node sizes at depth l are
// floor(n / 2^l) or ceil(n / 2^l), and a node of at most r particles is a leaf.
int split_levels(uint64_t n, uint32_t r) {
  int l = 0;
  while (((n + (1ull << l) - 1) >> l) > r) ++l;
  return l;
}

// Radix digit of the per-node histograms at one level (2^level nodes): wide
// at the top, narrower below so that a level's bins stay within 2^22.
uint32_t digit_bits_for(int level) {
  int d = 22 - level;
  if (d > 13) d = 13;
  if (d < 6) d = 6;
  return uint32_t(d);
}

// Bytes of one axis's code array: room for u32 codes and for the 16-byte
// loads of a tile's last group, which may reach up to 64 bytes past n.
inline uint64_t code_stride(uint64_t n) { return align_up(4 * n + 64); }

// Tiles per node at one level: node sizes are floor(n / 2^level) or one more.
uint64_t tiles_per_node(uint64_t n, int level, uint32_t tile) {
  const uint64_t big = (n >> level) + 1;
  const uint64_t t = (big + tile - 1) / tile;
  return t ? t : 1;
}

// smallest scatter tile over code widths: sizes the per-tile counts for any data
uint32_t min_scatter_tile(bool idx) {
  const uint32_t a = scatter_tile(2, idx), b = scatter_tile(4, idx);
  return a < b ? a : b;
}

int make_plan(uint64_t n, int dtype, const pc_config *cfg, bool idx, int sm_count, Plan &p, uint32_t r_min = 0) {
  if (dtype != PC_F32 && dtype != PC_F64) return PC_ERR_ARG;
  if (n > PC_MAX_PARTICLES) return PC_ERR_ARG;
  uint32_t r = PC_DEFAULT_LEAF_SIZE;
  p.tune = false;
  if (cfg) {
    if (cfg->flags & ~(PC_FLAG_AUTOTUNE_LEAF | PC_FLAG_BOX_REDUCTION | PC_FLAG_REORDER | PC_FLAG_WIDEST_AXIS |
                       PC_FLAG_AUTOTUNE_KNOBS))
      return PC_ERR_ARG;
    if (cfg->warp_node_max > PC_MAX_WARP_NODE_MAX || cfg->warp_leaf_max > PC_MAX_LEAF_SIZE) return PC_ERR_ARG;
    if (cfg->warp_node_max) p.warp_node_max = cfg->warp_node_max;
    if (cfg->warp_leaf_max) p.warp_leaf_max = cfg->warp_leaf_max;
    p.widest = (cfg->flags & PC_FLAG_WIDEST_AXIS) != 0;
    p.reduce = (cfg->flags & PC_FLAG_BOX_REDUCTION) != 0;
    p.reorder = (cfg->flags & PC_FLAG_REORDER) != 0;
    if (cfg->leaf_size) r = cfg->leaf_size;
    if (cfg->flags & PC_FLAG_AUTOTUNE_LEAF) {
      // candidates: depths d with ceil(n / 2^d) in [min(PC_AUTOTUNE_MIN_LEAF, max), max]
      p.tune = true;
      p.r_hi = cfg->leaf_size ? cfg->leaf_size : PC_MAX_LEAF_SIZE;
      if (p.r_hi < 16 || p.r_hi > PC_MAX_LEAF_SIZE) return PC_ERR_ARG;
      const uint32_t lo = r_min ? r_min : PC_AUTOTUNE_MIN_LEAF;
      r = p.r_hi < lo ? p.r_hi : lo;
    }
  }
  if (r < 1 || r > PC_MAX_LEAF_SIZE) return PC_ERR_ARG;
  p.n = n;
  p.dtype = dtype;
  p.r = r;
  p.idx = idx;
  p.num_leaves = leaves_for(n, r);
  p.levels = split_levels(n, r);
  if (p.tune) {
    // the first candidate has the largest leaves <= r_hi; descend while leaves stay >= r.
    // Leaves of >= 16 particles make every candidate a whole depth of the tree: no node
    // above it is already that small.
    p.tune_first = split_levels(n, p.r_hi);
    p.tune_last = p.tune_first;
    while (((n + (2ull << p.tune_last) - 1) >> (p.tune_last + 1)) >= r) ++p.tune_last;
  }
  p.range_blocks = 4 * (sm_count > 0 ? sm_count : 148);
  if (p.range_blocks > 1024) p.range_blocks = 1024;

  uint64_t o = 0;
  p.off_partial = o;
  o = align_up(o + 8ull * sizeof(double) * p.range_blocks);
  p.off_range = o;
  o = align_up(o + sizeof(RangeResult));
  p.off_codes_a = o;
  o = align_up(o + 3 * code_stride(n));
  p.off_codes_b = o;
  o = align_up(o + 3 * code_stride(n));
  // input indices carried through the partition: for the permutation output,
  // and for the lossless axes (the packing reads their coordinates through them),
  // which only the value range can reveal, so room for them is always planned
  p.off_idx_a = o;
  o = align_up(o + 4 * n);
  p.off_idx_b = o;
  o = align_up(o + 4 * n);
  uint64_t node_count = 0;
  for (int l = 0; l <= p.levels; ++l) node_count += 1ull << l;
  p.off_nodes = o;
  o = align_up(o + node_count * sizeof(LevelNode));
  p.off_leafrec = o;
  o = align_up(o + (p.num_leaves ? p.num_leaves : 1) * sizeof(LeafRec));
  p.off_words = o;
  o = align_up(o + 8);
  p.off_slices = o;  // slice totals of the many-leaf word scan
  o = align_up(o + 8 * ((p.num_leaves + 8191) / 8192 + 1));
  // group records of the scatter's classification, one level at a time
  uint64_t group_bytes = 16;
  for (int l = 0; l < p.levels; ++l)
    for (int cb = 2; cb <= 4; cb += 2)
      for (int wi = 0; wi < 2; ++wi) {
        const uint64_t g = (1ull << l) * tiles_per_node(n, l, scatter_tile(cb, wi)) * scatter_groups(cb, wi) * 16;
        if (g > group_bytes) group_bytes = g;
      }
  p.off_groups = o;
  o = align_up(o + group_bytes);
  if (p.reduce) {
    p.off_seqrec = o;
    o = align_up(o + (p.num_leaves ? p.num_leaves : 1) * sizeof(LeafRec));
    p.off_reduce = o;
    o = align_up(o + reduce_scratch_bytes(n, p.num_leaves));
  }
  if (p.reorder) {
    // a sequence holds at most r particles (the largest candidate when tuning), any number after the reduction
    const uint64_t most = p.reduce ? n : (p.tune ? p.r_hi : p.r);
    p.off_rorecs = o;
    o = align_up(o + (p.num_leaves ? p.num_leaves : 1) * sizeof(LeafRec));
    p.off_roscratch = o;
    o = align_up(o + reorder_scratch_bytes(n, p.num_leaves, most < n ? most : n));
  }
  // zeroed region
  p.off_zero = o;
  uint64_t hist_bins = 0, tiles = 0;
  for (int l = 0; l < p.levels; ++l) {
    const uint64_t b = (1ull << l) << digit_bits_for(l);
    if (b > hist_bins) hist_bins = b;
    tiles += (1ull << l) * tiles_per_node(n, l, min_scatter_tile(true));
  }
  p.off_hist = o;
  o = align_up(o + 4 * (hist_bins ? hist_bins : 1));
  p.off_tiles = o;
  o = align_up(o + 8 * (tiles ? tiles : 1));
  p.off_tickets = o;  // one per level over HBM, the subtree's, the leaf-size search pass's
  o = align_up(o + 4 * (p.levels + 2));
  p.off_tunecost = o;
  o = align_up(o + 8 * (kSubMaxLevels + 1));
  p.off_status = o;
  o = align_up(o + 8 * subtree_status_entries(p.levels));
  p.off_err = o;
  o = align_up(o + 4);
  p.off_total = o;
  o = align_up(o + 8);
  p.zero_bytes = o - p.off_zero;
  p.total = o;
  return PC_OK;
}

uint64_t stream_bound(uint64_t n, uint64_t leaves, int dtype) {
  // codes are at most 31 bits per axis (93 per particle); with lossless axes a
  // particle takes up to 3 M bits (96 for float, 192 for double), the centre included
  const uint64_t bits = dtype == PC_F64 ? 192 : 96;
  return PC_HEADER_BYTES + 36ull * leaves + 4ull * ((bits * n + 31) / 32);
}

// Spacing of the floating-point grid with `prec` significand bits at x > 0.
double grid_spacing(double x, int prec, int emin) {
  int e = 0;
  std::frexp(x, &e);
  int ex = e - 1;
  if (ex < emin) ex = emin;
  return std::ldexp(1.0, ex - (prec - 1));
}

struct Lattice {
  double eps = 0, s = 1, o[3] = {0, 0, 0};
  uint32_t qmax[3] = {0, 0, 0};
  double lo[3] = {0, 0, 0}, span[3] = {0, 0, 0};  // split keys of lossless axes
  uint32_t raw = 0;  // bit d: axis d stored losslessly (Sec. 4.1, m_d > M)
  int raw_cause = PC_OK;
};

// Split key of the largest coordinate of a lossless axis (k_quant.cu's rule).
uint32_t raw_key_top(double span) { return span > 0.0 ? (1u << 29) : 0u; }

// Sec. 3: eps from the absolute or value-range-relative bound; the lattice
// step s = 2 eb' keeps |p - (T)(o + s q)| <= eps after every rounding.
int lattice_from_range(const RangeResult &rr, int dtype, int mode, double eb, Lattice &L) {
  if (rr.nonfinite) return PC_ERR_NONFINITE;
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = rr.lo[d] == 0.0 ? 0.0 : rr.lo[d];
    hi[d] = rr.hi[d] == 0.0 ? 0.0 : rr.hi[d];
  }
  double dmax = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double r = hi[d] - lo[d];
    if (r > dmax) dmax = r;
  }
  L.eps = (mode == PC_EB_ABS) ? eb : eb * dmax;
  for (int d = 0; d < 3; ++d) L.o[d] = lo[d];
  if (dmax == 0.0) {
    L.s = 1.0;
    return PC_OK;
  }
  double m = 0.0;
  for (int d = 0; d < 3; ++d) {
    if (std::fabs(lo[d]) > m) m = std::fabs(lo[d]);
    if (std::fabs(hi[d]) > m) m = std::fabs(hi[d]);
  }
  const double m2 = 2.0 * (m > L.eps ? m : L.eps);
  const double tmax = dtype == PC_F32 ? double(FLT_MAX) : DBL_MAX;
  if (!(m2 <= tmax)) return PC_ERR_RANGE;
  const double ulp_t = dtype == PC_F32 ? grid_spacing(m2, 24, -126) : grid_spacing(m2, 53, -1022);
  const double ulp_d = grid_spacing(m2, 53, -1022);
  const double ebp = L.eps - ulp_t - 4.0 * ulp_d;
  if (!(ebp > 0.0)) {
    // no lattice keeps the bound through the rounding to T: every axis losslessly
    L.raw = 7u;
    L.raw_cause = PC_ERR_EB_TOO_SMALL;
    L.s = 1.0;
  } else {
    L.s = 2.0 * ebp;
    for (int d = 0; d < 3; ++d) {
      const double q = std::nearbyint((hi[d] - lo[d]) / L.s);
      if (!(q < double(kCodeLimit))) {  // codes of 2^30 or more: this axis losslessly
        L.raw |= 1u << d;
        L.raw_cause = PC_ERR_RANGE;
      } else {
        L.qmax[d] = uint32_t(q);
      }
    }
  }
  for (int d = 0; d < 3; ++d) {
    L.lo[d] = lo[d];
    L.span[d] = hi[d] - lo[d];
    if ((L.raw >> d) & 1u) L.qmax[d] = raw_key_top(L.span[d]);
  }
  return PC_OK;
}

#define PC_TRY(x)                        \
  do {                                   \
    cudaError_t e_ = (x);                \
    if (e_ != cudaSuccess) return PC_ERR_CUDA; \
  } while (0)

// With `sweep`, the leaf-size candidates are only measured: every candidate
// depth's stream size is recorded (sweep->count entries) and no stream is written.
struct Sweep {
  pc_sweep_point *points;
  uint32_t capacity, count;
  uint32_t r_min;
};

// Payload words an output of `capacity` bytes holds after the header and a
// table of `leaves` entries (0 when it holds not even those).
static uint64_t payload_words(uint64_t capacity, uint64_t leaves) {
  const uint64_t fixed = PC_HEADER_BYTES + uint64_t(PC_LEAF_BYTES) * leaves;
  return capacity > fixed ? (capacity - fixed) / 4 : 0;
}

// What one compression launched, for the launch-knob autotuner: which levels
// ran over HBM (the warp-per-node choice is made per level) and the leaf sizes
// the leaf kernels over HBM ran with (the warp-per-leaf choice is made per launch).
struct RunFacts {
  uint64_t hbm_levels = 0;  // bit l: level l ran over HBM
  uint32_t leaf_sizes[32] = {};
  int num_leaf_sizes = 0;
  bool leaf_overflow = false;  // more distinct leaf sizes than recorded
  void note_leaf_size(uint32_t r) {
    for (int i = 0; i < num_leaf_sizes; ++i)
      if (leaf_sizes[i] == r) return;
    if (num_leaf_sizes < 32) leaf_sizes[num_leaf_sizes++] = r;
    else leaf_overflow = true;
  }
};

int compress_impl(const void *positions, uint64_t n, int dtype, int eb_mode, double eb, const pc_config *cfg,
                  void *out, uint64_t out_capacity, uint64_t *out_size, void *workspace, uint64_t workspace_bytes,
                  uint32_t *perm, cudaStream_t st, Sweep *sweep = nullptr, RunFacts *facts = nullptr) {
  if (sweep) {
    if (!cfg || !(cfg->flags & PC_FLAG_AUTOTUNE_LEAF) || perm) return PC_ERR_ARG;
  } else if (!out || !out_size) {
    return PC_ERR_ARG;
  }
  if (n > 0 && !positions) return PC_ERR_ARG;
  if (sweep && n == 0) return PC_OK;
  if (eb_mode != PC_EB_ABS && eb_mode != PC_EB_REL) return PC_ERR_ARG;
  if (!(eb > 0.0) || !std::isfinite(eb)) return PC_ERR_ARG;
  if (!sweep && reinterpret_cast<uintptr_t>(out) % 16) return PC_ERR_ARG;
  const size_t esz = dtype == PC_F32 ? 4 : 8;
  if (n > 0 && reinterpret_cast<uintptr_t>(positions) % esz) return PC_ERR_ARG;
  Plan p;
  int rc = make_plan(n, dtype, cfg, perm != nullptr, device_sm_count(), p, sweep ? sweep->r_min : 0);
  if (rc) return rc;
  if (!workspace || reinterpret_cast<uintptr_t>(workspace) % kAlign) return PC_ERR_ARG;
  if (workspace_bytes < p.total) return PC_ERR_CAPACITY;
  if (!sweep && out_capacity < stream_bound(n, p.num_leaves, dtype)) return PC_ERR_CAPACITY;
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  uint32_t *err = reinterpret_cast<uint32_t *>(ws + p.off_err);
  uint64_t *total_dev = reinterpret_cast<uint64_t *>(ws + p.off_total);
  PC_TRY(cudaMemsetAsync(ws + p.off_zero, 0, p.zero_bytes, st));

  HeaderLaunch hl = {};
  hl.out = static_cast<uint8_t *>(out);
  hl.n = n;
  hl.dtype = dtype;
  hl.eb_mode = eb_mode;
  hl.eb = eb;
  hl.num_leaves = p.num_leaves;
  hl.leaf_size = p.r;
  hl.total_bytes = total_dev;
  hl.err = err;

  Lattice L;
  if (n == 0) {
    L.eps = eb_mode == PC_EB_ABS ? eb : 0.0;
  } else {
    // a1: value range (the one read-back before the launches that follow)
    RangeLaunch ra = {};
    ra.pos = positions;
    ra.n = n;
    ra.dtype = dtype;
    ra.vec = reinterpret_cast<uintptr_t>(positions) % 16 == 0;
    ra.partial = reinterpret_cast<double *>(ws + p.off_partial);
    ra.result = reinterpret_cast<RangeResult *>(ws + p.off_range);
    ra.blocks = p.range_blocks;
    PC_TRY(launch_range(ra, st));
    RangeResult rr;
    PC_TRY(read_back(&rr, ra.result, sizeof(rr), st));
    rc = lattice_from_range(rr, dtype, eb_mode, eb, L);
    if (rc) return rc;
    // lossless axes (Sec. 4.1, m_d > M): the plain stream only; the reduction,
    // the reordering and the leaf-size search need codes on every axis
    if (L.raw && (p.tune || p.reduce || p.reorder || sweep)) return L.raw_cause;
    const bool use_idx = p.idx || L.raw != 0;  // lossless axes are read through the input indices
    hl.raw = L.raw;

    const uint32_t qmax = L.qmax[0] > L.qmax[1] ? (L.qmax[0] > L.qmax[2] ? L.qmax[0] : L.qmax[2])
                                                 : (L.qmax[1] > L.qmax[2] ? L.qmax[1] : L.qmax[2]);
    const int cb = (qmax < 65536u && !L.raw) ? 2 : 4;
    void *codes_a[3], *codes_b[3];
    for (int d = 0; d < 3; ++d) {
      codes_a[d] = ws + p.off_codes_a + uint64_t(d) * code_stride(n);
      codes_b[d] = ws + p.off_codes_b + uint64_t(d) * code_stride(n);
    }
    uint32_t *idx_a = use_idx ? reinterpret_cast<uint32_t *>(ws + p.off_idx_a) : nullptr;
    uint32_t *idx_b = use_idx ? reinterpret_cast<uint32_t *>(ws + p.off_idx_b) : nullptr;

    // a2: quantize
    QuantLaunch qa = {};
    qa.pos = positions;
    qa.n = n;
    qa.dtype = dtype;
    qa.code_bytes = cb;
    qa.vec = ra.vec;
    for (int d = 0; d < 3; ++d) {
      qa.qp.o[d] = L.o[d];
      qa.qp.of[d] = float(L.o[d]);
      qa.q[d] = codes_a[d];
    }
    qa.qp.s = L.s;
    const double inv = 1.0 / L.s;
    qa.qp.rh = float(inv);
    qa.qp.rl = float(inv - double(qa.qp.rh));
    qa.qp.inv = inv;
    qa.fast = dtype == PC_F32 ? (qmax < (1u << 22) && inv > 0x1p-100 && inv < 0x1p100)
                              : (inv > 0x1p-1000 && inv < 0x1p1000);
    qa.qp.raw = L.raw;
    for (int d = 0; d < 3; ++d) {
      qa.qp.lo[d] = L.lo[d];
      qa.qp.span[d] = L.span[d];
    }
    qa.idx = idx_a;
    qa.blocks = 8 * device_sm_count();
    PC_TRY(launch_quantize(qa, st));

    // a3: the k-d levels, down to the leaves (autotuning: down to the deepest candidate at most);
    // the deep levels, bit boxes and packing on chip when the plain stream is asked for
    const int levels = p.tune ? p.tune_last : p.levels;
    const int sub_depth = (p.tune || p.reduce || p.reorder || sweep || L.raw)
                              ? -1
                              : subtree_depth(n, p.r, p.levels, cb, use_idx, device_sm_count());
    // the leaf-size search over the plain stream: levels over HBM down to tune_depth, then
    // the candidates below it costed on chip (the depth-mod-3 rule: a resumed level takes the
    // root's cell, which the widest-cell rule could not)
    const int tune_depth = (p.tune && !p.reduce && !p.reorder && !p.widest && !sweep && !L.raw)
                               ? tune_subtree_depth(n, p.tune_first, p.tune_last, cb, use_idx)
                               : -1;
    const int global_levels = sub_depth >= 0 ? sub_depth : (tune_depth >= 0 ? tune_depth : levels);
    // a4-a5 on the arrangement at depth `depth` (leaves = its 2^depth nodes when split_level = depth - 1)
    auto leaf_launch = [&](void *const *codes, const uint32_t *idxs, int split_level, uint32_t r,
                           uint64_t num_leaves, bool cost_only, bool box_only = false) {
      LeafLaunch lf = {};
      lf.n = n;
      lf.split_level = split_level;
      lf.code_bytes = cb;
      lf.leaf_size = r;
      lf.warp_leaf_max = p.warp_leaf_max;
      if (facts) facts->note_leaf_size(r);
      lf.num_leaves = num_leaves;
      for (int d = 0; d < 3; ++d) lf.codes[d] = codes[d];
      lf.idx = idxs;
      lf.out = static_cast<uint8_t *>(out);
      lf.perm = perm;
      lf.recs = reinterpret_cast<LeafRec *>(ws + p.off_leafrec);
      lf.total_words = reinterpret_cast<uint64_t *>(ws + p.off_words);
      lf.slice_tot = reinterpret_cast<uint64_t *>(ws + p.off_slices);
      lf.cost_only = cost_only;
      lf.box_only = box_only;
      lf.payload_cap = payload_words(out_capacity, num_leaves);
      lf.err = err;
      lf.raw = L.raw;
      lf.pos = positions;
      lf.dtype = dtype;
      return launch_leaves(lf, st);
    };
    // a5 from ready records: payload offsets and packing, after the reordering
    // when asked (from `codes` into `spare`, Sec. 4.2)
    auto pack_ready = [&](LeafRec *recs, uint64_t num_seq, void *const *codes, uint32_t *idxs, void *const *spare,
                          uint32_t *spare_idx, uint32_t r) -> int {
      if (p.reorder) {
        ReorderLaunch ro = {};
        ro.n = n;
        ro.code_bytes = cb;
        ro.num_seq = num_seq;
        ro.recs = recs;
        ro.out_recs = reinterpret_cast<LeafRec *>(ws + p.off_rorecs);
        for (int d = 0; d < 3; ++d) {
          ro.codes[d] = codes[d];
          ro.out_codes[d] = spare[d];
        }
        ro.idx = idxs;
        ro.out_idx = idxs ? spare_idx : nullptr;
        const uint64_t most = p.reduce ? n : (p.tune ? p.r_hi : p.r);
        ro.max_cnt = most < n ? most : n;
        ro.scratch = ws + p.off_roscratch;
        PC_TRY(launch_reorder(ro, st));
        recs = ro.out_recs;
        codes = spare;
        idxs = ro.out_idx;
      }
      LeafLaunch lf = {};
      lf.n = n;
      lf.code_bytes = cb;
      lf.leaf_size = r;
      lf.warp_leaf_max = p.warp_leaf_max;
      if (facts) facts->note_leaf_size(r);
      lf.num_leaves = num_seq;
      for (int d = 0; d < 3; ++d) lf.codes[d] = codes[d];
      lf.idx = idxs;
      lf.out = static_cast<uint8_t *>(out);
      lf.perm = perm;
      lf.recs = recs;
      lf.total_words = reinterpret_cast<uint64_t *>(ws + p.off_words);
      lf.slice_tot = reinterpret_cast<uint64_t *>(ws + p.off_slices);
      lf.recs_ready = true;
      lf.payload_cap = payload_words(out_capacity, num_seq);
      lf.err = err;
      PC_TRY(launch_leaves(lf, st));
      return PC_OK;
    };
    // The error word so far, read back: the paths that read back anyway (the
    // reduction, the reordering) stop before working on the partition of a
    // call that has failed; the leaf-size search reads it with each cost.
    auto error_so_far = [&]() -> int {
      uint32_t e = 0;
      PC_TRY(read_back(&e, err, 4, st));
      return (e & kErrTimeout) ? PC_ERR_TIMEOUT : (e ? PC_ERR_CUDA : PC_OK);
    };
    // autotuning: stream bytes of the leaves at `depth` (every node there is a leaf),
    // read back with the error word (the leaf kernels of a failed call do nothing)
    auto depth_cost = [&](void *const *codes, int depth, uint64_t *bytes) -> int {
      const uint64_t r = (n + (1ull << depth) - 1) >> depth;
      PC_TRY(leaf_launch(codes, nullptr, depth - 1, uint32_t(r), 1ull << depth, true));
      uint64_t words = 0;
      uint32_t e = 0;
      const ReadBack rb[2] = {{&words, ws + p.off_words, 8}, {&e, err, 4}};
      PC_TRY(read_back(rb, 2, st));
      if (e) return (e & kErrTimeout) ? PC_ERR_TIMEOUT : PC_ERR_CUDA;
      *bytes = uint64_t(PC_LEAF_BYTES) * (1ull << depth) + 4 * words;
      return PC_OK;
    };
    auto record = [&](int depth, uint64_t bytes) {
      if (sweep->count < sweep->capacity) {
        pc_sweep_point &pt = sweep->points[sweep->count];
        pt.leaf_size = uint32_t((n + (1ull << depth) - 1) >> depth);
        pt.depth = uint32_t(depth);
        pt.leaves = 1ull << depth;
        pt.header_bytes = PC_HEADER_BYTES;
        pt.table_bytes = uint64_t(PC_LEAF_BYTES) << depth;
        pt.payload_bytes = bytes - pt.table_bytes;
        pt.total_bytes = PC_HEADER_BYTES + bytes;
      }
      ++sweep->count;
    };
    int chosen = -1;            // autotuning: depth of the chosen leaves
    uint64_t best_bytes = 0;    // stream bytes (without header) at the shallower candidate
    const int first_depth = p.tune_first;
    LevelNode *nodes = reinterpret_cast<LevelNode *>(ws + p.off_nodes);
    void **src = codes_a, **dst = codes_b;
    uint32_t *isrc = idx_a, *idst = idx_b;
    int src_depth = 0;  // the depth of the arrangement in src; dst holds the one above
    // level l over HBM: splits the arrangement in src into dst, then swaps them
    auto global_level = [&](int l) -> int {
      LevelLaunch la = {};
      la.n = n;
      la.level = l;
      la.code_bytes = cb;
      la.with_idx = use_idx;
      la.leaf_size = p.r;
      la.warp_node_max = p.warp_node_max;
      if (facts && l < 64) facts->hbm_levels |= 1ull << l;
      // levels of at least 2048 nodes of at most kMedMaxNode particles: one warp per node
      la.warp_median = (1ull << l) >= 2048 && ((n + (1ull << l) - 1) >> l) <= kMedMaxNode;
      la.digit_bits = la.warp_median ? kMedD : digit_bits_for(l);
      const uint32_t widest_q = L.qmax[0] > L.qmax[1] ? (L.qmax[0] > L.qmax[2] ? L.qmax[0] : L.qmax[2])
                                                      : (L.qmax[1] > L.qmax[2] ? L.qmax[1] : L.qmax[2]);
      const uint32_t bits = bit_length(p.widest ? widest_q : L.qmax[l % 3]);
      la.widest = p.widest;
      la.passes = (bits + la.digit_bits - 1) / la.digit_bits;
      la.tiles_per_node = uint32_t(tiles_per_node(n, l, scatter_tile(cb, use_idx)));
      for (int d = 0; d < 3; ++d) la.root_hi[d] = L.qmax[d];
      for (int d = 0; d < 3; ++d) {
        la.src[d] = src[d];
        la.dst[d] = dst[d];
      }
      la.src_idx = isrc;
      la.dst_idx = idst;
      const uint64_t node_base = (1ull << l) - 1;  // the records of the levels above come first
      la.nodes = nodes + node_base;
      la.parents = l > 0 ? nodes + node_base - (1ull << (l - 1)) : nullptr;
      uint64_t tile_base = 0;
      for (int k = 0; k < l; ++k) tile_base += (1ull << k) * tiles_per_node(n, k, scatter_tile(cb, use_idx));
      la.hist = reinterpret_cast<uint32_t *>(ws + p.off_hist);
      la.tile_state = reinterpret_cast<unsigned long long *>(ws + p.off_tiles) + tile_base;
      la.groups = ws + p.off_groups;
      la.ticket = reinterpret_cast<uint32_t *>(ws + p.off_tickets) + l;
      la.err = err;
      la.hist_blocks = 2 * device_sm_count();
      la.drop_copies = t_drop_tile_copies;
      la.wait_limit = t_drop_tile_copies ? kSelftestSpinLimit : kBarSpinLimit;
      PC_TRY(launch_level(la, st));
      void **t = src;
      src = dst;
      dst = t;
      uint32_t *ti = isrc;
      isrc = idst;
      idst = ti;
      src_depth = l + 1;
      return PC_OK;
    };
    // a candidate depth's stream size against the shallower one (the arrangement at
    // depth l in src): the search stops at the first depth whose stream is not smaller
    auto judge = [&](int l, uint64_t bytes) {
      if (l > first_depth && bytes >= best_bytes) chosen = l - 1;
      else best_bytes = bytes;
    };
    for (int l = 0; l < global_levels; ++l) {
      if (p.tune && l >= first_depth) {
        uint64_t bytes = 0;
        rc = depth_cost(src, l, &bytes);
        if (rc) return rc;
        if (sweep) {
          record(l, bytes);
          best_bytes = bytes;
        } else {
          judge(l, bytes);
          if (chosen >= 0) break;
        }
      }
      rc = global_level(l);
      if (rc) return rc;
    }

    if (sweep) {
      // the deepest candidate, then nothing is written
      uint64_t bytes = 0;
      rc = depth_cost(src, levels, &bytes);
      if (rc) return rc;
      if (levels >= first_depth) record(levels, bytes);
      PC_TRY(cudaStreamSynchronize(st));
      trace_flush();
      return PC_OK;
    }
    // Sec. 4.1 bit-box reduction, then the packing of its sequences: codes and
    // indices go to the spare arrangement in sequence order
    auto reduce_launch = [&](void *const *codes, const uint32_t *idxs, void *const *spare, uint32_t *spare_idx,
                             int split_level, uint32_t r, uint64_t num_leaves) -> int {
      const int failed = error_so_far();
      if (failed) return failed;
      ReduceLaunch rl = {};
      rl.n = n;
      rl.code_bytes = cb;
      rl.split_level = split_level;
      rl.leaf_size = r;
      rl.num_leaves = num_leaves;
      for (int d = 0; d < 3; ++d) {
        rl.codes[d] = codes[d];
        rl.out_codes[d] = spare[d];
      }
      rl.idx = idxs;
      rl.out_idx = idxs ? spare_idx : nullptr;
      rl.leafs = reinterpret_cast<LeafRec *>(ws + p.off_leafrec);
      rl.seqs = reinterpret_cast<LeafRec *>(ws + p.off_seqrec);
      rl.scratch = ws + p.off_reduce;
      rl.err = err;
      uint64_t num_seq = 0, rounds = 0;
      PC_TRY(launch_reduce(rl, st, &num_seq, &rounds));
      hl.num_leaves = num_seq;
      // the leaf-ordered arrangement is free now: the reordering may write into it
      return pack_ready(rl.seqs, num_seq, spare, rl.out_idx, codes, const_cast<uint32_t *>(idxs), r);
    };
    // the leaves' bit boxes, then reordering and packing
    auto reorder_launch = [&](void *const *codes, uint32_t *idxs, void *const *spare, uint32_t *spare_idx,
                              int split_level, uint32_t r, uint64_t num_leaves) -> int {
      const int failed = error_so_far();
      if (failed) return failed;
      PC_TRY(leaf_launch(codes, idxs, split_level, r, num_leaves, false, true));
      return pack_ready(reinterpret_cast<LeafRec *>(ws + p.off_leafrec), num_leaves, codes, idxs, spare, spare_idx,
                        r);
    };
    // the on-chip subtree over the arrangement at `depth` (in src): `lv` levels
    // inside a CTA, leaves of at most r particles
    auto subtree_at = [&](int depth, int lv, uint32_t r, uint64_t num_leaves) {
      SubtreeLaunch sa = {};
      sa.n = n;
      sa.depth = depth;
      sa.levels = lv;
      sa.code_bytes = cb;
      sa.leaf_size = r;
      sa.widest = p.widest;
      for (int d = 0; d < 3; ++d) {
        sa.root_hi[d] = L.qmax[d];
        sa.codes[d] = src[d];
      }
      sa.parents = depth > 0 ? nodes + ((1ull << (depth - 1)) - 1) : nullptr;
      sa.idx = isrc;
      sa.out = static_cast<uint8_t *>(out);
      sa.perm = perm;
      sa.num_leaves = num_leaves;
      sa.leaves_small = leaves_for(n >> depth, r);
      sa.leaves_big = leaves_for((n >> depth) + 1, r);
      sa.status = reinterpret_cast<unsigned long long *>(ws + p.off_status);
      sa.ticket = reinterpret_cast<uint32_t *>(ws + p.off_tickets) + p.levels;
      sa.total_words = reinterpret_cast<uint64_t *>(ws + p.off_words);
      sa.payload_cap = payload_words(out_capacity, num_leaves);
      sa.err = err;
      return sa;
    };
    // a4-a5: bit boxes, payload offsets, packing
    if (sub_depth >= 0) {
      PC_TRY(launch_subtree(subtree_at(sub_depth, p.levels - sub_depth, p.r, p.num_leaves), st));
    } else if (!p.tune) {
      if (p.reduce) {
        rc = reduce_launch(src, isrc, dst, idst, levels - 1, p.r, p.num_leaves);
        if (rc) return rc;
      } else if (p.reorder) {
        rc = reorder_launch(src, isrc, dst, idst, levels - 1, p.r, p.num_leaves);
        if (rc) return rc;
      } else {
        PC_TRY(leaf_launch(src, isrc, levels - 1, p.r, p.num_leaves, false));
      }
    } else {
      bool packed = false;  // the chosen leaves were packed on chip
      if (chosen < 0 && tune_depth >= 0) {
        const int D = tune_depth;
        const int K = p.tune_last - D < kSubMaxLevels ? p.tune_last - D : kSubMaxLevels;
        // depth D itself: the last candidate judged on the levels over HBM (in src)
        if (D >= first_depth) {
          uint64_t bytes = 0;
          rc = depth_cost(src, D, &bytes);
          if (rc) return rc;
          judge(D, bytes);
        }
        if (chosen < 0) {
          // depths D + 1 .. D + K costed in one pass over the depth-D nodes, read back once;
          // when the search goes deeper the pass leaves depth D + K's arrangement in dst
          const bool deeper = D + K < p.tune_last;
          unsigned long long *cw = reinterpret_cast<unsigned long long *>(ws + p.off_tunecost);
          SubtreeLaunch ca = subtree_at(D, K, uint32_t((n + (1ull << (D + K)) - 1) >> (D + K)), 1ull << (D + K));
          ca.cost_words = cw;
          ca.ticket = reinterpret_cast<uint32_t *>(ws + p.off_tickets) + p.levels + 1;
          if (deeper) {
            for (int d = 0; d < 3; ++d) ca.wb_codes[d] = dst[d];
            ca.wb_idx = idst;
            ca.wb_nodes = nodes + ((1ull << (D + K - 1)) - 1);
          }
          PC_TRY(launch_subtree(ca, st));
          unsigned long long words[kSubMaxLevels + 1] = {};
          uint32_t e = 0;
          const ReadBack rb[2] = {{words, cw, 8ull * (K + 1)}, {&e, err, 4}};
          PC_TRY(read_back(rb, 2, st));
          if (e) return (e & kErrTimeout) ? PC_ERR_TIMEOUT : PC_ERR_CUDA;
          for (int d = D + 1; d <= D + K && chosen < 0; ++d)
            if (d >= first_depth) judge(d, uint64_t(PC_LEAF_BYTES) * (1ull << d) + 4ull * words[d - D]);
          if (chosen < 0 && !deeper) chosen = p.tune_last;  // every candidate's stream shrank: the deepest
          if (chosen >= D) {
            const uint64_t r = (n + (1ull << chosen) - 1) >> chosen;
            hl.leaf_size = uint32_t(r);
            hl.num_leaves = 1ull << chosen;
            PC_TRY(launch_subtree(subtree_at(D, chosen - D, uint32_t(r), 1ull << chosen), st));
            packed = true;
          } else if (chosen < 0) {
            // still shrinking at D + K: the search goes on over HBM from the arrangement and the
            // depth D + K - 1 records the pass wrote (src: depth D + K; dst: depth D, never the
            // one chosen from here)
            void **t = src;
            src = dst;
            dst = t;
            uint32_t *ti = isrc;
            isrc = idst;
            idst = ti;
            src_depth = D + K;
            for (int l = D + K; l < levels; ++l) {
              if (l > D + K && l >= first_depth) {
                uint64_t bytes = 0;
                rc = depth_cost(src, l, &bytes);
                if (rc) return rc;
                judge(l, bytes);
                if (chosen >= 0) break;
              }
              rc = global_level(l);
              if (rc) return rc;
            }
          }
        }
      }
      // the search stopped at the first depth whose stream is not smaller, or reached the
      // deepest candidate (in src), which is then judged too
      if (!packed && chosen < 0) {
        if (levels > first_depth) {
          uint64_t bytes = 0;
          rc = depth_cost(src, levels, &bytes);
          if (rc) return rc;
          judge(levels, bytes);
        }
        if (chosen < 0) chosen = levels;
      }
      if (!packed) {
        const int depth = chosen;
        const bool deepest = depth == src_depth;  // else dst holds it, one level above
        void **codes = deepest ? src : dst;
        uint32_t *idxs = deepest ? isrc : idst;
        const uint64_t r = depth ? (n + (1ull << depth) - 1) >> depth : n;
        hl.leaf_size = uint32_t(r);
        hl.num_leaves = 1ull << depth;
        if (p.reduce) {
          rc = reduce_launch(codes, idxs, deepest ? dst : src, deepest ? idst : isrc, depth - 1, uint32_t(r),
                             1ull << depth);
          if (rc) return rc;
        } else if (p.reorder) {
          rc = reorder_launch(codes, idxs, deepest ? dst : src, deepest ? idst : isrc, depth - 1, uint32_t(r),
                              1ull << depth);
          if (rc) return rc;
        } else {
          PC_TRY(leaf_launch(codes, idxs, depth - 1, uint32_t(r), 1ull << depth, false));
        }
      }
    }
    hl.total_words = reinterpret_cast<uint64_t *>(ws + p.off_words);
  }
  hl.eps = L.eps;
  hl.s = L.s;
  for (int d = 0; d < 3; ++d) hl.o[d] = L.o[d];
  PC_TRY(launch_header(hl, st));
  struct {
    uint64_t total;
    uint32_t err;
  } back = {0, 0};
  const ReadBack rb[2] = {{&back.total, total_dev, 8}, {&back.err, err, 4}};
  PC_TRY(read_back(rb, 2, st));
  trace_flush();
  if (back.err & kErrTimeout) return PC_ERR_TIMEOUT;
  if (back.err) return PC_ERR_CUDA;
  *out_size = back.total;
  return PC_OK;
}

// error word, then one u32 per decode chunk (its first particle's leaf)
// error word and code bounds, the dequantization table, the per-chunk facts
uint64_t decompress_ws_bytes(uint64_t n) {
  return kAlign + align_up(decode_table_bytes()) + align_up(decode_chunk_bytes(n));
}

int parse_header(const uint8_t *h, uint64_t avail, pc_info *info) {
  if (avail < PC_HEADER_BYTES) return PC_ERR_CORRUPT;
  if (std::memcmp(h, "PCB1", 4) != 0) return PC_ERR_CORRUPT;
  uint16_t ver;
  std::memcpy(&ver, h + 4, 2);
  if (ver != 1) return PC_ERR_CORRUPT;
  if (h[6] > 1 || h[7] > 1) return PC_ERR_CORRUPT;
  pc_info I = {};
  I.dtype = h[6];
  I.eb_mode = h[7];
  std::memcpy(&I.n, h + 8, 8);
  std::memcpy(&I.eb, h + 16, 8);
  std::memcpy(&I.eps, h + 24, 8);
  std::memcpy(&I.s, h + 32, 8);
  std::memcpy(I.o, h + 40, 24);
  std::memcpy(&I.num_leaves, h + 64, 8);
  std::memcpy(&I.payload_words, h + 72, 8);
  std::memcpy(&I.leaf_size, h + 80, 4);
  I.lossless_axes = h[84];  // Sec. 4.1, m_d > M: axes stored as the original coordinates
  if (I.lossless_axes > 7u) return PC_ERR_CORRUPT;
  for (int i = 85; i < 96; ++i)
    if (h[i]) return PC_ERR_CORRUPT;
  if (I.n > PC_MAX_PARTICLES || I.num_leaves > I.n || ((I.n > 0) != (I.num_leaves > 0))) return PC_ERR_CORRUPT;
  if (I.payload_words > (1ull << 40)) return PC_ERR_CORRUPT;
  if (!std::isfinite(I.s) || !(I.s > 0.0)) return PC_ERR_CORRUPT;
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(I.o[d])) return PC_ERR_CORRUPT;
  I.total_bytes = PC_HEADER_BYTES + PC_LEAF_BYTES * I.num_leaves + 4 * I.payload_words;
  *info = I;
  return PC_OK;
}

int decompress_impl(const void *stream_data, uint64_t stream_bytes, void *out_positions, uint64_t out_capacity_bytes,
                    void *workspace, uint64_t workspace_bytes, cudaStream_t st) {
  if (!stream_data || !workspace) return PC_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(stream_data) % 16 || reinterpret_cast<uintptr_t>(workspace) % kAlign)
    return PC_ERR_ARG;
  if (stream_bytes < PC_HEADER_BYTES) return PC_ERR_CORRUPT;
  if (workspace_bytes < 64) return PC_ERR_CAPACITY;
  uint32_t *err = static_cast<uint32_t *>(workspace);
  uint8_t *const ws = static_cast<uint8_t *>(workspace);
  int32_t *const qb = reinterpret_cast<int32_t *>(ws + 32);
  void *const tab = ws + kAlign;
  void *const chunks = ws + kAlign + align_up(decode_table_bytes());
  // the error word and code bounds are cleared and the header starts back to the host;
  // meanwhile the validation and the tables run on the device, reading the header
  // there (when the workspace holds the tables and a chunk's facts)
  HeaderCopy hc;
  PC_TRY(hc.start(stream_data, err, st));
  const uint64_t tab_end = kAlign + align_up(decode_table_bytes());
  const bool early = workspace_bytes >= tab_end + decode_chunk_bytes(1);
  if (early)
    PC_TRY(launch_decode_prologue(static_cast<const uint8_t *>(stream_data), stream_bytes,
                                  (workspace_bytes - tab_end) / decode_chunk_bytes(1), err, qb, tab, chunks, st));
  PC_TRY(hc.finish());
  pc_info I = {};
  int rc = parse_header(hc.h, PC_HEADER_BYTES, &I);
  if (!rc && I.total_bytes > stream_bytes) rc = PC_ERR_CORRUPT;
  const uint64_t esz = I.dtype == PC_F32 ? 4 : 8;
  if (!rc && out_capacity_bytes < 3 * esz * I.n) rc = PC_ERR_CAPACITY;
  if (!rc && I.n > 0 && (!out_positions || reinterpret_cast<uintptr_t>(out_positions) % esz)) rc = PC_ERR_ARG;
  if (!rc && I.n > 0 && workspace_bytes < decompress_ws_bytes(I.n)) rc = PC_ERR_CAPACITY;
  if (rc || I.n == 0) {
    // nothing of the early kernels outlives the call
    if (early) PC_TRY(cudaStreamSynchronize(st));
    return rc;
  }
  DecodeLaunch da = {};
  da.stream = static_cast<const uint8_t *>(stream_data);
  da.n = I.n;
  da.dtype = int(I.dtype);
  da.num_leaves = I.num_leaves;
  da.payload_words = I.payload_words;
  da.s = I.s;
  bool exact_o = true;
  for (int d = 0; d < 3; ++d) {
    da.o[d] = I.o[d];
    da.of[d] = float(I.o[d]);
    exact_o = exact_o && double(da.of[d]) == I.o[d];
  }
  da.sh = float(I.s);
  da.sl = float(I.s - double(da.sh));
  da.fast = I.dtype == PC_F32 && exact_o && I.s > 0x1p-100 && I.s < 0x1p100;
  da.out = out_positions;
  da.vec = reinterpret_cast<uintptr_t>(out_positions) % 16 == 0;
  da.err = err;
  da.qb = qb;
  da.tab = tab;
  da.chunks = chunks;
  da.raw = I.lossless_axes;
  da.prologue_done = early;
  // the decoder's last block leaves the error word in the header's staging block, over a
  // mark that stays when a block returned early (then the word is read back here)
  constexpr uint32_t kUnset = 0xffffffffu;
  da.host_err = da.raw ? nullptr : hc.host_err_dev();
  if (da.host_err) *hc.host_err() = kUnset;
  PC_TRY(launch_decode(da, st));
  uint32_t e = kUnset;
  if (da.host_err) {
    const cudaError_t se = cudaStreamSynchronize(st);
    if (se != cudaSuccess) {
      hc.done = false;  // the decoder may still write into the staging block: it is not reused
      return PC_ERR_CUDA;
    }
    e = *hc.host_err();
  }
  if (e == kUnset) PC_TRY(read_back(&e, err, 4, st));
  trace_flush();
  if (e & kErrCorrupt) return PC_ERR_CORRUPT;
  if (e) return PC_ERR_CUDA;
  return PC_OK;
}

// ---- Launch-knob autotuning (PC_FLAG_AUTOTUNE_KNOBS) --------------------------
// The classes live in a fixed table (no heap allocation, so pc_compress_noalloc
// may look them up).  The call that enters a class tunes it; a reset bumps the
// generation, and a tuning that started before it stores nothing.
constexpr int kKnobClasses = 256;
constexpr uint32_t kNodeCandidates[] = {512, 1024, 2048, 4096, 8192};
constexpr uint32_t kLeafCandidates[] = {256, 512, 1024, 2048, 4096};

struct KnobClass {
  int state;  // 0 free, 1 being tuned, 2 tuned
  uint64_t key;
  uint32_t leaf_size;
  uint32_t node_max, leaf_max;
};
std::mutex g_knob_mu;
KnobClass g_knob[kKnobClasses] = {};
uint64_t g_knob_gen = 0;

int bits_u64(uint64_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

// Class of a call: bit length of n, dtype, device and the flags other than this one (leaf_size apart).
uint64_t knob_key(uint64_t n, int dtype, const pc_config &c, int dev) {
  return uint64_t(bits_u64(n)) | (uint64_t(dtype & 1) << 7) | (uint64_t(dev & 0xff) << 8) |
         (uint64_t(c.flags & ~PC_FLAG_AUTOTUNE_KNOBS) << 16);
}

// Slot of the class (key, leaf_size), or -1.  With `claim`, a class not in the
// table is entered as being tuned (when a slot is free) and *claimed is set.
// Called with g_knob_mu held.
int knob_find(uint64_t key, uint32_t leaf_size, bool claim, bool *claimed) {
  *claimed = false;
  int free_slot = -1;
  for (int i = 0; i < kKnobClasses; ++i) {
    if (g_knob[i].state == 0) {
      if (free_slot < 0) free_slot = i;
    } else if (g_knob[i].key == key && g_knob[i].leaf_size == leaf_size) {
      return i;
    }
  }
  if (!claim || free_slot < 0) return -1;
  g_knob[free_slot] = KnobClass{1, key, leaf_size, 0, 0};
  *claimed = true;
  return free_slot;
}

// The tuning of one class: the call's own stream with cfg's knobs first, then
// every candidate that changes a launch for this input, timed on the host clock
// around the (synchronous) compression, best of two.  Threads per node first,
// then the packing tile with the best threads per node.  Every run writes the
// same stream into `out` (its size is checked).
int tune_knobs(const void *positions, uint64_t n, int dtype, int eb_mode, double eb, const pc_config &base,
               void *out, uint64_t out_capacity, uint64_t *out_size, void *workspace, uint64_t workspace_bytes,
               uint32_t *perm, cudaStream_t st, uint32_t *node_max, uint32_t *leaf_max) {
  RunFacts facts;
  int rc = compress_impl(positions, n, dtype, eb_mode, eb, &base, out, out_capacity, out_size, workspace,
                         workspace_bytes, perm, st, nullptr, &facts);
  if (rc) return rc;
  const uint64_t size0 = *out_size;
  uint32_t best_node = base.warp_node_max ? base.warp_node_max : PC_DEFAULT_WARP_NODE_MAX;
  uint32_t best_leaf = base.warp_leaf_max ? base.warp_leaf_max : PC_DEFAULT_WARP_LEAF_MAX;
  auto timed = [&](uint32_t nm, uint32_t lm, double *sec) -> int {
    pc_config c = base;
    c.warp_node_max = nm;
    c.warp_leaf_max = lm;
    double best = 0.0;
    for (int k = 0; k < 2; ++k) {
      uint64_t size = 0;
      const auto t0 = std::chrono::steady_clock::now();
      const int r = compress_impl(positions, n, dtype, eb_mode, eb, &c, out, out_capacity, &size, workspace,
                                  workspace_bytes, perm, st);
      const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (r) return r;
      if (size != size0) return PC_ERR_CUDA;  // a launch knob changed the stream: never expected
      if (k == 0 || t < best) best = t;
    }
    *sec = best;
    return PC_OK;
  };
  // what a candidate changes: the levels over HBM given a warp per node, or the
  // leaf-kernel launches given a warp per leaf
  auto signature = [&](bool node, uint32_t c) -> uint64_t {
    uint64_t m = 0;
    if (node) {
      for (int l = 0; l < 40; ++l)
        if (((facts.hbm_levels >> l) & 1ull) && ((n + (1ull << l) - 1) >> l) <= c) m |= 1ull << l;
    } else {
      for (int i = 0; i < facts.num_leaf_sizes; ++i)
        if (facts.leaf_sizes[i] <= c) m |= 1ull << i;
    }
    return m;
  };
  auto dist = [](uint32_t a, uint32_t b) { return a > b ? a - b : b - a; };
  // the current value and one candidate per other signature (the one nearest the current value)
  auto pass = [&](bool node, const uint32_t *cands, int nc, uint32_t &cur) -> int {
    uint64_t sig[8];
    uint32_t rep[8];
    int ns = 0;
    sig[ns] = signature(node, cur);
    rep[ns++] = cur;
    for (int i = 0; i < nc; ++i) {
      const uint64_t s = signature(node, cands[i]);
      int j = 0;
      while (j < ns && sig[j] != s) ++j;
      if (j == ns) {
        sig[ns] = s;
        rep[ns++] = cands[i];
      } else if (j > 0 && dist(cands[i], cur) < dist(rep[j], cur)) {
        rep[j] = cands[i];
      }
    }
    if (ns == 1) return PC_OK;  // no candidate changes a launch
    double best_t = 0.0;
    uint32_t best = cur;
    for (int j = 0; j < ns; ++j) {
      double t = 0.0;
      const int r = node ? timed(rep[j], best_leaf, &t) : timed(best_node, rep[j], &t);
      if (r) return r;
      if (j == 0 || t < best_t) {
        best_t = t;
        best = rep[j];
      }
    }
    cur = best;
    return PC_OK;
  };
  rc = pass(true, kNodeCandidates, int(sizeof(kNodeCandidates) / sizeof(kNodeCandidates[0])), best_node);
  if (rc) return rc;
  if (!facts.leaf_overflow) {
    rc = pass(false, kLeafCandidates, int(sizeof(kLeafCandidates) / sizeof(kLeafCandidates[0])), best_leaf);
    if (rc) return rc;
  }
  *node_max = best_node;
  *leaf_max = best_leaf;
  return PC_OK;
}

// Every compression entry point comes here: the plain call, or the knobs of
// the call's class (tuning the class when this call is its first).
int compress_entry(const void *positions, uint64_t n, int dtype, int eb_mode, double eb, const pc_config *cfg,
                   void *out, uint64_t out_capacity, uint64_t *out_size, void *workspace, uint64_t workspace_bytes,
                   uint32_t *perm, cudaStream_t st) {
  if (!cfg || !(cfg->flags & PC_FLAG_AUTOTUNE_KNOBS))
    return compress_impl(positions, n, dtype, eb_mode, eb, cfg, out, out_capacity, out_size, workspace,
                         workspace_bytes, perm, st);
  pc_config base = *cfg;
  base.flags &= ~PC_FLAG_AUTOTUNE_KNOBS;
  {
    Plan p;  // argument checks before the class table is touched
    const int rc = make_plan(n, dtype, &base, perm != nullptr, device_sm_count(), p);
    if (rc) return rc;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PC_ERR_CUDA;
  const uint64_t key = knob_key(n, dtype, base, dev);
  // tuning runs the compression many times and keeps a table entry: not for
  // empty inputs nor for callers that allocate nothing
  const bool may_tune = n > 0 && out && out_size && !no_host_alloc();
  int slot = -1;
  bool claimed = false;
  uint64_t gen = 0;
  {
    std::lock_guard<std::mutex> g(g_knob_mu);
    slot = knob_find(key, base.leaf_size, may_tune, &claimed);
    gen = g_knob_gen;
    if (slot >= 0 && g_knob[slot].state == 2) {
      base.warp_node_max = g_knob[slot].node_max;
      base.warp_leaf_max = g_knob[slot].leaf_max;
    }
  }
  if (!claimed)
    return compress_impl(positions, n, dtype, eb_mode, eb, &base, out, out_capacity, out_size, workspace,
                         workspace_bytes, perm, st);
  uint32_t node_max = 0, leaf_max = 0;
  const int rc = tune_knobs(positions, n, dtype, eb_mode, eb, base, out, out_capacity, out_size, workspace,
                            workspace_bytes, perm, st, &node_max, &leaf_max);
  std::lock_guard<std::mutex> g(g_knob_mu);
  if (g_knob_gen == gen) {
    if (rc == PC_OK) {
      g_knob[slot].node_max = node_max;
      g_knob[slot].leaf_max = leaf_max;
      g_knob[slot].state = 2;
    } else {
      g_knob[slot].state = 0;
    }
  }
  return rc;
}

}  // namespace

namespace pcx {

int compress_device(const void *positions, uint64_t n, int dtype, int eb_mode, double eb, const pc_config *cfg,
                    void *out, uint64_t out_capacity, uint64_t *out_size, void *workspace, uint64_t workspace_bytes,
                    cudaStream_t st) {
  return compress_entry(positions, n, dtype, eb_mode, eb, cfg, out, out_capacity, out_size, workspace,
                        workspace_bytes, nullptr, st);
}

}  // namespace pcx

extern "C" {

int pc_compress_bound(uint64_t n, int dtype, const pc_config *cfg, uint64_t *out_bytes) {
  if (!out_bytes) return PC_ERR_ARG;
  Plan p;
  int rc = make_plan(n, dtype, cfg, false, 148, p);
  if (rc) return rc;
  *out_bytes = stream_bound(n, p.num_leaves, dtype);
  return PC_OK;
}

int pc_compress_workspace_size(uint64_t n, int dtype, const pc_config *cfg, int with_perm, uint64_t *out_bytes) {
  if (!out_bytes) return PC_ERR_ARG;
  Plan p;
  // size for the largest block count the device may use
  int rc = make_plan(n, dtype, cfg, with_perm != 0, 256, p);
  if (rc) return rc;
  *out_bytes = p.total;
  return PC_OK;
}

int pc_compress(const void *positions, uint64_t n, int dtype, int eb_mode, double eb, const pc_config *cfg, void *out,
                uint64_t out_capacity, uint64_t *out_size, void *workspace, uint64_t workspace_bytes, uint32_t *perm,
                void *stream) {
  return compress_entry(positions, n, dtype, eb_mode, eb, cfg, out, out_capacity, out_size, workspace,
                        workspace_bytes, perm, static_cast<cudaStream_t>(stream));
}

int pc_tuned_config(uint64_t n, int dtype, const pc_config *cfg, pc_config *out, int *tuned) {
  if (!cfg || !out || !tuned || !(cfg->flags & PC_FLAG_AUTOTUNE_KNOBS)) return PC_ERR_ARG;
  pc_config c = *cfg;
  c.flags &= ~PC_FLAG_AUTOTUNE_KNOBS;
  Plan p;
  const int rc = make_plan(n, dtype, &c, false, 148, p);
  if (rc) return rc;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  const uint64_t key = knob_key(n, dtype, c, dev);
  c.warp_node_max = p.warp_node_max;
  c.warp_leaf_max = p.warp_leaf_max;
  *tuned = 0;
  {
    std::lock_guard<std::mutex> g(g_knob_mu);
    bool claimed = false;
    const int slot = knob_find(key, c.leaf_size, false, &claimed);
    if (slot >= 0 && g_knob[slot].state == 2) {
      c.warp_node_max = g_knob[slot].node_max;
      c.warp_leaf_max = g_knob[slot].leaf_max;
      *tuned = 1;
    }
  }
  *out = c;
  return PC_OK;
}

int pc_autotune_reset(void) {
  std::lock_guard<std::mutex> g(g_knob_mu);
  for (int i = 0; i < kKnobClasses; ++i) g_knob[i].state = 0;
  ++g_knob_gen;
  return PC_OK;
}

int pc_autotune_export(pc_tuned_class *out, uint32_t capacity, uint32_t *count) {
  if (!count || (capacity && !out)) return PC_ERR_ARG;
  std::lock_guard<std::mutex> g(g_knob_mu);
  uint32_t k = 0;
  for (int i = 0; i < kKnobClasses; ++i) {
    const KnobClass &c = g_knob[i];
    if (c.state != 2) continue;
    if (k < capacity) {
      pc_tuned_class t = {};
      t.n_bits = uint32_t(c.key & 0x7f);
      t.dtype = int32_t((c.key >> 7) & 1);
      t.device = int32_t((c.key >> 8) & 0xff);
      t.flags = uint32_t(c.key >> 16);
      t.leaf_size = c.leaf_size;
      t.warp_node_max = c.node_max;
      t.warp_leaf_max = c.leaf_max;
      out[k] = t;
    }
    ++k;
  }
  *count = k;
  return PC_OK;
}

int pc_autotune_import(const pc_tuned_class *classes, uint32_t count) {
  if (count && !classes) return PC_ERR_ARG;
  std::vector<uint64_t> keys(count);
  for (uint32_t i = 0; i < count; ++i) {
    const pc_tuned_class &t = classes[i];
    if (t.n_bits > 31 || (t.dtype != PC_F32 && t.dtype != PC_F64) || t.device < 0 || t.device > 255 ||
        t.reserved || (t.flags & PC_FLAG_AUTOTUNE_KNOBS) || !t.warp_node_max || !t.warp_leaf_max)
      return PC_ERR_ARG;
    // the class's config must be one a compression accepts (flags, leaf size, knob ranges)
    const pc_config c = {t.leaf_size, t.flags, t.warp_node_max, t.warp_leaf_max};
    const uint64_t n_rep = t.n_bits ? (1ull << (t.n_bits - 1)) : 0;  // a size of that bit length
    Plan p;
    if (make_plan(n_rep, t.dtype, &c, false, 148, p)) return PC_ERR_ARG;
    keys[i] = knob_key(n_rep, t.dtype, c, t.device);
  }
  std::lock_guard<std::mutex> g(g_knob_mu);
  auto slot_of = [&](uint64_t key, uint32_t leaf_size) {
    for (int s = 0; s < kKnobClasses; ++s)
      if (g_knob[s].state != 0 && g_knob[s].key == key && g_knob[s].leaf_size == leaf_size) return s;
    return -1;
  };
  // classes neither in the table nor earlier in the list need a free slot each
  int free_slots = 0, need = 0;
  for (int s = 0; s < kKnobClasses; ++s) free_slots += g_knob[s].state == 0;
  for (uint32_t i = 0; i < count; ++i) {
    bool seen = slot_of(keys[i], classes[i].leaf_size) >= 0;
    for (uint32_t j = 0; j < i && !seen; ++j) seen = keys[j] == keys[i] && classes[j].leaf_size == classes[i].leaf_size;
    need += !seen;
  }
  if (need > free_slots) return PC_ERR_CAPACITY;
  for (uint32_t i = 0; i < count; ++i) {
    int s = slot_of(keys[i], classes[i].leaf_size);
    if (s < 0) {
      s = 0;
      while (g_knob[s].state != 0) ++s;
    }
    g_knob[s] = KnobClass{2, keys[i], classes[i].leaf_size, classes[i].warp_node_max, classes[i].warp_leaf_max};
  }
  return PC_OK;
}

int pc_stream_info(const void *host_header, uint64_t header_bytes, pc_info *info) {
  if (!host_header || !info) return PC_ERR_ARG;
  return parse_header(static_cast<const uint8_t *>(host_header), header_bytes, info);
}

int pc_leaf_size_sweep_workspace_size(uint64_t n, int dtype, uint32_t r_min, uint32_t r_max, uint64_t *out_bytes) {
  if (!out_bytes || r_min < 16 || r_max < r_min || r_max > PC_MAX_LEAF_SIZE) return PC_ERR_ARG;
  pc_config cfg = {r_max, PC_FLAG_AUTOTUNE_LEAF};
  Plan p;
  int rc = make_plan(n, dtype, &cfg, false, 256, p, r_min);  // the largest block count a device may use
  if (rc) return rc;
  *out_bytes = p.total;
  return PC_OK;
}

int pc_leaf_size_sweep(const void *positions, uint64_t n, int dtype, int eb_mode, double eb, uint32_t r_min,
                       uint32_t r_max, pc_sweep_point *points, uint32_t capacity, uint32_t *count, void *workspace,
                       uint64_t workspace_bytes, void *stream) {
  if (!count || (capacity && !points) || r_min < 16 || r_max < r_min || r_max > PC_MAX_LEAF_SIZE)
    return PC_ERR_ARG;
  pc_config cfg = {r_max, PC_FLAG_AUTOTUNE_LEAF};
  Sweep sw = {points, capacity, 0, r_min};
  int rc = compress_impl(positions, n, dtype, eb_mode, eb, &cfg, nullptr, 0, nullptr, workspace, workspace_bytes,
                         nullptr, static_cast<cudaStream_t>(stream), &sw);
  *count = sw.count;
  return rc;
}

int pc_decompress_workspace_size(uint64_t n, uint64_t *out_bytes) {
  if (!out_bytes) return PC_ERR_ARG;
  *out_bytes = decompress_ws_bytes(n);
  return PC_OK;
}

int pc_decompress(const void *stream_data, uint64_t stream_bytes, void *out_positions, uint64_t out_capacity_bytes,
                  void *workspace, uint64_t workspace_bytes, void *stream) {
  return decompress_impl(stream_data, stream_bytes, out_positions, out_capacity_bytes, workspace, workspace_bytes,
                         static_cast<cudaStream_t>(stream));
}

int pc_compress_host_workspace_size(uint64_t n, int dtype, const pc_config *cfg, uint64_t *out_bytes) {
  if (!out_bytes) return PC_ERR_ARG;
  uint64_t ws = 0, bound = 0;
  int rc = pc_compress_workspace_size(n, dtype, cfg, 0, &ws);
  if (rc) return rc;
  rc = pc_compress_bound(n, dtype, cfg, &bound);
  if (rc) return rc;
  const uint64_t esz = dtype == PC_F32 ? 4 : 8;
  *out_bytes = align_up(3 * esz * n) + align_up(bound) + ws;
  return PC_OK;
}

int pc_compress_host(const void *host_positions, uint64_t n, int dtype, int eb_mode, double eb, const pc_config *cfg,
                     void *host_out, uint64_t out_capacity, uint64_t *out_size, void *workspace,
                     uint64_t workspace_bytes, void *stream) {
  if (!host_out || !out_size || !workspace || (n > 0 && !host_positions)) return PC_ERR_ARG;
  if (dtype != PC_F32 && dtype != PC_F64) return PC_ERR_ARG;
  uint64_t need = 0, bound = 0;
  int rc = pc_compress_host_workspace_size(n, dtype, cfg, &need);
  if (rc) return rc;
  if (workspace_bytes < need) return PC_ERR_CAPACITY;
  pc_compress_bound(n, dtype, cfg, &bound);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t esz = dtype == PC_F32 ? 4 : 8;
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  uint8_t *dpos = ws;
  uint8_t *dout = ws + align_up(3 * esz * n);
  uint8_t *rest = dout + align_up(bound);
  if (n) PC_TRY(cudaMemcpyAsync(dpos, host_positions, 3 * esz * n, cudaMemcpyHostToDevice, st));
  uint64_t size = 0;
  rc = compress_entry(dpos, n, dtype, eb_mode, eb, cfg, dout, bound, &size, rest, workspace_bytes - (rest - ws),
                      nullptr, st);
  if (rc) return rc;
  if (size > out_capacity) return PC_ERR_CAPACITY;
  PC_TRY(cudaMemcpyAsync(host_out, dout, size, cudaMemcpyDeviceToHost, st));
  PC_TRY(cudaStreamSynchronize(st));
  *out_size = size;
  return PC_OK;
}

int pc_decompress_host_workspace_size(uint64_t n, int dtype, uint64_t stream_bytes, uint64_t *out_bytes) {
  if (!out_bytes || (dtype != PC_F32 && dtype != PC_F64)) return PC_ERR_ARG;
  const uint64_t esz = dtype == PC_F32 ? 4 : 8;
  *out_bytes = align_up(stream_bytes) + align_up(3 * esz * n) + decompress_ws_bytes(n);
  return PC_OK;
}

int pc_decompress_host(const void *host_stream, uint64_t stream_bytes, void *host_positions,
                       uint64_t out_capacity_bytes, void *workspace, uint64_t workspace_bytes, void *stream) {
  if (!host_stream || !workspace) return PC_ERR_ARG;
  pc_info I;
  int rc = pc_stream_info(host_stream, stream_bytes, &I);
  if (rc) return rc;
  if (I.total_bytes > stream_bytes) return PC_ERR_CORRUPT;
  const uint64_t esz = I.dtype == PC_F32 ? 4 : 8;
  if (out_capacity_bytes < 3 * esz * I.n) return PC_ERR_CAPACITY;
  if (I.n > 0 && !host_positions) return PC_ERR_ARG;
  uint64_t need = 0;
  pc_decompress_host_workspace_size(I.n, int(I.dtype), I.total_bytes, &need);
  if (workspace_bytes < need) return PC_ERR_CAPACITY;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  uint8_t *dst_stream = ws;
  uint8_t *dpos = ws + align_up(I.total_bytes);
  uint8_t *rest = dpos + align_up(3 * esz * I.n);
  PC_TRY(cudaMemcpyAsync(dst_stream, host_stream, I.total_bytes, cudaMemcpyHostToDevice, st));
  rc = decompress_impl(dst_stream, I.total_bytes, dpos, 3 * esz * I.n, rest, decompress_ws_bytes(I.n), st);
  if (rc) return rc;
  if (I.n) PC_TRY(cudaMemcpyAsync(host_positions, dpos, 3 * esz * I.n, cudaMemcpyDeviceToHost, st));
  PC_TRY(cudaStreamSynchronize(st));
  return PC_OK;
}

const char *pc_error_string(int status) {
  switch (status) {
    case PC_OK: return "ok";
    case PC_ERR_ARG: return "invalid argument";
    case PC_ERR_NONFINITE: return "non-finite coordinate in the input";
    case PC_ERR_EB_TOO_SMALL: return "error bound below the rounding margin of the input type";
    case PC_ERR_RANGE: return "quantization codes or magnitudes out of range";
    case PC_ERR_CAPACITY: return "output or workspace buffer too small";
    case PC_ERR_CORRUPT: return "corrupt or inconsistent stream";
    case PC_ERR_TIMEOUT: return "a bounded device wait expired";
    case PC_ERR_CUDA: return "CUDA runtime error";
    default: return "unknown status";
  }
}

int pc_format_version(void) { return 1; }

}  // extern "C"
