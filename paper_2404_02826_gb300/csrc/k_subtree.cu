// The deep levels of the median k-d partition, the leaves' bit boxes and the
// packed sequences in one kernel (Sec. 4.1 and 4.2, Fig. 4 of arXiv 2404.02826).
//
// Once every node of a level fits in shared memory, a CTA takes one node (in
// ticket order), copies its code arrays in with bulk copies and finishes its
// subtree on chip, without returning to HBM:
//   - every remaining level: per subnode a radix select of the median code on
//     its split axis (histograms in shared memory), then a stable two-way
//     partition of every subnode (the median rule of Sec. 4.1: code < v, then
//     the first `tleft` codes equal to v in index order, go left), from warp
//     ballots and one block-wide scan, moved in place through registers;
//   - the leaves' bit boxes (AABB, the particle closest to its centre, Eq. 2);
//   - the CTA's first payload word, from the payload sizes of the CTAs before
//     it (decoupled look-back over one status word per node, bounded waits);
//   - the leaf records and the packed payload (Fig. 4), straight from shared
//     memory, and the optional permutation.
// The subnodes of a level are served by equal groups of warps: at relative
// depth k there are 2^k subnodes and 32 / 2^k warps each, and a thread takes
// positions row * (1024 / 2^k) + its index in the group, so it always holds at
// most kRows positions whatever k is.
#include <cstdint>

#include "pc_internal.cuh"
#include "pc_mbar.cuh"

namespace pcx {
namespace {

constexpr int kT = 1024;  // threads of a CTA
constexpr int kLgWarps = 5;
constexpr int kWarps = 1 << kLgWarps;
constexpr int kSubMaxLevels = kLgWarps + 1;  // splits inside a CTA: at least one warp per splitting subnode
constexpr uint32_t kSubBins = 2048;  // radix bins of a level, shared by its subnodes
constexpr uint32_t kLookSpin = 1u << 20;  // polls of a predecessor's status before giving up
constexpr uint32_t kTmemCols = 512;       // tensor-memory columns of a CTA (one CTA per SM)

// One subnode of the CTA's subtree at the current level.
struct SubNode {
  uint32_t off, cnt;        // position in the CTA's node, particles
  uint32_t blo[3], bhi[3];  // cell: code bounds on every axis, from the ancestors' splits
  uint32_t axis, split;     // split axis; 1 if the subnode splits (more than r particles)
  uint32_t lo, prefix, below, width;  // radix select: lowest code, chosen digits, count below them, digit bits
  int32_t shift;
  uint32_t v, tleft;        // split code; particles equal to v that go left
};

struct SubLeaf {
  uint32_t off, cnt, centre, m;
  int32_t qref[3];
  uint32_t words;
  unsigned long long word_off;
  uint32_t lo[3], hi[3];
};

struct SubMisc {
  unsigned long long bar;
  unsigned long long prefix;    // payload words of the nodes before this one
  unsigned long long wd[kWarps][2];
  uint32_t wp[kWarps][2];
  unsigned long long off, cnt;  // the node: first particle, particles
  uint32_t j, nl, lead, ilead, tmem;
  uint32_t skip;                // an earlier kernel of the call failed: the node is not worked
  uint32_t wt[kWarps];          // warp totals of the scans
  uint32_t gb[kWarps];          // scan value at the first entry of each group
  uint32_t fb[kWarps], fbefore[kWarps];
};

// Warps per leaf in the leaf phase: kWarps >> lgwl slots of 2^lgwl warps;
// more leaves than warps: a warp per leaf, in turns.
struct LeafSlots {
  uint32_t lgwl, WL, slots, lw, lt, lstep;
};
__device__ __forceinline__ LeafSlots leaf_slots(uint32_t nl, int warp, int lane) {
  LeafSlots q;
  uint32_t lgwl = kLgWarps;
  while (lgwl > 0 && (uint32_t(kWarps) >> lgwl) < nl) --lgwl;
  q.lgwl = lgwl;
  q.WL = 1u << lgwl;
  q.slots = uint32_t(kWarps) >> lgwl;
  q.lw = uint32_t(warp) & (q.WL - 1u);  // warp within its leaf group
  q.lt = q.lw * 32 + uint32_t(lane);
  q.lstep = q.WL * 32;
  return q;
}

__host__ __device__ constexpr uint32_t al128(uint32_t x) { return (x + 127u) & ~127u; }

// Shared-memory layout of one CTA: the code arrays of a node of up to
// kRows * 1024 particles (each with room for the lead and tail of a 16-byte
// aligned window), the optional index array, the radix bins, the partition's
// masks and scan (reused as the packing's word staging), the subnode and leaf
// records.  All offsets are compile-time constants.
template <typename C, bool IDX>
struct SubL {
  static constexpr int R = sizeof(C) == 2 ? (IDX ? 16 : 32) : (IDX ? 12 : 16);  // positions per thread
  // tensor-memory columns of one thread: every array's values of its positions, 32 bits per column
  static constexpr int kCodeCols = sizeof(C) == 2 ? R / 2 : R;
  static constexpr int kCols = 3 * kCodeCols + (IDX ? R : 0);
  static_assert(kCodeCols % 4 == 0 && (kWarps / 4) * kCols <= 512, "tensor-memory columns");
  static constexpr uint32_t kCap = uint32_t(R) * kT;
  static constexpr uint32_t kSlots = kCap + 16;
  static constexpr uint32_t kCodeStride = al128(kSlots * uint32_t(sizeof(C)));
  static constexpr uint32_t kIdx = 3 * kCodeStride;
  static constexpr uint32_t kBins = kIdx + (IDX ? al128(kSlots * 4) : 0u);
  static constexpr uint32_t kStage = kBins + al128(kSubBins * 4);
  static constexpr uint32_t kPart = uint32_t(R) * kWarps * 16, kPack = kWarps * 96u * 4;
  static constexpr uint32_t kSn0 = kStage + al128(kPart > kPack ? kPart : kPack);
  static constexpr uint32_t kSn1 = kSn0 + al128(kWarps * sizeof(SubNode));
  static constexpr uint32_t kLeaf = kSn1 + al128(kWarps * sizeof(SubNode));
  static constexpr uint32_t kMisc = kLeaf + al128(2 * kWarps * sizeof(SubLeaf));
  static constexpr uint32_t kTotal = kMisc + al128(sizeof(SubMisc));
  static_assert(kTotal <= 232448, "shared memory of one CTA");
};

constexpr unsigned long long kStAgg = 1ull << 62, kStIncl = 2ull << 62, kStVal = (1ull << 62) - 1;

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t widest_axis(const uint32_t *blo, const uint32_t *bhi) {
  uint32_t ax = 0;
  for (uint32_t d = 1; d < 3; ++d)
    if (bhi[d] - blo[d] > bhi[ax] - blo[ax]) ax = d;
  return ax;
}

// Radix-select state of a splitting subnode from its cell (k_prep's rule):
// all codes equal on the axis decides at once, else digits of at most hb bits.
__device__ __forceinline__ void sub_select_init(SubNode &s, uint32_t hb) {
  s.lo = s.blo[s.axis];
  const uint32_t B = bit_length(s.bhi[s.axis] - s.lo);
  s.prefix = 0;
  s.below = 0;
  if (!s.split) {
    s.width = 0;
  } else if (B == 0) {
    s.width = 0;
    s.v = s.lo;
    s.tleft = s.cnt >> 1;
  } else {
    s.width = B < hb ? B : hb;
    s.shift = int32_t(B - s.width);
  }
}

// ---- tensor memory (TMEM): where each thread keeps its rows between levels ----
// Between two levels a thread's positions (its rows of its group's subnode)
// live in its own TMEM lane (tcgen05.st / tcgen05.ld, shape 32x32b: a warp
// reaches the 32 lanes of its lane quarter, 32 bits per column).  Shared
// memory only serves the exchange of a level's move: every thread writes its
// values to their destinations, the block synchronises, and every thread reads
// its rows of the next level back into TMEM.  One warp allocates the columns
// at the start and frees them at the end.  Every tcgen05 instruction is
// .sync.aligned, so each helper first reconverges the warp.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
  __syncwarp();
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  __syncwarp();
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 4 consecutive columns of this thread's lane; completes by tmem_wait_st()
__device__ __forceinline__ void tmem_st4(uint32_t t, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  __syncwarp();
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(t), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  __syncwarp();
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// 8 consecutive columns, complete when the call returns
__device__ __forceinline__ void tmem_ld8(uint32_t t, uint32_t *v) {
  __syncwarp();
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
      : "r"(t)
      : "memory");
}
// 4 columns from each of three places (the x, y, z values of the same rows), one wait
__device__ __forceinline__ void tmem_ld4x3(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t *v) {
  __syncwarp();
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%12];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%13];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%14];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11])
      : "r"(t0), "r"(t1), "r"(t2)
      : "memory");
}
__device__ __forceinline__ void tmem_ld4(uint32_t t, uint32_t *v) {
  __syncwarp();
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
      : "r"(t)
      : "memory");
}

// Up to 8 columns (`left` of them remain in the array; a compile-time value
// after unrolling), the rest zero.
__device__ __forceinline__ void tmem_ld_cols(uint32_t t, uint32_t *v, int left) {
  if (left >= 8) {
    tmem_ld8(t, v);
  } else {
    tmem_ld4(t, v);
    v[4] = v[5] = v[6] = v[7] = 0;
  }
}

// Value of row r of a thread's array from its columns: 16-bit values two rows
// per column (rows 2c and 2c + 1 in column c), 32-bit values one row each.
template <typename E>
__device__ __forceinline__ uint32_t row_of(const uint32_t *cols, int r) {
  if constexpr (sizeof(E) == 2) return (cols[r >> 1] >> (16 * (r & 1))) & 0xffffu;
  else return cols[r];
}

// Reads the rows p = r * Tg + ltid (r < nv) of one array of a subnode from
// shared memory into the thread's columns from `taddr` (completion:
// tmem_wait_st).
template <int R, typename E>
__device__ __forceinline__ void load_rows(const E *A, uint32_t nv, uint32_t Tg, uint32_t ltid, uint32_t taddr) {
  constexpr int NC = sizeof(E) == 2 ? R / 2 : R;
  constexpr int RPC = sizeof(E) == 2 ? 2 : 1;  // rows per column
#pragma unroll
  for (int c0 = 0; c0 < NC; c0 += 4) {
    uint32_t v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      v[c] = 0;
#pragma unroll
      for (int h = 0; h < RPC; ++h) {
        const int r = RPC * (c0 + c) + h;
        if (uint32_t(r) < nv) v[c] |= uint32_t(A[uint32_t(r) * Tg + ltid]) << (16 * h);
      }
    }
    tmem_st4(taddr + uint32_t(c0), v[0], v[1], v[2], v[3]);
  }
}

// COST: the leaf-size search's pass.  Every subnode splits at every level;
// before the first level and after each one the leaves at that depth get their
// bit boxes, and their payload words are added to cost_words[level]; nothing
// is written to the stream.
template <typename C, bool IDX, bool WIDEST, bool COST>
__global__ void __launch_bounds__(kT, 1) k_subtree(SubtreeLaunch a) {
  using L = SubL<C, IDX>;
  constexpr int R = L::R;
  extern __shared__ __align__(128) unsigned char sm[];
  uint32_t *bins = reinterpret_cast<uint32_t *>(sm + L::kBins);
  // per (row, warp): scan of the packed counts, mask of code < v, mask of code == v
  uint4 *S4 = reinterpret_cast<uint4 *>(sm + L::kStage);
  SubNode *cur = reinterpret_cast<SubNode *>(sm + L::kSn0);
  SubNode *nxt = reinterpret_cast<SubNode *>(sm + L::kSn1);
  SubLeaf *LF = reinterpret_cast<SubLeaf *>(sm + L::kLeaf);
  SubMisc &M = *reinterpret_cast<SubMisc *>(sm + L::kMisc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t ltm = (1u << lane) - 1u;

  // ---- the node: ticket order, so every node before it has started ----
  if (threadIdx.x == 0) {
    M.j = atomicAdd(a.ticket, 1u);
    mbar_init(&M.bar, 1);
    mbar_fence_init();
  }
  constexpr uint32_t kV = 16 / sizeof(C);  // codes per 16 bytes
  if (threadIdx.x == 0) {
    const uint32_t j = M.j;
    uint64_t off64, cnt64;
    node_range(a.n, a.depth, j, off64, cnt64);
    M.off = off64;
    M.cnt = cnt64;
    const uint32_t lead = uint32_t(off64) & (kV - 1u), ilead = uint32_t(off64) & 3u;
    M.lead = lead;
    M.ilead = ilead;
    const uint32_t noff = uint32_t(off64), ncnt = uint32_t(cnt64);
    const uint32_t nwin = (lead + ncnt + kV - 1u) & ~(kV - 1u);
    const uint32_t niw = (ilead + ncnt + 3u) & ~3u;
    const bool dead = *reinterpret_cast<const volatile uint32_t *>(a.err) != 0u;
    M.skip = dead ? 1u : 0u;
    const bool ok = ncnt <= L::kCap && !dead;
    const uint32_t bytes = ok ? 3 * nwin * uint32_t(sizeof(C)) + (IDX ? 4 * niw : 0u) : 0u;
    if (!ok && !dead) atomicOr(a.err, kErrInternal);
    mbar_expect_tx(&M.bar, bytes);
    if (bytes) {
      for (int d = 0; d < 3; ++d)
        bulk_g2s(sm + d * L::kCodeStride, static_cast<const C *>(a.codes[d]) + (noff - lead),
                 nwin * uint32_t(sizeof(C)), &M.bar);
      if (IDX) bulk_g2s(sm + L::kIdx, a.idx + (noff - ilead), 4 * niw, &M.bar);
    }
    // the root of the subtree: its cell from the parent's split (k_prep's rule);
    // in a failed call the parents' records were never written and are not read
    SubNode &s = cur[0];
    if (a.depth == 0 || dead) {
      for (int d = 0; d < 3; ++d) {
        s.blo[d] = 0;
        s.bhi[d] = a.root_hi[d];
      }
    } else {
      const LevelNode &p = a.parents[j >> 1];
      for (int d = 0; d < 3; ++d) {
        s.blo[d] = p.blo[d];
        s.bhi[d] = p.bhi[d];
      }
      if (p.v != 0xffffffffu && p.axis < 3u) {
        if (j & 1) s.blo[p.axis] = p.v;
        else s.bhi[p.axis] = p.v;
      }
    }
    s.off = 0;
    s.cnt = ok ? ncnt : 0u;
    s.axis = WIDEST ? widest_axis(s.blo, s.bhi) : uint32_t(a.depth % 3);
    s.split = s.cnt > a.leaf_size;
  }
  // the radix bins start at zero (every select pass leaves them zero again)
  for (uint32_t b = threadIdx.x; b < kSubBins; b += kT) bins[b] = 0;
  if (warp == 0) tmem_alloc(&M.tmem, kTmemCols);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  // this thread's tensor-memory columns: lane quarter warp % 4, columns by warpgroup
  const uint32_t tcol = M.tmem + ((32u * (uint32_t(warp) & 3u)) << 16) + (uint32_t(warp) >> 2) * uint32_t(L::kCols);
  // A failed call (an earlier kernel, or this copy's wait giving up): the
  // node's status is published as complete, so that no later node waits for
  // it, and the CTA leaves.
  const bool late = wait_buffer(&M.bar, 0, a.err);
  if (__syncthreads_or(late || M.skip != 0u)) {
    if (!COST && threadIdx.x == 0) st_release_u64(a.status + M.j, kStIncl);
    tmem_fence_before();
    __syncthreads();
    if (warp == 0) {
      tmem_fence_after();
      tmem_dealloc(M.tmem, kTmemCols);
    }
    return;
  }
  // element i of the node (any array) sits at slot lead + i
  C *const X0 = reinterpret_cast<C *>(sm) + M.lead;

  // ---- the levels inside the CTA ----
  constexpr int NC = L::kCodeCols;                 // TMEM columns of one code array
  constexpr int RPC = sizeof(C) == 2 ? 2 : 1;      // rows per column
  constexpr uint32_t S = L::kCodeStride / sizeof(C);
  uint32_t *const XI = reinterpret_cast<uint32_t *>(sm + L::kIdx) + M.ilead;
  if (a.levels > 0) {  // the root's rows into TMEM (level 0: one group of all warps)
    const uint32_t cnt0 = cur[0].cnt;
    const uint32_t nv0 = cnt0 > threadIdx.x ? (cnt0 - threadIdx.x + kT - 1u) / kT : 0u;
    load_rows<R>(X0, nv0, kT, threadIdx.x, tcol);
    load_rows<R>(X0 + S, nv0, kT, threadIdx.x, tcol + NC);
    load_rows<R>(X0 + 2 * S, nv0, kT, threadIdx.x, tcol + 2 * NC);
    if (IDX) load_rows<R>(XI, nv0, kT, threadIdx.x, tcol + 3 * NC);
    tmem_wait_st();
  }
  const C *const Y0 = X0, *const Y1 = X0 + S, *const Y2 = X0 + 2 * S;
  // Leaves below the subnodes cur[0..G): the two halves of a splitting subnode
  // (with `halves`), else the subnode itself; their AABBs, centres (first
  // position on ties), widths (Eq. 2) and payload words, in LF.  Returns
  // their number.  Every thread calls it.
  auto leaf_boxes = [&](uint32_t G, bool halves) -> uint32_t {
    if (threadIdx.x == 0) {
      uint32_t nl = 0;
      for (uint32_t t = 0; t < G; ++t) {
        const SubNode &u = cur[t];
        if (halves && u.split) {
          const uint32_t kk = u.cnt >> 1;
          LF[nl].off = u.off;
          LF[nl++].cnt = kk;
          LF[nl].off = u.off + kk;
          LF[nl++].cnt = u.cnt - kk;
        } else {
          LF[nl].off = u.off;
          LF[nl++].cnt = u.cnt;
        }
      }
      M.nl = nl;
    }
    __syncthreads();
    const uint32_t nl = M.nl;
    if (threadIdx.x < nl) {
      for (int d = 0; d < 3; ++d) {
        LF[threadIdx.x].lo[d] = 0xffffffffu;
        LF[threadIdx.x].hi[d] = 0;
      }
    }
    const LeafSlots q = leaf_slots(nl, warp, lane);
    const uint32_t lgwl = q.lgwl, WL = q.WL, slots = q.slots, lt = q.lt, lstep = q.lstep;
    __syncthreads();
    // bit boxes: AABB
    for (uint32_t f = uint32_t(warp) >> lgwl; f < nl; f += slots) {
      const uint32_t off = LF[f].off, cnt = LF[f].cnt;
      uint32_t mn0 = 0xffffffffu, mn1 = 0xffffffffu, mn2 = 0xffffffffu, mx0 = 0, mx1 = 0, mx2 = 0;
      for (uint32_t i = lt; i < cnt; i += lstep) {
        const uint32_t c0 = Y0[off + i], c1 = Y1[off + i], c2 = Y2[off + i];
        mn0 = min(mn0, c0);
        mx0 = max(mx0, c0);
        mn1 = min(mn1, c1);
        mx1 = max(mx1, c1);
        mn2 = min(mn2, c2);
        mx2 = max(mx2, c2);
      }
      mn0 = __reduce_min_sync(0xffffffffu, mn0);
      mn1 = __reduce_min_sync(0xffffffffu, mn1);
      mn2 = __reduce_min_sync(0xffffffffu, mn2);
      mx0 = __reduce_max_sync(0xffffffffu, mx0);
      mx1 = __reduce_max_sync(0xffffffffu, mx1);
      mx2 = __reduce_max_sync(0xffffffffu, mx2);
      if (lane == 0) {
        atomicMin(&LF[f].lo[0], mn0);
        atomicMin(&LF[f].lo[1], mn1);
        atomicMin(&LF[f].lo[2], mn2);
        atomicMax(&LF[f].hi[0], mx0);
        atomicMax(&LF[f].hi[1], mx1);
        atomicMax(&LF[f].hi[2], mx2);
      }
    }
    __syncthreads();
    // centre: least squared distance to the AABB centre, first position on ties.
    // When every side of the box is below 2^15 codes, |2q - lo - hi| < 2^15 and
    // the squared distance is exact in 32 bits; otherwise it is formed in 64.
    {
      int it = 0;
      for (uint32_t f = uint32_t(warp) >> lgwl; f < nl; f += slots, ++it) {
        const uint32_t off = LF[f].off, cnt = LF[f].cnt;
        const uint32_t l0 = LF[f].lo[0], l1 = LF[f].lo[1], l2 = LF[f].lo[2];
        const uint32_t u0 = LF[f].hi[0], u1 = LF[f].hi[1], u2 = LF[f].hi[2];
        unsigned long long bd;
        uint32_t bp;
        if (max(u0 - l0, max(u1 - l1, u2 - l2)) < 32768u) {
          const int s0 = int(l0 + u0), s1 = int(l1 + u1), s2 = int(l2 + u2);
          uint32_t md = 0xffffffffu, mp = 0xffffffffu;
          for (uint32_t i = lt; i < cnt; i += lstep) {
            const int e0 = 2 * int(Y0[off + i]) - s0, e1 = 2 * int(Y1[off + i]) - s1, e2 = 2 * int(Y2[off + i]) - s2;
            const uint32_t d2 = uint32_t(e0 * e0) + uint32_t(e1 * e1) + uint32_t(e2 * e2);
            if (d2 < md) {  // positions rise within a thread: the first minimum is the lowest
              md = d2;
              mp = i;
            }
          }
          const uint32_t wmd = __reduce_min_sync(0xffffffffu, md);
          bp = __reduce_min_sync(0xffffffffu, md == wmd ? mp : 0xffffffffu);
          bd = wmd;
        } else {
          const long long s0 = (long long)l0 + u0, s1 = (long long)l1 + u1, s2 = (long long)l2 + u2;
          bd = ~0ull;
          bp = 0xffffffffu;
          for (uint32_t i = lt; i < cnt; i += lstep) {
            const long long e0 = 2ll * Y0[off + i] - s0, e1 = 2ll * Y1[off + i] - s1, e2 = 2ll * Y2[off + i] - s2;
            const unsigned long long d2 =
                (unsigned long long)(e0 * e0) + (unsigned long long)(e1 * e1) + (unsigned long long)(e2 * e2);
            if (d2 < bd) {
              bd = d2;
              bp = i;
            }
          }
  #pragma unroll
          for (int o = 16; o; o >>= 1) {
            const unsigned long long od = __shfl_xor_sync(0xffffffffu, bd, o);
            const uint32_t op = __shfl_xor_sync(0xffffffffu, bp, o);
            if (od < bd || (od == bd && op < bp)) {
              bd = od;
              bp = op;
            }
          }
        }
        if (lane == 0) {
          M.wd[warp][it] = bd;
          M.wp[warp][it] = bp;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < nl) {
      const uint32_t f = threadIdx.x;
      unsigned long long bd = ~0ull;
      uint32_t bp = 0xffffffffu;
      const bool turns = nl > uint32_t(kWarps);
      const uint32_t w0 = turns ? (f % kWarps) : (f << lgwl), wn = turns ? 1u : WL, it = turns ? (f / kWarps) : 0u;
      for (uint32_t w = w0; w < w0 + wn; ++w) {
        const unsigned long long od = M.wd[w][it];
        const uint32_t op = M.wp[w][it];
        if (od < bd || (od == bd && op < bp)) {
          bd = od;
          bp = op;
        }
      }
      SubLeaf &lf = LF[f];
      const uint32_t c = bp < lf.cnt ? bp : 0u;
      const uint32_t q0 = Y0[lf.off + c], q1 = Y1[lf.off + c], q2 = Y2[lf.off + c];
      const uint32_t m0 = bits_for_range(max(q0 - lf.lo[0], lf.hi[0] - q0));
      const uint32_t m1 = bits_for_range(max(q1 - lf.lo[1], lf.hi[1] - q1));
      const uint32_t m2 = bits_for_range(max(q2 - lf.lo[2], lf.hi[2] - q2));
      lf.qref[0] = int32_t(q0);
      lf.qref[1] = int32_t(q1);
      lf.qref[2] = int32_t(q2);
      lf.centre = c;
      lf.m = m0 | (m1 << 8) | (m2 << 16);
      lf.words = uint32_t((uint64_t(m0 + m1 + m2) * (lf.cnt ? lf.cnt - 1 : 0) + 31) >> 5);
    }
    __syncthreads();
    return nl;
  };
  // the leaf-size search: payload words of the leaves at in-CTA depth k
  auto add_cost = [&](uint32_t nl, int k) {
    if (warp == 0) {
      unsigned long long w = 0;
      for (uint32_t f = lane; f < nl; f += 32) w += LF[f].words;
#pragma unroll
      for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      if (lane == 0) atomicAdd(a.cost_words + k, w);
    }
  };
  if (COST) add_cost(leaf_boxes(1, false), 0);  // the node itself as one leaf
  for (int k = 0; k < a.levels; ++k) {
    const int lgW = kLgWarps - k;  // log2 of the warps per group
    const uint32_t G = 1u << k;
    const int g = warp >> lgW;
    const uint32_t Tg = uint32_t(kT) >> k;
    const uint32_t ltid = threadIdx.x & (Tg - 1u);
    const uint32_t BPG = kSubBins >> k, hb = 11u - uint32_t(k);
    const uint32_t soff = cur[g].off, scnt = cur[g].cnt;
    const uint32_t nv = scnt > ltid ? (scnt - ltid + Tg - 1u) / Tg : 0u;  // rows of this thread in its subnode
    const uint32_t tax = tcol + cur[g].axis * NC;                           // columns of the split axis
    if (threadIdx.x < G) sub_select_init(cur[threadIdx.x], hb);
    // radix select of every splitting subnode, one digit per pass, from the rows in TMEM
    bool any = __syncthreads_or(threadIdx.x < G && cur[threadIdx.x].width != 0);
    while (any) {
      const uint32_t width = cur[g].width;
      const bool act = width != 0;
      if (act) {
        const uint32_t lo = cur[g].lo, prefix = cur[g].prefix, shift = uint32_t(cur[g].shift);
        const uint32_t mask = (1u << width) - 1u;
        uint32_t *hg = bins + uint32_t(g) * BPG;
#pragma unroll
        for (int c0 = 0; c0 < NC; c0 += 8) {
          uint32_t v[8];
          tmem_ld_cols(tax + uint32_t(c0), v, NC - c0);
#pragma unroll
          for (int i = 0; i < 8 * RPC; ++i) {
            const int r = RPC * c0 + i;
            if (r < R && uint32_t(r) < nv) {
              const uint32_t hbk = (row_of<C>(v, i) - lo) >> shift;
              if ((hbk >> width) == prefix) atomicAdd(&hg[hbk & mask], 1u);
            }
          }
        }
      }
      __syncthreads();
      // the bucket holding rank cnt/2 - below: kBinsPer bins per thread, scanned within the group
      constexpr uint32_t kBinsPer = kSubBins / kT;
      const uint32_t b0 = kBinsPer * threadIdx.x;  // bins of this thread (in its own group's region)
      uint32_t h[kBinsPer], x = 0;
#pragma unroll
      for (uint32_t e = 0; e < kBinsPer; ++e) {
        h[e] = bins[b0 + e];
        bins[b0 + e] = 0;
        x += h[e];
      }
      if (!act) x = 0;
      uint32_t incl = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane == 31) M.wt[warp] = incl;
      __syncthreads();
      if (act) {
        uint32_t base = 0;
        for (int w = g << lgW; w < warp; ++w) base += M.wt[w];
        uint32_t ex = base + incl - x;
        const uint32_t target = (scnt >> 1) - cur[g].below;
        if (x && ex <= target && target < ex + x) {
          uint32_t e = 0;
          while (e + 1 < kBinsPer && target >= ex + h[e]) ex += h[e++];
          M.fb[g] = b0 - uint32_t(g) * BPG + e;
          M.fbefore[g] = ex;
        }
      }
      __syncthreads();
      bool still = false;
      if (act && ltid == 0) {
        SubNode &u = cur[g];
        u.below += M.fbefore[g];
        u.prefix = (u.prefix << u.width) | M.fb[g];
        if (u.shift == 0) {
          u.v = u.lo + u.prefix;
          u.tleft = (u.cnt >> 1) - u.below;
          u.width = 0;
        } else {
          const uint32_t w = uint32_t(u.shift) < hb ? uint32_t(u.shift) : hb;
          u.shift -= int32_t(w);
          u.width = w;
          still = true;
        }
      }
      any = __syncthreads_or(still);
    }

    const bool split = cur[g].split != 0;
    // classification: masks of code < v and code == v per (row, warp)
    {
      const uint32_t v = cur[g].v;
#pragma unroll
      for (int c0 = 0; c0 < NC; c0 += 8) {
        uint32_t cv[8];
        tmem_ld_cols(tax + uint32_t(c0), cv, NC - c0);
#pragma unroll
        for (int i = 0; i < 8 * RPC; ++i) {
          const int r = RPC * c0 + i;
          if (r >= R) break;
          const bool valid = split && uint32_t(r) < nv;
          const uint32_t c = row_of<C>(cv, i);
          const uint32_t lm = __ballot_sync(0xffffffffu, valid && c < v);
          const uint32_t tm = __ballot_sync(0xffffffffu, valid && c == v);
          if (lane == 0) {
            S4[r * kWarps + warp].y = lm;
            S4[r * kWarps + warp].z = tm;
          }
        }
      }
    }
    __syncthreads();
    // one block-wide exclusive scan over the entries (group, row, warp of the group),
    // the order of the positions within each subnode; kEPT consecutive entries per thread
    {
      constexpr uint32_t kE = uint32_t(R) * kWarps, kEPT = (kE + kT - 1) / kT;
      const uint32_t per_group = uint32_t(R) << lgW;
      uint32_t cx[kEPT], slot[kEPT], sum = 0;
#pragma unroll
      for (uint32_t e = 0; e < kEPT; ++e) {
        const uint32_t i = threadIdx.x * kEPT + e;
        cx[e] = 0;
        slot[e] = 0;
        if (i < kE) {
          const uint32_t gi = i / per_group;
          const uint32_t rem = i - gi * per_group;
          const uint32_t row = rem >> lgW, w = rem & ((1u << lgW) - 1u);
          slot[e] = row * kWarps + (gi << lgW) + w;
          cx[e] = (uint32_t(__popc(S4[slot[e]].y)) << 16) | uint32_t(__popc(S4[slot[e]].z));
        }
        sum += cx[e];
      }
      uint32_t inc = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane == 31) M.wt[warp] = inc;
      __syncthreads();
      if (warp == 0) {
        const uint32_t t = lane < kWarps ? M.wt[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
          if (lane >= o) ti += y;
        }
        if (lane < kWarps) M.wt[lane] = ti - t;
      }
      __syncthreads();
      uint32_t ex = M.wt[warp] + inc - sum;
#pragma unroll
      for (uint32_t e = 0; e < kEPT; ++e) {
        const uint32_t i = threadIdx.x * kEPT + e;
        if (i < kE) {
          S4[slot[e]].x = ex;
          if (i % per_group == 0) M.gb[i / per_group] = ex;
        }
        ex += cx[e];
      }
    }
    __syncthreads();
    // the move: every row from TMEM to its destination in shared memory
    {
      const uint32_t kk = scnt >> 1, gbase = M.gb[g], tleft = cur[g].tleft;
      C *const A0 = X0 + soff, *const A1 = X0 + S + soff, *const A2 = X0 + 2 * S + soff;
      uint32_t *const AI = XI + soff;
#pragma unroll
      for (int c0 = 0; c0 < NC; c0 += 4) {
        uint32_t v[12];
        tmem_ld4x3(tcol + uint32_t(c0), tcol + uint32_t(NC + c0), tcol + uint32_t(2 * NC + c0), v);
        uint32_t vi[4 * RPC];
        if (IDX) {
          tmem_ld4(tcol + uint32_t(3 * NC + RPC * c0), vi);
          if (RPC == 2) tmem_ld4(tcol + uint32_t(3 * NC + RPC * c0 + 4), vi + 4);
        }
#pragma unroll
        for (int i = 0; i < 4 * RPC; ++i) {
          const int r = RPC * c0 + i;
          if (uint32_t(r) < nv) {
            const uint32_t p = uint32_t(r) * Tg + ltid;
            uint32_t dst = p;
            if (split) {
              const uint4 e = S4[r * kWarps + warp];
              const uint32_t P = e.x - gbase;
              const uint32_t lb = (P >> 16) + uint32_t(__popc(e.y & ltm));
              uint32_t gl;
              bool left;
              if (e.z == 0) {  // no code of this warp's row equals v
                gl = lb + min(P & 0xffffu, tleft);
                left = (e.y >> lane) & 1u;
              } else {
                const uint32_t tb = (P & 0xffffu) + uint32_t(__popc(e.z & ltm));
                left = ((e.y >> lane) & 1u) || (((e.z >> lane) & 1u) && tb < tleft);
                gl = lb + min(tb, tleft);
              }
              dst = left ? gl : kk + p - gl;
              if (dst >= scnt) {
                atomicOr(a.err, kErrInternal);
                dst = p;
              }
            }
            A0[dst] = C(row_of<C>(v, i));
            A1[dst] = C(row_of<C>(v + 4, i));
            A2[dst] = C(row_of<C>(v + 8, i));
            if (IDX) AI[dst] = vi[i];
          }
        }
      }
    }
    // children of every subnode (every subnode above the last level splits)
    if (k + 1 < a.levels && threadIdx.x < G) {
      const SubNode &u = cur[threadIdx.x];
      if (!u.split) atomicOr(a.err, kErrInternal);
      const uint32_t kk = u.cnt >> 1;
      SubNode &cl = nxt[2 * threadIdx.x], &cr = nxt[2 * threadIdx.x + 1];
      for (int d = 0; d < 3; ++d) {
        cl.blo[d] = cr.blo[d] = u.blo[d];
        cl.bhi[d] = cr.bhi[d] = u.bhi[d];
      }
      cl.bhi[u.axis] = u.v;
      cr.blo[u.axis] = u.v;
      cl.off = u.off;
      cl.cnt = kk;
      cr.off = u.off + kk;
      cr.cnt = u.cnt - kk;
      const uint32_t ax = uint32_t((a.depth + k + 1) % 3);
      cl.axis = WIDEST ? widest_axis(cl.blo, cl.bhi) : ax;
      cr.axis = WIDEST ? widest_axis(cr.blo, cr.bhi) : ax;
      cl.split = cl.cnt > a.leaf_size;
      cr.split = cr.cnt > a.leaf_size;
    }
    __syncthreads();  // the level's arrangement is complete in shared memory
    if (COST) add_cost(leaf_boxes(G, true), k + 1);
    if (k + 1 < a.levels) {
      SubNode *t = cur;
      cur = nxt;
      nxt = t;
      // this thread's rows of the next level back into TMEM
      const int g2 = warp >> (lgW - 1);
      const uint32_t Tg2 = Tg >> 1, ltid2 = threadIdx.x & (Tg2 - 1u);
      const uint32_t off2 = cur[g2].off, cnt2 = cur[g2].cnt;
      const uint32_t nv2 = cnt2 > ltid2 ? (cnt2 - ltid2 + Tg2 - 1u) / Tg2 : 0u;
      load_rows<R>(X0 + off2, nv2, Tg2, ltid2, tcol);
      load_rows<R>(X0 + S + off2, nv2, Tg2, ltid2, tcol + NC);
      load_rows<R>(X0 + 2 * S + off2, nv2, Tg2, ltid2, tcol + 2 * NC);
      if (IDX) load_rows<R>(XI + off2, nv2, Tg2, ltid2, tcol + 3 * NC);
      tmem_wait_st();
      // the next level's moves overwrite shared memory only after its selection's barriers
    }
  }

  if (COST) {
    // the search pass: the deepest in-CTA arrangement back to HBM when asked
    // (a deeper search continues there); no leaf records, look-back or packing
    if (a.wb_codes[0]) {
      const uint64_t o = M.off;
      const uint32_t cnt = uint32_t(M.cnt);
      for (uint32_t i = threadIdx.x; i < cnt; i += kT) {
        static_cast<C *>(a.wb_codes[0])[o + i] = X0[i];
        static_cast<C *>(a.wb_codes[1])[o + i] = X0[S + i];
        static_cast<C *>(a.wb_codes[2])[o + i] = X0[2 * S + i];
        if (IDX) a.wb_idx[o + i] = XI[i];
      }
      // and the records of the last in-CTA level (depth + levels - 1), the parents of the
      // level over HBM that continues from there: their cells and splits (k_prep's fields)
      if (a.wb_nodes && a.levels > 0) {
        const uint32_t G = 1u << (a.levels - 1);
        if (threadIdx.x < G) {
          const SubNode &u = cur[threadIdx.x];
          LevelNode nd = {};
          for (int d = 0; d < 3; ++d) {
            nd.blo[d] = u.blo[d];
            nd.bhi[d] = u.bhi[d];
          }
          nd.axis = u.axis;
          nd.v = u.split ? u.v : 0xffffffffu;
          a.wb_nodes[(uint64_t(M.j) << (a.levels - 1)) + threadIdx.x] = nd;
        }
      }
    }
    tmem_fence_before();
    __syncthreads();
    if (warp == 0) {
      tmem_fence_after();
      tmem_dealloc(M.tmem, kTmemCols);
    }
    return;
  }
  // ---- leaves: the last level's subnodes, split or not, in order ----
  const uint32_t nl = leaf_boxes(a.levels > 0 ? 1u << (a.levels - 1) : 1u, true);
  const LeafSlots q = leaf_slots(nl, warp, lane);
  const uint32_t lgwl = q.lgwl, WL = q.WL, slots = q.slots, lw = q.lw, lt = q.lt, lstep = q.lstep;
  // ---- payload words before this node: decoupled look-back ----
  const uint32_t j = M.j;
  if (warp == 0) {
    unsigned long long agg = 0;
    for (uint32_t f = lane; f < nl; f += 32) agg += LF[f].words;
#pragma unroll
    for (int o = 16; o; o >>= 1) agg += __shfl_xor_sync(0xffffffffu, agg, o);
    if (lane == 0) st_release_u64(a.status + j, (j == 0 ? kStIncl : kStAgg) | agg);
    unsigned long long prefix = 0;
    if (j > 0) {
      long long i = (long long)j - 1;
      uint32_t spins = 0;
      for (;;) {
        const long long q = i - lane;
        const unsigned long long st = q >= 0 ? ld_acquire_u64(a.status + q) : kStIncl;
        const unsigned long long flag = st >> 62;
        const uint32_t incl = __ballot_sync(0xffffffffu, flag == 2), zero = __ballot_sync(0xffffffffu, flag == 0);
        const int fi = incl ? __ffs(incl) - 1 : 32;
        const uint32_t rel = fi >= 31 ? 0xffffffffu : ((2u << fi) - 1u);
        if (zero & rel) {
          if (++spins > kLookSpin) {
            if (lane == 0) atomicOr(a.err, kErrTimeout);
            break;
          }
          __nanosleep(64);
          continue;
        }
        unsigned long long v = lane <= fi ? (st & kStVal) : 0ull;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        prefix += v;
        if (fi < 32) break;
        i -= 32;
      }
      if (lane == 0) st_release_u64(a.status + j, kStIncl | (prefix + agg));
    }
    if (lane == 0) {
      if (uint64_t(j) + 1 == (1ull << a.depth)) *a.total_words = prefix + agg;
      unsigned long long run = prefix;
      for (uint32_t f = 0; f < nl; ++f) {
        LF[f].word_off = run;
        run += LF[f].words;
      }
    }
  }
  __syncthreads();

  // ---- leaf records, permutation and packed payload ----
  const uint64_t off64 = M.off;
  const uint64_t leaf0 =
      uint64_t(j) * a.leaves_small + (off64 - uint64_t(j) * (a.n >> a.depth)) * (a.leaves_big - a.leaves_small);
  uint32_t *sw = reinterpret_cast<uint32_t *>(sm + L::kStage) + warp * 96;
  uint32_t *payload0 = reinterpret_cast<uint32_t *>(a.out + kHeaderBytes + uint64_t(kLeafBytes) * a.num_leaves);
  for (uint32_t f = uint32_t(warp) >> lgwl; f < nl; f += slots) {
    const uint32_t foff = LF[f].off, fcnt = LF[f].cnt, centre = LF[f].centre, fm = LF[f].m, words = LF[f].words;
    const unsigned long long word_off = LF[f].word_off;
    const uint64_t gl = leaf0 + f, goff = off64 + foff;
    if (gl >= a.num_leaves || goff + fcnt > a.n || word_off + words > a.payload_cap) {
      if (lt == 0) atomicOr(a.err, kErrInternal);
      continue;
    }
    const uint32_t r0 = uint32_t(LF[f].qref[0]), r1 = uint32_t(LF[f].qref[1]), r2 = uint32_t(LF[f].qref[2]);
    if (lt == 0) {
      uint4 *rec = reinterpret_cast<uint4 *>(a.out + kHeaderBytes + uint64_t(kLeafBytes) * gl);
      rec[0] = make_uint4(uint32_t(goff), uint32_t(goff >> 32), uint32_t(word_off), uint32_t(word_off >> 32));
      rec[1] = make_uint4(r0, r1, r2, fm);
    }
    if (IDX && a.perm) {
      const uint32_t *XI = reinterpret_cast<const uint32_t *>(sm + L::kIdx) + M.ilead + foff;
      for (uint32_t i = lt; i < fcnt; i += lstep) {
        const uint32_t src = i == 0 ? centre : (i - 1 < centre ? i - 1 : i);
        a.perm[goff + i] = XI[src];
      }
    }
    const uint32_t m0 = fm & 0xffu, m1 = (fm >> 8) & 0xffu, m2 = (fm >> 16) & 0xffu;
    const uint32_t w = m0 + m1 + m2;
    if (w == 0 || fcnt < 2) continue;
    uint32_t *payload = payload0 + word_off;
    const uint32_t h0 = m0 ? (1u << (m0 - 1)) - 1u : 0u;
    const uint32_t h1 = m1 ? (1u << (m1 - 1)) - 1u : 0u;
    const uint32_t h2 = m2 ? (1u << (m2 - 1)) - 1u : 0u;
    const uint32_t nsl = fcnt - 1, chunks = (nsl + 31) / 32;
    // w <= 32: word k of a chunk takes bits from lanes i0 = 32k / w on (at most nit of them)
    const uint32_t i0 = w <= 32 ? (32u * lane) / w : 0u;
    const int sh0 = int(i0 * w) - int(32u * lane);
    const uint32_t nit = w <= 32 ? (31u + w) / w + 1u : 0u;
    const C *x0 = Y0 + foff, *x1 = Y1 + foff, *x2 = Y2 + foff;
    for (uint32_t ch = lw; ch < chunks; ch += WL) {
      // this lane's particle as one w-bit value c_x | c_y << m_x | c_z << (m_x + m_y), in three limbs
      const uint32_t sl = ch * 32 + lane;
      uint32_t v0 = 0, v1 = 0, v2 = 0;
      if (sl < nsl) {
        const uint32_t p = sl < centre ? sl : sl + 1;
        const uint32_t cx = m0 ? uint32_t(x0[p]) - r0 + h0 : 0u;
        const uint32_t cy = m1 ? uint32_t(x1[p]) - r1 + h1 : 0u;
        const uint32_t cz = m2 ? uint32_t(x2[p]) - r2 + h2 : 0u;
        const unsigned long long y = (unsigned long long)cy << m0;
        v0 = cx | uint32_t(y);
        v1 = uint32_t(y >> 32);
        const uint32_t s2 = m0 + m1;
        const unsigned long long z = (unsigned long long)cz << (s2 & 31);
        if (s2 < 32) {
          v0 |= uint32_t(z);
          v1 |= uint32_t(z >> 32);
        } else {
          v1 |= uint32_t(z);
          v2 = uint32_t(z >> 32);
        }
      }
      if (w <= 32) {
        // lane k assembles word k of the chunk from the lanes whose values overlap it
        uint32_t word = 0;
        for (uint32_t t = 0; t < nit; ++t) {
          const uint32_t i = i0 + t;
          const uint32_t vi = __shfl_sync(0xffffffffu, v0, i & 31u);
          const int sh = sh0 + int(t * w);
          if (i < 32 && sh < 32) word |= sh >= 0 ? (vi << sh) : (vi >> -sh);
        }
        const uint32_t gw = ch * w + lane;
        if (lane < w && gw < words) __stcs(payload + gw, word);
      } else {
        for (uint32_t t = lane; t < w; t += 32) sw[t] = 0;
        __syncwarp();
        if (sl < nsl) {
          const uint32_t b = lane * w, k0 = b >> 5, sh = b & 31;
          const uint32_t nwd = (sh + w + 31) >> 5;
          atomicOr(&sw[k0], v0 << sh);
          if (nwd > 1) atomicOr(&sw[k0 + 1], __funnelshift_l(v0, v1, sh));
          if (nwd > 2) atomicOr(&sw[k0 + 2], __funnelshift_l(v1, v2, sh));
          if (nwd > 3) atomicOr(&sw[k0 + 3], __funnelshift_l(v2, 0u, sh));
        }
        __syncwarp();
        for (uint32_t t = lane; t < w; t += 32) {
          const uint32_t gw = ch * w + t;
          if (gw < words) __stcs(payload + gw, sw[t]);
        }
        __syncwarp();
      }
    }
  }
  // every warp is done with tensor memory before warp 0 frees it
  tmem_fence_before();
  __syncthreads();
  if (warp == 0) {
    tmem_fence_after();
    tmem_dealloc(M.tmem, kTmemCols);
  }
}

template <typename C, bool IDX, bool WIDEST, bool COST>
cudaError_t subtree_launch_as(const SubtreeLaunch &a, cudaStream_t st) {
  const uint32_t smem = SubL<C, IDX>::kTotal;
  int per_sm = 0;
  cudaError_t e = resident_blocks<k_subtree<C, IDX, WIDEST, COST>>(kT, smem, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  TraceScope ts(COST ? "k_subtree_cost" : "k_subtree", st);
  k_subtree<C, IDX, WIDEST, COST><<<unsigned(1ull << a.depth), kT, smem, st>>>(a);
  return cudaGetLastError();
}
template <typename C, bool IDX, bool WIDEST>
cudaError_t subtree_launch(const SubtreeLaunch &a, cudaStream_t st) {
  return a.cost_words ? subtree_launch_as<C, IDX, WIDEST, true>(a, st) : subtree_launch_as<C, IDX, WIDEST, false>(a, st);
}

}  // namespace

uint32_t subtree_capacity(int code_bytes, bool with_idx) {
  return code_bytes == 2 ? (with_idx ? SubL<uint16_t, true>::kCap : SubL<uint16_t, false>::kCap)
                         : (with_idx ? SubL<uint32_t, true>::kCap : SubL<uint32_t, false>::kCap);
}

cudaError_t launch_subtree(const SubtreeLaunch &a, cudaStream_t st) {
  if (a.code_bytes == 2) {
    if (a.idx) return a.widest ? subtree_launch<uint16_t, true, true>(a, st) : subtree_launch<uint16_t, true, false>(a, st);
    return a.widest ? subtree_launch<uint16_t, false, true>(a, st) : subtree_launch<uint16_t, false, false>(a, st);
  }
  if (a.idx) return a.widest ? subtree_launch<uint32_t, true, true>(a, st) : subtree_launch<uint32_t, true, false>(a, st);
  return a.widest ? subtree_launch<uint32_t, false, true>(a, st) : subtree_launch<uint32_t, false, false>(a, st);
}

}  // namespace pcx
