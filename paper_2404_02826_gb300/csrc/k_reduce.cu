// Bit-box reduction (Sec. 4.1, "bit box reduction and bit box intersection
// update"; Alg. 1 of arXiv 2404.02826), in rounds of pairwise disjoint boxes.
//
// Input: the codes after the last k-d level, stored leaf after leaf ("slots").
// Every leaf starts as a box: the bit box of its particles that are not yet in
// a sequence ("live", one bit per slot).  Once a sequence holds a particle,
// owner[slot] is the box whose sequence it is and rank[slot] its place in it;
// the output position is the sequence's first position plus the rank.
//
// Intersection query: a 32-ary tree over the box indices.  Level 0 are the
// boxes; node j of level k >= 1 holds the union of the alive bit boxes below
// its children [32j, 32j + 32) of level k - 1 and the least (key, index) of
// those boxes (key = m_x + m_y + m_z).  It is updated bottom-up after every
// round (the paper's bottom-up update: only nodes above changed boxes, each
// by the warp that settles its last pending change) and searched top-down,
// 32 children per warp-wide test, so that boxes come out in increasing index.
//
// One round:
//   select   a warp per alive box a: a is taken when no other alive box with a
//            smaller (key, index) meets its bit box (the box found blocking it
//            in an earlier round is checked first).  Taken boxes are pairwise
//            disjoint, so no particle lies in two of them.
//   take     a block per taken box: ranks in its sequence for its centre, its
//            other live particles in slot order, then, for every alive box c
//            that is not taken and meets it, the live particles of c inside
//            its bit box, by c and slot (counted first, then ranked); boxes
//            that lost particles are listed.
//   scan     one block: each taken box's sequence index and first output
//            position, in box order, after the sequences of earlier rounds.
//   rebuild  a block per listed box: the bit box of what it keeps (the leaf
//            rules: AABB, the particle closest to its centre, Eq. 2); taken and
//            emptied boxes die; the tree nodes above them are recomputed.
// The host reads the alive count back every few rounds; rounds issued after
// the last box died return at once.  A final pass moves codes and input
// indices to their output positions for the packing kernels.
#include <climits>
#include <cstdint>

#include "pc_host.cuh"
#include "pc_internal.cuh"
#include "pc_reduce.cuh"

namespace pcx {
namespace {

constexpr int kMaxLevels = 8;  // 32^7 > 2^32 boxes
constexpr uint32_t kAlive = 1u, kTaken = 2u;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kListCap = 512;  // boxes met by a taken box, per batch
constexpr int kRoundsPerCheck = 8;

struct RBox {            // what the tree tests, 32 bytes
  int32_t lo[3], hi[3];  // bit box: q_ref -/+ (2^(m-1) - 1) per axis (q_ref where m = 0)
  uint32_t key;          // m_x + m_y + m_z
  uint32_t state;        // kAlive | kTaken
};
struct TNode {           // 32 bytes
  int32_t lo[3], hi[3];  // union of the alive bit boxes below (lo > hi: none)
  unsigned long long min;  // least key << 32 | index below, ~0 for none
};
struct RInfo {  // the rest of a box, 64 bytes
  int32_t qref[3];
  uint32_t m;       // m_x | m_y << 8 | m_z << 16
  uint32_t centre;  // slot of the centre
  uint32_t live;    // live particles
  uint32_t off, cnt;  // the leaf's slots
  uint32_t tlo[3], thi[3];  // AABB of the live particles
  uint32_t lost;    // set while listed for a rebuild
  uint32_t pad;
};
static_assert(sizeof(RBox) == 32 && sizeof(TNode) == 32 && sizeof(RInfo) == 64, "box layouts");

struct RCounters {
  uint32_t alive, taken, nlost, nseq, filled, rounds, done, pad;
};

struct Tree {
  RBox *box;
  TNode *node[kMaxLevels];       // node[k], 1 <= k <= top
  uint32_t *ticket[kMaxLevels];  // ticket[k], 2 <= k <= top: children of node j refitted so far
  uint32_t *pend[kMaxLevels];    // pend[k], 1 <= k < top: changes below node j not yet settled
  uint32_t count[kMaxLevels];    // count[0] = boxes, count[top] = 1
  int top;
};

struct State {
  Tree t;
  RInfo *info;
  uint32_t *live;     // [n / 32 + 1] bit s: slot s is live
  uint32_t *dest;     // [n] the box whose sequence holds the particle
  uint32_t *rank;     // [n] place in that sequence
  uint32_t *seq_cnt;  // [boxes] particles of a taken box's sequence, 0 otherwise
  uint32_t *seq_pos;  // [boxes] first output position of a taken box's sequence
  uint32_t *taken;    // [boxes] boxes taken in the round, any order
  uint32_t *lost;     // [boxes] boxes that lost particles in the round, any order
  uint32_t *tbits;    // [boxes / 32] bitmap of the boxes taken in the round
  uint32_t *blocker;  // [boxes] the box found blocking this one in an earlier round (~0: none yet)
  RCounters *ctr;
  uint32_t nl;
};

struct Layout {
  uint64_t live, dest, rank, blocker, box, info, node[kMaxLevels], ticket[kMaxLevels], pend[kMaxLevels], seq_cnt, seq_pos,
      taken, lost, tbits, ctr;
  uint64_t zero_begin, zero_end, total;
  uint32_t count[kMaxLevels];
  int top;
};

inline uint64_t align256(uint64_t x) { return (x + 255) / 256 * 256; }

Layout layout_of(uint64_t n, uint64_t nl) {
  Layout L = {};
  L.count[0] = uint32_t(nl);
  int k = 0;
  do {
    L.count[k + 1] = (L.count[k] + 31) / 32;
    ++k;
  } while (L.count[k] > 1);
  L.top = k;
  uint64_t o = 0;
  L.live = o;
  o = align256(o + 4 * (n / 32 + 2));
  L.dest = o;
  o = align256(o + 4 * n + 16);  // whole groups of four slots are read
  L.rank = o;
  o = align256(o + 4 * n);
  L.blocker = o;
  o = align256(o + 4 * nl);
  L.box = o;
  o = align256(o + sizeof(RBox) * nl);
  L.info = o;
  o = align256(o + sizeof(RInfo) * nl);
  for (int l = 1; l <= L.top; ++l) {
    L.node[l] = o;
    o = align256(o + sizeof(TNode) * L.count[l]);
  }
  L.seq_pos = o;
  o = align256(o + 4 * nl);
  L.taken = o;
  o = align256(o + 4 * nl);
  L.lost = o;
  o = align256(o + 4 * nl);
  L.zero_begin = o;  // zeroed once per call
  for (int l = 2; l <= L.top; ++l) {
    L.ticket[l] = o;
    o = align256(o + 4 * uint64_t(L.count[l]));
  }
  for (int l = 1; l < L.top; ++l) {
    L.pend[l] = o;
    o = align256(o + 4 * uint64_t(L.count[l]));
  }
  L.seq_cnt = o;
  o = align256(o + 4 * nl);
  L.tbits = o;
  o = align256(o + 4 * ((nl + 31) / 32));
  L.ctr = o;
  o = align256(o + sizeof(RCounters));
  L.zero_end = o;
  L.total = o;
  return L;
}

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

// A bit box in registers.
struct Box6 {
  int32_t lo[3], hi[3];
};
// Does the box stored as (p, q) = (lo0 lo1 lo2 hi0, hi1 hi2 ...) meet `a`?
__device__ __forceinline__ bool meets(const Box6 &a, const int4 &p, const int4 &q) {
  return a.lo[0] <= p.w && p.x <= a.hi[0] && a.lo[1] <= q.x && p.y <= a.hi[1] && a.lo[2] <= q.y && p.z <= a.hi[2];
}

// ---- top-down search ----------------------------------------------------

struct Descent {
  uint32_t mask[kMaxLevels];  // children of the current node at each level still to visit
  uint32_t base[kMaxLevels];  // index of child 0 at each level
  int lvl;
  bool done;
};

// One warp tests the children [first, first + 32) of level `level`.
template <class NodeOk, class BoxOk>
__device__ __forceinline__ uint32_t test_children(const Tree &t, int level, uint32_t first, NodeOk nok, BoxOk bok) {
  const uint32_t i = first + (threadIdx.x & 31);
  bool ok = false;
  if (i < t.count[level]) {
    if (level == 0) {
      const int4 *p = reinterpret_cast<const int4 *>(t.box + i);
      ok = bok(i, p[0], p[1]);
    } else {
      const int4 *p = reinterpret_cast<const int4 *>(t.node[level] + i);
      ok = nok(p[0], p[1]);
    }
  }
  return __ballot_sync(0xffffffffu, ok);
}

template <class NodeOk, class BoxOk>
__device__ void descent_start(Descent &d, const Tree &t, NodeOk nok, BoxOk bok) {
  d.lvl = t.top - 1;
  d.base[d.lvl] = 0;
  d.mask[d.lvl] = test_children(t, d.lvl, 0, nok, bok);
  d.done = false;
}

// Continues the search.  take(first, mask) gets each nonempty group of wanted
// boxes (bit i: box first + i) in increasing index and returns true to pause;
// returns true when paused, false when the search is complete.
template <class NodeOk, class BoxOk, class Take>
__device__ bool descent_run(Descent &d, const Tree &t, NodeOk nok, BoxOk bok, Take take) {
  while (!d.done) {
    const int l = d.lvl;
    const uint32_t m = d.mask[l];
    if (m == 0) {
      if (l + 1 >= t.top)
        d.done = true;
      else
        d.lvl = l + 1;
      continue;
    }
    if (l == 0) {
      d.mask[0] = 0;
      if (take(d.base[0], m)) return true;
      continue;
    }
    d.mask[l] = m & (m - 1);
    const uint32_t first = (d.base[l] + uint32_t(__ffs(int(m)) - 1)) * 32;
    d.base[l - 1] = first;
    d.mask[l - 1] = test_children(t, l - 1, first, nok, bok);
    d.lvl = l - 1;
  }
  return false;
}

// ---- refit ----------------------------------------------------------------

__device__ __forceinline__ void warp_union(int32_t lo[3], int32_t hi[3], unsigned long long &mn) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    lo[d] = __reduce_min_sync(0xffffffffu, lo[d]);
    hi[d] = __reduce_max_sync(0xffffffffu, hi[d]);
  }
  for (int o = 16; o; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mn, o);
    mn = y < mn ? y : mn;
  }
}

// Child c of level l (a box when l = 0) as its part of a node: bounds and
// key << 32 | index of an alive box, the node itself above; nothing otherwise.
__device__ __forceinline__ void load_child(const Tree &t, int l, uint32_t c, int32_t lo[3], int32_t hi[3],
                                           unsigned long long &mn) {
  lo[0] = lo[1] = lo[2] = INT_MAX;
  hi[0] = hi[1] = hi[2] = INT_MIN;
  mn = ~0ull;
  if (c >= t.count[l]) return;
  const int4 *q = l == 0 ? reinterpret_cast<const int4 *>(t.box + c) : reinterpret_cast<const int4 *>(t.node[l] + c);
  const int4 a = __ldcg(q), b = __ldcg(q + 1);
  if (l == 0 && !(uint32_t(b.w) & kAlive)) return;
  lo[0] = a.x;
  lo[1] = a.y;
  lo[2] = a.z;
  hi[0] = a.w;
  hi[1] = b.x;
  hi[2] = b.y;
  mn = l == 0 ? (static_cast<unsigned long long>(uint32_t(b.z)) << 32) | c
              : (static_cast<unsigned long long>(uint32_t(b.w)) << 32) | uint32_t(b.z);
}

// One warp recomputes node j of level l >= 1 from its 32 children.
__device__ __forceinline__ void warp_refit_node(const Tree &t, int l, uint32_t j) {
  int32_t lo[3], hi[3];
  unsigned long long mn;
  load_child(t, l - 1, j * 32 + (threadIdx.x & 31), lo, hi, mn);
  warp_union(lo, hi, mn);
  if ((threadIdx.x & 31) == 0) t.node[l][j] = TNode{{lo[0], lo[1], lo[2]}, {hi[0], hi[1], hi[2]}, mn};
}

// A box about to change this round (taken, or losing particles): one more
// pending change below each of its nodes that was clean (one thread).
__device__ __forceinline__ void mark_dirty(const Tree &t, uint32_t c) {
  uint32_t j = c;
  for (int l = 1; l < t.top; ++l) {
    j >>= 5;
    if (atomicAdd(t.pend[l] + j, 1u) != 0u) return;
  }
}

// After box c's new record is written: one pending change fewer; the warp
// that settles the last change below a node recomputes it and goes on up
// (the root is never searched and is not kept up to date).
__device__ __forceinline__ void warp_settle(const Tree &t, uint32_t c) {
  uint32_t j = c;
  for (int l = 1; l < t.top; ++l) {
    j >>= 5;
    uint32_t old = 0;
    if ((threadIdx.x & 31) == 0) {
      __threadfence();
      old = atomicSub(t.pend[l] + j, 1u);
    }
    old = __shfl_sync(0xffffffffu, old, 0);
    if (old != 1u) return;
    __threadfence();
    warp_refit_node(t, l, j);
  }
}

// The whole tree (after the first boxes): a warp per node of level 1; the
// warp that completes the last child of a node (ticket) goes on to compute
// that node, up to the root.
__global__ void __launch_bounds__(kThreads) k_rd_refit(State S) {
  const int lane = threadIdx.x & 31;
  uint32_t j = (blockIdx.x * kThreads + threadIdx.x) >> 5;
  if (j >= S.t.count[1]) return;
  warp_refit_node(S.t, 1, j);
  for (int l = 1; l < S.t.top; ++l) {
    const uint32_t p = j >> 5;
    const uint32_t kids = min(32u, S.t.count[l] - p * 32);
    uint32_t tk = 0;
    if (lane == 0) {
      __threadfence();
      tk = atomicAdd(S.t.ticket[l + 1] + p, 1u);
    }
    tk = __shfl_sync(0xffffffffu, tk, 0);
    if (tk + 1 != kids) return;
    if (lane == 0) S.t.ticket[l + 1][p] = 0;
    __threadfence();
    warp_refit_node(S.t, l + 1, p);
    j = p;
  }
}

// ---- select ---------------------------------------------------------------

__device__ __forceinline__ Box6 box6(const RBox &b) {
  Box6 x;
  for (int d = 0; d < 3; ++d) {
    x.lo[d] = b.lo[d];
    x.hi[d] = b.hi[d];
  }
  return x;
}

__global__ void __launch_bounds__(kThreads) k_rd_select(State S) {
  if (S.ctr->alive == 0) return;
  const uint32_t a = (blockIdx.x * kThreads + threadIdx.x) >> 5;
  if (a >= S.nl) return;
  const RBox A = S.t.box[a];
  if (!(A.state & kAlive)) return;
  const unsigned long long ka = (static_cast<unsigned long long>(A.key) << 32) | a;
  const Box6 bx = box6(A);
  // the box that blocked this one before usually still does: alive, a smaller key, meeting it
  const uint32_t bl = S.blocker[a];
  if (bl != 0xffffffffu) {
    const int4 *q = reinterpret_cast<const int4 *>(S.t.box + bl);
    const int4 p0 = q[0], p1 = q[1];
    const unsigned long long kb = (static_cast<unsigned long long>(uint32_t(p1.z)) << 32) | bl;
    if ((uint32_t(p1.w) & kAlive) && kb < ka && meets(bx, p0, p1)) return;
  }
  auto nok = [&](const int4 &p, const int4 &q) {
    const unsigned long long mn = (static_cast<unsigned long long>(uint32_t(q.w)) << 32) | uint32_t(q.z);
    return mn < ka && meets(bx, p, q);
  };
  auto bok = [&](uint32_t c, const int4 &p, const int4 &q) {
    const unsigned long long kc = (static_cast<unsigned long long>(uint32_t(q.z)) << 32) | c;
    return (uint32_t(q.w) & kAlive) && kc < ka && meets(bx, p, q);
  };
  Descent d;
  descent_start(d, S.t, nok, bok);
  uint32_t found = 0xffffffffu;
  const bool blocked = descent_run(d, S.t, nok, bok, [&](uint32_t first, uint32_t m) {
    found = first + uint32_t(__ffs(int(m)) - 1);
    return true;
  });
  if (blocked && (threadIdx.x & 31) == 0) S.blocker[a] = found;
  if (!blocked && (threadIdx.x & 31) == 0) {
    atomicOr(&S.t.box[a].state, kTaken);
    atomicOr(S.tbits + (a >> 5), 1u << (a & 31));
    S.taken[atomicAdd(&S.ctr->taken, 1u)] = a;
    mark_dirty(S.t, a);
  }
}

// ---- count and place ------------------------------------------------------

constexpr int kTakeThreads = 1024;
constexpr int kTakeWarps = kTakeThreads / 32;
static_assert(kTakeWarps >= 2 && kTakeWarps <= 32, "take: a search warp and an own-particle warp, one scan warp");

template <typename C>
struct Codes4;  // the codes of the aligned group of four slots g, as loaded (two or four words)
template <>
struct Codes4<uint16_t> {
  using Raw = uint2;
  static __device__ __forceinline__ Raw load(const uint16_t *q, uint32_t g) {
    return __ldg(reinterpret_cast<const uint2 *>(q) + g);
  }
  static __device__ __forceinline__ uint32_t at(const Raw &w, int j) {
    const uint32_t x = j < 2 ? w.x : w.y;
    return (j & 1) ? (x >> 16) : (x & 0xffffu);
  }
};
template <>
struct Codes4<uint32_t> {
  using Raw = uint4;
  static __device__ __forceinline__ Raw load(const uint32_t *q, uint32_t g) {
    return __ldg(reinterpret_cast<const uint4 *>(q) + g);
  }
  static __device__ __forceinline__ uint32_t at(const Raw &w, int j) {
    return j == 0 ? w.x : (j == 1 ? w.y : (j == 2 ? w.z : w.w));
  }
};

// A warp's picks over slots [off, end), recorded for the ranking pass: per
// lane, four bits (one group of four slots) for each group the lane visited,
// in visiting order.  Leaves hold at most PC_MAX_LEAF_SIZE particles, so a
// lane visits at most kRecWords * 8 groups of one leaf.
constexpr int kRecWords = 12;
template <typename C>
constexpr int kPickUnroll = sizeof(C) == 2 ? 4 : 2;  // groups per lane in flight: the same bytes for both widths
static_assert(((PC_MAX_LEAF_SIZE + 3) / 4 + 1 + 31) / 32 <= kRecWords * 8, "pick record too small");
struct Picks {
  uint32_t w[kRecWords];
};

// One warp walks the live slots of [off, end) in aligned groups of four (lane
// i takes every 32nd group), a few groups per lane at a time: all their loads
// are issued first (indices clamped into the range, so no load waits on a
// branch), then the slots are tested.  want(s, x, y, z) picks live slot s (x,
// y, z its codes when CODES).  Records the picks and returns their number.
template <typename C, bool CODES, class Want>
__device__ __forceinline__ uint32_t warp_pick(const State &S, const C *q0, const C *q1, const C *q2, uint32_t off,
                                              uint32_t end, Want want, Picks &rec) {
  using Raw = typename Codes4<C>::Raw;
  constexpr int U = kPickUnroll<C>;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t g0 = off >> 2, g1 = (end + 3) >> 2;
  uint32_t k = 0, nib = 0;
  for (uint32_t gb = g0; gb < g1; gb += 32 * U) {
    uint32_t lw[U];
    Raw cx[U], cy[U], cz[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t g = min(gb + uint32_t(u) * 32 + lane, g1 - 1);
      lw[u] = __ldcg(S.live + (g >> 3));
      if (CODES) {
        cx[u] = Codes4<C>::load(q0, g);
        cy[u] = Codes4<C>::load(q1, g);
        cz[u] = Codes4<C>::load(q2, g);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u, ++nib) {
      const uint32_t g = gb + uint32_t(u) * 32 + lane;
      const uint32_t lb = g < g1 ? (lw[u] >> (4 * (g & 7))) & 0xfu : 0u;
      uint32_t bits = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t s = 4 * g + uint32_t(j);
        if (!((lb >> j) & 1u) || s < off || s >= end) continue;
        uint32_t x = 0, y = 0, z = 0;
        if (CODES) {
          x = Codes4<C>::at(cx[u], j);
          y = Codes4<C>::at(cy[u], j);
          z = Codes4<C>::at(cz[u], j);
        }
        if (want(s, x, y, z)) bits |= 1u << j;
      }
      if ((nib & 7) == 0) rec.w[nib >> 3] = 0;
      rec.w[nib >> 3] |= bits << (4 * (nib & 7));
      k += __popc(bits);
    }
  }
  return __reduce_add_sync(0xffffffffu, k);
}

// Replays a warp's picks over [off, end): they stop being live and get
// dest[s] = tag and rank[s] = pos, pos + 1, ... in slot order.
__device__ __forceinline__ void warp_place(const State &S, uint32_t tag, uint32_t off, uint32_t end, uint32_t pos,
                                           const Picks &rec, int unroll) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t g0 = off >> 2, g1 = (end + 3) >> 2;
  uint32_t nib = 0;
  for (uint32_t gb = g0; gb < g1; gb += 32 * uint32_t(unroll)) {
    for (int u = 0; u < unroll; ++u, ++nib) {
      const uint32_t bits = (rec.w[nib >> 3] >> (4 * (nib & 7))) & 0xfu;
      const uint32_t c = __popc(bits);
      uint32_t incl = c;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= uint32_t(o)) incl += y;
      }
      uint32_t p = pos + incl - c;
      pos += __shfl_sync(0xffffffffu, incl, 31);
      if (!bits) continue;
      const uint32_t g = gb + uint32_t(u) * 32 + lane;
      atomicAnd(S.live + (g >> 3), ~(bits << (4 * (g & 7))));
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if ((bits >> j) & 1u) {
          S.dest[4 * g + uint32_t(j)] = tag;
          S.rank[4 * g + uint32_t(j)] = p++;
        }
    }
  }
}

// The slots of part t of `parts` of box c (whole groups of four, in slot
// order), or an empty range when c's live particles miss bit box b; `all`
// tells that every live particle of c lies inside b.
__device__ __forceinline__ void take_range(const RInfo &I, uint32_t t, uint32_t parts, const Box6 &b, uint32_t &off,
                                           uint32_t &end, bool &all) {
  bool meet = true;
  all = true;
  for (int d = 0; d < 3; ++d) {
    const int32_t lo = int32_t(I.tlo[d]), hi = int32_t(I.thi[d]);
    if (lo > b.hi[d] || hi < b.lo[d]) meet = false;
    if (lo < b.lo[d] || hi > b.hi[d]) all = false;
  }
  off = end = 0;
  if (!meet) return;
  const uint32_t g0 = I.off >> 2, ng = ((I.off + I.cnt + 3) >> 2) - g0;  // ng * parts < 2^32
  off = max(I.off, 4 * (g0 + ng * t / parts));
  end = min(I.off + I.cnt, 4 * (g0 + ng * (t + 1) / parts));
  if (off > end) off = end;
}

// Live particles of slots [off, end) of a box inside bit box b (every live
// one when `all`), by one warp; records them for warp_place.
template <typename C>
__device__ __forceinline__ uint32_t warp_pick_inside(const State &S, const C *q0, const C *q1, const C *q2,
                                                     uint32_t off, uint32_t end, bool all, const Box6 &b, Picks &rec) {
  if (off >= end) return 0;
  if (all)
    return warp_pick<C, false>(S, q0, q1, q2, off, end, [](uint32_t, uint32_t, uint32_t, uint32_t) { return true; },
                               rec);
  return warp_pick<C, true>(S, q0, q1, q2, off, end,
                            [&](uint32_t, uint32_t x, uint32_t y, uint32_t z) {
                              return b.lo[0] <= int32_t(x) && int32_t(x) <= b.hi[0] && b.lo[1] <= int32_t(y) &&
                                     int32_t(y) <= b.hi[1] && b.lo[2] <= int32_t(z) && int32_t(z) <= b.hi[2];
                            },
                            rec);
}

// Barrier of the first `nthreads` threads of the block (whole warps), apart
// from __syncthreads: the search warps meet here while the last warp ranks
// the taken box's own particles.
__device__ __forceinline__ void search_sync(int nthreads) { asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory"); }

// A block per taken box: the ranks of its sequence, its length into seq_cnt.
// The last warp ranks the box's own particles while the others search the
// tree breadth first (one level per step, all nodes of a level at once; a
// level of more than kListCap boxes falls back to a depth-first search in
// batches by warp 0).  Then every warp counts, and after a scan ranks, pieces
// of the boxes met.
template <typename C>
__global__ void __launch_bounds__(kTakeThreads) k_rd_take(State S, const C *__restrict__ q0,
                                                          const C *__restrict__ q1, const C *__restrict__ q2) {
  constexpr int kSearchWarps = kTakeWarps - 1;
  __shared__ uint32_t fr[2][kListCap];  // search frontiers; the boxes met end in one of them
  __shared__ uint32_t fmask[kListCap];
  __shared__ uint32_t lpos[kListCap];
  __shared__ uint32_t s_nf, s_over, s_cur, s_n, s_done, s_sum;
  if (S.ctr->alive == 0) return;
  const uint32_t ntaken = S.ctr->taken;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t i = blockIdx.x; i < ntaken; i += gridDim.x) {
    const uint32_t a = S.taken[i];
    const RBox A = S.t.box[a];
    const Box6 bx = box6(A);
    const RInfo IA = S.info[a];
    auto nok = [&](const int4 &p, const int4 &q) { return meets(bx, p, q); };
    auto bok = [&](uint32_t, const int4 &p, const int4 &q) {
      return (uint32_t(q.w) & (kAlive | kTaken)) == kAlive && meets(bx, p, q);
    };
    if (warp == kTakeWarps - 1) {  // the centre, then the box's other live particles in slot order
      const uint32_t centre = IA.centre;
      Picks rec;
      warp_pick<C, false>(S, q0, q1, q2, IA.off, IA.off + IA.cnt,
                          [=](uint32_t s, uint32_t, uint32_t, uint32_t) { return s != centre; }, rec);
      warp_place(S, a, IA.off, IA.off + IA.cnt, 1, rec, kPickUnroll<C>);
      if (lane == 0) {
        atomicAnd(S.live + (centre >> 5), ~(1u << (centre & 31)));
        S.dest[centre] = a;
        S.rank[centre] = 0;
      }
    } else {
      const Tree &t = S.t;
      int cur = 0;
      if (warp == 0) {
        const uint32_t m = test_children(t, t.top - 1, 0, nok, bok);
        if ((m >> lane) & 1u) fr[0][__popc(m & lanemask_lt())] = lane;
        if (lane == 0) {
          s_nf = __popc(m);
          s_over = 0;
        }
      }
      search_sync(kSearchWarps * 32);
      for (int l = t.top - 1; l >= 1; --l) {  // fr[cur] holds the nodes of level l to expand
        const uint32_t nf = s_nf;
        for (uint32_t j = warp; j < nf; j += kSearchWarps) {
          const uint32_t m = test_children(t, l - 1, fr[cur][j] * 32, nok, bok);
          if (lane == 0) fmask[j] = m;
        }
        search_sync(kSearchWarps * 32);
        if (warp == 0) {
          uint32_t run = 0;
          for (uint32_t j0 = 0; j0 < nf; j0 += 32) {
            const uint32_t x = j0 + lane < nf ? __popc(fmask[j0 + lane]) : 0u;
            uint32_t incl = x;
            for (int o = 1; o < 32; o <<= 1) {
              const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
              if (lane >= o) incl += y;
            }
            if (j0 + lane < nf) lpos[j0 + lane] = run + incl - x;
            run += __shfl_sync(0xffffffffu, incl, 31);
          }
          if (lane == 0) {
            s_nf = run;
            s_over = run > kListCap ? 1u : 0u;
          }
        }
        search_sync(kSearchWarps * 32);
        if (s_over) break;
        for (uint32_t j = warp; j < nf; j += kSearchWarps) {
          const uint32_t m = fmask[j];
          if ((m >> lane) & 1u) fr[cur ^ 1][lpos[j] + __popc(m & lanemask_lt())] = fr[cur][j] * 32 + lane;
        }
        search_sync(kSearchWarps * 32);
        cur ^= 1;
      }
      if (threadIdx.x == 0) s_cur = uint32_t(cur);
    }
    __syncthreads();
    uint32_t pos = IA.live;
    // counts, then ranks, of `parts` pieces of each of the nlist boxes in list,
    // at most one piece per warp at a time (its picks stay in the warp's registers)
    auto batch = [&](const uint32_t *list, uint32_t nlist) {
      const uint32_t parts = nlist ? max(1u, min(16u, uint32_t(kTakeWarps) / nlist)) : 1u;
      const uint32_t items = nlist * parts;
      for (uint32_t i0 = 0; i0 < items; i0 += kTakeWarps) {
        const uint32_t it = i0 + uint32_t(warp);
        uint32_t c = 0, off = 0, end = 0, k = 0;
        Picks rec;
        if (it < items) {
          c = list[it / parts];
          bool all;
          take_range(S.info[c], it % parts, parts, bx, off, end, all);
          k = warp_pick_inside<C>(S, q0, q1, q2, off, end, all, bx, rec);
        }
        if (lane == 0) lpos[warp] = k;
        __syncthreads();
        if (warp == 0) {  // exclusive scan of the pieces' counts (one per warp of the block)
          const uint32_t x = lane < kTakeWarps ? lpos[lane] : 0u;
          uint32_t incl = x;
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
          }
          lpos[lane] = incl - x;
          if (lane == 31) s_sum = incl;
        }
        __syncthreads();
        if (k) {
          warp_place(S, a, off, end, pos + lpos[warp], rec, kPickUnroll<C>);
          if (lane == 0 && atomicExch(&S.info[c].lost, 1u) == 0u) {
            S.lost[atomicAdd(&S.ctr->nlost, 1u)] = c;
            mark_dirty(S.t, c);
          }
        }
        pos += s_sum;
        __syncthreads();  // lpos and s_sum are reused
      }
    };
    if (!s_over) {
      batch(fr[s_cur], s_nf);
    } else {
      // more boxes than a batch holds: depth first, in batches, by warp 0
      Descent d;
      if (warp == 0) descent_start(d, S.t, nok, bok);
      for (;;) {
        if (warp == 0) {
          uint32_t nlist = 0;
          descent_run(d, S.t, nok, bok, [&](uint32_t first, uint32_t m) {
            if ((m >> lane) & 1u) fr[0][nlist + __popc(m & lanemask_lt())] = first + lane;
            nlist += __popc(m);
            return nlist + 32 > kListCap;
          });
          if (lane == 0) {
            s_n = nlist;
            s_done = d.done ? 1u : 0u;
          }
        }
        __syncthreads();
        const uint32_t nlist = s_n;
        const bool done = s_done != 0;
        batch(fr[0], nlist);
        if (done) break;
      }
    }
    if (threadIdx.x == 0) S.seq_cnt[a] = pos;
    __syncthreads();
  }
}

// ---- scan -----------------------------------------------------------------

// Sequence index and first position of every taken box, in box order: one
// block over the bitmap of taken boxes, which it clears for the next round.
__global__ void __launch_bounds__(1024) k_rd_scan(State S, LeafRec *seqs) {
  __shared__ uint32_t ws[32], wc[32];
  if (S.ctr->alive == 0) return;
  const uint32_t filled = S.ctr->filled, nseq = S.ctr->nseq;
  const uint32_t nw = (S.nl + 31) / 32;
  const uint32_t per = (nw + 1023) / 1024;
  const uint32_t w0 = min(nw, threadIdx.x * per), w1 = min(nw, w0 + per);
  uint32_t sum = 0, cnt = 0;
  for (uint32_t w = w0; w < w1; ++w) {
    uint32_t b = S.tbits[w];
    cnt += __popc(b);
    while (b) {
      const uint32_t a = 32 * w + uint32_t(__ffs(int(b)) - 1);
      b &= b - 1;
      sum += S.seq_cnt[a];
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t is = sum, ic = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t ys = __shfl_up_sync(0xffffffffu, is, o), yc = __shfl_up_sync(0xffffffffu, ic, o);
    if (lane >= o) {
      is += ys;
      ic += yc;
    }
  }
  if (lane == 31) {
    ws[warp] = is;
    wc[warp] = ic;
  }
  __syncthreads();
  if (warp == 0) {
    const uint32_t xs = ws[lane], xc = wc[lane];
    uint32_t js = xs, jc = xc;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t ys = __shfl_up_sync(0xffffffffu, js, o), yc = __shfl_up_sync(0xffffffffu, jc, o);
      if (lane >= o) {
        js += ys;
        jc += yc;
      }
    }
    ws[lane] = js - xs;
    wc[lane] = jc - xc;
    if (lane == 31) {  // every thread has read the counters above
      S.ctr->filled = filled + js;
      S.ctr->nseq = nseq + jc;
      S.ctr->rounds += 1;
    }
  }
  __syncthreads();
  uint32_t pos = filled + ws[warp] + is - sum, seq = nseq + wc[warp] + ic - cnt;
  for (uint32_t w = w0; w < w1; ++w) {
    uint32_t b = S.tbits[w];
    if (!b) continue;
    S.tbits[w] = 0;
    while (b) {
      const uint32_t a = 32 * w + uint32_t(__ffs(int(b)) - 1);
      b &= b - 1;
      const uint32_t x = S.seq_cnt[a];
      S.seq_pos[a] = pos;
      const RInfo I = S.info[a];
      LeafRec r = {};
      r.off = pos;
      r.cnt = x;
      r.centre = 0;
      r.m = I.m;
      for (int d = 0; d < 3; ++d) r.qref[d] = I.qref[d];
      const uint64_t wb = (I.m & 0xffu) + ((I.m >> 8) & 0xffu) + ((I.m >> 16) & 0xffu);
      r.words = uint32_t((wb * (x - 1) + 31) >> 5);
      seqs[seq] = r;
      pos += x;
      ++seq;
    }
  }
}

// ---- rebuild --------------------------------------------------------------

constexpr int kBoxThreads = 128;
constexpr int kBoxWarps = kBoxThreads / 32;

// The block's threads visit the live slots of [off, end) (every slot when
// INIT) in aligned groups of four, four groups per thread at a time with their
// loads issued first; f(s, x, y, z) sees each slot in increasing order per thread.
template <typename C, bool INIT, class F>
__device__ __forceinline__ void box_walk(const State &S, const C *q0, const C *q1, const C *q2, uint32_t off,
                                         uint32_t end, F f) {
  using Raw = typename Codes4<C>::Raw;
  constexpr int U = 4;
  const uint32_t g0 = off >> 2, g1 = (end + 3) >> 2;
  for (uint32_t gb = g0; gb < g1; gb += U * kBoxThreads) {
    uint32_t lw[U];
    Raw cx[U], cy[U], cz[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t g = min(gb + uint32_t(u) * kBoxThreads + threadIdx.x, g1 - 1);
      lw[u] = INIT ? 0xffffffffu : __ldcg(S.live + (g >> 3));
      cx[u] = Codes4<C>::load(q0, g);
      cy[u] = Codes4<C>::load(q1, g);
      cz[u] = Codes4<C>::load(q2, g);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t g = gb + uint32_t(u) * kBoxThreads + threadIdx.x;
      if (g >= g1) continue;
      const uint32_t lb = (lw[u] >> (4 * (g & 7))) & 0xfu;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t s = 4 * g + uint32_t(j);
        if (!((lb >> j) & 1u) || s < off || s >= end) continue;
        f(s, Codes4<C>::at(cx[u], j), Codes4<C>::at(cy[u], j), Codes4<C>::at(cz[u], j));
      }
    }
  }
}

// INIT: every leaf's first box (all particles live; the counters start).
// Otherwise: the boxes listed by place get the bit box of their live
// particles or die when none is left; taken boxes die.
template <typename C, bool INIT>
__global__ void __launch_bounds__(kBoxThreads) k_rd_rebuild(State S, const C *__restrict__ q0,
                                                            const C *__restrict__ q1, const C *__restrict__ q2,
                                                            const LeafRec *__restrict__ leafs) {
  __shared__ uint32_t red[7][kBoxWarps];
  __shared__ unsigned long long rd[kBoxWarps];
  __shared__ uint32_t rp[kBoxWarps];
  if (INIT) {
    if (blockIdx.x == 0 && threadIdx.x == 0) S.ctr->alive = S.nl;  // the rest starts zeroed
  } else if (S.ctr->alive == 0) {
    return;
  }
  const uint32_t nlost = INIT ? S.nl : S.ctr->nlost;
  const uint32_t ntaken = INIT ? 0u : S.ctr->taken;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t i = blockIdx.x; i < nlost + ntaken; i += gridDim.x) {
    if (i >= nlost) {
      if (warp == 0) {
        const uint32_t a = S.taken[i - nlost];
        if (lane == 0) {
          S.t.box[a].state = 0;
          atomicSub(&S.ctr->alive, 1u);
        }
        warp_settle(S.t, a);
      }
      continue;
    }
    const uint32_t c = INIT ? i : S.lost[i];
    uint32_t off, cnt;
    if (INIT) {
      off = leafs[c].off;
      cnt = leafs[c].cnt;
    } else {
      off = S.info[c].off;
      cnt = S.info[c].cnt;
    }
    const uint32_t end = off + cnt;
    uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0, 0, 0}, live = 0;
    box_walk<C, INIT>(S, q0, q1, q2, off, end, [&](uint32_t, uint32_t x, uint32_t y, uint32_t z) {
      lo[0] = min(lo[0], x);
      hi[0] = max(hi[0], x);
      lo[1] = min(lo[1], y);
      hi[1] = max(hi[1], y);
      lo[2] = min(lo[2], z);
      hi[2] = max(hi[2], z);
      ++live;
    });
    for (int d = 0; d < 3; ++d) {
      lo[d] = __reduce_min_sync(0xffffffffu, lo[d]);
      hi[d] = __reduce_max_sync(0xffffffffu, hi[d]);
    }
    live = __reduce_add_sync(0xffffffffu, live);
    if (lane == 0) {
      for (int d = 0; d < 3; ++d) {
        red[2 * d][warp] = lo[d];
        red[2 * d + 1][warp] = hi[d];
      }
      red[6][warp] = live;
    }
    __syncthreads();
    live = 0;
    for (int d = 0; d < 3; ++d) {
      lo[d] = red[2 * d][0];
      hi[d] = red[2 * d + 1][0];
    }
    for (int w = 0; w < kBoxWarps; ++w) {
      live += red[6][w];
      for (int d = 0; d < 3; ++d) {
        lo[d] = min(lo[d], red[2 * d][w]);
        hi[d] = max(hi[d], red[2 * d + 1][w]);
      }
    }
    if (live == 0) {  // emptied by the round
      if (threadIdx.x == 0) {
        S.t.box[c].state = 0;
        S.info[c].live = 0;
        S.info[c].lost = 0;
        atomicSub(&S.ctr->alive, 1u);
      }
      if (warp == 0) warp_settle(S.t, c);
      __syncthreads();
      continue;
    }
    // centre: least squared distance to the AABB centre, lowest slot on ties
    unsigned long long bd = ~0ull;
    uint32_t bp = 0xffffffffu;
    const long long s0 = (long long)lo[0] + hi[0], s1 = (long long)lo[1] + hi[1], s2 = (long long)lo[2] + hi[2];
    box_walk<C, INIT>(S, q0, q1, q2, off, end, [&](uint32_t s, uint32_t x, uint32_t y, uint32_t z) {
      const long long a = 2ll * x - s0, b = 2ll * y - s1, e = 2ll * z - s2;
      const unsigned long long d2 =
          (unsigned long long)(a * a) + (unsigned long long)(b * b) + (unsigned long long)(e * e);
      if (d2 < bd) {  // slots rise within a thread: the first minimum is the lowest
        bd = d2;
        bp = s;
      }
    });
    for (int o = 16; o; o >>= 1) {
      const unsigned long long od = __shfl_xor_sync(0xffffffffu, bd, o);
      const uint32_t op = __shfl_xor_sync(0xffffffffu, bp, o);
      if (od < bd || (od == bd && op < bp)) {
        bd = od;
        bp = op;
      }
    }
    if (lane == 0) {
      rd[warp] = bd;
      rp[warp] = bp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kBoxWarps; ++w)
        if (rd[w] < bd || (rd[w] == bd && rp[w] < bp)) {
          bd = rd[w];
          bp = rp[w];
        }
      const uint32_t qc[3] = {uint32_t(q0[bp]), uint32_t(q1[bp]), uint32_t(q2[bp])};
      RInfo I = {};
      RBox B = {};
      uint32_t m[3];
      for (int d = 0; d < 3; ++d) {
        m[d] = bits_for_range(max(qc[d] - lo[d], hi[d] - qc[d]));
        const int32_t h = m[d] ? int32_t((1u << (m[d] - 1)) - 1u) : 0;
        I.qref[d] = int32_t(qc[d]);
        I.tlo[d] = lo[d];
        I.thi[d] = hi[d];
        B.lo[d] = int32_t(qc[d]) - h;
        B.hi[d] = int32_t(qc[d]) + h;
      }
      I.m = m[0] | (m[1] << 8) | (m[2] << 16);
      I.centre = bp;
      I.live = live;
      I.off = off;
      I.cnt = cnt;
      I.lost = 0;
      B.key = m[0] + m[1] + m[2];
      B.state = kAlive;
      S.info[c] = I;
      S.t.box[c] = B;
    }
    if (!INIT && warp == 0) warp_settle(S.t, c);
    __syncthreads();
  }
  // the last block to finish empties the round's lists for the next round
  if (!INIT && threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&S.ctr->done, 1u) == gridDim.x - 1) {
      S.ctr->taken = 0;
      S.ctr->nlost = 0;
      S.ctr->done = 0;
    }
  }
}

// ---- sequence order ---------------------------------------------------------

template <typename C>
__global__ void k_rd_gather(State S, uint64_t n, const C *__restrict__ q0, const C *__restrict__ q1,
                            const C *__restrict__ q2, C *o0, C *o1, C *o2, const uint32_t *__restrict__ idx,
                            uint32_t *oidx, uint32_t *err) {
  for (uint64_t s = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t a = S.dest[s];
    const uint64_t p = a < S.nl ? uint64_t(S.seq_pos[a]) + S.rank[s] : n;
    if (p >= n) {  // every particle is in exactly one sequence
      atomicOr(err, kErrInternal);
      continue;
    }
    o0[p] = q0[s];
    o1[p] = q1[s];
    o2[p] = q2[s];
    if (idx) oidx[p] = idx[s];
  }
}

// A CUDA graph of launches captured from a private stream; destroyed with it.
struct RoundGraph {
  cudaGraphExec_t exec = nullptr;
  template <typename Fn>
  void capture(Fn issue) {
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      issue(cs);
      if (cudaStreamEndCapture(cs, &g) == cudaSuccess && g) {
        if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
        cudaGraphDestroy(g);
      }
    }
    cudaStreamDestroy(cs);
    (void)cudaGetLastError();  // a failed capture leaves the launches to be issued one by one
  }
  ~RoundGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

template <typename C>
cudaError_t reduce_dispatch(const ReduceLaunch &a, cudaStream_t st, uint64_t *num_seq, uint64_t *rounds) {
  const Layout L = layout_of(a.n, a.num_leaves);
  uint8_t *base = static_cast<uint8_t *>(a.scratch);
  State S = {};
  S.t.box = reinterpret_cast<RBox *>(base + L.box);
  for (int l = 1; l <= L.top; ++l) S.t.node[l] = reinterpret_cast<TNode *>(base + L.node[l]);
  for (int l = 2; l <= L.top; ++l) S.t.ticket[l] = reinterpret_cast<uint32_t *>(base + L.ticket[l]);
  for (int l = 1; l < L.top; ++l) S.t.pend[l] = reinterpret_cast<uint32_t *>(base + L.pend[l]);
  for (int l = 0; l <= L.top; ++l) S.t.count[l] = L.count[l];
  S.t.top = L.top;
  S.info = reinterpret_cast<RInfo *>(base + L.info);
  S.live = reinterpret_cast<uint32_t *>(base + L.live);
  S.dest = reinterpret_cast<uint32_t *>(base + L.dest);
  S.rank = reinterpret_cast<uint32_t *>(base + L.rank);
  S.seq_cnt = reinterpret_cast<uint32_t *>(base + L.seq_cnt);
  S.seq_pos = reinterpret_cast<uint32_t *>(base + L.seq_pos);
  S.taken = reinterpret_cast<uint32_t *>(base + L.taken);
  S.lost = reinterpret_cast<uint32_t *>(base + L.lost);
  S.tbits = reinterpret_cast<uint32_t *>(base + L.tbits);
  S.blocker = reinterpret_cast<uint32_t *>(base + L.blocker);
  S.ctr = reinterpret_cast<RCounters *>(base + L.ctr);
  S.nl = uint32_t(a.num_leaves);
  const C *q0 = static_cast<const C *>(a.codes[0]), *q1 = static_cast<const C *>(a.codes[1]),
          *q2 = static_cast<const C *>(a.codes[2]);

  cudaError_t e = cudaMemsetAsync(S.live, 0xff, 4 * (a.n / 32 + 2), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(S.dest, 0xff, 4 * a.n, st);  // no owner yet: the final pass checks every slot got one
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(S.blocker, 0xff, 4 * a.num_leaves, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(base + L.zero_begin, 0, L.zero_end - L.zero_begin, st);
  if (e != cudaSuccess) return e;
  e = launch_leaftable(a.n, a.split_level, a.leaf_size, a.leafs, a.num_leaves, st);
  if (e != cudaSuccess) return e;

  const uint32_t sms = uint32_t(device_sm_count());
  const unsigned box_blocks = unsigned(a.num_leaves < 16ull * sms ? a.num_leaves : 16ull * sms);
  const unsigned take_blocks = unsigned(a.num_leaves < 2ull * sms ? a.num_leaves : 2ull * sms);
  const unsigned refit_blocks = unsigned((uint64_t(L.count[1]) + kWarps - 1) / kWarps);
  const unsigned select_blocks = unsigned((a.num_leaves + kWarps - 1) / kWarps);
  {
    TraceScope ts("k_rd_rebuild", st);
    k_rd_rebuild<C, true><<<box_blocks, kBoxThreads, 0, st>>>(S, q0, q1, q2, a.leafs);
  }
  {
    TraceScope ts("k_rd_refit", st);
    k_rd_refit<<<refit_blocks, kThreads, 0, st>>>(S);
  }
  // kRoundsPerCheck rounds: the same launches with the same arguments every time
  auto issue_rounds = [&](cudaStream_t s) {
    for (int k = 0; k < kRoundsPerCheck; ++k) {
      {
        TraceScope ts("k_rd_select", s);
        k_rd_select<<<select_blocks, kThreads, 0, s>>>(S);
      }
      {
        TraceScope ts("k_rd_take", s);
        k_rd_take<C><<<take_blocks, kTakeThreads, 0, s>>>(S, q0, q1, q2);
      }
      {
        TraceScope ts("k_rd_scan", s);
        k_rd_scan<<<1, 1024, 0, s>>>(S, a.seqs);
      }
      {
        TraceScope ts("k_rd_rebuild", s);
        k_rd_rebuild<C, false><<<box_blocks, kBoxThreads, 0, s>>>(S, q0, q1, q2, a.leafs);
      }
    }
  };
  // The rounds between two read-backs are captured once into a CUDA graph (on a
  // private stream of this call, so that any stream, the legacy one included,
  // can launch it) and launched once per read-back: one launch in place of
  // 4 * kRoundsPerCheck.  Kernel tracing needs events around every launch, so
  // with it on (or when the capture fails) the launches go one by one; so do
  // they for a caller that may not allocate (no graph is instantiated).
  RoundGraph graph;
  if (!trace_enabled() && !no_host_alloc()) graph.capture(issue_rounds);
  uint64_t issued = 0;
  for (;;) {
    if (graph.exec) {
      e = cudaGraphLaunch(graph.exec, st);
      if (e != cudaSuccess) return e;
    } else {
      issue_rounds(st);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    issued += kRoundsPerCheck;
    RCounters h;
    e = read_back(&h, S.ctr, sizeof(h), st);
    if (e != cudaSuccess) return e;
    if (h.alive == 0) {
      *num_seq = h.nseq;
      *rounds = h.rounds;
      break;
    }
    // every round takes at least the alive box of least key
    if (issued > a.num_leaves + kRoundsPerCheck) return cudaErrorUnknown;
  }
  {
    TraceScope ts("k_rd_gather", st);
    const uint64_t blocks = (a.n + 255) / 256;
    const unsigned grid = unsigned(blocks < 16ull * sms ? blocks : 16ull * sms);
    k_rd_gather<C><<<grid, 256, 0, st>>>(S, a.n, q0, q1, q2, static_cast<C *>(a.out_codes[0]),
                                        static_cast<C *>(a.out_codes[1]), static_cast<C *>(a.out_codes[2]), a.idx,
                                        a.out_idx, a.err);
  }
  return cudaGetLastError();
}

}  // namespace

uint64_t reduce_scratch_bytes(uint64_t n, uint64_t num_leaves) { return layout_of(n, num_leaves).total; }

cudaError_t launch_reduce(const ReduceLaunch &a, cudaStream_t st, uint64_t *num_seq, uint64_t *rounds) {
  *num_seq = 0;
  *rounds = 0;
  if (a.n == 0 || a.num_leaves == 0) return cudaSuccess;
  if (a.code_bytes == 2) return reduce_dispatch<uint16_t>(a, st, num_seq, rounds);
  return reduce_dispatch<uint32_t>(a, st, num_seq, rounds);
}

}  // namespace pcx
