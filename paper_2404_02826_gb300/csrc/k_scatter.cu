// Stable two-way partition of every node of one k-d level (Sec. 4.1 of
// arXiv 2404.02826): particles with code < v, then the first `tleft`
// particles with code == v (in index order) go to the left child, the rest to
// the right child, both keeping their order.  A node that is already a leaf
// has v above every code and is copied unchanged.
//
// Three kernels per level:
//   k_count     per tile, in groups of 32 consecutive window slots: the bit
//               masks of "code < v" and "code == v" of every group, their
//               prefix counts within the tile, and the tile's totals;
//   k_tilescan  per node: exclusive scan of its tiles' totals;
//   k_scatter   persistent CTAs; while one tile is partitioned, the Tensor
//               Memory Accelerator copies the next tile's codes into the other
//               half of a shared-memory double buffer (cp.async.bulk completing
//               on an mbarrier), with the tile's group records.  Consecutive
//               lanes take consecutive particles, a warp one group; each
//               particle's place in its child follows from the group's prefix
//               and the popcount of the group's masks below its lane.  Stores
//               to each child are contiguous across a warp.
#include <cstdint>

#include "pc_internal.cuh"
#include "pc_mbar.cuh"

namespace pcx {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;

template <typename C, bool IDX>
struct Cfg {
  static constexpr int kBytesPer = 3 * int(sizeof(C)) + (IDX ? 4 : 0);
  static constexpr int kWin = kBytesPer <= 6 ? 8192 : 4096;  // window of particles held per buffer
  static constexpr int kTile = kWin - 16;                      // largest tile: an aligned window covers it
  static constexpr int kRounds = kWin / kThreads;              // window slots per thread
  static constexpr int kGroups = kWin / 32;                    // 32-slot groups of a window
};

// Group record: masks of "code < v" and "code == v" over 32 window slots, and
// (less << 16 | tie) of the tile's groups before it.
using GroupRec = uint4;

// Tile i of node j covers positions [i*ts, (i+1)*ts) of the node, clipped to
// its size, with ts = ceil(cnt / T).  Everything fits 32 bits (n < 2^31), and
// the host picks T so that ts never exceeds the largest tile.  Computed once
// per tile by one thread: 64-bit division would run on the FP64 pipe.
struct TileGeom {
  uint32_t j, off, cnt, tb, te;
};

template <typename C, bool IDX>
struct Smem {
  using F = Cfg<C, IDX>;
  C in[2][3][F::kWin];
  uint32_t idx[IDX ? 2 : 1][IDX ? F::kWin : 4];
  GroupRec grp[2][F::kGroups];
  unsigned long long bar[2];
  unsigned long long pre[2];  // (less << 31 | tie) of the node's tiles before this one
  uint32_t tile[2];
  uint32_t tleft[2];
  TileGeom geo[2];
};

__device__ __forceinline__ TileGeom tile_geom(const LevelLaunch &a, uint32_t t) {
  TileGeom g;
  const uint32_t T = a.tiles_per_node;
  g.j = t / T;
  const uint32_t i = t - g.j * T;
  uint64_t off, cnt;
  node_range(a.n, a.level, g.j, off, cnt);
  g.off = uint32_t(off);
  g.cnt = uint32_t(cnt);
  const uint32_t ts = (g.cnt + T - 1) / T;
  g.tb = g.off + min(i * ts, g.cnt);
  g.te = g.off + min(i * ts + ts, g.cnt);
  return g;
}

// What thread 0 reads for a tile it has just issued; the loads complete while
// the current tile is processed and are used at its end.
struct Pending {
  uint32_t tl;
  unsigned long long pre;
};

// Thread 0: copies the window of tile t into buffer b and starts the loads of
// its node and its prefix counts.
template <typename C, bool IDX>
__device__ __forceinline__ void issue_tile(const LevelLaunch &a, Smem<C, IDX> &S, uint32_t t, int b, Pending &p) {
  const TileGeom g = tile_geom(a, t);
  S.geo[b] = g;
  const uint32_t w0 = g.tb & ~15u;
  const uint32_t nwin = (g.te - w0 + 15) & ~15u;
  const uint32_t bytes = nwin * uint32_t(sizeof(C));
  const uint32_t ngrp = (g.te - w0 + 31) >> 5;
  if (!a.drop_copies) {
    mbar_expect_tx(&S.bar[b], 3 * bytes + (IDX ? 4 * nwin : 0) + ngrp * uint32_t(sizeof(GroupRec)));
  }
  if (nwin && !a.drop_copies) {
    for (int d = 0; d < 3; ++d) bulk_g2s(S.in[b][d], static_cast<const C *>(a.src[d]) + w0, bytes, &S.bar[b]);
    if (IDX) bulk_g2s(S.idx[b], a.src_idx + w0, 4 * nwin, &S.bar[b]);
    bulk_g2s(S.grp[b], static_cast<const GroupRec *>(a.groups) + uint64_t(t) * Cfg<C, IDX>::kGroups,
             ngrp * uint32_t(sizeof(GroupRec)), &S.bar[b]);
  }
  p.tl = a.nodes[g.j].tleft;
  p.pre = a.tile_state[t];
}

template <typename C, bool IDX>
__device__ __forceinline__ void publish(Smem<C, IDX> &S, int b, const Pending &p) {
  S.tleft[b] = p.tl;
  S.pre[b] = p.pre;
}

// Persistent CTA.  Thread 0 keeps one ticket and one tile copy ahead of the
// tile being partitioned, so neither the ticket atomic nor the copy is waited
// for; three block barriers per tile.  AXIS is the split axis of the level.
// When the wait for a tile's copy gives up, the block lets the copy of the
// next tile land (bounded) and leaves the loop: it issues no further copy and
// takes no further ticket, so one stuck copy costs one bounded wait per block.
template <typename C, bool IDX, int AXIS>
__global__ void __launch_bounds__(kThreads, 2) k_scatter(LevelLaunch a, uint32_t tiles) {
  extern __shared__ __align__(128) unsigned char smraw[];
  Smem<C, IDX> &S = *reinterpret_cast<Smem<C, IDX> *>(smraw);
  if (call_failed(a.err)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Pending pend = {};
  uint32_t next_t = tiles;  // thread 0: the tile after the one in flight
  if (threadIdx.x == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    mbar_fence_init();
    const uint32_t t0 = atomicAdd(a.ticket, 1u);
    S.tile[0] = t0;
    if (t0 < tiles) {
      issue_tile(a, S, t0, 0, pend);
      publish(S, 0, pend);
      next_t = atomicAdd(a.ticket, 1u);
    }
  }
  __syncthreads();
  uint32_t phase0 = 0u, phase1 = 0u;  // parity of the next completion of each buffer's barrier
  int b = 0;
  C *d0 = static_cast<C *>(a.dst[0]);
  C *d1 = static_cast<C *>(a.dst[1]);
  C *d2 = static_cast<C *>(a.dst[2]);
  const uint32_t lt_mask = (1u << lane) - 1u, lane_bit = 1u << lane;
  for (;;) {
    const uint32_t t = S.tile[b];
    if (t >= tiles) break;
    bool prefetched = false;
    uint32_t after = tiles;
    if (threadIdx.x == 0) {
      S.tile[b ^ 1] = next_t;
      if (next_t < tiles) {
        fence_proxy_async();  // earlier generic reads of that buffer precede the async writes
        issue_tile(a, S, next_t, b ^ 1, pend);
        prefetched = true;
        after = atomicAdd(a.ticket, 1u);
      }
    }
    const bool late = wait_buffer(&S.bar[b], b ? phase1 : phase0, a.err, a.wait_limit);
    if (b) phase1 ^= 1u;
    else phase0 ^= 1u;

    const TileGeom g = S.geo[b];
    const uint32_t k = g.cnt >> 1;
    const uint32_t lead = g.tb & 15u;
    const uint32_t nslots = lead + (g.te - g.tb);
    const uint32_t tl = S.tleft[b];
    C *n0 = d0 + g.off, *n1 = d1 + g.off, *n2 = d2 + g.off;
    uint32_t *ni = IDX ? a.dst_idx + g.off : nullptr;
    const C *x0s = S.in[b][0], *x1s = S.in[b][1], *x2s = S.in[b][2];

    // Window slot wp = r * kThreads + threadIdx.x in round r: warp w covers
    // group r * kWarps + w.  Slots outside [lead, nslots) are not particles of
    // the tile; only the first and the last round have any.
    const uint32_t rounds = (nslots + kThreads - 1) / kThreads;
    const unsigned long long pre = S.pre[b];
    const uint32_t less_before = uint32_t(pre >> 31), tie_before = uint32_t(pre & 0x7fffffffu);
    const uint32_t cnt = g.cnt;
    const uint32_t kpos = k + (g.tb - g.off) - lead;  // k + node position of window slot 0
    for (uint32_t r = 0; r < rounds; ++r) {
      const uint32_t wp = r * kThreads + threadIdx.x;
      const GroupRec gr = S.grp[b][r * kWarps + warp];
      const uint32_t lb = less_before + (gr.z >> 16), tb = tie_before + (gr.z & 0xffffu);
      bool left;
      uint32_t glrank;  // left-going particles of the node before this one
      if (gr.y == 0) {  // no particle of the group has code v
        left = (gr.x & lane_bit) != 0;
        glrank = lb + min(tb, tl) + __popc(gr.x & lt_mask);
      } else {
        const uint32_t run_t = tb + __popc(gr.y & lt_mask);
        left = (gr.x & lane_bit) || ((gr.y & lane_bit) && run_t < tl);
        glrank = lb + __popc(gr.x & lt_mask) + min(run_t, tl);
      }
      const bool valid = (r > 0 && r + 1 < rounds) || (wp >= lead && wp < nslots);
      if (valid) {
        const uint32_t dst = left ? glrank : kpos + wp - glrank;
        const C x0 = x0s[wp], x1 = x1s[wp], x2 = x2s[wp];
        if (dst < cnt) {
          __stcg(n0 + dst, x0);
          __stcg(n1 + dst, x1);
          __stcg(n2 + dst, x2);
          if (IDX) __stcg(ni + dst, S.idx[b][wp]);
        } else {
          atomicOr(a.err, kErrInternal);
        }
      }
    }
    if (threadIdx.x == 0) {
      if (prefetched) publish(S, b ^ 1, pend);
      next_t = after;
    }
    // the next tile's state is published; this tile's buffer may be refilled.
    // A wait that gave up (the stores above then wrote only inside this node,
    // from data never copied; the call fails) ends the block's work here.
    if (__syncthreads_or(late)) {
      if (threadIdx.x == 0 && prefetched) drain_buffer(&S.bar[b ^ 1], b ? phase0 : phase1, a.wait_limit);
      break;
    }
    b ^= 1;
  }
}

// Per tile (one block of 8 warps): for every 32-slot group of the tile's
// window, the masks of "code < v" and "code == v" and the counts of the
// groups before it; the tile's totals go to tile_state for the node scan.
// Warp w takes a contiguous run of kGroups / 8 groups.  A lane loads 16 bytes
// (kPerLane codes) at a time and classifies them; the lanes sharing a group
// OR their bits together with xor-shuffles.
template <typename C, bool IDX>
__global__ void __launch_bounds__(256) k_count(LevelLaunch a) {
  constexpr int kG = Cfg<C, IDX>::kGroups;
  constexpr int kPerWarp = kG / 8;                    // groups of one warp
  constexpr int kPerLane = 16 / int(sizeof(C));       // codes of one 16-byte load
  constexpr int kLanesPerGroup = 32 / kPerLane;       // 4 (u16) or 8 (u32)
  constexpr int kGroupsPerLoad = 32 / kLanesPerGroup;  // groups one warp-wide load covers
  constexpr int kLoads = kPerWarp / kGroupsPerLoad;
  static_assert(kPerWarp <= 32 && kLoads * kGroupsPerLoad == kPerWarp, "group layout");
  __shared__ uint32_t wtot[8];
  __shared__ TileGeom sg;
  __shared__ uint32_t sv, sax;
  if (call_failed(a.err)) return;
  if (threadIdx.x == 0) {
    sg = tile_geom(a, blockIdx.x);
    sv = a.nodes[sg.j].v;
    sax = a.nodes[sg.j].axis;
  }
  __syncthreads();
  const TileGeom g = sg;
  const uint32_t v = sv;
  const uint32_t vc = v < 0x7fffffffu ? v : 0x7fffffffu, vc1 = vc + 1u;  // a leaf's v: above every code
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const C *q = static_cast<const C *>(a.src[sax]);
  const uint32_t w0 = g.tb & ~15u;
  const uint32_t ngrp = (g.te - w0 + 31) >> 5;
  const uint32_t run0 = w0 + uint32_t(warp) * (32u * kPerWarp);  // first slot of this warp's run
  // all of the lane's loads first
  uint4 raw[kLoads];
#pragma unroll
  for (int i = 0; i < kLoads; ++i) {
    const uint32_t s0 = run0 + uint32_t(i) * (32u * kGroupsPerLoad) + uint32_t(lane) * kPerLane;
    raw[i] = s0 < g.te ? __ldcs(reinterpret_cast<const uint4 *>(q + s0)) : make_uint4(0u, 0u, 0u, 0u);
  }
  uint32_t mylm = 0, mytm = 0, mycnt = 0;  // lane i: group warp * kPerWarp + i
#pragma unroll
  for (int i = 0; i < kLoads; ++i) {
    const uint32_t s0 = run0 + uint32_t(i) * (32u * kGroupsPerLoad) + uint32_t(lane) * kPerLane;
    // valid slots of this lane's codes: [tb, te) relative to s0
    const int vlo = min(max(int(g.tb) - int(s0), 0), kPerLane), vhi = min(max(int(g.te) - int(s0), 0), kPerLane);
    const uint32_t vm = ((1u << vhi) - 1u) & ~((1u << vlo) - 1u);
    const uint32_t w[4] = {raw[i].x, raw[i].y, raw[i].z, raw[i].w};
    // Codes are below 2^30 and vc, vc + 1 at most 2^31, so the sign bit of
    // x - vc is x < vc and that of x - (vc + 1) is x <= vc; each bit is
    // shifted into its mask (code c at bit c), and the ties are le & ~lt.
    uint32_t l = 0, le = 0;
#pragma unroll
    for (int c = kPerLane - 1; c >= 0; --c) {
      const uint32_t x = sizeof(C) == 2 ? ((w[c >> 1] >> (16 * (c & 1))) & 0xffffu) : w[c];
      l = __funnelshift_l(x - vc, l, 1);
      le = __funnelshift_l(x - vc1, le, 1);
    }
    uint32_t t = le & ~l;
    const int sh = kPerLane * (lane % kLanesPerGroup);
    l = (l & vm) << sh;
    t = (t & vm) << sh;
#pragma unroll
    for (int o = 1; o < kLanesPerGroup; o <<= 1) {
      l |= __shfl_xor_sync(0xffffffffu, l, o);
      t |= __shfl_xor_sync(0xffffffffu, t, o);
    }
    // group i * kGroupsPerLoad + j sits in lanes j * kLanesPerGroup ...; hand it to lane i * kGroupsPerLoad + j
    const int src = (lane % kGroupsPerLoad) * kLanesPerGroup;
    const uint32_t gl = __shfl_sync(0xffffffffu, l, src), gt = __shfl_sync(0xffffffffu, t, src);
    if (lane / kGroupsPerLoad == i) {
      mylm = gl;
      mytm = gt;
      mycnt = (uint32_t(__popc(gl)) << 16) | uint32_t(__popc(gt));
    }
  }
  // prefix of the groups: within the warp, then across warps
  uint32_t incl = mycnt;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  uint32_t wbase = 0, total = 0;
  for (int w = 0; w < 8; ++w) {
    const uint32_t x = wtot[w];
    wbase += w < warp ? x : 0u;
    total += x;
  }
  const uint32_t m = uint32_t(warp * kPerWarp + lane);
  if (lane < kPerWarp && m < ngrp) {
    GroupRec *out = static_cast<GroupRec *>(a.groups) + uint64_t(blockIdx.x) * kG;
    out[m] = make_uint4(mylm, mytm, wbase + incl - mycnt, 0u);
  }
  if (threadIdx.x == 0) a.tile_state[blockIdx.x] = ((unsigned long long)(total >> 16) << 31) | (total & 0xffffu);
}

// Per node: exclusive scan of its tiles' (less << 31 | tie) counts, in place.
__global__ void __launch_bounds__(1024) k_tilescan(LevelLaunch a) {
  __shared__ unsigned long long wt[33];
  if (call_failed(a.err)) return;
  const uint64_t T = a.tiles_per_node;
  unsigned long long *s = a.tile_state + blockIdx.x * T;
  const uint64_t per = (T + blockDim.x - 1) / blockDim.x;
  const uint64_t t0 = threadIdx.x * per, t1 = (t0 + per) < T ? (t0 + per) : T;
  unsigned long long sum = 0;
  for (uint64_t t = t0; t < t1; ++t) sum += s[t];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long incl = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wt[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long x = wt[lane];
    unsigned long long xi = x;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += y;
    }
    wt[lane] = xi - x;
  }
  __syncthreads();
  unsigned long long run = wt[warp] + incl - sum;
  for (uint64_t t = t0; t < t1; ++t) {
    const unsigned long long x = s[t];
    s[t] = run;
    run += x;
  }
}

// The same scan for nodes of few tiles: one thread per node.
__global__ void k_tilescan_small(LevelLaunch a) {
  if (call_failed(a.err)) return;
  const uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= (1ull << a.level)) return;
  const uint32_t T = a.tiles_per_node;
  unsigned long long *s = a.tile_state + j * T;
  unsigned long long run = 0;
  for (uint32_t t = 0; t < T; ++t) {
    const unsigned long long x = s[t];
    s[t] = run;
    run += x;
  }
}

// Levels of small nodes (at most a.warp_node_max particles): one warp partitions a
// whole node in one pass, 32 consecutive particles per round, carrying the
// counts of "code < v" and "code == v" from round to round - no tiles, no
// count pass, no tile scan.  Same placement rule as k_scatter.  AXIS is the
// level's split axis, or 3 for each node's own (widest-cell variant).
template <typename C, bool IDX, int AXIS>
__global__ void __launch_bounds__(256) k_scatter_node(LevelLaunch a) {
  if (call_failed(a.err)) return;
  const int lane = threadIdx.x & 31;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint64_t count = 1ull << a.level;
  const uint64_t warps = uint64_t(gridDim.x) * (blockDim.x >> 5);
  const C *s0 = static_cast<const C *>(a.src[0]), *s1 = static_cast<const C *>(a.src[1]),
          *s2 = static_cast<const C *>(a.src[2]);
  for (uint64_t j = uint64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); j < count; j += warps) {
    uint64_t off64, cnt64;
    node_range(a.n, a.level, j, off64, cnt64);
    const uint32_t off = uint32_t(off64), cnt = uint32_t(cnt64), k = cnt >> 1;
    const uint32_t v = a.nodes[j].v, tl = a.nodes[j].tleft, ax = AXIS == 3 ? a.nodes[j].axis : uint32_t(AXIS);
    C *n0 = static_cast<C *>(a.dst[0]) + off, *n1 = static_cast<C *>(a.dst[1]) + off,
      *n2 = static_cast<C *>(a.dst[2]) + off;
    uint32_t *ni = IDX ? a.dst_idx + off : nullptr;
    uint32_t run_l = 0, run_t = 0;  // particles below v and equal to v before this round
    // each round's codes are loaded one round ahead, so their latency overlaps the current round
    C p0 = 0, p1 = 0, p2 = 0;
    uint32_t pxi = 0;
    if (lane < cnt) {
      p0 = s0[off + lane];
      p1 = s1[off + lane];
      p2 = s2[off + lane];
      if (IDX) pxi = a.src_idx[off + lane];
    }
    for (uint32_t base = 0; base < cnt; base += 32) {
      const uint32_t i = base + lane;
      const bool valid = i < cnt;
      const C x0 = p0, x1 = p1, x2 = p2;
      const uint32_t xi = pxi;
      if (i + 32 < cnt) {
        p0 = s0[off + i + 32];
        p1 = s1[off + i + 32];
        p2 = s2[off + i + 32];
        if (IDX) pxi = a.src_idx[off + i + 32];
      }
      const uint32_t q = ax == 0 ? x0 : (ax == 1 ? x1 : x2);
      const bool isless = valid && q < v, istie = valid && q == v;
      const uint32_t lm = __ballot_sync(0xffffffffu, isless), tm = __ballot_sync(0xffffffffu, istie);
      const uint32_t tie_rank = run_t + __popc(tm & lt_mask);
      const bool left = isless || (istie && tie_rank < tl);
      const uint32_t glrank = run_l + __popc(lm & lt_mask) + min(tie_rank, tl);  // left-going before this one
      if (valid) {
        const uint32_t dst = left ? glrank : k + (i - glrank);
        if (dst < cnt) {
          __stcg(n0 + dst, x0);
          __stcg(n1 + dst, x1);
          __stcg(n2 + dst, x2);
          if (IDX) __stcg(ni + dst, xi);
        } else {
          atomicOr(a.err, kErrInternal);
        }
      }
      run_l += __popc(lm);
      run_t += __popc(tm);
    }
  }
}

template <typename C, bool IDX, int AXIS>
cudaError_t scatter_launch(const LevelLaunch &a, uint32_t tiles, cudaStream_t st) {
  const size_t smem = sizeof(Smem<C, IDX>);
  int per_sm = 0;
  cudaError_t e = resident_blocks<k_scatter<C, IDX, AXIS>>(kThreads, smem, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  uint64_t grid = uint64_t(per_sm) * uint64_t(device_sm_count());
  if (grid > tiles) grid = tiles;
  TraceScope ts("k_scatter", st);
  k_scatter<C, IDX, AXIS><<<unsigned(grid), kThreads, smem, st>>>(a, tiles);
  return cudaGetLastError();
}

template <typename C, bool IDX, int AXIS>
cudaError_t scatter_node_launch(const LevelLaunch &a, cudaStream_t st) {
  const uint64_t nodes = 1ull << a.level;
  uint64_t grid = (nodes + 7) / 8;  // 8 warps per block, a warp per node
  const uint64_t cap = uint64_t(device_sm_count()) * 8 * 4;
  if (grid > cap) grid = cap;
  TraceScope ts("k_scatter_node", st);
  k_scatter_node<C, IDX, AXIS><<<unsigned(grid), 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename C, bool IDX>
cudaError_t scatter_dispatch(const LevelLaunch &a, cudaStream_t st) {
  if (((a.n + (1ull << a.level) - 1) >> a.level) <= a.warp_node_max) {
    if (a.widest) return scatter_node_launch<C, IDX, 3>(a, st);
    switch (a.level % 3) {
      case 0: return scatter_node_launch<C, IDX, 0>(a, st);
      case 1: return scatter_node_launch<C, IDX, 1>(a, st);
      default: return scatter_node_launch<C, IDX, 2>(a, st);
    }
  }
  const uint64_t tiles = (1ull << a.level) * a.tiles_per_node;
  {
    TraceScope ts("k_count", st);
    k_count<C, IDX><<<unsigned(tiles), 256, 0, st>>>(a);
  }
  {
    TraceScope ts("k_tilescan", st);
    if (a.tiles_per_node <= 16)
      k_tilescan_small<<<unsigned(((1ull << a.level) + 255) / 256), 256, 0, st>>>(a);
    else
      k_tilescan<<<unsigned(1ull << a.level), 1024, 0, st>>>(a);
  }
  switch (a.level % 3) {
    case 0: return scatter_launch<C, IDX, 0>(a, uint32_t(tiles), st);
    case 1: return scatter_launch<C, IDX, 1>(a, uint32_t(tiles), st);
    default: return scatter_launch<C, IDX, 2>(a, uint32_t(tiles), st);
  }
}

}  // namespace

uint32_t scatter_groups(int code_bytes, bool with_idx) {
  if (code_bytes == 2) return with_idx ? Cfg<uint16_t, true>::kGroups : Cfg<uint16_t, false>::kGroups;
  return with_idx ? Cfg<uint32_t, true>::kGroups : Cfg<uint32_t, false>::kGroups;
}

uint32_t scatter_tile(int code_bytes, bool with_idx) {
  if (code_bytes == 2) return with_idx ? Cfg<uint16_t, true>::kTile : Cfg<uint16_t, false>::kTile;
  return with_idx ? Cfg<uint32_t, true>::kTile : Cfg<uint32_t, false>::kTile;
}

cudaError_t launch_scatter(const LevelLaunch &a, cudaStream_t st) {
  if (a.code_bytes == 2)
    return a.with_idx ? scatter_dispatch<uint16_t, true>(a, st) : scatter_dispatch<uint16_t, false>(a, st);
  return a.with_idx ? scatter_dispatch<uint32_t, true>(a, st) : scatter_dispatch<uint32_t, false>(a, st);
}

}  // namespace pcx
