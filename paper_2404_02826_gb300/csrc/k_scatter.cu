// Stable two-way partition of every node of one k-d level (Sec. 4.1 of
// arXiv 2404.02826): particles with code < v, then the first `tleft`
// particles with code == v (in index order) go to the left child, the rest to
// the right child, both keeping their order.  A node that is already a leaf
// has v above every code and is copied unchanged.
//
// Three kernels per level:
//   k_count     per tile: how many particles have code < v and code == v;
//   k_tilescan  per node: exclusive scan of its tiles' counts;
//   k_scatter   persistent CTAs; while one tile is partitioned, the Tensor
//               Memory Accelerator copies the next tile's codes into the other
//               half of a shared-memory double buffer (cp.async.bulk completing
//               on an mbarrier).  Per tile: consecutive lanes take consecutive
//               particles; two warp ballots give the masks of "code < v" and
//               "code == v" of 32 particles, one block scan turns the counts of
//               every (round, warp) into prefixes, and each particle's place in
//               its child follows from its prefix and the popcount of the
//               masks below its lane.  Stores to each child are contiguous
//               across a warp.
#include <cstdint>

#include "pc_internal.cuh"

namespace pcx {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kBarSpinLimit = 1u << 22;

template <typename C, bool IDX>
struct Cfg {
  static constexpr int kBytesPer = 3 * int(sizeof(C)) + (IDX ? 4 : 0);
  static constexpr int kWin = kBytesPer <= 6 ? 8192 : 4096;  // window of particles held per buffer
  static constexpr int kTile = kWin - 16;                      // largest tile: an aligned window covers it
  static constexpr int kRounds = kWin / kThreads;              // window slots per thread
};

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
  alignas(16) uint32_t wc[F::kRounds * kWarps];  // (less << 16 | tie) per round and warp
  uint2 msk[F::kRounds * kWarps];                // ("code < v", "code == v") ballots per round and warp
  uint2 pref[F::kRounds * kWarps];               // (left-going, ties) in the node before each round and warp
  unsigned long long bar[2];
  unsigned long long pre[2];  // (less << 31 | tie) of the node's tiles before this one
  uint32_t tile[2];
  uint32_t v[2], tleft[2];
  TileGeom geo[2];
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for the copy into one buffer; bounded: on expiry the error bit is set
// and the wait is repeated once more (the copy itself always completes).
__device__ __forceinline__ void wait_buffer(unsigned long long *bar, uint32_t parity, uint32_t *err) {
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++spins > kBarSpinLimit) {
      if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
      spins = 0;
      while (!mbar_try_wait(bar, parity) && ++spins < kBarSpinLimit) {
      }
      return;
    }
  }
}

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
  uint32_t v, tl;
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
  mbar_expect_tx(&S.bar[b], 3 * bytes + (IDX ? 4 * nwin : 0));
  if (nwin) {
    for (int d = 0; d < 3; ++d) bulk_g2s(S.in[b][d], static_cast<const C *>(a.src[d]) + w0, bytes, &S.bar[b]);
    if (IDX) bulk_g2s(S.idx[b], a.src_idx + w0, 4 * nwin, &S.bar[b]);
  }
  p.v = a.nodes[g.j].v;
  p.tl = a.nodes[g.j].tleft;
  p.pre = a.tile_state[t];
}

template <typename C, bool IDX>
__device__ __forceinline__ void publish(Smem<C, IDX> &S, int b, const Pending &p) {
  S.v[b] = p.v;
  S.tleft[b] = p.tl;
  S.pre[b] = p.pre;
}

// Persistent CTA.  Thread 0 keeps one ticket and one tile copy ahead of the
// tile being partitioned, so neither the ticket atomic nor the copy is waited
// for; three block barriers per tile.  AXIS is the split axis of the level.
template <typename C, bool IDX, int AXIS>
__global__ void __launch_bounds__(kThreads, 2) k_scatter(LevelLaunch a, uint32_t tiles) {
  using F = Cfg<C, IDX>;
  constexpr int kPer = F::kRounds * kWarps / 32;  // scan entries per lane of warp 0
  static_assert(kPer == 4 || kPer == 8, "scan entries per lane");
  extern __shared__ __align__(128) unsigned char smraw[];
  Smem<C, IDX> &S = *reinterpret_cast<Smem<C, IDX> *>(smraw);
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
    wait_buffer(&S.bar[b], b ? phase1 : phase0, a.err);
    if (b) phase1 ^= 1u;
    else phase0 ^= 1u;

    const TileGeom g = S.geo[b];
    const uint32_t k = g.cnt >> 1;
    const uint32_t lead = g.tb & 15u;
    const uint32_t nslots = lead + (g.te - g.tb);
    const uint32_t v = S.v[b], tl = S.tleft[b];
    C *n0 = d0 + g.off, *n1 = d1 + g.off, *n2 = d2 + g.off;
    uint32_t *ni = IDX ? a.dst_idx + g.off : nullptr;
    const C *x0s = S.in[b][0], *x1s = S.in[b][1], *x2s = S.in[b][2];
    const C *qa = AXIS == 0 ? x0s : (AXIS == 1 ? x1s : x2s);

    // Window slot wp = r * kThreads + threadIdx.x in round r: a warp covers 32
    // consecutive slots, so two ballots give the "code < v" and "code == v"
    // masks of those 32 particles.  Slots outside [lead, nslots) are not
    // particles of the tile; only the first and the last round have any.
    const uint32_t rounds = (nslots + kThreads - 1) / kThreads;
    // 1. masks and counts per round and warp
    for (uint32_t r = 0; r < rounds; ++r) {
      const uint32_t wp = r * kThreads + threadIdx.x;
      const uint32_t q = qa[wp];
      const bool valid = wp >= lead && wp < nslots;
      const uint32_t lm = __ballot_sync(0xffffffffu, valid && q < v);
      const uint32_t tm = __ballot_sync(0xffffffffu, valid && q == v);
      if (lane == 0) {
        S.wc[r * kWarps + warp] = (uint32_t(__popc(lm)) << 16) | uint32_t(__popc(tm));
        S.msk[r * kWarps + warp] = make_uint2(lm, tm);
      }
    }
    __syncthreads();
    // 2. warp 0: exclusive scan of the counts, kPer entries per lane, turned
    //    into (left-going particles, ties) of the node before each entry
    if (warp == 0) {
      const unsigned long long pre = S.pre[b];
      const uint32_t less_before = uint32_t(pre >> 31), tie_before = uint32_t(pre & 0x7fffffffu);
      const uint32_t ne = rounds * kWarps;
      uint32_t e[kPer];
      const uint4 *w4 = reinterpret_cast<const uint4 *>(S.wc + kPer * lane);
#pragma unroll
      for (int h = 0; h < kPer / 4; ++h) {
        const uint4 x = w4[h];
        e[4 * h] = x.x;
        e[4 * h + 1] = x.y;
        e[4 * h + 2] = x.z;
        e[4 * h + 3] = x.w;
      }
      uint32_t sum = 0;
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const uint32_t x = (kPer * uint32_t(lane) + i) < ne ? e[i] : 0u;
        e[i] = sum;
        sum += x;
      }
      uint32_t incl = sum;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t base = incl - sum;
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const uint32_t ex = base + e[i];
        const uint32_t lb = less_before + (ex >> 16), tb = tie_before + (ex & 0xffffu);
        S.pref[kPer * lane + i] = make_uint2(lb + min(tb, tl), tb);
      }
    }
    __syncthreads();
    // 3. every particle's place in the node; stores with consecutive lanes on
    //    consecutive particles, so each child's run is contiguous across a warp
    const uint32_t cnt = g.cnt;
    const uint32_t kpos = k + (g.tb - g.off) - lead;  // k + node position of window slot 0
    for (uint32_t r = 0; r < rounds; ++r) {
      const uint32_t wp = r * kThreads + threadIdx.x;
      const uint2 mk = S.msk[r * kWarps + warp];
      const uint2 pf = S.pref[r * kWarps + warp];
      bool left;
      uint32_t glrank;  // left-going particles of the node before this one
      if (mk.y == 0) {  // no particle of this warp's 32 has code v
        left = (mk.x & lane_bit) != 0;
        glrank = pf.x + __popc(mk.x & lt_mask);
      } else {
        const uint32_t run_t = pf.y + __popc(mk.y & lt_mask);
        const uint32_t run_l = pf.x - min(pf.y, tl) + __popc(mk.x & lt_mask);
        left = (mk.x & lane_bit) || ((mk.y & lane_bit) && run_t < tl);
        glrank = run_l + min(run_t, tl);
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
    __syncthreads();  // the next tile's state is published; this tile's buffer may be refilled
    b ^= 1;
  }
}

// Per tile: how many particles have code < v and code == v (one block per tile).
template <typename C>
__global__ void __launch_bounds__(256) k_count(LevelLaunch a) {
  __shared__ uint32_t red[2][8];
  __shared__ TileGeom sg;
  __shared__ uint32_t sv;
  if (threadIdx.x == 0) {
    sg = tile_geom(a, blockIdx.x);
    sv = a.nodes[sg.j].v;
  }
  __syncthreads();
  const TileGeom g = sg;
  const uint32_t v = sv;
  const C *q = static_cast<const C *>(a.src[a.level % 3]);
  constexpr uint32_t kVec = 16 / sizeof(C);
  uint32_t less = 0, tie = 0;
  auto one = [&](uint32_t x) {
    less += x < v;
    tie += x == v;
  };
  const uint32_t a0 = (g.tb + kVec - 1) & ~(kVec - 1), a1 = g.te & ~(kVec - 1);
  if (a0 >= a1) {
    for (uint32_t e = g.tb + threadIdx.x; e < g.te; e += blockDim.x) one(__ldcg(q + e));
  } else {
    for (uint32_t e = g.tb + threadIdx.x; e < a0; e += blockDim.x) one(__ldcg(q + e));
    for (uint32_t e = a1 + threadIdx.x; e < g.te; e += blockDim.x) one(__ldcg(q + e));
    const uint4 *vp = reinterpret_cast<const uint4 *>(q + a0);
    const uint32_t nv = (a1 - a0) / kVec;
    for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) {
      const uint4 w = __ldcg(vp + i);
      const uint32_t x[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (sizeof(C) == 2) {
          one(x[c] & 0xffffu);
          one(x[c] >> 16);
        } else {
          one(x[c]);
        }
      }
    }
  }
  less = __reduce_add_sync(0xffffffffu, less);
  tie = __reduce_add_sync(0xffffffffu, tie);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = less;
    red[1][threadIdx.x >> 5] = tie;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t l = 0, t = 0;
    for (int w = 0; w < 8; ++w) {
      l += red[0][w];
      t += red[1][w];
    }
    a.tile_state[blockIdx.x] = ((unsigned long long)l << 31) | t;
  }
}

// Per node: exclusive scan of its tiles' (less << 31 | tie) counts, in place.
__global__ void __launch_bounds__(1024) k_tilescan(LevelLaunch a) {
  __shared__ unsigned long long wt[33];
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

template <typename C, bool IDX, int AXIS>
cudaError_t scatter_launch(const LevelLaunch &a, uint32_t tiles, cudaStream_t st) {
  const size_t smem = sizeof(Smem<C, IDX>);
  cudaError_t e =
      cudaFuncSetAttribute(k_scatter<C, IDX, AXIS>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter<C, IDX, AXIS>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  uint64_t grid = uint64_t(per_sm) * uint64_t(device_sm_count());
  if (grid > tiles) grid = tiles;
  TraceScope ts("k_scatter", st);
  k_scatter<C, IDX, AXIS><<<unsigned(grid), kThreads, smem, st>>>(a, tiles);
  return cudaGetLastError();
}

template <typename C, bool IDX>
cudaError_t scatter_dispatch(const LevelLaunch &a, cudaStream_t st) {
  const uint64_t tiles = (1ull << a.level) * a.tiles_per_node;
  {
    TraceScope ts("k_count", st);
    k_count<C><<<unsigned(tiles), 256, 0, st>>>(a);
  }
  {
    TraceScope ts("k_tilescan", st);
    k_tilescan<<<unsigned(1ull << a.level), 1024, 0, st>>>(a);
  }
  switch (a.level % 3) {
    case 0: return scatter_launch<C, IDX, 0>(a, uint32_t(tiles), st);
    case 1: return scatter_launch<C, IDX, 1>(a, uint32_t(tiles), st);
    default: return scatter_launch<C, IDX, 2>(a, uint32_t(tiles), st);
  }
}

}  // namespace

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
