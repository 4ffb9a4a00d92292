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
//               on an mbarrier).  Per tile: one thread per 16 consecutive
//               particles forms bit masks of "code < v" and "code == v"; after
//               a block scan of their counts the same thread walks its group
//               and records each particle's place in the tile's left or right
//               run as a 16-bit index; then consecutive threads take
//               consecutive particles and store them, so stores to each run are
//               contiguous across a warp.  The children's code bounds on the
//               next axis are reduced per CTA and folded in with an atomic only
//               when they improve the stored bound.
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
  uint16_t dst[F::kWin];       // tile-local destination of each window slot (0xffff: none)
  uint32_t scan[33];
  uint32_t red[4][kWarps];
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

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *warp_tot, uint32_t &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = x;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t t = lane < kWarps ? warp_tot[lane] : 0;
    uint32_t ti = t;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < kWarps) warp_tot[lane] = ti - t;
    if (lane == 31) warp_tot[32] = ti;
  }
  __syncthreads();
  total = warp_tot[32];
  const uint32_t r = warp_tot[warp] + incl - x;
  __syncthreads();
  return r;
}

// 16 consecutive codes starting at a 16-aligned slot, read with 16-byte loads.
template <typename C>
struct Group16;
template <>
struct Group16<uint16_t> {
  uint32_t w[8];  // two codes per word, element 2i in the low half
  __device__ __forceinline__ void load(const uint16_t *p) {
    const uint4 a = reinterpret_cast<const uint4 *>(p)[0], b = reinterpret_cast<const uint4 *>(p)[1];
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
  }
  __device__ __forceinline__ uint32_t get(int j) const { return (j & 1) ? (w[j >> 1] >> 16) : (w[j >> 1] & 0xffffu); }
};
template <>
struct Group16<uint32_t> {
  uint32_t w[16];
  __device__ __forceinline__ void load(const uint32_t *p) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint4 a = reinterpret_cast<const uint4 *>(p)[i];
      w[4 * i] = a.x; w[4 * i + 1] = a.y; w[4 * i + 2] = a.z; w[4 * i + 3] = a.w;
    }
  }
  __device__ __forceinline__ uint32_t get(int j) const { return w[j]; }
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

// Thread 0: copies the window of tile t into buffer b and reads its node and
// its prefix counts (the loads complete while the current tile is processed).
template <typename C, bool IDX>
__device__ __forceinline__ void issue_tile(const LevelLaunch &a, Smem<C, IDX> &S, uint32_t t, int b, uint32_t &v,
                                           uint32_t &tl, unsigned long long &pre) {
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
  v = a.nodes[g.j].v;
  tl = a.nodes[g.j].tleft;
  pre = a.tile_state[t];
}

template <typename C, bool IDX>
__global__ void __launch_bounds__(kThreads) k_scatter(LevelLaunch a, uint32_t tiles) {
  extern __shared__ __align__(128) unsigned char smraw[];
  Smem<C, IDX> &S = *reinterpret_cast<Smem<C, IDX> *>(smraw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int axis = a.level % 3, nxt = (a.level + 1) % 3;
  uint32_t pend_v = 0, pend_tl = 0;
  unsigned long long pend_pre = 0;
  if (threadIdx.x == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    mbar_fence_init();
    const uint32_t t0 = atomicAdd(a.ticket, 1u);
    S.tile[0] = t0;
    if (t0 < tiles) {
      issue_tile(a, S, t0, 0, pend_v, pend_tl, pend_pre);
      S.v[0] = pend_v;
      S.tleft[0] = pend_tl;
      S.pre[0] = pend_pre;
    }
  }
  __syncthreads();
  uint32_t phase0 = 0u, phase1 = 0u;  // parity of the next completion of each buffer's barrier
  int b = 0;
  C *d0 = static_cast<C *>(a.dst[0]);
  C *d1 = static_cast<C *>(a.dst[1]);
  C *d2 = static_cast<C *>(a.dst[2]);
  for (;;) {
    const uint32_t t = S.tile[b];
    if (t >= tiles) break;
    bool prefetched = false;
    if (threadIdx.x == 0) {
      const uint32_t tn = atomicAdd(a.ticket, 1u);
      S.tile[b ^ 1] = tn;
      if (tn < tiles) {
        fence_proxy_async();  // earlier generic reads of that buffer precede the async writes
        issue_tile(a, S, tn, b ^ 1, pend_v, pend_tl, pend_pre);
        prefetched = true;
      }
    }
    wait_buffer(&S.bar[b], b ? phase1 : phase0, a.err);
    if (b) phase1 ^= 1u;
    else phase0 ^= 1u;

    const TileGeom g = S.geo[b];
    const uint32_t k = g.cnt >> 1;
    const uint32_t sz = g.te - g.tb;
    const uint32_t lead = g.tb & 15u;
    const uint32_t ngroups = (lead + sz + 15) >> 4;
    const uint32_t v = S.v[b], tl = S.tleft[b];
    const unsigned long long pre = S.pre[b];
    const uint32_t less_before = uint32_t(pre >> 31), tie_before = uint32_t(pre & 0x7fffffffu);
    const uint32_t node_pos0 = g.tb - g.off;  // position of the tile's first particle in the node
    C *n0 = d0 + g.off, *n1 = d1 + g.off, *n2 = d2 + g.off;
    uint32_t *ni = IDX ? a.dst_idx + g.off : nullptr;

    // 1. each thread classifies its 16-particle group (registers only)
    const bool mine = threadIdx.x < ngroups;
    const uint32_t base = threadIdx.x * 16;
    const C *qa = S.in[b][axis];
    const C *qn = S.in[b][nxt];
    uint32_t lm = 0, tm = 0, vm = 0;
    if (mine) {
      Group16<C> ga;  // 16-byte loads: scalar loads 16 particles apart would hit the same bank
      ga.load(qa + base);
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const uint32_t wp = base + jj;
        const uint32_t q = ga.get(jj);
        const bool valid = wp >= lead && wp < lead + sz;
        vm |= uint32_t(valid) << jj;
        lm |= uint32_t(valid && q < v) << jj;
        tm |= uint32_t(valid && q == v) << jj;
      }
    }
    uint32_t total;
    const uint32_t ex = block_excl_scan((uint32_t(__popc(lm)) << 16) | uint32_t(__popc(tm)), S.scan, total);
    // the tile's particles split into a left run [0, left_tile) and a right run [left_tile, sz)
    const uint32_t left_before = less_before + min(tie_before, tl);
    const uint32_t left_tile = less_before + (total >> 16) + min(tie_before + (total & 0xffffu), tl) - left_before;
    const uint32_t right_before = node_pos0 - left_before;
    // 2. tile-local destination of every particle of the group, and the children bounds
    uint32_t cmin0 = 0xffffffffu, cmax0 = 0, cmin1 = 0xffffffffu, cmax1 = 0;
    if (mine) {
      uint32_t run_l = less_before + (ex >> 16), run_t = tie_before + (ex & 0xffffu);
      uint32_t pk[8];
      Group16<C> gn;
      gn.load(qn + base);
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const bool valid = (vm >> jj) & 1u, isless = (lm >> jj) & 1u, istie = (tm >> jj) & 1u;
        const bool left = isless || (istie && run_t < tl);
        const uint32_t glrank = run_l + min(run_t, tl);
        const uint32_t pos = node_pos0 + (base + jj - lead);  // position in the node
        uint32_t d = left ? glrank - left_before : left_tile + (pos - glrank - right_before);
        d = valid ? d : 0xffffu;
        if (jj & 1) pk[jj >> 1] |= d << 16;
        else pk[jj >> 1] = d & 0xffffu;
        run_l += isless;
        run_t += istie;
        if (valid) {
          const uint32_t xn = gn.get(jj);
          if (left) {
            cmin0 = min(cmin0, xn);
            cmax0 = max(cmax0, xn);
          } else {
            cmin1 = min(cmin1, xn);
            cmax1 = max(cmax1, xn);
          }
        }
      }
      uint4 *dv = reinterpret_cast<uint4 *>(S.dst + base);
      dv[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      dv[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
    __syncthreads();  // destinations visible to every thread
    // 3. stores, consecutive threads on consecutive particles
    const uint32_t cnt = g.cnt;
    const uint32_t baseR = k + right_before - left_tile;  // node position = local + baseR in the right run
    for (uint32_t p = threadIdx.x; p < sz; p += kThreads) {
      const uint32_t wp = lead + p;
      const uint32_t dl = S.dst[wp];
      const uint32_t dst = dl + (dl < left_tile ? left_before : baseR);
      if (dl < sz && dst < cnt) {
        __stcg(n0 + dst, S.in[b][0][wp]);
        __stcg(n1 + dst, S.in[b][1][wp]);
        __stcg(n2 + dst, S.in[b][2][wp]);
        if (IDX) __stcg(ni + dst, S.idx[b][wp]);
      } else {
        atomicOr(a.err, kErrInternal);
      }
    }
    // 4. children bounds on the next axis
    if (a.children) {
      cmin0 = __reduce_min_sync(0xffffffffu, cmin0);
      cmax0 = __reduce_max_sync(0xffffffffu, cmax0);
      cmin1 = __reduce_min_sync(0xffffffffu, cmin1);
      cmax1 = __reduce_max_sync(0xffffffffu, cmax1);
      if (lane == 0) {
        S.red[0][warp] = cmin0;
        S.red[1][warp] = cmax0;
        S.red[2][warp] = cmin1;
        S.red[3][warp] = cmax1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (a.children) {
        uint32_t m0 = S.red[0][0], x0 = S.red[1][0], m1 = S.red[2][0], x1 = S.red[3][0];
        for (int w = 1; w < kWarps; ++w) {
          m0 = min(m0, S.red[0][w]);
          x0 = max(x0, S.red[1][w]);
          m1 = min(m1, S.red[2][w]);
          x1 = max(x1, S.red[3][w]);
        }
        LevelNode *c0 = a.children + 2 * g.j, *c1 = c0 + 1;
        if (m0 <= x0) {
          if (m0 < ld_relaxed(&c0->lo)) atomicMin(&c0->lo, m0);
          if (x0 > ld_relaxed(&c0->hi)) atomicMax(&c0->hi, x0);
        }
        if (m1 <= x1) {
          if (m1 < ld_relaxed(&c1->lo)) atomicMin(&c1->lo, m1);
          if (x1 > ld_relaxed(&c1->hi)) atomicMax(&c1->hi, x1);
        }
      }
      if (prefetched) {
        S.v[b ^ 1] = pend_v;
        S.tleft[b ^ 1] = pend_tl;
        S.pre[b ^ 1] = pend_pre;
      }
    }
    __syncthreads();
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
  const size_t smem = sizeof(Smem<C, IDX>);
  cudaError_t e = cudaFuncSetAttribute(k_scatter<C, IDX>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter<C, IDX>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  uint64_t grid = uint64_t(per_sm) * uint64_t(device_sm_count());
  if (grid > tiles) grid = tiles;
  TraceScope ts("k_scatter", st);
  k_scatter<C, IDX><<<unsigned(grid), kThreads, smem, st>>>(a, uint32_t(tiles));
  return cudaGetLastError();
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
