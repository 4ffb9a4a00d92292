// Global levels of the median k-d partition (Sec. 4.1 of arXiv 2404.02826).
//
// A node at depth l splits on axis l mod 3.  Sorting its particles by
// (code, original index), the first floor(c/2) go left, so the median lies on
// the larger-coordinate side.  Particles of a node are stored contiguously and
// in original-index order (every partition below is stable), so "original
// index" is simply "position in the node".
//
// One level is four kernels:
//   prep     per node: code bounds -> first radix digit (or "all equal")
//   hist     per node and digit: histogram of the digit of (code - lo)
//   select   per node: the bucket that holds rank floor(c/2); after the last
//            digit this gives the split code v, the count below it and how
//            many particles equal to v go left
//   scatter  stable two-way partition of every node into its children, with
//            the node-local prefix counts obtained by a decoupled look-back
//            over the node's tiles; it also records each child's code bounds
//            on the next axis
#include <cuda/atomic>
#include <cstdint>

#include "pc_internal.cuh"

namespace pcx {
namespace {

constexpr int kHistThreads = 512;
constexpr int kSelThreads = 256;
constexpr int kScatThreads = 256;
constexpr int kScatWarps = kScatThreads / 32;
constexpr int kScatItems = 16;                         // per lane
constexpr int kTile = kScatThreads * kScatItems;       // 4096 particles

constexpr unsigned long long kFlagA = 1ull << 62;      // tile aggregate published
constexpr unsigned long long kFlagP = 2ull << 62;      // inclusive prefix published
constexpr unsigned long long kValMask = (1ull << 62) - 1;

__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v) {
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> r(*p);
  r.store(v, cuda::memory_order_release);
}
__device__ __forceinline__ unsigned long long ld_acquire(unsigned long long *p) {
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> r(*p);
  return r.load(cuda::memory_order_acquire);
}
__device__ __forceinline__ uint32_t ld_relaxed(uint32_t *p) {
  cuda::atomic_ref<uint32_t, cuda::thread_scope_device> r(*p);
  return r.load(cuda::memory_order_relaxed);
}

// Decoupled look-back: tile t publishes its aggregate, sums its predecessors
// back to the first inclusive prefix (or the node's first tile), publishes its
// own inclusive prefix and returns the exclusive one.  Every wait is bounded;
// on expiry the error word is set and the tile unblocks its successors.
__device__ unsigned long long lookback(unsigned long long *state, uint64_t t, uint64_t first,
                                       unsigned long long agg, uint32_t *err) {
  if (t == first) {
    st_release(&state[t], kFlagP | agg);
    return 0;
  }
  st_release(&state[t], kFlagA | agg);
  unsigned long long excl = 0;
  uint64_t pred = t - 1;
  for (;;) {
    unsigned long long s;
    uint32_t spins = 0;
    while (((s = ld_acquire(&state[pred])) >> 62) == 0) {
      if (++spins > kSpinLimit || (ld_relaxed(err) & kErrTimeout)) {
        atomicOr(err, kErrTimeout);
        st_release(&state[t], kFlagP | ((excl + agg) & kValMask));
        return excl;
      }
      __nanosleep(64);
    }
    excl += s & kValMask;
    if ((s & ~kValMask) == kFlagP || pred == first) break;
    --pred;
  }
  st_release(&state[t], kFlagP | ((excl + agg) & kValMask));
  return excl;
}

template <typename C>
__device__ __forceinline__ uint32_t ldc(const C *p) {
  return (uint32_t)__ldcg(p);
}

// --------------------------------------------------------------------------
// prep: first digit of every node; children bounds reset for the scatter
// --------------------------------------------------------------------------
__global__ void k_prep(LevelNode *nodes, LevelNode *children, uint64_t n, int level, uint32_t digit_bits,
                       uint32_t root_hi) {
  const uint64_t count = 1ull << level;
  const uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= count) return;
  LevelNode nd = {};
  if (level == 0) {
    nd.lo = 0;
    nd.hi = root_hi;
  } else {
    nd.lo = nodes[j].lo;
    nd.hi = nodes[j].hi;
  }
  uint64_t off, cnt;
  node_range(n, level, j, off, cnt);
  const uint32_t k = uint32_t(cnt >> 1);
  const uint32_t B = bit_length(nd.hi - nd.lo);
  if (B == 0) {
    nd.width = 0;
    nd.v = nd.lo;
    nd.less = 0;
    nd.tleft = k;
  } else {
    nd.width = B < digit_bits ? B : digit_bits;
    nd.shift = int32_t(B - nd.width);
    nd.prefix = 0;
    nd.below = 0;
  }
  nodes[j] = nd;
  if (children) {
    LevelNode c = {};
    c.lo = 0xffffffffu;
    c.hi = 0;
    children[2 * j] = c;
    children[2 * j + 1] = c;
  }
}

// --------------------------------------------------------------------------
// hist: each block walks a contiguous range of particles node by node
// --------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(kHistThreads) k_hist(const C *__restrict__ codes, const LevelNode *__restrict__ nodes,
                                                       uint32_t *__restrict__ hist, uint64_t n, int level,
                                                       uint32_t digit_bits) {
  extern __shared__ uint32_t sh[];
  uint64_t start = n * blockIdx.x / gridDim.x;
  const uint64_t end = n * (blockIdx.x + 1) / gridDim.x;
  if (start >= end) return;
  // node holding `start`: the last j with off(j) <= start
  uint64_t lo = 0, hi = (1ull << level) - 1;
  while (lo < hi) {
    uint64_t mid = (lo + hi + 1) >> 1, off, cnt;
    node_range(n, level, mid, off, cnt);
    if (off <= start) lo = mid;
    else hi = mid - 1;
  }
  uint64_t j = lo;
  while (start < end) {
    uint64_t off, cnt;
    node_range(n, level, j, off, cnt);
    const uint64_t seg_end = (off + cnt) < end ? (off + cnt) : end;
    const LevelNode nd = nodes[j];
    if (nd.width) {
      const uint32_t nb = 1u << nd.width, mask = nb - 1;
      for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) sh[b] = 0;
      __syncthreads();
      for (uint64_t e = start + threadIdx.x; e < seg_end; e += blockDim.x) {
        const uint32_t rel = ldc(codes + e) - nd.lo;
        const uint32_t hi_bits = rel >> nd.shift;
        if ((hi_bits >> nd.width) == nd.prefix) atomicAdd(&sh[hi_bits & mask], 1u);
      }
      __syncthreads();
      uint32_t *g = hist + (j << digit_bits);
      for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
        const uint32_t c = sh[b];
        if (c) atomicAdd(g + b, c);
      }
      __syncthreads();
    }
    start = seg_end;
    ++j;
  }
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *warp_tot, uint32_t &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  uint32_t incl = x;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < warps ? warp_tot[lane] : 0, ti = t;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < warps) warp_tot[lane] = ti - t;  // exclusive warp base
    if (lane == 31) warp_tot[32] = ti;
  }
  __syncthreads();
  total = warp_tot[32];
  uint32_t r = warp_tot[warp] + incl - x;
  __syncthreads();
  return r;
}

// --------------------------------------------------------------------------
// select: one block per node; finds the bucket of rank floor(c/2)
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kSelThreads) k_select(LevelNode *nodes, uint32_t *hist, uint64_t n, int level,
                                                        uint32_t digit_bits) {
  __shared__ uint32_t warp_tot[33];
  __shared__ uint32_t found_b, found_before;
  const uint64_t j = blockIdx.x;
  LevelNode nd = nodes[j];
  if (nd.width == 0) return;
  uint64_t off, cnt;
  node_range(n, level, j, off, cnt);
  const uint32_t k = uint32_t(cnt >> 1);
  const uint32_t target = k - nd.below;
  const uint32_t nb = 1u << nd.width;
  const uint32_t per = (nb + blockDim.x - 1) / blockDim.x;
  uint32_t *h = hist + (j << digit_bits);
  const uint32_t b0 = threadIdx.x * per;
  const uint32_t b1 = (b0 + per) < nb ? (b0 + per) : nb;
  uint32_t sum = 0;
  for (uint32_t b = b0; b < b1; ++b) sum += h[b];
  if (threadIdx.x == 0) {
    found_b = 0xffffffffu;
    found_before = 0;
  }
  uint32_t total;
  const uint32_t ex = block_excl_scan(sum, warp_tot, total);
  if (sum && ex <= target && target < ex + sum) {
    uint32_t c = ex;
    for (uint32_t b = b0; b < b1; ++b) {
      const uint32_t hb = h[b];
      if (target < c + hb) {
        found_b = b;
        found_before = c;
        break;
      }
      c += hb;
    }
  }
  for (uint32_t b = b0; b < b1; ++b) h[b] = 0;  // leave the histogram zero for the next pass
  __syncthreads();
  if (threadIdx.x == 0) {
    if (found_b == 0xffffffffu) {
      // cannot happen for a consistent histogram; keep the node well-formed
      found_b = 0;
      found_before = 0;
    }
    nd.below += found_before;
    nd.prefix = (nd.prefix << nd.width) | found_b;
    if (nd.shift == 0) {
      nd.v = nd.lo + nd.prefix;
      nd.less = nd.below;
      nd.tleft = k - nd.less;
      nd.width = 0;
    } else {
      const uint32_t w = uint32_t(nd.shift) < digit_bits ? uint32_t(nd.shift) : digit_bits;
      nd.shift -= int32_t(w);
      nd.width = w;
    }
    nodes[j] = nd;
  }
}

// --------------------------------------------------------------------------
// scatter: stable partition of each node into its two children
// --------------------------------------------------------------------------
template <typename C, bool IDX>
struct ScatShared {
  C q[3][kTile];
  uint32_t idx[IDX ? kTile : 1];
  uint32_t wless[kScatWarps], wtie[kScatWarps];
  uint32_t wless_ex[kScatWarps], wtie_ex[kScatWarps];
  uint64_t tile;
  uint32_t left_before, right_before, left_tile, less_before, tie_before;
};

template <typename C, bool IDX>
__global__ void __launch_bounds__(kScatThreads) k_scatter(LevelLaunch a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  ScatShared<C, IDX> &S = *reinterpret_cast<ScatShared<C, IDX> *>(smraw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int axis = a.level % 3, nxt = (a.level + 1) % 3;
  if (threadIdx.x == 0) S.tile = atomicAdd(a.ticket, 1u);
  __syncthreads();
  const uint64_t t = S.tile;
  const uint64_t T = a.tiles_per_node;
  const uint64_t j = t / T, i = t % T;
  uint64_t off, cnt;
  node_range(a.n, a.level, j, off, cnt);
  const uint64_t k = cnt >> 1;
  const uint64_t tb = off + (cnt * i) / T;
  const uint64_t te = off + (cnt * (i + 1)) / T;
  const uint32_t sz = uint32_t(te - tb);
  const LevelNode nd = a.nodes[j];
  const uint32_t v = nd.v, tl = nd.tleft;
  const C *src0 = static_cast<const C *>(a.src[0]);
  const C *src1 = static_cast<const C *>(a.src[1]);
  const C *src2 = static_cast<const C *>(a.src[2]);

  uint32_t q0[kScatItems], q1[kScatItems], q2[kScatItems], id[IDX ? kScatItems : 1];
  uint32_t wl = 0, wt = 0;
#pragma unroll
  for (int e = 0; e < kScatItems; ++e) {
    const uint32_t p = uint32_t(warp) * (32 * kScatItems) + uint32_t(e) * 32 + lane;
    const bool valid = p < sz;
    q0[e] = valid ? ldc(src0 + tb + p) : 0;
    q1[e] = valid ? ldc(src1 + tb + p) : 0;
    q2[e] = valid ? ldc(src2 + tb + p) : 0;
    if (IDX) id[e] = valid ? __ldcg(a.src_idx + tb + p) : 0;
    const uint32_t qa = axis == 0 ? q0[e] : (axis == 1 ? q1[e] : q2[e]);
    wl += __popc(__ballot_sync(0xffffffffu, valid && qa < v));
    wt += __popc(__ballot_sync(0xffffffffu, valid && qa == v));
  }
  if (lane == 0) {
    S.wless[warp] = wl;
    S.wtie[warp] = wt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t sl = 0, st = 0;
    for (int w = 0; w < kScatWarps; ++w) {
      S.wless_ex[w] = sl;
      S.wtie_ex[w] = st;
      sl += S.wless[w];
      st += S.wtie[w];
    }
    const unsigned long long agg = ((unsigned long long)sl << 31) | st;
    const unsigned long long ex = lookback(a.tile_state, t, j * T, agg, a.err);
    const uint32_t less_before = uint32_t(ex >> 31), tie_before = uint32_t(ex & 0x7fffffffu);
    const uint32_t lb = less_before + min(tie_before, tl);
    const uint32_t lincl = less_before + sl + min(tie_before + st, tl);
    S.less_before = less_before;
    S.tie_before = tie_before;
    S.left_before = lb;
    S.left_tile = lincl - lb;
    S.right_before = uint32_t(tb - off) - lb;
  }
  __syncthreads();
  const uint32_t less_before = S.less_before, tie_before = S.tie_before;
  const uint32_t left_before = S.left_before, left_tile = S.left_tile, right_before = S.right_before;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t run_l = S.wless_ex[warp], run_t = S.wtie_ex[warp];
  uint32_t cmin0 = 0xffffffffu, cmax0 = 0, cmin1 = 0xffffffffu, cmax1 = 0;
#pragma unroll
  for (int e = 0; e < kScatItems; ++e) {
    const uint32_t p = uint32_t(warp) * (32 * kScatItems) + uint32_t(e) * 32 + lane;
    const bool valid = p < sz;
    const uint32_t qa = axis == 0 ? q0[e] : (axis == 1 ? q1[e] : q2[e]);
    const bool isless = valid && qa < v, istie = valid && qa == v;
    const uint32_t bl = __ballot_sync(0xffffffffu, isless), bt = __ballot_sync(0xffffffffu, istie);
    const uint32_t less_ex = run_l + __popc(bl & lt_mask);
    const uint32_t tie_ex = run_t + __popc(bt & lt_mask);
    run_l += __popc(bl);
    run_t += __popc(bt);
    if (valid) {
      const uint32_t trank = tie_before + tie_ex;
      const bool left = isless || (istie && trank < tl);
      const uint32_t glrank = less_before + less_ex + min(trank, tl);
      uint32_t local;
      if (left) {
        local = glrank - left_before;
      } else {
        const uint32_t grrank = uint32_t(tb + p - off) - glrank;
        local = left_tile + (grrank - right_before);
      }
      if (local < sz) {
        S.q[0][local] = (C)q0[e];
        S.q[1][local] = (C)q1[e];
        S.q[2][local] = (C)q2[e];
        if (IDX) S.idx[local] = id[e];
      } else {
        atomicOr(a.err, kErrInternal);
      }
      const uint32_t qn = nxt == 0 ? q0[e] : (nxt == 1 ? q1[e] : q2[e]);
      if (left) {
        cmin0 = min(cmin0, qn);
        cmax0 = max(cmax0, qn);
      } else {
        cmin1 = min(cmin1, qn);
        cmax1 = max(cmax1, qn);
      }
    }
  }
  cmin0 = __reduce_min_sync(0xffffffffu, cmin0);
  cmax0 = __reduce_max_sync(0xffffffffu, cmax0);
  cmin1 = __reduce_min_sync(0xffffffffu, cmin1);
  cmax1 = __reduce_max_sync(0xffffffffu, cmax1);
  if (lane == 0 && a.children) {
    if (cmin0 <= cmax0) {
      atomicMin(&a.children[2 * j].lo, cmin0);
      atomicMax(&a.children[2 * j].hi, cmax0);
    }
    if (cmin1 <= cmax1) {
      atomicMin(&a.children[2 * j + 1].lo, cmin1);
      atomicMax(&a.children[2 * j + 1].hi, cmax1);
    }
  }
  __syncthreads();
  C *d0 = static_cast<C *>(a.dst[0]);
  C *d1 = static_cast<C *>(a.dst[1]);
  C *d2 = static_cast<C *>(a.dst[2]);
  for (uint32_t p = threadIdx.x; p < sz; p += kScatThreads) {
    const uint64_t dst = p < left_tile ? off + left_before + p : off + k + right_before + (p - left_tile);
    if (dst >= off + cnt) {
      atomicOr(a.err, kErrInternal);
      continue;
    }
    __stcg(d0 + dst, S.q[0][p]);
    __stcg(d1 + dst, S.q[1][p]);
    __stcg(d2 + dst, S.q[2][p]);
    if (IDX) __stcg(a.dst_idx + dst, S.idx[p]);
  }
}

template <typename C, bool IDX>
cudaError_t level_dispatch(const LevelLaunch &a, cudaStream_t st) {
  const uint64_t count = 1ull << a.level;
  {
    TraceScope ts("k_prep", st);
    k_prep<<<unsigned((count + 255) / 256), 256, 0, st>>>(a.nodes, a.children, a.n, a.level, a.digit_bits,
                                                          a.root_hi);
  }
  const int axis = a.level % 3;
  const C *codes = static_cast<const C *>(a.src[axis]);
  const size_t hsm = sizeof(uint32_t) << a.digit_bits;
  for (uint32_t p = 0; p < a.passes; ++p) {
    {
      TraceScope ts("k_hist", st);
      k_hist<C><<<a.hist_blocks, kHistThreads, hsm, st>>>(codes, a.nodes, a.hist, a.n, a.level, a.digit_bits);
    }
    TraceScope ts("k_select", st);
    k_select<<<unsigned(count), kSelThreads, 0, st>>>(a.nodes, a.hist, a.n, a.level, a.digit_bits);
  }
  const size_t ssm = sizeof(ScatShared<C, IDX>);
  cudaError_t e = cudaFuncSetAttribute(k_scatter<C, IDX>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ssm));
  if (e != cudaSuccess) return e;
  const uint64_t tiles = count * a.tiles_per_node;
  TraceScope ts("k_scatter", st);
  k_scatter<C, IDX><<<unsigned(tiles), kScatThreads, ssm, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

uint32_t scatter_tile() { return kTile; }

cudaError_t launch_level(const LevelLaunch &a, cudaStream_t st) {
  if (a.code_bytes == 2)
    return a.with_idx ? level_dispatch<uint16_t, true>(a, st) : level_dispatch<uint16_t, false>(a, st);
  return a.with_idx ? level_dispatch<uint32_t, true>(a, st) : level_dispatch<uint32_t, false>(a, st);
}

}  // namespace pcx
