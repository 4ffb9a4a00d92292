// Global levels of the median k-d partition (Sec. 4.1 of arXiv 2404.02826).
//
// A node at depth l splits on axis l mod 3, or (widest-cell variant) on the
// axis along which its cell (the root's code bounds cut by its ancestors'
// splits) is widest, the lowest of equal widths.  Sorting its particles by
// (code, original index), the first floor(c/2) go left, so the median lies on
// the larger-coordinate side.  Particles of a node are stored contiguously and
// in original-index order (every partition is stable), so "original index" is
// simply "position in the node".
//
// One level is four kernels:
//   prep     per node: code bounds -> first radix digit (or "all equal")
//   hist     per node and digit: histogram of the digit of (code - lo)
//   select   per node: the bucket that holds rank floor(c/2); after the last
//            digit this gives the split code v, the count below it and how
//            many particles equal to v go left
//   scatter  stable two-way partition of every node into its children
//            (k_scatter.cu)
// Levels of many small nodes replace hist and select by k_median: one warp per
// node with a private shared-memory histogram runs every digit of the radix
// select for its node, with no block barrier and no global histogram.
#include <cstdint>

#include "pc_internal.cuh"

namespace pcx {
namespace {

constexpr int kHistThreads = 512;
constexpr int kSelThreads = 256;
constexpr int kMedWarps = 16;                 // warps (nodes in flight) per k_median block
constexpr uint32_t kMedBins = 1u << kMedD;    // private histogram of one warp

// --------------------------------------------------------------------------
// prep: bounds of every node from its parent's split, then its first digit
// --------------------------------------------------------------------------
__global__ void k_prep(LevelNode *nodes, const LevelNode *parents, uint64_t n, int level, uint32_t digit_bits,
                       LevelLaunch::RootHi root_hi, uint32_t leaf_size, bool widest, const uint32_t *err) {
  if (call_failed(err)) return;
  const uint64_t count = 1ull << level;
  const uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= count) return;
  LevelNode nd = {};
  if (level == 0) {
    for (int d = 0; d < 3; ++d) {
      nd.blo[d] = 0;
      nd.bhi[d] = root_hi.v[d];
    }
  } else {
    const LevelNode &p = parents[j >> 1];
    for (int d = 0; d < 3; ++d) {
      nd.blo[d] = p.blo[d];
      nd.bhi[d] = p.bhi[d];
    }
    if (p.v != 0xffffffffu) {  // the parent was split at p.v on its axis
      const int pa = int(p.axis);
      if (j & 1) nd.blo[pa] = p.v;
      else nd.bhi[pa] = p.v;
    }
  }
  int axis = level % 3;
  if (widest) {
    axis = 0;
    for (int d = 1; d < 3; ++d)
      if (nd.bhi[d] - nd.blo[d] > nd.bhi[axis] - nd.blo[axis]) axis = d;
  }
  nd.axis = uint32_t(axis);
  nd.lo = nd.blo[axis];
  nd.hi = nd.bhi[axis];
  uint64_t off, cnt;
  node_range(n, level, j, off, cnt);
  const uint32_t k = uint32_t(cnt >> 1);
  const uint32_t B = bit_length(nd.hi - nd.lo);
  if (cnt <= leaf_size) {  // already a leaf: every code is below v, the node is copied as is
    nd.width = 0;
    nd.v = 0xffffffffu;
    nd.less = uint32_t(cnt);
    nd.tleft = 0;
  } else if (B == 0) {
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
}

// --------------------------------------------------------------------------
// hist: each block walks a contiguous, 16-aligned range node by node
// --------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(kHistThreads) k_hist(const C *__restrict__ q0, const C *__restrict__ q1,
                                                       const C *__restrict__ q2, const LevelNode *__restrict__ nodes,
                                                       uint32_t *__restrict__ hist, uint64_t n, int level,
                                                       uint32_t digit_bits, const uint32_t *err) {
  extern __shared__ uint32_t sh[];
  if (call_failed(err)) return;
  uint64_t start = ((n * blockIdx.x / gridDim.x) + 15) & ~15ull;
  uint64_t end = blockIdx.x + 1 == gridDim.x ? n : (((n * (blockIdx.x + 1) / gridDim.x) + 15) & ~15ull);
  if (end > n) end = n;
  if (start >= end) return;
  uint64_t lo = 0, hi = (1ull << level) - 1;  // node holding `start`
  while (lo < hi) {
    const uint64_t mid = (lo + hi + 1) >> 1;
    uint64_t off, cnt;
    node_range(n, level, mid, off, cnt);
    if (off <= start) lo = mid;
    else hi = mid - 1;
  }
  uint64_t j = lo;
  constexpr uint32_t kVec = 16 / sizeof(C);  // codes per 16-byte load
  while (start < end) {
    uint64_t off, cnt;
    node_range(n, level, j, off, cnt);
    const uint64_t seg_end = (off + cnt) < end ? (off + cnt) : end;
    const LevelNode nd = nodes[j];
    if (nd.width) {
      const C *codes = nd.axis == 0 ? q0 : (nd.axis == 1 ? q1 : q2);
      const uint32_t nb = 1u << nd.width, mask = nb - 1;
      const uint32_t lo_c = nd.lo, prefix = nd.prefix, width = nd.width;
      const int shift = nd.shift;
      for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) sh[b] = 0;
      __syncthreads();
      auto add = [&](uint32_t q) {
        const uint32_t hb = (q - lo_c) >> shift;
        if ((hb >> width) == prefix) atomicAdd(&sh[hb & mask], 1u);
      };
      auto add4 = [&](const uint4 &w) {
        const uint32_t x[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (sizeof(C) == 2) {
            add(x[c] & 0xffffu);
            add(x[c] >> 16);
          } else {
            add(x[c]);
          }
        }
      };
      const uint64_t a0 = (start + kVec - 1) / kVec * kVec;  // first aligned index
      const uint64_t a1 = seg_end / kVec * kVec;              // end of the aligned body
      if (a0 >= a1) {
        for (uint64_t e = start + threadIdx.x; e < seg_end; e += blockDim.x) add(__ldcg(codes + e));
      } else {
        for (uint64_t e = start + threadIdx.x; e < a0; e += blockDim.x) add(__ldcg(codes + e));
        for (uint64_t e = a1 + threadIdx.x; e < seg_end; e += blockDim.x) add(__ldcg(codes + e));
        const uint4 *v = reinterpret_cast<const uint4 *>(codes + a0);
        const uint64_t nv = (a1 - a0) / kVec;
        uint64_t i = threadIdx.x;
        // four 16-byte loads per thread and step; the next step's loads are issued
        // before this step's codes are counted, so their latency hides behind the atomics
        if (i + 3 * blockDim.x < nv) {
          uint4 w[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) w[u] = __ldcg(v + i + u * blockDim.x);
          for (;;) {
            const uint64_t in = i + 4 * blockDim.x;
            const bool more = in + 3 * blockDim.x < nv;
            uint4 nx[4];
            if (more) {
#pragma unroll
              for (int u = 0; u < 4; ++u) nx[u] = __ldcg(v + in + u * blockDim.x);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) add4(w[u]);
            i = in;
            if (!more) break;
#pragma unroll
            for (int u = 0; u < 4; ++u) w[u] = nx[u];
          }
        }
        for (; i < nv; i += blockDim.x) add4(__ldcg(v + i));
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
                                                        uint32_t digit_bits, const uint32_t *err) {
  __shared__ uint32_t warp_tot[33];
  __shared__ uint32_t found_b, found_before;
  if (call_failed(err)) return;
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
// median: one warp per node, all digits (levels of many small nodes)
// --------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(kMedWarps * 32) k_median(const C *__restrict__ q0, const C *__restrict__ q1,
                                                            const C *__restrict__ q2, LevelNode *nodes, uint64_t n,
                                                            int level, const uint32_t *err) {
  extern __shared__ uint32_t med_hist[];
  if (call_failed(err)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *h = med_hist + warp * kMedBins;
  const uint64_t count = 1ull << level;
  constexpr uint32_t kVec = 16 / sizeof(C);
  for (uint64_t j = uint64_t(blockIdx.x) * kMedWarps + warp; j < count; j += uint64_t(gridDim.x) * kMedWarps) {
    LevelNode nd = nodes[j];
    if (nd.width == 0) continue;  // a leaf, or all codes equal: prep has decided
    const C *codes = nd.axis == 0 ? q0 : (nd.axis == 1 ? q1 : q2);
    uint64_t off64, cnt64;
    node_range(n, level, j, off64, cnt64);
    const uint32_t off = uint32_t(off64), cnt = uint32_t(cnt64), k = cnt >> 1;
    for (;;) {
      const uint32_t lo_c = nd.lo, prefix = nd.prefix, width = nd.width, mask = (1u << width) - 1u;
      const int shift = nd.shift;
      for (uint32_t b = lane; b < kMedBins; b += 32) h[b] = 0;
      __syncwarp();
      auto add = [&](uint32_t q) {
        const uint32_t hb = (q - lo_c) >> shift;
        if ((hb >> width) == prefix) atomicAdd(&h[hb & mask], 1u);
      };
      const uint32_t a0 = min((off + kVec - 1) & ~(kVec - 1), off + cnt), a1 = max(a0, (off + cnt) & ~(kVec - 1));
      for (uint32_t e = off + lane; e < a0; e += 32) add(__ldcg(codes + e));
      for (uint32_t e = a1 + lane; e < off + cnt; e += 32) add(__ldcg(codes + e));
      const uint4 *v4 = reinterpret_cast<const uint4 *>(codes + a0);
      const uint32_t nv = (a1 - a0) / kVec;
      uint32_t i = lane;
      for (; i + 96 < nv; i += 128) {
        uint4 w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] = __ldcg(v4 + i + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t x[4] = {w[u].x, w[u].y, w[u].z, w[u].w};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (sizeof(C) == 2) {
              add(x[c] & 0xffffu);
              add(x[c] >> 16);
            } else {
              add(x[c]);
            }
          }
        }
      }
      for (; i < nv; i += 32) {
        const uint4 w = __ldcg(v4 + i);
        const uint32_t x[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (sizeof(C) == 2) {
            add(x[c] & 0xffffu);
            add(x[c] >> 16);
          } else {
            add(x[c]);
          }
        }
      }
      __syncwarp();
      // the bucket holding rank k - below: 32 bins at a time, one per lane
      const uint32_t target = k - nd.below;
      uint32_t run = 0, found_b = 0, found_before = 0;
      const uint32_t nb = 1u << width;
      for (uint32_t c0 = 0; c0 < nb; c0 += 32) {
        const uint32_t x = c0 + lane < nb ? h[c0 + lane] : 0u;
        uint32_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const uint32_t hit = __ballot_sync(0xffffffffu, x && run + incl - x <= target && target < run + incl);
        if (hit) {
          const int src = __ffs(hit) - 1;
          found_b = c0 + src;
          found_before = run + __shfl_sync(0xffffffffu, incl - x, src);
          break;
        }
        run += __shfl_sync(0xffffffffu, incl, 31);
      }
      __syncwarp();
      nd.below += found_before;
      nd.prefix = (nd.prefix << nd.width) | found_b;
      if (nd.shift == 0) {
        nd.v = nd.lo + nd.prefix;
        nd.less = nd.below;
        nd.tleft = k - nd.less;
        nd.width = 0;
        break;
      }
      const uint32_t w = uint32_t(nd.shift) < kMedD ? uint32_t(nd.shift) : kMedD;
      nd.shift -= int32_t(w);
      nd.width = w;
    }
    if (lane == 0) nodes[j] = nd;
  }
}

template <typename C>
cudaError_t level_dispatch(const LevelLaunch &a, cudaStream_t st) {
  const uint64_t count = 1ull << a.level;
  {
    TraceScope ts("k_prep", st);
    LevelLaunch::RootHi rh;
    for (int d = 0; d < 3; ++d) rh.v[d] = a.root_hi[d];
    k_prep<<<unsigned((count + 255) / 256), 256, 0, st>>>(a.nodes, a.parents, a.n, a.level, a.digit_bits, rh,
                                                          a.leaf_size, a.widest, a.err);
  }
  const C *q0 = static_cast<const C *>(a.src[0]), *q1 = static_cast<const C *>(a.src[1]),
          *q2 = static_cast<const C *>(a.src[2]);
  if (a.warp_median) {
    const size_t msm = sizeof(uint32_t) * kMedBins * kMedWarps;
    int per_sm = 0;
    cudaError_t e = resident_blocks<k_median<C>>(kMedWarps * 32, msm, &per_sm);
    if (e != cudaSuccess) return e;
    uint64_t grid = uint64_t(per_sm < 1 ? 1 : per_sm) * uint64_t(device_sm_count());
    const uint64_t need = (count + kMedWarps - 1) / kMedWarps;
    if (grid > need) grid = need;
    {
      TraceScope ts("k_median", st);
      k_median<C><<<unsigned(grid), kMedWarps * 32, msm, st>>>(q0, q1, q2, a.nodes, a.n, a.level, a.err);
    }
    return launch_scatter(a, st);
  }
  const size_t hsm = sizeof(uint32_t) << a.digit_bits;
  for (uint32_t p = 0; p < a.passes; ++p) {
    {
      TraceScope ts("k_hist", st);
      k_hist<C><<<a.hist_blocks, kHistThreads, hsm, st>>>(q0, q1, q2, a.nodes, a.hist, a.n, a.level, a.digit_bits,
                                                               a.err);
    }
    TraceScope ts("k_select", st);
    k_select<<<unsigned(count), kSelThreads, 0, st>>>(a.nodes, a.hist, a.n, a.level, a.digit_bits, a.err);
  }
  return launch_scatter(a, st);
}

}  // namespace

cudaError_t launch_level(const LevelLaunch &a, cudaStream_t st) {
  return a.code_bytes == 2 ? level_dispatch<uint16_t>(a, st) : level_dispatch<uint32_t>(a, st);
}

}  // namespace pcx
