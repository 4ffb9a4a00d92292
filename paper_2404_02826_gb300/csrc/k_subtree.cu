// Subtree kernel: everything below the global levels, one k-d subtree per CTA,
// held in shared memory (Sec. 4.1 partition and bit boxes, Sec. 4.2 layout).
//
// Per CTA (1024 threads, one per SM):
//   1. take the next subtree in order (ticket), load its codes into SMEM;
//   2. depth-first: split every node with more than r particles on axis
//      depth mod 3 (radix select of the median in SMEM, stable partition with
//      warp ballots, permutation through registers), so leaves come out in
//      left-to-right order;
//   3. per leaf, the bit box: AABB, the particle closest to the AABB centre
//      (squared distance in doubled lattice units, first in leaf order on
//      ties), R_d and m_d of Eq. 2, and the payload size (sum m)(n - 1) bits;
//   4. decoupled look-back over the subtrees for the first payload word;
//   5. leaf records and the packed payload: each output word is assembled
//      from the codes that overlap it, c_d = q_d - q_ref_d + 2^(m_d-1) - 1,
//      least significant bit first, so every word is written exactly once.
#include <cuda/atomic>
#include <cstdint>

#include "pc_internal.cuh"

namespace pcx {
namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kDigit = 11;  // radix digit of the in-SMEM select
constexpr unsigned long long kFlagA = 1ull << 62;
constexpr unsigned long long kFlagP = 2ull << 62;
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

// Register buffer of EMAX 16-bit values, two per register.
template <int EMAX>
struct Half16 {
  uint32_t w[(EMAX + 1) / 2];
  __device__ __forceinline__ void set(int e, uint32_t v) {
    if (e & 1) w[e >> 1] = (w[e >> 1] & 0xffffu) | (v << 16);
    else w[e >> 1] = (w[e >> 1] & 0xffff0000u) | (v & 0xffffu);
  }
  __device__ __forceinline__ uint32_t get(int e) const { return (e & 1) ? (w[e >> 1] >> 16) : (w[e >> 1] & 0xffffu); }
};
template <int EMAX>
struct Full32 {
  uint32_t w[EMAX];
  __device__ __forceinline__ void set(int e, uint32_t v) { w[e] = v; }
  __device__ __forceinline__ uint32_t get(int e) const { return w[e]; }
};
template <typename V, int EMAX>
struct RegBuf;
template <int EMAX>
struct RegBuf<uint16_t, EMAX> : Half16<EMAX> {};
template <int EMAX>
struct RegBuf<uint32_t, EMAX> : Full32<EMAX> {};

struct Frame {
  uint32_t off, cnt, depth;
};

struct Ctl {
  uint32_t warp_a[33], warp_b[33];
  unsigned long long warp_d[kWarps];
  uint32_t warp_p[kWarps];
  uint32_t red[6][kWarps];
  Frame stack[64];
  int sp;
  Frame cur;
  uint32_t s_lo, s_hi, found_b, found_before;
  uint32_t v, less, tleft;
  uint32_t leaves, words;
  uint64_t subtree;
  uint64_t word_base;
  unsigned long long best_d;
  uint32_t best_p;
  uint32_t bmin[3], bmax[3];
};

__device__ __forceinline__ uint32_t block_min(uint32_t x, uint32_t *slot) {
  x = __reduce_min_sync(0xffffffffu, x);
  if ((threadIdx.x & 31) == 0) slot[threadIdx.x >> 5] = x;
  __syncthreads();
  uint32_t r = slot[0];
  for (int w = 1; w < kWarps; ++w) r = min(r, slot[w]);
  __syncthreads();
  return r;
}
__device__ __forceinline__ uint32_t block_max(uint32_t x, uint32_t *slot) {
  x = __reduce_max_sync(0xffffffffu, x);
  if ((threadIdx.x & 31) == 0) slot[threadIdx.x >> 5] = x;
  __syncthreads();
  uint32_t r = slot[0];
  for (int w = 1; w < kWarps; ++w) r = max(r, slot[w]);
  __syncthreads();
  return r;
}

// Exclusive scan of one value per thread over the block; also the total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *warp_tot, uint32_t &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = x;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = warp_tot[lane], ti = t;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    warp_tot[lane] = ti - t;
    if (lane == 31) warp_tot[32] = ti;
  }
  __syncthreads();
  total = warp_tot[32];
  const uint32_t r = warp_tot[warp] + incl - x;
  __syncthreads();
  return r;
}

template <typename C, bool IDX, int EMAX>
struct Sub {
  static constexpr uint32_t kCap = uint32_t(EMAX) * kThreads;

  // Permute one array of the node in place: X[dst(e)] = X[src(e)].
  template <typename V>
  static __device__ __forceinline__ void permute(V *X, const Half16<EMAX> &dst, uint32_t E, uint32_t n, int warp,
                                                 int lane) {
    RegBuf<V, EMAX> vb;
#pragma unroll
    for (int e = 0; e < EMAX; ++e) {
      const uint32_t p = uint32_t(warp) * 32u * E + uint32_t(e) * 32u + lane;
      if (uint32_t(e) < E && p < n) vb.set(e, X[p]);
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < EMAX; ++e) {
      const uint32_t p = uint32_t(warp) * 32u * E + uint32_t(e) * 32u + lane;
      if (uint32_t(e) < E && p < n && dst.get(e) < n) X[dst.get(e)] = (V)vb.get(e);
    }
    __syncthreads();
  }

  // Median split of the node [off, off + n) in SMEM on the given axis.
  static __device__ void split(C *sq0, C *sq1, C *sq2, uint32_t *sidx, uint32_t *hist, Ctl &c, uint32_t off,
                               uint32_t n, int axis) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C *qa = (axis == 0 ? sq0 : (axis == 1 ? sq1 : sq2)) + off;
    const uint32_t k = n >> 1;
    // bounds of the node on its axis
    uint32_t mn = 0xffffffffu, mx = 0;
    for (uint32_t i = threadIdx.x; i < n; i += kThreads) {
      const uint32_t q = qa[i];
      mn = min(mn, q);
      mx = max(mx, q);
    }
    const uint32_t lo = block_min(mn, c.red[0]);
    const uint32_t hi = block_max(mx, c.red[1]);
    uint32_t v, less, tl;
    if (lo == hi) {
      v = lo;
      less = 0;
      tl = k;
    } else {
      // radix select of rank k on (code - lo), digits from the top
      int shift = int(bit_length(hi - lo));
      uint32_t prefix = 0, below = 0;
      while (shift > 0) {
        const int width = shift < kDigit ? shift : kDigit;
        shift -= width;
        const uint32_t nb = 1u << width, mask = nb - 1;
        for (uint32_t b = threadIdx.x; b < nb; b += kThreads) hist[b] = 0;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += kThreads) {
          const uint32_t rel = uint32_t(qa[i]) - lo;
          const uint32_t hb = rel >> shift;
          if ((hb >> width) == prefix) atomicAdd(&hist[hb & mask], 1u);
        }
        __syncthreads();
        const uint32_t b0 = 2 * threadIdx.x;
        const uint32_t h0 = b0 < nb ? hist[b0] : 0, h1 = (b0 + 1) < nb ? hist[b0 + 1] : 0;
        uint32_t total;
        const uint32_t ex = block_excl_scan(h0 + h1, c.warp_a, total);
        const uint32_t target = k - below;
        if (threadIdx.x == 0) {
          c.found_b = 0;
          c.found_before = 0;
        }
        __syncthreads();
        if (h0 && ex <= target && target < ex + h0) {
          c.found_b = b0;
          c.found_before = ex;
        } else if (h1 && ex + h0 <= target && target < ex + h0 + h1) {
          c.found_b = b0 + 1;
          c.found_before = ex + h0;
        }
        __syncthreads();
        below += c.found_before;
        prefix = (prefix << width) | c.found_b;
        __syncthreads();
      }
      v = lo + prefix;
      less = below;
      tl = k - less;
    }
    // stable partition: warp w owns positions [w*32E, (w+1)*32E), lane-minor
    const uint32_t E = (n + kThreads - 1) / kThreads;
    uint32_t wl = 0, wt = 0;
#pragma unroll
    for (int e = 0; e < EMAX; ++e) {
      if (uint32_t(e) < E) {
        const uint32_t p = uint32_t(warp) * 32u * E + uint32_t(e) * 32u + lane;
        const bool valid = p < n;
        const uint32_t q = valid ? uint32_t(qa[p]) : 0;
        wl += __popc(__ballot_sync(0xffffffffu, valid && q < v));
        wt += __popc(__ballot_sync(0xffffffffu, valid && q == v));
      }
    }
    if (lane == 0) {
      c.warp_a[warp] = wl;
      c.warp_b[warp] = wt;
    }
    __syncthreads();
    if (warp == 0) {
      const uint32_t a0 = c.warp_a[lane], b0 = c.warp_b[lane];
      uint32_t ai = a0, bi = b0;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, ai, o), y = __shfl_up_sync(0xffffffffu, bi, o);
        if (lane >= o) {
          ai += x;
          bi += y;
        }
      }
      c.warp_a[lane] = ai - a0;
      c.warp_b[lane] = bi - b0;
    }
    __syncthreads();
    uint32_t run_l = c.warp_a[warp], run_t = c.warp_b[warp];
    const uint32_t lt_mask = (1u << lane) - 1u;
    Half16<EMAX> dst;
#pragma unroll
    for (int e = 0; e < EMAX; ++e) {
      if (uint32_t(e) < E) {
        const uint32_t p = uint32_t(warp) * 32u * E + uint32_t(e) * 32u + lane;
        const bool valid = p < n;
        const uint32_t q = valid ? uint32_t(qa[p]) : 0;
        const bool isless = valid && q < v, istie = valid && q == v;
        const uint32_t bl = __ballot_sync(0xffffffffu, isless), bt = __ballot_sync(0xffffffffu, istie);
        const uint32_t less_ex = run_l + __popc(bl & lt_mask);
        const uint32_t trank = run_t + __popc(bt & lt_mask);
        run_l += __popc(bl);
        run_t += __popc(bt);
        const bool left = isless || (istie && trank < tl);
        const uint32_t lrank = less_ex + min(trank, tl);
        const uint32_t d = left ? lrank : k + (p - lrank);
        dst.set(e, d < n ? d : 0xffffu);  // never out of the node (0xffff > any capacity)
      }
    }
    C *qb = (axis == 0 ? sq1 : sq0) + off;
    C *qc = (axis == 2 ? sq1 : sq2) + off;
    permute<C>(qb, dst, E, n, warp, lane);
    permute<C>(qc, dst, E, n, warp, lane);
    if (IDX) permute<uint32_t>(sidx + off, dst, E, n, warp, lane);
    permute<C>(qa, dst, E, n, warp, lane);
  }

  // Bit box of the leaf [off, off + n): AABB, centre, m_d (Eq. 2).
  static __device__ void bitbox(const C *sq0, const C *sq1, const C *sq2, Ctl &c, uint32_t off, uint32_t n,
                                uint32_t &centre, uint32_t qref[3], uint32_t m[3]) {
    const C *q[3] = {sq0 + off, sq1 + off, sq2 + off};
    uint32_t lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      uint32_t mn = 0xffffffffu, mx = 0;
      for (uint32_t i = threadIdx.x; i < n; i += kThreads) {
        const uint32_t x = q[d][i];
        mn = min(mn, x);
        mx = max(mx, x);
      }
      mn = __reduce_min_sync(0xffffffffu, mn);
      mx = __reduce_max_sync(0xffffffffu, mx);
      if ((threadIdx.x & 31) == 0) {
        c.red[2 * d][threadIdx.x >> 5] = mn;
        c.red[2 * d + 1][threadIdx.x >> 5] = mx;
      }
    }
    __syncthreads();
    for (int d = 0; d < 3; ++d) {
      uint32_t a = c.red[2 * d][0], b = c.red[2 * d + 1][0];
      for (int w = 1; w < kWarps; ++w) {
        a = min(a, c.red[2 * d][w]);
        b = max(b, c.red[2 * d + 1][w]);
      }
      lo[d] = a;
      hi[d] = b;
    }
    __syncthreads();
    // argmin of squared distance to the AABB centre, lowest position on ties
    unsigned long long bd = ~0ull;
    uint32_t bp = 0xffffffffu;
    for (uint32_t i = threadIdx.x; i < n; i += kThreads) {
      unsigned long long d2 = 0;
      for (int d = 0; d < 3; ++d) {
        const long long t = 2ll * (long long)q[d][i] - (long long)lo[d] - (long long)hi[d];
        d2 += (unsigned long long)(t * t);
      }
      if (d2 < bd) {  // i increases, so the first minimum is kept
        bd = d2;
        bp = i;
      }
    }
    for (int o = 16; o; o >>= 1) {
      const unsigned long long od = __shfl_xor_sync(0xffffffffu, bd, o);
      const uint32_t op = __shfl_xor_sync(0xffffffffu, bp, o);
      if (od < bd || (od == bd && op < bp)) {
        bd = od;
        bp = op;
      }
    }
    if ((threadIdx.x & 31) == 0) {
      c.warp_d[threadIdx.x >> 5] = bd;
      c.warp_p[threadIdx.x >> 5] = bp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long d0 = c.warp_d[0];
      uint32_t p0 = c.warp_p[0];
      for (int w = 1; w < kWarps; ++w)
        if (c.warp_d[w] < d0 || (c.warp_d[w] == d0 && c.warp_p[w] < p0)) {
          d0 = c.warp_d[w];
          p0 = c.warp_p[w];
        }
      c.best_p = p0;
    }
    __syncthreads();
    centre = c.best_p;
    for (int d = 0; d < 3; ++d) {
      qref[d] = q[d][centre];
      const uint32_t R = max(qref[d] - lo[d], hi[d] - qref[d]);
      m[d] = bits_for_range(R);
    }
    __syncthreads();
  }
};

template <typename C, bool IDX, int EMAX>
__global__ void __launch_bounds__(kThreads, 1) k_subtree(SubtreeLaunch a) {
  using S = Sub<C, IDX, EMAX>;
  constexpr uint32_t kCap = S::kCap;
  extern __shared__ __align__(16) unsigned char smraw[];
  C *sq0 = reinterpret_cast<C *>(smraw);
  C *sq1 = sq0 + kCap;
  C *sq2 = sq1 + kCap;
  uint32_t *sidx = reinterpret_cast<uint32_t *>(sq2 + kCap);
  uint32_t *hist = sidx + (IDX ? kCap : 0);
  __shared__ Ctl c;

  if (threadIdx.x == 0) {
    c.subtree = atomicAdd(a.ticket, 1u);
    c.sp = 0;
    c.leaves = 0;
    c.words = 0;
  }
  __syncthreads();
  const uint64_t s = c.subtree;
  uint64_t off0, cnt0;
  node_range(a.n, a.root_level, s, off0, cnt0);
  const uint32_t n0 = uint32_t(cnt0);
  const uint64_t small = a.n >> a.root_level;
  const uint64_t big_before = off0 - s * small;
  const uint64_t leaf_base = s * a.leaves_small + big_before * (a.leaves_big - a.leaves_small);

  // 1. load the subtree
  const C *g0 = static_cast<const C *>(a.src[0]) + off0;
  const C *g1 = static_cast<const C *>(a.src[1]) + off0;
  const C *g2 = static_cast<const C *>(a.src[2]) + off0;
  for (uint32_t i = threadIdx.x; i < n0; i += kThreads) {
    sq0[i] = __ldcs(g0 + i);
    sq1[i] = __ldcs(g1 + i);
    sq2[i] = __ldcs(g2 + i);
    if (IDX) sidx[i] = __ldcs(a.src_idx + off0 + i);
  }
  if (threadIdx.x == 0) {
    c.stack[0] = Frame{0u, n0, uint32_t(a.root_level)};
    c.sp = n0 ? 1 : 0;
  }
  __syncthreads();

  // 2-3. depth-first: split, or finish a leaf
  for (;;) {
    const int sp = c.sp;
    __syncthreads();
    if (sp == 0) break;
    if (threadIdx.x == 0) c.cur = c.stack[--c.sp];
    __syncthreads();
    const Frame f = c.cur;
    __syncthreads();
    if (f.cnt <= a.leaf_size) {
      uint32_t centre, qref[3], m[3];
      S::bitbox(sq0, sq1, sq2, c, f.off, f.cnt, centre, qref, m);
      if (threadIdx.x == 0) {
        const uint32_t bits = (m[0] + m[1] + m[2]) * (f.cnt - 1);
        LeafInfo li;
        li.off = f.off;
        li.cnt = f.cnt;
        li.centre = centre;
        li.words = (bits + 31) / 32;
        li.lword = c.words;
        li.qref[0] = int32_t(qref[0]);
        li.qref[1] = int32_t(qref[1]);
        li.qref[2] = int32_t(qref[2]);
        li.m = m[0] | (m[1] << 8) | (m[2] << 16);
        li.pad = 0;
        if (leaf_base + c.leaves < a.num_leaves) {
          a.leaf_info[leaf_base + c.leaves] = li;
          c.leaves += 1;
          c.words += li.words;
        } else {
          atomicOr(a.err, kErrInternal);
        }
      }
      __syncthreads();
    } else {
      S::split(sq0, sq1, sq2, sidx, hist, c, f.off, f.cnt, int(f.depth % 3));
      if (threadIdx.x == 0) {
        const uint32_t k = f.cnt >> 1;
        c.stack[c.sp++] = Frame{f.off + k, f.cnt - k, f.depth + 1};  // right, popped second
        c.stack[c.sp++] = Frame{f.off, k, f.depth + 1};              // left, popped first
      }
      __syncthreads();
    }
  }

  // 4. first payload word of this subtree
  if (threadIdx.x == 0) {
    unsigned long long *st = a.state;
    const unsigned long long agg = c.words;
    unsigned long long excl = 0;
    if (s == 0) {
      st_release(&st[0], kFlagP | agg);
    } else {
      st_release(&st[s], kFlagA | agg);
      uint64_t pred = s - 1;
      bool timed_out = false;
      for (;;) {
        unsigned long long v;
        uint32_t spins = 0;
        while (((v = ld_acquire(&st[pred])) >> 62) == 0) {
          if (++spins > kSpinLimit || (ld_relaxed(a.err) & kErrTimeout)) {
            atomicOr(a.err, kErrTimeout);
            timed_out = true;
            break;
          }
          __nanosleep(64);
        }
        if (timed_out) break;
        excl += v & kValMask;
        if ((v & ~kValMask) == kFlagP || pred == 0) break;
        --pred;
      }
      st_release(&st[s], kFlagP | ((excl + agg) & kValMask));
    }
    c.word_base = excl;
  }
  __syncthreads();
  const uint64_t base = c.word_base;
  const uint32_t nl = c.leaves;

  // 5a. leaf records
  uint8_t *table = a.out + kHeaderBytes;
  uint32_t *payload = reinterpret_cast<uint32_t *>(a.out + kHeaderBytes + uint64_t(kLeafBytes) * a.num_leaves);
  for (uint32_t L = threadIdx.x; L < nl; L += kThreads) {
    const LeafInfo li = a.leaf_info[leaf_base + L];
    const uint64_t po = off0 + li.off, wo = base + li.lword;
    uint4 *rec = reinterpret_cast<uint4 *>(table + uint64_t(kLeafBytes) * (leaf_base + L));
    rec[0] = make_uint4(uint32_t(po), uint32_t(po >> 32), uint32_t(wo), uint32_t(wo >> 32));
    rec[1] = make_uint4(uint32_t(li.qref[0]), uint32_t(li.qref[1]), uint32_t(li.qref[2]), li.m);
  }
  // 5b. payload, word by word
  for (uint32_t L = 0; L < nl; ++L) {
    const LeafInfo li = a.leaf_info[leaf_base + L];
    if (li.words == 0) continue;
    const uint32_t m0 = li.m & 0xffu, m1 = (li.m >> 8) & 0xffu, m2 = (li.m >> 16) & 0xffu;
    const uint32_t w = m0 + m1 + m2;
    const uint32_t h0 = m0 ? (1u << (m0 - 1)) - 1u : 0u;
    const uint32_t h1 = m1 ? (1u << (m1 - 1)) - 1u : 0u;
    const uint32_t h2 = m2 ? (1u << (m2 - 1)) - 1u : 0u;
    const uint32_t r0 = uint32_t(li.qref[0]), r1 = uint32_t(li.qref[1]), r2 = uint32_t(li.qref[2]);
    const uint32_t last_slot = li.cnt - 2;
    const C *p0 = sq0 + li.off, *p1 = sq1 + li.off, *p2 = sq2 + li.off;
    uint32_t *outw = payload + base + li.lword;
    for (uint32_t j = threadIdx.x; j < li.words; j += kThreads) {
      const uint64_t bit0 = 32ull * j;
      const uint32_t first = uint32_t(bit0 / w);
      uint32_t last = uint32_t((bit0 + 31) / w);
      if (last > last_slot) last = last_slot;
      uint32_t word = 0;
      for (uint32_t sl = first; sl <= last; ++sl) {
        const uint32_t pp = sl < li.centre ? sl : sl + 1;
        const long long b = (long long)sl * w - (long long)bit0;
        if (m0) {
          const uint32_t cd = uint32_t(p0[pp]) - r0 + h0;
          const long long sh = b;
          if (sh >= 0) { if (sh < 32) word |= uint32_t((unsigned long long)cd << sh); }
          else if (-sh < (long long)m0) word |= cd >> (-sh);
        }
        if (m1) {
          const uint32_t cd = uint32_t(p1[pp]) - r1 + h1;
          const long long sh = b + m0;
          if (sh >= 0) { if (sh < 32) word |= uint32_t((unsigned long long)cd << sh); }
          else if (-sh < (long long)m1) word |= cd >> (-sh);
        }
        if (m2) {
          const uint32_t cd = uint32_t(p2[pp]) - r2 + h2;
          const long long sh = b + m0 + m1;
          if (sh >= 0) { if (sh < 32) word |= uint32_t((unsigned long long)cd << sh); }
          else if (-sh < (long long)m2) word |= cd >> (-sh);
        }
      }
      __stcs(outw + j, word);
    }
  }
  // 5c. optional permutation: decoded position -> input index
  if (IDX && a.perm) {
    for (uint32_t L = 0; L < nl; ++L) {
      const LeafInfo li = a.leaf_info[leaf_base + L];
      for (uint32_t i = threadIdx.x; i < li.cnt; i += kThreads) {
        const uint32_t src = i == 0 ? li.centre : (i - 1 < li.centre ? i - 1 : i);
        a.perm[off0 + li.off + i] = sidx[li.off + src];
      }
    }
  }
}

template <typename C, bool IDX, int EMAX>
cudaError_t subtree_dispatch(const SubtreeLaunch &a, cudaStream_t st) {
  constexpr uint32_t cap = uint32_t(EMAX) * kThreads;
  const size_t smem = size_t(cap) * (3 * sizeof(C) + (IDX ? 4 : 0)) + sizeof(uint32_t) * (1u << kDigit);
  cudaError_t e = cudaFuncSetAttribute(k_subtree<C, IDX, EMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem));
  if (e != cudaSuccess) return e;
  const uint64_t roots = 1ull << a.root_level;
  TraceScope ts("k_subtree", st);
  k_subtree<C, IDX, EMAX><<<unsigned(roots), kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

uint32_t subtree_capacity(int code_bytes, bool with_idx) {
  if (code_bytes == 2) return with_idx ? 16u * kThreads : 32u * kThreads;
  return with_idx ? 12u * kThreads : 16u * kThreads;
}

cudaError_t launch_subtree(const SubtreeLaunch &a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  if (a.code_bytes == 2)
    return a.with_idx ? subtree_dispatch<uint16_t, true, 16>(a, st) : subtree_dispatch<uint16_t, false, 32>(a, st);
  return a.with_idx ? subtree_dispatch<uint32_t, true, 12>(a, st) : subtree_dispatch<uint32_t, false, 16>(a, st);
}

}  // namespace pcx
