// Leaves of the k-d partition: bit boxes (Sec. 4.1, Eq. 2) and the packed
// sequences (Sec. 4.2, Fig. 4) of arXiv 2404.02826.
//
// After the last level the codes are stored leaf after leaf, each leaf in
// original-index order.  Four kernels:
//   k_leaftable  the leaf ranges, from the deterministic node sizes;
//   k_leafbox    one CTA per leaf: AABB, the particle closest to the AABB
//                centre (squared distance in doubled lattice units, first in
//                leaf order on ties), R_d and m_d = bit_length(R_d) + 1 (0 for
//                R_d = 0), and the leaf's payload size (sum m)(n - 1) bits;
//   k_leafscan   exclusive scan of the payload words: each leaf's first word;
//   k_leafpack   one CTA per leaf: its 32-byte record, its payload and the
//                optional permutation.  A warp packs 32 consecutive particles
//                at a time; 32 particles of w bits fill exactly w words: each
//                lane shifts its w-bit value to its bit offset (funnel shifts
//                on 32-bit limbs) and ORs the pieces into the warp's words in
//                shared memory, which then go out as whole, contiguous words.
#include <cstdint>

#include "pc_internal.cuh"

namespace pcx {
namespace {

constexpr int kBoxThreads = 256;
constexpr int kPackThreads = 256;
constexpr int kPackWarps = kPackThreads / 32;

__global__ void k_leaftable(uint64_t n, int level, uint32_t r, LeafRec *recs, uint64_t num_leaves) {
  const uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (level < 0) {  // no split at all: one leaf
    if (j == 0 && num_leaves == 1) {
      LeafRec z = {};
      z.off = 0;
      z.cnt = uint32_t(n);
      recs[0] = z;
    }
    return;
  }
  if (j >= (1ull << level)) return;
  uint64_t off, cnt;
  node_range(n, level, j, off, cnt);
  const uint64_t a = n >> level;
  // leaves before this node: 2 per earlier node if every node splits, else
  // one per earlier node plus one per earlier node of the larger size
  const uint64_t base = a > r ? 2 * j : j + (off - j * a);
  LeafRec x = {};
  if (cnt <= r) {
    x.off = uint32_t(off);
    x.cnt = uint32_t(cnt);
    if (base < num_leaves) recs[base] = x;
  } else {
    const uint64_t h = cnt >> 1;
    x.off = uint32_t(off);
    x.cnt = uint32_t(h);
    if (base < num_leaves) recs[base] = x;
    x.off = uint32_t(off + h);
    x.cnt = uint32_t(cnt - h);
    if (base + 1 < num_leaves) recs[base + 1] = x;
  }
}

template <typename C>
struct Vec16;  // codes per 16-byte vector
template <>
struct Vec16<uint16_t> {
  static constexpr int N = 8;
  static __device__ __forceinline__ uint32_t at(const uint4 &w, int i) {
    const uint32_t x = i < 2 ? w.x : (i < 4 ? w.y : (i < 6 ? w.z : w.w));
    return (i & 1) ? (x >> 16) : (x & 0xffffu);
  }
};
template <>
struct Vec16<uint32_t> {
  static constexpr int N = 4;
  static __device__ __forceinline__ uint32_t at(const uint4 &w, int i) {
    return i == 0 ? w.x : (i == 1 ? w.y : (i == 2 ? w.z : w.w));
  }
};

// Calls f(position in leaf, x, y, z) for every particle of [off, off + cnt),
// with 16-byte loads on the aligned body.
template <typename C, typename F>
__device__ __forceinline__ void for_leaf(const C *q0, const C *q1, const C *q2, uint32_t off, uint32_t cnt, F f) {
  constexpr uint32_t kV = Vec16<C>::N;
  const uint32_t a0 = min((off + kV - 1) / kV * kV, off + cnt);
  const uint32_t a1 = max(a0, (off + cnt) / kV * kV);
  for (uint32_t e = off + threadIdx.x; e < a0; e += blockDim.x) f(e - off, uint32_t(q0[e]), uint32_t(q1[e]), uint32_t(q2[e]));
  for (uint32_t e = a1 + threadIdx.x; e < off + cnt; e += blockDim.x)
    f(e - off, uint32_t(q0[e]), uint32_t(q1[e]), uint32_t(q2[e]));
  const uint32_t nv = (a1 - a0) / kV;
  const uint4 *v0 = reinterpret_cast<const uint4 *>(q0 + a0), *v1 = reinterpret_cast<const uint4 *>(q1 + a0),
              *v2 = reinterpret_cast<const uint4 *>(q2 + a0);
  for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) {
    const uint4 x = __ldcg(v0 + i), y = __ldcg(v1 + i), z = __ldcg(v2 + i);
#pragma unroll
    for (int c = 0; c < int(kV); ++c)
      f(a0 - off + i * kV + c, Vec16<C>::at(x, c), Vec16<C>::at(y, c), Vec16<C>::at(z, c));
  }
}

// Widths of a leaf: m_d by Eq. 2, or M on a lossless axis (q_ref_d then 0);
// payload words: (sum m)(n - 1) bits, or (sum widths) * n when the stream has
// lossless axes (every particle, the centre included, is in the payload).
__device__ __forceinline__ void leaf_widths(LeafRec &rec, const uint32_t qc[3], const uint32_t lo[3],
                                            const uint32_t hi[3], uint32_t cnt, uint32_t raw, uint32_t M) {
  uint32_t m[3];
  for (int d = 0; d < 3; ++d) {
    if ((raw >> d) & 1u) {
      m[d] = M;
      rec.qref[d] = 0;
    } else {
      m[d] = bits_for_range(max(qc[d] - lo[d], hi[d] - qc[d]));
      rec.qref[d] = int32_t(qc[d]);
    }
  }
  rec.m = m[0] | (m[1] << 8) | (m[2] << 16);
  const uint64_t w = m[0] + m[1] + m[2];
  rec.words = uint32_t((w * (raw ? uint64_t(cnt) : uint64_t(cnt - 1)) + 31) >> 5);
}

template <typename C>
__global__ void __launch_bounds__(kBoxThreads) k_leafbox(const C *__restrict__ q0, const C *__restrict__ q1,
                                                         const C *__restrict__ q2, LeafRec *recs, uint32_t raw,
                                                         uint32_t M, const uint32_t *err) {
  __shared__ uint32_t red[6][kBoxThreads / 32];
  __shared__ unsigned long long rd[kBoxThreads / 32];
  __shared__ uint32_t rp[kBoxThreads / 32];
  if (call_failed(err)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  LeafRec rec = recs[blockIdx.x];
  const uint32_t off = rec.off, cnt = rec.cnt;
  uint32_t mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0, 0, 0};
  for_leaf(q0, q1, q2, off, cnt, [&](uint32_t, uint32_t x, uint32_t y, uint32_t z) {
    mn[0] = min(mn[0], x);
    mx[0] = max(mx[0], x);
    mn[1] = min(mn[1], y);
    mx[1] = max(mx[1], y);
    mn[2] = min(mn[2], z);
    mx[2] = max(mx[2], z);
  });
  for (int d = 0; d < 3; ++d) {
    mn[d] = __reduce_min_sync(0xffffffffu, mn[d]);
    mx[d] = __reduce_max_sync(0xffffffffu, mx[d]);
    if (lane == 0) {
      red[2 * d][warp] = mn[d];
      red[2 * d + 1][warp] = mx[d];
    }
  }
  __syncthreads();
  uint32_t lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = red[2 * d][0];
    hi[d] = red[2 * d + 1][0];
    for (int w = 1; w < kBoxThreads / 32; ++w) {
      lo[d] = min(lo[d], red[2 * d][w]);
      hi[d] = max(hi[d], red[2 * d + 1][w]);
    }
  }
  // centre: least squared distance to the AABB centre, lowest position on ties
  unsigned long long bd = ~0ull;
  uint32_t bp = 0xffffffffu;
  const long long s0 = (long long)lo[0] + hi[0], s1 = (long long)lo[1] + hi[1], s2 = (long long)lo[2] + hi[2];
  for_leaf(q0, q1, q2, off, cnt, [&](uint32_t p, uint32_t x, uint32_t y, uint32_t z) {
    const long long a = 2ll * x - s0, b = 2ll * y - s1, c = 2ll * z - s2;
    const unsigned long long d2 = (unsigned long long)(a * a) + (unsigned long long)(b * b) + (unsigned long long)(c * c);
    if (d2 < bd || (d2 == bd && p < bp)) {
      bd = d2;
      bp = p;
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
    for (int w = 1; w < kBoxThreads / 32; ++w)
      if (rd[w] < bd || (rd[w] == bd && rp[w] < bp)) {
        bd = rd[w];
        bp = rp[w];
      }
    const uint32_t c = bp;
    const uint32_t qc[3] = {uint32_t(q0[off + c]), uint32_t(q1[off + c]), uint32_t(q2[off + c])};
    rec.centre = c;
    leaf_widths(rec, qc, lo, hi, cnt, raw, M);
    recs[blockIdx.x] = rec;
  }
}

// The same bit box with one warp per leaf (small leaves).  The squared
// distances of the centre search are formed in 32 bits when every side of the
// box is below 2^15 codes (|2q - lo - hi| < 2^15, so the sum of three squares
// stays below 2^32), else in 64; the next leaf's record is loaded while the
// current one is worked.
template <typename C>
__global__ void __launch_bounds__(256) k_leafbox_warp(const C *__restrict__ q0, const C *__restrict__ q1,
                                                      const C *__restrict__ q2, LeafRec *recs, uint64_t num_leaves,
                                                      uint32_t raw, uint32_t M, const uint32_t *err) {
  if (call_failed(err)) return;
  const int lane = threadIdx.x & 31;
  const uint64_t warps = uint64_t(gridDim.x) * 8;
  uint64_t L = uint64_t(blockIdx.x) * 8 + (threadIdx.x >> 5);
  uint4 nx = make_uint4(0u, 0u, 0u, 0u);  // offset and count of the next leaf (the record's first 16 bytes)
  if (L < num_leaves) nx = *reinterpret_cast<const uint4 *>(recs + L);
  for (; L < num_leaves; L += warps) {
    const uint32_t off = nx.x, cnt = nx.y;
    if (L + warps < num_leaves) nx = *reinterpret_cast<const uint4 *>(recs + L + warps);
    uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0, 0, 0};
    for (uint32_t i = lane; i < cnt; i += 32) {
      const uint32_t x[3] = {uint32_t(q0[off + i]), uint32_t(q1[off + i]), uint32_t(q2[off + i])};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        lo[d] = min(lo[d], x[d]);
        hi[d] = max(hi[d], x[d]);
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lo[d] = __reduce_min_sync(0xffffffffu, lo[d]);
      hi[d] = __reduce_max_sync(0xffffffffu, hi[d]);
    }
    // centre: least squared distance to the AABB centre, lowest position on ties
    // (positions rise within a lane: the first minimum is the lowest)
    uint32_t bp = 0xffffffffu;
    if (max(hi[0] - lo[0], max(hi[1] - lo[1], hi[2] - lo[2])) < 32768u) {
      const int s0 = int(lo[0] + hi[0]), s1 = int(lo[1] + hi[1]), s2 = int(lo[2] + hi[2]);
      uint32_t md = 0xffffffffu, mp = 0xffffffffu;
      for (uint32_t i = lane; i < cnt; i += 32) {
        const int e0 = 2 * int(q0[off + i]) - s0, e1 = 2 * int(q1[off + i]) - s1, e2 = 2 * int(q2[off + i]) - s2;
        const uint32_t d2 = uint32_t(e0 * e0) + uint32_t(e1 * e1) + uint32_t(e2 * e2);
        if (d2 < md) {
          md = d2;
          mp = i;
        }
      }
      const uint32_t wmd = __reduce_min_sync(0xffffffffu, md);
      bp = __reduce_min_sync(0xffffffffu, md == wmd ? mp : 0xffffffffu);
    } else {
      unsigned long long bd = ~0ull;
      const long long s0 = (long long)lo[0] + hi[0], s1 = (long long)lo[1] + hi[1], s2 = (long long)lo[2] + hi[2];
      for (uint32_t i = lane; i < cnt; i += 32) {
        const long long a = 2ll * q0[off + i] - s0, b = 2ll * q1[off + i] - s1, c = 2ll * q2[off + i] - s2;
        const unsigned long long d2 =
            (unsigned long long)(a * a) + (unsigned long long)(b * b) + (unsigned long long)(c * c);
        if (d2 < bd) {
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
    }
    if (lane == 0) {
      LeafRec rec = recs[L];
      const uint32_t c = bp;
      const uint32_t qc[3] = {uint32_t(q0[off + c]), uint32_t(q1[off + c]), uint32_t(q2[off + c])};
      rec.centre = c;
      leaf_widths(rec, qc, lo, hi, cnt, raw, M);
      recs[L] = rec;
    }
  }
}

// Payload word offsets over many leaves, in three steps: each block scans its
// slice of leaves (offsets within the slice, slice total), one block scans the
// slice totals, each block adds its slice's base.
constexpr uint32_t kScanSlice = 8192;  // leaves per block

__global__ void __launch_bounds__(1024) k_leafscan_slices(LeafRec *recs, uint64_t num_leaves, uint64_t *slice_tot) {
  __shared__ unsigned long long wt[33];
  const uint64_t s0 = uint64_t(blockIdx.x) * kScanSlice;
  const uint64_t s1 = (s0 + kScanSlice) < num_leaves ? (s0 + kScanSlice) : num_leaves;
  constexpr uint32_t per = kScanSlice / 1024;
  const uint64_t l0 = s0 + uint64_t(threadIdx.x) * per;
  const uint64_t l1 = (l0 + per) < s1 ? (l0 + per) : s1;
  unsigned long long sum = 0;
  for (uint64_t l = l0; l < l1; ++l) sum += recs[l].words;
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
    if (lane == 31) slice_tot[blockIdx.x] = xi;
  }
  __syncthreads();
  unsigned long long run = wt[warp] + incl - sum;
  for (uint64_t l = l0; l < l1; ++l) {
    recs[l].word_off = run;
    run += recs[l].words;
  }
}

__global__ void __launch_bounds__(1024) k_leafscan_totals(uint64_t *slice_tot, uint64_t slices, uint64_t *total_words) {
  // slices <= 1024 * 64: a sequential run per thread, then a block scan
  __shared__ unsigned long long wt[33];
  const uint64_t per = (slices + 1023) / 1024;
  const uint64_t t0 = threadIdx.x * per, t1 = (t0 + per) < slices ? (t0 + per) : slices;
  unsigned long long sum = 0;
  for (uint64_t t = t0; t < t1; ++t) sum += slice_tot[t];
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
    if (lane == 31) *total_words = xi;
  }
  __syncthreads();
  unsigned long long run = wt[warp] + incl - sum;
  for (uint64_t t = t0; t < t1; ++t) {
    const unsigned long long x = slice_tot[t];
    slice_tot[t] = run;
    run += x;
  }
}

__global__ void k_leafscan_add(LeafRec *recs, uint64_t num_leaves, const uint64_t *slice_base) {
  const uint64_t l = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l < num_leaves) recs[l].word_off += slice_base[l / kScanSlice];
}

// Exclusive scan of the leaves' payload words (one block).
__global__ void __launch_bounds__(1024) k_leafscan(LeafRec *recs, uint64_t num_leaves, uint64_t *total_words) {
  __shared__ unsigned long long wt[33];
  const uint64_t per = (num_leaves + blockDim.x - 1) / blockDim.x;
  const uint64_t l0 = threadIdx.x * per, l1 = (l0 + per) < num_leaves ? (l0 + per) : num_leaves;
  unsigned long long sum = 0;
  for (uint64_t l = l0; l < l1; ++l) sum += recs[l].words;
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
    if (lane == 31) wt[32] = xi;
  }
  __syncthreads();
  unsigned long long run = wt[warp] + incl - sum;
  for (uint64_t l = l0; l < l1; ++l) {
    recs[l].word_off = run;
    run += recs[l].words;
  }
  if (threadIdx.x == 0) *total_words = wt[32];
}

// One leaf by a group of `nw` warps (this thread is lane `lane` of warp `warp`
// of the group, thread `tid` of its nw * 32); sw: this warp's 96 staged words.
template <typename C, bool IDX>
__device__ __forceinline__ void pack_leaf(const C *__restrict__ q0, const C *__restrict__ q1, const C *__restrict__ q2,
                                          const uint32_t *__restrict__ idx, const LeafRec &rec, uint64_t leaf,
                                          uint8_t *out, uint64_t num_leaves, uint32_t *perm, int lane, int warp, int nw,
                                          uint32_t *sw, uint64_t n, uint64_t payload_cap, uint32_t *err) {
  const uint32_t tid = uint32_t(warp) * 32 + lane, group = uint32_t(nw) * 32;
  if (uint64_t(rec.off) + rec.cnt > n || rec.word_off + rec.words > payload_cap) {  // inconsistent: never written
    if (tid == 0) atomicOr(err, kErrInternal);
    return;
  }
  const uint32_t off = rec.off, cnt = rec.cnt, centre = rec.centre;
  const uint32_t m0 = rec.m & 0xffu, m1 = (rec.m >> 8) & 0xffu, m2 = (rec.m >> 16) & 0xffu;
  const uint32_t w = m0 + m1 + m2;
  if (tid == 0) {
    uint4 *r = reinterpret_cast<uint4 *>(out + kHeaderBytes + uint64_t(kLeafBytes) * leaf);
    const uint64_t po = off, wo = rec.word_off;
    r[0] = make_uint4(uint32_t(po), uint32_t(po >> 32), uint32_t(wo), uint32_t(wo >> 32));
    r[1] = make_uint4(uint32_t(rec.qref[0]), uint32_t(rec.qref[1]), uint32_t(rec.qref[2]), rec.m);
  }
  if (IDX && perm) {
    for (uint32_t i = tid; i < cnt; i += group) {
      const uint32_t src = i == 0 ? centre : (i - 1 < centre ? i - 1 : i);
      perm[off + i] = idx[off + src];
    }
  }
  if (w == 0 || cnt < 2) return;
  uint32_t *payload = reinterpret_cast<uint32_t *>(out + kHeaderBytes + uint64_t(kLeafBytes) * num_leaves) + rec.word_off;
  const uint32_t h0 = m0 ? (1u << (m0 - 1)) - 1u : 0u;
  const uint32_t h1 = m1 ? (1u << (m1 - 1)) - 1u : 0u;
  const uint32_t h2 = m2 ? (1u << (m2 - 1)) - 1u : 0u;
  const uint32_t r0 = uint32_t(rec.qref[0]), r1 = uint32_t(rec.qref[1]), r2 = uint32_t(rec.qref[2]);
  const uint32_t slots = cnt - 1;
  const uint32_t words = rec.words;
  const uint32_t chunks = (slots + 31) / 32;
  for (uint32_t ch = warp; ch < chunks; ch += nw) {
    // this lane's particle as one w-bit value c_x | c_y << m_x | c_z << (m_x + m_y), in three 32-bit limbs
    const uint32_t s = ch * 32 + lane;
    uint32_t v0 = 0, v1 = 0, v2 = 0;
    if (s < slots) {
      const uint32_t p = off + (s < centre ? s : s + 1);
      const uint32_t cx = m0 ? uint32_t(q0[p]) - r0 + h0 : 0u;
      const uint32_t cy = m1 ? uint32_t(q1[p]) - r1 + h1 : 0u;
      const uint32_t cz = m2 ? uint32_t(q2[p]) - r2 + h2 : 0u;
      const unsigned long long y = (unsigned long long)cy << m0;  // m_x <= 31
      v0 = cx | uint32_t(y);
      v1 = uint32_t(y >> 32);
      const uint32_t s2 = m0 + m1;  // <= 62
      const unsigned long long z = (unsigned long long)cz << (s2 & 31);
      if (s2 < 32) {
        v0 |= uint32_t(z);
        v1 |= uint32_t(z >> 32);
      } else {
        v1 |= uint32_t(z);
        v2 = uint32_t(z >> 32);
      }
    }
    // the 32 values fill exactly w words of this chunk; lane i's value starts at bit i * w
    for (uint32_t t = lane; t < w; t += 32) sw[t] = 0;
    __syncwarp();
    if (s < slots) {
      const uint32_t b = lane * w, k0 = b >> 5, sh = b & 31;
      const uint32_t nw = (sh + w + 31) >> 5;  // words this value touches, <= 4
      atomicOr(&sw[k0], v0 << sh);
      if (nw > 1) atomicOr(&sw[k0 + 1], __funnelshift_l(v0, v1, sh));
      if (nw > 2) atomicOr(&sw[k0 + 2], __funnelshift_l(v1, v2, sh));
      if (nw > 3) atomicOr(&sw[k0 + 3], __funnelshift_l(v2, 0u, sh));
    }
    __syncwarp();
    for (uint32_t t = lane; t < w; t += 32) {
      const uint32_t gw = ch * w + t;
      if (gw < words) __stcs(payload + gw, sw[t]);
    }
    __syncwarp();
  }
}

// One CTA per leaf (large leaves).
template <typename C, bool IDX>
__global__ void __launch_bounds__(kPackThreads) k_leafpack(const C *__restrict__ q0, const C *__restrict__ q1,
                                                           const C *__restrict__ q2, const uint32_t *__restrict__ idx,
                                                           const LeafRec *__restrict__ recs, uint8_t *out,
                                                           uint64_t num_leaves, uint32_t *perm, uint64_t n,
                                                           uint64_t payload_cap, uint32_t *err) {
  __shared__ uint32_t swords[kPackWarps][96];  // one chunk's words per warp (w <= 93)
  if (call_failed(err)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  pack_leaf<C, IDX>(q0, q1, q2, idx, recs[blockIdx.x], blockIdx.x, out, num_leaves, perm, lane, warp, kPackWarps,
                    swords[warp], n, payload_cap, err);
}

// One warp per leaf (small leaves).
template <typename C, bool IDX>
__global__ void __launch_bounds__(kPackThreads) k_leafpack_warp(const C *__restrict__ q0, const C *__restrict__ q1,
                                                                const C *__restrict__ q2,
                                                                const uint32_t *__restrict__ idx,
                                                                const LeafRec *__restrict__ recs, uint8_t *out,
                                                                uint64_t num_leaves, uint32_t *perm, uint64_t n,
                                                                uint64_t payload_cap, uint32_t *err) {
  __shared__ uint32_t swords[kPackWarps][96];
  if (call_failed(err)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t L = uint64_t(blockIdx.x) * kPackWarps + warp; L < num_leaves; L += uint64_t(gridDim.x) * kPackWarps)
    pack_leaf<C, IDX>(q0, q1, q2, idx, recs[L], L, out, num_leaves, perm, lane, 0, 1, swords[warp], n, payload_cap,
                      err);
}

// Packing of a stream with lossless axes (Sec. 4.1, m_d > M), one warp per
// leaf: every particle of the leaf, the centre first, as x, y, z fields of m_d
// bits (coded axes, Fig. 2 codes) or M bits (the coordinate's own bit pattern,
// read through the input index).  32 particles of w bits fill w words: each
// lane assembles its particle's bits (up to 192) and ORs them into the warp's
// staged words, which then go out whole.
template <typename T>
__global__ void __launch_bounds__(kPackThreads) k_leafpack_lossless(
    const uint32_t *__restrict__ q0, const uint32_t *__restrict__ q1, const uint32_t *__restrict__ q2,
    const uint32_t *__restrict__ idx, const LeafRec *__restrict__ recs, uint8_t *out, uint64_t num_leaves,
    uint32_t *perm, uint64_t n, uint64_t payload_cap, uint32_t *err, const T *__restrict__ pos, uint32_t raw) {
  constexpr uint32_t kMaxW = 3 * 8 * sizeof(T);  // widest particle: three lossless axes
  __shared__ uint32_t swords[kPackWarps][kMaxW + 8];
  if (call_failed(err)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *sw = swords[warp];
  const uint32_t *qs[3] = {q0, q1, q2};
  for (uint64_t L = uint64_t(blockIdx.x) * kPackWarps + warp; L < num_leaves; L += uint64_t(gridDim.x) * kPackWarps) {
    const LeafRec rec = recs[L];
    if (uint64_t(rec.off) + rec.cnt > n || rec.word_off + rec.words > payload_cap) {
      if (lane == 0) atomicOr(err, kErrInternal);
      continue;
    }
    const uint32_t off = rec.off, cnt = rec.cnt, centre = rec.centre;
    const uint32_t m[3] = {rec.m & 0xffu, (rec.m >> 8) & 0xffu, (rec.m >> 16) & 0xffu};
    const uint32_t w = m[0] + m[1] + m[2];
    if (lane == 0) {
      uint4 *r = reinterpret_cast<uint4 *>(out + kHeaderBytes + uint64_t(kLeafBytes) * L);
      const uint64_t po = off, wo = rec.word_off;
      r[0] = make_uint4(uint32_t(po), uint32_t(po >> 32), uint32_t(wo), uint32_t(wo >> 32));
      r[1] = make_uint4(uint32_t(rec.qref[0]), uint32_t(rec.qref[1]), uint32_t(rec.qref[2]), rec.m);
    }
    uint32_t *payload =
        reinterpret_cast<uint32_t *>(out + kHeaderBytes + uint64_t(kLeafBytes) * num_leaves) + rec.word_off;
    for (uint32_t c0 = 0; c0 < cnt; c0 += 32) {
      const uint32_t k = c0 + lane;  // payload entry: 0 is the centre, then leaf order without it
      uint32_t lim[kMaxW / 32] = {};
      if (k < cnt) {
        const uint32_t src = k == 0 ? centre : (k - 1 < centre ? k - 1 : k);
        const uint32_t id = idx[off + src];
        if (perm) perm[off + k] = id;
        uint32_t bp = 0;
        for (int d = 0; d < 3; ++d) {
          uint64_t v;
          if ((raw >> d) & 1u) {
            v = sizeof(T) == 4 ? uint64_t(__float_as_uint(float(pos[3 * uint64_t(id) + d])))
                               : uint64_t(__double_as_longlong(double(pos[3 * uint64_t(id) + d])));
          } else if (m[d]) {
            v = uint64_t(qs[d][off + src] - uint32_t(rec.qref[d]) + ((1u << (m[d] - 1)) - 1u));
          } else {
            continue;
          }
          for (uint32_t t = 0; t < m[d]; t += 32) {
            const uint32_t nb = min(32u, m[d] - t);
            uint32_t part = uint32_t(v >> t);
            if (nb < 32) part &= (1u << nb) - 1u;
            const uint32_t wj = bp >> 5, sh = bp & 31;
            lim[wj] |= part << sh;
            if (sh && wj + 1 < kMaxW / 32) lim[wj + 1] |= part >> (32 - sh);
            bp += nb;
          }
        }
      }
      for (uint32_t t = lane; t < w + 8; t += 32) sw[t] = 0;
      __syncwarp();
      if (k < cnt) {
        for (uint32_t j = 0; 32 * j < w; ++j) {
          const uint32_t g = lane * w + 32 * j, k0 = g >> 5, sh = g & 31;
          atomicOr(&sw[k0], lim[j] << sh);
          if (sh) atomicOr(&sw[k0 + 1], lim[j] >> (32 - sh));
        }
      }
      __syncwarp();
      for (uint32_t t = lane; t < w; t += 32) {
        const uint32_t gw = (c0 >> 5) * w + t;
        if (gw < rec.words) __stcs(payload + gw, sw[t]);
      }
      __syncwarp();
    }
  }
}

template <typename C, bool IDX>
cudaError_t leaves_dispatch(const LeafLaunch &a, cudaStream_t st) {
  const C *q0 = static_cast<const C *>(a.codes[0]), *q1 = static_cast<const C *>(a.codes[1]),
          *q2 = static_cast<const C *>(a.codes[2]);
  if (!a.recs_ready) {
    TraceScope ts("k_leaftable", st);
    const uint64_t nodes = a.split_level < 0 ? 1 : (1ull << a.split_level);
    k_leaftable<<<unsigned((nodes + 255) / 256), 256, 0, st>>>(a.n, a.split_level, a.leaf_size, a.recs,
                                                               a.num_leaves);
  }
  // threads per leaf: a CTA for large leaves, a warp for small ones
  const bool small = a.leaf_size <= a.warp_leaf_max;
  const uint64_t warp_blocks = (a.num_leaves + 7) / 8;
  const unsigned wgrid = unsigned(warp_blocks < uint64_t(device_sm_count()) * 32 ? warp_blocks
                                                                                 : uint64_t(device_sm_count()) * 32);
  if (!a.recs_ready) {
    TraceScope ts("k_leafbox", st);
    const uint32_t M = a.dtype == 0 ? 32u : 64u;
    if (small)
      k_leafbox_warp<C><<<wgrid, 256, 0, st>>>(q0, q1, q2, a.recs, a.num_leaves, a.raw, M, a.err);
    else
      k_leafbox<C><<<unsigned(a.num_leaves), kBoxThreads, 0, st>>>(q0, q1, q2, a.recs, a.raw, M, a.err);
  }
  if (a.box_only) return cudaGetLastError();
  {
    TraceScope ts("k_leafscan", st);
    if (a.num_leaves <= kScanSlice) {
      k_leafscan<<<1, 1024, 0, st>>>(a.recs, a.num_leaves, a.total_words);
    } else {
      const uint64_t slices = (a.num_leaves + kScanSlice - 1) / kScanSlice;
      k_leafscan_slices<<<unsigned(slices), 1024, 0, st>>>(a.recs, a.num_leaves, a.slice_tot);
      k_leafscan_totals<<<1, 1024, 0, st>>>(a.slice_tot, slices, a.total_words);
      k_leafscan_add<<<unsigned((a.num_leaves + 255) / 256), 256, 0, st>>>(a.recs, a.num_leaves, a.slice_tot);
    }
  }
  if (a.cost_only) return cudaGetLastError();
  TraceScope ts("k_leafpack", st);
  if (a.raw) {  // lossless axes: u32 codes and the input index are always there
    if (sizeof(C) != 4 || !IDX || !a.pos) return cudaErrorInvalidValue;
    const uint32_t *u0 = reinterpret_cast<const uint32_t *>(q0), *u1 = reinterpret_cast<const uint32_t *>(q1),
                   *u2 = reinterpret_cast<const uint32_t *>(q2);
    if (a.dtype == 0)
      k_leafpack_lossless<float><<<wgrid, kPackThreads, 0, st>>>(u0, u1, u2, a.idx, a.recs, a.out, a.num_leaves,
                                                                  a.perm, a.n, a.payload_cap, a.err,
                                                                  static_cast<const float *>(a.pos), a.raw);
    else
      k_leafpack_lossless<double><<<wgrid, kPackThreads, 0, st>>>(u0, u1, u2, a.idx, a.recs, a.out, a.num_leaves,
                                                                   a.perm, a.n, a.payload_cap, a.err,
                                                                   static_cast<const double *>(a.pos), a.raw);
    return cudaGetLastError();
  }
  if (small)
    k_leafpack_warp<C, IDX><<<wgrid, kPackThreads, 0, st>>>(q0, q1, q2, a.idx, a.recs, a.out, a.num_leaves, a.perm,
                                                            a.n, a.payload_cap, a.err);
  else
    k_leafpack<C, IDX><<<unsigned(a.num_leaves), kPackThreads, 0, st>>>(q0, q1, q2, a.idx, a.recs, a.out,
                                                                        a.num_leaves, a.perm, a.n, a.payload_cap,
                                                                        a.err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_leaftable(uint64_t n, int split_level, uint32_t leaf_size, LeafRec *recs, uint64_t num_leaves,
                             cudaStream_t st) {
  if (n == 0 || num_leaves == 0) return cudaSuccess;
  TraceScope ts("k_leaftable", st);
  const uint64_t nodes = split_level < 0 ? 1 : (1ull << split_level);
  k_leaftable<<<unsigned((nodes + 255) / 256), 256, 0, st>>>(n, split_level, leaf_size, recs, num_leaves);
  return cudaGetLastError();
}

cudaError_t launch_leaves(const LeafLaunch &a, cudaStream_t st) {
  if (a.n == 0 || a.num_leaves == 0) return cudaSuccess;
  if (a.code_bytes == 2)
    return a.idx ? leaves_dispatch<uint16_t, true>(a, st) : leaves_dispatch<uint16_t, false>(a, st);
  return a.idx ? leaves_dispatch<uint32_t, true>(a, st) : leaves_dispatch<uint32_t, false>(a, st);
}

}  // namespace pcx
