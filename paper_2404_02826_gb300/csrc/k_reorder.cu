// Reordering for the entropy coder (Sec. 4.2 of arXiv 2404.02826, after
// Fig. 4): the sequences go in increasing order of sum m_d (ties keep their
// order) and the particles of a sequence, its centre first, in increasing
// order of their R-index (ties keep their order).  The R-index joins a
// particle's codes, most significant first, in the order of the axes' entropy
// levels: the entropy of the distribution of m_d over all sequences, lowest
// first; entropies within 1e-9 tie and keep x, y, z (a stable insertion sort).
// Decoding ignores the order, so the stream format does not change.
//
//   k_ro_stats  histograms of m_x, m_y, m_z and of sum m_d; the largest sequence;
//   k_ro_plan   one block: the axis order, the first new index of every sum;
//   k_ro_rank   one block: each sequence's new index (a stable counting sort);
//   k_ro_counts, k_ro_scan, k_ro_records  new first particles (one block scans the
//               counts in the new order) and the records;
//   k_ro_sort   a block per sequence: keys R-index << 32 | position sorted in
//               shared memory (kRadixMin to kRadixMax keys of at most 64 bits:
//               stable radix passes over the R-index, 4 bits each; else
//               bitonic), then the codes and indices moved;
//               longer sequences with 8-byte keys are merge-sorted in global
//               memory (k_ro_big_*: runs of kSmemSort keys sorted in shared
//               memory, then merged pairwise, each key finding its place in the
//               other run by binary search); longer ones with 16-byte keys go
//               to k_ro_sort_big, one block sorting them one after the other.
#include <cstdint>

#include "pc_internal.cuh"
#include "pc_reorder.cuh"

namespace pcx {
namespace {

constexpr int kSums = 94;            // sum of m_d: 0 .. 93
constexpr int kRankThreads = 256;
constexpr uint32_t kSmemSort = 16384;  // keys sorted in shared memory: 8-byte keys (128 KB)
constexpr uint32_t kSmemWide = 8192;   // 16-byte keys (128 KB)
constexpr int kSortThreads = 1024;
constexpr uint32_t kRadixMin = 1000;   // narrow-key sequences of kRadixMin..kRadixMax particles after the centre
constexpr uint32_t kRadixMax = 8192;   // are sorted by radix passes instead of the bitonic network (shorter ones
                                       // sort faster in a warp's registers: 0.67 against 1.82 ms at 2^25, r = 128)
constexpr int kRadixRounds = 8;        // their keys per thread, at most (kRadixMax over 1024 threads)
constexpr uint32_t kRadixTable = 4096; // counters of one pass: 16 digits x rounds x warps <= kRadixMax / 2

struct RoPlan {
  uint32_t hist_m[3][32];
  uint32_t hist_sum[kSums];
  uint32_t start[kSums];
  uint32_t max_cnt;
  uint32_t nbig;   // sequences left to k_ro_sort_big (16-byte keys)
  uint32_t nbign;  // sequences left to the k_ro_big_* merge sort (8-byte keys)
  int32_t order[3];
  unsigned long long big_keys, big_runs;  // keys and runs of the merge sort
};

inline uint64_t align256(uint64_t x) { return (x + 255) / 256 * 256; }

struct RoLayout {
  uint64_t plan, seq_at, off, big_list, big_list_n, kbase, rbase, keys_a, keys_b, big, total;
};
constexpr int kScanThreads = 1024;

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

RoLayout ro_layout(uint64_t n, uint64_t num_seq, uint64_t max_cnt) {
  RoLayout L = {};
  uint64_t o = 0;
  L.plan = o;
  o = align256(o + sizeof(RoPlan));
  L.seq_at = o;
  o = align256(o + 4 * (num_seq ? num_seq : 1));
  L.off = o;
  o = align256(o + 4 * (num_seq ? num_seq : 1));
  L.big_list = o;  // [num_seq] 16-byte-key sequences, then [num_seq] 8-byte-key ones
  o = align256(o + 8 * (num_seq ? num_seq : 1));
  L.big_list_n = L.big_list;
  L.kbase = o;  // first key of each merge-sorted sequence, then its first run (u64 each, one more than sequences)
  o = align256(o + 8 * (num_seq + 1));
  L.rbase = o;
  o = align256(o + 8 * (num_seq + 1));
  const uint64_t merge_keys = max_cnt > kSmemSort + 1 ? n : 1;  // the merge-sorted keys, at most all particles
  L.keys_a = o;
  o = align256(o + 8 * merge_keys);
  L.keys_b = o;
  o = align256(o + 8 * merge_keys);
  L.big = o;  // global keys of a 16-byte-key sequence too long for shared memory
  const uint64_t big = max_cnt > kSmemWide + 1 ? next_pow2(max_cnt - 1) : 1;
  o = align256(o + 16 * big);
  L.total = o;
  return L;
}

__device__ __forceinline__ uint32_t m_of(const LeafRec &r, int d) { return (r.m >> (8 * d)) & 0xffu; }
__device__ __forceinline__ uint32_t msum(const LeafRec &r) { return m_of(r, 0) + m_of(r, 1) + m_of(r, 2); }
// Bits of a position within the sequence (positions < cnt).
__device__ __forceinline__ uint32_t pos_bits(uint32_t cnt) {
  uint32_t b = 1;
  while ((1u << b) < cnt) ++b;
  return b;
}
// Do the R-index and the position fit one 64-bit key?
__device__ __forceinline__ bool narrow_keys(const LeafRec &r) { return msum(r) + pos_bits(r.cnt) <= 64; }
// Sorted by k_ro_sort (shared memory) rather than k_ro_sort_big?
__device__ __forceinline__ bool fits_smem(const LeafRec &r, uint32_t cap) {
  const uint32_t L = r.cnt - 1;
  return narrow_keys(r) ? L <= cap : L <= (cap < kSmemWide ? cap : kSmemWide);
}

__global__ void k_ro_stats(const LeafRec *__restrict__ recs, uint64_t num_seq, RoPlan *plan) {
  __shared__ uint32_t hm[3][32], hs[kSums];
  for (int i = threadIdx.x; i < 96; i += blockDim.x) hm[i / 32][i % 32] = 0;
  for (int i = threadIdx.x; i < kSums; i += blockDim.x) hs[i] = 0;
  __syncthreads();
  uint32_t mx = 0;
  for (uint64_t s = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < num_seq; s += uint64_t(gridDim.x) * blockDim.x) {
    const LeafRec r = recs[s];
    for (int d = 0; d < 3; ++d) atomicAdd(&hm[d][m_of(r, d) & 31], 1u);
    atomicAdd(&hs[msum(r)], 1u);
    mx = max(mx, r.cnt);
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if ((threadIdx.x & 31) == 0) atomicMax(&plan->max_cnt, mx);
  __syncthreads();
  for (int i = threadIdx.x; i < 96; i += blockDim.x)
    if (hm[i / 32][i % 32]) atomicAdd(&plan->hist_m[i / 32][i % 32], hm[i / 32][i % 32]);
  for (int i = threadIdx.x; i < kSums; i += blockDim.x)
    if (hs[i]) atomicAdd(&plan->hist_sum[i], hs[i]);
}

__global__ void k_ro_plan(RoPlan *plan, uint64_t num_seq) {
  if (threadIdx.x != 0) return;
  double ent[3];
  for (int d = 0; d < 3; ++d) {
    double h = 0.0;
    for (int v = 0; v < 32; ++v) {
      const uint32_t c = plan->hist_m[d][v];
      if (c) {
        const double p = double(c) / double(num_seq);
        h -= p * log2(p);
      }
    }
    ent[d] = h;
  }
  int order[3] = {0, 1, 2};
  for (int i = 1; i < 3; ++i)
    for (int j = i; j > 0 && ent[order[j]] < ent[order[j - 1]] - 1e-9; --j) {
      const int t = order[j];
      order[j] = order[j - 1];
      order[j - 1] = t;
    }
  for (int d = 0; d < 3; ++d) plan->order[d] = order[d];
  uint32_t run = 0;
  for (int k = 0; k < kSums; ++k) {
    plan->start[k] = run;
    run += plan->hist_sum[k];
  }
}

// New index of every sequence: the first index of its sum plus the sequences
// of the same sum before it.  Thread t owns a contiguous range; cnt[k][t]
// counts its sequences of sum k, then becomes its first index of sum k.
__global__ void __launch_bounds__(kRankThreads) k_ro_rank(const LeafRec *__restrict__ recs, uint64_t num_seq,
                                                          const RoPlan *plan, uint32_t *seq_at) {
  extern __shared__ uint32_t cnt[];  // [kSums][kRankThreads]
  const uint32_t t = threadIdx.x;
  for (uint32_t i = t; i < uint32_t(kSums) * kRankThreads; i += kRankThreads) cnt[i] = 0;
  __syncthreads();
  const uint64_t per = (num_seq + kRankThreads - 1) / kRankThreads;
  const uint64_t s0 = min(num_seq, t * per), s1 = min(num_seq, s0 + per);
  for (uint64_t s = s0; s < s1; ++s) ++cnt[msum(recs[s]) * kRankThreads + t];
  __syncthreads();
  if (t < uint32_t(kSums)) {
    uint32_t run = plan->start[t];
    for (uint32_t u = 0; u < kRankThreads; ++u) {
      const uint32_t x = cnt[t * kRankThreads + u];
      cnt[t * kRankThreads + u] = run;
      run += x;
    }
  }
  __syncthreads();
  for (uint64_t s = s0; s < s1; ++s) seq_at[cnt[msum(recs[s]) * kRankThreads + t]++] = uint32_t(s);
}

// Counts in the new order (into off), then their exclusive scan by one block
// over contiguous ranges, then the records.
__global__ void k_ro_counts(const LeafRec *__restrict__ recs, uint64_t num_seq, const uint32_t *__restrict__ seq_at,
                            uint32_t *off) {
  for (uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < num_seq; j += uint64_t(gridDim.x) * blockDim.x)
    off[j] = recs[seq_at[j]].cnt;
}

__global__ void __launch_bounds__(kScanThreads) k_ro_scan(uint64_t num_seq, uint32_t *off) {
  __shared__ uint32_t ws[32];
  const uint64_t per = (num_seq + kScanThreads - 1) / kScanThreads;
  const uint64_t j0 = min(num_seq, threadIdx.x * per), j1 = min(num_seq, j0 + per);
  uint32_t sum = 0;
  for (uint64_t j = j0; j < j1; ++j) sum += off[j];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t x = ws[lane];
    uint32_t xi = x;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += y;
    }
    ws[lane] = xi - x;
  }
  __syncthreads();
  uint32_t run = ws[warp] + incl - sum;
  for (uint64_t j = j0; j < j1; ++j) {
    const uint32_t x = off[j];
    off[j] = run;
    run += x;
  }
}

__global__ void k_ro_records(const LeafRec *__restrict__ recs, uint64_t num_seq, const uint32_t *__restrict__ seq_at,
                             const uint32_t *__restrict__ off, LeafRec *out_recs) {
  for (uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < num_seq;
       j += uint64_t(gridDim.x) * blockDim.x) {
    LeafRec r = recs[seq_at[j]];
    r.off = off[j];
    r.centre = 0;
    r.words = uint32_t((uint64_t(msum(r)) * (r.cnt - 1) + 31) >> 5);
    r.word_off = 0;
    out_recs[j] = r;
  }
}

// 128-bit key of the particle at position p of a sequence: its R-index
// (codes c_d = q_d - q_ref_d + 2^(m_d-1) - 1, joined in the axis order, up to
// 93 bits) shifted left by 32, position p in the low 32 bits.
__device__ __forceinline__ void rkey(const uint32_t q[3], const LeafRec &r, const int32_t order[3], uint32_t p,
                                     unsigned long long &hi, unsigned long long &lo) {
  unsigned long long h = 0, l = 0;
  for (int k = 0; k < 3; ++k) {
    const int d = order[k];
    const uint32_t m = m_of(r, d);
    const uint32_t c = m ? q[d] - uint32_t(r.qref[d]) + ((1u << (m - 1)) - 1u) : 0u;
    if (m) {
      h = (h << m) | (l >> (64 - m));  // m <= 31
      l <<= m;
    }
    l |= c;
  }
  hi = (h << 32) | (l >> 32);
  lo = (l << 32) | p;
}

template <typename C>
__device__ __forceinline__ void load_q(const C *q0, const C *q1, const C *q2, uint64_t i, uint32_t q[3]) {
  q[0] = uint32_t(q0[i]);
  q[1] = uint32_t(q1[i]);
  q[2] = uint32_t(q2[i]);
}

// Bitonic sort of P keys (a power of two) held in kh/kl by the block.
__device__ __forceinline__ void block_bitonic(unsigned long long *kh, unsigned long long *kl, uint32_t P) {
  for (uint32_t k = 2; k <= P; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < P / 2; i += blockDim.x) {
        const uint32_t a = 2 * j * (i / j) + (i % j), b = a + j;  // pairs (a, a + j) with bit j of a clear
        const bool up = (a & k) == 0;
        const unsigned long long ah = kh[a], al = kl[a], bh = kh[b], bl = kl[b];
        const bool gt = ah > bh || (ah == bh && al > bl);
        if (gt == up) {
          kh[a] = bh;
          kl[a] = bl;
          kh[b] = ah;
          kl[b] = al;
        }
      }
      __syncthreads();
    }
}

// The same on 64-bit keys.
__device__ __forceinline__ void block_bitonic64(unsigned long long *k64, uint32_t P) {
  for (uint32_t k = 2; k <= P; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < P / 2; i += blockDim.x) {
        const uint32_t a = 2 * j * (i / j) + (i % j), b = a + j;
        const bool up = (a & k) == 0;
        const unsigned long long x = k64[a], y = k64[b];
        if ((x > y) == up) {
          k64[a] = y;
          k64[b] = x;
        }
      }
      __syncthreads();
    }
}

// Bitonic sort of P 64-bit keys (a power of two), E per thread in registers:
// thread t holds keys tE .. tE + E - 1.  Partners within a thread are compared
// in registers, partners within a warp through shuffles, the rest through
// shared memory `sm` (P keys).  Every thread of the block takes part.
template <int E, int J>
__device__ __forceinline__ void reg_stage(unsigned long long (&v)[E], uint32_t base, uint32_t k) {
#pragma unroll
  for (int i = 0; i < E; ++i) {
    if (i & J) continue;
    const bool up = ((base + uint32_t(i)) & k) == 0;
    const unsigned long long a = v[i], b = v[i + J];
    if ((a > b) == up) {
      v[i] = b;
      v[i + J] = a;
    }
  }
}

template <int E>
__device__ __forceinline__ void keep(unsigned long long (&v)[E], uint32_t base, uint32_t k, uint32_t j,
                                     const unsigned long long *o) {
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const uint32_t e = base + uint32_t(i);
    const bool keep_min = ((e & j) == 0) == ((e & k) == 0);
    v[i] = keep_min ? (o[i] < v[i] ? o[i] : v[i]) : (o[i] > v[i] ? o[i] : v[i]);
  }
}

template <int E>
__device__ void bitonic_regs(unsigned long long (&v)[E], uint32_t P, unsigned long long *sm) {
  const uint32_t base = threadIdx.x * E;
  for (uint32_t k = 2; k <= P; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      unsigned long long o[E];
      if (j >= 32u * E) {  // partner in another warp
        __syncthreads();
#pragma unroll
        for (int i = 0; i < E; ++i) sm[base + i] = v[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < E; ++i) o[i] = ((base + i) ^ j) < P ? sm[(base + i) ^ j] : v[i];
        keep(v, base, k, j, o);
      } else if (j >= uint32_t(E)) {  // partner in another lane of this warp
#pragma unroll
        for (int i = 0; i < E; ++i) o[i] = __shfl_xor_sync(0xffffffffu, v[i], j / E);
        keep(v, base, k, j, o);
      } else if (j == 4) {
        if (E > 4) reg_stage<E, (E > 4 ? 4 : 1)>(v, base, k);
      } else if (j == 2) {
        reg_stage<E, 2>(v, base, k);
      } else {
        reg_stage<E, 1>(v, base, k);
      }
    }
}

// Exclusive scan of n counters in shared memory by the whole block
// (n <= 4 * blockDim.x, blockDim.x a multiple of 32); wsum: 32 words.
__device__ __forceinline__ void block_scan_excl(uint32_t *c, uint32_t n, uint32_t *wsum) {
  const uint32_t T = blockDim.x, per = (n + T - 1) / T, lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t b = threadIdx.x * per, W = T >> 5;
  uint32_t v[4], sum = 0;
#pragma unroll
  for (uint32_t i = 0; i < 4; ++i) {
    v[i] = (i < per && b + i < n) ? c[b + i] : 0u;
    sum += v[i];
  }
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= uint32_t(o)) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t t = lane < W ? wsum[lane] : 0u;
    uint32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= uint32_t(o)) ti += y;
    }
    if (lane < W) wsum[lane] = ti - t;
  }
  __syncthreads();
  uint32_t run = wsum[warp] + inc - sum;
#pragma unroll
  for (uint32_t i = 0; i < 4; ++i)
    if (i < per && b + i < n) {
      c[b + i] = run;
      run += v[i];
    }
  __syncthreads();
}

// Stable LSD radix sort of the L narrow keys in a (R-index << pbits | position,
// in position order) by their R-index bits, 4 bits per pass; b is scratch of L
// keys, tab kRadixTable counters, wsum 32 words.  Equal R-indices keep their
// order, so the result is the keys' ascending order.  Round k of the block
// takes keys k * T + t; a key's place is the count of keys before it in
// (digit, round, warp, lane) order: its rank among its warp's equal digits
// (match_any) plus the scanned counter of (digit, round, warp).  Returns the
// array holding the sorted keys.
__device__ unsigned long long *radix_narrow(unsigned long long *a, unsigned long long *b, uint32_t *tab,
                                            uint32_t *wsum, uint32_t L, uint32_t pbits, uint32_t rbits) {
  const uint32_t T = blockDim.x, W = T >> 5, K = (L + T - 1) / T;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, lt = (1u << lane) - 1u;
  const uint32_t n = 16u * K * W;
  for (uint32_t sh = pbits; sh < pbits + rbits; sh += 4) {
    uint32_t dig[kRadixRounds], rank[kRadixRounds];
    for (uint32_t i = threadIdx.x; i < n; i += T) tab[i] = 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRadixRounds; ++k) {
      dig[k] = 16u;
      rank[k] = 0;
      if (uint32_t(k) < K) {  // block-uniform: every lane of a warp takes part in the match
        const uint32_t e = uint32_t(k) * T + threadIdx.x;
        const uint32_t d = e < L ? uint32_t(a[e] >> sh) & 15u : 16u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        dig[k] = d;
        rank[k] = __popc(peers & lt);
        if (d < 16u && (peers & lt) == 0) tab[(d * K + uint32_t(k)) * W + warp] = __popc(peers);
      }
    }
    __syncthreads();
    block_scan_excl(tab, n, wsum);
#pragma unroll
    for (int k = 0; k < kRadixRounds; ++k)
      if (dig[k] < 16u) b[tab[(dig[k] * K + uint32_t(k)) * W + warp] + rank[k]] = a[uint32_t(k) * T + threadIdx.x];
    __syncthreads();
    unsigned long long *t = a;
    a = b;
    b = t;
  }
  return a;
}

// Narrow keys of one sequence (P of them, a power of two, P <= E * blockDim)
// sorted with bitonic_regs; the sorted keys end in sm[0 .. P).
template <int E, typename C>
__device__ void sort_narrow(const LeafRec &r, uint32_t P, uint32_t pbits, const int32_t order[3], const C *q0,
                            const C *q1, const C *q2, unsigned long long *sm) {
  const uint32_t L = r.cnt - 1;
  unsigned long long v[E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const uint32_t e = threadIdx.x * E + i;
    v[i] = ~0ull;
    if (e < L) {
      const uint32_t p = e < r.centre ? e : e + 1;
      uint32_t q[3];
      load_q(q0, q1, q2, uint64_t(r.off) + p, q);
      unsigned long long h, l;
      rkey(q, r, order, p, h, l);
      v[i] = (((h << 32) | (l >> 32)) << pbits) | p;
    }
  }
  bitonic_regs<E>(v, P, sm);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < E; ++i)
    if (threadIdx.x * E + i < P) sm[threadIdx.x * E + i] = v[i];
  __syncthreads();
}

// The same for more keys than the block's registers hold: all in shared memory.
template <typename C>
__device__ void sort_narrow_smem(const LeafRec &r, uint32_t P, uint32_t pbits, const int32_t order[3], const C *q0,
                                 const C *q1, const C *q2, unsigned long long *sm) {
  const uint32_t L = r.cnt - 1;
  for (uint32_t e = threadIdx.x; e < P; e += blockDim.x) {
    unsigned long long v = ~0ull;
    if (e < L) {
      const uint32_t p = e < r.centre ? e : e + 1;
      uint32_t q[3];
      load_q(q0, q1, q2, uint64_t(r.off) + p, q);
      unsigned long long h, l;
      rkey(q, r, order, p, h, l);
      v = (((h << 32) | (l >> 32)) << pbits) | p;
    }
    sm[e] = v;
  }
  __syncthreads();
  block_bitonic64(sm, P);
}

// Sorts sequence j's keys in kh/kl (capacity P) and moves its particles.  When
// the R-index and the position fit in 64 bits together (sum m_d + bits of the
// count <= 64) the keys are R-index << pbits | position in kl alone.
template <typename C, bool IDX>
__device__ void sort_one(const LeafRec &r, uint32_t dst, const int32_t order[3], const C *q0, const C *q1,
                         const C *q2, const uint32_t *idx, C *o0, C *o1, C *o2, uint32_t *oidx,
                         unsigned long long *kh, unsigned long long *kl, uint32_t P) {
  const uint32_t L = r.cnt - 1;  // particles after the centre
  uint32_t pbits = 1;
  while ((1u << pbits) < r.cnt) ++pbits;  // positions < cnt
  const bool narrow = msum(r) + pbits <= 64;
  const unsigned long long pmask = narrow ? (1ull << pbits) - 1 : 0xffffffffull;
  for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
    if (i < L) {
      const uint32_t p = i < r.centre ? i : i + 1;  // position in the sequence, the centre skipped
      uint32_t q[3];
      load_q(q0, q1, q2, uint64_t(r.off) + p, q);
      unsigned long long h, l;
      rkey(q, r, order, p, h, l);
      if (narrow) {
        kl[i] = (((h << 32) | (l >> 32)) << pbits) | p;  // the R-index has at most 64 - pbits bits
      } else {
        kh[i] = h;
        kl[i] = l;
      }
    } else {
      kh[i] = ~0ull;
      kl[i] = ~0ull;
    }
  }
  __syncthreads();
  if (narrow)
    block_bitonic64(kl, P);
  else
    block_bitonic(kh, kl, P);
  for (uint32_t i = threadIdx.x; i <= L; i += blockDim.x) {
    const uint32_t p = i == 0 ? r.centre : uint32_t(kl[i - 1] & pmask);
    const uint64_t src = uint64_t(r.off) + p, d = uint64_t(dst) + i;
    o0[d] = q0[src];
    o1[d] = q1[src];
    o2[d] = q2[src];
    if (IDX) oidx[d] = idx[src];
  }
  __syncthreads();
}

template <typename C, bool IDX, int E>
__global__ void __launch_bounds__(kSortThreads) k_ro_sort(const LeafRec *__restrict__ recs, uint64_t num_seq,
                                                          const uint32_t *__restrict__ seq_at,
                                                          const uint32_t *__restrict__ off, const RoPlan *plan,
                                                          const C *q0, const C *q1, const C *q2, const uint32_t *idx,
                                                          C *o0, C *o1, C *o2, uint32_t *oidx, uint32_t cap,
                                                          RoPlan *wplan, uint32_t *big_list) {
  extern __shared__ unsigned long long keys[];
  // the radix passes: keys and scratch of rcap keys each, then their counters
  const uint32_t rcap = cap < kRadixMax ? cap : kRadixMax;
  uint32_t *const rtab = reinterpret_cast<uint32_t *>(keys + 2 * rcap);
  uint32_t *const rwsum = rtab + kRadixTable;
  const int32_t order[3] = {plan->order[0], plan->order[1], plan->order[2]};
  for (uint64_t j = blockIdx.x; j < num_seq; j += gridDim.x) {
    const LeafRec r = recs[seq_at[j]];
    const uint32_t L = r.cnt - 1;
    if (!fits_smem(r, cap)) {  // left to the merge sort or to k_ro_sort_big
      if (threadIdx.x == 0) {
        if (narrow_keys(r))
          big_list[num_seq + atomicAdd(&wplan->nbign, 1u)] = uint32_t(j);
        else
          big_list[atomicAdd(&wplan->nbig, 1u)] = uint32_t(j);
      }
      continue;
    }
    uint32_t P = 1;
    while (P < L) P <<= 1;
    const uint32_t pbits = pos_bits(r.cnt);
    if (narrow_keys(r)) {
      const unsigned long long *sorted = keys;
      if (L >= kRadixMin && L <= rcap) {
        // radix passes over the R-index bits
        for (uint32_t e = threadIdx.x; e < L; e += blockDim.x) {
          const uint32_t p = e < r.centre ? e : e + 1;
          uint32_t q[3];
          load_q(q0, q1, q2, uint64_t(r.off) + p, q);
          unsigned long long h, l;
          rkey(q, r, order, p, h, l);
          keys[e] = (((h << 32) | (l >> 32)) << pbits) | p;
        }
        __syncthreads();
        sorted = radix_narrow(keys, keys + rcap, rtab, rwsum, L, pbits, msum(r));
      } else {
        // narrow keys: in registers (padded to a warp's worth at least), or all in shared memory
        const uint32_t Pw = P < 32u * E ? 32u * E : P;
        if (Pw <= E * blockDim.x)
          sort_narrow<E, C>(r, Pw, pbits, order, q0, q1, q2, keys);
        else
          sort_narrow_smem<C>(r, P, pbits, order, q0, q1, q2, keys);
      }
      const unsigned long long pmask = (1ull << pbits) - 1;
      const uint32_t dst = off[j];
      for (uint32_t i = threadIdx.x; i <= L; i += blockDim.x) {
        const uint32_t p = i == 0 ? r.centre : uint32_t(sorted[i - 1] & pmask);
        const uint64_t src = uint64_t(r.off) + p, d = uint64_t(dst) + i;
        o0[d] = q0[src];
        o1[d] = q1[src];
        o2[d] = q2[src];
        if (IDX) oidx[d] = idx[src];
      }
      __syncthreads();
    } else {
      const uint32_t capw = cap < kSmemWide ? cap : kSmemWide;
      sort_one<C, IDX>(r, off[j], order, q0, q1, q2, idx, o0, o1, o2, oidx, keys, keys + capw, P);
    }
  }
}

template <typename C, bool IDX>
__global__ void __launch_bounds__(kSortThreads) k_ro_sort_big(const LeafRec *__restrict__ recs, uint64_t num_seq,
                                                              const uint32_t *__restrict__ seq_at,
                                                              const uint32_t *__restrict__ off, const RoPlan *plan,
                                                              const C *q0, const C *q1, const C *q2,
                                                              const uint32_t *idx, C *o0, C *o1, C *o2, uint32_t *oidx,
                                                              uint32_t cap, unsigned long long *big, uint64_t big_cap,
                                                              const uint32_t *big_list) {
  const int32_t order[3] = {plan->order[0], plan->order[1], plan->order[2]};
  for (uint32_t b = 0; b < plan->nbig; ++b) {
    const uint32_t j = big_list[b];
    const LeafRec r = recs[seq_at[j]];
    const uint32_t L = r.cnt - 1;
    uint32_t P = 1;
    while (P < L) P <<= 1;
    if (P > big_cap) continue;  // sized for the largest sequence: cannot happen
    sort_one<C, IDX>(r, off[j], order, q0, q1, q2, idx, o0, o1, o2, oidx, big, big + big_cap, P);
  }
}

// ---- merge sort of the long sequences with 8-byte keys --------------------

// Index b of the sequence whose range [base[b], base[b + 1]) holds t.
__device__ __forceinline__ uint32_t find_range(const unsigned long long *base, uint32_t count, unsigned long long t) {
  uint32_t lo = 0, hi = count;  // base[lo] <= t < base[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (base[mid] <= t)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// One block: first key and first run of every long sequence.
__global__ void __launch_bounds__(1024) k_ro_big_plan(const LeafRec *__restrict__ recs, const uint32_t *seq_at,
                                                      const uint32_t *list, RoPlan *plan, unsigned long long *kbase,
                                                      unsigned long long *rbase) {
  if (threadIdx.x != 0) return;
  unsigned long long k = 0, r = 0;
  for (uint32_t b = 0; b < plan->nbign; ++b) {
    const uint32_t L = recs[seq_at[list[b]]].cnt - 1;
    kbase[b] = k;
    rbase[b] = r;
    k += L;
    r += (L + kSmemSort - 1) / kSmemSort;
  }
  kbase[plan->nbign] = k;
  rbase[plan->nbign] = r;
  plan->big_keys = k;
  plan->big_runs = r;
}

__global__ void k_ro_big_keys(const LeafRec *__restrict__ recs, const uint32_t *seq_at, const uint32_t *list,
                              const RoPlan *plan, const unsigned long long *kbase, const void *c0, const void *c1,
                              const void *c2, int code_bytes, unsigned long long *keys) {
  const int32_t order[3] = {plan->order[0], plan->order[1], plan->order[2]};
  const unsigned long long T = plan->big_keys;
  for (unsigned long long t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < T;
       t += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t b = find_range(kbase, plan->nbign, t);
    const LeafRec r = recs[seq_at[list[b]]];
    const uint32_t e = uint32_t(t - kbase[b]);
    const uint32_t p = e < r.centre ? e : e + 1;
    uint32_t q[3];
    if (code_bytes == 2)
      load_q(static_cast<const uint16_t *>(c0), static_cast<const uint16_t *>(c1),
             static_cast<const uint16_t *>(c2), uint64_t(r.off) + p, q);
    else
      load_q(static_cast<const uint32_t *>(c0), static_cast<const uint32_t *>(c1),
             static_cast<const uint32_t *>(c2), uint64_t(r.off) + p, q);
    unsigned long long h, l;
    rkey(q, r, order, p, h, l);
    keys[t] = (((h << 32) | (l >> 32)) << pos_bits(r.cnt)) | p;
  }
}

// A block per run of up to kSmemSort keys: sorted in shared memory.
__global__ void __launch_bounds__(kSortThreads) k_ro_big_runs(const LeafRec *__restrict__ recs, const uint32_t *seq_at,
                                                              const uint32_t *list, const RoPlan *plan,
                                                              const unsigned long long *kbase,
                                                              const unsigned long long *rbase,
                                                              unsigned long long *keys) {
  extern __shared__ unsigned long long sm[];
  const unsigned long long R = plan->big_runs;
  for (unsigned long long g = blockIdx.x; g < R; g += gridDim.x) {
    const uint32_t b = find_range(rbase, plan->nbign, g);
    const uint32_t L = recs[seq_at[list[b]]].cnt - 1;
    const uint32_t k0 = uint32_t(g - rbase[b]) * kSmemSort;
    const uint32_t len = min(kSmemSort, L - k0);
    uint32_t P = 1;
    while (P < len) P <<= 1;
    unsigned long long *run = keys + kbase[b] + k0;
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) sm[i] = i < len ? run[i] : ~0ull;
    __syncthreads();
    block_bitonic64(sm, P);
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) run[i] = sm[i];
    __syncthreads();
  }
}

// Runs of w keys merged pairwise into runs of 2w: a key's place is its place
// in its run plus the number of smaller keys in the other run (keys differ).
__global__ void k_ro_big_merge(const LeafRec *__restrict__ recs, const uint32_t *seq_at, const uint32_t *list,
                               const RoPlan *plan, const unsigned long long *kbase, const unsigned long long *in,
                               unsigned long long *out, uint32_t w) {
  const unsigned long long T = plan->big_keys;
  for (unsigned long long t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < T;
       t += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t b = find_range(kbase, plan->nbign, t);
    const uint32_t L = recs[seq_at[list[b]]].cnt - 1;
    const unsigned long long *s = in + kbase[b];
    const uint32_t e = uint32_t(t - kbase[b]);
    const uint32_t r = e / w, start = (r & ~1u) * w;
    const unsigned long long key = s[e];
    // the other run of the pair
    const uint32_t o0 = (r & 1u) ? start : min(L, start + w);
    const uint32_t o1 = (r & 1u) ? start + w : min(L, start + 2 * w);
    uint32_t lo = o0, hi = o1;  // first key >= key in [o0, o1)
    while (lo < hi) {
      const uint32_t mid = (lo + hi) / 2;
      if (s[mid] < key)
        lo = mid + 1;
      else
        hi = mid;
    }
    out[kbase[b] + start + (e - r * w) + (lo - o0)] = key;
  }
}

template <typename C, bool IDX>
__global__ void k_ro_big_write(const LeafRec *__restrict__ recs, const uint32_t *seq_at, const uint32_t *list,
                               const RoPlan *plan, const unsigned long long *kbase, const unsigned long long *keys,
                               const uint32_t *__restrict__ off, const C *q0, const C *q1, const C *q2,
                               const uint32_t *idx, C *o0, C *o1, C *o2, uint32_t *oidx) {
  const unsigned long long T = plan->big_keys;
  for (unsigned long long t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < T;
       t += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t b = find_range(kbase, plan->nbign, t);
    const uint32_t j = list[b];
    const LeafRec r = recs[seq_at[j]];
    const uint32_t e = uint32_t(t - kbase[b]);
    const uint32_t p = uint32_t(keys[t] & ((1ull << pos_bits(r.cnt)) - 1));
    for (int k = 0; k < (e == 0 ? 2 : 1); ++k) {  // the first key's thread also moves the centre
      const uint32_t src_p = k ? r.centre : p;
      const uint64_t src = uint64_t(r.off) + src_p, d = uint64_t(off[j]) + (k ? 0 : e + 1);
      o0[d] = q0[src];
      o1[d] = q1[src];
      o2[d] = q2[src];
      if (IDX) oidx[d] = idx[src];
    }
  }
}

template <typename C, bool IDX>
cudaError_t reorder_dispatch(const ReorderLaunch &a, cudaStream_t st) {
  const RoLayout L = ro_layout(a.n, a.num_seq, a.max_cnt);
  uint8_t *base = static_cast<uint8_t *>(a.scratch);
  RoPlan *plan = reinterpret_cast<RoPlan *>(base + L.plan);
  uint32_t *seq_at = reinterpret_cast<uint32_t *>(base + L.seq_at);
  uint32_t *off = reinterpret_cast<uint32_t *>(base + L.off);
  const C *q0 = static_cast<const C *>(a.codes[0]), *q1 = static_cast<const C *>(a.codes[1]),
          *q2 = static_cast<const C *>(a.codes[2]);
  C *o0 = static_cast<C *>(a.out_codes[0]), *o1 = static_cast<C *>(a.out_codes[1]),
    *o2 = static_cast<C *>(a.out_codes[2]);
  cudaError_t e = cudaMemsetAsync(plan, 0, sizeof(RoPlan), st);
  if (e != cudaSuccess) return e;
  const uint32_t sms = uint32_t(device_sm_count());
  {
    TraceScope ts("k_ro_stats", st);
    const uint64_t blocks = (a.num_seq + 255) / 256;
    k_ro_stats<<<unsigned(blocks < 4ull * sms ? blocks : 4ull * sms), 256, 0, st>>>(a.recs, a.num_seq, plan);
  }
  {
    TraceScope ts("k_ro_plan", st);
    k_ro_plan<<<1, 32, 0, st>>>(plan, a.num_seq);
  }
  uint32_t max_cnt = 0;
  e = read_back(&max_cnt, &plan->max_cnt, 4, st);
  if (e != cudaSuccess) return e;
  {
    TraceScope ts("k_ro_rank", st);
    const size_t smem = size_t(kSums) * kRankThreads * 4;
    e = cudaFuncSetAttribute(k_ro_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_ro_rank<<<1, kRankThreads, smem, st>>>(a.recs, a.num_seq, plan, seq_at);
  }
  {
    TraceScope ts("k_ro_offsets", st);
    const uint64_t blocks = (a.num_seq + 255) / 256;
    const unsigned grid = unsigned(blocks < 8ull * sms ? blocks : 8ull * sms);
    k_ro_counts<<<grid, 256, 0, st>>>(a.recs, a.num_seq, seq_at, off);
    k_ro_scan<<<1, kScanThreads, 0, st>>>(a.num_seq, off);
    k_ro_records<<<grid, 256, 0, st>>>(a.recs, a.num_seq, seq_at, off, a.out_recs);
  }
  // shared-memory keys for the sequences up to kSmemSort particles after the centre
  uint32_t cap = 1;
  const uint32_t longest = max_cnt ? max_cnt - 1 : 0;
  while (cap < (longest < kSmemSort ? longest : kSmemSort)) cap <<= 1;
  {
    TraceScope ts("k_ro_sort", st);
    // E keys per thread in registers: cap / E threads (a warp at least, 1024 at most), 4 keys below 2048,
    // 8 from there; shared memory for 8-byte keys up to cap and 16-byte keys up to kSmemWide
    const uint32_t c2 = cap < 256 ? 256 : cap;
    size_t smem = size_t(c2) * 8 > size_t(c2 < kSmemWide ? c2 : kSmemWide) * 16
                      ? size_t(c2) * 8
                      : size_t(c2 < kSmemWide ? c2 : kSmemWide) * 16;
    // the radix passes' keys, scratch and counters, when a sequence can take them
    const size_t radix = size_t(c2 < kRadixMax ? c2 : kRadixMax) * 16 + 4 * (kRadixTable + 32);
    if (c2 >= kRadixMin && radix > smem) smem = radix;
    const bool wide = cap >= 2048;
    const uint32_t tpc = cap / (wide ? 8 : 4);
    const int threads = int(tpc < 32 ? 32 : (tpc > uint32_t(kSortThreads) ? kSortThreads : tpc));
    auto kern = wide ? k_ro_sort<C, IDX, 8> : k_ro_sort<C, IDX, 4>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const uint64_t grid = uint64_t(per_sm) * sms;
    kern<<<unsigned(a.num_seq < grid ? a.num_seq : grid), threads, smem, st>>>(
        a.recs, a.num_seq, seq_at, off, plan, q0, q1, q2, a.idx, o0, o1, o2, a.out_idx, c2, plan,
        reinterpret_cast<uint32_t *>(base + L.big_list));
  }
  if (longest > kSmemSort) {  // the merge sort of long sequences with 8-byte keys, if any
    const uint32_t *list = reinterpret_cast<const uint32_t *>(base + L.big_list) + a.num_seq;
    auto *kbase = reinterpret_cast<unsigned long long *>(base + L.kbase);
    auto *rbase = reinterpret_cast<unsigned long long *>(base + L.rbase);
    auto *ka = reinterpret_cast<unsigned long long *>(base + L.keys_a);
    auto *kb = reinterpret_cast<unsigned long long *>(base + L.keys_b);
    if (L.keys_b - L.keys_a < 8 * a.n) return cudaErrorInvalidValue;  // the scratch bound was too small
    TraceScope ts("k_ro_big", st);
    const unsigned grid = 8 * sms;
    k_ro_big_plan<<<1, 32, 0, st>>>(a.recs, seq_at, list, plan, kbase, rbase);
    k_ro_big_keys<<<grid, 256, 0, st>>>(a.recs, seq_at, list, plan, kbase, a.codes[0], a.codes[1], a.codes[2],
                                        a.code_bytes, ka);
    const size_t smem = size_t(kSmemSort) * 8;
    e = cudaFuncSetAttribute(k_ro_big_runs, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_ro_big_runs<<<2 * sms, kSortThreads, smem, st>>>(a.recs, seq_at, list, plan, kbase, rbase, ka);
    for (uint64_t w = kSmemSort; w < longest; w *= 2) {
      k_ro_big_merge<<<grid, 256, 0, st>>>(a.recs, seq_at, list, plan, kbase, ka, kb, uint32_t(w));
      auto *t = ka;
      ka = kb;
      kb = t;
    }
    k_ro_big_write<C, IDX><<<grid, 256, 0, st>>>(a.recs, seq_at, list, plan, kbase, ka, off, q0, q1, q2, a.idx, o0,
                                                 o1, o2, a.out_idx);
  }
  if (longest > kSmemWide) {  // 16-byte-key sequences left to the global-memory bitonic sort, if any
    cap = cap < 256 ? 256 : cap;
    const uint64_t big_cap = next_pow2(longest);
    if (L.total - L.big < 16 * big_cap) return cudaErrorInvalidValue;  // the scratch bound was too small
    TraceScope ts("k_ro_sort_big", st);
    k_ro_sort_big<C, IDX><<<1, kSortThreads, 0, st>>>(a.recs, a.num_seq, seq_at, off, plan, q0, q1, q2, a.idx, o0,
                                                     o1, o2, a.out_idx, cap,
                                                     reinterpret_cast<unsigned long long *>(base + L.big), big_cap,
                                                     reinterpret_cast<const uint32_t *>(base + L.big_list));
  }
  return cudaGetLastError();
}

}  // namespace

uint64_t reorder_scratch_bytes(uint64_t n, uint64_t num_seq, uint64_t max_cnt) {
  return ro_layout(n, num_seq, max_cnt).total;
}

cudaError_t launch_reorder(const ReorderLaunch &a, cudaStream_t st) {
  if (a.n == 0 || a.num_seq == 0) return cudaSuccess;
  if (a.code_bytes == 2)
    return a.idx ? reorder_dispatch<uint16_t, true>(a, st) : reorder_dispatch<uint16_t, false>(a, st);
  return a.idx ? reorder_dispatch<uint32_t, true>(a, st) : reorder_dispatch<uint32_t, false>(a, st);
}

}  // namespace pcx
