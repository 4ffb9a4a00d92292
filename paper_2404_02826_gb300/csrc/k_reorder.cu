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
//               shared memory (bitonic), then the codes and indices moved;
//               sequences too large for shared memory go to k_ro_sort_big, one
//               block sorting them one after the other in global memory.
#include <cstdint>

#include "pc_internal.cuh"
#include "pc_reorder.cuh"

namespace pcx {
namespace {

constexpr int kSums = 94;            // sum of m_d: 0 .. 93
constexpr int kRankThreads = 256;
constexpr uint32_t kSmemSort = 8192;  // keys sorted in shared memory (16 bytes each)
constexpr int kSortThreads = 1024;

struct RoPlan {
  uint32_t hist_m[3][32];
  uint32_t hist_sum[kSums];
  uint32_t start[kSums];
  uint32_t max_cnt;
  int32_t order[3];
};

inline uint64_t align256(uint64_t x) { return (x + 255) / 256 * 256; }

struct RoLayout {
  uint64_t plan, seq_at, off, big, total;
};
constexpr int kScanThreads = 1024;

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

RoLayout ro_layout(uint64_t num_seq, uint64_t max_cnt) {
  RoLayout L = {};
  uint64_t o = 0;
  L.plan = o;
  o = align256(o + sizeof(RoPlan));
  L.seq_at = o;
  o = align256(o + 4 * (num_seq ? num_seq : 1));
  L.off = o;
  o = align256(o + 4 * (num_seq ? num_seq : 1));
  L.big = o;  // global keys of a sequence above kSmemSort particles
  const uint64_t big = max_cnt > kSmemSort + 1 ? next_pow2(max_cnt - 1) : 1;
  o = align256(o + 16 * big);
  L.total = o;
  return L;
}

__device__ __forceinline__ uint32_t m_of(const LeafRec &r, int d) { return (r.m >> (8 * d)) & 0xffu; }
__device__ __forceinline__ uint32_t msum(const LeafRec &r) { return m_of(r, 0) + m_of(r, 1) + m_of(r, 2); }

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
                                                          C *o0, C *o1, C *o2, uint32_t *oidx, uint32_t cap) {
  extern __shared__ unsigned long long keys[];  // [2][cap]
  const int32_t order[3] = {plan->order[0], plan->order[1], plan->order[2]};
  for (uint64_t j = blockIdx.x; j < num_seq; j += gridDim.x) {
    const LeafRec r = recs[seq_at[j]];
    const uint32_t L = r.cnt - 1;
    if (L > cap) continue;  // k_ro_sort_big
    uint32_t P = 1;
    while (P < L) P <<= 1;
    uint32_t pbits = 1;
    while ((1u << pbits) < r.cnt) ++pbits;
    if (msum(r) + pbits <= 64 && P <= E * blockDim.x) {
      // narrow keys in registers (padded to a warp's worth at least)
      const uint32_t Pw = P < 32u * E ? 32u * E : P;
      sort_narrow<E, C>(r, Pw, pbits, order, q0, q1, q2, keys);
      const unsigned long long pmask = (1ull << pbits) - 1;
      const uint32_t dst = off[j];
      for (uint32_t i = threadIdx.x; i <= L; i += blockDim.x) {
        const uint32_t p = i == 0 ? r.centre : uint32_t(keys[i - 1] & pmask);
        const uint64_t src = uint64_t(r.off) + p, d = uint64_t(dst) + i;
        o0[d] = q0[src];
        o1[d] = q1[src];
        o2[d] = q2[src];
        if (IDX) oidx[d] = idx[src];
      }
      __syncthreads();
    } else {
      sort_one<C, IDX>(r, off[j], order, q0, q1, q2, idx, o0, o1, o2, oidx, keys, keys + cap, P);
    }
  }
}

template <typename C, bool IDX>
__global__ void __launch_bounds__(kSortThreads) k_ro_sort_big(const LeafRec *__restrict__ recs, uint64_t num_seq,
                                                              const uint32_t *__restrict__ seq_at,
                                                              const uint32_t *__restrict__ off, const RoPlan *plan,
                                                              const C *q0, const C *q1, const C *q2,
                                                              const uint32_t *idx, C *o0, C *o1, C *o2, uint32_t *oidx,
                                                              uint32_t cap, unsigned long long *big, uint64_t big_cap) {
  const int32_t order[3] = {plan->order[0], plan->order[1], plan->order[2]};
  for (uint64_t j = 0; j < num_seq; ++j) {
    const LeafRec r = recs[seq_at[j]];
    const uint32_t L = r.cnt - 1;
    if (L <= cap) continue;
    uint32_t P = 1;
    while (P < L) P <<= 1;
    if (P > big_cap) continue;  // sized for the largest sequence: cannot happen
    sort_one<C, IDX>(r, off[j], order, q0, q1, q2, idx, o0, o1, o2, oidx, big, big + big_cap, P);
  }
}

template <typename C, bool IDX>
cudaError_t reorder_dispatch(const ReorderLaunch &a, cudaStream_t st) {
  const RoLayout L = ro_layout(a.num_seq, a.max_cnt);
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
  e = cudaMemcpyAsync(&max_cnt, &plan->max_cnt, 4, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
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
    // E keys per thread in registers: cap / E threads (a warp at least), 4 keys below 2048, 8 from there
    // (fewer threads per sequence, two sequences per SM)
    const size_t smem = size_t(cap < 256 ? 256 : cap) * 16;
    const bool wide = cap >= 2048;
    const int threads = int(cap / (wide ? 8 : 4) < 32 ? 32 : cap / (wide ? 8 : 4));
    auto kern = wide ? k_ro_sort<C, IDX, 8> : k_ro_sort<C, IDX, 4>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const uint64_t grid = uint64_t(per_sm) * sms;
    kern<<<unsigned(a.num_seq < grid ? a.num_seq : grid), threads, smem, st>>>(
        a.recs, a.num_seq, seq_at, off, plan, q0, q1, q2, a.idx, o0, o1, o2, a.out_idx, cap < 256 ? 256 : cap);
  }
  if (longest > cap) {
    const uint64_t big_cap = next_pow2(longest);
    if (L.total - L.big < 16 * big_cap) return cudaErrorInvalidValue;  // the scratch bound was too small
    TraceScope ts("k_ro_sort_big", st);
    k_ro_sort_big<C, IDX><<<1, kSortThreads, 0, st>>>(a.recs, a.num_seq, seq_at, off, plan, q0, q1, q2, a.idx, o0,
                                                     o1, o2, a.out_idx, cap,
                                                     reinterpret_cast<unsigned long long *>(base + L.big), big_cap);
  }
  return cudaGetLastError();
}

}  // namespace

uint64_t reorder_scratch_bytes(uint64_t num_seq, uint64_t max_cnt) { return ro_layout(num_seq, max_cnt).total; }

cudaError_t launch_reorder(const ReorderLaunch &a, cudaStream_t st) {
  if (a.n == 0 || a.num_seq == 0) return cudaSuccess;
  if (a.code_bytes == 2)
    return a.idx ? reorder_dispatch<uint16_t, true>(a, st) : reorder_dispatch<uint16_t, false>(a, st);
  return a.idx ? reorder_dispatch<uint32_t, true>(a, st) : reorder_dispatch<uint32_t, false>(a, st);
}

}  // namespace pcx
