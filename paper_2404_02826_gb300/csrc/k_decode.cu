// Stream header, stream validation and decoding (Sec. 3 dequantization,
// Sec. 4.2 / Fig. 4 layout of arXiv 2404.02826).
//
// Decoding reconstructs p_hat = (T)(o + s q) with one double multiply and one
// double add, q = q_ref + c - (2^(m-1) - 1) and q = q_ref for the centre.  For
// float output the kernel evaluates that expression on the FP32 pipe: s q and
// o + s q are formed as an unevaluated float sum zh + zl with error-free
// products and sums (error below 2^-45 of max(|o|, |s q|)).  It then rounds
// zh + zl - tol and zh + zl + tol to float, tol = 2^-40 max(|o|, |s q|): when
// both give the same float, every real number in between - the exact value and
// the double-precision value, which is within 2^-51 of it - rounds to that
// float too (rounding to nearest is monotone).  Otherwise, and for tiny or
// huge magnitudes, the literal double expression decides.  Double output uses
// the double expression directly.
#include <cstdint>

#include "pc_internal.cuh"

namespace pcx {
namespace {

constexpr int kDecThreads = 256;
constexpr int kDecPer = 4;                          // particles per thread
constexpr int kChunk = kDecThreads * kDecPer;       // particles per block
constexpr int kChunkLeaves = 32;                    // leaves of one chunk held in shared memory
// Payload words staged per chunk: kChunk particles of at most 93 bits, up to
// kChunkLeaves word-aligned leaf starts, the alignment of the first staged
// word and a 4-word read window past the last particle fit in 3 * kChunk + 64.
constexpr int kWordCap = 3 * kChunk + 64;

struct Rec {
  uint64_t po, wo;
  int32_t q[3];
  uint32_t m[3];
  uint32_t zero;
};

__device__ __forceinline__ Rec load_rec(const uint8_t *table, uint64_t L) {
  const uint4 *p = reinterpret_cast<const uint4 *>(table + uint64_t(kLeafBytes) * L);
  const uint4 a = __ldg(p), b = __ldg(p + 1);
  Rec r;
  r.po = uint64_t(a.x) | (uint64_t(a.y) << 32);
  r.wo = uint64_t(a.z) | (uint64_t(a.w) << 32);
  r.q[0] = int32_t(b.x);
  r.q[1] = int32_t(b.y);
  r.q[2] = int32_t(b.z);
  r.m[0] = b.w & 0xffu;
  r.m[1] = (b.w >> 8) & 0xffu;
  r.m[2] = (b.w >> 16) & 0xffu;
  r.zero = b.w >> 24;
  return r;
}

__device__ __forceinline__ uint64_t leaf_words(const Rec &r, uint64_t cnt) {
  return ((uint64_t)(r.m[0] + r.m[1] + r.m[2]) * (cnt - 1) + 31) >> 5;
}

// One thread per leaf: every field and every neighbour relation is checked,
// and each decode chunk whose first particle lies in this leaf records it.
__global__ void k_validate(const uint8_t *__restrict__ stream, uint64_t n, uint64_t num_leaves, uint64_t words,
                           uint32_t *chunk_leaf, uint32_t *err) {
  const uint64_t L = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (L >= num_leaves) return;
  const uint8_t *table = stream + kHeaderBytes;
  const Rec r = load_rec(table, L);
  const uint64_t pend = (L + 1 < num_leaves) ? load_rec(table, L + 1).po : n;
  bool ok = r.zero == 0 && r.m[0] <= 31 && r.m[1] <= 31 && r.m[2] <= 31 && pend > r.po && pend <= n;
  if (L == 0) ok = ok && r.po == 0 && r.wo == 0;
  if (ok) {
    const uint64_t wend = r.wo + leaf_words(r, pend - r.po);
    const uint64_t wnext = (L + 1 < num_leaves) ? load_rec(table, L + 1).wo : words;
    ok = r.wo <= words && wend == wnext;
  }
  if (!ok) {
    atomicOr(err, kErrCorrupt);
    return;
  }
  for (uint64_t c = (r.po + kChunk - 1) / kChunk; c * kChunk < pend; ++c) chunk_leaf[c] = uint32_t(L);
}

__device__ __forceinline__ uint32_t word_at(const uint32_t *__restrict__ w, uint64_t nwords, uint64_t i) {
  return i < nwords ? __ldg(w + i) : 0u;
}

__device__ __forceinline__ float dequant_exact(int32_t q, double od, double s) {
  return __double2float_rn(__dadd_rn(od, __dmul_rn(s, (double)q)));
}
// The same, kept out of line so that the rare fallback below is a real branch:
// inlined, the compiler evaluates it speculatively on GB300's narrow FP64 pipe.
__device__ __noinline__ float dequant_exact_call(int32_t q, double od, double s) { return dequant_exact(q, od, s); }

// float-pair evaluation of (float)(o + s*q), exact by the monotonicity check
__device__ __forceinline__ float dequant_fast(int32_t q, float of, double od, double s, float sh, float sl) {
  const float qf = (float)q;  // exact while |q| < 2^24
  const float yh = __fmul_rn(sh, qf);
  const float ye = __fmaf_rn(sh, qf, -yh);
  const float yl = __fmaf_rn(sl, qf, ye);
  // TwoSum(of, yh): zh + ze == of + yh exactly
  const float zh = __fadd_rn(of, yh);
  const float bb = __fsub_rn(zh, of);
  const float ze = __fadd_rn(__fsub_rn(of, __fsub_rn(zh, bb)), __fsub_rn(yh, bb));
  const float zl = __fadd_rn(ze, yl);
  const float mag = fmaxf(fabsf(of), fabsf(yh));
  const float tol = __fmul_rn(mag, 0x1p-40f);
  const float r1 = __fadd_rn(zh, __fsub_rn(zl, tol));
  const float r2 = __fadd_rn(zh, __fadd_rn(zl, tol));
  if (__builtin_expect(r1 == r2 && mag > 0x1p-80f && mag < 0x1p100f && (unsigned)q < (1u << 24), 1)) return r1;
  return dequant_exact_call(q, od, s);
}

// Code of m bits at bit offset r (0 <= r < 96) of the window w0..w3.
__device__ __forceinline__ uint32_t window_bits(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t r,
                                                uint32_t m) {
  const uint32_t k = r >> 5;
  const uint32_t lo = k == 0 ? w0 : (k == 1 ? w1 : w2);
  const uint32_t hi = k == 0 ? w1 : (k == 1 ? w2 : w3);
  return __funnelshift_r(lo, hi, r & 31) & ((1u << m) - 1u);
}

// Dequantizes one particle's three codes into the chunk's staging area.
template <typename T, bool FAST>
__device__ __forceinline__ void put_particle(const DecodeLaunch &a, T *stage, uint32_t sl, int32_t q0, int32_t q1,
                                             int32_t q2) {
  const int32_t q[3] = {q0, q1, q2};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T v;
    if (sizeof(T) == 4) {
      if (FAST) v = (T)dequant_fast(q[d], a.of[d], a.o[d], a.s, a.sh, a.sl);
      else v = (T)dequant_exact(q[d], a.o[d], a.s);
    } else {
      v = (T)__dadd_rn(a.o[d], __dmul_rn(a.s, (double)q[d]));
    }
    stage[3 * sl + d] = v;
  }
}

// c = code - (2^(m-1) - 1) for the three fields of one particle starting at
// bit r0 of the 4-word window.
__device__ __forceinline__ void add_fields(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t r0,
                                           uint32_t mm, int32_t &q0, int32_t &q1, int32_t &q2) {
  const uint32_t m0 = mm & 0xffu, m1 = (mm >> 8) & 0xffu, m2 = (mm >> 16) & 0xffu;
  if (m0) q0 += int32_t(window_bits(w0, w1, w2, w3, r0, m0)) - int32_t((1u << (m0 - 1)) - 1u);
  if (m1) q1 += int32_t(window_bits(w0, w1, w2, w3, r0 + m0, m1)) - int32_t((1u << (m1 - 1)) - 1u);
  if (m2) q2 += int32_t(window_bits(w0, w1, w2, w3, r0 + m0 + m1, m2)) - int32_t((1u << (m2 - 1)) - 1u);
}

// One block decodes a chunk of kChunk consecutive particles.  When the chunk
// holds at most kChunkLeaves leaves (always, unless leaves are tiny), their
// records and the payload words the chunk spans are staged in shared memory
// with coalesced loads, and every particle is located with 32-bit arithmetic
// relative to the staged words.  Otherwise each particle searches the leaf
// table and reads its words from global memory.
template <typename T, bool FAST, bool VEC>
__global__ void __launch_bounds__(kDecThreads) k_decode(DecodeLaunch a) {
  __shared__ __align__(16) T stage[3 * kChunk];
  __shared__ __align__(16) uint32_t sw[kWordCap];
  __shared__ uint64_t s_po[kChunkLeaves + 1], s_wo[kChunkLeaves + 1];
  __shared__ int64_t s_base[kChunkLeaves];  // staged-relative bit of "particle 0" of the leaf, minus one field width
  __shared__ int32_t s_q[kChunkLeaves][3];
  __shared__ uint32_t s_m[kChunkLeaves + 1];
  __shared__ int s_count, s_staged;
  __shared__ uint64_t s_lo, s_hi, s_end;
  if (*a.err) return;  // validation failed: write nothing
  const uint64_t c0 = uint64_t(blockIdx.x) * kChunk;
  if (c0 >= a.n) return;
  const uint64_t c1 = (c0 + kChunk) < a.n ? (c0 + kChunk) : a.n;
  const uint8_t *table = a.stream + kHeaderBytes;
  const uint32_t *words = reinterpret_cast<const uint32_t *>(table + uint64_t(kLeafBytes) * a.num_leaves);
  const uint64_t first = a.chunk_leaf[blockIdx.x];
  if (threadIdx.x < kChunkLeaves + 1) {
    const uint64_t L = first + threadIdx.x;
    if (L < a.num_leaves) {
      const Rec r = load_rec(table, L);
      s_po[threadIdx.x] = r.po;
      s_wo[threadIdx.x] = r.wo;
      s_m[threadIdx.x] = r.m[0] | (r.m[1] << 8) | (r.m[2] << 16);
      if (threadIdx.x < kChunkLeaves) {
        s_q[threadIdx.x][0] = r.q[0];
        s_q[threadIdx.x][1] = r.q[1];
        s_q[threadIdx.x][2] = r.q[2];
      }
    } else {
      s_po[threadIdx.x] = a.n;
      s_wo[threadIdx.x] = a.payload_words;
      s_m[threadIdx.x] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 1;
    while (c < kChunkLeaves && s_po[c] < c1) ++c;
    s_count = c;
    const bool in_smem = c < kChunkLeaves || s_po[kChunkLeaves] >= c1;
    int staged = 0;
    if (in_smem) {
      // first bit of particle c0 and end bit of particle c1 - 1
      auto width = [](uint32_t mm) { return uint64_t((mm & 0xffu) + ((mm >> 8) & 0xffu) + ((mm >> 16) & 0xffu)); };
      const uint64_t i0 = c0 - s_po[0];
      const uint64_t b0 = 32 * s_wo[0] + (i0 ? (i0 - 1) * width(s_m[0]) : 0);
      const uint64_t il = (c1 - 1) - s_po[c - 1];
      const uint64_t b1 = 32 * s_wo[c - 1] + il * width(s_m[c - 1]);
      const uint64_t lo = (b0 >> 5) & ~3ull;  // 16-byte aligned start of the staged words
      const uint64_t end = ((b1 + 31) >> 5) + 4;  // words a particle's 4-word window may touch
      if (end - lo <= kWordCap) {
        staged = 1;
        s_lo = lo;
        s_end = end;
        s_hi = end < a.payload_words ? end : a.payload_words;
        for (int L = 0; L < c; ++L)
          s_base[L] = int64_t(32 * s_wo[L]) - int64_t(32 * lo) - int64_t(width(s_m[L]));
      }
    }
    s_staged = staged;
  }
  __syncthreads();
  const int count = s_count;
  T *stage_t = stage;
  if (s_staged) {
    const uint64_t lo = s_lo, hi = s_hi;
    const uint32_t nst = uint32_t(s_end - lo);
    const uint32_t nreal = hi > lo ? uint32_t(hi - lo) : 0u;
    if ((reinterpret_cast<uintptr_t>(words) & 15) == 0) {
      const uint32_t nvec = nreal >> 2;
      const uint4 *src = reinterpret_cast<const uint4 *>(words + lo);
      uint4 *dst = reinterpret_cast<uint4 *>(sw);
      for (uint32_t v = threadIdx.x; v < nvec; v += kDecThreads) dst[v] = __ldg(src + v);
      for (uint32_t w = 4 * nvec + threadIdx.x; w < nst; w += kDecThreads) sw[w] = w < nreal ? __ldg(words + lo + w) : 0u;
    } else {
      for (uint32_t w = threadIdx.x; w < nst; w += kDecThreads) sw[w] = w < nreal ? __ldg(words + lo + w) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kDecPer; ++k) {
      const uint32_t sl = uint32_t(k) * kDecThreads + threadIdx.x;
      const uint64_t g = c0 + sl;
      if (g >= c1) continue;
      int L = 0;
      while (L + 1 < count && s_po[L + 1] <= g) ++L;
      int32_t q0 = s_q[L][0], q1 = s_q[L][1], q2 = s_q[L][2];
      const uint32_t i = uint32_t(g - s_po[L]);
      if (i > 0) {
        const uint32_t mm = s_m[L];
        const uint32_t w = (mm & 0xffu) + ((mm >> 8) & 0xffu) + ((mm >> 16) & 0xffu);
        const uint32_t bit = uint32_t(s_base[L] + int64_t(uint64_t(i) * w));
        const uint32_t wi = bit >> 5;
        add_fields(sw[wi], sw[wi + 1], sw[wi + 2], sw[wi + 3], bit & 31u, mm, q0, q1, q2);
      }
      put_particle<T, FAST>(a, stage_t, sl, q0, q1, q2);
    }
  } else {
    const bool in_smem = count < kChunkLeaves || s_po[kChunkLeaves] >= c1;
#pragma unroll
    for (int k = 0; k < kDecPer; ++k) {
      const uint32_t sl = uint32_t(k) * kDecThreads + threadIdx.x;
      const uint64_t g = c0 + sl;
      if (g >= c1) continue;
      uint64_t po, wo;
      int32_t q0, q1, q2;
      uint32_t mm;
      if (in_smem) {
        int L = 0;
        while (L + 1 < count && s_po[L + 1] <= g) ++L;
        po = s_po[L];
        wo = s_wo[L];
        q0 = s_q[L][0];
        q1 = s_q[L][1];
        q2 = s_q[L][2];
        mm = s_m[L];
      } else {  // many small leaves in this chunk: search the table
        uint64_t lo = first, hi = a.num_leaves - 1;
        while (lo < hi) {
          const uint64_t mid = (lo + hi + 1) >> 1;
          if (load_rec(table, mid).po <= g) lo = mid;
          else hi = mid - 1;
        }
        const Rec r = load_rec(table, lo);
        po = r.po;
        wo = r.wo;
        q0 = r.q[0];
        q1 = r.q[1];
        q2 = r.q[2];
        mm = r.m[0] | (r.m[1] << 8) | (r.m[2] << 16);
      }
      const uint64_t i = g - po;
      if (i > 0) {
        const uint32_t w = (mm & 0xffu) + ((mm >> 8) & 0xffu) + ((mm >> 16) & 0xffu);
        const uint64_t bit = 32ull * wo + (i - 1) * uint64_t(w);
        const uint64_t wi = bit >> 5;
        add_fields(word_at(words, a.payload_words, wi), word_at(words, a.payload_words, wi + 1),
                   word_at(words, a.payload_words, wi + 2), word_at(words, a.payload_words, wi + 3),
                   uint32_t(bit & 31), mm, q0, q1, q2);
      }
      put_particle<T, FAST>(a, stage_t, sl, q0, q1, q2);
    }
  }
  __syncthreads();
  T *out = static_cast<T *>(a.out) + 3 * c0;
  const uint32_t total = uint32_t(3 * (c1 - c0));
  if (VEC && (total % (16 / sizeof(T))) == 0) {
    const uint32_t nv = total / (16 / sizeof(T));
    const uint4 *s4 = reinterpret_cast<const uint4 *>(stage);
    uint4 *o4 = reinterpret_cast<uint4 *>(out);
    for (uint32_t v = threadIdx.x; v < nv; v += kDecThreads) __stcs(o4 + v, s4[v]);
  } else {
    for (uint32_t v = threadIdx.x; v < total; v += kDecThreads) out[v] = stage[v];
  }
}

__global__ void k_header(HeaderLaunch a) {
  const uint64_t words = a.total_words ? *a.total_words : 0;
  __align__(16) uint8_t h[kHeaderBytes];
  for (int i = 0; i < int(kHeaderBytes); ++i) h[i] = 0;
  h[0] = 'P';
  h[1] = 'C';
  h[2] = 'B';
  h[3] = '1';
  h[4] = 1;
  h[5] = 0;
  h[6] = uint8_t(a.dtype);
  h[7] = uint8_t(a.eb_mode);
  auto put64 = [&](int at, uint64_t v) {
    for (int i = 0; i < 8; ++i) h[at + i] = uint8_t(v >> (8 * i));
  };
  put64(8, a.n);
  put64(16, (uint64_t)__double_as_longlong(a.eb));
  put64(24, (uint64_t)__double_as_longlong(a.eps));
  put64(32, (uint64_t)__double_as_longlong(a.s));
  for (int d = 0; d < 3; ++d) put64(40 + 8 * d, (uint64_t)__double_as_longlong(a.o[d]));
  put64(64, a.num_leaves);
  put64(72, words);
  for (int i = 0; i < 4; ++i) h[80 + i] = uint8_t(a.leaf_size >> (8 * i));
  uint4 *dst = reinterpret_cast<uint4 *>(a.out);
  const uint4 *src = reinterpret_cast<const uint4 *>(h);
  for (int i = 0; i < int(kHeaderBytes / 16); ++i) dst[i] = src[i];
  *a.total_bytes = uint64_t(kHeaderBytes) + uint64_t(kLeafBytes) * a.num_leaves + 4ull * words;
}

template <typename T, bool FAST>
void decode_dispatch(const DecodeLaunch &a, cudaStream_t st) {
  const unsigned blocks = unsigned(decode_chunks(a.n));
  TraceScope ts("k_decode", st);
  if (a.vec) k_decode<T, FAST, true><<<blocks, kDecThreads, 0, st>>>(a);
  else k_decode<T, FAST, false><<<blocks, kDecThreads, 0, st>>>(a);
}

}  // namespace

uint64_t decode_chunks(uint64_t n) { return (n + kChunk - 1) / kChunk; }

cudaError_t launch_header(const HeaderLaunch &a, cudaStream_t st) {
  TraceScope ts("k_header", st);
  k_header<<<1, 1, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_decode(const DecodeLaunch &a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  {
    TraceScope ts("k_validate", st);
    k_validate<<<unsigned((a.num_leaves + 255) / 256), 256, 0, st>>>(a.stream, a.n, a.num_leaves, a.payload_words,
                                                                        a.chunk_leaf, a.err);
  }
  if (a.dtype == 0) {
    if (a.fast) decode_dispatch<float, true>(a, st);
    else decode_dispatch<float, false>(a, st);
  } else {
    decode_dispatch<double, false>(a, st);
  }
  return cudaGetLastError();
}

}  // namespace pcx
