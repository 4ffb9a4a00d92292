// Stream header, stream validation and decoding (Sec. 3 dequantization,
// Sec. 4.2 / Fig. 4 layout of arXiv 2404.02826).
//
// Decoding reconstructs p_hat = (T)(o + s q) with one double multiply and one
// double add, q = q_ref + c - (2^(m-1) - 1) and q = q_ref for the centre.  For
// float output the kernel evaluates that expression on the FP32 pipe: s q and
// o + s q are formed as unevaluated float sums with error-free products and
// sums (relative error below 2^-45 of max(|o|, |s q|)), rounded once to float,
// and the literal double expression is used whenever that sum lies within
// 2^-40 of a rounding midpoint, sits on a power of two, or is tiny.  Elsewhere
// the two agree, because the double-precision value is within 2^-51 of the
// exact one.  Double output uses the double expression directly.
#include <cstdint>

#include "pc_internal.cuh"

namespace pcx {
namespace {

constexpr int kDecThreads = 256;
constexpr int kDecPer = 4;                          // particles per thread
constexpr int kChunk = kDecThreads * kDecPer;       // particles per block

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

// One thread per leaf: every field and every neighbour relation is checked.
__global__ void k_validate(const uint8_t *__restrict__ stream, uint64_t n, uint64_t num_leaves, uint64_t words,
                           uint32_t *err) {
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
  if (!ok) atomicOr(err, kErrCorrupt);
}

__device__ __forceinline__ uint32_t get_bits(const uint32_t *__restrict__ w, uint64_t nwords, uint64_t bit,
                                             uint32_t m) {
  const uint64_t i = bit >> 5;
  const uint32_t lo = i < nwords ? __ldg(w + i) : 0u;
  const uint32_t hi = (i + 1) < nwords ? __ldg(w + i + 1) : 0u;
  const unsigned long long v = ((unsigned long long)hi << 32 | lo) >> (bit & 31);
  return uint32_t(v) & ((1u << m) - 1u);
}

// float-pair evaluation of (float)(o + s*q) with a double fallback
__device__ __forceinline__ float dequant_fast(int32_t q, float of, double od, double s, float sh, float sl) {
  if (q < 0 || q >= (1 << 24)) return __double2float_rn(__dadd_rn(od, __dmul_rn(s, (double)q)));
  const float qf = (float)q;  // exact
  const float yh = __fmul_rn(sh, qf);
  const float ye = __fmaf_rn(sh, qf, -yh);
  const float yl = __fmaf_rn(sl, qf, ye);
  // TwoSum(of, yh)
  const float zh = __fadd_rn(of, yh);
  const float bb = __fsub_rn(zh, of);
  const float ze = __fadd_rn(__fsub_rn(of, __fsub_rn(zh, bb)), __fsub_rn(yh, bb));
  const float zl = __fadd_rn(ze, yl);
  const float out = __fadd_rn(zh, zl);
  // exact residual of the final rounding
  const float b2 = __fsub_rn(out, zh);
  const float err = __fadd_rn(__fsub_rn(zh, __fsub_rn(out, b2)), __fsub_rn(zl, b2));
  const uint32_t ob = __float_as_uint(out) & 0x7fffffffu;
  const uint32_t ex = ob >> 23;
  const float mag = fmaxf(fabsf(of), fabsf(yh));
  const uint32_t mb = __float_as_uint(mag) >> 23;
  if (ex >= 64 && ex < 255 && (ob & 0x7fffffu) != 0 && mb >= 64 && mb < 255) {
    const float half = __uint_as_float((ex - 24) << 23);  // half a unit in the last place of out
    const float tol = __uint_as_float((mb - 40) << 23);   // 2^-40 of max(|o|, |s q|), rounded down
    if (__fsub_rn(half, fabsf(err)) > tol) return out;
  }
  return __double2float_rn(__dadd_rn(od, __dmul_rn(s, (double)q)));
}

template <typename T, bool FAST, bool VEC>
__global__ void __launch_bounds__(kDecThreads) k_decode(DecodeLaunch a) {
  __shared__ __align__(16) T stage[3 * kChunk];
  __shared__ uint64_t first_leaf;
  if (*a.err) return;  // validation failed: write nothing
  const uint64_t c0 = uint64_t(blockIdx.x) * kChunk;
  if (c0 >= a.n) return;
  const uint64_t c1 = (c0 + kChunk) < a.n ? (c0 + kChunk) : a.n;
  const uint8_t *table = a.stream + kHeaderBytes;
  const uint32_t *words = reinterpret_cast<const uint32_t *>(table + uint64_t(kLeafBytes) * a.num_leaves);
  if (threadIdx.x == 0) {
    uint64_t lo = 0, hi = a.num_leaves - 1;  // last leaf with po <= c0
    while (lo < hi) {
      const uint64_t mid = (lo + hi + 1) >> 1;
      if (load_rec(table, mid).po <= c0) lo = mid;
      else hi = mid - 1;
    }
    first_leaf = lo;
  }
  __syncthreads();
  const uint64_t Lf = first_leaf;
  for (int k = 0; k < kDecPer; ++k) {
    const uint64_t g = c0 + uint64_t(k) * kDecThreads + threadIdx.x;
    if (g >= c1) break;
    // leaf of g: the last L >= Lf with po(L) <= g
    uint64_t lo = Lf, hi = a.num_leaves - 1;
    uint64_t span = 1;
    while (lo + span <= hi && load_rec(table, lo + span).po <= g) span <<= 1;  // gallop
    hi = (lo + span) < hi ? (lo + span) : hi;
    while (lo < hi) {
      const uint64_t mid = (lo + hi + 1) >> 1;
      if (load_rec(table, mid).po <= g) lo = mid;
      else hi = mid - 1;
    }
    const Rec r = load_rec(table, lo);
    const uint64_t i = g - r.po;
    int32_t q[3] = {r.q[0], r.q[1], r.q[2]};
    if (i > 0) {
      const uint32_t w = r.m[0] + r.m[1] + r.m[2];
      uint64_t bit = 32ull * r.wo + (i - 1) * (uint64_t)w;
      for (int d = 0; d < 3; ++d) {
        const uint32_t m = r.m[d];
        if (m) {
          const uint32_t c = get_bits(words, a.payload_words, bit, m);
          q[d] = r.q[d] + int32_t(c) - int32_t((1u << (m - 1)) - 1u);
          bit += m;
        }
      }
    }
    const uint32_t sl = uint32_t(g - c0);
    for (int d = 0; d < 3; ++d) {
      T v;
      if (sizeof(T) == 4) {
        if (FAST) v = (T)dequant_fast(q[d], a.of[d], a.o[d], a.s, a.sh, a.sl);
        else v = (T)__double2float_rn(__dadd_rn(a.o[d], __dmul_rn(a.s, (double)q[d])));
      } else {
        v = (T)__dadd_rn(a.o[d], __dmul_rn(a.s, (double)q[d]));
      }
      stage[3 * sl + d] = v;
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
  uint64_t words = 0;
  if (a.last_state) {
    const unsigned long long s = *a.last_state;
    if ((s >> 62) != 2) atomicOr(a.err, kErrInternal);
    words = s & ((1ull << 62) - 1);
  }
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
  const unsigned blocks = unsigned((a.n + kChunk - 1) / kChunk);
  TraceScope ts("k_decode", st);
  if (a.vec) k_decode<T, FAST, true><<<blocks, kDecThreads, 0, st>>>(a);
  else k_decode<T, FAST, false><<<blocks, kDecThreads, 0, st>>>(a);
}

}  // namespace

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
                                                                        a.err);
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
