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
#include "pc_mbar.cuh"

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

// A leaf record as stored (32 bytes, Fig. 4 layout of this format).
__device__ __forceinline__ Rec rec_from(const uint4 a, const uint4 b) {
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

__device__ __forceinline__ Rec load_rec(const uint8_t *table, uint64_t L) {
  const uint4 *p = reinterpret_cast<const uint4 *>(table + uint64_t(kLeafBytes) * L);
  return rec_from(__ldg(p), __ldg(p + 1));
}

__device__ __forceinline__ uint64_t leaf_words(const Rec &r, uint64_t cnt) {
  return ((uint64_t)(r.m[0] + r.m[1] + r.m[2]) * (cnt - 1) + 31) >> 5;
}

// What a decode chunk needs before it can start: its leaves and the payload
// words its particles span (from a 16-byte aligned word, plus the 4-word read
// window of its last particle).
struct ChunkInfo {
  uint64_t lo, end;     // staged words [lo, end) of the payload
  uint32_t first, last;  // leaves of the chunk's first and last particle
  uint32_t tag;          // a batch: index of the chunk's stream
  uint32_t pad;
};

// One thread per leaf: every field and every neighbour relation is checked,
// and each decode chunk whose first particle lies in this leaf gets its first
// leaf and first word, the chunk before it its last leaf and end word.
// The range of codes a leaf can produce, [q_ref - 2^(m-1) + 1, q_ref + 2^(m-1)]
// per axis (any m-bit field, the unused all-ones one included), is reduced
// per warp into qb: qb[d] = min(0, lowest code), qb[3 + d] = max(0, highest).
// Leaf L of one stream (a lane past its last leaf takes part in the warp
// reductions only).
__device__ __forceinline__ void validate_leaf(const uint8_t *__restrict__ stream, uint64_t n, uint64_t num_leaves,
                                              uint64_t words, ChunkInfo *info, uint32_t *err, int32_t *qb,
                                              uint32_t raw, uint32_t M, uint64_t L) {
  const bool mine = L < num_leaves;
  const uint8_t *table = stream + kHeaderBytes;
  int32_t low[3] = {0, 0, 0}, top[3] = {0, 0, 0};
  if (mine) {
    const Rec r = load_rec(table, L);
    const uint64_t pend = (L + 1 < num_leaves) ? load_rec(table, L + 1).po : n;
    bool ok = r.zero == 0 && pend > r.po && pend <= n;
    for (int d = 0; d < 3; ++d) ok = ok && ((raw >> d) & 1u ? r.m[d] == M : r.m[d] <= 31);
    if (L == 0) ok = ok && r.po == 0 && r.wo == 0;
    if (ok) {
      // with lossless axes every particle of the leaf, the centre included, is in the payload
      const uint64_t wend = r.wo + (raw ? ((uint64_t)(r.m[0] + r.m[1] + r.m[2]) * (pend - r.po) + 31) >> 5
                                        : leaf_words(r, pend - r.po));
      const uint64_t wnext = (L + 1 < num_leaves) ? load_rec(table, L + 1).wo : words;
      ok = r.wo <= words && wend == wnext;
    }
    if (!ok) {
      atomicOr(err, kErrCorrupt);
    } else {
      const uint64_t w = r.m[0] + r.m[1] + r.m[2];
      for (uint64_t c = (r.po + kChunk - 1) / kChunk; c * kChunk < pend; ++c) {
        const uint64_t c0 = c * kChunk;
        const uint64_t bit = 32 * r.wo + (c0 > r.po ? (c0 - r.po - 1) * w : 0);  // first bit of particle c0
        info[c].lo = (bit >> 5) & ~3ull;
        info[c].first = uint32_t(L);
        if (c > 0) {
          info[c - 1].end = ((bit + 31) >> 5) + 4;
          info[c - 1].last = c0 == r.po ? uint32_t(L - 1) : uint32_t(L);
        }
      }
      if (L + 1 == num_leaves) {
        const uint64_t c = (n - 1) / kChunk;
        info[c].end = words + 4;
        info[c].last = uint32_t(L);
      }
      for (int d = 0; d < 3; ++d) {
        if ((raw >> d) & 1u) continue;  // a lossless axis has no codes
        const int64_t half = r.m[d] ? (int64_t(1) << (r.m[d] - 1)) : 0;
        const int64_t lo = int64_t(r.q[d]) - (half ? half - 1 : 0), hi = int64_t(r.q[d]) + half;
        low[d] = int32_t(lo >= 0 ? 0 : (lo < -0x7fffffffll ? -0x7fffffffll : lo));
        top[d] = int32_t(hi <= 0 ? 0 : (hi > 0x7fffffffll ? 0x7fffffffll : hi));
      }
    }
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    low[d] = __reduce_min_sync(0xffffffffu, low[d]);
    top[d] = __reduce_max_sync(0xffffffffu, top[d]);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (low[d]) atomicMin(qb + d, low[d]);
      if (top[d]) atomicMax(qb + 3 + d, top[d]);
    }
  }
}

__global__ void k_validate(const uint8_t *__restrict__ stream, uint64_t n, uint64_t num_leaves, uint64_t words,
                           ChunkInfo *info, uint32_t *err, int32_t *qb, uint32_t raw, uint32_t M) {
  validate_leaf(stream, n, num_leaves, words, info, err, qb, raw, M, uint64_t(blockIdx.x) * blockDim.x + threadIdx.x);
}

// ---- the decoding prologue on the device, launched before the header is back on the host ----

// The header fields the prologue needs, with the host parser's checks
// (format, version, kinds, sizes, the stream's own length, finite s > 0 and
// o): a stream that fails them is not touched.
struct DevHeader {
  uint64_t n, num_leaves, payload_words;
  double s, o[3];
  uint32_t dtype, raw;
  bool ok;
};

__device__ __forceinline__ DevHeader read_header(const uint8_t *stream, uint64_t stream_bytes) {
  DevHeader H = {};
  const uint4 *p = reinterpret_cast<const uint4 *>(stream);
  uint32_t w[24];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const uint4 v = __ldg(p + i);
    w[4 * i] = v.x;
    w[4 * i + 1] = v.y;
    w[4 * i + 2] = v.z;
    w[4 * i + 3] = v.w;
  }
  auto u64 = [&](int byte) { return uint64_t(w[byte / 4]) | (uint64_t(w[byte / 4 + 1]) << 32); };
  const uint32_t magic = 'P' | ('C' << 8) | ('B' << 16) | (uint32_t('1') << 24);
  bool ok = w[0] == magic && (w[1] & 0xffffu) == 1u;
  H.dtype = (w[1] >> 16) & 0xffu;
  const uint32_t mode = w[1] >> 24;
  ok = ok && H.dtype <= 1u && mode <= 1u;
  H.n = u64(8);
  H.s = __longlong_as_double((long long)u64(32));
  for (int d = 0; d < 3; ++d) H.o[d] = __longlong_as_double((long long)u64(40 + 8 * d));
  H.num_leaves = u64(64);
  H.payload_words = u64(72);
  H.raw = w[21] & 0xffu;
  ok = ok && H.raw <= 7u && (w[21] >> 8) == 0u && w[22] == 0u && w[23] == 0u;
  ok = ok && H.n <= PC_MAX_PARTICLES && H.num_leaves <= H.n && ((H.n > 0) == (H.num_leaves > 0));
  ok = ok && H.payload_words <= (1ull << 40) && isfinite(H.s) && H.s > 0.0;
  for (int d = 0; d < 3; ++d) ok = ok && isfinite(H.o[d]);
  ok = ok && uint64_t(kHeaderBytes) + uint64_t(kLeafBytes) * H.num_leaves + 4 * H.payload_words <= stream_bytes;
  H.ok = ok;
  return H;
}

// The first launch of a decompression: clears the workspace's first 64 bytes
// (error word, the decoder's block count, code bounds) and copies the header
// into page-locked host memory.
__global__ void k_decode_start(const uint8_t *stream, uint32_t *ws64, uint8_t *host_header) {
  const uint32_t t = threadIdx.x;
  if (t < 16) ws64[t] = 0u;
  if (t < kHeaderBytes / 16)
    reinterpret_cast<uint4 *>(host_header)[t] = __ldg(reinterpret_cast<const uint4 *>(stream) + t);
}

// k_validate with the header read on the device: a fixed grid strides over the
// leaves (warp-uniform steps, as validate_leaf's reductions need); nothing is
// done when the header fails its checks or the chunk facts would not fit the
// `chunk_cap` entries the workspace holds (the host then returns the error).
__global__ void __launch_bounds__(256) k_validate_dev(const uint8_t *stream, uint64_t stream_bytes, uint64_t chunk_cap,
                                                      ChunkInfo *info, uint32_t *err, int32_t *qb) {
  const DevHeader H = read_header(stream, stream_bytes);
  if (!H.ok) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, kErrCorrupt);
    return;
  }
  if ((H.n + kChunk - 1) / kChunk > chunk_cap) return;
  const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t base = uint64_t(blockIdx.x) * blockDim.x; base < H.num_leaves; base += step)
    validate_leaf(stream, H.n, H.num_leaves, H.payload_words, info, err, qb, H.raw, H.dtype == 0 ? 32u : 64u,
                  base + threadIdx.x);
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

// Entries of the dequantization table (global memory, read through L1).
constexpr uint32_t kTabEntries = 24576;

// Constants of one leaf of the chunk being decoded.
struct LeafC {
  int32_t rel;       // first particle of the leaf minus the chunk's first particle
  int32_t base;      // bit of particle i is base + i * w, relative to the first staged word
  uint32_t w;        // m_x + m_y + m_z
  uint32_t m0;       // m_x
  uint32_t s2;       // m_x + m_y: first bit of the z field
  uint32_t mask[3];  // 2^m_d - 1
  int32_t off[3];    // q_ref_d - (2^(m_d - 1) - 1): the code of field value 0
  int32_t qref[3];
  uint32_t pad[2];
};

// One chunk's staging area: its payload words, from a 16-byte aligned word
// (room for the copy rounded up to whole 16 bytes), and its leaf records as
// stored in the stream.
struct DecBuf {
  uint32_t sw[kWordCap + 4];
  uint4 rec[2 * kChunkLeaves];
};

// Persistent decoder: two staging areas filled by bulk copies, the leaf
// constants of each, the chunk descriptors and the copies' barriers.
struct DecSmem {
  DecBuf buf[2];
  LeafC lc[2][kChunkLeaves];
  ChunkInfo ci[2];
  unsigned long long bar[2];
  uint32_t ncopy[2];  // words each area's copy brings
};

// Whether the code ranges [lo_d, hi_d] of the three axes fit kTabEntries
// entries together; tb[d] is where axis d's table starts.
__device__ __forceinline__ bool table_fits(const int32_t *qb, uint32_t tb[3], uint32_t &te) {
  uint64_t e = 0;
  for (int d = 0; d < 3; ++d) {
    tb[d] = uint32_t(e);
    e += uint64_t(int64_t(qb[3 + d]) - int64_t(qb[d]) + 1);
  }
  te = uint32_t(e < kTabEntries ? e : kTabEntries);
  return e <= kTabEntries;
}

// (T)(o_d + s q) by the double expression; float output on the FP32 pipe when exact.
template <typename T, bool FAST>
__device__ __forceinline__ T dequant(const DecodeLaunch &a, int d, int32_t q) {
  if (sizeof(T) == 4) {
    if (FAST) return (T)dequant_fast(q, a.of[d], a.o[d], a.s, a.sh, a.sl);
    return (T)dequant_exact(q, a.o[d], a.s);
  }
  return (T)__dadd_rn(a.o[d], __dmul_rn(a.s, (double)q));
}

// The same for the per-particle path when there are no tables.  Float output
// with the float-pair check stays inline (FP32 pipe); the double expression
// is kept out of line, so that it is not evaluated speculatively on GB300's
// narrow FP64 pipe beside the table lookups.
template <typename T>
__device__ __noinline__ T dequant_double_call(const DecodeLaunch &a, int d, int32_t q) {
  if (sizeof(T) == 4) return (T)dequant_exact(q, a.o[d], a.s);
  return (T)__dadd_rn(a.o[d], __dmul_rn(a.s, (double)q));
}
template <typename T, bool FAST>
__device__ __forceinline__ T dequant_particle(const DecodeLaunch &a, int d, int32_t q) {
  if (sizeof(T) == 4 && FAST) return (T)dequant_fast(q, a.of[d], a.o[d], a.s, a.sh, a.sl);
  return dequant_double_call<T>(a, d, q);
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

// (T)(o_d + s q) for every code q in [lo_d, hi_d] of the three axes, one
// table after another: the dequantization of a particle becomes three
// lookups, and the double expression is evaluated once per code.
template <typename T, bool FAST>
__device__ __forceinline__ void fill_table(const DecodeLaunch &a) {
  uint32_t tb[3], te;
  if (!table_fits(a.qb, tb, te)) return;
  T *tab = static_cast<T *>(a.tab);
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < te; e += gridDim.x * blockDim.x) {
    const int d = e < tb[1] ? 0 : (e < tb[2] ? 1 : 2);
    const int32_t q = a.qb[d] + int32_t(e - tb[d]);
    tab[e] = dequant<T, FAST>(a, d, q);
  }
}
// The decoder is launched as the tables' programmatic dependent: its blocks may
// be placed as soon as every block of the tables has begun, and wait for the
// tables' completion (griddepcontrol.wait) before they read anything.
template <typename T, bool FAST>
__global__ void k_dtable(DecodeLaunch a) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (*a.err) return;
  fill_table<T, FAST>(a);
}
// k_dtable with the header read on the device: the same tables, the float-pair
// path chosen by the host's rule (float output, o exact in float, s within
// 2^-100 .. 2^100).  Nothing for a failed validation or lossless axes.
__global__ void k_dtable_dev(const uint8_t *stream, uint64_t stream_bytes, const uint32_t *err, int32_t *qb,
                             void *tab) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (*reinterpret_cast<const volatile uint32_t *>(err)) return;
  const DevHeader H = read_header(stream, stream_bytes);
  if (!H.ok || H.raw || H.n == 0) return;
  DecodeLaunch a = {};
  a.s = H.s;
  bool exact_o = true;
  for (int d = 0; d < 3; ++d) {
    a.o[d] = H.o[d];
    a.of[d] = __double2float_rn(H.o[d]);
    exact_o = exact_o && double(a.of[d]) == H.o[d];
  }
  a.sh = __double2float_rn(H.s);
  a.sl = __double2float_rn(H.s - double(a.sh));
  a.qb = qb;
  a.tab = tab;
  if (H.dtype != 0) fill_table<double, false>(a);
  else if (exact_o && H.s > 0x1p-100 && H.s < 0x1p100) fill_table<float, true>(a);
  else fill_table<float, false>(a);
}

// Whether a chunk is decoded from shared memory: at most kChunkLeaves leaves
// and a payload span that fits the staging area.
__device__ __forceinline__ bool chunk_staged(const ChunkInfo &ci) {
  return ci.last - ci.first + 1 <= uint32_t(kChunkLeaves) && ci.end - ci.lo <= uint64_t(kWordCap);
}

// Thread 0: starts the bulk copies of a chunk into staging area b - its
// payload words in whole 16-byte units as far as the payload reaches, and its
// leaf records - or, for a chunk that is not staged, only arrives on b's
// barrier.  Source and destination are 16-byte aligned: the stream starts on
// 16 bytes, the leaf table at byte 96 in 32-byte records, the payload after
// it, and a chunk's first staged word is a multiple of 4.
__device__ __forceinline__ void dec_issue(uint64_t payload_words, DecSmem &S, int b, const ChunkInfo &ci,
                                          const uint32_t *words, const uint8_t *table) {
  S.ci[b] = ci;
  uint32_t nw = 0, bytes = 0;
  const bool staged = chunk_staged(ci);
  if (staged) {
    const uint64_t up = (ci.end - ci.lo + 3) & ~3ull;
    const uint64_t avail = payload_words > ci.lo ? payload_words - ci.lo : 0;
    nw = uint32_t(up <= avail ? up : (avail & ~3ull));
    bytes = 4 * nw + uint32_t(kLeafBytes) * (ci.last - ci.first + 1);
  }
  S.ncopy[b] = nw;
  mbar_expect_tx(&S.bar[b], bytes);
  if (staged) {
    if (nw) bulk_g2s(S.buf[b].sw, words + ci.lo, 4 * nw, &S.bar[b]);
    bulk_g2s(S.buf[b].rec, table + uint64_t(kLeafBytes) * ci.first, uint32_t(kLeafBytes) * (ci.last - ci.first + 1),
             &S.bar[b]);
  }
}

// Persistent blocks; block k decodes chunks k, k + G, k + 2G, ... of kChunk
// consecutive particles (G = grid size).
//  * Thread 0 starts the copies of the block's next chunk into the other
//    staging area while the current one is decoded, and keeps the descriptor
//    of the chunk after that in flight; one block barrier per chunk.
//  * Dequantization reads the code tables (k_dtable) when they exist; the
//    particles of a leaf have nearby codes, so a warp's lookups touch few
//    cache lines.
//  * Each particle's fields are cut from a 96-bit window of the staged words
//    with funnel shifts and per-leaf masks.  A chunk of more than
//    kChunkLeaves leaves (tiny leaves) or a longer span searches the leaf table
//    and reads its words from global memory instead.
//  * A copy whose wait gives up ends the block's work (error word set).
template <typename T, bool FAST, bool VEC>
__global__ void __launch_bounds__(kDecThreads) k_decode(DecodeLaunch a) {
  __shared__ __align__(16) DecSmem S;
  // launched as the tables' programmatic dependent: they (and the validation before
  // them) are complete and visible after this wait
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (call_failed(a.err)) return;  // validation failed: write nothing
  const uint64_t nchunks = (a.n + kChunk - 1) / kChunk;
  uint64_t chunk = blockIdx.x;
  if (chunk >= nchunks) return;
  const uint8_t *table = a.stream + kHeaderBytes;
  const uint32_t *words = reinterpret_cast<const uint32_t *>(table + uint64_t(kLeafBytes) * a.num_leaves);
  const ChunkInfo *cinfo = static_cast<const ChunkInfo *>(a.chunks);
  uint32_t tb[3], te = 0;
  const bool use_table = table_fits(a.qb, tb, te);
  // table of axis d indexed by the code itself: its start minus the lowest code
  const T *tabs = static_cast<const T *>(a.tab);
  const T *tab0 = tabs + (int64_t(tb[0]) - a.qb[0]), *tab1 = tabs + (int64_t(tb[1]) - a.qb[1]),
          *tab2 = tabs + (int64_t(tb[2]) - a.qb[2]);
  const int32_t qlow0 = a.qb[0], qlow1 = a.qb[1], qlow2 = a.qb[2];
  const uint64_t G = gridDim.x;
  ChunkInfo ahead = {};  // thread 0: the descriptor of the chunk after the next one
  if (threadIdx.x == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    mbar_fence_init();
    dec_issue(a.payload_words, S, 0, cinfo[chunk], words, table);
    if (chunk + G < nchunks) ahead = cinfo[chunk + G];
  }
  __syncthreads();
  uint32_t ph0 = 0u, ph1 = 0u;
  for (int b = 0; chunk < nchunks; chunk += G, b ^= 1) {
    const bool late = wait_buffer(&S.bar[b], b ? ph1 : ph0, a.err);
    if (b) ph1 ^= 1u;
    else ph0 ^= 1u;
    const ChunkInfo ci = S.ci[b];
    const uint32_t count = ci.last - ci.first + 1;
    const bool staged = chunk_staged(ci);
    const uint64_t c0 = chunk * kChunk;
    const int32_t nloc = int32_t(((c0 + kChunk) < a.n ? (c0 + kChunk) : a.n) - c0);
    if (staged && !late) {
      if (threadIdx.x < count) {
        const int L = threadIdx.x;
        const Rec r = rec_from(S.buf[b].rec[2 * L], S.buf[b].rec[2 * L + 1]);
        LeafC lc;
        lc.rel = int32_t(int64_t(r.po) - int64_t(c0));
        lc.w = r.m[0] + r.m[1] + r.m[2];
        lc.base = int32_t(int64_t(32 * r.wo) - int64_t(32 * ci.lo) - int64_t(lc.w));
        lc.m0 = r.m[0];
        lc.s2 = r.m[0] + r.m[1];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          lc.mask[d] = (1u << r.m[d]) - 1u;
          lc.qref[d] = r.q[d];
          lc.off[d] = r.q[d] - int32_t(r.m[d] ? (1u << (r.m[d] - 1)) - 1u : 0u);
        }
        lc.pad[0] = lc.pad[1] = 0;
        S.lc[b][L] = lc;
      }
      // the words the copy did not bring (the last chunks only): the payload's tail, then zeros
      const uint32_t nst = uint32_t(ci.end - ci.lo);
      for (uint32_t w = S.ncopy[b] + threadIdx.x; w < nst; w += kDecThreads)
        S.buf[b].sw[w] = ci.lo + w < a.payload_words ? __ldg(words + ci.lo + w) : 0u;
    }
    // this chunk's constants are in place; every thread is done with the other staging area
    if (__syncthreads_or(late)) break;
    if (threadIdx.x == 0 && chunk + G < nchunks) {
      fence_proxy_async();  // earlier generic reads of that area precede the async writes
      dec_issue(a.payload_words, S, b ^ 1, ahead, words, table);
      if (chunk + 2 * G < nchunks) ahead = cinfo[chunk + 2 * G];
    }
    __align__(16) T vals[3 * kDecPer];
    int32_t qs[3 * kDecPer];  // codes of the run; unused slots hold the lowest code, a valid table index
#pragma unroll
    for (int v = 0; v < 3 * kDecPer; v += 3) {
      qs[v] = qlow0;
      qs[v + 1] = qlow1;
      qs[v + 2] = qlow2;
    }
    const int32_t sl0 = int32_t(threadIdx.x) * kDecPer;
    if (staged) {
      const uint32_t *sw = S.buf[b].sw;
      const LeafC *lcs = S.lc[b];
      // kDecPer consecutive particles per thread: one leaf lookup for the run
      if (sl0 < nloc) {
        int L = 0;
        while (L + 1 < int(count) && lcs[L + 1].rel <= sl0) ++L;
        LeafC lc = lcs[L];
        int32_t next = L + 1 < int(count) ? lcs[L + 1].rel : 0x7fffffff;
#pragma unroll
        for (int k = 0; k < kDecPer; ++k) {
          const int32_t sl = sl0 + k;
          if (sl >= nloc) continue;
          if (sl >= next) {  // the run crosses into the next leaf
            ++L;
            lc = lcs[L];
            next = L + 1 < int(count) ? lcs[L + 1].rel : 0x7fffffff;
          }
          const uint32_t i = uint32_t(sl) - uint32_t(lc.rel);
          int32_t q0, q1, q2;
          if (i == 0) {
            q0 = lc.qref[0];
            q1 = lc.qref[1];
            q2 = lc.qref[2];
          } else {
            const uint32_t bit = uint32_t(lc.base) + i * lc.w;  // modulo 2^32; the result is below 2^17
            const uint32_t wi = bit >> 5, r0 = bit & 31u;
            const uint32_t a0 = sw[wi], a1 = sw[wi + 1], a2 = sw[wi + 2], a3 = sw[wi + 3];
            const uint32_t v0 = __funnelshift_r(a0, a1, r0);  // bits [bit, bit + 96) of the payload
            const uint32_t v1 = __funnelshift_r(a1, a2, r0);
            const uint32_t v2 = __funnelshift_r(a2, a3, r0);
            const bool hi2 = lc.s2 >= 32;
            q0 = lc.off[0] + int32_t(v0 & lc.mask[0]);
            q1 = lc.off[1] + int32_t(__funnelshift_r(v0, v1, lc.m0) & lc.mask[1]);
            q2 = lc.off[2] + int32_t(__funnelshift_r(hi2 ? v1 : v0, hi2 ? v2 : v1, lc.s2) & lc.mask[2]);
          }
          qs[3 * k] = q0;
          qs[3 * k + 1] = q1;
          qs[3 * k + 2] = q2;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < kDecPer; ++k) {
        const int32_t sl = sl0 + k;
        if (sl >= nloc) continue;
        const uint64_t g = c0 + uint64_t(sl);
        // many leaves, or a span beyond the staging area: search the leaf table
        uint64_t lo = ci.first, hi = ci.last;
        while (lo < hi) {
          const uint64_t mid = (lo + hi + 1) >> 1;
          if (load_rec(table, mid).po <= g) lo = mid;
          else hi = mid - 1;
        }
        const Rec r = load_rec(table, lo);
        const uint64_t po = r.po, wo = r.wo;
        int32_t q0 = r.q[0], q1 = r.q[1], q2 = r.q[2];
        const uint32_t mm = r.m[0] | (r.m[1] << 8) | (r.m[2] << 16);
        const uint64_t i = g - po;
        if (i > 0) {
          const uint32_t w = (mm & 0xffu) + ((mm >> 8) & 0xffu) + ((mm >> 16) & 0xffu);
          const uint64_t bit = 32ull * wo + (i - 1) * uint64_t(w);
          const uint64_t wi = bit >> 5;
          add_fields(word_at(words, a.payload_words, wi), word_at(words, a.payload_words, wi + 1),
                     word_at(words, a.payload_words, wi + 2), word_at(words, a.payload_words, wi + 3),
                     uint32_t(bit & 31), mm, q0, q1, q2);
        }
        qs[3 * k] = q0;
        qs[3 * k + 1] = q1;
        qs[3 * k + 2] = q2;
      }
    }
    // dequantize the run: all lookups issued together
    if (use_table) {
#pragma unroll
      for (int v = 0; v < 3 * kDecPer; ++v) vals[v] = __ldg((v % 3 == 0 ? tab0 : (v % 3 == 1 ? tab1 : tab2)) + qs[v]);
    } else {
#pragma unroll
      for (int v = 0; v < 3 * kDecPer; ++v) vals[v] = dequant_particle<T, FAST>(a, v % 3, qs[v]);
    }
    // the run's 3 * kDecPer values are consecutive in the output
    if (sl0 < nloc) {
      T *out = static_cast<T *>(a.out) + 3 * (c0 + uint64_t(sl0));
      if (VEC && sl0 + kDecPer <= nloc) {
        constexpr int kVec = 3 * kDecPer * int(sizeof(T)) / 16;
        uint4 *o4 = reinterpret_cast<uint4 *>(out);
        const uint4 *v4 = reinterpret_cast<const uint4 *>(vals);
#pragma unroll
        for (int v = 0; v < kVec; ++v) __stcs(o4 + v, v4[v]);
      } else {
        const int m = 3 * min(kDecPer, nloc - sl0);
#pragma unroll
        for (int v = 0; v < 3 * kDecPer; ++v)
          if (v < m) out[v] = vals[v];
      }
    }
  }
  // with host_err: the last block to get here leaves the error word there (a block that
  // returned early does not count, and the host then reads the word itself)
  if (a.host_err) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(a.err + 1, 1u) == gridDim.x - 1) {
        __threadfence();
        *reinterpret_cast<volatile uint32_t *>(a.host_err) = *reinterpret_cast<volatile uint32_t *>(a.err);
        __threadfence_system();
      }
    }
  }
}

// Decoding of a stream with lossless axes, one thread per particle: its leaf
// by binary search within its chunk's leaves, every particle in the payload
// (entry i of the leaf, the centre first), x, y, z fields of m_d bits (coded:
// q = q_ref + c - (2^(m-1) - 1), then (T)(o + s q)) or M bits (the
// coordinate's own pattern).
template <typename T>
__global__ void __launch_bounds__(kDecThreads) k_decode_lossless(DecodeLaunch a) {
  if (*a.err) return;
  const uint64_t g = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= a.n) return;
  const uint8_t *table = a.stream + kHeaderBytes;
  const uint32_t *words = reinterpret_cast<const uint32_t *>(table + uint64_t(kLeafBytes) * a.num_leaves);
  const ChunkInfo ci = static_cast<const ChunkInfo *>(a.chunks)[g / kChunk];
  uint64_t lo = ci.first, hi = ci.last;
  while (lo < hi) {
    const uint64_t mid = (lo + hi + 1) >> 1;
    if (load_rec(table, mid).po <= g) lo = mid;
    else hi = mid - 1;
  }
  const Rec r = load_rec(table, lo);
  const uint32_t w = r.m[0] + r.m[1] + r.m[2];
  uint64_t bit = 32ull * r.wo + (g - r.po) * uint64_t(w);
  T *out = static_cast<T *>(a.out) + 3 * g;
  for (int d = 0; d < 3; ++d) {
    const uint32_t md = r.m[d];
    uint64_t v = 0;
    for (uint32_t t = 0; t < md; t += 32) {  // md bits from `bit` on, 32 at a time
      const uint32_t nb = min(32u, md - t);
      const uint64_t b = bit + t, wi = b >> 5;
      const uint32_t x = __funnelshift_r(word_at(words, a.payload_words, wi), word_at(words, a.payload_words, wi + 1),
                                         uint32_t(b & 31));
      v |= uint64_t(nb < 32 ? x & ((1u << nb) - 1u) : x) << t;
    }
    bit += md;
    if ((a.raw >> d) & 1u) {
      if (sizeof(T) == 4) out[d] = T(__uint_as_float(uint32_t(v)));
      else out[d] = T(__longlong_as_double((long long)v));
    } else {
      const int32_t q = r.q[d] + (md ? int32_t(v) - int32_t((1u << (md - 1)) - 1u) : 0);
      out[d] = dequant_particle<T, false>(a, d, q);
    }
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
  h[84] = uint8_t(a.raw);
  uint4 *dst = reinterpret_cast<uint4 *>(a.out);
  const uint4 *src = reinterpret_cast<const uint4 *>(h);
  for (int i = 0; i < int(kHeaderBytes / 16); ++i) dst[i] = src[i];
  *a.total_bytes = uint64_t(kHeaderBytes) + uint64_t(kLeafBytes) * a.num_leaves + 4ull * words;
}

template <typename T, bool FAST, bool VEC>
cudaError_t decode_launch(const DecodeLaunch &a, cudaStream_t st, bool tables) {
  if (tables) {
    TraceScope ts("k_dtable", st);
    k_dtable<T, FAST><<<unsigned((kTabEntries + 255) / 256), 256, 0, st>>>(a);
  }
  // persistent: as many blocks as stay resident, at most one per chunk
  int per_sm = 0;
  const cudaError_t e = resident_blocks<k_decode<T, FAST, VEC>>(kDecThreads, 0, &per_sm);
  if (e != cudaSuccess) return e;
  uint64_t grid = uint64_t(per_sm < 1 ? 1 : per_sm) * uint64_t(device_sm_count());
  if (grid > decode_chunks(a.n)) grid = decode_chunks(a.n);
  TraceScope ts("k_decode", st);
  // a programmatic dependent of the tables: its blocks are placed while they are filled
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(kDecThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_decode<T, FAST, VEC>, a);
}

template <typename T, bool FAST>
cudaError_t decode_dispatch(const DecodeLaunch &a, cudaStream_t st, bool tables = true) {
  return a.vec ? decode_launch<T, FAST, true>(a, st, tables) : decode_launch<T, FAST, false>(a, st, tables);
}


// ---- many streams: one set of launches for a batch ----

__global__ void k_gather_headers(const uint8_t *const *streams, uint32_t count, uint8_t *dst) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;  // one 16-byte word of one header
  if (i >= count * (kHeaderBytes / 16)) return;
  const uint32_t item = i / (kHeaderBytes / 16), w = i % (kHeaderBytes / 16);
  reinterpret_cast<uint4 *>(dst)[i] = __ldg(reinterpret_cast<const uint4 *>(streams[item]) + w);
}

// The batch's leaf space, a warp per step: a warp's leaves belong to one
// stream (streams start on multiples of 32), found by binary search.
__global__ void k_validate_batch(const DecItem *items, const uint64_t *leaf_start, uint32_t count, uint64_t leaves) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t base = uint64_t(blockIdx.x) * blockDim.x; base < leaves; base += stride) {
    const uint64_t wbase = base + (threadIdx.x & ~31u);
    uint32_t lo = 0, hi = count - 1;  // the last stream whose leaves start at or before the warp's
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (leaf_start[mid] <= wbase) lo = mid;
      else hi = mid - 1;
    }
    const DecodeLaunch &a = items[lo].a;
    validate_leaf(a.stream, a.n, a.num_leaves, a.payload_words, static_cast<ChunkInfo *>(a.chunks), a.err, a.qb,
                  a.raw, a.dtype == 0 ? 32u : 64u, base + threadIdx.x - leaf_start[lo]);
  }
}

// Every chunk descriptor of a stream names the stream (one grid row per
// stream), whatever its validation finds: the batched decoder reads the tag
// before it trusts anything else in a descriptor.
__global__ void k_tag_chunks(const DecItem *items, uint32_t first) {
  const uint32_t item = first + blockIdx.y;
  const DecodeLaunch &a = items[item].a;
  ChunkInfo *info = static_cast<ChunkInfo *>(a.chunks);
  const uint64_t chunks = (a.n + kChunk - 1) / kChunk;
  for (uint64_t c = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < chunks; c += uint64_t(gridDim.x) * blockDim.x)
    info[c].tag = item;
}

// One grid row per stream.
__global__ void k_dtable_batch(const DecItem *items) {
  const DecodeLaunch &a = items[blockIdx.y].a;
  if (*a.err || a.raw) return;
  if (a.dtype == 0) {
    if (a.fast) fill_table<float, true>(a);
    else fill_table<float, false>(a);
  } else {
    fill_table<double, false>(a);
  }
}

// What every thread needs of the stream of a staged chunk (thread 0 writes it
// with the chunk's copies).
struct BatchMeta {
  const DecodeLaunch *a;  // the stream's launch fields
  const uint8_t *table;   // its leaf table
  const uint32_t *words;  // its payload
  uint64_t payload_words;
  void *out;
  const void *tab[3];     // code tables indexed by the code itself (with use_table)
  uint64_t c0;            // first particle of the chunk in its stream
  int32_t nloc;           // particles of the chunk
  int32_t qlow[3];
  uint32_t use_table;
  uint32_t failed;        // the stream's validation failed: its chunks are not decoded
};
struct DecBatchSmem {
  DecSmem d;
  BatchMeta meta[2];
  // thread 0's own state, kept here rather than in every thread's registers:
  // the stream it last described and the descriptor of the chunk after the next
  BatchMeta st;
  uint64_t chunk0, n;
  uint32_t cur;
  ChunkInfo ahead;
};

// The batch's decoder for the streams of one kind: persistent blocks take the
// kind's chunks k, k + G, ... as the single-stream decoder does; a chunk's
// descriptor names its stream (k_tag_chunks), and thread 0 refreshes what it
// keeps of a stream only when the stream changes.  A staging area's record is
// read only after its barrier completes (thread 0 writes it before arriving);
// a wait that gives up sets the batch's own error word `berr`.
template <typename T, bool FAST, bool VEC>
__global__ void __launch_bounds__(kDecThreads, 5) k_decode_batch(const DecItem *items, const ChunkInfo *cinfo,
                                                              uint64_t nchunks, uint32_t *berr) {
  __shared__ __align__(16) DecBatchSmem S;
  uint64_t chunk = blockIdx.x;
  if (chunk >= nchunks) return;
  const uint64_t G = gridDim.x;
  BatchMeta &st = S.st;
  auto issue = [&](int b, uint64_t g, const ChunkInfo &ci) {
    if (ci.tag != S.cur) {
      S.cur = ci.tag;
      const DecodeLaunch &a = items[S.cur].a;
      st.a = &a;
      st.table = a.stream + kHeaderBytes;
      st.words = reinterpret_cast<const uint32_t *>(st.table + uint64_t(kLeafBytes) * a.num_leaves);
      st.payload_words = a.payload_words;
      st.out = a.out;
      uint32_t tb[3], te = 0;
      st.use_table = table_fits(a.qb, tb, te) ? 1u : 0u;
      const T *tabs = static_cast<const T *>(a.tab);
      for (int d = 0; d < 3; ++d) {
        st.qlow[d] = a.qb[d];
        st.tab[d] = tabs + (int64_t(tb[d]) - a.qb[d]);
      }
      S.chunk0 = items[S.cur].chunk0;
      S.n = a.n;
      st.failed = *reinterpret_cast<const volatile uint32_t *>(a.err) != 0u ? 1u : 0u;
    }
    st.c0 = (g - S.chunk0) * kChunk;
    st.nloc = int32_t(((st.c0 + kChunk) < S.n ? (st.c0 + kChunk) : S.n) - st.c0);
    S.meta[b] = st;
    if (st.failed) {  // nothing of the descriptor is used: an arrival without copies
      S.d.ci[b] = ci;
      S.d.ncopy[b] = 0;
      mbar_expect_tx(&S.d.bar[b], 0);
    } else {
      dec_issue(st.payload_words, S.d, b, ci, st.words, st.table);
    }
  };
  if (threadIdx.x == 0) {
    mbar_init(&S.d.bar[0], 1);
    mbar_init(&S.d.bar[1], 1);
    mbar_fence_init();
    S.cur = 0xffffffffu;
    issue(0, chunk, cinfo[chunk]);
    if (chunk + G < nchunks) S.ahead = cinfo[chunk + G];
  }
  __syncthreads();
  uint32_t ph0 = 0u, ph1 = 0u;
  for (int b = 0; chunk < nchunks; chunk += G, b ^= 1) {
    const bool late = wait_buffer(&S.d.bar[b], b ? ph1 : ph0, berr);
    if (b) ph1 ^= 1u;
    else ph0 ^= 1u;
    const ChunkInfo ci = S.d.ci[b];
    const BatchMeta &M = S.meta[b];
    const DecodeLaunch &A = *M.a;
    const bool failed = M.failed != 0;  // the descriptor may be stale: nothing of it is read
    const uint32_t count = ci.last - ci.first + 1;
    const bool staged = !failed && chunk_staged(ci);
    const uint64_t c0 = M.c0;
    const int32_t nloc = M.nloc;
    const bool use_table = M.use_table != 0;
    const T *tab0 = static_cast<const T *>(M.tab[0]), *tab1 = static_cast<const T *>(M.tab[1]),
            *tab2 = static_cast<const T *>(M.tab[2]);
    const int32_t qlow0 = M.qlow[0], qlow1 = M.qlow[1], qlow2 = M.qlow[2];
    if (staged && !late) {
      if (threadIdx.x < count) {
        const int L = threadIdx.x;
        const Rec r = rec_from(S.d.buf[b].rec[2 * L], S.d.buf[b].rec[2 * L + 1]);
        LeafC lc;
        lc.rel = int32_t(int64_t(r.po) - int64_t(c0));
        lc.w = r.m[0] + r.m[1] + r.m[2];
        lc.base = int32_t(int64_t(32 * r.wo) - int64_t(32 * ci.lo) - int64_t(lc.w));
        lc.m0 = r.m[0];
        lc.s2 = r.m[0] + r.m[1];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          lc.mask[d] = (1u << r.m[d]) - 1u;
          lc.qref[d] = r.q[d];
          lc.off[d] = r.q[d] - int32_t(r.m[d] ? (1u << (r.m[d] - 1)) - 1u : 0u);
        }
        lc.pad[0] = lc.pad[1] = 0;
        S.d.lc[b][L] = lc;
      }
      // the words the copy did not bring (the stream's last chunks only): its payload's tail, then zeros
      const uint32_t nst = uint32_t(ci.end - ci.lo);
      for (uint32_t w = S.d.ncopy[b] + threadIdx.x; w < nst; w += kDecThreads)
        S.d.buf[b].sw[w] = ci.lo + w < M.payload_words ? __ldg(M.words + ci.lo + w) : 0u;
    }
    // this chunk's constants are in place; every thread is done with the other staging area
    if (__syncthreads_or(late)) break;
    if (threadIdx.x == 0 && chunk + G < nchunks) {
      fence_proxy_async();  // earlier generic reads of that area precede the async writes
      issue(b ^ 1, chunk + G, S.ahead);
      if (chunk + 2 * G < nchunks) S.ahead = cinfo[chunk + 2 * G];
    }
    if (failed) continue;
    __align__(16) T vals[3 * kDecPer];
    int32_t qs[3 * kDecPer];  // codes of the run; unused slots hold the lowest code, a valid table index
#pragma unroll
    for (int v = 0; v < 3 * kDecPer; v += 3) {
      qs[v] = qlow0;
      qs[v + 1] = qlow1;
      qs[v + 2] = qlow2;
    }
    const int32_t sl0 = int32_t(threadIdx.x) * kDecPer;
    if (staged) {
      const uint32_t *sw = S.d.buf[b].sw;
      const LeafC *lcs = S.d.lc[b];
      // kDecPer consecutive particles per thread: one leaf lookup for the run
      if (sl0 < nloc) {
        int L = 0;
        while (L + 1 < int(count) && lcs[L + 1].rel <= sl0) ++L;
        LeafC lc = lcs[L];
        int32_t next = L + 1 < int(count) ? lcs[L + 1].rel : 0x7fffffff;
#pragma unroll
        for (int k = 0; k < kDecPer; ++k) {
          const int32_t sl = sl0 + k;
          if (sl >= nloc) continue;
          if (sl >= next) {  // the run crosses into the next leaf
            ++L;
            lc = lcs[L];
            next = L + 1 < int(count) ? lcs[L + 1].rel : 0x7fffffff;
          }
          const uint32_t i = uint32_t(sl) - uint32_t(lc.rel);
          int32_t q0, q1, q2;
          if (i == 0) {
            q0 = lc.qref[0];
            q1 = lc.qref[1];
            q2 = lc.qref[2];
          } else {
            const uint32_t bit = uint32_t(lc.base) + i * lc.w;  // modulo 2^32; the result is below 2^17
            const uint32_t wi = bit >> 5, r0 = bit & 31u;
            const uint32_t a0 = sw[wi], a1 = sw[wi + 1], a2 = sw[wi + 2], a3 = sw[wi + 3];
            const uint32_t v0 = __funnelshift_r(a0, a1, r0);  // bits [bit, bit + 96) of the payload
            const uint32_t v1 = __funnelshift_r(a1, a2, r0);
            const uint32_t v2 = __funnelshift_r(a2, a3, r0);
            const bool hi2 = lc.s2 >= 32;
            q0 = lc.off[0] + int32_t(v0 & lc.mask[0]);
            q1 = lc.off[1] + int32_t(__funnelshift_r(v0, v1, lc.m0) & lc.mask[1]);
            q2 = lc.off[2] + int32_t(__funnelshift_r(hi2 ? v1 : v0, hi2 ? v2 : v1, lc.s2) & lc.mask[2]);
          }
          qs[3 * k] = q0;
          qs[3 * k + 1] = q1;
          qs[3 * k + 2] = q2;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < kDecPer; ++k) {
        const int32_t sl = sl0 + k;
        if (sl >= nloc) continue;
        const uint64_t g = c0 + uint64_t(sl);
        // many leaves, or a span beyond the staging area: search the leaf table
        uint64_t lo = ci.first, hi = ci.last;
        while (lo < hi) {
          const uint64_t mid = (lo + hi + 1) >> 1;
          if (load_rec(M.table, mid).po <= g) lo = mid;
          else hi = mid - 1;
        }
        const Rec r = load_rec(M.table, lo);
        const uint64_t po = r.po, wo = r.wo;
        int32_t q0 = r.q[0], q1 = r.q[1], q2 = r.q[2];
        const uint32_t mm = r.m[0] | (r.m[1] << 8) | (r.m[2] << 16);
        const uint64_t i = g - po;
        if (i > 0) {
          const uint32_t w = (mm & 0xffu) + ((mm >> 8) & 0xffu) + ((mm >> 16) & 0xffu);
          const uint64_t bit = 32ull * wo + (i - 1) * uint64_t(w);
          const uint64_t wi = bit >> 5;
          add_fields(word_at(M.words, M.payload_words, wi), word_at(M.words, M.payload_words, wi + 1),
                     word_at(M.words, M.payload_words, wi + 2), word_at(M.words, M.payload_words, wi + 3),
                     uint32_t(bit & 31), mm, q0, q1, q2);
        }
        qs[3 * k] = q0;
        qs[3 * k + 1] = q1;
        qs[3 * k + 2] = q2;
      }
    }
    // dequantize the run: all lookups issued together
    if (use_table) {
#pragma unroll
      for (int v = 0; v < 3 * kDecPer; ++v) vals[v] = __ldg((v % 3 == 0 ? tab0 : (v % 3 == 1 ? tab1 : tab2)) + qs[v]);
    } else {
#pragma unroll
      for (int v = 0; v < 3 * kDecPer; ++v) vals[v] = dequant_particle<T, FAST>(A, v % 3, qs[v]);
    }
    // the run's 3 * kDecPer values are consecutive in the output
    if (sl0 < nloc) {
      T *out = static_cast<T *>(M.out) + 3 * (c0 + uint64_t(sl0));
      if (VEC && sl0 + kDecPer <= nloc) {
        constexpr int kVec = 3 * kDecPer * int(sizeof(T)) / 16;
        uint4 *o4 = reinterpret_cast<uint4 *>(out);
        const uint4 *v4 = reinterpret_cast<const uint4 *>(vals);
#pragma unroll
        for (int v = 0; v < kVec; ++v) __stcs(o4 + v, v4[v]);
      } else {
        const int m = 3 * min(kDecPer, nloc - sl0);
#pragma unroll
        for (int v = 0; v < 3 * kDecPer; ++v)
          if (v < m) out[v] = vals[v];
      }
    }
  }
}
}  // namespace

uint64_t decode_chunks(uint64_t n) { return (n + kChunk - 1) / kChunk; }
uint64_t decode_table_bytes() { return uint64_t(kTabEntries) * sizeof(double); }
uint64_t decode_chunk_bytes(uint64_t n) { return decode_chunks(n) * sizeof(ChunkInfo); }

cudaError_t launch_header(const HeaderLaunch &a, cudaStream_t st) {
  TraceScope ts("k_header", st);
  k_header<<<1, 1, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gather_headers(const uint8_t *const *streams, uint32_t count, uint8_t *dst, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const uint32_t words = count * (kHeaderBytes / 16);
  k_gather_headers<<<(words + 255) / 256, 256, 0, st>>>(streams, count, dst);
  return cudaGetLastError();
}

cudaError_t launch_validate_batch(const DecItem *items, const uint64_t *leaf_start, uint32_t count, uint64_t leaves,
                                  cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  TraceScope ts("k_validate", st);
  for (uint32_t first = 0; first < count; first += 65535u) {  // one grid row per stream
    const uint32_t rows = count - first < 65535u ? count - first : 65535u;
    k_tag_chunks<<<dim3(8, rows), 256, 0, st>>>(items, first);
  }
  if (leaves) k_validate_batch<<<unsigned(8 * device_sm_count()), 64, 0, st>>>(items, leaf_start, count, leaves);
  return cudaGetLastError();
}

cudaError_t launch_dtable_batch(const DecItem *items, uint32_t count, cudaStream_t st) {
  TraceScope ts("k_dtable", st);
  for (uint32_t first = 0; first < count; first += 65535u) {  // one grid row per stream
    const uint32_t rows = count - first < 65535u ? count - first : 65535u;
    k_dtable_batch<<<dim3((kTabEntries + 255) / 256, rows), 256, 0, st>>>(items + first);
  }
  return cudaGetLastError();
}

namespace {
template <typename T, bool FAST, bool VEC>
cudaError_t decode_batch_as(const DecItem *items, const void *chunks, uint64_t num_chunks, uint32_t *berr,
                            cudaStream_t st) {
  int per_sm = 0;
  const cudaError_t e = resident_blocks<k_decode_batch<T, FAST, VEC>>(kDecThreads, 0, &per_sm);
  if (e != cudaSuccess) return e;
  uint64_t grid = uint64_t(per_sm < 1 ? 1 : per_sm) * uint64_t(device_sm_count());
  if (grid > num_chunks) grid = num_chunks;
  TraceScope ts("k_decode", st);
  k_decode_batch<T, FAST, VEC><<<unsigned(grid), kDecThreads, 0, st>>>(items, static_cast<const ChunkInfo *>(chunks),
                                                                       num_chunks, berr);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_decode_batch(int kind, bool vec, const DecItem *items, const void *chunks, uint64_t num_chunks,
                                uint32_t *berr, cudaStream_t st) {
  if (num_chunks == 0) return cudaSuccess;
  switch (kind) {
    case kDecKindF32Fast:
      return vec ? decode_batch_as<float, true, true>(items, chunks, num_chunks, berr, st)
                 : decode_batch_as<float, true, false>(items, chunks, num_chunks, berr, st);
    case kDecKindF32:
      return vec ? decode_batch_as<float, false, true>(items, chunks, num_chunks, berr, st)
                 : decode_batch_as<float, false, false>(items, chunks, num_chunks, berr, st);
    default:
      return vec ? decode_batch_as<double, false, true>(items, chunks, num_chunks, berr, st)
                 : decode_batch_as<double, false, false>(items, chunks, num_chunks, berr, st);
  }
}

cudaError_t launch_decode_lossless(const DecodeLaunch &a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  TraceScope ts("k_decode", st);
  const unsigned grid = unsigned((a.n + kDecThreads - 1) / kDecThreads);
  if (a.dtype == 0) k_decode_lossless<float><<<grid, kDecThreads, 0, st>>>(a);
  else k_decode_lossless<double><<<grid, kDecThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_decode_start(const uint8_t *stream, uint32_t *ws64, uint8_t *host_header, cudaStream_t st) {
  TraceScope ts("k_decode_start", st);
  k_decode_start<<<1, 32, 0, st>>>(stream, ws64, host_header);
  return cudaGetLastError();
}

cudaError_t launch_decode_prologue(const uint8_t *stream, uint64_t stream_bytes, uint64_t chunk_cap, uint32_t *err,
                                   int32_t *qb, void *tab, void *chunks, cudaStream_t st) {
  {
    TraceScope ts("k_validate", st);
    k_validate_dev<<<unsigned(4 * device_sm_count()), 256, 0, st>>>(stream, stream_bytes, chunk_cap,
                                                                    static_cast<ChunkInfo *>(chunks), err, qb);
  }
  TraceScope ts("k_dtable", st);
  k_dtable_dev<<<unsigned((kTabEntries + 255) / 256), 256, 0, st>>>(stream, stream_bytes, err, qb, tab);
  return cudaGetLastError();
}

cudaError_t launch_decode(const DecodeLaunch &a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  if (a.prologue_done) {  // validation and tables already launched (launch_decode_prologue)
    if (a.raw) return launch_decode_lossless(a, st);
    if (a.dtype == 0) return a.fast ? decode_dispatch<float, true>(a, st, false) : decode_dispatch<float, false>(a, st, false);
    return decode_dispatch<double, false>(a, st, false);
  }
  {
    TraceScope ts("k_validate", st);
    // 64 threads a block: the leaves spread over every SM (each thread waits on its records)
    k_validate<<<unsigned((a.num_leaves + 63) / 64), 64, 0, st>>>(a.stream, a.n, a.num_leaves, a.payload_words,
                                                                      static_cast<ChunkInfo *>(a.chunks), a.err, a.qb,
                                                                      a.raw, a.dtype == 0 ? 32u : 64u);
  }
  if (a.raw) {
    TraceScope ts("k_decode", st);
    const unsigned grid = unsigned((a.n + kDecThreads - 1) / kDecThreads);
    if (a.dtype == 0) k_decode_lossless<float><<<grid, kDecThreads, 0, st>>>(a);
    else k_decode_lossless<double><<<grid, kDecThreads, 0, st>>>(a);
    return cudaGetLastError();
  }
  if (a.dtype == 0) return a.fast ? decode_dispatch<float, true>(a, st) : decode_dispatch<float, false>(a, st);
  return decode_dispatch<double, false>(a, st);
}

}  // namespace pcx
