// Value range and quantization kernels (Sec. 3 of arXiv 2404.02826).
//
// Range: per-axis min / max of the input and a non-finite check, in the input
// type (min and max are exact), reduced per block and then by one block.
//
// Quantize: q_d = rint(((double)p_d - o_d) / s), round-half-even, one double
// division, exactly as the definition states.  GB300 runs FP64 at a small
// fraction of FP32, so for float input the kernel evaluates the same rule on
// the FP32 pipe: p - o is split exactly into dh + dl (TwoSum), multiplied by
// 1/s held as a float pair, and rounded; whenever the fractional part lies
// within 2^-20 of one half, the literal double-precision expression decides.
// Outside that window the float-pair value is within 2^-21 of the exact
// quotient (codes < 2^22), so it and the double-precision quotient round to
// the same integer.  For double input the subtraction stays in double, the
// quotient is formed as (p - o) * fl(1/s) and rounded with integer operations
// on its bits; within 2^-20 of one half (products are within 2^-51 relative,
// so under 2^-20 absolute, of the double quotient) the division decides.
// Codes are written as structure-of-arrays (u16 or u32).
#include <cfloat>
#include <cstdint>

#include "pc_internal.cuh"

namespace pcx {
namespace {

constexpr int kThreads = 256;

// -------------------------------------------------------------------------
// range
// -------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long f64_key(double v) {
  unsigned long long b = __double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double f64_from_key(unsigned long long k) {
  unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double(b);
}
__device__ __forceinline__ bool f64_bad(double v) {
  return ((__double_as_longlong(v) >> 52) & 0x7ff) == 0x7ff;
}

struct F32Acc {
  float mn[3], mx[3];
  bool bad;
  __device__ void init() {
    for (int d = 0; d < 3; ++d) {
      mn[d] = FLT_MAX;
      mx[d] = -FLT_MAX;
    }
    bad = false;
  }
  __device__ __forceinline__ void add(int d, float v) {
    bad |= !(fabsf(v) <= FLT_MAX);
    mn[d] = fminf(mn[d], v);
    mx[d] = fmaxf(mx[d], v);
  }
};

struct F64Acc {
  unsigned long long mn[3], mx[3];
  bool bad;
  __device__ void init() {
    for (int d = 0; d < 3; ++d) {
      mn[d] = ~0ull;
      mx[d] = 0ull;
    }
    bad = false;
  }
  __device__ __forceinline__ void add(int d, double v) {
    bad |= f64_bad(v);
    unsigned long long k = f64_key(v);
    mn[d] = k < mn[d] ? k : mn[d];
    mx[d] = k > mx[d] ? k : mx[d];
  }
};

template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_range_f32(const float *__restrict__ pos, uint64_t n,
                                                        double *__restrict__ partial) {
  F32Acc acc;
  acc.init();
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  uint64_t done = 0;
  if (VEC) {
    const float4 *p4 = reinterpret_cast<const float4 *>(pos);
    const uint64_t groups = n / 4;  // 4 particles = 3 float4
    for (uint64_t g = tid; g < groups; g += stride) {
      float4 a = __ldcs(p4 + 3 * g), b = __ldcs(p4 + 3 * g + 1), c = __ldcs(p4 + 3 * g + 2);
      acc.add(0, a.x); acc.add(1, a.y); acc.add(2, a.z); acc.add(0, a.w);
      acc.add(1, b.x); acc.add(2, b.y); acc.add(0, b.z); acc.add(1, b.w);
      acc.add(2, c.x); acc.add(0, c.y); acc.add(1, c.z); acc.add(2, c.w);
    }
    done = groups * 4;
  }
  for (uint64_t i = done + tid; i < n; i += stride)
    for (int d = 0; d < 3; ++d) acc.add(d, pos[3 * i + d]);

  __shared__ float smn[3][kThreads / 32], smx[3][kThreads / 32];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  for (int d = 0; d < 3; ++d) {
    float a = acc.mn[d], b = acc.mx[d];
    for (int o = 16; o; o >>= 1) {
      a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if ((threadIdx.x & 31) == 0) {
      smn[d][threadIdx.x >> 5] = a;
      smx[d][threadIdx.x >> 5] = b;
    }
  }
  if (acc.bad) sbad = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    double *out = partial + 8 * blockIdx.x;
    for (int d = 0; d < 3; ++d) {
      float a = smn[d][0], b = smx[d][0];
      for (int w = 1; w < kThreads / 32; ++w) {
        a = fminf(a, smn[d][w]);
        b = fmaxf(b, smx[d][w]);
      }
      out[d] = a;
      out[3 + d] = b;
    }
    out[6] = sbad ? 1.0 : 0.0;
  }
}

template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_range_f64(const double *__restrict__ pos, uint64_t n,
                                                        double *__restrict__ partial) {
  F64Acc acc;
  acc.init();
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  uint64_t done = 0;
  if (VEC) {
    const double2 *p2 = reinterpret_cast<const double2 *>(pos);
    const uint64_t groups = n / 2;  // 2 particles = 3 double2
    for (uint64_t g = tid; g < groups; g += stride) {
      double2 a = __ldcs(p2 + 3 * g), b = __ldcs(p2 + 3 * g + 1), c = __ldcs(p2 + 3 * g + 2);
      acc.add(0, a.x); acc.add(1, a.y); acc.add(2, b.x);
      acc.add(0, b.y); acc.add(1, c.x); acc.add(2, c.y);
    }
    done = groups * 2;
  }
  for (uint64_t i = done + tid; i < n; i += stride)
    for (int d = 0; d < 3; ++d) acc.add(d, pos[3 * i + d]);

  __shared__ unsigned long long smn[3][kThreads / 32], smx[3][kThreads / 32];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  for (int d = 0; d < 3; ++d) {
    unsigned long long a = acc.mn[d], b = acc.mx[d];
    for (int o = 16; o; o >>= 1) {
      unsigned long long x = __shfl_xor_sync(0xffffffffu, a, o), y = __shfl_xor_sync(0xffffffffu, b, o);
      a = x < a ? x : a;
      b = y > b ? y : b;
    }
    if ((threadIdx.x & 31) == 0) {
      smn[d][threadIdx.x >> 5] = a;
      smx[d][threadIdx.x >> 5] = b;
    }
  }
  if (acc.bad) sbad = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    double *out = partial + 8 * blockIdx.x;
    for (int d = 0; d < 3; ++d) {
      unsigned long long a = smn[d][0], b = smx[d][0];
      for (int w = 1; w < kThreads / 32; ++w) {
        a = smn[d][w] < a ? smn[d][w] : a;
        b = smx[d][w] > b ? smx[d][w] : b;
      }
      out[d] = f64_from_key(a);
      out[3 + d] = f64_from_key(b);
    }
    out[6] = sbad ? 1.0 : 0.0;
  }
}

// One block folds the per-block partials.  Comparisons go through the same
// order-preserving integer keys, so no FP64 arithmetic is involved.
__global__ void k_range_final(const double *__restrict__ partial, int blocks, RangeResult *__restrict__ res) {
  __shared__ unsigned long long smn[3][32], smx[3][32];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  unsigned long long mn[3], mx[3];
  bool bad = false;
  for (int d = 0; d < 3; ++d) {
    mn[d] = ~0ull;
    mx[d] = 0;
  }
  for (int b = threadIdx.x; b < blocks; b += blockDim.x) {
    const double *p = partial + 8 * b;
    for (int d = 0; d < 3; ++d) {
      unsigned long long a = f64_key(p[d]), c = f64_key(p[3 + d]);
      mn[d] = a < mn[d] ? a : mn[d];
      mx[d] = c > mx[d] ? c : mx[d];
    }
    bad |= p[6] != 0.0;
  }
  for (int d = 0; d < 3; ++d) {
    unsigned long long a = mn[d], b = mx[d];
    for (int o = 16; o; o >>= 1) {
      unsigned long long x = __shfl_xor_sync(0xffffffffu, a, o), y = __shfl_xor_sync(0xffffffffu, b, o);
      a = x < a ? x : a;
      b = y > b ? y : b;
    }
    if ((threadIdx.x & 31) == 0) {
      smn[d][threadIdx.x >> 5] = a;
      smx[d][threadIdx.x >> 5] = b;
    }
  }
  if (bad) sbad = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int warps = blockDim.x / 32;
    for (int d = 0; d < 3; ++d) {
      unsigned long long a = smn[d][0], b = smx[d][0];
      for (int w = 1; w < warps; ++w) {
        a = smn[d][w] < a ? smn[d][w] : a;
        b = smx[d][w] > b ? smx[d][w] : b;
      }
      res->lo[d] = f64_from_key(a);
      res->hi[d] = f64_from_key(b);
    }
    res->nonfinite = sbad ? 1u : 0u;
    res->pad = 0;
  }
}

// -------------------------------------------------------------------------
// quantize
// -------------------------------------------------------------------------

// The definition: one double subtraction, one double division, rint.
__device__ __forceinline__ uint32_t quant_exact(double p, double o, double s) {
  return (uint32_t)rint(__ddiv_rn(__dsub_rn(p, o), s));
}

// Out of line, so that the rare fallback stays a branch and is not evaluated
// speculatively on the narrow FP64 pipe.
__device__ __noinline__ uint32_t quant_exact_call(float p, double o, double s) { return quant_exact((double)p, o, s); }

// Same result for float input, evaluated on the FP32 pipe (see file comment).
__device__ __forceinline__ uint32_t quant_fast(float p, float o, double od, double s, float rh, float rl) {
  // TwoSum(p, -o): dh + dl == p - o exactly.
  float dh = __fsub_rn(p, o);
  float bb = __fsub_rn(dh, p);
  float dl = __fadd_rn(__fsub_rn(p, __fsub_rn(dh, bb)), __fsub_rn(-o, bb));
  // (dh + dl) * (rh + rl): th exact product head, tl the small remainder.
  float th = __fmul_rn(dh, rh);
  float pe = __fmaf_rn(dh, rh, -th);
  float tl = __fmaf_rn(dh, rl, __fmaf_rn(dl, rh, pe));
  float q0 = rintf(th);
  float r = __fadd_rn(__fsub_rn(th, q0), tl);
  if (__builtin_expect(fabsf(r) < 0.5f - 0x1p-20f, 1)) return (uint32_t)q0;
  return quant_exact_call(p, od, s);
}

__device__ __noinline__ uint32_t quant_exact_call64(double p, double o, double s) { return quant_exact(p, o, s); }

// Same result for double input with two double operations: t = (p - o) * inv
// and the round-to-nearest-even of t taken from its bits (t >= 0, as o is the
// minimum), unless t lies within 2^-20 of a half-integer or at 2^31 or above.
__device__ __forceinline__ uint32_t quant_fast64(double p, double o, double s, double inv) {
  const double t = __dmul_rn(__dsub_rn(p, o), inv);
  const unsigned long long b = (unsigned long long)__double_as_longlong(t);
  const int e = int((b >> 52) & 0x7ff) - 1023;  // t in [2^e, 2^(e+1))
  const unsigned long long mant = (b & 0xfffffffffffffull) | (1ull << 52);
  uint32_t q = 0;
  bool ok;
  if (e <= -3) {
    ok = true;  // t < 1/4
  } else if (e == -2) {
    ok = (b & 0xfffffffffffffull) < (1ull << 52) - (1ull << 34);  // t < 1/2 - 2^-20
  } else if (e <= 30) {
    const int F = 52 - e;  // fraction bits of t, 22 .. 53
    const unsigned long long fr = mant & ((1ull << F) - 1), half = 1ull << (F - 1), mg = 1ull << (F - 20);
    ok = fr + mg < half || fr > half + mg;
    q = uint32_t(mant >> F) + (fr > half ? 1u : 0u);
  } else {
    ok = false;
  }
  if (__builtin_expect(ok, 1)) return q;
  return quant_exact_call64(p, o, s);
}

template <typename C>
struct CodeVec;
template <>
struct CodeVec<uint16_t> {
  static __device__ __forceinline__ void put4(uint16_t *q, uint64_t i, uint32_t a, uint32_t b, uint32_t c,
                                              uint32_t d) {
    uint2 v;
    v.x = a | (b << 16);
    v.y = c | (d << 16);
    __stcs(reinterpret_cast<uint2 *>(q + i), v);
  }
  static __device__ __forceinline__ void put2(uint16_t *q, uint64_t i, uint32_t a, uint32_t b) {
    __stcs(reinterpret_cast<unsigned int *>(q + i), a | (b << 16));
  }
};
template <>
struct CodeVec<uint32_t> {
  static __device__ __forceinline__ void put4(uint32_t *q, uint64_t i, uint32_t a, uint32_t b, uint32_t c,
                                              uint32_t d) {
    __stcs(reinterpret_cast<uint4 *>(q + i), make_uint4(a, b, c, d));
  }
  static __device__ __forceinline__ void put2(uint32_t *q, uint64_t i, uint32_t a, uint32_t b) {
    __stcs(reinterpret_cast<uint2 *>(q + i), make_uint2(a, b));
  }
};

template <typename C, bool VEC, bool FAST>
__global__ void __launch_bounds__(kThreads) k_quant_f32(const float *__restrict__ pos, uint64_t n, QuantParams qp,
                                                        C *__restrict__ qx, C *__restrict__ qy, C *__restrict__ qz,
                                                        uint32_t *__restrict__ idx) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  auto Q = [&](float p, int d) -> uint32_t {
    if (FAST) return quant_fast(p, qp.of[d], qp.o[d], qp.s, qp.rh, qp.rl);
    return quant_exact((double)p, qp.o[d], qp.s);
  };
  uint64_t done = 0;
  if (VEC) {
    const float4 *p4 = reinterpret_cast<const float4 *>(pos);
    const uint64_t groups = n / 4;
    for (uint64_t g = tid; g < groups; g += stride) {
      float4 a = __ldcs(p4 + 3 * g), b = __ldcs(p4 + 3 * g + 1), c = __ldcs(p4 + 3 * g + 2);
      // particles 4g..4g+3: (a.x a.y a.z) (a.w b.x b.y) (b.z b.w c.x) (c.y c.z c.w)
      CodeVec<C>::put4(qx, 4 * g, Q(a.x, 0), Q(a.w, 0), Q(b.z, 0), Q(c.y, 0));
      CodeVec<C>::put4(qy, 4 * g, Q(a.y, 1), Q(b.x, 1), Q(b.w, 1), Q(c.z, 1));
      CodeVec<C>::put4(qz, 4 * g, Q(a.z, 2), Q(b.y, 2), Q(c.x, 2), Q(c.w, 2));
      if (idx) __stcs(reinterpret_cast<uint4 *>(idx + 4 * g),
                      make_uint4(uint32_t(4 * g), uint32_t(4 * g + 1), uint32_t(4 * g + 2), uint32_t(4 * g + 3)));
    }
    done = groups * 4;
  }
  for (uint64_t i = done + tid; i < n; i += stride) {
    qx[i] = (C)Q(pos[3 * i + 0], 0);
    qy[i] = (C)Q(pos[3 * i + 1], 1);
    qz[i] = (C)Q(pos[3 * i + 2], 2);
    if (idx) idx[i] = uint32_t(i);
  }
}

template <typename C, bool VEC, bool FAST>
__global__ void __launch_bounds__(kThreads) k_quant_f64(const double *__restrict__ pos, uint64_t n, QuantParams qp,
                                                        C *__restrict__ qx, C *__restrict__ qy, C *__restrict__ qz,
                                                        uint32_t *__restrict__ idx) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  auto quant_exact = [&](double p, double o, double s) -> uint32_t {
    if (FAST) return quant_fast64(p, o, s, qp.inv);
    return pcx::quant_exact(p, o, s);
  };
  uint64_t done = 0;
  if (VEC) {
    const double2 *p2 = reinterpret_cast<const double2 *>(pos);
    const uint64_t groups = n / 2;
    for (uint64_t g = tid; g < groups; g += stride) {
      double2 a = __ldcs(p2 + 3 * g), b = __ldcs(p2 + 3 * g + 1), c = __ldcs(p2 + 3 * g + 2);
      CodeVec<C>::put2(qx, 2 * g, quant_exact(a.x, qp.o[0], qp.s), quant_exact(b.y, qp.o[0], qp.s));
      CodeVec<C>::put2(qy, 2 * g, quant_exact(a.y, qp.o[1], qp.s), quant_exact(c.x, qp.o[1], qp.s));
      CodeVec<C>::put2(qz, 2 * g, quant_exact(b.x, qp.o[2], qp.s), quant_exact(c.y, qp.o[2], qp.s));
      if (idx) __stcs(reinterpret_cast<uint2 *>(idx + 2 * g), make_uint2(uint32_t(2 * g), uint32_t(2 * g + 1)));
    }
    done = groups * 2;
  }
  for (uint64_t i = done + tid; i < n; i += stride) {
    qx[i] = (C)quant_exact(pos[3 * i + 0], qp.o[0], qp.s);
    qy[i] = (C)quant_exact(pos[3 * i + 1], qp.o[1], qp.s);
    qz[i] = (C)quant_exact(pos[3 * i + 2], qp.o[2], qp.s);
    if (idx) idx[i] = uint32_t(i);
  }
}

// Streams with lossless axes (Sec. 4.1, m_d > M): a coded axis takes the
// definition's code, a lossless axis the split key floor((p - lo) / span * 2^29)
// in [0, 2^29] (the coordinate itself is stored by the packing).  Codes are u32.
__device__ __forceinline__ uint32_t raw_key(double p, double lo, double span) {
  if (!(span > 0.0)) return 0u;
  double t = floor(__dmul_rn(__ddiv_rn(__dsub_rn(p, lo), span), 536870912.0));
  t = t < 0.0 ? 0.0 : (t > 536870912.0 ? 536870912.0 : t);
  return uint32_t(t);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_quant_lossless(const T *__restrict__ pos, uint64_t n, QuantParams qp,
                                                             uint32_t *__restrict__ qx, uint32_t *__restrict__ qy,
                                                             uint32_t *__restrict__ qz, uint32_t *__restrict__ idx) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint32_t q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double p = (double)pos[3 * i + d];
      q[d] = (qp.raw >> d) & 1u ? raw_key(p, qp.lo[d], qp.span[d]) : quant_exact(p, qp.o[d], qp.s);
    }
    qx[i] = q[0];
    qy[i] = q[1];
    qz[i] = q[2];
    if (idx) idx[i] = uint32_t(i);
  }
}

template <typename C>
cudaError_t quant_dispatch(const QuantLaunch &a, cudaStream_t st) {
  C *qx = static_cast<C *>(a.q[0]), *qy = static_cast<C *>(a.q[1]), *qz = static_cast<C *>(a.q[2]);
  TraceScope ts("k_quantize", st);
  if (a.dtype == 0) {
    const float *p = static_cast<const float *>(a.pos);
    if (a.vec && a.fast) k_quant_f32<C, true, true><<<a.blocks, kThreads, 0, st>>>(p, a.n, a.qp, qx, qy, qz, a.idx);
    else if (a.vec) k_quant_f32<C, true, false><<<a.blocks, kThreads, 0, st>>>(p, a.n, a.qp, qx, qy, qz, a.idx);
    else if (a.fast) k_quant_f32<C, false, true><<<a.blocks, kThreads, 0, st>>>(p, a.n, a.qp, qx, qy, qz, a.idx);
    else k_quant_f32<C, false, false><<<a.blocks, kThreads, 0, st>>>(p, a.n, a.qp, qx, qy, qz, a.idx);
  } else {
    const double *p = static_cast<const double *>(a.pos);
    if (a.fast) {
      if (a.vec) k_quant_f64<C, true, true><<<a.blocks, kThreads, 0, st>>>(p, a.n, a.qp, qx, qy, qz, a.idx);
      else k_quant_f64<C, false, true><<<a.blocks, kThreads, 0, st>>>(p, a.n, a.qp, qx, qy, qz, a.idx);
    } else {
      if (a.vec) k_quant_f64<C, true, false><<<a.blocks, kThreads, 0, st>>>(p, a.n, a.qp, qx, qy, qz, a.idx);
      else k_quant_f64<C, false, false><<<a.blocks, kThreads, 0, st>>>(p, a.n, a.qp, qx, qy, qz, a.idx);
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_range(const RangeLaunch &a, cudaStream_t st) {
  TraceScope ts("k_range", st);
  if (a.dtype == 0) {
    const float *p = static_cast<const float *>(a.pos);
    if (a.vec) k_range_f32<true><<<a.blocks, kThreads, 0, st>>>(p, a.n, a.partial);
    else k_range_f32<false><<<a.blocks, kThreads, 0, st>>>(p, a.n, a.partial);
  } else {
    const double *p = static_cast<const double *>(a.pos);
    if (a.vec) k_range_f64<true><<<a.blocks, kThreads, 0, st>>>(p, a.n, a.partial);
    else k_range_f64<false><<<a.blocks, kThreads, 0, st>>>(p, a.n, a.partial);
  }
  k_range_final<<<1, 1024, 0, st>>>(a.partial, a.blocks, a.result);
  return cudaGetLastError();
}

cudaError_t launch_quantize(const QuantLaunch &a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  if (a.qp.raw) {
    if (a.code_bytes != 4) return cudaErrorInvalidValue;
    uint32_t *qx = static_cast<uint32_t *>(a.q[0]), *qy = static_cast<uint32_t *>(a.q[1]),
             *qz = static_cast<uint32_t *>(a.q[2]);
    TraceScope ts("k_quantize", st);
    if (a.dtype == 0)
      k_quant_lossless<float><<<a.blocks, kThreads, 0, st>>>(static_cast<const float *>(a.pos), a.n, a.qp, qx, qy,
                                                              qz, a.idx);
    else
      k_quant_lossless<double><<<a.blocks, kThreads, 0, st>>>(static_cast<const double *>(a.pos), a.n, a.qp, qx,
                                                               qy, qz, a.idx);
    return cudaGetLastError();
  }
  return a.code_bytes == 2 ? quant_dispatch<uint16_t>(a, st) : quant_dispatch<uint32_t>(a, st);
}

}  // namespace pcx
