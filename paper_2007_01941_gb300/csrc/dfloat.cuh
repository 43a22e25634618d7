// Paired-FP32 ("double-float") scalars for the mixed-precision path.
//
// A value is carried as hi + lo, two floats with |lo| <= ulp(hi) / 2 after every
// operation, which holds about 48 significant bits.  Products use Dekker's exact
// product through fma, sums Knuth's two-sum; the __f*_rn intrinsics keep the compiler
// from fusing the steps of these error-free transformations into other operations.
// This GPU issues FP32 instructions at 58 times its FP64 rate, so FP64-accurate
// arithmetic that is bound by its instruction count runs several times faster this way.
#pragma once

#include <cuda_runtime.h>

#include "device_util.cuh"

namespace ba {

struct DF {
  float h, l;
  DF() = default;
  __device__ __forceinline__ constexpr DF(float hi, float lo) : h(hi), l(lo) {}
  // exact for literals representable as a float; others are split
  __device__ __forceinline__ explicit DF(double x) { split_double(x, h, l); }
};

__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {   // requires |a| >= |b|
  const float s = __fadd_rn(a, b);
  return DF(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ DF operator+(DF a, DF b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return df_fast_two_sum(s, __fadd_rn(err, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ DF operator-(DF a) { return DF(-a.h, -a.l); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }

__device__ __forceinline__ DF operator*(DF a, DF b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return df_fast_two_sum(p, e);
}

// a / b: quotient of the heads, then one correction from the exact remainder
__device__ __forceinline__ DF operator/(DF a, DF b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  const DF r = a - b * DF(q1, 0.f);
  const float q2 = __fdiv_rn(r.h, b.h);
  return df_fast_two_sum(q1, q2);
}

__device__ __forceinline__ DF& operator+=(DF& a, DF b) { return a = a + b; }
__device__ __forceinline__ DF& operator-=(DF& a, DF b) { return a = a - b; }

__device__ __forceinline__ DF df_sqrt(DF a) {
  if (!(a.h > 0.f)) return DF(0.f, 0.f);
  const float s = __fsqrt_rn(a.h);
  const DF r = a - DF(s, 0.f) * DF(s, 0.f);
  return df_fast_two_sum(s, __fdiv_rn(r.h, __fmul_rn(2.f, s)));
}

__device__ __forceinline__ bool operator!=(DF a, float b) { return a.h != b || a.l != 0.f; }

// exact float -> double by integer bit operations (zeros and subnormals to signed zero,
// infinities and NaNs keep their class)
__device__ __forceinline__ double df_f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned s = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const unsigned ed = e == 0xffu ? 0x7ffu : e + 896u;
  const unsigned hi = e == 0u ? s : (s | (ed << 20) | (m >> 3));
  const unsigned lo = e == 0u ? 0u : (m & 7u) << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// hi + lo as one double (one FP64 addition, exact up to the double's last bit)
__device__ __forceinline__ double to_double(DF a) { return df_f2d(a.h) + df_f2d(a.l); }

__device__ __forceinline__ DF to_df(double x) { return DF(x); }
__device__ __forceinline__ double to_double(double x) { return x; }

// sum over the warp (every lane gets the total)
__device__ __forceinline__ DF warp_sum_df(DF v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += DF(__shfl_xor_sync(kFull, v.h, d), __shfl_xor_sync(kFull, v.l, d));
  return v;
}

// a += x * y with the product exact (Dekker through fma) and the running sum kept as an
// unnormalised head s and correction c (two-sum of s and the product's head; its error
// and the product's tail go into c), the compensated dot product of Ogita, Rump and
// Oishi carried over DF operands
__device__ __forceinline__ void dot2_fma(float& s, float& c, float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, e);
  e = __fmaf_rn(x.y, y.x, e);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}
__device__ __forceinline__ void dot2_fma(float& s, float& c, DF x, DF y) {
  dot2_fma(s, c, make_float2(x.h, x.l), make_float2(y.h, y.l));
}

// In-place Gauss-Jordan inverse of a BS x BS block without pivoting (the block is SPD),
// held by BS lanes of a warp: lane base + j keeps column j, with row (k + i) mod BS of it
// in a[i] during step k.  Step k takes the pivot and column k from lane base + k by
// shuffles; the rows then rotate by one register, so the pivot row is always a[0] and
// BS rotations restore the order.  The step loop stays rolled: unrolled over the pivots
// the code outgrows the instruction cache, and each warp runs it once.  Every lane of the
// warp must call it (full-mask shuffles); returns false if a pivot is not positive.
template <int BS>
__device__ __forceinline__ bool df_gauss_jordan_cols(DF (&a)[BS], int base, int j) {
  bool ok = true;
#pragma unroll 1
  for (int k = 0; k < BS; ++k) {
    const int src = base + k;
    const DF p(__shfl_sync(kFull, a[0].h, src), __shfl_sync(kFull, a[0].l, src));
    if (!(p.h > 0.f)) ok = false;
    const DF ip = DF(1.f, 0.f) / p;
    const bool piv = j == k;
    // row k: a_kj / p; column k: -a_ik / p (the pivot lane, from a zero start); others
    // a_ij - a_ik (a_kj / p)
    const DF f = piv ? ip : a[0] * ip;
#pragma unroll
    for (int i = 1; i < BS; ++i) {
      const DF ci(__shfl_sync(kFull, a[i].h, src), __shfl_sync(kFull, a[i].l, src));
      a[i - 1] = (piv ? DF(0.f, 0.f) : a[i]) - ci * f;
    }
    a[BS - 1] = f;
  }
  return ok;
}

}  // namespace ba
