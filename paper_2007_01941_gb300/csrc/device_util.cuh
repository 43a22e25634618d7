// Device-side helpers shared by the kernels: warp/block reductions, the
// deterministic two-stage grid reduction and small dense block routines.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ba {

constexpr unsigned kFull = 0xffffffffu;

// Programmatic dependent launch (launch_k with overlap): a kernel may be scheduled
// while the previous kernel of the stream is still running; pdl_wait() blocks until
// that kernel has completed and its writes are visible, pdl_trigger() lets the next
// kernel be scheduled.  Both are no-ops for an ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// float with the sign, exponent and top 23 mantissa bits of the double with bits b (the
// dropped bits are zero when called below); zero below the float range, infinity above
__device__ __forceinline__ float bits_to_float(unsigned long long b) {
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  const unsigned m = (unsigned)(b >> 29) & 0x7fffffu;
  const unsigned f = e <= 0 ? sign : (e >= 255 ? (sign | 0x7f800000u) : (sign | ((unsigned)e << 23) | m));
  return __uint_as_float(f);
}

// x = hi + lo with hi = x truncated to a float's 24 significant bits and lo the remainder
// truncated likewise (|x - hi - lo| <= 2^-46 |x|): one exact FP64 subtraction and integer
// bit operations, as FP64 conversions run on this GPU's narrow FP64 unit
__device__ __forceinline__ void split_double(double x, float& hi, float& lo) {
  const unsigned long long kKeep = 0xFFFFFFFFE0000000ull;
  const unsigned long long hb = (unsigned long long)__double_as_longlong(x) & kKeep;
  const double rem = x - __longlong_as_double((long long)hb);
  hi = bits_to_float(hb);
  lo = bits_to_float((unsigned long long)__double_as_longlong(rem) & kKeep);
}

// SplitMix64 (Steele, Lea & Flood 2014) of counter i: the Lanczos start vector
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long i) {
  unsigned long long z = 0x9E3779B97F4A7C15ull * (i + 1ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Per-observation Jacobian record: F_o (2 x 9, row-major) then E_o (2 x 3, row-major),
// 24 values, 96 bytes in FP32 / 192 bytes in FP64 (16-byte aligned).
constexpr int kRec = 24;
#define JF(J, o, k) (J)[(size_t)(o) * ::ba::kRec + (k)]
#define JE(J, o, k) (J)[(size_t)(o) * ::ba::kRec + 18 + (k)]

__device__ __forceinline__ void load_record(const float* __restrict__ r, float f[18], float e[6]) {
  const float4* v = reinterpret_cast<const float4*>(r);
  float4 q[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) q[i] = __ldcs(v + i);
  float t[24];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    t[4 * i] = q[i].x;
    t[4 * i + 1] = q[i].y;
    t[4 * i + 2] = q[i].z;
    t[4 * i + 3] = q[i].w;
  }
#pragma unroll
  for (int k = 0; k < 18; ++k) f[k] = t[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) e[k] = t[18 + k];
}

__device__ __forceinline__ void load_record(const double* __restrict__ r, double f[18], double e[6]) {
  const double2* v = reinterpret_cast<const double2*>(r);
  double2 q[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) q[i] = __ldcs(v + i);
  double t[24];
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    t[2 * i] = q[i].x;
    t[2 * i + 1] = q[i].y;
  }
#pragma unroll
  for (int k = 0; k < 18; ++k) f[k] = t[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) e[k] = t[18 + k];
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
  return v;
}

// Sum over a block of BS threads; result valid in thread 0.
template <int BS>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red_smem[BS / 32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red_smem[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = (l < BS / 32) ? red_smem[l] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

// Deterministic grid reduction: every block writes its partial sum; the last
// block to finish adds the partials in block order and stores the total.
template <int BS>
__device__ __forceinline__ void grid_sum_store(double v, double* partial, unsigned* counter,
                                               double* out) {
  __shared__ bool am_last;
  double s = block_sum<BS>(v);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s;
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) {
    __threadfence();
    double acc = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += BS) acc += __ldcg(partial + i);
    acc = block_sum<BS>(acc);
    if (threadIdx.x == 0) {
      *out = acc;
      *counter = 0u;
    }
  }
}

// In-place inverse of an n x n SPD matrix (row-major, n <= 16) held by one thread,
// via Cholesky A = L L^T, L^-1 and A^-1 = L^-T L^-1.  Returns false if a pivot is
// not positive (the matrix is then left partially overwritten).
template <int NMAX>
__device__ bool spd_inverse(double* a, int n) {
  // Cholesky, lower triangle in place
  for (int j = 0; j < n; ++j) {
    double d = a[j * n + j];
    for (int k = 0; k < j; ++k) d -= a[j * n + k] * a[j * n + k];
    if (!(d > 0.0)) return false;
    d = sqrt(d);
    a[j * n + j] = d;
    const double inv = 1.0 / d;
    for (int i = j + 1; i < n; ++i) {
      double s = a[i * n + j];
      for (int k = 0; k < j; ++k) s -= a[i * n + k] * a[j * n + k];
      a[i * n + j] = s * inv;
    }
  }
  // L^-1 in place (lower triangle)
  for (int j = 0; j < n; ++j) {
    a[j * n + j] = 1.0 / a[j * n + j];
    for (int i = j + 1; i < n; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s -= a[i * n + k] * a[k * n + j];
      a[i * n + j] = s / a[i * n + i];
    }
  }
  // A^-1 = L^-T L^-1 ; compute lower triangle then mirror
  double tmp[NMAX];
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = 0.0;
      for (int k = i; k < n; ++k) s += a[k * n + i] * a[k * n + j];
      tmp[j] = s;
    }
    // row i of result lower part stored after finishing (entries a[k*n+i] for k>=i are
    // still needed by later rows i' > i only through columns >= i', untouched here)
    for (int j = 0; j <= i; ++j) a[i * n + j] = tmp[j];
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) a[i * n + j] = a[j * n + i];
  return true;
}

// 16-byte asynchronous global -> shared copies (completion per thread at wait_group;
// a __syncwarp after it publishes them to the rest of the warp)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

}  // namespace ba
