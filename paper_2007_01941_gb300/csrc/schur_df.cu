// Outer implicit Schur product y += S x of the mixed-precision solve (Section 3.6's
// implicit operator, the same three-step product as the FP64 kernel in schur.cu) in
// paired-FP32 arithmetic: every FP64 quantity is carried as hi + lo, two floats whose
// sum holds ~48 significant bits, and multiplied and added with error-free float
// transformations (Dekker's product via fma; Knuth's two-sum).  This GPU issues FP64
// instructions at 1/58 of the FP32 rate, so the FP64 kernel is bound by its arithmetic;
// in paired FP32 the same product costs about a sixth of the issue slots and becomes
// bound by the Jacobian stream again.  Inputs: the FP32 Jacobian records (hi) and their
// rounding residuals (lo) written by the linearisation, C_p^-1 as hi/lo, and x split
// into hi/lo per component.  Camera sums are formed in the tile's camera order by a
// segmented shuffle reduction (as in the FP32 product) and added to the FP64 y by one
// lane per camera.
#include "ba_internal.h"
#include "device_util.cuh"

namespace ba {

struct F2 {
  float h, l;
};

// a * b with the lo*lo term dropped (relative size 2^-48); result not normalised.
// The _rn intrinsics keep the compiler from fusing these steps into other operations,
// which would break the error-free transformations.
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return {p, e};
}

// s += t: two-sum of the heads, plain sum of the tails
__device__ __forceinline__ void f2_add(F2& s, F2 t) {
  const float a = __fadd_rn(s.h, t.h);
  const float bb = __fsub_rn(a, s.h);
  const float err = __fadd_rn(__fsub_rn(s.h, __fsub_rn(a, bb)), __fsub_rn(t.h, bb));
  s.h = a;
  s.l = __fadd_rn(s.l, __fadd_rn(err, t.l));
}

__device__ __forceinline__ void f2_fma(F2& s, F2 a, F2 b) { f2_add(s, f2_mul(a, b)); }

// |l| <= ulp(h) / 2 again
__device__ __forceinline__ F2 f2_norm(F2 s) {
  const float a = __fadd_rn(s.h, s.l);
  return {a, __fsub_rn(s.l, __fsub_rn(a, s.h))};
}

__device__ __forceinline__ F2 f2_neg(F2 s) { return {-s.h, -s.l}; }

__device__ __forceinline__ F2 f2_shfl(F2 v, int src) {
  return {__shfl_sync(kFull, v.h, src), __shfl_sync(kFull, v.l, src)};
}
__device__ __forceinline__ F2 f2_shfl_down(F2 v, int d) {
  return {__shfl_down_sync(kFull, v.h, d), __shfl_down_sync(kFull, v.l, d)};
}
__device__ __forceinline__ F2 f2_shfl_xor(F2 v, int d) {
  return {__shfl_xor_sync(kFull, v.h, d), __shfl_xor_sync(kFull, v.l, d)};
}

// exact float -> double by bit manipulation on the integer pipe (this GPU runs FP64
// conversions on its narrow FP64 unit); zeros and subnormals map to signed zero,
// infinities and NaNs keep their class
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned s = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const unsigned ed = e == 0xffu ? 0x7ffu : e + 896u;
  const unsigned hi = e == 0u ? s : (s | (ed << 20) | (m >> 3));
  const unsigned lo = e == 0u ? 0u : (m & 7u) << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// y += hi + lo: one FP64 addition (exact: the pair's bits fit a double) and one atomic
__device__ __forceinline__ void f2_atomic_add(double* y, F2 v) {
  atomicAdd(y, f2d_bits(v.h) + f2d_bits(v.l));
}

__device__ __forceinline__ void load_record_pair(const float* __restrict__ hi, const float* __restrict__ lo,
                                                 F2 J[kRec]) {
  const float4* a = reinterpret_cast<const float4*>(hi);
  const float4* b = reinterpret_cast<const float4*>(lo);
#pragma unroll
  for (int i = 0; i < kRec / 4; ++i) {
    const float4 p = __ldcs(a + i), q = __ldcs(b + i);
    J[4 * i] = {p.x, q.x};
    J[4 * i + 1] = {p.y, q.y};
    J[4 * i + 2] = {p.z, q.z};
    J[4 * i + 3] = {p.w, q.w};
  }
}

__device__ __forceinline__ F2 load_f2(const float* __restrict__ hi, const float* __restrict__ lo, size_t i) {
  return {__ldg(hi + i), __ldg(lo + i)};
}

// u = F x_c for observation record J (F = J[0..17] row-major 2 x 9, E = J[18..23] 2 x 3)
__device__ __forceinline__ void df_u(const F2 J[kRec], const float2* __restrict__ xc, F2& u0, F2& u1) {
  u0 = {0.f, 0.f};
  u1 = {0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float2 xv = __ldg(xc + k);
    const F2 xk = {xv.x, xv.y};
    f2_fma(u0, J[k], xk);
    f2_fma(u1, J[9 + k], xk);
  }
  u0 = f2_norm(u0);
  u1 = f2_norm(u1);
}

constexpr int kDfWarps = 8;

__global__ void __launch_bounds__(kDfWarps * 32, 3)
k_schur_matvec_df(const float* __restrict__ Jh, const float* __restrict__ Jl, const float* __restrict__ Ch,
                  const float* __restrict__ Cl, int ldp, const int* __restrict__ obs_cam,
                  const int4* __restrict__ tile_desc, const unsigned char* __restrict__ tile_perm,
                  const int* __restrict__ chunk_tile, int n_chunks, const float2* __restrict__ xs,
                  double* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned le = (lane == 31) ? kFull : ((2u << lane) - 1u);
  for (int chunk = blockIdx.x; chunk < n_chunks; chunk += gridDim.x) {
    const int t_begin = chunk_tile[chunk], t_end = chunk_tile[chunk + 1];
    for (int t = t_begin + warp; t < t_end; t += kDfWarps) {
      const int4 desc = __ldg(tile_desc + t);
      const int ob = desc.x, nobs = desc.y, p0 = desc.z;
      if (nobs <= 32) {
        const unsigned pb = (unsigned)__ldg(tile_perm + (size_t)t * 32 + lane);
        const unsigned startmask = (unsigned)desc.w;
        const bool active = lane < nobs;
        const int seg_head = 31 - __clz(startmask & le);
        const unsigned after = startmask & ~le;
        const int seg_end = active ? (after ? (__ffs(after) - 2) : (nobs - 1)) : lane;
        const int ip = p0 + __popc(startmask & le) - 1;
        const int o = active ? ob + lane : ob;
        const int c = __ldg(obs_cam + o);
        F2 J[kRec];
        load_record_pair(Jh + (size_t)o * kRec, Jl + (size_t)o * kRec, J);
        const int seglen = __reduce_max_sync(kFull, (unsigned)(seg_end - seg_head + 1));
        F2 u0, u1;
        df_u(J, xs + 9 * (size_t)c, u0, u1);
        if (!active) u0 = u1 = {0.f, 0.f};
        // t_o = E^T u, summed over the point's observations
        F2 s0 = f2_mul(J[18], u0), s1 = f2_mul(J[19], u0), s2 = f2_mul(J[20], u0);
        f2_fma(s0, J[21], u1);
        f2_fma(s1, J[22], u1);
        f2_fma(s2, J[23], u1);
        for (int d = 1; d < seglen; d <<= 1) {
          const F2 a0 = f2_shfl_down(s0, d), a1 = f2_shfl_down(s1, d), a2 = f2_shfl_down(s2, d);
          if (lane + d <= seg_end) {
            f2_add(s0, a0);
            f2_add(s1, a1);
            f2_add(s2, a2);
          }
        }
        const F2 v0 = f2_norm(f2_shfl(s0, seg_head)), v1 = f2_norm(f2_shfl(s1, seg_head)),
                 v2 = f2_norm(f2_shfl(s2, seg_head));
        // z = C_p^-1 v
        const F2 c00 = load_f2(Ch, Cl, ip), c01 = load_f2(Ch, Cl, ldp + ip), c02 = load_f2(Ch, Cl, 2 * ldp + ip);
        const F2 c11 = load_f2(Ch, Cl, 3 * ldp + ip), c12 = load_f2(Ch, Cl, 4 * ldp + ip);
        const F2 c22 = load_f2(Ch, Cl, 5 * ldp + ip);
        F2 z0 = f2_mul(c00, v0), z1 = f2_mul(c01, v0), z2 = f2_mul(c02, v0);
        f2_fma(z0, c01, v1);
        f2_fma(z0, c02, v2);
        f2_fma(z1, c11, v1);
        f2_fma(z1, c12, v2);
        f2_fma(z2, c12, v1);
        f2_fma(z2, c22, v2);
        z0 = f2_norm(z0);
        z1 = f2_norm(z1);
        z2 = f2_norm(z2);
        // w = u - E z
        F2 w0 = u0, w1 = u1;
        f2_fma(w0, f2_neg(J[18]), z0);
        f2_fma(w0, f2_neg(J[19]), z1);
        f2_fma(w0, f2_neg(J[20]), z2);
        f2_fma(w1, f2_neg(J[21]), z0);
        f2_fma(w1, f2_neg(J[22]), z1);
        f2_fma(w1, f2_neg(J[23]), z2);
        w0 = f2_norm(w0);
        w1 = f2_norm(w1);
        if (!active) w0 = w1 = {0.f, 0.f};
        // y_c += F^T w, reduced over runs of equal cameras in the tile's camera order
        F2 yv[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          yv[k] = f2_mul(J[k], w0);
          f2_fma(yv[k], J[9 + k], w1);
        }
        const int src = pb & 31;
        const bool run_head = (pb >> 7) != 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) yv[k] = f2_shfl(yv[k], src);
        const int cs = __shfl_sync(kFull, c, src);
        const unsigned heads = __ballot_sync(kFull, run_head);
        const unsigned later = heads & ~le;
        const int run_end = later ? __ffs(later) - 2 : 31;
        const int runlen = __reduce_max_sync(kFull, run_head ? (unsigned)(run_end - lane + 1) : 1u);
        for (int d = 1; d < runlen; d <<= 1) {
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const F2 a = f2_shfl_down(yv[k], d);
            if (lane + d <= run_end) f2_add(yv[k], a);
          }
        }
        if (run_head && lane < nobs) {
          double* yc = y + 9 * (size_t)cs;
#pragma unroll
          for (int k = 0; k < 9; ++k) f2_atomic_add(yc + k, yv[k]);
        }
      } else {
        // one point with more than 32 observations: two passes over them
        const int ip = p0;
        F2 s0 = {0.f, 0.f}, s1 = {0.f, 0.f}, s2 = {0.f, 0.f};
        for (int base = 0; base < nobs; base += 32) {
          const int o = ob + base + lane;
          if (base + lane < nobs) {
            F2 J[kRec];
            load_record_pair(Jh + (size_t)o * kRec, Jl + (size_t)o * kRec, J);
            F2 u0, u1;
            df_u(J, xs + 9 * (size_t)__ldg(obs_cam + o), u0, u1);
            f2_fma(s0, J[18], u0);
            f2_fma(s0, J[21], u1);
            f2_fma(s1, J[19], u0);
            f2_fma(s1, J[22], u1);
            f2_fma(s2, J[20], u0);
            f2_fma(s2, J[23], u1);
          }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          f2_add(s0, f2_shfl_xor(s0, d));
          f2_add(s1, f2_shfl_xor(s1, d));
          f2_add(s2, f2_shfl_xor(s2, d));
        }
        const F2 v0 = f2_norm(s0), v1 = f2_norm(s1), v2 = f2_norm(s2);
        const F2 c00 = load_f2(Ch, Cl, ip), c01 = load_f2(Ch, Cl, ldp + ip), c02 = load_f2(Ch, Cl, 2 * ldp + ip);
        const F2 c11 = load_f2(Ch, Cl, 3 * ldp + ip), c12 = load_f2(Ch, Cl, 4 * ldp + ip);
        const F2 c22 = load_f2(Ch, Cl, 5 * ldp + ip);
        F2 z0 = f2_mul(c00, v0), z1 = f2_mul(c01, v0), z2 = f2_mul(c02, v0);
        f2_fma(z0, c01, v1);
        f2_fma(z0, c02, v2);
        f2_fma(z1, c11, v1);
        f2_fma(z1, c12, v2);
        f2_fma(z2, c12, v1);
        f2_fma(z2, c22, v2);
        z0 = f2_norm(z0);
        z1 = f2_norm(z1);
        z2 = f2_norm(z2);
        for (int base = 0; base < nobs; base += 32) {
          const int o = ob + base + lane;
          if (base + lane < nobs) {
            const int c = __ldg(obs_cam + o);
            F2 J[kRec];
            load_record_pair(Jh + (size_t)o * kRec, Jl + (size_t)o * kRec, J);
            F2 u0, u1;
            df_u(J, xs + 9 * (size_t)c, u0, u1);
            F2 w0 = u0, w1 = u1;
            f2_fma(w0, f2_neg(J[18]), z0);
            f2_fma(w0, f2_neg(J[19]), z1);
            f2_fma(w0, f2_neg(J[20]), z2);
            f2_fma(w1, f2_neg(J[21]), z0);
            f2_fma(w1, f2_neg(J[22]), z1);
            f2_fma(w1, f2_neg(J[23]), z2);
            w0 = f2_norm(w0);
            w1 = f2_norm(w1);
            double* yc = y + 9 * (size_t)c;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
              F2 v = f2_mul(J[k], w0);
              f2_fma(v, J[9 + k], w1);
              f2_atomic_add(yc + k, v);
            }
          }
        }
      }
    }
  }
}

// xs = hi/lo split of x; with Dc, also y = Dc o x (the product's diagonal term)
__global__ void k_split_diag(size_t n, const double* __restrict__ x, float2* __restrict__ xs,
                             const double* __restrict__ Dc, double* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  const float h = (float)v;
  xs[i] = make_float2(h, (float)(v - (double)h));
  if (Dc) y[i] = Dc[i] * v;
}

bool outer_df(ba_problem* P) { return P->opt.precision == BA_MIXED && P->opt.outer_product == BA_OUTER_PAIRED_FP32; }

void split_vector(ba_problem* P, const double* x, const double* Dc, double* y) {
  const size_t n = (size_t)P->n_c * 9;
  P->xsplit.ensure(sizeof(float2) * n + 64);
  launch_k(P, k_split_diag, cdiv((long long)n, 256), 256, 0, n, x, P->xsplit.as<float2>(), Dc, y);
}

// y += S x without the diagonal term; P->xsplit must hold the split of x
void matvec_df_accumulate(ba_problem* P, double* y) {
  if (P->n_chunks == 0) return;
  int& grid = P->k3_grid_df;
  if (grid == 0) {
    int per_sm = 0;
    BA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_schur_matvec_df, kDfWarps * 32, 0));
    grid = std::max(1, std::min(P->n_chunks, P->n_sm * std::max(per_sm, 1)));
  }
  KernelTimer kt(P, BA_KT_SCHUR_DF);
  launch_k(P, k_schur_matvec_df, grid, kDfWarps * 32, 0, P->J32.as<float>(), P->J32lo.as<float>(),
           P->Cinv32.as<float>(), P->Cinv32lo.as<float>(), (int)P->ldp, P->obs_cam.as<int>(),
           P->tile_desc.as<int4>(), P->tile_perm.as<unsigned char>(), P->chunk_tile.as<int>(), P->n_chunks,
           P->xsplit.as<float2>(), y);
}

}  // namespace ba
