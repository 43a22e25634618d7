// K2: Schur reduction (Section 2.1, Eq. 3-4) and K3: the implicit Schur product of
// Section 3.6, S x = A x - F^T (E (C^-1 (E^T (F x)))), with A = F^T F + D_c.
//
// Per-observation arrays are SoA with leading dimension ld (18 rows of F, 6 of E);
// per-point arrays SoA with leading dimension ldp; camera vectors are [n_c][9].
#include <algorithm>

#include "ba_internal.h"
#include "device_util.cuh"
#include "dfloat.cuh"
#include "camera_model.cuh"

namespace ba {

// ---------------------------------------------------------------------------
// point pass: C_p = sum E^T E + D_p, C_p^-1, g_p = -sum E^T f, w_p = C_p^-1 g_p
// ---------------------------------------------------------------------------
__global__ void k_point_setup(const double* __restrict__ E, const double* __restrict__ fres,
                              size_t ld, const int* __restrict__ pt_ptr, int n_p, int n_p_obs,
                              size_t ldp, double lambda, int damp_identity, double* __restrict__ Dp,
                              double* __restrict__ Cinv, float* __restrict__ Cinv32,
                              float* __restrict__ Cinv32lo, double* __restrict__ gp, double* __restrict__ wp,
                              int* flags) {
  int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= n_p) return;
  double c00 = 0, c01 = 0, c02 = 0, c11 = 0, c12 = 0, c22 = 0, g0 = 0, g1 = 0, g2 = 0;
  const int b = pt_ptr[ip], e = pt_ptr[ip + 1];
  for (int o = b; o < e; ++o) {
    const double a0 = JE(E, o, 0), a1 = JE(E, o, 1), a2 = JE(E, o, 2);
    const double b0 = JE(E, o, 3), b1 = JE(E, o, 4), b2 = JE(E, o, 5);
    const double f0 = fres[2 * (size_t)o], f1 = fres[2 * (size_t)o + 1];
    c00 += a0 * a0 + b0 * b0;
    c01 += a0 * a1 + b0 * b1;
    c02 += a0 * a2 + b0 * b2;
    c11 += a1 * a1 + b1 * b1;
    c12 += a1 * a2 + b1 * b2;
    c22 += a2 * a2 + b2 * b2;
    g0 -= a0 * f0 + b0 * f1;
    g1 -= a1 * f0 + b1 * f1;
    g2 -= a2 * f0 + b2 * f1;
  }
  double d0, d1, d2;
  if (damp_identity) {
    d0 = d1 = d2 = lambda;
  } else {
    d0 = lambda * fmax(c00, 1e-6);
    d1 = lambda * fmax(c11, 1e-6);
    d2 = lambda * fmax(c22, 1e-6);
  }
  Dp[ip] = d0;
  Dp[ldp + ip] = d1;
  Dp[2 * ldp + ip] = d2;
  gp[ip] = g0;
  gp[ldp + ip] = g1;
  gp[2 * ldp + ip] = g2;
  double inv[6] = {0, 0, 0, 0, 0, 0};
  if (ip < n_p_obs) {
    double a[9] = {c00 + d0, c01, c02, c01, c11 + d1, c12, c02, c12, c22 + d2};
    if (!spd_inverse<3>(a, 3)) {
      flags[F_NOT_SPD_POINT] = 1;
    } else {
      inv[0] = a[0]; inv[1] = a[1]; inv[2] = a[2]; inv[3] = a[4]; inv[4] = a[5]; inv[5] = a[8];
    }
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    Cinv[k * ldp + ip] = inv[k];
    if (Cinv32) {
      float hi, lo;
      split_double(inv[k], hi, lo);
      Cinv32[k * ldp + ip] = hi;
      Cinv32lo[k * ldp + ip] = lo;
    }
  }
  wp[ip] = inv[0] * g0 + inv[1] * g1 + inv[2] * g2;
  wp[ldp + ip] = inv[1] * g0 + inv[3] * g1 + inv[4] * g2;
  wp[2 * ldp + ip] = inv[2] * g0 + inv[4] * g1 + inv[5] * g2;
}

// ---------------------------------------------------------------------------
// camera pass (warp per camera): D_c, g_c = -F^T f, b_c = g_c - sum F^T E w_p
// ---------------------------------------------------------------------------
__global__ void k_camera_setup(const double* __restrict__ F, const double* __restrict__ E,
                               const double* __restrict__ fres, size_t ld,
                               const int* __restrict__ cam_ptr, const int* __restrict__ cam_obs,
                               const int* __restrict__ obs_pt, const double* __restrict__ wp,
                               size_t ldp, int n_c, double lambda, int damp_identity,
                               double* __restrict__ Dc, float* __restrict__ Dc32,
                               double* __restrict__ gc, double* __restrict__ rhs, int raw_diag) {
  // raw_diag (partitioned solve): Dc receives this rank's share of diag(J^T J); the damping
  // is applied once the shares are summed (k_finalize_damping)
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= n_c) return;
  double dg[9], g[9], bb[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) dg[k] = g[k] = bb[k] = 0.0;
  for (int i = cam_ptr[c] + lane; i < cam_ptr[c + 1]; i += 32) {
    const int o = cam_obs[i];
    const int ip = obs_pt[o];
    const double f0 = fres[2 * (size_t)o], f1 = fres[2 * (size_t)o + 1];
    const double w0 = wp[ip], w1 = wp[ldp + ip], w2 = wp[2 * ldp + ip];
    const double h0 = f0 + JE(E, o, 0) * w0 + JE(E, o, 1) * w1 + JE(E, o, 2) * w2;
    const double h1 = f1 + JE(E, o, 3) * w0 + JE(E, o, 4) * w1 + JE(E, o, 5) * w2;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double a = JF(F, o, k), b = JF(F, o, 9 + k);
      dg[k] += a * a + b * b;
      g[k] -= a * f0 + b * f1;
      bb[k] -= a * h0 + b * h1;
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    dg[k] = warp_sum(dg[k]);
    g[k] = warp_sum(g[k]);
    bb[k] = warp_sum(bb[k]);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double d = raw_diag ? dg[k] : (damp_identity ? lambda : lambda * fmax(dg[k], 1e-6));
      Dc[9 * c + k] = d;
      Dc32[9 * c + k] = (float)d;
      gc[9 * c + k] = g[k];
      rhs[9 * c + k] = bb[k];
    }
  }
}

// ---------------------------------------------------------------------------
// S_cc = D_c + sum_{o in c} F_o^T (I - E_o C_p^-1 E_o^T) F_o   (warp per camera)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_scc(const T* __restrict__ F, const T* __restrict__ E, size_t ld,
                      const T* __restrict__ Cinv, size_t ldp, const int* __restrict__ cam_ptr,
                      const int* __restrict__ cam_obs, const int* __restrict__ obs_pt,
                      const double* __restrict__ Dc, int n_c, double* __restrict__ Scc) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= n_c) return;
  T acc[45];
#pragma unroll
  for (int k = 0; k < 45; ++k) acc[k] = 0;
  for (int i = cam_ptr[c] + lane; i < cam_ptr[c + 1]; i += 32) {
    const int o = cam_obs[i];
    const int ip = obs_pt[o];
    T e[6], ci[6], f[18];
#pragma unroll
    for (int k = 0; k < 6; ++k) e[k] = JE(E, o, k);
#pragma unroll
    for (int k = 0; k < 6; ++k) ci[k] = Cinv[k * ldp + ip];
#pragma unroll
    for (int k = 0; k < 18; ++k) f[k] = JF(F, o, k);
    // Y = E C^-1 (2x3)
    T y0[3], y1[3];
    y0[0] = e[0] * ci[0] + e[1] * ci[1] + e[2] * ci[2];
    y0[1] = e[0] * ci[1] + e[1] * ci[3] + e[2] * ci[4];
    y0[2] = e[0] * ci[2] + e[1] * ci[4] + e[2] * ci[5];
    y1[0] = e[3] * ci[0] + e[4] * ci[1] + e[5] * ci[2];
    y1[1] = e[3] * ci[1] + e[4] * ci[3] + e[5] * ci[4];
    y1[2] = e[3] * ci[2] + e[4] * ci[4] + e[5] * ci[5];
    // N = I - Y E^T (2x2, symmetric)
    const T n00 = T(1) - (y0[0] * e[0] + y0[1] * e[1] + y0[2] * e[2]);
    const T n01 = -(y0[0] * e[3] + y0[1] * e[4] + y0[2] * e[5]);
    const T n11 = T(1) - (y1[0] * e[3] + y1[1] * e[4] + y1[2] * e[5]);
    int t = 0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const T ga0 = f[a] * n00 + f[9 + a] * n01;
      const T ga1 = f[a] * n01 + f[9 + a] * n11;
#pragma unroll
      for (int b = a; b < 9; ++b) acc[t++] += ga0 * f[b] + ga1 * f[9 + b];
    }
  }
#pragma unroll
  for (int k = 0; k < 45; ++k) acc[k] = warp_sum(acc[k]);
  if (lane == 0) {
    double* out = Scc + 81 * (size_t)c;
    int t = 0;
    for (int a = 0; a < 9; ++a)
      for (int b = a; b < 9; ++b) {
        double v = (double)acc[t++];
        if (a == b && Dc) v += Dc[9 * c + a];
        out[9 * a + b] = v;
        out[9 * b + a] = v;
      }
  }
}

// inverse of SPD blocks: in [n][BS*BS] -> out64 (and out32)
template <int BS>
__global__ void k_block_inverse(const double* __restrict__ in, int n, double* __restrict__ out64,
                                float* __restrict__ out32, int* flags, int flag_slot) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a[BS * BS];
  for (int k = 0; k < BS * BS; ++k) a[k] = in[(size_t)BS * BS * i + k];
  if (!spd_inverse<BS>(a, BS)) {
    flags[flag_slot] = 1;
    for (int k = 0; k < BS * BS; ++k) a[k] = 0.0;
  }
  for (int k = 0; k < BS * BS; ++k) {
    out64[(size_t)BS * BS * i + k] = a[k];
    if (out32) out32[(size_t)BS * BS * i + k] = (float)a[k];
  }
}

// inverse of SPD blocks, one warp per block: Gauss-Jordan elimination without pivoting
// (the pivots of an SPD matrix are its positive Schur-complement diagonals); each
// lane owns BS*BS/32 entries, every step reads the old pivot row and column before
// any lane writes.  A non-positive pivot raises the flag and zeroes the block.
template <int BS>
__global__ void __launch_bounds__(256) k_block_inverse_warp(const double* __restrict__ in, int n,
                                                            double* __restrict__ out64, float* __restrict__ out32,
                                                            int* flags, int flag_slot) {
  constexpr int PER = (BS * BS + 31) / 32;
  __shared__ double sa[8][BS * BS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int blk = blockIdx.x * 8 + warp;
  if (blk >= n) return;
  double* a = sa[warp];
  const double* src = in + (size_t)blk * BS * BS;
  for (int e = lane; e < BS * BS; e += 32) a[e] = src[e];
  __syncwarp();
  bool ok = true;
  for (int k = 0; k < BS; ++k) {
    const double p = a[k * BS + k];
    if (!(p > 0.0)) ok = false;
    const double ip = 1.0 / p;
    double nv[PER];
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int e = lane + 32 * t;
      if (e < BS * BS) {
        const int i = e / BS, j = e - (e / BS) * BS;
        double v;
        if (i == k && j == k) v = ip;
        else if (i == k) v = a[k * BS + j] * ip;
        else if (j == k) v = -a[i * BS + k] * ip;
        else v = a[e] - a[i * BS + k] * a[k * BS + j] * ip;
        nv[t] = v;
      }
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int e = lane + 32 * t;
      if (e < BS * BS) a[e] = nv[t];
    }
    __syncwarp();
  }
  if (!ok && lane == 0) flags[flag_slot] = 1;
  for (int e = lane; e < BS * BS; e += 32) {
    const double v = ok ? 0.5 * (a[e] + a[(e % BS) * BS + e / BS]) : 0.0;  // symmetrise
    out64[(size_t)blk * BS * BS + e] = v;
    if (out32) out32[(size_t)blk * BS * BS + e] = (float)v;
  }
}

// The same Gauss-Jordan inversion in DF (mixed precision): the FP64 unit of this GPU
// would take a warp's FP64 instruction over many cycles per SM sub-partition, while the
// paired-FP32 steps run on the FP32 pipes.  The inverse is accurate to about 2^-48 times
// the block's condition number, beyond what the FP32 smoother blocks it feeds can hold.
// One block per group of BS lanes (32 / BS groups per warp), inverted in registers by
// df_gauss_jordan_cols: no shared-memory round trip or warp barrier per pivot step.  One
// launch covers a list of block arrays (every level's smoother blocks at once).
template <int BS>
__global__ void __launch_bounds__(256) k_block_inverse_cols_df(BlockInvBatch B, int* flags, int flag_slot) {
  constexpr int G = 32 / BS;
  __shared__ float2 tile[8][G][BS][BS + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / BS, j = lane - (lane / BS) * BS;
  const int base = g < G ? g * BS : 0;      // lanes past the last group shadow group 0
  const int blk = (blockIdx.x * 8 + warp) * G + g;
  const bool live = g < G && blk < B.total;
  int si = 0;
  for (int q = 1; q < B.nseg; ++q)
    if (blk >= B.s[q].start) si = q;
  const BlockInvSeg S = B.s[si];
  const size_t o = ((size_t)(blk - S.start) * BS) * BS + j;
  DF a[BS];
#pragma unroll
  for (int i = 0; i < BS; ++i) a[i] = live ? DF(S.in[o + (size_t)i * BS]) : DF(i == j ? 1.f : 0.f, 0.f);
  const bool ok = df_gauss_jordan_cols<BS>(a, base, j);
  if (g < G) {
#pragma unroll
    for (int i = 0; i < BS; ++i) tile[warp][g][i][j] = make_float2(a[i].h, a[i].l);
  }
  __syncwarp();
  if (!live) return;
  if (!ok && j == 0) flags[flag_slot] = 1;
#pragma unroll
  for (int i = 0; i < BS; ++i) {
    DF v(0.f, 0.f);
    if (ok) {
      const float2 t = tile[warp][g][j][i];
      const DF sym = a[i] + DF(t.x, t.y);   // symmetrise
      v = DF(0.5f * sym.h, 0.5f * sym.l);
    }
    S.out64[o + (size_t)i * BS] = to_double(v);
    if (S.out32) S.out32[o + (size_t)i * BS] = v.h;
  }
}

void block_inverse_batch(ba_problem* P, const BlockInvBatch& B, int bs, int flag_slot) {
  if (B.total == 0) return;
  if (bs == 9)
    k_block_inverse_cols_df<9><<<cdiv(B.total, 8 * 3), 256, 0, P->stream>>>(B, P->flags.as<int>(), flag_slot);
  else
    k_block_inverse_cols_df<16><<<cdiv(B.total, 8 * 2), 256, 0, P->stream>>>(B, P->flags.as<int>(), flag_slot);
  launched(P);
}

void block_inverse(ba_problem* P, const double* in, int n, int bs, double* out64, float* out32,
                   int flag_slot) {
  if (n == 0) return;
  if (P->opt.precision == BA_MIXED) {
    BlockInvBatch B{};
    B.s[0] = BlockInvSeg{in, out64, out32, n, 0};
    B.nseg = 1;
    B.total = n;
    block_inverse_batch(P, B, bs, flag_slot);
    return;
  }
  if (bs == 9)
    k_block_inverse_warp<9><<<cdiv(n, 8), 256, 0, P->stream>>>(in, n, out64, out32, P->flags.as<int>(), flag_slot);
  else
    k_block_inverse_warp<16><<<cdiv(n, 8), 256, 0, P->stream>>>(in, n, out64, out32, P->flags.as<int>(), flag_slot);
  launched(P);
}

// ---------------------------------------------------------------------------
// Mixed precision: the per-observation sums of the Schur setup and of the point
// back-substitution in paired FP32 (DF) from the FP32 records and their remainders, with
// the FP64 results formed from the pairs.  The 3x3 inversions stay FP64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ DF rec_df(const float* __restrict__ h, const float* __restrict__ l, int o, int k) {
  return DF(__ldg(h + (size_t)o * kRec + k), __ldg(l + (size_t)o * kRec + k));
}

// record o (F row-major, then E) as DF, with 16-byte loads of the heads and remainders
// (records are 96 bytes, so every record starts on a 16-byte boundary)
__device__ __forceinline__ void rec_df_all(const float* __restrict__ h, const float* __restrict__ l, int o,
                                           DF r[kRec]) {
  const float4* H = reinterpret_cast<const float4*>(h + (size_t)o * kRec);
  const float4* L = reinterpret_cast<const float4*>(l + (size_t)o * kRec);
#pragma unroll
  for (int k = 0; k < kRec / 4; ++k) {
    const float4 a = __ldg(H + k), b = __ldg(L + k);
    r[4 * k] = DF(a.x, b.x);
    r[4 * k + 1] = DF(a.y, b.y);
    r[4 * k + 2] = DF(a.z, b.z);
    r[4 * k + 3] = DF(a.w, b.w);
  }
}

// E_o (record entries 18..23) as DF
__device__ __forceinline__ void rec_df_e(const float* __restrict__ h, const float* __restrict__ l, int o, DF e[6]) {
  const float4* H = reinterpret_cast<const float4*>(h + (size_t)o * kRec);
  const float4* L = reinterpret_cast<const float4*>(l + (size_t)o * kRec);
  const float4 a4 = __ldg(H + 4), b4 = __ldg(L + 4), a5 = __ldg(H + 5), b5 = __ldg(L + 5);
  e[0] = DF(a4.z, b4.z);
  e[1] = DF(a4.w, b4.w);
  e[2] = DF(a5.x, b5.x);
  e[3] = DF(a5.y, b5.y);
  e[4] = DF(a5.z, b5.z);
  e[5] = DF(a5.w, b5.w);
}

// One thread per point: C_p = sum E_o^T E_o (+ D_p), g_p = -sum E_o^T f_o, in DF; then, in
// DF as well, the Cholesky factor C_p = G G^T, X = G^-1 (lower triangular) and
// C_p^-1 = X^T X, written as FP64, as FP32 heads and remainders, and X itself (the factor
// W_o = X E_o^T F_o of the assembled S, since W_i^T W_j = F_i^T E_i C_p^-1 E_j^T F_j).
__global__ void k_point_setup_df(const float* __restrict__ Jh, const float* __restrict__ Jl,
                                 const double* __restrict__ fres, const int* __restrict__ pt_ptr, int n_p, int n_p_obs,
                                 size_t ldp, double lambda, int damp_identity, double* __restrict__ Dp,
                                 double* __restrict__ Cinv, float* __restrict__ Cinv32, float* __restrict__ Cinv32lo,
                                 double* __restrict__ gp, double* __restrict__ wp, float2* __restrict__ wpdf,
                                 float2* __restrict__ Xdf, int* flags) {
  int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= n_p) return;
  float ch[9], cc[9];   // C (6 unique) and g (3) as compensated sums
#pragma unroll
  for (int k = 0; k < 9; ++k) ch[k] = cc[k] = 0.f;
  const int b = pt_ptr[ip], e = pt_ptr[ip + 1];
  for (int o = b; o < e; ++o) {
    DF ev[6];
    rec_df_e(Jh, Jl, o, ev);
    const DF a0 = ev[0], a1 = ev[1], a2 = ev[2], b0 = ev[3], b1 = ev[4], b2 = ev[5];
    const DF f0(fres[2 * (size_t)o]), f1(fres[2 * (size_t)o + 1]);
    const DF nf0 = -f0, nf1 = -f1;
    dot2_fma(ch[0], cc[0], a0, a0); dot2_fma(ch[0], cc[0], b0, b0);
    dot2_fma(ch[1], cc[1], a0, a1); dot2_fma(ch[1], cc[1], b0, b1);
    dot2_fma(ch[2], cc[2], a0, a2); dot2_fma(ch[2], cc[2], b0, b2);
    dot2_fma(ch[3], cc[3], a1, a1); dot2_fma(ch[3], cc[3], b1, b1);
    dot2_fma(ch[4], cc[4], a1, a2); dot2_fma(ch[4], cc[4], b1, b2);
    dot2_fma(ch[5], cc[5], a2, a2); dot2_fma(ch[5], cc[5], b2, b2);
    dot2_fma(ch[6], cc[6], a0, nf0); dot2_fma(ch[6], cc[6], b0, nf1);
    dot2_fma(ch[7], cc[7], a1, nf0); dot2_fma(ch[7], cc[7], b1, nf1);
    dot2_fma(ch[8], cc[8], a2, nf0); dot2_fma(ch[8], cc[8], b2, nf1);
  }
  DF cv[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) cv[k] = DF(ch[k], 0.f) + DF(cc[k], 0.f);
  const double C00 = to_double(cv[0]), C11 = to_double(cv[3]), C22 = to_double(cv[5]);
  double d0, d1, d2;
  if (damp_identity) {
    d0 = d1 = d2 = lambda;
  } else {
    d0 = lambda * fmax(C00, 1e-6);
    d1 = lambda * fmax(C11, 1e-6);
    d2 = lambda * fmax(C22, 1e-6);
  }
  Dp[ip] = d0;
  Dp[ldp + ip] = d1;
  Dp[2 * ldp + ip] = d2;
  const double G0 = to_double(cv[6]), G1 = to_double(cv[7]), G2 = to_double(cv[8]);
  gp[ip] = G0;
  gp[ldp + ip] = G1;
  gp[2 * ldp + ip] = G2;
  const DF zero(0.f, 0.f), one(1.f, 0.f);
  DF inv[6] = {zero, zero, zero, zero, zero, zero}, X[6] = {zero, zero, zero, zero, zero, zero};
  if (ip < n_p_obs) {
    const DF m00 = cv[0] + DF(d0), m11 = cv[3] + DF(d1), m22 = cv[5] + DF(d2);
    const DF m01 = cv[1], m02 = cv[2], m12 = cv[4];
    // Cholesky G (lower) and X = G^-1: x00, x10, x11, x20, x21, x22
    const DF p1 = m00;
    const DF g00 = df_sqrt(p1);
    const DF i00 = p1.h > 0.f ? one / g00 : zero;
    const DF g10 = m01 * i00, g20 = m02 * i00;
    const DF p2 = m11 - g10 * g10;
    const DF g11 = df_sqrt(p2);
    const DF i11 = p2.h > 0.f ? one / g11 : zero;
    const DF g21 = (m12 - g20 * g10) * i11;
    const DF p3 = m22 - g20 * g20 - g21 * g21;
    const DF g22 = df_sqrt(p3);
    const DF i22 = p3.h > 0.f ? one / g22 : zero;
    if (!(p1.h > 0.f && p2.h > 0.f && p3.h > 0.f)) {
      flags[F_NOT_SPD_POINT] = 1;
    } else {
      const DF x10 = -(g10 * i00) * i11;
      const DF x21 = -(g21 * i11) * i22;
      const DF x20 = -(g20 * i00 + g21 * x10) * i22;
      X[0] = i00; X[1] = x10; X[2] = i11; X[3] = x20; X[4] = x21; X[5] = i22;
      // C^-1 = X^T X
      inv[0] = i00 * i00 + x10 * x10 + x20 * x20;
      inv[1] = x10 * i11 + x20 * x21;
      inv[2] = x20 * i22;
      inv[3] = i11 * i11 + x21 * x21;
      inv[4] = x21 * i22;
      inv[5] = i22 * i22;
    }
  }
  double invd[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    invd[k] = to_double(inv[k]);
    Cinv[k * ldp + ip] = invd[k];
    Cinv32[k * ldp + ip] = inv[k].h;
    Cinv32lo[k * ldp + ip] = inv[k].l;
    Xdf[k * ldp + ip] = make_float2(X[k].h, X[k].l);
  }
  // w_p = C^-1 g_p
  const DF g0(G0), g1(G1), g2(G2);
  const DF w[3] = {inv[0] * g0 + inv[1] * g1 + inv[2] * g2, inv[1] * g0 + inv[3] * g1 + inv[4] * g2,
                   inv[2] * g0 + inv[4] * g1 + inv[5] * g2};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    wp[k * ldp + ip] = to_double(w[k]);
    wpdf[k * ldp + ip] = make_float2(w[k].h, w[k].l);
  }
}

constexpr int kCamBS = 128;

// one CTA per camera (threads over its observations): D_c, g_c = -F^T f and the reduced
// right-hand side b_c = g_c - F^T E w_p (w_p = C_p^-1 g_p, as float pairs), sums in DF
__global__ void __launch_bounds__(kCamBS)
k_camera_setup_df(const float* __restrict__ Jh, const float* __restrict__ Jl,
                  const double* __restrict__ fres, const int* __restrict__ cam_ptr,
                  const int* __restrict__ cam_obs, const int* __restrict__ obs_pt,
                  const float2* __restrict__ wpdf, size_t ldp, int n_c, double lambda,
                  int damp_identity, double* __restrict__ Dc, float* __restrict__ Dc32,
                  double* __restrict__ gc, double* __restrict__ rhs) {
  __shared__ float2 red[kCamBS / 32][27];
  const int c = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // dg (9), g (9), bb (9) as compensated sums
  float hs[27], cs[27];
#pragma unroll
  for (int k = 0; k < 27; ++k) hs[k] = cs[k] = 0.f;
  // the next observation's indices are fetched one iteration ahead
  const int iend = cam_ptr[c + 1];
  int i = cam_ptr[c] + t;
  int o = i < iend ? cam_obs[i] : 0;
  int ip = i < iend ? obs_pt[o] : 0;
  for (; i < iend; i += kCamBS) {
    const int on = i + kCamBS < iend ? __ldg(cam_obs + i + kCamBS) : 0;
    const int ipn = i + kCamBS < iend ? __ldg(obs_pt + on) : 0;
    const DF f0(fres[2 * (size_t)o]), f1(fres[2 * (size_t)o + 1]);
    const float2 q0 = __ldg(wpdf + ip), q1 = __ldg(wpdf + ldp + ip), q2 = __ldg(wpdf + 2 * ldp + ip);
    const DF w0(q0.x, q0.y), w1(q1.x, q1.y), w2(q2.x, q2.y);
    DF rv[kRec];
    rec_df_all(Jh, Jl, o, rv);
    const DF h0 = f0 + rv[18] * w0 + rv[19] * w1 + rv[20] * w2;
    const DF h1 = f1 + rv[21] * w0 + rv[22] * w1 + rv[23] * w2;
    const DF nf0 = -f0, nf1 = -f1, nh0 = -h0, nh1 = -h1;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const DF a = rv[k], b = rv[9 + k];
      dot2_fma(hs[k], cs[k], a, a);
      dot2_fma(hs[k], cs[k], b, b);
      dot2_fma(hs[9 + k], cs[9 + k], a, nf0);
      dot2_fma(hs[9 + k], cs[9 + k], b, nf1);
      dot2_fma(hs[18 + k], cs[18 + k], a, nh0);
      dot2_fma(hs[18 + k], cs[18 + k], b, nh1);
    }
    o = on;
    ip = ipn;
  }
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const DF v = warp_sum_df(DF(hs[k], 0.f) + DF(cs[k], 0.f));
    if (lane == 0) red[warp][k] = make_float2(v.h, v.l);
  }
  __syncthreads();
  if (t < 27) {
    DF v(0.f, 0.f);
#pragma unroll
    for (int w = 0; w < kCamBS / 32; ++w) v += DF(red[w][t].x, red[w][t].y);
    const int k = t % 9;
    const double d = to_double(v);
    if (t < 9) {
      const double dd = damp_identity ? lambda : lambda * fmax(d, 1e-6);
      Dc[9 * c + k] = dd;
      Dc32[9 * c + k] = (float)dd;
    } else if (t < 18) {
      gc[9 * c + k] = d;
    } else {
      rhs[9 * c + k] = d;
    }
  }
}

// S_cc = D_c + sum_{o in c} F_o^T N_o F_o, N_o = I - E_o C_p^-1 E_o^T, in DF (the
// counterpart of k_scc): A_cc and the point terms cancel in S_cc, so its FP64 value,
// which the assembled S and the point-block-Jacobi blocks take, needs the extra bits.
// One CTA per camera, one thread per observation; each thread keeps the 45 upper
// entries as compensated sums (dot2_fma), the CTA adds them up through shared memory.
constexpr int kSccBS = 128;

__global__ void __launch_bounds__(kSccBS)
k_scc_df(const float* __restrict__ Jh, const float* __restrict__ Jl, const float* __restrict__ Ch,
         const float* __restrict__ Cl, size_t ldp, const int* __restrict__ cam_ptr, const int* __restrict__ cam_obs,
         const int* __restrict__ obs_pt, const double* __restrict__ Dc, int n_c, double* __restrict__ Scc,
         float* __restrict__ ubnd) {
  __shared__ float2 part[45][kSccBS + 1];
  const int c = blockIdx.x;
  const int t = threadIdx.x;
  float as[45], ac[45], ub[9];
#pragma unroll
  for (int k = 0; k < 45; ++k) as[k] = ac[k] = 0.f;
#pragma unroll
  for (int a = 0; a < 9; ++a) ub[a] = 0.f;
  // the next observation's indices are fetched one iteration ahead
  const int iend = cam_ptr[c + 1];
  int i = cam_ptr[c] + t;
  int o = i < iend ? cam_obs[i] : 0;
  int ip = i < iend ? obs_pt[o] : 0;
  for (; i < iend; i += kSccBS) {
    const int on = i + kSccBS < iend ? __ldg(cam_obs + i + kSccBS) : 0;
    const int ipn = i + kSccBS < iend ? __ldg(obs_pt + on) : 0;
    DF rv[kRec], ci[6];
    rec_df_all(Jh, Jl, o, rv);
    const DF* f = rv;
    const DF* e = rv + 18;
#pragma unroll
    for (int k = 0; k < 6; ++k) ci[k] = DF(__ldg(Ch + k * ldp + ip), __ldg(Cl + k * ldp + ip));
    // Y = E C^-1 (2x3), N = I - Y E^T (2x2, symmetric)
    DF y0[3], y1[3];
    y0[0] = e[0] * ci[0] + e[1] * ci[1] + e[2] * ci[2];
    y0[1] = e[0] * ci[1] + e[1] * ci[3] + e[2] * ci[4];
    y0[2] = e[0] * ci[2] + e[1] * ci[4] + e[2] * ci[5];
    y1[0] = e[3] * ci[0] + e[4] * ci[1] + e[5] * ci[2];
    y1[1] = e[3] * ci[1] + e[4] * ci[3] + e[5] * ci[4];
    y1[2] = e[3] * ci[2] + e[4] * ci[4] + e[5] * ci[5];
    const DF one(1.f, 0.f);
    const DF n00 = one - (y0[0] * e[0] + y0[1] * e[1] + y0[2] * e[2]);
    const DF n01 = -(y0[0] * e[3] + y0[1] * e[4] + y0[2] * e[5]);
    const DF n11 = one - (y1[0] * e[3] + y1[1] * e[4] + y1[2] * e[5]);
#pragma unroll
    for (int a = 0; a < 9; ++a) ub[a] = fmaf(f[a].h, f[a].h, fmaf(f[9 + a].h, f[9 + a].h, ub[a]));
    int k = 0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const DF ga0 = f[a] * n00 + f[9 + a] * n01;
      const DF ga1 = f[a] * n01 + f[9 + a] * n11;
#pragma unroll
      for (int b = a; b < 9; ++b, ++k) {
        dot2_fma(as[k], ac[k], ga0, f[b]);
        dot2_fma(as[k], ac[k], ga1, f[9 + b]);
      }
    }
    o = on;
    ip = ipn;
  }
#pragma unroll
  for (int k = 0; k < 45; ++k) {
    const DF v = DF(as[k], 0.f) + DF(ac[k], 0.f);
    part[k][t] = make_float2(v.h, v.l);
  }
  __syncthreads();
  if (t < 45) {
    DF v(0.f, 0.f);
    for (int j = 0; j < kSccBS; ++j) v += DF(part[t][j].x, part[t][j].y);
    // entry t of the upper triangle in row order -> (a, b)
    int a = 0, r = t;
    while (r >= 9 - a) {
      r -= 9 - a;
      ++a;
    }
    const int b = a + r;
    double d = to_double(v);
    if (a == b) d += Dc[9 * c + a];
    double* out = Scc + 81 * (size_t)c;
    out[9 * a + b] = d;
    out[9 * b + a] = d;
  }
  // diag(sum_o F_o^T F_o): since E_o C_p^-1 E_o^T <= I for every observation, it bounds
  // the column sums sum_o |W_o(:, a)|^2 of the assembly's factors W_o = L_p^T E_o^T F_o
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 9; ++a) part[a][t].x = ub[a];
  __syncthreads();
  if (t < 9) {
    float v = 0.f;
    for (int j = 0; j < kSccBS; ++j) v += part[t][j].x;
    ubnd[9 * (size_t)c + t] = v;
  }
}

// delta_p = C_p^-1 (v_p - sum_{o in p} E_o^T F_o delta_c), delta_c given as float pairs
__global__ void k_back_substitute_df(const float* __restrict__ Jh, const float* __restrict__ Jl,
                                     const double* __restrict__ Cinv, size_t ldp, const int* __restrict__ pt_ptr,
                                     const int* __restrict__ obs_cam, const int* __restrict__ pt_user,
                                     const double* __restrict__ vp, int vp_user, const float2* __restrict__ dcs,
                                     int n_p, double* __restrict__ out_int, double* __restrict__ out_user) {
  int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= n_p) return;
  const int pu = pt_user[ip];
  DF h0, h1, h2;
  if (vp_user) {
    h0 = DF(vp[3 * pu]);
    h1 = DF(vp[3 * pu + 1]);
    h2 = DF(vp[3 * pu + 2]);
  } else {
    h0 = DF(vp[ip]);
    h1 = DF(vp[ldp + ip]);
    h2 = DF(vp[2 * ldp + ip]);
  }
  // the next observation's record and camera index are loaded one iteration ahead
  const int oe = pt_ptr[ip + 1];
  int o = pt_ptr[ip];
  DF rv[kRec];
  int cam = 0;
  if (o < oe) {
    cam = obs_cam[o];
    rec_df_all(Jh, Jl, o, rv);
  }
  for (; o < oe; ++o) {
    DF rn[kRec];
    int camn = 0;
    if (o + 1 < oe) {
      camn = obs_cam[o + 1];
      rec_df_all(Jh, Jl, o + 1, rn);
    } else {
#pragma unroll
      for (int k = 0; k < kRec; ++k) rn[k] = DF(0.f, 0.f);
    }
    const float2* x = dcs + 9 * (size_t)cam;
    DF u0(0.f, 0.f), u1(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float2 xv = __ldg(x + k);
      const DF xk(xv.x, xv.y);
      u0 += rv[k] * xk;
      u1 += rv[9 + k] * xk;
    }
    h0 -= rv[18] * u0 + rv[21] * u1;
    h1 -= rv[19] * u0 + rv[22] * u1;
    h2 -= rv[20] * u0 + rv[23] * u1;
#pragma unroll
    for (int k = 0; k < kRec; ++k) rv[k] = rn[k];
    cam = camn;
  }
  const double H0 = to_double(h0), H1 = to_double(h1), H2 = to_double(h2);
  const double c00 = Cinv[ip], c01 = Cinv[ldp + ip], c02 = Cinv[2 * ldp + ip];
  const double c11 = Cinv[3 * ldp + ip], c12 = Cinv[4 * ldp + ip], c22 = Cinv[5 * ldp + ip];
  const double d0 = c00 * H0 + c01 * H1 + c02 * H2;
  const double d1 = c01 * H0 + c11 * H1 + c12 * H2;
  const double d2 = c02 * H0 + c12 * H1 + c22 * H2;
  if (out_int) {
    out_int[ip] = d0;
    out_int[ldp + ip] = d1;
    out_int[2 * ldp + ip] = d2;
  }
  if (out_user) {
    out_user[3 * pu] = d0;
    out_user[3 * pu + 1] = d1;
    out_user[3 * pu + 2] = d2;
  }
}

// The mixed-precision hierarchy is built from S at damping mu = max(lambda,
// precond_lambda_min): its diagonal gets s_i = (mu - lambda) max(diag(J^T J)_i, 1e-6)
// (s_i = mu - lambda with identity damping), the difference between D at mu and at
// lambda.  FP32 copies only: the PCG's own operator keeps the damping lambda.
__global__ void k_precond_shift(int n, float s, int damp_identity, const float* __restrict__ ubnd,
                                float* __restrict__ pcd, float* __restrict__ Dc32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = damp_identity ? s : s * fmaxf(ubnd[i], 1e-6f);
  pcd[i] = v;
  Dc32[i] += v;
}

// partitioned solve: D_c from the summed diag(J^T J), and its addition to the summed S_cc
__global__ void k_finalize_damping(int n, double lambda, int damp_identity, double* __restrict__ Dc,
                                   float* __restrict__ Dc32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = damp_identity ? lambda : lambda * fmax(Dc[i], 1e-6);
  Dc[i] = d;
  Dc32[i] = (float)d;
}

__global__ void k_scc_add_damping(int n_c, const double* __restrict__ Dc, double* __restrict__ Scc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9 * n_c) return;
  Scc[81 * (size_t)(i / 9) + 10 * (i % 9)] += Dc[i];
}

__global__ void k_add_block_diag(int n_c, const double* __restrict__ Scc, const float* __restrict__ pcd,
                                 double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 81 * n_c) return;
  const int c = i / 81, k = i - 81 * c;
  out[i] = Scc[i] + ((k % 10 == 0) ? (double)pcd[9 * c + k / 10] : 0.0);
}

void schur_setup(ba_problem* P, double lambda, bool check) {
  const bool mixed = P->opt.precision == BA_MIXED;
  const int n_c = P->n_c, n_p = P->n_p;
  const size_t ldp = P->ldp;
  P->lambda = lambda;
  P->Dc.ensure(sizeof(double) * 9 * n_c + 64);
  P->Dc32.ensure(sizeof(float) * 9 * n_c + 64);
  P->Dp.ensure(sizeof(double) * 3 * ldp);
  P->Cinv64.ensure(sizeof(double) * 6 * ldp);
  if (mixed) {
    P->Cinv32.ensure(sizeof(float) * 6 * ldp);
    P->Cinv32lo.ensure(sizeof(float) * 6 * ldp);
  }
  P->gc.ensure(sizeof(double) * 9 * n_c + 64);
  P->gp.ensure(sizeof(double) * 3 * ldp);
  P->wp.ensure(sizeof(double) * 3 * ldp);
  P->rhs.ensure(sizeof(double) * 9 * n_c + 64);
  P->Scc.ensure(sizeof(double) * 81 * n_c + 64);
  P->Scc_inv.ensure(sizeof(double) * 81 * n_c + 64);
  P->Scc_inv32.ensure(sizeof(float) * 81 * n_c + 64);
  if (mixed) P->cam_ubnd.ensure(sizeof(float) * 9 * n_c + 64);
  if (check) clear_flags(P);   // else the linearisation's flags stay for the caller's check
  const int damp_id = P->opt.damping == BA_DAMP_IDENTITY;
  if (n_p) {
    if (mixed) {
      P->wpdf.ensure(sizeof(float2) * 3 * ldp);
      P->Xdf.ensure(sizeof(float2) * 6 * ldp);
      k_point_setup_df<<<cdiv(n_p, 128), 128, 0, P->stream>>>(
          P->J32.as<float>(), P->J32lo.as<float>(), P->fres.as<double>(), P->pt_ptr.as<int>(), n_p, P->n_p_obs, ldp,
          lambda, damp_id, P->Dp.as<double>(), P->Cinv64.as<double>(), P->Cinv32.as<float>(),
          P->Cinv32lo.as<float>(), P->gp.as<double>(), P->wp.as<double>(), P->wpdf.as<float2>(),
          P->Xdf.as<float2>(), P->flags.as<int>());
    } else {
      k_point_setup<<<cdiv(n_p, 128), 128, 0, P->stream>>>(
          P->J64.as<double>(), P->fres.as<double>(), P->ld, P->pt_ptr.as<int>(), n_p, P->n_p_obs, ldp,
          lambda, damp_id, P->Dp.as<double>(), P->Cinv64.as<double>(), nullptr, nullptr, P->gp.as<double>(),
          P->wp.as<double>(), P->flags.as<int>());
    }
    launched(P);
  }
  if (mixed && n_p)
    k_camera_setup_df<<<n_c, kCamBS, 0, P->stream>>>(
        P->J32.as<float>(), P->J32lo.as<float>(), P->fres.as<double>(), P->cam_ptr.as<int>(), P->cam_obs.as<int>(),
        P->obs_pt.as<int>(), P->wpdf.as<float2>(), ldp, n_c, lambda, damp_id, P->Dc.as<double>(),
        P->Dc32.as<float>(), P->gc.as<double>(), P->rhs.as<double>());
  else
    k_camera_setup<<<cdiv((long long)n_c * 32, 128), 128, 0, P->stream>>>(
        jacobian64(P), jacobian64(P), P->fres.as<double>(), P->ld, P->cam_ptr.as<int>(),
        P->cam_obs.as<int>(), P->obs_pt.as<int>(), P->wp.as<double>(), ldp, n_c, lambda, damp_id,
        P->Dc.as<double>(), P->Dc32.as<float>(), P->gc.as<double>(), P->rhs.as<double>(), partitioned(P) ? 1 : 0);
  launched(P);
  if (partitioned(P)) {
    // the camera sums over all ranks' points, then the damping from the summed diagonal
    part_allreduce(P, P->Dc.as<double>(), 9 * (size_t)n_c);
    part_allreduce(P, P->gc.as<double>(), 9 * (size_t)n_c);
    part_allreduce(P, P->rhs.as<double>(), 9 * (size_t)n_c);
    k_finalize_damping<<<cdiv(9 * n_c, 256), 256, 0, P->stream>>>(9 * n_c, lambda, damp_id, P->Dc.as<double>(),
                                                                   P->Dc32.as<float>());
    launched(P);
  }
  // point-block-Jacobi blocks S_cc (in the mode's storage precision) and FP64 inverses
  double* Scc = P->Scc.as<double>();
  if (mixed)
    k_scc_df<<<n_c, kSccBS, 0, P->stream>>>(
        P->J32.as<float>(), P->J32lo.as<float>(), P->Cinv32.as<float>(), P->Cinv32lo.as<float>(), ldp,
        P->cam_ptr.as<int>(), P->cam_obs.as<int>(), P->obs_pt.as<int>(), P->Dc.as<double>(), n_c, Scc,
        P->cam_ubnd.as<float>());
  else
    k_scc<double><<<cdiv((long long)n_c * 32, 128), 128, 0, P->stream>>>(
        P->J64.as<double>(), P->J64.as<double>(), P->ld, P->Cinv64.as<double>(), ldp,
        P->cam_ptr.as<int>(), P->cam_obs.as<int>(), P->obs_pt.as<int>(),
        partitioned(P) ? nullptr : P->Dc.as<double>(), n_c, Scc);
  launched(P);
  if (partitioned(P)) {
    part_allreduce(P, Scc, 81 * (size_t)n_c);
    k_scc_add_damping<<<cdiv(9 * n_c, 256), 256, 0, P->stream>>>(n_c, P->Dc.as<double>(), Scc);
    launched(P);
  }
  // mixed precision: the FP32 hierarchy's extra damping below precond_lambda_min
  const double mu = P->opt.precond_lambda_min;
  P->pc_shift = mixed && mu > lambda;
  if (P->pc_shift) {
    P->pc_diag.ensure(sizeof(float) * 9 * n_c + 64);
    k_precond_shift<<<cdiv(9 * n_c, 256), 256, 0, P->stream>>>(9 * n_c, (float)(mu - lambda), damp_id,
                                                                 P->cam_ubnd.as<float>(), P->pc_diag.as<float>(),
                                                                 P->Dc32.as<float>());
    launched(P);
  }
  block_inverse(P, Scc, n_c, 9, P->Scc_inv.as<double>(), P->Scc_inv32.as<float>(), F_NOT_SPD_JACOBI);
  if (P->pc_shift) {
    // the hierarchy's level-0 Jacobi blocks (the FP32 inverses) are those of the damped copy
    P->Scc_pc.ensure(sizeof(double) * 81 * (2 * (size_t)n_c) + 64);
    double* shifted = P->Scc_pc.as<double>();
    k_add_block_diag<<<cdiv(81 * n_c, 256), 256, 0, P->stream>>>(n_c, Scc, P->pc_diag.as<float>(), shifted);
    launched(P);
    block_inverse(P, shifted, n_c, 9, shifted + 81 * (size_t)n_c, P->Scc_inv32.as<float>(), F_NOT_SPD_JACOBI);
  }
  // the PCG graph captures the FP64 outer product, so its records must exist beforehand
  if (mixed && !outer_df(P) && !P->opt.recompute_jacobian) jacobian64(P);
  if (check) check_flags(P);
}

// ---------------------------------------------------------------------------
// K3: implicit Schur product.  One CTA per chunk of consecutive warp tiles; a warp
// tile is a run of whole points with <= 32 observations (a point with more is a
// tile of its own and is processed in 32-observation passes), described by one
// int4 {first observation, count, first point, mask of lanes that start a point}.
// Lane l of a warp handles observation ob + l:
//   u_o = F_o x_c ; t_o = E_o^T u_o ; v_p = sum_{o in p} t_o (segmented warp scan)
//   z_p = C_p^-1 v_p ; w_o = u_o - E_o z_p ; y_c += F_o^T w_o
// Camera sums: with WINDOW (FP32) they go to a shared-memory window of the chunk's
// cameras (points are ordered by their first camera, so a chunk touches a narrow
// camera range), flushed once per CTA, and cameras outside the window go straight
// to global memory; without WINDOW (FP64, whose shared-memory atomics are slow
// compare-and-swap loops on this GPU) every contribution is a global L2 atomic.
// y must hold D_c x on entry.
// ---------------------------------------------------------------------------
constexpr int kK3Warps = 8;

// component k of a lane's 9-vector is camera component rot_index(rot, k)
__device__ __forceinline__ int rot_index(int rot, int k) {
  const int j = rot + k;
  return j >= 9 ? j - 9 : j;
}

// Bulk staging of the FP32 product's records (one 1-D cp.async.bulk per warp tile into
// shared memory, completion counted on an mbarrier).  Every wait has an iteration limit,
// after which the kernel sets F_WAIT_TIMEOUT and goes on without the data.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* m) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(m)) : "memory");
}

// lane-0 issue of a bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned),
// after the warp's reads of the destination (generic proxy) and before the copy's writes
// (async proxy)
__device__ __forceinline__ void bulk_stage(void* dst, const void* src, unsigned bytes, unsigned long long* m) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(m))
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(unsigned long long* m, unsigned parity) {
  const unsigned a = smem_addr(m);
  for (int it = 0; it < (1 << 22); ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Recompute mode of the product (FP64): instead of streaming each observation's stored
// record (192 bytes), F and E are rebuilt in registers from the camera's rotation data and
// parameters (read from L2: few cameras) and the point (shared by the point's lanes), the
// same camera model as the linearisation, scaled by the robust weight under the Huber
// loss.  It trades 192 streamed bytes per observation for about 300 FP64 operations.
struct RecompSrc {
  const double* camx;     // [n_c][kCamx] R, J_l, first-order flag of the linearisation point
  const double* cams;     // [n_c][9] the linearisation point's cameras
  const double* pts;      // [n_p][3] its points, in the caller's point order
  const double* obs;      // [n_o][2] observations, in the caller's order (Huber weights only)
  const int* obs_ptu;     // internal observation -> caller point
  const int* obs_user;    // internal observation -> caller observation
  double huber;           // Huber scale a, or 0 for the squared loss
};

__device__ __forceinline__ void recompute_record(const RecompSrc& r, int o, int c, double f[18], double e[6]) {
  const double* cx = r.camx + (size_t)kCamx * c;
  const double* cp = r.cams + 9 * (size_t)c;
  double c9[9], cr[18];
#pragma unroll
  for (int i = 0; i < 9; ++i) c9[i] = __ldg(cp + i);
#pragma unroll
  for (int i = 0; i < 18; ++i) cr[i] = __ldg(cx + i);
  const int pu = __ldg(r.obs_ptu + o);
  const double X[3] = {__ldg(r.pts + 3 * (size_t)pu), __ldg(r.pts + 3 * (size_t)pu + 1),
                       __ldg(r.pts + 3 * (size_t)pu + 2)};
  double ob[2] = {0.0, 0.0};
  if (r.huber > 0.0) {
    const int ou = __ldg(r.obs_user + o);
    ob[0] = __ldg(r.obs + 2 * (size_t)ou);
    ob[1] = __ldg(r.obs + 2 * (size_t)ou + 1);
  }
  CamObsT<double> v;
  project_obs_t<true, double>(c9, cr, __ldg(cx + 18) != 0.0, X, ob, v);
  double w = 1.0;
  if (r.huber > 0.0) {
    double half_rho;
    w = robust_weight(v.res[0] * v.res[0] + v.res[1] * v.res[1], r.huber, half_rho);
  }
#pragma unroll
  for (int k = 0; k < 18; ++k) f[k] = w * v.F[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) e[k] = w * v.E[k];
}

template <typename T, bool WINDOW>
__device__ __forceinline__ void k3_scatter(T* acc, T* __restrict__ y, int c, int cam_lo, int span,
                                           const T yv[9], int rot) {
  const int rel = c - cam_lo;
  T* dst = (WINDOW && rel < span) ? acc + 9 * rel : y + 9 * (size_t)c;
#pragma unroll
  for (int k = 0; k < 9; ++k) atomicAdd(dst + rot_index(rot, k), yv[k]);
}

// STAGES > 0 (BULK; FP32 with the camera window): each warp stages the records of its
// coming tiles (at most 32 x 96 contiguous bytes each) into a ring of STAGES shared-memory
// buffers with 1-D bulk copies, STAGES - 1 tiles ahead of the one it reduces, so the
// record stream stays in flight without holding registers.  stage_off: byte offset of the
// buffers after the camera window; then kK3Warps x STAGES buffers, then as many mbarriers.
// Measured on the street chain and the city grid, the ring costs the product a third of its
// speed: its shared memory halves the resident warps, and the tile reduction, not the load
// latency, bounds the product (register loads keep 32 warps per SM).
constexpr int kK3StageFloats = 32 * kRec;   // one buffer: 32 records
constexpr int kK3BulkStages = 2;

template <typename T, bool WINDOW, bool RECOMP = false, int STAGES = 0>
__global__ void __launch_bounds__(kK3Warps * 32, STAGES ? 2 : (sizeof(T) == 4 ? 4 : (RECOMP ? 2 : 3)))
k_schur_matvec(const T* __restrict__ F, const T* __restrict__ E, int ld,
               const T* __restrict__ Cinv, int ldp, const int* __restrict__ obs_cam,
               const int4* __restrict__ tile_desc, const unsigned char* __restrict__ tile_perm,
               const int* __restrict__ chunk_tile, const int* __restrict__ chunk_cam, int n_chunks, const T* __restrict__ x,
               T* __restrict__ y, int win, int reverse, RecompSrc rs, int stage_off, int* flags) {
  constexpr bool BULK = STAGES > 0;
  constexpr int kK3Stages = BULK ? STAGES : 1;
  static_assert(!RECOMP || sizeof(T) == 8, "the recompute mode is the FP64 product");
  static_assert(!BULK || (sizeof(T) == 4 && WINDOW && !RECOMP), "bulk staging is for the FP32 product");
  constexpr bool kPermute = sizeof(T) == 4;
  extern __shared__ __align__(128) unsigned char k3_smem[];
  T* acc = reinterpret_cast<T*>(k3_smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // BULK: narrow tiles take the buffers in turn, in the order the warp visits its tiles;
  // the producer (pbuf) runs kK3Stages - 1 narrow tiles ahead of the consumer (cbuf)
  float* stage = nullptr;
  unsigned long long* mbar = nullptr;
  int pbuf = 0, cbuf = 0;
  unsigned ph = 0;        // bit b: parity of buffer b's next phase
  unsigned pending = 0;   // bit b: a copy into buffer b not yet waited for
  bool stalled = false;   // a wait ran out: stage nothing more
  if constexpr (BULK) {
    stage = reinterpret_cast<float*>(k3_smem + stage_off) + (size_t)warp * kK3Stages * kK3StageFloats;
    mbar = reinterpret_cast<unsigned long long*>(k3_smem + stage_off +
                                                 sizeof(float) * kK3Warps * kK3Stages * kK3StageFloats) +
           kK3Stages * warp;
    if (lane == 0)
      for (int b = 0; b < kK3Stages; ++b) mbar_init(mbar + b);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
  }
  // a CTA takes chunks blockIdx.x, blockIdx.x + gridDim.x, ...: the grid is one wave of
  // resident CTAs and the chunks are small enough to balance the SMs
  for (int chunk = blockIdx.x; chunk < n_chunks; chunk += gridDim.x) {
    const int cam_lo = chunk_cam[2 * chunk];
    const int cam_hi = chunk_cam[2 * chunk + 1];
    const int span = WINDOW ? min(cam_hi - cam_lo + 1, win) : 0;
    if (WINDOW) {
      for (int i = threadIdx.x; i < span * 9; i += blockDim.x) acc[i] = T(0);
      __syncthreads();
    }
    // reverse != 0 walks the chunk's tiles from its end, where the previous product left
    // the most recently used lines in L2
    const int t_begin = chunk_tile[chunk], t_end = chunk_tile[chunk + 1];
    // BULK: stage the chunk's i-th tile if it exists and is narrow (a point with more than
    // 32 observations is read directly); its buffer held the narrow tile kK3Stages before,
    // which this warp has finished
    auto stage_tile = [&](int i) {
      if (i >= t_end - t_begin) return;
      const int4 d = __ldg(tile_desc + (reverse ? t_end - 1 - i : t_begin + i));
      if (d.y > 32) return;
      const int b = pbuf;
      pbuf = pbuf + 1 == kK3Stages ? 0 : pbuf + 1;
      if (stalled) return;
      pending |= 1u << b;
      if (lane == 0)
        bulk_stage(stage + (size_t)b * kK3StageFloats, F + (size_t)d.x * kRec, (unsigned)(d.y * kRec * 4), mbar + b);
    };
    if constexpr (BULK) {
#pragma unroll
      for (int s = 0; s < kK3Stages - 1; ++s) stage_tile(warp + s * kK3Warps);
    }
    for (int i = warp; i < t_end - t_begin; i += kK3Warps) {
      const int t = reverse ? t_end - 1 - i : t_begin + i;
      if constexpr (BULK) stage_tile(i + (kK3Stages - 1) * kK3Warps);
      const int4 desc = __ldg(tile_desc + t);
      const unsigned pb = kPermute ? (unsigned)__ldg(tile_perm + (size_t)t * 32 + lane) : 0u;
      const int ob = desc.x, nobs = desc.y, p0 = desc.z;
      if (nobs <= 32) {
        const unsigned startmask = (unsigned)desc.w;
        const bool active = lane < nobs;
        const unsigned le = (lane == 31) ? kFull : ((2u << lane) - 1u);
        const int seg_head = 31 - __clz(startmask & le);
        const unsigned after = startmask & ~le;
        const int seg_end = active ? (after ? (__ffs(after) - 2) : (nobs - 1)) : lane;
        const int ip = p0 + __popc(startmask & le) - 1;
        const int o = active ? ob + lane : ob;
        // C_p^-1 is needed only after the point sums; in FP32 its loads go out now so that
        // they overlap the record loads instead of adding a round trip after the scan (the
        // FP64 kernel is arithmetic-bound and has no registers to spare for them)
        const T* Ci = Cinv + ip;
        T c00, c01, c02, c11, c12, c22;
        if constexpr (kPermute) {
          c00 = __ldg(Ci), c01 = __ldg(Ci + ldp), c02 = __ldg(Ci + 2 * ldp);
          c11 = __ldg(Ci + 3 * ldp), c12 = __ldg(Ci + 4 * ldp), c22 = __ldg(Ci + 5 * ldp);
        }
        const int c = __ldg(obs_cam + o);
        // FP64: lane l visits the 9 camera components starting at l mod 9, so that lanes
        // of one camera add into different words of y at the same time (not in the
        // recompute mode, whose rebuilt blocks sit in registers in their natural order)
        const int rot = (kPermute || RECOMP) ? 0 : lane % 9;
        T f[18], e[6];
        if constexpr (RECOMP) {
          recompute_record(rs, o, c, f, e);
        } else if constexpr (BULK) {
          const int b = cbuf;
          cbuf = cbuf + 1 == kK3Stages ? 0 : cbuf + 1;
          bool ok = false;
          if (!stalled) {
            ok = mbar_wait(mbar + b, (ph >> b) & 1u);
            if (ok) {
              ph ^= 1u << b;
              pending &= ~(1u << b);
            } else {
              stalled = true;
              if (lane == 0) atomicExch(flags + F_WAIT_TIMEOUT, 1);
            }
          }
          // every lane reads a record it owns (inactive lanes: the tile's first)
          const float4* r = reinterpret_cast<const float4*>(stage + (size_t)b * kK3StageFloats +
                                                            (size_t)(active ? lane : 0) * kRec);
          float t[24];
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            const float4 q = ok ? r[k] : make_float4(0.f, 0.f, 0.f, 0.f);
            t[4 * k] = q.x, t[4 * k + 1] = q.y, t[4 * k + 2] = q.z, t[4 * k + 3] = q.w;
          }
#pragma unroll
          for (int k = 0; k < 18; ++k) f[k] = t[k];
#pragma unroll
          for (int k = 0; k < 6; ++k) e[k] = t[18 + k];
        } else if constexpr (kPermute) {
          load_record(F + (size_t)o * kRec, f, e);
        } else {
          const T* r = F + (size_t)o * kRec;
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const int j = rot_index(rot, k);
            f[k] = __ldcs(r + j);
            f[9 + k] = __ldcs(r + 9 + j);
          }
#pragma unroll
          for (int k = 0; k < 6; ++k) e[k] = __ldcs(r + 18 + k);
        }
        // scan steps needed: ceil(log2(longest point segment of the tile))
        const int seglen = __reduce_max_sync(kFull, (unsigned)(seg_end - seg_head + 1));
        const T* xc = x + 9 * (size_t)c;
        T u0 = T(0), u1 = T(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const T xv = __ldg(xc + rot_index(rot, k));
          u0 += f[k] * xv;
          u1 += f[9 + k] * xv;
        }
        if (!active) {
          u0 = T(0);
          u1 = T(0);
        }
        T s0 = e[0] * u0 + e[3] * u1;
        T s1 = e[1] * u0 + e[4] * u1;
        T s2 = e[2] * u0 + e[5] * u1;
        for (int d = 1; d < seglen; d <<= 1) {
          const T a0 = __shfl_down_sync(kFull, s0, d);
          const T a1 = __shfl_down_sync(kFull, s1, d);
          const T a2 = __shfl_down_sync(kFull, s2, d);
          if (lane + d <= seg_end) {
            s0 += a0;
            s1 += a1;
            s2 += a2;
          }
        }
        const T v0 = __shfl_sync(kFull, s0, seg_head);
        const T v1 = __shfl_sync(kFull, s1, seg_head);
        const T v2 = __shfl_sync(kFull, s2, seg_head);
        if constexpr (!kPermute) {
          c00 = __ldg(Ci), c01 = __ldg(Ci + ldp), c02 = __ldg(Ci + 2 * ldp);
          c11 = __ldg(Ci + 3 * ldp), c12 = __ldg(Ci + 4 * ldp), c22 = __ldg(Ci + 5 * ldp);
        }
        const T z0 = c00 * v0 + c01 * v1 + c02 * v2;
        const T z1 = c01 * v0 + c11 * v1 + c12 * v2;
        const T z2 = c02 * v0 + c12 * v1 + c22 * v2;
        T w0 = u0 - (e[0] * z0 + e[1] * z1 + e[2] * z2);
        T w1 = u1 - (e[3] * z0 + e[4] * z1 + e[5] * z2);
        if (!active) {
          w0 = T(0);
          w1 = T(0);
        }
        T yv[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) yv[k] = f[k] * w0 + f[9 + k] * w1;
        if constexpr (kPermute) {
          // camera sums: move the lanes into the tile's camera order, add each run of
          // equal cameras into its first lane with a segmented shuffle reduction, and let
          // that lane alone add the camera's 9 values into the window (no two lanes of a
          // warp then update one address)
          const int src = pb & 31;
          const bool run_head = (pb >> 7) != 0;
#pragma unroll
          for (int k = 0; k < 9; ++k) yv[k] = __shfl_sync(kFull, yv[k], src);
          const int cs = __shfl_sync(kFull, c, src);
          const unsigned heads = __ballot_sync(kFull, run_head);
          const unsigned later = heads & ~le;
          const int run_end = later ? __ffs(later) - 2 : 31;
          const int runlen = __reduce_max_sync(kFull, run_head ? (unsigned)(run_end - lane + 1) : 1u);
          for (int d = 1; d < runlen; d <<= 1) {
#pragma unroll
            for (int k = 0; k < 9; ++k) {
              const T a = __shfl_down_sync(kFull, yv[k], d);
              if (lane + d <= run_end) yv[k] += a;
            }
          }
          if (run_head && lane < nobs) k3_scatter<T, WINDOW>(acc, y, cs, cam_lo, span, yv, 0);
        } else if (active) {
          k3_scatter<T, WINDOW>(acc, y, c, cam_lo, span, yv, rot);
        }
        // BULK: every lane has read this buffer before the next staging refills it
        if constexpr (BULK) __syncwarp();
      } else {
        // one point with more than 32 observations
        const int ip = p0;
        auto blocks = [&](int o, int c, T f[18], T e[6]) {
          if constexpr (RECOMP) {
            recompute_record(rs, o, c, f, e);
          } else {
#pragma unroll
            for (int k = 0; k < 18; ++k) f[k] = JF(F, o, k);
#pragma unroll
            for (int k = 0; k < 6; ++k) e[k] = JE(E, o, k);
          }
        };
        T s0 = T(0), s1 = T(0), s2 = T(0);
        for (int base = 0; base < nobs; base += 32) {
          const int o = ob + base + lane;
          if (base + lane < nobs) {
            const int c = obs_cam[o];
            const T* xc = x + 9 * (size_t)c;
            T f[18], e[6];
            blocks(o, c, f, e);
            T u0 = T(0), u1 = T(0);
#pragma unroll
            for (int k = 0; k < 9; ++k) {
              u0 += f[k] * xc[k];
              u1 += f[9 + k] * xc[k];
            }
            s0 += e[0] * u0 + e[3] * u1;
            s1 += e[1] * u0 + e[4] * u1;
            s2 += e[2] * u0 + e[5] * u1;
          }
        }
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        const T c00 = Cinv[ip], c01 = Cinv[ldp + ip], c02 = Cinv[2 * ldp + ip];
        const T c11 = Cinv[3 * ldp + ip], c12 = Cinv[4 * ldp + ip], c22 = Cinv[5 * ldp + ip];
        const T z0 = c00 * s0 + c01 * s1 + c02 * s2;
        const T z1 = c01 * s0 + c11 * s1 + c12 * s2;
        const T z2 = c02 * s0 + c12 * s1 + c22 * s2;
        for (int base = 0; base < nobs; base += 32) {
          const int o = ob + base + lane;
          if (base + lane < nobs) {
            const int c = obs_cam[o];
            const T* xc = x + 9 * (size_t)c;
            T f[18], e[6];
            blocks(o, c, f, e);
            T u0 = T(0), u1 = T(0);
#pragma unroll
            for (int k = 0; k < 9; ++k) {
              u0 += f[k] * xc[k];
              u1 += f[9 + k] * xc[k];
            }
            const T w0 = u0 - (e[0] * z0 + e[1] * z1 + e[2] * z2);
            const T w1 = u1 - (e[3] * z0 + e[4] * z1 + e[5] * z2);
            T yv[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) yv[k] = f[k] * w0 + f[9 + k] * w1;
            k3_scatter<T, WINDOW>(acc, y, c, cam_lo, span, yv, 0);
          }
        }
      }
    }
    if (WINDOW) {
      __syncthreads();
      T* yb = y + 9 * (size_t)cam_lo;
      for (int i = threadIdx.x; i < span * 9; i += blockDim.x) {
        const T v = acc[i];
        if (v != T(0)) atomicAdd(yb + i, v);
      }
      __syncthreads();
    }
  }
  // BULK: after a wait that ran out, let the copies still in flight land (again bounded)
  // before the CTA's shared memory is released
  if constexpr (BULK) {
    for (int b = 0; b < kK3Stages; ++b)
      if ((pending >> b) & 1u) (void)mbar_wait(mbar + b, (ph >> b) & 1u);
  }
}

template <typename TD, typename T>
__global__ void k_diag_init(const TD* __restrict__ Dc, const T* __restrict__ x, T* __restrict__ y, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (T)Dc[i] * x[i];
}

// the FP32 product with STAGES record buffers per warp
template <int STAGES>
static void launch_bulk(ba_problem* P, const float* F, const float* Cinv, const float* x, float* y) {
  auto kern = k_schur_matvec<float, true, false, STAGES>;
  // window, then the warps' record buffers (16-byte aligned), then their mbarriers
  const int stage_off = (int)((sizeof(float) * 9 * (size_t)P->k3_window + 127) / 128 * 128);
  const size_t smem_b = stage_off + sizeof(float) * kK3Warps * STAGES * kK3StageFloats +
                        sizeof(unsigned long long) * kK3Warps * STAGES;
  int& g = P->k3_grid_bulk;
  if (g == 0) {
    constexpr size_t kMax = sizeof(float) * 9 * 1024 + sizeof(float) * kK3Warps * STAGES * kK3StageFloats +
                            sizeof(unsigned long long) * kK3Warps * STAGES;
    BA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMax));
    int per_sm = 0;
    BA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kK3Warps * 32, smem_b));
    g = std::max(1, std::min(P->n_chunks, P->n_sm * std::max(per_sm, 1)));
  }
  KernelTimer kt(P, BA_KT_SCHUR_FP32);
  kern<<<g, kK3Warps * 32, smem_b, P->stream>>>(F, F, (int)P->ld, Cinv, (int)P->ldp, P->obs_cam.as<int>(),
                                                P->tile_desc.as<int4>(), P->tile_perm.as<unsigned char>(),
                                                P->chunk_tile.as<int>(), P->chunk_cam.as<int>(), P->n_chunks, x, y,
                                                P->k3_window, (P->k3_calls++) & 1, RecompSrc{}, stage_off,
                                                P->flags.as<int>());
  launched(P);
}

template <typename T>
static void launch_matvec(ba_problem* P, const T* F, const T* E, const T* Cinv, const T* x, T* y) {
  if (P->n_chunks == 0) return;
  constexpr bool window = sizeof(T) == 4;
  const size_t smem = window ? sizeof(T) * 9 * (size_t)P->k3_window : 0;
  int& grid = P->k3_grid[sizeof(T) == 8];
  if (grid == 0) {
    // first product of this problem: the shared-memory limit is an attribute of the
    // kernel on the problem's device (a problem lives on one device)
    if (window)
      BA_CUDA(cudaFuncSetAttribute(k_schur_matvec<T, window>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(T) * 9 * 1024)));
    // one wave: every SM holds as many CTAs as registers and shared memory allow
    int per_sm = 0;
    BA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_schur_matvec<T, window>,
                                                          kK3Warps * 32, smem));
    grid = std::max(1, std::min(P->n_chunks, P->n_sm * std::max(per_sm, 1)));
  }
  if constexpr (sizeof(T) == 8) {
    if (P->opt.recompute_jacobian) {
      int& g = P->k3_grid_rc;
      if (g == 0) {
        int per_sm = 0;
        BA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_schur_matvec<double, false, true>,
                                                              kK3Warps * 32, 0));
        g = std::max(1, std::min(P->n_chunks, P->n_sm * std::max(per_sm, 1)));
      }
      const RecompSrc rs{P->camx.as<double>(), P->cams_lin.as<double>(), P->pts_lin.as<double>(),
                         P->obs_lin.as<double>(), P->obs_ptu.as<int>(), P->obs_user.as<int>(),
                         P->opt.loss == BA_LOSS_HUBER ? P->opt.loss_scale : 0.0};
      KernelTimer kt(P, BA_KT_SCHUR_RECOMPUTE);
      k_schur_matvec<double, false, true><<<g, kK3Warps * 32, 0, P->stream>>>(
          nullptr, nullptr, (int)P->ld, Cinv, (int)P->ldp, P->obs_cam.as<int>(), P->tile_desc.as<int4>(),
          P->tile_perm.as<unsigned char>(), P->chunk_tile.as<int>(), P->chunk_cam.as<int>(), P->n_chunks, x, y,
          P->k3_window, (P->k3_calls++) & 1, rs, 0, nullptr);
      launched(P);
      return;
    }
  }
  if constexpr (sizeof(T) == 4) {
    if (P->opt.schur_staging) {
      launch_bulk<kK3BulkStages>(P, F, Cinv, x, y);
      return;
    }
  }
  KernelTimer kt(P, sizeof(T) == 8 ? BA_KT_SCHUR_FP64 : BA_KT_SCHUR_FP32);
  k_schur_matvec<T, window><<<grid, kK3Warps * 32, smem, P->stream>>>(
      F, E, (int)P->ld, Cinv, (int)P->ldp, P->obs_cam.as<int>(), P->tile_desc.as<int4>(),
      P->tile_perm.as<unsigned char>(), P->chunk_tile.as<int>(), P->chunk_cam.as<int>(), P->n_chunks, x, y, P->k3_window,
      (P->k3_calls++) & 1, RecompSrc{}, 0, nullptr);
  launched(P);
}

// the FP64 records, unless the product rebuilds its blocks (recompute mode)
static double* records64(ba_problem* P) { return P->opt.recompute_jacobian ? nullptr : jacobian64(P); }

void matvec64(ba_problem* P, const double* x, double* y) {
  if (outer_df(P)) {
    split_vector(P, x, P->Dc.as<double>(), y);
    matvec_df_accumulate(P, y);
    return;
  }
  const int n = 9 * P->n_c;
  k_diag_init<double, double><<<cdiv(n, 256), 256, 0, P->stream>>>(P->Dc.as<double>(), x, y, n);
  launched(P);
  double* J = records64(P);
  launch_matvec<double>(P, J, J, P->Cinv64.as<double>(), x, y);
}

void matvec32(ba_problem* P, const float* x, float* y) {
  const int n = 9 * P->n_c;
  k_diag_init<float, float><<<cdiv(n, 256), 256, 0, P->stream>>>(P->Dc32.as<float>(), x, y, n);
  launched(P);
  launch_matvec<float>(P, P->J32.as<float>(), P->J32.as<float>(), P->Cinv32.as<float>(), x, y);
}

// the products alone, for callers whose producing kernel already wrote y = D_c x (and,
// for the paired-FP32 product, the split of x into P->xsplit)
void matvec64_accumulate(ba_problem* P, const double* x, double* y) {
  if (outer_df(P)) {
    matvec_df_accumulate(P, y);
    return;
  }
  double* J = records64(P);
  launch_matvec<double>(P, J, J, P->Cinv64.as<double>(), x, y);
}
void matvec32_accumulate(ba_problem* P, const float* x, float* y) {
  launch_matvec<float>(P, P->J32.as<float>(), P->J32.as<float>(), P->Cinv32.as<float>(), x, y);
}

// ---------------------------------------------------------------------------
// explicit level-0 operator S (for the Galerkin product and, when chosen, the PCG
// product and the V-cycle's finest level).  With C_p^-1 = L_p L_p^T (Cholesky) and
// W_o = L_p^T E_o^T F_o (3 x 9) per observation o = (c, p), an off-diagonal block is
//   S_cc' = - sum_{p seen by c and c'} W_(c,p)^T W_(c',p),
// and the diagonal block S_cc is the one the Schur setup already formed.  S is
// symmetric, so only the blocks on and above the diagonal are work items: the pairs
// (o, o') that meet in each upper block are listed once per problem (symbolic), and
// each block is also written, transposed, to its mirror below the diagonal.  k_schur_w
// writes W (one thread per observation, rows padded to 28 entries) and
// k_explicit_pairs gives each block to one warp, whose lane (a, g) (27 lanes)
// accumulates entries (a, 3g .. 3g+2) over the block's pairs in registers.
// ---------------------------------------------------------------------------
constexpr int kWld = 28;   // W row stride (entries)

template <typename T>
__global__ void k_schur_w(const T* __restrict__ J, const T* __restrict__ Cinv, int ldp,
                          const int* __restrict__ obs_pt, int n_o, T* __restrict__ W) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_o) return;
  const int ip = obs_pt[o];
  T f[18], e[6];
  load_record(J + (size_t)o * kRec, f, e);
  // H = E^T F (3 x 9): H[t][b] = E[0][t] F[0][b] + E[1][t] F[1][b]
  T h[27];
#pragma unroll
  for (int t = 0; t < 3; ++t)
#pragma unroll
    for (int b = 0; b < 9; ++b) h[9 * t + b] = e[t] * f[b] + e[3 + t] * f[9 + b];
  const T c00 = Cinv[ip], c01 = Cinv[ldp + ip], c02 = Cinv[2 * ldp + ip];
  const T c11 = Cinv[3 * ldp + ip], c12 = Cinv[4 * ldp + ip], c22 = Cinv[5 * ldp + ip];
  // lower Cholesky factor of C_p^-1 (clamped at zero if rounding makes a pivot negative)
  const T l00 = sqrt(c00 > T(0) ? c00 : T(0));
  const T i00 = l00 > T(0) ? T(1) / l00 : T(0);
  const T l10 = c01 * i00, l20 = c02 * i00;
  const T p11 = c11 - l10 * l10;
  const T l11 = sqrt(p11 > T(0) ? p11 : T(0));
  const T i11 = l11 > T(0) ? T(1) / l11 : T(0);
  const T l21 = (c12 - l20 * l10) * i11;
  const T p22 = c22 - l20 * l20 - l21 * l21;
  const T l22 = sqrt(p22 > T(0) ? p22 : T(0));
  // W = L^T H
  T w[kWld];
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    w[b] = l00 * h[b] + l10 * h[9 + b] + l20 * h[18 + b];
    w[9 + b] = l11 * h[9 + b] + l21 * h[18 + b];
    w[18 + b] = l22 * h[18 + b];
  }
  w[27] = T(0);
  T* out = W + (size_t)o * kWld;
  if (sizeof(T) == 4) {
    float4* o4 = reinterpret_cast<float4*>(out);
#pragma unroll
    for (int i = 0; i < kWld / 4; ++i) o4[i] = make_float4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
  } else {
    double2* o2 = reinterpret_cast<double2*>(out);
#pragma unroll
    for (int i = 0; i < kWld / 2; ++i) o2[i] = make_double2(w[2 * i], w[2 * i + 1]);
  }
}

// The same W in DF from the FP32 records and their remainders, with the point's factor X
// (C_p^-1 = X^T X, X lower triangular, from the point setup): W_o = X E_o^T F_o, so that
// W_i^T W_j = F_i^T E_i C_p^-1 E_j^T F_j; row o holds its 27 entries as (hi, lo) pairs,
// padded to 28.
__global__ void __launch_bounds__(128)
k_schur_w_df(const float* __restrict__ Jh, const float* __restrict__ Jl, const float2* __restrict__ Xdf, int ldp,
             const int* __restrict__ obs_pt, int n_o, float2* __restrict__ W2) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_o) return;
  const int ip = obs_pt[o];
  DF x[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float2 v = __ldg(Xdf + (size_t)k * ldp + ip);
    x[k] = DF(v.x, v.y);
  }
  DF rv[kRec];
  rec_df_all(Jh, Jl, o, rv);
  const DF* e = rv + 18;
  DF w[kWld];
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    const DF f0 = rv[b], f1 = rv[9 + b];
    const DF h0 = e[0] * f0 + e[3] * f1, h1 = e[1] * f0 + e[4] * f1, h2 = e[2] * f0 + e[5] * f1;
    w[b] = x[0] * h0;
    w[9 + b] = x[1] * h0 + x[2] * h1;
    w[18 + b] = x[3] * h0 + x[4] * h1 + x[5] * h2;
  }
  w[27] = DF(0.f, 0.f);
  float4* o4 = reinterpret_cast<float4*>(W2 + (size_t)o * kWld);
#pragma unroll
  for (int i = 0; i < kWld / 2; ++i) o4[i] = make_float4(w[2 * i].h, w[2 * i].l, w[2 * i + 1].h, w[2 * i + 1].l);
}

constexpr int kExWarps = 4;

// Double-buffered staging of a block's pair rows, shared by the kernels below: both W
// rows of each of a batch's kB pairs (E bytes per entry) are copied into shared memory
// with 16-byte asynchronous copies, so all of a batch's gathers are in flight at once
// and the next batch loads while this one is summed.
template <typename E, int kB>
struct PairStage {
  static constexpr int kV = 16 / (int)sizeof(E);   // entries per 16-byte copy
  static constexpr int kCh = kWld / kV;            // copies per W row
  E (*buf)[2 * kB][kWld];                          // [2][2 pair + side][entry]
  const E* W;
  const int2* pairs;
  int q1, lane;
  __device__ __forceinline__ void issue(int base, int b) {
    const int nb = min(kB, q1 - base);
    for (int t = lane; t < nb * 2 * kCh; t += 32) {
      const int r = t / kCh, ch = t - r * kCh;
      const int2 pq = __ldg(pairs + base + (r >> 1));
      const int row = (r & 1) ? pq.y : pq.x;
      cp_async16(&buf[b][r][ch * kV], W + (size_t)row * kWld + ch * kV);
    }
    cp_async_commit();
  }
  // waits for the batch at `base` (buffer b) after starting the next one
  __device__ __forceinline__ void advance(int base, int b) {
    if (base + kB < q1) {
      issue(base + kB, b ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
  }
};

template <typename T>
__global__ void __launch_bounds__(kExWarps * 32)
k_explicit_pairs(const T* __restrict__ W, int n_up, const int* __restrict__ up_blk, const int* __restrict__ mirror,
                 const int* __restrict__ blk_row, const int* __restrict__ cols, const int* __restrict__ pair_ptr,
                 const int2* __restrict__ pairs, const double* __restrict__ Scc, const float* __restrict__ pcd,
                 T* __restrict__ vals) {
  constexpr int kB = 64 / (int)sizeof(T);            // pairs per batch
  __shared__ __align__(16) T stage[kExWarps][2][2 * kB][kWld];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int w = blockIdx.x * kExWarps + wid;
  if (w >= n_up) return;
  const int e = up_blk[w];
  const int c = blk_row[e];
  T* out = vals + (size_t)e * 81;
  if (cols[e] == c) {
    // (pcd: the mixed-precision hierarchy's extra damping on the FP32 diagonal)
    for (int i = lane; i < 81; i += 32)
      out[i] = (T)Scc[(size_t)c * 81 + i] + ((pcd && i % 10 == 0) ? (T)pcd[9 * (size_t)c + i / 10] : T(0));
    return;
  }
  // lane -> (row a, column group g); lanes 27..31 repeat lane 0's reads and discard them
  const int la = lane < 27 ? lane / 3 : 0, lg = lane < 27 ? lane - 3 * (lane / 3) : 0;
  T s0 = T(0), s1 = T(0), s2 = T(0);
  const int q0 = pair_ptr[w], q1 = pair_ptr[w + 1];
  PairStage<T, kB> st{stage[wid], W, pairs, q1, lane};
  if (q0 < q1) st.issue(q0, 0);
  int buf = 0;
  for (int base = q0; base < q1; base += kB) {
    st.advance(base, buf);
    const int nb = min(kB, q1 - base);
    for (int k = 0; k < nb; ++k) {
      const T* wi = &stage[wid][buf][2 * k][la];
      const T* wj = &stage[wid][buf][2 * k + 1][3 * lg];
      const T a0 = wi[0], a1 = wi[9], a2 = wi[18];
      s0 += a0 * wj[0] + a1 * wj[9] + a2 * wj[18];
      s1 += a0 * wj[1] + a1 * wj[10] + a2 * wj[19];
      s2 += a0 * wj[2] + a1 * wj[11] + a2 * wj[20];
    }
    __syncwarp();  // every lane is done with this buffer before it is refilled
    buf ^= 1;
  }
  if (lane < 27) {
    T* o = out + 9 * la + 3 * lg;
    T* m = vals + (size_t)mirror[w] * 81 + la;
    o[0] = -s0;
    o[1] = -s1;
    o[2] = -s2;
    m[9 * (3 * lg)] = -s0;
    m[9 * (3 * lg + 1)] = -s1;
    m[9 * (3 * lg + 2)] = -s2;
  }
}

// Paired-FP32 assembly (mixed precision): the same blocks from the DF rows of
// k_schur_w_df; writes each block as (hi, lo) float pairs (its FP64 value, for the PCG
// product) and its FP32 rounding (for the V-cycle and the Galerkin product).
//
// The sums use an offset accumulator.  By Cauchy-Schwarz every partial sum of entry
// (a, b) of block (c, c'), and every product in it, is bounded by
// M = sqrt(V_c(a) V_c'(b)) with V_c(a) = sum_o |W_o(:, a)|^2 <= diag(F^T F)_c(a, a).
// With sigma a power of two >= 4 M the head s starts at sigma and takes each product
// of the heads with one fma, s' = fl(x y + s); s and s' both stay in [sigma/2, 2 sigma],
// so d = s' - s is exact (Sterbenz) and the heads' total is s - sigma exactly, while
// fma(x, y, -d) recovers the step's rounding error to within 2^-48 sigma (the same
// error-free-transformation idea as the two-sum, with the exponent fixed in advance as
// in Rump, Ogita and Oishi's extraction of a sum's leading part).  The step errors and
// the cross terms with the tails go into a plain FP32 sum that is folded into a DF
// accumulator after every batch of pairs.  Six FP32 operations per term instead of
// the twelve of the compensated dot product.
__device__ __forceinline__ float assembly_offset(float m) {
  const unsigned e = (__float_as_uint(m * 1.01f) >> 23) & 0xffu;   // 1.01 m < 2^(e - 126)
  const unsigned es = min(e + 3u, 252u);
  return __uint_as_float(es << 23);                                 // 2^(es - 127) > 4 m
}

__device__ __forceinline__ void offset_term(float& s, float& c, float2 x, float2 y) {
  const float sn = __fmaf_rn(x.x, y.x, s);
  const float d = __fsub_rn(sn, s);
  float t = __fmaf_rn(x.x, y.x, -d);
  t = __fmaf_rn(x.x, y.y, t);
  t = __fmaf_rn(x.y, y.x, t);
  c = __fadd_rn(c, t);
  s = sn;
}

__global__ void __launch_bounds__(kExWarps * 32)
k_explicit_pairs_df(const float2* __restrict__ W2, int n_up, const int* __restrict__ up_blk,
                    const int* __restrict__ mirror, const int* __restrict__ blk_row, const int* __restrict__ cols,
                    const int* __restrict__ pair_ptr, const int2* __restrict__ pairs, const double* __restrict__ Scc,
                    const float* __restrict__ ubnd, const float* __restrict__ pcd, float2* __restrict__ valsdf,
                    float* __restrict__ vals32) {
  constexpr int kB = 8;
  __shared__ __align__(16) float2 stage[kExWarps][2][2 * kB][kWld];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int w = blockIdx.x * kExWarps + wid;
  if (w >= n_up) return;
  const int e = up_blk[w];
  const int c = blk_row[e], c2 = cols[e];
  if (c2 == c) {
    for (int i = lane; i < 81; i += 32) {
      const DF v(Scc[(size_t)c * 81 + i]);
      valsdf[(size_t)e * 81 + i] = make_float2(v.h, v.l);
      // the FP32 copy feeds the hierarchy: with its extra damping on the diagonal
      vals32[(size_t)e * 81 + i] = (pcd && i % 10 == 0) ? v.h + pcd[9 * (size_t)c + i / 10] : v.h;
    }
    return;
  }
  const int la = lane < 27 ? lane / 3 : 0, lg = lane < 27 ? lane - 3 * (lane / 3) : 0;
  // two heads per entry (terms 0, 2 and term 1 of each pair) for more independent chains
  float sig[3], sh[3], th[3];
  const float va = ubnd[9 * (size_t)c + la];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    sig[u] = assembly_offset(sqrtf(va * ubnd[9 * (size_t)c2 + 3 * lg + u]));
    sh[u] = th[u] = sig[u];
  }
  DF acc[3] = {DF(0.f, 0.f), DF(0.f, 0.f), DF(0.f, 0.f)};
  const int q0 = pair_ptr[w], q1 = pair_ptr[w + 1];
  PairStage<float2, kB> st{stage[wid], W2, pairs, q1, lane};
  if (q0 < q1) st.issue(q0, 0);
  int buf = 0;
  for (int base = q0; base < q1; base += kB) {
    st.advance(base, buf);
    const int nb = min(kB, q1 - base);
    float sc[3] = {0.f, 0.f, 0.f}, tc[3] = {0.f, 0.f, 0.f};
#pragma unroll 2
    for (int k = 0; k < nb; ++k) {
      const float2* wi = &stage[wid][buf][2 * k][la];
      const float2* wj = &stage[wid][buf][2 * k + 1][3 * lg];
      const float2 a0 = wi[0], a1 = wi[9], a2 = wi[18];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        offset_term(sh[u], sc[u], a0, wj[u]);
        offset_term(th[u], tc[u], a1, wj[9 + u]);
        offset_term(sh[u], sc[u], a2, wj[18 + u]);
      }
    }
    __syncwarp();
    buf ^= 1;
#pragma unroll
    for (int u = 0; u < 3; ++u) acc[u] += DF(sc[u], 0.f) + DF(tc[u], 0.f);
  }
  if (lane < 27) {
    const size_t o = (size_t)e * 81 + 9 * la + 3 * lg, m = (size_t)mirror[w] * 81 + la;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      // the heads' totals s - sigma are exact
      const DF v = -((DF(__fsub_rn(sh[u], sig[u]), 0.f) + DF(__fsub_rn(th[u], sig[u]), 0.f)) + acc[u]);
      const float2 d = make_float2(v.h, v.l);
      valsdf[o + u] = d;
      vals32[o + u] = v.h;
      valsdf[m + 9 * (3 * lg + u)] = d;
      vals32[m + 9 * (3 * lg + u)] = v.h;
    }
  }
}

// index of block (c, c2) in camera row c of the level-0 pattern (columns ascending), or -1
__device__ __forceinline__ int pattern_block(const int* __restrict__ row_ptr, const int* __restrict__ cols, int c,
                                             int c2) {
  int lo = row_ptr[c], hi = row_ptr[c + 1];
  const int end = hi;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cols[mid] < c2) lo = mid + 1;
    else hi = mid;
  }
  return lo < end && cols[lo] == c2 ? lo : -1;
}

// The observation pairs (o, q) of block (c, c') with c < c': the observations o of camera c
// in its order, for each the observations q of the same point seen by c' > c.  One warp per
// camera: lane j takes the j-th of 32 contiguous segments of the camera's observations and
// counts its pairs per block of row c in shared memory (every block of row c is camera c's
// alone); COUNT adds the lanes' counts into cnt[up_of[e]], the fill gives each lane its
// start in each block (the earlier lanes' counts added to pos[e]) and writes its segment's
// pairs in order, so the lists are those of a sequential walk.  Rows of more than
// kPairRowMax blocks are walked by lane 0 alone.
constexpr int kPairRowMax = 64;
constexpr int kPairWarps = 4;

template <bool COUNT>
__global__ void __launch_bounds__(kPairWarps * 32)
k_pair_lists(int n_c, const int* __restrict__ row_ptr, const int* __restrict__ cols, const int* __restrict__ cam_ptr,
             const int* __restrict__ cam_obs, const int* __restrict__ obs_pt, const int* __restrict__ obs_cam,
             const int* __restrict__ pt_ptr, const int* __restrict__ up_of, int* __restrict__ cnt,
             int* __restrict__ pos, int2* __restrict__ pairs, int* flags) {
  __shared__ int lc[kPairWarps][kPairRowMax][33];   // [warp][block of the row][lane]
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int c = blockIdx.x * kPairWarps + wi;
  if (c >= n_c) return;
  const int r0 = row_ptr[c], R = row_ptr[c + 1] - r0;
  const int k0 = cam_ptr[c], k1 = cam_ptr[c + 1];
  // visits the pairs of observations [ka, kb) of camera c in order
  auto walk = [&](int ka, int kb, auto&& f) {
    for (int k = ka; k < kb; ++k) {
      const int o = cam_obs[k], p = obs_pt[o];
      for (int q = pt_ptr[p]; q < pt_ptr[p + 1]; ++q) {
        const int c2 = obs_cam[q];
        if (c2 <= c) continue;
        const int e = pattern_block(row_ptr, cols, c, c2);
        if (e < 0) {
          flags[F_PATTERN] = 1;
          continue;
        }
        f(e, o, q);
      }
    }
  };
  if (R > kPairRowMax) {
    if (lane != 0) return;
    if (COUNT) {
      walk(k0, k1, [&](int e, int, int) { ++cnt[up_of[e]]; });
    } else {
      // this row's start slots, advanced in place (the row is this thread's alone)
      walk(k0, k1, [&](int e, int o, int q) { pairs[pos[e]++] = make_int2(o, q); });
    }
    return;
  }
  // lane j's segment [ka, kb) and its counts per block of the row
  const int nk = k1 - k0, per = (nk + 31) / 32;
  const int ka = min(k0 + lane * per, k1), kb = min(ka + per, k1);
  for (int s = 0; s < R; ++s) lc[wi][s][lane] = 0;
  walk(ka, kb, [&](int e, int, int) { ++lc[wi][e - r0][lane]; });
  __syncwarp();
  if (COUNT) {
    for (int s = lane; s < R; s += 32) {
      const int e = r0 + s;
      if (up_of[e] < 0) continue;
      int t = 0;
      for (int j = 0; j < 32; ++j) t += lc[wi][s][j];
      cnt[up_of[e]] += t;
    }
    return;
  }
  // exclusive prefix over the lanes, per block: lane j's first slot in each block
  for (int s = lane; s < R; s += 32) {
    int run = pos[r0 + s];
    for (int j = 0; j < 32; ++j) {
      const int v = lc[wi][s][j];
      lc[wi][s][j] = run;
      run += v;
    }
  }
  __syncwarp();
  walk(ka, kb, [&](int e, int o, int q) { pairs[lc[wi][e - r0][lane]++] = make_int2(o, q); });
}

// pairs of observations of one point seen by different cameras c < c', grouped by the
// level-0 block (c, c') they contribute to, and the work list of blocks on and above
// the diagonal with their mirrors; built once per problem, in camera-row then observation
// order (deterministic sums).  The block lists are formed on the host (O(blocks)), the
// pairs on the device (k_pair_lists: two passes over every pair).
static void explicit_pairs_symbolic(ba_problem* P, Level& L0) {
  const int n_c = P->n_c;
  std::vector<int> row_ptr(n_c + 1), cols(std::max(L0.nnzb, 1));
  BA_CUDA(cudaMemcpyAsync(row_ptr.data(), L0.row_ptr.p, sizeof(int) * (n_c + 1), cudaMemcpyDeviceToHost, P->stream));
  if (L0.nnzb)
    BA_CUDA(cudaMemcpyAsync(cols.data(), L0.cols.p, sizeof(int) * L0.nnzb, cudaMemcpyDeviceToHost, P->stream));
  sync(P);
  auto block_of = [&](int c, int c2) {
    int lo = row_ptr[c], hi = row_ptr[c + 1];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cols[mid] < c2) lo = mid + 1;
      else hi = mid;
    }
    BA_REQUIRE(lo < row_ptr[c + 1] && cols[lo] == c2, BA_ERR_STATE, "covisibility pattern is not symmetric");
    return lo;
  };
  std::vector<int> blk_row(std::max(L0.nnzb, 1)), up_of(std::max(L0.nnzb, 1), -1), up_blk, mirror;
  for (int c = 0; c < n_c; ++c)
    for (int e = row_ptr[c]; e < row_ptr[c + 1]; ++e) {
      blk_row[e] = c;
      if (cols[e] >= c) {
        up_of[e] = (int)up_blk.size();
        up_blk.push_back(e);
        mirror.push_back(block_of(cols[e], c));
      }
    }
  const int n_up = (int)up_blk.size();
  const int nz = std::max(L0.nnzb, 1);
  // device scratch: up_of [nnzb], then the counts [n_up + 1], then the fill positions [nnzb]
  P->scratch.ensure(sizeof(int) * (2 * (size_t)nz + n_up + 1) + 64);
  int* d_up_of = P->scratch.as<int>();
  int* d_cnt = d_up_of + nz;
  int* d_pos = d_cnt + n_up + 1;
  BA_CUDA(cudaMemcpyAsync(d_up_of, up_of.data(), sizeof(int) * nz, cudaMemcpyHostToDevice, P->stream));
  BA_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(int) * (n_up + 1), P->stream));
  const int g = cdiv(std::max(n_c, 1), kPairWarps);
  k_pair_lists<true><<<g, kPairWarps * 32, 0, P->stream>>>(n_c, L0.row_ptr.as<int>(), L0.cols.as<int>(), P->cam_ptr.as<int>(),
                                               P->cam_obs.as<int>(), P->obs_pt.as<int>(), P->obs_cam.as<int>(),
                                               P->pt_ptr.as<int>(), d_up_of, d_cnt, nullptr, nullptr,
                                               P->flags.as<int>());
  launched(P);
  std::vector<int> cnt(n_up + 1, 0);
  if (n_up) BA_CUDA(cudaMemcpyAsync(cnt.data() + 1, d_cnt, sizeof(int) * n_up, cudaMemcpyDeviceToHost, P->stream));
  sync(P);
  // work items in decreasing order of their pair counts, so that the longest blocks start
  // first and the grid's tail is short (each block's own pair order is kept).  This order
  // re-reads each W row from DRAM about k_p - 1 times (4x the algorithmic bytes), but the
  // two orders that keep the blocks sharing a row together were both slower on the street
  // chain: block-row order 0.59 ms, groups of 256 block rows each in decreasing pair count
  // 0.52 ms, against 0.37 ms (3.6 against 4.8 and 3.7 ms on the city grid)
  std::vector<int> perm(n_up), rank(n_up);
  for (int u = 0; u < n_up; ++u) perm[u] = u;
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return cnt[a + 1] > cnt[b + 1]; });
  std::vector<int> up2(n_up), mir2(n_up), ptr(n_up + 1, 0);
  for (int r = 0; r < n_up; ++r) {
    rank[perm[r]] = r;
    up2[r] = up_blk[perm[r]];
    mir2[r] = mirror[perm[r]];
    ptr[r + 1] = ptr[r] + cnt[perm[r] + 1];
  }
  // each block's first pair slot, for the fill
  std::vector<int> pos(nz, 0);
  for (int e = 0; e < L0.nnzb; ++e)
    if (up_of[e] >= 0) pos[e] = ptr[rank[up_of[e]]];
  upload(P, L0.pair_ptr, ptr);
  upload(P, L0.blk_row, blk_row);
  upload(P, L0.up_blk, up2);
  upload(P, L0.mirror, mir2);
  L0.pairs.ensure(sizeof(int2) * (size_t)std::max(ptr[n_up], 1) + 64);
  BA_CUDA(cudaMemcpyAsync(d_pos, pos.data(), sizeof(int) * nz, cudaMemcpyHostToDevice, P->stream));
  k_pair_lists<false><<<g, kPairWarps * 32, 0, P->stream>>>(n_c, L0.row_ptr.as<int>(), L0.cols.as<int>(), P->cam_ptr.as<int>(),
                                                P->cam_obs.as<int>(), P->obs_pt.as<int>(), P->obs_cam.as<int>(),
                                                P->pt_ptr.as<int>(), d_up_of, nullptr, d_pos,
                                                L0.pairs.as<int2>(), P->flags.as<int>());
  launched(P);
  L0.n_up = n_up;
  sync(P);
}

// partitioned solve: after the ranks' block shares are summed, the diagonal blocks (copied
// from S_cc, which every rank already holds summed) are written again
__global__ void k_restore_diag_blocks(int n_c, const int* __restrict__ row_ptr, const int* __restrict__ cols,
                                      const double* __restrict__ Scc, double* __restrict__ vals) {
  const int c = blockIdx.x;
  __shared__ int diag;
  if (threadIdx.x == 0) {
    diag = -1;
    for (int e = row_ptr[c]; e < row_ptr[c + 1]; ++e)
      if (cols[e] == c) diag = e;
  }
  __syncthreads();
  if (diag < 0) return;
  for (int i = threadIdx.x; i < 81; i += blockDim.x) vals[81 * (size_t)diag + i] = Scc[81 * (size_t)c + i];
}

void explicit_schur(ba_problem* P, Level& L0, ExplicitMode mode) {
  if (!L0.pairs.p) explicit_pairs_symbolic(P, L0);
  const int g = cdiv(std::max(P->n_o, 1), 128);
  const int gb = cdiv(std::max(L0.n_up, 1), kExWarps);
  const int ldp = (int)P->ldp;
  if (mode == EX_PAIRED) {
    L0.vals32.ensure(sizeof(float) * 81 * (size_t)L0.nnzb + 64);
    L0.valsdf.ensure(sizeof(float2) * 81 * (size_t)L0.nnzb + 64);
    P->scratch.ensure(sizeof(float2) * kWld * (size_t)std::max(P->n_o, 1) + 64);
    float2* W2 = P->scratch.as<float2>();
    if (P->n_o) {
      k_schur_w_df<<<g, 128, 0, P->stream>>>(P->J32.as<float>(), P->J32lo.as<float>(), P->Xdf.as<float2>(), ldp,
                                             P->obs_pt.as<int>(), P->n_o, W2);
      launched(P);
    }
    KernelTimer kt(P, BA_KT_ASSEMBLY);
    k_explicit_pairs_df<<<gb, kExWarps * 32, 0, P->stream>>>(
        W2, L0.n_up, L0.up_blk.as<int>(), L0.mirror.as<int>(), L0.blk_row.as<int>(), L0.cols.as<int>(),
        L0.pair_ptr.as<int>(), L0.pairs.as<int2>(), P->Scc.as<double>(), P->cam_ubnd.as<float>(),
        P->pc_shift ? P->pc_diag.as<float>() : nullptr, L0.valsdf.as<float2>(), L0.vals32.as<float>());
  } else if (mode == EX_FP32) {
    L0.vals32.ensure(sizeof(float) * 81 * (size_t)L0.nnzb + 64);
    P->scratch.ensure(sizeof(float) * kWld * (size_t)std::max(P->n_o, 1) + 64);
    float* W = P->scratch.as<float>();
    if (P->n_o) {
      k_schur_w<float><<<g, 128, 0, P->stream>>>(P->J32.as<float>(), P->Cinv32.as<float>(), ldp,
                                                 P->obs_pt.as<int>(), P->n_o, W);
      launched(P);
    }
    KernelTimer kt(P, BA_KT_ASSEMBLY);
    k_explicit_pairs<float><<<gb, kExWarps * 32, 0, P->stream>>>(
        W, L0.n_up, L0.up_blk.as<int>(), L0.mirror.as<int>(), L0.blk_row.as<int>(), L0.cols.as<int>(),
        L0.pair_ptr.as<int>(), L0.pairs.as<int2>(), P->Scc.as<double>(),
        P->pc_shift ? P->pc_diag.as<float>() : nullptr, L0.vals32.as<float>());
  } else {
    L0.vals64.ensure(sizeof(double) * 81 * (size_t)L0.nnzb + 64);
    P->scratch.ensure(sizeof(double) * kWld * (size_t)std::max(P->n_o, 1) + 64);
    double* W = P->scratch.as<double>();
    if (P->n_o) {
      k_schur_w<double><<<g, 128, 0, P->stream>>>(jacobian64(P), P->Cinv64.as<double>(), ldp,
                                                  P->obs_pt.as<int>(), P->n_o, W);
      launched(P);
    }
    KernelTimer kt(P, BA_KT_ASSEMBLY);
    k_explicit_pairs<double><<<gb, kExWarps * 32, 0, P->stream>>>(
        W, L0.n_up, L0.up_blk.as<int>(), L0.mirror.as<int>(), L0.blk_row.as<int>(), L0.cols.as<int>(),
        L0.pair_ptr.as<int>(), L0.pairs.as<int2>(), P->Scc.as<double>(), nullptr, L0.vals64.as<double>());
  }
  launched(P);
  if (partitioned(P) && mode == EX_FP64) {
    part_allreduce(P, L0.vals64.as<double>(), 81 * (size_t)L0.nnzb);
    k_restore_diag_blocks<<<P->n_c, 128, 0, P->stream>>>(P->n_c, L0.row_ptr.as<int>(), L0.cols.as<int>(),
                                                          P->Scc.as<double>(), L0.vals64.as<double>());
    launched(P);
  }
}

// ---------------------------------------------------------------------------
// back-substitution delta_p = C_p^-1 (v_p - sum_{o in p} E_o^T F_o delta_c)
// (v_p = g_p, or a caller vector for the adjoint); writes the internal SoA layout
// and, if out_user is given, the caller's [n_p][3] layout.
// ---------------------------------------------------------------------------
__global__ void k_back_substitute(const double* __restrict__ F, const double* __restrict__ E, size_t ld,
                                  const double* __restrict__ Cinv, size_t ldp,
                                  const int* __restrict__ pt_ptr, const int* __restrict__ obs_cam,
                                  const int* __restrict__ pt_user, const double* __restrict__ vp,
                                  int vp_user, const double* __restrict__ dc, int n_p,
                                  double* __restrict__ out_int, double* __restrict__ out_user) {
  int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= n_p) return;
  const int pu = pt_user[ip];
  double h0, h1, h2;
  if (vp_user) {
    h0 = vp[3 * pu];
    h1 = vp[3 * pu + 1];
    h2 = vp[3 * pu + 2];
  } else {
    h0 = vp[ip];
    h1 = vp[ldp + ip];
    h2 = vp[2 * ldp + ip];
  }
  for (int o = pt_ptr[ip]; o < pt_ptr[ip + 1]; ++o) {
    const double* x = dc + 9 * (size_t)obs_cam[o];
    double u0 = 0, u1 = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      u0 += JF(F, o, k) * x[k];
      u1 += JF(F, o, 9 + k) * x[k];
    }
    h0 -= JE(E, o, 0) * u0 + JE(E, o, 3) * u1;
    h1 -= JE(E, o, 1) * u0 + JE(E, o, 4) * u1;
    h2 -= JE(E, o, 2) * u0 + JE(E, o, 5) * u1;
  }
  const double c00 = Cinv[ip], c01 = Cinv[ldp + ip], c02 = Cinv[2 * ldp + ip];
  const double c11 = Cinv[3 * ldp + ip], c12 = Cinv[4 * ldp + ip], c22 = Cinv[5 * ldp + ip];
  const double d0 = c00 * h0 + c01 * h1 + c02 * h2;
  const double d1 = c01 * h0 + c11 * h1 + c12 * h2;
  const double d2 = c02 * h0 + c12 * h1 + c22 * h2;
  if (out_int) {
    out_int[ip] = d0;
    out_int[ldp + ip] = d1;
    out_int[2 * ldp + ip] = d2;
  }
  if (out_user) {
    out_user[3 * pu] = d0;
    out_user[3 * pu + 1] = d1;
    out_user[3 * pu + 2] = d2;
  }
}

static void back_substitute_impl(ba_problem* P, const double* vp, int vp_user, const double* dc, double* out_int,
                                 double* out_user) {
  if (P->n_p == 0) return;
  if (P->opt.precision == BA_MIXED) {
    split_vector(P, dc, nullptr, nullptr);
    k_back_substitute_df<<<cdiv(P->n_p, 128), 128, 0, P->stream>>>(
        P->J32.as<float>(), P->J32lo.as<float>(), P->Cinv64.as<double>(), P->ldp, P->pt_ptr.as<int>(),
        P->obs_cam.as<int>(), P->pt_user.as<int>(), vp, vp_user, P->xsplit.as<float2>(), P->n_p, out_int, out_user);
  } else {
    k_back_substitute<<<cdiv(P->n_p, 128), 128, 0, P->stream>>>(
        P->J64.as<double>(), P->J64.as<double>(), P->ld, P->Cinv64.as<double>(), P->ldp, P->pt_ptr.as<int>(),
        P->obs_cam.as<int>(), P->pt_user.as<int>(), vp, vp_user, dc, P->n_p, out_int, out_user);
  }
  launched(P);
}

void back_substitute_to(ba_problem* P, const double* dc, double* out_int, double* out_user) {
  back_substitute_impl(P, P->gp.as<double>(), 0, dc, out_int, out_user);
}

void back_substitute_general(ba_problem* P, const double* vp_user, const double* dc, double* out_int,
                             double* out_user) {
  back_substitute_impl(P, vp_user, 1, dc, out_int, out_user);
}

// reduced RHS for a general right-hand side: out_c = v_c - sum_o F_o^T E_o C_p^-1 v_p
__global__ void k_point_cinv_apply(const double* __restrict__ Cinv, size_t ldp, const int* __restrict__ pt_user,
                                   const double* __restrict__ vp_user, int n_p, double* __restrict__ wp) {
  int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= n_p) return;
  const int pu = pt_user[ip];
  const double h0 = vp_user[3 * pu], h1 = vp_user[3 * pu + 1], h2 = vp_user[3 * pu + 2];
  const double c00 = Cinv[ip], c01 = Cinv[ldp + ip], c02 = Cinv[2 * ldp + ip];
  const double c11 = Cinv[3 * ldp + ip], c12 = Cinv[4 * ldp + ip], c22 = Cinv[5 * ldp + ip];
  wp[ip] = c00 * h0 + c01 * h1 + c02 * h2;
  wp[ldp + ip] = c01 * h0 + c11 * h1 + c12 * h2;
  wp[2 * ldp + ip] = c02 * h0 + c12 * h1 + c22 * h2;
}

__global__ void k_camera_reduce_rhs(const double* __restrict__ F, const double* __restrict__ E, size_t ld,
                                    const int* __restrict__ cam_ptr, const int* __restrict__ cam_obs,
                                    const int* __restrict__ obs_pt, const double* __restrict__ wp,
                                    size_t ldp, const double* __restrict__ vc, int n_c,
                                    double* __restrict__ out) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= n_c) return;
  double bb[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) bb[k] = 0.0;
  for (int i = cam_ptr[c] + lane; i < cam_ptr[c + 1]; i += 32) {
    const int o = cam_obs[i];
    const int ip = obs_pt[o];
    const double w0 = wp[ip], w1 = wp[ldp + ip], w2 = wp[2 * ldp + ip];
    const double h0 = JE(E, o, 0) * w0 + JE(E, o, 1) * w1 + JE(E, o, 2) * w2;
    const double h1 = JE(E, o, 3) * w0 + JE(E, o, 4) * w1 + JE(E, o, 5) * w2;
#pragma unroll
    for (int k = 0; k < 9; ++k) bb[k] += JF(F, o, k) * h0 + JF(F, o, 9 + k) * h1;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) bb[k] = warp_sum(bb[k]);
  if (lane == 0)
    for (int k = 0; k < 9; ++k) out[9 * c + k] = vc[9 * c + k] - bb[k];
}

void reduced_rhs(ba_problem* P, const double* vc, const double* vp_user, double* out) {
  P->scratch2.ensure(sizeof(double) * 3 * P->ldp + 64);
  double* w = P->scratch2.as<double>();
  if (P->n_p) {
    k_point_cinv_apply<<<cdiv(P->n_p, 128), 128, 0, P->stream>>>(P->Cinv64.as<double>(), P->ldp,
                                                                P->pt_user.as<int>(), vp_user, P->n_p, w);
    launched(P);
  }
  double* J = jacobian64(P);
  k_camera_reduce_rhs<<<cdiv((long long)P->n_c * 32, 128), 128, 0, P->stream>>>(
      J, J, P->ld, P->cam_ptr.as<int>(), P->cam_obs.as<int>(),
      P->obs_pt.as<int>(), w, P->ldp, vc, P->n_c, out);
  launched(P);
}

}  // namespace ba
