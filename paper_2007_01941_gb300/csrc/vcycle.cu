// One V-cycle of Algorithm 1 (Section 2.3) for hierarchies whose every level has an
// assembled block-sparse operator (level 0 the 9x9-block S, coarse levels the 16x16-block
// Galerkin products) and whose coarsest level has an explicit inverse.  The smoother is
// the Chebyshev / point-block-Jacobi iteration of Section 3.4 (Saad, Iterative Methods,
// Alg. 12.1), as in the step-per-launch path of solve.cu, which this one replaces when
// the level-0 operator is assembled.
//
// Each block-sparse product is fused into the kernel of the element-wise step that
// consumes it: one CTA owns a block row, its threads split the row's blocks, and the
// row of the product meets in shared memory next to the row's vector entries.  One
// launch per phase:
//   pre-smoothing  step 0:   r = b, d = D^-1 r / theta, x = d
//                  step k:   q = A d; r' = r - q; d' = rho_k rho_{k-1} d + 2 rho_k / delta D^-1 r'; x += d'
//   residual:                s = r - A d
//   restriction:             b_c[a] = sum_{i in a} Q_i^T s_i     (one warp per aggregate)
//   coarsest:                x_c = A_c^-1 b_c
//   prolongation and post-smoothing step 0, from A P and the residual s of the pre-smoothed
//                            x: r = s - (A P) x_c; d = D^-1 r / theta; x' = x + Q x_c[agg] + d
//                  step k:   as in pre-smoothing
// d and r alternate between two buffers per level, and x moves to its second buffer
// at post-smoothing step 0, so that no kernel writes a vector that its own warps read.
#include <algorithm>
#include <type_traits>

#include "ba_internal.h"
#include "device_util.cuh"
#include "pcg_update.cuh"

namespace ba {

bool level_fp32(ba_problem* P);

template <typename T>
struct VLevel {
  int n, bs, coarsest;
  int N, Np;          // coarsest: dense size n * bs and the row stride of Ainv
  const int* row_ptr;
  const int* cols;
  const T* vals;
  const T* Dinv;
  const T* Q;        // [n][bs][16] prolongator blocks (not on the coarsest level)
  const int* agg;
  const int* agg_ptr;
  const int* agg_mem;
  const double* cheb;
  const double* Ainv;  // coarsest: [N][Np]
  const int* ap_ptr;   // A P: blocks (bs x 16) of fine row i, their aggregates and values
  const int* ap_cols;
  const T* ap_vals;
  const int* gptr;     // folded coarse level: fine members of each block's aggregate
  const int* gmem;
  const T* mvals;      // folded coarse level: M_aj = A_aj D_j^-1 / theta
  T* rt;               // level above a folded one: t_i = Q_i^T s_i [n][16]
  T* b;
  T* x[2];
  T* r[2];
  T* d[2];
};

constexpr int kPhaseBS = 256;
constexpr int kPhaseWarps = kPhaseBS / 32;

// Every kernel below first loads the data that no kernel of the cycle writes (block
// rows of the operators, prolongator and Jacobi blocks, the coarse inverse, index
// lists) into registers, then lets the next kernel of the stream launch, then waits for
// its predecessor: with programmatic dependent launch those loads overlap the previous
// kernel, and only the vector reads stay on the cycle's critical path.

// Chebyshev coefficients (c1, c2) of step k >= 1, d_k = c1 d_{k-1} + c2 D^-1 r_k, from the
// level's table (formed on the device at each setup, so that a captured cycle stays valid)
__device__ __forceinline__ void cheb_step(const double* __restrict__ ch, int k, double& c1, double& c2) {
  c1 = ch[24 + 2 * (k - 1)];
  c2 = ch[25 + 2 * (k - 1)];
}

// row u of D_i^-1 (u = lane < BS) for block_apply
template <typename T, int BS>
__device__ __forceinline__ void dinv_row(const T* __restrict__ Dinv_i, int lane, T dr[BS]) {
  const int u = lane < BS ? lane : 0;
#pragma unroll
  for (int v = 0; v < BS; ++v) dr[v] = Dinv_i[u * BS + v];
}

// (D_i^-1 w)_u where lane v < BS holds w_v and dr is row u of D_i^-1
template <typename T, int BS>
__device__ __forceinline__ T block_apply(const T dr[BS], T w, int lane) {
  T acc = T(0);
#pragma unroll
  for (int v = 0; v < BS; ++v) acc += dr[v] * __shfl_sync(kFull, w, v);
  return lane < BS ? acc : T(0);
}

// CTA shape of the row phases: G groups of BS threads split a block row's blocks
template <int BS>
struct RowCta {
  static constexpr int G = BS == 16 ? 8 : 10;
  static constexpr int kThreads = BS == 16 ? 128 : 96;
  // 9 x 9 blocks are read by columns (kCol): the per-column partial rows of every group,
  // then each group's row sums, meet in shared memory
  static constexpr bool kCol = BS == 9;
  static constexpr int kPart = kCol ? G * BS * BS + G * BS : G * BS;
};

// FP32 level-0 phases: at least N CTAs per SM (N x 152 >= 2,000 rows), so that a
// 2,000-camera level runs in one wave (the step kernel had 13 per SM at 48 registers)
template <typename T, int BS, int N>
constexpr int phase_min_blocks() { return BS == 9 && sizeof(T) == 4 ? N : 1; }

// the first kPre blocks of thread (u, h)'s share of block row i (row u of each; column u
// for 9 x 9 blocks, so that a group's loads cover its block contiguously) and where its
// remaining blocks start
template <typename T, int BS>
struct RowPrefetch {
  static constexpr int kPre = 2;
  int e, e1, n;
  int col[kPre];
  T a[kPre][BS];
};

template <typename T, int BS>
__device__ __forceinline__ void row_prefetch(const VLevel<T>& L, int i, RowPrefetch<T, BS>& p) {
  constexpr int G = RowCta<BS>::G;
  const int t = threadIdx.x;
  const int u = t % BS, h = t / BS;
  p.n = 0;
  p.e = 0;
  p.e1 = 0;
  if (h >= G) return;
  p.e1 = L.row_ptr[i + 1];
  int e = L.row_ptr[i] + h;
#pragma unroll
  for (int k = 0; k < RowPrefetch<T, BS>::kPre; ++k) {
    if (e < p.e1) {
      p.col[k] = L.cols[e];
      constexpr bool kCol = RowCta<BS>::kCol;
      const T* a = L.vals + (size_t)e * (BS * BS) + (kCol ? u : u * BS);
#pragma unroll
      for (int c = 0; c < BS; ++c) p.a[k][c] = a[kCol ? c * BS : c];
      p.n = k + 1;
      e += G;
    }
  }
  p.e = e;
}

// q = (A v)_i by the whole CTA from the prefetched blocks and the rest of the row; on
// return q[u], u < BS, in shared memory (all threads)
template <typename T, int BS>
__device__ __forceinline__ void cta_row_product(const VLevel<T>& L, const RowPrefetch<T, BS>& p,
                                                const T* __restrict__ v, T* part, T* q) {
  constexpr int G = RowCta<BS>::G;
  const int t = threadIdx.x;
  const int u = t % BS, h = t / BS;
  if constexpr (RowCta<BS>::kCol) {
    // thread (u, h) holds column u of its blocks: acc[c] += A_i,col(c, u) v_col(u)
    if (h < G) {
      T acc[BS];
#pragma unroll
      for (int c = 0; c < BS; ++c) acc[c] = T(0);
#pragma unroll
      for (int k = 0; k < RowPrefetch<T, BS>::kPre; ++k) {
        if (k < p.n) {
          const T xu = v[(size_t)p.col[k] * BS + u];
#pragma unroll
          for (int c = 0; c < BS; ++c) acc[c] += p.a[k][c] * xu;
        }
      }
#pragma unroll 2
      for (int e = p.e; e < p.e1; e += G) {
        const T* a = L.vals + (size_t)e * (BS * BS) + u;
        const T xu = v[(size_t)L.cols[e] * BS + u];
#pragma unroll
        for (int c = 0; c < BS; ++c) acc[c] += a[c * BS] * xu;
      }
#pragma unroll
      for (int c = 0; c < BS; ++c) part[(h * BS + c) * BS + u] = acc[c];   // [group][row][column]
    }
    __syncthreads();
    T* rows = part + G * BS * BS;
    if (t < G * BS) {
      const T* pr = part + (size_t)t * BS;   // group t / BS, row t % BS
      T s = T(0);
#pragma unroll
      for (int c = 0; c < BS; ++c) s += pr[c];
      rows[t] = s;
    }
    __syncthreads();
    if (t < BS) {
      T s = T(0);
#pragma unroll
      for (int g = 0; g < G; ++g) s += rows[g * BS + t];
      q[t] = s;
    }
    __syncthreads();
    return;
  }
  if (h < G) {
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < RowPrefetch<T, BS>::kPre; ++k) {
      if (k < p.n) {
        const T* xv = v + (size_t)p.col[k] * BS;
#pragma unroll
        for (int c = 0; c < BS; ++c) acc += p.a[k][c] * xv[c];
      }
    }
#pragma unroll 2
    for (int e = p.e; e < p.e1; e += G) {
      const T* a = L.vals + (size_t)e * (BS * BS) + u * BS;
      const T* xv = v + (size_t)L.cols[e] * BS;
#pragma unroll
      for (int c = 0; c < BS; ++c) acc += a[c] * xv[c];
    }
    part[h * BS + u] = acc;
  }
  __syncthreads();
  if (t < BS) {
    T s = T(0);
#pragma unroll
    for (int g = 0; g < G; ++g) s += part[g * BS + t];
    q[t] = s;
  }
  __syncthreads();
}

// ROWS x 16 FP32 blocks (16 x 16 operator blocks of the coarse levels; A P blocks, 9 x 16
// on level 0 and 16 x 16 below): the NW warps of the row's CTA take its blocks in turn,
// and a warp reads a block (ROWS x 64 bytes, 16-byte aligned) with 16-byte loads: lane l
// holds float4 l (row l / 4, columns 4 (l % 4) .. + 3) and, for the rows past 8, float4
// 32 + l (row 8 + l / 4), multiplies them by the four matching entries of v (one 16-byte
// load) and the four lanes of each row add their sums by shuffles.  (Per-thread rows of
// 16 scalar loads made each warp load touch 32 separate 64-byte rows.)
template <int ROWS>
struct RowPrefetch16 {
  static constexpr int kPre = 2;
  int e, e1, n;
  int col[kPre];
  float4 a[kPre][2];
};

template <int ROWS, int NW>
__device__ __forceinline__ void row_prefetch16(const int* __restrict__ row_ptr, const int* __restrict__ cols,
                                               const float* __restrict__ vals, int i, RowPrefetch16<ROWS>& p) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kSecond = (ROWS - 8) * 4;   // lanes holding a float4 of rows 8 ..
  p.n = 0;
  p.e1 = row_ptr[i + 1];
  int e = row_ptr[i] + w;
#pragma unroll
  for (int k = 0; k < RowPrefetch16<ROWS>::kPre; ++k) {
    if (e < p.e1) {
      p.col[k] = cols[e];
      const float4* a = reinterpret_cast<const float4*>(vals + (size_t)e * (ROWS * 16));
      p.a[k][0] = a[lane];
      p.a[k][1] = lane < kSecond ? a[32 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
      p.n = k + 1;
      e += NW;
    }
  }
  p.e = e;
}

__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }

// q = (A v)_i (ROWS values in shared memory on return, all threads) for an NW-warp CTA;
// part holds at least 16 NW floats
template <int ROWS, int NW>
__device__ __forceinline__ void cta_row_product16(const int* __restrict__ cols, const float* __restrict__ vals,
                                                  const RowPrefetch16<ROWS>& p, const float* __restrict__ v,
                                                  float* part, float* q) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, cq = 4 * (lane & 3);
  constexpr int kSecond = (ROWS - 8) * 4;
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int k = 0; k < RowPrefetch16<ROWS>::kPre; ++k) {
    if (k < p.n) {
      const float4 xv = *reinterpret_cast<const float4*>(v + (size_t)p.col[k] * 16 + cq);
      s0 += dot4(p.a[k][0], xv);
      s1 += dot4(p.a[k][1], xv);
    }
  }
#pragma unroll 2
  for (int e = p.e; e < p.e1; e += NW) {
    const float4* a = reinterpret_cast<const float4*>(vals + (size_t)e * (ROWS * 16));
    const float4 a0 = a[lane];
    const float4 a1 = lane < kSecond ? a[32 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 xv = *reinterpret_cast<const float4*>(v + (size_t)cols[e] * 16 + cq);
    s0 += dot4(a0, xv);
    s1 += dot4(a1, xv);
  }
  s0 += __shfl_xor_sync(kFull, s0, 1);
  s0 += __shfl_xor_sync(kFull, s0, 2);
  s1 += __shfl_xor_sync(kFull, s1, 1);
  s1 += __shfl_xor_sync(kFull, s1, 2);
  if ((lane & 3) == 0) {
    part[w * 16 + (lane >> 2)] = s0;
    if (lane < kSecond) part[w * 16 + 8 + (lane >> 2)] = s1;
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < ROWS) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NW; ++k) s += part[k * 16 + t];
    q[t] = s;
  }
  __syncthreads();
}

// row u of Dinv_i times the vector w held in shared memory
template <typename T, int BS>
__device__ __forceinline__ T row_dinv(const T dr[BS], const T* w) {
  T acc = T(0);
#pragma unroll
  for (int v = 0; v < BS; ++v) acc += dr[v] * w[v];
  return acc;
}

// pre-smoothing step 0 with x = 0: r = b, d = D^-1 b / theta, x = d (one warp per row);
// on level 0 b comes in as the FP64 right-hand side
template <typename T, int BS>
__global__ void __launch_bounds__(256) k_ph_first(VLevel<T> L, const double* __restrict__ in) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const T inv_theta = (T)(1.0 / L.cheb[0]);
  T dr[BS];
  if (gw < L.n) dinv_row<T, BS>(L.Dinv + (size_t)gw * BS * BS, lane, dr);
  pdl_trigger();
  pdl_wait();
  for (int i = gw; i < L.n; i += nw) {
    if (i != gw) dinv_row<T, BS>(L.Dinv + (size_t)i * BS * BS, lane, dr);
    const size_t idx = (size_t)i * BS + lane;
    T bv = T(0);
    if (lane < BS) {
      bv = in ? (T)in[idx] : L.b[idx];
      if (in) L.b[idx] = bv;
    }
    const T dv = block_apply<T, BS>(dr, bv, lane) * inv_theta;
    if (lane < BS) {
      L.r[0][idx] = bv;
      L.d[0][idx] = dv;
      L.x[0][idx] = dv;
    }
  }
}

// The PCG update with the assembled S (alpha = r.z / p.q, x += alpha p, r -= alpha q,
// r.r and the stopping test) fused with the next V-cycle's level-0 pre-smoothing step 0 on
// the new r (the work of k_ph_first with `in` = r): each CTA takes groups of kUpdRows
// block rows, thread (row, u) entry u of its row; the row's new r meets in shared memory
// for D_i^-1 r.  The graph's last iteration forms a step 0 that no cycle uses.
constexpr int kUpdRows = 32;
constexpr int kUpdBS = kUpdRows * 9;

template <typename T>
__global__ void __launch_bounds__(kUpdBS)
k_pcg_update_first(VLevel<T> L, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                   const double* __restrict__ q, PcgCheck ck) {
  __shared__ T bsm[kUpdBS];
  const int t = threadIdx.x, lr = t / 9, u = t - 9 * lr;
  const int ngroups = (L.n + kUpdRows - 1) / kUpdRows;
  const T inv_theta = (T)(1.0 / L.cheb[0]);
  T dr[9];
  {
    const int row = blockIdx.x * kUpdRows + lr;
    if (row < L.n) dinv_row<T, 9>(L.Dinv + (size_t)row * 81, u, dr);
  }
  pdl_trigger();
  pdl_wait();
  const double pq = pcg_pq<kUpdBS>(ck), rz = ck.scal[S_TMP2];
  const double alpha = rz / pq;
  const bool ok = pq > 0.0 && isfinite(alpha);
  double acc = 0.0;
  for (int g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const int row = g * kUpdRows + lr;
    const bool live = row < L.n;
    if (live && g != (int)blockIdx.x) dinv_row<T, 9>(L.Dinv + (size_t)row * 81, u, dr);
    const size_t idx = (size_t)row * 9 + u;
    double ri = 0.0;
    if (live) {
      ri = r[idx];
      if (ok) {
        x[idx] += alpha * p[idx];
        ri -= alpha * q[idx];
        r[idx] = ri;
      }
      acc += ri * ri;
    }
    const T bv = (T)ri;
    bsm[t] = bv;
    __syncthreads();
    if (live) {
      T s = T(0);
#pragma unroll
      for (int v = 0; v < 9; ++v) s += dr[v] * bsm[9 * lr + v];
      const T dv = s * inv_theta;
      L.b[idx] = bv;
      L.r[0][idx] = bv;
      L.d[0][idx] = dv;
      L.x[0][idx] = dv;
    }
    __syncthreads();
  }
  pcg_update_finish<kUpdBS>(acc, ok, alpha, rz, ck);
}

// Chebyshev step k >= 1 on row blockIdx.x: q = A din; rout = rin - q;
// dout = c1 din + c2 D^-1 rout; x += dout (out: FP64 copy of the new x, level 0's last step)
template <typename T, int BS>
__global__ void __launch_bounds__(RowCta<BS>::kThreads, phase_min_blocks<T, BS, 16>()) k_ph_step(VLevel<T> L, int dc, int rc, int xc, int k,
                                                                 double* __restrict__ out, const double* __restrict__ rdot,
                                                                 double* __restrict__ dpart) {
  __shared__ T part[RowCta<BS>::kPart];
  __shared__ T q[BS], w[BS];
  const int i = blockIdx.x, t = threadIdx.x;
  constexpr bool kVec = BS == 16 && sizeof(T) == 4;
  constexpr int kNW = RowCta<BS>::kThreads / 32;
  std::conditional_t<kVec, RowPrefetch16<16>, RowPrefetch<T, BS>> pf;
  if constexpr (kVec) row_prefetch16<16, kNW>(L.row_ptr, L.cols, L.vals, i, pf);
  else row_prefetch<T, BS>(L, i, pf);
  T dr[BS];
  __shared__ T cc[2];   // this step's (c1, c2), read after the product's barriers
  if (t < BS) dinv_row<T, BS>(L.Dinv + (size_t)i * BS * BS, t, dr);
  if (t == 32) {
    double c1d, c2d;
    cheb_step(L.cheb, k, c1d, c2d);
    cc[0] = (T)c1d;
    cc[1] = (T)c2d;
  }
  pdl_trigger();
  pdl_wait();
  const T* din = L.d[dc];
  if constexpr (kVec) cta_row_product16<16, kNW>(L.cols, L.vals, pf, din, part, q);
  else cta_row_product<T, BS>(L, pf, din, part, q);
  const size_t idx = (size_t)i * BS + t;
  if (t < BS) w[t] = L.r[rc][idx] - q[t];
  __syncthreads();
  double dot = 0.0;
  if (t < BS) {
    const T acc = row_dinv<T, BS>(dr, w);
    const T dn = cc[0] * din[idx] + cc[1] * acc;
    const T xn = L.x[xc][idx] + dn;
    L.r[1 - rc][idx] = w[t];
    L.d[1 - dc][idx] = dn;
    L.x[xc][idx] = xn;
    if (out) {
      out[idx] = (double)xn;
      if (dpart) dot = (double)xn * rdot[idx];
    }
  }
  // this row's share of r.z (rows are CTAs; no cross-CTA reduction here)
  if (dpart && t < 32) {
    dot = warp_sum(dot);
    if (t == 0) dpart[i] = dot;
  }
}

// residual of the pre-smoothed iterate on row blockIdx.x: s = r - A d, into the free r buffer;
// RT (the next level's restriction folded into its first smoothing kernel): also this
// row's restriction term t_i = Q_i^T s_i into L.rt
template <typename T, int BS, bool RT = false>
__global__ void __launch_bounds__(RowCta<BS>::kThreads) k_ph_residual(VLevel<T> L, int dc, int rc) {
  __shared__ T part[RowCta<BS>::kPart];
  __shared__ T q[BS], sv[BS];
  const int i = blockIdx.x, t = threadIdx.x;
  constexpr bool kVec = BS == 16 && sizeof(T) == 4;
  constexpr int kNW = RowCta<BS>::kThreads / 32;
  std::conditional_t<kVec, RowPrefetch16<16>, RowPrefetch<T, BS>> pf;
  if constexpr (kVec) row_prefetch16<16, kNW>(L.row_ptr, L.cols, L.vals, i, pf);
  else row_prefetch<T, BS>(L, i, pf);
  // RT: column t of Q_i (t < 16)
  T qc[RT ? BS : 1];
  if constexpr (RT) {
    if (t < 16) {
      const T* Qi = L.Q + (size_t)i * BS * 16 + t;
#pragma unroll
      for (int u = 0; u < BS; ++u) qc[u] = Qi[u * 16];
    }
  }
  pdl_trigger();
  pdl_wait();
  if constexpr (kVec) cta_row_product16<16, kNW>(L.cols, L.vals, pf, L.d[dc], part, q);
  else cta_row_product<T, BS>(L, pf, L.d[dc], part, q);
  if (t < BS) {
    const size_t idx = (size_t)i * BS + t;
    const T s = L.r[rc][idx] - q[t];
    L.r[1 - rc][idx] = s;
    if constexpr (RT) sv[t] = s;
  }
  if constexpr (RT) {
    __syncthreads();
    if (t < 16) {
      T acc = T(0);
#pragma unroll
      for (int u = 0; u < BS; ++u) acc += qc[u] * sv[u];
      L.rt[(size_t)i * 16 + t] = acc;
    }
  }
}

// restriction b_c[a] = sum_{i in a} Q_i^T s_i (one warp per aggregate, lane s < 16); when
// the coarse level is smoothed, also its pre-smoothing step 0 for row a (x_c = 0):
// r_c = b_c, d_c = D_c^-1 b_c / theta_c, x_c = d_c
template <typename T, int BS>
__global__ void __launch_bounds__(256) k_ph_restrict(VLevel<T> L, VLevel<T> C, const T* __restrict__ res) {
  constexpr int kPre = 2;   // members per half-warp whose Q columns are prefetched
  const int lane = threadIdx.x & 31;
  const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const bool live = a < C.n;
  // lane s + 16h adds members h, h + 2, ... of the aggregate into output s
  const int s = lane & 15, h = lane >> 4;
  int m0 = 0, m1 = 0, mi[kPre];
  T qa[kPre][BS];
  T dr[16];
  if (live) {
    m0 = L.agg_ptr[a] + h;
    m1 = L.agg_ptr[a + 1];
#pragma unroll
    for (int k = 0; k < kPre; ++k) {
      const int m = m0 + 2 * k;
      mi[k] = m < m1 ? L.agg_mem[m] : 0;
      const T* Qi = L.Q + (size_t)mi[k] * BS * 16 + s;
#pragma unroll
      for (int u = 0; u < BS; ++u) qa[k][u] = m < m1 ? Qi[u * 16] : T(0);
    }
    if (!C.coarsest) dinv_row<T, 16>(C.Dinv + (size_t)a * 256, lane, dr);
  }
  pdl_trigger();
  pdl_wait();
  if (!live) return;
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < kPre; ++k) {
    if (m0 + 2 * k < m1) {
      const T* ri = res + (size_t)mi[k] * BS;
#pragma unroll
      for (int u = 0; u < BS; ++u) acc += qa[k][u] * ri[u];
    }
  }
  for (int m = m0 + 2 * kPre; m < m1; m += 2) {
    const int i = L.agg_mem[m];
    const T* Qi = L.Q + (size_t)i * BS * 16 + s;
    const T* ri = res + (size_t)i * BS;
#pragma unroll
    for (int u = 0; u < BS; ++u) acc += Qi[u * 16] * ri[u];
  }
  acc += __shfl_xor_sync(kFull, acc, 16);
  if (lane >= 16) acc = T(0);
  const size_t idx = (size_t)a * 16 + lane;
  if (lane < 16) C.b[idx] = acc;
  if (C.coarsest) return;
  const T dv = block_apply<T, 16>(dr, acc, lane) * (T)(1.0 / C.cheb[0]);
  if (lane < 16) {
    C.r[0][idx] = acc;
    C.d[0][idx] = dv;
    C.x[0][idx] = dv;
  }
}

// Restriction folded into the coarse level's first smoothing kernel (FP32 hierarchy).  The
// fine level's residual kernel leaves t_i = Q_i^T s_i per fine row, so b_a = sum_{i in a}
// t_i, and with x = 0 the coarse pre-smoothing steps 0 and 1 on row a are
//   d0 = D_a^-1 b_a / theta,  q = (A d0)_a = sum_j M_aj b_j  (M_aj = A_aj D_j^-1 / theta),
//   r1 = b_a - q,  d1 = c1 d0 + c2 D_a^-1 r1,  x = d0 + d1:
// the same iterate as the restriction kernel followed by step 1, one launch fewer.  The NW
// warps split row a's blocks; a warp reads a 16 x 16 block of M with 16-byte loads (lane
// l: float4 l and 32 + l, as cta_row_product16) and the matching four entries of b_j as
// the sum of t over j's fine members (listed per block in gptr / gmem).
constexpr int kGMem = 4;   // members per prefetched block kept in registers

struct GatherPrefetch {
  static constexpr int kPre = 2;
  int e, e1, n;
  int g0[kPre], g1[kPre];
  int m[kPre][kGMem];
  float4 a[kPre][2];
};

// sum over the members [g0, g1) (the first kGMem of them in m) of t's float4 at column cq
__device__ __forceinline__ float4 gather_t4(const float* __restrict__ rt, const int* __restrict__ gmem, int g0,
                                            int g1, const int* m, int cq) {
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < kGMem; ++k) {
    if (g0 + k < g1) {
      const float4 v = *reinterpret_cast<const float4*>(rt + (size_t)m[k] * 16 + cq);
      s.x += v.x, s.y += v.y, s.z += v.z, s.w += v.w;
    }
  }
  for (int g = g0 + kGMem; g < g1; ++g) {
    const float4 v = *reinterpret_cast<const float4*>(rt + (size_t)gmem[g] * 16 + cq);
    s.x += v.x, s.y += v.y, s.z += v.z, s.w += v.w;
  }
  return s;
}

template <int NW>
__global__ void __launch_bounds__(NW * 32) k_ph_cstep(VLevel<float> F, VLevel<float> C, int dc, int rc, int xc) {
  __shared__ float part[16 * NW];
  __shared__ float q[16], bsm[16], w[16];
  const int a = blockIdx.x, t = threadIdx.x, wi = t >> 5, lane = t & 31, cq = 4 * (lane & 3);
  // static data first: this warp's first blocks of row a of M with their member lists, row
  // t of D_a^-1 and the aggregate's own members
  GatherPrefetch p;
  p.n = 0;
  p.e1 = C.row_ptr[a + 1];
  int e = C.row_ptr[a] + wi;
#pragma unroll
  for (int k = 0; k < GatherPrefetch::kPre; ++k) {
    if (e < p.e1) {
      p.g0[k] = C.gptr[e];
      p.g1[k] = C.gptr[e + 1];
#pragma unroll
      for (int j = 0; j < kGMem; ++j) p.m[k][j] = p.g0[k] + j < p.g1[k] ? C.gmem[p.g0[k] + j] : 0;
      const float4* ab = reinterpret_cast<const float4*>(C.mvals + (size_t)e * 256);
      p.a[k][0] = ab[lane];
      p.a[k][1] = ab[32 + lane];
      p.n = k + 1;
      e += NW;
    }
  }
  p.e = e;
  float dr[16];
  int o0 = 0, o1 = 0, om[kGMem];
  if (t < 16) {
    dinv_row<float, 16>(C.Dinv + (size_t)a * 256, t, dr);
    o0 = F.agg_ptr[a];
    o1 = F.agg_ptr[a + 1];
#pragma unroll
    for (int j = 0; j < kGMem; ++j) om[j] = o0 + j < o1 ? F.agg_mem[o0 + j] : 0;
  }
  const float inv_theta = (float)(1.0 / C.cheb[0]);
  float c1 = 0.f, c2 = 0.f;
  if (t < 16) {
    double c1d, c2d;
    cheb_step(C.cheb, 1, c1d, c2d);
    c1 = (float)c1d;
    c2 = (float)c2d;
  }
  pdl_trigger();
  pdl_wait();
  // b_a
  if (t < 16) {
    float b = 0.f;
#pragma unroll
    for (int j = 0; j < kGMem; ++j)
      if (o0 + j < o1) b += F.rt[(size_t)om[j] * 16 + t];
    for (int g = o0 + kGMem; g < o1; ++g) b += F.rt[(size_t)F.agg_mem[g] * 16 + t];
    bsm[t] = b;
  }
  // q = sum_j M_aj b_j
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int k = 0; k < GatherPrefetch::kPre; ++k) {
    if (k < p.n) {
      const float4 xv = gather_t4(F.rt, C.gmem, p.g0[k], p.g1[k], p.m[k], cq);
      s0 += dot4(p.a[k][0], xv);
      s1 += dot4(p.a[k][1], xv);
    }
  }
  for (int e2 = p.e; e2 < p.e1; e2 += NW) {
    const float4* ab = reinterpret_cast<const float4*>(C.mvals + (size_t)e2 * 256);
    const float4 a0 = ab[lane], a1 = ab[32 + lane];
    const int g0 = C.gptr[e2], g1 = C.gptr[e2 + 1];
    int m[kGMem];
#pragma unroll
    for (int j = 0; j < kGMem; ++j) m[j] = g0 + j < g1 ? C.gmem[g0 + j] : 0;
    const float4 xv = gather_t4(F.rt, C.gmem, g0, g1, m, cq);
    s0 += dot4(a0, xv);
    s1 += dot4(a1, xv);
  }
  s0 += __shfl_xor_sync(kFull, s0, 1);
  s0 += __shfl_xor_sync(kFull, s0, 2);
  s1 += __shfl_xor_sync(kFull, s1, 1);
  s1 += __shfl_xor_sync(kFull, s1, 2);
  if ((lane & 3) == 0) {
    part[wi * 16 + (lane >> 2)] = s0;
    part[wi * 16 + 8 + (lane >> 2)] = s1;
  }
  __syncthreads();
  float d0 = 0.f;
  if (t < 16) {
    float qs = 0.f;
#pragma unroll
    for (int k = 0; k < NW; ++k) qs += part[k * 16 + t];
    d0 = row_dinv<float, 16>(dr, bsm) * inv_theta;
    w[t] = bsm[t] - qs;
  }
  __syncthreads();
  if (t < 16) {
    const float d1 = c1 * d0 + c2 * row_dinv<float, 16>(dr, w);
    const size_t idx = (size_t)a * 16 + t;
    C.r[1 - rc][idx] = w[t];
    C.d[1 - dc][idx] = d1;
    C.x[xc][idx] = d0 + d1;
  }
}

// x_c = A_c^-1 b_c, one warp per row of the dense inverse (the row prefetched while the
// previous kernel runs)
constexpr int kCoarseRowMax = 16;   // doubles of an inverse row per lane held in registers

template <typename T>
__global__ void __launch_bounds__(256) k_ph_coarsest(VLevel<T> C) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  double ar[kCoarseRowMax];
  const bool pre = gw < C.N && C.N <= 32 * kCoarseRowMax;
  if (pre) {
    const double* a = C.Ainv + (size_t)gw * C.Np;
#pragma unroll
    for (int k = 0; k < kCoarseRowMax; ++k) {
      const int j = lane + 32 * k;
      ar[k] = j < C.N ? a[j] : 0.0;
    }
  }
  pdl_trigger();
  pdl_wait();
  for (int row = gw; row < C.N; row += nw) {
    double acc = 0.0;
    if (pre && row == gw) {
#pragma unroll
      for (int k = 0; k < kCoarseRowMax; ++k) {
        const int j = lane + 32 * k;
        if (j < C.N) acc += ar[k] * (double)C.b[j];
      }
    } else {
      const double* a = C.Ainv + (size_t)row * C.Np;
      for (int j = lane; j < C.N; j += 32) acc += a[j] * (double)C.b[j];
    }
    acc = warp_sum(acc);
    if (lane == 0) C.x[0][row] = (T)acc;
  }
}

// The coarsest solve with the restriction into it folded in (coarsest level of at most
// kCoarseFoldMax dofs): every CTA forms b_c[16 a + s] = sum_{i in a} t_i[s] in shared
// memory from the t left by the last smoothed level's residual kernel, then x_c = A_c^-1
// b_c as k_ph_coarsest.  (Every CTA repeats the 4.6 KB gather of a 21-node coarsest
// level; the restriction launch it replaces cost about as much as a V-cycle phase.)
constexpr int kCoarseFoldMax = 32 * kCoarseRowMax;

template <typename T>
__global__ void __launch_bounds__(256) k_ph_coarsest_t(VLevel<T> F, VLevel<T> C) {
  __shared__ T bsm[kCoarseFoldMax];
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  // static data first: this warp's row of the inverse, and for this thread's entries of
  // b_c (k = threadIdx.x + 256 h) their members
  double ar[kCoarseRowMax];
  if (gw < C.N) {
    const double* a = C.Ainv + (size_t)gw * C.Np;
#pragma unroll
    for (int k = 0; k < kCoarseRowMax; ++k) {
      const int j = lane + 32 * k;
      ar[k] = j < C.N ? a[j] : 0.0;
    }
  }
  constexpr int kH = kCoarseFoldMax / 256;
  int g0[kH], g1[kH], m[kH][kGMem];
#pragma unroll
  for (int h = 0; h < kH; ++h) {
    const int k = threadIdx.x + 256 * h;
    g0[h] = g1[h] = 0;
    if (k < C.N) {
      g0[h] = F.agg_ptr[k >> 4];
      g1[h] = F.agg_ptr[(k >> 4) + 1];
    }
#pragma unroll
    for (int j = 0; j < kGMem; ++j) m[h][j] = g0[h] + j < g1[h] ? F.agg_mem[g0[h] + j] : 0;
  }
  pdl_trigger();
  pdl_wait();
#pragma unroll
  for (int h = 0; h < kH; ++h) {
    const int k = threadIdx.x + 256 * h;
    if (k < C.N) {
      T s = T(0);
#pragma unroll
      for (int j = 0; j < kGMem; ++j)
        if (g0[h] + j < g1[h]) s += F.rt[(size_t)m[h][j] * 16 + (k & 15)];
      for (int g = g0[h] + kGMem; g < g1[h]; ++g) s += F.rt[(size_t)F.agg_mem[g] * 16 + (k & 15)];
      bsm[k] = s;
    }
  }
  __syncthreads();
  for (int row = gw; row < C.N; row += nw) {
    double acc = 0.0;
    if (row == gw) {
#pragma unroll
      for (int k = 0; k < kCoarseRowMax; ++k) {
        const int j = lane + 32 * k;
        if (j < C.N) acc += ar[k] * (double)bsm[j];
      }
    } else {
      const double* a = C.Ainv + (size_t)row * C.Np;
      for (int j = lane; j < C.N; j += 32) acc += a[j] * (double)bsm[j];
    }
    acc = warp_sum(acc);
    if (lane == 0) C.x[0][row] = (T)acc;
  }
}

// Prolongation and post-smoothing step 0 in one launch, from A P (assembled with the
// hierarchy): with s = b - A x the residual of the pre-smoothed iterate (left in the free
// r buffer by the residual kernel) and x' = x + P x_c,
//   r = b - A x' = s - (A P) x_c,  d = D^-1 r / theta,  x'' = x' + d,
// so row i needs x_c only, not its neighbours' prolonged x'.
template <typename T, int BS>
__global__ void __launch_bounds__(RowCta<BS>::kThreads, phase_min_blocks<T, BS, 14>()) k_ph_post_first_ap(VLevel<T> L, VLevel<T> C, int xc, int xcl,
                                                                          int rc, int dc, double* __restrict__ out,
                                                                          const double* __restrict__ rdot,
                                                                          double* __restrict__ dpart) {
  constexpr int G = RowCta<BS>::G;
  constexpr int kPre = 2;
  constexpr bool kVec = sizeof(T) == 4;   // A P blocks are BS x 16 floats, 16-byte aligned
  constexpr int kNW = RowCta<BS>::kThreads / 32;
  __shared__ T part[RowCta<BS>::kPart];
  __shared__ T q[BS], w[BS];
  const int i = blockIdx.x, t = threadIdx.x;
  const int u = t % BS, h = t / BS;
  // static data first: this thread's first kPre blocks of (A P)_i (row u), Q_i row u, D_i^-1
  // row u and the aggregate of row i
  int e = 0, e1 = 0, np = 0;
  int pc[kPre];
  T pa[kPre][16];
  RowPrefetch16<BS> pf16;
  if constexpr (kVec) {
    row_prefetch16<BS, kNW>(L.ap_ptr, L.ap_cols, L.ap_vals, i, pf16);
  } else if (h < G) {
    e1 = L.ap_ptr[i + 1];
    e = L.ap_ptr[i] + h;
#pragma unroll
    for (int k = 0; k < kPre; ++k) {
      if (e < e1) {
        pc[k] = L.ap_cols[e];
        const T* a = L.ap_vals + (size_t)e * (BS * 16) + u * 16;
#pragma unroll
        for (int c = 0; c < 16; ++c) pa[k][c] = a[c];
        np = k + 1;
        e += G;
      }
    }
  }
  T dr[BS], qr[16];
  int ai = 0;
  if (t < BS) {
    dinv_row<T, BS>(L.Dinv + (size_t)i * BS * BS, t, dr);
    const T* Qi = L.Q + ((size_t)i * BS + t) * 16;
#pragma unroll
    for (int c = 0; c < 16; ++c) qr[c] = Qi[c];
    ai = L.agg[i];
  }
  pdl_trigger();
  pdl_wait();
  const T* xcv = C.x[xcl];
  if constexpr (kVec) {
    // (A P x_c)_i in q (the product synchronises the CTA)
    cta_row_product16<BS, kNW>(L.ap_cols, L.ap_vals, pf16, xcv, part, q);
  } else {
    if (h < G) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < kPre; ++k) {
        if (k < np) {
          const T* xa = xcv + (size_t)pc[k] * 16;
#pragma unroll
          for (int c = 0; c < 16; ++c) acc += pa[k][c] * xa[c];
        }
      }
      for (; e < e1; e += G) {
        const T* a = L.ap_vals + (size_t)e * (BS * 16) + u * 16;
        const T* xa = xcv + (size_t)L.ap_cols[e] * 16;
#pragma unroll
        for (int c = 0; c < 16; ++c) acc += a[c] * xa[c];
      }
      part[h * BS + u] = acc;
    }
    __syncthreads();
    if (t < BS) {
      T sq = T(0);
#pragma unroll
      for (int g = 0; g < G; ++g) sq += part[g * BS + t];
      q[t] = sq;
    }
  }
  __syncthreads();
  const size_t idx = (size_t)i * BS + t;
  T xp = T(0);
  if (t < BS) {
    const T sq = q[t];
    const T* xa = xcv + (size_t)ai * 16;
    T pq = T(0);
#pragma unroll
    for (int c = 0; c < 16; ++c) pq += qr[c] * xa[c];
    xp = L.x[xc][idx] + pq;
    w[t] = L.r[1 - rc][idx] - sq;
  }
  __syncthreads();
  double dot = 0.0;
  if (t < BS) {
    const T dv = row_dinv<T, BS>(dr, w) * (T)(1.0 / L.cheb[0]);
    const T xn = xp + dv;
    L.r[rc][idx] = w[t];
    L.d[dc][idx] = dv;
    L.x[1 - xc][idx] = xn;
    if (out) {
      out[idx] = (double)xn;
      if (dpart) dot = (double)xn * rdot[idx];
    }
  }
  if (dpart && t < 32) {
    dot = warp_sum(dot);
    if (t == 0) dpart[i] = dot;
  }
}

// (A P) blocks of a level, one CTA per block and one thread per entry (u, s): the sum over
// the listed A blocks of (A_ij Q_j)[u][s]
template <typename T, int BS>
__global__ void __launch_bounds__(256) k_ap_values(int nap, const int* __restrict__ lptr, const int* __restrict__ list,
                                                  const int* __restrict__ cols, const T* __restrict__ vals,
                                                  const T* __restrict__ Q, T* __restrict__ ap) {
  const int c = blockIdx.x, o = threadIdx.x;
  if (o >= BS * 16) return;
  const int uu = o / 16, ss = o - uu * 16;
  T acc = T(0);
  for (int k = lptr[c]; k < lptr[c + 1]; ++k) {
    const int e = list[k], j = cols[e];
    const T* a = vals + (size_t)e * BS * BS + uu * BS;
    const T* qj = Q + (size_t)j * BS * 16 + ss;
#pragma unroll
    for (int v = 0; v < BS; ++v) acc += a[v] * qj[v * 16];
  }
  ap[(size_t)c * BS * 16 + o] = acc;
}

// pattern of A P for a level (the distinct aggregates of each fine row's neighbours, in
// increasing order) and, per block, its contributing A blocks in row order
static void ap_symbolic(ba_problem* P, Level& L) {
  std::vector<int> rp(L.n + 1), cl(std::max(L.nnzb, 1)), agg(std::max(L.n, 1));
  BA_CUDA(cudaMemcpyAsync(rp.data(), L.row_ptr.p, sizeof(int) * (L.n + 1), cudaMemcpyDeviceToHost, P->stream));
  if (L.nnzb)
    BA_CUDA(cudaMemcpyAsync(cl.data(), L.cols.p, sizeof(int) * L.nnzb, cudaMemcpyDeviceToHost, P->stream));
  BA_CUDA(cudaMemcpyAsync(agg.data(), L.agg.p, sizeof(int) * L.n, cudaMemcpyDeviceToHost, P->stream));
  sync(P);
  std::vector<int> ap_ptr(L.n + 1, 0), ap_cols, lptr(1, 0), list;
  std::vector<int> aggs;
  for (int i = 0; i < L.n; ++i) {
    aggs.clear();
    for (int e = rp[i]; e < rp[i + 1]; ++e) aggs.push_back(agg[cl[e]]);
    std::sort(aggs.begin(), aggs.end());
    aggs.erase(std::unique(aggs.begin(), aggs.end()), aggs.end());
    for (int a : aggs) {
      ap_cols.push_back(a);
      for (int e = rp[i]; e < rp[i + 1]; ++e)
        if (agg[cl[e]] == a) list.push_back(e);
      lptr.push_back((int)list.size());
    }
    ap_ptr[i + 1] = (int)ap_cols.size();
  }
  L.ap_nnzb = (int)ap_cols.size();
  upload(P, L.ap_ptr, ap_ptr);
  upload(P, L.ap_cols, ap_cols);
  upload(P, L.ap_lptr, lptr);
  upload(P, L.ap_list, list);
  sync(P);
}

template <typename T>
static void ap_numeric(ba_problem* P, Level& L) {
  const bool fp32 = sizeof(T) == 4;
  L.ap_vals.ensure(sizeof(T) * (size_t)L.bs * 16 * std::max(L.ap_nnzb, 1) + 64);
  const int g = std::max(L.ap_nnzb, 1);
  const T* vals = fp32 ? (const T*)L.vals32.p : (const T*)L.vals64.p;
  const T* Q = fp32 ? (const T*)L.Q32.p : (const T*)L.Q64.p;
  if (L.ap_nnzb == 0) return;
  if (L.bs == 9)
    k_ap_values<T, 9><<<g, 160, 0, P->stream>>>(L.ap_nnzb, L.ap_lptr.as<int>(), L.ap_list.as<int>(), L.cols.as<int>(),
                                               vals, Q, L.ap_vals.as<T>());
  else
    k_ap_values<T, 16><<<g, 256, 0, P->stream>>>(L.ap_nnzb, L.ap_lptr.as<int>(), L.ap_list.as<int>(),
                                                L.cols.as<int>(), vals, Q, L.ap_vals.as<T>());
  launched(P);
}

void build_ap(ba_problem* P, Level& L) {
  if (!L.ap_ptr.p) ap_symbolic(P, L);
  if (level_fp32(P)) ap_numeric<float>(P, L);
  else ap_numeric<double>(P, L);
}

template <typename T>
static VLevel<T> describe(Level& L) {
  const bool fp32 = sizeof(T) == 4;
  VLevel<T> v{};
  v.n = L.n;
  v.bs = L.bs;
  v.coarsest = L.coarsest ? 1 : 0;
  v.N = L.n * L.bs;
  v.Np = L.N;
  v.row_ptr = L.row_ptr.as<int>();
  v.cols = L.cols.as<int>();
  v.vals = fp32 ? (const T*)L.vals32.p : (const T*)L.vals64.p;
  v.Dinv = fp32 ? (const T*)L.Dinv32.p : (const T*)L.Dinv64.p;
  v.Q = fp32 ? (const T*)L.Q32.p : (const T*)L.Q64.p;
  v.agg = L.agg.as<int>();
  v.agg_ptr = L.agg_ptr.as<int>();
  v.agg_mem = L.agg_mem.as<int>();
  v.cheb = L.cheb.as<double>();
  v.Ainv = L.Ainv.as<double>();
  v.ap_ptr = L.ap_ptr.as<int>();
  v.ap_cols = L.ap_cols.as<int>();
  v.ap_vals = (const T*)L.ap_vals.p;
  v.gptr = L.gptr.as<int>();
  v.gmem = L.gmem.as<int>();
  v.mvals = (const T*)L.mvals32.p;
  v.rt = (T*)L.rt.p;
  v.b = L.vb.as<T>();
  v.x[0] = L.vx.as<T>();
  v.x[1] = L.vt.as<T>();
  v.r[0] = L.vr.as<T>();
  v.r[1] = L.vs.as<T>();
  v.d[0] = L.vd.as<T>();
  v.d[1] = L.vq.as<T>();
  return v;
}

static int warps_grid(int warps) { return std::max(1, cdiv((long long)warps, kPhaseWarps)); }

template <typename T>
static void run(ba_problem* P, const double* r, double* z, double* dpart, bool first_done) {
  const int nl = P->n_levels;
  const int pre = std::max(1, P->opt.pre_smooth), post = std::max(1, P->opt.post_smooth);
  std::vector<VLevel<T>> V(nl);
  for (int l = 0; l < nl; ++l) V[l] = describe<T>(P->levels[l]);
  unsigned xm = 0, rm = 0, dm = 0;
  auto bit = [](unsigned m, int l) { return (int)((m >> l) & 1u); };
  cudaStream_t st = P->stream;
  for (int l = 0; l + 1 < nl; ++l) {
    const VLevel<T>& L = V[l];
    const bool folded = P->levels[l].folded, fold_next = P->levels[l + 1].folded;
    // step 0 of the coarse levels is done by the restriction that produces their b (on a
    // folded level: with step 1, by k_ph_cstep), and of level 0 by the PCG update when
    // first_done
    if (l == 0 && !first_done) {
      const int g = warps_grid(L.n);
      if (L.bs == 9) launch_k(P, k_ph_first<T, 9>, g, kPhaseBS, 0, L, r);
      else launch_k(P, k_ph_first<T, 16>, g, kPhaseBS, 0, L, r);
    }
    int k1 = 1;
    if constexpr (std::is_same_v<T, float>) {
      if (folded) {
        launch_k(P, k_ph_cstep<RowCta<16>::kThreads / 32>, L.n, RowCta<16>::kThreads, 0, V[l - 1], L, bit(dm, l),
                 bit(rm, l), bit(xm, l));
        rm ^= 1u << l;
        dm ^= 1u << l;
        k1 = 2;
      }
    }
    for (int k = k1; k < pre; ++k) {
      if (L.bs == 9)
        launch_k(P, k_ph_step<T, 9>, L.n, RowCta<9>::kThreads, 0, L, bit(dm, l), bit(rm, l), bit(xm, l), k,
                 (double*)nullptr, (const double*)nullptr, (double*)nullptr);
      else
        launch_k(P, k_ph_step<T, 16>, L.n, RowCta<16>::kThreads, 0, L, bit(dm, l), bit(rm, l), bit(xm, l), k,
                 (double*)nullptr, (const double*)nullptr, (double*)nullptr);
      rm ^= 1u << l;
      dm ^= 1u << l;
    }
    if (fold_next) {
      // the next level's restriction terms with the residual; no restriction launch
      if (L.bs == 9) launch_k(P, k_ph_residual<T, 9, true>, L.n, RowCta<9>::kThreads, 0, L, bit(dm, l), bit(rm, l));
      else launch_k(P, k_ph_residual<T, 16, true>, L.n, RowCta<16>::kThreads, 0, L, bit(dm, l), bit(rm, l));
      continue;
    }
    if (L.bs == 9) launch_k(P, k_ph_residual<T, 9>, L.n, RowCta<9>::kThreads, 0, L, bit(dm, l), bit(rm, l));
    else launch_k(P, k_ph_residual<T, 16>, L.n, RowCta<16>::kThreads, 0, L, bit(dm, l), bit(rm, l));
    const T* res = L.r[1 - bit(rm, l)];
    const int gc = warps_grid(V[l + 1].n);
    if (L.bs == 9) launch_k(P, k_ph_restrict<T, 9>, gc, kPhaseBS, 0, L, V[l + 1], res);
    else launch_k(P, k_ph_restrict<T, 16>, gc, kPhaseBS, 0, L, V[l + 1], res);
  }
  if (P->levels[nl - 1].folded)
    launch_k(P, k_ph_coarsest_t<T>, warps_grid(V[nl - 1].N), kPhaseBS, 0, V[nl - 2], V[nl - 1]);
  else
    launch_k(P, k_ph_coarsest<T>, warps_grid(V[nl - 1].N), kPhaseBS, 0, V[nl - 1]);
  for (int l = nl - 2; l >= 0; --l) {
    const VLevel<T>& L = V[l];
    double* o = (l == 0 && post == 1) ? z : nullptr;
    double* op = o ? dpart : nullptr;
    if (L.bs == 9)
      launch_k(P, k_ph_post_first_ap<T, 9>, L.n, RowCta<9>::kThreads, 0, L, V[l + 1], bit(xm, l), bit(xm, l + 1),
               bit(rm, l), bit(dm, l), o, r, op);
    else
      launch_k(P, k_ph_post_first_ap<T, 16>, L.n, RowCta<16>::kThreads, 0, L, V[l + 1], bit(xm, l), bit(xm, l + 1),
               bit(rm, l), bit(dm, l), o, r, op);
    xm ^= 1u << l;
    for (int k = 1; k < post; ++k) {
      double* ok = (l == 0 && k == post - 1) ? z : nullptr;
      double* okp = ok ? dpart : nullptr;
      if (L.bs == 9)
        launch_k(P, k_ph_step<T, 9>, L.n, RowCta<9>::kThreads, 0, L, bit(dm, l), bit(rm, l), bit(xm, l), k, ok, r,
                 okp);
      else
        launch_k(P, k_ph_step<T, 16>, L.n, RowCta<16>::kThreads, 0, L, bit(dm, l), bit(rm, l), bit(xm, l), k, ok, r,
                 okp);
      rm ^= 1u << l;
      dm ^= 1u << l;
    }
  }
}

// M_aj = A_aj D_j^-1 / theta of the folded coarse levels, all in one launch: CTA b is block
// b - off[k] of level k (off[k] <= b < off[k + 1]), thread (u, v) entry (u, v)
struct FoldBatch {
  int n;
  int off[17];
  const int* cols[16];
  const float* vals[16];
  const float* dinv[16];
  const double* cheb[16];
  float* out[16];
};

__global__ void __launch_bounds__(256) k_fold_blocks(FoldBatch FB) {
  __shared__ float A[256], D[256];
  const int t = threadIdx.x, u = t >> 4, v = t & 15;
  int k = 0;
  while (k + 1 < FB.n && (int)blockIdx.x >= FB.off[k + 1]) ++k;
  const int e = (int)blockIdx.x - FB.off[k];
  if (e >= FB.off[k + 1] - FB.off[k]) return;
  A[t] = FB.vals[k][(size_t)e * 256 + t];
  D[t] = FB.dinv[k][(size_t)FB.cols[k][e] * 256 + t];
  __syncthreads();
  float s = 0.f;
#pragma unroll
  for (int w = 0; w < 16; ++w) s += A[u * 16 + w] * D[w * 16 + v];
  FB.out[k][(size_t)e * 256 + t] = s * (float)(1.0 / FB.cheb[k][0]);
}

// per block (a, j) of coarse level C, the fine members of aggregate j (F's member lists),
// once per hierarchy
static void fold_symbolic(ba_problem* P, Level& F, Level& C) {
  std::vector<int> rp(C.n + 1), cl(std::max(C.nnzb, 1)), ap(C.n + 1), am(std::max(F.n, 1));
  BA_CUDA(cudaMemcpyAsync(rp.data(), C.row_ptr.p, sizeof(int) * (C.n + 1), cudaMemcpyDeviceToHost, P->stream));
  if (C.nnzb) BA_CUDA(cudaMemcpyAsync(cl.data(), C.cols.p, sizeof(int) * C.nnzb, cudaMemcpyDeviceToHost, P->stream));
  BA_CUDA(cudaMemcpyAsync(ap.data(), F.agg_ptr.p, sizeof(int) * (C.n + 1), cudaMemcpyDeviceToHost, P->stream));
  if (F.n) BA_CUDA(cudaMemcpyAsync(am.data(), F.agg_mem.p, sizeof(int) * F.n, cudaMemcpyDeviceToHost, P->stream));
  sync(P);
  BA_REQUIRE(ap[C.n] == F.n, BA_ERR_STATE, "aggregates do not cover the fine level");
  std::vector<int> gptr(1, 0), gmem;
  gmem.reserve((size_t)C.nnzb * 4);
  for (int e = 0; e < C.nnzb; ++e) {
    const int j = cl[e];
    for (int g = ap[j]; g < ap[j + 1]; ++g) gmem.push_back(am[g]);
    gptr.push_back((int)gmem.size());
  }
  if (gmem.empty()) gmem.push_back(0);
  upload(P, C.gptr, gptr);
  upload(P, C.gmem, gmem);
  sync(P);
}

// A folded level's first step reads M instead of A, so A loses its L2 reuse between that
// step and the residual, and M is formed at every setup: the fold saves a launch only on
// levels whose operator costs less than a launch (about 2.5 us) to stream again.  Measured:
// street chain (levels of 11, 3 and 0.6 MB) V-cycle 67.0 -> 63.8 us; city grid with every
// level folded (level 1: 110 MB) PCG 9.0 -> 9.3 ms and setup 8.0 -> 8.3 ms.
constexpr size_t kFoldMaxBytes = size_t(16) << 20;

// Called at the end of the multigrid setup: whether the fused-phase cycle applies, and
// which coarse levels take their restriction folded into their first smoothing kernel
// (FP32 hierarchy with at least two pre-smoothing steps; smoothed coarse levels whose FP32
// operator is at most kFoldMaxBytes)
void fused_vcycle_setup(ba_problem* P) {
  P->vc_ready = false;
  for (int l = 0; l < P->n_levels; ++l) P->levels[l].folded = false;
  if (!P->opt.fused_vcycle || !P->l0_explicit || P->n_levels < 2) return;
  for (int l = 0; l + 1 < P->n_levels; ++l) {
    const int bs = P->levels[l].bs;
    if (bs != 9 && bs != 16) return;
  }
  // (A P of every smoothed level, for the fused prolongation + post-smoothing start, was
  // assembled with the Galerkin products)
  P->vc_ready = true;
  {
    // the restriction into a small coarsest level goes into its solve (k_ph_coarsest_t)
    Level& C = P->levels[P->n_levels - 1];
    Level& F = P->levels[P->n_levels - 2];
    if (C.coarsest && C.bs == 16 && C.n * C.bs <= kCoarseFoldMax) {
      F.rt.ensure((level_fp32(P) ? sizeof(float) : sizeof(double)) * 16 * (size_t)std::max(F.n, 1) + 64);
      C.folded = true;
    }
  }
  if (!level_fp32(P) || P->opt.pre_smooth < 2) return;
  FoldBatch FB{};
  FB.off[0] = 0;
  for (int l = 1; l + 1 < P->n_levels && FB.n < 16; ++l) {
    Level& C = P->levels[l];
    Level& F = P->levels[l - 1];
    if (C.coarsest || C.bs != 16 || sizeof(float) * 256 * (size_t)C.nnzb > kFoldMaxBytes) continue;
    if (!C.gptr.p) fold_symbolic(P, F, C);
    C.mvals32.ensure(sizeof(float) * 256 * (size_t)std::max(C.nnzb, 1) + 64);
    F.rt.ensure(sizeof(float) * 16 * (size_t)std::max(F.n, 1) + 64);
    const int k = FB.n++;
    FB.cols[k] = C.cols.as<int>();
    FB.vals[k] = C.vals32.as<float>();
    FB.dinv[k] = C.Dinv32.as<float>();
    FB.cheb[k] = C.cheb.as<double>();
    FB.out[k] = C.mvals32.as<float>();
    FB.off[k + 1] = FB.off[k] + C.nnzb;
    C.folded = true;
  }
  if (FB.n > 0 && FB.off[FB.n] > 0) {
    k_fold_blocks<<<FB.off[FB.n], 256, 0, P->stream>>>(FB);
    launched(P);
  }
}

void fused_vcycle(ba_problem* P, const double* r, double* z, double* rz_part, bool first_done) {
  if (level_fp32(P)) run<float>(P, r, z, rz_part, first_done);
  else run<double>(P, r, z, rz_part, first_done);
}

template <typename T>
static void update_first(ba_problem* P, double* x, double* r, const double* p, const double* q, const PcgCheck& ck) {
  const VLevel<T> L = describe<T>(P->levels[0]);
  // at most 16 CTAs per SM: the r.r partials have one slot per CTA
  const int grid = std::max(1, std::min(cdiv((long long)L.n, kUpdRows), 8 * P->n_sm));
  launch_k(P, k_pcg_update_first<T>, grid, kUpdBS, 0, L, x, r, p, q, ck);
}

void fused_update_first(ba_problem* P, double* x, double* r, const double* p, const double* q, const PcgCheck& ck) {
  BA_REQUIRE(P->vc_ready && P->levels[0].bs == 9, BA_ERR_STATE, "fused update without the fused V-cycle");
  if (level_fp32(P)) update_first<float>(P, x, r, p, q, ck);
  else update_first<double>(P, x, r, p, q, ck);
}

}  // namespace ba
