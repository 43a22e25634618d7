// V-cycle (Algorithm 1) with the Chebyshev / point-block-Jacobi smoother of
// Section 3.4, PCG on S (Section 3.6) and one Levenberg-Marquardt step (Section 2.1).
#include <algorithm>
#include <cmath>

#include "ba_internal.h"
#include "device_util.cuh"
#include "dfloat.cuh"
#include "pcg_update.cuh"

namespace ba {

void back_substitute_to(ba_problem* P, const double* dc, double* out_int, double* out_user);

bool level_fp32(ba_problem* P) { return P->opt.precision == BA_MIXED; }

// ---------------------------------------------------------------------------
// level operators
// ---------------------------------------------------------------------------
// y = A x for a 16x16-block BSR operator; 16 threads per block row.
template <typename T>
__global__ void k_bsr16_spmv(int n, const int* __restrict__ row_ptr, const int* __restrict__ cols,
                             const T* __restrict__ vals, const T* __restrict__ x, T* __restrict__ y) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gid >> 4, u = gid & 15;
  if (i >= n) return;
  float accf = 0.0f;
  double accd = 0.0;
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
    const T* a = vals + (size_t)e * 256 + u * 16;
    const T* xv = x + (size_t)cols[e] * 16;
#pragma unroll
    for (int v = 0; v < 16; ++v) {
      if (sizeof(T) == 4) accf += (float)a[v] * (float)xv[v];
      else accd += (double)a[v] * (double)xv[v];
    }
  }
  y[(size_t)i * 16 + u] = sizeof(T) == 4 ? (T)accf : (T)accd;
}

// y = S x for the assembled 9x9-block camera system: one warp per block row; lane
// r + 9k (k < 3) takes output row r of blocks k, k+3, ... of the row, and the three
// partial sums of row r meet in lane r.
template <typename T>
__global__ void k_bsr9_spmv(int n, const int* __restrict__ row_ptr, const int* __restrict__ cols,
                            const T* __restrict__ vals, const T* __restrict__ x, T* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const int r = lane % 9, k = lane / 9;
  T acc = T(0);
  if (k < 3) {
    const int e1 = row_ptr[i + 1];
    for (int e = row_ptr[i] + k; e < e1; e += 3) {
      const T* a = vals + (size_t)e * 81 + r * 9;
      const T* xv = x + (size_t)cols[e] * 9;
#pragma unroll
      for (int c = 0; c < 9; ++c) acc += __ldg(a + c) * __ldg(xv + c);
    }
  }
  const T a1 = __shfl_sync(kFull, acc, min(lane + 9, 31));
  const T a2 = __shfl_sync(kFull, acc, min(lane + 18, 31));
  if (lane < 9) y[(size_t)i * 9 + r] = acc + a1 + a2;
}

// y = A_l x.  At level 0 with `ready`, y already holds D_c x (written by the kernel
// that produced x) and the product only accumulates.
void level_matvec(ba_problem* P, int l, const void* x, void* y, bool ready) {
  Level& L = P->levels[l];
  const bool fp32 = level_fp32(P);
  if (l == 0 && P->l0_explicit) {
    // the assembled S already holds D_c: overwrite y
    const int g = cdiv(L.n, 4);
    if (fp32)
      k_bsr9_spmv<float><<<g, 128, 0, P->stream>>>(L.n, L.row_ptr.as<int>(), L.cols.as<int>(),
                                                   L.vals32.as<float>(), (const float*)x, (float*)y);
    else
      k_bsr9_spmv<double><<<g, 128, 0, P->stream>>>(L.n, L.row_ptr.as<int>(), L.cols.as<int>(),
                                                    L.vals64.as<double>(), (const double*)x, (double*)y);
    launched(P);
    return;
  }
  if (l == 0) {
    if (fp32) {
      if (ready) matvec32_accumulate(P, (const float*)x, (float*)y);
      else matvec32(P, (const float*)x, (float*)y);
    } else {
      if (ready) matvec64_accumulate(P, (const double*)x, (double*)y);
      else matvec64(P, (const double*)x, (double*)y);
    }
    return;
  }
  const int g = cdiv((long long)L.n * 16, 64);   // small blocks: spread coarse rows over all SMs
  if (fp32)
    k_bsr16_spmv<float><<<g, 64, 0, P->stream>>>(L.n, L.row_ptr.as<int>(), L.cols.as<int>(), L.vals32.as<float>(),
                                                  (const float*)x, (float*)y);
  else
    k_bsr16_spmv<double><<<g, 64, 0, P->stream>>>(L.n, L.row_ptr.as<int>(), L.cols.as<int>(),
                                                   L.vals64.as<double>(), (const double*)x, (double*)y);
  launched(P);
}

// ---------------------------------------------------------------------------
// Chebyshev semi-iteration (Saad, Iterative Methods, Alg. 12.1) preconditioned by
// point-block Jacobi on [lo, hi]; cheb = {theta, delta, sigma_1, lambda_max}.
// rho_0 = 1/sigma_1, rho_k = 1/(2 sigma_1 - rho_{k-1}).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cheb_rho(const double* cheb, int k) {
  double rho = 1.0 / cheb[2];
  for (int j = 1; j <= k; ++j) rho = 1.0 / (2.0 * cheb[2] - rho);
  return rho;
}

// Every kernel that produces the vector a level-0 product is applied to next also writes
// yn = Dn o (that vector), the product's diagonal term, so the product itself only
// accumulates (Dn = null at the block-sparse coarse levels).

// step 0: r = b - q (q null: x = 0), d = D^-1 r / theta, x = x + d, yn = Dn o d
template <typename T>
__global__ void k_cheb_first(int n, int bs, const T* __restrict__ Dinv, const T* __restrict__ b,
                             const T* __restrict__ q, T* __restrict__ r, T* __restrict__ d, T* __restrict__ x,
                             int x_zero, const double* __restrict__ cheb, const T* __restrict__ Dn,
                             T* __restrict__ yn) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * bs) return;
  const size_t i = idx / bs;
  const int u = (int)(idx - i * bs);
  const T* Di = Dinv + (i * bs + u) * bs;
  const T* bi = b + i * bs;
  const T* qi = q ? q + i * bs : nullptr;
  T acc = T(0);
  for (int v = 0; v < bs; ++v) acc += Di[v] * (qi ? bi[v] - qi[v] : bi[v]);
  const T ri = q ? b[idx] - q[idx] : b[idx];
  const T di = acc * (T)(1.0 / cheb[0]);
  r[idx] = ri;
  d[idx] = di;
  x[idx] = x_zero ? di : x[idx] + di;
  if (Dn) yn[idx] = Dn[idx] * di;
}

// step k >= 1: r_out = r_in - q; d = rho_k rho_{k-1} d + (2 rho_k / delta) D^-1 r_out;
// x = x + d; yn = Dn o d   (r_in and r_out are different buffers)
template <typename T>
__global__ void k_cheb_step(int n, int bs, const T* __restrict__ Dinv, const T* __restrict__ r_in,
                            const T* __restrict__ q, T* __restrict__ r_out, T* __restrict__ d, T* __restrict__ x,
                            const double* __restrict__ cheb, int k, const T* __restrict__ Dn,
                            T* __restrict__ yn) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * bs) return;
  const size_t i = idx / bs;
  const int u = (int)(idx - i * bs);
  const T* Di = Dinv + (i * bs + u) * bs;
  const T* ri = r_in + i * bs;
  const T* qi = q + i * bs;
  T acc = T(0);
  for (int v = 0; v < bs; ++v) acc += Di[v] * (ri[v] - qi[v]);
  r_out[idx] = r_in[idx] - q[idx];
  const double rk = cheb_rho(cheb, k), rk1 = cheb_rho(cheb, k - 1);
  const T dn = (T)(rk * rk1) * d[idx] + (T)(2.0 * rk / cheb[1]) * acc;
  d[idx] = dn;
  x[idx] += dn;
  if (Dn) yn[idx] = Dn[idx] * dn;
}

// rc[a][s] = sum_{i in a} sum_u Q_i[u][s] (r_i[u] - q_i[u])   (restriction R = P^T)
template <typename T>
__global__ void k_restrict(int n_agg, int bs, const int* __restrict__ mptr, const int* __restrict__ mem,
                           const T* __restrict__ Q, const T* __restrict__ r, const T* __restrict__ q,
                           T* __restrict__ rc) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = gid >> 4, s = gid & 15;
  if (a >= n_agg) return;
  T acc = T(0);
  for (int k = mptr[a]; k < mptr[a + 1]; ++k) {
    const int i = mem[k];
    const T* Qi = Q + (size_t)i * bs * 16;
    for (int u = 0; u < bs; ++u) {
      const T rv = q ? r[(size_t)i * bs + u] - q[(size_t)i * bs + u] : r[(size_t)i * bs + u];
      acc += Qi[u * 16 + s] * rv;
    }
  }
  rc[(size_t)a * 16 + s] = acc;
}

// x_i += Q_i xc_{agg(i)} (prolongation); yn = Dn o x
template <typename T>
__global__ void k_prolong(int n, int bs, const int* __restrict__ agg, const T* __restrict__ Q,
                          const T* __restrict__ xc, T* __restrict__ x, const T* __restrict__ Dn,
                          T* __restrict__ yn) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * bs) return;
  const size_t i = idx / bs;
  const int u = (int)(idx - i * bs);
  const T* Qi = Q + (i * bs + u) * 16;
  const T* xa = xc + (size_t)agg[i] * 16;
  T acc = T(0);
#pragma unroll
  for (int s = 0; s < 16; ++s) acc += Qi[s] * xa[s];
  const T xn = x[idx] + acc;
  x[idx] = xn;
  if (Dn) yn[idx] = Dn[idx] * xn;
}

// coarsest level: x = Ainv b (FP64 inverse, padded to Np; b beyond N is zero)
template <typename T>
__global__ void k_dense_apply(int N, int Np, const double* __restrict__ Ainv, const T* __restrict__ b,
                              T* __restrict__ x) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  const double* a = Ainv + (size_t)row * Np;
  double acc = 0.0;
  for (int j = lane; j < N; j += 32) acc += a[j] * (double)b[j];
  acc = warp_sum(acc);
  if (lane == 0) x[row] = (T)acc;
}

template <typename T>
static const T* dinv(Level& L) {
  return sizeof(T) == 4 ? (const T*)L.Dinv32.p : (const T*)L.Dinv64.p;
}
template <typename T>
static const T* qblk(Level& L) {
  return sizeof(T) == 4 ? (const T*)L.Q32.p : (const T*)L.Q64.p;
}
// D_c in the V-cycle's precision (level 0 only)
template <typename T>
static const T* diag0(ba_problem* P, int l) {
  if (l != 0) return nullptr;
  return sizeof(T) == 4 ? (const T*)P->Dc32.p : (const T*)P->Dc.p;
}

// Chebyshev smoothing of A x = b with residual buffers rr[2] and product buffers qq[2].
// On entry with x_zero false, qq[qi] holds A x.  On exit rr[ri] = b - A (x - d), d is
// the last update and (level 0) qq[qi] holds D_c d, ready for the product A d.
template <typename T>
static void smooth(ba_problem* P, int l, T* x, const T* b, T** rr, int& ri, T* d, T** qq, int& qi, int steps,
                   bool x_zero) {
  Level& L = P->levels[l];
  const size_t n = (size_t)L.n * L.bs;
  const int g = cdiv((long long)n, 256);
  const double* cheb = L.cheb.as<double>();
  const T* Dn = diag0<T>(P, l);
  const T* qin = x_zero ? nullptr : qq[qi];
  const int qn = x_zero ? qi : 1 - qi;
  k_cheb_first<T><<<g, 256, 0, P->stream>>>(L.n, L.bs, dinv<T>(L), b, qin, rr[ri], d, x, x_zero, cheb, Dn, qq[qn]);
  launched(P);
  qi = qn;
  for (int k = 1; k < steps; ++k) {
    level_matvec(P, l, d, qq[qi], true);
    const int qn2 = 1 - qi;
    k_cheb_step<T><<<g, 256, 0, P->stream>>>(L.n, L.bs, dinv<T>(L), rr[ri], qq[qi], rr[1 - ri], d, x, cheb, k, Dn,
                                            qq[qn2]);
    launched(P);
    ri = 1 - ri;
    qi = qn2;
  }
}

// x = mgcycle(l, 0, b)   (Algorithm 1)
template <typename T>
static void vcycle(ba_problem* P, int l, const T* b, T* x) {
  Level& L = P->levels[l];
  if (L.coarsest) {
    const int N = L.n * L.bs;
    k_dense_apply<T><<<cdiv((long long)N * 32, 256), 256, 0, P->stream>>>(N, L.N, L.Ainv.as<double>(), b, x);
    launched(P);
    return;
  }
  T* rr[2] = {L.vr.as<T>(), L.vs.as<T>()};
  T* qq[2] = {L.vq.as<T>(), L.vt.as<T>()};
  T* d = L.vd.as<T>();
  int ri = 0, qi = 0;
  const int pre = std::max(1, P->opt.pre_smooth), post = std::max(1, P->opt.post_smooth);
  smooth<T>(P, l, x, b, rr, ri, d, qq, qi, pre, true);         // pre-smoothing
  level_matvec(P, l, d, qq[qi], true);                         // residual b - A x = r - A d
  Level& C = P->levels[l + 1];
  T* rc = C.vb.as<T>();
  T* xc = C.vx.as<T>();
  k_restrict<T><<<cdiv((long long)C.n * 16, 64), 64, 0, P->stream>>>(C.n, L.bs, L.agg_ptr.as<int>(),
                                                                   L.agg_mem.as<int>(), qblk<T>(L), rr[ri],
                                                                   qq[qi], rc);
  launched(P);                                                 // restriction
  vcycle<T>(P, l + 1, rc, xc);                                 // coarse-level solve
  qi = 1 - qi;
  k_prolong<T><<<cdiv((long long)L.n * L.bs, 256), 256, 0, P->stream>>>(L.n, L.bs, L.agg.as<int>(), qblk<T>(L),
                                                                      xc, x, diag0<T>(P, l), qq[qi]);
  launched(P);                                                 // prolongation
  level_matvec(P, l, x, qq[qi], true);                         // A x for the post-smoothing
  smooth<T>(P, l, x, b, rr, ri, d, qq, qi, post, false);       // post-smoothing
}

// ---------------------------------------------------------------------------
// preconditioner application on FP64 camera vectors
// ---------------------------------------------------------------------------
__global__ void k_to_float(size_t n, const double* __restrict__ a, float* __restrict__ b) {
  pdl_wait();
  pdl_trigger();
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_to_double(size_t n, const float* __restrict__ a, double* __restrict__ b) {
  pdl_wait();
  pdl_trigger();
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}
__global__ void k_blockdiag9(int n, const double* __restrict__ B, const double* __restrict__ x,
                             double* __restrict__ y) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * 9) return;
  const size_t i = idx / 9;
  const int u = (int)(idx - i * 9);
  const double* b = B + i * 81 + u * 9;
  const double* xi = x + i * 9;
  double acc = 0.0;
#pragma unroll
  for (int v = 0; v < 9; ++v) acc += b[v] * xi[v];
  y[idx] = acc;
}

void precond_apply(ba_problem* P, const double* r, double* z) {
  const size_t n = (size_t)P->n_c * 9;
  const int g = cdiv((long long)n, 256);
  const int pc = P->opt.preconditioner;
  if (pc == BA_PRECOND_NONE) {
    BA_CUDA(cudaMemcpyAsync(z, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream));
    return;
  }
  if (pc == BA_PRECOND_JACOBI) {
    k_blockdiag9<<<g, 256, 0, P->stream>>>(P->n_c, P->Scc_inv.as<double>(), r, z);
    launched(P);
    return;
  }
  BA_REQUIRE(P->n_levels > 0, BA_ERR_STATE, "ba_mg_setup has not been run");
  KernelTimer kt(P, BA_KT_VCYCLE);
  if (P->vc_ready) {
    fused_vcycle(P, r, z, nullptr, false);
    return;
  }
  Level& L0 = P->levels[0];
  if (level_fp32(P)) {
    float* b = L0.vb.as<float>();
    float* x = L0.vx.as<float>();
    launch_k(P, k_to_float, g, 256, 0, n, r, b);
    vcycle<float>(P, 0, b, x);
    launch_k(P, k_to_double, g, 256, 0, n, x, z);
  } else {
    double* b = L0.vb.as<double>();
    BA_CUDA(cudaMemcpyAsync(b, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream));
    vcycle<double>(P, 0, b, z);
  }
}

// ---------------------------------------------------------------------------
// PCG
// ---------------------------------------------------------------------------
constexpr int kVecBS = 256;

// x += alpha p; r -= alpha q; S_RR = r.r ; alpha = scal[rz] / scal[pq]
__global__ void __launch_bounds__(kVecBS)
k_pcg_update(size_t n, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
             const double* __restrict__ q, double* scal, int s_rz, double* partial, unsigned* counter,
             int* flags) {
  pdl_wait();
  pdl_trigger();
  const double pq = scal[S_PQ];
  const double alpha = scal[s_rz] / pq;
  const bool ok = pq > 0.0 && isfinite(alpha);
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * kVecBS + threadIdx.x; i < n; i += (size_t)gridDim.x * kVecBS) {
    double ri = r[i];
    if (ok) {
      x[i] += alpha * p[i];
      ri -= alpha * q[i];
      r[i] = ri;
    }
    acc += ri * ri;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (!ok) flags[F_BREAKDOWN] = 1;
    // quadratic model: Q_i - Q_{i-1} = -alpha (r.z) / 2
    const double dq = ok ? -0.5 * alpha * scal[s_rz] : 0.0;
    scal[S_DQ] = dq;
    scal[S_Q] += dq;
  }
  grid_sum_store<kVecBS>(acc, partial, counter, scal + S_RR);
}

// p = z + beta p, beta = scal[rz_new] / scal[rz_old] (s_new < 0: p = z); q = D_c p, the
// diagonal term of the next product S p; ps (if given) = hi/lo float split of p, the
// input of the paired-FP32 product
__global__ void k_pcg_direction(size_t n, double* __restrict__ p, const double* __restrict__ z,
                                const double* __restrict__ scal, int s_new, int s_old,
                                const double* __restrict__ Dc, double* __restrict__ q, float2* __restrict__ ps) {
  pdl_wait();
  pdl_trigger();
  const double beta = s_new >= 0 ? scal[s_new] / scal[s_old] : 0.0;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double pi = s_new >= 0 ? z[i] + beta * p[i] : z[i];
    p[i] = pi;
    if (q) q[i] = Dc[i] * pi;
    if (ps) {
      const float h = (float)pi;
      ps[i] = make_float2(h, (float)(pi - (double)h));
    }
  }
}

static float2* split_target(ba_problem* P) {
  if (!outer_df(P) || P->outer_explicit) return nullptr;
  P->xsplit.ensure(sizeof(float2) * 9 * (size_t)P->n_c + 64);
  return P->xsplit.as<float2>();
}

// q = S p for the PCG with the implicit operator: the product added to q = D_c p,
// written with p
static void outer_product(ba_problem* P, const double* p, double* q) { matvec64_accumulate(P, p, q); }

// one PCG iteration's head: q = S p; alpha = rz / p.q; x += alpha p; r -= alpha q; rr = r.r
static void pcg_head(ba_problem* P, double* x) {
  const size_t n = (size_t)P->n_c * 9;
  double *r = P->r.as<double>(), *p = P->p.as<double>(), *q = P->q.as<double>();
  outer_product(P, p, q);
  dot64(P, p, q, n, S_PQ);
  launch_k(P, k_pcg_update, reduce_blocks(P, n), kVecBS, 0, n, x, r, p, q, P->scal.as<double>(), S_RZ,
                                                              P->partial.as<double>(), P->counter.as<unsigned>(),
                                                              P->flags.as<int>());
}

// counts the iteration and sets the loop condition: continue while not converged
// (pcg_converged), no breakdown and fewer than max_iters iterations
__global__ void k_pcg_check(double* scal, const int* flags, int max_iters, double rtol2, int rule, double tau,
                            cudaGraphConditionalHandle h) {
  pdl_wait();
  pdl_trigger();
  const double it = scal[S_ITER] + 1.0;
  scal[S_ITER] = it;
  const double rr = scal[S_RR], bb = scal[S_BB];
  const bool stop = pcg_converged(rule, it, rr, bb, rtol2, scal[S_Q], scal[S_DQ], tau) ||
                    flags[F_BREAKDOWN] != 0 || it >= (double)max_iters;
  cudaGraphSetConditional(h, stop ? 0u : 1u);
}

__global__ void k_copy_slot(double* scal, int dst, int src) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x == 0) scal[dst] = scal[src];
}

// one PCG iteration's tail: z = M r; beta = r.z / rz; p = z + beta p; rz = r.z
static void pcg_tail(ba_problem* P) {
  const size_t n = (size_t)P->n_c * 9;
  double *r = P->r.as<double>(), *z = P->z.as<double>(), *p = P->p.as<double>();
  precond_apply(P, r, z);
  dot64(P, r, z, n, S_TMP2);
  launch_k(P, k_pcg_direction, cdiv((long long)n, 256), 256, 0, n, p, z, P->scal.as<double>(), S_TMP2, S_RZ,
                                                                   P->Dc.as<double>(), P->q.as<double>(),
                                                                   split_target(P));
  launch_k(P, k_copy_slot, 1, 32, 0, P->scal.as<double>(), S_RZ, S_TMP2);
}

// ---------------------------------------------------------------------------
// PCG with the assembled S (the PCG product of Section 3.6's choice when level 0 is
// assembled): an iteration is the V-cycle, r.z, the direction update and two kernels,
//   k_pcg_spmv_pq:       q = S p and p.q
//   k_pcg_update_check:  alpha = r.z / p.q, x += alpha p, r -= alpha q, r.r, the
//                        quadratic model, the stopping test and the graph condition
// so the recurrences are the ones of the launch-per-operation path above, fused.
// ---------------------------------------------------------------------------
constexpr int kSpmvBS = 128;

// the product's p.q: summed over the grid by its last CTA into pq_out, or (pq_out null)
// left as one share per CTA for the update kernel to add
__device__ __forceinline__ void spmv_pq_store(double dot, double* partial, unsigned* counter, double* pq_out) {
  if (pq_out) {
    grid_sum_store<kSpmvBS>(dot, partial, counter, pq_out);
    return;
  }
  const double s = block_sum<kSpmvBS>(dot);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// q = S p with the FP64 blocks (one warp per block row: lane r + 9k takes row r of
// blocks k, k + 3, ...; its first block is loaded before the programmatic wait) and p.q
__global__ void __launch_bounds__(kSpmvBS)
k_pcg_spmv_pq(int n, const int* __restrict__ row_ptr, const int* __restrict__ cols, const double* __restrict__ vals,
              const double* __restrict__ p, double* __restrict__ q, double* partial, unsigned* counter,
              double* pq_out) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (kSpmvBS / 32) + (threadIdx.x >> 5);
  const int r = lane % 9, k = lane / 9;
  const bool live = i < n && k < 3;
  int e0 = 0, e1 = 0, c0 = 0;
  double a0[9];
  if (live) {
    e0 = row_ptr[i] + k;
    e1 = row_ptr[i + 1];
    const int ef = min(e0, max(e1 - 1, 0));
    c0 = cols[ef];
    const double* a = vals + (size_t)ef * 81 + r * 9;
#pragma unroll
    for (int c = 0; c < 9; ++c) a0[c] = a[c];
  }
  pdl_trigger();
  pdl_wait();
  double acc = 0.0;
  if (live && e0 < e1) {
    const double* x0 = p + (size_t)c0 * 9;
#pragma unroll
    for (int c = 0; c < 9; ++c) acc += a0[c] * x0[c];
    for (int e = e0 + 3; e < e1; e += 3) {
      const double* a = vals + (size_t)e * 81 + r * 9;
      const double* xv = p + (size_t)cols[e] * 9;
#pragma unroll
      for (int c = 0; c < 9; ++c) acc += a[c] * xv[c];
    }
  }
  const double a1 = __shfl_sync(kFull, acc, min(lane + 9, 31));
  const double a2 = __shfl_sync(kFull, acc, min(lane + 18, 31));
  double dot = 0.0;
  if (i < n && lane < 9) {
    const size_t idx = (size_t)i * 9 + r;
    const double qi = acc + a1 + a2;
    q[idx] = qi;
    dot = p[idx] * qi;
  }
  spmv_pq_store(dot, partial, counter, pq_out);
}

__global__ void __launch_bounds__(kVecBS)
k_pcg_update_check(size_t n, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                   const double* __restrict__ q, PcgCheck ck) {
  pdl_trigger();
  pdl_wait();
  const double pq = pcg_pq<kVecBS>(ck), rz = ck.scal[S_TMP2];
  const double alpha = rz / pq;
  const bool ok = pq > 0.0 && isfinite(alpha);
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * kVecBS + threadIdx.x; i < n; i += (size_t)gridDim.x * kVecBS) {
    double ri = r[i];
    if (ok) {
      x[i] += alpha * p[i];
      ri -= alpha * q[i];
      r[i] = ri;
    }
    acc += ri * ri;
  }
  pcg_update_finish<kVecBS>(acc, ok, alpha, rz, ck);
}

// The same product in mixed precision from the blocks as (hi, lo) float pairs and the
// direction split the same way (written with p): each lane's terms in a compensated sum
// (dot2_fma), the three partial rows added in DF, q formed as a double.
__global__ void __launch_bounds__(kSpmvBS)
k_pcg_spmv_pq_df(int n, const int* __restrict__ row_ptr, const int* __restrict__ cols,
                 const float2* __restrict__ vals, const float2* __restrict__ ps, const double* __restrict__ p,
                 double* __restrict__ q, double* partial, unsigned* counter, double* pq_out) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (kSpmvBS / 32) + (threadIdx.x >> 5);
  const int r = lane % 9, k = lane / 9;
  const bool live = i < n && k < 3;
  // the first two blocks of this lane's share (blocks k and k + 3 of the row), loaded
  // before the wait; the rest two at a time into independent sums
  int e0 = 0, e1 = 0, c0 = 0, c1 = 0;
  float2 a0[9], a1[9];
  if (live) {
    e0 = row_ptr[i] + k;
    e1 = row_ptr[i + 1];
    const int last = max(e1 - 1, 0);
    const int f0 = min(e0, last), f1 = min(e0 + 3, last);
    c0 = cols[f0];
    c1 = cols[f1];
    const float2* x0 = vals + (size_t)f0 * 81 + r * 9;
    const float2* x1 = vals + (size_t)f1 * 81 + r * 9;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      a0[c] = x0[c];
      a1[c] = x1[c];
    }
  }
  pdl_trigger();
  pdl_wait();
  float sh = 0.f, sc = 0.f, th = 0.f, tc = 0.f;
  if (live && e0 < e1) {
    const float2* x0 = ps + (size_t)c0 * 9;
#pragma unroll
    for (int c = 0; c < 9; ++c) dot2_fma(sh, sc, a0[c], x0[c]);
    if (e0 + 3 < e1) {
      const float2* x1 = ps + (size_t)c1 * 9;
#pragma unroll
      for (int c = 0; c < 9; ++c) dot2_fma(th, tc, a1[c], x1[c]);
    }
    int e = e0 + 6;
    for (; e + 3 < e1; e += 6) {
      const float2* a = vals + (size_t)e * 81 + r * 9;
      const float2* b = vals + (size_t)(e + 3) * 81 + r * 9;
      const float2* xa = ps + (size_t)cols[e] * 9;
      const float2* xb = ps + (size_t)cols[e + 3] * 9;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        dot2_fma(sh, sc, a[c], xa[c]);
        dot2_fma(th, tc, b[c], xb[c]);
      }
    }
    if (e < e1) {
      const float2* a = vals + (size_t)e * 81 + r * 9;
      const float2* xa = ps + (size_t)cols[e] * 9;
#pragma unroll
      for (int c = 0; c < 9; ++c) dot2_fma(sh, sc, a[c], xa[c]);
    }
  }
  DF acc = (DF(sh, 0.f) + DF(sc, 0.f)) + (DF(th, 0.f) + DF(tc, 0.f));
  const int l1 = min(lane + 9, 31), l2 = min(lane + 18, 31);
  const DF s1(__shfl_sync(kFull, acc.h, l1), __shfl_sync(kFull, acc.l, l1));
  const DF s2(__shfl_sync(kFull, acc.h, l2), __shfl_sync(kFull, acc.l, l2));
  double dot = 0.0;
  if (i < n && lane < 9) {
    const size_t idx = (size_t)i * 9 + r;
    const double qi = to_double(acc + s1 + s2);
    q[idx] = qi;
    dot = p[idx] * qi;
  }
  spmv_pq_store(dot, partial, counter, pq_out);
}

// p = z + beta p with beta = rz / scal[S_RZ] (p = z when first), rz the sum of the rows'
// shares of r.z left by the V-cycle (every CTA adds them in the same order; CTA 0 stores
// it for the update kernel); ps (if given) the float-pair split of p
__global__ void __launch_bounds__(256)
k_pcg_direction_rz(size_t n, double* __restrict__ p, const double* __restrict__ z, double* scal, int first,
                   const double* __restrict__ part, int npart, float2* __restrict__ ps) {
  pdl_wait();
  pdl_trigger();
  double s = 0.0;
  for (int k = threadIdx.x; k < npart; k += 256) s += part[k];
  __shared__ double rz_sm;
  s = block_sum<256>(s);
  if (threadIdx.x == 0) {
    rz_sm = s;
    if (blockIdx.x == 0) scal[S_TMP2] = s;
  }
  __syncthreads();
  const double rz = rz_sm;
  const double beta = first ? 0.0 : rz / scal[S_RZ];
  const size_t i = (size_t)blockIdx.x * 256 + threadIdx.x;
  if (i < n) {
    const double pi = first ? z[i] : z[i] + beta * p[i];
    p[i] = pi;
    if (ps) {
      const float h = (float)pi;
      ps[i] = make_float2(h, (float)(pi - (double)h));
    }
  }
}

// the split of p that the mixed-precision product reads
static float2* assembled_split(ba_problem* P) {
  if (P->opt.precision != BA_MIXED) return nullptr;
  P->xsplit.ensure(sizeof(float2) * 9 * (size_t)P->n_c + 64);
  return P->xsplit.as<float2>();
}

// z = M r, r.z into scal[S_TMP2] and the direction p = z + (r.z / rz_old) p (p = z when
// first); the r.z of the previous iteration is in scal[S_RZ]
static void assembled_precond_direction(ba_problem* P, int first) {
  const size_t n = (size_t)P->n_c * 9;
  double *r = P->r.as<double>(), *z = P->z.as<double>(), *p = P->p.as<double>();
  if (P->opt.preconditioner == BA_PRECOND_MG && P->vc_ready) {
    // the V-cycle's last kernel leaves each row's share of r.z; every CTA of the direction
    // kernel adds them up in the same order
    double* part = P->rzpart.as<double>();
    {
      KernelTimer kt(P, BA_KT_VCYCLE);
      // after the first iteration the update kernel has done the cycle's first phase
      fused_vcycle(P, r, z, part, !first);
    }
    launch_k(P, k_pcg_direction_rz, cdiv((long long)n, 256), 256, 0, n, p, z, P->scal.as<double>(), first,
             (const double*)part, P->n_c, assembled_split(P));
    return;
  }
  precond_apply(P, r, z);
  dot64(P, r, z, n, S_TMP2);
  launch_k(P, k_pcg_direction, cdiv((long long)n, 256), 256, 0, n, p, z, P->scal.as<double>(), first ? -1 : S_TMP2,
           S_RZ, P->Dc.as<double>(), (double*)nullptr, assembled_split(P));
}

// CTAs of the product; up to kPqShares of them, the update kernel adds their p.q shares
// (in every CTA: a few hundred loads each) instead of the product's last CTA
constexpr int kPqShares = 1024;
static int spmv_blocks(ba_problem* P) { return cdiv(P->levels[0].n, kSpmvBS / 32); }

static void assembled_spmv(ba_problem* P) {
  const Level& L0 = P->levels[0];
  const int nb = spmv_blocks(P);
  double* pq_out = nb <= kPqShares ? nullptr : P->scal.as<double>() + S_PQ;
  KernelTimer kt(P, BA_KT_OUTER_BSR);
  if (P->opt.precision == BA_MIXED)
    launch_k(P, k_pcg_spmv_pq_df, nb, kSpmvBS, 0, L0.n, L0.row_ptr.as<int>(), L0.cols.as<int>(),
             L0.valsdf.as<float2>(), P->xsplit.as<float2>(), P->p.as<double>(), P->q.as<double>(),
             P->partial2.as<double>(), P->counter.as<unsigned>() + 1, pq_out);
  else
    launch_k(P, k_pcg_spmv_pq, nb, kSpmvBS, 0, L0.n, L0.row_ptr.as<int>(), L0.cols.as<int>(),
             L0.vals64.as<double>(), P->p.as<double>(), P->q.as<double>(), P->partial2.as<double>(),
             P->counter.as<unsigned>() + 1, pq_out);
}

// the update kernel; with the fused V-cycle it also forms the next cycle's level-0
// pre-smoothing step 0 from the new r (the cycle then starts at step 1)
static bool update_starts_vcycle(ba_problem* P) { return P->opt.preconditioner == BA_PRECOND_MG && P->vc_ready; }

static void assembled_update(ba_problem* P, double* x, int use_cond, cudaGraphConditionalHandle h) {
  const size_t n = (size_t)P->n_c * 9;
  const int nb = spmv_blocks(P);
  const PcgCheck ck{P->scal.as<double>(), P->partial.as<double>(), P->counter.as<unsigned>(), P->flags.as<int>(),
                    P->opt.max_iters, P->opt.rtol * P->opt.rtol, P->opt.stop_rule, P->opt.tau, use_cond, h,
                    P->partial2.as<double>(), nb <= kPqShares ? nb : 0};
  if (update_starts_vcycle(P)) {
    fused_update_first(P, x, P->r.as<double>(), P->p.as<double>(), P->q.as<double>(), ck);
    return;
  }
  launch_k(P, k_pcg_update_check, reduce_blocks(P, n), kVecBS, 0, n, x, P->r.as<double>(), P->p.as<double>(),
           P->q.as<double>(), ck);
}

// Signature of what the captured PCG graph takes from the host: every buffer's address and
// capacity, the hierarchy's shape, the launch geometry and the options.  The numbers a
// setup changes (operators, Jacobi blocks, Chebyshev coefficients, the coarse inverse) are
// read on the device, so the graph is captured again only when this signature changes.
static uint64_t pcg_graph_key(ba_problem* P) {
  uint64_t h = 1469598103934665603ull;   // FNV-1a
  auto val = [&](auto v) {
    const unsigned char* b = reinterpret_cast<const unsigned char*>(&v);
    for (size_t i = 0; i < sizeof(v); ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  };
  for_each_problem_buf(P, [&](DBuf& b) {
    val(b.p);
    val(b.cap);
  });
  val(P->n_levels);
  for (int l = 0; l < P->n_levels; ++l) {
    Level& L = P->levels[l];
    val(L.n);
    val(L.bs);
    val(L.nnzb);
    val(L.coarsest);
    val(L.N);
    val(L.folded);
    val(L.ap_nnzb);
    for_each_level_buf(L, [&](DBuf& b) {
      val(b.p);
      val(b.cap);
    });
  }
  val(P->n_c);
  val(P->n_p);
  val(P->n_o);
  val(P->n_sm);
  val(P->vc_ready);
  val(P->l0_explicit);
  val(P->outer_explicit);
  val(P->pc_shift);
  val(P->n_chunks);
  val(P->k3_window);
  val(P->k3_grid[0]);
  val(P->k3_grid[1]);
  val(P->k3_grid_bulk);
  val(P->k3_grid_df);
  val(P->k3_grid_rc);
  const ba_options& o = P->opt;
  val(o.lambda);
  val(o.rtol);
  val(o.max_iters);
  val(o.precision);
  val(o.preconditioner);
  val(o.damping);
  val(o.recompute_jacobian);
  val(o.max_agg);
  val(o.pre_smooth);
  val(o.post_smooth);
  val(o.lanczos_steps);
  val(o.coarse_max_nodes);
  val(o.max_levels);
  val(o.cheb_lo);
  val(o.cheb_hi);
  val(o.level0_operator);
  val(o.fused_vcycle);
  val(o.outer_product);
  val(o.stop_rule);
  val(o.tau);
  val(o.overlap_launches);
  val(o.loss);
  val(o.loss_scale);
  val(o.precond_lambda_min);
  val(o.schur_staging);
  return h;
}

// Builds [head, check] -> while(cond) { tail, head, check } as one executable graph that
// works on the problem's own vectors (x = P->x).
static void build_pcg_graph(ba_problem* P) {
  if (P->pcg_exec) {
    cudaGraphExecDestroy(P->pcg_exec);
    P->pcg_exec = nullptr;
  }
  if (!P->cap_stream) BA_CUDA(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
  cudaStream_t user = P->stream;
  const long long launches0 = P->launches;
  cudaGraph_t g = nullptr;
  try {
    const double rtol2 = P->opt.rtol * P->opt.rtol;
    double* x = P->x.as<double>();
    BA_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    BA_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    P->stream = P->cap_stream;
    const bool assembled = P->outer_explicit;
    BA_CUDA(cudaStreamBeginCaptureToGraph(P->cap_stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if (assembled) {
      assembled_spmv(P);
      assembled_update(P, x, 1, h);
    } else {
      pcg_head(P, x);
      launch_k(P, k_pcg_check, 1, 1, 0, P->scal.as<double>(), P->flags.as<int>(), P->opt.max_iters, rtol2,
                                           P->opt.stop_rule, P->opt.tau, h);
    }
    const long long head_kernels = P->launches - launches0;
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t ndeps = 0;
    cudaGraph_t cg_graph = nullptr;
    BA_CUDA(cudaStreamGetCaptureInfo(P->cap_stream, &status, nullptr, &cg_graph, &deps, &edges, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    BA_CUDA(cudaGraphAddNode(&cnode, cg_graph, deps, edges, ndeps, &cp));
    BA_CUDA(cudaStreamUpdateCaptureDependencies(P->cap_stream, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    BA_CUDA(cudaStreamEndCapture(P->cap_stream, &g));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    BA_CUDA(cudaStreamBeginCaptureToGraph(P->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const long long body0 = P->launches;
    if (assembled) {
      assembled_precond_direction(P, 0);
      assembled_spmv(P);
      assembled_update(P, x, 1, h);
    } else {
      pcg_tail(P);
      pcg_head(P, x);
      launch_k(P, k_pcg_check, 1, 1, 0, P->scal.as<double>(), P->flags.as<int>(), P->opt.max_iters, rtol2,
                                           P->opt.stop_rule, P->opt.tau, h);
    }
    BA_CUDA(cudaStreamEndCapture(P->cap_stream, &body));
    BA_CUDA(cudaGraphInstantiate(&P->pcg_exec, g, 0));
    cudaGraphDestroy(g);
    P->pcg_graph_head = head_kernels;
    P->pcg_graph_body = P->launches - body0;
    P->stream = user;
    P->launches = launches0;
    P->pcg_graph_key = pcg_graph_key(P);
  } catch (...) {
    cudaStreamCaptureStatus st;
    if (cudaStreamIsCapturing(P->cap_stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(P->cap_stream, &junk);
      if (junk) cudaGraphDestroy(junk);
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    P->stream = user;
    P->launches = launches0;
    P->pcg_exec = nullptr;
    P->graphs_ok = false;
  }
}

// PCG pieces shared by the synchronous solve and the LM step's enqueue-only path.
// pcg_begin: buffers, delta_c = 0, r = rhs, b.b into S_BB (not fetched)
static void pcg_begin(ba_problem* P, const double* rhs, double* dc) {
  const size_t n = (size_t)P->n_c * 9;
  P->r.ensure(sizeof(double) * n + 64);
  P->z.ensure(sizeof(double) * n + 64);
  P->p.ensure(sizeof(double) * n + 64);
  P->q.ensure(sizeof(double) * n + 64);
  P->x.ensure(sizeof(double) * n + 64);
  BA_CUDA(cudaMemsetAsync(dc, 0, sizeof(double) * n, P->stream));
  BA_CUDA(cudaMemcpyAsync(P->r.as<double>(), rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream));
  dot64(P, P->r.as<double>(), P->r.as<double>(), n, S_BB);
}

// the first preconditioning and direction p = z, and the loop's scalars S_ITER, S_Q, S_DQ
// set to 0
static void pcg_first_direction(ba_problem* P) {
  const size_t n = (size_t)P->n_c * 9;
  double* scal = P->scal.as<double>();
  if (P->outer_explicit) {
    // per-row-group partial sums of the fused p.q and the rows' shares of r.z, sized
    // before any graph capture
    P->partial2.ensure(sizeof(double) * ((size_t)cdiv(P->n_c, kSpmvBS / 32) + 64));
    P->rzpart.ensure(sizeof(double) * ((size_t)P->n_c + 64));
    assembled_precond_direction(P, 1);
  } else {
    precond_apply(P, P->r.as<double>(), P->z.as<double>());
    dot64(P, P->r.as<double>(), P->z.as<double>(), n, S_RZ);
    launch_k(P, k_pcg_direction, cdiv((long long)n, 256), 256, 0, n, P->p.as<double>(), P->z.as<double>(), scal,
             -1, 0, P->Dc.as<double>(), P->q.as<double>(), split_target(P));  // p = z
  }
  static_assert(S_Q == S_ITER + 1 && S_DQ == S_ITER + 2, "scalar slots");
  BA_CUDA(cudaMemsetAsync(scal + S_ITER, 0, 3 * sizeof(double), P->stream));
}

// the graph path: captured (again) when its signature changed; false when graphs are not
// used (kernel timing) or the capture failed
static bool pcg_graph_ready(ba_problem* P) {
  if (P->ktime || !P->graphs_ok) return false;
  if (!P->pcg_exec || P->pcg_graph_key != pcg_graph_key(P)) build_pcg_graph(P);
  return P->pcg_exec != nullptr;
}

// the whole loop as one graph launch, then delta_c = x
static void pcg_graph_launch(ba_problem* P, double* dc) {
  const size_t n = (size_t)P->n_c * 9;
  double* x = P->x.as<double>();
  BA_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, P->stream));
  BA_CUDA(cudaGraphLaunch(P->pcg_exec, P->stream));
  BA_CUDA(cudaMemcpyAsync(dc, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream));
}

// iterations and relative residual of a graph solve from the fetched scalars (bb > 0);
// whether it converged
static bool pcg_graph_result(ba_problem* P, double bb) {
  const int it = (int)P->h_scal[S_ITER];
  P->launches += P->pcg_graph_head + (long long)std::max(it - 1, 0) * P->pcg_graph_body;
  const double rel = std::sqrt(P->h_scal[S_RR] / bb);
  P->pcg_iters = it;
  P->pcg_rel = rel;
  BA_REQUIRE(std::isfinite(rel), BA_ERR_BREAKDOWN, "non-finite PCG residual");
  return pcg_converged(P->opt.stop_rule, (double)it, P->h_scal[S_RR], bb, P->opt.rtol * P->opt.rtol,
                       P->h_scal[S_Q], P->h_scal[S_DQ], P->opt.tau);
}

void pcg(ba_problem* P, const double* rhs, double* dc, bool check_setup) {
  const size_t n = (size_t)P->n_c * 9;
  const int g = cdiv((long long)n, 256);
  if (!check_setup) clear_flags(P);
  pcg_begin(P, rhs, dc);
  double *r = P->r.as<double>(), *z = P->z.as<double>(), *p = P->p.as<double>(), *q = P->q.as<double>();
  double* scal = P->scal.as<double>();
  if (check_setup) {
    // the setup's flags come back with b.b (one synchronisation), then start clean
    fetch_checked(P, S_BB, 1);
    clear_flags(P);
  } else {
    fetch_scalars(P, S_BB, 1);
  }
  const double bb = P->h_scal[S_BB];
  P->pcg_iters = 0;
  P->pcg_rel = 0.0;
  if (!(bb > 0.0)) {
    BA_REQUIRE(bb == 0.0, BA_ERR_INVALID_ARG, "non-finite right-hand side");
    return;
  }
  const bool assembled = P->outer_explicit;
  int s_rz = S_RZ, s_new = S_TMP2;
  pcg_first_direction(P);
  const int rg = reduce_blocks(P, n);
  const double rtol2 = P->opt.rtol * P->opt.rtol;
  double rel = 1.0;
  int it = 0;
  bool done = false;
  // graph-driven loop: no host round trip per iteration
  if (pcg_graph_ready(P)) {
    pcg_graph_launch(P, dc);
    fetch_checked(P, S_RR, S_DQ - S_RR + 1);
    if (!pcg_graph_result(P, bb))
      throw Error(BA_ERR_NOT_CONVERGED,
                  "PCG reached max_iters with relative residual " + std::to_string(P->pcg_rel));
    return;
  }
  while (it < P->opt.max_iters) {
    if (assembled) {
      assembled_spmv(P);
      assembled_update(P, dc, 0, 0);
    } else {
      outer_product(P, p, q);
      dot64(P, p, q, n, S_PQ);
      launch_k(P, k_pcg_update, rg, kVecBS, 0, n, dc, r, p, q, scal, s_rz, P->partial.as<double>(),
                                                 P->counter.as<unsigned>(), P->flags.as<int>());
    }
    ++it;
    fetch_checked(P, S_RR, S_DQ - S_RR + 1);
    rel = std::sqrt(P->h_scal[S_RR] / bb);
    BA_REQUIRE(std::isfinite(rel), BA_ERR_BREAKDOWN, "non-finite PCG residual");
    done = pcg_converged(P->opt.stop_rule, (double)it, P->h_scal[S_RR], bb, rtol2, P->h_scal[S_Q],
                         P->h_scal[S_DQ], P->opt.tau);
    if (done) break;
    if (assembled) {
      assembled_precond_direction(P, 0);
      continue;
    }
    precond_apply(P, r, z);
    dot64(P, r, z, n, s_new);
    launch_k(P, k_pcg_direction, g, 256, 0, n, p, z, scal, s_new, s_rz, P->Dc.as<double>(), q,
                                              split_target(P));
    std::swap(s_rz, s_new);
  }
  P->pcg_iters = it;
  P->pcg_rel = rel;
  if (!done)
    throw Error(BA_ERR_NOT_CONVERGED, "PCG reached max_iters with relative residual " + std::to_string(rel));
}

// ---------------------------------------------------------------------------
// LM step
// ---------------------------------------------------------------------------
__global__ void k_add(size_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = a[i] + b[i];
}

// sum_i d_i (g_i + D_i d_i) over camera vectors and the internal point SoA
__global__ void __launch_bounds__(kVecBS)
k_model_terms(int n_c9, const double* __restrict__ dc, const double* __restrict__ gc, const double* __restrict__ Dc,
              int n_p, size_t ldp, const double* __restrict__ dp, const double* __restrict__ gp,
              const double* __restrict__ Dp, double* partial, unsigned* counter, double* out) {
  double acc = 0.0;
  const size_t total = (size_t)n_c9 + 3 * (size_t)n_p;
  for (size_t i = (size_t)blockIdx.x * kVecBS + threadIdx.x; i < total; i += (size_t)gridDim.x * kVecBS) {
    if (i < (size_t)n_c9) {
      acc += dc[i] * (gc[i] + Dc[i] * dc[i]);
    } else {
      const size_t j = i - n_c9;
      const size_t k = j / n_p, ip = j - k * n_p;
      const size_t s = k * ldp + ip;
      acc += dp[s] * (gp[s] + Dp[s] * dp[s]);
    }
  }
  grid_sum_store<kVecBS>(acc, partial, counter, out);
}

void lm_step(ba_problem* P, double* cams, double* pts, const double* obs, double* lam, int* accepted,
             double* cost_out) {
  linearize(P, cams, pts, obs);
  // An unpartitioned step with the PCG graph is enqueued whole (linearisation, setups, the
  // PCG graph, back-substitution, trial cost and model decrease) and synchronises once for
  // its decision: the scalars and flags of every stage come back together, the deferred
  // setup checks are raised then (the PCG loop itself stops at once when a setup flag is
  // set), and a zero right-hand side gives delta_c = 0.  Otherwise the stages synchronise
  // where the host needs them: the flags of the linearisation and the setups with the
  // PCG's b.b, the PCG's result with its flags, the trial cost with the model decrease.  A
  // partitioned problem sums the cost over its ranks here, in the same order on every rank.
  const bool part = partitioned(P);
  double cost0 = part ? fetch_sum_checked(P, S_COST) : 0.0;
  const size_t nc = (size_t)P->n_c * 9, np = (size_t)P->n_p * 3;
  P->delta_c.ensure(sizeof(double) * nc + 64);
  double* dc = P->delta_c.as<double>();
  // A linear solve that fails (a block found not positive definite by its pivots, or a
  // PCG breakdown; near the optimum lambda becomes small enough for S to be numerically
  // singular along the gauge and the focal-length / depth directions) makes the step
  // unsuccessful, as in the Ceres trust-region loop the paper uses: x is kept and lambda
  // grows as after a rejection.
  bool solved = true, enqueued = false;
  try {
    schur_setup(P, *lam, false);
    if (P->opt.preconditioner == BA_PRECOND_MG) mg_setup(P, false);
    if (!part) {
      pcg_begin(P, P->rhs.as<double>(), dc);
      pcg_first_direction(P);
      enqueued = pcg_graph_ready(P);
      if (enqueued) {
        pcg_graph_launch(P, dc);
        // the flags as the solve left them (the trial cost below may flag a non-finite
        // residual, which only rejects the step), into pinned memory in stream order
        BA_CUDA(cudaMemcpyAsync(P->h_flags, P->flags.p, sizeof(int) * F_COUNT, cudaMemcpyDeviceToHost, P->stream));
      }
    }
    if (!enqueued) {
      try {
        pcg(P, P->rhs.as<double>(), dc, true);
      } catch (const Error& e) {
        if (e.status != BA_ERR_NOT_CONVERGED) throw;  // an inexact step is still a step
      }
    }
  } catch (const Error& e) {
    if (e.status != BA_ERR_NOT_SPD && e.status != BA_ERR_BREAKDOWN) throw;
    solved = false;
  }
  auto reject = [&](bool failed_solve) {
    P->cost = cost0;
    *lam = *lam * P->lm_nu;
    P->lm_nu *= 2.0;
    *accepted = 0;
    *cost_out = cost0;
    if (failed_solve) P->stage = 1;   // linearised; the setup must run again before a solve
    sync(P);
  };
  if (!solved) {
    if (!part) {
      fetch_scalars(P, S_COST, 1);
      cost0 = P->h_scal[S_COST];
    }
    reject(true);
    return;
  }
  P->scratch.ensure(sizeof(double) * (nc + 2 * np) + 64);
  double* cams1 = P->scratch.as<double>();
  double* dp_user = cams1 + nc;
  double* pts1 = dp_user + np;
  P->delta_p.ensure(sizeof(double) * 3 * P->ldp);
  back_substitute_to(P, dc, P->delta_p.as<double>(), dp_user);
  k_add<<<cdiv((long long)nc, 256), 256, 0, P->stream>>>(nc, cams, dc, cams1);
  launched(P);
  if (np) {
    k_add<<<cdiv((long long)np, 256), 256, 0, P->stream>>>(np, pts, dp_user, pts1);
    launched(P);
  }
  // the model decrease 1/2 (delta.g + delta.D.delta); partitioned: the point terms are this
  // rank's share (summed over the ranks), the camera terms are the same on every rank
  auto model_terms = [&](int n_c9, int n_pts) {
    k_model_terms<<<reduce_blocks(P, (size_t)n_c9 + 3 * (size_t)n_pts), kVecBS, 0, P->stream>>>(
        n_c9, dc, P->gc.as<double>(), P->Dc.as<double>(), n_pts, P->ldp, P->delta_p.as<double>(),
        P->gp.as<double>(), P->Dp.as<double>(), P->partial.as<double>(), P->counter.as<unsigned>(),
        P->scal.as<double>() + S_MODEL);
    launched(P);
  };
  double model_sum, cost1;
  if (part) {
    cost1 = cost_at(P, cams1, pts1, obs);
    model_terms(0, P->n_p);
    model_sum = fetch_sum(P, S_MODEL);
    model_terms((int)nc, 0);
    fetch_scalars(P, S_MODEL, 1);
    model_sum += P->h_scal[S_MODEL];
  } else {
    cost_at_async(P, cams1, pts1, obs);
    model_terms((int)nc, P->n_p);
    static_assert(S_COST == 0 && S_COST_NEW == S_MODEL + 1 && S_DQ > S_COST_NEW && S_BB < S_MODEL,
                  "scalar slots");
    if (enqueued) {
      // the step's one synchronisation: every scalar up to the PCG's (the flags were copied
      // after the solve)
      fetch_scalars(P, S_COST, S_DQ + 1);
      const double bb = P->h_scal[S_BB];
      BA_REQUIRE(bb >= 0.0 && std::isfinite(bb), BA_ERR_INVALID_ARG, "non-finite right-hand side");
      if (bb == 0.0) P->h_flags[F_BREAKDOWN] = 0;   // r = 0: delta_c = 0, no iteration
      try {
        raise_flags(P);
        if (bb > 0.0) {
          pcg_graph_result(P, bb);   // not converged: an inexact step is still a step
        } else {
          P->pcg_iters = 0;
          P->pcg_rel = 0.0;
        }
      } catch (const Error& e) {
        if (e.status != BA_ERR_NOT_SPD && e.status != BA_ERR_BREAKDOWN) throw;
        solved = false;
      }
    } else {
      fetch_scalars(P, S_COST, S_COST_NEW + 1);
    }
    cost0 = P->h_scal[S_COST];
    model_sum = P->h_scal[S_MODEL];
    cost1 = P->h_scal[S_COST_NEW];
    if (!solved) {
      reject(true);
      return;
    }
  }
  P->cost = cost0;
  const double model = 0.5 * model_sum;
  const double rho = model > 0.0 ? (cost0 - cost1) / model : -INFINITY;
  if (rho > 1e-3 && std::isfinite(cost1)) {
    BA_CUDA(cudaMemcpyAsync(cams, cams1, sizeof(double) * nc, cudaMemcpyDeviceToDevice, P->stream));
    if (np) BA_CUDA(cudaMemcpyAsync(pts, pts1, sizeof(double) * np, cudaMemcpyDeviceToDevice, P->stream));
    const double t = 2.0 * rho - 1.0;
    *lam = *lam * std::max(1.0 / 3.0, 1.0 - t * t * t);
    P->lm_nu = 2.0;
    *accepted = 1;
    *cost_out = cost1;
    sync(P);
  } else {
    reject(false);
  }
}

}  // namespace ba
