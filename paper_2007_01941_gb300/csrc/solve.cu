// V-cycle (Algorithm 1) with the Chebyshev / point-block-Jacobi smoother of
// Section 3.4, PCG on S (Section 3.6) and one Levenberg-Marquardt step (Section 2.1).
#include <algorithm>
#include <cmath>

#include "ba_internal.h"
#include "device_util.cuh"

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

void level_matvec(ba_problem* P, int l, const void* x, void* y) {
  Level& L = P->levels[l];
  const bool fp32 = level_fp32(P);
  if (l == 0) {
    if (fp32) matvec32(P, (const float*)x, (float*)y);
    else matvec64(P, (const double*)x, (double*)y);
    return;
  }
  const int g = cdiv((long long)L.n * 16, 256);
  if (fp32)
    k_bsr16_spmv<float><<<g, 256, 0, P->stream>>>(L.n, L.row_ptr.as<int>(), L.cols.as<int>(), L.vals32.as<float>(),
                                                  (const float*)x, (float*)y);
  else
    k_bsr16_spmv<double><<<g, 256, 0, P->stream>>>(L.n, L.row_ptr.as<int>(), L.cols.as<int>(),
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

// step 0: r = b - q (q may be null: x = 0), d = D^-1 r / theta, x = x + d
template <typename T>
__global__ void k_cheb_first(int n, int bs, const T* __restrict__ Dinv, const T* __restrict__ b,
                             const T* __restrict__ q, T* __restrict__ r, T* __restrict__ d, T* __restrict__ x,
                             int x_zero, const double* __restrict__ cheb) {
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
}

// step k >= 1: r = r - q; d = rho_k rho_{k-1} d + (2 rho_k / delta) D^-1 r; x = x + d
// (r is updated by a separate pass first so every thread sees the new r)
template <typename T>
__global__ void k_sub(size_t n, T* __restrict__ r, const T* __restrict__ q) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] -= q[i];
}

template <typename T>
__global__ void k_cheb_step(int n, int bs, const T* __restrict__ Dinv, const T* __restrict__ r,
                            T* __restrict__ d, T* __restrict__ x, const double* __restrict__ cheb, int k) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * bs) return;
  const size_t i = idx / bs;
  const int u = (int)(idx - i * bs);
  const T* Di = Dinv + (i * bs + u) * bs;
  const T* ri = r + i * bs;
  T acc = T(0);
  for (int v = 0; v < bs; ++v) acc += Di[v] * ri[v];
  const double rk = cheb_rho(cheb, k), rk1 = cheb_rho(cheb, k - 1);
  const T dn = (T)(rk * rk1) * d[idx] + (T)(2.0 * rk / cheb[1]) * acc;
  d[idx] = dn;
  x[idx] += dn;
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

// x_i += Q_i xc_{agg(i)}   (prolongation)
template <typename T>
__global__ void k_prolong(int n, int bs, const int* __restrict__ agg, const T* __restrict__ Q,
                          const T* __restrict__ xc, T* __restrict__ x) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * bs) return;
  const size_t i = idx / bs;
  const int u = (int)(idx - i * bs);
  const T* Qi = Q + (i * bs + u) * 16;
  const T* xa = xc + (size_t)agg[i] * 16;
  T acc = T(0);
#pragma unroll
  for (int s = 0; s < 16; ++s) acc += Qi[s] * xa[s];
  x[idx] += acc;
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

// smooth(x, b) with `steps` Chebyshev steps; x_zero: x = 0 on entry.  On exit r holds
// the residual b - A x_{steps-1} and d the last update (so b - A x = r - A d).
template <typename T>
static void smooth(ba_problem* P, int l, T* x, const T* b, T* r, T* d, T* q, int steps, bool x_zero) {
  Level& L = P->levels[l];
  const size_t n = (size_t)L.n * L.bs;
  const int g = cdiv((long long)n, 256);
  const double* cheb = L.cheb.as<double>();
  if (!x_zero) level_matvec(P, l, x, q);
  k_cheb_first<T><<<g, 256, 0, P->stream>>>(L.n, L.bs, dinv<T>(L), b, x_zero ? nullptr : q, r, d, x, x_zero, cheb);
  launched(P);
  for (int k = 1; k < steps; ++k) {
    level_matvec(P, l, d, q);
    k_sub<T><<<g, 256, 0, P->stream>>>(n, r, q);
    launched(P);
    k_cheb_step<T><<<g, 256, 0, P->stream>>>(L.n, L.bs, dinv<T>(L), r, d, x, cheb, k);
    launched(P);
  }
}

// x = mgcycle(l, 0, b)
template <typename T>
static void vcycle(ba_problem* P, int l, const T* b, T* x) {
  Level& L = P->levels[l];
  if (L.coarsest) {
    const int N = L.n * L.bs;
    k_dense_apply<T><<<cdiv((long long)N * 32, 256), 256, 0, P->stream>>>(N, L.N, L.Ainv.as<double>(), b, x);
    launched(P);
    return;
  }
  T* r = L.vr.as<T>();
  T* d = L.vd.as<T>();
  T* q = L.vq.as<T>();
  const int pre = std::max(1, P->opt.pre_smooth), post = std::max(1, P->opt.post_smooth);
  smooth<T>(P, l, x, b, r, d, q, pre, true);                   // pre-smoothing
  level_matvec(P, l, d, q);                                     // residual b - A x = r - A d
  Level& C = P->levels[l + 1];
  T* rc = C.vb.as<T>();
  T* xc = C.vx.as<T>();
  k_restrict<T><<<cdiv((long long)C.n * 16, 256), 256, 0, P->stream>>>(C.n, L.bs, L.agg_ptr.as<int>(),
                                                                     L.agg_mem.as<int>(), qblk<T>(L), r, q, rc);
  launched(P);                                                  // restriction
  vcycle<T>(P, l + 1, rc, xc);                                  // coarse-level solve
  k_prolong<T><<<cdiv((long long)L.n * L.bs, 256), 256, 0, P->stream>>>(L.n, L.bs, L.agg.as<int>(), qblk<T>(L),
                                                                      xc, x);
  launched(P);                                                  // prolongation
  smooth<T>(P, l, x, b, r, d, q, post, false);                  // post-smoothing
}

// ---------------------------------------------------------------------------
// preconditioner application on FP64 camera vectors
// ---------------------------------------------------------------------------
__global__ void k_to_float(size_t n, const double* __restrict__ a, float* __restrict__ b) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_to_double(size_t n, const float* __restrict__ a, double* __restrict__ b) {
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
  Level& L0 = P->levels[0];
  if (level_fp32(P)) {
    float* b = L0.vb.as<float>();
    float* x = L0.vx.as<float>();
    k_to_float<<<g, 256, 0, P->stream>>>(n, r, b);
    launched(P);
    vcycle<float>(P, 0, b, x);
    k_to_double<<<g, 256, 0, P->stream>>>(n, x, z);
    launched(P);
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
  if (!ok && blockIdx.x == 0 && threadIdx.x == 0) flags[F_BREAKDOWN] = 1;
  grid_sum_store<kVecBS>(acc, partial, counter, scal + S_RR);
}

// p = z + beta p, beta = scal[rz_new] / scal[rz_old]
__global__ void k_pcg_direction(size_t n, double* __restrict__ p, const double* __restrict__ z,
                                const double* __restrict__ scal, int s_new, int s_old) {
  const double beta = scal[s_new] / scal[s_old];
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = z[i] + beta * p[i];
}

void pcg(ba_problem* P, const double* rhs, double* dc) {
  const size_t n = (size_t)P->n_c * 9;
  const int g = cdiv((long long)n, 256);
  P->r.ensure(sizeof(double) * n + 64);
  P->z.ensure(sizeof(double) * n + 64);
  P->p.ensure(sizeof(double) * n + 64);
  P->q.ensure(sizeof(double) * n + 64);
  double *r = P->r.as<double>(), *z = P->z.as<double>(), *p = P->p.as<double>(), *q = P->q.as<double>();
  double* scal = P->scal.as<double>();
  clear_flags(P);
  BA_CUDA(cudaMemsetAsync(dc, 0, sizeof(double) * n, P->stream));
  BA_CUDA(cudaMemcpyAsync(r, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream));
  dot64(P, r, r, n, S_BB);
  fetch_scalars(P, S_BB, 1);
  const double bb = P->h_scal[S_BB];
  P->pcg_iters = 0;
  P->pcg_rel = 0.0;
  if (!(bb > 0.0)) {
    BA_REQUIRE(bb == 0.0, BA_ERR_INVALID_ARG, "non-finite right-hand side");
    return;
  }
  precond_apply(P, r, z);
  int s_rz = S_RZ, s_new = S_TMP2;
  dot64(P, r, z, n, s_rz);
  BA_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream));
  const int rg = reduce_blocks(P, n);
  double rel = 1.0;
  int it = 0;
  while (it < P->opt.max_iters) {
    matvec64(P, p, q);
    dot64(P, p, q, n, S_PQ);
    k_pcg_update<<<rg, kVecBS, 0, P->stream>>>(n, dc, r, p, q, scal, s_rz, P->partial.as<double>(),
                                               P->counter.as<unsigned>(), P->flags.as<int>());
    launched(P);
    ++it;
    fetch_scalars(P, S_RR, 1);
    rel = std::sqrt(P->h_scal[S_RR] / bb);
    check_flags(P);
    BA_REQUIRE(std::isfinite(rel), BA_ERR_BREAKDOWN, "non-finite PCG residual");
    if (rel <= P->opt.rtol) break;
    precond_apply(P, r, z);
    dot64(P, r, z, n, s_new);
    k_pcg_direction<<<g, 256, 0, P->stream>>>(n, p, z, scal, s_new, s_rz);
    launched(P);
    std::swap(s_rz, s_new);
  }
  P->pcg_iters = it;
  P->pcg_rel = rel;
  if (rel > P->opt.rtol)
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
  fetch_scalars(P, S_COST, 1);
  check_flags(P);
  const double cost0 = P->h_scal[S_COST];
  P->cost = cost0;
  schur_setup(P, *lam);
  if (P->opt.preconditioner == BA_PRECOND_MG) mg_setup(P);
  const size_t nc = (size_t)P->n_c * 9, np = (size_t)P->n_p * 3;
  P->delta_c.ensure(sizeof(double) * nc + 64);
  try {
    pcg(P, P->rhs.as<double>(), P->delta_c.as<double>());
  } catch (const Error& e) {
    if (e.status != BA_ERR_NOT_CONVERGED) throw;  // an inexact step is still a step
  }
  P->scratch.ensure(sizeof(double) * (nc + 2 * np) + 64);
  double* cams1 = P->scratch.as<double>();
  double* dp_user = cams1 + nc;
  double* pts1 = dp_user + np;
  P->delta_p.ensure(sizeof(double) * 3 * P->ldp);
  back_substitute_to(P, P->delta_c.as<double>(), P->delta_p.as<double>(), dp_user);
  k_add<<<cdiv((long long)nc, 256), 256, 0, P->stream>>>(nc, cams, P->delta_c.as<double>(), cams1);
  launched(P);
  if (np) {
    k_add<<<cdiv((long long)np, 256), 256, 0, P->stream>>>(np, pts, dp_user, pts1);
    launched(P);
  }
  const double cost1 = cost_at(P, cams1, pts1, obs);
  k_model_terms<<<reduce_blocks(P, nc + np), kVecBS, 0, P->stream>>>(
      (int)nc, P->delta_c.as<double>(), P->gc.as<double>(), P->Dc.as<double>(), P->n_p, P->ldp,
      P->delta_p.as<double>(), P->gp.as<double>(), P->Dp.as<double>(), P->partial.as<double>(),
      P->counter.as<unsigned>(), P->scal.as<double>() + S_MODEL);
  launched(P);
  fetch_scalars(P, S_MODEL, 1);
  const double model = 0.5 * P->h_scal[S_MODEL];
  const double rho = model > 0.0 ? (cost0 - cost1) / model : -INFINITY;
  if (rho > 1e-3 && std::isfinite(cost1)) {
    BA_CUDA(cudaMemcpyAsync(cams, cams1, sizeof(double) * nc, cudaMemcpyDeviceToDevice, P->stream));
    if (np) BA_CUDA(cudaMemcpyAsync(pts, pts1, sizeof(double) * np, cudaMemcpyDeviceToDevice, P->stream));
    const double t = 2.0 * rho - 1.0;
    *lam = *lam * std::max(1.0 / 3.0, 1.0 - t * t * t);
    P->lm_nu = 2.0;
    *accepted = 1;
    *cost_out = cost1;
  } else {
    *lam = *lam * P->lm_nu;
    P->lm_nu *= 2.0;
    *accepted = 0;
    *cost_out = cost0;
  }
  sync(P);
}

}  // namespace ba
