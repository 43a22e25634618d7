// K14: adjoint of one LM step (gradient of a loss of delta through the linear solve).
//
// delta solves H delta = g with H = J^T J + D, g = -J^T f (Section 2.1).  For a
// cotangent vbar = dL/ddelta, with mu = H^-1 vbar (obtained through the Schur
// complement and the same multigrid hierarchy, H being symmetric):
//   dL/dobs_o   = J_o mu_o                                  (f_o = pi - obs_o)
//   dL/dtheta_o = -d/dtheta [ (J_o mu)^T f_o + (J_o mu)^T (J_o delta)
//                             + lam sum_k m_k mu_k delta_k |J_o[:,k]|^2 ]
// with mu, delta held fixed and m_k = 1 where D_kk = lam diag(J^T J)_kk is above its
// floor (Marquardt damping).  With u = J mu, w = J delta, h = f + w and the 2 x 12
// matrix a[:,k] = mu_k h + delta_k u + 2 lam m_k mu_k delta_k J[:,k], the bracket's
// gradient is  H_0 a[0,:] + H_1 a[1,:] + J^T u,  where H_i is the Hessian of f_i in
// the observation's 12 parameters.  The two Hessian-vector products come from one
// forward-mode pass over the Jacobian with two tangent directions (a[0,:], a[1,:]).
// F and E are recomputed in that pass rather than read back.
#include <cmath>

#include "ba_internal.h"
#include "device_util.cuh"

namespace ba {

void reduced_rhs(ba_problem* P, const double* vc, const double* vp_user, double* out);
void back_substitute_general(ba_problem* P, const double* vp_user, const double* dc, double* out_int,
                             double* out_user);

struct Dual2 {
  double v, d0, d1;
  __device__ Dual2() : v(0), d0(0), d1(0) {}
  __device__ Dual2(double a) : v(a), d0(0), d1(0) {}
  __device__ Dual2(double a, double b, double c) : v(a), d0(b), d1(c) {}
};
__device__ __forceinline__ Dual2 operator+(Dual2 a, Dual2 b) { return {a.v + b.v, a.d0 + b.d0, a.d1 + b.d1}; }
__device__ __forceinline__ Dual2 operator-(Dual2 a, Dual2 b) { return {a.v - b.v, a.d0 - b.d0, a.d1 - b.d1}; }
__device__ __forceinline__ Dual2 operator-(Dual2 a) { return {-a.v, -a.d0, -a.d1}; }
__device__ __forceinline__ Dual2 operator*(Dual2 a, Dual2 b) {
  return {a.v * b.v, a.d0 * b.v + a.v * b.d0, a.d1 * b.v + a.v * b.d1};
}
__device__ __forceinline__ Dual2 operator/(Dual2 a, Dual2 b) {
  const double iv = 1.0 / b.v;
  const double q = a.v * iv;
  return {q, (a.d0 - q * b.d0) * iv, (a.d1 - q * b.d1) * iv};
}
__device__ __forceinline__ Dual2 dsqrt(Dual2 a) {
  const double s = sqrt(a.v);
  const double k = 0.5 / s;
  return {s, a.d0 * k, a.d1 * k};
}
__device__ __forceinline__ void dsincos(Dual2 a, Dual2* s, Dual2* c) {
  double sv, cv;
  sincos(a.v, &sv, &cv);
  *s = Dual2(sv, cv * a.d0, cv * a.d1);
  *c = Dual2(cv, -sv * a.d0, -sv * a.d1);
}
__device__ __forceinline__ double val(const Dual2& a) { return a.v; }
__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ void dsincos(double a, double* s, double* c) { sincos(a, s, c); }

// Residual and Jacobian of one observation in the same formulation as K1, with the
// rotation data computed inline (generic scalar type S).
template <typename S>
__device__ void obs_jacobian(const S cam[9], const S X[3], const double ob[2], S res[2], S F[18], S E[6]) {
  const S r0 = cam[0], r1 = cam[1], r2 = cam[2];
  const S th2 = r0 * r0 + r1 * r1 + r2 * r2;
  const bool small = val(th2) < 1e-16;
  S RX[3], Dr[9], Dx[9];
  if (small) {
    RX[0] = X[0] + (r1 * X[2] - r2 * X[1]);
    RX[1] = X[1] + (r2 * X[0] - r0 * X[2]);
    RX[2] = X[2] + (r0 * X[1] - r1 * X[0]);
    const S z(0.0), one(1.0);
    Dr[0] = z;     Dr[1] = X[2];  Dr[2] = -X[1];
    Dr[3] = -X[2]; Dr[4] = z;     Dr[5] = X[0];
    Dr[6] = X[1];  Dr[7] = -X[0]; Dr[8] = z;
    Dx[0] = one;   Dx[1] = -r2;   Dx[2] = r1;
    Dx[3] = r2;    Dx[4] = one;   Dx[5] = -r0;
    Dx[6] = -r1;   Dx[7] = r0;    Dx[8] = one;
  } else {
    const S th = dsqrt(th2);
    S s, co;
    dsincos(th, &s, &co);
    const S a = (S(1.0) - co) / th2;
    const S b = (th - s) / (th2 * th);
    const S al = s / th;
    const S Km[9] = {S(0.0), -r2, r1, r2, S(0.0), -r0, -r1, r0, S(0.0)};
    const S rv[3] = {r0, r1, r2};
    S R[9], Jl[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const S K2 = rv[i] * rv[j] - (i == j ? th2 : S(0.0));
        const S I = S(i == j ? 1.0 : 0.0);
        R[3 * i + j] = I + al * Km[3 * i + j] + a * K2;
        Jl[3 * i + j] = I + a * Km[3 * i + j] + b * K2;
      }
    for (int i = 0; i < 3; ++i) RX[i] = R[3 * i] * X[0] + R[3 * i + 1] * X[1] + R[3 * i + 2] * X[2];
    for (int j = 0; j < 3; ++j) {
      const S m0 = Jl[j], m1 = Jl[3 + j], m2 = Jl[6 + j];
      Dr[0 + j] = -(RX[1] * m2 - RX[2] * m1);
      Dr[3 + j] = -(RX[2] * m0 - RX[0] * m2);
      Dr[6 + j] = -(RX[0] * m1 - RX[1] * m0);
    }
    for (int i = 0; i < 9; ++i) Dx[i] = R[i];
  }
  const S P0 = RX[0] + cam[3], P1 = RX[1] + cam[4], P2 = RX[2] + cam[5];
  const S iz = S(1.0) / P2;
  const S px = -P0 * iz, py = -P1 * iz;
  const S f = cam[6], k1 = cam[7], k2 = cam[8];
  const S rr = px * px + py * py;
  const S d = S(1.0) + k1 * rr + k2 * rr * rr;
  res[0] = f * d * px - S(ob[0]);
  res[1] = f * d * py - S(ob[1]);
  const S gd = S(2.0) * (k1 + S(2.0) * k2 * rr);
  const S A00 = f * (d + px * gd * px), A01 = f * (px * gd * py);
  const S A10 = f * (py * gd * px), A11 = f * (d + py * gd * py);
  const S iz2 = iz * iz;
  S G[6];
  G[0] = -A00 * iz;
  G[1] = -A01 * iz;
  G[2] = (A00 * P0 + A01 * P1) * iz2;
  G[3] = -A10 * iz;
  G[4] = -A11 * iz;
  G[5] = (A10 * P0 + A11 * P1) * iz2;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      F[9 * i + j] = G[3 * i] * Dr[j] + G[3 * i + 1] * Dr[3 + j] + G[3 * i + 2] * Dr[6 + j];
      F[9 * i + 3 + j] = G[3 * i + j];
      E[3 * i + j] = G[3 * i] * Dx[j] + G[3 * i + 1] * Dx[3 + j] + G[3 * i + 2] * Dx[6 + j];
    }
  F[6] = d * px;
  F[15] = d * py;
  F[7] = f * rr * px;
  F[16] = f * rr * py;
  F[8] = f * rr * rr * px;
  F[17] = f * rr * rr * py;
}

__global__ void k_adjoint_obs(int n_o, const double* __restrict__ cams, const double* __restrict__ pts,
                              const double* __restrict__ obs, const int* __restrict__ obs_cam,
                              const int* __restrict__ obs_pt, const int* __restrict__ obs_ptu,
                              const int* __restrict__ obs_user, const double* __restrict__ mu_c,
                              const double* __restrict__ mu_p, const double* __restrict__ dl_c,
                              const double* __restrict__ dl_p, size_t ldp, const double* __restrict__ Dc,
                              const double* __restrict__ Dp, double lam, int marquardt,
                              double* __restrict__ g_obs, double* __restrict__ g_cam, double* __restrict__ g_pt) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_o) return;
  const int c = obs_cam[o], ip = obs_pt[o], pu = obs_ptu[o], ou = obs_user[o];
  double th[12], mu[12], dl[12], mk[12];
  for (int k = 0; k < 9; ++k) {
    th[k] = cams[9 * c + k];
    mu[k] = mu_c[9 * c + k];
    dl[k] = dl_c[9 * c + k];
    mk[k] = (marquardt && Dc[9 * c + k] > lam * 1e-6) ? 1.0 : 0.0;
  }
  for (int k = 0; k < 3; ++k) {
    th[9 + k] = pts[3 * pu + k];
    mu[9 + k] = mu_p[k * ldp + ip];
    dl[9 + k] = dl_p[k * ldp + ip];
    mk[9 + k] = (marquardt && Dp[k * ldp + ip] > lam * 1e-6) ? 1.0 : 0.0;
  }
  const double ob[2] = {obs[2 * ou], obs[2 * ou + 1]};
  // plain pass: J (2 x 12) and f
  double res[2], F[18], E[6];
  obs_jacobian<double>(th, th + 9, ob, res, F, E);
  double J[2][12];
  for (int i = 0; i < 2; ++i) {
    for (int k = 0; k < 9; ++k) J[i][k] = F[9 * i + k];
    for (int k = 0; k < 3; ++k) J[i][9 + k] = E[3 * i + k];
  }
  double u[2] = {0, 0}, w[2] = {0, 0};
  for (int i = 0; i < 2; ++i)
    for (int k = 0; k < 12; ++k) {
      u[i] += J[i][k] * mu[k];
      w[i] += J[i][k] * dl[k];
    }
  const double h[2] = {res[0] + w[0], res[1] + w[1]};
  double a[2][12];
  for (int k = 0; k < 12; ++k)
    for (int i = 0; i < 2; ++i)
      a[i][k] = mu[k] * h[i] + dl[k] * u[i] + 2.0 * lam * mk[k] * mu[k] * dl[k] * J[i][k];
  // dual pass with tangents a[0,:] and a[1,:]
  Dual2 tc[9], tx[3];
  for (int k = 0; k < 9; ++k) tc[k] = Dual2(th[k], a[0][k], a[1][k]);
  for (int k = 0; k < 3; ++k) tx[k] = Dual2(th[9 + k], a[0][9 + k], a[1][9 + k]);
  Dual2 dres[2], dF[18], dE[6];
  obs_jacobian<Dual2>(tc, tx, ob, dres, dF, dE);
  double grad[12];
  for (int k = 0; k < 9; ++k) grad[k] = dF[k].d0 + dF[9 + k].d1 + J[0][k] * u[0] + J[1][k] * u[1];
  for (int k = 0; k < 3; ++k)
    grad[9 + k] = dE[k].d0 + dE[3 + k].d1 + J[0][9 + k] * u[0] + J[1][9 + k] * u[1];
  if (g_obs) {
    g_obs[2 * ou] = u[0];
    g_obs[2 * ou + 1] = u[1];
  }
  if (g_cam)
    for (int k = 0; k < 9; ++k) atomicAdd(g_cam + 9 * c + k, -grad[k]);
  if (g_pt)
    for (int k = 0; k < 3; ++k) atomicAdd(g_pt + 3 * pu + k, -grad[9 + k]);
}

void adjoint(ba_problem* P, const double* dL_ddelta, double* dL_dobs, double* dL_dcams, double* dL_dpts) {
  const size_t nc = (size_t)P->n_c * 9, np = (size_t)P->n_p * 3;
  // mu_c = S^-1 (vbar_c - F^T E C^-1 vbar_p)
  P->scratch.ensure(sizeof(double) * (2 * nc + 3 * P->ldp) + 64);
  double* rhs = P->scratch.as<double>();
  double* mu_c = rhs + nc;
  double* mu_p = mu_c + nc;
  reduced_rhs(P, dL_ddelta, dL_ddelta + nc, rhs);
  // the reduced RHS uses scratch2; PCG does not touch scratch
  pcg(P, rhs, mu_c);
  back_substitute_general(P, dL_ddelta + nc, mu_c, mu_p, nullptr);
  if (dL_dcams) BA_CUDA(cudaMemsetAsync(dL_dcams, 0, sizeof(double) * nc, P->stream));
  if (dL_dpts && np) BA_CUDA(cudaMemsetAsync(dL_dpts, 0, sizeof(double) * np, P->stream));
  if (P->n_o) {
    k_adjoint_obs<<<cdiv(P->n_o, 128), 128, 0, P->stream>>>(
        P->n_o, P->cams_lin.as<double>(), P->pts_lin.as<double>(), P->obs_lin.as<double>(), P->obs_cam.as<int>(),
        P->obs_pt.as<int>(), P->obs_ptu.as<int>(), P->obs_user.as<int>(), mu_c, mu_p, P->delta_c.as<double>(),
        P->delta_p.as<double>(), P->ldp, P->Dc.as<double>(), P->Dp.as<double>(), P->lambda,
        P->opt.damping == BA_DAMP_MARQUARDT, dL_dobs, dL_dcams, dL_dpts);
    launched(P);
  }
  sync(P);
}

}  // namespace ba
