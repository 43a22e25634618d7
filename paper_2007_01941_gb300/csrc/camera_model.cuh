// The 9-parameter camera model of the linearisation (Section 2.1, Eq. 1-2; BAL
// convention): residual and Jacobian blocks of one observation, written once over the
// arithmetic type (double, or DF for paired FP32), and the robust weight of Section 5.
// Shared by the linearisation kernels and by the implicit Schur product's recompute mode.
//
// P = R(r) X + t, p = -P_xy / P_z, d = 1 + k1 |p|^2 + k2 |p|^4, f_o = f d p - obs_o.
// Per camera, R(r) and the left Jacobian of SO(3) J_l(r) are precomputed (camx rows);
// per observation d(RX)/dr = -[R X]_x J_l(r) and d(RX)/dX = R.  For th^2 < 1e-16 the
// rotation is taken to first order: R X = X + r x X, d(RX)/dr = -[X]_x,
// d(RX)/dX = I + [r]_x.
#ifndef BA_CAMERA_MODEL_CUH_
#define BA_CAMERA_MODEL_CUH_

namespace ba {

constexpr int kCamx = 24;   // doubles of per-camera rotation data: R (9), J_l (9), first-order flag

template <typename R>
struct CamObsT {
  R res[2];
  R F[18];
  R E[6];
};
using CamObs = CamObsT<double>;

// residual and (JAC) Jacobian of one observation; cam: the 9 parameters, cx: R(r) (9),
// J_l(r) (9), small: first-order rotation; R is double or DF (paired FP32)
template <bool JAC, typename R>
__device__ __forceinline__ void project_obs_t(const R cam[9], const R cx[18], bool small, const R X[3],
                                              const R ob[2], CamObsT<R>& out) {
  const R one = R(1.0), two = R(2.0);
  R RX[3];
  if (small) {
    const R r0 = cam[0], r1 = cam[1], r2 = cam[2];
    RX[0] = X[0] + (r1 * X[2] - r2 * X[1]);
    RX[1] = X[1] + (r2 * X[0] - r0 * X[2]);
    RX[2] = X[2] + (r0 * X[1] - r1 * X[0]);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) RX[i] = cx[3 * i] * X[0] + cx[3 * i + 1] * X[1] + cx[3 * i + 2] * X[2];
  }
  const R P0 = RX[0] + cam[3], P1 = RX[1] + cam[4], P2 = RX[2] + cam[5];
  const R iz = one / P2;
  const R px = -P0 * iz, py = -P1 * iz;
  const R f = cam[6], k1 = cam[7], k2 = cam[8];
  const R r2 = px * px + py * py;
  const R d = one + k1 * r2 + k2 * r2 * r2;
  out.res[0] = f * d * px - ob[0];
  out.res[1] = f * d * py - ob[1];
  if (!JAC) return;
  // d pi / d p = f (d I + p (grad d)^T),  grad d = 2 (k1 + 2 k2 r2) p
  const R gd = two * (k1 + two * k2 * r2);
  const R A00 = f * (d + px * gd * px), A01 = f * (px * gd * py);
  const R A10 = f * (py * gd * px), A11 = f * (d + py * gd * py);
  // d p / d P = [[-iz, 0, P0 iz^2], [0, -iz, P1 iz^2]]
  const R iz2 = iz * iz;
  R G[6];  // d pi / d P (2x3)
  G[0] = -A00 * iz;
  G[1] = -A01 * iz;
  G[2] = (A00 * P0 + A01 * P1) * iz2;
  G[3] = -A10 * iz;
  G[4] = -A11 * iz;
  G[5] = (A10 * P0 + A11 * P1) * iz2;
  // d P / d r
  R Dr[9];
  const R zero = R(0.0);
  if (small) {
    // -[X]_x
    Dr[0] = zero;   Dr[1] = X[2];   Dr[2] = -X[1];
    Dr[3] = -X[2];  Dr[4] = zero;   Dr[5] = X[0];
    Dr[6] = X[1];   Dr[7] = -X[0];  Dr[8] = zero;
  } else {
    // -[RX]_x J_l : column j = -(RX x J_l[:, j])
    const R* J = cx + 9;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const R m0 = J[j], m1 = J[3 + j], m2 = J[6 + j];
      Dr[0 + j] = -(RX[1] * m2 - RX[2] * m1);
      Dr[3 + j] = -(RX[2] * m0 - RX[0] * m2);
      Dr[6 + j] = -(RX[0] * m1 - RX[1] * m0);
    }
  }
  // d P / d X
  R Dx[9];
  if (small) {
    const R r0 = cam[0], r1 = cam[1], r2c = cam[2];
    Dx[0] = one;  Dx[1] = -r2c; Dx[2] = r1;
    Dx[3] = r2c;  Dx[4] = one;  Dx[5] = -r0;
    Dx[6] = -r1;  Dx[7] = r0;   Dx[8] = one;
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) Dx[i] = cx[i];
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      out.F[9 * i + j] = G[3 * i] * Dr[j] + G[3 * i + 1] * Dr[3 + j] + G[3 * i + 2] * Dr[6 + j];
      out.F[9 * i + 3 + j] = G[3 * i + j];
      out.E[3 * i + j] = G[3 * i] * Dx[j] + G[3 * i + 1] * Dx[3 + j] + G[3 * i + 2] * Dx[6 + j];
    }
  }
  out.F[6] = d * px;
  out.F[15] = d * py;
  out.F[7] = f * r2 * px;
  out.F[16] = f * r2 * py;
  out.F[8] = f * r2 * r2 * px;
  out.F[17] = f * r2 * r2 * py;
}

// Robust loss of Section 5 on s = |f_o|^2: returns w = sqrt(rho'(s)) and sets half_rho =
// rho(s) / 2; ha > 0 selects Huber with scale ha (rho = s inside ha^2, 2 ha sqrt(s) - ha^2
// beyond, so w = (ha^2 / s)^(1/4) there), ha <= 0 the squared loss (w = 1)
__device__ __forceinline__ double robust_weight(double s, double ha, double& half_rho) {
  if (ha > 0.0 && s > ha * ha) {
    const double rs = sqrt(s);
    half_rho = ha * rs - 0.5 * ha * ha;
    return sqrt(ha / rs);
  }
  half_rho = 0.5 * s;
  return 1.0;
}

}  // namespace ba

#endif
