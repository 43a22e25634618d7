// K1: residuals and Jacobian blocks of the 9-parameter camera (Section 2.1, Eq. 1-2).
//
// Camera model (BAL convention, see ba.h): P = R(r) X + t, p = -P_xy / P_z,
// d = 1 + k1 |p|^2 + k2 |p|^4, f_o = f d p - obs_o.
//
// Formulation used on the GPU: per camera, R(r) and the left Jacobian of SO(3)
// J_l(r) = I + ((1-cos th)/th^2) [r]_x + ((th - sin th)/th^3) [r]_x^2 are computed
// once; per observation d(RX)/dr = -[R X]_x J_l(r) and d(RX)/dX = R.  For
// th^2 < 1e-16 the rotation is taken to first order: R X = X + r x X with
// d(RX)/dr = -[X]_x and d(RX)/dX = I + [r]_x.
#include "ba_internal.h"
#include "device_util.cuh"
#include "dfloat.cuh"
#include "camera_model.cuh"

namespace ba {

constexpr int kLinBS = 256;

// per camera: R (9), J_l (9), first-order flag (1) in camx; with camdf also the same
// values and the 9 parameters split into float pairs ([n_c][kCamdf]: 0..17 R and J_l,
// 18 the flag, 19..27 the parameters), for the paired-FP32 linearisation
constexpr int kCamdf = 28;

__device__ __forceinline__ void camdf_write(float2* __restrict__ camdf, int c, const double* o, const double* cam) {
  if (!camdf) return;
  float2* d = camdf + (size_t)kCamdf * c;
  for (int i = 0; i < 19; ++i) {
    float h, l;
    split_double(o[i], h, l);
    d[i] = make_float2(h, l);
  }
  for (int i = 0; i < 9; ++i) {
    float h, l;
    split_double(cam[i], h, l);
    d[19 + i] = make_float2(h, l);
  }
}

__global__ void k_camera_rotation(const double* __restrict__ cams, int n_c, double* __restrict__ camx,
                                  float2* __restrict__ camdf) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_c) return;
  const double r0 = cams[9 * c + 0], r1 = cams[9 * c + 1], r2 = cams[9 * c + 2];
  const double th2 = r0 * r0 + r1 * r1 + r2 * r2;
  double* o = camx + (size_t)kCamx * c;
  if (th2 < 1e-16) {
    // first-order rotation; J_l unused
    const double R[9] = {1.0, -r2, r1, r2, 1.0, -r0, -r1, r0, 1.0};
    for (int i = 0; i < 9; ++i) o[i] = R[i];
    for (int i = 0; i < 9; ++i) o[9 + i] = (i % 4 == 0) ? 1.0 : 0.0;
    o[18] = 1.0;
    camdf_write(camdf, c, o, cams + 9 * c);
    return;
  }
  const double th = sqrt(th2);
  double s, co;
  sincos(th, &s, &co);
  const double a = (1.0 - co) / th2;           // (1 - cos)/th^2
  const double b = (th - s) / (th2 * th);      // (th - sin)/th^3
  const double al = s / th;                    // sin/th
  // K = [r]_x ; K^2 = r r^T - th^2 I
  const double K[9] = {0.0, -r2, r1, r2, 0.0, -r0, -r1, r0, 0.0};
  const double rv[3] = {r0, r1, r2};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K2[3 * i + j] = rv[i] * rv[j] - (i == j ? th2 : 0.0);
  for (int i = 0; i < 9; ++i) {
    const double I = (i % 4 == 0) ? 1.0 : 0.0;
    o[i] = I + al * K[i] + a * K2[i];          // Rodrigues R = I + sin/th K + (1-cos)/th^2 K^2
    o[9 + i] = I + a * K[i] + b * K2[i];       // J_l
  }
  o[18] = 0.0;
  camdf_write(camdf, c, o, cams + 9 * c);
}

template <bool JAC>
__device__ __forceinline__ void project_obs(const double* __restrict__ cam, const double* __restrict__ cx,
                                            const double X[3], const double ob[2], CamObs& out) {
  double c9[9], cr[18];
#pragma unroll
  for (int i = 0; i < 9; ++i) c9[i] = cam[i];
#pragma unroll
  for (int i = 0; i < 18; ++i) cr[i] = cx[i];
  project_obs_t<JAC, double>(c9, cr, cx[18] != 0.0, X, ob, out);
}

template <bool JAC, bool MIXED>
__global__ void __launch_bounds__(kLinBS)
k_linearize(const double* __restrict__ cams, const double* __restrict__ pts,
            const double* __restrict__ obs, const double* __restrict__ camx,
            const int* __restrict__ obs_cam, const int* __restrict__ obs_ptu,
            const int* __restrict__ obs_user, int n_o, size_t ld, double* __restrict__ fres,
            double* __restrict__ J64, float* __restrict__ J32, float* __restrict__ J32lo,
            double* partial, unsigned* counter, double* cost_out, int* flags, double ha) {
  double acc = 0.0;
  for (int o = blockIdx.x * kLinBS + threadIdx.x; o < n_o; o += gridDim.x * kLinBS) {
    const int c = obs_cam[o];
    const int pu = obs_ptu[o];
    const int ou = obs_user[o];
    const double X[3] = {pts[3 * pu], pts[3 * pu + 1], pts[3 * pu + 2]};
    const double ob[2] = {obs[2 * ou], obs[2 * ou + 1]};
    CamObs v;
    project_obs<JAC>(cams + 9 * c, camx + (size_t)kCamx * c, X, ob, v);
    double half_rho;
    const double w = robust_weight(v.res[0] * v.res[0] + v.res[1] * v.res[1], ha, half_rho);
    acc += half_rho;
    if (w != 1.0) {
      v.res[0] *= w;
      v.res[1] *= w;
      if (JAC) {
#pragma unroll
        for (int k = 0; k < 18; ++k) v.F[k] *= w;
#pragma unroll
        for (int k = 0; k < 6; ++k) v.E[k] *= w;
      }
    }
    if (fres) reinterpret_cast<double2*>(fres)[o] = make_double2(v.res[0], v.res[1]);
    if (JAC) {
      bool finite = isfinite(v.res[0]) && isfinite(v.res[1]);
      double rec[kRec];
#pragma unroll
      for (int k = 0; k < 18; ++k) rec[k] = v.F[k];
#pragma unroll
      for (int k = 0; k < 6; ++k) rec[18 + k] = v.E[k];
#pragma unroll
      for (int k = 0; k < kRec; ++k) finite = finite && isfinite(rec[k]);
      double2* d64 = reinterpret_cast<double2*>(J64 + (size_t)o * kRec);
#pragma unroll
      for (int k = 0; k < kRec / 2; ++k) d64[k] = make_double2(rec[2 * k], rec[2 * k + 1]);
      if (MIXED) {
        // FP32 copy (hi) and the remainder (lo): hi + lo carries ~47 bits
        float hi[kRec], lo[kRec];
#pragma unroll
        for (int k = 0; k < kRec; ++k) split_double(rec[k], hi[k], lo[k]);
        float4* d32 = reinterpret_cast<float4*>(J32 + (size_t)o * kRec);
        float4* l32 = reinterpret_cast<float4*>(J32lo + (size_t)o * kRec);
#pragma unroll
        for (int k = 0; k < kRec / 4; ++k) {
          d32[k] = make_float4(hi[4 * k], hi[4 * k + 1], hi[4 * k + 2], hi[4 * k + 3]);
          l32[k] = make_float4(lo[4 * k], lo[4 * k + 1], lo[4 * k + 2], lo[4 * k + 3]);
        }
      }
      if (!finite) flags[F_NONFINITE] = 1;
    }
  }
  grid_sum_store<kLinBS>(acc, partial, counter, cost_out);
}

// points as float pairs, once per point (the observations of a point share the split)
__global__ void k_split_points(size_t n, const double* __restrict__ pts, float2* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const DF v(pts[i]);
    out[i] = make_float2(v.h, v.l);
  }
}

// The mixed-precision linearisation: the camera model of project_obs_t in paired FP32
// (DF), from the per-camera split of camdf, the point split of ptsdf and the observations
// split on load.  Writes the residuals and, directly from the pairs, the FP32 records (hi)
// and their remainders (lo); the FP64 records (hi + lo) only when J64 is given.  With the
// squared loss the cost terms are summed in DF too, so that an observation takes only the
// FP64 additions that form its residual.
template <bool JAC>
__global__ void __launch_bounds__(kLinBS)
k_linearize_df(const float2* __restrict__ ptsdf, const double* __restrict__ obs, const float2* __restrict__ camdf,
               const int* __restrict__ obs_cam, const int* __restrict__ obs_ptu, const int* __restrict__ obs_user,
               int n_o, double* __restrict__ fres, double* __restrict__ J64, float* __restrict__ J32,
               float* __restrict__ J32lo, double* partial, unsigned* counter, double* cost_out, int* flags,
               double ha) {
  double acc = 0.0;
  DF accdf(0.f, 0.f);
  for (int o = blockIdx.x * kLinBS + threadIdx.x; o < n_o; o += gridDim.x * kLinBS) {
    const int c = obs_cam[o];
    const int pu = obs_ptu[o];
    const int ou = obs_user[o];
    const float2* cd = camdf + (size_t)kCamdf * c;
    DF cx[18], cam[9];
#pragma unroll
    for (int i = 0; i < 18; ++i) {
      const float2 v = __ldg(cd + i);
      cx[i] = DF(v.x, v.y);
    }
    const bool small = __ldg(cd + 18).x != 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float2 v = __ldg(cd + 19 + i);
      cam[i] = DF(v.x, v.y);
    }
    const float2 x0 = __ldg(ptsdf + 3 * (size_t)pu), x1 = __ldg(ptsdf + 3 * (size_t)pu + 1),
                 x2 = __ldg(ptsdf + 3 * (size_t)pu + 2);
    const DF X[3] = {DF(x0.x, x0.y), DF(x1.x, x1.y), DF(x2.x, x2.y)};
    const DF ob[2] = {DF(obs[2 * ou]), DF(obs[2 * ou + 1])};
    CamObsT<DF> v;
    project_obs_t<JAC, DF>(cam, cx, small, X, ob, v);
    double r0 = to_double(v.res[0]), r1 = to_double(v.res[1]);
    double w = 1.0;
    bool scaled = false;
    if (ha > 0.0) {
      double half_rho;
      w = robust_weight(r0 * r0 + r1 * r1, ha, half_rho);
      acc += half_rho;
      scaled = w != 1.0;
      if (scaled) {
        r0 *= w;
        r1 *= w;
      }
    } else {
      const DF s2 = v.res[0] * v.res[0] + v.res[1] * v.res[1];
      accdf += DF(0.5f * s2.h, 0.5f * s2.l);
    }
    if (fres) reinterpret_cast<double2*>(fres)[o] = make_double2(r0, r1);
    if (JAC) {
      bool finite = isfinite(r0) && isfinite(r1);
      DF rec[kRec];
#pragma unroll
      for (int k = 0; k < 18; ++k) rec[k] = v.F[k];
#pragma unroll
      for (int k = 0; k < 6; ++k) rec[18 + k] = v.E[k];
      if (scaled) {
        const DF wd(w);
#pragma unroll
        for (int k = 0; k < kRec; ++k) rec[k] = rec[k] * wd;
      }
#pragma unroll
      for (int k = 0; k < kRec; ++k) finite = finite && isfinite(rec[k].h);
      if (J64) {
        double2* d64 = reinterpret_cast<double2*>(J64 + (size_t)o * kRec);
#pragma unroll
        for (int k = 0; k < kRec / 2; ++k) d64[k] = make_double2(to_double(rec[2 * k]), to_double(rec[2 * k + 1]));
      }
      float4* d32 = reinterpret_cast<float4*>(J32 + (size_t)o * kRec);
      float4* l32 = reinterpret_cast<float4*>(J32lo + (size_t)o * kRec);
#pragma unroll
      for (int k = 0; k < kRec / 4; ++k) {
        d32[k] = make_float4(rec[4 * k].h, rec[4 * k + 1].h, rec[4 * k + 2].h, rec[4 * k + 3].h);
        l32[k] = make_float4(rec[4 * k].l, rec[4 * k + 1].l, rec[4 * k + 2].l, rec[4 * k + 3].l);
      }
      if (!finite) flags[F_NONFINITE] = 1;
    }
  }
  acc += to_double(accdf);
  grid_sum_store<kLinBS>(acc, partial, counter, cost_out);
}

static void camera_rotation(ba_problem* P, const double* cams, double* camx, float2* camdf) {
  // one warp per CTA: the cameras' FP64 work spread over as many SMs as possible
  k_camera_rotation<<<cdiv(P->n_c, 32), 32, 0, P->stream>>>(cams, P->n_c, camx, camdf);
  launched(P);
}

// the kernels' loss argument: the Huber scale a, or 0 for the squared loss
static double huber_scale(const ba_problem* P) {
  return P->opt.loss == BA_LOSS_HUBER ? P->opt.loss_scale : 0.0;
}

static void split_points(ba_problem* P, const double* pts) {
  const size_t n = 3 * (size_t)P->n_p;
  P->ptsdf.ensure(sizeof(float2) * std::max<size_t>(n, 1) + 64);
  if (n) {
    k_split_points<<<cdiv((long long)n, 256), 256, 0, P->stream>>>(n, pts, P->ptsdf.as<float2>());
    launched(P);
  }
}

static int lin_grid(ba_problem* P) {
  int g = cdiv(P->n_o, kLinBS);
  return std::max(1, std::min(g, P->n_sm * 8));
}

void linearize(ba_problem* P, const double* cams, const double* pts, const double* obs) {
  const size_t ld = P->ld;
  const bool mixed = P->opt.precision == BA_MIXED;
  P->camx.ensure(sizeof(double) * kCamx * std::max(P->n_c, 1));
  P->fres.ensure(sizeof(double) * 2 * ld);
  if (!mixed) P->J64.ensure(sizeof(double) * kRec * ld);
  P->j64_valid = !mixed;
  if (mixed) {
    P->J32.ensure(sizeof(float) * kRec * ld);
    P->J32lo.ensure(sizeof(float) * kRec * ld);
  }
  // keep the linearisation point (near-nullspace and adjoint use it)
  P->cams_lin.ensure(sizeof(double) * 9 * std::max(P->n_c, 1));
  P->pts_lin.ensure(sizeof(double) * 3 * std::max(P->n_p, 1));
  BA_CUDA(cudaMemcpyAsync(P->cams_lin.p, cams, sizeof(double) * 9 * P->n_c, cudaMemcpyDeviceToDevice, P->stream));
  if (P->n_p)
    BA_CUDA(cudaMemcpyAsync(P->pts_lin.p, pts, sizeof(double) * 3 * P->n_p, cudaMemcpyDeviceToDevice, P->stream));
  P->obs_lin.ensure(sizeof(double) * 2 * std::max(P->n_o, 1));
  if (P->n_o)
    BA_CUDA(cudaMemcpyAsync(P->obs_lin.p, obs, sizeof(double) * 2 * P->n_o, cudaMemcpyDeviceToDevice, P->stream));
  clear_flags(P);
  if (mixed) P->camdf.ensure(sizeof(float2) * kCamdf * std::max(P->n_c, 1));
  camera_rotation(P, cams, P->camx.as<double>(), mixed ? P->camdf.as<float2>() : nullptr);
  int g = lin_grid(P);
  double* cost = P->scal.as<double>() + S_COST;
  KernelTimer kt(P, BA_KT_LINEARIZE);
  if (mixed) split_points(P, pts);
  if (mixed)
    k_linearize_df<true><<<g, kLinBS, 0, P->stream>>>(
        P->ptsdf.as<float2>(), obs, P->camdf.as<float2>(), P->obs_cam.as<int>(), P->obs_ptu.as<int>(), P->obs_user.as<int>(), P->n_o,
        P->fres.as<double>(), nullptr, P->J32.as<float>(), P->J32lo.as<float>(), P->partial.as<double>(),
        P->counter.as<unsigned>(), cost, P->flags.as<int>(), huber_scale(P));
  else
    k_linearize<true, false><<<g, kLinBS, 0, P->stream>>>(
        cams, pts, obs, P->camx.as<double>(), P->obs_cam.as<int>(), P->obs_ptu.as<int>(),
        P->obs_user.as<int>(), P->n_o, ld, P->fres.as<double>(), P->J64.as<double>(), nullptr, nullptr,
        P->partial.as<double>(), P->counter.as<unsigned>(), cost, P->flags.as<int>(), huber_scale(P));
  launched(P);
}

__global__ void k_pair_sum(size_t n, const float* __restrict__ hi, const float* __restrict__ lo,
                           double* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)hi[i] + (double)lo[i];
}

double* jacobian64(ba_problem* P) {
  if (!P->j64_valid) {
    P->J64.ensure(sizeof(double) * kRec * P->ld);
    const size_t n = (size_t)kRec * P->n_o;
    if (n) {
      k_pair_sum<<<cdiv((long long)n, 256), 256, 0, P->stream>>>(n, P->J32.as<float>(), P->J32lo.as<float>(),
                                                                 P->J64.as<double>());
      launched(P);
    }
    P->j64_valid = true;
  }
  return P->J64.as<double>();
}

double cost_at(ba_problem* P, const double* cams, const double* pts, const double* obs) {
  cost_at_async(P, cams, pts, obs);
  return fetch_sum(P, S_COST_NEW);
}

void cost_at_async(ba_problem* P, const double* cams, const double* pts, const double* obs) {
  const bool mixed = P->opt.precision == BA_MIXED;
  // rotation data in the front of scratch2, the camera split behind it
  const size_t rot_bytes = (sizeof(double) * kCamx * std::max(P->n_c, 1) + 255) / 256 * 256;
  P->scratch2.ensure(rot_bytes + sizeof(float2) * kCamdf * std::max(P->n_c, 1));
  float2* camdf = mixed ? reinterpret_cast<float2*>(P->scratch2.as<char>() + rot_bytes) : nullptr;
  camera_rotation(P, cams, P->scratch2.as<double>(), camdf);
  int g = lin_grid(P);
  if (mixed) split_points(P, pts);
  if (mixed)
    k_linearize_df<false><<<g, kLinBS, 0, P->stream>>>(
        P->ptsdf.as<float2>(), obs, camdf, P->obs_cam.as<int>(), P->obs_ptu.as<int>(), P->obs_user.as<int>(), P->n_o, nullptr, nullptr,
        nullptr, nullptr, P->partial.as<double>(), P->counter.as<unsigned>(), P->scal.as<double>() + S_COST_NEW,
        P->flags.as<int>(), huber_scale(P));
  else
    k_linearize<false, false><<<g, kLinBS, 0, P->stream>>>(
        cams, pts, obs, P->scratch2.as<double>(), P->obs_cam.as<int>(), P->obs_ptu.as<int>(),
        P->obs_user.as<int>(), P->n_o, P->ld, nullptr, nullptr, nullptr, nullptr,
        P->partial.as<double>(), P->counter.as<unsigned>(), P->scal.as<double>() + S_COST_NEW,
        P->flags.as<int>(), huber_scale(P));
  launched(P);
}

}  // namespace ba
