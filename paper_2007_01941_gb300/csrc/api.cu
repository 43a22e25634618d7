// extern "C" entry points of ba.h: argument checks, stage bookkeeping and the
// conversion of internal errors into ba_status codes.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ba_internal.h"
#include "device_util.cuh"

namespace ba {
void back_substitute_to(ba_problem* P, const double* dc, double* out_int, double* out_user);
}

namespace {

using ba::Error;

template <typename Fn>
ba_status guard(ba_problem* P, Fn&& fn) {
  try {
    fn();
    if (P) P->err.clear();
    return BA_OK;
  } catch (const Error& e) {
    if (P) P->err = e.what();
    return e.status;
  } catch (const std::exception& e) {
    if (P) P->err = e.what();
    return BA_ERR_CUDA;
  }
}

void require_stage(ba_problem* P, int stage, const char* what) {
  BA_REQUIRE(P->stage >= stage, BA_ERR_STATE, std::string(what));
}

__global__ void k_soa_to_user(const double* __restrict__ src, size_t ld, int rows, int n, const int* __restrict__ perm,
                              double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int u = perm[i];
  for (int k = 0; k < rows; ++k) dst[(size_t)u * rows + k] = src[k * ld + i];
}

// interleaved per-observation records (stride values each, `rows` of them from `offset`)
__global__ void k_rec_to_user(const double* __restrict__ src, int stride, int offset, int rows, int n,
                              const int* __restrict__ perm, double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int u = perm[i];
  for (int k = 0; k < rows; ++k) dst[(size_t)u * rows + k] = src[(size_t)i * stride + offset + k];
}

__global__ void k_cinv_to_user(const double* __restrict__ src, size_t ldp, int n, const int* __restrict__ perm,
                               double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int idx[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
  double* d = dst + 9 * (size_t)perm[i];
  for (int k = 0; k < 9; ++k) d[k] = src[idx[k] * ldp + i];
}

// (hi, lo) float pairs -> their double sums
__global__ void k_df2d(size_t n, const float2* __restrict__ in, double* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i].x + (double)in[i].y;
}

__global__ void k_f2d(size_t n, const float* __restrict__ a, double* __restrict__ b) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}
__global__ void k_d2f(size_t n, const double* __restrict__ a, float* __restrict__ b) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

}  // namespace

extern "C" {

void ba_default_options(ba_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->lambda = 1e-4;
  o->rtol = 1e-6;
  o->max_iters = 1000;
  o->precision = BA_FP64;
  o->preconditioner = BA_PRECOND_MG;
  o->damping = BA_DAMP_MARQUARDT;
  o->recompute_jacobian = 1;
  o->max_agg = 20;
  o->pre_smooth = 2;
  o->post_smooth = 2;
  o->lanczos_steps = 5;
  o->coarse_max_nodes = 32;
  o->max_levels = 10;
  o->cheb_lo = 0.3;
  o->cheb_hi = 1.1;
  o->level0_operator = BA_OP_AUTO;
  o->fused_vcycle = 1;
  o->outer_product = BA_OUTER_PAIRED_FP32;
  o->stop_rule = BA_STOP_RELRES;
  o->tau = 0.1;
  o->overlap_launches = 1;
  o->loss = BA_LOSS_SQUARED;
  o->loss_scale = 1.0;
  o->precond_lambda_min = 1e-5;
  o->schur_staging = 0;
}

size_t ba_struct_size(int which) {
  return which == 0 ? sizeof(ba_options) : which == 1 ? sizeof(ba_info) : 0;
}

ba_status ba_create(int n_cams, int n_pts, int n_obs, const int32_t* cam_idx, const int32_t* pt_idx,
                    const ba_options* opt, void* stream, ba_problem** out) {
  if (!out) return BA_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_cams < 1 || n_pts < 0 || n_obs < 0) return BA_ERR_INVALID_ARG;
  if (n_obs > 0 && (!cam_idx || !pt_idx)) return BA_ERR_INVALID_ARG;
  ba_problem* P = new ba_problem();
  if (opt) P->opt = *opt;
  else ba_default_options(&P->opt);
  P->stream = static_cast<cudaStream_t>(stream);
  P->n_c = n_cams;
  P->n_p = n_pts;
  P->n_o = n_obs;
  P->levels.reserve(16);
  ba_status st = guard(P, [&] {
    const ba_options& o = P->opt;
    BA_REQUIRE(o.precision == BA_FP64 || o.precision == BA_MIXED, BA_ERR_INVALID_ARG, "bad precision");
    BA_REQUIRE(o.preconditioner >= 0 && o.preconditioner <= 2, BA_ERR_INVALID_ARG, "bad preconditioner");
    BA_REQUIRE(o.max_agg >= 2 && o.max_agg <= 64, BA_ERR_INVALID_ARG, "max_agg must be in [2, 64]");
    BA_REQUIRE(o.pre_smooth >= 1 && o.post_smooth >= 1 && o.pre_smooth <= ba::kMaxSmooth &&
                   o.post_smooth <= ba::kMaxSmooth,
               BA_ERR_INVALID_ARG, "smoothing steps must be in 1 .. 8");
    BA_REQUIRE(o.lanczos_steps >= 1 && o.lanczos_steps <= 8, BA_ERR_INVALID_ARG, "lanczos_steps in [1, 8]");
    BA_REQUIRE(o.max_iters >= 1 && o.rtol >= 0.0, BA_ERR_INVALID_ARG, "bad PCG limits");
    BA_REQUIRE(o.cheb_hi > o.cheb_lo && o.cheb_lo > 0.0, BA_ERR_INVALID_ARG, "bad Chebyshev interval");
    BA_REQUIRE(o.max_levels >= 1 && o.coarse_max_nodes >= 1, BA_ERR_INVALID_ARG, "bad hierarchy limits");
    BA_REQUIRE(o.level0_operator >= BA_OP_IMPLICIT && o.level0_operator <= BA_OP_AUTO, BA_ERR_INVALID_ARG,
               "bad level0_operator");
    BA_REQUIRE(o.outer_product == BA_OUTER_FP64 || o.outer_product == BA_OUTER_PAIRED_FP32, BA_ERR_INVALID_ARG,
               "bad outer_product");
    BA_REQUIRE(o.stop_rule == BA_STOP_RELRES || (o.stop_rule == BA_STOP_NASH_SOFER && o.tau > 0.0),
               BA_ERR_INVALID_ARG, "bad stop_rule / tau");
    BA_REQUIRE(o.loss == BA_LOSS_SQUARED || (o.loss == BA_LOSS_HUBER && o.loss_scale > 0.0 &&
                                             std::isfinite(o.loss_scale)),
               BA_ERR_INVALID_ARG, "bad loss / loss_scale");
    BA_REQUIRE(o.precond_lambda_min >= 0.0 && std::isfinite(o.precond_lambda_min), BA_ERR_INVALID_ARG,
               "bad precond_lambda_min");
    BA_REQUIRE(o.schur_staging == 0 || o.schur_staging == 1, BA_ERR_INVALID_ARG, "bad schur_staging");
    int dev = 0;
    BA_CUDA(cudaGetDevice(&dev));
    BA_CUDA(cudaDeviceGetAttribute(&P->n_sm, cudaDevAttrMultiProcessorCount, dev));
    P->scal.ensure(sizeof(double) * ba::kScalars);
    // one partial sum per block of any grid reduction (at most 8 blocks per SM)
    P->partial.ensure(sizeof(double) * (16 * (size_t)P->n_sm + 64));
    P->counter.ensure(sizeof(unsigned) * 8);
    P->flags.ensure(sizeof(int) * ba::F_COUNT);
    BA_CUDA(cudaMemsetAsync(P->scal.p, 0, sizeof(double) * ba::kScalars, P->stream));
    BA_CUDA(cudaMemsetAsync(P->counter.p, 0, sizeof(unsigned) * 8, P->stream));
    BA_CUDA(cudaMemsetAsync(P->flags.p, 0, sizeof(int) * ba::F_COUNT, P->stream));
    BA_CUDA(cudaMallocHost(&P->h_scal, sizeof(double) * ba::kScalars));
    BA_CUDA(cudaMallocHost(&P->h_flags, sizeof(int) * ba::F_COUNT));
    BA_CUDA(cudaMallocHost(&P->h_cheb, sizeof(double) * 16 * ba::kChebSlots));
    ba::build_graph(P, cam_idx, pt_idx);
  });
  if (st != BA_OK) {
    ba_destroy(P);
    return st;
  }
  *out = P;
  return BA_OK;
}

void ba_destroy(ba_problem* P) {
  if (!P) return;
  cudaStreamSynchronize(P->stream);
  if (P->side_stream) {
    cudaStreamSynchronize(P->side_stream);
    cudaStreamDestroy(P->side_stream);
    cudaEventDestroy(P->ev_fork);
    cudaEventDestroy(P->ev_join);
  }
  ba::for_each_problem_buf(P, [](ba::DBuf& b) { b.release(); });
  for (ba::Level& L : P->levels) ba::for_each_level_buf(L, [](ba::DBuf& b) { b.release(); });
  if (P->h_scal) cudaFreeHost(P->h_scal);
  if (P->h_flags) cudaFreeHost(P->h_flags);
  if (P->h_cheb) cudaFreeHost(P->h_cheb);
  for (auto& r : P->krec) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : P->ev_pool) cudaEventDestroy(e);
  if (P->pcg_exec) cudaGraphExecDestroy(P->pcg_exec);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  delete P;
}

const char* ba_last_error(const ba_problem* P) { return P ? P->err.c_str() : "null problem"; }

ba_status ba_linearize(ba_problem* P, const double* cams, const double* pts, const double* obs, double* cost_out) {
  if (!P) return BA_ERR_INVALID_ARG;
  return guard(P, [&] {
    BA_REQUIRE(cams && (pts || P->n_p == 0) && (obs || P->n_o == 0), BA_ERR_INVALID_ARG, "null array");
    P->stage = 0;
    ba::linearize(P, cams, pts, obs);
    ba::check_flags(P);
    P->cost = ba::fetch_sum(P, ba::S_COST);
    if (cost_out) *cost_out = P->cost;
    P->stage = 1;
  });
}

ba_status ba_schur_setup(ba_problem* P, double lambda) {
  if (!P) return BA_ERR_INVALID_ARG;
  return guard(P, [&] {
    require_stage(P, 1, "ba_schur_setup needs ba_linearize first");
    BA_REQUIRE(lambda >= 0.0, BA_ERR_INVALID_ARG, "lambda must be >= 0");
    P->stage = 1;
    ba::schur_setup(P, lambda);
    P->stage = 2;
  });
}

ba_status ba_mg_setup(ba_problem* P) {
  if (!P) return BA_ERR_INVALID_ARG;
  return guard(P, [&] {
    require_stage(P, 2, "ba_mg_setup needs ba_schur_setup first");
    P->stage = 2;
    if (P->opt.preconditioner == BA_PRECOND_MG) ba::mg_setup(P);
    P->stage = 3;
  });
}

ba_status ba_pcg_solve(ba_problem* P, const double* rhs, double* delta_c, int* iters, double* rel_res) {
  if (!P) return BA_ERR_INVALID_ARG;
  ba_status st = guard(P, [&] {
    require_stage(P, P->opt.preconditioner == BA_PRECOND_MG ? 3 : 2, "ba_pcg_solve needs the setup calls first");
    BA_REQUIRE(delta_c, BA_ERR_INVALID_ARG, "null delta_c");
    ba::pcg(P, rhs ? rhs : P->rhs.as<double>(), delta_c);
  });
  if (st == BA_OK || st == BA_ERR_NOT_CONVERGED) {
    if (iters) *iters = P->pcg_iters;
    if (rel_res) *rel_res = P->pcg_rel;
    if (!rhs) {
      ba_status st2 = guard(P, [&] {
        const size_t nc = (size_t)P->n_c * 9;
        P->delta_c.ensure(sizeof(double) * nc + 64);
        BA_CUDA(cudaMemcpyAsync(P->delta_c.p, delta_c, sizeof(double) * nc, cudaMemcpyDeviceToDevice, P->stream));
        P->delta_p.ensure(sizeof(double) * 3 * P->ldp);
        ba::back_substitute_to(P, delta_c, P->delta_p.as<double>(), nullptr);
        ba::sync(P);
        P->stage = 4;
      });
      if (st2 != BA_OK) return st2;
    }
  }
  return st;
}

ba_status ba_back_substitute(ba_problem* P, const double* delta_c, double* delta_p) {
  if (!P) return BA_ERR_INVALID_ARG;
  return guard(P, [&] {
    require_stage(P, 2, "ba_back_substitute needs ba_schur_setup first");
    BA_REQUIRE(delta_c && (delta_p || P->n_p == 0), BA_ERR_INVALID_ARG, "null array");
    ba::back_substitute_to(P, delta_c, nullptr, delta_p);
    ba::sync(P);
  });
}

ba_status ba_lm_step(ba_problem* P, double* cams, double* pts, const double* obs, double* lambda_inout,
                     int* accepted, double* cost_out) {
  if (!P) return BA_ERR_INVALID_ARG;
  return guard(P, [&] {
    BA_REQUIRE(cams && lambda_inout && accepted && cost_out, BA_ERR_INVALID_ARG, "null argument");
    BA_REQUIRE(*lambda_inout >= 0.0, BA_ERR_INVALID_ARG, "lambda must be >= 0");
    P->stage = 0;
    ba::lm_step(P, cams, pts, obs, lambda_inout, accepted, cost_out);
    if (P->stage != 1) P->stage = 4;   // 1: the step's linear solve failed (step rejected)
  });
}

ba_status ba_set_partition(ba_problem* P, int n_obs_all, const int32_t* cam_idx_all, const int32_t* pt_idx_all,
                           ba_allreduce_fn allreduce, void* user) {
  if (!P) return BA_ERR_INVALID_ARG;
  return guard(P, [&] {
    BA_REQUIRE(P->stage == 0 && !P->sym_ready && !P->part_fn, BA_ERR_STATE,
               "ba_set_partition must come once, after ba_create and before the first ba_linearize");
    BA_REQUIRE(allreduce, BA_ERR_INVALID_ARG, "null all-reduce hook");
    BA_REQUIRE(n_obs_all >= P->n_o && (n_obs_all == 0 || (cam_idx_all && pt_idx_all)), BA_ERR_INVALID_ARG,
               "the whole problem's observation graph must include this rank's observations");
    BA_REQUIRE(P->opt.precision == BA_FP64, BA_ERR_INVALID_ARG, "a partitioned solve runs in BA_FP64");
    BA_REQUIRE(P->opt.preconditioner == BA_PRECOND_MG, BA_ERR_INVALID_ARG,
               "a partitioned solve needs the multigrid preconditioner (its assembled S)");
    BA_REQUIRE(P->opt.level0_operator != BA_OP_IMPLICIT, BA_ERR_INVALID_ARG,
               "a partitioned solve uses the assembled level-0 operator");
    for (int o = 0; o < n_obs_all; ++o)
      BA_REQUIRE(cam_idx_all[o] >= 0 && cam_idx_all[o] < P->n_c && pt_idx_all[o] >= 0, BA_ERR_INVALID_ARG,
                 "observation index out of range in the partition's observation graph");
    P->part_cam.assign(cam_idx_all, cam_idx_all + n_obs_all);
    P->part_pt.assign(pt_idx_all, pt_idx_all + n_obs_all);
    P->opt.level0_operator = BA_OP_EXPLICIT;
    P->part_user = user;
    P->part_fn = allreduce;
  });
}

ba_status ba_adjoint(ba_problem* P, const double* dL_ddelta, double* dL_dobs, double* dL_dcams, double* dL_dpts) {
  if (!P) return BA_ERR_INVALID_ARG;
  return guard(P, [&] {
    require_stage(P, 4, "ba_adjoint needs a completed solve (ba_pcg_solve with rhs = NULL, or ba_lm_step)");
    BA_REQUIRE(dL_ddelta, BA_ERR_INVALID_ARG, "null cotangent");
    BA_REQUIRE(P->opt.loss == BA_LOSS_SQUARED, BA_ERR_INVALID_ARG,
               "ba_adjoint differentiates the squared loss only");
    BA_REQUIRE(!ba::partitioned(P), BA_ERR_INVALID_ARG, "ba_adjoint is not available on a partitioned problem");
    ba::adjoint(P, dL_ddelta, dL_dobs, dL_dcams, dL_dpts);
  });
}

ba_status ba_schur_matvec(ba_problem* P, const double* x, double* y, int precision) {
  if (!P) return BA_ERR_INVALID_ARG;
  return guard(P, [&] {
    require_stage(P, 2, "ba_schur_matvec needs ba_schur_setup first");
    BA_REQUIRE(x && y, BA_ERR_INVALID_ARG, "null array");
    BA_REQUIRE(!ba::partitioned(P), BA_ERR_INVALID_ARG,
               "the implicit product of a partitioned problem holds only this rank's points");
    const size_t n = (size_t)P->n_c * 9;
    if (precision == BA_MIXED) {
      BA_REQUIRE(P->opt.precision == BA_MIXED, BA_ERR_STATE, "FP32 Jacobian storage exists only in mixed precision");
      P->y32b.ensure(sizeof(float) * 2 * n + 64);
      float* xf = P->y32b.as<float>();
      float* yf = xf + n;
      k_d2f<<<ba::cdiv((long long)n, 256), 256, 0, P->stream>>>(n, x, xf);
      ba::launched(P);
      ba::matvec32(P, xf, yf);
      k_f2d<<<ba::cdiv((long long)n, 256), 256, 0, P->stream>>>(n, yf, y);
      ba::launched(P);
    } else {
      ba::matvec64(P, x, y);
    }
    ba::sync(P);
  });
}

ba_status ba_precond_apply(ba_problem* P, const double* r, double* z) {
  if (!P) return BA_ERR_INVALID_ARG;
  return guard(P, [&] {
    require_stage(P, P->opt.preconditioner == BA_PRECOND_MG ? 3 : 2, "preconditioner not set up");
    BA_REQUIRE(r && z, BA_ERR_INVALID_ARG, "null array");
    ba::precond_apply(P, r, z);
    ba::sync(P);
  });
}

ba_status ba_set_kernel_timing(ba_problem* P, int enable) {
  if (!P) return BA_ERR_INVALID_ARG;
  return guard(P, [&] { ba::kernel_timing_enable(P, enable != 0); });
}

ba_status ba_get_kernel_timing(ba_problem* P, int kernel_class, double* total_ms, long long* launches) {
  if (!P || !total_ms || !launches) return BA_ERR_INVALID_ARG;
  return guard(P, [&] {
    BA_REQUIRE(kernel_class >= 0 && kernel_class < BA_KT_COUNT, BA_ERR_INVALID_ARG, "bad kernel class");
    ba::kernel_timing_get(P, kernel_class, total_ms, launches);
  });
}

ba_status ba_get_info(ba_problem* P, ba_info* info) {
  if (!P || !info) return BA_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  const bool mg = P->opt.preconditioner == BA_PRECOND_MG && P->stage >= 3;
  info->n_levels = mg ? P->n_levels : 0;
  for (int l = 0; l < info->n_levels && l < 16; ++l) {
    const ba::Level& L = P->levels[l];
    info->level_nodes[l] = L.n;
    info->level_block[l] = L.bs;
    info->level_nnzb[l] = L.nnzb;
    // the Lanczos estimate lives on the device (slot 3 of the level's Chebyshev data)
    double lam = 0.0;
    if (!L.coarsest && L.cheb.p &&
        cudaMemcpyAsync(P->h_cheb, L.cheb.p, sizeof(double) * 4, cudaMemcpyDeviceToHost, P->stream) == cudaSuccess &&
        cudaStreamSynchronize(P->stream) == cudaSuccess)
      lam = P->h_cheb[3];
    info->level_lambda_max[l] = lam;
  }
  info->pcg_iters = P->pcg_iters;
  info->pcg_rel_res = P->pcg_rel;
  info->cost = P->cost;
  info->lambda = P->lambda;
  info->kernel_launches = P->launches;
  info->level0_explicit = P->l0_explicit ? 1 : 0;
  return BA_OK;
}

ba_status ba_get_array(ba_problem* P, int which, int level, void* dst, size_t bytes, size_t* needed) {
  if (!P) return BA_ERR_INVALID_ARG;
  return guard(P, [&] {
    const int n_o = P->n_o, n_p = P->n_p, n_c = P->n_c;
    const bool lvl = which >= BA_ARR_LEVEL_ROWPTR && which <= BA_ARR_COARSE_INV;
    const ba::Level* L = nullptr;
    if (lvl) {
      require_stage(P, 3, "no multigrid hierarchy");
      BA_REQUIRE(level >= 0 && level < P->n_levels, BA_ERR_INVALID_ARG, "level out of range");
      L = &P->levels[level];
    }
    size_t need = 0;
    switch (which) {
      case BA_ARR_RESIDUAL: need = sizeof(double) * 2 * n_o; break;
      case BA_ARR_JAC_F: need = sizeof(double) * 18 * n_o; break;
      case BA_ARR_JAC_E: need = sizeof(double) * 6 * n_o; break;
      case BA_ARR_DAMP_C: case BA_ARR_GRAD_C: case BA_ARR_RHS: need = sizeof(double) * 9 * n_c; break;
      case BA_ARR_DAMP_P: case BA_ARR_GRAD_P: need = sizeof(double) * 3 * n_p; break;
      case BA_ARR_CINV: need = sizeof(double) * 9 * n_p; break;
      case BA_ARR_SCC_INV: need = sizeof(double) * 81 * n_c; break;
      case BA_ARR_LEVEL_ROWPTR: need = sizeof(int) * (L->n + 1); break;
      case BA_ARR_LEVEL_COLS: need = sizeof(int) * L->nnzb; break;
      case BA_ARR_LEVEL_VALS: need = sizeof(double) * (size_t)L->nnzb * L->bs * L->bs; break;
      case BA_ARR_LEVEL_W: need = sizeof(long long) * L->nnzb; break;
      case BA_ARR_STRENGTH_PTR: BA_REQUIRE(!L->coarsest, BA_ERR_INVALID_ARG, "coarsest level"); need = sizeof(int) * (L->n + 1); break;
      case BA_ARR_STRENGTH_IDX: BA_REQUIRE(!L->coarsest, BA_ERR_INVALID_ARG, "coarsest level"); need = sizeof(int) * L->n_strength; break;
      case BA_ARR_AGG: BA_REQUIRE(!L->coarsest, BA_ERR_INVALID_ARG, "coarsest level"); need = sizeof(int) * L->n; break;
      case BA_ARR_NULLSPACE: need = sizeof(double) * (size_t)L->n * L->bs * ba::kNull; break;
      case BA_ARR_PROLONG: BA_REQUIRE(!L->coarsest, BA_ERR_INVALID_ARG, "coarsest level"); need = sizeof(double) * (size_t)L->n * L->bs * ba::kNull; break;
      case BA_ARR_KEPT: need = sizeof(unsigned) * L->n; break;
      case BA_ARR_JACOBI_INV: BA_REQUIRE(!L->coarsest, BA_ERR_INVALID_ARG, "coarsest level"); need = sizeof(double) * (size_t)L->n * L->bs * L->bs; break;
      case BA_ARR_COARSE_INV: BA_REQUIRE(L->coarsest, BA_ERR_INVALID_ARG, "not the coarsest level"); need = sizeof(double) * (size_t)L->N * L->N; break;
      default: throw Error(BA_ERR_INVALID_ARG, "unknown array");
    }
    if (needed) *needed = need;
    if (!dst) return;
    BA_REQUIRE(bytes >= need, BA_ERR_INVALID_ARG, "destination too small");
    if (which <= BA_ARR_RHS || which == BA_ARR_SCC_INV) require_stage(P, which <= BA_ARR_JAC_E ? 1 : 2, "not computed yet");
    double* d = static_cast<double*>(dst);
    auto D2D = [&](const void* src, size_t b) {
      BA_CUDA(cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToDevice, P->stream));
    };
    const int go = ba::cdiv(std::max(n_o, 1), 256), gp = ba::cdiv(std::max(n_p, 1), 256);
    switch (which) {
      case BA_ARR_RESIDUAL:
        k_rec_to_user<<<go, 256, 0, P->stream>>>(P->fres.as<double>(), 2, 0, 2, n_o, P->obs_user.as<int>(), d); break;
      case BA_ARR_JAC_F:
        k_rec_to_user<<<go, 256, 0, P->stream>>>(ba::jacobian64(P), ba::kRec, 0, 18, n_o, P->obs_user.as<int>(), d); break;
      case BA_ARR_JAC_E:
        k_rec_to_user<<<go, 256, 0, P->stream>>>(ba::jacobian64(P), ba::kRec, 18, 6, n_o, P->obs_user.as<int>(), d); break;
      case BA_ARR_DAMP_C: D2D(P->Dc.p, need); break;
      case BA_ARR_GRAD_C: D2D(P->gc.p, need); break;
      case BA_ARR_RHS: D2D(P->rhs.p, need); break;
      case BA_ARR_SCC_INV: D2D(P->Scc_inv.p, need); break;
      case BA_ARR_DAMP_P:
        k_soa_to_user<<<gp, 256, 0, P->stream>>>(P->Dp.as<double>(), P->ldp, 3, n_p, P->pt_user.as<int>(), d); break;
      case BA_ARR_GRAD_P:
        k_soa_to_user<<<gp, 256, 0, P->stream>>>(P->gp.as<double>(), P->ldp, 3, n_p, P->pt_user.as<int>(), d); break;
      case BA_ARR_CINV:
        k_cinv_to_user<<<gp, 256, 0, P->stream>>>(P->Cinv64.as<double>(), P->ldp, n_p, P->pt_user.as<int>(), d); break;
      case BA_ARR_LEVEL_ROWPTR: D2D(L->row_ptr.p, need); break;
      case BA_ARR_LEVEL_COLS: D2D(L->cols.p, need); break;
      case BA_ARR_LEVEL_W: D2D(L->W.p, need); break;
      case BA_ARR_LEVEL_VALS: {
        const size_t n = (size_t)L->nnzb * L->bs * L->bs;
        if (P->opt.precision == BA_MIXED && level == 0 && P->outer_explicit)
          k_df2d<<<ba::cdiv((long long)std::max<size_t>(n, 1), 256), 256, 0, P->stream>>>(n, L->valsdf.as<float2>(), d);
        else if (P->opt.precision == BA_MIXED)
          k_f2d<<<ba::cdiv((long long)std::max<size_t>(n, 1), 256), 256, 0, P->stream>>>(n, L->vals32.as<float>(), d);
        else
          D2D(L->vals64.p, need);
        break;
      }
      case BA_ARR_STRENGTH_PTR: D2D(L->sptr.p, need); break;
      case BA_ARR_STRENGTH_IDX: D2D(L->sidx.p, need); break;
      case BA_ARR_AGG: D2D(L->agg.p, need); break;
      case BA_ARR_NULLSPACE: D2D(L->K.p, need); break;
      case BA_ARR_PROLONG: D2D(L->Q64.p, need); break;
      case BA_ARR_KEPT: D2D(L->kept.p, need); break;
      case BA_ARR_JACOBI_INV: D2D(L->Dinv64.p, need); break;
      case BA_ARR_COARSE_INV: D2D(L->Ainv.p, need); break;
      default: break;
    }
    ba::launched(P);
    ba::sync(P);
  });
}

}  // extern "C"
