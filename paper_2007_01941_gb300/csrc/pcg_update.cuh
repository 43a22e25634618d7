// The end of a PCG iteration with the assembled S, shared by the plain update kernel
// and the one that also starts the next V-cycle: the quadratic model, r.r by a
// deterministic grid reduction, the iteration count, the stopping test and the graph's
// loop condition.
#pragma once

#include "ba_internal.h"
#include "device_util.cuh"

namespace ba {

// stopping test: |r|^2 <= rtol^2 |b|^2, or the Nash-Sofer rule of Section 2.1 on the
// quadratic model Q (q) and its last decrease (dq)
__device__ __host__ inline bool pcg_converged(int rule, double it, double rr, double bb, double rtol2, double q,
                                              double dq, double tau) {
  if (rule == BA_STOP_NASH_SOFER) return q < 0.0 && it * dq / q <= tau;
  return !(rr > rtol2 * bb);
}

struct PcgCheck {
  double* scal;
  double* partial;    // one slot per CTA
  unsigned* counter;  // zero between launches
  int* flags;
  int max_iters;
  double rtol2;
  int rule;
  double tau;
  int use_cond;       // 1: set the graph's while condition
  cudaGraphConditionalHandle h;
  const double* pq_part;  // the product's per-CTA shares of p.q (n_pq_part > 0), else
  int n_pq_part;          // p.q is in scal[S_PQ]
};

// p.q for every thread of the CTA: the product's per-CTA shares added in the same order by
// every CTA (so that the product needs no grid-wide reduction of its own), or scal[S_PQ]
template <int BS>
__device__ __forceinline__ double pcg_pq(const PcgCheck& ck) {
  if (ck.n_pq_part == 0) return ck.scal[S_PQ];
  __shared__ double pq_sm;
  double s = 0.0;
  for (int k = threadIdx.x; k < ck.n_pq_part; k += BS) s += __ldcg(ck.pq_part + k);
  s = block_sum<BS>(s);
  if (threadIdx.x == 0) {
    pq_sm = s;
    if (blockIdx.x == 0) ck.scal[S_PQ] = s;
  }
  __syncthreads();
  return pq_sm;
}

// acc: this thread's share of r.r; ok: alpha was usable (p.q > 0, finite)
template <int BS>
__device__ __forceinline__ void pcg_update_finish(double acc, bool ok, double alpha, double rz, const PcgCheck& ck) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (!ok) ck.flags[F_BREAKDOWN] = 1;
    // quadratic model: Q_i - Q_{i-1} = -alpha (r.z) / 2
    const double dq = ok ? -0.5 * alpha * rz : 0.0;
    ck.scal[S_DQ] = dq;
    ck.scal[S_Q] += dq;
    ck.scal[S_RZ] = rz;   // the next direction's beta divides by this r.z
  }
  // the last block adds the blocks' partial sums in block order, counts the iteration and
  // sets the loop condition (continue while not converged, no breakdown, below max_iters)
  __shared__ bool am_last;
  const double s = block_sum<BS>(acc);
  if (threadIdx.x == 0) {
    ck.partial[blockIdx.x] = s;
    __threadfence();
    am_last = atomicAdd(ck.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (am_last) {
    __threadfence();
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += BS) t += __ldcg(ck.partial + b);
    t = block_sum<BS>(t);
    if (threadIdx.x == 0) {
      double* scal = ck.scal;
      scal[S_RR] = t;
      *ck.counter = 0u;
      const double it = scal[S_ITER] + 1.0;
      scal[S_ITER] = it;
      // a setup whose check was deferred (the LM step) may have failed: stop at once
      const bool setup_failed = __ldcg(ck.flags + F_NOT_SPD_POINT) != 0 || __ldcg(ck.flags + F_NOT_SPD_JACOBI) != 0 ||
                                __ldcg(ck.flags + F_NOT_SPD_COARSE) != 0 || __ldcg(ck.flags + F_NONFINITE) != 0;
      const bool stop =
          pcg_converged(ck.rule, it, t, scal[S_BB], ck.rtol2, __ldcg(scal + S_Q), __ldcg(scal + S_DQ), ck.tau) ||
          __ldcg(ck.flags + F_BREAKDOWN) != 0 || setup_failed || it >= (double)ck.max_iters;
      if (ck.use_cond) cudaGraphSetConditional(ck.h, stop ? 0u : 1u);
    }
  }
}

}  // namespace ba
