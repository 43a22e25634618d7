// One V-cycle of Algorithm 1 (Section 2.3) for hierarchies whose every level has an
// assembled block-sparse operator (level 0 the 9x9-block S, coarse levels the 16x16-block
// Galerkin products) and whose coarsest level has an explicit inverse.  The smoother is
// the Chebyshev / point-block-Jacobi iteration of Section 3.4 (Saad, Iterative Methods,
// Alg. 12.1), as in the step-per-launch path of solve.cu, which this one replaces when
// the level-0 operator is assembled.
//
// Each block-sparse product is fused into the kernel of the element-wise step that
// consumes it, because the warp that owns a block row holds the whole row of the
// product; one launch per phase:
//   pre-smoothing  step 0:   r = b, d = D^-1 r / theta, x = d
//                  step k:   q = A d; r' = r - q; d' = rho_k rho_{k-1} d + 2 rho_k / delta D^-1 r'; x += d'
//   restriction:             b_c[a] = sum_{i in a} Q_i^T (r_i - (A d)_i)     (one warp per aggregate)
//   coarsest:                x_c = A_c^-1 b_c
//   prolongation:            x_i += Q_i x_c[agg(i)]
//   post-smoothing step 0:   q = A x; r = b - q; d = D^-1 r / theta; x' = x + d
//                  step k:   as in pre-smoothing
// d and r alternate between two buffers per level, and x moves to its second buffer
// at post-smoothing step 0, so that no kernel writes a vector that its own warps read.
#include <algorithm>

#include "ba_internal.h"
#include "device_util.cuh"

namespace ba {

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
  T* b;
  T* x[2];
  T* r[2];
  T* d[2];
};

__device__ __forceinline__ double vc_rho(const double* cheb, int k) {
  double rho = 1.0 / cheb[2];
  for (int j = 1; j <= k; ++j) rho = 1.0 / (2.0 * cheb[2] - rho);
  return rho;
}

// (A v)_i for block row i, computed by one warp: lane u < BS returns component u.
// The row's block columns are read once, coalesced, and handed out by shuffles, so the
// loads of the blocks and of v are independent of each other and can all be in flight.
template <typename T, int BS>
__device__ __forceinline__ T row_product(const VLevel<T>& L, int i, const T* __restrict__ v, int lane) {
  const int e0 = L.row_ptr[i], e1 = L.row_ptr[i + 1];
  const int nb = e1 - e0;
  T acc = T(0);
  // BS = 9: lane = r + 9k (k < 3) takes row r of blocks k, k+3, ...; BS = 16: lane =
  // u + 16h takes row u of blocks h, h+2, ...
  constexpr int kGroups = BS == 9 ? 3 : 2;
  const int r = BS == 9 ? lane % 9 : (lane & 15);
  const int k = BS == 9 ? lane / 9 : (lane >> 4);
  for (int base = 0; base < nb; base += 32) {
    const int cl = base + lane < nb ? L.cols[e0 + base + lane] : 0;
    const int lim = min(32, nb - base);
    const int steps = (lim + kGroups - 1) / kGroups;   // the same in every lane
#pragma unroll 2
    for (int m = 0; m < steps; ++m) {
      const int j = k + m * kGroups;
      const int col = __shfl_sync(kFull, cl, j & 31);
      if (k < kGroups && j < lim) {
        const T* a = L.vals + (size_t)(e0 + base + j) * (BS * BS) + r * BS;
        const T* xv = v + (size_t)col * BS;
#pragma unroll
        for (int c = 0; c < BS; ++c) acc += a[c] * xv[c];
      }
    }
  }
  if (BS == 9) {
    const T a1 = __shfl_sync(kFull, acc, min(lane + 9, 31));
    const T a2 = __shfl_sync(kFull, acc, min(lane + 18, 31));
    return acc + a1 + a2;
  }
  return acc + __shfl_xor_sync(kFull, acc, 16);
}

// (D_i^-1 w)_u where lane v < BS holds w_v
template <typename T, int BS>
__device__ __forceinline__ T block_apply(const T* __restrict__ Dinv_i, T w, int lane) {
  const int u = lane < BS ? lane : 0;
  T dr[BS];
#pragma unroll
  for (int v = 0; v < BS; ++v) dr[v] = Dinv_i[u * BS + v];
  T acc = T(0);
#pragma unroll
  for (int v = 0; v < BS; ++v) acc += dr[v] * __shfl_sync(kFull, w, v);
  return lane < BS ? acc : T(0);
}

// pre-smoothing step 0 with x = 0: r = b, d = D^-1 b / theta, x = d (one warp per row);
// on level 0 b comes in as the FP64 right-hand side
template <typename T, int BS>
__device__ __forceinline__ void phase_first(const VLevel<T>& L, const double* __restrict__ in, int gw, int nw,
                                            int lane) {
  const T inv_theta = (T)(1.0 / L.cheb[0]);
  for (int i = gw; i < L.n; i += nw) {
    const size_t idx = (size_t)i * BS + lane;
    T bv = T(0);
    if (lane < BS) {
      bv = in ? (T)in[idx] : L.b[idx];
      if (in) L.b[idx] = bv;
    }
    const T dv = block_apply<T, BS>(L.Dinv + (size_t)i * BS * BS, bv, lane) * inv_theta;
    if (lane < BS) {
      L.r[0][idx] = bv;
      L.d[0][idx] = dv;
      L.x[0][idx] = dv;
    }
  }
}

// Chebyshev step k >= 1: q = A din; rout = rin - q; dout = c1 din + c2 D^-1 rout; x += dout
template <typename T, int BS>
__device__ __forceinline__ void phase_step(const VLevel<T>& L, const T* __restrict__ din, T* __restrict__ dout,
                                           const T* __restrict__ rin, T* __restrict__ rout, T* __restrict__ x,
                                           T c1, T c2, double* __restrict__ out, int gw, int nw, int lane) {
  for (int i = gw; i < L.n; i += nw) {
    const T q = row_product<T, BS>(L, i, din, lane);
    const size_t idx = (size_t)i * BS + lane;
    const T rv = lane < BS ? rin[idx] - q : T(0);
    const T acc = block_apply<T, BS>(L.Dinv + (size_t)i * BS * BS, rv, lane);
    if (lane < BS) {
      const T dn = c1 * din[idx] + c2 * acc;
      const T xn = x[idx] + dn;
      rout[idx] = rv;
      dout[idx] = dn;
      x[idx] = xn;
      if (out) out[idx] = (double)xn;
    }
  }
}

// restriction b_c[a] = sum_{i in a} Q_i^T (r_i - (A d)_i), one warp per aggregate
template <typename T, int BS>
__device__ __forceinline__ void phase_restrict(const VLevel<T>& L, const VLevel<T>& C, const T* __restrict__ dv,
                                               const T* __restrict__ rv, int gw, int nw, int lane) {
  for (int a = gw; a < C.n; a += nw) {
    T acc = T(0);
    for (int m = L.agg_ptr[a]; m < L.agg_ptr[a + 1]; ++m) {
      const int i = L.agg_mem[m];
      const T q = row_product<T, BS>(L, i, dv, lane);
      const T res = lane < BS ? rv[(size_t)i * BS + lane] - q : T(0);
      const T* Qi = L.Q + (size_t)i * BS * 16 + (lane & 15);
      T qv[BS];
#pragma unroll
      for (int u = 0; u < BS; ++u) qv[u] = Qi[u * 16];
#pragma unroll
      for (int u = 0; u < BS; ++u) acc += qv[u] * __shfl_sync(kFull, res, u);
    }
    if (lane < 16) C.b[(size_t)a * 16 + lane] = acc;
  }
}

// post-smoothing step 0: q = A xin; r = b - q; d = D^-1 r / theta; xout = xin + d
template <typename T, int BS>
__device__ __forceinline__ void phase_post_first(const VLevel<T>& L, const T* __restrict__ xin, T* __restrict__ xout,
                                                 T* __restrict__ r, T* __restrict__ d, double* __restrict__ out,
                                                 int gw, int nw, int lane) {
  const T inv_theta = (T)(1.0 / L.cheb[0]);
  for (int i = gw; i < L.n; i += nw) {
    const T q = row_product<T, BS>(L, i, xin, lane);
    const size_t idx = (size_t)i * BS + lane;
    const T rv = lane < BS ? L.b[idx] - q : T(0);
    const T dv = block_apply<T, BS>(L.Dinv + (size_t)i * BS * BS, rv, lane) * inv_theta;
    if (lane < BS) {
      const T xn = xin[idx] + dv;
      r[idx] = rv;
      d[idx] = dv;
      xout[idx] = xn;
      if (out) out[idx] = (double)xn;
    }
  }
}

constexpr int kPhaseBS = 256;
constexpr int kPhaseWarps = kPhaseBS / 32;

__device__ __forceinline__ int warp_id() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int warp_count() { return (gridDim.x * blockDim.x) >> 5; }

template <typename T, int BS>
__global__ void __launch_bounds__(kPhaseBS) k_ph_first(VLevel<T> L, const double* __restrict__ in) {
  phase_first<T, BS>(L, in, warp_id(), warp_count(), threadIdx.x & 31);
}

template <typename T, int BS>
__global__ void __launch_bounds__(kPhaseBS) k_ph_step(VLevel<T> L, int dc, int rc, int xc, T c1, T c2,
                                                     double* __restrict__ out) {
  phase_step<T, BS>(L, L.d[dc], L.d[1 - dc], L.r[rc], L.r[1 - rc], L.x[xc], c1, c2, out, warp_id(), warp_count(),
                    threadIdx.x & 31);
}

template <typename T, int BS>
__global__ void __launch_bounds__(kPhaseBS) k_ph_restrict(VLevel<T> L, VLevel<T> C, int dc, int rc) {
  phase_restrict<T, BS>(L, C, L.d[dc], L.r[rc], warp_id(), warp_count(), threadIdx.x & 31);
}

template <typename T>
__global__ void __launch_bounds__(kPhaseBS) k_ph_coarsest(VLevel<T> C) {
  const int lane = threadIdx.x & 31;
  for (int row = warp_id(); row < C.N; row += warp_count()) {
    const double* a = C.Ainv + (size_t)row * C.Np;
    double acc = 0.0;
    for (int j = lane; j < C.N; j += 32) acc += a[j] * (double)C.b[j];
    acc = warp_sum(acc);
    if (lane == 0) C.x[0][row] = (T)acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kPhaseBS) k_ph_prolong(VLevel<T> L, VLevel<T> C, int xl, int xcl) {
  const int bs = L.bs;
  T* x = L.x[xl];
  const T* xc = C.x[xcl];
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.n * bs; idx += gridDim.x * blockDim.x) {
    const int i = idx / bs, u = idx - i * bs;
    const T* Qi = L.Q + ((size_t)i * bs + u) * 16;
    const T* xa = xc + (size_t)L.agg[i] * 16;
    T acc = T(0);
#pragma unroll
    for (int s = 0; s < 16; ++s) acc += Qi[s] * xa[s];
    x[idx] += acc;
  }
}

template <typename T, int BS>
__global__ void __launch_bounds__(kPhaseBS) k_ph_post_first(VLevel<T> L, int xc, int rc, int dc,
                                                           double* __restrict__ out) {
  phase_post_first<T, BS>(L, L.x[xc], L.x[1 - xc], L.r[rc], L.d[dc], out, warp_id(), warp_count(),
                          threadIdx.x & 31);
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

// host-side Chebyshev coefficients of step k (the same recurrence as vc_rho)
static void cheb_coeffs(const Level& L, int k, double& c1, double& c2) {
  const double* ch = L.cheb_host;
  double rho = 1.0 / ch[2], rho_prev = 0.0;
  for (int j = 1; j <= k; ++j) {
    rho_prev = rho;
    rho = 1.0 / (2.0 * ch[2] - rho);
  }
  c1 = rho * rho_prev;
  c2 = 2.0 * rho / ch[1];
}

template <typename T>
static void run(ba_problem* P, const double* r, double* z) {
  const int nl = P->n_levels;
  const int pre = std::max(1, P->opt.pre_smooth), post = std::max(1, P->opt.post_smooth);
  std::vector<VLevel<T>> V(nl);
  for (int l = 0; l < nl; ++l) V[l] = describe<T>(P->levels[l]);
  unsigned xm = 0, rm = 0, dm = 0;
  auto bit = [](unsigned m, int l) { return (int)((m >> l) & 1u); };
  cudaStream_t st = P->stream;
  for (int l = 0; l + 1 < nl; ++l) {
    const VLevel<T>& L = V[l];
    const int g = warps_grid(L.n);
    if (L.bs == 9) k_ph_first<T, 9><<<g, kPhaseBS, 0, st>>>(L, l == 0 ? r : nullptr);
    else k_ph_first<T, 16><<<g, kPhaseBS, 0, st>>>(L, l == 0 ? r : nullptr);
    launched(P);
    for (int k = 1; k < pre; ++k) {
      double c1, c2;
      cheb_coeffs(P->levels[l], k, c1, c2);
      if (L.bs == 9)
        k_ph_step<T, 9><<<g, kPhaseBS, 0, st>>>(L, bit(dm, l), bit(rm, l), bit(xm, l), (T)c1, (T)c2, nullptr);
      else
        k_ph_step<T, 16><<<g, kPhaseBS, 0, st>>>(L, bit(dm, l), bit(rm, l), bit(xm, l), (T)c1, (T)c2, nullptr);
      launched(P);
      rm ^= 1u << l;
      dm ^= 1u << l;
    }
    const int gc = warps_grid(V[l + 1].n);
    if (L.bs == 9) k_ph_restrict<T, 9><<<gc, kPhaseBS, 0, st>>>(L, V[l + 1], bit(dm, l), bit(rm, l));
    else k_ph_restrict<T, 16><<<gc, kPhaseBS, 0, st>>>(L, V[l + 1], bit(dm, l), bit(rm, l));
    launched(P);
  }
  k_ph_coarsest<T><<<warps_grid(V[nl - 1].N), kPhaseBS, 0, st>>>(V[nl - 1]);
  launched(P);
  for (int l = nl - 2; l >= 0; --l) {
    const VLevel<T>& L = V[l];
    const int g = warps_grid(L.n);
    k_ph_prolong<T><<<cdiv((long long)L.n * L.bs, kPhaseBS), kPhaseBS, 0, st>>>(L, V[l + 1], bit(xm, l),
                                                                               bit(xm, l + 1));
    launched(P);
    double* o = (l == 0 && post == 1) ? z : nullptr;
    if (L.bs == 9) k_ph_post_first<T, 9><<<g, kPhaseBS, 0, st>>>(L, bit(xm, l), bit(rm, l), bit(dm, l), o);
    else k_ph_post_first<T, 16><<<g, kPhaseBS, 0, st>>>(L, bit(xm, l), bit(rm, l), bit(dm, l), o);
    launched(P);
    xm ^= 1u << l;
    for (int k = 1; k < post; ++k) {
      double c1, c2;
      cheb_coeffs(P->levels[l], k, c1, c2);
      double* ok = (l == 0 && k == post - 1) ? z : nullptr;
      if (L.bs == 9)
        k_ph_step<T, 9><<<g, kPhaseBS, 0, st>>>(L, bit(dm, l), bit(rm, l), bit(xm, l), (T)c1, (T)c2, ok);
      else
        k_ph_step<T, 16><<<g, kPhaseBS, 0, st>>>(L, bit(dm, l), bit(rm, l), bit(xm, l), (T)c1, (T)c2, ok);
      launched(P);
      rm ^= 1u << l;
      dm ^= 1u << l;
    }
  }
}

bool level_fp32(ba_problem* P);

// Called at the end of the multigrid setup: whether the fused-phase cycle applies.
void fused_vcycle_setup(ba_problem* P) {
  P->vc_ready = false;
  if (!P->opt.fused_vcycle || !P->l0_explicit || P->n_levels < 2) return;
  for (int l = 0; l + 1 < P->n_levels; ++l) {
    const int bs = P->levels[l].bs;
    if (bs != 9 && bs != 16) return;
  }
  P->vc_ready = true;
}

void fused_vcycle(ba_problem* P, const double* r, double* z) {
  if (level_fp32(P)) run<float>(P, r, z);
  else run<double>(P, r, z);
}

}  // namespace ba
