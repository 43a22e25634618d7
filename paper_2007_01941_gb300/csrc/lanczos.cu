// Lanczos estimate of lambda_max(D^-1 A) in the D-inner product (Section 3.4), for all
// assembled smoothed levels at once: each kernel of the recurrence covers the block rows
// of every level (one warp per block row, each CTA within one level), and the inner products are per-level
// deterministic grid reductions written straight into the level's Chebyshev buffer
// (alpha_j at slot 8 + j, beta_j at slot 16 + j).  The same recurrence, level by level,
// is the path of mg_setup.cu for an implicit level 0:
//   q_0 = v / |v|_D;  for j: Aq = A q_j, alpha_j = q_j^T A q_j,
//   w = D^-1 Aq - alpha_j q_j - beta_{j-1} q_{j-1},  beta_j = |w|_D,  q_{j+1} = w / beta_j.
// Scalings by 1/|.|_D are applied lazily by the kernel that next reads the vector, so a
// step is two launches for every level together.
#include <algorithm>

#include "ba_internal.h"
#include "device_util.cuh"

namespace ba {

constexpr int kLzMax = 16;
constexpr int kLzBS = 128;

template <typename T>
struct LzLevel {
  int n, bs, cta0, nct;   // rows, block size, first CTA of the level in the batched grid, its CTAs
  const int* row_ptr;
  const int* cols;
  const T* vals;
  const T* D;           // diagonal blocks [n][bs][bs] in the level's precision
  const T* Dinv;        // their inverses
  T* v;                 // start vector
  T* w;                 // unscaled next direction
  T* q[2];              // current / previous direction (by step parity)
  T* Aq;
  double* cheb;         // level buffer: [8 + j] alpha_j, [16 + j] beta_j
  double* s;            // [0] |v|_D^2, [1 + j] |w_j|_D^2
  double* partial;      // one slot per CTA of the level
  unsigned* counter;
};

template <typename T>
struct LzArgs {
  int nl;
  LzLevel<T> L[kLzMax];
};

// one warp per block row, kLzBS / 32 rows per CTA; every CTA holds rows of one level
constexpr int kLzRows = kLzBS / 32;

template <typename T>
__device__ __forceinline__ int lz_level(const LzArgs<T>& A, int b) {
  int l = 0;
  while (l + 1 < A.nl && A.L[l + 1].cta0 <= b) ++l;
  return l;
}

// CTA-wide sum of one value per thread (result valid in thread 0)
__device__ __forceinline__ double lz_block_sum(double v) {
  __shared__ double red[kLzBS / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kLzBS / 32; ++w) s += red[w];
  __syncthreads();
  return s;
}

// deterministic per-level sum: every CTA of the level stores its partial (thread 0's
// v), the last CTA to arrive adds them in a fixed order
__device__ __forceinline__ void lz_reduce(double v, double* partial, unsigned* counter, int n, int slot,
                                          double* out) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partial[slot] = v;
    __threadfence();
    last = atomicAdd(counter, 1u) == (unsigned)(n - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kLzBS) s += ((volatile double*)partial)[i];
    s = lz_block_sum(s);
    if (threadIdx.x == 0) {
      *out = s;
      *counter = 0u;
    }
  }
}

// (B x)_i row u for the warp's row i (lane u < bs), in the level's precision
template <typename T>
__device__ __forceinline__ T lz_block_row(const T* __restrict__ B, int bs, int i, const T* x, int u) {
  if (u >= bs) return T(0);
  const T* b = B + ((size_t)i * bs + u) * bs;
  const T* xi = x + (size_t)i * bs;
  T acc = T(0);
  for (int c = 0; c < bs; ++c) acc += b[c] * xi[c];
  return acc;
}

// (A x)_i row u for the warp's row i: lane u + bs h takes blocks h, h + G, ... (G = 32 / bs)
// and lane u < bs gets the row's sum
// lane (h, u) adds row u of blocks h, h + G, ... (G = 32 / BS groups); two blocks per
// iteration into independent sums, so that their loads are in flight together
template <typename T, int BS>
__device__ __forceinline__ T lz_row_product_bs(const LzLevel<T>& L, int i, const T* __restrict__ x, int lane) {
  constexpr int G = 32 / BS;
  const int u = lane % BS, h = lane / BS;
  T acc0 = T(0), acc1 = T(0);
  if (h < G) {
    const int e1 = L.row_ptr[i + 1];
    int e = L.row_ptr[i] + h;
    for (; e + G < e1; e += 2 * G) {
      const T* a = L.vals + (size_t)e * BS * BS + u * BS;
      const T* b = L.vals + (size_t)(e + G) * BS * BS + u * BS;
      const T* xa = x + (size_t)L.cols[e] * BS;
      const T* xb = x + (size_t)L.cols[e + G] * BS;
#pragma unroll
      for (int c = 0; c < BS; ++c) {
        acc0 += a[c] * xa[c];
        acc1 += b[c] * xb[c];
      }
    }
    if (e < e1) {
      const T* a = L.vals + (size_t)e * BS * BS + u * BS;
      const T* xa = x + (size_t)L.cols[e] * BS;
#pragma unroll
      for (int c = 0; c < BS; ++c) acc0 += a[c] * xa[c];
    }
  }
  const T acc = acc0 + acc1;
  // groups h = 1 .. G-1 to group 0 (lane u)
  T tot = acc;
#pragma unroll
  for (int g = 1; g < 32 / 9 + 1; ++g) {
    const int src = lane + g * BS;
    const T o = __shfl_sync(kFull, acc, src < 32 ? src : 31);
    if (g < G && src < G * BS) tot += o;
  }
  return tot;
}

template <typename T>
__device__ __forceinline__ T lz_row_product(const LzLevel<T>& L, int i, const T* __restrict__ x, int lane) {
  return L.bs == 9 ? lz_row_product_bs<T, 9>(L, i, x, lane) : lz_row_product_bs<T, 16>(L, i, x, lane);
}

// v = start vector (SplitMix64 of the level-local index, mapped to [-1, 1)); s[0] = v^T D v
template <typename T>
__global__ void __launch_bounds__(kLzBS) k_lz_init(LzArgs<T> A) {
  pdl_wait();
  pdl_trigger();
  const int l = lz_level(A, blockIdx.x);
  const LzLevel<T>& L = A.L[l];
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x - L.cta0) * kLzRows + (threadIdx.x >> 5), bs = L.bs;
  const bool live = i < L.n;
  if (live && lane < bs) {
    const size_t idx = (size_t)i * bs + lane;
    L.v[idx] = (T)(2.0 * ((double)(splitmix64(idx) >> 11) * 0x1.0p-53) - 1.0);
  }
  __syncwarp();
  double part = 0.0;
  if (live && lane < bs) part = (double)lz_block_row(L.D, bs, i, L.v, lane) * (double)L.v[(size_t)i * bs + lane];
  lz_reduce(lz_block_sum(part), L.partial, L.counter, L.nct, blockIdx.x - L.cta0, L.s);
}

// step j: q_j = src / sqrt(s[j]) (src = v for j = 0, w otherwise); Aq = A q_j; alpha_j
template <typename T>
__global__ void __launch_bounds__(kLzBS) k_lz_product(LzArgs<T> A, int j) {
  pdl_wait();
  pdl_trigger();
  const int l = lz_level(A, blockIdx.x);
  const LzLevel<T>& L = A.L[l];
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x - L.cta0) * kLzRows + (threadIdx.x >> 5), bs = L.bs;
  const bool live = i < L.n;
  const T* src = j == 0 ? L.v : L.w;
  const double scale = 1.0 / sqrt(L.s[j]);
  // the row's products in the level's precision (an estimate of lambda_max needs no
  // more; FP32 arithmetic also keeps this off the GPU's narrow FP64 unit)
  const T rowsum = live ? lz_row_product(L, i, src, lane) : T(0);
  double contrib = 0.0;
  if (live && lane < bs) {
    const size_t idx = (size_t)i * bs + lane;
    const double aq = (double)rowsum * scale;
    const double qv = (double)src[idx] * scale;
    L.Aq[idx] = (T)aq;
    L.q[j & 1][idx] = (T)qv;
    contrib = qv * aq;
  }
  lz_reduce(lz_block_sum(contrib), L.partial, L.counter, L.nct, blockIdx.x - L.cta0, L.cheb + 8 + j);
}

// w = D^-1 Aq - alpha_j q_j - beta_{j-1} q_{j-1}; s[j + 1] = w^T D w; beta_j = sqrt(s[j + 1])
template <typename T>
__global__ void __launch_bounds__(kLzBS) k_lz_direction(LzArgs<T> A, int j) {
  pdl_wait();
  pdl_trigger();
  const int l = lz_level(A, blockIdx.x);
  const LzLevel<T>& L = A.L[l];
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x - L.cta0) * kLzRows + (threadIdx.x >> 5), bs = L.bs;
  const bool live = i < L.n;
  const double alpha = L.cheb[8 + j];
  const double beta = j > 0 ? sqrt(L.s[j]) : 0.0;   // beta_{j-1} = |w_{j-1}|_D
  double wv = 0.0;
  if (live && lane < bs) {
    const size_t idx = (size_t)i * bs + lane;
    wv = (double)lz_block_row(L.Dinv, bs, i, L.Aq, lane);
    wv -= alpha * (double)L.q[j & 1][idx];
    if (j > 0) wv -= beta * (double)L.q[(j + 1) & 1][idx];
    L.w[idx] = (T)wv;
  }
  __syncwarp();
  double part = 0.0;
  if (live && lane < bs)
    part = (double)lz_block_row(L.D, bs, i, L.w, lane) * (double)L.w[(size_t)i * bs + lane];
  lz_reduce(lz_block_sum(part), L.partial, L.counter, L.nct, blockIdx.x - L.cta0, L.s + 1 + j);   // beta_j^2
}

__global__ void k_lz_betas(double* const* cheb, double* const* s, int nl, int m) {
  const int l = threadIdx.x;
  if (l >= nl) return;
  for (int j = 0; j + 1 < m; ++j) cheb[l][16 + j] = sqrt(s[l][1 + j]);
}

bool level_fp32(ba_problem* P);

// Lanczos for levels [first, last] of the hierarchy, all assembled.
template <typename T>
static void run(ba_problem* P, int first, int last) {
  const int nl = last - first + 1;
  const int m = std::min(std::max(P->opt.lanczos_steps, 1), 8);
  LzArgs<T> A{};
  A.nl = nl;
  size_t vec = 0;
  int ctas = 0;
  for (int k = 0; k < nl; ++k) {
    Level& L = P->levels[first + k];
    vec += (size_t)L.n * L.bs + 32;
    ctas += cdiv(L.n, kLzRows);
  }
  P->lz_vec.ensure(sizeof(T) * vec * 5 + 256);
  P->lz_red.ensure(sizeof(double) * ((size_t)ctas + 16 * (size_t)nl) + 256);
  P->lz_cnt.ensure(sizeof(unsigned) * (size_t)nl + 64);
  BA_CUDA(cudaMemsetAsync(P->lz_cnt.p, 0, sizeof(unsigned) * nl, P->stream));
  T* vb = P->lz_vec.as<T>();
  double* red = P->lz_red.as<double>();
  double* sbase = red + ctas;
  int cta0 = 0;
  for (int k = 0; k < nl; ++k) {
    Level& L = P->levels[first + k];
    L.cheb.ensure(sizeof(double) * kChebSlots);
    const size_t n = (size_t)L.n * L.bs;
    LzLevel<T>& d = A.L[k];
    BA_REQUIRE(L.bs == 9 || L.bs == 16, BA_ERR_STATE, "Lanczos: block size other than 9 or 16");
    d.n = L.n;
    d.bs = L.bs;
    d.cta0 = cta0;
    d.nct = cdiv(L.n, kLzRows);
    d.row_ptr = L.row_ptr.as<int>();
    d.cols = L.cols.as<int>();
    d.vals = sizeof(T) == 4 ? (const T*)L.vals32.p : (const T*)L.vals64.p;
    d.D = sizeof(T) == 4 ? (const T*)L.Dblk32.p : (const T*)L.Dblk.p;
    d.Dinv = sizeof(T) == 4 ? (const T*)L.Dinv32.p : (const T*)L.Dinv64.p;
    d.v = vb;
    d.w = vb + n;
    d.q[0] = vb + 2 * n;
    d.q[1] = vb + 3 * n;
    d.Aq = vb + 4 * n;
    vb += 5 * n + 32;
    d.cheb = L.cheb.as<double>();
    d.s = sbase + 16 * k;
    d.partial = red + cta0;
    d.counter = P->lz_cnt.as<unsigned>() + k;
    cta0 += d.nct;
  }
  // zero the alpha / beta slots so that unused ones read as 0
  for (int k = 0; k < nl; ++k)
    BA_CUDA(cudaMemsetAsync(A.L[k].cheb + 8, 0, sizeof(double) * 16, P->stream));
  launch_k(P, k_lz_init<T>, ctas, kLzBS, 0, A);
  for (int j = 0; j < m; ++j) {
    launch_k(P, k_lz_product<T>, ctas, kLzBS, 0, A, j);
    if (j == m - 1) break;
    launch_k(P, k_lz_direction<T>, ctas, kLzBS, 0, A, j);
  }
  // beta_j = sqrt(s[j + 1])
  std::vector<double*> hc(nl), hs(nl);
  for (int k = 0; k < nl; ++k) {
    hc[k] = A.L[k].cheb;
    hs[k] = A.L[k].s;
  }
  P->lz_ptr.ensure(sizeof(double*) * 2 * (size_t)nl + 64);
  BA_CUDA(cudaMemcpyAsync(P->lz_ptr.p, hc.data(), sizeof(double*) * nl, cudaMemcpyHostToDevice, P->stream));
  BA_CUDA(cudaMemcpyAsync((double**)P->lz_ptr.p + nl, hs.data(), sizeof(double*) * nl, cudaMemcpyHostToDevice,
                          P->stream));
  launch_k(P, k_lz_betas, 1, 32, 0, (double* const*)P->lz_ptr.p, (double* const*)((double**)P->lz_ptr.p + nl), nl,
           m);
}

void lanczos_batched(ba_problem* P, int first, int last) {
  if (last < first) return;
  BA_REQUIRE(last - first + 1 <= kLzMax, BA_ERR_LIMIT, "too many levels for the batched Lanczos");
  if (level_fp32(P)) run<float>(P, first, last);
  else run<double>(P, first, last);
}

}  // namespace ba
