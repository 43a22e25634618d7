// Multigrid setup of Section 3 on the GPU:
//   covisibility counts W = V^T V and the block pattern of S (K5),
//   strength-of-connection ordering (Section 3.2) and Algorithm 2 aggregation (K6),
//   near-nullspace (Section 3.1) and per-aggregate QR prolongators (Section 3.3, K7),
//   Galerkin coarse operators P^T A P (Section 2.3, K8),
//   block-Jacobi inverses (K4), Lanczos lambda_max (Section 3.4, K10) and the
//   coarsest direct solver (an explicit FP64 inverse, K12).
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <cmath>

#include "ba_internal.h"
#include "device_util.cuh"
#include "dfloat.cuh"

namespace cg = cooperative_groups;

namespace ba {

void block_inverse(ba_problem* P, const double* in, int n, int bs, double* out64, float* out32,
                   int flag_slot);
void block_inverse_batch(ba_problem* P, const BlockInvBatch& B, int bs, int flag_slot);
void level_matvec(ba_problem* P, int l, const void* x, void* y, bool ready);
bool level_fp32(ba_problem* P);

// ---------------------------------------------------------------------------
// exclusive scan of n ints (single CTA; n is at most a few million)
// ---------------------------------------------------------------------------
constexpr int kScanBS = 1024;
__global__ void __launch_bounds__(kScanBS) k_scan_exclusive(const int* __restrict__ in, int* __restrict__ out,
                                                            int n) {
  __shared__ int s[kScanBS];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += kScanBS) {
    const int i = base + threadIdx.x;
    const int v = (i < n) ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int d = 1; d < kScanBS; d <<= 1) {
      const int t = (threadIdx.x >= d) ? s[threadIdx.x - d] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < n) out[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == kScanBS - 1) carry += s[kScanBS - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

static int scan(ba_problem* P, const int* in, int* out, int n) {
  k_scan_exclusive<<<1, kScanBS, 0, P->stream>>>(in, out, n);
  launched(P);
  int total = 0;
  BA_CUDA(cudaMemcpyAsync(&total, out + n, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  sync(P);
  return total;
}

// ---------------------------------------------------------------------------
// Row-wise accumulation of (key, value) contributions in a shared-memory hash
// table; then the distinct keys of the row sorted ascending.  MODE 0: level 0,
// contributions of camera c are the cameras of every point c sees (value 1), plus
// the diagonal key.  MODE 1: coarse level, contributions of aggregate a are
// (agg[j], W_ij) for every entry (i, j) of every member i.
// ---------------------------------------------------------------------------
constexpr int kHashBS = 256;
constexpr int kEmpty = INT_MAX;

template <int MODE>
__global__ void __launch_bounds__(kHashBS)
k_row_hash(int n_rows, int H, const int* __restrict__ a_ptr, const int* __restrict__ a_list,
           const int* __restrict__ b_ptr, const int* __restrict__ b_idx, const int* __restrict__ map,
           const long long* __restrict__ Win, const int* __restrict__ out_ptr, int* __restrict__ out_cnt,
           int* __restrict__ out_cols, long long* __restrict__ out_W, int* flags) {
  extern __shared__ __align__(16) unsigned char hsm[];
  long long* hv = reinterpret_cast<long long*>(hsm);      // [H]
  int* hk = reinterpret_cast<int*>(hv + H);                 // [H]
  int* ck = hk + H;                                          // [H] slots of the distinct keys
  __shared__ int n_keys;
  __shared__ int overflow;
  const int row = blockIdx.x;
  if (row >= n_rows) return;
  for (int i = threadIdx.x; i < H; i += kHashBS) {
    hk[i] = kEmpty;
    hv[i] = 0;
  }
  if (threadIdx.x == 0) {
    n_keys = 0;
    overflow = 0;
  }
  __syncthreads();
  auto insert = [&](int key, long long val) {
    unsigned h = ((unsigned)key * 2654435761u) & (unsigned)(H - 1);
    for (int probe = 0; probe < H; ++probe) {
      const int prev = atomicCAS(hk + h, kEmpty, key);
      if (prev == kEmpty || prev == key) {
        atomicAdd(reinterpret_cast<unsigned long long*>(hv + h), (unsigned long long)val);
        return;
      }
      h = (h + 1) & (unsigned)(H - 1);
    }
    overflow = 1;
  };
  if (MODE == 0) {
    if (threadIdx.x == 0) insert(row, 0);
    // a_ptr/a_list: camera -> internal obs; b_ptr: point -> obs range; b_idx: obs -> point;
    // map: obs -> camera
    const int ab = a_ptr[row], ae = a_ptr[row + 1];
    for (int k = ab + (threadIdx.x >> 5); k < ae; k += kHashBS / 32) {
      const int o = a_list[k];
      const int ip = b_idx[o];
      for (int q = b_ptr[ip] + (threadIdx.x & 31); q < b_ptr[ip + 1]; q += 32) insert(map[q], 1);
    }
  } else {
    // a_ptr/a_list: members of aggregate; b_ptr/b_idx: BSR pattern of the fine level;
    // map: fine node -> aggregate; Win: fine W
    const int ab = a_ptr[row], ae = a_ptr[row + 1];
    for (int k = ab; k < ae; ++k) {
      const int i = a_list[k];
      for (int e = b_ptr[i] + threadIdx.x; e < b_ptr[i + 1]; e += kHashBS) insert(map[b_idx[e]], Win[e]);
    }
  }
  __syncthreads();
  if (overflow) {
    if (threadIdx.x == 0) flags[F_HASH_OVERFLOW] = 1;
    return;
  }
  // compact keys (order is fixed later by the sort)
  for (int i = threadIdx.x; i < H; i += kHashBS) {
    if (hk[i] != kEmpty) {
      const int pos = atomicAdd(&n_keys, 1);
      ck[pos] = i;  // slot index
    }
  }
  __syncthreads();
  const int nk = n_keys;
  int m = 1;
  while (m < nk) m <<= 1;
  // sort slot indices by key (bitonic, keys looked up through the slots)
  for (int i = nk + threadIdx.x; i < m; i += kHashBS) ck[i] = -1;
  __syncthreads();
  for (int size = 2; size <= m; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < m; i += kHashBS) {
        const int j = i ^ stride;
        if (j > i) {
          const int si = ck[i], sj = ck[j];
          const int ki = si < 0 ? INT_MAX : hk[si];
          const int kj = sj < 0 ? INT_MAX : hk[sj];
          const bool up = (i & size) == 0;
          if ((ki > kj) == up) {
            ck[i] = sj;
            ck[j] = si;
          }
        }
      }
      __syncthreads();
    }
  }
  if (out_cnt) {
    if (threadIdx.x == 0) out_cnt[row] = nk;
  } else {
    const int base = out_ptr[row];
    for (int i = threadIdx.x; i < nk; i += kHashBS) {
      out_cols[base + i] = hk[ck[i]];
      out_W[base + i] = hv[ck[i]];
    }
  }
}

static int hash_size(int bound) {
  int H = 64;
  while (H < 2 * bound && H < 8192) H <<= 1;
  return H;
}

static size_t hash_smem(int H) { return (size_t)H * (8 + 4 + 4); }

template <int MODE>
static void row_hash(ba_problem* P, int n_rows, int H, const int* a_ptr, const int* a_list,
                     const int* b_ptr, const int* b_idx, const int* map, const long long* Win,
                     Level& out) {
  const size_t smem = hash_smem(H);
  BA_CUDA(cudaFuncSetAttribute(k_row_hash<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // pass 1: counts
  P->scratch.ensure(sizeof(int) * ((size_t)n_rows + 1) * 2 + 64);
  int* cnt = P->scratch.as<int>();
  // (the flags are not cleared here: a setup whose check is deferred keeps its earlier
  // flags, which this check then raises)
  k_row_hash<MODE><<<n_rows, kHashBS, smem, P->stream>>>(n_rows, H, a_ptr, a_list, b_ptr, b_idx, map, Win,
                                                         nullptr, cnt, nullptr, nullptr, P->flags.as<int>());
  launched(P);
  check_flags(P);
  out.row_ptr.ensure(sizeof(int) * ((size_t)n_rows + 1));
  out.nnzb = scan(P, cnt, out.row_ptr.as<int>(), n_rows);
  out.cols.ensure(sizeof(int) * (size_t)std::max(out.nnzb, 1));
  out.W.ensure(sizeof(long long) * (size_t)std::max(out.nnzb, 1));
  k_row_hash<MODE><<<n_rows, kHashBS, smem, P->stream>>>(n_rows, H, a_ptr, a_list, b_ptr, b_idx, map, Win,
                                                         out.row_ptr.as<int>(), nullptr, out.cols.as<int>(),
                                                         out.W.as<long long>(), P->flags.as<int>());
  launched(P);
  check_flags(P);
}

// Partitioned solve: W = V^T V of the whole problem from its observation graph (host,
// global point ids), by a sparse accumulator per camera row; every rank builds the same.
static void covisibility_level0_host(ba_problem* P, Level& L) {
  const int n_c = P->n_c;
  const size_t n_o = P->part_cam.size();
  int n_pts = 0;
  for (size_t o = 0; o < n_o; ++o) n_pts = std::max(n_pts, P->part_pt[o] + 1);
  std::vector<int> pptr(n_pts + 1, 0), cptr(n_c + 1, 0);
  for (size_t o = 0; o < n_o; ++o) {
    ++pptr[P->part_pt[o] + 1];
    ++cptr[P->part_cam[o] + 1];
  }
  for (int p = 0; p < n_pts; ++p) pptr[p + 1] += pptr[p];
  for (int c = 0; c < n_c; ++c) cptr[c + 1] += cptr[c];
  std::vector<int> pcam(std::max<size_t>(n_o, 1)), cpt(std::max<size_t>(n_o, 1));
  {
    std::vector<int> pf(pptr.begin(), pptr.end() - 1), cf(cptr.begin(), cptr.end() - 1);
    for (size_t o = 0; o < n_o; ++o) {
      pcam[pf[P->part_pt[o]]++] = P->part_cam[o];
      cpt[cf[P->part_cam[o]]++] = P->part_pt[o];
    }
  }
  std::vector<long long> acc(n_c, 0);
  std::vector<int> touched, rp(n_c + 1, 0), cols;
  std::vector<long long> W;
  for (int c = 0; c < n_c; ++c) {
    touched.clear();
    for (int k = cptr[c]; k < cptr[c + 1]; ++k) {
      const int p = cpt[k];
      for (int q = pptr[p]; q < pptr[p + 1]; ++q) {
        const int c2 = pcam[q];
        if (acc[c2]++ == 0) touched.push_back(c2);
      }
    }
    std::sort(touched.begin(), touched.end());
    for (int c2 : touched) {
      // a point seen twice by camera c counts twice on the diagonal: duplicates are invalid
      BA_REQUIRE(c2 != c || acc[c2] == cptr[c + 1] - cptr[c], BA_ERR_INVALID_ARG,
                 "duplicate (camera, point) pair in the partition's observation graph");
      cols.push_back(c2);
      W.push_back(acc[c2]);
      acc[c2] = 0;
    }
    rp[c + 1] = (int)cols.size();
  }
  L.nnzb = (int)cols.size();
  L.row_ptr.ensure(sizeof(int) * ((size_t)n_c + 1));
  L.cols.ensure(sizeof(int) * (size_t)std::max(L.nnzb, 1));
  L.W.ensure(sizeof(long long) * (size_t)std::max(L.nnzb, 1));
  BA_CUDA(cudaMemcpyAsync(L.row_ptr.p, rp.data(), sizeof(int) * (n_c + 1), cudaMemcpyHostToDevice, P->stream));
  if (L.nnzb) {
    BA_CUDA(cudaMemcpyAsync(L.cols.p, cols.data(), sizeof(int) * L.nnzb, cudaMemcpyHostToDevice, P->stream));
    BA_CUDA(cudaMemcpyAsync(L.W.p, W.data(), sizeof(long long) * L.nnzb, cudaMemcpyHostToDevice, P->stream));
  }
  sync(P);
}

void covisibility_level0(ba_problem* P, Level& L) {
  L.n = P->n_c;
  L.bs = 9;
  if (partitioned(P)) {
    covisibility_level0_host(P, L);
    return;
  }
  const int H = hash_size(std::min(P->n_c, std::max(P->max_row_contrib, 1)));
  row_hash<0>(P, P->n_c, H, P->cam_ptr.as<int>(), P->cam_obs.as<int>(), P->pt_ptr.as<int>(),
              P->obs_pt.as<int>(), P->obs_cam.as<int>(), nullptr, L);
}

// ---------------------------------------------------------------------------
// strength ordering: neighbours j != i by decreasing W_ij / sqrt(W_jj) (the
// common factor sqrt(W_ii) does not change the order), compared exactly as
// W_ij^2 W_kk > W_ik^2 W_jj in 128-bit integers; ties to the smaller index.
// ---------------------------------------------------------------------------
__global__ void k_diag_w(int n, const int* __restrict__ row_ptr, const int* __restrict__ cols,
                         const long long* __restrict__ W, long long* __restrict__ Wd) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long d = 0;
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
    if (cols[e] == i) d = W[e];
  Wd[i] = d;
}

struct StrengthKey {
  int j;
  long long w;   // W_ij
  long long wd;  // W_jj
};

__device__ __forceinline__ bool stronger(const StrengthKey& a, const StrengthKey& b) {
  // true if a precedes b
  const unsigned __int128 lhs = (unsigned __int128)((unsigned long long)a.w * (unsigned long long)a.w) *
                                (unsigned long long)b.wd;
  const unsigned __int128 rhs = (unsigned __int128)((unsigned long long)b.w * (unsigned long long)b.w) *
                                (unsigned long long)a.wd;
  if (lhs != rhs) return lhs > rhs;
  return a.j < b.j;
}

constexpr int kStrBS = 128;
__global__ void __launch_bounds__(kStrBS)
k_strength_order(int n, const int* __restrict__ row_ptr, const int* __restrict__ cols,
                 const long long* __restrict__ W, const long long* __restrict__ Wd,
                 int* __restrict__ sptr_out, int* __restrict__ sidx) {
  extern __shared__ __align__(16) unsigned char ssm[];
  StrengthKey* keys = reinterpret_cast<StrengthKey*>(ssm);
  __shared__ int cnt;
  const int i = blockIdx.x;
  const int rb = row_ptr[i], re = row_ptr[i + 1];
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int m = 1;
  while (m < re - rb) m <<= 1;
  for (int e = rb + threadIdx.x; e < re; e += kStrBS) {
    const int j = cols[e];
    if (j != i && W[e] > 0) {
      const int pos = atomicAdd(&cnt, 1);
      keys[pos] = StrengthKey{j, W[e], Wd[j]};
    }
  }
  __syncthreads();
  const int nk = cnt;
  for (int k = nk + threadIdx.x; k < m; k += kStrBS) keys[k] = StrengthKey{INT_MAX, 0, 1};
  __syncthreads();
  for (int size = 2; size <= m; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int a = threadIdx.x; a < m; a += kStrBS) {
        const int b = a ^ stride;
        if (b > a) {
          const StrengthKey ka = keys[a], kb = keys[b];
          const bool up = (a & size) == 0;
          // padding (j == INT_MAX) always sorts last
          bool a_first;
          if (ka.j == INT_MAX) a_first = false;
          else if (kb.j == INT_MAX) a_first = true;
          else a_first = stronger(ka, kb);
          if (a_first != up) {
            keys[a] = kb;
            keys[b] = ka;
          }
        }
      }
      __syncthreads();
    }
  }
  const int base = sptr_out[i];
  for (int k = threadIdx.x; k < nk; k += kStrBS) sidx[base + k] = keys[k].j;
}

__global__ void k_strength_count(int n, const int* __restrict__ row_ptr, const int* __restrict__ cols,
                                 const long long* __restrict__ W, int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = 0;
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) c += (cols[e] != i && W[e] > 0);
  cnt[i] = c;
}

// ---------------------------------------------------------------------------
// Algorithm 2 (sequential greedy pass; one thread, state in shared memory when it
// fits).  A node left unaggregated becomes a singleton aggregate afterwards.
// ---------------------------------------------------------------------------
// Two warps: warp 1 prefetches, for the next 32 nodes, the bounds of their strength
// lists and their strongest neighbour into shared memory while lane 0 of warp 0 runs
// the greedy pass over the current 32 nodes (further neighbours, rarely needed, are
// read from global memory).
template <bool SMEM>
__global__ void __launch_bounds__(64) k_aggregate(int n, const int* __restrict__ sptr, const int* __restrict__ sidx,
                                                  int max_agg, int* __restrict__ agg_out, int* __restrict__ gsize,
                                                  int* __restrict__ n_agg_out) {
  extern __shared__ __align__(16) unsigned char asm_[];
  __shared__ int pb[2][32], pe[2][32], pf[2][32];
  int* agg = SMEM ? reinterpret_cast<int*>(asm_) : agg_out;
  int* size = SMEM ? (agg + n) : gsize;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    agg[i] = -1;
    size[i] = 0;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto prefetch = [&](int chunk) {
    const int i = chunk * 32 + lane;
    int b = 0, e = 0, f = -1;
    if (i < n) {
      b = sptr[i];
      e = sptr[i + 1];
      if (b < e) f = __ldg(sidx + b);
    }
    pb[chunk & 1][lane] = b;
    pe[chunk & 1][lane] = e;
    pf[chunk & 1][lane] = f;
  };
  if (warp == 1) prefetch(0);
  __syncthreads();
  const int nchunks = (n + 31) / 32;
  int na = 0;
  for (int c = 0; c < nchunks; ++c) {
    if (warp == 1 && c + 1 < nchunks) prefetch(c + 1);
    if (threadIdx.x == 0) {
      const int buf = c & 1;
      for (int k = 0; k < 32; ++k) {
        const int i = c * 32 + k;
        if (i >= n) break;
        if (agg[i] >= 0) continue;
        const int e1 = pe[buf][k];
        for (int e = pb[buf][k]; e < e1; ++e) {
          const int j = (e == pb[buf][k]) ? pf[buf][k] : __ldg(sidx + e);
          const int a = agg[j];
          if (a < 0) {
            agg[i] = na;
            agg[j] = na;
            size[na] = 2;
            ++na;
            break;
          }
          if (size[a] < max_agg) {
            agg[i] = a;
            size[a] += 1;
            break;
          }
        }
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i)
      if (agg[i] < 0) agg[i] = na++;
    *n_agg_out = na;
  }
  __syncthreads();
  if (SMEM)
    for (int i = threadIdx.x; i < n; i += blockDim.x) agg_out[i] = agg[i];
}

__global__ void k_count_members(int n, const int* __restrict__ agg, int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(cnt + agg[i], 1);
}

__global__ void k_fill_members(int n, const int* __restrict__ agg, const int* __restrict__ ptr,
                               int* __restrict__ fill, int* __restrict__ mem) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int a = agg[i];
    mem[ptr[a] + atomicAdd(fill + a, 1)] = i;
  }
}

__global__ void k_sort_members(int n_agg, const int* __restrict__ ptr, int* __restrict__ mem) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_agg) return;
  const int b = ptr[a], e = ptr[a + 1];
  for (int i = b + 1; i < e; ++i) {
    const int v = mem[i];
    int j = i - 1;
    while (j >= b && mem[j] > v) {
      mem[j + 1] = mem[j];
      --j;
    }
    mem[j + 1] = v;
  }
}

// ---------------------------------------------------------------------------
// near-nullspace of level 0 (Section 3.1): per camera, 9 x 16 rows
//   translation e_k: dt = -R e_k;  rotation e_k: dr = -J_l(r)^-1 R e_k;  scale: dt = t;
//   then the 9 per-parameter constant columns.
// J_l^-1 = I - 1/2 [r]_x + (1/th^2 - (1 + cos th) / (2 th sin th)) [r]_x^2 (1/12 for th < 1e-6).
// ---------------------------------------------------------------------------
__global__ void k_nullspace0(const double* __restrict__ cams, int n_c, double* __restrict__ K) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_c) return;
  const double* cam = cams + 9 * c;
  const double r0 = cam[0], r1 = cam[1], r2 = cam[2];
  const double th2 = r0 * r0 + r1 * r1 + r2 * r2;
  const double Km[9] = {0.0, -r2, r1, r2, 0.0, -r0, -r1, r0, 0.0};
  double K2[9];
  const double rv[3] = {r0, r1, r2};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K2[3 * i + j] = rv[i] * rv[j] - (i == j ? th2 : 0.0);
  double R[9], Jli[9];
  // one sine and cosine serve R and J_l^-1 (the FP64 unit bounds this kernel)
  const double th = sqrt(th2);
  double s = 0.0, co = 1.0;
  if (th2 >= 1e-16) sincos(th, &s, &co);
  if (th2 < 1e-16) {
    for (int i = 0; i < 9; ++i) R[i] = ((i % 4 == 0) ? 1.0 : 0.0) + Km[i];
  } else {
    for (int i = 0; i < 9; ++i) R[i] = ((i % 4 == 0) ? 1.0 : 0.0) + s / th * Km[i] + (1.0 - co) / th2 * K2[i];
  }
  double coef;
  if (th < 1e-6) {
    coef = 1.0 / 12.0;
  } else {
    coef = 1.0 / th2 - (1.0 + co) / (2.0 * th * s);
  }
  for (int i = 0; i < 9; ++i) Jli[i] = ((i % 4 == 0) ? 1.0 : 0.0) - 0.5 * Km[i] + coef * K2[i];
  double* out = K + (size_t)c * 9 * kNull;
  for (int i = 0; i < 9 * kNull; ++i) out[i] = 0.0;
  for (int k = 0; k < 3; ++k) {
    // translation: rows 3..5 of column k = -R e_k
    for (int i = 0; i < 3; ++i) out[(3 + i) * kNull + k] = -R[3 * i + k];
    // rotation: rows 0..2 of column 3+k = -J_l^-1 R e_k
    for (int i = 0; i < 3; ++i) {
      double v = 0.0;
      for (int m = 0; m < 3; ++m) v += Jli[3 * i + m] * R[3 * m + k];
      out[i * kNull + 3 + k] = -v;
    }
  }
  for (int i = 0; i < 3; ++i) out[(3 + i) * kNull + 6] = cam[3 + i];
  for (int i = 0; i < 9; ++i) out[i * kNull + 7 + i] = 1.0;
}

// ---------------------------------------------------------------------------
// per-aggregate thin QR (Section 3.3) by Gram-Schmidt with one re-orthogonalisation
// pass; a column whose remaining norm is <= 1e-10 of its original norm is dropped
// (zero Q column, zero R row).  One warp per aggregate (four per CTA), rows spread over
// the lanes.  Each pass projects column j on all earlier columns at once (classical
// Gram-Schmidt: the j inner products come out of one 16-value warp reduction, so the
// dependency chain per column is two reductions long instead of 2j); with the second
// pass this is as accurate as the modified variant with re-orthogonalisation.  FP64
// throughput per SM is what limits this kernel, so no warp works on an empty share.
// ---------------------------------------------------------------------------
// row stride of the aggregate matrix in shared memory: 17 doubles, so the rows that
// consecutive threads touch fall in different banks
constexpr int kQrStride = kNull + 1;

// sums over the warp of p[0..15] (16 values per lane), into every lane's h[0..15]: each
// step halves the values a lane carries (it keeps one half and adds its partner's copy
// of that half), so the 16 sums take 15 shuffles; 16 more broadcast them.
__device__ __forceinline__ void qr_warp_sum16(double p[kNull], double h[kNull], int lane) {
#pragma unroll
  for (int half = 8, off = 16; half >= 1; half >>= 1, off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const double send = up ? p[k] : p[k + half];
      const double keep = up ? p[k + half] : p[k];
      p[k] = keep + __shfl_xor_sync(kFull, send, off);
    }
  }
  // p[0] holds the partial of index idx(lane); lanes l and l ^ 1 hold the same index
  const double v = p[0] + __shfl_xor_sync(kFull, p[0], 1);
#pragma unroll
  for (int i = 0; i < kNull; ++i) {
    // lane holding index i: bits 4..1 of the lane are the bits 3..0 of i
    const int src = ((i >> 3) & 1) << 4 | ((i >> 2) & 1) << 3 | ((i >> 1) & 1) << 2 | (i & 1) << 1;
    h[i] = __shfl_sync(kFull, v, src);
  }
}

constexpr int kQrWarps = 4;   // aggregates per CTA (one warp each)

__global__ void __launch_bounds__(kQrWarps * 32)
k_aggregate_qr(int n_agg, int bs, int max_rows, const int* __restrict__ mptr, const int* __restrict__ mem,
               const double* __restrict__ K, double* __restrict__ Q64, float* __restrict__ Q32,
               double* __restrict__ Kc, unsigned* __restrict__ kept_out) {
  extern __shared__ __align__(16) unsigned char qsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int a = blockIdx.x * kQrWarps + warp;
  if (a >= n_agg) return;
  double* A = reinterpret_cast<double*>(qsm) + (size_t)warp * max_rows * kQrStride;  // [rows][kQrStride]
  const int mb = mptr[a], me = mptr[a + 1];
  const int rows = (me - mb) * bs;
  for (int e = lane; e < rows * kNull; e += 32) {
    const int r = e / kNull, j = e - r * kNull;
    const int s = r / bs, u = r - s * bs;
    A[r * kQrStride + j] = K[((size_t)mem[mb + s] * bs + u) * kNull + j];
  }
  __shared__ double Rs[kQrWarps][kNull][kNull + 1];
  double(*R)[kNull + 1] = Rs[warp];
  for (int e = lane; e < kNull * kNull; e += 32) R[e / kNull][e % kNull] = 0.0;
  __syncwarp();
  unsigned kept = 0;
  for (int j = 0; j < kNull; ++j) {
    double n2 = 0.0;
    for (int r = lane; r < rows; r += 32) n2 += A[r * kQrStride + j] * A[r * kQrStride + j];
    const double n0 = sqrt(warp_sum(n2));
    double rc[kNull];
#pragma unroll
    for (int i = 0; i < kNull; ++i) rc[i] = 0.0;
    if (j > 0) {
      for (int pass = 0; pass < 2; ++pass) {
        double p[kNull], h[kNull];
#pragma unroll
        for (int i = 0; i < kNull; ++i) p[i] = 0.0;
        for (int r = lane; r < rows; r += 32) {
          const double aj = A[r * kQrStride + j];
#pragma unroll
          for (int i = 0; i < kNull; ++i)
            if (i < j) p[i] += A[r * kQrStride + i] * aj;
        }
        qr_warp_sum16(p, h, lane);
        for (int r = lane; r < rows; r += 32) {
          double aj = A[r * kQrStride + j];
#pragma unroll
          for (int i = 0; i < kNull; ++i)
            if (i < j) aj -= h[i] * A[r * kQrStride + i];
          A[r * kQrStride + j] = aj;
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < kNull; ++i)
          if (i < j) rc[i] += h[i];
      }
    }
    double v2 = 0.0;
    for (int r = lane; r < rows; r += 32) v2 += A[r * kQrStride + j] * A[r * kQrStride + j];
    const double nv = sqrt(warp_sum(v2));
    const bool keep = n0 > 0.0 && nv > 1e-10 * n0;
    const double scale = keep ? 1.0 / nv : 0.0;
    for (int r = lane; r < rows; r += 32) A[r * kQrStride + j] *= scale;
    __syncwarp();
    if (keep) kept |= 1u << j;
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < kNull; ++i)
        if (i < j) R[i][j] = rc[i];
      R[j][j] = keep ? nv : 0.0;
    }
  }
  __syncwarp();
  // Q blocks back to the member nodes
  for (int e = lane; e < rows * kNull; e += 32) {
    const int r = e / kNull, j = e - r * kNull;
    const int s = r / bs, u = r - s * bs;
    const size_t dst = ((size_t)mem[mb + s] * bs + u) * kNull + j;
    const double q = A[r * kQrStride + j];
    Q64[dst] = q;
    Q32[dst] = (float)q;
  }
  for (int e = lane; e < kNull * kNull; e += 32) Kc[(size_t)a * kNull * kNull + e] = R[e / kNull][e % kNull];
  if (lane == 0) kept_out[a] = kept;
}

// The same factorisation in paired FP32 (DF) for the mixed-precision hierarchy (the FP64
// unit of this GPU issues a warp's FMA over many cycles per SM sub-partition, DF runs on
// the FP32 pipes), with one CTA of kQrDfBS threads per aggregate: the inner products
// of a pass are split over the CTA (thread i + 16 k: column i, rows k, k + 8, ...), the
// projection over rows (one row per thread), so the dependency chain of a column is a few
// block reductions long instead of one warp's walk over all rows.
constexpr int kQrDfBS = 128;
constexpr int kQrDfParts = kQrDfBS / 16;

// sum over the CTA of one DF value per thread; every thread gets the total
__device__ __forceinline__ DF qr_block_sum_df(DF v, float2* red /*[kQrDfBS / 32]*/) {
  v = warp_sum_df(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = make_float2(v.h, v.l);
  __syncthreads();
  DF s(0.f, 0.f);
#pragma unroll
  for (int w = 0; w < kQrDfBS / 32; ++w) s += DF(red[w].x, red[w].y);
  return s;
}

__global__ void __launch_bounds__(kQrDfBS)
k_aggregate_qr_df_cta(int n_agg, int bs, const int* __restrict__ mptr, const int* __restrict__ mem,
                      const double* __restrict__ K, double* __restrict__ Q64, float* __restrict__ Q32,
                      double* __restrict__ Kc, unsigned* __restrict__ kept_out) {
  extern __shared__ __align__(16) unsigned char qsm[];
  float2* A = reinterpret_cast<float2*>(qsm);  // [rows][kQrStride]
  __shared__ float2 R[kNull][kNull + 1];
  __shared__ float2 gpart[kQrDfParts / 2][kNull];   // per-warp partial inner products
  __shared__ float2 g[kNull];
  __shared__ float2 red[kQrDfBS / 32];
  __shared__ float2 n0s[kNull];
  const int a = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int mb = mptr[a], me = mptr[a + 1];
  const int rows = (me - mb) * bs;
  for (int e = t; e < rows * kNull; e += kQrDfBS) {
    const int r = e / kNull, j = e - r * kNull;
    const int s = r / bs, u = r - s * bs;
    const DF v(K[((size_t)mem[mb + s] * bs + u) * kNull + j]);
    A[r * kQrStride + j] = make_float2(v.h, v.l);
  }
  for (int e = t; e < kNull * kNull; e += kQrDfBS) R[e / kNull][e % kNull] = make_float2(0.f, 0.f);
  __syncthreads();
  auto at = [&](int r, int j) {
    const float2 v = A[r * kQrStride + j];
    return DF(v.x, v.y);
  };
  const int gi = t & 15, part = t >> 4;   // part = 2 warp + (lane >> 4)
  // the rank test's reference: every column's norm before orthogonalisation, at once
  {
    float s = 0.f, c = 0.f;
    for (int r = part; r < rows; r += kQrDfParts) {
      const DF v = at(r, gi);
      dot2_fma(s, c, v, v);
    }
    DF nv = DF(s, 0.f) + DF(c, 0.f);
    nv += DF(__shfl_xor_sync(kFull, nv.h, 16), __shfl_xor_sync(kFull, nv.l, 16));
    if (lane < 16) gpart[warp][lane] = make_float2(nv.h, nv.l);
    __syncthreads();
    if (t < kNull) {
      DF tot(0.f, 0.f);
#pragma unroll
      for (int w = 0; w < kQrDfParts / 2; ++w) tot += DF(gpart[w][t].x, gpart[w][t].y);
      const DF n = df_sqrt(tot);
      n0s[t] = make_float2(n.h, n.l);
    }
    __syncthreads();
  }
  unsigned kept = 0;
  DF rc(0.f, 0.f);   // threads t < 16: R[t][j] of the current column
  for (int j = 0; j < kNull; ++j) {
    const DF n0(n0s[j].x, n0s[j].y);
    DF nv = n0;
    rc = DF(0.f, 0.f);
    if (j > 0) {
      for (int pass = 0; pass < 2; ++pass) {
        // g_i = A[:, i] . A[:, j] for i < j
        float s = 0.f, c = 0.f;
        if (gi < j) {
#pragma unroll 2
          for (int r = part; r < rows; r += kQrDfParts) dot2_fma(s, c, at(r, gi), at(r, j));
        }
        DF gv = DF(s, 0.f) + DF(c, 0.f);
        gv += DF(__shfl_xor_sync(kFull, gv.h, 16), __shfl_xor_sync(kFull, gv.l, 16));
        if (lane < 16) gpart[warp][lane] = make_float2(gv.h, gv.l);
        __syncthreads();
        if (t < kNull) {
          DF tot(0.f, 0.f);
#pragma unroll
          for (int w = 0; w < kQrDfParts / 2; ++w) tot += DF(gpart[w][t].x, gpart[w][t].y);
          if (t >= j) tot = DF(0.f, 0.f);
          g[t] = make_float2(tot.h, tot.l);
          rc += tot;
        }
        __syncthreads();
        // A[:, j] -= sum_{i<j} g_i A[:, i]; the second pass also sums the new column's
        // squares, and the reduction's first barrier orders the column's writes
        float ns = 0.f, nc = 0.f;
        for (int r = t; r < rows; r += kQrDfBS) {
          float ps = 0.f, pc = 0.f;
#pragma unroll 4
          for (int i = 0; i < j; ++i) dot2_fma(ps, pc, g[i], A[r * kQrStride + i]);
          const DF v = at(r, j) - (DF(ps, 0.f) + DF(pc, 0.f));
          A[r * kQrStride + j] = make_float2(v.h, v.l);
          dot2_fma(ns, nc, v, v);
        }
        if (pass == 0) __syncthreads();
        else nv = df_sqrt(qr_block_sum_df(DF(ns, 0.f) + DF(nc, 0.f), red));
      }
    }
    const bool keep = n0.h > 0.f && nv.h > 1e-10f * n0.h;
    const DF scale = keep ? DF(1.f, 0.f) / nv : DF(0.f, 0.f);
    for (int r = t; r < rows; r += kQrDfBS) {
      const DF v = at(r, j) * scale;
      A[r * kQrStride + j] = make_float2(v.h, v.l);
    }
    if (keep) kept |= 1u << j;
    if (t < j) R[t][j] = make_float2(rc.h, rc.l);
    if (t == 0) R[j][j] = keep ? make_float2(nv.h, nv.l) : make_float2(0.f, 0.f);
    __syncthreads();
  }
  // Q blocks back to the member nodes
  for (int e = t; e < rows * kNull; e += kQrDfBS) {
    const int r = e / kNull, j = e - r * kNull;
    const int s = r / bs, u = r - s * bs;
    const size_t dst = ((size_t)mem[mb + s] * bs + u) * kNull + j;
    const DF q = at(r, j);
    Q64[dst] = to_double(q);
    Q32[dst] = q.h;
  }
  for (int e = t; e < kNull * kNull; e += kQrDfBS) {
    const float2 v = R[e / kNull][e % kNull];
    Kc[(size_t)a * kNull * kNull + e] = to_double(DF(v.x, v.y));
  }
  if (t == 0) kept_out[a] = kept;
}

// The same factorisation with one CTA of kQrBS threads per aggregate, rows spread over
// the threads: shorter dependency chains for the few large aggregates of the coarse
// levels, where there are too few aggregates to fill the GPU with warps.
constexpr int kQrBS = 128;
constexpr int kQrCtaWarps = kQrBS / 32;

// sqrt of the sum over the CTA of v (one value per thread); result in every thread.
// The square root runs once (thread 0): FP64 square roots and divisions are long
// sequences on this GPU's narrow FP64 unit, which all CTAs of an SM share.
__device__ __forceinline__ double qr_block_norm(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kQrCtaWarps; ++w) s += red[w];
    red[kQrCtaWarps * kNull] = sqrt(s);
  }
  __syncthreads();
  return red[kQrCtaWarps * kNull];
}

// sums over the CTA of p[0..15] (16 values per thread); h[0..15] in shared memory on
// return.  Within a warp, each step halves the values a lane carries (it keeps one half
// and adds its partner's copy of that half), so the 16 sums take 15 shuffles.
__device__ __forceinline__ void qr_block_sum16(double p[kNull], double* red /*[kQrCtaWarps][16]*/, double* h) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int half = 8, off = 16; half >= 1; half >>= 1, off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const double send = up ? p[k] : p[k + half];
      const double keep = up ? p[k + half] : p[k];
      p[k] = keep + __shfl_xor_sync(kFull, send, off);
    }
  }
  // p[0] now holds the warp's partial of index idx; lanes l and l ^ 1 hold the same index
  const double v = p[0] + __shfl_xor_sync(kFull, p[0], 1);
  const int idx = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
  __syncthreads();
  if ((lane & 1) == 0) red[warp * kNull + idx] = v;
  __syncthreads();
  if (threadIdx.x < kNull) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kQrCtaWarps; ++w) s += red[w * kNull + threadIdx.x];
    h[threadIdx.x] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kQrBS)
k_aggregate_qr_cta(int n_agg, int bs, const int* __restrict__ mptr, const int* __restrict__ mem,
               const double* __restrict__ K, double* __restrict__ Q64, float* __restrict__ Q32,
               double* __restrict__ Kc, unsigned* __restrict__ kept_out) {
  extern __shared__ __align__(16) unsigned char qsm[];
  double* A = reinterpret_cast<double*>(qsm);  // [rows][kQrStride]
  __shared__ double red[kQrCtaWarps * kNull + 2];
  __shared__ double h[kNull];
  __shared__ double Rs[kNull][kNull + 1];
  const int a = blockIdx.x;
  const int t = threadIdx.x;
  const int mb = mptr[a], me = mptr[a + 1];
  const int rows = (me - mb) * bs;
  for (int e = t; e < rows * kNull; e += kQrBS) {
    const int r = e / kNull, j = e - r * kNull;
    const int s = r / bs, u = r - s * bs;
    A[r * kQrStride + j] = K[((size_t)mem[mb + s] * bs + u) * kNull + j];
  }
  for (int e = t; e < kNull * kNull; e += kQrBS) Rs[e / kNull][e % kNull] = 0.0;
  __syncthreads();
  unsigned kept = 0;
  for (int j = 0; j < kNull; ++j) {
    double n2 = 0.0;
    for (int r = t; r < rows; r += kQrBS) n2 += A[r * kQrStride + j] * A[r * kQrStride + j];
    const double n0 = qr_block_norm(n2, red);
    double rc[kNull];
#pragma unroll
    for (int i = 0; i < kNull; ++i) rc[i] = 0.0;
    if (j > 0) {
      for (int pass = 0; pass < 2; ++pass) {
        double p[kNull];
#pragma unroll
        for (int i = 0; i < kNull; ++i) p[i] = 0.0;
        for (int r = t; r < rows; r += kQrBS) {
          const double aj = A[r * kQrStride + j];
#pragma unroll
          for (int i = 0; i < kNull; ++i)
            if (i < j) p[i] += A[r * kQrStride + i] * aj;
        }
        qr_block_sum16(p, red, h);
        for (int r = t; r < rows; r += kQrBS) {
          double aj = A[r * kQrStride + j];
#pragma unroll
          for (int i = 0; i < kNull; ++i)
            if (i < j) aj -= h[i] * A[r * kQrStride + i];
          A[r * kQrStride + j] = aj;
        }
#pragma unroll
        for (int i = 0; i < kNull; ++i)
          if (i < j) rc[i] += h[i];
        __syncthreads();
      }
    }
    double v2 = 0.0;
    for (int r = t; r < rows; r += kQrBS) v2 += A[r * kQrStride + j] * A[r * kQrStride + j];
    const double nv = qr_block_norm(v2, red);
    const bool keep = n0 > 0.0 && nv > 1e-10 * n0;
    if (threadIdx.x == 0) red[kQrCtaWarps * kNull + 1] = keep ? 1.0 / nv : 0.0;
    __syncthreads();
    const double scale = red[kQrCtaWarps * kNull + 1];
    for (int r = t; r < rows; r += kQrBS) A[r * kQrStride + j] *= scale;
    if (keep) kept |= 1u << j;
    if (t == 0) {
#pragma unroll
      for (int i = 0; i < kNull; ++i)
        if (i < j) Rs[i][j] = rc[i];
      Rs[j][j] = keep ? nv : 0.0;
    }
    __syncthreads();
  }
  // Q blocks back to the member nodes
  for (int e = t; e < rows * kNull; e += kQrBS) {
    const int r = e / kNull, j = e - r * kNull;
    const int s = r / bs, u = r - s * bs;
    const size_t dst = ((size_t)mem[mb + s] * bs + u) * kNull + j;
    const double q = A[r * kQrStride + j];
    Q64[dst] = q;
    Q32[dst] = (float)q;
  }
  for (int e = t; e < kNull * kNull; e += kQrBS) Kc[(size_t)a * kNull * kNull + e] = Rs[e / kNull][e % kNull];
  if (t == 0) kept_out[a] = kept;
}

// ---------------------------------------------------------------------------
// Galerkin product A_{l+1} = P^T A_l P (Section 2.3) on the coarse pattern, from the
// blocks of A_l P_l (assembled first, one per fine row and neighbouring aggregate):
//   A_{l+1}[a, b] = sum_{i in a} Q_i^T (A P)[i, b].
// The A P blocks that meet in each coarse block are listed once per problem (members of a
// in list order), and one CTA owns a coarse block: its warps take every kGalWarps-th A P
// block, lane s + 16 h keeping entries (8 h .. 8 h + 7, s) in registers, and the warps'
// sums are added in warp order.  A coarse dof dropped by the QR (zero Q column) gets a
// unit diagonal, which decouples it.  The diagonal blocks also go to cD (FP64) and cD32
// (FP32, if given): the coarse level's Jacobi blocks.
// ---------------------------------------------------------------------------
constexpr int kGalWarps = 4;   // warps per coarse block; each takes every kGalWarps-th A P block

template <typename T, int BS>
__global__ void __launch_bounds__(kGalWarps * 32)
k_galerkin(int nnzb_c, const int* __restrict__ gal_ptr, const int2* __restrict__ gal_list,
           const int* __restrict__ gal_row, const int* __restrict__ ccols, const T* __restrict__ ap,
           const T* __restrict__ Q, const unsigned* __restrict__ ckept, T* __restrict__ cvals, double* __restrict__ cD,
           float* __restrict__ cD32) {
  __shared__ T part[kGalWarps][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ce = blockIdx.x;
  const int s = lane & 15, r0 = (lane >> 4) * 8;
  T out[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) out[k] = T(0);
  for (int q = gal_ptr[ce] + warp; q < gal_ptr[ce + 1]; q += kGalWarps) {
    const int2 ci = gal_list[q];
    const T* apc = ap + (size_t)ci.x * BS * 16 + s;
    const T* qi = Q + (size_t)ci.y * BS * 16 + r0;
    T acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = T(0);
#pragma unroll
    for (int u = 0; u < BS; ++u) {
      const T a = apc[u * 16];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] += qi[u * 16 + k] * a;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) out[k] += acc[k];
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) part[warp][(r0 + k) * 16 + s] = out[k];
  __syncthreads();
  // the warps' partial blocks in warp order; entry e = r * 16 + s per thread
  const int a = gal_row[ce];
  const bool diag = ccols[ce] == a;
  const unsigned kept = ckept[a];
  for (int e = threadIdx.x; e < 256; e += kGalWarps * 32) {
    T v = T(0);
#pragma unroll
    for (int w = 0; w < kGalWarps; ++w) v += part[w][e];
    const int r = e >> 4, sc = e & 15;
    if (diag && r == sc && !((kept >> r) & 1u)) v = T(1);
    cvals[(size_t)ce * 256 + e] = v;
    if (diag && cD) {
      cD[(size_t)a * 256 + e] = (double)v;
      if (cD32) cD32[(size_t)a * 256 + e] = (float)v;
    }
  }
}

// the A P blocks of level L that meet in each block of level L1 (built on the host once)
static void galerkin_symbolic(ba_problem* P, Level& L, Level& L1) {
  auto down = [&](std::vector<int>& hv, const DBuf& d, size_t n) {
    hv.resize(std::max<size_t>(n, 1));
    if (n) BA_CUDA(cudaMemcpyAsync(hv.data(), d.p, sizeof(int) * n, cudaMemcpyDeviceToHost, P->stream));
  };
  std::vector<int> app, apc, aptr, amem, crp, ccl;
  down(app, L.ap_ptr, L.n + 1);
  down(apc, L.ap_cols, L.ap_nnzb);
  down(aptr, L.agg_ptr, L1.n + 1);
  down(amem, L.agg_mem, L.n);
  down(crp, L1.row_ptr, L1.n + 1);
  down(ccl, L1.cols, L1.nnzb);
  sync(P);
  std::vector<int> crow(std::max(L1.nnzb, 1)), cnt(L1.nnzb + 1, 0);
  for (int a = 0; a < L1.n; ++a)
    for (int c = crp[a]; c < crp[a + 1]; ++c) crow[c] = a;
  auto slot = [&](int a, int b) {
    int lo = crp[a], hi = crp[a + 1];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (ccl[mid] < b) lo = mid + 1;
      else hi = mid;
    }
    BA_REQUIRE(lo < crp[a + 1] && ccl[lo] == b, BA_ERR_STATE, "coarse pattern misses a Galerkin block");
    return lo;
  };
  std::vector<int2> list(std::max(L.ap_nnzb, 1));
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<int> fill;
    if (pass == 1) fill.assign(cnt.begin(), cnt.end() - 1);
    for (int a = 0; a < L1.n; ++a)
      for (int m = aptr[a]; m < aptr[a + 1]; ++m) {
        const int i = amem[m];
        for (int c = app[i]; c < app[i + 1]; ++c) {
          const int sl = slot(a, apc[c]);
          if (pass == 0) ++cnt[sl + 1];
          else list[fill[sl]++] = make_int2(c, i);
        }
      }
    if (pass == 0)
      for (int c = 0; c < L1.nnzb; ++c) cnt[c + 1] += cnt[c];
  }
  upload(P, L.gal_ptr, cnt);
  upload(P, L.gal_list, list);
  upload(P, L.gal_row, crow);
  sync(P);
}

// diagonal blocks of a BSR level as double
// level 0's Jacobi data from the Schur setup's: S_cc blocks (and their FP32 copy, if d32 is
// given, for the batched Lanczos) and their FP64 and FP32 inverses
__global__ void k_copy_jacobi0(size_t n, const double* __restrict__ s, const double* __restrict__ si,
                               const float* __restrict__ si32, double* __restrict__ d, float* __restrict__ d32,
                               double* __restrict__ di, float* __restrict__ di32) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = s[i];
    d[i] = v;
    if (d32) d32[i] = (float)v;
    di[i] = si[i];
    di32[i] = si32[i];
  }
}

// ---------------------------------------------------------------------------
// Lanczos helpers (D-inner product): start vector from SplitMix64, block-diagonal
// products, recurrence updates with scalars read from device memory.
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_start_vector(T* __restrict__ v, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (T)(2.0 * ((double)(splitmix64(i) >> 11) * 0x1.0p-53) - 1.0);
}

// y = B x for block-diagonal B (double blocks), T vectors
template <typename T>
__global__ void k_blockdiag_apply(int n, int bs, const double* __restrict__ B, const T* __restrict__ x,
                                  T* __restrict__ y) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * bs) return;
  const size_t i = idx / bs;
  const int u = (int)(idx - i * bs);
  const double* b = B + (i * bs + u) * bs;
  const T* xi = x + i * bs;
  double acc = 0.0;
  for (int v = 0; v < bs; ++v) acc += b[v] * (double)xi[v];
  y[idx] = (T)acc;
}

// q = v / sqrt(scal[s])
template <typename T>
__global__ void k_scale_rsqrt(size_t n, const T* __restrict__ v, T* __restrict__ q, const double* __restrict__ scal,
                              int s) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double f = 1.0 / sqrt(scal[s]);
  if (i < n) q[i] = (T)((double)v[i] * f);
}

// w = Dinv Aq - alpha q - beta qprev  (Dinv applied blockwise), alpha = scal[sa], beta = scal[sb] or 0
template <typename T>
__global__ void k_lanczos_w(int n, int bs, const double* __restrict__ Dinv, const T* __restrict__ Aq,
                            const T* __restrict__ q, const T* __restrict__ qprev, const double* __restrict__ scal,
                            int sa, int sb, T* __restrict__ w) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * bs) return;
  const size_t i = idx / bs;
  const int u = (int)(idx - i * bs);
  const double* b = Dinv + (i * bs + u) * bs;
  double acc = 0.0;
  for (int v = 0; v < bs; ++v) acc += b[v] * (double)Aq[i * bs + v];
  const double alpha = scal[sa];
  const double beta = sb >= 0 ? scal[sb] : 0.0;
  acc -= alpha * (double)q[idx];
  if (sb >= 0) acc -= beta * (double)qprev[idx];
  w[idx] = (T)acc;
}

__global__ void k_sqrt_slot(double* scal, int src, int dst) {
  if (threadIdx.x == 0) scal[dst] = sqrt(scal[src]);
}

template <typename T>
static void lanczos(ba_problem* P, int l) {
  Level& L = P->levels[l];
  const size_t n = (size_t)L.n * L.bs;
  const int m = std::min(std::max(P->opt.lanczos_steps, 1), 8);
  P->scratch2.ensure(sizeof(T) * n * 5 + 256);
  T* v = P->scratch2.as<T>();
  T* q = v + n;
  T* qprev = q + n;
  T* w = qprev + n;
  T* Aq = w + n;
  const int g = cdiv((long long)n, 256);
  double* scal = P->scal.as<double>();
  k_start_vector<T><<<g, 256, 0, P->stream>>>(v, n);
  launched(P);
  k_blockdiag_apply<T><<<g, 256, 0, P->stream>>>(L.n, L.bs, L.Dblk.as<double>(), v, w);
  launched(P);
  if (sizeof(T) == 8) dot64(P, (const double*)v, (const double*)w, n, S_TMP0);
  else dot32(P, (const float*)v, (const float*)w, n, S_TMP0);
  k_scale_rsqrt<T><<<g, 256, 0, P->stream>>>(n, v, q, scal, S_TMP0);
  launched(P);
  for (int j = 0; j < m; ++j) {
    level_matvec(P, l, q, Aq, false);
    if (sizeof(T) == 8) dot64(P, (const double*)q, (const double*)Aq, n, S_LANCZOS + j);
    else dot32(P, (const float*)q, (const float*)Aq, n, S_LANCZOS + j);
    k_lanczos_w<T><<<g, 256, 0, P->stream>>>(L.n, L.bs, L.Dinv64.as<double>(), Aq, q, qprev, scal,
                                            S_LANCZOS + j, j > 0 ? S_LANCZOS + 8 + j - 1 : -1, w);
    launched(P);
    if (j == m - 1) break;
    k_blockdiag_apply<T><<<g, 256, 0, P->stream>>>(L.n, L.bs, L.Dblk.as<double>(), w, v);
    launched(P);
    if (sizeof(T) == 8) dot64(P, (const double*)w, (const double*)v, n, S_TMP1);
    else dot32(P, (const float*)w, (const float*)v, n, S_TMP1);
    // beta_j = sqrt(w.Dw); q_prev <- q; q <- w / beta_j
    k_scale_rsqrt<T><<<g, 256, 0, P->stream>>>(n, w, v, scal, S_TMP1);  // v = w / beta
    launched(P);
    std::swap(qprev, q);   // qprev = old q
    std::swap(q, v);       // q = w / beta, v free
    k_sqrt_slot<<<1, 1, 0, P->stream>>>(scal, S_TMP1, S_LANCZOS + 8 + j);  // beta_j
    launched(P);
  }
  // park alpha_0..7 and beta_0..7 in the level's buffer (slots 8..23); the largest Ritz
  // value is found on the device once every level is done (finish_lanczos, k_cheb_params)
  L.cheb.ensure(sizeof(double) * kChebSlots);
  BA_CUDA(cudaMemcpyAsync(L.cheb.as<double>() + 8, scal + S_LANCZOS, sizeof(double) * 16, cudaMemcpyDeviceToDevice,
                          P->stream));
}

// Largest eigenvalue of each level's Lanczos tridiagonal (alpha_0..m-1 in slots 8..,
// beta_0..m-2 in slots 16..) by multisection with Sturm counts, and from it the Chebyshev
// parameters {theta, delta, sigma_1, lambda_max} of the interval [lo_f, hi_f] lambda_max
// (Section 3.4) in slots 0..3 and the step coefficients in slots 24...  One warp per level
// (each in its own CTA), on the device, so that the V-cycle's kernels read them there and the setup needs no host
// round trip: each round the 32 lanes count the eigenvalues below 32 points of the current
// interval and keep the sub-interval where the count reaches m, a factor 33 per round.
struct ChebLevels {
  double* cheb[16];
  int n;
};

__global__ void __launch_bounds__(32) k_cheb_params(ChebLevels CL, int m, double lo_f, double hi_f) {
  // one CTA (one warp) per level, so that the levels' FP64 recurrences run on different SMs
  const int k = blockIdx.x, lane = threadIdx.x;
  if (k >= CL.n) return;
  double* c = CL.cheb[k];
  double al[8], be2[8];
  int mm = m;
  for (int j = 0; j < m; ++j) al[j] = c[8 + j];
  for (int j = 0; j + 1 < m; ++j) {
    const double b = c[16 + j];
    be2[j] = b;
    if (!(b > 0.0)) {  // invariant subspace found: truncate
      mm = j + 1;
      break;
    }
  }
  // Gershgorin interval, and the matrix scaled by its bound s so that the characteristic
  // polynomials below stay within range
  double lo = al[0], hi = al[0];
  for (int j = 0; j < mm; ++j) {
    const double rad = (j > 0 ? fabs(be2[j - 1]) : 0.0) + (j + 1 < mm ? fabs(be2[j]) : 0.0);
    lo = fmin(lo, al[j] - rad);
    hi = fmax(hi, al[j] + rad);
  }
  const double s = fmax(fabs(lo), fabs(hi)) > 0.0 ? fmax(fabs(lo), fabs(hi)) : 1.0;
  for (int j = 0; j < mm; ++j) al[j] /= s;
  for (int j = 0; j + 1 < mm; ++j) be2[j] = (be2[j] / s) * (be2[j] / s);
  lo /= s;
  hi /= s;
  for (int round = 0; round < 64; ++round) {
    if (hi - lo <= 4.0 * 2.220446049250313e-16 * fabs(hi)) break;
    // lane j tests x = lo + (j + 1) (hi - lo) / 33: the eigenvalues below x are the sign
    // changes of p_0 = 1, p_1 = a_0 - x, p_j = (a_{j-1} - x) p_{j-1} - b_{j-2}^2 p_{j-2}
    // (a zero p_j takes the sign opposite to p_{j-1})
    const double x = lo + (double)(lane + 1) * ((hi - lo) / 33.0);
    int below = 0;
    double pm2 = 1.0, pm1 = al[0] - x;
    if (!(pm1 > 0.0)) ++below;
    for (int j = 1; j < mm; ++j) {
      const double pj = (al[j] - x) * pm1 - be2[j - 1] * pm2;
      if (pm1 == 0.0 ? true : (pm1 > 0.0 ? !(pj > 0.0) : (pj > 0.0))) ++below;
      pm2 = pm1;
      pm1 = pj == 0.0 ? -copysign(1e-300, pm2) : pj;
    }
    const bool all_below = below >= mm && x > lo && x < hi;
    const unsigned ball = __ballot_sync(0xffffffffu, all_below);
    double nlo, nhi;
    if (ball) {
      const int f = __ffs(ball) - 1;   // first point with every eigenvalue below it
      nhi = __shfl_sync(0xffffffffu, x, f);
      nlo = f > 0 ? __shfl_sync(0xffffffffu, x, f - 1) : lo;
    } else {
      nlo = __shfl_sync(0xffffffffu, x, 31);
      nhi = hi;
    }
    if (!(nlo > lo || nhi < hi)) break;   // the interval no longer shrinks
    lo = fmax(lo, nlo);
    hi = fmin(hi, nhi);
  }
  hi *= s;
  if (lane != 0) return;
  const double lam = hi;
  const double a = lo_f * lam, b = hi_f * lam;
  c[0] = 0.5 * (b + a);
  c[1] = 0.5 * (b - a);
  c[2] = c[0] / c[1];
  c[3] = lam;
  // step coefficients (Saad, Alg. 12.1): d_k = c1 d_{k-1} + c2 D^-1 r_k with rho_0 = 1 /
  // sigma_1, rho_j = 1 / (2 sigma_1 - rho_{j-1}), c1 = rho_k rho_{k-1}, c2 = 2 rho_k / delta
  double rho = 1.0 / c[2];
  for (int j = 1; j < kMaxSmooth; ++j) {
    const double rho_prev = rho;
    rho = 1.0 / (2.0 * c[2] - rho);
    c[24 + 2 * (j - 1)] = rho * rho_prev;
    c[25 + 2 * (j - 1)] = 2.0 * rho / c[1];
  }
}

// the Chebyshev parameters of every smoothed level from its Lanczos coefficients
static void finish_lanczos(ba_problem* P) {
  const int nl = P->n_levels - 1;
  if (nl <= 0) return;
  BA_REQUIRE(nl <= 16, BA_ERR_LIMIT, "more than 16 smoothed levels");
  ChebLevels CL{};
  CL.n = nl;
  for (int k = 0; k < nl; ++k) CL.cheb[k] = P->levels[k].cheb.as<double>();
  const int m = std::min(std::max(P->opt.lanczos_steps, 1), 8);
  k_cheb_params<<<nl, 32, 0, P->stream>>>(CL, m, P->opt.cheb_lo, P->opt.cheb_hi);
  launched(P);
}

// ---------------------------------------------------------------------------
// coarsest level: dense FP64 matrix from the BSR blocks, padded with identity to a
// multiple of the pivot width, inverted by blocked Gauss-Jordan (SPD, no pivoting) in a
// cooperative kernel with one grid barrier per pivot block.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_bsr_to_dense(int n, int bs, const int* __restrict__ row_ptr, const int* __restrict__ cols,
                               const T* __restrict__ vals, int Np, double* __restrict__ A) {
  const int i = blockIdx.x;
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
    const int j = cols[e];
    for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) {
      const int u = t / bs, v = t - u * bs;
      A[(size_t)(i * bs + u) * Np + j * bs + v] = (double)vals[(size_t)e * bs * bs + t];
    }
  }
}

__global__ void k_dense_identity_pad(int N, int Np, double* __restrict__ A) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)Np * Np) return;
  const int i = (int)(idx / Np), j = (int)(idx % Np);
  if (i >= N || j >= N) A[idx] = (i == j) ? 1.0 : 0.0;
}

constexpr int kGJ = 16;   // pivot block: its inversion is the serial part of every step
constexpr int kGJBS = kGJ * kGJ;
// in-place inverse of the SPD kGJ x kGJ matrix in shared memory (Gauss-Jordan, no
// pivoting; one thread per entry); returns false in thread 0 if a pivot is not positive
__device__ __forceinline__ bool gj_invert(double piv[kGJ][kGJ + 1], double* gj_row, double* gj_col, double& gj_ip) {
  const int t = threadIdx.x, u = t / kGJ, v = t % kGJ;
  bool ok = true;
  for (int k = 0; k < kGJ; ++k) {
    if (t == 0) {
      const double pk = piv[k][k];
      if (!(pk > 0.0)) ok = false;
      gj_ip = 1.0 / pk;
    }
    __syncthreads();
    const double ip = gj_ip;
    if (t < kGJ) {
      gj_row[t] = t == k ? ip : piv[k][t] * ip;
      gj_col[t] = piv[t][k];
    }
    __syncthreads();
    double nv;
    if (u == k) nv = gj_row[v];
    else if (v == k) nv = -gj_col[u] * ip;
    else nv = piv[u][v] - gj_col[u] * gj_row[v];
    piv[u][v] = nv;
    __syncthreads();
  }
  return ok;
}

// Per pivot block K (kGJ wide) every CTA reads P^-1 = (A_KK)^-1 and writes its tiles of
// the next matrix:
//   A'_KK = P^-1,  A'_KJ = P^-1 A_KJ,  A'_IK = -A_IK P^-1,  A'_IJ = A_IJ - A_IK (P^-1 A_KJ)
// reading A and writing A' (two buffers that swap roles every step).  The CTA that
// writes the next pivot block A'_{K+1,K+1} inverts it before the step's grid barrier, so
// a step needs one barrier and the inversion overlaps the other CTAs' tiles.
__global__ void __launch_bounds__(kGJBS) k_gauss_jordan(double* Aa, double* Ab, int Np, double* pinv, int* flags) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double piv[kGJ][kGJ + 1];
  __shared__ double gj_row[kGJ], gj_col[kGJ];
  __shared__ double gj_ip;
  __shared__ double sa[kGJ][kGJ + 1], sb[kGJ][kGJ + 1], st[kGJ][kGJ + 1];
  const int nb = Np / kGJ;
  const int t = threadIdx.x, u = t / kGJ, v = t % kGJ;
  if (blockIdx.x == 0) {
    piv[u][v] = Aa[(size_t)u * Np + v];
    __syncthreads();
    const bool ok = gj_invert(piv, gj_row, gj_col, gj_ip);
    if (t == 0 && !ok) flags[F_NOT_SPD_COARSE] = 1;
    pinv[t] = piv[u][v];
  }
  grid.sync();
  for (int K = 0; K < nb; ++K) {
    const double* A = (K & 1) ? Ab : Aa;
    double* An = (K & 1) ? Aa : Ab;
    const int K0 = K * kGJ;
    piv[u][v] = pinv[(size_t)(K & 1) * kGJBS + t];
    __syncthreads();
    bool owner = false;
    for (int w = blockIdx.x; w < nb * nb; w += gridDim.x) {
      const int I = w / nb, J = w - I * nb;
      if (I == K + 1 && J == K + 1) owner = true;
      double out;
      if (I == K && J == K) {
        out = piv[u][v];
      } else if (I == K) {
        sb[u][v] = A[(size_t)(K0 + u) * Np + J * kGJ + v];
        __syncthreads();
        out = 0.0;
#pragma unroll
        for (int k = 0; k < kGJ; ++k) out += piv[u][k] * sb[k][v];
      } else if (J == K) {
        sa[u][v] = A[(size_t)(I * kGJ + u) * Np + K0 + v];
        __syncthreads();
        out = 0.0;
#pragma unroll
        for (int k = 0; k < kGJ; ++k) out -= sa[u][k] * piv[k][v];
      } else {
        sa[u][v] = A[(size_t)(I * kGJ + u) * Np + K0 + v];
        sb[u][v] = A[(size_t)(K0 + u) * Np + J * kGJ + v];
        const double aij = A[(size_t)(I * kGJ + u) * Np + J * kGJ + v];
        __syncthreads();
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kGJ; ++k) s += piv[u][k] * sb[k][v];
        st[u][v] = s;
        __syncthreads();
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < kGJ; ++k) acc += sa[u][k] * st[k][v];
        out = aij - acc;
      }
      An[(size_t)(I * kGJ + u) * Np + J * kGJ + v] = out;
      __syncthreads();   // the tile buffers are refilled by the next work item
    }
    if (owner) {
      // the next pivot block, just written by this CTA, inverted for every CTA's next step
      const int K1 = K0 + kGJ;
      piv[u][v] = An[(size_t)(K1 + u) * Np + K1 + v];
      __syncthreads();
      const bool ok = gj_invert(piv, gj_row, gj_col, gj_ip);
      if (t == 0 && !ok) flags[F_NOT_SPD_COARSE] = 1;
      pinv[(size_t)((K + 1) & 1) * kGJBS + t] = piv[u][v];
    }
    grid.sync();
  }
}

// The same inversion in paired FP32 (mixed precision): the matrix as (hi, lo) float pairs,
// products as compensated sums, the pivot reciprocal as a DF division.  The FP64 unit of
// this GPU takes a warp's FMA over many cycles per SM sub-partition; the pairs run on the
// FP32 pipes and carry ~48 bits, well beyond what the FP32 coarse operator holds.
// the pivot block's inverse in place, alternating between piv and tmp (kGJ is even, so the
// result ends in piv): every thread forms the pivot's reciprocal and reads row and column
// k of the current tile itself, so a step has one barrier
__device__ __forceinline__ bool gj_invert_df(float2 piv[kGJ][kGJ + 1], float2 tmp[kGJ][kGJ + 1]) {
  static_assert(kGJ % 2 == 0, "the ping-pong must end in the input tile");
  const int t = threadIdx.x, u = t / kGJ, v = t % kGJ;
  bool ok = true;
#pragma unroll 1
  for (int k = 0; k < kGJ; ++k) {
    float2 (*src)[kGJ + 1] = (k & 1) ? tmp : piv;
    float2 (*dst)[kGJ + 1] = (k & 1) ? piv : tmp;
    const DF pk(src[k][k].x, src[k][k].y);
    if (!(pk.h > 0.f)) ok = false;
    const DF ip = DF(1.f, 0.f) / pk;
    const DF rv = v == k ? ip : DF(src[k][v].x, src[k][v].y) * ip;
    const DF cu(src[u][k].x, src[u][k].y);
    DF nv;
    if (u == k) nv = rv;
    else if (v == k) nv = -(cu * ip);
    else nv = DF(src[u][v].x, src[u][v].y) - cu * rv;
    dst[u][v] = make_float2(nv.h, nv.l);
    __syncthreads();
  }
  return ok;
}

// sum_k x[u][k] y[k][v] of two kGJ x kGJ tiles in shared memory, compensated
__device__ __forceinline__ DF gj_tile_dot(const float2 x[kGJ][kGJ + 1], const float2 y[kGJ][kGJ + 1], int u, int v) {
  float s = 0.f, c = 0.f;
#pragma unroll
  for (int k = 0; k < kGJ; ++k) dot2_fma(s, c, x[u][k], y[k][v]);
  return DF(s, 0.f) + DF(c, 0.f);
}

__global__ void __launch_bounds__(kGJBS) k_gauss_jordan_df(float2* Aa, float2* Ab, int Np, float2* pinv, int* flags) {
  cg::grid_group grid = cg::this_grid();
  __shared__ float2 piv[kGJ][kGJ + 1], piv2[kGJ][kGJ + 1], gj_tmp[kGJ][kGJ + 1];
  __shared__ float2 sa[kGJ][kGJ + 1], sb[kGJ][kGJ + 1], st[kGJ][kGJ + 1];
  const int nb = Np / kGJ;
  const int t = threadIdx.x, u = t / kGJ, v = t % kGJ;
  if (blockIdx.x == 0) {
    piv[u][v] = Aa[(size_t)u * Np + v];
    __syncthreads();
    const bool ok = gj_invert_df(piv, gj_tmp);
    if (t == 0 && !ok) flags[F_NOT_SPD_COARSE] = 1;
    pinv[t] = piv[u][v];
  }
  grid.sync();
  for (int K = 0; K < nb; ++K) {
    const float2* A = (K & 1) ? Ab : Aa;
    float2* An = (K & 1) ? Aa : Ab;
    const int K0 = K * kGJ;
    piv[u][v] = pinv[(size_t)(K & 1) * kGJBS + t];
    __syncthreads();
    // this CTA's tiles; the next pivot block first if it is one of them, so that its
    // inverse is formed while the other CTAs update their tiles
    const int wn = K + 1 < nb ? (K + 1) * nb + (K + 1) : -1;
    const bool owner = wn >= 0 && wn % (int)gridDim.x == (int)blockIdx.x;
    for (int it = 0, w = owner ? wn : (int)blockIdx.x; w < nb * nb; ++it) {
      const int I = w / nb, J = w - I * nb;
      DF out;
      if (I == K && J == K) {
        out = DF(piv[u][v].x, piv[u][v].y);
      } else if (I == K) {
        sb[u][v] = A[(size_t)(K0 + u) * Np + J * kGJ + v];
        __syncthreads();
        out = gj_tile_dot(piv, sb, u, v);
      } else if (J == K) {
        sa[u][v] = A[(size_t)(I * kGJ + u) * Np + K0 + v];
        __syncthreads();
        out = -gj_tile_dot(sa, piv, u, v);
      } else {
        sa[u][v] = A[(size_t)(I * kGJ + u) * Np + K0 + v];
        sb[u][v] = A[(size_t)(K0 + u) * Np + J * kGJ + v];
        const float2 aij = A[(size_t)(I * kGJ + u) * Np + J * kGJ + v];
        __syncthreads();
        const DF sv = gj_tile_dot(piv, sb, u, v);
        st[u][v] = make_float2(sv.h, sv.l);
        __syncthreads();
        out = DF(aij.x, aij.y) - gj_tile_dot(sa, st, u, v);
      }
      An[(size_t)(I * kGJ + u) * Np + J * kGJ + v] = make_float2(out.h, out.l);
      __syncthreads();
      if (w == wn) {
        piv2[u][v] = make_float2(out.h, out.l);
        __syncthreads();
        const bool ok = gj_invert_df(piv2, gj_tmp);
        if (t == 0 && !ok) flags[F_NOT_SPD_COARSE] = 1;
        pinv[(size_t)((K + 1) & 1) * kGJBS + t] = piv2[u][v];
        __syncthreads();
      }
      // next tile in this CTA's order, the pivot block (done first) skipped
      if (owner && it == 0) w = (int)blockIdx.x;
      else w += gridDim.x;
      if (owner && w == wn) w += gridDim.x;
    }
    grid.sync();
  }
}

__global__ void k_df2d_vec(size_t n, const float2* __restrict__ a, double* __restrict__ b) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = to_double(DF(a[i].x, a[i].y));
}

__global__ void k_d2f_vec(size_t n, const double* __restrict__ a, float* __restrict__ b) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// the coarsest operator's FP32 blocks as a dense float-pair matrix (value, 0), padded with
// the identity up to Np (Da zeroed beforehand)
__global__ void k_bsr_to_dense_df(int n, int bs, const int* __restrict__ row_ptr, const int* __restrict__ cols,
                                  const float* __restrict__ vals, int N, int Np, float2* __restrict__ Da) {
  const int i = blockIdx.x;
  if (i < n) {
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      const int j = cols[e];
      for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) {
        const int u = t / bs, v = t - u * bs;
        Da[(size_t)(i * bs + u) * Np + j * bs + v] = make_float2(vals[(size_t)e * bs * bs + t], 0.f);
      }
    }
  } else {
    for (int k = N + (int)threadIdx.x; k < Np; k += blockDim.x) Da[(size_t)k * Np + k] = make_float2(1.f, 0.f);
  }
}

static void dense_inverse(ba_problem* P, Level& L, cudaStream_t st) {
  const int N = L.n * L.bs;
  const int Np = (N + kGJ - 1) / kGJ * kGJ;
  BA_REQUIRE(Np <= 16384, BA_ERR_LIMIT, "coarsest level too large for the dense solver (" + std::to_string(N) + " dofs)");
  L.N = Np;
  L.Ainv.ensure(sizeof(double) * (size_t)Np * Np);
  double* A = L.Ainv.as<double>();
  if (level_fp32(P)) {
    if (!L.vals32.p) throw Error(BA_ERR_STATE, "missing coarse operator");
    // paired FP32: both buffers of the ping-pong and the pivot inverses as float pairs; the
    // matrix goes straight from the blocks into the first buffer
    const size_t nn = (size_t)Np * Np;
    P->scratch.ensure(sizeof(float2) * (2 * nn + 2 * kGJBS) + 64);
    float2* Da = P->scratch.as<float2>();
    float2* Db = Da + nn;
    float2* pinv = Db + nn;
    BA_CUDA(cudaMemsetAsync(Da, 0, sizeof(float2) * nn, st));
    k_bsr_to_dense_df<<<L.n + 1, 256, 0, st>>>(L.n, L.bs, L.row_ptr.as<int>(), L.cols.as<int>(),
                                                       L.vals32.as<float>(), N, Np, Da);
    launched(P);
    int nblk = 0;
    BA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, k_gauss_jordan_df, kGJBS, 0));
    const int nbk = Np / kGJ;
    int grid = std::max(1, std::min(nblk * P->n_sm, nbk * nbk));
    int* flags = P->flags.as<int>();
    void* args[] = {(void*)&Da, (void*)&Db, (void*)&Np, (void*)&pinv, (void*)&flags};
    BA_CUDA(cudaLaunchCooperativeKernel((void*)k_gauss_jordan_df, grid, kGJBS, args, 0, st));
    launched(P);
    k_df2d_vec<<<cdiv((long long)nn, 256), 256, 0, st>>>(nn, (nbk & 1) ? Db : Da, A);
    launched(P);
    return;
  }
  BA_CUDA(cudaMemsetAsync(A, 0, sizeof(double) * (size_t)Np * Np, st));
  k_bsr_to_dense<double><<<L.n, 256, 0, st>>>(L.n, L.bs, L.row_ptr.as<int>(), L.cols.as<int>(),
                                                     L.vals64.as<double>(), Np, A);
  launched(P);
  k_dense_identity_pad<<<cdiv((long long)Np * Np, 256), 256, 0, st>>>(N, Np, A);
  launched(P);
  // second buffer of the ping-pong and the two pivot inverses
  P->scratch.ensure(sizeof(double) * ((size_t)Np * Np + 2 * kGJBS) + 64);
  double* B = P->scratch.as<double>();
  double* pinv = B + (size_t)Np * Np;
  int nblk = 0;
  BA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, k_gauss_jordan, kGJBS, 0));
  const int nbk = Np / kGJ;
  int grid = std::max(1, std::min(nblk * P->n_sm, nbk * nbk));
  int* flags = P->flags.as<int>();
  void* args[] = {(void*)&A, (void*)&B, (void*)&Np, (void*)&pinv, (void*)&flags};
  BA_CUDA(cudaLaunchCooperativeKernel((void*)k_gauss_jordan, grid, kGJBS, args, 0, st));
  launched(P);
  // after an odd number of steps the inverse is in the second buffer
  if (nbk & 1) BA_CUDA(cudaMemcpyAsync(A, B, sizeof(double) * (size_t)Np * Np, cudaMemcpyDeviceToDevice, st));
}

// ---------------------------------------------------------------------------
// orchestration
//
// The symbolic hierarchy (covisibility counts and block patterns of every level,
// strength orderings, Algorithm 2 aggregates and their member lists) depends only on
// the observation graph, so it is built on the first call and reused by every later
// LM step; each call recomputes only the numerical parts (level-0 blocks, the
// near-nullspace at the current cameras, QR prolongators, Galerkin products,
// smoother blocks, Lanczos estimates and the coarsest inverse).
// ---------------------------------------------------------------------------
static int max_row_length(ba_problem* P, const Level& L) {
  std::vector<int> hptr(L.n + 1);
  BA_CUDA(cudaMemcpyAsync(hptr.data(), L.row_ptr.p, sizeof(int) * (L.n + 1), cudaMemcpyDeviceToHost, P->stream));
  sync(P);
  int maxrow = 1;
  for (int i = 0; i < L.n; ++i) maxrow = std::max(maxrow, hptr[i + 1] - hptr[i]);
  return maxrow;
}

static void mg_symbolic(ba_problem* P) {
  const ba_options& o = P->opt;
  if ((int)P->levels.size() < 1) P->levels.resize(1);
  Level& L0 = P->levels[0];
  covisibility_level0(P, L0);
  L0.n = P->n_c;
  L0.bs = 9;
  L0.maxrow = max_row_length(P, L0);
  int l = 0;
  while (true) {
    Level& L = P->levels[l];
    L.coarsest = false;
    bool coarsest = L.n <= o.coarse_max_nodes || l + 1 >= o.max_levels || l + 1 >= 16;
    if (!coarsest) {
      // strength ordering
      L.sptr.ensure(sizeof(int) * ((size_t)L.n + 1));
      P->scratch.ensure(sizeof(int) * ((size_t)L.n + 1) + sizeof(long long) * (size_t)L.n + 64);
      int* cnt = P->scratch.as<int>();
      k_strength_count<<<cdiv(L.n, 128), 128, 0, P->stream>>>(L.n, L.row_ptr.as<int>(), L.cols.as<int>(),
                                                              L.W.as<long long>(), cnt);
      launched(P);
      L.n_strength = scan(P, cnt, L.sptr.as<int>(), L.n);
      L.sidx.ensure(sizeof(int) * (size_t)std::max(L.n_strength, 1));
      P->scratch2.ensure(sizeof(long long) * (size_t)L.n + 64);
      long long* Wd = P->scratch2.as<long long>();
      k_diag_w<<<cdiv(L.n, 128), 128, 0, P->stream>>>(L.n, L.row_ptr.as<int>(), L.cols.as<int>(),
                                                     L.W.as<long long>(), Wd);
      launched(P);
      int mpow = 1;
      while (mpow < L.maxrow) mpow <<= 1;
      const size_t ssm = sizeof(StrengthKey) * mpow;
      BA_REQUIRE(ssm <= 200 * 1024, BA_ERR_LIMIT, "too many covisible neighbours for the strength sort");
      BA_CUDA(cudaFuncSetAttribute(k_strength_order, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm));
      k_strength_order<<<L.n, kStrBS, ssm, P->stream>>>(L.n, L.row_ptr.as<int>(), L.cols.as<int>(),
                                                        L.W.as<long long>(), Wd, L.sptr.as<int>(), L.sidx.as<int>());
      launched(P);
      // Algorithm 2
      L.agg.ensure(sizeof(int) * (size_t)L.n + 64);
      P->scratch.ensure(sizeof(int) * (2 * (size_t)L.n + 8));
      int* gsize = P->scratch.as<int>();
      int* d_nagg = gsize + L.n + 4;
      const size_t asmem = sizeof(int) * 2 * (size_t)L.n;
      if (asmem <= 160 * 1024) {
        BA_CUDA(cudaFuncSetAttribute(k_aggregate<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asmem));
        k_aggregate<true><<<1, 64, asmem, P->stream>>>(L.n, L.sptr.as<int>(), L.sidx.as<int>(), o.max_agg,
                                                        L.agg.as<int>(), gsize, d_nagg);
      } else {
        k_aggregate<false><<<1, 64, 0, P->stream>>>(L.n, L.sptr.as<int>(), L.sidx.as<int>(), o.max_agg,
                                                     L.agg.as<int>(), gsize, d_nagg);
      }
      launched(P);
      BA_CUDA(cudaMemcpyAsync(&L.n_agg, d_nagg, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
      sync(P);
      if (L.n_agg >= L.n) coarsest = true;
    }
    if (coarsest) {
      L.coarsest = true;
      break;
    }
    // members of each aggregate
    L.agg_ptr.ensure(sizeof(int) * ((size_t)L.n_agg + 1));
    L.agg_mem.ensure(sizeof(int) * (size_t)L.n + 64);
    P->scratch.ensure(sizeof(int) * 2 * ((size_t)L.n_agg + 1) + 64);
    int* mc = P->scratch.as<int>();
    int* fill = mc + L.n_agg + 1;
    BA_CUDA(cudaMemsetAsync(mc, 0, sizeof(int) * 2 * (L.n_agg + 1), P->stream));
    k_count_members<<<cdiv(L.n, 256), 256, 0, P->stream>>>(L.n, L.agg.as<int>(), mc);
    launched(P);
    scan(P, mc, L.agg_ptr.as<int>(), L.n_agg);
    {
      std::vector<int> hp(L.n_agg + 1);
      BA_CUDA(cudaMemcpyAsync(hp.data(), L.agg_ptr.p, sizeof(int) * (L.n_agg + 1), cudaMemcpyDeviceToHost, P->stream));
      sync(P);
      L.agg_max = 1;
      for (int k = 0; k < L.n_agg; ++k) L.agg_max = std::max(L.agg_max, hp[k + 1] - hp[k]);
    }
    k_fill_members<<<cdiv(L.n, 256), 256, 0, P->stream>>>(L.n, L.agg.as<int>(), L.agg_ptr.as<int>(), fill,
                                                          L.agg_mem.as<int>());
    launched(P);
    k_sort_members<<<cdiv(L.n_agg, 128), 128, 0, P->stream>>>(L.n_agg, L.agg_ptr.as<int>(), L.agg_mem.as<int>());
    launched(P);
    // next level's pattern and covisibility W_{l+1} = Agg^T W_l Agg
    if ((int)P->levels.size() < l + 2) P->levels.resize(l + 2);
    Level& L1 = P->levels[l + 1];
    Level& Lc = P->levels[l];
    L1.n = Lc.n_agg;
    L1.bs = kNull;
    const int H = hash_size(std::min(L1.n, 4096));
    row_hash<1>(P, L1.n, H, Lc.agg_ptr.as<int>(), Lc.agg_mem.as<int>(), Lc.row_ptr.as<int>(), Lc.cols.as<int>(),
                Lc.agg.as<int>(), Lc.W.as<long long>(), L1);
    L1.maxrow = max_row_length(P, L1);
    ++l;
  }
  P->n_levels = l + 1;
  P->sym_ready = true;
}

// The near-nullspace of level 0 and every level's per-aggregate QR (Section 3.3): they need
// only the cameras and the aggregates, not the operators, so they run on the side stream
// while the main stream assembles S.
static void prolongator_chain(ba_problem* P, cudaStream_t st) {
  const bool fp32 = level_fp32(P);
  Level& L0 = P->levels[0];
  L0.K.ensure(sizeof(double) * 9 * kNull * (size_t)P->n_c + 64);
  // one warp per CTA: the cameras' FP64 work spread over as many SMs as possible
  k_nullspace0<<<cdiv(P->n_c, 32), 32, 0, st>>>(P->cams_lin.as<double>(), P->n_c, L0.K.as<double>());
  launched(P);
  L0.kept.ensure(sizeof(unsigned) * P->n_c + 64);
  BA_CUDA(cudaMemsetAsync(L0.kept.p, 0xff, sizeof(unsigned) * P->n_c, st));
  for (int l = 0; l < P->n_levels; ++l) {
    Level& L = P->levels[l];
    if (L.coarsest) break;
    Level& L1 = P->levels[l + 1];
    // QR prolongators, coarse nullspace and kept masks
    L.Q64.ensure(sizeof(double) * L.bs * kNull * (size_t)L.n + 64);
    L.Q32.ensure(sizeof(float) * L.bs * kNull * (size_t)L.n + 64);
    L1.K.ensure(sizeof(double) * kNull * kNull * (size_t)L1.n + 64);
    L1.kept.ensure(sizeof(unsigned) * (size_t)L1.n + 64);
    const int max_rows = std::max(1, L.agg_max) * L.bs;
    const size_t qsm = sizeof(double) * (size_t)kQrWarps * max_rows * kQrStride;
    BA_REQUIRE(qsm <= 200 * 1024, BA_ERR_LIMIT, "aggregates too large for the aggregate QR");
    if (fp32) {
      // mixed precision: the DF factorisation, one CTA per aggregate at every level
      const size_t dsm = sizeof(float2) * (size_t)max_rows * kQrStride;
      BA_CUDA(cudaFuncSetAttribute(k_aggregate_qr_df_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
      k_aggregate_qr_df_cta<<<L1.n, kQrDfBS, dsm, st>>>(
          L1.n, L.bs, L.agg_ptr.as<int>(), L.agg_mem.as<int>(), L.K.as<double>(), L.Q64.as<double>(),
          L.Q32.as<float>(), L1.K.as<double>(), L1.kept.as<unsigned>());
    } else if (L1.n >= 2 * P->n_sm) {
      BA_CUDA(cudaFuncSetAttribute(k_aggregate_qr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsm));
      k_aggregate_qr<<<cdiv(L1.n, kQrWarps), kQrWarps * 32, qsm, st>>>(
          L1.n, L.bs, max_rows, L.agg_ptr.as<int>(), L.agg_mem.as<int>(), L.K.as<double>(), L.Q64.as<double>(),
          L.Q32.as<float>(), L1.K.as<double>(), L1.kept.as<unsigned>());
    } else {
      const size_t csm = sizeof(double) * (size_t)max_rows * kQrStride;
      BA_CUDA(cudaFuncSetAttribute(k_aggregate_qr_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
      k_aggregate_qr_cta<<<L1.n, kQrBS, csm, st>>>(L1.n, L.bs, L.agg_ptr.as<int>(), L.agg_mem.as<int>(),
                                                          L.K.as<double>(), L.Q64.as<double>(), L.Q32.as<float>(),
                                                          L1.K.as<double>(), L1.kept.as<unsigned>());
    }
    launched(P);
  }
}

void mg_setup(ba_problem* P, bool check) {
  const bool fp32 = level_fp32(P);
  const ba_options& o = P->opt;
  // check = false (the LM step): the flags of the linearisation and the Schur setup stay
  // for the step's next fetch_checked
  if (check) clear_flags(P);
  if (!P->sym_ready) mg_symbolic(P);
  Level& L0 = P->levels[0];
  {
    // Section 3.6: each level uses the cheaper of the implicit and the assembled operator;
    // level 0 is S itself, so the choice covers the PCG product as well
    const size_t elem = fp32 ? 4 : 8;
    const double explicit_bytes = (double)L0.nnzb * (81.0 * elem + 4.0);
    const double implicit_bytes = (double)P->n_o * (24.0 * elem + 4.0) + (double)P->n_p * 6.0 * elem;
    P->l0_explicit = o.level0_operator == BA_OP_EXPLICIT ||
                     (o.level0_operator == BA_OP_AUTO && explicit_bytes < implicit_bytes);
    P->outer_explicit = P->l0_explicit;
  }
  // the prolongators beside the assembly: fork the side stream after everything the main
  // stream has queued (the cameras of the linearisation, the aggregates)
  if (!P->side_stream) {
    BA_CUDA(cudaStreamCreateWithFlags(&P->side_stream, cudaStreamNonBlocking));
    BA_CUDA(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
    BA_CUDA(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
  }
  BA_CUDA(cudaEventRecord(P->ev_fork, P->stream));
  BA_CUDA(cudaStreamWaitEvent(P->side_stream, P->ev_fork, 0));
  prolongator_chain(P, P->side_stream);
  BA_CUDA(cudaEventRecord(P->ev_join, P->side_stream));
  // the Galerkin product needs S assembled in any case; the PCG product needs its FP64
  // value, which mixed precision forms in paired FP32
  explicit_schur(P, L0, !fp32 ? EX_FP64 : P->outer_explicit ? EX_PAIRED : EX_FP32);
  // level-0 smoother blocks: S_cc from the Schur setup
  L0.Dblk.ensure(sizeof(double) * 81 * (size_t)P->n_c + 64);
  L0.Dinv64.ensure(sizeof(double) * 81 * (size_t)P->n_c + 64);
  L0.Dinv32.ensure(sizeof(float) * 81 * (size_t)P->n_c + 64);
  {
    const size_t n81 = 81 * (size_t)P->n_c;
    if (fp32) L0.Dblk32.ensure(sizeof(float) * n81 + 64);
    k_copy_jacobi0<<<std::max(1, std::min(cdiv((long long)n81, 256), 4 * P->n_sm)), 256, 0, P->stream>>>(
        n81, P->Scc.as<double>(), P->Scc_inv.as<double>(), P->Scc_inv32.as<float>(), L0.Dblk.as<double>(),
        fp32 ? L0.Dblk32.as<float>() : nullptr, L0.Dinv64.as<double>(), L0.Dinv32.as<float>());
    launched(P);
  }

  const bool batch_inv = P->opt.precision == BA_MIXED;
  BlockInvBatch inv{};
  BA_CUDA(cudaStreamWaitEvent(P->stream, P->ev_join, 0));
  bool coarse_forked = false;
  for (int l = 0; l < P->n_levels; ++l) {
    Level& L = P->levels[l];
    if (l > 0) {
      L.Dblk.ensure(sizeof(double) * L.bs * L.bs * (size_t)L.n + 64);
      L.Dinv64.ensure(sizeof(double) * L.bs * L.bs * (size_t)L.n + 64);
      L.Dinv32.ensure(sizeof(float) * L.bs * L.bs * (size_t)L.n + 64);
    }
    if (L.coarsest) {
      // the coarsest inverse (a cooperative kernel of nb = N / 16 grid barriers) beside the
      // smoother blocks and the Lanczos runs, which do not read it; joined below
      BA_CUDA(cudaEventRecord(P->ev_fork, P->stream));
      BA_CUDA(cudaStreamWaitEvent(P->side_stream, P->ev_fork, 0));
      dense_inverse(P, L, P->side_stream);
      BA_CUDA(cudaEventRecord(P->ev_join, P->side_stream));
      coarse_forked = true;
      break;
    }
    // smoother for this level: its diagonal blocks (FP64, and FP32 for the batched Lanczos)
    // were written by the Galerkin product that formed the level
    const size_t nb2 = (size_t)L.bs * L.bs * L.n;
    if (fp32) L.Dblk32.ensure(sizeof(float) * nb2 + 64);
    if (l > 0) {
      if (batch_inv && L.bs == 16 && inv.nseg < kMaxInvSegs) {
        // inverted with the other coarse levels' blocks in one launch after the loop (only
        // the batched Lanczos and the V-cycle read them)
        inv.s[inv.nseg++] = BlockInvSeg{L.Dblk.as<double>(), L.Dinv64.as<double>(), L.Dinv32.as<float>(), L.n,
                                        inv.total};
        inv.total += L.n;
      } else {
        block_inverse(P, L.Dblk.as<double>(), L.n, L.bs, L.Dinv64.as<double>(), L.Dinv32.as<float>(),
                      F_NOT_SPD_JACOBI);
      }
    }
    // assembled levels get their Lanczos estimate in one batch after the loop
    if (l == 0 && !P->l0_explicit) {
      if (fp32) lanczos<float>(P, l);
      else lanczos<double>(P, l);
    }
    Level& L1 = P->levels[l + 1];
    // Galerkin from A P (which the fused V-cycle also uses)
    build_ap(P, L);
    if (!L.gal_ptr.p) galerkin_symbolic(P, L, L1);
    const int gg = std::max(L1.nnzb, 1);
    // the next level's Jacobi blocks come out of the same product (not for the coarsest,
    // which is inverted whole)
    double* cD = nullptr;
    float* cD32 = nullptr;
    if (!L1.coarsest) {
      const size_t nb2c = (size_t)L1.bs * L1.bs * L1.n;
      L1.Dblk.ensure(sizeof(double) * nb2c + 64);
      cD = L1.Dblk.as<double>();
      if (fp32) {
        L1.Dblk32.ensure(sizeof(float) * nb2c + 64);
        cD32 = L1.Dblk32.as<float>();
      }
    }
    if (fp32) {
      L1.vals32.ensure(sizeof(float) * 256 * (size_t)L1.nnzb + 64);
      if (L.bs == 9)
        k_galerkin<float, 9><<<gg, kGalWarps * 32, 0, P->stream>>>(L1.nnzb, L.gal_ptr.as<int>(), L.gal_list.as<int2>(),
                                                          L.gal_row.as<int>(), L1.cols.as<int>(),
                                                          L.ap_vals.as<float>(), L.Q32.as<float>(),
                                                          L1.kept.as<unsigned>(), L1.vals32.as<float>(), cD, cD32);
      else
        k_galerkin<float, 16><<<gg, kGalWarps * 32, 0, P->stream>>>(L1.nnzb, L.gal_ptr.as<int>(), L.gal_list.as<int2>(),
                                                           L.gal_row.as<int>(), L1.cols.as<int>(),
                                                           L.ap_vals.as<float>(), L.Q32.as<float>(),
                                                           L1.kept.as<unsigned>(), L1.vals32.as<float>(), cD, cD32);
    } else {
      L1.vals64.ensure(sizeof(double) * 256 * (size_t)L1.nnzb + 64);
      if (L.bs == 9)
        k_galerkin<double, 9><<<gg, kGalWarps * 32, 0, P->stream>>>(L1.nnzb, L.gal_ptr.as<int>(), L.gal_list.as<int2>(),
                                                           L.gal_row.as<int>(), L1.cols.as<int>(),
                                                           L.ap_vals.as<double>(), L.Q64.as<double>(),
                                                           L1.kept.as<unsigned>(), L1.vals64.as<double>(), cD, nullptr);
      else
        k_galerkin<double, 16><<<gg, kGalWarps * 32, 0, P->stream>>>(L1.nnzb, L.gal_ptr.as<int>(), L.gal_list.as<int2>(),
                                                            L.gal_row.as<int>(), L1.cols.as<int>(),
                                                            L.ap_vals.as<double>(), L.Q64.as<double>(),
                                                            L1.kept.as<unsigned>(), L1.vals64.as<double>(), cD, nullptr);
    }
    launched(P);
  }
  block_inverse_batch(P, inv, 16, F_NOT_SPD_JACOBI);
  lanczos_batched(P, P->l0_explicit ? 0 : 1, P->n_levels - 2);
  finish_lanczos(P);
  if (coarse_forked) BA_CUDA(cudaStreamWaitEvent(P->stream, P->ev_join, 0));
  if (check) check_flags(P);
  // V-cycle work vectors
  for (int k = 0; k < P->n_levels; ++k) {
    Level& L = P->levels[k];
    const size_t n = (size_t)(L.coarsest ? L.N : L.n * L.bs) + 64;
    const size_t es = fp32 ? sizeof(float) : sizeof(double);
    L.vx.ensure(es * n);
    L.vb.ensure(es * n);
    L.vr.ensure(es * n);
    L.vd.ensure(es * n);
    L.vq.ensure(es * n);
    L.vt.ensure(es * n);
    L.vs.ensure(es * n);
  }
  fused_vcycle_setup(P);
}

}  // namespace ba
