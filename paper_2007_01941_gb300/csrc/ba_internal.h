// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ba.h"

namespace ba {

constexpr int kNull = 16;        // near-nullspace dimension (Section 3.3)

// arrays of dense blocks inverted by one launch (each: n blocks from `in`, written to
// out64 and, if given, out32; `start` is the first block's index in the launch)
struct BlockInvSeg {
  const double* in;
  double* out64;
  float* out32;
  int n, start;
};
constexpr int kMaxInvSegs = 16;
struct BlockInvBatch {
  BlockInvSeg s[kMaxInvSegs];
  int nseg, total;
};
constexpr int kMaxSmooth = 8;    // Chebyshev steps per smoothing pass
// per level: theta, delta, sigma_1, lambda_max, pad, Lanczos alphas (8..15) and betas
// (16..23), then (c1, c2) of Chebyshev steps 1 .. kMaxSmooth - 1 (24 + 2 (k - 1))
constexpr int kChebSlots = 24 + 2 * kMaxSmooth;
constexpr int kScalars = 64;     // device scalar slots per problem

// Error raised inside the library; converted to a ba_status at the C boundary.
struct Error : std::runtime_error {
  ba_status status;
  Error(ba_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define BA_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      throw ::ba::Error(e_ == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA, \
                        std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)

#define BA_REQUIRE(cond, status, msg)                   \
  do {                                                  \
    if (!(cond)) throw ::ba::Error((status), (msg));    \
  } while (0)

// Device buffer that keeps its capacity across calls.
struct DBuf {
  void* p = nullptr;
  size_t cap = 0;
  template <typename T> T* as() const { return static_cast<T*>(p); }
  void ensure(size_t bytes) {
    if (bytes <= cap && p) return;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t b = bytes ? bytes : 16;
    BA_CUDA(cudaMalloc(&p, b));
    cap = b;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

// Slots of the device scalar array.
enum Scalar : int {
  S_COST = 0,      // 1/2 sum |f|^2
  S_RR = 1,        // r.r
  S_RZ = 2,        // r.z (current)
  S_PQ = 3,        // p.q
  S_ALPHA = 4,
  S_BETA = 5,
  S_BB = 6,        // b.b
  S_TMP0 = 7,
  S_TMP1 = 8,
  S_TMP2 = 9,
  S_MODEL = 10,    // model reduction terms
  S_COST_NEW = 11,
  S_ITER = 12,     // PCG iterations done (graph path)
  S_Q = 13,        // PCG quadratic model Q_i = 1/2 x^T S x - x^T b
  S_DQ = 14,       // Q_i - Q_{i-1}
  S_LANCZOS = 16,  // 16 .. 31: alphas / betas of the Lanczos recurrences
  S_LANCZOS_END = 32,
};

// Device error flags.
enum Flag : int {
  F_NOT_SPD_POINT = 0,
  F_NOT_SPD_JACOBI = 1,
  F_NOT_SPD_COARSE = 2,
  F_BREAKDOWN = 3,
  F_HASH_OVERFLOW = 4,
  F_NONFINITE = 5,
  F_WAIT_TIMEOUT = 6,   // a bounded wait in a kernel gave up (its results are not valid)
  F_PATTERN = 7,        // a level-0 block's mirror is missing from the covisibility pattern
  F_COUNT = 8
};

struct Level {
  int n = 0, bs = 0;            // nodes, dofs per node
  int nnzb = 0;                 // block nonzeros of the operator / covisibility pattern
  int maxrow = 1;               // longest block row
  DBuf row_ptr, cols, W;        // BSR pattern (int32) and covisibility counts (int64)
  DBuf vals64, vals32;          // operator blocks [nnzb][bs][bs]
  DBuf valsdf;                  // level 0 in mixed precision: FP64 blocks as (hi, lo) float pairs
  DBuf sptr, sidx;              // strength-ordered neighbour lists
  int n_strength = 0;
  DBuf agg;                     // int32 [n] aggregate (= next-level node) of each node
  int n_agg = 0;
  int agg_max = 1;              // members of the largest aggregate
  DBuf agg_ptr, agg_mem;        // member lists of the next-level nodes
  DBuf pair_ptr, pairs, blk_row; // level 0: observation pairs per work block (int [n_up+1], int2), block rows
  DBuf up_blk, mirror;          // level 0: blocks on and above the diagonal and their transposes
  DBuf gal_ptr, gal_list, gal_row;  // A P blocks (block, fine row) per block of the next level, its rows
  DBuf ap_ptr, ap_cols, ap_lptr, ap_list, ap_vals;  // A P blocks (bs x 16) per fine row, their A blocks
  int ap_nnzb = 0;
  int n_up = 0;
  DBuf K;                       // double [n][bs][16] near-nullspace rows
  DBuf Q64, Q32;                // double/float [n][bs][16] prolongator blocks
  DBuf kept;                    // uint32 [n] kept-dof masks of this level's nodes
  DBuf Dblk, Dinv64, Dinv32;    // diagonal blocks and their inverses [n][bs][bs]
  DBuf Dblk32;                  // FP32 copy of the diagonal blocks (mixed precision)
  DBuf cheb;                    // double[kChebSlots]: Chebyshev parameters, Lanczos data, step coefficients
  bool coarsest = false;
  int N = 0;                    // coarsest: dense size n*bs
  DBuf Ainv;                    // coarsest: double [N][N]
  DBuf vx, vb, vr, vd, vq, vt, vs;  // V-cycle vectors in the level's precision
  // restriction into this level folded into the V-cycle's next kernel (a small coarsest
  // level's solve; the first smoothing kernel of a smoothed coarse level, FP32 hierarchy,
  // >= 2 pre-smoothing steps): on a smoothed coarse level, its fine members per operator
  // block (gptr, gmem) and the blocks M_aj = A_aj D_j^-1 / theta; on the level above it,
  // t_i = Q_i^T s_i
  bool folded = false;
  DBuf gptr, gmem, mvals32;
  DBuf rt;
};

}  // namespace ba

struct ba_problem {
  ba_options opt;
  cudaStream_t stream = nullptr;
  int n_c = 0, n_p = 0, n_o = 0;
  int n_p_obs = 0;              // points with at least one observation (internal prefix)
  int n_sm = 0;
  std::string err;
  long long launches = 0;
  int stage = 0;                // 0 created, 1 linearized, 2 schur, 3 mg, 4 solved

  // observation graph in internal order (points sorted by first camera, obs by point, camera)
  ba::DBuf obs_user;            // int32 [n_o] internal obs -> caller obs index
  ba::DBuf obs_cam;             // int32 [n_o] camera of each internal obs
  ba::DBuf obs_ptu;             // int32 [n_o] caller point index of each internal obs
  ba::DBuf obs_pt;              // int32 [n_o] internal point of each internal obs
  ba::DBuf pt_ptr;              // int32 [n_p + 1]
  ba::DBuf pt_user;             // int32 [n_p] internal point -> caller point
  ba::DBuf cam_ptr, cam_obs;    // camera-major CSR over internal obs
  int n_tiles = 0, n_chunks = 0, k3_window = 0;
  int k3_grid[2] = {0, 0};       // Schur product CTAs per launch (FP32, FP64), set at first use
  int k3_grid_bulk = 0;          // the same for the FP32 product with bulk-staged records
  int k3_grid_df = 0;           // the same for the paired-FP32 product
  int k3_grid_rc = 0;           // the same for the FP64 product in recompute mode
  bool l0_explicit = false;     // V-cycle level 0 uses the assembled S (set by the multigrid setup)
  bool outer_explicit = false;  // the PCG product uses the FP64-valued blocks of the assembled S
  bool vc_ready = false;        // the fused-phase V-cycle applies (set by the multigrid setup)
  bool j64_valid = false;       // J64 holds the current records (mixed precision forms it on demand)
  ba::DBuf lz_vec, lz_red, lz_cnt, lz_ptr;  // batched Lanczos vectors, reductions, counters, pointers
  unsigned k3_calls = 0;        // alternates the tile order of successive Schur products
  ba::DBuf tile_pt;             // int32 [n_tiles + 1] point ranges of <=32-obs warp tiles
  ba::DBuf tile_desc;           // int4 [n_tiles] {first obs, obs count, first point, start mask}
  ba::DBuf tile_perm;           // uint8 [n_tiles][32] camera order of a tile's lanes (bit 7: run start)
  ba::DBuf chunk_tile;          // int32 [n_chunks + 1] tile ranges per matvec CTA
  ba::DBuf chunk_cam;           // int32 [2 n_chunks] lowest / highest camera of a chunk
  size_t ld = 0;                // leading dimension of per-observation SoA arrays
  size_t ldp = 0;               // leading dimension of per-point SoA arrays
  int max_row_contrib = 0;      // max_c sum_{o in c} |obs(point(o))| (hash sizing)
  int max_pt_obs = 0;           // most observations of one point

  // linearisation (SoA, internal order)
  ba::DBuf camx;                // double [n_c][24] per-camera rotation data
  ba::DBuf fres;                // double [n_o][2] residuals
  ba::DBuf J64;                 // double [n_o][24] Jacobian records (F row-major, then E)
  ba::DBuf J32;                 // float copy of the records (mixed precision)
  ba::DBuf J32lo;               // float rounding residual J64 - J32 (mixed precision)
  ba::DBuf cams_lin, pts_lin;   // copies of the linearisation point (adjoint, nullspace)
  ba::DBuf obs_lin;             // copy of the observations of the last linearisation

  // Schur reduction
  double lambda = 0.0;
  ba::DBuf Dc, Dp;              // double [n_c*9], [ldp][3] (internal points, SoA)
  ba::DBuf Cinv64, Cinv32;      // [6][ldp]
  ba::DBuf Cinv32lo;            // [6][ldp] float rounding residual Cinv64 - Cinv32
  ba::DBuf xsplit;              // float2 [n_c][9] hi/lo split of a camera vector
  ba::DBuf camdf;               // float2 [n_c][28] split rotation data and parameters (mixed)
  ba::DBuf wpdf;                // float2 [3][ldp] split C_p^-1 g_p (mixed)
  ba::DBuf Xdf;                 // float2 [6][ldp] X = G^-1 (C_p + D_p = G G^T) as float pairs (mixed)
  ba::DBuf gc, gp, wp, rhs;     // g_c [n_c*9], g_p [3][ldp], C^-1 g_p [3][ldp], b [n_c*9]
  ba::DBuf Dc32;                // float copy of D_c
  ba::DBuf Scc;                 // double [n_c][81] diagonal blocks S_cc
  ba::DBuf Scc_inv, Scc_inv32;  // their inverses (point-block-Jacobi), FP64 and FP32
  ba::DBuf ptsdf;               // float2 [n_p][3]: the points of the current linearisation as float pairs
  ba::DBuf cam_ubnd;            // float [n_c][9]: diag(sum_o F_o^T F_o), bounds of the assembly's column sums
  ba::DBuf pc_diag;             // float [n_c][9]: the mixed-precision hierarchy's extra damping (see below)
  ba::DBuf Scc_pc;              // double [2][n_c][81]: S_cc with that damping, and its FP64 inverse (scratch)
  bool pc_shift = false;        // pc_diag holds (mu - lambda) max(diag(J^T J), 1e-6), mu = precond_lambda_min

  // multigrid hierarchy
  std::vector<ba::Level> levels;
  int n_levels = 0;
  bool sym_ready = false;       // symbolic hierarchy built (depends on the graph only)

  // PCG
  ba::DBuf x, r, z, p, q, y32a, y32b;
  ba::DBuf delta_c, delta_p;    // last solve (internal layout: [n_c*9], [3][ldp])
  int pcg_iters = 0;
  double pcg_rel = 0.0;
  double cost = 0.0;
  double lm_nu = 2.0;

  // reductions and flags
  ba::DBuf scal;                // double [kScalars]
  ba::DBuf partial;             // double [partial_cap]
  ba::DBuf partial2;            // double: per-CTA partial sums of the PCG's fused p.q
  ba::DBuf rzpart;              // double [n_c]: each level-0 row's share of r.z (fused V-cycle)
  ba::DBuf counter;             // unsigned [8]
  ba::DBuf flags;               // int [F_COUNT]
  double* h_scal = nullptr;     // pinned host mirror
  double* h_cheb = nullptr;     // pinned [16][kChebSlots] host copies of the levels' Chebyshev data
  int* h_flags = nullptr;
  ba::DBuf scratch;             // general scratch
  ba::DBuf scratch2;

  // PCG as one CUDA graph (a first iteration, then a device-driven while loop);
  // rebuilt whenever a setup call may have moved buffers
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t pcg_exec = nullptr;
  uint64_t pcg_graph_key = 0;   // signature of what the PCG graph was captured with
  bool graphs_ok = true;        // false after a failed build: eager fallback
  long long pcg_graph_head = 0, pcg_graph_body = 0;  // kernels per graph part

  // side stream of the multigrid setup (the prolongator QR chain runs beside the assembly)
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // point-partitioned solve: the all-reduce hook and the whole problem's observation graph
  // (host, global point ids), from which the level-0 covisibility is built
  ba_allreduce_fn part_fn = nullptr;
  void* part_user = nullptr;
  std::vector<int> part_cam, part_pt;
  std::vector<double> part_buf;

  // optional CUDA-event timing of selected kernel classes
  bool ktime = false;
  std::vector<cudaEvent_t> ev_pool;
  struct KRec { int cls; cudaEvent_t a, b; };
  std::vector<KRec> krec;
};

namespace ba {
// Records a CUDA event pair around the launches made during its lifetime when
// kernel timing is enabled on the problem.
struct KernelTimer {
  ba_problem* P;
  int cls;
  cudaEvent_t a = nullptr, b = nullptr;
  KernelTimer(ba_problem* p, int c);
  ~KernelTimer();
};
void kernel_timing_enable(ba_problem* P, bool on);
void kernel_timing_get(ba_problem* P, int cls, double* ms, long long* n);
}  // namespace ba

namespace ba {

// ---- stream helpers -------------------------------------------------------
void sync(ba_problem* P);
void fetch_scalars(ba_problem* P, int first, int count);  // async copy + sync
// point-partitioned solve: sum a device array (n doubles, in place) or a scalar slot over
// the ranks through the caller's hook (no-ops on an unpartitioned problem)
void part_allreduce(ba_problem* P, double* dev, size_t n);
double fetch_sum(ba_problem* P, int slot);
inline bool partitioned(const ba_problem* P) { return P->part_fn != nullptr; }
void check_flags(ba_problem* P);                          // sync, read, raise
// check_flags without its own synchronisation: raises from the flags last copied to the host
void raise_flags(ba_problem* P);
// scalars [first, first + count) and the flags to the host in one synchronisation, then
// raise_flags; fetch_sum_checked also sums the slot over a partitioned problem's ranks
void fetch_checked(ba_problem* P, int first, int count);
double fetch_sum_checked(ba_problem* P, int slot);
void clear_flags(ba_problem* P);
void launched(ba_problem* P);                              // count + check launch error

// host vector -> device buffer (grown as needed) on the problem's stream
template <typename T>
void upload(ba_problem* P, DBuf& dst, const std::vector<T>& src) {
  dst.ensure(sizeof(T) * std::max<size_t>(src.size(), 1));
  if (!src.empty())
    BA_CUDA(cudaMemcpyAsync(dst.p, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, P->stream));
}

// Launches kern on the problem's stream; with opt.overlap_launches as a programmatic
// dependent launch (the kernel must call pdl_wait() before it touches memory).
template <typename... KArgs, typename... Args>
void launch_k(ba_problem* P, void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = P->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = P->opt.overlap_launches ? 1 : 0;
  BA_CUDA(cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...));
  launched(P);
}

// ---- graph preprocessing (graph.cu) ----------------------------------------
void build_graph(ba_problem* P, const int32_t* cam_idx_dev, const int32_t* pt_idx_dev);

// ---- linearisation (linearize.cu) ------------------------------------------
void linearize(ba_problem* P, const double* cams, const double* pts, const double* obs);
double cost_at(ba_problem* P, const double* cams, const double* pts, const double* obs);
// the same cost into scalar S_COST_NEW, not fetched
void cost_at_async(ba_problem* P, const double* cams, const double* pts, const double* obs);
// the FP64 Jacobian records; in mixed precision formed on first use from J32 + J32lo
// (exactly the doubles the paired-FP32 linearisation computed), never inside a capture
double* jacobian64(ba_problem* P);

// ---- Schur reduction and implicit operator (schur.cu) -----------------------
// check = false leaves the flags for the caller's next fetch_checked (the LM step's PCG)
void schur_setup(ba_problem* P, double lambda, bool check = true);
// y = S x on internal camera vectors; T selects the FP64 or FP32 storage kernel.
void matvec64(ba_problem* P, const double* x, double* y);
void matvec32(ba_problem* P, const float* x, float* y);
// the same products without writing D_c x first (y must already hold it)
void matvec64_accumulate(ba_problem* P, const double* x, double* y);
void matvec32_accumulate(ba_problem* P, const float* x, float* y);
bool outer_df(ba_problem* P);                                         // mixed mode, paired-FP32 outer product
void split_vector(ba_problem* P, const double* x, const double* Dc, double* y);  // xsplit = split(x); y = Dc o x
void matvec_df_accumulate(ba_problem* P, double* y);                   // y += S x - Dc x from xsplit
void lanczos_batched(ba_problem* P, int first, int last);  // levels first..last, all assembled
// A_l P_l of a smoothed level: pattern (once per problem) and blocks
void build_ap(ba_problem* P, Level& L);
void fused_vcycle_setup(ba_problem* P);
// z = M r; rz_part (optional): per level-0 row, its share of r.z (one value per block row)
// first_done: the level-0 pre-smoothing step 0 on r was already formed (by
// fused_update_first), so the cycle starts at step 1
void fused_vcycle(ba_problem* P, const double* r, double* z, double* rz_part, bool first_done);
struct PcgCheck;
// the PCG update with the assembled S (x += alpha p, r -= alpha q, r.r, the stopping test)
// fused with the next V-cycle's level-0 pre-smoothing step 0 on the new r
void fused_update_first(ba_problem* P, double* x, double* r, const double* p, const double* q, const PcgCheck& ck);
// assembled level-0 S: FP32 blocks only (the Galerkin product's input), FP64 blocks, or
// paired-FP32 arithmetic giving the FP64 blocks and their FP32 roundings
enum ExplicitMode { EX_FP32, EX_FP64, EX_PAIRED };
void explicit_schur(ba_problem* P, Level& L0, ExplicitMode mode);
void back_substitute_to(ba_problem* P, const double* dc, double* out_int, double* out_user);
void reduced_rhs(ba_problem* P, const double* vc, const double* vp_user, double* out);

// ---- multigrid setup (mg_setup.cu) ------------------------------------------
void mg_setup(ba_problem* P, bool check = true);
void covisibility_level0(ba_problem* P, Level& L);

// ---- solve (solve.cu) -------------------------------------------------------
void precond_apply(ba_problem* P, const double* r, double* z);
// check_setup: raise the flags left by an unchecked schur_setup / mg_setup first
void pcg(ba_problem* P, const double* rhs, double* dc, bool check_setup = false);
void lm_step(ba_problem* P, double* cams, double* pts, const double* obs, double* lam,
             int* accepted, double* cost);

// ---- adjoint (adjoint.cu) ---------------------------------------------------
void adjoint(ba_problem* P, const double* dL_ddelta, double* dL_dobs, double* dL_dcams,
             double* dL_dpts);

// ---- reductions (reduce.cu) -------------------------------------------------
// out_slot = sum_i a_i b_i (a, b of type T, length n), deterministic two-stage.
void dot64(ba_problem* P, const double* a, const double* b, size_t n, int slot);
void dot32(ba_problem* P, const float* a, const float* b, size_t n, int slot);
int reduce_blocks(ba_problem* P, size_t n);

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// Every device buffer of a problem and of a level (released by ba_destroy; their addresses
// and capacities are part of the PCG graph's signature).
template <class F>
void for_each_problem_buf(ba_problem* P, F&& f) {
  DBuf* bufs[] = {&P->obs_user, &P->obs_cam, &P->obs_ptu, &P->obs_pt, &P->pt_ptr, &P->pt_user, &P->cam_ptr,
                  &P->cam_obs, &P->tile_pt, &P->tile_desc, &P->tile_perm, &P->lz_vec, &P->lz_red, &P->lz_cnt,
                  &P->lz_ptr, &P->chunk_tile, &P->chunk_cam, &P->camx, &P->fres, &P->J64, &P->J32, &P->J32lo,
                  &P->cams_lin, &P->pts_lin, &P->obs_lin, &P->Dc, &P->Dp, &P->Cinv64, &P->Cinv32, &P->Cinv32lo,
                  &P->xsplit, &P->camdf, &P->wpdf, &P->Xdf, &P->gc, &P->gp, &P->wp, &P->rhs, &P->Dc32, &P->Scc,
                  &P->Scc_inv, &P->Scc_inv32, &P->cam_ubnd, &P->pc_diag, &P->Scc_pc, &P->ptsdf, &P->x, &P->r,
                  &P->z, &P->p, &P->q, &P->y32a, &P->y32b, &P->delta_c, &P->delta_p, &P->scal, &P->partial,
                  &P->partial2, &P->rzpart, &P->counter, &P->flags, &P->scratch, &P->scratch2};
  for (DBuf* b : bufs) f(*b);
}

template <class F>
void for_each_level_buf(Level& L, F&& f) {
  DBuf* bufs[] = {&L.row_ptr, &L.cols, &L.W, &L.vals64, &L.vals32, &L.sptr, &L.sidx, &L.agg, &L.agg_ptr,
                  &L.agg_mem, &L.K, &L.Q64, &L.Q32, &L.kept, &L.Dblk, &L.Dinv64, &L.Dinv32, &L.cheb, &L.Ainv,
                  &L.vx, &L.vb, &L.vr, &L.vd, &L.vq, &L.vt, &L.vs, &L.pair_ptr, &L.pairs, &L.blk_row, &L.up_blk,
                  &L.mirror, &L.Dblk32, &L.valsdf, &L.ap_ptr, &L.ap_cols, &L.ap_lptr, &L.ap_list, &L.ap_vals,
                  &L.gal_ptr, &L.gal_list, &L.gal_row, &L.gptr, &L.gmem, &L.mvals32, &L.rt};
  for (DBuf* b : bufs) f(*b);
}

}  // namespace ba
