// Deterministic FP64 reductions and stream/flag helpers.
#include "ba_internal.h"
#include "device_util.cuh"

namespace ba {

constexpr int kRedBS = 256;

template <typename T>
__global__ void __launch_bounds__(kRedBS) k_dot(const T* __restrict__ a, const T* __restrict__ b,
                                                size_t n, double* partial, unsigned* counter,
                                                double* out) {
  pdl_wait();
  pdl_trigger();
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * kRedBS + threadIdx.x; i < n; i += (size_t)gridDim.x * kRedBS)
    acc += (double)a[i] * (double)b[i];
  grid_sum_store<kRedBS>(acc, partial, counter, out);
}

int reduce_blocks(ba_problem* P, size_t n) {
  long long b = (long long)((n + kRedBS * 4 - 1) / (kRedBS * 4));
  if (b < 1) b = 1;
  if (b > 2LL * P->n_sm) b = 2LL * P->n_sm;
  return (int)b;
}

void dot64(ba_problem* P, const double* a, const double* b, size_t n, int slot) {
  int g = reduce_blocks(P, n);
  launch_k(P, k_dot<double>, g, kRedBS, 0, a, b, n, P->partial.as<double>(), P->counter.as<unsigned>(),
           P->scal.as<double>() + slot);
}

void dot32(ba_problem* P, const float* a, const float* b, size_t n, int slot) {
  int g = reduce_blocks(P, n);
  launch_k(P, k_dot<float>, g, kRedBS, 0, a, b, n, P->partial.as<double>(), P->counter.as<unsigned>(),
           P->scal.as<double>() + slot);
}

void launched(ba_problem* P) {
  P->launches++;
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(BA_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
  }
}

void sync(ba_problem* P) { BA_CUDA(cudaStreamSynchronize(P->stream)); }

static cudaEvent_t take_event(ba_problem* P) {
  if (!P->ev_pool.empty()) {
    cudaEvent_t e = P->ev_pool.back();
    P->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  BA_CUDA(cudaEventCreate(&e));
  return e;
}

KernelTimer::KernelTimer(ba_problem* p, int c) : P(p), cls(c) {
  if (!P->ktime) return;
  cudaStreamCaptureStatus st;
  if (cudaStreamIsCapturing(P->stream, &st) != cudaSuccess || st != cudaStreamCaptureStatusNone) return;
  a = take_event(P);
  b = take_event(P);
  cudaEventRecord(a, P->stream);
}

KernelTimer::~KernelTimer() {
  if (!a) return;
  cudaEventRecord(b, P->stream);
  P->krec.push_back({cls, a, b});
}

void kernel_timing_enable(ba_problem* P, bool on) {
  sync(P);
  for (auto& r : P->krec) {
    P->ev_pool.push_back(r.a);
    P->ev_pool.push_back(r.b);
  }
  P->krec.clear();
  P->ktime = on;
}

void kernel_timing_get(ba_problem* P, int cls, double* ms, long long* n) {
  sync(P);
  double tot = 0.0;
  long long cnt = 0;
  for (auto& r : P->krec) {
    if (r.cls != cls) continue;
    float t = 0.f;
    BA_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    tot += t;
    ++cnt;
  }
  *ms = tot;
  *n = cnt;
}

void fetch_scalars(ba_problem* P, int first, int count) {
  BA_CUDA(cudaMemcpyAsync(P->h_scal + first, P->scal.as<double>() + first, sizeof(double) * count,
                          cudaMemcpyDeviceToHost, P->stream));
  sync(P);
}

void part_allreduce(ba_problem* P, double* dev, size_t n) {
  if (!P->part_fn || n == 0) return;
  P->part_buf.resize(n);
  BA_CUDA(cudaMemcpyAsync(P->part_buf.data(), dev, sizeof(double) * n, cudaMemcpyDeviceToHost, P->stream));
  sync(P);
  BA_REQUIRE(P->part_fn(P->part_buf.data(), n, P->part_user) == 0, BA_ERR_STATE, "the all-reduce hook failed");
  BA_CUDA(cudaMemcpyAsync(dev, P->part_buf.data(), sizeof(double) * n, cudaMemcpyHostToDevice, P->stream));
  sync(P);
}

double fetch_sum(ba_problem* P, int slot) {
  fetch_scalars(P, slot, 1);
  if (P->part_fn) {
    double v = P->h_scal[slot];
    BA_REQUIRE(P->part_fn(&v, 1, P->part_user) == 0, BA_ERR_STATE, "the all-reduce hook failed");
    P->h_scal[slot] = v;
  }
  return P->h_scal[slot];
}

void clear_flags(ba_problem* P) {
  BA_CUDA(cudaMemsetAsync(P->flags.p, 0, sizeof(int) * F_COUNT, P->stream));
}

static void read_flags_async(ba_problem* P) {
  BA_CUDA(cudaMemcpyAsync(P->h_flags, P->flags.p, sizeof(int) * F_COUNT, cudaMemcpyDeviceToHost, P->stream));
}

void fetch_checked(ba_problem* P, int first, int count) {
  BA_CUDA(cudaMemcpyAsync(P->h_scal + first, P->scal.as<double>() + first, sizeof(double) * count,
                          cudaMemcpyDeviceToHost, P->stream));
  read_flags_async(P);
  sync(P);
  raise_flags(P);
}

double fetch_sum_checked(ba_problem* P, int slot) {
  fetch_checked(P, slot, 1);
  if (P->part_fn) {
    double v = P->h_scal[slot];
    BA_REQUIRE(P->part_fn(&v, 1, P->part_user) == 0, BA_ERR_STATE, "the all-reduce hook failed");
    P->h_scal[slot] = v;
  }
  return P->h_scal[slot];
}

void check_flags(ba_problem* P) {
  read_flags_async(P);
  sync(P);
  raise_flags(P);
}

void raise_flags(ba_problem* P) {
  if (P->part_fn) {
    // partitioned solve: every rank raises the same error at the same point (a rank that
    // stopped alone would leave the others waiting in their next reduction)
    double fs[F_COUNT];
    for (int i = 0; i < F_COUNT; ++i) fs[i] = P->h_flags[i];
    BA_REQUIRE(P->part_fn(fs, F_COUNT, P->part_user) == 0, BA_ERR_STATE, "the all-reduce hook failed");
    for (int i = 0; i < F_COUNT; ++i) P->h_flags[i] = fs[i] > 0.0 ? 1 : 0;
  }
  const int* f = P->h_flags;
  if (f[F_HASH_OVERFLOW])
    throw Error(BA_ERR_LIMIT, "a covisibility row has more distinct neighbours than the hash capacity");
  if (f[F_NONFINITE]) throw Error(BA_ERR_INVALID_ARG, "non-finite value in the linearisation");
  if (f[F_NOT_SPD_POINT]) throw Error(BA_ERR_NOT_SPD, "a 3x3 point block C_p is not positive definite");
  if (f[F_NOT_SPD_JACOBI]) throw Error(BA_ERR_NOT_SPD, "a block-Jacobi diagonal block is not positive definite");
  if (f[F_NOT_SPD_COARSE]) throw Error(BA_ERR_NOT_SPD, "the coarsest operator is not positive definite");
  if (f[F_BREAKDOWN]) throw Error(BA_ERR_BREAKDOWN, "PCG breakdown");
  if (f[F_WAIT_TIMEOUT]) throw Error(BA_ERR_CUDA, "a kernel's bounded wait for its staged data gave up");
  if (f[F_PATTERN]) throw Error(BA_ERR_STATE, "covisibility pattern is not symmetric");
}

}  // namespace ba
