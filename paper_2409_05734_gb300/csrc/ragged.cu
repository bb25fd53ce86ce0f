// Ragged batches of independent problems: buckets of equal (n, m, L), each a
// batched plan with per-problem phases, run as concurrent stream branches that
// fork from and join into the caller's stream (graph-capturable).
#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "sr_internal.h"

namespace {

sr_status rfail(sr_status st, const std::string& msg) {
  sr::set_last_error(msg);
  return st;
}

#define SR_RCUDA(call, what)                                                               \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      cudaGetLastError();                                                                  \
      return rfail(SR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_));      \
    }                                                                                      \
  } while (0)

struct Bucket {
  int64_t n = 0, m = 0;
  int L = 0;
  std::vector<int> members;  // caller indices, in slot order
  int slot0 = 0;             // first slot of the bucket
  int64_t x_base = 0, y_base = 0;
  sr_plan* plan = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

// loss[t][member[s]] = scratch[iters * slot0(s) + t * B(s) + (s - slot0(s))]
__global__ void k_scatter_loss(const float* __restrict__ scratch, const int* __restrict__ member,
                               const int* __restrict__ slot0, const int* __restrict__ bsize, int count, int iters,
                               float* __restrict__ loss) {
  const int64_t total = (int64_t)count * iters;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(i % count);
    const int t = (int)(i / count);
    const int s0 = slot0[s], bs = bsize[s];
    loss[(int64_t)t * count + member[s]] = scratch[(int64_t)iters * s0 + (int64_t)t * bs + (s - s0)];
  }
}

}  // namespace

struct sr_ragged {
  int count = 0;
  int device = 0;
  std::vector<int64_t> x_off, y_off;
  int64_t x_total = 0, y_total = 0;
  std::vector<Bucket> buckets;
  cudaEvent_t fork = nullptr;
  int iters_cap = 0;
  float* d_loss = nullptr;   // [iters_cap * count] scratch
  int* d_member = nullptr;   // [count] per slot
  int* d_slot0 = nullptr;
  int* d_bsize = nullptr;
};

namespace {

// Runs fn(bucket) on every bucket's stream between a fork from and a join into `s`.
template <class F>
sr_status run_buckets(sr_ragged* r, cudaStream_t s, F fn) {
  SR_RCUDA(cudaEventRecord(r->fork, s), "cudaEventRecord(fork)");
  for (Bucket& b : r->buckets) {
    SR_RCUDA(cudaStreamWaitEvent(b.stream, r->fork, 0), "cudaStreamWaitEvent(fork)");
    sr_status st = fn(b);
    if (st != SR_OK) return st;
    SR_RCUDA(cudaEventRecord(b.done, b.stream), "cudaEventRecord(join)");
    SR_RCUDA(cudaStreamWaitEvent(s, b.done, 0), "cudaStreamWaitEvent(join)");
  }
  return SR_OK;
}

sr_status check_ragged(sr_ragged* r) {
  if (!r) return rfail(SR_ERR_INVALID_ARG, "ragged handle is NULL");
  int dev = -1;
  SR_RCUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != r->device) return rfail(SR_ERR_INVALID_ARG, "current CUDA device differs from the handle's device");
  return SR_OK;
}

}  // namespace

extern "C" {

sr_status sr_ragged_destroy(sr_ragged* r) {
  if (!r) return SR_OK;
  for (Bucket& b : r->buckets) {
    sr_plan_destroy(b.plan);
    if (b.stream) cudaStreamDestroy(b.stream);
    if (b.done) cudaEventDestroy(b.done);
  }
  if (r->fork) cudaEventDestroy(r->fork);
  cudaFree(r->d_loss);
  cudaFree(r->d_member);
  cudaFree(r->d_slot0);
  cudaFree(r->d_bsize);
  delete r;
  return SR_OK;
}

sr_status sr_ragged_create(int count, const int64_t* n, const int64_t* m, const int* L, const uint64_t* seeds,
                           int autotune, sr_ragged** out) {
  if (!out || !n || !m || !L || !seeds) return rfail(SR_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (count < 1) return rfail(SR_ERR_INVALID_ARG, "count must be >= 1");
  for (int i = 0; i < count; ++i)
    if (n[i] > m[i]) return rfail(SR_ERR_UNSUPPORTED, "ragged batches need n <= m (alpha >= 1)");
  sr_ragged* r = new (std::nothrow) sr_ragged();
  if (!r) return rfail(SR_ERR_OOM, "host allocation failed");
  r->count = count;
  if (cudaGetDevice(&r->device) != cudaSuccess) {
    delete r;
    return rfail(SR_ERR_CUDA, "cudaGetDevice");
  }
  // buckets of equal shape, largest work first
  std::map<std::tuple<int64_t, int64_t, int>, std::vector<int>> by_shape;
  for (int i = 0; i < count; ++i) by_shape[std::make_tuple(n[i], m[i], L[i])].push_back(i);
  for (auto& kv : by_shape) {
    Bucket b;
    std::tie(b.n, b.m, b.L) = kv.first;
    b.members = kv.second;
    r->buckets.push_back(b);
  }
  std::stable_sort(r->buckets.begin(), r->buckets.end(), [](const Bucket& a, const Bucket& b) {
    return (double)a.m * a.L * a.members.size() > (double)b.m * b.L * b.members.size();
  });
  r->x_off.assign(count, 0);
  r->y_off.assign(count, 0);
  std::vector<int> member, slot0, bsize;
  int slot = 0;
  for (Bucket& b : r->buckets) {
    b.slot0 = slot;
    b.x_base = r->x_total;
    b.y_base = r->y_total;
    for (size_t j = 0; j < b.members.size(); ++j) {
      const int i = b.members[j];
      r->x_off[i] = b.x_base + (int64_t)j * b.n;
      r->y_off[i] = b.y_base + (int64_t)j * b.m;
      member.push_back(i);
      slot0.push_back(b.slot0);
      bsize.push_back((int)b.members.size());
    }
    slot += (int)b.members.size();
    r->x_total += (int64_t)b.members.size() * b.n;
    r->y_total += (int64_t)b.members.size() * b.m;
  }
  sr_status st = SR_OK;
  for (Bucket& b : r->buckets) {
    const int B = (int)b.members.size();
    std::vector<uint64_t> sd(B);
    for (int j = 0; j < B; ++j) sd[j] = seeds[b.members[j]];
    if ((st = sr_plan_create(b.n, b.m, b.L, sd[0], &b.plan)) != SR_OK ||
        (st = sr::plan_set_problem_phases(b.plan, B, sd.data())) != SR_OK ||
        (st = sr_plan_reserve(b.plan, B)) != SR_OK) {
      sr_ragged_destroy(r);
      return st;
    }
    if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess) {
      sr_ragged_destroy(r);
      return rfail(SR_ERR_CUDA, "stream or event creation failed");
    }
    if (autotune && (st = sr_plan_autotune(b.plan, B, b.stream)) != SR_OK) {
      sr_ragged_destroy(r);
      return st;
    }
  }
  cudaError_t e = cudaEventCreateWithFlags(&r->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&r->d_member, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMalloc(&r->d_slot0, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMalloc(&r->d_bsize, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMemcpy(r->d_member, member.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r->d_slot0, slot0.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r->d_bsize, bsize.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    sr_ragged_destroy(r);
    return rfail(SR_ERR_CUDA, std::string("ragged setup: ") + cudaGetErrorString(e));
  }
  *out = r;
  return SR_OK;
}

sr_status sr_ragged_layout(const sr_ragged* r, int64_t* x_off, int64_t* y_off, int64_t* x_total, int64_t* y_total,
                           int* buckets) {
  if (!r) return rfail(SR_ERR_INVALID_ARG, "ragged handle is NULL");
  if (x_off) std::copy(r->x_off.begin(), r->x_off.end(), x_off);
  if (y_off) std::copy(r->y_off.begin(), r->y_off.end(), y_off);
  if (x_total) *x_total = r->x_total;
  if (y_total) *y_total = r->y_total;
  if (buckets) *buckets = (int)r->buckets.size();
  return SR_OK;
}

sr_status sr_ragged_reserve(sr_ragged* r, int iters) {
  sr_status st = check_ragged(r);
  if (st != SR_OK) return st;
  if (iters <= r->iters_cap) return SR_OK;
  cudaFree(r->d_loss);
  r->d_loss = nullptr;
  r->iters_cap = 0;
  SR_RCUDA(cudaMalloc(&r->d_loss, sizeof(float) * (size_t)iters * r->count), "cudaMalloc(loss scratch)");
  r->iters_cap = iters;
  return SR_OK;
}

sr_status sr_ragged_forward(sr_ragged* r, const void* x_cat, void* z_cat, void* stream) {
  sr_status st = check_ragged(r);
  if (st != SR_OK) return st;
  if (!x_cat || !z_cat) return rfail(SR_ERR_INVALID_ARG, "NULL array argument");
  const float2* x = static_cast<const float2*>(x_cat);
  float2* z = static_cast<float2*>(z_cat);
  return run_buckets(r, (cudaStream_t)stream, [&](Bucket& b) {
    return sr_forward(b.plan, x + b.x_base, z + b.y_base, (int)b.members.size(), b.stream);
  });
}

sr_status sr_ragged_spectral_init(sr_ragged* r, const float* y_cat, const void* v0_cat, int iters,
                                  const sr_spectral_opts* opts, void* x_cat, void* stream) {
  sr_status st = check_ragged(r);
  if (st != SR_OK) return st;
  if (!y_cat || !v0_cat || !x_cat) return rfail(SR_ERR_INVALID_ARG, "NULL array argument");
  const float2* v0 = static_cast<const float2*>(v0_cat);
  float2* x = static_cast<float2*>(x_cat);
  return run_buckets(r, (cudaStream_t)stream, [&](Bucket& b) {
    return sr_spectral_init(b.plan, y_cat + b.y_base, v0 + b.x_base, iters, opts, x + b.x_base,
                            (int)b.members.size(), b.stream);
  });
}

sr_status sr_ragged_gd_solve(sr_ragged* r, const float* y_cat, void* x_cat, int iters, const sr_gd_opts* opts,
                             float* loss_hist, void* stream) {
  sr_status st = check_ragged(r);
  if (st != SR_OK) return st;
  if (!y_cat || !x_cat) return rfail(SR_ERR_INVALID_ARG, "NULL array argument");
  if (iters < 0) return rfail(SR_ERR_INVALID_ARG, "iters must be >= 0");
  if (loss_hist && iters > r->iters_cap)
    return rfail(SR_ERR_INVALID_ARG, "loss history needs sr_ragged_reserve(iters) first");
  float2* x = static_cast<float2*>(x_cat);
  cudaStream_t s = (cudaStream_t)stream;
  st = run_buckets(r, s, [&](Bucket& b) {
    float* lh = loss_hist ? r->d_loss + (size_t)iters * b.slot0 : nullptr;
    return sr_gd_solve(b.plan, y_cat + b.y_base, x + b.x_base, iters, opts, lh, (int)b.members.size(), b.stream);
  });
  if (st != SR_OK || !loss_hist || iters == 0) return st;
  const int64_t total = (int64_t)iters * r->count;
  const int blocks = (int)std::min<int64_t>(1024, (total + 255) / 256);
  k_scatter_loss<<<blocks, 256, 0, s>>>(r->d_loss, r->d_member, r->d_slot0, r->d_bsize, r->count, iters, loss_hist);
  sr::count_launch();
  SR_RCUDA(cudaGetLastError(), "launch(scatter loss)");
  return SR_OK;
}

sr_status sr_ragged_check(sr_ragged* r) {
  sr_status st = check_ragged(r);
  if (st != SR_OK) return st;
  for (Bucket& b : r->buckets)
    if ((st = sr_plan_check(b.plan)) != SR_OK) return st;
  return SR_OK;
}

}  // extern "C"
