// sr_metrics: the accuracy measures of the recovery experiments (Sec. IV-A)
// on the device -- the cosine similarity of Eq. 6 and the relative error up
// to a global phase -- for a batch of estimates against reference signals.
//
// One thread-block cluster per problem. Every CTA of the cluster sums its
// slice of the vectors (compensated two-sum: Re and Im of <x_hat, x>,
// ||x_hat||^2, ||x||^2); rank 0 gathers the CTAs' totals through distributed
// shared memory in a fixed order, forms the optimal phase
// c = <x_hat, x> / |<x_hat, x>|, and every CTA then sums its slice of
// |c x_hat - x|^2 directly (the expanded form ||x_hat||^2 + ||x||^2 -
// 2 |<x_hat, x>| loses the small errors to cancellation in FP32). No global
// scratch, no atomics: the result is the same bit for bit on every call.
#include <cooperative_groups.h>

#include <algorithm>
#include <string>

#include "sr_device.cuh"
#include "sr_internal.h"

namespace cg = cooperative_groups;

namespace sr {
namespace {

constexpr int kMetricThreads = 512;
constexpr int kMaxClusterCtas = 8;  // portable cluster size

// Block-wide compensated sums of K values; results valid in thread 0.
// red holds 2 * K * 32 floats.
template <int K>
__device__ __forceinline__ void block_sums(fsum2 (&acc)[K], float* red, float (&out)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      fsum2 o{__shfl_down_sync(0xffffffffu, acc[k].s, off), __shfl_down_sync(0xffffffffu, acc[k].c, off)};
      if ((threadIdx.x & 31) + off < 32) acc[k] = acc_merge(acc[k], o);
    }
  }
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      red[(k * 32 + warp) * 2] = acc[k].s;
      red[(k * 32 + warp) * 2 + 1] = acc[k].c;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      fsum2 T{red[k * 64], red[k * 64 + 1]};
      for (int w = 1; w < nwarp; ++w) T = acc_merge(T, fsum2{red[(k * 32 + w) * 2], red[(k * 32 + w) * 2 + 1]});
      out[k] = T.s + T.c;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kMetricThreads) k_metrics(const float2* __restrict__ xh, const float2* __restrict__ xr,
                                                           int64_t n, float* __restrict__ cos_out,
                                                           float* __restrict__ err_out) {
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ float red[2 * 4 * 32];
  __shared__ float s_tot[4];    // this CTA's slice totals: Re ip, Im ip, ||x_hat||^2, ||x||^2 (then residual)
  __shared__ float2 s_phase;    // rank 0: the optimal phase c
  const int b = blockIdx.y;
  const int rank = (int)cluster.block_rank(), nrank = (int)cluster.num_blocks();
  const int64_t len = (n + nrank - 1) / nrank;
  const int64_t lo = (int64_t)rank * len, hi = min(n, lo + len);
  const float2* a = xh + (size_t)b * n;
  const float2* r = xr + (size_t)b * n;

  // pass 1: <x_hat, x> = sum conj(x_hat) x, and the two squared norms
  fsum2 acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const float2 u = a[i], v = r[i];
    acc_add(acc[0], fmaf(u.x, v.x, u.y * v.y));
    acc_add(acc[1], fmaf(u.x, v.y, -u.y * v.x));
    acc_add(acc[2], cabs2(u));
    acc_add(acc[3], cabs2(v));
  }
  float tot[4];
  block_sums<4>(acc, red, tot);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) s_tot[k] = tot[k];
  cluster.sync();
  float nr = 0.f;
  if (rank == 0 && threadIdx.x == 0) {
    fsum2 T[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int q = 0; q < nrank; ++q) {
      const float* t = cluster.map_shared_rank(s_tot, q);
      for (int k = 0; k < 4; ++k) acc_add(T[k], t[k]);
    }
    const float ipr = T[0].s + T[0].c, ipi = T[1].s + T[1].c;
    const float nh = T[2].s + T[2].c;
    nr = T[3].s + T[3].c;
    const float mag = hypotf(ipr, ipi);
    s_phase = mag > 0.f ? make_float2(ipr / mag, ipi / mag) : make_float2(1.f, 0.f);
    if (cos_out) cos_out[b] = mag / (sqrtf(nh) * sqrtf(nr));
  }
  cluster.sync();  // rank 0 has read every slice total and published the phase
  const float2 c = *cluster.map_shared_rank(&s_phase, 0);

  // pass 2: || c x_hat - x ||^2
  fsum2 res[1] = {{0.f, 0.f}};
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const float2 d = csub(cmul(c, a[i]), r[i]);
    acc_add(res[0], cabs2(d));
  }
  float rt[1];
  block_sums<1>(res, red, rt);
  if (threadIdx.x == 0) s_tot[0] = rt[0];
  cluster.sync();
  if (rank == 0 && threadIdx.x == 0) {
    fsum2 T{0.f, 0.f};
    for (int q = 0; q < nrank; ++q) acc_add(T, *cluster.map_shared_rank(&s_tot[0], q));
    if (err_out) err_out[b] = sqrtf(T.s + T.c) / sqrtf(nr);
  }
  cluster.sync();  // no CTA leaves while rank 0 still reads its shared memory
}

}  // namespace
}  // namespace sr

extern "C" {

sr_status sr_metrics(const void* x_hat, const void* x_ref, int64_t n, int B, float* cos_out, float* relerr_out,
                     void* stream) {
  if (!x_hat || !x_ref) {
    sr::set_last_error("NULL array argument");
    return SR_ERR_INVALID_ARG;
  }
  if (n < 1 || B < 1) {
    sr::set_last_error("need n >= 1 and B >= 1");
    return SR_ERR_INVALID_ARG;
  }
  if (B > 65535) {
    sr::set_last_error("B must be <= 65535");
    return SR_ERR_UNSUPPORTED;
  }
  if (!cos_out && !relerr_out) return SR_OK;
  // CTAs per problem: one per 16k elements, a power of two up to 8
  int ctas = 1;
  while (ctas < sr::kMaxClusterCtas && (int64_t)ctas * 16384 < n) ctas *= 2;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas, B, 1);
  cfg.blockDim = dim3(sr::kMetricThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = static_cast<cudaStream_t>(stream);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, sr::k_metrics, static_cast<const float2*>(x_hat),
                                           static_cast<const float2*>(x_ref), n, cos_out, relerr_out);
  sr::count_launch();
  if (e != cudaSuccess) {
    cudaGetLastError();
    sr::set_last_error(std::string("launch(metrics): ") + cudaGetErrorString(e));
    return SR_ERR_CUDA;
  }
  return SR_OK;
}

}  // extern "C"
