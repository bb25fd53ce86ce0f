// Persistent passes over ragged batches: one launch runs the same pass index
// of a GD or power-iteration step (Sec. II-B) for every problem of a ragged
// batch whose four-step geometry it covers, whatever the problem's length.
//
// A launch covers segments: buckets of problems of one shape (n, m, L), each
// with its own batched plan (per-problem phases, exchange buffers, partial
// sums). A segment's descriptor holds the pass arguments the bucket's plan
// would launch its own kernel with, its first tile in the launch, and which
// line length and pass kind it runs; the values that change from call to call
// or step to step (the caller's concatenated x and y, the step's warm-up
// factor, the loss-history row, the power iteration's ping-pong banks) come
// as kernel parameters. Every CTA of the persistent grid takes a contiguous
// chunk of the launch's tiles, so it mostly stays within one segment; per
// tile it finds the segment and runs the FIRST / MID / LAST / fused body of
// passes.cuh for that line length, with the same TMA staging and prefetch of
// the next tile as the single-plan kernels (lines of up to 512 points; the
// 4-line tiles of 1024-point lines read their input directly).
//
// Every CTA has 256 threads and tiles of 4096 values: lines of 128, 256, 512
// and 1024 points as 32, 16, 8 and 4 lines per tile. The line twiddles come
// from one table of W_1024^k in global memory (L1-resident), read with the
// stride 1024 / ELL, so shared memory holds only the staging buffer, the FFT
// scratch and the row twiddles.
#include <algorithm>

#include "passes.cuh"
#include "sr_ragged.h"

namespace sr {
namespace {

constexpr int kRgThreads = 256;

// Byte layout of the dynamic shared memory (relative to a 1024-byte-aligned
// base): TMA staging (32 KB), FFT scratch (the padded layout of 4096 values),
// row twiddles (16 x up to 32 lines), two copies of the segment arguments,
// the barrier.
struct RgSmem {
  static constexpr size_t stage = 0;
  static constexpr size_t scratch = 4096 * 8;
  static constexpr size_t rowtw = scratch + 4096 * 17 / 16 * 8;
  static constexpr size_t args = rowtw + 16 * 32 * 8;
  static constexpr size_t bar = args + 2 * sizeof(PassArgs);
  static constexpr size_t total = bar + 16;
};

__device__ __forceinline__ int rg_find(const int* tile0, int nseg, int s, int idx) {
  while (s + 1 < nseg && idx >= tile0[s + 1]) ++s;
  return s;
}

// The pass arguments of segment sg for this launch: its descriptor with the
// call's and the step's values filled in.
__device__ __forceinline__ void rg_patch(PassArgs& a, const RaggedSeg& sg, const RaggedDyn& d) {
  a.xin = d.x ? d.x + sg.x_off : nullptr;
  a.xout = d.xo ? d.xo + sg.x_off : nullptr;
  if (a.op == kOpGdEpilogue || a.op == kOpSpecEpilogue) a.y = d.y + sg.y_off;
  a.mu_scale = d.mu_scale;
  a.loss_out = (d.loss_base && sg.record_loss)
                   ? d.loss_base + (int64_t)d.iters * sg.slot0 + (int64_t)d.t * sg.bsize
                   : nullptr;
  a.lam = d.lam;
  a.weight_mode = d.weight_mode;
  a.shift = d.shift;
  if (sg.spec) {
    // step `parity` writes bank[parity] and reads the previous step's bank
    a.norm_in = sg.bank[1 - d.parity];
    a.norm_in_count = d.first_step ? sg.count_first : sg.count_steady;
    if (sg.kind == kRgLF || sg.kind == kRgLast) a.part_out = sg.bank[d.parity];
  }
}

// Copies segment s's descriptor into shared-memory copy `slot` and patches it
// (warp 0; the caller synchronises before any thread reads it).
__device__ __forceinline__ void rg_load_args(PassArgs* dst, const RaggedSeg& sg, const RaggedDyn& d) {
  if (threadIdx.x >= 32) return;
  const uint4* src = reinterpret_cast<const uint4*>(&sg.a);
  uint4* out = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(PassArgs) / 16); i += 32) out[i] = src[i];
  __syncwarp();
  if (threadIdx.x == 0) rg_patch(*dst, sg, d);
  __syncwarp();
}

// Problem and first line of local tile `local` of a segment with T lines per tile.
__device__ __forceinline__ void rg_tile_pos(const PassArgs& a, int local, int& b, int& g0) {
  b = local / a.cpp;
  g0 = (local - b * a.cpp) * a.T;
}

struct RgCtx {
  const RaggedSeg* segs;
  const int* tile0;  // shared
  int nseg;
  int c1;            // end of this CTA's chunk
  unsigned char* smem;
  float2* scratch;
  float2* rowtw;
  const float2* tw;  // W_1024 table
  uint32_t bar, stage;
  int waits;         // staged tiles consumed so far (mbarrier phase)
};

// Thread 0: issues the TMA loads of tile idx (if it is a staged tile).
__device__ __forceinline__ void rg_issue(const RgCtx& cx, int idx, int s) {
  if (idx >= cx.c1) return;
  s = rg_find(cx.tile0, cx.nseg, s, idx);
  const RaggedSeg& sg = cx.segs[s];
  if (!sg.tma) return;
  int b, g0;
  rg_tile_pos(sg.a, idx - cx.tile0[s], b, g0);
  fence_proxy_async_smem();
  issue_rows(&sg.a.tmap, b * sg.a.nl + g0, sg.a.ell, sg.a.T, sg.a.T * 128, cx.stage, cx.bar);
}

// A run of tiles [i0, i1) of one segment of a pipelined pass (MID, fused
// LAST/FIRST, LAST) with lines of ELL points: per tile, its input lines into
// registers (from the staging buffer, or straight from the exchange buffer for
// unstaged tiles), the refill of the staging buffer with the next tile of the
// chunk, then the body. False when a staged load never completed (recorded in
// a.err).
template <int ELL, int KIND>
__device__ __noinline__ bool rg_run(RgCtx& cx, const PassArgs& a, int s, int i0, int i1, TileScalars& sh) {
  constexpr int T = 4096 / ELL;
  using TL = Tile<ELL, T>;
  constexpr int TWS = 1024 / ELL;
  static_assert(TL::THREADS == kRgThreads, "ragged tiles are 256 threads");
  int t, p;
  thread_coords<TL>(t, p);
  const int cpp = a.cpp, tile0 = cx.tile0[s];
  for (int idx = i0; idx < i1; ++idx) {
    const int local = idx - tile0;
    const int b = local / cpp, g0 = (local - b * cpp) * T;
    float2 v[TL::E];
    if constexpr (TL::TMA) {
      const bool ok = mbar_wait_bounded(cx.bar, (uint32_t)(cx.waits & 1));
      ++cx.waits;
      if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) atomicExch(a.err, (int)SR_ERR_TIMEOUT);
        return false;
      }
      load_staged<TL>(cx.smem + RgSmem::stage, t, p, v);
      __syncthreads();  // every thread has its slots before the buffer is refilled
      if (threadIdx.x == 0) rg_issue(cx, idx + 1, s);
    } else {
      __syncthreads();  // the previous tile's scratch reads are done
      if (threadIdx.x == 0) rg_issue(cx, idx + 1, s);
      const float2* src = a.ein + (size_t)b * a.m + (size_t)(g0 + t) * ELL;
#pragma unroll
      for (int j = 0; j < TL::E; ++j) v[j] = src[p + j * TL::P];
    }
    if constexpr (KIND == kRgMidFF) mid_tile<TL, -1, -1, TWS>(a, v, b, g0, t, p, cx.scratch, cx.tw, cx.rowtw, sh);
    else if constexpr (KIND == kRgMidFI) mid_tile<TL, -1, 1, TWS>(a, v, b, g0, t, p, cx.scratch, cx.tw, cx.rowtw, sh);
    else if constexpr (KIND == kRgMidII) mid_tile<TL, 1, 1, TWS>(a, v, b, g0, t, p, cx.scratch, cx.tw, cx.rowtw, sh);
    else if constexpr (KIND == kRgLF) last_first_tile<TL, 0, TWS>(a, v, b, g0, t, p, cx.scratch, cx.tw, cx.rowtw, sh);
    else last_tile<TL, 1, 0, TWS>(a, v, b, g0, t, p, cx.scratch, cx.tw, sh);
  }
  return true;
}

// A run of FIRST tiles [i0, i1) of one segment (lines of ELL points).
template <int ELL>
__device__ __noinline__ void rg_first_run(const PassArgs& a, int tile0, int i0, int i1, float2* scratch,
                                          const float2* tw, float2* rowtw, TileScalars& sh) {
  constexpr int T = 4096 / ELL;
  using TL = Tile<ELL, T>;
  int t, p;
  thread_coords<TL>(t, p);
  const int cpp = a.cpp;
  for (int idx = i0; idx < i1; ++idx) {
    const int local = idx - tile0;
    const int b = local / cpp, g0 = (local - b * cpp) * T;
    first_tile<TL, -1, 0, 1024 / ELL>(a, b, g0, t, p, scratch, tw, rowtw, sh);
    __syncthreads();  // scratch, row twiddles and shared scalars are reused by the next tile
  }
}

#define SR_RG_CLASSES(X) X(0, 128) X(1, 256) X(2, 512) X(3, 1024)

__global__ void __launch_bounds__(kRgThreads, 3)
    k_ragged_pipe(const RaggedSeg* __restrict__ segs, int nseg, int ntiles, const __grid_constant__ RaggedDyn dyn,
                  int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ TileScalars sh;
  __shared__ int tile0[kRgMaxSeg + 1];
  unsigned char* smem = aligned_smem(smem_raw);
  const int tid = threadIdx.x;
  for (int i = tid; i < nseg; i += blockDim.x) tile0[i] = segs[i].tile0;
  if (tid == 0) tile0[nseg] = ntiles;
  // an earlier pass gave up (see mbar_wait_bounded): do nothing
  if (__syncthreads_or(tid == 0 && *(volatile int*)err != 0)) return;
  const int per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int c0 = blockIdx.x * per, c1 = min(ntiles, c0 + per);
  if (c0 >= c1) return;
  RgCtx cx;
  cx.segs = segs;
  cx.tile0 = tile0;
  cx.nseg = nseg;
  cx.c1 = c1;
  cx.smem = smem;
  cx.scratch = reinterpret_cast<float2*>(smem + RgSmem::scratch);
  cx.rowtw = reinterpret_cast<float2*>(smem + RgSmem::rowtw);
  cx.tw = dyn.w1024;
  cx.bar = smem_addr(smem + RgSmem::bar);
  cx.stage = smem_addr(smem + RgSmem::stage);
  cx.waits = 0;
  PassArgs* args = reinterpret_cast<PassArgs*>(smem + RgSmem::args);
  if (tid == 0) {
    mbar_init(cx.bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  int s = rg_find(tile0, nseg, 0, c0);
  if (tid == 0) rg_issue(cx, c0, s);
  int cur = 0;
  for (int idx = c0; idx < c1;) {
    s = rg_find(tile0, nseg, s, idx);
    const int i1 = min(c1, tile0[s + 1]);
    // The copy written here was last read by the run before the previous one,
    // which ended before the previous run's first barrier.
    cur ^= 1;
    rg_load_args(&args[cur], segs[s], dyn);
    __syncthreads();
    bool ok = true;
    switch (segs[s].variant) {
#define SR_RG_CASE(C, ELL)                                                            \
  case kRgMidFF * 4 + C: ok = rg_run<ELL, kRgMidFF>(cx, args[cur], s, idx, i1, sh); break; \
  case kRgMidFI * 4 + C: ok = rg_run<ELL, kRgMidFI>(cx, args[cur], s, idx, i1, sh); break; \
  case kRgMidII * 4 + C: ok = rg_run<ELL, kRgMidII>(cx, args[cur], s, idx, i1, sh); break; \
  case kRgLF * 4 + C: ok = rg_run<ELL, kRgLF>(cx, args[cur], s, idx, i1, sh); break;       \
  case kRgLast * 4 + C: ok = rg_run<ELL, kRgLast>(cx, args[cur], s, idx, i1, sh); break;
      SR_RG_CLASSES(SR_RG_CASE)
#undef SR_RG_CASE
      default: break;
    }
    if (!ok) return;
    idx = i1;
  }
}

// FIRST passes (the input U x, D_1, step 1 of DFT 0) of every segment.
__global__ void __launch_bounds__(kRgThreads, 3)
    k_ragged_first(const RaggedSeg* __restrict__ segs, int nseg, int ntiles, const __grid_constant__ RaggedDyn dyn,
                   int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ TileScalars sh;
  __shared__ int tile0[kRgMaxSeg + 1];
  unsigned char* smem = aligned_smem(smem_raw);
  const int tid = threadIdx.x;
  for (int i = tid; i < nseg; i += blockDim.x) tile0[i] = segs[i].tile0;
  if (tid == 0) tile0[nseg] = ntiles;
  if (__syncthreads_or(tid == 0 && *(volatile int*)err != 0)) return;
  const int per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int c0 = blockIdx.x * per, c1 = min(ntiles, c0 + per);
  float2* scratch = reinterpret_cast<float2*>(smem + RgSmem::scratch);
  float2* rowtw = reinterpret_cast<float2*>(smem + RgSmem::rowtw);
  PassArgs* args = reinterpret_cast<PassArgs*>(smem + RgSmem::args);
  int s = 0, cur = 0;
  for (int idx = c0; idx < c1;) {
    s = rg_find(tile0, nseg, s, idx);
    const int i1 = min(c1, tile0[s + 1]);
    cur ^= 1;
    rg_load_args(&args[cur], segs[s], dyn);
    __syncthreads();
    switch (segs[s].variant & 3) {
#define SR_RG_FIRST(C, ELL) \
  case C: rg_first_run<ELL>(args[cur], tile0[s], idx, i1, scratch, dyn.w1024, rowtw, sh); break;
      SR_RG_CLASSES(SR_RG_FIRST)
#undef SR_RG_FIRST
      default: break;
    }
    idx = i1;
  }
}

// ------------------------------------------------ per-problem set-up / finish

// Compensated block sum (256 threads); valid in thread 0.
__device__ __forceinline__ float rg_block_sum(fsum2 acc, float* red) { return block_sum(acc, red); }

__global__ void __launch_bounds__(256) k_ragged_prepare(const RaggedProblem* __restrict__ pr, const float* __restrict__ y,
                                                        float mu0) {
  __shared__ float red[64];
  const RaggedProblem q = pr[blockIdx.x];
  const float* yb = y + q.y_off;
  fsum2 acc{0.f, 0.f};
  for (int i = threadIdx.x; i < q.m; i += blockDim.x) acc_add(acc, yb[i]);
  const float s = rg_block_sum(acc, red);
  if (threadIdx.x == 0) {
    q.scal[q.b] = s;
    if (mu0 > 0.f) q.scal[q.B + q.b] = mu0 * (float)q.m / s;
  }
}

__global__ void __launch_bounds__(256) k_ragged_start(const RaggedProblem* __restrict__ pr, const float2* __restrict__ v0,
                                                      float2* __restrict__ x) {
  __shared__ float red[64];
  const RaggedProblem q = pr[blockIdx.x];
  fsum2 acc{0.f, 0.f};
  for (int i = threadIdx.x; i < q.n; i += blockDim.x) {
    const float2 v = v0[q.x_off + i];
    x[q.x_off + i] = v;
    acc_add(acc, cabs2(v));
  }
  const float s = rg_block_sum(acc, red);
  if (threadIdx.x == 0) q.bank[1][q.b] = s;
}

__global__ void __launch_bounds__(256) k_ragged_finish(const RaggedProblem* __restrict__ pr, float2* __restrict__ x,
                                                       int prev, int first) {
  __shared__ float s_f;
  const RaggedProblem q = pr[blockIdx.x];
  if (threadIdx.x == 0) {
    const int cnt = first ? 1 : q.count_steady;
    s_f = sqrtf(q.scal[q.b]) / sqrtf(sum_partials(q.bank[prev] + (size_t)q.b * cnt, cnt));
  }
  __syncthreads();
  const float f = s_f;
  for (int i = threadIdx.x; i < q.n; i += blockDim.x) x[q.x_off + i] = cscale(x[q.x_off + i], f);
}

}  // namespace

cudaError_t launch_ragged_prepare(const RaggedProblem* pr, int count, const float* y, float mu0, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_ragged_prepare<<<count, 256, 0, s>>>(pr, y, mu0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_ragged_start(const RaggedProblem* pr, int count, const float2* v0, float2* x, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_ragged_start<<<count, 256, 0, s>>>(pr, v0, x);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_ragged_finish(const RaggedProblem* pr, int count, float2* x, int prev, int first, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_ragged_finish<<<count, 256, 0, s>>>(pr, x, prev, first);
  count_launch();
  return cudaGetLastError();
}

size_t ragged_smem_bytes() { return RgSmem::total + 1024; }

int ragged_class(int ell) {
  switch (ell) {
    case 128: return 0;
    case 256: return 1;
    case 512: return 2;
    case 1024: return 3;
    default: return -1;
  }
}

cudaError_t ragged_occupancy(int* per_sm) {
  const size_t smem = ragged_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_ragged_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ragged_first, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_ragged_pipe, kRgThreads, smem);
  if (e == cudaSuccess) *per_sm = std::max(1, *per_sm);
  return e;
}

cudaError_t launch_ragged_pass(bool first, const RaggedSeg* segs, int nseg, int ntiles, const RaggedDyn& d, int grid,
                               int* err, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  grid = std::max(1, std::min(grid, ntiles));
  const size_t smem = ragged_smem_bytes();
  if (first) k_ragged_first<<<grid, kRgThreads, smem, s>>>(segs, nseg, ntiles, d, err);
  else k_ragged_pipe<<<grid, kRgThreads, smem, s>>>(segs, nseg, ntiles, d, err);
  count_launch();
  return cudaGetLastError();
}

}  // namespace sr
