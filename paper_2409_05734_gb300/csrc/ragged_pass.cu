// The queue-driven solve over ragged batches: ONE launch runs a whole GD or
// power-iteration call (Sec. II-B, Eq. 2-4) for every problem of a ragged
// batch whose four-step geometry it covers, whatever the problem's length.
//
// The problems come from buckets of one shape (n, m, L), each with its own
// batched plan (per-problem phases, exchange buffers, partial sums). A
// descriptor per (bucket, pass kind) holds the pass arguments the bucket's plan
// would launch its own kernel with and which line length and pass kind it
// runs; the values that change from call to call or step to step (the caller's
// concatenated x and y, the step's warm-up factor, the loss-history row, the
// power iteration's ping-pong banks) are filled in on the device.
//
// Work items are tiles: (problem, pass, tile), dealt out by an atomic ticket in
// a fixed order -- group by group (problems of one L whose data fits in L2),
// pass by pass, problem by problem. A tile of pass q of problem p starts once
// all tiles of pass q - 1 of p are done (a per-problem completion count, read
// with acquire semantics). Every dependency points to a lower ticket and a CTA
// takes a ticket only while it runs, so the lowest unfinished ticket can always
// proceed: the grid needs no co-residency guarantee. Each wait is bounded; one
// that gives up records SR_ERR_TIMEOUT and ends its CTA.
//
// Every CTA has 256 threads and tiles of 4096 values: lines of 128, 256, 512
// and 1024 points as 32, 16, 8 and 4 lines per tile. A CTA holds two items:
// the one it runs and the next, whose input it stages by TMA as soon as the
// current tile's values are in registers and the next tile's inputs are
// complete (lines of up to 512 points; the 4-line tiles of 1024-point lines
// read their input directly). The line twiddles come from one table of
// W_1024^k in global memory (L1-resident), read with the stride 1024 / ELL, so
// shared memory holds only the staging buffer, the FFT scratch and the row
// twiddles.
#include <algorithm>

#include "passes.cuh"
#include "sr_ragged.h"

namespace sr {
namespace {

constexpr int kRgThreads = 256;

// Byte layout of the dynamic shared memory (relative to a 1024-byte-aligned
// base): TMA staging (32 KB), FFT scratch (the padded layout of 4096 values),
// row twiddles (16 x up to 32 lines), the descriptors of the current and the
// next item, the barrier.
struct RgSmem {
  static constexpr size_t stage = 0;
  static constexpr size_t scratch = 4096 * 8;
  static constexpr size_t rowtw = scratch + 4096 * 17 / 16 * 8;
  static constexpr size_t args = rowtw + 16 * 32 * 8;
  static constexpr size_t bar = args + 2 * sizeof(RaggedSeg);
  static constexpr size_t total = bar + 16;
};

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

// ------------------------------------------------------- queue-driven solve

// A decoded work item: tile `tile` of pass q of problem p, at step t.
struct RgItem {
  int valid;
  int ready;    // inputs known to be complete (the first pass needs none)
  int p, q, tile, t;
  int b;        // the problem's index in its bucket
  int si;       // descriptor
  int need;     // completed tiles of p before this tile may start (q * C)
  int variant;
  int tma;
  int row;      // first exchange-buffer row of the tile (staged tiles)
  int ell, T;   // line length; lines per tile
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// The pass data a producer wrote with ordinary stores is read by this CTA's
// TMA loads (the async proxy): order them after the acquire.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// 16-byte asynchronous copy global -> shared (cp.async, L2 only).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared tables of the queue: the first ticket of every group (and the total
// after the last), its tiles per pass and its first record.
struct RgQTables {
  unsigned gstart[kRgMaxGroups + 1];
  int ipq[kRgMaxGroups];
  int rec0[kRgMaxGroups];
};

// Decodes ticket tk: the group by binary search in shared memory, pass and tile
// slot by division, then one 32-byte record load; the pass kind, layout, line
// length and descriptor follow from the record and the pass index.
__device__ __forceinline__ void rg_decode(RgItem& it, const RgSolveArgs& sa, const RgQTables& tb, unsigned tk) {
  it.valid = 0;
  if (tk >= tb.gstart[sa.ngrp]) return;
  int lo = 0, hi = sa.ngrp - 1;  // the group g with gstart[g] <= tk < gstart[g + 1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tb.gstart[mid] <= tk) lo = mid;
    else hi = mid - 1;
  }
  const unsigned within = tk - tb.gstart[lo];
  const int ipq = tb.ipq[lo];
  const int q = (int)(within / (unsigned)ipq), r = (int)within - q * ipq;
  const RgTileRec R = sa.rec[tb.rec0[lo] + r];
  // pass sequence of a problem: FIRST; then per step MID_1 .. MID_{2L-1} and
  // the fused LAST/FIRST (LAST after the final step)
  const int per = 2 * R.L;
  int kidx = 0, t = 0;
  if (q > 0) {
    t = (q - 1) / per;
    const int k = q - t * per;
    kidx = k < per ? k : (t + 1 < sa.T ? per : per + 1);
  }
  int kind;
  if (kidx == 0) kind = kRgFirst;
  else if (kidx < R.L) kind = kRgMidFF;
  else if (kidx == R.L) kind = kRgMidFI;
  else if (kidx < per) kind = kRgMidII;
  else kind = kidx == per ? kRgLF : kRgLast;
  // layouts: FIRST, LAST and the fused pass work on layout X; MID k on Y for
  // odd k, X for even k
  const int lay_y = (kidx > 0 && kidx < per && (kidx & 1)) ? 1 : 0;
  const int code = (R.lay >> (8 * lay_y)) & 0xff;
  const int cls = code & 15;
  it.p = R.p;
  it.q = q;
  it.tile = R.tile;
  it.t = t;
  it.b = R.b;
  it.si = R.si0 + kidx;
  it.need = q * R.C;
  it.variant = kind * 4 + cls;
  it.tma = kind != kRgFirst && (code >> 4);
  it.ell = 128 << cls;
  it.T = 32 >> cls;
  it.row = R.b * (1 << (R.lgm - 7 - cls)) + R.tile * it.T;
  it.ready = q == 0;
  it.valid = 1;
}

// Thread 0: waits (bounded) until problem p has `need` completed tiles.
__device__ __forceinline__ bool rg_wait_done(const int* done, int p, int need) {
  if (need <= 0 || ld_acquire_gpu(done + p) >= need) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    __nanosleep(64);
    if (ld_acquire_gpu(done + p) >= need) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

struct RgQCtx {
  const RgSolveArgs* sa;
  unsigned char* smem;
  float2* scratch;
  float2* rowtw;
  const float2* tw;
  uint32_t bar, stage;
  int waits;
  RgItem* items;     // shared: [2] the current and the next item (slot = item count & 1)
  int* issued;       // shared: [2] whether the item's TMA load is in flight
  RaggedSeg* args;   // shared: [2] the items' descriptors, patched for their step
  int cur;
  int* err;
};

// Thread 0: issues the TMA load of items[slot] when it is a staged tile whose
// inputs are complete (the caller has freed the staging buffer).
__device__ __forceinline__ void rg_issue(RgQCtx& cx, int slot) {
  const RgItem& nx = cx.items[slot];
  if (!nx.valid || !nx.tma) return;
  if (!nx.ready && ld_acquire_gpu(cx.sa->done + nx.p) < nx.need) return;
  fence_proxy_async_global();
  fence_proxy_async_smem();
  issue_rows(&cx.sa->segs[nx.si].a.tmap, nx.row, nx.ell, nx.T, nx.T * 128, cx.stage, cx.bar);
  cx.issued[slot] = 1;
}

// Warp 0, once the current tile's input is in registers: the next item's TMA
// load (lane 0) and the asynchronous copy of its descriptor into its argument
// slot (patched after the current item, see rg_finish_item).
__device__ __forceinline__ void rg_prep_next(RgQCtx& cx) {
  const int nxt = cx.cur ^ 1;
  if (threadIdx.x == 0) rg_issue(cx, nxt);
  const RgItem& nx = cx.items[nxt];
  if (nx.valid) {
    const uint4* src = reinterpret_cast<const uint4*>(&cx.sa->segs[nx.si]);
    uint4* dst = reinterpret_cast<uint4*>(&cx.args[nxt]);
    constexpr int kChunks = (int)(sizeof(RaggedSeg) / 16);
    for (int i = threadIdx.x; i < kChunks; i += 32) cp_async16(dst + i, src + i);
  }
  cp_async_commit();
}

// The descriptor copy sg for step t of the call: the call's pointers, the
// step's warm-up factor and loss row, the power iteration's banks.
__device__ __forceinline__ void rg_patch_step(RaggedSeg& sg, const RaggedDyn& d, int t, float tau0) {
  RaggedDyn e = d;
  e.t = t;
  e.mu_scale = tau0 > 0.f ? 1.0f - expf(-(float)(t + 1) / tau0) : 1.0f;
  e.parity = t & 1;
  e.first_step = t == 0;
  rg_patch(sg.a, sg, e);
}

// One item of a pipelined pass kind (MID, fused LAST/FIRST, LAST) with lines
// of ELL points: its input lines into registers (from the staging buffer, or
// straight from the exchange buffer for unstaged tiles), the next item's
// prefetch, then the body. False when a wait gave up (recorded in err).
template <int ELL, int KIND>
__device__ __noinline__ bool rg_qtile(RgQCtx& cx, const PassArgs& a, const RgItem& it, TileScalars& sh) {
  constexpr int T = 4096 / ELL;
  using TL = Tile<ELL, T>;
  constexpr int TWS = 1024 / ELL;
  int t, p, rho;
  thread_coords<TL>(t, p, rho);
  const int b = it.b, g0 = it.tile * T;  // tiles of a pass hold T consecutive lines
  float2 v[TL::E];
  if constexpr (TL::TMA) {
    if (cx.issued[cx.cur] == 0) {  // the load waits for the producers of this pass (this CTA holds nothing)
      bool ok = true;
      if (threadIdx.x == 0) {
        ok = rg_wait_done(cx.sa->done, it.p, it.need);
        if (ok) {
          fence_proxy_async_global();
          fence_proxy_async_smem();
          issue_rows(&cx.sa->segs[it.si].a.tmap, it.row, ELL, T, T * 128, cx.stage, cx.bar);
        } else {
          atomicExch(cx.err, (int)SR_ERR_TIMEOUT);
        }
      }
      if (!__syncthreads_and(ok)) return false;
    }
    const bool ok = mbar_wait_bounded(cx.bar, (uint32_t)(cx.waits & 1));
    ++cx.waits;
    // the slots are read whatever the wait's outcome (in bounds either way);
    // one barrier then frees the staging buffer and tells every thread
    // whether a wait gave up
    load_staged<TL>(cx.smem + RgSmem::stage, t, p, rho, v);
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) atomicExch(cx.err, (int)SR_ERR_TIMEOUT);
      return false;
    }
    if (threadIdx.x < 32) rg_prep_next(cx);
  } else {
    bool ok = true;
    if (threadIdx.x == 0) {
      ok = rg_wait_done(cx.sa->done, it.p, it.need);
      if (!ok) atomicExch(cx.err, (int)SR_ERR_TIMEOUT);
    }
    if (!__syncthreads_and(ok)) return false;
    if (threadIdx.x < 32) rg_prep_next(cx);
    const float2* src = a.ein + (size_t)b * a.m + (size_t)(g0 + t) * ELL;
#pragma unroll
    for (int j = 0; j < TL::E; ++j) v[j] = src[p + j * TL::P];
  }
  if constexpr (KIND == kRgMidFF) mid_tile<TL, -1, -1, TWS>(a, v, b, g0, t, p, rho, cx.scratch, cx.tw, cx.rowtw, sh);
  else if constexpr (KIND == kRgMidFI) mid_tile<TL, -1, 1, TWS>(a, v, b, g0, t, p, rho, cx.scratch, cx.tw, cx.rowtw, sh);
  else if constexpr (KIND == kRgMidII) mid_tile<TL, 1, 1, TWS>(a, v, b, g0, t, p, rho, cx.scratch, cx.tw, cx.rowtw, sh);
  else if constexpr (KIND == kRgLF) last_first_tile<TL, 0, TWS>(a, v, b, g0, t, p, rho, cx.scratch, cx.tw, cx.rowtw, sh);
  else last_tile<TL, 1, 0, TWS>(a, v, b, g0, t, p, rho, cx.scratch, cx.tw, sh);
  return true;
}

// One FIRST item (lines of ELL points): natural-order input, no wait.
template <int ELL>
__device__ __noinline__ bool rg_qfirst(RgQCtx& cx, const PassArgs& a, const RgItem& it, TileScalars& sh) {
  constexpr int T = 4096 / ELL;
  using TL = Tile<ELL, T>;
  int t, p, rho;
  thread_coords<TL>(t, p, rho);
  const int b = it.b, g0 = it.tile * T;
  __syncthreads();  // the item's arguments visible
  if (threadIdx.x < 32) rg_prep_next(cx);
  first_tile<TL, -1, 0, 1024 / ELL>(a, b, g0, t, p, rho, cx.scratch, cx.tw, cx.rowtw, sh);
  return true;
}

// Runs one item of line length ELL (any pass kind). Each (length, kind) body
// is a function of its own: one register allocation per body, not one for the
// union of all of them.
template <int ELL>
__device__ __forceinline__ bool rg_qitem(RgQCtx& cx, const PassArgs& a, const RgItem& it, TileScalars& sh) {
  switch (it.variant >> 2) {
    case kRgMidFF: return rg_qtile<ELL, kRgMidFF>(cx, a, it, sh);
    case kRgMidFI: return rg_qtile<ELL, kRgMidFI>(cx, a, it, sh);
    case kRgMidII: return rg_qtile<ELL, kRgMidII>(cx, a, it, sh);
    case kRgLF: return rg_qtile<ELL, kRgLF>(cx, a, it, sh);
    case kRgLast: return rg_qtile<ELL, kRgLast>(cx, a, it, sh);
    default: return rg_qfirst<ELL>(cx, a, it, sh);
  }
}

// Warp 0 after an item's closing barrier: the item's completion is released
// (thread 0), the next item's descriptor copy is awaited and patched for its
// step, the prefetched ticket is decoded into the finished item's slot (the
// item after the next) and a new ticket is requested, whose value is needed
// only after the next item.
__device__ __forceinline__ void rg_finish_item(RgQCtx& cx, const RgSolveArgs& sa, const RaggedDyn& dyn,
                                               const RgQTables& tb, unsigned& tk_pf) {
  cp_async_wait_all();
  __syncwarp();
  if (threadIdx.x == 0) {
    const int cur = cx.cur, nxt = cur ^ 1;
    fence_proxy_async_global();
    __threadfence();
    atomicAdd(sa.done + cx.items[cur].p, 1);
    if (cx.items[nxt].valid) rg_patch_step(cx.args[nxt], dyn, cx.items[nxt].t, sa.tau0);
    rg_decode(cx.items[cur], sa, tb, tk_pf);
    cx.issued[cur] = 0;
    tk_pf = atomicAdd(sa.ticket, 1u);
  }
}

__global__ void __launch_bounds__(kRgThreads, 3)
    k_ragged_solve(const __grid_constant__ RgSolveArgs sa, const __grid_constant__ RaggedDyn dyn, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ TileScalars sh;
  __shared__ RgQTables tb;
  __shared__ RgItem items[2];
  __shared__ int issued[2];
  unsigned char* smem = aligned_smem(smem_raw);
  const int tid = threadIdx.x;
  if (tid == 0) {
    unsigned acc = 0;
    for (int g = 0; g < sa.ngrp; ++g) {
      const RgGroup G = sa.grp[g];
      const int L = sa.rec[G.rec0].L;
      tb.gstart[g] = acc;
      tb.ipq[g] = G.ipq;
      tb.rec0[g] = G.rec0;
      acc += (unsigned)(1 + 2 * L * sa.T) * (unsigned)G.ipq;
    }
    tb.gstart[sa.ngrp] = acc;
  }
  // an earlier pass gave up (see mbar_wait_bounded): do nothing
  if (__syncthreads_or(tid == 0 && *(volatile int*)err != 0)) return;
  RgQCtx cx;
  cx.sa = &sa;
  cx.smem = smem;
  cx.scratch = reinterpret_cast<float2*>(smem + RgSmem::scratch);
  cx.rowtw = reinterpret_cast<float2*>(smem + RgSmem::rowtw);
  cx.tw = dyn.w1024;
  cx.bar = smem_addr(smem + RgSmem::bar);
  cx.stage = smem_addr(smem + RgSmem::stage);
  cx.waits = 0;
  cx.items = items;
  cx.issued = issued;
  cx.args = reinterpret_cast<RaggedSeg*>(smem + RgSmem::args);
  cx.cur = 0;
  cx.err = err;
  // the first two items, the first one's descriptor and TMA load, and a
  // ticket in flight for the third
  unsigned tk_pf = 0;
  if (tid == 0) {
    mbar_init(cx.bar, 1);
    mbar_init_fence();
    rg_decode(items[0], sa, tb, atomicAdd(sa.ticket, 1u));
    rg_decode(items[1], sa, tb, atomicAdd(sa.ticket, 1u));
    issued[0] = issued[1] = 0;
    tk_pf = atomicAdd(sa.ticket, 1u);
  }
  __syncthreads();
  if (tid < 32 && items[0].valid) {
    const uint4* src = reinterpret_cast<const uint4*>(&sa.segs[items[0].si]);
    uint4* dst = reinterpret_cast<uint4*>(&cx.args[0]);
    for (int i = tid; i < (int)(sizeof(RaggedSeg) / 16); i += 32) dst[i] = src[i];
    __syncwarp();
    if (tid == 0) {
      rg_patch_step(cx.args[0], dyn, items[0].t, sa.tau0);
      rg_issue(cx, 0);
    }
  }
  __syncthreads();
  for (;;) {
    const RgItem& it = items[cx.cur];
    if (!it.valid) break;
    const PassArgs& a = cx.args[cx.cur].a;
    bool ok = true;
    switch (it.variant & 3) {
      case 0: ok = rg_qitem<128>(cx, a, it, sh); break;
      case 1: ok = rg_qitem<256>(cx, a, it, sh); break;
      case 2: ok = rg_qitem<512>(cx, a, it, sh); break;
      default: ok = rg_qitem<1024>(cx, a, it, sh); break;
    }
    if (!ok) {
      if (tid < 32) cp_async_wait_all();  // no copy into shared memory outlives the CTA
      return;
    }
    __syncthreads();  // every store of the tile issued; every thread is done with the item
    if (tid < 32) rg_finish_item(cx, sa, dyn, tb, tk_pf);
    cx.cur ^= 1;
  }
  if (tid < 32) cp_async_wait_all();
}

// ------------------------------------------------ per-problem set-up / finish

// Chunk c = blockIdx.x of problem blockIdx.y (kRgChunks chunks per problem).
__device__ __forceinline__ void rg_chunk(int len, int& lo, int& hi) {
  const int per = (len + kRgChunks - 1) / kRgChunks;
  lo = min(len, (int)blockIdx.x * per);
  hi = min(len, lo + per);
}

__global__ void __launch_bounds__(256) k_ragged_sum_y(const RaggedProblem* __restrict__ pr, const float* __restrict__ y) {
  __shared__ float red[64];
  const RaggedProblem q = pr[blockIdx.y];
  int lo, hi;
  rg_chunk(q.m, lo, hi);
  const float* yb = y + q.y_off;
  fsum2 acc{0.f, 0.f};
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) acc_add(acc, yb[i]);
  const float s = block_sum(acc, red);
  if (threadIdx.x == 0) q.sums[(size_t)q.b * kRgChunks + blockIdx.x] = s;
}

__global__ void k_ragged_finish_y(const RaggedProblem* __restrict__ pr, int count, float mu0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const RaggedProblem q = pr[i];
  const float s = sum_partials(q.sums + (size_t)q.b * kRgChunks, kRgChunks);
  q.scal[q.b] = s;
  if (mu0 > 0.f) q.scal[q.B + q.b] = mu0 * (float)q.m / s;
}

__global__ void __launch_bounds__(256) k_ragged_start(const RaggedProblem* __restrict__ pr, const float2* __restrict__ v0,
                                                      float2* __restrict__ x) {
  __shared__ float red[64];
  const RaggedProblem q = pr[blockIdx.y];
  int lo, hi;
  rg_chunk(q.n, lo, hi);
  fsum2 acc{0.f, 0.f};
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const float2 v = v0[q.x_off + i];
    x[q.x_off + i] = v;
    acc_add(acc, cabs2(v));
  }
  const float s = block_sum(acc, red);
  if (threadIdx.x == 0) q.bank[1][(size_t)q.b * kRgChunks + blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_ragged_finish(const RaggedProblem* __restrict__ pr, float2* __restrict__ x,
                                                       int prev, int first) {
  __shared__ float s_f;
  const RaggedProblem q = pr[blockIdx.y];
  if (threadIdx.x == 0) {
    const int cnt = first ? kRgChunks : q.count_steady;
    s_f = sqrtf(q.scal[q.b]) / sqrtf(sum_partials(q.bank[prev] + (size_t)q.b * cnt, cnt));
  }
  __syncthreads();
  const float f = s_f;
  int lo, hi;
  rg_chunk(q.n, lo, hi);
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) x[q.x_off + i] = cscale(x[q.x_off + i], f);
}

}  // namespace

cudaError_t launch_ragged_prepare(const RaggedProblem* pr, int count, const float* y, float mu0, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_ragged_sum_y<<<dim3(kRgChunks, count), 256, 0, s>>>(pr, y);
  count_launch();
  k_ragged_finish_y<<<(count + 127) / 128, 128, 0, s>>>(pr, count, mu0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_ragged_start(const RaggedProblem* pr, int count, const float2* v0, float2* x, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_ragged_start<<<dim3(kRgChunks, count), 256, 0, s>>>(pr, v0, x);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_ragged_finish(const RaggedProblem* pr, int count, float2* x, int prev, int first, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_ragged_finish<<<dim3(kRgChunks, count), 256, 0, s>>>(pr, x, prev, first);
  count_launch();
  return cudaGetLastError();
}

size_t ragged_smem_bytes() { return RgSmem::total + 1024; }

cudaError_t ragged_solve_occupancy(int* per_sm) {
  const size_t smem = ragged_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_ragged_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_ragged_solve, kRgThreads, smem);
  if (e == cudaSuccess) *per_sm = std::max(1, *per_sm);
  return e;
}

cudaError_t launch_ragged_solve(const RgSolveArgs& sa, const RaggedDyn& d, int grid, int* err, cudaStream_t s) {
  k_ragged_solve<<<std::max(1, grid), kRgThreads, ragged_smem_bytes(), s>>>(sa, d, err);
  count_launch();
  return cudaGetLastError();
}

int ragged_class(int ell) {
  switch (ell) {
    case 128: return 0;
    case 256: return 1;
    case 512: return 2;
    case 1024: return 3;
    default: return -1;
  }
}

}  // namespace sr
