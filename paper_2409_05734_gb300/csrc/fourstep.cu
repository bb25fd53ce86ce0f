// Four-step pass kernels of the structured operator A = F D_L ... F D_1 U
// (Sec. III, Eq. 5) and the helper kernels of the solvers (Sec. II-B).
//
// A chain of DFTs (the L transforms of A, then the L of A^H for a gradient or
// power-iteration step) runs as: one FIRST pass (natural-order input, fused
// zero-padding U / input scaling / D_1, step 1 of DFT 0), one MID pass per
// interior boundary (step 2 of DFT k-1, fused elementwise operation, step 1 of
// DFT k), and one LAST pass (step 2 of the final DFT, fused D_1^H and the
// natural-order output or solver update). Between passes the data crosses HBM
// (or L2) once, through an exchange buffer.
//
// Threads are numbered line-fastest (tid = t + T*p), so every natural-order
// access (x, y, D_l) and every exchange-buffer write is T consecutive elements
// per warp instruction straight from registers. The exchange rows a MID/LAST
// pass reads are brought into shared memory by 2D TMA loads with 128-byte
// swizzle, double-buffered across the tiles of a persistent grid so that the
// next tile's load overlaps the current tile's FFTs.
#include <algorithm>
#include <atomic>

#include "sr_device.cuh"
#include "sr_internal.h"
#include "sr_tma.cuh"

namespace sr {

std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------ shared-memory layout
struct PipeSmem {
  size_t in0, in1, scratch, tw, rowtw, bar, total;
};

__host__ __device__ inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Bytes one TMA box (16 complex values x T rows) occupies in shared memory:
// every box starts on a 1024-byte boundary (the period of the 128-byte swizzle).
__host__ __device__ inline int box_bytes(int T) { return (int)round_up((size_t)T * 128, 1024); }

// Layout relative to a 1024-byte-aligned base. tma: the pass stages its input
// tiles (T rows of ell complex values, ell/16 boxes) in `nbuf` swizzled buffers.
__host__ __device__ inline PipeSmem pipe_layout(int ell, int T, int nbuf, bool tma) {
  PipeSmem L;
  const size_t tile = tma ? (size_t)(ell / 16) * box_bytes(T) : 0;
  const int E = ell < 16 ? ell : 16;
  L.in0 = 0;
  L.in1 = tile;
  size_t off = tile * (tma ? nbuf : 0);
  L.scratch = off;
  off += (size_t)T * (ell + ell / 16) * 8;
  L.tw = off;
  off += (size_t)ell * 8;
  L.rowtw = off;
  off += (size_t)E * T * 8;
  L.bar = round_up(off, 8);
  L.total = L.bar + 16;
  return L;
}

__device__ __forceinline__ unsigned char* aligned_smem(unsigned char* raw) {
  const uint32_t a = smem_addr(raw);
  return raw + (((a + 1023u) & ~1023u) - a);
}

// ------------------------------------------------------------------ tables

// W_m^e = W_m^(hi part) * W_m^(lo part), both tables rounded from double.
__device__ __forceinline__ float2 tw_m(const PassArgs& a, int e) {
  return cmul(__ldg(&a.tw_hi[e >> a.tw_shift]), __ldg(&a.tw_lo[e & ((1 << a.tw_shift) - 1)]));
}

// Line twiddles W_ELL^k, k < ELL, into shared memory.
template <int ELL>
__device__ __forceinline__ void load_line_twiddles(const PassArgs& a, float2* tw) {
  for (int i = threadIdx.x; i < ELL; i += blockDim.x) tw[i] = __ldg(&a.twl[i * a.tws]);
}

// Four-step twiddle of (line g, frequency f = p + j*P) is W_m^(g p) * W_m^(g P j);
// the second factor is tabulated per tile: rowtw[j*T + t] = W_m^((g0 + t) P j).
template <int ELL>
__device__ __forceinline__ void fill_row_twiddles(const PassArgs& a, int g0, float2* rowtw) {
  constexpr int E = LineShape<ELL>::E, P = LineShape<ELL>::P;
  for (int i = threadIdx.x; i < E * a.T; i += blockDim.x) {
    const int t = i & (a.T - 1), j = i >> a.lgT;
    rowtw[i] = tw_m(a, (g0 + t) * P * j);
  }
}

// Step-1 outputs of line g times W_m^(dir g f), stored to the exchange buffer
// at f*NL + g (T consecutive elements per frequency across the warp).
template <int ELL>
__device__ __forceinline__ void twiddle_store(float2 (&v)[LineShape<ELL>::E], const PassArgs& a, int b, int g,
                                              int t, int p, const float2* rowtw) {
  constexpr int E = LineShape<ELL>::E, P = LineShape<ELL>::P;
  const float2 A = tw_m(a, g * p);
  float2* eb = a.eout + (size_t)b * a.m + g;
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const float2 w = cmul(A, rowtw[j * a.T + t]);
    const float2 o = a.out_dir > 0 ? cmulc(v[j], w) : cmul(v[j], w);
    eb[(size_t)(p + j * P) * a.nl] = o;
  }
}

// Elementwise operation at (line g, frequency f): natural index f*NL + g.
template <int ELL>
__device__ __forceinline__ void mid_op(float2 (&v)[LineShape<ELL>::E], const PassArgs& a, int b, int g, int p,
                                       fsum2& acc) {
  constexpr int E = LineShape<ELL>::E, P = LineShape<ELL>::P;
  if (a.op == kOpDiag) {
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = cmul(v[j], __ldg(&a.dp[(p + j * P) * a.nl + g]));
  } else if (a.op == kOpDiagConj) {
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = cmulc(v[j], __ldg(&a.dp[(p + j * P) * a.nl + g]));
  } else if (a.op == kOpGdEpilogue) {
    // z -> r = |z|^2 - y, w = r z (Eq. 2); loss partial sum of r^2
    const float* y = a.y + (size_t)b * a.m + g;
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const float r = cabs2(v[j]) - __ldg(&y[(p + j * P) * a.nl]);
      acc_add(acc, r * r);
      v[j] = cscale(v[j], r);
    }
  } else if (a.op == kOpSpecEpilogue) {
    // z -> T(y_hat) z, y_hat = m y / sum(y) (Eq. 3)
    const float* y = a.y + (size_t)b * a.m + g;
    const float scale = (float)a.m / __ldg(&a.sumy[b]);
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const float yh = __ldg(&y[(p + j * P) * a.nl]) * scale;
      float w;
      if (a.weight_mode == SR_WEIGHT_IDENTITY) w = yh;
      else w = yh > 0.f ? fmaxf(1.0f - 1.0f / yh, a.lam) : a.lam;
      v[j] = cscale(v[j], w);
    }
  }
}

// ------------------------------------------------------------ FIRST pass

// Threads per CTA of the passes over lines of length ELL (make_geom keeps
// T * P within this bound): 256 up to ELL = 512, 512 beyond; at least two
// CTAs per SM for the shorter lines.
__host__ __device__ constexpr int pass_threads(int ell) { return ell <= 512 ? 256 : 512; }
__host__ __device__ constexpr int pass_min_ctas(int ell) { return ell <= 512 ? 2 : 1; }

template <int ELL>
__global__ void __launch_bounds__(pass_threads(ELL), pass_min_ctas(ELL)) k_first(const __grid_constant__ PassArgs a) {
  using S = LineShape<ELL>;
  constexpr int E = S::E, P = S::P;
  extern __shared__ unsigned char smem_raw[];
  __shared__ float s_scale;
  unsigned char* smem = aligned_smem(smem_raw);
  const PipeSmem L = pipe_layout(ELL, a.T, 1, false);
  float2* scratch = reinterpret_cast<float2*>(smem + L.scratch);
  float2* tw = reinterpret_cast<float2*>(smem + L.tw);
  float2* rowtw = reinterpret_cast<float2*>(smem + L.rowtw);
  const int tid = threadIdx.x, lgT = a.lgT, t = tid & (a.T - 1), p = tid >> lgT;
  const int b = blockIdx.x / a.cpp, g0 = (blockIdx.x - b * a.cpp) << lgT, g = g0 + t;
  load_line_twiddles<ELL>(a, tw);
  fill_row_twiddles<ELL>(a, g0, rowtw);
  if (tid == 0)
    s_scale = a.norm_in ? 1.0f / sqrtf(sum_partials(a.norm_in + (size_t)b * a.norm_in_count, a.norm_in_count))
                        : 1.0f;
  // Natural-order input, zero beyond n_in (the padding U): element (line g,
  // position q) is x[q*NL + g]; the warp reads T consecutive elements.
  const float2* xb = a.xin + (size_t)b * a.n_in;
  float2 v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int nat = (p + j * P) * a.nl + g;
    v[j] = nat < a.n_in ? xb[nat] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float sc = s_scale;
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = cscale(v[j], sc);
  if (a.op == kOpDiag) {
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = cmul(v[j], __ldg(&a.dp[(p + j * P) * a.nl + g]));
  }
  line_fft<ELL>(v, scratch, p, t, lgT, a.out_dir, tw);
  twiddle_store<ELL>(v, a, b, g, t, p, rowtw);
}

// ------------------------------------------------------ MID and LAST passes

// Issues the TMA loads of tile `tile` (T rows of ELL complex values, boxes of
// 16 values x T rows) into `buf`, completing on barrier `bar`.
template <int ELL>
__device__ __forceinline__ void issue_tile(const PassArgs& a, int tile, uint32_t buf, uint32_t bar) {
  const int b = tile / a.cpp, g0 = (tile - b * a.cpp) << a.lgT;
  const int row = b * a.nl + g0;
  mbar_arrive_expect_tx(bar, (uint32_t)(a.T * ELL * 8));
#pragma unroll 1
  const int bb = box_bytes(a.T);
  for (int kb = 0; kb < ELL / 16; ++kb) tma_load_2d(buf + (uint32_t)(kb * bb), &a.tmap, kb * 32, row, bar);
}

// Shared pipeline of the persistent MID / LAST passes: for every tile of this
// CTA, loads the T input lines (rows of the exchange buffer) into registers
// (slot j = position p + j*P) and calls body(v, b, g0).
template <int ELL, class Body>
__device__ __forceinline__ void pipe_tiles(const PassArgs& a, int nbuf, unsigned char* smem, const PipeSmem& L,
                                           Body&& body) {
  constexpr int E = LineShape<ELL>::E, P = LineShape<ELL>::P;
  constexpr bool kTma = ELL >= 16;
  const int tid = threadIdx.x, lgT = a.lgT, t = tid & (a.T - 1), p = tid >> lgT;
  // an earlier pass gave up (see mbar_wait_bounded): do nothing
  if (__syncthreads_or(tid == 0 && *(volatile int*)a.err != 0)) return;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar);
  const uint32_t bar0 = smem_addr(&bars[0]), bar1 = smem_addr(&bars[1]);
  const uint32_t in0 = smem_addr(smem + L.in0), in1 = smem_addr(smem + L.in1);
  int tile = blockIdx.x;
  if constexpr (kTma) {
    if (tid == 0) {
      mbar_init(bar0, 1);
      mbar_init(bar1, 1);
      mbar_init_fence();
    }
    __syncthreads();
    if (tid == 0 && tile < a.ntiles) issue_tile<ELL>(a, tile, in0, bar0);
  }
  for (int k = 0; tile < a.ntiles; ++k, tile += gridDim.x) {
    const int b = tile / a.cpp, g0 = (tile - b * a.cpp) << lgT, g = g0 + t;
    const int next = tile + (int)gridDim.x;
    float2 v[E];
    if constexpr (kTma) {
      const int buf = nbuf == 2 ? (k & 1) : 0;
      const uint32_t parity = nbuf == 2 ? (uint32_t)((k >> 1) & 1) : (uint32_t)(k & 1);
      const uint32_t bar = buf ? bar1 : bar0;
      if (nbuf == 2 && tid == 0 && next < a.ntiles) {
        fence_proxy_async_smem();
        issue_tile<ELL>(a, next, buf ? in0 : in1, buf ? bar0 : bar1);
      }
      const bool ok = mbar_wait_bounded(bar, parity);
      if (!__syncthreads_and(ok)) {
        // a load never completed: record it, let a pending prefetch land, stop
        if (tid == 0) {
          atomicExch(a.err, (int)SR_ERR_TIMEOUT);
          if (nbuf == 2 && next < a.ntiles) mbar_wait_bounded(buf ? bar0 : bar1, (uint32_t)(((k + 1) >> 1) & 1));
        }
        return;
      }
      const unsigned char* src = smem + (buf ? L.in1 : L.in0);
      const int bb = box_bytes(a.T);
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = *reinterpret_cast<const float2*>(src + swz128_offset(bb, t, p + j * P));
      if (nbuf == 1) {
        __syncthreads();  // every thread has its slots before the buffer is refilled
        if (tid == 0 && next < a.ntiles) {
          fence_proxy_async_smem();
          issue_tile<ELL>(a, next, in0, bar0);
        }
      }
    } else {
      const float2* src = a.ein + (size_t)b * a.m + (size_t)g * ELL;
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = src[p + j * P];
    }
    body(v, b, g0);
    __syncthreads();  // scratch, tables and input buffer free for the next tile
  }
}

template <int ELL>
__global__ void __launch_bounds__(pass_threads(ELL), pass_min_ctas(ELL)) k_mid(const __grid_constant__ PassArgs a, int nbuf) {
  using S = LineShape<ELL>;
  constexpr int E = S::E;
  extern __shared__ unsigned char smem_raw[];
  __shared__ float red[64];
  unsigned char* smem = aligned_smem(smem_raw);
  const PipeSmem L = pipe_layout(ELL, a.T, nbuf, ELL >= 16);
  float2* scratch = reinterpret_cast<float2*>(smem + L.scratch);
  float2* tw = reinterpret_cast<float2*>(smem + L.tw);
  float2* rowtw = reinterpret_cast<float2*>(smem + L.rowtw);
  const int tid = threadIdx.x, lgT = a.lgT, t = tid & (a.T - 1), p = tid >> lgT;
  load_line_twiddles<ELL>(a, tw);
  __syncthreads();
  pipe_tiles<ELL>(a, nbuf, smem, L, [&](float2 (&v)[E], int b, int g0) {
    const int g = g0 + t;
    fill_row_twiddles<ELL>(a, g0, rowtw);
    line_fft<ELL>(v, scratch, p, t, lgT, a.in_dir, tw);
    fsum2 acc{0.f, 0.f};
    mid_op<ELL>(v, a, b, g, p, acc);
    if (a.op == kOpGdEpilogue) {
      const float s = block_sum(acc, red);
      if (tid == 0) a.part_out[(size_t)b * a.cpp + (g0 >> lgT)] = s;
    }
    __syncthreads();  // first FFT's scratch reads done; row twiddles visible
    line_fft<ELL>(v, scratch, p, t, lgT, a.out_dir, tw);
    twiddle_store<ELL>(v, a, b, g, t, p, rowtw);
  });
}

template <int ELL>
__global__ void __launch_bounds__(pass_threads(ELL), pass_min_ctas(ELL)) k_last(const __grid_constant__ PassArgs a, int nbuf) {
  using S = LineShape<ELL>;
  constexpr int E = S::E, P = S::P;
  extern __shared__ unsigned char smem_raw[];
  __shared__ float red[64];
  __shared__ float s_inv_old, s_mu;
  unsigned char* smem = aligned_smem(smem_raw);
  const PipeSmem L = pipe_layout(ELL, a.T, nbuf, ELL >= 16);
  float2* scratch = reinterpret_cast<float2*>(smem + L.scratch);
  float2* tw = reinterpret_cast<float2*>(smem + L.tw);
  const int tid = threadIdx.x, lgT = a.lgT, t = tid & (a.T - 1), p = tid >> lgT;
  load_line_twiddles<ELL>(a, tw);
  __syncthreads();
  pipe_tiles<ELL>(a, nbuf, smem, L, [&](float2 (&v)[E], int b, int g0) {
    const int g = g0 + t;
    if (tid == 0) {
      s_inv_old = (a.out_mode == kOutSpec && a.norm_in)
                      ? 1.0f / sqrtf(sum_partials(a.norm_in + (size_t)b * a.norm_in_count, a.norm_in_count))
                      : 1.0f;
      s_mu = a.mu ? a.mu[b] : 0.f;
    }
    line_fft<ELL>(v, scratch, p, t, lgT, a.in_dir, tw);
    __syncthreads();  // tile scalars visible
    if (a.op == kOpDiagConj) {
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = cmulc(v[j], __ldg(&a.dp[(p + j * P) * a.nl + g]));
    }
    // natural index of (line g, frequency f) is f*NL + g; keep those < n_out (U^H)
    float2* xb = a.xout + (size_t)b * a.n_out;
    const float inv_old = s_inv_old, mu2 = 2.0f * s_mu * a.mu_scale, sh = a.shift * inv_old;
    fsum2 acc{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int nat = (p + j * P) * a.nl + g;
      if (nat >= a.n_out) continue;
      const float2 val = v[j];
      if (a.out_mode == kOutStore) {
        xb[nat] = val;
      } else if (a.out_mode == kOutGrad) {
        xb[nat] = cscale(val, 2.0f);
      } else if (a.out_mode == kOutGd) {
        float2 x = xb[nat];
        x.x = fmaf(-mu2, val.x, x.x);
        x.y = fmaf(-mu2, val.y, x.y);
        xb[nat] = x;
      } else {  // kOutSpec
        const float2 old = xb[nat];
        const float2 u = make_float2(fmaf(sh, old.x, val.x), fmaf(sh, old.y, val.y));
        xb[nat] = u;
        acc_add(acc, cabs2(u));
      }
    }
    if (a.out_mode == kOutSpec) {
      const float s = block_sum(acc, red);
      if (tid == 0) a.part_out[(size_t)b * a.cpp + (g0 >> lgT)] = s;
    }
    if (a.loss_out && g0 == 0 && tid == 0)
      a.loss_out[b] = sum_partials(a.loss_part + (size_t)b * a.loss_cpp, a.loss_cpp);
  });
}

// ------------------------------------------------------------------ helpers

// part[b*chunks + c] = compensated sum of chunk c of row b.
__global__ void k_sum_rows(const float* __restrict__ y, int m, float* __restrict__ part, int chunks) {
  __shared__ float red[64];
  const int b = blockIdx.y, c = blockIdx.x;
  const int len = (m + chunks - 1) / chunks;
  const int lo = c * len, hi = min(m, lo + len);
  const float* yb = y + (size_t)b * m;
  fsum2 acc{0.f, 0.f};
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) acc_add(acc, yb[i]);
  const float s = block_sum(acc, red);
  if (threadIdx.x == 0) part[(size_t)b * chunks + c] = s;
}

__global__ void k_norm_rows(const float2* __restrict__ v, int n, float* __restrict__ part, int chunks) {
  __shared__ float red[64];
  const int b = blockIdx.y, c = blockIdx.x;
  const int len = (n + chunks - 1) / chunks;
  const int lo = c * len, hi = min(n, lo + len);
  const float2* vb = v + (size_t)b * n;
  fsum2 acc{0.f, 0.f};
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) acc_add(acc, cabs2(vb[i]));
  const float s = block_sum(acc, red);
  if (threadIdx.x == 0) part[(size_t)b * chunks + c] = s;
}

__global__ void k_finish_scalars(const float* __restrict__ part, int chunks, int B, float mu0, int m,
                                 float* __restrict__ sumy, float* __restrict__ mu) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float s = sum_partials(part + (size_t)b * chunks, chunks);
  sumy[b] = s;
  if (mu) mu[b] = mu0 * (float)m / s;
}

// v[b] *= sqrt(sumy[b]) / ||v[b]|| with ||v||^2 the sum of `chunks` partials.
__global__ void k_scale_rows(float2* __restrict__ v, int n, const float* __restrict__ part, int chunks,
                             const float* __restrict__ sumy) {
  __shared__ float s_f;
  const int b = blockIdx.y;
  if (threadIdx.x == 0) s_f = sqrtf(sumy[b]) / sqrtf(sum_partials(part + (size_t)b * chunks, chunks));
  __syncthreads();
  const float f = s_f;
  float2* vb = v + (size_t)b * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) vb[i] = cscale(vb[i], f);
}

// ------------------------------------------------------------------ launchers

constexpr size_t kSmemBudget = 220 * 1024;

LineGeom make_geom(int64_t m, int ell) {
  LineGeom g;
  g.ell = ell;
  g.nl = (int)(m / ell);
  const int E = ell < 16 ? ell : 16;
  g.P = ell / E;
  int T = std::max(8, 256 / g.P);
  T = std::min(T, pass_threads(ell) / g.P);
  T = std::min(T, g.nl);
  const bool tma = ell >= 16;
  while (T > 1 && pipe_layout(ell, T, 1, tma).total + 1024 > kSmemBudget) T >>= 1;
  g.T = T;
  g.lgT = 0;
  while ((1 << g.lgT) < T) ++g.lgT;
  g.cpp = g.nl / T;
  g.threads = T * g.P;
  g.nbuf = (tma && pipe_layout(ell, T, 2, tma).total + 1024 <= kSmemBudget) ? 2 : 1;
  g.smem_pipe = pipe_layout(ell, T, g.nbuf, tma).total + 1024;
  g.smem_first = pipe_layout(ell, T, 1, false).total + 1024;
  return g;
}

// Step 1 of a DFT with decomposition parity 0 works on layout X, parity 1 on Y;
// its step 2 on the other layout.
Layout s1_layout(int parity) { return parity == 0 ? kLayoutX : kLayoutY; }
Layout s2_layout(int parity) { return parity == 0 ? kLayoutY : kLayoutX; }

#define SR_ELL_SWITCH(ell, KERNEL, fn)     \
  switch (ell) {                           \
    case 2: fn = KERNEL<2>; break;         \
    case 4: fn = KERNEL<4>; break;         \
    case 8: fn = KERNEL<8>; break;         \
    case 16: fn = KERNEL<16>; break;       \
    case 32: fn = KERNEL<32>; break;       \
    case 64: fn = KERNEL<64>; break;       \
    case 128: fn = KERNEL<128>; break;     \
    case 256: fn = KERNEL<256>; break;     \
    case 512: fn = KERNEL<512>; break;     \
    case 1024: fn = KERNEL<1024>; break;   \
    case 2048: fn = KERNEL<2048>; break;   \
    case 4096: fn = KERNEL<4096>; break;   \
    default: return cudaErrorInvalidValue; \
  }

static cudaError_t allow_smem(const void* fn, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

static PassArgs with_geom(const PassArgs& a0, const Plan& p, const LineGeom& g, int B) {
  PassArgs a = a0;
  a.m = (int)p.m;
  a.nl = g.nl;
  a.ell = g.ell;
  a.T = g.T;
  a.lgT = g.lgT;
  a.cpp = g.cpp;
  a.ntiles = B * g.cpp;
  a.tws = p.lmax / g.ell;
  return a;
}

cudaError_t launch_first(const Plan& p, Layout lay, const PassArgs& a0, int B, cudaStream_t s) {
  const LineGeom& g = p.geom[lay];
  void (*fn)(PassArgs) = nullptr;
  SR_ELL_SWITCH(g.ell, k_first, fn);
  cudaError_t e = allow_smem((const void*)fn, g.smem_first);
  if (e != cudaSuccess) return e;
  const PassArgs a = with_geom(a0, p, g, B);
  fn<<<a.ntiles, g.threads, g.smem_first, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

static cudaError_t launch_pipe(bool last, const Plan& p, Layout lay, const PassArgs& a0, int B, cudaStream_t s) {
  const LineGeom& g = p.geom[lay];
  void (*fn)(PassArgs, int) = nullptr;
  if (last) {
    SR_ELL_SWITCH(g.ell, k_last, fn);
  } else {
    SR_ELL_SWITCH(g.ell, k_mid, fn);
  }
  cudaError_t e = allow_smem((const void*)fn, g.smem_pipe);
  if (e != cudaSuccess) return e;
  const PassArgs a = with_geom(a0, p, g, B);
  const int per_sm = last ? p.per_sm_last[lay] : p.per_sm_mid[lay];
  const int grid = std::max(1, std::min(a.ntiles, per_sm * p.num_sms));
  fn<<<grid, g.threads, g.smem_pipe, s>>>(a, g.nbuf);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_mid(const Plan& p, Layout lay, const PassArgs& a, int B, cudaStream_t s) {
  return launch_pipe(false, p, lay, a, B, s);
}
cudaError_t launch_last(const Plan& p, Layout lay, const PassArgs& a, int B, cudaStream_t s) {
  return launch_pipe(true, p, lay, a, B, s);
}

cudaError_t pass_occupancy(const LineGeom& g, int* per_sm_mid, int* per_sm_last) {
  void (*fm)(PassArgs, int) = nullptr;
  void (*fl)(PassArgs, int) = nullptr;
  SR_ELL_SWITCH(g.ell, k_mid, fm);
  SR_ELL_SWITCH(g.ell, k_last, fl);
  cudaError_t e;
  if ((e = allow_smem((const void*)fm, g.smem_pipe)) != cudaSuccess) return e;
  if ((e = allow_smem((const void*)fl, g.smem_pipe)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm_mid, fm, g.threads, g.smem_pipe)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm_last, fl, g.threads, g.smem_pipe)) != cudaSuccess)
    return e;
  *per_sm_mid = std::max(1, *per_sm_mid);
  *per_sm_last = std::max(1, *per_sm_last);
  return cudaSuccess;
}

cudaError_t launch_sum_rows(const float* y, int B, int m, float* part, int chunks, cudaStream_t s) {
  k_sum_rows<<<dim3(chunks, B), 256, 0, s>>>(y, m, part, chunks);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_norm_rows(const float2* v, int B, int n, float* part, int chunks, cudaStream_t s) {
  k_norm_rows<<<dim3(chunks, B), 256, 0, s>>>(v, n, part, chunks);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_finish_scalars(const float* part, int chunks, int B, float mu0, int m, float* sumy, float* mu,
                                  cudaStream_t s) {
  k_finish_scalars<<<(B + 127) / 128, 128, 0, s>>>(part, chunks, B, mu0, m, sumy, mu);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_scale_rows(float2* v, int B, int n, const float* part, int chunks, const float* sumy,
                              cudaStream_t s) {
  const int blocks = std::min(64, (n + 255) / 256);
  k_scale_rows<<<dim3(blocks, B), 256, 0, s>>>(v, n, part, chunks, sumy);
  count_launch();
  return cudaGetLastError();
}

}  // namespace sr
