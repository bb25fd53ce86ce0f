// Four-step pass kernels of the structured operator A = F D_L ... F D_1 U
// (Sec. III, Eq. 5) and the helper kernels of the solvers (Sec. II-B).
//
// A chain of DFTs (the L transforms of A, then the L of A^H for a gradient or
// power-iteration step) runs as: one FIRST pass (natural-order input, fused
// zero-padding U / input scaling / D_1, step 1 of DFT 0), one MID pass per
// interior boundary (step 2 of DFT k-1, fused elementwise operation, step 1 of
// DFT k), and one LAST pass (step 2 of the final DFT, fused D_1^H and the
// natural-order output or solver update). Between passes the data crosses HBM
// (or L2) once, through an exchange buffer written in the order the next pass
// reads contiguously.
#include <algorithm>
#include <atomic>

#include "sr_device.cuh"
#include "sr_internal.h"

namespace sr {

std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// W_m^e = W_m^(hi part) * W_m^(lo part), both tables rounded from double.
__device__ __forceinline__ float2 tw_m(const PassArgs& a, int e) {
  return cmul(__ldg(&a.tw_hi[e >> a.tw_shift]), __ldg(&a.tw_lo[e & ((1 << a.tw_shift) - 1)]));
}

// Multiplies the step-1 outputs of line g by the four-step twiddles
// W_m^(dir * g * f), transposes the CTA's T lines through shared memory and
// writes them to the exchange buffer at (f * NL + g): for each frequency f
// the CTA writes T consecutive elements.
template <int ELL>
__device__ __forceinline__ void store_exchange(float2 (&v)[LineShape<ELL>::E], const PassArgs& a, int b,
                                               int g0, int t, int p, float2* sm) {
  constexpr int E = LineShape<ELL>::E, P = LineShape<ELL>::P;
  const int g = g0 + t;
  const int T = a.T, TP = a.T + 1;
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int f = p + j * P;
    const float2 w = tw_m(a, g * f);
    v[j] = a.out_dir > 0 ? cmulc(v[j], w) : cmul(v[j], w);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < E; ++j) sm[(p + j * P) * TP + t] = v[j];
  __syncthreads();
  float2* eb = a.eout + (size_t)b * a.m;
  for (int idx = threadIdx.x; idx < ELL * T; idx += blockDim.x) {
    const int f = idx / T, tt = idx - f * T;
    eb[(size_t)f * a.nl + g0 + tt] = sm[f * TP + tt];
  }
}

// Threads per CTA of a pass over lines of length ELL (see geom_for): 256 up to
// ELL = 1024, then 4 lines of ELL/16 threads.
__host__ __device__ constexpr int max_threads(int ell) { return ell <= 1024 ? 256 : 4 * (ell / 16); }

template <int ELL>
__global__ void __launch_bounds__(max_threads(ELL)) k_first(PassArgs a) {
  using S = LineShape<ELL>;
  constexpr int E = S::E, P = S::P, LS = S::LS;
  extern __shared__ float2 sm[];
  __shared__ float s_scale;
  const int T = a.T, NL = a.nl, TP = a.T + 1;
  const int tid = threadIdx.x, t = tid / P, p = tid % P;
  const int cta = blockIdx.x, b = cta / a.cpp, g0 = (cta % a.cpp) * T, g = g0 + t;
  const bool warp_ok = (blockDim.x % 32) == 0;
  if (tid == 0) {
    s_scale = a.norm_in ? 1.0f / sqrtf(sum_partials(a.norm_in + (size_t)b * a.norm_in_count, a.norm_in_count))
                        : 1.0f;
  }
  // Natural-order input, zero-padded beyond n_in (the operator U): element
  // (line g, position q) is x[q*NL + g]. Transposed through shared memory so
  // that global reads are T consecutive elements per position.
  const int n_in = a.n_in;
  const int qmax = n_in > g0 ? min(ELL, (n_in - g0 + NL - 1) / NL) : 0;
  const float2* xb = a.xin + (size_t)b * n_in;
  for (int idx = tid; idx < qmax * T; idx += blockDim.x) {
    const int q = idx / T, tt = idx - q * T;
    const long nat = (long)q * NL + g0 + tt;
    sm[q * TP + tt] = nat < n_in ? xb[nat] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float sc = s_scale;
  float2 v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int q = p + j * P;
    v[j] = q < qmax ? cscale(sm[q * TP + t], sc) : make_float2(0.f, 0.f);
  }
  if (a.op == kOpDiag) {
    const float2* d = a.dp + (size_t)g * ELL;
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = cmul(v[j], __ldg(&d[p + j * P]));
  }
  __syncthreads();
  line_fft<ELL>(v, sm + t * LS, p, a.out_dir, a.twl, a.tws, warp_ok);
  store_exchange<ELL>(v, a, b, g0, t, p, sm);
}

template <int ELL>
__device__ __forceinline__ void mid_op(float2 (&v)[LineShape<ELL>::E], const PassArgs& a, int b, int g, int p,
                                       fsum2& acc) {
  constexpr int E = LineShape<ELL>::E, P = LineShape<ELL>::P;
  if (a.op == kOpDiag || a.op == kOpDiagConj) {
    const float2* d = a.dp + (size_t)g * ELL;
    if (a.op == kOpDiag) {
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = cmul(v[j], __ldg(&d[p + j * P]));
    } else {
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = cmulc(v[j], __ldg(&d[p + j * P]));
    }
  } else if (a.op == kOpGdEpilogue) {
    // z -> r = |z|^2 - y, w = r z (Eq. 2); loss partial sum of r^2
    const float* y = a.yp + (size_t)b * a.m + (size_t)g * ELL;
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const float r = cabs2(v[j]) - __ldg(&y[p + j * P]);
      acc_add(acc, r * r);
      v[j] = cscale(v[j], r);
    }
  } else if (a.op == kOpSpecEpilogue) {
    // z -> T(y_hat) z, y_hat = m y / sum(y) (Eq. 3)
    const float* y = a.yp + (size_t)b * a.m + (size_t)g * ELL;
    const float scale = (float)a.m / __ldg(&a.sumy[b]);
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const float yh = __ldg(&y[p + j * P]) * scale;
      float w;
      if (a.weight_mode == SR_WEIGHT_IDENTITY) w = yh;
      else w = yh > 0.f ? fmaxf(1.0f - 1.0f / yh, a.lam) : a.lam;
      v[j] = cscale(v[j], w);
    }
  }
}

template <int ELL>
__global__ void __launch_bounds__(max_threads(ELL)) k_mid(PassArgs a) {
  using S = LineShape<ELL>;
  constexpr int E = S::E, P = S::P, LS = S::LS;
  extern __shared__ float2 sm[];
  __shared__ float red[64];
  const int T = a.T;
  const int tid = threadIdx.x, t = tid / P, p = tid % P;
  const int cta = blockIdx.x, b = cta / a.cpp, g0 = (cta % a.cpp) * T, g = g0 + t;
  const bool warp_ok = (blockDim.x % 32) == 0;
  // lines of the exchange buffer are contiguous: element (g, q) at g*ELL + q
  const float2* src = a.ein + (size_t)b * a.m + (size_t)g * ELL;
  float2 v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = src[p + j * P];
  line_fft<ELL>(v, sm + t * LS, p, a.in_dir, a.twl, a.tws, warp_ok);
  fsum2 acc{0.f, 0.f};
  mid_op<ELL>(v, a, b, g, p, acc);
  if (a.op == kOpGdEpilogue) {
    const float s = block_sum(acc, red);
    if (tid == 0) a.part_out[(size_t)b * a.cpp + (cta % a.cpp)] = s;
  }
  line_sync<P>(warp_ok);
  line_fft<ELL>(v, sm + t * LS, p, a.out_dir, a.twl, a.tws, warp_ok);
  store_exchange<ELL>(v, a, b, g0, t, p, sm);
}

template <int ELL>
__global__ void __launch_bounds__(max_threads(ELL)) k_last(PassArgs a) {
  using S = LineShape<ELL>;
  constexpr int E = S::E, P = S::P, LS = S::LS;
  extern __shared__ float2 sm[];
  __shared__ float red[64];
  __shared__ float s_inv_old, s_mu;
  const int T = a.T, NL = a.nl, TP = a.T + 1;
  const int tid = threadIdx.x, t = tid / P, p = tid % P;
  const int cta = blockIdx.x, b = cta / a.cpp, g0 = (cta % a.cpp) * T, g = g0 + t;
  const bool warp_ok = (blockDim.x % 32) == 0;
  const float2* src = a.ein + (size_t)b * a.m + (size_t)g * ELL;
  float2 v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = src[p + j * P];
  line_fft<ELL>(v, sm + t * LS, p, a.in_dir, a.twl, a.tws, warp_ok);
  if (a.op == kOpDiagConj) {
    const float2* d = a.dp + (size_t)g * ELL;
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = cmulc(v[j], __ldg(&d[p + j * P]));
  }
  if (tid == 0) {
    s_inv_old = (a.out_mode == kOutSpec && a.norm_in)
                    ? 1.0f / sqrtf(sum_partials(a.norm_in + (size_t)b * a.norm_in_count, a.norm_in_count))
                    : 1.0f;
    s_mu = a.mu ? a.mu[b] : 0.f;
  }
  // natural index of (line g, frequency f) is f*NL + g; keep those < n_out (U^H)
  const int n_out = a.n_out;
  const int fmax = n_out > g0 ? min(ELL, (n_out - g0 + NL - 1) / NL) : 0;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int f = p + j * P;
    if (f < fmax) sm[f * TP + t] = v[j];
  }
  __syncthreads();
  float2* xb = a.xout + (size_t)b * n_out;
  const float inv_old = s_inv_old, mu2 = 2.0f * s_mu;
  fsum2 acc{0.f, 0.f};
  for (int idx = tid; idx < fmax * T; idx += blockDim.x) {
    const int f = idx / T, tt = idx - f * T;
    const long nat = (long)f * NL + g0 + tt;
    if (nat >= n_out) continue;
    const float2 val = sm[f * TP + tt];
    switch (a.out_mode) {
      case kOutStore:
        xb[nat] = val;
        break;
      case kOutGrad:
        xb[nat] = cscale(val, 2.0f);
        break;
      case kOutGd: {
        float2 x = xb[nat];
        x.x = fmaf(-mu2, val.x, x.x);
        x.y = fmaf(-mu2, val.y, x.y);
        xb[nat] = x;
        break;
      }
      case kOutSpec: {
        const float2 old = xb[nat];
        const float s = a.shift * inv_old;
        const float2 u = make_float2(fmaf(s, old.x, val.x), fmaf(s, old.y, val.y));
        xb[nat] = u;
        acc_add(acc, cabs2(u));
        break;
      }
    }
  }
  if (a.out_mode == kOutSpec) {
    const float s = block_sum(acc, red);
    if (tid == 0) a.part_out[(size_t)b * a.cpp + (cta % a.cpp)] = s;
  }
  if (a.loss_out && (cta % a.cpp) == 0 && tid == 0)
    a.loss_out[b] = sum_partials(a.loss_part + (size_t)b * a.loss_cpp, a.loss_cpp);
}

// ------------------------------------------------------------------ helpers

// yp[b][g*ell + f] = y[b][f*nl + g]: 32x32 tiles through shared memory.
__global__ void k_permute_real(const float* __restrict__ y, float* __restrict__ yp, int m, int nl, int ell) {
  __shared__ float tile[32][33];
  const int b = blockIdx.z;
  const int g_base = blockIdx.x * 32, f_base = blockIdx.y * 32;
  const float* yb = y + (size_t)b * m;
  float* ob = yp + (size_t)b * m;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int f = f_base + i, g = g_base + threadIdx.x;
    if (f < ell && g < nl) tile[i][threadIdx.x] = yb[(size_t)f * nl + g];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int g = g_base + i, f = f_base + threadIdx.x;
    if (f < ell && g < nl) ob[(size_t)g * ell + f] = tile[threadIdx.x][i];
  }
}

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

LineGeom geom_for(const Plan& p, Layout lay) {
  LineGeom g;
  g.ell = lay == kLayoutX ? p.m1 : p.m2;
  g.nl = (int)(p.m / g.ell);
  const int E = g.ell < 16 ? g.ell : 16;
  g.P = g.ell / E;
  int T = std::max(4, 256 / g.P);
  T = std::min(T, 1024 / g.P);
  T = std::min(T, g.nl);
  g.T = T;
  g.cpp = g.nl / T;
  g.threads = T * g.P;
  const int LS = g.ell + g.ell / 16;
  g.smem = (size_t)std::max(T * LS, g.ell * (T + 1)) * sizeof(float2);
  return g;
}

// Step-1 of a DFT with decomposition parity 0 works on layout X, parity 1 on Y;
// its step 2 on the other layout.
Layout s1_layout(int parity) { return parity == 0 ? kLayoutX : kLayoutY; }
Layout s2_layout(int parity) { return parity == 0 ? kLayoutY : kLayoutX; }
// D_1 (index 0) is applied at the first/last pass (layout X); D_{d+1} (d >= 1)
// between DFT d-1 and DFT d, i.e. at step 2 of a DFT of parity (d-1) mod 2.
Layout diag_layout(int d) { return d == 0 ? kLayoutX : s2_layout((d - 1) % 2); }

#define SR_DEFINE_DISPATCH(KERNEL)                                                               \
  static cudaError_t launch_##KERNEL(int ell, dim3 grid, dim3 block, size_t smem, cudaStream_t s, \
                                     const PassArgs& a) {                                        \
    void (*fn)(PassArgs) = nullptr;                                                              \
    switch (ell) {                                                                               \
      case 2: fn = KERNEL<2>; break;                                                             \
      case 4: fn = KERNEL<4>; break;                                                             \
      case 8: fn = KERNEL<8>; break;                                                             \
      case 16: fn = KERNEL<16>; break;                                                           \
      case 32: fn = KERNEL<32>; break;                                                           \
      case 64: fn = KERNEL<64>; break;                                                           \
      case 128: fn = KERNEL<128>; break;                                                         \
      case 256: fn = KERNEL<256>; break;                                                         \
      case 512: fn = KERNEL<512>; break;                                                         \
      case 1024: fn = KERNEL<1024>; break;                                                       \
      case 2048: fn = KERNEL<2048>; break;                                                       \
      case 4096: fn = KERNEL<4096>; break;                                                       \
      default: return cudaErrorInvalidValue;                                                     \
    }                                                                                            \
    if (smem > 48 * 1024) {                                                                      \
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                           (int)smem);                                           \
      if (e != cudaSuccess) return e;                                                            \
    }                                                                                            \
    fn<<<grid, block, smem, s>>>(a);                                                             \
    count_launch();                                                                              \
    return cudaGetLastError();                                                                   \
  }

SR_DEFINE_DISPATCH(k_first)
SR_DEFINE_DISPATCH(k_mid)
SR_DEFINE_DISPATCH(k_last)

static PassArgs with_geom(const PassArgs& a0, const Plan& p, const LineGeom& g) {
  PassArgs a = a0;
  a.m = (int)p.m;
  a.nl = g.nl;
  a.ell = g.ell;
  a.T = g.T;
  a.cpp = g.cpp;
  a.tws = p.lmax / g.ell;
  return a;
}

cudaError_t launch_first(const Plan& p, Layout lay, const PassArgs& a0, int B, cudaStream_t s) {
  const LineGeom g = geom_for(p, lay);
  return launch_k_first(g.ell, dim3(B * g.cpp), dim3(g.threads), g.smem, s, with_geom(a0, p, g));
}
cudaError_t launch_mid(const Plan& p, Layout lay, const PassArgs& a0, int B, cudaStream_t s) {
  const LineGeom g = geom_for(p, lay);
  return launch_k_mid(g.ell, dim3(B * g.cpp), dim3(g.threads), g.smem, s, with_geom(a0, p, g));
}
cudaError_t launch_last(const Plan& p, Layout lay, const PassArgs& a0, int B, cudaStream_t s) {
  const LineGeom g = geom_for(p, lay);
  return launch_k_last(g.ell, dim3(B * g.cpp), dim3(g.threads), g.smem, s, with_geom(a0, p, g));
}

cudaError_t launch_permute_real(const float* y, float* yp, int B, int m, int nl, int ell, cudaStream_t s) {
  dim3 grid((nl + 31) / 32, (ell + 31) / 32, B), block(32, 8);
  k_permute_real<<<grid, block, 0, s>>>(y, yp, m, nl, ell);
  count_launch();
  return cudaGetLastError();
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
