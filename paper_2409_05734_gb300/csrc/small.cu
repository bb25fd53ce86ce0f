// Whole solves for short transforms: power-of-two m <= 8192 (1D plans, n <= m).
//
// The length-m DFT of one problem is a single line FFT (line_fft, radix-16
// Stockham in shared memory), so every A and A^H of Sec. III, Eq. 5 runs
// inside one CTA: each problem is one line of a CTA (T problems per CTA, P =
// m/16 threads per problem, thread (t, p) holding entries p + j P of problem
// t in registers). The iterate x (and y, or the spectral weights) stay in
// registers for all iterations, which loop inside the kernel; only the
// diagonals D_l are re-read (from L2) per use. One launch replaces the 2L
// passes of an iteration times the iteration count.
//
// k_small_gd: GD steps x <- x - mu_t 2 A^H((|Ax|^2 - y) Ax) (Sec. II-B-1,
// Eq. 2), one gradient evaluation (loss and 2 A^H(r z)), or the operator
// alone (z = A x, x = A^H w).
// k_small_spec: power-iteration steps u = A^H diag(T(y_hat)) A v + s v,
// v = u / ||u|| (Sec. II-B-2, Eq. 3-4), with the norms of the last two steps.
#include <algorithm>

#include "sr_device.cuh"
#include "sr_internal.h"

namespace sr {
namespace {

// W_m^k for k < M from the plan's two-level table (forward sign).
template <int M>
__device__ __forceinline__ void small_twiddles(const SmallArgs& a, float2* tw) {
  const int mask = (1 << a.tw_shift) - 1;
  for (int k = threadIdx.x; k < M; k += blockDim.x) tw[k] = cmul(__ldg(&a.tw_hi[k >> a.tw_shift]), __ldg(&a.tw_lo[k & mask]));
}

// Compensated sum over the P threads of each line (problem) t; every thread
// gets its line's sum. red: P*T float2.
template <int T, int P>
__device__ __forceinline__ float line_sum(fsum2 acc, int t, int p, float2* red) {
  red[p * T + t] = make_float2(acc.s, acc.c);
  __syncthreads();
#pragma unroll 1
  for (int h = P / 2; h >= 1; h >>= 1) {
    if (p < h) {
      const float2 u = red[p * T + t], w = red[(p + h) * T + t];
      const fsum2 r = acc_merge(fsum2{u.x, u.y}, fsum2{w.x, w.y});
      red[p * T + t] = make_float2(r.s, r.c);
    }
    __syncthreads();
  }
  const float2 r = red[t];
  __syncthreads();  // red is reused by the next call
  return r.x + r.y;
}

// v <- A v from v = U x (slots j at entries k = p + j P): D_l then F, l = 1..L.
template <int M, int T>
__device__ __forceinline__ void small_forward(float2 (&v)[LineShape<M>::E], const float2* dpb, int m, int L, int p,
                                              int t, float2* scratch, const float2* tw) {
  constexpr int E = LineShape<M>::E, P = LineShape<M>::P;
#pragma unroll 1
  for (int l = 0; l < L; ++l) {
    const float2* d = dpb + (size_t)l * m;
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = cmul(v[j], __ldg(&d[p + j * P]));
    if constexpr (LineShape<M>::NSTAGE > 1) __syncthreads();  // the scratch's previous reads are done
    line_fft<M, T, -1>(v, scratch, p, t, tw);
  }
}

// v <- D_1^H F^H ... D_L^H F^H v.
template <int M, int T>
__device__ __forceinline__ void small_adjoint(float2 (&v)[LineShape<M>::E], const float2* dpb, int m, int L, int p,
                                              int t, float2* scratch, const float2* tw) {
  constexpr int E = LineShape<M>::E, P = LineShape<M>::P;
#pragma unroll 1
  for (int l = L - 1; l >= 0; --l) {
    if constexpr (LineShape<M>::NSTAGE > 1) __syncthreads();
    line_fft<M, T, 1>(v, scratch, p, t, tw);
    const float2* d = dpb + (size_t)l * m;
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = cmulc(v[j], __ldg(&d[p + j * P]));
  }
}

template <int M, int T>
struct SmallSmem {
  static constexpr int P = LineShape<M>::P;
  static constexpr size_t scratch = (size_t)T * LineShape<M>::LS * 8;
  static constexpr size_t tw = (size_t)M * 8;
  static constexpr size_t red = (size_t)P * T * 8;
  static constexpr size_t total = scratch + tw + red;
};

template <int M, int T>
__global__ void __launch_bounds__(T * LineShape<M>::P) k_small_gd(const SmallArgs a) {
  constexpr int E = LineShape<M>::E, P = LineShape<M>::P;
  using SM = SmallSmem<M, T>;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* scratch = reinterpret_cast<float2*>(smem);
  float2* tw = reinterpret_cast<float2*>(smem + SM::scratch);
  float2* red = reinterpret_cast<float2*>(smem + SM::scratch + SM::tw);
  const int t = threadIdx.x % T, p = threadIdx.x / T;
  const int b = blockIdx.x * T + t;
  const bool valid = b < a.B;
  const int m = a.m, n = a.n;
  small_twiddles<M>(a, tw);
  const float2* dpb = a.dp + (size_t)(valid ? b : 0) * a.dp_stride;
  if (a.op != 0) {  // the operator alone (Sec. III, Eq. 5): z = A x or x = A^H w
    float2 v[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int k = p + j * P;
      const bool inwin = (unsigned)(k - a.off) < (unsigned)a.mo;  // S^H: zero outside the window
      if (a.op == 1) v[j] = valid && k < n ? a.x[(size_t)b * n + k] : make_float2(0.f, 0.f);
      else v[j] = valid && inwin ? a.win[(size_t)b * a.mo + (k - a.off)] : make_float2(0.f, 0.f);
    }
    __syncthreads();  // twiddles
    if (a.op == 1) {
      small_forward<M, T>(v, dpb, m, a.L, p, t, scratch, tw);
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int k = p + j * P;
        if (valid && (unsigned)(k - a.off) < (unsigned)a.mo) a.zout[(size_t)b * a.mo + (k - a.off)] = v[j];  // S
      }
    } else {
      small_adjoint<M, T>(v, dpb, m, a.L, p, t, scratch, tw);
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int k = p + j * P;
        if (valid && k < n) a.x[(size_t)b * n + k] = v[j];
      }
    }
    return;
  }
  float2 xr[E];
  float yr[E];
  unsigned inwin = 0;  // bit j: entry p + j P is measured (the window of the alpha < 1 branch)
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int k = p + j * P;
    const bool in = (unsigned)(k - a.off) < (unsigned)a.mo;
    inwin |= in ? (1u << j) : 0u;
    xr[j] = valid && k < n ? a.x[(size_t)b * n + k] : make_float2(0.f, 0.f);
    yr[j] = valid && in ? __ldg(&a.y[(size_t)b * a.mo + (k - a.off)]) : 0.f;
  }
  const float mu = valid && a.mu ? __ldg(&a.mu[b]) : 0.f;
  __syncthreads();  // twiddles
#pragma unroll 1
  for (int it = 0; it < a.count; ++it) {
    const int step = a.t0 + it;
    float2 v[E];
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = xr[j];
    small_forward<M, T>(v, dpb, m, a.L, p, t, scratch, tw);
    // z -> r = |z|^2 - y, w = r z (Eq. 2); loss = sum r^2
    fsum2 acc{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const float r = cabs2(v[j]) - yr[j];
      if (inwin & (1u << j)) {
        acc_add(acc, r * r);
        v[j] = cscale(v[j], r);
      } else {
        v[j] = make_float2(0.f, 0.f);  // S^H S: unmeasured entries carry no residual
      }
    }
    float* lrow = a.grad ? a.loss_out
                         : (a.loss_hist && step >= a.loss_first ? a.loss_hist + (size_t)(step - a.loss_first) * a.B
                                                                : nullptr);
    if (lrow) {
      const float loss = line_sum<T, P>(acc, t, p, red);
      if (valid && p == 0) lrow[b] = loss;
    }
    small_adjoint<M, T>(v, dpb, m, a.L, p, t, scratch, tw);
    if (a.grad) {  // the gradient 2 A^H(r z) of the incoming x
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int k = p + j * P;
        if (valid && k < n) a.g[(size_t)b * n + k] = cscale(v[j], 2.0f);
      }
      return;
    }
    const float ramp = a.tau0 > 0.f ? 1.0f - expf(-(float)(step + 1) / a.tau0) : 1.0f;
    const float mu2 = 2.0f * mu * ramp;
#pragma unroll
    for (int j = 0; j < E; ++j) {
      if (p + j * P < n) {
        xr[j].x = fmaf(-mu2, v[j].x, xr[j].x);
        xr[j].y = fmaf(-mu2, v[j].y, xr[j].y);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int k = p + j * P;
    if (valid && k < n) a.x[(size_t)b * n + k] = xr[j];
  }
}

template <int M, int T>
__global__ void __launch_bounds__(T * LineShape<M>::P) k_small_spec(const SmallArgs a) {
  constexpr int E = LineShape<M>::E, P = LineShape<M>::P;
  using SM = SmallSmem<M, T>;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* scratch = reinterpret_cast<float2*>(smem);
  float2* tw = reinterpret_cast<float2*>(smem + SM::scratch);
  float2* red = reinterpret_cast<float2*>(smem + SM::scratch + SM::tw);
  const int t = threadIdx.x % T, p = threadIdx.x / T;
  const int b = blockIdx.x * T + t;
  const bool valid = b < a.B;
  const int m = a.m, n = a.n;
  small_twiddles<M>(a, tw);
  const float2* dpb = a.dp + (size_t)(valid ? b : 0) * a.dp_stride;
  // weights T(y_hat), y_hat = m y / sum(y) (Eq. 3)
  const float ysc = valid ? (float)a.mo / __ldg(&a.sumy[b]) : 0.f;
  float2 ur[E];
  float wr[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int k = p + j * P;
    const bool in = (unsigned)(k - a.off) < (unsigned)a.mo;
    ur[j] = valid && k < n ? a.x[(size_t)b * n + k] : make_float2(0.f, 0.f);
    const float yh = valid && in ? __ldg(&a.y[(size_t)b * a.mo + (k - a.off)]) * ysc : 0.f;
    float w = yh;
    if (a.weight_mode == SR_WEIGHT_OPTIMAL) w = yh > 0.f ? fmaxf(1.0f - 1.0f / yh, a.lam) : a.lam;
    wr[j] = in ? w : 0.f;  // S^H S: unmeasured entries carry no weight
  }
  // ||u||^2 of the incoming iterate
  float nrm = valid ? sum_partials(a.norm_in + (size_t)b * a.norm_in_count, a.norm_in_count) : 1.f;
  float nrm_prev = nrm;
  __syncthreads();  // twiddles
#pragma unroll 1
  for (int it = 0; it < a.count; ++it) {
    const float inv = nrm > 0.f ? 1.0f / sqrtf(nrm) : 0.f;
    float2 v[E];
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = cscale(ur[j], inv);
    small_forward<M, T>(v, dpb, m, a.L, p, t, scratch, tw);
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = cscale(v[j], wr[j]);
    small_adjoint<M, T>(v, dpb, m, a.L, p, t, scratch, tw);
    // u = M v + s v on the kept entries (U^H), and its norm
    const float sh = a.shift * inv;
    fsum2 acc{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < E; ++j) {
      if (p + j * P < n) {
        ur[j] = make_float2(fmaf(sh, ur[j].x, v[j].x), fmaf(sh, ur[j].y, v[j].y));
        acc_add(acc, cabs2(ur[j]));
      }
    }
    nrm_prev = nrm;
    nrm = line_sum<T, P>(acc, t, p, red);
  }
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int k = p + j * P;
    if (valid && k < n) a.x[(size_t)b * n + k] = ur[j];
  }
  if (valid && p == 0) {
    a.norm_last[b] = nrm;
    if (a.count >= 2) a.norm_prev[b] = nrm_prev;
  }
}

template <int M, int T>
cudaError_t launch_small_t(const SmallArgs& a, bool spec, cudaStream_t s) {
  using SM = SmallSmem<M, T>;
  constexpr int threads = T * LineShape<M>::P;
  const void* fn = spec ? reinterpret_cast<const void*>(&k_small_spec<M, T>)
                        : reinterpret_cast<const void*>(&k_small_gd<M, T>);
  if (SM::total > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::total);
    if (e != cudaSuccess) return e;
  }
  const int grid = (a.B + T - 1) / T;
  if (spec) k_small_spec<M, T><<<grid, threads, SM::total, s>>>(a);
  else k_small_gd<M, T><<<grid, threads, SM::total, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

// Problems per CTA: 256 threads per CTA while that gives every SM a CTA, else
// one warp's worth of threads, else one problem per CTA (small batches of
// short transforms are latency-bound: spreading them over more SMs wins).
template <int M>
cudaError_t launch_small_m(const SmallArgs& a, bool spec, int num_sms, cudaStream_t s) {
  constexpr int P = LineShape<M>::P;
  constexpr int TB = P >= 256 ? 1 : 256 / P;
  constexpr int TS = P >= 32 ? 1 : 32 / P;
  if ((a.B + TB - 1) / TB >= num_sms || TB == 1) return launch_small_t<M, TB>(a, spec, s);
  if constexpr (TS != TB) {
    if ((a.B + TS - 1) / TS >= num_sms || TS == 1) return launch_small_t<M, TS>(a, spec, s);
  }
  return launch_small_t<M, 1>(a, spec, s);
}

}  // namespace

bool small_eligible(const Plan& p) {
  return !p.inner && !p.two_d && p.m >= 4 && p.m <= kSmallMaxM && (p.m & (p.m - 1)) == 0 && p.n <= p.m;
}

cudaError_t launch_small(const Plan& p, const SmallArgs& a, bool spec, cudaStream_t s) {
  switch (p.m) {
    case 4: return launch_small_m<4>(a, spec, p.num_sms, s);
    case 8: return launch_small_m<8>(a, spec, p.num_sms, s);
    case 16: return launch_small_m<16>(a, spec, p.num_sms, s);
    case 32: return launch_small_m<32>(a, spec, p.num_sms, s);
    case 64: return launch_small_m<64>(a, spec, p.num_sms, s);
    case 128: return launch_small_m<128>(a, spec, p.num_sms, s);
    case 256: return launch_small_m<256>(a, spec, p.num_sms, s);
    case 512: return launch_small_m<512>(a, spec, p.num_sms, s);
    case 1024: return launch_small_m<1024>(a, spec, p.num_sms, s);
    case 2048: return launch_small_m<2048>(a, spec, p.num_sms, s);
    case 4096: return launch_small_m<4096>(a, spec, p.num_sms, s);
    case 8192: return launch_small_m<8192>(a, spec, p.num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sr
