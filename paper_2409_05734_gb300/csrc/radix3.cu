// Lengths m = 3 * mp (mp a power of two): the unitary DFT of Sec. III, Eq. 5 by
// one radix-3 step of decimation in time around power-of-two DFTs.
//
// With u_r[j] = v[3j + r] (r = 0, 1, 2; j < mp) and U_r = DFT_mp(u_r),
//   DFT_m(v)[k' + s mp] = sum_r W_m^{r k'} W_3^{r s} U_r[k'],   k' < mp, s < 3,
// where W_N = exp(-2 pi i / N) (forward sign; the inverse conjugates every W).
// A chain step is then: the power-of-two DFT of the 3B sequences u_r by the
// four-step passes, whose first pass gathers the stride-3 subsequences of the
// natural-order vector and applies the operation that precedes the DFT (a
// diagonal, the GD or spectral epilogue) at the outer index, and a combine
// kernel (twiddles, radix-3 butterfly, natural-order output with the chain's
// output mode).
#include <algorithm>

#include "sr_device.cuh"
#include "sr_internal.h"

namespace sr {
namespace {

// sqrt(3)/2: imaginary part of exp(-2 pi i / 3) up to sign.
constexpr float kS3 = 0.86602540378443864676f;

template <int DIR>
__global__ void k_r3_combine(const R3CombineArgs a) {
  __shared__ float red[64];
  __shared__ float s_inv_old, s_mu;
  const int b = blockIdx.y, c = blockIdx.x;
  const int64_t mp = a.mp;
  const int64_t kmax = mp < a.n_out ? mp : a.n_out;  // outputs k' + s mp < n_out need k' < n_out
  const int64_t len = (mp + a.chunks - 1) / a.chunks;
  const int64_t lo = c * len, hi = min(kmax, lo + len);
  if (threadIdx.x == 0) {
    s_inv_old = (a.out_mode == kOutSpec && a.norm_in)
                    ? 1.0f / sqrtf(sum_partials(a.norm_in + (size_t)b * a.norm_in_count, a.norm_in_count))
                    : 1.0f;
    s_mu = a.mu ? a.mu[b] : 0.f;
  }
  __syncthreads();
  const float inv_old = s_inv_old, mu2 = 2.0f * s_mu * a.mu_scale, sh = a.shift * inv_old;
  const float2* U = a.U + (size_t)(3 * b) * mp;
  float2* xb = a.xout + (size_t)b * a.n_out;
  fsum2 acc{0.f, 0.f};
  for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
    float2 w1 = __ldg(&a.tw3[k]), w2 = __ldg(&a.tw3[2 * k]);
    if (DIR > 0) {
      w1.y = -w1.y;
      w2.y = -w2.y;
    }
    const float2 t0 = U[k];
    const float2 t1 = cmul(U[mp + k], w1);
    const float2 t2 = cmul(U[2 * mp + k], w2);
    // radix-3 butterfly: X_s = t0 + W3^s t1 + W3^{2s} t2
    const float2 sum = cadd(t1, t2), dif = csub(t1, t2);
    const float2 mid = make_float2(fmaf(-0.5f, sum.x, t0.x), fmaf(-0.5f, sum.y, t0.y));
    // -i sqrt(3)/2 * dif for the forward sign (+i for the inverse)
    const float2 rot = DIR > 0 ? make_float2(-kS3 * dif.y, kS3 * dif.x) : make_float2(kS3 * dif.y, -kS3 * dif.x);
    float2 X[3];
    X[0] = cadd(t0, sum);
    X[1] = cadd(mid, rot);
    X[2] = csub(mid, rot);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int64_t nat = k + s * mp;
      if (nat >= a.n_out) continue;
      float2 val = X[s];
      if (a.op == kOpDiagConj) val = cmulc(val, __ldg(&a.dp[(size_t)b * a.dp_stride + nat]));
      if (a.out_mode == kOutStore) {
        xb[nat] = val;
      } else if (a.out_mode == kOutGrad) {
        xb[nat] = cscale(val, 2.0f);
      } else if (a.out_mode == kOutGd) {
        float2 x = xb[nat];
        x.x = fmaf(-mu2, val.x, x.x);
        x.y = fmaf(-mu2, val.y, x.y);
        xb[nat] = x;
      } else {  // kOutSpec: u = M v + shift v, v = old / ||old||
        const float2 old = xb[nat];
        const float2 uu = make_float2(fmaf(sh, old.x, val.x), fmaf(sh, old.y, val.y));
        xb[nat] = uu;
        acc_add(acc, cabs2(uu));
      }
    }
  }
  if (a.out_mode == kOutSpec) {
    const float s = block_sum(acc, red);
    if (threadIdx.x == 0) a.part_out[(size_t)b * a.chunks + c] = s;
  }
  if (a.loss_out && c == 0 && threadIdx.x == 0)
    a.loss_out[b] = sum_partials(a.loss_part + (size_t)b * a.loss_cpp, a.loss_cpp);
}

}  // namespace

cudaError_t launch_r3_combine(const R3CombineArgs& a, int dir, int B, cudaStream_t s) {
  if (dir > 0) k_r3_combine<1><<<dim3(a.chunks, B), 256, 0, s>>>(a);
  else k_r3_combine<-1><<<dim3(a.chunks, B), 256, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace sr
