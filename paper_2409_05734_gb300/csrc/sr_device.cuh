// Device building blocks of the structured-operator kernels: complex helpers,
// radix-2/4/8/16 DFT butterflies, the per-line Stockham FFT held in registers
// and shared memory, and compensated (two-sum) float reductions.
//
// All FFTs here are unnormalised, with the forward sign exp(-2*pi*i*jk/N) or
// the inverse sign exp(+2*pi*i*jk/N) chosen at compile time; the unitary
// 1/sqrt(m) of F (Sec. III, Eq. 5) is folded into the diagonal tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sr {

// ------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// Packed FP32x2 arithmetic of the sm_100 family: one instruction adds or
// subtracts both parts of a complex value (the float2 stays one 64-bit
// register pair).
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, exact as a fused multiply-add by -1 (one rounding, like a subtraction)
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// ------------------------------------------------------ small DFTs (sign S)
// X_k = sum_j a_j exp(S 2 pi i jk/R) for S = -1 (forward) or S = +1 (inverse),
// unnormalised, natural order in and out. The inverse is written out with the
// conjugate roots rather than as conj(DFT(conj(.))) so that the real and
// imaginary parts of every value stay in their register pair.
// Constants of the 8th and 16th roots of unity: cos(pi/4), cos(pi/8), sin(pi/8).
constexpr float kC4 = 0.70710678118654752440f;
constexpr float kC8 = 0.92387953251128675613f;
constexpr float kS8 = 0.38268343236508977173f;

// a * exp(S i pi/2): -i a for S = -1, +i a for S = +1
template <int S>
__device__ __forceinline__ float2 mul_si(float2 a) {
  return S < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// a times the forward-sign root w (S = -1) or its conjugate (S = +1)
template <int S>
__device__ __forceinline__ float2 mul_root(float2 a, float2 w) {
  return S < 0 ? cmul(a, w) : cmulc(a, w);
}

__device__ __forceinline__ void dft2(float2& a0, float2& a1) {
  const float2 t = a0;
  a0 = padd(t, a1);
  a1 = psub(t, a1);
}

template <int S>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = padd(a0, a2), t1 = psub(a0, a2);
  const float2 t2 = padd(a1, a3), d = mul_si<S>(psub(a1, a3));
  a0 = padd(t0, t2);
  a2 = psub(t0, t2);
  a1 = make_float2(t1.x + d.x, t1.y + d.y);
  a3 = make_float2(t1.x - d.x, t1.y - d.y);
}

// Radix-2 split into two length-4 DFTs (even / odd inputs), roots w8^k, w8 = exp(S i pi/4).
template <int S>
__device__ __forceinline__ void dft8(float2* a) {
  float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  float2 o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<S>(e0, e1, e2, e3);
  dft4<S>(o0, o1, o2, o3);
  o1 = mul_root<S>(o1, make_float2(kC4, -kC4));
  o2 = mul_si<S>(o2);
  o3 = mul_root<S>(o3, make_float2(-kC4, -kC4));
  a[0] = padd(e0, o0); a[4] = psub(e0, o0);
  a[1] = padd(e1, o1); a[5] = psub(e1, o1);
  a[2] = padd(e2, o2); a[6] = psub(e2, o2);
  a[3] = padd(e3, o3); a[7] = psub(e3, o3);
}

// 16 = 4 x 4: length-4 DFTs over the stride-4 groups, roots w16^(j2*k1),
// length-4 DFTs across groups; input index j2 + 4*j1, output index k1 + 4*k2.
template <int S>
__device__ __forceinline__ void dft16(float2* a) {
#pragma unroll
  for (int j2 = 0; j2 < 4; ++j2) dft4<S>(a[j2], a[j2 + 4], a[j2 + 8], a[j2 + 12]);
  // now a[j2 + 4*k1] = B[k1][j2]; multiply by w16^(j2*k1) (forward w16 = exp(-i pi/8))
  const float2 w1 = make_float2(kC8, -kS8), w2 = make_float2(kC4, -kC4), w3 = make_float2(kS8, -kC8);
  a[5] = mul_root<S>(a[5], w1);                          // j2=1,k1=1
  a[6] = mul_root<S>(a[6], w2);                          // j2=2,k1=1
  a[7] = mul_root<S>(a[7], w3);                          // j2=3,k1=1
  a[9] = mul_root<S>(a[9], w2);                          // j2=1,k1=2
  a[10] = mul_si<S>(a[10]);                              // j2=2,k1=2: w^4
  a[11] = mul_root<S>(a[11], make_float2(-kC4, -kC4));   // j2=3,k1=2: w^6
  a[13] = mul_root<S>(a[13], w3);                        // j2=1,k1=3: w^3
  a[14] = mul_root<S>(a[14], make_float2(-kC4, -kC4));   // j2=2,k1=3: w^6
  a[15] = mul_root<S>(a[15], make_float2(-kC8, kS8));    // j2=3,k1=3: w^9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<S>(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
  // a[4*k1 + k2] = X[k1 + 4*k2]: transpose the 4x4 index grid
  float2 t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = a[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = t[4 * k1 + k2];
}

template <int R, int S>
__device__ __forceinline__ void dft_small(float2* a) {
  if constexpr (R == 2) dft2(a[0], a[1]);
  else if constexpr (R == 4) dft4<S>(a[0], a[1], a[2], a[3]);
  else if constexpr (R == 8) dft8<S>(a);
  else if constexpr (R == 16) dft16<S>(a);
  else static_assert(R == 1, "radix must be 1, 2, 4, 8 or 16");
}

// ------------------------------------------------------------ line FFT shape
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// A line of N points is held by P = N/E threads with E elements each. Threads
// are numbered tid = t + T*p (line index t fastest, T lines per CTA): thread
// (t, p) holds "slot" j = position p + j*P of line t. Stages: radix 16 while
// >= 16 remains, then one stage of the remaining radix (N < 16: a single stage
// of radix N).
template <int N>
struct LineShape {
  static constexpr int E = N < 16 ? N : 16;
  static constexpr int P = N / E;
  static constexpr int LOGN = ilog2c(N);
  static constexpr int NSTAGE = N < 16 ? 1 : (LOGN + 3) / 4;
  static constexpr int LS = N + N / 16;  // padded positions per line in the scratch
  __host__ __device__ static constexpr int radix(int s) { return N < 16 ? N : (s < LOGN / 4 ? 16 : (1 << (LOGN % 4))); }
  __host__ __device__ static constexpr int span(int s) { return s == 0 ? 1 : 16 * span(s - 1); }  // Ns of stage s
};

// Padded position: one spare row after every 16 (bank-conflict relief for the
// stride-16 writes of the first stage when fewer than 16 lines share a row).
__host__ __device__ constexpr int pad16(int i) { return i + (i >> 4); }

// Scratch layout: position-major, line-minor -- element (pos, t) at
// pad16(pos) * T + t, so the T lines of one position are contiguous and the
// line-fastest threads of a warp touch consecutive words.
template <int T>
__device__ __forceinline__ int sidx(int pos, int t) { return pad16(pos) * T + t; }

// One Stockham radix-R stage (Govindaraju et al., SC'08 formulation): butterfly b
// reads positions b + r*N/R, applies twiddles W_{Ns R}^{r (b mod Ns)}, a radix-R
// DFT, and writes position (b/Ns)*Ns*R + (b mod Ns) + r*Ns. Butterflies of this
// thread: b = p + q*P, q < E/R; their inputs are slots q + r*E/R.
// tw: shared-memory table W_N^k, k < N.
//
// Addressing is written as a per-thread base plus compile-time offsets. With
// P and 16 powers of two and p < P: pad16(p + j*P) = pad16(p) + pad16(j*P);
// the stages that write back are radix 16: stage 0 (Ns = 1: position
// 16(p + qP) + r, padded 17(p + qP) + r) and later stages with one butterfly
// b = p per thread (P >= Ns): position 16 Ns (p / Ns) + (p mod Ns) + r Ns,
// padded pad16(16 Ns (p / Ns) + (p mod Ns)) + r 17 Ns / 16 (stage 1 of lines
// up to 4096 points, stages 1 and 2 of 8192-point lines); and
// b mod Ns = (p mod Ns) + (qP mod Ns).
template <int N, int T, int S, int DIR, int TWS>
__device__ __forceinline__ void fft_stage(float2 (&v)[LineShape<N>::E], float2* sm, int p, int t, const float2* tw) {
  using LS_ = LineShape<N>;
  constexpr int E = LS_::E, P = LS_::P;
  constexpr int R = LS_::radix(S);
  constexpr int Q = E / R;
  constexpr int Ns = LS_::span(S);
  constexpr bool LAST = (S == LS_::NSTAGE - 1);
  static_assert(LAST || S == 0 || (R == 16 && Q == 1 && P >= Ns), "write-back stages: stage 0 or one butterfly per thread");
  if constexpr (S > 0) {
    const float2* rb = sm + pad16(p) * T + t;
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = rb[pad16(j * P) * T];
    if constexpr (!LAST) __syncthreads();  // everyone read before anyone overwrites
  }
  float2* wb = sm + t;
  if constexpr (!LAST) {
    static_assert(R == 16, "write-back stages are radix 16");
    if constexpr (S == 0) wb += 17 * p * T;
    else wb += pad16(16 * Ns * (p / Ns) + (p & (Ns - 1))) * T;
  }
  const int kp = (P >= Ns) ? (p & (Ns - 1)) : p;  // runtime part of b mod Ns
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float2 a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = v[q + r * Q];
    if constexpr (S > 0) {
      const int kq = (P >= Ns) ? 0 : ((q * P) & (Ns - 1));
      constexpr int step = N / (Ns * R);  // W_{Ns R}^{r k} = W_N^{r k step}
      const int k = kp + kq;
#pragma unroll
      for (int r = 1; r < R; ++r) a[r] = mul_root<DIR>(a[r], tw[r * step * k * TWS]);
    }
    dft_small<R, DIR>(a);
    if constexpr (LAST) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[q + r * Q] = a[r];
    } else if constexpr (S == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) wb[(17 * q * P + r) * T] = a[r];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) wb[r * (Ns + Ns / 16) * T] = a[r];
    }
  }
  if constexpr (!LAST) __syncthreads();
}

// A callable that does nothing (the default hook of line_fft).
struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

template <int N, int T, int S, int DIR, int TWS, class Hook>
__device__ __forceinline__ void fft_stages(float2 (&v)[LineShape<N>::E], float2* sm, int p, int t, const float2* tw,
                                           const Hook& hook) {
  if constexpr (S < LineShape<N>::NSTAGE) {
    fft_stage<N, T, S, DIR, TWS>(v, sm, p, t, tw);
    if constexpr (S == 0 && LineShape<N>::NSTAGE >= 2) hook();  // after stage 0's CTA barrier
    fft_stages<N, T, S + 1, DIR, TWS>(v, sm, p, t, tw, hook);
  }
}

// Unnormalised length-N DFT of line t, sign -1 (DIR < 0) or +1 (DIR > 0).
// In: slot j = position p + j*P; out: slot j = frequency p + j*P (natural order).
// The inverse sign uses the conjugate roots: the table tw holds the forward
// roots, entry k * TWS = W_N^k (a table of W_{N TWS} serves every N that
// divides its length), conjugated where applied. The scratch is shared by the
// CTA's lines: every thread of the block calls this together, and the caller
// synchronises before the call if the scratch was in use. For lines of two or
// more stages, hook() runs once, right after the CTA barrier that ends stage 0
// (every thread is then past all its earlier shared-memory accesses).
template <int N, int T, int DIR, int TWS = 1, class Hook = NoHook>
__device__ __forceinline__ void line_fft(float2 (&v)[LineShape<N>::E], float2* sm, int p, int t, const float2* tw,
                                         const Hook& hook = Hook()) {
  fft_stages<N, T, 0, (DIR > 0 ? 1 : -1), TWS>(v, sm, p, t, tw, hook);
}

// ---------------------------------------------------- compensated summation
// Value = s + c, accumulated with Knuth's error-free two-sum so that the
// rounding error of each addition is carried in c.
struct fsum2 {
  float s, c;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void acc_add(fsum2& A, float x) {
  float s, e;
  two_sum(A.s, x, s, e);
  A.s = s;
  A.c += e;
}

__device__ __forceinline__ fsum2 acc_merge(fsum2 A, fsum2 B) {
  float s, e;
  two_sum(A.s, B.s, s, e);
  return fsum2{s, A.c + B.c + e};
}

// Warp-wide compensated sum (fixed order); result valid in lane 0.
__device__ __forceinline__ float warp_sum(fsum2 A) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    fsum2 B{__shfl_down_sync(0xffffffffu, A.s, off), __shfl_down_sync(0xffffffffu, A.c, off)};
    if ((threadIdx.x & 31) + off < 32) A = acc_merge(A, B);
  }
  return A.s + A.c;
}

// Block-wide compensated sum; result valid in thread 0. `red` holds >= 64 floats.
// Blocks that are not whole warps (tiny sizes, < 32 threads) reduce serially.
__device__ __forceinline__ float block_sum(fsum2 A, float* red) {
  if (blockDim.x % 32 != 0) {
    __syncthreads();
    red[2 * threadIdx.x] = A.s;
    red[2 * threadIdx.x + 1] = A.c;
    __syncthreads();
    float out = 0.f;
    if (threadIdx.x == 0) {
      fsum2 T{red[0], red[1]};
      for (unsigned w = 1; w < blockDim.x; ++w) T = acc_merge(T, fsum2{red[2 * w], red[2 * w + 1]});
      out = T.s + T.c;
    }
    __syncthreads();
    return out;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    fsum2 B{__shfl_down_sync(0xffffffffu, A.s, off), __shfl_down_sync(0xffffffffu, A.c, off)};
    if ((threadIdx.x & 31) + off < 32) A = acc_merge(A, B);
  }
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[2 * warp] = A.s;
    red[2 * warp + 1] = A.c;
  }
  __syncthreads();
  float out = 0.f;
  if (threadIdx.x == 0) {
    fsum2 T{red[0], red[1]};
    for (int w = 1; w < nwarp; ++w) T = acc_merge(T, fsum2{red[2 * w], red[2 * w + 1]});
    out = T.s + T.c;
  }
  __syncthreads();
  return out;
}

// Deterministic compensated sum of `count` partials (serial, fixed order).
__device__ __forceinline__ float sum_partials(const float* __restrict__ part, int count) {
  fsum2 A{0.f, 0.f};
  for (int i = 0; i < count; ++i) acc_add(A, part[i]);
  return A.s + A.c;
}

}  // namespace sr
