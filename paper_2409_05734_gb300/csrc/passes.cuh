// Device templates of the four-step pass kernels (FIRST, MID, LAST) of the
// structured operator A = F D_L ... F D_1 U (Sec. III, Eq. 5).
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
// swizzle; in the persistent grid the staging buffer then serves as the
// scratch of the tile's first line FFT, and the next tile's load is issued
// after the second FFT's first barrier, so it overlaps the rest of the tile.
// Kernels are instantiated per tile shape (line length ELL, lines
// per CTA T) and per transform direction, so that index arithmetic folds and
// the inverse-transform exchanges resolve at compile time.
#pragma once

#include "sr_device.cuh"
#include "sr_internal.h"
#include "sr_tma.cuh"

namespace sr {

// Threads per CTA allowed for lines of length ELL: 256 up to ELL = 512, 512 beyond.
__host__ __device__ constexpr int pass_threads(int ell) { return ell <= 512 ? 256 : 512; }

// Input tiles are staged by TMA when a box row is a whole 128-byte line and the
// box (T rows) fills a 1024-byte swizzle period.
__host__ __device__ constexpr bool uses_tma(int ell, int T) { return ell >= 16 && T >= 8; }

// Tile shape: lines of ELL points, T lines per CTA. NLC is the number of lines
// NL = m / ELL when it is fixed at compile time (specialised kernels for the
// most used lengths: every per-slot offset of the natural-order and exchange
// accesses then folds into an immediate), or 0 to read it from the arguments.
//
// Lines of ELL = 3 M points (M a power of two: the radix-3 lengths m = 3 * 2^a)
// are three interleaved sub-lines of M points with one radix-3 step: thread
// (t, p, rho) holds 16 points of sub-line rho (P threads per sub-line, 3P per
// line). Two slot orders exist per thread, for slot j < 16:
//   block order     position p + rho M + j P            (BSTR = P)
//   stride-3 order  position 3 (p + j P) + rho          (SSTR = 3 P)
// A radix-3 line FFT by decimation in time (fft_s3_to_blk) takes its input in
// stride-3 order and leaves the output in block order; by decimation in
// frequency (fft_blk_to_s3) the other way round. Power-of-two lines have one
// order, p + j P, for both (R = 1, rho = 0).
template <int ELL, int T_, int NLC_ = 0>
struct Tile {
  static constexpr bool R3 = (ELL % 3 == 0);
  static constexpr int R = R3 ? 3 : 1;         // sub-lines per line
  static constexpr int M = ELL / R;            // points per sub-line (a power of two)
  static constexpr int T = T_;
  static constexpr int NLC = NLC_;
  static constexpr int E = LineShape<M>::E, P = LineShape<M>::P;  // P: threads per sub-line
  static constexpr int PL = R * P;             // threads per line
  static constexpr int BSTR = P, SSTR = R * P; // slot strides of the block and stride-3 orders
  static constexpr int THREADS = T * PL;
  static constexpr bool TMA = uses_tma(ELL, T);
  static constexpr int BOX = T * 128;  // bytes of one box: 16 complex values x T rows
  static constexpr int MIN_CTAS = THREADS <= 256 ? 3 : THREADS <= 384 ? 2 : 1;
  // Staged tiles whose line FFT runs through the scratch (two or more stages,
  // or a radix-3 step): the staging buffer, free once the tile is in
  // registers, serves as the first line FFT's scratch, and the next tile's
  // load is issued after the second FFT's first barrier.
  static constexpr bool LATE = TMA && (R3 || LineShape<M>::NSTAGE >= 2);
  static_assert(THREADS <= 512, "tile too large");
  static_assert(NLC == 0 || NLC % T == 0, "lines per CTA must divide the line count");
  __device__ __forceinline__ static int nl(const PassArgs& a) { return NLC ? NLC : a.nl; }
  __device__ __forceinline__ static int m(const PassArgs& a) { return NLC ? NLC * ELL : a.m; }
  __device__ __forceinline__ static int cpp(const PassArgs& a) { return NLC ? NLC / T : a.cpp; }
  // split point of the two-level W_m table: ceil(log2(m) / 2)
  __device__ __forceinline__ static int tw_shift(const PassArgs& a) {
    return NLC ? (ilog2c(NLC * ELL) + 1) / 2 : a.tw_shift;
  }
};

// Thread coordinates (line t, butterfly column p, sub-line rho) with their
// ranges stated to the compiler, which lets it fold the per-slot index
// arithmetic (padding, swizzle, Stockham positions) into immediate offsets.
template <class TL>
__device__ __forceinline__ void thread_coords(int& t, int& p, int& rho) {
  const int tid = threadIdx.x;
  __builtin_assume(tid >= 0 && tid < TL::THREADS);
  t = tid % TL::T;
  const int pl = tid / TL::T;
  __builtin_assume(pl >= 0 && pl < TL::PL);
  p = TL::R3 ? pl % TL::P : pl;
  rho = TL::R3 ? pl / TL::P : 0;
  __builtin_assume(t >= 0 && t < TL::T);
  __builtin_assume(p >= 0 && p < TL::P);
  __builtin_assume(rho >= 0 && rho < TL::R);
}

// First position of this thread's slots in block order (stride BSTR) and in
// stride-3 order (stride SSTR); equal for power-of-two lines.
template <class TL>
__device__ __forceinline__ int blk0(int p, int rho) { return p + rho * TL::M; }
template <class TL>
__device__ __forceinline__ int s30(int p, int rho) { return TL::R * p + rho; }

// ------------------------------------------------------ shared-memory layout
struct PipeSmem {
  size_t in0, in1, scratch, tw, rowtw, bar, total;
};

__host__ __device__ inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Layout relative to a 1024-byte-aligned base; input tiles (T rows of ell
// complex values as ell/16 boxes) in `nbuf` swizzled buffers when staged,
// each large enough to serve as a line-FFT scratch once its tile is in
// registers.
__host__ __device__ inline PipeSmem pipe_layout(int ell, int T, int nbuf, bool stage_input) {
  PipeSmem L;
  const bool tma = stage_input && uses_tma(ell, T);
  const size_t box_bytes = (size_t)(ell / 16) * T * 128, scr_bytes = (size_t)T * (ell + ell / 16) * 8;
  const size_t tile = tma ? round_up(box_bytes > scr_bytes ? box_bytes : scr_bytes, 1024) : 0;
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

// W_m^e = W_m^(hi part) * W_m^(lo part), both tables rounded from double;
// conjugated when dir > 0.
template <class TL>
__device__ __forceinline__ float2 tw_m(const PassArgs& a, int e, int dir) {
  const int sh = TL::tw_shift(a);
  const float2 w = cmul(__ldg(&a.tw_hi[e >> sh]), __ldg(&a.tw_lo[e & ((1 << sh) - 1)]));
  return dir > 0 ? conjf2(w) : w;
}

// Line twiddles W_ELL^k, k < ELL, into shared memory.
template <int ELL>
__device__ __forceinline__ void load_line_twiddles(const PassArgs& a, float2* tw) {
  for (int i = threadIdx.x; i < ELL; i += blockDim.x) tw[i] = __ldg(&a.twl[i * a.tws]);
}

// ------------------------------------------------------------ line FFTs

// W_3^(k mod 3) in the transform's sign (forward exp(-2 pi i / 3); the
// inverse conjugates), for k = 0 .. 4.
template <int DIR>
__device__ __forceinline__ float2 root3(int k) {
  constexpr float kS3 = 0.86602540378443864676f;  // sqrt(3) / 2
  const int r = k % 3;
  const float s = DIR > 0 ? kS3 : -kS3;
  return r == 0 ? make_float2(1.f, 0.f) : make_float2(-0.5f, r == 1 ? s : -s);
}

// Unnormalised DFT of the T lines of a tile, input slots in stride-3 order,
// output slots in block order. Radix-3 lines by decimation in time: with
// u_r[j] = x[3 j + r] and U_r = DFT_M(u_r) (one sub-line each),
//   X[k + s M] = sum_r W_ELL^(r k) W_3^(r s) U_r[k],   k < M, s < 3;
// thread (t, p, rho) forms the outputs s = rho of its k = p + j P, reading the
// three U_r[k] from the scratch. tw: table of W_ELL (entry i * TWS). With
// XSEP the U_r go through a second scratch `xsm` (free on entry), so no
// barrier separates the sub-line FFTs' last reads from the exchange.
template <class TL, int DIR, int TWS, bool XSEP = false>
__device__ __forceinline__ void fft_s3_to_blk(float2 (&v)[TL::E], float2* sm, int p, int rho, int t,
                                              const float2* tw, float2* xsm = nullptr) {
  if constexpr (!TL::R3) {
    line_fft<TL::M, TL::T, DIR, TWS>(v, sm, p, t, tw);
  } else {
    constexpr int T = TL::T, T3 = 3 * TL::T, P = TL::P;
    line_fft<TL::M, T3, DIR, 3 * TWS>(v, sm, p, t + T * rho, tw);
    if constexpr (!XSEP) {
      __syncthreads();  // the sub-line FFTs' last scratch reads are done
      xsm = sm;
    }
#pragma unroll
    for (int j = 0; j < TL::E; ++j) xsm[sidx<T3>(p + j * P, t + T * rho)] = v[j];
    __syncthreads();
    const float2 c1 = root3<DIR>(rho), c2 = root3<DIR>(2 * rho);
#pragma unroll
    for (int j = 0; j < TL::E; ++j) {
      const int k = p + j * P;
      const float2 u0 = xsm[sidx<T3>(k, t)];
      const float2 u1 = mul_root<DIR>(xsm[sidx<T3>(k, t + T)], tw[k * TWS]);
      const float2 u2 = mul_root<DIR>(xsm[sidx<T3>(k, t + 2 * T)], tw[2 * k * TWS]);
      v[j] = padd(u0, padd(cmul(u1, c1), cmul(u2, c2)));
    }
  }
}

// Unnormalised DFT of the T lines of a tile, input slots in block order,
// output slots in stride-3 order. Radix-3 lines by decimation in frequency:
//   X[3 k + s] = DFT_M(u_s)[k],  u_s[k] = W_ELL^(k s) sum_r W_3^(r s) x[k + r M];
// thread (t, p, rho) forms u_rho at its k = p + j P from the three block
// values read from the scratch, then the sub-line FFT. The caller
// synchronises before the call if the scratch was in use. hook() runs once
// after a CTA barrier that every thread reaches after its last access to the
// scratch it ran in before the call (none for single-stage lines). With XSEP
// the block values go through a second scratch `xsm` (free on entry), so no
// barrier separates their reads from the sub-line FFTs; hook() then runs
// after the sub-line FFTs' first barrier, once every thread has read xsm.
template <class TL, int DIR, int TWS, bool XSEP = false, class Hook = NoHook>
__device__ __forceinline__ void fft_blk_to_s3(float2 (&v)[TL::E], float2* sm, int p, int rho, int t,
                                              const float2* tw, const Hook& hook = Hook(), float2* xsm = nullptr) {
  if constexpr (TL::R3) {
    constexpr int T = TL::T, T3 = 3 * TL::T, P = TL::P;
    if constexpr (!XSEP) xsm = sm;
#pragma unroll
    for (int j = 0; j < TL::E; ++j) xsm[sidx<T3>(p + j * P, t + T * rho)] = v[j];
    __syncthreads();
    if constexpr (!XSEP) hook();
    const float2 c1 = root3<DIR>(rho), c2 = root3<DIR>(2 * rho);
#pragma unroll
    for (int j = 0; j < TL::E; ++j) {
      const int k = p + j * P;
      const float2 x0 = xsm[sidx<T3>(k, t)], x1 = xsm[sidx<T3>(k, t + T)], x2 = xsm[sidx<T3>(k, t + 2 * T)];
      const float2 u = padd(x0, padd(cmul(x1, c1), cmul(x2, c2)));
      v[j] = mul_root<DIR>(u, tw[rho * k * TWS]);
    }
    if constexpr (XSEP) {
      fence_proxy_async_smem();  // xsm may next be written by a TMA load (issued by hook)
      line_fft<TL::M, T3, DIR, 3 * TWS>(v, sm, p, t + T * rho, tw, hook);
    } else {
      __syncthreads();  // every block value read before the sub-line FFT writes the scratch
      line_fft<TL::M, T3, DIR, 3 * TWS>(v, sm, p, t + T * rho, tw);
    }
  } else {
    line_fft<TL::M, TL::T, DIR, TWS>(v, sm, p, t, tw, hook);
  }
}

// The four-step twiddle of (line g, frequency f = f0 + j*SSTR), f0 the
// thread's first stride-3-order position (p for power-of-two lines), is
// W_m^(g f0) * W_m^(g SSTR j); the second factor is tabulated per tile,
// rowtw[j*T + t] = W_m^((g0 + t) SSTR j). RowTw holds this thread's entries of
// the table between their (early) load and their (late) store to shared memory.
template <class TL>
struct RowTw {
  static constexpr int N = (TL::E * TL::T + TL::THREADS - 1) / TL::THREADS;
  float2 w[N];
  __device__ __forceinline__ void load(const PassArgs& a, int g0, int dir) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int i = threadIdx.x + k * TL::THREADS;
      if (i < TL::E * TL::T) w[k] = tw_m<TL>(a, (g0 + i % TL::T) * TL::SSTR * (i / TL::T), dir);
    }
  }
  __device__ __forceinline__ void store(float2* rowtw) const {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int i = threadIdx.x + k * TL::THREADS;
      if (i < TL::E * TL::T) rowtw[i] = w[k];
    }
  }
};

// Step-1 outputs of line g (slots in stride-3 order from f0) times the
// four-step twiddles (already conjugated for an inverse transform), stored to
// the exchange buffer at f*NL + g (T consecutive elements per frequency across
// the warp).
template <class TL>
__device__ __forceinline__ void twiddle_store(float2 (&v)[TL::E], const PassArgs& a, int b, int g, int t, int f0,
                                              float2 A, const float2* rowtw) {
  float2* eb = a.eout + (size_t)b * TL::m(a) + g;
#pragma unroll
  for (int j = 0; j < TL::E; ++j) {
    const float2 w = cmul(A, rowtw[j * TL::T + t]);
    eb[(size_t)(f0 + j * TL::SSTR) * TL::nl(a)] = cmul(v[j], w);
  }
}

// Measurements an epilogue needs at (line g, frequency f), natural index
// f*NL + g, loaded before the pass's first FFT so that their latency overlaps
// it. (Diagonal entries are read where they are applied: they are shared by
// all problems of a batch -- or, with dp_stride != 0, one table per problem --
// and stay in L2.)
template <class TL>
struct OpData {
  float y[TL::E];
  float vscale = 1.0f;  // spectral epilogue: 1/||u|| of the current iterate (when applied here)
  // q0: the thread's first block-order position (slot j at q0 + j*BSTR)
  __device__ __forceinline__ void load_y(const PassArgs& a, int op, int b, int g, int q0) {
    if (op == kOpGdEpilogue || op == kOpSpecEpilogue) {
      const float* yb = a.y + (size_t)b * TL::m(a) + g;
#pragma unroll
      for (int j = 0; j < TL::E; ++j) y[j] = __ldg(&yb[(q0 + j * TL::BSTR) * TL::nl(a)]);
    }
  }
};

// The operation at natural index (q0 + j*BSTR)*NL + g of slot j (block order).
template <class TL, bool EPI = true, bool DIAG = true>
__device__ __forceinline__ void apply_op(float2 (&v)[TL::E], const PassArgs& a, const OpData<TL>& od, int b, int g,
                                         int q0, fsum2& acc) {
  if (DIAG && a.op == kOpDiag) {
    const float2* dp = a.dp + (size_t)b * a.dp_stride;
#pragma unroll
    for (int j = 0; j < TL::E; ++j) v[j] = cmul(v[j], __ldg(&dp[(q0 + j * TL::BSTR) * TL::nl(a) + g]));
  } else if (DIAG && a.op == kOpDiagConj) {
    const float2* dp = a.dp + (size_t)b * a.dp_stride;
#pragma unroll
    for (int j = 0; j < TL::E; ++j) v[j] = cmulc(v[j], __ldg(&dp[(q0 + j * TL::BSTR) * TL::nl(a) + g]));
  } else if (EPI && a.op == kOpGdEpilogue) {
    // z -> r = |z|^2 - y, w = r z (Eq. 2); loss partial sum of r^2
#pragma unroll
    for (int j = 0; j < TL::E; ++j) {
      const float r = cabs2(v[j]) - od.y[j];
      acc_add(acc, r * r);
      v[j] = cscale(v[j], r);
    }
  } else if (EPI && a.op == kOpSpecEpilogue) {
    // z -> T(y_hat) z, y_hat = m y / sum(y) (Eq. 3); times 1/||u|| when the
    // iterate's normalisation is applied here rather than at the chain's input
    const float scale = (float)TL::m(a) / __ldg(&a.sumy[b]);
#pragma unroll
    for (int j = 0; j < TL::E; ++j) {
      const float yh = od.y[j] * scale;
      float w;
      if (a.weight_mode == SR_WEIGHT_IDENTITY) w = yh;
      else w = yh > 0.f ? fmaxf(1.0f - 1.0f / yh, a.lam) : a.lam;
      v[j] = cscale(v[j], w * od.vscale);
    }
  }
}

// 2D grids (S x S, row-major; MAP = 1 kernels). Without its twiddles the
// four-step DFT of a grid is the 2D DFT with its output transposed, so a chain
// alternates between the grid and its transpose: layout element (row, col)
// holds signal entry (col, row) when `tr` is set. Flat index of the entry of an
// h x w row-major signal that layout element (row, col) holds, or -1 outside
// the h x w corner (the zero padding U2 and the crop U2^H).
__device__ __forceinline__ int grid_index(int row, int col, int h, int w, int tr) {
  if (tr) {
    const int t = row;
    row = col;
    col = t;
  }
  return (row < h && col < w) ? row * w + col : -1;
}

// Shared scalars of one tile (every pass kernel declares one in shared memory).
struct TileScalars {
  float red[64];   // block reductions
  float scale;     // FIRST: input scale; MID (spectral epilogue): 1/||u||
  float inv_old;   // LAST / fused: 1/||v_old|| of the power iterate
  float mu;        // LAST / fused: the problem's step
};

// The T input lines of a tile staged by TMA (boxes of 16 values x T rows,
// 128-byte swizzle) into registers: slot j = position p + j*P.
// swz128_offset(BOX, t, p + j*P) as a per-thread base plus a per-slot
// constant: for P >= 16 the slot only moves the box; for P < 16 it adds
// (j*P) & 15 to the 16-byte chunk index, whose bits are disjoint from p's.
// Radix-3 lines: slot j is position q = s30 + j*SSTR (stride-3 order), at
// byte (q / 16) * BOX + t * 128 + ((q % 16) * 8 ^ (t % 8) * 16).
template <class TL>
__device__ __forceinline__ void load_staged(const unsigned char* src, int t, int p, int rho, float2 (&v)[TL::E]) {
  constexpr int E = TL::E, P = TL::P;
  const int t7 = t & 7;
  if constexpr (TL::R3) {
    const int q0 = s30<TL>(p, rho);
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int q = q0 + j * TL::SSTR;
      v[j] = *reinterpret_cast<const float2*>(src + (q >> 4) * TL::BOX + t * 128 + (((q & 15) << 3) ^ (t7 << 4)));
    }
  } else if constexpr (P >= 16) {
    const unsigned char* base = src + (p >> 4) * TL::BOX + t * 128 + (((p & 15) << 3) ^ (t7 << 4));
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = *reinterpret_cast<const float2*>(base + j * (P / 16) * TL::BOX);
  } else {
    const int base = t * 128 + ((p << 3) ^ (t7 << 4));
#pragma unroll
    for (int j = 0; j < E; ++j)
      v[j] = *reinterpret_cast<const float2*>(src + ((j * P) >> 4) * TL::BOX + (base ^ (((j * P) & 15) << 3)));
  }
}

// ------------------------------------------------------------ FIRST pass

// One tile of a FIRST pass: natural-order input of problem b (zero beyond
// n_in: the padding U), the operation before DFT 0, step 1 of DFT 0 and the
// four-step twiddles, into the exchange buffer. tw: line twiddles, entry
// k * TWS = W_ELL^k. The caller synchronises before the next tile.
template <class TL, int DB, int MAP, int TWS>
__device__ __forceinline__ void first_tile(const PassArgs& a, int b, int g0, int t, int p, int rho, float2* scratch,
                                           const float2* tw, float2* rowtw, TileScalars& sh) {
  constexpr int E = TL::E, P = TL::P, T = TL::T;
  const int q0 = blk0<TL>(p, rho), f0 = s30<TL>(p, rho);
  const int tid = threadIdx.x;
  const int g = g0 + t;
  RowTw<TL> rw;
  rw.load(a, g0, DB);
  rw.store(rowtw);
  const float2 A = tw_m<TL>(a, g * f0, DB);
  // Radix-3 lengths (a.r3): inner problem b = 3 bo + r holds the stride-3
  // subsequence r of outer problem bo (element 3 nat + r), and the operation
  // that precedes this DFT is applied at that outer natural index.
  const int bo = a.r3 ? b / 3 : b, rr = a.r3 ? b - 3 * bo : 0;
  if (tid == 0)
    sh.scale = a.norm_in ? 1.0f / sqrtf(sum_partials(a.norm_in + (size_t)bo * a.norm_in_count, a.norm_in_count))
                         : 1.0f;
  // Natural-order input, zero beyond n_in (the padding U): element (line g,
  // position q) is x[q*NL + g], slot j at q = q0 + j*P (block order); the
  // warp reads T consecutive elements.
  const float2* xb = a.xin + (size_t)bo * a.n_in;
  // (2D grids: the signal entry at grid_index, tables at the layout index nat)
  float2 v[E];
  int idx[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int nat = (q0 + j * P) * TL::nl(a) + g;
    if constexpr (MAP) {
      idx[j] = nat;
      const int xi = grid_index(q0 + j * P, g, a.in_h, a.in_w, a.in_tr);
      v[j] = xi >= 0 ? xb[xi] : make_float2(0.f, 0.f);
    } else {
      // in_off: the input is the window off .. off+n_in-1 of the length-m
      // vector (S^H of the alpha < 1 branch; zero outside)
      idx[j] = a.r3 ? 3 * nat + rr : nat - a.in_off;
      v[j] = (unsigned)idx[j] < (unsigned)a.n_in ? xb[idx[j]] : make_float2(0.f, 0.f);
    }
  }
  if (a.op == kOpDiag) {
    const float2* dp = a.dp + (size_t)bo * a.dp_stride;
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = cmul(v[j], __ldg(&dp[idx[j]]));
  } else if (a.op == kOpDiagConj) {
    const float2* dp = a.dp + (size_t)bo * a.dp_stride;
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = cmulc(v[j], __ldg(&dp[idx[j]]));
  } else if (a.op == kOpGdEpilogue) {  // (radix-3, alpha < 1 chains) r = |z|^2 - y, w = r z, loss partials
    const float* yb = a.y + (size_t)bo * a.ym;
    fsum2 acc{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < E; ++j) {
      if ((unsigned)idx[j] < (unsigned)a.ym) {  // outside the measurement window: w = 0
        const float res = cabs2(v[j]) - __ldg(&yb[idx[j]]);
        acc_add(acc, res * res);
        v[j] = cscale(v[j], res);
      }
    }
    const float sum = block_sum(acc, sh.red);
    if (tid == 0) a.part_out[(size_t)b * TL::cpp(a) + g0 / T] = sum;
  } else if (a.op == kOpSpecEpilogue) {  // (radix-3, alpha < 1 chains) w = T(y_hat) z
    const float* yb = a.y + (size_t)bo * a.ym;
    const float ysc = (float)a.ym / __ldg(&a.sumy[bo]);
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const float yh = (unsigned)idx[j] < (unsigned)a.ym ? __ldg(&yb[idx[j]]) * ysc : 0.f;
      float w = yh;
      if (a.weight_mode == SR_WEIGHT_OPTIMAL) w = yh > 0.f ? fmaxf(1.0f - 1.0f / yh, a.lam) : a.lam;
      v[j] = cscale(v[j], w);
    }
  }
  __syncthreads();  // sh.scale and the row twiddles visible
  const float sc = sh.scale;
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = cscale(v[j], sc);
  fft_blk_to_s3<TL, DB, TWS>(v, scratch, p, rho, t, tw);
  twiddle_store<TL>(v, a, b, g, t, f0, A, rowtw);
}

template <int ELL, int T, int DB, int MAP = 0>
__global__ void __launch_bounds__(Tile<ELL, T>::THREADS, Tile<ELL, T>::MIN_CTAS)
    k_first(const __grid_constant__ PassArgs a) {
  using TL = Tile<ELL, T>;
  extern __shared__ unsigned char smem_raw[];
  __shared__ TileScalars sh;
  unsigned char* smem = aligned_smem(smem_raw);
  const PipeSmem L = pipe_layout(ELL, T, 1, false);
  float2* scratch = reinterpret_cast<float2*>(smem + L.scratch);
  float2* tw = reinterpret_cast<float2*>(smem + L.tw);
  float2* rowtw = reinterpret_cast<float2*>(smem + L.rowtw);
  int t, p, rho;
  thread_coords<TL>(t, p, rho);
  load_line_twiddles<ELL>(a, tw);  // once per CTA: the grid is persistent over the tiles
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int b = tile / a.cpp, g0 = (tile - b * a.cpp) * T;
    first_tile<TL, DB, MAP, 1>(a, b, g0, t, p, rho, scratch, tw, rowtw, sh);
    __syncthreads();  // scratch, row twiddles and sh.scale are reused by the next tile
  }
}

// ------------------------------------------------------ MID and LAST passes

// Issues the TMA loads of one tile -- T rows of ELL complex values starting at
// row `row` of the tensor `map`, as boxes of 16 values x T rows -- into `buf`,
// completing on barrier `bar`.
__device__ __forceinline__ void issue_rows(const CUtensorMap* map, int row, int ell, int T, int box, uint32_t buf,
                                           uint32_t bar) {
  mbar_arrive_expect_tx(bar, (uint32_t)(T * ell * 8));
#pragma unroll 1
  for (int kb = 0; kb < ell / 16; ++kb) tma_load_2d(buf + (uint32_t)(kb * box), map, kb * 32, row, bar);
}

template <class TL, int ELL>
__device__ __forceinline__ void issue_tile(const PassArgs& a, int tile, uint32_t buf, uint32_t bar) {
  const int b = tile / TL::cpp(a), g0 = (tile - b * TL::cpp(a)) * TL::T;
  issue_rows(&a.tmap, b * TL::nl(a) + g0, ELL, TL::T, TL::BOX, buf, bar);
}

// The request of the next tile's load (thread 0 acts; nothing when the tile
// does not exist or the pass issues its loads early).
template <class TL, int ELL>
struct NextLoad {
  const PassArgs* a;
  int next;
  uint32_t buf, bar;
  __device__ __forceinline__ void operator()() const {
    if constexpr (TL::LATE) {
      if (threadIdx.x == 0 && next < a->ntiles) {
        fence_proxy_async_smem();
        issue_tile<TL, ELL>(*a, next, buf, bar);
      }
    }
  }
};

// Shared pipeline of the persistent MID / LAST passes: for every tile of this
// CTA, loads the T input lines (rows of the exchange buffer) into registers
// (slots in stride-3 order: slot j = position s30 + j*SSTR, which is p + j*P
// for power-of-two lines) and calls body(v, b, g0, scr1, issue): scr1 is the
// scratch for the tile's first line FFT and issue() the request of the next
// tile's load. With TL::LATE, scr1 is the staging buffer itself and the body
// calls issue() (every thread; thread 0 acts) once every thread is past its
// last access to scr1; otherwise scr1 is the regular scratch, the next load
// is already in flight and issue() does nothing. One staging buffer (nbuf = 1).
template <int ELL, class TL, class Body>
__device__ __forceinline__ void pipe_tiles(const PassArgs& a, int nbuf, unsigned char* smem, const PipeSmem& L,
                                           float2* scratch, Body&& body) {
  constexpr int E = TL::E, T = TL::T;
  (void)nbuf;
  const int tid = threadIdx.x;
  int t, p, rho;
  thread_coords<TL>(t, p, rho);
  // an earlier pass gave up (see mbar_wait_bounded): do nothing
  if (__syncthreads_or(tid == 0 && *(volatile int*)a.err != 0)) return;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar);
  const uint32_t bar0 = smem_addr(&bars[0]);
  const uint32_t in0 = smem_addr(smem + L.in0);
  float2* stage_scr = reinterpret_cast<float2*>(smem + L.in0);
  int tile = blockIdx.x;
  if constexpr (TL::TMA) {
    if (tid == 0) {
      mbar_init(bar0, 1);
      mbar_init_fence();
    }
    __syncthreads();
    if (tid == 0 && tile < a.ntiles) issue_tile<TL, ELL>(a, tile, in0, bar0);
  }
  for (int k = 0; tile < a.ntiles; ++k, tile += gridDim.x) {
    const int b = tile / TL::cpp(a), g0 = (tile - b * TL::cpp(a)) * T, g = g0 + t;
    const int next = tile + (int)gridDim.x;
    float2 v[E];
    const NextLoad<TL, ELL> issue{&a, next, in0, bar0};
    if constexpr (TL::TMA) {
      const bool ok = mbar_wait_bounded(bar0, (uint32_t)(k & 1));
      if (ok) load_staged<TL>(smem + L.in0, t, p, rho, v);
      // one barrier: every thread has its slots before the buffer is reused,
      // and every thread learns whether any wait gave up
      if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicExch(a.err, (int)SR_ERR_TIMEOUT);  // a load never completed: record it, stop
        return;
      }
      if (!TL::LATE && tid == 0 && next < a.ntiles) {
        fence_proxy_async_smem();
        issue_tile<TL, ELL>(a, next, in0, bar0);
      }
    } else {
      const float2* src = a.ein + (size_t)b * TL::m(a) + (size_t)g * ELL + s30<TL>(p, rho);
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = src[j * TL::SSTR];
    }
    body(v, b, g0, TL::LATE ? stage_scr : scratch, issue);
    // Scratch, tables and shared scalars are free for the next tile. With TMA
    // staging the barrier that follows the next tile's register load already
    // orders this tile's last shared-memory reads before the next tile's first
    // writes, so no barrier is needed here.
    if (!TL::TMA) __syncthreads();
  }
}

// One tile of a MID pass: step 2 of the previous DFT (direction DA) on the T
// lines in v, the fused operation (D_l, D_l^H, the GD residual with loss
// partials, or the spectral weights), step 1 of the next DFT (direction DB)
// and the four-step twiddles, into the exchange buffer. With SPLIT the first
// FFT runs in scr1 (the staging buffer) and the second in `scratch`, so no
// barrier separates them; issue() runs after the second FFT's first barrier.
template <class TL, int DA, int DB, int TWS, bool SPLIT = false, class Hook = NoHook>
__device__ __forceinline__ void mid_tile(const PassArgs& a, float2 (&v)[TL::E], int b, int g0, int t, int p, int rho,
                                         float2* scratch, const float2* tw, float2* rowtw, TileScalars& sh,
                                         float2* scr1 = nullptr, const Hook& issue = Hook()) {
  constexpr int T = TL::T;
  // the first FFT leaves its output in block order (slot j at frequency
  // q0 + j*BSTR), where the operation applies; the second writes stride-3
  // order (f0 + j*SSTR)
  const int q0 = blk0<TL>(p, rho), f0 = s30<TL>(p, rho);
  // The chains apply an epilogue (GD residual or spectral weights) exactly
  // between a forward and an inverse DFT, and diagonals (or nothing) between
  // two DFTs of one direction, so each direction pair compiles only its own
  // operations (fewer live registers: no spills at three CTAs per SM).
  constexpr bool EPI = DA < 0 && DB > 0;
  constexpr bool DIAG = !EPI;
  const int tid = threadIdx.x;
  const int g = g0 + t;
  OpData<TL> od;
  if constexpr (EPI) od.load_y(a, a.op, b, g, q0);
  const bool vs = EPI && a.op == kOpSpecEpilogue && a.norm_in;
  if (vs && tid == 0)
    sh.scale = 1.0f / sqrtf(sum_partials(a.norm_in + (size_t)b * a.norm_in_count, a.norm_in_count));
  // Diagonal passes with a phase table: theta_l (4 bytes an entry, half of
  // D_l) is loaded before the first FFT so that its latency overlaps it, and
  // exp(i theta) is formed in registers (__sincosf: absolute error below
  // 4e-7 on [-pi, pi)); D_l's 1/sqrt(m) rides on the four-step twiddle.
  float th[TL::E];
  const bool phs = DIAG && a.ph != nullptr && (a.op == kOpDiag || a.op == kOpDiagConj);
  if (phs) {
    const float* pb = a.ph + (size_t)b * a.dp_stride;
#pragma unroll
    for (int j = 0; j < TL::E; ++j) th[j] = __ldg(&pb[(q0 + j * TL::BSTR) * TL::nl(a) + g]);
  }
  // four-step twiddles of the second FFT, loaded early so that their latency
  // overlaps the first FFT
  RowTw<TL> rw;
  rw.load(a, g0, DB);
  float2 A = tw_m<TL>(a, g * f0, DB);
  fft_s3_to_blk<TL, DA, TWS, SPLIT>(v, SPLIT ? scr1 : scratch, p, rho, t, tw, scratch);
  fsum2 acc{0.f, 0.f};
  if (vs) {
    __syncthreads();  // sh.scale visible
    od.vscale = sh.scale;
  }
  if (phs) {
    const bool cj = a.op == kOpDiagConj;
#pragma unroll
    for (int j = 0; j < TL::E; ++j) {
      float sn, cs;
      __sincosf(th[j], &sn, &cs);
      v[j] = cj ? cmulc(v[j], make_float2(cs, sn)) : cmul(v[j], make_float2(cs, sn));
    }
    A = cscale(A, a.dscale);
  } else {
    apply_op<TL, EPI, DIAG>(v, a, od, b, g, q0, acc);
  }
  if (EPI && a.op == kOpGdEpilogue) {
    if constexpr (TL::THREADS % 32 == 0) {
      // one partial per warp (no CTA barrier): [B][tiles][warps]
      const float s = warp_sum(acc);
      if ((tid & 31) == 0) a.part_out[((size_t)b * TL::cpp(a) + g0 / T) * (TL::THREADS / 32) + (tid >> 5)] = s;
    } else {
      const float s = block_sum(acc, sh.red);
      if (tid == 0) a.part_out[(size_t)b * TL::cpp(a) + g0 / T] = s;
    }
  }
  rw.store(rowtw);
  if constexpr (SPLIT) {
    // the second FFT's first barrier orders the row twiddles before their use
    // and every access to scr1 before the next tile's load into it
    fence_proxy_async_smem();
    fft_blk_to_s3<TL, DB, TWS, SPLIT>(v, scratch, p, rho, t, tw, issue, scr1);
  } else {
    __syncthreads();  // first FFT's scratch reads done; row twiddles visible
    fft_blk_to_s3<TL, DB, TWS>(v, scratch, p, rho, t, tw);
  }
  twiddle_store<TL>(v, a, b, g, t, f0, A, rowtw);
}

template <int ELL, int T, int DA, int DB, int NLC = 0>
__global__ void __launch_bounds__(Tile<ELL, T>::THREADS, Tile<ELL, T>::MIN_CTAS)
    k_mid(const __grid_constant__ PassArgs a, int nbuf) {
  using TL = Tile<ELL, T, NLC>;
  constexpr int E = TL::E;
  extern __shared__ unsigned char smem_raw[];
  __shared__ TileScalars sh;
  unsigned char* smem = aligned_smem(smem_raw);
  const PipeSmem L = pipe_layout(ELL, T, nbuf, true);
  float2* scratch = reinterpret_cast<float2*>(smem + L.scratch);
  float2* tw = reinterpret_cast<float2*>(smem + L.tw);
  float2* rowtw = reinterpret_cast<float2*>(smem + L.rowtw);
  int t, p, rho;
  thread_coords<TL>(t, p, rho);
  load_line_twiddles<ELL>(a, tw);
  __syncthreads();
  pipe_tiles<ELL, TL>(a, nbuf, smem, L, scratch, [&](float2 (&v)[E], int b, int g0, float2* scr1, const NextLoad<TL, ELL>& issue) {
    mid_tile<TL, DA, DB, 1, TL::LATE>(a, v, b, g0, t, p, rho, scratch, tw, rowtw, sh, scr1, issue);
  });
}

// One tile of a LAST pass: step 2 of the final DFT (direction DA), D_1^H on
// the kept entries and the natural-order output or solver update (U^H: only
// entries < n_out are written).
template <class TL, int DA, int MAP, int TWS, bool SPLIT = false, class Hook = NoHook>
__device__ __forceinline__ void last_tile(const PassArgs& a, float2 (&v)[TL::E], int b, int g0, int t, int p, int rho,
                                          float2* scratch, const float2* tw, TileScalars& sh,
                                          float2* scr1 = nullptr, const Hook& issue = Hook()) {
  constexpr int E = TL::E, P = TL::P, T = TL::T;
  const int q0 = blk0<TL>(p, rho);  // the output's block order: slot j at frequency q0 + j*P
  const int tid = threadIdx.x;
  const int g = g0 + t;
  if (tid == 0) {
    sh.inv_old = (a.out_mode == kOutSpec && a.norm_in)
                     ? 1.0f / sqrtf(sum_partials(a.norm_in + (size_t)b * a.norm_in_count, a.norm_in_count))
                     : 1.0f;
    sh.mu = a.mu ? a.mu[b] : 0.f;
  }
  fft_s3_to_blk<TL, DA, TWS, SPLIT>(v, SPLIT ? scr1 : scratch, p, rho, t, tw, scratch);
  if constexpr (SPLIT) fence_proxy_async_smem();
  __syncthreads();  // tile scalars visible (and, with SPLIT, scr1 free for the next load)
  if constexpr (SPLIT) issue();
  // natural index of (line g, frequency f) is f*NL + g; keep those < n_out
  // (U^H), and apply D_1^H only to the kept entries
  float2* xb = a.xout + (size_t)b * a.n_out;
  const float inv_old = sh.inv_old, mu2 = 2.0f * sh.mu * a.mu_scale, shv = a.shift * inv_old;
  fsum2 acc{0.f, 0.f};
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int nat = (q0 + j * P) * TL::nl(a) + g;
    // output index: the prefix n_out (U^H), the window out_off .. out_off+n_out-1
    // (S of the alpha < 1 branch), or grid_index (2D grids); tables stay at nat
    int oi = nat - a.out_off;
    if constexpr (MAP) {
      oi = grid_index(q0 + j * P, g, a.out_h, a.out_w, a.out_tr);
      if (oi < 0) continue;
    } else {
      if ((unsigned)oi >= (unsigned)a.n_out) continue;
    }
    float2 val = v[j];
    if (a.op == kOpDiagConj) val = cmulc(val, __ldg(&a.dp[(size_t)b * a.dp_stride + nat]));
    if (a.out_mode == kOutStore) {
      xb[oi] = val;
    } else if (a.out_mode == kOutGrad) {
      xb[oi] = cscale(val, 2.0f);
    } else if (a.out_mode == kOutGd) {
      float2 x = xb[oi];
      x.x = fmaf(-mu2, val.x, x.x);
      x.y = fmaf(-mu2, val.y, x.y);
      xb[oi] = x;
    } else {  // kOutSpec
      const float2 old = xb[oi];
      const float2 u = make_float2(fmaf(shv, old.x, val.x), fmaf(shv, old.y, val.y));
      xb[oi] = u;
      acc_add(acc, cabs2(u));
    }
  }
  if (a.out_mode == kOutSpec) {
    const float s = block_sum(acc, sh.red);
    if (tid == 0) a.part_out[(size_t)b * TL::cpp(a) + g0 / T] = s;
  }
  if (a.loss_out && g0 == 0 && tid == 0)
    a.loss_out[b] = sum_partials(a.loss_part + (size_t)b * a.loss_cpp, a.loss_cpp);
}

template <int ELL, int T, int DA, int NLC = 0, int MAP = 0>
__global__ void __launch_bounds__(Tile<ELL, T>::THREADS, Tile<ELL, T>::MIN_CTAS)
    k_last(const __grid_constant__ PassArgs a, int nbuf) {
  using TL = Tile<ELL, T, NLC>;
  constexpr int E = TL::E;
  extern __shared__ unsigned char smem_raw[];
  __shared__ TileScalars sh;
  unsigned char* smem = aligned_smem(smem_raw);
  const PipeSmem L = pipe_layout(ELL, T, nbuf, true);
  float2* scratch = reinterpret_cast<float2*>(smem + L.scratch);
  float2* tw = reinterpret_cast<float2*>(smem + L.tw);
  int t, p, rho;
  thread_coords<TL>(t, p, rho);
  load_line_twiddles<ELL>(a, tw);
  __syncthreads();
  pipe_tiles<ELL, TL>(a, nbuf, smem, L, scratch, [&](float2 (&v)[E], int b, int g0, float2* scr1, const NextLoad<TL, ELL>& issue) {
    last_tile<TL, DA, MAP, 1, TL::LATE>(a, v, b, g0, t, p, rho, scratch, tw, sh, scr1, issue);
  });
}


// LAST of one GD or power-iteration step fused with FIRST of the next. Both
// work on the lines of layout X: step 2 of the final inverse DFT, D_1^H, the
// update on the kept entries (U^H) -- x <- x - mu_t 2 (.) for GD, or
// u <- (.) + shift v (with norm partials of u) for the power iteration, whose
// 1/||u|| the next step applies in its spectral epilogue -- and then, still in
// registers, U (zeros beyond n), D_1 and step 1 of the next step's first
// forward DFT, with the four-step twiddles, into the exchange buffer `eout`.
// Each D_1 entry is loaded once for both uses.
template <class TL, int MAP, int TWS, bool SPLIT = false, class Hook = NoHook>
__device__ __forceinline__ void last_first_tile(const PassArgs& a, float2 (&v)[TL::E], int b, int g0, int t, int p,
                                                int rho, float2* scratch, const float2* tw, float2* rowtw,
                                                TileScalars& sh, float2* scr1 = nullptr,
                                                const Hook& issue = Hook()) {
  constexpr int E = TL::E, P = TL::P, T = TL::T;
  // the inverse DFT's output and the update in block order (q0 + j*P); the
  // next forward DFT's step-1 output in stride-3 order (f0 + j*SSTR)
  const int q0 = blk0<TL>(p, rho), f0 = s30<TL>(p, rho);
  const int tid = threadIdx.x;
  const int g = g0 + t;
  const bool spec = a.out_mode == kOutSpec;
  if (tid == 0) {
    sh.mu = spec ? 0.f : a.mu[b];
    sh.inv_old = spec && a.norm_in
                     ? 1.0f / sqrtf(sum_partials(a.norm_in + (size_t)b * a.norm_in_count, a.norm_in_count))
                     : 1.0f;
  }
  RowTw<TL> rw;
  rw.load(a, g0, -1);
  const float2 A = tw_m<TL>(a, g * f0, -1);
  fft_s3_to_blk<TL, 1, TWS, SPLIT>(v, SPLIT ? scr1 : scratch, p, rho, t, tw, scratch);
  // tile scalars visible: with SPLIT the first FFT's own barriers publish them
  // (it runs through the scratch), otherwise a barrier here
  if constexpr (!SPLIT) __syncthreads();
  const float mu2 = 2.0f * sh.mu * a.mu_scale, shv = a.shift * sh.inv_old;
  float2* xb = a.xout + (size_t)b * a.n_out;
  const float2* dp = a.dp + (size_t)b * a.dp_stride;
  fsum2 acc{0.f, 0.f};
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int nat = (q0 + j * P) * TL::nl(a) + g;
    // signal index (2D grids: grid_index, with U2 and U2^H the same corner)
    int xi = nat;
    bool keep;
    if constexpr (MAP) {
      xi = grid_index(q0 + j * P, g, a.out_h, a.out_w, 0);
      keep = xi >= 0;
    } else {
      keep = nat < a.n_out;
    }
    if (keep) {
      const float2 d = __ldg(&dp[nat]);
      const float2 gr = cmulc(v[j], d);
      float2 x = xb[xi];
      if (spec) {  // u = M v + shift v with v = x / ||x|| (x unnormalised)
        x = make_float2(fmaf(shv, x.x, gr.x), fmaf(shv, x.y, gr.y));
        acc_add(acc, cabs2(x));
      } else {     // x <- x - mu_t 2 A^H(r z)
        x.x = fmaf(-mu2, gr.x, x.x);
        x.y = fmaf(-mu2, gr.y, x.y);
      }
      xb[xi] = x;
      v[j] = cmul(x, d);
    } else {
      v[j] = make_float2(0.f, 0.f);
    }
  }
  if (spec) {
    const float s = block_sum(acc, sh.red);
    if (tid == 0) a.part_out[(size_t)b * TL::cpp(a) + g0 / T] = s;
  }
  if (a.loss_out && g0 == 0 && tid == 0)
    a.loss_out[b] = sum_partials(a.loss_part + (size_t)b * a.loss_cpp, a.loss_cpp);
  rw.store(rowtw);
  if constexpr (SPLIT) {
    // the first FFT ran in scr1; the second FFT's first barrier orders the row
    // twiddles before their use and every access to scr1 before the next
    // tile's load into it
    fence_proxy_async_smem();
    fft_blk_to_s3<TL, -1, TWS, SPLIT>(v, scratch, p, rho, t, tw, issue, scr1);
  } else {
    __syncthreads();  // the first FFT's scratch reads done; row twiddles visible
    fft_blk_to_s3<TL, -1, TWS>(v, scratch, p, rho, t, tw);
  }
  twiddle_store<TL>(v, a, b, g, t, f0, A, rowtw);
}

template <int ELL, int T, int NLC = 0, int MAP = 0>
__global__ void __launch_bounds__(Tile<ELL, T>::THREADS, Tile<ELL, T>::MIN_CTAS)
    k_last_first(const __grid_constant__ PassArgs a, int nbuf) {
  using TL = Tile<ELL, T, NLC>;
  constexpr int E = TL::E;
  extern __shared__ unsigned char smem_raw[];
  __shared__ TileScalars sh;
  unsigned char* smem = aligned_smem(smem_raw);
  const PipeSmem L = pipe_layout(ELL, T, nbuf, true);
  float2* scratch = reinterpret_cast<float2*>(smem + L.scratch);
  float2* tw = reinterpret_cast<float2*>(smem + L.tw);
  float2* rowtw = reinterpret_cast<float2*>(smem + L.rowtw);
  int t, p, rho;
  thread_coords<TL>(t, p, rho);
  load_line_twiddles<ELL>(a, tw);
  __syncthreads();
  pipe_tiles<ELL, TL>(a, nbuf, smem, L, scratch, [&](float2 (&v)[E], int b, int g0, float2* scr1,
                                                     const NextLoad<TL, ELL>& issue) {
    last_first_tile<TL, MAP, 1, TL::LATE>(a, v, b, g0, t, p, rho, scratch, tw, rowtw, sh, scr1, issue);
  });
}

// Every (line length, lines per CTA) pair make_geom produces for m = 4 .. 2^24.
// The radix-3 lines of m = 3 * 2^a: 192, 384 and 768 points (sub-lines of 64,
// 128 and 256; 192 or 384 threads per CTA).
#define SR_TILE_SHAPES(X)                                                                                      \
  X(2, 2) X(2, 4) X(4, 2) X(4, 4) X(4, 8) X(8, 4) X(8, 8) X(8, 16) X(16, 8) X(16, 16) X(16, 32) X(32, 16)    \
  X(32, 32) X(32, 64) X(64, 32) X(64, 64) X(128, 32) X(256, 16) X(512, 8) X(1024, 8) X(2048, 4) X(4096, 2)  \
  X(192, 16) X(384, 16) X(768, 8)

// The (line length, lines per CTA) pairs of square grids m = S * S, S = 2 .. 4096
// (line length S): the shapes with 2D-grid (MAP = 1) kernels.
#define SR_SQUARE_SHAPES(X) \
  X(2, 2) X(4, 4) X(8, 8) X(16, 16) X(32, 32) X(64, 64) X(128, 32) X(256, 16) X(512, 8) X(1024, 8) X(2048, 4) X(4096, 2)

// Kernel entry points by tile shape and transform direction (nullptr when the
// combination is not instantiated). Defined in pass_first.cu / pass_mid.cu /
// pass_last.cu / pass_last_first.cu. map != 0 selects the 2D-grid variants.
const void* pick_first(int ell, int T, int db, int map);
// nl selects a kernel specialised for that line count when one exists.
const void* pick_mid(int ell, int T, int da, int db, int nl);
const void* pick_last(int ell, int T, int da, int nl, int map);
const void* pick_last_first(int ell, int T, int nl, int map);

// Line counts with specialised kernels: (ELL, T, NL) = (256, 16, 256), i.e. m = 2^16.
#define SR_NL_SPECIAL(ell, T, nl) ((ell) == 256 && (T) == 16 && (nl) == 256)

}  // namespace sr
