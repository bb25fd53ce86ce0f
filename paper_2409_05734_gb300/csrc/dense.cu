// Dense i.i.d. comparison model (Sec. II-A): z = A x and A^H w for a dense
// complex A in C^{m x n}, as real GEMMs on the fifth-generation tensor cores.
//
// Number formats. A is stored in BF16 (tcgen05 kind::f16) or in TF32
// (kind::tf32, FP32 containers, twice the bytes) and is, by definition, the
// model's matrix: the caller's entries are rounded once when the model is
// created (BF16: to nearest even; TF32: to nearest, ties away from zero), so
// the product involves no further error from A. The vector operand (x, or the
// residual-weighted w) is split into a high and a low part of the same format
// (v = hi + lo to about 2^-17 relative in BF16, 2^-22 in TF32); each A tile
// staged in shared memory is multiplied with both parts, accumulating in FP32
// in tensor memory, so the split costs no extra HBM traffic.
//
// Complex products as one real GEMM with interleaved layouts:
//   forward  Z'[i][c] = sum_k Af[i][k] X'[c][k],  Af[i][2j] = Re A_ij, Af[i][2j+1] = Im A_ij,
//            X'[b][(2j,2j+1)] = (Re x_j, -Im x_j), X'[B+b][(2j,2j+1)] = (Im x_j, Re x_j)
//            -> Z'[i][b] = Re z_i, Z'[i][B+b] = Im z_i;
//   adjoint  G'[r][c] = sum_i Aa[r][i] W'[c][i],  Aa[2j][i] = Re A_ij, Aa[2j+1][i] = Im A_ij,
//            W'[b][i] = Re w_i, W'[B+b][i] = Im w_i
//            -> Re (A^H w)_j = G'[2j][b] + G'[2j+1][B+b], Im = G'[2j][B+b] - G'[2j+1][b].
// Both operands of both GEMMs are K-major (A is stored twice, Af and its
// transpose Aa), so one kernel serves both.
//
// Both operands live in HBM pre-tiled: A as tiles of 128 rows x VPR values
// (VPR = 64 BF16 or 32 TF32 values: one 128-byte row) and the vector operand
// X'/W' as blocks of VPR columns (high part, then low part),
// each stored as the exact 128-byte-swizzled shared-memory image the MMA reads.
// A stage of the main loop is then two contiguous bulk copies (16 KB of A and
// 2 x 2B x 128 bytes of the vector operand), with no tensor maps. The kernels
// that produce X' and W' (the operand preparation and the fused epilogues)
// write the tiled form directly.
//
// Throughput: the main loop is bound by the latency of the stage ring (about
// 2 us from issuing a stage's copies to the MMAs releasing it), with four
// 48 KB stages in flight per SM; the vector operand takes two thirds of each
// stage. Pairing SMs on one 256-row tile (cta_group::2, each SM holding half
// of the vector operand) would raise the matrix bytes in flight per SM.
//
// Kernel: one CTA per 128-row tile of the output, 4 warps. Warp 0 lane 0 issues
// the loads of a multi-stage ring; warp 1 lane 0 issues tcgen05.mma (M = 128,
// N = 2B, K = 16 BF16 or 8 TF32 values per instruction, four per stage, high
// and low parts) into TMEM accumulators and
// frees each stage with tcgen05.commit; then all four warps read their 32 TMEM
// lanes and run the fused epilogue. All waits are bounded by the global timer.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "sr_device.cuh"
#include "sr_internal.h"
#include "sr_tcgen05.cuh"

namespace sr {
namespace {

constexpr int kBM = 128;      // output rows per CTA (TMEM lanes)
constexpr int kThreads = 128;
constexpr int kMaxStages = 6;

// Operand formats: element type, values per 128-byte row (VPR) and per
// 16-byte swizzle chunk (VPC), reduction length of one MMA instruction (KPM).
template <int FMT>
struct Fmt;
template <>
struct Fmt<SR_DENSE_BF16> {
  using El = __nv_bfloat16;
  static constexpr int VPR = 64, VPC = 8, KPM = 16;
  __device__ __forceinline__ static void split(float v, El& hi, El& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
};
template <>
struct Fmt<SR_DENSE_TF32> {
  using El = uint32_t;  // TF32 in an FP32 container (low 13 mantissa bits zero)
  static constexpr int VPR = 32, VPC = 4, KPM = 8;
  __device__ __forceinline__ static uint32_t round(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
  }
  __device__ __forceinline__ static void split(float v, El& hi, El& lo) {
    hi = round(v);
    lo = round(v - __uint_as_float(hi));
  }
};

enum DenseMode {
  kDenseStoreZ = 0,  // forward: z = A x
  kDenseGdFwd = 1,   // forward: r = |z|^2 - y, w = r z as the adjoint's operand, loss partials
  kDenseStoreX = 2,  // adjoint: x = A^H w
  kDenseGdAdj = 3,   // adjoint: x -= mu_t 2 A^H w, next forward operand, loss history
  kDenseSpecFwd = 4, // forward: w = T(y_hat) z / ||u|| as the adjoint's operand (Eq. 3)
  kDenseSpecAdj = 5  // adjoint: u = A^H w + s u / ||u||, norm partials, next forward operand (Eq. 4)
};

struct GemmArgs {
  const void* a_tiles;  // A operand, tiled: [M/128][K/VPR] images of 128 x VPR (16 KB, swizzled)
  const void* b_tiles;  // vector operand, tiled (vtile_index): [K/VPR][high, low][2B][VPR]
  int M, K, B;      // output rows, reduction length, problems (N = 2B)
  int mode;
  int n, m;         // model sizes
  float2* z;                 // kDenseStoreZ: [B][m]
  const float* y;            // kDenseGdFwd: [B][m]
  void* w_out;               // kDenseGdFwd / kDenseSpecFwd: W' [2B][m], tiled
  float* loss_part;          // kDenseGdFwd writes [tiles][B]; kDenseGdAdj reads
  int loss_tiles;
  float* loss_out;           // kDenseGdAdj: [B] or nullptr
  float2* x;                 // kDenseStoreX / kDenseGdAdj: [B][n]
  const float* mu;           // kDenseGdAdj: [B]
  float mu_scale;
  void* xo_out;              // kDenseGdAdj / kDenseSpecAdj: next X' [2B][2n], tiled
  // spectral initialisation
  const float* inv_norm;     // [B]: 1/||u|| of the current iterate
  const float* sumy;         // [B]
  float lam, shift;
  int weight_mode;
  float* norm_part;          // kDenseSpecAdj: [tiles][B] partial sums of |u_new|^2
  int* err;
};

// Contiguous global -> shared copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned) completing on barrier `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Position of element (c, k) of a [2B][K] vector operand (X' or W') in its
// tiled form: per block of VPR columns, the high part's shared-memory image (2B
// rows of 128 bytes, 128-byte swizzle) followed by the low part's; the low
// part of an element sits 2B * VPR values after its high part. One stage of
// the GEMM is then one contiguous copy of 2 * 2B * 128 bytes.
template <int FMT>
__host__ __device__ __forceinline__ size_t vtile_index(int c, int64_t k, int twoB) {
  constexpr int V = Fmt<FMT>::VPR, C = Fmt<FMT>::VPC;
  return (size_t)(k / V) * (size_t)(2 * twoB * V) + (size_t)c * V + (size_t)((((k % V) / C) ^ (c % 8)) * C) +
         (size_t)(k % C);
}

// Splits v into high and low parts and stores both at (c, k) of a tiled operand.
template <int FMT>
__device__ __forceinline__ void store_split(void* t, int twoB, int c, int64_t k, float v) {
  using F = Fmt<FMT>;
  typename F::El h, l;
  F::split(v, h, l);
  typename F::El* te = static_cast<typename F::El*>(t);
  const size_t i = vtile_index<FMT>(c, k, twoB);
  te[i] = h;
  te[i + (size_t)twoB * F::VPR] = l;
}

// Thread-block-cluster helpers (split-K pairs): barrier over both CTAs, the
// address in CTA `rank` of a shared location, and a store there.
__device__ __forceinline__ void pair_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t pair_map(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void pair_store(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void pair_store_i(uint32_t addr, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// split = 1: one CTA per 128-row output tile. split = 2 (launched as clusters
// of two CTAs): the two CTAs of a cluster share a tile and each sums half of
// the K range; after both main loops, rank 1 stores its FP32 sums into rank
// 0's (drained) stage ring through distributed shared memory, and rank 0 adds
// them and runs the epilogue.
template <int FMT>
__global__ void __launch_bounds__(kThreads, 1) k_dense_gemm(const __grid_constant__ GemmArgs a, int stages,
                                                              int split) {
  using F = Fmt<FMT>;
  using El = typename F::El;
  constexpr int kBK = F::VPR;
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail, s_peer_ok;
  __shared__ float red[4][128];
  const int tile = blockIdx.x / split, rank = split == 2 ? (int)(blockIdx.x & 1) : 0;
  const int ntiles = (int)gridDim.x / split;
  const uint32_t base_a = smem_addr(smem_raw);
  const uint32_t base = (base_a + 1023u) & ~1023u;
  const int N = 2 * a.B;
  const uint32_t a_bytes = kBM * 128, b_bytes = (uint32_t)N * 128;
  const uint32_t stage_bytes = a_bytes + 2 * b_bytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = tile * kBM;
  // TMEM columns of one accumulator: N, and every column the epilogue reads
  // (32-column loads at c0 and B + c0 for c0 < B). Successive K-stages rotate
  // over `nacc` accumulators (as many as the 512 columns hold, up to 4) that the
  // epilogue adds in FP32: shorter accumulation chains inside the tensor core.
  const int need = max(N, a.B + ((a.B - 1) / 32) * 32 + 32);
  uint32_t acc_cols = 32;
  while ((int)acc_cols < need) acc_cols <<= 1;
  const int nacc = (int)min(4u, 512u / acc_cols);
  const uint32_t ncols = acc_cols * (uint32_t)nacc;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_addr(&full_bar[s]), 1);
      mbar_init(smem_addr(&empty_bar[s]), 1);
    }
    mbar_init(smem_addr(&done_bar), 1);
    mbar_init_fence();
    s_fail = 0;
  }
  if (warp == 0) tmem_alloc(&tmem_slot, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const int KT = a.K / kBK / split;   // k-tiles of this CTA
  const int kbeg = rank * KT;          // its first k-tile
  // CTAs start their K sweep at staggered offsets so that the vector operand's
  // tiles are not requested by every CTA at the same moment (K order only
  // changes the FP32 summation order, which stays fixed per output row).
  const int kt0 = (int)(((long long)tile * KT) / ntiles);

  // Lanes 1-31 of the producer and MMA warps park at __syncwarp (not in a spin
  // on the done barrier, which would steal the warp's issue slots from lane 0).
  if (warp == 0) {
    if (lane == 0) {
      // producer: TMA loads into the stage ring
      for (int kt = 0; kt < KT; ++kt) {
        const int s = kt % stages, round = kt / stages;
        if (!mbar_wait_bounded(smem_addr(&empty_bar[s]), (uint32_t)((round & 1) ^ 1))) {
          s_fail = 1;
          break;
        }
        const uint32_t st = base + (uint32_t)s * stage_bytes;
        const uint32_t fb = smem_addr(&full_bar[s]);
        mbar_arrive_expect_tx(fb, stage_bytes);
        const int kx = (kbeg + (kt + kt0) % KT) * kBK;
        bulk_load(st, static_cast<const El*>(a.a_tiles) + ((size_t)tile * (a.K / kBK) + (kx / kBK)) * (kBM * kBK),
                  a_bytes, fb);
        bulk_load(st + a_bytes, static_cast<const El*>(a.b_tiles) + (size_t)(kx / kBK) * (2 * N * kBK), 2 * b_bytes,
                  fb);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: 4 K-steps of KPM values (32 bytes of each row) per stage,
      // high and low parts
      const uint32_t idesc = FMT == SR_DENSE_TF32 ? idesc_tf32_f32(kBM, N) : idesc_bf16_f32(kBM, N);
      for (int kt = 0; kt < KT; ++kt) {
        const int s = kt % stages, round = kt / stages;
        if (!mbar_wait_bounded(smem_addr(&full_bar[s]), (uint32_t)(round & 1))) {
          s_fail = 1;
          break;
        }
        tc_fence_after();
        const uint32_t st = base + (uint32_t)s * stage_bytes;
        const uint32_t dacc = tmem + (uint32_t)(kt % nacc) * acc_cols;
#pragma unroll
        for (int kk = 0; kk < kBK / F::KPM; ++kk) {
          const uint64_t da = sw128_desc(st + kk * 32);
          const uint64_t dh = sw128_desc(st + a_bytes + kk * 32), dl = sw128_desc(st + a_bytes + b_bytes + kk * 32);
          if constexpr (FMT == SR_DENSE_TF32) {
            tc_mma_tf32(dacc, da, dh, idesc, (kt >= nacc || kk != 0) ? 1u : 0u);
            tc_mma_tf32(dacc, da, dl, idesc, 1u);
          } else {
            tc_mma_bf16(dacc, da, dh, idesc, (kt >= nacc || kk != 0) ? 1u : 0u);
            tc_mma_bf16(dacc, da, dl, idesc, 1u);
          }
        }
        tc_commit(smem_addr(&empty_bar[s]));
      }
      tc_commit(smem_addr(&done_bar));
    }
    __syncwarp();
  }

  // epilogue: each warp reads its 32 TMEM lanes = 32 output rows
  bool ok = mbar_wait_bounded_sleep(smem_addr(&done_bar), 0, 256);
  tc_fence_after();
  ok = __syncthreads_and(ok) && !s_fail;
  const int row = m0 + warp * 32 + lane;  // output row of this thread
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
  // split-K: partial sums of rank 1 at part[((c0 / 32) * 2 + re/im) * 32 + i][128 rows]
  const float* part = reinterpret_cast<const float*>(smem_raw + (base - base_a));
  if (split == 2) {
    pair_sync();  // both main loops done: rank 0's stage ring is free
    if (rank == 1) {
      if (ok) {
        const uint32_t rbase = pair_map(base, 0);
        const int rl = warp * 32 + lane;
        for (int c0 = 0; c0 < a.B; c0 += 32) {
          float re[32], im[32];
          tmem_ld32(tl + (uint32_t)c0, re);
          tmem_ld32(tl + (uint32_t)(a.B + c0), im);
          for (int q = 1; q < nacc && q < KT; ++q) {
            float r2[32], i2[32];
            tmem_ld32(tl + (uint32_t)q * acc_cols + (uint32_t)c0, r2);
            tmem_ld32(tl + (uint32_t)q * acc_cols + (uint32_t)(a.B + c0), i2);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              re[i] += r2[i];
              im[i] += i2[i];
            }
          }
          const uint32_t cb = rbase + (uint32_t)(((c0 / 32) * 2) * 32 * 128 + rl) * 4u;
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            pair_store(cb + (uint32_t)(i * 128) * 4u, re[i]);
            pair_store(cb + (uint32_t)((32 + i) * 128) * 4u, im[i]);
          }
        }
      }
      if (threadIdx.x == 0) pair_store_i(pair_map(smem_addr(&s_peer_ok), 0), ok ? 1 : 0);
    }
    pair_sync();  // rank 1's partial sums and status are in rank 0's shared memory
    if (rank == 0) ok = ok && s_peer_ok;
  }
  if (ok && rank == 0) {
    for (int c0 = 0; c0 < a.B; c0 += 32) {
      float re[32], im[32];
      tmem_ld32(tl + (uint32_t)c0, re);
      tmem_ld32(tl + (uint32_t)(a.B + c0), im);
      for (int q = 1; q < nacc && q < KT; ++q) {
        float r2[32], i2[32];
        tmem_ld32(tl + (uint32_t)q * acc_cols + (uint32_t)c0, r2);
        tmem_ld32(tl + (uint32_t)q * acc_cols + (uint32_t)(a.B + c0), i2);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          re[i] += r2[i];
          im[i] += i2[i];
        }
      }
      if (split == 2) {
        const float* pc = part + ((c0 / 32) * 2) * 32 * 128 + warp * 32 + lane;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          re[i] += pc[i * 128];
          im[i] += pc[(32 + i) * 128];
        }
      }
      const int nb = min(32, a.B - c0);
      if (a.mode == kDenseStoreZ) {
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (q < nb) a.z[(size_t)(c0 + q) * a.m + row] = make_float2(re[q], im[q]);
      } else if (a.mode == kDenseGdFwd) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          if (q >= nb) continue;
          const int b = c0 + q;
          const float r = fmaf(re[q], re[q], im[q] * im[q]) - a.y[(size_t)b * a.m + row];
          store_split<FMT>(a.w_out, N, b, row, r * re[q]);
          store_split<FMT>(a.w_out, N, a.B + b, row, r * im[q]);
          float s = r * r;
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
          if (lane == 0) red[warp][q] = s;
        }
        __syncthreads();
        if ((int)threadIdx.x < nb)
          a.loss_part[(size_t)tile * a.B + c0 + threadIdx.x] =
              ((red[0][threadIdx.x] + red[1][threadIdx.x]) + red[2][threadIdx.x]) + red[3][threadIdx.x];
        __syncthreads();
      } else if (a.mode == kDenseSpecFwd) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          if (q >= nb) continue;
          const int b = c0 + q;
          const float yh = a.y[(size_t)b * a.m + row] * ((float)a.m / a.sumy[b]);
          float t;
          if (a.weight_mode == SR_WEIGHT_IDENTITY) t = yh;
          else t = yh > 0.f ? fmaxf(1.0f - 1.0f / yh, a.lam) : a.lam;
          t *= a.inv_norm[b];
          store_split<FMT>(a.w_out, N, b, row, t * re[q]);
          store_split<FMT>(a.w_out, N, a.B + b, row, t * im[q]);
        }
      } else {
        // adjoint: rows 2j (Re A^T) and 2j+1 (Im A^T) sit in neighbouring lanes
        const int j = row >> 1;
        const bool even = (row & 1) == 0;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          if (q >= nb) continue;
          const float o_re = __shfl_xor_sync(0xffffffffu, re[q], 1);
          const float o_im = __shfl_xor_sync(0xffffffffu, im[q], 1);
          if (!even) continue;
          const int b = c0 + q;
          const float gr = re[q] + o_im;  // G[2j][b] + G[2j+1][B+b]
          const float gi = im[q] - o_re;  // G[2j][B+b] - G[2j+1][b]
          float2* xp = &a.x[(size_t)b * a.n + j];
          if (a.mode == kDenseStoreX) {
            *xp = make_float2(gr, gi);
          } else {
            float2 xv = *xp;
            if (a.mode == kDenseGdAdj) {
              const float s = 2.0f * a.mu[b] * a.mu_scale;
              xv.x = fmaf(-s, gr, xv.x);
              xv.y = fmaf(-s, gi, xv.y);
            } else {  // kDenseSpecAdj: u = M v + s v with v = u_old / ||u_old||
              const float s = a.shift * a.inv_norm[b];
              xv.x = fmaf(s, xv.x, gr);
              xv.y = fmaf(s, xv.y, gi);
            }
            *xp = xv;
            // next forward operand: X'[b] = (Re x, -Im x), X'[B+b] = (Im x, Re x)
            store_split<FMT>(a.xo_out, N, b, 2 * j, xv.x);
            store_split<FMT>(a.xo_out, N, b, 2 * j + 1, -xv.y);
            store_split<FMT>(a.xo_out, N, a.B + b, 2 * j, xv.y);
            store_split<FMT>(a.xo_out, N, a.B + b, 2 * j + 1, xv.x);
          }
        }
        if (a.mode == kDenseSpecAdj) {
          // partial sums of |u_new|^2 over this tile, per problem (even lanes hold u)
          __syncthreads();
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            if (q >= nb) continue;
            float v2 = 0.f;
            if ((row & 1) == 0) {
              const float2 u = a.x[(size_t)(c0 + q) * a.n + (row >> 1)];
              v2 = fmaf(u.x, u.x, u.y * u.y);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v2 += __shfl_xor_sync(0xffffffffu, v2, off);
            if (lane == 0) red[warp][q] = v2;
          }
          __syncthreads();
          if ((int)threadIdx.x < nb)
            a.norm_part[(size_t)tile * a.B + c0 + threadIdx.x] =
                ((red[0][threadIdx.x] + red[1][threadIdx.x]) + red[2][threadIdx.x]) + red[3][threadIdx.x];
          __syncthreads();
        }
      }
    }
    if (a.mode == kDenseGdAdj && a.loss_out && tile == 0) {
      for (int b = threadIdx.x; b < a.B; b += blockDim.x) {
        fsum2 acc{0.f, 0.f};
        for (int t = 0; t < a.loss_tiles; ++t) acc_add(acc, a.loss_part[(size_t)t * a.B + b]);
        a.loss_out[b] = acc.s + acc.c;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
  if (!ok && threadIdx.x == 0) atomicExch(a.err, (int)SR_ERR_TIMEOUT);
}

// inv[b] = 1 / sqrt(sum of `count` partials of problem b), partials laid out [count][B].
__global__ void k_dense_inv_norm(const float* __restrict__ part, int count, int B, float* __restrict__ inv) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  fsum2 acc{0.f, 0.f};
  for (int t = 0; t < count; ++t) acc_add(acc, part[(size_t)t * B + b]);
  inv[b] = 1.0f / sqrtf(acc.s + acc.c);
}

// X' (tiled, high and low) from x: rows b = (Re x, -Im x), rows B+b = (Im x, Re x).
template <int FMT>
__global__ void k_dense_prep_x(const float2* __restrict__ x, int n, int B, void* __restrict__ xt) {
  const size_t total = (size_t)B * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / n);
    const int64_t j = (int64_t)(i - (size_t)b * n);
    const float2 v = x[i];
    store_split<FMT>(xt, 2 * B, b, 2 * j, v.x);
    store_split<FMT>(xt, 2 * B, b, 2 * j + 1, -v.y);
    store_split<FMT>(xt, 2 * B, B + b, 2 * j, v.y);
    store_split<FMT>(xt, 2 * B, B + b, 2 * j + 1, v.x);
  }
}

// W' (tiled, high and low) from a complex vector w: rows b = Re w, rows B+b = Im w.
template <int FMT>
__global__ void k_dense_prep_w(const float2* __restrict__ w, int m, int B, void* __restrict__ wt) {
  const size_t total = (size_t)B * m;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / m);
    const int64_t k = (int64_t)(i - (size_t)b * m);
    const float2 v = w[i];
    store_split<FMT>(wt, 2 * B, b, k, v.x);
    store_split<FMT>(wt, 2 * B, B + b, k, v.y);
  }
}

}  // namespace
}  // namespace sr

// ---------------------------------------------------------------- host side

namespace {

}  // namespace

struct sr_dense {
  int64_t n = 0, m = 0;
  int fmt = SR_DENSE_BF16;  // operand format (SR_DENSE_BF16 or SR_DENSE_TF32)
  int vpr = 64;             // values per 128-byte tile row: 64 (BF16) or 32 (TF32)
  int eb = 2;               // bytes per operand value
  int device = 0;
  int num_sms = 0;
  void* d_af = nullptr;  // Af [m][2n] as tiles [m/128][2n/vpr][128][vpr] (swizzled images)
  void* d_aa = nullptr;  // Aa [2n][m] as tiles [2n/128][m/vpr][128][vpr]
  int* d_err = nullptr;
  // workspace for B problems
  int B_cap = 0;
  void* d_xt = nullptr;  // X' [2B][2n], tiled high + low (2 * 2B * 2n values)
  void* d_wt = nullptr;  // W' [2B][m], tiled high + low
  float* d_part = nullptr;                          // [m/128][B]
  float* d_npart = nullptr;                         // [max(2n/128, 64)][B]: norm partials
  float* d_scal = nullptr;                          // [3][B]: sum(y), mu, 1/||u||
};

namespace {

sr_status dfail(sr_status st, const std::string& msg) {
  sr::set_last_error(msg);
  return st;
}

#define SR_DCUDA(call, where)                                                                     \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return dfail(SR_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void dense_free_ws(sr_dense* d) {
  cudaFree(d->d_xt);
  cudaFree(d->d_wt);
  cudaFree(d->d_part);
  cudaFree(d->d_npart);
  cudaFree(d->d_scal);
  d->d_xt = d->d_wt = nullptr;
  d->d_part = d->d_npart = d->d_scal = nullptr;
  d->B_cap = 0;
}

sr_status dense_ws(sr_dense* d, int B) {
  if (B <= d->B_cap) return SR_OK;
  dense_free_ws(d);
  const size_t xs = (size_t)2 * B * 2 * d->n, ws = (size_t)2 * B * d->m;
  cudaError_t e;
  if ((e = cudaMalloc(&d->d_xt, 2 * xs * d->eb)) != cudaSuccess || (e = cudaMalloc(&d->d_wt, 2 * ws * d->eb)) != cudaSuccess ||
      (e = cudaMalloc(&d->d_part, sizeof(float) * (size_t)std::max<int64_t>(d->m / 128, 64) * B)) != cudaSuccess ||
      (e = cudaMalloc(&d->d_npart, sizeof(float) * (size_t)std::max<int64_t>(2 * d->n / 128, 64) * B)) !=
          cudaSuccess ||
      (e = cudaMalloc(&d->d_scal, sizeof(float) * 3 * (size_t)B)) != cudaSuccess) {
    cudaGetLastError();
    dense_free_ws(d);
    return dfail(SR_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  d->B_cap = B;
  return SR_OK;
}

size_t gemm_smem(int B, int* stages) {
  const size_t stage = (size_t)sr::kBM * 128 + 2 * (size_t)(2 * B) * 128;
  int s = (int)std::min<size_t>(sr::kMaxStages, (200 * 1024) / stage);
  *stages = std::max(2, s);
  return (size_t)(*stages) * stage + 1024;
}

sr_status check_call(sr_dense* d, int B) {
  if (!d) return dfail(SR_ERR_INVALID_ARG, "model is NULL");
  if (B < 1 || B > 128 || B % 8 != 0) return dfail(SR_ERR_UNSUPPORTED, "dense model: B must be a multiple of 8 in [8, 128]");
  int dev = -1;
  SR_DCUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != d->device) return dfail(SR_ERR_INVALID_ARG, "current CUDA device differs from the model's device");
  return dense_ws(d, B);
}

// One GEMM launch: output rows M (multiple of 128), reduction K (multiple of 64).
sr_status run_gemm(sr_dense* d, sr::GemmArgs& g, const void* a_op, int64_t M, int64_t K, const void* bt, int B,
                   cudaStream_t s) {
  g.a_tiles = a_op;
  g.b_tiles = bt;
  g.M = (int)M;
  g.K = (int)K;
  g.B = B;
  g.n = (int)d->n;
  g.m = (int)d->m;
  g.err = d->d_err;
  int stages = 2;
  const size_t smem = gemm_smem(B, &stages);
  const void* kern = d->fmt == SR_DENSE_TF32 ? (const void*)sr::k_dense_gemm<SR_DENSE_TF32>
                                              : (const void*)sr::k_dense_gemm<SR_DENSE_BF16>;
  SR_DCUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
           "cudaFuncSetAttribute");
  // Split the K range over a pair of CTAs when the tiles alone would leave
  // SMs idle and twice as many CTAs still fit (the adjoint at n << m).
  const int tiles = (int)(M / sr::kBM);
  const int split = (2 * tiles <= d->num_sms && (K / d->vpr) % 2 == 0) ? 2 : 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(tiles * split));
  cfg.blockDim = dim3(sr::kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)split;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = split == 2 ? 1 : 0;
  void* args[] = {(void*)&g, (void*)&stages, (void*)&split};
  SR_DCUDA(cudaLaunchKernelExC(&cfg, kern, args), "launch(dense gemm)");
  sr::count_launch();
  return SR_OK;
}

// Position of element (r, k) of a row-major [rows][K] matrix in its tiled
// form: tiles of 128 rows x vpr columns (one 128-byte row: vpr = 64 BF16 or 32
// TF32 values), ordered (r / 128, k / vpr), each the exact shared-memory image
// the MMA reads -- rows of 128 bytes whose 16-byte chunks are permuted by the
// 128-byte swizzle (chunk c of row r at c ^ (r % 8)).
size_t tiled_index(int64_t r, int64_t k, int64_t K, int vpr) {
  const int vpc = vpr / 8;  // values per 16-byte chunk
  const int64_t tile = (r / sr::kBM) * (K / vpr) + k / vpr;
  const int64_t rr = r % sr::kBM, kk = k % vpr;
  const int64_t chunk = (kk / vpc) ^ (rr % 8);
  return (size_t)(tile * sr::kBM * vpr + rr * vpr + chunk * vpc + kk % vpc);
}

// Rounds to TF32 (10 fraction bits) to nearest, ties away from zero: the
// rounding of cvt.rna.tf32.f32, written out on the host.
uint32_t tf32_rna(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (u & 0x007fffffu) ? 0x7fc00000u : u;  // NaN, +-Inf
  return (u + 0x1000u) & 0xffffe000u;
}

sr_status prep_x(sr_dense* d, const float2* x, int B, cudaStream_t s) {
  const size_t total = (size_t)B * d->n;
  const unsigned grid = (unsigned)std::min<size_t>(4096, (total + 255) / 256);
  if (d->fmt == SR_DENSE_TF32) sr::k_dense_prep_x<SR_DENSE_TF32><<<grid, 256, 0, s>>>(x, (int)d->n, B, d->d_xt);
  else sr::k_dense_prep_x<SR_DENSE_BF16><<<grid, 256, 0, s>>>(x, (int)d->n, B, d->d_xt);
  sr::count_launch();
  SR_DCUDA(cudaGetLastError(), "launch(dense prep x)");
  return SR_OK;
}

// Af and Aa of a row-major complex m x n matrix (interleaved re, im), as
// tiled host images of element type El, with round(.) applied to every entry.
template <class El, class Round>
void tile_matrix(const float* a_host, int64_t n, int64_t m, int vpr, Round round, std::vector<El>& af,
                 std::vector<El>& aa) {
  const size_t cnt = (size_t)m * n * 2;
  af.assign(cnt, El());
  aa.assign(cnt, El());
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      const El re = round(a_host[(i * n + j) * 2]);
      const El im = round(a_host[(i * n + j) * 2 + 1]);
      af[tiled_index(i, 2 * j, 2 * n, vpr)] = re;
      af[tiled_index(i, 2 * j + 1, 2 * n, vpr)] = im;
      aa[tiled_index(2 * j, i, m, vpr)] = re;
      aa[tiled_index(2 * j + 1, i, m, vpr)] = im;
    }
}

}  // namespace

extern "C" {

sr_status sr_dense_create(int64_t n, int64_t m, const float* a_host, sr_dense** out) {
  return sr_dense_create_format(n, m, a_host, SR_DENSE_BF16, out);
}

sr_status sr_dense_create_format(int64_t n, int64_t m, const float* a_host, int format, sr_dense** out) {
  if (!out || !a_host) return dfail(SR_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (format != SR_DENSE_BF16 && format != SR_DENSE_TF32) return dfail(SR_ERR_INVALID_ARG, "unknown dense format");
  if (n < 64 || m < 128 || n % 64 != 0 || m % 128 != 0 || n > (1 << 20) || m > (1 << 22) || n > m)
    return dfail(SR_ERR_UNSUPPORTED, "dense model: n a multiple of 64, m a multiple of 128, 64 <= n <= m");
  sr_dense* d = new (std::nothrow) sr_dense();
  if (!d) return dfail(SR_ERR_OOM, "host allocation failed");
  d->n = n;
  d->m = m;
  d->fmt = format;
  d->vpr = format == SR_DENSE_TF32 ? 32 : 64;
  d->eb = format == SR_DENSE_TF32 ? 4 : 2;
  cudaError_t e = cudaGetDevice(&d->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d->num_sms, cudaDevAttrMultiProcessorCount, d->device);
  const size_t cnt = (size_t)m * n * 2, bytes = cnt * (size_t)d->eb;
  std::vector<__nv_bfloat16> af16, aa16;
  std::vector<uint32_t> af32, aa32;
  if (format == SR_DENSE_TF32) tile_matrix(a_host, n, m, d->vpr, tf32_rna, af32, aa32);
  else tile_matrix(a_host, n, m, d->vpr, [](float v) { return __float2bfloat16_rn(v); }, af16, aa16);
  const void* af = format == SR_DENSE_TF32 ? (const void*)af32.data() : (const void*)af16.data();
  const void* aa = format == SR_DENSE_TF32 ? (const void*)aa32.data() : (const void*)aa16.data();
  if (e == cudaSuccess) e = cudaMalloc(&d->d_af, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&d->d_aa, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&d->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(d->d_af, af, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d->d_aa, aa, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(d->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    sr_dense_destroy(d);
    return dfail(e == cudaErrorMemoryAllocation ? SR_ERR_OOM : SR_ERR_CUDA,
                 std::string("dense model setup: ") + cudaGetErrorString(e));
  }
  *out = d;
  return SR_OK;
}

sr_status sr_dense_destroy(sr_dense* d) {
  if (!d) return SR_OK;
  dense_free_ws(d);
  cudaFree(d->d_af);
  cudaFree(d->d_aa);
  cudaFree(d->d_err);
  delete d;
  return SR_OK;
}

sr_status sr_dense_forward(sr_dense* d, const void* x, void* z, int B, void* stream) {
  sr_status st = check_call(d, B);
  if (st != SR_OK) return st;
  if (!x || !z) return dfail(SR_ERR_INVALID_ARG, "NULL array argument");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = prep_x(d, (const float2*)x, B, s)) != SR_OK) return st;
  sr::GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.mode = sr::kDenseStoreZ;
  g.z = (float2*)z;
  return run_gemm(d, g, d->d_af, d->m, 2 * d->n, d->d_xt, B, s);
}

sr_status sr_dense_adjoint(sr_dense* d, const void* w, void* x, int B, void* stream) {
  sr_status st = check_call(d, B);
  if (st != SR_OK) return st;
  if (!x || !w) return dfail(SR_ERR_INVALID_ARG, "NULL array argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t total = (size_t)B * d->m;
  const unsigned grid = (unsigned)std::min<size_t>(4096, (total + 255) / 256);
  if (d->fmt == SR_DENSE_TF32)
    sr::k_dense_prep_w<SR_DENSE_TF32><<<grid, 256, 0, s>>>((const float2*)w, (int)d->m, B, d->d_wt);
  else
    sr::k_dense_prep_w<SR_DENSE_BF16><<<grid, 256, 0, s>>>((const float2*)w, (int)d->m, B, d->d_wt);
  sr::count_launch();
  SR_DCUDA(cudaGetLastError(), "launch(dense prep w)");
  sr::GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.mode = sr::kDenseStoreX;
  g.x = (float2*)x;
  return run_gemm(d, g, d->d_aa, 2 * d->n, d->m, d->d_wt, B, s);
}

sr_status sr_dense_gd_solve(sr_dense* d, const float* y, void* x, int iters, const sr_gd_opts* opts,
                            float* loss_hist, int B, void* stream) {
  sr_status st = check_call(d, B);
  if (st != SR_OK) return st;
  if (!y || !x) return dfail(SR_ERR_INVALID_ARG, "NULL array argument");
  if (iters < 0) return dfail(SR_ERR_INVALID_ARG, "iters must be >= 0");
  const float mu0 = opts ? opts->mu0 : 0.1f;
  const float tau0 = opts ? opts->tau0 : 0.f;
  if (!(mu0 > 0.f && std::isfinite(mu0)) || !(tau0 >= 0.f && std::isfinite(tau0)))
    return dfail(SR_ERR_INVALID_ARG, "mu0 must be > 0 and tau0 >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  // step mu = mu0 * m / sum(y): the structured model's helpers compute sum(y)
  const int chunks = (int)std::min<int64_t>(64, (d->m + 4095) / 4096);
  SR_DCUDA(sr::launch_sum_rows(y, B, (int)d->m, d->d_part, chunks, s), "launch(sum y)");
  SR_DCUDA(sr::launch_finish_scalars(d->d_part, chunks, B, mu0, (int)d->m, d->d_scal, d->d_scal + B, s),
           "launch(step size)");
  if ((st = prep_x(d, (const float2*)x, B, s)) != SR_OK) return st;
  for (int it = 0; it < iters; ++it) {
    sr::GemmArgs f;
    memset(&f, 0, sizeof(f));
    f.mode = sr::kDenseGdFwd;
    f.y = y;
    f.w_out = d->d_wt;
    f.loss_part = d->d_part;
    if ((st = run_gemm(d, f, d->d_af, d->m, 2 * d->n, d->d_xt, B, s)) != SR_OK) return st;
    sr::GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.mode = sr::kDenseGdAdj;
    g.x = (float2*)x;
    g.mu = d->d_scal + B;
    g.mu_scale = tau0 > 0.f ? (float)(1.0 - std::exp(-(double)(it + 1) / (double)tau0)) : 1.0f;
    g.xo_out = d->d_xt;
    g.loss_part = d->d_part;
    g.loss_tiles = (int)(d->m / sr::kBM);
    g.loss_out = loss_hist ? loss_hist + (size_t)it * B : nullptr;
    if ((st = run_gemm(d, g, d->d_aa, 2 * d->n, d->m, d->d_wt, B, s)) != SR_OK) return st;
  }
  return SR_OK;
}

sr_status sr_dense_spectral_init(sr_dense* d, const float* y, const void* v0, int iters,
                                 const sr_spectral_opts* opts, void* x_out, int B, void* stream) {
  sr_status st = check_call(d, B);
  if (st != SR_OK) return st;
  if (!y || !v0 || !x_out) return dfail(SR_ERR_INVALID_ARG, "NULL array argument");
  if (iters < 0) return dfail(SR_ERR_INVALID_ARG, "iters must be >= 0");
  sr_spectral_opts o{SR_WEIGHT_OPTIMAL, -1.0f};
  if (opts) o = *opts;
  if (o.weight_mode != SR_WEIGHT_IDENTITY && o.weight_mode != SR_WEIGHT_OPTIMAL)
    return dfail(SR_ERR_INVALID_ARG, "unknown weight_mode");
  if (o.weight_mode == SR_WEIGHT_OPTIMAL && !(o.lambda < 0.f && std::isfinite(o.lambda)))
    return dfail(SR_ERR_INVALID_ARG, "lambda must be finite and < 0");
  cudaStream_t s = (cudaStream_t)stream;
  const int n = (int)d->n, m = (int)d->m;
  float2* u = (float2*)x_out;
  if (x_out != v0)
    SR_DCUDA(cudaMemcpyAsync(x_out, v0, (size_t)B * n * sizeof(float2), cudaMemcpyDeviceToDevice, s),
             "cudaMemcpyAsync(v0)");
  const int chunks = (int)std::min<int64_t>(64, (m + 4095) / 4096);
  SR_DCUDA(sr::launch_sum_rows(y, B, m, d->d_part, chunks, s), "launch(sum y)");
  SR_DCUDA(sr::launch_finish_scalars(d->d_part, chunks, B, 0.f, m, d->d_scal, nullptr, s), "launch(sum y)");
  // ||v0||^2 as one partial per problem ([B][1] = [1][B])
  SR_DCUDA(sr::launch_norm_rows(u, B, n, d->d_npart, 1, s), "launch(norm v0)");
  float* inv = d->d_scal + 2 * B;
  sr::k_dense_inv_norm<<<(B + 127) / 128, 128, 0, s>>>(d->d_npart, 1, B, inv);
  sr::count_launch();
  if ((st = prep_x(d, u, B, s)) != SR_OK) return st;
  const int adj_tiles = 2 * n / sr::kBM;
  for (int it = 0; it < iters; ++it) {
    sr::GemmArgs f;
    memset(&f, 0, sizeof(f));
    f.mode = sr::kDenseSpecFwd;
    f.y = y;
    f.sumy = d->d_scal;
    f.inv_norm = inv;
    f.lam = o.lambda;
    f.weight_mode = o.weight_mode;
    f.w_out = d->d_wt;
    if ((st = run_gemm(d, f, d->d_af, m, 2 * n, d->d_xt, B, s)) != SR_OK) return st;
    sr::GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.mode = sr::kDenseSpecAdj;
    g.x = u;
    g.inv_norm = inv;
    g.shift = o.weight_mode == SR_WEIGHT_IDENTITY ? 0.f : -2.0f * o.lambda;
    g.xo_out = d->d_xt;
    g.norm_part = d->d_npart;
    if ((st = run_gemm(d, g, d->d_aa, 2 * n, m, d->d_wt, B, s)) != SR_OK) return st;
    sr::k_dense_inv_norm<<<(B + 127) / 128, 128, 0, s>>>(d->d_npart, adj_tiles, B, inv);
    sr::count_launch();
    SR_DCUDA(cudaGetLastError(), "launch(inverse norm)");
  }
  // x0 = sqrt(sum y) u / ||u||
  SR_DCUDA(sr::launch_norm_rows(u, B, n, d->d_npart, 1, s), "launch(norm u)");
  SR_DCUDA(sr::launch_scale_rows(u, B, n, d->d_npart, 1, d->d_scal, s), "launch(scale)");
  return SR_OK;
}

sr_status sr_dense_check(sr_dense* d) {
  if (!d) return dfail(SR_ERR_INVALID_ARG, "model is NULL");
  SR_DCUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  int code = 0;
  SR_DCUDA(cudaMemcpy(&code, d->d_err, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy(status)");
  if (code != 0) {
    SR_DCUDA(cudaMemset(d->d_err, 0, sizeof(int)), "cudaMemset(status)");
    return dfail((sr_status)code, "a device-side wait of the dense model gave up");
  }
  return SR_OK;
}

}  // extern "C"
