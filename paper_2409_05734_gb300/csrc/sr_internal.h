// Internal definitions shared by the C-ABI layer and the kernel launchers:
// the plan, the line-space geometry of the four-step decomposition, and the
// argument block of the pass kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sr.h"

namespace sr {

// A length-m DFT is split m = m1 * m2 (m1 >= m2, both powers of two). Each
// DFT runs as two passes over "lines": step 1 transforms lines of one
// decomposition, a global exchange follows, step 2 transforms lines of the
// other. Two line spaces occur (index of element (line g, position q) in the
// natural-order vector is q * NL + g):
//   layout X: NL = m2 lines of length ELL = m1
//   layout Y: NL = m1 lines of length ELL = m2
// Consecutive DFTs alternate their decomposition so that step 2 of one DFT
// and step 1 of the next run on the same lines inside one kernel.
enum Layout { kLayoutX = 0, kLayoutY = 1 };

struct LineGeom {
  int ell;   // line length
  int nl;    // number of lines
  int T;     // lines per CTA
  int P;     // threads per line
  int cpp;   // CTAs per problem = nl / T
  int threads;
  size_t smem;  // dynamic shared memory bytes
};

// Operations fused between the two line FFTs of a pass (or before the first /
// after the last FFT of a chain).
enum PassOp {
  kOpNone = 0,
  kOpDiag = 1,       // v *= Dp[g*ell + f]
  kOpDiagConj = 2,   // v *= conj(Dp[g*ell + f])
  kOpGdEpilogue = 3, // z -> r = |z|^2 - y, w = r z, loss partial sum r^2
  kOpSpecEpilogue = 4 // z -> T(y_hat) z
};

enum OutMode {
  kOutStore = 0,  // out = value
  kOutGrad = 1,   // out = 2 value
  kOutGd = 2,     // x -= mu * 2 value
  kOutSpec = 3    // v = value + shift * v_old / ||v_old||, norm partial
};

struct PassArgs {
  int m;
  int nl, ell, T, cpp;
  int in_dir, out_dir;     // FFT signs of the pass's step-2 and step-1 transforms
  // tables
  const float2* twl;       // W_Lmax^j, j < Lmax
  int tws;                 // Lmax / ell
  const float2* tw_hi;     // W_m^(h << tw_shift)
  const float2* tw_lo;     // W_m^l, l < 2^tw_shift
  int tw_shift;
  // exchange buffers (c64[B][m])
  const float2* ein;
  float2* eout;
  // natural-order vectors (first pass input / last pass output)
  const float2* xin;
  int n_in;
  float2* xout;
  int n_out;
  // fused operation
  int op;
  const float2* dp;        // permuted diagonal, line layout of this pass
  const float* yp;         // permuted y, line layout of this pass, [B][m]
  const float* sumy;       // [B]
  float lam;
  int weight_mode;
  float* part_out;         // per-CTA partial sums [B * cpp]
  // first pass: optional scaling of the input by 1/sqrt(sum of partials)
  const float* norm_in;
  int norm_in_count;
  // last pass
  int out_mode;
  const float* mu;         // [B]
  float shift;
  const float* loss_part;  // partials of the epilogue pass
  int loss_cpp;
  float* loss_out;         // [B] (one row of the history) or nullptr
};

struct Plan {
  int64_t n = 0, m = 0;
  int L = 0;
  uint64_t seed = 0;
  int device = 0;
  int m1 = 0, m2 = 0, lmax = 0;
  int tw_shift = 0;
  std::vector<double> theta;     // host copy, [L][m]
  float2* d_dp = nullptr;        // permuted diagonals, [L][m]
  float2* d_twl = nullptr;       // [lmax]
  float2* d_tw_hi = nullptr;
  float2* d_tw_lo = nullptr;
  // workspace
  int B_cap = 0;
  float2* d_e0 = nullptr;
  float2* d_e1 = nullptr;
  float* d_yp = nullptr;         // [B][m]
  float* d_part = nullptr;       // partial sums, 4 banks of B * kMaxCpp
  float* d_scal = nullptr;       // [4][B]: sum(y), mu, spare
  // optional per-pass event timing (sr_plan_set_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev[3];  // pairs (start, end) per pass class
  size_t ev_used[3] = {0, 0, 0};
};

// Counts every kernel launch of the library (sr_kernel_launches).
void count_launch();
uint64_t launches_so_far();

constexpr int kMaxCpp = 1 << 14;  // max CTAs per problem of any pass (lines per problem)

LineGeom geom_for(const Plan& p, Layout lay);
Layout s1_layout(int parity);
Layout s2_layout(int parity);
Layout diag_layout(int d);

// Pass launchers (fourstep.cu)
cudaError_t launch_first(const Plan& p, Layout lay, const PassArgs& a, int B, cudaStream_t s);
cudaError_t launch_mid(const Plan& p, Layout lay, const PassArgs& a, int B, cudaStream_t s);
cudaError_t launch_last(const Plan& p, Layout lay, const PassArgs& a, int B, cudaStream_t s);
// Helpers (fourstep.cu)
cudaError_t launch_permute_real(const float* y, float* yp, int B, int m, int nl, int ell, cudaStream_t s);
cudaError_t launch_sum_rows(const float* y, int B, int m, float* part, int chunks, cudaStream_t s);
cudaError_t launch_norm_rows(const float2* v, int B, int n, float* part, int chunks, cudaStream_t s);
cudaError_t launch_finish_scalars(const float* part, int chunks, int B, float mu0, int m,
                                  float* sumy, float* mu, cudaStream_t s);
cudaError_t launch_scale_rows(float2* v, int B, int n, const float* part, int chunks,
                              const float* sumy, cudaStream_t s);

}  // namespace sr
