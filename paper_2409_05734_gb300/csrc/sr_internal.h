// Internal definitions shared by the C-ABI layer and the kernel launchers:
// the plan, the line-space geometry of the four-step decomposition, and the
// argument block of the pass kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sr.h"

namespace sr {

// A length-m DFT is split m = m1 * m2 (m1 >= m2, both powers of two). Each
// DFT runs as two steps over "lines": step 1 transforms lines of one
// decomposition, a global exchange follows, step 2 transforms lines of the
// other. Two line spaces occur; element (line g, position q) of either is the
// natural-order index q * NL + g:
//   layout X: NL = m2 lines of length ELL = m1
//   layout Y: NL = m1 lines of length ELL = m2
// Consecutive DFTs alternate their decomposition so that step 2 of one DFT
// and step 1 of the next run on the same lines inside one kernel. The
// exchange buffer between the steps of one DFT holds element (line g, output
// frequency f) of step 1 at f * NL + g, so step 2 reads its lines as
// contiguous rows.
enum Layout { kLayoutX = 0, kLayoutY = 1 };

struct LineGeom {
  int ell;      // line length
  int nl;       // number of lines
  int T;        // lines per CTA (power of two)
  int lgT;
  int P;        // threads per line
  int cpp;      // CTAs (tiles) per problem = nl / T
  int threads;  // T * P
  int nbuf;     // input stages of the persistent passes (1 or 2)
  size_t smem_first, smem_pipe;  // dynamic shared memory of the first / middle+last passes
};

// Operations fused between the two line FFTs of a pass (or before the first /
// after the last FFT of a chain). Tables are in natural order.
enum PassOp {
  kOpNone = 0,
  kOpDiag = 1,        // v *= D[q*NL + g]
  kOpDiagConj = 2,    // v *= conj(D[q*NL + g])
  kOpGdEpilogue = 3,  // z -> r = |z|^2 - y, w = r z, loss partial sum r^2
  kOpSpecEpilogue = 4 // z -> T(y_hat) z
};

enum OutMode {
  kOutStore = 0,  // out = value
  kOutGrad = 1,   // out = 2 value
  kOutGd = 2,     // x -= mu * mu_scale * 2 value
  kOutSpec = 3    // v = value + shift * v_old / ||v_old||, norm partial
};

struct PassArgs {
  CUtensorMap tmap;        // rows of the input exchange buffer (middle/last passes, ELL >= 16)
  int m;
  int nl, ell, T, lgT, cpp, ntiles;
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
  const float2* dp;        // diagonal D_l (natural order, 1/sqrt(m) folded in)
  int64_t dp_stride;       // complex values between problems' tables (0: one table for the batch)
  // middle passes: the phases theta_l of the same diagonal (float, in
  // [-pi, pi), indexed like dp), from which the pass forms exp(i theta) itself
  // (nullptr: use dp); the 1/sqrt(m) of D_l is then applied as `dscale` with
  // the pass's four-step twiddles
  const float* ph;
  float dscale;
  const float* y;          // measurements [B][m], natural order
  const float* sumy;       // [B]
  float lam;
  int weight_mode;
  float* part_out;         // per-tile partial sums [B * cpp]
  // first pass of a radix-3 chain: inner problem 3 bo + r reads element
  // 3 nat + r of outer problem bo; y and D are the outer plan's (length ym)
  int r3;
  int ym;
  // 2D grids (MAP = 1 kernels): signal shapes and transposition of the first
  // pass's input and the last pass's output (see grid_index)
  int in_h, in_w, in_tr;
  int out_h, out_w, out_tr;
  // alpha < 1: first pass input / last pass output is the window of the
  // length-m vector starting at this offset (0 otherwise)
  int in_off, out_off;
  // first pass: optional scaling of the input by 1/sqrt(sum of partials)
  const float* norm_in;
  int norm_in_count;
  // last pass
  int out_mode;
  const float* mu;         // [B]
  float mu_scale;          // step warm-up factor of this iteration
  float shift;
  const float* loss_part;  // partials of the epilogue pass
  int loss_cpp;
  float* loss_out;         // [B] (one row of the history) or nullptr
  int* err;                // device status word (SR_ERR_TIMEOUT on a failed wait)
};

// Radix-3 chain step (radix3.cu): the stride-3 de-interleave and the operation
// before each DFT happen in the inner plan's first pass (PassArgs::r3); combine
// = twiddles and radix-3 butterfly back to natural order, with the chain's
// output mode.
struct R3CombineArgs {
  const float2* U;         // [3B][mp]
  int64_t mp;
  int chunks;
  const float2* tw3;       // W_m^j (forward sign), j < 2 mp
  int op;                  // kOpNone or kOpDiagConj (D_1^H)
  const float2* dp;
  int64_t dp_stride;
  float2* xout;            // [B][n_out], natural order
  int64_t n_out;
  int out_mode;            // OutMode
  const float* mu;
  float mu_scale, shift;
  const float* norm_in;
  int norm_in_count;
  float* part_out;         // kOutSpec: norm partials [B][chunks]
  const float* loss_part;  // loss history: partials [B][loss_cpp]
  int loss_cpp;
  float* loss_out;
};

cudaError_t launch_r3_combine(const R3CombineArgs& a, int dir, int B, cudaStream_t s);

struct Plan {
  int64_t n = 0, m = 0;
  int L = 0;
  uint64_t seed = 0;
  int device = 0;
  int num_sms = 0;
  int m1 = 0, m2 = 0, lmax = 0;
  int tw_shift = 0;
  std::vector<double> theta;     // host copy, [L][m]
  float2* d_dp = nullptr;        // diagonals, [L][m] natural order (per problem: [B][L][m])
  float* d_ph = nullptr;         // their phases as float in [-pi, pi), same layout
  int64_t dp_stride = 0;         // L * m when every problem of the batch has its own phases
  int batch_fixed = 0;           // with per-problem phases: the only valid batch size
  int tuned_per_sm = 0;          // persistent-grid CTAs per SM chosen by sr_plan_autotune (0: occupancy)
  // 2D model on h x w images in an S x S grid (m = S * S, n = h * w): unit
  // four-step twiddles, diagonals of even layers stored transposed, and for
  // odd L a transposed copy of y (d_yt, [B][m]) for the epilogues
  // alpha < 1 (m < n): the DFTs have length m = n here and the operator keeps
  // the mo entries off .. off+mo-1 of the result (mo = m otherwise); the
  // solver steps run a forward chain into d_zw ([B][mo]) and an adjoint chain
  // whose first pass applies the epilogue
  int64_t mo = 0;
  int64_t off = 0;
  float2* d_zw = nullptr;
  float* d_es = nullptr;  // early stopping: the last two losses of a chunk, [2][B]
  bool two_d = false;
  int gh = 0, gw = 0, gS = 0;
  float* d_yt = nullptr;
  float2* d_twl = nullptr;       // [lmax]
  float2* d_tw_hi = nullptr;
  float2* d_tw_lo = nullptr;
  int* d_err = nullptr;          // device status word
  LineGeom geom[2];              // per layout
  int per_sm_mid[2][3] = {{1, 1, 1}, {1, 1, 1}};  // co-resident CTAs per SM: [layout][direction pair]
  int per_sm_last[2][2] = {{1, 1}, {1, 1}};       // [layout][inverse]
  int per_sm_lf[2] = {1, 1};                      // fused LAST + FIRST, [layout]
  int per_sm_first[2] = {1, 1};                   // FIRST (persistent over its tiles), [layout]
  // workspace
  int B_cap = 0;
  float2* d_e0 = nullptr;
  float2* d_e1 = nullptr;
  float* d_part = nullptr;       // partial sums, 4 banks
  float* d_scal = nullptr;       // [4][B]: sum(y), mu, spare
  // backward pass: two natural-order vectors per problem (grown on first use)
  int W_cap = 0;
  float2* d_w0 = nullptr;
  float2* d_w1 = nullptr;
  // phases set from the device (sr_plan_set_phases_device): float copy; the
  // host copy `theta` is refreshed from it on demand
  float* d_theta_f = nullptr;
  bool host_theta_stale = false;
  CUtensorMap tmap[2][2];  // [buffer e0/e1][layout]: rows of the exchange buffer
  // m = 3 mp: DFTs of length mp over 3B sequences run on `inner` (a power-of-two
  // plan, n = m = mp; its first pass gathers the stride-3 subsequences), then
  // the radix-3 combine
  Plan* inner = nullptr;
  int64_t mp = 0;
  int r3_chunks = 0;             // blocks per problem of the combine kernel
  float2* d_tw3 = nullptr;       // W_m^j, j < 2 mp
  // optional per-pass event timing (sr_plan_set_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev[3];  // pairs (start, end) per pass class
  size_t ev_used[3] = {0, 0, 0};
};

// Encodes `rows` rows of `ell` complex values starting at `base` (an exchange
// buffer) as a 2D tensor for the TMA loads of the passes that read it: boxes of
// 16 complex values (128 bytes) x T rows, 128-byte swizzle. cudaErrorNotSupported
// when the driver has no tensor-map encoder, cudaErrorInvalidValue when the
// encoder rejects the description (api.cu).
cudaError_t encode_rows(CUtensorMap* map, float2* base, int ell, int64_t rows, int T);

// Sets the thread-local message sr_last_error() returns.
void set_last_error(const std::string& msg);

// Counts every kernel launch of the library (sr_kernel_launches).
void count_launch();
uint64_t launches_so_far();

LineGeom make_geom(int64_t m, int ell);
Layout s1_layout(int parity);
Layout s2_layout(int parity);

// Pass launchers (fourstep.cu). B problems; the middle and last passes run a
// persistent grid of min(tiles, per_sm * SMs) CTAs.
cudaError_t launch_first(const Plan& p, Layout lay, const PassArgs& a, int B, cudaStream_t s);
// Loss partials a middle pass writes per tile: one per warp when the CTA is
// whole warps, else one.
inline int epilogue_partials_per_tile(const LineGeom& g) { return g.threads % 32 == 0 ? g.threads / 32 : 1; }

// Whole solves for short transforms (small.cu): power-of-two m <= kSmallMaxM
// (the DFT length; both alpha branches), 1D plans. One CTA line per problem;
// all iterations in one launch.
constexpr int kSmallMaxM = 8192;
struct SmallArgs {
  int m, n, L, B;
  int mo, off;             // measurements: entries off .. off+mo-1 of the length-m result (alpha < 1), else m, 0
  const float2* dp;        // diagonals, D_l at dp + b * dp_stride + l * m
  int64_t dp_stride;
  const float2* tw_hi;     // the plan's two-level W_m table
  const float2* tw_lo;
  int tw_shift;
  const float* y;          // [B][mo]
  const float* sumy;       // [B]
  float2* x;               // [B][n], updated in place (GD, power iteration)
  int count;               // steps in this launch
  // GD
  const float* mu;         // [B]: mu0 m / sum(y)
  int t0;                  // global index of the first step (warm-up factor)
  float tau0;
  float* loss_hist;        // rows of steps >= loss_first, [B] each, or nullptr
  int loss_first;
  int grad;                // one gradient evaluation: g = 2 A^H(r z), loss_out
  float2* g;
  float* loss_out;
  // the operator alone: z = A x (op = 1, zout [B][mo]) or x = A^H w (op = 2,
  // win [B][mo] in, x [B][n] out); op = 0 for the solver modes
  int op;
  const float2* win;
  float2* zout;
  // power iteration
  int weight_mode;
  float lam, shift;
  const float* norm_in;    // partials of ||x||^2 of the incoming iterate
  int norm_in_count;
  float* norm_last;        // [B]: ||u||^2 of the last step
  float* norm_prev;        // [B]: of the step before (count >= 2)
};
bool small_eligible(const Plan& p);
cudaError_t launch_small(const Plan& p, const SmallArgs& a, bool spec, cudaStream_t s);
// yt[b] = y[b]^T for B row-major S x S float grids (2D plans with odd L)
cudaError_t launch_transpose_grids(const float* y, float* yt, int S, int B, cudaStream_t s);
cudaError_t launch_mid(const Plan& p, Layout lay, const PassArgs& a, int B, cudaStream_t s);
cudaError_t launch_last(const Plan& p, Layout lay, const PassArgs& a, int B, cudaStream_t s);
// LAST of a GD step fused with FIRST of the next (same layout X lines).
cudaError_t launch_last_first(const Plan& p, Layout lay, const PassArgs& a, int B, cudaStream_t s);
// Max co-resident CTAs per SM of the middle pass kernels (3 direction pairs)
// and of the last pass kernels (2 directions) of a geometry.
cudaError_t pass_occupancy(const LineGeom& g, int* per_sm_mid, int* per_sm_last, int* per_sm_lf, int* per_sm_first);
// Helpers (fourstep.cu)
cudaError_t launch_sum_rows(const float* y, int B, int m, float* part, int chunks, cudaStream_t s);
cudaError_t launch_norm_rows(const float2* v, int B, int n, float* part, int chunks, cudaStream_t s);
cudaError_t launch_finish_scalars(const float* part, int chunks, int B, float mu0, int m,
                                  float* sumy, float* mu, cudaStream_t s);
cudaError_t launch_scale_rows(float2* v, int B, int n, const float* part, int chunks,
                              const float* sumy, cudaStream_t s);
// d = exp(i theta) * scale and ph = theta wrapped to [-pi, pi), count entries.
cudaError_t launch_set_diag(const float* theta, float2* d, float* ph, size_t count, float scale, cudaStream_t s);
cudaError_t launch_theta_grad(const float2* q, int nq, const float2* d, const float2* h, int m, int B, float* out,
                              cudaStream_t s);
cudaError_t launch_conj_diag_prune(const float2* h, const float2* d, int m, int n, int B, float2* out,
                                   cudaStream_t s);

// Kernel whose bounded wait never completes and records SR_ERR_TIMEOUT in *err.
cudaError_t launch_wait_probe(int* err, cudaStream_t s);

// Bank `bank` of the plan's per-problem partial sums for batches of B problems
// (0, 1: power-iteration norms, 2: loss, 3: sums) (api.cu).
float* plan_part_bank(const Plan& p, int bank, int B);

// Per-problem phases for a batch of B problems of one shape (api.cu).
sr_status plan_set_problem_phases(sr_plan* plan, int B, const uint64_t* seeds);

}  // namespace sr
