/*
 * sr.h -- C ABI of the GB300 library for the structured random phase-retrieval
 * model of Hu, Tachella, Unser and Dong, "Structured Random Model for Fast and
 * Robust Phase Retrieval" (arXiv 2409.05734).
 *
 * The sensing operator (Sec. III, Eq. 5, oversampling branch alpha = m/n >= 1) is
 *
 *     A = F D_L ... F D_1 U,      A in C^{m x n},
 *
 * where U zero-pads x in C^n to C^m (x occupies entries 0..n-1), F is the
 * unitary length-m DFT, F[k, j] = m^{-1/2} exp(-2 pi i j k / m), and
 * D_l = diag(exp(i theta_l)) with theta_l[k] ~ U[0, 2 pi) (D_1 acts first).
 * The measurements are y = |A x|^2 (Sec. II-A, Eq. 1).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Complex data is interleaved single precision (re, im) = 8 bytes per
 *   element ("c64"); a batch of B problems is stored problem-major:
 *   x is c64[B][n], z is c64[B][m], y is float[B][m].
 * - All array arguments of the compute calls are DEVICE pointers on the
 *   current CUDA device, owned by the caller, aligned to at least 8 bytes.
 *   Outputs must not overlap inputs unless a call says so.
 * - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls
 *   enqueue their kernels on it and return without synchronising; errors of
 *   the launches themselves are reported through the return value.
 * - The plan owns its device tables (diagonals, twiddles) and a workspace for
 *   up to B_cap problems (2 exchange buffers of B_cap*m c64, a permuted copy
 *   of y, per-block partial sums). A call with B > B_cap grows the workspace
 *   (cudaMalloc) first; call sr_plan_reserve() beforehand to keep later calls
 *   free of allocation. Concurrent calls on one plan must not overlap in time
 *   (they share the workspace); use one plan per stream.
 * - Supported sizes: m = 2^a with 4 <= m <= 2^24, or m = 3 * 2^a with
 *   4 <= 2^a <= 2^22 (oversampling ratios such as 1.5, 3 and 6). For
 *   3 * 2^12 <= m <= 3 * 2^20 the four-step passes take lines of 192, 384 or
 *   768 points with a radix-3 step inside the line FFT; other radix-3 lengths
 *   run one radix-3 step around three power-of-two DFTs on an inner plan that
 *   holds a second workspace of 2 * B_cap * m c64 (B <= 21845 there);
 *   1 <= n <= m, 1 <= L <= 8, 1 <= B <= 65535.
 *   Other sizes return SR_ERR_UNSUPPORTED. sr_forward_noalloc takes
 *   power-of-two m only.
 * - Every call returns SR_OK or an error code; sr_last_error() gives a
 *   thread-local message for the last failing call on the calling thread.
 */
#ifndef SR_H
#define SR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sr_plan sr_plan; /* opaque, owned by the library */

typedef enum sr_status {
  SR_OK = 0,
  SR_ERR_INVALID_ARG = 1,  /* null pointer, B < 1, iters < 0, bad option value */
  SR_ERR_UNSUPPORTED = 2,  /* size outside the supported set */
  SR_ERR_OOM = 3,          /* device or host allocation failed */
  SR_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed */
  SR_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
  SR_ERR_NUMERIC = 6       /* non-finite or invalid numeric input */
} sr_status;

/* Spectral weights T applied to y_hat = m * y / sum(y) (Sec. II-B-2, Eq. 3). */
typedef enum sr_weight_mode {
  SR_WEIGHT_IDENTITY = 0, /* T(y_hat) = y_hat: M = A^H diag(y_hat) A, no shift */
  SR_WEIGHT_OPTIMAL = 1   /* T(y_hat) = max(1 - 1/y_hat, lambda), T = lambda where
                             y_hat <= 0; shift -2*lambda (Eq. 4) */
} sr_weight_mode;

/* Passing NULL for the options selects SR_WEIGHT_OPTIMAL with lambda = -1:
 * Sec. IV runs its spectral methods with the optimal preprocessing function. */
typedef struct sr_spectral_opts {
  int weight_mode; /* sr_weight_mode */
  float lambda;    /* lower threshold, < 0, used by SR_WEIGHT_OPTIMAL */
} sr_spectral_opts;

typedef struct sr_gd_opts {
  float mu0;  /* step scale, > 0 */
  float tau0; /* warm-up length, >= 0 (0: constant step) */
} sr_gd_opts;

/* ---- phases (host only; no GPU needed) ------------------------------------
 * sr_phases: the diffuser phases a plan created with `seed` uses (Sec. III:
 * theta ~ U[0, 2 pi)). theta[l*m + k] = 2*pi*u with u = (w >> 8) * 2^-24 and
 * w the first word of Philox4x32-10 (Salmon et al., SC'11) at counter
 * (k mod 2^32, k div 2^32, l, 1) under key (seed mod 2^32, seed div 2^32).
 * theta: host double[L*m], caller-owned. Needs L >= 1, m >= 1. */
sr_status sr_phases(uint64_t seed, int L, int64_t m, double* theta);

/* ---- plan ------------------------------------------------------------------
 * sr_plan_create: operator A of Sec. III, Eq. 5 for sizes (n, m, L) with the
 * phases of sr_phases(seed, L, m), on the current CUDA device. Builds the
 * device tables (D_l = exp(i theta_l)/sqrt(m) rounded to float, twiddles
 * computed in double and rounded). *out receives the plan; release it with
 * sr_plan_destroy.
 * m < n selects the undersampling branch of Sec. III (the paragraph after
 * Eq. 5): A = S F D_L ... F D_1 with DFTs of length n (n = 2^a in [4, 2^24],
 * else SR_ERR_UNSUPPORTED), phases sr_phases(seed, L, n), and S keeping the m
 * entries off .. off+m-1 of the result, off = floor((n - m) / 2). Every
 * m-length array (z, y, the adjoint's input) holds those m entries. Such plans
 * refuse sr_backward, sr_forward_noalloc and the ragged calls. */
sr_status sr_plan_create(int64_t n, int64_t m, int L, uint64_t seed, sr_plan** out);
sr_status sr_plan_destroy(sr_plan* plan); /* NULL is accepted (no-op) */

/* sr_plan_create_2d: the 2D form of the operator that the experiments of
 * Sec. IV run (a 2D FFT on zero-padded images): A = F2 D_L ... F2 D_1 U2 with
 * x an h x w image (row-major, n = h*w entries, pixel (r, c) at r*w + c), U2
 * placing it in the top-left corner of an S x S grid (zeros elsewhere), F2 the
 * unitary 2D DFT of the grid, F2[(a,b),(r,c)] = exp(-2 pi i (r a + c b)/S) / S,
 * and D_l = diag(exp(i theta_l)) over the grid in row-major order (m = S*S;
 * theta as sr_phases(seed, L, S*S)). z = A x and every m-length array (y, the
 * adjoint's input) are row-major grids. S must be a power of two in
 * [2, 4096] and 1 <= h, w <= S (else SR_ERR_UNSUPPORTED). The plan accepts
 * every call of a 1D plan except sr_plan_set_phases_device, sr_backward,
 * sr_forward_noalloc and the ragged calls (SR_ERR_UNSUPPORTED). */
sr_status sr_plan_create_2d(int64_t h, int64_t w, int64_t S, int L, uint64_t seed, sr_plan** out);

/* Copies the plan's phases (double[L*N], host, N = max(n, m) the DFT length)
 * out / replaces them from host memory (the diagonal tables are rebuilt
 * synchronously). */
sr_status sr_plan_get_phases(const sr_plan* plan, double* theta);
sr_status sr_plan_set_phases(sr_plan* plan, const double* theta);

/* sr_plan_set_batch_phases: gives each of B problems its own operator, with
 * the phases of sr_phases(seeds[b], L, N) for problem b (independent trials of
 * the random model, as in a recovery sweep). The diagonal tables become
 * [B][L][N] (host-built, synchronous); afterwards every call on the plan must
 * use this batch size B (else SR_ERR_INVALID_ARG), and sr_plan_get_phases
 * returns problem 0's phases. seeds: host uint64_t[B]. 2D plans return
 * SR_ERR_UNSUPPORTED. */
sr_status sr_plan_set_batch_phases(sr_plan* plan, int B, const uint64_t* seeds);

/* Replaces the phases from DEVICE memory (float[L*N], e.g. a trainable
 * tensor): the diagonal tables are rebuilt on `stream` (D = exp(i theta)/sqrt(m)
 * in float). The host copy returned by sr_plan_get_phases is refreshed from
 * them on its next call (which then synchronises the device). */
sr_status sr_plan_set_phases_device(sr_plan* plan, const float* theta, void* stream);

/* Reports the plan's sizes (any output pointer may be NULL). */
sr_status sr_plan_info(const sr_plan* plan, int64_t* n, int64_t* m, int* L);

/* Grows the workspace to hold B problems (synchronous cudaMalloc). */
sr_status sr_plan_reserve(sr_plan* plan, int B);

/* Autotunes the plan for batches of B problems: the four-step split of the
 * DFT length (m = m1 m2: the balanced split and its neighbours by a factor of
 * two, with lines of 16 to 4096 points; 1D plans on the four-step passes
 * only) and, for each split, the persistent grid of the middle and last pass
 * kernels (co-resident CTAs per SM from the kernels' occupancy down to 1).
 * Times a few GD steps per candidate on scratch data and keeps the fastest for
 * later calls. Results differ between splits only by rounding. Synchronises
 * the stream; allocates and frees scratch and may rebuild the workspace (not
 * capturable; call before capturing a graph and before handing the plan's
 * buffers to anything else). The paper has no counterpart (launch parameters
 * of this implementation). */
sr_status sr_plan_autotune(sr_plan* plan, int B, void* stream);
/* Sets the four-step split m = m1 * m2 of a 1D plan (for a radix-3 length
 * run on an inner plan, of that plan; one of m1, m2 may be a radix-3 line of
 * 192, 384 or 768 points): layout X holds m2 lines of m1
 * points, layout Y m1 lines of m2 points. SR_ERR_UNSUPPORTED (plan unchanged)
 * when m1 does not divide m or a line length of the split has no pass kernels,
 * and for 2D plans (their split is the S x S grid). Waits for the device and
 * rebuilds the workspace (synchronous cudaMalloc). The paper has no
 * counterpart (it states the DFT, not how it is factored). */
sr_status sr_plan_set_split(sr_plan* plan, int m1);
/* Reports the plan's four-step split and the persistent-grid CTAs per SM that
 * sr_plan_autotune chose (0: the kernels' occupancy). Any output may be NULL. */
sr_status sr_plan_tuning(const sr_plan* plan, int* m1, int* m2, int* ctas_per_sm);

/* ---- operator applications (Sec. III, Eq. 5) --------------------------------
 * sr_forward: z = A x.    x: c64[B][n] (input), z: c64[B][m] (output).
 * sr_adjoint: x = A^H z = U^H D_1^H F^H ... D_L^H F^H z.
 *             z: c64[B][m] (input), x: c64[B][n] (output). */
sr_status sr_forward(sr_plan* plan, const void* x, void* z, int B, void* stream);
sr_status sr_adjoint(sr_plan* plan, const void* z, void* x, int B, void* stream);

/* ---- backward of the operator (phases theta_l are the model's parameters) ----
 * For z = A x (Sec. III, Eq. 5) and the gradient G_z of a real loss with
 * respect to z (convention G_w = dL/dRe w + i dL/dIm w, as in PyTorch):
 *   grad_x     = A^H G_z                                  (c64[B][n], or NULL)
 *   grad_theta = sum over b of Im(conj(p_l) * h_l)         (float[L][m], or NULL)
 * where p_l = D_l q_l is layer l's value right after D_l (q_1 = U x,
 * q_{l+1} = F p_l) and h_l = F^H D_{l+1}^H ... D_L^H F^H G_z is the gradient
 * arriving at p_l (dp_l/dtheta_l = i p_l). The q_l are recomputed from x, not
 * stored: L(L+1)/2 DFT applications in all (3 for L = 2). x: c64[B][n],
 * G_z: c64[B][m]. Uses two extra B*m workspace vectors (grown on first use). */
sr_status sr_backward(sr_plan* plan, const void* x, const void* gz, void* grad_x, float* grad_theta, int B,
                      void* stream);

/* ---- loss and gradient (Sec. II-B-1, Eq. 2) ----------------------------------
 * With z = A x and r = |z|^2 - y:
 *   loss[b] = sum_k r_k^2                   (float[B], device)
 *   grad    = 2 A^H (r * z)                 (c64[B][n], device)
 * Eq. 2 prints diag(x); it is read as diag(A x), which makes grad the
 * Wirtinger derivative dL/d conj(x). x: c64[B][n], y: float[B][m].
 * loss may be NULL. */
sr_status sr_loss_grad(sr_plan* plan, const void* x, const float* y, float* loss,
                       void* grad, int B, void* stream);

/* ---- spectral initialisation (Sec. II-B-2, Eq. 3-4) --------------------------
 * Power iteration on M = A^H diag(T(y_hat)) A with shift s (0 for the identity
 * weight, -2*lambda for the optimal weight): v <- v0/||v0||, then `iters`
 * times u = M v + s v, v = u/||u||; finally x_out = sqrt(sum(y)) * v.
 * y: float[B][m]; v0: c64[B][n] start vectors (random draws are inputs);
 * x_out: c64[B][n]; x_out may equal v0. opts may be NULL (optimal weight, lambda = -1). */
sr_status sr_spectral_init(sr_plan* plan, const float* y, const void* v0, int iters,
                           const sr_spectral_opts* opts, void* x_out, int B, void* stream);

/* sr_spectral_init_early_stop: the same power iteration with early stopping
 * (Sec. IV-A runs it "with early stopping" and states no rule). lambda_t =
 * ||u_t|| estimates the top eigenvalue of M + s I; after every check_every
 * (>= 2) steps it stops once, for every problem, |lambda_{t-1} - lambda_t| <=
 * rel_tol * lambda_{t-1}; at most max_iters steps. *iters_run (host int)
 * receives the number run. Each check synchronises `stream` (a copy of the
 * norm partials to the host), so the call cannot be captured in a graph.
 * rel_tol must be finite and >= 0. */
sr_status sr_spectral_init_early_stop(sr_plan* plan, const float* y, const void* v0, int max_iters,
                                      const sr_spectral_opts* opts, float rel_tol, int check_every,
                                      void* x_out, int* iters_run, int B, void* stream);

/* ---- gradient descent (Sec. II-B-1, Sec. IV-A) ------------------------------
 * `iters` steps x <- x - mu_t * 2 A^H((|Ax|^2 - y) * Ax) with
 *   mu_t = mu0 * (1 - exp(-(t+1)/tau0)) * m / sum(y)   (tau0 > 0), or
 *   mu_t = mu0 * m / sum(y)                             (tau0 == 0),
 * t = 0..iters-1 counted from this call (the paper gives no step size; the
 * warm-up follows the Wirtinger-flow schedule of Candes et al. 2015), updating
 * x (c64[B][n], device) in place. loss_hist (float[iters][B], device)
 * receives the loss at each iterate before its update, or is NULL.
 * opts may be NULL (mu0 = 0.1, tau0 = 0). */
sr_status sr_gd_solve(sr_plan* plan, const float* y, void* x, int iters,
                      const sr_gd_opts* opts, float* loss_hist, int B, void* stream);

/* sr_gd_solve_early_stop: the same iteration with early stopping (Sec. IV-A
 * runs GD "with early stopping" and states no rule). Runs chunks of
 * check_every (>= 2) iterations; after each chunk it reads the losses of the
 * chunk's last two iterations t-1, t and stops once, for every problem,
 * |L(x_{t-1}) - L(x_t)| <= rel_tol * L(x_{t-1}); at most max_iters
 * iterations. *iters_run (host int) receives the number run. loss_hist
 * (float[max_iters][B], device) or NULL as for sr_gd_solve. Each check
 * synchronises `stream` (one 8*B-byte device-to-host copy), so the call cannot
 * be captured in a CUDA graph. B <= 65535. rel_tol must be finite and >= 0. */
sr_status sr_gd_solve_early_stop(sr_plan* plan, const float* y, void* x, int max_iters,
                                 const sr_gd_opts* opts, float rel_tol, int check_every,
                                 float* loss_hist, int* iters_run, int B, void* stream);

/* ---- accuracy metrics (Sec. IV-A, Eq. 6) --------------------------------------
 * For B estimates x_hat[b] and references x[b] (both c64[B][n], device):
 *   cos_out[b]    = |<x_hat, x>| / (||x_hat|| ||x||),  <a, b> = a^H b  (Eq. 6)
 *   relerr_out[b] = min over phi of ||exp(i phi) x_hat - x|| / ||x||
 * (recovery is only possible up to a global phase, Sec. II-A). The minimum is
 * attained at exp(i phi) = <x_hat, x> / |<x_hat, x>| (phi = 0 when the inner
 * product is zero), and the distance is summed directly at that phase. Sums
 * are compensated FP32 in a fixed order (deterministic); each problem is one
 * thread-block cluster of up to 8 CTAs that reduce through distributed shared
 * memory, so the call uses no workspace and never allocates. A zero-norm
 * vector gives NaN (cos) or NaN/inf (relerr), as the definitions do.
 * cos_out, relerr_out: float[B] on the device; either may be NULL.
 * n >= 1, 1 <= B <= 65535. */
sr_status sr_metrics(const void* x_hat, const void* x_ref, int64_t n, int B, float* cos_out, float* relerr_out,
                     void* stream);

/* ---- forward without allocation (the paper has no counterpart) ---------------
 * sr_forward_noalloc: z = A x exactly like sr_forward, for callers that cannot
 * allocate device memory when they make the call -- code running while a CUDA
 * graph is being captured on its stream (cudaMalloc is not allowed there), or
 * hosts whose device memory is owned by their own allocator. It never calls
 * cudaMalloc/cudaFree and never touches the plan's workspace: its two exchange
 * buffers live in a fixed scratch array compiled into the library (2 x
 * SR_FORWARD_NOALLOC_MAX_ELEMENTS complex values, 8 MiB, held by every GPU
 * that loads the library until the process exits). The plan must already
 * exist (sr_plan_create allocates its tables once).
 * - B * m must not exceed SR_FORWARD_NOALLOC_MAX_ELEMENTS; larger calls
 *   return SR_ERR_UNSUPPORTED and launch nothing.
 * - The first call on a device looks up the scratch array's device address
 *   (cudaGetSymbolAddress); make that first call before any stream capture.
 *   The address is cached per device and CUDA context: after cudaDeviceReset
 *   the next call looks it up again (again before any capture).
 * - A plan given per-problem phases (sr_plan_set_batch_phases) accepts only
 *   that batch size; another B returns SR_ERR_INVALID_ARG.
 * - All calls share the one scratch array, which keeps the last call's
 *   contents (every element is rewritten before it is read, so nothing needs
 *   clearing). Calls that overlap on the GPU -- concurrent streams, or several
 *   host threads -- race on it; serialise them.
 * x: c64[B][n], z: c64[B][m], device pointers as for sr_forward. */
#define SR_FORWARD_NOALLOC_MAX_ELEMENTS ((size_t)1 << 19)
sr_status sr_forward_noalloc(const sr_plan* plan, const void* x, void* z, int B, void* stream);

/* ---- dense i.i.d. comparison model (Sec. II-A) -----------------------------
 * The random model the paper compares against: a dense A in C^{m x n} with
 * i.i.d. entries, here supplied by the caller (host float[m][n][2], interleaved
 * re/im) and rounded once to BF16: the rounded matrix IS the model's A. The
 * products run on the tensor cores (tcgen05, BF16 inputs, FP32 accumulation);
 * the vector operand is split into BF16 high and low parts, so a product carries
 * about 2^-16 relative error beyond the FP32 accumulation.
 * Sizes: n a multiple of 64, m a multiple of 128, 64 <= n <= m <= 2^22,
 * B a multiple of 8 in [8, 128]. The model owns two copies of A (A and its
 * transpose, 2 * 4 * m * n bytes) and a workspace for B problems. */
typedef struct sr_dense sr_dense;
/* Operand formats of the dense model (tensor-core input types). */
enum { SR_DENSE_BF16 = 0, SR_DENSE_TF32 = 1 };
/* The BF16 model (sr_dense_create_format with SR_DENSE_BF16). */
sr_status sr_dense_create(int64_t n, int64_t m, const float* a_host, sr_dense** out);
/* The model with its matrix in `format`:
 * - SR_DENSE_BF16: A rounded to BF16 (nearest even); tcgen05 kind::f16; the
 *   vector operand split into BF16 high and low parts (about 2^-16 relative).
 * - SR_DENSE_TF32: A rounded to TF32 (10 fraction bits, to nearest with ties
 *   away from zero, as cvt.rna.tf32.f32); tcgen05 kind::tf32 on FP32-sized
 *   operands (twice the bytes of BF16: 2 * 8 * m * n for A and its transpose);
 *   the vector operand split into TF32 high and low parts (about 2^-21).
 * The rounded matrix is the model's A in both cases. Same sizes and calls as
 * above; SR_ERR_INVALID_ARG for an unknown format. */
sr_status sr_dense_create_format(int64_t n, int64_t m, const float* a_host, int format, sr_dense** out);
sr_status sr_dense_destroy(sr_dense* model); /* NULL accepted */
/* z = A x (x: c64[B][n], z: c64[B][m], device) and x = A^H w (w: c64[B][m]). */
sr_status sr_dense_forward(sr_dense* model, const void* x, void* z, int B, void* stream);
sr_status sr_dense_adjoint(sr_dense* model, const void* w, void* x, int B, void* stream);
/* Gradient descent as sr_gd_solve (same loss, gradient, step rule and loss
 * history), with the dense A. */
sr_status sr_dense_gd_solve(sr_dense* model, const float* y, void* x, int iters, const sr_gd_opts* opts,
                            float* loss_hist, int B, void* stream);
/* Spectral initialisation as sr_spectral_init (same weights T(y_hat), shift,
 * normalisation and output sqrt(sum y) v), with the dense A: per iteration one
 * forward GEMM whose epilogue forms T(y_hat) (A u) / ||u|| and one adjoint GEMM
 * whose epilogue forms u + shift u / ||u|| and the partial sums of ||u||^2
 * (Eq. 3-4). y: f32[B][m], v0 and x_out: c64[B][n] (x_out may equal v0). */
sr_status sr_dense_spectral_init(sr_dense* model, const float* y, const void* v0, int iters,
                                 const sr_spectral_opts* opts, void* x_out, int B, void* stream);
/* As sr_plan_check, for the dense model's kernels. */
sr_status sr_dense_check(sr_dense* model);

/* ---- ragged batches of independent problems -------------------------------
 * A batch of `count` problems with their own sizes n_i, m_i, L_i and phase
 * seeds (the paper's recovery experiments solve many independent problems;
 * Sec. IV). The library buckets problems of equal (n, m, L) into one batched
 * plan whose diagonal tables hold each problem's own phases theta(seed_i).
 * Buckets with power-of-two m from 2^14 to 2^20 form one queue-driven group: a
 * whole GD or power-iteration call on all of the group's problems is ONE
 * persistent launch (plus a few per-problem set-up and finish launches). The
 * other buckets (short transforms, which the resident solver runs whole,
 * radix-3 and longer lengths) run as concurrent branches (one stream each,
 * forked from and joined back into the caller's stream). Every call is one
 * capturable sequence.
 *
 * Data layout: the library chooses where each problem lives in the
 * concatenated buffers: x_cat (c64, problem i at x_off[i], n_i values) and
 * y_cat (f32 for measurements, or c64 for sr_ragged_forward's output; problem
 * i at y_off[i], m_i values), both from sr_ragged_layout; problems of a
 * bucket are adjacent. Sizes as for sr_plan_create; autotune != 0 runs
 * sr_plan_autotune at creation on every bucket outside the queue-driven group
 * (the group runs on its own tile geometry and grid). */
typedef struct sr_ragged sr_ragged;
sr_status sr_ragged_create(int count, const int64_t* n, const int64_t* m, const int* L, const uint64_t* seeds,
                           int autotune, sr_ragged** out);
sr_status sr_ragged_destroy(sr_ragged* r); /* NULL accepted */
/* x_off, y_off: int64[count] (either may be NULL); totals in values. */
sr_status sr_ragged_layout(const sr_ragged* r, int64_t* x_off, int64_t* y_off, int64_t* x_total,
                           int64_t* y_total, int* buckets);
/* z_cat (c64, y layout) = A_i x_i for every problem. */
sr_status sr_ragged_forward(sr_ragged* r, const void* x_cat, void* z_cat, void* stream);
/* Spectral initialisation of every problem (as sr_spectral_init). */
sr_status sr_ragged_spectral_init(sr_ragged* r, const float* y_cat, const void* v0_cat, int iters,
                                  const sr_spectral_opts* opts, void* x_cat, void* stream);
/* GD on every problem in place (as sr_gd_solve). loss_hist: NULL or
 * float[iters][count] (problem i in column i), written at the end of the call;
 * it needs sr_ragged_reserve(r, iters) beforehand (scratch of iters * count
 * floats), which keeps the call free of allocation. */
sr_status sr_ragged_reserve(sr_ragged* r, int iters);
sr_status sr_ragged_gd_solve(sr_ragged* r, const float* y_cat, void* x_cat, int iters, const sr_gd_opts* opts,
                             float* loss_hist, void* stream);
/* As sr_plan_check, over every bucket's plan and the queue-driven solve. */
sr_status sr_ragged_check(sr_ragged* r);
/* Exercises the failure path of the queue-driven solve (the paper has no
 * counterpart): runs one solve step whose tiles after the first pass can never
 * see their inputs complete, so each of their bounded waits gives up after the
 * library's limit (100 ms of GPU time), records SR_ERR_TIMEOUT and returns.
 * Synchronises `stream`; the next sr_ragged_check reports SR_ERR_TIMEOUT (and
 * clears it), and the context stays usable. SR_ERR_UNSUPPORTED when no problem
 * of the batch runs in the queue-driven solve. Allocates scratch inputs. */
sr_status sr_ragged_selftest_timeout(sr_ragged* r, void* stream);

/* ---- device status -----------------------------------------------------------
 * sr_plan_check: waits for the device (cudaDeviceSynchronize) and reports the
 * status the plan's kernels recorded since the last check: SR_ERR_TIMEOUT if
 * a pass kernel's bounded wait for its input tile gave up (the kernel then
 * stops early and its outputs are invalid), SR_OK otherwise. Clears the
 * recorded status. */
sr_status sr_plan_check(sr_plan* plan);

/* Exercises the failure path (the paper has no counterpart): launches one
 * kernel that waits, through the pass kernels' bounded wait, on an mbarrier
 * that nothing completes. The wait gives up after the library's limit (100 ms
 * of GPU time), records SR_ERR_TIMEOUT in the plan's status and returns, so
 * the next sr_plan_check reports SR_ERR_TIMEOUT (and clears it) while the CUDA
 * context stays usable. */
sr_status sr_plan_selftest_timeout(sr_plan* plan, void* stream);

/* ---- profiling ------------------------------------------------------------
 * sr_kernel_launches: number of CUDA kernels this library has launched in the
 * process so far (all plans, all devices).
 * sr_plan_set_timing: when enable != 0, every pass kernel the plan launches
 * afterwards is bracketed by two CUDA events on its stream (a small extra
 * cost per launch); enable == 0 stops recording.
 * sr_plan_get_timing: waits for the recorded events, returns the summed
 * device time (ms) and launch count of each pass class -- index 0 the first
 * pass of a chain, 1 the middle passes, 2 the last pass -- and clears the
 * record. ms and count are host arrays of 3 elements (either may be NULL). */
uint64_t sr_kernel_launches(void);
sr_status sr_plan_set_timing(sr_plan* plan, int enable);
sr_status sr_plan_get_timing(sr_plan* plan, double* ms, int64_t* count);

/* ---- errors --------------------------------------------------------------- */
const char* sr_status_string(sr_status status);
const char* sr_last_error(void); /* thread-local; "" when none */

#ifdef __cplusplus
}
#endif

#endif /* SR_H */
