// C ABI of the structured random phase-retrieval library (include/sr.h):
// argument validation, plan construction (host Philox phases, diagonal and
// twiddle tables computed in double and rounded to float), workspace, and the
// orchestration of the pass kernels into the operator applications and solver
// loops of the paper (Sec. II-B, Sec. III).
#include <algorithm>
#include <numeric>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sr_internal.h"

using sr::Plan;

namespace {

thread_local std::string g_last_error;

sr_status fail(sr_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

sr_status cuda_fail(cudaError_t e, const char* where) {
  return fail(SR_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define SR_CUDA(call, where)                       \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

constexpr double kTwoPi = 6.283185307179586476925286766559;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplications with the published round constants and Weyl key increments.
void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

constexpr uint32_t kStreamTheta = 1;

void gen_phases(uint64_t seed, int L, int64_t m, double* theta) {
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
  for (int l = 0; l < L; ++l) {
    for (int64_t k = 0; k < m; ++k) {
      uint32_t c[4] = {(uint32_t)((uint64_t)k & 0xFFFFFFFFu), (uint32_t)((uint64_t)k >> 32), (uint32_t)l,
                       kStreamTheta};
      philox4x32_10(c, k0, k1);
      const double u = (double)(c[0] >> 8) * 0x1p-24;
      theta[(size_t)l * m + k] = 2.0 * M_PI * u;
    }
  }
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int64_t v) {
  int r = 0;
  while ((int64_t(1) << r) < v) ++r;
  return r;
}

// m = 3 * 2^k with 2^k >= 4 (the radix-3 lengths)
bool is_three_pow2(int64_t m) { return m % 3 == 0 && is_pow2(m / 3) && m / 3 >= 4; }

sr_status check_sizes(int64_t n, int64_t m, int L) {
  if (L < 1 || L > 8) return fail(SR_ERR_UNSUPPORTED, "L must be in [1, 8]");
  const bool ok = (is_pow2(m) && m >= 4 && m <= (int64_t(1) << 24)) ||
                  (is_three_pow2(m) && m / 3 <= (int64_t(1) << 22));
  if (!ok) return fail(SR_ERR_UNSUPPORTED, "m must be 2^a in [4, 2^24] or 3 * 2^a with 2^a in [4, 2^22]");
  if (n < 1 || n > m) return fail(SR_ERR_UNSUPPORTED, "n must satisfy 1 <= n <= m");
  return SR_OK;
}

sr_status check_device(const Plan* p) {
  int dev = -1;
  SR_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != p->device) return fail(SR_ERR_INVALID_ARG, "current CUDA device differs from the plan's device");
  return SR_OK;
}

template <typename T>
sr_status dalloc(T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) return SR_OK;
  cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(SR_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return SR_OK;
}

void free_workspace(Plan* p) {
  cudaFree(p->d_e0);
  cudaFree(p->d_e1);
  cudaFree(p->d_part);
  cudaFree(p->d_scal);
  cudaFree(p->d_yt);
  cudaFree(p->d_zw);
  p->d_zw = nullptr;
  p->d_e0 = p->d_e1 = nullptr;
  p->d_part = p->d_scal = nullptr;
  p->d_yt = nullptr;
  p->B_cap = 0;
}

// Size of one bank of per-tile partial sums per problem.
int part_stride(const Plan& p) {
  int s = std::max(std::max(std::max(p.geom[0].cpp, p.geom[1].cpp), p.r3_chunks), 64);
  for (int lay = 0; lay < 2; ++lay)  // the GD epilogue's per-warp loss partials
    s = std::max(s, p.geom[lay].cpp * sr::epilogue_partials_per_tile(p.geom[lay]));
  // radix-3: the inner first pass writes 3 banks of its tile partials per problem
  if (p.inner) s = std::max(s, 3 * std::max(p.inner->geom[0].cpp, p.inner->geom[1].cpp));
  return s;
}

// sr::encode_rows (defined below the anonymous namespace) with its failures
// reported through sr_last_error.
sr_status encode_exchange_rows(CUtensorMap* map, float2* base, int ell, int64_t rows, int T) {
  const cudaError_t e = sr::encode_rows(map, base, ell, rows, T);
  if (e == cudaErrorNotSupported) return fail(SR_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if (e != cudaSuccess) return fail(SR_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return SR_OK;
}
constexpr int kPartBanks = 4;  // 0,1: power-iteration norms (ping-pong), 2: loss, 3: sums

sr_status ensure_workspace(Plan* p, int B) {
  if (B <= p->B_cap) return SR_OK;
  free_workspace(p);
  const size_t bm = (size_t)B * (size_t)p->m;
  sr_status st;
  if ((st = dalloc(&p->d_e0, bm)) != SR_OK || (st = dalloc(&p->d_e1, bm)) != SR_OK ||
      (st = dalloc(&p->d_part, (size_t)kPartBanks * B * part_stride(*p))) != SR_OK ||
      (st = dalloc(&p->d_scal, (size_t)4 * B)) != SR_OK ||
      (p->two_d && p->L % 2 == 1 && (st = dalloc(&p->d_yt, bm)) != SR_OK) ||
      (p->mo < p->m && (st = dalloc(&p->d_zw, (size_t)B * (size_t)p->mo)) != SR_OK)) {
    free_workspace(p);
    return st;
  }
  for (int lay = 0; lay < 2; ++lay) {
    const sr::LineGeom& g = p->geom[lay];
    if (g.ell < 16) continue;  // short lines are read without TMA
    for (int buf = 0; buf < 2; ++buf) {
      st = encode_exchange_rows(&p->tmap[buf][lay], buf ? p->d_e1 : p->d_e0, g.ell, (int64_t)B * g.nl, g.T);
      if (st != SR_OK) {
        free_workspace(p);
        return st;
      }
    }
  }
  p->B_cap = B;
  return SR_OK;
}

sr_status ensure_backward_buffers(Plan* p, int B) {
  if (B <= p->W_cap) return SR_OK;
  cudaFree(p->d_w0);
  cudaFree(p->d_w1);
  p->d_w0 = p->d_w1 = nullptr;
  p->W_cap = 0;
  const size_t bm = (size_t)B * (size_t)p->m;
  sr_status st;
  if ((st = dalloc(&p->d_w0, bm)) != SR_OK || (st = dalloc(&p->d_w1, bm)) != SR_OK) {
    cudaFree(p->d_w0);
    p->d_w0 = nullptr;
    return st;
  }
  p->W_cap = B;
  return SR_OK;
}

float* part_bank(const Plan& p, int bank, int B) { return p.d_part + (size_t)bank * B * part_stride(p); }
}  // namespace

namespace sr {
float* plan_part_bank(const Plan& p, int bank, int B) { return part_bank(p, bank, B); }
}  // namespace sr

namespace {

// theta wrapped to [-pi, pi).
double wrap_phase(double t) {
  double w = std::remainder(t, kTwoPi);
  if (w >= 0.5 * kTwoPi) w -= kTwoPi;
  return w;
}

// Rebuilds the device diagonal tables from p->theta: D_l = exp(i theta_l)/sqrt(m)
// (the 1/sqrt(m) of each unitary F folded in), natural order, computed in
// double and rounded to float.
sr_status upload_diagonals(Plan* p) {
  const int64_t m = p->m;
  const double scale = 1.0 / std::sqrt((double)m);
  std::vector<float2> host((size_t)p->L * m);
  std::vector<float> ph((size_t)p->L * m);
  for (size_t i = 0; i < host.size(); ++i) {
    // 2D grids: layers 2, 4, ... act on the transposed grid (see grid_index),
    // so their tables are stored transposed: entry (r, c) holds D(c, r)
    size_t src = i;
    const int64_t l = (int64_t)(i / m), k = (int64_t)(i % m);
    if (p->two_d && l % 2 == 1) src = (size_t)(l * m + (k % p->gS) * p->gS + k / p->gS);
    const double t = p->theta[src];
    host[i] = make_float2((float)(std::cos(t) * scale), (float)(std::sin(t) * scale));
    ph[i] = (float)wrap_phase(t);
  }
  SR_CUDA(cudaMemcpy(p->d_dp, host.data(), host.size() * sizeof(float2), cudaMemcpyHostToDevice),
          "cudaMemcpy(diagonals)");
  SR_CUDA(cudaMemcpy(p->d_ph, ph.data(), ph.size() * sizeof(float), cudaMemcpyHostToDevice), "cudaMemcpy(phases)");
  return SR_OK;
}

float2 root_of_unity(int64_t j, int64_t N) {
  // exp(-2 pi i j / N) in double, rounded to float
  const double a = -kTwoPi * (double)j / (double)N;
  return make_float2((float)std::cos(a), (float)std::sin(a));
}

// Line twiddles W_lmax^j, j < lmax (lmax: the longer line of the split).
sr_status upload_line_twiddles(Plan* p) {
  std::vector<float2> twl(p->lmax);
  for (int j = 0; j < p->lmax; ++j) twl[j] = root_of_unity(j, p->lmax);
  cudaFree(p->d_twl);
  p->d_twl = nullptr;
  sr_status st;
  if ((st = dalloc(&p->d_twl, twl.size())) != SR_OK) return st;
  SR_CUDA(cudaMemcpy(p->d_twl, twl.data(), twl.size() * sizeof(float2), cudaMemcpyHostToDevice), "cudaMemcpy");
  return SR_OK;
}

// The two-level W_m tables (the split-independent four-step twiddles).
sr_status upload_twiddles(Plan* p) {
  const int64_t nlo = int64_t(1) << p->tw_shift, nhi = (p->m + nlo - 1) / nlo;
  std::vector<float2> lo(nlo), hi(nhi);
  for (int64_t j = 0; j < nlo; ++j) lo[j] = root_of_unity(j, p->m);
  for (int64_t j = 0; j < nhi; ++j) hi[j] = root_of_unity(j * nlo, p->m);
  if (p->two_d) {
    // the 2D DFT of an S x S grid is the four-step DFT without its twiddles
    std::fill(lo.begin(), lo.end(), make_float2(1.f, 0.f));
    std::fill(hi.begin(), hi.end(), make_float2(1.f, 0.f));
  }
  sr_status st;
  if ((st = dalloc(&p->d_tw_lo, lo.size())) != SR_OK || (st = dalloc(&p->d_tw_hi, hi.size())) != SR_OK) return st;
  SR_CUDA(cudaMemcpy(p->d_tw_lo, lo.data(), lo.size() * sizeof(float2), cudaMemcpyHostToDevice), "cudaMemcpy");
  SR_CUDA(cudaMemcpy(p->d_tw_hi, hi.data(), hi.size() * sizeof(float2), cudaMemcpyHostToDevice), "cudaMemcpy");
  return SR_OK;
}

// Four-step split m = m1 m2 (layout X: m2 lines of m1 points; layout Y: m1
// lines of m2 points): geometry, pass occupancy and the line-twiddle table.
// SR_ERR_UNSUPPORTED (plan unchanged) when a line length of the split has no
// pass kernels. The workspace (its tensor maps and partial-sum banks depend on
// the split) is released; the next call rebuilds it.
sr_status set_split(Plan* p, int m1) {
  if (m1 < 2 || p->m % m1 != 0 || p->m / m1 < 2) return fail(SR_ERR_UNSUPPORTED, "invalid four-step split");
  const int m2 = (int)(p->m / m1);
  sr::LineGeom g[2] = {sr::make_geom(p->m, m1), sr::make_geom(p->m, m2)};
  int mid[2][3], last[2][2], lf[2], first[2];
  for (int lay = 0; lay < 2; ++lay) {
    const cudaError_t e = sr::pass_occupancy(g[lay], mid[lay], last[lay], &lf[lay], &first[lay]);
    if (e == cudaErrorInvalidValue) {
      cudaGetLastError();
      return fail(SR_ERR_UNSUPPORTED, "no pass kernels for this four-step split");
    }
    if (e != cudaSuccess) return cuda_fail(e, "plan geometry");
  }
  p->m1 = m1;
  p->m2 = m2;
  // one line-twiddle table W_lmax serves both line lengths: lmax = lcm(m1, m2)
  // (the longer line for powers of two, 3 x the longer power for radix-3 lines)
  p->lmax = (int)std::lcm((int64_t)m1, (int64_t)m2);
  for (int lay = 0; lay < 2; ++lay) {
    p->geom[lay] = g[lay];
    std::memcpy(p->per_sm_mid[lay], mid[lay], sizeof(mid[lay]));
    std::memcpy(p->per_sm_last[lay], last[lay], sizeof(last[lay]));
    p->per_sm_lf[lay] = lf[lay];
    p->per_sm_first[lay] = first[lay];
  }
  p->tuned_per_sm = 0;
  free_workspace(p);
  return upload_line_twiddles(p);
}

// ------------------------------------------------------------ chains of DFTs

struct MidOp {
  int op = sr::kOpNone;
  int d = 0;  // diagonal index for the diagonal operations
};

struct Chain {
  int nfft = 0;
  int s0 = 0;                 // decomposition parity of DFT 0
  int dir[16] = {0};
  int first_op = sr::kOpNone; // kOpNone, kOpDiag or kOpDiagConj
  int first_d = 0;            // index of the diagonal the first pass applies
  MidOp mid[16];              // mid[k], k = 1..nfft-1
  int last_op = sr::kOpNone;  // kOpNone or kOpDiagConj (D_1^H)
  // input of the first pass
  const float2* xin = nullptr;
  int n_in = 0;
  const float* norm_in = nullptr;
  int norm_in_count = 0;
  // output of the last pass
  float2* xout = nullptr;
  int n_out = 0;
  int out_mode = sr::kOutStore;
  const float* mu = nullptr;
  float mu_scale = 1.f;
  float shift = 0.f;
  float* spec_part_out = nullptr;
  float* loss_out = nullptr;
  // epilogue data
  const float* y = nullptr;
  const float* sumy = nullptr;
  float lam = 0.f;
  int weight_mode = SR_WEIGHT_IDENTITY;
  float* loss_part = nullptr;
  // GD loop fusion (power-of-two plans): the exchange buffer e0 already holds
  // the FIRST output of this step (written by the previous step's fused last
  // pass), and/or the last pass also runs the next step's FIRST into e0.
  bool skip_first = false;
  bool fuse_next_first = false;
  // power iteration: apply 1/||v|| (norm_in) in the spectral epilogue instead
  // of at the chain's input (the operations before it are linear)
  bool norm_at_epilogue = false;
  // radix-3 chains: the first pass of this inner chain reads the outer
  // vector (PassArgs::r3), applying first_op with the outer plan's tables
  bool r3_first = false;
  int ym = 0;
  // 2D plans: the chain's input / output is the transpose of the grid
  // (the forward's output and the adjoint's input when L is odd)
  int in_tr = 0;
  int out_tr = 0;
  const float2* first_dp = nullptr;
  int64_t first_dp_stride = 0;
  // alpha < 1: the first pass reads / the last pass writes the window of the
  // length-m vector starting at this offset (S^H / S)
  int in_off = 0;
  int out_off = 0;
};

sr::PassArgs base_args(const Plan& p) {
  sr::PassArgs a;
  std::memset(&a, 0, sizeof(a));
  a.m = (int)p.m;
  a.dp_stride = p.dp_stride;
  a.twl = p.d_twl;
  a.tw_hi = p.d_tw_hi;
  a.tw_lo = p.d_tw_lo;
  a.tw_shift = p.tw_shift;
  a.err = p.d_err;
  return a;
}

// Event pair around one pass launch when the plan records timing.
struct PassTimer {
  Plan* p;
  int cls;
  cudaStream_t s;
  cudaEvent_t end = nullptr;
  PassTimer(const Plan& plan, int k, cudaStream_t st) : p(const_cast<Plan*>(&plan)), cls(k), s(st) {
    if (!p->timing) return;
    std::vector<cudaEvent_t>& v = p->ev[cls];
    const size_t i = p->ev_used[cls];
    while (v.size() < i + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      v.push_back(e);
    }
    cudaEventRecord(v[i], s);
    end = v[i + 1];
    p->ev_used[cls] = i + 2;
  }
  ~PassTimer() {
    if (end) cudaEventRecord(end, s);
  }
};

sr_status run_chain_r3(const Plan& p, const Chain& c, int B, cudaStream_t s);

// Number of partial sums per problem the last stage of a chain writes (norm
// partials of the spectral update).
int final_partials(const Plan& p, int nfft, int s0) {
  if (sr::small_eligible(p)) return 1;  // the resident solver writes each norm whole
  if (p.inner) return p.r3_chunks;
  return p.geom[sr::s2_layout((s0 + nfft - 1) % 2)].cpp;
}

sr_status run_chain(const Plan& p, const Chain& c, int B, cudaStream_t s) {
  if (p.inner) return run_chain_r3(p, c, B, s);
  const sr::PassArgs base = base_args(p);
  float2* cur = p.d_e0;
  float2* nxt = p.d_e1;
  int cur_idx = 0;  // which exchange buffer `cur` is (selects its tensor maps)
  int loss_cpp = 0;
  // FIRST
  if (!c.skip_first) {
    sr::PassArgs a = base;
    a.out_dir = c.dir[0];
    a.xin = c.xin;
    a.n_in = c.n_in;
    a.norm_in = c.norm_at_epilogue ? nullptr : c.norm_in;
    a.norm_in_count = c.norm_in_count;
    a.op = c.first_op;
    a.dp = p.d_dp + (size_t)c.first_d * p.m;
    if (p.two_d) {
      a.in_h = c.n_in == p.m ? p.gS : p.gh;
      a.in_w = c.n_in == p.m ? p.gS : p.gw;
      a.in_tr = c.in_tr;
    }
    a.in_off = c.in_off;
    if (c.first_op == sr::kOpGdEpilogue || c.first_op == sr::kOpSpecEpilogue) {
      // the epilogue in the first pass (radix-3 chains, alpha < 1 adjoint chains)
      a.ym = c.ym;
      a.y = c.y;
      a.sumy = c.sumy;
      a.lam = c.lam;
      a.weight_mode = c.weight_mode;
      a.part_out = c.loss_part;
      if (c.first_op == sr::kOpGdEpilogue) loss_cpp = p.geom[sr::s1_layout(c.s0)].cpp;
    }
    if (c.r3_first) {
      a.r3 = 1;
      a.ym = c.ym;
      a.dp = c.first_dp;
      a.dp_stride = c.first_dp_stride;
    }
    a.eout = cur;
    PassTimer tm(p, 0, s);
    SR_CUDA(sr::launch_first(p, sr::s1_layout(c.s0), a, B, s), "launch(first pass)");
  }
  for (int k = 1; k < c.nfft; ++k) {
    const sr::Layout lay = sr::s2_layout((c.s0 + k - 1) % 2);
    sr::PassArgs a = base;
    a.in_dir = c.dir[k - 1];
    a.out_dir = c.dir[k];
    a.ein = cur;
    a.eout = nxt;
    a.tmap = p.tmap[cur_idx][lay];
    a.op = c.mid[k].op;
    a.dp = p.d_dp + (size_t)c.mid[k].d * p.m;
    if (a.op == sr::kOpDiag || a.op == sr::kOpDiagConj) {
      a.ph = p.d_ph + (size_t)c.mid[k].d * p.m;
      a.dscale = (float)(1.0 / std::sqrt((double)p.m));
    }
    if (a.op == sr::kOpGdEpilogue) {
      a.y = c.y;
      a.part_out = c.loss_part;
      loss_cpp = p.geom[lay].cpp * sr::epilogue_partials_per_tile(p.geom[lay]);
    } else if (a.op == sr::kOpSpecEpilogue) {
      a.y = c.y;
      a.sumy = c.sumy;
      a.lam = c.lam;
      a.weight_mode = c.weight_mode;
      if (c.norm_at_epilogue) {
        a.norm_in = c.norm_in;
        a.norm_in_count = c.norm_in_count;
      }
    }
    {
      PassTimer tm(p, 1, s);
      SR_CUDA(sr::launch_mid(p, lay, a, B, s), "launch(mid pass)");
    }
    std::swap(cur, nxt);
    cur_idx ^= 1;
  }
  // LAST
  {
    const sr::Layout lay = sr::s2_layout((c.s0 + c.nfft - 1) % 2);
    sr::PassArgs a = base;
    a.in_dir = c.dir[c.nfft - 1];
    a.ein = cur;
    a.tmap = p.tmap[cur_idx][lay];
    a.op = c.last_op;
    a.dp = p.d_dp;
    a.xout = c.xout;
    a.n_out = c.n_out;
    a.out_mode = c.out_mode;
    a.mu = c.mu;
    a.mu_scale = c.mu_scale;
    a.shift = c.shift;
    a.norm_in = c.norm_in;
    a.norm_in_count = c.norm_in_count;
    a.part_out = c.spec_part_out;
    a.loss_part = c.loss_part;
    a.loss_cpp = loss_cpp;
    a.loss_out = c.loss_out;
    a.out_off = c.out_off;
    if (p.two_d) {
      a.out_h = c.n_out == p.m ? p.gS : p.gh;
      a.out_w = c.n_out == p.m ? p.gS : p.gw;
      a.out_tr = c.out_tr;
    }
    PassTimer tm(p, 2, s);
    if (c.fuse_next_first) {
      a.eout = p.d_e0;  // the next step's FIRST output (cur is e1 here: 2L - 1 middle passes)
      SR_CUDA(sr::launch_last_first(p, lay, a, B, s), "launch(fused last/first pass)");
    } else {
      SR_CUDA(sr::launch_last(p, lay, a, B, s), "launch(last pass)");
    }
  }
  return SR_OK;
}

// A chain on a plan of length m = 3 mp: every DFT is a power-of-two DFT of
// length mp over 3B sequences on the inner plan, whose first pass gathers the
// stride-3 subsequences of the outer vector (with the operation that precedes
// the DFT), then a combine; the last combine applies D_1^H (if asked), prunes
// to n_out and applies the output mode. Buffers: the inner chain writes the 3B
// transformed sequences to e0, e1 holds the natural-order vector between DFTs.
sr_status run_chain_r3(const Plan& p, const Chain& c, int B, cudaStream_t s) {
  const Plan& in = *p.inner;
  const float2* src = c.xin;
  int64_t n_src = c.n_in;
  // loss partials of the GD epilogue: [3B][inner cpp] = [B][3 inner cpp]
  const int loss_cpp = 3 * in.geom[sr::s1_layout(0)].cpp;
  for (int k = 0; k < c.nfft; ++k) {
    Chain ic;
    ic.nfft = 1;
    ic.dir[0] = c.dir[k];
    ic.xin = src;
    ic.n_in = (int)n_src;
    ic.xout = p.d_e0;
    ic.n_out = (int)p.mp;
    ic.r3_first = true;
    ic.first_op = k == 0 ? c.first_op : c.mid[k].op;
    ic.first_dp = p.d_dp + (size_t)(k == 0 ? c.first_d : c.mid[k].d) * p.m;
    ic.first_dp_stride = p.dp_stride;
    ic.ym = (int)p.m;
    if (k == 0) {
      ic.norm_in = c.norm_in;
      ic.norm_in_count = c.norm_in_count;
    }
    ic.y = c.y;
    ic.sumy = c.sumy;
    ic.lam = c.lam;
    ic.weight_mode = c.weight_mode;
    ic.loss_part = c.loss_part;
    sr_status st = run_chain(in, ic, 3 * B, s);
    if (st != SR_OK) return st;
    sr::R3CombineArgs ca;
    std::memset(&ca, 0, sizeof(ca));
    ca.U = p.d_e0;
    ca.mp = p.mp;
    ca.chunks = p.r3_chunks;
    ca.tw3 = p.d_tw3;
    if (k + 1 < c.nfft) {
      ca.op = sr::kOpNone;
      ca.xout = p.d_e1;
      ca.n_out = p.m;
      ca.out_mode = sr::kOutStore;
    } else {
      ca.op = c.last_op;
      ca.dp = p.d_dp;
      ca.dp_stride = p.dp_stride;
      ca.xout = c.xout;
      ca.n_out = c.n_out;
      ca.out_mode = c.out_mode;
      ca.mu = c.mu;
      ca.mu_scale = c.mu_scale;
      ca.shift = c.shift;
      ca.norm_in = c.norm_in;
      ca.norm_in_count = c.norm_in_count;
      ca.part_out = c.spec_part_out;
      ca.loss_part = c.loss_part;
      ca.loss_cpp = loss_cpp;
      ca.loss_out = c.loss_out;
    }
    SR_CUDA(sr::launch_r3_combine(ca, c.dir[k], B, s), "launch(radix-3 combine)");
    src = p.d_e1;
    n_src = p.m;
  }
  return SR_OK;
}

// The 2L DFTs of one gradient or power-iteration step: A (D_1 first), then A^H.
Chain round_trip_chain(const Plan& p, int epilogue_op) {
  Chain c;
  const int L = p.L;
  c.nfft = 2 * L;
  c.s0 = 0;
  for (int k = 0; k < L; ++k) c.dir[k] = -1;
  for (int k = L; k < 2 * L; ++k) c.dir[k] = +1;
  c.first_op = sr::kOpDiag;  // D_1
  for (int k = 1; k < L; ++k) c.mid[k] = MidOp{sr::kOpDiag, k};  // D_{k+1}
  c.mid[L] = MidOp{epilogue_op, 0};
  for (int k = L + 1; k < 2 * L; ++k) c.mid[k] = MidOp{sr::kOpDiagConj, 2 * L - k};  // D_{2L-k+1}^H
  c.last_op = sr::kOpDiagConj;  // D_1^H
  return c;
}

// The measurements in the layout of the epilogue pass: y itself, or for 2D
// plans with odd L (the grid is transposed after L twiddle-free DFTs) a
// transposed copy in the plan's workspace.
sr_status epilogue_y(Plan* p, const float* y, int B, cudaStream_t s, const float** out) {
  *out = y;
  if (!(p->two_d && p->L % 2 == 1)) return SR_OK;
  SR_CUDA(sr::launch_transpose_grids(y, p->d_yt, p->gS, B, s), "launch(transpose y)");
  *out = p->d_yt;
  return SR_OK;
}

// z = A x: L forward DFTs, D_l before DFT l; for 2D plans with odd L the
// output is stored through the transposition, for alpha < 1 only the window.
Chain forward_chain(const Plan& p) {
  Chain c;
  c.nfft = p.L;
  c.s0 = 0;
  for (int k = 0; k < p.L; ++k) c.dir[k] = -1;
  c.first_op = sr::kOpDiag;
  for (int k = 1; k < p.L; ++k) c.mid[k] = MidOp{sr::kOpDiag, k};
  c.last_op = sr::kOpNone;
  c.n_in = (int)p.n;
  c.n_out = (int)p.mo;
  c.out_off = (int)p.off;
  c.out_mode = sr::kOutStore;
  c.out_tr = p.two_d && p.L % 2 == 1;  // 2D: L twiddle-free DFTs leave the grid transposed for odd L
  return c;
}

// x = A^H w: L inverse DFTs; the first pass reads the window (alpha < 1) or the
// grid in the layout the forward leaves it in (2D, odd L).
Chain adjoint_chain(const Plan& p) {
  Chain c;
  c.nfft = p.L;
  c.s0 = p.L % 2;  // keeps every D_l in the layout it was stored in
  for (int k = 0; k < p.L; ++k) c.dir[k] = +1;
  c.first_op = sr::kOpNone;
  for (int k = 1; k < p.L; ++k) c.mid[k] = MidOp{sr::kOpDiagConj, p.L - k};
  c.last_op = sr::kOpDiagConj;
  c.n_in = (int)p.mo;
  c.in_off = (int)p.off;
  c.in_tr = p.two_d && p.L % 2 == 1;
  c.n_out = (int)p.n;
  c.out_mode = sr::kOutStore;
  return c;
}

// alpha < 1 solver steps: the adjoint half reads A v from the window buffer
// and applies the epilogue (GD residual or spectral weights) in its first pass.
Chain window_adjoint_chain(const Plan& p, int epilogue_op, const float* y) {
  Chain c = adjoint_chain(p);
  c.first_op = epilogue_op;
  c.xin = p.d_zw;  // the window: entry i sits at off + i of the length-m vector (in_off)
  c.y = y;
  c.ym = (int)p.mo;
  return c;
}

// sum(y) per problem (and the GD step mu0 * m / sum(y)) into the scalar workspace.
sr_status prepare_y(Plan* p, const float* y, int B, float mu0, cudaStream_t s) {
  const int chunks = (int)std::min<int64_t>(64, (p->mo + 4095) / 4096);
  float* part = part_bank(*p, 3, B);
  SR_CUDA(sr::launch_sum_rows(y, B, (int)p->mo, part, chunks, s), "launch(sum y)");
  SR_CUDA(sr::launch_finish_scalars(part, chunks, B, mu0, (int)p->mo, p->d_scal, p->d_scal + B, s),
          "launch(step size)");
  return SR_OK;
}

sr_status check_plan_call(sr_plan* plan, int B) {
  if (!plan) return fail(SR_ERR_INVALID_ARG, "plan is NULL");
  if (B < 1) return fail(SR_ERR_INVALID_ARG, "B must be >= 1");
  if (B > 65535) return fail(SR_ERR_UNSUPPORTED, "B must be <= 65535");
  Plan* p = reinterpret_cast<Plan*>(plan);
  sr_status st = check_device(p);
  if (st != SR_OK) return st;
  if ((double)B * (double)p->m > 4.0e9) return fail(SR_ERR_UNSUPPORTED, "B*m too large");
  if (p->batch_fixed && B != p->batch_fixed)
    return fail(SR_ERR_INVALID_ARG, "this plan holds per-problem phases for a fixed batch size");
  if (p->inner) {
    if (3 * B > 65535) return fail(SR_ERR_UNSUPPORTED, "B must be <= 21845 when m = 3 * 2^a");
    if ((st = ensure_workspace(p->inner, 3 * B)) != SR_OK) return st;
  }
  return ensure_workspace(p, B);
}

}  // namespace

struct sr_plan : public Plan {};

namespace sr {
void set_last_error(const std::string& msg) { g_last_error = msg; }

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once per process (the static's
// initialisation is thread-safe); nullptr when the driver lacks it.
EncodeTiledFn tensor_map_encoder() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    const cudaError_t e =
        cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}
}  // namespace

cudaError_t encode_rows(CUtensorMap* map, float2* base, int ell, int64_t rows, int T) {
  const EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * ell), (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ell * 8};
  const cuuint32_t box[2] = {32, (cuuint32_t)T};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Gives each of B problems of the plan its own phases theta(seed_b): the
// diagonal table becomes [B][L][m] (problem stride L * m), filled from the same
// generator as sr_plan_create. Calls with another batch size are then invalid;
// used for batches of independent problems of one shape.
sr_status plan_set_problem_phases(sr_plan* plan, int B, const uint64_t* seeds) {
  if (!plan || !seeds || B < 1) return fail(SR_ERR_INVALID_ARG, "bad arguments");
  Plan& p = *plan;
  const int64_t lm = (int64_t)p.L * p.m;
  const double scale = 1.0 / std::sqrt((double)p.m);
  std::vector<double> th((size_t)lm);
  std::vector<float2> host((size_t)B * lm);
  std::vector<float> phh((size_t)B * lm);
  for (int b = 0; b < B; ++b) {
    gen_phases(seeds[b], p.L, p.m, th.data());
    for (int64_t i = 0; i < lm; ++i) {
      host[(size_t)b * lm + i] = make_float2((float)(std::cos(th[i]) * scale), (float)(std::sin(th[i]) * scale));
      phh[(size_t)b * lm + i] = (float)wrap_phase(th[i]);
    }
  }
  float2* d = nullptr;
  float* ph = nullptr;
  sr_status st = dalloc(&d, host.size());
  if (st != SR_OK) return st;
  if ((st = dalloc(&ph, phh.size())) != SR_OK) {
    cudaFree(d);
    return st;
  }
  cudaError_t e = cudaMemcpy(d, host.data(), host.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ph, phh.data(), phh.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    cudaFree(ph);
    return cuda_fail(e, "cudaMemcpy(problem diagonals)");
  }
  cudaFree(p.d_dp);
  cudaFree(p.d_ph);
  p.d_dp = d;
  p.d_ph = ph;
  p.dp_stride = lm;
  p.batch_fixed = B;
  gen_phases(seeds[0], p.L, p.m, p.theta.data());
  return SR_OK;
}
}  // namespace sr

extern "C" {

sr_status sr_phases(uint64_t seed, int L, int64_t m, double* theta) {
  if (!theta) return fail(SR_ERR_INVALID_ARG, "theta is NULL");
  if (L < 1 || m < 1) return fail(SR_ERR_INVALID_ARG, "need L >= 1 and m >= 1");
  gen_phases(seed, L, m, theta);
  return SR_OK;
}

}  // extern "C"

namespace {
// Plan construction shared by the 1D and the 2D entry points; gS > 0 makes a
// 2D plan of gh x gw images in a gS x gS grid (n = gh * gw, m = gS * gS).
sr_status create_plan(int64_t n, int64_t m, int L, uint64_t seed, int gh, int gw, int gS, sr_plan** out) {
  if (!out) return fail(SR_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  sr_status st = check_sizes(n, m, L);
  if (st != SR_OK) return st;
  sr_plan* p = new (std::nothrow) sr_plan();
  if (!p) return fail(SR_ERR_OOM, "host allocation failed");
  p->n = n;
  p->m = m;
  p->mo = m;
  p->off = 0;
  p->L = L;
  p->seed = seed;
  p->two_d = gS > 0;
  p->gh = gh;
  p->gw = gw;
  p->gS = gS;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaGetDevice");
  }
  // m = 3 * 2^a: lines of 192, 384 or 768 points (a radix-3 step inside the
  // line FFT) against power-of-two lines of 16 .. 4096 points, the most
  // balanced split the pass kernels cover
  std::vector<int> r3_splits;
  if (is_three_pow2(m) && gS == 0) {
    std::vector<std::pair<double, int>> c;
    for (int r : {192, 384, 768}) {
      if (m % r != 0 || !is_pow2(m / r) || m / r < 16 || m / r > 4096) continue;
      const int q = (int)(m / r);
      const double bal = std::fabs(std::log2((double)r / (double)q));
      c.push_back({bal, r});
      c.push_back({bal + 1e-3, q});  // the same lines, radix-3 ones in layout Y
    }
    std::sort(c.begin(), c.end());
    for (auto& e2 : c) r3_splits.push_back(e2.second);
  }
  bool r3_lines = false;
  if (!r3_splits.empty()) {
    const int a = ilog2(m);
    p->tw_shift = (a + 1) / 2;
    e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
      delete p;
      return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    for (int m1 : r3_splits)
      if (set_split(p, m1) == SR_OK) {
        r3_lines = true;
        break;
      }
    if (r3_lines && (st = upload_twiddles(p)) != SR_OK) {
      sr_plan_destroy(p);
      return st;
    }
    if (!r3_lines) sr::set_last_error("");
  }
  if (r3_lines) {
    // (set up above)
  } else if (is_three_pow2(m)) {
    // m = 3 mp without a radix-3 line split: the power-of-two DFTs run on an
    // inner plan of length mp
    p->mp = m / 3;
    p->r3_chunks = (int)std::min<int64_t>(256, std::max<int64_t>(1, p->mp / 1024));
    sr_plan* in = nullptr;
    if ((st = sr_plan_create(p->mp, p->mp, 1, 0, &in)) != SR_OK) {
      delete p;
      return st;
    }
    p->inner = in;
    p->num_sms = in->num_sms;
    std::vector<float2> tw3((size_t)(2 * p->mp));
    for (int64_t j = 0; j < 2 * p->mp; ++j) tw3[j] = root_of_unity(j, m);
    if ((st = dalloc(&p->d_tw3, tw3.size())) != SR_OK) {
      sr_plan_destroy(p);
      return st;
    }
    e = cudaMemcpy(p->d_tw3, tw3.data(), tw3.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      sr_plan_destroy(p);
      return cuda_fail(e, "cudaMemcpy(radix-3 twiddles)");
    }
  } else {
    const int a = ilog2(m);
    p->tw_shift = (a + 1) / 2;
    e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
      delete p;
      return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    // the balanced split (the longer line first); sr_plan_autotune may choose another
    if ((st = set_split(p, 1 << ((a + 1) / 2))) != SR_OK || (st = upload_twiddles(p)) != SR_OK) {
      sr_plan_destroy(p);
      return st;
    }
  }
  p->theta.resize((size_t)L * m);
  gen_phases(seed, L, m, p->theta.data());
  if ((st = dalloc(&p->d_dp, (size_t)L * m)) != SR_OK || (st = dalloc(&p->d_ph, (size_t)L * m)) != SR_OK ||
      (st = upload_diagonals(p)) != SR_OK ||
      (st = dalloc(&p->d_err, 1)) != SR_OK) {
    sr_plan_destroy(p);
    return st;
  }
  e = cudaMemset(p->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    sr_plan_destroy(p);
    return cuda_fail(e, "cudaMemset");
  }
  *out = p;
  return SR_OK;
}
// The fields of the resident small-m solver's arguments common to every call.
sr::SmallArgs small_args(const Plan& p, const float* y, void* x, int B) {
  sr::SmallArgs a;
  std::memset(&a, 0, sizeof(a));
  a.m = (int)p.m;
  a.n = (int)p.n;
  a.mo = (int)p.mo;
  a.off = (int)p.off;
  a.L = p.L;
  a.B = B;
  a.dp = p.d_dp;
  a.dp_stride = p.dp_stride;
  a.tw_hi = p.d_tw_hi;
  a.tw_lo = p.d_tw_lo;
  a.tw_shift = p.tw_shift;
  a.y = y;
  a.sumy = p.d_scal;
  a.x = (float2*)x;
  return a;
}

// Power iteration shared by the spectral entry points: the step chains, the
// ping-pong banks of norm partials and the bank of the latest iterate.
struct SpectralRun {
  Plan* p = nullptr;
  int B = 0;
  cudaStream_t s = nullptr;
  float2* v = nullptr;
  float* bank[2] = {nullptr, nullptr};
  int prev = 1, prev_count = 0, last_cpp = 0;
  int done = 0;  // steps run so far
  bool window = false, fuse = false, small = false;
  const float* ye = nullptr;
  sr_spectral_opts o{SR_WEIGHT_OPTIMAL, -1.0f};
  Chain c, f, a;

  sr_status setup(sr_plan* plan, const float* y, const void* v0, const sr_spectral_opts* opts, void* x_out, int nb,
                  cudaStream_t st_) {
    sr_status st = check_plan_call(plan, nb);
    if (st != SR_OK) return st;
    if (!y || !v0 || !x_out) return fail(SR_ERR_INVALID_ARG, "NULL array argument");
    if (opts) o = *opts;
    if (o.weight_mode != SR_WEIGHT_IDENTITY && o.weight_mode != SR_WEIGHT_OPTIMAL)
      return fail(SR_ERR_INVALID_ARG, "unknown weight_mode");
    if (o.weight_mode == SR_WEIGHT_OPTIMAL && !(o.lambda < 0.f && std::isfinite(o.lambda)))
      return fail(SR_ERR_INVALID_ARG, "lambda must be finite and < 0");
    p = plan;
    B = nb;
    s = st_;
    const int n = (int)p->n;
    if (x_out != v0)
      SR_CUDA(cudaMemcpyAsync(x_out, v0, (size_t)B * n * sizeof(float2), cudaMemcpyDeviceToDevice, s),
              "cudaMemcpyAsync(v0)");
    if ((st = prepare_y(p, y, B, 0.f, s)) != SR_OK) return st;
    if ((st = epilogue_y(p, y, B, s, &ye)) != SR_OK) return st;
    v = (float2*)x_out;
    prev_count = std::min(64, (n + 4095) / 4096);
    bank[0] = part_bank(*p, 0, B);
    bank[1] = part_bank(*p, 1, B);
    SR_CUDA(sr::launch_norm_rows(v, B, n, bank[1], prev_count, s), "launch(norm v0)");
    last_cpp = final_partials(*p, 2 * p->L, 0);
    const float shift = o.weight_mode == SR_WEIGHT_IDENTITY ? 0.f : -2.0f * o.lambda;
    small = sr::small_eligible(*p);
    window = p->mo < p->m;
    if (window) {
      // alpha < 1: forward chain of v / ||v|| into the window, adjoint chain with
      // the spectral weights in its first pass and the update u = M v + s v last
      f = forward_chain(*p);
      f.xin = v;
      f.xout = p->d_zw;
      a = window_adjoint_chain(*p, sr::kOpSpecEpilogue, ye);
      a.sumy = p->d_scal;
      a.lam = o.lambda;
      a.weight_mode = o.weight_mode;
      a.norm_at_epilogue = true;  // no input scale in its first pass; the last pass uses norm_in
      a.xout = v;
      a.out_mode = sr::kOutSpec;
      a.shift = shift;
      return SR_OK;
    }
    c = round_trip_chain(*p, sr::kOpSpecEpilogue);
    c.xin = v;
    c.n_in = n;
    c.xout = v;
    c.n_out = n;
    c.out_mode = sr::kOutSpec;
    c.shift = shift;
    c.y = ye;
    c.sumy = p->d_scal;
    c.lam = o.lambda;
    c.weight_mode = o.weight_mode;
    // Consecutive steps share a kernel (see sr_gd_solve); the iterate then enters
    // each step unnormalised and its 1/||u|| is applied in the spectral epilogue.
    fuse = !p->inner;
    c.norm_at_epilogue = fuse;
    return SR_OK;
  }

  // `count` more steps u = M v + s v (v = previous u / ||u||); the last of them
  // does not fuse into a following FIRST, so calls can be chained.
  sr_status steps(int count) {
    sr_status st;
    if (small) {  // all `count` steps in one launch of the resident solver
      if (count <= 0) return SR_OK;
      sr::SmallArgs sa = small_args(*p, ye, v, B);
      sa.count = count;
      sa.weight_mode = o.weight_mode;
      sa.lam = o.lambda;
      sa.shift = o.weight_mode == SR_WEIGHT_IDENTITY ? 0.f : -2.0f * o.lambda;
      sa.norm_in = bank[prev];
      sa.norm_in_count = prev_count;
      const int last = (done + count - 1) % 2;
      sa.norm_last = bank[last];
      sa.norm_prev = bank[1 - last];
      SR_CUDA(sr::launch_small(*p, sa, true, s), "launch(small power iteration)");
      done += count;
      prev = last;
      prev_count = 1;
      return SR_OK;
    }
    for (int it = 0; it < count; ++it, ++done) {
      const int cur = done % 2;
      if (window) {
        f.norm_in = a.norm_in = bank[prev];
        f.norm_in_count = a.norm_in_count = prev_count;
        a.spec_part_out = bank[cur];
        if ((st = run_chain(*p, f, B, s)) != SR_OK) return st;
        if ((st = run_chain(*p, a, B, s)) != SR_OK) return st;
      } else {
        c.norm_in = bank[prev];
        c.norm_in_count = prev_count;
        c.spec_part_out = bank[cur];
        c.skip_first = fuse && it > 0;
        c.fuse_next_first = fuse && it + 1 < count;
        if ((st = run_chain(*p, c, B, s)) != SR_OK) return st;
      }
      prev = cur;
      prev_count = last_cpp;
    }
    return SR_OK;
  }

  // x = sqrt(sum y) v / ||v||
  sr_status finish() {
    SR_CUDA(sr::launch_scale_rows(v, B, (int)p->n, bank[prev], prev_count, p->d_scal, s), "launch(scale)");
    return SR_OK;
  }
};

// Validation and the per-problem step mu0 * m / sum(y) shared by the GD entry points.
sr_status gd_setup(sr_plan* plan, const float* y, void* x, int iters, const sr_gd_opts* opts, int B, void* stream,
                   float* mu0_out, float* tau0_out) {
  sr_status st = check_plan_call(plan, B);
  if (st != SR_OK) return st;
  if (!y || !x) return fail(SR_ERR_INVALID_ARG, "NULL array argument");
  if (iters < 0) return fail(SR_ERR_INVALID_ARG, "iters must be >= 0");
  const float mu0 = opts ? opts->mu0 : 0.1f;
  const float tau0 = opts ? opts->tau0 : 0.f;
  if (!(mu0 > 0.f && std::isfinite(mu0))) return fail(SR_ERR_INVALID_ARG, "mu0 must be finite and > 0");
  if (!(tau0 >= 0.f && std::isfinite(tau0))) return fail(SR_ERR_INVALID_ARG, "tau0 must be finite and >= 0");
  *mu0_out = mu0;
  *tau0_out = tau0;
  return prepare_y(plan, y, B, mu0, (cudaStream_t)stream);
}

// GD iterations t0 .. t0+count-1 on x (the warm-up factor uses the global
// index t); loss_row(t) is where iteration t's loss goes, or nullptr.
template <class RowFn>
sr_status gd_iterations(Plan& p, const float* ye, void* x, int t0, int count, float tau0, int B, cudaStream_t s,
                        RowFn loss_row) {
  sr_status st;
  if (sr::small_eligible(p)) {  // all `count` steps in one launch of the resident solver
    if (count <= 0) return SR_OK;
    sr::SmallArgs a = small_args(p, ye, x, B);
    a.count = count;
    a.mu = p.d_scal + B;
    a.t0 = t0;
    a.tau0 = tau0;
    for (int t = t0; t < t0 + count; ++t) {
      if (float* row = loss_row(t)) {  // rows are B apart from the first recorded step on
        a.loss_hist = row;
        a.loss_first = t;
        break;
      }
    }
    SR_CUDA(sr::launch_small(p, a, false, s), "launch(small solve)");
    return SR_OK;
  }
  auto ramp = [&](int t) {
    return tau0 > 0.f ? (float)(1.0 - std::exp(-(double)(t + 1) / (double)tau0)) : 1.0f;
  };
  if (p.mo < p.m) {
    // alpha < 1: forward chain into the window, adjoint chain with the GD
    // residual in its first pass and the update x -= mu_t 2 A^H(r z) last
    Chain f = forward_chain(p);
    f.xin = (const float2*)x;
    f.xout = p.d_zw;
    Chain a = window_adjoint_chain(p, sr::kOpGdEpilogue, ye);
    a.loss_part = part_bank(p, 2, B);
    a.xout = (float2*)x;
    a.out_mode = sr::kOutGd;
    a.mu = p.d_scal + B;
    for (int t = t0; t < t0 + count; ++t) {
      a.loss_out = loss_row(t);
      a.mu_scale = ramp(t);
      if ((st = run_chain(p, f, B, s)) != SR_OK) return st;
      if ((st = run_chain(p, a, B, s)) != SR_OK) return st;
    }
    return SR_OK;
  }
  Chain c = round_trip_chain(p, sr::kOpGdEpilogue);
  c.xin = (const float2*)x;
  c.n_in = (int)p.n;
  c.xout = (float2*)x;
  c.n_out = (int)p.n;
  c.out_mode = sr::kOutGd;
  c.mu = p.d_scal + B;
  c.y = ye;
  c.loss_part = part_bank(p, 2, B);
  // Consecutive steps share a kernel: the last pass of step t also runs the
  // first pass of step t+1 (same lines, x_{t+1} still in registers).
  const bool fuse = !p.inner && (2 * p.L - 1) % 2 == 1;
  for (int t = t0; t < t0 + count; ++t) {
    c.loss_out = loss_row(t);
    c.mu_scale = ramp(t);
    c.skip_first = fuse && t > t0;
    c.fuse_next_first = fuse && t + 1 < t0 + count;
    if ((st = run_chain(p, c, B, s)) != SR_OK) return st;
  }
  return SR_OK;
}

}  // namespace

extern "C" {

sr_status sr_plan_create(int64_t n, int64_t m, int L, uint64_t seed, sr_plan** out) {
  if (m >= 1 && m < n) {
    // alpha < 1: DFTs of length n, then S keeps the m central entries
    if (!out) return fail(SR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!(is_pow2(n) && n >= 4 && n <= (int64_t(1) << 24)))
      return fail(SR_ERR_UNSUPPORTED, "with m < n, n must be 2^a in [4, 2^24]");
    sr_status st = create_plan(n, n, L, seed, 0, 0, 0, out);
    if (st != SR_OK) return st;
    (*out)->mo = m;
    (*out)->off = (n - m) / 2;
    return SR_OK;
  }
  return create_plan(n, m, L, seed, 0, 0, 0, out);
}

sr_status sr_plan_create_2d(int64_t h, int64_t w, int64_t S, int L, uint64_t seed, sr_plan** out) {
  if (!out) return fail(SR_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (S < 2 || S > 4096 || !is_pow2(S)) return fail(SR_ERR_UNSUPPORTED, "S must be a power of two in [2, 4096]");
  if (h < 1 || w < 1 || h > S || w > S) return fail(SR_ERR_UNSUPPORTED, "need 1 <= h <= S and 1 <= w <= S");
  return create_plan(h * w, S * S, L, seed, (int)h, (int)w, (int)S, out);
}

sr_status sr_plan_destroy(sr_plan* plan) {
  if (!plan) return SR_OK;
  for (auto& v : plan->ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  free_workspace(plan);
  cudaFree(plan->d_w0);
  cudaFree(plan->d_w1);
  cudaFree(plan->d_theta_f);
  cudaFree(plan->d_ph);
  cudaFree(plan->d_err);
  cudaFree(plan->d_dp);
  cudaFree(plan->d_twl);
  cudaFree(plan->d_tw_hi);
  cudaFree(plan->d_tw_lo);
  cudaFree(plan->d_tw3);
  cudaFree(plan->d_es);
  if (plan->inner) sr_plan_destroy(static_cast<sr_plan*>(plan->inner));
  delete plan;
  return SR_OK;
}

sr_status sr_plan_set_batch_phases(sr_plan* plan, int B, const uint64_t* seeds) {
  if (!plan || !seeds || B < 1) return fail(SR_ERR_INVALID_ARG, "NULL argument or B < 1");
  if (plan->two_d) return fail(SR_ERR_UNSUPPORTED, "per-problem phases are not supported on 2D plans");
  if (plan->inner && 3 * B > 65535) return fail(SR_ERR_UNSUPPORTED, "B must be <= 21845 when m = 3 * 2^a");
  sr_status st = check_device(plan);
  if (st != SR_OK) return st;
  return sr::plan_set_problem_phases(plan, B, seeds);
}

sr_status sr_plan_get_phases(const sr_plan* plan_c, double* theta) {
  if (!plan_c || !theta) return fail(SR_ERR_INVALID_ARG, "NULL argument");
  sr_plan* plan = const_cast<sr_plan*>(plan_c);
  if (plan->host_theta_stale) {
    // phases were last set from the device: refresh the host copy
    std::vector<float> f(plan->theta.size());
    SR_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    SR_CUDA(cudaMemcpy(f.data(), plan->d_theta_f, f.size() * sizeof(float), cudaMemcpyDeviceToHost), "cudaMemcpy");
    for (size_t i = 0; i < f.size(); ++i) plan->theta[i] = f[i];
    plan->host_theta_stale = false;
  }
  std::memcpy(theta, plan->theta.data(), plan->theta.size() * sizeof(double));
  return SR_OK;
}

sr_status sr_plan_set_phases_device(sr_plan* plan, const float* theta, void* stream) {
  if (!plan || !theta) return fail(SR_ERR_INVALID_ARG, "NULL argument");
  if (plan->two_d) return fail(SR_ERR_UNSUPPORTED, "device phases are not supported on 2D plans");
  sr_status st = check_device(plan);
  if (st != SR_OK) return st;
  const size_t count = (size_t)plan->L * plan->m;
  if (!plan->d_theta_f && (st = dalloc(&plan->d_theta_f, count)) != SR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  SR_CUDA(cudaMemcpyAsync(plan->d_theta_f, theta, count * sizeof(float), cudaMemcpyDeviceToDevice, s),
          "cudaMemcpyAsync(theta)");
  SR_CUDA(sr::launch_set_diag(plan->d_theta_f, plan->d_dp, plan->d_ph, count,
                              (float)(1.0 / std::sqrt((double)plan->m)), s),
          "launch(diagonals)");
  plan->host_theta_stale = true;
  return SR_OK;
}

sr_status sr_plan_set_phases(sr_plan* plan, const double* theta) {
  if (!plan || !theta) return fail(SR_ERR_INVALID_ARG, "NULL argument");
  sr_status st = check_device(plan);
  if (st != SR_OK) return st;
  for (size_t i = 0; i < plan->theta.size(); ++i)
    if (!std::isfinite(theta[i])) return fail(SR_ERR_NUMERIC, "non-finite phase");
  std::memcpy(plan->theta.data(), theta, plan->theta.size() * sizeof(double));
  plan->host_theta_stale = false;
  SR_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  return upload_diagonals(plan);
}

sr_status sr_plan_info(const sr_plan* plan, int64_t* n, int64_t* m, int* L) {
  if (!plan) return fail(SR_ERR_INVALID_ARG, "plan is NULL");
  if (n) *n = plan->n;
  if (m) *m = plan->mo;  // measurements (the DFT length is max(n, m))
  if (L) *L = plan->L;
  return SR_OK;
}

sr_status sr_plan_reserve(sr_plan* plan, int B) { return check_plan_call(plan, B); }

// Times `reps` GD steps of the plan over B problems of scratch data (after two
// untimed steps); 0 on success.
static sr_status time_gd_steps(sr_plan* plan, const float* y, float2* x, int B, cudaStream_t s, cudaEvent_t e0,
                               cudaEvent_t e1, float* ms) {
  const sr_gd_opts o{1e-6f, 0.f};
  sr_status st;
  if ((st = sr_gd_solve(plan, y, x, 2, &o, nullptr, B, s)) != SR_OK) return st;
  SR_CUDA(cudaEventRecord(e0, s), "cudaEventRecord");
  if ((st = sr_gd_solve(plan, y, x, 5, &o, nullptr, B, s)) != SR_OK) return st;
  SR_CUDA(cudaEventRecord(e1, s), "cudaEventRecord");
  SR_CUDA(cudaEventSynchronize(e1), "cudaEventSynchronize");
  SR_CUDA(cudaEventElapsedTime(ms, e0, e1), "cudaEventElapsedTime");
  return SR_OK;
}

// Caps every persistent-pass grid of the plan at c CTAs per SM (c <= 0: the
// kernels' occupancy).
static void cap_grids(Plan& p, const int (&mid)[2][3], const int (&last)[2][2], const int (&lf)[2], int c) {
  for (int l = 0; l < 2; ++l) {
    for (int k = 0; k < 3; ++k) p.per_sm_mid[l][k] = c > 0 ? std::min(c, mid[l][k]) : mid[l][k];
    for (int k = 0; k < 2; ++k) p.per_sm_last[l][k] = c > 0 ? std::min(c, last[l][k]) : last[l][k];
    p.per_sm_lf[l] = c > 0 ? std::min(c, lf[l]) : lf[l];
  }
  p.tuned_per_sm = c > 0 ? c : 0;
}

sr_status sr_plan_autotune(sr_plan* plan, int B, void* stream) {
  sr_status st = check_plan_call(plan, B);
  if (st != SR_OK) return st;
  Plan& p = plan->inner ? *plan->inner : *plan;
  cudaStream_t s = (cudaStream_t)stream;
  const int cap_outer = plan->B_cap;
  // Candidate four-step splits (1D plans on the four-step passes): the
  // balanced one and its neighbours by a factor of two, each line of 16 to
  // 4096 points with pass kernels for both line lengths.
  std::vector<int> splits{p.m1};
  if (!p.two_d && !sr::small_eligible(p)) {
    for (int m1 : {p.m1 / 2, p.m1 * 2}) {
      const int64_t m2 = p.m / std::max(1, m1);
      if (m1 >= 16 && m1 <= 4096 && m2 >= 16 && m2 <= 4096) splits.push_back(m1);
    }
  }
  float* y = nullptr;
  float2* x = nullptr;
  if ((st = dalloc(&y, (size_t)B * plan->m)) != SR_OK) return st;
  if ((st = dalloc(&x, (size_t)B * plan->n)) != SR_OK) {
    cudaFree(y);
    return st;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemsetAsync(y, 0x3F, sizeof(float) * (size_t)B * plan->m, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0x3F, sizeof(float2) * (size_t)B * plan->n, s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // For every split the kernels support, the persistent-grid sizes of the
  // middle and last passes from the kernels' occupancy down to 1 CTA per SM.
  float best_ms = 0.f;
  int best_split = p.m1, best_c = 0;
  bool have = false;
  for (size_t si = 0; si < splits.size() && e == cudaSuccess && st == SR_OK; ++si) {
    if (splits[si] != p.m1 && set_split(&p, splits[si]) != SR_OK) continue;  // no kernels for this split
    if (plan->inner) free_workspace(plan);  // the outer plan's banks follow the inner geometry
    int mid[2][3], last[2][2], lf[2];
    std::memcpy(mid, p.per_sm_mid, sizeof(mid));
    std::memcpy(last, p.per_sm_last, sizeof(last));
    std::memcpy(lf, p.per_sm_lf, sizeof(lf));
    int max_occ = 1;
    for (int l = 0; l < 2; ++l) {
      for (int k = 0; k < 3; ++k) max_occ = std::max(max_occ, mid[l][k]);
      for (int k = 0; k < 2; ++k) max_occ = std::max(max_occ, last[l][k]);
      max_occ = std::max(max_occ, lf[l]);
    }
    for (int c = max_occ; c >= 1 && st == SR_OK; --c) {
      cap_grids(p, mid, last, lf, c);
      float ms = 0.f;
      if ((st = time_gd_steps(plan, y, x, B, s, e0, e1, &ms)) != SR_OK) break;
      if (!have || ms < best_ms) {
        have = true;
        best_ms = ms;
        best_split = p.m1;
        best_c = c;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(y);
  cudaFree(x);
  if (st == SR_OK && e != cudaSuccess) st = cuda_fail(e, "autotune");
  // the winner (the balanced split if nothing was timed) with its grid size,
  // and the workspace the plan held before
  sr_status st2 = set_split(&p, best_split);
  if (st2 == SR_OK) {
    int mid[2][3], last[2][2], lf[2];
    std::memcpy(mid, p.per_sm_mid, sizeof(mid));
    std::memcpy(last, p.per_sm_last, sizeof(last));
    std::memcpy(lf, p.per_sm_lf, sizeof(lf));
    cap_grids(p, mid, last, lf, best_c);
    if (plan->inner) free_workspace(plan);
    st2 = check_plan_call(plan, plan->batch_fixed ? B : std::max(B, cap_outer));
  }
  return st != SR_OK ? st : st2;
}

sr_status sr_plan_set_split(sr_plan* plan, int m1) {
  if (!plan) return fail(SR_ERR_INVALID_ARG, "plan is NULL");
  sr_status st = check_device(plan);
  if (st != SR_OK) return st;
  if (plan->two_d) return fail(SR_ERR_UNSUPPORTED, "2D plans keep the S x S split");
  Plan& p = plan->inner ? *plan->inner : *plan;
  const int cap = plan->B_cap;
  SR_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  if ((st = set_split(&p, m1)) != SR_OK) return st;
  if (plan->inner) free_workspace(plan);
  return cap > 0 ? check_plan_call(plan, plan->batch_fixed ? plan->batch_fixed : cap) : SR_OK;
}

sr_status sr_plan_tuning(const sr_plan* plan, int* m1, int* m2, int* ctas_per_sm) {
  if (!plan) return fail(SR_ERR_INVALID_ARG, "plan is NULL");
  const Plan& p = plan->inner ? *static_cast<const Plan*>(plan->inner) : *static_cast<const Plan*>(plan);
  if (m1) *m1 = p.m1;
  if (m2) *m2 = p.m2;
  if (ctas_per_sm) *ctas_per_sm = p.tuned_per_sm;
  return SR_OK;
}

sr_status sr_forward(sr_plan* plan, const void* x, void* z, int B, void* stream) {
  sr_status st = check_plan_call(plan, B);
  if (st != SR_OK) return st;
  if (!x || !z) return fail(SR_ERR_INVALID_ARG, "NULL array argument");
  Plan& p = *plan;
  if (sr::small_eligible(p)) {  // one launch: the whole operator inside one CTA per problem
    sr::SmallArgs a = small_args(p, nullptr, const_cast<void*>(x), B);
    a.op = 1;
    a.zout = (float2*)z;
    SR_CUDA(sr::launch_small(p, a, false, (cudaStream_t)stream), "launch(small forward)");
    return SR_OK;
  }
  Chain c = forward_chain(p);
  c.xin = (const float2*)x;
  c.xout = (float2*)z;
  return run_chain(p, c, B, (cudaStream_t)stream);
}

sr_status sr_adjoint(sr_plan* plan, const void* z, void* x, int B, void* stream) {
  sr_status st = check_plan_call(plan, B);
  if (st != SR_OK) return st;
  if (!x || !z) return fail(SR_ERR_INVALID_ARG, "NULL array argument");
  Plan& p = *plan;
  if (sr::small_eligible(p)) {
    sr::SmallArgs a = small_args(p, nullptr, x, B);
    a.op = 2;
    a.win = (const float2*)z;
    SR_CUDA(sr::launch_small(p, a, false, (cudaStream_t)stream), "launch(small adjoint)");
    return SR_OK;
  }
  Chain c = adjoint_chain(p);
  c.xin = (const float2*)z;
  c.xout = (float2*)x;
  return run_chain(p, c, B, (cudaStream_t)stream);
}

sr_status sr_loss_grad(sr_plan* plan, const void* x, const float* y, float* loss, void* grad, int B,
                       void* stream) {
  sr_status st = check_plan_call(plan, B);
  if (st != SR_OK) return st;
  if (!x || !y || !grad) return fail(SR_ERR_INVALID_ARG, "NULL array argument");
  Plan& p = *plan;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = prepare_y(&p, y, B, 0.f, s)) != SR_OK) return st;
  const float* ye = nullptr;
  if ((st = epilogue_y(&p, y, B, s, &ye)) != SR_OK) return st;
  if (sr::small_eligible(p)) {
    sr::SmallArgs a = small_args(p, ye, const_cast<void*>(x), B);
    a.count = 1;
    a.grad = 1;
    a.g = (float2*)grad;
    a.loss_out = loss;
    SR_CUDA(sr::launch_small(p, a, false, s), "launch(small gradient)");
    return SR_OK;
  }
  if (p.mo < p.m) {
    Chain f = forward_chain(p);
    f.xin = (const float2*)x;
    f.xout = p.d_zw;
    if ((st = run_chain(p, f, B, s)) != SR_OK) return st;
    Chain a = window_adjoint_chain(p, sr::kOpGdEpilogue, ye);
    a.loss_part = part_bank(p, 2, B);
    a.loss_out = loss;
    a.xout = (float2*)grad;
    a.out_mode = sr::kOutGrad;
    return run_chain(p, a, B, s);
  }
  Chain c = round_trip_chain(p, sr::kOpGdEpilogue);
  c.xin = (const float2*)x;
  c.n_in = (int)p.n;
  c.xout = (float2*)grad;
  c.n_out = (int)p.n;
  c.out_mode = sr::kOutGrad;
  c.y = ye;
  c.loss_part = part_bank(p, 2, B);
  c.loss_out = loss;
  return run_chain(p, c, B, s);
}

sr_status sr_spectral_init(sr_plan* plan, const float* y, const void* v0, int iters, const sr_spectral_opts* opts,
                           void* x_out, int B, void* stream) {
  if (iters < 0) return fail(SR_ERR_INVALID_ARG, "iters must be >= 0");
  SpectralRun r;
  sr_status st = r.setup(plan, y, v0, opts, x_out, B, (cudaStream_t)stream);
  if (st != SR_OK) return st;
  if ((st = r.steps(iters)) != SR_OK) return st;
  return r.finish();
}

sr_status sr_spectral_init_early_stop(sr_plan* plan, const float* y, const void* v0, int max_iters,
                                      const sr_spectral_opts* opts, float rel_tol, int check_every, void* x_out,
                                      int* iters_run, int B, void* stream) {
  if (!iters_run) return fail(SR_ERR_INVALID_ARG, "iters_run is NULL");
  *iters_run = 0;
  if (max_iters < 0) return fail(SR_ERR_INVALID_ARG, "max_iters must be >= 0");
  if (check_every < 2) return fail(SR_ERR_INVALID_ARG, "check_every must be >= 2");
  if (!(rel_tol >= 0.f && std::isfinite(rel_tol))) return fail(SR_ERR_INVALID_ARG, "rel_tol must be finite and >= 0");
  SpectralRun r;
  sr_status st = r.setup(plan, y, v0, opts, x_out, B, (cudaStream_t)stream);
  if (st != SR_OK) return st;
  const int stride = part_stride(*plan);
  std::vector<float> banks(2 * (size_t)B * stride);
  while (r.done < max_iters) {
    const int count = std::min(check_every, max_iters - r.done);
    if ((st = r.steps(count)) != SR_OK) return st;
    *iters_run = r.done;
    if (count < check_every || r.done >= max_iters) break;
    // lambda_t^2 and lambda_{t-1}^2 are the sums of the two banks' partials
    // (bank k holds problem b's last_cpp partials at k B stride + b last_cpp)
    SR_CUDA(cudaMemcpyAsync(banks.data(), r.bank[0], banks.size() * sizeof(float), cudaMemcpyDeviceToHost, r.s),
            "cudaMemcpyAsync(norm partials)");
    SR_CUDA(cudaStreamSynchronize(r.s), "cudaStreamSynchronize");
    bool all = true;
    for (int b = 0; b < B && all; ++b) {
      double sq[2] = {0.0, 0.0};
      for (int k = 0; k < 2; ++k)
        for (int i = 0; i < r.last_cpp; ++i) sq[k] += banks[(size_t)k * B * stride + (size_t)b * r.last_cpp + i];
      const double cur = std::sqrt(sq[r.prev]), prev = std::sqrt(sq[1 - r.prev]);
      all = std::fabs(prev - cur) <= (double)rel_tol * prev;
    }
    if (all) break;
  }
  return r.finish();
}

sr_status sr_gd_solve(sr_plan* plan, const float* y, void* x, int iters, const sr_gd_opts* opts, float* loss_hist,
                      int B, void* stream) {
  float mu0 = 0.f, tau0 = 0.f;
  sr_status st = gd_setup(plan, y, x, iters, opts, B, stream, &mu0, &tau0);
  if (st != SR_OK) return st;
  const float* ye = nullptr;
  if ((st = epilogue_y(plan, y, B, (cudaStream_t)stream, &ye)) != SR_OK) return st;
  return gd_iterations(*plan, ye, x, 0, iters, tau0, B, (cudaStream_t)stream,
                       [&](int t) { return loss_hist ? loss_hist + (size_t)t * B : nullptr; });
}

sr_status sr_gd_solve_early_stop(sr_plan* plan, const float* y, void* x, int max_iters, const sr_gd_opts* opts,
                                 float rel_tol, int check_every, float* loss_hist, int* iters_run, int B,
                                 void* stream) {
  if (!iters_run) return fail(SR_ERR_INVALID_ARG, "iters_run is NULL");
  *iters_run = 0;
  if (check_every < 2) return fail(SR_ERR_INVALID_ARG, "check_every must be >= 2");
  if (!(rel_tol >= 0.f && std::isfinite(rel_tol))) return fail(SR_ERR_INVALID_ARG, "rel_tol must be finite and >= 0");
  float mu0 = 0.f, tau0 = 0.f;
  sr_status st = gd_setup(plan, y, x, max_iters, opts, B, stream, &mu0, &tau0);
  if (st != SR_OK) return st;
  Plan& p = *plan;
  cudaStream_t s = (cudaStream_t)stream;
  const float* ye = nullptr;
  if ((st = epilogue_y(&p, y, B, s, &ye)) != SR_OK) return st;
  if (!p.d_es && (st = dalloc(&p.d_es, (size_t)2 * 65535)) != SR_OK) return st;
  std::vector<float> last(2 * (size_t)B);
  for (int t0 = 0; t0 < max_iters; t0 += check_every) {
    const int count = std::min(check_every, max_iters - t0);
    const int t1 = t0 + count;
    // the losses of the chunk's last two iterations go to d_es as well
    // (rows of loss_hist when it is given)
    st = gd_iterations(p, ye, x, t0, count, tau0, B, s, [&](int t) -> float* {
      if (loss_hist) return loss_hist + (size_t)t * B;
      return t >= t1 - 2 ? p.d_es + (size_t)(t - (t1 - 2)) * B : nullptr;
    });
    if (st != SR_OK) return st;
    *iters_run = t1;
    if (count < check_every || t1 >= max_iters) break;
    const float* rows = loss_hist ? loss_hist + (size_t)(t1 - 2) * B : p.d_es;
    SR_CUDA(cudaMemcpyAsync(last.data(), rows, last.size() * sizeof(float), cudaMemcpyDeviceToHost, s),
            "cudaMemcpyAsync(losses)");
    SR_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    bool all = true;
    for (int b = 0; b < B && all; ++b) {
      const double prev = last[b], cur = last[(size_t)B + b];
      all = std::fabs(prev - cur) <= (double)rel_tol * prev;
    }
    if (all) break;
  }
  return SR_OK;
}

sr_status sr_plan_check(sr_plan* plan) {
  if (!plan) return fail(SR_ERR_INVALID_ARG, "plan is NULL");
  sr_status st = check_device(plan);
  if (st != SR_OK) return st;
  SR_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  int code = 0;
  SR_CUDA(cudaMemcpy(&code, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy(status)");
  if (code != 0) {
    SR_CUDA(cudaMemset(plan->d_err, 0, sizeof(int)), "cudaMemset(status)");
    return fail((sr_status)code, "a device-side wait of a pass kernel gave up");
  }
  if (plan->inner) return sr_plan_check(static_cast<sr_plan*>(plan->inner));
  return SR_OK;
}

sr_status sr_plan_selftest_timeout(sr_plan* plan, void* stream) {
  if (!plan) return fail(SR_ERR_INVALID_ARG, "plan is NULL");
  sr_status st = check_device(plan);
  if (st != SR_OK) return st;
  SR_CUDA(sr::launch_wait_probe(plan->d_err, (cudaStream_t)stream), "launch(wait probe)");
  return SR_OK;
}

uint64_t sr_kernel_launches(void) {
  return sr::launches_so_far();
}

sr_status sr_plan_set_timing(sr_plan* plan, int enable) {
  if (!plan) return fail(SR_ERR_INVALID_ARG, "plan is NULL");
  plan->timing = enable != 0;
  return SR_OK;
}

sr_status sr_plan_get_timing(sr_plan* plan, double* ms, int64_t* count) {
  if (!plan) return fail(SR_ERR_INVALID_ARG, "plan is NULL");
  for (int k = 0; k < 3; ++k) {
    double total = 0.0;
    const size_t used = plan->ev_used[k];
    if (used) SR_CUDA(cudaEventSynchronize(plan->ev[k][used - 1]), "cudaEventSynchronize");
    for (size_t i = 0; i + 1 < used; i += 2) {
      float t = 0.f;
      SR_CUDA(cudaEventElapsedTime(&t, plan->ev[k][i], plan->ev[k][i + 1]), "cudaEventElapsedTime");
      total += t;
    }
    if (ms) ms[k] = total;
    if (count) count[k] = (int64_t)(used / 2);
    plan->ev_used[k] = 0;
  }
  return SR_OK;
}

sr_status sr_backward(sr_plan* plan, const void* x, const void* gz, void* grad_x, float* grad_theta, int B,
                      void* stream) {
  sr_status st = check_plan_call(plan, B);
  if (st != SR_OK) return st;
  if (!x || !gz) return fail(SR_ERR_INVALID_ARG, "NULL array argument");
  if (plan->two_d) return fail(SR_ERR_UNSUPPORTED, "the backward pass is not supported on 2D plans");
  if (plan->mo < plan->m) return fail(SR_ERR_UNSUPPORTED, "the backward pass is not supported for m < n");
  if (!grad_x && !grad_theta) return SR_OK;
  if ((st = ensure_backward_buffers(plan, B)) != SR_OK) return st;
  Plan& p = *plan;
  cudaStream_t s = (cudaStream_t)stream;
  const int L = p.L, n = (int)p.n, m = (int)p.m;
  float2* h = p.d_w0;  // gradient at p_l, carried with a factor sqrt(m)
  float2* q = p.d_w1;  // recomputed layer input q_l
  // h_L = F^H G_z (one inverse DFT, unnormalised: sqrt(m) F^H)
  {
    Chain c;
    c.nfft = 1;
    c.dir[0] = +1;
    c.xin = (const float2*)gz;
    c.n_in = m;
    c.xout = h;
    c.n_out = m;
    if ((st = run_chain(p, c, B, s)) != SR_OK) return st;
  }
  for (int l = L - 1; l >= 0; --l) {
    if (grad_theta) {
      const float2* ql = (const float2*)x;  // q_1 = U x
      int nq = n;
      if (l > 0) {
        // recompute q_l = F D_{l-1} ... F D_1 U x instead of storing it
        Chain c;
        c.nfft = l;
        for (int k = 0; k < l; ++k) c.dir[k] = -1;
        c.first_op = sr::kOpDiag;
        for (int k = 1; k < l; ++k) c.mid[k] = MidOp{sr::kOpDiag, k};
        c.xin = (const float2*)x;
        c.n_in = n;
        c.xout = q;
        c.n_out = m;
        if ((st = run_chain(p, c, B, s)) != SR_OK) return st;
        ql = q;
        nq = m;
      }
      SR_CUDA(sr::launch_theta_grad(ql, nq, p.d_dp + (size_t)l * m, h, m, B, grad_theta + (size_t)l * m, s),
              "launch(theta grad)");
    }
    if (l > 0) {
      // h_{l-1} = F^H D_l^H h_l (the input is consumed by the first pass before
      // the last pass overwrites it)
      Chain c;
      c.nfft = 1;
      c.dir[0] = +1;
      c.first_op = sr::kOpDiagConj;
      c.first_d = l;
      c.xin = h;
      c.n_in = m;
      c.xout = h;
      c.n_out = m;
      if ((st = run_chain(p, c, B, s)) != SR_OK) return st;
    }
  }
  if (grad_x) SR_CUDA(sr::launch_conj_diag_prune(h, p.d_dp, m, n, B, (float2*)grad_x, s), "launch(grad x)");
  return SR_OK;
}

const char* sr_status_string(sr_status status) {
  switch (status) {
    case SR_OK: return "ok";
    case SR_ERR_INVALID_ARG: return "invalid argument";
    case SR_ERR_UNSUPPORTED: return "unsupported size";
    case SR_ERR_OOM: return "out of memory";
    case SR_ERR_CUDA: return "CUDA error";
    case SR_ERR_TIMEOUT: return "device wait timed out";
    case SR_ERR_NUMERIC: return "numeric error";
  }
  return "unknown status";
}

const char* sr_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
