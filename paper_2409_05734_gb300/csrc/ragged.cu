// Ragged batches of independent problems: buckets of equal (n, m, L), each a
// batched plan with per-problem phases. Buckets whose four-step geometry the
// queue-driven solve covers (power-of-two m from 2^14 to 2^20) form one group:
// a whole GD or power-iteration call runs as ONE launch over all of the
// group's problems (ragged_pass.cu), plus a few launches for the per-problem
// set-up and finish. The other buckets (short transforms,
// which the resident solver runs whole, radix-3 lengths, longer lines) run as
// concurrent stream branches that fork from and join into the caller's
// stream. Everything is graph-capturable.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "sr_internal.h"
#include "sr_ragged.h"

namespace {

sr_status rfail(sr_status st, const std::string& msg) {
  sr::set_last_error(msg);
  return st;
}

#define SR_RCUDA(call, what)                                                               \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      cudaGetLastError();                                                                  \
      return rfail(SR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_));      \
    }                                                                                      \
  } while (0)

struct Bucket {
  int64_t n = 0, m = 0;
  int L = 0;
  std::vector<int> members;  // caller indices, in slot order
  int slot0 = 0;             // first slot of the bucket
  int64_t x_base = 0, y_base = 0;
  sr_plan* plan = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool fused = false;         // runs in the persistent ragged passes
};

// The buckets that run in the persistent ragged passes, and the launch
// descriptors of every pass kind (built once at creation).
struct Fused {
  std::vector<int> buckets;
  int count = 0;                           // problems in the group
  sr::RaggedProblem* d_prob = nullptr;
  float2* d_w1024 = nullptr;
  int* d_err = nullptr;
  int num_sms = 1;
  // queue-driven solve: per bucket [FIRST, MID_1 .. MID_{2L-1}, LF, LAST] for
  // GD ([0]) and the power iteration ([1]), problems in group order, groups of
  // one L whose passes hold about group_tiles tiles (their data stays in L2)
  sr::RaggedSeg* d_qsegs[2] = {nullptr, nullptr};
  sr::RgTileRec* d_rec = nullptr;
  sr::RgGroup* d_grp = nullptr;
  int ngrp = 0;
  int* d_done = nullptr;
  unsigned* d_ticket = nullptr;
  int max_iters = 0;  // longest call of one launch (tickets < 2^31)
  int qgrid = 0;
  int group_tiles = 1024;
};

// loss[t][member[s]] = scratch[iters * slot0(s) + t * B(s) + (s - slot0(s))]
__global__ void k_scatter_loss(const float* __restrict__ scratch, const int* __restrict__ member,
                               const int* __restrict__ slot0, const int* __restrict__ bsize, int count, int iters,
                               float* __restrict__ loss) {
  const int64_t total = (int64_t)count * iters;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(i % count);
    const int t = (int)(i / count);
    const int s0 = slot0[s], bs = bsize[s];
    loss[(int64_t)t * count + member[s]] = scratch[(int64_t)iters * s0 + (int64_t)t * bs + (s - s0)];
  }
}

}  // namespace

struct sr_ragged {
  int count = 0;
  int device = 0;
  std::vector<int64_t> x_off, y_off;
  int64_t x_total = 0, y_total = 0;
  std::vector<Bucket> buckets;
  cudaEvent_t fork = nullptr;
  int iters_cap = 0;
  float* d_loss = nullptr;   // [iters_cap * count] scratch
  int* d_member = nullptr;   // [count] per slot
  int* d_slot0 = nullptr;
  int* d_bsize = nullptr;
  Fused fz;
};

namespace {

// Runs fn(bucket) on every bucket's stream between a fork from and a join into
// `s` (with skip_fused, on the buckets outside the persistent-pass group only),
// and pre() on `s` itself between the fork and the join, so that the branches
// overlap the group's work. The branches are launched first: their kernels use
// few CTAs each and run for the whole call, while the group's persistent grid
// takes its work from a queue, so CTAs of it that find no room start later
// and still share the work.
template <class F, class G>
sr_status run_buckets(sr_ragged* r, cudaStream_t s, F fn, bool skip_fused, G pre) {
  SR_RCUDA(cudaEventRecord(r->fork, s), "cudaEventRecord(fork)");
  for (Bucket& b : r->buckets) {
    if (skip_fused && b.fused) continue;
    SR_RCUDA(cudaStreamWaitEvent(b.stream, r->fork, 0), "cudaStreamWaitEvent(fork)");
    sr_status st = fn(b);
    if (st != SR_OK) return st;
    SR_RCUDA(cudaEventRecord(b.done, b.stream), "cudaEventRecord(join)");
  }
  sr_status st0 = pre();
  if (st0 != SR_OK) return st0;
  for (Bucket& b : r->buckets) {
    if (skip_fused && b.fused) continue;
    SR_RCUDA(cudaStreamWaitEvent(s, b.done, 0), "cudaStreamWaitEvent(join)");
  }
  return SR_OK;
}

template <class F>
sr_status run_buckets(sr_ragged* r, cudaStream_t s, F fn) {
  return run_buckets(r, s, fn, false, []() { return SR_OK; });
}

// ------------------------------------------------------- persistent passes

constexpr double kTwoPiR = 6.283185307179586476925286766559;

// Whether a bucket's plan can run in the persistent ragged passes: a 1D
// power-of-two plan whose two line lengths are 128 .. 1024 points.
bool fusable(const sr_plan* pl) {
  const sr::Plan& p = *reinterpret_cast<const sr::Plan*>(pl);
  if (p.inner || p.two_d || p.mo < p.m || p.m < (1 << 14) || p.m > (1 << 20)) return false;
  for (int lay = 0; lay < 2; ++lay)
    if (sr::ragged_class(p.geom[lay].ell) < 0) return false;
  return true;
}

// Pass arguments of a bucket plan common to every pass, with the ragged tile
// geometry of layout `lay` (tiles of 4096 values: T = 4096 / ell lines).
sr::PassArgs seg_base(const sr::Plan& p, sr::Layout lay, int B, int* err) {
  sr::PassArgs a;
  std::memset(&a, 0, sizeof(a));
  a.m = (int)p.m;
  a.dp_stride = p.dp_stride;
  a.twl = p.d_twl;
  a.tw_hi = p.d_tw_hi;
  a.tw_lo = p.d_tw_lo;
  a.tw_shift = p.tw_shift;
  a.err = err;
  const int ell = p.geom[lay].ell;
  a.ell = ell;
  a.T = 4096 / ell;
  a.lgT = 0;
  while ((1 << a.lgT) < a.T) ++a.lgT;
  a.nl = (int)(p.m / ell);
  a.cpp = a.nl / a.T;
  a.ntiles = B * a.cpp;
  a.tws = p.lmax / ell;
  return a;
}

// The descriptor of bucket `bk`'s pass of kind `kind` (MID index k for the
// middle passes) in a GD step (spec = 0) or a power-iteration step (spec = 1):
// the arguments run_chain would pass for the round trip A^H (epilogue) A of
// the bucket's plan, with the tile geometry of the ragged passes.
sr::RaggedSeg make_seg(const Bucket& bk, int kind, int k, int spec, int* err) {
  const sr::Plan& p = *reinterpret_cast<const sr::Plan*>(bk.plan);
  const int B = (int)bk.members.size(), L = p.L;
  sr::RaggedSeg g;
  std::memset(&g, 0, sizeof(g));
  sr::Layout lay = sr::kLayoutX;
  if (kind != sr::kRgFirst && kind != sr::kRgLF && kind != sr::kRgLast) lay = sr::s2_layout((k - 1) % 2);
  g.a = seg_base(p, lay, B, err);
  sr::PassArgs& a = g.a;
  g.kind = kind;
  g.x_off = bk.x_base;
  g.y_off = bk.y_base;
  g.slot0 = bk.slot0;
  g.bsize = B;
  // staged by TMA: the passes that read exchange-buffer rows (not FIRST, whose
  // input is the natural-order signal), with the plan's row tensor map
  g.tma = kind != sr::kRgFirst && a.ell <= 512 && p.geom[lay].T == a.T;
  const float* loss_part = sr::plan_part_bank(p, 2, B);
  const sr::Layout lay_epi = sr::s2_layout((L - 1) % 2);
  const int epi_cpp = (int)(p.m / p.geom[lay_epi].ell) / (4096 / p.geom[lay_epi].ell);
  if (kind == sr::kRgFirst) {
    a.out_dir = -1;
    a.n_in = (int)p.n;
    a.op = sr::kOpDiag;  // D_1
    a.dp = p.d_dp;
    a.eout = p.d_e0;
  } else if (kind == sr::kRgLF || kind == sr::kRgLast) {
    // after 2L - 1 middle passes the step's data is in e1
    a.in_dir = 1;
    a.ein = p.d_e1;
    a.tmap = p.tmap[1][lay];
    a.dp = p.d_dp;  // D_1 (conjugated for the update, then again for the next FIRST)
    a.op = kind == sr::kRgLast ? sr::kOpDiagConj : sr::kOpNone;
    a.eout = p.d_e0;
    a.n_out = (int)p.n;
    a.loss_part = loss_part;
    a.loss_cpp = epi_cpp * (sr::kRgThreadsPerTile / 32);
    if (spec) {
      a.out_mode = sr::kOutSpec;
      g.spec = 1;
    } else {
      a.out_mode = sr::kOutGd;
      a.mu = p.d_scal + B;
      g.record_loss = 1;
    }
  } else {
    // middle pass k: step 2 of DFT k-1, the operation, step 1 of DFT k
    const int da = (k - 1) < L ? -1 : 1, db = k < L ? -1 : 1;
    g.kind = da < 0 ? (db < 0 ? sr::kRgMidFF : sr::kRgMidFI) : sr::kRgMidII;
    const int src = (k % 2 == 1) ? 0 : 1;  // FIRST / fused passes write e0, then the buffers alternate
    a.in_dir = da;
    a.out_dir = db;
    a.ein = src ? p.d_e1 : p.d_e0;
    a.eout = src ? p.d_e0 : p.d_e1;
    a.tmap = p.tmap[src][lay];
    if (k != L) {
      const int d = k < L ? k : 2 * L - k;
      a.op = k < L ? sr::kOpDiag : sr::kOpDiagConj;
      a.dp = p.d_dp + (size_t)d * p.m;
      a.ph = p.d_ph + (size_t)d * p.m;
      a.dscale = (float)(1.0 / std::sqrt((double)p.m));
    } else if (spec) {
      a.op = sr::kOpSpecEpilogue;
      a.sumy = p.d_scal;
      g.spec = 1;
    } else {
      a.op = sr::kOpGdEpilogue;
      a.part_out = const_cast<float*>(loss_part);
    }
  }
  if (g.spec) {
    g.bank[0] = sr::plan_part_bank(p, 0, B);
    g.bank[1] = sr::plan_part_bank(p, 1, B);
    g.count_first = sr::kRgChunks;
    g.count_steady = seg_base(p, sr::kLayoutX, B, err).cpp;
  }
  g.variant = g.kind * 4 + sr::ragged_class(a.ell);
  return g;
}

void free_fused(Fused& f) {
  for (int k = 0; k < 2; ++k) cudaFree(f.d_qsegs[k]);
  cudaFree(f.d_rec);
  cudaFree(f.d_grp);
  cudaFree(f.d_done);
  cudaFree(f.d_ticket);
  cudaFree(f.d_prob);
  cudaFree(f.d_w1024);
  cudaFree(f.d_err);
  f = Fused();
}

// Line-length class and TMA staging of layout `lay` of a bucket's ragged
// tiles, packed as in RgTileRec::lay.
int lay_code(const sr::Plan& p, sr::Layout lay) {
  const int ell = p.geom[lay].ell;
  const int tma = ell <= 512 && p.geom[lay].T == 4096 / ell;
  return sr::ragged_class(ell) | (tma << 4);
}

// The queue-driven solve's tables: every fused bucket's descriptors in pass
// order, and the problems in groups of one L of about f.group_tiles tiles per
// pass (a group's exchange buffers, phases and measurements then fit in L2
// while its passes run), as one record per tile slot of a group's pass.
sr_status build_queue(sr_ragged* r) {
  Fused& f = r->fz;
  std::vector<sr::RaggedSeg> segs[2];
  std::vector<int> base(r->buckets.size(), 0);
  for (int bi : f.buckets) {
    const Bucket& bk = r->buckets[bi];
    base[bi] = (int)segs[0].size();
    for (int spec = 0; spec < 2; ++spec) {
      segs[spec].push_back(make_seg(bk, sr::kRgFirst, 0, spec, f.d_err));
      for (int k = 1; k <= 2 * bk.L - 1; ++k) segs[spec].push_back(make_seg(bk, sr::kRgMidFF, k, spec, f.d_err));
      segs[spec].push_back(make_seg(bk, sr::kRgLF, 0, spec, f.d_err));
      segs[spec].push_back(make_seg(bk, sr::kRgLast, 0, spec, f.d_err));
    }
  }
  // problems by L (a group has one L), buckets kept together; the group size
  // grows until the groups fit the kernel's table
  std::vector<int> order(f.buckets.begin(), f.buckets.end());
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return r->buckets[a].L < r->buckets[b].L; });
  std::vector<sr::RgTileRec> rec;
  std::vector<sr::RgGroup> grp;
  for (;;) {
    rec.clear();
    grp.clear();
    int gL = -1, p = 0;
    for (int bi : order) {
      const Bucket& bk = r->buckets[bi];
      const sr::Plan& pl = *reinterpret_cast<const sr::Plan*>(bk.plan);
      const int C = (int)(bk.m / 4096);
      int lgm = 0;
      while ((1ll << lgm) < bk.m) ++lgm;
      const int lay = lay_code(pl, sr::kLayoutX) | (lay_code(pl, sr::kLayoutY) << 8);
      for (int j = 0; j < (int)bk.members.size(); ++j, ++p) {
        if (grp.empty() || gL != bk.L || grp.back().ipq + C > f.group_tiles) {
          sr::RgGroup g;
          g.ipq = 0;
          g.rec0 = (int)rec.size();
          grp.push_back(g);
          gL = bk.L;
        }
        for (int c = 0; c < C; ++c) {
          sr::RgTileRec q;
          q.p = p;
          q.b = j;
          q.tile = c;
          q.C = C;
          q.si0 = base[bi];
          q.L = bk.L;
          q.lgm = lgm;
          q.lay = lay;
          rec.push_back(q);
        }
        grp.back().ipq += C;
      }
    }
    if ((int)grp.size() <= sr::kRgMaxGroups) break;
    f.group_tiles *= 2;
  }
  // tickets of the longest call the tables can deal in one launch (< 2^31)
  int64_t per_step = 0, first = 0;
  for (size_t g = 0; g < grp.size(); ++g) {
    const int L = rec[grp[g].rec0].L;
    per_step += 2 * L * (int64_t)grp[g].ipq;
    first += grp[g].ipq;
  }
  f.max_iters = (int)std::min<int64_t>(INT32_MAX, ((int64_t)INT32_MAX - first) / std::max<int64_t>(1, per_step));
  f.ngrp = (int)grp.size();
  for (int k = 0; k < 2; ++k) {
    SR_RCUDA(cudaMalloc(&f.d_qsegs[k], sizeof(sr::RaggedSeg) * segs[k].size()), "cudaMalloc(queue descriptors)");
    SR_RCUDA(cudaMemcpy(f.d_qsegs[k], segs[k].data(), sizeof(sr::RaggedSeg) * segs[k].size(), cudaMemcpyHostToDevice),
             "cudaMemcpy(queue descriptors)");
  }
  SR_RCUDA(cudaMalloc(&f.d_rec, sizeof(sr::RgTileRec) * rec.size()), "cudaMalloc(queue records)");
  SR_RCUDA(cudaMemcpy(f.d_rec, rec.data(), sizeof(sr::RgTileRec) * rec.size(), cudaMemcpyHostToDevice),
           "cudaMemcpy(queue records)");
  SR_RCUDA(cudaMalloc(&f.d_grp, sizeof(sr::RgGroup) * grp.size()), "cudaMalloc(queue groups)");
  SR_RCUDA(cudaMemcpy(f.d_grp, grp.data(), sizeof(sr::RgGroup) * grp.size(), cudaMemcpyHostToDevice),
           "cudaMemcpy(queue groups)");
  SR_RCUDA(cudaMalloc(&f.d_done, sizeof(int) * f.count), "cudaMalloc(completion counts)");
  SR_RCUDA(cudaMalloc(&f.d_ticket, sizeof(unsigned)), "cudaMalloc(ticket)");
  int occ = 1;
  SR_RCUDA(sr::ragged_solve_occupancy(&occ), "ragged solve occupancy");
  f.qgrid = occ * f.num_sms;
  return SR_OK;
}

// One queue-driven launch running `iters` steps (GD: spec = 0; power
// iteration: spec = 1) of every problem of the group, after the completion
// counts and the ticket are cleared.
sr_status fused_queue(const Fused& f, int spec, int iters, float tau0, const sr::RaggedDyn& d, cudaStream_t s) {
  if (iters > f.max_iters) return rfail(SR_ERR_UNSUPPORTED, "too many steps for one call of this ragged batch");
  SR_RCUDA(cudaMemsetAsync(f.d_done, 0, sizeof(int) * f.count, s), "cudaMemsetAsync(completion counts)");
  SR_RCUDA(cudaMemsetAsync(f.d_ticket, 0, sizeof(unsigned), s), "cudaMemsetAsync(ticket)");
  sr::RgSolveArgs sa;
  std::memset(&sa, 0, sizeof(sa));
  sa.segs = f.d_qsegs[spec];
  sa.rec = f.d_rec;
  sa.grp = f.d_grp;
  sa.ngrp = f.ngrp;
  sa.T = iters;
  sa.tau0 = tau0;
  sa.done = f.d_done;
  sa.ticket = f.d_ticket;
  SR_RCUDA(sr::launch_ragged_solve(sa, d, f.qgrid, f.d_err, s), "launch(ragged solve)");
  return SR_OK;
}

// Builds the queue-driven group: every fusable bucket, the per-problem table of
// the set-up and finish kernels, the W_1024 line-twiddle table and the queue's
// tables (build_queue).
sr_status build_fused(sr_ragged* r) {
  Fused& f = r->fz;
  for (size_t i = 0; i < r->buckets.size(); ++i) {
    if (!fusable(r->buckets[i].plan)) continue;
    r->buckets[i].fused = true;
    f.buckets.push_back((int)i);
  }
  if (f.buckets.empty()) return SR_OK;
  SR_RCUDA(cudaMalloc(&f.d_err, sizeof(int)), "cudaMalloc(ragged status)");
  SR_RCUDA(cudaMemset(f.d_err, 0, sizeof(int)), "cudaMemset(ragged status)");
  std::vector<sr::RaggedProblem> prob;
  for (int bi : f.buckets) {
    const Bucket& bk = r->buckets[bi];
    const sr::Plan& p = *reinterpret_cast<const sr::Plan*>(bk.plan);
    const int B = (int)bk.members.size();
    for (int j = 0; j < B; ++j) {
      sr::RaggedProblem q;
      std::memset(&q, 0, sizeof(q));
      q.x_off = bk.x_base + (int64_t)j * bk.n;
      q.y_off = bk.y_base + (int64_t)j * bk.m;
      q.n = (int)bk.n;
      q.m = (int)bk.m;
      q.b = j;
      q.B = B;
      q.scal = p.d_scal;
      q.bank[0] = sr::plan_part_bank(p, 0, B);
      q.bank[1] = sr::plan_part_bank(p, 1, B);
      q.sums = sr::plan_part_bank(p, 3, B);
      q.count_steady = seg_base(p, sr::kLayoutX, B, f.d_err).cpp;
      prob.push_back(q);
    }
  }
  f.count = (int)prob.size();
  std::vector<float2> w(1024);
  for (int k = 0; k < 1024; ++k) {
    const double ang = -kTwoPiR * (double)k / 1024.0;
    w[k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  SR_RCUDA(cudaMalloc(&f.d_prob, sizeof(sr::RaggedProblem) * prob.size()), "cudaMalloc(ragged problems)");
  SR_RCUDA(cudaMemcpy(f.d_prob, prob.data(), sizeof(sr::RaggedProblem) * prob.size(), cudaMemcpyHostToDevice),
           "cudaMemcpy(ragged problems)");
  SR_RCUDA(cudaMalloc(&f.d_w1024, sizeof(float2) * 1024), "cudaMalloc(line twiddles)");
  SR_RCUDA(cudaMemcpy(f.d_w1024, w.data(), sizeof(float2) * 1024, cudaMemcpyHostToDevice), "cudaMemcpy(line twiddles)");
  SR_RCUDA(cudaDeviceGetAttribute(&f.num_sms, cudaDevAttrMultiProcessorCount, r->device), "device attributes");
  return build_queue(r);
}

// `iters` GD steps on every problem of the group (Sec. II-B-1): one
// queue-driven launch after the per-problem set-up.
sr_status fused_gd(sr_ragged* r, const float* y, float2* x, int iters, float mu0, float tau0, float* loss_scratch,
                   cudaStream_t s) {
  const Fused& f = r->fz;
  if (f.buckets.empty()) return SR_OK;
  SR_RCUDA(sr::launch_ragged_prepare(f.d_prob, f.count, y, mu0, s), "launch(ragged prepare)");
  if (iters == 0) return SR_OK;
  sr::RaggedDyn d;
  std::memset(&d, 0, sizeof(d));
  d.x = x;
  d.xo = x;
  d.y = y;
  d.w1024 = f.d_w1024;
  d.loss_base = loss_scratch;
  d.iters = iters;
  return fused_queue(f, 0, iters, tau0, d, s);
}

// `iters` power-iteration steps (Sec. II-B-2, Eq. 3-4) on every problem of the
// group, from x = v0, ending with x = sqrt(sum y) v / ||v||.
sr_status fused_spectral(sr_ragged* r, const float* y, const float2* v0, float2* x, int iters,
                         const sr_spectral_opts& o, cudaStream_t s) {
  const Fused& f = r->fz;
  if (f.buckets.empty()) return SR_OK;
  SR_RCUDA(sr::launch_ragged_prepare(f.d_prob, f.count, y, 0.f, s), "launch(ragged prepare)");
  SR_RCUDA(sr::launch_ragged_start(f.d_prob, f.count, v0, x, s), "launch(ragged start)");
  sr::RaggedDyn d;
  std::memset(&d, 0, sizeof(d));
  d.x = x;
  d.xo = x;
  d.y = y;
  d.w1024 = f.d_w1024;
  d.lam = o.lambda;
  d.weight_mode = o.weight_mode;
  d.shift = o.weight_mode == SR_WEIGHT_IDENTITY ? 0.f : -2.0f * o.lambda;
  sr_status st;
  if (iters > 0 && (st = fused_queue(f, 1, iters, 0.f, d, s)) != SR_OK) return st;
  const int prev = iters == 0 ? 1 : (iters - 1) % 2;
  SR_RCUDA(sr::launch_ragged_finish(f.d_prob, f.count, x, prev, iters == 0, s), "launch(ragged finish)");
  return SR_OK;
}

sr_status check_ragged(sr_ragged* r) {
  if (!r) return rfail(SR_ERR_INVALID_ARG, "ragged handle is NULL");
  int dev = -1;
  SR_RCUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != r->device) return rfail(SR_ERR_INVALID_ARG, "current CUDA device differs from the handle's device");
  return SR_OK;
}

}  // namespace

extern "C" {

sr_status sr_ragged_destroy(sr_ragged* r) {
  if (!r) return SR_OK;
  for (Bucket& b : r->buckets) {
    sr_plan_destroy(b.plan);
    if (b.stream) cudaStreamDestroy(b.stream);
    if (b.done) cudaEventDestroy(b.done);
  }
  if (r->fork) cudaEventDestroy(r->fork);
  free_fused(r->fz);
  cudaFree(r->d_loss);
  cudaFree(r->d_member);
  cudaFree(r->d_slot0);
  cudaFree(r->d_bsize);
  delete r;
  return SR_OK;
}

sr_status sr_ragged_create(int count, const int64_t* n, const int64_t* m, const int* L, const uint64_t* seeds,
                           int autotune, sr_ragged** out) {
  if (!out || !n || !m || !L || !seeds) return rfail(SR_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (count < 1) return rfail(SR_ERR_INVALID_ARG, "count must be >= 1");
  for (int i = 0; i < count; ++i)
    if (n[i] > m[i]) return rfail(SR_ERR_UNSUPPORTED, "ragged batches need n <= m (alpha >= 1)");
  sr_ragged* r = new (std::nothrow) sr_ragged();
  if (!r) return rfail(SR_ERR_OOM, "host allocation failed");
  r->count = count;
  if (cudaGetDevice(&r->device) != cudaSuccess) {
    delete r;
    return rfail(SR_ERR_CUDA, "cudaGetDevice");
  }
  // buckets of equal shape, largest work first
  std::map<std::tuple<int64_t, int64_t, int>, std::vector<int>> by_shape;
  for (int i = 0; i < count; ++i) by_shape[std::make_tuple(n[i], m[i], L[i])].push_back(i);
  for (auto& kv : by_shape) {
    Bucket b;
    std::tie(b.n, b.m, b.L) = kv.first;
    b.members = kv.second;
    r->buckets.push_back(b);
  }
  std::stable_sort(r->buckets.begin(), r->buckets.end(), [](const Bucket& a, const Bucket& b) {
    return (double)a.m * a.L * a.members.size() > (double)b.m * b.L * b.members.size();
  });
  r->x_off.assign(count, 0);
  r->y_off.assign(count, 0);
  std::vector<int> member, slot0, bsize;
  int slot = 0;
  for (Bucket& b : r->buckets) {
    b.slot0 = slot;
    b.x_base = r->x_total;
    b.y_base = r->y_total;
    for (size_t j = 0; j < b.members.size(); ++j) {
      const int i = b.members[j];
      r->x_off[i] = b.x_base + (int64_t)j * b.n;
      r->y_off[i] = b.y_base + (int64_t)j * b.m;
      member.push_back(i);
      slot0.push_back(b.slot0);
      bsize.push_back((int)b.members.size());
    }
    slot += (int)b.members.size();
    r->x_total += (int64_t)b.members.size() * b.n;
    r->y_total += (int64_t)b.members.size() * b.m;
  }
  sr_status st = SR_OK;
  for (Bucket& b : r->buckets) {
    const int B = (int)b.members.size();
    std::vector<uint64_t> sd(B);
    for (int j = 0; j < B; ++j) sd[j] = seeds[b.members[j]];
    if ((st = sr_plan_create(b.n, b.m, b.L, sd[0], &b.plan)) != SR_OK ||
        (st = sr::plan_set_problem_phases(b.plan, B, sd.data())) != SR_OK ||
        (st = sr_plan_reserve(b.plan, B)) != SR_OK) {
      sr_ragged_destroy(r);
      return st;
    }
    if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess) {
      sr_ragged_destroy(r);
      return rfail(SR_ERR_CUDA, "stream or event creation failed");
    }
    // (buckets of the queue-driven group run on that group's own tile
    // geometry and grid, so only the others are tuned; tuning must not move a
    // bucket out of the group by choosing a split the group does not cover)
    if (autotune && !fusable(b.plan) && (st = sr_plan_autotune(b.plan, B, b.stream)) != SR_OK) {
      sr_ragged_destroy(r);
      return st;
    }
  }
  cudaError_t e = cudaEventCreateWithFlags(&r->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&r->d_member, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMalloc(&r->d_slot0, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMalloc(&r->d_bsize, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMemcpy(r->d_member, member.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r->d_slot0, slot0.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r->d_bsize, bsize.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    sr_ragged_destroy(r);
    return rfail(SR_ERR_CUDA, std::string("ragged setup: ") + cudaGetErrorString(e));
  }
  if ((st = build_fused(r)) != SR_OK) {
    sr_ragged_destroy(r);
    return st;
  }
  *out = r;
  return SR_OK;
}

sr_status sr_ragged_layout(const sr_ragged* r, int64_t* x_off, int64_t* y_off, int64_t* x_total, int64_t* y_total,
                           int* buckets) {
  if (!r) return rfail(SR_ERR_INVALID_ARG, "ragged handle is NULL");
  if (x_off) std::copy(r->x_off.begin(), r->x_off.end(), x_off);
  if (y_off) std::copy(r->y_off.begin(), r->y_off.end(), y_off);
  if (x_total) *x_total = r->x_total;
  if (y_total) *y_total = r->y_total;
  if (buckets) *buckets = (int)r->buckets.size();
  return SR_OK;
}

sr_status sr_ragged_reserve(sr_ragged* r, int iters) {
  sr_status st = check_ragged(r);
  if (st != SR_OK) return st;
  if (iters <= r->iters_cap) return SR_OK;
  cudaFree(r->d_loss);
  r->d_loss = nullptr;
  r->iters_cap = 0;
  SR_RCUDA(cudaMalloc(&r->d_loss, sizeof(float) * (size_t)iters * r->count), "cudaMalloc(loss scratch)");
  r->iters_cap = iters;
  return SR_OK;
}

sr_status sr_ragged_forward(sr_ragged* r, const void* x_cat, void* z_cat, void* stream) {
  sr_status st = check_ragged(r);
  if (st != SR_OK) return st;
  if (!x_cat || !z_cat) return rfail(SR_ERR_INVALID_ARG, "NULL array argument");
  const float2* x = static_cast<const float2*>(x_cat);
  float2* z = static_cast<float2*>(z_cat);
  return run_buckets(r, (cudaStream_t)stream, [&](Bucket& b) {
    return sr_forward(b.plan, x + b.x_base, z + b.y_base, (int)b.members.size(), b.stream);
  });
}

sr_status sr_ragged_spectral_init(sr_ragged* r, const float* y_cat, const void* v0_cat, int iters,
                                  const sr_spectral_opts* opts, void* x_cat, void* stream) {
  sr_status st = check_ragged(r);
  if (st != SR_OK) return st;
  if (!y_cat || !v0_cat || !x_cat) return rfail(SR_ERR_INVALID_ARG, "NULL array argument");
  if (iters < 0) return rfail(SR_ERR_INVALID_ARG, "iters must be >= 0");
  sr_spectral_opts o{SR_WEIGHT_OPTIMAL, -1.0f};
  if (opts) o = *opts;
  if (o.weight_mode != SR_WEIGHT_IDENTITY && o.weight_mode != SR_WEIGHT_OPTIMAL)
    return rfail(SR_ERR_INVALID_ARG, "unknown weight_mode");
  if (o.weight_mode == SR_WEIGHT_OPTIMAL && !(o.lambda < 0.f && std::isfinite(o.lambda)))
    return rfail(SR_ERR_INVALID_ARG, "lambda must be finite and < 0");
  const float2* v0 = static_cast<const float2*>(v0_cat);
  float2* x = static_cast<float2*>(x_cat);
  cudaStream_t s = (cudaStream_t)stream;
  return run_buckets(
      r, s,
      [&](Bucket& b) {
        return sr_spectral_init(b.plan, y_cat + b.y_base, v0 + b.x_base, iters, &o, x + b.x_base,
                                (int)b.members.size(), b.stream);
      },
      true, [&]() { return fused_spectral(r, y_cat, v0, x, iters, o, s); });
}

sr_status sr_ragged_gd_solve(sr_ragged* r, const float* y_cat, void* x_cat, int iters, const sr_gd_opts* opts,
                             float* loss_hist, void* stream) {
  sr_status st = check_ragged(r);
  if (st != SR_OK) return st;
  if (!y_cat || !x_cat) return rfail(SR_ERR_INVALID_ARG, "NULL array argument");
  if (iters < 0) return rfail(SR_ERR_INVALID_ARG, "iters must be >= 0");
  if (loss_hist && iters > r->iters_cap)
    return rfail(SR_ERR_INVALID_ARG, "loss history needs sr_ragged_reserve(iters) first");
  const float mu0 = opts ? opts->mu0 : 0.1f;
  const float tau0 = opts ? opts->tau0 : 0.f;
  if (!(mu0 > 0.f && std::isfinite(mu0))) return rfail(SR_ERR_INVALID_ARG, "mu0 must be finite and > 0");
  if (!(tau0 >= 0.f && std::isfinite(tau0))) return rfail(SR_ERR_INVALID_ARG, "tau0 must be finite and >= 0");
  float2* x = static_cast<float2*>(x_cat);
  cudaStream_t s = (cudaStream_t)stream;
  st = run_buckets(
      r, s,
      [&](Bucket& b) {
        float* lh = loss_hist ? r->d_loss + (size_t)iters * b.slot0 : nullptr;
        return sr_gd_solve(b.plan, y_cat + b.y_base, x + b.x_base, iters, opts, lh, (int)b.members.size(),
                           b.stream);
      },
      true, [&]() { return fused_gd(r, y_cat, x, iters, mu0, tau0, loss_hist ? r->d_loss : nullptr, s); });
  if (st != SR_OK || !loss_hist || iters == 0) return st;
  const int64_t total = (int64_t)iters * r->count;
  const int blocks = (int)std::min<int64_t>(1024, (total + 255) / 256);
  k_scatter_loss<<<blocks, 256, 0, s>>>(r->d_loss, r->d_member, r->d_slot0, r->d_bsize, r->count, iters, loss_hist);
  sr::count_launch();
  SR_RCUDA(cudaGetLastError(), "launch(scatter loss)");
  return SR_OK;
}

sr_status sr_ragged_selftest_timeout(sr_ragged* r, void* stream) {
  sr_status st = check_ragged(r);
  if (st != SR_OK) return st;
  const Fused& f = r->fz;
  if (f.buckets.empty()) return rfail(SR_ERR_UNSUPPORTED, "the batch has no problems in the queue-driven solve");
  cudaStream_t s = (cudaStream_t)stream;
  // scratch inputs for the FIRST tiles (which need nothing and run normally)
  float2* x = nullptr;
  float* y = nullptr;
  SR_RCUDA(cudaMalloc(&x, sizeof(float2) * (size_t)std::max<int64_t>(1, r->x_total)), "cudaMalloc(selftest x)");
  cudaError_t e = cudaMalloc(&y, sizeof(float) * (size_t)std::max<int64_t>(1, r->y_total));
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, sizeof(float2) * (size_t)std::max<int64_t>(1, r->x_total), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(y, 0, sizeof(float) * (size_t)std::max<int64_t>(1, r->y_total), s);
  // every completion count starts far below zero, so no tile after FIRST
  // ever sees its inputs complete: each such wait gives up after the
  // library's limit, records SR_ERR_TIMEOUT and its CTA returns
  if (e == cudaSuccess) e = cudaMemsetAsync(f.d_done, 0x80, sizeof(int) * f.count, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(f.d_ticket, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    sr::RgSolveArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.segs = f.d_qsegs[0];
    sa.rec = f.d_rec;
    sa.grp = f.d_grp;
    sa.ngrp = f.ngrp;
    sa.T = 1;
    sa.done = f.d_done;
    sa.ticket = f.d_ticket;
    sr::RaggedDyn d;
    std::memset(&d, 0, sizeof(d));
    d.x = x;
    d.xo = x;
    d.y = y;
    d.w1024 = f.d_w1024;
    d.iters = 1;
    e = sr::launch_ragged_solve(sa, d, f.qgrid, f.d_err, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(x);
  cudaFree(y);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return rfail(SR_ERR_CUDA, std::string("ragged selftest: ") + cudaGetErrorString(e));
  }
  return SR_OK;
}

sr_status sr_ragged_check(sr_ragged* r) {
  sr_status st = check_ragged(r);
  if (st != SR_OK) return st;
  for (Bucket& b : r->buckets)
    if ((st = sr_plan_check(b.plan)) != SR_OK) return st;
  if (r->fz.d_err) {
    int h = 0;
    SR_RCUDA(cudaMemcpy(&h, r->fz.d_err, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy(ragged status)");
    if (h != 0) {
      SR_RCUDA(cudaMemset(r->fz.d_err, 0, sizeof(int)), "cudaMemset(ragged status)");
      return rfail((sr_status)h, "a persistent ragged pass gave up waiting for its input tile");
    }
  }
  return SR_OK;
}

}  // extern "C"
