// Descriptors of the persistent ragged passes (ragged_pass.cu), shared with
// the ragged-batch orchestration (ragged.cu).
#pragma once

#include "sr_internal.h"

namespace sr {

// Pass kinds of a ragged launch (combined with the line-length class
// 0..3 = 128, 256, 512, 1024 points as variant = kind * 4 + class).
enum RaggedKind {
  kRgMidFF = 0,  // MID, forward -> forward (inside A)
  kRgMidFI = 1,  // MID, forward -> inverse (the epilogue between A and A^H)
  kRgMidII = 2,  // MID, inverse -> inverse (inside A^H)
  kRgLF = 3,     // LAST of a step fused with FIRST of the next
  kRgLast = 4,   // LAST of the final step
  kRgFirst = 5   // FIRST of the first step (k_ragged_first)
};

constexpr int kRgThreadsPerTile = 256;  // threads of a ragged-pass CTA

// One segment (bucket) of a ragged launch. `a` holds the bucket plan's pass
// arguments with the ragged tile geometry (T = 4096 / ell lines per tile);
// the per-call and per-step fields are filled in from RaggedDyn.
struct RaggedSeg {
  PassArgs a;
  int variant;        // kind * 4 + line-length class
  int kind;
  int tma;            // the input lines are staged by TMA
  int spec;           // power-iteration step (norm banks in use)
  int record_loss;    // GD: the step's loss goes to the loss history
  int slot0;          // the bucket's first slot (problem index in bucket order)
  int bsize;          // problems in the bucket
  int count_first;    // norm partials per problem of the start vector
  int count_steady;   // norm partials per problem written by a step
  int64_t x_off;      // offset of the bucket in the call's x (values)
  int64_t y_off;      // offset of the bucket in the call's y (values)
  float* bank[2];     // power iteration: norm-partial banks (ping-pong)
};

// Per-launch values.
struct RaggedDyn {
  const float2* x;       // concatenated x (FIRST input), or nullptr
  float2* xo;            // concatenated x (LAST / fused output), or nullptr
  const float* y;        // concatenated y
  float* loss_base;      // loss scratch: bucket with first slot s0 and B problems keeps its
                         // [iters][B] block at loss_base + iters * s0; or nullptr
  int iters, t;          // steps of the call and this step's index (loss rows)
  const float2* w1024;   // W_1024^k, k < 1024
  float mu_scale;        // warm-up factor of the step
  int parity;            // power iteration: the bank the step writes
  int first_step;        // power iteration: the input norm is the start vector's
  float lam;
  int weight_mode;
  float shift;
};

// Line-length class of a ragged segment (0..3), or -1 for lengths the ragged
// passes do not cover.
int ragged_class(int ell);
size_t ragged_smem_bytes();
// One problem of the ragged group, for the per-problem set-up and finish kernels.
struct RaggedProblem {
  int64_t x_off, y_off;  // offsets in the concatenated x and y (values)
  int n, m;
  int b, B;              // index in its bucket and the bucket's size
  float* scal;           // the bucket plan's scalars: sum(y) at [b], the GD step at [B + b]
  float* bank[2];        // the bucket plan's norm-partial banks (power iteration)
  float* sums;           // the bucket plan's bank of sum partials
  int count_steady;      // norm partials per problem written by a power-iteration step
};
// ----------------------------------------------------- queue-driven solve
// One launch runs a whole GD or power-iteration call over every problem of
// the group: work items (problem, pass, tile) are handed out by an atomic
// ticket in a fixed order; a tile of pass q of problem p starts once all
// tiles of pass q - 1 of p are done (a per-problem completion count).
constexpr int kRgMaxGroups = 64;

// One tile slot of a group's pass: everything a ticket decodes to, in one
// 32-byte record (one load).
struct alignas(32) RgTileRec {
  int p;        // problem index (completion counts)
  int b;        // index in its bucket
  int tile;     // tile within the pass
  int C;        // tiles per pass of the problem (m / 4096)
  int si0;      // the bucket's first descriptor (FIRST); pass k is si0 + k
  int L;        // layers
  int lgm;      // log2 m
  int lay;      // per layout (X: bits 0-7, Y: bits 8-15): line-length class | staged-by-TMA << 4
};

struct RgGroup {
  int ipq;      // tiles per pass of the whole group
  int rec0;     // the group's first record
};

struct RgSolveArgs {
  const RaggedSeg* segs;   // per bucket: FIRST, MID_1 .. MID_{2L-1}, fused LAST/FIRST, LAST
  const RgTileRec* rec;    // per group: ipq records, problem-major
  const RgGroup* grp;
  int ngrp;
  int T;                   // steps of the call (>= 1)
  float tau0;              // GD step warm-up: mu_t = mu0 (1 - exp(-(t+1)/tau0)) m / sum(y)
  int* done;               // per problem: completed tiles (zero at launch)
  unsigned* ticket;        // next work item (zero at launch); a launch deals < 2^31 tickets
};

// The queue-driven solve (one launch).
cudaError_t launch_ragged_solve(const RgSolveArgs& sa, const RaggedDyn& d, int grid, int* err, cudaStream_t s);
cudaError_t ragged_solve_occupancy(int* per_sm);

// The set-up and finish kernels split every problem into kRgChunks chunks.
constexpr int kRgChunks = 64;
// sum(y) and the GD step mu0 m / sum(y) (mu0 > 0) of every problem (two launches).
cudaError_t launch_ragged_prepare(const RaggedProblem* pr, int count, const float* y, float mu0, cudaStream_t s);
// Power-iteration start: x = v0 and ||v0||^2 as kRgChunks partials into bank[1].
cudaError_t launch_ragged_start(const RaggedProblem* pr, int count, const float2* v0, float2* x, cudaStream_t s);
// x = sqrt(sum y) v / ||v|| with ||v||^2 from bank[prev] (`first`: kRgChunks
// partials, else count_steady).
cudaError_t launch_ragged_finish(const RaggedProblem* pr, int count, float2* x, int prev, int first, cudaStream_t s);

}  // namespace sr
