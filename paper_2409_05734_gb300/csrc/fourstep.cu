// Launchers of the four-step pass kernels (passes.cuh) and the helper kernels
// of the solvers (Sec. II-B): per-problem sums, norms and scalings.
#include <algorithm>
#include <atomic>

#include "passes.cuh"

namespace sr {

std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------------ helpers

// part[b*chunks + c] = compensated sum of chunk c of row b.
__global__ void k_sum_rows(const float* __restrict__ y, int m, float* __restrict__ part, int chunks) {
  __shared__ float red[64];
  const int b = blockIdx.y, c = blockIdx.x;
  const int len = (m + chunks - 1) / chunks;
  const int lo = c * len, hi = min(m, lo + len);
  const float* yb = y + (size_t)b * m;
  fsum2 acc{0.f, 0.f};
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) acc_add(acc, yb[i]);
  const float s = block_sum(acc, red);
  if (threadIdx.x == 0) part[(size_t)b * chunks + c] = s;
}

__global__ void k_norm_rows(const float2* __restrict__ v, int n, float* __restrict__ part, int chunks) {
  __shared__ float red[64];
  const int b = blockIdx.y, c = blockIdx.x;
  const int len = (n + chunks - 1) / chunks;
  const int lo = c * len, hi = min(n, lo + len);
  const float2* vb = v + (size_t)b * n;
  fsum2 acc{0.f, 0.f};
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) acc_add(acc, cabs2(vb[i]));
  const float s = block_sum(acc, red);
  if (threadIdx.x == 0) part[(size_t)b * chunks + c] = s;
}

__global__ void k_finish_scalars(const float* __restrict__ part, int chunks, int B, float mu0, int m,
                                 float* __restrict__ sumy, float* __restrict__ mu) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float s = sum_partials(part + (size_t)b * chunks, chunks);
  sumy[b] = s;
  if (mu) mu[b] = mu0 * (float)m / s;
}

// v[b] *= sqrt(sumy[b]) / ||v[b]|| with ||v||^2 the sum of `chunks` partials.
__global__ void k_scale_rows(float2* __restrict__ v, int n, const float* __restrict__ part, int chunks,
                             const float* __restrict__ sumy) {
  __shared__ float s_f;
  const int b = blockIdx.y;
  if (threadIdx.x == 0) s_f = sqrtf(sumy[b]) / sqrtf(sum_partials(part + (size_t)b * chunks, chunks));
  __syncthreads();
  const float f = s_f;
  float2* vb = v + (size_t)b * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) vb[i] = cscale(vb[i], f);
}

// D_l[k] = exp(i theta_l[k]) / sqrt(m) from device phases (float), all layers,
// and the phases wrapped to [-pi, pi) for the passes that form exp(i theta).
__global__ void k_set_diag(const float* __restrict__ theta, float2* __restrict__ d, float* __restrict__ ph,
                           size_t count, float scale) {
  constexpr float kTwoPiF = 6.28318530717958647692f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float th = theta[i];
    float sn, cs;
    sincosf(th, &sn, &cs);
    d[i] = make_float2(cs * scale, sn * scale);
    float w = th - kTwoPiF * rintf(th / kTwoPiF);
    if (w >= 0.5f * kTwoPiF) w -= kTwoPiF;
    ph[i] = w;
  }
}

// Phase gradient of one layer, summed over the batch (compensated):
// out[k] = sum_b Im(conj(D[k] q[b][k]) h[b][k]), with q[b][k] = 0 for k >= nq.
// D carries 1/sqrt(m) and h carries the matching sqrt(m) (unnormalised inverse
// DFTs), so the product is the unscaled gradient.
__global__ void k_theta_grad(const float2* __restrict__ q, int nq, const float2* __restrict__ d,
                             const float2* __restrict__ h, int m, int B, float* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  if (k >= nq) {
    out[k] = 0.f;
    return;
  }
  const float2 dk = __ldg(&d[k]);
  fsum2 acc{0.f, 0.f};
  for (int b = 0; b < B; ++b) {
    const float2 pk = cmul(dk, q[(size_t)b * nq + k]);
    const float2 hk = h[(size_t)b * m + k];
    acc_add(acc, pk.x * hk.y - pk.y * hk.x);  // Im(conj(p) h)
  }
  out[k] = acc.s + acc.c;
}

// out[b][k] = conj(D[k]) h[b][k] for k < n (the last step of the backward: U^H D_1^H).
__global__ void k_conj_diag_prune(const float2* __restrict__ h, const float2* __restrict__ d, int m, int n, int B,
                                  float2* __restrict__ out) {
  const size_t total = (size_t)B * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / n, k = i - b * n;
    out[i] = cmulc(h[b * m + k], __ldg(&d[k]));
  }
}

// yt[b] = transpose of the S x S row-major grid y[b], through 32 x 32 tiles in
// shared memory (both sides coalesced). Grid (S/32 or 1, S/32 or 1, B) of
// 32 x 8 threads; S a power of two.
__global__ void k_transpose_grids(const float* __restrict__ y, float* __restrict__ yt, int S) {
  __shared__ float tile[32][33];
  const size_t base = (size_t)blockIdx.z * S * S;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < S && c < S) tile[k][threadIdx.x] = y[base + (size_t)r * S + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = c0 + k, c = r0 + threadIdx.x;  // output row = input column
    if (r < S && c < S) yt[base + (size_t)r * S + c] = tile[threadIdx.x][k];
  }
}

cudaError_t launch_transpose_grids(const float* y, float* yt, int S, int B, cudaStream_t s) {
  const int t = (S + 31) / 32;
  k_transpose_grids<<<dim3(t, t, B), dim3(32, 8), 0, s>>>(y, yt, S);
  count_launch();
  return cudaGetLastError();
}

// Failure-path probe: one thread waits on an mbarrier that nothing ever
// completes, through the same bounded wait the pass kernels use; when the wait
// gives up it records SR_ERR_TIMEOUT in the plan's status word and returns.
// No copy is in flight, so the kernel ends cleanly.
__global__ void k_wait_probe(int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(smem_addr(&bar), 1);
  mbar_init_fence();
  if (!mbar_wait_bounded(smem_addr(&bar), 0)) atomicExch(err, (int)SR_ERR_TIMEOUT);
}

cudaError_t launch_wait_probe(int* err, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(err);
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers

constexpr size_t kSmemBudget = 220 * 1024;

LineGeom make_geom(int64_t m, int ell) {
  LineGeom g;
  g.ell = ell;
  g.nl = (int)(m / ell);
  const int E = ell < 16 ? ell : 16;
  g.P = ell / E;  // threads per line
  int T;
  if (ell % 3 == 0) {
    T = ell == 768 ? 8 : 16;  // the radix-3 tile shapes: 384 threads (192 for lines of 192)
  } else {
    T = std::max(8, 256 / g.P);
    T = std::min(T, pass_threads(ell) / g.P);
  }
  T = std::min(T, g.nl);
  while (T & (T - 1)) T &= T - 1;          // a power of two
  while (T > 1 && g.nl % T != 0) T >>= 1;  // tiles of whole lines (3 * 2^a lines in the other layout)
  while (T > 1 && pipe_layout(ell, T, 1, true).total + 1024 > kSmemBudget) T >>= 1;
  g.T = T;
  g.lgT = 0;
  while ((1 << g.lgT) < T) ++g.lgT;
  g.cpp = g.nl / T;
  g.threads = T * g.P;
  // One staging buffer: the next tile's load is issued once the current tile is
  // in registers, so it overlaps the current tile's compute without a second buffer.
  g.nbuf = 1;
  g.smem_pipe = pipe_layout(ell, T, g.nbuf, true).total + 1024;
  g.smem_first = pipe_layout(ell, T, 1, false).total + 1024;
  return g;
}

// Step 1 of a DFT with decomposition parity 0 works on layout X, parity 1 on Y;
// its step 2 on the other layout.
Layout s1_layout(int parity) { return parity == 0 ? kLayoutX : kLayoutY; }
Layout s2_layout(int parity) { return parity == 0 ? kLayoutY : kLayoutX; }

static int pair_index(int da, int db) { return da < 0 ? (db < 0 ? 0 : 1) : 2; }

static cudaError_t allow_smem(const void* fn, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

static PassArgs with_geom(const PassArgs& a0, const Plan& p, const LineGeom& g, int B) {
  PassArgs a = a0;
  a.m = (int)p.m;
  a.nl = g.nl;
  a.ell = g.ell;
  a.T = g.T;
  a.lgT = g.lgT;
  a.cpp = g.cpp;
  a.ntiles = B * g.cpp;
  a.tws = p.lmax / g.ell;
  return a;
}

cudaError_t launch_first(const Plan& p, Layout lay, const PassArgs& a0, int B, cudaStream_t s) {
  const LineGeom& g = p.geom[lay];
  auto fn = reinterpret_cast<void (*)(PassArgs)>(const_cast<void*>(pick_first(g.ell, g.T, a0.out_dir, p.two_d)));
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = allow_smem((const void*)fn, g.smem_first);
  if (e != cudaSuccess) return e;
  const PassArgs a = with_geom(a0, p, g, B);
  const int grid = std::max(1, std::min(a.ntiles, p.per_sm_first[lay] * p.num_sms));
  fn<<<grid, g.threads, g.smem_first, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

static cudaError_t launch_pipe(bool last, const Plan& p, Layout lay, const PassArgs& a0, int B, cudaStream_t s) {
  const LineGeom& g = p.geom[lay];
  auto fn = reinterpret_cast<void (*)(PassArgs, int)>(
      const_cast<void*>(last ? pick_last(g.ell, g.T, a0.in_dir, g.nl, p.two_d) : pick_mid(g.ell, g.T, a0.in_dir, a0.out_dir, g.nl)));
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = allow_smem((const void*)fn, g.smem_pipe);
  if (e != cudaSuccess) return e;
  const PassArgs a = with_geom(a0, p, g, B);
  const int per_sm = last ? p.per_sm_last[lay][a0.in_dir > 0] : p.per_sm_mid[lay][pair_index(a0.in_dir, a0.out_dir)];
  const int grid = std::max(1, std::min(a.ntiles, per_sm * p.num_sms));
  fn<<<grid, g.threads, g.smem_pipe, s>>>(a, g.nbuf);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_mid(const Plan& p, Layout lay, const PassArgs& a, int B, cudaStream_t s) {
  return launch_pipe(false, p, lay, a, B, s);
}
cudaError_t launch_last(const Plan& p, Layout lay, const PassArgs& a, int B, cudaStream_t s) {
  return launch_pipe(true, p, lay, a, B, s);
}

cudaError_t launch_last_first(const Plan& p, Layout lay, const PassArgs& a0, int B, cudaStream_t s) {
  const LineGeom& g = p.geom[lay];
  auto fn = reinterpret_cast<void (*)(PassArgs, int)>(const_cast<void*>(pick_last_first(g.ell, g.T, g.nl, p.two_d)));
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = allow_smem((const void*)fn, g.smem_pipe);
  if (e != cudaSuccess) return e;
  const PassArgs a = with_geom(a0, p, g, B);
  const int grid = std::max(1, std::min(a.ntiles, p.per_sm_lf[lay] * p.num_sms));
  fn<<<grid, g.threads, g.smem_pipe, s>>>(a, g.nbuf);
  count_launch();
  return cudaGetLastError();
}

cudaError_t pass_occupancy(const LineGeom& g, int* per_sm_mid, int* per_sm_last, int* per_sm_lf, int* per_sm_first) {
  {
    const void* fn = pick_first(g.ell, g.T, -1, 0);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem(fn, g.smem_first);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm_first, fn, g.threads, g.smem_first);
    if (e != cudaSuccess) return e;
    *per_sm_first = std::max(1, *per_sm_first);
  }
  // per_sm_mid[3]: direction pairs (-,-), (-,+), (+,+); per_sm_last[2]: (-), (+); per_sm_lf: fused
  const int pairs[3][2] = {{-1, -1}, {-1, 1}, {1, 1}};
  for (int k = 0; k < 6; ++k) {
    const void* fn = k < 3   ? pick_mid(g.ell, g.T, pairs[k][0], pairs[k][1], g.nl)
                     : k < 5 ? pick_last(g.ell, g.T, k == 3 ? -1 : 1, g.nl, 0)
                             : pick_last_first(g.ell, g.T, g.nl, 0);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem(fn, g.smem_pipe);
    if (e != cudaSuccess) return e;
    int* out = k < 3 ? &per_sm_mid[k] : k < 5 ? &per_sm_last[k - 3] : per_sm_lf;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fn, g.threads, g.smem_pipe);
    if (e != cudaSuccess) return e;
    *out = std::max(1, *out);
  }
  return cudaSuccess;
}

cudaError_t launch_sum_rows(const float* y, int B, int m, float* part, int chunks, cudaStream_t s) {
  k_sum_rows<<<dim3(chunks, B), 256, 0, s>>>(y, m, part, chunks);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_norm_rows(const float2* v, int B, int n, float* part, int chunks, cudaStream_t s) {
  k_norm_rows<<<dim3(chunks, B), 256, 0, s>>>(v, n, part, chunks);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_finish_scalars(const float* part, int chunks, int B, float mu0, int m, float* sumy, float* mu,
                                  cudaStream_t s) {
  k_finish_scalars<<<(B + 127) / 128, 128, 0, s>>>(part, chunks, B, mu0, m, sumy, mu);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_scale_rows(float2* v, int B, int n, const float* part, int chunks, const float* sumy,
                              cudaStream_t s) {
  const int blocks = std::min(64, (n + 255) / 256);
  k_scale_rows<<<dim3(blocks, B), 256, 0, s>>>(v, n, part, chunks, sumy);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_set_diag(const float* theta, float2* d, float* ph, size_t count, float scale, cudaStream_t s) {
  const int blocks = (int)std::min<size_t>(4096, (count + 255) / 256);
  k_set_diag<<<blocks, 256, 0, s>>>(theta, d, ph, count, scale);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_theta_grad(const float2* q, int nq, const float2* d, const float2* h, int m, int B, float* out,
                              cudaStream_t s) {
  k_theta_grad<<<(m + 255) / 256, 256, 0, s>>>(q, nq, d, h, m, B, out);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_conj_diag_prune(const float2* h, const float2* d, int m, int n, int B, float2* out,
                                   cudaStream_t s) {
  const size_t total = (size_t)B * n;
  const int blocks = (int)std::min<size_t>(4096, (total + 255) / 256);
  k_conj_diag_prune<<<blocks, 256, 0, s>>>(h, d, m, n, B, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace sr
