// sr_forward_noalloc: z = A x like sr_forward, for callers that cannot
// allocate device memory at the time of the call -- for example code that
// runs while a CUDA graph is being captured on its stream (cudaMalloc is not
// permitted there), or a host that has handed all device memory to its own
// allocator and must not let a library take more. The plan itself is created
// beforehand (sr_plan_create allocates its tables once); this entry point then
// runs the same pass kernels without touching the plan's workspace, using a
// fixed scratch area compiled into the library instead of cudaMalloc.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "sr_internal.h"

namespace {

// Scratch of the two exchange buffers: 2 x 2^19 complex values (8 MiB), a
// file-scope device array. Every GPU that loads the library holds it until
// the process exits.
constexpr size_t kNoallocMaxElements = SR_FORWARD_NOALLOC_MAX_ELEMENTS;  // B * m limit per call
static __device__ __align__(256) float2 g_noalloc_scratch[2 * kNoallocMaxElements];

// Device address of the scratch, looked up once per device and CUDA context.
// In host code the array's name is only a host-side stand-in, so the address
// must come from cudaGetSymbolAddress with that device current. The context
// is part of the key: after cudaDeviceReset the primary context (and the
// module holding the array) is created anew, and an address cached from the
// old context would no longer belong to the library.
constexpr int kMaxDevices = 64;
struct ScratchSlot {
  CUcontext ctx = nullptr;
  float2* ptr = nullptr;
};
ScratchSlot g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

sr_status noalloc_fail(sr_status st, const std::string& msg) {
  sr::set_last_error(msg);
  return st;
}

// The calling thread's current CUDA context (the driver's cuCtxGetCurrent,
// looked up once per process; the static's initialisation is thread-safe).
bool current_context(CUcontext* ctx) {
  using GetCurrentFn = CUresult (*)(CUcontext*);
  static const GetCurrentFn fn = []() -> GetCurrentFn {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<GetCurrentFn>(f);
  }();
  return fn && fn(ctx) == CUDA_SUCCESS && *ctx != nullptr;
}

}  // namespace

extern "C" {

sr_status sr_forward_noalloc(const sr_plan* plan_in, const void* x, void* z, int B, void* stream) {
  const sr::Plan* plan = reinterpret_cast<const sr::Plan*>(plan_in);
  if (!plan || !x || !z) return noalloc_fail(SR_ERR_INVALID_ARG, "NULL argument");
  if (B < 1) return noalloc_fail(SR_ERR_INVALID_ARG, "B must be >= 1");
  if (plan->inner || (plan->m & (plan->m - 1)) != 0)
    return noalloc_fail(SR_ERR_UNSUPPORTED, "only power-of-two m is supported");
  if (plan->two_d) return noalloc_fail(SR_ERR_UNSUPPORTED, "2D plans are not supported");
  if (plan->mo < plan->m) return noalloc_fail(SR_ERR_UNSUPPORTED, "m < n is not supported");
  // A plan with per-problem phases holds diagonal tables for exactly
  // batch_fixed problems; any other B would read past them.
  if (plan->batch_fixed && B != plan->batch_fixed)
    return noalloc_fail(SR_ERR_INVALID_ARG, "this plan holds per-problem phases for a batch of " +
                                                std::to_string(plan->batch_fixed) + " problems");
  if ((size_t)B * (size_t)plan->m > kNoallocMaxElements)
    return noalloc_fail(SR_ERR_UNSUPPORTED, "B*m = " + std::to_string((size_t)B * plan->m) +
                                                " exceeds the static scratch of " +
                                                std::to_string(kNoallocMaxElements) + " complex values");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(SR_ERR_INVALID_ARG, "current CUDA device differs from the plan's device");
  // cudaSetDevice on the current device makes its primary context current on
  // this thread (a thread whose first CUDA call this is has none yet).
  CUcontext ctx = nullptr;
  if (cudaSetDevice(dev) != cudaSuccess || !current_context(&ctx)) {
    cudaGetLastError();
    return noalloc_fail(SR_ERR_CUDA, "no current CUDA context on this thread");
  }
  float2* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchSlot& slot = g_scratch[dev];
    if (!slot.ptr || slot.ctx != ctx) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return noalloc_fail(SR_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      slot.ptr = static_cast<float2*>(p);
      slot.ctx = ctx;
    }
    scratch = slot.ptr;
  }
  float2* e0 = scratch;
  float2* e1 = scratch + kNoallocMaxElements;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // The forward chain of sr_forward: FIRST (U, D_1, step 1 of DFT 0), one MID
  // per later DFT (step 2, D_{k+1}, step 1), LAST (step 2 of DFT L-1, store z).
  // Every exchange-buffer element is written before it is read, so the
  // scratch needs no clearing between calls.
  sr::PassArgs base;
  memset(&base, 0, sizeof(base));
  base.m = (int)plan->m;
  base.dp_stride = plan->dp_stride;
  base.twl = plan->d_twl;
  base.tw_hi = plan->d_tw_hi;
  base.tw_lo = plan->d_tw_lo;
  base.tw_shift = plan->tw_shift;
  base.err = plan->d_err;
  const int L = plan->L;
  float2* cur = e0;
  float2* nxt = e1;
  {
    sr::PassArgs a = base;
    a.out_dir = -1;
    a.xin = static_cast<const float2*>(x);
    a.n_in = (int)plan->n;
    a.op = sr::kOpDiag;
    a.dp = plan->d_dp;
    a.eout = cur;
    cudaError_t e = sr::launch_first(*plan, sr::s1_layout(0), a, B, s);
    if (e != cudaSuccess) return noalloc_fail(SR_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  }
  for (int k = 1; k <= L; ++k) {
    const bool last = (k == L);
    const sr::Layout lay = sr::s2_layout((k - 1) % 2);
    const sr::LineGeom& g = plan->geom[lay];
    sr::PassArgs a = base;
    a.in_dir = -1;
    a.out_dir = -1;
    a.ein = cur;
    if (g.ell >= 16 && g.T >= 8 && sr::encode_rows(&a.tmap, cur, g.ell, (int64_t)B * g.nl, g.T) != cudaSuccess)
      return noalloc_fail(SR_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    cudaError_t e;
    if (!last) {
      a.eout = nxt;
      a.op = sr::kOpDiag;
      a.dp = plan->d_dp + (size_t)k * plan->m;
      a.ph = plan->d_ph + (size_t)k * plan->m;
      a.dscale = (float)(1.0 / std::sqrt((double)plan->m));
      e = sr::launch_mid(*plan, lay, a, B, s);
      std::swap(cur, nxt);
    } else {
      a.op = sr::kOpNone;
      a.xout = static_cast<float2*>(z);
      a.n_out = (int)plan->m;
      a.out_mode = sr::kOutStore;
      e = sr::launch_last(*plan, lay, a, B, s);
    }
    if (e != cudaSuccess) return noalloc_fail(SR_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  }
  return SR_OK;
}

}  // extern "C"
