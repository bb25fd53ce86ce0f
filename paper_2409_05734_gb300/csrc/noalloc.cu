// sr_forward_noalloc: z = A x like sr_forward, for callers that cannot
// allocate device memory at the time of the call -- for example code that
// runs while a CUDA graph is being captured on its stream (cudaMalloc is not
// permitted there), or a host that has handed all device memory to its own
// allocator and must not let a library take more. The plan itself is created
// beforehand (sr_plan_create allocates its tables once); this entry point then
// runs the same pass kernels without touching the plan's workspace, using a
// fixed scratch area compiled into the library instead of cudaMalloc.
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

// Device address of the scratch, looked up once per device. In host code the
// array's name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with that device current.
constexpr int kMaxDevices = 64;
float2* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

sr_status noalloc_fail(sr_status st, const std::string& msg) {
  sr::set_last_error(msg);
  return st;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Same tensor description the plan uses for its own exchange buffers: rows of
// `ell` complex values, boxes of 16 values x T rows, 128-byte swizzle.
bool encode_rows(CUtensorMap* map, float2* base, int ell, int64_t rows, int T) {
  static EncodeTiledFn enc = nullptr;
  if (!enc) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f)
      return false;
    enc = reinterpret_cast<EncodeTiledFn>(f);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * ell), (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ell * 8};
  const cuuint32_t box[2] = {32, (cuuint32_t)T};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

extern "C" {

sr_status sr_forward_noalloc(const sr_plan* plan_in, const void* x, void* z, int B, void* stream) {
  const sr::Plan* plan = reinterpret_cast<const sr::Plan*>(plan_in);
  if (!plan || !x || !z) return noalloc_fail(SR_ERR_INVALID_ARG, "NULL argument");
  if (B < 1) return noalloc_fail(SR_ERR_INVALID_ARG, "B must be >= 1");
  if (plan->inner) return noalloc_fail(SR_ERR_UNSUPPORTED, "only power-of-two m is supported");
  if (plan->two_d) return noalloc_fail(SR_ERR_UNSUPPORTED, "2D plans are not supported");
  if (plan->mo < plan->m) return noalloc_fail(SR_ERR_UNSUPPORTED, "m < n is not supported");
  if ((size_t)B * (size_t)plan->m > kNoallocMaxElements)
    return noalloc_fail(SR_ERR_UNSUPPORTED, "B*m = " + std::to_string((size_t)B * plan->m) +
                                                " exceeds the static scratch of " +
                                                std::to_string(kNoallocMaxElements) + " complex values");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(SR_ERR_INVALID_ARG, "current CUDA device differs from the plan's device");
  float2* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return noalloc_fail(SR_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<float2*>(p);
    }
    scratch = g_scratch_ptr[dev];
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
    if (g.ell >= 16 && g.T >= 8 && !encode_rows(&a.tmap, cur, g.ell, (int64_t)B * g.nl, g.T))
      return noalloc_fail(SR_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    cudaError_t e;
    if (!last) {
      a.eout = nxt;
      a.op = sr::kOpDiag;
      a.dp = plan->d_dp + (size_t)k * plan->m;
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
