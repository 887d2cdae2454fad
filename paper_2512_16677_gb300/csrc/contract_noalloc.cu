// contract_noalloc.cu -- the tensor-core contraction with no allocation.
//
// Some callers cannot call cudaMalloc: code that runs while another runtime
// owns the device memory budget (a framework's caching allocator or a fixed
// memory pool, where a stray cudaMalloc can fragment the pool or fail at an
// arbitrary point), code on a latency-critical path where the implicit
// device synchronisation of cudaMalloc/cudaFree is unacceptable, and code
// that must not fail halfway for lack of memory once it has started.  This
// entry point gives them the split-bf16 / TF32 contraction of
// qk_contract_device with its scratch in a fixed device array instead.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes; every
// GPU that loads the library holds it until the process exits.  Host code
// cannot use the array's name as a device address (on the host it names a
// stand-in), so the device address is looked up with cudaGetSymbolAddress,
// with that device current, on the first call made on that device (and
// again after a reset of the device gave it a new context).
#include <cuda.h>

#include <mutex>

#include "internal.h"

namespace qk {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr size_t kFlagBytes = 256;                         // device error word
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array, cached per device together with the CUDA
// context it was looked up in: a reset of the device (cudaDeviceReset)
// gives the next call a new primary context, in which the module and the
// array are loaded afresh, so a cached address counts only while the
// current context is the one it came from.
struct ScratchAddr {
  void* ctx = nullptr;
  void* addr = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

CtxGetCurrentFn ctx_get_current_fn() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)p;
  });
  return fn;
}

// Device address of the scratch array in the current device's context (set-up
// on the first call per device and context, with that device current).
cudaError_t scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  CtxGetCurrentFn get = ctx_get_current_fn();
  if (!get) return cudaErrorInitializationError;
  CUcontext ctx = nullptr;  // NULL until the runtime first touches the device
  if (get(&ctx) != CUDA_SUCCESS) return cudaErrorInitializationError;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchAddr& slot = g_scratch_addr[dev];
  if (!ctx || slot.ctx != (void*)ctx || !slot.addr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the context current if need be
    if (e != cudaSuccess) return e;
    if (get(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorInitializationError;
    slot.ctx = (void*)ctx;
    slot.addr = p;
  }
  *out = slot.addr;
  return cudaSuccess;
}

inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }
inline int64_t up8(int64_t x) { return (x + 7) / 8 * 8; }

unsigned grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// FP32 [rows][cols] -> bf16 hi/lo planes [rows][ld], padding columns zeroed
__global__ void noalloc_split_kernel(const float* src, int64_t rows, int64_t cols, int64_t ld,
                                     __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const int64_t n = rows * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ld, c = i % ld;
    const float v = c < cols ? src[r * cols + c] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// FP32 [rows][cols] -> FP32 [rows][ld] with 16-byte aligned rows
__global__ void noalloc_pad_kernel(const float* src, int64_t rows, int64_t cols, int64_t ld,
                                   float* dst) {
  const int64_t n = rows * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ld, c = i % ld;
    dst[i] = c < cols ? src[r * cols + c] : 0.0f;
  }
}

}  // namespace
}  // namespace qk

using namespace qk;

extern "C" qk_status qk_contract_device_noalloc(int32_t mode, int64_t M, int64_t N, int64_t K,
                                                const float* A, const float* B, float* D,
                                                void* stream) {
  if (!A || !B || !D) return QK_ERR_NULL_POINTER;
  if (mode != QK_BF16X3 && mode != QK_TF32) return QK_ERR_INVALID_ARG;
  if (M < 0 || N < 0 || K < 1) return QK_ERR_BAD_SIZE;
  if (M == 0 || N == 0) return QK_SUCCESS;
  const int64_t ld = up8(K);
  const size_t es = mode == QK_BF16X3 ? 2 : 4;
  const int planes = mode == QK_BF16X3 ? 2 : 1;
  // sizes beyond the fixed scratch are refused before any work is queued
  if (M > (int64_t)kNoAllocScratchBytes || N > (int64_t)kNoAllocScratchBytes ||
      ld > (int64_t)kNoAllocScratchBytes)
    return QK_ERR_BAD_SIZE;
  const size_t a_b = align256((size_t)M * ld * es), b_b = align256((size_t)N * ld * es);
  if (kFlagBytes + planes * (a_b + b_b) > kNoAllocScratchBytes) return QK_ERR_BAD_SIZE;

  void* base_v = nullptr;
  cudaError_t e = scratch_address(&base_v);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return QK_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = (unsigned char*)base_v;
  int* flag = (int*)base;  // the array keeps the previous call's contents: clear the word
  unsigned char* pa = base + kFlagBytes;
  unsigned char* pb = pa + planes * a_b;
  e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  AOTensor t{};
  t.rows = M;
  t.ld = ld;
  t.a = pa;
  if (e == cudaSuccess) {
    if (mode == QK_BF16X3) {
      noalloc_split_kernel<<<grid_for(M * ld), 256, 0, s>>>(A, M, K, ld, (__nv_bfloat16*)pa,
                                                            (__nv_bfloat16*)(pa + a_b));
      noalloc_split_kernel<<<grid_for(N * ld), 256, 0, s>>>(B, N, K, ld, (__nv_bfloat16*)pb,
                                                            (__nv_bfloat16*)(pb + b_b));
      t.a_lo = pa + a_b;
      e = cudaGetLastError();
      if (e == cudaSuccess)
        e = launch_mo_tc(mode, t, K, pb, pb + b_b, ld, N, D, tc_default_config(mode, N), flag,
                         s);
    } else {
      noalloc_pad_kernel<<<grid_for(M * ld), 256, 0, s>>>(A, M, K, ld, (float*)pa);
      noalloc_pad_kernel<<<grid_for(N * ld), 256, 0, s>>>(B, N, K, ld, (float*)pb);
      e = cudaGetLastError();
      if (e == cudaSuccess)
        e = launch_mo_tc(mode, t, K, pb, nullptr, ld, N, D, tc_default_config(mode, N), flag, s);
    }
  }
  int hflag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorNotSupported ? QK_ERR_NOT_IMPLEMENTED : QK_ERR_CUDA;
  }
  return hflag != 0 ? QK_ERR_DEVICE_TIMEOUT : QK_SUCCESS;
}
