// contract.cu -- the contraction step of Eqs. 5-7 on a caller's tensor.
//
// D[M][N] = sum_k A[m][k] B[n][k] with the arithmetic of a compute mode, for
// callers that hold their own AO-like tensor (and for checking each
// contraction kernel in isolation).  The bf16 split planes and padded
// copies live in library-owned scratch that is kept between calls.
#include "internal.h"

namespace qk {
namespace {

DevBuf g_scratch;

inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }
inline int64_t up8(int64_t x) { return (x + 7) / 8 * 8; }

__global__ void split_f32_kernel(const float* src, int64_t rows, int64_t cols, int64_t ld,
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

__global__ void pad_f32_kernel(const float* src, int64_t rows, int64_t cols, int64_t ld,
                               float* dst) {
  const int64_t n = rows * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ld, c = i % ld;
    dst[i] = c < cols ? src[r * cols + c] : 0.0f;
  }
}

unsigned grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace
}  // namespace qk

using namespace qk;

extern "C" qk_status qk_contract_device(int32_t mode, int64_t M, int64_t N, int64_t K,
                                        const void* A, const void* B, void* D, void* stream) {
  if (!A || !B || !D) return QK_ERR_NULL_POINTER;
  if (M < 0 || N < 0 || K < 1) return QK_ERR_BAD_SIZE;
  if (M == 0 || N == 0) return QK_SUCCESS;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  switch (mode) {
    case QK_FP64:
      e = launch_gemm_f64(M, N, K, (const double*)A, K, 1, (const double*)B, K, 1, (double*)D, N,
                          1, s);
      break;
    case QK_FP32:
      e = launch_gemm_f32(M, N, K, (const float*)A, K, 1, (const float*)B, K, 1, (float*)D, N, 1,
                          s);
      break;
    case QK_BF16X3:
    case QK_TF32: {
      const int64_t ld = up8(K);
      const size_t es = mode == QK_BF16X3 ? 2 : 4;
      const int planes = mode == QK_BF16X3 ? 2 : 1;
      const size_t a_b = align256(M * ld * es), b_b = align256(N * ld * es);
      e = g_scratch.ensure(256 + planes * (a_b + b_b));
      if (e != cudaSuccess) break;
      unsigned char* base = (unsigned char*)g_scratch.p;
      int* flag = (int*)base;
      unsigned char* pa = base + 256;
      unsigned char* pb = pa + planes * a_b;
      e = cudaMemsetAsync(flag, 0, sizeof(int), s);
      if (e != cudaSuccess) break;
      AOTensor t{};
      t.rows = M;
      t.ld = ld;
      if (mode == QK_BF16X3) {
        split_f32_kernel<<<grid_for(M * ld), 256, 0, s>>>(
            (const float*)A, M, K, ld, (__nv_bfloat16*)pa, (__nv_bfloat16*)(pa + a_b));
        split_f32_kernel<<<grid_for(N * ld), 256, 0, s>>>(
            (const float*)B, N, K, ld, (__nv_bfloat16*)pb, (__nv_bfloat16*)(pb + b_b));
        t.a = pa;
        t.a_lo = pa + a_b;
        e = cudaGetLastError();
        if (e == cudaSuccess)
          e = launch_mo_tc(mode, t, K, pb, pb + b_b, ld, N, (float*)D,
                           tc_default_config(mode, N), flag, s);
      } else {
        pad_f32_kernel<<<grid_for(M * ld), 256, 0, s>>>((const float*)A, M, K, ld, (float*)pa);
        pad_f32_kernel<<<grid_for(N * ld), 256, 0, s>>>((const float*)B, N, K, ld, (float*)pb);
        t.a = pa;
        e = cudaGetLastError();
        if (e == cudaSuccess)
          e = launch_mo_tc(mode, t, K, pb, nullptr, ld, N, (float*)D, tc_default_config(mode, N),
                           flag, s);
      }
      if (e != cudaSuccess) break;
      int hflag = 0;
      e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e == cudaSuccess && hflag != 0) return QK_ERR_DEVICE_TIMEOUT;
      break;
    }
    default:
      return QK_ERR_INVALID_ARG;
  }
  if (e == cudaErrorNotSupported) return QK_ERR_NOT_IMPLEMENTED;
  if (e == cudaErrorMemoryAllocation) return QK_ERR_OUT_OF_MEMORY;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return QK_ERR_CUDA;
  }
  return QK_SUCCESS;
}
