// density.cu -- helpers of the electron density on grid points (Sec. 5.4):
// rho(p) = sum_i w_i phi_i(p)^2 over the MOs with a nonzero weight.
//
// The tensor-core modes get rho from the contraction's density epilogue
// (per N tile partial sums, added here in a fixed order); the FP64 / FP32
// modes contract into D [points][occupied MOs] with the SIMT GEMM and sum
// w_i D_i^2 here.
#include "internal.h"

namespace qk {
namespace {

// dst row r = src row rows[r]; rows are ld elements of `elem` bytes.
__global__ void gather_rows_kernel(const unsigned char* src, int64_t row_bytes, const int* rows,
                                   int64_t nrows, unsigned char* dst) {
  const int64_t words = row_bytes / 4;
  const int64_t total = nrows * words;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / words, w = i % words;
    reinterpret_cast<uint32_t*>(dst)[r * words + w] =
        reinterpret_cast<const uint32_t*>(src + (int64_t)rows[r] * row_bytes)[w];
  }
}

__global__ void density_reduce_kernel(const float* part, int parts, int64_t n, float* rho) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int k = 0; k < parts; ++k) s += part[k * n + i];
    rho[i] = s;
  }
}

// One warp per point: lanes stride over the MOs, then a butterfly sum
// (a fixed order for a given m).
template <typename T>
__global__ void density_from_mo_kernel(const T* D, int64_t n, int64_t m, const double* w,
                                       T* rho) {
  const int lane = threadIdx.x & 31;
  const int64_t wstep = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t p = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); p < n;
       p += wstep) {
    T s = T(0);
    for (int64_t i = lane; i < m; i += 32) {
      const T v = D[p * m + i];
      s += (T)w[i] * v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rho[p] = s;
  }
}

unsigned grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_gather_rows(const void* src, int64_t ld, size_t elem, const int* rows,
                               int64_t nrows, void* dst, cudaStream_t s) {
  const int64_t row_bytes = ld * (int64_t)elem;
  if (nrows == 0) return cudaSuccess;
  if (row_bytes % 4 != 0) return cudaErrorInvalidValue;
  gather_rows_kernel<<<grid_for(nrows * row_bytes / 4), 256, 0, s>>>(
      (const unsigned char*)src, row_bytes, rows, nrows, (unsigned char*)dst);
  return cudaGetLastError();
}

cudaError_t launch_density_reduce(const float* part, int parts, int64_t n, float* rho,
                                  cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  density_reduce_kernel<<<grid_for(n), 256, 0, s>>>(part, parts, n, rho);
  return cudaGetLastError();
}

cudaError_t launch_density_from_mo(bool f64, const void* D, int64_t n, int64_t m,
                                   const double* w, void* rho, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 7) / 8;
  const unsigned g = (unsigned)(blocks < 8192 ? blocks : 8192);
  if (f64)
    density_from_mo_kernel<double><<<g, 256, 0, s>>>((const double*)D, n, m, w, (double*)rho);
  else
    density_from_mo_kernel<float><<<g, 256, 0, s>>>((const float*)D, n, m, w, (float*)rho);
  return cudaGetLastError();
}

}  // namespace qk
