// single.cu -- single-electron moves: the proposed positions of one
// electron in every walker written into the context's point arrays once
// the move is accepted (point w * elec_num + elec of walker w).
#include "internal.h"

namespace qk {
namespace {

__global__ void scatter_points_kernel(PointsDev src, PointsDev dst, int64_t elec_num,
                                      int64_t elec) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < src.n;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = w * elec_num + elec;
    double* x = const_cast<double*>(dst.x);
    double* y = const_cast<double*>(dst.y);
    double* z = const_cast<double*>(dst.z);
    float* hi = const_cast<float*>(dst.hi);
    float* lo = const_cast<float*>(dst.lo);
    x[i] = src.x[w];
    y[i] = src.y[w];
    z[i] = src.z[w];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      hi[k * dst.ld + i] = src.hi[k * src.ld + w];
      lo[k * dst.ld + i] = src.lo[k * src.ld + w];
    }
  }
}

}  // namespace

cudaError_t launch_scatter_points(const PointsDev& src, const PointsDev& dst, int64_t elec_num,
                                  int64_t elec, cudaStream_t s) {
  if (src.n == 0) return cudaSuccess;
  const int64_t blocks = (src.n + 255) / 256;
  scatter_points_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, s>>>(src, dst,
                                                                                 elec_num, elec);
  return cudaGetLastError();
}

}  // namespace qk
