// selftest.cu -- a check of the bounded device-side waits every tcgen05
// kernel of the library relies on (mbarrier waits that give up after a
// clock limit and raise the CTA's abort flag, plus the caller's error word).
//
// The kernel waits on an mbarrier that nothing ever arrives at: one thread
// with a short limit, which must give up, record its code in the error word
// and raise the abort flag; a second thread with the library's normal limit
// (about two seconds), which must leave through the abort flag well before
// its own limit.  Nothing faults, traps or spins without bound.
#include "tc_common.cuh"

namespace qk {
namespace {

// out[0]: error word (flag_error code 1 once the short wait gave up);
// out[1]: 1 if the second waiter left through the abort flag, 2 if its own
// limit ran out instead; out[2], out[3]: cycles each waiter spent.
__global__ void wait_timeout_kernel(long long limit, int* out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  const uint32_t b = tc::smem_u32(&bar);
  if (threadIdx.x == 0) {
    tc::mbar_init(b, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  volatile int* ab = &abort_flag;
  const long long t0 = clock64();
  if (threadIdx.x == 0) {
    if (!tc::mbar_wait(b, 0u, ab, limit)) tc::flag_error(out, ab, 1);
    out[2] = (int)min(clock64() - t0, (long long)INT32_MAX);
  } else if (threadIdx.x == 32) {
    const bool got = tc::mbar_wait(b, 0u, ab);
    const long long dt = clock64() - t0;
    out[1] = got ? 0 : (dt < tc::kWaitCycles ? 1 : 2);
    out[3] = (int)min(dt, (long long)INT32_MAX);
  }
}

}  // namespace
}  // namespace qk

extern "C" qk_status qk_selftest_wait_timeout(int64_t limit_cycles, int32_t* info) {
  if (limit_cycles < 1 || limit_cycles > 100000000) return QK_ERR_BAD_SIZE;
  int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 4 * sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return QK_ERR_CUDA;
  }
  int h[4] = {0, 0, 0, 0};
  e = cudaMemset(d, 0, 4 * sizeof(int));
  if (e == cudaSuccess) {
    qk::wait_timeout_kernel<<<1, 64>>>((long long)limit_cycles, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return QK_ERR_CUDA;
  }
  if (info) {
    for (int i = 0; i < 4; ++i) info[i] = h[i];
  }
  return h[0] != 0 ? QK_ERR_DEVICE_TIMEOUT : QK_SUCCESS;
}
