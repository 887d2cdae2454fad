// mo_simt.cu -- SIMT (CUDA-core) contractions in FP64 and FP32.
//
// The MO vgl of Eqs. 5-7 is one matrix product over the concatenated
// (point, component) rows of the AO tensor (Sec. 3.2: values, gradients and
// Laplacians in a single GEMM so that C is reused):
//   D[5P x N_mo] = AO[5P x N_ao] . C^T
// These kernels are the FP64 accuracy path and the plain FP32 path; the
// same kernel with other strides computes the adjoint products
// Abar = W . C and dL/dC = W^T . AO (split over K into partial sums).
//
// Tiling: a CTA computes a BM x BN tile of D with 256 threads, each owning a
// TM x TN register tile; K advances in BK slices staged through shared
// memory (double-buffered, next slice prefetched into registers while the
// current one is consumed).  Element (m, k) of A is A[m*sam + k*sak] and
// (n, k) of B is B[n*sbn + k*sbk]; the load pattern follows whichever
// stride is 1 so that global loads stay coalesced.
#include "internal.h"

namespace qk {

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    gemm_simt_kernel(int64_t M, int64_t N, int64_t K, const T* __restrict__ A, int64_t sam,
                     int64_t sak, const T* __restrict__ B, int64_t sbn, int64_t sbk,
                     T* __restrict__ D, int64_t ldd, int64_t k_per_split, int64_t m_tiles) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int LA = BM * BK / NT;
  constexpr int LB = BN * BK / NT;
  constexpr int PAD = 16 / sizeof(T);
  static_assert(BM * BK % NT == 0 && BN * BK % NT == 0, "tile/thread mismatch");
  __shared__ __align__(16) T As[2][BK][BM + PAD];
  __shared__ __align__(16) T Bs[2][BK][BN + PAD];

  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN);
  const int ty = tid / (BN / TN);
  const int64_t n0 = (int64_t)blockIdx.x * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * k_per_split;
  const int64_t kend = min(K, kbeg + k_per_split);
  T* Dz = D + (int64_t)blockIdx.z * M * ldd;
  const bool a_kfast = (sak == 1);
  const bool b_kfast = (sbk == 1);

  for (int64_t mt = blockIdx.y; mt < m_tiles; mt += gridDim.y) {
    const int64_t m0 = mt * BM;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    T ra[LA], rb[LB];
    auto load = [&](int64_t k0) {
#pragma unroll
      for (int l = 0; l < LA; ++l) {
        const int i = tid + l * NT;
        const int kk = a_kfast ? i % BK : i / BM;
        const int mm = a_kfast ? i / BK : i % BM;
        const int64_t m = m0 + mm, k = k0 + kk;
        ra[l] = (m < M && k < kend) ? A[m * sam + k * sak] : T(0);
      }
#pragma unroll
      for (int l = 0; l < LB; ++l) {
        const int i = tid + l * NT;
        const int kk = b_kfast ? i % BK : i / BN;
        const int nn = b_kfast ? i / BK : i % BN;
        const int64_t n = n0 + nn, k = k0 + kk;
        rb[l] = (n < N && k < kend) ? B[n * sbn + k * sbk] : T(0);
      }
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int l = 0; l < LA; ++l) {
        const int i = tid + l * NT;
        const int kk = a_kfast ? i % BK : i / BM;
        const int mm = a_kfast ? i / BK : i % BM;
        As[buf][kk][mm] = ra[l];
      }
#pragma unroll
      for (int l = 0; l < LB; ++l) {
        const int i = tid + l * NT;
        const int kk = b_kfast ? i % BK : i / BN;
        const int nn = b_kfast ? i / BK : i % BN;
        Bs[buf][kk][nn] = rb[l];
      }
    };

    if (kbeg < kend) {
      load(kbeg);
      store(0);
    }
    __syncthreads();
    int buf = 0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
      const bool has_next = k0 + BK < kend;
      if (has_next) load(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = Bs[buf][kk][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * bv[j];
      }
      if (has_next) store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t m = m0 + ty * TM + i;
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t n = n0 + tx * TN + j;
        if (n < N) Dz[m * ldd + n] = acc[i][j];
      }
    }
    __syncthreads();
  }
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
static cudaError_t launch_gemm(int64_t M, int64_t N, int64_t K, const T* A, int64_t sam,
                               int64_t sak, const T* B, int64_t sbn, int64_t sbk, T* D,
                               int64_t ldd, int k_split, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (k_split < 1) k_split = 1;
  const int64_t kps = ((K + k_split - 1) / k_split + BK - 1) / BK * BK;
  const int64_t m_tiles = (M + BM - 1) / BM;
  const int64_t n_tiles = (N + BN - 1) / BN;
  if (n_tiles > 65535 || k_split > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)n_tiles, (unsigned)(m_tiles < 65535 ? m_tiles : 65535), (unsigned)k_split);
  gemm_simt_kernel<T, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(
      M, N, K, A, sam, sak, B, sbn, sbk, D, ldd, kps, m_tiles);
  return cudaGetLastError();
}

cudaError_t launch_gemm_f32(int64_t M, int64_t N, int64_t K, const float* A, int64_t sam,
                            int64_t sak, const float* B, int64_t sbn, int64_t sbk, float* D,
                            int64_t ldd, int k_split, cudaStream_t s) {
  return launch_gemm<float, 128, 128, 16, 8, 8>(M, N, K, A, sam, sak, B, sbn, sbk, D, ldd,
                                                k_split, s);
}

cudaError_t launch_gemm_f64(int64_t M, int64_t N, int64_t K, const double* A, int64_t sam,
                            int64_t sak, const double* B, int64_t sbn, int64_t sbk, double* D,
                            int64_t ldd, int k_split, cudaStream_t s) {
  return launch_gemm<double, 64, 64, 16, 4, 4>(M, N, K, A, sam, sak, B, sbn, sbk, D, ldd,
                                               k_split, s);
}

template <typename T>
__global__ void reduce_partials_kernel(const T* part, int k_split, int64_t n, double* dst,
                                       const int* col_map, int64_t ncol) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < k_split; ++z) s += (double)part[(int64_t)z * n + i];
    // col_map: column j of each row goes to column col_map[j]
    dst[col_map ? (i / ncol) * ncol + col_map[i % ncol] : i] = s;
  }
}

cudaError_t launch_reduce_partials_f32(const float* part, int k_split, int64_t n, double* dst,
                                       cudaStream_t s, const int* col_map, int64_t ncol) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  reduce_partials_kernel<float><<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(
      part, k_split, n, dst, col_map, ncol);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials_f64(const double* part, int k_split, int64_t n, double* dst,
                                       cudaStream_t s, const int* col_map, int64_t ncol) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  reduce_partials_kernel<double><<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(
      part, k_split, n, dst, col_map, ncol);
  return cudaGetLastError();
}

}  // namespace qk
