// adjoint_tc.cu -- the two products of the MO vgl adjoint on the tcgen05
// tensor cores, in split bf16 (hi*hi + hi*lo + lo*hi, FP32 accumulation).
//
// For L = sum_{p,c,i} W[p][c][i] mo_vgl[p][c][i] with mo_vgl = AO . C^T
// (Eqs. 5-7, all five components as rows r = 5p + c):
//   Abar = W . C             [5P x N_ao]   (feeds dL/dR_nuc, Sec. 3.6)
//   dL/dC = W^T . AO         [N_mo x N_ao]
// Both run on the K-major tcgen05 kernel of the forward (mo_tc.cu), which
// wants each operand with its contraction index contiguous:
//   Abar:  A = W hi/lo [5P][N_mo] as given, B = C^T hi/lo [N_ao][N_mo];
//   dL/dC: A = W^T hi/lo [N_mo][5P], B = AO^T hi/lo [N_ao][5P],
// so W, W^T and AO^T are split (and transposed) here; C^T is split once per
// upload of C.  dL/dC sums over every row of every point: the rows are cut
// into slices, one problem of a multi-problem launch each, and the FP32
// partials are summed in FP64 in a fixed order.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace qk {
namespace {

unsigned grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// x = hi + lo + r with hi = bf16(x), lo = bf16(x - hi): |r| <= 2^-18 |x|.
__device__ __forceinline__ void split(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// FP32 [rows][cols] (row stride lds) -> bf16 hi/lo [rows][ld] (ld even), padding zero.
__global__ void split_rows_kernel(const float* __restrict__ src, int64_t rows, int64_t cols,
                                  int64_t lds, int64_t ld, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo) {
  // two adjacent columns per thread (ld is even), stored as bf16 pairs
  const int64_t n = rows * ld / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = 2 * i / ld, c = 2 * i % ld;
    const float* row = src + r * lds;
    __nv_bfloat162 hp, lp;
    split(c < cols ? row[c] : 0.0f, hp.x, lp.x);
    split(c + 1 < cols ? row[c + 1] : 0.0f, hp.y, lp.y);
    reinterpret_cast<__nv_bfloat162*>(hi)[i] = hp;
    reinterpret_cast<__nv_bfloat162*>(lo)[i] = lp;
  }
}

// FP32 [rows][cols] (row stride lds) -> transposed bf16 hi/lo [cols][ldt]
// (ldt >= rows and even, columns past rows zero), through 64 x 64 shared tiles.
__global__ void __launch_bounds__(256)
    transpose_split_kernel(const float* __restrict__ src, int64_t rows, int64_t cols,
                           int64_t lds, int64_t ldt, bool vec, __nv_bfloat16* __restrict__ hi,
                           __nv_bfloat16* __restrict__ lo) {
  // 64 x 64 tile: rows r0.. of src become columns of out[c][r] = src[r][c].
  // Loads are float4 along src rows (16 threads per row) when the rows are
  // 16-byte aligned; stores are bf16 pairs, one warp per output row, so each
  // warp instruction writes 128 contiguous bytes of each plane.  Columns
  // r in [rows, ldt) are written as zeros (ldt is even).
  __shared__ float t[64][65];
  const int64_t r0 = (int64_t)blockIdx.x * 64, c0 = (int64_t)blockIdx.y * 64;
  const int q = threadIdx.x & 15, rr = threadIdx.x >> 4;  // 16 x 16 threads
  if (vec && c0 + 64 <= cols) {
    for (int k = rr; k < 64; k += 16) {
      const int64_t r = r0 + k;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows) v = __ldg(reinterpret_cast<const float4*>(src + r * lds + c0) + q);
      t[k][4 * q] = v.x;
      t[k][4 * q + 1] = v.y;
      t[k][4 * q + 2] = v.z;
      t[k][4 * q + 3] = v.w;
    }
  } else {
    for (int k = rr; k < 64; k += 16) {
      const int64_t r = r0 + k;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t c = c0 + 16 * j + q;
        t[k][16 * j + q] = (r < rows && c < cols) ? src[r * lds + c] : 0.0f;
      }
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t r = r0 + 2 * lane;
  for (int k = w; k < 64; k += 8) {
    const int64_t c = c0 + k;
    if (c >= cols || r >= ldt) continue;
    __nv_bfloat16 h0, l0, h1, l1;
    split(t[2 * lane][k], h0, l0);
    split(t[2 * lane + 1][k], h1, l1);
    __nv_bfloat162 hp, lp;
    hp.x = h0;
    hp.y = h1;
    lp.x = l0;
    lp.y = l1;
    *reinterpret_cast<__nv_bfloat162*>(hi + c * ldt + r) = hp;
    *reinterpret_cast<__nv_bfloat162*>(lo + c * ldt + r) = lp;
  }
}

// C^T: FP64 [mo][ao] -> bf16 hi/lo [ao][ld] (split from the FP64 value).
__global__ void ct_split_kernel(const double* __restrict__ C, int64_t mo, int64_t ao, int64_t ld,
                                __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t n = ao * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = i / ld, m = i % ld;
    const double v = m < mo ? C[m * ao + a] : 0.0;
    const __nv_bfloat16 h = __double2bfloat16(v);
    hi[i] = h;
    lo[i] = __double2bfloat16(v - (double)__bfloat162float(h));
  }
}

inline int64_t up8(int64_t x) { return (x + 7) / 8 * 8; }
inline size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// The slices of the 5P rows for dL/dC: enough problems to fill the GPU with
// the N tiles of one problem, each slice a multiple of 64 rows (one K block).
struct Slices {
  int64_t n, rows;  // slice count, rows per slice
};
Slices slices_for(int64_t R, int64_t n_tiles_n) {
  const int64_t want = std::max<int64_t>(1, (2 * (int64_t)device_sms() + n_tiles_n - 1) / n_tiles_n);
  int64_t per = (R + want - 1) / want;
  per = std::max<int64_t>(1024, (per + 63) / 64 * 64);
  return Slices{(R + per - 1) / per, per};
}

int bn_for(int64_t n) {
  // as few N tiles of at most 160 as possible, each a multiple of 16
  const int64_t tiles = (n + 159) / 160;
  const int64_t per = (n + tiles - 1) / tiles;
  return (int)((per + 15) / 16 * 16);
}

}  // namespace

size_t adjoint_tc_ct_bytes(int64_t mo_num, int64_t ao_num) {
  return 2 * up256(sizeof(__nv_bfloat16) * (size_t)ao_num * up8(mo_num));
}

cudaError_t launch_adjoint_ct_split(const double* C64, int64_t mo_num, int64_t ao_num,
                                    void* ct, cudaStream_t s) {
  const int64_t ld = up8(mo_num);
  __nv_bfloat16* hi = (__nv_bfloat16*)ct;
  __nv_bfloat16* lo = (__nv_bfloat16*)((unsigned char*)ct + up256(sizeof(__nv_bfloat16) * ao_num * ld));
  if (ao_num * ld == 0) return cudaSuccess;
  ct_split_kernel<<<grid_for(ao_num * ld), 256, 0, s>>>(C64, mo_num, ao_num, ld, hi, lo);
  return cudaGetLastError();
}

size_t adjoint_tc_scratch_bytes(int64_t rows, int64_t mo_num, int64_t ao_num) {
  const int64_t ldw = up8(mo_num), R = up8(rows);
  const int bn = bn_for(ao_num);
  const int64_t ntn = (ao_num + bn - 1) / bn;
  const Slices sl = slices_for(R, ntn);
  size_t b = 0;
  b += 2 * up256(sizeof(__nv_bfloat16) * (size_t)rows * ldw);    // W hi/lo
  b += 2 * up256(sizeof(__nv_bfloat16) * (size_t)mo_num * R);    // W^T hi/lo
  b += 2 * up256(sizeof(__nv_bfloat16) * (size_t)ao_num * R);    // AO^T hi/lo
  b += up256(sizeof(float) * (size_t)sl.n * mo_num * ao_num);    // dL/dC partials
  b += up256(sizeof(TcProblem) * (size_t)sl.n);                  // problem descriptors
  b += up256(sizeof(int4) * (size_t)sl.n * ntn * ((mo_num + kTileRows - 1) / kTileRows));
  return b;
}

cudaError_t launch_adjoint_tc(const float* W, int64_t rows, int64_t mo_num, const float* ao,
                              int64_t ld_ao, int64_t ao_num, const void* ct, float* abar,
                              double* d_dC, const int* col_map, void* scratch, int* err_flag,
                              cudaStream_t s) {
  if (rows == 0 || mo_num == 0 || ao_num == 0) return cudaSuccess;
  if (rows > INT32_MAX || ao_num > INT32_MAX) return cudaErrorInvalidValue;
  const int64_t ldw = up8(mo_num), R = up8(rows);
  const int bn = bn_for(ao_num);
  const int64_t ntn = (ao_num + bn - 1) / bn;
  const Slices sl = slices_for(R, ntn);
  unsigned char* p = (unsigned char*)scratch;
  auto take = [&](size_t bytes) {
    unsigned char* q = p;
    p += up256(bytes);
    return q;
  };
  __nv_bfloat16* w_hi = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * rows * ldw);
  __nv_bfloat16* w_lo = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * rows * ldw);
  __nv_bfloat16* wt_hi = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * mo_num * R);
  __nv_bfloat16* wt_lo = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * mo_num * R);
  __nv_bfloat16* at_hi = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * ao_num * R);
  __nv_bfloat16* at_lo = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * ao_num * R);
  float* part = (float*)take(sizeof(float) * sl.n * mo_num * ao_num);
  TcProblem* probs = (TcProblem*)take(sizeof(TcProblem) * sl.n);
  int4* items = (int4*)take(sizeof(int4) * sl.n * ntn * ((mo_num + kTileRows - 1) / kTileRows));
  const __nv_bfloat16* ct_hi = (const __nv_bfloat16*)ct;
  const __nv_bfloat16* ct_lo =
      (const __nv_bfloat16*)((const unsigned char*)ct + up256(sizeof(__nv_bfloat16) * ao_num * ldw));

  // operands in bf16 hi/lo planes
  split_rows_kernel<<<grid_for(rows * ldw / 2), 256, 0, s>>>(W, rows, mo_num, mo_num, ldw, w_hi,
                                                            w_lo);
  auto aligned16 = [](const float* q, int64_t ld) {
    return ((uintptr_t)q & 15) == 0 && ld % 4 == 0;
  };
  const dim3 tw((unsigned)((R + 63) / 64), (unsigned)((mo_num + 63) / 64));
  transpose_split_kernel<<<tw, 256, 0, s>>>(W, rows, mo_num, mo_num, R, aligned16(W, mo_num),
                                            wt_hi, wt_lo);
  const dim3 ta((unsigned)((R + 63) / 64), (unsigned)((ao_num + 63) / 64));
  transpose_split_kernel<<<ta, 256, 0, s>>>(ao, rows, ao_num, ld_ao, R, aligned16(ao, ld_ao),
                                            at_hi, at_lo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  // Abar [rows][ao_num] = W . C
  AOTensor wv{};
  wv.a = w_hi;
  wv.a_lo = w_lo;
  wv.rows = rows;
  wv.ld = ldw;
  TcConfig cfg = tc_default_config(QK_BF16X3, ao_num);
  e = launch_mo_tc(QK_BF16X3, wv, mo_num, ct_hi, ct_lo, ldw, ao_num, abar, cfg, err_flag, s,
                   rows);
  if (e != cudaSuccess) return e;
  if (!d_dC) return cudaSuccess;

  // dL/dC partials: one problem per slice of rows
  std::vector<TcProblem> hp((size_t)sl.n);
  std::vector<int4> hi_items;
  for (int64_t k = 0; k < sl.n; ++k) {
    const int64_t r0 = k * sl.rows, r1 = std::min(R, r0 + sl.rows);
    AOTensor a{};
    a.a = wt_hi + r0;
    a.a_lo = wt_lo + r0;
    a.rows = mo_num;
    a.ld = R;
    if (!tc_make_problem(QK_BF16X3, a, r1 - r0, at_hi + r0, at_lo + r0, R, ao_num,
                         part + k * mo_num * ao_num, bn, mo_num, &hp[(size_t)k]))
      return cudaErrorInvalidValue;
    for (int64_t m = 0; m < (mo_num + kTileRows - 1) / kTileRows; ++m)
      for (int64_t n = 0; n < ntn; ++n) hi_items.push_back(make_int4((int)k, (int)m, (int)n, 0));
  }
  e = cudaMemcpyAsync(probs, hp.data(), sizeof(TcProblem) * hp.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(items, hi_items.data(), sizeof(int4) * hi_items.size(),
                        cudaMemcpyHostToDevice, s);
  // (copies from pageable host memory are staged before the call returns,
  // so the host vectors may go out of scope)
  if (e != cudaSuccess) return e;
  e = launch_mo_tc_batch(QK_BF16X3, 160, probs, items, (int64_t)hi_items.size(), err_flag, s);
  if (e != cudaSuccess) return e;
  return launch_reduce_partials_f32(part, (int)sl.n, mo_num * ao_num, d_dC, s, col_map, ao_num);
}

}  // namespace qk
