// mo_sparse64.cu -- the FP64 MO contraction over the block-sparse AO tensor.
//
// Eqs. 5-7 in FP64, D[5P x N_mo] = AO[5P x N_ao] . C^T, restricted to what
// screening (Eq. 3) leaves: the AO tensor is in the tiled layout (25 points
// = 125 rows of a 128-row tile, 64-AO column chunks) and only the live 16-AO
// column groups of its live (tile, chunk) blocks are multiplied, as the
// sparse-AO MO product of Sec. 3.2 does; skipped terms are exact zeros.
//
// A CTA computes a 128-row x 64-column tile of D.  Per live column group it
// stages the 128 x 16 AO block (one contiguous 16 KB slice of the blocked
// layout; k-major in shared memory) and the 64 x 16 block of C in shared
// memory, double buffered so that the next group loads while this one is
// multiplied; each thread accumulates an 8-row x 4-column block in FP64
// registers.  The output rows go to the caller's points through the tile
// permutation.  Every product and sum is an FP64 fused multiply-add, in a
// fixed order (groups ascending, k ascending within a group).
#include "internal.h"

namespace qk {
namespace {

constexpr int kThreads = 256;
constexpr int kBN = 64;    // output columns per CTA
constexpr int kBK = 16;    // one column group

struct Sparse64Args {
  const double* A;        // tiled AO tensor, blocked: a 16-column group is one 16 KB slice
  const uint8_t* mask;    // [tiles][mask_ld(nchunk)] live column groups
  int nchunk;
  const double* C;        // [N][ldc] chunked columns (padding zero)
  int64_t ldc;
  int64_t N;
  double* D;              // [M][N]
  int64_t M;              // output rows (5 x points)
  const int32_t* perm;    // slot -> point (NULL: identity)
  int64_t m_tiles;
};

__global__ void __launch_bounds__(kThreads)
    mo_sparse64_kernel(const Sparse64Args a) {
  // staged blocks, double buffered: AO [2][16][128] and C [2][16][64]
  extern __shared__ __align__(16) double smem64[];
  double(*As)[kBK][kTileRows] = reinterpret_cast<double(*)[kBK][kTileRows]>(smem64);
  double(*Cs)[kBK][kBN] = reinterpret_cast<double(*)[kBK][kBN]>(smem64 + 2 * kBK * kTileRows);
  __shared__ uint8_t gm[256];  // this tile's mask byte per chunk
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;  // 16 x 16 threads
  const int n0 = blockIdx.x * kBN;
  griddep_wait();
  for (int64_t mt = blockIdx.y; mt < a.m_tiles; mt += gridDim.y) {
    __syncthreads();  // previous tile's readers of gm are done
    const int mld = mask_ld(a.nchunk);
    for (int q = tid; q < a.nchunk; q += kThreads) gm[q] = a.mask[mt * mld + q] & 0xFu;
    __syncthreads();
    double acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    // walk the live groups: (q, g) pairs in ascending order
    int q = 0, g = -1;
    auto next_group = [&](int& qq, int& gg) -> bool {
      for (;;) {
        ++gg;
        if (gg == 4) {
          gg = 0;
          ++qq;
        }
        if (qq >= a.nchunk) return false;
        if ((gm[qq] >> gg) & 1u) return true;
      }
    };
    // staging of one group into buffer b (k-major): AO rows r of the tile,
    // columns 64 q + 16 g + k; C rows n0 + n, same columns
    auto stage = [&](int b, int qq, int gg) {
      const int64_t col = (int64_t)qq * kChunkAO + 16 * gg;
      {
        // 128 rows x 16 columns (one contiguous slice): thread -> row tid / 2,
        // columns 8 (tid & 1) .. + 7
        const int r = tid >> 1, k0 = (tid & 1) * 8;
        const double2* src = reinterpret_cast<const double2*>(
            a.A + blocked_offset(mt, qq, a.nchunk, 1, 0, r, 16 * gg + k0, 8));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double2 v = src[k];
          As[b][k0 + 2 * k][r] = v.x;
          As[b][k0 + 2 * k + 1][r] = v.y;
        }
      }
      {
        // 64 rows x 16 columns: thread -> row tid / 4, columns 4 (tid & 3) .. + 3
        const int n = tid >> 2, k0 = (tid & 3) * 4;
        const int64_t row = n0 + n;
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        if (row < a.N) {
          const double2* src = reinterpret_cast<const double2*>(a.C + row * a.ldc + col + k0);
          const double2 v0 = src[0], v1 = src[1];
          v[0] = v0.x;
          v[1] = v0.y;
          v[2] = v1.x;
          v[3] = v1.y;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) Cs[b][k0 + k][n] = v[k];
      }
    };
    bool have = next_group(q, g);
    int buf = 0;
    if (have) stage(0, q, g);
    __syncthreads();
    while (have) {
      int q2 = q, g2 = g;
      const bool more = next_group(q2, g2);
      if (more) stage(buf ^ 1, q2, g2);  // the next group loads while this one multiplies
#pragma unroll
      for (int k = 0; k < kBK; ++k) {
        double av[8], cv[4];
        const double2* ap = reinterpret_cast<const double2*>(&As[buf][k][ty * 8]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const double2 t = ap[i];
          av[2 * i] = t.x;
          av[2 * i + 1] = t.y;
        }
        const double2* cp = reinterpret_cast<const double2*>(&Cs[buf][k][tx * 4]);
        const double2 c0 = cp[0], c1 = cp[1];
        cv[0] = c0.x;
        cv[1] = c0.y;
        cv[2] = c1.x;
        cv[3] = c1.y;
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], cv[j], acc[i][j]);
      }
      __syncthreads();
      buf ^= 1;
      q = q2;
      g = g2;
      have = more;
    }
    // epilogue: rows 8 ty .. + 7 of the tile, columns n0 + 4 tx .. + 3
    const int64_t row0 = mt * (5 * kTilePoints);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int loc = ty * 8 + i;
      const int64_t lin = row0 + loc;
      if (loc >= 5 * kTilePoints || lin >= a.M) continue;
      const int64_t orow = a.perm ? 5 * (int64_t)a.perm[lin / 5] + lin % 5 : lin;
      double* dst = a.D + orow * a.N;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t col = n0 + 4 * tx + j;
        if (col < a.N) dst[col] = acc[i][j];
      }
    }
  }
}

}  // namespace

cudaError_t launch_mo_sparse64(const AOTensor& ao, const double* C, int64_t ldc, int64_t N,
                               double* D, int64_t out_rows, cudaStream_t s) {
  if (!ao.tiled || !ao.blocked || ao.comps == 1) return cudaErrorInvalidValue;
  if (ao.nchunk > 256) return cudaErrorInvalidValue;
  const int64_t m_tiles = ao.rows / kTileRows;
  if (m_tiles == 0 || N == 0) return cudaSuccess;
  Sparse64Args a;
  a.A = static_cast<const double*>(ao.a);
  a.mask = ao.mask;
  a.nchunk = ao.nchunk;
  a.C = C;
  a.ldc = ldc;
  a.N = N;
  a.D = D;
  a.M = out_rows;
  a.perm = ao.perm;
  a.m_tiles = m_tiles;
  const int64_t nt = (N + kBN - 1) / kBN;
  if (nt > 65535) return cudaErrorInvalidValue;
  // enough CTAs for a few waves; each walks M tiles
  const int64_t want = 8 * (int64_t)device_sms();
  int64_t gy = (want + nt - 1) / nt;
  if (gy > m_tiles) gy = m_tiles;
  if (gy > 65535) gy = 65535;
  constexpr size_t smem = sizeof(double) * 2 * kBK * (kTileRows + kBN);
  KernelFacts f;
  cudaError_t e = kernel_facts<mo_sparse64_kernel>(smem, kThreads, &f);
  if (e != cudaSuccess) return e;
  return launch_pdl(mo_sparse64_kernel, dim3((unsigned)nt, (unsigned)gy), kThreads, smem, s, a);
}

}  // namespace qk
