// adjoint.cu -- nuclear-coordinate part of the MO vgl adjoint.
//
// For L = sum_{p,c,i} W[p][c][i] mo_vgl[p][c][i] (Eqs. 5-7) the gradient with
// respect to nucleus A is
//   dL/dR_A = - sum_p sum_{k on A} ( Abar_v grad chi_k
//                                    + sum_i Abar_i grad d_i chi_k
//                                    + Abar_lap grad lap chi_k ),
//   Abar[p][c][k] = sum_i W[p][c][i] C_ik,
// since an AO on A depends on r - R_A only.  This needs AO derivatives up to
// third order (Sec. 3.6 notes that forces need them).  They are recomputed
// here, never stored: with S_m = sum_k c_k gamma_k^m e^{-gamma_k r^2}
// (m = 0..3), d_j S_m = -2 d_j S_{m+1}, and P = X(dx) Y(dy) Z(dz),
//   d_j chi        = M (P_j S0 - 2 d_j P S1)
//   d_j d_i chi    = M (P_ij S0 - 2 (d_i P_j + d_j P_i) S1 - 2 delta_ij P S1
//                       + 4 d_i d_j P S2)
//   d_j lap chi    = M ((lapP)_j S0 - 2 d_j lapP S1 - 2(2l+3) P_j S1
//                       + (4(2l+3) + 8) d_j P S2 + 4 r^2 P_j S2 - 8 r^2 d_j P S3)
// (the Laplacian of Eq. 1 uses d . grad P = l P for the homogeneous P).
//
// Dense Abar (FP64, FP32): one CTA covers 32 points x one AO column chunk;
// each warp handles the 32 points of one shell, reduces over them with
// shuffles and adds into a per-shell accumulator that only it writes, so
// the sum order is fixed.  Abar in live (tile, chunk) blocks (split bf16):
// one CTA per chunk walks the tiles where the chunk is live, lists the
// (point, shell) pairs inside the shell's radius, gives each its own
// shared slot and sums the slots per shell in point order.  Either way the
// per-CTA shell sums go to a partial buffer; two small kernels then sum the
// partials over point-tile blocks and over the shells of each nucleus, in
// fixed orders.
#include "ao_common.cuh"

namespace qk {
namespace {


constexpr int kThreads = 256;
constexpr int kMaxTileBlocks = 512;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The gradient terms of shell s at point ip: g += sum over the shell's AOs
// j of M_j (Abar_v grad chi + sum_i Abar_i grad d_i chi + Abar_lap grad lap
// chi), with ab0 the Abar entry (value component) of the shell's first AO
// and ld the distance between components.
template <typename T>
__device__ __forceinline__ void dR_point_shell(const BasisDev& b, const PointsDev& pts,
                                               int64_t ip, int s, const T* ab0, int64_t ld,
                                               T Tthr, T g[3]) {
  using A = Arith<T>;
  T dx, dy, dz;
  A::diff(b, pts, ip, b.shell_nuc[s], dx, dy, dz);
  const T r2 = A::add(A::add(A::mul(dx, dx), A::mul(dy, dy)), A::mul(dz, dz));
  T S0 = T(0), S1 = T(0), S2 = T(0), S3 = T(0);
  if (r2 < A::r2max(b, s)) {
    const int k0 = b.shell_prim0[s];
    const int k1 = k0 + b.shell_nprim[s];
    for (int k = k0; k < k1; ++k) {
      const T gm = A::gam(b, k);
      const T t = A::mul(gm, r2);
      if (!(t < Tthr)) break;
      const T ce = A::coef(b, k) * A::ex(-t);
      S0 += ce;
      S1 += gm * ce;
      S2 += gm * gm * ce;
      S3 += gm * gm * gm * ce;
    }
  }
  if (S0 == T(0) && S1 == T(0) && S2 == T(0) && S3 == T(0)) return;
  const int l = b.shell_l[s];
  const int ao0 = b.shell_ao0[s];
  const int nc = (l + 1) * (l + 2) / 2;
  const T d[3] = {dx, dy, dz};
  const T x2 = dx * dx, y2 = dy * dy, z2 = dz * dz;
  const T k1 = T(2 * (2 * l + 3));
  for (int j = 0; j < nc; ++j) {
    const int a = c_pow[l][j][0], bb = c_pow[l][j][1], c = c_pow[l][j][2];
    // 1-D factors of P and their derivatives up to third order
    const T X[4] = {sel4(a, T(1), dx, x2, x2 * dx), sel4(a, T(0), T(1), T(2) * dx, T(3) * x2),
                    sel4(a, T(0), T(0), T(2), T(6) * dx), sel4(a, T(0), T(0), T(0), T(6))};
    const T Y[4] = {sel4(bb, T(1), dy, y2, y2 * dy), sel4(bb, T(0), T(1), T(2) * dy, T(3) * y2),
                    sel4(bb, T(0), T(0), T(2), T(6) * dy), sel4(bb, T(0), T(0), T(0), T(6))};
    const T Z[4] = {sel4(c, T(1), dz, z2, z2 * dz), sel4(c, T(0), T(1), T(2) * dz, T(3) * z2),
                    sel4(c, T(0), T(0), T(2), T(6) * dz), sel4(c, T(0), T(0), T(0), T(6))};
    const T P = X[0] * Y[0] * Z[0];
    const T Pi[3] = {X[1] * Y[0] * Z[0], X[0] * Y[1] * Z[0], X[0] * Y[0] * Z[1]};
    // Pij[i][j] symmetric
    const T Pxx = X[2] * Y[0] * Z[0], Pyy = X[0] * Y[2] * Z[0], Pzz = X[0] * Y[0] * Z[2];
    const T Pxy = X[1] * Y[1] * Z[0], Pxz = X[1] * Y[0] * Z[1], Pyz = X[0] * Y[1] * Z[1];
    const T Pij[3][3] = {{Pxx, Pxy, Pxz}, {Pxy, Pyy, Pyz}, {Pxz, Pyz, Pzz}};
    const T lapP = Pxx + Pyy + Pzz;
    const T lapPj[3] = {X[3] * Y[0] * Z[0] + X[1] * Y[2] * Z[0] + X[1] * Y[0] * Z[2],
                        X[2] * Y[1] * Z[0] + X[0] * Y[3] * Z[0] + X[0] * Y[1] * Z[2],
                        X[2] * Y[0] * Z[1] + X[0] * Y[2] * Z[1] + X[0] * Y[0] * Z[3]};
    const T M = A::aofac(b, ao0 + j);
    const T* ab = ab0 + j;
    const T Av = ab[0], Ag[3] = {ab[ld], ab[2 * ld], ab[3 * ld]}, Al = ab[4 * ld];
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) {
      const T dj = d[jj];
      T G = Av * (Pi[jj] * S0 - T(2) * dj * P * S1);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const T h = Pij[i][jj] * S0 - T(2) * (d[i] * Pi[jj] + dj * Pi[i]) * S1 +
                    T(4) * d[i] * dj * P * S2 - (i == jj ? T(2) * P * S1 : T(0));
        G += Ag[i] * h;
      }
      const T tl = lapPj[jj] * S0 - T(2) * dj * lapP * S1 - k1 * Pi[jj] * S1 +
                   (T(2) * k1 + T(8)) * dj * P * S2 + T(4) * r2 * Pi[jj] * S2 -
                   T(8) * r2 * dj * P * S3;
      G += Al * tl;
      g[jj] += M * G;
    }
  }
}

// Abar dense [5P][ld] in the points' order: CTA (chunk, point-tile block y)
// over point tiles y, y + gridDim.y, ...
template <typename T>
__global__ void __launch_bounds__(kThreads)
    adjoint_dR_kernel(BasisDev b, PointsDev pts, const T* __restrict__ abar, int64_t ld,
                      double* __restrict__ partial, int64_t n_ptiles) {
  using A = Arith<T>;
  __shared__ double s_acc[kChunkAO * 3];
  const int4 ch = b.chunk[blockIdx.x];
  const int ns = ch.y - ch.x;
  for (int i = threadIdx.x; i < kChunkAO * 3; i += kThreads) s_acc[i] = 0.0;
  __syncthreads();
  const T Tthr = A::thr(b);
  const int lane = threadIdx.x & 31;

  for (int64_t ptile = blockIdx.y; ptile < n_ptiles; ptile += gridDim.y) {
    const int64_t p0 = ptile * kPT;
    // kPT == 32 and kThreads % 32 == 0: each warp iteration is one shell
    for (int idx = threadIdx.x; idx < kPT * ns; idx += kThreads) {
      const int pl = idx % kPT;
      const int sl = idx / kPT;
      const int64_t ip = p0 + pl;
      const int s = ch.x + sl;
      T g[3] = {T(0), T(0), T(0)};
      if (ip < pts.n) dR_point_shell(b, pts, ip, s, abar + 5 * ip * ld + b.shell_ao0[s], ld, Tthr, g);
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) g[jj] = warp_sum(g[jj]);
      if (lane == 0) {
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) s_acc[3 * sl + jj] += (double)g[jj];
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ns * 3; i += kThreads)
    partial[((int64_t)blockIdx.y * b.shell_num + ch.x) * 3 + i] = s_acc[i];
}

// Abar in live (tile, chunk) blocks [tiles][nchunk][128][64] (FP32), the
// points in the tiles' order (25 per tile, rows 5 j + c): CTA (chunk,
// block y) over the tiles y, y + gridDim.y, ... where the chunk is live.
// Per tile the (point, shell) pairs that pass the radius test are listed
// first, so that the threads take only pairs with work (about a third of a
// live block's pairs on a chain); each pair's gradient goes to its own
// shared slot and the slots are added per shell in point order.
constexpr int kBlkThreads = 128;
__global__ void __launch_bounds__(kBlkThreads, 8)
    adjoint_dR_blocked_kernel(BasisDev b, PointsDev pts, const float* __restrict__ abar,
                              const uint8_t* __restrict__ mask, int64_t tiles,
                              double* __restrict__ partial) {
  using A = Arith<float>;
  __shared__ double s_acc[kMaxShellsChunk * 3];
  __shared__ float gbuf[kMaxShellsChunk][kTilePoints][3];
  __shared__ uint16_t list[kMaxShellsChunk * kTilePoints];
  __shared__ int cnt;
  const int q = blockIdx.x;
  const int4 ch = b.chunk[q];
  const int ns = ch.y - ch.x;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < kMaxShellsChunk * 3; i += kBlkThreads) s_acc[i] = 0.0;
  const float Tthr = A::thr(b);
  const int mld = mask_ld(b.nchunk);

  for (int64_t t = blockIdx.y; t < tiles; t += gridDim.y) {
    if (!(mask[t * mld + q] & 0xFu)) continue;  // no AO of the chunk reaches the tile
    const float* blk = abar + (t * b.nchunk + q) * (int64_t)(kTileRows * kChunkAO);
    __syncthreads();  // the previous tile's slots are summed
    if (tid == 0) cnt = 0;
    for (int i = tid; i < ns * kTilePoints * 3; i += kBlkThreads) (&gbuf[0][0][0])[i] = 0.0f;
    __syncthreads();
    // pairs that pass the radius test (the same test the gradient makes)
    for (int base = 0; base < ns * kTilePoints; base += kBlkThreads) {
      const int idx = base + tid;
      bool pass = false;
      int pl = 0, sl = 0;
      if (idx < ns * kTilePoints) {
        pl = idx % kTilePoints;
        sl = idx / kTilePoints;
        const int64_t ip = t * kTilePoints + pl;
        if (ip < pts.n) {
          const int s = ch.x + sl;
          float dx, dy, dz;
          A::diff(b, pts, ip, b.shell_nuc[s], dx, dy, dz);
          const float r2 = A::add(A::add(A::mul(dx, dx), A::mul(dy, dy)), A::mul(dz, dz));
          pass = r2 < A::r2max(b, s);
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, pass);
      int at = 0;
      if (lane == 0 && bal) at = atomicAdd(&cnt, __popc(bal));
      at = __shfl_sync(0xffffffffu, at, 0);
      if (pass) list[at + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)(pl | (sl << 5));
    }
    __syncthreads();
    const int n_pairs = cnt;
    for (int k = tid; k < n_pairs; k += kBlkThreads) {
      const int e = list[k];
      const int pl = e & 31, sl = e >> 5;
      const int s = ch.x + sl;
      float g[3] = {0.0f, 0.0f, 0.0f};
      dR_point_shell(b, pts, t * kTilePoints + pl, s,
                     blk + 5 * pl * kChunkAO + (b.shell_ao0[s] - ch.z), (int64_t)kChunkAO, Tthr, g);
      gbuf[sl][pl][0] = g[0];
      gbuf[sl][pl][1] = g[1];
      gbuf[sl][pl][2] = g[2];
    }
    __syncthreads();
    for (int i = tid; i < ns * 3; i += kBlkThreads) {
      const int sl = i / 3, ax = i % 3;
      float sum = 0.0f;
#pragma unroll 5
      for (int pl = 0; pl < kTilePoints; ++pl) sum += gbuf[sl][pl][ax];
      s_acc[i] += (double)sum;
    }
  }
  __syncthreads();
  for (int i = tid; i < ns * 3; i += kBlkThreads)
    partial[((int64_t)blockIdx.y * b.shell_num + ch.x) * 3 + i] = s_acc[i];
}

// Shell totals: sum over the point-tile blocks in a fixed order.  A CTA of
// 32 x 16 threads covers 32 (shell, axis) columns: row ty sums the blocks
// ty, ty + 16, ... in order, then the 16 row sums are added in order, so
// the result does not depend on the schedule.  Shells not touched by any
// block (none here: every chunk writes all its shells) stay 0.
constexpr int kSumCols = 32, kSumRows = 16;
__global__ void __launch_bounds__(kSumCols * kSumRows)
    dR_shell_sum_kernel(const double* partial, int blocks, int shell_num, double* shell_tot) {
  __shared__ double red[kSumRows][kSumCols];
  const int tx = threadIdx.x % kSumCols, ty = threadIdx.x / kSumCols;
  const int i = blockIdx.x * kSumCols + tx;
  const int n = shell_num * 3;
  double s = 0.0;
  if (i < n)
    for (int y = ty; y < blocks; y += kSumRows) s += partial[(int64_t)y * n + i];
  red[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && i < n) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < kSumRows; ++k) t += red[k][tx];
    shell_tot[i] = t;
  }
}

// dR[A][j] = - sum over shells of A: a warp per (A, j), lane i adding the
// shells i, i + 32, ... of A in order, then a fixed shuffle tree.
__global__ void dR_nucleus_sum_kernel(const double* shell_tot, const int* shell_nuc,
                                      int shell_num, int nucl_num, double* dR) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nucl_num * 3) return;  // whole warps leave together
  const int A = w / 3, j = w % 3;
  double s = 0.0;
  for (int sh = lane; sh < shell_num; sh += 32)
    if (shell_nuc[sh] == A) s += shell_tot[3 * sh + j];
  s = warp_sum(s);
  if (lane == 0) dR[w] = -s;
}

// Partials [blocks][shell][3] -> shell totals -> d_dR [nucl][3].
cudaError_t reduce_dR(const BasisDev& b, double* partial, int blocks, double* d_dR,
                      cudaStream_t s) {
  double* shell_tot = partial + (size_t)3 * b.shell_num * blocks;
  dR_shell_sum_kernel<<<(b.shell_num * 3 + kSumCols - 1) / kSumCols, kSumCols * kSumRows, 0, s>>>(
      partial, blocks, b.shell_num, shell_tot);
  dR_nucleus_sum_kernel<<<(b.nucl_num * 3 + 7) / 8, 256, 0, s>>>(shell_tot, b.shell_nuc,
                                                                 b.shell_num, b.nucl_num, d_dR);
  return cudaGetLastError();
}

int tile_blocks(int64_t point_num) {
  const int64_t t = (point_num + kPT - 1) / kPT;
  return (int)(t < kMaxTileBlocks ? (t > 0 ? t : 1) : kMaxTileBlocks);
}

}  // namespace

size_t adjoint_dR_partial_bytes(const BasisDev& b, int64_t point_num) {
  return sizeof(double) * 3 * (size_t)b.shell_num * ((size_t)tile_blocks(point_num) + 1);
}

cudaError_t launch_adjoint_dR(const BasisDev& b, const PointsDev& p, int mode, const void* abar,
                              int64_t ld, double* partial, double* d_dR, cudaStream_t s) {
  const int blocks = tile_blocks(p.n);
  const int64_t n_ptiles = (p.n + kPT - 1) / kPT;
  if (b.nchunk == 0) return cudaSuccess;
  dim3 grid((unsigned)b.nchunk, (unsigned)blocks);
  if (mode == QK_FP64)
    adjoint_dR_kernel<double><<<grid, kThreads, 0, s>>>(b, p, (const double*)abar, ld, partial,
                                                        n_ptiles);
  else
    adjoint_dR_kernel<float><<<grid, kThreads, 0, s>>>(b, p, (const float*)abar, ld, partial,
                                                       n_ptiles);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return reduce_dR(b, partial, blocks, d_dR, s);
}

cudaError_t launch_adjoint_dR_blocked(const BasisDev& b, const PointsDev& p, const float* abar,
                                      const uint8_t* mask, double* partial, double* d_dR,
                                      cudaStream_t s) {
  // point-tile blocks as for the dense kernel (the partial buffer's size);
  // never more than the 25-point tiles
  const int blocks = tile_blocks(p.n);
  const int64_t tiles = (p.n + kTilePoints - 1) / kTilePoints;
  if (b.nchunk == 0 || p.n == 0) return cudaSuccess;
  dim3 grid((unsigned)b.nchunk, (unsigned)blocks);
  adjoint_dR_blocked_kernel<<<grid, kBlkThreads, 0, s>>>(b, p, abar, mask, tiles, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return reduce_dR(b, partial, blocks, d_dR, s);
}

}  // namespace qk
