// ao_vgl.cu -- atomic-orbital values, gradients and Laplacians at every point.
//
// Sec. 3.1 of the QMCkl paper: chi_n = M_n R_s P_abc (Eq. 1), a contracted
// Gaussian radial part (Eq. 2, p = 2), primitives skipped when
// gamma r^2 >= T (Eq. 3), Cartesian polynomial (Eq. 4) built from repeated
// products of the coordinate differences.
//
// For one (point, shell) the radial part and its derivatives need only
//   S_m = sum_k c_k gamma_k^m exp(-gamma_k r^2),  m = 0, 1, 2,  c_k = N_s a_k f_k
// because grad R = -2 d S_1 and lap R = 4 r^2 S_2 - 6 S_1.  With P
// homogeneous of degree l (d . grad P = l P):
//   chi   = M P S_0
//   d_i   = M (d_iP S_0 - 2 d_i P S_1)
//   lap   = M (lapP S_0 - 2 (2l+3) P S_1 + 4 r^2 P S_2)
//
// Work decomposition.  The AOs are cut into column chunks of at most 64 AOs
// and 32 shells that end on shell boundaries.  A CTA owns one chunk and
// loops over tiles of 32 points (persistent in the point direction), with the
// chunk's shell, primitive and AO tables staged once in shared memory:
//   phase 0  the tile's point coordinates -> shared memory
//   phase 1  one warp per shell, one lane per point: d = r - R_A, the shell
//            radius test (r^2 >= T/gamma_min screens every primitive), then
//            the Eq. 3 test on primitives sorted by ascending exponent (the
//            first screened one ends the loop); S_0..S_2 and d -> shared
//   phase 2  one lane per pair of AOs, one warp per point: assemble the five
//            components and store them.
// In the contraction layout (AOTensor::chunked) chunk q owns the 64 columns
// [64q, 64q + 64) of the AO tensor, padding included, so each warp store is
// one aligned 128-byte (bf16 plane) / 256-byte (FP32) / 512-byte (FP64) row
// segment, and the contraction's K blocks coincide with the chunks.  The
// caller-facing layout writes the AOs densely (column = AO index).
//
// Precision: FP64 mode does everything in FP64 and forms r^2 and gamma r^2
// without fused multiply-adds, so its screening decisions are those of the
// plain definition.  The reduced modes form d from float hi/lo pairs of the
// coordinates, then run exp and the assembly in FP32.
#include "ao_common.cuh"

namespace qk {
namespace {

constexpr int kThreads = 256;
constexpr int kPT = 32;  // points per tile: one lane per point in phase 1
static_assert(kTilePoints <= kPT, "a tiled tile fits the 32 lanes of phase 1");

// Shared memory of one CTA (templated on the arithmetic type).
template <typename T>
struct AOShared {
  // chunk tables (loaded once)
  T nuc[kMaxShellsChunk][3];     // FP64: R_A; FP32: float(R_A)
  T nuc_lo[kMaxShellsChunk][3];  // FP32: residual R_A - float(R_A)
  T r2max[kMaxShellsChunk];
  int prim0[kMaxShellsChunk];    // first primitive, local to the chunk
  int nprim[kMaxShellsChunk];
  T g[kMaxPrimsChunk];
  T c[kMaxPrimsChunk];
  T M[kChunkAO];
  int ao_info[kChunkAO];  // local shell | l << 8 | Cartesian index << 12
  // per tile: [point][shell] with one pad column, so that phase 1 (lanes over
  // points) and phase 2 (lanes over AOs of one point) hit distinct banks
  T pt[kPT][3];
  T pt_lo[kPT][3];
  T d[3][kPT][kMaxShellsChunk + 1];
  T S[3][kPT][kMaxShellsChunk + 1];
};

// Two adjacent AOs (local columns 2q, 2q+1) of one component row.
template <typename T, bool kSplit>
struct PairStore;

template <typename T>
struct PairStore<T, false> {
  static __device__ __forceinline__ void put(const AOTensor& o, int64_t row, int64_t col, T v0,
                                             T v1) {
    T* p = static_cast<T*>(o.a) + row * o.ld + col;
    if constexpr (sizeof(T) == 8)
      *reinterpret_cast<double2*>(p) = make_double2(v0, v1);
    else
      *reinterpret_cast<float2*>(p) = make_float2(v0, v1);
  }
};

template <>
struct PairStore<float, true> {
  static __device__ __forceinline__ void put(const AOTensor& o, int64_t row, int64_t col, float v0,
                                             float v1) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
    const int64_t off = row * o.ld + col;
    *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(o.a) + off) =
        __halves2bfloat162(h0, h1);
    *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(o.a_lo) + off) =
        __halves2bfloat162(l0, l1);
  }
};

// The five components of local AO `al` at tile point `pl`.
template <typename T>
__device__ __forceinline__ void assemble(const AOShared<T>& sh, int al, int pl, T out[5]) {
  const int info = sh.ao_info[al];
  const int sl = info & 0xff;
  const T S0 = sh.S[0][pl][sl], S1 = sh.S[1][pl][sl], S2 = sh.S[2][pl][sl];
  if (S0 == T(0) && S1 == T(0) && S2 == T(0)) {
#pragma unroll
    for (int c = 0; c < 5; ++c) out[c] = T(0);
    return;
  }
  const int l = (info >> 8) & 0xf;
  const int j = info >> 12;
  const T dx = sh.d[0][pl][sl], dy = sh.d[1][pl][sl], dz = sh.d[2][pl][sl];
  const int a = c_pow[l][j][0], bb = c_pow[l][j][1], c = c_pow[l][j][2];
  const T x2 = dx * dx, y2 = dy * dy, z2 = dz * dz;
  const T X = sel4(a, T(1), dx, x2, x2 * dx);
  const T Y = sel4(bb, T(1), dy, y2, y2 * dy);
  const T Z = sel4(c, T(1), dz, z2, z2 * dz);
  const T X1 = sel4(a, T(0), T(1), T(2) * dx, T(3) * x2);
  const T Y1 = sel4(bb, T(0), T(1), T(2) * dy, T(3) * y2);
  const T Z1 = sel4(c, T(0), T(1), T(2) * dz, T(3) * z2);
  const T X2 = sel4(a, T(0), T(0), T(2), T(6) * dx);
  const T Y2 = sel4(bb, T(0), T(0), T(2), T(6) * dy);
  const T Z2 = sel4(c, T(0), T(0), T(2), T(6) * dz);
  const T P = X * Y * Z;
  const T M = sh.M[al];
  const T r2 = x2 + y2 + z2;
  const T MS0 = M * S0;
  const T MS1x2 = T(2) * M * S1;
  out[0] = MS0 * P;
  out[1] = MS0 * (X1 * Y * Z) - MS1x2 * dx * P;
  out[2] = MS0 * (X * Y1 * Z) - MS1x2 * dy * P;
  out[3] = MS0 * (X * Y * Z1) - MS1x2 * dz * P;
  const T lapP = X2 * Y * Z + X * Y2 * Z + X * Y * Z2;
  out[4] = M * (lapP * S0 - T(2 * (2 * l + 3)) * P * S1 + T(4) * r2 * P * S2);
}

// Chunk q of one problem over point tiles t_begin, t_begin + t_step, ...
// below t_end (the whole CTA calls this; it starts with a block barrier).
template <typename T, bool kSplit, bool kChunked, bool kTiled>
__device__ __forceinline__ void ao_chunk_tiles(const BasisDev& b, const PointsDev& pts,
                                               const AOTensor& out, int q, int64_t t_begin,
                                               int64_t t_end, int64_t t_step, AOShared<T>& sh) {
  constexpr int TP = kTiled ? kTilePoints : kPT;  // points per tile
  using A = Arith<T>;
  __syncthreads();  // the previous call's readers of the shared tables are done
  const int4 ch = b.chunk[q];
  const int ns = ch.y - ch.x;
  const int na = ch.w - ch.z;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;

  // ---- chunk tables, once per CTA
  const int p_first = b.shell_prim0[ch.x];
  for (int i = tid; i < ns; i += kThreads) {
    const int s = ch.x + i;
    const int A_ = b.shell_nuc[s];
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int k = 0; k < 3; ++k) sh.nuc[i][k] = b.nucl_xyz[3 * A_ + k];
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        sh.nuc[i][k] = b.nucl_hi[3 * A_ + k];
        sh.nuc_lo[i][k] = b.nucl_lo[3 * A_ + k];
      }
    }
    sh.r2max[i] = A::r2max(b, s);
    sh.prim0[i] = b.shell_prim0[s] - p_first;
    sh.nprim[i] = b.shell_nprim[s];
  }
  const int np_chunk = b.shell_prim0[ch.y - 1] + b.shell_nprim[ch.y - 1] - p_first;
  for (int i = tid; i < np_chunk; i += kThreads) {
    sh.g[i] = A::gam(b, p_first + i);
    sh.c[i] = A::coef(b, p_first + i);
  }
  for (int i = tid; i < na; i += kThreads) {
    const int ao = ch.z + i;
    const int s = b.ao_shell[ao];
    sh.ao_info[i] = (s - ch.x) | (b.shell_l[s] << 8) | ((ao - b.shell_ao0[s]) << 12);
    sh.M[i] = A::aofac(b, ao);
  }
  const T Tthr = A::thr(b);
  const int64_t n = pts.n;
  const int64_t col0 = kChunked ? (int64_t)q * kChunkAO : ch.z;

  for (int64_t ptile = t_begin; ptile < t_end; ptile += t_step) {
    const int64_t p0 = ptile * TP;
    __syncthreads();  // tables ready / previous tile's phase 2 done with shared data
    // ---- phase 0: the tile's points
    if (tid < TP) {
      const int64_t ip = p0 + tid;
      if (ip < n) {
        if constexpr (sizeof(T) == 8) {
          sh.pt[tid][0] = pts.x[ip];
          sh.pt[tid][1] = pts.y[ip];
          sh.pt[tid][2] = pts.z[ip];
        } else {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            sh.pt[tid][k] = pts.hi[k * n + ip];
            sh.pt_lo[tid][k] = pts.lo[k * n + ip];
          }
        }
      }
    }
    __syncthreads();
    // ---- phase 1: one warp per shell, lanes over the tile's points
    int live = 0;
    for (int sl = warp; sl < ns; sl += kThreads / 32) {
      const int pl = lane;
      T dx = T(0), dy = T(0), dz = T(0), S0 = T(0), S1 = T(0), S2 = T(0);
      if (pl < TP && p0 + pl < n) {
        if constexpr (sizeof(T) == 8) {
          dx = __dsub_rn(sh.pt[pl][0], sh.nuc[sl][0]);
          dy = __dsub_rn(sh.pt[pl][1], sh.nuc[sl][1]);
          dz = __dsub_rn(sh.pt[pl][2], sh.nuc[sl][2]);
        } else {
          // hi parts cancel exactly when close; the residuals restore FP32
          // accuracy of the difference
          dx = (sh.pt[pl][0] - sh.nuc[sl][0]) + (sh.pt_lo[pl][0] - sh.nuc_lo[sl][0]);
          dy = (sh.pt[pl][1] - sh.nuc[sl][1]) + (sh.pt_lo[pl][1] - sh.nuc_lo[sl][1]);
          dz = (sh.pt[pl][2] - sh.nuc[sl][2]) + (sh.pt_lo[pl][2] - sh.nuc_lo[sl][2]);
        }
        const T r2 = A::add(A::add(A::mul(dx, dx), A::mul(dy, dy)), A::mul(dz, dz));
        if (r2 < sh.r2max[sl]) {
          const int k0 = sh.prim0[sl];
          const int k1 = k0 + sh.nprim[sl];
          for (int k = k0; k < k1; ++k) {
            const T gm = sh.g[k];
            const T t = A::mul(gm, r2);
            if (!(t < Tthr)) break;  // ascending exponents: the rest is screened too
            const T ce = sh.c[k] * A::ex(-t);
            S0 += ce;
            S1 += gm * ce;
            S2 += gm * gm * ce;
          }
        }
      }
      sh.d[0][pl][sl] = dx;
      sh.d[1][pl][sl] = dy;
      sh.d[2][pl][sl] = dz;
      sh.S[0][pl][sl] = S0;
      sh.S[1][pl][sl] = S1;
      sh.S[2][pl][sl] = S2;
      live |= (S0 != T(0) || S1 != T(0) || S2 != T(0));
    }
    // block barrier; in the tiled layout it also tells whether any entry of
    // block (tile, chunk) survived screening
    live = __syncthreads_or(live);
    if constexpr (kTiled) {
      if (tid == 0) out.mask[ptile * out.nchunk + q] = live ? 1 : 0;
      if (!live) continue;  // not written: the contraction skips this block
      // rows 125..127 of the tile are zero
      if (warp < kTileRows - 5 * kTilePoints) {
        const int64_t prow = ptile * kTileRows + 5 * kTilePoints + warp;
        PairStore<T, kSplit>::put(out, prow, col0 + 2 * lane, T(0), T(0));
      }
    }
    // ---- phase 2: one warp per point, lane = AO pair (2 lane, 2 lane + 1)
    for (int pl = warp; pl < TP; pl += kThreads / 32) {
      const int64_t ip = p0 + pl;
      if (ip >= n) break;
      const int a0 = 2 * lane, a1 = 2 * lane + 1;
      T v0[5], v1[5];
      if (a0 < na) {
        assemble(sh, a0, pl, v0);
      } else {
#pragma unroll
        for (int c = 0; c < 5; ++c) v0[c] = T(0);
      }
      if (a1 < na) {
        assemble(sh, a1, pl, v1);
      } else {
#pragma unroll
        for (int c = 0; c < 5; ++c) v1[c] = T(0);
      }
      const int64_t row = kTiled ? ptile * kTileRows + 5 * pl : 5 * ip;
      if constexpr (kChunked) {
        // chunk window: padding columns are written as zeros
#pragma unroll
        for (int c = 0; c < 5; ++c)
          PairStore<T, kSplit>::put(out, row + c, col0 + a0, v0[c], v1[c]);
      } else {
        T* o = static_cast<T*>(out.a);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          if (a0 < na) o[(row + c) * out.ld + col0 + a0] = v0[c];
          if (a1 < na) o[(row + c) * out.ld + col0 + a1] = v1[c];
        }
      }
    }
  }
}

template <typename T, bool kSplit, bool kChunked, bool kTiled>
__global__ void __launch_bounds__(kThreads)
    ao_vgl_kernel(BasisDev b, PointsDev pts, AOTensor out, int64_t n_ptiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AOShared<T>& sh = *reinterpret_cast<AOShared<T>*>(smem_raw);
  ao_chunk_tiles<T, kSplit, kChunked, kTiled>(b, pts, out, blockIdx.x, blockIdx.y, n_ptiles,
                                              gridDim.y, sh);
}

// Several problems in one persistent launch: CTAs stride over a work list of
// (problem, chunk, first tile, end tile), longest first.
template <bool kSplit>
__global__ void __launch_bounds__(kThreads)
    ao_vgl_batch_kernel(const AOProblem* __restrict__ probs, const int4* __restrict__ items,
                        int64_t n_items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AOShared<float>& sh = *reinterpret_cast<AOShared<float>*>(smem_raw);
  for (int64_t i = blockIdx.x; i < n_items; i += gridDim.x) {
    const int4 w = items[i];
    const AOProblem& P = probs[w.x];
    ao_chunk_tiles<float, kSplit, true, true>(P.b, P.p, P.out, w.y, w.z, w.w, 1, sh);
  }
}

template <typename T, bool kSplit, bool kChunked, bool kTiled = false>
cudaError_t launch_ao(const BasisDev& b, const PointsDev& p, const AOTensor& out,
                      cudaStream_t s) {
  constexpr size_t smem = sizeof(AOShared<T>);
  constexpr int TP = kTiled ? kTilePoints : kPT;
  auto kern = ao_vgl_kernel<T, kSplit, kChunked, kTiled>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t n_ptiles = (p.n + TP - 1) / TP;
  if (n_ptiles == 0 || b.nchunk == 0) return cudaSuccess;
  int occ = 1, sms = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
  if (occ < 1) occ = 1;
  // about four waves of resident CTAs, each CTA walking several point tiles
  int64_t gy = ((int64_t)sms * occ * 4 + b.nchunk - 1) / b.nchunk;
  if (gy > n_ptiles) gy = n_ptiles;
  if (gy > 65535) gy = 65535;
  dim3 grid((unsigned)b.nchunk, (unsigned)gy);
  kern<<<grid, kThreads, smem, s>>>(b, p, out, n_ptiles);
  return cudaGetLastError();
}

template <bool kSplit>
cudaError_t launch_ao_batch(const AOProblem* probs, const int4* items, int64_t n_items,
                            cudaStream_t s) {
  constexpr size_t smem = sizeof(AOShared<float>);
  auto kern = ao_vgl_batch_kernel<kSplit>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (n_items == 0) return cudaSuccess;
  int occ = 1, sms = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
  if (occ < 1) occ = 1;
  const int64_t grid = n_items < (int64_t)sms * occ ? n_items : (int64_t)sms * occ;
  kern<<<(unsigned)grid, kThreads, smem, s>>>(probs, items, n_items);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ao_vgl_batch(bool split, const AOProblem* probs, const int4* items,
                                int64_t n_items, cudaStream_t s) {
  return split ? launch_ao_batch<true>(probs, items, n_items, s)
               : launch_ao_batch<false>(probs, items, n_items, s);
}

cudaError_t launch_ao_vgl(const BasisDev& b, const PointsDev& p, int out_mode,
                          const AOTensor& out, cudaStream_t s) {
  if (out.tiled) {
    switch (out_mode) {
      case QK_FP32:
      case QK_TF32:
        return launch_ao<float, false, true, true>(b, p, out, s);
      case QK_BF16X3:
        return launch_ao<float, true, true, true>(b, p, out, s);
      default:
        return cudaErrorInvalidValue;
    }
  }
  if (out.chunked) {
    switch (out_mode) {
      case QK_FP64:
        return launch_ao<double, false, true>(b, p, out, s);
      case QK_FP32:
      case QK_TF32:
        return launch_ao<float, false, true>(b, p, out, s);
      case QK_BF16X3:
        return launch_ao<float, true, true>(b, p, out, s);
      default:
        return cudaErrorInvalidValue;
    }
  }
  switch (out_mode) {
    case QK_FP64:
      return launch_ao<double, false, false>(b, p, out, s);
    case QK_FP32:
    case QK_TF32:
      return launch_ao<float, false, false>(b, p, out, s);
    default:
      return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------ helpers ---

__global__ void points_soa_kernel(const double* raw, char transp, int64_t n, double* x,
                                  double* y, double* z, float* hi, float* lo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double c[3];
    if (transp == 'N') {
      c[0] = raw[3 * i + 0];
      c[1] = raw[3 * i + 1];
      c[2] = raw[3 * i + 2];
    } else {
      c[0] = raw[i];
      c[1] = raw[n + i];
      c[2] = raw[2 * n + i];
    }
    x[i] = c[0];
    y[i] = c[1];
    z[i] = c[2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float h = __double2float_rn(c[d]);
      hi[d * n + i] = h;
      lo[d * n + i] = __double2float_rn(c[d] - (double)h);
    }
  }
}

cudaError_t launch_points_soa(const double* raw, char transp, int64_t n, double* x, double* y,
                              double* z, float* hi, float* lo, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  points_soa_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(raw, transp, n, x,
                                                                              y, z, hi, lo);
  return cudaGetLastError();
}

// C [rows][cols] (FP64) -> the contraction's chunked column layout
// ([rows][nchunk*64], padding zeroed) as FP64, FP32 and bf16 hi/lo planes.
__global__ void mo_chunked_kernel(const double* src, int64_t rows, int64_t cols,
                                  const int4* chunk, int nchunk, double* d64, float* d32,
                                  __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const int64_t ld = (int64_t)nchunk * kChunkAO;
  const int64_t n = rows * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ld, col = i % ld;
    const int q = (int)(col / kChunkAO), loc = (int)(col % kChunkAO);
    const int4 ch = chunk[q];
    const double v = loc < ch.w - ch.z ? src[r * cols + ch.z + loc] : 0.0;
    d64[i] = v;
    d32[i] = __double2float_rn(v);
    const __nv_bfloat16 h = __double2bfloat16(v);
    hi[i] = h;
    lo[i] = __double2bfloat16(v - (double)__bfloat162float(h));
  }
}

cudaError_t launch_mo_chunked(const double* src, int64_t rows, int64_t cols, const int4* chunk,
                              int nchunk, double* d64, float* d32, __nv_bfloat16* hi,
                              __nv_bfloat16* lo, cudaStream_t s) {
  const int64_t n = rows * (int64_t)nchunk * kChunkAO;
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  mo_chunked_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(
      src, rows, cols, chunk, nchunk, d64, d32, hi, lo);
  return cudaGetLastError();
}

__global__ void split_bf16_kernel(const double* src, int64_t rows, int64_t cols, int64_t ld,
                                  __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const int64_t n = rows * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ld, c = i % ld;
    const double v = c < cols ? src[r * cols + c] : 0.0;
    const __nv_bfloat16 h = __double2bfloat16(v);
    hi[i] = h;
    lo[i] = __double2bfloat16(v - (double)__bfloat162float(h));
  }
}

cudaError_t launch_split_bf16(const double* src, int64_t rows, int64_t cols, int64_t ld,
                              __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t s) {
  const int64_t n = rows * ld;
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  split_bf16_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(src, rows, cols, ld,
                                                                              hi, lo);
  return cudaGetLastError();
}

__global__ void to_f32_kernel(const double* src, int64_t rows, int64_t cols, int64_t ld,
                              float* dst) {
  const int64_t n = rows * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ld, c = i % ld;
    dst[i] = c < cols ? __double2float_rn(src[r * cols + c]) : 0.0f;
  }
}

cudaError_t launch_to_f32(const double* src, int64_t rows, int64_t cols, int64_t ld, float* dst,
                          cudaStream_t s) {
  const int64_t n = rows * ld;
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  to_f32_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(src, rows, cols, ld,
                                                                          dst);
  return cudaGetLastError();
}

}  // namespace qk
