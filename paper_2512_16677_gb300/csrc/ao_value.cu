// ao_value.cu -- atomic-orbital values only, for the density on a grid
// (Sec. 5.4: orbitals evaluated at grid points, no derivatives).
//
// chi_n = M_n P(d) S_0, S_0 = sum_k c_k exp(-gamma_k r^2) over the primitives
// that pass Eq. 3 (Eqs. 1, 2, 4).  One row per point, so a 128-row
// contraction tile holds 128 points; chunk q owns columns [64q, 64q + 64)
// as in the vgl layout.
//
// A CTA owns one chunk and walks tiles of 128 points in four groups of 32:
//   phase 0  warps 0-3 load a group each and form its bounding box; warp 0
//            marks, per group, the shells whose screening sphere reaches
//            the box (as ao_vgl does per tile) and lists the (shell, group)
//            items to visit, costliest shells first
//   phase 1  warps take items: a lane per point of the group, the radial
//            sum and every Cartesian component of the shell with
//            compile-time exponents, into a shared staging tile [128][65];
//            unreached items only clear their columns, and only when an
//            earlier tile left values there
//   phase 2  copy-out of the 128 rows (bf16 hi/lo planes or FP32 / FP64;
//            tiled: 16-byte stores per lane, dead 16-AO groups skipped).
// Tiled output (tensor-core modes) writes live (tile, chunk) blocks only and
// a mask byte per block; the dense output (FP64 / FP32 modes) writes every
// row below the point count.
#include "ao_common.cuh"

namespace qk {
namespace {

constexpr int kThreads = 256;
constexpr int kGroups = 4;
constexpr int kTP = 32 * kGroups;  // points per tile = rows per tile

template <typename T>
struct AOValueSmem {
  using value_type = T;
  static constexpr int kRows = kTP;
  T nuc[kMaxShellsChunk][3];
  T nuc_lo[kMaxShellsChunk][3];
  T r2max[kMaxShellsChunk];
  T g[kMaxPrimsChunk];
  T c[kMaxPrimsChunk];
  T M[kChunkAO];
  T pt[kTP][3];
  T pt_lo[kTP][3];
  T box[kGroups][6];
  int prim0[kMaxShellsChunk];
  int nprim[kMaxShellsChunk];
  int col[kMaxShellsChunk];
  int lsh[kMaxShellsChunk];
  int order[kMaxShellsChunk];
  unsigned char dirty[kMaxShellsChunk];  // set by the table loader; unused here
  // gdirty[g][s]: group g's staging columns of shell s may hold values (one
  // byte each: warps on different groups of a shell update them at once)
  unsigned char gdirty[kGroups][kMaxShellsChunk];
  unsigned reach[kGroups];
  unsigned gmask;  // bit g: 16-AO column group g holds a nonzero entry
  int work[kMaxShellsChunk * kGroups];   // shell | group << 8
  int nwork;
  int next;
  T stage[kTP][kStagePitch];
};

// Values of component J.. of a momentum-L shell at one point.
template <typename T, int L, int J>
__device__ __forceinline__ void cart_values(const T (&px)[4], const T (&py)[4], const T (&pz)[4],
                                            const T* M, T S0, T* st) {
  if constexpr (J < (L + 1) * (L + 2) / 2) {
    constexpr int a = cart_exp(L, J, 0), b = cart_exp(L, J, 1), c = cart_exp(L, J, 2);
    st[J] = M[J] * S0 * (px[a] * py[b] * pz[c]);
    cart_values<T, L, J + 1>(px, py, pz, M, S0, st);
  }
}

template <typename T, int L>
__device__ __forceinline__ void shell_values(T dx, T dy, T dz, T S0, const T* M, T* st) {
  const T x2 = dx * dx, y2 = dy * dy, z2 = dz * dz;
  const T px[4] = {T(1), dx, x2, x2 * dx};
  const T py[4] = {T(1), dy, y2, y2 * dy};
  const T pz[4] = {T(1), dz, z2, z2 * dz};
  cart_values<T, L, 0>(px, py, pz, M, S0, st);
}

template <typename T>
__device__ __forceinline__ void clear_columns(AOValueSmem<T>& sh, int sl, int grp, int lane) {
  if (!sh.gdirty[grp][sl]) return;
  const int l = sh.lsh[sl];
  const int nc = (l + 1) * (l + 2) / 2;
  T* st = &sh.stage[32 * grp + lane][sh.col[sl]];
  for (int j = 0; j < nc; ++j) st[j] = T(0);
  __syncwarp();
  if (lane == 0) sh.gdirty[grp][sl] = 0;
}

// Shell sl at point 32 grp + lane of the tile; returns, on every lane,
// whether the S_0 of any lane was nonzero.
template <typename T>
__device__ __forceinline__ bool shell_value_at_point(AOValueSmem<T>& sh, int sl, int grp,
                                                     int lane, bool valid, T Tthr) {
  using A = Arith<T>;
  const int pl = 32 * grp + lane;
  T dx = T(0), dy = T(0), dz = T(0), S0 = T(0);
  if (valid) {
    if constexpr (sizeof(T) == 8) {
      dx = __dsub_rn(sh.pt[pl][0], sh.nuc[sl][0]);
      dy = __dsub_rn(sh.pt[pl][1], sh.nuc[sl][1]);
      dz = __dsub_rn(sh.pt[pl][2], sh.nuc[sl][2]);
    } else {
      dx = (sh.pt[pl][0] - sh.nuc[sl][0]) + (sh.pt_lo[pl][0] - sh.nuc_lo[sl][0]);
      dy = (sh.pt[pl][1] - sh.nuc[sl][1]) + (sh.pt_lo[pl][1] - sh.nuc_lo[sl][1]);
      dz = (sh.pt[pl][2] - sh.nuc[sl][2]) + (sh.pt_lo[pl][2] - sh.nuc_lo[sl][2]);
    }
    const T r2 = A::add(A::add(A::mul(dx, dx), A::mul(dy, dy)), A::mul(dz, dz));
    if (r2 < sh.r2max[sl]) {
      const int k0 = sh.prim0[sl];
      const int k1 = k0 + sh.nprim[sl];
      for (int k = k0; k < k1; ++k) {
        const T t = A::mul(sh.g[k], r2);
        if (!(t < Tthr)) break;  // ascending exponents: the rest is screened too
        S0 += sh.c[k] * A::ex(-t);
      }
    }
  }
  const bool nz = S0 != T(0);
  const bool any = __any_sync(0xffffffffu, nz);
  if (any) {
    const int c0 = sh.col[sl];
    T* st = &sh.stage[pl][c0];
    const T* M = &sh.M[c0];
    switch (sh.lsh[sl]) {
      case 0: shell_values<T, 0>(dx, dy, dz, S0, M, st); break;
      case 1: shell_values<T, 1>(dx, dy, dz, S0, M, st); break;
      case 2: shell_values<T, 2>(dx, dy, dz, S0, M, st); break;
      default: shell_values<T, 3>(dx, dy, dz, S0, M, st); break;
    }
    if (lane == 0) sh.gdirty[grp][sl] = 1;
  } else {
    clear_columns(sh, sl, grp, lane);
  }
  return any;
}

template <typename T, bool kSplit, bool kTiled>
__global__ void __launch_bounds__(kThreads)
    ao_value_kernel(BasisDev b, PointsDev pts, AOTensor out, int64_t n_tiles) {
  using A = Arith<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AOValueSmem<T>& sh = *reinterpret_cast<AOValueSmem<T>*>(smem_raw);
  // the last chunks (diffuse shells: the longest CTAs) start first
  const int q = b.nchunk - 1 - (int)blockIdx.y;
  const int4 ch = b.chunk[q];
  const int ns = ch.y - ch.x;
  const int na = ch.w - ch.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kThreads / 32;
  load_stage_tables(b, q, sh, tid, kThreads);
  griddep_wait();  // the points are the previous kernel's output
  for (int i = tid; i < ns; i += kThreads)
    for (int g = 0; g < kGroups; ++g) sh.gdirty[g][i] = 1;  // the stage holds anything
  const T Tthr = A::thr(b);
  const int64_t n = pts.n;
  const int64_t col0 = (int64_t)q * kChunkAO;

  // warps 0..3 hold their group's points of the next tile in registers,
  // loaded while the current tile is evaluated
  TilePoint<T> next;
  if (warp < kGroups && (int64_t)blockIdx.x < n_tiles)
    next = tile_point<T>(pts, lane, 32, (int64_t)blockIdx.x * kTP + 32 * warp);
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t p0 = tile * kTP;
    __syncthreads();  // tables ready / previous tile's copy-out done
    // ---- phase 0: points and group boxes
    if (warp < kGroups) {
      const int pl = 32 * warp + lane;
      const TilePoint<T> P = next;
      if (tile + gridDim.x < n_tiles)
        next = tile_point<T>(pts, lane, 32, (tile + gridDim.x) * kTP + 32 * warp);
      const bool pv = P.pv;
      const T x = P.x, y = P.y, z = P.z;
      if (pv) {
        if constexpr (sizeof(T) != 8) {
          sh.pt_lo[pl][0] = P.lx;
          sh.pt_lo[pl][1] = P.ly;
          sh.pt_lo[pl][2] = P.lz;
        }
        sh.pt[pl][0] = x;
        sh.pt[pl][1] = y;
        sh.pt[pl][2] = z;
      }
      T lo[3], hi[3];
      warp_box(pv, x, y, z, lo, hi);
      if (lane == 0)
        for (int k = 0; k < 3; ++k) {
          sh.box[warp][k] = lo[k];
          sh.box[warp][3 + k] = hi[k];
        }
    }
    __syncthreads();
    if (warp == 0) {
      unsigned rg[kGroups];
#pragma unroll
      for (int g = 0; g < kGroups; ++g) {
        const T lo[3] = {sh.box[g][0], sh.box[g][1], sh.box[g][2]};
        const T hi[3] = {sh.box[g][3], sh.box[g][4], sh.box[g][5]};
        const bool keep = lane < ns && shell_reaches_box(lo, hi, sh.nuc[lane][0],
                                                         sh.nuc[lane][1], sh.nuc[lane][2],
                                                         sh.r2max[lane]);
        rg[g] = __ballot_sync(0xffffffffu, keep);
      }
      // items of the lane-th costliest shell, then their places in the list
      int sl = 0, cnt = 0;
      unsigned mine = 0;
      if (lane < ns) {
        sl = sh.order[lane];
#pragma unroll
        for (int g = 0; g < kGroups; ++g)
          if (((rg[g] >> sl) & 1u) || sh.gdirty[g][sl]) {
            mine |= 1u << g;
            ++cnt;
          }
      }
      int pos = cnt;  // inclusive scan over lanes
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pos, o);
        if (lane >= o) pos += v;
      }
      int w = pos - cnt;
#pragma unroll
      for (int g = 0; g < kGroups; ++g)
        if ((mine >> g) & 1u) sh.work[w++] = sl | (g << 8);
      if (lane == 31) sh.nwork = pos;
      if (lane < kGroups) sh.reach[lane] = rg[lane];
      if (lane == 0) {
        sh.next = 0;
        sh.gmask = 0;
      }
    }
    __syncthreads();
    const bool reached = (sh.reach[0] | sh.reach[1] | sh.reach[2] | sh.reach[3]) != 0u;
    if constexpr (kTiled) {
      if (!reached) {  // no shell reaches any point of the tile: block not written
        if (tid == 0) out.mask[tile * mask_ld(out.nchunk) + q] = 0;
        continue;
      }
    }
    // ---- phase 1
    const int nwork = sh.nwork;
    unsigned groups = 0;  // warp-uniform: column groups this warp made nonzero
    for (;;) {
      int k = 0;
      if (lane == 0) k = atomicAdd(&sh.next, 1);
      k = __shfl_sync(0xffffffffu, k, 0);
      if (k >= nwork) break;
      const int item = sh.work[k];
      const int sl = item & 0xff, grp = item >> 8;
      const bool valid = p0 + 32 * grp + lane < n;
      if ((sh.reach[grp] >> sl) & 1u) {
        if (shell_value_at_point(sh, sl, grp, lane, valid, Tthr))
          groups |= shell_group_bits(sh.col[sl], sh.lsh[sl]);
      } else {
        clear_columns(sh, sl, grp, lane);
      }
    }
    if constexpr (kTiled) {
      if (lane == 0 && groups) atomicOr(&sh.gmask, groups);
    }
    __syncthreads();
    if constexpr (kTiled) {
      const unsigned gm = sh.gmask;  // the vgl layout's mask byte: live column groups
      if (tid == 0) out.mask[tile * mask_ld(out.nchunk) + q] = (uint8_t)gm;
      if (!gm) continue;
      // ---- phase 2, tiled: 16-byte stores, dead 16-AO groups not written
      // (the contraction never reads them), as in ao_vgl
      const int64_t row0 = tile * kTileRows;
      if constexpr (kSplit) {
        const int rsub = lane >> 3, c8 = lane & 7;
        const bool store = (gm >> (c8 >> 1)) & 1u;
#pragma unroll
        for (int it = 0; it < kTP / (4 * kWarps); ++it) {
          const int r = 4 * (warp + kWarps * it) + rsub;
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float v0 = sh.stage[r][8 * c8 + 2 * j];
            const float v1 = sh.stage[r][8 * c8 + 2 * j + 1];
            const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
            const float2 hf = __bfloat1622float2(h);
            const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
            memcpy(&hw[j], &h, 4);
            memcpy(&lw[j], &l, 4);
          }
          if (store) {
            const int64_t e = (row0 + r) * out.ld + col0 + 8 * c8;
            *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out.a) + e) =
                make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out.a_lo) + e) =
                make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
        }
      } else {
        const int rsub = lane >> 4, c4 = lane & 15;
        const bool store = (gm >> (c4 >> 2)) & 1u;
#pragma unroll
        for (int it = 0; it < kTP / (2 * kWarps); ++it) {
          const int r = 2 * (warp + kWarps * it) + rsub;
          const float4 w = make_float4(sh.stage[r][4 * c4], sh.stage[r][4 * c4 + 1],
                                       sh.stage[r][4 * c4 + 2], sh.stage[r][4 * c4 + 3]);
          if (store)
            *reinterpret_cast<float4*>(static_cast<float*>(out.a) + (row0 + r) * out.ld + col0 +
                                       4 * c4) = w;
        }
      }
      continue;
    }
    // ---- phase 2, dense: one warp per row, lanes over columns lane, lane + 32
    for (int r = warp; r < kTP; r += kWarps) {
      if (p0 + r >= n) break;
      const int64_t grow = p0 + r;
      const T v0 = sh.stage[r][lane];
      const T v1 = sh.stage[r][lane + 32];
      T* o = static_cast<T*>(out.a) + grow * out.ld + col0;
      o[lane] = v0;
      o[lane + 32] = v1;
    }
  }
  (void)na;
}

template <typename T, bool kSplit, bool kTiled>
cudaError_t launch_value(const BasisDev& b, const PointsDev& p, const AOTensor& out,
                         cudaStream_t s) {
  constexpr size_t smem = sizeof(AOValueSmem<T>);
  auto kern = ao_value_kernel<T, kSplit, kTiled>;
  KernelFacts f;
  cudaError_t e = kernel_facts<ao_value_kernel<T, kSplit, kTiled>>(smem, kThreads, &f);
  if (e != cudaSuccess) return e;
  const int64_t n_tiles = (p.n + kTP - 1) / kTP;
  if (n_tiles == 0 || b.nchunk == 0) return cudaSuccess;
  const int occ = f.occ < 1 ? 1 : f.occ, sms = f.sms;
  int64_t gy = ((int64_t)sms * occ * 4 + b.nchunk - 1) / b.nchunk;
  if (gy > n_tiles) gy = n_tiles;
  if (b.nchunk > 65535) return cudaErrorInvalidValue;
  return launch_pdl(kern, dim3((unsigned)gy, (unsigned)b.nchunk), kThreads, smem, s, b, p, out,
                    n_tiles);
}

}  // namespace

int ao_value_tile_points() { return kTP; }

cudaError_t launch_ao_value(const BasisDev& b, const PointsDev& p, int out_mode,
                            const AOTensor& out, cudaStream_t s) {
  if (out.tiled) {
    if (out_mode == QK_BF16X3) return launch_value<float, true, true>(b, p, out, s);
    if (out_mode == QK_TF32 || out_mode == QK_FP32)
      return launch_value<float, false, true>(b, p, out, s);
    return cudaErrorInvalidValue;
  }
  if (out_mode == QK_FP64) return launch_value<double, false, false>(b, p, out, s);
  if (out_mode == QK_FP32) return launch_value<float, false, false>(b, p, out, s);
  return cudaErrorInvalidValue;
}

}  // namespace qk
