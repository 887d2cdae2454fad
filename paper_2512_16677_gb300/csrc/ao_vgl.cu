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
// loops over tiles of points (persistent in the point direction), with the
// chunk's shell, primitive and AO tables staged once in shared memory:
//   phase 0  the tile's point coordinates -> shared memory
//   phase 1  warps take shells from a shared counter, costliest first; one
//            lane per point: d = r - R_A, the shell radius test
//            (r^2 >= T/gamma_min screens every primitive), then the Eq. 3
//            test on primitives sorted by ascending exponent (the first
//            screened one ends the loop) gives S_0..S_2, and every Cartesian
//            component of the shell follows with compile-time exponents
//            into a shared staging tile [5 points][64 AOs]
//   phase 2  copy-out, converted to the output type: in the tiled layout a
//            lane takes 8 (bf16 planes) or 4 (FP32) consecutive columns of a
//            row and writes them with 16-byte stores, skipping dead 16-AO
//            groups; otherwise one warp per (point, component) row, lanes
//            over the 64 columns.
// In the contraction layout (AOTensor::chunked) chunk q owns the 64 columns
// [64q, 64q + 64) of the AO tensor, padding included, so each warp store is
// an aligned row segment, and the contraction's K blocks coincide with the
// chunks.  The caller-facing layout writes the AOs densely (column = AO
// index).
//
// Precision: FP64 mode does everything in FP64 and forms r^2 and gamma r^2
// without fused multiply-adds, so its screening decisions are those of the
// plain definition.  The reduced modes form d from float hi/lo pairs of the
// coordinates, then run exp and the assembly in FP32.
#include "ao_common.cuh"

namespace qk {
namespace {

constexpr int kThreads = 256;
static_assert(kTilePoints < kPT, "a tiled tile fits the 32 lanes of phase 1");

// Point lanes that own staging rows: 32-point tiles use every lane; 25-point
// tiles use 26, lane 25's zero rows doubling as the tile's rows 125..127.
template <bool kTiled>
constexpr int stage_lanes() {
  return kTiled ? kTilePoints + 1 : kPT;
}
template <typename T, bool kTiled>
using StageOf = AOStageSmem<T, stage_lanes<kTiled>()>;

// Chunk q of one problem over point tiles t_begin, t_begin + t_step, ...
// below t_end (the whole CTA calls this; it starts with a block barrier).
template <typename T, bool kSplit, bool kChunked, bool kTiled>
__device__ __forceinline__ void ao_chunk_tiles(const BasisDev& b, const PointsDev& pts,
                                               const AOTensor& out, int q, int64_t t_begin,
                                               int64_t t_end, int64_t t_step,
                                               StageOf<T, kTiled>& sh) {
  constexpr int TP = kTiled ? kTilePoints : kPT;  // points per tile
  constexpr int kWarps = kThreads / 32;
  using A = Arith<T>;
  __syncthreads();  // the previous call's readers of the shared tables are done
  const int4 ch = b.chunk[q];
  const int ns = ch.y - ch.x;
  const int na = ch.w - ch.z;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;

  // ---- chunk tables, once per call (static: they may load while the
  // previous kernel in the stream finishes)
  load_stage_tables(b, q, sh, tid, kThreads);
  griddep_wait();
  const T Tthr = A::thr(b);
  const int64_t n = pts.n;
  const int64_t col0 = kChunked ? (int64_t)q * kChunkAO : ch.z;

  // Tiles go in batches of 32: lane i of every warp reads the pre-pass's
  // reach word of tile base + i t_step, so that unreached blocks (most of
  // them) cost neither a barrier nor a dependent load each; their mask bytes
  // are written here.
  const bool culled = kTiled && out.reach != nullptr;
  for (int64_t base = t_begin; base < t_end; base += 32 * t_step) {
    const int64_t mine = base + (int64_t)lane * t_step;
    unsigned word = 0u, pword = 0u;
    if (mine < t_end) word = culled ? out.reach[mine * out.nchunk + q] : ~0u;
    // the partner tile's reach word (the contraction multiplies tiles 2i and
    // 2i + 1 together over the union of their live column groups)
    if (kTiled && culled && out.pair_zero && mine < t_end && (mine ^ 1) < t_end)
      pword = out.reach[(mine ^ 1) * out.nchunk + q];
    if (culled && warp == 0 && mine < t_end && word == 0u)
      out.mask[mine * mask_ld(out.nchunk) + q] = 0;
    unsigned todo = __ballot_sync(0xffffffffu, word != 0u);
    // warp 0 holds the next tile's points in registers, loaded while the
    // current tile is evaluated
    TilePoint<T> next;
    if (warp == 0 && todo)
      next = tile_point<T>(pts, lane, TP, (base + (int64_t)(__ffs(todo) - 1) * t_step) * TP);
    while (todo) {
      const int i = __ffs(todo) - 1;
      todo &= todo - 1u;
      const int64_t ptile = base + (int64_t)i * t_step;
      const int64_t p0 = ptile * TP;
      const unsigned pre = culled ? __shfl_sync(0xffffffffu, word, i) : ~0u;
      const unsigned ppre = __shfl_sync(0xffffffffu, pword, i);
      __syncthreads();  // tables ready / previous tile's copy-out done with the stage
      // ---- phase 0 (warp 0): the tile's points, its bounding box and the
      // shells that may reach it
      if (warp == 0) {
        const TilePoint<T> cur = next;
        if (todo)
          next = tile_point<T>(pts, lane, TP, (base + (int64_t)(__ffs(todo) - 1) * t_step) * TP);
        tile_reach(sh, cur, ns, lane, pre);
      }
      __syncthreads();
      const unsigned reach = sh.reach;
      if constexpr (kTiled) {
        if (reach == 0u) {  // no shell reaches the tile: block not written
          if (tid == 0) out.mask[ptile * mask_ld(out.nchunk) + q] = 0;
          continue;
        }
      }
      // ---- phase 1: warps take shells (costliest first), lanes are points;
      // culled shells only get their staging columns cleared
      const bool valid = lane < TP && p0 + lane < n;
      const int nwork = sh.nwork;
      unsigned groups = 0;  // warp-uniform: column groups this warp made nonzero
      for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(&sh.next, 1);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= nwork) break;
        const int sl = sh.work[k];
        if ((reach >> sl) & 1u) {
          if (shell_at_point(sh, sl, lane, valid, Tthr))
            groups |= shell_group_bits(sh.col[sl], sh.lsh[sl]);
        } else {
          shell_zero_columns(sh, sl, lane);
        }
      }
      if constexpr (kTiled) {
        if (lane == 0 && groups) atomicOr(&sh.gmask, groups);
      }
      __syncthreads();
      if constexpr (kTiled) {
        // mask byte: bit g set when column group g of block (tile, chunk) holds
        // an entry that survived screening; 0: block not written, the
        // contraction skips it
        const unsigned gm = sh.gmask;
        if (tid == 0) out.mask[ptile * mask_ld(out.nchunk) + q] = (uint8_t)gm;
        if (!gm) continue;
        // groups written: the live ones, plus (pairs) those the partner tile
        // may make live, which hold zeros here (their staging columns are
        // zero: no shell of theirs had a nonzero value at this tile)
        unsigned wm = gm;
        if (out.pair_zero) {
          const bool on = lane < ns && ((ppre >> lane) & 1u);
          const unsigned gb = on ? shell_group_bits(sh.col[lane], sh.lsh[lane]) : 0u;
          wm |= __reduce_or_sync(0xffffffffu, gb) & 0xFu;
        }
        // ---- phase 2, tiled: all 128 rows (stage rows 125..127 belong to the
        // lane past the tile and hold zeros) in 16-byte stores into the
        // block's 128-byte column slices; the columns of dead 16-AO groups
        // are not written (the contraction never reads them)
        if constexpr (kSplit) {
          // a lane splits 8 consecutive columns of one row into 16 bytes of each
          // bf16 plane: hi = rn(v), lo = rn(v - hi); a warp covers 4 rows
          const int rsub = lane >> 3, c8 = lane & 7;
          const bool store = (wm >> (c8 >> 1)) & 1u;
  #pragma unroll
          for (int it = 0; it < kTileRows / (4 * kWarps); ++it) {
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
              __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out.a) +
                                 blocked_offset(ptile, q, out.nchunk, 2, 0, r, 8 * c8, 2);
              *reinterpret_cast<uint4*>(o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              *reinterpret_cast<uint4*>(o + kBlockElems) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
          }
        } else if constexpr (sizeof(T) == 8) {
          // a lane stores 2 consecutive columns (16 bytes) of one row; a warp
          // covers a row
          const bool store = (wm >> (lane >> 3)) & 1u;
  #pragma unroll 4
          for (int it = 0; it < kTileRows / kWarps; ++it) {
            const int r = warp + kWarps * it;
            const double2 w = make_double2(sh.stage[r][2 * lane], sh.stage[r][2 * lane + 1]);
            if (store)
              *reinterpret_cast<double2*>(
                  static_cast<double*>(out.a) +
                  blocked_offset(ptile, q, out.nchunk, 1, 0, r, 2 * lane, 8)) = w;
          }
        } else {
          // a lane stores 4 consecutive columns of one row; a warp covers 2 rows
          const int rsub = lane >> 4, c4 = lane & 15;
          const bool store = (wm >> (c4 >> 2)) & 1u;
  #pragma unroll
          for (int it = 0; it < kTileRows / (2 * kWarps); ++it) {
            const int r = 2 * (warp + kWarps * it) + rsub;
            const float4 w = make_float4(sh.stage[r][4 * c4], sh.stage[r][4 * c4 + 1],
                                         sh.stage[r][4 * c4 + 2], sh.stage[r][4 * c4 + 3]);
            if (store)
              *reinterpret_cast<float4*>(
                  static_cast<float*>(out.a) +
                  blocked_offset(ptile, q, out.nchunk, 1, 0, r, 4 * c4, 4)) = w;
          }
        }
        continue;
      }
      // ---- phase 2: copy-out, one warp per row, lanes over columns lane and
      // lane + 32.
      constexpr int kRows = 5 * kPT;
      for (int r = warp; r < kRows; r += kWarps) {
        if (p0 + r / 5 >= n) break;
        const int64_t grow = 5 * p0 + r;
        const T v0 = sh.stage[r][lane];
        const T v1 = sh.stage[r][lane + 32];
        if constexpr (kSplit) {
          // hi = rn(v), lo = rn(v - hi), both columns at once
          const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
          const float2 hf = __bfloat1622float2(h);
          const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
          __nv_bfloat16* oh = static_cast<__nv_bfloat16*>(out.a) + grow * out.ld + col0;
          __nv_bfloat16* ol = static_cast<__nv_bfloat16*>(out.a_lo) + grow * out.ld + col0;
          oh[lane] = h.x;
          oh[lane + 32] = h.y;
          ol[lane] = l.x;
          ol[lane + 32] = l.y;
        } else {
          if constexpr (kChunked) {
            // chunk window: padding columns are written as zeros
            T* o = static_cast<T*>(out.a) + grow * out.ld + col0;
            o[lane] = v0;
            o[lane + 32] = v1;
          } else {
            T* o = static_cast<T*>(out.a) + grow * out.ld;
            const int* cmap = out.caller_cols ? b.ao_caller : nullptr;
            if (lane < na) o[cmap ? cmap[col0 + lane] : col0 + lane] = v0;
            if (lane + 32 < na) o[cmap ? cmap[col0 + lane + 32] : col0 + lane + 32] = v1;
          }
        }
      }
    }
  }
}

template <typename T, bool kSplit, bool kChunked, bool kTiled>
__global__ void __launch_bounds__(kThreads)
    ao_vgl_kernel(BasisDev b, PointsDev pts, AOTensor out, int64_t n_ptiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sh = *reinterpret_cast<StageOf<T, kTiled>*>(smem_raw);
  // CTAs start in grid order with the last chunk first: the internal shell
  // order puts the diffuse shells, whose chunks reach the most tiles, at the
  // end, so the longest CTAs start early and the tail is made of short ones
  ao_chunk_tiles<T, kSplit, kChunked, kTiled>(b, pts, out, b.nchunk - 1 - (int)blockIdx.y,
                                              blockIdx.x, n_ptiles, gridDim.x, sh);
}

// Several problems in one persistent launch: CTAs stride over a work list of
// (problem, chunk, first tile, end tile), longest first.
template <bool kSplit>
__global__ void __launch_bounds__(kThreads)
    ao_vgl_batch_kernel(const AOProblem* __restrict__ probs, const int4* __restrict__ items,
                        int64_t n_items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sh = *reinterpret_cast<StageOf<float, true>*>(smem_raw);
  for (int64_t i = blockIdx.x; i < n_items; i += gridDim.x) {
    const int4 w = items[i];
    const AOProblem& P = probs[w.x];
    const int64_t tiles = (P.p.n + kTilePoints - 1) / kTilePoints;
    ao_chunk_tiles<float, kSplit, true, true>(P.b, P.p, P.out, w.y, w.z, tiles, w.w, sh);
  }
}

// Pre-pass of the tiled layout: one warp per 25-point tile forms the tile's
// bounding box (float hi parts of the coordinates) and, for every chunk,
// the bit mask of the chunk's shells that may reach it (shell_reaches_box,
// the test ao_vgl applies itself when no table is given).  Each block first
// copies the shells' centres and radii^2 into shared memory (when they fit).
constexpr int kReachThreads = 256;
constexpr int kReachSmemShells = 8192;  // 128 KB of float4

// Tiles first, first + step, ... of one problem, one warp each.
__device__ __forceinline__ void reach_tiles(const BasisDev& b, const PointsDev& pts,
                                            uint32_t* reach, int64_t tiles, bool staged,
                                            const float4* shell_tab, int64_t first,
                                            int64_t step) {
  const int lane = threadIdx.x & 31;
  for (int64_t t = first; t < tiles; t += step) {
    const int64_t ip = t * kTilePoints + lane;
    const bool pv = lane < kTilePoints && ip < pts.n;
    float x = 0.0f, y = 0.0f, z = 0.0f;
    if (pv) {
      x = pts.hi[ip];
      y = pts.hi[pts.ld + ip];
      z = pts.hi[2 * pts.ld + ip];
    }
    float lo[3], hi[3];
    warp_box(pv, x, y, z, lo, hi);
    for (int q = 0; q < b.nchunk; ++q) {
      const int4 ch = b.chunk[q];
      const int s = ch.x + lane;
      bool keep = false;
      if (s < ch.y) {
        float4 c;
        if (staged) {
          c = shell_tab[s];
        } else {
          const int A = b.shell_nuc[s];
          c = make_float4(b.nucl_hi[3 * A], b.nucl_hi[3 * A + 1], b.nucl_hi[3 * A + 2],
                          b.shell_r2_f[s]);
        }
        keep = shell_reaches_box(lo, hi, c.x, c.y, c.z, c.w);
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) reach[t * b.nchunk + q] = m;
    }
  }
}

// The shells' centres and radii^2 into shared memory.
__device__ __forceinline__ void stage_shells(const BasisDev& b, float4* shell_tab) {
  for (int s = threadIdx.x; s < b.shell_num; s += blockDim.x) {
    const int A = b.shell_nuc[s];
    shell_tab[s] = make_float4(b.nucl_hi[3 * A], b.nucl_hi[3 * A + 1], b.nucl_hi[3 * A + 2],
                               b.shell_r2_f[s]);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kReachThreads)
    tile_reach_kernel(BasisDev b, PointsDev pts, uint32_t* reach, int64_t tiles, int staged) {
  extern __shared__ float4 shell_tab[];  // [shell] (X, Y, Z, r2max), float
  griddep_wait();
  if (staged) stage_shells(b, shell_tab);
  const int64_t warps = blockDim.x >> 5;
  reach_tiles(b, pts, reach, tiles, staged != 0, shell_tab,
              blockIdx.x * warps + (threadIdx.x >> 5), (int64_t)gridDim.x * warps);
}

// Several problems: blockIdx.y is the problem; a problem's table is staged
// when it has at most `cap` shells.
__global__ void __launch_bounds__(kReachThreads)
    tile_reach_batch_kernel(const AOProblem* probs, int cap) {
  extern __shared__ float4 shell_tab[];
  griddep_wait();
  const AOProblem& P = probs[blockIdx.y];
  if (P.out.reach == nullptr) return;
  const int64_t tiles = (P.p.n + kTilePoints - 1) / kTilePoints;
  const bool staged = P.b.shell_num <= cap;
  if (staged) stage_shells(P.b, shell_tab);
  const int64_t warps = blockDim.x >> 5;
  reach_tiles(P.b, P.p, P.out.reach, tiles, staged, shell_tab,
              blockIdx.x * warps + (threadIdx.x >> 5), (int64_t)gridDim.x * warps);
}

cudaError_t launch_tile_reach(const BasisDev& b, const PointsDev& p, uint32_t* reach,
                              int64_t tiles, cudaStream_t s) {
  const int staged = b.shell_num <= kReachSmemShells ? 1 : 0;
  const size_t smem = staged ? sizeof(float4) * (size_t)b.shell_num : 0;
  KernelFacts f;
  cudaError_t e = kernel_facts<tile_reach_kernel>(sizeof(float4) * kReachSmemShells,
                                                  kReachThreads, &f);
  if (e != cudaSuccess) return e;
  // a few blocks per SM, each staging the table once and walking tiles
  const int64_t want = (tiles + 7) / 8;
  const int64_t blocks = want < 4 * (int64_t)f.sms ? want : 4 * (int64_t)f.sms;
  return launch_pdl(tile_reach_kernel, (unsigned)(blocks > 0 ? blocks : 1), kReachThreads, smem, s,
                    b, p, reach, tiles, staged);
}

cudaError_t launch_tile_reach_batch_impl(const AOProblem* d_probs, int nprob, int64_t max_tiles,
                                         int max_shells, cudaStream_t s) {
  if (nprob < 1 || nprob > 65535 || max_tiles == 0) return cudaSuccess;
  const int cap = max_shells < kReachSmemShells ? max_shells : kReachSmemShells;
  const size_t smem = sizeof(float4) * (size_t)cap;
  KernelFacts f;
  cudaError_t e = kernel_facts<tile_reach_batch_kernel>(sizeof(float4) * kReachSmemShells,
                                                        kReachThreads, &f);
  if (e != cudaSuccess) return e;
  // about four blocks per SM over all problems, each walking its problem's tiles
  int64_t gx = (4 * (int64_t)f.sms + nprob - 1) / nprob;
  const int64_t want = (max_tiles + 7) / 8;
  if (gx > want) gx = want;
  if (gx < 1) gx = 1;
  return launch_pdl(tile_reach_batch_kernel, dim3((unsigned)gx, (unsigned)nprob), kReachThreads,
                    smem, s, d_probs, cap);
}

template <typename T, bool kSplit, bool kChunked, bool kTiled = false>
cudaError_t launch_ao(const BasisDev& b, const PointsDev& p, const AOTensor& out,
                      cudaStream_t s) {
  constexpr size_t smem = sizeof(StageOf<T, kTiled>);
  constexpr int TP = kTiled ? kTilePoints : kPT;
  auto kern = ao_vgl_kernel<T, kSplit, kChunked, kTiled>;
  KernelFacts f;
  cudaError_t e = kernel_facts<ao_vgl_kernel<T, kSplit, kChunked, kTiled>>(smem, kThreads, &f);
  if (e != cudaSuccess) return e;
  const int64_t n_ptiles = (p.n + TP - 1) / TP;
  if (n_ptiles == 0 || b.nchunk == 0) return cudaSuccess;
  if (kTiled && out.reach) {
    e = launch_tile_reach(b, p, out.reach, n_ptiles, s);
    if (e != cudaSuccess) return e;
  }
  const int occ = f.occ < 1 ? 1 : f.occ, sms = f.sms;
  // about four waves of resident CTAs, each CTA walking several point tiles
  int64_t gy = ((int64_t)sms * occ * 4 + b.nchunk - 1) / b.nchunk;
  if (gy > n_ptiles) gy = n_ptiles;
  if (b.nchunk > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)gy, (unsigned)b.nchunk);
  return launch_pdl(kern, grid, kThreads, smem, s, b, p, out, n_ptiles);
}

template <bool kSplit>
cudaError_t launch_ao_batch(const AOProblem* probs, const int4* items, int64_t n_items,
                            cudaStream_t s) {
  constexpr size_t smem = sizeof(StageOf<float, true>);
  auto kern = ao_vgl_batch_kernel<kSplit>;
  KernelFacts f;
  cudaError_t e = kernel_facts<ao_vgl_batch_kernel<kSplit>>(smem, kThreads, &f);
  if (e != cudaSuccess) return e;
  if (n_items == 0) return cudaSuccess;
  const int occ = f.occ < 1 ? 1 : f.occ, sms = f.sms;
  const int64_t grid = n_items < (int64_t)sms * occ ? n_items : (int64_t)sms * occ;
  return launch_pdl(kern, (unsigned)grid, kThreads, smem, s, probs, items, n_items);
}

}  // namespace

cudaError_t launch_tile_reach_batch(const AOProblem* d_probs, int nprob, int64_t max_tiles,
                                    int max_shells, cudaStream_t s) {
  return launch_tile_reach_batch_impl(d_probs, nprob, max_tiles, max_shells, s);
}

cudaError_t launch_ao_vgl_batch(bool split, const AOProblem* probs, const int4* items,
                                int64_t n_items, cudaStream_t s) {
  return split ? launch_ao_batch<true>(probs, items, n_items, s)
               : launch_ao_batch<false>(probs, items, n_items, s);
}

cudaError_t launch_ao_vgl(const BasisDev& b, const PointsDev& p, int out_mode,
                          const AOTensor& out, cudaStream_t s) {
  if (out.tiled) {
    if (!out.blocked || !out.chunked) return cudaErrorInvalidValue;  // the one tiled vgl layout
    switch (out_mode) {
      case QK_FP64:
        return launch_ao<double, false, true, true>(b, p, out, s);
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

// Nonzero (point, AO) pairs of a tiled (blocked) vgl AO tensor: the AO of a point
// counts when any of its five rows holds a nonzero entry at that column
// (either bf16 plane when split; the sign bit ignored; kEs bytes per entry).  Blocks whose mask
// byte is zero, and the dead 16-AO groups of live blocks, were not written
// and count nothing.  Statistics only.
template <int kEs>
__global__ void __launch_bounds__(256)
    ao_nnz_kernel(AOTensor t, int64_t n, int64_t tiles, unsigned long long* out) {
  __shared__ unsigned long long tot;
  if (threadIdx.x == 0) tot = 0ull;
  __syncthreads();
  unsigned cnt = 0;
  const int64_t blocks = tiles * t.nchunk;
  for (int64_t bi = blockIdx.x; bi < blocks; bi += gridDim.x) {
    const int64_t tile = bi / t.nchunk;
    const int q = (int)(bi % t.nchunk);
    const unsigned gm = t.mask[tile * mask_ld(t.nchunk) + q];
    if (gm == 0) continue;
    const int64_t left = n - tile * kTilePoints;
    const int pts = left < kTilePoints ? (int)left : kTilePoints;
    for (int i = threadIdx.x; i < pts * kChunkAO; i += blockDim.x) {
      const int j = i / kChunkAO, c = i % kChunkAO;
      if (!((gm >> (c >> 4)) & 1u)) continue;  // dead groups are not written
      bool nz = false;
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        const int64_t e =
            blocked_offset(tile, q, t.nchunk, kEs == 2 ? 2 : 1, 0, 5 * j + r, c, kEs);
        if constexpr (kEs == 2) {
          nz |= (static_cast<const uint16_t*>(t.a)[e] & 0x7fffu) != 0u;
          nz |= (static_cast<const uint16_t*>(t.a)[e + kBlockElems] & 0x7fffu) != 0u;
        } else if constexpr (kEs == 4) {
          nz |= (static_cast<const uint32_t*>(t.a)[e] & 0x7fffffffu) != 0u;
        } else {
          nz |= (static_cast<const uint64_t*>(t.a)[e] & 0x7fffffffffffffffull) != 0ull;
        }
      }
      cnt += nz ? 1u : 0u;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&tot, (unsigned long long)cnt);
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(out, tot);
}

cudaError_t launch_ao_nnz(const AOTensor& t, int es, int64_t n, unsigned long long* out,
                          cudaStream_t s) {
  if (!t.tiled || !t.blocked) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + kTilePoints - 1) / kTilePoints;
  const int64_t blocks = tiles * t.nchunk;
  if (blocks == 0) return cudaSuccess;
  const unsigned g = (unsigned)(blocks < 8 * (int64_t)device_sms() ? blocks
                                                                    : 8 * (int64_t)device_sms());
  if (es == 2)
    ao_nnz_kernel<2><<<g, 256, 0, s>>>(t, n, tiles, out);
  else if (es == 4)
    ao_nnz_kernel<4><<<g, 256, 0, s>>>(t, n, tiles, out);
  else
    ao_nnz_kernel<8><<<g, 256, 0, s>>>(t, n, tiles, out);
  return cudaGetLastError();
}


__global__ void points_soa_kernel(const double* raw, char transp, int64_t n, double* x,
                                  double* y, double* z, float* hi, float* lo) {
  griddep_wait();
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
  return launch_pdl(points_soa_kernel, (unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s, raw,
                    transp, n, x, y, z, hi, lo);
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
