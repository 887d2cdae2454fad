// adjoint_sparse.cu -- the split-bf16 MO vgl adjoint over the forward pass's
// blocked, block-sparse AO tensor (Sec. 3.6 for what the adjoint needs,
// Eqs. 5-7 for the product it differentiates).
//
// For L = sum_{p,c,i} W[p][c][i] mo_vgl[p][c][i]:
//   dL/dC[i][k]   = sum_{p,c} W[p][c][i] AO[p][c][k]     (W^T . AO)
//   Abar[p][c][k] = sum_i W[p][c][i] C[i][k]             (W . C)
// and dL/dR from Abar (adjoint.cu).  Both products need the AO blocks that
// screening left live, nothing else:
//   * the AO tensor is the forward's own: tiles of 25 points in the spatial
//     order, 128 rows each (25 x 5 components, 3 zero rows), 64-AO chunks,
//     bf16 hi/lo planes per block, a mask byte of live 16-AO groups per
//     (tile, chunk).  Dead groups of live blocks are never written by the
//     forward (its contraction skips them); one pass zeroes them before they
//     enter a product here.
//   * W is gathered into the same tile rows and split into bf16 hi/lo.
//   * dL/dC^T[k][i] is accumulated on tcgen05 with A = the AO columns of
//     two chunks (M = 128, MN-major: a blocked slice holds 128-byte rows of
//     64 AOs per tensor row) and B = the W rows of the same tile (N = MOs,
//     MN-major), K = the tile's rows, over the tiles where either chunk is
//     live.  The tiles are cut into slices whose FP32 partials are added in
//     a fixed order (FP64) by a last small kernel.
//   * Abar is formed for live (tile, chunk) blocks only: A = the W rows of
//     the tile (K-major, K = MOs), B = the rows of C^T of up to four live
//     chunks of the tile (K-major, one MMA of N = 64 per chunk); each block
//     leaves through swizzled shared-memory staging and TMA tensor stores.
// The three split products hi.hi + hi.lo + lo.hi accumulate in FP32 in TMEM.
// Every wait is bounded; a wait that gives up records a code in the error
// word, stops the pipeline, lets the copies and MMAs in flight finish,
// frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "tc_common.cuh"

namespace qk {
namespace {

using namespace tc;

constexpr int kThreads = 192;               // warps 0-3 epilogue, 4 TMA, 5 MMA
constexpr size_t kSmemCap = 232448;         // opt-in shared memory per block
constexpr int kHalf = 64;                   // tile rows per dL/dC stage
constexpr uint32_t kSlice = kHalf * 128;    // one plane of a 64-wide atom: 8 KB
constexpr uint32_t kAtom = 2 * kSlice;      // hi + lo: 16 KB

inline int64_t up16(int64_t x) { return (x + 15) / 16 * 16; }
inline size_t up256(size_t x) { return (x + 255) / 256 * 256; }

unsigned grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// Shared-memory matrix descriptor, MN-major, 128-byte swizzle: rows of 64
// bf16 along M (or N) at 128-byte pitch, 8-row K groups 1024 bytes apart
// (SBO), 64-element M/N atoms `lbo` bytes apart (LBO); descriptor version 1,
// layout type 2 = SWIZZLE_128B.
__device__ __forceinline__ uint64_t sw128_desc_mn(uint32_t addr, uint32_t lbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor bits 15 / 16: A / B read MN-major.
constexpr uint32_t kAMajorMN = 1u << 15;
constexpr uint32_t kBMajorMN = 1u << 16;

// ---------------------------------------------------------------- set-up --

// Zero the dead 16-AO groups of live blocks (both planes, all 128 rows): a
// warp per block, 16-byte stores.
__global__ void zero_dead_groups_kernel(__nv_bfloat16* ao, const uint8_t* mask, int64_t tiles,
                                        int nchunk) {
  const int lane = threadIdx.x & 31;
  const int64_t nblk = tiles * nchunk;
  const int64_t step = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w < nblk;
       w += step) {
    const int64_t t = w / nchunk;
    const int q = (int)(w % nchunk);
    const unsigned m = mask[t * mask_ld(nchunk) + q] & 0xFu;
    if (m == 0u || m == 0xFu) continue;
    __nv_bfloat16* blk = ao + blocked_offset(t, q, nchunk, 2, 0, 0, 0, 2);
    // plane (2) x row (128) x 16-byte piece (8); piece c covers group c / 2
    for (int i = lane; i < 2 * kTileRows * 8; i += 32) {
      const int c = i & 7, r = (i >> 3) & (kTileRows - 1), pl = i >> 10;
      if ((m >> (c >> 1)) & 1u) continue;
      reinterpret_cast<uint4*>(blk + pl * kBlockElems + r * 64)[c] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

// W [P][5][mo] (FP32, the caller's points) -> bf16 hi/lo [tiles * 128][ldw]
// in the AO tensor's tile rows: row 128 t + 5 j + c holds component c of
// point perm[25 t + j] (perm NULL: that point itself).  Rows 125..127 of a
// tile, rows past the last point and columns past mo are zero.  A warp per
// row, lanes over column pairs (ldw is even), stored as bf16 pairs; the
// next row's point index is loaded while the current row is copied.
__device__ __forceinline__ const float* w_row(const float* W, const int32_t* perm, int64_t P,
                                              int64_t mo, int64_t row) {
  const int j = (int)(row % kTileRows);
  if (j >= 5 * kTilePoints) return nullptr;
  const int64_t s = row / kTileRows * kTilePoints + j / 5;
  if (s >= P) return nullptr;
  return W + (5 * (perm ? (int64_t)perm[s] : s) + j % 5) * mo;
}

__global__ void gather_split_w_kernel(const float* __restrict__ W, const int32_t* __restrict__ perm,
                                      int64_t P, int64_t mo, int64_t ldw, int64_t tiles,
                                      __nv_bfloat16* __restrict__ hi,
                                      __nv_bfloat16* __restrict__ lo) {
  const int lane = threadIdx.x & 31;
  const int64_t rows = tiles * kTileRows;
  const int64_t step = (int64_t)gridDim.x * (blockDim.x >> 5);
  const bool pairs = (mo & 1) == 0;  // rows start on 8-byte boundaries: float2 loads
  // rows on 16-byte boundaries and whole quads of columns: float4 loads
  const bool quads = (mo & 3) == 0 && (ldw & 3) == 0 && ((uintptr_t)W & 15) == 0;
  int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const float* src = row < rows ? w_row(W, perm, P, mo, row) : nullptr;
  for (; row < rows; row += step) {
    const int64_t nrow = row + step;
    const float* nsrc = nrow < rows ? w_row(W, perm, P, mo, nrow) : nullptr;
    if (quads) {
      // four columns per lane: one 16-byte load, 8 bytes into each plane
      uint2* oh = reinterpret_cast<uint2*>(hi + row * ldw);
      uint2* ol = reinterpret_cast<uint2*>(lo + row * ldw);
      for (int64_t c = 4 * lane; c < ldw; c += 128) {
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (src && c < mo) v = *reinterpret_cast<const float4*>(src + c);
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y);
        const __nv_bfloat162 h1 = __floats2bfloat162_rn(v.z, v.w);
        const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
        const __nv_bfloat162 l0 = __floats2bfloat162_rn(v.x - f0.x, v.y - f0.y);
        const __nv_bfloat162 l1 = __floats2bfloat162_rn(v.z - f1.x, v.w - f1.y);
        uint2 hw, lw;
        memcpy(&hw.x, &h0, 4);
        memcpy(&hw.y, &h1, 4);
        memcpy(&lw.x, &l0, 4);
        memcpy(&lw.y, &l1, 4);
        oh[c / 4] = hw;
        ol[c / 4] = lw;
      }
      src = nsrc;
      continue;
    }
    __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(hi + row * ldw);
    __nv_bfloat162* ol = reinterpret_cast<__nv_bfloat162*>(lo + row * ldw);
    for (int64_t c = 2 * lane; c < ldw; c += 64) {
      float v0 = 0.0f, v1 = 0.0f;
      if (src && c < mo) {
        if (pairs) {
          const float2 v = *reinterpret_cast<const float2*>(src + c);
          v0 = v.x;
          v1 = v.y;
        } else {
          v0 = src[c];
          if (c + 1 < mo) v1 = src[c + 1];
        }
      }
      const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
      const float2 hf = __bfloat1622float2(h);
      oh[c / 2] = h;
      ol[c / 2] = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
    }
    src = nsrc;
  }
}

// C^T in the chunked column order: C [mo][kpad] (FP64) -> bf16 hi/lo
// [kpad][ldw], split from the FP64 value; columns past mo are zero.
__global__ void ctk_split_kernel(const double* __restrict__ C, int64_t mo, int64_t kpad,
                                 int64_t ldw, __nv_bfloat16* __restrict__ hi,
                                 __nv_bfloat16* __restrict__ lo) {
  const int64_t n = kpad * ldw;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / ldw, m = i % ldw;
    const double v = m < mo ? C[m * kpad + k] : 0.0;
    const __nv_bfloat16 h = __double2bfloat16(v);
    hi[i] = h;
    lo[i] = __double2bfloat16(v - (double)__bfloat162float(h));
  }
}

// ------------------------------------------------------------- dL/dC^T --

template <int NA>  // 64-MO atoms of the widest N tile (1..4)
struct DcShape {
  static constexpr uint32_t A_BYTES = 2 * kAtom;  // two chunks, hi + lo each
  static constexpr uint32_t STAGE = A_BYTES + NA * kAtom;
  static constexpr int STAGES =
      (int)((kSmemCap - 4096) / STAGE) > 4 ? 4 : (int)((kSmemCap - 4096) / STAGE);
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 8 * (2 * STAGES + 1);
  static constexpr uint32_t TMEM = tmem_cols<NA * 64>();
  static_assert(STAGES >= 2 && SMEM <= kSmemCap, "shared memory budget");
};

struct DcParams {
  CUtensorMap a;         // AO blocked slices: box (64 AOs, 64 rows, hi + lo)
  CUtensorMap w;         // W tile rows, hi/lo planes: box (64 MOs, 64 rows, 2 planes)
  const uint8_t* mask;   // [tiles][mask_ld(nchunk)]
  float* part;           // [slices][kpad][ldp]
  int64_t kpad;
  int ldp;               // MOs rounded up to 16 (the N extent of all N tiles)
  int nchunk, tiles, per_slice, slices, n_tiles, bn;
  int zero_slice;        // a slice coordinate past the map: reads zeros
};

// CTA (chunk pair cp, N tile nt, slice): dC^T rows 128 cp .. + 127 (AO
// columns of chunks 2 cp and 2 cp + 1), columns of N tile nt, summed over
// the tiles of the slice where either chunk is live (two stages per tile,
// one per 64-row half).  One accumulator per CTA.
//   full[s]   TMA bytes of stage s landed    (producer -> MMA)
//   empty[s]  MMAs reading stage s finished  (MMA -> producer, commit)
//   tfull     accumulator complete           (MMA -> epilogue, commit)
template <int NA>
__global__ void __launch_bounds__(kThreads, 1)
    dct_kernel(const __grid_constant__ DcParams P, int* err_flag) {
  using S = DcShape<NA>;
  constexpr int ST = S::STAGES;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t bar0 = base + ST * S::STAGE;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (ST + s); };
  const uint32_t tfull_bar = bar0 + 8u * (2 * ST);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  volatile int* abort_v = &abort_flag;
  const int slice = blockIdx.x % P.slices;
  const int rest = blockIdx.x / P.slices;
  const int nt = rest % P.n_tiles;
  const int cp = rest / P.n_tiles;
  const int t0 = slice * P.per_slice;
  const int t1 = min(P.tiles, t0 + P.per_slice);
  const int q0 = 2 * cp, q1 = 2 * cp + 1;
  const int n0 = nt * P.bn;
  const int bn = min(P.bn, P.ldp - n0);  // multiple of 16
  const int na = (bn + 63) / 64;
  // live groups of the two chunks at tile t (chunk q1 in bits 4-7)
  auto live_of = [&](int t) -> uint32_t {
    const uint8_t* row = P.mask + (int64_t)t * mask_ld(P.nchunk);
    const uint32_t m0 = row[q0] & 0xFu;
    const uint32_t m1 = q1 < P.nchunk ? (row[q1] & 0xFu) : 0u;
    return m0 | (m1 << 4);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(tfull_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(S::TMEM)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  griddep_wait();

  if (warp == 4) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_map(&P.a);
      tma_prefetch_map(&P.w);
      const uint32_t bytes = S::A_BYTES + (uint32_t)na * kAtom;
      uint32_t it = 0;
      bool ok = true;
      uint32_t nxt = t0 < t1 ? live_of(t0) : 0u;
      for (int t = t0; t < t1 && ok; ++t) {
        const uint32_t lv = nxt;
        nxt = t + 1 < t1 ? live_of(t + 1) : 0u;  // the next tile's mask bytes, early
        if (!lv) continue;
        const int z0 = (lv & 0xFu) ? 2 * (t * P.nchunk + q0) : P.zero_slice;
        const int z1 = (lv >> 4) ? 2 * (t * P.nchunk + q1) : P.zero_slice;
        for (int h = 0; h < 2; ++h) {
          const int s = it % ST;
          const uint32_t ph = (it / ST) & 1u;
          ++it;
          if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_v)) {
            flag_error(err_flag, abort_v, 1);
            ok = false;
            break;
          }
          mbar_expect_tx(full_bar(s), bytes);
          const uint32_t st = base + s * S::STAGE;
          tma_load_3d(st, &P.a, full_bar(s), 0, kHalf * h, z0);
          tma_load_3d(st + kAtom, &P.a, full_bar(s), 0, kHalf * h, z1);
          for (int j = 0; j < na; ++j)
            tma_load_3d(st + S::A_BYTES + j * kAtom, &P.w, full_bar(s), n0 + 64 * j,
                        t * kTileRows + kHalf * h, 0);
        }
      }
      if (*abort_v) {
        // drain: the copies already issued land before the CTA leaves
        const uint32_t first = it > (uint32_t)ST ? it - ST : 0u;
        for (uint32_t k = first; k < it; ++k) {
          const long long c0 = clock64();
          while (!mbar_try_wait(full_bar(k % ST), (k / ST) & 1u) && clock64() - c0 < kWaitCycles) {
          }
        }
      }
    }
  } else if (warp == 5) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = make_idesc(1u, kBM, bn) | kAMajorMN | kBMajorMN;
      uint32_t it = 0;
      bool first = true;
      uint32_t nxt = t0 < t1 ? live_of(t0) : 0u;
      for (int t = t0; t < t1; ++t) {
        const uint32_t lv = nxt;
        nxt = t + 1 < t1 ? live_of(t + 1) : 0u;  // the next tile's mask bytes, early
        if (!lv) continue;
        bool ok = true;
        for (int h = 0; h < 2; ++h) {
          const int s = it % ST;
          const uint32_t ph = (it / ST) & 1u;
          ++it;
          if (!mbar_wait(full_bar(s), ph, abort_v)) {
            flag_error(err_flag, abort_v, 2);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = base + s * S::STAGE;
#pragma unroll
          for (int kk = 0; kk < kHalf / 16; ++kk) {
            const uint32_t ko = kk * 16 * 128;  // 16 rows of 128 bytes
            const uint64_t a_hi = sw128_desc_mn(st + ko, kAtom);
            const uint64_t a_lo = sw128_desc_mn(st + kSlice + ko, kAtom);
            const uint64_t b_hi = sw128_desc_mn(st + S::A_BYTES + ko, kAtom);
            const uint64_t b_lo = sw128_desc_mn(st + S::A_BYTES + kSlice + ko, kAtom);
            umma<QK_BF16X3>(tmem, a_hi, b_hi, idesc, first ? 0u : 1u);
            umma<QK_BF16X3>(tmem, a_hi, b_lo, idesc, 1u);
            umma<QK_BF16X3>(tmem, a_lo, b_hi, idesc, 1u);
            first = false;
          }
          umma_commit(empty_bar(s));
        }
        if (!ok) break;
      }
      // the accumulator is complete (or the pipeline stopped) once these
      // MMAs finish; the epilogue waits for this commit in every case
      umma_commit(tfull_bar);
      const long long c0 = clock64();
      while (!mbar_try_wait(tfull_bar, 0u) && clock64() - c0 < kWaitCycles) {
      }
    }
  } else {
    // ------------------------------------------------ epilogue (warps 0-3)
    const long long c0 = clock64();
    bool ok = true;
    while (!mbar_try_wait(tfull_bar, 0u)) {
      if (clock64() - c0 > kWaitCycles) {
        ok = false;
        break;
      }
    }
    if (!ok) flag_error(err_flag, abort_v, 3);
    ok = __all_sync(0xffffffffu, ok) && !*abort_v;
    if (ok) {
      tc_fence_after();
      bool any = false;
      for (int t = t0 + lane; t < t1; t += 32) any |= live_of(t) != 0u;
      any = __any_sync(0xffffffffu, any);
      const int64_t k = (int64_t)kBM * cp + 32 * warp + lane;
      float* dst = P.part + ((int64_t)slice * P.kpad + k) * P.ldp + n0;
      const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
      for (int c = 0; c < bn; c += 32) {
        const bool two = c + 16 < bn;
        float v[32];
        if (any) {
          tmem_ld16x2(tb + c, v, two);
        } else {  // no live block in the slice: the partial is exactly zero
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = 0.0f;
        }
        if (k < P.kpad) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            reinterpret_cast<float4*>(dst + c)[j] =
                make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          if (two) {
#pragma unroll
            for (int j = 4; j < 8; ++j)
              reinterpret_cast<float4*>(dst + c)[j] =
                  make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(S::TMEM)
                 : "memory");
  }
}

// dL/dC [mo][ao] (FP64, the caller's AO order) = sum over slices of the
// partials, in slice order: a thread per (chunked column k, MO), MOs
// fastest (reads along a partial's rows), the slices' loads unrolled;
// padding columns of a chunk are skipped.
__global__ void reduce_dct_kernel(const float* __restrict__ part, int slices, int64_t kpad,
                                  int ldp, int64_t mo, const int4* chunk, const int* ao_caller,
                                  int64_t ao_num, double* __restrict__ dC) {
  const int64_t n = kpad * mo;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / mo, m = i % mo;
    const int4 ch = chunk[k / kChunkAO];
    const int a = ch.z + (int)(k % kChunkAO);  // internal AO index
    if (a >= ch.w) continue;
    const float* src = part + k * ldp + m;
    const int64_t stride = kpad * ldp;
    double s = 0.0;
#pragma unroll 8
    for (int z = 0; z < slices; ++z) s += (double)src[z * stride];
    dC[m * ao_num + (ao_caller ? ao_caller[a] : a)] = s;
  }
}

// ------------------------------------------------------------ Abar blocks --

// An Abar item is one tile and up to kAbGroup of its live chunks: one MMA
// of N = 64 per chunk multiplies the tile's W rows by the chunks' C^T rows.
constexpr int kAbGroup = 4;
constexpr uint32_t kAbA = 2 * kTileRows * 128;  // W rows of a tile, one K block, hi + lo
constexpr uint32_t kAbPlane = 64 * 128;         // C^T rows of a chunk, one K block, one plane
constexpr uint32_t kAbB = 2 * kAbGroup * kAbPlane;  // hi rows of the group, then lo rows
constexpr uint32_t kAbStage = kAbA + kAbB;
constexpr int kAbStages = 2;
constexpr int kAbBuf = 2;                       // accumulators of kAbGroup x 64 columns
constexpr uint32_t kAbStg = 2 * 32 * 128;       // per epilogue warp: 32 rows x 64 FP32, two halves
constexpr size_t kAbSmem =
    1024 + (size_t)kAbStages * kAbStage + 4 * kAbStg + 8 * (2 * kAbStages + 2 * kAbBuf);
static_assert(kAbSmem <= kSmemCap, "shared memory budget");

// Tiled TMA store of a box from shared memory (bulk-group completion).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
          (uint64_t)map),
      "r"(src), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// The stores committed so far have read their shared-memory source.
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// The stores committed so far are complete.
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

struct AbParams {
  CUtensorMap w;        // W tile rows hi/lo: box (64 MOs, 128 rows, 2 planes)
  CUtensorMap c;        // C^T hi/lo [kpad][ldw]: box (64 MOs, 64 AOs, 1 plane)
  CUtensorMap out;      // Abar blocks as rows of 64 FP32: box (32 columns, 32 rows), 128B swizzle
  const uint8_t* mask;
  float* abar;          // blocks [tiles][nchunk][128][64]
  int nchunk, tiles, num_kb;
};

// Live chunks 64 w .. 64 w + 63 of tile t as bits, from up to four 16-byte
// loads of the mask row (rows are mask_ld bytes, 16-byte aligned; bytes
// past the last chunk are never written and are masked off).
__device__ __forceinline__ uint64_t live_window(const uint8_t* mask, int nchunk, int t, int w) {
  const int mld = mask_ld(nchunk);
  const uint4* row = reinterpret_cast<const uint4*>(mask + (int64_t)t * mld + 64 * w);
  const int nv = (mld - 64 * w) / 16;
  uint4 x[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) x[v] = v < nv ? row[v] : make_uint4(0u, 0u, 0u, 0u);
  uint64_t bits = 0;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const uint32_t wd[4] = {x[v].x, x[v].y, x[v].z, x[v].w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int by = 0; by < 4; ++by)
        if ((wd[k] >> (8 * by)) & 0xFu) bits |= 1ull << (16 * v + 4 * k + by);
  }
  const int valid = nchunk - 64 * w;
  if (valid < 64) bits &= (1ull << valid) - 1ull;
  return bits;
}

// The next item's chunks: up to kAbGroup of the live chunks left in bits
// (window w), lowest first; returns their count.
__device__ __forceinline__ int take_group(uint64_t& bits, int w, int* q) {
  int n = 0;
  while (bits && n < kAbGroup) {
    q[n++] = 64 * w + __ffsll((long long)bits) - 1;
    bits &= bits - 1ull;
  }
  return n;
}

// Persistent: CTA c walks tiles c, c + gridDim.x, ... and, in each, its
// live chunks in groups of up to kAbGroup; an item (tile, group) takes
// num_kb stages (K = MOs in blocks of 64) and one of kAbBuf TMEM
// accumulators, so that the epilogue of an item overlaps the MMAs of the
// next.  The three roles enumerate the items from the mask in the same
// order.
//   full[s] / empty[s]   stage s loaded / read by the MMAs
//   tfull[b]  accumulator b complete            (MMA -> epilogue, commit)
//   tempty[b] accumulator b read out            (epilogue warps -> MMA)
__global__ void __launch_bounds__(kThreads, 1)
    abar_kernel(const __grid_constant__ AbParams P, int* err_flag) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t bar0 = base + kAbStages * kAbStage + 4 * kAbStg;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (kAbStages + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * kAbStages + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * kAbStages + kAbBuf + b); };
  constexpr uint32_t kAcc = kAbGroup * 64;
  constexpr uint32_t kTmem = tmem_cols<kAbBuf * kAcc>();

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  volatile int* abort_v = &abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kAbStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < kAbBuf; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), 4);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTmem)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  griddep_wait();

  if (warp == 4) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_map(&P.w);
      tma_prefetch_map(&P.c);
      uint32_t it = 0;
      bool ok = true;
      uint64_t cur = (int)blockIdx.x < P.tiles ? live_window(P.mask, P.nchunk, blockIdx.x, 0) : 0;
      for (int t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
        const int tn = t + gridDim.x;
        const uint64_t nxt = tn < P.tiles ? live_window(P.mask, P.nchunk, tn, 0) : 0;  // early
        for (int w = 0; 64 * w < P.nchunk && ok; ++w) {
          uint64_t bits = w == 0 ? cur : live_window(P.mask, P.nchunk, t, w);
          while (bits && ok) {
            int q[kAbGroup];
            const int n = take_group(bits, w, q);
            for (int kb = 0; kb < P.num_kb; ++kb) {
              const int s = it % kAbStages;
              const uint32_t ph = (it / kAbStages) & 1u;
              ++it;
              if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_v)) {
                flag_error(err_flag, abort_v, 1);
                ok = false;
                break;
              }
              mbar_expect_tx(full_bar(s), kAbA + 2u * n * kAbPlane);
              const uint32_t st = base + s * kAbStage;
              tma_load_3d(st, &P.w, full_bar(s), 64 * kb, t * kTileRows, 0);
              for (int j = 0; j < n; ++j) {
                tma_load_3d(st + kAbA + j * kAbPlane, &P.c, full_bar(s), 64 * kb, 64 * q[j], 0);
                tma_load_3d(st + kAbA + (kAbGroup + j) * kAbPlane, &P.c, full_bar(s), 64 * kb,
                            64 * q[j], 1);
              }
            }
          }
        }
        cur = nxt;
      }
      if (*abort_v) {
        const uint32_t first = it > (uint32_t)kAbStages ? it - kAbStages : 0u;
        for (uint32_t k = first; k < it; ++k) {
          const long long c0 = clock64();
          while (!mbar_try_wait(full_bar(k % kAbStages), (k / kAbStages) & 1u) &&
                 clock64() - c0 < kWaitCycles) {
          }
        }
      }
    }
  } else if (warp == 5) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t it = 0, i = 0;
      bool ok = true, in_item = false;
      uint32_t b = 0;
      uint64_t cur = (int)blockIdx.x < P.tiles ? live_window(P.mask, P.nchunk, blockIdx.x, 0) : 0;
      for (int t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
        const int tn = t + gridDim.x;
        const uint64_t nxt = tn < P.tiles ? live_window(P.mask, P.nchunk, tn, 0) : 0;  // early
        for (int w = 0; 64 * w < P.nchunk && ok; ++w) {
          uint64_t bits = w == 0 ? cur : live_window(P.mask, P.nchunk, t, w);
          while (bits && ok) {
            int q[kAbGroup];
            const int n = take_group(bits, w, q);
            b = i % kAbBuf;
            if (!mbar_wait(tempty_bar(b), ((i / kAbBuf) & 1u) ^ 1u, abort_v)) {
              flag_error(err_flag, abort_v, 2);
              ok = false;
              break;
            }
            in_item = true;
            const uint32_t dacc = tmem + b * kAcc;
            const uint32_t idesc = make_idesc(1u, kBM, 64 * n);
            for (int kb = 0; kb < P.num_kb; ++kb) {
              const int s = it % kAbStages;
              const uint32_t ph = (it / kAbStages) & 1u;
              ++it;
              if (!mbar_wait(full_bar(s), ph, abort_v)) {
                flag_error(err_flag, abort_v, 2);
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t st = base + s * kAbStage;
              const uint64_t a_hi = sw128_desc(st);
              const uint64_t a_lo = sw128_desc(st + kAbA / 2);
              const uint64_t b_hi = sw128_desc(st + kAbA);
              const uint64_t b_lo = sw128_desc(st + kAbA + kAbGroup * kAbPlane);
#pragma unroll
              for (int kk = 0; kk < kRowBytes / kUmmaKBytes; ++kk) {
                const uint64_t ko = (uint64_t)(kk * kUmmaKBytes) >> 4;
                umma<QK_BF16X3>(dacc, a_hi + ko, b_hi + ko, idesc, (kb | kk) ? 1u : 0u);
                umma<QK_BF16X3>(dacc, a_hi + ko, b_lo + ko, idesc, 1u);
                umma<QK_BF16X3>(dacc, a_lo + ko, b_hi + ko, idesc, 1u);
              }
              umma_commit(empty_bar(s));
            }
            if (!ok) break;
            umma_commit(tfull_bar(b));
            in_item = false;
            ++i;
          }
        }
        cur = nxt;
      }
      if (!ok) {
        // aborted: the MMAs in flight finish before TMEM is freed
        uint32_t wb = 0, wi = 0;
        bool wait = false;
        if (in_item) {
          umma_commit(tfull_bar(b));
          wb = b;
          wi = i;
          wait = true;
        } else if (i > 0) {
          wb = (i - 1) % kAbBuf;
          wi = i - 1;
          wait = true;
        }
        const long long c0 = clock64();
        while (wait && !mbar_try_wait(tfull_bar(wb), (wi / kAbBuf) & 1u) &&
               clock64() - c0 < kWaitCycles) {
        }
      }
    }
  } else {
    // ------------------------------------------------ epilogue (warps 0-3)
    // Per chunk of an item, warp w's 32 rows of the block go TMEM -> shared
    // (two 32-column halves in the 128-byte swizzled layout: 16-byte piece j
    // of row r at j ^ (r & 7), free of bank conflicts) -> global by two
    // tensor stores; the staging buffer is reused once the previous stores
    // have read it.
    const uint32_t stg = base + kAbStages * kAbStage + warp * kAbStg;
    uint32_t i = 0;
    bool ok = true;
    uint64_t cur = (int)blockIdx.x < P.tiles ? live_window(P.mask, P.nchunk, blockIdx.x, 0) : 0;
    for (int t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
      const int tn = t + gridDim.x;
      const uint64_t nxt = tn < P.tiles ? live_window(P.mask, P.nchunk, tn, 0) : 0;  // early
      for (int w = 0; 64 * w < P.nchunk && ok; ++w) {
        uint64_t bits = w == 0 ? cur : live_window(P.mask, P.nchunk, t, w);
        while (bits) {
          int q[kAbGroup];
          const int n = take_group(bits, w, q);
          const uint32_t b = i % kAbBuf;
          const long long c0 = clock64();
          bool got = true;
          while (!mbar_try_wait(tfull_bar(b), (i / kAbBuf) & 1u)) {
            if (clock64() - c0 > kWaitCycles) {
              got = false;
              break;
            }
          }
          if (!got) flag_error(err_flag, abort_v, 3);
          ok = __all_sync(0xffffffffu, got) && !*abort_v;
          __syncwarp();
          if (!ok) break;
          tc_fence_after();
          for (int j = 0; j < n; ++j) {
            if (lane == 0) bulk_wait_read_all();
            __syncwarp();
            const uint32_t tb = tmem + b * kAcc + 64 * j + ((uint32_t)(warp * 32) << 16);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float v[32];
              tmem_ld16x2(tb + 32 * h, v, true);
              const uint32_t rowp = stg + h * (kAbStg / 2) + lane * 128;
#pragma unroll
              for (int k = 0; k < 8; ++k)
                asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(
                                 rowp + (uint32_t)((k ^ (lane & 7)) * 16)),
                             "f"(v[4 * k]), "f"(v[4 * k + 1]), "f"(v[4 * k + 2]),
                             "f"(v[4 * k + 3])
                             : "memory");
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
              const int row0 = ((t * P.nchunk + q[j]) * kTileRows) + 32 * warp;
              tma_store_2d(&P.out, stg, 0, row0);
              tma_store_2d(&P.out, stg + kAbStg / 2, 32, row0);
              bulk_commit();
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty_bar(b));
          ++i;
        }
      }
      cur = nxt;
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmem)
                 : "memory");
  }
}

// N tiles of the dL/dC^T product: as few as possible of at most 256 MOs,
// each a multiple of 16.
int dc_bn(int64_t ldp) {
  const int64_t tiles = (ldp + 255) / 256;
  const int64_t per = (ldp + tiles - 1) / tiles;
  return (int)((per + 15) / 16 * 16);
}

struct SparseLayout {
  size_t w_hi, w_lo, part, abar, total;
  int slices, per_slice, n_tiles, bn;
};

SparseLayout sparse_layout(int64_t tiles, int nchunk, int64_t mo_num) {
  SparseLayout L{};
  const int64_t ldw = (mo_num + 7) / 8 * 8;
  const int64_t ldp = up16(mo_num);
  const int64_t rows = tiles * kTileRows;
  const int64_t kpad = (int64_t)nchunk * kChunkAO;
  L.bn = dc_bn(ldp);
  L.n_tiles = (int)((ldp + L.bn - 1) / L.bn);
  const int64_t pairs = (nchunk + 1) / 2;
  // slices: enough for a CTA per SM (one is resident per SM), and of at
  // most 32 tiles (4096 rows summed in FP32 before the FP64 sum over
  // slices) while the partials stay within 64 MB; at least 4 tiles each
  int64_t sl = ((int64_t)device_sms() + pairs * L.n_tiles - 1) / (pairs * L.n_tiles);
  sl = std::max<int64_t>(sl, (tiles + 31) / 32);
  const int64_t slice_bytes = (int64_t)sizeof(float) * kpad * ldp;
  sl = std::min<int64_t>(sl, std::max<int64_t>(1, ((int64_t)64 << 20) / slice_bytes));
  sl = std::max<int64_t>(1, std::min<int64_t>(sl, (tiles + 3) / 4));
  L.per_slice = (int)((tiles + sl - 1) / sl);
  L.slices = (int)((tiles + L.per_slice - 1) / L.per_slice);
  size_t off = 0;
  L.w_hi = off;
  off += up256(sizeof(__nv_bfloat16) * (size_t)rows * ldw);
  L.w_lo = off;
  off += up256(sizeof(__nv_bfloat16) * (size_t)rows * ldw);
  L.part = off;
  off += up256(sizeof(float) * (size_t)L.slices * kpad * ldp);
  L.abar = off;
  off += up256(sizeof(float) * (size_t)tiles * nchunk * kTileRows * 64);
  L.total = off;
  return L;
}

template <int NA>
cudaError_t launch_dct(const DcParams& p, unsigned grid, int* err_flag, cudaStream_t s) {
  using S = DcShape<NA>;
  KernelFacts f;
  cudaError_t e = kernel_facts<dct_kernel<NA>>(S::SMEM, kThreads, &f);
  if (e != cudaSuccess) return e;
  if (f.occ < 1 || f.occ * (int)S::TMEM > 512) return cudaErrorInvalidConfiguration;
  return launch_pdl(dct_kernel<NA>, grid, kThreads, S::SMEM, s, p, err_flag);
}

}  // namespace

size_t adjoint_sparse_ctk_bytes(int nchunk, int64_t mo_num) {
  const int64_t ldw = (mo_num + 7) / 8 * 8;
  return 2 * up256(sizeof(__nv_bfloat16) * (size_t)nchunk * kChunkAO * ldw);
}

cudaError_t launch_adjoint_ctk_split(const double* C64p, int64_t mo_num, int nchunk, void* ctk,
                                     cudaStream_t s) {
  const int64_t ldw = (mo_num + 7) / 8 * 8, kpad = (int64_t)nchunk * kChunkAO;
  if (kpad * ldw == 0) return cudaSuccess;
  __nv_bfloat16* hi = (__nv_bfloat16*)ctk;
  __nv_bfloat16* lo =
      (__nv_bfloat16*)((unsigned char*)ctk + up256(sizeof(__nv_bfloat16) * kpad * ldw));
  ctk_split_kernel<<<grid_for(kpad * ldw), 256, 0, s>>>(C64p, mo_num, kpad, ldw, hi, lo);
  return cudaGetLastError();
}

size_t adjoint_sparse_scratch_bytes(int64_t point_num, int nchunk, int64_t mo_num) {
  const int64_t tiles = (point_num + kTilePoints - 1) / kTilePoints;
  return sparse_layout(tiles, nchunk, mo_num).total;
}

cudaError_t launch_adjoint_sparse(const BasisDev& b, const PointsDev& p, const AOTensor& ao,
                                  const float* W, int64_t mo_num, const void* ctk, bool zero_groups,
                                  double* d_dC, double* d_dR, void* scratch, double* dr_partial,
                                  int* err_flag, cudaStream_t s) {
  const int64_t P = p.n;
  if (P == 0 || mo_num == 0) return cudaSuccess;
  if (!ao.tiled || !ao.blocked || !ao.a_lo || !ao.mask) return cudaErrorInvalidValue;
  const int nchunk = ao.nchunk;
  const int64_t tiles = (P + kTilePoints - 1) / kTilePoints;
  if ((int64_t)nchunk * tiles * kTileRows > INT32_MAX || mo_num > INT32_MAX)
    return cudaErrorInvalidValue;
  const int64_t ldw = (mo_num + 7) / 8 * 8;
  const int64_t ldp = up16(mo_num);
  const int64_t kpad = (int64_t)nchunk * kChunkAO;
  const SparseLayout L = sparse_layout(tiles, nchunk, mo_num);
  unsigned char* base = (unsigned char*)scratch;
  __nv_bfloat16* w_hi = (__nv_bfloat16*)(base + L.w_hi);
  __nv_bfloat16* w_lo = (__nv_bfloat16*)(base + L.w_lo);
  float* part = (float*)(base + L.part);
  float* abar = (float*)(base + L.abar);
  const __nv_bfloat16* c_hi = (const __nv_bfloat16*)ctk;
  const __nv_bfloat16* c_lo =
      (const __nv_bfloat16*)((const unsigned char*)ctk + up256(sizeof(__nv_bfloat16) * kpad * ldw));

  // 1. dead groups of live blocks to zero; W into the tile rows, split
  if (zero_groups) {
    const int64_t warps = tiles * nchunk;
    const int64_t blocks = (warps + 7) / 8;
    zero_dead_groups_kernel<<<(unsigned)std::min<int64_t>(blocks, 8 * device_sms()), 256, 0, s>>>(
        (__nv_bfloat16*)ao.a, ao.mask, tiles, nchunk);
  }
  gather_split_w_kernel<<<(unsigned)std::min<int64_t>((tiles * kTileRows + 7) / 8,
                                                      16 * (int64_t)device_sms()),
                          256, 0, s>>>(W, ao.perm, P, mo_num, ldw, tiles, w_hi, w_lo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  // 2. dL/dC^T partials over slices of tiles, then their fixed-order sum
  if (d_dC) {
    DcParams dp;
    memset(&dp, 0, sizeof(dp));
    {
      // AO slices with a 64-row box (half a tile per stage)
      EncodeTiledFn enc = encode_fn();
      if (!enc) return cudaErrorInvalidValue;
      const int64_t nblocks = tiles * nchunk;
      cuuint64_t dims[3] = {64, (cuuint64_t)kTileRows, (cuuint64_t)(2 * nblocks)};
      cuuint64_t strides[2] = {128, 128 * 128};
      cuuint32_t box[3] = {64, (cuuint32_t)kHalf, 2};
      cuuint32_t estr[3] = {1, 1, 1};
      if (enc(&dp.a, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ao.a), dims, strides,
              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
      dp.zero_slice = (int)(2 * nblocks);
    }
    if (!make_map_planes(&dp.w, w_hi, w_lo, ldw, tiles * kTileRows, ldw, 64, kHalf))
      return cudaErrorInvalidValue;
    dp.mask = ao.mask;
    dp.part = part;
    dp.kpad = kpad;
    dp.ldp = (int)ldp;
    dp.nchunk = nchunk;
    dp.tiles = (int)tiles;
    dp.per_slice = L.per_slice;
    dp.slices = L.slices;
    dp.n_tiles = L.n_tiles;
    dp.bn = L.bn;
    const int64_t pairs = (nchunk + 1) / 2;
    const unsigned grid = (unsigned)(pairs * L.n_tiles * L.slices);
    switch ((L.bn + 63) / 64) {
      case 1: e = launch_dct<1>(dp, grid, err_flag, s); break;
      case 2: e = launch_dct<2>(dp, grid, err_flag, s); break;
      case 3: e = launch_dct<3>(dp, grid, err_flag, s); break;
      case 4: e = launch_dct<4>(dp, grid, err_flag, s); break;
      default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    reduce_dct_kernel<<<grid_for(mo_num * kpad), 256, 0, s>>>(
        part, L.slices, kpad, (int)ldp, mo_num, b.chunk, b.ao_caller, b.ao_num, d_dC);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (!d_dR) return cudaSuccess;

  // 3. Abar at the live blocks, then dL/dR from them
  AbParams ap;
  memset(&ap, 0, sizeof(ap));
  if (!make_map_planes(&ap.w, w_hi, w_lo, ldw, tiles * kTileRows, ldw, 64, kTileRows))
    return cudaErrorInvalidValue;
  {
    // C^T planes as a 3-D map with a one-plane box: the hi rows of a group's
    // chunks land together, then the lo rows
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorInvalidValue;
    const intptr_t gap = (const char*)c_lo - (const char*)c_hi;
    cuuint64_t dims[3] = {(cuuint64_t)ldw, (cuuint64_t)kpad, 2};
    cuuint64_t strides[2] = {(cuuint64_t)(ldw * 2), (cuuint64_t)gap};
    cuuint32_t box[3] = {64, 64, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    if (gap <= 0 || gap % 16 != 0 ||
        enc(&ap.c, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(c_hi), dims,
            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorInvalidValue;
    cuuint64_t dims[2] = {64, (cuuint64_t)(tiles * nchunk * kTileRows)};
    cuuint64_t strides[1] = {64 * sizeof(float)};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t estr[2] = {1, 1};
    if (enc(&ap.out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, abar, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  ap.mask = ao.mask;
  ap.abar = abar;
  ap.nchunk = nchunk;
  ap.tiles = (int)tiles;
  ap.num_kb = (int)((ldw + 63) / 64);
  {
    KernelFacts f;
    e = kernel_facts<abar_kernel>(kAbSmem, kThreads, &f);
    if (e != cudaSuccess) return e;
    if (f.occ < 1 || f.occ * (int)tmem_cols<kAbBuf * kAbGroup * 64>() > 512)
      return cudaErrorInvalidConfiguration;
    const int64_t g = std::min<int64_t>(tiles, (int64_t)f.sms * f.occ);
    e = launch_pdl(abar_kernel, (unsigned)g, kThreads, kAbSmem, s, ap, err_flag);
    if (e != cudaSuccess) return e;
  }
  return launch_adjoint_dR_blocked(b, p, abar, ao.mask, dr_partial, d_dR, s);
}

}  // namespace qk
