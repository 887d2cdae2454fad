// tc_common.cuh -- building blocks of the tcgen05 kernels: mbarrier waits
// (bounded), TMA tile loads, shared-memory matrix and instruction
// descriptors, MMA issue / commit, TMEM loads, and the host-side tensor map
// encoder.  Used by the contraction (mo_tc.cu) and the fused AO + MO kernel
// (mo_fused.cu).
#pragma once

#include <cuda.h>

#include "internal.h"

namespace qk {
namespace tc {

constexpr int kBM = 128;            // MMA M (TMEM lanes)
constexpr int kRowBytes = 128;      // one K block = one 128-byte swizzle row
constexpr int kUmmaKBytes = 32;     // bytes of K consumed by one MMA
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

template <int MODE>
struct TcTraits;
template <>
struct TcTraits<QK_BF16X3> {
  static constexpr int kBK = 64;      // bf16 elements per K block
  static constexpr int kPlanes = 2;   // hi and lo
  static constexpr uint32_t kFmt = 1; // BF16
};
template <>
struct TcTraits<QK_TF32> {
  static constexpr int kBK = 32;
  static constexpr int kPlanes = 1;
  static constexpr uint32_t kFmt = 2; // TF32
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false if it gave up
// (after `limit` SM clock cycles) or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          volatile int* abort_flag,
                                          long long limit = kWaitCycles) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Bring the box at (c0, c1, c2) of a 3-D map into L2 (no shared memory).
__device__ __forceinline__ void tma_prefetch_l2_3d(const CUtensorMap* map, int c0, int c1,
                                                   int c2) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                   (uint64_t)map),
               "r"(c0), "r"(c1), "r"(c2)
               : "memory");
}

// Fetch a tensor map (kernel parameter or global memory) into the TMA
// unit's descriptor cache.
__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), start address in 16-byte units; descriptor
// version 1 (bits 46-47); layout type 2 = SWIZZLE_128B (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: f32 accumulator, A/B format, K-major A and B,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, int m, int n) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

template <int MODE>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t accumulate) {
  if constexpr (MODE == QK_BF16X3) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  }
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Columns taddr .. + 15 and, when two, taddr + 16 .. + 31 of this warp's 32
// TMEM lanes, with one wait for both loads.
__device__ __forceinline__ void tmem_ld16x2(uint32_t taddr, float* v, bool two) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  if (two) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr + 16));
  } else {
#pragma unroll
    for (int i = 16; i < 32; ++i) r[i] = 0u;
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void flag_error(int* err_flag, volatile int* abort_flag, int code) {
  *abort_flag = 1;
  atomicCAS(err_flag, 0, code);
}

template <int BNT>
constexpr uint32_t tmem_cols() {
  return BNT <= 32 ? 32 : BNT <= 64 ? 64 : BNT <= 128 ? 128 : BNT <= 256 ? 256 : 512;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}


typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 2-D tiled map over a row-major [outer][ld] matrix with `inner` valid
// columns; box = box_inner x box_outer, 128-byte swizzle, zero fill outside.
inline bool make_map(CUtensorMap* m, const void* ptr, bool f32, int64_t inner, int64_t outer,
              int64_t ld, int box_inner, int box_outer) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const int es = f32 ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
             const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The bf16 hi and lo planes of one matrix as a 3-D map (plane = third
// dimension, stride lo - hi bytes), so that one copy brings a box of both
// planes: plane 0 then plane 1, box_outer rows of 128 bytes each.  False if
// lo does not follow hi at a positive multiple of 16 bytes.
inline bool make_map_planes(CUtensorMap* m, const void* hi, const void* lo, int64_t inner,
                            int64_t outer, int64_t ld, int box_inner, int box_outer) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const intptr_t gap = (const char*)lo - (const char*)hi;
  if (gap <= 0 || gap % 16 != 0) return false;
  cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)outer, 2};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)gap};
  cuuint32_t box[3] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer, 2};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(hi), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The blocked AO tensor (AOTensor::blocked) as a 3-D map over its 128-byte
// column slices: (w columns, 128 rows, slice), slice z = block * 2 + j with
// j the plane (split bf16: hi, lo; box of 2 slices = the whole 32 KB block,
// the same shared-memory image as the row layout's 3-D box of both planes)
// or the 32-column half (TF32: box of 1 slice = one K block).  A box at
// slice 2 * nblocks (past the end) reads zeros.
inline bool make_map_blocked(CUtensorMap* m, const void* base, bool split, int64_t nblocks) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t w = split ? 64 : 32;
  cuuint64_t dims[3] = {w, 128, (cuuint64_t)(2 * nblocks)};
  cuuint64_t strides[2] = {128, 128 * 128};
  cuuint32_t box[3] = {(cuuint32_t)w, 128, split ? 2u : 1u};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, split ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
             const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Slice coordinate of K block kb of M tile mt in the blocked map: a split
// K block is one chunk (both planes), a TF32 K block half a chunk.
template <int MODE>
__device__ __forceinline__ int blocked_slice(int mt, int kb, int nchunk) {
  if constexpr (TcTraits<MODE>::kBK == 64)
    return 2 * (mt * nchunk + kb);
  else
    return 2 * (mt * nchunk + (kb >> 1)) + (kb & 1);
}

}  // namespace tc
}  // namespace qk
