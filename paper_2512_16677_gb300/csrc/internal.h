// internal.h -- declarations shared by the library's translation units.
// Not part of the public ABI (include/qmckl_gpu.h is).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>
#include <string>
#include <vector>

#include "../../include/qmckl_gpu.h"

namespace qk {

// Largest angular momentum handled by the kernels (f shells).
constexpr int kMaxL = 3;
// AOs per ao_vgl column chunk; chunks end on shell boundaries and also hold
// at most kMaxShellsChunk shells and kMaxPrimsChunk primitives.  In the
// contraction layout chunk q owns AO-tensor columns [64q, 64q + 64).
constexpr int kChunkAO = 64;
constexpr int kMaxShellsChunk = 32;
constexpr int kMaxPrimsChunk = 256;

// Device-side basis tables, passed to kernels by value.  Every pointer
// points into one allocation owned by the context.  Primitives of each
// shell are sorted by ascending exponent.
struct BasisDev {
  int nucl_num, shell_num, ao_num, prim_num, nchunk;
  const double* nucl_xyz;   // [nucl][3]
  const float* nucl_hi;     // [nucl][3] float(x)
  const float* nucl_lo;     // [nucl][3] float(x - float(x))
  const int* shell_nuc;     // [shell]
  const int* shell_l;       // [shell]
  const int* shell_prim0;   // [shell] first primitive
  const int* shell_nprim;   // [shell]
  const int* shell_ao0;     // [shell] first AO
  const double* shell_r2;   // [shell] T / gamma_min: r^2 at or beyond it screens every primitive
  const float* shell_r2_f;  // [shell] same, rounded up to float
  const double* prim_g;     // [prim] gamma
  const double* prim_c;     // [prim] N_s * a * f
  const float* prim_g_f;
  const float* prim_c_f;
  const double* ao_fac;     // [ao] M_n
  const float* ao_fac_f;
  const int* ao_shell;      // [ao] shell of each AO
  const int4* chunk;        // [nchunk] (shell_begin, shell_end, ao_begin, ao_end)
  const int* shell_chunk;   // [shell] chunk holding each shell
  const int* ao_caller;     // [ao] the caller's index of each AO (NULL: the same order)
  double T;                 // Eq. 3 threshold on gamma r^2
  float T_f;
};

// Points in structure-of-arrays form (device, library-owned).  A view of a
// contiguous range of points offsets every pointer and keeps ld.
struct PointsDev {
  int64_t n;
  const double* x;  // [n] each
  const double* y;
  const double* z;
  const float* hi;  // [3][ld] float(x), float(y), float(z)
  const float* lo;  // [3][ld] residuals
  int64_t ld;       // distance between the coordinate planes of hi and lo
};

// Bytes per tile row of the live-group mask of a tiled AO tensor.
__host__ __device__ inline int mask_ld(int nchunk) { return (nchunk + 15) & ~15; }

// Layout of the AO tensor: rows are (point, component) pairs, row r = 5p + c,
// ld elements apart.  chunked: AO n of chunk q sits in column
// 64q + (n - first AO of q) and the padding columns hold zeros (the layout the
// contraction reads); otherwise column = AO index.
//
// tiled (tensor-core modes): points go in tiles of kTilePoints; the 125
// (point, component) rows of tile t are rows 128 t .. 128 t + 124, rows
// 125..127 of each tile are zero, and bit g of mask[t * mask_ld(nchunk) + q]
// says whether columns 16 g .. 16 g + 15 of block (t, q) hold any entry that
// survived screening (rows padded to 16 bytes, so that a reader takes 16
// chunks with one load; the padding bytes are never written).  Blocks with a
// zero mask byte are not written, nor are the dead column groups of live
// blocks; the contraction skips both (K blocks, and MMA k-steps over dead
// groups: the sparse-AO MO product of Sec. 3.2 at tile granularity).
struct AOTensor {
  void* a;        // FP64 / FP32 values, or bf16 "hi" plane
  void* a_lo;     // bf16 "lo" plane (QK_BF16X3 only)
  int64_t rows;   // rows of the tensor: 5 * point_num, or 128 * tiles when tiled
  int64_t ld;     // row stride in elements
  bool chunked;
  bool tiled;
  uint8_t* mask;  // [tiles][mask_ld(nchunk)] live 16-column groups when tiled
  int nchunk;
  // tiled, optional: [tiles][nchunk] bit s set when shell s of the chunk may
  // reach a point of the tile (filled by a pre-pass in launch_ao_vgl; NULL:
  // each ao_vgl tile works it out itself)
  uint32_t* reach;
  // tiled, optional: point slot s of the tiles holds the caller's point
  // perm[s] (spatial order); the contraction writes its rows there.  NULL:
  // slot s is point s.
  const int32_t* perm;
  // tiled: 0 or 5 -> the vgl layout (25 points x 5 components per 128-row
  // tile); 1 -> values only (128 points per tile, one row each)
  int comps;
  // dense layout only: columns in the caller's AO order (BasisDev::ao_caller)
  bool caller_cols;
  // tiled vgl layout, blocked: block b = tile * nchunk + chunk holds its
  // planes (bf16 hi then lo; one otherwise) one after the other, each plane
  // as 128-byte-wide column slices ([64 / w][128 rows][w columns], w = 128
  // bytes / element size), blocks in b order: a live block is one contiguous
  // read and a slice one TMA box (element offset: blocked_offset below).
  // a_lo then points at the lo plane of block 0.  Otherwise rows of ld
  // elements.
  bool blocked;
  // tiled, with reach: the contraction multiplies tiles in pairs (2i, 2i+1)
  // over the union of their live column groups, so ao_vgl also writes zeros
  // into the groups of a live block that the partner tile's reach word says
  // may be live there
  bool pair_zero;
};
constexpr int kTilePoints = 25;   // 125 rows of a 128-row contraction tile
constexpr int kTileRows = 128;
constexpr int64_t kBlockElems = (int64_t)kTileRows * 64;  // one plane of one block

// Element offset of (tile row r, chunk column c, plane p) of block
// (tile, chunk) in the blocked layout, for elements of `es` bytes.
__host__ __device__ __forceinline__ int64_t blocked_offset(int64_t tile, int chunk, int nchunk,
                                                           int planes, int plane, int r, int c,
                                                           int es) {
  const int w = 128 / es;  // columns of one slice
  return ((tile * nchunk + chunk) * planes + plane) * kBlockElems +
         (int64_t)(c / w) * (kTileRows * w) + (int64_t)r * w + c % w;
}

// Launch facts of a kernel on the current device, worked out once per
// (kernel, device): its opt-in dynamic shared memory set, resident blocks
// per SM at that size and the SM count.  Small calls (a single-electron
// move) would otherwise spend more time in these queries than on the GPU.
struct KernelFacts {
  int occ;
  int sms;
};
constexpr int kMaxDevices = 64;
template <auto Kern>
cudaError_t kernel_facts(size_t smem, int threads, KernelFacts* out) {
  static std::atomic<int> ready[kMaxDevices];
  static KernelFacts facts[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cache = dev >= 0 && dev < kMaxDevices;
  if (cache && ready[dev].load(std::memory_order_acquire)) {
    *out = facts[dev];
    return cudaSuccess;
  }
  e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  KernelFacts f{0, 1};
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&f.occ, Kern, threads, smem);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&f.sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (cache) {
    facts[dev] = f;
    ready[dev].store(1, std::memory_order_release);
  }
  *out = f;
  return cudaSuccess;
}
// The SM count of the current device (cached per device).
inline int device_sms() {
  static std::atomic<int> sms[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev < 0 || dev >= kMaxDevices) return 1;
  int v = sms[dev].load(std::memory_order_acquire);
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
      v = 1;
    sms[dev].store(v, std::memory_order_release);
  }
  return v;
}

// Programmatic dependent launch: the kernel may be scheduled while the
// previous kernel in the stream finishes (its set-up overlapping that
// kernel's tail); it must call griddep_wait() before it reads anything the
// previous kernel wrote or writes anything it reads.  In a launch without
// the attribute griddep_wait() returns at once.
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// A device allocation owned by the library.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t n);
  void release();
  ~DevBuf() { release(); }
};

// ---------------------------------------------------------------- kernels --
// All launchers return the launch status (cudaGetLastError) and run on `s`.

// AO vgl at every point.  out_mode: QK_FP64 -> double, QK_FP32/QK_TF32 ->
// float, QK_BF16X3 -> bf16 hi/lo planes.
cudaError_t launch_ao_vgl(const BasisDev& b, const PointsDev& p, int out_mode,
                          const AOTensor& out, cudaStream_t s);

// Nonzero (point, AO) pairs of the tiled vgl AO tensor t of n points
// (es = 2: bf16 hi/lo planes; 4: FP32; 8: FP64) summed into *out (device;
// zeroed first).
cudaError_t launch_ao_nnz(const AOTensor& t, int es, int64_t n, unsigned long long* out,
                          cudaStream_t s);

// Point coordinates [n][3] ('N') or [3][n] ('T') -> SoA + hi/lo floats.
cudaError_t launch_points_soa(const double* raw, char transp, int64_t n, double* x,
                              double* y, double* z, float* hi, float* lo, cudaStream_t s);

// C [rows][cols] (FP64) -> chunked column layout [rows][nchunk*64] in FP64,
// FP32 and bf16 hi/lo planes (padding zeroed).
cudaError_t launch_mo_chunked(const double* src, int64_t rows, int64_t cols, const int4* chunk,
                              int nchunk, double* d64, float* d32, __nv_bfloat16* hi,
                              __nv_bfloat16* lo, cudaStream_t s);

// Split an FP64 matrix [rows][cols] into bf16 hi and lo planes (ld columns,
// padding zeroed), or convert it to FP32.
cudaError_t launch_split_bf16(const double* src, int64_t rows, int64_t cols, int64_t ld,
                              __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t s);
cudaError_t launch_to_f32(const double* src, int64_t rows, int64_t cols, int64_t ld,
                          float* dst, cudaStream_t s);

// SIMT contraction D[M][N] = sum_k A[m][k] B[n][k] (FP32 or FP64), with
// generic strides: element (m,k) of A at A[m*sam + k*sak], (n,k) of B at
// B[n*sbn + k*sbk], D[m*ldd + n].  k_split > 1 writes k_split partial
// results D + z*M*ldd.
cudaError_t launch_gemm_f32(int64_t M, int64_t N, int64_t K, const float* A, int64_t sam,
                            int64_t sak, const float* B, int64_t sbn, int64_t sbk, float* D,
                            int64_t ldd, int k_split, cudaStream_t s);
cudaError_t launch_gemm_f64(int64_t M, int64_t N, int64_t K, const double* A, int64_t sam,
                            int64_t sak, const double* B, int64_t sbn, int64_t sbk, double* D,
                            int64_t ldd, int k_split, cudaStream_t s);
// Sum k_split partials [k_split][n] into dst (FP64 out).  col_map (optional):
// the partials are rows of ncol columns and column j lands in column col_map[j].
cudaError_t launch_reduce_partials_f32(const float* part, int k_split, int64_t n, double* dst,
                                       cudaStream_t s, const int* col_map = nullptr,
                                       int64_t ncol = 0);
cudaError_t launch_reduce_partials_f64(const double* part, int k_split, int64_t n, double* dst,
                                       cudaStream_t s, const int* col_map = nullptr,
                                       int64_t ncol = 0);

// tcgen05 contraction (QK_BF16X3 / QK_TF32): D[rows][mo] float.
struct TcConfig {
  int bn;      // MMA N per instruction (multiple of 16, <= 256)
  int nsub;    // MMA instructions along N per CTA
  int stages;  // shared-memory pipeline depth
};
// out_rows: rows of D (5 * points); -1 = ao.rows (dense layout).
// Density epilogue (wdens != NULL): instead of D, each output row r gets
// sum_n wdens[n] D[r][n]^2 over the columns of its N tile, written to
// rho_part[N tile][r]; out is then unused.
cudaError_t launch_mo_tc(int mode, const AOTensor& ao, int64_t ao_num, const void* c_hi,
                         const void* c_lo, int64_t ldc, int64_t mo_num, float* out,
                         const TcConfig& cfg, int* err_flag, cudaStream_t s,
                         int64_t out_rows = -1, const float* wdens = nullptr,
                         float* rho_part = nullptr);
// FP64 contraction over a tiled vgl AO tensor (mo_sparse64.cu): only the
// live 16-AO column groups of live blocks are multiplied; C [N][ldc] in the
// chunked column layout; D [out_rows][N] double, rows through ao.perm.
cudaError_t launch_mo_sparse64(const AOTensor& ao, const double* C, int64_t ldc, int64_t N,
                               double* D, int64_t out_rows, cudaStream_t s);
// Default tile configuration for a problem shape.
TcConfig tc_default_config(int mode, int64_t mo_num);
// The same contraction on pairs of SMs (mo_tc_pair.cu): tiled vgl AO tensors
// only (25 points per tile, written with pair_zero), MMA N = bn (64, 96,
// 128, 160, 192 or 256) per pair of tiles; D[out_rows][mo] float.  C comes
// blocked (launch_pair_c): for each half h of an N tile (the rows one CTA
// of the pair multiplies, bn / 2 of them, zero-padded) and each K block, a
// contiguous [planes][bn / 2][128 bytes] block, so that each stage's C
// copy is one contiguous box.
// half_rows: the rows each half block holds (bn / 2 for a launch of MMA N
// bn; a multi-problem launch pads every problem's halves to bn_max / 2).
size_t pair_c_bytes(int mode, int64_t mo_num, int64_t ao_num, int bn, int half_rows);
// c_hi / c_lo: [mo][ldc] bf16 planes (QK_BF16X3) or c_hi [mo][ldc] FP32 (QK_TF32).
cudaError_t launch_pair_c(int mode, const void* c_hi, const void* c_lo, int64_t ldc,
                          int64_t mo_num, int64_t ao_num, int bn, int half_rows, void* c_blk,
                          cudaStream_t s);
cudaError_t launch_mo_tc_pair(int mode, const AOTensor& ao, int64_t ao_num, const void* c_blk,
                              int64_t mo_num, float* out, int bn, int* err_flag, cudaStream_t s,
                              int64_t out_rows);
// One problem of a multi-problem pair launch (device-resident; the tensor
// maps, 64-byte aligned by their type, are written by the host).
struct PairProblem {
  CUtensorMap a, b;      // blocked AO tensor; blocked C with halves of bn_max / 2 rows
  const uint8_t* mask;   // [tiles][mask_ld(nchunk)]
  const int32_t* perm;   // slot -> point (NULL: identity)
  float* D;              // [M][N] output
  int64_t M, N;          // output rows (5 * points) and columns
  int m_tiles, n_tiles, num_kb, nchunk;
  int bn, last_bn;       // MMA N of the N tiles and of the last one
  int zero_slice;        // a slice past the AO tensor's end
};
// Fill a PairProblem (host): the AO tensor written with pair_zero, C blocked
// by launch_pair_c(bn, bn_max / 2); bn <= bn_max.
bool tc_make_pair_problem(int mode, const AOTensor& ao, int64_t K, const void* c_blk, int64_t N,
                          float* out, int bn, int bn_max, int64_t out_rows, PairProblem* p);
// Persistent pair launch over a work list of int4 (problem, M-tile pair, N tile, 0).
cudaError_t launch_mo_tc_pair_batch(int mode, int bn_max, const PairProblem* probs,
                                    const int4* items, int64_t n_items, int* err_flag,
                                    cudaStream_t s);

// One contraction problem of a multi-problem launch (device-resident; the
// tensor maps, 64-byte aligned by their type, are written by the host
// before the launch).
struct TcProblem {
  CUtensorMap a, b;  // AO and C; QK_BF16X3: 3-D maps over the hi and lo planes
  float* D;                      // [M][N] output
  const uint8_t* mask;           // tiled AO tensor: [tiles][mask_ld(nchunk)] (else NULL)
  const int32_t* perm;           // tiled AO tensor: point of each slot (NULL: identity)
  int64_t M, N;                  // output rows (5 * points) and columns
  int num_kb;                    // K blocks
  int bn;                        // MMA N (multiple of 16, <= the launch's bn_max)
  int nchunk;
  int blocked;                   // AO tensor in the blocked layout (map over its slices)
};
// BN_MAX values instantiated for multi-problem launches.
extern const int kBatchBnMax[6];
// Fill a TcProblem (host): tensor maps over the AO tensor and C planes.
bool tc_make_problem(int mode, const AOTensor& ao, int64_t K, const void* c_hi, const void* c_lo,
                     int64_t ldc, int64_t N, float* out, int bn, int64_t out_rows,
                     TcProblem* p);
// Persistent launch over a work list of int4 (problem, m tile, n tile, 0).
cudaError_t launch_mo_tc_batch(int mode, int bn_max, const TcProblem* probs, const int4* items,
                               int64_t n_items, int* err_flag, cudaStream_t s);

// One AO problem of a multi-problem ao_vgl launch.
struct AOProblem {
  BasisDev b;
  PointsDev p;
  AOTensor out;  // chunked layout
};
// Persistent ao_vgl over a work list of int4 (problem, chunk, first tile,
// tile stride): an item takes tiles first, first + stride, ... of the
// problem's tiled AO tensor (kTilePoints points per tile).  split: bf16
// hi/lo planes, else FP32.
cudaError_t launch_ao_vgl_batch(bool split, const AOProblem* probs, const int4* items,
                                int64_t n_items, cudaStream_t s);

// Values-only AO tensor (ao_value.cu): tiled (128 points per tile, bf16
// hi/lo or FP32) for the tensor-core modes, dense rows = points (FP32 or
// FP64) otherwise; chunked columns in both.
int ao_value_tile_points();
cudaError_t launch_ao_value(const BasisDev& b, const PointsDev& p, int out_mode,
                            const AOTensor& out, cudaStream_t s);
// Single-electron moves in FP64 (single_mo.cu): C^T [ao][single_ct_ld] from
// C [mo][ao], then the MO vgl of the W moved points p into out [W][5][mo] in
// one launch (f64 must be true).
int64_t single_ct_ld(bool f64, int64_t mo_num);
cudaError_t launch_single_ct(bool f64, const double* C, int64_t mo_num, int64_t ao_num, void* ct,
                             cudaStream_t s);
cudaError_t launch_single_mo(bool f64, const BasisDev& b, const PointsDev& p, const void* ct,
                             int64_t mo_num, void* out, cudaStream_t s);
// Whether the one-launch kernel applies (FP64, and the basis tables fit its
// shared memory).
bool single_mo_fits(bool f64, const BasisDev& b);
// Single-electron moves (single.cu): src point w -> dst point w * elec_num + elec.
cudaError_t launch_scatter_points(const PointsDev& src, const PointsDev& dst, int64_t elec_num,
                                  int64_t elec, cudaStream_t s);
// Density helpers (density.cu).
cudaError_t launch_gather_rows(const void* src, int64_t ld, size_t elem, const int* rows,
                               int64_t nrows, void* dst, cudaStream_t s);
cudaError_t launch_density_reduce(const float* part, int parts, int64_t n, float* rho,
                                  cudaStream_t s);
// rho[p] = sum_i w[i] D[p][i]^2 for D [n][m] (FP64 or FP32, rho of the same type).
cudaError_t launch_density_from_mo(bool f64, const void* D, int64_t n, int64_t m,
                                   const double* w, void* rho, cudaStream_t s);

// Spatial order of the points (sort.cu): a permutation perm (slot -> point)
// and the point arrays in that order, in `scratch` of spatial_order_bytes(n)
// bytes; box_lo/box_hi bound the region the order resolves.
size_t spatial_order_bytes(int64_t n);
cudaError_t launch_spatial_order(const PointsDev& p, const float box_lo[3],
                                 const float box_hi[3], void* scratch, int32_t** perm,
                                 PointsDev* sorted, cudaStream_t s);
// Kernel launches launch_spatial_order makes for n points.
int spatial_order_kernels(int64_t n);
// Cell grid of the spatial order over a box: cell = (x - lo) * inv per axis.
void cell_grid(const float box_lo[3], const float box_hi[3], float3* lo, float3* inv);
// Several problems' points in one spatial order (sort.cu): the key of a
// point is (problem << cell bits) | its cell key in its problem's own grid,
// so each problem's points stay contiguous, problem after problem, in the
// order of a single problem within.
struct SortProblem {
  PointsDev p;      // the problem's points, caller order
  float3 lo, inv;   // its cell grid (cell_grid of its nuclear box)
  int spatial;      // 0: the problem keeps its caller order
};
struct BatchOrder {
  uint32_t* hist;
  uint32_t* key[2];
  int32_t* val[2];
  PointsDev sorted;  // every problem's points in order, problem j from off[j]; ld = total
  int32_t* perm;     // slot -> the problem's own point index
  int64_t total;
  int nprob, passes;
};
size_t spatial_order_batch_bytes(int64_t total, int nprob);
// Pointers into `scratch` (host arithmetic only).
BatchOrder spatial_order_batch_layout(void* scratch, int64_t total, int nprob);
// d_probs [nprob], d_off [nprob + 1] (off[0] = 0, off[nprob] = total) in device memory.
cudaError_t launch_spatial_order_batch(const BatchOrder& o, const SortProblem* d_probs,
                                       const int64_t* d_off, cudaStream_t s);
// Reach pre-pass of several tiled AO problems in one launch (problems whose
// out.reach is NULL are skipped); max_shells: the largest shell count.
cudaError_t launch_tile_reach_batch(const AOProblem* d_probs, int nprob, int64_t max_tiles,
                                    int max_shells, cudaStream_t s);

// MO cusp correction (cusp.cu, Sec. 3.3).
struct CuspDev {
  const double* rc;      // [nucl] sphere radius in bohr (0: no correction at A)
  const float* rc_f;     // [nucl] float(rc)
  const double* charge;  // [nucl] Z_A
  const int* s_start;    // [nucl + 1] range of each nucleus in s_shell
  const int* s_shell;    // the s shells of each nucleus
};
// Coefficients f [nucl][mo][4] (FP64 and FP32) of the current basis, C
// ([mo][ao] FP64) and radii; X [nucl][ao] and Q [nucl][mo] are scratch.
cudaError_t launch_cusp_setup(const BasisDev& b, const CuspDev& cu, int64_t mo_num,
                              const double* C, double* X, double* Q, double* f64, float* f32,
                              cudaStream_t s);
// Adds the correction to D [points][5][mo] (FP64 or FP32) at the points.
// FP64 output: C64 [mo][ao] and f64; FP32 output: C32 [mo][ldc32] and f32.
// scratch: cusp_list_bytes(p.n) bytes of device memory.  scan (optional):
// the same points in another order (the spatial order), perm[slot] = the
// point's index in p; the sphere search walks tiles of that order.
size_t cusp_list_bytes(int64_t n);
cudaError_t launch_cusp_apply(const BasisDev& b, const CuspDev& cu, const PointsDev& p,
                              const PointsDev* scan, const int32_t* perm, int64_t mo_num,
                              const double* C64, const float* C32, int64_t ldc32,
                              const double* f64, const float* f32, bool f64_out, void* D,
                              void* scratch, cudaStream_t s);

// Adjoint dR kernel: dR partials from Abar [5P][ld] (value type T) at the
// points, reduced into d_dR [nucl][3] (FP64).
cudaError_t launch_adjoint_dR(const BasisDev& b, const PointsDev& p, int mode,
                              const void* abar, int64_t ld, double* partial, double* d_dR,
                              cudaStream_t s);
size_t adjoint_dR_partial_bytes(const BasisDev& b, int64_t point_num);
// The same from Abar in live (tile, chunk) blocks [tiles][nchunk][128][64]
// (FP32) of the blocked AO tensor whose mask is `mask`; p: the points in the
// tiles' order.
cudaError_t launch_adjoint_dR_blocked(const BasisDev& b, const PointsDev& p, const float* abar,
                                      const uint8_t* mask, double* partial, double* d_dR,
                                      cudaStream_t s);

// Split-bf16 adjoint over the forward's blocked AO tensor (adjoint_sparse.cu).
// ctk: C^T hi/lo planes in the chunked column order, made from C [mo][kpad]
// (FP64) by launch_adjoint_ctk_split (adjoint_sparse_ctk_bytes).  Then, for
// W [P][5][mo] (FP32, the caller's points), the AO tensor `ao` (tiled,
// blocked, bf16 hi/lo, mask; ao.perm the tiles' points) and p the points in
// the tiles' order: d_dC [mo][ao] (FP64, the caller's AO order; NULL: not
// formed) and d_dR [nucl][3] (NULL: not formed).  zero_groups: zero the
// dead groups of live blocks first (once per AO tensor: the forward leaves
// them unwritten).  scratch: adjoint_sparse_scratch_bytes; dr_partial:
// adjoint_dR_partial_bytes.
size_t adjoint_sparse_ctk_bytes(int nchunk, int64_t mo_num);
cudaError_t launch_adjoint_ctk_split(const double* C64p, int64_t mo_num, int nchunk, void* ctk,
                                     cudaStream_t s);
size_t adjoint_sparse_scratch_bytes(int64_t point_num, int nchunk, int64_t mo_num);
cudaError_t launch_adjoint_sparse(const BasisDev& b, const PointsDev& p, const AOTensor& ao,
                                  const float* W, int64_t mo_num, const void* ctk, bool zero_groups,
                                  double* d_dC, double* d_dR, void* scratch, double* dr_partial,
                                  int* err_flag, cudaStream_t s);

// Fused AO + MO evaluation (split-bf16): live-chunk lists per 25-point tile,
// then one persistent kernel that builds AO blocks in shared memory and
// multiplies them on the tensor cores.
size_t fused_workspace_bytes(int64_t point_num, int nchunk);
cudaError_t launch_fused_live(const BasisDev& b, const PointsDev& p, int* live_count,
                              uint16_t* live_list, cudaStream_t s);
cudaError_t launch_mo_fused(int bn, const BasisDev& b, const PointsDev& p, const void* c_hi,
                            const void* c_lo, int64_t kpad, int64_t N, float* out,
                            const int* live_count, const uint16_t* live_list, int* err_flag,
                            cudaStream_t s);

// What a multi-molecule launch needs from one context (context.cu): makes
// the tables, MO planes and AO workspace of the current state valid and
// returns views of them.
struct ForwardViews {
  BasisDev b;
  PointsDev p;
  AOTensor ao;          // chunked
  const void* c_hi;     // contraction B planes (c_lo NULL for TF32)
  const void* c_lo;
  int64_t kpad, mo_num, walk_num, elec_num;
  int mode;
  uint64_t basis_version;  // bumped by every change of nuclei, basis, cutoff or order
  float box_lo[3], box_hi[3];  // nuclear box of the spatial point order
  bool spatial;                // whether the context cuts its tiles from that order
  uint64_t mo_version;         // bumped by every upload of C
};
qk_status context_forward_views(qk_context c, ForwardViews* v);
// Whether the context applies the MO cusp correction.
bool context_cusp_on(qk_context c);
// C blocked for the pair contraction at MMA N bn with halves of half_rows
// rows (built on the context's stream once per upload of C, tile shape and
// mode; *out stays valid until the next call with another shape).
qk_status context_pair_c(qk_context c, int bn, int half_rows, const void** out);
// Record that the workspace's AO tensor is not the context's own any more
// (a multi-molecule launch wrote it in its own point order).
void context_forget_ao(qk_context c);
qk_status context_fail(qk_context c, qk_status code, const char* msg);

}  // namespace qk
