// mo_tc.cu -- MO contraction on the 5th-generation (tcgen05) tensor cores.
//
// Eqs. 5-7 of the QMCkl paper as one product over the concatenated
// (point, component) rows (Sec. 3.2):  D[5P x N_mo] = AO[5P x N_ao] . C^T.
//
// Arithmetic:
//   QK_BF16X3  AO and C are each split into bf16 hi + lo (x = hi + lo + r,
//              |r| <= 2^-18 |x|) and D accumulates hi*hi + hi*lo + lo*hi in
//              FP32 (tcgen05.mma kind::f16, bf16 inputs, f32 accumulator).
//   QK_TF32    FP32 AO and C read as TF32 (kind::tf32), one product.
//
// Design: one CTA computes a 128-row x (NSUB*BN)-column tile of D.
//   warp 4     TMA producer: 128B-swizzled K-major tiles of AO and C into a
//              STAGES-deep shared-memory ring (mbarrier complete_tx).
//   warp 5     allocates TMEM; one thread issues the MMAs for each stage and
//              commits them to the stage's "empty" barrier.
//   warps 0-3  epilogue: wait for the last commit, read the FP32 accumulator
//              from TMEM (warp w owns TMEM lanes 32w..32w+31 = rows), turn
//              each 32 x 16 slice around in shared memory and store it as
//              64-byte row segments of D, 8 rows per instruction.
// Every wait is bounded (clock64); a wait that gives up records a code in the
// caller's error word, stops the pipeline, drains its own copies and MMAs,
// frees TMEM and returns.
#include <cuda.h>

#include "tc_common.cuh"

namespace qk {
namespace {

using namespace tc;

constexpr int kThreads = 192;       // 4 epilogue warps + producer + MMA
// Epilogue staging: each epilogue warp turns a 32-row x 16-column slice of
// the accumulator (one row per lane) around in shared memory so that each
// 16-byte global store instruction covers 8 rows x 64 contiguous bytes.
// 16-byte chunk q of row r sits at chunk q ^ ((r / 2) % 4): row writes (8
// lanes = 8 rows per phase) and row-pair reads are both free of bank
// conflicts.
constexpr int kEpiCols = 16;
constexpr int kEpiPitch = kEpiCols;
constexpr size_t kEpiBytes = 4 * 32 * kEpiPitch * sizeof(float);
constexpr size_t kSmemLimit = 232448;  // opt-in shared memory per block

template <int MODE, int BN_MAX, int STAGES>
struct TcShape {
  using TR = TcTraits<MODE>;
  static constexpr uint32_t A_BYTES = kBM * kRowBytes;
  static constexpr uint32_t B_BYTES = BN_MAX * kRowBytes;  // room for the widest B tile
  static constexpr uint32_t STAGE_BYTES = TR::kPlanes * (A_BYTES + B_BYTES);
  // accumulator buffers: as many BN_MAX-column regions (32-column aligned)
  // as the 512 TMEM columns hold, at most 4, so that the epilogue may trail
  // the MMAs by up to NBUF - 1 tiles
  static constexpr uint32_t ACC = (BN_MAX + 31) / 32 * 32;
  static constexpr int NBUF = 512 / ACC > 4 ? 4 : (int)(512 / ACC);
  static constexpr uint32_t TMEM_ALLOC = tmem_cols<NBUF * ACC>();
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES + 8 * (2 * STAGES + 2 * NBUF);
  static_assert(SMEM + kEpiBytes + 64 <= kSmemLimit, "shared memory budget");
  static_assert(BN_MAX % 16 == 0 && BN_MAX >= 16 && BN_MAX <= 256, "MMA N: 16..256, step 16");
};

// Stage word from the TMA producer to the MMA thread: bits 0-3 the k-steps
// to issue, kStageFirst / kStageLast on the first / last stage of a tile,
// the tile's MMA N / 16 from bit kStageBnShift (on every stage: the C lo
// plane sits N rows after the hi plane).
constexpr uint32_t kStageFirst = 1u << 4;
constexpr uint32_t kStageLast = 1u << 5;
constexpr int kStageBnShift = 8;

// One output tile as the three roles see it.
struct TileInfo {
  const CUtensorMap* a;  // AO tiles (QK_BF16X3: hi and lo planes in one 3-D map;
                         // blocked: a 3-D map over the tensor's column slices)
  const CUtensorMap* b;  // C tiles (likewise)
  float* D;
  const uint8_t* kmask;  // live 16-column groups of this M tile's chunks (NULL: all)
  const int32_t* perm;   // tiled: point of each slot (NULL: slot = point)
  int64_t M, N;          // output rows and columns
  int m0, n0;            // AO-tensor row and output column of the tile
  int num_kb;
  int bn;                // MMA N of this tile (multiple of 16, <= BN_MAX)
  int ntile;             // index of the tile's N range (density partials)
  bool tiled;            // rows: rows_per_tile live of 128, output row = rpt (m0/128) + local
  int rows_per_tile;     // tiled: 125 (vgl) or 128 (values only)
  int nchunk;
  bool ablocked;         // AO tensor in the blocked layout (coordinates: blocked_slice)
  const float* wdens;    // density epilogue: column weights (NULL: store D)
  float* rho;            // density epilogue: [N tiles][M] partial sums
};

// The MMA k-steps of a K block: bit kk = k-step kk meets a nonzero AO.  The
// mask byte of a 64-column chunk has a bit per 16-column group.  A K block
// of 64 bf16 columns is one chunk, its four k-steps of 16 one group each; a
// K block of 32 TF32 columns is half kb & 1 of chunk kb >> 1, and its
// k-steps of 8 take two per group.
template <int MODE>
constexpr int kb_per_chunk() {
  return TcTraits<MODE>::kBK == 64 ? 1 : 2;
}

// Whether any chunk of the tile holds a live group (whole warp: lanes take
// 16-chunk windows of the mask row; padding bytes past the last chunk are
// never written and are ignored).
template <int MODE>
__device__ __forceinline__ bool tile_live(const TileInfo& x, int lane) {
  if (x.kmask == nullptr) return true;
  const int nq = (x.num_kb + kb_per_chunk<MODE>() - 1) / kb_per_chunk<MODE>();
  const uint4* row = reinterpret_cast<const uint4*>(x.kmask);
  bool live = false;
  for (int w = lane; 16 * w < nq; w += 32) {
    const uint4 v = row[w];
    const int valid = nq - 16 * w;  // bytes of this window that are chunks
    const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int nb = valid - 4 * k;
      const uint32_t keep = nb >= 4 ? 0x0F0F0F0Fu : (nb <= 0 ? 0u : (0x0F0F0F0Fu >> (8 * (4 - nb))));
      live |= (wd[k] & keep) != 0u;
    }
  }
  return __any_sync(0xffffffffu, live);
}

// One problem: tile t -> (m, n) = (t / n_tiles, t % n_tiles), N tile fastest
// so that the N tiles of one M tile run together and share A through L2.
template <int BN>
struct SingleSched {
  CUtensorMap a, b;
  CUtensorMap b_last;  // the last N tile's C rows (box last_bn), when last_bn < BN
  int last_bn;         // MMA N of the last N tile: the MOs left, rounded up to 16
  float* D;
  const uint8_t* mask;  // [m tiles][mask_ld(nchunk)] when tiled
  const int32_t* perm;
  const float* wdens;
  float* rho;
  int64_t M, N, total;
  int num_kb, n_tiles, nchunk, rows_per_tile;
  bool tiled, blocked;
  __device__ __forceinline__ int64_t count() const { return total; }
  // the tensor maps into the TMA unit's cache before the first copy
  __device__ __forceinline__ void prefetch_maps() const {
    tma_prefetch_map(&a);
    tma_prefetch_map(&b);
    if (last_bn != BN) tma_prefetch_map(&b_last);
  }
  __device__ __forceinline__ TileInfo tile(int64_t t) const {
    TileInfo x;
    const int64_t mt =
        total <= 0x7fffffff ? (int64_t)((uint32_t)t / (uint32_t)n_tiles) : t / n_tiles;
    const int nt = (int)(t - mt * n_tiles);
    const bool last = nt == n_tiles - 1 && last_bn != BN;
    x.a = &a;
    x.b = last ? &b_last : &b;
    x.D = D;
    x.kmask = tiled ? mask + mt * mask_ld(nchunk) : nullptr;
    x.perm = perm;
    x.M = M;
    x.N = N;
    x.m0 = (int)(mt * kBM);
    x.n0 = nt * BN;
    x.num_kb = num_kb;
    x.bn = last ? last_bn : BN;
    x.ntile = nt;
    x.tiled = tiled;
    x.rows_per_tile = rows_per_tile;
    x.nchunk = nchunk;
    x.ablocked = blocked;
    x.wdens = wdens;
    x.rho = rho;
    return x;
  }
};

// Several problems: a work list of (problem, m tile, n tile) over descriptors
// in global memory (tensor maps written by the host before the launch).
struct BatchSched {
  const TcProblem* probs;
  const int4* items;
  int64_t n_items;
  __device__ __forceinline__ int64_t count() const { return n_items; }
  __device__ __forceinline__ void prefetch_maps() const {}  // maps differ per problem
  __device__ __forceinline__ TileInfo tile(int64_t t) const {
    const int4 it = items[t];
    const TcProblem& p = probs[it.x];
    TileInfo x;
    x.a = &p.a;
    x.b = &p.b;
    x.D = p.D;
    x.kmask = p.mask ? p.mask + (int64_t)it.y * mask_ld(p.nchunk) : nullptr;
    x.perm = p.perm;
    x.M = p.M;
    x.N = p.N;
    x.m0 = it.y * kBM;
    x.n0 = it.z * p.bn;
    x.num_kb = p.num_kb;
    x.bn = p.bn;
    x.ntile = it.z;
    x.tiled = p.mask != nullptr;
    x.rows_per_tile = 5 * kTilePoints;
    x.nchunk = p.nchunk;
    x.ablocked = p.blocked != 0;
    x.wdens = nullptr;
    x.rho = nullptr;
    return x;
  }
};

// Persistent: CTA c walks tiles t = c, c + gridDim.x, ...  The shared-memory
// ring runs on a k-block counter that continues across tiles; the
// accumulator cycles through NBUF TMEM buffers so that the epilogue of tile
// i overlaps the MMAs of the next tiles (tiles of few live K blocks take
// less MMA time than their epilogue, so a lag of more than one tile pays).
//   full[s]   TMA bytes of stage s landed        (producer -> MMA)
//   empty[s]  MMAs reading stage s finished      (MMA -> producer, commit)
//   tfull[b]  accumulator b complete             (MMA -> epilogue, commit)
//   tempty[b] accumulator b drained to global    (epilogue warps -> MMA)
template <int MODE, int BN_MAX, int STAGES, class Sched>
__global__ void __launch_bounds__(kThreads, 1)
    mo_tc_kernel(const __grid_constant__ Sched sched, int* err_flag) {
  using S = TcShape<MODE, BN_MAX, STAGES>;
  using TR = TcTraits<MODE>;
  constexpr uint32_t ACC = S::ACC;  // columns of one accumulator buffer
  constexpr uint32_t NBUF = S::NBUF;

  extern __shared__ unsigned char smem_raw[];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ uint32_t stage_info[STAGES];  // producer -> MMA, per stage (see kStageFirst)
  __shared__ uint16_t elist[64];           // producer's stage list (one 32-chunk window)
  __shared__ __align__(16) float epi[4][32][kEpiPitch];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // swizzle atoms need 1024-byte alignment
  const uint32_t bar0 = base + STAGES * S::STAGE_BYTES;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + NBUF + b); };

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  volatile int* abort_v = &abort_flag;
  const int64_t total = sched.count();

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < (int)NBUF; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), 4);  // one arrival per epilogue warp
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(S::TMEM_ALLOC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  // set-up done: from here on the previous kernel's results are read
  griddep_wait();

  if (warp == 4) {
    // ------------------------------------------------ TMA producer (warp)
    // Walks the tiles' live K blocks (blocks of screened AOs are never read)
    // and tells the MMA thread, per stage, which k-steps to issue and where
    // tiles begin and end; a tile with no live block still takes one stage
    // (no copies, no MMAs) so that the MMA thread walks stages only.  The
    // warp reads the mask bytes of 32 chunks at once and writes that
    // window's stages as a list in shared memory (entry: K block, bits
    // 0-9; its live k-steps, bits 10-13); lanes 0 and 1 walk the list
    // together, lane 0 taking the barriers and the AO copy, lane 1 the C
    // copy (each both planes in QK_BF16X3).
    constexpr int kPer = kb_per_chunk<MODE>();  // K blocks per chunk
    if (lane == 0) sched.prefetch_maps();
    uint32_t it = 0;  // stages taken (lanes 0 and 1)
    bool ok = true;
    for (int64_t t = blockIdx.x; t < total && ok; t += gridDim.x) {
      const TileInfo x = sched.tile(t);
      const uint32_t bytes = TR::kPlanes * (S::A_BYTES + (uint32_t)x.bn * kRowBytes);
      const int nq = (x.num_kb + kPer - 1) / kPer;  // chunks (the last may be half one)
      auto groups_of = [&](int q) -> uint32_t {
        if (q >= nq) return 0u;
        return x.kmask ? (uint32_t)x.kmask[q] & 0xFu : 0xFu;
      };
      // the tile's last live K block (-1: none)
      int lastkb = -1;
      for (int q0 = 0; q0 < nq; q0 += 32) {
        const uint32_t g = groups_of(q0 + lane);
        const unsigned live = __ballot_sync(0xffffffffu, g != 0u);
        if (live) {
          const int j = 31 - __clz(live);
          const uint32_t gj = __shfl_sync(0xffffffffu, g, j);
          lastkb = (q0 + j) * kPer + ((kPer == 2 && (gj & 0xCu)) ? 1 : 0);
        }
      }
      if (lastkb >= x.num_kb) lastkb = x.num_kb - 1;  // no mask, odd K block count
      // this lane's copy of a stage: lane 0 the AO tile, lane 1 the C tile
      const CUtensorMap* map = lane ? x.b : x.a;
      const uint32_t dst_off = lane ? TR::kPlanes * S::A_BYTES : 0u;
      const int row0 = lane ? x.n0 : x.m0;
      const uint32_t bn_bits = (uint32_t)(x.bn >> 4) << kStageBnShift;  // on every stage
      uint32_t flags = kStageFirst;
      // one stage (lanes 0 and 1): wait for the slot, post the stage word
      // (lane 0), issue this lane's copy
      auto stage = [&](int kb, uint32_t steps) -> bool {
        const int s = it % STAGES;
        const uint32_t ph = (it / STAGES) & 1u;
        ++it;
        if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_v)) {
          flag_error(err_flag, abort_v, 1);
          return false;
        }
        if (lane == 0) {
          stage_info[s] = steps | flags | bn_bits | (kb == lastkb ? kStageLast : 0u);
          mbar_expect_tx(full_bar(s), kb >= 0 ? bytes : 0u);
        }
        flags = 0;
        if (kb >= 0) {
          const uint32_t dst = base + s * S::STAGE_BYTES + dst_off;
          if (lane == 0 && x.ablocked)
            tma_load_3d(dst, map, full_bar(s), 0, 0,
                        blocked_slice<MODE>(x.m0 / kBM, kb, x.nchunk));
          else if constexpr (TR::kPlanes == 2)
            tma_load_3d(dst, map, full_bar(s), kb * TR::kBK, row0, 0);
          else
            tma_load_2d(dst, map, full_bar(s), kb * TR::kBK, row0);
        }
        return true;
      };
      if (lastkb < 0) {
        if (lane < 2) ok = stage(-1, 0u);
        ok = __all_sync(0xffffffffu, ok);
        continue;
      }
      for (int q0 = 0; q0 < nq && ok; q0 += 32) {
        const uint32_t g = groups_of(q0 + lane);
        uint32_t e[2] = {0u, 0u};
#pragma unroll
        for (int h = 0; h < kPer; ++h) {
          uint32_t steps = g;
          if constexpr (kPer == 2) {
            const uint32_t hh = (g >> (2 * h)) & 3u;
            steps = (hh & 1u ? 0x3u : 0u) | (hh & 2u ? 0xCu : 0u);
          }
          const int kb = (q0 + lane) * kPer + h;
          if (steps && kb < x.num_kb) e[h] = (uint32_t)kb | (steps << 10);
        }
        const unsigned b0 = __ballot_sync(0xffffffffu, e[0] != 0u);
        const unsigned b1 = __ballot_sync(0xffffffffu, e[1] != 0u);
        const unsigned lt = (1u << lane) - 1u;
        const int pos = __popc(b0 & lt) + __popc(b1 & lt);
        if (e[0]) elist[pos] = (uint16_t)e[0];
        if (e[1]) elist[pos + (e[0] ? 1 : 0)] = (uint16_t)e[1];
        const int n_e = __popc(b0) + __popc(b1);
        __syncwarp();
        if (lane < 2) {
          for (int k = 0; k < n_e && ok; ++k) {
            const uint32_t v = elist[k];
            // the next entry's AO block into L2 now, so that its copy into
            // the ring (a stage later) does not wait on HBM
            if constexpr (kPer == 1) {
              if (lane == 0 && k + 1 < n_e) {
                const int kn = (int)(elist[k + 1] & 0x3FFu);
                if (x.ablocked)
                  tma_prefetch_l2_3d(x.a, 0, 0, blocked_slice<MODE>(x.m0 / kBM, kn, x.nchunk));
                else
                  tma_prefetch_l2_3d(x.a, kn * TR::kBK, x.m0, 0);
              }
            }
            ok = stage((int)(v & 0x3FFu), (v >> 10) & 0xFu);
          }
        }
        ok = __all_sync(0xffffffffu, ok);  // also: the list may be rewritten
      }
    }
    if (lane == 0 && *abort_v) {
      // drain: let the copies already issued land before the CTA leaves
      const uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0u;
      for (uint32_t k = first; k < it; ++k) {
        const long long t0 = clock64();
        while (!mbar_try_wait(full_bar(k % STAGES), (k / STAGES) & 1u) &&
               clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp == 5 && lane == 0) {
    // ------------------------------------------------ MMA issuer
    // Stage by stage: the producer's stage word gives the k-steps to issue
    // and marks the first and last stage of each tile.  Descriptors are
    // those of stage 0 plus the byte offset / 16 (the start-address field
    // cannot carry: shared addresses stay below 256 KB).
    const int64_t my_tiles =
        total > (int64_t)blockIdx.x ? (total - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint64_t d0 = sw128_desc(base);
    uint32_t it = 0, i = 0, b = 0, dacc = tmem, idesc = 0;
    bool first = true, in_tile = false, ok = true;
    while ((int64_t)i < my_tiles) {
      const int s = it % STAGES;
      const uint32_t ph = (it / STAGES) & 1u;
      ++it;
      if (!mbar_wait(full_bar(s), ph, abort_v)) {
        flag_error(err_flag, abort_v, 2);
        ok = false;
        break;
      }
      const uint32_t info = stage_info[s];
      if (info & kStageFirst) {
        b = i % NBUF;
        if (!mbar_wait(tempty_bar(b), ((i / NBUF) & 1u) ^ 1u, abort_v)) {
          flag_error(err_flag, abort_v, 2);
          ok = false;
          break;
        }
        in_tile = true;
        dacc = tmem + b * ACC;
        idesc = make_idesc(TR::kFmt, kBM, (int)((info >> kStageBnShift) << 4));
        first = true;  // the tile's first MMA overwrites the accumulator
      }
      tc_fence_after();
      const uint64_t da = d0 + ((uint64_t)(s * S::STAGE_BYTES) >> 4);
      const uint64_t da_lo = da + (S::A_BYTES >> 4);
      const uint64_t db = da + ((TR::kPlanes * S::A_BYTES) >> 4);
      // the C lo plane follows the hi plane's bn rows (one 3-D box)
      const uint64_t db_lo = db + ((((info >> kStageBnShift) << 4) * kRowBytes) >> 4);
#pragma unroll
      for (int kk = 0; kk < kRowBytes / kUmmaKBytes; ++kk) {
        // k-steps over AO columns that are zero at every row of the tile
        // would add exact zeros
        if (!((info >> kk) & 1u)) continue;
        const uint64_t ko = (uint64_t)(kk * kUmmaKBytes) >> 4;
        const uint32_t acc = first ? 0u : 1u;
        first = false;
        umma<MODE>(dacc, da + ko, db + ko, idesc, acc);
        if constexpr (MODE == QK_BF16X3) {
          umma<MODE>(dacc, da + ko, db_lo + ko, idesc, 1u);
          umma<MODE>(dacc, da_lo + ko, db + ko, idesc, 1u);
        }
      }
      umma_commit(empty_bar(s));  // stage s is free once these MMAs finish
      if (info & kStageLast) {
        umma_commit(tfull_bar(b));  // accumulator b complete
        in_tile = false;
        ++i;
      }
    }
    if (!ok) {
      // aborted: the MMAs in flight must finish before TMEM can be freed;
      // a tile cut short still gets its commit (the epilogue sees the abort
      // flag and does not read it)
      uint32_t wb = 0, wi = 0;
      bool wait = false;
      if (in_tile) {
        umma_commit(tfull_bar(b));
        wb = b;
        wi = i;
        wait = true;
      } else if (i > 0) {
        wb = (i - 1) % NBUF;
        wi = i - 1;
        wait = true;
      }
      const long long t0 = clock64();
      while (wait && !mbar_try_wait(tfull_bar(wb), (wi / NBUF) & 1u) &&
             clock64() - t0 < kWaitCycles) {
      }
    }
  } else if (warp < 4) {
    // ------------------------------------------------ epilogue
    uint32_t i = 0;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x, ++i) {
      const uint32_t b = i % NBUF;
      const long long t0 = clock64();
      bool ok = true;
      while (!mbar_try_wait(tfull_bar(b), (i / NBUF) & 1u)) {
        if (clock64() - t0 > kWaitCycles) {
          ok = false;
          break;
        }
      }
      if (!ok) flag_error(err_flag, abort_v, 3);
      ok = __all_sync(0xffffffffu, ok) && !*abort_v;
      __syncwarp();
      if (!ok) break;
      tc_fence_after();
      const TileInfo x = sched.tile(t);
      const bool any_live = tile_live<MODE>(x, lane);
      const uint32_t tbase = tmem + b * ACC + ((uint32_t)(warp * 32) << 16);
      const int64_t N = x.N;
      // store phase: lane -> row 8 i + lane / 4 of the warp's 32, columns
      // 4 (lane % 4) .. + 3 of the slice
      const int rq = lane >> 2;
      const int cq = (lane & 3) * 4;
      const bool vec = (N % 4) == 0 && (reinterpret_cast<uintptr_t>(x.D) & 15) == 0;
      const int64_t row0 = x.tiled ? (int64_t)(x.m0 / kBM) * x.rows_per_tile : (int64_t)x.m0;
      const int rows_here = x.tiled ? x.rows_per_tile : kBM;  // tile rows that exist in D
      if (x.rho) {
        // density: this thread's TMEM lane is its row; sum w_n D_n^2 over the tile's columns
        const int loc = warp * 32 + lane;
        float acc = 0.0f;
#pragma unroll 1
        for (int c = 0; c < x.bn; c += 16) {
          float v[16];
          if (any_live) {
            tmem_ld16(tbase + c, v);
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = 0.0f;
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int64_t col = x.n0 + c + q;
            if (col < N) acc += x.wdens[col] * v[q] * v[q];
          }
        }
        if (loc < rows_here && row0 + loc < x.M)
          x.rho[(int64_t)x.ntile * x.M + row0 + loc] = acc;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty_bar(b));
        continue;
      }
      // the four output rows this lane writes (slot rows mapped to the
      // caller's points when the tiles hold a spatial order); -1: none
      int64_t orow[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int loc = warp * 32 + 8 * i + rq;
        const int64_t lin = row0 + loc;
        orow[i] = (loc < rows_here && lin < x.M)
                      ? (x.perm ? 5 * (int64_t)x.perm[lin / 5] + lin % 5 : lin)
                      : -1;
      }
      float(*stg)[kEpiPitch] = epi[warp];
      float* rowp[4];  // start of each output row of this lane
#pragma unroll
      for (int i = 0; i < 4; ++i) rowp[i] = x.D + (orow[i] >= 0 ? orow[i] : 0) * N;
      // one 16-column slice through the staging buffer to D
      auto store_slice = [&](const float* v, int c) {
        float4* srow = reinterpret_cast<float4*>(&stg[lane][0]);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          srow[q ^ ((lane >> 1) & 3)] =
              make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        __syncwarp();
        const int64_t col = x.n0 + c + cq;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = 8 * i + rq;
          if (orow[i] >= 0) {
            const float4 w =
                reinterpret_cast<const float4*>(&stg[r][0])[(lane & 3) ^ ((r >> 1) & 3)];
            float* dst = rowp[i] + col;
            if (vec && col + 3 < N) {
              *reinterpret_cast<float4*>(dst) = w;
            } else {
              if (col < N) dst[0] = w.x;
              if (col + 1 < N) dst[1] = w.y;
              if (col + 2 < N) dst[2] = w.z;
              if (col + 3 < N) dst[3] = w.w;
            }
          }
        }
        __syncwarp();
      };
      // 32 columns per TMEM round trip (two loads, one wait)
#pragma unroll 1
      for (int c = 0; c < x.bn; c += 32) {
        const bool two = c + 16 < x.bn;
        float v[32];
        if (any_live) {
          tmem_ld16x2(tbase + c, v, two);
        } else {  // every AO of the tile was screened: the MOs are exactly zero
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = 0.0f;
        }
        store_slice(v, c);
        if (two) store_slice(v + 16, c + 16);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar(b));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(S::TMEM_ALLOC)
                 : "memory");
  }
}

// ----------------------------------------------------------------- host ---

constexpr int stages_for(int mode, int bn) {
  // as many stages as the shared memory left by the epilogue staging holds, at most 8
  return (int)((kSmemLimit - kEpiBytes - 1024 - 512) /
               ((mode == QK_BF16X3 ? 2 : 1) * (kBM + bn) * kRowBytes)) > 8
             ? 8
             : (int)((kSmemLimit - kEpiBytes - 1024 - 512) /
                     ((mode == QK_BF16X3 ? 2 : 1) * (kBM + bn) * kRowBytes));
}

// Grid of resident CTAs for a kernel instance (TMEM never oversubscribed).
template <auto Kern>
cudaError_t persistent_grid(size_t smem, uint32_t tmem_cols, int64_t work, int64_t* grid) {
  KernelFacts f;
  cudaError_t e = kernel_facts<Kern>(smem, kThreads, &f);
  if (e != cudaSuccess) return e;
  const int occ = f.occ;
  if (occ < 1 || occ * (int)tmem_cols > 512) return cudaErrorInvalidConfiguration;
  *grid = work < (int64_t)f.sms * occ ? work : (int64_t)f.sms * occ;
  return cudaSuccess;
}

template <int MODE, int BN>
cudaError_t launch_single(const AOTensor& ao, int64_t K, const void* c_hi, const void* c_lo,
                          int64_t ldc, int64_t N, float* out, int64_t out_rows, int* err_flag,
                          cudaStream_t s, const float* wdens, float* rho) {
  constexpr int ST = stages_for(MODE, BN);
  using S = TcShape<MODE, BN, ST>;
  using TR = TcTraits<MODE>;
  static_assert(S::SMEM <= 232448, "shared memory budget");
  const bool f32 = MODE == QK_TF32;
  const int64_t M = ao.rows;
  if (M == 0 || N == 0) return cudaSuccess;
  if (M > INT32_MAX || K > INT32_MAX || N > INT32_MAX) return cudaErrorInvalidValue;
  if (ao.tiled && M % kBM != 0) return cudaErrorInvalidValue;
  if (ao.blocked && (!ao.tiled || K > (int64_t)ao.nchunk * kChunkAO)) return cudaErrorInvalidValue;
  SingleSched<BN> sc;
  // the last N tile multiplies only the MOs it has, rounded up to 16
  const int64_t n_tiles = (N + BN - 1) / BN;
  const int last_bn = (int)((N - (n_tiles - 1) * BN + 15) / 16 * 16);
  sc.last_bn = last_bn;
  if (ao.blocked) {
    if (!make_map_blocked(&sc.a, ao.a, TR::kPlanes == 2, M / kBM * ao.nchunk))
      return cudaErrorInvalidValue;
  } else if (TR::kPlanes == 2) {
    if (!make_map_planes(&sc.a, ao.a, ao.a_lo, K, M, ao.ld, TR::kBK, kBM))
      return cudaErrorInvalidValue;
  } else {
    if (!make_map(&sc.a, ao.a, f32, K, M, ao.ld, TR::kBK, kBM)) return cudaErrorInvalidValue;
  }
  if (TR::kPlanes == 2) {
    if (!make_map_planes(&sc.b, c_hi, c_lo, K, N, ldc, TR::kBK, BN)) return cudaErrorInvalidValue;
    if (last_bn != BN && !make_map_planes(&sc.b_last, c_hi, c_lo, K, N, ldc, TR::kBK, last_bn))
      return cudaErrorInvalidValue;
  } else {
    if (!make_map(&sc.b, c_hi, f32, K, N, ldc, TR::kBK, BN)) return cudaErrorInvalidValue;
    if (last_bn != BN && !make_map(&sc.b_last, c_hi, f32, K, N, ldc, TR::kBK, last_bn))
      return cudaErrorInvalidValue;
  }
  sc.D = out;
  sc.mask = ao.tiled ? ao.mask : nullptr;
  sc.perm = ao.tiled ? ao.perm : nullptr;
  sc.rows_per_tile = ao.comps == 1 ? kBM : 5 * kTilePoints;
  sc.wdens = wdens;
  sc.rho = rho;
  sc.tiled = ao.tiled;
  sc.blocked = ao.blocked;
  sc.nchunk = ao.nchunk;
  sc.M = ao.tiled ? out_rows : M;
  sc.N = N;
  sc.num_kb = (int)((K + TR::kBK - 1) / TR::kBK);
  sc.n_tiles = (int)((N + BN - 1) / BN);
  sc.total = ((M + kBM - 1) / kBM) * sc.n_tiles;
  auto kern = mo_tc_kernel<MODE, BN, ST, SingleSched<BN>>;
  int64_t grid = 0;
  cudaError_t e = persistent_grid<mo_tc_kernel<MODE, BN, ST, SingleSched<BN>>>(
      S::SMEM, S::TMEM_ALLOC, sc.total, &grid);
  if (e != cudaSuccess) return e;
  return launch_pdl(kern, (unsigned)grid, kThreads, S::SMEM, s, sc, err_flag);
}

template <int MODE>
cudaError_t launch_mode(const TcConfig& cfg, const AOTensor& ao, int64_t K, const void* c_hi,
                        const void* c_lo, int64_t ldc, int64_t N, float* out, int64_t out_rows,
                        int* err_flag, cudaStream_t s, const float* wdens, float* rho) {
  switch (cfg.bn) {
    case 16: return launch_single<MODE, 16>(ao, K, c_hi, c_lo, ldc, N, out, out_rows, err_flag, s, wdens, rho);
    case 32: return launch_single<MODE, 32>(ao, K, c_hi, c_lo, ldc, N, out, out_rows, err_flag, s, wdens, rho);
    case 64: return launch_single<MODE, 64>(ao, K, c_hi, c_lo, ldc, N, out, out_rows, err_flag, s, wdens, rho);
    case 96: return launch_single<MODE, 96>(ao, K, c_hi, c_lo, ldc, N, out, out_rows, err_flag, s, wdens, rho);
    case 128: return launch_single<MODE, 128>(ao, K, c_hi, c_lo, ldc, N, out, out_rows, err_flag, s, wdens, rho);
    case 160: return launch_single<MODE, 160>(ao, K, c_hi, c_lo, ldc, N, out, out_rows, err_flag, s, wdens, rho);
    case 192: return launch_single<MODE, 192>(ao, K, c_hi, c_lo, ldc, N, out, out_rows, err_flag, s, wdens, rho);
    case 256: return launch_single<MODE, 256>(ao, K, c_hi, c_lo, ldc, N, out, out_rows, err_flag, s, wdens, rho);
    default: return cudaErrorInvalidValue;
  }
}

template <int MODE, int BN_MAX>
cudaError_t launch_batch_bn(const TcProblem* probs, const int4* items, int64_t n_items,
                            int* err_flag, cudaStream_t s) {
  constexpr int ST = stages_for(MODE, BN_MAX);
  using S = TcShape<MODE, BN_MAX, ST>;
  static_assert(S::SMEM <= 232448, "shared memory budget");
  if (n_items == 0) return cudaSuccess;
  BatchSched sc{probs, items, n_items};
  auto kern = mo_tc_kernel<MODE, BN_MAX, ST, BatchSched>;
  int64_t grid = 0;
  cudaError_t e = persistent_grid<mo_tc_kernel<MODE, BN_MAX, ST, BatchSched>>(
      S::SMEM, S::TMEM_ALLOC, n_items, &grid);
  if (e != cudaSuccess) return e;
  return launch_pdl(kern, (unsigned)grid, kThreads, S::SMEM, s, sc, err_flag);
}

template <int MODE>
cudaError_t launch_batch_mode(int bn_max, const TcProblem* probs, const int4* items,
                              int64_t n_items, int* err_flag, cudaStream_t s) {
  switch (bn_max) {
    case 64: return launch_batch_bn<MODE, 64>(probs, items, n_items, err_flag, s);
    case 96: return launch_batch_bn<MODE, 96>(probs, items, n_items, err_flag, s);
    case 128: return launch_batch_bn<MODE, 128>(probs, items, n_items, err_flag, s);
    case 160: return launch_batch_bn<MODE, 160>(probs, items, n_items, err_flag, s);
    case 192: return launch_batch_bn<MODE, 192>(probs, items, n_items, err_flag, s);
    case 256: return launch_batch_bn<MODE, 256>(probs, items, n_items, err_flag, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

TcConfig tc_default_config(int mode, int64_t mo_num) {
  (void)mode;
  static const int bns[] = {16, 32, 64, 96, 128, 160, 192, 256};
  const int64_t tiles = (mo_num + 255) / 256;
  const int64_t per = (mo_num + tiles - 1) / tiles;
  int bn = 256;
  for (int b : bns)
    if (b >= per) {
      bn = b;
      break;
    }
  return TcConfig{bn, 1, 0};
}

const int kBatchBnMax[] = {64, 96, 128, 160, 192, 256};

bool tc_make_problem(int mode, const AOTensor& ao, int64_t K, const void* c_hi, const void* c_lo,
                     int64_t ldc, int64_t N, float* out, int bn, int64_t out_rows,
                     TcProblem* p) {
  const bool f32 = mode == QK_TF32;
  const int bk = f32 ? TcTraits<QK_TF32>::kBK : TcTraits<QK_BF16X3>::kBK;
  if (bn % 16 != 0 || bn < 16 || bn > 256) return false;
  if (ao.rows > INT32_MAX || K > INT32_MAX || N > INT32_MAX) return false;
  if (ao.blocked) {
    if (!ao.tiled || ao.rows % kBM != 0 || K > (int64_t)ao.nchunk * kChunkAO) return false;
    if (!make_map_blocked(&p->a, ao.a, !f32, ao.rows / kBM * ao.nchunk)) return false;
  } else if (!f32) {
    if (!make_map_planes(&p->a, ao.a, ao.a_lo, K, ao.rows, ao.ld, bk, kBM)) return false;
  } else {
    if (!make_map(&p->a, ao.a, f32, K, ao.rows, ao.ld, bk, kBM)) return false;
  }
  if (!f32) {
    if (!make_map_planes(&p->b, c_hi, c_lo, K, N, ldc, bk, bn)) return false;
  } else {
    if (!make_map(&p->b, c_hi, f32, K, N, ldc, bk, bn)) return false;
  }
  p->D = out;
  p->mask = ao.tiled ? ao.mask : nullptr;
  p->perm = ao.tiled ? ao.perm : nullptr;
  p->nchunk = ao.nchunk;
  p->blocked = ao.blocked ? 1 : 0;
  p->M = out_rows;
  p->N = N;
  p->num_kb = (int)((K + bk - 1) / bk);
  p->bn = bn;
  return true;
}

cudaError_t launch_mo_tc_batch(int mode, int bn_max, const TcProblem* probs, const int4* items,
                               int64_t n_items, int* err_flag, cudaStream_t s) {
  if (mode == QK_BF16X3)
    return launch_batch_mode<QK_BF16X3>(bn_max, probs, items, n_items, err_flag, s);
  if (mode == QK_TF32)
    return launch_batch_mode<QK_TF32>(bn_max, probs, items, n_items, err_flag, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_mo_tc(int mode, const AOTensor& ao, int64_t ao_num, const void* c_hi,
                         const void* c_lo, int64_t ldc, int64_t mo_num, float* out,
                         const TcConfig& cfg, int* err_flag, cudaStream_t s, int64_t out_rows,
                         const float* wdens, float* rho_part) {
  if (out_rows < 0) out_rows = ao.rows;
  if ((wdens == nullptr) != (rho_part == nullptr)) return cudaErrorInvalidValue;
  if (mode == QK_BF16X3)
    return launch_mode<QK_BF16X3>(cfg, ao, ao_num, c_hi, c_lo, ldc, mo_num, out, out_rows,
                                  err_flag, s, wdens, rho_part);
  if (mode == QK_TF32)
    return launch_mode<QK_TF32>(cfg, ao, ao_num, c_hi, c_lo, ldc, mo_num, out, out_rows,
                                err_flag, s, wdens, rho_part);
  return cudaErrorInvalidValue;
}

}  // namespace qk
