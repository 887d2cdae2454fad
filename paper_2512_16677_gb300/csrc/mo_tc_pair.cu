// mo_tc_pair.cu -- the MO contraction of Eqs. 5-7 on pairs of SMs.
//
// Same product as mo_tc.cu, D[5P x N_mo] = AO[5P x N_ao] . C^T over the
// tiled block-sparse AO tensor (Sec. 3.2's sparse-AO MO product at tile
// granularity), with split-bf16 (hi*hi + hi*lo + lo*hi, FP32 accumulation
// in TMEM) or TF32 operands.  The difference is the tensor-core issue: the
// two CTAs of a cluster run one tcgen05.mma.cta_group::2 with M = 256 (two
// consecutive 25-point tiles, one per CTA), and each CTA stages only half of
// the C tile (N / 2 rows).  Per SM a pipeline stage then carries the AO
// block (32 KB, one contiguous box of the blocked layout) and half the C
// block (20 KB at N = 160, one contiguous box of C blocked per half N tile
// and K block) instead of the whole C block (40 KB), so four stages fit
// where three did, and every C byte fetched from L2 serves twice the MMA
// work.  The kernel takes a scheduler: one problem (pair-tile p -> M-tile
// pair, N tile), or a work list over several molecules' problems.
//
// The two tiles of a pair share one K sequence: the union of their live AO
// blocks and 16-AO column groups.  A block dead in this CTA's own tile is
// loaded from outside the tensor (TMA zero fill, no memory traffic); a
// column group live in the partner only holds zeros in this tile's block,
// because ao_vgl writes zeros there (it reads the partner's reach word).
//
// Roles (224 threads per CTA):
//   warps 4, 6 TMA producers in both CTAs: warp 4 the own AO block, warp 6
//              the own half of the C block (a thread's copies complete one
//              after another, so each operand gets its own issuing warp); the
//              copies of both CTAs complete on the leader CTA's full barrier.
//              Each warp builds a 32-chunk window's stage list, one lane walks
//              it (wait, stage word, copy) and prefetches the next own AO
//              block into L2.
//   warp 5     TMEM allocation (cta_group::2, both CTAs); lane 0 of the
//              leader issues the MMAs and commits them to both CTAs'
//              barriers (multicast).
//   warps 0-3  epilogue in both CTAs: own 128 TMEM lanes = own tile's rows,
//              written through the point permutation; each warp then
//              arrives on the leader's accumulator-free barrier.
// Every wait is bounded (clock64); a wait that gives up records a code in
// the caller's error word and raises the CTA's abort flag.
#include <cuda.h>

#include <algorithm>

#include "tc_common.cuh"

namespace qk {
namespace {

using namespace tc;

constexpr int kThreads = 224;  // 4 epilogue warps, AO producer, MMA, C producer
constexpr size_t kEpiBytes = 4 * 32 * 32 * sizeof(float);  // epilogue staging
constexpr size_t kSmemLimit = 232448;

constexpr uint32_t kStageFirst = 1u << 4;
constexpr uint32_t kStageLast = 1u << 5;
constexpr int kStageBnShift = 8;

template <int MODE, int BN, int STAGES>
struct PairShape {
  using TR = TcTraits<MODE>;
  static constexpr uint32_t A_BYTES = kBM * kRowBytes;            // own 128 rows
  static constexpr uint32_t BH_BYTES = (BN / 2) * kRowBytes;      // own half of C
  static constexpr uint32_t STAGE_BYTES = TR::kPlanes * (A_BYTES + BH_BYTES);
  static constexpr uint32_t ACC = (BN + 31) / 32 * 32;
  static constexpr int NBUF = 512 / ACC > 4 ? 4 : (int)(512 / ACC);
  static constexpr uint32_t TMEM_ALLOC = tmem_cols<NBUF * ACC>();
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES + 8 * (2 * STAGES + 2 * NBUF);
  static_assert(SMEM + kEpiBytes + 512 <= kSmemLimit, "shared memory budget");
  static_assert(BN % 16 == 0, "MMA N: multiple of 16 (halves of whole 8-row groups)");
  static_assert(BN >= 32 && BN <= 256, "MMA N of a pair: 32..256");
};

constexpr int stages_for_pair(int mode, int bn) {
  return (int)((kSmemLimit - kEpiBytes - 1024 - 1024) /
               ((mode == QK_BF16X3 ? 2 : 1) * (kBM + bn / 2) * kRowBytes)) > 8
             ? 8
             : (int)((kSmemLimit - kEpiBytes - 1024 - 1024) /
                     ((mode == QK_BF16X3 ? 2 : 1) * (kBM + bn / 2) * kRowBytes));
}

// One pair-tile as the roles see it: M tiles 2 mp (leader) and 2 mp + 1
// (partner) of a problem, N tile nt.
struct PairTile {
  const CUtensorMap* a;  // blocked AO tensor: 3-D map over its column slices (one box = one K block)
  const CUtensorMap* b;  // blocked C: 3-D map over its [BN / 2][128-byte] slices
  const uint8_t* mask;   // [m tiles][mask_ld(nchunk)]
  const int32_t* perm;   // slot -> point (NULL: identity)
  float* D;
  int64_t M, N;          // output rows (5 points) and columns
  int mp, nt;            // M-tile pair and N tile
  int n0, bn;            // first output column and MMA N of the tile
  int m_tiles, num_kb, nchunk;
  int zero_slice;        // a slice past the AO tensor's end: its box reads zeros
};

// One problem: pair-tile p -> (M tile pair p / n_tiles, N tile p % n_tiles).
template <int BN>
struct PairSched {
  CUtensorMap a, b;
  int last_bn;           // MMA N of the last N tile (the MOs left, rounded up to 16)
  float* D;
  const uint8_t* mask;
  const int32_t* perm;
  int64_t M, N;
  int zero_slice, m_tiles, n_tiles, num_kb, nchunk;
  int64_t total;         // pair-tiles
  __device__ __forceinline__ int64_t count() const { return total; }
  __device__ __forceinline__ void prefetch_map(bool a_side) const {
    tma_prefetch_map(a_side ? &a : &b);
  }
  __device__ __forceinline__ PairTile tile(int64_t p) const {
    PairTile x;
    x.mp = (int)(p / n_tiles);
    x.nt = (int)(p - (int64_t)x.mp * n_tiles);
    x.bn = x.nt == n_tiles - 1 ? last_bn : BN;
    x.n0 = x.nt * BN;
    x.a = &a;
    x.b = &b;
    x.mask = mask;
    x.perm = perm;
    x.D = D;
    x.M = M;
    x.N = N;
    x.m_tiles = m_tiles;
    x.num_kb = num_kb;
    x.nchunk = nchunk;
    x.zero_slice = zero_slice;
    return x;
  }
};

// Several problems: a work list of (problem, M-tile pair, N tile) over
// descriptors in global memory (tensor maps written by the host).
struct PairBatchSched {
  const PairProblem* probs;
  const int4* items;
  int64_t n_items;
  __device__ __forceinline__ int64_t count() const { return n_items; }
  __device__ __forceinline__ void prefetch_map(bool) const {}  // maps differ per problem
  __device__ __forceinline__ PairTile tile(int64_t p) const {
    const int4 it = items[p];
    const PairProblem& P = probs[it.x];
    PairTile x;
    x.mp = it.y;
    x.nt = it.z;
    x.bn = x.nt == P.n_tiles - 1 ? P.last_bn : P.bn;
    x.n0 = x.nt * P.bn;
    x.a = &P.a;
    x.b = &P.b;
    x.mask = P.mask;
    x.perm = P.perm;
    x.D = P.D;
    x.M = P.M;
    x.N = P.N;
    x.m_tiles = P.m_tiles;
    x.num_kb = P.num_kb;
    x.nchunk = P.nchunk;
    x.zero_slice = P.zero_slice;
    return x;
  }
};

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Shared-memory address `addr` of this CTA as seen in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// Arrive on an mbarrier of a CTA of the cluster (cluster address), without
// ordering this thread's earlier memory operations before the arrival.
__device__ __forceinline__ void mbar_arrive_cluster_relaxed(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}

// TMA tile loads whose completion may be counted on the peer CTA's barrier.
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap* map,
                                                 uint32_t bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map,
                                                 uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}

template <int MODE>
__device__ __forceinline__ void umma_pair(uint32_t tmem_d, uint64_t a, uint64_t b,
                                          uint32_t idesc, uint32_t accumulate) {
  if constexpr (MODE == QK_BF16X3) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  }
}

// Commit the leader's MMAs issued so far to the barrier at the same offset in
// both CTAs of the pair.
__device__ __forceinline__ void umma_commit_pair(uint32_t bar) {
  asm volatile(
      "{\n\t.reg .b16 m;\n\tmov.b16 m, 3;\n\t"
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
      "[%0], m;\n\t}\n" ::"r"(bar)
      : "memory");
}

// Mask windows of 32 chunks a lane holds for one pair-tile (chunks <= 256).
constexpr int kMaxWin = 8;

__device__ __forceinline__ uint32_t pick_window(const uint32_t (&g)[kMaxWin], int w) {
  uint32_t v = g[0];
#pragma unroll
  for (int k = 1; k < kMaxWin; ++k) v = w == k ? g[k] : v;
  return v;
}

template <int MODE>
constexpr int kb_per_chunk() {
  return TcTraits<MODE>::kBK == 64 ? 1 : 2;
}

template <int MODE, int BN, int STAGES, class Sched>
__global__ void __launch_bounds__(kThreads, 1)
    mo_tc_pair_kernel(const __grid_constant__ Sched sc, int* err_flag) {
  using S = PairShape<MODE, BN, STAGES>;
  using TR = TcTraits<MODE>;
  constexpr uint32_t ACC = S::ACC;
  constexpr uint32_t NBUF = S::NBUF;
  constexpr int kPer = kb_per_chunk<MODE>();

  extern __shared__ unsigned char smem_raw[];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ uint32_t stage_info[STAGES];
  __shared__ uint16_t elist[2][64];  // producers' stage lists (one 32-chunk window each)
  __shared__ __align__(16) float epi[4][32][32];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t bar0 = base + STAGES * S::STAGE_BYTES;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + NBUF + b); };

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int64_t cluster = blockIdx.x >> 1;
  const int64_t nclusters = gridDim.x >> 1;
  volatile int* abort_v = &abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < (int)NBUF; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), 8);  // four epilogue warps in each CTA
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(S::TMEM_ALLOC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers initialised before either signals the other
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  griddep_wait();

  const int64_t total = sc.count();
  // chunks of a tile's K range (the last may be half one) and the 32-chunk
  // windows of its mask row
  auto chunks_of = [&](const PairTile& x) { return (x.num_kb + kPer - 1) / kPer; };

  if (warp == 4 || warp == 6) {
    // ------------------------------------------------ TMA producers (both CTAs)
    // Warp 4 copies the AO blocks (and, in the leader, posts the stage word
    // and the stage's byte count), warp 6 the C blocks: the copies one thread
    // issues complete one after another, so the two operands of a stage come
    // from two warps.  All four producers of a pair walk the same stage
    // sequence: the union of the pair's live K blocks.  The two mask rows of
    // a pair-tile are read one pair-tile ahead, a byte per lane and 32-chunk
    // window, and kept in registers: per chunk the union groups (bits 0-3)
    // and this CTA's own groups (bits 4-7).
    const bool a_warp = warp == 4;
    if (lane == 0) sc.prefetch_map(a_warp);
    auto load_groups = [&](const PairTile& x, uint32_t (&g)[kMaxWin]) {
      const int nq = chunks_of(x), nwin = (nq + 31) / 32;
      const int mld = mask_ld(x.nchunk);
      const int mo = 2 * x.mp + (int)rank, mr = 2 * x.mp + 1 - (int)rank;
      const uint8_t* own_row = mo < x.m_tiles ? x.mask + (int64_t)mo * mld : nullptr;
      const uint8_t* par_row = mr < x.m_tiles ? x.mask + (int64_t)mr * mld : nullptr;
#pragma unroll
      for (int w = 0; w < kMaxWin; ++w) {
        const int q = 32 * w + lane;
        uint32_t o = 0u, r = 0u;
        if (w < nwin && q < nq) {
          if (own_row) o = (uint32_t)own_row[q] & 0xFu;
          if (par_row) r = (uint32_t)par_row[q] & 0xFu;
        }
        g[w] = (o | r) | (o << 4);
      }
    };
    // The stages of one 32-chunk window as a list in shared memory (built by
    // the whole warp), walked by lane 0 alone: the per-stage work of a
    // producer is then a wait, a word and a copy, with no warp-wide step.
    // Entry: K block (bits 0-9), its live k-steps (bits 10-13), the block
    // live in this CTA's own tile (bit 14); never 0.
    uint16_t* list = elist[a_warp ? 0 : 1];
    uint32_t gnext[kMaxWin];
    PairTile xnext{};
    if (cluster < total) {
      xnext = sc.tile(cluster);
      load_groups(xnext, gnext);
    }
    uint32_t it = 0;  // stages taken (lane 0)
    bool ok = true;
    for (int64_t p = cluster; p < total && ok; p += nclusters) {
      uint32_t gcur[kMaxWin];
#pragma unroll
      for (int w = 0; w < kMaxWin; ++w) gcur[w] = gnext[w];
      const PairTile x = xnext;
      if (p + nclusters < total) {
        xnext = sc.tile(p + nclusters);
        load_groups(xnext, gnext);
      }
      const int nwin = (chunks_of(x) + 31) / 32;
      const int nt = x.nt;
      const int mt_own = 2 * x.mp + (int)rank;
      const int bn = x.bn;
      // the pair-tile's last live K block (-1: none)
      int lastkb = -1;
#pragma unroll
      for (int w = 0; w < kMaxWin; ++w) {
        const unsigned live = __ballot_sync(0xffffffffu, (gcur[w] & 0xFu) != 0u);
        if (live) {
          const int j = 31 - __clz(live);
          const uint32_t gj = __shfl_sync(0xffffffffu, gcur[w], j);
          lastkb = (32 * w + j) * kPer + ((kPer == 2 && (gj & 0xCu)) ? 1 : 0);
        }
      }
      if (lastkb >= x.num_kb) lastkb = x.num_kb - 1;
      // a C block is always BN / 2 rows (the last N tile's are zero-padded)
      const uint32_t cta_bytes = S::STAGE_BYTES;
      const uint32_t bn_bits = (uint32_t)(bn >> 4) << kStageBnShift;
      uint32_t flags = kStageFirst;
      // one stage (lane 0): wait for the slot, post the stage word (leader's
      // AO producer), issue this CTA's copy of the operand
      auto stage = [&](int kb, uint32_t steps, bool own_live) -> bool {
        const int s = it % STAGES;
        const uint32_t ph = (it / STAGES) & 1u;
        ++it;
        if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_v)) {
          flag_error(err_flag, abort_v, 1);
          return false;
        }
        if (a_warp && leader) {
          stage_info[s] = steps | flags | bn_bits | (kb == lastkb ? kStageLast : 0u);
          mbar_expect_tx(full_bar(s), kb >= 0 ? 2u * cta_bytes : 0u);
        }
        flags = 0;
        if (kb >= 0) {
          const uint32_t bar = map_to_rank(full_bar(s), 0);  // the leader's full[s]
          const uint32_t dst = base + s * S::STAGE_BYTES + (a_warp ? 0u : TR::kPlanes * S::A_BYTES);
          // own AO block (one contiguous box), or zeros from past the
          // tensor's end when the block is dead in this CTA's tile; own half
          // of the C block
          if (a_warp) {
            const int z = own_live ? blocked_slice<MODE>(mt_own, kb, x.nchunk) : x.zero_slice;
            tma_load_3d_pair(dst, x.a, bar, 0, 0, z);
          } else {
            const int z = ((2 * nt + (int)rank) * x.num_kb + kb) * TR::kPlanes;
            tma_load_3d_pair(dst, x.b, bar, 0, 0, z);
          }
        }
        return true;
      };
      if (lastkb < 0) {
        if (lane == 0) ok = stage(-1, 0u, false);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        continue;
      }
#pragma unroll 1
      for (int w = 0; w < nwin && ok; ++w) {
        const uint32_t g = pick_window(gcur, w);
        const int q = 32 * w + lane;
        const uint32_t own = (g >> 4) != 0u ? 1u << 14 : 0u;
        uint32_t e[2] = {0u, 0u};
#pragma unroll
        for (int h = 0; h < kPer; ++h) {
          uint32_t steps = g & 0xFu;
          if constexpr (kPer == 2) {
            const uint32_t hh = (g >> (2 * h)) & 3u;
            steps = (hh & 1u ? 0x3u : 0u) | (hh & 2u ? 0xCu : 0u);
          }
          const int kb = q * kPer + h;
          if (steps && kb < x.num_kb) e[h] = (uint32_t)kb | (steps << 10) | own;
        }
        const unsigned b0 = __ballot_sync(0xffffffffu, e[0] != 0u);
        const unsigned b1 = __ballot_sync(0xffffffffu, e[1] != 0u);
        const unsigned lt = (1u << lane) - 1u;
        const int pos = __popc(b0 & lt) + __popc(b1 & lt);
        if (e[0]) list[pos] = (uint16_t)e[0];
        if (e[1]) list[pos + (e[0] ? 1 : 0)] = (uint16_t)e[1];
        const int n_e = __popc(b0) + __popc(b1);
        __syncwarp();
        if (lane == 0) {
          if constexpr (kPer == 1) {
            // the window's first own AO block into L2 as soon as the list is known
            if (a_warp && n_e > 0 && (list[0] & (1u << 14)))
              tma_prefetch_l2_3d(x.a, 0, 0,
                                 blocked_slice<MODE>(mt_own, (int)(list[0] & 0x3FFu), x.nchunk));
          }
          for (int k = 0; k < n_e && ok; ++k) {
            const uint32_t v = list[k];
            if constexpr (kPer == 1) {
              // the next entry's own AO block into L2 now, so that its copy
              // into the ring (a stage later) does not wait on HBM
              if (a_warp && k + 1 < n_e) {
                const uint32_t vn = list[k + 1];
                if (vn & (1u << 14))
                  tma_prefetch_l2_3d(x.a, 0, 0,
                                     blocked_slice<MODE>(mt_own, (int)(vn & 0x3FFu), x.nchunk));
              }
            }
            ok = stage((int)(v & 0x3FFu), (v >> 10) & 0xFu, (v >> 14) & 1u);
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);  // also: the list may be rewritten
      }
    }
    if (a_warp && leader && lane == 0 && *abort_v) {
      // drain: the copies of both CTAs complete on the leader's barriers
      const uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0u;
      for (uint32_t k = first; k < it; ++k) {
        const long long t0 = clock64();
        while (!mbar_try_wait(full_bar(k % STAGES), (k / STAGES) & 1u) &&
               clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp == 5 && lane == 0 && leader) {
    // ------------------------------------------------ MMA issuer (leader)
    const int64_t my_tiles =
        total > cluster ? (total - 1 - cluster) / nclusters + 1 : 0;
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
        const int bn = (int)((info >> kStageBnShift) << 4);
        idesc = make_idesc(TR::kFmt, 2 * kBM, bn);
        first = true;
      }
      tc_fence_after();
      const uint64_t da = d0 + ((uint64_t)(s * S::STAGE_BYTES) >> 4);
      const uint64_t da_lo = da + (S::A_BYTES >> 4);
      const uint64_t db = da + ((TR::kPlanes * S::A_BYTES) >> 4);
      // the C block's lo plane follows BN / 2 rows of hi (padded on the last N tile)
      const uint64_t db_lo = db + (((uint32_t)(BN / 2) * kRowBytes) >> 4);
#pragma unroll
      for (int kk = 0; kk < kRowBytes / kUmmaKBytes; ++kk) {
        if (!((info >> kk) & 1u)) continue;
        const uint64_t ko = (uint64_t)(kk * kUmmaKBytes) >> 4;
        const uint32_t acc = first ? 0u : 1u;
        first = false;
        umma_pair<MODE>(dacc, da + ko, db + ko, idesc, acc);
        if constexpr (MODE == QK_BF16X3) {
          umma_pair<MODE>(dacc, da + ko, db_lo + ko, idesc, 1u);
          umma_pair<MODE>(dacc, da_lo + ko, db + ko, idesc, 1u);
        }
      }
      umma_commit_pair(empty_bar(s));
      if (info & kStageLast) {
        umma_commit_pair(tfull_bar(b));
        in_tile = false;
        ++i;
      }
    }
    if (!ok) {
      uint32_t wb = 0, wi = 0;
      bool wait = false;
      if (in_tile) {
        umma_commit_pair(tfull_bar(b));
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
    // ------------------------------------------------ epilogue (both CTAs)
    // Warp w drains TMEM lanes 32 w .. 32 w + 31 (its rows of this CTA's
    // tile), 32 columns per round trip: each lane's row goes into a staging
    // tile [32 rows][32 floats] (16-byte chunk q of row r at q ^ (r % 8), free
    // of bank conflicts both ways), then each store instruction writes 4 rows
    // x 128 contiguous bytes.  The output rows (through the point
    // permutation) and the tile's live flag are read one pair-tile ahead.
    // The leader's accumulator-free barrier gets this warp's arrival as soon
    // as its last TMEM load of the tile has completed.
    auto load_setup = [&](const PairTile& x, int64_t (&orow)[8], uint32_t& livebits) {
      const int mt = 2 * x.mp + (int)rank;
      const int64_t row0 = (int64_t)mt * (5 * kTilePoints);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int loc = warp * 32 + 4 * k + (lane >> 3);
        const int64_t lin = row0 + loc;
        orow[k] = (mt < x.m_tiles && loc < 5 * kTilePoints && lin < x.M)
                      ? (x.perm ? 5 * (int64_t)x.perm[lin / 5] + lin % 5 : lin)
                      : -1;
      }
      livebits = 0u;
      if (mt < x.m_tiles) {
        const uint8_t* row = x.mask + (int64_t)mt * mask_ld(x.nchunk);
        const int nq = chunks_of(x);
        for (int q = lane; q < nq; q += 32) livebits |= (uint32_t)row[q] & 0xFu;
      }
    };
    int64_t onext[8];
    uint32_t lnext = 0u;
    PairTile xnext{};
    if (cluster < total) {
      xnext = sc.tile(cluster);
      load_setup(xnext, onext, lnext);
    }
    float(*stg)[32] = epi[warp];
    uint32_t i = 0;
    for (int64_t p = cluster; p < total; p += nclusters, ++i) {
      int64_t orow[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) orow[k] = onext[k];
      const uint32_t lcur = lnext;
      const PairTile x = xnext;
      if (p + nclusters < total) {
        xnext = sc.tile(p + nclusters);
        load_setup(xnext, onext, lnext);
      }
      const int64_t N = x.N;
      const bool vec = (N % 4) == 0 && (reinterpret_cast<uintptr_t>(x.D) & 15) == 0;
      const uint32_t b = i % NBUF;
      const long long t0 = clock64();
      bool ok = true;
      while (!mbar_try_wait(tfull_bar(b), (i / NBUF) & 1u)) {
        if (*abort_v || clock64() - t0 > kWaitCycles) {
          ok = false;
          break;
        }
      }
      if (!ok) flag_error(err_flag, abort_v, 3);
      ok = __all_sync(0xffffffffu, ok) && !*abort_v;
      __syncwarp();
      if (!ok) break;
      tc_fence_after();
      const int bn = x.bn;
      const int n0 = x.n0;
      const bool any_live = __any_sync(0xffffffffu, lcur != 0u);
      const uint32_t tbase = tmem + b * ACC + ((uint32_t)(warp * 32) << 16);
      const int cq = lane & 7;
      float* rowp[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) rowp[k] = x.D + (orow[k] >= 0 ? orow[k] : 0) * N;
#pragma unroll 1
      for (int c = 0; c < bn; c += 32) {
        const bool two = c + 16 < bn;
        float v[32];
        if (any_live) {
          tmem_ld16x2(tbase + c, v, two);
        } else {  // every AO of this tile was screened: the MOs are exactly zero
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = 0.0f;
        }
        if (c + 32 >= bn) {
          // the tile's TMEM reads are complete: the buffer may be refilled
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster_relaxed(map_to_rank(tempty_bar(b), 0));
        }
        float4* srow = reinterpret_cast<float4*>(&stg[lane][0]);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          srow[q ^ (lane & 7)] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        __syncwarp();
        const int64_t col = n0 + c + 4 * cq;
        const bool in_tile = cq < (two ? 8 : 4);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int r = 4 * k + (lane >> 3);
          if (orow[k] >= 0 && in_tile) {
            const float4 w = reinterpret_cast<const float4*>(&stg[r][0])[cq ^ (r & 7)];
            float* dst = rowp[k] + col;
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
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // no role of either CTA touches the other's barriers or TMEM after this
  if (warp == 5) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(S::TMEM_ALLOC)
                 : "memory");
  }
}

// The blocked C as a 3-D map: slices of `hb` rows x 128 bytes, box = the
// planes of one block.
template <int MODE>
bool make_map_pair_c(CUtensorMap* m, const void* c_blk, int hb, int64_t nslices) {
  using TR = TcTraits<MODE>;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t w = 128 / (TR::kPlanes == 2 ? 2 : 4);
  cuuint64_t dims[3] = {w, (cuuint64_t)hb, (cuuint64_t)nslices};
  cuuint64_t strides[2] = {128, (cuuint64_t)hb * 128};
  cuuint32_t box[3] = {(cuuint32_t)w, (cuuint32_t)hb, (cuuint32_t)TR::kPlanes};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, TR::kPlanes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
             3, const_cast<void*>(c_blk), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One persistent launch: one CTA per SM (TMEM is taken whole), in pairs.
template <int MODE, int BN, class Sched>
cudaError_t launch_pair_kernel(const Sched& sc, int64_t total, int* err_flag, cudaStream_t s) {
  constexpr int ST = stages_for_pair(MODE, BN);
  using S = PairShape<MODE, BN, ST>;
  if (total == 0) return cudaSuccess;
  auto kern = mo_tc_pair_kernel<MODE, BN, ST, Sched>;
  KernelFacts f;
  cudaError_t e = kernel_facts<mo_tc_pair_kernel<MODE, BN, ST, Sched>>(S::SMEM, kThreads, &f);
  if (e != cudaSuccess) return e;
  if (f.occ < 1) return cudaErrorInvalidConfiguration;
  int64_t clusters = f.sms / 2;
  if (clusters > total) clusters = total;
  if (clusters < 1) clusters = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * clusters));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = S::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kern, sc, err_flag);
}

// Checks and the shared fields of one problem (single or batch).
template <int MODE>
bool pair_problem_fields(const AOTensor& ao, int64_t K, int64_t N, int bn, int bn_max,
                         const void* c_blk, CUtensorMap* a, CUtensorMap* b, int* last_bn,
                         int* zero_slice, int* m_tiles, int* n_tiles, int* num_kb) {
  using TR = TcTraits<MODE>;
  const int64_t M = ao.rows;
  if (M > INT32_MAX / 2 || K > INT32_MAX || N > INT32_MAX) return false;
  if (!ao.tiled || !ao.blocked || M % kBM != 0 || ao.comps == 1) return false;
  if (K > (int64_t)ao.nchunk * kChunkAO || K % kChunkAO != 0) return false;
  if (bn % 16 != 0 || bn < 32 || bn > bn_max) return false;
  const int64_t nt = (N + bn - 1) / bn;
  const int64_t nblocks = M / kBM * ao.nchunk;
  const int64_t kbs = K / TR::kBK;
  if (2 * nblocks + 2 > INT32_MAX || 2 * nt * kbs * TR::kPlanes > INT32_MAX) return false;
  if (!make_map_blocked(a, ao.a, TR::kPlanes == 2, nblocks)) return false;
  if (!make_map_pair_c<MODE>(b, c_blk, bn_max / 2, 2 * nt * kbs * TR::kPlanes)) return false;
  // the last N tile multiplies only the MOs it has, rounded up to 16 (halves
  // of whole 8-row groups)
  *last_bn = (int)((N - (nt - 1) * bn + 15) / 16 * 16);
  *zero_slice = (int)(2 * nblocks);
  *m_tiles = (int)(M / kBM);
  *n_tiles = (int)nt;
  *num_kb = (int)kbs;
  return true;
}

template <int MODE, int BN>
cudaError_t launch_pair_bn(const AOTensor& ao, int64_t K, const void* c_blk, int64_t N, float* out,
                           int64_t out_rows, int* err_flag, cudaStream_t s) {
  if (ao.rows == 0 || N == 0) return cudaSuccess;
  PairSched<BN> sc;
  if (!pair_problem_fields<MODE>(ao, K, N, BN, BN, c_blk, &sc.a, &sc.b, &sc.last_bn,
                                 &sc.zero_slice, &sc.m_tiles, &sc.n_tiles, &sc.num_kb))
    return cudaErrorInvalidValue;
  sc.D = out;
  sc.mask = ao.mask;
  sc.perm = ao.perm;
  sc.M = out_rows;
  sc.N = N;
  sc.nchunk = ao.nchunk;
  sc.total = (int64_t)((sc.m_tiles + 1) / 2) * sc.n_tiles;
  return launch_pair_kernel<MODE, BN>(sc, sc.total, err_flag, s);
}

template <int MODE, int BN>
cudaError_t launch_pair_batch_bn(const PairProblem* probs, const int4* items, int64_t n_items,
                                 int* err_flag, cudaStream_t s) {
  PairBatchSched sc{probs, items, n_items};
  return launch_pair_kernel<MODE, BN>(sc, n_items, err_flag, s);
}

// Blocked C of one (half, K block): [planes][hb][w] with w = 128 bytes of
// elements; half h = 2 nt + r holds rows nt bn + r bn_t / 2 .. + bn_t / 2 of
// C (bn_t the tile's MMA N, bn_t / 2 <= hb), zeros past them and past the
// last MO.
template <typename E>
__global__ void pair_c_kernel(const E* c_hi, const E* c_lo, int64_t ldc, int64_t N, int bn,
                              int last_bn, int hb, int64_t n_tiles, int64_t num_kb, int planes,
                              E* out) {
  constexpr int w = 128 / (int)sizeof(E);
  const int64_t total = 2 * n_tiles * num_kb * planes * hb * w;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % w);
    int64_t t = i / w;
    const int r = (int)(t % hb);
    t /= hb;
    const int p = (int)(t % planes);
    t /= planes;
    const int64_t kb = t % num_kb;
    const int64_t h = t / num_kb;
    const int64_t nt = h / 2;
    const int bnt = nt == n_tiles - 1 ? last_bn : bn;
    const int64_t row = nt * bn + (h & 1) * (bnt / 2) + r;
    E v = E(0.0f);
    if (r < bnt / 2 && row < N) v = (p ? c_lo : c_hi)[row * ldc + kb * w + c];
    out[i] = v;
  }
}

int pair_last_bn(int64_t N, int bn) {
  const int64_t n_tiles = (N + bn - 1) / bn;
  return (int)((N - (n_tiles - 1) * bn + 15) / 16 * 16);
}

}  // namespace

size_t pair_c_bytes(int mode, int64_t mo_num, int64_t ao_num, int bn, int half_rows) {
  const int64_t n_tiles = (mo_num + bn - 1) / bn;
  const int64_t kb = mode == QK_TF32 ? ao_num / 32 : ao_num / 64;
  const int planes = mode == QK_BF16X3 ? 2 : 1;
  return (size_t)(2 * n_tiles * kb * planes) * (size_t)half_rows * 128;
}

cudaError_t launch_pair_c(int mode, const void* c_hi, const void* c_lo, int64_t ldc,
                          int64_t mo_num, int64_t ao_num, int bn, int half_rows, void* c_blk,
                          cudaStream_t s) {
  if (bn % 16 != 0 || bn < 32 || bn > 256 || ao_num % kChunkAO != 0 || 2 * half_rows < bn ||
      half_rows % 8 != 0)
    return cudaErrorInvalidValue;
  const int64_t n_tiles = (mo_num + bn - 1) / bn;
  const int last_bn = pair_last_bn(mo_num, bn);
  const int64_t elems =
      (int64_t)pair_c_bytes(mode, mo_num, ao_num, bn, half_rows) / (mode == QK_TF32 ? 4 : 2);
  const unsigned grid = (unsigned)std::min<int64_t>((elems + 255) / 256, 4096);
  if (elems == 0) return cudaSuccess;
  if (mode == QK_BF16X3) {
    pair_c_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(
        (const __nv_bfloat16*)c_hi, (const __nv_bfloat16*)c_lo, ldc, mo_num, bn, last_bn,
        half_rows, n_tiles, ao_num / 64, 2, (__nv_bfloat16*)c_blk);
  } else if (mode == QK_TF32) {
    pair_c_kernel<float><<<grid, 256, 0, s>>>((const float*)c_hi, nullptr, ldc, mo_num, bn,
                                              last_bn, half_rows, n_tiles, ao_num / 32, 1,
                                              (float*)c_blk);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

bool tc_make_pair_problem(int mode, const AOTensor& ao, int64_t K, const void* c_blk, int64_t N,
                          float* out, int bn, int bn_max, int64_t out_rows, PairProblem* p) {
  bool ok;
  if (mode == QK_BF16X3)
    ok = pair_problem_fields<QK_BF16X3>(ao, K, N, bn, bn_max, c_blk, &p->a, &p->b, &p->last_bn,
                                        &p->zero_slice, &p->m_tiles, &p->n_tiles, &p->num_kb);
  else if (mode == QK_TF32)
    ok = pair_problem_fields<QK_TF32>(ao, K, N, bn, bn_max, c_blk, &p->a, &p->b, &p->last_bn,
                                      &p->zero_slice, &p->m_tiles, &p->n_tiles, &p->num_kb);
  else
    ok = false;
  if (!ok) return false;
  p->mask = ao.mask;
  p->perm = ao.perm;
  p->D = out;
  p->M = out_rows;
  p->N = N;
  p->nchunk = ao.nchunk;
  p->bn = bn;
  return true;
}

cudaError_t launch_mo_tc_pair_batch(int mode, int bn_max, const PairProblem* probs,
                                    const int4* items, int64_t n_items, int* err_flag,
                                    cudaStream_t s) {
#define QK_PAIR_BATCH_CASE(M_, B_) \
  case B_:                         \
    return launch_pair_batch_bn<M_, B_>(probs, items, n_items, err_flag, s);
  if (mode == QK_BF16X3) {
    switch (bn_max) {
      QK_PAIR_BATCH_CASE(QK_BF16X3, 64)
      QK_PAIR_BATCH_CASE(QK_BF16X3, 96)
      QK_PAIR_BATCH_CASE(QK_BF16X3, 128)
      QK_PAIR_BATCH_CASE(QK_BF16X3, 160)
      QK_PAIR_BATCH_CASE(QK_BF16X3, 192)
      QK_PAIR_BATCH_CASE(QK_BF16X3, 256)
      default: return cudaErrorInvalidValue;
    }
  }
  if (mode == QK_TF32) {
    switch (bn_max) {
      QK_PAIR_BATCH_CASE(QK_TF32, 64)
      QK_PAIR_BATCH_CASE(QK_TF32, 96)
      QK_PAIR_BATCH_CASE(QK_TF32, 128)
      QK_PAIR_BATCH_CASE(QK_TF32, 160)
      QK_PAIR_BATCH_CASE(QK_TF32, 192)
      QK_PAIR_BATCH_CASE(QK_TF32, 256)
      default: return cudaErrorInvalidValue;
    }
  }
#undef QK_PAIR_BATCH_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_mo_tc_pair(int mode, const AOTensor& ao, int64_t ao_num, const void* c_blk,
                              int64_t mo_num, float* out, int bn, int* err_flag, cudaStream_t s,
                              int64_t out_rows) {
#define QK_PAIR_CASE(M_, B_)                                                                   \
  case B_:                                                                                     \
    return launch_pair_bn<M_, B_>(ao, ao_num, c_blk, mo_num, out, out_rows, err_flag, s);
  if (mode == QK_BF16X3) {
    switch (bn) {
      QK_PAIR_CASE(QK_BF16X3, 64)
      QK_PAIR_CASE(QK_BF16X3, 96)
      QK_PAIR_CASE(QK_BF16X3, 128)
      QK_PAIR_CASE(QK_BF16X3, 160)
      QK_PAIR_CASE(QK_BF16X3, 192)
      QK_PAIR_CASE(QK_BF16X3, 256)
      default: return cudaErrorInvalidValue;
    }
  }
  if (mode == QK_TF32) {
    switch (bn) {
      QK_PAIR_CASE(QK_TF32, 64)
      QK_PAIR_CASE(QK_TF32, 96)
      QK_PAIR_CASE(QK_TF32, 128)
      QK_PAIR_CASE(QK_TF32, 160)
      QK_PAIR_CASE(QK_TF32, 192)
      QK_PAIR_CASE(QK_TF32, 256)
      default: return cudaErrorInvalidValue;
    }
  }
#undef QK_PAIR_CASE
  return cudaErrorInvalidValue;
}

}  // namespace qk
