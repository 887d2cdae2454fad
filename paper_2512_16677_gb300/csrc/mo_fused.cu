// mo_fused.cu -- AO evaluation fused into the tcgen05 MO contraction.
//
// The split-bf16 MO vgl (Eqs. 5-7) without an AO tensor in HBM.  Points go
// in tiles of 25 (125 (point, component) rows of a 128-row MMA tile) and AOs
// in chunks of <= 64 (one 64-column K block).
//
//  1. fused_live_kernel: for every tile, the chunks with at least one shell
//     whose radius (r^2 < T / gamma_min, Eq. 3) reaches one of the tile's
//     points, as an ascending list; only those K blocks are multiplied (the
//     sparse-AO MO product of Sec. 3.2 at tile granularity).
//  2. mo_fused_kernel, persistent over (tile, N tile) items, 13 warps:
//       warps 5-12  AO producers: for each live chunk, the shell-major AO
//                   evaluation of ao_vgl (one warp per shell, one lane per
//                   point: radial sums of Eq. 2 with the Eq. 3 screen, then
//                   every Cartesian component of Eqs. 1 and 4) into an FP32
//                   staging tile, then split into bf16 hi + lo and written
//                   into the MMA's shared memory stage in the 128-byte
//                   swizzled K-major layout; the group leader also loads the
//                   matching C chunk by TMA
//       warp 4      one thread issues hi*hi + hi*lo + lo*hi MMAs into a
//                   double-buffered TMEM accumulator
//       warps 0-3   epilogue: TMEM -> registers -> shared memory (32 x 16
//                   slices turned around) -> whole row segments of the output
// The producer group synchronises on named barrier 1.  Every wait is bounded
// and a wait that gives up records a code in the caller's error word.
#include "ao_common.cuh"
#include "tc_common.cuh"

namespace qk {
namespace {

using namespace tc;

constexpr int kMmaWarp = 4;
constexpr int kProdWarp0 = 5;
constexpr int kProdWarps = 8;
constexpr int kProdThreads = 32 * kProdWarps;
constexpr int kFThreads = 32 * (kProdWarp0 + kProdWarps);  // 416
constexpr int kStages = 2;
constexpr uint32_t kABytes = kBM * kRowBytes;  // one bf16 plane of a 128 x 64 block
// staging rows of lanes 0..25; lane 25 is past the tile, so rows 125..127
// read back as zeros
using FusedStage = AOStageSmem<float, kTilePoints + 1>;
// MMA N of the fused kernel: the AO staging tile leaves room for two stages
// of B up to 192 columns
constexpr int kFusedBnMax = 192;
// epilogue staging, as in the two-kernel contraction: per warp a 32 x 16
// accumulator slice, 16-byte chunk q of row r at chunk q ^ ((r / 2) % 4)
constexpr int kEpiPitch = 16;

__device__ __forceinline__ void prod_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kProdThreads) : "memory");
}

struct FusedParams {
  BasisDev b;
  PointsDev p;
  CUtensorMap c_hi, c_lo;     // C planes [N][nchunk * 64], box {64, BN}
  float* D;                   // [5P][N]
  const int* live_count;      // [tiles]
  const uint16_t* live_list;  // [tiles][nchunk]
  int64_t P, N, total;
  int n_tiles, nchunk;
};

template <int BN>
struct FusedShape {
  static constexpr uint32_t B_BYTES = BN * kRowBytes;
  static constexpr uint32_t STAGE_BYTES = 2 * (kABytes + B_BYTES);
  static constexpr uint32_t RING = kStages * STAGE_BYTES;
  static constexpr uint32_t TMEM_COLS = tmem_cols<BN>();  // per accumulator buffer (two)
  static constexpr size_t SMEM = 1024 + RING + sizeof(FusedStage);
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "MMA N: 16..256, step 16");
};

template <int BN>
__global__ void __launch_bounds__(kFThreads, 1)
    mo_fused_kernel(const __grid_constant__ FusedParams prm, int* err_flag) {
  using Sh = FusedShape<BN>;
  constexpr uint32_t idesc = make_idesc(TcTraits<QK_BF16X3>::kFmt, kBM, BN);
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[2 * kStages + 4];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int stage_last[kStages];
  __shared__ int prod_ok;
  __shared__ __align__(16) float epi[4][32][kEpiPitch];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // swizzle atoms need 1024-byte alignment
  unsigned char* gbase = smem_raw + (base - raw);
  FusedStage& sh = *reinterpret_cast<FusedStage*>(gbase + Sh::RING);
  auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
  auto empty_bar = [&](int s) { return smem_u32(&bars[kStages + s]); };
  auto tfull_bar = [&](int b) { return smem_u32(&bars[2 * kStages + b]); };
  auto tempty_bar = [&](int b) { return smem_u32(&bars[2 * kStages + 2 + b]); };

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  volatile int* abort_v = &abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full_bar(s), kProdWarps + 1);  // 8 producer warps + the TMA expect_tx
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), 4);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(2 * Sh::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp >= kProdWarp0) {
    // ------------------------------------------------ AO producers
    const int pw = warp - kProdWarp0;
    const int ptid = threadIdx.x - 32 * kProdWarp0;
    const float Tthr = prm.b.T_f;
    const int64_t n = prm.P;
    uint32_t it = 0;
    bool alive = true;
    for (int64_t t = blockIdx.x; t < prm.total && alive; t += gridDim.x) {
      const int64_t mt = t / prm.n_tiles;
      const int n0 = (int)(t % prm.n_tiles) * BN;
      const int64_t p0 = mt * kTilePoints;
      int cnt = prm.live_count[mt];
      const uint16_t* lst = prm.live_list + mt * prm.nchunk;
      const bool forced = cnt == 0;  // nothing live: one all-zero block keeps the flow uniform
      if (forced) cnt = 1;
      prod_sync();  // the previous tile's readers of the points are done
      if (ptid < kTilePoints) {
        const int64_t ip = p0 + ptid;
        if (ip < n) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            sh.pt[ptid][k] = prm.p.hi[k * prm.p.ld + ip];
            sh.pt_lo[ptid][k] = prm.p.lo[k * prm.p.ld + ip];
          }
        }
      }
      const bool valid = lane < kTilePoints && p0 + lane < n;
      for (int i = 0; i < cnt; ++i) {
        const int q = forced ? 0 : (int)lst[i];
        prod_sync();  // previous block's conversion done with the tables and staging tile
        load_stage_tables(prm.b, q, sh, ptid, kProdThreads);
        if (ptid == 0) sh.next = 0;
        prod_sync();
        const int4 ch = prm.b.chunk[q];
        const int ns = ch.y - ch.x;
        for (;;) {
          int k = 0;
          if (lane == 0) k = atomicAdd(&sh.next, 1);
          k = __shfl_sync(0xffffffffu, k, 0);
          if (k >= ns) break;
          shell_at_point(sh, sh.order[k], lane, valid, Tthr);
        }
        const int s = it % kStages;
        const uint32_t ph = (it / kStages) & 1u;
        ++it;
        if (ptid == 0) {
          const bool ok = mbar_wait(empty_bar(s), ph ^ 1u, abort_v);
          if (!ok) flag_error(err_flag, abort_v, 4);
          prod_ok = ok ? 1 : 0;
          if (ok) {
            stage_last[s] = (i == cnt - 1) ? 1 : 0;
            const uint32_t bst = base + s * Sh::STAGE_BYTES + 2 * kABytes;
            mbar_expect_tx(full_bar(s), 2 * Sh::B_BYTES);
            tma_load_2d(bst, &prm.c_hi, full_bar(s), q * kChunkAO, n0);
            tma_load_2d(bst + Sh::B_BYTES, &prm.c_lo, full_bar(s), q * kChunkAO, n0);
          }
        }
        prod_sync();  // staging tile complete, stage granted
        if (!prod_ok) {
          alive = false;
          break;
        }
        // rows r of both planes in the SWIZZLE_128B layout (16-byte chunk j
        // of row r at chunk j ^ (r & 7)); lane = AO pair (2 lane, 2 lane + 1)
        unsigned char* a_hi = gbase + s * Sh::STAGE_BYTES;
        unsigned char* a_lo = a_hi + kABytes;
        for (int r = pw; r < kTileRows; r += kProdWarps) {
          const float v0 = sh.stage[r][2 * lane], v1 = sh.stage[r][2 * lane + 1];
          const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
          const float2 hf = __bfloat1622float2(h);
          const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
          const uint32_t off = r * kRowBytes + ((((uint32_t)lane >> 2) ^ (r & 7)) << 4) +
                               (((uint32_t)lane & 3) << 2);
          *reinterpret_cast<__nv_bfloat162*>(a_hi + off) = h;
          *reinterpret_cast<__nv_bfloat162*>(a_lo + off) = l;
        }
        // generic-proxy writes must be visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(full_bar(s));
      }
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t it = 0, i = 0;
      for (int64_t t = blockIdx.x; t < prm.total; t += gridDim.x, ++i) {
        const uint32_t b = i & 1u;
        if (!mbar_wait(tempty_bar(b), ((i >> 1) & 1u) ^ 1u, abort_v)) {
          flag_error(err_flag, abort_v, 5);
          break;
        }
        tc_fence_after();
        const uint32_t dacc = tmem + b * Sh::TMEM_COLS;
        bool ok = true, first = true;
        for (;;) {
          const int s = it % kStages;
          const uint32_t ph = (it / kStages) & 1u;
          ++it;
          if (!mbar_wait(full_bar(s), ph, abort_v)) {
            flag_error(err_flag, abort_v, 5);
            ok = false;
            break;
          }
          tc_fence_after();
          const int last = stage_last[s];
          const uint32_t a_hi = base + s * Sh::STAGE_BYTES;
          const uint32_t a_lo = a_hi + kABytes;
          const uint32_t b_hi = a_hi + 2 * kABytes;
          const uint32_t b_lo = b_hi + Sh::B_BYTES;
#pragma unroll
          for (int kk = 0; kk < kRowBytes / kUmmaKBytes; ++kk) {
            const uint32_t koff = kk * kUmmaKBytes;
            const uint32_t acc = (!first || kk != 0) ? 1u : 0u;
            umma<QK_BF16X3>(dacc, sw128_desc(a_hi + koff), sw128_desc(b_hi + koff), idesc, acc);
            umma<QK_BF16X3>(dacc, sw128_desc(a_hi + koff), sw128_desc(b_lo + koff), idesc, 1u);
            umma<QK_BF16X3>(dacc, sw128_desc(a_lo + koff), sw128_desc(b_hi + koff), idesc, 1u);
          }
          umma_commit(empty_bar(s));
          first = false;
          if (last) break;
        }
        umma_commit(tfull_bar(b));
        if (!ok) {
          const long long t0 = clock64();
          while (!mbar_try_wait(tfull_bar(b), (i >> 1) & 1u) && clock64() - t0 < kWaitCycles) {
          }
          break;
        }
      }
    }
  } else {
    // ------------------------------------------------ epilogue (warps 0-3)
    uint32_t i = 0;
    for (int64_t t = blockIdx.x; t < prm.total; t += gridDim.x, ++i) {
      const uint32_t b = i & 1u;
      const long long t0 = clock64();
      bool ok = true;
      while (!mbar_try_wait(tfull_bar(b), (i >> 1) & 1u)) {
        if (clock64() - t0 > kWaitCycles) {
          ok = false;
          break;
        }
      }
      if (!ok) flag_error(err_flag, abort_v, 6);
      ok = __all_sync(0xffffffffu, ok) && !*abort_v;
      __syncwarp();
      if (!ok) break;
      tc_fence_after();
      const int64_t mt = t / prm.n_tiles;
      const int64_t n0 = (t % prm.n_tiles) * BN;
      const int64_t N = prm.N;
      const int64_t M = 5 * prm.P;
      const uint32_t tbase = tmem + b * Sh::TMEM_COLS + ((uint32_t)(warp * 32) << 16);
      // store phase: lane -> row 8 i + lane / 4 of the warp's 32, columns
      // 4 (lane % 4) .. + 3 of the slice
      const int rq = lane >> 2;
      const int cq = (lane & 3) * 4;
      const bool vec = (N % 4) == 0 && (reinterpret_cast<uintptr_t>(prm.D) & 15) == 0;
      float(*stg)[kEpiPitch] = epi[warp];
#pragma unroll 1
      for (int c = 0; c < BN; c += 16) {
        float v[16];
        tmem_ld16(tbase + c, v);
        float4* srow = reinterpret_cast<float4*>(&stg[lane][0]);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          srow[q ^ ((lane >> 1) & 3)] =
              make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        __syncwarp();
        const int64_t col = n0 + c + cq;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = 8 * i + rq;
          const int loc = warp * 32 + r;
          const int64_t row = mt * (5 * kTilePoints) + loc;
          if (loc < 5 * kTilePoints && row < M) {
            const float4 w =
                reinterpret_cast<const float4*>(&stg[r][0])[(lane & 3) ^ ((r >> 1) & 3)];
            float* dst = prm.D + row * N + col;
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
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar(b));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * Sh::TMEM_COLS)
                 : "memory");
  }
}

// Live chunks of every 25-point tile, from distances only: chunk q is live
// when some shell of q has r^2 below its screening radius for some point
// (with a 1e-5 margin, so that a chunk the radial pass would find nonzero is
// never dropped; a chunk kept by the margin alone just adds zeros).
__global__ void __launch_bounds__(256)
    fused_live_kernel(BasisDev b, PointsDev p, int* live_count, uint16_t* live_list,
                      int64_t tiles) {
  extern __shared__ unsigned char live[];  // [nchunk]
  __shared__ float pt[kTilePoints][3], pt_lo[kTilePoints][3];
  const int tid = threadIdx.x;
  const int64_t n = p.n;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    __syncthreads();
    for (int q = tid; q < b.nchunk; q += blockDim.x) live[q] = 0;
    const int64_t p0 = t * kTilePoints;
    const int np = (int)(n - p0 < kTilePoints ? n - p0 : kTilePoints);
    if (tid < np) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        pt[tid][k] = p.hi[k * p.ld + p0 + tid];
        pt_lo[tid][k] = p.lo[k * p.ld + p0 + tid];
      }
    }
    __syncthreads();
    for (int idx = tid; idx < np * b.shell_num; idx += blockDim.x) {
      const int pl = idx % np;
      const int s = idx / np;
      const int A = b.shell_nuc[s];
      const float dx = (pt[pl][0] - b.nucl_hi[3 * A]) + (pt_lo[pl][0] - b.nucl_lo[3 * A]);
      const float dy = (pt[pl][1] - b.nucl_hi[3 * A + 1]) + (pt_lo[pl][1] - b.nucl_lo[3 * A + 1]);
      const float dz = (pt[pl][2] - b.nucl_hi[3 * A + 2]) + (pt_lo[pl][2] - b.nucl_lo[3 * A + 2]);
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < b.shell_r2_f[s] * (1.0f + 1e-5f)) live[b.shell_chunk[s]] = 1;
    }
    __syncthreads();
    if (tid < 32) {
      int cnt = 0;
      for (int q0 = 0; q0 < b.nchunk; q0 += 32) {
        const int q = q0 + tid;
        const bool f = q < b.nchunk && live[q];
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (f) live_list[t * b.nchunk + cnt + __popc(m & ((1u << tid) - 1u))] = (uint16_t)q;
        cnt += __popc(m);
      }
      if (tid == 0) live_count[t] = cnt;
    }
  }
}

template <int BN>
cudaError_t launch_fused_bn(const BasisDev& b, const PointsDev& p, const void* c_hi,
                            const void* c_lo, int64_t kpad, int64_t N, float* out,
                            const int* live_count, const uint16_t* live_list, int* err_flag,
                            cudaStream_t s) {
  using Sh = FusedShape<BN>;
  static_assert(Sh::SMEM + sizeof(float) * 4 * 32 * kEpiPitch + 1024 <= 232448,
                "shared memory budget");
  FusedParams prm;
  prm.b = b;
  prm.p = p;
  if (!make_map(&prm.c_hi, c_hi, false, kpad, N, kpad, kChunkAO, BN) ||
      !make_map(&prm.c_lo, c_lo, false, kpad, N, kpad, kChunkAO, BN))
    return cudaErrorInvalidValue;
  prm.D = out;
  prm.live_count = live_count;
  prm.live_list = live_list;
  prm.P = p.n;
  prm.N = N;
  prm.nchunk = b.nchunk;
  prm.n_tiles = (int)((N + BN - 1) / BN);
  const int64_t tiles = (p.n + kTilePoints - 1) / kTilePoints;
  prm.total = tiles * prm.n_tiles;
  auto kern = mo_fused_kernel<BN>;
  KernelFacts f;
  cudaError_t e = kernel_facts<mo_fused_kernel<BN>>(Sh::SMEM, kFThreads, &f);
  if (e != cudaSuccess) return e;
  const int occ = f.occ;
  if (occ < 1 || occ * 2 * (int)Sh::TMEM_COLS > 512) return cudaErrorInvalidConfiguration;
  const int64_t grid = prm.total < (int64_t)f.sms * occ ? prm.total : (int64_t)f.sms * occ;
  if (grid == 0) return cudaSuccess;
  kern<<<(unsigned)grid, kFThreads, Sh::SMEM, s>>>(prm, err_flag);
  return cudaGetLastError();
}

}  // namespace

size_t fused_workspace_bytes(int64_t point_num, int nchunk) {
  const int64_t tiles = (point_num + kTilePoints - 1) / kTilePoints;
  return (size_t)((tiles * 4 + 255) / 256 * 256) +
         (size_t)((tiles * nchunk * 2 + 255) / 256 * 256);
}

cudaError_t launch_fused_live(const BasisDev& b, const PointsDev& p, int* live_count,
                              uint16_t* live_list, cudaStream_t s) {
  const int64_t tiles = (p.n + kTilePoints - 1) / kTilePoints;
  if (tiles == 0) return cudaSuccess;
  const size_t smem = (size_t)b.nchunk;
  if (smem > 48 * 1024) return cudaErrorInvalidValue;
  const int64_t grid = tiles < 4096 ? tiles : 4096;
  fused_live_kernel<<<(unsigned)grid, 256, smem, s>>>(b, p, live_count, live_list, tiles);
  return cudaGetLastError();
}

cudaError_t launch_mo_fused(int bn, const BasisDev& b, const PointsDev& p, const void* c_hi,
                            const void* c_lo, int64_t kpad, int64_t N, float* out,
                            const int* live_count, const uint16_t* live_list, int* err_flag,
                            cudaStream_t s) {
  if (bn > kFusedBnMax) {
    // the fewest N tiles of at most kFusedBnMax columns, each as narrow as it can be
    static const int bns[] = {16, 32, 64, 96, 128, 160, 192};
    const int64_t tiles = (N + kFusedBnMax - 1) / kFusedBnMax;
    const int64_t per = (N + tiles - 1) / tiles;
    bn = kFusedBnMax;
    for (int c : bns)
      if (c >= per) {
        bn = c;
        break;
      }
  }
  switch (bn) {
    case 16: return launch_fused_bn<16>(b, p, c_hi, c_lo, kpad, N, out, live_count, live_list, err_flag, s);
    case 32: return launch_fused_bn<32>(b, p, c_hi, c_lo, kpad, N, out, live_count, live_list, err_flag, s);
    case 64: return launch_fused_bn<64>(b, p, c_hi, c_lo, kpad, N, out, live_count, live_list, err_flag, s);
    case 96: return launch_fused_bn<96>(b, p, c_hi, c_lo, kpad, N, out, live_count, live_list, err_flag, s);
    case 128: return launch_fused_bn<128>(b, p, c_hi, c_lo, kpad, N, out, live_count, live_list, err_flag, s);
    case 160: return launch_fused_bn<160>(b, p, c_hi, c_lo, kpad, N, out, live_count, live_list, err_flag, s);
    case 192: return launch_fused_bn<192>(b, p, c_hi, c_lo, kpad, N, out, live_count, live_list, err_flag, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qk
