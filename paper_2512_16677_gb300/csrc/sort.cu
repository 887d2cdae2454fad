// sort.cu -- spatial order of the points for the block-sparse tensor-core
// path.
//
// Tiles of 25 consecutive points decide which (tile, AO chunk) blocks the
// contraction multiplies (Sec. 3.2's sparse AO matrix at tile granularity).
// Points that are close in space share their nonzero AOs, so tiles cut from
// a spatial order carry fewer live blocks than tiles cut from the caller's
// order.  The order here: cells of a 32 x 32 x 32 grid over the nuclear
// bounding box (points outside are clamped to the border cells) visited in
// Morton (Z-curve) order, points of one cell by ascending index: a stable
// radix sort of the cell keys, so the permutation depends on the
// coordinates only.  The permutation changes which points share a tile, never a point's
// own values: each AO value and each output row is computed from that point
// alone.
#include "internal.h"

namespace qk {
namespace {

constexpr int kCellBits = 5;  // per axis

__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  // bit i of v -> bit 3 i
  uint32_t r = 0;
#pragma unroll
  for (int i = 0; i < kCellBits; ++i) r |= ((v >> i) & 1u) << (3 * i);
  return r;
}

__device__ __forceinline__ uint32_t cell_of(float x, float lo, float inv) {
  const float f = (x - lo) * inv;
  const int c = f <= 0.0f ? 0 : (f >= (float)((1 << kCellBits) - 1) ? (1 << kCellBits) - 1 : (int)f);
  return (uint32_t)c;
}

__global__ void cell_key_kernel(PointsDev p, float3 lo, float3 inv, uint32_t* key) {
  griddep_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t cx = cell_of(p.hi[i], lo.x, inv.x);
    const uint32_t cy = cell_of(p.hi[p.ld + i], lo.y, inv.y);
    const uint32_t cz = cell_of(p.hi[2 * p.ld + i], lo.z, inv.z);
    key[i] = spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2);
  }
}

// Stable LSD radix sort of the cell keys, 8-bit digits.  Block b owns keys
// [b * kSortBlock, (b + 1) * kSortBlock), taken in kRounds rounds of
// kSortThreads.  A pass: per-block digit counts, an exclusive scan of the
// counts in digit-major order (so the offset of (digit d, block b) counts
// every key of a smaller digit and every key of digit d in an earlier
// block), then a scatter in which a key's place among the equal digits of
// its block follows round, warp and lane order.  Equal keys therefore keep
// their index order and the result is unique.
constexpr int kSortThreads = 1024;
constexpr int kRounds = 4;
constexpr int kSortBlock = kSortThreads * kRounds;
constexpr int kDigitBits = 8;
constexpr int kBins = 1 << kDigitBits;

__global__ void __launch_bounds__(kSortThreads)
    digit_count_kernel(const uint32_t* key, int64_t n, int shift, int nblocks, uint32_t* hist) {
  griddep_wait();
  __shared__ uint32_t cnt[kBins];
  for (int d = threadIdx.x; d < kBins; d += blockDim.x) cnt[d] = 0;
  __syncthreads();
  for (int r = 0; r < kRounds; ++r) {
    const int64_t i = (int64_t)blockIdx.x * kSortBlock + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(key[i] >> shift) & (kBins - 1)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kBins; d += blockDim.x)
    hist[(int64_t)d * nblocks + blockIdx.x] = cnt[d];
}

// Exclusive scan of m counts in place (one block).
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) exclusive_scan_kernel(uint32_t* v, int64_t m) {
  griddep_wait();
  __shared__ uint32_t part[kScanThreads];
  const int t = threadIdx.x;
  const int64_t per = (m + kScanThreads - 1) / kScanThreads;
  const int64_t b = t * per;
  const int64_t e = b + per < m ? b + per : m;
  uint32_t s = 0;
  for (int64_t k = b; k < e; ++k) s += v[k];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {  // inclusive Hillis-Steele scan
    const uint32_t x = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  uint32_t run = t > 0 ? part[t - 1] : 0u;
  for (int64_t k = b; k < e; ++k) {
    const uint32_t c = v[k];
    v[k] = run;
    run += c;
  }
}

__global__ void __launch_bounds__(kSortThreads)
    digit_scatter_kernel(const uint32_t* key_in, const int32_t* val_in, uint32_t* key_out,
                         int32_t* val_out, int64_t n, int shift, int nblocks,
                         const uint32_t* offset) {
  griddep_wait();
  constexpr int kWarps = kSortThreads / 32;
  __shared__ uint32_t wcnt[kWarps][kBins];
  __shared__ uint32_t run[kBins];  // keys of each digit placed by earlier rounds
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int d = t; d < kBins; d += kSortThreads) run[d] = 0;
  for (int r = 0; r < kRounds; ++r) {
    for (int k = t; k < kWarps * kBins; k += kSortThreads) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kSortBlock + r * kSortThreads + t;
    const bool live = i < n;
    const uint32_t k = live ? key_in[i] : 0u;
    // keys past the end get a digit of their own so that they match no live key
    const int d = live ? (int)((k >> shift) & (kBins - 1)) : kBins;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int wrank = __popc(peers & ((1u << lane) - 1u));
    if (live && wrank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (live) {
      uint32_t before = run[d];
      for (int w = 0; w < warp; ++w) before += wcnt[w][d];
      const uint32_t pos = offset[(int64_t)d * nblocks + blockIdx.x] + before + wrank;
      key_out[pos] = k;
      val_out[pos] = val_in ? val_in[i] : (int32_t)i;
    }
    __syncthreads();
    for (int dd = t; dd < kBins; dd += kSortThreads) {
      uint32_t s = 0;
      for (int w = 0; w < kWarps; ++w) s += wcnt[w][dd];
      run[dd] += s;
    }
    // the next round's clearing of wcnt starts after this barrier
    __syncthreads();
  }
}

// Sorted copy of the point arrays: slot s holds point perm[s].
__global__ void gather_points_kernel(PointsDev p, const int32_t* perm, double* x, double* y,
                                     double* z, float* hi, float* lo) {
  griddep_wait();
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < p.n;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = perm[s];
    x[s] = p.x[i];
    y[s] = p.y[i];
    z[s] = p.z[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      hi[k * p.n + s] = p.hi[k * p.ld + i];
      lo[k * p.n + s] = p.lo[k * p.ld + i];
    }
  }
}

// ---- several problems in one order

// The problem that global index g falls in: the largest j with off[j] <= g
// (empty problems share their offset with the next one and are passed over).
__device__ __forceinline__ int problem_of(const int64_t* off, int nprob, int64_t g) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__global__ void batch_cell_key_kernel(const SortProblem* probs, const int64_t* off, int nprob,
                                      int64_t total, uint32_t* key) {
  griddep_wait();
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int j = problem_of(off, nprob, g);
    const SortProblem& P = probs[j];
    const int64_t i = g - off[j];
    uint32_t cell = 0u;
    if (P.spatial) {
      const uint32_t cx = cell_of(P.p.hi[i], P.lo.x, P.inv.x);
      const uint32_t cy = cell_of(P.p.hi[P.p.ld + i], P.lo.y, P.inv.y);
      const uint32_t cz = cell_of(P.p.hi[2 * P.p.ld + i], P.lo.z, P.inv.z);
      cell = spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2);
    }
    key[g] = ((uint32_t)j << (3 * kCellBits)) | cell;
  }
}

// Sorted copy of every problem's points (slot s holds global point perm[s],
// of the problem that owns slot s) and the problem-local permutation.
__global__ void batch_gather_kernel(const SortProblem* probs, const int64_t* off, int nprob,
                                   int64_t total, const int32_t* perm, double* x, double* y,
                                   double* z, float* hi, float* lo, int32_t* perm_local) {
  griddep_wait();
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < total;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int j = problem_of(off, nprob, s);
    const PointsDev& p = probs[j].p;
    const int64_t i = (int64_t)perm[s] - off[j];
    x[s] = p.x[i];
    y[s] = p.y[i];
    z[s] = p.z[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      hi[k * total + s] = p.hi[k * p.ld + i];
      lo[k * total + s] = p.lo[k * p.ld + i];
    }
    perm_local[s] = (int32_t)i;
  }
}

unsigned grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

int sort_blocks(int64_t n) { return (int)((n + kSortBlock - 1) / kSortBlock); }

}  // namespace

void cell_grid(const float box_lo[3], const float box_hi[3], float3* lo, float3* inv) {
  const float span = (float)(1 << kCellBits);
  lo->x = box_lo[0];
  lo->y = box_lo[1];
  lo->z = box_lo[2];
  inv->x = span / fmaxf(box_hi[0] - box_lo[0], 1e-3f);
  inv->y = span / fmaxf(box_hi[1] - box_lo[1], 1e-3f);
  inv->z = span / fmaxf(box_hi[2] - box_lo[2], 1e-3f);
}

size_t spatial_order_bytes(int64_t n) {
  const auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  return al(sizeof(uint32_t) * (size_t)kBins * sort_blocks(n)) + 2 * al(sizeof(uint32_t) * n) +
         2 * al(sizeof(int32_t) * n) + al(3 * sizeof(double) * n) + al(6 * sizeof(float) * n);
}

int spatial_order_kernels(int64_t n) {
  constexpr int kPasses = (3 * kCellBits + kDigitBits - 1) / kDigitBits;
  return n == 0 ? 0 : 2 + 3 * kPasses;
}

cudaError_t launch_spatial_order(const PointsDev& p, const float box_lo[3],
                                 const float box_hi[3], void* scratch, int32_t** perm_out,
                                 PointsDev* sorted, cudaStream_t s) {
  const auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const int64_t n = p.n;
  const int nb = sort_blocks(n);
  unsigned char* w = (unsigned char*)scratch;
  uint32_t* hist = (uint32_t*)w;
  w += al(sizeof(uint32_t) * (size_t)kBins * nb);
  uint32_t* key[2] = {(uint32_t*)w, nullptr};
  w += al(sizeof(uint32_t) * n);
  key[1] = (uint32_t*)w;
  w += al(sizeof(uint32_t) * n);
  int32_t* val[2] = {(int32_t*)w, nullptr};
  w += al(sizeof(int32_t) * n);
  val[1] = (int32_t*)w;
  w += al(sizeof(int32_t) * n);
  double* x = (double*)w;
  w += al(3 * sizeof(double) * n);
  float* hi = (float*)w;
  sorted->n = n;
  sorted->x = x;
  sorted->y = x + n;
  sorted->z = x + 2 * n;
  sorted->hi = hi;
  sorted->lo = hi + 3 * n;
  sorted->ld = n;
  constexpr int kKeyBits = 3 * kCellBits;
  constexpr int kPasses = (kKeyBits + kDigitBits - 1) / kDigitBits;
  *perm_out = val[kPasses & 1];  // where the last pass leaves the values
  if (n == 0) return cudaSuccess;
  float3 lo, inv;
  cell_grid(box_lo, box_hi, &lo, &inv);
  // each kernel waits for its predecessor's results first thing
  // (programmatic dependent launches: only the launch latency overlaps)
  cudaError_t e = launch_pdl(cell_key_kernel, grid_for(n), 256, 0, s, p, lo, inv, key[0]);
  for (int pass = 0; pass < kPasses && e == cudaSuccess; ++pass) {
    const int in = pass & 1, out = in ^ 1;
    e = launch_pdl(digit_count_kernel, nb, kSortThreads, 0, s, (const uint32_t*)key[in], n,
                   kDigitBits * pass, nb, hist);
    if (e == cudaSuccess)
      e = launch_pdl(exclusive_scan_kernel, 1, kScanThreads, 0, s, hist,
                     (int64_t)kBins * nb);
    if (e == cudaSuccess)
      e = launch_pdl(digit_scatter_kernel, nb, kSortThreads, 0, s, (const uint32_t*)key[in],
                     (const int32_t*)(pass == 0 ? nullptr : val[in]), key[out], val[out], n,
                     kDigitBits * pass, nb, (const uint32_t*)hist);
  }
  if (e == cudaSuccess)
    e = launch_pdl(gather_points_kernel, grid_for(n), 256, 0, s, p, (const int32_t*)*perm_out, x,
                   x + n, x + 2 * n, hi, hi + 3 * n);
  return e;
}

namespace {
int problem_bits(int nprob) {
  int b = 0;
  while (b < 31 && ((int64_t)1 << b) < nprob) ++b;
  return b;
}
size_t al256(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

size_t spatial_order_batch_bytes(int64_t total, int nprob) {
  (void)nprob;
  return al256(sizeof(uint32_t) * (size_t)kBins * sort_blocks(total)) +
         2 * al256(sizeof(uint32_t) * total) + 3 * al256(sizeof(int32_t) * total) +
         al256(3 * sizeof(double) * total) + al256(6 * sizeof(float) * total);
}

BatchOrder spatial_order_batch_layout(void* scratch, int64_t total, int nprob) {
  BatchOrder o{};
  unsigned char* w = (unsigned char*)scratch;
  o.hist = (uint32_t*)w;
  w += al256(sizeof(uint32_t) * (size_t)kBins * sort_blocks(total));
  for (int k = 0; k < 2; ++k) {
    o.key[k] = (uint32_t*)w;
    w += al256(sizeof(uint32_t) * total);
  }
  for (int k = 0; k < 2; ++k) {
    o.val[k] = (int32_t*)w;
    w += al256(sizeof(int32_t) * total);
  }
  o.perm = (int32_t*)w;
  w += al256(sizeof(int32_t) * total);
  double* x = (double*)w;
  w += al256(3 * sizeof(double) * total);
  float* hi = (float*)w;
  o.sorted.n = total;
  o.sorted.x = x;
  o.sorted.y = x + total;
  o.sorted.z = x + 2 * total;
  o.sorted.hi = hi;
  o.sorted.lo = hi + 3 * total;
  o.sorted.ld = total;
  o.total = total;
  o.nprob = nprob;
  const int bits = 3 * kCellBits + problem_bits(nprob);
  o.passes = (bits + kDigitBits - 1) / kDigitBits;
  return o;
}

cudaError_t launch_spatial_order_batch(const BatchOrder& o, const SortProblem* d_probs,
                                       const int64_t* d_off, cudaStream_t s) {
  const int64_t n = o.total;
  if (n == 0) return cudaSuccess;
  if (3 * kCellBits + problem_bits(o.nprob) > 32) return cudaErrorInvalidValue;
  const int nb = sort_blocks(n);
  cudaError_t e = launch_pdl(batch_cell_key_kernel, grid_for(n), 256, 0, s, d_probs, d_off,
                             o.nprob, n, o.key[0]);
  for (int pass = 0; pass < o.passes && e == cudaSuccess; ++pass) {
    const int in = pass & 1, out = in ^ 1;
    e = launch_pdl(digit_count_kernel, nb, kSortThreads, 0, s, (const uint32_t*)o.key[in], n,
                   kDigitBits * pass, nb, o.hist);
    if (e == cudaSuccess)
      e = launch_pdl(exclusive_scan_kernel, 1, kScanThreads, 0, s, o.hist, (int64_t)kBins * nb);
    if (e == cudaSuccess)
      e = launch_pdl(digit_scatter_kernel, nb, kSortThreads, 0, s, (const uint32_t*)o.key[in],
                     (const int32_t*)(pass == 0 ? nullptr : o.val[in]), o.key[out], o.val[out], n,
                     kDigitBits * pass, nb, (const uint32_t*)o.hist);
  }
  if (e == cudaSuccess) {
    double* x = const_cast<double*>(o.sorted.x);
    float* hi = const_cast<float*>(o.sorted.hi);
    e = launch_pdl(batch_gather_kernel, grid_for(n), 256, 0, s, d_probs, d_off, o.nprob, n,
                   (const int32_t*)o.val[o.passes & 1], x, x + n, x + 2 * n, hi, hi + 3 * n,
                   o.perm);
  }
  return e;
}

}  // namespace qk
