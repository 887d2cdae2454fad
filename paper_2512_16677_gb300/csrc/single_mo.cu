// single_mo.cu -- MO vgl at the proposed position of one electron per walker
// (single-electron moves, the usage of Sec. 4) in FP64: one launch per move.
//
// CTA (w, j) evaluates walker w's moved point for MOs [j * kMoBlock,
// (j + 1) * kMoBlock), kMoBlock = 32 lanes x NV vectors (float4 / double2):
//   1. the point's AO row (Eqs. 1-4 under the Eq. 3 screening, the same
//      arithmetic as ao_vgl) for every shell whose screening radius holds the
//      point, written as a compact list (AO index, 5 components) in shared
//      memory, shells in rounds of kThreads (one per thread), in shell order
//      (a block-wide prefix sum places each shell's entries);
//   2. the GEMV D[w][c][mo] = sum over the list of AO[c][k] C^T[k][mo]
//      (Eqs. 5-7): warp i takes entries i, i + 4, ..., its lanes NV vectors
//      of MOs each (float4 / double2 pieces of C^T rows, coalesced), several
//      entries deep; the four warps' partial sums are added in a fixed
//      order, one component at a time, in the space the list used.
// C^T is kept per upload of C in the output precision ([ao][ldm], padding
// zero).  Every step has a fixed order, so results are reproducible.
#include "ao_common.cuh"

namespace qk {
namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
constexpr int kCap = kThreads * 10;  // list entries per round: f shells have 10 components

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using V = float4;
  static constexpr int N = 4;
};
template <>
struct Vec<double> {
  using V = double2;
  static constexpr int N = 2;
};

template <typename T>
__device__ __forceinline__ void unpack(const typename Vec<T>::V& v, T* out) {
  if constexpr (Vec<T>::N == 4) {
    out[0] = v.x;
    out[1] = v.y;
    out[2] = v.z;
    out[3] = v.w;
  } else {
    out[0] = v.x;
    out[1] = v.y;
  }
}

// Basis tables staged in shared memory once per CTA: per shell its centre
// (FP64, or the float hi and lo parts) with the screening radius^2, and
// (first primitive, primitive count, l, first AO); per primitive the
// exponent and coefficient; per AO its factor M_n.
template <typename T>
struct StagedBasis {
  static size_t bytes(const BasisDev& b) {
    return sizeof(T) * 8 * (size_t)b.shell_num + sizeof(int4) * (size_t)b.shell_num +
           sizeof(T) * 2 * (size_t)b.prim_num + sizeof(T) * (size_t)b.ao_num;
  }
};

template <typename T, int NV>
__global__ void __launch_bounds__(kThreads)
    single_mo_kernel(BasisDev b, PointsDev pts, const T* __restrict__ ct, int64_t ldm,
                     int64_t mo_num, T* __restrict__ out) {
  using A = Arith<T>;
  constexpr int VN = Vec<T>::N;
  constexpr int kMoBlock = 32 * VN * NV;  // MOs of one CTA
  static_assert(kWarps * kMoBlock <= 5 * kCap, "partial sums fit in the list's space");
  extern __shared__ __align__(16) unsigned char smem[];
  T* val = reinterpret_cast<T*>(smem);                      // [5][kCap]
  int* idx = reinterpret_cast<int*>(val + 5 * kCap);        // [kCap]
  T* part = val;                                            // [kWarps][kMoBlock], after the list
  // staged tables
  T* shc = reinterpret_cast<T*>(idx + kCap);                // [shell][8]: x, y, z, r2max, xl, yl, zl, -
  int4* meta = reinterpret_cast<int4*>(shc + 8 * (size_t)b.shell_num);  // [shell]
  T* pg = reinterpret_cast<T*>(meta + b.shell_num);         // [prim]
  T* pc = pg + b.prim_num;                                  // [prim]
  T* Mf = pc + b.prim_num;                                  // [ao]
  __shared__ int wsum[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t w = blockIdx.x;
  const int64_t m0 = (int64_t)blockIdx.y * kMoBlock;
  griddep_wait();
  for (int s = tid; s < b.shell_num; s += kThreads) {
    const int a = b.shell_nuc[s];
    T* c = shc + 8 * s;
    if constexpr (sizeof(T) == 8) {
      c[0] = b.nucl_xyz[3 * a];
      c[1] = b.nucl_xyz[3 * a + 1];
      c[2] = b.nucl_xyz[3 * a + 2];
    } else {
      c[0] = b.nucl_hi[3 * a];
      c[1] = b.nucl_hi[3 * a + 1];
      c[2] = b.nucl_hi[3 * a + 2];
      c[4] = b.nucl_lo[3 * a];
      c[5] = b.nucl_lo[3 * a + 1];
      c[6] = b.nucl_lo[3 * a + 2];
    }
    c[3] = A::r2max(b, s);
    meta[s] = make_int4(b.shell_prim0[s], b.shell_nprim[s], b.shell_l[s], b.shell_ao0[s]);
  }
  for (int k = tid; k < b.prim_num; k += kThreads) {
    pg[k] = A::gam(b, k);
    pc[k] = A::coef(b, k);
  }
  for (int k = tid; k < b.ao_num; k += kThreads) Mf[k] = A::aofac(b, k);
  // the moved point (FP64, or the float hi/lo pair)
  T X, Y, Z, Xl = T(0), Yl = T(0), Zl = T(0);
  if constexpr (sizeof(T) == 8) {
    X = pts.x[w];
    Y = pts.y[w];
    Z = pts.z[w];
  } else {
    X = pts.hi[w];
    Y = pts.hi[pts.ld + w];
    Z = pts.hi[2 * pts.ld + w];
    Xl = pts.lo[w];
    Yl = pts.lo[pts.ld + w];
    Zl = pts.lo[2 * pts.ld + w];
  }
  const T Tthr = A::thr(b);
  T acc[NV][5][VN];
#pragma unroll
  for (int j = 0; j < NV; ++j)
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int v = 0; v < VN; ++v) acc[j][c][v] = T(0);
  // this lane's MO vectors: m0 + (j * 32 + lane) * VN, j < NV
  int64_t mo_vec[NV];
  bool vec_in[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    mo_vec[j] = m0 + (int64_t)(j * 32 + lane) * VN;
    vec_in[j] = mo_vec[j] < mo_num;
  }
  __syncthreads();

  for (int s0 = 0; s0 < b.shell_num; s0 += kThreads) {
    // ---- 1. AO row entries of shells s0 .. s0 + kThreads - 1
    const int s = s0 + tid;
    int n = 0, l = 0, ao0 = 0;
    T dx = T(0), dy = T(0), dz = T(0), S0 = T(0), S1 = T(0), S2 = T(0);
    if (s < b.shell_num) {
      const T* c = shc + 8 * s;
      if constexpr (sizeof(T) == 8) {
        dx = __dsub_rn(X, c[0]);
        dy = __dsub_rn(Y, c[1]);
        dz = __dsub_rn(Z, c[2]);
      } else {
        dx = (X - c[0]) + (Xl - c[4]);
        dy = (Y - c[1]) + (Yl - c[5]);
        dz = (Z - c[2]) + (Zl - c[6]);
      }
      const T r2 = A::add(A::add(A::mul(dx, dx), A::mul(dy, dy)), A::mul(dz, dz));
      if (r2 < c[3]) {
        const int4 m = meta[s];
        for (int k = m.x; k < m.x + m.y; ++k) {
          const T gm = pg[k];
          const T t = A::mul(gm, r2);
          if (!(t < Tthr)) break;  // ascending exponents: the rest is screened too
          const T ce = pc[k] * A::ex(-t);
          S0 += ce;
          S1 += gm * ce;
          S2 += gm * gm * ce;
        }
        if (S0 != T(0) || S1 != T(0) || S2 != T(0)) {
          l = m.z;
          ao0 = m.w;
          n = (l + 1) * (l + 2) / 2;
        }
      }
    }
    // block-wide exclusive prefix sum of n (shell order)
    int x = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) {
      const int v = wsum[k];
      before += k < warp ? v : 0;
      total += v;
    }
    const int off = before + x - n;
    if (n) {
      const T* M = Mf + ao0;
      T* st = val + off;
      switch (l) {
        case 0: shell_components<T, 0, kCap>(dx, dy, dz, S0, S1, S2, M, st); break;
        case 1: shell_components<T, 1, kCap>(dx, dy, dz, S0, S1, S2, M, st); break;
        case 2: shell_components<T, 2, kCap>(dx, dy, dz, S0, S1, S2, M, st); break;
        default: shell_components<T, 3, kCap>(dx, dy, dz, S0, S1, S2, M, st); break;
      }
      for (int j = 0; j < n; ++j) idx[off + j] = ao0 + j;
    }
    __syncthreads();
    // ---- 2. this round's entries into the accumulators, four deep
    constexpr int kU = 4;
    int e = warp;
    for (; e + (kU - 1) * kWarps < total; e += kU * kWarps) {
      typename Vec<T>::V cv[kU][NV];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const T* row = ct + (int64_t)idx[e + u * kWarps] * ldm;
#pragma unroll
        for (int j = 0; j < NV; ++j)
          if (vec_in[j]) cv[u][j] = *reinterpret_cast<const typename Vec<T>::V*>(row + mo_vec[j]);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int eu = e + u * kWarps;
        T a[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) a[c] = val[c * kCap + eu];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
          if (!vec_in[j]) continue;
          T cc[VN];
          unpack<T>(cv[u][j], cc);
#pragma unroll
          for (int c = 0; c < 5; ++c)
#pragma unroll
            for (int v = 0; v < VN; ++v) acc[j][c][v] = fma(a[c], cc[v], acc[j][c][v]);
        }
      }
    }
    for (; e < total; e += kWarps) {
      const T* row = ct + (int64_t)idx[e] * ldm;
      T a[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) a[c] = val[c * kCap + e];
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        if (!vec_in[j]) continue;
        T cc[VN];
        unpack<T>(*reinterpret_cast<const typename Vec<T>::V*>(row + mo_vec[j]), cc);
#pragma unroll
        for (int c = 0; c < 5; ++c)
#pragma unroll
          for (int v = 0; v < VN; ++v) acc[j][c][v] = fma(a[c], cc[v], acc[j][c][v]);
      }
    }
    __syncthreads();  // the list is rebuilt in the next round
  }
  // ---- the warps' partial sums, added in warp order, a component at a time
#pragma unroll
  for (int c = 0; c < 5; ++c) {
#pragma unroll
    for (int j = 0; j < NV; ++j)
#pragma unroll
      for (int v = 0; v < VN; ++v) part[warp * kMoBlock + (j * 32 + lane) * VN + v] = acc[j][c][v];
    __syncthreads();
    for (int m = tid; m < kMoBlock; m += kThreads) {
      T sum = T(0);
#pragma unroll
      for (int k = 0; k < kWarps; ++k) sum += part[k * kMoBlock + m];
      if (m0 + m < mo_num) out[(w * 5 + c) * mo_num + m0 + m] = sum;
    }
    __syncthreads();
  }
}

// C [mo][ao] (FP64) -> C^T [ao][ldm] in T, padding zero
template <typename T>
__global__ void ct_kernel(const double* __restrict__ C, int64_t mo, int64_t ao, int64_t ldm,
                          T* __restrict__ ct) {
  const int64_t n = ao * ldm;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = i / ldm, m = i % ldm;
    ct[i] = m < mo ? (T)C[m * ao + a] : T(0);
  }
}

template <typename T>
size_t single_smem(const BasisDev& b) {
  return sizeof(T) * 5 * kCap + sizeof(int) * kCap + StagedBasis<T>::bytes(b);
}

// Whether the kernel's shared memory (list + staged basis) fits a CTA.
template <typename T>
bool single_fits(const BasisDev& b) {
  return single_smem<T>(b) <= 160 * 1024;
}

template <typename T, int NV>
cudaError_t launch_nv(const BasisDev& b, const PointsDev& p, const T* ct, int64_t ldm,
                      int64_t mo_num, T* out, cudaStream_t s) {
  constexpr int64_t kMoBlock = 32 * Vec<T>::N * NV;
  const int64_t gy = (mo_num + kMoBlock - 1) / kMoBlock;
  if (gy > 65535 || p.n > INT32_MAX) return cudaErrorInvalidValue;
  const size_t smem = single_smem<T>(b);
  KernelFacts f;
  // the attribute is set once, for the largest size the kernel accepts
  cudaError_t e = kernel_facts<single_mo_kernel<T, NV>>(160 * 1024, kThreads, &f);
  if (e != cudaSuccess) return e;
  return launch_pdl(single_mo_kernel<T, NV>, dim3((unsigned)p.n, (unsigned)gy), kThreads, smem,
                    s, b, p, ct, ldm, mo_num, out);
}

template <typename T>
cudaError_t launch_t(const BasisDev& b, const PointsDev& p, const T* ct, int64_t ldm,
                     int64_t mo_num, T* out, cudaStream_t s) {
  // one CTA per point when at most three (FP32) or four (FP64) vectors per
  // lane cover the MOs, else several
  const int64_t per_vec = 32 * Vec<T>::N;
  const int64_t nv = (mo_num + per_vec - 1) / per_vec;
  if (nv <= 1) return launch_nv<T, 1>(b, p, ct, ldm, mo_num, out, s);
  if (nv == 2) return launch_nv<T, 2>(b, p, ct, ldm, mo_num, out, s);
  if (sizeof(T) == 4) return launch_nv<T, 3>(b, p, ct, ldm, mo_num, out, s);
  return launch_nv<T, 4>(b, p, ct, ldm, mo_num, out, s);
}

}  // namespace

bool single_mo_fits(bool f64, const BasisDev& b) { return f64 && single_fits<double>(b); }

int64_t single_ct_ld(bool f64, int64_t mo_num) {
  const int64_t v = f64 ? 2 : 4;
  return (mo_num + v - 1) / v * v;
}

cudaError_t launch_single_ct(bool f64, const double* C, int64_t mo_num, int64_t ao_num, void* ct,
                             cudaStream_t s) {
  const int64_t ldm = single_ct_ld(f64, mo_num);
  const int64_t n = ao_num * ldm;
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  const unsigned g = (unsigned)(blocks < 4096 ? blocks : 4096);
  if (f64)
    ct_kernel<double><<<g, 256, 0, s>>>(C, mo_num, ao_num, ldm, (double*)ct);
  else
    ct_kernel<float><<<g, 256, 0, s>>>(C, mo_num, ao_num, ldm, (float*)ct);
  return cudaGetLastError();
}

cudaError_t launch_single_mo(bool f64, const BasisDev& b, const PointsDev& p, const void* ct,
                             int64_t mo_num, void* out, cudaStream_t s) {
  if (!f64) return cudaErrorInvalidValue;  // the reduced modes take the tile kernels
  if (p.n == 0 || mo_num == 0) return cudaSuccess;
  const int64_t ldm = single_ct_ld(f64, mo_num);
  return launch_t<double>(b, p, (const double*)ct, ldm, mo_num, (double*)out, s);
}

}  // namespace qk
