// ao_vgl.cu -- atomic-orbital values, gradients and Laplacians at every point.
//
// Sec. 3.1 of the QMCkl paper: chi_n = M_n R_s P_abc (Eq. 1), a contracted
// Gaussian radial part (Eq. 2, p = 2), primitives skipped when
// gamma r^2 >= T (Eq. 3), Cartesian polynomial (Eq. 4) built from iterated
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
// One CTA covers PT points x one column chunk of <= 64 AOs (chunks end on
// shell boundaries).  Phase 1: threads over (point, shell) pairs compute
// d = r - R_A, apply the per-shell radius (r^2 >= T/gamma_min screens the
// whole shell) and then the per-primitive test of Eq. 3 on primitives
// sorted by ascending exponent (the first screened primitive ends the loop),
// leaving S_0..S_2 and d in shared memory.  Phase 2: threads over
// (point, AO) pairs, consecutive lanes on consecutive AOs, assemble the five
// components and store them as coalesced row segments of the AO tensor
// [5*point][ld] (row 5p + c).
//
// Precision: FP64 mode does everything in FP64 and forms r^2 and gamma r^2
// without fused multiply-adds, so its screening decisions are those of the
// plain definition.  The reduced modes form d from float hi/lo pairs of the
// coordinates (exact-ish difference, then FP32), and run exp and the
// assembly in FP32.
#include "ao_common.cuh"

namespace qk {

// Output writers: plain element type, or bf16 hi/lo planes.
template <typename T>
struct StorePlain {
  static __device__ __forceinline__ void put(const AOTensor& o, int64_t row, int col, T v) {
    static_cast<T*>(o.a)[row * o.ld + col] = v;
  }
};
struct StoreSplit {
  static __device__ __forceinline__ void put(const AOTensor& o, int64_t row, int col, float v) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    static_cast<__nv_bfloat16*>(o.a)[row * o.ld + col] = hi;
    static_cast<__nv_bfloat16*>(o.a_lo)[row * o.ld + col] = lo;
  }
};

constexpr int kThreads = 256;


// shared layout: 6 arrays [PT][kChunkAO] of T: dx, dy, dz, S0, S1, S2
template <int PT, typename T>
constexpr size_t ao_smem_bytes() {
  return sizeof(T) * 6 * PT * kChunkAO;
}

template <int PT, typename T, typename Store>
__global__ void __launch_bounds__(kThreads)
    ao_vgl_kernel(BasisDev b, PointsDev pts, AOTensor out, int64_t n_ptiles) {
  using A = Arith<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* s_dx = sm;
  T* s_dy = sm + 1 * PT * kChunkAO;
  T* s_dz = sm + 2 * PT * kChunkAO;
  T* s_S0 = sm + 3 * PT * kChunkAO;
  T* s_S1 = sm + 4 * PT * kChunkAO;
  T* s_S2 = sm + 5 * PT * kChunkAO;

  const int4 ch = b.chunk[blockIdx.x];
  const int ns = ch.y - ch.x;
  const int na = ch.w - ch.z;
  const T Tthr = A::thr(b);

  for (int64_t ptile = blockIdx.y; ptile < n_ptiles; ptile += gridDim.y) {
    const int64_t p0 = ptile * PT;
    // ---- phase 1: radial sums per (point, shell)
    for (int idx = threadIdx.x; idx < PT * ns; idx += kThreads) {
      const int pl = idx % PT;
      const int sl = idx / PT;
      const int64_t ip = p0 + pl;
      const int s = ch.x + sl;
      T dx = T(0), dy = T(0), dz = T(0), S0 = T(0), S1 = T(0), S2 = T(0);
      if (ip < pts.n) {
        A::diff(b, pts, ip, b.shell_nuc[s], dx, dy, dz);
        const T r2 = A::add(A::add(A::mul(dx, dx), A::mul(dy, dy)), A::mul(dz, dz));
        if (r2 < A::r2max(b, s)) {
          const int k0 = b.shell_prim0[s];
          const int k1 = k0 + b.shell_nprim[s];
          for (int k = k0; k < k1; ++k) {
            const T g = A::gam(b, k);
            const T t = A::mul(g, r2);
            if (!(t < Tthr)) break;  // ascending exponents: the rest is screened too
            const T ce = A::coef(b, k) * A::ex(-t);
            S0 += ce;
            S1 += g * ce;
            S2 += g * g * ce;
          }
        }
      }
      const int o = pl * kChunkAO + sl;
      s_dx[o] = dx;
      s_dy[o] = dy;
      s_dz[o] = dz;
      s_S0[o] = S0;
      s_S1[o] = S1;
      s_S2[o] = S2;
    }
    __syncthreads();
    // ---- phase 2: Cartesian assembly per (point, AO), lanes along AOs
    for (int idx = threadIdx.x; idx < PT * kChunkAO; idx += kThreads) {
      const int al = idx % kChunkAO;
      const int pl = idx / kChunkAO;
      const int64_t ip = p0 + pl;
      if (al >= na || ip >= pts.n) continue;
      const int ao = ch.z + al;
      const int s = b.ao_shell[ao];
      const int l = b.shell_l[s];
      const int j = ao - b.shell_ao0[s];
      const int o = pl * kChunkAO + (s - ch.x);
      const T S0 = s_S0[o], S1 = s_S1[o], S2 = s_S2[o];
      T v = T(0), gx = T(0), gy = T(0), gz = T(0), lap = T(0);
      if (S0 != T(0) || S1 != T(0) || S2 != T(0)) {
        const T dx = s_dx[o], dy = s_dy[o], dz = s_dz[o];
        const int a = c_pow[l][j][0], bb = c_pow[l][j][1], c = c_pow[l][j][2];
        // iterated powers d^0..d^3 (Eq. 4 without pow), picked by selects so
        // that they stay in registers
        const T x2 = dx * dx, y2 = dy * dy, z2 = dz * dz;
        const T X = sel4(a, T(1), dx, x2, x2 * dx);
        const T Y = sel4(bb, T(1), dy, y2, y2 * dy);
        const T Z = sel4(c, T(1), dz, z2, z2 * dz);
        const T X1 = sel4(a, T(0), T(1), T(2) * dx, T(3) * x2);
        const T Y1 = sel4(bb, T(0), T(1), T(2) * dy, T(3) * y2);
        const T Z1 = sel4(c, T(0), T(1), T(2) * dz, T(3) * z2);
        const T X2 = sel4(a, T(0), T(0), T(2), T(6) * dx);
        const T Y2 = sel4(bb, T(0), T(0), T(2), T(6) * dy);
        const T Z2 = sel4(c, T(0), T(0), T(2), T(6) * dz);
        const T P = X * Y * Z;
        const T M = A::aofac(b, ao);
        const T r2 = x2 + y2 + z2;
        const T MS1x2 = T(2) * M * S1;
        v = M * P * S0;
        gx = M * (X1 * Y * Z) * S0 - MS1x2 * dx * P;
        gy = M * (X * Y1 * Z) * S0 - MS1x2 * dy * P;
        gz = M * (X * Y * Z1) * S0 - MS1x2 * dz * P;
        const T lapP = X2 * Y * Z + X * Y2 * Z + X * Y * Z2;
        lap = M * (lapP * S0 - T(2 * (2 * l + 3)) * P * S1 + T(4) * r2 * P * S2);
      }
      const int64_t row = 5 * ip;
      Store::put(out, row + 0, ao, v);
      Store::put(out, row + 1, ao, gx);
      Store::put(out, row + 2, ao, gy);
      Store::put(out, row + 3, ao, gz);
      Store::put(out, row + 4, ao, lap);
    }
    __syncthreads();
  }
}

template <int PT, typename T, typename Store>
static cudaError_t launch_ao(const BasisDev& b, const PointsDev& p, const AOTensor& out,
                             cudaStream_t s) {
  constexpr size_t smem = ao_smem_bytes<PT, T>();
  auto kern = ao_vgl_kernel<PT, T, Store>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t n_ptiles = (p.n + PT - 1) / PT;
  if (n_ptiles == 0 || b.nchunk == 0) return cudaSuccess;
  dim3 grid((unsigned)b.nchunk, (unsigned)(n_ptiles < 65535 ? n_ptiles : 65535));
  kern<<<grid, kThreads, smem, s>>>(b, p, out, n_ptiles);
  return cudaGetLastError();
}

cudaError_t launch_ao_vgl(const BasisDev& b, const PointsDev& p, int out_mode,
                          const AOTensor& out, cudaStream_t s) {
  switch (out_mode) {
    case QK_FP64:
      return launch_ao<16, double, StorePlain<double>>(b, p, out, s);
    case QK_FP32:
    case QK_TF32:
      return launch_ao<32, float, StorePlain<float>>(b, p, out, s);
    case QK_BF16X3:
      return launch_ao<32, float, StoreSplit>(b, p, out, s);
    default:
      return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------ helpers ---

__global__ void points_soa_kernel(const double* raw, char transp, int64_t n, double* x,
                                  double* y, double* z, float* hi, float* lo) {
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
  points_soa_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(raw, transp, n, x,
                                                                              y, z, hi, lo);
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
