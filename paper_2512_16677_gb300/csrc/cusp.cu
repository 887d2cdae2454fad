// cusp.cu -- MO cusp correction (Sec. 3.3).
//
// Inside a sphere of radius rc_A around nucleus A each MO becomes
//   phi_i^cusp = phi_i - phi_i^{s_A} + sum_{k=0}^{3} f_k^{(A,i)} rho^k,  rho = |r - R_A|,
// phi_i^{s_A} being the part of MO i carried by the s AOs on A.  The f_k
// make value, first and second radial derivative continuous at rc_A and
// satisfy Kato's cusp at the nucleus, f_1 = -Z_A (q + f_0) with
// q = phi_i(R_A) - phi_i^{s_A}(R_A).
//
// Set-up (FP64, when the basis, C, the radii or T change):
//   1. X[A][n] = chi_n(R_A), zero for the s AOs of A themselves;
//   2. Q = X C^T, so Q[A][i] = q of (A, i)          (SIMT FP64 GEMM);
//   3. one thread per (A, i): g, g', g'' of the s part at rc_A with the same
//      Eq. 3 screening as the MO evaluation, then the 4 x 4 solve.
// Correction (after the contraction, on the output rows in the caller's
// point order): pass 1 lists the points inside a sphere (a warp per 32
// points of the spatial order, spheres culled against the tile's box);
// pass 2 gives each listed point a CTA whose warps split the MOs and add
//   value      -g + p(rho)
//   gradient   (p'(rho)/rho + 2 G_1) d,          d/d rho of an s AO is -2 rho M S_1
//   Laplacian  (2 f_1/rho + 6 f_2 + 12 f_3 rho) - (4 rho^2 G_2 - 6 G_1)
// with G_m = sum over the s AOs of A of C_in M_n S_m(rho).  Whether a point
// is inside a sphere is decided in FP64 (after an FP32 prefilter); the
// correction itself runs in the output's precision: FP64 in the FP64 mode,
// FP32 (float tables, FP32 C, the coefficients rounded to float) in the
// reduced modes, whose outputs are FP32.
#include "ao_common.cuh"

namespace qk {
namespace {

__device__ __forceinline__ void s_sums(const BasisDev& b, int s, double rho2, double& S0,
                                       double& S1, double& S2) {
  S0 = S1 = S2 = 0.0;
  const int k0 = b.shell_prim0[s], k1 = k0 + b.shell_nprim[s];
  for (int k = k0; k < k1; ++k) {
    const double g = b.prim_g[k];
    const double t = __dmul_rn(g, rho2);
    if (!(t < b.T)) break;  // ascending exponents: the rest is screened too
    const double ce = b.prim_c[k] * exp(-t);
    S0 += ce;
    S1 += g * ce;
    S2 += g * g * ce;
  }
}

// X[A][n]: AO n at the position of nucleus A (value only, Eq. 1 with the
// Eq. 3 screen), zero for the s AOs on A.
__global__ void cusp_ao_at_nuclei_kernel(BasisDev b, double* X) {
  const int64_t total = (int64_t)b.nucl_num * b.ao_num;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int A = (int)(idx / b.ao_num);
    const int n = (int)(idx % b.ao_num);
    const int s = b.ao_shell[n];
    const int B = b.shell_nuc[s];
    const int l = b.shell_l[s];
    double v = 0.0;
    if (!(B == A && l == 0)) {
      const double dx = __dsub_rn(b.nucl_xyz[3 * A], b.nucl_xyz[3 * B]);
      const double dy = __dsub_rn(b.nucl_xyz[3 * A + 1], b.nucl_xyz[3 * B + 1]);
      const double dz = __dsub_rn(b.nucl_xyz[3 * A + 2], b.nucl_xyz[3 * B + 2]);
      const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                  __dmul_rn(dz, dz));
      if (r2 < b.shell_r2[s]) {
        double S0, S1, S2;
        s_sums(b, s, r2, S0, S1, S2);
        const int j = n - b.shell_ao0[s];
        double P = 1.0;
        for (int e = 0; e < c_pow[l][j][0]; ++e) P *= dx;
        for (int e = 0; e < c_pow[l][j][1]; ++e) P *= dy;
        for (int e = 0; e < c_pow[l][j][2]; ++e) P *= dz;
        v = b.ao_fac[n] * P * S0;
      }
    }
    X[idx] = v;
  }
}

// f[A][i][0..3] from the four conditions; rows A with rc_A = 0 get zeros.
__global__ void cusp_solve_kernel(BasisDev b, CuspDev cu, int64_t mo_num, const double* C,
                                  const double* Q, double* f64, float* f32) {
  const int64_t total = (int64_t)b.nucl_num * mo_num;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int A = (int)(idx / mo_num);
    const int64_t i = idx % mo_num;
    double f[4] = {0.0, 0.0, 0.0, 0.0};
    const double r = cu.rc[A];
    if (r > 0.0) {
      double g = 0.0, g1 = 0.0, g2 = 0.0;
      for (int t = cu.s_start[A]; t < cu.s_start[A + 1]; ++t) {
        const int s = cu.s_shell[t];
        const int ao = b.shell_ao0[s];
        double S0, S1, S2;
        s_sums(b, s, r * r, S0, S1, S2);
        const double w = C[i * b.ao_num + ao] * b.ao_fac[ao];
        g += w * S0;
        g1 += w * (-2.0 * r * S1);
        g2 += w * (4.0 * r * r * S2 - 2.0 * S1);
      }
      const double Z = cu.charge[A];
      const double q = Q[(int64_t)A * mo_num + i];
      // rows: value, slope, curvature at rc; Kato at the nucleus
      double M[4][5] = {{1.0, r, r * r, r * r * r, g},
                        {0.0, 1.0, 2.0 * r, 3.0 * r * r, g1},
                        {0.0, 0.0, 2.0, 6.0 * r, g2},
                        {Z, 1.0, 0.0, 0.0, -Z * q}};
      // Gaussian elimination with partial pivoting
      for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int rr = c + 1; rr < 4; ++rr)
          if (fabs(M[rr][c]) > fabs(M[piv][c])) piv = rr;
        if (piv != c)
          for (int k = 0; k < 5; ++k) {
            const double tmp = M[c][k];
            M[c][k] = M[piv][k];
            M[piv][k] = tmp;
          }
        for (int rr = c + 1; rr < 4; ++rr) {
          const double m = M[rr][c] / M[c][c];
          for (int k = c; k < 5; ++k) M[rr][k] -= m * M[c][k];
        }
      }
      for (int c = 3; c >= 0; --c) {
        double s = M[c][4];
        for (int k = c + 1; k < 4; ++k) s -= M[c][k] * f[k];
        f[c] = s / M[c][c];
      }
    }
    for (int k = 0; k < 4; ++k) {
      f64[idx * 4 + k] = f[k];
      f32[idx * 4 + k] = (float)f[k];
    }
  }
}

// s_sums in the reduced precision: float tables, FP32 exp, the same
// ascending-exponent screen.
__device__ __forceinline__ void s_sums(const BasisDev& b, int s, float rho2, float& S0, float& S1,
                                       float& S2) {
  S0 = S1 = S2 = 0.0f;
  const int k0 = b.shell_prim0[s], k1 = k0 + b.shell_nprim[s];
  for (int k = k0; k < k1; ++k) {
    const float g = b.prim_g_f[k];
    const float t = g * rho2;
    if (!(t < b.T_f)) break;
    const float ce = b.prim_c_f[k] * __expf(-t);
    S0 += ce;
    S1 += g * ce;
    S2 += g * g * ce;
  }
}

__device__ __forceinline__ double ao_factor(const BasisDev& b, int ao, double) {
  return b.ao_fac[ao];
}
__device__ __forceinline__ float ao_factor(const BasisDev& b, int ao, float) {
  return b.ao_fac_f[ao];
}

// The correction of MO columns [i0, i0 + 32) of point ip for the sphere of
// nucleus A (one warp; every lane runs the shuffles, lanes past the last MO
// skip the update).  T: arithmetic and output type; C [mo][ldc] and
// f [nucl][mo][4] in T.
template <typename T>
__device__ __forceinline__ void correct_columns(const BasisDev& b, const CuspDev& cu,
                                                const PointsDev& p, int64_t ip, int A,
                                                int64_t mo_num, int64_t i0, const T* C,
                                                int64_t ldc, const T* f, T* D, int lane) {
  const double d[3] = {__dsub_rn(p.x[ip], b.nucl_xyz[3 * A]),
                       __dsub_rn(p.y[ip], b.nucl_xyz[3 * A + 1]),
                       __dsub_rn(p.z[ip], b.nucl_xyz[3 * A + 2])};
  const double rho2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                                __dmul_rn(d[2], d[2]));
  const T rho = (T)sqrt(rho2);
  const T r2 = (T)rho2;
  const T dv[3] = {(T)d[0], (T)d[1], (T)d[2]};
  // radial sums of A's s shells, one lane per shell
  const int t0 = cu.s_start[A], ns = cu.s_start[A + 1] - t0;
  T S0 = T(0), S1 = T(0), S2 = T(0);
  if (lane < ns) s_sums(b, cu.s_shell[t0 + lane], r2, S0, S1, S2);
  const int64_t i = i0 + lane;
  const bool mine = i < mo_num;
  T G0 = T(0), G1 = T(0), G2 = T(0);
  for (int j = 0; j < ns; ++j) {
    const int ao = b.shell_ao0[cu.s_shell[t0 + j]];
    const T w = mine ? C[i * ldc + ao] * ao_factor(b, ao, T(0)) : T(0);
    G0 += w * __shfl_sync(0xffffffffu, S0, j);
    G1 += w * __shfl_sync(0xffffffffu, S1, j);
    G2 += w * __shfl_sync(0xffffffffu, S2, j);
  }
  if (!mine) return;
  const T* fi = f + ((int64_t)A * mo_num + i) * 4;
  const T inv = T(1) / rho;
  const T pv = fi[0] + rho * (fi[1] + rho * (fi[2] + rho * fi[3]));
  const T p1r = fi[1] * inv + T(2) * fi[2] + T(3) * fi[3] * rho;
  const T lapp = T(2) * fi[1] * inv + T(6) * fi[2] + T(12) * fi[3] * rho;
  const T lapg = T(4) * r2 * G2 - T(6) * G1;
  const T gs = p1r + T(2) * G1;
  T* row = D + 5 * ip * mo_num + i;
  row[0] += pv - G0;
#pragma unroll
  for (int k = 0; k < 3; ++k) row[(k + 1) * mo_num] += gs * dv[k];
  row[4 * mo_num] += lapp - lapg;
}

// Pass 1: which spheres hold each point, one warp per 32 consecutive points
// of a scan order (the spatial order when the points have one; perm maps a
// scan slot to the point's index in the output order).  A point inside
// 1..3 spheres is listed once as (point, nuclei ascending, -1 padding); a
// point inside more is listed once as (point, -2, -2, -2) and pass 2 tests
// every nucleus for it.  The tile's bounding box (float
// coordinates) is tested against every sphere, lanes over nuclei; only the
// spheres that reach the box are tested point by point (the same FP32
// prefilter and exact FP64 test as above).  The distance from a nucleus to
// the box never exceeds the distance to a point inside it, also after
// rounding (each term is the same or a smaller float difference and float
// sums are monotone), so the cull drops no point that the prefilter keeps.
__global__ void __launch_bounds__(256)
    cusp_find_tiles_kernel(BasisDev b, CuspDev cu, PointsDev q, const int32_t* perm,
                           int4* list, int* count) {
  const int lane = threadIdx.x & 31;
  const int64_t tiles = (q.n + 31) / 32;
  const int64_t wstep = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < tiles;
       t += wstep) {
    const int64_t sl = t * 32 + lane;
    const bool pv = sl < q.n;
    float xf = 0.0f, yf = 0.0f, zf = 0.0f;
    if (pv) {
      xf = q.hi[sl];
      yf = q.hi[q.ld + sl];
      zf = q.hi[2 * q.ld + sl];
    }
    float lo[3], hi[3];
    warp_box(pv, xf, yf, zf, lo, hi);
    int found[3] = {-1, -1, -1};
    int nfound = 0;
    for (int a0 = 0; a0 < b.nucl_num; a0 += 32) {
      const int a = a0 + lane;
      bool cand = false;
      if (a < b.nucl_num) {
        const float rcf = cu.rc_f[a];
        const float c[3] = {b.nucl_hi[3 * a], b.nucl_hi[3 * a + 1], b.nucl_hi[3 * a + 2]};
        float d2 = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float e = fmaxf(0.0f, fmaxf(lo[k] - c[k], c[k] - hi[k]));
          d2 += e * e;
        }
        cand = rcf > 0.0f && d2 <= rcf * rcf * 1.001f + 1e-4f;
      }
      unsigned m = __ballot_sync(0xffffffffu, cand);
      while (m) {
        const int A = a0 + __ffs(m) - 1;
        m &= m - 1u;
        if (!pv) continue;
        const float rcf = cu.rc_f[A];
        const float ex = xf - b.nucl_hi[3 * A], ey = yf - b.nucl_hi[3 * A + 1],
                    ez = zf - b.nucl_hi[3 * A + 2];
        if (!(ex * ex + ey * ey + ez * ez <= rcf * rcf * 1.001f + 1e-4f)) continue;
        const double dx = __dsub_rn(q.x[sl], b.nucl_xyz[3 * A]);
        const double dy = __dsub_rn(q.y[sl], b.nucl_xyz[3 * A + 1]);
        const double dz = __dsub_rn(q.z[sl], b.nucl_xyz[3 * A + 2]);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                    __dmul_rn(dz, dz));
        if (!(r2 < cu.rc[A] * cu.rc[A])) continue;
        if (nfound < 3) found[nfound] = A;
        ++nfound;
      }
    }
    if (!pv || nfound == 0) continue;
    const int ip = perm ? perm[sl] : (int)sl;
    const int4 it = nfound <= 3 ? make_int4(ip, found[0], found[1], found[2])
                                : make_int4(ip, -2, -2, -2);
    list[atomicAdd(count, 1)] = it;
  }
}

// Pass 2, one CTA per listed point: warps split the MO columns and apply the
// point's spheres in ascending nucleus order (each output element is
// written by one thread, so the result does not depend on scheduling).
template <typename T>
__global__ void __launch_bounds__(256)
    cusp_apply_list_kernel(BasisDev b, CuspDev cu, PointsDev p, int64_t mo_num, const T* C,
                           int64_t ldc, const T* f, T* D, const int4* list, const int* count) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  griddep_wait();  // the list is the previous kernel's output
  const int n = *count;
  for (int e = blockIdx.x; e < n; e += gridDim.x) {
    const int4 it = list[e];
    if (it.y == -2) {
      // inside more than three spheres: every nucleus, ascending
      for (int A = 0; A < b.nucl_num; ++A) {
        if (!(cu.rc[A] > 0.0)) continue;
        const double dx = __dsub_rn(p.x[it.x], b.nucl_xyz[3 * A]);
        const double dy = __dsub_rn(p.y[it.x], b.nucl_xyz[3 * A + 1]);
        const double dz = __dsub_rn(p.z[it.x], b.nucl_xyz[3 * A + 2]);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                    __dmul_rn(dz, dz));
        if (!(r2 < cu.rc[A] * cu.rc[A])) continue;
        for (int64_t i0 = 32 * (int64_t)warp; i0 < mo_num; i0 += 32 * (int64_t)nw)
          correct_columns(b, cu, p, it.x, A, mo_num, i0, C, ldc, f, D, lane);
      }
      continue;
    }
    const int nuc[3] = {it.y, it.z, it.w};
    for (int k = 0; k < 3; ++k) {
      if (nuc[k] < 0) break;
      for (int64_t i0 = 32 * (int64_t)warp; i0 < mo_num; i0 += 32 * (int64_t)nw)
        correct_columns(b, cu, p, it.x, nuc[k], mo_num, i0, C, ldc, f, D, lane);
    }
  }
}

// float copies of the radii (rounded up, so the prefilter never drops a point)
__global__ void cusp_radii_f_kernel(const double* rc, float* rc_f, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rc_f[i] = __double2float_ru(rc[i]);
}

unsigned grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_cusp_setup(const BasisDev& b, const CuspDev& cu, int64_t mo_num,
                              const double* C, double* X, double* Q, double* f64, float* f32,
                              cudaStream_t s) {
  if (b.nucl_num == 0 || mo_num == 0) return cudaSuccess;
  cusp_radii_f_kernel<<<(b.nucl_num + 255) / 256, 256, 0, s>>>(cu.rc, const_cast<float*>(cu.rc_f),
                                                               b.nucl_num);
  cusp_ao_at_nuclei_kernel<<<grid_for((int64_t)b.nucl_num * b.ao_num), 256, 0, s>>>(b, X);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // Q[A][i] = sum_n X[A][n] C[i][n]
  e = launch_gemm_f64(b.nucl_num, mo_num, b.ao_num, X, b.ao_num, 1, C, b.ao_num, 1, Q, mo_num, 1,
                      s);
  if (e != cudaSuccess) return e;
  cusp_solve_kernel<<<grid_for((int64_t)b.nucl_num * mo_num), 256, 0, s>>>(b, cu, mo_num, C, Q,
                                                                          f64, f32);
  return cudaGetLastError();
}

size_t cusp_list_bytes(int64_t n) { return sizeof(int4) * (size_t)(n > 0 ? n : 1) + 256; }

cudaError_t launch_cusp_apply(const BasisDev& b, const CuspDev& cu, const PointsDev& p,
                              const PointsDev* scan, const int32_t* perm, int64_t mo_num,
                              const double* C64, const float* C32, int64_t ldc32,
                              const double* f64, const float* f32, bool f64_out, void* D,
                              void* scratch, cudaStream_t s) {
  if (p.n == 0 || mo_num == 0) return cudaSuccess;
  int* count = (int*)scratch;
  int4* list = (int4*)((unsigned char*)scratch + 256);
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const PointsDev& q = scan ? *scan : p;
  if (q.n != p.n) return cudaErrorInvalidValue;
  // a warp per 32 scan-order points, eight warps per block
  const int64_t blocks = ((q.n + 31) / 32 + 7) / 8;
  const unsigned g = (unsigned)(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096);
  const unsigned g2 = (unsigned)(8 * device_sms());
  cusp_find_tiles_kernel<<<g, 256, 0, s>>>(b, cu, q, scan ? perm : nullptr, list, count);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (f64_out)
    return launch_pdl(cusp_apply_list_kernel<double>, g2, 256, 0, s, b, cu, p, mo_num, C64,
                      (int64_t)b.ao_num, f64, (double*)D, (const int4*)list, (const int*)count);
  return launch_pdl(cusp_apply_list_kernel<float>, g2, 256, 0, s, b, cu, p, mo_num, C32, ldc32,
                    f32, (float*)D, (const int4*)list, (const int*)count);
}

}  // namespace qk
