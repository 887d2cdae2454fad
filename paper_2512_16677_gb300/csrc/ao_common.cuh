// ao_common.cuh -- device helpers shared by the AO evaluation kernels
// (forward ao_vgl and the adjoint): Cartesian exponent table, the FP64 /
// FP32 arithmetic policies and register selects.
#pragma once

#include "internal.h"

namespace qk {

// (a, b, c) of Cartesian component j of a shell of momentum l.
static __constant__ signed char c_pow[4][10][3] = {
    {{0, 0, 0}},
    {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {{2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}},
    {{3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1}, {1, 0, 2}, {0, 3, 0}, {0, 2, 1},
     {0, 1, 2}, {0, 0, 3}}};

template <typename T>
struct Arith;

template <>
struct Arith<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double ex(double x) { return exp(x); }
  static __device__ __forceinline__ void diff(const BasisDev& b, const PointsDev& p, int64_t ip,
                                              int a, double& dx, double& dy, double& dz) {
    dx = __dsub_rn(p.x[ip], b.nucl_xyz[3 * a + 0]);
    dy = __dsub_rn(p.y[ip], b.nucl_xyz[3 * a + 1]);
    dz = __dsub_rn(p.z[ip], b.nucl_xyz[3 * a + 2]);
  }
  static __device__ __forceinline__ double r2max(const BasisDev& b, int s) { return b.shell_r2[s]; }
  static __device__ __forceinline__ double gam(const BasisDev& b, int k) { return b.prim_g[k]; }
  static __device__ __forceinline__ double coef(const BasisDev& b, int k) { return b.prim_c[k]; }
  static __device__ __forceinline__ double aofac(const BasisDev& b, int k) { return b.ao_fac[k]; }
  static __device__ __forceinline__ double thr(const BasisDev& b) { return b.T; }
};

template <>
struct Arith<float> {
  static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ float ex(float x) { return __expf(x); }
  static __device__ __forceinline__ void diff(const BasisDev& b, const PointsDev& p, int64_t ip,
                                              int a, float& dx, float& dy, float& dz) {
    const int64_t n = p.n;
    // (x_hi - X_hi) is exact when the two are close (Sterbenz) and otherwise
    // rounds once; adding the residual difference restores FP32 accuracy of d.
    dx = (p.hi[ip] - b.nucl_hi[3 * a + 0]) + (p.lo[ip] - b.nucl_lo[3 * a + 0]);
    dy = (p.hi[n + ip] - b.nucl_hi[3 * a + 1]) + (p.lo[n + ip] - b.nucl_lo[3 * a + 1]);
    dz = (p.hi[2 * n + ip] - b.nucl_hi[3 * a + 2]) + (p.lo[2 * n + ip] - b.nucl_lo[3 * a + 2]);
  }
  static __device__ __forceinline__ float r2max(const BasisDev& b, int s) { return b.shell_r2_f[s]; }
  static __device__ __forceinline__ float gam(const BasisDev& b, int k) { return b.prim_g_f[k]; }
  static __device__ __forceinline__ float coef(const BasisDev& b, int k) { return b.prim_c_f[k]; }
  static __device__ __forceinline__ float aofac(const BasisDev& b, int k) { return b.ao_fac_f[k]; }
  static __device__ __forceinline__ float thr(const BasisDev& b) { return b.T_f; }
};

template <typename T>
__device__ __forceinline__ T sel4(int i, T v0, T v1, T v2, T v3) {
  return i == 0 ? v0 : (i == 1 ? v1 : (i == 2 ? v2 : v3));
}

}  // namespace qk
