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
    const int64_t n = p.ld;
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

constexpr int kPT = 32;  // points per tile slot: one lane per point in the radial phase

// Shared memory of one CTA (templated on the arithmetic type).
template <typename T>
struct AOShared {
  // chunk tables (loaded once)
  T nuc[kMaxShellsChunk][3];     // FP64: R_A; FP32: float(R_A)
  T nuc_lo[kMaxShellsChunk][3];  // FP32: residual R_A - float(R_A)
  T r2max[kMaxShellsChunk];
  int prim0[kMaxShellsChunk];    // first primitive, local to the chunk
  int nprim[kMaxShellsChunk];
  T g[kMaxPrimsChunk];
  T c[kMaxPrimsChunk];
  T M[kChunkAO];
  int ao_info[kChunkAO];  // local shell | l << 8 | Cartesian index << 12
  // per tile: [point][shell] with one pad column, so that phase 1 (lanes over
  // points) and phase 2 (lanes over AOs of one point) hit distinct banks
  T pt[kPT][3];
  T pt_lo[kPT][3];
  T d[3][kPT][kMaxShellsChunk + 1];
  T S[3][kPT][kMaxShellsChunk + 1];
};

// The chunk's shell, primitive and AO tables into shared memory (threads
// tid = 0..nthreads-1 of the calling group share the work).
template <typename T>
__device__ __forceinline__ void load_chunk_tables(const BasisDev& b, int q, AOShared<T>& sh,
                                                  int tid, int nthreads) {
  using A = Arith<T>;
  const int4 ch = b.chunk[q];
  const int ns = ch.y - ch.x;
  const int na = ch.w - ch.z;
  const int p_first = b.shell_prim0[ch.x];
  for (int i = tid; i < ns; i += nthreads) {
    const int s = ch.x + i;
    const int A_ = b.shell_nuc[s];
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int k = 0; k < 3; ++k) sh.nuc[i][k] = b.nucl_xyz[3 * A_ + k];
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        sh.nuc[i][k] = b.nucl_hi[3 * A_ + k];
        sh.nuc_lo[i][k] = b.nucl_lo[3 * A_ + k];
      }
    }
    sh.r2max[i] = A::r2max(b, s);
    sh.prim0[i] = b.shell_prim0[s] - p_first;
    sh.nprim[i] = b.shell_nprim[s];
  }
  const int np_chunk = b.shell_prim0[ch.y - 1] + b.shell_nprim[ch.y - 1] - p_first;
  for (int i = tid; i < np_chunk; i += nthreads) {
    sh.g[i] = A::gam(b, p_first + i);
    sh.c[i] = A::coef(b, p_first + i);
  }
  for (int i = tid; i < na; i += nthreads) {
    const int ao = ch.z + i;
    const int s = b.ao_shell[ao];
    sh.ao_info[i] = (s - ch.x) | (b.shell_l[s] << 8) | ((ao - b.shell_ao0[s]) << 12);
    sh.M[i] = A::aofac(b, ao);
  }
}

// Radial phase for one tile: warp w of `nwarps` takes shells w, w + nwarps,
// ...; lane pl < tp is point p0 + pl.  Leaves d and S_0..S_2 in shared
// memory; returns whether this thread saw a nonzero S.
template <typename T>
__device__ __forceinline__ int radial_phase(AOShared<T>& sh, int ns, int warp, int nwarps,
                                            int lane, int tp, int64_t p0, int64_t n, T Tthr) {
  using A = Arith<T>;
  int live = 0;
  for (int sl = warp; sl < ns; sl += nwarps) {
    const int pl = lane;
    T dx = T(0), dy = T(0), dz = T(0), S0 = T(0), S1 = T(0), S2 = T(0);
    if (pl < tp && p0 + pl < n) {
      if constexpr (sizeof(T) == 8) {
        dx = __dsub_rn(sh.pt[pl][0], sh.nuc[sl][0]);
        dy = __dsub_rn(sh.pt[pl][1], sh.nuc[sl][1]);
        dz = __dsub_rn(sh.pt[pl][2], sh.nuc[sl][2]);
      } else {
        // hi parts cancel exactly when close; the residuals restore FP32
        // accuracy of the difference
        dx = (sh.pt[pl][0] - sh.nuc[sl][0]) + (sh.pt_lo[pl][0] - sh.nuc_lo[sl][0]);
        dy = (sh.pt[pl][1] - sh.nuc[sl][1]) + (sh.pt_lo[pl][1] - sh.nuc_lo[sl][1]);
        dz = (sh.pt[pl][2] - sh.nuc[sl][2]) + (sh.pt_lo[pl][2] - sh.nuc_lo[sl][2]);
      }
      const T r2 = A::add(A::add(A::mul(dx, dx), A::mul(dy, dy)), A::mul(dz, dz));
      if (r2 < sh.r2max[sl]) {
        const int k0 = sh.prim0[sl];
        const int k1 = k0 + sh.nprim[sl];
        for (int k = k0; k < k1; ++k) {
          const T gm = sh.g[k];
          const T t = A::mul(gm, r2);
          if (!(t < Tthr)) break;  // ascending exponents: the rest is screened too
          const T ce = sh.c[k] * A::ex(-t);
          S0 += ce;
          S1 += gm * ce;
          S2 += gm * gm * ce;
        }
      }
    }
    sh.d[0][pl][sl] = dx;
    sh.d[1][pl][sl] = dy;
    sh.d[2][pl][sl] = dz;
    sh.S[0][pl][sl] = S0;
    sh.S[1][pl][sl] = S1;
    sh.S[2][pl][sl] = S2;
    live |= (S0 != T(0) || S1 != T(0) || S2 != T(0));
  }
  return live;
}

// The five components of local AO `al` at tile point `pl`.
template <typename T>
__device__ __forceinline__ void assemble(const AOShared<T>& sh, int al, int pl, T out[5]) {
  const int info = sh.ao_info[al];
  const int sl = info & 0xff;
  const T S0 = sh.S[0][pl][sl], S1 = sh.S[1][pl][sl], S2 = sh.S[2][pl][sl];
  if (S0 == T(0) && S1 == T(0) && S2 == T(0)) {
#pragma unroll
    for (int c = 0; c < 5; ++c) out[c] = T(0);
    return;
  }
  const int l = (info >> 8) & 0xf;
  const int j = info >> 12;
  const T dx = sh.d[0][pl][sl], dy = sh.d[1][pl][sl], dz = sh.d[2][pl][sl];
  const int a = c_pow[l][j][0], bb = c_pow[l][j][1], c = c_pow[l][j][2];
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
  const T M = sh.M[al];
  const T r2 = x2 + y2 + z2;
  const T MS0 = M * S0;
  const T MS1x2 = T(2) * M * S1;
  out[0] = MS0 * P;
  out[1] = MS0 * (X1 * Y * Z) - MS1x2 * dx * P;
  out[2] = MS0 * (X * Y1 * Z) - MS1x2 * dy * P;
  out[3] = MS0 * (X * Y * Z1) - MS1x2 * dz * P;
  const T lapP = X2 * Y * Z + X * Y2 * Z + X * Y * Z2;
  out[4] = M * (lapP * S0 - T(2 * (2 * l + 3)) * P * S1 + T(4) * r2 * P * S2);
}

// ------------------------------------------------------------------------
// Shell-major evaluation.  One warp takes one shell, one lane one point: the
// radial sums S_0..S_2 and the 1-D power tables of d are formed once per
// (point, shell) and every Cartesian component of the shell follows with
// its exponents known at compile time.  Results land in a shared staging
// tile [5 * points][kStagePitch] (row 5 p + c, column = AO in the chunk);
// the odd pitch keeps both the column writes (lanes over points) and the
// row reads (lanes over AOs) free of bank conflicts.  kLanes point lanes
// own staging rows; lanes at or past kLanes - 1 share the last lane's rows
// (with 25-point tiles, kLanes = 26 leaves zeros in rows 125..129).
constexpr int kStagePitch = kChunkAO + 1;

// (a, b, c) of Cartesian component j of momentum l: a from l down to 0, then
// b from l - a down to 0 (the order of the c_pow table).
__host__ __device__ constexpr int cart_exp(int l, int j, int axis) {
  int idx = 0;
  for (int a = l; a >= 0; --a)
    for (int b = l - a; b >= 0; --b) {
      if (idx == j) return axis == 0 ? a : (axis == 1 ? b : l - a - b);
      ++idx;
    }
  return 0;
}

template <typename T, int kLanes>
struct AOStageSmem {
  using value_type = T;
  static constexpr int kRows = 5 * kLanes;  // staging rows
  T nuc[kMaxShellsChunk][3];     // FP64: R_A; FP32: float(R_A)
  T nuc_lo[kMaxShellsChunk][3];  // FP32: residual R_A - float(R_A)
  T r2max[kMaxShellsChunk];
  T g[kMaxPrimsChunk];
  T c[kMaxPrimsChunk];
  T M[kChunkAO];
  T pt[kPT][3];
  T pt_lo[kPT][3];
  int prim0[kMaxShellsChunk];  // first primitive, local to the chunk
  int nprim[kMaxShellsChunk];
  int col[kMaxShellsChunk];    // first column of the shell in the chunk
  int lsh[kMaxShellsChunk];
  int order[kMaxShellsChunk];  // shells by descending estimated cost
  int work[kMaxShellsChunk];   // this tile's shells to visit, in `order` order
  unsigned char dirty[kMaxShellsChunk];  // staging columns of the shell may be nonzero
  unsigned reach;              // bit s: shell s may reach a point of the tile
  unsigned gmask;              // bit g: 16-AO column group g holds a nonzero entry
  int nwork;
  int next;                    // next entry of `work` to hand out
  T stage[5 * kLanes][kStagePitch];
};

// Chunk tables into shared memory and zeros into the staging columns past
// the chunk's last AO (nothing else writes them).  Smem: a shared-memory
// layout with the table fields of AOStageSmem, a staging tile of
// Smem::kRows rows and a dirty flag per shell.
template <class Smem>
__device__ __forceinline__ void load_stage_tables(const BasisDev& b, int q, Smem& sh, int tid,
                                                  int nthreads) {
  using T = typename Smem::value_type;
  using A = Arith<T>;
  const int4 ch = b.chunk[q];
  const int ns = ch.y - ch.x;
  const int na = ch.w - ch.z;
  const int p_first = b.shell_prim0[ch.x];
  for (int i = tid; i < ns; i += nthreads) {
    const int s = ch.x + i;
    const int A_ = b.shell_nuc[s];
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int k = 0; k < 3; ++k) sh.nuc[i][k] = b.nucl_xyz[3 * A_ + k];
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        sh.nuc[i][k] = b.nucl_hi[3 * A_ + k];
        sh.nuc_lo[i][k] = b.nucl_lo[3 * A_ + k];
      }
    }
    sh.r2max[i] = A::r2max(b, s);
    sh.prim0[i] = b.shell_prim0[s] - p_first;
    sh.nprim[i] = b.shell_nprim[s];
    sh.col[i] = b.shell_ao0[s] - ch.z;
    const int l = b.shell_l[s];
    sh.lsh[i] = l;
    sh.dirty[i] = 1;  // columns hold whatever the previous chunk left
    // cost ~ primitives (radial sums) + Cartesian components (assembly);
    // rank by descending cost, ties by position
    auto cost = [&](int ss) {
      const int ll = b.shell_l[ss];
      return 8 * b.shell_nprim[ss] + 15 * (ll + 1) * (ll + 2);
    };
    const int ci = cost(s);
    int rank = 0;
    for (int j = 0; j < ns; ++j) {
      const int cj = cost(ch.x + j);
      rank += (cj > ci) || (cj == ci && j < i);
    }
    sh.order[rank] = i;
  }
  const int np_chunk = b.shell_prim0[ch.y - 1] + b.shell_nprim[ch.y - 1] - p_first;
  for (int i = tid; i < np_chunk; i += nthreads) {
    sh.g[i] = A::gam(b, p_first + i);
    sh.c[i] = A::coef(b, p_first + i);
  }
  for (int i = tid; i < na; i += nthreads) sh.M[i] = A::aofac(b, ch.z + i);
  const int npad = kChunkAO - na;
  for (int i = tid; i < Smem::kRows * npad; i += nthreads)
    sh.stage[i / npad][na + i % npad] = T(0);
}

// Cartesian component J of a momentum-L shell at one point:
//   chi = M S0 P,  d_i chi = M (S0 d_iP - 2 S1 d_i P),
//   lap chi = M (S0 lapP + (4 r^2 S2 - 2 (2L+3) S1) P),
// with u_i = 2 S1 d_i and Lr = 4 r^2 S2 - 2 (2L+3) S1 formed once per shell.
template <typename T, int L, int J, int kPitch = kStagePitch>
__device__ __forceinline__ void cart_component(const T (&px)[4], const T (&py)[4],
                                               const T (&pz)[4], const T* M, T S0, T ux, T uy,
                                               T uz, T Lr, T* st) {
  if constexpr (J < (L + 1) * (L + 2) / 2) {
    constexpr int a = cart_exp(L, J, 0), b = cart_exp(L, J, 1), c = cart_exp(L, J, 2);
    const T P = px[a] * py[b] * pz[c];
    const T mS0 = M[J] * S0;
    const T mP = M[J] * P;
    st[J] = mS0 * P;
    if constexpr (a > 0)
      st[kPitch + J] = mS0 * (T(a) * px[a > 0 ? a - 1 : 0] * py[b] * pz[c]) - ux * mP;
    else
      st[kPitch + J] = -(ux * mP);
    if constexpr (b > 0)
      st[2 * kPitch + J] = mS0 * (T(b) * px[a] * py[b > 0 ? b - 1 : 0] * pz[c]) - uy * mP;
    else
      st[2 * kPitch + J] = -(uy * mP);
    if constexpr (c > 0)
      st[3 * kPitch + J] = mS0 * (T(c) * px[a] * py[b] * pz[c > 0 ? c - 1 : 0]) - uz * mP;
    else
      st[3 * kPitch + J] = -(uz * mP);
    if constexpr (a > 1 || b > 1 || c > 1) {
      T lapP = T(0);
      bool first = true;
      if constexpr (a > 1) {
        lapP = T(a * (a - 1)) * px[a > 1 ? a - 2 : 0] * py[b] * pz[c];
        first = false;
      }
      if constexpr (b > 1) {
        const T t = T(b * (b - 1)) * px[a] * py[b > 1 ? b - 2 : 0] * pz[c];
        lapP = first ? t : lapP + t;
        first = false;
      }
      if constexpr (c > 1) {
        const T t = T(c * (c - 1)) * px[a] * py[b] * pz[c > 1 ? c - 2 : 0];
        lapP = first ? t : lapP + t;
      }
      st[4 * kPitch + J] = mS0 * lapP + Lr * mP;
    } else {
      st[4 * kPitch + J] = Lr * mP;
    }
    cart_component<T, L, J + 1, kPitch>(px, py, pz, M, S0, ux, uy, uz, Lr, st);
  }
}

// All components of a momentum-L shell at one point into the staging rows
// st[c * kPitch + j] (c = value, d/dx, d/dy, d/dz, Laplacian).
template <typename T, int L, int kPitch = kStagePitch>
__device__ __forceinline__ void shell_components(T dx, T dy, T dz, T S0, T S1, T S2, const T* M,
                                                 T* st) {
  const T x2 = dx * dx, y2 = dy * dy, z2 = dz * dz;
  const T px[4] = {T(1), dx, x2, x2 * dx};
  const T py[4] = {T(1), dy, y2, y2 * dy};
  const T pz[4] = {T(1), dz, z2, z2 * dz};
  const T r2 = x2 + y2 + z2;
  const T S1x2 = T(2) * S1;
  const T Lr = T(4) * r2 * S2 - T(2 * (2 * L + 3)) * S1;
  cart_component<T, L, 0, kPitch>(px, py, pz, M, S0, S1x2 * dx, S1x2 * dy, S1x2 * dz, Lr, st);
}

// Zeros into the staging columns of shell `sl` if they may hold values of
// an earlier tile (whole warp; only this warp touches the shell this tile).
template <typename T, int kLanes>
__device__ __forceinline__ void shell_zero_columns(AOStageSmem<T, kLanes>& sh, int sl, int lane) {
  if (!sh.dirty[sl]) return;
  const int l = sh.lsh[sl];
  const int nc = (l + 1) * (l + 2) / 2;
  T* st = &sh.stage[5 * (lane < kLanes ? lane : kLanes - 1)][sh.col[sl]];
  for (int j = 0; j < nc; ++j) {
#pragma unroll
    for (int c = 0; c < 5; ++c) st[c * kStagePitch + j] = T(0);
  }
  __syncwarp();
  if (lane == 0) sh.dirty[sl] = 0;
}

// Whether a shell centred at c with screening radius^2 r2max may reach a
// point of the box [lo, hi]: the squared distance from c to the box bounds
// r^2 from below for every point in it, so the shell is kept unless that
// bound, less a relative and absolute margin for the rounding of both
// sides, is at least r2max.
template <typename T>
__device__ __forceinline__ bool shell_reaches_box(const T (&lo)[3], const T (&hi)[3], T cx, T cy,
                                                  T cz, T r2max) {
  const T c[3] = {cx, cy, cz};
  T d2 = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T e = max(T(0), max(lo[k] - c[k], c[k] - hi[k]));
    d2 += e * e;
  }
  return d2 * T(0.9999) - T(1e-3) < r2max;
}

// Bounding box of the valid points held one per lane (whole warp).
template <typename T>
__device__ __forceinline__ void warp_box(bool pv, T x, T y, T z, T (&lo)[3], T (&hi)[3]) {
  const T big = T(3.0e38);
  lo[0] = pv ? x : big;
  lo[1] = pv ? y : big;
  lo[2] = pv ? z : big;
  hi[0] = pv ? x : -big;
  hi[1] = pv ? y : -big;
  hi[2] = pv ? z : -big;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  }
}

// The coordinates of point p0 + lane of a tile (lane < tp, inside the point
// set), held in registers: FP64 values, or the float hi/lo pairs.
template <typename T>
struct TilePoint {
  T x, y, z;     // FP64: the coordinates; FP32: their float hi parts
  T lx, ly, lz;  // FP32: the residuals
  bool pv;
};

template <typename T>
__device__ __forceinline__ TilePoint<T> tile_point(const PointsDev& pts, int lane, int tp,
                                                   int64_t p0) {
  TilePoint<T> r;
  const int64_t ip = p0 + lane;
  r.pv = lane < tp && ip < pts.n;
  r.x = r.y = r.z = r.lx = r.ly = r.lz = T(0);
  if (r.pv) {
    if constexpr (sizeof(T) == 8) {
      r.x = pts.x[ip];
      r.y = pts.y[ip];
      r.z = pts.z[ip];
    } else {
      const int64_t ld = pts.ld;
      r.x = pts.hi[ip];
      r.y = pts.hi[ld + ip];
      r.z = pts.hi[2 * ld + ip];
      r.lx = pts.lo[ip];
      r.ly = pts.lo[ld + ip];
      r.lz = pts.lo[2 * ld + ip];
    }
  }
  return r;
}

// Phase 0 of a tile, one warp: each lane's point (P, from tile_point) into
// shared memory.  Shells that cannot reach the tile's bounding box
// (shell_reaches_box) are culled, from `pre` when a pre-pass worked that
// out (pre != ~0u) or from the box here.  Writes sh.reach, the list of
// shells to visit (kept ones, and culled ones whose staging columns are
// dirty) in `order` order, and resets the work counter and the group mask.
template <typename T, int kLanes>
__device__ __forceinline__ void tile_reach(AOStageSmem<T, kLanes>& sh, const TilePoint<T>& P,
                                           int ns, int lane, unsigned pre) {
  if (P.pv) {
    sh.pt[lane][0] = P.x;
    sh.pt[lane][1] = P.y;
    sh.pt[lane][2] = P.z;
    if constexpr (sizeof(T) != 8) {
      sh.pt_lo[lane][0] = P.lx;
      sh.pt_lo[lane][1] = P.ly;
      sh.pt_lo[lane][2] = P.lz;
    }
  }
  unsigned reach = pre;
  if (pre == ~0u) {
    T lo[3], hi[3];
    warp_box(P.pv, P.x, P.y, P.z, lo, hi);
    const bool keep = lane < ns && shell_reaches_box(lo, hi, sh.nuc[lane][0], sh.nuc[lane][1],
                                                     sh.nuc[lane][2], sh.r2max[lane]);
    reach = __ballot_sync(0xffffffffu, keep);
  }
  bool visit = false;
  int sl = 0;
  if (lane < ns) {
    sl = sh.order[lane];
    visit = ((reach >> sl) & 1u) || sh.dirty[sl];
  }
  const unsigned vm = __ballot_sync(0xffffffffu, visit);
  if (visit) sh.work[__popc(vm & ((1u << lane) - 1u))] = sl;
  if (lane == 0) {
    sh.reach = reach;
    sh.gmask = 0;
    sh.nwork = __popc(vm);
    sh.next = 0;
  }
}

// The 16-AO column groups of a 64-column chunk (one tensor-core k-step
// each) that the columns of a shell of angular momentum l starting at
// column c0 fall in.
__device__ __forceinline__ unsigned shell_group_bits(int c0, int l) {
  const int nc = (l + 1) * (l + 2) / 2;
  const int g0 = c0 >> 4, g1 = (c0 + nc - 1) >> 4;
  return ((2u << g1) - 1u) & ~((1u << g0) - 1u);
}

// Radial sums and every component of shell `sl` at tile point `lane` (valid
// lanes only; the others get zeros), written to the staging tile.  Returns,
// on every lane, whether the S of any lane were nonzero.
template <typename T, int kLanes>
__device__ __forceinline__ bool shell_at_point(AOStageSmem<T, kLanes>& sh, int sl, int lane,
                                               bool valid, T Tthr) {
  using A = Arith<T>;
  T dx = T(0), dy = T(0), dz = T(0), S0 = T(0), S1 = T(0), S2 = T(0);
  if (valid) {
    if constexpr (sizeof(T) == 8) {
      dx = __dsub_rn(sh.pt[lane][0], sh.nuc[sl][0]);
      dy = __dsub_rn(sh.pt[lane][1], sh.nuc[sl][1]);
      dz = __dsub_rn(sh.pt[lane][2], sh.nuc[sl][2]);
    } else {
      // hi parts cancel exactly when close; the residuals restore FP32
      // accuracy of the difference
      dx = (sh.pt[lane][0] - sh.nuc[sl][0]) + (sh.pt_lo[lane][0] - sh.nuc_lo[sl][0]);
      dy = (sh.pt[lane][1] - sh.nuc[sl][1]) + (sh.pt_lo[lane][1] - sh.nuc_lo[sl][1]);
      dz = (sh.pt[lane][2] - sh.nuc[sl][2]) + (sh.pt_lo[lane][2] - sh.nuc_lo[sl][2]);
    }
    const T r2 = A::add(A::add(A::mul(dx, dx), A::mul(dy, dy)), A::mul(dz, dz));
    if (r2 < sh.r2max[sl]) {
      const int k0 = sh.prim0[sl];
      const int k1 = k0 + sh.nprim[sl];
      for (int k = k0; k < k1; ++k) {
        const T gm = sh.g[k];
        const T t = A::mul(gm, r2);
        if (!(t < Tthr)) break;  // ascending exponents: the rest is screened too
        const T ce = sh.c[k] * A::ex(-t);
        S0 += ce;
        S1 += gm * ce;
        S2 += gm * gm * ce;
      }
    }
  }
  const bool nz = S0 != T(0) || S1 != T(0) || S2 != T(0);
  const bool any = __any_sync(0xffffffffu, nz);
  if (any) {
    const int c0 = sh.col[sl];
    T* st = &sh.stage[5 * (lane < kLanes ? lane : kLanes - 1)][c0];
    const T* M = &sh.M[c0];
    switch (sh.lsh[sl]) {
      case 0: shell_components<T, 0>(dx, dy, dz, S0, S1, S2, M, st); break;
      case 1: shell_components<T, 1>(dx, dy, dz, S0, S1, S2, M, st); break;
      case 2: shell_components<T, 2>(dx, dy, dz, S0, S1, S2, M, st); break;
      default: shell_components<T, 3>(dx, dy, dz, S0, S1, S2, M, st); break;
    }
    if (lane == 0) sh.dirty[sl] = 1;
  } else {
    shell_zero_columns(sh, sl, lane);
  }
  return any;
}


}  // namespace qk
