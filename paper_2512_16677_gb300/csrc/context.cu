// context.cu -- the C-ABI context: inputs, device tables, memoisation and
// dispatch of the AO/MO vgl kernels.
//
// Sec. 2.2 of the QMCkl paper: a context holds every input and every cached
// intermediate with its time stamp; setting new electron coordinates bumps
// the stamp and a "get" recomputes only what is out of date.  Here the cached
// intermediate is the AO tensor (the input of the contraction of Eqs. 5-7):
// it is keyed by (time stamp, compute mode, basis version, workspace).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace qk {

cudaError_t DevBuf::ensure(size_t n) {
  if (n <= bytes && p) return cudaSuccess;
  release();
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    p = nullptr;
    bytes = 0;
    return e;
  }
  bytes = n;
  return cudaSuccess;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

static inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
static inline int64_t round_up8(int64_t x) { return (x + 7) / 8 * 8; }

}  // namespace qk

using namespace qk;

// timer classes: 0 = ao_vgl, 1 = contraction, 2 = everything else
static constexpr int kTimerClasses = 3;

struct qk_context_s {
  int device = -1;
  cudaStream_t stream = nullptr;
  std::string err;
  // settings
  int bits = 53;
  double eps = 0.0;  // > 0: explicit cutoff instead of bits
  int mode = QK_FP64;
  bool fused = false;  // split-bf16: AO blocks built inside the contraction kernel
  bool spatial = true;  // tensor-core modes: tiles cut from a spatial point order
  bool sm_pairs = true;  // tensor-core modes: contraction on pairs of SMs (cta_group::2)
  uint64_t basis_version = 1;
  // nuclei
  int64_t nucl_num = 0;
  std::vector<double> nucl_charge, nucl_coord;
  float nbox_lo[3] = {0, 0, 0}, nbox_hi[3] = {0, 0, 0};  // nuclear box with a margin
  // basis, primitives sorted by ascending exponent inside each shell
  bool has_basis = false;
  int64_t shell_num = 0, prim_num = 0, ao_num = 0;
  std::vector<int> shell_nuc, shell_l, shell_prim0, shell_nprim, shell_ao0, ao_shell;
  std::vector<double> prim_g, prim_c, ao_fac, shell_gmin;
  std::vector<int4> chunks;
  // internal shell order: 0 = chosen from the nuclei (default), 1 = the
  // caller's, 2 = spatial; ao_caller[internal AO] = the caller's AO index
  int order_mode = 0;
  std::vector<int64_t> shell_perm;  // caller's shell at each internal position
  bool order_spatial = false;   // nuclei taken in Morton order
  bool order_permuted = false;  // internal shell order differs from the caller's
  std::vector<int> ao_caller;
  DevBuf d_tables;
  BasisDev bdev{};
  bool tables_dirty = true;
  // MO coefficients
  bool has_mo = false;
  int64_t mo_num = 0, ldc = 0;
  std::vector<double> mo_coef;
  DevBuf d_mo;
  double* c64 = nullptr;   // [mo][ao]     dense (adjoint)
  float* c32 = nullptr;    // [mo][ldc]    dense (adjoint)
  double* c64p = nullptr;  // [mo][kpad]   chunked column layout (contraction)
  float* c32p = nullptr;
  __nv_bfloat16* c_hi = nullptr;
  __nv_bfloat16* c_lo = nullptr;
  int64_t kpad = 0;
  bool mo_dirty = true;
  // points
  bool has_points = false;
  int64_t walk_num = 0, elec_num = 0, point_num = 0;
  uint64_t date = 0;
  DevBuf d_points, d_raw;
  PointsDev pdev{};
  // spatial order of the current points (tensor-core modes)
  DevBuf d_sort;
  int32_t* perm = nullptr;
  PointsDev psort{};
  uint64_t sort_date = ~0ull;
  // workspace and memo
  void* ws_user = nullptr;
  size_t ws_user_bytes = 0;
  DevBuf ws_own;
  uint64_t ao_date = ~0ull, ao_version = 0;
  uint64_t fused_date = ~0ull;             // time stamp of the last fused evaluation
  unsigned char* fused_lists = nullptr;    // its live-chunk lists
  int ao_mode = -1;
  void* ao_ws = nullptr;
  bool ao_sorted = false;
  bool ao_pairs = false;  // the AO tensor holds the zeros a pair contraction reads
  bool ao_zeroed = false;  // its dead groups of live blocks hold zeros (adjoint)
  // host-output staging, device error word, backward scratch
  DevBuf d_out;
  cudaStream_t copy_stream = nullptr;   // device -> host copies of output ranges
  // MO cusp correction (Sec. 3.3)
  bool cusp_on = false;
  bool cusp_dirty = true;
  std::vector<double> cusp_rc;
  uint64_t cusp_basis = 0, cusp_mo = 0;
  DevBuf d_cusp;
  DevBuf d_cusp_list;  // points inside a sphere, per MO call
  DevBuf d_dens;       // density: occupied-MO tables, weights, partial sums
  // single-electron moves: proposed positions of electron single_elec of
  // every walker, and the AO tensor at them
  DevBuf d_single, d_single_ws, d_single_ct;
  uint64_t single_ct_version = ~0ull;  // C^T for single moves, per upload of C
  bool single_ct_f64 = false;
  PointsDev psingle{};
  int64_t single_elec = -1;
  CuspDev cudev{};
  double* cusp_f64 = nullptr;
  float* cusp_f32 = nullptr;
  uint64_t mo_version = 0;  // bumped by every upload of C
  DevBuf d_ct;              // C^T bf16 hi/lo planes (chunked order) for the split-bf16 adjoint
  uint64_t ct_version = ~0ull;
  // C blocked for the pair contraction (per upload of C, tile width and mode)
  DevBuf d_cpair;
  uint64_t cpair_version = ~0ull;
  int cpair_bn = 0, cpair_half = 0, cpair_mode = -1;
  std::vector<cudaEvent_t> range_done;  // one per output range of a host call
  DevBuf d_flag;
  DevBuf bwd_own;
  // optional per-kernel-class timing with events on the context's stream
  bool timing = false;
  int64_t kernels = 0;  // kernel launches of the timed classes since the last read
  std::vector<cudaEvent_t> ev_start[kTimerClasses], ev_stop[kTimerClasses];
  size_t ev_used[kTimerClasses] = {0, 0, 0};
  ~qk_context_s() {
    for (auto e : range_done) cudaEventDestroy(e);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    for (int k = 0; k < kTimerClasses; ++k) {
      for (auto e : ev_start[k]) cudaEventDestroy(e);
      for (auto e : ev_stop[k]) cudaEventDestroy(e);
    }
  }
};

namespace {

qk_status fail(qk_context c, qk_status code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

qk_status cuda_fail(qk_context c, cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky launch error so later calls start clean
  if (e == cudaErrorMemoryAllocation)
    return fail(c, QK_ERR_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorNotSupported)
    return fail(c, QK_ERR_NOT_IMPLEMENTED, "%s: not supported on this device", what);
  return fail(c, QK_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CHECK_CTX(c) \
  if (!(c)) return QK_ERR_NULL_POINTER

// Event pair around one launch of class k (no-op unless timing is on).
struct TimedLaunch {
  qk_context c;
  int k;
  bool on;
  // nk: kernels the wrapped call launches (counted whether or not timing is on)
  TimedLaunch(qk_context c_, int k_, int nk = 1) : c(c_), k(k_), on(c_->timing) {
    c->kernels += nk;
    if (!on) return;
    size_t i = c->ev_used[k];
    if (i == c->ev_start[k].size()) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        on = false;
        return;
      }
      c->ev_start[k].push_back(a);
      c->ev_stop[k].push_back(b);
    }
    cudaEventRecord(c->ev_start[k][i], c->stream);
  }
  ~TimedLaunch() {
    if (!on) return;
    cudaEventRecord(c->ev_stop[k][c->ev_used[k]], c->stream);
    c->ev_used[k]++;
  }
};

double threshold(const qk_context c) {
  if (c->eps > 0.0) return -std::log(c->eps);
  return (double)(c->bits - 1) * std::log(2.0);
}

// Internal shell order.  AO chunks are cut from consecutive shells, and
// the contraction skips (tile, chunk) blocks and 16-AO column groups that
// hold no entry surviving Eq. 3, so the shells that share a column group
// should reach the same points: nearby nuclei, and similar screening radii
// (r^2 < T / gamma_min).
//  - Nuclei: bases listed along a chain or molecule by molecule already
//    are in a spatial order; bases listed in random atom order are not.
//    Spatial order: nuclei ranked by the Morton code of a 1024^3 grid over
//    their box, a nucleus's shells keep the caller's order.  The default
//    takes it when the path through the nuclei in shell order gets shorter
//    than 0.7 of the caller's.
//  - Radii: the shells are then split, stably, into a compact class
//    (gamma_min at least that of the AO-weighted median shell) followed by
//    a diffuse class.  A diffuse shell reaches far, so a column group that
//    mixes one with compact shells is live wherever the diffuse one is;
//    the split is threshold-free because r^2 scales with 1 / gamma_min for
//    every shell alike.
// Mode 1 keeps the caller's order as it is.
std::vector<int64_t> nucleus_order(qk_context c, int64_t S, const int64_t* shell_nucleus) {
  std::vector<int64_t> caller(S);
  std::iota(caller.begin(), caller.end(), 0);
  if (S < 2) return caller;
  const int64_t NN = c->nucl_num;
  const double* R = c->nucl_coord.data();
  double lo[3], hi[3];
  for (int k = 0; k < 3; ++k) {
    lo[k] = hi[k] = R[k];
    for (int64_t a = 1; a < NN; ++a) {
      lo[k] = std::min(lo[k], R[3 * a + k]);
      hi[k] = std::max(hi[k], R[3 * a + k]);
    }
  }
  auto spread = [](uint64_t v) {
    uint64_t r = 0;
    for (int i = 0; i < 10; ++i) r |= ((v >> i) & 1ull) << (3 * i);
    return r;
  };
  std::vector<uint64_t> key(NN);
  for (int64_t a = 0; a < NN; ++a) {
    uint64_t q[3];
    for (int k = 0; k < 3; ++k) {
      const double span = hi[k] - lo[k];
      const double f = span > 0 ? (R[3 * a + k] - lo[k]) / span * 1023.0 : 0.0;
      q[k] = (uint64_t)std::min(1023.0, std::max(0.0, f));
    }
    key[a] = spread(q[0]) | (spread(q[1]) << 1) | (spread(q[2]) << 2);
  }
  std::vector<int64_t> spatial(caller);
  std::stable_sort(spatial.begin(), spatial.end(), [&](int64_t x, int64_t y) {
    const int64_t ax = shell_nucleus[x], ay = shell_nucleus[y];
    return key[ax] != key[ay] ? key[ax] < key[ay] : ax < ay;
  });
  if (c->order_mode == 2) return spatial;
  auto path = [&](const std::vector<int64_t>& o) {
    double L = 0.0;
    for (int64_t i = 1; i < S; ++i) {
      const int64_t a = shell_nucleus[o[i - 1]], b = shell_nucleus[o[i]];
      if (a == b) continue;
      const double dx = R[3 * a] - R[3 * b], dy = R[3 * a + 1] - R[3 * b + 1],
                   dz = R[3 * a + 2] - R[3 * b + 2];
      L += std::sqrt(dx * dx + dy * dy + dz * dz);
    }
    return L;
  };
  return path(spatial) < 0.7 * path(caller) ? spatial : caller;
}

// *morton: the nuclei were taken in Morton order.
std::vector<int64_t> shell_order(qk_context c, int64_t S, const int64_t* shell_nucleus,
                                 const int32_t* shell_ang_mom, const int64_t* shell_prim_num,
                                 const double* exponent, bool* morton) {
  std::vector<int64_t> order(S);
  std::iota(order.begin(), order.end(), 0);
  *morton = false;
  if (c->order_mode == 1 || S < 2) return order;
  order = nucleus_order(c, S, shell_nucleus);
  for (int64_t i = 0; i < S; ++i)
    if (order[i] != i) *morton = true;
  std::vector<double> gmin(S);
  int64_t p = 0, na = 0;
  for (int64_t s = 0; s < S; ++s) {
    gmin[s] = exponent[p];
    for (int64_t k = 1; k < shell_prim_num[s]; ++k) gmin[s] = std::min(gmin[s], exponent[p + k]);
    p += shell_prim_num[s];
    na += (shell_ang_mom[s] + 1) * (shell_ang_mom[s] + 2) / 2;
  }
  // gamma_min of the shell that holds the middle AO, shells by descending gamma_min
  std::vector<int64_t> by_g(S);
  std::iota(by_g.begin(), by_g.end(), 0);
  std::stable_sort(by_g.begin(), by_g.end(),
                   [&](int64_t x, int64_t y) { return gmin[x] > gmin[y]; });
  double gmed = gmin[by_g[0]];
  for (int64_t i = 0, a = 0; i < S; ++i) {
    a += (shell_ang_mom[by_g[i]] + 1) * (shell_ang_mom[by_g[i]] + 2) / 2;
    if (2 * a >= na) {
      gmed = gmin[by_g[i]];
      break;
    }
  }
  std::stable_partition(order.begin(), order.end(),
                        [&](int64_t s) { return gmin[s] >= gmed; });
  return order;
}

qk_status ensure_tables(qk_context c) {
  if (!c->tables_dirty) return QK_SUCCESS;
  const double T = threshold(c);
  const int S = (int)c->shell_num, NP = (int)c->prim_num, NA = (int)c->ao_num,
            NN = (int)c->nucl_num, NC = (int)c->chunks.size();
  std::vector<double> r2(S);
  std::vector<float> r2f(S), gf(NP), cf(NP), af(NA), nhi(3 * NN), nlo(3 * NN);
  std::vector<int> sch(S);
  for (int q = 0; q < NC; ++q)
    for (int sh = c->chunks[q].x; sh < c->chunks[q].y; ++sh) sch[sh] = q;
  for (int s = 0; s < S; ++s) {
    // any r^2 >= r2[s] gives fl(gamma_min r^2) > T, so no primitive would pass
    r2[s] = std::isinf(T) ? INFINITY : T / c->shell_gmin[s] * (1.0 + 1e-13);
    r2f[s] = std::isinf(T) ? INFINITY : std::nextafter((float)r2[s], INFINITY) * (1.0f + 1e-6f);
  }
  for (int k = 0; k < NP; ++k) {
    gf[k] = (float)c->prim_g[k];
    cf[k] = (float)c->prim_c[k];
  }
  for (int k = 0; k < NA; ++k) af[k] = (float)c->ao_fac[k];
  for (int k = 0; k < 3 * NN; ++k) {
    nhi[k] = (float)c->nucl_coord[k];
    nlo[k] = (float)(c->nucl_coord[k] - (double)nhi[k]);
  }
  // pack everything into one allocation, 256-byte aligned pieces
  struct Piece {
    const void* src;
    size_t bytes;
    size_t off;
  };
  std::vector<Piece> pieces = {
      {c->nucl_coord.data(), sizeof(double) * 3 * NN, 0},
      {nhi.data(), sizeof(float) * 3 * NN, 0},
      {nlo.data(), sizeof(float) * 3 * NN, 0},
      {c->shell_nuc.data(), sizeof(int) * S, 0},
      {c->shell_l.data(), sizeof(int) * S, 0},
      {c->shell_prim0.data(), sizeof(int) * S, 0},
      {c->shell_nprim.data(), sizeof(int) * S, 0},
      {c->shell_ao0.data(), sizeof(int) * S, 0},
      {r2.data(), sizeof(double) * S, 0},
      {r2f.data(), sizeof(float) * S, 0},
      {c->prim_g.data(), sizeof(double) * NP, 0},
      {c->prim_c.data(), sizeof(double) * NP, 0},
      {gf.data(), sizeof(float) * NP, 0},
      {cf.data(), sizeof(float) * NP, 0},
      {c->ao_fac.data(), sizeof(double) * NA, 0},
      {af.data(), sizeof(float) * NA, 0},
      {c->ao_shell.data(), sizeof(int) * NA, 0},
      {c->chunks.data(), sizeof(int4) * NC, 0},
      {sch.data(), sizeof(int) * S, 0},
      {c->ao_caller.data(), sizeof(int) * NA, 0},
  };
  size_t total = 0;
  for (auto& p : pieces) {
    p.off = total;
    total = align_up(total + p.bytes, 256);
  }
  std::vector<unsigned char> host(total, 0);
  for (auto& p : pieces)
    if (p.bytes) std::memcpy(host.data() + p.off, p.src, p.bytes);
  cudaError_t e = c->d_tables.ensure(total);
  if (e != cudaSuccess) return cuda_fail(c, e, "basis tables");
  e = cudaMemcpy(c->d_tables.p, host.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "basis tables upload");
  auto at = [&](int i) { return (void*)((unsigned char*)c->d_tables.p + pieces[i].off); };
  BasisDev& b = c->bdev;
  b.nucl_num = NN;
  b.shell_num = S;
  b.ao_num = NA;
  b.prim_num = NP;
  b.nchunk = NC;
  b.nucl_xyz = (const double*)at(0);
  b.nucl_hi = (const float*)at(1);
  b.nucl_lo = (const float*)at(2);
  b.shell_nuc = (const int*)at(3);
  b.shell_l = (const int*)at(4);
  b.shell_prim0 = (const int*)at(5);
  b.shell_nprim = (const int*)at(6);
  b.shell_ao0 = (const int*)at(7);
  b.shell_r2 = (const double*)at(8);
  b.shell_r2_f = (const float*)at(9);
  b.prim_g = (const double*)at(10);
  b.prim_c = (const double*)at(11);
  b.prim_g_f = (const float*)at(12);
  b.prim_c_f = (const float*)at(13);
  b.ao_fac = (const double*)at(14);
  b.ao_fac_f = (const float*)at(15);
  b.ao_shell = (const int*)at(16);
  b.chunk = (const int4*)at(17);
  b.shell_chunk = (const int*)at(18);
  b.ao_caller = c->order_permuted ? (const int*)at(19) : nullptr;
  b.T = T;
  b.T_f = std::isinf(T) ? INFINITY : (float)T;
  c->tables_dirty = false;
  return QK_SUCCESS;
}

qk_status ensure_mo(qk_context c) {
  if (!c->mo_dirty) return QK_SUCCESS;
  qk_status st = ensure_tables(c);  // the chunk table defines the padded layout
  if (st) return st;
  const int64_t nm = c->mo_num, na = c->ao_num, ldc = round_up8(na);
  const int64_t kp = (int64_t)c->chunks.size() * kChunkAO;
  const size_t b64 = align_up(sizeof(double) * nm * na, 256);
  const size_t b32 = align_up(sizeof(float) * nm * ldc, 256);
  const size_t b64p = align_up(sizeof(double) * nm * kp, 256);
  const size_t b32p = align_up(sizeof(float) * nm * kp, 256);
  const size_t b16 = align_up(sizeof(__nv_bfloat16) * nm * kp, 256);
  cudaError_t e = c->d_mo.ensure(b64 + b32 + b64p + b32p + 2 * b16);
  if (e != cudaSuccess) return cuda_fail(c, e, "MO coefficient tables");
  unsigned char* base = (unsigned char*)c->d_mo.p;
  c->c64 = (double*)base;
  c->c32 = (float*)(base + b64);
  c->c64p = (double*)(base + b64 + b32);
  c->c32p = (float*)(base + b64 + b32 + b64p);
  c->c_hi = (__nv_bfloat16*)(base + b64 + b32 + b64p + b32p);
  c->c_lo = (__nv_bfloat16*)(base + b64 + b32 + b64p + b32p + b16);
  c->ldc = ldc;
  c->kpad = kp;
  // C in the internal AO order (columns follow ao_caller)
  std::vector<double> cint;
  const double* csrc = c->mo_coef.data();
  if (c->order_permuted) {
    cint.resize((size_t)nm * na);
    for (int64_t i = 0; i < nm; ++i)
      for (int64_t a = 0; a < na; ++a) cint[i * na + a] = c->mo_coef[i * na + c->ao_caller[a]];
    csrc = cint.data();
  }
  e = cudaMemcpyAsync(c->c64, csrc, sizeof(double) * nm * na, cudaMemcpyHostToDevice,
                      c->stream);
  if (e == cudaSuccess) e = launch_to_f32(c->c64, nm, na, ldc, c->c32, c->stream);
  if (e == cudaSuccess)
    e = launch_mo_chunked(c->c64, nm, na, c->bdev.chunk, c->bdev.nchunk, c->c64p, c->c32p,
                          c->c_hi, c->c_lo, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "MO coefficient upload");
  c->mo_dirty = false;
  c->mo_version++;
  return QK_SUCCESS;
}

// The cusp coefficients of the current basis, C and radii (FP64 set-up on
// the device, once per change).
qk_status ensure_cusp(qk_context c) {
  if (!c->cusp_on) return QK_SUCCESS;
  qk_status st = ensure_tables(c);
  if (st) return st;
  st = ensure_mo(c);
  if (st) return st;
  if (!c->cusp_dirty && c->cusp_basis == c->basis_version && c->cusp_mo == c->mo_version)
    return QK_SUCCESS;
  const int64_t nn = c->nucl_num, nm = c->mo_num, na = c->ao_num;
  std::vector<int> start(nn + 1, 0), list;
  for (int64_t A = 0; A < nn; ++A) {
    start[A] = (int)list.size();
    for (int64_t s = 0; s < c->shell_num; ++s)
      if (c->shell_nuc[s] == A && c->shell_l[s] == 0) list.push_back((int)s);
    if ((int)list.size() - start[A] > 32)
      return fail(c, QK_ERR_NOT_IMPLEMENTED, "cusp correction: more than 32 s shells on a nucleus");
  }
  start[nn] = (int)list.size();
  if (list.empty()) list.push_back(0);
  const size_t b_rc = align_up(sizeof(double) * nn, 256);
  const size_t b_rf = align_up(sizeof(float) * nn, 256);
  const size_t b_st = align_up(sizeof(int) * (nn + 1), 256);
  const size_t b_ls = align_up(sizeof(int) * list.size(), 256);
  const size_t b_x = align_up(sizeof(double) * nn * na, 256);
  const size_t b_q = align_up(sizeof(double) * nn * nm, 256);
  const size_t b_f = align_up(sizeof(double) * nn * nm * 4, 256);
  const size_t b_g = align_up(sizeof(float) * nn * nm * 4, 256);
  cudaError_t e = c->d_cusp.ensure(2 * b_rc + b_st + b_ls + b_x + b_q + b_f + b_g + b_rf);
  if (e != cudaSuccess) return cuda_fail(c, e, "cusp tables");
  unsigned char* p = (unsigned char*)c->d_cusp.p;
  double* rc = (double*)p;
  double* charge = (double*)(p + b_rc);
  int* dstart = (int*)(p + 2 * b_rc);
  int* dlist = (int*)(p + 2 * b_rc + b_st);
  double* X = (double*)(p + 2 * b_rc + b_st + b_ls);
  double* Q = (double*)((unsigned char*)X + b_x);
  c->cusp_f64 = (double*)((unsigned char*)Q + b_q);
  c->cusp_f32 = (float*)((unsigned char*)c->cusp_f64 + b_f);
  c->cudev.rc_f = (float*)((unsigned char*)c->cusp_f32 + b_g);
  c->cudev.rc = rc;
  c->cudev.charge = charge;
  c->cudev.s_start = dstart;
  c->cudev.s_shell = dlist;
  e = cudaMemcpyAsync(rc, c->cusp_rc.data(), sizeof(double) * nn, cudaMemcpyHostToDevice,
                      c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(charge, c->nucl_charge.data(), sizeof(double) * nn,
                        cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dstart, start.data(), sizeof(int) * (nn + 1), cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dlist, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess)
    e = launch_cusp_setup(c->bdev, c->cudev, nm, c->c64, X, Q, c->cusp_f64, c->cusp_f32,
                          c->stream);
  // the host vectors above must outlive the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cusp set-up");
  c->cusp_dirty = false;
  c->cusp_basis = c->basis_version;
  c->cusp_mo = c->mo_version;
  return QK_SUCCESS;
}

// Adds the cusp correction to MO rows D of the points p (caller's order).
// The cusp correction on D at points p; `whole`: p are the context's current
// points, whose spatial order (when they have one) the sphere search walks.
qk_status apply_cusp(qk_context c, const PointsDev& p, void* D, bool whole = false) {
  if (!c->cusp_on) return QK_SUCCESS;
  cudaError_t e = c->d_cusp_list.ensure(cusp_list_bytes(p.n));
  if (e != cudaSuccess) return cuda_fail(c, e, "cusp point list");
  const bool sorted = whole && c->perm && c->sort_date == c->date && c->psort.n == p.n;
  {
    TimedLaunch t(c, 2, 2);
    e = launch_cusp_apply(c->bdev, c->cudev, p, sorted ? &c->psort : nullptr,
                          sorted ? c->perm : nullptr, c->mo_num, c->c64, c->c32, c->ldc,
                          c->cusp_f64, c->cusp_f32, c->mode == QK_FP64, D, c->d_cusp_list.p,
                          c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "cusp correction");
  return QK_SUCCESS;
}

// Columns of the contraction's AO tensor: one 64-wide window per chunk.
int64_t kpad_of(qk_context c) { return (int64_t)c->chunks.size() * kChunkAO; }

// Tensor-core modes use the tiled layout: kTilePoints points per 128-row
// tile, plus one live-block byte per (tile, chunk).
bool tiled_mode(int mode) { return mode == QK_BF16X3 || mode == QK_TF32; }
// The MO vgl AO tensor is tiled and block-sparse in the tensor-core modes and
// in FP64 (whose contraction multiplies live column groups only); the plain
// FP32 path keeps the dense layout.
bool vgl_tiled(int mode) { return tiled_mode(mode) || mode == QK_FP64; }
size_t ao_elem_bytes(int mode) {
  return mode == QK_FP64 ? sizeof(double)
                         : (mode == QK_BF16X3 ? sizeof(__nv_bfloat16) : sizeof(float));
}
int64_t ao_tiles(qk_context c) { return (c->point_num + kTilePoints - 1) / kTilePoints; }

bool use_fused(qk_context c) { return c->mode == QK_BF16X3 && c->fused; }

size_t ao_tensor_bytes(qk_context c, int mode) {
  const size_t ld = (size_t)kpad_of(c);
  if (vgl_tiled(mode)) {
    const size_t rows = (size_t)ao_tiles(c) * kTileRows;
    const size_t mask = align_up((size_t)ao_tiles(c) * mask_ld((int)c->chunks.size()), 256) +
                        align_up((size_t)ao_tiles(c) * c->chunks.size() * sizeof(uint32_t), 256);
    const size_t planes = mode == QK_BF16X3 ? 2 : 1;
    return planes * align_up(rows * ld * ao_elem_bytes(mode), 256) + mask;
  }
  const size_t rows = (size_t)5 * c->point_num;
  if (mode == QK_FP64) return align_up(rows * ld * sizeof(double), 256);
  return align_up(rows * ld * sizeof(float), 256);
}

// Bind the context to the current device on first use; allocate the
// device error word.
qk_status ensure_device(qk_context c) {
  if (c->device >= 0) return QK_SUCCESS;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = c->d_flag.ensure(256);
  if (e == cudaSuccess) e = cudaMemset(c->d_flag.p, 0, 256);
  if (e != cudaSuccess) return cuda_fail(c, e, "no usable CUDA device");
  c->device = dev;
  return QK_SUCCESS;
}

qk_status require(qk_context c, bool need_mo) {
  if (c->nucl_num == 0) return fail(c, QK_ERR_NOT_PROVIDED, "nuclei not set");
  if (!c->has_basis) return fail(c, QK_ERR_NOT_PROVIDED, "AO basis not set");
  if (need_mo && !c->has_mo) return fail(c, QK_ERR_NOT_PROVIDED, "MO coefficients not set");
  if (!c->has_points) return fail(c, QK_ERR_NOT_PROVIDED, "points not set");
  return ensure_device(c);
}

// Pointer to a workspace of at least `need` bytes (caller's or the library's).
qk_status workspace(qk_context c, size_t need, void** out) {
  if (c->ws_user) {
    if (c->ws_user_bytes < need)
      return fail(c, QK_ERR_BAD_SIZE, "workspace holds %zu bytes, %zu needed", c->ws_user_bytes,
                  need);
    *out = c->ws_user;
    return QK_SUCCESS;
  }
  cudaError_t e = c->ws_own.ensure(need);
  if (e != cudaSuccess) return cuda_fail(c, e, "workspace");
  *out = c->ws_own.p;
  return QK_SUCCESS;
}

AOTensor ao_view(qk_context c, void* ws, int mode) {
  AOTensor t{};
  t.ld = kpad_of(c);
  t.chunked = true;
  t.nchunk = (int)c->chunks.size();
  t.a = ws;
  if (vgl_tiled(mode)) {
    t.tiled = true;
    t.blocked = true;
    t.rows = ao_tiles(c) * kTileRows;
    const size_t es = ao_elem_bytes(mode);
    const size_t plane = align_up((size_t)t.rows * t.ld * es, 256);
    unsigned char* p = (unsigned char*)ws + plane;
    if (mode == QK_BF16X3) {
      t.a_lo = (unsigned char*)ws + kBlockElems * es;  // planes interleave by block
      p += plane;
    }
    t.mask = p;
    t.reach = (uint32_t*)(p + align_up((size_t)ao_tiles(c) * mask_ld(t.nchunk), 256));
  } else {
    t.rows = 5 * c->point_num;
  }
  return t;
}

// The AO tensor's place in the workspace; *valid says whether it already
// holds the current date/mode/basis.
qk_status ao_workspace(qk_context c, AOTensor* out, bool* valid, bool sorted) {
  qk_status st = ensure_tables(c);
  if (st) return st;
  void* ws = nullptr;
  st = workspace(c, ao_tensor_bytes(c, c->mode), &ws);
  if (st) return st;
  *out = ao_view(c, ws, c->mode);
  if (sorted) out->perm = c->perm;
  out->pair_zero = tiled_mode(c->mode) && out->tiled && out->reach != nullptr && c->sm_pairs;
  *valid = c->ao_date == c->date && c->ao_mode == c->mode && c->ao_ws == ws &&
           c->ao_version == c->basis_version && c->ao_sorted == sorted &&
           c->ao_pairs == out->pair_zero;
  return QK_SUCCESS;
}

void mark_ao(qk_context c, const AOTensor& ao, bool sorted) {
  c->ao_date = c->date;
  c->ao_mode = c->mode;
  c->ao_ws = ao.a;
  c->ao_version = c->basis_version;
  c->ao_sorted = sorted;
  c->ao_pairs = ao.pair_zero;
  c->ao_zeroed = false;
}

// Whether the device path cuts its tiles from a spatial point order.
bool use_spatial(qk_context c) {
  return vgl_tiled(c->mode) && c->spatial && c->point_num >= 2 * kTilePoints;
}

// The spatial order of the current points (once per time stamp).
qk_status ensure_spatial(qk_context c) {
  if (c->sort_date == c->date) return QK_SUCCESS;
  cudaError_t e = c->d_sort.ensure(spatial_order_bytes(c->point_num));
  if (e != cudaSuccess) return cuda_fail(c, e, "spatial order scratch");
  {
    TimedLaunch t(c, 2, spatial_order_kernels(c->point_num));
    e = launch_spatial_order(c->pdev, c->nbox_lo, c->nbox_hi, c->d_sort.p, &c->perm, &c->psort,
                             c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "spatial order");
  c->sort_date = c->date;
  return QK_SUCCESS;
}

// Points [p0, p1) and the matching rows of the AO tensor (p0 a multiple of
// the layout's point tile).
PointsDev points_range(const PointsDev& p, int64_t p0, int64_t p1) {
  PointsDev v = p;
  v.n = p1 - p0;
  v.x += p0;
  v.y += p0;
  v.z += p0;
  v.hi += p0;
  v.lo += p0;
  return v;
}

AOTensor ao_range(const AOTensor& t, int mode, int64_t p0, int64_t p1) {
  AOTensor v = t;
  const size_t es = ao_elem_bytes(mode);
  if (t.tiled) {
    const int64_t t0 = p0 / kTilePoints;
    v.rows = (p1 - p0 + kTilePoints - 1) / kTilePoints * kTileRows;
    v.mask = t.mask + t0 * mask_ld(t.nchunk);
    if (t.reach) v.reach = t.reach + t0 * t.nchunk;
    // the blocks of tile t0 onwards (both planes in each block)
    const size_t off = (size_t)blocked_offset(t0, 0, t.nchunk, t.a_lo ? 2 : 1, 0, 0, 0, (int)es);
    v.a = (unsigned char*)t.a + off * es;
    if (t.a_lo) v.a_lo = (unsigned char*)v.a + kBlockElems * es;
    return v;
  }
  const int64_t r0 = 5 * p0;
  v.rows = 5 * (p1 - p0);
  v.a = (unsigned char*)t.a + (size_t)r0 * t.ld * es;
  if (t.a_lo) v.a_lo = (unsigned char*)t.a_lo + (size_t)r0 * t.ld * es;
  return v;
}

// Make the AO tensor of the current date/mode valid in the workspace.
qk_status provide_ao(qk_context c, AOTensor* out) {
  const bool sorted = use_spatial(c);
  if (sorted) {
    qk_status st = ensure_spatial(c);
    if (st) return st;
  }
  bool valid = false;
  qk_status st = ao_workspace(c, out, &valid, sorted);
  if (st || valid) return st;
  cudaError_t e;
  {
    TimedLaunch t(c, 0, out->tiled && out->reach ? 2 : 1);  // reach pre-pass + ao_vgl
    e = launch_ao_vgl(c->bdev, sorted ? c->psort : c->pdev, c->mode, *out, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "ao_vgl launch");
  mark_ao(c, *out, sorted);
  return QK_SUCCESS;
}

// D[M][mo] = AO rows . C^T for the AO rows of `ao` (M = 5 x its points).
qk_status contract(qk_context c, const AOTensor& ao, int64_t M, void* dout) {
  const int64_t N = c->mo_num;
  const int64_t KP = c->kpad;  // the contraction runs over the chunked columns
  cudaError_t e = cudaSuccess;
  TimedLaunch timer(c, 1);
  switch (c->mode) {
    case QK_FP64:
      if (ao.tiled)  // live 16-AO column groups only (Sec. 3.2's sparse product)
        e = launch_mo_sparse64(ao, c->c64p, KP, N, (double*)dout, M, c->stream);
      else
        e = launch_gemm_f64(M, N, KP, (const double*)ao.a, ao.ld, 1, c->c64p, KP, 1,
                            (double*)dout, N, 1, c->stream);
      break;
    case QK_FP32:
      e = launch_gemm_f32(M, N, KP, (const float*)ao.a, ao.ld, 1, c->c32p, KP, 1, (float*)dout,
                          N, 1, c->stream);
      break;
    default: {
      const bool split = c->mode == QK_BF16X3;
      const void* b_hi = split ? (const void*)c->c_hi : (const void*)c->c32p;
      const void* b_lo = split ? (const void*)c->c_lo : nullptr;
      const TcConfig cfg = tc_default_config(c->mode, N);
      if (ao.pair_zero && cfg.bn >= 64 && cfg.bn % 32 == 0) {
        const void* cblk = nullptr;
        qk_status st = context_pair_c(c, cfg.bn, cfg.bn / 2, &cblk);
        if (st) return st;
        e = launch_mo_tc_pair(c->mode, ao, KP, cblk, N, (float*)dout, cfg.bn,
                              (int*)c->d_flag.p, c->stream, M);
      } else
        e = launch_mo_tc(c->mode, ao, KP, b_hi, b_lo, KP, N, (float*)dout, cfg,
                         (int*)c->d_flag.p, c->stream, M);
    }
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "mo_vgl contraction");
  return QK_SUCCESS;
}

// Output ranges of a host-memory MO call: enough points per range for full
// launches, at most 8 ranges, each a multiple of 800 points (whole 25- and
// 32-point tiles, so every range sees the tiles of the one-launch path).
constexpr int64_t kRangeQuantum = 800;
constexpr int64_t kMinRangePoints = 9600;
int64_t host_range_points(qk_context c) {
  int64_t parts = c->point_num / kMinRangePoints;
  if (parts > 8) parts = 8;
  if (parts < 2) return c->point_num;
  const int64_t per = (c->point_num + parts - 1) / parts;
  return (per + kRangeQuantum - 1) / kRangeQuantum * kRangeQuantum;
}

void invalidate(qk_context c) {
  c->basis_version++;
  c->tables_dirty = true;
}

qk_status set_points_common(qk_context c, char transp, int64_t walk_num, int64_t elec_num) {
  if (transp != 'N' && transp != 'T')
    return fail(c, QK_ERR_INVALID_ARG, "transp must be 'N' or 'T'");
  if (walk_num < 1 || elec_num < 1)
    return fail(c, QK_ERR_BAD_SIZE, "walk_num and elec_num must be >= 1");
  qk_status st = ensure_device(c);
  if (st) return st;
  const int64_t n = walk_num * elec_num;
  cudaError_t e = c->d_points.ensure(align_up(sizeof(double) * 3 * n, 256) +
                                     align_up(sizeof(float) * 6 * n, 256));
  if (e != cudaSuccess) return cuda_fail(c, e, "point buffers");
  double* base = (double*)c->d_points.p;
  c->pdev.n = n;
  c->pdev.x = base;
  c->pdev.y = base + n;
  c->pdev.z = base + 2 * n;
  float* fb = (float*)((unsigned char*)c->d_points.p + align_up(sizeof(double) * 3 * n, 256));
  c->pdev.hi = fb;
  c->pdev.lo = fb + 3 * n;
  c->pdev.ld = n;
  c->walk_num = walk_num;
  c->elec_num = elec_num;
  c->point_num = n;
  return QK_SUCCESS;
}

}  // namespace

extern "C" {

qk_status qk_context_create(qk_context* out) {
  if (!out) return QK_ERR_NULL_POINTER;
  qk_context c = new (std::nothrow) qk_context_s();
  if (!c) return QK_ERR_OUT_OF_MEMORY;
  // the device is bound at the first call that touches it, so that the
  // host-side setters and their validation work without a GPU
  *out = c;
  return QK_SUCCESS;
}

qk_status qk_context_destroy(qk_context c) {
  CHECK_CTX(c);
  delete c;
  return QK_SUCCESS;
}

qk_status qk_last_error(qk_context c, char* buf, int64_t size) {
  CHECK_CTX(c);
  if (!buf) return QK_ERR_NULL_POINTER;
  if (size < 1) return QK_ERR_BAD_SIZE;
  const size_t n = std::min((size_t)(size - 1), c->err.size());
  std::memcpy(buf, c->err.data(), n);
  buf[n] = '\0';
  return QK_SUCCESS;
}

qk_status qk_set_precision(qk_context c, int32_t bits) {
  CHECK_CTX(c);
  if (bits < 2 || bits > 53) return fail(c, QK_ERR_INVALID_ARG, "bits must be in [2, 53]");
  c->bits = bits;
  c->eps = 0.0;
  invalidate(c);
  return QK_SUCCESS;
}

qk_status qk_set_cutoff(qk_context c, double eps) {
  CHECK_CTX(c);
  if (!(eps > 0.0 && eps < 1.0)) return fail(c, QK_ERR_INVALID_ARG, "eps must be in (0, 1)");
  c->eps = eps;
  invalidate(c);
  return QK_SUCCESS;
}

qk_status qk_set_compute_mode(qk_context c, int32_t mode) {
  CHECK_CTX(c);
  if (mode != QK_FP64 && mode != QK_FP32 && mode != QK_BF16X3 && mode != QK_TF32)
    return fail(c, QK_ERR_INVALID_ARG, "unknown compute mode %d", mode);
  c->mode = mode;
  return QK_SUCCESS;
}

qk_status qk_set_nucleus(qk_context c, int64_t nucl_num, const double* charge,
                         const double* coord) {
  CHECK_CTX(c);
  if (!charge || !coord) return fail(c, QK_ERR_NULL_POINTER, "charge/coord is NULL");
  if (nucl_num < 1 || nucl_num > (1 << 30))
    return fail(c, QK_ERR_BAD_SIZE, "nucl_num must be >= 1");
  for (int64_t i = 0; i < 3 * nucl_num; ++i)
    if (!std::isfinite(coord[i])) return fail(c, QK_ERR_INVALID_ARG, "non-finite nuclear coordinate");
  if (nucl_num != c->nucl_num) {
    c->has_basis = false;
    c->has_mo = false;
    c->cusp_on = false;  // radii were given per nucleus of the old system
  }
  c->cusp_dirty = true;
  c->nucl_num = nucl_num;
  c->nucl_charge.assign(charge, charge + nucl_num);
  c->nucl_coord.assign(coord, coord + 3 * nucl_num);
  // region the spatial point order resolves: the nuclei plus 4 bohr
  for (int k = 0; k < 3; ++k) {
    double lo = coord[k], hi = coord[k];
    for (int64_t a = 1; a < nucl_num; ++a) {
      lo = std::min(lo, coord[3 * a + k]);
      hi = std::max(hi, coord[3 * a + k]);
    }
    c->nbox_lo[k] = (float)(lo - 4.0);
    c->nbox_hi[k] = (float)(hi + 4.0);
  }
  invalidate(c);
  return QK_SUCCESS;
}

qk_status qk_set_ao_basis(qk_context c, int64_t shell_num, int64_t prim_num,
                          const int64_t* shell_nucleus, const int32_t* shell_ang_mom,
                          const int64_t* shell_prim_num, const double* shell_factor,
                          const double* exponent, const double* coefficient,
                          const double* prim_factor, int64_t ao_num, const double* ao_factor) {
  CHECK_CTX(c);
  if (c->nucl_num == 0) return fail(c, QK_ERR_NOT_PROVIDED, "set the nuclei before the basis");
  if (!shell_nucleus || !shell_ang_mom || !shell_prim_num || !shell_factor || !exponent ||
      !coefficient || !prim_factor || !ao_factor)
    return fail(c, QK_ERR_NULL_POINTER, "a basis array is NULL");
  if (shell_num < 1 || prim_num < 1 || ao_num < 1 || shell_num > (1 << 30) ||
      prim_num > (1 << 30) || ao_num > (1 << 30))
    return fail(c, QK_ERR_BAD_SIZE, "shell/prim/ao counts must be >= 1");
  int64_t np = 0, na = 0;
  for (int64_t s = 0; s < shell_num; ++s) {
    if (shell_nucleus[s] < 0 || shell_nucleus[s] >= c->nucl_num)
      return fail(c, QK_ERR_INVALID_ARG, "shell %lld: nucleus index out of range", (long long)s);
    if (shell_ang_mom[s] < 0) return fail(c, QK_ERR_INVALID_ARG, "negative angular momentum");
    if (shell_ang_mom[s] > kMaxL)
      return fail(c, QK_ERR_NOT_IMPLEMENTED, "shell %lld: l = %d > 3", (long long)s,
                  shell_ang_mom[s]);
    if (shell_prim_num[s] < 1)
      return fail(c, QK_ERR_INVALID_ARG, "shell %lld has no primitive", (long long)s);
    if (shell_prim_num[s] > kMaxPrimsChunk)
      return fail(c, QK_ERR_NOT_IMPLEMENTED, "shell %lld has more than %d primitives",
                  (long long)s, kMaxPrimsChunk);
    np += shell_prim_num[s];
    na += (shell_ang_mom[s] + 1) * (shell_ang_mom[s] + 2) / 2;
  }
  if (np != prim_num) return fail(c, QK_ERR_BAD_SIZE, "prim_num does not match shell_prim_num");
  if (na != ao_num) return fail(c, QK_ERR_BAD_SIZE, "ao_num does not match the shells");
  for (int64_t k = 0; k < prim_num; ++k)
    if (!(exponent[k] > 0.0) || !std::isfinite(exponent[k]) || !std::isfinite(coefficient[k]) ||
        !std::isfinite(prim_factor[k]))
      return fail(c, QK_ERR_INVALID_ARG, "primitive %lld: exponent must be > 0 and finite",
                  (long long)k);
  for (int64_t s = 0; s < shell_num; ++s)
    if (!std::isfinite(shell_factor[s])) return fail(c, QK_ERR_INVALID_ARG, "non-finite N_s");
  for (int64_t k = 0; k < ao_num; ++k)
    if (!std::isfinite(ao_factor[k])) return fail(c, QK_ERR_INVALID_ARG, "non-finite M_n");

  // internal shell order (see shell_order)
  std::vector<int64_t> caller_p0(shell_num + 1, 0), caller_a0(shell_num + 1, 0);
  for (int64_t s = 0; s < shell_num; ++s) {
    caller_p0[s + 1] = caller_p0[s] + shell_prim_num[s];
    caller_a0[s + 1] = caller_a0[s] + (shell_ang_mom[s] + 1) * (shell_ang_mom[s] + 2) / 2;
  }
  bool morton = false;
  std::vector<int64_t> order =
      shell_order(c, shell_num, shell_nucleus, shell_ang_mom, shell_prim_num, exponent, &morton);
  c->order_spatial = morton;
  c->order_permuted = false;
  for (int64_t i = 0; i < shell_num; ++i)
    if (order[i] != i) c->order_permuted = true;
  c->shell_perm = order;

  c->shell_num = shell_num;
  c->prim_num = prim_num;
  c->ao_num = ao_num;
  c->shell_nuc.resize(shell_num);
  c->shell_l.resize(shell_num);
  c->shell_prim0.resize(shell_num);
  c->shell_nprim.resize(shell_num);
  c->shell_ao0.resize(shell_num);
  c->shell_gmin.resize(shell_num);
  c->prim_g.resize(prim_num);
  c->prim_c.resize(prim_num);
  c->ao_fac.resize(ao_num);
  c->ao_caller.resize(ao_num);
  c->ao_shell.resize(ao_num);
  c->chunks.clear();
  int64_t p0 = 0, a0 = 0, chunk_prims = 0;
  int4 cur = make_int4(0, 0, 0, 0);
  for (int64_t s = 0; s < shell_num; ++s) {
    const int64_t cs = order[s];  // the caller's shell at internal position s
    const int l = shell_ang_mom[cs];
    const int nc = (l + 1) * (l + 2) / 2;
    const int64_t npr = shell_prim_num[cs];
    std::vector<int64_t> idx(npr);
    std::iota(idx.begin(), idx.end(), caller_p0[cs]);
    // Sec. 3.1: primitives sorted by ascending exponent, so the first one that
    // fails Eq. 3 ends the loop
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int64_t x, int64_t y) { return exponent[x] < exponent[y]; });
    for (int64_t k = 0; k < npr; ++k) {
      c->prim_g[p0 + k] = exponent[idx[k]];
      c->prim_c[p0 + k] = shell_factor[cs] * coefficient[idx[k]] * prim_factor[idx[k]];
    }
    for (int j = 0; j < nc; ++j) {
      c->ao_fac[a0 + j] = ao_factor[caller_a0[cs] + j];
      c->ao_caller[a0 + j] = (int)(caller_a0[cs] + j);
    }
    c->shell_nuc[s] = (int)shell_nucleus[cs];
    c->shell_l[s] = l;
    c->shell_prim0[s] = (int)p0;
    c->shell_nprim[s] = (int)npr;
    c->shell_ao0[s] = (int)a0;
    c->shell_gmin[s] = c->prim_g[p0];
    for (int j = 0; j < nc; ++j) c->ao_shell[a0 + j] = (int)s;
    if (cur.w - cur.z + nc > kChunkAO || cur.y - cur.x + 1 > kMaxShellsChunk ||
        chunk_prims + npr > kMaxPrimsChunk) {
      c->chunks.push_back(cur);
      cur = make_int4((int)s, (int)s, (int)a0, (int)a0);
      chunk_prims = 0;
    }
    chunk_prims += npr;
    cur.y = (int)s + 1;
    cur.w = (int)(a0 + nc);
    p0 += npr;
    a0 += nc;
  }
  c->chunks.push_back(cur);
  c->has_basis = true;
  c->has_mo = c->has_mo && c->mo_num > 0 && (int64_t)c->mo_coef.size() == c->mo_num * ao_num;
  c->mo_dirty = true;
  invalidate(c);
  return QK_SUCCESS;
}

qk_status qk_set_mo_coefficient(qk_context c, int64_t mo_num, const double* coef) {
  CHECK_CTX(c);
  if (!c->has_basis) return fail(c, QK_ERR_NOT_PROVIDED, "set the AO basis before the MOs");
  if (!coef) return fail(c, QK_ERR_NULL_POINTER, "coef is NULL");
  if (mo_num < 1 || mo_num > (1 << 24)) return fail(c, QK_ERR_BAD_SIZE, "mo_num must be >= 1");
  for (int64_t i = 0; i < mo_num * c->ao_num; ++i)
    if (!std::isfinite(coef[i])) return fail(c, QK_ERR_INVALID_ARG, "non-finite MO coefficient");
  c->mo_num = mo_num;
  c->mo_coef.assign(coef, coef + mo_num * c->ao_num);
  c->has_mo = true;
  c->mo_dirty = true;
  return QK_SUCCESS;
}

qk_status qk_set_points(qk_context c, char transp, int64_t walk_num, int64_t elec_num,
                        const double* coord) {
  CHECK_CTX(c);
  if (!coord) return fail(c, QK_ERR_NULL_POINTER, "coord is NULL");
  qk_status st = set_points_common(c, transp, walk_num, elec_num);
  if (st) return st;
  const int64_t n = c->point_num;
  cudaError_t e = c->d_raw.ensure(sizeof(double) * 3 * n);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_raw.p, coord, sizeof(double) * 3 * n, cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess)
    e = launch_points_soa((const double*)c->d_raw.p, transp, n, (double*)c->pdev.x,
                          (double*)c->pdev.y, (double*)c->pdev.z, (float*)c->pdev.hi,
                          (float*)c->pdev.lo, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "set_points");
  c->has_points = true;
  c->date++;
  return QK_SUCCESS;
}

qk_status qk_set_points_device(qk_context c, char transp, int64_t walk_num, int64_t elec_num,
                               const double* dcoord) {
  CHECK_CTX(c);
  if (!dcoord) return fail(c, QK_ERR_NULL_POINTER, "dcoord is NULL");
  qk_status st = set_points_common(c, transp, walk_num, elec_num);
  if (st) return st;
  TimedLaunch timer(c, 2);
  cudaError_t e = launch_points_soa(dcoord, transp, c->point_num, (double*)c->pdev.x,
                                    (double*)c->pdev.y, (double*)c->pdev.z, (float*)c->pdev.hi,
                                    (float*)c->pdev.lo, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "set_points_device");
  c->has_points = true;
  c->date++;
  return QK_SUCCESS;
}

qk_status qk_get_nucl_num(qk_context c, int64_t* n) {
  CHECK_CTX(c);
  if (!n) return QK_ERR_NULL_POINTER;
  if (c->nucl_num == 0) return fail(c, QK_ERR_NOT_PROVIDED, "nuclei not set");
  *n = c->nucl_num;
  return QK_SUCCESS;
}

qk_status qk_get_ao_num(qk_context c, int64_t* n) {
  CHECK_CTX(c);
  if (!n) return QK_ERR_NULL_POINTER;
  if (!c->has_basis) return fail(c, QK_ERR_NOT_PROVIDED, "AO basis not set");
  *n = c->ao_num;
  return QK_SUCCESS;
}

qk_status qk_get_mo_num(qk_context c, int64_t* n) {
  CHECK_CTX(c);
  if (!n) return QK_ERR_NULL_POINTER;
  if (!c->has_mo) return fail(c, QK_ERR_NOT_PROVIDED, "MO coefficients not set");
  *n = c->mo_num;
  return QK_SUCCESS;
}

qk_status qk_get_point_num(qk_context c, int64_t* n) {
  CHECK_CTX(c);
  if (!n) return QK_ERR_NULL_POINTER;
  if (!c->has_points) return fail(c, QK_ERR_NOT_PROVIDED, "points not set");
  *n = c->point_num;
  return QK_SUCCESS;
}

qk_status qk_workspace_size(qk_context c, size_t* bytes) {
  CHECK_CTX(c);
  if (!bytes) return QK_ERR_NULL_POINTER;
  qk_status st = require(c, false);
  if (st) return st;
  // room for both the fused path's live lists and the two-kernel path's AO
  // tensor, so that switching qk_set_fusion needs no new workspace
  *bytes = ao_tensor_bytes(c, c->mode) +
           (c->mode == QK_BF16X3 ? fused_workspace_bytes(c->point_num, (int)c->chunks.size())
                                 : 0);
  return QK_SUCCESS;
}

qk_status qk_set_fusion(qk_context c, int32_t enable) {
  CHECK_CTX(c);
  c->fused = enable != 0;
  return QK_SUCCESS;
}

qk_status qk_set_mo_cusp(qk_context c, const double* rc) {
  CHECK_CTX(c);
  if (!rc) {
    c->cusp_on = false;
    return QK_SUCCESS;
  }
  if (c->nucl_num < 1) return fail(c, QK_ERR_NOT_PROVIDED, "set the nuclei before cusp radii");
  for (int64_t A = 0; A < c->nucl_num; ++A)
    if (!(std::isfinite(rc[A]) && rc[A] >= 0.0))
      return fail(c, QK_ERR_INVALID_ARG, "cusp radii must be finite and >= 0");
  c->cusp_rc.assign(rc, rc + c->nucl_num);
  c->cusp_on = true;
  c->cusp_dirty = true;
  return QK_SUCCESS;
}

qk_status qk_get_mo_cusp_coefficients_device(qk_context c, double* df, int64_t size) {
  CHECK_CTX(c);
  if (!df) return fail(c, QK_ERR_NULL_POINTER, "df is NULL");
  if (!c->cusp_on) return fail(c, QK_ERR_NOT_PROVIDED, "no cusp radii set");
  qk_status st = require(c, true);
  if (st) return st;
  if (size < c->nucl_num * c->mo_num * 4)
    return fail(c, QK_ERR_BAD_SIZE, "df holds %lld elements, %lld needed", (long long)size,
                (long long)(c->nucl_num * c->mo_num * 4));
  st = ensure_cusp(c);
  if (st) return st;
  cudaError_t e = cudaMemcpyAsync(df, c->cusp_f64, sizeof(double) * c->nucl_num * c->mo_num * 4,
                                  cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cusp coefficients");
  return QK_SUCCESS;
}

qk_status qk_get_density_device(qk_context c, const double* w, void* drho, int64_t size) {
  CHECK_CTX(c);
  if (!w || !drho) return fail(c, QK_ERR_NULL_POINTER, "w/drho is NULL");
  qk_status st = require(c, true);
  if (st) return st;
  const int64_t P = c->point_num;
  if (size < P)
    return fail(c, QK_ERR_BAD_SIZE, "drho holds %lld elements, %lld needed", (long long)size,
                (long long)P);
  std::vector<int> occ;
  std::vector<double> w64;
  std::vector<float> w32;
  for (int64_t i = 0; i < c->mo_num; ++i) {
    if (!std::isfinite(w[i])) return fail(c, QK_ERR_INVALID_ARG, "non-finite occupation");
    if (w[i] != 0.0) {
      occ.push_back((int)i);
      w64.push_back(w[i]);
      w32.push_back((float)w[i]);
    }
  }
  st = ensure_tables(c);
  if (st) return st;
  st = ensure_mo(c);
  if (st) return st;
  const int mode = c->mode;
  const bool f64 = mode == QK_FP64;
  const bool tiled = tiled_mode(mode);
  const bool split = mode == QK_BF16X3;
  cudaError_t e;
  const int64_t no = (int64_t)occ.size();
  if (no == 0) {
    e = cudaMemsetAsync(drho, 0, (f64 ? sizeof(double) : sizeof(float)) * P, c->stream);
    return e == cudaSuccess ? QK_SUCCESS : cuda_fail(c, e, "density");
  }
  const int64_t kp = c->kpad;
  const TcConfig cfg = tc_default_config(mode, no);
  const int64_t n_tiles_n = (no + cfg.bn - 1) / cfg.bn;
  const size_t ce = f64 ? sizeof(double) : (split ? sizeof(__nv_bfloat16) : sizeof(float));
  const size_t b_idx = align_up(sizeof(int) * no, 256);
  const size_t b_w64 = align_up(sizeof(double) * no, 256);
  const size_t b_w32 = align_up(sizeof(float) * no, 256);
  const size_t b_c = align_up(ce * no * kp, 256);
  const size_t b_extra = tiled ? align_up(sizeof(float) * n_tiles_n * P, 256)
                               : align_up((f64 ? sizeof(double) : sizeof(float)) * P * no, 256);
  e = c->d_dens.ensure(b_idx + b_w64 + b_w32 + (split ? 2 : 1) * b_c + b_extra);
  if (e != cudaSuccess) return cuda_fail(c, e, "density scratch");
  unsigned char* q = (unsigned char*)c->d_dens.p;
  int* didx = (int*)q;
  double* dw64 = (double*)(q + b_idx);
  float* dw32 = (float*)(q + b_idx + b_w64);
  unsigned char* c0 = q + b_idx + b_w64 + b_w32;
  unsigned char* c1 = c0 + b_c;
  unsigned char* extra = c0 + (split ? 2 : 1) * b_c;
  e = cudaMemcpyAsync(didx, occ.data(), sizeof(int) * no, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dw64, w64.data(), sizeof(double) * no, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dw32, w32.data(), sizeof(float) * no, cudaMemcpyHostToDevice, c->stream);
  // the host vectors above must outlive the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  // the occupied MOs' rows of the chunked C planes
  if (e == cudaSuccess) {
    if (split) {
      e = launch_gather_rows(c->c_hi, kp, ce, didx, no, c0, c->stream);
      if (e == cudaSuccess) e = launch_gather_rows(c->c_lo, kp, ce, didx, no, c1, c->stream);
    } else {
      e = launch_gather_rows(f64 ? (const void*)c->c64p : (const void*)c->c32p, kp, ce, didx, no,
                             c0, c->stream);
    }
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "density tables");
  // the values-only AO tensor, in the workspace (the vgl AO tensor's memo is lost)
  const int64_t tp = ao_value_tile_points();
  const int64_t tiles = (P + tp - 1) / tp;
  AOTensor av{};
  av.ld = kp;
  av.chunked = true;
  av.nchunk = (int)c->chunks.size();
  av.comps = 1;
  av.tiled = tiled;
  av.rows = tiled ? tiles * kTileRows : P;
  const size_t ae = f64 ? sizeof(double) : (split ? sizeof(__nv_bfloat16) : sizeof(float));
  const size_t plane = align_up((size_t)av.rows * kp * ae, 256);
  const size_t need = (split ? 2 : 1) * plane +
                      (tiled ? align_up((size_t)tiles * mask_ld(av.nchunk), 256) : 0);
  void* ws = nullptr;
  st = workspace(c, need, &ws);
  if (st) return st;
  c->ao_date = ~0ull;
  av.a = ws;
  if (split) av.a_lo = (unsigned char*)ws + plane;
  if (tiled) av.mask = (uint8_t*)ws + (split ? 2 : 1) * plane;
  {
    TimedLaunch t(c, 0);
    e = launch_ao_value(c->bdev, c->pdev, mode, av, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "density ao values");
  {
    TimedLaunch t(c, 1);
    if (tiled) {
      float* part = (float*)extra;
      e = launch_mo_tc(mode, av, kp, c0, split ? (const void*)c1 : nullptr, kp, no, nullptr, cfg,
                       (int*)c->d_flag.p, c->stream, P, dw32, part);
      if (e == cudaSuccess)
        e = launch_density_reduce(part, (int)n_tiles_n, P, (float*)drho, c->stream);
    } else if (f64) {
      e = launch_gemm_f64(P, no, kp, (const double*)av.a, kp, 1, (const double*)c0, kp, 1,
                          (double*)extra, no, 1, c->stream);
      if (e == cudaSuccess) e = launch_density_from_mo(true, extra, P, no, dw64, drho, c->stream);
    } else {
      e = launch_gemm_f32(P, no, kp, (const float*)av.a, kp, 1, (const float*)c0, kp, 1,
                          (float*)extra, no, 1, c->stream);
      if (e == cudaSuccess) e = launch_density_from_mo(false, extra, P, no, dw64, drho, c->stream);
    }
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "density contraction");
  return QK_SUCCESS;
}

}  // extern "C"

namespace {

// Single-electron moves for a basis whose tables do not fit the one-launch
// kernel's shared memory: the W moved points through the full path's
// kernels (ao_vgl in a workspace of its own, then the contraction), so that
// the cached AO tensor of the full configuration stays valid.
qk_status single_move_tiled(qk_context c, int64_t W, void* dout) {
  AOTensor av{};
  av.ld = c->kpad;
  av.chunked = true;
  av.nchunk = (int)c->chunks.size();
  const bool tiled = vgl_tiled(c->mode);
  const size_t es = ao_elem_bytes(c->mode);
  size_t need = 0, plane = 0, mask = 0;
  if (tiled) {
    const int64_t tiles = (W + kTilePoints - 1) / kTilePoints;
    av.tiled = true;
    av.blocked = true;
    av.rows = tiles * kTileRows;
    plane = align_up((size_t)av.rows * av.ld * es, 256);
    mask = align_up((size_t)tiles * mask_ld(av.nchunk), 256);
    need = (c->mode == QK_BF16X3 ? 2 : 1) * plane + mask;
  } else {
    av.rows = 5 * W;
    plane = align_up((size_t)av.rows * av.ld * es, 256);
    need = plane;
  }
  cudaError_t e = c->d_single_ws.ensure(need);
  if (e != cudaSuccess) return cuda_fail(c, e, "single-move workspace");
  unsigned char* p = (unsigned char*)c->d_single_ws.p;
  av.a = p;
  if (tiled) {
    if (c->mode == QK_BF16X3) av.a_lo = p + kBlockElems * es;  // planes interleave by block
    // a few tiles only: each ao_vgl tile culls for itself (no pre-pass launch)
    av.mask = p + (c->mode == QK_BF16X3 ? 2 : 1) * plane;
  }
  {
    TimedLaunch t(c, 0);
    e = launch_ao_vgl(c->bdev, c->psingle, c->mode, av, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "single-move ao_vgl");
  qk_status st = contract(c, av, 5 * W, dout);
  if (st) return st;
  return apply_cusp(c, c->psingle, dout);
}

}  // namespace

extern "C" {

qk_status qk_set_single_point_device(qk_context c, int64_t elec, const double* dcoord) {
  CHECK_CTX(c);
  if (!dcoord) return fail(c, QK_ERR_NULL_POINTER, "dcoord is NULL");
  if (!c->has_points) return fail(c, QK_ERR_NOT_PROVIDED, "set the points first");
  if (elec < 0 || elec >= c->elec_num)
    return fail(c, QK_ERR_INVALID_ARG, "electron index %lld outside [0, %lld)", (long long)elec,
                (long long)c->elec_num);
  qk_status st = ensure_device(c);
  if (st) return st;
  const int64_t W = c->walk_num;
  cudaError_t e = c->d_single.ensure(align_up(sizeof(double) * 3 * W, 256) +
                                     align_up(sizeof(float) * 6 * W, 256));
  if (e != cudaSuccess) return cuda_fail(c, e, "single-point buffers");
  double* base = (double*)c->d_single.p;
  float* fb = (float*)((unsigned char*)c->d_single.p + align_up(sizeof(double) * 3 * W, 256));
  c->psingle.n = W;
  c->psingle.x = base;
  c->psingle.y = base + W;
  c->psingle.z = base + 2 * W;
  c->psingle.hi = fb;
  c->psingle.lo = fb + 3 * W;
  c->psingle.ld = W;
  {
    TimedLaunch t(c, 2);
    e = launch_points_soa(dcoord, 'N', W, base, base + W, base + 2 * W, fb, fb + 3 * W,
                          c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "set_single_point_device");
  c->single_elec = elec;
  return QK_SUCCESS;
}

qk_status qk_get_mo_vgl_single_device(qk_context c, void* dout, int64_t size) {
  CHECK_CTX(c);
  if (!dout) return fail(c, QK_ERR_NULL_POINTER, "dout is NULL");
  qk_status st = require(c, true);
  if (st) return st;
  if (c->single_elec < 0) return fail(c, QK_ERR_NOT_PROVIDED, "no single-electron move set");
  const int64_t W = c->psingle.n, N = c->mo_num;
  if (size < 5 * W * N)
    return fail(c, QK_ERR_BAD_SIZE, "output holds %lld elements, %lld needed", (long long)size,
                (long long)(5 * W * N));
  st = ensure_tables(c);
  if (st) return st;
  st = ensure_mo(c);
  if (st) return st;
  st = ensure_cusp(c);
  if (st) return st;
  // FP64: one launch, each moved point's AO row and its product with C^T
  // (kept per upload of C), when the basis tables fit the kernel's shared
  // memory; the reduced modes (and larger bases) run the moved points through
  // the tile kernels, whose shared C blocks move far fewer bytes than a
  // product per point.  The cached AO tensor of the full configuration stays
  // valid either way.
  const bool f64 = c->mode == QK_FP64;
  if (!f64 || !single_mo_fits(f64, c->bdev)) return single_move_tiled(c, W, dout);
  if (c->single_ct_version != c->mo_version || c->single_ct_f64 != f64 || !c->d_single_ct.p) {
    const size_t es = f64 ? sizeof(double) : sizeof(float);
    cudaError_t e = c->d_single_ct.ensure(es * (size_t)c->ao_num * single_ct_ld(f64, N));
    if (e == cudaSuccess) e = launch_single_ct(f64, c->c64, N, c->ao_num, c->d_single_ct.p, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "single-move C^T");
    c->single_ct_version = c->mo_version;
    c->single_ct_f64 = f64;
  }
  cudaError_t e;
  {
    TimedLaunch t(c, 1);
    e = launch_single_mo(f64, c->bdev, c->psingle, c->d_single_ct.p, N, dout, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "single-move MO vgl");
  return apply_cusp(c, c->psingle, dout);
}

qk_status qk_accept_single_point(qk_context c) {
  CHECK_CTX(c);
  if (c->single_elec < 0) return fail(c, QK_ERR_NOT_PROVIDED, "no single-electron move set");
  cudaError_t e;
  {
    TimedLaunch t(c, 2);
    e = launch_scatter_points(c->psingle, c->pdev, c->elec_num, c->single_elec, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "accept_single_point");
  c->single_elec = -1;
  c->date++;  // new configuration: cached AOs and point order are stale
  return QK_SUCCESS;
}

qk_status qk_set_basis_order(qk_context c, int32_t mode) {
  CHECK_CTX(c);
  if (mode < 0 || mode > 2) return fail(c, QK_ERR_INVALID_ARG, "order mode must be 0, 1 or 2");
  c->order_mode = mode;
  return QK_SUCCESS;
}

qk_status qk_get_basis_order(qk_context c, int32_t* spatial) {
  CHECK_CTX(c);
  if (!spatial) return fail(c, QK_ERR_NULL_POINTER, "spatial is NULL");
  if (!c->has_basis) return fail(c, QK_ERR_NOT_PROVIDED, "AO basis not set");
  *spatial = c->order_spatial ? 1 : 0;
  return QK_SUCCESS;
}

qk_status qk_get_shell_order(qk_context c, int64_t* order, int64_t n) {
  CHECK_CTX(c);
  if (!order) return fail(c, QK_ERR_NULL_POINTER, "order is NULL");
  if (!c->has_basis) return fail(c, QK_ERR_NOT_PROVIDED, "AO basis not set");
  if (n < c->shell_num)
    return fail(c, QK_ERR_BAD_SIZE, "order holds %lld entries, %lld needed", (long long)n,
                (long long)c->shell_num);
  std::copy(c->shell_perm.begin(), c->shell_perm.end(), order);
  return QK_SUCCESS;
}

qk_status qk_set_spatial_order(qk_context c, int32_t enable) {
  CHECK_CTX(c);
  c->spatial = enable != 0;
  return QK_SUCCESS;
}

qk_status qk_set_sm_pairs(qk_context c, int32_t enable) {
  CHECK_CTX(c);
  c->sm_pairs = enable != 0;
  return QK_SUCCESS;
}

qk_status qk_set_workspace(qk_context c, void* dev, size_t bytes) {
  CHECK_CTX(c);
  if (dev && ((uintptr_t)dev % 256 != 0))
    return fail(c, QK_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  c->ws_user = dev;
  c->ws_user_bytes = dev ? bytes : 0;
  if (dev) c->ws_own.release();
  c->ao_date = ~0ull;  // cached AO tensor lived in the previous workspace
  return QK_SUCCESS;
}

qk_status qk_set_stream(qk_context c, void* stream) {
  CHECK_CTX(c);
  c->stream = (cudaStream_t)stream;
  return QK_SUCCESS;
}

qk_status qk_synchronize(qk_context c) {
  CHECK_CTX(c);
  qk_status st = ensure_device(c);
  if (st) return st;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
  int flag = 0;
  e = cudaMemcpy(&flag, c->d_flag.p, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "error flag read");
  if (flag != 0) {
    cudaMemset(c->d_flag.p, 0, sizeof(int));
    return fail(c, QK_ERR_DEVICE_TIMEOUT, "a device-side wait gave up (code %d)", flag);
  }
  return QK_SUCCESS;
}

qk_status qk_get_ao_vgl_device(qk_context c, void* dout, int64_t size) {
  CHECK_CTX(c);
  if (!dout) return fail(c, QK_ERR_NULL_POINTER, "dout is NULL");
  qk_status st = require(c, false);
  if (st) return st;
  if (size < 5 * c->point_num * c->ao_num)
    return fail(c, QK_ERR_BAD_SIZE, "output holds %lld elements, %lld needed", (long long)size,
                (long long)(5 * c->point_num * c->ao_num));
  st = ensure_tables(c);
  if (st) return st;
  AOTensor t{};
  t.a = dout;
  t.rows = 5 * c->point_num;
  t.ld = c->ao_num;
  t.caller_cols = true;  // the caller's AO order
  const int m = c->mode == QK_FP64 ? QK_FP64 : QK_FP32;
  cudaError_t e = launch_ao_vgl(c->bdev, c->pdev, m, t, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "ao_vgl launch");
  return QK_SUCCESS;
}

qk_status qk_get_ao_vgl(qk_context c, void* out, int64_t size) {
  CHECK_CTX(c);
  if (!out) return fail(c, QK_ERR_NULL_POINTER, "out is NULL");
  qk_status st = require(c, false);
  if (st) return st;
  const int64_t n = 5 * c->point_num * c->ao_num;
  if (size < n) return fail(c, QK_ERR_BAD_SIZE, "output too small");
  const size_t es = c->mode == QK_FP64 ? sizeof(double) : sizeof(float);
  cudaError_t e = c->d_out.ensure(es * n);
  if (e != cudaSuccess) return cuda_fail(c, e, "output staging");
  st = qk_get_ao_vgl_device(c, c->d_out.p, n);
  if (st) return st;
  e = cudaMemcpyAsync(out, c->d_out.p, es * n, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "get_ao_vgl copy");
  return qk_synchronize(c);
}

qk_status qk_get_mo_vgl_device(qk_context c, void* dout, int64_t size) {
  CHECK_CTX(c);
  if (!dout) return fail(c, QK_ERR_NULL_POINTER, "dout is NULL");
  qk_status st = require(c, true);
  if (st) return st;
  const int64_t M = 5 * c->point_num, N = c->mo_num;
  if (size < M * N)
    return fail(c, QK_ERR_BAD_SIZE, "output holds %lld elements, %lld needed", (long long)size,
                (long long)(M * N));
  st = ensure_mo(c);
  if (st) return st;
  st = ensure_cusp(c);
  if (st) return st;
  if (use_fused(c)) {
    void* ws = nullptr;
    const size_t fb = fused_workspace_bytes(c->point_num, (int)c->chunks.size());
    st = workspace(c, ao_tensor_bytes(c, c->mode) + fb, &ws);
    if (st) return st;
    // the live lists sit behind the (unused here) AO tensor area
    unsigned char* lp = (unsigned char*)ws + ao_tensor_bytes(c, c->mode);
    const int64_t tiles = ao_tiles(c);
    int* live_count = (int*)lp;
    uint16_t* live_list = (uint16_t*)(lp + align_up((size_t)tiles * 4, 256));
    cudaError_t e;
    {
      TimedLaunch t0(c, 0);
      e = launch_fused_live(c->bdev, c->pdev, live_count, live_list, c->stream);
    }
    if (e == cudaSuccess) {
      TimedLaunch t1(c, 1);
      e = launch_mo_fused(tc_default_config(c->mode, N).bn, c->bdev, c->pdev, c->c_hi, c->c_lo,
                          c->kpad, N, (float*)dout, live_count, live_list, (int*)c->d_flag.p,
                          c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "fused mo_vgl");
    c->fused_date = c->date;
    c->fused_lists = lp;
    c->ao_date = ~0ull;  // no AO tensor was written
    return apply_cusp(c, c->pdev, dout, true);
  }
  AOTensor ao{};
  st = provide_ao(c, &ao);
  if (st) return st;
  st = contract(c, ao, M, dout);
  if (st) return st;
  return apply_cusp(c, c->pdev, dout, true);
}

qk_status qk_get_mo_vgl(qk_context c, void* out, int64_t size) {
  CHECK_CTX(c);
  if (!out) return fail(c, QK_ERR_NULL_POINTER, "out is NULL");
  qk_status st = require(c, true);
  if (st) return st;
  const int64_t n = 5 * c->point_num * c->mo_num;
  if (size < n) return fail(c, QK_ERR_BAD_SIZE, "output too small");
  const size_t es = c->mode == QK_FP64 ? sizeof(double) : sizeof(float);
  cudaError_t e = c->d_out.ensure(es * n);
  if (e != cudaSuccess) return cuda_fail(c, e, "output staging");
  const int64_t per = host_range_points(c);
  if (per >= c->point_num || use_fused(c)) {
    st = qk_get_mo_vgl_device(c, c->d_out.p, n);
    if (st) return st;
    e = cudaMemcpyAsync(out, c->d_out.p, es * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_mo_vgl copy");
    return qk_synchronize(c);
  }
  // Point ranges in turn: range r's output goes to the host on a second
  // stream while range r + 1 is evaluated (the copy link is the slower part).
  st = ensure_mo(c);
  if (st) return st;
  st = ensure_cusp(c);
  if (st) return st;
  AOTensor ao{};
  bool have_ao = false;
  st = ao_workspace(c, &ao, &have_ao, false);  // ranges are contiguous in the caller's order
  if (st) return st;
  if (!c->copy_stream) {
    e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy stream");
  }
  const int64_t N = c->mo_num;
  const int64_t ranges = (c->point_num + per - 1) / per;
  while ((int64_t)c->range_done.size() < ranges) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(c, e, "range events");
    c->range_done.push_back(ev);
  }
  unsigned char* dbase = (unsigned char*)c->d_out.p;
  unsigned char* hbase = (unsigned char*)out;
  for (int64_t r = 0; r < ranges; ++r) {
    const int64_t p0 = r * per;
    const int64_t p1 = p0 + per < c->point_num ? p0 + per : c->point_num;
    const AOTensor av = ao_range(ao, c->mode, p0, p1);
    if (!have_ao) {
      TimedLaunch t(c, 0, av.tiled && av.reach ? 2 : 1);
      e = launch_ao_vgl(c->bdev, points_range(c->pdev, p0, p1), c->mode, av, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "ao_vgl launch");
    }
    const size_t off = (size_t)5 * p0 * N * es;
    st = contract(c, av, 5 * (p1 - p0), dbase + off);
    if (st) return st;
    st = apply_cusp(c, points_range(c->pdev, p0, p1), dbase + off);
    if (st) return st;
    e = cudaEventRecord(c->range_done[r], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy_stream, c->range_done[r], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hbase + off, dbase + off, (size_t)5 * (p1 - p0) * N * es,
                          cudaMemcpyDeviceToHost, c->copy_stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_mo_vgl range copy");
  }
  if (!have_ao) mark_ao(c, ao, false);
  e = cudaStreamSynchronize(c->copy_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "get_mo_vgl copy");
  return qk_synchronize(c);
}

qk_status qk_set_timing(qk_context c, int32_t enable) {
  CHECK_CTX(c);
  c->timing = enable != 0;
  for (int k = 0; k < kTimerClasses; ++k) c->ev_used[k] = 0;
  return QK_SUCCESS;
}

qk_status qk_get_kernel_count(qk_context c, int64_t* count) {
  CHECK_CTX(c);
  if (!count) return fail(c, QK_ERR_NULL_POINTER, "count is NULL");
  *count = c->kernels;
  c->kernels = 0;
  return QK_SUCCESS;
}

qk_status qk_get_timing(qk_context c, double* ms, int64_t* launches, int32_t n) {
  CHECK_CTX(c);
  if (!ms || !launches) return fail(c, QK_ERR_NULL_POINTER, "ms/launches is NULL");
  if (n < 1 || n > kTimerClasses) return fail(c, QK_ERR_BAD_SIZE, "n must be in [1, 3]");
  for (int k = 0; k < n; ++k) {
    double tot = 0.0;
    for (size_t i = 0; i < c->ev_used[k]; ++i) {
      cudaError_t e = cudaEventSynchronize(c->ev_stop[k][i]);
      float t = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, c->ev_start[k][i], c->ev_stop[k][i]);
      if (e != cudaSuccess) return cuda_fail(c, e, "timing events");
      tot += t;
    }
    ms[k] = tot;
    launches[k] = (int64_t)c->ev_used[k];
    c->ev_used[k] = 0;
  }
  return QK_SUCCESS;
}

}  // extern "C"

namespace {

// Layout of the backward scratch.  FP64 / FP32: recomputed AO tensor, Abar
// (both [5P][ld]), split-K partials of dL/dC, then the dR partials.
// Split bf16: the block-sparse products' scratch (the AO tensor is the
// forward's, in the workspace), then the dR partials.
struct BwdLayout {
  size_t ao, abar, dc, dr, total;
  int k_split;
  bool tc;  // split-bf16 products on the tensor cores (dc: their scratch)
};

BwdLayout bwd_layout(qk_context c) {
  BwdLayout L{};
  if (c->mode == QK_BF16X3) {
    L.tc = true;
    L.dc = 0;
    L.dr = align_up(adjoint_sparse_scratch_bytes(c->point_num, (int)c->chunks.size(), c->mo_num),
                    256);
    L.total = L.dr + align_up(adjoint_dR_partial_bytes(c->bdev, c->point_num), 256);
    return L;
  }
  const bool f64 = c->mode == QK_FP64;
  const size_t es = f64 ? sizeof(double) : sizeof(float);
  const int64_t rows = 5 * c->point_num, ld = round_up8(c->ao_num);
  // enough split-K blocks to fill the GPU: SIMT tiles are 64x64 (FP64) or
  // 128x128 (FP32); keep >= 1024 rows per split
  const int64_t tile = f64 ? 64 : 128;
  const int64_t tiles = ((c->mo_num + tile - 1) / tile) * ((c->ao_num + tile - 1) / tile);
  int64_t ks = (304 + tiles - 1) / tiles;
  const int64_t kmax = (rows + 1023) / 1024;
  if (ks > kmax) ks = kmax;
  if (ks < 1) ks = 1;
  L.k_split = (int)ks;
  L.ao = 0;
  L.abar = align_up(rows * ld * es, 256);
  L.dc = L.abar + align_up(rows * ld * es, 256);
  L.dr = L.dc + align_up((size_t)ks * c->mo_num * c->ao_num * es, 256);
  L.total = L.dr + align_up(adjoint_dR_partial_bytes(c->bdev, c->point_num), 256);
  return L;
}

}  // namespace

extern "C" {

qk_status qk_get_block_stats(qk_context c, int64_t* live_blocks, int64_t* total_blocks,
                             int64_t* live_entries) {
  CHECK_CTX(c);
  if (!live_blocks || !total_blocks || !live_entries)
    return fail(c, QK_ERR_NULL_POINTER, "output pointer is NULL");
  if (c->fused_date == c->date && c->fused_lists && use_fused(c)) {
    const int64_t tiles = ao_tiles(c), nq = (int64_t)c->chunks.size();
    std::vector<int> cnt((size_t)tiles);
    std::vector<uint16_t> lst((size_t)(tiles * nq));
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy(cnt.data(), c->fused_lists, sizeof(int) * tiles, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(lst.data(), c->fused_lists + align_up((size_t)tiles * 4, 256),
                     sizeof(uint16_t) * lst.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "live list read");
    int64_t live = 0, entries = 0;
    for (int64_t ti = 0; ti < tiles; ++ti) {
      const int64_t pts = std::min<int64_t>(kTilePoints, c->point_num - ti * kTilePoints);
      for (int i = 0; i < cnt[ti]; ++i) {
        const int4 ch = c->chunks[lst[ti * nq + i]];
        ++live;
        entries += pts * (ch.w - ch.z);
      }
    }
    *live_blocks = live;
    *total_blocks = tiles * nq;
    *live_entries = entries;
    return QK_SUCCESS;
  }
  if (!vgl_tiled(c->ao_mode) || c->ao_ws == nullptr || c->ao_date != c->date)
    return fail(c, QK_ERR_NOT_PROVIDED,
                "no AO tensor of the current points in a block-sparse mode");
  const AOTensor t = ao_view(c, c->ao_ws, c->ao_mode);
  const int64_t tiles = ao_tiles(c), nq = t.nchunk, ld = mask_ld(t.nchunk);
  std::vector<uint8_t> mask((size_t)(tiles * ld));
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(mask.data(), t.mask, mask.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "block mask read");
  int64_t live = 0, entries = 0;
  for (int64_t ti = 0; ti < tiles; ++ti) {
    const int64_t pts = std::min<int64_t>(kTilePoints, c->point_num - ti * kTilePoints);
    for (int64_t q = 0; q < nq; ++q)
      if (mask[ti * ld + q]) {
        ++live;
        entries += pts * (c->chunks[q].w - c->chunks[q].z);
      }
  }
  *live_blocks = live;
  *total_blocks = tiles * nq;
  *live_entries = entries;
  return QK_SUCCESS;
}

qk_status qk_get_sparsity_stats(qk_context c, int64_t* live_groups, int64_t* nnz) {
  CHECK_CTX(c);
  if (!live_groups || !nnz) return fail(c, QK_ERR_NULL_POINTER, "output pointer is NULL");
  if (use_fused(c) || !vgl_tiled(c->ao_mode) || c->ao_ws == nullptr ||
      c->ao_date != c->date)
    return fail(c, QK_ERR_NOT_PROVIDED,
                "no AO tensor of the current points in a two-kernel tensor-core mode");
  const AOTensor t = ao_view(c, c->ao_ws, c->ao_mode);
  const int64_t tiles = ao_tiles(c), nq = t.nchunk, ld = mask_ld(t.nchunk);
  std::vector<uint8_t> mask((size_t)(tiles * ld));
  // the counter lives in the second half of the 256-byte error-word buffer
  auto* cnt = reinterpret_cast<unsigned long long*>(static_cast<char*>(c->d_flag.p) + 128);
  unsigned long long h = 0;
  cudaError_t e = launch_ao_nnz(t, (int)ao_elem_bytes(c->ao_mode), c->point_num, cnt, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(mask.data(), t.mask, mask.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "sparsity count");
  int64_t g = 0;
  for (int64_t ti = 0; ti < tiles; ++ti)
    for (int64_t q = 0; q < nq; ++q) g += __builtin_popcount(mask[ti * ld + q] & 0xFu);
  *live_groups = g;
  *nnz = (int64_t)h;
  return QK_SUCCESS;
}

qk_status qk_get_tile_layout(qk_context c, int32_t* perm, int64_t n, int32_t* live,
                             int64_t ntiles, uint8_t* groups, int64_t gsize) {
  CHECK_CTX(c);
  if (use_fused(c) || !vgl_tiled(c->ao_mode) || c->ao_ws == nullptr ||
      c->ao_date != c->date)
    return fail(c, QK_ERR_NOT_PROVIDED,
                "no AO tensor of the current points in a two-kernel tensor-core mode");
  const int64_t tiles = ao_tiles(c);
  const int64_t nchunk = (int64_t)c->chunks.size();
  if ((perm && n < c->point_num) || (live && ntiles < tiles) ||
      (groups && gsize < tiles * nchunk))
    return fail(c, QK_ERR_BAD_SIZE, "perm needs %lld, live %lld and groups %lld elements",
                (long long)c->point_num, (long long)tiles, (long long)(tiles * nchunk));
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "tile layout");
  if (perm) {
    if (c->ao_sorted && c->perm) {
      e = cudaMemcpy(perm, c->perm, sizeof(int32_t) * c->point_num, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(c, e, "point order read");
    } else {
      for (int64_t s = 0; s < c->point_num; ++s) perm[s] = (int32_t)s;
    }
  }
  if (live || groups) {
    const AOTensor t = ao_view(c, c->ao_ws, c->ao_mode);
    const int64_t nq = t.nchunk, ld = mask_ld(t.nchunk);
    std::vector<uint8_t> mask((size_t)(tiles * ld));
    e = cudaMemcpy(mask.data(), t.mask, mask.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "block mask read");
    for (int64_t ti = 0; ti < tiles; ++ti) {
      int32_t k = 0;
      for (int64_t q = 0; q < nq; ++q) {
        k += mask[ti * ld + q] != 0;
        if (groups) groups[ti * nq + q] = mask[ti * ld + q] & 0xFu;
      }
      if (live) live[ti] = k;
    }
  }
  return QK_SUCCESS;
}

qk_status qk_get_ao_chunk_num(qk_context c, int64_t* nchunk) {
  CHECK_CTX(c);
  if (!nchunk) return fail(c, QK_ERR_NULL_POINTER, "output pointer is NULL");
  if (!c->has_basis) return fail(c, QK_ERR_NOT_PROVIDED, "AO basis not set");
  *nchunk = (int64_t)c->chunks.size();
  return QK_SUCCESS;
}

qk_status qk_backward_workspace_size(qk_context c, size_t* bytes) {
  CHECK_CTX(c);
  if (!bytes) return QK_ERR_NULL_POINTER;
  qk_status st = require(c, true);
  if (st) return st;
  st = ensure_tables(c);
  if (st) return st;
  *bytes = bwd_layout(c).total;
  return QK_SUCCESS;
}

qk_status qk_mo_vgl_backward_device(qk_context c, const void* dW, int64_t size, double* d_dC,
                                    double* d_dR) {
  CHECK_CTX(c);
  if (!dW) return fail(c, QK_ERR_NULL_POINTER, "dW is NULL");
  qk_status st = require(c, true);
  if (st) return st;
  if (c->cusp_on)
    return fail(c, QK_ERR_NOT_IMPLEMENTED, "the adjoint does not cover the cusp correction");
  const int64_t rows = 5 * c->point_num, N = c->mo_num, K = c->ao_num;
  if (size < rows * N)
    return fail(c, QK_ERR_BAD_SIZE, "dW holds %lld elements, %lld needed", (long long)size,
                (long long)(rows * N));
  st = ensure_tables(c);
  if (st) return st;
  st = ensure_mo(c);
  if (st) return st;
  const BwdLayout L = bwd_layout(c);
  // split bf16: the forward's AO tensor of the current points (computed
  // here if the last forward pass did not leave it in the workspace)
  AOTensor fao{};
  if (L.tc) {
    st = provide_ao(c, &fao);
    if (st) return st;
  }
  // scratch: behind the forward's AO tensor in the caller's workspace when it
  // is large enough, else library-owned
  unsigned char* base = nullptr;
  const size_t fwd = ao_tensor_bytes(c, c->mode);
  if (c->ws_user && c->ws_user_bytes >= fwd + L.total) {
    base = (unsigned char*)c->ws_user + fwd;
  } else {
    cudaError_t e = c->bwd_own.ensure(L.total);
    if (e != cudaSuccess) return cuda_fail(c, e, "backward scratch");
    base = (unsigned char*)c->bwd_own.p;
  }
  const bool f64 = c->mode == QK_FP64;
  const int64_t ld = round_up8(K);
  AOTensor ao{};
  ao.a = base + L.ao;
  ao.rows = rows;
  ao.ld = ld;
  ao.chunked = false;
  void* abar = base + L.abar;
  void* dcp = base + L.dc;
  double* drp = (double*)(base + L.dr);
  cudaError_t e;
  TimedLaunch timer(c, 2);
  if (L.tc) {
    // split bf16 on the tensor cores over the live blocks of the forward's
    // AO tensor: dL/dC = W^T . AO, Abar = W . C at the live blocks, dL/dR
    if (c->ct_version != c->mo_version || !c->d_ct.p) {
      const int nq = (int)c->chunks.size();
      e = c->d_ct.ensure(adjoint_sparse_ctk_bytes(nq, N));
      if (e == cudaSuccess) e = launch_adjoint_ctk_split(c->c64p, N, nq, c->d_ct.p, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "backward C^T planes");
      c->ct_version = c->mo_version;
    }
    const PointsDev& tp = c->ao_sorted ? c->psort : c->pdev;  // the tiles' points
    e = launch_adjoint_sparse(c->bdev, tp, fao, (const float*)dW, N, c->d_ct.p, !c->ao_zeroed,
                              d_dC, d_dR, base + L.dc, drp, (int*)c->d_flag.p, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "backward tensor-core products");
    c->ao_zeroed = true;
    return QK_SUCCESS;
  }
  // 1. AO values recomputed, not kept from the forward pass
  e = launch_ao_vgl(c->bdev, c->pdev, f64 ? QK_FP64 : QK_FP32, ao, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "backward ao_vgl");
  // 2. Abar[row][k] = sum_i W[row][i] C[i][k]
  if (f64)
    e = launch_gemm_f64(rows, K, N, (const double*)dW, N, 1, c->c64, 1, K, (double*)abar, ld, 1,
                        c->stream);
  else
    e = launch_gemm_f32(rows, K, N, (const float*)dW, N, 1, c->c32, 1, c->ldc, (float*)abar, ld,
                        1, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "backward Abar");
  // 3. dL/dC[i][k] = sum_row W[row][i] AO[row][k], split over rows
  if (d_dC) {
    if (f64) {
      e = launch_gemm_f64(N, K, rows, (const double*)dW, 1, N, (const double*)ao.a, 1, ld,
                          (double*)dcp, K, L.k_split, c->stream);
      if (e == cudaSuccess)
        e = launch_reduce_partials_f64((const double*)dcp, L.k_split, N * K, d_dC, c->stream,
                                       c->bdev.ao_caller, K);
    } else {
      e = launch_gemm_f32(N, K, rows, (const float*)dW, 1, N, (const float*)ao.a, 1, ld,
                          (float*)dcp, K, L.k_split, c->stream);
      if (e == cudaSuccess)
        e = launch_reduce_partials_f32((const float*)dcp, L.k_split, N * K, d_dC, c->stream,
                                       c->bdev.ao_caller, K);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "backward dL/dC");
  }
  // 4. dL/dR_nuc from Abar and third-order AO derivatives
  if (d_dR) {
    e = launch_adjoint_dR(c->bdev, c->pdev, f64 ? QK_FP64 : QK_FP32, abar, ld, drp, d_dR,
                          c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "backward dL/dR");
  }
  return QK_SUCCESS;
}

}  // extern "C"

namespace qk {

qk_status context_fail(qk_context c, qk_status code, const char* msg) {
  return fail(c, code, "%s", msg);
}

qk_status context_forward_views(qk_context c, ForwardViews* v) {
  CHECK_CTX(c);
  qk_status st = require(c, true);
  if (st) return st;
  st = ensure_tables(c);
  if (st) return st;
  st = ensure_mo(c);
  if (st) return st;
  void* ws = nullptr;
  st = workspace(c, ao_tensor_bytes(c, c->mode), &ws);
  if (st) return st;
  v->b = c->bdev;
  v->p = c->pdev;
  v->ao = ao_view(c, ws, c->mode);
  const bool split = c->mode == QK_BF16X3;
  v->c_hi = split ? (const void*)c->c_hi : (const void*)c->c32p;
  v->c_lo = split ? (const void*)c->c_lo : nullptr;
  v->kpad = c->kpad;
  v->mo_num = c->mo_num;
  v->walk_num = c->walk_num;
  v->elec_num = c->elec_num;
  v->mode = c->mode;
  v->basis_version = c->basis_version;
  for (int k = 0; k < 3; ++k) {
    v->box_lo[k] = c->nbox_lo[k];
    v->box_hi[k] = c->nbox_hi[k];
  }
  v->spatial = c->spatial;
  v->mo_version = c->mo_version;
  return QK_SUCCESS;
}

bool context_cusp_on(qk_context c) { return c->cusp_on; }

void context_forget_ao(qk_context c) { c->ao_date = ~0ull; }

qk_status context_pair_c(qk_context c, int bn, int half_rows, const void** out) {
  qk_status st = ensure_mo(c);
  if (st) return st;
  if (c->cpair_version != c->mo_version || c->cpair_bn != bn || c->cpair_half != half_rows ||
      c->cpair_mode != c->mode) {
    const bool split = c->mode == QK_BF16X3;
    const void* b_hi = split ? (const void*)c->c_hi : (const void*)c->c32p;
    const void* b_lo = split ? (const void*)c->c_lo : nullptr;
    cudaError_t e = c->d_cpair.ensure(pair_c_bytes(c->mode, c->mo_num, c->kpad, bn, half_rows));
    if (e == cudaSuccess)
      e = launch_pair_c(c->mode, b_hi, b_lo, c->kpad, c->mo_num, c->kpad, bn, half_rows,
                        c->d_cpair.p, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "blocked C");
    c->cpair_version = c->mo_version;
    c->cpair_bn = bn;
    c->cpair_half = half_rows;
    c->cpair_mode = c->mode;
  }
  *out = c->d_cpair.p;
  return QK_SUCCESS;
}

}  // namespace qk
