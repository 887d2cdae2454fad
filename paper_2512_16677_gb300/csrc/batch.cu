// batch.cu -- walkers of several molecules of uneven sizes in one launch.
//
// A batch holds contexts that are fully set (basis, MO coefficients, points)
// in a tensor-core mode.  One run evaluates every molecule's MO vgl as the
// single-molecule path does, each step one launch (or one sort) for all
// molecules: a spatial order of every molecule's points in one radix sort
// (problem index above the cell key), the tiles' reach pre-pass, ao_vgl
// over a work list of (molecule, AO chunk, point tiles) items, then the
// tcgen05 contraction over (molecule, M-tile pair, N tile) items on pairs of
// SMs (or (molecule, M tile, N tile) on single SMs), the two lists
// ordered longest first (LPT) so that the largest pieces start early and
// the tail is made of small ones.  The launches are captured once in a CUDA
// graph and replayed on later runs; the work lists
// and per-molecule descriptors (tensor maps, pointers, sizes) live in device
// memory and are rebuilt only when a shape or pointer changes.  The MMA N
// of each molecule is chosen below the launch's BN_MAX, which the autotuner
// picks by timing every instantiated BN_MAX on the batch itself.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

using namespace qk;

struct qk_batch_s {
  std::vector<qk_context> ctxs;
  int mode = -1;
  cudaStream_t stream = nullptr;
  int bn_max = 160;
  bool use_graph = true;
  std::string err;
  // device descriptors and work lists
  DevBuf d_ao_probs, d_tc_probs, d_ao_items, d_tc_items, d_flag;
  int64_t n_ao_items = 0, n_tc_items = 0;
  // the spatial order of all molecules' points
  DevBuf d_sort, d_sort_probs, d_off;
  // contraction on pairs of SMs: per molecule C blocked with halves of
  // bn_max / 2 rows, and the pair problem descriptors
  bool sm_pairs = true;
  std::vector<DevBuf> d_cpair;
  DevBuf d_pair_probs;
  BatchOrder order{};
  int64_t max_tiles = 0;
  int max_shells = 0;
  std::vector<uintptr_t> signature;  // what the descriptors were built from
  cudaGraphExec_t graph = nullptr;
  int graph_bn = -1;
  ~qk_batch_s() {
    if (graph) cudaGraphExecDestroy(graph);
  }
};

namespace {

qk_status bfail(qk_batch b, qk_status code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

qk_status bcuda(qk_batch b, cudaError_t e, const char* what) {
  cudaGetLastError();
  return bfail(b, e == cudaErrorMemoryAllocation ? QK_ERR_OUT_OF_MEMORY : QK_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

// ao_vgl work items of a batch: about four waves of resident CTAs.
constexpr int64_t kAoItemsTarget = 3000;

// MMA N for a molecule with n MOs under bn_max: as few N tiles as possible,
// then the smallest multiple of 16 that covers n in that many tiles.
int pick_bn(int64_t n, int bn_max) {
  const int64_t tiles = (n + bn_max - 1) / bn_max;
  const int64_t per = (n + tiles - 1) / tiles;
  return (int)((per + 15) / 16 * 16);
}

// Build descriptors and work lists for the current contexts and outputs.
qk_status build(qk_batch b, float* const* outs) {
  // the descriptors, work lists and error word are rewritten below with
  // blocking copies on the legacy stream: first let every earlier launch on
  // the batch stream finish, and report a wait of one of them that gave up
  // before its error word is cleared
  if (b->d_flag.p) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flag, b->d_flag.p, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "batch rebuild");
    if (flag != 0) {
      cudaMemset(b->d_flag.p, 0, sizeof(int));
      return bfail(b, QK_ERR_DEVICE_TIMEOUT, "a device-side wait of an earlier run gave up");
    }
  }
  const int n = (int)b->ctxs.size();
  std::vector<ForwardViews> views(n);
  std::vector<int64_t> off(n + 1, 0);
  std::vector<SortProblem> sp(n);
  for (int i = 0; i < n; ++i) {
    ForwardViews& v = views[i];
    if (context_cusp_on(b->ctxs[i]))
      return bfail(b, QK_ERR_NOT_IMPLEMENTED,
                   "context " + std::to_string(i) + " has the cusp correction on");
    qk_status st = context_forward_views(b->ctxs[i], &v);
    if (st) return bfail(b, st, "context " + std::to_string(i) + " is not ready");
    off[i + 1] = off[i] + v.p.n;
    sp[i].p = v.p;
    cell_grid(v.box_lo, v.box_hi, &sp[i].lo, &sp[i].inv);
    sp[i].spatial = v.spatial && v.p.n >= 2 * kTilePoints ? 1 : 0;
  }
  const int64_t total = off[n];
  if (total > INT32_MAX) return bfail(b, QK_ERR_BAD_SIZE, "more than 2^31 points in one batch");
  {
    cudaError_t e = b->d_sort.ensure(spatial_order_batch_bytes(total, n));
    if (e == cudaSuccess) e = b->d_sort_probs.ensure(sizeof(SortProblem) * n);
    if (e == cudaSuccess) e = b->d_off.ensure(sizeof(int64_t) * (n + 1));
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_sort_probs.p, sp.data(), sizeof(SortProblem) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_off.p, off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(b, e, "batch point order");
  }
  b->order = spatial_order_batch_layout(b->d_sort.p, total, n);
  // tiles per ao_vgl item: about kAoItemsTarget items over the whole batch,
  // so that each item loads its chunk's tables once for many tiles
  int64_t blocks = 0;
  for (int i = 0; i < n; ++i)
    blocks += (views[i].p.n + kTilePoints - 1) / kTilePoints * views[i].b.nchunk;
  const int64_t ao_tiles_per_item = std::max<int64_t>(8, (blocks + kAoItemsTarget - 1) / kAoItemsTarget);
  b->max_tiles = 0;
  b->max_shells = 0;
  std::vector<AOProblem> aop(n);
  std::vector<TcProblem> tcp(n);
  std::vector<PairProblem> pp(b->sm_pairs ? n : 0);
  if (b->sm_pairs) b->d_cpair.resize(n);
  std::vector<int4> ao_items, tc_items;
  std::vector<double> ao_cost, tc_cost;
  for (int i = 0; i < n; ++i) {
    ForwardViews& v = views[i];
    // molecule i's points in the batch order, its AO tensor cut in tiles of
    // that order, output rows written back through the permutation
    PointsDev ps = b->order.sorted;
    ps.n = v.p.n;
    ps.x += off[i];
    ps.y += off[i];
    ps.z += off[i];
    ps.hi += off[i];
    ps.lo += off[i];
    v.ao.perm = b->order.perm + off[i];
    aop[i].b = v.b;
    aop[i].p = ps;
    aop[i].out = v.ao;
    // pairs multiply tiles 2i and 2i + 1 over the union of their live
    // groups: ao_vgl writes zeros into the groups the partner may light
    aop[i].out.pair_zero = b->sm_pairs;
    b->max_tiles = std::max<int64_t>(b->max_tiles, (v.p.n + kTilePoints - 1) / kTilePoints);
    b->max_shells = std::max(b->max_shells, v.b.shell_num);
    int bn = pick_bn(v.mo_num, b->bn_max);
    if (b->sm_pairs) {
      bn = std::max(bn, 32);  // the pair kernel's smallest MMA N
      const int half = b->bn_max / 2;
      cudaError_t e = b->d_cpair[i].ensure(pair_c_bytes(b->mode, v.mo_num, v.kpad, bn, half));
      if (e == cudaSuccess)
        e = launch_pair_c(b->mode, v.c_hi, v.c_lo, v.kpad, v.mo_num, v.kpad, bn, half,
                          b->d_cpair[i].p, b->stream);
      if (e != cudaSuccess) return bcuda(b, e, "blocked C");
      if (!tc_make_pair_problem(b->mode, v.ao, v.kpad, b->d_cpair[i].p, v.mo_num, outs[i], bn,
                                b->bn_max, 5 * v.p.n, &pp[i]))
        return bfail(b, QK_ERR_CUDA, "tensor map encoding failed");
    } else if (!tc_make_problem(b->mode, v.ao, v.kpad, v.c_hi, v.c_lo, v.kpad, v.mo_num, outs[i],
                                bn, 5 * v.p.n, &tcp[i])) {
      return bfail(b, QK_ERR_CUDA, "tensor map encoding failed");
    }
    // ao items: one chunk of every stride-th tile (strided, so that each
    // item samples the whole molecule and items of one molecule cost alike)
    const int64_t tiles = (v.p.n + kTilePoints - 1) / kTilePoints;
    const int64_t stride = std::max<int64_t>(1, (tiles + ao_tiles_per_item - 1) / ao_tiles_per_item);
    for (int q = 0; q < v.b.nchunk; ++q)
      for (int64_t t = 0; t < stride && t < tiles; ++t) {
        ao_items.push_back(make_int4(i, q, (int)t, (int)stride));
        ao_cost.push_back((double)((tiles - t + stride - 1) / stride));
      }
    // contraction items: every (M tile, N tile), or every (M-tile pair, N
    // tile); cost ~ K blocks x MMA N
    const int64_t mt = v.ao.rows / kTileRows, nt = (v.mo_num + bn - 1) / bn;
    const int64_t nm = b->sm_pairs ? (mt + 1) / 2 : mt;
    const int nkb = b->sm_pairs ? pp[i].num_kb : tcp[i].num_kb;
    for (int64_t m = 0; m < nm; ++m)
      for (int64_t k = 0; k < nt; ++k) {
        tc_items.push_back(make_int4(i, (int)m, (int)k, 0));
        tc_cost.push_back((double)nkb * bn);
      }
  }
  // longest first (stable: N tiles of one M tile stay adjacent)
  auto lpt = [](std::vector<int4>& items, const std::vector<double>& cost) {
    std::vector<size_t> idx(items.size());
    for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
    std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
    std::vector<int4> out(items.size());
    for (size_t k = 0; k < idx.size(); ++k) out[k] = items[idx[k]];
    items.swap(out);
  };
  lpt(ao_items, ao_cost);
  lpt(tc_items, tc_cost);
  cudaError_t e = b->d_ao_probs.ensure(sizeof(AOProblem) * n);
  if (e == cudaSuccess) e = b->d_tc_probs.ensure(sizeof(TcProblem) * n);
  if (e == cudaSuccess && b->sm_pairs) e = b->d_pair_probs.ensure(sizeof(PairProblem) * n);
  if (e == cudaSuccess && b->sm_pairs)
    e = cudaMemcpy(b->d_pair_probs.p, pp.data(), sizeof(PairProblem) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = b->d_ao_items.ensure(sizeof(int4) * std::max<size_t>(1, ao_items.size()));
  if (e == cudaSuccess) e = b->d_tc_items.ensure(sizeof(int4) * std::max<size_t>(1, tc_items.size()));
  if (e == cudaSuccess) e = b->d_flag.ensure(256);
  if (e == cudaSuccess) e = cudaMemset(b->d_flag.p, 0, 256);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_ao_probs.p, aop.data(), sizeof(AOProblem) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_tc_probs.p, tcp.data(), sizeof(TcProblem) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !ao_items.empty())
    e = cudaMemcpy(b->d_ao_items.p, ao_items.data(), sizeof(int4) * ao_items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !tc_items.empty())
    e = cudaMemcpy(b->d_tc_items.p, tc_items.data(), sizeof(int4) * tc_items.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bcuda(b, e, "batch descriptors");
  b->n_ao_items = (int64_t)ao_items.size();
  b->n_tc_items = (int64_t)tc_items.size();
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return QK_SUCCESS;
}

// The pointers and sizes the descriptors depend on.
qk_status signature(qk_batch b, float* const* outs, std::vector<uintptr_t>* sig) {
  sig->clear();
  sig->push_back((uintptr_t)b->bn_max);
  sig->push_back((uintptr_t)b->sm_pairs);
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    ForwardViews v;
    if (context_cusp_on(b->ctxs[i]))
      return bfail(b, QK_ERR_NOT_IMPLEMENTED,
                   "context " + std::to_string(i) + " has the cusp correction on");
    qk_status st = context_forward_views(b->ctxs[i], &v);
    if (st) return bfail(b, st, "context " + std::to_string(i) + " is not ready");
    // tables re-uploaded in place (same sizes) keep their addresses: the
    // basis version, the Eq. 3 threshold and the chunking say whether the
    // AO problem copied into the descriptors is still the context's
    sig->push_back((uintptr_t)v.basis_version);
    uint64_t tbits = 0;
    std::memcpy(&tbits, &v.b.T, sizeof tbits);
    sig->push_back((uintptr_t)tbits);
    sig->push_back((uintptr_t)v.b.nchunk);
    sig->push_back((uintptr_t)v.ao.a);
    sig->push_back((uintptr_t)v.ao.a_lo);
    sig->push_back((uintptr_t)v.ao.mask);
    sig->push_back((uintptr_t)v.p.x);
    sig->push_back((uintptr_t)v.p.n);
    sig->push_back((uintptr_t)v.b.chunk);
    sig->push_back((uintptr_t)v.c_hi);
    sig->push_back((uintptr_t)v.mo_num);
    sig->push_back((uintptr_t)v.mo_version);  // C is blocked per upload for pairs
    sig->push_back((uintptr_t)outs[i]);
  }
  return QK_SUCCESS;
}

// The point order, the reach pre-pass and ao_vgl of every molecule.
cudaError_t launch_ao_side(qk_batch b, cudaStream_t s) {
  cudaError_t e = launch_spatial_order_batch(b->order, (const SortProblem*)b->d_sort_probs.p,
                                             (const int64_t*)b->d_off.p, s);
  if (e == cudaSuccess)
    e = launch_tile_reach_batch((const AOProblem*)b->d_ao_probs.p, (int)b->ctxs.size(),
                                b->max_tiles, b->max_shells, s);
  if (e == cudaSuccess)
    e = launch_ao_vgl_batch(b->mode == QK_BF16X3, (const AOProblem*)b->d_ao_probs.p,
                            (const int4*)b->d_ao_items.p, b->n_ao_items, s);
  return e;
}

cudaError_t launch_contraction(qk_batch b, int bn_max, cudaStream_t s) {
  if (b->sm_pairs)
    return launch_mo_tc_pair_batch(b->mode, bn_max, (const PairProblem*)b->d_pair_probs.p,
                                   (const int4*)b->d_tc_items.p, b->n_tc_items, (int*)b->d_flag.p,
                                   s);
  return launch_mo_tc_batch(b->mode, bn_max, (const TcProblem*)b->d_tc_probs.p,
                            (const int4*)b->d_tc_items.p, b->n_tc_items, (int*)b->d_flag.p, s);
}

cudaError_t launch_both(qk_batch b, cudaStream_t s) {
  cudaError_t e = launch_ao_side(b, s);
  if (e != cudaSuccess) return e;
  return launch_contraction(b, b->bn_max, s);
}

qk_status prepare(qk_batch b, float* const* outs, const int64_t* sizes) {
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    if (!outs[i]) return bfail(b, QK_ERR_NULL_POINTER, "output " + std::to_string(i) + " is NULL");
    ForwardViews v;
    if (context_cusp_on(b->ctxs[i]))
      return bfail(b, QK_ERR_NOT_IMPLEMENTED,
                   "context " + std::to_string(i) + " has the cusp correction on");
    qk_status st = context_forward_views(b->ctxs[i], &v);
    if (st) return bfail(b, st, "context " + std::to_string(i) + " is not ready");
    if (v.mode != b->mode)
      return bfail(b, QK_ERR_INVALID_ARG, "context " + std::to_string(i) + " changed mode");
    if (sizes && sizes[i] < 5 * v.p.n * v.mo_num)
      return bfail(b, QK_ERR_BAD_SIZE, "output " + std::to_string(i) + " too small");
  }
  std::vector<uintptr_t> sig;
  qk_status st = signature(b, outs, &sig);
  if (st) return st;
  if (sig != b->signature) {
    st = build(b, outs);
    if (st) return st;
    b->signature = sig;
  }
  return QK_SUCCESS;
}

}  // namespace

extern "C" {

qk_status qk_batch_create(qk_batch* out, int32_t n_ctx, const qk_context* ctxs) {
  if (!out || !ctxs) return QK_ERR_NULL_POINTER;
  if (n_ctx < 1) return QK_ERR_BAD_SIZE;
  qk_batch b = new (std::nothrow) qk_batch_s();
  if (!b) return QK_ERR_OUT_OF_MEMORY;
  for (int i = 0; i < n_ctx; ++i) {
    if (!ctxs[i]) {
      delete b;
      return QK_ERR_NULL_POINTER;
    }
    ForwardViews v;
    qk_status st = context_forward_views(ctxs[i], &v);
    if (st) {
      delete b;
      return st;
    }
    if (v.mode != QK_BF16X3 && v.mode != QK_TF32) {
      delete b;
      return QK_ERR_INVALID_ARG;
    }
    if (i == 0) b->mode = v.mode;
    if (v.mode != b->mode) {
      delete b;
      return QK_ERR_INVALID_ARG;
    }
    b->ctxs.push_back(ctxs[i]);
  }
  *out = b;
  return QK_SUCCESS;
}

qk_status qk_batch_destroy(qk_batch b) {
  if (!b) return QK_ERR_NULL_POINTER;
  delete b;
  return QK_SUCCESS;
}

qk_status qk_batch_last_error(qk_batch b, char* buf, int64_t size) {
  if (!b || !buf) return QK_ERR_NULL_POINTER;
  if (size < 1) return QK_ERR_BAD_SIZE;
  const size_t n = std::min((size_t)(size - 1), b->err.size());
  std::memcpy(buf, b->err.data(), n);
  buf[n] = '\0';
  return QK_SUCCESS;
}

qk_status qk_batch_set_stream(qk_batch b, void* stream) {
  if (!b) return QK_ERR_NULL_POINTER;
  if ((cudaStream_t)stream != b->stream && b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->stream = (cudaStream_t)stream;
  return QK_SUCCESS;
}

qk_status qk_batch_set_graph(qk_batch b, int32_t enable) {
  if (!b) return QK_ERR_NULL_POINTER;
  b->use_graph = enable != 0;
  return QK_SUCCESS;
}

qk_status qk_batch_set_sm_pairs(qk_batch b, int32_t enable) {
  if (!b) return QK_ERR_NULL_POINTER;
  b->sm_pairs = enable != 0;
  return QK_SUCCESS;
}

qk_status qk_batch_set_tile(qk_batch b, int32_t bn_max) {
  if (!b) return QK_ERR_NULL_POINTER;
  bool known = false;
  for (int v : kBatchBnMax) known = known || v == bn_max;
  if (!known) return bfail(b, QK_ERR_INVALID_ARG, "bn_max must be 64, 96, 128, 160, 192 or 256");
  b->bn_max = bn_max;
  return QK_SUCCESS;
}

qk_status qk_batch_get_tile(qk_batch b, int32_t* bn_max) {
  if (!b || !bn_max) return QK_ERR_NULL_POINTER;
  *bn_max = b->bn_max;
  return QK_SUCCESS;
}

qk_status qk_batch_run(qk_batch b, float* const* douts, const int64_t* sizes) {
  if (!b || !douts) return QK_ERR_NULL_POINTER;
  qk_status st = prepare(b, douts, sizes);
  if (st) return st;
  cudaError_t e = cudaSuccess;
  if (b->use_graph) {
    if (!b->graph || b->graph_bn != b->bn_max) {
      if (b->graph) cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
      cudaGraph_t g = nullptr;
      // capture on a private stream, then launch the graph on the batch stream
      cudaStream_t cap = nullptr;
      e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t el = launch_both(b, cap);
        e = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = el;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (cap) cudaStreamDestroy(cap);
      if (e != cudaSuccess) return bcuda(b, e, "batch graph capture");
      b->graph_bn = b->bn_max;
    }
    e = cudaGraphLaunch(b->graph, b->stream);
  } else {
    e = launch_both(b, b->stream);
  }
  if (e != cudaSuccess) return bcuda(b, e, "batch launch");
  for (qk_context c : b->ctxs) context_forget_ao(c);
  return QK_SUCCESS;
}

qk_status qk_batch_synchronize(qk_batch b) {
  if (!b) return QK_ERR_NULL_POINTER;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "batch synchronize");
  int flag = 0;
  if (b->d_flag.p) {
    e = cudaMemcpy(&flag, b->d_flag.p, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "batch error flag");
  }
  if (flag != 0) {
    cudaMemset(b->d_flag.p, 0, sizeof(int));
    return bfail(b, QK_ERR_DEVICE_TIMEOUT, "a device-side wait gave up");
  }
  return QK_SUCCESS;
}

qk_status qk_batch_autotune(qk_batch b, float* const* douts, int32_t reps, double* best_ms) {
  if (!b || !douts) return QK_ERR_NULL_POINTER;
  if (reps < 1) reps = 3;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return bcuda(b, e, "autotune events");
  const int keep_bn = b->bn_max;
  const bool keep_graph = b->use_graph;
  b->use_graph = false;
  double best = 1e300;
  int best_bn = keep_bn;
  qk_status st = QK_SUCCESS;
  for (int bn : kBatchBnMax) {
    b->bn_max = bn;
    st = prepare(b, douts, nullptr);
    if (st) break;
    // the AO tensors are filled once; only the contraction is timed
    e = launch_ao_side(b, b->stream);
    for (int r = 0; r < reps + 1 && e == cudaSuccess; ++r) {
      if (r == 1) e = cudaEventRecord(e0, b->stream);
      if (e == cudaSuccess) e = launch_contraction(b, bn, b->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaErrorInvalidConfiguration) {  // this tile does not fit: skip it
      cudaGetLastError();
      e = cudaSuccess;
      continue;
    }
    if (e != cudaSuccess) {
      st = bcuda(b, e, "autotune");
      break;
    }
    if (ms / reps < best) {
      best = ms / reps;
      best_bn = bn;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->bn_max = best_bn;
  b->use_graph = keep_graph;
  if (st) return st;
  st = qk_batch_synchronize(b);
  if (st) return st;
  if (best_ms) *best_ms = best;
  return QK_SUCCESS;
}

}  // extern "C"
