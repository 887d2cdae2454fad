/*
 * qmckl_gpu.h -- C ABI of the GB300 (sm_103a) AO/MO "vgl" library.
 *
 * The library evaluates, at every electron of a batch of walkers, the values,
 * gradients and Laplacians ("vgl") of contracted Gaussian atomic orbitals and
 * of the molecular orbitals built from them, following the QMCkl paper
 * (arXiv 2512.16677):
 *
 *   chi_n(r)  = M_n R_s(r) P_abc(r - R_A)                      Sec. 3.1, Eq. 1
 *   R_s(r)    = N_s sum_k a_ks f_ks exp(-gamma_ks |r - R_A|^2)  Eq. 2 (p = 2, n_s = 0)
 *   screening: primitive k is evaluated only if
 *              gamma_ks |r - R_A|^2 < T,  T = (B-1) ln 2        Eq. 3
 *   P_abc     = (x-X_A)^a (y-Y_A)^b (z-Z_A)^c                   Eq. 4
 *   phi_i, grad phi_i, lap phi_i = sum_k C_ik (chi_k, grad chi_k, lap chi_k)
 *                                                              Sec. 3.2, Eqs. 5-7
 *
 * The calling sequence follows the paper's usage (Sec. 2.2 context and
 * memoisation, Sec. 2.3 C ABI, Sec. 5.1 example): create a context, set the
 * nuclei, the shells and primitives and the MO coefficients, set the points,
 * then get the MO vgl.  Units: bohr for lengths, bohr^-2 for exponents.
 *
 * Conventions shared by every call:
 *  - Every function returns a qk_status: QK_SUCCESS (0) or a negative code.
 *    On failure the context keeps a message, read with qk_last_error.
 *    Outputs are left untouched when an argument is rejected.
 *  - Setters copy host inputs; the caller keeps ownership of its arrays.
 *    The context owns its device tables and frees them in
 *    qk_context_destroy.
 *  - Arrays are C order (row-major).  Cartesian components within a shell
 *    are ordered by descending a, then descending b (l = 2: xx, xy, xz, yy,
 *    yz, zz).  vgl outputs are [walk][elec][5][n] with the five components
 *    (value, d/dx, d/dy, d/dz, Laplacian).
 *  - Element type of AO/MO outputs and of loss weights: double in QK_FP64
 *    mode, float in every other mode.
 *  - A context is not thread-safe (Sec. 2.4); separate contexts may be used
 *    concurrently.  All device work of a context runs on its stream (the
 *    legacy default stream unless qk_set_stream is called).
 */
#ifndef QMCKL_GPU_H
#define QMCKL_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t qk_status;

#define QK_SUCCESS 0
#define QK_ERR_INVALID_ARG -1      /* a value is out of its domain */
#define QK_ERR_NULL_POINTER -2     /* a required pointer is NULL */
#define QK_ERR_BAD_SIZE -3         /* a size argument is too small or inconsistent */
#define QK_ERR_NOT_PROVIDED -4     /* a required setter has not been called */
#define QK_ERR_NOT_IMPLEMENTED -5  /* valid input outside what the library implements */
#define QK_ERR_CUDA -6             /* a CUDA runtime/driver call failed */
#define QK_ERR_DEVICE_TIMEOUT -7   /* a bounded device-side wait gave up */
#define QK_ERR_OUT_OF_MEMORY -8    /* device or host allocation failed */

/* Arithmetic of the evaluation (qk_set_compute_mode). */
#define QK_FP64 0    /* FP64 AOs and FP64 contraction: the accuracy anchor */
#define QK_FP32 1    /* FP32 AOs (FP64 coordinate differences) and FP32 SIMT contraction */
#define QK_BF16X3 2  /* FP32 AOs split into bf16 hi+lo, contraction on tcgen05 tensor
                        cores as hi*hi + hi*lo + lo*hi with FP32 accumulation */
#define QK_TF32 3    /* FP32 AOs, contraction on tcgen05 tensor cores in TF32 */

typedef struct qk_context_s* qk_context;
typedef struct qk_batch_s* qk_batch;

/* ----------------------------------------------------------- lifetime --- */

/* Create a context on the current CUDA device (Sec. 2.2: the context holds all
   inputs, cached intermediates and their time stamps).  *out receives the
   handle.  Errors: QK_ERR_NULL_POINTER, QK_ERR_OUT_OF_MEMORY, QK_ERR_CUDA. */
qk_status qk_context_create(qk_context* out);

/* Free the context and every device table it owns.  A NULL handle is
   QK_ERR_NULL_POINTER.  Caller-owned workspace is not freed. */
qk_status qk_context_destroy(qk_context ctx);

/* Copy the last error message (NUL-terminated, truncated to size) into buf. */
qk_status qk_last_error(qk_context ctx, char* buf, int64_t size);

/* ----------------------------------------------------------- settings --- */

/* Precision parameter B of Eq. 3 (default 53): primitives with
   gamma r^2 >= (B-1) ln 2 are skipped.  2 <= bits <= 53, else
   QK_ERR_INVALID_ARG.  Clears a cutoff set by qk_set_cutoff. */
qk_status qk_set_precision(qk_context ctx, int32_t bits);

/* Alternative to B: skip primitives with exp(-gamma r^2) <= eps, i.e.
   T = ln(1/eps).  0 < eps < 1, else QK_ERR_INVALID_ARG. */
qk_status qk_set_cutoff(qk_context ctx, double eps);

/* One of QK_FP64, QK_FP32, QK_BF16X3, QK_TF32 (default QK_FP64). */
qk_status qk_set_compute_mode(qk_context ctx, int32_t mode);

/* QK_BF16X3 only: 1 builds the AO blocks inside the tensor-core contraction
   kernel, in shared memory, so no AO tensor goes through HBM; 0 (default)
   runs ao_vgl and the contraction as two kernels through an AO tensor in the
   workspace.  Both give the same arithmetic.  Other modes ignore it. */
qk_status qk_set_fusion(qk_context ctx, int32_t enable);

/* Internal order of the shells (a layout choice of this library, not a
   step of the paper's method).  AO chunks and the contraction's 16-AO
   column groups are cut from consecutive shells, and blocks and groups
   that no point of a tile reaches are skipped, so the shells of a group
   should be close in space and alike in screening radius.
   Nuclei, mode 0 (default): in Morton (Z-curve) order when that shortens
   the path through the nuclei in shell order below 0.7 of the caller's
   order (bases listed in random atom order), else in the caller's order;
   mode 2: always in Morton order.  In both modes the shells are then split
   stably into a compact class (minimum exponent >= that of the shell
   holding the AO-weighted median) followed by a diffuse class.
   Mode 1: the caller's shell order as it is.  Takes effect at the next
   qk_set_ao_basis.  Every input and output keeps the caller's AO order
   (C columns, AO tensors, dL/dC).  Other values: QK_ERR_INVALID_ARG.
   qk_get_basis_order: *spatial = 1 when the current basis takes its
   nuclei in Morton order.
   qk_get_shell_order: order[i] = the caller's shell at internal position
   i (n >= shell_num, else QK_ERR_BAD_SIZE; QK_ERR_NOT_PROVIDED before a
   basis). */
qk_status qk_set_basis_order(qk_context ctx, int32_t mode);
qk_status qk_get_basis_order(qk_context ctx, int32_t* spatial);
qk_status qk_get_shell_order(qk_context ctx, int64_t* order, int64_t n);

/* QK_BF16X3 / QK_TF32, device-memory calls: 1 (default) cuts the point tiles
   of the block-sparse contraction from a spatial (Morton cell) order of the
   points, so that a tile's points share their nonzero AOs and fewer
   (tile, AO chunk) blocks are multiplied; outputs stay in the caller's
   point order and every value is the same as with 0, which cuts tiles in
   the caller's order.  This is a layout choice of this library, not a step
   of the paper's method.  Other modes and the host-memory calls ignore it. */
qk_status qk_set_spatial_order(qk_context ctx, int32_t enable);

/* Tensor-core modes, two-kernel path: 1 (default) runs the contraction of
   Eqs. 5-7 on pairs of SMs (one tcgen05 MMA with M = 256 over two
   consecutive point tiles, each SM holding half of the C tile), 0 on single
   SMs.  Both multiply the same live blocks; a pair multiplies the union of
   its two tiles' live column groups, whose extra terms are exact zeros, so
   the results are the same.  A layout choice of this library, not a step
   of the paper's method. */
qk_status qk_set_sm_pairs(qk_context ctx, int32_t enable);

/* MO cusp correction (Sec. 3.3).  rc [nucl_num]: sphere radius in bohr
   around each nucleus (>= 0, 0 = no correction there); NULL switches the
   correction off.  Inside the sphere of A every MO output becomes
   phi - phi^{s_A} + f_0 + f_1 rho + f_2 rho^2 + f_3 rho^3 (rho = |r - R_A|,
   phi^{s_A} the part of the MO carried by the s AOs on A), with value
   gradient and Laplacian of that expression.  The f_k (per nucleus and MO)
   make value, first and second radial derivative continuous at rc and
   satisfy Kato's cusp f_1 = -Z_A (phi(R_A) - phi^{s_A}(R_A) + f_0); the
   paper names the first two conditions and the cusp, the second-derivative
   one is this library's reading.  Z_A is the charge given to
   qk_set_nucleus.  The coefficients are set up in FP64 on the device and
   the correction is added in FP64 to the output of every MO call.  A point
   exactly on a nucleus gets an infinite Laplacian.  Copies rc; changing the
   number of nuclei switches the correction off.  Non-finite or negative
   radii are QK_ERR_INVALID_ARG; more than 32 s shells on one nucleus gives
   QK_ERR_NOT_IMPLEMENTED at the next evaluation, as do
   qk_mo_vgl_backward_device and multi-molecule batches on a context with
   the correction on. */
qk_status qk_set_mo_cusp(qk_context ctx, const double* rc);

/* Single-electron moves (the usage of Sec. 4, CHAMP: one electron of every
   walker moved, its MOs needed at the proposed position).
   qk_set_single_point_device: dcoord [walk_num][3] (device, bohr) are the
   proposed positions of electron `elec` (0 <= elec < elec_num, else
   QK_ERR_INVALID_ARG) in each walker; copied.  The context's points are not
   changed and its cached AO tensor stays valid.
   qk_get_mo_vgl_single_device: MO vgl [walk_num][5][mo_num] at the proposed
   positions (FP64 in QK_FP64 mode, else FP32), with the same arithmetic as
   qk_get_mo_vgl_device (so each row equals the row the full evaluation gives
   that point), cusp correction included; size >= 5 * walk_num * mo_num.
   qk_accept_single_point: the proposed positions replace electron `elec`
   of every walker in the context's points (a new time stamp).
   QK_ERR_NOT_PROVIDED without a proposal. */
qk_status qk_set_single_point_device(qk_context ctx, int64_t elec, const double* dcoord);
qk_status qk_get_mo_vgl_single_device(qk_context ctx, void* dout, int64_t size);
qk_status qk_accept_single_point(qk_context ctx);

/* Electron density on the current points (Sec. 5.4, e.g. a grid):
   rho(p) = sum_i w[i] phi_i(p)^2 with the MO values of Eqs. 5-7 (no
   derivatives are formed).  w [mo_num] (host, copied): occupation weights,
   e.g. 2 for doubly occupied MOs; MOs with w = 0 cost nothing.  drho
   [point_num] on the device, FP64 in QK_FP64 mode and FP32 otherwise;
   size >= point_num.  The tensor-core modes contract values-only AO tiles
   of 128 points and reduce sum w phi^2 in the contraction's epilogue; the
   FP64 / FP32 modes go through the SIMT GEMM.  Runs on the context's stream
   after a short synchronisation (the weights' upload); uses the AO
   workspace, so the next MO call evaluates its AOs again.  The cusp
   correction does not apply.  Non-finite weights are QK_ERR_INVALID_ARG. */
qk_status qk_get_density_device(qk_context ctx, const double* w, void* drho, int64_t size);

/* The coefficients f [nucl_num][mo_num][4] (device memory, FP64) of the
   current cusp correction; size >= 4 * nucl_num * mo_num.  QK_ERR_NOT_PROVIDED
   without radii. */
qk_status qk_get_mo_cusp_coefficients_device(qk_context ctx, double* df, int64_t size);

/* ------------------------------------------------------------- system --- */

/* Nuclei (Sec. 3.1): charge [nucl_num] (kept for reference only) and
   coord [nucl_num][3] in bohr.  nucl_num >= 1.  Non-finite coordinates are
   QK_ERR_INVALID_ARG.  Resets the basis if nucl_num changed. */
qk_status qk_set_nucleus(qk_context ctx, int64_t nucl_num, const double* charge,
                         const double* coord);

/* Contracted Gaussian shells (Eqs. 1, 2, 4).
   shell_nucleus [shell_num]  nucleus of each shell, 0 <= . < nucl_num
   shell_ang_mom [shell_num]  l, 0 <= l <= 3 (l > 3: QK_ERR_NOT_IMPLEMENTED)
   shell_prim_num [shell_num] primitives per shell, >= 1; primitives are
                              stored shell after shell
   shell_factor [shell_num]   N_s
   exponent, coefficient, prim_factor [prim_num]: gamma_ks > 0, a_ks, f_ks
   ao_num = sum over shells of (l+1)(l+2)/2, else QK_ERR_BAD_SIZE
   ao_factor [ao_num]         M_n
   The primitives of each shell are sorted by ascending exponent inside the
   library (Sec. 3.1); results do not depend on the input order.
   Requires qk_set_nucleus first (QK_ERR_NOT_PROVIDED). */
qk_status qk_set_ao_basis(qk_context ctx, int64_t shell_num, int64_t prim_num,
                          const int64_t* shell_nucleus, const int32_t* shell_ang_mom,
                          const int64_t* shell_prim_num, const double* shell_factor,
                          const double* exponent, const double* coefficient,
                          const double* prim_factor, int64_t ao_num,
                          const double* ao_factor);

/* MO coefficients C [mo_num][ao_num] (Eqs. 5-7).  Passing only the occupied
   MOs is the paper's MO-subset selection (Sec. 3.2).  Requires the basis. */
qk_status qk_set_mo_coefficient(qk_context ctx, int64_t mo_num, const double* coef);

/* ------------------------------------------------------------- points --- */

/* Electron coordinates from host memory.  transp 'N': coord [walk][elec][3];
   'T': coord [3][walk*elec].  walk_num, elec_num >= 1.  Bumps the context's
   time stamp, which invalidates every cached intermediate (Sec. 2.2). */
qk_status qk_set_points(qk_context ctx, char transp, int64_t walk_num, int64_t elec_num,
                        const double* coord);

/* Same, from device memory (read on the context's stream before return of
   the next get; the caller keeps the buffer alive until then). */
qk_status qk_set_points_device(qk_context ctx, char transp, int64_t walk_num,
                               int64_t elec_num, const double* dcoord);

/* --------------------------------------------------------------- sizes --- */

qk_status qk_get_nucl_num(qk_context ctx, int64_t* n);
qk_status qk_get_ao_num(qk_context ctx, int64_t* n);
qk_status qk_get_mo_num(qk_context ctx, int64_t* n);
qk_status qk_get_point_num(qk_context ctx, int64_t* n);

/* ---------------------------------------------------------- workspace --- */

/* Device bytes the next evaluation needs (points, mode and basis must be
   set).  The workspace holds the coordinate copies and the AO tensor. */
qk_status qk_workspace_size(qk_context ctx, size_t* bytes);

/* Caller-owned device workspace (e.g. a torch allocation), 256-byte
   aligned, at least qk_workspace_size bytes (QK_ERR_BAD_SIZE otherwise).
   Once set, the library allocates nothing per evaluation.  NULL reverts to
   library-owned workspace. */
qk_status qk_set_workspace(qk_context ctx, void* dev, size_t bytes);

/* Stream for all device work of this context (a cudaStream_t). */
qk_status qk_set_stream(qk_context ctx, void* stream);

/* Synchronise the context's stream and report device-side errors (bounded
   waits that gave up: QK_ERR_DEVICE_TIMEOUT). */
qk_status qk_synchronize(qk_context ctx);

/* Profiling aid (no counterpart in the paper): when enabled, the library
   records a CUDA event pair on the context's stream around every launch,
   in three classes: 0 = ao_vgl, 1 = MO contraction, 2 = other (point
   layout).  Enabling or disabling resets the record. */
qk_status qk_set_timing(qk_context ctx, int32_t enable);

/* Wait for the recorded events and return, for classes 0..n-1, the summed
   device time in ms and the number of launches since the last reset; then
   reset.  1 <= n <= 3, else QK_ERR_BAD_SIZE. */
qk_status qk_get_timing(qk_context ctx, double* ms, int64_t* launches, int32_t n);

/* Kernel launches the context made in the timed classes above (whether or
   not timing is enabled) since the last call; then reset. */
qk_status qk_get_kernel_count(qk_context ctx, int64_t* count);

/* Block sparsity of the AO tensor of the current points (tensor-core modes,
   after a get_mo_vgl at this time stamp; else QK_ERR_NOT_PROVIDED).  Points
   are grouped in tiles of 25 and AOs in chunks of <= 64; a block is live
   when any primitive of its shells passed Eq. 3 at any of its points.
   live_entries = sum over live blocks of (points x AOs) of the block: the
   (point, AO) pairs the contraction multiplies.  Synchronises the stream. */
qk_status qk_get_block_stats(qk_context ctx, int64_t* live_blocks, int64_t* total_blocks,
                             int64_t* live_entries);

/* Finer sparsity of the same AO tensor (two-kernel tensor-core path, after
   a get_mo_vgl at this time stamp; else QK_ERR_NOT_PROVIDED).
   live_groups = (tile, 16-AO column group) pairs holding an entry that
   survived Eq. 3 screening: the contraction issues its tensor-core
   k-steps over these only.  nnz = sum over points p of nnz_AO(p), the
   (point, AO) pairs with any nonzero component (Sec. 3.2's sparse MO
   product needs 2 * 5 * mo_num * nnz flops).  Runs a counting kernel and
   synchronises the stream. */
qk_status qk_get_sparsity_stats(qk_context ctx, int64_t* live_groups, int64_t* nnz);

/* Tile layout of the same AO tensor (tensor-core path, after a get_mo_vgl at
   this time stamp; else QK_ERR_NOT_PROVIDED), for tests and profiling:
   perm[s] (host int32, n >= point_num) = the caller's point held by point
   slot s (slots 25 t .. 25 t + 24 make contraction tile t: the spatial
   order of the points, or the identity when it is off); live[t] (host
   int32, ntiles >= ceil(point_num / 25)) = the (tile, AO chunk) blocks of
   tile t holding an entry that survived Eq. 3; groups (host uint8,
   gsize >= ntiles * nchunk, nchunk = ceil(padded AO columns / 64)) =
   [tile][chunk] bit g set when 16-AO column group g of the block holds
   such an entry.  Any of the three may be NULL.  Synchronises the
   context's stream. */
qk_status qk_get_tile_layout(qk_context ctx, int32_t* perm, int64_t n, int32_t* live,
                             int64_t ntiles, uint8_t* groups, int64_t gsize);

/* Number of 64-column AO chunks of the current basis (the contraction's K
   blocks; chunks end on shell boundaries, so it may exceed ao_num / 64). */
qk_status qk_get_ao_chunk_num(qk_context ctx, int64_t* nchunk);

/* ----------------------------------------------------------- evaluate --- */

/* AO vgl [walk][elec][5][ao_num] into host memory; size = number of elements
   the buffer holds (>= point_num*5*ao_num, else QK_ERR_BAD_SIZE).
   Blocks until the copy is done. */
qk_status qk_get_ao_vgl(qk_context ctx, void* out, int64_t size);

/* Same into device memory on the context's stream (asynchronous). */
qk_status qk_get_ao_vgl_device(qk_context ctx, void* dout, int64_t size);

/* MO vgl [walk][elec][5][mo_num] into host memory (Eqs. 5-7); size as above
   with mo_num.  Blocks until the copy is done. */
qk_status qk_get_mo_vgl(qk_context ctx, void* out, int64_t size);

/* Same into device memory on the context's stream (asynchronous).  The AO
   tensor is memoised: a second call at the same time stamp and mode reuses
   it and runs only the contraction (Sec. 2.2). */
qk_status qk_get_mo_vgl_device(qk_context ctx, void* dout, int64_t size);

/* The contraction of Eqs. 5-7 on a caller-supplied tensor, without a
   context: D[m][n] = sum_k A[m][k] B[n][k], A [M][K], B [N][K], D [M][N]
   row-major in device memory; double in QK_FP64 mode, float otherwise.
   mode selects the kernel (QK_BF16X3 splits A and B into bf16 hi/lo planes
   first).  Runs on `stream` (a cudaStream_t, NULL = legacy default);
   tensor-core modes synchronise the stream to read the device error word.
   Scratch is library-owned and shared by all calls: not thread-safe.
   Errors: QK_ERR_NULL_POINTER, QK_ERR_BAD_SIZE (K < 1 or a negative size),
   QK_ERR_INVALID_ARG (mode), QK_ERR_DEVICE_TIMEOUT, QK_ERR_CUDA. */
qk_status qk_contract_device(int32_t mode, int64_t M, int64_t N, int64_t K, const void* A,
                             const void* B, void* D, void* stream);

/* Allocation-free variant of qk_contract_device for the tensor-core modes.
   The paper has no counterpart: this entry point exists for callers that
   cannot call cudaMalloc (a framework or memory pool owns the device memory
   budget, a latency-critical loop cannot take the synchronisation that
   cudaMalloc/cudaFree imply, or the caller must not fail for lack of memory
   once started).  Same arguments and result as qk_contract_device, with
   mode QK_BF16X3 or QK_TF32 (else QK_ERR_INVALID_ARG) and float data.
   Scratch: a fixed 32 MiB device array inside the library, which every GPU
   that loads the library holds until the process exits.  Limit:
     256 + planes * (round256(M*ld*es) + round256(N*ld*es)) <= 32 MiB,
   ld = K rounded up to a multiple of 8; bf16x3: planes 2, es 2; tf32:
   planes 1, es 4; so about (M + N) * ld <= 8.38e6.  Larger problems are
   refused with QK_ERR_BAD_SIZE before any work is queued.
   The first call on a device looks up the array's device address (once per
   device and CUDA context, with that device current: again after a device
   reset).  All calls share the one array and it keeps the previous call's
   contents (the error word is cleared on every call): calls that overlap on
   the GPU race, so serialise them (one stream, or events).  Every call
   synchronises `stream` to read the error word, so no call can be made
   while that stream is being captured into a CUDA graph.  Allocates no
   device or host memory. */
qk_status qk_contract_device_noalloc(int32_t mode, int64_t M, int64_t N, int64_t K,
                                     const float* A, const float* B, float* D, void* stream);

/* Self-test of the bounded device-side waits (the paper has no counterpart:
   every tcgen05 kernel here waits on mbarriers with a clock limit, and a
   wait that gives up records a code in the caller's error word, which the
   host reports as QK_ERR_DEVICE_TIMEOUT).  One small kernel waits on an
   mbarrier that nothing arrives at: one thread with limit_cycles (1 ..
   1e8 SM clock cycles, else QK_ERR_BAD_SIZE), which gives up and raises the
   CTA's abort flag, and one with the library's normal limit (about 2 s),
   which must leave through that flag.  Returns QK_ERR_DEVICE_TIMEOUT when
   the short wait gave up as it should (QK_SUCCESS would mean it did not).
   info (host, 4 int32, may be NULL): [0] the error word, [1] 1 if the
   second waiter left through the abort flag (2: by its own limit),
   [2], [3] the cycles each waiter spent.  Allocates 16 bytes of device
   memory; synchronises the device. */
qk_status qk_selftest_wait_timeout(int64_t limit_cycles, int32_t* info);

/* ------------------------------------------------------------ adjoint --- */

/* Gradients of L = sum_{p,c,i} W[p][c][i] * mo_vgl[p][c][i] at the current
   points (Sec. 3.6 needs nuclear derivatives of the orbitals up to third
   order).  dW has the mo_vgl layout and element type, in device memory.
   d_dC [mo_num][ao_num] (dL/dC) and d_dR [nucl_num][3] (dL/dR_nuc) are
   device FP64 arrays; either may be NULL to skip it.  QK_FP64 and QK_FP32
   / QK_TF32 recompute the AO values densely and multiply with SIMT GEMMs.
   QK_BF16X3 multiplies on the tensor cores over the block-sparse AO tensor
   of the current points: the one the last forward call left in the
   workspace, else one computed here (it is kept, as a forward call keeps
   it); its derivatives for dL/dR_nuc are recomputed.  Runs on the
   context's stream. */
qk_status qk_mo_vgl_backward_device(qk_context ctx, const void* dW, int64_t size,
                                    double* d_dC, double* d_dR);

/* Device bytes qk_mo_vgl_backward_device needs beyond the forward workspace
   (it allocates them itself unless qk_set_workspace covered both sizes). */
qk_status qk_backward_workspace_size(qk_context ctx, size_t* bytes);

/* ------------------------------------------------------------- batch --- */
/* Walkers of several molecules of uneven sizes, evaluated together: one
   persistent ao_vgl launch over (molecule, AO chunk, point tiles) items and
   one persistent tcgen05 contraction over (molecule, M tile, N tile) items,
   each ordered longest first, captured once in a CUDA graph and replayed.
   The paper evaluates one system per context (Sec. 2.2); a batch runs the
   same Eqs. 1-7 for each of its contexts. */

/* Create a batch over n_ctx contexts, each with nuclei, basis, MO
   coefficients and points set, all in QK_BF16X3 or all in QK_TF32 mode
   (else QK_ERR_INVALID_ARG; unset inputs: QK_ERR_NOT_PROVIDED).  The batch
   keeps the handles, not copies: the contexts must outlive it, and their
   points may be updated between runs (qk_set_points*). */
qk_status qk_batch_create(qk_batch* out, int32_t n_ctx, const qk_context* ctxs);
qk_status qk_batch_destroy(qk_batch b);
qk_status qk_batch_last_error(qk_batch b, char* buf, int64_t size);

/* Stream for the batch's launches (a cudaStream_t; NULL = legacy default).
   Point updates of the contexts must be ordered before a run on it. */
qk_status qk_batch_set_stream(qk_batch b, void* stream);

/* 1 (default): capture the two launches in a CUDA graph on the first run and
   replay it; 0: plain launches. */
qk_status qk_batch_set_graph(qk_batch b, int32_t enable);

/* 1 (default): the batch's contraction multiplies pairs of point tiles on
   pairs of SMs (tcgen05.mma.cta_group::2), as qk_set_sm_pairs does for one
   context; 0: one tile per SM.  Both give the same values.  Takes effect at
   the next run (descriptors and graph are rebuilt).  Sec. 3.2's one-GEMM
   contraction; the pairing is a GPU execution choice with no counterpart
   in the paper. */
qk_status qk_batch_set_sm_pairs(qk_batch b, int32_t enable);

/* Largest MMA N of the contraction (64, 96, 128, 160, 192 or 256; default
   160).  Each molecule uses the smallest multiple of 16 that covers its MOs
   in the fewest N tiles under this bound (at least 32 on pairs of SMs). */
qk_status qk_batch_set_tile(qk_batch b, int32_t bn_max);
qk_status qk_batch_get_tile(qk_batch b, int32_t* bn_max);

/* Evaluate the MO vgl of every context: douts[i] is a device float array
   [walk][elec][5][mo] of context i holding at least sizes[i] elements
   (sizes may be NULL).  Asynchronous on the batch stream. */
qk_status qk_batch_run(qk_batch b, float* const* douts, const int64_t* sizes);

/* Wait for the batch stream; QK_ERR_DEVICE_TIMEOUT if a bounded device wait
   gave up. */
qk_status qk_batch_synchronize(qk_batch b);

/* Autotuner: time the contraction for every instantiated bn_max on this
   batch (reps timed launches each, after one warm-up) and keep the fastest;
   *best_ms (optional) receives its time per launch.  Writes douts. */
qk_status qk_batch_autotune(qk_batch b, float* const* douts, int32_t reps, double* best_ms);

#ifdef __cplusplus
}
#endif

#endif /* QMCKL_GPU_H */
