/*
 * cdl.h -- C ABI of the GB300 (sm_103a) CADDeLaG hot path.
 *
 * The library computes, on one GPU, the commute-time embedding of dense,
 * fully connected similarity graphs and the CAD anomaly scores between two
 * graphs (Basak, Das, Mengshoel, "CADDeLaG: Framework for distributed anomaly
 * detection in large dense graph sequences", arXiv 1802.05421):
 *
 *   cdl_build_graph   Gaussian-kernel graph A, degrees D = A 1, volume
 *                     (Sec. 2; kernel of Sec. 4.2.1; D = A 1 of Sec. 3.2)
 *   cdl_chain_build   inverse-chain levels of Alg. 2, ChainProduct
 *   cdl_project       random projection Y = (Q W^{1/2} B)^T of Alg. 1 / Alg. 3
 *   cdl_chain_solve   L Z = Y by chain-preconditioned Richardson iteration
 *                     (Alg. 2, EstimateSolution; multi-RHS loop of Sec. 4.1)
 *   cdl_cad_score     node scores F_i = sum_j |A1-A2|_ij |c2-c1|_ij and the
 *                     top anomalies (Alg. 4; CAD edge score of Sec. 2)
 *   cdl_caddelag_pair the whole of Alg. 4 for one graph pair
 *
 * Conventions (all entry points):
 *  - Return value: CDL_OK (0) or a negative CDL_ERR_* status.
 *  - Pointers named "device" are CUDA device pointers on the context's
 *    device; "host" pointers are ordinary host memory. The caller owns every
 *    pointer it passes. The library owns cdl_ctx, cdl_chain and the
 *    workspace inside them, and nothing else.
 *  - Matrices are dense and row-major: element (i, j) of an n x n matrix is
 *    at i * n + j; Y and Z (n x k) hold node i's k values in row i.
 *  - Work is enqueued asynchronously on the context's stream unless the
 *    entry point says it synchronises. cdl_sync() waits and reports deferred
 *    device errors. A call that fails validation launches nothing.
 *  - There is no CPU fallback and no silent change of precision.
 */
#ifndef CDL_H
#define CDL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
  CDL_OK = 0,
  CDL_ERR_INVALID_ARG = -1,   /* bad size, null or misaligned pointer, bad enum  */
  CDL_ERR_OOM = -2,           /* device allocation failed or workspace cap hit   */
  CDL_ERR_CUDA = -3,          /* a CUDA runtime/driver call failed               */
  CDL_ERR_NOT_CONVERGED = -4, /* solve stopped at max_iter above rel_tol         */
  CDL_ERR_TIMEOUT = -5,       /* a bounded device-side wait expired              */
  CDL_ERR_UNSUPPORTED = -6    /* valid request the library does not implement    */
};

typedef enum {
  CDL_F64 = 0,      /* IEEE binary64                                    */
  CDL_F32 = 1,      /* IEEE binary32                                    */
  CDL_BF16 = 2,     /* bfloat16, tensor-core chain (tcgen05)            */
  CDL_FP8E4M3 = 3,  /* float8 e4m3 with one scale per level (tcgen05)   */
  CDL_FP8E4M3_T128 = 4  /* float8 e4m3, one scale per 128 x 128 tile    */
} cdl_dtype;

typedef struct cdl_ctx cdl_ctx;
typedef struct cdl_chain cdl_chain;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`. `cuda_stream` is a borrowed
 * cudaStream_t (NULL = the legacy default stream); every kernel of every call
 * on this context is launched on it. `ws_cap_bytes` caps the device workspace
 * the context may allocate (0 = no cap); a call that would exceed it returns
 * CDL_ERR_OOM without launching. *out receives the context. */
int cdl_ctx_create(cdl_ctx** out, int device, void* cuda_stream, size_t ws_cap_bytes);

/* Synchronise the stream, free all workspace and the context. NULL is a no-op. */
int cdl_ctx_destroy(cdl_ctx* ctx);

/* Wait for all work on the context's stream; returns CDL_ERR_CUDA on a
 * deferred device error and CDL_ERR_TIMEOUT if a kernel reported an expired
 * bounded wait (the kernel returned early; the context stays usable). */
int cdl_sync(cdl_ctx* ctx);

/* Static, human-readable name of a status code. */
const char* cdl_status_string(int status);

/* Text of the last CUDA failure recorded by the calling thread (the CUDA
 * error string and where it was caught); empty if none. Diagnostics only. */
const char* cdl_last_error_detail(void);

/* Kernel-class timing. With timing enabled (nonzero), every launch is
 * bracketed by CUDA events on the context's stream and its duration is
 * added to the class totals when they are read. `cdl_ctx_timing` synchronises
 * and returns, for class `kernel_class` (CDL_KC_*), the summed device time in
 * ms, the number of launches and the algorithmic work (flops or bytes, see
 * CDL_KC_*) those launches performed. `cdl_ctx_reset_counters` zeroes all
 * class totals and the launch counter. */
enum {
  CDL_KC_DISTANCE = 0,   /* pairwise squared distances; work = n^2/2 T terms  */
  CDL_KC_SELECT = 1,     /* median radix select; work = bytes read             */
  CDL_KC_KERNEL = 2,     /* exp kernel + degrees; work = bytes moved           */
  CDL_KC_CHAIN_INIT = 3, /* deflated level-0 formation; work = bytes moved     */
  CDL_KC_SQUARE = 4,     /* chain squaring GEMM; work = flops (n^2 (n+1))      */
  CDL_KC_APPLY = 5,      /* chain apply GEMM; work = bytes of levels read      */
  CDL_KC_RESIDUAL = 6,   /* Y - L Z; work = multiply-adds n^2 k                */
  CDL_KC_PROJECT = 7,    /* random projection; work = n(n-1) k signed adds     */
  CDL_KC_SCORE = 8,      /* CAD scores; work = bytes of A1, A2 read            */
  CDL_KC_TOPK = 9,
  CDL_KC_MISC = 10,      /* small vector kernels (norms, centring, updates)    */
  CDL_KC_HOST_LINK = 11, /* chain levels copied over the host link (CDL_CHAIN_HOST_LEVELS):
                            copies, not kernels: "launches" counts copies and the
                            launch counter excludes them; ms = summed copy time on
                            the chain's copy stream; work = bytes copied           */
  CDL_KC_COUNT = 12
};
int cdl_ctx_set_timing(cdl_ctx* ctx, int enable);
int cdl_ctx_timing(cdl_ctx* ctx, int kernel_class, double* total_ms, int64_t* launches,
                   double* work);
int cdl_ctx_reset_counters(cdl_ctx* ctx);
/* Total kernels this context launched since creation or the last reset. */
int cdl_ctx_launch_count(cdl_ctx* ctx, int64_t* launches);

/* Test hooks (0 = none). CDL_DEBUG_WITHHOLD_TC_LOAD: the next tensor-core
 * squarings never issue their first tile load, so the kernel's bounded wait
 * for it expires (about 2 s); the kernel records the expiry and returns, and
 * cdl_sync reports CDL_ERR_TIMEOUT. Used to test the bounded-wait path; the
 * outputs of such a launch are meaningless. CDL_DEBUG_BATCH_VARIANT: a
 * batched plan built while it is set skips the autotuner and uses squaring
 * variant ((flags >> 8) & 15) and projection variant ((flags >> 12) & 15)
 * (clamped to the variants the plan has), so tests can check every variant. */
enum { CDL_DEBUG_WITHHOLD_TC_LOAD = 1, CDL_DEBUG_BATCH_VARIANT = 2 };
int cdl_ctx_set_debug(cdl_ctx* ctx, int flags);

/* ---------------------------------------------------------------- graph */

/* Gaussian-kernel graph of n node series (Sec. 4.2.1 kernel; Sec. 2: no
 * self edges; Sec. 3.2: D = A 1; Eq. 1: vol = sum_i D_i):
 *   A_ij = exp(-||x_i - x_j||^2 / (2 sigma^2)) for i != j, A_ii = 0,
 *   D_i = sum_j A_ij, vol = sum_i D_i.
 * X:  device, n x T float64 row-major (node i's series in row i).
 * sigma: kernel width; sigma <= 0 selects the lower median of the
 *   n(n-1)/2 distances ||x_i - x_j||, i < j (exact selection). A median of
 *   0 (at least half of the pairs coincide) leaves the kernel undefined:
 *   the selection runs on the device without a host round trip, so this is
 *   not detected and A is not meaningful; pass sigma > 0 for such inputs.
 *   A node with no neighbour of nonzero weight has degree 0; the chain of
 *   that graph is then not finite, and cdl_chain_solve's residual check
 *   (which treats a non-finite residual as divergence) stops it with
 *   CDL_ERR_NOT_CONVERGED.
 * a_dtype: must be CDL_F64 (A is always produced in float64).
 * A:  device, n x n float64 output. D: device, n float64 output.
 * vol, sigma_out: device, one float64 each (sigma_out receives the sigma used).
 * Squared distances are exact when every x is a multiple of 2^-16 below 2^7
 * in magnitude (int64 arithmetic); otherwise they are computed in float64
 * with one rounding per subtraction, product and sum, samples in order.
 * Requires 2 <= n <= 2^20, 1 <= T <= 4096. */
int cdl_build_graph(cdl_ctx* ctx, const double* X, int64_t n, int32_t T, double sigma,
                    cdl_dtype a_dtype, void* A, double* D, double* vol, double* sigma_out);

/* Same computation and results as cdl_build_graph (float64 A), for callers
 * that cannot let a library allocate device memory: for example a process
 * whose device memory is all handed to its own pool allocator, where an
 * extra cudaMalloc would fail or fragment the pool, or a service that must
 * not allocate once it is running. The paper has no counterpart; this entry
 * point exists for such deployments.
 * It needs no context and calls no cudaMalloc, cudaFree or other allocating
 * routine: all scratch lives in one statically allocated device array of
 * about 4 MiB inside the library, held by every GPU that loads it until the
 * process exits. Work is enqueued on `cuda_stream` (NULL = legacy default
 * stream) on the CURRENT device, which must own X and the outputs.
 * Limit: n * T <= 2^20 (e.g. n = 4096 with T = 256); larger inputs return
 * CDL_ERR_INVALID_ARG before launching anything. X and the outputs may be
 * device memory of the current device or managed memory, 8-byte aligned.
 * Other limits and argument meanings as for cdl_build_graph.
 * Each CUDA context has its own copy of the array at its own address: the
 * first call in a context (with that context current) looks the address up
 * and caches it under the context's unique ID, so a context the caller
 * makes current through the driver API, or a primary context re-created
 * after cudaDeviceReset, gets its own lookup. Make the first call in each
 * context before any stream capture.
 * Every call uses the same array: calls that may overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller. */
int cdl_build_graph_static(const double* X, int64_t n, int32_t T, double sigma, double* A,
                           double* D, double* vol, double* sigma_out, void* cuda_stream);

/* Graph of n points under a chosen kernel: kernel = CDL_KERNEL_GAUSSIAN is
 * cdl_build_graph; CDL_KERNEL_EXP is the kernel of the synthetic
 * experiments (Sec. 4.2.1, "Synthetic Data", written there as exp(-d(i,j))
 * with d the Euclidean distance, i.e. sigma = 1):
 *   A_ij = exp(-||x_i - x_j|| / sigma) for i != j, A_ii = 0,
 * computed as exp(-(sqrt(d2) * (1 / sigma))) with the correctly rounded
 * float64 square root. sigma <= 0 selects the lower median distance, as for
 * the Gaussian kernel. Other arguments, limits and errors as for
 * cdl_build_graph; an unknown kernel returns CDL_ERR_INVALID_ARG. */
enum { CDL_KERNEL_GAUSSIAN = 0, CDL_KERNEL_EXP = 1 };
int cdl_build_graph_kernel(cdl_ctx* ctx, const double* X, int64_t n, int32_t T, int32_t kernel,
                           double sigma, cdl_dtype a_dtype, void* A, double* D, double* vol,
                           double* sigma_out);

/* Degrees of a caller's graph (Sec. 3.2: D = A 1; Eq. 1: vol = sum_i D_i),
 * for adjacency matrices not made by cdl_build_graph (the paper's election
 * graphs use their own similarity; the synthetic experiments add random
 * edges). A: device n x n float64, symmetric, non-negative, zero diagonal
 * (not checked). D: device n float64 output; vol: device one float64.
 * Row sums are compensated float64 sums (a few units in the last place of
 * the exact sum). Requires 1 <= n <= 2^20; a_dtype must be CDL_F64
 * (else CDL_ERR_UNSUPPORTED). Asynchronous. */
int cdl_graph_degrees(cdl_ctx* ctx, const void* A, cdl_dtype a_dtype, int64_t n, double* D,
                      double* vol);

/* Symmetric edge weights added to a graph: A_ij += w_e and A_ji += w_e for
 * every listed pair e = (i, j). This forms the second graph of the synthetic
 * experiments, A_2 = Q + (R + R^T) / 2 (Sec. 4.2.1), with w_e = (R_ij +
 * R_ji) / 2 over the pairs where it is nonzero. A: device n x n float64,
 * updated in place (degrees are not updated: call cdl_graph_degrees after).
 * ij: device m x 2 int64, row-major (i, j) pairs, the layout of
 * cdl_cad_edges' edge list; w: device m float64. Pairs must be distinct as
 * unordered pairs for exact, order-free results (each entry then receives
 * one float64 addition); repeated pairs are added in an unspecified order.
 * Entries with an index outside [0, n), i == j, or w negative, infinite or
 * NaN are skipped; their count goes to *n_bad (host, may be NULL) and the
 * call returns CDL_ERR_INVALID_ARG after applying the valid entries.
 * Requires 2 <= n <= 2^20, m >= 0 (ij and w may be NULL when m == 0).
 * Synchronises the context's stream. */
int cdl_graph_add_edges(cdl_ctx* ctx, void* A, cdl_dtype a_dtype, int64_t n, int64_t m,
                        const int64_t* ij, const double* w, int64_t* n_bad);

/* ---------------------------------------------------------------- chain */

/* Inverse chain of Alg. 2 (ChainProduct) for M = L = D - A.
 * Stored levels are the deflated powers
 *   S~_0 = D^{-1/2} A D^{-1/2} - u u^T,  u = D^{1/2} 1 / sqrt(vol),
 *   S~_{i+1} = S~_i S~_i,  i = 0 .. d-2,
 * which equal S^{2^i} - u u^T (u is the eigenvector of S for eigenvalue 1)
 * and act like S^{2^i} on every vector D^{-1/2} b with b orthogonal to the
 * ones vector, the only vectors the solve applies them to.
 * A (device, n x n, a_dtype = CDL_F64; weights finite and non-negative),
 * D (device, n), vol (device, 1).
 * chain_dtype: CDL_F64, CDL_F32 (CUDA-core GEMM), CDL_BF16 (tcgen05
 *   tensor-core GEMM, float32 accumulation, bfloat16 levels) or CDL_FP8E4M3
 *   (tcgen05 kind::f8f6f4 GEMM, float32 accumulation, e4m3 levels with one
 *   scale per level: level i stores value / s_i, s_i = m_i / 448 where m_0 =
 *   max |S~_0| and m_{i+1} = max_r |row r of S~_i|^2 bounds every entry of
 *   S~_i^2 (|(S S)_ab| <= |row a| |row b|; attained on the diagonal); a bf16
 *   copy of each level is kept for the solve's apply), or CDL_FP8E4M3_T128
 *   (e4m3 levels with one scale per 128 x 128 tile, a power of two: the
 *   least 2^e with tile max <= 448 * 2^e; each squaring runs on tcgen05
 *   kind::mxf8f6f4 with block scaling, the tensor core applying the tiles'
 *   e8m0 scales to every 32-element K block, so the whole K range
 *   accumulates in float32 in TMEM; the finished tile's maximum sets its
 *   scale; bf16 copies kept for the apply).
 * flags: CDL_CHAIN_* below.
 * inout: if *inout is NULL a chain is allocated (cdl_chain_free releases it);
 *   if it points to a chain created with the same (n, d, chain_dtype) its
 *   storage is reused; any other chain returns CDL_ERR_INVALID_ARG.
 * Levels occupy d * npad^2 elements, npad = n rounded up to 256; tensor
 * chains (bf16, e4m3) also keep A as two bf16 matrices (A_hi + A_lo,
 * 4 npad^2 bytes), the operand of the solve's tensor-core residual update,
 * and A / 2^q as six exact bf16 slices (12 npad^2 bytes; 2^q, q >= 0, the
 * least power of two not below max A, found by one pass over A), the operand
 * of its full residual.
 * CDL_CHAIN_HOST_LEVELS (bf16 chains): the levels live in pinned host memory
 * (d * npad^2 * 2 bytes, allocated by the library) and two device slots of
 * npad^2 bf16 hold the ones in use: each squaring writes level i + 1 to a
 * slot that is copied to the host on a copy stream while the next squaring
 * runs, and each application of the chain loads level l + 1 over the link
 * while level l is applied. Results are identical to device levels;
 * cdl_chain_level then returns host pointers (and waits for the copies).
 * CDL_CHAIN_TRUNCATE (opt-in; not with CDL_CHAIN_HOST_LEVELS): after each
 * squaring, stop when the new level's max absolute row sum (a bound on its
 * spectral norm, the level being symmetric) is at most 2^-24: neither it nor
 * any later level (their norms square) can change a float32 x + S~ x, so the
 * chain keeps d_eff <= d levels (cdl_chain_depth) and the solve applies only
 * those. For well-connected dense graphs the deflated levels decay like
 * lambda_2^(2^i) and d_eff is a few levels. Changes the configured d, hence
 * opt-in. */
enum { CDL_CHAIN_DEFAULT = 0, CDL_CHAIN_HOST_LEVELS = 1, CDL_CHAIN_TRUNCATE = 2 };
/* With CDL_CHAIN_HOST_LEVELS, bits 8-15 of the flags = r keep levels
 * 0 .. r - 1 in device memory and only the others on the host (a chain
 * larger than the host's memory keeps what fits on the device); 0 = every
 * level on the host. Only cdl_caddelag_pair with CDL_PAIR_REGEN_GRAPHS takes
 * r = 255: as many as fit in the free device memory beside the pair's own
 * buffers. */
enum { CDL_CHAIN_RESIDENT_SHIFT = 8, CDL_CHAIN_RESIDENT_MASK = 0xFF00 };
#define CDL_CHAIN_RESIDENT(r) ((((int32_t)(r)) << CDL_CHAIN_RESIDENT_SHIFT) & CDL_CHAIN_RESIDENT_MASK)
/* Levels in use: d, or fewer after CDL_CHAIN_TRUNCATE. */
int cdl_chain_depth(const cdl_chain* chain, int32_t* d_eff);
int cdl_chain_build(cdl_ctx* ctx, const void* A, cdl_dtype a_dtype, const double* D,
                    const double* vol, int64_t n, int32_t d, cdl_dtype chain_dtype,
                    int32_t flags, cdl_chain** inout);
int cdl_chain_free(cdl_chain* chain);
/* Device pointer to level i (npad x npad, chain dtype, zero padded) and npad;
 * i < d_eff (levels past a truncation are not formed). */
int cdl_chain_level(const cdl_chain* chain, int32_t i, void** level, int64_t* npad);
/* Device pointer to the bf16 view of level i that the solve's tensor-core
 * apply reads (npad x npad): the level itself for CDL_BF16 chains, its bf16
 * copy for CDL_FP8E4M3 and CDL_FP8E4M3_T128 chains; NULL (and
 * CDL_ERR_INVALID_ARG) otherwise. */
int cdl_chain_apply_level(const cdl_chain* chain, int32_t i, void** level);
/* CDL_FP8E4M3_T128 chains: device pointer to the nt x nt float32 tile scales
 * of level i (nt = npad / 128; value of tile (I, J) = scale[I nt + J] times
 * the stored e4m3 values; every scale a power of two). CDL_ERR_INVALID_ARG
 * for other chains. */
int cdl_chain_tile_scales(const cdl_chain* chain, int32_t i, float** scales, int64_t* nt);
/* Scale of level i: stored value times *scale is the level's value (1 for
 * every dtype but CDL_FP8E4M3). Synchronises the chain's device. */
int cdl_chain_level_scale(const cdl_chain* chain, int32_t i, double* scale);

/* ---------------------------------------------------------------- projection */

/* Random projection of Alg. 1 (line "y = W^{1/2} B q") and Alg. 3, formed
 * edge by edge without materialising B or Q (Sec. 4.1: Map + ReduceByKey):
 *   Y[i, r] = k^{-1/2} sum_{j != i} o_ij s_r(min(i,j), max(i,j)) sqrt(A_ij),
 * o_ij = +1 if i < j (edge (i,j) has head i, tail j; Sec. 2), -1 otherwise.
 * s_r(i, j) = +1 if bit (r mod 32) of word ((r mod 128) / 32) of
 * Philox4x32-10(counter = (i, j, r / 128, 0), key = (seed & 0xffffffff,
 * seed >> 32)) is set, else -1.
 * The exact Y has zero column sums (B^T 1 = 0); the computed columns have
 * their means subtracted, which removes the rounding residue of the row sums
 * (a component in the null space of L that no solve could match).
 * A: device n x n (a_dtype = CDL_F64), weights finite, non-negative and
 * below 2^200 (any graph, not only kernel graphs: the terms are split on
 * grids scaled to sqrt(max A), found by one pass over A). Y: device n x k
 * float64 output. Requires 1 <= k <= 1024. */
int cdl_project(cdl_ctx* ctx, const void* A, cdl_dtype a_dtype, int64_t n, int32_t k,
                uint64_t seed, double* Y);

/* ---------------------------------------------------------------- solve */

typedef struct {
  int32_t max_iter;   /* preconditioner applications, >= 1 (paper's q - 1)   */
  double rel_tol;     /* stop when ||Y - L Z||_F <= rel_tol ||Y||_F; 0 = run
                         exactly max_iter applications                       */
  int32_t flags;      /* CDL_SOLVE_* bits                                    */
} cdl_solve_opts;
/* Form the float-float residual after every application (default: after the
 * first one, then update it recursively, R -= L dZ, in float32). */
enum { CDL_SOLVE_FULL_RESIDUAL = 1 };

typedef struct {
  int32_t iters;              /* preconditioner applications performed        */
  double rel_res;             /* final ||Y - L Z||_F / ||Y||_F                 */
  double history[64];         /* rel_res after each application (first iters) */
} cdl_solve_stats;

/* Solve L Z = Y (L = D - A, Y's columns orthogonal to the ones vector) with
 * the chain as preconditioner P (Alg. 2, EstimateSolution, all k right-hand
 * sides at once as in Sec. 4.1):
 *   Z_0 = 0;  Z_{t+1} = Z_t + P (Y - L Z_t),
 *   P R = D^{-1/2} prod_{i<d} (I + S~_i) D^{-1/2} R,
 * then Z is shifted to D-weighted zero column means (sum_i D_i Z[i,:] = 0).
 * For Z_0 = 0 this is the paper's y_{t+1} = y_t - P2 y_t + chi with
 * chi = P1 b and P2 = P1 L. The residual Y - L Z is formed from float64 A,
 * D, Y, Z after the first application: for tensor-core chains A Z runs on
 * the tensor cores from exact bf16 slices (A and Z / c_r, c_r a power of two
 * per column, each as six signed base-256 digits on the grids 2^-8s; every
 * slice product and every 256-term chunk sum is exact in float32; chunk sums
 * are added as integers and scaled into float64), leaving about 2^-50 of
 * |A||Z|; for CUDA-core chains in float-float arithmetic (about 48
 * significant bits). Later steps update it recursively, R -= D dZ - A dZ,
 * with A dZ in float32 (error about 1e-7 of ||L dZ||, i.e. of the previous
 * residual). A bound on the accumulated error of these updates is kept; when
 * the stopping test passes with that bound above rel_tol / 10, the residual
 * is formed in float-float again before stopping. flags =
 * CDL_SOLVE_FULL_RESIDUAL forms it in float-float after every application.
 * Synchronises once per application to read the residual norm.
 * chain: from cdl_chain_build on the same graph. A: device n x n (CDL_F64).
 * Y: device n x k float64. Z: device n x k float64 output; 1 <= k <= 1024.
 * Tensor-core chains apply a level to at most 128 columns at a time, so
 * with k > 128 they solve the columns as independent blocks of at most 128
 * (the iteration acts on each column on its own): each block stops on its
 * own test against its own ||Y_b||; stats then give the residual of all k
 * columns, the largest block iteration count and, per step, the blocks'
 * combined residual (a block that stopped earlier counts with its last).
 * stats: host, may be NULL. Returns CDL_ERR_NOT_CONVERGED (Z still written)
 * when rel_tol > 0 was not reached within max_iter applications, and stops
 * early with it when the residual is not finite or exceeds 1e6 ||Y|| (a
 * preconditioner that does not contract, e.g. an e4m3 chain whose single
 * per-level scale cannot hold the graph's dynamic range). */
int cdl_chain_solve(cdl_ctx* ctx, const cdl_chain* chain, const void* A, cdl_dtype a_dtype,
                    const double* Y, int32_t k, const cdl_solve_opts* opts, double* Z,
                    cdl_solve_stats* stats);

/* ---------------------------------------------------------------- scores */

/* CAD scores between two graphs on the same nodes (Alg. 4; Sec. 2):
 *   c_t(i,j) = vol_t ||Z_t[i,:] - Z_t[j,:]||^2   (Eq. 1 via the embedding),
 *   F_i = sum_{j != i} |A1_ij - A2_ij| * |c_2(i,j) - c_1(i,j)|,
 * and top_idx = the `topk` nodes of highest F, ties to the lower index.
 * The commute-time difference is formed as (a_i - a_j).(b_i - b_j) with
 * a = sqrt(vol2) Z2 - sqrt(vol1) Z1 and b = sqrt(vol2) Z2 + sqrt(vol1) Z1,
 * which avoids cancelling two large commute times.
 * score_dtype: CDL_F64 forms the k-term products and sums in float64;
 *   CDL_F32 forms them on the float32 pipes (much faster on this GPU):
 *   a and b split per column into hi + lo with hi on a fixed grid (23 bits
 *   of the column maximum, so hi_i - hi_j is exact), products made exact by
 *   fused multiply-add and the k-term sum compensated (TwoSum); each
 *   difference c_2 - c_1 is within about 2^-44 sum_r |a_ir - a_jr||b_ir -
 *   b_jr| even where the k terms cancel. Scores accumulate in float64.
 *   CDL_BF16 forms the k-term sums on the bf16 tensor cores, exactly:
 *   c_2 - c_1 = d_i + d_j - M_ij with d_i = a_i.b_i and M_ij = a_i.b_j +
 *   b_i.a_j, M from six exact bf16 slices of [a/g | b g] and [b g | a/g] (g a
 *   power of two per column, c a power of two above every entry; slice
 *   products and 128-term chunk sums exact in float32, combined in int64 in
 *   units of c^2 2^-48), so c_2 - c_1 is within about 2^-47 c^2 of its
 *   value wherever the terms cancel. Edge scores and sums in float64.
 *   (cdl_cad_edges and cdl_cad_score_changed take CDL_F64 or CDL_F32.)
 * A1, A2: device n x n (CDL_F64). Z1, Z2: device n x k float64.
 * vol1, vol2: device, one float64 each. F: device n float64 output.
 * top_idx: device topk int64 output (may be NULL when topk == 0).
 * Requires 0 <= topk <= min(n, 1024). */
int cdl_cad_score(cdl_ctx* ctx, const void* A1, const void* A2, cdl_dtype a_dtype,
                  const double* Z1, const double* Z2, const double* vol1, const double* vol2,
                  int64_t n, int32_t k, cdl_dtype score_dtype, int32_t topk, double* F,
                  int64_t* top_idx);

/* CAD's anomalous edge set (Sec. 3.3): the smallest set S of edges (i < j)
 * whose removal leaves sum_{e not in S} Delta E_e < delta, with
 * Delta E_ij = |A1_ij - A2_ij| |c2(i,j) - c1(i,j)| (the per-edge term of
 * cdl_cad_score). Taking edges in descending Delta E, ties to the lower
 * (i, j), is optimal for this cardinality problem; S = {Delta E > tau} plus
 * the first ties at tau, tau found by bisection on the float64 bit patterns
 * with fixed-order sums (deterministic). The remaining sum is decided in
 * float64 (a different summation order than a sequential sum: decisions
 * within about 1e-15 relative of delta can differ from one).
 * Outputs: edge_ij (device, 2 x max_edges int64, (i, j) pairs in (i, j)
 * order) and edge_dE (device, max_edges) receive the first min(|S|,
 * max_edges) edges of S; for each of the n_nodes nodes in `nodes` (device
 * int64), its top_per_node largest edges (partner j, ties to the lower j;
 * -1 past the end) go to partner / partner_dE (device, n_nodes x
 * top_per_node); F (device n, may be NULL) receives the node scores; *res
 * (host) the counts and sums. Needs n x n float64 workspace (8 n^2 bytes).
 * Requires delta > 0, 0 <= top_per_node <= 1024. Synchronises. */
typedef struct {
  int64_t n_edges;        /* |S| (may exceed max_edges: then only max_edges written) */
  int64_t n_ties_taken;   /* edges of S with Delta E equal to the threshold */
  double threshold;       /* tau as a value (+inf when S is empty)          */
  double remaining;       /* sum of Delta E outside S (< delta)             */
  double total;           /* sum of Delta E over all edges                  */
} cdl_edge_result;
int cdl_cad_edges(cdl_ctx* ctx, const void* A1, const void* A2, cdl_dtype a_dtype, const double* Z1,
                  const double* Z2, const double* vol1, const double* vol2, int64_t n, int32_t k,
                  cdl_dtype score_dtype, double delta, int64_t max_edges, int64_t* edge_ij,
                  double* edge_dE, const int64_t* nodes, int32_t n_nodes, int32_t top_per_node,
                  int64_t* partner, double* partner_dE, double* F, cdl_edge_result* res);

/* Nodes whose series differ between X1 and X2 (any sample unequal; exact
 * comparison): changed[0 .. *n_changed) in ascending order. X1, X2: device
 * n x T float64; changed: device n int32 (capacity); n_changed: host.
 * Synchronises the context's stream. */
int cdl_changed_nodes(cdl_ctx* ctx, const double* X1, const double* X2, int64_t n, int32_t T,
                      int32_t* changed, int32_t* n_changed);

/* CAD scores over the edges of the changed nodes only (Sec. 3.3: commute
 * times are needed only for node pairs whose weight changed). When the two
 * graphs share sigma (cdl_build_graph with the same sigma > 0), A1 and A2
 * differ only in the rows and columns of the nodes whose series changed, so
 * every edge with Delta A != 0 has an endpoint in `changed` and the scores
 * equal cdl_cad_score's (same per-edge arithmetic, sums in another order).
 * Work is n_changed x n edges instead of n^2 / 2. Precondition (not
 * checked): A1_ij == A2_ij whenever neither i nor j is in `changed`.
 * changed: device, n_changed node indices (distinct), 0 <= n_changed <=
 * min(n, 65535). Other arguments as in cdl_cad_score. */
int cdl_cad_score_changed(cdl_ctx* ctx, const void* A1, const void* A2, cdl_dtype a_dtype,
                          const double* Z1, const double* Z2, const double* vol1, const double* vol2,
                          int64_t n, int32_t k, cdl_dtype score_dtype, const int32_t* changed,
                          int32_t n_changed, int32_t topk, double* F, int64_t* top_idx);
/* cdl_pair_opts.score_flags: with a shared sigma (sigma > 0), find the
 * changed nodes (cdl_changed_nodes) and score only their edges
 * (cdl_cad_score_changed); needs sigma > 0, else CDL_ERR_INVALID_ARG. */
enum { CDL_SCORE_CHANGED_ONLY = 1 };

/* ---------------------------------------------------------------- Alg. 4 */

typedef struct {
  int32_t k;               /* projection dimension                          */
  int32_t d;               /* chain length (levels)                         */
  cdl_dtype chain_dtype;   /* CDL_F64, CDL_F32 or CDL_BF16                  */
  cdl_dtype score_dtype;   /* CDL_F64, CDL_F32 or CDL_BF16 (see
                              cdl_cad_score; CDL_BF16 not with
                              CDL_SCORE_CHANGED_ONLY)                       */
  uint64_t seed;           /* projection seed, shared by both graphs        */
  double sigma;            /* <= 0: median rule per graph                   */
  cdl_solve_opts solve;
  int32_t topk;
  int32_t host_io;         /* 1: X1, X2, F, top_idx are host pointers and
                              the call copies them in and out (synchronous);
                              0: device pointers (asynchronous)            */
  int32_t chain_flags;     /* CDL_CHAIN_* flags of cdl_chain_build, and
                              CDL_PAIR_REGEN_GRAPHS / CDL_PAIR_PANEL below  */
  int32_t score_flags;     /* CDL_SCORE_* flags                             */
} cdl_pair_opts;

/* cdl_pair_opts.chain_flags for graphs too large to keep (the paper's
 * larger-than-memory aim, Sec. 1 and Sec. 3.2). With CDL_PAIR_REGEN_GRAPHS
 * neither n x n graph is stored: each is regenerated from its node series
 * in row panels (default 4096 rows; bits 16-23 = log2 of the panel rows,
 * 8 .. 16) wherever it is needed: the exact median sigma (radix select,
 * every pass over the upper-triangle distances of each panel), the degrees,
 * level 0 of the chain and the projection (one pass), the full residual of
 * every refinement step (A Z summed over the panels' exact bf16 slices on
 * the tensor cores) and the scores (both graphs' panels side by side). The
 * panels hold the same A values as cdl_build_graph; degrees and sums differ
 * only in summation order. Needs chain_dtype = score_dtype = CDL_BF16, node
 * series on the 2^-16 grid (else CDL_ERR_UNSUPPORTED) and no
 * CDL_CHAIN_TRUNCATE; the solve forms the full residual after every step.
 * Levels: all in device memory, or with CDL_CHAIN_HOST_LEVELS levels
 * 0 .. r - 1 on the device and the rest in pinned host memory, r from
 * CDL_CHAIN_RESIDENT(r) (255: as many as fit; at least one is needed,
 * level 0 being formed in place). Device memory: the levels on the device,
 * two level slots with host levels, two P x n float64 panels, 12 npad P
 * bytes of slices and the O(n k) vectors. */
enum { CDL_PAIR_REGEN_GRAPHS = 4, CDL_PAIR_PANEL_SHIFT = 16, CDL_PAIR_PANEL_MASK = 0xFF0000 };

/* One graph pair end to end (Alg. 4): graph build, chain, projection and
 * solve for each graph (Alg. 3), then scores and top anomalies.
 * X1, X2: n x T float64 (host or device per host_io). F: n float64,
 * top_idx: topk int64 (host or device per host_io). stats1/stats2: host
 * solve statistics, may be NULL. Device buffers (graphs, chain, embeddings)
 * are owned by the context and reused across calls with the same sizes.
 * Returns CDL_ERR_NOT_CONVERGED (scores still written) when either solve
 * missed its tolerance. */
int cdl_caddelag_pair(cdl_ctx* ctx, const double* X1, const double* X2, int64_t n, int32_t T,
                      const cdl_pair_opts* opts, double* F, int64_t* top_idx,
                      cdl_solve_stats* stats1, cdl_solve_stats* stats2);

/* The embeddings of the last cdl_caddelag_pair call on this context (Alg. 3,
 * what the scores were computed from), for inspection and checking: Z1, Z2
 * receive n x k float64 each (device or host memory, NULL to skip);
 * scalars (4 float64, device or host, NULL to skip) = vol1, vol2, sigma1,
 * sigma2. The values stay valid until the next call that uses the
 * context's workspace. Synchronises. CDL_ERR_INVALID_ARG if no pair has
 * run on the context. */
int cdl_pair_embeddings(cdl_ctx* ctx, double* Z1, double* Z2, double* scalars);

/* ---------------------------------------------------------------- batched form */

typedef struct {
  int32_t k;               /* projection dimension, 1..128                  */
  int32_t d;               /* chain length (levels), 1..64                  */
  cdl_dtype chain_dtype;   /* CDL_BF16 (tensor-core chain)                  */
  cdl_dtype score_dtype;   /* CDL_F64 or CDL_F32 (see cdl_cad_score)        */
  uint64_t seed;           /* projection seed, shared by every graph        */
  double sigma;            /* <= 0: median rule per graph                   */
  cdl_solve_opts solve;    /* per graph (see cdl_caddelag_batched)          */
  int32_t topk;            /* per pair; <= the smallest n                   */
  int32_t host_io;         /* 1: X1, X2, F, top_idx are host pointers       */
  int32_t use_graph;       /* 1: record the whole batch as a CUDA graph on
                              the first call and replay it on later calls
                              with the same sizes and options              */
} cdl_batch_opts;

/* G independent graph pairs of uneven order, end to end (Alg. 4 for each
 * pair), run together: per step, one launch covers every graph of the batch
 * (one grouped tcgen05 launch per chain level, one grouped launch per
 * refinement kernel, one grouped launch per scoring kernel). Each pair's
 * results equal what cdl_caddelag_pair computes for it up to the rounding
 * order of the chain apply (no split-K here).
 * n: host array of G orders, 2 <= n[p] <= 32768, sum <= 2^26.
 * X1, X2: (sum n) x T float64, row-major; pair p's nodes are rows
 *   off_p .. off_p + n[p] - 1 with off_p = n[0] + ... + n[p-1].
 * F: sum n float64 output at the same offsets. top_idx: G x topk int64
 *   output (pair-major; node indices within the pair).
 * stats: host array of 2G entries (graph 2p is pair p's first graph, 2p+1
 *   its second) or NULL.
 * Refinement: each graph follows the rules of cdl_chain_solve, decided on
 * the device; the host issues max_iter + 4 step slots (max_iter with
 * CDL_SOLVE_FULL_RESIDUAL), where a slot is one application of the
 * preconditioner or one certification of a recursively updated residual; a
 * graph that has stopped skips the remaining slots. Full residuals (first
 * step, certifications) are formed on the tensor cores from six exact bf16
 * slices of A and of Z / c, as for a single tensor chain (float64-class).
 * Device buffers of the batch (graphs, chains, A's slices, embeddings; about
 * sum over graphs of (2 d + 16) npad^2 + 8 n^2 bytes, npad = n rounded up to
 * 128) are owned by the context and kept for the next call with the same
 * sizes and options. The call returns after the results are written (it
 * synchronises); it returns CDL_ERR_NOT_CONVERGED (results still written)
 * when any solve missed its tolerance, CDL_ERR_UNSUPPORTED without tcgen05. */
int cdl_caddelag_batched(cdl_ctx* ctx, int32_t G, const int64_t* n, int32_t T, const double* X1,
                         const double* X2, const cdl_batch_opts* opts, double* F, int64_t* top_idx,
                         cdl_solve_stats* stats);

/* What the batched plan of the context holds: the autotuner's choices and
 * timings and the refinement slots recorded in the CUDA graph. The tuner
 * runs once per plan, on the first call, over the batch's own data: each
 * squaring variant (128 x 128 tiles for graphs up to an order, 128 x 256
 * above; max_npad_128 = -1: 256 x 256 blocks on CTA pairs for every graph)
 * squares level 0 of every graph, each projection variant (node rows per
 * block) projects every graph; the fastest of each is kept. */
typedef struct {
  int32_t ready;                        /* 1 once a batched call built a plan  */
  int32_t square_max_npad_128;          /* chosen squaring variant             */
  int32_t project_rows_per_block;       /* chosen projection variant           */
  int32_t residual_tile_m, residual_tile_n;
  int32_t slots_captured;               /* refinement slots in the CUDA graph  */
  int32_t slots_seen;                   /* most slots a call has needed        */
  int32_t n_square_variants, n_project_variants;
  int32_t square_variant_max_npad_128[8];
  double square_variant_ms[8];
  int32_t project_variant_rows[8];
  double project_variant_ms[8];
  uint64_t device_bytes;                /* device memory owned by the plan     */
} cdl_batch_info;
int cdl_batch_plan_info(const cdl_ctx* ctx, cdl_batch_info* info);

#ifdef __cplusplus
}
#endif
#endif /* CDL_H */
