/*
 * hps.h -- C ABI of libhps.so, a GB300 (sm_103a) implementation of the
 * multigrid-preconditioned Hierarchical Poincare-Steklov (HPS) skeleton solver
 * for the variable-coefficient Helmholtz problem
 *
 *     -Lap u - kappa^2 (1 - b(x)) u = s  in (0,1)^2,   du/dn + i eta u = t  on the boundary
 *
 * ("Towards a Multigrid Preconditioner Interpretation of Hierarchical
 * Poincare-Steklov Solvers", arXiv 2511.00735, section 2, eq. diffhelm).
 *
 * Conventions shared by every call
 * --------------------------------
 *  Complex numbers are interleaved (re, im) doubles (C99 double complex /
 *  numpy complex128).  Lower-precision internals (the mixed path) are hidden.
 *
 *  Elements: e = ix + nx*iy (x fastest).  Element nodes: tensor GLL grid of
 *  order N, node(i,j) = i*(N+1) + j (x index slow), physical coordinates
 *  x = ix*h + (xi_i + 1) h/2, h = 1/nx.  q = N-1 edge (non-corner) nodes per
 *  side; sides ordered l, r, b, t; along a side by increasing coordinate.
 *
 *  Skeleton ("face") order, length n_skel = 2 * nfaces * q: vertical faces
 *  v(ix,iy) (between (ix,iy) and (ix+1,iy)) numbered ix + (nx-1)*iy, then
 *  horizontal faces h(ix,iy) (between (ix,iy) and (ix,iy+1)) numbered
 *  (nx-1)*ny + ix + nx*iy.  Face f holds [incoming impedance of the
 *  left/bottom element on its side r/t ; incoming impedance of the right/top
 *  element on its side l/b], q values each: index (2f + slot) q + k.
 *  Row k of M is the outgoing relation (section 3.2, eq. localiti) of the
 *  element across the face from unknown k, so M = I + Pi T and
 *      M g = RHS,  RHS_k = -( H^(e)_a + sum_{b on the boundary} T^(e)_{ab} t_b ).
 *
 *  Boundary-data order, length n_bdry = 4 nx q: domain sides left (ix = 0,
 *  iy = 0..ny-1), right, bottom (iy = 0, ix = 0..nx-1), top; each element side
 *  with its q edge nodes by increasing coordinate.
 *
 *  Batches of right-hand sides are RHS-major: [nrhs][n] complex128.
 *
 *  Pointers: "device" arguments must be device (or managed) memory of the
 *  context's device; "host or device" arguments are classified with
 *  cudaPointerGetAttributes.  The caller owns every buffer it passes; the
 *  library owns the leaf maps, the merge tree and its workspaces until
 *  hps_destroy, a new hps_mesh or hps_set_coeff.
 *
 *  Streams: every call enqueues on the context's stream (hps_create); calls
 *  return after enqueueing except where stated (hps_gmres_solve reads scalars
 *  back every outer iteration and returns when the solve is done).  One
 *  context per stream; a context is not thread-safe.
 *
 *  Errors: every call returns HPS_OK (0) or a negative status below; nothing
 *  aborts, traps or throws across the ABI.  hps_last_error(ctx) gives a
 *  message for the last failure on that context.  There is no CPU fallback:
 *  without a usable CUDA device hps_create returns HPS_ENODEV.
 */
#ifndef HPS_H
#define HPS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hps_ctx hps_ctx;

enum {
  HPS_OK = 0,
  HPS_EINVAL = -1,      /* bad argument (size, pointer, order, state)            */
  HPS_ENOMEM = -2,      /* device allocation failed                              */
  HPS_ENOTBUILT = -3,   /* a prerequisite call (mesh, coeff, leaves, merges) missing */
  HPS_ENOTCONV = -4,    /* FGMRES stopped before the tolerance (info still filled) */
  HPS_ETIMEOUT = -5,    /* a bounded device wait gave up                         */
  HPS_ECUDA = -6,       /* a CUDA runtime call failed                            */
  HPS_ENODEV = -7,      /* no usable CUDA device                                 */
  HPS_EUNSUPPORTED = -8,/* valid input this build does not handle (stated in the message) */
  HPS_ENUMERIC = -9     /* a factorisation broke down (non-positive pivot, zero pivot) */
};

enum { HPS_FP64 = 0, HPS_MIXED = 1 };

/* Arithmetic of the outer FGMRES (hps_set_outer_arith). */
enum { HPS_OUTER_DEFAULT = -1, HPS_OUTER_FP64 = 0, HPS_OUTER_DF64 = 1 };

/* Method of the double-float Arnoldi matvec (hps_set_arnoldi_matvec). */
enum { HPS_MV_DEFAULT = -1, HPS_MV_SIMT = 0, HPS_MV_TENSOR = 1 };

/* Arithmetic of the sweep products of an HPS_MIXED tree (hps_set_sweep_arith). */
enum { HPS_SWEEP_DEFAULT = -1, HPS_SWEEP_FP32 = 0, HPS_SWEEP_BF16X3 = 1 };

/* Per-solve report of hps_gmres_solve. */
typedef struct {
  int outer_iterations;     /* FGMRES iterations (max over right-hand sides)         */
  int converged;            /* number of right-hand sides with true residual <= tol  */
  double max_rel_residual;  /* max over RHS of ||RHS - M g||_2 / ||RHS||_2 of the returned g,
                               formed with the FP64 matvec on both paths */
  int* iterations;          /* optional caller array [nrhs]: iterations per RHS (may be NULL) */
  double* rel_residual;     /* optional caller array [nrhs]: explicit residual per RHS (may be NULL) */
  double ms_rhs;            /* device time of the RHS assembly                        */
  double ms_solve;          /* wall time of the FGMRES loop                           */
} hps_info;

/* Device-memory allocator used for every library-owned buffer.  alloc returns
 * a device pointer of at least `bytes` bytes aligned to 256 bytes, or NULL;
 * free releases it.  Default: cudaMalloc / cudaFree. */
typedef void* (*hps_alloc_fn)(size_t bytes, void* user);
typedef void (*hps_free_fn)(void* ptr, void* user);

/* Create a context on `device`, enqueuing on `stream` (a cudaStream_t, NULL =
 * the legacy default stream).  *ctx receives the handle.  HPS_ENODEV when the
 * device cannot be used. */
int hps_create(hps_ctx** ctx, int device, void* stream);

/* Release every library-owned buffer and the context (safe on NULL). */
int hps_destroy(hps_ctx* ctx);

/* Replace the allocator (before hps_mesh; EINVAL afterwards). */
int hps_set_allocator(hps_ctx* ctx, hps_alloc_fn alloc, hps_free_fn free_fn, void* user);

/* Message of the last failure on ctx (static storage of the context). */
const char* hps_last_error(hps_ctx* ctx);
const char* hps_strerror(int status);

/* Structured mesh of nx x ny square elements with tensor GLL grids of order N
 * (section 3).  Requires nx == ny == 2^k (k >= 1) so that the nested-dissection
 * levels alternate x, y, x, y (section 4.2, Fig. 1), and 2 <= N <= 24.
 * Builds every index map on the host and uploads it.  Invalidates coefficient,
 * leaves and tree. */
int hps_mesh(hps_ctx* ctx, int nx, int ny, int N);

/* Sizes after hps_mesh: skeleton unknowns, boundary-data length, number of
 * merge levels L = log2(nx*ny), and the device bytes currently held. */
int hps_sizes(hps_ctx* ctx, long long* n_skel, long long* n_bdry, int* levels,
              long long* bytes_held);

/* Host arrays [E][(N+1)^2]: physical coordinates of every element node
 * (the points where the caller samples b). */
int hps_node_coords(hps_ctx* ctx, double* x, double* y);

/* Host arrays [n_bdry]: coordinates and outward normal of every physical
 * boundary node, in boundary-data order (where the caller evaluates t). */
int hps_boundary_points(hps_ctx* ctx, double* x, double* y, double* nx, double* ny);

/* Host int32 arrays [E*4*q] indexed by element-side position
 * p = (e*4 + side)*q + k: skel_in[p] = skeleton unknown incoming to e there,
 * skel_out[p] = skeleton unknown incoming to the neighbour across it,
 * bdry[p] = boundary-data index; -1 where not applicable.  Any may be NULL. */
int hps_index_maps(hps_ctx* ctx, int* skel_in, int* skel_out, int* bdry);

/* Coefficient c = kappa^2 (1 - b) (section 2).  b: [E][(N+1)^2] doubles at
 * the points of hps_node_coords, host or device.  eta is the impedance
 * parameter (the paper takes eta = kappa).  Invalidates leaves and tree. */
int hps_set_coeff(hps_ctx* ctx, double kappa, double eta, const double* b);

/* Build every leaf impedance-to-impedance map T = I_o L^{-1} I(:, iota_Gamma)
 * (section 3.1, eq. ItIOperator), one batched launch over the elements, FP64
 * result kept on the device in side order l, r, b, t.  `precision` selects the
 * precision of the merge tree built later (HPS_FP64 or HPS_MIXED); the leaf
 * maps themselves are FP64 in both (the outer matvec needs them).
 * Elements whose interior operator is provably positive definite
 * (kappa^2 (1-b) (h/2)^2 below the smallest interior Dirichlet eigenvalue of
 * the reference element, with a 2% margin) eliminate the interior by a real
 * L D L^T factorisation (N <= 16; for 17 <= N <= 24, whose factor does not fit
 * on chip, by conjugate gradients preconditioned by fast diagonalisation, as
 * hps_volume_solution); the others (near or past an interior resonance) use
 * a pivoted complex elimination of the edge rows first.  HPS_ENUMERIC if an
 * element system is singular. */
int hps_build_leaves(hps_ctx* ctx, int precision);

/* hps_build_leaves for n contexts at once (section 3.1): the elements of all
 * contexts on the Cholesky route are built by one kernel launch per GLL order
 * (one CTA per SM striding over a per-element list of coefficient pointer,
 * output pointer, h and eta), the others by the pivoted route.  Every context
 * needs hps_set_coeff; all must live on one device.  Work is enqueued on the
 * stream of ctxs[0] and the call returns after it completes, so every
 * context's maps are ready on return.  Errors are reported on ctxs[0]. */
int hps_build_leaves_batch(hps_ctx** ctxs, int n, int precision);

/* Free the per-solve workspaces (FGMRES basis, sweep and coarse vectors,
 * staging) and keep the leaf maps and the merge tree; the next solve
 * allocates them again.  Synchronises the context's stream. */
int hps_release_workspace(hps_ctx* ctx);

/* Host copy of leaf maps e0 .. e0+count-1: [count][4q][4q] complex128, row-major. */
int hps_leaf_T(hps_ctx* ctx, int e0, int count, void* T_host);

/* Nested-dissection merges l = 1..L_exact (section 4.1 eq. globalfacesystem,
 * section 4.2): per level, batched pair merges T_pair = D - C A^{-1} B with
 * the interface blocks A kept (inverted) for the preconditioner.  0 <= L_exact
 * <= L.  exact_coarse != 0 also inverts the coarse system M_{L_exact+1}
 * densely (direct HPS when combined with L_exact = L-1; section 4.2). */
int hps_merge_levels(hps_ctx* ctx, int L_exact, int exact_coarse);

/* Host copy of the ItI map of subdomain `sub` after `stage` merges (stage 0 =
 * leaves), in the subdomain's natural boundary order l, r, b, t:
 * [n][n] complex128, n = 2 (a+b) q for an a x b element block. */
int hps_stage_T(hps_ctx* ctx, int stage, int sub, void* T_host);

/* RHS of M g = RHS from boundary data (section 3.2; sources s = 0):
 * t [nrhs][n_bdry] -> rhs [nrhs][n_skel], both device, complex128. */
int hps_rhs(hps_ctx* ctx, const void* t, void* rhs, int nrhs);

/* y = M x for x, y [nrhs][n_skel] device complex128 (FP64, leaf maps). */
int hps_skel_matvec(hps_ctx* ctx, const void* x, void* y, int nrhs);

/* z = MG(M) r (section 4.3): the V-cycle over the merged levels 1..L_exact
 * (smoother A^{-1}, restriction, prolongation), the coarse system solved by
 * inner_iters unpreconditioned GMRES steps from zero (or exactly when the tree
 * was built with exact_coarse).  r, z [nrhs][n_skel] device complex128. */
int hps_precond_apply(hps_ctx* ctx, const void* r, void* z, int nrhs, int inner_iters);

/* Solve M g = RHS(t) for nrhs right-hand sides by flexible GMRES (restart
 * `restart`, zero initial guess, at most max_outer restart cycles) with MG(M)
 * as the preconditioner (inner_iters coarse GMRES steps), until
 * ||RHS - M g||_2 <= tol ||RHS||_2 per right-hand side (section 4.3, 5).
 * inner_iters < 0 runs unpreconditioned FGMRES.  t [nrhs][n_bdry] and
 * g_out [nrhs][n_skel] are complex128, host or device.  s (may be NULL: no
 * source) holds the source of each right-hand side at every element node,
 * [nrhs][E][(N+1)^2] complex128 in the node order of hps_node_coords, host or
 * device; its interior values enter as b~ = w_i w_j s (physical GLL weights)
 * and the RHS gets the interior contributions H = I_o L^{-1} I(:, iota_i) b~ of
 * eq. ItIOperator (section 3.1; the RHS of the header's conventions).  info
 * may be NULL.  HPS_ENOTCONV when a right-hand side did not reach tol (g_out
 * and info are filled). */
int hps_gmres_solve(hps_ctx* ctx, const void* t, const void* s, int nrhs, double tol,
                    int inner_iters, int restart, int max_outer, void* g_out,
                    hps_info* info);

/* Element fields u at every node of every element (section 3.1: L u = b with
 * b(iota_Gamma) = I_i u, b(iota_i) = b~) from the skeleton solution g
 * [nrhs][n_skel] of hps_gmres_solve, the boundary data t [nrhs][n_bdry] (NULL:
 * zero) and the sources s [nrhs][E][(N+1)^2] (NULL: none), all complex128, host
 * or device.  u [nrhs][E][(N+1)^2] complex128, host or device, node order of
 * hps_node_coords.  The corner nodes, which the discretization leaves out, are
 * filled afterwards: each is the mean of the two one-sided extrapolations along
 * the element edges meeting there (the degree N-2 polynomial through an edge's
 * N-1 other nodes, evaluated at the corner).  Interior solves: positive-definite
 * elements by conjugate gradients preconditioned by fast diagonalisation of the
 * constant-coefficient operator (FP32) inside FP64 refinement; the others by the
 * pivoted route of hps_build_leaves.  Returns when u is written. */
int hps_volume_solution(hps_ctx* ctx, const void* t, const void* s, const void* g, int nrhs, void* u);

/* Coarse calls per level of the preconditioner of later hps_precond_apply and
 * hps_gmres_solve calls on ctx (section 4.3: "a single coarse call yields a
 * V-cycle; multiple ones define a gamma-cycle").  At every merge level the
 * correction of the next level's system S r_c is made by `gamma` calls of MG,
 * each on the current residual, e_k = e_{k-1} + MG(S)(r_c - S e_{k-1}); at the
 * coarsest level MG(S) is the coarse solver (inner_iters GMRES steps or the
 * exact inverse).  gamma = 1 (the initial state) is the V-cycle; the coarse
 * solver then runs gamma^L_exact times per application.  1 <= gamma <= 8,
 * HPS_EINVAL otherwise.  Buffers for gamma > 1 are allocated by the next
 * application (one extra pair of stage vectors per merged level). */
int hps_set_gamma(hps_ctx* ctx, int gamma);

/* Arithmetic of the outer FGMRES of later hps_gmres_solve calls on ctx:
 *   HPS_OUTER_FP64     matvec, Gram-Schmidt and basis in FP64 (section 4.3);
 *   HPS_OUTER_DF64     (with HPS_MIXED leaves only) the Arnoldi steps (matvec,
 *                      Gram-Schmidt, basis) on pairs of FP32 numbers (about 48
 *                      significand bits, error-free TwoSum/TwoProduct
 *                      accumulation), the preconditioned directions kept in
 *                      FP32 (they are the FP32 tree's output).  Every restart
 *                      residual and the residual of the returned solution are
 *                      formed in FP64 (the iterate rounded to FP64, the FP64
 *                      leaf maps, FP64 norms), so every convergence decision
 *                      and the reported residual are FP64;
 *   HPS_OUTER_DEFAULT  DF64 for HPS_MIXED, FP64 for HPS_FP64 (the initial state).
 * HPS_EINVAL for other values.  DF64 needs HPS_MIXED leaves: with HPS_FP64
 * leaves hps_gmres_solve returns HPS_EINVAL (there is no silent fallback). */
int hps_set_outer_arith(hps_ctx* ctx, int mode);

/* Method of the Arnoldi matvec w = Pi M z of later HPS_OUTER_DF64 solves on ctx
 * (section 4.3: the skeleton operator applied once per FGMRES iteration), with
 * the FP64 leaf maps, the preconditioned direction z in FP32 and w in
 * double-float:
 *   HPS_MV_SIMT     error-free FP32 products and TwoSum accumulation on the
 *                   FP32 pipes (about 48 significant bits);
 *   HPS_MV_TENSOR   exact splitting on the tensor cores (Ozaki, Ogita, Oishi,
 *                   Rump 2012): the rows of T and the columns of the expanded z
 *                   cut into seven 7-bit slices aligned to their largest entry,
 *                   the 28 slice products with s + t <= 8 formed exactly in
 *                   bf16 MMAs with FP32 accumulation, summed in double-float;
 *                   error below about 2^-45 |T_i.|max |z_.r|max (4q) per entry.
 *                   Used when 4q <= 92 and nrhs <= 32, else HPS_MV_SIMT;
 *   HPS_MV_DEFAULT  HPS_MV_TENSOR (the initial state).
 * HPS_EINVAL for other values. */
int hps_set_arnoldi_matvec(hps_ctx* ctx, int method);

/* The Arnoldi matvec as the current method forms it, for checking it: y = Pi M x
 * with x rounded to FP32 first (the Arnoldi multiplies FP32 directions) and the
 * double-float result returned in FP64.  x, y: [nrhs][n_skel] complex128 in the
 * hps_skel_matvec layout, device pointers; 1 <= nrhs <= 64.  HPS_ENOTBUILT
 * before hps_build_leaves; HPS_ETIMEOUT if a tensor-core wait gave up. */
int hps_skel_matvec_mixed(hps_ctx* ctx, const void* x, void* y, int nrhs);

/* Arithmetic of the preconditioner's sweep products (section 4.3: the up-sweep
 * rho' = rho - U f and the down-sweep x = Dm [.;.] of every merge level, which
 * the V-cycle applies once per FGMRES iteration) for trees built by later
 * hps_merge_levels calls with HPS_MIXED leaves; the FP64 tree ignores it:
 *   HPS_SWEEP_FP32     FP32 products (3xTF32 on the tensor cores where the
 *                      operator has at least 32 interface rows per child);
 *   HPS_SWEEP_BF16X3   the operators U, Dm of those levels are stored as bf16
 *                      pairs x = hi + lo (hi = bf16(x), lo = bf16(x - hi),
 *                      2^-16 relative) and multiplied as hi*hi + hi*lo + lo*hi
 *                      with FP32 accumulation: about 3 * 2^-16 relative error
 *                      per product, the same 8 bytes per complex entry as FP32,
 *                      no splitting of the operator at application time.  The
 *                      preconditioner is applied inside flexible GMRES whose
 *                      residuals are formed in FP64, so the solution's accuracy
 *                      is unchanged; only the iteration count can differ;
 *   HPS_SWEEP_DEFAULT  HPS_SWEEP_BF16X3 (the initial state).
 * HPS_EINVAL for other values.  The tree in use keeps the arithmetic it was
 * built with. */
int hps_set_sweep_arith(hps_ctx* ctx, int mode);

/* Profiling phases of hps_profile_read. */
enum {
  HPS_PH_LEAF = 0,   /* hps_build_leaves: the leaf kernel alone                     */
  HPS_PH_MERGE,      /* hps_merge_levels                                            */
  HPS_PH_RHS,        /* RHS assembly inside hps_gmres_solve                         */
  HPS_PH_MATVEC,     /* skeleton matvec inside hps_gmres_solve (one kernel each)     */
  HPS_PH_PRECOND,    /* MG(M) applications inside hps_gmres_solve                   */
  HPS_PH_ORTHO,      /* Gram-Schmidt inside hps_gmres_solve                         */
  HPS_PH_OTHER,      /* final residual and output                                   */
  HPS_NPHASE
};

/* Number of CUDA kernels this library has launched in this process (all
 * contexts); a cheap host-side counter, no device synchronisation. */
long long hps_kernel_launches(void);

/* enable != 0: clear the per-phase counters and start bracketing the phases
 * above with CUDA events on the context's stream; enable == 0: stop.
 * Profiling adds two event records per phase instance and no synchronisation. */
int hps_profile(hps_ctx* ctx, int enable);

/* Device milliseconds, kernel launches and phase instances accumulated since
 * the last hps_profile(ctx, 1), per phase; host arrays [HPS_NPHASE], any may be
 * NULL.  Synchronises the context's stream. */
int hps_profile_read(hps_ctx* ctx, double* ms, long long* launches, long long* calls);

/* Kernel classes of hps_profile_kernels_read. */
enum {
  HPS_KC_SWEEP = 0,    /* the V-cycle's sweep products on the tensor cores (the tiled
                          operators of every merge level, up- and down-sweep); work =
                          algorithmic bytes: the operator (8 B per complex entry), the
                          block vector B, C0 when present and C, each once            */
  HPS_KC_MERGE_GEMM,   /* the batched complex GEMMs of hps_merge_levels (section 4.1 /
                          Algorithm 1: S, X1, X2, T_pair, U, Dm); work = algorithmic
                          flops 8 m n k per product                                     */
  HPS_NKC
};

/* enable != 0: clear the per-class counters and bracket every launch of the
 * classes above with CUDA events on the context's stream (launches being
 * captured into the V-cycle's CUDA graph inside hps_gmres_solve are not
 * bracketed: time the class through hps_precond_apply, which launches
 * directly); enable == 0: stop.  Two event records per launch, no
 * synchronisation. */
int hps_profile_kernels(hps_ctx* ctx, int enable);

/* Per class (host arrays [HPS_NKC], any may be NULL): device milliseconds,
 * bracketed launches, algorithmic bytes and algorithmic flops accumulated
 * since the last hps_profile_kernels(ctx, 1).  Synchronises the context's
 * stream. */
int hps_profile_kernels_read(hps_ctx* ctx, double* ms, long long* launches, double* bytes, double* flops);

/* Tile autotuner of the tensor-core GEMMs (the merge products, the sweep
 * products and the coarse products): per GEMM shape (kernel family, rows,
 * columns, k, batch entries, SM count) it times a short list of candidate
 * launch configurations -- column-tile width, CTAs per SM of the persistent
 * kernels, and how far k is split to fill the GPU -- with CUDA events on the
 * context's stream and keeps the fastest in a process-wide table that every
 * context shares.
 *   HPS_TUNE_OFF       (default) the fixed heuristics (candidate 0 of each list)
 *   HPS_TUNE_ON        table lookups; a shape not in the table is tuned on its
 *                      first launch outside graph capture whose output does not
 *                      alias its inputs (each candidate runs once untimed and
 *                      twice timed, then the winner once more, so the call's
 *                      result is the winner's); a product that cannot be
 *                      re-run, or that is being captured, takes candidate 0
 *   HPS_TUNE_FORCE + i candidate i (modulo the list's length) for every shape,
 *                      without timing (tests of every candidate's numerics)
 * Switching the mode re-captures the V-cycle graph on its next use; with
 * HPS_TUNE_ON the first V-cycle after that runs without the graph, so that
 * its sweep shapes are tuned before they are captured.  Candidates differ
 * only in tiling and in the order of the k summation (split k), so results
 * agree to FP32 rounding.  Tuning synchronises the stream once per new shape. */
enum { HPS_TUNE_OFF = 0, HPS_TUNE_ON = 1, HPS_TUNE_FORCE = 16 };
int hps_set_autotune(hps_ctx* ctx, int mode);

/* The process-wide tuning table as text, one line per shape ("family m n k
 * batch sms -> candidate: nc, CTAs per SM, split; ms of candidate 0 and of
 * the winner"), NUL-terminated and cut to len bytes; returns the number of
 * shapes in the table (buf may be NULL to count). */
int hps_autotune_table(char* buf, int len);

/* Empty the process-wide tuning table. */
void hps_autotune_clear(void);

/* Leaf ItI maps without any device allocation (no counterpart in the paper:
 * a deployment variant of hps_build_leaves).  For callers that cannot
 * allocate device memory while they run, e.g. a process whose device memory
 * all belongs to its own pool, or a loop that must not call cudaMalloc /
 * cudaFree because those calls can synchronise the device.
 *
 *   device, stream  where to run (stream: a cudaStream_t, NULL = legacy default)
 *   N               GLL order, 2 <= N <= 16 (larger orders exceed the static
 *                   workspace: HPS_EINVAL)
 *   h, eta          element width and impedance parameter
 *   c               device [E][(N+1)^2]: c = kappa^2 (1 - b) at the element
 *                   nodes (node order of hps_node_coords)
 *   T               device output [E][4(N-1)][4(N-1)] complex128, side order
 *                   l, r, b, t (the same maps hps_build_leaves keeps)
 *
 * All workspace lives in one file-scope device array of about 4.6 MB that
 * every GPU which loads the library holds until the process exits.  Its
 * device address is looked up on the first call on each device, with that
 * device current; make that first call before any stream capture.  Every call
 * shares the array: calls whose work overlaps on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  The call synchronises
 * `stream` once to read the breakdown flag: HPS_ENUMERIC when an interior
 * operator is not positive definite (this entry has no pivoted fallback), and
 * T is then undefined for every element.  The caller's current device is the
 * same on return as on entry. */
int hps_leaf_maps_noalloc(int device, void* stream, int N, double h, double eta, const double* c, int E,
                          void* T);

#ifdef __cplusplus
}
#endif

#endif /* HPS_H */
