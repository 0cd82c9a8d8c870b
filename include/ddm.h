/*
 * ddm.h -- C ABI of the GB300 (sm_103a) additive overlapping domain
 * decomposition solver for the Helmholtz equation with PML
 * (Leng & Ju, "An Additive Overlapping Domain Decomposition Method for the
 * Helmholtz Equation", 2018).
 *
 * Problem (Sections 1, 2.1, 3.1):  Delta u + k^2 u = f, k(x) = omega / c(x),
 * truncated by a uniaxial PML (alpha = 1 + i sigma) and discretised by the
 * 5-point (2D) / 7-point (3D) finite-difference operator in its J-scaled,
 * complex-symmetric form
 *     (A u)(x) = sum_a prod_{b!=a} alpha_b [ (u(x+e_a)-u(x))/alpha_a(x_a+1/2)
 *                                           - (u(x)-u(x-e_a))/alpha_a(x_a-1/2) ]
 *                + h^2 k^2 prod_a alpha_a u(x),          A u = b = h^2 J f,
 * with homogeneous Dirichlet values beyond the extended grid.
 *
 * Method (Algorithm 3.1): the interior is cut into N1 x N2 (x N3) boxes; each
 * box plus an overlap of `overlap` cells and a PML of `pml` cells is a
 * subdomain.  Step 1 solves every subdomain problem with its restricted
 * source; step s >= 2 solves them with the directional residuals Psi of the
 * neighbours (8 directions in 2D, 26 in 3D; faces lagged one step, corners
 * two, 3D vertices three).  The DDM solution is sum beta_0 * sum_s u^s.
 * The same steps form the preconditioner M_K of flexible GMRES (Section 4.2).
 *
 * Grid and memory layout
 *   - Physical axis 0 is x (fastest varying), 1 is y, 2 is z.  Interior node p
 *     sits at (p + 1/2) h; the global extended grid adds e = overlap + pml
 *     nodes per side, so it has (n[a] + 2e) nodes along axis a.
 *   - "Global vectors" are complex128 (interleaved re, im doubles) arrays over
 *     the global extended grid, x fastest, then y, then z, one after another
 *     for several right-hand sides (stride = number of global nodes).
 *   - The wave speed `c` is a float64 array over the global extended grid.
 *   - "Local vectors" (debug/parity entry points only) concatenate every
 *     subdomain's extended grid (x fastest), subdomains in C order of their
 *     index (z slowest, x fastest); ddm_local_layout() gives the offsets.
 *     With nrhs right-hand sides they are subdomain-major: subdomain s's
 *     nrhs vectors are adjacent, right-hand side r at element
 *     offsets[s] * nrhs + r * (ext_x[s] * ext_y[s] * ext_z[s]).
 *
 * Conventions for every entry point
 *   - Returns a ddm_status; never aborts or exits.  On error the context keeps
 *     a message, readable with ddm_last_error().
 *   - Pointers named *_dev are CUDA device pointers owned by the caller and
 *     valid only during the call; *_host are host pointers.  The library never
 *     frees caller memory.  Work is enqueued on the stream given at set-up;
 *     entry points that return results to the host synchronise that stream.
 *   - A context is not thread-safe: serialise calls on one context.
 */
#ifndef DDM_H
#define DDM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DDM_OK = 0,
  DDM_E_INVAL = 1,     /* bad argument or parameter combination            */
  DDM_E_NOMEM = 2,     /* device allocation failed                          */
  DDM_E_CUDA = 3,      /* a CUDA call or kernel launch failed               */
  DDM_E_STATE = 4,     /* call out of order (e.g. solve before factor)      */
  DDM_E_SINGULAR = 5,  /* a pivot of a subdomain factor was (near) zero     */
  DDM_E_NOCONV = 6,    /* tolerance not reached within the iteration limit  */
  DDM_E_TIMEOUT = 7,   /* a bounded device-side wait gave up                */
  DDM_E_BUDGET = 8     /* request exceeds the configured memory budget      */
} ddm_status;

enum { DDM_FP64 = 0, DDM_MIXED = 1 };         /* precision of the local solves  */
enum { DDM_STEPPING = 0, DDM_FGMRES = 1 };    /* solver mode of ddm_solve       */

typedef struct ddm_ctx ddm_ctx;

typedef struct {
  int dim;                  /* 2 or 3                                                   */
  int64_t n[3];             /* interior nodes per physical axis (x, y, z)               */
  double h;                 /* uniform spacing                                          */
  int parts[3];             /* N1, N2 (, N3): subdomains per axis (Section 2.2)         */
  const int64_t *cuts[3];   /* host arrays of parts[a]+1 increasing node offsets from 0
                               to n[a] (uneven partitions); NULL = uniform cuts         */
  int overlap;              /* ov >= 1 cells: overlap width d~ = ov h (Eq. (11))      */
  int pml;                  /* PML cells beyond the overlap                             */
  double sigma0;            /* PML profile sigma(t) = sigma0 ((t - ov)/pml)^pml_power   */
  double pml_power;         /*   for t > ov cells beyond a box face, 0 otherwise        */
  int precision;            /* DDM_FP64, or DDM_MIXED: complex64 factors, local solves
                               and transfers inside complex128 Krylov / residuals       */
  int max_rhs;              /* largest nrhs passed to ddm_apply / ddm_solve             */
} ddm_params;

typedef struct {
  int iters;                /* FGMRES iterations (or DDM steps in stepping mode)        */
  int ddm_steps;            /* DDM steps taken = local solves per subdomain             */
  int converged;            /* 1 if rel_residual <= tol                                  */
  int n_unique_factors;     /* distinct subdomain factors actually computed             */
  double rel_residual;      /* explicit ||b - A u||_2 / ||b||_2 in FP64 at exit         */
  double rel_residual_est;  /* last Krylov / strip-residual estimate                    */
  double factor_ms;         /* device time of the last ddm_factor                       */
  double solve_ms;          /* wall time of this ddm_solve call                         */
} ddm_info;

/* Set-up (Sections 2.1, 3.1; assembly step of the path).  Validates `p`,
 * copies the wave speed c_dev (float64, global extended grid, device) and
 * builds on the device the PML stretching tables (alpha = 1 + i sigma at nodes
 * and half nodes, Eq. (11)), k^2 = (omega / c)^2 and the partition
 * descriptors.  Allocates all device workspace for up to p->max_rhs
 * right-hand sides.  `stream` is a cudaStream_t (NULL = legacy default).
 * Does not factor.  Errors: DDM_E_INVAL, DDM_E_NOMEM, DDM_E_CUDA.           */
ddm_status ddm_setup(const ddm_params *p, double omega, const double *c_dev, void *stream, ddm_ctx **out);

/* Replace the medium: recompute k^2 = (omega / c)^2 from c_dev (float64, global
 * extended grid, device) on the context's stream (the assembly step of the
 * path) and mark the context unfactored; call ddm_factor before solving.
 * Errors: DDM_E_INVAL, DDM_E_CUDA.                                          */
ddm_status ddm_set_medium(ddm_ctx *ctx, double omega, const double *c_dev);

/* ddm_set_medium with the wave speed in host memory (float64, global
 * extended grid): copied to a library-owned device buffer on the context's
 * stream, then as ddm_set_medium.                                            */
ddm_status ddm_set_medium_host(ddm_ctx *ctx, double omega, const double *c_host);

/* Factor every distinct subdomain operator (Algorithm 3.1's local problems;
 * the paper uses a sparse direct solver).  Subdomains whose extended grids
 * carry identical operators share one factor.  Each factor is the block
 * tridiagonal LU in explicit-inverse form: G_k = D_k^{-1} with
 * D_k = T_k - L_k G_{k-1} U_{k-1} over the x-lines (2D) or z-planes (3D) of
 * the subdomain, each D_k inverted by Gauss-Jordan with partial pivoting
 * inside the block: in registers / shared memory in 2D when the x-lines are
 * at most 128 nodes (complex64) or 96 (complex128) wide, otherwise (wider
 * 2D subdomains such as the paper's 300^2 + PML, and every 3D partition) as
 * dense blocks in global memory, each block step of the local solves then a
 * contraction over all subdomains and right-hand sides sharing a factor.
 * Errors: DDM_E_SINGULAR if a pivot fell below 1e-30 relative to its column,
 * DDM_E_CUDA, DDM_E_STATE.                                                  */
ddm_status ddm_factor(ddm_ctx *ctx);

/* dst = M_K(src): K steps of Algorithm 3.1 with right-hand side src, then the
 * assembled DDM solution sum_R beta_{0;R} sum_s u^s_R (Eq. (39)).  src and
 * dst are global complex128 vectors (nrhs of them, device).  src is in the
 * J-scaled space of b.  Requires ddm_factor.  Errors: DDM_E_INVAL (K < 1,
 * nrhs > max_rhs), DDM_E_STATE, DDM_E_CUDA.                                 */
ddm_status ddm_apply(ddm_ctx *ctx, int K, const void *src_dev, void *dst_dev, int nrhs);

/* Solve A u = h^2 J f for nrhs right-hand sides f (global complex128, device)
 * into u (device).  mode DDM_FGMRES: flexible GMRES(restart) right-
 * preconditioned by M_K, x0 = 0, classical Gram-Schmidt twice, stop when the
 * least-squares residual estimate <= tol (Section 4.2.2).  mode DDM_STEPPING:
 * Algorithm 3.1 continued as an iteration (Section 4.2.1), residual of the
 * assembled solution from the transfers of the last steps; in DDM_MIXED it
 * runs as iterative refinement around complex64 steps.  max_it bounds
 * FGMRES iterations (or DDM steps).  Every exit is checked with an explicit
 * FP64 residual, reported in info (may be NULL).  Errors: DDM_E_NOCONV,
 * DDM_E_INVAL, DDM_E_STATE, DDM_E_CUDA.                                     */
ddm_status ddm_solve(ddm_ctx *ctx, const void *f_dev, void *u_dev, int nrhs, double tol, int max_it,
                     int mode, int K, int restart, ddm_info *info);

/* ddm_solve with host buffers: copies f_host (complex128, nrhs global
 * vectors) to the device, solves, copies u back to u_host, synchronising the
 * stream.  Pinned host memory makes the copies asynchronous.                */
ddm_status ddm_solve_host(ddm_ctx *ctx, const void *f_host, void *u_host, int nrhs, double tol, int max_it,
                          int mode, int K, int restart, ddm_info *info);

/* enable != 0: every preconditioner application M_K (ddm_apply, and inside
 * ddm_solve's FGMRES) replays a CUDA graph of its kernels -- restriction, K
 * batched local solves, K-1 transfers, assembly -- captured on the first use
 * of each (nrhs, K) on a library-owned non-blocking stream and ordered with
 * the context's stream by events.  Inputs and outputs pass through staging
 * vectors held by the context.  0 turns it off.  2D partitions on the 2D
 * kernels only (x-lines of at most 128 / 96 nodes, see ddm_factor).
 * Errors: DDM_E_INVAL (3D, or wider 2D subdomains).                          */
ddm_status ddm_set_graph(ddm_ctx *ctx, int enable);

/* Block solves of Algorithm 3.1 on the tensor cores (DDM_MIXED only).  In 3D
 * every plane step of the forward and backward sweeps is a complex
 * contraction G_k Y over all subdomains and right-hand sides sharing a factor
 * (Section 3, the block LDU solve); with enable != 0 (the default) it runs
 * on tcgen05 in split TF32 ("3xTF32": hi*hi + hi*lo + lo*hi, FP32
 * accumulation, FP32-level accuracy), from a packed copy of the factor that
 * ddm_factor writes; 0 selects the CUDA-core FP32 kernels.  DDM_FP64 contexts
 * always use FP64 CUDA cores.  Takes effect from the next solve.
 * Errors: DDM_E_INVAL (null context).                                       */
ddm_status ddm_set_tensor_cores(ddm_ctx *ctx, int enable);

/* Kernel choice of the 2D local solves (Algorithm 3.1's block solves) for
 * nrhs > 1: nr = 1, 2, 4, 8 right-hand sides per CTA on the CUDA cores
 * (8: DDM_MIXED only), or nr = 64 per CTA on the tensor cores (DDM_MIXED
 * contexts with max_rhs >= 16, after ddm_factor, which then keeps a packed
 * split-TF32 copy of the factors; blocks of at most 128 rows).  0 (the
 * default) picks the fastest candidate by timing each once per context and
 * nrhs (ddm_autotune_log; the tensor-core candidate from nrhs >= 8).
 * Errors: DDM_E_INVAL (value not listed, or the tensor-core conditions not
 * met).                                                                     */
ddm_status ddm_set_rhs_per_cta(ddm_ctx *ctx, int nr);

/* Pivoting of the dense-block factorisation: 3D partitions, and 2D subdomains
 * wider than the 2D kernels (see ddm_factor).  Each Schur block D_k is
 * inverted by Gauss-Jordan in panels of 16 columns (8 in complex128).  With
 * tau > 0 (the default is 4) a panel's pivots are searched among its own
 * diagonal rows only.  Every CTA then eliminates the panel without waiting
 * for the others, instead of taking one cluster-wide search per pivot.  The
 * choice is checked: if an unpivoted row outside the panel holds more than
 * tau times its column's pivot (threshold pivoting with u = 1/tau), or a
 * panel has no usable pivot, ddm_factor redoes the whole factorisation with
 * partial pivoting over all rows.  The result then equals that of tau = 0,
 * which always searches all rows.  The Schur blocks of this method contain a
 * PML layer; partial pivoting over all rows takes their diagonal entries in
 * practice, so the check rarely fails.  Takes effect at the next ddm_factor.
 * ddm_pivoting_info returns tau and the number of factorisations redone so
 * far.  Errors: DDM_E_INVAL (null context, tau outside [0, 1e6]).           */
ddm_status ddm_set_pivoting(ddm_ctx *ctx, double tau);
ddm_status ddm_pivoting_info(const ddm_ctx *ctx, double *tau, int64_t *redone);

/* Local solver of Algorithm 3.1's subdomain problems.  The paper factors
 * each subdomain with a sparse direct (multifrontal) solver (Section 4).
 * DDM_LOCAL_BLOCK (the default): the block-tridiagonal LU in explicit-inverse
 * form described at ddm_factor.  DDM_LOCAL_ND (2D partitions only): a
 * multifrontal factorisation in nested-dissection order.  Each subdomain grid
 * is bisected recursively by grid lines until boxes of at most `leaf` nodes
 * remain (leaf 0: DDM_ND_LEAF_DEFAULT).  Every tree node's front is swept by
 * Gauss-Jordan over its separator, with partial pivoting inside the
 * separator.  A solve is one forward and one backward pass over the tree
 * heights, all subdomains and right-hand sides in the same launches.  At the
 * paper's 300^2 + PML subdomains it stores about 1/6 of the block factor's
 * entries and needs about 1/14 of its flops.  Its fronts, blocks and
 * arithmetic are FP64 in both precisions (CUDA cores): an interior front is
 * a box problem without PML damping, and near a resonance its pivot block is
 * too ill-conditioned for complex64.  In DDM_MIXED contexts only the source,
 * the output and U are complex64.  A change takes effect
 * at the next ddm_factor: the context is unfactored until then.  It also
 * drops captured graphs.  ddm_workspace_bytes bounds the default solver only.
 * Errors: DDM_E_INVAL (unknown solver, leaf outside 0..4096, DDM_LOCAL_ND on
 * a 3D partition, or DDM_LOCAL_BLOCK with graph replay on where the block
 * solver cannot replay).                                                    */
enum { DDM_LOCAL_BLOCK = 0, DDM_LOCAL_ND = 1 };
#define DDM_ND_LEAF_DEFAULT 32
ddm_status ddm_set_local_solver(ddm_ctx *ctx, int solver, int leaf);

/* The nested-dissection plan of an nx x ny subdomain grid (x fastest, node
 * index y*nx + x) with leaves of at most `leaf` nodes (0: the default).  Pure
 * host computation, no CUDA call.  Fills *info; each array that is not NULL
 * receives, with indices local to the plan:
 *   fronts  nfront x 12 ints, children before parents, the root last:
 *           s (pivots), d (boundary nodes), height (leaves 0), offset of its
 *           pivots in piv, offset of its boundary nodes in bnd, child 0,
 *           child 1 (-1 if none), offsets in cmap of child 0's and child 1's
 *           boundary positions, offset and count of its entries in ent,
 *           offset of its update vector;
 *   piv     n_piv node indices, the pivots of every front in elimination order;
 *   bnd     n_bnd node indices, each front's boundary nodes in ascending order;
 *   cmap    n_cmap positions (0..s+d-1) in the parent front of each child
 *           boundary node;
 *   ent     n_ent x 4 ints (row, col, node, plane): front[row][col] gets the
 *           operator's plane `plane` (0 centre, 1 x-, 2 x+, 3 y-, 4 y+) at
 *           local node `node`.
 * The factor stores factor_entries = sum over fronts of (s+d)*s elements.
 * Errors: DDM_E_INVAL (NULL info, nx or ny outside 1..4096, bad leaf).       */
typedef struct {
  int nfront, height;
  int64_t n_piv, n_bnd, n_cmap, n_ent;
  int64_t factor_entries, scratch_entries, update_entries;
} ddm_nd_plan_info;
ddm_status ddm_nd_plan(int nx, int ny, int leaf, ddm_nd_plan_info *info, int *fronts, int *piv, int *bnd, int *cmap,
                       int *ent);

/* Upper bound of the device bytes a context for `p` holds after ddm_setup,
 * ddm_factor (every subdomain counted with its own factor) and an FGMRES
 * solve of p->max_rhs right-hand sides with the given restart (0: no FGMRES
 * workspace).  Pure arithmetic on the parameters: no CUDA call, usable for
 * admission control before any allocation.  Errors: DDM_E_INVAL.            */
ddm_status ddm_workspace_bytes(const ddm_params *p, int restart, int64_t *bytes);

/* Release every device allocation of the context.  NULL is a no-op.        */
ddm_status ddm_destroy(ddm_ctx *ctx);

/* Message of the last error on ctx (or of the last failed ddm_setup when
 * ctx is NULL).  The string lives until the next call on the context.      */
const char *ddm_last_error(const ddm_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Building blocks, exported for parity tests and measurement.  All operate
 * on the context's partition and stream.
 * ------------------------------------------------------------------------ */

/* b = h^2 J f on the global grid (right-hand side of the J-scaled system,
 * Eq. (32)).  Global complex128 vectors, device.                      */
ddm_status ddm_rhs(ddm_ctx *ctx, const void *f_dev, void *b_dev, int nrhs);

/* y = A x with the global truncated operator (Section 3.1), FP64.          */
ddm_status ddm_global_apply(ddm_ctx *ctx, const void *x_dev, void *y_dev, int nrhs);

/* r = b - A x and, per right-hand side, norms_host[2*i] = ||r_i||_2,
 * norms_host[2*i+1] = ||b_i||_2 (FP64; synchronises).                       */
ddm_status ddm_residual(ddm_ctx *ctx, const void *b_dev, const void *x_dev, void *r_dev, int nrhs,
                        double *norms_host);

/* Local layout: number of subdomains, total local length (one right-hand
 * side), and (optional, host arrays of n_sub entries) each subdomain's
 * element offset for one right-hand side and its extended size along x, y,
 * z.  With nrhs right-hand sides, right-hand side r of subdomain s starts at
 * offsets[s] * nrhs + r * ext_x[s] * ext_y[s] * ext_z[s].                   */
ddm_status ddm_local_layout(const ddm_ctx *ctx, int *n_sub, int64_t *total, int64_t *offsets,
                            int *ext_x, int *ext_y, int *ext_z);

/* u_R = L^_R^{-1} src_R for every subdomain R (the batched local solves of
 * Eqs. (37)/(38)); local complex vectors (total * nrhs elements,
 * subdomain-major as above), device, in the context's local precision
 * (complex128 for DDM_FP64, complex64 for DDM_MIXED).                       */
ddm_status ddm_local_solve(ddm_ctx *ctx, const void *src_dev, void *u_dev, int nrhs);

/* Run `nsteps` steps of Algorithm 3.1 from the global right-hand side b_dev
 * (one right-hand side) and return: w_dev = the assembled solution after the
 * last step (global complex128, device, may be NULL); u_last_dev = the last
 * step's local solutions (local layout/precision, device, may be NULL); and
 * res_host[s-1] = || sum of the directional residuals of steps s, s-1(, s-2)
 * on the own regions ||_2 (= ||b - A w_s|| in exact arithmetic), s = 1..nsteps
 * (host array of nsteps doubles, may be NULL; res_host[0] is computed from
 * step 1's transfers).  Synchronises.                                       */
ddm_status ddm_steps(ddm_ctx *ctx, const void *b_dev, int nsteps, void *w_dev, void *u_last_dev,
                     double *res_host);

/* Device time of the kernels launched since the last reset, accumulated with
 * CUDA events on the context's stream when timing is enabled:
 * out_ms[0] local solves, [1] transfers, [2] assembly/restriction,
 * [3] global operator, [4] Krylov (Arnoldi, updates), [5] factorisation,
 * [6] graph replays of M_K (ddm_set_graph; their kernels are not in 0-2);
 * out_launches[i] the matching launch counts (arrays of 7; either may be
 * NULL).
 * enable != 0 turns recording on, 0 off; reset clears the sums.            */
ddm_status ddm_timing(ddm_ctx *ctx, int enable, int reset, double *out_ms, int64_t *out_launches);

/* Number of kernels this context has launched (since creation or the last
 * reset); reset != 0 clears the counter after reading it.                    */
ddm_status ddm_kernel_launches(ddm_ctx *ctx, int64_t *count, int reset);

/* Autotuner record of the 2D local solve: the first local solve of nrhs > 1
 * right-hand sides on a context times every right-hand-side grouping per CTA
 * (1, 2, 4, 8; 8 only in complex64) on its own input and keeps the fastest
 * for that nrhs.  Fills up to cap entries (nrhs, grouping, device ms) and
 * sets *count to the number recorded (any output may be NULL).              */
ddm_status ddm_autotune_log(const ddm_ctx *ctx, int cap, int *nrhs, int *nr, float *ms, int *count);

/* Bytes of subdomain factors read by one batched local solve of one
 * right-hand side per subdomain (each distinct factor streamed twice, once
 * per sweep, per subdomain using it), and bytes of factor storage.          */
ddm_status ddm_factor_bytes(const ddm_ctx *ctx, int64_t *bytes_per_solve, int64_t *bytes_stored);

/* ---------------------------------------------------------------------------
 * Allocation-free helper.  The paper has no counterpart: this is a service
 * for callers that cannot allocate device memory where they need it (a fixed
 * device-memory budget, a caching allocator that must not be re-entered, or a
 * section where cudaMalloc's implicit device synchronisation is not allowed).
 * ------------------------------------------------------------------------ */

/* norms_dev[i] = ||x_i||_2 for nvec complex128 vectors of n elements each,
 * stored one after another at x_dev (device).  norms_dev is a caller-owned
 * device array of nvec doubles.  Work is enqueued on `stream` (a
 * cudaStream_t, NULL = legacy default) and the call returns without
 * synchronising; read norms_dev after the stream has reached it.
 *
 * Allocates nothing: its reduction scratch is one static device array of
 * 304 x 16 + 16 doubles (about 39 KB) that every GPU which loads the library
 * keeps until the process exits.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress, with the device current) and
 * caches it; make that first call outside any stream capture.  The cached
 * address is valid for the device's primary context only: after
 * cudaDeviceReset the call must not be used again in that process.  All calls
 * share the one array, so calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 * Errors: DDM_E_INVAL for null pointers, n < 1 or nvec outside [1, 16] (the
 * static scratch holds 16 vectors), DDM_E_CUDA; the message is readable with
 * ddm_last_error(NULL).                                                      */
ddm_status ddm_norms_noalloc(const void *x_dev, int64_t n, int nvec, void *stream, double *norms_dev);

#ifdef __cplusplus
}
#endif
#endif /* DDM_H */
