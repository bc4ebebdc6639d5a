/*
 * nnmg.h - C interface of the GB300 non-nested matrix-free multigrid library.
 *
 * The library solves A_L u = f (Sec. 2, Eq. linear_system) for continuous
 * Q_k Lagrange elements (k = 1..4) on quadrilateral or hexahedral meshes with
 * conjugate gradients preconditioned by one non-nested multigrid V-cycle
 * (Sec. 2, Algorithm 1; Sec. 4 solver settings).  Levels are independent
 * meshes of the same domain (Sec. 2: T_{l-1} is not contained in T_l); the
 * transfer between them evaluates coarse basis functions at fine support
 * points (Sec. 2, Eqs. pointwise, residual2; Sec. 3.2, Eq.
 * tensor_product_evaluation) and restriction is its exact transpose.
 *
 * Conventions shared by every call
 * --------------------------------
 * Status: every call returns an int status (NNMG_OK = 0).  On failure the
 *   library records a message readable with nnmg_last_error() (per host
 *   thread) and leaves caller-owned outputs unspecified.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Device work is enqueued on it; calls that return host data
 *   synchronise it.
 * Ownership: the library copies every host input it needs; it owns all
 *   hierarchy memory until nnmg_destroy.  Device vectors passed to compute
 *   calls are owned by the caller and must stay valid until the stream has
 *   finished the call's work.
 * Precision: NNMG_F32 (float) or NNMG_F64 (double) for vector arguments
 *   declared as void*.
 * Vector layout: a vector on level l has n_nodes(l) * n_components rows; row
 *   r = node * n_components + component; each row holds nrhs contiguous
 *   values (right-hand side index fastest).  Element (node, comp, rhs) sits at
 *   ((node * n_components + comp) * nrhs + rhs).  Entries at Dirichlet-
 *   constrained DoFs are ignored on input and written as 0 on output.
 * Node numbering: a local node of a cell is identified by the combination of
 *   the cell's corner vertices that places it (integer weights
 *   W_v = prod_d (b_d(v) ? m_d : k - m_d) for local multi-index m and corner
 *   bits b(v)); nodes are numbered in order of first appearance, walking cells
 *   in index order and each cell's (k+1)^d local nodes lexicographically
 *   (x fastest).  Local node (m_0, m_1, m_2) sits at the Gauss-Lobatto point
 *   (xi_{m_0}, xi_{m_1}, xi_{m_2}) of the reference cell [0,1]^d.
 * Dirichlet set: all nodes on a boundary face (a face of exactly one cell)
 *   whose corner vertices are all flagged in dirichlet_vertex.
 * nrhs: 1 .. options.max_nrhs (<= 16).
 */
#ifndef NNMG_H
#define NNMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nnmg_handle nnmg_handle;

enum nnmg_status {
  NNMG_OK = 0,
  NNMG_INVALID_ARG = 1,     /* bad pointer, size, level index, nrhs or option   */
  NNMG_BAD_MESH = 2,        /* non-positive Jacobian determinant at a quadrature point, or a
                               non-conforming mesh (a shared face with inconsistent vertex order) */
  NNMG_POINT_NOT_FOUND = 3, /* a fine support point could not be located         */
  NNMG_CHOLESKY_FAIL = 4,   /* coarsest matrix not positive definite             */
  NNMG_OUT_OF_MEMORY = 5,   /* device or host allocation failed                  */
  NNMG_CUDA_ERROR = 6,      /* a CUDA runtime call failed                         */
  NNMG_NOT_CONVERGED = 7,   /* PCG reached maxit before rtol for some column      */
  NNMG_BREAKDOWN = 8        /* PCG met p.Ap <= 0 or a non-finite scalar           */
};

/* NNMG_F64_DW (nnmg_apply_operator only): FP64 vectors, arithmetic in
 * double-word form (pairs of floats, about 48 significand bits) on the FP32
 * pipes, which GB300 runs 61x faster than its FP64 pipe. */
enum nnmg_precision { NNMG_F32 = 0, NNMG_F64 = 1, NNMG_F64_DW = 2 };

enum nnmg_mode {
  NNMG_FP64_MG = 0,          /* V-cycle and CG in double precision                */
  NNMG_FP32_MG_FP64_CG = 1,  /* V-cycle in single precision inside a double CG (Sec. 4) */
  NNMG_FP32_MG_DW_CG = 2     /* as 1, with the CG's operator A p in double-word
                                arithmetic (vectors, dots and updates stay FP64) */
};

/* One level of the hierarchy: a conforming quad (dim 2) or hex (dim 3) mesh.
 * vertices: host, [n_vertices][dim] doubles.
 * cells: host, [n_cells][2^dim] vertex indices; local corner v = b0 + 2 b1 + 4 b2
 *   where b_d is the corner's offset bit in reference direction d.
 * dirichlet_vertex: host, [n_vertices] flags (NULL = no Dirichlet boundary).
 * degree: polynomial degree of this level, 1..4, or 0 for options.degree.
 *   Repeating the coarsest mesh with degrees 1, 2, .., k below the Q_k levels
 *   gives the polynomial-multigrid coarse solver of Sec. 2 ("Coarse grid
 *   solvers", Fig. hp_MG): the transfers between degrees on one mesh are the
 *   same point evaluations (nested there), and the direct solve acts on Q1. */
typedef struct {
  int dim;
  int64_t n_vertices;
  const double* vertices;
  int64_t n_cells;
  const int32_t* cells;
  const uint8_t* dirichlet_vertex;
  int degree;
} nnmg_level_desc;

/* Solver options (Sec. 4 solver settings; values in brackets are defaults).
 * degree k [1] of Q_k; n_components [1] (1 = Poisson, 3 = linear elasticity in
 * 3D, Sec. 4.4 Eq. linear_elasticity with Lame parameters lambda [1], mu [1]);
 * cheb_degree [3] Chebyshev steps per smoothing; smoothing_range [20] and
 * eig_safety [1.2] place the Chebyshev interval at
 * [eig_safety*lam/smoothing_range, eig_safety*lam] for lam the Lanczos
 * estimate after lanczos_steps [12] steps; max_nrhs [16] sizes work buffers.
 * deterministic [0] (no counterpart in the paper): 1 makes every result
 * bitwise reproducible from run to run.  Each level's cells are colored
 * greedily in input order so that no two cells of a color share a vertex,
 * and stored grouped by color (input order within a color; the DoF numbering
 * is that of the input order); the cell loops (operator, Jacobi diagonal,
 * load vector) run one launch per color, so that every output entry receives
 * at most one addition per launch and the additions' order is fixed.  Queries
 * and inputs that are per cell (nnmg_cell_nodes, nnmg_quadrature_points, a
 * load given per quadrature point) then use the stored order.  The operator
 * kernels follow the fixed default rule (no timed choice, which could differ
 * between two hierarchies), and the persistent smoother is not used.  A mesh
 * that needs more than 64 colors is BAD_MESH. */
typedef struct {
  int degree;
  int n_components;
  double lambda;
  double mu;
  int cheb_degree;
  double smoothing_range;
  int lanczos_steps;
  double eig_safety;
  int max_nrhs;
  int deterministic;
} nnmg_options;

/* Fill *opt with the defaults above. */
void nnmg_default_options(nnmg_options* opt);

/* Build a hierarchy from n_levels >= 1 meshes ordered coarse -> fine (Sec. 2:
 * level 1 coarsest, level L finest; here index 0 is the coarsest).  Setup
 * (Sec. 3.1, 3.2): DoF numbering, geometry at quadrature points, support
 * points, location of every free fine support point in the next coarser mesh
 * (bounding-box buckets, Newton inversion of the Q1 cell map, first accepting
 * cell by index, nearest-point projection onto [0,1]^d otherwise, Sec. 3.3
 * Eq. closest_point), point-Jacobi diagonals, Lanczos eigenvalue estimates and
 * the FP64 factorization of the coarsest operator.  Errors: INVALID_ARG,
 * BAD_MESH, POINT_NOT_FOUND, CHOLESKY_FAIL, OUT_OF_MEMORY, CUDA_ERROR. */
int nnmg_setup_hierarchy(const nnmg_level_desc* levels, int n_levels,
                         const nnmg_options* opt, void* stream, nnmg_handle** out);

/* Release all memory of a hierarchy (NULL is accepted). */
int nnmg_destroy(nnmg_handle* h);

/* Number of levels. */
int nnmg_n_levels(const nnmg_handle* h);

/* Sizes of one level: nodes, free (unconstrained) nodes and cells. */
int nnmg_level_info(const nnmg_handle* h, int level, int64_t* n_nodes,
                    int64_t* n_free_nodes, int64_t* n_cells);

/* Device bytes held by the hierarchy (used to admit work against a budget). */
size_t nnmg_hierarchy_bytes(const nnmg_handle* h);

/* Device bytes the work buffers of one solve with nrhs columns will add. */
size_t nnmg_solve_bytes(const nnmg_handle* h, int nrhs);

/* The same two sizes before anything is built (no counterpart in the paper:
 * it serves admission by a device-memory budget).  From the level
 * descriptions and options of nnmg_setup_hierarchy, on the host only (it
 * numbers the nodes of every level; no CUDA call, no device allocation):
 * *hierarchy_bytes (may be NULL) = what nnmg_hierarchy_bytes will report after
 * setup; *solve_bytes (may be NULL) = nnmg_solve_bytes(h, nrhs) of that
 * hierarchy.  Errors: INVALID_ARG (bad levels, options or nrhs outside
 * 1..16), BAD_MESH (non-conforming mesh), OUT_OF_MEMORY (host). */
int nnmg_estimate_bytes(const nnmg_level_desc* levels, int n_levels, const nnmg_options* opt,
                        int nrhs, size_t* hierarchy_bytes, size_t* solve_bytes);

/* Host copies of setup products of a level:
 * support points x_i = F_K(xi_i) [n_nodes][dim] (Sec. 2 Eq. pointwise);
 * constrained flags [n_nodes]; cell-to-node map [n_cells][(k+1)^d];
 * physical quadrature points [n_cells][(k+1)^d][dim] (Gauss-Legendre, Sec. 4). */
int nnmg_support_points(const nnmg_handle* h, int level, double* points);
int nnmg_constrained_nodes(const nnmg_handle* h, int level, uint8_t* flags);
int nnmg_cell_nodes(const nnmg_handle* h, int level, int32_t* cell_nodes);
int nnmg_quadrature_points(const nnmg_handle* h, int level, double* xq);

/* Cell colors of the deterministic mode (no counterpart in the paper).
 * nnmg_color_cells (host only, no handle): greedy coloring of the cells
 * [n_cells][2^dim] (vertex indices < n_vertices) in cell order, each cell
 * taking the smallest color no earlier cell sharing a vertex took;
 * color [n_cells] receives the colors, *n_colors their count.  INVALID_ARG
 * for bad arguments or vertex indices, BAD_MESH if more than 64 colors would
 * be needed.
 * nnmg_level_colors: *n_colors of a level of a hierarchy (0 when it was not
 * built deterministic) and, if color_start is not NULL, the first stored cell
 * of every color and the cell count [n_colors + 1]. */
int nnmg_color_cells(const int32_t* cells, int64_t n_cells, int64_t n_vertices, int dim,
                     uint8_t* color, int* n_colors);
int nnmg_level_colors(const nnmg_handle* h, int level, int64_t* color_start, int* n_colors);

/* The located coarse cell and reference point of every free fine node of
 * level fine_level >= 1 (Sec. 3.1), in increasing fine node order:
 * cell [n_free_fine], xi [n_free_fine][dim] (clamped to [0,1]^d). */
int nnmg_transfer_points(const nnmg_handle* h, int fine_level, int32_t* cell, double* xi);

/* Whether nnmg_pcg_solve / nnmg_pcg_solve_host for (mode, nrhs) now run as
 * one device-side graph loop (a CUDA graph WHILE node around one PCG
 * iteration; the host waits once per solve): *state = 1 built, 0 not built
 * yet (it is built on the second solve, after the first has tuned and
 * captured the iteration), -1 could not be built (the host-driven loop runs).
 * The environment variable NNMG_DEVICE_LOOP=0 keeps the host-driven loop.
 * No counterpart in the paper.  INVALID_ARG for a null handle or pointer. */
int nnmg_pcg_device_loop(const nnmg_handle* h, int mode, int nrhs, int* state);

/* Wall seconds of the setup phases of this hierarchy (no counterpart in the
 * paper, which does not time setup): seconds[NNMG_SETUP_PHASES] =
 * {0 node numbering (host), 1 per-level device geometry: metric terms,
 * support points, diagonal, 2 point location and transfer lists,
 * 3 restriction gather lists (host), 4 Lanczos eigenvalue estimates,
 * 5 coarsest operator assembly and dense inverse}.  INVALID_ARG for a null
 * handle or pointer. */
#define NNMG_SETUP_PHASES 6
int nnmg_setup_seconds(const nnmg_handle* h, double* seconds);

/* Which operator kernel serves level `level` in arithmetic `precision`
 * (enum nnmg_precision) for nrhs columns, as chosen so far on this handle
 * (no counterpart in the paper: an implementation detail exposed for
 * profiling).  *choice: -1 register-resident kernel (one thread per cell and
 * column), -2 its paired FP32 form (one thread per cell and two columns), U > 0
 * shared-memory kernel with U (cell, column) units per block, -100 - U its
 * paired FP32 form (3D Poisson, U (cell, column pair) units), 0 the default
 * rule (not tuned yet, autotuning off, or first used inside a stream capture).
 * INVALID_ARG for a null handle or pointer, a bad level, precision or nrhs. */
int nnmg_operator_choice(const nnmg_handle* h, int level, int precision, int nrhs, int* choice);

/* Lanczos estimate of lambda_max(D^-1 A_l) per level ([n_levels]; 0 on level 0). */
int nnmg_eigen_estimates(const nnmg_handle* h, double* lam_max);

/* Load vector b_(i,c) = sum_K sum_q w_q |det J| f_c(x_q) phi_i(xi_q) (Sec. 2,
 * (f_l, v) = b(v)) written into column rhs_col of the device FP64 vector b
 * [rows][nrhs].  f: host; if f_per_qp == 0 it holds n_components constants,
 * else values [n_cells][(k+1)^d][n_components] at nnmg_quadrature_points.
 * Constrained rows are written 0; other columns are left untouched. */
int nnmg_load_vector(nnmg_handle* h, int level, const double* f, int f_per_qp,
                     double* b, int nrhs, int rhs_col, void* stream);

/* y = A_l x (Sec. 2, (A_l w, v) = a(w, v)), matrix-free with sum
 * factorization (Sec. 3.2); x and y are device vectors of level `level` in
 * `precision`, distinct, [rows][nrhs]. */
int nnmg_apply_operator(nnmg_handle* h, int level, int precision, const void* x,
                        void* y, int nrhs, void* stream);

/* fine = P coarse (Sec. 2 transfer matrix P^(c,f); Sec. 3.2 evaluation at
 * reference points).  fine_level >= 1; `coarse` lives on fine_level-1.
 * Overwrites fine. */
int nnmg_prolongate(nnmg_handle* h, int fine_level, int precision, const void* coarse,
                    void* fine, int nrhs, void* stream);

/* coarse = P^T fine (Sec. 2 Eq. residual2), a deterministic two-phase gather:
 * bitwise reproducible for fixed inputs.  Overwrites coarse. */
int nnmg_restrict(nnmg_handle* h, int fine_level, int precision, const void* fine,
                  void* coarse, int nrhs, void* stream);

/* coarse = P^T fine, as nnmg_restrict, without allocating anything.  The paper
 * has no counterpart: this entry point exists for callers that must not
 * allocate device memory while they run (allocator-free real-time loops,
 * memory handed out by an external pool or budget, host callbacks, where
 * cudaMalloc may not be called).  Its scratch is a fixed 64 MiB array inside
 * the library, held by every GPU that loads the library until the process
 * exits; the call fails with INVALID_ARG when coarse cells x (k+1)^d x
 * components x nrhs x value size exceeds it.  The array's device address is
 * looked up by nnmg_setup_hierarchy (with the hierarchy's device current) and
 * kept with the handle, so even the first call allocates nothing; call it
 * with that device current (INVALID_ARG otherwise).  A device reset ends the
 * handle: set up a new one.  The array is shared by all calls: calls that
 * overlap on the GPU race, so order them on one stream.  Nothing needs
 * clearing between calls: the first phase writes every entry the second
 * reads. */
int nnmg_restrict_noalloc(nnmg_handle* h, int fine_level, int precision, const void* fine,
                          void* coarse, int nrhs, void* stream);

/* Switch the transfer between fine_level and fine_level-1 to the nested
 * (global-coarsening) form, the comparison system of the paper's Sec. 5: the
 * fine mesh must be the uniform 2^d refinement of the coarse one (same
 * degree, fine cells obtained by mapping the reference sub-cells through the
 * coarse Q1 map, corner order aligned with the parent).  parent_cell
 * [n_fine_cells] gives each fine cell's coarse cell, child_index
 * [n_fine_cells] its position (bit d = upper half in direction d).  The
 * transfer is then sum-factorized per child (the same operator P as the
 * point evaluation, evaluated differently).  parent_cell = NULL switches back
 * to the non-nested transfer.  Captured graphs are dropped. */
int nnmg_set_nested(nnmg_handle* h, int fine_level, const int32_t* parent_cell,
                    const uint8_t* child_index);

/* One V-cycle (Algorithm 1) on the finest level from a zero guess: z ~ A_L^-1 r.
 * Chebyshev-Jacobi pre- and post-smoothing, residual, restriction, recursion,
 * prolongation; coarsest level solved directly in FP64.  With the environment
 * variable NNMG_FUSED_SMOOTHER=1 each smoothing sweep of a small level served
 * by the register operator runs as one persistent cooperative kernel (grid
 * barriers between its operator and vector phases; not used by handles in
 * continuous batching).  With NNMG_FUSED_STEP=1 each Chebyshev step with an
 * operator pass on such a level is one launch without any wait (the cells add
 * A x, count themselves done on every node, and the block that completes a
 * node's count updates that node).  By default every step is an operator
 * kernel and a vector kernel, which measured faster than both. */
int nnmg_vcycle(nnmg_handle* h, int precision, const void* r, void* z, int nrhs,
                void* stream);

/* One V-cycle exactly as nnmg_vcycle (same kernels, same z), run eagerly with
 * CUDA events around every kernel, to time its parts per level as the paper's
 * Sec. 5 does (Fig. breakdown_serial: pre-smoother, residual, restrictor,
 * coarse-grid solver, prolongator, post-smoother).  Waits for `stream`.
 * ms (host, [n_levels][NNMG_PROF_COLS], overwritten): milliseconds summed
 * over the launches of each (level, column); columns NNMG_PROF_PRE ..
 * NNMG_PROF_POST are the six components (the coarse solve on level 0, the
 * others on levels >= 1; restriction and prolongation are booked on the fine
 * level of their pair), NNMG_PROF_OPERATOR and NNMG_PROF_VECTOR the same
 * launches by kernel class (operator applications; Chebyshev vector
 * updates).  The residual r_l = f_l - A_l x_l is formed inside the
 * restriction's first kernel, so the residual column holds the operator
 * application A_l x_l and the restrictor column the subtraction with the
 * transfer.  launches (host, same shape, may be NULL): how many
 * launches each entry sums.  Event timing adds a few microseconds per launch
 * on small levels.  INVALID_ARG for bad arguments or when called inside a
 * stream capture. */
#define NNMG_PROF_PRE 0
#define NNMG_PROF_RESIDUAL 1
#define NNMG_PROF_RESTRICT 2
#define NNMG_PROF_COARSE 3
#define NNMG_PROF_PROLONG 4
#define NNMG_PROF_POST 5
#define NNMG_PROF_OPERATOR 6
#define NNMG_PROF_VECTOR 7
#define NNMG_PROF_COLS 8
int nnmg_vcycle_profile(nnmg_handle* h, int precision, const void* r, void* z, int nrhs,
                        void* stream, double* ms, int* launches);

/* PCG in FP64 from x0 = 0, preconditioned by one V-cycle per iteration
 * (Sec. 4), per column until ||r_k||_2 <= rtol ||b||_2 (recursive residual).
 * b, x: device FP64 [rows][nrhs]; iters_out, relres_out: host [nrhs] (may be
 * NULL).  Returns NOT_CONVERGED (x still written) if a column misses rtol in
 * maxit iterations, BREAKDOWN on p.Ap <= 0 or a non-finite scalar. */
int nnmg_pcg_solve(nnmg_handle* h, int mode, const double* b, double* x, int nrhs,
                   double rtol, int maxit, int* iters_out, double* relres_out,
                   void* stream);

/* As nnmg_pcg_solve with HOST b and x (pinned or pageable); the copies to and
 * from the device are part of the call. */
int nnmg_pcg_solve_host(nnmg_handle* h, int mode, const double* b_host, double* x_host,
                        int nrhs, double rtol, int maxit, int* iters_out,
                        double* relres_out, void* stream);

/* Continuous batching (serving).  The PCG of nnmg_pcg_solve runs over
 * `nslots` independent columns; columns can be started and emptied between
 * iterations while the others continue, so requests that arrive while the GPU
 * works on earlier ones join the running solve as slots free up.  A column's
 * arithmetic does not depend on the other columns.  All calls of one handle
 * must use the same stream; different handles may run on different streams
 * concurrently.
 * nnmg_batch_reset: empty all nslots (<= max_nrhs) columns; mode, rtol (per
 *   column ||r|| <= rtol ||b||) and maxit (per column) as for nnmg_pcg_solve.
 * nnmg_batch_admit: start column `slot` from the FP64 right-hand side b [rows]
 *   (device, or host if b_on_host) with x0 = 0.
 * nnmg_batch_admit_cols: start columns first_slot .. first_slot + ncols - 1
 *   from columns 0 .. ncols - 1 of b [rows][ldb] (row-major, ldb >= ncols;
 *   device, or host if b_on_host with ldb <= max_nrhs: one contiguous copy of
 *   rows x ldb values, then the columns are spread on the device).
 * nnmg_batch_step: enqueue `iterations` PCG iterations of all columns
 *   (inactive columns stay frozen; a column that converges stops updating)
 *   and an asynchronous copy of the per-column state.
 * nnmg_batch_poll: if the last step has finished (or, with wait != 0, after
 *   waiting for it) set *ready = 1 and fill host arrays [nslots] (may be
 *   NULL): active flags, iteration counts, relative residuals and per-column
 *   status (NNMG_OK, NNMG_NOT_CONVERGED, NNMG_BREAKDOWN); else *ready = 0.
 * nnmg_batch_retire: enqueue the copy of column `slot` of x into x [rows]
 *   (device, or host if x_on_host; host memory should be pinned) and mark the
 *   slot empty.  The copy is asynchronous: read x after synchronising the
 *   stream or after the next nnmg_batch_poll that reports ready.
 * nnmg_batch_repack: change the batch to new_slots (1..max_nrhs) columns;
 *   column j < new_slots continues old column src[j] (host array of
 *   new_slots entries, distinct old slots or -1 for an empty column) with
 *   its iterate, residual, search direction and scalars unchanged; old
 *   columns not listed are dropped (retire them first).  Every later step
 *   costs in proportion to new_slots, so a server keeps the occupied columns
 *   packed into a batch no wider than it needs.  Call only when no step is
 *   in flight (after nnmg_batch_poll reported ready); enqueued on `stream`,
 *   no allocation.  Errors: INVALID_ARG, CUDA_ERROR. */
int nnmg_batch_reset(nnmg_handle* h, int mode, int nslots, double rtol, int maxit, void* stream);
int nnmg_batch_admit(nnmg_handle* h, int slot, const double* b, int b_on_host, void* stream);
int nnmg_batch_admit_cols(nnmg_handle* h, int first_slot, int ncols, const double* b, int ldb,
                          int b_on_host, void* stream);
int nnmg_batch_step(nnmg_handle* h, int iterations, void* stream);
int nnmg_batch_poll(nnmg_handle* h, int wait, int* ready, int* active, int* iters,
                    double* relres, int* status);
int nnmg_batch_retire(nnmg_handle* h, int slot, double* x, int x_on_host, void* stream);
int nnmg_batch_repack(nnmg_handle* h, int new_slots, const int* src, void* stream);

/* Arithmetic pipe rate of the current GPU (no counterpart in the paper: the
 * denominator of the rooflines of ALU-bound kernels).  Runs independent
 * fused multiply-add chains on every SM (8 per thread, 2048 threads per SM,
 * no memory traffic) for `iters` x 32 steps per chain, once to warm up and
 * once timed with CUDA events on `stream`; *fma_per_s = multiply-adds per
 * second.  kind: 0 FP64 (DFMA), 1 FP32 (FFMA), 2 packed FP32 pairs (FFMA2,
 * two multiply-adds per instruction).  Allocates a small device buffer.
 * Errors: INVALID_ARG, CUDA_ERROR. */
int nnmg_pipe_rate(int kind, int iters, void* stream, double* fma_per_s);

/* Message of the last failed call on this host thread ("" if none). */
const char* nnmg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NNMG_H */
