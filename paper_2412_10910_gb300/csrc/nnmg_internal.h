// Internal declarations of the GB300 non-nested multigrid library.
//
// Data layout in device memory (one hierarchy):
//   per level: cell_nodes [n_cells][(k+1)^d] int32 with -1 at Dirichlet nodes;
//   metric terms per quadrature point, [n_cells][n_metric][nqp] (component
//   outer, quadrature point inner, so neighbouring threads read neighbouring
//   words; rows padded to nqp = (k+1)^d rounded up to a multiple of 4, so a
//   row starts on a 16-byte boundary and loads as 16-byte vectors) in FP64 and
//   FP32; inverse Jacobi diagonals per row in FP64 and FP32;
//   for a level l >= 1 the located fine points sorted by coarse cell
//   (fine node, reference point) with a CSR start per coarse cell; for a level
//   used as coarse level the restriction gather list node -> (cell*nloc+local).
//   Vectors are [rows][nrhs] with rows = n_nodes * n_components.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/nnmg.h"

namespace nnmg {

constexpr int kMaxDegree = 4;
constexpr int kMaxN = kMaxDegree + 1;
constexpr int kMaxRhs = 16;
constexpr int kCoarseMaxSegments = 16;  // column segments of the coarse solve

// 1D tables for one degree k (n = k+1 points), passed to kernels by value.
//   S[q][l]  = L_l(g_q): Gauss-Lobatto Lagrange basis at Gauss point q
//   Dg[q][p] = derivative at g_q of the Lagrange basis on the Gauss points
//   DS[q][l] = L_l'(g_q)
//   gl[l]    = Gauss-Lobatto node l on [0,1]; gl_scale[l] = 1/prod_{m!=l}(gl_l-gl_m)
//   gx[q], gw[q] = Gauss-Legendre points and weights on [0,1]
template <typename T>
struct Basis1D {
  T S[kMaxN][kMaxN];
  T Dg[kMaxN][kMaxN];
  T DS[kMaxN][kMaxN];
  T gl[kMaxN];
  T gl_scale[kMaxN];
  T gx[kMaxN];
  T gw[kMaxN];
};

// Host side: tables in double for degree k (Newton on Legendre polynomials).
void make_basis(int k, Basis1D<double>* b64, Basis1D<float>* b32);

// Error record set by every entry point.
void set_error(const std::string& msg);
const char* get_error();

#define NNMG_CUDA(call)                                                         \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      ::nnmg::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));    \
      return NNMG_CUDA_ERROR;                                                   \
    }                                                                           \
  } while (0)

// ------------------------------------------------ programmatic dependent launch
// The V-cycle and PCG kernels are launched with programmatic stream
// serialization: a kernel may be scheduled before its predecessor in the
// stream has finished, and calls pdl_wait() before it reads or writes
// anything its predecessors produce (pdl_wait() returns at once when the
// kernel was launched without the attribute).  With the predecessor's
// implicit trigger (its blocks' exit) this hides launch latency between
// kernels: V-cycle 1.335 -> 1.326 ms, solve 31.86 -> 31.74 ms on config 2.
// An explicit trigger at every block's start (pdl_trigger(), built with
// NNMG_PDL_EARLY_TRIGGER=1) lets dependents occupy SM slots early and
// measured slower (V-cycle 1.343 -> 1.378 ms, solve 31.9 -> 33.4 ms), so
// pdl_trigger() compiles to nothing by default.  NNMG_PDL=0 in the
// environment launches without the attribute.
#ifndef NNMG_PDL_EARLY_TRIGGER
#define NNMG_PDL_EARLY_TRIGGER 0
#endif
__device__ __forceinline__ void pdl_trigger() {
#if NNMG_PDL_EARLY_TRIGGER
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

bool pdl_enabled();

template <typename... P, typename... A>
cudaError_t launch_k(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  if (pdl_enabled()) {
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// ---------------------------------------------------------------- host mesh
struct HostNumbering {
  std::vector<int32_t> cell_nodes;   // [nc][nloc]
  int64_t n_nodes = 0;
  std::vector<int32_t> owner_cell;   // [n_nodes]
  std::vector<int32_t> owner_local;  // [n_nodes]
  std::vector<uint8_t> constrained;  // [n_nodes]
};
int number_nodes(const int32_t* cells, int64_t nc, int64_t nv, int dim, int k,
                 const uint8_t* dirichlet_vertex, HostNumbering* out);

// Greedy vertex-disjoint coloring of cells (at most 64 colors; -1 if more
// would be needed), colors in [0, returned count).
int color_cells(const int32_t* cells, int64_t nc, int64_t nv, int dim, std::vector<uint8_t>* color);

struct BucketGeom {            // plain data, passed to the location kernel
  double lo[3], inv_w[3];
  int nb[3];
  double eps;                  // bounding-box widening
};
struct BucketGrid {
  BucketGeom geo;
  std::vector<int32_t> start;  // [n_buckets+1]
  std::vector<int32_t> cells;  // ascending within a bucket
};
void build_buckets(const double* vertices, const int32_t* cells, int64_t nc, int dim,
                   BucketGrid* g, std::vector<double>* aabb);



// ------------------------------------------------------------ device levels
struct DevLevel {
  int dim = 0, k = 0, n1 = 0, nloc = 0, ncomp = 1, nmetric = 0;
  int nqp = 0;                       // metric row stride: nloc rounded up to a multiple of 4
  int64_t n_vertices = 0, n_cells = 0, n_nodes = 0, n_free_nodes = 0, rows = 0;
  HostNumbering num;                 // host numbering (kept for queries)
  std::vector<double> h_vertices;
  std::vector<int32_t> h_cells;
  double* vertices = nullptr;        // [nv][dim]
  int32_t* cells = nullptr;          // [nc][2^dim]
  int32_t* cell_nodes = nullptr;     // [nc][nloc], -1 = constrained
  int32_t* owner_cell = nullptr;     // [n_nodes]
  int32_t* owner_local = nullptr;    // [n_nodes]
  double* metric64 = nullptr;        // [nc][nmetric][nqp], entries nloc..nqp-1 zero
  float* metric32 = nullptr;
  float* metric_dw = nullptr;        // double-word pairs (hi, lo) [nc][nmetric][nloc][2], on demand
  double* diag64 = nullptr;          // [rows] (0 at constrained rows)
  double* dinv64 = nullptr;          // [rows] (0 at constrained rows)
  float* dinv32 = nullptr;
  uint8_t* row_free = nullptr;       // [rows]
  double* points = nullptr;          // [n_nodes][dim]
  int32_t* valence = nullptr;        // [n_nodes] cells holding the node (0 if constrained)
  int32_t* node_count = nullptr;     // [n_nodes] finished cells of a fused step (0 at rest)
  double lam_max = 0.0;
  double cheb_a = 0.0, cheb_b = 0.0;
  // transfer from the next coarser level (this level is the fine one), l >= 1
  int64_t n_pts = 0;
  int32_t* pt_node = nullptr;        // [n_pts] fine node, sorted by coarse cell
  int32_t* pt_cell = nullptr;        // [n_pts] its coarse cell
  double* pt_xi64 = nullptr;         // [n_pts][dim]
  float* pt_xi32 = nullptr;
  int32_t* cell_pt_start = nullptr;  // [n_cells(coarse)+1]
  std::vector<int32_t> h_loc_cell;   // by increasing free fine node
  std::vector<double> h_loc_xi;
  // nested transfer from the next coarser level (global-coarsening comparison):
  // children of every coarse cell ordered by child index [n_cells(coarse)][2^d]
  int32_t* gc_children = nullptr;
  bool gc_active = false;
  // restriction gather lists of this level as a coarse level
  int32_t* gather_start = nullptr;   // [n_nodes+1]
  int32_t* gather_pos = nullptr;     // [..] cell*nloc + local, ascending
  // coarsest level direct solve
  int n_free_rows = 0;
  int32_t* free_rows = nullptr;      // [n_free_rows]
  double* coarse_inv = nullptr;      // [n_free_rows][n_free_rows]
  double* coarse_partial = nullptr;  // [kCoarseMaxSegments][n_free_rows][kMaxRhs]
  // deterministic mode: cells stored grouped by color, no two cells of a
  // color sharing a vertex; color c holds cells color_start[c] ..
  // color_start[c+1]-1 (empty: cells in input order, one launch per loop)
  std::vector<int64_t> color_start;
};

// Cells c0 .. c1-1 of L as a level of their own, for the cell-loop launchers
// (operator, diagonal, load vector): the per-cell device arrays are offset,
// node- and row-indexed arrays are shared, host data is not copied.
inline void cell_range_view(const DevLevel& L, int64_t c0, int64_t c1, DevLevel* V) {
  V->dim = L.dim;
  V->k = L.k;
  V->n1 = L.n1;
  V->nloc = L.nloc;
  V->ncomp = L.ncomp;
  V->nmetric = L.nmetric;
  V->nqp = L.nqp;
  V->n_vertices = L.n_vertices;
  V->n_nodes = L.n_nodes;
  V->n_free_nodes = L.n_free_nodes;
  V->rows = L.rows;
  V->n_cells = c1 - c0;
  V->vertices = L.vertices;
  V->cells = L.cells ? L.cells + c0 * (1 << L.dim) : nullptr;
  V->cell_nodes = L.cell_nodes ? L.cell_nodes + c0 * L.nloc : nullptr;
  const int64_t mrow = (int64_t)L.nmetric * L.nqp;
  V->metric64 = L.metric64 ? L.metric64 + c0 * mrow : nullptr;
  V->metric32 = L.metric32 ? L.metric32 + c0 * mrow : nullptr;
  V->metric_dw = L.metric_dw ? L.metric_dw + 2 * c0 * mrow : nullptr;
  V->diag64 = L.diag64;
  V->dinv64 = L.dinv64;
  V->dinv32 = L.dinv32;
  V->row_free = L.row_free;
  V->points = L.points;
  V->valence = L.valence;
  V->node_count = L.node_count;
}

// Run launch(level) once, or once per color on the color's cell range (the
// launches of one color add at most once into every output entry, so the
// result does not depend on the order of the atomic additions).
template <typename F>
cudaError_t for_each_color(const DevLevel& L, F launch) {
  if (L.color_start.empty()) return launch(L);
  for (size_t c = 0; c + 1 < L.color_start.size(); ++c) {
    const int64_t c0 = L.color_start[c], c1 = L.color_start[c + 1];
    if (c1 == c0) continue;
    DevLevel V;
    cell_range_view(L, c0, c1, &V);
    const cudaError_t e = launch(V);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------- kernels
// Launchers return cudaGetLastError() of the launch.
cudaError_t launch_metric(const DevLevel& L, int* d_err, cudaStream_t s);
cudaError_t launch_support_points(const DevLevel& L, cudaStream_t s);
cudaError_t launch_diag(const DevLevel& L, double lambda, double mu, cudaStream_t s);
cudaError_t launch_quad_points(const DevLevel& L, double* xq, cudaStream_t s);
cudaError_t launch_load_vector(const DevLevel& L, const double* f, int f_per_qp, double* b,
                               int nrhs, int col, cudaStream_t s);
cudaError_t launch_locate(const DevLevel& coarse, const double* points, const int32_t* pt_nodes,
                          int64_t n_pts, const int32_t* bucket_start, const int32_t* bucket_cells,
                          const double* aabb, const BucketGeom& g, int32_t* out_cell,
                          double* out_xi, cudaStream_t s);

// units = (cell, right-hand side) pairs per block; 0 selects the default rule.
template <typename T>
cudaError_t launch_operator(const DevLevel& L, const T* x, T* y, int nrhs, double lambda,
                            double mu, cudaStream_t s, int units = 0);
// y = A x with FP64 vectors and double-word arithmetic on the FP32 pipes
// (needs L.metric_dw).
cudaError_t launch_operator_dw(const DevLevel& L, const double* x, double* y, int nrhs,
                               double lambda, double mu, cudaStream_t s, int units = 0);
cudaError_t launch_split_dw(const double* a, float* hl, int64_t n, cudaStream_t s);
// Legal units-per-block choices of the operator kernel for this level (for the
// autotuner); returns how many were written to out.
template <typename T>
int operator_unit_candidates(const DevLevel& L, int nrhs, int* out, int max_out);
template <typename T>
cudaError_t launch_prolongate_add(const DevLevel& fine, const DevLevel& coarse, const T* xc,
                                  T* xf, int nrhs, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict(const DevLevel& fine, const DevLevel& coarse, const T* rf, T* rc,
                            T* scratch, int nrhs, cudaStream_t s);
// The non-nested transfer's kernels (k_prolong.cu, k_restrict.cu): x_f += P x_c;
// phase one of r_c = P^T r_f into the cell-local buffer [coarse cells][(k+1)^d]
// [ncomp * nrhs]; phase two, the fixed-order gather of that buffer into r_c.
template <typename T>
cudaError_t launch_prolongate_points(const DevLevel& fine, const DevLevel& coarse, const T* xc,
                                     T* xf, int nrhs, cudaStream_t s);
// With tres != nullptr, phase one forms the residual r_f = rf - tres itself
// and resets tres to zero at every free fine row.
template <typename T>
cudaError_t launch_restrict_points(const DevLevel& fine, const DevLevel& coarse, const T* rf,
                                   T* tres, T* scratch, int nrhs, cudaStream_t s);
// The residual r_l = f_l - t (t = A_l x_l) restricted to the coarse level in
// one pass (no residual vector): rc = P^T (f - t), t reset to zero.  The
// nested transfer forms the residual first.
template <typename T>
cudaError_t launch_restrict_residual(const DevLevel& fine, const DevLevel& coarse, const T* f,
                                     T* t, T* r_tmp, T* rc, T* scratch, int nrhs, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict_gather(const DevLevel& coarse, const T* scratch, T* rc, int nch,
                                   cudaStream_t s);
template <typename TI, typename TO>
cudaError_t launch_coarse_solve(const DevLevel& L, const TI* r, TO* z, int nrhs, cudaStream_t s);
// The free-row block of level L's operator into D [n][n] and its inverse in
// place (n = L.n_free_rows; blocked Gauss-Jordan, FP64).  X, Y: L.rows x
// kMaxRhs doubles; work: n x 64 + 64 x 64 doubles; *err set to 1 on a
// non-positive pivot.  Enqueued on s.
cudaError_t launch_coarse_inverse(const DevLevel& L, double lambda, double mu, double* D, double* X,
                                  double* Y, double* work, int* err, cudaStream_t s);

// One Chebyshev-Jacobi smoothing sweep as a single persistent (cooperative)
// kernel for small levels served by the register operator (Poisson, 3D k <= 2,
// 2D; at most a few waves of operator work, see cheb_smoother_supported):
// steps m; from_zero: start x = d = c_init D^-1 f (pre-smoothing) instead of
// an operator pass; step j (j >= 1 from zero, j >= 0 otherwise) computes
// t = A x, then d = cd[j] d + cr[j] D^-1 (f - t), x += d, t = 0; final_op
// ends with t = A x.  bar: two zeroed device words (barrier count and
// generation) owned by the caller; err: set to 1 if a grid barrier gave up.
// Returns cudaErrorNotSupported when the level has no fused form.
constexpr int kMaxChebSteps = 16;
struct SmootherPlan {
  int steps = 0, from_zero = 0, final_op = 0;
  double c_init = 0.0;
  double cd[kMaxChebSteps] = {0}, cr[kMaxChebSteps] = {0};
};
// Whether launch_cheb_smoother serves this level with m steps and nrhs columns.
bool cheb_smoother_supported(const DevLevel& L, int m, int nrhs);
// One Chebyshev step with its operator pass in one launch (Poisson levels the
// register kernel serves, not in the deterministic mode): t += A x, then at
// every node whose cells are all done d = cd d + cr D^-1 (f - t), x += d, t = 0.
bool cheb_step_fused_supported(const DevLevel& L);
template <typename T>
cudaError_t launch_cheb_step_fused(const DevLevel& L, const T* f, T* t, const T* dinv, T* d, T* x,
                                   double cd, double cr, int nrhs, cudaStream_t s);
template <typename T>
cudaError_t launch_cheb_smoother(const DevLevel& L, const T* f, T* t, const T* dinv, T* d, T* x,
                                 int nrhs, const SmootherPlan& P, unsigned* bar, int* err,
                                 cudaStream_t s);

// vector kernels, rows x nrhs
template <typename T>
cudaError_t launch_cheb_init(const T* f, const T* dinv, T* d, T* x, double c, int64_t rows,
                             int nrhs, cudaStream_t s);
template <typename T>
cudaError_t launch_cheb_step(const T* f, T* t, const T* dinv, T* d, T* x, double cd, double cr,
                             int64_t rows, int nrhs, cudaStream_t s);
template <typename T>
cudaError_t launch_residual(const T* f, T* t, T* r, int64_t rows, int nrhs, cudaStream_t s);
template <typename TI, typename TO>
cudaError_t launch_cast(const TI* a, TO* b, int64_t n, cudaStream_t s);

// PCG (FP64) helpers.  Per-column scalars live in a device struct.
// Per-column state: columns are independent, so a column can be (re)started
// between iterations while the others continue (continuous batching).
struct PcgScalars {
  double rho[kMaxRhs];
  double alpha[kMaxRhs];
  double beta[kMaxRhs];
  double bnorm[kMaxRhs];
  double rnorm[kMaxRhs];
  int active[kMaxRhs];
  int iters[kMaxRhs];
  int first[kMaxRhs];    // 1 until the column's first beta step (beta = 0)
  int failed[kMaxRhs];   // reached maxit without convergence
  int broken[kMaxRhs];   // p.Ap <= 0 or a non-finite scalar
  int any_active;
  int breakdown;         // any column broken
  int maxit;
  double rtol;
};
constexpr int kDotBlocks = 152 * 4;
constexpr int kDotThreads = 256;
template <typename TB>
cudaError_t launch_dot_partial(const double* a, const TB* b, double* partial, int64_t rows,
                               int nrhs, cudaStream_t s);
// The PCG writers of r also write r32 = (float) r, the FP32 V-cycle's input.
cudaError_t launch_pcg_init(const double* b, const uint8_t* row_free, double* r, float* r32,
                            double* x, double* p, double* partial, int64_t rows, int nrhs,
                            cudaStream_t s);
cudaError_t launch_pcg_start(PcgScalars* sc, const double* partial, int nrhs, double rtol,
                             int maxit, cudaStream_t s);
// Continuous batching: reset every column to inactive; start column `slot`
// from the right-hand side b [rows] (r = b on free rows, x = p = 0).
cudaError_t launch_batch_reset(PcgScalars* sc, double rtol, int maxit, cudaStream_t s);
// Start columns first_slot .. first_slot + ncols - 1 of the batch from the
// columns of b [rows][ldb].
cudaError_t launch_batch_admit(const double* b, int ldb, const uint8_t* row_free, double* r,
                               float* r32, double* x, double* p, double* partial, PcgScalars* sc,
                               int64_t rows, int nslots, int first_slot, int ncols, cudaStream_t s);
// out [rows] = column `slot` of v [rows][nslots].
cudaError_t launch_column_gather(const double* v, double* out, int64_t rows, int nslots, int slot,
                                 cudaStream_t s);
// Repack the batch's x, r (and its FP32 copy) and p from [rows][old_slots] to
// [rows][new_slots], column j taking old column m.s[j] (empty if < 0), through
// tmp [rows * new_slots], which is left zero; the per-column scalars move with
// their columns.
struct SlotMap {
  int s[kMaxRhs];
};
cudaError_t launch_batch_repack(double* x, double* r, float* r32, double* p, double* tmp,
                                PcgScalars* sc, int64_t rows, int old_slots, int new_slots,
                                const SlotMap& m, cudaStream_t s);
template <typename TZ>
cudaError_t launch_pcg_beta_p(PcgScalars* sc, const double* partial, const TZ* z, double* p,
                              int64_t rows, int nrhs, cudaStream_t s);
cudaError_t launch_pcg_alpha(PcgScalars* sc, const double* partial, int nrhs, cudaStream_t s);
cudaError_t launch_pcg_update(const PcgScalars* sc, const double* p, double* q, double* x,
                              double* r, float* r32, double* partial, int64_t rows, int nrhs,
                              cudaStream_t s);
// smoother_err (may be null): a set flag marks every active column broken.
cudaError_t launch_pcg_check(PcgScalars* sc, const double* partial, int nrhs, const int* smoother_err,
                             cudaStream_t s);
// Loop control of the device-side PCG loop (graph conditional WHILE node).
cudaError_t launch_pcg_loop_begin(cudaGraphConditionalHandle hc, const PcgScalars* sc, int* count,
                                  cudaStream_t s);
cudaError_t launch_pcg_loop_next(cudaGraphConditionalHandle hc, const PcgScalars* sc, int* count,
                                 cudaStream_t s);
// Lanczos helper: w = dinv .* u - beta * vprev  (nrhs = 1)
cudaError_t launch_axpby_dinv(const double* u, const double* dinv, const double* vprev,
                              double beta, double* w, int64_t rows, cudaStream_t s);
cudaError_t launch_dot_weighted(const double* a, const double* b, const double* wgt,
                                double* partial, int64_t rows, cudaStream_t s);
cudaError_t launch_axpy(double a, const double* x, double* y, double scale_y, int64_t rows,
                        cudaStream_t s);

}  // namespace nnmg
