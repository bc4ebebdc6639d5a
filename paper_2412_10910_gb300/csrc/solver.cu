// Hierarchy setup, V-cycle (Sec. 2 Algorithm 1), PCG (Sec. 4) and the C
// entry points declared in include/nnmg.h.
//
// The V-cycle and each PCG iteration are enqueued as a fixed sequence of
// kernels on internal buffers; after a first eager run they are captured once
// per (precision or mode, nrhs) into a CUDA graph and replayed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <map>
#include <new>
#include <tuple>
#include <type_traits>

#include "nnmg_internal.h"

using namespace nnmg;

namespace nnmg {
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = getenv("NNMG_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}
cudaError_t launch_finalize_diag(const double* diag, const uint8_t* row_free, double* dinv64,
                                 float* dinv32, int64_t rows, cudaStream_t s);
}

template <typename T>
struct WorkSet {
  bool ready = false;
  std::vector<T*> f, x, t, d, scratch;
};

struct nnmg_handle {
  nnmg_options opt;
  int device = -1;                  // the device current at setup
  // persistent smoother: grid barrier count and generation, then its error flag
  unsigned* smoother_sync = nullptr;
  // cooperative (persistent) smoother kernels allowed; off once the handle
  // serves continuous batching, whose engines run concurrently on other streams
  bool cooperative_ok = true;
  void* noalloc_scratch = nullptr;  // device address of nnmg_restrict_noalloc's array there
  std::vector<DevLevel> lv;
  cudaStream_t cap = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
  size_t work_bytes = 0;
  WorkSet<float> w32;
  WorkSet<double> w64;
  bool pcg_ready = false;
  double *px = nullptr, *pr = nullptr, *pp = nullptr, *pq = nullptr, *pb = nullptr;
  float* pr32 = nullptr;   // (float) pr: the FP32 V-cycle's input, written with pr
  double* partial = nullptr;
  PcgScalars* sc = nullptr;
  PcgScalars* h_sc = nullptr;
  std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;  // (kind, prec/mode, nrhs)
  std::map<std::tuple<int, int, int>, int> runs;
  // device-side PCG loops per (mode, nrhs); nullptr marks a failed build
  std::map<std::tuple<int, int>, cudaGraphExec_t> loops;
  int* loop_count = nullptr;
  std::map<std::tuple<int, int, int>, int> op_units;  // (level, precision, nrhs) -> units
  // wall seconds of the setup phases (see nnmg_setup_seconds in nnmg.h)
  double setup_s[NNMG_SETUP_PHASES] = {0};
  // continuous batching state
  int batch_mode = -1, batch_slots = 0;
  cudaEvent_t batch_ev = nullptr;
  bool batch_inflight = false;
};

namespace {

double wall_seconds() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

template <typename T>
cudaError_t dalloc(nnmg_handle* h, T** p, size_t count, bool work = false) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) return e;
  h->allocs.push_back((void*)*p);
  if (work)
    h->work_bytes += count * sizeof(T);
  else
    h->bytes += count * sizeof(T);
  return cudaSuccess;
}

#define CK(...)                                                                    \
  do {                                                                             \
    cudaError_t e_ = (__VA_ARGS__);                                                \
    if (e_ != cudaSuccess) {                                                       \
      set_error(std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));        \
      return e_ == cudaErrorMemoryAllocation ? NNMG_OUT_OF_MEMORY : NNMG_CUDA_ERROR; \
    }                                                                              \
  } while (0)

template <typename T>
const T* dinv_of(const DevLevel& L);
template <>
const float* dinv_of<float>(const DevLevel& L) { return L.dinv32; }
template <>
const double* dinv_of<double>(const DevLevel& L) { return L.dinv64; }

template <typename T>
WorkSet<T>& work_of(nnmg_handle* h);
template <>
WorkSet<float>& work_of<float>(nnmg_handle* h) { return h->w32; }
template <>
WorkSet<double>& work_of<double>(nnmg_handle* h) { return h->w64; }

template <typename T>
int ensure_work(nnmg_handle* h) {
  WorkSet<T>& W = work_of<T>(h);
  if (W.ready) return NNMG_OK;
  const int n = (int)h->lv.size();
  const int mr = h->opt.max_nrhs;
  if (!h->smoother_sync) {
    CK(dalloc(h, &h->smoother_sync, 4, true));
    CK(cudaMemset(h->smoother_sync, 0, 4 * sizeof(unsigned)));
  }
  W.f.assign(n, nullptr);
  W.x.assign(n, nullptr);
  W.t.assign(n, nullptr);
  W.d.assign(n, nullptr);
  W.scratch.assign(n, nullptr);
  for (int l = 0; l < n; ++l) {
    const DevLevel& L = h->lv[l];
    const size_t m = (size_t)L.rows * mr;
    CK(dalloc(h, &W.f[l], m, true));
    CK(dalloc(h, &W.x[l], m, true));
    CK(cudaMemset(W.f[l], 0, m * sizeof(T)));
    CK(cudaMemset(W.x[l], 0, m * sizeof(T)));
    if (l >= 1) {
      CK(dalloc(h, &W.t[l], m, true));
      CK(dalloc(h, &W.d[l], m, true));
      CK(cudaMemset(W.t[l], 0, m * sizeof(T)));
      CK(cudaMemset(W.d[l], 0, m * sizeof(T)));
      const DevLevel& C = h->lv[l - 1];
      const size_t sm = (size_t)C.n_cells * C.nloc * L.ncomp * mr;
      CK(dalloc(h, &W.scratch[l], sm, true));
    }
  }
  W.ready = true;
  return NNMG_OK;
}

// Double-word copies of the metric terms, made on first use of the
// double-word operator.
int ensure_dw(nnmg_handle* h, int level) {
  DevLevel& L = h->lv[level];
  if (L.metric_dw) return NNMG_OK;
  const size_t nm = (size_t)L.n_cells * L.nmetric * L.nqp;
  CK(dalloc(h, &L.metric_dw, 2 * nm));
  CK(launch_split_dw(L.metric64, L.metric_dw, (int64_t)nm, 0));
  CK(cudaStreamSynchronize(0));
  return NNMG_OK;
}

int ensure_pcg(nnmg_handle* h) {
  if (h->pcg_ready) return NNMG_OK;
  const DevLevel& L = h->lv.back();
  const size_t m = (size_t)L.rows * h->opt.max_nrhs;
  CK(dalloc(h, &h->px, m, true));
  CK(dalloc(h, &h->pr, m, true));
  CK(dalloc(h, &h->pp, m, true));
  CK(dalloc(h, &h->pq, m, true));
  CK(dalloc(h, &h->pb, m, true));
  CK(dalloc(h, &h->pr32, m, true));
  CK(cudaMemset(h->pq, 0, m * sizeof(double)));
  CK(dalloc(h, &h->partial, (size_t)kDotBlocks * kMaxRhs, true));
  CK(dalloc(h, &h->sc, 1, true));
  CK(dalloc(h, &h->loop_count, 1, true));
  CK(cudaMallocHost((void**)&h->h_sc, sizeof(PcgScalars)));
  h->pcg_ready = true;
  return NNMG_OK;
}

// ------------------------------------------------------------------ autotuner
// Operator kernel choice for (level, precision, nrhs): -1 the register-resident
// kernel, -2 its paired FP32 form, U > 0 the shared-memory kernel with U units
// per block, -100 - U its paired FP32 form, 0 the default rule.  On first use
// every legal choice is timed (two warm-ups and six timed launches on scratch
// vectors, CUDA events) and the fastest is kept for the handle's lifetime.
// Never runs during stream capture or in the deterministic mode (the default
// rule is used then);
// NNMG_AUTOTUNE=0 in the environment keeps the default rule, NNMG_OP_CHOICE=<c>
// forces choice c on every level (a choice that does not apply to a level
// falls back to the default there).
template <typename T, typename Launch>
int tune_units(nnmg_handle* h, int level, int prec_key, int nrhs, cudaStream_t s, Launch launch) {
  auto key = std::make_tuple(level, prec_key, nrhs);
  auto it = h->op_units.find(key);
  if (it != h->op_units.end()) return it->second;
  if (const char* f = getenv("NNMG_OP_CHOICE")) {
    const int c = atoi(f);
    h->op_units[key] = c;
    return c;
  }
  static const bool enabled = [] {
    const char* e = getenv("NNMG_AUTOTUNE");
    return !(e && e[0] == '0');
  }();
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  // the deterministic mode keeps the default rule: a choice made by timing
  // could differ between two hierarchies and with it the rounding
  if (!enabled || h->opt.deterministic || cudaStreamIsCapturing(s, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone)
    return 0;
  const DevLevel& L = h->lv[level];
  int cand[16];
  const int nc = operator_unit_candidates<T>(L, nrhs, cand, 16);
  int best = 0;
  if (nc > 1 && L.n_cells > 0) {
    using IO = std::conditional_t<sizeof(T) == 4, float, double>;
    IO *x = nullptr, *y = nullptr;
    const size_t n = (size_t)L.rows * nrhs;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&x, n * sizeof(IO)) == cudaSuccess && cudaMalloc(&y, n * sizeof(IO)) == cudaSuccess &&
        cudaMemsetAsync(x, 0, n * sizeof(IO), s) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
      float best_ms = 1e30f;
      for (int c = 0; c < nc; ++c) {
        bool ok = launch(L, x, y, cand[c]) == cudaSuccess;
        ok = ok && launch(L, x, y, cand[c]) == cudaSuccess;
        ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
        for (int r = 0; r < 6 && ok; ++r) ok = launch(L, x, y, cand[c]) == cudaSuccess;
        ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0.f;
        if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
          best_ms = ms;
          best = cand[c];
        }
      }
    }
    cudaGetLastError();  // a rejected candidate must not leave a sticky launch error
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (x) cudaFree(x);
    if (y) cudaFree(y);
  }
  h->op_units[key] = best;
  return best;
}

template <typename T>
int op_units(nnmg_handle* h, int level, int nrhs, cudaStream_t s) {
  return tune_units<T>(h, level, sizeof(T) == 8 ? NNMG_F64 : NNMG_F32, nrhs, s,
                       [&](const DevLevel& L, T* x, T* y, int c) {
                         return launch_operator<T>(L, x, y, nrhs, h->opt.lambda, h->opt.mu, s, c);
                       });
}

// The double-word operator (FP64 vectors, FP32 pipes).
int op_units_dw(nnmg_handle* h, int level, int nrhs, cudaStream_t s) {
  return tune_units<double>(h, level, NNMG_F64_DW, nrhs, s,
                            [&](const DevLevel& L, double* x, double* y, int c) {
                              return launch_operator_dw(L, x, y, nrhs, h->opt.lambda, h->opt.mu, s, c);
                            });
}

// ------------------------------------------------------------------ V-cycle
// Algorithm 1 with Chebyshev-Jacobi smoothing (Sec. 4): pre-smoothing from a
// zero guess (m steps, m-1 operator applications), residual, restriction
// r_{l-1} = P^T r_l, recursion, prolongation x_l += P delta_{l-1},
// post-smoothing continuing from x_l (m steps), FP64 direct solve on level 0.
//
// With a VcycleTimer (nnmg_vcycle_profile) every launch is bracketed by CUDA
// events and attributed to its level, its component of the paper's Sec. 5
// breakdown and its kernel class; all other runs pass none.
struct VcycleTimer {
  struct Mark {
    int level, col_component, col_kind;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  ~VcycleTimer() {
    for (auto& m : marks) {
      if (m.a) cudaEventDestroy(m.a);
      if (m.b) cudaEventDestroy(m.b);
    }
  }
  cudaError_t start(int level, int comp, int kind, cudaStream_t s) {
    Mark m{level, comp, kind, nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&m.a);
    if (e == cudaSuccess) e = cudaEventCreate(&m.b);
    marks.push_back(m);
    return e == cudaSuccess ? cudaEventRecord(m.a, s) : e;
  }
  cudaError_t stop(cudaStream_t s) { return cudaEventRecord(marks.back().b, s); }
};

// Forget the captured V-cycle, iteration and loop graphs (they are captured
// again on later calls).  The caller makes sure none is running.
void drop_graphs(nnmg_handle* h) {
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  h->runs.clear();
  for (auto& kv : h->loops)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  h->loops.clear();
}

bool fused_residual_allowed() {
  const char* e = getenv("NNMG_FUSED_RESIDUAL");    // read when a V-cycle is enqueued or captured
  return !(e && e[0] == '0');
}

int* smoother_err(nnmg_handle* h) {
  return h->smoother_sync ? reinterpret_cast<int*>(h->smoother_sync + 2) : nullptr;
}

// The persistent smoother (one cooperative kernel per Chebyshev sweep) serves
// small levels whose operator is the register kernel (autotuned choice -1, or
// the default rule) when NNMG_FUSED_SMOOTHER=1 is set.  It is off by default:
// inside the captured V-cycle graph a kernel boundary costs about a
// microsecond and the grid barriers more, so the kernel-per-step sequence is
// faster (config 2 V-cycle 1.327 ms without, 1.358 ms with the smoother on its
// three coarser levels, 1.622 ms with it on every level; config 1 solve 0.83 ms
// either way).
bool fused_smoother_allowed(const nnmg_handle* h, const DevLevel& L, int op_choice, int m,
                            int nrhs) {
  const char* e = getenv("NNMG_FUSED_SMOOTHER");    // read when a V-cycle is enqueued or captured
  const bool on = e && e[0] == '1';
  return on && h->cooperative_ok && L.color_start.empty() && (op_choice == -1 || op_choice == 0) &&
         cheb_smoother_supported(L, m, nrhs);
}

// The fused operator + Chebyshev step (opt-in: NNMG_FUSED_STEP=1 in the
// environment; measured slower than the operator and vector kernels apart)
// serves a level where the register kernel is the operator choice.
bool fused_step_allowed(const DevLevel& L, int op_choice) {
  const char* e = getenv("NNMG_FUSED_STEP");          // read when a V-cycle is enqueued or captured
  const bool on = e && e[0] == '1';
  return on && (op_choice == -1 || op_choice == 0) && cheb_step_fused_supported(L);
}

// Chebyshev coefficients of one sweep (Sec. 4 smoother; the recurrence of
// the kernel-per-step path): pre-smoothing from zero, or continuing from x.
SmootherPlan smoother_plan(const DevLevel& L, int m, bool pre) {
  SmootherPlan P;
  const double a = L.cheb_a, b = L.cheb_b;
  const double theta = 0.5 * (a + b), delta = 0.5 * (b - a), sigma = theta / delta;
  P.steps = m;
  P.from_zero = pre ? 1 : 0;
  P.final_op = pre ? 1 : 0;
  P.c_init = 1.0 / theta;
  P.cd[0] = 0.0;
  P.cr[0] = 1.0 / theta;
  double rho = 1.0 / sigma;
  for (int j = 1; j < m && j < kMaxChebSteps; ++j) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    P.cd[j] = rn * rho;
    P.cr[j] = 2.0 * rn / delta;
    rho = rn;
  }
  return P;
}

template <typename T>
cudaError_t enqueue_vcycle(nnmg_handle* h, const T* f_top, int nrhs, cudaStream_t s,
                           VcycleTimer* P = nullptr) {
  WorkSet<T>& W = work_of<T>(h);
  const int top = (int)h->lv.size() - 1;
  const int m = h->opt.cheb_degree;
  const double lam = h->opt.lambda, mu = h->opt.mu;
  cudaError_t e;
#define RET(...)                        \
  do {                                  \
    e = (__VA_ARGS__);                  \
    if (e != cudaSuccess) return e;     \
  } while (0)
  // a launch of component `comp` (NNMG_PROF_*) and kernel class `kind`
#define RUN(level, comp, kind, ...)                   \
  do {                                                \
    if (P) RET(P->start(level, comp, kind, s));       \
    RET(__VA_ARGS__);                                 \
    if (P) RET(P->stop(s));                           \
  } while (0)
  for (int l = top; l >= 1; --l) {
    const DevLevel& L = h->lv[l];
    const T* f = l == top ? f_top : W.f[l];
    T *x = W.x[l], *t = W.t[l], *d = W.d[l];
    const T* dinv = dinv_of<T>(L);
    const int ou = op_units<T>(h, l, nrhs, s);
    const double a = L.cheb_a, b = L.cheb_b;
    const double theta = 0.5 * (a + b), delta = 0.5 * (b - a), sigma = theta / delta;
    // pre-smoothing and the residual's operator pass in one persistent kernel
    // where the level has one, else kernel by kernel
    bool fused = false;
    if (fused_smoother_allowed(h, L, ou, m, nrhs)) {
      RUN(l, NNMG_PROF_PRE, NNMG_PROF_OPERATOR,
          launch_cheb_smoother<T>(L, f, t, dinv, d, x, nrhs, smoother_plan(L, m, true),
                                  h->smoother_sync, smoother_err(h), s));
      fused = true;
    }
    if (!fused) {
      RUN(l, NNMG_PROF_PRE, NNMG_PROF_VECTOR,
          launch_cheb_init<T>(f, dinv, d, x, 1.0 / theta, L.rows, nrhs, s));
      double rho = 1.0 / sigma;
      const bool fs = fused_step_allowed(L, ou);
      for (int j = 1; j < m; ++j) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        if (fs) {
          RUN(l, NNMG_PROF_PRE, NNMG_PROF_OPERATOR,
              launch_cheb_step_fused<T>(L, f, t, dinv, d, x, rn * rho, 2.0 * rn / delta, nrhs, s));
        } else {
          RUN(l, NNMG_PROF_PRE, NNMG_PROF_OPERATOR,
              launch_operator<T>(L, x, t, nrhs, lam, mu, s, ou));
          RUN(l, NNMG_PROF_PRE, NNMG_PROF_VECTOR,
              launch_cheb_step<T>(f, t, dinv, d, x, rn * rho, 2.0 * rn / delta, L.rows, nrhs, s));
        }
        rho = rn;
      }
      RUN(l, NNMG_PROF_RESIDUAL, NNMG_PROF_OPERATOR,
          launch_operator<T>(L, x, t, nrhs, lam, mu, s, ou));
    }
    // r_l = f_l - A_l x_l formed inside the restriction (t reset to zero there);
    // NNMG_FUSED_RESIDUAL=0 runs the residual kernel and the plain restriction
    if (fused_residual_allowed()) {
      RUN(l, NNMG_PROF_RESTRICT, NNMG_PROF_RESTRICT,
          launch_restrict_residual<T>(L, h->lv[l - 1], f, t, d, W.f[l - 1], W.scratch[l], nrhs, s));
    } else {
      RUN(l, NNMG_PROF_RESIDUAL, NNMG_PROF_VECTOR, launch_residual<T>(f, t, d, L.rows, nrhs, s));
      RUN(l, NNMG_PROF_RESTRICT, NNMG_PROF_RESTRICT,
          launch_restrict<T>(L, h->lv[l - 1], d, W.f[l - 1], W.scratch[l], nrhs, s));
    }
  }
  {
    const T* f0 = top == 0 ? f_top : W.f[0];
    RUN(0, NNMG_PROF_COARSE, NNMG_PROF_COARSE,
        launch_coarse_solve<T, T>(h->lv[0], f0, W.x[0], nrhs, s));
  }
  for (int l = 1; l <= top; ++l) {
    const DevLevel& L = h->lv[l];
    const T* f = l == top ? f_top : W.f[l];
    T *x = W.x[l], *t = W.t[l], *d = W.d[l];
    const T* dinv = dinv_of<T>(L);
    RUN(l, NNMG_PROF_PROLONG, NNMG_PROF_PROLONG,
        launch_prolongate_add<T>(L, h->lv[l - 1], W.x[l - 1], x, nrhs, s));
    const int ou = op_units<T>(h, l, nrhs, s);
    const double a = L.cheb_a, b = L.cheb_b;
    const double theta = 0.5 * (a + b), delta = 0.5 * (b - a), sigma = theta / delta;
    if (fused_smoother_allowed(h, L, ou, m, nrhs)) {
      RUN(l, NNMG_PROF_POST, NNMG_PROF_OPERATOR,
          launch_cheb_smoother<T>(L, f, t, dinv, d, x, nrhs, smoother_plan(L, m, false),
                                  h->smoother_sync, smoother_err(h), s));
      continue;
    }
    double rho = 1.0 / sigma;
    const bool fs = fused_step_allowed(L, ou);
    for (int j = 0; j < m; ++j) {
      double cd = 0.0, cr = 1.0 / theta;
      if (j > 0) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        cd = rn * rho;
        cr = 2.0 * rn / delta;
        rho = rn;
      }
      if (fs) {
        RUN(l, NNMG_PROF_POST, NNMG_PROF_OPERATOR,
            launch_cheb_step_fused<T>(L, f, t, dinv, d, x, cd, cr, nrhs, s));
      } else {
        RUN(l, NNMG_PROF_POST, NNMG_PROF_OPERATOR,
            launch_operator<T>(L, x, t, nrhs, lam, mu, s, ou));
        RUN(l, NNMG_PROF_POST, NNMG_PROF_VECTOR,
            launch_cheb_step<T>(f, t, dinv, d, x, cd, cr, L.rows, nrhs, s));
      }
    }
  }
#undef RUN
#undef RET
  return cudaSuccess;
}

// One PCG iteration: z = M r, beta, p = z + beta p, q = A p, alpha, x, r updates,
// convergence check.  All per-column scalars stay on the device.
cudaError_t enqueue_pcg_iter(nnmg_handle* h, int mode, int nrhs, cudaStream_t s) {
  const DevLevel& L = h->lv.back();
  const int top = (int)h->lv.size() - 1;
  const int64_t rows = L.rows;
  cudaError_t e;
  if (mode == NNMG_FP32_MG_FP64_CG || mode == NNMG_FP32_MG_DW_CG) {
    e = enqueue_vcycle<float>(h, h->pr32, nrhs, s);
    if (e != cudaSuccess) return e;
    const float* z = h->w32.x[top];
    if ((e = launch_dot_partial<float>(h->pr, z, h->partial, rows, nrhs, s)) != cudaSuccess) return e;
    if ((e = launch_pcg_beta_p<float>(h->sc, h->partial, z, h->pp, rows, nrhs, s)) != cudaSuccess) return e;
  } else {
    e = enqueue_vcycle<double>(h, h->pr, nrhs, s);
    if (e != cudaSuccess) return e;
    const double* z = h->w64.x[top];
    if ((e = launch_dot_partial<double>(h->pr, z, h->partial, rows, nrhs, s)) != cudaSuccess) return e;
    if ((e = launch_pcg_beta_p<double>(h->sc, h->partial, z, h->pp, rows, nrhs, s)) != cudaSuccess) return e;
  }
  if (mode == NNMG_FP32_MG_DW_CG)
    e = launch_operator_dw(L, h->pp, h->pq, nrhs, h->opt.lambda, h->opt.mu, s,
                           op_units_dw(h, top, nrhs, s));
  else
    e = launch_operator<double>(L, h->pp, h->pq, nrhs, h->opt.lambda, h->opt.mu, s,
                                op_units<double>(h, top, nrhs, s));
  if (e != cudaSuccess) return e;
  if ((e = launch_dot_partial<double>(h->pp, h->pq, h->partial, rows, nrhs, s)) != cudaSuccess) return e;
  if ((e = launch_pcg_alpha(h->sc, h->partial, nrhs, s)) != cudaSuccess) return e;
  if ((e = launch_pcg_update(h->sc, h->pp, h->pq, h->px, h->pr, h->pr32, h->partial, rows, nrhs, s)) != cudaSuccess) return e;
  return launch_pcg_check(h->sc, h->partial, nrhs, smoother_err(h), s);
}

// Run `body` on stream s: eagerly on the first call for `key`, from a captured
// CUDA graph afterwards.
template <typename F>
int run_graph(nnmg_handle* h, std::tuple<int, int, int> key, cudaStream_t s, F body) {
  auto it = h->graphs.find(key);
  if (it != h->graphs.end()) {
    CK(cudaGraphLaunch(it->second, s));
    return NNMG_OK;
  }
  int& runs = h->runs[key];
  if (runs == 0) {
    runs = 1;
    CK(body(s));
    return NNMG_OK;
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t eb = body(h->cap);
  cudaError_t ee = cudaStreamEndCapture(h->cap, &g);
  if (eb != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    set_error(std::string("graph capture failed: ") +
              cudaGetErrorString(eb != cudaSuccess ? eb : ee));
    return NNMG_CUDA_ERROR;
  }
  cudaGraphExec_t ex = nullptr;
  cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    set_error(std::string("graph instantiate: ") + cudaGetErrorString(ei));
    return NNMG_CUDA_ERROR;
  }
  h->graphs[key] = ex;
  CK(cudaGraphLaunch(ex, s));
  return NNMG_OK;
}

// The whole PCG loop as one graph: a kernel arms a WHILE node whose body is
// one iteration (the kernels of enqueue_pcg_iter) and the re-arming kernel;
// the host then waits once per solve instead of once per iteration.  Built
// after the iteration has run eagerly (so the autotuner's choices exist);
// returns nullptr if the graph cannot be built (the host-driven loop runs).
cudaGraphExec_t build_pcg_loop(nnmg_handle* h, int mode, int nrhs) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaGraphConditionalHandle hc;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&hc, g, 0, 0) == cudaSuccess;
  cudaGraphNode_t pre = nullptr;
  if (ok) {
    ok = cudaStreamBeginCaptureToGraph(h->cap, g, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const bool launched = launch_pcg_loop_begin(hc, h->sc, h->loop_count, h->cap) == cudaSuccess;
      cudaGraph_t gg = g;
      ok = cudaStreamEndCapture(h->cap, &gg) == cudaSuccess && launched;
    }
    size_t nn = 0;
    ok = ok && cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn == 1 &&
         cudaGraphGetNodes(g, &pre, &nn) == cudaSuccess;
  }
  cudaGraph_t body = nullptr;
  if (ok) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn;
    ok = cudaGraphAddNode(&cn, g, &pre, nullptr, 1, &cp) == cudaSuccess;
    if (ok) body = cp.conditional.phGraph_out[0];
  }
  if (ok) {
    ok = cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      bool launched = enqueue_pcg_iter(h, mode, nrhs, h->cap) == cudaSuccess;
      launched = launched && launch_pcg_loop_next(hc, h->sc, h->loop_count, h->cap) == cudaSuccess;
      cudaGraph_t bb = body;
      ok = cudaStreamEndCapture(h->cap, &bb) == cudaSuccess && launched;
    }
  }
  if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    if (ex) cudaGraphExecDestroy(ex);
    ex = nullptr;
    cudaGetLastError();   // leave no sticky error behind
  }
  return ex;
}

// ------------------------------------------------------------------ setup
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int n = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {  // Sturm count of eigenvalues < x
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < n; ++i) {
      d = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 300; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (count_below(mid) == n)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

double sum_partial_host(const std::vector<double>& p) {
  double s = 0.0;
  for (int b = 0; b < kDotBlocks; ++b) s += p[(size_t)b * kMaxRhs];
  return s;
}

int lanczos(nnmg_handle* h, DevLevel& L, cudaStream_t s) {
  const int64_t n = L.rows;
  if (L.n_free_nodes == 0) {
    L.lam_max = 1.0;
    return NNMG_OK;
  }
  std::vector<double> v0((size_t)n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    if (!L.num.constrained[i / L.ncomp]) v0[i] = 1.0 + 0.01 * (double)((i % 17) - 8);
  double *v, *vp, *w, *u, *part;
  CK(cudaMalloc(&v, n * sizeof(double)));
  CK(cudaMalloc(&vp, n * sizeof(double)));
  CK(cudaMalloc(&w, n * sizeof(double)));
  CK(cudaMalloc(&u, n * sizeof(double)));
  CK(cudaMalloc(&part, (size_t)kDotBlocks * kMaxRhs * sizeof(double)));
  std::vector<double> hp((size_t)kDotBlocks * kMaxRhs);
  auto dotD = [&](const double* a, const double* b, double* out) -> int {
    CK(launch_dot_weighted(a, b, L.diag64, part, n, s));
    CK(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *out = sum_partial_host(hp);
    return NNMG_OK;
  };
  int rc = NNMG_OK;
  std::vector<double> al, be;
  do {
    CK(cudaMemcpyAsync(v, v0.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(vp, 0, n * sizeof(double), s));
    CK(cudaMemsetAsync(w, 0, n * sizeof(double), s));
    double nn;
    if ((rc = dotD(v, v, &nn)) != NNMG_OK) break;
    CK(launch_axpy(0.0, v, v, 1.0 / std::sqrt(nn), n, s));
    double beta = 0.0;
    for (int j = 0; j < h->opt.lanczos_steps; ++j) {
      CK(cudaMemsetAsync(u, 0, n * sizeof(double), s));
      CK(launch_operator<double>(L, v, u, 1, h->opt.lambda, h->opt.mu, s));
      CK(launch_axpby_dinv(u, L.dinv64, vp, beta, w, n, s));
      double alpha;
      if ((rc = dotD(w, v, &alpha)) != NNMG_OK) break;
      CK(launch_axpy(-alpha, v, w, 1.0, n, s));
      double ww;
      if ((rc = dotD(w, w, &ww)) != NNMG_OK) break;
      beta = std::sqrt(std::max(ww, 0.0));
      al.push_back(alpha);
      be.push_back(beta);
      if (beta == 0.0) break;
      std::swap(vp, v);                                 // vp <- v
      CK(launch_axpy(1.0 / beta, w, v, 0.0, n, s));     // v <- w / beta
    }
  } while (false);
  cudaFree(v);
  cudaFree(vp);
  cudaFree(w);
  cudaFree(u);
  cudaFree(part);
  if (rc != NNMG_OK) return rc;
  L.lam_max = tridiag_max_eig(al, be);
  return NNMG_OK;
}

// The coarsest level's direct solve: the dense free-row block of its operator
// and the inverse, both built on the device (k_dense.cu).
int setup_coarse(nnmg_handle* h, DevLevel& L, cudaStream_t s) {
  std::vector<int32_t> rows;
  for (int64_t r = 0; r < L.rows; ++r)
    if (!L.num.constrained[r / L.ncomp]) rows.push_back((int32_t)r);
  const int n = (int)rows.size();
  L.n_free_rows = n;
  CK(dalloc(h, &L.free_rows, std::max(n, 1)));
  if (n == 0) return NNMG_OK;
  CK(cudaMemcpy(L.free_rows, rows.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(dalloc(h, &L.coarse_inv, (size_t)n * n));
  CK(dalloc(h, &L.coarse_partial, (size_t)kCoarseMaxSegments * n * kMaxRhs));
  double *X = nullptr, *Y = nullptr, *work = nullptr;
  int* err = nullptr;
  int herr = 0;
  cudaError_t e = cudaMalloc(&X, (size_t)L.rows * kMaxRhs * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&Y, (size_t)L.rows * kMaxRhs * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&work, ((size_t)n * 64 + 64 * 64) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = launch_coarse_inverse(L, h->opt.lambda, h->opt.mu, L.coarse_inv, X, Y, work, err, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(X);
  cudaFree(Y);
  cudaFree(work);
  cudaFree(err);
  if (e != cudaSuccess) {
    set_error(std::string("coarse inverse: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? NNMG_OUT_OF_MEMORY : NNMG_CUDA_ERROR;
  }
  if (herr) {
    set_error("coarsest operator is not positive definite");
    return NNMG_CHOLESKY_FAIL;
  }
  return NNMG_OK;
}

int setup_level(nnmg_handle* h, const nnmg_level_desc& d, DevLevel& L, cudaStream_t s) {
  const nnmg_options& o = h->opt;
  L.dim = d.dim;
  L.k = d.degree > 0 ? d.degree : o.degree;
  L.n1 = L.k + 1;
  L.nloc = d.dim == 2 ? L.n1 * L.n1 : L.n1 * L.n1 * L.n1;
  L.ncomp = o.n_components;
  L.nmetric = o.n_components == 1 ? d.dim * (d.dim + 1) / 2 : d.dim * d.dim;
  L.nqp = (L.nloc + 3) / 4 * 4;
  L.n_vertices = d.n_vertices;
  L.n_cells = d.n_cells;
  const int nc4 = 1 << d.dim;
  for (int64_t i = 0; i < d.n_cells * nc4; ++i) {
    if (d.cells[i] < 0 || d.cells[i] >= d.n_vertices) {
      set_error("cell vertex index out of range");
      return NNMG_INVALID_ARG;
    }
  }
  const double t0 = wall_seconds();
  int rc = number_nodes(d.cells, d.n_cells, d.n_vertices, d.dim, L.k, d.dirichlet_vertex, &L.num);
  if (rc != NNMG_OK) return rc;
  L.h_cells.assign(d.cells, d.cells + d.n_cells * nc4);
  if (o.deterministic) {
    // store the cells grouped by color (in input order within a color); the
    // node numbering above stays that of the input order
    std::vector<uint8_t> color;
    const int nk = color_cells(d.cells, d.n_cells, d.n_vertices, d.dim, &color);
    if (nk < 0) {
      set_error("deterministic mode: a cell needs more than 64 colors");
      return NNMG_BAD_MESH;
    }
    L.color_start.assign((size_t)nk + 1, 0);
    for (auto k : color) L.color_start[(size_t)k + 1]++;
    for (int k = 0; k < nk; ++k) L.color_start[(size_t)k + 1] += L.color_start[(size_t)k];
    std::vector<int64_t> fill(L.color_start.begin(), L.color_start.end() - 1);
    std::vector<int32_t> new_of((size_t)d.n_cells);
    for (int64_t c = 0; c < d.n_cells; ++c) new_of[(size_t)c] = (int32_t)fill[color[(size_t)c]]++;
    std::vector<int32_t> cn(L.num.cell_nodes.size());
    for (int64_t c = 0; c < d.n_cells; ++c) {
      const int64_t n = new_of[(size_t)c];
      std::copy(d.cells + c * nc4, d.cells + (c + 1) * nc4, L.h_cells.begin() + n * nc4);
      std::copy(L.num.cell_nodes.begin() + c * L.nloc, L.num.cell_nodes.begin() + (c + 1) * L.nloc,
                cn.begin() + n * L.nloc);
    }
    L.num.cell_nodes.swap(cn);
    for (auto& oc : L.num.owner_cell) oc = new_of[(size_t)oc];
  }
  const double t1 = wall_seconds();
  h->setup_s[0] += t1 - t0;
  L.n_nodes = L.num.n_nodes;
  L.rows = L.n_nodes * L.ncomp;
  L.n_free_nodes = 0;
  for (auto c : L.num.constrained) L.n_free_nodes += c ? 0 : 1;
  L.h_vertices.assign(d.vertices, d.vertices + d.n_vertices * d.dim);
  CK(dalloc(h, &L.vertices, (size_t)d.n_vertices * d.dim));
  CK(dalloc(h, &L.cells, (size_t)d.n_cells * nc4));
  CK(cudaMemcpy(L.vertices, d.vertices, (size_t)d.n_vertices * d.dim * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(L.cells, L.h_cells.data(), (size_t)d.n_cells * nc4 * sizeof(int32_t), cudaMemcpyHostToDevice));
  std::vector<int32_t> masked(L.num.cell_nodes);
  for (auto& v : masked)
    if (L.num.constrained[v]) v = -1;
  CK(dalloc(h, &L.cell_nodes, masked.size()));
  CK(cudaMemcpy(L.cell_nodes, masked.data(), masked.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(dalloc(h, &L.owner_cell, (size_t)L.n_nodes));
  CK(dalloc(h, &L.owner_local, (size_t)L.n_nodes));
  CK(cudaMemcpy(L.owner_cell, L.num.owner_cell.data(), L.n_nodes * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(L.owner_local, L.num.owner_local.data(), L.n_nodes * sizeof(int32_t), cudaMemcpyHostToDevice));
  {
    // cells holding each free node, and the zeroed counts of the fused
    // operator + Chebyshev step
    std::vector<int32_t> val((size_t)L.n_nodes, 0);
    for (auto v : masked)
      if (v >= 0) val[(size_t)v]++;
    CK(dalloc(h, &L.valence, (size_t)L.n_nodes));
    CK(dalloc(h, &L.node_count, (size_t)L.n_nodes));
    CK(cudaMemcpy(L.valence, val.data(), L.n_nodes * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemset(L.node_count, 0, L.n_nodes * sizeof(int32_t)));
  }
  std::vector<uint8_t> rf((size_t)L.rows);
  for (int64_t r = 0; r < L.rows; ++r) rf[r] = L.num.constrained[r / L.ncomp] ? 0 : 1;
  CK(dalloc(h, &L.row_free, (size_t)L.rows));
  CK(cudaMemcpy(L.row_free, rf.data(), L.rows, cudaMemcpyHostToDevice));
  // geometry
  const size_t nm = (size_t)L.n_cells * L.nmetric * L.nqp;
  CK(dalloc(h, &L.metric64, nm));
  CK(dalloc(h, &L.metric32, nm));
  CK(cudaMemsetAsync(L.metric64, 0, nm * sizeof(double), s));     // the row padding stays zero
  CK(cudaMemsetAsync(L.metric32, 0, nm * sizeof(float), s));
  int* derr;
  CK(cudaMalloc(&derr, sizeof(int)));
  CK(cudaMemsetAsync(derr, 0, sizeof(int), s));
  CK(launch_metric(L, derr, s));
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  cudaFree(derr);
  if (herr) {
    set_error("non-positive Jacobian determinant at a quadrature point");
    return NNMG_BAD_MESH;
  }
  CK(dalloc(h, &L.points, (size_t)L.n_nodes * d.dim));
  CK(launch_support_points(L, s));
  CK(dalloc(h, &L.diag64, (size_t)L.rows));
  CK(dalloc(h, &L.dinv64, (size_t)L.rows));
  CK(dalloc(h, &L.dinv32, (size_t)L.rows));
  CK(cudaMemsetAsync(L.diag64, 0, L.rows * sizeof(double), s));
  CK(launch_diag(L, o.lambda, o.mu, s));
  CK(launch_finalize_diag(L.diag64, L.row_free, L.dinv64, L.dinv32, L.rows, s));
  CK(cudaStreamSynchronize(s));
  h->setup_s[1] += wall_seconds() - t1;
  return NNMG_OK;
}

// Locate the free fine nodes of level `fi` in level fi-1 and build the sorted
// point lists (fine side) and the restriction gather lists (coarse side).
int setup_transfer(nnmg_handle* h, int fi, cudaStream_t s) {
  DevLevel& F = h->lv[fi];
  DevLevel& C = h->lv[fi - 1];
  const int dim = F.dim;
  std::vector<int32_t> pts;
  for (int64_t i = 0; i < F.n_nodes; ++i)
    if (!F.num.constrained[i]) pts.push_back((int32_t)i);
  const int64_t np = (int64_t)pts.size();
  F.n_pts = np;
  BucketGrid g;
  std::vector<double> aabb;
  build_buckets(C.h_vertices.data(), C.h_cells.data(), C.n_cells, dim, &g, &aabb);
  int32_t *dstart, *dcells, *dpts, *dcell;
  double *daabb, *dxi;
  CK(cudaMalloc(&dstart, g.start.size() * sizeof(int32_t)));
  CK(cudaMalloc(&dcells, std::max<size_t>(g.cells.size(), 1) * sizeof(int32_t)));
  CK(cudaMalloc(&daabb, aabb.size() * sizeof(double)));
  CK(cudaMalloc(&dpts, std::max<int64_t>(np, 1) * sizeof(int32_t)));
  CK(cudaMalloc(&dcell, std::max<int64_t>(np, 1) * sizeof(int32_t)));
  CK(cudaMalloc(&dxi, std::max<int64_t>(np, 1) * dim * sizeof(double)));
  CK(cudaMemcpy(dstart, g.start.data(), g.start.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  if (!g.cells.empty())
    CK(cudaMemcpy(dcells, g.cells.data(), g.cells.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(daabb, aabb.data(), aabb.size() * sizeof(double), cudaMemcpyHostToDevice));
  if (np) CK(cudaMemcpy(dpts, pts.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(launch_locate(C, F.points, dpts, np, dstart, dcells, daabb, g.geo, dcell, dxi, s));
  F.h_loc_cell.assign((size_t)np, -1);
  F.h_loc_xi.assign((size_t)np * dim, 0.0);
  if (np) {
    CK(cudaMemcpyAsync(F.h_loc_cell.data(), dcell, np * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(F.h_loc_xi.data(), dxi, np * dim * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  cudaFree(dstart);
  cudaFree(dcells);
  cudaFree(daabb);
  cudaFree(dpts);
  cudaFree(dcell);
  cudaFree(dxi);
  for (int64_t p = 0; p < np; ++p) {
    if (F.h_loc_cell[p] < 0) {
      set_error("fine support point not located in the coarser mesh");
      return NNMG_POINT_NOT_FOUND;
    }
  }
  // counting sort by coarse cell (stable: ascending fine node within a cell)
  std::vector<int32_t> start((size_t)C.n_cells + 1, 0);
  for (int64_t p = 0; p < np; ++p) start[F.h_loc_cell[p] + 1]++;
  for (int64_t c = 0; c < C.n_cells; ++c) start[c + 1] += start[c];
  std::vector<int32_t> fill(start.begin(), start.end() - 1);
  std::vector<int32_t> snode((size_t)np), scell((size_t)np);
  std::vector<double> sxi((size_t)np * dim);
  std::vector<float> sxi32((size_t)np * dim);
  for (int64_t p = 0; p < np; ++p) {
    const int32_t q = fill[F.h_loc_cell[p]]++;
    snode[q] = pts[p];
    scell[q] = F.h_loc_cell[p];
    for (int d = 0; d < dim; ++d) {
      sxi[(size_t)q * dim + d] = F.h_loc_xi[(size_t)p * dim + d];
      sxi32[(size_t)q * dim + d] = (float)F.h_loc_xi[(size_t)p * dim + d];
    }
  }
  CK(dalloc(h, &F.pt_node, (size_t)np));
  CK(dalloc(h, &F.pt_cell, (size_t)np));
  CK(dalloc(h, &F.pt_xi64, (size_t)np * dim));
  CK(dalloc(h, &F.pt_xi32, (size_t)np * dim));
  CK(dalloc(h, &F.cell_pt_start, start.size()));
  if (np) {
    CK(cudaMemcpy(F.pt_node, snode.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(F.pt_cell, scell.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(F.pt_xi64, sxi.data(), np * dim * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(F.pt_xi32, sxi32.data(), np * dim * sizeof(float), cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(F.cell_pt_start, start.data(), start.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  return NNMG_OK;
}

int setup_gather(nnmg_handle* h, DevLevel& C) {
  std::vector<int32_t> start((size_t)C.n_nodes + 1, 0);
  const auto& cn = C.num.cell_nodes;
  for (size_t i = 0; i < cn.size(); ++i)
    if (!C.num.constrained[cn[i]]) start[cn[i] + 1]++;
  for (int64_t n = 0; n < C.n_nodes; ++n) start[n + 1] += start[n];
  std::vector<int32_t> fill(start.begin(), start.end() - 1), pos((size_t)start.back());
  for (size_t i = 0; i < cn.size(); ++i)
    if (!C.num.constrained[cn[i]]) pos[fill[cn[i]]++] = (int32_t)i;
  CK(dalloc(h, &C.gather_start, start.size()));
  CK(dalloc(h, &C.gather_pos, std::max<size_t>(pos.size(), 1)));
  CK(cudaMemcpy(C.gather_start, start.data(), start.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  if (!pos.empty())
    CK(cudaMemcpy(C.gather_pos, pos.data(), pos.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  return NNMG_OK;
}

int check_vec_args(nnmg_handle* h, int level, int precision, int nrhs, bool allow_dw = false) {
  if (!h) {
    set_error("null handle");
    return NNMG_INVALID_ARG;
  }
  if (level < 0 || level >= (int)h->lv.size()) {
    set_error("level out of range");
    return NNMG_INVALID_ARG;
  }
  if (precision != NNMG_F32 && precision != NNMG_F64 && !(allow_dw && precision == NNMG_F64_DW)) {
    set_error("precision must be NNMG_F32 or NNMG_F64 (or NNMG_F64_DW for the operator)");
    return NNMG_INVALID_ARG;
  }
  if (nrhs < 1 || nrhs > h->opt.max_nrhs) {
    set_error("nrhs must be in 1..max_nrhs");
    return NNMG_INVALID_ARG;
  }
  return NNMG_OK;
}

void destroy_impl(nnmg_handle* h) {
  if (h->batch_ev) cudaEventDestroy(h->batch_ev);
  for (auto& kv : h->loops)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_sc) cudaFreeHost(h->h_sc);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
}

}  // namespace

namespace nnmg {
// Level data of a handle for entry points defined in other translation units
// (nullptr for a bad handle or level).
const DevLevel* handle_level(const nnmg_handle* h, int level) {
  if (!h || level < 0 || level >= (int)h->lv.size()) return nullptr;
  return &h->lv[level];
}
int handle_max_nrhs(const nnmg_handle* h) { return h ? h->opt.max_nrhs : 0; }
int handle_device(const nnmg_handle* h, void** noalloc_scratch) {
  *noalloc_scratch = h ? h->noalloc_scratch : nullptr;
  return h ? h->device : -1;
}
int noalloc_scratch_lookup(void** out);
}  // namespace nnmg

namespace {
// Sizes that decide the device memory of a hierarchy, from a level's mesh and
// host numbering alone: used by nnmg_estimate_bytes before anything is
// allocated, and by nnmg_solve_bytes.
struct LevelPlan {
  int dim = 0, k = 0, ncomp = 1, nloc = 0, nmetric = 0;
  int64_t n_vertices = 0, n_cells = 0, n_nodes = 0, rows = 0, n_free_nodes = 0;
  int64_t gather_entries = 0;   // cell-local slots holding a free node
};

LevelPlan level_plan(int dim, int k, int ncomp, int64_t nv, int64_t nc, const HostNumbering& num) {
  LevelPlan p;
  p.dim = dim;
  p.k = k;
  p.ncomp = ncomp;
  p.nloc = dim == 2 ? (k + 1) * (k + 1) : (k + 1) * (k + 1) * (k + 1);
  p.nmetric = ncomp == 1 ? dim * (dim + 1) / 2 : dim * dim;
  p.n_vertices = nv;
  p.n_cells = nc;
  p.n_nodes = num.n_nodes;
  p.rows = num.n_nodes * ncomp;
  for (auto c : num.constrained) p.n_free_nodes += c ? 0 : 1;
  for (auto n : num.cell_nodes) p.gather_entries += num.constrained[n] ? 0 : 1;
  return p;
}

// One dalloc of `count` elements of T (at least one, as dalloc does).
template <typename T>
size_t bytes_of(int64_t count) {
  return (size_t)std::max<int64_t>(count, 1) * sizeof(T);
}

// The device bytes nnmg_setup_hierarchy allocates (what nnmg_hierarchy_bytes
// reports right after setup), allocation by allocation: setup_level,
// setup_transfer, setup_gather and setup_coarse.
size_t planned_hierarchy_bytes(const std::vector<LevelPlan>& P) {
  size_t b = 0;
  const int n = (int)P.size();
  for (int l = 0; l < n; ++l) {
    const LevelPlan& L = P[l];
    const int64_t nm = L.n_cells * L.nmetric * ((L.nloc + 3) / 4 * 4);
    b += bytes_of<double>(L.n_vertices * L.dim) + bytes_of<int32_t>(L.n_cells << L.dim) +
         bytes_of<int32_t>(L.n_cells * L.nloc) + 4 * bytes_of<int32_t>(L.n_nodes) +
         bytes_of<uint8_t>(L.rows) + bytes_of<double>(nm) + bytes_of<float>(nm) +
         bytes_of<double>(L.n_nodes * L.dim) + 2 * bytes_of<double>(L.rows) + bytes_of<float>(L.rows);
    if (l >= 1) {
      const int64_t np = L.n_free_nodes;
      b += 2 * bytes_of<int32_t>(np) + bytes_of<double>(np * L.dim) + bytes_of<float>(np * L.dim) +
           bytes_of<int32_t>(P[l - 1].n_cells + 1);
    }
    if (l + 1 < n) b += bytes_of<int32_t>(L.n_nodes + 1) + bytes_of<int32_t>(L.gather_entries);
  }
  const int64_t nfr = P[0].n_free_nodes * P[0].ncomp;
  b += bytes_of<int32_t>(nfr);
  if (nfr > 0)
    b += bytes_of<double>(nfr * nfr) + bytes_of<double>((int64_t)kCoarseMaxSegments * nfr * kMaxRhs);
  return b;
}

// Device bytes the work buffers of solves with nrhs columns add (V-cycle
// vectors and cell buffers in both precisions, PCG vectors).
size_t planned_solve_bytes(const std::vector<LevelPlan>& P, int nrhs) {
  size_t b = 0;
  for (size_t l = 0; l < P.size(); ++l) {
    const LevelPlan& L = P[l];
    size_t per = (size_t)L.rows * nrhs * (l ? 4 : 2);
    if (l) per += (size_t)P[l - 1].n_cells * P[l - 1].nloc * L.ncomp * nrhs;
    b += per * (sizeof(float) + sizeof(double));
  }
  b += (size_t)P.back().rows * nrhs * (5 * sizeof(double) + sizeof(float));
  return b;
}
}  // namespace

// ====================================================================== C ABI
extern "C" {

void nnmg_default_options(nnmg_options* o) {
  if (!o) return;
  o->degree = 1;
  o->n_components = 1;
  o->lambda = 1.0;
  o->mu = 1.0;
  o->cheb_degree = 3;
  o->smoothing_range = 20.0;
  o->lanczos_steps = 12;
  o->eig_safety = 1.2;
  o->max_nrhs = 16;
  o->deterministic = 0;
}

const char* nnmg_last_error(void) { return get_error(); }

int nnmg_setup_hierarchy(const nnmg_level_desc* levels, int n_levels, const nnmg_options* opt,
                         void* stream, nnmg_handle** out) {
  set_error("");
  if (!out || !levels || !opt || n_levels < 1) {
    set_error("null argument or n_levels < 1");
    return NNMG_INVALID_ARG;
  }
  *out = nullptr;
  if (opt->degree < 1 || opt->degree > kMaxDegree || (opt->n_components != 1 && opt->n_components != 3) ||
      opt->cheb_degree < 1 || opt->lanczos_steps < 1 || opt->max_nrhs < 1 || opt->max_nrhs > kMaxRhs ||
      !(opt->smoothing_range > 1.0) || !(opt->eig_safety > 0.0) ||
      (opt->deterministic != 0 && opt->deterministic != 1)) {
    set_error("invalid options");
    return NNMG_INVALID_ARG;
  }
  for (int l = 0; l < n_levels; ++l) {
    const nnmg_level_desc& d = levels[l];
    if ((d.dim != 2 && d.dim != 3) || d.dim != levels[0].dim || d.n_cells < 1 || d.n_vertices < 1 ||
        !d.vertices || !d.cells || (opt->n_components == 3 && d.dim != 3) || d.degree < 0 ||
        d.degree > kMaxDegree) {
      set_error("invalid level description");
      return NNMG_INVALID_ARG;
    }
  }
  nnmg_handle* h = nullptr;
  try {
    h = new nnmg_handle();
    h->opt = *opt;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("cannot create capture stream");
      destroy_impl(h);
      return NNMG_CUDA_ERROR;
    }
    h->lv.resize(n_levels);
    int rc = NNMG_OK;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
      set_error("cudaGetDevice failed");
      rc = NNMG_CUDA_ERROR;
    }
    if (rc == NNMG_OK) rc = noalloc_scratch_lookup(&h->noalloc_scratch);
    for (int l = 0; l < n_levels && rc == NNMG_OK; ++l) rc = setup_level(h, levels[l], h->lv[l], s);
    double t = wall_seconds();
    for (int l = 1; l < n_levels && rc == NNMG_OK; ++l) rc = setup_transfer(h, l, s);
    h->setup_s[2] = wall_seconds() - t;
    t += h->setup_s[2];
    for (int l = 0; l + 1 < n_levels && rc == NNMG_OK; ++l) rc = setup_gather(h, h->lv[l]);
    h->setup_s[3] = wall_seconds() - t;
    t += h->setup_s[3];
    for (int l = 1; l < n_levels && rc == NNMG_OK; ++l) {
      rc = lanczos(h, h->lv[l], s);
      DevLevel& L = h->lv[l];
      L.cheb_b = h->opt.eig_safety * L.lam_max;
      L.cheb_a = L.cheb_b / h->opt.smoothing_range;
    }
    h->setup_s[4] = wall_seconds() - t;
    t += h->setup_s[4];
    if (rc == NNMG_OK) rc = setup_coarse(h, h->lv[0], s);
    if (rc == NNMG_OK && cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("setup: stream synchronize failed");
      rc = NNMG_CUDA_ERROR;
    }
    h->setup_s[5] = wall_seconds() - t;
    if (rc != NNMG_OK) {
      std::string msg = get_error();
      destroy_impl(h);
      set_error(msg);
      return rc;
    }
    *out = h;
    return NNMG_OK;
  } catch (const std::bad_alloc&) {
    if (h) destroy_impl(h);
    set_error("host allocation failed");
    return NNMG_OUT_OF_MEMORY;
  }
}

int nnmg_destroy(nnmg_handle* h) {
  if (h) destroy_impl(h);
  return NNMG_OK;
}

int nnmg_n_levels(const nnmg_handle* h) { return h ? (int)h->lv.size() : 0; }

int nnmg_level_info(const nnmg_handle* h, int level, int64_t* n_nodes, int64_t* n_free,
                    int64_t* n_cells) {
  if (!h || level < 0 || level >= (int)h->lv.size()) {
    set_error("bad handle or level");
    return NNMG_INVALID_ARG;
  }
  const DevLevel& L = h->lv[level];
  if (n_nodes) *n_nodes = L.n_nodes;
  if (n_free) *n_free = L.n_free_nodes;
  if (n_cells) *n_cells = L.n_cells;
  return NNMG_OK;
}

size_t nnmg_hierarchy_bytes(const nnmg_handle* h) { return h ? h->bytes : 0; }

int nnmg_estimate_bytes(const nnmg_level_desc* levels, int n_levels, const nnmg_options* opt,
                        int nrhs, size_t* hierarchy_bytes, size_t* solve_bytes) {
  set_error("");
  if (!levels || !opt || n_levels < 1 || nrhs < 1 || nrhs > kMaxRhs || opt->degree < 1 ||
      opt->degree > kMaxDegree || (opt->n_components != 1 && opt->n_components != 3)) {
    set_error("nnmg_estimate_bytes: bad argument");
    return NNMG_INVALID_ARG;
  }
  try {
    std::vector<HostNumbering> num((size_t)n_levels);
    std::vector<LevelPlan> plan((size_t)n_levels);
    for (int l = 0; l < n_levels; ++l) {
      const nnmg_level_desc& d = levels[l];
      if ((d.dim != 2 && d.dim != 3) || d.n_cells < 1 || d.n_vertices < 1 || !d.cells ||
          d.degree < 0 || d.degree > kMaxDegree) {
        set_error("nnmg_estimate_bytes: invalid level description");
        return NNMG_INVALID_ARG;
      }
      for (int64_t i = 0; i < d.n_cells * (1 << d.dim); ++i)
        if (d.cells[i] < 0 || d.cells[i] >= d.n_vertices) {
          set_error("nnmg_estimate_bytes: cell vertex index out of range");
          return NNMG_INVALID_ARG;
        }
      const int k = d.degree > 0 ? d.degree : opt->degree;
      int rc = number_nodes(d.cells, d.n_cells, d.n_vertices, d.dim, k, d.dirichlet_vertex, &num[l]);
      if (rc != NNMG_OK) return rc;
      plan[l] = level_plan(d.dim, k, opt->n_components, d.n_vertices, d.n_cells, num[l]);
    }
    if (hierarchy_bytes) *hierarchy_bytes = planned_hierarchy_bytes(plan);
    if (solve_bytes) *solve_bytes = planned_solve_bytes(plan, nrhs);
    return NNMG_OK;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return NNMG_OUT_OF_MEMORY;
  }
}

size_t nnmg_solve_bytes(const nnmg_handle* h, int nrhs) {
  if (!h) return 0;
  std::vector<LevelPlan> plan(h->lv.size());
  for (size_t l = 0; l < h->lv.size(); ++l) {
    const DevLevel& L = h->lv[l];
    plan[l] = level_plan(L.dim, L.k, L.ncomp, L.n_vertices, L.n_cells, L.num);
  }
  return planned_solve_bytes(plan, nrhs);
}

int nnmg_support_points(const nnmg_handle* h, int level, double* pts) {
  if (!h || !pts || level < 0 || level >= (int)h->lv.size()) {
    set_error("bad argument");
    return NNMG_INVALID_ARG;
  }
  const DevLevel& L = h->lv[level];
  NNMG_CUDA(cudaMemcpy(pts, L.points, (size_t)L.n_nodes * L.dim * sizeof(double), cudaMemcpyDeviceToHost));
  return NNMG_OK;
}

int nnmg_constrained_nodes(const nnmg_handle* h, int level, uint8_t* flags) {
  if (!h || !flags || level < 0 || level >= (int)h->lv.size()) {
    set_error("bad argument");
    return NNMG_INVALID_ARG;
  }
  const DevLevel& L = h->lv[level];
  std::memcpy(flags, L.num.constrained.data(), (size_t)L.n_nodes);
  return NNMG_OK;
}

int nnmg_cell_nodes(const nnmg_handle* h, int level, int32_t* cn) {
  if (!h || !cn || level < 0 || level >= (int)h->lv.size()) {
    set_error("bad argument");
    return NNMG_INVALID_ARG;
  }
  const DevLevel& L = h->lv[level];
  std::memcpy(cn, L.num.cell_nodes.data(), L.num.cell_nodes.size() * sizeof(int32_t));
  return NNMG_OK;
}

int nnmg_color_cells(const int32_t* cells, int64_t n_cells, int64_t n_vertices, int dim,
                     uint8_t* color, int* n_colors) {
  if (!cells || !color || !n_colors || n_cells < 0 || n_vertices < 1 || (dim != 2 && dim != 3)) {
    set_error("nnmg_color_cells: bad argument");
    return NNMG_INVALID_ARG;
  }
  for (int64_t i = 0; i < n_cells * (1 << dim); ++i)
    if (cells[i] < 0 || cells[i] >= n_vertices) {
      set_error("nnmg_color_cells: vertex index out of range");
      return NNMG_INVALID_ARG;
    }
  std::vector<uint8_t> c;
  const int nk = color_cells(cells, n_cells, n_vertices, dim, &c);
  if (nk < 0) {
    set_error("nnmg_color_cells: more than 64 colors needed");
    return NNMG_BAD_MESH;
  }
  std::copy(c.begin(), c.end(), color);
  *n_colors = nk;
  return NNMG_OK;
}

int nnmg_level_colors(const nnmg_handle* h, int level, int64_t* color_start, int* n_colors) {
  if (!h || !n_colors || level < 0 || level >= (int)h->lv.size()) {
    set_error("bad argument");
    return NNMG_INVALID_ARG;
  }
  const DevLevel& L = h->lv[level];
  *n_colors = L.color_start.empty() ? 0 : (int)L.color_start.size() - 1;
  if (color_start) std::copy(L.color_start.begin(), L.color_start.end(), color_start);
  return NNMG_OK;
}

int nnmg_quadrature_points(const nnmg_handle* h, int level, double* xq) {
  if (!h || !xq || level < 0 || level >= (int)h->lv.size()) {
    set_error("bad argument");
    return NNMG_INVALID_ARG;
  }
  const DevLevel& L = h->lv[level];
  const size_t n = (size_t)L.n_cells * L.nloc * L.dim;
  double* d;
  NNMG_CUDA(cudaMalloc(&d, n * sizeof(double)));
  cudaError_t e = launch_quad_points(L, d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(xq, d, n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d);
  NNMG_CUDA(e);
  return NNMG_OK;
}

int nnmg_transfer_points(const nnmg_handle* h, int fine_level, int32_t* cell, double* xi) {
  if (!h || fine_level < 1 || fine_level >= (int)h->lv.size()) {
    set_error("bad argument");
    return NNMG_INVALID_ARG;
  }
  const DevLevel& F = h->lv[fine_level];
  if (cell) std::memcpy(cell, F.h_loc_cell.data(), F.h_loc_cell.size() * sizeof(int32_t));
  if (xi) std::memcpy(xi, F.h_loc_xi.data(), F.h_loc_xi.size() * sizeof(double));
  return NNMG_OK;
}

int nnmg_pcg_device_loop(const nnmg_handle* h, int mode, int nrhs, int* state) {
  if (!h || !state) {
    set_error("nnmg_pcg_device_loop: null handle or pointer");
    return NNMG_INVALID_ARG;
  }
  auto it = h->loops.find(std::make_tuple(mode, nrhs));
  *state = it == h->loops.end() ? 0 : (it->second ? 1 : -1);
  return NNMG_OK;
}

int nnmg_setup_seconds(const nnmg_handle* h, double* seconds) {
  if (!h || !seconds) {
    set_error("nnmg_setup_seconds: null handle or pointer");
    return NNMG_INVALID_ARG;
  }
  for (int i = 0; i < NNMG_SETUP_PHASES; ++i) seconds[i] = h->setup_s[i];
  return NNMG_OK;
}

int nnmg_operator_choice(const nnmg_handle* h, int level, int precision, int nrhs, int* choice) {
  if (!h || !choice || level < 0 || level >= (int)h->lv.size() || nrhs < 1 ||
      nrhs > kMaxRhs || (precision != NNMG_F32 && precision != NNMG_F64 && precision != NNMG_F64_DW)) {
    set_error("nnmg_operator_choice: bad handle, pointer, level, precision or nrhs");
    return NNMG_INVALID_ARG;
  }
  auto it = h->op_units.find(std::make_tuple(level, precision, nrhs));
  *choice = it == h->op_units.end() ? 0 : it->second;
  return NNMG_OK;
}

int nnmg_eigen_estimates(const nnmg_handle* h, double* lam) {
  if (!h || !lam) {
    set_error("bad argument");
    return NNMG_INVALID_ARG;
  }
  for (size_t l = 0; l < h->lv.size(); ++l) lam[l] = l ? h->lv[l].lam_max : 0.0;
  return NNMG_OK;
}

int nnmg_load_vector(nnmg_handle* h, int level, const double* f, int f_per_qp, double* b,
                     int nrhs, int col, void* stream) {
  int rc = check_vec_args(h, level, NNMG_F64, nrhs);
  if (rc) return rc;
  if (!f || !b || col < 0 || col >= nrhs) {
    set_error("bad argument");
    return NNMG_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const DevLevel& L = h->lv[level];
  const size_t nf = f_per_qp ? (size_t)L.n_cells * L.nloc * L.ncomp : (size_t)L.ncomp;
  double* df;
  NNMG_CUDA(cudaMalloc(&df, nf * sizeof(double)));
  cudaError_t e = cudaMemcpyAsync(df, f, nf * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemset2DAsync(b + col, (size_t)nrhs * sizeof(double), 0, sizeof(double), (size_t)L.rows, s);
  if (e == cudaSuccess) e = launch_load_vector(L, df, f_per_qp, b, nrhs, col, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(df);
  NNMG_CUDA(e);
  return NNMG_OK;
}

int nnmg_apply_operator(nnmg_handle* h, int level, int precision, const void* x, void* y,
                        int nrhs, void* stream) {
  int rc = check_vec_args(h, level, precision, nrhs, true);
  if (rc) return rc;
  if (!x || !y || x == y) {
    set_error("x and y must be distinct device vectors");
    return NNMG_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const DevLevel& L = h->lv[level];
  const size_t ts = precision == NNMG_F64 ? sizeof(double) : sizeof(float);
  if (precision == NNMG_F64_DW) {
    if ((rc = ensure_dw(h, level))) return rc;
    const int ou = op_units_dw(h, level, nrhs, s);
    NNMG_CUDA(cudaMemsetAsync(y, 0, (size_t)L.rows * nrhs * sizeof(double), s));
    NNMG_CUDA(launch_operator_dw(L, (const double*)x, (double*)y, nrhs, h->opt.lambda, h->opt.mu, s, ou));
    return NNMG_OK;
  }
  const int ou = precision == NNMG_F64 ? op_units<double>(h, level, nrhs, s)
                                        : op_units<float>(h, level, nrhs, s);
  NNMG_CUDA(cudaMemsetAsync(y, 0, (size_t)L.rows * nrhs * ts, s));
  if (precision == NNMG_F64)
    NNMG_CUDA(launch_operator<double>(L, (const double*)x, (double*)y, nrhs, h->opt.lambda, h->opt.mu, s, ou));
  else
    NNMG_CUDA(launch_operator<float>(L, (const float*)x, (float*)y, nrhs, h->opt.lambda, h->opt.mu, s, ou));
  return NNMG_OK;
}

int nnmg_prolongate(nnmg_handle* h, int fine_level, int precision, const void* coarse, void* fine,
                    int nrhs, void* stream) {
  int rc = check_vec_args(h, fine_level, precision, nrhs);
  if (rc) return rc;
  if (fine_level < 1 || !coarse || !fine) {
    set_error("fine_level must be >= 1 and vectors non-null");
    return NNMG_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const DevLevel& F = h->lv[fine_level];
  const DevLevel& C = h->lv[fine_level - 1];
  const size_t ts = precision == NNMG_F64 ? sizeof(double) : sizeof(float);
  NNMG_CUDA(cudaMemsetAsync(fine, 0, (size_t)F.rows * nrhs * ts, s));
  if (precision == NNMG_F64)
    NNMG_CUDA(launch_prolongate_add<double>(F, C, (const double*)coarse, (double*)fine, nrhs, s));
  else
    NNMG_CUDA(launch_prolongate_add<float>(F, C, (const float*)coarse, (float*)fine, nrhs, s));
  return NNMG_OK;
}

int nnmg_restrict(nnmg_handle* h, int fine_level, int precision, const void* fine, void* coarse,
                  int nrhs, void* stream) {
  int rc = check_vec_args(h, fine_level, precision, nrhs);
  if (rc) return rc;
  if (fine_level < 1 || !coarse || !fine) {
    set_error("fine_level must be >= 1 and vectors non-null");
    return NNMG_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const DevLevel& F = h->lv[fine_level];
  const DevLevel& C = h->lv[fine_level - 1];
  if (precision == NNMG_F64) {
    if ((rc = ensure_work<double>(h))) return rc;
    NNMG_CUDA(launch_restrict<double>(F, C, (const double*)fine, (double*)coarse,
                                      h->w64.scratch[fine_level], nrhs, s));
  } else {
    if ((rc = ensure_work<float>(h))) return rc;
    NNMG_CUDA(launch_restrict<float>(F, C, (const float*)fine, (float*)coarse,
                                     h->w32.scratch[fine_level], nrhs, s));
  }
  return NNMG_OK;
}

int nnmg_vcycle(nnmg_handle* h, int precision, const void* r, void* z, int nrhs, void* stream) {
  int rc = check_vec_args(h, 0, precision, nrhs);
  if (rc) return rc;
  if (!r || !z) {
    set_error("null vector");
    return NNMG_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int top = (int)h->lv.size() - 1;
  const size_t n = (size_t)h->lv[top].rows * nrhs;
  if (precision == NNMG_F64) {
    if ((rc = ensure_work<double>(h))) return rc;
    NNMG_CUDA(cudaMemcpyAsync(h->w64.f[top], r, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (top == 0) NNMG_CUDA(cudaMemsetAsync(h->w64.x[0], 0, n * sizeof(double), s));
    rc = run_graph(h, {0, NNMG_F64, nrhs}, s, [&](cudaStream_t st) {
      return enqueue_vcycle<double>(h, h->w64.f[top], nrhs, st);
    });
    if (rc) return rc;
    NNMG_CUDA(cudaMemcpyAsync(z, h->w64.x[top], n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    if ((rc = ensure_work<float>(h))) return rc;
    NNMG_CUDA(cudaMemcpyAsync(h->w32.f[top], r, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (top == 0) NNMG_CUDA(cudaMemsetAsync(h->w32.x[0], 0, n * sizeof(float), s));
    rc = run_graph(h, {0, NNMG_F32, nrhs}, s, [&](cudaStream_t st) {
      return enqueue_vcycle<float>(h, h->w32.f[top], nrhs, st);
    });
    if (rc) return rc;
    NNMG_CUDA(cudaMemcpyAsync(z, h->w32.x[top], n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  return NNMG_OK;
}

int nnmg_vcycle_profile(nnmg_handle* h, int precision, const void* r, void* z, int nrhs,
                        void* stream, double* ms, int* launches) {
  int rc = check_vec_args(h, 0, precision, nrhs);
  if (rc) return rc;
  if (!r || !z || !ms) {
    set_error("null vector or output array");
    return NNMG_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  NNMG_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) {
    set_error("nnmg_vcycle_profile cannot run inside a stream capture");
    return NNMG_INVALID_ARG;
  }
  const int nl = (int)h->lv.size(), top = nl - 1;
  const size_t n = (size_t)h->lv[top].rows * nrhs;
  VcycleTimer P;
  auto run = [&](auto tag, WorkSet<decltype(tag)>& W) -> int {
    using T = decltype(tag);
    int rr = ensure_work<T>(h);
    if (rr) return rr;
    for (int l = 1; l <= top; ++l) op_units<T>(h, l, nrhs, s);   // tune outside the timed launches
    NNMG_CUDA(cudaMemcpyAsync(W.f[top], r, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    if (top == 0) NNMG_CUDA(cudaMemsetAsync(W.x[0], 0, n * sizeof(T), s));
    NNMG_CUDA(enqueue_vcycle<T>(h, W.f[top], nrhs, s, &P));
    NNMG_CUDA(cudaMemcpyAsync(z, W.x[top], n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    return NNMG_OK;
  };
  rc = precision == NNMG_F64 ? run(0.0, h->w64) : run(0.0f, h->w32);
  if (rc) return rc;
  NNMG_CUDA(cudaStreamSynchronize(s));
  std::fill(ms, ms + (size_t)nl * NNMG_PROF_COLS, 0.0);
  if (launches) std::fill(launches, launches + (size_t)nl * NNMG_PROF_COLS, 0);
  for (const auto& m : P.marks) {
    float t = 0.f;
    NNMG_CUDA(cudaEventElapsedTime(&t, m.a, m.b));
    int cols[2] = {m.col_component, m.col_kind};
    const int nc = m.col_kind == m.col_component ? 1 : 2;
    for (int c = 0; c < nc; ++c) {
      ms[(size_t)m.level * NNMG_PROF_COLS + cols[c]] += t;
      if (launches) ++launches[(size_t)m.level * NNMG_PROF_COLS + cols[c]];
    }
  }
  return NNMG_OK;
}

// ------------------------------------------------------- nested transfer
int nnmg_set_nested(nnmg_handle* h, int fine_level, const int32_t* parent_cell,
                    const uint8_t* child_index) {
  if (!h || fine_level < 1 || fine_level >= (int)h->lv.size()) {
    set_error("nnmg_set_nested: bad handle or fine_level");
    return NNMG_INVALID_ARG;
  }
  DevLevel& F = h->lv[fine_level];
  const DevLevel& C = h->lv[fine_level - 1];
  drop_graphs(h);                                                  // the V-cycle changes
  if (!parent_cell) {
    F.gc_active = false;
    return NNMG_OK;
  }
  if (!child_index) {
    set_error("nnmg_set_nested: child_index is required with parent_cell");
    return NNMG_INVALID_ARG;
  }
  const int nchild = 1 << F.dim;
  if (F.k != C.k || F.n_cells != C.n_cells * nchild) {
    set_error("nnmg_set_nested: the fine level must be the 2^d refinement of the coarse one, same degree");
    return NNMG_INVALID_ARG;
  }
  std::vector<int32_t> ch((size_t)C.n_cells * nchild, -1);
  for (int64_t f = 0; f < F.n_cells; ++f) {
    const int64_t p = parent_cell[f];
    const int b = child_index[f];
    if (p < 0 || p >= C.n_cells || b >= nchild || ch[(size_t)p * nchild + b] >= 0) {
      set_error("nnmg_set_nested: parent/child lists are not a 2^d refinement");
      return NNMG_INVALID_ARG;
    }
    ch[(size_t)p * nchild + b] = (int32_t)f;
  }
  if (!F.gc_children) CK(dalloc(h, &F.gc_children, ch.size()));
  CK(cudaMemcpy(F.gc_children, ch.data(), ch.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  F.gc_active = true;
  return NNMG_OK;
}

// ------------------------------------------------------- continuous batching
int nnmg_batch_reset(nnmg_handle* h, int mode, int nslots, double rtol, int maxit, void* stream) {
  int rc = check_vec_args(h, 0, NNMG_F64, nslots);
  if (rc) return rc;
  if ((mode != NNMG_FP64_MG && mode != NNMG_FP32_MG_FP64_CG && mode != NNMG_FP32_MG_DW_CG) ||
      !(rtol > 0.0) || maxit < 1) {
    set_error("bad mode, rtol or maxit");
    return NNMG_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (h->cooperative_ok) {
    // from now on kernel-per-step smoothing: drop graphs captured with the
    // cooperative smoother
    h->cooperative_ok = false;
    NNMG_CUDA(cudaStreamSynchronize(s));
    drop_graphs(h);
  }
  if ((rc = ensure_pcg(h))) return rc;
  if ((rc = (mode == NNMG_FP64_MG ? ensure_work<double>(h) : ensure_work<float>(h)))) return rc;
  if (mode == NNMG_FP32_MG_DW_CG && (rc = ensure_dw(h, (int)h->lv.size() - 1))) return rc;
  if (!h->batch_ev) NNMG_CUDA(cudaEventCreateWithFlags(&h->batch_ev, cudaEventDisableTiming));
  const size_t n = (size_t)h->lv.back().rows * nslots * sizeof(double);
  NNMG_CUDA(cudaMemsetAsync(h->px, 0, n, s));
  NNMG_CUDA(cudaMemsetAsync(h->pr, 0, n, s));
  NNMG_CUDA(cudaMemsetAsync(h->pr32, 0, n / 2, s));
  NNMG_CUDA(cudaMemsetAsync(h->pp, 0, n, s));
  NNMG_CUDA(cudaMemsetAsync(h->pq, 0, n, s));
  NNMG_CUDA(launch_batch_reset(h->sc, rtol, maxit, s));
  h->batch_mode = mode;
  h->batch_slots = nslots;
  h->batch_inflight = false;
  return NNMG_OK;
}

int nnmg_batch_admit(nnmg_handle* h, int slot, const double* b, int b_on_host, void* stream) {
  if (!h || h->batch_mode < 0 || slot < 0 || slot >= h->batch_slots || !b) {
    set_error("nnmg_batch_admit: no batch started, bad slot or null b");
    return NNMG_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const DevLevel& L = h->lv.back();
  const double* src = b;
  if (b_on_host) {
    NNMG_CUDA(cudaMemcpyAsync(h->pb, b, (size_t)L.rows * sizeof(double), cudaMemcpyHostToDevice, s));
    src = h->pb;
  }
  NNMG_CUDA(launch_batch_admit(src, 1, L.row_free, h->pr, h->pr32, h->px, h->pp, h->partial, h->sc,
                               L.rows, h->batch_slots, slot, 1, s));
  return NNMG_OK;
}

int nnmg_batch_admit_cols(nnmg_handle* h, int first_slot, int ncols, const double* b, int ldb,
                          int b_on_host, void* stream) {
  if (!h || h->batch_mode < 0 || !b || ncols < 1 || first_slot < 0 ||
      first_slot + ncols > h->batch_slots || ldb < ncols || (b_on_host && ldb > h->opt.max_nrhs)) {
    set_error("nnmg_batch_admit_cols: no batch started, null b, slots outside the batch, "
              "ldb < ncols or (host b) ldb > max_nrhs");
    return NNMG_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const DevLevel& L = h->lv.back();
  const double* src = b;
  if (b_on_host) {
    NNMG_CUDA(cudaMemcpyAsync(h->pb, b, (size_t)L.rows * ldb * sizeof(double),
                              cudaMemcpyHostToDevice, s));
    src = h->pb;
  }
  NNMG_CUDA(launch_batch_admit(src, ldb, L.row_free, h->pr, h->pr32, h->px, h->pp, h->partial,
                               h->sc, L.rows, h->batch_slots, first_slot, ncols, s));
  return NNMG_OK;
}

int nnmg_batch_step(nnmg_handle* h, int iterations, void* stream) {
  if (!h || h->batch_mode < 0 || iterations < 1) {
    set_error("nnmg_batch_step: no batch started or iterations < 1");
    return NNMG_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int mode = h->batch_mode, nslots = h->batch_slots;
  for (int it = 0; it < iterations; ++it) {
    int rc = run_graph(h, {1, mode, nslots}, s, [&](cudaStream_t st) {
      return enqueue_pcg_iter(h, mode, nslots, st);
    });
    if (rc) return rc;
  }
  NNMG_CUDA(cudaMemcpyAsync(h->h_sc, h->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
  NNMG_CUDA(cudaEventRecord(h->batch_ev, s));
  h->batch_inflight = true;
  return NNMG_OK;
}

int nnmg_batch_repack(nnmg_handle* h, int new_slots, const int* src, void* stream) {
  if (!h || h->batch_mode < 0 || !src || new_slots < 1 || new_slots > h->opt.max_nrhs) {
    set_error("nnmg_batch_repack: no batch started, null src or new_slots not in 1..max_nrhs");
    return NNMG_INVALID_ARG;
  }
  if (h->batch_inflight) {
    set_error("nnmg_batch_repack: a step is in flight (poll until it reports ready)");
    return NNMG_INVALID_ARG;
  }
  SlotMap m;
  bool seen[kMaxRhs] = {};
  for (int j = 0; j < kMaxRhs; ++j) m.s[j] = -1;
  for (int j = 0; j < new_slots; ++j) {
    const int q = src[j];
    if (q < -1 || q >= h->batch_slots || (q >= 0 && seen[q])) {
      set_error("nnmg_batch_repack: src entries must be distinct old slots or -1");
      return NNMG_INVALID_ARG;
    }
    if (q >= 0) seen[q] = true;
    m.s[j] = q;
  }
  cudaStream_t s = (cudaStream_t)stream;
  NNMG_CUDA(launch_batch_repack(h->px, h->pr, h->pr32, h->pp, h->pq, h->sc, h->lv.back().rows,
                                h->batch_slots, new_slots, m, s));
  h->batch_slots = new_slots;
  return NNMG_OK;
}

int nnmg_batch_poll(nnmg_handle* h, int wait, int* ready, int* active, int* iters, double* relres,
                    int* status) {
  if (!h || h->batch_mode < 0 || !ready) {
    set_error("nnmg_batch_poll: no batch started");
    return NNMG_INVALID_ARG;
  }
  *ready = 0;
  if (h->batch_inflight) {
    cudaError_t e = wait ? cudaEventSynchronize(h->batch_ev) : cudaEventQuery(h->batch_ev);
    if (e == cudaErrorNotReady) return NNMG_OK;
    NNMG_CUDA(e);
    h->batch_inflight = false;
  } else {
    return NNMG_OK;
  }
  *ready = 1;
  const PcgScalars& sc = *h->h_sc;
  for (int q = 0; q < h->batch_slots; ++q) {
    if (active) active[q] = sc.active[q];
    if (iters) iters[q] = sc.iters[q];
    if (relres) relres[q] = sc.bnorm[q] > 0 ? sc.rnorm[q] / sc.bnorm[q] : 0.0;
    if (status)
      status[q] = sc.broken[q] ? NNMG_BREAKDOWN : (sc.failed[q] ? NNMG_NOT_CONVERGED : NNMG_OK);
  }
  return NNMG_OK;
}

int nnmg_batch_retire(nnmg_handle* h, int slot, double* x, int x_on_host, void* stream) {
  if (!h || h->batch_mode < 0 || slot < 0 || slot >= h->batch_slots || !x) {
    set_error("nnmg_batch_retire: no batch started, bad slot or null x");
    return NNMG_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const DevLevel& L = h->lv.back();
  // the column is gathered on the device (a copy engine moves a column of
  // 8-byte pieces slowly), then copied contiguously
  if (x_on_host) {
    NNMG_CUDA(launch_column_gather(h->px, h->pb, L.rows, h->batch_slots, slot, s));
    NNMG_CUDA(cudaMemcpyAsync(x, h->pb, (size_t)L.rows * sizeof(double), cudaMemcpyDeviceToHost, s));
  } else {
    NNMG_CUDA(launch_column_gather(h->px, x, L.rows, h->batch_slots, slot, s));
  }
  NNMG_CUDA(cudaMemsetAsync(&h->sc->active[slot], 0, sizeof(int), s));
  return NNMG_OK;
}

}  // extern "C"

namespace {
int pcg_result(nnmg_handle* h, int nrhs, double rtol, int* iters_out, double* relres_out);

// PCG from x0 = 0 on device right-hand sides b; the solution stays in h->px.
int pcg_run(nnmg_handle* h, int mode, const double* b, int nrhs, double rtol, int maxit,
            int* iters_out, double* relres_out, cudaStream_t s) {
  int rc;
  if ((rc = ensure_pcg(h))) return rc;
  if ((rc = (mode == NNMG_FP64_MG ? ensure_work<double>(h) : ensure_work<float>(h)))) return rc;
  if (mode == NNMG_FP32_MG_DW_CG && (rc = ensure_dw(h, (int)h->lv.size() - 1))) return rc;
  const DevLevel& L = h->lv.back();
  NNMG_CUDA(launch_pcg_init(b, L.row_free, h->pr, h->pr32, h->px, h->pp, h->partial, L.rows, nrhs, s));
  NNMG_CUDA(launch_pcg_start(h->sc, h->partial, nrhs, rtol, maxit, s));
  // device-side loop once the single-iteration graph exists (NNMG_DEVICE_LOOP=0
  // keeps the host-driven loop)
  const char* dl = getenv("NNMG_DEVICE_LOOP");
  const auto lkey = std::make_tuple(mode, nrhs);
  if (!(dl && dl[0] == '0') && h->graphs.count(std::make_tuple(1, mode, nrhs))) {
    auto it = h->loops.find(lkey);
    if (it == h->loops.end()) it = h->loops.emplace(lkey, build_pcg_loop(h, mode, nrhs)).first;
    if (it->second) {
      NNMG_CUDA(cudaGraphLaunch(it->second, s));
      NNMG_CUDA(cudaMemcpyAsync(h->h_sc, h->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
      NNMG_CUDA(cudaStreamSynchronize(s));
      return pcg_result(h, nrhs, rtol, iters_out, relres_out);
    }
  }
  NNMG_CUDA(cudaMemcpyAsync(h->h_sc, h->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
  NNMG_CUDA(cudaStreamSynchronize(s));
  bool active = h->h_sc->any_active != 0;
  for (int it = 0; it < maxit && active; ++it) {
    rc = run_graph(h, {1, mode, nrhs}, s, [&](cudaStream_t st) {
      return enqueue_pcg_iter(h, mode, nrhs, st);
    });
    if (rc) return rc;
    NNMG_CUDA(cudaMemcpyAsync(h->h_sc, h->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    NNMG_CUDA(cudaStreamSynchronize(s));
    active = h->h_sc->any_active != 0;
  }
  return pcg_result(h, nrhs, rtol, iters_out, relres_out);
}

// Per-column results of the finished PCG (host copy of the scalars).
int pcg_result(nnmg_handle* h, int nrhs, double rtol, int* iters_out, double* relres_out) {
  const PcgScalars& sc = *h->h_sc;
  bool conv = true;
  for (int q = 0; q < nrhs; ++q) {
    if (iters_out) iters_out[q] = sc.iters[q];
    const double rel = sc.bnorm[q] > 0 ? sc.rnorm[q] / sc.bnorm[q] : 0.0;
    if (relres_out) relres_out[q] = rel;
    conv = conv && (rel <= rtol);
  }
  if (sc.breakdown) {
    set_error("PCG breakdown (p.Ap <= 0 or non-finite scalar)");
    return NNMG_BREAKDOWN;
  }
  if (!conv) {
    set_error("PCG did not reach rtol within maxit");
    return NNMG_NOT_CONVERGED;
  }
  return NNMG_OK;
}

int pcg_args(nnmg_handle* h, int mode, int nrhs, double rtol, int maxit) {
  int rc = check_vec_args(h, 0, NNMG_F64, nrhs);
  if (rc) return rc;
  if ((mode != NNMG_FP64_MG && mode != NNMG_FP32_MG_FP64_CG && mode != NNMG_FP32_MG_DW_CG) ||
      !(rtol > 0.0) || maxit < 1) {
    set_error("bad mode, rtol or maxit");
    return NNMG_INVALID_ARG;
  }
  return NNMG_OK;
}
}  // namespace

extern "C" {

int nnmg_pcg_solve(nnmg_handle* h, int mode, const double* b, double* x, int nrhs, double rtol,
                   int maxit, int* iters_out, double* relres_out, void* stream) {
  int rc = pcg_args(h, mode, nrhs, rtol, maxit);
  if (rc) return rc;
  if (!b || !x) {
    set_error("null vector");
    return NNMG_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  rc = pcg_run(h, mode, b, nrhs, rtol, maxit, iters_out, relres_out, s);
  if (rc != NNMG_OK && rc != NNMG_NOT_CONVERGED && rc != NNMG_BREAKDOWN) return rc;
  const size_t n = (size_t)h->lv.back().rows * nrhs * sizeof(double);
  NNMG_CUDA(cudaMemcpyAsync(x, h->px, n, cudaMemcpyDeviceToDevice, s));
  return rc;
}

int nnmg_pcg_solve_host(nnmg_handle* h, int mode, const double* b_host, double* x_host, int nrhs,
                        double rtol, int maxit, int* iters_out, double* relres_out, void* stream) {
  int rc = pcg_args(h, mode, nrhs, rtol, maxit);
  if (rc) return rc;
  if (!b_host || !x_host) {
    set_error("null host vector");
    return NNMG_INVALID_ARG;
  }
  if ((rc = ensure_pcg(h))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)h->lv.back().rows * nrhs * sizeof(double);
  NNMG_CUDA(cudaMemcpyAsync(h->pb, b_host, n, cudaMemcpyHostToDevice, s));
  rc = pcg_run(h, mode, h->pb, nrhs, rtol, maxit, iters_out, relres_out, s);
  if (rc != NNMG_OK && rc != NNMG_NOT_CONVERGED && rc != NNMG_BREAKDOWN) return rc;
  cudaError_t e = cudaMemcpyAsync(x_host, h->px, n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  NNMG_CUDA(e);
  return rc;
}

}  // extern "C"
