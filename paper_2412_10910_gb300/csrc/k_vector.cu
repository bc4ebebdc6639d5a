// Vector kernels: Chebyshev-Jacobi updates (Sec. 4 smoother), residuals,
// precision casts, deterministic dot products and the per-column scalar
// steps of PCG (Sec. 4: CG in double precision, one V-cycle as preconditioner).
//
// Layout: vectors are [rows][nrhs]; the Jacobi inverse diagonal is per row.
// Dot products are two-pass: each of kDotBlocks blocks writes per-column
// partial sums, and a single-block kernel adds them in block order, so the
// result does not depend on scheduling.
#include "nnmg_internal.h"

namespace nnmg {
namespace {

// FP32 -> FP64 widening on the integer pipes.  The conversion instruction runs
// on GB300's FP64 pipe (2 operations per clock per SM, shared with the FMAs of
// the FP64 dot products and updates), so kernels that widen every element
// re-pack the IEEE-754 fields instead: a normal float's exponent is rebiased
// (127 -> 1023) and its 23 fraction bits move to the top of the 52, which is
// exact.  Zeros keep their sign; subnormals, infinities and NaNs (not produced
// by the solver) take the conversion instruction.
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xffu;
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  if ((u & 0x7fffffffu) == 0) return __longlong_as_double((long long)sign);
  if (ex == 0 || ex == 0xffu) return (double)f;
  return __longlong_as_double(
      (long long)(sign | ((uint64_t)(ex + 896u) << 52) | ((uint64_t)(u & 0x7fffffu) << 29)));
}
__device__ __forceinline__ double widen(double d) { return d; }

inline unsigned vblocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// Vectors handled here hold fewer than 2^31 elements (checked by the
// launchers), so element and row indices use 32-bit unsigned arithmetic; the
// row of element e is e / nrhs.

template <typename T>
__global__ void cheb_init_kernel(const T* __restrict__ f, const T* __restrict__ dinv,
                                 T* __restrict__ d, T* __restrict__ x, T c, int64_t n, int nrhs) {
  pdl_trigger();
  pdl_wait();
  const unsigned un = (unsigned)n, ur = (unsigned)nrhs;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < un; e += gridDim.x * blockDim.x) {
    const T v = c * dinv[e / ur] * f[e];
    d[e] = v;
    x[e] = v;
  }
}

// r = f - t (t then reset to 0); d = cd*d + cr*Dinv r; x += d.
// All loads of an element are issued before its stores: a store placed
// between loads serialises the memory round trips (measured 8x slower).
template <typename T>
__global__ void cheb_step_kernel(const T* __restrict__ f, T* __restrict__ t,
                                 const T* __restrict__ dinv, T* __restrict__ d, T* __restrict__ x,
                                 T cd, T cr, int64_t n, int nrhs) {
  pdl_trigger();
  pdl_wait();
  const unsigned un = (unsigned)n, ur = (unsigned)nrhs;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < un; e += gridDim.x * blockDim.x) {
    const T fe = f[e], te = t[e], de = d[e], xe = x[e], di = dinv[e / ur];
    const T dn = cd * de + cr * di * (fe - te);
    d[e] = dn;
    x[e] = xe + dn;
    t[e] = T(0);
  }
}

template <typename T>
__global__ void residual_kernel(const T* __restrict__ f, T* __restrict__ t, T* __restrict__ r,
                                int64_t n) {
  pdl_trigger();
  pdl_wait();
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < (unsigned)n;
       e += gridDim.x * blockDim.x) {
    r[e] = f[e] - t[e];
    t[e] = T(0);
  }
}

template <typename TI, typename TO>
__global__ void cast_kernel(const TI* __restrict__ a, TO* __restrict__ b, int64_t n) {
  pdl_trigger();
  pdl_wait();
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < (unsigned)n;
       e += gridDim.x * blockDim.x)
    b[e] = (TO)a[e];
}

// Dot-product layout: a block has kDotThreads - (kDotThreads % nrhs) active
// threads and the grid stride is a multiple of nrhs, so thread t always visits
// column t % nrhs.  Each block writes one partial sum per column to
// partial[block][column]; partials are added in block order by
// sum_partials_warp.  Both steps have a fixed order: results are reproducible.
__device__ __forceinline__ unsigned dot_threads(int nrhs) {
  return kDotThreads - (kDotThreads % (unsigned)nrhs);
}

__device__ __forceinline__ void block_store_partials(double v, int nrhs, double* partial) {
  __shared__ double sh[kDotThreads];
  const unsigned active = dot_threads(nrhs);
  sh[threadIdx.x] = threadIdx.x < active ? v : 0.0;
  __syncthreads();
  if (threadIdx.x < (unsigned)nrhs) {
    double s = 0.0;
    for (unsigned t = threadIdx.x; t < active; t += nrhs) s += sh[t];
    partial[blockIdx.x * kMaxRhs + threadIdx.x] = s;
  }
}

template <typename TB>
__global__ void __launch_bounds__(kDotThreads) dot_kernel(const double* __restrict__ a,
                                                          const TB* __restrict__ b,
                                                          double* __restrict__ partial,
                                                          int64_t rows, int nrhs) {
  pdl_trigger();
  pdl_wait();
  const unsigned act = dot_threads(nrhs);
  const unsigned n = (unsigned)(rows * nrhs);
  double v = 0.0;
  if (threadIdx.x < act) {
    // four independent chains keep eight loads in flight per thread; the
    // order of the additions is still fixed
    const unsigned st = gridDim.x * act;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    unsigned e = blockIdx.x * act + threadIdx.x;
    for (; (uint64_t)e + 3ull * st < n; e += 4 * st) {
      v0 += a[e] * widen(b[e]);
      v1 += a[e + st] * widen(b[e + st]);
      v2 += a[e + 2 * st] * widen(b[e + 2 * st]);
      v3 += a[e + 3 * st] * widen(b[e + 3 * st]);
    }
    for (; e < n; e += st) v0 += a[e] * widen(b[e]);
    v = (v0 + v1) + (v2 + v3);
  }
  block_store_partials(v, nrhs, partial);
}

__global__ void __launch_bounds__(kDotThreads) pcg_init_kernel(
    const double* __restrict__ b, const uint8_t* __restrict__ row_free, double* __restrict__ r,
    float* __restrict__ r32, double* __restrict__ x, double* __restrict__ p,
    double* __restrict__ partial, int64_t rows, int nrhs) {
  pdl_trigger();
  pdl_wait();
  const unsigned act = dot_threads(nrhs);
  const unsigned n = (unsigned)(rows * nrhs);
  double v = 0.0;
  if (threadIdx.x < act)
    for (unsigned e = blockIdx.x * act + threadIdx.x; e < n; e += gridDim.x * act) {
      const double bv = row_free[e / (unsigned)nrhs] ? b[e] : 0.0;
      r[e] = bv;
      r32[e] = (float)bv;
      x[e] = 0.0;
      p[e] = 0.0;
      v += bv * bv;
    }
  block_store_partials(v, nrhs, partial);
}

// Sum of the kDotBlocks partials of column q, by one warp (lanes take blocks
// lane, lane+32, ...; then a fixed butterfly).  Every lane returns the total.
__device__ __forceinline__ double sum_partials_warp(const double* partial, int q) {
  const int lane = threadIdx.x & 31;
  static_assert(kDotBlocks % 32 == 0, "every lane reads the same number of partials");
  double acc[4] = {0.0, 0.0, 0.0, 0.0};      // four independent chains
#pragma unroll
  for (int i = 0; i < kDotBlocks / 32; ++i) acc[i % 4] += partial[(lane + 32 * i) * kMaxRhs + q];
  double s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Scalar kernels run one warp per column (blockDim = 32 * kMaxRhs).
__device__ __forceinline__ void start_column(PcgScalars* sc, int q, double bn, bool used) {
  sc->bnorm[q] = bn;
  sc->rnorm[q] = bn;
  sc->rho[q] = 0.0;
  sc->alpha[q] = 0.0;
  sc->beta[q] = 0.0;
  sc->iters[q] = 0;
  sc->first[q] = 1;
  sc->failed[q] = 0;
  sc->broken[q] = 0;
  sc->active[q] = (used && bn > 0.0) ? 1 : 0;
}

__global__ void pcg_start_kernel(PcgScalars* sc, const double* partial, int nrhs, double rtol,
                                 int maxit) {
  pdl_trigger();
  pdl_wait();
  __shared__ int act[kMaxRhs];
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double bn = q < nrhs ? sqrt(sum_partials_warp(partial, q)) : 0.0;
  if (lane == 0) {
    start_column(sc, q, bn, q < nrhs);
    act[q] = sc->active[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = 0;
    for (int j = 0; j < kMaxRhs; ++j) any |= act[j];
    sc->any_active = any;
    sc->breakdown = 0;
    sc->rtol = rtol;
    sc->maxit = maxit;
  }
}

__global__ void batch_reset_kernel(PcgScalars* sc, double rtol, int maxit) {
  const int q = threadIdx.x;
  if (q < kMaxRhs) start_column(sc, q, 0.0, false);
  if (q == 0) {
    sc->any_active = 0;
    sc->breakdown = 0;
    sc->rtol = rtol;
    sc->maxit = maxit;
  }
}

// Columns first_slot .. first_slot + ncols - 1 of the [rows][nslots] batch
// vectors start from columns 0 .. ncols - 1 of b [rows][ldb]: r = b on free
// rows, x = p = 0; partial sums of ||b||^2 per column.  A thread keeps one
// column (threadIdx.x mod ncols) and strides over rows.
__global__ void __launch_bounds__(kDotThreads) batch_admit_kernel(
    const double* __restrict__ b, int ldb, const uint8_t* __restrict__ row_free,
    double* __restrict__ r, float* __restrict__ r32, double* __restrict__ x, double* __restrict__ p,
    double* __restrict__ partial, int64_t rows, int nslots, int first_slot, int ncols) {
  const unsigned act = dot_threads(ncols);
  const int64_t per_block = act / ncols;
  double v = 0.0;
  if (threadIdx.x < act) {
    const int c = threadIdx.x % ncols;
    for (int64_t i = blockIdx.x * per_block + threadIdx.x / ncols; i < rows;
         i += (int64_t)gridDim.x * per_block) {
      const double bv = row_free[i] ? b[i * ldb + c] : 0.0;
      const int64_t e = i * nslots + first_slot + c;
      r[e] = bv;
      r32[e] = (float)bv;
      x[e] = 0.0;
      p[e] = 0.0;
      v += bv * bv;
    }
  }
  block_store_partials(v, ncols, partial);
}

// One warp per admitted column: ||b|| and the column's start state.
__global__ void batch_admit_scalar_kernel(PcgScalars* sc, const double* partial, int first_slot,
                                          int ncols) {
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c < ncols) {
    const double bn = sqrt(sum_partials_warp(partial, c));
    if (lane == 0) start_column(sc, first_slot + c, bn, true);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = sc->any_active;
    for (int j = 0; j < ncols; ++j) any |= sc->active[first_slot + j];
    sc->any_active = any;
  }
}

// out [rows] = column `slot` of v [rows][nslots].
__global__ void column_gather_kernel(const double* __restrict__ v, double* __restrict__ out,
                                     int64_t rows, int nslots, int slot) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v[i * nslots + slot];
}

// Repacking a batch: column j < new_slots of [rows][new_slots] takes column
// m.s[j] of [rows][old_slots] (zero where m.s[j] < 0); out32, if given,
// receives the same values rounded to FP32.
__global__ void __launch_bounds__(kDotThreads) batch_repack_vec_kernel(
    const double* __restrict__ in, double* __restrict__ out, float* __restrict__ out32,
    int64_t rows, int old_slots, int new_slots, SlotMap m) {
  const int64_t n = rows * new_slots;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / new_slots;
    const int q = m.s[e - i * new_slots];
    const double v = q >= 0 ? in[i * old_slots + q] : 0.0;
    out[e] = v;
    if (out32) out32[e] = (float)v;
  }
}

// The per-column PCG state follows its column; new empty columns start
// inactive.  One thread per column.
__global__ void batch_repack_scalar_kernel(PcgScalars* sc, int new_slots, SlotMap m) {
  __shared__ int act[kMaxRhs];
  const int j = threadIdx.x;
  const int q = j < new_slots ? m.s[j] : -1;
  double rho = 0.0, alpha = 0.0, beta = 0.0, bn = 0.0, rn = 0.0;
  int a = 0, it = 0, first = 1, failed = 0, broken = 0;
  if (q >= 0) {
    rho = sc->rho[q];
    alpha = sc->alpha[q];
    beta = sc->beta[q];
    bn = sc->bnorm[q];
    rn = sc->rnorm[q];
    a = sc->active[q];
    it = sc->iters[q];
    first = sc->first[q];
    failed = sc->failed[q];
    broken = sc->broken[q];
  }
  __syncthreads();
  sc->rho[j] = rho;
  sc->alpha[j] = alpha;
  sc->beta[j] = beta;
  sc->bnorm[j] = bn;
  sc->rnorm[j] = rn;
  sc->active[j] = a;
  sc->iters[j] = it;
  sc->first[j] = first;
  sc->failed[j] = failed;
  sc->broken[j] = broken;
  act[j] = a;
  __syncthreads();
  if (j == 0) {
    int any = 0;
    for (int c = 0; c < kMaxRhs; ++c) any |= act[c];
    sc->any_active = any;
  }
}

// rho_new = r.z; beta = rho_new/rho (0 on the first iteration); rho = rho_new
__global__ void pcg_beta_kernel(PcgScalars* sc, const double* partial, int nrhs) {
  pdl_trigger();
  pdl_wait();
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q < nrhs) {
    const double rn = sum_partials_warp(partial, q);
    if (lane == 0 && sc->active[q]) {
      double beta = 0.0;
      if (!sc->first[q] && sc->rho[q] != 0.0) beta = rn / sc->rho[q];
      if (!isfinite(rn) || !isfinite(beta)) {
        sc->broken[q] = 1;
        sc->breakdown = 1;
        beta = 0.0;
      }
      sc->beta[q] = beta;
      sc->rho[q] = rn;
      sc->first[q] = 0;
    }
  }
}

template <typename TZ>
__global__ void __launch_bounds__(kDotThreads) pcg_p_kernel(const PcgScalars* __restrict__ sc,
                                                            const TZ* __restrict__ z,
                                                            double* __restrict__ p, int64_t n,
                                                            int nrhs) {
  pdl_trigger();
  pdl_wait();
  // the dot-product layout: this thread's elements all lie in column t % nrhs
  const unsigned act = dot_threads(nrhs);
  if (threadIdx.x >= act) return;
  const unsigned q = threadIdx.x % (unsigned)nrhs;
  if (!sc->active[q]) return;
  const double beta = sc->beta[q];
  const unsigned un = (unsigned)n, st = gridDim.x * act;
  unsigned e = blockIdx.x * act + threadIdx.x;
  for (; (uint64_t)e + 3ull * st < un; e += 4 * st) {
    const double z0 = widen(z[e]), z1 = widen(z[e + st]), z2 = widen(z[e + 2 * st]),
                 z3 = widen(z[e + 3 * st]);
    const double p0 = p[e], p1 = p[e + st], p2 = p[e + 2 * st], p3 = p[e + 3 * st];
    p[e] = z0 + beta * p0;
    p[e + st] = z1 + beta * p1;
    p[e + 2 * st] = z2 + beta * p2;
    p[e + 3 * st] = z3 + beta * p3;
  }
  for (; e < un; e += st) p[e] = widen(z[e]) + beta * p[e];
}

// alpha = rho / (p.q); breakdown if p.q <= 0 or non-finite on an active column
__global__ void pcg_alpha_kernel(PcgScalars* sc, const double* partial, int nrhs) {
  pdl_trigger();
  pdl_wait();
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= nrhs) return;
  const double pq = sum_partials_warp(partial, q);
  if (lane != 0) return;
  double alpha = 0.0;
  if (sc->active[q] && !sc->broken[q]) {
    if (!(pq > 0.0) || !isfinite(pq)) {
      sc->broken[q] = 1;
      sc->breakdown = 1;
    } else {
      alpha = sc->rho[q] / pq;
      if (!isfinite(alpha)) {
        sc->broken[q] = 1;
        sc->breakdown = 1;
        alpha = 0.0;
      }
    }
  }
  sc->alpha[q] = alpha;
}

// x += alpha p; r -= alpha q; q = 0; partial ||r||^2
__global__ void __launch_bounds__(kDotThreads) pcg_update_kernel(
    const PcgScalars* __restrict__ sc, const double* __restrict__ p, double* __restrict__ qv,
    double* __restrict__ x, double* __restrict__ r, float* __restrict__ r32,
    double* __restrict__ partial, int64_t rows, int nrhs) {
  pdl_trigger();
  pdl_wait();
  const unsigned act = dot_threads(nrhs);
  const unsigned n = (unsigned)(rows * nrhs);
  double v = 0.0;
  if (threadIdx.x < act) {
    const double al = sc->alpha[threadIdx.x % nrhs];
    for (unsigned e = blockIdx.x * act + threadIdx.x; e < n; e += gridDim.x * act) {
      const double qq = qv[e], pe = p[e], xe = x[e], re = r[e];   // loads before stores
      const double rr = re - al * qq;
      x[e] = xe + al * pe;
      r[e] = rr;
      r32[e] = (float)rr;
      qv[e] = 0.0;
      v += rr * rr;
    }
  }
  block_store_partials(v, nrhs, partial);
}

// Device-side PCG loop (a CUDA graph WHILE node around one captured
// iteration): the first kernel arms the loop if any column is active, the
// last kernel of every iteration re-arms it while a column is active and
// fewer than maxit iterations ran, so the loop always ends.
__global__ void pcg_loop_begin_kernel(cudaGraphConditionalHandle hc, const PcgScalars* sc,
                                      int* count) {
  *count = 0;
  cudaGraphSetConditional(hc, sc->any_active ? 1u : 0u);
}
__global__ void pcg_loop_next_kernel(cudaGraphConditionalHandle hc, const PcgScalars* sc,
                                     int* count) {
  const int c = *count + 1;
  *count = c;
  cudaGraphSetConditional(hc, (sc->any_active && c < sc->maxit) ? 1u : 0u);
}

__global__ void pcg_check_kernel(PcgScalars* sc, const double* partial, int nrhs,
                                 const int* __restrict__ smoother_err) {
  pdl_trigger();
  pdl_wait();
  const bool serr = smoother_err && *smoother_err;     // a smoother's grid barrier gave up
  __shared__ int act[kMaxRhs];
  __shared__ int bad[kMaxRhs];
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double rn = q < nrhs ? sqrt(sum_partials_warp(partial, q)) : 0.0;
  if (lane == 0) {
    int a = 0, b = 0;
    if (q < nrhs && sc->active[q]) {
      if (sc->broken[q] || serr || !isfinite(rn)) {
        sc->broken[q] = 1;
        b = 1;
      } else {
        sc->rnorm[q] = rn;
        sc->iters[q] += 1;
        a = rn <= sc->rtol * sc->bnorm[q] ? 0 : 1;
        if (a && sc->iters[q] >= sc->maxit) {
          sc->failed[q] = 1;
          a = 0;
        }
      }
      sc->active[q] = a;
    }
    act[q] = a;
    bad[q] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = 0, brk = 0;
    for (int j = 0; j < kMaxRhs; ++j) {
      any |= act[j];
      brk |= bad[j];
    }
    if (brk) sc->breakdown = 1;
    sc->any_active = any;
  }
}

__global__ void axpby_dinv_kernel(const double* __restrict__ u, const double* __restrict__ dinv,
                                  const double* __restrict__ vprev, double beta,
                                  double* __restrict__ w, int64_t n) {
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < (unsigned)n;
       e += gridDim.x * blockDim.x)
    w[e] = dinv[e] * u[e] - beta * vprev[e];
}

__global__ void __launch_bounds__(kDotThreads) dotw_kernel(const double* __restrict__ a,
                                                           const double* __restrict__ b,
                                                           const double* __restrict__ wgt,
                                                           double* __restrict__ partial, int64_t n) {
  double v = 0.0;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < (unsigned)n;
       e += gridDim.x * blockDim.x)
    v += a[e] * b[e] * wgt[e];
  block_store_partials(v, 1, partial);
}

// hl[2i] + hl[2i+1] = a[i] to about 2^-48 relative (double-word split)
__global__ void split_dw_kernel(const double* __restrict__ a, float* __restrict__ hl, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = a[i];
    const float h = __double2float_rn(v);
    hl[2 * i] = h;
    hl[2 * i + 1] = __double2float_rn(v - (double)h);
  }
}

__global__ void axpy_kernel(double a, const double* __restrict__ x, double* __restrict__ y,
                            double sy, int64_t n) {
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < (unsigned)n;
       e += gridDim.x * blockDim.x)
    y[e] = sy * y[e] + a * x[e];
}

}  // namespace

inline bool too_big(int64_t n) { return n > (int64_t)INT32_MAX; }

template <typename T>
cudaError_t launch_cheb_init(const T* f, const T* dinv, T* d, T* x, double c, int64_t rows,
                             int nrhs, cudaStream_t s) {
  const int64_t n = rows * nrhs;
  if (n == 0) return cudaSuccess;
  if (too_big(n)) return cudaErrorInvalidValue;
  return launch_k(cheb_init_kernel<T>, vblocks(n), 256, 0, s, f, dinv, d, x, (T)c, n, nrhs);
}
template <typename T>
cudaError_t launch_cheb_step(const T* f, T* t, const T* dinv, T* d, T* x, double cd, double cr,
                             int64_t rows, int nrhs, cudaStream_t s) {
  const int64_t n = rows * nrhs;
  if (n == 0) return cudaSuccess;
  if (too_big(n)) return cudaErrorInvalidValue;
  return launch_k(cheb_step_kernel<T>, vblocks(n), 256, 0, s, f, t, dinv, d, x, (T)cd, (T)cr, n, nrhs);
}
template <typename T>
cudaError_t launch_residual(const T* f, T* t, T* r, int64_t rows, int nrhs, cudaStream_t s) {
  const int64_t n = rows * nrhs;
  if (n == 0) return cudaSuccess;
  if (too_big(n)) return cudaErrorInvalidValue;
  return launch_k(residual_kernel<T>, vblocks(n), 256, 0, s, f, t, r, n);
}
template <typename TI, typename TO>
cudaError_t launch_cast(const TI* a, TO* b, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (too_big(n)) return cudaErrorInvalidValue;
  return launch_k(cast_kernel<TI, TO>, vblocks(n), 256, 0, s, a, b, n);
}
template <typename TB>
cudaError_t launch_dot_partial(const double* a, const TB* b, double* partial, int64_t rows,
                               int nrhs, cudaStream_t s) {
  if (too_big(rows * nrhs)) return cudaErrorInvalidValue;
  return launch_k(dot_kernel<TB>, kDotBlocks, kDotThreads, 0, s, a, b, partial, rows, nrhs);
}
cudaError_t launch_pcg_init(const double* b, const uint8_t* row_free, double* r, float* r32,
                            double* x, double* p, double* partial, int64_t rows, int nrhs,
                            cudaStream_t s) {
  if (too_big(rows * nrhs)) return cudaErrorInvalidValue;
  return launch_k(pcg_init_kernel, kDotBlocks, kDotThreads, 0, s, b, row_free, r, r32, x, p, partial,
                  rows, nrhs);
}
cudaError_t launch_pcg_start(PcgScalars* sc, const double* partial, int nrhs, double rtol,
                             int maxit, cudaStream_t s) {
  return launch_k(pcg_start_kernel, 1, 32 * kMaxRhs, 0, s, sc, partial, nrhs, rtol, maxit);
}
cudaError_t launch_batch_reset(PcgScalars* sc, double rtol, int maxit, cudaStream_t s) {
  batch_reset_kernel<<<1, 32, 0, s>>>(sc, rtol, maxit);
  return cudaGetLastError();
}
cudaError_t launch_batch_admit(const double* b, int ldb, const uint8_t* row_free, double* r,
                               float* r32, double* x, double* p, double* partial, PcgScalars* sc,
                               int64_t rows, int nslots, int first_slot, int ncols, cudaStream_t s) {
  batch_admit_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(b, ldb, row_free, r, r32, x, p, partial,
                                                       rows, nslots, first_slot, ncols);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_admit_scalar_kernel<<<1, 32 * kMaxRhs, 0, s>>>(sc, partial, first_slot, ncols);
  return cudaGetLastError();
}
cudaError_t launch_column_gather(const double* v, double* out, int64_t rows, int nslots, int slot,
                                 cudaStream_t s) {
  column_gather_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(v, out, rows, nslots, slot);
  return cudaGetLastError();
}
cudaError_t launch_batch_repack(double* x, double* r, float* r32, double* p, double* tmp,
                                PcgScalars* sc, int64_t rows, int old_slots, int new_slots,
                                const SlotMap& m, cudaStream_t s) {
  const size_t bytes = (size_t)rows * new_slots * sizeof(double);
  double* vec[3] = {x, r, p};
  for (int v = 0; v < 3; ++v) {
    batch_repack_vec_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(vec[v], tmp, v == 1 ? r32 : nullptr,
                                                               rows, old_slots, new_slots, m);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(vec[v], tmp, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  // tmp is the operator's output A p, which is zero between iterations (the
  // operator adds into it)
  cudaError_t e = cudaMemsetAsync(tmp, 0, bytes, s);
  if (e != cudaSuccess) return e;
  batch_repack_scalar_kernel<<<1, kMaxRhs, 0, s>>>(sc, new_slots, m);
  return cudaGetLastError();
}
template <typename TZ>
cudaError_t launch_pcg_beta_p(PcgScalars* sc, const double* partial, const TZ* z, double* p,
                              int64_t rows, int nrhs, cudaStream_t s) {
  cudaError_t eb = launch_k(pcg_beta_kernel, 1, 32 * kMaxRhs, 0, s, sc, partial, nrhs);
  if (eb != cudaSuccess) return eb;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t n = rows * nrhs;
  if (too_big(n)) return cudaErrorInvalidValue;
  return launch_k(pcg_p_kernel<TZ>, kDotBlocks, kDotThreads, 0, s, sc, z, p, n, nrhs);
}
cudaError_t launch_pcg_alpha(PcgScalars* sc, const double* partial, int nrhs, cudaStream_t s) {
  return launch_k(pcg_alpha_kernel, 1, 32 * kMaxRhs, 0, s, sc, partial, nrhs);
}
cudaError_t launch_pcg_update(const PcgScalars* sc, const double* p, double* q, double* x,
                              double* r, float* r32, double* partial, int64_t rows, int nrhs,
                              cudaStream_t s) {
  if (too_big(rows * nrhs)) return cudaErrorInvalidValue;
  return launch_k(pcg_update_kernel, kDotBlocks, kDotThreads, 0, s, sc, p, q, x, r, r32, partial, rows, nrhs);
}
cudaError_t launch_pcg_loop_begin(cudaGraphConditionalHandle hc, const PcgScalars* sc, int* count,
                                  cudaStream_t s) {
  pcg_loop_begin_kernel<<<1, 1, 0, s>>>(hc, sc, count);
  return cudaGetLastError();
}
cudaError_t launch_pcg_loop_next(cudaGraphConditionalHandle hc, const PcgScalars* sc, int* count,
                                 cudaStream_t s) {
  pcg_loop_next_kernel<<<1, 1, 0, s>>>(hc, sc, count);
  return cudaGetLastError();
}
cudaError_t launch_pcg_check(PcgScalars* sc, const double* partial, int nrhs, const int* smoother_err,
                             cudaStream_t s) {
  return launch_k(pcg_check_kernel, 1, 32 * kMaxRhs, 0, s, sc, partial, nrhs, smoother_err);
}
cudaError_t launch_axpby_dinv(const double* u, const double* dinv, const double* vprev,
                              double beta, double* w, int64_t rows, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  if (too_big(rows)) return cudaErrorInvalidValue;
  axpby_dinv_kernel<<<vblocks(rows), 256, 0, s>>>(u, dinv, vprev, beta, w, rows);
  return cudaGetLastError();
}
cudaError_t launch_dot_weighted(const double* a, const double* b, const double* wgt,
                                double* partial, int64_t rows, cudaStream_t s) {
  if (too_big(rows)) return cudaErrorInvalidValue;
  dotw_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(a, b, wgt, partial, rows);
  return cudaGetLastError();
}
cudaError_t launch_split_dw(const double* a, float* hl, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  split_dw_kernel<<<vblocks(n), 256, 0, s>>>(a, hl, n);
  return cudaGetLastError();
}
cudaError_t launch_axpy(double a, const double* x, double* y, double sy, int64_t rows,
                        cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  if (too_big(rows)) return cudaErrorInvalidValue;
  axpy_kernel<<<vblocks(rows), 256, 0, s>>>(a, x, y, sy, rows);
  return cudaGetLastError();
}

#define NNMG_VT(T)                                                                              \
  template cudaError_t launch_cheb_init<T>(const T*, const T*, T*, T*, double, int64_t, int,   \
                                           cudaStream_t);                                       \
  template cudaError_t launch_cheb_step<T>(const T*, T*, const T*, T*, T*, double, double,     \
                                           int64_t, int, cudaStream_t);                         \
  template cudaError_t launch_residual<T>(const T*, T*, T*, int64_t, int, cudaStream_t);       \
  template cudaError_t launch_dot_partial<T>(const double*, const T*, double*, int64_t, int,   \
                                             cudaStream_t);                                     \
  template cudaError_t launch_pcg_beta_p<T>(PcgScalars*, const double*, const T*, double*,     \
                                            int64_t, int, cudaStream_t);
NNMG_VT(float)
NNMG_VT(double)
#undef NNMG_VT
template cudaError_t launch_cast<double, float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_cast<float, double>(const float*, double*, int64_t, cudaStream_t);

}  // namespace nnmg
