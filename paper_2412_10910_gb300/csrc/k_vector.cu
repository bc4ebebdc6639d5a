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

inline unsigned vblocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (unsigned)b;
}

template <typename T>
__global__ void cheb_init_kernel(const T* __restrict__ f, const T* __restrict__ dinv,
                                 T* __restrict__ d, T* __restrict__ x, T c, int64_t n, int nrhs) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const T v = c * dinv[e / nrhs] * f[e];
    d[e] = v;
    x[e] = v;
  }
}

// r = f - t (t then reset to 0); d = cd*d + cr*Dinv r; x += d
template <typename T>
__global__ void cheb_step_kernel(const T* __restrict__ f, T* __restrict__ t,
                                 const T* __restrict__ dinv, T* __restrict__ d, T* __restrict__ x,
                                 T cd, T cr, int64_t n, int nrhs) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const T r = f[e] - t[e];
    t[e] = T(0);
    const T dn = cd * d[e] + cr * dinv[e / nrhs] * r;
    d[e] = dn;
    x[e] += dn;
  }
}

template <typename T>
__global__ void residual_kernel(const T* __restrict__ f, T* __restrict__ t, T* __restrict__ r,
                                int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    r[e] = f[e] - t[e];
    t[e] = T(0);
  }
}

template <typename TI, typename TO>
__global__ void cast_kernel(const TI* __restrict__ a, TO* __restrict__ b, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    b[e] = (TO)a[e];
}

// block reduction of nrhs per-thread values into partial[blockIdx.x][kMaxRhs]
__device__ __forceinline__ void block_reduce_store(double (&v)[kMaxRhs], int nrhs, double* partial) {
  __shared__ double sh[kDotThreads / 32][kMaxRhs];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kMaxRhs; ++q) {
    if (q < nrhs) {
      double s = v[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) sh[wid][q] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x < nrhs) {
    double s = 0.0;
    for (int w = 0; w < kDotThreads / 32; ++w) s += sh[w][threadIdx.x];
    partial[blockIdx.x * kMaxRhs + threadIdx.x] = s;
  }
}

template <typename TB>
__global__ void __launch_bounds__(kDotThreads) dot_kernel(const double* __restrict__ a,
                                                          const TB* __restrict__ b,
                                                          double* __restrict__ partial,
                                                          int64_t rows, int nrhs) {
  double v[kMaxRhs];
#pragma unroll
  for (int q = 0; q < kMaxRhs; ++q) v[q] = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int q = 0; q < kMaxRhs; ++q)
      if (q < nrhs) v[q] += a[r * nrhs + q] * (double)b[r * nrhs + q];
  }
  block_reduce_store(v, nrhs, partial);
}

__global__ void __launch_bounds__(kDotThreads) pcg_init_kernel(
    const double* __restrict__ b, const uint8_t* __restrict__ row_free, double* __restrict__ r,
    double* __restrict__ x, double* __restrict__ p, double* __restrict__ partial, int64_t rows,
    int nrhs) {
  double v[kMaxRhs];
#pragma unroll
  for (int q = 0; q < kMaxRhs; ++q) v[q] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool fr = row_free[i] != 0;
#pragma unroll
    for (int q = 0; q < kMaxRhs; ++q) {
      if (q < nrhs) {
        const double bv = fr ? b[i * nrhs + q] : 0.0;
        r[i * nrhs + q] = bv;
        x[i * nrhs + q] = 0.0;
        p[i * nrhs + q] = 0.0;
        v[q] += bv * bv;
      }
    }
  }
  block_reduce_store(v, nrhs, partial);
}

__device__ __forceinline__ double sum_partials(const double* partial, int q) {
  double s = 0.0;
  for (int bk = 0; bk < kDotBlocks; ++bk) s += partial[bk * kMaxRhs + q];
  return s;
}

__global__ void pcg_start_kernel(PcgScalars* sc, const double* partial, int nrhs, double rtol) {
  if (threadIdx.x != 0) return;
  int any = 0;
  for (int q = 0; q < kMaxRhs; ++q) {
    const double bn = q < nrhs ? sqrt(sum_partials(partial, q)) : 0.0;
    sc->bnorm[q] = bn;
    sc->rnorm[q] = bn;
    sc->rho[q] = 0.0;
    sc->alpha[q] = 0.0;
    sc->beta[q] = 0.0;
    sc->iters[q] = 0;
    sc->active[q] = (q < nrhs && bn > 0.0) ? 1 : 0;
    any |= sc->active[q];
  }
  sc->first = 1;
  sc->any_active = any;
  sc->breakdown = 0;
  sc->rtol = rtol;
}

// rho_new = r.z; beta = rho_new/rho (0 on the first iteration); rho = rho_new
__global__ void pcg_beta_kernel(PcgScalars* sc, const double* partial, int nrhs) {
  const int q = threadIdx.x;
  const int first = sc->first;
  __syncwarp();
  if (q < nrhs) {
    const double rn = sum_partials(partial, q);
    double beta = 0.0;
    if (!first && sc->rho[q] != 0.0) beta = rn / sc->rho[q];
    if (!isfinite(rn) || !isfinite(beta)) {
      if (sc->active[q]) sc->breakdown = 1;
      beta = 0.0;
    }
    sc->beta[q] = beta;
    sc->rho[q] = rn;
  }
  if (q == 0) sc->first = 0;
}

template <typename TZ>
__global__ void pcg_p_kernel(const PcgScalars* __restrict__ sc, const TZ* __restrict__ z,
                             double* __restrict__ p, int64_t n, int nrhs) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % nrhs);
    if (sc->active[q]) p[e] = (double)z[e] + sc->beta[q] * p[e];
  }
}

// alpha = rho / (p.q); breakdown if p.q <= 0 or non-finite on an active column
__global__ void pcg_alpha_kernel(PcgScalars* sc, const double* partial, int nrhs) {
  const int q = threadIdx.x;
  if (q >= nrhs) return;
  const double pq = sum_partials(partial, q);
  double alpha = 0.0;
  if (sc->active[q]) {
    if (!(pq > 0.0) || !isfinite(pq)) {
      sc->breakdown = 1;
    } else {
      alpha = sc->rho[q] / pq;
      if (!isfinite(alpha)) {
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
    double* __restrict__ x, double* __restrict__ r, double* __restrict__ partial, int64_t rows,
    int nrhs) {
  double v[kMaxRhs];
  double al[kMaxRhs];
#pragma unroll
  for (int q = 0; q < kMaxRhs; ++q) {
    v[q] = 0.0;
    al[q] = q < nrhs ? sc->alpha[q] : 0.0;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int q = 0; q < kMaxRhs; ++q) {
      if (q < nrhs) {
        const int64_t e = i * nrhs + q;
        const double qq = qv[e];
        x[e] += al[q] * p[e];
        const double rr = r[e] - al[q] * qq;
        r[e] = rr;
        qv[e] = 0.0;
        v[q] += rr * rr;
      }
    }
  }
  block_reduce_store(v, nrhs, partial);
}

__global__ void pcg_check_kernel(PcgScalars* sc, const double* partial, int nrhs) {
  if (threadIdx.x != 0) return;
  int any = 0;
  for (int q = 0; q < nrhs; ++q) {
    if (sc->active[q]) {
      const double rn = sqrt(sum_partials(partial, q));
      sc->rnorm[q] = rn;
      sc->iters[q] += 1;
      if (rn <= sc->rtol * sc->bnorm[q]) sc->active[q] = 0;
      if (!isfinite(rn)) sc->breakdown = 1;
    }
    any |= sc->active[q];
  }
  sc->any_active = sc->breakdown ? 0 : any;
}

__global__ void axpby_dinv_kernel(const double* __restrict__ u, const double* __restrict__ dinv,
                                  const double* __restrict__ vprev, double beta,
                                  double* __restrict__ w, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    w[e] = dinv[e] * u[e] - beta * vprev[e];
}

__global__ void __launch_bounds__(kDotThreads) dotw_kernel(const double* __restrict__ a,
                                                           const double* __restrict__ b,
                                                           const double* __restrict__ wgt,
                                                           double* __restrict__ partial, int64_t n) {
  double v[kMaxRhs];
#pragma unroll
  for (int q = 0; q < kMaxRhs; ++q) v[q] = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    v[0] += a[e] * b[e] * wgt[e];
  block_reduce_store(v, 1, partial);
}

__global__ void axpy_kernel(double a, const double* __restrict__ x, double* __restrict__ y,
                            double sy, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = sy * y[e] + a * x[e];
}

}  // namespace

template <typename T>
cudaError_t launch_cheb_init(const T* f, const T* dinv, T* d, T* x, double c, int64_t rows,
                             int nrhs, cudaStream_t s) {
  const int64_t n = rows * nrhs;
  if (n == 0) return cudaSuccess;
  cheb_init_kernel<T><<<vblocks(n), 256, 0, s>>>(f, dinv, d, x, (T)c, n, nrhs);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cheb_step(const T* f, T* t, const T* dinv, T* d, T* x, double cd, double cr,
                             int64_t rows, int nrhs, cudaStream_t s) {
  const int64_t n = rows * nrhs;
  if (n == 0) return cudaSuccess;
  cheb_step_kernel<T><<<vblocks(n), 256, 0, s>>>(f, t, dinv, d, x, (T)cd, (T)cr, n, nrhs);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_residual(const T* f, T* t, T* r, int64_t rows, int nrhs, cudaStream_t s) {
  const int64_t n = rows * nrhs;
  if (n == 0) return cudaSuccess;
  residual_kernel<T><<<vblocks(n), 256, 0, s>>>(f, t, r, n);
  return cudaGetLastError();
}
template <typename TI, typename TO>
cudaError_t launch_cast(const TI* a, TO* b, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cast_kernel<TI, TO><<<vblocks(n), 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}
template <typename TB>
cudaError_t launch_dot_partial(const double* a, const TB* b, double* partial, int64_t rows,
                               int nrhs, cudaStream_t s) {
  dot_kernel<TB><<<kDotBlocks, kDotThreads, 0, s>>>(a, b, partial, rows, nrhs);
  return cudaGetLastError();
}
cudaError_t launch_pcg_init(const double* b, const uint8_t* row_free, double* r, double* x,
                            double* p, double* partial, int64_t rows, int nrhs, cudaStream_t s) {
  pcg_init_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(b, row_free, r, x, p, partial, rows, nrhs);
  return cudaGetLastError();
}
cudaError_t launch_pcg_start(PcgScalars* sc, const double* partial, int nrhs, double rtol,
                             cudaStream_t s) {
  pcg_start_kernel<<<1, 32, 0, s>>>(sc, partial, nrhs, rtol);
  return cudaGetLastError();
}
template <typename TZ>
cudaError_t launch_pcg_beta_p(PcgScalars* sc, const double* partial, const TZ* z, double* p,
                              int64_t rows, int nrhs, cudaStream_t s) {
  pcg_beta_kernel<<<1, 32, 0, s>>>(sc, partial, nrhs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t n = rows * nrhs;
  pcg_p_kernel<TZ><<<vblocks(n), 256, 0, s>>>(sc, z, p, n, nrhs);
  return cudaGetLastError();
}
cudaError_t launch_pcg_alpha(PcgScalars* sc, const double* partial, int nrhs, cudaStream_t s) {
  pcg_alpha_kernel<<<1, 32, 0, s>>>(sc, partial, nrhs);
  return cudaGetLastError();
}
cudaError_t launch_pcg_update(const PcgScalars* sc, const double* p, double* q, double* x,
                              double* r, double* partial, int64_t rows, int nrhs, cudaStream_t s) {
  pcg_update_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(sc, p, q, x, r, partial, rows, nrhs);
  return cudaGetLastError();
}
cudaError_t launch_pcg_check(PcgScalars* sc, const double* partial, int nrhs, cudaStream_t s) {
  pcg_check_kernel<<<1, 32, 0, s>>>(sc, partial, nrhs);
  return cudaGetLastError();
}
cudaError_t launch_axpby_dinv(const double* u, const double* dinv, const double* vprev,
                              double beta, double* w, int64_t rows, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  axpby_dinv_kernel<<<vblocks(rows), 256, 0, s>>>(u, dinv, vprev, beta, w, rows);
  return cudaGetLastError();
}
cudaError_t launch_dot_weighted(const double* a, const double* b, const double* wgt,
                                double* partial, int64_t rows, cudaStream_t s) {
  dotw_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(a, b, wgt, partial, rows);
  return cudaGetLastError();
}
cudaError_t launch_axpy(double a, const double* x, double* y, double sy, int64_t rows,
                        cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
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
