// The coarsest level's dense operator and its inverse, built on the device at
// setup (the direct coarse solve of Algorithm 1, applied per V-cycle as a
// matrix-vector product with the inverse).
//
// Assembly: the operator is applied to batches of unit vectors at the free
// rows; the free rows of the results are the matrix's columns.  The matrix is
// symmetrised (the operator is symmetric up to rounding).
//
// Inverse: blocked Gauss-Jordan elimination in place, without pivoting, with
// pivot blocks of kGJ rows.  For pivot block p and the rest q of the index
// set, one step maps M to
//   M_pp <- M_pp^-1,  M_pq <- M_pp^-1 M_pq,  M_qq <- M_qq - M_qp M_pp^-1 M_pq,
//   M_qp <- -M_qp M_pp^-1,
// so that after the last block M holds the inverse.  For a symmetric positive
// definite matrix every pivot block is a diagonal block of a Schur complement,
// itself symmetric positive definite, so no pivoting is needed; a
// non-positive scalar pivot inside a block (a matrix that is not positive
// definite) sets the error flag.  The trailing update M_qq - M_qp (M_pp^-1 M_pq)
// is a rank-kGJ product computed in 64 x 64 tiles from shared memory: n^3
// multiply-adds in all, on the FP64 pipe.
#include <algorithm>

#include "nnmg_internal.h"

namespace nnmg {
namespace {

constexpr int kGJ = 64;        // pivot block
constexpr int kTile = 64;      // update tile (rows and columns)

// D[i][j0 + c] = Y[rows[i]][c] for the m columns of a batch (Y is [rows][m]).
__global__ void gather_columns_kernel(const double* __restrict__ Y, int m,
                                      const int32_t* __restrict__ rows, int n, int j0,
                                      double* __restrict__ D) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * m) return;
  const int i = (int)(e / m), c = (int)(e - (int64_t)i * m);
  D[(int64_t)i * n + j0 + c] = Y[(int64_t)rows[i] * m + c];
}

// X = the m unit vectors e_{rows[j0 + c]} (X is [nrows][m], zeroed before).
__global__ void unit_columns_kernel(double* __restrict__ X, int m, const int32_t* __restrict__ rows,
                                    int j0) {
  const int c = threadIdx.x;
  if (c < m) X[(int64_t)rows[j0 + c] * m + c] = 1.0;
}

// D <- (D + D^T) / 2, one thread per pair (i > j).
__global__ void symmetrize_kernel(double* __restrict__ D, int n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t pairs = (int64_t)n * (n - 1) / 2;
  if (e >= pairs) return;
  // e = i (i - 1) / 2 + j with 0 <= j < i
  int i = (int)((1.0 + sqrt(1.0 + 8.0 * (double)e)) * 0.5);
  while ((int64_t)i * (i - 1) / 2 > e) --i;
  while ((int64_t)(i + 1) * i / 2 <= e) ++i;
  const int j = (int)(e - (int64_t)i * (i - 1) / 2);
  const double v = 0.5 * (D[(int64_t)i * n + j] + D[(int64_t)j * n + i]);
  D[(int64_t)i * n + j] = v;
  D[(int64_t)j * n + i] = v;
}

// Invert the pivot block M[k0..k0+b)[k0..k0+b) in place (b <= kGJ) by scalar
// Gauss-Jordan steps in shared memory; also writes it to pinv [b][b].
__global__ void __launch_bounds__(256) gj_pivot_kernel(double* __restrict__ M, int n, int k0, int b,
                                                       double* __restrict__ pinv, int* err) {
  __shared__ double P[kGJ][kGJ + 1];
  __shared__ double row[kGJ], col[kGJ];
  for (int e = threadIdx.x; e < b * b; e += blockDim.x)
    P[e / b][e % b] = M[(int64_t)(k0 + e / b) * n + k0 + e % b];
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    for (int t = threadIdx.x; t < b; t += blockDim.x) {
      row[t] = P[j][t];
      col[t] = P[t][j];
    }
    __syncthreads();
    const double piv = row[j];
    if (!(piv > 0.0)) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      return;                                   // the whole block leaves (piv is uniform)
    }
    const double ip = 1.0 / piv;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
      const int r = e / b, c = e - r * b;
      double v;
      if (r == j)
        v = c == j ? ip : row[c] * ip;
      else if (c == j)
        v = -col[r] * ip;
      else
        v = P[r][c] - col[r] * (row[c] * ip);
      P[r][c] = v;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const double v = P[e / b][e % b];
    M[(int64_t)(k0 + e / b) * n + k0 + e % b] = v;
    pinv[e] = v;
  }
}

// C = M[:, k0..k0+b) (old column panel, rows outside the pivot block; pivot
// rows set to zero), [n][b].
__global__ void gj_copy_col_kernel(const double* __restrict__ M, int n, int k0, int b,
                                   double* __restrict__ C) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * b) return;
  const int i = (int)(e / b), s = (int)(e - (int64_t)i * b);
  C[e] = (i >= k0 && i < k0 + b) ? 0.0 : M[(int64_t)i * n + k0 + s];
}

// Row panel: M[k0+r][j] <- sum_s pinv[r][s] M[k0+s][j] for the kTile columns
// j of this block outside the pivot block (in place: the block's columns are
// read into shared memory first).
__global__ void __launch_bounds__(256) gj_row_kernel(double* __restrict__ M, int n, int k0, int b,
                                                     const double* __restrict__ pinv) {
  __shared__ double V[kGJ][kTile + 1];
  const int j0 = blockIdx.x * kTile;
  for (int e = threadIdx.x; e < b * kTile; e += blockDim.x) {
    const int s = e / kTile, c = e - s * kTile, j = j0 + c;
    V[s][c] = j < n ? M[(int64_t)(k0 + s) * n + j] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < b * kTile; e += blockDim.x) {
    const int r = e / kTile, c = e - r * kTile, j = j0 + c;
    if (j >= n || (j >= k0 && j < k0 + b)) continue;
    double acc = 0.0;
    const double* pr = pinv + r * b;              // one row, shared by the block's threads (L1)
    for (int s = 0; s < b; ++s) acc += pr[s] * V[s][c];
    M[(int64_t)(k0 + r) * n + j] = acc;
  }
}

// Trailing update and column panel, one 64 x 64 tile per block, rows outside
// the pivot block: M[i][j] <- base - sum_s C[i][s] R[s][j], with base = M[i][j]
// and R = the new row panel for columns outside the pivot block, base = 0 and
// R = pinv for the pivot block's columns (the new column panel -C pinv).
// 256 threads, each a 4 x 4 sub-tile.
__global__ void __launch_bounds__(256) gj_update_kernel(double* __restrict__ M, int n, int k0,
                                                        int b, const double* __restrict__ C,
                                                        const double* __restrict__ pinv) {
  extern __shared__ double smem_gj[];
  double(*Cs)[kGJ + 1] = reinterpret_cast<double(*)[kGJ + 1]>(smem_gj);               // [kTile][kGJ+1]
  double(*Rs)[kTile + 1] = reinterpret_cast<double(*)[kTile + 1]>(smem_gj + kTile * (kGJ + 1));
  const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
  for (int e = threadIdx.x; e < kTile * b; e += blockDim.x) {
    const int r = e / b, s = e - r * b, i = i0 + r;
    Cs[r][s] = i < n ? C[(int64_t)i * b + s] : 0.0;
  }
  for (int e = threadIdx.x; e < b * kTile; e += blockDim.x) {
    const int s = e / kTile, c = e - s * kTile, j = j0 + c;
    double v = 0.0;
    if (j < n) v = (j >= k0 && j < k0 + b) ? pinv[s * b + (j - k0)] : M[(int64_t)(k0 + s) * n + j];
    Rs[s][c] = v;
  }
  __syncthreads();
  const int tr = (threadIdx.x / 16) * 4, tc = (threadIdx.x % 16) * 4;
  double acc[4][4] = {{0.0}};
  for (int s = 0; s < b; ++s) {
    double a[4], r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[q] = Cs[tr + q][s];
      r[q] = Rs[s][tc + q];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * r[q];
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = i0 + tr + p;
    if (i >= n || (i >= k0 && i < k0 + b)) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + tc + q;
      if (j >= n) continue;
      const bool piv_col = j >= k0 && j < k0 + b;
      double* m = M + (int64_t)i * n + j;
      *m = (piv_col ? 0.0 : *m) - acc[p][q];
    }
  }
}

}  // namespace

// The free-row block of the coarsest operator into D [n][n] (n = L.n_free_rows,
// rows = L.free_rows) and its inverse in place.  X, Y: device work vectors of
// L.rows x kMaxRhs doubles; work: n x kGJ + kGJ x kGJ doubles; err: device int.
// Everything is enqueued on s; the caller synchronises and reads *err.
cudaError_t launch_coarse_inverse(const DevLevel& L, double lambda, double mu, double* D, double* X,
                                  double* Y, double* work, int* err, cudaStream_t s) {
  const int n = L.n_free_rows;
  if (n == 0) return cudaSuccess;
  cudaError_t e;
  for (int j0 = 0; j0 < n; j0 += kMaxRhs) {
    const int m = std::min(kMaxRhs, n - j0);
    if ((e = cudaMemsetAsync(X, 0, (size_t)L.rows * m * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Y, 0, (size_t)L.rows * m * sizeof(double), s)) != cudaSuccess) return e;
    unit_columns_kernel<<<1, kMaxRhs, 0, s>>>(X, m, L.free_rows, j0);
    if ((e = launch_operator<double>(L, X, Y, m, lambda, mu, s)) != cudaSuccess) return e;
    const int64_t t = (int64_t)n * m;
    gather_columns_kernel<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(Y, m, L.free_rows, n, j0, D);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int64_t pairs = (int64_t)n * (n - 1) / 2;
  if (pairs > 0) symmetrize_kernel<<<(unsigned)((pairs + 255) / 256), 256, 0, s>>>(D, n);
  double* C = work;
  double* pinv = work + (size_t)n * kGJ;
  const unsigned tiles = (unsigned)((n + kTile - 1) / kTile);
  const size_t usmem = ((size_t)kTile * (kGJ + 1) + (size_t)kGJ * (kTile + 1)) * sizeof(double);
  static bool granted = false;
  if (!granted) {
    if ((e = cudaFuncSetAttribute(gj_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)usmem)) != cudaSuccess)
      return e;
    granted = true;
  }
  for (int k0 = 0; k0 < n; k0 += kGJ) {
    const int b = std::min(kGJ, n - k0);
    gj_pivot_kernel<<<1, 256, 0, s>>>(D, n, k0, b, pinv, err);
    gj_copy_col_kernel<<<(unsigned)(((int64_t)n * b + 255) / 256), 256, 0, s>>>(D, n, k0, b, C);
    gj_row_kernel<<<tiles, 256, 0, s>>>(D, n, k0, b, pinv);
    gj_update_kernel<<<dim3(tiles, tiles), 256, usmem, s>>>(D, n, k0, b, C, pinv);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace nnmg
