// Nested (global-coarsening) transfer kernels for the comparison of the
// paper's Sec. 5, the transfer dispatch and the coarsest-level solve.  The
// non-nested point-evaluation transfer itself lives in k_prolong.cu and
// k_restrict.cu.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "nnmg_internal.h"

namespace nnmg {
namespace {

// z[free_i] = sum_j Ainv[i][j] r[free_j] in FP64.  Every lane owns one
// (row, right-hand side) pair: a warp covers 32 / npad rows (npad = nrhs
// rounded up to a power of two), a block kCoarseWarps warps.  The gathered
// right-hand sides of a tile of kCoarseTile columns pass through shared
// memory as [column][npad] (lanes of one row read consecutive banks, lanes of
// one right-hand side the same word), and every lane accumulates its row's
// products over the tile with four independent chains: no cross-lane sums.
constexpr int kCoarseWarps = 8;
constexpr int kCoarseTile = 128;

// The column range of every row is split over gridDim.y segments; segment s
// writes partial[s][row][rhs] and coarse_sum_kernel adds the segments in order
// (deterministic).  With gridDim.y == 1 the kernel writes z directly.
template <typename TI, typename TO>
__global__ void __launch_bounds__(32 * kCoarseWarps) coarse_solve_kernel(
    const double* __restrict__ Ainv, const int32_t* __restrict__ rows, int n,
    const TI* __restrict__ r, TO* __restrict__ z, int nrhs, int npad,
    double* __restrict__ partial) {
  pdl_trigger();
  pdl_wait();
  __shared__ double sr[kCoarseTile * kMaxRhs];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rpw = 32 / npad;                       // rows per warp
  const int q = lane % npad;
  const int i = (blockIdx.x * kCoarseWarps + warp) * rpw + lane / npad;
  const bool own = q < nrhs && i < n;
  const int seg = (n + gridDim.y - 1) / gridDim.y;
  const int jb = blockIdx.y * seg, je = min(n, jb + seg);
  const double* arow = Ainv + (int64_t)(own ? i : 0) * n;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j0 = jb; j0 < je; j0 += kCoarseTile) {
    const int nt = min(kCoarseTile, je - j0);
    for (int t = threadIdx.x; t < nt * npad; t += blockDim.x) {
      const int jj = t / npad, qq = t - jj * npad;
      sr[t] = qq < nrhs ? (double)r[(int64_t)rows[j0 + jj] * nrhs + qq] : 0.0;
    }
    __syncthreads();
    if (own) {
      int jj = 0;
      for (; jj + 4 <= nt; jj += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += arow[j0 + jj + u] * sr[(jj + u) * npad + q];
      }
      for (; jj < nt; ++jj) acc[0] += arow[j0 + jj] * sr[jj * npad + q];
    }
    __syncthreads();
  }
  if (!own) return;
  const double v = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  if (gridDim.y == 1)
    z[(int64_t)rows[i] * nrhs + q] = (TO)v;
  else
    partial[((int64_t)blockIdx.y * n + i) * kMaxRhs + q] = v;
}

template <typename TO>
__global__ void coarse_sum_kernel(const double* __restrict__ partial, const int32_t* __restrict__ rows,
                                  int n, int nseg, TO* __restrict__ z, int nrhs) {
  pdl_trigger();
  pdl_wait();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * nrhs) return;
  const int i = e / nrhs, q = e - i * nrhs;
  double s = 0.0;
  for (int g = 0; g < nseg; ++g) s += partial[((int64_t)g * n + i) * kMaxRhs + q];
  z[(int64_t)rows[i] * nrhs + q] = (TO)s;
}

// Opt a kernel in to `dyn` bytes of dynamic shared memory when its static
// and dynamic shared memory together exceed the default 48 KB per block;
// `granted` remembers the largest size already allowed for this kernel.
template <typename F>
cudaError_t allow_smem(F kern, size_t dyn, size_t* granted) {
  if (dyn <= *granted) return cudaSuccess;
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kern);
  if (e != cudaSuccess) return e;
  if (dyn + a.sharedSizeBytes > 48 * 1024) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  *granted = dyn;
  return cudaSuccess;
}

// ---------------------------------------------------------------- nested (GC)
// Transfer between nested levels (the global-coarsening comparison of the
// paper's Sec. 5): a fine cell that is child b = (b_0, b_1, b_2) of coarse
// cell c carries u_f = (E_{b_2} x E_{b_1} x E_{b_0}) u_c with the 1D matrices
// E_b[m][l] = L_l((b + t_m) / 2) (t_m the Gauss-Lobatto nodes): sum
// factorization, d sweeps of (k+1)^(d+1) FMAs per child.  One block per coarse
// cell; a fine node is written by the child cell that numbered it first, so
// each is written once.  Restriction applies the transposed sweeps and adds
// the children in fixed order into the per-coarse-cell buffer of the
// non-nested restriction, whose second phase then gathers (deterministic).
template <typename T>
struct GcTables {
  T E[2][kMaxN][kMaxN];
};

template <int D, int N, typename T>
__device__ __forceinline__ void gc_sweep(const T (&E)[kMaxN][kMaxN], const T* in, T* out, int dir,
                                         bool transpose, int nch) {
  constexpr int NL = D == 2 ? N * N : N * N * N;
  const int stride = dir == 0 ? 1 : (dir == 1 ? N : N * N);
  for (int e = threadIdx.x; e < NL * nch; e += blockDim.x) {
    const int i = e / nch, ch = e - i * nch;
    const int m = (i / stride) % N;
    const int base = i - m * stride;
    T v = 0;
#pragma unroll
    for (int l = 0; l < N; ++l)
      v += (transpose ? E[l][m] : E[m][l]) * in[(base + l * stride) * nch + ch];
    out[e] = v;
  }
}

template <int D, int K, typename T>
__global__ void gc_prolong_kernel(const int32_t* __restrict__ coarse_cell_nodes,
                                  const T* __restrict__ xc, T* __restrict__ xf,
                                  const int32_t* __restrict__ children,
                                  const int32_t* __restrict__ fine_cell_nodes,
                                  const int32_t* __restrict__ owner_cell,
                                  const int32_t* __restrict__ owner_local, int nch,
                                  GcTables<T> G) {
  constexpr int N = K + 1;
  constexpr int NL = D == 2 ? N * N : N * N * N;
  extern __shared__ unsigned char smem_raw[];
  T* u = reinterpret_cast<T*>(smem_raw);  // [NL][nch] coarse values
  T* a = u + NL * nch;                      // sweep buffers
  T* b = a + NL * nch;
  const int64_t c = blockIdx.x;
  for (int e = threadIdx.x; e < NL * nch; e += blockDim.x) {
    const int j = e / nch, ch = e - j * nch;
    const int node = coarse_cell_nodes[c * NL + j];
    u[e] = node >= 0 ? xc[(int64_t)node * nch + ch] : T(0);
  }
  __syncthreads();
  for (int cb = 0; cb < (1 << D); ++cb) {
    const int f = children[c * (1 << D) + cb];
    gc_sweep<D, N, T>(G.E[cb & 1], u, a, 0, false, nch);
    __syncthreads();
    gc_sweep<D, N, T>(G.E[(cb >> 1) & 1], a, b, 1, false, nch);
    __syncthreads();
    const T* res = b;
    if constexpr (D == 3) {
      gc_sweep<D, N, T>(G.E[(cb >> 2) & 1], b, a, 2, false, nch);
      __syncthreads();
      res = a;
    }
    for (int e = threadIdx.x; e < NL * nch; e += blockDim.x) {
      const int i = e / nch, ch = e - i * nch;
      const int node = fine_cell_nodes[(int64_t)f * NL + i];
      if (node >= 0 && owner_cell[node] == f && owner_local[node] == i)
        xf[(int64_t)node * nch + ch] += res[e];
    }
    __syncthreads();
  }
}

template <int D, int K, typename T>
__global__ void gc_restrict1_kernel(const T* __restrict__ rf, T* __restrict__ buf,
                                    const int32_t* __restrict__ children,
                                    const int32_t* __restrict__ fine_cell_nodes,
                                    const int32_t* __restrict__ owner_cell,
                                    const int32_t* __restrict__ owner_local, int nch,
                                    GcTables<T> G) {
  constexpr int N = K + 1;
  constexpr int NL = D == 2 ? N * N : N * N * N;
  extern __shared__ unsigned char smem_raw[];
  T* acc = reinterpret_cast<T*>(smem_raw);  // [NL][nch]
  T* a = acc + NL * nch;
  T* b = a + NL * nch;
  const int64_t c = blockIdx.x;
  for (int e = threadIdx.x; e < NL * nch; e += blockDim.x) acc[e] = T(0);
  for (int cb = 0; cb < (1 << D); ++cb) {
    const int f = children[c * (1 << D) + cb];
    for (int e = threadIdx.x; e < NL * nch; e += blockDim.x) {
      const int i = e / nch, ch = e - i * nch;
      const int node = fine_cell_nodes[(int64_t)f * NL + i];
      const bool own = node >= 0 && owner_cell[node] == f && owner_local[node] == i;
      a[e] = own ? rf[(int64_t)node * nch + ch] : T(0);
    }
    __syncthreads();
    T* in = a;
    T* out = b;
    if constexpr (D == 3) {
      gc_sweep<D, N, T>(G.E[(cb >> 2) & 1], in, out, 2, true, nch);
      __syncthreads();
      in = b;
      out = a;
    }
    gc_sweep<D, N, T>(G.E[(cb >> 1) & 1], in, out, 1, true, nch);
    __syncthreads();
    gc_sweep<D, N, T>(G.E[cb & 1], out, in, 0, true, nch);
    __syncthreads();
    for (int e = threadIdx.x; e < NL * nch; e += blockDim.x) acc[e] += in[e];
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NL * nch; e += blockDim.x) buf[(c * NL) * nch + e] = acc[e];
}

template <typename T>
GcTables<T> gc_tables(int k) {
  Basis1D<double> d;
  Basis1D<float> f;
  make_basis(k, &d, &f);
  GcTables<T> g;
  std::memset(&g, 0, sizeof(g));
  const int n = k + 1;
  for (int b = 0; b < 2; ++b)
    for (int m = 0; m < n; ++m) {
      const double x = 0.5 * (b + d.gl[m]);
      for (int l = 0; l < n; ++l) {
        double v = d.gl_scale[l];
        for (int q = 0; q < n; ++q)
          if (q != l) v *= x - d.gl[q];
        g.E[b][m][l] = (T)v;
      }
    }
  return g;
}

template <int D, int K, typename T>
cudaError_t gc_prolong_dk(const DevLevel& f, const DevLevel& c, const T* xc, T* xf, int nch,
                          cudaStream_t s) {
  constexpr int N = K + 1;
  constexpr int NL = D == 2 ? N * N : N * N * N;
  const size_t smem = 3 * (size_t)NL * nch * sizeof(T);
  auto kern = gc_prolong_kernel<D, K, T>;
  static size_t granted = 0;
  cudaError_t e = allow_smem(kern, smem, &granted);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)c.n_cells, 128, smem, s>>>(c.cell_nodes, xc, xf, f.gc_children, f.cell_nodes,
                                              f.owner_cell, f.owner_local, nch, gc_tables<T>(K));
  return cudaGetLastError();
}

template <int D, int K, typename T>
cudaError_t gc_restrict_dk(const DevLevel& f, const DevLevel& c, const T* rf, T* rc, T* scratch,
                           int nch, cudaStream_t s) {
  constexpr int N = K + 1;
  constexpr int NL = D == 2 ? N * N : N * N * N;
  const size_t smem = 3 * (size_t)NL * nch * sizeof(T);
  auto kern = gc_restrict1_kernel<D, K, T>;
  static size_t granted = 0;
  cudaError_t e = allow_smem(kern, smem, &granted);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)c.n_cells, 128, smem, s>>>(rf, scratch, f.gc_children, f.cell_nodes,
                                              f.owner_cell, f.owner_local, nch, gc_tables<T>(K));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_restrict_gather<T>(c, scratch, rc, nch, s);
}

}  // namespace

template <typename T>
cudaError_t launch_prolongate_add(const DevLevel& fine, const DevLevel& coarse, const T* xc,
                                  T* xf, int nrhs, cudaStream_t s) {
  if (coarse.n_cells == 0) return cudaSuccess;
  const int nch = fine.ncomp * nrhs;
  if (fine.gc_active) {
#define NNMG_G(D, K) \
  if (fine.dim == D && coarse.k == K) return gc_prolong_dk<D, K, T>(fine, coarse, xc, xf, nch, s);
    NNMG_G(2, 1) NNMG_G(2, 2) NNMG_G(2, 3) NNMG_G(2, 4)
    NNMG_G(3, 1) NNMG_G(3, 2) NNMG_G(3, 3) NNMG_G(3, 4)
#undef NNMG_G
    return cudaErrorInvalidValue;
  }
  return launch_prolongate_points<T>(fine, coarse, xc, xf, nrhs, s);
}

template <typename T>
cudaError_t launch_restrict(const DevLevel& fine, const DevLevel& coarse, const T* rf, T* rc,
                            T* scratch, int nrhs, cudaStream_t s) {
  if (coarse.n_cells == 0) return cudaSuccess;
  const int nch = fine.ncomp * nrhs;
  if (fine.gc_active) {
#define NNMG_G(D, K) \
  if (fine.dim == D && coarse.k == K) return gc_restrict_dk<D, K, T>(fine, coarse, rf, rc, scratch, nch, s);
    NNMG_G(2, 1) NNMG_G(2, 2) NNMG_G(2, 3) NNMG_G(2, 4)
    NNMG_G(3, 1) NNMG_G(3, 2) NNMG_G(3, 3) NNMG_G(3, 4)
#undef NNMG_G
    return cudaErrorInvalidValue;
  }
  cudaError_t e = launch_restrict_points<T>(fine, coarse, rf, nullptr, scratch, nrhs, s);
  if (e != cudaSuccess) return e;
  return launch_restrict_gather<T>(coarse, scratch, rc, nch, s);
}

template <typename T>
cudaError_t launch_restrict_residual(const DevLevel& fine, const DevLevel& coarse, const T* f,
                                     T* t, T* r_tmp, T* rc, T* scratch, int nrhs, cudaStream_t s) {
  if (fine.gc_active || coarse.n_cells == 0) {
    cudaError_t e = launch_residual<T>(f, t, r_tmp, fine.rows, nrhs, s);
    if (e != cudaSuccess) return e;
    return launch_restrict<T>(fine, coarse, r_tmp, rc, scratch, nrhs, s);
  }
  cudaError_t e = launch_restrict_points<T>(fine, coarse, f, t, scratch, nrhs, s);
  if (e != cudaSuccess) return e;
  return launch_restrict_gather<T>(coarse, scratch, rc, fine.ncomp * nrhs, s);
}

template <typename TI, typename TO>
cudaError_t launch_coarse_solve(const DevLevel& L, const TI* r, TO* z, int nrhs, cudaStream_t s) {
  if (L.n_free_rows == 0) return cudaSuccess;
  const int n = L.n_free_rows;
  int npad = 1;
  while (npad < nrhs) npad *= 2;
  const int rows_per_block = kCoarseWarps * (32 / npad);
  const unsigned blocks = (unsigned)((n + rows_per_block - 1) / rows_per_block);
  // enough segments for ~4 blocks per SM, each segment at least one tile long
  int nseg = (int)std::min<int64_t>(kCoarseMaxSegments, std::max<int64_t>(1, (4 * 152) / blocks));
  nseg = std::max(1, std::min(nseg, (n + kCoarseTile - 1) / kCoarseTile));
  if (!L.coarse_partial) nseg = 1;
  cudaError_t e = launch_k(coarse_solve_kernel<TI, TO>, dim3(blocks, nseg), 32 * kCoarseWarps, 0, s,
                           L.coarse_inv, L.free_rows, n, r, z, nrhs, npad, L.coarse_partial);
  if (e != cudaSuccess || nseg == 1) return e;
  return launch_k(coarse_sum_kernel<TO>, (n * nrhs + 255) / 256, 256, 0, s, L.coarse_partial,
                  L.free_rows, n, nseg, z, nrhs);
}

template cudaError_t launch_prolongate_add<float>(const DevLevel&, const DevLevel&, const float*,
                                                  float*, int, cudaStream_t);
template cudaError_t launch_prolongate_add<double>(const DevLevel&, const DevLevel&, const double*,
                                                   double*, int, cudaStream_t);
template cudaError_t launch_restrict<float>(const DevLevel&, const DevLevel&, const float*, float*,
                                            float*, int, cudaStream_t);
template cudaError_t launch_restrict<double>(const DevLevel&, const DevLevel&, const double*,
                                             double*, double*, int, cudaStream_t);
template cudaError_t launch_restrict_residual<float>(const DevLevel&, const DevLevel&, const float*,
                                                     float*, float*, float*, float*, int,
                                                     cudaStream_t);
template cudaError_t launch_restrict_residual<double>(const DevLevel&, const DevLevel&,
                                                      const double*, double*, double*, double*,
                                                      double*, int, cudaStream_t);
template cudaError_t launch_coarse_solve<float, float>(const DevLevel&, const float*, float*, int,
                                                      cudaStream_t);
template cudaError_t launch_coarse_solve<double, double>(const DevLevel&, const double*, double*,
                                                         int, cudaStream_t);

}  // namespace nnmg
