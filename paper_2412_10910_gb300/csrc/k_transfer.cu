// Non-nested transfer kernels and the coarsest-level solve.
//
// The kernels are instantiated on the coarse level's degree (the basis they
// evaluate); the fine level may have another degree (polynomial coarsening on
// one mesh, Sec. 2 "Coarse grid solvers").
//
// Prolongation x_f += P x_c (Sec. 2, P[i,j] = phi^{l-1}_j(x_i); Sec. 3.2,
// Eqs. local_evaluation, tensor_product_evaluation): the fine points are
// grouped by coarse cell; at each point the 1D Lagrange bases are evaluated at
// its reference coordinates and contracted with the cell's (k+1)^d coarse
// values direction by direction.  Every fine point belongs to exactly one
// coarse cell, so its output is written once (no atomics).
//
// Restriction r_c = P^T r_f (Sec. 2, Eq. residual2) in two deterministic
// phases: (1) per coarse cell, phi_j(xi_p) r_f(p) is summed over the cell's
// fine points into a cell-local buffer, in an order fixed by the code;
// (2) per coarse node, the buffer entries of the cells that share it are
// summed in ascending (cell, local) order.  No atomics: results are bitwise
// reproducible.
//
// Two forms of each: a register form (a warp per coarse cell, the cell's
// values or buffer entries of one channel held by each thread; up to 128 FP32
// or 64 FP64 values per cell) and a shared-memory form for FP64 3D degree 4
// (a block per coarse cell stages the cell's values for all channels).
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "nnmg_internal.h"

namespace nnmg {
namespace {

template <int N, typename T>
__device__ __forceinline__ void lagrange1d(const Basis1D<T>& B, T xi, T* L) {
#pragma unroll
  for (int l = 0; l < N; ++l) {
    T v = B.gl_scale[l];
#pragma unroll
    for (int m = 0; m < N; ++m)
      if (m != l) v *= xi - B.gl[m];
    L[l] = v;
  }
}

// Shared-memory forms (FP64 3D degree 4, whose 125 coarse values or buffer
// entries per channel do not fit a thread's registers).  Fine points of a coarse cell
// are handled in chunks of kChunk: a cell holds
// about (refinement ratio)^d points, ~66-68 for the 2.1-2.2x coarsening of the
// configurations, so one chunk (one gather round, two barriers) covers it.
constexpr int kChunk = 128;

template <int D, int K, typename T>
__global__ void prolong_kernel(const int32_t* __restrict__ coarse_cell_nodes,
                               const T* __restrict__ xc, T* __restrict__ xf,
                               const int32_t* __restrict__ cell_pt_start,
                               const int32_t* __restrict__ pt_node, const T* __restrict__ pt_xi,
                               int nch, Basis1D<T> B) {
  constexpr int N = K + 1;
  constexpr int NL = D == 2 ? N * N : N * N * N;
  extern __shared__ unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);  // [NL][nch]
  const int64_t c = blockIdx.x;
  for (int e = threadIdx.x; e < NL * nch; e += blockDim.x) {
    const int j = e / nch, ch = e - j * nch;
    const int node = coarse_cell_nodes[c * NL + j];
    su[e] = node >= 0 ? xc[(int64_t)node * nch + ch] : T(0);
  }
  __syncthreads();
  __shared__ T sL[kChunk][D][N];      // 1D bases of the chunk's points
  const int p0 = cell_pt_start[c], p1 = cell_pt_start[c + 1];
  for (int q0 = p0; q0 < p1; q0 += kChunk) {
    const int np = min(kChunk, p1 - q0);
    __syncthreads();                   // the previous chunk's readers are done
    for (int t = threadIdx.x; t < np * D; t += blockDim.x) {
      const int pp = t / D, d = t - pp * D;
      lagrange1d<N, T>(B, pt_xi[(int64_t)(q0 + pp) * D + d], sL[pp][d]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < np * nch; e += blockDim.x) {
      const int pl = e / nch, ch = e - pl * nch;
      const T(&L)[D][N] = sL[pl];
      T val = 0;
      if constexpr (D == 2) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          T s = 0;
#pragma unroll
          for (int i = 0; i < N; ++i) s += L[0][i] * su[(i + N * j) * nch + ch];
          val += L[1][j] * s;
        }
      } else {
#pragma unroll
        for (int l = 0; l < N; ++l) {
          T s1 = 0;
#pragma unroll
          for (int j = 0; j < N; ++j) {
            T s0 = 0;
#pragma unroll
            for (int i = 0; i < N; ++i) s0 += L[0][i] * su[(i + N * j + N * N * l) * nch + ch];
            s1 += L[1][j] * s0;
          }
          val += L[2][l] * s1;
        }
      }
      T* o = xf + (int64_t)pt_node[q0 + pl] * nch + ch;
      *o += val;
    }
  }
}

// Phase one: thread (m_0[, m_1], channel) owns the N buffer entries that
// differ in the last local index; per fine point it forms
// phi_{m_0}(xi_0) [phi_{m_1}(xi_1)] r_p once and adds it times each of the
// last direction's N basis values (points in stored order: deterministic).
template <int D, int K, typename T>
__global__ void restrict1_kernel(const T* __restrict__ rf, T* __restrict__ buf,
                                 const int32_t* __restrict__ cell_pt_start,
                                 const int32_t* __restrict__ pt_node, const T* __restrict__ pt_xi,
                                 int nch, Basis1D<T> B) {
  constexpr int N = K + 1;
  constexpr int NL = D == 2 ? N * N : N * N * N;
  constexpr int NP = NL / N;                   // (m_0[, m_1]) combinations
  __shared__ T sL[kChunk][D][N];
  extern __shared__ unsigned char smem_raw[];
  T* sr = reinterpret_cast<T*>(smem_raw);  // [kChunk][nch]
  const int64_t c = blockIdx.x;
  const int e = blockIdx.y * blockDim.x + threadIdx.x;
  const bool valid = e < NP * nch;
  const int jp = valid ? e / nch : 0;
  const int ch = valid ? e - jp * nch : 0;
  const int m0 = jp % N, m1 = jp / N;          // m1 unused in 2D
  const int p0 = cell_pt_start[c], p1 = cell_pt_start[c + 1];
  T acc[N];
#pragma unroll
  for (int m = 0; m < N; ++m) acc[m] = 0;
  for (int q0 = p0; q0 < p1; q0 += kChunk) {
    const int np = min(kChunk, p1 - q0);
    for (int t = threadIdx.x; t < np * D; t += blockDim.x) {
      const int pp = t / D, d = t - pp * D;
      lagrange1d<N, T>(B, pt_xi[(int64_t)(q0 + pp) * D + d], sL[pp][d]);
    }
    for (int t = threadIdx.x; t < np * nch; t += blockDim.x) {
      const int pp = t / nch, cc = t - pp * nch;
      sr[t] = rf[(int64_t)pt_node[q0 + pp] * nch + cc];
    }
    __syncthreads();
    if (valid) {
      for (int pp = 0; pp < np; ++pp) {
        T w = sL[pp][0][m0] * sr[pp * nch + ch];
        if constexpr (D == 3) w *= sL[pp][1][m1];
#pragma unroll
        for (int m = 0; m < N; ++m) acc[m] += w * sL[pp][D - 1][m];
      }
    }
    __syncthreads();
  }
  if (valid) {
#pragma unroll
    for (int m = 0; m < N; ++m) buf[(c * NL + jp + NP * m) * nch + ch] = acc[m];
  }
}

// Register forms (FP32: every degree; FP64: 2D k <= 4, 3D k <= 3).
// A coarse cell's fine points are split into P parts (points p0 + part,
// p0 + part + P, ...), and each (cell, part, channel) goes to one thread.
// With nch <= 32 channels a cell gets one warp: lane = part * nch + channel,
// P = 32 / nch, and the 32 % nch remaining lanes idle; the parts of a cell are
// combined by shuffles.  With more channels a cell gets nch threads (P = 1).
// No shared memory and no barriers: a thread's loads are the cell's data and,
// per point, its reference point, fine node and one value.
// Register forms serve cells of at most kRegWords 4-byte words of values per
// channel: 128 FP32 values (3D Q4) or 64 FP64 values.
constexpr int kRegWords = 128;
template <typename T>
constexpr bool reg_transfer(int nl) {
  return nl * (int)(sizeof(T) / 4) <= kRegWords;
}
constexpr int kPts = 4;   // points per batch of loads
__host__ __device__ inline int transfer_lanes(int nch) { return nch <= 32 ? 32 : nch; }

// Prolongation: the thread keeps its channel's NL coarse values in registers
// and evaluates the coarse polynomial at each of its points (the contraction
// order of the shared-memory form).
template <int D, int K, typename T>
__device__ __forceinline__ void prolong_reg_body(
    const int32_t* __restrict__ coarse_cell_nodes, const T* __restrict__ xc, T* __restrict__ xf,
    const int32_t* __restrict__ cell_pt_start, const int32_t* __restrict__ pt_node,
    const T* __restrict__ pt_xi, int64_t n_cells, int nch, const Basis1D<T>& B) {
  constexpr int N = K + 1;
  constexpr int NL = D == 2 ? N * N : N * N * N;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lanes = transfer_lanes(nch), P = lanes / nch;
  const int64_t c = e / lanes;
  const int r = (int)(e - c * lanes), part = r / nch, ch = r - part * nch;
  if (c >= n_cells || part >= P) return;
  const int32_t* cn = coarse_cell_nodes + c * NL;
  T u[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    const int node = cn[j];
    u[j] = node >= 0 ? xc[(int64_t)node * nch + ch] : T(0);
  }
  const int p0 = cell_pt_start[c], p1 = cell_pt_start[c + 1];
  // kPts points at a time: their indices, reference points and old fine
  // values are loaded before any of them is evaluated
  for (int p = p0 + part; p < p1; p += kPts * P) {
    int node[kPts];
    T xi[kPts][D], old[kPts];
#pragma unroll
    for (int b = 0; b < kPts; ++b) {
      const int q = p + b * P;
      node[b] = q < p1 ? pt_node[q] : -1;
#pragma unroll
      for (int d = 0; d < D; ++d) xi[b][d] = q < p1 ? pt_xi[(int64_t)q * D + d] : T(0);
    }
#pragma unroll
    for (int b = 0; b < kPts; ++b) old[b] = node[b] >= 0 ? xf[(int64_t)node[b] * nch + ch] : T(0);
#pragma unroll
    for (int b = 0; b < kPts; ++b) {
      if (node[b] < 0) continue;
      T L[D][N];
#pragma unroll
      for (int d = 0; d < D; ++d) lagrange1d<N, T>(B, xi[b][d], L[d]);
      T val = 0;
      if constexpr (D == 2) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          T s = 0;
#pragma unroll
          for (int i = 0; i < N; ++i) s += L[0][i] * u[i + N * j];
          val += L[1][j] * s;
        }
      } else {
#pragma unroll
        for (int l = 0; l < N; ++l) {
          T s1 = 0;
#pragma unroll
          for (int j = 0; j < N; ++j) {
            T s0 = 0;
#pragma unroll
            for (int i = 0; i < N; ++i) s0 += L[0][i] * u[i + N * j + N * N * l];
            s1 += L[1][j] * s0;
          }
          val += L[2][l] * s1;
        }
      }
      xf[(int64_t)node[b] * nch + ch] = old[b] + val;
    }
  }
}

template <int D, int K, typename T>
__global__ void __launch_bounds__(128) prolong_reg_kernel(
    const int32_t* __restrict__ coarse_cell_nodes, const T* __restrict__ xc, T* __restrict__ xf,
    const int32_t* __restrict__ cell_pt_start, const int32_t* __restrict__ pt_node,
    const T* __restrict__ pt_xi, int64_t n_cells, int nch, Basis1D<T> B) {
  prolong_reg_body<D, K, T>(coarse_cell_nodes, xc, xf, cell_pt_start, pt_node, pt_xi, n_cells,
                            nch, B);
}

// The 3D Q4 FP32 instance bounded to three blocks per SM: 168 registers
// instead of 217 (125 coarse values per thread), 12 warps per SM instead of
// 8; 0.197 vs 0.233 ms on config 3's finest pair.  (The same bound on the
// smaller instances slows them: config 2's Q2, 0.058 vs 0.053 ms.)
template <int D, int K, typename T>
__global__ void __launch_bounds__(128, 3) prolong_reg_kernel_3b(
    const int32_t* __restrict__ coarse_cell_nodes, const T* __restrict__ xc, T* __restrict__ xf,
    const int32_t* __restrict__ cell_pt_start, const int32_t* __restrict__ pt_node,
    const T* __restrict__ pt_xi, int64_t n_cells, int nch, Basis1D<T> B) {
  prolong_reg_body<D, K, T>(coarse_cell_nodes, xc, xf, cell_pt_start, pt_node, pt_xi, n_cells,
                            nch, B);
}

// Restriction phase one: the thread accumulates phi_m(xi_p) r_p over its
// points for all NL local nodes m of the cell (sum-factorized outer product,
// points in stored order); the P parts of a cell are then added by shuffles
// in a fixed tree, so the result does not depend on scheduling.
template <int D, int K, typename T>
__global__ void __launch_bounds__(128) restrict1_reg_kernel(
    const T* __restrict__ rf, T* __restrict__ buf, const int32_t* __restrict__ cell_pt_start,
    const int32_t* __restrict__ pt_node, const T* __restrict__ pt_xi, int64_t n_cells, int nch,
    Basis1D<T> B) {
  constexpr int N = K + 1;
  constexpr int NL = D == 2 ? N * N : N * N * N;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lanes = transfer_lanes(nch), P = lanes / nch;
  const int64_t c = e / lanes;
  // with nch <= 32 a warp is exactly one cell: whole warps leave here together
  if (c >= n_cells) return;
  const int r = (int)(e - c * lanes), part = r / nch, ch = r - part * nch;
  const bool idle = part >= P;                 // one of the 32 % nch spare lanes
  T acc[NL];
#pragma unroll
  for (int m = 0; m < NL; ++m) acc[m] = 0;
  const int p0 = cell_pt_start[c], p1 = cell_pt_start[c + 1];
  for (int p = idle ? p1 : p0 + part; p < p1; p += kPts * P) {
    int node[kPts];
    T xi[kPts][D], rv[kPts];
#pragma unroll
    for (int b = 0; b < kPts; ++b) {
      const int q = p + b * P;
      node[b] = q < p1 ? pt_node[q] : -1;
#pragma unroll
      for (int d = 0; d < D; ++d) xi[b][d] = q < p1 ? pt_xi[(int64_t)q * D + d] : T(0);
    }
#pragma unroll
    for (int b = 0; b < kPts; ++b) rv[b] = node[b] >= 0 ? rf[(int64_t)node[b] * nch + ch] : T(0);
#pragma unroll
    for (int b = 0; b < kPts; ++b) {
      if (node[b] < 0) continue;
      T L[D][N];
#pragma unroll
      for (int d = 0; d < D; ++d) lagrange1d<N, T>(B, xi[b][d], L[d]);
      if constexpr (D == 2) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const T w = L[1][j] * rv[b];
#pragma unroll
          for (int i = 0; i < N; ++i) acc[i + N * j] += L[0][i] * w;
        }
      } else {
#pragma unroll
        for (int l = 0; l < N; ++l) {
          const T w2 = L[2][l] * rv[b];
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const T w1 = L[1][j] * w2;
#pragma unroll
            for (int i = 0; i < N; ++i) acc[i + N * j + N * N * l] += L[0][i] * w1;
          }
        }
      }
    }
  }
  if (P > 1) {
    // fixed tree over the parts: at step h, part q < h adds part q + h
    int h = 1;
    while (2 * h < P) h *= 2;
    for (; h >= 1; h >>= 1) {
      const bool take = part < h && part + h < P;
#pragma unroll
      for (int m = 0; m < NL; ++m) {
        const T o = __shfl_down_sync(0xffffffffu, acc[m], h * nch);
        if (take) acc[m] += o;
      }
    }
  }
  if (part == 0) {
#pragma unroll
    for (int m = 0; m < NL; ++m) buf[(c * NL + m) * nch + ch] = acc[m];
  }
}

// Phase two: per (coarse node, channel) the buffer entries of the cells that
// share the node, added in ascending list order (kBatch list entries and
// their values loaded at a time, so the loads of one node overlap).
constexpr int kBatch = 8;
template <typename T>
__global__ void restrict2_kernel(const T* __restrict__ buf, const int32_t* __restrict__ gstart,
                                 const int32_t* __restrict__ gpos, T* __restrict__ rc,
                                 int64_t n_nodes, int nch) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_nodes * nch) return;
  const int64_t node = e / nch;
  const int ch = (int)(e - node * nch);
  const int k0 = gstart[node], k1 = gstart[node + 1];
  T s = 0;
  for (int k = k0; k < k1; k += kBatch) {
    int pos[kBatch];
    T v[kBatch];
#pragma unroll
    for (int i = 0; i < kBatch; ++i) pos[i] = k + i < k1 ? gpos[k + i] : -1;
#pragma unroll
    for (int i = 0; i < kBatch; ++i) v[i] = pos[i] >= 0 ? buf[(int64_t)pos[i] * nch + ch] : T(0);
#pragma unroll
    for (int i = 0; i < kBatch; ++i)
      if (k + i < k1) s += v[i];
  }
  rc[e] = s;
}

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
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * nrhs) return;
  const int i = e / nrhs, q = e - i * nrhs;
  double s = 0.0;
  for (int g = 0; g < nseg; ++g) s += partial[((int64_t)g * n + i) * kMaxRhs + q];
  z[(int64_t)rows[i] * nrhs + q] = (TO)s;
}

template <typename T>
void basis_of(int k, Basis1D<T>* b);
template <>
void basis_of<double>(int k, Basis1D<double>* b) {
  Basis1D<float> f;
  make_basis(k, b, &f);
}
template <>
void basis_of<float>(int k, Basis1D<float>* b) {
  Basis1D<double> d;
  make_basis(k, &d, b);
}

template <typename T>
const T* xi_of(const DevLevel& L);
template <>
const double* xi_of<double>(const DevLevel& L) { return L.pt_xi64; }
template <>
const float* xi_of<float>(const DevLevel& L) { return L.pt_xi32; }


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

template <int D, int K, typename T>
cudaError_t prolong_dk(const DevLevel& f, const DevLevel& c, const T* xc, T* xf, int nch,
                       cudaStream_t s) {
  Basis1D<T> B;
  basis_of<T>(K, &B);
  constexpr int N = K + 1;
  constexpr int NL = D == 2 ? N * N : N * N * N;
  const size_t smem = (size_t)NL * nch * sizeof(T);
  if constexpr (reg_transfer<T>(NL)) {
    const int64_t threads = c.n_cells * transfer_lanes(nch);
    const unsigned blocks = (unsigned)((threads + 127) / 128);
    if constexpr (D == 3 && K == 4 && std::is_same<T, float>::value)
      prolong_reg_kernel_3b<D, K, T><<<blocks, 128, 0, s>>>(
          c.cell_nodes, xc, xf, f.cell_pt_start, f.pt_node, xi_of<T>(f), c.n_cells, nch, B);
    else
      prolong_reg_kernel<D, K, T><<<blocks, 128, 0, s>>>(
          c.cell_nodes, xc, xf, f.cell_pt_start, f.pt_node, xi_of<T>(f), c.n_cells, nch, B);
  } else {
    auto kern = prolong_kernel<D, K, T>;
    static size_t granted = 0;
    cudaError_t e = allow_smem(kern, smem, &granted);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)c.n_cells, 128, smem, s>>>(c.cell_nodes, xc, xf, f.cell_pt_start, f.pt_node,
                                                xi_of<T>(f), nch, B);
  }
  return cudaGetLastError();
}

template <int D, int K, typename T>
cudaError_t restrict_dk(const DevLevel& f, const DevLevel& c, const T* rf, T* rc, T* scratch,
                        int nch, cudaStream_t s) {
  Basis1D<T> B;
  basis_of<T>(K, &B);
  constexpr int N = K + 1;
  constexpr int NL = D == 2 ? N * N : N * N * N;
  const size_t smem = (size_t)kChunk * nch * sizeof(T);
  cudaError_t e;
  if constexpr (reg_transfer<T>(NL)) {
    const int64_t threads = c.n_cells * transfer_lanes(nch);
    restrict1_reg_kernel<D, K, T><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(
        rf, scratch, f.cell_pt_start, f.pt_node, xi_of<T>(f), c.n_cells, nch, B);
  } else {
    auto kern = restrict1_kernel<D, K, T>;
    static size_t granted = 0;
    e = allow_smem(kern, smem, &granted);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)c.n_cells, (unsigned)((NL / N * nch + 127) / 128));
    kern<<<grid, 128, smem, s>>>(rf, scratch, f.cell_pt_start, f.pt_node, xi_of<T>(f), nch, B);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t n = c.n_nodes * nch;
  restrict2_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(scratch, c.gather_start,
                                                                  c.gather_pos, rc, c.n_nodes, nch);
  return cudaGetLastError();
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
  const int64_t n = c.n_nodes * nch;
  restrict2_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(scratch, c.gather_start,
                                                                  c.gather_pos, rc, c.n_nodes, nch);
  return cudaGetLastError();
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
#define NNMG_P(D, K) \
  if (fine.dim == D && coarse.k == K) return prolong_dk<D, K, T>(fine, coarse, xc, xf, nch, s);
  NNMG_P(2, 1) NNMG_P(2, 2) NNMG_P(2, 3) NNMG_P(2, 4)
  NNMG_P(3, 1) NNMG_P(3, 2) NNMG_P(3, 3) NNMG_P(3, 4)
#undef NNMG_P
  return cudaErrorInvalidValue;
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
#define NNMG_R(D, K) \
  if (fine.dim == D && coarse.k == K) return restrict_dk<D, K, T>(fine, coarse, rf, rc, scratch, nch, s);
  NNMG_R(2, 1) NNMG_R(2, 2) NNMG_R(2, 3) NNMG_R(2, 4)
  NNMG_R(3, 1) NNMG_R(3, 2) NNMG_R(3, 3) NNMG_R(3, 4)
#undef NNMG_R
  return cudaErrorInvalidValue;
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
  coarse_solve_kernel<TI, TO><<<dim3(blocks, nseg), 32 * kCoarseWarps, 0, s>>>(
      L.coarse_inv, L.free_rows, n, r, z, nrhs, npad, L.coarse_partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || nseg == 1) return e;
  coarse_sum_kernel<TO><<<(n * nrhs + 255) / 256, 256, 0, s>>>(L.coarse_partial, L.free_rows, n,
                                                               nseg, z, nrhs);
  return cudaGetLastError();
}

template cudaError_t launch_prolongate_add<float>(const DevLevel&, const DevLevel&, const float*,
                                                  float*, int, cudaStream_t);
template cudaError_t launch_prolongate_add<double>(const DevLevel&, const DevLevel&, const double*,
                                                   double*, int, cudaStream_t);
template cudaError_t launch_restrict<float>(const DevLevel&, const DevLevel&, const float*, float*,
                                            float*, int, cudaStream_t);
template cudaError_t launch_restrict<double>(const DevLevel&, const DevLevel&, const double*,
                                             double*, double*, int, cudaStream_t);
template cudaError_t launch_coarse_solve<float, float>(const DevLevel&, const float*, float*, int,
                                                      cudaStream_t);
template cudaError_t launch_coarse_solve<double, double>(const DevLevel&, const double*, double*,
                                                         int, cudaStream_t);

}  // namespace nnmg
