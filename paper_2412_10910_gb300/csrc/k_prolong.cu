// Non-nested prolongation x_f += P x_c (Sec. 2: P[i, j] = phi^{l-1}_j(x_i);
// Sec. 3.2, Eqs. local_evaluation and tensor_product_evaluation).
//
// Every free fine node i was located at setup in one coarse cell K with
// reference point xi (Sec. 3.1); the points are stored sorted by coarse cell.
// At a point, the coarse field is u_K(xi) = sum_{i,j,l} L_i(xi_0) L_j(xi_1)
// L_l(xi_2) u_K[i, j, l], contracted one direction at a time (sum
// factorization: (k+1)^3 + (k+1)^2 + (k+1) multiply-adds per channel).
//
// Thread mapping: a block owns G consecutive coarse cells.  It first copies
// their (k+1)^d coarse values for all channels into shared memory (gathered
// once through the coarse cell-to-node map), then walks the points of those
// cells with one thread per (point, group of CH channels): the thread
// evaluates the point's d (k+1) Lagrange factors once, contracts them with the
// staged values of its channel group in packed FP32 (or FP64) arithmetic and
// adds the result to the fine row with vector accesses.  Every fine point
// belongs to exactly one coarse cell, so each output is written by one thread
// (no atomics).
#include <algorithm>

#include "transfer_pts.h"

namespace nnmg {
namespace {

using namespace pts;

constexpr int kProlongThreads = 256;
constexpr size_t kProlongSmemCap = 24 * 1024;   // staged values per block, keeps 8 blocks/SM

// Contract the staged coarse values u (one channel group, rows nch apart) with
// the point's 1D factors L: val = sum_l L2[l] sum_j L1[j] sum_i L0[i] u[i,j,l].
template <int D, int N, typename T, int CH>
__device__ __forceinline__ void evaluate(const T* u, const T (&L)[D][N], int nch,
                                         typename Pack<T, CH>::type* val) {
  using P = typename Pack<T, CH>::type;
  constexpr int NP = Pack<T, CH>::n;
  if constexpr (D == 2) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      P s[NP];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        P uv[NP];
        load_group<T, CH>(u + (i + N * j) * nch, uv);
#pragma unroll
        for (int q = 0; q < NP; ++q)
          s[q] = i == 0 ? pmul(pbcast(L[0][0], P()), uv[q]) : pfma(pbcast(L[0][i], P()), uv[q], s[q]);
      }
#pragma unroll
      for (int q = 0; q < NP; ++q)
        val[q] = j == 0 ? pmul(pbcast(L[1][0], P()), s[q]) : pfma(pbcast(L[1][j], P()), s[q], val[q]);
    }
  } else {
#pragma unroll
    for (int l = 0; l < N; ++l) {
      P s1[NP];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        P s0[NP];
#pragma unroll
        for (int i = 0; i < N; ++i) {
          P uv[NP];
          load_group<T, CH>(u + (i + N * j + N * N * l) * nch, uv);
#pragma unroll
          for (int q = 0; q < NP; ++q)
            s0[q] = i == 0 ? pmul(pbcast(L[0][0], P()), uv[q]) : pfma(pbcast(L[0][i], P()), uv[q], s0[q]);
        }
#pragma unroll
        for (int q = 0; q < NP; ++q)
          s1[q] = j == 0 ? pmul(pbcast(L[1][0], P()), s0[q]) : pfma(pbcast(L[1][j], P()), s0[q], s1[q]);
      }
#pragma unroll
      for (int q = 0; q < NP; ++q)
        val[q] = l == 0 ? pmul(pbcast(L[2][0], P()), s1[q]) : pfma(pbcast(L[2][l], P()), s1[q], val[q]);
    }
  }
}

// Loads in flight per thread: the staging copies kStage (cell node, channel
// group) units at a time and the point pass kBatch points at a time, every
// load of a batch issued before any of its values is used (the index -> value
// chains of the batch overlap instead of following one another).
constexpr int kStage = 4;
#ifndef NNMG_PROLONG_BATCH
#define NNMG_PROLONG_BATCH 2
#endif
#ifndef NNMG_PROLONG_MIN_BLOCKS
#define NNMG_PROLONG_MIN_BLOCKS 3
#endif
constexpr int kBatch = NNMG_PROLONG_BATCH;
// channel-group items per coarse cell from which a warp per cell pays
#ifndef NNMG_PROLONG_CELL_ITEMS
#define NNMG_PROLONG_CELL_ITEMS 128
#endif
constexpr double kCellItems = NNMG_PROLONG_CELL_ITEMS;

template <int D, int K, typename T, int CH>
__global__ void __launch_bounds__(kProlongThreads, NNMG_PROLONG_MIN_BLOCKS) prolong_pts_kernel(
    const int32_t* __restrict__ ccell_nodes, const T* __restrict__ xc, T* __restrict__ xf,
    const int32_t* __restrict__ cell_pt_start, const int32_t* __restrict__ pt_node,
    const int32_t* __restrict__ pt_cell, const T* __restrict__ pt_xi, int64_t n_cells, int nch,
    int G, Basis1D<T> B) {
  pdl_trigger();
  pdl_wait();
  constexpr int N = K + 1;
  constexpr int NL = ipow<N, D>::value;
  using P = typename Pack<T, CH>::type;
  constexpr int NP = Pack<T, CH>::n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);  // [G][NL][nch]
  const int64_t c0 = (int64_t)blockIdx.x * G;
  const int cg = (int)(n_cells - c0 < G ? n_cells - c0 : G);
  const int ng = nch / CH;
  // stage the coarse values of the block's cells (zero at Dirichlet nodes)
  const int units = cg * NL * ng;
  for (int e0 = threadIdx.x; e0 < units; e0 += kStage * blockDim.x) {
    int node[kStage];
#pragma unroll
    for (int b = 0; b < kStage; ++b) {
      const int e = e0 + b * blockDim.x;
      node[b] = e < units ? ccell_nodes[c0 * NL + e / ng] : -2;
    }
    P v[kStage][NP];
#pragma unroll
    for (int b = 0; b < kStage; ++b) {
      const int e = e0 + b * blockDim.x;
      if (node[b] >= 0) {
        load_group<T, CH>(xc + (int64_t)node[b] * nch + (e % ng) * CH, v[b]);
      } else {
#pragma unroll
        for (int q = 0; q < NP; ++q) v[b][q] = pzero(P());
      }
    }
#pragma unroll
    for (int b = 0; b < kStage; ++b) {
      const int e = e0 + b * blockDim.x;
      if (node[b] != -2) store_group<T, CH>(su + (e / ng) * nch + (e % ng) * CH, v[b]);
    }
  }
  __syncthreads();
  const int p0 = cell_pt_start[c0], p1 = cell_pt_start[c0 + cg];
  const int items = (p1 - p0) * ng;
  for (int it0 = threadIdx.x; it0 < items; it0 += kBatch * blockDim.x) {
    int node[kBatch], off[kBatch];
    T xi[kBatch][D];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int it = it0 + b * blockDim.x;
      node[b] = -1;
      off[b] = 0;
      if (it < items) {
        const int pl = it / ng, g = it - pl * ng;
        const int p = p0 + pl;
        node[b] = pt_node[p];
        off[b] = (pt_cell[p] - (int)c0) * NL * nch + g * CH;
#pragma unroll
        for (int d = 0; d < D; ++d) xi[b][d] = pt_xi[(int64_t)p * D + d];
        node[b] = node[b] * ng + g;        // row group index: node * ng + g
      }
    }
    P old[kBatch][NP];
#pragma unroll
    for (int b = 0; b < kBatch; ++b)
      if (node[b] >= 0) load_group<T, CH>(xf + (int64_t)node[b] * CH, old[b]);
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      if (node[b] < 0) continue;
      T L[D][N];
#pragma unroll
      for (int d = 0; d < D; ++d) lagrange<N, T>(B, xi[b][d], L[d]);
      P val[NP];
      evaluate<D, N, T, CH>(su + off[b], L, nch, val);
#pragma unroll
      for (int q = 0; q < NP; ++q) old[b][q] = padd(old[b][q], val[q]);
      store_group<T, CH>(xf + (int64_t)node[b] * CH, old[b]);
    }
  }
}

// The same with one warp per coarse cell, for cells holding many points (3D
// Q3/Q4 coarse cells hold hundreds): every lane of a warp reads the same
// cell's staged values, so a shared-memory read is one broadcast instead of
// one access per cell that the warp's points straddle.
template <int D, int K, typename T, int CH>
__global__ void __launch_bounds__(128) prolong_cell_kernel(
    const int32_t* __restrict__ ccell_nodes, const T* __restrict__ xc, T* __restrict__ xf,
    const int32_t* __restrict__ cell_pt_start, const int32_t* __restrict__ pt_node,
    const T* __restrict__ pt_xi, int64_t n_cells, int nch, Basis1D<T> B) {
  pdl_trigger();
  pdl_wait();
  constexpr int N = K + 1;
  constexpr int NL = ipow<N, D>::value;
  using P = typename Pack<T, CH>::type;
  constexpr int NP = Pack<T, CH>::n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= n_cells) return;                       // whole warps leave (no block barrier below)
  T* su = reinterpret_cast<T*>(smem_raw) + (size_t)warp * NL * nch;   // [NL][nch]
  const int ng = nch / CH;
  const int units = NL * ng;
  for (int e0 = lane; e0 < units; e0 += kStage * 32) {
    int node[kStage];
#pragma unroll
    for (int b = 0; b < kStage; ++b) {
      const int e = e0 + b * 32;
      node[b] = e < units ? ccell_nodes[c * NL + e / ng] : -2;
    }
    P v[kStage][NP];
#pragma unroll
    for (int b = 0; b < kStage; ++b) {
      const int e = e0 + b * 32;
      if (node[b] >= 0) {
        load_group<T, CH>(xc + (int64_t)node[b] * nch + (e % ng) * CH, v[b]);
      } else {
#pragma unroll
        for (int q = 0; q < NP; ++q) v[b][q] = pzero(P());
      }
    }
#pragma unroll
    for (int b = 0; b < kStage; ++b) {
      const int e = e0 + b * 32;
      if (node[b] != -2) store_group<T, CH>(su + (e / ng) * nch + (e % ng) * CH, v[b]);
    }
  }
  __syncwarp();
  const int p0 = cell_pt_start[c], p1 = cell_pt_start[c + 1];
  const int items = (p1 - p0) * ng;
  for (int it0 = lane; it0 < items; it0 += kBatch * 32) {
    int node[kBatch], off[kBatch];
    T xi[kBatch][D];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int it = it0 + b * 32;
      node[b] = -1;
      off[b] = 0;
      if (it < items) {
        const int pl = it / ng, g = it - pl * ng;
        const int p = p0 + pl;
        off[b] = g * CH;
#pragma unroll
        for (int d = 0; d < D; ++d) xi[b][d] = pt_xi[(int64_t)p * D + d];
        node[b] = pt_node[p] * ng + g;      // row group index
      }
    }
    P old[kBatch][NP];
#pragma unroll
    for (int b = 0; b < kBatch; ++b)
      if (node[b] >= 0) load_group<T, CH>(xf + (int64_t)node[b] * CH, old[b]);
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      if (node[b] < 0) continue;
      T L[D][N];
#pragma unroll
      for (int d = 0; d < D; ++d) lagrange<N, T>(B, xi[b][d], L[d]);
      P val[NP];
      evaluate<D, N, T, CH>(su + off[b], L, nch, val);
#pragma unroll
      for (int q = 0; q < NP; ++q) old[b][q] = padd(old[b][q], val[q]);
      store_group<T, CH>(xf + (int64_t)node[b] * CH, old[b]);
    }
  }
}

template <typename T>
void basis_for(int k, Basis1D<T>* b);
template <>
void basis_for<double>(int k, Basis1D<double>* b) {
  Basis1D<float> f;
  make_basis(k, b, &f);
}
template <>
void basis_for<float>(int k, Basis1D<float>* b) {
  Basis1D<double> d;
  make_basis(k, &d, b);
}

template <typename T>
const T* xi_for(const DevLevel& L);
template <>
const double* xi_for<double>(const DevLevel& L) { return L.pt_xi64; }
template <>
const float* xi_for<float>(const DevLevel& L) { return L.pt_xi32; }

template <int D, int K, typename T, int CH>
cudaError_t prolong_run(const DevLevel& f, const DevLevel& c, const T* xc, T* xf, int nch,
                        cudaStream_t s) {
  constexpr int NL = ipow<K + 1, D>::value;
  Basis1D<T> B;
  basis_for<T>(K, &B);
  const size_t per_cell = (size_t)NL * nch * sizeof(T);
  const double pts_per_cell = (double)f.n_pts / (double)std::max<int64_t>(c.n_cells, 1);
  const double items_per_cell = std::max(1.0, pts_per_cell * (nch / CH));
  if (items_per_cell >= kCellItems) {
    // a warp per cell: up to four cells per block, fewer when a cell's values are large
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, (96 * 1024) / per_cell));
    const size_t smem = warps * per_cell;
    auto kern = prolong_cell_kernel<D, K, T, CH>;
    static size_t granted_cell = 48 * 1024;
    if (smem > granted_cell) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      granted_cell = smem;
    }
    const unsigned blocks = (unsigned)((c.n_cells + warps - 1) / warps);
    return launch_k(kern, blocks, 32 * warps, smem, s, c.cell_nodes, xc, xf, f.cell_pt_start,
                    f.pt_node, xi_for<T>(f), c.n_cells, nch, B);
  }
  // cells per block: about as many points as one batched pass of the block
  // takes, and no more cells than the staging budget allows (at least one)
  int G = (int)(kBatch * kProlongThreads / items_per_cell);
  G = std::max(1, std::min<int>(G, (int)(kProlongSmemCap / per_cell)));
  G = (int)std::min<int64_t>(G, c.n_cells);
  const size_t smem = (size_t)G * per_cell;
  auto kern = prolong_pts_kernel<D, K, T, CH>;
  static size_t granted = 48 * 1024;
  if (smem > granted) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    granted = smem;
  }
  const unsigned blocks = (unsigned)((c.n_cells + G - 1) / G);
  return launch_k(kern, blocks, kProlongThreads, smem, s, c.cell_nodes, xc, xf, f.cell_pt_start,
                  f.pt_node, f.pt_cell, xi_for<T>(f), c.n_cells, nch, G, B);
}

template <int D, int K, typename T>
cudaError_t prolong_dk(const DevLevel& f, const DevLevel& c, const T* xc, T* xf, int nch,
                       cudaStream_t s) {
  switch (channel_group<T>(nch, xc, xf)) {
    case 8:
      if constexpr (sizeof(T) == 4) return prolong_run<D, K, T, 8>(f, c, xc, xf, nch, s);
      break;
    case 4: return prolong_run<D, K, T, 4>(f, c, xc, xf, nch, s);
    case 2: return prolong_run<D, K, T, 2>(f, c, xc, xf, nch, s);
    default: return prolong_run<D, K, T, 1>(f, c, xc, xf, nch, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// x_f += P x_c for the non-nested transfer from level `coarse` to `fine`
// (instantiated on the coarse level's degree).
template <typename T>
cudaError_t launch_prolongate_points(const DevLevel& fine, const DevLevel& coarse, const T* xc,
                                     T* xf, int nrhs, cudaStream_t s) {
  if (coarse.n_cells == 0 || fine.n_pts == 0) return cudaSuccess;
  const int nch = fine.ncomp * nrhs;
#define NNMG_P(D, K) \
  if (fine.dim == D && coarse.k == K) return prolong_dk<D, K, T>(fine, coarse, xc, xf, nch, s);
  NNMG_P(2, 1) NNMG_P(2, 2) NNMG_P(2, 3) NNMG_P(2, 4)
  NNMG_P(3, 1) NNMG_P(3, 2) NNMG_P(3, 3) NNMG_P(3, 4)
#undef NNMG_P
  return cudaErrorInvalidValue;
}

template cudaError_t launch_prolongate_points<float>(const DevLevel&, const DevLevel&, const float*,
                                                     float*, int, cudaStream_t);
template cudaError_t launch_prolongate_points<double>(const DevLevel&, const DevLevel&,
                                                      const double*, double*, int, cudaStream_t);

}  // namespace nnmg
