// Non-nested restriction r_c = P^T r_f (Sec. 2, Eq. residual2), the exact
// transpose of the point-evaluation prolongation, in two deterministic phases
// without atomics (results are bitwise reproducible):
//
// (1) per coarse cell K and local node (i, j, l): the sum over the fine points
//     p located in K, in their stored order, of L_i(xi_0) L_j(xi_1) L_l(xi_2)
//     r_f(p), written to a cell-local buffer [cell][(k+1)^d][channels];
// (2) per coarse node, the buffer entries of the cells that share it, added in
//     ascending (cell, local node) order.
//
// Phase one, thread mapping: a warp owns one coarse cell and walks its points
// 128 at a time.  Each lane first stages four points: it evaluates a point's
// d (k+1) Lagrange factors and loads the point's residual row into the warp's
// shared memory (so a point's factors are computed and its row is read once).
// Then every lane that owns an output line (i[, j]) and a group of CH channels
// adds, per staged point, the point's contribution to its k+1 entries
// l = 0..k (sum factorization of the outer product), in packed FP32 or FP64
// arithmetic.  When a cell needs fewer than 32 owners, the staged points are
// split into parts over the spare lanes, and the parts are added at the end by
// a fixed shuffle tree; with more than 32 owners the lanes take them in rounds.
#include <algorithm>

#include "transfer_pts.h"

namespace nnmg {
namespace {

using namespace pts;

// A warp stages kLanePts points per lane, 32 kLanePts points per round (all
// loads of a lane's points issued before their values are used).
#ifndef NNMG_RESTRICT_LANE_PTS
#define NNMG_RESTRICT_LANE_PTS 2
#endif
#ifndef NNMG_RESTRICT_MIN_BLOCKS
#define NNMG_RESTRICT_MIN_BLOCKS 6
#endif
constexpr int kLanePts = NNMG_RESTRICT_LANE_PTS;
constexpr int kStagePts = 32 * kLanePts;

// F = 1: a lane owns a line (i[, j]) and its k+1 entries along the last
// direction; F = 2 (3D): a lane owns a plane i and its (k+1)^2 entries (j, l),
// which shares each loaded factor and product over more entries (3D Q3/Q4).
template <int D, int K, typename T, int CH, int F>
__global__ void __launch_bounds__(128, F == 1 ? NNMG_RESTRICT_MIN_BLOCKS : 4) restrict_pts_kernel(
    const T* __restrict__ rf, T* __restrict__ tres, T* __restrict__ buf,
    const int32_t* __restrict__ cell_pt_start, const int32_t* __restrict__ pt_node,
    const T* __restrict__ pt_xi, int64_t n_cells, int nch, Basis1D<T> B) {
  pdl_trigger();
  pdl_wait();
  constexpr int N = K + 1;
  constexpr int NL = ipow<N, D>::value;
  constexpr int NO = F == 1 ? NL / N : N;         // owned lines (i[, j]) or planes (i)
  constexpr int NA = F == 1 ? N : N * N;          // entries per owner: l, or (j, l)
  using P = typename Pack<T, CH>::type;
  constexpr int NP = Pack<T, CH>::n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= n_cells) return;                       // whole warps leave (no block barrier below)
  // per warp: residual rows [kStagePts][nch], then Lagrange factors [kStagePts][D][N]
  T* sr = reinterpret_cast<T*>(smem_raw) + (size_t)warp * kStagePts * (nch + D * N);
  T* sL = sr + kStagePts * nch;
  const int ng = nch / CH;
  const int owners = NO * ng;
  const int parts = owners <= 32 ? 32 / owners : 1;
  const int rounds = (owners + 31) / 32;
  const int p0 = cell_pt_start[c], p1 = cell_pt_start[c + 1];
  for (int rd = 0; rd < rounds; ++rd) {
    const int part = owners <= 32 ? lane / owners : 0;
    const int own = owners <= 32 ? lane - part * owners : rd * 32 + lane;
    const bool active = owners <= 32 ? part < parts : own < owners;
    const int g = active ? own % ng : 0;
    const int line = active ? own / ng : 0;
    const int i0 = line % N, j0 = line / N;        // j0 unused in 2D and for F = 2
    P acc[NA][NP];
#pragma unroll
    for (int m = 0; m < NA; ++m)
#pragma unroll
      for (int q = 0; q < NP; ++q) acc[m][q] = pzero(P());
    for (int q0 = p0; q0 < p1; q0 += kStagePts) {
      const int nq = min(kStagePts, p1 - q0);
      __syncwarp();                               // the previous round has been read
      {
        int node[kLanePts];
        T xi[kLanePts][D];
#pragma unroll
        for (int b = 0; b < kLanePts; ++b) {
          const int pl = lane + 32 * b;
          node[b] = pl < nq ? pt_node[q0 + pl] : -1;
#pragma unroll
          for (int d = 0; d < D; ++d) xi[b][d] = pl < nq ? pt_xi[(int64_t)(q0 + pl) * D + d] : T(0);
        }
        for (int gg = 0; gg < ng; ++gg) {
          P v[kLanePts][NP];
#pragma unroll
          for (int b = 0; b < kLanePts; ++b)
            if (node[b] >= 0) load_group<T, CH>(rf + (int64_t)node[b] * nch + gg * CH, v[b]);
          if (tres) {
            // fused residual: r = f - t at the point's row
            P tv[kLanePts][NP];
#pragma unroll
            for (int b = 0; b < kLanePts; ++b)
              if (node[b] >= 0) load_group<T, CH>(tres + (int64_t)node[b] * nch + gg * CH, tv[b]);
#pragma unroll
            for (int b = 0; b < kLanePts; ++b)
              if (node[b] >= 0)
#pragma unroll
                for (int q = 0; q < NP; ++q) v[b][q] = psub(v[b][q], tv[b][q]);
          }
#pragma unroll
          for (int b = 0; b < kLanePts; ++b)
            if (node[b] >= 0) store_group<T, CH>(sr + (lane + 32 * b) * nch + gg * CH, v[b]);
        }
        if (tres && rd == rounds - 1) {
          // t = 0 at the points' rows, in the last round over the points (every
          // free fine node is exactly one point, so all of t is reset; earlier
          // rounds still read t).  The stores follow all of this round's
          // loads: a global store between them would serialise their round
          // trips (the rows of t may alias as far as the compiler knows).
          P zero[NP];
#pragma unroll
          for (int q = 0; q < NP; ++q) zero[q] = pzero(P());
          for (int gg = 0; gg < ng; ++gg)
#pragma unroll
            for (int b = 0; b < kLanePts; ++b)
              if (node[b] >= 0) store_group<T, CH>(tres + (int64_t)node[b] * nch + gg * CH, zero);
        }
#pragma unroll
        for (int b = 0; b < kLanePts; ++b)
          if (node[b] >= 0)
#pragma unroll
            for (int d = 0; d < D; ++d) lagrange<N, T>(B, xi[b][d], sL + ((lane + 32 * b) * D + d) * N);
      }
      __syncwarp();
      if (active) {
        for (int pp = part; pp < nq; pp += parts) {
          const T* Lp = sL + pp * D * N;
          P rv[NP];
          load_group<T, CH>(sr + pp * nch + g * CH, rv);
          if constexpr (F == 1) {
            T w = Lp[i0];
            if constexpr (D == 3) w *= Lp[N + j0];
#pragma unroll
            for (int q = 0; q < NP; ++q) rv[q] = pmul(pbcast(w, P()), rv[q]);
#pragma unroll
            for (int m = 0; m < N; ++m) {
              const P lm = pbcast(Lp[(D - 1) * N + m], P());
#pragma unroll
              for (int q = 0; q < NP; ++q) acc[m][q] = pfma(lm, rv[q], acc[m][q]);
            }
          } else {
            const P w = pbcast(Lp[i0], P());
#pragma unroll
            for (int q = 0; q < NP; ++q) rv[q] = pmul(w, rv[q]);
            T l2[N];
#pragma unroll
            for (int m = 0; m < N; ++m) l2[m] = Lp[2 * N + m];
#pragma unroll
            for (int j = 0; j < N; ++j) {
              const P lj = pbcast(Lp[N + j], P());
              P u[NP];
#pragma unroll
              for (int q = 0; q < NP; ++q) u[q] = pmul(lj, rv[q]);
#pragma unroll
              for (int m = 0; m < N; ++m)
#pragma unroll
                for (int q = 0; q < NP; ++q) acc[j + N * m][q] = pfma(pbcast(l2[m], P()), u[q], acc[j + N * m][q]);
            }
          }
        }
      }
    }
    if (parts > 1) {
      // fixed tree over the parts: at step h, part q < h adds part q + h
      int h = 1;
      while (2 * h < parts) h *= 2;
      for (; h >= 1; h >>= 1) {
        const bool take = active && part < h && part + h < parts;
#pragma unroll
        for (int m = 0; m < NA; ++m)
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            const P o = pshfl_down(acc[m][q], h * owners);
            if (take) acc[m][q] = padd(acc[m][q], o);
          }
      }
    }
    if (active && part == 0) {
#pragma unroll
      for (int m = 0; m < NA; ++m)      // local node line + NO m: (i[, j], l) or (i, j + N l)
        store_group<T, CH>(buf + ((c * NL + line + NO * m) * nch + g * CH), acc[m]);
    }
  }
}

// Phase two: per (coarse node, channel) the buffer entries of the cells that
// share the node, added in ascending list order (kBatch list entries and
// their values loaded at a time, so the loads of one node overlap).
constexpr int kBatch = 8;
template <typename T>
__global__ void restrict_gather_kernel(const T* __restrict__ buf, const int32_t* __restrict__ gstart,
                                       const int32_t* __restrict__ gpos, T* __restrict__ rc,
                                       int64_t n_nodes, int nch) {
  pdl_trigger();
  pdl_wait();
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

template <int D, int K, typename T, int CH, int F>
cudaError_t restrict_run(const DevLevel& f, const DevLevel& c, const T* rf, T* tres, T* buf,
                         int nch, cudaStream_t s) {
  constexpr int N = K + 1;
  Basis1D<T> B;
  basis_for<T>(K, &B);
  // warps (cells) per block: up to four, fewer when a warp's staging area is large
  const size_t per_warp = (size_t)kStagePts * (nch + D * N) * sizeof(T);
  const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, (96 * 1024) / per_warp));
  const size_t smem = warps * per_warp;
  auto kern = restrict_pts_kernel<D, K, T, CH, F>;
  static size_t granted = 48 * 1024;
  if (smem > granted) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    granted = smem;
  }
  const unsigned blocks = (unsigned)((c.n_cells + warps - 1) / warps);
  return launch_k(kern, blocks, 32 * warps, smem, s, rf, tres, buf, f.cell_pt_start, f.pt_node,
                  xi_for<T>(f), c.n_cells, nch, B);
}

template <int D, int K, typename T>
cudaError_t restrict_dk(const DevLevel& f, const DevLevel& c, const T* rf, T* tres, T* buf,
                        int nch, cudaStream_t s) {
  // the buffer rows are allocated by cudaMalloc or the no-allocation array
  // (256-byte aligned): only the fine vector's alignment can vary.  3D Q3/Q4
  // own planes (F = 2) of up to 25 entries, with at most 2 FP32 channels (a
  // float pair) or 1 FP64 channel per lane.
  constexpr bool planes = D == 3 && K >= 3;
  int ch = channel_group<T>(nch, rf, tres ? (const void*)tres : (const void*)buf);
  if (planes) ch = std::min(ch, sizeof(T) == 4 ? 2 : 1);
  if constexpr (planes) {
    switch (ch) {
      case 2:
        if constexpr (sizeof(T) == 4) return restrict_run<D, K, T, 2, 2>(f, c, rf, tres, buf, nch, s);
        break;
      default: return restrict_run<D, K, T, 1, 2>(f, c, rf, tres, buf, nch, s);
    }
  } else {
    switch (ch) {
      case 8:
        if constexpr (sizeof(T) == 4) return restrict_run<D, K, T, 8, 1>(f, c, rf, tres, buf, nch, s);
        break;
      case 4: return restrict_run<D, K, T, 4, 1>(f, c, rf, tres, buf, nch, s);
      case 2: return restrict_run<D, K, T, 2, 1>(f, c, rf, tres, buf, nch, s);
      default: return restrict_run<D, K, T, 1, 1>(f, c, rf, tres, buf, nch, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// Phase one of r_c = P^T r_f into the cell-local buffer `scratch`
// [coarse cells][(k+1)^d][ncomp * nrhs] (instantiated on the coarse degree).
// With tres != nullptr the residual is fused: r_f = rf - tres at the located
// points, and tres is reset to zero there.
template <typename T>
cudaError_t launch_restrict_points(const DevLevel& fine, const DevLevel& coarse, const T* rf,
                                   T* tres, T* scratch, int nrhs, cudaStream_t s) {
  if (coarse.n_cells == 0) return cudaSuccess;
  const int nch = fine.ncomp * nrhs;
#define NNMG_R(D, K) \
  if (fine.dim == D && coarse.k == K) return restrict_dk<D, K, T>(fine, coarse, rf, tres, scratch, nch, s);
  NNMG_R(2, 1) NNMG_R(2, 2) NNMG_R(2, 3) NNMG_R(2, 4)
  NNMG_R(3, 1) NNMG_R(3, 2) NNMG_R(3, 3) NNMG_R(3, 4)
#undef NNMG_R
  return cudaErrorInvalidValue;
}

// Phase two: r_c from the cell-local buffer (also used by the nested transfer).
template <typename T>
cudaError_t launch_restrict_gather(const DevLevel& coarse, const T* scratch, T* rc, int nch,
                                   cudaStream_t s) {
  const int64_t n = coarse.n_nodes * nch;
  if (n == 0) return cudaSuccess;
  return launch_k(restrict_gather_kernel<T>, (unsigned)((n + 255) / 256), 256, 0, s, scratch,
                  coarse.gather_start, coarse.gather_pos, rc, coarse.n_nodes, nch);
}

template cudaError_t launch_restrict_points<float>(const DevLevel&, const DevLevel&, const float*,
                                                   float*, float*, int, cudaStream_t);
template cudaError_t launch_restrict_points<double>(const DevLevel&, const DevLevel&,
                                                    const double*, double*, double*, int,
                                                    cudaStream_t);
template cudaError_t launch_restrict_gather<float>(const DevLevel&, const float*, float*, int,
                                                   cudaStream_t);
template cudaError_t launch_restrict_gather<double>(const DevLevel&, const double*, double*, int,
                                                    cudaStream_t);

}  // namespace nnmg
