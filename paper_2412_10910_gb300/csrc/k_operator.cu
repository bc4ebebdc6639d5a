// Matrix-free cell operator y = A_l x with sum factorization (Sec. 3.2,
// Eq. tensor_product_evaluation for tensor point sets; Sec. 2 operator A_l).
//
// Per cell: gather the (k+1)^d nodal values, interpolate to the (k+1)^d
// Gauss points (one 1D sweep per direction), take reference derivatives by
// collocation on the Gauss points, apply the stored metric terms (Poisson:
// G = |det J| w J^-1 J^-T; elasticity: sigma = lambda tr(eps) I + 2 mu eps,
// Sec. 4.4), run the transposed sweeps and scatter-add into y.
//
// Thread mapping: a "unit" is one (cell, right-hand side) pair; a block holds
// U units (right-hand side fastest, then cells) and (k+1)^(d-1) lines per
// unit; thread t has unit t % U and line t / U, so a warp reads one node's
// contiguous right-hand sides and neighbouring cells.  A thread keeps one
// line of k+1 values in registers per sweep; sweeps along other directions go
// through shared memory laid out [array][point][unit] (bank-conflict free).
// In the paired FP32 form (T = f2) a unit is a (cell, pair of right-hand
// sides) and every value a float pair.  The register-resident kernels further
// down keep a whole cell of one unit in a thread.  Dirichlet nodes carry index
// -1: read as 0, never written.  y must be zero on entry (scatter is atomic).
#include <algorithm>
#include <type_traits>

#include "dword.h"
#include "nnmg_internal.h"

namespace nnmg {
namespace {

// Arithmetic type T and the type of vectors in memory: float and double work
// in place; the double-word type dw reads and writes FP64 vectors.
template <typename T>
struct io_of {
  using type = T;
};
template <>
struct io_of<dw> {
  using type = double;
};
__device__ __forceinline__ float to_arith(float v, float) { return v; }
__device__ __forceinline__ double to_arith(double v, double) { return v; }
__device__ __forceinline__ dw to_arith(double v, dw) { return dw_from_double(v); }
__device__ __forceinline__ void add_out(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void add_out(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void add_out(double* p, dw v) { atomicAdd(p, dw_to_double(v)); }

// Two right-hand sides of one cell packed in a float pair: every operation is
// one Blackwell packed FP32 instruction (add, multiply, fused multiply-add on
// both halves, each rounded as its scalar FP32 counterpart).
struct f2 {
  float2 v;
  __host__ __device__ f2() : v(make_float2(0.f, 0.f)) {}
  __host__ __device__ f2(float a) : v(make_float2(a, a)) {}
  __host__ __device__ f2(float2 a) : v(a) {}
};
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }

// s + m u: one FMA for float and double (contracted), one packed FMA for f2,
// the double-word product and sum for dw.
template <typename T>
__device__ __forceinline__ T mac(T s, T m, T u) {
  return s + m * u;
}
__device__ __forceinline__ f2 mac(f2 s, f2 m, f2 u) { return f2(__ffma2_rn(m.v, u.v, s.v)); }

// The paired type reads and writes float pairs (two right-hand sides) and
// FP32 metric terms; the other types read metric terms of their own type.
template <>
struct io_of<f2> {
  using type = float2;
};
template <typename T>
struct metric_type {
  using type = T;
};
template <>
struct metric_type<f2> {
  using type = float;
};
__device__ __forceinline__ f2 to_arith(float2 v, f2) { return f2(v); }
__device__ __forceinline__ void add_out(float2* p, f2 v) { atomicAdd(p, v.v); }

// Metric rows are padded to NQP = NQ rounded up to a multiple of 4 entries, so
// every row of every cell starts on a 16-byte boundary; the register kernels
// load a row four (FP32) or two (FP64, double-word) quadrature points at a time.
__host__ __device__ constexpr int padded_nq(int nq) { return (nq + 3) / 4 * 4; }
template <typename T>
struct MetricVec {
  static constexpr int W = 16 / (int)sizeof(T);
};
__device__ __forceinline__ void load_metric(const float* p, float (&o)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  o[0] = a.x;
  o[1] = a.y;
  o[2] = a.z;
  o[3] = a.w;
}
__device__ __forceinline__ void load_metric(const float* p, float (&o)[2]) {
  const float2 a = *reinterpret_cast<const float2*>(p);
  o[0] = a.x;
  o[1] = a.y;
}
__device__ __forceinline__ void load_metric(const double* p, double (&o)[2]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  o[0] = a.x;
  o[1] = a.y;
}
__device__ __forceinline__ void load_metric(const dw* p, dw (&o)[2]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  o[0] = dw(a.x, a.y);
  o[1] = dw(a.z, a.w);
}

// The two 1D matrices of the sweeps: S interpolates from the Lobatto nodes to
// the Gauss points, Dg differentiates by collocation on the Gauss points.  For
// odd N the middle Gauss point is the middle Lobatto node (both are 1/2), so
// S's middle row is the unit row and Dg's middle diagonal entry is zero (the
// derivative there of the Lagrange polynomial of a symmetric point set at its
// own, central node).  The host stores these entries exactly; the sweeps skip
// them, which removes N of the N^2 products of every S sweep and one of every
// Dg sweep.  A chain of products starts with its first product, so no type
// (the double-word one in particular) pays for an addition of zero.
enum { kInterp = 0, kDeriv = 1 };

template <int N, int KIND>
__host__ __device__ constexpr bool unit_row(int q) {
  return KIND == kInterp && N % 2 == 1 && q == N / 2;
}
template <int N, int KIND>
__host__ __device__ constexpr bool zero_entry(int q, int l) {
  return N % 2 == 1 && (KIND == kInterp ? (q == N / 2 && l != N / 2)
                                        : (q == N / 2 && l == N / 2));
}

// out = M in
template <int N, int KIND, typename T>
__device__ __forceinline__ void apply(const T (&M)[kMaxN][kMaxN], const T* in, T* out) {
#pragma unroll
  for (int q = 0; q < N; ++q) {
    if (unit_row<N, KIND>(q)) {
      out[q] = in[q];
      continue;
    }
    T s;
    bool first = true;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      if (zero_entry<N, KIND>(q, l)) continue;
      s = first ? M[q][l] * in[l] : mac(s, M[q][l], in[l]);
      first = false;
    }
    out[q] = s;
  }
}

// out = M^T in (add = false) or out += M^T in (add = true)
template <int N, int KIND, bool ADD = false, typename T>
__device__ __forceinline__ void apply_t(const T (&M)[kMaxN][kMaxN], const T* in, T* out) {
#pragma unroll
  for (int l = 0; l < N; ++l) {
    T s;
    bool first = true;
    if (ADD) {
      s = out[l];
      first = false;
    }
    if (unit_row<N, KIND>(l)) {   // the unit entry M[l][l] = 1
      s = first ? in[l] : s + in[l];
      first = false;
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
      if (zero_entry<N, KIND>(q, l) || unit_row<N, KIND>(q)) continue;
      s = first ? M[q][l] * in[q] : mac(s, M[q][l], in[q]);
      first = false;
    }
    out[l] = s;
  }
}

// Stress flux at one quadrature point for elasticity: g[c][a] = d u_c / d xi_a
// in, F[c][a] out.  K = sqrt(|det J| w) J^-1, H = g K (scaled physical
// gradient), sigma = lambda tr(H) I + mu (H + H^T), F = sigma K^T.
template <typename T>
__device__ __forceinline__ void elastic_flux(const T (&g)[3][3], const T (&K)[3][3], T lambda,
                                             T mu, T (&F)[3][3]) {
  T H[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b) H[c][b] = g[c][0] * K[0][b] + g[c][1] * K[1][b] + g[c][2] * K[2][b];
  const T tr = lambda * (H[0][0] + H[1][1] + H[2][2]);
  T s[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b) s[c][b] = mu * (H[c][b] + H[b][c]) + (c == b ? tr : T(0));
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int a = 0; a < 3; ++a) F[c][a] = s[c][0] * K[a][0] + s[c][1] * K[a][1] + s[c][2] * K[a][2];
}

template <int K, typename T, int NC>
__device__ __forceinline__ void op3d_body(const int32_t* __restrict__ cell_nodes,
                                          const typename metric_type<T>::type* __restrict__ metric,
                                          const typename io_of<T>::type* __restrict__ x,
                                          typename io_of<T>::type* __restrict__ y, int64_t n_cells,
                                          int nrhs, int U, const Basis1D<T>& B, T lambda, T mu) {
  pdl_trigger();
  pdl_wait();
  constexpr int N = K + 1, N2 = N * N, NQ = N2 * N, NQP = padded_nq(NQ);
  constexpr int NM = NC == 1 ? 6 : 9;
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int unit = threadIdx.x % U;
  const int line = threadIdx.x / U;
  const int a = line % N, b = line / N;
  const int rhs = unit % nrhs;
  const int64_t cell = (int64_t)blockIdx.x * (U / nrhs) + unit / nrhs;
  const bool act = cell < n_cells;
  // shared arrays: for component c: A = 3c, Gx = 3c+1, Gy = 3c+2
  auto S = [&](int arr, int idx) -> T& { return sm[(arr * NQ + idx) * U + unit]; };
  const int rs = NC * nrhs;  // stride between node rows of one right-hand side

  int dof[N];
  // P0 + P1: gather the z-line (i=a, j=b) and interpolate along z in registers
#pragma unroll
  for (int l = 0; l < N; ++l) dof[l] = act ? cell_nodes[cell * NQ + a + N * b + N2 * l] : -1;
  const typename metric_type<T>::type* mc = metric + (act ? cell : 0) * NM * NQP;
  // Poisson: fetch the metric terms of this thread's quadrature column now, so
  // that their latency overlaps the first sweeps (used in P5)
  T Gp[NC == 1 ? 6 : 1][N];
  if constexpr (NC == 1) {
#pragma unroll
    for (int q = 0; q < N; ++q)
#pragma unroll
      for (int m = 0; m < 6; ++m) Gp[m][q] = act ? T(mc[m * NQP + a + N * b + N2 * q]) : T(0);
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T u[N], v[N];
#pragma unroll
    for (int l = 0; l < N; ++l)
      u[l] = dof[l] >= 0 ? to_arith(x[(int64_t)dof[l] * rs + c * nrhs + rhs], T()) : T(0);
    apply<N, kInterp>(B.S, u, v);
#pragma unroll
    for (int q = 0; q < N; ++q) S(3 * c, a + N * b + N2 * q) = v[q];
  }
  __syncthreads();
  // P2: interpolate along y, line (i=a, z=b)
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T u[N], v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) u[j] = S(3 * c, a + N * j + N2 * b);
    apply<N, kInterp>(B.S, u, v);
#pragma unroll
    for (int q = 0; q < N; ++q) S(3 * c, a + N * q + N2 * b) = v[q];
  }
  __syncthreads();
  // P3: interpolate along x and take the x derivative, line (y=a, z=b)
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T u[N], v[N], g[N];
#pragma unroll
    for (int i = 0; i < N; ++i) u[i] = S(3 * c, i + N * a + N2 * b);
    apply<N, kInterp>(B.S, u, v);
    apply<N, kDeriv>(B.Dg, v, g);
#pragma unroll
    for (int q = 0; q < N; ++q) {
      S(3 * c, q + N * a + N2 * b) = v[q];
      S(3 * c + 1, q + N * a + N2 * b) = g[q];
    }
  }
  __syncthreads();
  // P4: y derivative, line (x=a, z=b)
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T u[N], g[N];
#pragma unroll
    for (int p = 0; p < N; ++p) u[p] = S(3 * c, a + N * p + N2 * b);
    apply<N, kDeriv>(B.Dg, u, g);
#pragma unroll
    for (int q = 0; q < N; ++q) S(3 * c + 2, a + N * q + N2 * b) = g[q];
  }
  __syncthreads();
  // P5: z derivative, physics at the quadrature points of column (a, b),
  // transposed z derivative
  {
    T gz[NC][N];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T u[N];
#pragma unroll
      for (int p = 0; p < N; ++p) u[p] = S(3 * c, a + N * b + N2 * p);
      apply<N, kDeriv>(B.Dg, u, gz[c]);
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
      const int idx = a + N * b + N2 * q;
      if constexpr (NC == 1) {
        const T gx = S(1, idx), gy = S(2, idx), g3 = gz[0][q];
        T G[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) G[m] = Gp[m][q];
        if constexpr (std::is_same<T, f2>::value) {
          S(1, idx) = mac(mac(G[0] * gx, G[1], gy), G[2], g3);
          S(2, idx) = mac(mac(G[1] * gx, G[3], gy), G[4], g3);
          gz[0][q] = mac(mac(G[2] * gx, G[4], gy), G[5], g3);
        } else {
          S(1, idx) = G[0] * gx + G[1] * gy + G[2] * g3;
          S(2, idx) = G[1] * gx + G[3] * gy + G[4] * g3;
          gz[0][q] = G[2] * gx + G[4] * gy + G[5] * g3;
        }
      } else {
        T g[3][3], Km[3][3], F[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          g[c][0] = S(3 * c + 1, idx);
          g[c][1] = S(3 * c + 2, idx);
          g[c][2] = gz[c][q];
        }
#pragma unroll
        for (int m = 0; m < 9; ++m) Km[m / 3][m % 3] = act ? T(mc[m * NQP + idx]) : T(0);
        elastic_flux(g, Km, lambda, mu, F);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          S(3 * c + 1, idx) = F[c][0];
          S(3 * c + 2, idx) = F[c][1];
          gz[c][q] = F[c][2];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T w[N];
      apply_t<N, kDeriv>(B.Dg, gz[c], w);
#pragma unroll
      for (int p = 0; p < N; ++p) S(3 * c, a + N * b + N2 * p) = w[p];
    }
  }
  __syncthreads();
  // P6: add the transposed y derivative, line (x=a, z=b)
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T f[N], w[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      f[q] = S(3 * c + 2, a + N * q + N2 * b);
      w[q] = S(3 * c, a + N * q + N2 * b);
    }
    apply_t<N, kDeriv, true>(B.Dg, f, w);
#pragma unroll
    for (int p = 0; p < N; ++p) S(3 * c, a + N * p + N2 * b) = w[p];
  }
  __syncthreads();
  // P7: add the transposed x derivative and integrate along x, line (y=a, z=b)
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T f[N], w[N], o[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      f[q] = S(3 * c + 1, q + N * a + N2 * b);
      w[q] = S(3 * c, q + N * a + N2 * b);
    }
    apply_t<N, kDeriv, true>(B.Dg, f, w);
    apply_t<N, kInterp>(B.S, w, o);
#pragma unroll
    for (int i = 0; i < N; ++i) S(3 * c, i + N * a + N2 * b) = o[i];
  }
  __syncthreads();
  // P8: integrate along y, line (x=a, z=b)
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T f[N], o[N];
#pragma unroll
    for (int q = 0; q < N; ++q) f[q] = S(3 * c, a + N * q + N2 * b);
    apply_t<N, kInterp>(B.S, f, o);
#pragma unroll
    for (int j = 0; j < N; ++j) S(3 * c, a + N * j + N2 * b) = o[j];
  }
  __syncthreads();
  // P9: integrate along z and scatter, column (a, b)
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T f[N], o[N];
#pragma unroll
    for (int q = 0; q < N; ++q) f[q] = S(3 * c, a + N * b + N2 * q);
    apply_t<N, kInterp>(B.S, f, o);
#pragma unroll
    for (int l = 0; l < N; ++l)
      if (dof[l] >= 0) add_out(&y[(int64_t)dof[l] * rs + c * nrhs + rhs], o[l]);
  }
}

template <int K, typename T, int NC>
__global__ void op3d_kernel(const int32_t* __restrict__ cell_nodes,
                            const typename metric_type<T>::type* __restrict__ metric,
                            const typename io_of<T>::type* __restrict__ x,
                            typename io_of<T>::type* __restrict__ y, int64_t n_cells, int nrhs,
                            int U, Basis1D<T> B, T lambda, T mu) {
  op3d_body<K, T, NC>(cell_nodes, metric, x, y, n_cells, nrhs, U, B, lambda, mu);
}

// The same for FP64 3D Q4 Poisson, limited to 400-thread blocks, two per SM:
// at 72 registers (a few spilled) two blocks of 16 units share an SM and one
// block's barriers overlap the other's FP64 work (3.62 vs 3.84 ms on config
// 3's fine level, 4 RHS; the unbounded kernel takes 96 registers, one block).
template <int K, typename T, int NC>
__global__ void __launch_bounds__(400, 2) op3d_kernel_2b(
    const int32_t* __restrict__ cell_nodes, const typename metric_type<T>::type* __restrict__ metric,
    const typename io_of<T>::type* __restrict__ x, typename io_of<T>::type* __restrict__ y,
    int64_t n_cells, int nrhs, int U, Basis1D<T> B, T lambda, T mu) {
  op3d_body<K, T, NC>(cell_nodes, metric, x, y, n_cells, nrhs, U, B, lambda, mu);
}

// The paired FP32 Q4 form with blocks of at most 100 threads (4 (cell, pair)
// units), five per SM: 96 registers instead of 128 (four blocks of 4 warps)
// and 0.194 vs 0.205 ms on config 3's fine level (4 RHS).  Serves up to 4
// pairs of right-hand sides per cell (a block must hold a whole cell).
template <int K, typename T, int NC>
__global__ void __launch_bounds__(100, 5) op3d_kernel_f2b(
    const int32_t* __restrict__ cell_nodes, const typename metric_type<T>::type* __restrict__ metric,
    const typename io_of<T>::type* __restrict__ x, typename io_of<T>::type* __restrict__ y,
    int64_t n_cells, int nrhs, int U, Basis1D<T> B, T lambda, T mu) {
  op3d_body<K, T, NC>(cell_nodes, metric, x, y, n_cells, nrhs, U, B, lambda, mu);
}
constexpr int kF2bMaxPairs = 4;

// The kernel entry for (K, T, NC); `cols` = vector columns per node row in T
// units (right-hand sides, or pairs of them for f2).
template <int K, typename T, int NC>
auto op3d_kernel_for(int cols) {
  if constexpr (K == 4 && NC == 1 && std::is_same<T, double>::value) {
    return op3d_kernel_2b<K, T, NC>;
  } else if constexpr (K == 4 && NC == 1 && std::is_same<T, f2>::value) {
    return cols <= kF2bMaxPairs ? op3d_kernel_f2b<K, T, NC> : op3d_kernel<K, T, NC>;
  } else {
    (void)cols;
    return op3d_kernel<K, T, NC>;
  }
}

// 2D Poisson: one thread per x-column (i = a) or y-row.
template <int K, typename T>
__global__ void op2d_kernel(const int32_t* __restrict__ cell_nodes, const T* __restrict__ metric,
                            const typename io_of<T>::type* __restrict__ x,
                            typename io_of<T>::type* __restrict__ y, int64_t n_cells, int nrhs,
                            int U, Basis1D<T> B) {
  pdl_trigger();
  pdl_wait();
  constexpr int N = K + 1, NQ = N * N;
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int unit = threadIdx.x % U;
  const int a = threadIdx.x / U;
  const int rhs = unit % nrhs;
  const int64_t cell = (int64_t)blockIdx.x * (U / nrhs) + unit / nrhs;
  const bool act = cell < n_cells;
  auto S = [&](int arr, int idx) -> T& { return sm[(arr * NQ + idx) * U + unit]; };
  int dof[N];
  {
    T u[N], v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      dof[j] = act ? cell_nodes[cell * NQ + a + N * j] : -1;
      u[j] = dof[j] >= 0 ? to_arith(x[(int64_t)dof[j] * nrhs + rhs], T()) : T(0);
    }
    apply<N, kInterp>(B.S, u, v);
#pragma unroll
    for (int q = 0; q < N; ++q) S(0, a + N * q) = v[q];
  }
  __syncthreads();
  {  // x interpolation and derivative, row y = a
    T u[N], v[N], g[N];
#pragma unroll
    for (int i = 0; i < N; ++i) u[i] = S(0, i + N * a);
    apply<N, kInterp>(B.S, u, v);
    apply<N, kDeriv>(B.Dg, v, g);
#pragma unroll
    for (int q = 0; q < N; ++q) {
      S(0, q + N * a) = v[q];
      S(1, q + N * a) = g[q];
    }
  }
  __syncthreads();
  {  // y derivative, metric, transposed y derivative, column x = a
    T u[N], gy[N], w[N];
#pragma unroll
    for (int p = 0; p < N; ++p) u[p] = S(0, a + N * p);
    apply<N, kDeriv>(B.Dg, u, gy);
    constexpr int NQP = padded_nq(NQ);
    const T* mc = metric + (act ? cell : 0) * 3 * NQP;
#pragma unroll
    for (int q = 0; q < N; ++q) {
      const int idx = a + N * q;
      const T gx = S(1, idx);
      const T G0 = act ? mc[idx] : T(0), G1 = act ? mc[NQP + idx] : T(0),
              G2 = act ? mc[2 * NQP + idx] : T(0);
      S(1, idx) = G0 * gx + G1 * gy[q];
      gy[q] = G1 * gx + G2 * gy[q];
    }
    apply_t<N, kDeriv>(B.Dg, gy, w);
#pragma unroll
    for (int p = 0; p < N; ++p) S(0, a + N * p) = w[p];
  }
  __syncthreads();
  {  // transposed x derivative + x integration, row y = a
    T f[N], w[N], o[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      f[q] = S(1, q + N * a);
      w[q] = S(0, q + N * a);
    }
    apply_t<N, kDeriv, true>(B.Dg, f, w);
    apply_t<N, kInterp>(B.S, w, o);
#pragma unroll
    for (int i = 0; i < N; ++i) S(0, i + N * a) = o[i];
  }
  __syncthreads();
  {  // y integration and scatter, column x = a
    T f[N], o[N];
#pragma unroll
    for (int q = 0; q < N; ++q) f[q] = S(0, a + N * q);
    apply_t<N, kInterp>(B.S, f, o);
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (dof[j] >= 0) add_out(&y[(int64_t)dof[j] * nrhs + rhs], o[j]);
  }
}


// Register-resident variant for small cells (3D k <= 2, 2D k <= 4, Poisson):
// one thread per (cell, right-hand side) unit keeps all (k+1)^d values, the
// reference gradients and the fluxes in registers, so the sweeps need no
// shared memory and no barriers.  Consecutive threads are consecutive units
// (right-hand side fastest), so a warp's gathers of one local node cover
// whole 32-byte rows of right-hand sides.  In FP64 (and double-word) the
// 1/64-rate FP64 pipe bounds the kernel and the barrier-free schedule keeps
// it busy; 253 registers a thread still fit two 128-thread blocks per SM.
template <int D, int N, int KIND, bool TRANSPOSE, bool ADD = false, typename T>
__device__ __forceinline__ void sweep(const T (&M)[kMaxN][kMaxN], const T* f, T* v, int dir) {
  // v = M (or M^T) applied along direction dir to every line of the N^D
  // array f; with ADD the result is added to v instead (TRANSPOSE only)
  constexpr int NQ = D == 2 ? N * N : N * N * N;
  const int stride = dir == 0 ? 1 : (dir == 1 ? N : N * N);
#pragma unroll
  for (int base = 0; base < NQ; ++base) {
    const int coord = (base / stride) % N;
    if (coord != 0) continue;
    T in[N], out[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      in[i] = f[base + i * stride];
      if (ADD) out[i] = v[base + i * stride];
    }
    if constexpr (TRANSPOSE)
      apply_t<N, KIND, ADD>(M, in, out);
    else
      apply<N, KIND>(M, in, out);
#pragma unroll
    for (int i = 0; i < N; ++i) v[base + i * stride] = out[i];
  }
}

// y += A_K x on one (cell, right-hand side) unit (the body of the register
// kernel and of the persistent smoother's operator phase).
template <int D, int K, typename T>
__device__ __forceinline__ void op_reg_unit(const int32_t* __restrict__ cell_nodes,
                                            const T* __restrict__ metric,
                                            const typename io_of<T>::type* __restrict__ x,
                                            typename io_of<T>::type* __restrict__ y, int64_t cell,
                                            int rhs, int nrhs, const Basis1D<T>& B) {
  constexpr int N = K + 1;
  constexpr int NQ = D == 2 ? N * N : N * N * N;
  constexpr int NM = D == 2 ? 3 : 6;
  const int32_t* cn = cell_nodes + cell * NQ;
  T v[NQ], gx[NQ], gy[NQ];
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    const int dof = cn[i];
    v[i] = dof >= 0 ? to_arith(x[(int64_t)dof * nrhs + rhs], T()) : T(0);
  }
  // values at the Gauss points, then collocation derivatives
#pragma unroll
  for (int d = 0; d < D; ++d) sweep<D, N, kInterp, false>(B.S, v, v, d);
  sweep<D, N, kDeriv, false>(B.Dg, v, gx, 0);
  sweep<D, N, kDeriv, false>(B.Dg, v, gy, 1);
  if constexpr (D == 3) sweep<D, N, kDeriv, false>(B.Dg, v, v, 2);  // v now holds d/dz
  // metric terms: flux = G grad^ (FP32 rows loaded four quadrature points at a
  // time; the FP64-pipe-bound types load one, which keeps their registers)
  constexpr int NQP = padded_nq(NQ);
#ifndef NNMG_METRIC_VEC
#define NNMG_METRIC_VEC 2
#endif
  constexpr int W = std::is_same<T, float>::value ? NNMG_METRIC_VEC : 1;
  const T* mc = metric + cell * NM * NQP;
#pragma unroll
  for (int q0 = 0; q0 < NQ; q0 += W) {
    T G[NM][W];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      if constexpr (W > 1)
        load_metric(mc + m * NQP + q0, G[m]);
      else
        G[m][0] = mc[m * NQP + q0];
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const int q = q0 + w;
      if (q >= NQ) break;
      if constexpr (D == 3) {
        const T a = gx[q], b = gy[q], c = v[q];
        gx[q] = G[0][w] * a + G[1][w] * b + G[2][w] * c;
        gy[q] = G[1][w] * a + G[3][w] * b + G[4][w] * c;
        v[q] = G[2][w] * a + G[4][w] * b + G[5][w] * c;
      } else {
        const T a = gx[q], b = gy[q];
        gx[q] = G[0][w] * a + G[1][w] * b;
        gy[q] = G[1][w] * a + G[2][w] * b;
      }
    }
  }
  // w = Dx^T fx + Dy^T fy (+ Dz^T fz), then integrate with S^T
  if constexpr (D == 3) {
    sweep<D, N, kDeriv, true>(B.Dg, v, v, 2);
    sweep<D, N, kDeriv, true, true>(B.Dg, gy, v, 1);
    sweep<D, N, kDeriv, true, true>(B.Dg, gx, v, 0);
  } else {
    sweep<D, N, kDeriv, true>(B.Dg, gy, v, 1);
    sweep<D, N, kDeriv, true, true>(B.Dg, gx, v, 0);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) sweep<D, N, kInterp, true>(B.S, v, v, d);
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    const int dof = cn[i];
    if (dof >= 0) add_out(&y[(int64_t)dof * nrhs + rhs], v[i]);
  }
}

template <int D, int K, typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1) op_reg_kernel(
    const int32_t* __restrict__ cell_nodes,
                                                     const T* __restrict__ metric,
                                                     const typename io_of<T>::type* __restrict__ x,
                                                     typename io_of<T>::type* __restrict__ y,
                                                     int64_t n_cells, int nrhs, Basis1D<T> B) {
  pdl_trigger();
  pdl_wait();
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t cell = u / nrhs;
  if (cell >= n_cells) return;
  op_reg_unit<D, K, T>(cell_nodes, metric, x, y, cell, (int)(u - cell * nrhs), nrhs, B);
}

// ------------------------------------------------- operator + Chebyshev step
// One Chebyshev-Jacobi step (Sec. 4 smoother) in one launch without any wait:
// the register kernel adds t += A_K x for the block's cells; then the block
// counts, per cell and node, one finished cell on cnt[node].  A count that
// reaches valence[node] (the number of cells holding the node) means the
// node's row of A x is complete: the block lists the node and, after a
// barrier, applies the step to the listed rows, one (node, right-hand side)
// element per thread: d = cd d + cr D^-1 (f - t), x += d, t = 0, cnt = 0.
// x at a node changes only after every cell holding the node has gathered
// it.  Blocks hold whole cells (blockDim = cells per block x nrhs).
__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

template <int D, int K, typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1) op_cheb_kernel(
    const int32_t* __restrict__ cell_nodes, const T* __restrict__ metric, const T* __restrict__ f,
    T* __restrict__ t, const T* __restrict__ dinv, T* __restrict__ d, T* __restrict__ x,
    int32_t* __restrict__ cnt, const int32_t* __restrict__ valence, int64_t n_cells, int nrhs,
    Basis1D<T> B, T cd, T cr) {
  pdl_trigger();
  pdl_wait();
  constexpr int N = K + 1;
  constexpr int NQ = D == 2 ? N * N : N * N * N;
  __shared__ int32_t done[128 * NQ];   // nodes this block completes (at most its cell slots)
  __shared__ int n_done;
  const int cells_per_block = blockDim.x / nrhs;
  const int64_t c0 = (int64_t)blockIdx.x * cells_per_block;
  const int64_t cell = c0 + threadIdx.x / nrhs;
  if (threadIdx.x == 0) n_done = 0;
  if (cell < n_cells)
    op_reg_unit<D, K, T>(cell_nodes, metric, x, t, cell, (int)(threadIdx.x % nrhs), nrhs, B);
  // release: the block's additions (ordered before this thread by the
  // barrier) before this thread's counts; acquire: a node's counts before the
  // block's reads of its t.  Acquire-release fences, not the sequentially
  // consistent __threadfence().
  __syncthreads();
  fence_acq_rel_gpu();
  const int64_t nc = n_cells - c0 < cells_per_block ? n_cells - c0 : cells_per_block;
  for (int i = threadIdx.x; i < nc * NQ; i += blockDim.x) {
    const int dof = cell_nodes[c0 * NQ + i];
    if (dof >= 0 && atomicAdd(&cnt[dof], 1) == valence[dof] - 1) done[atomicAdd(&n_done, 1)] = dof;
  }
  fence_acq_rel_gpu();
  __syncthreads();
  fence_acq_rel_gpu();
  // the completed nodes' rows, one (node, right-hand side) element per thread
  const int ne = n_done * nrhs;
  for (int i = threadIdx.x; i < ne; i += blockDim.x) {
    const int64_t dof = done[i / nrhs];
    const int64_t e = dof * nrhs + i % nrhs;
    const T fe = f[e], te = __ldcg(&t[e]), de = d[e], xe = x[e], di = dinv[dof];
    const T dn = cd * de + cr * di * (fe - te);
    d[e] = dn;
    x[e] = xe + dn;
    t[e] = T(0);
    if (i % nrhs == 0) cnt[dof] = 0;
  }
}

// ------------------------------------------------------ persistent smoother
// One Chebyshev-Jacobi smoothing sweep (Sec. 4) in a single cooperative
// launch: the operator phase t = A x (the register kernel's cell body over a
// grid-stride range of units) and the vector phase d = cd d + cr D^-1 (f - t),
// x += d, t = 0 alternate, separated by grid-wide barriers.  Pre-smoothing
// starts from x = d = D^-1 f / theta and ends with t = A x (the residual's
// operator pass, read by the restriction); post-smoothing starts with an
// operator pass.  A barrier gives up after kBarrierSpins polls, sets *err and
// the kernel returns (with a cooperative launch every block is resident, so
// the limit is a guard, not a schedule).
constexpr unsigned kBarrierSpins = 1u << 26;   // with a 64 ns pause: a few seconds

__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    ok = 1;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);                       // the next barrier counts from zero
      __threadfence();
      atomicAdd(bar + 1, 1u);                    // release the other blocks
    } else {
      unsigned it = 0;
      while (*gen == g) {
        if (++it > kBarrierSpins) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        if (it > 4096) __nanosleep(64);        // poll at full rate first
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

constexpr int kSmootherThreads = 128;

template <int D, int K, typename T>
__global__ void __launch_bounds__(kSmootherThreads) cheb_smoother_kernel(
    const int32_t* __restrict__ cell_nodes, const T* __restrict__ metric, const T* __restrict__ f,
    T* __restrict__ t, const T* __restrict__ dinv, T* __restrict__ d, T* __restrict__ x,
    int64_t n_cells, int64_t rows, int nrhs, Basis1D<T> B, SmootherPlan P, unsigned* bar, int* err) {
  const int64_t units = n_cells * nrhs, n = rows * nrhs;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int kU = 4;                          // vector elements in flight per thread
  int j = 0;
  if (P.from_zero) {
    const T c = (T)P.c_init;
    for (int64_t e0 = t0; e0 < n; e0 += kU * stride) {
      T fe[kU], di[kU];
#pragma unroll
      for (int b = 0; b < kU; ++b) {
        const int64_t e = e0 + b * stride;
        fe[b] = e < n ? f[e] : T(0);
        di[b] = e < n ? dinv[e / nrhs] : T(0);
      }
#pragma unroll
      for (int b = 0; b < kU; ++b) {
        const int64_t e = e0 + b * stride;
        if (e < n) {
          const T v = c * di[b] * fe[b];
          d[e] = v;
          x[e] = v;
        }
      }
    }
    j = 1;
    if (!grid_barrier(bar, err)) return;
  }
  for (; j < P.steps; ++j) {
    for (int64_t u = t0; u < units; u += stride) {
      const int64_t cell = u / nrhs;
      op_reg_unit<D, K, T>(cell_nodes, metric, x, t, cell, (int)(u - cell * nrhs), nrhs, B);
    }
    if (!grid_barrier(bar, err)) return;
    const T cd = (T)P.cd[j], cr = (T)P.cr[j];
    for (int64_t e0 = t0; e0 < n; e0 += kU * stride) {
      T fe[kU], te[kU], de[kU], xe[kU], di[kU];
#pragma unroll
      for (int b = 0; b < kU; ++b) {
        const int64_t e = e0 + b * stride;
        const bool in = e < n;
        fe[b] = in ? f[e] : T(0);
        te[b] = in ? t[e] : T(0);
        de[b] = in ? d[e] : T(0);
        xe[b] = in ? x[e] : T(0);
        di[b] = in ? dinv[e / nrhs] : T(0);
      }
#pragma unroll
      for (int b = 0; b < kU; ++b) {
        const int64_t e = e0 + b * stride;
        if (e < n) {
          const T dn = cd * de[b] + cr * di[b] * (fe[b] - te[b]);
          d[e] = dn;
          x[e] = xe[b] + dn;
          t[e] = T(0);
        }
      }
    }
    if (j + 1 < P.steps || P.final_op) {
      if (!grid_barrier(bar, err)) return;
    }
  }
  if (P.final_op) {
    for (int64_t u = t0; u < units; u += stride) {
      const int64_t cell = u / nrhs;
      op_reg_unit<D, K, T>(cell_nodes, metric, x, t, cell, (int)(u - cell * nrhs), nrhs, B);
    }
  }
}

// Paired FP32 variant (even number of right-hand sides): one thread per cell
// and pair of right-hand sides, each value an f2.  Every FMA, index load,
// metric load and atomic then serves two right-hand sides, which halves the
// instruction count of this issue-bound kernel; vectors are read and written
// as float pairs (8-byte aligned rows of right-hand sides).
#ifndef NNMG_REG2_MIN_BLOCKS
#define NNMG_REG2_MIN_BLOCKS 1
#endif
template <int D, int K>
__global__ void __launch_bounds__(128, NNMG_REG2_MIN_BLOCKS) op_reg2_kernel(const int32_t* __restrict__ cell_nodes,
                                                      const float* __restrict__ metric,
                                                      const float2* __restrict__ x,
                                                      float2* __restrict__ y, int64_t n_cells,
                                                      int npair, Basis1D<f2> B) {
  pdl_trigger();
  pdl_wait();
  constexpr int N = K + 1;
  constexpr int NQ = D == 2 ? N * N : N * N * N;
  constexpr int NM = D == 2 ? 3 : 6;
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t cell = u / npair;
  if (cell >= n_cells) return;
  const int pr = (int)(u - cell * npair);
  const int32_t* cn = cell_nodes + cell * NQ;
  f2 v[NQ], gx[NQ], gy[NQ];
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    const int dof = cn[i];
    v[i] = dof >= 0 ? f2(x[(int64_t)dof * npair + pr]) : f2();
  }
#pragma unroll
  for (int d = 0; d < D; ++d) sweep<D, N, kInterp, false>(B.S, v, v, d);
  sweep<D, N, kDeriv, false>(B.Dg, v, gx, 0);
  sweep<D, N, kDeriv, false>(B.Dg, v, gy, 1);
  if constexpr (D == 3) sweep<D, N, kDeriv, false>(B.Dg, v, v, 2);
  constexpr int NQP = padded_nq(NQ);
  const float* mc = metric + cell * NM * NQP;
#pragma unroll
  for (int q0 = 0; q0 < NQ; q0 += 4) {
    float G[NM][4];
#pragma unroll
    for (int m = 0; m < NM; ++m) load_metric(mc + m * NQP + q0, G[m]);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int q = q0 + w;
      if (q >= NQ) break;
      if constexpr (D == 3) {
        const f2 a = gx[q], b = gy[q], c = v[q];
        const f2 G0(G[0][w]), G1(G[1][w]), G2(G[2][w]), G3(G[3][w]), G4(G[4][w]), G5(G[5][w]);
        gx[q] = mac(mac(G0 * a, G1, b), G2, c);
        gy[q] = mac(mac(G1 * a, G3, b), G4, c);
        v[q] = mac(mac(G2 * a, G4, b), G5, c);
      } else {
        const f2 a = gx[q], b = gy[q];
        const f2 G0(G[0][w]), G1(G[1][w]), G2(G[2][w]);
        gx[q] = mac(G0 * a, G1, b);
        gy[q] = mac(G1 * a, G2, b);
      }
    }
  }
  if constexpr (D == 3) {
    sweep<D, N, kDeriv, true>(B.Dg, v, v, 2);
    sweep<D, N, kDeriv, true, true>(B.Dg, gy, v, 1);
    sweep<D, N, kDeriv, true, true>(B.Dg, gx, v, 0);
  } else {
    sweep<D, N, kDeriv, true>(B.Dg, gy, v, 1);
    sweep<D, N, kDeriv, true, true>(B.Dg, gx, v, 0);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) sweep<D, N, kInterp, true>(B.S, v, v, d);
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    const int dof = cn[i];
    if (dof >= 0) atomicAdd(&y[(int64_t)dof * npair + pr], v[i].v);
  }
}

// Paired FP32 3D form with z-slices streamed: the values at the Gauss points
// and their z-derivatives are kept for the whole cell, but the x/y gradients
// and fluxes only for one slice at a time (a slice's values are dead once its
// gradients and the cell's z-derivatives exist, so its transposed x/y
// derivatives take their registers).  About 72 live float pairs instead of
// 81, which fits three 128-thread blocks per SM without spilling.
#ifndef NNMG_REG2S_MIN_BLOCKS
#define NNMG_REG2S_MIN_BLOCKS 3
#endif
template <int K>
__global__ void __launch_bounds__(128, NNMG_REG2S_MIN_BLOCKS) op_reg2s_kernel(const int32_t* __restrict__ cell_nodes,
                                                          const float* __restrict__ metric,
                                                          const float2* __restrict__ x,
                                                          float2* __restrict__ y, int64_t n_cells,
                                                          int npair, Basis1D<f2> B) {
  pdl_trigger();
  pdl_wait();
  constexpr int N = K + 1, N2 = N * N, NQ = N2 * N, NQP = padded_nq(NQ);
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t cell = u / npair;
  if (cell >= n_cells) return;
  const int pr = (int)(u - cell * npair);
  const int32_t* cn = cell_nodes + cell * NQ;
  f2 v[NQ], gz[NQ];
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    const int dof = cn[i];
    v[i] = dof >= 0 ? f2(x[(int64_t)dof * npair + pr]) : f2();
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) sweep<3, N, kInterp, false>(B.S, v, v, d);
  sweep<3, N, kDeriv, false>(B.Dg, v, gz, 2);
  const float* mc = metric + cell * 6 * NQP;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    f2 gx[N2], gy[N2];
#pragma unroll
    for (int j = 0; j < N; ++j) {            // x-lines of the slice
      f2 in[N], out[N];
#pragma unroll
      for (int i = 0; i < N; ++i) in[i] = v[i + N * j + N2 * c];
      apply<N, kDeriv>(B.Dg, in, out);
#pragma unroll
      for (int i = 0; i < N; ++i) gx[i + N * j] = out[i];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {            // y-lines of the slice
      f2 in[N], out[N];
#pragma unroll
      for (int j = 0; j < N; ++j) in[j] = v[i + N * j + N2 * c];
      apply<N, kDeriv>(B.Dg, in, out);
#pragma unroll
      for (int j = 0; j < N; ++j) gy[i + N * j] = out[j];
    }
#pragma unroll
    for (int p = 0; p < N2; ++p) {           // flux = G grad^ at the slice's points
      const int q = p + N2 * c;
      const f2 a = gx[p], b = gy[p], cz = gz[q];
      const f2 G0(mc[q]), G1(mc[NQP + q]), G2(mc[2 * NQP + q]), G3(mc[3 * NQP + q]),
          G4(mc[4 * NQP + q]), G5(mc[5 * NQP + q]);
      gx[p] = mac(mac(G0 * a, G1, b), G2, cz);
      gy[p] = mac(mac(G1 * a, G3, b), G4, cz);
      gz[q] = mac(mac(G2 * a, G4, b), G5, cz);
    }
    // the slice's transposed x and y derivatives replace its values
#pragma unroll
    for (int j = 0; j < N; ++j) {
      f2 in[N], out[N];
#pragma unroll
      for (int i = 0; i < N; ++i) in[i] = gx[i + N * j];
      apply_t<N, kDeriv>(B.Dg, in, out);
#pragma unroll
      for (int i = 0; i < N; ++i) v[i + N * j + N2 * c] = out[i];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      f2 in[N], out[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        in[j] = gy[i + N * j];
        out[j] = v[i + N * j + N2 * c];
      }
      apply_t<N, kDeriv, true>(B.Dg, in, out);
#pragma unroll
      for (int j = 0; j < N; ++j) v[i + N * j + N2 * c] = out[j];
    }
  }
  sweep<3, N, kDeriv, true, true>(B.Dg, gz, v, 2);   // + transposed z derivative
#pragma unroll
  for (int d = 0; d < 3; ++d) sweep<3, N, kInterp, true>(B.S, v, v, d);
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    const int dof = cn[i];
    if (dof >= 0) atomicAdd(&y[(int64_t)dof * npair + pr], v[i].v);
  }
}

template <typename T>
void pick_basis(int k, Basis1D<T>* b);
template <>
void pick_basis<double>(int k, Basis1D<double>* b) {
  Basis1D<float> f;
  make_basis(k, b, &f);
}
template <>
void pick_basis<float>(int k, Basis1D<float>* b) {
  Basis1D<double> d;
  make_basis(k, &d, b);
}
template <>
void pick_basis<dw>(int k, Basis1D<dw>* b) {
  Basis1D<double> d;
  Basis1D<float> f;
  make_basis(k, &d, &f);
  for (int i = 0; i < kMaxN; ++i) {
    for (int j = 0; j < kMaxN; ++j) {
      b->S[i][j] = dw_split_host(d.S[i][j]);
      b->Dg[i][j] = dw_split_host(d.Dg[i][j]);
      b->DS[i][j] = dw_split_host(d.DS[i][j]);
    }
    b->gl[i] = dw_split_host(d.gl[i]);
    b->gl_scale[i] = dw_split_host(d.gl_scale[i]);
    b->gx[i] = dw_split_host(d.gx[i]);
    b->gw[i] = dw_split_host(d.gw[i]);
  }
}

template <>
void pick_basis<f2>(int k, Basis1D<f2>* b) {
  Basis1D<double> d;
  Basis1D<float> f;
  make_basis(k, &d, &f);
  for (int i = 0; i < kMaxN; ++i) {
    for (int j = 0; j < kMaxN; ++j) {
      b->S[i][j] = f2(f.S[i][j]);
      b->Dg[i][j] = f2(f.Dg[i][j]);
      b->DS[i][j] = f2(f.DS[i][j]);
    }
    b->gl[i] = f2(f.gl[i]);
    b->gl_scale[i] = f2(f.gl_scale[i]);
    b->gx[i] = f2(f.gx[i]);
    b->gw[i] = f2(f.gw[i]);
  }
}

template <typename T>
T arith_from_double(double v) {
  return (T)v;
}
template <>
dw arith_from_double<dw>(double v) {
  return dw_split_host(v);
}

struct OpConfig {
  int U;
  unsigned blocks;
  int threads;
  size_t smem;
};

// Units per block: the largest multiple of nrhs not above 32, so a warp is one
// tensor line of consecutive units (conflict-free shared memory); doubled for
// small line counts to reach 128 threads; halved while the block exceeds the
// largest block this kernel can launch with (its registers decide that).
constexpr size_t kMaxSmem = 227 * 1024;

inline OpConfig op_config(int lines, int nq, int arrays, size_t tsize, int64_t n_cells, int nrhs,
                          int max_threads, int units) {
  const size_t per_unit = (size_t)arrays * nq * tsize;
  int u0 = 32 - (32 % nrhs);
  int U = u0;
  while (U * lines < 128 && U * 2 * lines <= 1024) U *= 2;
  while (U > nrhs && (U * lines > max_threads || U * per_unit > kMaxSmem))
    U = std::max(nrhs, (U / 2) / nrhs * nrhs);
  if (units > 0 && units % nrhs == 0 && units * lines <= max_threads && units * per_unit <= kMaxSmem)
    U = units;
  OpConfig c;
  const int cpb = U / nrhs;
  c.U = U;
  c.threads = U * lines;
  c.blocks = (unsigned)((n_cells + cpb - 1) / cpb);
  c.smem = (size_t)arrays * nq * U * tsize;
  return c;
}

template <typename F>
int kernel_max_threads(F kern) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, kern) != cudaSuccess) return 256;
  return a.maxThreadsPerBlock;
}

// Candidate units per block: multiples of nrhs from nrhs up to the kernel's
// largest block, doubling from the warp-aligned default.
inline int unit_candidates(int lines, int nrhs, int max_threads, size_t per_unit, int* out,
                           int max_out) {
  int n = 0;
  int u0 = 32 - (32 % nrhs);
  for (int U = std::max(nrhs, u0 / 4 / nrhs * nrhs);
       U * lines <= max_threads && U * per_unit <= kMaxSmem && n < max_out; U *= 2)
    if (U * lines >= 32) out[n++] = U;
  if (n == 0 && n < max_out) out[n++] = nrhs;
  return n;
}

template <int K, typename T, int NC>
cudaError_t run3d(const DevLevel& L, const typename metric_type<T>::type* metric,
                  const typename io_of<T>::type* x,
                  typename io_of<T>::type* y, int nrhs, double lambda, double mu, cudaStream_t s,
                  int units) {
  constexpr int N = K + 1;
  Basis1D<T> B;
  pick_basis<T>(K, &B);
  auto kern = op3d_kernel_for<K, T, NC>(nrhs);
  // per entry (the plain kernel, or the bounded one op3d_kernel_for picked):
  // its largest block and the opt-in shared memory already granted to it
  const int which = kern == op3d_kernel<K, T, NC> ? 0 : 1;
  static int max_threads_of[2] = {0, 0};
  static size_t smem_set[2] = {48 * 1024, 48 * 1024};
  if (max_threads_of[which] == 0) max_threads_of[which] = kernel_max_threads(kern);
  OpConfig c = op_config(N * N, N * N * N, 3 * NC, sizeof(T), L.n_cells, nrhs,
                         max_threads_of[which], units);
  if (c.smem > smem_set[which]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
    if (e != cudaSuccess) return e;
    smem_set[which] = c.smem;
  }
  return launch_k(kern, c.blocks, c.threads, c.smem, s, L.cell_nodes, metric, x, y, L.n_cells, nrhs,
                  c.U, B, arith_from_double<T>(lambda), arith_from_double<T>(mu));
}

template <int K, typename T>
cudaError_t run2d(const DevLevel& L, const T* metric, const typename io_of<T>::type* x,
                  typename io_of<T>::type* y, int nrhs, cudaStream_t s, int units) {
  constexpr int N = K + 1;
  Basis1D<T> B;
  pick_basis<T>(K, &B);
  static const int max_threads = kernel_max_threads(op2d_kernel<K, T>);
  OpConfig c = op_config(N, N * N, 2, sizeof(T), L.n_cells, nrhs, max_threads, units);
  return launch_k(op2d_kernel<K, T>, c.blocks, c.threads, c.smem, s, L.cell_nodes, metric, x, y,
                  L.n_cells, nrhs, c.U, B);
}

template <typename T>
const T* metric_of(const DevLevel& L);
template <>
const double* metric_of<double>(const DevLevel& L) { return L.metric64; }
template <>
const float* metric_of<float>(const DevLevel& L) { return L.metric32; }
template <>
const dw* metric_of<dw>(const DevLevel& L) { return reinterpret_cast<const dw*>(L.metric_dw); }

}  // namespace

template <int D, int K, typename T>
cudaError_t run_reg(const DevLevel& L, const T* metric, const typename io_of<T>::type* x,
                    typename io_of<T>::type* y, int nrhs, cudaStream_t s) {
  Basis1D<T> B;
  pick_basis<T>(K, &B);
  const int64_t units = L.n_cells * nrhs;
  return launch_k(op_reg_kernel<D, K, T>, (unsigned)((units + 127) / 128), 128, 0, s, L.cell_nodes,
                  metric, x, y, L.n_cells, nrhs, B);
}

template <int D, int K>
cudaError_t run_reg2(const DevLevel& L, const float* metric, const float* x, float* y, int nrhs,
                     cudaStream_t s) {
  Basis1D<f2> B;
  pick_basis<f2>(K, &B);
  const int npair = nrhs / 2;
  const int64_t units = L.n_cells * npair;
  if constexpr (D == 3)
    return launch_k(op_reg2s_kernel<K>, (unsigned)((units + 127) / 128), 128, 0, s, L.cell_nodes,
                    metric, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(y),
                    L.n_cells, npair, B);
  return launch_k(op_reg2_kernel<D, K>, (unsigned)((units + 127) / 128), 128, 0, s, L.cell_nodes,
                  metric, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(y), L.n_cells,
                  npair, B);
}

template <int D, int K, typename T>
cudaError_t run_smoother(const DevLevel& L, const T* f, T* t, const T* dinv, T* d, T* x, int nrhs,
                         const SmootherPlan& P, unsigned* bar, int* err, cudaStream_t s) {
  Basis1D<T> B;
  pick_basis<T>(K, &B);
  auto kern = cheb_smoother_kernel<D, K, T>;
  static int per_sm = -1, sms = 0;
  if (per_sm < 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSmootherThreads, 0);
    if (e != cudaSuccess) return e;
  }
  const int64_t units = L.n_cells * nrhs;
  const int64_t want = std::max<int64_t>(1, (units + kSmootherThreads - 1) / kSmootherThreads);
  const unsigned blocks = (unsigned)std::min<int64_t>(want, (int64_t)per_sm * sms);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = blocks;
  cfg.blockDim = kSmootherThreads;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, (const int32_t*)L.cell_nodes, (const T*)metric_of<T>(L), f,
                            t, dinv, d, x, L.n_cells, L.rows, nrhs, B, P, bar, err);
}

// The register-resident kernel serves Poisson cells with at most 27 (3D) or
// 25 (2D) nodes, in every arithmetic type; units < 0 asks for it explicitly,
// units = -2 for its paired FP32 form (even
// nrhs, 8-byte aligned vectors; otherwise the unpaired one runs), units > 0
// for the shared-memory kernel with that many units per block (autotuner
// choices), units = 0 for the default: the register kernel where it applies
// in FP32 and FP64, the shared-memory kernel in double-word arithmetic (whose
// register kernel, at 255 registers, measured 1.9x slower on 3D Q2).
// units <= kPairedSmem selects the paired FP32 form of the 3D Poisson
// shared-memory kernel (two right-hand sides per thread, packed FP32
// instructions) with kPairedSmem - units (cell, pair) units per block; it
// runs for an even nrhs on 8-byte aligned vectors (otherwise the default).
constexpr int kPairedSmem = -100;

template <typename T>
bool reg_eligible(const DevLevel& L) {
  return L.ncomp == 1 && (L.dim == 2 || L.k <= 2);
}

template <typename T>
cudaError_t launch_operator_impl(const DevLevel& L, const typename io_of<T>::type* x,
                                 typename io_of<T>::type* y, int nrhs, double lambda, double mu,
                                 cudaStream_t s, int units) {
  if (L.n_cells == 0) return cudaSuccess;
  const T* m = metric_of<T>(L);
  if (!m) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 4) {
    if (reg_eligible<T>(L) && units == -2 && nrhs % 2 == 0 && (uintptr_t)x % 8 == 0 &&
        (uintptr_t)y % 8 == 0) {
#define NNMG_REG2(D, K) if (L.dim == D && L.k == K) return run_reg2<D, K>(L, m, x, y, nrhs, s);
      NNMG_REG2(2, 1) NNMG_REG2(2, 2) NNMG_REG2(2, 3) NNMG_REG2(2, 4) NNMG_REG2(3, 1) NNMG_REG2(3, 2)
#undef NNMG_REG2
    }
  }
  if constexpr (sizeof(T) == 4) {
    if (units <= kPairedSmem && L.dim == 3 && L.ncomp == 1 && nrhs % 2 == 0 &&
        (uintptr_t)x % 8 == 0 && (uintptr_t)y % 8 == 0) {
      const float2* x2 = reinterpret_cast<const float2*>(x);
      float2* y2 = reinterpret_cast<float2*>(y);
      const int U = kPairedSmem - units;
      switch (L.k) {
        case 1: return run3d<1, f2, 1>(L, m, x2, y2, nrhs / 2, 0.0, 0.0, s, U);
        case 2: return run3d<2, f2, 1>(L, m, x2, y2, nrhs / 2, 0.0, 0.0, s, U);
        case 3: return run3d<3, f2, 1>(L, m, x2, y2, nrhs / 2, 0.0, 0.0, s, U);
        case 4: return run3d<4, f2, 1>(L, m, x2, y2, nrhs / 2, 0.0, 0.0, s, U);
      }
    }
  }
  constexpr bool reg_default = !std::is_same<T, dw>::value;
  if (reg_eligible<T>(L) && (units < 0 || (units == 0 && reg_default))) {
#define NNMG_REG(D, K) if (L.dim == D && L.k == K) return run_reg<D, K, T>(L, m, x, y, nrhs, s);
    NNMG_REG(2, 1) NNMG_REG(2, 2) NNMG_REG(2, 3) NNMG_REG(2, 4) NNMG_REG(3, 1) NNMG_REG(3, 2)
#undef NNMG_REG
  }
  if (L.dim == 2) {
    switch (L.k) {
      case 1: return run2d<1, T>(L, m, x, y, nrhs, s, units);
      case 2: return run2d<2, T>(L, m, x, y, nrhs, s, units);
      case 3: return run2d<3, T>(L, m, x, y, nrhs, s, units);
      case 4: return run2d<4, T>(L, m, x, y, nrhs, s, units);
    }
  } else if (L.ncomp == 1) {
    switch (L.k) {
      case 1: return run3d<1, T, 1>(L, m, x, y, nrhs, lambda, mu, s, units);
      case 2: return run3d<2, T, 1>(L, m, x, y, nrhs, lambda, mu, s, units);
      case 3: return run3d<3, T, 1>(L, m, x, y, nrhs, lambda, mu, s, units);
      case 4: return run3d<4, T, 1>(L, m, x, y, nrhs, lambda, mu, s, units);
    }
  } else {
    switch (L.k) {
      case 1: return run3d<1, T, 3>(L, m, x, y, nrhs, lambda, mu, s, units);
      case 2: return run3d<2, T, 3>(L, m, x, y, nrhs, lambda, mu, s, units);
      case 3: return run3d<3, T, 3>(L, m, x, y, nrhs, lambda, mu, s, units);
      case 4: return run3d<4, T, 3>(L, m, x, y, nrhs, lambda, mu, s, units);
    }
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_operator(const DevLevel& L, const T* x, T* y, int nrhs, double lambda,
                            double mu, cudaStream_t s, int units) {
  return for_each_color(L, [&](const DevLevel& V) {
    return launch_operator_impl<T>(V, x, y, nrhs, lambda, mu, s, units);
  });
}

cudaError_t launch_operator_dw(const DevLevel& L, const double* x, double* y, int nrhs,
                               double lambda, double mu, cudaStream_t s, int units) {
  return for_each_color(L, [&](const DevLevel& V) {
    return launch_operator_impl<dw>(V, x, y, nrhs, lambda, mu, s, units);
  });
}

bool cheb_step_fused_supported(const DevLevel& L) {
  return L.color_start.empty() && L.ncomp == 1 && L.valence && L.node_count &&
         ((L.dim == 3 && L.k <= 2) || (L.dim == 2 && L.k <= 4));
}

template <typename T>
cudaError_t launch_cheb_step_fused(const DevLevel& L, const T* f, T* t, const T* dinv, T* d, T* x,
                                   double cd, double cr, int nrhs, cudaStream_t s) {
  if (!cheb_step_fused_supported(L) || nrhs < 1 || nrhs > 128) return cudaErrorInvalidValue;
  if (L.n_cells == 0) return cudaSuccess;
  const int cpb = 128 / nrhs;
  const unsigned blocks = (unsigned)((L.n_cells + cpb - 1) / cpb);
  const T* m = metric_of<T>(L);
  Basis1D<T> B;
#define NNMG_OPCHEB(DD, KK)                                                                   \
  if (L.dim == DD && L.k == KK) {                                                            \
    pick_basis<T>(KK, &B);                                                                   \
    return launch_k(op_cheb_kernel<DD, KK, T>, blocks, cpb * nrhs, 0, s, L.cell_nodes, m, f, t, \
                    dinv, d, x, L.node_count, L.valence, L.n_cells, nrhs, B, (T)cd, (T)cr);  \
  }
  NNMG_OPCHEB(2, 1) NNMG_OPCHEB(2, 2) NNMG_OPCHEB(2, 3) NNMG_OPCHEB(2, 4)
  NNMG_OPCHEB(3, 1) NNMG_OPCHEB(3, 2)
#undef NNMG_OPCHEB
  return cudaErrorInvalidValue;
}
template cudaError_t launch_cheb_step_fused<float>(const DevLevel&, const float*, float*,
                                                   const float*, float*, float*, double, double,
                                                   int, cudaStream_t);
template cudaError_t launch_cheb_step_fused<double>(const DevLevel&, const double*, double*,
                                                    const double*, double*, double*, double,
                                                    double, int, cudaStream_t);

template <typename T>
int operator_unit_candidates(const DevLevel& L, int nrhs, int* out, int max_out) {
  int lines = 0, mt = 256;
  size_t per_unit = 0;
#define NNMG_C(D, K, NC)                                                              \
  if (L.dim == D && L.k == K && L.ncomp == NC) {                                      \
    lines = D == 2 ? K + 1 : (K + 1) * (K + 1);                                       \
    per_unit = (D == 2 ? 2 : 3 * NC) * (size_t)lines * (K + 1) * sizeof(T);          \
    mt = D == 2 ? kernel_max_threads(op2d_kernel<K, T>) : kernel_max_threads(op3d_kernel_for<K, T, NC>(nrhs)); \
  }
  NNMG_C(2, 1, 1) NNMG_C(2, 2, 1) NNMG_C(2, 3, 1) NNMG_C(2, 4, 1)
  NNMG_C(3, 1, 1) NNMG_C(3, 2, 1) NNMG_C(3, 3, 1) NNMG_C(3, 4, 1)
  NNMG_C(3, 1, 3) NNMG_C(3, 2, 3) NNMG_C(3, 3, 3) NNMG_C(3, 4, 3)
#undef NNMG_C
  if (lines == 0) return 0;
  int n = 0;
  if (reg_eligible<T>(L) && max_out > 0) out[n++] = -1;   // the register-resident kernel
  if (sizeof(T) == 4 && reg_eligible<T>(L) && nrhs % 2 == 0 && n < max_out) out[n++] = -2;
  n += unit_candidates(lines, nrhs, mt, per_unit, out + n, max_out - n);
  if (sizeof(T) == 4 && L.dim == 3 && L.ncomp == 1 && nrhs % 2 == 0 && n < max_out) {
    int mt2 = 256;
#define NNMG_C2(K) if (L.k == K) mt2 = kernel_max_threads(op3d_kernel_for<K, f2, 1>(nrhs / 2));
    NNMG_C2(1) NNMG_C2(2) NNMG_C2(3) NNMG_C2(4)
#undef NNMG_C2
    // (cell, pair) units per block: from half the unpaired kernel's smallest
    // block (the same cells per block) upwards, doubling
    const int npair = nrhs / 2;
    const int u0 = 32 - (32 % nrhs);
    for (int U = std::max(npair, std::max(nrhs, u0 / 4 / nrhs * nrhs) / 2);
         U * lines <= mt2 && (size_t)U * per_unit * 2 <= kMaxSmem && n < max_out; U *= 2)
      if (U * lines >= 32) out[n++] = kPairedSmem - U;
  }
  return n;
}

// The persistent smoother is meant for levels where launches dominate: those
// whose operator fills at most kSmootherWaves waves of the GPU (4 blocks of
// 128 threads per SM at the register operator's 128 registers).  On larger
// levels its vector phase, at the operator's occupancy, loses to the separate
// vector kernels (config 2's 55^3 fine level: 1.321 vs 1.103 ms per level and
// V-cycle, eager).
constexpr int64_t kSmootherWaves = 4;
bool cheb_smoother_supported(const DevLevel& L, int m, int nrhs) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return false;
  }
  const int64_t wave = (int64_t)sms * 4 * 128;
  return L.n_cells > 0 && reg_eligible<float>(L) && m >= 1 && m <= kMaxChebSteps &&
         L.n_cells * nrhs <= kSmootherWaves * wave;
}

template <typename T>
cudaError_t launch_cheb_smoother(const DevLevel& L, const T* f, T* t, const T* dinv, T* d, T* x,
                                 int nrhs, const SmootherPlan& P, unsigned* bar, int* err,
                                 cudaStream_t s) {
  if (!cheb_smoother_supported(L, P.steps, nrhs)) return cudaErrorNotSupported;
#define NNMG_S(D, K) \
  if (L.dim == D && L.k == K) return run_smoother<D, K, T>(L, f, t, dinv, d, x, nrhs, P, bar, err, s);
  NNMG_S(2, 1) NNMG_S(2, 2) NNMG_S(2, 3) NNMG_S(2, 4) NNMG_S(3, 1) NNMG_S(3, 2)
#undef NNMG_S
  return cudaErrorNotSupported;
}

template cudaError_t launch_cheb_smoother<float>(const DevLevel&, const float*, float*, const float*,
                                                 float*, float*, int, const SmootherPlan&,
                                                 unsigned*, int*, cudaStream_t);
template cudaError_t launch_cheb_smoother<double>(const DevLevel&, const double*, double*,
                                                  const double*, double*, double*, int,
                                                  const SmootherPlan&, unsigned*, int*,
                                                  cudaStream_t);
template cudaError_t launch_operator<float>(const DevLevel&, const float*, float*, int, double,
                                            double, cudaStream_t, int);
template cudaError_t launch_operator<double>(const DevLevel&, const double*, double*, int, double,
                                             double, cudaStream_t, int);
template int operator_unit_candidates<float>(const DevLevel&, int, int*, int);
template int operator_unit_candidates<double>(const DevLevel&, int, int*, int);
template int operator_unit_candidates<dw>(const DevLevel&, int, int*, int);

}  // namespace nnmg
