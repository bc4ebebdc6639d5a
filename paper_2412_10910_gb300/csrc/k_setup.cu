// Setup kernels in FP64: metric terms at quadrature points, support points,
// point-Jacobi diagonal, load vectors and location of fine support points in
// the coarse mesh (Sec. 3.1: candidate cells from a bounding-box grid, Newton
// inversion of the Q1 cell map, first accepting cell by index, nearest-point
// projection otherwise, Sec. 3.3 Eq. closest_point).
#include <cmath>

#include "nnmg_internal.h"

namespace nnmg {
namespace {

// Q1 map: x(xi) and J[a][b] = dx_a/dxi_b from the 2^D corners.
template <int D>
__device__ __forceinline__ void q1_map(const double* __restrict__ X /*[2^D][D]*/,
                                       const double* xi, double* x, double (*J)[3]) {
  for (int a = 0; a < D; ++a) {
    x[a] = 0.0;
    for (int b = 0; b < D; ++b) J[a][b] = 0.0;
  }
#pragma unroll
  for (int v = 0; v < (1 << D); ++v) {
    double f[3], df[3];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int bit = (v >> d) & 1;
      f[d] = bit ? xi[d] : 1.0 - xi[d];
      df[d] = bit ? 1.0 : -1.0;
    }
    double N = 1.0;
#pragma unroll
    for (int d = 0; d < D; ++d) N *= f[d];
    double dN[3];
#pragma unroll
    for (int b = 0; b < D; ++b) {
      double t = df[b];
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (d != b) t *= f[d];
      dN[b] = t;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double Xa = X[v * D + a];
      x[a] += N * Xa;
#pragma unroll
      for (int b = 0; b < D; ++b) J[a][b] += Xa * dN[b];
    }
  }
}

// determinant and inverse of a DxD matrix
template <int D>
__device__ __forceinline__ double inv_det(const double (*J)[3], double (*Ji)[3]) {
  if (D == 2) {
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double r = 1.0 / det;
    Ji[0][0] = J[1][1] * r;
    Ji[0][1] = -J[0][1] * r;
    Ji[1][0] = -J[1][0] * r;
    Ji[1][1] = J[0][0] * r;
    return det;
  } else {
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    const double r = 1.0 / det;
    Ji[0][0] = c00 * r;
    Ji[1][0] = c01 * r;
    Ji[2][0] = c02 * r;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * r;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * r;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * r;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * r;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * r;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * r;
    return det;
  }
}

template <int D>
__device__ __forceinline__ void load_corners(const double* __restrict__ vertices,
                                             const int32_t* __restrict__ cells, int64_t c,
                                             double* X) {
#pragma unroll
  for (int v = 0; v < (1 << D); ++v) {
    const int64_t g = cells[c * (1 << D) + v];
#pragma unroll
    for (int d = 0; d < D; ++d) X[v * D + d] = vertices[g * D + d];
  }
}

// Metric terms per (cell, quadrature point).  Poisson: the symmetric
// G = |det J| w J^-1 J^-T (upper triangle, D(D+1)/2 values).  Elasticity:
// K = sqrt(|det J| w) J^-1 (9 values), so that the reference flux of the
// stress is K sigma(grad^u K) (Sec. 4.4).
template <int D>
__global__ void metric_kernel(const double* __restrict__ vertices, const int32_t* __restrict__ cells,
                              int64_t nc, int n1, int ncomp, int nqp, Basis1D<double> B,
                              double* __restrict__ m64, float* __restrict__ m32, int* err) {
  const int nq = D == 2 ? n1 * n1 : n1 * n1 * n1;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= nc * nq) return;
  const int64_t c = tid / nq;
  const int q = (int)(tid % nq);
  const int qi[3] = {q % n1, (q / n1) % n1, q / (n1 * n1)};
  double X[(1 << D) * D];
  load_corners<D>(vertices, cells, c, X);
  double xi[3], x[3], J[3][3], Ji[3][3];
  double w = 1.0;
  for (int d = 0; d < D; ++d) {
    xi[d] = B.gx[qi[d]];
    w *= B.gw[qi[d]];
  }
  q1_map<D>(X, xi, x, J);
  const double det = inv_det<D>(J, Ji);
  if (!(det > 0.0)) atomicExch(err, 1);
  const double dw = fabs(det) * w;
  if (ncomp == 1) {
    const int nm = D * (D + 1) / 2;
    int j = 0;
    for (int a = 0; a < D; ++a)
      for (int b = a; b < D; ++b) {
        double g = 0.0;
        for (int e = 0; e < D; ++e) g += Ji[a][e] * Ji[b][e];
        g *= dw;
        const int64_t o = (c * nm + j) * nqp + q;
        m64[o] = g;
        m32[o] = (float)g;
        ++j;
      }
  } else {
    const double s = sqrt(dw);
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) {
        const double g = s * Ji[a][b];
        const int64_t o = (c * (D * D) + a * D + b) * nqp + q;
        m64[o] = g;
        m32[o] = (float)g;
      }
  }
}

// Support point of every node from its first-touch (cell, local node).
template <int D>
__global__ void support_kernel(const double* __restrict__ vertices, const int32_t* __restrict__ cells,
                               const int32_t* __restrict__ owner_cell,
                               const int32_t* __restrict__ owner_local, int64_t n, int n1,
                               Basis1D<double> B, double* __restrict__ pts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double X[(1 << D) * D];
  load_corners<D>(vertices, cells, owner_cell[i], X);
  const int l = owner_local[i];
  const int m[3] = {l % n1, (l / n1) % n1, l / (n1 * n1)};
  double xi[3], x[3], J[3][3];
  for (int d = 0; d < D; ++d) xi[d] = B.gl[m[d]];
  q1_map<D>(X, xi, x, J);
  for (int d = 0; d < D; ++d) pts[i * D + d] = x[d];
}

// Physical quadrature points.
template <int D>
__global__ void quad_points_kernel(const double* __restrict__ vertices,
                                   const int32_t* __restrict__ cells, int64_t nc, int n1,
                                   Basis1D<double> B, double* __restrict__ xq) {
  const int nq = D == 2 ? n1 * n1 : n1 * n1 * n1;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= nc * nq) return;
  const int64_t c = tid / nq;
  const int q = (int)(tid % nq);
  const int qi[3] = {q % n1, (q / n1) % n1, q / (n1 * n1)};
  double X[(1 << D) * D];
  load_corners<D>(vertices, cells, c, X);
  double xi[3], x[3], J[3][3];
  for (int d = 0; d < D; ++d) xi[d] = B.gx[qi[d]];
  q1_map<D>(X, xi, x, J);
  for (int d = 0; d < D; ++d) xq[tid * D + d] = x[d];
}

// Diagonal of the cell operators summed into diag[row] (FP64 atomics).
// Poisson: sum_q grad^phi_i . G_q grad^phi_i.  Elasticity, row (i, c):
// sum_q lambda h_c^2 + mu (|h|^2 + h_c^2) with h = K^T grad^phi_i.
template <int D>
__global__ void diag_kernel(const int32_t* __restrict__ cell_nodes, const double* __restrict__ m64,
                            int64_t nc, int n1, int ncomp, int nqp, double lambda, double mu,
                            Basis1D<double> B, double* __restrict__ diag) {
  const int nloc = D == 2 ? n1 * n1 : n1 * n1 * n1;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= nc * nloc) return;
  const int64_t c = tid / nloc;
  const int i = (int)(tid % nloc);
  const int node = cell_nodes[tid];
  if (node < 0) return;
  const int mi[3] = {i % n1, (i / n1) % n1, i / (n1 * n1)};
  double acc[3] = {0.0, 0.0, 0.0};
  for (int q = 0; q < nloc; ++q) {
    const int qi[3] = {q % n1, (q / n1) % n1, q / (n1 * n1)};
    double g[3];
    for (int a = 0; a < D; ++a) {
      double t = 1.0;
      for (int d = 0; d < D; ++d) t *= (d == a) ? B.DS[qi[d]][mi[d]] : B.S[qi[d]][mi[d]];
      g[a] = t;
    }
    if (ncomp == 1) {
      const int nm = D * (D + 1) / 2;
      int j = 0;
      double s = 0.0;
      for (int a = 0; a < D; ++a)
        for (int b = a; b < D; ++b) {
          const double Gab = m64[(c * nm + j) * nqp + q];
          s += (a == b ? 1.0 : 2.0) * Gab * g[a] * g[b];
          ++j;
        }
      acc[0] += s;
    } else {
      double h[3] = {0.0, 0.0, 0.0};
      for (int b = 0; b < D; ++b)
        for (int a = 0; a < D; ++a) h[b] += g[a] * m64[(c * (D * D) + a * D + b) * nqp + q];
      double hh = 0.0;
      for (int b = 0; b < D; ++b) hh += h[b] * h[b];
      for (int e = 0; e < D; ++e) acc[e] += lambda * h[e] * h[e] + mu * (hh + h[e] * h[e]);
    }
  }
  for (int e = 0; e < ncomp; ++e) atomicAdd(&diag[(int64_t)node * ncomp + e], acc[e]);
}

// b[(node*ncomp + e)*nrhs + col] += sum_q |det J| w_q f_e(x_q) phi_i(xi_q)
template <int D>
__global__ void load_kernel(const double* __restrict__ vertices, const int32_t* __restrict__ cells,
                            const int32_t* __restrict__ cell_nodes, int64_t nc, int n1, int ncomp,
                            const double* __restrict__ f, int f_per_qp, Basis1D<double> B,
                            double* __restrict__ b, int nrhs, int col) {
  const int nloc = D == 2 ? n1 * n1 : n1 * n1 * n1;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= nc * nloc) return;
  const int64_t c = tid / nloc;
  const int i = (int)(tid % nloc);
  const int node = cell_nodes[tid];
  if (node < 0) return;
  const int mi[3] = {i % n1, (i / n1) % n1, i / (n1 * n1)};
  double X[(1 << D) * D];
  load_corners<D>(vertices, cells, c, X);
  double acc[3] = {0.0, 0.0, 0.0};
  for (int q = 0; q < nloc; ++q) {
    const int qi[3] = {q % n1, (q / n1) % n1, q / (n1 * n1)};
    double xi[3], x[3], J[3][3], Ji[3][3];
    double w = 1.0, phi = 1.0;
    for (int d = 0; d < D; ++d) {
      xi[d] = B.gx[qi[d]];
      w *= B.gw[qi[d]];
      phi *= B.S[qi[d]][mi[d]];
    }
    q1_map<D>(X, xi, x, J);
    const double dw = fabs(inv_det<D>(J, Ji)) * w;
    for (int e = 0; e < ncomp; ++e) {
      const double fv = f_per_qp ? f[(c * nloc + q) * ncomp + e] : f[e];
      acc[e] += dw * fv * phi;
    }
  }
  for (int e = 0; e < ncomp; ++e)
    atomicAdd(&b[((int64_t)node * ncomp + e) * nrhs + col], acc[e]);
}

// Newton inversion of the Q1 map: start (1/2,..), at most 30 steps, stop when
// max|dxi| < 1e-14.  Returns true only if the map was inverted: the last step
// was below 1e-10 (iterates that wander without converging, as for a point
// outside a strongly distorted cell, are not preimages) and no Jacobian was
// singular.
template <int D>
__device__ bool newton(const double* X, const double* p, double* xi) {
  for (int d = 0; d < D; ++d) xi[d] = 0.5;
  double last = INFINITY;
  for (int it = 0; it < 30; ++it) {
    double x[3], J[3][3], Ji[3][3];
    q1_map<D>(X, xi, x, J);
    const double det = inv_det<D>(J, Ji);
    if (!(det != 0.0) || !isfinite(det)) {
      for (int d = 0; d < D; ++d) xi[d] = nan("");
      return false;
    }
    double r[3], mx = 0.0;
    for (int d = 0; d < D; ++d) r[d] = x[d] - p[d];
    for (int a = 0; a < D; ++a) {
      double dx = 0.0;
      for (int b = 0; b < D; ++b) dx += Ji[a][b] * r[b];
      xi[a] -= dx;
      const double adx = fabs(dx);
      if (!(adx <= mx)) mx = adx;  // a NaN step propagates and counts as not converged
    }
    last = mx;
    if (!(mx >= 1e-14)) break;
  }
  return last < 1e-10;
}

template <int D>
__global__ void locate_kernel(const double* __restrict__ vertices, const int32_t* __restrict__ cells,
                              int64_t nc, const double* __restrict__ points,
                              const int32_t* __restrict__ pt_nodes, int64_t n_pts,
                              const int32_t* __restrict__ bstart, const int32_t* __restrict__ bcells,
                              const double* __restrict__ aabb, BucketGeom g,
                              int32_t* __restrict__ out_cell, double* __restrict__ out_xi) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pts) return;
  const int64_t node = pt_nodes[i];
  double p[3];
  for (int d = 0; d < D; ++d) p[d] = points[node * D + d];
  int bi[3] = {0, 0, 0};
  for (int d = 0; d < D; ++d) {
    int b = (int)floor((p[d] - g.lo[d]) * g.inv_w[d]);
    bi[d] = min(max(b, 0), g.nb[d] - 1);
  }
  const int64_t b = bi[0] + (int64_t)g.nb[0] * (bi[1] + (int64_t)g.nb[1] * bi[2]);
  const double tol = 1e-10;
  int found = -1;
  double xi[3], X[(1 << D) * D];
  for (int j = bstart[b]; j < bstart[b + 1] && found < 0; ++j) {
    const int c = bcells[j];
    bool in = true;
    for (int d = 0; d < D; ++d)
      in = in && p[d] >= aabb[c * 6 + d] - g.eps && p[d] <= aabb[c * 6 + 3 + d] + g.eps;
    if (!in) continue;
    load_corners<D>(vertices, cells, c, X);
    if (!newton<D>(X, p, xi)) continue;
    bool ok = true;
    for (int d = 0; d < D; ++d) ok = ok && xi[d] >= -tol && xi[d] <= 1.0 + tol;
    if (ok) found = c;
  }
  if (found < 0) {
    // Nearest point (Sec. 3.3 Eq. closest_point): the converged cell whose xi
    // is nearest to [0,1]^d, first searched among the cells listed in the 3^d
    // buckets around the point (a point outside a curved boundary lies within
    // about one coarse cell of its owner), then, if none converged, over all
    // cells.  Ties keep the lowest cell index.
    double best = INFINITY;
    double bxi[3] = {0, 0, 0};
    auto consider = [&](int c) {
      load_corners<D>(vertices, cells, c, X);
      if (!newton<D>(X, p, xi)) return;
      double dd = 0.0;
      for (int d = 0; d < D; ++d) {
        const double e = xi[d] - fmin(fmax(xi[d], 0.0), 1.0);
        dd += e * e;
      }
      dd = sqrt(dd);
      if (dd < best || (dd == best && c < found)) {
        best = dd;
        found = c;
        for (int d = 0; d < D; ++d) bxi[d] = xi[d];
      }
    };
    const int lo0 = max(bi[0] - 1, 0), hi0 = min(bi[0] + 1, g.nb[0] - 1);
    const int lo1 = D > 1 ? max(bi[1] - 1, 0) : 0, hi1 = D > 1 ? min(bi[1] + 1, g.nb[1] - 1) : 0;
    const int lo2 = D > 2 ? max(bi[2] - 1, 0) : 0, hi2 = D > 2 ? min(bi[2] + 1, g.nb[2] - 1) : 0;
    for (int z = lo2; z <= hi2; ++z)
      for (int y = lo1; y <= hi1; ++y)
        for (int x = lo0; x <= hi0; ++x) {
          const int64_t nbk = x + (int64_t)g.nb[0] * (y + (int64_t)g.nb[1] * z);
          for (int j = bstart[nbk]; j < bstart[nbk + 1]; ++j) consider(bcells[j]);
        }
    if (found < 0)
      for (int64_t c = 0; c < nc; ++c) consider((int)c);
    for (int d = 0; d < D; ++d) xi[d] = bxi[d];
  }
  out_cell[i] = found;
  for (int d = 0; d < D; ++d) out_xi[i * D + d] = fmin(fmax(xi[d], 0.0), 1.0);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_metric(const DevLevel& L, int* d_err, cudaStream_t s) {
  Basis1D<double> b64;
  Basis1D<float> b32;
  make_basis(L.k, &b64, &b32);
  const int64_t n = L.n_cells * L.nloc;
  if (n == 0) return cudaSuccess;
  if (L.dim == 2)
    metric_kernel<2><<<blocks_for(n, 128), 128, 0, s>>>(L.vertices, L.cells, L.n_cells, L.n1,
                                                        L.ncomp, L.nqp, b64, L.metric64, L.metric32,
                                                        d_err);
  else
    metric_kernel<3><<<blocks_for(n, 128), 128, 0, s>>>(L.vertices, L.cells, L.n_cells, L.n1,
                                                        L.ncomp, L.nqp, b64, L.metric64, L.metric32,
                                                        d_err);
  return cudaGetLastError();
}

cudaError_t launch_support_points(const DevLevel& L, cudaStream_t s) {
  Basis1D<double> b64;
  Basis1D<float> b32;
  make_basis(L.k, &b64, &b32);
  if (L.n_nodes == 0) return cudaSuccess;
  if (L.dim == 2)
    support_kernel<2><<<blocks_for(L.n_nodes, 128), 128, 0, s>>>(
        L.vertices, L.cells, L.owner_cell, L.owner_local, L.n_nodes, L.n1, b64, L.points);
  else
    support_kernel<3><<<blocks_for(L.n_nodes, 128), 128, 0, s>>>(
        L.vertices, L.cells, L.owner_cell, L.owner_local, L.n_nodes, L.n1, b64, L.points);
  return cudaGetLastError();
}

cudaError_t launch_quad_points(const DevLevel& L, double* xq, cudaStream_t s) {
  Basis1D<double> b64;
  Basis1D<float> b32;
  make_basis(L.k, &b64, &b32);
  const int64_t n = L.n_cells * L.nloc;
  if (n == 0) return cudaSuccess;
  if (L.dim == 2)
    quad_points_kernel<2><<<blocks_for(n, 128), 128, 0, s>>>(L.vertices, L.cells, L.n_cells, L.n1, b64, xq);
  else
    quad_points_kernel<3><<<blocks_for(n, 128), 128, 0, s>>>(L.vertices, L.cells, L.n_cells, L.n1, b64, xq);
  return cudaGetLastError();
}

namespace {
cudaError_t launch_diag_range(const DevLevel& L, double lambda, double mu, cudaStream_t s) {
  Basis1D<double> b64;
  Basis1D<float> b32;
  make_basis(L.k, &b64, &b32);
  const int64_t n = L.n_cells * L.nloc;
  if (n == 0) return cudaSuccess;
  if (L.dim == 2)
    diag_kernel<2><<<blocks_for(n, 128), 128, 0, s>>>(L.cell_nodes, L.metric64, L.n_cells, L.n1,
                                                      L.ncomp, L.nqp, lambda, mu, b64, L.diag64);
  else
    diag_kernel<3><<<blocks_for(n, 128), 128, 0, s>>>(L.cell_nodes, L.metric64, L.n_cells, L.n1,
                                                      L.ncomp, L.nqp, lambda, mu, b64, L.diag64);
  return cudaGetLastError();
}

cudaError_t launch_load_range(const DevLevel& L, const double* f, int f_per_qp, double* b,
                              int nrhs, int col, cudaStream_t s) {
  Basis1D<double> b64;
  Basis1D<float> b32;
  make_basis(L.k, &b64, &b32);
  const int64_t n = L.n_cells * L.nloc;
  if (n == 0) return cudaSuccess;
  if (L.dim == 2)
    load_kernel<2><<<blocks_for(n, 128), 128, 0, s>>>(L.vertices, L.cells, L.cell_nodes, L.n_cells,
                                                      L.n1, L.ncomp, f, f_per_qp, b64, b, nrhs, col);
  else
    load_kernel<3><<<blocks_for(n, 128), 128, 0, s>>>(L.vertices, L.cells, L.cell_nodes, L.n_cells,
                                                      L.n1, L.ncomp, f, f_per_qp, b64, b, nrhs, col);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_diag(const DevLevel& L, double lambda, double mu, cudaStream_t s) {
  return for_each_color(L, [&](const DevLevel& V) { return launch_diag_range(V, lambda, mu, s); });
}

// f per quadrature point is [n_cells][nloc][ncomp] in the level's cell order.
cudaError_t launch_load_vector(const DevLevel& L, const double* f, int f_per_qp, double* b,
                               int nrhs, int col, cudaStream_t s) {
  return for_each_color(L, [&](const DevLevel& V) {
    const double* fv = f_per_qp ? f + (V.cell_nodes - L.cell_nodes) * L.ncomp : f;
    return launch_load_range(V, fv, f_per_qp, b, nrhs, col, s);
  });
}

cudaError_t launch_locate(const DevLevel& coarse, const double* points, const int32_t* pt_nodes,
                          int64_t n_pts, const int32_t* bucket_start, const int32_t* bucket_cells,
                          const double* aabb, const BucketGeom& gg, int32_t* out_cell,
                          double* out_xi, cudaStream_t s) {
  if (n_pts == 0) return cudaSuccess;
  if (coarse.dim == 2)
    locate_kernel<2><<<blocks_for(n_pts, 128), 128, 0, s>>>(
        coarse.vertices, coarse.cells, coarse.n_cells, points, pt_nodes, n_pts, bucket_start,
        bucket_cells, aabb, gg, out_cell, out_xi);
  else
    locate_kernel<3><<<blocks_for(n_pts, 128), 128, 0, s>>>(
        coarse.vertices, coarse.cells, coarse.n_cells, points, pt_nodes, n_pts, bucket_start,
        bucket_cells, aabb, gg, out_cell, out_xi);
  return cudaGetLastError();
}

}  // namespace nnmg

namespace nnmg {
namespace {
__global__ void finalize_diag_kernel(const double* __restrict__ diag, const uint8_t* __restrict__ row_free,
                                     double* __restrict__ dinv64, float* __restrict__ dinv32,
                                     int64_t rows) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const double v = (row_free[i] && diag[i] > 0.0) ? 1.0 / diag[i] : 0.0;
  dinv64[i] = v;
  dinv32[i] = (float)v;
}
}  // namespace

cudaError_t launch_finalize_diag(const double* diag, const uint8_t* row_free, double* dinv64,
                                 float* dinv32, int64_t rows, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  finalize_diag_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(diag, row_free, dinv64, dinv32, rows);
  return cudaGetLastError();
}
}  // namespace nnmg
