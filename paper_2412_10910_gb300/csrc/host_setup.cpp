// Host-side setup: 1D basis tables, continuous Q_k node numbering, Dirichlet
// set, coarse-cell bucket grid for point location and the dense FP64
// factorisation of the coarsest operator.
#include <algorithm>
#include <cmath>
#include <thread>
#include <unordered_map>

#include "nnmg_internal.h"

namespace nnmg {

static thread_local std::string g_error;
void set_error(const std::string& msg) { g_error = msg; }
const char* get_error() { return g_error.c_str(); }

// ------------------------------------------------------------ 1D tables
// Legendre P_n and P_n' at x by the three-term recurrence.
static void legendre(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int j = 2; j <= n; ++j) {
    double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

// Gauss-Legendre points and weights on [0,1] (Newton on P_n).
static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double t = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, t, &p, &dp);
      double dt = p / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double p, dp;
    legendre(n, t, &p, &dp);
    x[i] = 0.5 * (t + 1.0);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2/((1-t^2)P'^2) halved for [0,1]
  }
}

// Gauss-Lobatto nodes on [0,1]: end points and roots of P_k' (Newton using the
// Legendre equation (1-x^2)P'' = 2xP' - k(k+1)P).
static void gauss_lobatto(int k, double* x) {
  x[0] = 0.0;
  x[k] = 1.0;
  for (int j = 1; j < k; ++j) {
    double t = -std::cos(M_PI * j / k);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(k, t, &p, &dp);
      double d2p = (2.0 * t * dp - k * (k + 1.0) * p) / (1.0 - t * t);
      double dt = dp / d2p;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[j] = 0.5 * (t + 1.0);
  }
}

static double lagrange_val(const double* nodes, int n, int l, double x) {
  double v = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != l) v *= (x - nodes[m]) / (nodes[l] - nodes[m]);
  return v;
}

static double lagrange_der(const double* nodes, int n, int l, double x) {
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == l) continue;
    double t = 1.0 / (nodes[l] - nodes[m]);
    for (int q = 0; q < n; ++q)
      if (q != l && q != m) t *= (x - nodes[q]) / (nodes[l] - nodes[q]);
    s += t;
  }
  return s;
}

static void make_basis_uncached(int k, Basis1D<double>* b64, Basis1D<float>* b32);

void make_basis(int k, Basis1D<double>* b64, Basis1D<float>* b32) {
  struct Cache {
    Basis1D<double> d[kMaxDegree + 1];
    Basis1D<float> f[kMaxDegree + 1];
    Cache() {
      for (int j = 1; j <= kMaxDegree; ++j) make_basis_uncached(j, &d[j], &f[j]);
    }
  };
  static const Cache cache;
  *b64 = cache.d[k];
  *b32 = cache.f[k];
}

static void make_basis_uncached(int k, Basis1D<double>* b64, Basis1D<float>* b32) {
  const int n = k + 1;
  double gl[kMaxN] = {0}, gx[kMaxN] = {0}, gw[kMaxN] = {0};
  gauss_lobatto(k, gl);
  gauss_legendre(n, gx, gw);
  // For odd n both point sets contain the centre 1/2; store it exactly, so
  // that S's middle row is exactly the unit row (the sweeps skip it).
  if (n % 2 == 1) gl[n / 2] = gx[n / 2] = 0.5;
  Basis1D<double> b;
  std::memset(&b, 0, sizeof(b));
  for (int q = 0; q < n; ++q) {
    for (int l = 0; l < n; ++l) {
      b.S[q][l] = lagrange_val(gl, n, l, gx[q]);
      b.DS[q][l] = lagrange_der(gl, n, l, gx[q]);
      b.Dg[q][l] = lagrange_der(gx, n, l, gx[q]);
    }
  }
  if (n % 2 == 1) {
    // the central Lagrange polynomial of a symmetric point set is even about
    // 1/2: its derivative there vanishes exactly
    b.Dg[n / 2][n / 2] = 0.0;
    b.DS[n / 2][n / 2] = 0.0;
  }
  for (int l = 0; l < n; ++l) {
    b.gl[l] = gl[l];
    double p = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != l) p *= gl[l] - gl[m];
    b.gl_scale[l] = 1.0 / p;
    b.gx[l] = gx[l];
    b.gw[l] = gw[l];
  }
  *b64 = b;
  for (int i = 0; i < kMaxN; ++i) {
    for (int j = 0; j < kMaxN; ++j) {
      b32->S[i][j] = (float)b.S[i][j];
      b32->Dg[i][j] = (float)b.Dg[i][j];
      b32->DS[i][j] = (float)b.DS[i][j];
    }
    b32->gl[i] = (float)b.gl[i];
    b32->gl_scale[i] = (float)b.gl_scale[i];
    b32->gx[i] = (float)b.gx[i];
    b32->gw[i] = (float)b.gw[i];
  }
}

// ------------------------------------------------------------ numbering
namespace {
struct Key {
  int32_t v[4];
  int32_t w[4];
  int n;
  bool operator==(const Key& o) const {
    if (n != o.n) return false;
    for (int i = 0; i < n; ++i)
      if (v[i] != o.v[i] || w[i] != o.w[i]) return false;
    return true;
  }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = 1469598103934665603ull ^ (uint64_t)k.n;
    for (int i = 0; i < k.n; ++i) {
      h = (h ^ (uint64_t)(uint32_t)k.v[i]) * 1099511628211ull;
      h = (h ^ (uint64_t)(uint32_t)k.w[i]) * 1099511628211ull;
    }
    return (size_t)(h ^ (h >> 29));
  }
};
struct FaceKey {
  int32_t v[4];
  int n;
  bool operator==(const FaceKey& o) const {
    for (int i = 0; i < n; ++i)
      if (v[i] != o.v[i]) return false;
    return n == o.n;
  }
};
struct FaceHash {
  size_t operator()(const FaceKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < k.n; ++i) h = (h ^ (uint64_t)(uint32_t)k.v[i]) * 1099511628211ull;
    return (size_t)(h ^ (h >> 31));
  }
};
}  // namespace

int number_nodes(const int32_t* cells, int64_t nc, int64_t nv, int dim, int k,
                 const uint8_t* dirichlet_vertex, HostNumbering* out) {
  const int n1 = k + 1;
  const int nloc = dim == 2 ? n1 * n1 : n1 * n1 * n1;
  const int ncorner = 1 << dim;
  // corner weights W[i][v] = prod_d (bit_d(v) ? m_d : k - m_d)
  std::vector<int> W((size_t)nloc * ncorner);
  std::vector<int> mi((size_t)nloc * 3);
  for (int i = 0; i < nloc; ++i) {
    int m[3] = {i % n1, (i / n1) % n1, i / (n1 * n1)};
    for (int d = 0; d < 3; ++d) mi[i * 3 + d] = m[d];
    for (int v = 0; v < ncorner; ++v) {
      int w = 1;
      for (int d = 0; d < dim; ++d) w *= ((v >> d) & 1) ? m[d] : (k - m[d]);
      W[(size_t)i * ncorner + v] = w;
    }
  }
  out->cell_nodes.assign((size_t)nc * nloc, -1);
  out->owner_cell.clear();
  out->owner_local.clear();
  std::vector<int32_t> vertex_node((size_t)nv, -1);
  std::unordered_map<Key, int32_t, KeyHash> shared;
  shared.reserve((size_t)nc * (nloc - 1) / 2 + 16);
  int64_t next = 0;
  for (int64_t c = 0; c < nc; ++c) {
    const int32_t* cv = cells + c * ncorner;
    for (int i = 0; i < nloc; ++i) {
      int nz = 0;
      int32_t vv[8];
      int32_t ww[8];
      for (int v = 0; v < ncorner; ++v) {
        int w = W[(size_t)i * ncorner + v];
        if (w) {
          vv[nz] = cv[v];
          ww[nz] = w;
          ++nz;
        }
      }
      int32_t id;
      if (nz == 1) {
        int32_t& slot = vertex_node[vv[0]];
        if (slot < 0) {
          slot = (int32_t)next++;
          out->owner_cell.push_back((int32_t)c);
          out->owner_local.push_back(i);
        }
        id = slot;
      } else if (nz == ncorner) {
        id = (int32_t)next++;
        out->owner_cell.push_back((int32_t)c);
        out->owner_local.push_back(i);
      } else {
        Key key;
        key.n = nz;
        int order[4] = {0, 1, 2, 3};
        std::sort(order, order + nz, [&](int a, int b) { return vv[a] < vv[b]; });
        for (int j = 0; j < nz; ++j) {
          key.v[j] = vv[order[j]];
          key.w[j] = ww[order[j]];
        }
        auto it = shared.find(key);
        if (it == shared.end()) {
          id = (int32_t)next++;
          shared.emplace(key, id);
          out->owner_cell.push_back((int32_t)c);
          out->owner_local.push_back(i);
        } else {
          id = it->second;
        }
      }
      out->cell_nodes[(size_t)c * nloc + i] = id;
    }
  }
  if (next > INT32_MAX / 16) {
    set_error("too many nodes for 32-bit indices");
    return NNMG_INVALID_ARG;
  }
  out->n_nodes = next;
  out->constrained.assign((size_t)next, 0);
  if (!dirichlet_vertex) return NNMG_OK;
  // boundary faces: faces of exactly one cell
  std::unordered_map<FaceKey, int32_t, FaceHash> faces;
  faces.reserve((size_t)nc * dim * 2);
  auto face_key = [&](int64_t c, int a, int s) {
    FaceKey f;
    f.n = 0;
    for (int v = 0; v < ncorner; ++v)
      if (((v >> a) & 1) == s) f.v[f.n++] = cells[c * ncorner + v];
    std::sort(f.v, f.v + f.n);
    return f;
  };
  for (int64_t c = 0; c < nc; ++c)
    for (int a = 0; a < dim; ++a)
      for (int s = 0; s < 2; ++s) faces[face_key(c, a, s)] += 1;
  for (int64_t c = 0; c < nc; ++c) {
    for (int a = 0; a < dim; ++a) {
      for (int s = 0; s < 2; ++s) {
        FaceKey f = face_key(c, a, s);
        if (faces[f] != 1) continue;
        bool flagged = true;
        for (int j = 0; j < f.n; ++j) flagged = flagged && dirichlet_vertex[f.v[j]];
        if (!flagged) continue;
        for (int i = 0; i < nloc; ++i)
          if (mi[i * 3 + a] == s * k)
            out->constrained[out->cell_nodes[(size_t)c * nloc + i]] = 1;
      }
    }
  }
  return NNMG_OK;
}

// ------------------------------------------------------------ buckets
void build_buckets(const double* vertices, const int32_t* cells, int64_t nc, int dim,
                   BucketGrid* g, std::vector<double>* aabb) {
  const int ncorner = 1 << dim;
  double glo[3] = {1e300, 1e300, 1e300}, ghi[3] = {-1e300, -1e300, -1e300};
  aabb->assign((size_t)nc * 6, 0.0);
  for (int64_t c = 0; c < nc; ++c) {
    for (int d = 0; d < dim; ++d) {
      double lo = 1e300, hi = -1e300;
      for (int v = 0; v < ncorner; ++v) {
        double x = vertices[(size_t)cells[c * ncorner + v] * dim + d];
        lo = std::min(lo, x);
        hi = std::max(hi, x);
      }
      (*aabb)[c * 6 + d] = lo;
      (*aabb)[c * 6 + 3 + d] = hi;
      glo[d] = std::min(glo[d], lo);
      ghi[d] = std::max(ghi[d], hi);
    }
  }
  double span = 0.0, vol = 1.0;
  for (int d = 0; d < dim; ++d) {
    span = std::max(span, ghi[d] - glo[d]);
  }
  g->geo.eps = 1e-9 * span;
  for (int d = 0; d < dim; ++d) {
    glo[d] -= 2 * g->geo.eps;
    ghi[d] += 2 * g->geo.eps;
    vol *= ghi[d] - glo[d];
  }
  double w = std::pow(vol / (double)std::max<int64_t>(nc, 1), 1.0 / dim);
  int64_t nbt = 1;
  for (int d = 0; d < 3; ++d) {
    if (d < dim) {
      g->geo.nb[d] = std::max(1, (int)std::ceil((ghi[d] - glo[d]) / w));
      g->geo.lo[d] = glo[d];
      g->geo.inv_w[d] = g->geo.nb[d] / (ghi[d] - glo[d]);
    } else {
      g->geo.nb[d] = 1;
      g->geo.lo[d] = 0.0;
      g->geo.inv_w[d] = 0.0;
    }
    nbt *= g->geo.nb[d];
  }
  auto bidx = [&](int d, double x) {
    int b = (int)std::floor((x - g->geo.lo[d]) * g->geo.inv_w[d]);
    return std::min(std::max(b, 0), g->geo.nb[d] - 1);
  };
  std::vector<int32_t> count((size_t)nbt + 1, 0);
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      for (int64_t b = 0; b < nbt; ++b) count[b + 1] += count[b];
      g->start = count;
      g->cells.assign((size_t)count[nbt], 0);
    }
    std::vector<int32_t> fill = pass == 1 ? g->start : std::vector<int32_t>();
    for (int64_t c = 0; c < nc; ++c) {
      int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) {
        lo[d] = bidx(d, (*aabb)[c * 6 + d] - g->geo.eps);
        hi[d] = bidx(d, (*aabb)[c * 6 + 3 + d] + g->geo.eps);
      }
      for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
          for (int x = lo[0]; x <= hi[0]; ++x) {
            int64_t b = x + (int64_t)g->geo.nb[0] * (y + (int64_t)g->geo.nb[1] * z);
            if (pass == 0)
              count[b + 1]++;
            else
              g->cells[fill[b]++] = (int32_t)c;
          }
    }
  }
}

// ------------------------------------------------------------ dense SPD
// Blocked right-looking Cholesky (lower, row-major) with the trailing update
// split over host threads, then A^-1 column by column from L and L^T.
bool dense_spd_inverse(std::vector<double>& a, int n, std::vector<double>* inv) {
  const int nb = 64;
  unsigned nt = std::max(1u, std::thread::hardware_concurrency());
  auto par = [&](int64_t lo, int64_t hi, auto fn) {
    int64_t m = hi - lo;
    if (m <= 0) return;
    unsigned t = (unsigned)std::min<int64_t>(nt, m);
    std::vector<std::thread> th;
    for (unsigned i = 0; i < t; ++i) {
      th.emplace_back([&, i]() {
        for (int64_t r = lo + i; r < hi; r += t) fn(r);
      });
    }
    for (auto& x : th) x.join();
  };
  double* A = a.data();
  for (int k0 = 0; k0 < n; k0 += nb) {
    int k1 = std::min(n, k0 + nb);
    // factor the diagonal block
    for (int j = k0; j < k1; ++j) {
      double s = A[(size_t)j * n + j];
      for (int p = k0; p < j; ++p) s -= A[(size_t)j * n + p] * A[(size_t)j * n + p];
      if (!(s > 0.0)) return false;
      double ljj = std::sqrt(s);
      A[(size_t)j * n + j] = ljj;
      for (int i = j + 1; i < k1; ++i) {
        double t = A[(size_t)i * n + j];
        for (int p = k0; p < j; ++p) t -= A[(size_t)i * n + p] * A[(size_t)j * n + p];
        A[(size_t)i * n + j] = t / ljj;
      }
    }
    // panel below: L21 = A21 L11^-T
    par(k1, n, [&](int64_t i) {
      double* ri = A + (size_t)i * n;
      for (int j = k0; j < k1; ++j) {
        double t = ri[j];
        const double* rj = A + (size_t)j * n;
        for (int p = k0; p < j; ++p) t -= ri[p] * rj[p];
        ri[j] = t / rj[j];
      }
    });
    // trailing update A22 -= L21 L21^T (lower triangle)
    par(k1, n, [&](int64_t i) {
      double* ri = A + (size_t)i * n;
      for (int64_t j = k1; j <= i; ++j) {
        const double* rj = A + (size_t)j * n;
        double t = 0.0;
        for (int p = k0; p < k1; ++p) t += ri[p] * rj[p];
        ri[j] -= t;
      }
    });
  }
  // U = L^T (row-major) for the backward solves
  std::vector<double> U((size_t)n * n, 0.0);
  par(0, n, [&](int64_t i) {
    for (int j = 0; j <= i; ++j) U[(size_t)j * n + i] = A[(size_t)i * n + j];
  });
  inv->assign((size_t)n * n, 0.0);
  par(0, n, [&](int64_t col) {
    std::vector<double> y((size_t)n, 0.0);
    for (int64_t i = col; i < n; ++i) {       // L y = e_col
      const double* ri = A + (size_t)i * n;
      double t = (i == col) ? 1.0 : 0.0;
      for (int64_t p = col; p < i; ++p) t -= ri[p] * y[p];
      y[i] = t / ri[i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {    // L^T x = y
      const double* ui = U.data() + (size_t)i * n;
      double t = y[i];
      for (int64_t p = i + 1; p < n; ++p) t -= ui[p] * y[p];
      y[i] = t / ui[i];
    }
    for (int64_t i = 0; i < n; ++i) (*inv)[(size_t)i * n + col] = y[i];
  });
  return true;
}

}  // namespace nnmg
