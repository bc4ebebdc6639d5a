// Host-side setup: 1D basis tables, continuous Q_k node numbering, Dirichlet
// set and the coarse-cell bucket grid for point location.
#include <algorithm>
#include <cmath>

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
// Mesh entities shared between cells: edges (2 vertices) and, in 3D, faces
// (4 vertices), each identified by its vertex set.  An entity is filed under
// its smallest vertex: per vertex a chain of the entities it is the smallest
// vertex of, holding the other vertices in increasing order, so a lookup
// walks a handful of entries.
struct Entities {
  int nv;                          // vertices per entity
  std::vector<int32_t> head;       // per mesh vertex: first entity of its chain or -1
  std::vector<int32_t> next;       // per entity: next entity in the chain or -1
  std::vector<int32_t> rest;       // per entity: its nv - 1 larger vertices
  Entities(int nverts_per, int64_t n_mesh_vertices) : nv(nverts_per), head((size_t)n_mesh_vertices, -1) {}
  int32_t size() const { return (int32_t)next.size(); }
  // id of the entity with these vertices (sorted increasingly), added if new
  int32_t find_or_add(const int32_t* v) {
    for (int32_t e = head[v[0]]; e >= 0; e = next[e]) {
      const int32_t* r = &rest[(size_t)e * (nv - 1)];
      bool eq = true;
      for (int j = 1; j < nv; ++j) eq = eq && r[j - 1] == v[j];
      if (eq) return e;
    }
    const int32_t e = size();
    next.push_back(head[v[0]]);
    head[v[0]] = e;
    for (int j = 1; j < nv; ++j) rest.push_back(v[j]);
    return e;
  }
};

// The nodes inside one kind of entity: per entity up to `cap` slots, each
// holding the node's corner weights (packed, in increasing vertex order) and
// its node number.
struct EntityNodes {
  int cap;
  std::vector<uint8_t> count;
  std::vector<uint32_t> key;
  std::vector<int32_t> node;
  EntityNodes(int c, int32_t n) : cap(c), count((size_t)n, 0), key((size_t)n * c), node((size_t)n * c) {}
  // node number of the node with weights `w` in entity e, or -1 if not numbered yet
  int32_t find(int32_t e, uint32_t w) const {
    for (int j = 0; j < count[e]; ++j)
      if (key[(size_t)e * cap + j] == w) return node[(size_t)e * cap + j];
    return -1;
  }
  // false when the entity's slots are full: more distinct nodes than a
  // conforming edge or face has (a twisted face)
  bool add(int32_t e, uint32_t w, int32_t id) {
    if (count[e] >= cap) return false;
    const size_t j = (size_t)e * cap + count[e]++;
    key[j] = w;
    node[j] = id;
    return true;
  }
};

void sort_small(int32_t* v, uint32_t* w, int n) {  // by vertex, weights alongside
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && v[j] < v[j - 1]; --j) {
      std::swap(v[j], v[j - 1]);
      std::swap(w[j], w[j - 1]);
    }
}
}  // namespace

// Continuous node numbering, first touch in (cell, local node) order: a node
// is identified by the mesh vertices whose multilinear weight at it is
// nonzero, W_v = prod_d (bit_d(v) ? m_d : k - m_d) for local node
// (m_0, m_1, m_2), together with those weights.  Vertex nodes are indexed by
// their vertex, nodes strictly inside a cell are new, edge and face nodes are
// looked up in their entity's slots.
int number_nodes(const int32_t* cells, int64_t nc, int64_t nv, int dim, int k,
                 const uint8_t* dirichlet_vertex, HostNumbering* out) {
  const int n1 = k + 1;
  const int nloc = dim == 2 ? n1 * n1 : n1 * n1 * n1;
  const int ncorner = 1 << dim;
  const int nedge = dim == 2 ? 4 : 12, nface = dim == 3 ? 6 : 0;
  // local edges: corner pairs differing in one bit; local faces: (axis a, side s) -> 2a + s
  int edge_corners[12][2], edge_of[8][8];
  {
    int e = 0;
    for (int a = 0; a < dim; ++a)
      for (int v = 0; v < ncorner; ++v)
        if (!((v >> a) & 1)) {
          edge_corners[e][0] = v;
          edge_corners[e][1] = v | (1 << a);
          edge_of[v][v | (1 << a)] = edge_of[v | (1 << a)][v] = e;
          ++e;
        }
  }
  // per local node: corners with nonzero weight, those weights, its local entity
  std::vector<int> nz((size_t)nloc), ent((size_t)nloc, -1), mi((size_t)nloc * 3);
  std::vector<int> corner((size_t)nloc * 8);
  std::vector<uint32_t> weight((size_t)nloc * 8);
  for (int i = 0; i < nloc; ++i) {
    int m[3] = {i % n1, (i / n1) % n1, i / (n1 * n1)};
    if (dim == 2) m[2] = 0;
    for (int d = 0; d < 3; ++d) mi[i * 3 + d] = m[d];
    int z = 0;
    for (int v = 0; v < ncorner; ++v) {
      int w = 1;
      for (int d = 0; d < dim; ++d) w *= ((v >> d) & 1) ? m[d] : (k - m[d]);
      if (w) {
        corner[(size_t)i * 8 + z] = v;
        weight[(size_t)i * 8 + z] = (uint32_t)w;
        ++z;
      }
    }
    nz[i] = z;
    if (z == 2) {
      ent[i] = edge_of[corner[(size_t)i * 8]][corner[(size_t)i * 8 + 1]];
    } else if (z == 4 && dim == 3) {
      for (int a = 0; a < 3; ++a)
        if (m[a] == 0 || m[a] == k) ent[i] = 2 * a + (m[a] == k ? 1 : 0);
    }
  }
  // pass 1: entity numbers of every cell's edges and faces
  Entities edges(2, nv), faces(4, nv);
  std::vector<int32_t> cell_edge((size_t)nc * nedge), cell_face((size_t)nc * nface);
  for (int64_t c = 0; c < nc; ++c) {
    const int32_t* cv = cells + c * ncorner;
    for (int e = 0; e < nedge; ++e) {
      int32_t v[2] = {cv[edge_corners[e][0]], cv[edge_corners[e][1]]};
      if (v[1] < v[0]) std::swap(v[0], v[1]);
      cell_edge[(size_t)c * nedge + e] = edges.find_or_add(v);
    }
    for (int f = 0; f < nface; ++f) {
      int32_t v[4];
      int n = 0;
      for (int u = 0; u < ncorner; ++u)
        if (((u >> (f / 2)) & 1) == (f & 1)) v[n++] = cv[u];
      auto cs = [&](int a, int b) {
        if (v[b] < v[a]) std::swap(v[a], v[b]);
      };
      cs(0, 1), cs(2, 3), cs(0, 2), cs(1, 3), cs(1, 2);   // sorting network for 4
      cell_face[(size_t)c * nface + f] = faces.find_or_add(v);
    }
  }
  // pass 2: node numbers
  const int ecap = std::max(k - 1, 1), fcap = std::max((k - 1) * (k - 1), 1);
  EntityNodes enodes(ecap, edges.size()), fnodes(fcap, faces.size());
  out->cell_nodes.assign((size_t)nc * nloc, -1);
  out->owner_cell.clear();
  out->owner_local.clear();
  {  // nodes: vertices + edge nodes + face nodes + cell interiors
    const int64_t interior = dim == 2 ? (int64_t)(k - 1) * (k - 1) : (int64_t)(k - 1) * (k - 1) * (k - 1);
    const int64_t est = nv + (int64_t)edges.size() * (k - 1) + (int64_t)faces.size() * (k - 1) * (k - 1) +
                        nc * interior;
    out->owner_cell.reserve((size_t)est);
    out->owner_local.reserve((size_t)est);
  }
  std::vector<int32_t> vertex_node((size_t)nv, -1);
  int64_t next = 0;
  auto fresh = [&](int64_t c, int i) {
    out->owner_cell.push_back((int32_t)c);
    out->owner_local.push_back(i);
    return (int32_t)next++;
  };
  for (int64_t c = 0; c < nc; ++c) {
    const int32_t* cv = cells + c * ncorner;
    for (int i = 0; i < nloc; ++i) {
      const int z = nz[i];
      int32_t id;
      if (z == 1) {
        int32_t& slot = vertex_node[cv[corner[(size_t)i * 8]]];
        if (slot < 0) slot = fresh(c, i);
        id = slot;
      } else if (z == ncorner) {
        id = fresh(c, i);
      } else {
        int32_t v[4];
        uint32_t w[4];
        for (int j = 0; j < z; ++j) {
          v[j] = cv[corner[(size_t)i * 8 + j]];
          w[j] = weight[(size_t)i * 8 + j];
        }
        sort_small(v, w, z);
        uint32_t packed = 0;
        for (int j = 0; j < z; ++j) packed |= w[j] << (8 * j);
        EntityNodes& en = z == 2 ? enodes : fnodes;
        const int32_t e = z == 2 ? cell_edge[(size_t)c * nedge + ent[i]] : cell_face[(size_t)c * nface + ent[i]];
        id = en.find(e, packed);
        if (id < 0) {
          id = fresh(c, i);
          if (!en.add(e, packed, id)) {
            set_error("non-conforming mesh: an edge or face is shared with inconsistent vertex order");
            return NNMG_BAD_MESH;
          }
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
  // boundary faces (edges in 2D): those of exactly one cell
  const Entities& bent = dim == 3 ? faces : edges;
  std::vector<int32_t> uses((size_t)bent.size(), 0);
  auto boundary_entity = [&](int64_t c, int a, int side) {
    if (dim == 3) return cell_face[(size_t)c * nface + 2 * a + side];
    return cell_edge[(size_t)c * nedge + edge_of[side << a][(side << a) | (1 << (1 - a))]];
  };
  for (int64_t c = 0; c < nc; ++c)
    for (int a = 0; a < dim; ++a)
      for (int side = 0; side < 2; ++side) uses[boundary_entity(c, a, side)]++;
  for (int64_t c = 0; c < nc; ++c) {
    for (int a = 0; a < dim; ++a) {
      for (int side = 0; side < 2; ++side) {
        if (uses[boundary_entity(c, a, side)] != 1) continue;
        bool flagged = true;
        for (int u = 0; u < ncorner; ++u)
          if (((u >> a) & 1) == side) flagged = flagged && dirichlet_vertex[cells[c * ncorner + u]];
        if (!flagged) continue;
        for (int i = 0; i < nloc; ++i)
          if (mi[i * 3 + a] == side * k) out->constrained[out->cell_nodes[(size_t)c * nloc + i]] = 1;
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

// ------------------------------------------------------------ cell colors
// Greedy coloring in cell order: a cell takes the smallest color that no
// earlier cell sharing one of its vertices took.  Cells that share no vertex
// share no node of a continuous Q_k space (edge, face and interior nodes
// belong to the entities spanned by the cell's vertices), so the cells of one
// color write disjoint output rows.  Returns the number of colors, or -1 if a
// cell would need more than 64.
int color_cells(const int32_t* cells, int64_t nc, int64_t nv, int dim, std::vector<uint8_t>* color) {
  const int nvc = 1 << dim;
  std::vector<int64_t> start((size_t)nv + 1, 0);
  for (int64_t i = 0; i < nc * nvc; ++i) start[(size_t)cells[i] + 1]++;
  for (int64_t v = 0; v < nv; ++v) start[(size_t)v + 1] += start[(size_t)v];
  std::vector<int32_t> vcells((size_t)(nc * nvc));
  std::vector<int64_t> fill(start.begin(), start.end() - 1);
  for (int64_t c = 0; c < nc; ++c)
    for (int j = 0; j < nvc; ++j) vcells[(size_t)fill[(size_t)cells[c * nvc + j]]++] = (int32_t)c;
  color->assign((size_t)nc, 0xff);
  int ncolors = 0;
  for (int64_t c = 0; c < nc; ++c) {
    uint64_t used = 0;
    for (int j = 0; j < nvc; ++j) {
      const int32_t v = cells[c * nvc + j];
      for (int64_t t = start[(size_t)v]; t < start[(size_t)v + 1]; ++t) {
        const uint8_t k = (*color)[(size_t)vcells[(size_t)t]];
        if (k != 0xff) used |= uint64_t(1) << k;
      }
    }
    if (used == ~uint64_t(0)) return -1;
    int k = 0;
    while (used >> k & 1) ++k;
    (*color)[(size_t)c] = (uint8_t)k;
    ncolors = std::max(ncolors, k + 1);
  }
  return ncolors;
}

}  // namespace nnmg
