// Host-side model: mesh numbering, spline tables, tree-cotree gauge and DOF
// classes of the dual-primal method (Sec. 2, Sec. 2.2, Fig. "weights").
#include "model.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <set>
#include <tuple>

#include "../../include/ieti.h"

namespace ieti {

namespace {

// Ordering of the interior (r_V) DOFs of a subdomain for the dense blocked
// factorisation: lexicographic in the control-grid index of the edge, the
// axis with the longest extent outermost and the shortest innermost, the
// direction last. Basis functions couple only within p + 1 control indices
// in every axis, so K_rr^(k) is banded with a bandwidth of a few cross
// sections of the shortest two axes, and its Cholesky factor fills only the
// band (about 40 % of the 64 x 64 tiles on a 2 x 2 x 1-patch subdomain, where
// edge-id order fills them all). The r_I DOFs stay after all r_V DOFs.
void order_interior(const Mesh& m, std::vector<int64_t>& V) {
  if (V.size() < 2) return;
  struct Key {
    int c[3];
    int d;
    int64_t e;
  };
  std::vector<Key> key(V.size());
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
  for (size_t q = 0; q < V.size(); ++q) {
    Key& K = key[q];
    m.edge_decode(V[q], K.d, K.c[0], K.c[1], K.c[2]);
    K.e = V[q];
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], K.c[a]);
      hi[a] = std::max(hi[a], K.c[a]);
    }
  }
  int ax[3] = {0, 1, 2};
  std::stable_sort(ax, ax + 3, [&](int a, int b) { return hi[a] - lo[a] > hi[b] - lo[b]; });
  std::sort(key.begin(), key.end(), [&](const Key& x, const Key& y) {
    for (int a = 0; a < 3; ++a)
      if (x.c[ax[a]] != y.c[ax[a]]) return x.c[ax[a]] < y.c[ax[a]];
    if (x.d != y.d) return x.d < y.d;
    return x.e < y.e;
  });
  for (size_t q = 0; q < V.size(); ++q) V[q] = key[q].e;
}

}  // namespace

// ---------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------

void Mesh::init(int p_, const int P_[3], const int* const nsp[3], bool periodic0) {
  p = p_;
  per0 = periodic0;
  for (int d = 0; d < 3; ++d) {
    P[d] = P_[d];
    nspan[d].assign(nsp[d], nsp[d] + P[d]);
    start[d].resize(P[d]);
    spanoff[d].resize(P[d]);
    int acc = 0, sacc = 0;
    for (int a = 0; a < P[d]; ++a) {
      start[d][a] = acc;
      spanoff[d][a] = sacc;
      acc += nspan[d][a] + p - 1;
      sacc += nspan[d][a];
    }
    N[d] = acc + ((d == 0 && per0) ? 0 : 1);
    nspan_tot[d] = sacc;
  }
  int64_t tot = 0;
  for (int d = 0; d < 3; ++d) {
    for (int e = 0; e < 3; ++e) ext[d][e] = N[e];
    if (!(d == 0 && per0)) ext[d][d] -= 1;
    off[d] = tot;
    tot += ext[d][0] * ext[d][1] * ext[d][2];
  }
  nedge = tot;
  nnode = (int64_t)N[0] * N[1] * N[2];
}

void Mesh::edge_decode(int64_t e, int& d, int& i, int& j, int& k) const {
  d = (e >= off[2]) ? 2 : (e >= off[1] ? 1 : 0);
  int64_t r = e - off[d];
  i = (int)(r % ext[d][0]);
  r /= ext[d][0];
  j = (int)(r % ext[d][1]);
  k = (int)(r / ext[d][1]);
}

void Mesh::edge_nodes(int64_t e, int64_t& tail, int64_t& head) const {
  int d, i, j, k;
  edge_decode(e, d, i, j, k);
  tail = node_id(i, j, k);
  int h[3] = {i, j, k};
  h[d] += 1;
  if (d == 0) h[0] = wrap0(h[0]);
  head = node_id(h[0], h[1], h[2]);
}

bool Mesh::edge_dirichlet(int64_t e) const {
  int d, ijk[3];
  edge_decode(e, d, ijk[0], ijk[1], ijk[2]);
  for (int c = 0; c < 3; ++c) {
    if (c == d || (c == 0 && per0)) continue;
    if (ijk[c] == 0 || ijk[c] == N[c] - 1) return true;
  }
  return false;
}

bool Mesh::node_boundary(int64_t n) const {
  int ijk[3] = {(int)(n % N[0]), (int)((n / N[0]) % N[1]), (int)(n / ((int64_t)N[0] * N[1]))};
  for (int c = 0; c < 3; ++c) {
    if (c == 0 && per0) continue;
    if (ijk[c] == 0 || ijk[c] == N[c] - 1) return true;
  }
  return false;
}

void Mesh::patch_edge_ext(int q, int d, int e[3]) const {
  int a[3];
  patch_abc(q, a);
  for (int c = 0; c < 3; ++c) e[c] = nspan[c][a[c]] + p - (c == d ? 1 : 0);
}

int64_t Mesh::patch_nedge(int q) const {
  int64_t s = 0;
  for (int d = 0; d < 3; ++d) {
    int e[3];
    patch_edge_ext(q, d, e);
    s += (int64_t)e[0] * e[1] * e[2];
  }
  return s;
}

int64_t Mesh::patch_edge_gid(int q, int d, int i, int j, int k) const {
  int a[3];
  patch_abc(q, a);
  return edge_id(d, wrap0(start[0][a[0]] + i), start[1][a[1]] + j, start[2][a[2]] + k);
}

int Mesh::nelem(int q) const {
  int a[3];
  patch_abc(q, a);
  return nspan[0][a[0]] * nspan[1][a[1]] * nspan[2][a[2]];
}

// ---------------------------------------------------------------------------
// spline tables: nonzero B-splines on a span by the triangular recurrence
// (left/right differences), derivatives through the edge basis
// D_i = p/(t_{i+p+1}-t_{i+1}) N_{i+1,p-1}, with N_i' = D_{i-1} - D_i.
// ---------------------------------------------------------------------------

static std::vector<double> open_knots(int p, int n) {
  std::vector<double> t;
  for (int i = 0; i <= p; ++i) t.push_back(0.0);
  for (int i = 1; i < n; ++i) t.push_back((double)i / n);
  for (int i = 0; i <= p; ++i) t.push_back(1.0);
  return t;
}

// values of the q+1 B-splines of degree q that are nonzero on knot interval
// [t[s], t[s+1]) at x: out[r] = N_{s-q+r, q}(x)
static void nonzero_basis(const std::vector<double>& t, int s, int q, double x, double* out) {
  std::vector<double> left(q + 1), right(q + 1);
  out[0] = 1.0;
  for (int j = 1; j <= q; ++j) {
    left[j] = x - t[s + 1 - j];
    right[j] = t[s + j] - x;
    double saved = 0.0;
    for (int r = 0; r < j; ++r) {
      double tmp = out[r] / (right[r + 1] + left[j - r]);
      out[r] = saved + right[r + 1] * tmp;
      saved = left[j - r] * tmp;
    }
    out[j] = saved;
  }
}

static void gauss_rule(int nq, std::vector<double>& x, std::vector<double>& w) {
  // Newton iteration on the Legendre polynomial for each root on [-1, 1]
  x.assign(nq, 0.0);
  w.assign(nq, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < nq; ++i) {
    double z = std::cos(pi * (i + 0.75) / (nq + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int k = 1; k <= nq; ++k) {
        double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
      }
      dp = nq * (z * p0 - p1) / (z * z - 1.0);
      double dz = p0 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged root
    double p0 = 1.0, p1 = 0.0;
    for (int k = 1; k <= nq; ++k) {
      double p2 = p1;
      p1 = p0;
      p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
    }
    dp = nq * (z * p0 - p1) / (z * z - 1.0);
    x[nq - 1 - i] = 0.5 * (z + 1.0);
    w[nq - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);   // (2/((1-z^2)p'^2)) * 1/2
  }
}

void build_tables(const Mesh& m, Tables1D& t) {
  const int p = m.p;
  t.nq = p + 1;
  gauss_rule(t.nq, t.xq, t.wq);
  for (int d = 0; d < 3; ++d) {
    int G = m.nspan_tot[d];
    t.N[d].assign((size_t)G * (p + 1) * t.nq, 0.0);
    t.dN[d].assign((size_t)G * (p + 1) * t.nq, 0.0);
    t.D[d].assign((size_t)G * p * t.nq, 0.0);
    for (int a = 0; a < m.P[d]; ++a) {
      int n = m.nspan[d][a];
      std::vector<double> kn = open_knots(p, n);
      for (int s = 0; s < n; ++s) {
        int g = m.spanoff[d][a] + s;
        int ks = s + p;  // knot interval index [t[ks], t[ks+1])
        for (int x = 0; x < t.nq; ++x) {
          double xi = (s + t.xq[x]) / n;
          std::vector<double> Np(p + 1), Nm(p);
          nonzero_basis(kn, ks, p, xi, Np.data());
          nonzero_basis(kn, ks, p - 1, xi, Nm.data());
          // Nm[r] = N_{ks-(p-1)+r, p-1} = N_{s+1+r, p-1}; D_{s+r} uses N_{s+r+1,p-1}
          std::vector<double> Dv(p);
          for (int r = 0; r < p; ++r) {
            int i = s + r;
            double den = kn[i + p + 1] - kn[i + 1];
            Dv[r] = p / den * Nm[r];
          }
          for (int r = 0; r <= p; ++r) {
            // local H1 function s+r: derivative D_{s+r-1} - D_{s+r}
            double dl = (r >= 1) ? Dv[r - 1] : 0.0;
            double dr = (r < p) ? Dv[r] : 0.0;
            t.N[d][((size_t)g * (p + 1) + r) * t.nq + x] = Np[r];
            t.dN[d][((size_t)g * (p + 1) + r) * t.nq + x] = dl - dr;
          }
          for (int r = 0; r < p; ++r) t.D[d][((size_t)g * p + r) * t.nq + x] = Dv[r];
        }
      }
    }
  }
}

void build_gram(const Mesh& m, const Tables1D& t, int d, Gram1D& out) {
  const int p = m.p, nq = t.nq;
  out.band = 2 * p + 1;
  out.nfun_max = 0;
  for (int a = 0; a < m.P[d]; ++a) out.nfun_max = std::max(out.nfun_max, m.nspan[d][a] + p);
  out.slab_off.resize(m.P[d]);
  size_t per = (size_t)9 * out.nfun_max * out.band;
  out.g.assign(per * m.P[d], 0.0);
  for (int a = 0; a < m.P[d]; ++a) {
    out.slab_off[a] = (int64_t)(per * a);
    double* G = out.g.data() + per * a;
    int n = m.nspan[d][a];
    for (int s = 0; s < n; ++s) {
      int g = m.spanoff[d][a] + s;
      for (int x = 0; x < nq; ++x) {
        double w = t.wq[x] / n;
        // family values of the functions nonzero on span s: index, value
        for (int f1 = 0; f1 < 3; ++f1) {
          int n1 = (f1 == 2) ? p : p + 1;
          for (int r1 = 0; r1 < n1; ++r1) {
            double v1 = (f1 == 0) ? t.N[d][((size_t)g * (p + 1) + r1) * nq + x]
                      : (f1 == 1) ? t.dN[d][((size_t)g * (p + 1) + r1) * nq + x]
                                  : t.D[d][((size_t)g * p + r1) * nq + x];
            int i = s + r1;
            for (int f2 = 0; f2 < 3; ++f2) {
              int n2 = (f2 == 2) ? p : p + 1;
              for (int r2 = 0; r2 < n2; ++r2) {
                double v2 = (f2 == 0) ? t.N[d][((size_t)g * (p + 1) + r2) * nq + x]
                          : (f2 == 1) ? t.dN[d][((size_t)g * (p + 1) + r2) * nq + x]
                                      : t.D[d][((size_t)g * p + r2) * nq + x];
                int j = s + r2;
                G[((size_t)(f1 * 3 + f2) * out.nfun_max + i) * out.band + (j - i + p)] += w * v1 * v2;
              }
            }
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// topology
// ---------------------------------------------------------------------------

namespace {

struct DSU {
  std::vector<int64_t> par;
  explicit DSU(int64_t n) : par(n) { std::iota(par.begin(), par.end(), 0); }
  int64_t root(int64_t x) {
    while (par[x] != x) {
      par[x] = par[par[x]];
      x = par[x];
    }
    return x;
  }
  bool join(int64_t a, int64_t b) {
    a = root(a);
    b = root(b);
    if (a == b) return false;
    par[b] = a;
    return true;
  }
};

int neighbour_patch(const Mesh& m, int q, int d, int side) {
  int a[3];
  m.patch_abc(q, a);
  a[d] += side ? 1 : -1;
  if (d == 0 && m.per0) {
    a[0] = (a[0] + m.P[0]) % m.P[0];
  } else if (a[d] < 0 || a[d] >= m.P[d]) {
    return -1;
  }
  return m.patch_index(a[0], a[1], a[2]);
}

// edges in the closure of face (d, side) of patch q
void face_edges(const Mesh& m, int q, int d, int side, std::vector<int64_t>& out) {
  for (int de = 0; de < 3; ++de) {
    if (de == d) continue;
    int e[3];
    m.patch_edge_ext(q, de, e);
    int lo[3] = {0, 0, 0}, hi[3] = {e[0], e[1], e[2]};
    int a[3];
    m.patch_abc(q, a);
    int fix = side ? (m.nspan[d][a[d]] + m.p - 1) : 0;
    lo[d] = fix;
    hi[d] = fix + 1;
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) out.push_back(m.patch_edge_gid(q, de, i, j, k));
  }
}

// contractibility of a union of patch cubes: connected, Euler characteristic 1,
// and no enclosed cavity (the complement in the padded grid is connected).
bool simply_connected(const Mesh& m, const std::vector<int>& members) {
  if (members.empty()) return false;
  std::set<int> mem(members.begin(), members.end());
  // connectivity over face neighbours
  std::set<int> seen{members[0]};
  std::vector<int> st{members[0]};
  while (!st.empty()) {
    int q = st.back();
    st.pop_back();
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        int nb = neighbour_patch(m, q, d, s);
        if (nb >= 0 && mem.count(nb) && !seen.count(nb)) {
          seen.insert(nb);
          st.push_back(nb);
        }
      }
  }
  if (seen.size() != mem.size()) return false;
  // Euler characteristic of the cube complex (coordinates wrap in a periodic direction 0)
  auto w0 = [&](int x) { return m.per0 ? ((x % m.P[0]) + m.P[0]) % m.P[0] : x; };
  std::set<std::tuple<int, int, int>> V;
  std::set<std::tuple<int, int, int, int>> E, F;
  for (int q : members) {
    int a[3];
    m.patch_abc(q, a);
    for (int dx = 0; dx < 2; ++dx)
      for (int dy = 0; dy < 2; ++dy)
        for (int dz = 0; dz < 2; ++dz) V.insert({w0(a[0] + dx), a[1] + dy, a[2] + dz});
    for (int d = 0; d < 3; ++d) {
      int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
      for (int s1 = 0; s1 < 2; ++s1)
        for (int s2 = 0; s2 < 2; ++s2) {
          int b[3] = {a[0], a[1], a[2]};
          b[o1] += s1;
          b[o2] += s2;
          E.insert({d, w0(b[0]), b[1], b[2]});
        }
      for (int s = 0; s < 2; ++s) {
        int b[3] = {a[0], a[1], a[2]};
        b[d] += s;
        F.insert({d, w0(b[0]), b[1], b[2]});
      }
    }
  }
  long chi = (long)V.size() - (long)E.size() + (long)F.size() - (long)members.size();
  if (chi != 1) return false;
  // cavities: flood the complement from outside (non-periodic directions padded)
  int lo0 = m.per0 ? 0 : -1, hi0 = m.per0 ? m.P[0] - 1 : m.P[0];
  auto inside = [&](int a, int b, int c) {
    return a >= 0 && a < m.P[0] && b >= 0 && b < m.P[1] && c >= 0 && c < m.P[2];
  };
  std::set<std::tuple<int, int, int>> vis;
  std::vector<std::tuple<int, int, int>> stack;
  // start from every padding cell adjacent to the boundary (outside region)
  stack.push_back({lo0, -1, -1});
  vis.insert({lo0, -1, -1});
  while (!stack.empty()) {
    auto [a, b, c] = stack.back();
    stack.pop_back();
    for (int d = 0; d < 3; ++d)
      for (int s = -1; s <= 1; s += 2) {
        int n[3] = {a, b, c};
        n[d] += s;
        if (m.per0) n[0] = ((n[0] % m.P[0]) + m.P[0]) % m.P[0];
        if (n[0] < lo0 || n[0] > hi0 || n[1] < -1 || n[1] > m.P[1] || n[2] < -1 || n[2] > m.P[2]) continue;
        auto t = std::make_tuple(n[0], n[1], n[2]);
        if (vis.count(t)) continue;
        if (inside(n[0], n[1], n[2]) && mem.count(m.patch_index(n[0], n[1], n[2]))) continue;
        vis.insert(t);
        stack.push_back(t);
      }
  }
  long n_out = 0;
  for (auto& t : vis)
    if (inside(std::get<0>(t), std::get<1>(t), std::get<2>(t))) ++n_out;
  return n_out == (long)m.npatch() - (long)members.size();
}

}  // namespace

std::string build_topology(const Mesh& m, const std::vector<int>& sub_of_patch,
                           const std::vector<double>& nu, int panel, Topology& topo, int* code) {
  const int np = m.npatch();
  int nsub = 0;
  for (int q = 0; q < np; ++q) nsub = std::max(nsub, sub_of_patch[q] + 1);
  topo.nsub = nsub;
  topo.subs.assign(nsub, SubDofs());
  for (int q = 0; q < np; ++q) topo.subs[sub_of_patch[q]].patches.push_back(q);
  for (int k = 0; k < nsub; ++k) {
    if (topo.subs[k].patches.empty()) {
      *code = IETI_ERR_INVALID_ARG;
      return "subdomain " + std::to_string(k) + " has no patch";
    }
    if (!simply_connected(m, topo.subs[k].patches)) {
      *code = IETI_ERR_NOT_SIMPLY_CONNECTED;
      return "subdomain " + std::to_string(k) + " is not a simply connected union of patches";
    }
  }
  const int64_t ne = m.nedge;
  // subdomain membership of every edge (an edge lies in at most 4 patches' closures
  // around a line, hence in at most 4 subdomains)
  std::vector<int32_t> subs_of(ne * 4, -1);
  std::vector<uint8_t> mult(ne, 0);
  std::vector<std::vector<int64_t>> sub_edges(nsub);
  for (int k = 0; k < nsub; ++k) {
    std::vector<int64_t>& se = sub_edges[k];
    for (int q : topo.subs[k].patches) {
      for (int d = 0; d < 3; ++d) {
        int e[3];
        m.patch_edge_ext(q, d, e);
        for (int kk = 0; kk < e[2]; ++kk)
          for (int j = 0; j < e[1]; ++j)
            for (int i = 0; i < e[0]; ++i) se.push_back(m.patch_edge_gid(q, d, i, j, kk));
      }
    }
    std::sort(se.begin(), se.end());
    se.erase(std::unique(se.begin(), se.end()), se.end());
    for (int64_t e : se) {
      if (mult[e] >= 4) {
        *code = IETI_ERR_INVALID_ARG;
        return "edge in more than four subdomains";
      }
      subs_of[e * 4 + mult[e]] = k;
      mult[e]++;
    }
  }
  topo.dirichlet.assign(ne, 0);
  for (int64_t e = 0; e < ne; ++e) topo.dirichlet[e] = m.edge_dirichlet(e) ? 1 : 0;

  // wire basket: in >2 subdomains, or in the closure of >= 2 facets of one subdomain
  std::vector<uint8_t> wire(ne, 0);
  for (int64_t e = 0; e < ne; ++e) wire[e] = mult[e] > 2;
  for (int k = 0; k < nsub; ++k) {
    std::vector<std::pair<int64_t, int64_t>> edge_facet;   // (edge, facet key)
    struct DirFace { int q, d, s; };
    std::vector<DirFace> dfaces;
    std::vector<int64_t> buf;
    for (int q : topo.subs[k].patches) {
      for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s) {
          int nb = neighbour_patch(m, q, d, s);
          if (nb < 0) {
            dfaces.push_back({q, d, s});
          } else if (sub_of_patch[nb] != k) {
            buf.clear();
            face_edges(m, q, d, s, buf);
            for (int64_t e : buf) edge_facet.push_back({e, (int64_t)sub_of_patch[nb]});
          }
        }
    }
    // Dirichlet facets: components of same-label boundary patch-facets
    DSU dsu((int64_t)dfaces.size());
    for (size_t a = 0; a < dfaces.size(); ++a)
      for (size_t b = a + 1; b < dfaces.size(); ++b) {
        if (dfaces[a].d != dfaces[b].d || dfaces[a].s != dfaces[b].s) continue;
        int x[3], y[3];
        m.patch_abc(dfaces[a].q, x);
        m.patch_abc(dfaces[b].q, y);
        int dist = 0;
        bool ok = true;
        for (int c = 0; c < 3; ++c) {
          int df = std::abs(x[c] - y[c]);
          if (c == 0 && m.per0) df = std::min(df, m.P[0] - df);
          if (c == dfaces[a].d && df != 0) ok = false;
          dist += df;
        }
        if (ok && dist == 1) dsu.join((int64_t)a, (int64_t)b);
      }
    for (size_t a = 0; a < dfaces.size(); ++a) {
      buf.clear();
      face_edges(m, dfaces[a].q, dfaces[a].d, dfaces[a].s, buf);
      int64_t key = (int64_t)nsub + dsu.root((int64_t)a);   // distinct from interface keys
      for (int64_t e : buf) edge_facet.push_back({e, key});
    }
    std::sort(edge_facet.begin(), edge_facet.end());
    edge_facet.erase(std::unique(edge_facet.begin(), edge_facet.end()), edge_facet.end());
    for (size_t a = 0; a < edge_facet.size();) {
      size_t b = a;
      while (b < edge_facet.size() && edge_facet[b].first == edge_facet[a].first) ++b;
      if (b - a >= 2) wire[edge_facet[a].first] = 1;
      a = b;
    }
  }

  // weights: first matching rule of Fig. "weights"
  topo.weight.assign(ne, 5);
  for (int64_t e = 0; e < ne; ++e) {
    bool dir = topo.dirichlet[e], intf = mult[e] >= 2;
    uint8_t w;
    if (dir && intf) w = 1;
    else if (mult[e] > 2) w = 2;
    else if (wire[e]) w = 3;
    else if (dir || intf) w = 4;
    else w = 5;
    topo.weight[e] = w;
  }

  // Kruskal on (weight, edge id); rerun with boundary edges first if the tree
  // is not a tree on the Dirichlet boundary (Sec. 2.2)
  int64_t nbnode = 0;
  for (int64_t n = 0; n < m.nnode; ++n) nbnode += m.node_boundary(n) ? 1 : 0;
  auto kruskal = [&](bool boundary_first) {
    std::vector<uint8_t> tree(ne, 0);
    DSU dsu(m.nnode);
    std::vector<std::vector<int64_t>> buckets(6);
    for (int64_t e = 0; e < ne; ++e) {
      int w = topo.weight[e];
      if (boundary_first && topo.dirichlet[e]) w = 1;
      buckets[w].push_back(e);   // ascending edge id inside each bucket
    }
    for (int w = 1; w <= 5; ++w)
      for (int64_t e : buckets[w]) {
        int64_t t, h;
        m.edge_nodes(e, t, h);
        if (dsu.join(t, h)) tree[e] = 1;
      }
    return tree;
  };
  auto boundary_ok = [&](const std::vector<uint8_t>& tree) {
    int64_t c = 0;
    for (int64_t e = 0; e < ne; ++e) c += (tree[e] && topo.dirichlet[e]) ? 1 : 0;
    return c == nbnode - 1;
  };
  topo.tree = kruskal(false);
  topo.rerun = false;
  if (!boundary_ok(topo.tree)) {
    topo.tree = kruskal(true);
    topo.rerun = true;
    if (!boundary_ok(topo.tree)) {
      *code = IETI_ERR_TREE_INCONSISTENT;
      return "spanning tree is not a tree on the Dirichlet boundary";
    }
  }

  // DOF classes
  topo.primal_edges.clear();
  topo.dual_edges.clear();
  std::vector<int64_t> dual_index(ne, -1), primal_index(ne, -1);
  topo.n_tree = topo.n_dirichlet = topo.n_gauged = 0;
  for (int64_t e = 0; e < ne; ++e) {
    topo.n_tree += topo.tree[e];
    topo.n_dirichlet += topo.dirichlet[e];
    bool keep = !topo.dirichlet[e] && !topo.tree[e];
    if (!keep) continue;
    topo.n_gauged++;
    if (topo.weight[e] == 2) {
      primal_index[e] = (int64_t)topo.primal_edges.size();
      topo.primal_edges.push_back(e);
    } else if (mult[e] >= 2) {
      if (mult[e] != 2) {
        *code = IETI_ERR_TREE_INCONSISTENT;
        return "a multiplier would couple more than two subdomains";
      }
      dual_index[e] = (int64_t)topo.dual_edges.size();
      topo.dual_edges.push_back(e);
    }
  }
  for (int k = 0; k < nsub; ++k) {
    SubDofs& s = topo.subs[k];
    s.V.clear(); s.I.clear(); s.Pr.clear();
    for (int64_t e : sub_edges[k]) {
      if (topo.dirichlet[e] || topo.tree[e]) continue;
      if (primal_index[e] >= 0) s.Pr.push_back(e);
      else if (dual_index[e] >= 0) s.I.push_back(e);
      else s.V.push_back(e);
    }
    order_interior(m, s.V);
    s.nV = (int)s.V.size();
    s.nI = (int)s.I.size();
    s.nP = (int)s.Pr.size();
    s.nVp = (s.nV + panel - 1) / panel * panel;
    s.n = s.nVp + s.nI;
    s.I_dual.resize(s.nI);
    s.I_sign.resize(s.nI);
    for (int i = 0; i < s.nI; ++i) {
      int64_t e = s.I[i];
      s.I_dual[i] = dual_index[e];
      int lo = std::min(subs_of[e * 4 + 0], subs_of[e * 4 + 1]);
      s.I_sign[i] = (lo == k) ? 1.0 : -1.0;
    }
    s.P_glob.resize(s.nP);
    for (int i = 0; i < s.nP; ++i) s.P_glob[i] = primal_index[s.Pr[i]];
  }
  // the two local positions of every multiplier
  topo.dual_pair.assign(topo.dual_edges.size() * 4, -1);
  for (int k = 0; k < nsub; ++k) {
    const SubDofs& s = topo.subs[k];
    for (int i = 0; i < s.nI; ++i) {
      int64_t l = s.I_dual[i];
      int slot = (s.I_sign[i] > 0) ? 0 : 2;
      topo.dual_pair[l * 4 + slot] = k;
      topo.dual_pair[l * 4 + slot + 1] = i;
    }
  }
  update_nu(m, sub_of_patch, nu, topo);
  *code = 0;
  return std::string();
}

void update_nu(const Mesh& m, const std::vector<int>& sub_of_patch, const std::vector<double>& nu,
               Topology& topo) {
  // nu of subdomain k at an interface edge: max over its patches containing the edge
  for (int k = 0; k < topo.nsub; ++k) {
    SubDofs& s = topo.subs[k];
    s.I_nu.assign(s.nI, 0.0);
    for (int i = 0; i < s.nI; ++i) {
      int d, ijk[3];
      m.edge_decode(s.I[i], d, ijk[0], ijk[1], ijk[2]);
      for (int q : s.patches) {
        int a[3];
        m.patch_abc(q, a);
        bool in = true;
        for (int c = 0; c < 3 && in; ++c) {
          int lo = m.start[c][a[c]];
          int hi = lo + m.nspan[c][a[c]] + m.p - 1 - (c == d ? 1 : 0);
          int x = ijk[c];
          if (c == 0 && m.per0) {
            int rel = ((x - lo) % m.N[0] + m.N[0]) % m.N[0];
            in = rel <= hi - lo;
          } else {
            in = x >= lo && x <= hi;
          }
        }
        if (in) s.I_nu[i] = std::max(s.I_nu[i], nu[q]);
      }
    }
  }
  (void)sub_of_patch;
}

// ---------------------------------------------------------------------------
// non-homogeneous tangential Dirichlet data (Sec. 2 boundary condition with
// the data of the manufactured field of Sec. 3)
// ---------------------------------------------------------------------------

static void trig_field(const double X[3], double A[3]) {
  const double cx = std::cos(X[0]), cy = std::cos(X[1]), cz = std::cos(X[2]);
  const double sx = std::sin(X[0]), sy = std::sin(X[1]), sz = std::sin(X[2]);
  A[0] = cy * cz * sx;
  A[1] = -2.0 * cx * cz * sy;
  A[2] = cx * cy * sz;
}

// On a face normal to axis n of an affine box patch (DF = diag(L)), the edge
// function of direction d != n whose index along n is the boundary index has
// the single tangential component D_i(xi_d) N_j(xi_e) / L_d (covariant map;
// the factor along n is 1 there), and every other edge function has a zero
// tangential trace. The face mass matrix of these traces and the moments of
// the trace of A_ana use the assembly's Gauss rule (p + 1 points per span);
// the system over all Dirichlet edges is solved by conjugate gradients with
// the diagonal as preconditioner (the mass matrix is well conditioned).
std::string boundary_projection_trig(const Mesh& m, const Tables1D& t, const std::vector<double>& ctrl,
                                     std::vector<double>& gD) {
  if (m.per0) return "the boundary data needs a box domain without a periodic direction";
  const int p = m.p, nq = t.nq;
  std::vector<int64_t> cidx((size_t)m.nedge, -1);
  std::vector<int64_t> ids;
  for (int64_t e = 0; e < m.nedge; ++e)
    if (m.edge_dirichlet(e)) {
      cidx[(size_t)e] = (int64_t)ids.size();
      ids.push_back(e);
    }
  const int64_t nb = (int64_t)ids.size();
  gD.assign((size_t)m.nedge, 0.0);
  if (nb == 0) return "";
  std::vector<std::tuple<int64_t, int64_t, double>> trip;
  std::vector<double> rhs((size_t)nb, 0.0);
  auto cp = [&](int i, int j, int k, int r) {
    return ctrl[(((size_t)k * m.N[1] + j) * m.N[0] + i) * 4 + r];
  };
  for (int q = 0; q < m.npatch(); ++q) {
    int a[3], st[3], n[3];
    m.patch_abc(q, a);
    for (int d = 0; d < 3; ++d) {
      st[d] = m.start[d][a[d]];
      n[d] = m.nspan[d][a[d]];
    }
    const double lo[3] = {cp(st[0], st[1], st[2], 0), cp(st[0], st[1], st[2], 1), cp(st[0], st[1], st[2], 2)};
    const double L[3] = {cp(st[0] + n[0] + p - 1, st[1], st[2], 0) - lo[0],
                         cp(st[0], st[1] + n[1] + p - 1, st[2], 1) - lo[1],
                         cp(st[0], st[1], st[2] + n[2] + p - 1, 2) - lo[2]};
    for (int ax = 0; ax < 3; ++ax)
      for (int side = 0; side < 2; ++side) {
        if (a[ax] != (side == 0 ? 0 : m.P[ax] - 1)) continue;
        const int bidx = side == 0 ? 0 : m.N[ax] - 1;
        const double xn = lo[ax] + (side == 0 ? 0.0 : L[ax]);
        for (int d = 0; d < 3; ++d) {
          if (d == ax) continue;
          const int e = 3 - ax - d;
          const int nloc = p * (p + 1);
          std::vector<int64_t> loc(nloc);
          std::vector<double> T((size_t)nloc * nq * nq), gq((size_t)nq * nq), wq((size_t)nq * nq);
          for (int sd = 0; sd < n[d]; ++sd)
            for (int se = 0; se < n[e]; ++se) {
              const int gd = m.spanoff[d][a[d]] + sd, ge = m.spanoff[e][a[e]] + se;
              for (int x = 0; x < nq; ++x)
                for (int y = 0; y < nq; ++y) {
                  double X[3];
                  X[ax] = xn;
                  X[d] = lo[d] + L[d] * (sd + t.xq[x]) / n[d];
                  X[e] = lo[e] + L[e] * (se + t.xq[y]) / n[e];
                  double A[3];
                  trig_field(X, A);
                  gq[(size_t)x * nq + y] = A[d];
                  wq[(size_t)x * nq + y] = t.wq[x] * t.wq[y] * (L[d] / n[d]) * (L[e] / n[e]);
                }
              for (int i = 0; i < p; ++i)
                for (int j = 0; j <= p; ++j) {
                  const int l = i * (p + 1) + j;
                  int c[3];
                  c[ax] = bidx;
                  c[d] = st[d] + sd + i;
                  c[e] = st[e] + se + j;
                  loc[l] = cidx[(size_t)m.edge_id(d, c[0], c[1], c[2])];
                  for (int x = 0; x < nq; ++x)
                    for (int y = 0; y < nq; ++y)
                      T[((size_t)l * nq + x) * nq + y] =
                          t.D[d][((size_t)gd * p + i) * nq + x] * t.N[e][((size_t)ge * (p + 1) + j) * nq + y] / L[d];
                }
              for (int l = 0; l < nloc; ++l) {
                if (loc[l] < 0) return "a boundary edge is not a Dirichlet edge";
                double f = 0;
                for (int u = 0; u < nq * nq; ++u) f += T[(size_t)l * nq * nq + u] * wq[u] * gq[u];
                rhs[(size_t)loc[l]] += f;
                for (int l2 = 0; l2 < nloc; ++l2) {
                  double v = 0;
                  for (int u = 0; u < nq * nq; ++u)
                    v += T[(size_t)l * nq * nq + u] * wq[u] * T[(size_t)l2 * nq * nq + u];
                  trip.emplace_back(loc[l], loc[l2], v);
                }
              }
            }
        }
      }
  }
  // CSR of the boundary mass matrix (duplicates summed)
  std::sort(trip.begin(), trip.end());
  std::vector<int64_t> rp((size_t)nb + 1, 0), ci;
  std::vector<double> va;
  for (size_t u = 0; u < trip.size();) {
    const int64_t r = std::get<0>(trip[u]), c = std::get<1>(trip[u]);
    double v = 0;
    while (u < trip.size() && std::get<0>(trip[u]) == r && std::get<1>(trip[u]) == c) v += std::get<2>(trip[u++]);
    ci.push_back(c);
    va.push_back(v);
    rp[(size_t)r + 1] = (int64_t)ci.size();
  }
  for (int64_t r = 0; r < nb; ++r) rp[(size_t)r + 1] = std::max(rp[(size_t)r + 1], rp[(size_t)r]);
  std::vector<double> dg((size_t)nb, 0.0);
  for (int64_t r = 0; r < nb; ++r)
    for (int64_t u = rp[(size_t)r]; u < rp[(size_t)r + 1]; ++u)
      if (ci[(size_t)u] == r) dg[(size_t)r] = va[(size_t)u];
  for (double v : dg)
    if (!(v > 0)) return "the boundary mass matrix has a non-positive diagonal";
  auto mv = [&](const std::vector<double>& x, std::vector<double>& y) {
    for (int64_t r = 0; r < nb; ++r) {
      double s = 0;
      for (int64_t u = rp[(size_t)r]; u < rp[(size_t)r + 1]; ++u) s += va[(size_t)u] * x[(size_t)ci[(size_t)u]];
      y[(size_t)r] = s;
    }
  };
  std::vector<double> x((size_t)nb, 0.0), r = rhs, z((size_t)nb), pv((size_t)nb), Ap((size_t)nb);
  auto dot = [&](const std::vector<double>& u, const std::vector<double>& v) {
    double s = 0;
    for (int64_t i = 0; i < nb; ++i) s += u[(size_t)i] * v[(size_t)i];
    return s;
  };
  const double r0 = std::sqrt(dot(r, r));
  for (int64_t i = 0; i < nb; ++i) z[(size_t)i] = r[(size_t)i] / dg[(size_t)i];
  pv = z;
  double rz = dot(r, z);
  bool ok = r0 == 0;
  for (int it = 0; it < 20000 && !ok; ++it) {
    mv(pv, Ap);
    const double al = rz / dot(pv, Ap);
    for (int64_t i = 0; i < nb; ++i) {
      x[(size_t)i] += al * pv[(size_t)i];
      r[(size_t)i] -= al * Ap[(size_t)i];
    }
    if (std::sqrt(dot(r, r)) <= 1e-13 * r0) {
      ok = true;
      break;
    }
    for (int64_t i = 0; i < nb; ++i) z[(size_t)i] = r[(size_t)i] / dg[(size_t)i];
    const double rz2 = dot(r, z);
    for (int64_t i = 0; i < nb; ++i) pv[(size_t)i] = z[(size_t)i] + rz2 / rz * pv[(size_t)i];
    rz = rz2;
  }
  if (!ok) return "the boundary projection did not converge";
  for (int64_t i = 0; i < nb; ++i) gD[(size_t)ids[(size_t)i]] = x[(size_t)i];
  return "";
}

}  // namespace ieti
