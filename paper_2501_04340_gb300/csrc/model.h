// Host-side model of the multipatch problem: glued control mesh, 1D spline
// tables at the Gauss points, facets / wire basket / weights / Kruskal tree
// (Sec. 2, Sec. 2.2, Fig. "weights") and the per-subdomain DOF classes.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace ieti {

struct Mesh {
  int p = 0;
  int P[3] = {0, 0, 0};          // patch grid
  int N[3] = {0, 0, 0};          // glued control points per direction
  bool per0 = false;             // direction 0 periodic
  std::vector<int> nspan[3];     // spans of each slab
  std::vector<int> start[3];     // first control index of each slab
  std::vector<int> spanoff[3];   // first global span index of each slab
  int nspan_tot[3] = {0, 0, 0};
  int64_t ext[3][3];             // index extents of the edge block of direction d
  int64_t off[3];                // first edge id of direction d
  int64_t nedge = 0, nnode = 0;

  void init(int p_, const int P_[3], const int* const nsp[3], bool periodic0);
  int64_t node_id(int64_t i, int64_t j, int64_t k) const { return i + N[0] * (j + (int64_t)N[1] * k); }
  int64_t edge_id(int d, int64_t i, int64_t j, int64_t k) const {
    return off[d] + i + ext[d][0] * (j + ext[d][1] * k);
  }
  void edge_decode(int64_t e, int& d, int& i, int& j, int& k) const;
  void edge_nodes(int64_t e, int64_t& tail, int64_t& head) const;
  bool edge_dirichlet(int64_t e) const;
  bool node_boundary(int64_t n) const;
  int npatch() const { return P[0] * P[1] * P[2]; }
  void patch_abc(int q, int a[3]) const { a[0] = q % P[0]; a[1] = (q / P[0]) % P[1]; a[2] = q / (P[0] * P[1]); }
  int patch_index(int a, int b, int c) const { return a + P[0] * (b + P[1] * c); }
  int wrap0(int i) const { return per0 ? (i % N[0]) : i; }
  // number of patch-local edges of direction d (functions D in d, N elsewhere)
  void patch_edge_ext(int q, int d, int e[3]) const;
  int64_t patch_nedge(int q) const;
  // global edge id of patch-local edge (d, i, j, k)
  int64_t patch_edge_gid(int q, int d, int i, int j, int k) const;
  int nelem(int q) const;
};

// 1D tables of one direction: for each global span g and Gauss point x:
// N[(g*(p+1)+a)*nq + x], dN likewise (d/dxi in patch parameter), D[(g*p+a)*nq + x]
struct Tables1D {
  int nq = 0;
  std::vector<double> xq, wq;            // Gauss rule on [0, 1]
  std::vector<double> N[3], dN[3], D[3];
};
void build_tables(const Mesh& m, Tables1D& t);

// Banded 1D Gram matrices of one slab for the families {N, dN, D} (index 0,1,2):
// G[((f1*3+f2) * nfun_max + i) * (2p+1) + (j - i + p)] = int_0^1 f1_i f2_j dxi
struct Gram1D {
  int nfun_max = 0, band = 0;
  std::vector<double> g;                 // per slab, concatenated
  std::vector<int64_t> slab_off;         // offset of each slab's block
};
void build_gram(const Mesh& m, const Tables1D& t, int d, Gram1D& out);

struct SubDofs {
  std::vector<int> patches;
  std::vector<int64_t> V, I, Pr;         // global edge ids (sorted)
  std::vector<int64_t> I_dual;           // global dual index of each I dof
  std::vector<double> I_sign;            // +1 / -1
  std::vector<double> I_nu;              // nu of this subdomain at each I dof
  std::vector<int64_t> P_glob;           // global primal index of each primal dof
  int nV = 0, nVp = 0, nI = 0, nP = 0, n = 0;   // n = nVp + nI (dense dimension)
};

struct Topology {
  int nsub = 0;
  std::vector<uint8_t> dirichlet, tree, weight;
  std::vector<int64_t> primal_edges, dual_edges;
  std::vector<SubDofs> subs;
  // per dual dof: (k1, i1, k2, i2) with k1 < k2, local I positions
  std::vector<int32_t> dual_pair;
  bool rerun = false;
  int64_t n_tree = 0, n_dirichlet = 0, n_gauged = 0;
};

// Returns an empty string on success, else an error message; *code receives
// an ieti_status on error.
std::string build_topology(const Mesh& m, const std::vector<int>& sub_of_patch,
                           const std::vector<double>& nu, int panel, Topology& topo, int* code);
void update_nu(const Mesh& m, const std::vector<int>& sub_of_patch, const std::vector<double>& nu,
               Topology& topo);

// Coefficients (nedge, zero off the Dirichlet faces) of the boundary L2
// projection of the tangential trace of the manufactured field A_ana of Sec. 3
// onto the traces of the edge functions, over all Dirichlet faces at once.
// Axis-aligned affine box patches only (the control net is checked by the
// caller). Returns an empty string, else an error message.
std::string boundary_projection_trig(const Mesh& m, const Tables1D& t, const std::vector<double>& ctrl,
                                     std::vector<double>& gD);

}  // namespace ieti
