// C ABI of the library: context creation (mesh, tables, gauge, DOF maps,
// device layout), parameter updates, and the thin entry points over the
// assembly, factorisation and solver modules.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"

using namespace ieti;

struct ieti_ctx {
  Ctx c;
};

namespace {

template <typename T>
ieti_status dalloc(Ctx* c, T** p, size_t count) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e);
    return IETI_ERR_OOM;
  }
  c->allocs.push_back({q, bytes});
  *p = (T*)q;
  return IETI_OK;
}

template <typename T>
ieti_status upload(Ctx* c, T** p, const std::vector<T>& h) {
  ieti_status r = dalloc(c, p, h.size());
  if (r != IETI_OK) return r;
  if (!h.empty()) IETI_CUDA_TRY(c, cudaMemcpy(*p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return IETI_OK;
}

#define TRY(x)                       \
  do {                               \
    ieti_status r__ = (x);           \
    if (r__ != IETI_OK) return r__;  \
  } while (0)

void compute_scaling(Ctx* c, std::vector<double>& scale) {
  // rho-scaling of Eq. (10): the row of the multiplier coupling k and l is
  // weighted in k's block by nu_l / (nu_k + nu_l)
  const Topology& t = c->topo;
  scale.assign(c->tot_iv, 0.0);
  for (int64_t l = 0; l < (int64_t)t.dual_edges.size(); ++l) {
    int k1 = t.dual_pair[l * 4], i1 = t.dual_pair[l * 4 + 1];
    int k2 = t.dual_pair[l * 4 + 2], i2 = t.dual_pair[l * 4 + 3];
    double n1 = t.subs[k1].I_nu[i1], n2 = t.subs[k2].I_nu[i2];
    scale[c->sd_host[k1].iv + i1] = n2 / (n1 + n2);
    scale[c->sd_host[k2].iv + i2] = n1 / (n1 + n2);
  }
}

// true if every patch map is an axis-aligned affine map: unit weights and
// control point (i, j, k) of each patch at (x0 + L0 g_i, y0 + L1 g_j, z0 + L2 g_k)
// with g the Greville abscissae of the patch's knot vectors (the only control
// nets of an open uniform knot vector that give such a map)
// the source parameters hold everything the kind reads for every load case
std::string check_source(int kind, const std::vector<double>& src, int nrhs, int np) {
  switch (kind) {
    case IETI_SOURCE_SINE:
    case IETI_SOURCE_TRIG:
      return (int64_t)src.size() < nrhs ? "the source needs one amplitude per load case" : "";
    case IETI_SOURCE_PATCHWISE:
      return (int64_t)src.size() < (int64_t)nrhs * np * 3 ? "the patchwise source needs nrhs x npatch x 3 values"
                                                           : "";
    case IETI_SOURCE_FOURIER: {
      size_t pos = 0;
      for (int r = 0; r < nrhs; ++r) {
        if (pos >= src.size()) return "the Fourier source parameters end before the last load case";
        const double nm = src[pos];
        if (!(nm >= 0 && nm <= 1e6) || nm != std::floor(nm)) return "bad number of Fourier modes";
        pos += 1 + 9 * (size_t)nm;
        if (pos > src.size()) return "the Fourier source parameters end before the last load case";
      }
      return "";
    }
    default:
      return "unknown source kind";
  }
}

bool nets_are_boxes(const Mesh& m, const std::vector<double>& ctrl, std::string& why) {
  if (m.per0) {
    why = "a periodic direction cannot be an affine box";
    return false;
  }
  const int p = m.p;
  for (int q = 0; q < m.npatch(); ++q) {
    int a[3];
    m.patch_abc(q, a);
    std::vector<double> g[3];
    int lo[3], cnt[3];
    for (int d = 0; d < 3; ++d) {
      const int n = m.nspan[d][a[d]];
      lo[d] = m.start[d][a[d]];
      cnt[d] = n + p;
      for (int i = 0; i < n + p; ++i) {
        double acc = 0;
        for (int l = i + 1; l <= i + p; ++l) acc += (l <= p) ? 0.0 : (l >= n + p ? 1.0 : (double)(l - p) / n);
        g[d].push_back(acc / p);
      }
    }
    auto X = [&](int i, int j, int k, int r) {
      return ctrl[(((size_t)(lo[2] + k) * m.N[1] + (lo[1] + j)) * m.N[0] + (lo[0] + i)) * 4 + r];
    };
    double x0[3] = {X(0, 0, 0, 0), X(0, 0, 0, 1), X(0, 0, 0, 2)};
    double L[3] = {X(cnt[0] - 1, 0, 0, 0) - x0[0], X(0, cnt[1] - 1, 0, 1) - x0[1], X(0, 0, cnt[2] - 1, 2) - x0[2]};
    const double tol = 1e-12 * std::max({std::fabs(L[0]), std::fabs(L[1]), std::fabs(L[2]), std::fabs(x0[0]),
                                         std::fabs(x0[1]), std::fabs(x0[2])});
    for (int k = 0; k < cnt[2]; ++k)
      for (int j = 0; j < cnt[1]; ++j)
        for (int i = 0; i < cnt[0]; ++i) {
          const double want[3] = {x0[0] + L[0] * g[0][i], x0[1] + L[1] * g[1][j], x0[2] + L[2] * g[2][k]};
          bool ok = X(i, j, k, 3) == 1.0;
          for (int r = 0; r < 3; ++r) ok = ok && std::fabs(X(i, j, k, r) - want[r]) <= tol;
          if (!ok) {
            why = "patch " + std::to_string(q) + " is not an axis-aligned affine box (control point (" +
                  std::to_string(i) + "," + std::to_string(j) + "," + std::to_string(k) + "))";
            return false;
          }
        }
  }
  return true;
}

void compute_gq(Ctx* c) {
  // per patch nu * L_c^2 / (L0 L1 L2) from the control net (axis-aligned affine maps)
  const Mesh& m = c->mesh;
  c->gq_host.assign((size_t)m.npatch() * 3, 0.0);
  for (int q = 0; q < m.npatch(); ++q) {
    int a[3];
    m.patch_abc(q, a);
    double L[3];
    for (int d = 0; d < 3; ++d) {
      int lo[3] = {m.start[0][a[0]], m.start[1][a[1]], m.start[2][a[2]]};
      int hi[3] = {lo[0], lo[1], lo[2]};
      hi[d] = lo[d] + m.nspan[d][a[d]] + m.p - 1;
      if (d == 0 && m.per0) hi[0] %= m.N[0];
      auto X = [&](int i, int j, int k) { return c->ctrl[(((size_t)k * m.N[1] + j) * m.N[0] + i) * 4 + d]; };
      L[d] = X(hi[0], hi[1], hi[2]) - X(lo[0], lo[1], lo[2]);
    }
    double vol = L[0] * L[1] * L[2];
    for (int d = 0; d < 3; ++d) c->gq_host[q * 3 + d] = c->nu[q] * L[d] * L[d] / vol;
  }
}

ieti_status build(Ctx* c, const ieti_problem_desc* desc, bool device) {
  const int p = desc->degree;
  if (p < 1 || p > 3) {
    c->err = "degree must be 1, 2 or 3";
    return IETI_ERR_INVALID_ARG;
  }
  if (desc->nrhs < 1 || desc->nrhs > MAX_RHS) {
    c->err = "nrhs must be in 1..64";
    return IETI_ERR_INVALID_ARG;
  }
  for (int d = 0; d < 3; ++d) {
    if (desc->npatch[d] < 1 || !desc->nspan_host[d]) {
      c->err = "bad patch grid";
      return IETI_ERR_INVALID_ARG;
    }
    for (int a = 0; a < desc->npatch[d]; ++a)
      if (desc->nspan_host[d][a] < 1) {
        c->err = "every slab needs at least one span";
        return IETI_ERR_INVALID_ARG;
      }
  }
  if (desc->periodic0 && desc->npatch[0] < 3) {
    c->err = "a periodic direction needs at least three patches";
    return IETI_ERR_INVALID_ARG;
  }
  Mesh& m = c->mesh;
  m.init(p, desc->npatch, desc->nspan_host, desc->periodic0 != 0);
  const int np = m.npatch();
  c->nrhs = desc->nrhs;
  c->affine = desc->affine != 0;
  c->source_kind = desc->source_kind;
  c->sub_of_patch.assign(desc->sub_of_patch_host, desc->sub_of_patch_host + np);
  c->nu.assign(desc->nu_host, desc->nu_host + np);
  for (double v : c->nu)
    if (!(v > 0)) {
      c->err = "reluctivity must be positive";
      return IETI_ERR_INVALID_ARG;
    }
  c->ctrl.assign(desc->ctrl_host, desc->ctrl_host + (size_t)m.nnode * 4);
  if (c->affine) {
    // the Kronecker assembly is exact only for boxes: check the claim
    std::string why;
    if (!nets_are_boxes(m, c->ctrl, why)) {
      c->err = "affine = 1 but " + why;
      return IETI_ERR_INVALID_ARG;
    }
  }
  if (desc->n_source_params < 0 || (desc->n_source_params > 0 && !desc->source_params_host)) {
    c->err = "bad source parameters";
    return IETI_ERR_INVALID_ARG;
  }
  c->src.assign(desc->source_params_host, desc->source_params_host + desc->n_source_params);
  {
    std::string why = check_source(c->source_kind, c->src, desc->nrhs, np);
    if (!why.empty()) {
      c->err = why;
      return IETI_ERR_INVALID_ARG;
    }
  }
  if (c->source_kind == IETI_SOURCE_TRIG && !c->affine) {
    c->err = "IETI_SOURCE_TRIG needs axis-aligned affine box patches (affine = 1)";
    return IETI_ERR_INVALID_ARG;
  }
  if (c->src.empty()) c->src.push_back(0.0);
  for (int q = 0; q < np; ++q)
    if (c->sub_of_patch[q] < 0) {
      c->err = "negative subdomain id";
      return IETI_ERR_INVALID_ARG;
    }
  build_tables(m, c->tab);
  for (int d = 0; d < 3; ++d) build_gram(m, c->tab, d, c->gram[d]);
  int code = 0;
  std::string msg = build_topology(m, c->sub_of_patch, c->nu, NB, c->topo, &code);
  if (!msg.empty()) {
    c->err = msg;
    return (ieti_status)code;
  }
  Topology& t = c->topo;
  c->nsub = t.nsub;
  c->m_r = (int64_t)t.dual_edges.size();
  c->n_gp = (int64_t)t.primal_edges.size();

  // ---- per-subdomain layout
  c->sd_host.resize(c->nsub);
  int64_t oA = 0, oKp = 0, oKpp = 0, oS = 0, oL = 0, oD = 0, orv = 0, opv = 0, oiv = 0, wsz_ii = 0;
  for (int k = 0; k < c->nsub; ++k) {
    const SubDofs& s = t.subs[k];
    SubDev& d = c->sd_host[k];
    int nIp = (int)(ceil_div(s.nI, NB) * NB);
    d.nVp = s.nVp;
    d.nI = s.nI;
    d.nP = s.nP;
    d.n = s.nVp + nIp;
    if (d.n == 0) d.n = NB;
    d.nblk = d.n / NB;
    d.A = oA; oA += (int64_t)d.n * d.n;
    d.Kp = oKp; oKp += (int64_t)d.n * d.nP;
    d.Kpp = oKpp; oKpp += (int64_t)d.nP * d.nP;
    d.ldI = (int)(ceil_div(d.nI, 4) * 4);
    d.S = oS; oS += (int64_t)d.ldI * d.nI;
    c->max_ldI = std::max(c->max_ldI, d.ldI);
    d.linv = oL; oL += (int64_t)d.nblk * NB * NB;
    d.dof = oD; oD += d.n + d.nP;
    d.rv = orv; orv += d.n;
    d.pv = opv; opv += d.nP;
    d.iv = oiv; oiv += d.nI;
    wsz_ii += (int64_t)(d.n - d.nVp) * d.nI;
    c->max_n = std::max(c->max_n, d.n);
    c->max_nI = std::max(c->max_nI, d.nI);
    c->max_nP = std::max(c->max_nP, d.nP);
    c->max_nblk = std::max(c->max_nblk, d.nblk);
  }
  c->tot_A = oA; c->tot_Kp = oKp; c->tot_Kpp = oKpp; c->tot_S = oS; c->tot_linv = oL; c->tot_dof = oD;
  c->tot_rv = orv; c->tot_pv = opv; c->tot_iv = oiv;

  // ---- DOF tables
  std::vector<DofDev> dof(oD);
  std::vector<int64_t> r_edge(oD, -1);
  std::vector<int32_t> I_dual(oiv), P_glob(opv);
  std::vector<double> I_sign(oiv);
  auto fill = [&](int64_t pos, int64_t e) {
    int dd, i, j, kk;
    m.edge_decode(e, dd, i, j, kk);
    dof[pos] = {dd, i, j, kk};
    r_edge[pos] = e;
  };
  for (int k = 0; k < c->nsub; ++k) {
    const SubDofs& s = t.subs[k];
    const SubDev& d = c->sd_host[k];
    for (int64_t i = 0; i < d.n + d.nP; ++i) dof[d.dof + i] = {-1, 0, 0, 0};
    for (int i = 0; i < s.nV; ++i) fill(d.dof + i, s.V[i]);
    for (int i = 0; i < s.nI; ++i) {
      fill(d.dof + d.nVp + i, s.I[i]);
      I_dual[d.iv + i] = (int32_t)s.I_dual[i];
      I_sign[d.iv + i] = s.I_sign[i];
    }
    for (int i = 0; i < s.nP; ++i) {
      fill(d.dof + d.n + i, s.Pr[i]);
      P_glob[d.pv + i] = (int32_t)s.P_glob[i];
    }
  }
  std::vector<double> scale;
  compute_scaling(c, scale);
  // ---- patch codes: patch-local edge -> local DOF index of its subdomain
  std::vector<int32_t> loc(m.nedge, -1);
  std::vector<int64_t> pc_off(np + 1, 0);
  for (int q = 0; q < np; ++q) pc_off[q + 1] = pc_off[q] + m.patch_nedge(q);
  std::vector<int32_t> pcode(pc_off[np], -1);
  for (int k = 0; k < c->nsub; ++k) {
    const SubDofs& s = t.subs[k];
    const SubDev& d = c->sd_host[k];
    for (int i = 0; i < s.nV; ++i) loc[s.V[i]] = i;
    for (int i = 0; i < s.nI; ++i) loc[s.I[i]] = d.nVp + i;
    for (int i = 0; i < s.nP; ++i) loc[s.Pr[i]] = d.n + i;
    for (int q : s.patches) {
      int64_t pos = pc_off[q];
      for (int dd = 0; dd < 3; ++dd) {
        int e[3];
        m.patch_edge_ext(q, dd, e);
        for (int kk = 0; kk < e[2]; ++kk)
          for (int j = 0; j < e[1]; ++j)
            for (int i = 0; i < e[0]; ++i) pcode[pos++] = loc[m.patch_edge_gid(q, dd, i, j, kk)];
      }
    }
    for (int64_t e : s.V) loc[e] = -1;
    for (int64_t e : s.I) loc[e] = -1;
    for (int64_t e : s.Pr) loc[e] = -1;
  }
  // ---- elements
  c->elem_host.clear();
  for (int q = 0; q < np; ++q) {
    int a[3];
    m.patch_abc(q, a);
    for (int s2 = 0; s2 < m.nspan[2][a[2]]; ++s2)
      for (int s1 = 0; s1 < m.nspan[1][a[1]]; ++s1)
        for (int s0 = 0; s0 < m.nspan[0][a[0]]; ++s0) {
          c->elem_host.push_back(q);
          c->elem_host.push_back(s0);
          c->elem_host.push_back(s1);
          c->elem_host.push_back(s2);
        }
  }
  c->nelem = (int64_t)c->elem_host.size() / 4;
  // ---- non-homogeneous Dirichlet data: boundary coefficients and the
  // elements that touch a Dirichlet face (the only ones the lifting changes)
  c->gD_host.clear();
  c->belem_host.clear();
  if (c->source_kind == IETI_SOURCE_TRIG) {
    std::string why = boundary_projection_trig(m, c->tab, c->ctrl, c->gD_host);
    if (!why.empty()) {
      c->err = why;
      return IETI_ERR_INVALID_ARG;
    }
    for (int64_t e = 0; e < c->nelem; ++e) {
      int a[3];
      m.patch_abc(c->elem_host[4 * e], a);
      bool touch = false;
      for (int d = 0; d < 3; ++d) {
        const int s = c->elem_host[4 * e + 1 + d];
        touch = touch || (a[d] == 0 && s == 0) || (a[d] == m.P[d] - 1 && s == m.nspan[d][a[d]] - 1);
      }
      if (touch) c->belem_host.push_back((int32_t)e);
    }
  }
  c->nbelem = (int64_t)c->belem_host.size();
  // ---- coarse contributors (CSR by coarse DOF)
  std::vector<int64_t> pcsr_off(c->n_gp + 1, 0);
  for (int k = 0; k < c->nsub; ++k)
    for (int i = 0; i < t.subs[k].nP; ++i) pcsr_off[t.subs[k].P_glob[i] + 1]++;
  for (int64_t g = 0; g < c->n_gp; ++g) pcsr_off[g + 1] += pcsr_off[g];
  std::vector<int2> pcsr(pcsr_off[c->n_gp]);
  {
    std::vector<int64_t> fillp(pcsr_off.begin(), pcsr_off.end() - 1);
    for (int k = 0; k < c->nsub; ++k)
      for (int i = 0; i < t.subs[k].nP; ++i) pcsr[fillp[t.subs[k].P_glob[i]]++] = make_int2(k, i);
  }
  compute_gq(c);
  // slab lookup per direction
  std::vector<int32_t> slab_of[3], startspan[3], nspan_v[3];
  for (int d = 0; d < 3; ++d) {
    slab_of[d].assign(m.N[d], 0);
    for (int x = 0; x < m.N[d]; ++x) {
      int a = 0;
      for (int b = 0; b < m.P[d]; ++b)
        if (m.start[d][b] <= x) a = b;
      slab_of[d][x] = a;
    }
    startspan[d].assign(m.start[d].begin(), m.start[d].end());
    startspan[d].insert(startspan[d].end(), m.spanoff[d].begin(), m.spanoff[d].end());
    nspan_v[d].assign(m.nspan[d].begin(), m.nspan[d].end());
  }

  c->host_only = !device;
  if (!device) return IETI_OK;
  c->syrk_tc = false;   // the CUDA-core trailing update (tensor cores: IETI_DEBUG_SYRK_TC)
  c->autotune = true;
  {
    int dev = 0, optin = 48 * 1024;
    IETI_CUDA_TRY(c, cudaGetDevice(&dev));
    IETI_CUDA_TRY(c, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    TRY(assemble_kernel_attrs(c, optin));
    TRY(flux_kernel_attrs(c, optin));
    TRY(solve_kernel_attrs(c, optin));
    TRY(factor_kernel_attrs(c));
    TRY(syrk_tc_attrs(c));
    TRY(dep_sweep_attrs(c));
    if ((size_t)c->max_ldI * sizeof(double) * 2 > (size_t)optin) {
      c->err = "interface block too large for the shared-memory staging of the local products";
      return IETI_ERR_INVALID_ARG;
    }
  }
  // ---- device uploads
  TRY(upload(c, &c->d_sd, c->sd_host));
  TRY(upload(c, &c->d_dof, dof));
  TRY(upload(c, &c->d_r_edge, r_edge));
  TRY(upload(c, &c->d_I_dual, I_dual));
  TRY(upload(c, &c->d_I_sign, I_sign));
  TRY(upload(c, &c->d_I_scale, scale));
  TRY(upload(c, &c->d_P_glob, P_glob));
  TRY(upload(c, &c->d_pair, t.dual_pair));
  TRY(upload(c, &c->d_patch_code, pcode));
  TRY(upload(c, &c->d_patch_code_off, pc_off));
  if (c->affine) {
    // the separable loads of box patches sum the patch contributions of every
    // local DOF in a fixed order (ascending patch-local edge): no atomics, so
    // repeated assemblies give bit-identical loads
    const int64_t nslot = c->tot_rv + c->tot_pv;
    std::vector<int64_t> gofs(nslot + 1, 0), gbase(std::max<int64_t>(nslot, 1), 0);
    std::vector<int32_t> gstride(std::max<int64_t>(nslot, 1), 0);
    auto slot_of = [&](int q, int32_t code) -> int64_t {
      const SubDev& d = c->sd_host[c->sub_of_patch[q]];
      return code < d.n ? d.rv + code : c->tot_rv + d.pv + (code - d.n);
    };
    for (int q = 0; q < np; ++q)
      for (int64_t g = pc_off[q]; g < pc_off[q + 1]; ++g)
        if (pcode[g] >= 0) gofs[slot_of(q, pcode[g]) + 1]++;
    for (int64_t t = 0; t < nslot; ++t) gofs[t + 1] += gofs[t];
    std::vector<int64_t> glist(std::max<int64_t>(gofs[nslot], 1)), fillp(gofs.begin(), gofs.end() - 1);
    for (int q = 0; q < np; ++q)
      for (int64_t g = pc_off[q]; g < pc_off[q + 1]; ++g)
        if (pcode[g] >= 0) glist[fillp[slot_of(q, pcode[g])]++] = g;
    for (int k = 0; k < c->nsub; ++k) {
      const SubDev& d = c->sd_host[k];
      for (int i = 0; i < d.n; ++i) {
        gbase[d.rv + i] = RV(d, i, 0, c->nrhs);
        gstride[d.rv + i] = d.n;
      }
      for (int i = 0; i < d.nP; ++i) {
        gbase[c->tot_rv + d.pv + i] = PV(d, i, 0, c->nrhs);
        gstride[c->tot_rv + d.pv + i] = d.nP;
      }
    }
    TRY(upload(c, &c->d_sep_gofs, gofs));
    TRY(upload(c, &c->d_sep_glist, glist));
    TRY(upload(c, &c->d_sep_gbase, gbase));
    TRY(upload(c, &c->d_sep_gstride, gstride));
    c->sep_nslot = nslot;
    c->sep_npl = pc_off[np];
  }
  TRY(upload(c, &c->d_sub_of_patch, c->sub_of_patch));
  TRY(upload(c, &c->d_elem, c->elem_host));
  if (!c->gD_host.empty()) {
    TRY(upload(c, &c->d_gD, c->gD_host));
    TRY(upload(c, &c->d_belem, c->belem_host));
  }
  {
    std::vector<int64_t> eoff(np + 1, 0);
    for (int q = 0; q < np; ++q) eoff[q + 1] = eoff[q] + m.nelem(q);
    TRY(upload(c, &c->d_patch_eoff, eoff));
    TRY(dalloc(c, &c->d_flux_out, (size_t)2 * np * MAX_RHS));
    TRY(dalloc(c, &c->d_flux_amp, MAX_RHS));
  }
  for (int d = 0; d < 3; ++d) {
    TRY(upload(c, &c->d_tabN[d], c->tab.N[d]));
    TRY(upload(c, &c->d_tabdN[d], c->tab.dN[d]));
    TRY(upload(c, &c->d_tabD[d], c->tab.D[d]));
    TRY(upload(c, &c->d_gram[d], c->gram[d].g));
    TRY(upload(c, &c->d_slab_of[d], slab_of[d]));
    TRY(upload(c, &c->d_start[d], startspan[d]));
    TRY(upload(c, &c->d_nspan[d], nspan_v[d]));
  }
  TRY(upload(c, &c->d_wq, c->tab.wq));
  TRY(upload(c, &c->d_ctrl, c->ctrl));
  TRY(upload(c, &c->d_nu, c->nu));
  TRY(upload(c, &c->d_src, c->src));
  TRY(upload(c, &c->d_gq, c->gq_host));
  TRY(upload(c, &c->d_pcsr, pcsr));
  TRY(upload(c, &c->d_pcsr_off, pcsr_off));
  TRY(upload(c, &c->d_primal_edges, t.primal_edges));

  const int nr = c->nrhs;
  TRY(dalloc(c, &c->K64, c->tot_A));
  double* Lb;
  TRY(dalloc(c, &Lb, c->tot_A));
  c->L = Lb;
  double* Li;
  TRY(dalloc(c, &Li, c->tot_linv));
  c->Linv = Li;
  TRY(dalloc(c, &c->Kp64, c->tot_Kp));
  TRY(dalloc(c, &c->Phi, c->tot_Kp));
  double* psi;
  TRY(dalloc(c, &psi, std::max<int64_t>(c->tot_Kp, 1)));
  c->Psi = psi;
  TRY(dalloc(c, &c->Kpp64, c->tot_Kpp));
  double *Sb, *Wb;
  TRY(dalloc(c, &Sb, c->tot_S));
  TRY(dalloc(c, &Wb, c->tot_S));
  c->S = Sb;
  c->W = Wb;
  TRY(dalloc(c, &c->jr, c->tot_rv * nr));
  TRY(dalloc(c, &c->jp, std::max<int64_t>(c->tot_pv, 1) * nr));
  int64_t wsz = std::max<int64_t>(c->tot_rv * std::max<int64_t>(nr, c->max_nP), wsz_ii);
  for (int i = 0; i < 3; ++i) {
    double* w;
    TRY(dalloc(c, &w, wsz));
    c->wr[i] = w;
    TRY(dalloc(c, &c->wr64[i], c->tot_rv * nr));
  }
  // apply_F / apply_precond accept up to MAX_RHS columns
  for (int i = 0; i < 2; ++i) TRY(dalloc(c, &c->wi[i], c->tot_iv * MAX_RHS));
  TRY(dalloc(c, &c->wq_part, std::max<int64_t>(c->tot_pv, 1) * MAX_RHS));
  for (int i = 0; i < 2; ++i) TRY(dalloc(c, &c->wc[i], std::max<int64_t>(c->n_gp, 1) * MAX_RHS));
  for (int i = 0; i < 8; ++i) TRY(dalloc(c, &c->wlam[i], std::max<int64_t>(c->m_r, 1) * nr));
  TRY(dalloc(c, &c->wlam_acc, std::max<int64_t>(c->m_r, 1) * nr));
  TRY(dalloc(c, &c->wvf, 5 * std::max<int64_t>(c->m_r, 1) * nr));
  TRY(dalloc(c, &c->wscal, 16 * MAX_RHS));
  TRY(dalloc(c, &c->wred, 512 * MAX_RHS));
  TRY(dalloc(c, &c->wflag, 64));
  TRY(dalloc(c, &c->wglob, m.nedge * nr));
  TRY(dalloc(c, &c->whist, 2 * 4096));
  TRY(dalloc(c, &c->wnorm, MAX_RHS));
  TRY(dalloc(c, &c->wres_r, c->tot_rv * nr));
  TRY(dalloc(c, &c->wres_p, std::max<int64_t>(c->tot_pv, 1) * nr));
  TRY(dalloc(c, &c->wxp, std::max<int64_t>(c->tot_pv, 1) * nr));
  double* wyk;
  TRY(dalloc(c, &wyk, c->tot_rv * nr));
  c->wyk = wyk;
  {
    // sweep ranges of the r-vector solves: the whole r range, and the r_I rows
    // (panels from nVp / 64 on; a subdomain without r_I DOFs takes no part)
    std::vector<SolveDesc> dh(2 * (size_t)c->nsub);
    int min_b0 = 1 << 30;
    for (int k = 0; k < c->nsub; ++k) {
      const SubDev& s = c->sd_host[k];
      dh[k] = SolveDesc{s.rv * nr, 0, s.n, nr, 0};
      dh[c->nsub + k] = SolveDesc{s.rv * nr + s.nVp, s.nVp / NB, s.n, s.nI > 0 ? nr : 0, 0};
      if (s.nI > 0) min_b0 = std::min(min_b0, s.nVp / NB);
    }
    c->min_b0_I = min_b0 == (1 << 30) ? c->max_nblk : min_b0;
    TRY(upload(c, &c->d_desc_rv, dh));
  }
  TRY(dep_sweep_alloc(c));
  char* desc_buf;
  TRY(dalloc(c, &desc_buf, 64 * (size_t)c->nsub + 64));
  c->d_descbuf = desc_buf;
  const int64_t ldc = ceil_div(std::max<int64_t>(c->n_gp, 1), NB) * NB;
  TRY(dalloc(c, &c->SPi, ldc * ldc));
  TRY(dalloc(c, &c->SPiInv, 5 * ldc * ldc + ldc * NB + 64));
  TRY(dalloc(c, &c->d_err, 4));
  IETI_CUDA_TRY(c, cudaMallocHost(&c->h_err, sizeof(int) * 4));
  TRY(iface_alloc(c));
  TRY(syrk_tc_alloc(c));
  return IETI_OK;
}

}  // namespace

extern "C" {

ieti_status ieti_create(const ieti_problem_desc* desc, ieti_ctx** out) {
  if (!desc || !out) return IETI_ERR_INVALID_ARG;
  *out = nullptr;
  ieti_ctx* x = new (std::nothrow) ieti_ctx();
  if (!x) return IETI_ERR_OOM;
  ieti_status r = build(&x->c, desc, true);
  *out = x;   // returned even on error so that ieti_last_error can be read
  return r;
}

ieti_status ieti_create_host(const ieti_problem_desc* desc, ieti_ctx** out) {
  if (!desc || !out) return IETI_ERR_INVALID_ARG;
  *out = nullptr;
  ieti_ctx* x = new (std::nothrow) ieti_ctx();
  if (!x) return IETI_ERR_OOM;
  ieti_status r = build(&x->c, desc, false);
  *out = x;
  return r;
}

ieti_status ieti_set_params(ieti_ctx* x, const double* nu, const double* src, int nsrc) {
  if (!x) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  const int np = c->mesh.npatch();
  if (c->host_only) {
    c->err = "context was created without a device";
    return IETI_ERR_STATE;
  }
  if (nu) {
    for (int q = 0; q < np; ++q)
      if (!(nu[q] > 0)) {
        c->err = "reluctivity must be positive";
        return IETI_ERR_INVALID_ARG;
      }
    c->nu.assign(nu, nu + np);
    update_nu(c->mesh, c->sub_of_patch, c->nu, c->topo);
    std::vector<double> scale;
    compute_scaling(c, scale);
    compute_gq(c);
    IETI_CUDA_TRY(c, cudaMemcpy(c->d_nu, c->nu.data(), sizeof(double) * np, cudaMemcpyHostToDevice));
    IETI_CUDA_TRY(c, cudaMemcpy(c->d_I_scale, scale.data(), sizeof(double) * scale.size(), cudaMemcpyHostToDevice));
    IETI_CUDA_TRY(c, cudaMemcpy(c->d_gq, c->gq_host.data(), sizeof(double) * c->gq_host.size(), cudaMemcpyHostToDevice));
  }
  if (src) {
    std::vector<double> v(src, src + std::max(nsrc, 0));
    std::string why = nsrc < 0 ? std::string("bad source parameters") : check_source(c->source_kind, v, c->nrhs, np);
    if (!why.empty()) {
      c->err = why;
      return IETI_ERR_INVALID_ARG;
    }
    if (nsrc > (int)c->src.size()) {
      // grow the device copy
      double* d;
      ieti_status r = dalloc(c, &d, nsrc);
      if (r != IETI_OK) return r;
      c->d_src = d;
    }
    c->src.assign(src, src + nsrc);
    IETI_CUDA_TRY(c, cudaMemcpy(c->d_src, c->src.data(), sizeof(double) * nsrc, cudaMemcpyHostToDevice));
  }
  c->assembled = false;
  c->factored = false;
  return IETI_OK;
}

ieti_status ieti_assemble(ieti_ctx* x, void* stream) {
  if (!x) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  if (c->host_only) {
    c->err = "context was created without a device";
    return IETI_ERR_STATE;
  }
  ieti_status r = assemble_all(c, (cudaStream_t)stream);
  if (r != IETI_OK) return r;
  c->assembled = true;
  c->factored = false;
  return IETI_OK;
}

ieti_status ieti_factor(ieti_ctx* x, ieti_precision prec, void* stream) {
  if (!x) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  if (!c->assembled) {
    c->err = "ieti_factor before ieti_assemble";
    return IETI_ERR_STATE;
  }
  if (prec != IETI_FP64 && prec != IETI_FP32_IR) {
    c->err = "unknown precision";
    return IETI_ERR_INVALID_ARG;
  }
  c->prec = prec;
  ieti_status r = factor_all(c, (cudaStream_t)stream);
  c->factored = (r == IETI_OK);
  return r;
}

ieti_status ieti_apply_F(ieti_ctx* x, const double* lam, double* y, int nrhs, void* stream) {
  if (!x || !lam || !y) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  if (!c->factored) {
    c->err = "ieti_apply_F before ieti_factor";
    return IETI_ERR_STATE;
  }
  if (nrhs < 1 || nrhs > MAX_RHS) {
    c->err = "nrhs out of range";
    return IETI_ERR_INVALID_ARG;
  }
  return apply_F(c, lam, y, nrhs, c->prec == IETI_FP32_IR, (cudaStream_t)stream);
}

ieti_status ieti_apply_F_implicit(ieti_ctx* x, const double* lam, double* y, int nrhs, void* stream) {
  if (!x || !lam || !y) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  if (!c->factored) {
    c->err = "ieti_apply_F_implicit before ieti_factor";
    return IETI_ERR_STATE;
  }
  if (nrhs != c->nrhs) {
    c->err = "ieti_apply_F_implicit: nrhs must equal the context's number of load cases";
    return IETI_ERR_INVALID_ARG;
  }
  const cudaStream_t st = (cudaStream_t)stream;
  IETI_CUDA_TRY(c, cudaMemsetAsync(c->d_dep_err, 0, sizeof(int), st));
  ieti_status r = apply_F_implicit(c, lam, y, st);
  if (r != IETI_OK) return r;
  IETI_CUDA_TRY(c, cudaMemcpyAsync(c->h_err + 1, c->d_dep_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  IETI_CUDA_TRY(c, cudaStreamSynchronize(st));
  if (c->h_err[1]) {
    c->err = "a triangular-sweep wait timed out";
    return IETI_ERR_TIMEOUT;
  }
  return IETI_OK;
}

ieti_status ieti_apply_precond(ieti_ctx* x, const double* r, double* z, int nrhs, void* stream) {
  if (!x || !r || !z) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  if (!c->factored) {
    c->err = "ieti_apply_precond before ieti_factor";
    return IETI_ERR_STATE;
  }
  if (nrhs < 1 || nrhs > MAX_RHS) {
    c->err = "nrhs out of range";
    return IETI_ERR_INVALID_ARG;
  }
  return apply_precond(c, r, z, nrhs, c->prec == IETI_FP32_IR, (cudaStream_t)stream);
}

ieti_status ieti_solve(ieti_ctx* x, const double* lam0, double tol, int maxit, double tol_field, double* a,
                       double* lam_out, ieti_solve_info* info, void* stream) {
  if (!x || !a) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  if (!c->factored) {
    c->err = "ieti_solve before ieti_factor";
    return IETI_ERR_STATE;
  }
  if (!(tol > 0) || maxit < 1) {
    c->err = "tol must be > 0 and maxit >= 1";
    return IETI_ERR_INVALID_ARG;
  }
  return solve_all(c, lam0, tol, maxit, tol_field, a, lam_out, info, (cudaStream_t)stream);
}

ieti_status ieti_interface_rhs(ieti_ctx* x, double* b, void* stream) {
  if (!x || !b) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  if (!c->factored) {
    c->err = "ieti_interface_rhs before ieti_factor";
    return IETI_ERR_STATE;
  }
  return interface_rhs(c, c->jr, c->jp, b, c->wc[1], c->nrhs, (cudaStream_t)stream);
}

ieti_status ieti_eval_B(ieti_ctx* x, const double* a, int nrhs, int ref_kind, const double* amp, double* nB2,
                        double* err2, double* Bq, void* stream) {
  if (!x) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  if (c->host_only) {
    c->err = "context was created without a device";
    return IETI_ERR_STATE;
  }
  if (!a || !nB2 || nrhs < 1 || nrhs > MAX_RHS || ref_kind < IETI_BREF_NONE || ref_kind > IETI_BREF_TRIG ||
      (ref_kind != IETI_BREF_NONE && !amp)) {
    c->err = "ieti_eval_B: bad arguments";
    return IETI_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t need = c->nelem * nrhs * 2;
  if (need > c->flux_part_cap) {
    double* p = nullptr;
    TRY(dalloc(c, &p, need));
    c->d_flux_part = p;
    c->flux_part_cap = need;
  }
  std::vector<double> amp_h(MAX_RHS, 0.0);
  if (ref_kind != IETI_BREF_NONE) std::copy(amp, amp + nrhs, amp_h.begin());
  IETI_CUDA_TRY(c, cudaMemcpyAsync(c->d_flux_amp, amp_h.data(), sizeof(double) * MAX_RHS, cudaMemcpyHostToDevice, st));
  TRY(eval_flux(c, a, nrhs, ref_kind, c->d_flux_amp, c->d_flux_part, c->d_flux_out, Bq, st));
  const int np = c->mesh.npatch();
  std::vector<double> out((size_t)2 * np * nrhs);
  IETI_CUDA_TRY(c, cudaMemcpyAsync(out.data(), c->d_flux_out, sizeof(double) * out.size(), cudaMemcpyDeviceToHost, st));
  IETI_CUDA_TRY(c, cudaStreamSynchronize(st));
  std::copy(out.begin(), out.begin() + (size_t)np * nrhs, nB2);
  if (err2) std::copy(out.begin() + (size_t)np * nrhs, out.end(), err2);
  return IETI_OK;
}

ieti_status ieti_query(const ieti_ctx* x, ieti_sizes* o) {
  if (!x || !o) return IETI_ERR_INVALID_ARG;
  const Ctx* c = &x->c;
  std::memset(o, 0, sizeof(*o));
  o->nedge = c->mesh.nedge;
  o->nnode = c->mesh.nnode;
  o->n_dirichlet = c->topo.n_dirichlet;
  o->n_tree = c->topo.n_tree;
  o->n_gauged = c->topo.n_gauged;
  o->m_r = c->m_r;
  o->n_gp = c->n_gp;
  o->nsub = c->nsub;
  o->nrhs = c->nrhs;
  for (const SubDofs& s : c->topo.subs) {
    o->max_nr = std::max<int64_t>(o->max_nr, s.nV + s.nI);
    o->max_nI = std::max<int64_t>(o->max_nI, s.nI);
    o->sum_nr2 += (int64_t)(s.nV + s.nI) * (s.nV + s.nI);
    o->sum_nI2 += (int64_t)s.nI * s.nI;
  }
  for (const DeviceBuf& b : c->allocs) o->bytes_device += (int64_t)b.bytes;
  o->tree_rerun = c->topo.rerun ? 1 : 0;
  return IETI_OK;
}

ieti_status ieti_get_dofmap(const ieti_ctx* x, int which, int sub, int64_t* out, int64_t cap, int64_t* count) {
  if (!x || !count) return IETI_ERR_INVALID_ARG;
  const Ctx* c = &x->c;
  const Topology& t = c->topo;
  std::vector<int64_t> v;
  if (which == 0) v.assign(t.tree.begin(), t.tree.end());
  else if (which == 1) v.assign(t.weight.begin(), t.weight.end());
  else if (which == 2) v = t.primal_edges;
  else if (which == 3) v = t.dual_edges;
  else {
    if (sub < 0 || sub >= t.nsub) return IETI_ERR_INVALID_ARG;
    const SubDofs& s = t.subs[sub];
    if (which == 4) v = s.V;
    else if (which == 5) v = s.I;
    else if (which == 6) v = s.Pr;
    else if (which == 7) for (double sg : s.I_sign) v.push_back((int64_t)sg);
    else return IETI_ERR_INVALID_ARG;
  }
  *count = (int64_t)v.size();
  if (out) std::memcpy(out, v.data(), sizeof(int64_t) * std::min<int64_t>(cap, (int64_t)v.size()));
  return IETI_OK;
}

ieti_status ieti_get_boundary_data(const ieti_ctx* x, double* out, int64_t cap, int64_t* count) {
  if (!x || !count || cap < 0 || (cap > 0 && !out)) return IETI_ERR_INVALID_ARG;
  const Ctx* c = &x->c;
  const int64_t n = (int64_t)c->gD_host.size();
  *count = n;
  std::copy(c->gD_host.begin(), c->gD_host.begin() + std::min(n, cap), out);
  return IETI_OK;
}

ieti_status ieti_get_block(ieti_ctx* x, int which, int sub, double* out, int64_t cap, int64_t* rows_out,
                           int64_t* cols_out) {
  if (!x || sub < 0) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  if (sub >= c->nsub) return IETI_ERR_INVALID_ARG;
  const SubDev& s = c->sd_host[sub];
  const int nV = c->topo.subs[sub].nV, nI = s.nI, nP = s.nP, nr = c->nrhs;
  std::vector<int> ridx;   // rows of the r block without padding
  for (int i = 0; i < nV; ++i) ridx.push_back(i);
  for (int i = 0; i < nI; ++i) ridx.push_back(s.nVp + i);
  int64_t R = 0, C = 0;
  switch (which) {
    case 0: R = C = (int64_t)ridx.size(); break;
    case 1: R = (int64_t)ridx.size(); C = nP; break;
    case 2: R = C = nP; break;
    case 3: R = (int64_t)ridx.size(); C = nr; break;
    case 4: R = nP; C = nr; break;
    case 5: case 6: R = C = nI; break;
    default: return IETI_ERR_INVALID_ARG;
  }
  if (rows_out) *rows_out = R;
  if (cols_out) *cols_out = C;
  if (!out) return IETI_OK;
  if (cap < R * C) return IETI_ERR_INVALID_ARG;
  if ((which >= 5) && !c->factored) {
    c->err = "factor first";
    return IETI_ERR_STATE;
  }
  IETI_CUDA_TRY(c, cudaDeviceSynchronize());
  std::vector<double> tmp;
  auto fetch = [&](const void* base, int64_t off, int64_t cnt, bool f32) -> ieti_status {
    tmp.resize(cnt);
    if (f32) {
      std::vector<float> tf(cnt);
      IETI_CUDA_TRY(c, cudaMemcpy(tf.data(), (const float*)base + off, sizeof(float) * cnt, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < cnt; ++i) tmp[i] = tf[i];
    } else {
      IETI_CUDA_TRY(c, cudaMemcpy(tmp.data(), (const double*)base + off, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
    }
    return IETI_OK;
  };
  ieti_status r;
  if (which == 0) {
    if ((r = fetch(c->K64, s.A, (int64_t)s.n * s.n, false)) != IETI_OK) return r;
    for (int64_t j = 0; j < C; ++j)
      for (int64_t i = 0; i < R; ++i) out[i + R * j] = tmp[ridx[i] + (int64_t)s.n * ridx[j]];
  } else if (which == 1) {
    if ((r = fetch(c->Kp64, s.Kp, (int64_t)s.n * nP, false)) != IETI_OK) return r;
    for (int64_t j = 0; j < C; ++j)
      for (int64_t i = 0; i < R; ++i) out[i + R * j] = tmp[ridx[i] + (int64_t)s.n * j];
  } else if (which == 2) {
    if ((r = fetch(c->Kpp64, s.Kpp, (int64_t)nP * nP, false)) != IETI_OK) return r;
    std::memcpy(out, tmp.data(), sizeof(double) * R * C);
  } else if (which == 3) {
    if ((r = fetch(c->jr, s.rv * nr, (int64_t)s.n * nr, false)) != IETI_OK) return r;
    for (int64_t j = 0; j < C; ++j)
      for (int64_t i = 0; i < R; ++i) out[i + R * j] = tmp[ridx[i] + (int64_t)s.n * j];
  } else if (which == 4) {
    if ((r = fetch(c->jp, s.pv * nr, (int64_t)nP * nr, false)) != IETI_OK) return r;
    std::memcpy(out, tmp.data(), sizeof(double) * R * C);
  } else {
    const void* base = (which == 5) ? c->S : c->W;
    if ((r = fetch(base, s.S, (int64_t)s.ldI * nI, c->prec == IETI_FP32_IR)) != IETI_OK) return r;
    for (int64_t j = 0; j < C; ++j)
      for (int64_t i = 0; i < R; ++i) out[i + R * j] = tmp[i + (int64_t)s.ldI * j];
  }
  return IETI_OK;
}

ieti_status ieti_get_coarse(ieti_ctx* x, double* out, int64_t cap) {
  if (!x || !out) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  if (!c->factored) return IETI_ERR_STATE;
  const int64_t ngp = c->n_gp, ldc = ceil_div(std::max<int64_t>(ngp, 1), NB) * NB;
  if (cap < ngp * ngp) return IETI_ERR_INVALID_ARG;
  std::vector<double> tmp(ldc * ldc);
  IETI_CUDA_TRY(c, cudaMemcpy(tmp.data(), c->SPi, sizeof(double) * ldc * ldc, cudaMemcpyDeviceToHost));
  for (int64_t j = 0; j < ngp; ++j)
    for (int64_t i = 0; i < ngp; ++i) out[i + ngp * j] = tmp[i + ldc * j];
  return IETI_OK;
}

int64_t ieti_launch_count(const ieti_ctx* x) { return x ? x->c.launches : 0; }

ieti_status ieti_debug_set(ieti_ctx* x, int what, int64_t value) {
  if (!x) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  if (c->host_only) {
    c->err = "context was created without a device";
    return IETI_ERR_STATE;
  }
  switch (what) {
    case IETI_DEBUG_WAIT_POLLS:
      return dep_set_poll_limit(c, value < 0 ? (1LL << 22) : (long long)value);
    case IETI_DEBUG_PIVOT_FAULT:
      if (value >= c->nsub) {
        c->err = "ieti_debug_set: subdomain out of range";
        return IETI_ERR_INVALID_ARG;
      }
      c->fault_pivot_sub = value < 0 ? -1 : (int)value;
      return IETI_OK;
    case IETI_DEBUG_FP64_FALLBACK:
      c->force_fallback = value != 0;
      return IETI_OK;
    case IETI_DEBUG_SYRK_TC:
      if (c->symb_ready) {   // the factorisation work lists depend on it
        c->err = "ieti_debug_set: the trailing-update path is chosen before the first factorisation";
        return IETI_ERR_STATE;
      }
      c->syrk_tc = value != 0;
      return IETI_OK;
    case IETI_DEBUG_NO_AUTOTUNE:
      c->autotune = value == 0;
      return IETI_OK;
    case IETI_DEBUG_ELEMENT_LOADS:
      c->sep_loads = value == 0;
      return IETI_OK;
    case IETI_DEBUG_SYRK_RESERVE:
      if (value >= std::max(c->sm_count, 1)) {
        c->err = "ieti_debug_set: reserve must be below the SM count";
        return IETI_ERR_INVALID_ARG;
      }
      c->syrk_reserve = value < 0 ? 24 : (int)value;
      return IETI_OK;
    default:
      c->err = "ieti_debug_set: unknown setting";
      return IETI_ERR_INVALID_ARG;
  }
}

ieti_status ieti_profile(ieti_ctx* x, int enable) {
  if (!x) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  prof_collect(c);
  c->prof.on = enable != 0;
  c->prof.mask = enable > 1 ? (unsigned)(((unsigned)enable >> 1) & ((1u << PROF_NCAT) - 1)) : ~0u;
  for (int i = 0; i < PROF_NCAT; ++i) {
    c->prof.ms[i] = 0;
    c->prof.calls[i] = 0;
  }
  return IETI_OK;
}

ieti_status ieti_profile_read(ieti_ctx* x, double* ms_host, int64_t* calls_host, int n) {
  if (!x || !ms_host || !calls_host) return IETI_ERR_INVALID_ARG;
  Ctx* c = &x->c;
  prof_collect(c);
  for (int i = 0; i < n && i < PROF_NCAT; ++i) {
    ms_host[i] = c->prof.ms[i];
    calls_host[i] = c->prof.calls[i];
  }
  return IETI_OK;
}

void ieti_destroy(ieti_ctx* x) {
  if (!x) return;
  for (DeviceBuf& b : x->c.allocs) cudaFree(b.p);
  if (x->c.h_err) cudaFreeHost(x->c.h_err);
  for (cudaEvent_t e : x->c.ev_fact)
    if (e) cudaEventDestroy(e);
  if (x->c.aux_stream) cudaStreamDestroy(x->c.aux_stream);
  for (auto& g : x->c.sgraph)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (x->c.cap_stream) cudaStreamDestroy(x->c.cap_stream);
  delete x;
}

const char* ieti_last_error(const ieti_ctx* x) { return x ? x->c.err.c_str() : "null context"; }

}  // extern "C"
