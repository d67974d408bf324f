// Batched assembly of the subdomain stiffness blocks and loads, Eq. (3):
//   (K)_ij = int nu curl w_j . curl w_i dV,  (j)_i = int J . w_i dV,
// with covariant Piola push-forward w = DF^-T w_hat, curl w = DF curl_hat w_hat / det DF.
//
// Two paths produce K^(k) = sum of the patch contributions of subdomain k:
//  * k_kron (axis-aligned affine patches): every dense entry is generated
//    directly from 1D Gram matrices of the spline families {N, N', D}; with a
//    constant diagonal Jacobian the Gauss quadrature of Eq. (3) factorises into
//    these 1D integrals, so the value equals the quadrature result. One thread
//    per dense entry, coalesced column-major stores, no atomics.
//  * k_elem_K (any NURBS map): one CTA per knot-span element, Gauss quadrature
//    with p+1 points per direction, element matrix in shared memory, atomic
//    scatter into the dense blocks.
// The loads always use the element path (k_elem_j).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace ieti {

struct AsmParams {
  int p, nq, nsub, nrhs, source_kind, n_src;
  int P0, P1, P2, N0, N1, N2, per0;
  const SubDev* sd;
  const DofDev* dof;
  const int32_t* patch_code;
  const int64_t* patch_code_off;
  const int32_t* sub_of_patch;
  const int32_t* elem;
  const double* tabN[3];
  const double* tabdN[3];
  const double* tabD[3];
  const double* wq;
  const double* ctrl;
  const double* nu;
  const double* src;
  const double* gq;
  double* geo;        // per element and Gauss point: X (3), weight * |det DF| DF^-1 (9); null: not kept
  int geo_ready;      // 1: geo holds the values (the geometry of the mesh is fixed)
  const double* gram[3];
  int64_t gram_per[3];
  int gram_nfun[3];
  const int32_t* slab_of[3];
  const int32_t* start[3];
  const int32_t* nspan[3];
  const int32_t* spanoff[3];
  double* K64;
  double* Kp;
  double* Kpp;
  double* jr;
  double* jp;
  int64_t eoff[3];    // first edge id of each direction (global numbering)
  int64_t eext[3][3]; // index extents of each direction's edge block
};

// ---------------------------------------------------------------------------
// shared device helpers
// ---------------------------------------------------------------------------

__device__ inline void patch_abc_d(const AsmParams& P, int q, int a[3]) {
  a[0] = q % P.P0;
  a[1] = (q / P.P0) % P.P1;
  a[2] = q / (P.P0 * P.P1);
}

// curl of a reference edge function of direction d, component c != d:
// sign and 1D families (0 = N, 1 = N', 2 = D) per direction
__device__ inline int curl_term(int d, int c, int fam[3]) {
  if (d == 0) {
    if (c == 1) { fam[0] = 2; fam[1] = 0; fam[2] = 1; return +1; }
    fam[0] = 2; fam[1] = 1; fam[2] = 0; return -1;           // c == 2
  } else if (d == 1) {
    if (c == 0) { fam[0] = 0; fam[1] = 2; fam[2] = 1; return -1; }
    fam[0] = 1; fam[1] = 2; fam[2] = 0; return +1;           // c == 2
  }
  if (c == 0) { fam[0] = 0; fam[1] = 1; fam[2] = 2; return +1; }
  fam[0] = 1; fam[1] = 0; fam[2] = 2; return -1;             // c == 1
}

// Fourier modes with integer wave numbers up to FT_KMAX per axis come from
// per-point tables of e^{2 pi i k x_d} (k = 0..FT_KMAX, one sincospi each), so
// a mode costs two complex products instead of an FP64 cosine and sine (the
// FP64 pipe of GB300 is narrow); other modes are evaluated directly.
constexpr int FT_KMAX = 8;

__device__ inline void fourier_factor(const double2* Et, double kd, double x, double& c, double& s) {
  const double a = fabs(kd);
  if (a == rint(a) && a <= FT_KMAX) {
    const double2 v = Et[(int)a];
    c = v.x;
    s = kd < 0 ? -v.y : v.y;
  } else {
    sincospi(2.0 * kd * x, &s, &c);
  }
}

// the source of load case r at the point X (tab: the point's tables, 3 x
// (FT_KMAX + 1), used by the Fourier kind)
__device__ inline void source_eval_r(const AsmParams& P, int q, int r, const double X[3], const double2* tab,
                                     double J[3]) {
  const double pi = 3.14159265358979323846;
  if (P.source_kind == IETI_SOURCE_SINE) {
    const double sx = sin(pi * X[0]), sy = sin(pi * X[1]), sz = sin(pi * X[2]);
    const double sc = P.src[r];
    J[0] = sc * 2 * pi * pi * sy * sz;
    J[1] = sc * 2 * pi * pi * sx * sz;
    J[2] = sc * 2 * pi * pi * sx * sy;
  } else if (P.source_kind == IETI_SOURCE_FOURIER) {
    int pos = 0;
    for (int rr = 0; rr < r; ++rr) pos += 1 + 9 * (int)P.src[pos];
    const int nm = (int)P.src[pos++];
    double a0 = 0, a1 = 0, a2 = 0;
    for (int m = 0; m < nm; ++m) {
      const double* M = P.src + pos + 9 * m;
      // e^{i theta}, theta = 2 pi k . X, as the product of the three axis factors
      double c0, s0, c1, s1, c2, s2;
      fourier_factor(tab, M[0], X[0], c0, s0);
      fourier_factor(tab + (FT_KMAX + 1), M[1], X[1], c1, s1);
      fourier_factor(tab + 2 * (FT_KMAX + 1), M[2], X[2], c2, s2);
      const double c01 = c0 * c1 - s0 * s1, s01 = s0 * c1 + c0 * s1;
      const double cs = c01 * c2 - s01 * s2, sn = s01 * c2 + c01 * s2;
      a0 += cs * M[3] - sn * M[6];
      a1 += cs * M[4] - sn * M[7];
      a2 += cs * M[5] - sn * M[8];
    }
    J[0] = a0; J[1] = a1; J[2] = a2;
  } else if (P.source_kind == IETI_SOURCE_TRIG) {
    // 3 A_ana of Sec. 3 (curl curl A_ana = 3 A_ana), scaled by the amplitude
    double sx, cx, sy, cy, sz, cz;
    sincos(X[0], &sx, &cx);
    sincos(X[1], &sy, &cy);
    sincos(X[2], &sz, &cz);
    const double sc = 3.0 * P.src[r];
    J[0] = sc * cy * cz * sx;
    J[1] = -2.0 * sc * cx * cz * sy;
    J[2] = sc * cx * cy * sz;
  } else {
    const int np = P.P0 * P.P1 * P.P2;
    const double* v = P.src + ((size_t)r * np + q) * 3;
    J[0] = v[0]; J[1] = v[1]; J[2] = v[2];
  }
}

// destination of the (ci, cj) entry of subdomain k (codes: [0,n) r, [n,n+nP) primal)
__device__ inline void add_entry(const AsmParams& P, const SubDev& s, int ci, int cj, double v) {
  if (ci < 0 || cj < 0) return;
  if (ci < s.n) {
    if (cj < s.n) atomicAdd(P.K64 + s.A + ci + (int64_t)s.n * cj, v);
    else atomicAdd(P.Kp + s.Kp + ci + (int64_t)s.n * (cj - s.n), v);
  } else if (cj >= s.n) {
    atomicAdd(P.Kpp + s.Kpp + (ci - s.n) + (int64_t)s.nP * (cj - s.n), v);
  }
}

// element setup common to the K and j kernels: 1D tables of the element's spans,
// local control points, geometry at the Gauss points
template <int PD>
struct ElemShared {
  static constexpr int NQ = PD + 1, NQ3 = NQ * NQ * NQ, NF = 3 * PD * (PD + 1) * (PD + 1);
  double N[3][PD + 1][NQ], dN[3][PD + 1][NQ], D[3][PD][NQ];
  double X[NQ3][3];
  double DF[NQ3][9];
  double det[NQ3], wt[NQ3];
  int code[NF];
};

template <int PD>
__device__ void elem_setup(const AsmParams& P, int e, ElemShared<PD>& sh, int& q, int& k, bool geom = true) {
  constexpr int NQ = PD + 1, NQ3 = NQ * NQ * NQ, NF = ElemShared<PD>::NF;
  const int tid = threadIdx.x;
  q = P.elem[4 * e];
  int s[3] = {P.elem[4 * e + 1], P.elem[4 * e + 2], P.elem[4 * e + 3]};
  int a[3];
  patch_abc_d(P, q, a);
  k = P.sub_of_patch[q];
  int nsp[3], g[3], st[3];
  for (int d = 0; d < 3; ++d) {
    nsp[d] = P.nspan[d][a[d]];
    g[d] = P.spanoff[d][a[d]] + s[d];
    st[d] = P.start[d][a[d]];
  }
  for (int t = tid; t < 3 * (PD + 1) * NQ; t += blockDim.x) {
    int d = t / ((PD + 1) * NQ), r = (t / NQ) % (PD + 1), x = t % NQ;
    sh.N[d][r][x] = P.tabN[d][((int64_t)g[d] * (PD + 1) + r) * NQ + x];
    sh.dN[d][r][x] = P.tabdN[d][((int64_t)g[d] * (PD + 1) + r) * NQ + x];
  }
  for (int t = tid; t < 3 * PD * NQ; t += blockDim.x) {
    int d = t / (PD * NQ), r = (t / NQ) % PD, x = t % NQ;
    sh.D[d][r][x] = P.tabD[d][((int64_t)g[d] * PD + r) * NQ + x];
  }
  // codes of the element functions (patch-local edge index -> local DOF)
  for (int f = tid; f < NF; f += blockDim.x) {
    constexpr int NFD = PD * (PD + 1) * (PD + 1);
    int d = f / NFD, r = f % NFD;
    int ext[3] = {PD + 1, PD + 1, PD + 1};
    ext[d] = PD;
    int la = r % ext[0], lb = (r / ext[0]) % ext[1], lc = r / (ext[0] * ext[1]);
    // patch-local edge extents
    int64_t doff = 0;
    int pe[3];
    for (int dd = 0; dd <= d; ++dd) {
      for (int c = 0; c < 3; ++c) pe[c] = nsp[c] + PD - (c == dd ? 1 : 0);
      if (dd < d) doff += (int64_t)pe[0] * pe[1] * pe[2];
    }
    int64_t li = doff + (s[0] + la) + (int64_t)pe[0] * ((s[1] + lb) + (int64_t)pe[1] * (s[2] + lc));
    sh.code[f] = P.patch_code[P.patch_code_off[q] + li];
  }
  __syncthreads();
  if (!geom) return;
  // geometry at the Gauss points
  for (int t = tid; t < NQ3; t += blockDim.x) {
    int x = t % NQ, y = (t / NQ) % NQ, z = t / (NQ * NQ);
    double W = 0, dW[3] = {0, 0, 0}, S[3] = {0, 0, 0}, dS[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int c = 0; c <= PD; ++c)
      for (int b = 0; b <= PD; ++b)
        for (int aa = 0; aa <= PD; ++aa) {
          int gi = st[0] + s[0] + aa;
          if (P.per0) gi %= P.N0;
          int gj = st[1] + s[1] + b, gk = st[2] + s[2] + c;
          const double* cp = P.ctrl + (((int64_t)gk * P.N1 + gj) * P.N0 + gi) * 4;
          double w = cp[3];
          double B = sh.N[0][aa][x] * sh.N[1][b][y] * sh.N[2][c][z];
          double B0 = sh.dN[0][aa][x] * sh.N[1][b][y] * sh.N[2][c][z];
          double B1 = sh.N[0][aa][x] * sh.dN[1][b][y] * sh.N[2][c][z];
          double B2 = sh.N[0][aa][x] * sh.N[1][b][y] * sh.dN[2][c][z];
          W += w * B;
          dW[0] += w * B0; dW[1] += w * B1; dW[2] += w * B2;
          for (int r = 0; r < 3; ++r) {
            double wp = w * cp[r];
            S[r] += wp * B;
            dS[r][0] += wp * B0; dS[r][1] += wp * B1; dS[r][2] += wp * B2;
          }
        }
    double Xr[3];
    for (int r = 0; r < 3; ++r) Xr[r] = S[r] / W;
    double F[9];
    for (int r = 0; r < 3; ++r)
      for (int cc = 0; cc < 3; ++cc) F[r * 3 + cc] = (dS[r][cc] - Xr[r] * dW[cc]) / W;
    double det = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                 F[2] * (F[3] * F[7] - F[4] * F[6]);
    for (int r = 0; r < 3; ++r) sh.X[t][r] = Xr[r];
    for (int r = 0; r < 9; ++r) sh.DF[t][r] = F[r];
    sh.det[t] = det;
    sh.wt[t] = P.wq[x] * P.wq[y] * P.wq[z] / ((double)nsp[0] * nsp[1] * nsp[2]);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// K: element quadrature (any geometry)
// ---------------------------------------------------------------------------

template <int PD>
__global__ void __launch_bounds__(256) k_elem_K(AsmParams P) {
  constexpr int NQ = PD + 1, NQ3 = NQ * NQ * NQ, NF = ElemShared<PD>::NF;
  constexpr int NFD = PD * (PD + 1) * (PD + 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ElemShared<PD>& sh = *reinterpret_cast<ElemShared<PD>*>(smem_raw);
  double* M = reinterpret_cast<double*>(smem_raw + sizeof(ElemShared<PD>));   // NQ3 x 9
  double* C = M + NQ3 * 9;                                                      // NF x NQ3 x 2
  const int e = blockIdx.x;
  int q, k;
  elem_setup<PD>(P, e, sh, q, k);
  const SubDev s = P.sd[k];
  const double nu = P.nu[q];
  const int tid = threadIdx.x;
  for (int t = tid; t < NQ3; t += blockDim.x) {
    const double* F = sh.DF[t];
    // dV = |det DF| dxi: a patch map may reverse orientation
    double f = nu * sh.wt[t] / fabs(sh.det[t]);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double v = 0;
        for (int r = 0; r < 3; ++r) v += F[r * 3 + a] * F[r * 3 + b];
        M[t * 9 + a * 3 + b] = f * v;
      }
  }
  // reference curls, two nonzero components per function
  for (int t = tid; t < NF * NQ3; t += blockDim.x) {
    int f = t / NQ3, qq = t % NQ3;
    int x = qq % NQ, y = (qq / NQ) % NQ, z = qq / (NQ * NQ);
    int d = f / NFD, r = f % NFD;
    int ext[3] = {PD + 1, PD + 1, PD + 1};
    ext[d] = PD;
    int la = r % ext[0], lb = (r / ext[0]) % ext[1], lc = r / (ext[0] * ext[1]);
    double c0, c1;
    if (d == 0) {        // D N N' , -D N' N   (components 1, 2)
      c0 = sh.D[0][la][x] * sh.N[1][lb][y] * sh.dN[2][lc][z];
      c1 = -sh.D[0][la][x] * sh.dN[1][lb][y] * sh.N[2][lc][z];
    } else if (d == 1) { // -N D N' , N' D N   (components 0, 2)
      c0 = -sh.N[0][la][x] * sh.D[1][lb][y] * sh.dN[2][lc][z];
      c1 = sh.dN[0][la][x] * sh.D[1][lb][y] * sh.N[2][lc][z];
    } else {             // N N' D , -N' N D   (components 0, 1)
      c0 = sh.N[0][la][x] * sh.dN[1][lb][y] * sh.D[2][lc][z];
      c1 = -sh.dN[0][la][x] * sh.N[1][lb][y] * sh.D[2][lc][z];
    }
    C[(f * NQ3 + qq) * 2 + 0] = c0;
    C[(f * NQ3 + qq) * 2 + 1] = c1;
  }
  __syncthreads();
  // 2x2 tiles (I <= J) of the symmetric element matrix
  constexpr int NT = NF / 2;
  constexpr int NTILE = NT * (NT + 1) / 2;
  for (int t = tid; t < NTILE; t += blockDim.x) {
    // decode t -> (I, J), I <= J, row-major over the upper triangle
    int I = 0, rem = t;
    while (rem >= NT - I) { rem -= NT - I; ++I; }
    int J = I + rem;
    int i0 = 2 * I, j0 = 2 * J;
    int di = i0 / NFD, dj = j0 / NFD;
    int ci[2] = {di == 0 ? 1 : 0, di == 2 ? 1 : 2};
    int cj[2] = {dj == 0 ? 1 : 0, dj == 2 ? 1 : 2};
    double e00 = 0, e01 = 0, e10 = 0, e11 = 0;
    for (int qq = 0; qq < NQ3; ++qq) {
      const double* Mq = M + qq * 9;
      double m00 = Mq[ci[0] * 3 + cj[0]], m01 = Mq[ci[0] * 3 + cj[1]];
      double m10 = Mq[ci[1] * 3 + cj[0]], m11 = Mq[ci[1] * 3 + cj[1]];
      const double* a0 = C + ((i0 + 0) * NQ3 + qq) * 2;
      const double* a1 = C + ((i0 + 1) * NQ3 + qq) * 2;
      const double* b0 = C + ((j0 + 0) * NQ3 + qq) * 2;
      const double* b1 = C + ((j0 + 1) * NQ3 + qq) * 2;
      double y00 = m00 * b0[0] + m01 * b0[1], y01 = m10 * b0[0] + m11 * b0[1];
      double y10 = m00 * b1[0] + m01 * b1[1], y11 = m10 * b1[0] + m11 * b1[1];
      e00 += a0[0] * y00 + a0[1] * y01;
      e01 += a0[0] * y10 + a0[1] * y11;
      e10 += a1[0] * y00 + a1[1] * y01;
      e11 += a1[0] * y10 + a1[1] * y11;
    }
    double ev[2][2] = {{e00, e01}, {e10, e11}};
    for (int u = 0; u < 2; ++u)
      for (int v = 0; v < 2; ++v) {
        int fi = i0 + u, fj = j0 + v;
        if (I == J && fj < fi) continue;
        int cI = sh.code[fi], cJ = sh.code[fj];
        add_entry(P, s, cI, cJ, ev[u][v]);
        if (fi != fj) add_entry(P, s, cJ, cI, ev[u][v]);
      }
  }
}

// ---------------------------------------------------------------------------
// j: element quadrature of int J . w_i (any geometry)
// ---------------------------------------------------------------------------

template <int PD>
__global__ void __launch_bounds__(256) k_elem_j(AsmParams P) {
  constexpr int NQ = PD + 1, NQ3 = NQ * NQ * NQ, NF = ElemShared<PD>::NF;
  constexpr int NFD = PD * (PD + 1) * (PD + 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ElemShared<PD>& sh = *reinterpret_cast<ElemShared<PD>*>(smem_raw);
  double* G = reinterpret_cast<double*>(smem_raw + sizeof(ElemShared<PD>));   // NQ3 x nrhs x 3
  double* As = G + (size_t)NQ3 * P.nrhs * 3;                                   // NQ3 x 9: weighted adj(DF)
  double* Xs = As + NQ3 * 9;                                                   // NQ3 x 3: the points
  // NQ3 x 3 x (FT_KMAX + 1) axis exponentials, on a 16-byte boundary (the
  // shared arrays before it end on an 8-byte one for some degrees)
  double2* Et = reinterpret_cast<double2*>((reinterpret_cast<uintptr_t>(Xs + NQ3 * 3) + 15) & ~uintptr_t(15));
  const int e = blockIdx.x;
  int q, k;
  // the geometry at the Gauss points does not change between assemblies: it
  // is computed once and kept (X and the weighted adjugate of DF)
  const bool cached = P.geo && P.geo_ready;
  elem_setup<PD>(P, e, sh, q, k, !cached);
  const SubDev s = P.sd[k];
  const int tid = threadIdx.x;
  for (int t = tid; t < NQ3; t += blockDim.x) {
    double* gk = P.geo ? P.geo + ((int64_t)e * NQ3 + t) * 12 : nullptr;
    double X[3], A[9];
    if (cached) {
      for (int r = 0; r < 3; ++r) X[r] = gk[r];
      for (int r = 0; r < 9; ++r) A[r] = gk[3 + r];
    } else {
      const double* F = sh.DF[t];
      // adjugate of DF (inverse times det)
      A[0] = F[4] * F[8] - F[5] * F[7]; A[1] = F[2] * F[7] - F[1] * F[8]; A[2] = F[1] * F[5] - F[2] * F[4];
      A[3] = F[5] * F[6] - F[3] * F[8]; A[4] = F[0] * F[8] - F[2] * F[6]; A[5] = F[2] * F[3] - F[0] * F[5];
      A[6] = F[3] * F[7] - F[4] * F[6]; A[7] = F[1] * F[6] - F[0] * F[7]; A[8] = F[0] * F[4] - F[1] * F[3];
      // |det DF| DF^-1 = sign(det) adj(DF), times the quadrature weight
      const double w = sh.det[t] < 0 ? -sh.wt[t] : sh.wt[t];
      for (int r = 0; r < 9; ++r) A[r] *= w;
      for (int r = 0; r < 3; ++r) X[r] = sh.X[t][r];
      if (gk) {
        for (int r = 0; r < 3; ++r) gk[r] = X[r];
        for (int r = 0; r < 9; ++r) gk[3 + r] = A[r];
      }
    }
    for (int r = 0; r < 9; ++r) As[t * 9 + r] = A[r];
    for (int r = 0; r < 3; ++r) Xs[t * 3 + r] = X[r];
  }
  __syncthreads();
  if (P.source_kind == IETI_SOURCE_FOURIER) {
    constexpr int KT = FT_KMAX + 1;
    for (int u = tid; u < NQ3 * 3 * KT; u += blockDim.x) {
      const int t = u / (3 * KT), d = (u / KT) % 3, kk = u % KT;
      double sn, cs;
      sincospi(2.0 * kk * Xs[t * 3 + d], &sn, &cs);
      Et[u] = make_double2(cs, sn);
    }
    __syncthreads();
  }
  // the source at every (point, load case), spread over all threads
  for (int u = tid; u < NQ3 * P.nrhs; u += blockDim.x) {
    const int t = u / P.nrhs, r = u % P.nrhs;
    double J[3];
    source_eval_r(P, q, r, Xs + t * 3, Et + t * 3 * (FT_KMAX + 1), J);
    const double* A = As + t * 9;
    for (int a = 0; a < 3; ++a)
      G[(t * P.nrhs + r) * 3 + a] = A[a * 3 + 0] * J[0] + A[a * 3 + 1] * J[1] + A[a * 3 + 2] * J[2];
  }
  __syncthreads();
  for (int t = tid; t < NF * P.nrhs; t += blockDim.x) {
    int f = t / P.nrhs, r = t % P.nrhs;
    int cf = sh.code[f];
    if (cf < 0) continue;
    int d = f / NFD, rr = f % NFD;
    int ext[3] = {PD + 1, PD + 1, PD + 1};
    ext[d] = PD;
    int la = rr % ext[0], lb = (rr / ext[0]) % ext[1], lc = rr / (ext[0] * ext[1]);
    double acc = 0;
    for (int qq = 0; qq < NQ3; ++qq) {
      int x = qq % NQ, y = (qq / NQ) % NQ, z = qq / (NQ * NQ);
      double v = (d == 0) ? sh.D[0][la][x] * sh.N[1][lb][y] * sh.N[2][lc][z]
               : (d == 1) ? sh.N[0][la][x] * sh.D[1][lb][y] * sh.N[2][lc][z]
                          : sh.N[0][la][x] * sh.N[1][lb][y] * sh.D[2][lc][z];
      acc += v * G[(qq * P.nrhs + r) * 3 + d];
    }
    if (cf < s.n) atomicAdd(P.jr + RV(s, cf, r, P.nrhs), acc);
    else atomicAdd(P.jp + PV(s, cf - s.n, r, P.nrhs), acc);
  }
}

// ---------------------------------------------------------------------------
// lifting of the loads by the boundary coefficients of non-homogeneous
// Dirichlet data: j_i -= s_r sum_f K_if gD_f (Eq. (3) for the coefficients off
// the Dirichlet faces), over the elements that touch a Dirichlet face
// ---------------------------------------------------------------------------

// the two nonzero components (into components c0i, c1i) of the reference curl
// of element function f at the Gauss point (x, y, z)
template <int PD>
__device__ inline void ref_curl(const ElemShared<PD>& sh, int f, int x, int y, int z, double& c0, double& c1,
                                int& c0i, int& c1i) {
  constexpr int NFD = PD * (PD + 1) * (PD + 1);
  const int d = f / NFD, r = f % NFD;
  int ext[3] = {PD + 1, PD + 1, PD + 1};
  ext[d] = PD;
  const int la = r % ext[0], lb = (r / ext[0]) % ext[1], lc = r / (ext[0] * ext[1]);
  c0i = d == 0 ? 1 : 0;
  c1i = d == 2 ? 1 : 2;
  if (d == 0) {        // D N N' , -D N' N   (components 1, 2)
    c0 = sh.D[0][la][x] * sh.N[1][lb][y] * sh.dN[2][lc][z];
    c1 = -sh.D[0][la][x] * sh.dN[1][lb][y] * sh.N[2][lc][z];
  } else if (d == 1) { // -N D N' , N' D N   (components 0, 2)
    c0 = -sh.N[0][la][x] * sh.D[1][lb][y] * sh.dN[2][lc][z];
    c1 = sh.dN[0][la][x] * sh.D[1][lb][y] * sh.N[2][lc][z];
  } else {             // N N' D , -N' N D   (components 0, 1)
    c0 = sh.N[0][la][x] * sh.dN[1][lb][y] * sh.D[2][lc][z];
    c1 = -sh.dN[0][la][x] * sh.N[1][lb][y] * sh.D[2][lc][z];
  }
}

template <int PD>
__global__ void __launch_bounds__(256) k_elem_lift(AsmParams P, const int32_t* __restrict__ belem,
                                                   const double* __restrict__ gD) {
  constexpr int NQ = PD + 1, NQ3 = NQ * NQ * NQ, NF = ElemShared<PD>::NF;
  constexpr int NFD = PD * (PD + 1) * (PD + 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ElemShared<PD>& sh = *reinterpret_cast<ElemShared<PD>*>(smem_raw);
  double* g = reinterpret_cast<double*>(smem_raw + sizeof(ElemShared<PD>));   // NF: boundary coefficients
  double* ell = g + NF;                                                        // NF: (K_e gD)_f
  double* v = ell + NF;                                                        // NQ3 x 3
  const int e = belem[blockIdx.x];
  int q, k;
  elem_setup<PD>(P, e, sh, q, k);
  const SubDev s = P.sd[k];
  const int tid = threadIdx.x;
  int a3[3];
  patch_abc_d(P, q, a3);
  const int st[3] = {P.start[0][a3[0]], P.start[1][a3[1]], P.start[2][a3[2]]};
  const int sp[3] = {P.elem[4 * e + 1], P.elem[4 * e + 2], P.elem[4 * e + 3]};
  for (int f = tid; f < NF; f += blockDim.x) {
    const int d = f / NFD, r = f % NFD;
    int ext[3] = {PD + 1, PD + 1, PD + 1};
    ext[d] = PD;
    const int64_t ix[3] = {st[0] + sp[0] + r % ext[0], st[1] + sp[1] + (r / ext[0]) % ext[1],
                           st[2] + sp[2] + r / (ext[0] * ext[1])};
    g[f] = gD[P.eoff[d] + ix[0] + P.eext[d][0] * (ix[1] + P.eext[d][1] * ix[2])];
  }
  __syncthreads();
  const double nu = P.nu[q];
  // v = nu w / |det DF| DF^T DF curl_hat(gD) at every Gauss point
  for (int t = tid; t < NQ3; t += blockDim.x) {
    const int x = t % NQ, y = (t / NQ) % NQ, z = t / (NQ * NQ);
    double ch[3] = {0, 0, 0};
    for (int f = 0; f < NF; ++f) {
      if (g[f] == 0.0) continue;
      double c0, c1;
      int i0, i1;
      ref_curl<PD>(sh, f, x, y, z, c0, c1, i0, i1);
      ch[i0] += g[f] * c0;
      ch[i1] += g[f] * c1;
    }
    const double* F = sh.DF[t];
    double y3[3];
    for (int r = 0; r < 3; ++r) y3[r] = F[r * 3 + 0] * ch[0] + F[r * 3 + 1] * ch[1] + F[r * 3 + 2] * ch[2];
    const double fac = nu * sh.wt[t] / fabs(sh.det[t]);
    for (int c = 0; c < 3; ++c) v[t * 3 + c] = fac * (F[0 * 3 + c] * y3[0] + F[1 * 3 + c] * y3[1] + F[2 * 3 + c] * y3[2]);
  }
  __syncthreads();
  for (int f = tid; f < NF; f += blockDim.x) {
    double acc = 0;
    for (int qq = 0; qq < NQ3; ++qq) {
      double c0, c1;
      int i0, i1;
      ref_curl<PD>(sh, f, qq % NQ, (qq / NQ) % NQ, qq / (NQ * NQ), c0, c1, i0, i1);
      acc += c0 * v[qq * 3 + i0] + c1 * v[qq * 3 + i1];
    }
    ell[f] = acc;
  }
  __syncthreads();
  for (int t = tid; t < NF * P.nrhs; t += blockDim.x) {
    const int f = t / P.nrhs, r = t % P.nrhs;
    const int cf = sh.code[f];
    if (cf < 0) continue;
    const double val = -P.src[r] * ell[f];
    if (cf < s.n) atomicAdd(P.jr + RV(s, cf, r, P.nrhs), val);
    else atomicAdd(P.jp + PV(s, cf - s.n, r, P.nrhs), val);
  }
}

// ---------------------------------------------------------------------------
// j on axis-aligned box patches from separable 1D integrals
//
// With DF = diag(L) the Gauss rule of Eq. (3) is a tensor product, and every
// source kind is a sum of products of 1D factors,
//   J_d(x) = Re sum_{fz,fy,fx} C_d[fz][fy][fx] phi_fx(x) phi_fy(y) phi_fz(z),
// with phi_f(t) = e^{2 pi i (f - KG) t} for Fourier modes with integer wave
// numbers |k| <= KG, and phi in {1, sin(pi t), sin t, cos t} for the sine,
// manufactured and patchwise kinds. So the load of the edge function
// D_a(xi_x) N_b(xi_y) N_c(xi_z) e_x (likewise for the other directions) is
//   (L_y L_z) Re sum C_x[fz][fy][fx] I^D_x[a][fx] I^N_y[b][fy] I^N_z[c][fz],
// the 1D sums I[i][f] = sum_spans sum_q (w_q / n) B_i(xi_q) phi_f(x(xi_q)) being
// the same Gauss rule, one axis at a time. The triple sum is contracted one
// axis at a time in shared memory (one CTA per patch, direction and load case).
// ---------------------------------------------------------------------------

struct SepArgs {
  int NF, KG, kind;        // kind 0: Fourier exponentials, 1: the four real factors
  int maxfun, Pmax;        // functions per slab at most (n + p), slabs per axis at most
  int per_patch;           // C per patch (patchwise source, NF = 1)
  const double* geo;       // per axis and slab: lower coordinate, length
  const double* xq;        // Gauss points on [0, 1]
  double2* tab;            // [axis][slab][family N/D][function][factor]
  const double2* C;        // [load case][(patch)][direction][fz][fy][fx]
  double* ploc;            // per patch-local edge and load case: the patch's part of its load
  int64_t npl;             // patch-local edges (column stride of ploc)
};

__global__ void k_sep_tab(AsmParams P, SepArgs S) {
  const int64_t tot = (int64_t)3 * S.Pmax * 2 * S.maxfun * S.NF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(t % S.NF);
    int64_t r = t / S.NF;
    const int i = (int)(r % S.maxfun);
    r /= S.maxfun;
    const int fam = (int)(r % 2);    // 0: N, 1: D
    r /= 2;
    const int sl = (int)(r % S.Pmax), ax = (int)(r / S.Pmax);
    const int Pa = ax == 0 ? P.P0 : (ax == 1 ? P.P1 : P.P2);
    double vr = 0, vi = 0;
    if (sl < Pa) {
      const int n = P.nspan[ax][sl];
      if (i < n + P.p - fam) {
        const double lo = S.geo[(ax * S.Pmax + sl) * 2], L = S.geo[(ax * S.Pmax + sl) * 2 + 1];
        const int g0 = P.spanoff[ax][sl];
        const int rmax = P.p - fam;   // local functions of a span: p + 1 (N), p (D)
        for (int sp = max(0, i - rmax); sp <= min(n - 1, i); ++sp) {
          const int rr = i - sp;
          for (int q = 0; q < P.nq; ++q) {
            const double B = fam ? P.tabD[ax][((int64_t)(g0 + sp) * P.p + rr) * P.nq + q]
                                 : P.tabN[ax][((int64_t)(g0 + sp) * (P.p + 1) + rr) * P.nq + q];
            const double w = P.wq[q] / n * B;
            const double x = lo + L * (sp + S.xq[q]) / n;
            if (S.kind == 0) {
              double sn, cs;
              sincospi(2.0 * (f - S.KG) * x, &sn, &cs);
              vr += w * cs;
              vi += w * sn;
            } else {
              vr += w * (f == 0 ? 1.0 : f == 1 ? sinpi(x) : f == 2 ? sin(x) : cos(x));
            }
          }
        }
      }
    }
    S.tab[t] = make_double2(vr, vi);
  }
}

__device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void __launch_bounds__(256) k_sep_load(AsmParams P, SepArgs S) {
  const int q = blockIdx.x, d = blockIdx.y, r = blockIdx.z;
  int a3[3];
  patch_abc_d(P, q, a3);
  const SubDev s = P.sd[P.sub_of_patch[q]];
  const int NF = S.NF, NF2 = NF * NF, NF3 = NF2 * NF;
  const int tid = threadIdx.x;
  int ext[3];
  for (int e = 0; e < 3; ++e) ext[e] = P.nspan[e][a3[e]] + P.p - (e == d ? 1 : 0);
  int64_t doff = 0;
  for (int dd = 0; dd < d; ++dd) {
    int64_t v = 1;
    for (int e = 0; e < 3; ++e) v *= P.nspan[e][a3[e]] + P.p - (e == dd ? 1 : 0);
    doff += v;
  }
  extern __shared__ __align__(16) double2 sm[];
  double2* Cs = sm;                            // [fz][fy][fx]
  double2* Tx = Cs + NF3;                      // [a][fx]
  double2* Ty = Tx + ext[0] * NF;              // [b][fy]
  double2* Tz = Ty + ext[1] * NF;              // [c][fz]
  double2* T1 = Tz + ext[2] * NF;              // [c][fy][fx]
  double2* T2 = T1 + (size_t)ext[2] * NF2;     // [c][b][fx]
  const int np = P.P0 * P.P1 * P.P2;
  const double2* Cg = S.C + (((int64_t)r * (S.per_patch ? np : 1) + (S.per_patch ? q : 0)) * 3 + d) * NF3;
  for (int t = tid; t < NF3; t += blockDim.x) Cs[t] = Cg[t];
  double2* T[3] = {Tx, Ty, Tz};
  for (int e = 0; e < 3; ++e) {
    const double2* src = S.tab + ((int64_t)((e * S.Pmax + a3[e]) * 2 + (e == d ? 1 : 0)) * S.maxfun) * NF;
    for (int t = tid; t < ext[e] * NF; t += blockDim.x) T[e][t] = src[t];
  }
  __syncthreads();
  for (int t = tid; t < ext[2] * NF2; t += blockDim.x) {
    const int c = t / NF2, yx = t % NF2;
    double2 acc = make_double2(0.0, 0.0);
    for (int fz = 0; fz < NF; ++fz) {
      const double2 v = cmul(Cs[fz * NF2 + yx], Tz[c * NF + fz]);
      acc.x += v.x;
      acc.y += v.y;
    }
    T1[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < ext[2] * ext[1] * NF; t += blockDim.x) {
    const int fx = t % NF, b = (t / NF) % ext[1], c = t / (NF * ext[1]);
    double2 acc = make_double2(0.0, 0.0);
    for (int fy = 0; fy < NF; ++fy) {
      const double2 v = cmul(T1[(c * NF + fy) * NF + fx], Ty[b * NF + fy]);
      acc.x += v.x;
      acc.y += v.y;
    }
    T2[t] = acc;
  }
  __syncthreads();
  // covariant map and measure: |L_x L_y L_z| / L_d
  double vol = 1.0;
  for (int e = 0; e < 3; ++e) vol *= S.geo[(e * S.Pmax + a3[e]) * 2 + 1];
  const double scale = fabs(vol) / S.geo[(d * S.Pmax + a3[d]) * 2 + 1];
  const int64_t nloc = (int64_t)ext[0] * ext[1] * ext[2];
  const int64_t cbase = P.patch_code_off[q] + doff;
  for (int64_t t = tid; t < nloc; t += blockDim.x) {
    const int a = (int)(t % ext[0]), bc = (int)(t / ext[0]);   // bc = b + ext1 c
    if (P.patch_code[cbase + t] < 0) continue;
    double v = 0;
    for (int fx = 0; fx < NF; ++fx) {
      const double2 u = T2[(int64_t)bc * NF + fx], w = Tx[a * NF + fx];
      v += u.x * w.x - u.y * w.y;
    }
    // this patch's part of the DOF's load; k_sep_gather sums the parts
    S.ploc[cbase + t + S.npl * r] = v * scale;
  }
}

// loads of the local DOFs: the parts of their patch-local edges summed in a
// fixed order (deterministic, no atomics)
__global__ void k_sep_gather(AsmParams P, SepArgs S, const int64_t* __restrict__ gofs,
                             const int64_t* __restrict__ glist, const int64_t* __restrict__ gbase,
                             const int32_t* __restrict__ gstride, int64_t nslot, int64_t nslot_r) {
  const int r = blockIdx.y;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nslot; t += (int64_t)gridDim.x * blockDim.x) {
    double v = 0;
    for (int64_t e = gofs[t]; e < gofs[t + 1]; ++e) v += S.ploc[glist[e] + S.npl * r];
    double* dst = t < nslot_r ? P.jr : P.jp;
    dst[gbase[t] + (int64_t)gstride[t] * r] = v;
  }
}

// ---------------------------------------------------------------------------
// K: Kronecker generation of every dense entry (axis-aligned affine patches)
// ---------------------------------------------------------------------------

__device__ inline int slab_cands(const AsmParams& P, int c, int idx, bool isD, int out[2]) {
  int Pc = (c == 0) ? P.P0 : (c == 1 ? P.P1 : P.P2);
  int a = P.slab_of[c][idx];
  int n = 0;
  out[n++] = a;
  if (!isD && idx == P.start[c][a]) {
    if (a > 0) out[n++] = a - 1;
    else if (c == 0 && P.per0) out[n++] = Pc - 1;
  }
  return n;
}

__device__ inline int local_index(const AsmParams& P, int c, int a, int idx, bool isD) {
  int li = idx - P.start[c][a];
  if (c == 0 && P.per0) li = ((li % P.N0) + P.N0) % P.N0;
  int hi = P.nspan[c][a] + P.p - 1 - (isD ? 1 : 0);
  return (li >= 0 && li <= hi) ? li : -1;
}

template <typename T>
__device__ __forceinline__ void kron_entry(const AsmParams& P, T* Lout, int k, const SubDev& s, int i, int j);

template <typename T>
__global__ void __launch_bounds__(256) k_kron(AsmParams P, T* Lout, int prim_only) {
  // grid: (row chunks of 256, column groups, subdomain); columns j = blockIdx.y + gridDim.y t,
  // from the first primal column if prim_only (the K_rp and K_pp blocks)
  const int k = blockIdx.z;
  const SubDev s = P.sd[k];
  const int R = s.n + s.nP;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= R) return;
  for (int j = (prim_only ? s.n : 0) + blockIdx.y; j < R; j += gridDim.y) kron_entry<T>(P, Lout, k, s, i, j);
}

// slab candidates and slab-local indices of one DOF per direction (the
// DOF-dependent part of a Kronecker entry, formed once per row and column)
struct KronInfo {
  int x[3], d;
  int n[3], cand[3][2], loc[3][2];
};

__device__ inline void kron_info(const AsmParams& P, const DofDev& a, KronInfo& I) {
  I.d = a.d;
  I.x[0] = a.i;
  I.x[1] = a.j;
  I.x[2] = a.k;
  if (a.d < 0) return;
  for (int c = 0; c < 3; ++c) {
    I.n[c] = slab_cands(P, c, I.x[c], a.d == c, I.cand[c]);
    for (int u = 0; u < I.n[c]; ++u) I.loc[c][u] = local_index(P, c, I.cand[c][u], I.x[c], a.d == c);
  }
}

// the K_rr entry of rows with infos A and B in subdomain k: the same terms, in
// the same order, as kron_entry
__device__ inline double kron_value(const AsmParams& P, int k, const KronInfo& A, const KronInfo& B, bool diag) {
  if (A.d < 0 || B.d < 0) return diag ? 1.0 : 0.0;
  const int p = P.p;
  for (int c = 0; c < 3; ++c) {
    int dl = A.x[c] - B.x[c];
    if (c == 0 && P.per0) {
      dl = ((dl % P.N0) + P.N0) % P.N0;
      if (dl > P.N0 / 2) dl -= P.N0;
    }
    if (dl > p || dl < -p) return 0.0;
  }
  double v = 0.0;
  for (int u0 = 0; u0 < A.n[0]; ++u0)
    for (int w0 = 0; w0 < B.n[0]; ++w0) {
      if (A.cand[0][u0] != B.cand[0][w0]) continue;
      for (int u1 = 0; u1 < A.n[1]; ++u1)
        for (int w1 = 0; w1 < B.n[1]; ++w1) {
          if (A.cand[1][u1] != B.cand[1][w1]) continue;
          for (int u2 = 0; u2 < A.n[2]; ++u2)
            for (int w2 = 0; w2 < B.n[2]; ++w2) {
              if (A.cand[2][u2] != B.cand[2][w2]) continue;
              const int sl[3] = {A.cand[0][u0], A.cand[1][u1], A.cand[2][u2]};
              const int q = sl[0] + P.P0 * (sl[1] + P.P1 * sl[2]);
              if (P.sub_of_patch[q] != k) continue;
              const int la[3] = {A.loc[0][u0], A.loc[1][u1], A.loc[2][u2]};
              const int lb[3] = {B.loc[0][w0], B.loc[1][w1], B.loc[2][w2]};
              if (la[0] < 0 || la[1] < 0 || la[2] < 0 || lb[0] < 0 || lb[1] < 0 || lb[2] < 0) continue;
              for (int comp = 0; comp < 3; ++comp) {
                if (comp == A.d || comp == B.d) continue;
                int fa[3], fb[3];
                const int sgn = curl_term(A.d, comp, fa) * curl_term(B.d, comp, fb);
                double prod = P.gq[q * 3 + comp] * sgn;
                for (int c = 0; c < 3; ++c) {
                  const int off = lb[c] - la[c] + p;
                  if (off < 0 || off > 2 * p) {
                    prod = 0;
                    break;
                  }
                  prod *= P.gram[c][P.gram_per[c] * sl[c] +
                                    ((int64_t)(fa[c] * 3 + fb[c]) * P.gram_nfun[c] + la[c]) * (2 * p + 1) + off];
                }
                v += prod;
              }
            }
        }
    }
  return v;
}

// K_rr entries of the listed nonzero 64 x 64 tiles (k, I, J), I >= J, only;
// the other tiles of K_rr are structurally zero and keep the zeros of the first
// assembly. The column infos are formed once per tile in shared memory, the
// row's once per thread (row 64 I + t % 64, columns 64 J + 16 (t / 64) ..);
// the tile is staged in shared memory and written with its mirror (J, I),
// both with coalesced stores.
__global__ void __launch_bounds__(256) k_kron_tiles(AsmParams P, const int4* tiles) {
  const int4 tl = tiles[blockIdx.x];
  const int k = tl.x;
  const SubDev s = P.sd[k];
  __shared__ KronInfo cinfo[NB];
  __shared__ double T[NB][NB + 1];
  const int tid = threadIdx.x;
  if (tid < NB) kron_info(P, P.dof[s.dof + tl.z * NB + tid], cinfo[tid]);
  KronInfo A;
  const int ii = tid % NB, j0 = 16 * (tid / NB);
  kron_info(P, P.dof[s.dof + tl.y * NB + ii], A);
  __syncthreads();
  const bool dtile = tl.y == tl.z;
  for (int jj = j0; jj < j0 + 16; ++jj) T[ii][jj] = kron_value(P, k, A, cinfo[jj], dtile && ii == jj);
  __syncthreads();
  double* K = P.K64 + s.A;
  for (int t = tid; t < NB * NB; t += blockDim.x) {
    const int r = t % NB, c = t / NB;
    // (a diagonal tile takes its lower half for both halves: K_rr exactly symmetric)
    K[(int64_t)tl.y * NB + r + (int64_t)s.n * (tl.z * NB + c)] = (dtile && r < c) ? T[c][r] : T[r][c];
    if (!dtile) K[(int64_t)tl.z * NB + r + (int64_t)s.n * (tl.y * NB + c)] = T[c][r];
  }
}

template <typename T>
__device__ __forceinline__ void kron_entry(const AsmParams& P, T* Lout, int k, const SubDev& s, int i, int j) {
  if (i >= s.n && j < s.n) return;           // K_pr is not stored
  const DofDev a = P.dof[s.dof + i];
  const DofDev b = P.dof[s.dof + j];
  double v = 0.0;
  if (a.d < 0 || b.d < 0) {
    v = (i == j) ? 1.0 : 0.0;
  } else {
    const int p = P.p;
    int xa[3] = {a.i, a.j, a.k}, xb[3] = {b.i, b.j, b.k};
    bool near = true;
    for (int c = 0; c < 3; ++c) {
      int dl = xa[c] - xb[c];
      if (c == 0 && P.per0) {
        dl = ((dl % P.N0) + P.N0) % P.N0;
        if (dl > P.N0 / 2) dl -= P.N0;
      }
      if (dl > p || dl < -p) near = false;
    }
    if (near) {
      int ca[3][2], cb[3][2], na[3], nb[3];
      for (int c = 0; c < 3; ++c) {
        na[c] = slab_cands(P, c, xa[c], a.d == c, ca[c]);
        nb[c] = slab_cands(P, c, xb[c], b.d == c, cb[c]);
      }
      // common slabs per direction
      int cs[3][2], ncs[3];
      for (int c = 0; c < 3; ++c) {
        ncs[c] = 0;
        for (int u = 0; u < na[c]; ++u)
          for (int w = 0; w < nb[c]; ++w)
            if (ca[c][u] == cb[c][w]) cs[c][ncs[c]++] = ca[c][u];
      }
      for (int u0 = 0; u0 < ncs[0]; ++u0)
        for (int u1 = 0; u1 < ncs[1]; ++u1)
          for (int u2 = 0; u2 < ncs[2]; ++u2) {
            int sl[3] = {cs[0][u0], cs[1][u1], cs[2][u2]};
            int q = sl[0] + P.P0 * (sl[1] + P.P1 * sl[2]);
            if (P.sub_of_patch[q] != k) continue;
            int la[3], lb[3];
            bool ok = true;
            for (int c = 0; c < 3; ++c) {
              la[c] = local_index(P, c, sl[c], xa[c], a.d == c);
              lb[c] = local_index(P, c, sl[c], xb[c], b.d == c);
              if (la[c] < 0 || lb[c] < 0) ok = false;
            }
            if (!ok) continue;
            for (int comp = 0; comp < 3; ++comp) {
              if (comp == a.d || comp == b.d) continue;
              int fa[3], fb[3];
              int sgn = curl_term(a.d, comp, fa) * curl_term(b.d, comp, fb);
              double prod = P.gq[q * 3 + comp] * sgn;
              for (int c = 0; c < 3; ++c) {
                int off = lb[c] - la[c] + p;
                if (off < 0 || off > 2 * p) { prod = 0; break; }
                prod *= P.gram[c][P.gram_per[c] * sl[c] +
                                  ((int64_t)(fa[c] * 3 + fb[c]) * P.gram_nfun[c] + la[c]) * (2 * p + 1) + off];
              }
              v += prod;
            }
          }
    }
  }
  if (i < s.n) {
    if (j < s.n) {
      P.K64[s.A + i + (int64_t)s.n * j] = v;
      if (Lout) Lout[s.A + i + (int64_t)s.n * j] = (T)v;
    } else {
      P.Kp[s.Kp + i + (int64_t)s.n * (j - s.n)] = v;
    }
  } else {
    P.Kpp[s.Kpp + (i - s.n) + (int64_t)s.nP * (j - s.n)] = v;
  }
}

__global__ void k_pad_diag(const SubDev* sd, const DofDev* dof, double* K64) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x)
    if (dof[s.dof + i].d < 0) K64[s.A + i + (int64_t)s.n * i] = 1.0;
}

template <typename T>
__global__ void k_copy_convert(const double* __restrict__ src, T* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}

// ---------------------------------------------------------------------------

static AsmParams make_params(Ctx* c) {
  AsmParams P;
  P.p = c->mesh.p;
  P.nq = c->tab.nq;
  P.nsub = c->nsub;
  P.nrhs = c->nrhs;
  P.source_kind = c->source_kind;
  P.n_src = (int)c->src.size();
  P.P0 = c->mesh.P[0]; P.P1 = c->mesh.P[1]; P.P2 = c->mesh.P[2];
  P.N0 = c->mesh.N[0]; P.N1 = c->mesh.N[1]; P.N2 = c->mesh.N[2];
  P.per0 = c->mesh.per0 ? 1 : 0;
  P.sd = c->d_sd;
  P.dof = c->d_dof;
  P.patch_code = c->d_patch_code;
  P.patch_code_off = c->d_patch_code_off;
  P.sub_of_patch = c->d_sub_of_patch;
  P.elem = c->d_elem;
  for (int d = 0; d < 3; ++d) {
    P.tabN[d] = c->d_tabN[d];
    P.tabdN[d] = c->d_tabdN[d];
    P.tabD[d] = c->d_tabD[d];
    P.gram[d] = c->d_gram[d];
    P.gram_per[d] = c->gram[d].slab_off.size() > 1 ? c->gram[d].slab_off[1] : 0;
    P.gram_nfun[d] = c->gram[d].nfun_max;
    P.slab_of[d] = c->d_slab_of[d];
    P.start[d] = c->d_start[d];
    P.nspan[d] = c->d_nspan[d];
    P.spanoff[d] = c->d_start[d] + c->mesh.P[d];   // stored right after start
  }
  P.wq = c->d_wq;
  P.ctrl = c->d_ctrl;
  P.nu = c->d_nu;
  P.src = c->d_src;
  P.gq = c->d_gq;
  P.geo = c->d_geo;
  P.geo_ready = c->geo_ready ? 1 : 0;
  P.K64 = c->K64;
  P.Kp = c->Kp64;
  P.Kpp = c->Kpp64;
  P.jr = c->jr;
  P.jp = c->jp;
  for (int d = 0; d < 3; ++d) {
    P.eoff[d] = c->mesh.off[d];
    for (int e = 0; e < 3; ++e) P.eext[d][e] = c->mesh.ext[d][e];
  }
  return P;
}

template <int PD>
static ieti_status launch_elem(Ctx* c, const AsmParams& P, bool do_K, bool do_j, cudaStream_t st) {
  constexpr int NQ3 = (PD + 1) * (PD + 1) * (PD + 1), NF = ElemShared<PD>::NF;
  if (do_K) {
    size_t smem = sizeof(ElemShared<PD>) + sizeof(double) * (NQ3 * 9 + (size_t)NF * NQ3 * 2);
    cudaEvent_t p0 = prof_begin(c, st);
    k_elem_K<PD><<<(unsigned)c->nelem, 256, smem, st>>>(P);
    prof_end(c, PROF_ASM_K, p0, st);
    IETI_LAUNCH_CHECK(c);
  }
  size_t smem = sizeof(ElemShared<PD>) + sizeof(double) * (size_t)NQ3 * (c->nrhs * 3 + 9 + 3) + 16 +
                sizeof(double2) * (size_t)NQ3 * 3 * (FT_KMAX + 1);
  cudaEvent_t p0 = prof_begin(c, st);
  if (do_j) {
    k_elem_j<PD><<<(unsigned)c->nelem, 256, smem, st>>>(P);
    IETI_LAUNCH_CHECK(c);
  }
  if (c->d_gD && c->nbelem > 0) {
    const size_t lsm = sizeof(ElemShared<PD>) + sizeof(double) * (2 * (size_t)NF + 3 * (size_t)NQ3);
    k_elem_lift<PD><<<(unsigned)c->nbelem, 256, lsm, st>>>(P, c->d_belem, c->d_gD);
    IETI_LAUNCH_CHECK(c);
  }
  prof_end(c, PROF_ASM_J, p0, st);
  return IETI_OK;
}

// raises the dynamic shared-memory limit of the element kernels
ieti_status assemble_kernel_attrs(Ctx* c, int smem_max) {
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_elem_K<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_elem_K<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_elem_K<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_elem_j<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_elem_j<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_elem_j<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_sep_load, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  return IETI_OK;
}

// device buffer of at least n elements, grown (and kept) on demand
template <typename T>
static ieti_status grow(Ctx* c, T** p, int64_t* cap, int64_t n) {
  if (n <= *cap) return IETI_OK;
  void* q = nullptr;
  const size_t bytes = sizeof(T) * (size_t)std::max<int64_t>(n, 1);
  if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed";
    return IETI_ERR_OOM;
  }
  c->allocs.push_back({q, bytes});
  *p = (T*)q;
  *cap = n;
  return IETI_OK;
}

// the loads of box patches from separable 1D integrals (above), when the
// source is a sum of products of the supported 1D factors and the contraction
// fits in shared memory; *done = false leaves them to the element quadrature
static ieti_status sep_loads(Ctx* c, const AsmParams& P, bool* done, cudaStream_t st) {
  *done = false;
  if (!c->d_sep_gofs) return IETI_OK;
  const Mesh& m = c->mesh;
  const int nr = c->nrhs, np = m.npatch();
  int NF = 0, KG = 0, kind = 1, per_patch = 0;
  std::vector<double2>& C = c->sep_C_host;   // kept: read by the asynchronous copy below
  const std::vector<double>& src = c->src;
  auto fill = [&](int NFv) {
    NF = NFv;
    C.assign((size_t)nr * (per_patch ? np : 1) * 3 * NF * NF * NF, make_double2(0.0, 0.0));
  };
  auto at = [&](int r, int d, int fz, int fy, int fx) -> double2& {
    return C[((size_t)r * 3 + d) * NF * NF * NF + ((size_t)fz * NF + fy) * NF + fx];
  };
  const double pi = 3.14159265358979323846;
  if (c->source_kind == IETI_SOURCE_FOURIER) {
    // integer wave numbers up to 4 per axis: the grid of exponentials
    size_t pos = 0;
    for (int r = 0; r < nr; ++r) {
      const int nm = (int)src[pos++];
      for (int mm = 0; mm < nm; ++mm, pos += 9)
        for (int a = 0; a < 3; ++a) {
          const double k = src[pos + a];
          if (k != std::rint(k) || std::fabs(k) > 4) return IETI_OK;
          KG = std::max(KG, (int)std::fabs(k));
        }
    }
    kind = 0;
    fill(2 * KG + 1);
    pos = 0;
    for (int r = 0; r < nr; ++r) {
      const int nm = (int)src[pos++];
      for (int mm = 0; mm < nm; ++mm, pos += 9) {
        const int kx = (int)src[pos] + KG, ky = (int)src[pos + 1] + KG, kz = (int)src[pos + 2] + KG;
        for (int d = 0; d < 3; ++d) {
          double2& v = at(r, d, kz, ky, kx);
          v.x += src[pos + 3 + d];
          v.y += src[pos + 6 + d];
        }
      }
    }
  } else if (c->source_kind == IETI_SOURCE_SINE) {
    // factors 0: 1, 1: sin(pi t)
    fill(4);
    for (int r = 0; r < nr; ++r) {
      const double a = src[r] * 2 * pi * pi;
      at(r, 0, 1, 1, 0).x = a;
      at(r, 1, 1, 0, 1).x = a;
      at(r, 2, 0, 1, 1).x = a;
    }
  } else if (c->source_kind == IETI_SOURCE_TRIG) {
    // factors 2: sin t, 3: cos t; 3 A_ana of Sec. 3
    fill(4);
    for (int r = 0; r < nr; ++r) {
      at(r, 0, 3, 3, 2).x = 3.0 * src[r];
      at(r, 1, 3, 2, 3).x = -6.0 * src[r];
      at(r, 2, 2, 3, 3).x = 3.0 * src[r];
    }
  } else if (c->source_kind == IETI_SOURCE_PATCHWISE) {
    per_patch = 1;
    fill(1);
    for (size_t t = 0; t < C.size(); ++t) C[t].x = src[t];
  } else {
    return IETI_OK;
  }
  int maxfun = 0, Pmax = 0;
  for (int a = 0; a < 3; ++a) {
    Pmax = std::max(Pmax, m.P[a]);
    for (int sl = 0; sl < m.P[a]; ++sl) maxfun = std::max(maxfun, m.nspan[a][sl] + m.p);
  }
  const size_t smem = sizeof(double2) * ((size_t)NF * NF * NF + 3 * (size_t)maxfun * NF +
                                         (size_t)maxfun * NF * NF + (size_t)maxfun * maxfun * NF);
  if (smem > (size_t)c->smem_optin) return IETI_OK;
  // slab geometry of the box net: lower corner and length per axis and slab
  std::vector<double> geo((size_t)3 * Pmax * 2, 0.0);
  for (int a = 0; a < 3; ++a)
    for (int sl = 0; sl < m.P[a]; ++sl) {
      int i0[3] = {0, 0, 0}, i1[3] = {0, 0, 0};
      i0[a] = m.start[a][sl];
      i1[a] = m.start[a][sl] + m.nspan[a][sl] + m.p - 1;
      auto X = [&](const int* ix) {
        return c->ctrl[(((size_t)ix[2] * m.N[1] + ix[1]) * m.N[0] + ix[0]) * 4 + a];
      };
      geo[(a * Pmax + sl) * 2] = X(i0);
      geo[(a * Pmax + sl) * 2 + 1] = X(i1) - X(i0);
    }
  ieti_status rs;
  int64_t cap = 0;
  if (!c->d_sep_geo) {
    if ((rs = grow(c, &c->d_sep_geo, &cap, (int64_t)geo.size())) != IETI_OK) return rs;
    cap = 0;
    if ((rs = grow(c, &c->d_xq, &cap, (int64_t)c->tab.xq.size())) != IETI_OK) return rs;
    IETI_CUDA_TRY(c, cudaMemcpy(c->d_sep_geo, geo.data(), sizeof(double) * geo.size(), cudaMemcpyHostToDevice));
    IETI_CUDA_TRY(c, cudaMemcpy(c->d_xq, c->tab.xq.data(), sizeof(double) * c->tab.xq.size(),
                                cudaMemcpyHostToDevice));
  }
  if ((rs = grow(c, &c->d_sep_C, &c->sep_C_cap, (int64_t)C.size())) != IETI_OK) return rs;
  if ((rs = grow(c, &c->d_sep_ploc, &c->sep_ploc_cap, c->sep_npl * nr)) != IETI_OK) return rs;
  const int64_t ntab = (int64_t)3 * Pmax * 2 * maxfun * NF;
  if ((rs = grow(c, &c->d_sep_tab, &c->sep_tab_cap, ntab)) != IETI_OK) return rs;
  IETI_CUDA_TRY(c, cudaMemcpyAsync(c->d_sep_C, C.data(), sizeof(double2) * C.size(), cudaMemcpyHostToDevice, st));
  SepArgs S;
  S.NF = NF;
  S.KG = KG;
  S.kind = kind;
  S.maxfun = maxfun;
  S.Pmax = Pmax;
  S.per_patch = per_patch;
  S.geo = c->d_sep_geo;
  S.xq = c->d_xq;
  S.tab = c->d_sep_tab;
  S.C = c->d_sep_C;
  S.ploc = c->d_sep_ploc;
  S.npl = c->sep_npl;
  cudaEvent_t p0 = prof_begin(c, st);
  k_sep_tab<<<(unsigned)std::min<int64_t>(ceil_div(ntab, 256), 4096), 256, 0, st>>>(P, S);
  IETI_LAUNCH_CHECK(c);
  k_sep_load<<<dim3((unsigned)np, 3, (unsigned)nr), 256, smem, st>>>(P, S);
  IETI_LAUNCH_CHECK(c);
  k_sep_gather<<<dim3((unsigned)std::min<int64_t>(ceil_div(std::max<int64_t>(c->sep_nslot, 1), 256), 1184),
                      (unsigned)nr), 256, 0, st>>>(P, S, c->d_sep_gofs, c->d_sep_glist, c->d_sep_gbase,
                                                   c->d_sep_gstride, c->sep_nslot, c->tot_rv);
  IETI_LAUNCH_CHECK(c);
  prof_end(c, PROF_ASM_J, p0, st);
  *done = true;
  return IETI_OK;
}

ieti_status assemble_all(Ctx* c, cudaStream_t st) {
  AsmParams P = make_params(c);
  IETI_CUDA_TRY(c, cudaMemsetAsync(c->jr, 0, sizeof(double) * c->tot_rv * c->nrhs, st));
  IETI_CUDA_TRY(c, cudaMemsetAsync(c->jp, 0, sizeof(double) * std::max<int64_t>(c->tot_pv, 1) * c->nrhs, st));
  const bool kron = c->affine;
  if (kron) {
    const int64_t R = c->max_n + c->max_nP;
    cudaEvent_t p0 = prof_begin(c, st);
    if (c->ktile_ready && c->n_ktiles > 0) {
      // the nonzero tiles of K_rr (pattern of an earlier assembly), then K_rp and K_pp
      k_kron_tiles<<<(unsigned)c->n_ktiles, 256, 0, st>>>(P, c->d_ktile_list);
      IETI_LAUNCH_CHECK(c);
      if (c->max_nP > 0) {
        dim3 grid((unsigned)ceil_div(R, 256), (unsigned)c->max_nP, (unsigned)c->nsub);
        k_kron<double><<<grid, 256, 0, st>>>(P, (double*)nullptr, 1);
      }
    } else {
      dim3 grid((unsigned)ceil_div(R, 256), (unsigned)std::min<int64_t>(R, 65535), (unsigned)c->nsub);
      k_kron<double><<<grid, 256, 0, st>>>(P, (double*)nullptr, 0);
    }
    prof_end(c, PROF_ASM_K, p0, st);
    IETI_LAUNCH_CHECK(c);
  } else {
    IETI_CUDA_TRY(c, cudaMemsetAsync(c->K64, 0, sizeof(double) * c->tot_A, st));
    IETI_CUDA_TRY(c, cudaMemsetAsync(c->Kp64, 0, sizeof(double) * std::max<int64_t>(c->tot_Kp, 1), st));
    IETI_CUDA_TRY(c, cudaMemsetAsync(c->Kpp64, 0, sizeof(double) * std::max<int64_t>(c->tot_Kpp, 1), st));
    k_pad_diag<<<dim3(8, c->nsub), 256, 0, st>>>(c->d_sd, c->d_dof, c->K64);
    IETI_LAUNCH_CHECK(c);
  }
  ieti_status r;
  bool sep = false;
  if (kron && c->sep_loads && (r = sep_loads(c, P, &sep, st)) != IETI_OK) return r;
  if (!sep && !c->d_geo && !c->geo_failed) {
    // geometry kept per element and Gauss point (12 doubles each)
    const int nq3 = (c->mesh.p + 1) * (c->mesh.p + 1) * (c->mesh.p + 1);
    const size_t bytes = sizeof(double) * 12 * (size_t)nq3 * (size_t)std::max<int64_t>(c->nelem, 1);
    void* g = nullptr;
    if (cudaMalloc(&g, bytes) == cudaSuccess) {
      c->allocs.push_back({g, bytes});
      c->d_geo = (double*)g;
      P.geo = c->d_geo;
    } else {
      cudaGetLastError();   // not kept: every assembly recomputes the geometry
      c->geo_failed = true;
    }
  }
  switch (c->mesh.p) {
    case 1: r = launch_elem<1>(c, P, !kron, !sep, st); break;
    case 2: r = launch_elem<2>(c, P, !kron, !sep, st); break;
    case 3: r = launch_elem<3>(c, P, !kron, !sep, st); break;
    default: c->err = "degree p must be 1, 2 or 3"; return IETI_ERR_INVALID_ARG;
  }
  if (r == IETI_OK && c->d_geo && !sep) c->geo_ready = true;
  return r;
}

// ---------------------------------------------------------------------------
// B = curl a at the Gauss points and its L2 norms (Sec. 3 error norm)
// ---------------------------------------------------------------------------

constexpr int FLUX_CG = 8;   // load cases per pass of the flux kernel

struct FluxArgs {
  const double* a;       // nedge x nrhs, global edge numbering
  int64_t nedge;
  int nrhs;
  int ref_kind;          // ieti_bref_kind
  const double* amp;     // nrhs amplitudes of the reference field
  double* part;          // per element and load case: |B|^2 and |B_ref - B|^2 integrals
  double* Bq;            // optional: B at the Gauss points (nelem x NQ3 x 3 per load case)
};

// reference flux density curl(amp (sin pi y sin pi z, sin pi x sin pi z, sin pi x sin pi y))
__device__ inline void sine_flux(const double X[3], double amp, double B[3]) {
  const double pi = 3.14159265358979323846;
  const double sx = sin(pi * X[0]), sy = sin(pi * X[1]), sz = sin(pi * X[2]);
  const double cx = cos(pi * X[0]), cy = cos(pi * X[1]), cz = cos(pi * X[2]);
  B[0] = amp * pi * sx * (cy - cz);
  B[1] = amp * pi * sy * (cz - cx);
  B[2] = amp * pi * sz * (cx - cy);
}

// reference flux density amp B_ana = amp curl A_ana of Sec. 3
__device__ inline void trig_flux(const double X[3], double amp, double B[3]) {
  double sx, cx, sy, cy, sz, cz;
  sincos(X[0], &sx, &cx);
  sincos(X[1], &sy, &cy);
  sincos(X[2], &sz, &cz);
  B[0] = -3.0 * amp * cx * sy * sz;
  B[1] = 0.0;
  B[2] = 3.0 * amp * cz * sx * sy;
}

// one CTA per element: the field's coefficients of the element functions, the
// reference curls of those functions at the Gauss points (two nonzero
// components each), B = DF curl_hat / det DF, and the element integrals
// sum_q w |det DF| |B|^2 (and |B_ref - B|^2) per load case
template <int PD>
__global__ void __launch_bounds__(256) k_elem_B(AsmParams P, FluxArgs F) {
  constexpr int NQ = PD + 1, NQ3 = NQ * NQ * NQ, NF = ElemShared<PD>::NF;
  constexpr int NFD = PD * (PD + 1) * (PD + 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ElemShared<PD>& sh = *reinterpret_cast<ElemShared<PD>*>(smem_raw);
  double* C = reinterpret_cast<double*>(smem_raw + sizeof(ElemShared<PD>));   // NF x NQ3 x 2
  double* coef = C + (size_t)NF * NQ3 * 2;                                     // NF x FLUX_CG
  double* acc = coef + (size_t)NF * FLUX_CG;                                   // NQ3 x FLUX_CG x 2
  __shared__ int64_t gid[NF];
  const int e = blockIdx.x;
  int q, k;
  elem_setup<PD>(P, e, sh, q, k);
  const int tid = threadIdx.x;
  int a3[3];
  patch_abc_d(P, q, a3);
  int st[3] = {P.start[0][a3[0]], P.start[1][a3[1]], P.start[2][a3[2]]};
  int s[3] = {P.elem[4 * e + 1], P.elem[4 * e + 2], P.elem[4 * e + 3]};
  for (int f = tid; f < NF; f += blockDim.x) {
    const int d = f / NFD, r = f % NFD;
    int ext[3] = {PD + 1, PD + 1, PD + 1};
    ext[d] = PD;
    int64_t ix[3] = {st[0] + s[0] + r % ext[0], st[1] + s[1] + (r / ext[0]) % ext[1],
                     st[2] + s[2] + r / (ext[0] * ext[1])};
    if (P.per0) ix[0] %= P.N0;
    gid[f] = P.eoff[d] + ix[0] + P.eext[d][0] * (ix[1] + P.eext[d][1] * ix[2]);
  }
  for (int t = tid; t < NF * NQ3; t += blockDim.x) {
    int f = t / NQ3, qq = t % NQ3;
    int x = qq % NQ, y = (qq / NQ) % NQ, z = qq / (NQ * NQ);
    int d = f / NFD, r = f % NFD;
    int ext[3] = {PD + 1, PD + 1, PD + 1};
    ext[d] = PD;
    int la = r % ext[0], lb = (r / ext[0]) % ext[1], lc = r / (ext[0] * ext[1]);
    double c0, c1;
    if (d == 0) {        // components 1, 2
      c0 = sh.D[0][la][x] * sh.N[1][lb][y] * sh.dN[2][lc][z];
      c1 = -sh.D[0][la][x] * sh.dN[1][lb][y] * sh.N[2][lc][z];
    } else if (d == 1) { // components 0, 2
      c0 = -sh.N[0][la][x] * sh.D[1][lb][y] * sh.dN[2][lc][z];
      c1 = sh.dN[0][la][x] * sh.D[1][lb][y] * sh.N[2][lc][z];
    } else {             // components 0, 1
      c0 = sh.N[0][la][x] * sh.dN[1][lb][y] * sh.D[2][lc][z];
      c1 = -sh.dN[0][la][x] * sh.N[1][lb][y] * sh.D[2][lc][z];
    }
    C[(f * NQ3 + qq) * 2 + 0] = c0;
    C[(f * NQ3 + qq) * 2 + 1] = c1;
  }
  __syncthreads();
  for (int c0 = 0; c0 < F.nrhs; c0 += FLUX_CG) {
    const int ng = min(FLUX_CG, F.nrhs - c0);
    for (int t = tid; t < NF * ng; t += blockDim.x) {
      const int f = t % NF, col = t / NF;
      coef[f * FLUX_CG + col] = F.a[gid[f] + F.nedge * (c0 + col)];
    }
    __syncthreads();
    for (int t = tid; t < NQ3 * ng; t += blockDim.x) {
      const int qq = t % NQ3, col = t / NQ3;
      double ch[3] = {0, 0, 0};
      for (int f = 0; f < NF; ++f) {
        const int d = f / NFD;
        const double v = coef[f * FLUX_CG + col];
        const double* cf = C + (f * NQ3 + qq) * 2;
        ch[d == 0 ? 1 : 0] += v * cf[0];
        ch[d == 2 ? 1 : 2] += v * cf[1];
      }
      const double* Df = sh.DF[qq];
      const double det = sh.det[qq];
      double B[3];
      for (int r = 0; r < 3; ++r) B[r] = (Df[r * 3 + 0] * ch[0] + Df[r * 3 + 1] * ch[1] + Df[r * 3 + 2] * ch[2]) / det;
      const double w = sh.wt[qq] * fabs(det);
      acc[(qq * FLUX_CG + col) * 2 + 0] = w * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
      double e2 = 0;
      if (F.ref_kind != IETI_BREF_NONE) {
        double R[3];
        if (F.ref_kind == IETI_BREF_SINE) sine_flux(sh.X[qq], F.amp[c0 + col], R);
        else trig_flux(sh.X[qq], F.amp[c0 + col], R);
        e2 = w * ((R[0] - B[0]) * (R[0] - B[0]) + (R[1] - B[1]) * (R[1] - B[1]) + (R[2] - B[2]) * (R[2] - B[2]));
      }
      acc[(qq * FLUX_CG + col) * 2 + 1] = e2;
      if (F.Bq) {
        double* o = F.Bq + (((int64_t)e * NQ3 + qq) * 3) + (int64_t)gridDim.x * NQ3 * 3 * (c0 + col);
        o[0] = B[0]; o[1] = B[1]; o[2] = B[2];
      }
    }
    __syncthreads();
    // element sums in a fixed order
    if (tid < 2 * ng) {
      const int col = tid / 2, which = tid % 2;
      double v = 0;
      for (int qq = 0; qq < NQ3; ++qq) v += acc[(qq * FLUX_CG + col) * 2 + which];
      F.part[((int64_t)e * F.nrhs + c0 + col) * 2 + which] = v;
    }
    __syncthreads();
  }
}

// per patch and load case: sums of the element integrals of its elements
// (contiguous, [eoff[q], eoff[q+1])) in element order
__global__ void k_flux_patch(const double* part, const int64_t* eoff, int npatch, int nrhs, double* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npatch * nrhs * 2) return;
  const int which = t % 2, col = (t / 2) % nrhs, q = t / (2 * nrhs);
  double v = 0;
  for (int64_t e = eoff[q]; e < eoff[q + 1]; ++e) v += part[(e * nrhs + col) * 2 + which];
  out[((int64_t)which * nrhs + col) * npatch + q] = v;
}

template <int PD>
static size_t flux_smem() {
  constexpr int NQ3 = (PD + 1) * (PD + 1) * (PD + 1), NF = ElemShared<PD>::NF;
  return sizeof(ElemShared<PD>) + sizeof(double) * ((size_t)NF * NQ3 * 2 + (size_t)NF * FLUX_CG + NQ3 * FLUX_CG * 2);
}

// the dynamic shared memory of the flux kernels is exactly flux_smem (their
// static shared memory comes on top, within the opt-in limit)
template <int PD>
static ieti_status flux_attr(Ctx* c, int smem_max) {
  cudaFuncAttributes fa;
  IETI_CUDA_TRY(c, cudaFuncGetAttributes(&fa, k_elem_B<PD>));
  if (flux_smem<PD>() + fa.sharedSizeBytes > (size_t)smem_max) {
    c->err = "shared memory of the flux kernel exceeds the device limit";
    return IETI_ERR_INVALID_ARG;
  }
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_elem_B<PD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)flux_smem<PD>()));
  return IETI_OK;
}

ieti_status flux_kernel_attrs(Ctx* c, int smem_max) {
  ieti_status r;
  if ((r = flux_attr<1>(c, smem_max)) != IETI_OK) return r;
  if ((r = flux_attr<2>(c, smem_max)) != IETI_OK) return r;
  return flux_attr<3>(c, smem_max);
}

// B = curl a for nrhs fields; out = [npatch x nrhs] squared norms, then the
// squared errors against the reference field (device, 2 npatch nrhs values)
ieti_status eval_flux(Ctx* c, const double* a, int nrhs, int ref_kind, const double* amp_dev, double* part,
                      double* out, double* Bq, cudaStream_t st) {
  AsmParams P = make_params(c);
  FluxArgs F;
  F.a = a;
  F.nedge = c->mesh.nedge;
  F.nrhs = nrhs;
  F.ref_kind = ref_kind;
  F.amp = amp_dev;
  F.part = part;
  F.Bq = Bq;
  const unsigned ne = (unsigned)c->nelem;
  switch (c->mesh.p) {
    case 1: k_elem_B<1><<<ne, 256, flux_smem<1>(), st>>>(P, F); break;
    case 2: k_elem_B<2><<<ne, 256, flux_smem<2>(), st>>>(P, F); break;
    case 3: k_elem_B<3><<<ne, 256, flux_smem<3>(), st>>>(P, F); break;
    default: c->err = "degree p must be 1, 2 or 3"; return IETI_ERR_INVALID_ARG;
  }
  IETI_LAUNCH_CHECK(c);
  const int npatch = c->mesh.npatch();
  const int nt = npatch * nrhs * 2;
  k_flux_patch<<<(nt + 255) / 256, 256, 0, st>>>(part, c->d_patch_eoff, npatch, nrhs, out);
  IETI_LAUNCH_CHECK(c);
  return IETI_OK;
}

// dst <- src on the listed 64 x 64 tiles (k, I, J) of the K_rr blocks
template <typename T>
__global__ void __launch_bounds__(256) k_convert_tiles(const SubDev* sd, const int4* tiles, const double* src,
                                                       T* dst) {
  const int4 tl = tiles[blockIdx.x];
  const SubDev s = sd[tl.x];
  const int i = tl.y * NB + (int)threadIdx.x % NB;
  const int64_t base = s.A + i + (int64_t)s.n * (tl.z * NB + 16 * ((int)threadIdx.x / NB));
#pragma unroll 4
  for (int c = 0; c < 16; ++c) dst[base + (int64_t)s.n * c] = (T)src[base + (int64_t)s.n * c];
}

template <typename T>
ieti_status convert_tiles(Ctx* c, const int4* tiles, int ntiles, const double* src, T* dst, cudaStream_t st) {
  if (ntiles <= 0) return IETI_OK;
  k_convert_tiles<T><<<ntiles, 256, 0, st>>>(c->d_sd, tiles, src, dst);
  IETI_LAUNCH_CHECK(c);
  return IETI_OK;
}
template ieti_status convert_tiles<float>(Ctx*, const int4*, int, const double*, float*, cudaStream_t);
template ieti_status convert_tiles<double>(Ctx*, const int4*, int, const double*, double*, cudaStream_t);

// conversion used by the factorisation set-up
template <typename T>
ieti_status convert_copy(Ctx* c, const double* src, T* dst, int64_t n, cudaStream_t st) {
  k_copy_convert<T><<<1216, 256, 0, st>>>(src, dst, n);
  IETI_LAUNCH_CHECK(c);
  return IETI_OK;
}
template ieti_status convert_copy<float>(Ctx*, const double*, float*, int64_t, cudaStream_t);
template ieti_status convert_copy<double>(Ctx*, const double*, double*, int64_t, cudaStream_t);

}  // namespace ieti
