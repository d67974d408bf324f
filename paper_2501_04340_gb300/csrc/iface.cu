// Streamed interface products: the subdomain-local parts of the F-apply
// (Eq. (7)) and of the Dirichlet preconditioner (Eq. (10)).
//
// Both are batched dense GEMVs with the per-subdomain blocks M_k (W_k =
// S_rIrI^-1 for F, S_rIrI for the preconditioner): t_k = M_k u_k with
// u_k = D_k B_k^T x. For F the rows of Phi_I^(k)T are streamed with W_k, so the
// same pass also yields the primal partials q_k = Phi_I^(k)T u_k of the coarse
// correction G S_Pi^-1 G^T.
//
// The blocks are read exactly once per product, so the pass is bound by HBM
// bandwidth. Rows are cut into tiles of about 32 KB (whole rows, contiguous in
// memory); one CTA per SM owns a contiguous run of tiles with balanced bytes
// and streams them through a ring of shared-memory stages with bulk async
// copies (cp.async.bulk, completion on an mbarrier), several tiles ahead of the
// warps that consume them. u_k is gathered into shared memory while the first
// copies are in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "internal.h"
#include "stream.cuh"

namespace ieti {

namespace {

constexpr int ROW_TARGET_DEFAULT = 32 * 1024;   // bytes per row-mode tile before autotuning

struct StreamArgs {
  StreamCtx C;
  const int* cta;      // tile range start of every CTA (grid + 1 entries)
  double* t;
  double* qpart;
  int nrhs;
};

template <typename T, int CT, bool ROWS>
__global__ void __launch_bounds__(STREAM_THREADS, 1) k_stream(StreamArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  stream_init_bars(smem, A.C.stages);
  const int tb = A.cta[blockIdx.x], te = A.cta[blockIdx.x + 1];
  const int col0 = blockIdx.y * CT;
  uint32_t seq = 0, useq = 0;
  // the first tiles of the blocks do not depend on the u scatter before this
  // launch: they are in flight while it finishes
  int npre = 0;
  if (threadIdx.x >= NCONS) npre = stream_prefetch<T>(A.C, tb, te, smem, seq, CT);
  griddep_wait();
  stream_tiles<T, CT, ROWS>(A.C, tb, te, smem, seq, useq, A.t, A.qpart, A.nrhs, col0, min(CT, A.nrhs - col0),
                            npre);
  griddep_launch();
}

// u vectors of all subdomains: for both sides of multiplier l,
// u[col * utot + uoff_k + i] = sign * (scale) * x[l, col]; entries beyond nI_k
// stay zero
template <typename T>
__global__ void k_scatter_u(const int4* gs, const int2* gu, const double* I_sign, const double* I_scale,
                            const double* x, int64_t m, int nrhs, int64_t utot, T* uall) {
  griddep_launch();   // the streamed product may start fetching its tiles
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m * nrhs;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = q % m, col = q / m;
    const int4 a = gs[l];
    const int2 o = gu[l];
    const double v = x[l + m * col];
    const int i0 = a.x + a.y, i1 = a.z + a.w;
    const double w0 = I_sign[i0] * (I_scale ? I_scale[i0] : 1.0);
    const double w1 = I_sign[i1] * (I_scale ? I_scale[i1] : 1.0);
    uall[col * utot + o.x] = (T)(w0 * v);
    uall[col * utot + o.y] = (T)(w1 * v);
  }
  // the product reads u with bulk copies (async proxy), possibly launched
  // before this kernel has ended
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// y[l] = t_k0[i0] - t_k1[i1] + sum_e G[l, e] yc[g_e] (+ partial <y, dotv>), one
// column per blockIdx.y. yc = S_Pi^-1 qg is either read (yc_in) or, for a small
// coarse space, formed in every block: qg[g] = sum of the partials q_k[c] of
// the contributors of g, then the product with the explicit inverse.
__global__ void __launch_bounds__(256) k_gather_F3(const int4* gs, const int2* gn, const int32_t* gi,
                                                   const double* gv, int E, const double* t,
                                                   const int64_t* pcsr_off, const int4* pcon, const double* qpart,
                                                   const double* SPiInv, int ldc, const double* yc_in, int ngp,
                                                   int64_t m, int nrhs, double* y, const double* dotv, double* part) {
  griddep_wait();   // t and the primal partials come from the streamed product
  extern __shared__ double sm[];   // qg[ngp], yc[ngp]
  __shared__ double red[8];
  const int col = blockIdx.y;
  double* qg = sm;
  double* yc = sm + ngp;
  if (ngp > 0) {
    if (yc_in) {
      for (int g = threadIdx.x; g < ngp; g += blockDim.x) yc[g] = yc_in[g + (int64_t)ngp * col];
    } else {
      for (int g = threadIdx.x; g < ngp; g += blockDim.x) {
        double acc = 0;
        for (int64_t e = pcsr_off[g]; e < pcsr_off[g + 1]; ++e) {
          const int4 pc = pcon[e];   // pv, c, nP of a contributor
          acc += qpart[(int64_t)pc.x * nrhs + pc.y + (int64_t)pc.z * col];
        }
        qg[g] = acc;
      }
      __syncthreads();
      for (int g = threadIdx.x; g < ngp; g += blockDim.x) {
        const double* col_g = SPiInv + (int64_t)ldc * g;
        double acc = 0;
        for (int h = 0; h < ngp; ++h) acc += col_g[h] * qg[h];
        yc[g] = acc;
      }
    }
    __syncthreads();
  }
  double mydot = 0;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < m; l += (int64_t)gridDim.x * blockDim.x) {
    const int4 a = gs[l];
    const int2 nn = gn[l];
    double v = t[(int64_t)a.x * nrhs + a.y + (int64_t)nn.x * col] - t[(int64_t)a.z * nrhs + a.w + (int64_t)nn.y * col];
    if (ngp > 0) {
#pragma unroll 8
      for (int e = 0; e < E; ++e) v += gv[e * m + l] * yc[gi[e * m + l]];
    }
    y[l + m * col] = v;
    if (dotv) mydot += v * dotv[l + m * col];
  }
  if (part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mydot += __shfl_xor_sync(0xffffffffu, mydot, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = mydot;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
      part[blockIdx.x + gridDim.x * col] = s;
    }
  }
}

// z[l] = D t2_k0[i0] - D t2_k1[i1] (+ partial <z, dotv>)
__global__ void __launch_bounds__(256) k_gather_P2(const int4* gs, const int2* gn, const double* I_scale,
                                                   const double* t, int64_t m, int nrhs, double* z,
                                                   const double* dotv, double* part) {
  griddep_wait();   // t comes from the streamed product
  __shared__ double red[8];
  const int col = blockIdx.y;
  double mydot = 0;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < m; l += (int64_t)gridDim.x * blockDim.x) {
    const int4 a = gs[l];
    const int2 nn = gn[l];
    const double v = I_scale[a.x + a.y] * t[(int64_t)a.x * nrhs + a.y + (int64_t)nn.x * col] -
                     I_scale[a.z + a.w] * t[(int64_t)a.z * nrhs + a.w + (int64_t)nn.y * col];
    z[l + m * col] = v;
    if (dotv) mydot += v * dotv[l + m * col];
  }
  if (part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mydot += __shfl_xor_sync(0xffffffffu, mydot, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = mydot;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
      part[blockIdx.x + gridDim.x * col] = s;
    }
  }
}

// Phi_I^(k)T rows in the factor precision: PhiT[phio_k + c ldI + i] = Phi[nVp + i, c]
template <typename T>
__global__ void k_build_phiT(const SubDev* sd, const int64_t* phio, const double* Phi, T* PhiT) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  const int64_t tot = (int64_t)s.nP * s.ldI;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q / s.ldI), i = (int)(q % s.ldI);
    PhiT[phio[k] + q] = i < s.nI ? (T)Phi[s.Kp + s.nVp + i + (int64_t)s.n * c] : (T)0;
  }
}

// coarse part of the F gather as an ELL matrix G (m x E, column e contiguous):
// side 0 contributes +Phi_I^(k0)[i0, c], side 1 -Phi_I^(k1)[i1, c], at coarse
// index P_glob[c]; unused slots hold (0, 0.0)
__global__ void k_build_gell(const SubDev* sd, const int32_t* pair, const int32_t* P_glob, const double* Phi,
                             int64_t m, int E, int32_t* gi, double* gv) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < m; l += (int64_t)gridDim.x * blockDim.x) {
    int e = 0;
    for (int side = 0; side < 2; ++side) {
      const int k = pair[l * 4 + 2 * side], i = pair[l * 4 + 2 * side + 1];
      const SubDev s = sd[k];
      for (int c = 0; c < s.nP && e < E; ++c, ++e) {
        gi[e * m + l] = P_glob[s.pv + c];
        const double v = Phi[s.Kp + s.nVp + i + (int64_t)s.n * c];
        gv[e * m + l] = side == 0 ? v : -v;
      }
    }
    for (; e < E; ++e) {
      gi[e * m + l] = 0;
      gv[e * m + l] = 0.0;
    }
  }
}

template <typename T, int CT>
void set_stream_attr(int smem) {
  cudaFuncSetAttribute(k_stream<T, CT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (CT == 1) cudaFuncSetAttribute(k_stream<T, CT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <typename T>
ieti_status alloc_dev(Ctx* c, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed (interface streaming)";
    return IETI_ERR_OOM;
  }
  c->allocs.push_back({q, bytes});
  *p = (T*)q;
  return IETI_OK;
}

// tile table of one precision: rows of M_k (and of Phi_I^(k)T if with_phi) cut
// into whole-row tiles of about TILE_TARGET bytes, subdomain by subdomain; CTA
// j owns the tiles whose cost offsets start in [j C / grid, (j+1) C / grid),
// the cost being the bytes plus a fixed charge per subdomain entered
// Row mode (row_target > 0, one column): a warp reduces whole rows, so a tile
// may hold more than RMAX rows; tiles of about row_target bytes keep the same
// bytes in flight in every stage whatever the row length of the subdomain
// (with a fixed row count, CTAs on subdomains with short rows streamed fewer
// bytes per round trip and finished last).
ieti_status build_plan(Ctx* c, int es, bool with_phi, StreamPlan* P, int rcap = RMAX, int row_target = 0) {
  std::vector<LTile> tiles;
  std::vector<int64_t> start;   // balancing cost before each tile
  int64_t bytes = 0, cost = 0;
  // a CTA pays for the u vector of every subdomain its run enters (one bulk
  // copy waited for before the first product): about 1.5 us, the time of
  // streaming this many bytes at one SM's share of the bandwidth
  constexpr int64_t U_COST = 48 * 1024;
  int stage_bytes = 0;
  for (int k = 0; k < c->nsub; ++k) {
    const SubDev& s = c->sd_host[k];
    if (s.nI == 0) {
      if (with_phi && s.nP > 0) P->incomplete = true;
      continue;
    }
    const int64_t rb = (int64_t)s.ldI * es;
    // whole rows, at most RMAX of them, about TILE_TARGET bytes
    const int rpt = row_target > 0
                        ? (int)std::max<int64_t>(1, std::min<int64_t>(RROW_MAX, row_target / rb))
                        : (int)std::max<int64_t>(1, std::min<int64_t>(std::min(rcap, RMAX), TILE_TARGET / rb));
    stage_bytes = std::max<int>(stage_bytes, (int)(rpt * rb));
    for (int kind = 0; kind < (with_phi ? 2 : 1); ++kind) {
      const int rows = kind == 0 ? s.nI : s.nP;
      for (int r0 = 0; r0 < rows; r0 += rpt) {
        LTile tl{};
        tl.k = k;
        tl.row0 = r0;
        tl.nrows = std::min(rpt, rows - r0);
        tl.kind = kind;
        tl.ldI = s.ldI;
        tl.src = (kind == 0 ? s.S : c->phio[k]) + (int64_t)r0 * s.ldI;
        tl.obase = kind == 0 ? s.iv : s.pv;
        tl.ostride = kind == 0 ? s.nI : s.nP;
        tl.bytes = (int)(tl.nrows * rb);
        tl.uoff = c->uoff[k];
        if (kind == 0 && r0 == 0) cost += U_COST;
        start.push_back(cost);
        bytes += tl.nrows * rb;
        cost += tl.nrows * rb;
        tiles.push_back(tl);
      }
    }
  }
  const int grid = c->sm_count;
  std::vector<int> cta(grid + 1, (int)tiles.size());
  {
    int j = 0;
    for (int g = 0; g < grid; ++g) {
      const int64_t lo = (int64_t)((double)cost * g / grid);
      while (j < (int)tiles.size() && start[j] < lo) ++j;
      cta[g] = j;
    }
    cta[grid] = (int)tiles.size();
  }
  // the subdomains of every CTA's run (tiles are ordered by subdomain)
  std::vector<int2> ckr(grid, make_int2(0, 0));
  for (int g = 0; g < grid; ++g)
    if (cta[g] < cta[g + 1]) ckr[g] = make_int2(tiles[cta[g]].k, tiles[cta[g + 1] - 1].k + 1);
  LTile* dt;
  int* dc;
  int2* dk;
  ieti_status r;
  if ((r = alloc_dev(c, &dt, tiles.size())) != IETI_OK) return r;
  if ((r = alloc_dev(c, &dc, cta.size())) != IETI_OK) return r;
  if ((r = alloc_dev(c, &dk, ckr.size())) != IETI_OK) return r;
  IETI_CUDA_TRY(c, cudaMemcpy(dt, tiles.data(), sizeof(LTile) * tiles.size(), cudaMemcpyHostToDevice));
  IETI_CUDA_TRY(c, cudaMemcpy(dc, cta.data(), sizeof(int) * cta.size(), cudaMemcpyHostToDevice));
  IETI_CUDA_TRY(c, cudaMemcpy(dk, ckr.data(), sizeof(int2) * ckr.size(), cudaMemcpyHostToDevice));
  P->d_tiles = dt;
  P->d_cta = dc;
  P->d_ckr = dk;
  P->ntiles = (int)tiles.size();
  P->grid = grid;
  P->stage_bytes = stage_bytes;
  P->bytes = bytes;
  P->rows_cap = row_target > 0 ? RROW_MAX : rcap;
  P->row_target = row_target;
  P->built = true;
  return IETI_OK;
}

template <typename T>
size_t u_bytes(const Ctx* c, int ct) {
  return ((sizeof(T) * (size_t)c->max_ldI * ct + 127) / 128) * 128;
}


// largest column group (<= want) and stage count that fit in shared memory
template <typename T>
bool pick_shape(const Ctx* c, const StreamPlan& P, int want, int* ct, int* stages) {
  for (int g = want; g >= 1; g /= 2) {
    const long long avail = (long long)c->smem_optin - stream_hdr(g) - 2 * (long long)u_bytes<T>(c, g);
    const int st = (int)std::min<long long>(MAX_STAGES, avail / std::max(P.stage_bytes, 1));
    if (st >= 2) {
      *ct = g;
      *stages = st;
      return true;
    }
  }
  return false;
}

template <typename T, int CT>
ieti_status launch_stream(Ctx* c, const StreamPlan& P, bool with_phi, const double* x, const double* scale,
                          double* t, double* qpart, int nrhs, int stages, cudaStream_t st) {
  k_scatter_u<T><<<(unsigned)std::min<int64_t>(1024, ceil_div(c->m_r * nrhs, 256)), 256, 0, st>>>(
      c->d_gs, c->d_gu, c->d_I_sign, scale, x, c->m_r, nrhs, c->utot, (T*)c->uall);
  IETI_LAUNCH_CHECK(c);
  StreamArgs A;
  A.C.M = with_phi ? c->W : c->S;
  A.C.PhiT = c->PhiT;
  A.C.uall = c->uall;
  A.C.tiles = (const LTile*)P.d_tiles;
  A.C.utot = c->utot;
  A.C.u_ld = c->max_ldI;
  A.C.stages = stages;
  A.C.stage_bytes = P.stage_bytes;
  A.C.err = c->d_stream_err;
  A.C.l2_hint = 0;
  A.cta = P.d_cta;
  A.t = t;
  A.qpart = qpart;
  A.nrhs = nrhs;
  const size_t smem = stream_hdr(CT) + 2 * u_bytes<T>(c, CT) + (size_t)stages * P.stage_bytes;
  // one column with rows short enough for u in registers: row mode
  const bool rows = CT == 1 && c->max_ldI <= ROW_MAX_ELEMS;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(STREAM_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (rows) {
    cfg.gridDim = dim3(P.grid, (unsigned)nrhs);
    IETI_CUDA_TRY(c, cudaLaunchKernelEx(&cfg, k_stream<T, CT, true>, A));
  } else {
    cfg.gridDim = dim3(P.grid, (unsigned)ceil_div(nrhs, CT));
    IETI_CUDA_TRY(c, cudaLaunchKernelEx(&cfg, k_stream<T, CT, false>, A));
  }
  IETI_LAUNCH_CHECK(c);
  return IETI_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// host entry points
// ---------------------------------------------------------------------------

ieti_status iface_alloc(Ctx* c) {
  int dev = 0;
  IETI_CUDA_TRY(c, cudaGetDevice(&dev));
  IETI_CUDA_TRY(c, cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev));
  IETI_CUDA_TRY(c, cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  set_stream_attr<float, 1>(c->smem_optin);
  set_stream_attr<float, 2>(c->smem_optin);
  set_stream_attr<float, 4>(c->smem_optin);
  set_stream_attr<float, 8>(c->smem_optin);
  set_stream_attr<double, 1>(c->smem_optin);
  set_stream_attr<double, 2>(c->smem_optin);
  set_stream_attr<double, 4>(c->smem_optin);
  set_stream_attr<double, 8>(c->smem_optin);
  IETI_CUDA_TRY(c, cudaGetLastError());
  // Phi_I^T rows (allocated for FP64, used in the factor precision)
  c->phio.assign(c->nsub, 0);
  int64_t tot = 0;
  for (int k = 0; k < c->nsub; ++k) {
    c->phio[k] = tot;
    tot += (int64_t)c->sd_host[k].nP * c->sd_host[k].ldI;
  }
  ieti_status r;
  double* pt;
  if ((r = alloc_dev(c, &pt, tot)) != IETI_OK) return r;
  c->PhiT = pt;
  if ((r = alloc_dev(c, &c->d_phio, c->nsub)) != IETI_OK) return r;
  IETI_CUDA_TRY(c, cudaMemcpy(c->d_phio, c->phio.data(), sizeof(int64_t) * c->nsub, cudaMemcpyHostToDevice));
  // per multiplier: (iv, i) of both sides, their nI, and the ELL width
  const int64_t m = c->m_r;
  std::vector<int4> gs(std::max<int64_t>(m, 1));
  std::vector<int2> gn(std::max<int64_t>(m, 1));
  int E = 0;
  for (int64_t l = 0; l < m; ++l) {
    const int k0 = c->topo.dual_pair[l * 4], i0 = c->topo.dual_pair[l * 4 + 1];
    const int k1 = c->topo.dual_pair[l * 4 + 2], i1 = c->topo.dual_pair[l * 4 + 3];
    const SubDev &s0 = c->sd_host[k0], &s1 = c->sd_host[k1];
    gs[l] = make_int4((int)s0.iv, i0, (int)s1.iv, i1);
    gn[l] = make_int2(s0.nI, s1.nI);
    E = std::max(E, s0.nP + s1.nP);
  }
  c->gell_E = E;
  {
    // per local interface DOF: its multiplier and the other side's (iv, i, nI)
    std::vector<int4> jt(std::max<int64_t>(c->tot_iv, 1), make_int4(0, 0, 0, 0));
    for (int64_t l = 0; l < m; ++l) {
      const int k0 = c->topo.dual_pair[l * 4], i0 = c->topo.dual_pair[l * 4 + 1];
      const int k1 = c->topo.dual_pair[l * 4 + 2], i1 = c->topo.dual_pair[l * 4 + 3];
      const SubDev &s0 = c->sd_host[k0], &s1 = c->sd_host[k1];
      jt[s0.iv + i0] = make_int4((int)l, (int)s1.iv, i1, s1.nI);
      jt[s1.iv + i1] = make_int4((int)l, (int)s0.iv, i0, s0.nI);
    }
    ieti_status r2;
    if ((r2 = alloc_dev(c, &c->d_jt, jt.size())) != IETI_OK) return r2;
    IETI_CUDA_TRY(c, cudaMemcpy(c->d_jt, jt.data(), sizeof(int4) * jt.size(), cudaMemcpyHostToDevice));
  }
  // prepared u vectors: subdomain k's block at uoff_k (ldI_k entries), MAX_RHS columns
  c->uoff.assign(c->nsub, 0);
  int64_t ut = 0;
  for (int k = 0; k < c->nsub; ++k) {
    c->uoff[k] = ut;
    ut += c->sd_host[k].ldI;
  }
  c->utot = std::max<int64_t>(ut, 4);
  if ((r = alloc_dev(c, &c->d_uoff, c->uoff.size())) != IETI_OK) return r;
  IETI_CUDA_TRY(c, cudaMemcpy(c->d_uoff, c->uoff.data(), sizeof(int64_t) * c->uoff.size(), cudaMemcpyHostToDevice));
  std::vector<int2> gu(std::max<int64_t>(m, 1));
  for (int64_t l = 0; l < m; ++l) {
    const int k0 = c->topo.dual_pair[l * 4], i0 = c->topo.dual_pair[l * 4 + 1];
    const int k1 = c->topo.dual_pair[l * 4 + 2], i1 = c->topo.dual_pair[l * 4 + 3];
    gu[l] = make_int2((int)(c->uoff[k0] + i0), (int)(c->uoff[k1] + i1));
  }
  if ((r = alloc_dev(c, &c->d_gu, gu.size())) != IETI_OK) return r;
  IETI_CUDA_TRY(c, cudaMemcpy(c->d_gu, gu.data(), sizeof(int2) * gu.size(), cudaMemcpyHostToDevice));
  double* ua;
  if ((r = alloc_dev(c, &ua, (size_t)c->utot * MAX_RHS)) != IETI_OK) return r;
  IETI_CUDA_TRY(c, cudaMemset(ua, 0, sizeof(double) * (size_t)c->utot * MAX_RHS));
  c->uall = ua;
  if ((r = alloc_dev(c, &c->d_gs, gs.size())) != IETI_OK) return r;
  if ((r = alloc_dev(c, &c->d_gn, gn.size())) != IETI_OK) return r;
  IETI_CUDA_TRY(c, cudaMemcpy(c->d_gs, gs.data(), sizeof(int4) * gs.size(), cudaMemcpyHostToDevice));
  IETI_CUDA_TRY(c, cudaMemcpy(c->d_gn, gn.data(), sizeof(int2) * gn.size(), cudaMemcpyHostToDevice));
  if ((r = alloc_dev(c, &c->d_gell_i, std::max<int64_t>(m, 1) * std::max(E, 1))) != IETI_OK) return r;
  if ((r = alloc_dev(c, &c->d_gell_v, std::max<int64_t>(m, 1) * std::max(E, 1))) != IETI_OK) return r;
  // contributors of every coarse DOF as (pv_k, c, nP_k), for the gather
  if (c->n_gp > 0) {
    std::vector<int64_t> po(c->n_gp + 1);
    IETI_CUDA_TRY(c, cudaMemcpy(po.data(), c->d_pcsr_off, sizeof(int64_t) * po.size(), cudaMemcpyDeviceToHost));
    std::vector<int2> pc(std::max<int64_t>(po.back(), 1));
    if (po.back() > 0)
      IETI_CUDA_TRY(c, cudaMemcpy(pc.data(), c->d_pcsr, sizeof(int2) * po.back(), cudaMemcpyDeviceToHost));
    std::vector<int4> pcon(pc.size());
    for (int64_t e = 0; e < po.back(); ++e) {
      const SubDev& sk = c->sd_host[pc[e].x];
      pcon[e] = make_int4((int)sk.pv, pc[e].y, sk.nP, 0);
    }
    c->pcon_count = po.back();
    if ((r = alloc_dev(c, &c->d_pcon, pcon.size())) != IETI_OK) return r;
    IETI_CUDA_TRY(c, cudaMemcpy(c->d_pcon, pcon.data(), sizeof(int4) * pcon.size(), cudaMemcpyHostToDevice));
  }
  if ((r = alloc_dev(c, &c->d_stream_err, 4)) != IETI_OK) return r;
  IETI_CUDA_TRY(c, cudaMemset(c->d_stream_err, 0, sizeof(int)));
  return IETI_OK;
}

// Tile-shape autotuner: for each product (S, and W with the Phi_I^T rows) the
// rows per tile are chosen among 2, 4 and 8 by timing a few single-column
// products of this context's blocks with CUDA events (smaller tiles give more
// pipeline stages in the same shared memory, larger ones fewer copies); runs
// once per precision, after the blocks of the first factorisation exist
static ieti_status autotune_plans(Ctx* c, bool fp32, cudaStream_t st) {
  const int es = fp32 ? 4 : 8;
  double* x = c->wlam[6];
  // the multi-column plans are timed on all columns (a single column runs on
  // the row-mode plans when they exist)
  const int tn = c->nrhs;
  IETI_CUDA_TRY(c, cudaMemsetAsync(x, 0, sizeof(double) * std::max<int64_t>(c->m_r, 1) * tn, st));
  const bool trace = std::getenv("IETI_TRACE") != nullptr;
  cudaEvent_t e0, e1;
  IETI_CUDA_TRY(c, cudaEventCreate(&e0));
  IETI_CUDA_TRY(c, cudaEventCreate(&e1));
  const bool prof = c->prof.on;
  c->prof.on = false;
  ieti_status res = IETI_OK;
  for (int wp = 0; wp < 2 && res == IETI_OK && !(tn == 1 && c->rplan[fp32][wp].built); ++wp) {
    const StreamPlan def = c->splan[fp32][wp];
    StreamPlan best = def;
    float best_ms = -1.f;
    for (int rcap : {2, 4, RMAX}) {
      StreamPlan cand;
      if (rcap == def.rows_cap) cand = def;
      else if ((res = build_plan(c, es, wp == 1, &cand, rcap)) != IETI_OK) break;
      if (cand.incomplete || cand.ntiles == 0) continue;
      c->splan[fp32][wp] = cand;
      ieti_status r = IETI_OK;
      for (int it = 0; it < 3 && r == IETI_OK; ++it)
        r = iface_local(c, fp32, wp == 1, x, wp == 1 ? nullptr : c->d_I_scale, c->wi[0], c->wq_part, tn, st);
      if (r != IETI_OK) continue;   // this shape does not fit: not a candidate
      IETI_CUDA_TRY(c, cudaEventRecord(e0, st));
      for (int it = 0; it < 10 && r == IETI_OK; ++it)
        r = iface_local(c, fp32, wp == 1, x, wp == 1 ? nullptr : c->d_I_scale, c->wi[0], c->wq_part, tn, st);
      IETI_CUDA_TRY(c, cudaEventRecord(e1, st));
      IETI_CUDA_TRY(c, cudaEventSynchronize(e1));
      float ms = 0.f;
      IETI_CUDA_TRY(c, cudaEventElapsedTime(&ms, e0, e1));
      if (trace) std::fprintf(stderr, "[ieti] plan fp32=%d phi=%d rows<=%d: %.1f us\n", (int)fp32, wp, rcap, 100.f * ms);
      if (r == IETI_OK && (best_ms < 0.f || ms < best_ms)) {
        best_ms = ms;
        best = cand;
      }
    }
    c->splan[fp32][wp] = best;
  }
  // row-mode plans: the bytes per tile
  for (int wp = 0; wp < 2 && res == IETI_OK && c->rplan[fp32][0].built; ++wp) {
    const StreamPlan def = c->rplan[fp32][wp];
    StreamPlan best = def;
    float best_ms = -1.f;
    for (int target : {16 * 1024, 24 * 1024, 32 * 1024, 48 * 1024}) {
      StreamPlan cand;
      if (target == def.row_target) cand = def;
      else if ((res = build_plan(c, es, wp == 1, &cand, RMAX, target)) != IETI_OK) break;
      if (cand.incomplete || cand.ntiles == 0) continue;
      c->rplan[fp32][wp] = cand;
      ieti_status r = IETI_OK;
      for (int it = 0; it < 3 && r == IETI_OK; ++it)
        r = iface_local(c, fp32, wp == 1, x, wp == 1 ? nullptr : c->d_I_scale, c->wi[0], c->wq_part, 1, st);
      if (r != IETI_OK) continue;
      IETI_CUDA_TRY(c, cudaEventRecord(e0, st));
      for (int it = 0; it < 10 && r == IETI_OK; ++it)
        r = iface_local(c, fp32, wp == 1, x, wp == 1 ? nullptr : c->d_I_scale, c->wi[0], c->wq_part, 1, st);
      IETI_CUDA_TRY(c, cudaEventRecord(e1, st));
      IETI_CUDA_TRY(c, cudaEventSynchronize(e1));
      float ms = 0.f;
      IETI_CUDA_TRY(c, cudaEventElapsedTime(&ms, e0, e1));
      if (trace)
        std::fprintf(stderr, "[ieti] row plan fp32=%d phi=%d %d KB tiles: %.1f us\n", (int)fp32, wp, target / 1024,
                     100.f * ms);
      if (r == IETI_OK && (best_ms < 0.f || ms < best_ms)) {
        best_ms = ms;
        best = cand;
      }
    }
    c->rplan[fp32][wp] = best;
  }
  c->prof.on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  IETI_CUDA_TRY(c, cudaMemsetAsync(c->uall, 0, sizeof(double) * (size_t)c->utot * MAX_RHS, st));
  return res;
}

ieti_status iface_prepare(Ctx* c, cudaStream_t st) {
  const bool fp32 = c->prec == IETI_FP32_IR;
  const int es = fp32 ? 4 : 8;
  ieti_status r;
  for (int wp = 0; wp < 2; ++wp)
    if (!c->splan[fp32][wp].built && (r = build_plan(c, es, wp == 1, &c->splan[fp32][wp])) != IETI_OK) return r;
  if (c->max_ldI <= ROW_MAX_ELEMS)
    for (int wp = 0; wp < 2; ++wp)
      if (!c->rplan[fp32][wp].built &&
          (r = build_plan(c, es, wp == 1, &c->rplan[fp32][wp], RMAX, ROW_TARGET_DEFAULT)) != IETI_OK)
        return r;
  // the u vectors are read in the factor precision: clear them (their padding
  // entries must be zero in that view)
  IETI_CUDA_TRY(c, cudaMemsetAsync(c->uall, 0, sizeof(double) * (size_t)c->utot * MAX_RHS, st));
  if (c->max_nP > 0) {
    if (fp32) k_build_phiT<float><<<dim3(64, c->nsub), 256, 0, st>>>(c->d_sd, c->d_phio, c->Phi, (float*)c->PhiT);
    else k_build_phiT<double><<<dim3(64, c->nsub), 256, 0, st>>>(c->d_sd, c->d_phio, c->Phi, (double*)c->PhiT);
    IETI_LAUNCH_CHECK(c);
  }
  if (c->m_r > 0 && c->gell_E > 0) {
    k_build_gell<<<(unsigned)std::min<int64_t>(1024, ceil_div(c->m_r, 256)), 256, 0, st>>>(
        c->d_sd, c->d_pair, c->d_P_glob, c->Phi, c->m_r, c->gell_E, c->d_gell_i, c->d_gell_v);
    IETI_LAUNCH_CHECK(c);
  }
  if (c->autotune && !c->tuned[fp32] && c->m_r > 0) {
    if ((r = autotune_plans(c, fp32, st)) != IETI_OK) return r;
    c->tuned[fp32] = true;
  }
  return IETI_OK;
}

// t_k = M_k D_k B_k^T x for every subdomain (and q_k = Phi_I^(k)T B_k^T x if
// with_phi); IETI_ERR_STATE if the streamed form does not fit this context
ieti_status iface_local(Ctx* c, bool fp32, bool with_phi, const double* x, const double* scale, double* t,
                        double* qpart, int nrhs, cudaStream_t st) {
  // one column in row mode: the plan with tiles of equal bytes
  const bool rowp = nrhs == 1 && c->rplan[fp32][with_phi].built;
  const StreamPlan& P = rowp ? c->rplan[fp32][with_phi] : c->splan[fp32][with_phi];
  if (!P.built || P.ntiles == 0 || P.incomplete) return IETI_ERR_STATE;
  const int want = nrhs == 1 ? 1 : nrhs == 2 ? 2 : nrhs <= 4 ? 4 : 8;
  int ct = 0, stages = 0;
  const bool ok = fp32 ? pick_shape<float>(c, P, want, &ct, &stages) : pick_shape<double>(c, P, want, &ct, &stages);
  if (!ok) return IETI_ERR_STATE;
  const int cat = with_phi ? PROF_LOCAL_W : PROF_LOCAL_S;
  cudaEvent_t p0 = prof_begin(c, st);
  ieti_status r;
#define IETI_STREAM_CASE(TT, CC) \
  r = launch_stream<TT, CC>(c, P, with_phi, x, scale, t, qpart, nrhs, stages, st)
  if (fp32) {
    if (ct == 1) IETI_STREAM_CASE(float, 1);
    else if (ct == 2) IETI_STREAM_CASE(float, 2);
    else if (ct == 4) IETI_STREAM_CASE(float, 4);
    else IETI_STREAM_CASE(float, 8);
  } else {
    if (ct == 1) IETI_STREAM_CASE(double, 1);
    else if (ct == 2) IETI_STREAM_CASE(double, 2);
    else if (ct == 4) IETI_STREAM_CASE(double, 4);
    else IETI_STREAM_CASE(double, 8);
  }
#undef IETI_STREAM_CASE
  prof_end(c, cat, p0, st);
  return r;
}

// y = F lam from the local products t and the primal partials (qpart): the
// coarse solve is folded into the gather when the coarse space is small, else
// it runs first as its own kernel (k_coarse, into yc_buf)
bool iface_coarse_fused(const Ctx* c) { return c->n_gp * c->n_gp <= 32768; }

ieti_status iface_gather_F(Ctx* c, const double* t, const double* qpart, const double* yc, int nrhs, double* y,
                           const double* dotv, double* part, int blocks, cudaStream_t st) {
  cudaEvent_t p0 = prof_begin(c, st);
  const int ngp = (int)c->n_gp;
  const int ldc = (int)(ceil_div(std::max<int64_t>(c->n_gp, 1), NB) * NB);
  const size_t smem = sizeof(double) * 2 * std::max(ngp, 1);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks, nrhs);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const int E = c->gell_E;
  const int64_t m = c->m_r;
  IETI_CUDA_TRY(c, cudaLaunchKernelEx(&cfg, k_gather_F3, (const int4*)c->d_gs, (const int2*)c->d_gn,
                                      (const int32_t*)c->d_gell_i, (const double*)c->d_gell_v, E, t,
                                      (const int64_t*)c->d_pcsr_off, (const int4*)c->d_pcon, qpart,
                                      (const double*)c->SPiInv, ldc, yc, ngp, m, nrhs, y, dotv, part));
  prof_end(c, PROF_GATHER, p0, st);
  IETI_LAUNCH_CHECK(c);
  return IETI_OK;
}

ieti_status iface_gather_P(Ctx* c, const double* t, int nrhs, double* z, const double* dotv, double* part,
                           int blocks, cudaStream_t st) {
  cudaEvent_t p0 = prof_begin(c, st);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks, nrhs);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const int64_t m = c->m_r;
  IETI_CUDA_TRY(c, cudaLaunchKernelEx(&cfg, k_gather_P2, (const int4*)c->d_gs, (const int2*)c->d_gn,
                                      (const double*)c->d_I_scale, t, m, nrhs, z, dotv, part));
  prof_end(c, PROF_GATHER, p0, st);
  IETI_LAUNCH_CHECK(c);
  return IETI_OK;
}

// 1 if a bounded wait of the streamed products timed out since the last call
ieti_status iface_check(Ctx* c, cudaStream_t st) {
  IETI_CUDA_TRY(c, cudaMemcpyAsync(c->h_err + 1, c->d_stream_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  IETI_CUDA_TRY(c, cudaStreamSynchronize(st));
  if (c->h_err[1]) {
    c->err = "a bulk-copy wait of the interface products timed out";
    return IETI_ERR_TIMEOUT;
  }
  return IETI_OK;
}

}  // namespace ieti
