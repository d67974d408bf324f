// The PCG iteration on F_DP lam = b with the Dirichlet preconditioner
// (Eqs. (7), (10)) as one persistent launch built on the streamed interface
// products. One CTA per SM; the CTA streams its byte-balanced run of W (and
// Phi_I^T) tiles and of S tiles exactly as the stand-alone products do, and
// owns a contiguous slice of the multipliers for the vector work.
//
// Per iteration, four grid barriers:
//   A  t1_k = W_k u_k, q_k = Phi_I^(k)T u_k          (u = D_W p, written in F)
//   B  p = z + beta p on the owned slice (deferred from F);
//      yc = S_Pi^-1 sum C^T q_k (every CTA); q = F p = B t1 + G yc; <p, q>
//   C  alpha = rz / <p, q>; lam += alpha p; <r', r'> with r' = r - alpha q;
//      u = D_S r' for the subdomains of the CTA's S run; t2_k = S_k u_k
//   E  r = r'  on the owned slice (deferred from C); convergence test;
//      z = sum_k B_k D_k t2_k; <r, z>
//   F  beta = rz_new / rz; u = D_W (z + beta p) for the subdomains of the
//      CTA's W run
// The deferred updates keep r and p unchanged while other CTAs read them.
// Every CTA that streams tiles of subdomain k writes the whole u_k itself
// (all of them store identical values) and fences the async proxy before its
// bulk copies read it, so no barrier separates u from the product. Every CTA
// sums the per-CTA partials in the same order, so all CTAs take the same
// alpha, beta and convergence decisions.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "stream.cuh"

namespace cg = cooperative_groups;

namespace ieti {

namespace {

constexpr int PS_SC = 16;        // scalars per column: 0 rz, 2 rr, 3 bb, 4 alpha, 5 beta, 7 done, 8 its
constexpr int PS_MAXGP = 181;    // coarse DOFs handled inside every CTA (n_gp^2 <= 32768)

struct PcgStreamArgs {
  StreamCtx CW, CS;              // W (+ Phi_I^T) and S streams
  const int* ctaW;
  const int* ctaS;
  const int2* ckrW;              // subdomains of every CTA's W and S runs
  const int2* ckrS;
  const SubDev* sd;
  const int64_t* uoff;
  const int32_t* I_dual;
  double *x, *r, *z, *p, *q;
  double *t1, *t2, *qpart;
  double* part;                  // per-CTA partials [3][grid][CT]
  double* scal;
  double* hist;
  int hist_cap;
  const int4* gs;
  const int2* gn;
  const int2* gu;
  const int32_t* gi;
  const double* gv;
  int E;
  const double* I_sign;
  const double* I_scale;
  const int64_t* pcsr_off;
  const int4* pcon;
  const double* SPiInv;
  int ldc, ngp;
  int64_t m;
  int nrhs, maxit;
  double tol2;
  int* err;
  int64_t ncontrib;              // contributors of all coarse DOFs (pcsr entries)
  size_t cache_off;              // dynamic shared memory offset of the per-CTA caches
  int cache_slice;               // 1: the slice metadata is cached in shared memory
  int cache_coarse;              // 1: S_Pi^-1 and the contributor lists are cached
};

// Per-CTA caches (dynamic shared memory after the stream buffers): the
// metadata of the owned multipliers, read in every vector phase, and the
// coarse data, read in every gather. Layout (nl = owned multipliers):
//   gs int4[nl] | gn int2[nl] | gu int2[nl] | sg double2[nl] (signs of both
//   sides) | sc double2[nl] (rho-scaling of both sides) | gv double[E nl] |
//   gi int32[E nl] | then, if cached, S_Pi^-1 (ngp x ngp) | contributor values
//   double[ncontrib] | contributor offsets int32[ngp + 1] | contributors int4
struct Slice {
  int64_t l0, nl;
  const int4* gs;
  const int2* gn;
  const int2* gu;
  const double2* sg;
  const double2* sc;
  const double* gv;
  const int32_t* gi;
};

__host__ __device__ inline size_t slice_bytes(int64_t nl, int E) {
  return (size_t)nl * (16 + 8 + 8 + 16 + 16) + (size_t)nl * E * (8 + 4);
}
__host__ __device__ inline size_t round16(size_t b) { return (b + 15) / 16 * 16; }
__host__ __device__ inline size_t coarse_bytes(int ngp, int64_t ncontrib) {
  return round16((size_t)ngp * ngp * 8) + round16((size_t)ncontrib * 8) + round16((size_t)(ngp + 1) * 4) +
         (size_t)ncontrib * 16;
}

// CTA sum in a fixed order (all STREAM_THREADS threads; every thread gets it)
__device__ inline double ps_cta_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0;
  for (int w = 0; w < STREAM_THREADS / 32; ++w) s += red[w];
  return s;
}

// sum of one column's per-CTA partials, thread-strided then a fixed tree
__device__ inline double ps_sum_part(const double* part, int col, int ct, double* red) {
  double v = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += part[(int64_t)i * ct + col];
  return ps_cta_sum(v, red);
}

__device__ inline void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// u_k = D_k v at the r_I DOFs of every subdomain k in kr (D = sign, times the
// rho-scaling if scaled), v = a + s[col] b (b == nullptr: v = a); a column
// with keep[col] set takes v = b. Each local r_I DOF has one multiplier.
template <typename T, int CT>
__device__ inline void write_u_run(const PcgStreamArgs& A, int2 kr, const double* a, const double* b,
                                   const double* s, const int* keep, bool scaled) {
  T* u = (T*)A.CW.uall;
  for (int k = kr.x; k < kr.y; ++k) {
    const int64_t iv = A.sd[k].iv;
    const int nI = A.sd[k].nI;
    const int64_t uo = A.uoff[k];
    for (int q = threadIdx.x; q < nI * A.nrhs; q += blockDim.x) {
      const int i = q % nI, col = q / nI;
      const int64_t j = iv + i;
      const int64_t l = A.I_dual[j] + A.m * col;
      const double w = scaled ? A.I_sign[j] * A.I_scale[j] : A.I_sign[j];
      double v;
      if (b == nullptr) v = a[l];
      else if (keep[col]) v = b[l];
      else v = a[l] + s[col] * b[l];
      u[col * A.CW.utot + uo + i] = (T)(w * v);
    }
  }
  fence_async_global();
}

template <typename T, int CT, bool ROWS>
__global__ void __launch_bounds__(STREAM_THREADS, 1) k_pcg_stream(PcgStreamArgs A) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[STREAM_THREADS / 32];
  __shared__ double qg[PS_MAXGP * CT], yc[PS_MAXGP * CT];
  __shared__ double rz[CT], bb[CT], alpha[CT], beta[CT];
  __shared__ int done[CT];
  __shared__ int zero_keep[CT];
  __shared__ int its;
  const int tid = threadIdx.x, G = gridDim.x, bid = blockIdx.x;
  const int nrhs = A.nrhs, ngp = A.ngp;
  const int64_t m = A.m;
  const int64_t l0 = m * bid / G, l1 = m * (bid + 1) / G;   // owned multipliers
  stream_init_bars(smem, A.CW.stages);
  // ---- per-CTA caches
  const int64_t nl = l1 - l0;
  const int E = A.E;
  unsigned char* cbase = smem + A.cache_off;
  int4* c_gs = reinterpret_cast<int4*>(cbase);
  int2* c_gn = reinterpret_cast<int2*>(c_gs + nl);
  int2* c_gu = c_gn + nl;
  double2* c_sg = reinterpret_cast<double2*>(c_gu + nl);
  double2* c_sc = c_sg + nl;
  double* c_gv = reinterpret_cast<double*>(c_sc + nl);
  int32_t* c_gi = reinterpret_cast<int32_t*>(c_gv + (size_t)E * nl);
  unsigned char* cend = A.cache_slice ? reinterpret_cast<unsigned char*>(c_gi + (size_t)E * nl) : cbase;
  cend = reinterpret_cast<unsigned char*>(((uintptr_t)cend + 15) / 16 * 16);
  double* c_spi = reinterpret_cast<double*>(cend);   // each coarse buffer starts on 16 bytes
  double* c_cv = reinterpret_cast<double*>(cend + round16((size_t)ngp * ngp * 8));
  int32_t* c_co = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(c_cv) + round16((size_t)A.ncontrib * 8));
  int4* c_pc = reinterpret_cast<int4*>(reinterpret_cast<unsigned char*>(c_co) + round16((size_t)(ngp + 1) * 4));
  if (A.cache_slice) {
    for (int64_t i = tid; i < nl; i += blockDim.x) {
      const int64_t l = l0 + i;
      const int4 a = A.gs[l];
      c_gs[i] = a;
      c_gn[i] = A.gn[l];
      c_gu[i] = A.gu[l];
      c_sg[i] = make_double2(A.I_sign[a.x + a.y], A.I_sign[a.z + a.w]);
      c_sc[i] = make_double2(A.I_scale[a.x + a.y], A.I_scale[a.z + a.w]);
      for (int e = 0; e < E; ++e) {
        c_gv[(size_t)e * nl + i] = A.gv[e * m + l];
        c_gi[(size_t)e * nl + i] = A.gi[e * m + l];
      }
    }
  }
  if (A.cache_coarse) {
    for (int t = tid; t < ngp * ngp; t += blockDim.x) c_spi[t] = A.SPiInv[(int64_t)A.ldc * (t / ngp) + t % ngp];
    for (int g = tid; g <= ngp; g += blockDim.x) c_co[g] = (int32_t)A.pcsr_off[g];
    for (int64_t e = tid; e < A.ncontrib; e += blockDim.x) c_pc[e] = A.pcon[e];
  }
  Slice SL;
  SL.l0 = l0;
  SL.nl = nl;
  if (A.cache_slice) {
    SL.gs = c_gs; SL.gn = c_gn; SL.gu = c_gu; SL.sg = c_sg; SL.sc = c_sc; SL.gv = c_gv; SL.gi = c_gi;
  } else {
    SL.gs = A.gs + l0; SL.gn = A.gn + l0; SL.gu = A.gu + l0; SL.sg = nullptr; SL.sc = nullptr;
    SL.gv = A.gv + l0; SL.gi = A.gi + l0;
  }
  const int64_t estride = A.cache_slice ? nl : m;
  __syncthreads();
  if (tid < CT) {
    rz[tid] = tid < nrhs ? A.scal[PS_SC * tid + 0] : 0.0;
    bb[tid] = tid < nrhs ? A.scal[PS_SC * tid + 3] : 1.0;
    done[tid] = tid < nrhs ? (A.scal[PS_SC * tid + 7] != 0.0) : 1;
  }
  if (tid == 0) its = (int)A.scal[8];
  if (tid < CT) zero_keep[tid] = 0;
  uint32_t seq = 0, useq = 0;
  const bool producer = tid >= NCONS;
  int npreW = 0, npreS = 0;   // tiles of the next W / S pass already in flight (producer warp)
  double* pq_part = A.part;
  double* rr_part = A.part + (int64_t)G * CT;
  double* rz_part = A.part + 2 * (int64_t)G * CT;
  const int2 krW = A.ckrW[bid], krS = A.ckrS[bid];
  // u = D_W p for the first product; the first W tiles are fetched meanwhile
  if (producer) npreW = stream_prefetch<T>(A.CW, A.ctaW[bid], A.ctaW[bid + 1], smem, seq, CT);
  write_u_run<T, CT>(A, krW, A.p, nullptr, nullptr, nullptr, false);
  __syncthreads();   // every thread's u stores and fence precede the bulk copies
  bool pend_p = false;   // p = z + beta p still to be applied to the owned slice
  int upd[CT];           // columns that this iteration's alpha updates
  for (int iter = 0; iter < A.maxit; ++iter) {
    bool all = true;
    for (int cc = 0; cc < nrhs; ++cc) all &= done[cc] != 0;
    if (all || *(volatile int*)A.err) break;
    // ---- A: local products with W and the primal partials
    stream_tiles<T, CT, ROWS>(A.CW, A.ctaW[bid], A.ctaW[bid + 1], smem, seq, useq, A.t1, A.qpart, nrhs, 0, nrhs,
                              npreW);
    npreW = 0;
    grid.sync();
    // the first S tiles are fetched while the vector phases run
    if (producer) npreS = stream_prefetch<T>(A.CS, A.ctaS[bid], A.ctaS[bid + 1], smem, seq, CT);
    // ---- B: deferred p update; coarse correction (every CTA), q = F p, partial <p, q>
    if (pend_p) {
      for (int64_t l = l0 + tid; l < l1; l += blockDim.x)
#pragma unroll
        for (int col = 0; col < CT; ++col) {
          if (col >= nrhs) break;
          if (!done[col]) A.p[l + m * col] = A.z[l + m * col] + beta[col] * A.p[l + m * col];
        }
      pend_p = false;
      __syncthreads();
    }
    if (ngp > 0) {
      if (A.cache_coarse) {
        // contributor values in parallel, then ordered sums per coarse DOF
        for (int col = 0; col < nrhs; ++col) {
          for (int64_t e = tid; e < A.ncontrib; e += blockDim.x) {
            const int4 pc = c_pc[e];
            c_cv[e] = A.qpart[(int64_t)pc.x * nrhs + pc.y + (int64_t)pc.z * col];
          }
          __syncthreads();
          for (int g = tid; g < ngp; g += blockDim.x) {
            double acc = 0;
            for (int e = c_co[g]; e < c_co[g + 1]; ++e) acc += c_cv[e];
            qg[g + ngp * col] = acc;
          }
          __syncthreads();
        }
        for (int t = tid; t < ngp * nrhs; t += blockDim.x) {
          const int g = t % ngp, col = t / ngp;
          const double* sp = c_spi + (size_t)ngp * g;
          double acc = 0;
          for (int h = 0; h < ngp; ++h) acc += sp[h] * qg[h + ngp * col];
          yc[t] = acc;
        }
      } else {
        for (int t = tid; t < ngp * nrhs; t += blockDim.x) {
          const int g = t % ngp, col = t / ngp;
          double acc = 0;
          for (int64_t e = A.pcsr_off[g]; e < A.pcsr_off[g + 1]; ++e) {
            const int4 pc = A.pcon[e];
            acc += A.qpart[(int64_t)pc.x * nrhs + pc.y + (int64_t)pc.z * col];
          }
          qg[t] = acc;
        }
        __syncthreads();
        for (int t = tid; t < ngp * nrhs; t += blockDim.x) {
          const int g = t % ngp, col = t / ngp;
          const double* cg_ = A.SPiInv + (int64_t)A.ldc * g;
          double acc = 0;
          for (int h = 0; h < ngp; ++h) acc += cg_[h] * qg[h + ngp * col];
          yc[t] = acc;
        }
      }
      __syncthreads();
    }
    double mine[CT];
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) mine[cc] = 0;
    for (int64_t i = tid; i < nl; i += blockDim.x) {
      const int64_t l = l0 + i;
      const int4 a = SL.gs[i];
      const int2 nn = SL.gn[i];
#pragma unroll
      for (int col = 0; col < CT; ++col) {
        if (col >= nrhs) break;
        double v = A.t1[(int64_t)a.x * nrhs + a.y + (int64_t)nn.x * col] -
                   A.t1[(int64_t)a.z * nrhs + a.w + (int64_t)nn.y * col];
        if (ngp > 0) {
#pragma unroll 8
          for (int e = 0; e < E; ++e) v += SL.gv[e * estride + i] * yc[SL.gi[e * estride + i] + ngp * col];
        }
        A.q[l + m * col] = v;
        mine[col] += v * A.p[l + m * col];
      }
    }
    for (int cc = 0; cc < nrhs; ++cc) {
      const double s = ps_cta_sum(mine[cc], red);
      if (tid == 0) pq_part[(int64_t)bid * CT + cc] = s;
    }
    grid.sync();
    // ---- C: alpha; lam update; partial <r', r'>; u = D_S r'; products with S
    for (int cc = 0; cc < nrhs; ++cc) {
      const double pq = ps_sum_part(pq_part, cc, CT, red);
      if (tid == 0) alpha[cc] = (done[cc] || pq == 0.0) ? 0.0 : rz[cc] / pq;
    }
    __syncthreads();
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) {
      mine[cc] = 0;
      upd[cc] = cc < nrhs && !done[cc];
    }
    for (int64_t l = l0 + tid; l < l1; l += blockDim.x) {
#pragma unroll
      for (int col = 0; col < CT; ++col) {
        if (col >= nrhs) break;
        const int64_t o = l + m * col;
        double rv = A.r[o];
        if (upd[col]) {
          A.x[o] += alpha[col] * A.p[o];
          rv -= alpha[col] * A.q[o];
        }
        mine[col] += rv * rv;
      }
    }
    for (int cc = 0; cc < nrhs; ++cc) {
      const double s = ps_cta_sum(mine[cc], red);
      if (tid == 0) rr_part[(int64_t)bid * CT + cc] = s;
    }
    {
      // r' = r - alpha q (alpha = 0 for finished columns)
      double nalpha[CT];
#pragma unroll
      for (int cc = 0; cc < CT; ++cc) nalpha[cc] = -alpha[cc];
      write_u_run<T, CT>(A, krS, A.r, A.q, nalpha, zero_keep, true);
      __syncthreads();   // every thread's u stores and fence precede the bulk copies
    }
    stream_tiles<T, CT, ROWS>(A.CS, A.ctaS[bid], A.ctaS[bid + 1], smem, seq, useq, A.t2, nullptr, nrhs, 0, nrhs,
                              npreS);
    npreS = 0;
    grid.sync();
    if (producer) npreW = stream_prefetch<T>(A.CW, A.ctaW[bid], A.ctaW[bid + 1], smem, seq, CT);
    // ---- E: deferred r update; convergence test; z = preconditioned r, partial <r, z>
    for (int64_t l = l0 + tid; l < l1; l += blockDim.x)
#pragma unroll
      for (int col = 0; col < CT; ++col) {
        if (col >= nrhs) break;
        if (upd[col]) A.r[l + m * col] -= alpha[col] * A.q[l + m * col];
      }
    for (int cc = 0; cc < nrhs; ++cc) {
      const double rr = ps_sum_part(rr_part, cc, CT, red);
      if (tid == 0 && !done[cc]) {
        if (bid == 0) {
          A.scal[PS_SC * cc + 2] = rr;
          A.scal[PS_SC * cc + 4] = alpha[cc];
          A.scal[PS_SC * cc + 8] += 1.0;
        }
        if (rr <= A.tol2 * bb[cc]) done[cc] = 1;
      }
    }
    if (tid == 0) {
      ++its;
      if (bid == 0 && A.hist && its <= A.hist_cap) A.hist[2 * (its - 1)] = alpha[0];
    }
    __syncthreads();
    {
      bool fin = true;
      for (int cc = 0; cc < nrhs; ++cc) fin &= done[cc] != 0;
      if (fin) break;
    }
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) mine[cc] = 0;
    for (int64_t i = tid; i < nl; i += blockDim.x) {
      const int64_t l = l0 + i;
      const int4 a = SL.gs[i];
      const int2 nn = SL.gn[i];
      double s0, s1;
      if (SL.sc) {
        const double2 sc = SL.sc[i];
        s0 = sc.x;
        s1 = sc.y;
      } else {
        s0 = A.I_scale[a.x + a.y];
        s1 = A.I_scale[a.z + a.w];
      }
#pragma unroll
      for (int col = 0; col < CT; ++col) {
        if (col >= nrhs) break;
        const double v = s0 * A.t2[(int64_t)a.x * nrhs + a.y + (int64_t)nn.x * col] -
                         s1 * A.t2[(int64_t)a.z * nrhs + a.w + (int64_t)nn.y * col];
        A.z[l + m * col] = v;
        mine[col] += v * A.r[l + m * col];
      }
    }
    for (int cc = 0; cc < nrhs; ++cc) {
      const double s = ps_cta_sum(mine[cc], red);
      if (tid == 0) rz_part[(int64_t)bid * CT + cc] = s;
    }
    grid.sync();
    // ---- F: beta; u = D_W (z + beta p) (the owned p follows in B)
    for (int cc = 0; cc < nrhs; ++cc) {
      const double rzn = ps_sum_part(rz_part, cc, CT, red);
      if (tid == 0) {
        beta[cc] = (done[cc] || rz[cc] == 0.0) ? 0.0 : rzn / rz[cc];
        if (!done[cc]) {
          rz[cc] = rzn;
          if (bid == 0) {
            A.scal[PS_SC * cc + 0] = rzn;
            A.scal[PS_SC * cc + 5] = beta[cc];
          }
        }
      }
    }
    __syncthreads();
    if (bid == 0 && tid == 0 && A.hist && its <= A.hist_cap) A.hist[2 * (its - 1) + 1] = beta[0];
    write_u_run<T, CT>(A, krW, A.z, A.p, beta, done, false);
    pend_p = true;
    __syncthreads();   // every thread's u stores and fence precede the bulk copies
  }
  if (pend_p) {
    for (int64_t l = l0 + tid; l < l1; l += blockDim.x)
#pragma unroll
      for (int col = 0; col < CT; ++col) {
        if (col >= nrhs) break;
        if (!done[col]) A.p[l + m * col] = A.z[l + m * col] + beta[col] * A.p[l + m * col];
      }
  }
  // tiles fetched ahead for a pass that will not run
  if (producer) stream_drain(smem, seq, npreW + npreS, A.CW.stages);
  if (bid == 0 && tid < nrhs) A.scal[PS_SC * tid + 7] = done[tid] ? 1.0 : 0.0;
}

template <typename T, int CT, bool ROWS>
ieti_status launch_pcg_stream(Ctx* c, PcgStreamArgs A, int stages_max, size_t ubytes, cudaStream_t st) {
  auto kern = k_pcg_stream<T, CT, ROWS>;
  cudaFuncAttributes fa;
  IETI_CUDA_TRY(c, cudaFuncGetAttributes(&fa, kern));
  const StreamPlan& PW = c->splan[sizeof(T) == 4][1];
  const StreamPlan& PS = c->splan[sizeof(T) == 4][0];
  const int stage_bytes = std::max(PW.stage_bytes, PS.stage_bytes);
  // caches: the slice metadata if it takes at most 40 KB, the coarse data if
  // n_gp <= 64
  const int64_t nlmax = ceil_div(A.m, PW.grid) + 1;
  A.cache_slice = slice_bytes(nlmax, A.E) <= 40 * 1024;
  A.cache_coarse = A.ngp > 0 && A.ngp <= 64;
  const size_t cache = (A.cache_slice ? (slice_bytes(nlmax, A.E) + 15) / 16 * 16 : 0) +
                       (A.cache_coarse ? coarse_bytes(A.ngp, A.ncontrib) : 0);
  const long long avail = (long long)c->smem_optin - (long long)fa.sharedSizeBytes - stream_hdr(CT) -
                          2 * (long long)ubytes - (long long)cache - 128;
  const int stages = (int)std::min<long long>(stages_max, avail / std::max(stage_bytes, 1));
  if (stages < 2) return IETI_ERR_STATE;
  A.CW.stages = A.CS.stages = stages;
  A.CW.stage_bytes = A.CS.stage_bytes = stage_bytes;
  A.cache_off = ((size_t)stream_hdr(CT) + 2 * ubytes + (size_t)stages * stage_bytes + 127) / 128 * 128;
  const size_t smem = A.cache_off + cache;
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  IETI_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, STREAM_THREADS, smem));
  if (per_sm < 1 || PW.grid > per_sm * c->sm_count) return IETI_ERR_STATE;
  void* args[] = {(void*)&A};
  cudaEvent_t p0 = prof_begin(c, st, PROF_PCG);
  IETI_CUDA_TRY(c, cudaLaunchCooperativeKernel((void*)kern, dim3(PW.grid), dim3(STREAM_THREADS), args, smem, st));
  prof_end(c, PROF_PCG, p0, st);
  IETI_LAUNCH_CHECK(c);
  return IETI_OK;
}

}  // namespace

// The whole PCG loop in one cooperative launch on the streamed products.
// IETI_ERR_STATE when this form does not apply (more than 8 columns, a coarse
// space larger than PS_MAXGP, tile plans missing, no cooperative launch).
ieti_status pcg_stream(Ctx* c, double* lam, double* r, double* z, double* p, double* q, double tol2, int maxit,
                       bool fp32, cudaStream_t st) {
  const int nrhs = c->nrhs;
  const StreamPlan& PW = c->splan[fp32][1];
  const StreamPlan& PS = c->splan[fp32][0];
  if (nrhs > 8 || c->n_gp > PS_MAXGP || !PW.built || !PS.built || PW.incomplete || PW.ntiles == 0 ||
      PS.ntiles == 0 || PW.grid != PS.grid)
    return IETI_ERR_STATE;
  int dev = 0, coop = 0;
  IETI_CUDA_TRY(c, cudaGetDevice(&dev));
  IETI_CUDA_TRY(c, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return IETI_ERR_STATE;
  PcgStreamArgs A;
  A.CW.M = c->W;
  A.CW.PhiT = c->PhiT;
  A.CW.uall = c->uall;
  A.CW.tiles = (const LTile*)PW.d_tiles;
  A.CW.utot = c->utot;
  A.CW.u_ld = c->max_ldI;
  A.CW.err = c->d_stream_err;
  A.CS = A.CW;
  A.CS.M = c->S;
  A.CS.tiles = (const LTile*)PS.d_tiles;
  A.ctaW = PW.d_cta;
  A.ctaS = PS.d_cta;
  A.ckrW = PW.d_ckr;
  A.ckrS = PS.d_ckr;
  A.sd = c->d_sd;
  A.uoff = c->d_uoff;
  A.I_dual = c->d_I_dual;
  A.x = lam;
  A.r = r;
  A.z = z;
  A.p = p;
  A.q = q;
  A.t1 = c->wi[0];
  A.t2 = c->wi[1];
  A.qpart = c->wq_part;
  A.part = c->wred;
  A.scal = c->wscal;
  A.hist = c->whist;
  A.hist_cap = 4096;
  A.gs = c->d_gs;
  A.gn = c->d_gn;
  A.gu = c->d_gu;
  A.gi = c->d_gell_i;
  A.gv = c->d_gell_v;
  A.E = c->gell_E;
  A.I_sign = c->d_I_sign;
  A.I_scale = c->d_I_scale;
  A.pcsr_off = c->d_pcsr_off;
  A.pcon = c->d_pcon;
  A.SPiInv = c->SPiInv;
  A.ldc = (int)(ceil_div(std::max<int64_t>(c->n_gp, 1), NB) * NB);
  A.ngp = (int)c->n_gp;
  A.m = c->m_r;
  A.nrhs = nrhs;
  A.maxit = maxit;
  A.tol2 = tol2;
  A.err = c->d_stream_err;
  A.ncontrib = c->pcon_count;
  const bool rows = nrhs == 1 && c->max_ldI <= ROW_MAX_ELEMS;
  const size_t ub1 = ((size_t)c->max_ldI * (fp32 ? 4 : 8) + 127) / 128 * 128;
  if (nrhs == 1) {
    if (fp32)
      return rows ? launch_pcg_stream<float, 1, true>(c, A, MAX_STAGES, ub1, st)
                  : launch_pcg_stream<float, 1, false>(c, A, MAX_STAGES, ub1, st);
    return rows ? launch_pcg_stream<double, 1, true>(c, A, MAX_STAGES, ub1, st)
                : launch_pcg_stream<double, 1, false>(c, A, MAX_STAGES, ub1, st);
  }
  return fp32 ? launch_pcg_stream<float, 8, false>(c, A, MAX_STAGES, ub1 * 8, st)
              : launch_pcg_stream<double, 8, false>(c, A, MAX_STAGES, ub1 * 8, st);
}

}  // namespace ieti
