// The PCG iteration on F_DP lam = b with the Dirichlet preconditioner
// (Eqs. (7), (10)) as one persistent launch built on the streamed interface
// products. One CTA per SM; the CTA streams its byte-balanced run of W (and
// Phi_I^T) tiles and of S tiles exactly as the stand-alone products do, and
// owns a contiguous slice of the multipliers for the vector work.
//
// Both inner products of an iteration are sums over the rows the products
// produce: <p, B t1> = sum_k u_k . t1_k with u_k = D_W,k B_k^T p, and
// <r', z'> = sum_k u_k . t2_k with u_k = D_S,k B_k^T r' (D diagonal), so the
// streaming passes form them on the fly and no reduction phase follows a
// gather. r and p are double-buffered, so a CTA never reads a value another
// CTA rewrites in the same phase, and the owner of a multiplier writes the
// entries of the next u vectors at both of its sides. Per iteration, four
// grid barriers, two of them after balanced vector phases:
//   P1  t1_k = W_k u_k, q_k = Phi_I^(k)T u_k (u = D_W p) and the CTA's share
//       of <p, B t1>                                                   | barrier
//   P2  every CTA: yc = S_Pi^-1 sum C^T q_k, <p, F p> = sum of the shares
//       + (G^T p) . yc, alpha. Owned slice: q = B t1 + G yc, lam += alpha p,
//       r' = r - alpha q into the other r buffer, u = D_S r' at both sides,
//       share of <r', r'>                                              | barrier
//   P3  t2_k = S_k u_k and the CTA's share of <r', z'>                 | barrier
//   P4  every CTA: convergence test on <r', r'>, beta = <r', z'> / <r, z>.
//       Owned slice: z' = sum_k B_k D_k t2_k, p' = z' + beta p into the other
//       p buffer, u = D_W p' at both sides                             | barrier
// Every CTA sums the per-CTA shares in the same order, so all CTAs take the
// same alpha, beta and convergence decisions. The loads of a vector phase are
// issued in one round before its block reductions, since the data were
// written by other SMs and every round trip costs an L2 latency. The W tiles
// are fetched with the L2 evict-last priority and the S tiles with
// evict-first, so that W stays in L2 from one iteration to the next when W and
// S together exceed it.
//
// The vectors and scalars of the loop are kept in the operators' precision V:
// FP64 with FP64 operators, FP32 with FP32 operators (the inner solve of the
// refinement, which stops at a relative residual of 1e-3 or above). GB300
// issues an FP64 fused multiply-add at 2 per clock per SM with a dependent
// latency of 64 clocks, so FP64 chains in the latency-bound vector phases cost
// far more than the FP32 ones. The FP32 vectors are normalised per column by
// ||b|| so that no value leaves the FP32 range; the shared scalars written for
// the host are scaled back.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

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
  void *x, *r, *z, *p, *q;       // lam, r, p, and the second r (q) and p (z) buffers (V)
  double *t1, *t2, *qpart;
  double* part;                  // per-CTA shares [3][grid][CT]: <p, B t1>, <r', r'>, <r', z'>
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
  int vscaled;                   // 1: the vectors are divided by ||b|| per column (FP32 vectors)
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
template <typename V>
using Vec2 = typename std::conditional<sizeof(V) == 4, float2, double2>::type;

template <typename V>
struct Slice {
  int64_t l0, nl;
  const int4* gs;
  const int2* gn;
  const int2* gu;
  const Vec2<V>* sg;
  const Vec2<V>* sc;
  const V* gv;                   // cached coarse map, else nullptr and gv64 (FP64, in global memory)
  const double* gv64;
  const int32_t* gi;
};

// vs: bytes of V
__host__ __device__ inline size_t slice_bytes(int64_t nl, int E, int vs) {
  return (size_t)nl * (16 + 8 + 8 + 4 * vs) + (size_t)nl * E * (vs + 4);
}
__host__ __device__ inline size_t round16(size_t b) { return (b + 15) / 16 * 16; }
__host__ __device__ inline size_t coarse_bytes(int ngp, int64_t ncontrib, int vs) {
  return round16((size_t)ngp * ngp * vs) + round16((size_t)ncontrib * vs) + round16((size_t)(ngp + 1) * 4) +
         (size_t)ncontrib * 16;
}

__device__ inline void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// u_k = D_k v at the r_I DOFs of every subdomain k in kr (D = sign, times the
// rho-scaling if scaled), v = a + s[col] b (b == nullptr: v = a); a column
// with keep[col] set takes v = b. Each local r_I DOF has one multiplier.
template <typename T, int CT, typename V>
__device__ inline void write_u_run(const PcgStreamArgs& A, int2 kr, const V* a, const V* b,
                                   const V* s, const int* keep, bool scaled) {
  T* u = (T*)A.CW.uall;
  for (int k = kr.x; k < kr.y; ++k) {
    const int64_t iv = A.sd[k].iv;
    const int nI = A.sd[k].nI;
    const int64_t uo = A.uoff[k];
    for (int q = threadIdx.x; q < nI * A.nrhs; q += blockDim.x) {
      const int i = q % nI, col = q / nI;
      const int64_t j = iv + i;
      const int64_t l = A.I_dual[j] + A.m * col;
      const V w = (V)(scaled ? A.I_sign[j] * A.I_scale[j] : A.I_sign[j]);
      V v;
      if (b == nullptr) v = a[l];
      else if (keep[col]) v = b[l];
      else v = a[l] + s[col] * b[l];
      u[col * A.CW.utot + uo + i] = (T)(w * v);
    }
  }
  fence_async_global();
}

// Vector phases run on the consumer warps alone (named barrier 2), so that the
// producer warp can issue the bulk copies of the next pass meanwhile.
__device__ __forceinline__ void cons_sync() { asm volatile("bar.sync 2, 256;" ::: "memory"); }

// The producer warp starts the bulk copies of the next pass only once the
// consumers hold the loads of their vector phase (named barrier 3): issued at
// the start of the phase, the copies of all SMs held those L2 loads up by
// about 2 us. (Whatever part of the phase runs under the copies slows down by
// about as much; the copies ahead still pay for themselves at the pass start.)
__device__ __forceinline__ void gate_open() { asm volatile("bar.arrive 3, 288;" ::: "memory"); }
__device__ __forceinline__ void gate_wait() { asm volatile("bar.sync 3, 288;" ::: "memory"); }

// Block sum over the consumer warps of one value per thread, in the warps
// [0, nw) that hold nonzero values; red: [8] values; cons_sum_end (after the
// next cons_sync) adds the warp sums. The partial sums are formed once, not in
// every thread.
template <typename V>
__device__ __forceinline__ void cons_sum_begin(V v, int nw, V* red) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (warp < nw) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
  }
}
template <typename V>
__device__ __forceinline__ V cons_sum_end(int nw, const V* red) {
  V s = 0;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// z' = s0 t2(side 0) - s1 t2(side 1) of the multiplier, as one expression
template <typename V>
__device__ __forceinline__ V zgather(V s0, V ta, V s1, V tb) {
  return fma(s0, ta, -(s1 * tb));
}

// state of the vector phases of one CTA: the shared-memory caches and
// scalars of the kernel
template <typename V, int CT>
struct PhaseCtx {
  Slice<V> SL;
  int64_t l0, nl, estride, m;
  int E, ngp, nrhs, G, bid, nwG, nwL;
  V* c_spi;
  V* c_cv;
  const int32_t* c_co;
  const int4* c_pc;
  V *qg, *yc, *redA, *redB, *rz, *bb, *alpha_s, *beta_s;
  double* s2;                    // ||b||^2 per column when the vectors are normalised, else 1
  int* done;
  int* its;
  int* itc;                      // iterations per column
  double *pW, *pR, *pZ;          // per-CTA shares (FP64 in memory)
};

// The vector phases are out-of-line functions of the consumer warps: compiled
// inside the register-capped kernel body, the same straight-line code
// scheduled far worse (P4 took 6.8 us per iteration inline against 2 us as a
// separate body).
template <typename T, int CT>
__device__ __noinline__ void pcg_phase2(const PcgStreamArgs& A, const PhaseCtx<T, CT>& X, T* rc, T* rn, T* pc) {
  using V = T;
  const int tid = threadIdx.x;
  const Slice<V>& SL = X.SL;
  const int64_t l0 = X.l0, nl = X.nl, estride = X.estride, m = X.m;
  const int E = X.E, ngp = X.ngp, nrhs = X.nrhs, G = X.G, bid = X.bid, nwG = X.nwG, nwL = X.nwL;
  V* xv = static_cast<V*>(A.x);
  // ---- P2 (consumers): one round of loads (the shares of <p, B t1>, the
  // primal partials of the coarse DOFs, the owned entries of t1, lam, p,
  // r); the coarse correction and alpha (one thread per column); the owned
  // updates and the u = D_S r' entries of both sides of every owned
  // multiplier
  V sv[CT];
#pragma unroll
  for (int cc = 0; cc < CT; ++cc) sv[cc] = (cc < nrhs && tid < G) ? (V)X.pW[(int64_t)tid * CT + cc] : (V)0;
  const bool own0 = tid < nl;
  V ta[CT], tb[CT], xo[CT], po[CT], ro[CT];
  if (own0) {
    const int4 a0 = SL.gs[tid];
    const int2 n0 = SL.gn[tid];
#pragma unroll
    for (int col = 0; col < CT; ++col) {
      if (col >= nrhs) break;
      const int64_t o = l0 + tid + m * col;
      ta[col] = (V)A.t1[(int64_t)a0.x * nrhs + a0.y + (int64_t)n0.x * col];
      tb[col] = (V)A.t1[(int64_t)a0.z * nrhs + a0.w + (int64_t)n0.y * col];
      xo[col] = xv[o];
      po[col] = pc[o];
      ro[col] = rc[o];
    }
  }
  if (ngp > 0 && A.cache_coarse && nrhs == 1) {
    // contributor values of G^T p in parallel (one round with the loads above)
    for (int64_t e = tid; e < A.ncontrib; e += NCONS) {
      const int4 pc4 = X.c_pc[e];
      X.c_cv[e] = (V)A.qpart[(int64_t)pc4.x + pc4.y];
    }
  }
#pragma unroll
  for (int cc = 0; cc < CT; ++cc)
    if (cc < nrhs) cons_sum_begin(sv[cc], nwG, X.redA + 8 * cc);
  cons_sync();
  gate_open();
  V* qg = X.qg;
  V* yc = X.yc;
  const int warp = tid / 32, lane = tid % 32;
  constexpr int NWC = NCONS / 32;
  // the coarse step and the scalars are spread over warps and lanes with
  // shuffle sums: serial chains of shared loads are slow while the bulk copies
  // of the next pass write shared memory
  if (ngp > 0) {
    // qg = G^T p from the contributors: one warp per coarse DOF and column
    for (int t = warp; t < ngp * nrhs; t += NWC) {
      const int g = t % ngp, col = t / ngp;
      V acc = 0;
      if (A.cache_coarse && nrhs == 1) {
        for (int e = X.c_co[g] + lane; e < X.c_co[g + 1]; e += 32) acc += X.c_cv[e];
      } else {
        for (int64_t e = A.pcsr_off[g] + lane; e < A.pcsr_off[g + 1]; e += 32) {
          const int4 pc4 = A.cache_coarse ? X.c_pc[e] : A.pcon[e];
          acc += (V)A.qpart[(int64_t)pc4.x * nrhs + pc4.y + (int64_t)pc4.z * col];
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) qg[t] = acc;
    }
    cons_sync();
    // yc = S_Pi^-1 qg: one warp per row and column
    for (int t = warp; t < ngp * nrhs; t += NWC) {
      const int g = t % ngp, col = t / ngp;
      V acc = 0;
      if (A.cache_coarse) {
        const V* sp = X.c_spi + (size_t)ngp * g;
        for (int h = lane; h < ngp; h += 32) acc += sp[h] * qg[h + ngp * col];
      } else {
        const double* sp = A.SPiInv + (int64_t)A.ldc * g;
        for (int h = lane; h < ngp; h += 32) acc += (V)sp[h] * qg[h + ngp * col];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) yc[t] = acc;
    }
    cons_sync();
  }
  // alpha of column cc (warp cc): <p, F p> = sum of the shares + (G^T p) . S_Pi^-1 (G^T p)
  for (int cc = warp; cc < nrhs; cc += NWC) {
    V v = lane < nwG ? X.redA[8 * cc + lane] : (V)0;
    for (int g = lane; g < ngp; g += 32) v += qg[g + ngp * cc] * yc[g + ngp * cc];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) X.alpha_s[cc] = (X.done[cc] || v == (V)0) ? (V)0 : X.rz[cc] / v;
  }
  cons_sync();
  V rrp[CT];
#pragma unroll
  for (int cc = 0; cc < CT; ++cc) rrp[cc] = 0;
  T* u = (T*)A.CW.uall;
  for (int64_t i = tid; i < nl; i += NCONS) {
    const bool first = i == tid;
    const int64_t l = l0 + i;
    const int4 a = SL.gs[i];
    const int2 nn = SL.gn[i];
    const int2 gu = SL.gu[i];
    V w0, w1;   // D_S at both sides: sign times rho-scaling
    if (SL.sg) {
      const Vec2<V> sg = SL.sg[i], sc = SL.sc[i];
      w0 = sg.x * sc.x;
      w1 = sg.y * sc.y;
    } else {
      w0 = (V)(A.I_sign[a.x + a.y] * A.I_scale[a.x + a.y]);
      w1 = (V)(A.I_sign[a.z + a.w] * A.I_scale[a.z + a.w]);
    }
#pragma unroll
    for (int col = 0; col < CT; ++col) {
      if (col >= nrhs) break;
      const int64_t o = l + m * col;
      const V al = X.alpha_s[col];
      V v = (first ? ta[col] : (V)A.t1[(int64_t)a.x * nrhs + a.y + (int64_t)nn.x * col]) -
            (first ? tb[col] : (V)A.t1[(int64_t)a.z * nrhs + a.w + (int64_t)nn.y * col]);
      if (ngp > 0) {
        if (SL.gv) {
#pragma unroll 8
          for (int e = 0; e < E; ++e) v += SL.gv[e * estride + i] * yc[SL.gi[e * estride + i] + ngp * col];
        } else {
          for (int e = 0; e < E; ++e) v += (V)SL.gv64[e * estride + i] * yc[SL.gi[e * estride + i] + ngp * col];
        }
      }
      xv[o] = fma(al, first ? po[col] : pc[o], first ? xo[col] : xv[o]);
      const V rv = fma(-al, v, first ? ro[col] : rc[o]);
      rn[o] = rv;
      rrp[col] += rv * rv;
      u[col * A.CW.utot + gu.x] = (T)(w0 * rv);
      u[col * A.CW.utot + gu.y] = (T)(w1 * rv);
    }
  }
  fence_async_global();   // the S pass reads u with bulk copies after the barrier
#pragma unroll
  for (int cc = 0; cc < CT; ++cc)
    if (cc < nrhs) cons_sum_begin(rrp[cc], nwL, X.redB + 8 * cc);
  cons_sync();
  if (tid < nrhs) {
    // a CTA whose bulk-copy wait timed out poisons its share, so that every
    // CTA sees the same non-finite <r', r'> and leaves the loop with it
    const double share = (double)cons_sum_end(nwL, X.redB + 8 * tid);
    X.pR[(int64_t)bid * CT + tid] = *(volatile int*)A.err ? __longlong_as_double(0x7ff8000000000000ll) : share;
  }
}

template <typename T, int CT>
__device__ __noinline__ void pcg_phase4(const PcgStreamArgs& A, const PhaseCtx<T, CT>& X, T* pc, T* pn) {
  using V = T;
  const int tid = threadIdx.x;
  const Slice<V>& SL = X.SL;
  const int64_t l0 = X.l0, nl = X.nl, m = X.m;
  const int nrhs = X.nrhs, G = X.G, bid = X.bid, nwG = X.nwG;
  // ---- P4 (consumers): one round of loads (the shares of <r', r'> and
  // <r', z'>, the owned entries of t2 and p); convergence test and beta
  // (one thread per column); owned p' and the u = D_W p' entries
  V sr[CT], sz[CT];
#pragma unroll
  for (int cc = 0; cc < CT; ++cc) {
    sr[cc] = (cc < nrhs && tid < G) ? (V)X.pR[(int64_t)tid * CT + cc] : (V)0;
    sz[cc] = (cc < nrhs && tid < G) ? (V)X.pZ[(int64_t)tid * CT + cc] : (V)0;
  }
  const bool own0 = tid < nl;
  V zt[CT], po[CT];
  if (own0) {
    const int4 a0 = SL.gs[tid];
    const int2 n0 = SL.gn[tid];
    V s0, s1;
    if (SL.sc) {
      const Vec2<V> sc = SL.sc[tid];
      s0 = sc.x;
      s1 = sc.y;
    } else {
      s0 = (V)A.I_scale[a0.x + a0.y];
      s1 = (V)A.I_scale[a0.z + a0.w];
    }
#pragma unroll
    for (int col = 0; col < CT; ++col) {
      if (col >= nrhs) break;
      const int64_t o = l0 + tid + m * col;
      zt[col] = zgather(s0, (V)A.t2[(int64_t)a0.x * nrhs + a0.y + (int64_t)n0.x * col], s1,
                        (V)A.t2[(int64_t)a0.z * nrhs + a0.w + (int64_t)n0.y * col]);
      po[col] = pc[o];
    }
  }
#pragma unroll
  for (int cc = 0; cc < CT; ++cc)
    if (cc < nrhs) {
      cons_sum_begin(sr[cc], nwG, X.redA + 8 * cc);
      cons_sum_begin(sz[cc], nwG, X.redB + 8 * cc);
    }
  cons_sync();
  gate_open();
  const int warp = tid / 32, lane = tid % 32;
  for (int cc = warp; cc < nrhs; cc += NCONS / 32) {
    // column cc on warp cc: the warp sums of the shares, then lane 0
    V rr = lane < nwG ? X.redA[8 * cc + lane] : (V)0, rzn = lane < nwG ? X.redB[8 * cc + lane] : (V)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rr += __shfl_xor_sync(0xffffffffu, rr, o);
      rzn += __shfl_xor_sync(0xffffffffu, rzn, o);
    }
    if (lane != 0) continue;
    const bool was = X.done[cc] != 0;
    // a non-finite residual (a timed-out wait somewhere, see P2) ends the loop
    const bool now = was || (double)rr <= A.tol2 * (double)X.bb[cc] || !isfinite(rr);
    const V b = (now || X.rz[cc] == (V)0) ? (V)0 : rzn / X.rz[cc];
    X.beta_s[cc] = b;
    if (!was) {
      ++X.itc[cc];
      if (bid == 0) {   // stores only: a read here would hold CTA 0 up by an L2 round trip
        A.scal[PS_SC * cc + 2] = (double)rr * X.s2[cc];
        A.scal[PS_SC * cc + 4] = (double)X.alpha_s[cc];
        A.scal[PS_SC * cc + 8] = (double)X.itc[cc];
      }
      X.done[cc] = now ? 1 : 0;
      if (!now) {
        X.rz[cc] = rzn;
        if (bid == 0) {
          A.scal[PS_SC * cc + 0] = (double)rzn * X.s2[cc];
          A.scal[PS_SC * cc + 5] = (double)b;
        }
      }
    }
    if (cc == 0) {
      ++*X.its;
      if (bid == 0 && A.hist && *X.its <= A.hist_cap) {
        A.hist[2 * (*X.its - 1)] = (double)X.alpha_s[0];
        A.hist[2 * (*X.its - 1) + 1] = (double)b;
      }
    }
  }
  cons_sync();
  T* u = (T*)A.CW.uall;
  for (int64_t i = tid; i < nl; i += NCONS) {
    const bool first = i == tid;
    const int64_t l = l0 + i;
    const int2 gu = SL.gu[i];
    V w0, w1;   // D_W at both sides: the signs
    if (SL.sg) {
      const Vec2<V> sg = SL.sg[i];
      w0 = sg.x;
      w1 = sg.y;
    } else {
      const int4 a = SL.gs[i];
      w0 = (V)A.I_sign[a.x + a.y];
      w1 = (V)A.I_sign[a.z + a.w];
    }
    V zr[CT];
    if (!first) {
      const int4 a = SL.gs[i];
      const int2 nn = SL.gn[i];
      V s0, s1;
      if (SL.sc) {
        const Vec2<V> sc = SL.sc[i];
        s0 = sc.x;
        s1 = sc.y;
      } else {
        s0 = (V)A.I_scale[a.x + a.y];
        s1 = (V)A.I_scale[a.z + a.w];
      }
#pragma unroll
      for (int col = 0; col < CT; ++col) {
        if (col >= nrhs) break;
        zr[col] = zgather(s0, (V)A.t2[(int64_t)a.x * nrhs + a.y + (int64_t)nn.x * col], s1,
                          (V)A.t2[(int64_t)a.z * nrhs + a.w + (int64_t)nn.y * col]);
      }
    }
#pragma unroll
    for (int col = 0; col < CT; ++col) {
      if (col >= nrhs) break;
      const int64_t o = l + m * col;
      const V pv = fma(X.beta_s[col], first ? po[col] : pc[o], first ? zt[col] : zr[col]);
      pn[o] = pv;
      u[col * A.CW.utot + gu.x] = (T)(w0 * pv);
      u[col * A.CW.utot + gu.y] = (T)(w1 * pv);
    }
  }
  fence_async_global();   // the W pass reads u with bulk copies after the barrier
}

template <typename T, int CT, bool ROWS>
__global__ void __launch_bounds__(STREAM_THREADS, 1) k_pcg_stream(PcgStreamArgs A) {
  using V = T;   // vectors and scalars in the operators' precision
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double dred[8 * CT];
  __shared__ V redA[8 * CT], redB[8 * CT];
  __shared__ V qg[PS_MAXGP * CT], yc[PS_MAXGP * CT];
  __shared__ V rz[CT], bb[CT], alpha_s[CT], beta_s[CT];
  __shared__ double s2[CT];
  __shared__ int done[CT];
  __shared__ int its, itc[CT];
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
  Vec2<V>* c_sg = reinterpret_cast<Vec2<V>*>(c_gu + nl);
  Vec2<V>* c_sc = c_sg + nl;
  V* c_gv = reinterpret_cast<V*>(c_sc + nl);
  int32_t* c_gi = reinterpret_cast<int32_t*>(c_gv + (size_t)E * nl);
  unsigned char* cend = A.cache_slice ? reinterpret_cast<unsigned char*>(c_gi + (size_t)E * nl) : cbase;
  cend = reinterpret_cast<unsigned char*>(((uintptr_t)cend + 15) / 16 * 16);
  V* c_spi = reinterpret_cast<V*>(cend);   // each coarse buffer starts on 16 bytes
  V* c_cv = reinterpret_cast<V*>(cend + round16((size_t)ngp * ngp * sizeof(V)));
  int32_t* c_co =
      reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(c_cv) + round16((size_t)A.ncontrib * sizeof(V)));
  int4* c_pc = reinterpret_cast<int4*>(reinterpret_cast<unsigned char*>(c_co) + round16((size_t)(ngp + 1) * 4));
  if (A.cache_slice) {
    for (int64_t i = tid; i < nl; i += blockDim.x) {
      const int64_t l = l0 + i;
      const int4 a = A.gs[l];
      c_gs[i] = a;
      c_gn[i] = A.gn[l];
      c_gu[i] = A.gu[l];
      c_sg[i] = {(V)A.I_sign[a.x + a.y], (V)A.I_sign[a.z + a.w]};
      c_sc[i] = {(V)A.I_scale[a.x + a.y], (V)A.I_scale[a.z + a.w]};
      for (int e = 0; e < E; ++e) {
        c_gv[(size_t)e * nl + i] = (V)A.gv[e * m + l];
        c_gi[(size_t)e * nl + i] = A.gi[e * m + l];
      }
    }
  }
  if (A.cache_coarse) {
    for (int t = tid; t < ngp * ngp; t += blockDim.x) c_spi[t] = (V)A.SPiInv[(int64_t)A.ldc * (t / ngp) + t % ngp];
    for (int g = tid; g <= ngp; g += blockDim.x) c_co[g] = (int32_t)A.pcsr_off[g];
    for (int64_t e = tid; e < A.ncontrib; e += blockDim.x) c_pc[e] = A.pcon[e];
  }
  Slice<V> SL;
  SL.l0 = l0;
  SL.nl = nl;
  if (A.cache_slice) {
    SL.gs = c_gs; SL.gn = c_gn; SL.gu = c_gu; SL.sg = c_sg; SL.sc = c_sc; SL.gv = c_gv; SL.gv64 = nullptr;
    SL.gi = c_gi;
  } else {
    SL.gs = A.gs + l0; SL.gn = A.gn + l0; SL.gu = A.gu + l0; SL.sg = nullptr; SL.sc = nullptr;
    SL.gv = nullptr; SL.gv64 = A.gv + l0; SL.gi = A.gi + l0;
  }
  const int64_t estride = A.cache_slice ? nl : m;
  __syncthreads();
  if (tid < CT) {
    // normalised vectors: <r, z> and ||b||^2 in units of ||b||^2
    const double b2 = tid < nrhs ? A.scal[PS_SC * tid + 3] : 1.0;
    s2[tid] = (A.vscaled && b2 > 0.0) ? b2 : 1.0;
    rz[tid] = tid < nrhs ? (V)(A.scal[PS_SC * tid + 0] / s2[tid]) : (V)0;
    bb[tid] = (V)(b2 / s2[tid]);
    done[tid] = tid < nrhs ? (A.scal[PS_SC * tid + 7] != 0.0) : 1;
    itc[tid] = tid < nrhs ? (int)A.scal[PS_SC * tid + 8] : 0;
  }
  if (tid == 0) its = (int)A.scal[8];
  uint32_t seq = 0, useq = 0;
  const bool producer = tid >= NCONS;
  int npreW = 0, npreS = 0;   // tiles of the next W / S pass already in flight (producer warp)
  double* pW = A.part;                          // shares of <p, B t1>
  double* pR = A.part + (int64_t)G * CT;        // shares of <r', r'>
  double* pZ = A.part + 2 * (int64_t)G * CT;    // shares of <r', z'>
  V* rb[2] = {static_cast<V*>(A.r), static_cast<V*>(A.q)};
  V* pb[2] = {static_cast<V*>(A.p), static_cast<V*>(A.z)};
  int cur = 0;
  const int2 krW = A.ckrW[bid];
  // u = D_W p for the first product; the first W tiles are fetched meanwhile
  if (producer) npreW = stream_prefetch<T>(A.CW, A.ctaW[bid], A.ctaW[bid + 1], smem, seq, CT);
  write_u_run<T, CT, V>(A, krW, pb[0], nullptr, nullptr, nullptr, false);
  __syncthreads();   // every thread's u stores and fence precede the bulk copies
  const int nwG = (G + 31) / 32;                       // warps holding per-CTA shares
  const int nwL = (int)((std::min<int64_t>(nl, NCONS) + 31) / 32);   // warps holding owned entries
  PhaseCtx<V, CT> X;
  X.SL = SL;
  X.l0 = l0;
  X.nl = nl;
  X.estride = estride;
  X.m = m;
  X.E = E;
  X.ngp = ngp;
  X.nrhs = nrhs;
  X.G = G;
  X.bid = bid;
  X.nwG = nwG;
  X.nwL = nwL;
  X.c_spi = c_spi;
  X.c_cv = c_cv;
  X.c_co = c_co;
  X.c_pc = c_pc;
  X.qg = qg;
  X.yc = yc;
  X.redA = redA;
  X.redB = redB;
  X.rz = rz;
  X.bb = bb;
  X.alpha_s = alpha_s;
  X.beta_s = beta_s;
  X.s2 = s2;
  X.done = done;
  X.its = &its;
  X.itc = itc;
  X.pW = pW;
  X.pR = pR;
  X.pZ = pZ;
  for (int iter = 0; iter < A.maxit; ++iter) {
    bool all = true;
    for (int cc = 0; cc < nrhs; ++cc) all &= done[cc] != 0;
    if (all) break;
    V* rc = rb[cur];
    V* rn = rb[cur ^ 1];
    V* pc = pb[cur];
    V* pn = pb[cur ^ 1];
    // ---- P1: local products with W, the primal partials, share of <p, B t1>
    stream_tiles<T, CT, ROWS, true>(A.CW, A.ctaW[bid], A.ctaW[bid + 1], smem, seq, useq, A.t1, A.qpart, nrhs, 0,
                                    nrhs, npreW, pW + (int64_t)bid * CT, dred);
    npreW = 0;
    grid.sync();
    if (producer) {
      // the first S tiles are fetched while the consumers run the vector phase
      gate_wait();
      npreS = stream_prefetch<T>(A.CS, A.ctaS[bid], A.ctaS[bid + 1], smem, seq, CT);
    } else {
      pcg_phase2<T, CT>(A, X, rc, rn, pc);
    }
    grid.sync();
    // ---- P3: local products with S, share of <r', z'>
    stream_tiles<T, CT, ROWS, true>(A.CS, A.ctaS[bid], A.ctaS[bid + 1], smem, seq, useq, A.t2, nullptr, nrhs, 0,
                                    nrhs, npreS, pZ + (int64_t)bid * CT, dred);
    npreS = 0;
    grid.sync();
    if (producer) {
      gate_wait();
      npreW = stream_prefetch<T>(A.CW, A.ctaW[bid], A.ctaW[bid + 1], smem, seq, CT);
    } else {
      pcg_phase4<T, CT>(A, X, pc, pn);
    }
    grid.sync();   // every CTA's u entries (and the done flags) before the next W pass
    cur ^= 1;
  }
  // tiles fetched ahead for a pass that will not run
  if (producer) stream_drain(smem, seq, npreW + npreS, A.CW.stages);
  if (bid == 0 && tid < nrhs) A.scal[PS_SC * tid + 7] = done[tid] ? 1.0 : 0.0;
}

// FP32 copies of lam, r and p, each column divided by ||b|| (||b||^2 is
// scalar 3 of the column), and the way back for lam
__global__ void k_vec_to_f32(const double* lam, const double* r, const double* p, const double* scal, int64_t m,
                             float* xf, float* rf, float* pf) {
  const int col = blockIdx.y;
  const double b2 = scal[PS_SC * col + 3];
  const double is = b2 > 0.0 ? 1.0 / sqrt(b2) : 1.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = i + m * col;
    xf[o] = (float)(lam[o] * is);
    rf[o] = (float)(r[o] * is);
    pf[o] = (float)(p[o] * is);
  }
}
__global__ void k_vec_from_f32(const float* xf, const double* scal, int64_t m, double* lam) {
  const int col = blockIdx.y;
  const double b2 = scal[PS_SC * col + 3];
  const double sc = b2 > 0.0 ? sqrt(b2) : 1.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = i + m * col;
    lam[o] = (double)xf[o] * sc;
  }
}

template <typename T, int CT, bool ROWS>
ieti_status launch_pcg_stream(Ctx* c, PcgStreamArgs A, int stages_max, size_t ubytes, cudaStream_t st) {
  auto kern = k_pcg_stream<T, CT, ROWS>;
  cudaFuncAttributes fa;
  IETI_CUDA_TRY(c, cudaFuncGetAttributes(&fa, kern));
  const StreamPlan& PW = ROWS ? c->rplan[sizeof(T) == 4][1] : c->splan[sizeof(T) == 4][1];
  const StreamPlan& PS = ROWS ? c->rplan[sizeof(T) == 4][0] : c->splan[sizeof(T) == 4][0];
  const int stage_bytes = std::max(PW.stage_bytes, PS.stage_bytes);
  // caches: the slice metadata if it takes at most 40 KB, the coarse data if
  // n_gp <= 64
  const int64_t nlmax = ceil_div(A.m, PW.grid) + 1;
  A.cache_slice = slice_bytes(nlmax, A.E, sizeof(T)) <= 40 * 1024;
  A.cache_coarse = A.ngp > 0 && A.ngp <= 64;
  const size_t cache = (A.cache_slice ? (slice_bytes(nlmax, A.E, sizeof(T)) + 15) / 16 * 16 : 0) +
                       (A.cache_coarse ? coarse_bytes(A.ngp, A.ncontrib, sizeof(T)) : 0);
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
  const bool rows = nrhs == 1 && c->max_ldI <= ROW_MAX_ELEMS && c->rplan[fp32][0].built && c->rplan[fp32][1].built;
  const StreamPlan& PW = rows ? c->rplan[fp32][1] : c->splan[fp32][1];
  const StreamPlan& PS = rows ? c->rplan[fp32][0] : c->splan[fp32][0];
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
  A.CW.l2_hint = 1;   // W stays in L2 across iterations
  A.CS = A.CW;
  A.CS.l2_hint = 2;   // S streams through
  A.CS.M = c->S;
  A.CS.tiles = (const LTile*)PS.d_tiles;
  A.ctaW = PW.d_cta;
  A.ctaS = PS.d_cta;
  A.ckrW = PW.d_ckr;
  A.ckrS = PS.d_ckr;
  A.sd = c->d_sd;
  A.uoff = c->d_uoff;
  A.I_dual = c->d_I_dual;
  const int64_t mn = c->m_r * nrhs;
  float* xf = c->wvf;   // FP32 vectors: lam, r, second r, p, second p
  if (fp32) {
    A.x = xf;
    A.r = xf + mn;
    A.q = xf + 2 * mn;
    A.p = xf + 3 * mn;
    A.z = xf + 4 * mn;
    A.vscaled = 1;
  } else {
    A.x = lam;
    A.r = r;
    A.z = z;
    A.p = p;
    A.q = q;
    A.vscaled = 0;
  }
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
  const size_t ub1 = ((size_t)c->max_ldI * (fp32 ? 4 : 8) + 127) / 128 * 128;
  const dim3 vg((unsigned)std::min<int64_t>(ceil_div(c->m_r, 256), 1024), nrhs);
  if (fp32) {
    k_vec_to_f32<<<vg, 256, 0, st>>>(lam, r, p, c->wscal, c->m_r, xf, xf + mn, xf + 3 * mn);
    IETI_LAUNCH_CHECK(c);
  }
  ieti_status res;
  if (nrhs == 1) {
    if (fp32)
      res = rows ? launch_pcg_stream<float, 1, true>(c, A, MAX_STAGES, ub1, st)
                 : launch_pcg_stream<float, 1, false>(c, A, MAX_STAGES, ub1, st);
    else
      res = rows ? launch_pcg_stream<double, 1, true>(c, A, MAX_STAGES, ub1, st)
                 : launch_pcg_stream<double, 1, false>(c, A, MAX_STAGES, ub1, st);
  } else {
    res = fp32 ? launch_pcg_stream<float, 8, false>(c, A, MAX_STAGES, ub1 * 8, st)
               : launch_pcg_stream<double, 8, false>(c, A, MAX_STAGES, ub1 * 8, st);
  }
  if (res == IETI_OK && fp32) {
    k_vec_from_f32<<<vg, 256, 0, st>>>(xf, c->wscal, c->m_r, lam);
    IETI_LAUNCH_CHECK(c);
  }
  return res;
}

}  // namespace ieti
