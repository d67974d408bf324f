// Persistent (cooperative) PCG with per-item local products: the PCG loop when
// the streamed products do not apply (for example a coarse space too large
// for the per-CTA caches of the streamed form).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace cg = cooperative_groups;

namespace ieti {

// ---------------------------------------------------------------------------
// k_pcg_coop: the PCG iteration on F_DP lam = b with the Dirichlet
// preconditioner (Eqs. (7), (10)) as one persistent launch. Per iteration:
//   A  t1_k = W_k B_k^T p,  q_k = Phi_I^(k)T B_k^T p            | grid barrier
//   B  yc = S_Pi^-1 sum C^T q_k (every CTA), q = B (t1 + Phi_I C yc), <p,q> partials
//   C  alpha = rz / <p,q>;  lam += alpha p;  r -= alpha q; <r,r> partials
//   D  convergence test; t2_k = S_k D_k B_k^T r                  | grid barrier
//   E  z = sum_k B_k D_k t2_k; <r,z> partials                    | grid barrier
//   F  beta = rz_new / rz;  p = z + beta p                        | grid barrier
// Every CTA reduces the same per-CTA partials in the same order, so every CTA
// takes the same alpha, beta and convergence decisions.
// ---------------------------------------------------------------------------

struct PcgArgs {
  const SubDev* sd;
  int nsub, nrhs, ngp, ldc, maxit, hist_cap;
  int64_t m;
  const void* W;
  const void* S;
  const int32_t* I_dual;
  const double* I_sign;
  const double* I_scale;
  const int32_t* pair;
  const double* Phi;
  const int32_t* P_glob;
  const int64_t* pcsr_off;
  const int2* pcsr;
  const double* SPiInv;
  double *x, *r, *z, *p, *q;
  double *t1, *t2, *qpart;
  double *part_pq, *part_rr, *part_rz;
  double* scal;     // per column (stride 16): 0 rz, 2 rr, 3 bb, 4 alpha, 5 beta, 7 done, 8 its
  double* hist;
  double tol2;
  int total_items;
  int u_ld;         // rows of the staged u (>= every ldI)
};

constexpr int PC_ROWS = 16;    // rows of a local block per work item
constexpr int PCG_COOP_MAX_GRID = 1024;
constexpr int PC_SC = 16;

// CTA sum in a fixed order: butterfly within each warp (lane 0's value), then
// the warp sums in warp order; every thread returns the same value
__device__ inline double cta_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  __syncthreads();   // red is free
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0;
  for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
  return s;
}

// sum of the per-CTA partials of one column: thread-strided sums, then a fixed
// tree, so every CTA obtains the bitwise same value
__device__ inline double sum_part(const double* part, int col, double* red) {
  double v = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += part[i + gridDim.x * col];
  return cta_sum(v, red);
}

// local products of one work item: rows [r0, r0 + PC_ROWS) of M_k times u_k
template <typename T, int CT>
__device__ void pc_local(const PcgArgs& A, const T* M, const double* src, bool scaled, double* out, int k, int chunk,
                         T* u, bool gather) {
  const SubDev s = A.sd[k];
  const int nI = s.nI;
  __syncthreads();
  for (int i = threadIdx.x; gather && i < s.ldI; i += blockDim.x) {
    if (i < nI) {
      const double w = A.I_sign[s.iv + i] * (scaled ? A.I_scale[s.iv + i] : 1.0);
      const int l = A.I_dual[s.iv + i];
#pragma unroll
      for (int cc = 0; cc < CT; ++cc) u[i * CT + cc] = (cc < A.nrhs) ? (T)(w * src[l + A.m * cc]) : (T)0;
    } else {
#pragma unroll
      for (int cc = 0; cc < CT; ++cc) u[i * CT + cc] = (T)0;
    }
  }
  __syncthreads();
  constexpr int VEC = 16 / sizeof(T);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const T* Mk = M + s.S;
  const int nv = s.ldI / VEC;
  for (int rr = warp; rr < PC_ROWS; rr += 8) {
    const int i = chunk * PC_ROWS + rr;
    if (i >= nI) break;
    const T* row = Mk + (int64_t)s.ldI * i;
    T acc[CT];
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) acc[cc] = 0;
#pragma unroll 4
    for (int jv = lane; jv < nv; jv += 32) {
      T mv[VEC];
      if constexpr (VEC == 4) {
        float4 qv = reinterpret_cast<const float4*>(row)[jv];
        mv[0] = qv.x; mv[1] = qv.y; mv[2] = qv.z; mv[3] = qv.w;
      } else {
        double2 qv = reinterpret_cast<const double2*>(row)[jv];
        mv[0] = qv.x; mv[1] = qv.y;
      }
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const T* uj = u + (jv * VEC + e) * CT;
#pragma unroll
        for (int cc = 0; cc < CT; ++cc) acc[cc] += mv[e] * uj[cc];
      }
    }
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) {
      T v = acc[cc];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && cc < A.nrhs) out[IV(s, i, cc, A.nrhs)] = (double)v;
    }
  }
}

template <typename T, int CT>
__global__ void __launch_bounds__(256) k_pcg_coop(PcgArgs A) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char dyn[];
  T* u = reinterpret_cast<T*>(dyn);                                        // u_ld x CT
  double* yc = reinterpret_cast<double*>(dyn + sizeof(T) * A.u_ld * CT);   // ngp x CT
  __shared__ double red[256];
  __shared__ double rz[CT], bb[CT], alpha[CT], beta[CT];
  __shared__ int done[CT];
  __shared__ int its;
  const int tid = threadIdx.x;
  if (tid < CT) {
    rz[tid] = (tid < A.nrhs) ? A.scal[PC_SC * tid + 0] : 0.0;
    bb[tid] = (tid < A.nrhs) ? A.scal[PC_SC * tid + 3] : 1.0;
    done[tid] = (tid < A.nrhs) ? (A.scal[PC_SC * tid + 7] != 0.0) : 1;
  }
  if (tid == 0) its = (int)A.scal[8];
  __syncthreads();
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + tid;
  for (int iter = 0; iter < A.maxit; ++iter) {
    bool all = true;
    for (int cc = 0; cc < A.nrhs; ++cc) all &= done[cc] != 0;
    if (all) break;
    // ---- A: local products with W and primal partials. Each CTA takes a
    // contiguous run of items (ordered by subdomain) and stages u_k once per
    // subdomain of the run.
    const int per = (A.total_items + (int)gridDim.x - 1) / (int)gridDim.x;
    const int ibeg = blockIdx.x * per, iend = min(A.total_items, ibeg + per);
    int k0 = 0, base0 = 0;
    while (k0 < A.nsub && ibeg >= base0 + (A.sd[k0].nI + PC_ROWS - 1) / PC_ROWS) {
      base0 += (A.sd[k0].nI + PC_ROWS - 1) / PC_ROWS;
      ++k0;
    }
    for (int item = ibeg, k = k0, base = base0, lastk = -1; item < iend; ++item) {
      while (item >= base + (A.sd[k].nI + PC_ROWS - 1) / PC_ROWS) {
        base += (A.sd[k].nI + PC_ROWS - 1) / PC_ROWS;
        ++k;
      }
      const int chunk = item - base;
      pc_local<T, CT>(A, (const T*)A.W, A.p, false, A.t1, k, chunk, u, k != lastk);
      lastk = k;
      if (chunk == 0) {
        const SubDev s = A.sd[k];
        const int warp = tid / 32, lane = tid % 32;
        for (int t = warp; t < s.nP * A.nrhs; t += 8) {
          const int c = t % s.nP, col = t / s.nP;
          const double* ph = A.Phi + s.Kp + s.nVp + (int64_t)s.n * c;
          double acc = 0;
          for (int i = lane; i < s.nI; i += 32) acc += ph[i] * A.I_sign[s.iv + i] * A.p[A.I_dual[s.iv + i] + A.m * col];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == 0) A.qpart[PV(s, c, col, A.nrhs)] = acc;
        }
      }
    }
    grid.sync();
    // ---- B: coarse correction (every CTA), q = F p, partial <p, q>
    if (A.ngp > 0) {
      double* qg = yc;   // reuse: gather, then overwrite with the product
      __syncthreads();
      for (int t = tid; t < A.ngp * A.nrhs; t += blockDim.x) {
        const int g = t % A.ngp, col = t / A.ngp;
        double acc = 0;
        for (int64_t e = A.pcsr_off[g]; e < A.pcsr_off[g + 1]; ++e) {
          const int2 kc = A.pcsr[e];
          acc += A.qpart[PV(A.sd[kc.x], kc.y, col, A.nrhs)];
        }
        qg[A.ngp * CT + t] = acc;   // gathered q after the product slots
      }
      __syncthreads();
      for (int t = tid; t < A.ngp * A.nrhs; t += blockDim.x) {
        const int g = t % A.ngp, col = t / A.ngp;
        double acc = 0;
        for (int h = 0; h < A.ngp; ++h) acc += A.SPiInv[h + (int64_t)A.ldc * g] * qg[A.ngp * CT + h + A.ngp * col];
        yc[t] = acc;
      }
      __syncthreads();
    }
    double mypq[CT];
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) mypq[cc] = 0;
    for (int64_t l = g0; l < A.m; l += gstride) {
      for (int col = 0; col < A.nrhs; ++col) {
        double v = 0;
        for (int side = 0; side < 2; ++side) {
          const int k = A.pair[l * 4 + 2 * side], i = A.pair[l * 4 + 2 * side + 1];
          const SubDev s = A.sd[k];
          double w = A.t1[IV(s, i, col, A.nrhs)];
          if (A.ngp > 0) {
            const double* ph = A.Phi + s.Kp + s.nVp + i;
            for (int c = 0; c < s.nP; ++c) w += ph[(int64_t)s.n * c] * yc[A.P_glob[s.pv + c] + A.ngp * col];
          }
          v += (side == 0) ? w : -w;
        }
        A.q[l + A.m * col] = v;
        mypq[col] += v * A.p[l + A.m * col];
      }
    }
    for (int cc = 0; cc < A.nrhs; ++cc) {
      const double s = cta_sum(mypq[cc], red);
      if (tid == 0) A.part_pq[blockIdx.x + gridDim.x * cc] = s;
    }
    grid.sync();
    // ---- C: alpha, x and r updates, partial <r, r>
    for (int cc = 0; cc < A.nrhs; ++cc) {
      const double pq = sum_part(A.part_pq, cc, red);
      if (tid == 0) alpha[cc] = (done[cc] || pq == 0.0) ? 0.0 : rz[cc] / pq;
    }
    __syncthreads();
    double myrr[CT];
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) myrr[cc] = 0;
    for (int64_t l = g0; l < A.m; l += gstride) {
      for (int col = 0; col < A.nrhs; ++col) {
        const int64_t o = l + A.m * col;
        double rv = A.r[o];
        if (!done[col]) {
          A.x[o] += alpha[col] * A.p[o];
          rv -= alpha[col] * A.q[o];
          A.r[o] = rv;
        }
        myrr[col] += rv * rv;
      }
    }
    for (int cc = 0; cc < A.nrhs; ++cc) {
      const double s = cta_sum(myrr[cc], red);
      if (tid == 0) A.part_rr[blockIdx.x + gridDim.x * cc] = s;
    }
    grid.sync();
    // ---- D: convergence test, local products with S
    for (int cc = 0; cc < A.nrhs; ++cc) {
      const double rr = sum_part(A.part_rr, cc, red);
      if (tid == 0 && !done[cc]) {
        if (blockIdx.x == 0) {
          A.scal[PC_SC * cc + 2] = rr;
          A.scal[PC_SC * cc + 4] = alpha[cc];
          A.scal[PC_SC * cc + 8] += 1.0;
        }
        if (rr <= A.tol2 * bb[cc]) done[cc] = 1;
      }
    }
    if (tid == 0) {
      ++its;
      if (blockIdx.x == 0 && A.hist && its <= A.hist_cap) A.hist[2 * (its - 1)] = alpha[0];
    }
    __syncthreads();
    for (int item = ibeg, k = k0, base = base0, lastk = -1; item < iend; ++item) {
      while (item >= base + (A.sd[k].nI + PC_ROWS - 1) / PC_ROWS) {
        base += (A.sd[k].nI + PC_ROWS - 1) / PC_ROWS;
        ++k;
      }
      pc_local<T, CT>(A, (const T*)A.S, A.r, true, A.t2, k, item - base, u, k != lastk);
      lastk = k;
    }
    grid.sync();
    // ---- E: z = preconditioned r, partial <r, z>
    double myrz[CT];
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) myrz[cc] = 0;
    for (int64_t l = g0; l < A.m; l += gstride) {
      for (int col = 0; col < A.nrhs; ++col) {
        double v = 0;
        for (int side = 0; side < 2; ++side) {
          const int k = A.pair[l * 4 + 2 * side], i = A.pair[l * 4 + 2 * side + 1];
          const SubDev s = A.sd[k];
          const double w = A.I_scale[s.iv + i] * A.t2[IV(s, i, col, A.nrhs)];
          v += (side == 0) ? w : -w;
        }
        A.z[l + A.m * col] = v;
        myrz[col] += v * A.r[l + A.m * col];
      }
    }
    for (int cc = 0; cc < A.nrhs; ++cc) {
      const double s = cta_sum(myrz[cc], red);
      if (tid == 0) A.part_rz[blockIdx.x + gridDim.x * cc] = s;
    }
    grid.sync();
    // ---- F: beta, p update
    for (int cc = 0; cc < A.nrhs; ++cc) {
      const double rzn = sum_part(A.part_rz, cc, red);
      if (tid == 0) {
        beta[cc] = (done[cc] || rz[cc] == 0.0) ? 0.0 : rzn / rz[cc];
        if (!done[cc]) {
          rz[cc] = rzn;
          if (blockIdx.x == 0) {
            A.scal[PC_SC * cc + 0] = rzn;
            A.scal[PC_SC * cc + 5] = beta[cc];
          }
        }
      }
    }
    __syncthreads();
    if (blockIdx.x == 0 && tid == 0 && A.hist && its <= A.hist_cap) A.hist[2 * (its - 1) + 1] = beta[0];
    for (int64_t l = g0; l < A.m; l += gstride)
      for (int col = 0; col < A.nrhs; ++col)
        if (!done[col]) A.p[l + A.m * col] = A.z[l + A.m * col] + beta[col] * A.p[l + A.m * col];
    grid.sync();
  }
  if (blockIdx.x == 0 && tid < A.nrhs) A.scal[PC_SC * tid + 7] = done[tid] ? 1.0 : 0.0;
}

template <typename T, int CT>
static ieti_status launch_pcg(Ctx* c, PcgArgs A, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  IETI_CUDA_TRY(c, cudaGetDevice(&dev));
  IETI_CUDA_TRY(c, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return IETI_ERR_STATE;
  IETI_CUDA_TRY(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t smem = sizeof(T) * (size_t)A.u_ld * CT + sizeof(double) * (size_t)A.ngp * CT * 2 + 64;
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_pcg_coop<T, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  IETI_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_coop<T, CT>, 256, smem));
  if (per_sm < 1) return IETI_ERR_STATE;
  const int grid = std::min(sms * per_sm, PCG_COOP_MAX_GRID);
  void* args[] = {(void*)&A};
  cudaEvent_t p0 = prof_begin(c, st, PROF_PCG);
  IETI_CUDA_TRY(c, cudaLaunchCooperativeKernel((void*)k_pcg_coop<T, CT>, dim3(grid), dim3(256), args, smem, st));
  prof_end(c, PROF_PCG, p0, st);
  IETI_LAUNCH_CHECK(c);
  return IETI_OK;
}

ieti_status pcg_coop(Ctx* c, double* lam, double* r, double* z, double* p, double* q, double tol2, int maxit,
                     bool fp32, cudaStream_t st) {
  if (c->nrhs > 8) return IETI_ERR_STATE;
  PcgArgs A;
  A.sd = c->d_sd;
  A.nsub = c->nsub;
  A.nrhs = c->nrhs;
  A.ngp = (int)c->n_gp;
  A.ldc = (int)(ceil_div(std::max<int64_t>(c->n_gp, 1), NB) * NB);
  A.maxit = maxit;
  A.hist_cap = 4096;
  A.m = c->m_r;
  A.W = c->W;
  A.S = c->S;
  A.I_dual = c->d_I_dual;
  A.I_sign = c->d_I_sign;
  A.I_scale = c->d_I_scale;
  A.pair = c->d_pair;
  A.Phi = c->Phi;
  A.P_glob = c->d_P_glob;
  A.pcsr_off = c->d_pcsr_off;
  A.pcsr = c->d_pcsr;
  A.SPiInv = c->SPiInv;
  A.x = lam;
  A.r = r;
  A.z = z;
  A.p = p;
  A.q = q;
  A.t1 = c->wi[0];
  A.t2 = c->wi[1];
  A.qpart = c->wq_part;
  A.part_pq = c->wred;
  A.part_rr = c->wred + PCG_COOP_MAX_GRID * 8;
  A.part_rz = c->wred + PCG_COOP_MAX_GRID * 16;
  A.scal = c->wscal;
  A.hist = c->whist;
  A.tol2 = tol2;
  int items = 0;
  for (const SubDev& s : c->sd_host) items += (int)ceil_div(s.nI, PC_ROWS);
  A.total_items = items;
  A.u_ld = std::max(c->max_ldI, 4);
  if (c->nrhs == 1)
    return fp32 ? launch_pcg<float, 1>(c, A, st) : launch_pcg<double, 1>(c, A, st);
  return fp32 ? launch_pcg<float, 8>(c, A, st) : launch_pcg<double, 8>(c, A, st);
}


}  // namespace ieti
