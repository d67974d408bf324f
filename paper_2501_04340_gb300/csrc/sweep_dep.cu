// Triangular sweeps with the blocked Cholesky factors of all subdomains as
// dependency-driven block tasks: one cooperative launch per sweep and no grid
// barrier. Forward, block row b of subdomain k:
//   y_b = Linv_b (b_b - sum_{b0 <= j < b} L_bj y_j)
// backward, block column b:
//   x_b = Linv_b^T (y_b - sum_{j > b} L_jb^T x_j)
// (the local solves K_rr^(k) x = f of Eqs. (8), (9) and of the right-hand
// side of Eq. (7); with many columns, the W and Phi solves of the
// factorisation), over the nonzero tiles of the factor only (symbolic.cu).
// A task is one 64-wide block of one subdomain (times one tile of up to 64
// columns for many right-hand sides). The tasks are ordered by b (ascending
// forward, descending backward) and dealt round-robin to the CTAs; a CTA runs
// its tasks in that order. A task reads the finished blocks as they are
// published and publishes its own block by raising its progress counter (one
// per subdomain, or per subdomain and column tile) with a release store after
// writing it, once its predecessor in the order has been published (so the
// counter says that every block up to it is final); readers poll the counter
// with acquire loads (bounded, with an error flag on time-out) and read the
// blocks through L2. Every wait is on a task that comes earlier in the order
// and all CTAs are resident (cooperative launch), so every wait ends. The
// single-column sweeps zero their counters before each launch; the
// multi-column solves' counters carry an epoch in their upper bits instead.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace ieti {

namespace {

constexpr int DEP_THREADS = 256;
constexpr int DEP_EPOCH_SHIFT = 20;            // blocks per subdomain < 2^20
constexpr long long DEP_SPIN_MAX = 1LL << 22;  // default poll limit (polls of about 0.1 us)

template <typename T>
using Vec16 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// waits until *p >= need (bounded); on time-out, or once another wait has
// timed out, records the error and returns so that the launch ends. err[0] is
// the error flag; the poll limit is the 64-bit value at err + 2 (set by the host)
__device__ unsigned long long dep_wait(const unsigned long long* p, unsigned long long need, int* err) {
  unsigned long long v = ld_acquire_u64(p);
  const long long lim = v < need ? *reinterpret_cast<const volatile long long*>(err + 2) : 0;
  for (long long it = 0; v < need; ++it) {
    if (it >= lim || *(volatile int*)err) {
      atomicExch(err, 1);
      return need;
    }
    __nanosleep(64);
    v = ld_acquire_u64(p);
  }
  return v;
}

// all threads: the block's stores are done; one thread waits until the
// counter reaches prev (the blocks before this one in the order are
// published: with zero tiles a task may finish before its predecessor, and
// the counter must mean that every block up to it is final), then publishes.
// seen: the counter value thread 0 has already observed (no second poll when
// it covers prev). The release store orders the stores of the whole CTA,
// which the barrier has made visible to thread 0, before the new counter.
__device__ __forceinline__ void dep_publish(unsigned long long* p, unsigned long long prev, unsigned long long v,
                                            int* err, unsigned long long seen = 0) {
  __syncthreads();
  if (threadIdx.x == 0) {
    if (seen < prev) dep_wait(p, prev, err);
    st_release_u64(p, v);
  }
}

// 16 consecutive entries of a published vector, read through L2
template <typename T>
__device__ __forceinline__ void load16_cg(const T* src, T (&v)[16]) {
  constexpr int VL = 16 / sizeof(T);
  const Vec16<T>* s = reinterpret_cast<const Vec16<T>*>(src);
#pragma unroll
  for (int q = 0; q < 16 / VL; ++q) {
    const Vec16<T> w = __ldcg(s + q);
    if constexpr (VL == 4) {
      v[4 * q] = w.x; v[4 * q + 1] = w.y; v[4 * q + 2] = w.z; v[4 * q + 3] = w.w;
    } else {
      v[2 * q] = w.x; v[2 * q + 1] = w.y;
    }
  }
}

// Forward task (k, b): thread (i, cs) = (tid % 64, tid / 64) accumulates row
// b*64+i over the 16 columns cs*16.. of every block j; two blocks per round
// keep 32 loads of L in flight per thread.
template <typename T>
__global__ void __launch_bounds__(DEP_THREADS, 2)
    k_dep_fwd(const SubDev* sd, const SolveDesc* dsc, const int2* tasks, int ntask, const T* L, const T* Linv,
              const T* B, T* Y, unsigned long long* prog, unsigned long long base, int* err,
              const int64_t* lptr, const int32_t* lidx, const int* bbase) {
  extern __shared__ __align__(16) unsigned char dsm[];
  T* Lis = reinterpret_cast<T*>(dsm);    // Linv_b, column-major 64 x 64
  T* part = Lis + NB * NB;               // [4][64]
  T* rhs = part + 4 * NB;                // [64]
  const int tid = threadIdx.x, i = tid % NB, cs = tid / NB;
  constexpr int VL = 16 / sizeof(T);
  for (int t = blockIdx.x; t < ntask; t += gridDim.x) {
    const int2 tk = tasks[t];
    const int k = tk.x, b = tk.y;
    const SubDev s = sd[k];
    const SolveDesc d = dsc[k];
    const int64_t n = s.n;
    const T* Lr = L + s.A + (int64_t)b * NB + i + n * (cs * 16);   // row b*64+i, columns cs*16.. of block 0
    T* Yk = Y + d.boff - (int64_t)d.b0 * NB;                         // indexed by row of the subdomain
    __syncthreads();   // the previous task is done with the shared buffers
    {
      const Vec16<T>* src = reinterpret_cast<const Vec16<T>*>(Linv + s.linv + (int64_t)b * NB * NB);
      Vec16<T>* dst = reinterpret_cast<Vec16<T>*>(Lis);
      for (int q = tid; q < NB * NB / VL; q += DEP_THREADS) dst[q] = src[q];
    }
    // the right-hand side of the block, loaded before the waits
    const T bv = tid < NB ? B[d.boff + (int64_t)(b - d.b0) * NB + tid] : (T)0;
    T acc = 0;
    unsigned long long seen = 0;
    // the nonzero tiles L_bj of block row b (ascending j), from the range start
    int64_t e = lptr[bbase[k] + b];
    const int64_t e1 = lptr[bbase[k] + b + 1];
    while (e < e1 && lidx[e] < d.b0) ++e;
    for (; e + 1 < e1; e += 2) {
      const int ja = lidx[e], jb = lidx[e + 1];
      T l0[16], l1[16], y0[16], y1[16];
      const T* La = Lr + n * ((int64_t)ja * NB);
      const T* Lb2 = Lr + n * ((int64_t)jb * NB);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        l0[c] = La[n * c];
        l1[c] = Lb2[n * c];
      }
      if (seen < base + jb + 1) seen = dep_wait(prog + k, base + jb + 1, err);
      load16_cg(Yk + (int64_t)ja * NB + cs * 16, y0);
      load16_cg(Yk + (int64_t)jb * NB + cs * 16, y1);
#pragma unroll
      for (int c = 0; c < 16; ++c) acc += l0[c] * y0[c];
#pragma unroll
      for (int c = 0; c < 16; ++c) acc += l1[c] * y1[c];
    }
    if (e < e1) {
      const int ja = lidx[e];
      T l0[16], y0[16];
      const T* La = Lr + n * ((int64_t)ja * NB);
#pragma unroll
      for (int c = 0; c < 16; ++c) l0[c] = La[n * c];
      if (seen < base + ja + 1) seen = dep_wait(prog + k, base + ja + 1, err);
      load16_cg(Yk + (int64_t)ja * NB + cs * 16, y0);
#pragma unroll
      for (int c = 0; c < 16; ++c) acc += l0[c] * y0[c];
    }
    part[cs * NB + i] = acc;
    __syncthreads();
    if (tid < NB) rhs[tid] = bv - (part[tid] + part[NB + tid] + part[2 * NB + tid] + part[3 * NB + tid]);
    __syncthreads();
    // y_b = Linv_b rhs (zero above the diagonal): part cs sums columns cs*16..
    T v = 0;
#pragma unroll
    for (int c = 0; c < 16; ++c) v += Lis[i + NB * (cs * 16 + c)] * rhs[cs * 16 + c];
    part[cs * NB + i] = v;
    __syncthreads();
    if (tid < NB) Yk[(int64_t)b * NB + tid] = part[tid] + part[NB + tid] + part[2 * NB + tid] + part[3 * NB + tid];
    dep_publish(prog + k, b > d.b0 ? base + (unsigned long long)b : 0ull, base + (unsigned long long)(b + 1), err,
                seen);
  }
}

// Backward task (k, b): thread (i, cs) reads row i of every block (j, b) below
// the diagonal, columns cs*16.., and accumulates the 16 column sums; the sums
// over i meet in shared memory.
template <typename T>
__global__ void __launch_bounds__(DEP_THREADS, 2)
    k_dep_bwd(const SubDev* sd, const SolveDesc* dsc, const int2* tasks, int ntask, const T* L, const T* Linv,
              const T* Y, T* X, unsigned long long* prog, unsigned long long base, int* err,
              const int64_t* lptr, const int32_t* lidx, const int* bbase) {
  extern __shared__ __align__(16) unsigned char dsm[];
  T* Lis = reinterpret_cast<T*>(dsm);          // Lis[l * 65 + i] = Linv_b[l][i]
  T* red = Lis + NB * (NB + 1);                // red[i * 65 + c]: partial column sums of row i
  T* part = red + NB * (NB + 1);               // [4][64]
  T* rhs = part + 4 * NB;                      // [64]
  const int tid = threadIdx.x, i = tid % NB, cs = tid / NB;
  for (int t = blockIdx.x; t < ntask; t += gridDim.x) {
    const int2 tk = tasks[t];
    const int k = tk.x, b = tk.y;
    const SubDev s = sd[k];
    const SolveDesc d = dsc[k];
    const int64_t n = s.n;
    const int nb = s.nblk;
    const T* Lc = L + s.A + i + n * ((int64_t)b * NB + cs * 16);   // row i of block row 0, columns of block b
    const T* Yk = Y + d.boff - (int64_t)d.b0 * NB;
    T* Xk = X + d.boff - (int64_t)d.b0 * NB;
    __syncthreads();   // the previous task is done with the shared buffers
    {
      const T* Lb = Linv + s.linv + (int64_t)b * NB * NB;   // Lb[l + 64 i] = Linv_b[l][i]
      for (int q = tid; q < NB * NB; q += DEP_THREADS) Lis[(q % NB) * (NB + 1) + q / NB] = Lb[q];
    }
    // the right-hand side of the block (written by the forward sweep), loaded before the waits
    const T yv = tid < NB ? Yk[(int64_t)b * NB + tid] : (T)0;
    T acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0;
    unsigned long long seen = 0;
    // the nonzero tiles L_jb of block column b (descending j > b)
    int64_t e = lptr[bbase[k] + b];
    const int64_t e1 = lptr[bbase[k] + b + 1];
    for (; e + 1 < e1; e += 2) {
      const int ja = lidx[e], jb = lidx[e + 1];   // ja > jb
      T l0[16], l1[16];
      const T* La = Lc + (int64_t)ja * NB;
      const T* Lb2 = Lc + (int64_t)jb * NB;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        l0[c] = La[n * c];
        l1[c] = Lb2[n * c];
      }
      const unsigned long long need = base + (unsigned long long)(nb - jb);
      if (seen < need) seen = dep_wait(prog + k, need, err);
      const T x0 = __ldcg(Xk + (int64_t)ja * NB + i);
      const T x1 = __ldcg(Xk + (int64_t)jb * NB + i);
#pragma unroll
      for (int c = 0; c < 16; ++c) acc[c] += l0[c] * x0 + l1[c] * x1;
    }
    if (e < e1) {
      const int ja = lidx[e];
      T l0[16];
      const T* La = Lc + (int64_t)ja * NB;
#pragma unroll
      for (int c = 0; c < 16; ++c) l0[c] = La[n * c];
      const unsigned long long need = base + (unsigned long long)(nb - ja);
      if (seen < need) seen = dep_wait(prog + k, need, err);
      const T x0 = __ldcg(Xk + (int64_t)ja * NB + i);
#pragma unroll
      for (int c = 0; c < 16; ++c) acc[c] += l0[c] * x0;
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) red[i * (NB + 1) + cs * 16 + c] = acc[c];
    __syncthreads();
    {
      // column c = tid % 64 summed over the rows of quarter tid / 64
      const int c = tid % NB, qr = tid / NB;
      T v = 0;
#pragma unroll
      for (int r = 0; r < 16; ++r) v += red[(qr * 16 + r) * (NB + 1) + c];
      part[qr * NB + c] = v;
    }
    __syncthreads();
    if (tid < NB) rhs[tid] = yv - (part[tid] + part[NB + tid] + part[2 * NB + tid] + part[3 * NB + tid]);
    __syncthreads();
    // x_b = Linv_b^T rhs: x_i = sum_{l >= i} Linv_b[l][i] rhs_l, part cs sums l = cs*16..
    T v = 0;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int l = cs * 16 + c;
      v += Lis[l * (NB + 1) + i] * rhs[l];
    }
    part[cs * NB + i] = v;
    __syncthreads();
    if (tid < NB) Xk[(int64_t)b * NB + tid] = part[tid] + part[NB + tid] + part[2 * NB + tid] + part[3 * NB + tid];
    dep_publish(prog + k, b < nb - 1 ? base + (unsigned long long)(nb - b - 1) : 0ull,
                base + (unsigned long long)(nb - b), err, seen);
  }
}

// Tasks of two blocks (FP32 sweeps). The single-column sweep is bound by its
// chain of dependent blocks: after block b-1 is published, block b still
// reads it through L2, reduces, solves its diagonal block and publishes, about
// 3.5 us per link. A task that solves two consecutive blocks on chip halves the
// number of links. Both block rows (columns) of the pair walk the merged list
// of their nonzero tiles, so that the tiles of both are loaded before the
// waits and each published block is read once for both; the in-pair coupling
// tile is applied from registers once the first block of the pair is solved,
// and the pair is published with one counter store (the counter advances by
// two).
//
// Forward pair (b, b+1): y_b as in k_dep_fwd, then
//   y_{b+1} = Linv_{b+1} (b_{b+1} - sum_{j < b} L_{b+1,j} y_j - L_{b+1,b} y_b).
template <typename T>
__global__ void __launch_bounds__(DEP_THREADS, 2)
    k_dep_fwd2(const SubDev* sd, const SolveDesc* dsc, const int2* tasks, int ntask, const T* L, const T* Linv,
               const T* B, T* Y, unsigned long long* prog, unsigned long long base, int* err,
               const int64_t* lptr, const int32_t* lidx, const int* bbase) {
  extern __shared__ __align__(16) unsigned char dsm[];
  T* Lis0 = reinterpret_cast<T*>(dsm);   // Linv_b, column-major 64 x 64
  T* Lis1 = Lis0 + NB * NB;              // Linv_{b+1}
  T* part = Lis1 + NB * NB;              // [4][64]
  T* rhs = part + 4 * NB;                // [64]
  T* y0s = rhs + NB;                     // [64] y_b
  const int tid = threadIdx.x, i = tid % NB, cs = tid / NB;
  constexpr int VL = 16 / sizeof(T);
  constexpr int JEND = 1 << 30;
  for (int t = blockIdx.x; t < ntask; t += gridDim.x) {
    const int2 tk = tasks[t];
    const int k = tk.x, b = tk.y;
    const SubDev s = sd[k];
    const SolveDesc d = dsc[k];
    const int64_t n = s.n;
    const bool two = b + 1 < s.nblk;
    const T* Lr0 = L + s.A + (int64_t)b * NB + i + n * (cs * 16);   // row b*64+i, columns cs*16.. of block 0
    const T* Lr1 = Lr0 + NB;                                          // row (b+1)*64+i
    T* Yk = Y + d.boff - (int64_t)d.b0 * NB;
    __syncthreads();   // the previous task is done with the shared buffers
    {
      const Vec16<T>* src = reinterpret_cast<const Vec16<T>*>(Linv + s.linv + (int64_t)b * NB * NB);
      Vec16<T>* dst = reinterpret_cast<Vec16<T>*>(Lis0);
      for (int q = tid; q < (two ? 2 : 1) * NB * NB / VL; q += DEP_THREADS) dst[q] = src[q];
    }
    const T bv0 = tid < NB ? B[d.boff + (int64_t)(b - d.b0) * NB + tid] : (T)0;
    const T bv1 = (two && tid < NB) ? B[d.boff + (int64_t)(b + 1 - d.b0) * NB + tid] : (T)0;
    // tile lists of both rows from the range start; the in-pair tile L_{b+1,b}
    // is the last entry of row b+1 if nonzero
    int64_t e0 = lptr[bbase[k] + b];
    const int64_t e0e = lptr[bbase[k] + b + 1];
    int64_t e1 = two ? lptr[bbase[k] + b + 1] : 0;
    int64_t e1e = two ? lptr[bbase[k] + b + 2] : 0;
    const bool has_in = two && e1e > e1 && lidx[e1e - 1] == b;
    if (has_in) --e1e;
    while (e0 < e0e && lidx[e0] < d.b0) ++e0;
    while (e1 < e1e && lidx[e1] < d.b0) ++e1;
    T lin[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) lin[c] = has_in ? Lr1[n * ((int64_t)b * NB + c)] : (T)0;
    unsigned long long seen = 0;
    T acc0 = 0, acc1 = 0;
    while (e0 < e0e || e1 < e1e) {
      const int j0 = e0 < e0e ? lidx[e0] : JEND, j1 = e1 < e1e ? lidx[e1] : JEND;
      const int j = min(j0, j1);
      const bool h0 = j0 == j, h1 = j1 == j;
      T l0[16], l1[16], y[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        l0[c] = h0 ? Lr0[n * ((int64_t)j * NB + c)] : (T)0;
        l1[c] = h1 ? Lr1[n * ((int64_t)j * NB + c)] : (T)0;
      }
      if (seen < base + j + 1) seen = dep_wait(prog + k, base + j + 1, err);
      load16_cg(Yk + (int64_t)j * NB + cs * 16, y);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        acc0 += l0[c] * y[c];
        acc1 += l1[c] * y[c];
      }
      e0 += h0 ? 1 : 0;
      e1 += h1 ? 1 : 0;
    }
    // block b
    part[cs * NB + i] = acc0;
    __syncthreads();
    if (tid < NB) rhs[tid] = bv0 - (part[tid] + part[NB + tid] + part[2 * NB + tid] + part[3 * NB + tid]);
    __syncthreads();
    T v = 0;
#pragma unroll
    for (int c = 0; c < 16; ++c) v += Lis0[i + NB * (cs * 16 + c)] * rhs[cs * 16 + c];
    part[cs * NB + i] = v;
    __syncthreads();
    if (tid < NB) {
      const T yb = part[tid] + part[NB + tid] + part[2 * NB + tid] + part[3 * NB + tid];
      Yk[(int64_t)b * NB + tid] = yb;
      y0s[tid] = yb;
    }
    if (two) {
      __syncthreads();   // y_b in shared memory; part is free
      T a1 = acc1;
#pragma unroll
      for (int c = 0; c < 16; ++c) a1 += lin[c] * y0s[cs * 16 + c];
      part[cs * NB + i] = a1;
      __syncthreads();
      if (tid < NB) rhs[tid] = bv1 - (part[tid] + part[NB + tid] + part[2 * NB + tid] + part[3 * NB + tid]);
      __syncthreads();
      T v1 = 0;
#pragma unroll
      for (int c = 0; c < 16; ++c) v1 += Lis1[i + NB * (cs * 16 + c)] * rhs[cs * 16 + c];
      part[cs * NB + i] = v1;
      __syncthreads();
      if (tid < NB)
        Yk[(int64_t)(b + 1) * NB + tid] = part[tid] + part[NB + tid] + part[2 * NB + tid] + part[3 * NB + tid];
    }
    dep_publish(prog + k, b > d.b0 ? base + (unsigned long long)b : 0ull,
                base + (unsigned long long)(b + (two ? 2 : 1)), err, seen);
  }
}

// Backward pair (b, b-1), b the upper block: x_b as in k_dep_bwd, then
//   x_{b-1} = Linv_{b-1}^T (y_{b-1} - sum_{j > b} L_{j,b-1}^T x_j - L_{b,b-1}^T x_b).
template <typename T>
__global__ void __launch_bounds__(DEP_THREADS, 2)
    k_dep_bwd2(const SubDev* sd, const SolveDesc* dsc, const int2* tasks, int ntask, const T* L, const T* Linv,
               const T* Y, T* X, unsigned long long* prog, unsigned long long base, int* err,
               const int64_t* lptr, const int32_t* lidx, const int* bbase) {
  extern __shared__ __align__(16) unsigned char dsm[];
  T* Lis0 = reinterpret_cast<T*>(dsm);         // Lis0[l * 65 + i] = Linv_b[l][i]
  T* Lis1 = Lis0 + NB * (NB + 1);              // Linv_{b-1}, same layout
  T* red = Lis1 + NB * (NB + 1);               // red[i * 65 + c]: partial column sums of row i
  T* part = red + NB * (NB + 1);               // [4][64]
  T* rhs = part + 4 * NB;                      // [64]
  T* xbs = rhs + NB;                           // [64] x_b
  const int tid = threadIdx.x, i = tid % NB, cs = tid / NB;
  for (int t = blockIdx.x; t < ntask; t += gridDim.x) {
    const int2 tk = tasks[t];
    const int k = tk.x, b = tk.y;
    const SubDev s = sd[k];
    const SolveDesc d = dsc[k];
    const int64_t n = s.n;
    const int nb = s.nblk;
    const bool two = b - 1 >= d.b0;
    const T* Lc0 = L + s.A + i + n * ((int64_t)b * NB + cs * 16);   // row i of block row 0, columns of block b
    const T* Lc1 = Lc0 - n * NB;                                      // columns of block b-1
    const T* Yk = Y + d.boff - (int64_t)d.b0 * NB;
    T* Xk = X + d.boff - (int64_t)d.b0 * NB;
    __syncthreads();   // the previous task is done with the shared buffers
    {
      const T* Lb = Linv + s.linv + (int64_t)b * NB * NB;   // Lb[l + 64 i] = Linv_b[l][i]
      for (int q = tid; q < NB * NB; q += DEP_THREADS) Lis0[(q % NB) * (NB + 1) + q / NB] = Lb[q];
      if (two) {
        const T* Lm = Lb - NB * NB;
        for (int q = tid; q < NB * NB; q += DEP_THREADS) Lis1[(q % NB) * (NB + 1) + q / NB] = Lm[q];
      }
    }
    const T yv0 = tid < NB ? Yk[(int64_t)b * NB + tid] : (T)0;
    const T yv1 = (two && tid < NB) ? Yk[(int64_t)(b - 1) * NB + tid] : (T)0;
    // column lists (descending j) of both columns; the in-pair tile L_{b,b-1}
    // is the last entry (smallest j) of column b-1 if nonzero
    int64_t e0 = lptr[bbase[k] + b];
    const int64_t e0e = lptr[bbase[k] + b + 1];
    int64_t e1 = two ? lptr[bbase[k] + b - 1] : 0;
    int64_t e1e = two ? lptr[bbase[k] + b] : 0;
    const bool has_in = two && e1e > e1 && lidx[e1e - 1] == b;
    if (has_in) --e1e;
    T lin[16];
    {
      const T* Li = Lc1 + (int64_t)b * NB;   // row b*64+i, columns (b-1)*64 + cs*16..
#pragma unroll
      for (int c = 0; c < 16; ++c) lin[c] = has_in ? Li[n * c] : (T)0;
    }
    unsigned long long seen = 0;
    T acc0[16], acc1[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc0[c] = acc1[c] = 0;
    while (e0 < e0e || e1 < e1e) {
      const int j0 = e0 < e0e ? lidx[e0] : -1, j1 = e1 < e1e ? lidx[e1] : -1;
      const int j = max(j0, j1);   // descending
      const bool h0 = j0 == j, h1 = j1 == j;
      T l0[16], l1[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        l0[c] = h0 ? Lc0[(int64_t)j * NB + n * c] : (T)0;
        l1[c] = h1 ? Lc1[(int64_t)j * NB + n * c] : (T)0;
      }
      const unsigned long long need = base + (unsigned long long)(nb - j);
      if (seen < need) seen = dep_wait(prog + k, need, err);
      const T x = __ldcg(Xk + (int64_t)j * NB + i);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        acc0[c] += l0[c] * x;
        acc1[c] += l1[c] * x;
      }
      e0 += h0 ? 1 : 0;
      e1 += h1 ? 1 : 0;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !two) break;
      const T* Lis = h == 0 ? Lis0 : Lis1;
      if (h == 1) {
        // x_b is in shared memory: add the in-pair products to the sums of block b-1
        const T xb = xbs[i];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc1[c] += lin[c] * xb;
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) red[i * (NB + 1) + cs * 16 + c] = h == 0 ? acc0[c] : acc1[c];
      __syncthreads();
      {
        const int c = tid % NB, qr = tid / NB;
        T v = 0;
#pragma unroll
        for (int r = 0; r < 16; ++r) v += red[(qr * 16 + r) * (NB + 1) + c];
        part[qr * NB + c] = v;
      }
      __syncthreads();
      if (tid < NB)
        rhs[tid] = (h == 0 ? yv0 : yv1) - (part[tid] + part[NB + tid] + part[2 * NB + tid] + part[3 * NB + tid]);
      __syncthreads();
      T v = 0;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int l = cs * 16 + c;
        v += Lis[l * (NB + 1) + i] * rhs[l];
      }
      part[cs * NB + i] = v;
      __syncthreads();
      if (tid < NB) {
        const T x = part[tid] + part[NB + tid] + part[2 * NB + tid] + part[3 * NB + tid];
        Xk[(int64_t)(b - h) * NB + tid] = x;
        if (h == 0) xbs[tid] = x;
      }
      __syncthreads();   // x_b visible; red and part free
    }
    dep_publish(prog + k, b < nb - 1 ? base + (unsigned long long)(nb - b - 1) : 0ull,
                base + (unsigned long long)(nb - b + (two ? 1 : 0)), err, seen);
  }
}

// Many right-hand sides (the W and Phi solves of the factorisation): a task is
// one 64-wide block of one subdomain times one tile of up to 64 columns, and
// every column tile of a subdomain has its own progress counter. Forward,
// block b: Y_b = Linv_b (B_b - sum_j L_bj Y_j) with 64 x 64 tile products
// staged in shared memory (4 x 4 outputs per thread); backward, block b:
// X_b = Linv_b^T (Y_b - sum_{j > b} L_jb^T X_j).
template <typename T>
__global__ void __launch_bounds__(DEP_THREADS)
    k_depmc(const SubDev* sd, const SolveDesc* dsc, const int4* tasks, int ntask, const T* L, const T* Linv,
            const T* In, T* Out, unsigned long long* prog, unsigned long long base, int* err,
            const int64_t* lptr, const int32_t* lidx, const int* bbase, int fwd) {
  extern __shared__ __align__(16) unsigned char dsm[];
  T(*As)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(dsm);
  T(*Bs)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(dsm + sizeof(T) * NB * (NB + 1));
  const int tid = threadIdx.x, ti = tid % 16, tj = tid / 16;
  for (int t = blockIdx.x; t < ntask; t += gridDim.x) {
    const int4 tk = tasks[t];
    const int k = tk.x, b = tk.y, c0 = tk.z * NB, v = tk.w;
    const SubDev s = sd[k];
    const SolveDesc d = dsc[k];
    const int64_t n = s.n;
    const int nb = s.nblk;
    const int nc = min(NB, d.ncol - c0);
    // In (forward: B, backward: Y) and Out (Y, X) indexed by subdomain row
    const T* Ik = In + d.boff + (int64_t)d.ldb * c0 - (int64_t)d.b0 * NB;
    T* Ok = Out + d.boff + (int64_t)d.ldb * c0 - (int64_t)d.b0 * NB;
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < 4; ++w) acc[u][w] = 0;
    unsigned long long seen = 0;
    int64_t e = lptr[bbase[k] + b];
    const int64_t e1 = lptr[bbase[k] + b + 1];
    if (fwd)
      while (e < e1 && lidx[e] < d.b0) ++e;
    for (; e < e1; ++e) {
      const int j = lidx[e];
      __syncthreads();   // the previous tiles are consumed
      // forward: As[i][l] = L[64 b + i, 64 j + l]; backward: As[l][i] = L[64 j + l, 64 b + i]
      for (int q = tid; q < NB * NB; q += DEP_THREADS) {
        const int x = q % NB, y = q / NB;
        if (fwd) As[x][y] = L[s.A + (int64_t)b * NB + x + n * ((int64_t)j * NB + y)];
        else As[x][y] = L[s.A + (int64_t)j * NB + x + n * ((int64_t)b * NB + y)];
      }
      const unsigned long long need = fwd ? base + (unsigned long long)(j + 1) : base + (unsigned long long)(nb - j);
      if (seen < need) seen = dep_wait(prog + v, need, err);
      for (int q = tid; q < NB * NB; q += DEP_THREADS) {
        const int l = q % NB, cc = q / NB;
        Bs[l][cc] = cc < nc ? __ldcg(Ok + (int64_t)j * NB + l + (int64_t)d.ldb * cc) : (T)0;
      }
      __syncthreads();
#pragma unroll 4
      for (int l = 0; l < NB; ++l) {
        T a[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = fwd ? As[4 * ti + u][l] : As[l][4 * ti + u];
#pragma unroll
        for (int w = 0; w < 4; ++w) y[w] = Bs[l][4 * tj + w];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[u][w] += a[u] * y[w];
      }
    }
    __syncthreads();
    // right-hand side of the diagonal block, and the inverse of the diagonal
    // block (forward As[i][l] = Linv_b[i][l], backward As[l][i] = Linv_b[l][i])
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int i = 4 * ti + u, cc = 4 * tj + w;
        Bs[i][cc] = (cc < nc ? Ik[(int64_t)b * NB + i + (int64_t)d.ldb * cc] : (T)0) - acc[u][w];
      }
    for (int q = tid; q < NB * NB; q += DEP_THREADS) As[q % NB][q / NB] = Linv[s.linv + (int64_t)b * NB * NB + q];
    __syncthreads();
    T o[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < 4; ++w) o[u][w] = 0;
#pragma unroll 4
    for (int l = 0; l < NB; ++l) {
      T a[4], y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = fwd ? As[4 * ti + u][l] : As[l][4 * ti + u];
#pragma unroll
      for (int w = 0; w < 4; ++w) y[w] = Bs[l][4 * tj + w];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) o[u][w] += a[u] * y[w];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int i = 4 * ti + u, cc = 4 * tj + w;
        if (cc < nc) Ok[(int64_t)b * NB + i + (int64_t)d.ldb * cc] = o[u][w];
      }
    if (fwd)
      dep_publish(prog + v, b > d.b0 ? base + (unsigned long long)b : 0ull, base + (unsigned long long)(b + 1), err,
                  seen);
    else
      dep_publish(prog + v, b < nb - 1 ? base + (unsigned long long)(nb - b - 1) : 0ull,
                  base + (unsigned long long)(nb - b), err, seen);
  }
}

template <typename T>
size_t mc_smem() { return sizeof(T) * 2 * (size_t)NB * (NB + 1); }

template <typename T>
size_t fwd_smem() { return sizeof(T) * ((size_t)NB * NB + 5 * NB); }
template <typename T>
size_t bwd_smem() { return sizeof(T) * (2 * (size_t)NB * (NB + 1) + 5 * NB); }
template <typename T>
size_t fwd2_smem() { return sizeof(T) * (2 * (size_t)NB * NB + 6 * NB); }
template <typename T>
size_t bwd2_smem() { return sizeof(T) * (3 * (size_t)NB * (NB + 1) + 6 * NB); }

template <typename T>
ieti_status launch_dep(Ctx* c, bool fwd, int range, const T* B, const T* Yin, T* Yout, cudaStream_t st) {
  const int which = fwd ? 0 : 1;
  // FP32: tasks of two blocks (the FP64 pair kernels would need more registers
  // than two CTAs per SM leave)
  constexpr bool pairs = sizeof(T) == 4;
  const int ntask = pairs ? c->dep_ntask2[range][which] : c->dep_ntask[range][which];
  if (ntask == 0) return IETI_OK;
  if (!c->symb_ready) return IETI_ERR_STATE;   // tile lists of the factor
  int dev = 0, coop = 0;
  IETI_CUDA_TRY(c, cudaGetDevice(&dev));
  IETI_CUDA_TRY(c, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop || c->sm_count < 1) return IETI_ERR_STATE;
  const SolveDesc* dd = c->d_desc_rv + (range == RV_IRANGE ? c->nsub : 0);
  const int2* tasks = pairs ? c->d_dep_tasks2[range][which] : c->d_dep_tasks[range][which];
  const size_t smem = pairs ? (fwd ? fwd2_smem<T>() : bwd2_smem<T>()) : (fwd ? fwd_smem<T>() : bwd_smem<T>());
  void* kern;
  if constexpr (pairs) kern = fwd ? (void*)k_dep_fwd2<T> : (void*)k_dep_bwd2<T>;
  else kern = fwd ? (void*)k_dep_fwd<T> : (void*)k_dep_bwd<T>;
  int per_sm = 0;
  IETI_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, DEP_THREADS, smem));
  if (per_sm < 1) return IETI_ERR_STATE;
  const int grid = std::min(ntask, per_sm * c->sm_count);
  // the progress counters start from zero at every sweep (a memset before the
  // launch), so the launch's arguments are the same every time and a graph of
  // the step can replay it
  const unsigned long long base = 1ull << DEP_EPOCH_SHIFT;
  unsigned long long* prog = c->d_dep_prog;
  IETI_CUDA_TRY(c, cudaMemsetAsync(prog, 0, sizeof(unsigned long long) * std::max(c->nsub, 1), st));
  const T* L = (const T*)c->L;
  const T* Linv = (const T*)c->Linv;
  const SubDev* sd = c->d_sd;
  int* err = c->d_dep_err;
  const int64_t* lptr = fwd ? c->d_lrow_ptr : c->d_lcol_ptr;
  const int32_t* lidx = fwd ? c->d_lrow_col : c->d_lcol_row;
  const int* bbase = c->d_ktile_base;
  void* args[] = {(void*)&sd, (void*)&dd, (void*)&tasks, (void*)&ntask, (void*)&L, (void*)&Linv,
                  (void*)(fwd ? &B : &Yin), (void*)&Yout, (void*)&prog, (void*)&base, (void*)&err,
                  (void*)&lptr, (void*)&lidx, (void*)&bbase};
  cudaEvent_t p0 = prof_begin(c, st);
  IETI_CUDA_TRY(c, cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(DEP_THREADS), args, smem, st));
  prof_end(c, fwd ? PROF_FWD : PROF_BWD, p0, st);
  IETI_LAUNCH_CHECK(c);
  return IETI_OK;
}

}  // namespace

ieti_status dep_sweep_attrs(Ctx* c) {
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_depmc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)mc_smem<float>()));
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_depmc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)mc_smem<double>()));
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_dep_fwd<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)fwd_smem<float>()));
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_dep_fwd<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)fwd_smem<double>()));
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_dep_bwd<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)bwd_smem<float>()));
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_dep_bwd<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)bwd_smem<double>()));
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_dep_fwd2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)fwd2_smem<float>()));
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_dep_bwd2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)bwd2_smem<float>()));
  return IETI_OK;
}

#define TRY_DEP(x)                   \
  do {                               \
    ieti_status r__ = (x);           \
    if (r__ != IETI_OK) return r__;  \
  } while (0)

// poll limit of the dependency waits (polls of about 0.1 us each)
ieti_status dep_set_poll_limit(Ctx* c, long long polls) {
  const long long v = std::max(0LL, polls);
  IETI_CUDA_TRY(c, cudaMemcpy(reinterpret_cast<char*>(c->d_dep_err) + 8, &v, sizeof(v), cudaMemcpyHostToDevice));
  return IETI_OK;
}

// task tables of the r-vector sweeps (whole r range and r_I rows, forward and
// backward), progress counters and the error flag
ieti_status dep_sweep_alloc(Ctx* c) {
  for (int range = 0; range < 2; ++range) {
    for (int which = 0; which < 2; ++which) {
      std::vector<int2> tk;
      for (int b = 0; b < c->max_nblk; ++b)
        for (int k = 0; k < c->nsub; ++k) {
          const SubDev& s = c->sd_host[k];
          const int b0 = range == RV_IRANGE ? s.nVp / NB : 0;
          if (range == RV_IRANGE && s.nI == 0) continue;
          const int bb = which == 0 ? b : c->max_nblk - 1 - b;
          if (bb >= b0 && bb < s.nblk) tk.push_back(make_int2(k, bb));
        }
      c->dep_ntask[range][which] = (int)tk.size();
      int2* d = nullptr;
      const size_t bytes = sizeof(int2) * std::max<size_t>(tk.size(), 1);
      IETI_CUDA_TRY(c, cudaMalloc(&d, bytes));
      c->allocs.push_back({d, bytes});
      if (!tk.empty()) IETI_CUDA_TRY(c, cudaMemcpy(d, tk.data(), sizeof(int2) * tk.size(), cudaMemcpyHostToDevice));
      c->d_dep_tasks[range][which] = d;
      // pairs of blocks, aligned at the start of the sweep: forward (b0, b0+1),
      // (b0+2, b0+3), ...; backward (nblk-1, nblk-2), ...; a lone block ends it
      std::vector<int2> t2;
      for (int q = 0; 2 * q < c->max_nblk; ++q)
        for (int k = 0; k < c->nsub; ++k) {
          const SubDev& sk = c->sd_host[k];
          if (range == RV_IRANGE && sk.nI == 0) continue;
          const int b0 = range == RV_IRANGE ? sk.nVp / NB : 0;
          const int b = which == 0 ? b0 + 2 * q : sk.nblk - 1 - 2 * q;
          if (b >= b0 && b < sk.nblk) t2.push_back(make_int2(k, b));
        }
      c->dep_ntask2[range][which] = (int)t2.size();
      int2* d2 = nullptr;
      const size_t bytes2 = sizeof(int2) * std::max<size_t>(t2.size(), 1);
      IETI_CUDA_TRY(c, cudaMalloc(&d2, bytes2));
      c->allocs.push_back({d2, bytes2});
      if (!t2.empty()) IETI_CUDA_TRY(c, cudaMemcpy(d2, t2.data(), sizeof(int2) * t2.size(), cudaMemcpyHostToDevice));
      c->d_dep_tasks2[range][which] = d2;
    }
  }
  unsigned long long* pg = nullptr;
  IETI_CUDA_TRY(c, cudaMalloc(&pg, sizeof(unsigned long long) * std::max(c->nsub, 1)));
  c->allocs.push_back({pg, sizeof(unsigned long long) * std::max(c->nsub, 1)});
  IETI_CUDA_TRY(c, cudaMemset(pg, 0, sizeof(unsigned long long) * std::max(c->nsub, 1)));
  c->d_dep_prog = pg;
  // error flag (int) at offset 0, poll limit of the waits (int64) at offset 8
  int* e = nullptr;
  IETI_CUDA_TRY(c, cudaMalloc(&e, 16));
  c->allocs.push_back({e, 16});
  IETI_CUDA_TRY(c, cudaMemset(e, 0, 16));
  c->d_dep_err = e;
  TRY_DEP(dep_set_poll_limit(c, DEP_SPIN_MAX));
  c->dep_epoch = 0;
  return IETI_OK;
}

// multi-column solves of a fixed descriptor set (slot 0: W, 1: Phi); the task
// lists and progress counters are built on the first call
template <typename T>
ieti_status dep_mc_solve(Ctx* c, int slot, const std::vector<SolveDesc>& dh, const SolveDesc* dd, int which,
                         const T* B, T* Y, T* X, cudaStream_t st) {
  if (!c->symb_ready) return IETI_ERR_STATE;
  int dev = 0, coop = 0;
  IETI_CUDA_TRY(c, cudaGetDevice(&dev));
  IETI_CUDA_TRY(c, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop || c->sm_count < 1) return IETI_ERR_STATE;
  McPlan& P = c->mcplan[slot];
  if (!P.built) {
    std::vector<int> vb(c->nsub + 1, 0);
    for (int k = 0; k < c->nsub; ++k) vb[k + 1] = vb[k] + (int)((std::max(dh[k].ncol, 0) + NB - 1) / NB);
    for (int dir = 0; dir < 2; ++dir) {
      std::vector<int4> tk;
      for (int bb = 0; bb < c->max_nblk; ++bb) {
        const int b = dir == 0 ? bb : c->max_nblk - 1 - bb;
        for (int k = 0; k < c->nsub; ++k) {
          const SubDev& s = c->sd_host[k];
          if (b < dh[k].b0 || b >= s.nblk || dh[k].ncol <= 0) continue;
          for (int ct = 0; ct < vb[k + 1] - vb[k]; ++ct) tk.push_back(make_int4(k, b, ct, vb[k] + ct));
        }
      }
      P.ntask[dir] = (int)tk.size();
      if (tk.empty()) tk.push_back(make_int4(0, 0, 0, 0));
      ieti_status r;
      if ((r = dev_upload(c, &P.d_tasks[dir], tk)) != IETI_OK) return r;
    }
    std::vector<unsigned long long> z(std::max(vb[c->nsub], 1), 0ull);
    ieti_status r;
    if ((r = dev_upload(c, &P.d_prog, z)) != IETI_OK) return r;
    P.built = true;
  }
  const size_t smem = mc_smem<T>();
  int per_sm = 0;
  IETI_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_depmc<T>, DEP_THREADS, smem));
  if (per_sm < 1) return IETI_ERR_STATE;
  const T* L = (const T*)c->L;
  const T* Linv = (const T*)c->Linv;
  const SubDev* sd = c->d_sd;
  int* err = c->d_dep_err;
  const int* bbase = c->d_ktile_base;
  for (int dir = 0; dir < 2; ++dir) {
    if (!(which & (dir == 0 ? SWEEP_FWD : SWEEP_BWD))) continue;
    const int ntask = P.ntask[dir];
    if (ntask == 0) continue;
    const int4* tasks = P.d_tasks[dir];
    const int grid = std::min(ntask, per_sm * c->sm_count);
    const unsigned long long base = (++c->dep_epoch) << DEP_EPOCH_SHIFT;
    const T* In = dir == 0 ? B : Y;
    T* Out = dir == 0 ? Y : X;
    const int64_t* lptr = dir == 0 ? c->d_lrow_ptr : c->d_lcol_ptr;
    const int32_t* lidx = dir == 0 ? c->d_lrow_col : c->d_lcol_row;
    int fwd = dir == 0 ? 1 : 0;
    unsigned long long* prog = P.d_prog;
    void* args[] = {(void*)&sd, (void*)&dd, (void*)&tasks, (void*)&ntask, (void*)&L, (void*)&Linv,
                    (void*)&In, (void*)&Out, (void*)&prog, (void*)&base, (void*)&err,
                    (void*)&lptr, (void*)&lidx, (void*)&bbase, (void*)&fwd};
    cudaEvent_t p0 = prof_begin(c, st);
    IETI_CUDA_TRY(c, cudaLaunchCooperativeKernel((void*)k_depmc<T>, dim3(grid), dim3(DEP_THREADS), args, smem, st));
    prof_end(c, dir == 0 ? PROF_FWD : PROF_BWD, p0, st);
    IETI_LAUNCH_CHECK(c);
  }
  return IETI_OK;
}
template ieti_status dep_mc_solve<float>(Ctx*, int, const std::vector<SolveDesc>&, const SolveDesc*, int,
                                         const float*, float*, float*, cudaStream_t);
template ieti_status dep_mc_solve<double>(Ctx*, int, const std::vector<SolveDesc>&, const SolveDesc*, int,
                                          const double*, double*, double*, cudaStream_t);

template <typename T>
ieti_status dep_sweep(Ctx* c, int range, int which, const T* B, T* Y, T* X, cudaStream_t st) {
  ieti_status r;
  if ((which & SWEEP_FWD) && (r = launch_dep<T>(c, true, range, B, nullptr, Y, st)) != IETI_OK) return r;
  if ((which & SWEEP_BWD) && (r = launch_dep<T>(c, false, range, nullptr, Y, X, st)) != IETI_OK) return r;
  return IETI_OK;
}
template ieti_status dep_sweep<float>(Ctx*, int, int, const float*, float*, float*, cudaStream_t);
template ieti_status dep_sweep<double>(Ctx*, int, int, const double*, double*, double*, cudaStream_t);

}  // namespace ieti
