// Batched dense factorisations of the local blocks (Sec. 2.1: K_rr block
// diagonal, "every K_rr^(k) invertible after tree and primal removal").
//
// Right-looking blocked Cholesky with NB x NB panels over all subdomains at
// once (uneven sizes: a subdomain whose panel count is exhausted skips the
// launch). The r DOFs are ordered [r_V, pad, r_I, pad]; right after the r_V
// panels the trailing block is exactly S_rIrI = K_II - K_IV K_VV^-1 K_VI
// (Eq. (10)), which is snapshotted. The inverses of the diagonal blocks are kept
// so that every triangular solve is a sequence of small dense products.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace ieti {

template <typename T>
ieti_status convert_copy(Ctx* c, const double* src, T* dst, int64_t n, cudaStream_t st);
template <typename T>
ieti_status convert_tiles(Ctx* c, const int4* tiles, int ntiles, const double* src, T* dst, cudaStream_t st);


// ---------------------------------------------------------------------------
// Cholesky kernels
// ---------------------------------------------------------------------------

// Cholesky of the 64 x 64 block a (lower part) by all threads: one column per
// step, two barriers a step (the FP64 path: its register form would spill)
template <typename T>
__device__ void chol64_cta(T (*a)[NB + 1], int* bad) {
  const int tid = threadIdx.x;
  // thread (row i, column group g) updates a[i][16 g .. 16 g + 15]: the lanes of
  // a warp share g, so a[l][c] is a broadcast and a[i][l] is conflict-free
  const int ri = tid % NB, g = tid / NB;
  for (int c = 0; c < NB; ++c) {
    // every thread forms the pivot itself; the threads below it scale column c
    // (a[c][c] itself is written after the barrier, once nobody reads it)
    const T v0 = a[c][c];
    const T piv = sqrt(v0 > (T)0 ? v0 : (T)1);
    if (tid > c && tid < NB) a[tid][c] /= piv;
    __syncthreads();
    if (tid == 0) {
      if (!(v0 > (T)0)) *bad = 1;
      a[c][c] = piv;
    }
    if (ri > c && 16 * g <= ri && 16 * g + 15 > c) {
      const T aic = a[ri][c];
      // unrolled with predicates: the 16 updates are independent
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int l = 16 * g + u;
        if (l > c && l <= ri) a[ri][l] -= aic * a[l][c];
      }
    }
    __syncthreads();
  }
}

// Cholesky of the 64 x 64 block a (lower part) in the registers of warp 0:
// lane l holds rows l (columns 0..l) and l + 32 (columns 0..l + 32); column c
// is scaled by the lanes below the pivot and its entries reach the other
// lanes by shuffles for the rank-1 update, with no barrier at all
__device__ void chol64_warp(float (*a)[NB + 1], int* bad) {
  const int lane = threadIdx.x & 31;
  float ra[32], rb[64];
#pragma unroll
  for (int l = 0; l < 32; ++l) ra[l] = l <= lane ? a[lane][l] : 0.f;
#pragma unroll
  for (int l = 0; l < 64; ++l) rb[l] = l <= lane + 32 ? a[lane + 32][l] : 0.f;
  bool nonpos = false;
#pragma unroll
  for (int c = 0; c < 64; ++c) {
    // (the indices are clamped so that every array index is in range; the
    // loops are unrolled, so each select is resolved at compile time)
    const int cc = c < 32 ? c : 0;
    const float d = __shfl_sync(0xffffffffu, c < 32 ? ra[cc] : rb[c], c & 31);
    nonpos |= !(d > 0.f);
    // the pivot and its reciprocal from one reciprocal square root (a
    // shorter dependent chain than a square root and a division; the FP32
    // factor is refined in FP64 anyway)
    const float dd = d > 0.f ? d : 1.f;
    const float rp = rsqrtf(dd);
    const float piv = dd * rp;
    if (c < 32) ra[cc] = lane > c ? ra[cc] * rp : (lane == c ? piv : ra[cc]);
    rb[c] = lane + 32 > c ? rb[c] * rp : (lane + 32 == c ? piv : rb[c]);
#pragma unroll
    for (int l = c + 1; l < 64; ++l) {
      const float llc = __shfl_sync(0xffffffffu, l < 32 ? ra[cc] : rb[c], l & 31);
      if (l < 32 && lane >= l) ra[l < 32 ? l : 0] -= ra[cc] * llc;
      if (lane + 32 >= l) rb[l] -= rb[c] * llc;
    }
  }
#pragma unroll
  for (int l = 0; l < 32; ++l)
    if (l <= lane) a[lane][l] = ra[l];
#pragma unroll
  for (int l = 0; l < 64; ++l)
    if (l <= lane + 32) a[lane + 32][l] = rb[l];
  if (lane == 0 && nonpos) *bad = 1;
}

// inverse of the lower triangular factor in a into inv (zero above the
// diagonal) by block doubling, all threads: the four 16 x 16 diagonal blocks
// by forward substitution (one warp each, one column per lane), then
// [X11 0; X21 X22] with X21 = -X22 L21 X11 at 32 and at 64. The two products of
// each level go through the unused upper triangle of a as scratch.
template <typename T>
__device__ void inv64_blocks(T (*a)[NB + 1], T (*inv)[NB + 1], T* rd) {
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  for (int t = tid; t < NB * NB; t += blockDim.x) inv[t % NB][t / NB] = (T)0;
  if (tid < NB) rd[tid] = (T)1 / a[tid][tid];
  __syncthreads();
  if (warp < 4 && lane < 16) {
    const int o = 16 * warp, j = lane;
    T x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      T acc = i == j ? (T)1 : (T)0;
#pragma unroll
      for (int l = 0; l < i; ++l) acc -= a[o + i][o + l] * x[l];
      x[i] = i >= j ? acc * rd[o + i] : (T)0;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) inv[o + i][o + j] = x[i];
  }
  __syncthreads();
  {
    // 32 x 32 blocks at o = 0 and 32 (128 threads each): scratch
    // a[o + i][o + 16 + j], above the diagonal
    const int B = tid / 128, e = tid % 128, o = 32 * B;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = e % 16, j = e / 16 + 8 * h;
      T acc = 0;
#pragma unroll
      for (int l = 0; l < 16; ++l) acc += a[o + 16 + i][o + l] * inv[o + l][o + j];
      a[o + i][o + 16 + j] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = e % 16, j = e / 16 + 8 * h;
      T acc = 0;
#pragma unroll
      for (int l = 0; l < 16; ++l) acc += inv[o + 16 + i][o + 16 + l] * a[o + l][o + 16 + j];
      inv[o + 16 + i][o + j] = -acc;
    }
  }
  __syncthreads();
  // 64 x 64: scratch a[i][32 + j], the upper right block
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const int i = tid % 32, j = tid / 32 + 8 * h;
    T acc = 0;
#pragma unroll 8
    for (int l = 0; l < 32; ++l) acc += a[32 + i][l] * inv[l][j];
    a[i][32 + j] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const int i = tid % 32, j = tid / 32 + 8 * h;
    T acc = 0;
#pragma unroll 8
    for (int l = 0; l < 32; ++l) acc += inv[32 + i][32 + l] * a[l][32 + j];
    inv[32 + i][j] = -acc;
  }
  __syncthreads();
}

// diagonal block b of every subdomain: Cholesky factor (lower part written
// back, zeros above) and the inverse of the factor (to Linv); 256 threads
template <typename T>
__global__ void __launch_bounds__(256) k_potrf_diag(const SubDev* sd, T* L, T* Linv, int b, int* err) {
  const int k = blockIdx.x;
  const SubDev s = sd[k];
  if (b >= s.nblk) return;
  __shared__ T a[NB][NB + 1];
  __shared__ T inv[NB][NB + 1];
  __shared__ T rd[NB];
  __shared__ int bad;
  const int tid = threadIdx.x;
  T* A = L + s.A + (int64_t)b * NB + (int64_t)s.n * b * NB;
  for (int t = tid; t < NB * NB; t += blockDim.x) {
    int i = t % NB, j = t / NB;
    a[i][j] = A[i + (int64_t)s.n * j];
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  if constexpr (sizeof(T) == 4) {
    if (tid < 32) chol64_warp(a, &bad);
  } else {
    chol64_cta(a, &bad);
  }
  __syncthreads();
  if (tid == 0 && bad) atomicCAS(err, 0, k + 1);
  inv64_blocks<T>(a, inv, rd);
  T* Li = Linv + s.linv + (int64_t)b * NB * NB;
  for (int t = tid; t < NB * NB; t += blockDim.x) {
    int i = t % NB, j = t / NB;
    A[i + (int64_t)s.n * j] = (i >= j) ? a[i][j] : (T)0;
    Li[i + NB * j] = inv[i][j];
  }
}

// four consecutive entries of a shared-memory row (16-byte aligned)
__device__ __forceinline__ void lds4(const float* p, float v[4]) {
  const float4 w = *reinterpret_cast<const float4*>(p);
  v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
}
__device__ __forceinline__ void lds4(const double* p, double v[4]) {
  const double2 w0 = *reinterpret_cast<const double2*>(p), w1 = *reinterpret_cast<const double2*>(p + 2);
  v[0] = w0.x; v[1] = w0.y; v[2] = w1.x; v[3] = w1.y;
}

template <typename T>
__global__ void __launch_bounds__(256) k_trsm_panel(const SubDev* sd, T* L, const T* Linv, int b,
                                                    const int2* items) {
  // items: (subdomain, block row) of the nonzero tiles, else every tile below b
  const int k = items ? items[blockIdx.x].x : (int)blockIdx.y;
  const int r = items ? items[blockIdx.x].y : b + 1 + (int)blockIdx.x;
  const SubDev s = sd[k];
  if (r >= s.nblk) return;
  // the tile and the inverse of the diagonal block, both transposed in shared
  // memory (rows of 64 + 4 entries, 16-byte aligned), so that a thread reads
  // its four rows and its four columns with one vector load each
  constexpr int LD = NB + 4;
  __shared__ __align__(16) T At[NB][LD];    // At[l][i] = A[i][l]
  __shared__ __align__(16) T LiT[NB][LD];   // LiT[l][j] = Linv[j][l]
  const int tid = threadIdx.x;
  T* Ab = L + s.A + (int64_t)r * NB + (int64_t)s.n * b * NB;
  const T* Lb = Linv + s.linv + (int64_t)b * NB * NB;
  for (int t = tid; t < NB * NB; t += blockDim.x) {
    const int i = t % NB, l = t / NB;
    At[l][i] = Ab[i + (int64_t)s.n * l];
    LiT[l][i] = Lb[i + NB * l];
  }
  __syncthreads();
  // X = A Linv^T: X[i][j] = sum_l A[i][l] Linv[j][l]; rows 4 ti .., columns 4 tj ..
  const int ti = tid % 16, tj = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0;
#pragma unroll 8
  for (int l = 0; l < NB; ++l) {
    T a[4], y[4];
    lds4(&At[l][4 * ti], a);
    lds4(&LiT[l][4 * tj], y);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * y[v];
  }
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) Ab[4 * ti + u + (int64_t)s.n * (4 * tj + v)] = acc[u][v];
}

template <typename T>
__global__ void __launch_bounds__(256) k_syrk(const SubDev* sd, T* L, int b, const int4* items) {
  // items: (subdomain, block row, block column) of the tiles to update, else
  // every tile of the trailing lower triangle
  int k, r, c;
  if (items) {
    const int4 it = items[blockIdx.x];
    k = it.x;
    r = it.y;
    c = it.z;
  } else {
    k = blockIdx.y;
    // triangular decode of the tile index: rr >= cc
    const int t = blockIdx.x;
    int rr = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while (rr * (rr + 1) / 2 > t) --rr;
    while ((rr + 1) * (rr + 2) / 2 <= t) ++rr;
    const int cc = t - rr * (rr + 1) / 2;
    if (rr >= sd[k].nblk - b - 1) return;
    r = b + 1 + rr;
    c = b + 1 + cc;
  }
  const SubDev s = sd[k];
  // panels stored transposed (Lr[l][i] = L[r-block row i, panel column l]) with
  // 16-byte aligned rows, so a thread reads its 4 rows / 4 columns as vectors
  constexpr int LDS = NB + 16 / (int)sizeof(T);
  __shared__ __align__(16) T Lr[NB][LDS];
  __shared__ __align__(16) T Lc[NB][LDS];
  const int tid = threadIdx.x;
  const T* Pr = L + s.A + (int64_t)r * NB + (int64_t)s.n * b * NB;
  const T* Pc = L + s.A + (int64_t)c * NB + (int64_t)s.n * b * NB;
  for (int x = tid; x < NB * NB; x += blockDim.x) {
    int i = x % NB, j = x / NB;
    Lr[j][i] = Pr[i + (int64_t)s.n * j];
    Lc[j][i] = Pc[i + (int64_t)s.n * j];
  }
  __syncthreads();
  const int ti = tid % 16, tj = tid / 16;   // rows 4ti..4ti+3, columns 4tj..4tj+3
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0;
#pragma unroll 8
  for (int l = 0; l < NB; ++l) {
    T x[4], y[4];
    if constexpr (sizeof(T) == 4) {
      float4 xv = *reinterpret_cast<const float4*>(&Lr[l][4 * ti]);
      float4 yv = *reinterpret_cast<const float4*>(&Lc[l][4 * tj]);
      x[0] = xv.x; x[1] = xv.y; x[2] = xv.z; x[3] = xv.w;
      y[0] = yv.x; y[1] = yv.y; y[2] = yv.z; y[3] = yv.w;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x[u] = Lr[l][4 * ti + u];
        y[u] = Lc[l][4 * tj + u];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += x[u] * y[v];
  }
  T* Out = L + s.A + (int64_t)r * NB + (int64_t)s.n * c * NB;
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int i = 4 * ti + u, j = 4 * tj + v;
      Out[i + (int64_t)s.n * j] -= acc[u][v];
    }
}

// FP32 trailing update on 128 x 128 tiles with the kb panels b .. b+kb-1
// (K = 64 kb): the tile covers block rows r0, r0+1 and block columns c0, c0+1
// of the trailing matrix (pairs counted from b+kb); 256 threads with 8 x 8
// outputs each, each 64-wide panel chunk staged transposed in shared memory in
// turn. Sub-blocks above the block diagonal are skipped. With col_only the
// update covers block column b+kb alone (one tile column, blockIdx.x = R).
constexpr int S2_LDS = 128 + 4;
constexpr int S2_SMEM = 2 * NB * S2_LDS * 4;
constexpr int S2_THREADS = 128;   // 8 x 16 outputs per thread

// 16-byte global -> shared copy that bypasses registers; valid == false
// writes zeros (no bytes are read from src)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  const int bytes = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(bytes) : "memory");
}

// one pair tile (R, C) of subdomain s (pairs counted from b+kb); returns with
// the block-uniform early exits before its first barrier
__device__ __forceinline__ void syrk2_tile(const SubDev& s, float* L, int b, int kb, int col_only, int R, int C,
                                           float* s2) {
  const int t0 = b + kb;          // first trailing block
  const int Tk = s.nblk - t0;
  if (Tk <= 0) return;
  const int Tt = (Tk + 1) / 2;   // block pairs
  if (R >= Tt) return;
  const int r0 = t0 + 2 * R, c0 = t0 + 2 * C;
  const int nr = min(2, s.nblk - r0), nc = col_only ? 1 : min(2, s.nblk - c0);   // blocks present (1 or 2)
  const int tid = threadIdx.x;
  const int64_t n = s.n;
  // rows 8 ti .. 8 ti + 7, columns 16 tj .. 16 tj + 15: 8 x 16 outputs per
  // thread, so that each operand loaded from shared memory feeds more products
  const int ti = tid % 16, tj = tid / 16;
  const int rb = r0 + (8 * ti) / NB, cb = c0 + (16 * tj) / NB;
  const bool writes = (8 * ti) / NB < nr && (16 * tj) / NB < nc && rb >= cb;
  float* Out = L + s.A + (int64_t)r0 * NB + 8 * ti + n * ((int64_t)c0 * NB + 16 * tj);
  float acc[8][16];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 16; ++v) acc[u][v] = 0.f;
  // the panels in pieces of S2_K columns, double buffered: the copies of piece
  // h + 1 are in flight while piece h is multiplied (two buffers of the row and
  // column panels, transposed, in the same shared memory as one 64-wide chunk)
  constexpr int S2_K = NB / 2;
  auto stage = [&](int h) {
    float(*Pr)[S2_LDS] = reinterpret_cast<float(*)[S2_LDS]>(s2 + (h & 1) * 2 * S2_K * S2_LDS);
    float(*Pc)[S2_LDS] = reinterpret_cast<float(*)[S2_LDS]>(s2 + (h & 1) * 2 * S2_K * S2_LDS + S2_K * S2_LDS);
    const float* P = L + s.A + n * ((int64_t)(b + h / 2) * NB + (h % 2) * S2_K);
    // 4 consecutive rows per 16-byte asynchronous copy (zero filled past the
    // blocks present)
#pragma unroll
    for (int q = 0; q < 1024 / S2_THREADS; ++q) {
      const int x = tid + S2_THREADS * q;           // 1024 vectors of 4 rows: i4 = x % 32, l = x / 32
      const int i = 4 * (x % 32), l = x / 32;
      const bool vr = i < nr * NB, vc = i < nc * NB;
      cp_async16(&Pr[l][i], vr ? P + (int64_t)r0 * NB + i + n * l : P, vr);
      cp_async16(&Pc[l][i], vc ? P + (int64_t)c0 * NB + i + n * l : P, vc);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  const int npieces = 2 * kb;
  stage(0);
  for (int h = 0; h < npieces; ++h) {
    if (h + 1 < npieces) {
      stage(h + 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();   // piece h is in shared memory for every thread
    const float(*Pr)[S2_LDS] = reinterpret_cast<const float(*)[S2_LDS]>(s2 + (h & 1) * 2 * S2_K * S2_LDS);
    const float(*Pc)[S2_LDS] =
        reinterpret_cast<const float(*)[S2_LDS]>(s2 + (h & 1) * 2 * S2_K * S2_LDS + S2_K * S2_LDS);
#pragma unroll 4
    for (int l = 0; l < S2_K; ++l) {
      const float4 x0 = *reinterpret_cast<const float4*>(&Pr[l][8 * ti]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Pr[l][8 * ti + 4]);
      const float4 y0 = *reinterpret_cast<const float4*>(&Pc[l][16 * tj]);
      const float4 y1 = *reinterpret_cast<const float4*>(&Pc[l][16 * tj + 4]);
      const float4 y2 = *reinterpret_cast<const float4*>(&Pc[l][16 * tj + 8]);
      const float4 y3 = *reinterpret_cast<const float4*>(&Pc[l][16 * tj + 12]);
      const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      const float y[16] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w,
                           y2.x, y2.y, y2.z, y2.w, y3.x, y3.y, y3.z, y3.w};
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 16; ++v) acc[u][v] = fmaf(x[u], y[v], acc[u][v]);
    }
    __syncthreads();   // every thread is done with buffer h & 1 before piece h + 2 is copied into it
  }
  if (!writes) return;   // beyond the trailing matrix or above the block diagonal
  // the C tile in two halves of 8 columns, each half's loads in flight together
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    float4 cv[16];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const float4* o = reinterpret_cast<const float4*>(Out + n * (8 * hh + v));
      cv[2 * v] = o[0];
      cv[2 * v + 1] = o[1];
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      float4* o = reinterpret_cast<float4*>(Out + n * (8 * hh + v));
      float4 a = cv[2 * v], c = cv[2 * v + 1];
      const int w = 8 * hh + v;
      a.x -= acc[0][w]; a.y -= acc[1][w]; a.z -= acc[2][w]; a.w -= acc[3][w];
      c.x -= acc[4][w]; c.y -= acc[5][w]; c.z -= acc[6][w]; c.w -= acc[7][w];
      o[0] = a;
      o[1] = c;
    }
  }
}

// items: (subdomain, R, C) of the nitems pair tiles to update, each CTA taking
// every gridDim.x-th (a grid smaller than nitems leaves SMs to other kernels);
// without items every pair tile, one per CTA (subdomain blockIdx.y)
__global__ void __launch_bounds__(S2_THREADS, 2) k_syrk2(const SubDev* sd, float* L, int b, int kb, int col_only,
                                                 const int4* items, int nitems) {
  extern __shared__ __align__(16) float s2[];
  if (items) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
      if (it != (int)blockIdx.x) __syncthreads();   // the previous tile's shared panels are no longer read
      const int4 w = items[it];
      syrk2_tile(sd[w.x], L, b, kb, col_only, w.y, w.z, s2);
    }
    return;
  }
  int R, C;
  if (col_only) {
    R = blockIdx.x;
    C = 0;
  } else {
    // triangular decode of the pair-tile index: R >= C
    const int t = blockIdx.x;
    R = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while (R * (R + 1) / 2 > t) --R;
    while ((R + 1) * (R + 2) / 2 <= t) ++R;
    C = t - R * (R + 1) / 2;
  }
  syrk2_tile(sd[blockIdx.y], L, b, kb, col_only, R, C, s2);
}

// S_rIrI snapshot: symmetrised copy of the lower trailing block at the r_I panel
template <typename T>
__global__ void k_snapshot(const SubDev* sd, const T* L, T* S, int b) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  if (s.nVp != b * NB || s.nI == 0) return;
  const int64_t tot = (int64_t)s.ldI * s.nI;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t % s.ldI), j = (int)(t / s.ldI);
    if (i >= s.nI) {
      S[s.S + t] = (T)0;
      continue;
    }
    int hi = i > j ? i : j, lo = i > j ? j : i;
    S[s.S + t] = L[s.A + (s.nVp + hi) + (int64_t)s.n * (s.nVp + lo)];
  }
}

// ---------------------------------------------------------------------------
// triangular solves L Y = B (forward) and L^T X = Y (backward) on a panel range
// ---------------------------------------------------------------------------

// Many right-hand sides (W = S_rIrI^-1 from identity columns, Phi from K_rp):
// blocked substitution whose work is 64 x 64 x 64 tile products. Forward,
// panel b: Y_b = Linv_b B_b, then B_below -= L_below,b Y_b. Backward, panel b:
// X_b = Linv_b^T Y_b, then Y_above -= L_b,above^T X_b. One CTA per 64 x 64 output
// tile, 4 x 4 outputs per thread from shared-memory copies of both operands.

constexpr int BWD_COLS = 64;    // single-column backward: rows above the panel per CTA

// C(i, j) = (or -=) sum_l P(i, l) Q(l, j) on one 64 x 64 tile with K = 64;
// P(i, l) = P[i pi + l pl], Q(l, j) = Q[l ql + j qj], C(i, j) = C[i + j ldc];
// rows i >= mi and columns j >= nj are not touched (their operands read as 0)
template <typename T, bool SUB>
__device__ __forceinline__ void tile_gemm64(const T* P, int64_t pi, int64_t pl, int mi, const T* Q, int64_t ql,
                                            int64_t qj, int nj, T* C, int64_t ldc) {
  constexpr int LDS = NB + 16 / (int)sizeof(T);
  __shared__ __align__(16) T Ps[NB][LDS];
  __shared__ __align__(16) T Qs[NB][LDS];
  const int tid = threadIdx.x;
  // the index with unit stride runs fastest over the threads (coalesced loads)
  const bool p_i_fast = pi == 1, q_l_fast = ql == 1;
  for (int x = tid; x < NB * NB; x += blockDim.x) {
    const int i = p_i_fast ? x % NB : x / NB, l = p_i_fast ? x / NB : x % NB;
    Ps[l][i] = i < mi ? P[i * pi + l * pl] : (T)0;
    const int lq = q_l_fast ? x % NB : x / NB, j = q_l_fast ? x / NB : x % NB;
    Qs[lq][j] = j < nj ? Q[lq * ql + j * qj] : (T)0;
  }
  __syncthreads();
  const int ti = tid % 16, tj = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0;
#pragma unroll 8
  for (int l = 0; l < NB; ++l) {
    T x[4], y[4];
    if constexpr (sizeof(T) == 4) {
      const float4 xv = *reinterpret_cast<const float4*>(&Ps[l][4 * ti]);
      const float4 yv = *reinterpret_cast<const float4*>(&Qs[l][4 * tj]);
      x[0] = xv.x; x[1] = xv.y; x[2] = xv.z; x[3] = xv.w;
      y[0] = yv.x; y[1] = yv.y; y[2] = yv.z; y[3] = yv.w;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x[u] = Ps[l][4 * ti + u];
        y[u] = Qs[l][4 * tj + u];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += x[u] * y[v];
  }
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = 4 * ti + u, j = 4 * tj + v;
      if (i < mi && j < nj) {
        if (SUB) C[i + j * ldc] -= acc[u][v];
        else C[i + j * ldc] = acc[u][v];
      }
    }
}

// diagonal block of panel b for column tile blockIdx.x: Dst_b = Linv_b Src_b
// (forward) or Linv_b^T Src_b (backward)
template <typename T, bool TRANS>
__global__ void __launch_bounds__(256) k_tsolve_diag(const SubDev* sd, const SolveDesc* dsc, const T* Linv,
                                                     const T* Src, T* Dst, int b) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  const SolveDesc d = dsc[k];
  if (b < d.b0 || b >= s.nblk || d.ncol == 0) return;
  const int j0 = blockIdx.x * NB;
  if (j0 >= d.ncol) return;
  const int row0 = (b - d.b0) * NB;
  const T* Lb = Linv + s.linv + (int64_t)b * NB * NB;
  const int64_t o = d.boff + row0 + (int64_t)d.ldb * j0;
  if (TRANS) tile_gemm64<T, false>(Lb, NB, 1, NB, Src + o, 1, d.ldb, min(NB, d.ncol - j0), Dst + o, d.ldb);
  else tile_gemm64<T, false>(Lb, 1, NB, NB, Src + o, 1, d.ldb, min(NB, d.ncol - j0), Dst + o, d.ldb);
}

// forward update of panel b: B[rows below] -= L[rows below, panel b] Y_b
template <typename T>
__global__ void __launch_bounds__(256) k_tsolve_fwd(const SubDev* sd, const SolveDesc* dsc, const T* L, T* B,
                                                    const T* Y, int b, const unsigned char* lf, const int64_t* lfo) {
  const int k = blockIdx.z;
  const SubDev s = sd[k];
  const SolveDesc d = dsc[k];
  if (b < d.b0 || b >= s.nblk || d.ncol == 0) return;
  const int j0 = blockIdx.y * NB;
  if (j0 >= d.ncol) return;
  const int row0 = (b - d.b0) * NB, rows = s.n - d.b0 * NB;
  const int r0 = row0 + NB + blockIdx.x * NB;
  if (r0 >= rows) return;
  if (lf && !lf[lfo[k] + d.b0 + r0 / NB + (int64_t)s.nblk * b]) return;   // zero tile of the factor
  const T* P = L + s.A + (d.b0 * NB + r0) + (int64_t)s.n * (b * NB);
  tile_gemm64<T, true>(P, 1, s.n, min(NB, rows - r0), Y + d.boff + row0 + (int64_t)d.ldb * j0, 1, d.ldb,
                       min(NB, d.ncol - j0), B + d.boff + r0 + (int64_t)d.ldb * j0, d.ldb);
}

// backward update of panel b: Y[rows above] -= L[panel b, rows above]^T X_b
template <typename T>
__global__ void __launch_bounds__(256) k_tsolve_bwd(const SubDev* sd, const SolveDesc* dsc, const T* L, T* Y,
                                                    const T* X, int b, const unsigned char* lf, const int64_t* lfo) {
  const int k = blockIdx.z;
  const SubDev s = sd[k];
  const SolveDesc d = dsc[k];
  if (b < d.b0 || b >= s.nblk || d.ncol == 0) return;
  const int j0 = blockIdx.y * NB;
  if (j0 >= d.ncol) return;
  const int row0 = (b - d.b0) * NB;
  const int a0 = blockIdx.x * NB;
  if (a0 >= row0) return;
  if (lf && !lf[lfo[k] + b + (int64_t)s.nblk * (d.b0 + a0 / NB)]) return;   // zero tile of the factor
  // P(i, l) = L[b NB + l, d.b0 NB + a0 + i]
  const T* P = L + s.A + (int64_t)b * NB + (int64_t)s.n * (d.b0 * NB + a0);
  tile_gemm64<T, true>(P, s.n, 1, min(NB, row0 - a0), X + d.boff + row0 + (int64_t)d.ldb * j0, 1, d.ldb,
                       min(NB, d.ncol - j0), Y + d.boff + a0 + (int64_t)d.ldb * j0, d.ldb);
}

// Single right-hand side: the diagonal solve reads the stored block inverse
// directly (coalesced, no shared-memory staging) and the update of the rows
// below spreads each row's 64-term dot product over 4 threads, so a launch has
// 4x more CTAs in flight for the same rows.
constexpr int FWD1_ROWS = 64;

template <typename T>
__global__ void __launch_bounds__(256) k_fwd1(const SubDev* sd, const SolveDesc* dsc, const T* L, const T* Linv,
                                              T* B, T* Y, int b) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  const SolveDesc d = dsc[k];
  if (b < d.b0 || b >= s.nblk || d.ncol == 0) return;
  const int row0 = (b - d.b0) * NB;
  const int rows = s.n - d.b0 * NB;
  const int rbeg = row0 + NB + blockIdx.x * FWD1_ROWS;
  if (blockIdx.x != 0 && rbeg >= rows) return;
  __shared__ T y[NB], bb[NB];
  const int tid = threadIdx.x;
  T* Bk = B + d.boff;
  if (tid < NB) bb[tid] = Bk[row0 + tid];
  __syncthreads();
  {
    // y_i = sum_{l <= i} Linv[i][l] b_l: 4 threads per row i, 16 terms each
    const T* Lb = Linv + s.linv + (int64_t)b * NB * NB;
    const int i = tid / 4, part = tid % 4;
    T acc = 0;
#pragma unroll
    for (int l = part * 16; l < part * 16 + 16; ++l) acc += Lb[i + NB * l] * bb[l];   // Linv[i][l] = 0 for l > i
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (part == 0) {
      y[i] = acc;
      if (blockIdx.x == 0) Y[d.boff + row0 + i] = acc;
    }
  }
  __syncthreads();
  const int r = rbeg + tid / 4, part = tid % 4;
  T acc = 0;
  if (r < rows) {
    const T* Lrow = L + s.A + (d.b0 * NB + r) + (int64_t)s.n * (b * NB + part * 16);
#pragma unroll
    for (int l = 0; l < 16; ++l) acc += Lrow[(int64_t)s.n * l] * y[part * 16 + l];
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  if (r < rows && part == 0) Bk[r] -= acc;
}

template <typename T>
__global__ void __launch_bounds__(256) k_bwd1(const SubDev* sd, const SolveDesc* dsc, const T* L, const T* Linv,
                                              T* Y, T* X, int b) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  const SolveDesc d = dsc[k];
  if (b < d.b0 || b >= s.nblk || d.ncol == 0) return;
  const int row0 = (b - d.b0) * NB;
  if (blockIdx.x != 0 && blockIdx.x * BWD_COLS >= row0) return;
  __shared__ T x[NB];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  T* Yk = Y + d.boff;
  {
    // x_i = sum_{l >= i} Linv[l][i] y_l: warp w computes x_i for i = w, w+8, ...
    const T* Lb = Linv + s.linv + (int64_t)b * NB * NB;
    const T y0 = Yk[row0 + lane], y1 = Yk[row0 + lane + 32];
#pragma unroll
    for (int i = warp; i < NB; i += 8) {
      T v = (lane >= i ? Lb[lane + NB * i] * y0 : (T)0) + (lane + 32 >= i ? Lb[lane + 32 + NB * i] * y1 : (T)0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) x[i] = v;
    }
  }
  __syncthreads();
  if (blockIdx.x == 0 && tid < NB) X[d.boff + row0 + tid] = x[tid];
  for (int w = warp; w < BWD_COLS; w += 8) {
    const int ccol = blockIdx.x * BWD_COLS + w;
    if (ccol >= row0) break;
    const T* Lc = L + s.A + (int64_t)b * NB + (int64_t)s.n * (d.b0 * NB + ccol);
    T v = Lc[lane] * x[lane] + Lc[lane + 32] * x[lane + 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) Yk[ccol] -= v;
  }
}

template <typename T>
ieti_status tri_solve(Ctx* c, const SubDev* d_sd, int nsub, int max_nblk, int max_rows, int max_ncol,
                      const SolveDesc* d_desc, int min_b0, const T* L, const T* Linv, T* B, T* Y, T* X,
                      cudaStream_t st, int which = SWEEP_BOTH, const unsigned char* lf = nullptr,
                      const int64_t* lfo = nullptr) {
  if (max_ncol <= 0) return IETI_OK;
  const bool one = max_ncol == 1;   // single right-hand side: one-column kernels
  const unsigned ctiles = (unsigned)ceil_div(max_ncol, NB);
  const unsigned rtiles = (unsigned)std::max<int64_t>(1, ceil_div(max_rows, NB));
  cudaEvent_t p0 = prof_begin(c, st);
  for (int b = min_b0; (which & SWEEP_FWD) && b < max_nblk; ++b) {
    if (one) {
      k_fwd1<T><<<dim3((unsigned)std::max<int64_t>(1, ceil_div(max_rows, FWD1_ROWS)), nsub), 256, 0, st>>>(
          d_sd, d_desc, L, Linv, B, Y, b);
      IETI_LAUNCH_CHECK(c);
    } else {
      k_tsolve_diag<T, false><<<dim3(ctiles, nsub), 256, 0, st>>>(d_sd, d_desc, Linv, B, Y, b);
      IETI_LAUNCH_CHECK(c);
      k_tsolve_fwd<T><<<dim3(rtiles, ctiles, nsub), 256, 0, st>>>(d_sd, d_desc, L, B, Y, b, lf, lfo);
      IETI_LAUNCH_CHECK(c);
    }
  }
  prof_end(c, PROF_FWD, p0, st);
  p0 = prof_begin(c, st);
  for (int b = max_nblk - 1; (which & SWEEP_BWD) && b >= min_b0; --b) {
    if (one) {
      k_bwd1<T><<<dim3((unsigned)std::max<int64_t>(1, ceil_div(max_rows, BWD_COLS)), nsub), 256, 0, st>>>(
          d_sd, d_desc, L, Linv, Y, X, b);
      IETI_LAUNCH_CHECK(c);
    } else {
      k_tsolve_diag<T, true><<<dim3(ctiles, nsub), 256, 0, st>>>(d_sd, d_desc, Linv, Y, X, b);
      IETI_LAUNCH_CHECK(c);
      k_tsolve_bwd<T><<<dim3(rtiles, ctiles, nsub), 256, 0, st>>>(d_sd, d_desc, L, Y, X, b, lf, lfo);
      IETI_LAUNCH_CHECK(c);
    }
  }
  prof_end(c, PROF_BWD, p0, st);
  return IETI_OK;
}

// ---------------------------------------------------------------------------
// helpers for the derived operators
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_identity_rhs(const SubDev* sd, const SolveDesc* dsc, T* B) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  const SolveDesc d = dsc[k];
  const int64_t tot = (int64_t)d.ldb * d.ncol;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t % d.ldb), j = (int)(t / d.ldb);
    B[d.boff + t] = (i == j) ? (T)1 : (T)0;
  }
  (void)s;
}

template <typename T>
__global__ void k_extract_W(const SubDev* sd, const SolveDesc* dsc, const T* X, T* W) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  const SolveDesc d = dsc[k];
  const int64_t tot = (int64_t)s.ldI * s.nI;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t % s.ldI), j = (int)(t / s.ldI);
    if (i >= s.nI) {
      W[s.S + t] = (T)0;
      continue;
    }
    // symmetrise (the two triangles agree up to rounding)
    T a = X[d.boff + i + (int64_t)d.ldb * j], bb = X[d.boff + j + (int64_t)d.ldb * i];
    W[s.S + t] = (T)0.5 * (a + bb);
  }
}

// B (n x nP, type T) <- K_rp
template <typename T>
__global__ void k_load_Kp(const SubDev* sd, const SolveDesc* dsc, const double* Kp, T* B) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  const SolveDesc d = dsc[k];
  const int64_t tot = (int64_t)s.n * s.nP;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    B[d.boff + t] = (T)Kp[s.Kp + t];
}

template <typename T>
__global__ void k_store_Phi(const SubDev* sd, const SolveDesc* dsc, const T* X, double* Phi) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  const SolveDesc d = dsc[k];
  const int64_t tot = (int64_t)s.n * s.nP;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    Phi[s.Kp + t] = (double)X[d.boff + t];
}

// Psi = L^-1 K_rp (the forward sweep of the Phi solve), kept in the factor
// precision for the recovery of the local field
template <typename T>
__global__ void k_store_Psi(const SubDev* sd, const SolveDesc* dsc, const T* Y, T* Psi) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  const SolveDesc d = dsc[k];
  const int64_t tot = (int64_t)s.n * s.nP;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    Psi[s.Kp + t] = Y[d.boff + t];
}

// S_Pi += C^T (K_pp - K_rp^T Phi) C, one CTA per subdomain, FP64
__global__ void k_coarse_assemble(const SubDev* sd, const double* Kp, const double* Kpp, const double* Phi,
                                  const int32_t* P_glob, double* SPi, int ldc) {
  const int k = blockIdx.x;
  const SubDev s = sd[k];
  const int np = s.nP;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int t = warp; t < np * np; t += nw) {
    int i = t % np, j = t / np;
    const double* a = Kp + s.Kp + (int64_t)s.n * i;
    const double* ph = Phi + s.Kp + (int64_t)s.n * j;
    double acc = 0;
    for (int r = lane; r < s.n; r += 32) acc += a[r] * ph[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      double v = Kpp[s.Kpp + i + (int64_t)np * j] - acc;
      int gi = P_glob[s.pv + i], gj = P_glob[s.pv + j];
      atomicAdd(SPi + gi + (int64_t)ldc * gj, v);
    }
  }
}

__global__ void k_pad_identity(double* A, int n0, int ld) {
  for (int i = n0 + blockIdx.x * blockDim.x + threadIdx.x; i < ld; i += gridDim.x * blockDim.x)
    A[i + (int64_t)ld * i] = 1.0;
}

// ---------------------------------------------------------------------------

ieti_status factor_kernel_attrs(Ctx* c) {
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_syrk2, cudaFuncAttributeMaxDynamicSharedMemorySize, S2_SMEM));
  return IETI_OK;
}

template <typename T>
static ieti_status cholesky(Ctx* c, const SubDev* d_sd, const std::vector<SubDev>& sdh, T* L, T* Linv,
                            T* S, bool snapshot, cudaStream_t st, const FactorPlan* plan = nullptr) {
  int nsub = (int)sdh.size();
  int max_nblk = 0;
  for (auto& s : sdh) max_nblk = std::max(max_nblk, s.nblk);
  auto snap_at = [&](int b) {
    bool any = false;
    for (auto& s : sdh) any |= (s.nVp == b * NB && s.nI > 0);
    return snapshot && any;
  };
  // diagonal block b and the panel below it (the nonzero tiles only with a plan)
  auto panel = [&](int b, const int2* items, int cnt) -> ieti_status {
    cudaEvent_t p0 = prof_begin(c, st);
    k_potrf_diag<T><<<nsub, 256, 0, st>>>(d_sd, L, Linv, b, c->d_err);
    prof_end(c, PROF_POTRF, p0, st);
    IETI_LAUNCH_CHECK(c);
    const int Tm = max_nblk - b - 1;
    if (items ? cnt > 0 : Tm > 0) {
      p0 = prof_begin(c, st);
      if (items) k_trsm_panel<T><<<cnt, 256, 0, st>>>(d_sd, L, Linv, b, items);
      else k_trsm_panel<T><<<dim3(Tm, nsub), 256, 0, st>>>(d_sd, L, Linv, b, nullptr);
      prof_end(c, PROF_TRSM, p0, st);
      IETI_LAUNCH_CHECK(c);
    }
    return IETI_OK;
  };
  const size_t nsteps = plan ? plan->steps.size() : 0;
  // lookahead: with a plan, a step's trailing update is split into the tiles
  // of the next panels (on st, so the next panel work follows them directly)
  // and the rest (on a low-priority second stream, overlapping the next panel
  // work, which touches other tiles); the next trailing update and any
  // snapshot wait for that rest
  const bool ahead = plan && !c->syrk_tc && nsteps > 1;
  if (ahead && !c->aux_stream) {
    int lo = 0, hi = 0;
    IETI_CUDA_TRY(c, cudaDeviceGetStreamPriorityRange(&lo, &hi));
    IETI_CUDA_TRY(c, cudaStreamCreateWithPriority(&c->aux_stream, cudaStreamNonBlocking, lo));
    for (cudaEvent_t& e : c->ev_fact) IETI_CUDA_TRY(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  bool rest_pending = false;
  auto wait_rest = [&]() -> ieti_status {
    if (rest_pending) IETI_CUDA_TRY(c, cudaStreamWaitEvent(st, c->ev_fact[1], 0));
    rest_pending = false;
    return IETI_OK;
  };
  for (int b = 0, si = 0; plan ? si < (int)nsteps : b < max_nblk; ++si) {
    FactorStep stp{};
    if (plan) {
      stp = plan->steps[si];
      b = stp.b;
    } else {
      // FP32: two panels per trailing update (K = 128 halves the passes over
      // the trailing matrix), unless the S_rIrI snapshot falls between them
      stp.b = b;
      stp.kb = 1;
      if constexpr (sizeof(T) == 4) stp.kb = (!c->syrk_tc && b + 2 < max_nblk && !snap_at(b + 1)) ? 2 : 1;
    }
    if (snap_at(b)) {
      ieti_status rw = wait_rest();
      if (rw != IETI_OK) return rw;
      k_snapshot<T><<<dim3(256, nsub), 256, 0, st>>>(d_sd, L, S, b);
      IETI_LAUNCH_CHECK(c);
    }
    const int kb = stp.kb;
    ieti_status r;
    if ((r = panel(b, plan ? plan->d_trsm + stp.trsm_off[0] : nullptr, stp.trsm_cnt[0])) != IETI_OK) return r;
    if (kb == 2) {
      if constexpr (sizeof(T) == 4) {
        // block column b+1 takes panel b's update before its own factorisation
        cudaEvent_t p0 = prof_begin(c, st);
        if (plan) {
          if (stp.col_cnt > 0)
            k_syrk2<<<stp.col_cnt, S2_THREADS, S2_SMEM, st>>>(d_sd, (float*)L, b, 1, 1, plan->d_items + stp.col_off,
                                                         stp.col_cnt);
        } else {
          const int Tp1 = (max_nblk - b - 1 + 1) / 2;
          k_syrk2<<<dim3(Tp1, nsub), S2_THREADS, S2_SMEM, st>>>(d_sd, (float*)L, b, 1, 1, nullptr, 0);
        }
        prof_end(c, PROF_SYRK, p0, st);
        IETI_LAUNCH_CHECK(c);
      }
      if ((r = panel(b + 1, plan ? plan->d_trsm + stp.trsm_off[1] : nullptr, stp.trsm_cnt[1])) != IETI_OK) return r;
    }
    const int Tm = max_nblk - b - kb;
    if ((r = wait_rest()) != IETI_OK) return r;
    if (ahead && stp.trail_cnt > 0) {
      // the next panels' tiles on st, the rest on the second stream
      const int4* items = plan->d_items + stp.trail_off;
      const int n0 = stp.trail_cnt0, n1 = stp.trail_cnt - stp.trail_cnt0;
      cudaEvent_t p0 = prof_begin(c, st);
      if (n0 > 0) {
        if constexpr (sizeof(T) == 4) k_syrk2<<<n0, S2_THREADS, S2_SMEM, st>>>(d_sd, (float*)L, b, kb, 0, items, n0);
        else k_syrk<T><<<n0, 256, 0, st>>>(d_sd, L, b, items);
        IETI_LAUNCH_CHECK(c);
      }
      prof_end(c, PROF_SYRK, p0, st);
      if (n1 > 0) {
        IETI_CUDA_TRY(c, cudaEventRecord(c->ev_fact[0], st));
        IETI_CUDA_TRY(c, cudaStreamWaitEvent(c->aux_stream, c->ev_fact[0], 0));
        cudaEvent_t p1 = prof_begin(c, c->aux_stream);
        // the overlapped rest runs on a grid that leaves SMs free for the
        // next panels' kernels: at two CTAs per SM this kernel holds the whole
        // register file of an SM, so a full grid keeps them waiting for SMs
        if constexpr (sizeof(T) == 4)
          k_syrk2<<<std::min(n1, 2 * std::max(1, c->sm_count - c->syrk_reserve)), S2_THREADS, S2_SMEM, c->aux_stream>>>(
              d_sd, (float*)L, b, kb, 0, items + n0, n1);
        else k_syrk<T><<<n1, 256, 0, c->aux_stream>>>(d_sd, L, b, items + n0);
        prof_end(c, PROF_SYRK, p1, c->aux_stream);
        IETI_LAUNCH_CHECK(c);
        IETI_CUDA_TRY(c, cudaEventRecord(c->ev_fact[1], c->aux_stream));
        rest_pending = true;
      }
    } else if (plan ? stp.trail_cnt > 0 : Tm > 0) {
      cudaEvent_t p0 = prof_begin(c, st);
      const int4* items = plan ? plan->d_items + stp.trail_off : nullptr;
      if constexpr (sizeof(T) == 4) {
        if (c->syrk_tc) {
          // opt-in: split TF32 products on the tensor cores (slower than the
          // CUDA-core kernel at this panel width, see syrk_tc.cu); it updates
          // every trailing tile, which is exact for the zero ones as well
          ieti_status r2 = syrk_tc(c, d_sd, (float*)L, b, max_nblk, nsub, st);
          if (r2 != IETI_OK) return r2;
        } else if (plan) {
          k_syrk2<<<stp.trail_cnt, S2_THREADS, S2_SMEM, st>>>(d_sd, (float*)L, b, kb, 0, items, stp.trail_cnt);
        } else {
          const int Tp = (Tm + 1) / 2;   // block pairs
          k_syrk2<<<dim3(Tp * (Tp + 1) / 2, nsub), S2_THREADS, S2_SMEM, st>>>(d_sd, (float*)L, b, kb, 0, nullptr, 0);
        }
      } else {
        if (plan) k_syrk<T><<<stp.trail_cnt, 256, 0, st>>>(d_sd, L, b, items);
        else k_syrk<T><<<dim3(Tm * (Tm + 1) / 2, nsub), 256, 0, st>>>(d_sd, L, b, nullptr);
      }
      prof_end(c, PROF_SYRK, p0, st);
      IETI_LAUNCH_CHECK(c);
    }
    b += kb;
  }
  return wait_rest();
}

template <typename T>
static ieti_status factor_t(Ctx* c, cudaStream_t st) {
  T* L = (T*)c->L;
  T* Linv = (T*)c->Linv;
  T* S = (T*)c->S;
  T* W = (T*)c->W;
  ieti_status r;
  // work lists over the nonzero tiles, found once from the assembled K_rr
  if (!c->symb_ready && (r = build_symbolic(c, st)) != IETI_OK) return r;
  // factor buffer <- K_rr: in full the first time in this precision (which
  // zeroes the tiles outside the factor's pattern for good: no step changes
  // them), then the pattern's tiles only
  const int pk = sizeof(T) == 4 ? 1 : 0;
  if (c->l_init_prec != pk) {
    if ((r = convert_copy<T>(c, c->K64, L, c->tot_A, st)) != IETI_OK) return r;
    c->l_init_prec = pk;
  } else if ((r = convert_tiles<T>(c, c->d_ltile_list, c->n_ltiles, c->K64, L, st)) != IETI_OK) {
    return r;
  }
  if (c->fault_pivot_sub >= 0 && c->fault_pivot_sub < c->nsub) {
    // testing aid: a negative first diagonal entry, found by the pivot check below
    const T v = (T)-1;
    IETI_CUDA_TRY(c, cudaMemcpyAsync(L + c->sd_host[c->fault_pivot_sub].A, &v, sizeof(T), cudaMemcpyHostToDevice, st));
    IETI_CUDA_TRY(c, cudaStreamSynchronize(st));
  }
  IETI_CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
  IETI_CUDA_TRY(c, cudaMemsetAsync(c->d_dep_err, 0, sizeof(int), st));   // bounded waits of the W and Phi solves
  const FactorPlan* plan = &c->fplan[sizeof(T) == 4 ? 1 : 0];
  if ((r = cholesky<T>(c, c->d_sd, c->sd_host, L, Linv, S, true, st, plan)) != IETI_OK) return r;
  IETI_CUDA_TRY(c, cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  IETI_CUDA_TRY(c, cudaStreamSynchronize(st));
  if (*c->h_err) {
    // the failed factorisation may have written non-finite values into tiles
    // outside the pattern (products with overflowed entries): the next one
    // starts from a full copy of K_rr
    c->l_init_prec = -1;
    c->err = "non-positive pivot in the factorisation of subdomain " + std::to_string(*c->h_err - 1);
    return IETI_ERR_SINGULAR_LOCAL;
  }
  const int nsub = c->nsub;
  T* B = (T*)c->wr[0];
  T* Y = (T*)c->wr[1];
  T* X = (T*)c->wr[2];
  // --- W = S_rIrI^-1 from the trailing factor block (identity right-hand sides)
  {
    std::vector<SolveDesc> dh(nsub);
    int64_t off = 0;
    int min_b0 = 1 << 30, max_rows = 0, max_col = 0;
    for (int k = 0; k < nsub; ++k) {
      const SubDev& s = c->sd_host[k];
      dh[k].boff = off;
      dh[k].b0 = s.nVp / NB;
      dh[k].ldb = s.n - s.nVp;
      dh[k].ncol = s.nI;
      off += (int64_t)dh[k].ldb * dh[k].ncol;
      min_b0 = std::min(min_b0, dh[k].b0);
      max_rows = std::max(max_rows, dh[k].ldb);
      max_col = std::max(max_col, s.nI);
    }
    SolveDesc* dd = (SolveDesc*)c->d_descbuf;   // scratch for descriptors (host-sized)
    IETI_CUDA_TRY(c, cudaMemcpyAsync(dd, dh.data(), sizeof(SolveDesc) * nsub, cudaMemcpyHostToDevice, st));
    k_identity_rhs<T><<<dim3(256, nsub), 256, 0, st>>>(c->d_sd, dd, B);
    IETI_LAUNCH_CHECK(c);
    r = dep_mc_solve<T>(c, 0, dh, dd, SWEEP_BOTH, B, Y, X, st);
    if (r == IETI_ERR_STATE)
      r = tri_solve<T>(c, c->d_sd, nsub, c->max_nblk, max_rows, max_col, dd, min_b0, L, Linv, B, Y, X, st,
                       SWEEP_BOTH, c->d_lflags, c->d_tile_off);
    if (r != IETI_OK) return r;
    k_extract_W<T><<<dim3(256, nsub), 256, 0, st>>>(c->d_sd, dd, X, W);
    IETI_LAUNCH_CHECK(c);
    IETI_CUDA_TRY(c, cudaStreamSynchronize(st));
  }
  // --- Phi = K_rr^-1 K_rp (FP64 storage)
  if (c->max_nP > 0) {
    std::vector<SolveDesc> dh(nsub);
    int64_t off = 0;
    for (int k = 0; k < nsub; ++k) {
      const SubDev& s = c->sd_host[k];
      dh[k].boff = off;
      dh[k].b0 = 0;
      dh[k].ldb = s.n;
      dh[k].ncol = s.nP;
      off += (int64_t)s.n * s.nP;
    }
    SolveDesc* dd = (SolveDesc*)c->d_descbuf;
    IETI_CUDA_TRY(c, cudaMemcpyAsync(dd, dh.data(), sizeof(SolveDesc) * nsub, cudaMemcpyHostToDevice, st));
    k_load_Kp<T><<<dim3(256, nsub), 256, 0, st>>>(c->d_sd, dd, c->Kp64, B);
    IETI_LAUNCH_CHECK(c);
    r = dep_mc_solve<T>(c, 1, dh, dd, SWEEP_FWD, B, Y, X, st);
    if (r == IETI_ERR_STATE)
      r = tri_solve<T>(c, c->d_sd, nsub, c->max_nblk, c->max_n, c->max_nP, dd, 0, L, Linv, B, Y, X, st, SWEEP_FWD,
                       c->d_lflags, c->d_tile_off);
    if (r != IETI_OK) return r;
    k_store_Psi<T><<<dim3(256, nsub), 256, 0, st>>>(c->d_sd, dd, Y, (T*)c->Psi);
    IETI_LAUNCH_CHECK(c);
    r = dep_mc_solve<T>(c, 1, dh, dd, SWEEP_BWD, B, Y, X, st);
    if (r == IETI_ERR_STATE)
      r = tri_solve<T>(c, c->d_sd, nsub, c->max_nblk, c->max_n, c->max_nP, dd, 0, L, Linv, B, Y, X, st, SWEEP_BWD,
                       c->d_lflags, c->d_tile_off);
    if (r != IETI_OK) return r;
    k_store_Phi<T><<<dim3(256, nsub), 256, 0, st>>>(c->d_sd, dd, X, c->Phi);
    IETI_LAUNCH_CHECK(c);
    IETI_CUDA_TRY(c, cudaStreamSynchronize(st));
  }
  IETI_CUDA_TRY(c, cudaMemcpyAsync(c->h_err + 1, c->d_dep_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  IETI_CUDA_TRY(c, cudaStreamSynchronize(st));
  if (c->h_err[1]) {
    c->err = "a wait of the W or Phi solves timed out";
    return IETI_ERR_TIMEOUT;
  }
  return IETI_OK;
}

// coarse S_Pi (always FP64): assemble, factor, explicit inverse
static ieti_status coarse_factor(Ctx* c, cudaStream_t st) {
  const int ngp = (int)c->n_gp;
  if (ngp == 0) return IETI_OK;
  const int ldc = (int)(ceil_div(ngp, NB) * NB);
  IETI_CUDA_TRY(c, cudaMemsetAsync(c->SPi, 0, sizeof(double) * ldc * ldc, st));
  k_coarse_assemble<<<c->nsub, 256, 0, st>>>(c->d_sd, c->Kp64, c->Kpp64, c->Phi, c->d_P_glob,
                                             c->SPi, ldc);
  IETI_LAUNCH_CHECK(c);
  k_pad_identity<<<1, 256, 0, st>>>(c->SPi, ngp, ldc);
  IETI_LAUNCH_CHECK(c);
  // one "subdomain" holding the coarse matrix; its factor lives in SPiInv's second half
  SubDev cs{};
  cs.A = 0;
  cs.n = ldc;
  cs.nblk = ldc / NB;
  cs.nVp = 0;
  cs.nI = 0;
  cs.linv = 0;
  std::vector<SubDev> csh{cs};
  double* Lc = c->SPiInv + (int64_t)ldc * ldc;          // factor
  double* Lci = Lc + (int64_t)ldc * ldc;                 // diagonal-block inverses
  double* Bc = Lci + (int64_t)ldc * NB;
  double* Yc = Bc + (int64_t)ldc * ldc;
  SubDev* d_cs = (SubDev*)(Yc + (int64_t)ldc * ldc);
  SolveDesc* d_desc = (SolveDesc*)(d_cs + 1);
  IETI_CUDA_TRY(c, cudaMemcpyAsync(d_cs, &cs, sizeof(SubDev), cudaMemcpyHostToDevice, st));
  IETI_CUDA_TRY(c, cudaMemcpyAsync(Lc, c->SPi, sizeof(double) * ldc * ldc, cudaMemcpyDeviceToDevice, st));
  IETI_CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
  ieti_status r;
  if ((r = cholesky<double>(c, d_cs, csh, Lc, Lci, nullptr, false, st)) != IETI_OK) return r;
  SolveDesc dh{0, 0, ldc, ldc, 0};
  IETI_CUDA_TRY(c, cudaMemcpyAsync(d_desc, &dh, sizeof(SolveDesc), cudaMemcpyHostToDevice, st));
  k_identity_rhs<double><<<dim3(64, 1), 256, 0, st>>>(d_cs, d_desc, Bc);
  IETI_LAUNCH_CHECK(c);
  if ((r = tri_solve<double>(c, d_cs, 1, cs.nblk, ldc, ldc, d_desc, 0, Lc, Lci, Bc, Yc, c->SPiInv, st)) != IETI_OK)
    return r;
  IETI_CUDA_TRY(c, cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  IETI_CUDA_TRY(c, cudaStreamSynchronize(st));
  if (*c->h_err) {
    c->err = "coarse matrix S_Pi is not positive definite";
    return IETI_ERR_SINGULAR_LOCAL;
  }
  return IETI_OK;
}

ieti_status factor_all(Ctx* c, cudaStream_t st) {
  IETI_CUDA_TRY(c, cudaMemsetAsync(c->d_stream_err, 0, sizeof(int), st));
  ieti_status r = (c->prec == IETI_FP64) ? factor_t<double>(c, st) : factor_t<float>(c, st);
  if (r == IETI_ERR_SINGULAR_LOCAL && c->prec == IETI_FP32_IR && c->fault_pivot_sub < 0) {
    // a non-positive pivot in FP32 (a local block too ill-conditioned for
    // single precision): the factors are redone in FP64
    c->prec = IETI_FP64;
    c->fp64_fallbacks++;
    r = factor_t<double>(c, st);
  }
  if (r != IETI_OK) return r;
  if ((r = coarse_factor(c, st)) != IETI_OK) return r;
  if ((r = iface_prepare(c, st)) != IETI_OK) return r;
  return iface_check(c, st);   // timed-out waits of the tensor-core update
}

// sweeps on nrhs-column r-vectors with the range descriptors built at creation
template <typename T>
ieti_status rv_solve(Ctx* c, int range, int which, T* B, T* Y, T* X, cudaStream_t st) {
  if (c->nrhs == 1) {
    const ieti_status r = dep_sweep<T>(c, range, which, B, Y, X, st);
    if (r != IETI_ERR_STATE) return r;
  }
  const bool irange = range == RV_IRANGE;
  const SolveDesc* dd = c->d_desc_rv + (irange ? c->nsub : 0);
  return tri_solve<T>(c, c->d_sd, c->nsub, c->max_nblk, c->max_n, c->nrhs, dd, irange ? c->min_b0_I : 0,
                      (const T*)c->L, (const T*)c->Linv, B, Y, X, st, which);
}
template ieti_status rv_solve<float>(Ctx*, int, int, float*, float*, float*, cudaStream_t);
template ieti_status rv_solve<double>(Ctx*, int, int, double*, double*, double*, cudaStream_t);

}  // namespace ieti
