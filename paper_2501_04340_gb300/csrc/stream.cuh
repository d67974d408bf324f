// Shared device code of the streamed interface products (bulk async copies
// of whole-row tiles through a ring of shared-memory stages); used by the
// stand-alone products and by the persistent PCG kernel.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "internal.h"

namespace ieti {

constexpr int TILE_TARGET = 64 * 1024;   // bytes per tile at most (whole rows, at most RMAX)
constexpr int RMAX = 8;                  // rows per tile at most (multi-column mode)
constexpr int RROW_MAX = 64;             // rows per tile at most (single-column row mode)
constexpr int MAX_STAGES = 12;
constexpr int NCONS = 256;               // consumer threads (8 warps); one producer warp follows
constexpr int STREAM_THREADS = NCONS + 32;
constexpr int ROW_MAX_ELEMS = 2048;      // row mode: u chunks of a whole row in registers
constexpr int BAR_BYTES = 256;           // mbarriers: full/empty per stage, ufull/uempty x 2; abort flag
constexpr int WIN = 32;                  // tile descriptors per window (two windows in shared memory)

// One tile: nrows whole rows of one subdomain's block, contiguous in memory.
struct LTile {
  int64_t src;      // element offset of the first row in the source buffer
  int64_t obase;    // output block: iv (kind 0) or pv (kind 1) of the subdomain
  int64_t uoff;     // offset of the subdomain's u_k in the u vectors (column 0)
  int k;            // subdomain
  int row0;         // first row (kind 0: row of M_k; kind 1: primal DOF c)
  int nrows;
  int kind;         // 0: rows of M_k -> t, 1: rows of Phi_I^(k)T -> qpart
  int ldI;          // row length (elements)
  int ostride;      // column stride of the output block (nI or nP)
  int bytes;        // nrows * ldI * element size
  int pad_;
};
static_assert(sizeof(LTile) == 56, "tile descriptor layout");

constexpr int WIN_BYTES = 2 * WIN * (int)sizeof(LTile);

// shared-memory header: barriers, two windows of tile descriptors, then the
// partial sums of the tile reduction, [2 buffers][8 warps][RMAX * CT] doubles
__host__ __device__ constexpr int stream_hdr(int ct) {
  return ((BAR_BYTES + WIN_BYTES + 2 * 8 * RMAX * ct * 8) + 127) / 128 * 128;
}

// ---- PTX wrappers: mbarrier and bulk async copy --------------------------------

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(bar))
               : "memory");
}

// the same copy with an L2 eviction priority (a policy from l2_policy)
__device__ __forceinline__ void bulk_load_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                               uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar)), "l"(policy)
      : "memory");
}

// L2 policies: 1 = keep (evict last), 2 = stream through (evict first)
__device__ __forceinline__ uint64_t l2_policy(int hint) {
  uint64_t pol = 0;
  if (hint == 1) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  else if (hint == 2) asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// a tile copy with the stream's L2 priority
__device__ __forceinline__ void tile_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar, int hint,
                                          uint64_t policy) {
  if (hint) bulk_load_hint(dst, src, bytes, bar, policy);
  else bulk_load(dst, src, bytes, bar);
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase with the given parity: gives up after 2^31 SM
// clocks (about one second at 2 GHz)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}

// ---- the streaming loop (shared by the stand-alone products and the
// persistent PCG kernel) ------------------------------------------------------

// The vectors u_k = D_k B_k^T x of all subdomains are prepared beforehand in
// one array (T, column col of subdomain k at col * utot + uoff_k, zero beyond
// nI_k), so that a CTA fetches u_k with bulk copies like the tiles.
struct StreamCtx {
  const void* M;       // rows of M_k (T), row-major with leading dimension ldI
  const void* PhiT;    // rows of Phi_I^(k)T (T), same layout
  const void* uall;    // prepared u vectors (T)
  const LTile* tiles;
  int64_t utot;        // column stride of uall (elements)
  int u_ld, stages, stage_bytes;
  int* err;            // device error word (set on a timed-out wait)
  int l2_hint;         // L2 priority of the tile copies: 0 normal, 1 evict last, 2 evict first
};

__device__ __forceinline__ void consumer_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Sum of V values over the 32 lanes of a warp by halving exchanges: after the
// call lane L holds max(1, V / 32) complete sums v[0..]; their value indices
// are  sum_s ((L >> (4 - s)) & 1) * (V >> (s + 1)) + i  over the first
// min(5, log2 V) steps s (lanes that differ only in the remaining low bits hold
// the same sums).
template <typename T, int V>
__device__ __forceinline__ void warp_transpose_sum(T (&v)[V], int lane) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int o = 16 >> s;
    const int n = V >> s;
    if (n > 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < n / 2; ++i) {
        const T send = up ? v[i] : v[i + n / 2];
        const T keep = up ? v[i + n / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    }
  }
}

template <int V>
__device__ __forceinline__ int transpose_index(int lane, int i) {
  int idx = i;
#pragma unroll
  for (int s = 0; s < 5; ++s)
    if ((V >> s) > 1) idx += ((lane >> (4 - s)) & 1) * (V >> (s + 1));
  return idx;
}

// barrier layout in the header: full[MAX_STAGES], empty[MAX_STAGES], ufull[2],
// uempty[2], abort flag
struct StreamBars {
  uint64_t* full;
  uint64_t* empty;
  uint64_t* ufull;
  uint64_t* uempty;
  volatile int* abort_flag;
  __device__ explicit StreamBars(unsigned char* smem) {
    full = reinterpret_cast<uint64_t*>(smem);
    empty = full + MAX_STAGES;
    ufull = empty + MAX_STAGES;
    uempty = ufull + 2;
    abort_flag = reinterpret_cast<volatile int*>(uempty + 2);
  }
};
static_assert((2 * MAX_STAGES + 4) * 8 + 4 <= BAR_BYTES, "barrier area");

// full: one arrival (the producer's expect_tx) plus the copy's bytes;
// empty: one arrival per consumer warp
__device__ __forceinline__ void stream_init_bars(unsigned char* smem, int stages) {
  StreamBars B(smem);
  if (threadIdx.x == 0) {
    for (int i = 0; i < stages; ++i) {
      mbar_init(&B.full[i], 1);
      mbar_init(&B.empty[i], NCONS / 32);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&B.ufull[i], 1);
      mbar_init(&B.uempty[i], NCONS / 32);
    }
    *B.abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();
}

// Producer warp only: copies the descriptors of the first WIN tiles of
// [tb, te) into window 0 and issues the bulk copies of the first `stages`
// tiles (they do not depend on u), so that a later stream_tiles call with the
// same range, seq and npre = the return value finds them in flight. The
// consumers of the previous range must be done with the window and the
// stages they used (the caller places a barrier in between). Returns the
// number of tiles issued (0 after a timed-out wait, which sets the abort flag).
template <typename T>
__device__ __noinline__ int stream_prefetch(const StreamCtx& C, int tb, int te, unsigned char* smem, uint32_t seq, int ct) {
  const int n = te - tb;
  if (n <= 0) return 0;
  StreamBars B(smem);
  LTile* win = reinterpret_cast<LTile*>(smem + BAR_BYTES);
  const size_t ubytes = ((sizeof(T) * (size_t)C.u_ld * ct + 127) / 128) * 128;
  unsigned char* stage_base = smem + stream_hdr(ct) + 2 * ubytes;
  const int lane = threadIdx.x % 32;
  const uint32_t S = (uint32_t)C.stages;
  if (lane < n && lane < WIN) win[lane] = C.tiles[tb + lane];
  __syncwarp();
  int npre = 0;
  if (lane == 0) {
    const uint64_t pol = l2_policy(C.l2_hint);
    const int want = min(n, (int)S);
    for (int j = 0; j < want && !*B.abort_flag; ++j) {
      const LTile tl = win[j];
      const uint32_t sq = seq + (uint32_t)j;
      const uint32_t st = sq % S, use = sq / S;
      if (use > 0 && !mbar_wait(&B.empty[st], (use - 1) & 1u)) {
        atomicExch(C.err, 1);
        *B.abort_flag = 1;
        break;
      }
      const T* src = (tl.kind ? (const T*)C.PhiT : (const T*)C.M) + tl.src;
      mbar_expect_tx(&B.full[st], (uint32_t)tl.bytes);
      tile_load(stage_base + (size_t)st * C.stage_bytes, src, (uint32_t)tl.bytes, &B.full[st], C.l2_hint, pol);
      npre = j + 1;
    }
  }
  return __shfl_sync(0xffffffffu, npre, 0);
}

// programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start before its predecessor ends; it waits for it here
// before touching the predecessor's output (a no-op for an ordinary launch)
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// lets the successor launch while this kernel finishes
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Producer warp only: waits (bounded) for tiles issued by stream_prefetch that
// will not be consumed (the loop ended), so that no copy is in flight when the
// CTA exits.
__device__ inline void stream_drain(unsigned char* smem, uint32_t seq, int npre, int stages) {
  StreamBars B(smem);
  if (threadIdx.x % 32 == 0)
    for (int j = 0; j < npre; ++j) {
      const uint32_t sq = seq + (uint32_t)j;
      mbar_wait(&B.full[sq % (uint32_t)stages], (sq / (uint32_t)stages) & 1u);
    }
  __syncwarp();
}

// Streams tiles [tb, te) and writes t (kind 0) and qpart (kind 1) for columns
// col0 .. col0+nc-1 of an nrhs-column layout. Called by all STREAM_THREADS
// threads: warps 0-7 consume, warp 8 (lane 0) issues the bulk copies: u_k at
// the first tile of every subdomain (into one of two u buffers), and the tiles
// up to `stages` ahead, each after the empty barrier of its buffer or stage
// reports that the consumers are done with the previous contents. seq and useq
// count the tiles and u vectors this CTA has streamed since the barriers were
// initialised (buffer = count % buffers, phase parity = (count / buffers) & 1);
// every thread advances them by the same amounts. A wait that times out sets
// *err and the CTA's abort flag; after that no further copy is issued,
// consumers skip the work, and the producer waits (bounded) for the copies it
// issued.
//
// Consumer mapping: thread t owns the 16-byte column chunks t, t + 256, ... of
// every row of the tile; it reads its u chunk once per tile and accumulates
// the partial products of all rows (at most RMAX) for all CT columns. The
// partials are summed by a halving exchange within each warp and a fixed-order
// sum over the 8 warps.
//
// With DOT, the consumers also form sum_k u_k . t_k over the rows of M_k that
// this range produces, per column (the CTA's share of an inner product such
// as <p, B W B^T p>), and consumer thread 0 writes it to dot_out[col]
// (dred: 8 CT doubles of shared scratch; zero for an empty range).
// Kept out of line: the persistent PCG kernel calls it for both passes, and
// two inlined copies of the streaming loop left one of them with a far worse
// register allocation (the FP64 W pass ran at half the speed of the S pass).
template <typename T, int CT, bool ROWS = false, bool DOT = false>
__device__ __noinline__ void stream_tiles(const StreamCtx& C, int tb, int te, unsigned char* smem, uint32_t& seq,
                             uint32_t& useq, double* t, double* qpart, int nrhs, int col0, int nc,
                             int npre = 0, double* dot_out = nullptr, double* dred = nullptr) {
  constexpr int VEC = 16 / sizeof(T);
  constexpr int V = RMAX * CT;
  const int n = te - tb;
  if (n <= 0) {
    if (DOT && threadIdx.x < nc) dot_out[threadIdx.x] = 0.0;
    return;
  }
  double dacc[CT];
#pragma unroll
  for (int cc = 0; cc < CT; ++cc) dacc[cc] = 0.0;
  StreamBars B(smem);
  LTile* win = reinterpret_cast<LTile*>(smem + BAR_BYTES);      // [2][WIN]
  double* red = reinterpret_cast<double*>(smem + BAR_BYTES + WIN_BYTES);   // [2][8 warps][V]
  const size_t ubytes = ((sizeof(T) * (size_t)C.u_ld * CT + 127) / 128) * 128;
  unsigned char* ubase = smem + stream_hdr(CT);
  unsigned char* stage_base = ubase + 2 * ubytes;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const uint32_t S = (uint32_t)C.stages;

  uint32_t uq_end;   // useq after this range (the same in every thread unless aborted)
  if (warp == NCONS / 32) {
    // u may have been written by other CTAs (generic proxy) before a grid
    // barrier: order the bulk copies (async proxy) after that view
    asm volatile("fence.proxy.async.global;" ::: "memory");
    // ---- producer warp: every WIN tiles all lanes copy the next WIN
    // descriptors into a shared window (the consumers read them there once the
    // tile has landed); lane 0 waits for free buffers and issues the copies
    uint32_t uq = useq;
    int issued = 0, pk = -1;
    bool stop = false;
    const uint64_t pol = lane == 0 ? l2_policy(C.l2_hint) : 0;
    for (int j = 0; j < n && !stop; ++j) {
      if (j % WIN == 0 && !(j == 0 && npre > 0)) {   // window 0 is filled by stream_prefetch
        const int jj = j + lane;
        if (jj < n) win[((j / WIN) & 1) * WIN + lane] = C.tiles[tb + jj];
        __syncwarp();
      }
      if (lane == 0) {
        const LTile tl = win[((j / WIN) & 1) * WIN + j % WIN];
        if (*B.abort_flag) stop = true;
        if (!stop && tl.k != pk) {
          const uint32_t ub = uq & 1u, use = uq >> 1;
          if (use > 0 && !mbar_wait(&B.uempty[ub], (use - 1) & 1u)) {
            atomicExch(C.err, 1);
            *B.abort_flag = 1;
            stop = true;
          } else {
            const uint32_t rowb = (uint32_t)((size_t)tl.ldI * sizeof(T));
            mbar_expect_tx(&B.ufull[ub], rowb * (uint32_t)nc);
            for (int cc = 0; cc < nc; ++cc)
              bulk_load(ubase + ub * ubytes + (size_t)cc * C.u_ld * sizeof(T),
                        (const T*)C.uall + (int64_t)(col0 + cc) * C.utot + tl.uoff, rowb, &B.ufull[ub]);
            ++uq;
            pk = tl.k;
          }
        }
        if (!stop && j < npre) {
          issued = j + 1;   // copied ahead by stream_prefetch
        } else if (!stop) {
          const uint32_t sq = seq + (uint32_t)j;
          const uint32_t st = sq % S, use = sq / S;
          if (use > 0 && !mbar_wait(&B.empty[st], (use - 1) & 1u)) {
            atomicExch(C.err, 1);
            *B.abort_flag = 1;
            stop = true;
          } else {
            const T* src = (tl.kind ? (const T*)C.PhiT : (const T*)C.M) + tl.src;
            mbar_expect_tx(&B.full[st], (uint32_t)tl.bytes);
            tile_load(stage_base + (size_t)st * C.stage_bytes, src, (uint32_t)tl.bytes, &B.full[st], C.l2_hint,
                      pol);
            issued = j + 1;
          }
        }
      }
      stop = __shfl_sync(0xffffffffu, stop, 0);
    }
    if (lane == 0 && *B.abort_flag) {
      for (int j = max(0, issued - (int)S); j < issued; ++j) {
        const uint32_t sq = seq + (uint32_t)j;
        mbar_wait(&B.full[sq % S], (sq / S) & 1u);
      }
      if (uq > useq) mbar_wait(&B.ufull[(uq - 1) & 1u], ((uq - 1) >> 1) & 1u);
    }
    uq_end = __shfl_sync(0xffffffffu, uq, 0);
  } else if constexpr (ROWS) {
    // ---- consumers, row mode (one column, rows of at most ROW_MAX_ELEMS):
    // each warp reduces whole rows against the 16-byte chunks lane,
    // lane + 32, ... of u, so no cross-warp step is needed. Warp w takes the
    // rows w, w + 8, ... of the CTA's run, whatever the tile boundaries, and
    // issues the shared loads of a group of chunks before their
    // multiply-adds. The u buffer stays in shared memory until the run leaves
    // the subdomain: the inner product reads u at the row from there.
    constexpr int UREG = ROW_MAX_ELEMS / (32 * VEC);
    constexpr int QG = 8;                // chunks per load group
    constexpr int NW = NCONS / 32;
    // FP32: u in registers (64 of them); FP64: u would take 128 registers of
    // the 168 a thread has here, so its chunks are read from shared memory
    // with the rows
    constexpr bool UREGS = VEC == 4;
    static_assert(UREG % QG == 0, "load groups");
    using V4 = typename std::conditional<VEC == 4, float4, double2>::type;
    V4 ur[UREGS ? UREG : 1];
    T dtacc = 0;             // lane 0: this warp's share of the inner product
    const T* us = nullptr;   // the subdomain's u in shared memory
    int curk = -1;
    int rdone = 0;           // rows of this range before the current tile
    uint32_t uq = useq;
    for (int j = 0; j < n; ++j) {
      const uint32_t sq = seq + (uint32_t)j;
      const uint32_t st = sq % S;
      bool ok = !*B.abort_flag;
      if (ok && !mbar_wait(&B.full[st], (sq / S) & 1u)) {
        atomicExch(C.err, 1);
        *B.abort_flag = 1;
        ok = false;
      }
      ok = __all_sync(0xffffffffu, ok);
      const LTile tl = win[((j / WIN) & 1) * WIN + j % WIN];
      const int nv = tl.ldI / VEC;
      if (tl.k != curk) {
        if (curk >= 0) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&B.uempty[(uq - 1) & 1u]);   // done with the previous u
        }
        const uint32_t ub = uq & 1u;
        bool uok = ok && mbar_wait(&B.ufull[ub], (uq >> 1) & 1u);
        if (ok && !uok) {
          atomicExch(C.err, 1);
          *B.abort_flag = 1;
        }
        ok = __all_sync(0xffffffffu, uok);
        us = reinterpret_cast<const T*>(ubase + ub * ubytes);
        if constexpr (UREGS) {
          const V4* u4 = reinterpret_cast<const V4*>(us);
#pragma unroll
          for (int q = 0; q < UREG; ++q) {
            const int jv = lane + 32 * q;
            if (jv < nv) ur[q] = u4[jv];
          }
        }
        ++uq;
        curk = tl.k;
      }
      const T* buf = reinterpret_cast<const T*>(stage_base + (size_t)st * C.stage_bytes);
      const int rfirst = (warp - rdone % NW + NW) % NW;
      rdone += tl.nrows;
      for (int r = rfirst; ok && r < tl.nrows; r += NW) {
        const V4* row = reinterpret_cast<const V4*>(buf + (size_t)r * tl.ldI);
        const T ue = (DOT && tl.kind == 0 && lane == 0) ? us[tl.row0 + r] : (T)0;
        T a0 = 0, a1 = 0;   // two chains of fused multiply-adds
#pragma unroll
        for (int g = 0; g < UREG; g += QG) {
          if (32 * g >= nv) break;   // the same in every lane
          V4 m[QG], xs[UREGS ? 1 : QG];
#pragma unroll
          for (int q = 0; q < QG; ++q) {
            const int jv = lane + 32 * (g + q);
            if (jv < nv) {
              m[q] = row[jv];
              if constexpr (!UREGS) xs[UREGS ? 0 : q] = reinterpret_cast<const V4*>(us)[jv];
            }
          }
#pragma unroll
          for (int q = 0; q < QG; ++q) {
            const int jv = lane + 32 * (g + q);
            if (jv < nv) {
              V4 x;
              if constexpr (UREGS) x = ur[g + q];
              else x = xs[UREGS ? 0 : q];
              if constexpr (VEC == 4) {
                a0 = fma(m[q].x, x.x, a0);
                a1 = fma(m[q].y, x.y, a1);
                a0 = fma(m[q].z, x.z, a0);
                a1 = fma(m[q].w, x.w, a1);
              } else {
                a0 = fma(m[q].x, x.x, a0);
                a1 = fma(m[q].y, x.y, a1);
              }
            }
          }
        }
        T acc = a0 + a1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0 && nc > 0) {
          double* out = tl.kind == 0 ? t : qpart;
          out[tl.obase * nrhs + tl.row0 + r + (int64_t)tl.ostride * col0] = (double)acc;
        }
        // in the operator's precision: GB300's FP64 pipe is narrow
        if constexpr (DOT) dtacc += acc * ue;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&B.empty[st]);   // this warp has read the stage
    }
    __syncwarp();
    if (curk >= 0 && lane == 0) mbar_arrive(&B.uempty[(uq - 1) & 1u]);   // done with the last u
    if constexpr (DOT) dacc[0] = (double)dtacc;
    uq_end = uq;
  } else {
    // ---- consumers: wait for the tile, then read its descriptor from the
    // window (written by the producer before it issued the copy)
    int curk = -1;
    uint32_t uq = useq;
    const T* u = nullptr;
    for (int j = 0; j < n; ++j) {
      const uint32_t sq = seq + (uint32_t)j;
      const uint32_t st = sq % S;
      bool ok = !*B.abort_flag;
      if (ok && !mbar_wait(&B.full[st], (sq / S) & 1u)) {
        atomicExch(C.err, 1);
        *B.abort_flag = 1;
        ok = false;
      }
      ok = __all_sync(0xffffffffu, ok);
      const LTile tl = win[((j / WIN) & 1) * WIN + j % WIN];
      if (tl.k != curk) {
        if (curk >= 0) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&B.uempty[(uq - 1) & 1u]);   // done with the previous u
        }
        const uint32_t ub = uq & 1u;
        if (ok && !mbar_wait(&B.ufull[ub], (uq >> 1) & 1u)) {
          atomicExch(C.err, 1);
          *B.abort_flag = 1;
          ok = false;
        }
        ok = __all_sync(0xffffffffu, ok);
        u = reinterpret_cast<const T*>(ubase + ub * ubytes);
        ++uq;
        curk = tl.k;
      }
      const T* buf = reinterpret_cast<const T*>(stage_base + (size_t)st * C.stage_bytes);
      const int ldI = tl.ldI, nv = ldI / VEC, nr = tl.nrows;
      T acc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = (T)0;
      for (int jv = tid; ok && jv < nv; jv += NCONS) {
        if constexpr (VEC == 4) {
          float4 x[CT];
#pragma unroll
          for (int cc = 0; cc < CT; ++cc) x[cc] = reinterpret_cast<const float4*>(u + (size_t)cc * C.u_ld)[jv];
#pragma unroll
          for (int r = 0; r < RMAX; ++r)
            if (r < nr) {
              const float4 m = reinterpret_cast<const float4*>(buf + (size_t)r * ldI)[jv];
#pragma unroll
              for (int cc = 0; cc < CT; ++cc)
                acc[r * CT + cc] += m.x * x[cc].x + m.y * x[cc].y + m.z * x[cc].z + m.w * x[cc].w;
            }
        } else {
          double2 x[CT];
#pragma unroll
          for (int cc = 0; cc < CT; ++cc) x[cc] = reinterpret_cast<const double2*>(u + (size_t)cc * C.u_ld)[jv];
#pragma unroll
          for (int r = 0; r < RMAX; ++r)
            if (r < nr) {
              const double2 m = reinterpret_cast<const double2*>(buf + (size_t)r * ldI)[jv];
#pragma unroll
              for (int cc = 0; cc < CT; ++cc) acc[r * CT + cc] += m.x * x[cc].x + m.y * x[cc].y;
            }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&B.empty[st]);   // this warp has read the stage
      warp_transpose_sum<T, V>(acc, lane);
      double* rd = red + (j & 1) * 8 * V;
      constexpr int PER = V >= 32 ? V / 32 : 1;
      constexpr int LOWMASK = V >= 32 ? 0 : (32 / V) - 1;
      if ((lane & LOWMASK) == 0)
#pragma unroll
        for (int i = 0; i < PER; ++i) rd[warp * V + transpose_index<V>(lane, i)] = (double)acc[i];
      consumer_bar();
      if (ok)
        for (int q = tid; q < nr * nc; q += NCONS) {
          const int r = q / nc, cc = q % nc;
          const int v = r * CT + cc;
          double sum = 0;
#pragma unroll
          for (int w = 0; w < 8; ++w) sum += rd[w * V + v];
          double* out = tl.kind == 0 ? t : qpart;
          out[tl.obase * nrhs + tl.row0 + r + (int64_t)tl.ostride * (col0 + cc)] = sum;
          if constexpr (DOT) {
            if (tl.kind == 0) {
              const double pr = sum * (double)u[(size_t)cc * C.u_ld + tl.row0 + r];
#pragma unroll
              for (int c2 = 0; c2 < CT; ++c2)
                if (c2 == cc) dacc[c2] += pr;
            }
          }
        }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&B.uempty[(uq - 1) & 1u]);   // done with the last u
    uq_end = uq;
  }
  if constexpr (DOT) {
    // the CTA's share per column: warp sums, then the 8 consumer warps in order
    if (warp < NCONS / 32) {
#pragma unroll
      for (int cc = 0; cc < CT; ++cc) {
        double v = dacc[cc];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) dred[warp * CT + cc] = v;
      }
      consumer_bar();
      if (tid < nc) {
        double s = 0;
#pragma unroll
        for (int w = 0; w < NCONS / 32; ++w) s += dred[w * CT + tid];
        dot_out[tid] = s;
      }
    }
  }
  seq += (uint32_t)n;
  useq = uq_end;
}

}  // namespace ieti
