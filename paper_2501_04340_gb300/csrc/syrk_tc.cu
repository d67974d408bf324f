// Trailing update of the FP32 blocked Cholesky (Sec. 2.1: the local blocks
// K_rr^(k) are factored) on the 5th-generation tensor cores.
//
// After panel b is factored, every trailing block (r, c), r >= c > b, takes
//   C_rc -= L_rb L_cb^T      (K = 64, the panel width).
// FP32 accuracy from TF32 products: every panel entry is split into three TF32
// terms x = h + m + l (h and m rounded to TF32, l the exact remainder), and the
// six products h h, h m, m h, m m, h l, l h are accumulated in FP32 in tensor
// memory; the dropped terms are below 2^-33 relative. The tensor cores round
// the accumulator toward zero, so the leading products h h go to one
// accumulator and the five small ones to a second: adding the small terms into
// the leading sum would round that sum once per MMA, a bias that left the
// factor too inaccurate for the refinement. The two sums are added with
// round-to-nearest in the epilogue.
//
// Two kernels per panel:
//  k_split  writes the three terms of the rows below the diagonal block as
//           "tile images": for every 128-row group and 32-column half of the
//           panel, a 16 KB array in the K-major 128-byte-swizzled layout that
//           tcgen05.mma reads from shared memory;
//  k_syrk_tc one CTA per 128 x 128 tile (two block rows x two block columns):
//           per 32-column half, bulk copies (cp.async.bulk, mbarrier
//           completion) of the six images into shared memory, 24 MMAs
//           (M = N = 128, K = 8) issued by one thread and committed to an
//           mbarrier; the accumulator is read with tcgen05.ld and subtracted
//           from C.
//
// Measured on the 64-patch cube (FP32 factor): 82.9 ms for all trailing updates
// against 79.0 ms for the CUDA-core kernel, and 8 refinement steps instead of 7
// (the leading accumulator is still rounded toward zero 16 times per tile). At
// K = 64 the update is bound by the C traffic and the image writes, not by
// arithmetic, so this path is opt-in (IETI_SYRK_TC=1); it pays off only with
// wider outer panels (fewer passes over C).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace ieti {

namespace {

constexpr int IMG_BYTES = 128 * 32 * 4;   // one 128 x 32 TF32 image (16 KB)
constexpr int TC_THREADS = 256;
constexpr int TC_SMEM = 6 * IMG_BYTES + 1024;   // six images + alignment slack

__device__ __forceinline__ uint32_t tc_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool tc_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(tc_saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait (about one second at 2 GHz)
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!tc_try_wait(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}

// shared-memory matrix descriptor for a K-major operand in 128-byte swizzle
// atoms: start address >> 4 in bits [0,14), leading byte offset >> 4 in
// [16,30) (not used by swizzled K-major operands), stride byte offset >> 4 in
// [32,46) (1024 B between 8-row groups), version 1 in [46,48), layout type 2
// (128-byte swizzle) in [61,64)
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// instruction descriptor: FP32 accumulator (bits [4,6) = 1), A and B TF32
// ([7,10) = [10,13) = 2), both K-major, N >> 3 in [17,23), M >> 4 in [24,29)
constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row m, column k < 32) in a 128 x 32 image: rows in
// groups of 8 (1024 B), 128 B per row, 16-byte chunk index XORed with m mod 8
__device__ __forceinline__ uint32_t img_off(int m, int k) {
  return (uint32_t)((m >> 3) * 1024 + (m & 7) * 128 + ((((k >> 2) ^ (m & 7))) << 4) + (k & 3) * 4);
}

// 32 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t ta, uint32_t (&d)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]), "=r"(d[8]),
        "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15]), "=r"(d[16]),
        "=r"(d[17]), "=r"(d[18]), "=r"(d[19]), "=r"(d[20]), "=r"(d[21]), "=r"(d[22]), "=r"(d[23]), "=r"(d[24]),
        "=r"(d[25]), "=r"(d[26]), "=r"(d[27]), "=r"(d[28]), "=r"(d[29]), "=r"(d[30]), "=r"(d[31])
      : "r"(ta));
}

// round to the nearest TF32 value (10 mantissa bits)
__device__ __forceinline__ float tf32_rn(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// images of panel b: grid (row groups, subdomains); image (g, half, term) of
// subdomain k at img + ((grp_off[k] + g) * 2 + half) * 3 + term
__global__ void __launch_bounds__(256) k_split(const SubDev* sd, const int* grp_off, const float* L, float* img,
                                               int b) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  const int rows0 = (b + 1) * NB;   // first row below the diagonal block
  if (rows0 >= s.n) return;
  const int g = blockIdx.x;
  if (g * 128 >= s.n - rows0) return;
  const float* P = L + s.A + (int64_t)s.n * b * NB + rows0 + g * 128;
  unsigned char* base = reinterpret_cast<unsigned char*>(img) + (int64_t)(grp_off[k] + g) * 6 * IMG_BYTES;
  const int valid = min(128, s.n - rows0 - g * 128);
  for (int e = threadIdx.x; e < 128 * NB; e += blockDim.x) {
    const int m = e % 128, kk = e / 128;
    const float x = m < valid ? P[m + (int64_t)s.n * kk] : 0.f;
    const float h = tf32_rn(x);
    const float r = x - h;
    const float mm = tf32_rn(r);
    const float l = r - mm;
    unsigned char* half = base + (kk >> 5) * 3 * IMG_BYTES;
    const uint32_t o = img_off(m, kk & 31);
    *reinterpret_cast<float*>(half + o) = h;
    *reinterpret_cast<float*>(half + IMG_BYTES + o) = mm;
    *reinterpret_cast<float*>(half + 2 * IMG_BYTES + o) = l;
  }
}

__global__ void __launch_bounds__(TC_THREADS, 2) k_syrk_tc(const SubDev* sd, const int* grp_off, float* L,
                                                           const float* img, int b, int* err) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  const int Tk = s.nblk - b - 1;
  if (Tk <= 0) return;
  const int Tt = (Tk + 1) / 2;   // block pairs = row groups
  const int t = blockIdx.x;
  int R = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while (R * (R + 1) / 2 > t) --R;
  while ((R + 1) * (R + 2) / 2 <= t) ++R;
  const int C = t - R * (R + 1) / 2;
  if (R >= Tt) return;
  const int r0 = b + 1 + 2 * R, c0 = b + 1 + 2 * C;
  const int nr = min(2, s.nblk - r0), nc = min(2, s.nblk - c0);
  extern __shared__ unsigned char tc_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full_bar, mma_bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int64_t n = s.n;
  // epilogue mapping: warp w handles rows 32 (w % 4) + lane, columns 64 (w / 4) .. +63
  const int m = 32 * (warp % 4) + lane;
  const int col0 = 64 * (warp / 4);
  const int rb = r0 + m / NB, cb = c0 + col0 / NB;
  const bool writes = m / NB < nr && col0 / NB < nc && rb >= cb;
  float* Crow = L + s.A + (int64_t)r0 * NB + m + n * ((int64_t)c0 * NB + col0);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_saddr(&full_bar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_saddr(&mma_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(tc_saddr(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = tmem_base;
  const unsigned char* imgA = reinterpret_cast<const unsigned char*>(img) + (int64_t)(grp_off[k] + R) * 6 * IMG_BYTES;
  const unsigned char* imgB = reinterpret_cast<const unsigned char*>(img) + (int64_t)(grp_off[k] + C) * 6 * IMG_BYTES;
  bool ok = true;
  for (int half = 0; half < 2; ++half) {
    if (tid == 0) {
      // images A (h, m, l) then B (h, m, l) of this half into the six slots
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_saddr(&full_bar)),
                   "r"(6 * IMG_BYTES)
                   : "memory");
      for (int q = 0; q < 6; ++q) {
        const unsigned char* src = (q < 3 ? imgA : imgB) + (half * 3 + q % 3) * IMG_BYTES;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                tc_saddr(sm + q * IMG_BYTES)),
            "l"(src), "r"(IMG_BYTES), "r"(tc_saddr(&full_bar))
            : "memory");
      }
    }
    ok &= tc_wait(&full_bar, (uint32_t)half);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0 && ok) {
      constexpr uint32_t idesc = tc_idesc(128, 128);
      // term pairs (a, b): h h, h m, m h, m m, h l, l h
      constexpr int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        const uint32_t aa = tc_saddr(sm + pa[p] * IMG_BYTES), bb = tc_saddr(sm + (3 + pb[p]) * IMG_BYTES);
#pragma unroll
        for (int st = 0; st < 4; ++st) {   // K = 8 per instruction: 32 bytes within the 128-byte rows
          const uint64_t ad = tc_desc(aa + st * 32), bd = tc_desc(bb + st * 32);
          // leading products into columns 0..127, small ones into 128..255
          const uint32_t dst = p == 0 ? taddr : taddr + 128;
          const uint32_t acc = (half > 0 || st > 0 || p > 1) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred pp;\n setp.ne.u32 pp, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, pp;\n}\n" ::"r"(dst),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       tc_saddr(&mma_bar))
                   : "memory");
    }
    // the MMAs of this half must have read the slots before they are refilled
    // (and before the accumulator is read)
    ok &= tc_wait(&mma_bar, (uint32_t)half);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (!ok && lane == 0) atomicExch(err, 1);
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    float cv[32];   // C loads and the tensor-memory load in flight together
    if (writes) {
#pragma unroll
      for (int j = 0; j < 32; ++j) cv[j] = Crow[n * (32 * h2 + j)];
    }
    uint32_t d[32], e[32];
    const uint32_t ta = taddr + ((uint32_t)(32 * (warp % 4)) << 16) + (uint32_t)(col0 + 32 * h2);
    tmem_ld32(ta, d);
    tmem_ld32(ta + 128, e);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (writes && ok) {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        Crow[n * (32 * h2 + j)] = cv[j] - (__uint_as_float(d[j]) + __uint_as_float(e[j]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(taddr) : "memory");
}

}  // namespace

ieti_status syrk_tc_attrs(Ctx* c) {
  IETI_CUDA_TRY(c, cudaFuncSetAttribute(k_syrk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  return IETI_OK;
}

// image scratch (one 128-row group = 96 KB) and per-subdomain group offsets
ieti_status syrk_tc_alloc(Ctx* c) {
  std::vector<int> off(c->nsub);
  int tot = 0;
  for (int k = 0; k < c->nsub; ++k) {
    off[k] = tot;
    tot += (int)ceil_div(c->sd_host[k].n, 128);
  }
  void* p = nullptr;
  const size_t bytes = (size_t)std::max(tot, 1) * 6 * IMG_BYTES;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->err = "cudaMalloc of the tensor-core image scratch failed";
    return IETI_ERR_OOM;
  }
  c->allocs.push_back({p, bytes});
  c->tc_img = (float*)p;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int) * std::max(c->nsub, 1)) != cudaSuccess) {
    cudaGetLastError();
    c->err = "cudaMalloc failed";
    return IETI_ERR_OOM;
  }
  c->allocs.push_back({d, sizeof(int) * (size_t)std::max(c->nsub, 1)});
  IETI_CUDA_TRY(c, cudaMemcpy(d, off.data(), sizeof(int) * c->nsub, cudaMemcpyHostToDevice));
  c->d_grp_off = d;
  return IETI_OK;
}

// trailing update after panel b of every subdomain's FP32 factor
ieti_status syrk_tc(Ctx* c, const SubDev* d_sd, float* L, int b, int max_nblk, int nsub, cudaStream_t st) {
  const int Tk = max_nblk - b - 1;
  if (Tk <= 0) return IETI_OK;
  const int Tt = (Tk + 1) / 2;
  k_split<<<dim3((unsigned)Tt, (unsigned)nsub), 256, 0, st>>>(d_sd, c->d_grp_off, L, c->tc_img, b);
  IETI_LAUNCH_CHECK(c);
  k_syrk_tc<<<dim3((unsigned)(Tt * (Tt + 1) / 2), (unsigned)nsub), TC_THREADS, TC_SMEM, st>>>(
      d_sd, c->d_grp_off, L, c->tc_img, b, c->d_stream_err);
  IETI_LAUNCH_CHECK(c);
  return IETI_OK;
}

}  // namespace ieti
