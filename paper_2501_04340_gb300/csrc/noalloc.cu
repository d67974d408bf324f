// Batched interface product that allocates nothing: its scratch lives in a
// fixed file-scope device array instead of memory obtained from cudaMalloc.
//
// Computes y = sum_k B_k^T diag(w_k) M_k diag(w_k) B_k x for caller-owned blocks
// M_k and maps. With M_k = S_rIrI^(k) and w_k the signed rho-scaling weights this
// is the Dirichlet preconditioner; with M_k = S_rIrI^(k)-1 and w_k the signs it is
// the local part of the F-apply. The descriptors of the blocks are built on the
// device from the block sizes, which travel as the kernel parameter, so nothing
// is copied from host memory.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/ieti.h"

namespace {

// Scratch for one call: the per-subdomain descriptors and the local products
// t_k (sum_k nI_k x nrhs doubles). Held by every GPU that loads the library
// until the process exits.
constexpr int64_t kScratchDoubles = int64_t(1) << 22;   // 32 MiB
constexpr int kMaxSub = 4096;
static __device__ __align__(256) double g_scratch[kScratchDoubles];

struct Desc {
  int64_t moff;   // offset of M_k in the caller's block array
  int64_t ioff;   // offset of subdomain k's interface DOFs in the maps
  int64_t toff;   // offset of t_k in the scratch (after the descriptors)
  int nI;
  int pad;
};

constexpr int kDescDoubles = (int)((sizeof(Desc) * kMaxSub + sizeof(double) - 1) / sizeof(double));

std::mutex g_mutex;
double* g_ptr[128] = {};   // device address of g_scratch, per device (set up once)

// block sizes of one call, passed by value as the kernel parameter (16 KB, within
// the 32 KB parameter limit), so that no host buffer has to outlive the call
struct Sizes {
  int nsub, nrhs;
  int nI[kMaxSub];
};

// descriptors of all subdomains from the block sizes (one CTA: prefix sums in
// chunks of 1024 subdomains)
__global__ void __launch_bounds__(1024) k_descriptors(const Sizes sz, Desc* desc) {
  __shared__ int64_t part[1024];
  __shared__ int64_t carry[2];
  if (threadIdx.x == 0) carry[0] = carry[1] = 0;
  __syncthreads();
  for (int k0 = 0; k0 < sz.nsub; k0 += 1024) {
    const int k = k0 + threadIdx.x;
    const int64_t n = k < sz.nsub ? sz.nI[k] : 0;
    // inclusive scan of n and n^2 (two passes over the same buffer)
    int64_t scan[2];
    for (int which = 0; which < 2; ++which) {
      part[threadIdx.x] = which == 0 ? n : n * n;
      __syncthreads();
      for (int o = 1; o < 1024; o <<= 1) {
        const int64_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
      }
      scan[which] = part[threadIdx.x];
      __syncthreads();
    }
    const int64_t ioff = carry[0] + scan[0] - n, moff = carry[1] + scan[1] - n * n;
    if (k < sz.nsub) desc[k] = {moff, ioff, kDescDoubles + ioff * sz.nrhs, (int)n, 0};
    __syncthreads();
    if (threadIdx.x == 1023) {
      carry[0] += scan[0];
      carry[1] += scan[1];
    }
    __syncthreads();
  }
}

__global__ void k_product(const Desc* desc, const double* M, const int* dual, const double* w, const double* x,
                          int64_t m, int nrhs, double* t) {
  const int k = blockIdx.y;
  const Desc d = desc[k];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int i = blockIdx.x * 8 + warp;          // row of M_k
  if (i >= d.nI) return;
  const double* row = M + d.moff + (int64_t)d.nI * i;   // symmetric: row i = column i
  for (int col = 0; col < nrhs; ++col) {
    double acc = 0;
    for (int j = lane; j < d.nI; j += 32) {
      const int l = dual[d.ioff + j];
      if (l >= 0 && l < m) acc += row[j] * w[d.ioff + j] * x[l + m * col];   // entries outside [0, m) are skipped
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) t[d.toff + i + (int64_t)d.nI * col] = acc;
  }
}

__global__ void k_scatter(const Desc* desc, const int* dual, const double* w, const double* t, int64_t m, int nrhs,
                          double* y) {
  const int k = blockIdx.y;
  const Desc d = desc[k];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)d.nI * nrhs;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e % d.nI), col = (int)(e / d.nI);
    const int l = dual[d.ioff + i];
    if (l >= 0 && l < m) atomicAdd(y + l + m * col, w[d.ioff + i] * t[d.toff + i + (int64_t)d.nI * col]);
  }
}

// one-time set-up per device: the device address of the static scratch
double* scratch_ptr(int dev) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (dev < 0 || dev >= 128) return nullptr;
  if (!g_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      std::fprintf(stderr, "ieti_interface_product_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
      return nullptr;
    }
    g_ptr[dev] = (double*)p;
  }
  return g_ptr[dev];
}

}  // namespace

extern "C" ieti_status ieti_interface_product_noalloc(int nsub, const int* nI_host, const double* M_dev,
                                                      const int* dual_dev, const double* weight_dev, int64_t m,
                                                      const double* x_dev, double* y_dev, int nrhs, void* stream) {
  auto fail = [](ieti_status code, const std::string& msg) {
    std::fprintf(stderr, "ieti_interface_product_noalloc: %s\n", msg.c_str());
    return code;
  };
  if (nsub < 1 || nsub > kMaxSub || !nI_host || !M_dev || !dual_dev || !weight_dev || !x_dev || !y_dev ||
      nrhs < 1 || m < 1) {
    return fail(IETI_ERR_INVALID_ARG, "invalid argument (nsub must be 1..4096, nrhs >= 1, pointers non-null)");
  }
  Sizes sz;
  sz.nsub = nsub;
  sz.nrhs = nrhs;
  int64_t toff = kDescDoubles;
  int max_nI = 0;
  for (int k = 0; k < nsub; ++k) {
    if (nI_host[k] < 0) {
      return fail(IETI_ERR_INVALID_ARG, "negative interface size");
    }
    sz.nI[k] = nI_host[k];
    toff += (int64_t)nI_host[k] * nrhs;
    if (toff > kScratchDoubles) break;
    if (nI_host[k] > max_nI) max_nI = nI_host[k];
  }
  if (toff > kScratchDoubles) {
    return fail(IETI_ERR_INVALID_ARG, "sum_k nI_k x nrhs exceeds the fixed scratch of " +
                                          std::to_string(kScratchDoubles - kDescDoubles) + " doubles");
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    return fail(IETI_ERR_CUDA, "no current CUDA device");
  }
  double* base = scratch_ptr(dev);
  if (!base) return IETI_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  Desc* d_desc = (Desc*)base;
  double* t = base;   // t_k at toff (past the descriptors)
  k_descriptors<<<1, 1024, 0, st>>>(sz, d_desc);
  cudaError_t e = cudaMemsetAsync(y_dev, 0, sizeof(double) * m * nrhs, st);
  if (e != cudaSuccess) {
    return fail(IETI_ERR_CUDA, std::string("memset: ") + cudaGetErrorString(e));
  }
  if (max_nI > 0) {
    k_product<<<dim3((unsigned)((max_nI + 7) / 8), (unsigned)nsub), 256, 0, st>>>(d_desc, M_dev, dual_dev,
                                                                                weight_dev, x_dev, m, nrhs, t);
    k_scatter<<<dim3(64, (unsigned)nsub), 256, 0, st>>>(d_desc, dual_dev, weight_dev, t, m, nrhs, y_dev);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    return fail(IETI_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  }
  return IETI_OK;
}
