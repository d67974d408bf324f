// Warm-start network for the interface multipliers: a 3-layer perceptron
// x -> lambda0 (ReLU hidden layers) with BF16 operands and FP32 accumulation,
// trained with mean squared error and Adam; forward, backward and optimiser are
// all kernels of this file. The paper has no learned component; the network
// only supplies the initial guess of PCG on the interface problem (Eq. (7)),
// which keeps its own stopping test, so a poor guess costs iterations, never
// accuracy.
//
// GEMMs use the BF16 tensor-core MMA (m16n8k16, FP32 accumulators) on 64x64
// CTA tiles staged in shared memory; operands are addressed through (row,
// column) strides so that the transposed products of the backward pass need
// no copies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ieti.h"

struct ieti_mlp {
  int n_in = 0, n_hidden = 0, n_out = 0, max_batch = 0;
  int64_t nparam = 0;
  int64_t off[6] = {};        // W1 b1 W2 b2 W3 b3 in the parameter vector
  float* P = nullptr;         // FP32 master parameters
  float* G = nullptr;         // gradients
  float* M1 = nullptr;        // Adam moments
  float* M2 = nullptr;
  __nv_bfloat16* Wb = nullptr;   // BF16 copies of W1, W2, W3 (same offsets as in P, weights only)
  __nv_bfloat16 *Xb = nullptr, *A1b = nullptr, *A2b = nullptr, *dYb = nullptr, *dZb = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *dY = nullptr, *dZ = nullptr;
  float* shift = nullptr;     // input normalisation x' = (x - shift) * scale
  float* scale = nullptr;
  float out_scale = 1.0f;     // lambda = out_scale * y
  float* red = nullptr;       // loss partials
  float* loss_dev = nullptr;
  float* loss_acc = nullptr;  // sum of batch losses over the last epoch of a fit
  float *Xg = nullptr, *Tg = nullptr;   // gathered mini-batch (fit)
  int* perm = nullptr;        // shuffled sample order of every epoch (fit)
  int64_t perm_cap = 0;
  int step = 0;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

constexpr int TM = 64, TN = 64, TK = 32;

enum Epi { EPI_STORE = 0, EPI_BIAS_RELU = 1, EPI_BIAS = 2, EPI_RELU_GRAD = 3 };

__device__ inline uint32_t pack2(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// C(m, n) = sum_k A(m, k) B(k, n); A(m, k) = A[m*sam + k*sak], B(k, n) = B[k*sbk + n*sbn]
template <int EPI>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int64_t sam,
                                              int64_t sak, const __nv_bfloat16* __restrict__ B, int64_t sbk,
                                              int64_t sbn, float* __restrict__ C, const float* __restrict__ bias,
                                              __nv_bfloat16* __restrict__ Cb, const float* __restrict__ mask) {
  __shared__ __align__(16) __nv_bfloat16 As[TM][TK + 8];
  __shared__ __align__(16) __nv_bfloat16 Bs[TN][TK + 8];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int g = lane / 4, t = lane % 4;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int wm = (warp / 2) * 32, wn = (warp % 2) * 32;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  for (int k0 = 0; k0 < K; k0 += TK) {
    __syncthreads();
    for (int idx = tid; idx < TM * TK; idx += blockDim.x) {
      const int r = idx / TK, kk = idx % TK;
      const int m = m0 + r, k = k0 + kk;
      As[r][kk] = (m < M && k < K) ? A[m * sam + k * sak] : __float2bfloat16(0.f);
      const int n = n0 + r;
      Bs[r][kk] = (n < N && k < K) ? B[k * sbk + n * sbn] : __float2bfloat16(0.f);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < TK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r = wm + mi * 16 + g, c = ks + 2 * t;
        af[mi][0] = pack2(&As[r][c]);
        af[mi][1] = pack2(&As[r + 8][c]);
        af[mi][2] = pack2(&As[r][c + 8]);
        af[mi][3] = pack2(&As[r + 8][c + 8]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int n = wn + ni * 8 + g, c = ks + 2 * t;
        bfr[ni][0] = pack2(&Bs[n][c]);
        bfr[ni][1] = pack2(&Bs[n][c + 8]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
              : "r"(af[mi][0]), "r"(af[mi][1]), "r"(af[mi][2]), "r"(af[mi][3]), "r"(bfr[ni][0]), "r"(bfr[ni][1]));
    }
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + mi * 16 + g + (q >= 2 ? 8 : 0);
        const int n = n0 + wn + ni * 8 + 2 * t + (q & 1);
        if (m >= M || n >= N) continue;
        float v = acc[mi][ni][q];
        const int64_t o = (int64_t)m * N + n;
        if (EPI == EPI_STORE) {
          C[o] = v;
        } else if (EPI == EPI_BIAS_RELU) {
          v += bias[n];
          C[o] = v;
          Cb[o] = __float2bfloat16(v > 0.f ? v : 0.f);
        } else if (EPI == EPI_BIAS) {
          C[o] = v + bias[n];
        } else {   // EPI_RELU_GRAD: dZ = dA * [Z > 0]
          v = mask[o] > 0.f ? v : 0.f;
          C[o] = v;
          Cb[o] = __float2bfloat16(v);
        }
      }
}

__global__ void k_input(const float* x, const float* shift, const float* scale, int n_in, int64_t n,
                        __nv_bfloat16* xb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(i % n_in);
    xb[i] = __float2bfloat16((x[i] - shift[f]) * scale[f]);
  }
}

// dY = 2 (Y - T/out_scale) / (B n_out); per-block partial sums of the squared error
__global__ void k_loss(const float* Y, const float* T, float inv_out_scale, int64_t n, float gscale, float* dY,
                       __nv_bfloat16* dYb, float* red) {
  __shared__ float s[256];
  float acc = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i] * inv_out_scale;
    acc += d * d;
    const float gv = gscale * d;
    dY[i] = gv;
    dYb[i] = __float2bfloat16(gv);
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) red[blockIdx.x] = s[0];
}

__global__ void k_sum(const float* red, int n, float div, float* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += red[i];
    *out = s / div;
  }
}

// db[n] = sum over the batch of dZ[b, n] (fixed order)
__global__ void k_colsum(const float* dZ, int B, int N, float* db) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dZ[(int64_t)b * N + n];
    db[n] = s;
  }
}

// Adam with bias correction; omb1 = 1 - beta1 and omb2 = 1 - beta2 are passed
// separately (rounded from FP64) because 1 - beta2 formed from an FP32 beta2 is
// off by 1.3e-5 relative.
__global__ void k_adam(float* P, const float* G, float* M1, float* M2, int64_t n, float lr, float b1, float omb1,
                       float b2, float omb2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = b1 * M1[i] + omb1 * g;
    const float v = b2 * M2[i] + omb2 * g * g;
    M1[i] = m;
    M2[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

__global__ void k_to_bf16(const float* src, int64_t n, __nv_bfloat16* dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16(src[i]);
}

// per-feature mean and 1/std over the samples (FP64 accumulation, two passes)
__global__ void k_feature_stats(const float* X, int n, int n_in, float* shift, float* scale) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < n_in; f += gridDim.x * blockDim.x) {
    double mean = 0.0;
    for (int i = 0; i < n; ++i) mean += X[(int64_t)i * n_in + f];
    mean /= n;
    double var = 0.0;
    for (int i = 0; i < n; ++i) {
      const double d = X[(int64_t)i * n_in + f] - mean;
      var += d * d;
    }
    var /= n;
    shift[f] = (float)mean;
    scale[f] = var > 1e-24 ? (float)(1.0 / sqrt(var)) : 1.0f;
  }
}

// out = sqrt(mean of T^2), one block
__global__ void k_rms(const float* T, int64_t n, float* out) {
  __shared__ double s[1024];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += (double)T[i] * T[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (float)sqrt(s[0] / (double)n);
}

// dst[r, :] = src[idx[r], :] for r < rows
__global__ void k_gather_rows(const float* src, const int* idx, int rows, int width, float* dst) {
  const int64_t n = (int64_t)rows * width;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / width, c = i % width;
    dst[i] = src[(int64_t)idx[r] * width + c];
  }
}

__global__ void k_accumulate(const float* v, float* acc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *acc += *v;
}

__global__ void k_scale_out_f64(const float* Y, int64_t n, float s, double* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)s * (double)Y[i];
}

// lam[b, j] = s * sum_c coef[b, c] Y[b, c m + j] (FP64 sum of the FP32 outputs)
__global__ void k_combine(const float* Y, const double* coef, int batch, int ncoef, int m, float s, double* lam) {
  const int64_t n = (int64_t)batch * m;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / m, j = i % m;
    const float* y = Y + b * (int64_t)ncoef * m + j;
    const double* c = coef + b * ncoef;
    double acc = 0.0;
    for (int q = 0; q < ncoef; ++q) acc += c[q] * (double)y[(int64_t)q * m];
    lam[i] = (double)s * acc;
  }
}

__global__ void k_scale_out(const float* Y, int64_t n, float s, float* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = s * Y[i];
}

template <typename T>
bool alloc(ieti_mlp* m, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
    cudaGetLastError();
    m->err = "cudaMalloc failed";
    return false;
  }
  m->allocs.push_back(q);
  *p = (T*)q;
  return true;
}

template <int EPI>
ieti_status gemm(ieti_mlp* m, int M, int N, int K, const __nv_bfloat16* A, int64_t sam, int64_t sak,
                 const __nv_bfloat16* B, int64_t sbk, int64_t sbn, float* C, const float* bias, __nv_bfloat16* Cb,
                 const float* mask, cudaStream_t st) {
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  k_gemm<EPI><<<grid, 128, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, bias, Cb, mask);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    m->err = std::string("gemm launch: ") + cudaGetErrorString(e);
    return IETI_ERR_CUDA;
  }
  return IETI_OK;
}

#define MLP_TRY(x)                    \
  do {                                \
    ieti_status r__ = (x);            \
    if (r__ != IETI_OK) return r__;   \
  } while (0)

ieti_status refresh_bf16(ieti_mlp* m, cudaStream_t st) {
  for (int l = 0; l < 3; ++l) {
    const int64_t o = m->off[2 * l], cnt = m->off[2 * l + 1] - o;
    k_to_bf16<<<256, 256, 0, st>>>(m->P + o, cnt, m->Wb + o);
  }
  return cudaGetLastError() == cudaSuccess ? IETI_OK : IETI_ERR_CUDA;
}

ieti_status forward_impl(ieti_mlp* m, const float* x, int B, cudaStream_t st) {
  const int I = m->n_in, H = m->n_hidden, O = m->n_out;
  k_input<<<256, 256, 0, st>>>(x, m->shift, m->scale, I, (int64_t)B * I, m->Xb);
  const __nv_bfloat16 *W1 = m->Wb + m->off[0], *W2 = m->Wb + m->off[2], *W3 = m->Wb + m->off[4];
  // Z1 = X W1^T + b1: A(b, i) = X[b, i], B(i, h) = W1[h, i]
  MLP_TRY(gemm<EPI_BIAS_RELU>(m, B, H, I, m->Xb, I, 1, W1, 1, I, m->Z1, m->P + m->off[1], m->A1b, nullptr, st));
  MLP_TRY(gemm<EPI_BIAS_RELU>(m, B, H, H, m->A1b, H, 1, W2, 1, H, m->Z2, m->P + m->off[3], m->A2b, nullptr, st));
  MLP_TRY(gemm<EPI_BIAS>(m, B, O, H, m->A2b, H, 1, W3, 1, H, m->Y, m->P + m->off[5], nullptr, nullptr, st));
  return IETI_OK;
}

ieti_status backward_impl(ieti_mlp* m, const float* x_dev, const float* t_dev, int batch, cudaStream_t st) {
  const int I = m->n_in, H = m->n_hidden, O = m->n_out, B = batch;
  MLP_TRY(forward_impl(m, x_dev, B, st));
  const int64_t nY = (int64_t)B * O;
  const int lb = 256;
  k_loss<<<lb, 256, 0, st>>>(m->Y, t_dev, 1.0f / m->out_scale, nY, 2.0f / (float)nY, m->dY, m->dYb, m->red);
  k_sum<<<1, 32, 0, st>>>(m->red, lb, (float)nY, m->loss_dev);
  float* G = m->G;
  const __nv_bfloat16 *W2 = m->Wb + m->off[2], *W3 = m->Wb + m->off[4];
  // layer 3: dW3 = dY^T A2 (A(o, b) = dY[b, o]; B(b, h) = A2[b, h]), db3, dA2 = dY W3
  MLP_TRY(gemm<EPI_STORE>(m, O, H, B, m->dYb, 1, O, m->A2b, H, 1, G + m->off[4], nullptr, nullptr, nullptr, st));
  k_colsum<<<(O + 255) / 256, 256, 0, st>>>(m->dY, B, O, G + m->off[5]);
  MLP_TRY(gemm<EPI_RELU_GRAD>(m, B, H, O, m->dYb, O, 1, W3, H, 1, m->dZ, nullptr, m->dZb, m->Z2, st));
  // layer 2
  MLP_TRY(gemm<EPI_STORE>(m, H, H, B, m->dZb, 1, H, m->A1b, H, 1, G + m->off[2], nullptr, nullptr, nullptr, st));
  k_colsum<<<(H + 255) / 256, 256, 0, st>>>(m->dZ, B, H, G + m->off[3]);
  // dA1 = dZ2 W2 -> dZ1 (written to the same buffers after the layer-2 products used them)
  MLP_TRY(gemm<EPI_RELU_GRAD>(m, B, H, H, m->dZb, H, 1, W2, H, 1, m->dY, nullptr, m->dYb, m->Z1, st));
  // layer 1: dW1 = dZ1^T X, db1
  MLP_TRY(gemm<EPI_STORE>(m, H, I, B, m->dYb, 1, H, m->Xb, I, 1, G + m->off[0], nullptr, nullptr, nullptr, st));
  k_colsum<<<(H + 255) / 256, 256, 0, st>>>(m->dY, B, H, G + m->off[1]);
  return cudaGetLastError() == cudaSuccess ? IETI_OK : IETI_ERR_CUDA;
}

ieti_status adam_impl(ieti_mlp* m, float lr, cudaStream_t st) {
  m->step += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - pow(b1, (double)m->step)), c2 = (float)(1.0 - pow(b2, (double)m->step));
  k_adam<<<512, 256, 0, st>>>(m->P, m->G, m->M1, m->M2, m->nparam, lr, (float)b1, (float)(1.0 - b1), (float)b2,
                              (float)(1.0 - b2), 1e-8f, c1, c2);
  return refresh_bf16(m, st);
}

uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

ieti_status ieti_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, ieti_mlp** out) {
  if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || max_batch < 1) return IETI_ERR_INVALID_ARG;
  ieti_mlp* m = new ieti_mlp();
  *out = m;
  m->n_in = n_in;
  m->n_hidden = n_hidden;
  m->n_out = n_out;
  m->max_batch = max_batch;
  const int64_t sizes[6] = {(int64_t)n_hidden * n_in, n_hidden, (int64_t)n_hidden * n_hidden, n_hidden,
                            (int64_t)n_out * n_hidden, n_out};
  int64_t acc = 0;
  for (int i = 0; i < 6; ++i) {
    m->off[i] = acc;
    acc += sizes[i];
  }
  m->nparam = acc;
  // dY / dYb later hold dZ1 (batch x hidden) as well
  const int64_t BH = (int64_t)max_batch * n_hidden,
                BO = (int64_t)max_batch * (n_out > n_hidden ? n_out : n_hidden);
  bool ok = alloc(m, &m->P, acc) && alloc(m, &m->G, acc) && alloc(m, &m->M1, acc) && alloc(m, &m->M2, acc) &&
            alloc(m, &m->Wb, acc) && alloc(m, &m->Xb, (size_t)max_batch * n_in) && alloc(m, &m->A1b, BH) &&
            alloc(m, &m->A2b, BH) && alloc(m, &m->dYb, BO) && alloc(m, &m->dZb, BH) && alloc(m, &m->Z1, BH) &&
            alloc(m, &m->Z2, BH) && alloc(m, &m->Y, BO) && alloc(m, &m->dY, BO) && alloc(m, &m->dZ, BH) &&
            alloc(m, &m->shift, n_in) && alloc(m, &m->scale, n_in) && alloc(m, &m->red, 1024) &&
            alloc(m, &m->loss_dev, 1) && alloc(m, &m->loss_acc, 1) &&
            alloc(m, &m->Xg, (size_t)max_batch * n_in) && alloc(m, &m->Tg, (size_t)max_batch * n_out);
  if (!ok) return IETI_ERR_OOM;
  std::vector<float> one(n_in, 1.0f), zero(n_in, 0.0f);
  cudaMemcpy(m->scale, one.data(), sizeof(float) * n_in, cudaMemcpyHostToDevice);
  cudaMemcpy(m->shift, zero.data(), sizeof(float) * n_in, cudaMemcpyHostToDevice);
  cudaMemset(m->P, 0, sizeof(float) * acc);
  cudaMemset(m->M1, 0, sizeof(float) * acc);
  cudaMemset(m->M2, 0, sizeof(float) * acc);
  return cudaGetLastError() == cudaSuccess ? IETI_OK : IETI_ERR_CUDA;
}

ieti_status ieti_mlp_query(const ieti_mlp* m, int* sizes4, int64_t* nparam) {
  if (!m || !sizes4 || !nparam) return IETI_ERR_INVALID_ARG;
  sizes4[0] = m->n_in;
  sizes4[1] = m->n_hidden;
  sizes4[2] = m->n_out;
  sizes4[3] = m->max_batch;
  *nparam = m->nparam;
  return IETI_OK;
}

ieti_status ieti_mlp_set_params(ieti_mlp* m, const float* params_host, int64_t count) {
  if (!m || !params_host || count != m->nparam) return IETI_ERR_INVALID_ARG;
  if (cudaMemcpy(m->P, params_host, sizeof(float) * count, cudaMemcpyHostToDevice) != cudaSuccess)
    return IETI_ERR_CUDA;
  cudaMemset(m->M1, 0, sizeof(float) * count);
  cudaMemset(m->M2, 0, sizeof(float) * count);
  m->step = 0;
  return refresh_bf16(m, 0) == IETI_OK && cudaDeviceSynchronize() == cudaSuccess ? IETI_OK : IETI_ERR_CUDA;
}

ieti_status ieti_mlp_set_scaling(ieti_mlp* m, const float* shift_host, const float* scale_host, float out_scale) {
  if (!m || !shift_host || !scale_host || !(out_scale > 0)) return IETI_ERR_INVALID_ARG;
  cudaMemcpy(m->shift, shift_host, sizeof(float) * m->n_in, cudaMemcpyHostToDevice);
  cudaMemcpy(m->scale, scale_host, sizeof(float) * m->n_in, cudaMemcpyHostToDevice);
  m->out_scale = out_scale;
  return cudaGetLastError() == cudaSuccess ? IETI_OK : IETI_ERR_CUDA;
}

ieti_status ieti_mlp_get(ieti_mlp* m, int which, float* out_host, int64_t cap, int64_t* count) {
  if (!m || !count) return IETI_ERR_INVALID_ARG;
  if (which < 0 || which > 2) return IETI_ERR_INVALID_ARG;
  *count = which == 2 ? 2 * (int64_t)m->n_in + 1 : m->nparam;
  if (!out_host) return IETI_OK;
  if (cap < *count) return IETI_ERR_INVALID_ARG;
  if (which == 2) {
    if (cudaMemcpy(out_host, m->shift, sizeof(float) * m->n_in, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(out_host + m->n_in, m->scale, sizeof(float) * m->n_in, cudaMemcpyDeviceToHost) != cudaSuccess)
      return IETI_ERR_CUDA;
    out_host[2 * m->n_in] = m->out_scale;
    return IETI_OK;
  }
  const float* src = which == 0 ? m->P : m->G;
  return cudaMemcpy(out_host, src, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost) == cudaSuccess
             ? IETI_OK
             : IETI_ERR_CUDA;
}

ieti_status ieti_mlp_forward(ieti_mlp* m, const float* x_dev, float* y_dev, int batch, void* stream) {
  if (!m || !x_dev || !y_dev || batch < 1 || batch > m->max_batch) return IETI_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  MLP_TRY(forward_impl(m, x_dev, batch, st));
  k_scale_out<<<256, 256, 0, st>>>(m->Y, (int64_t)batch * m->n_out, m->out_scale, y_dev);
  return cudaGetLastError() == cudaSuccess ? IETI_OK : IETI_ERR_CUDA;
}

ieti_status ieti_mlp_backward(ieti_mlp* m, const float* x_dev, const float* t_dev, int batch, float* loss_host,
                              void* stream) {
  if (!m || !x_dev || !t_dev || batch < 1 || batch > m->max_batch) return IETI_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  MLP_TRY(backward_impl(m, x_dev, t_dev, batch, st));
  if (loss_host) {
    if (cudaMemcpyAsync(loss_host, m->loss_dev, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return IETI_ERR_CUDA;
  }
  return IETI_OK;
}

ieti_status ieti_mlp_adam(ieti_mlp* m, float lr, void* stream) {
  if (!m || !(lr > 0)) return IETI_ERR_INVALID_ARG;
  return adam_impl(m, lr, (cudaStream_t)stream);
}

ieti_status ieti_mlp_forward_f64(ieti_mlp* m, const float* x_dev, double* lam_dev, int batch, void* stream) {
  if (!m || !x_dev || !lam_dev || batch < 1 || batch > m->max_batch) return IETI_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  MLP_TRY(forward_impl(m, x_dev, batch, st));
  k_scale_out_f64<<<256, 256, 0, st>>>(m->Y, (int64_t)batch * m->n_out, m->out_scale, lam_dev);
  return cudaGetLastError() == cudaSuccess ? IETI_OK : IETI_ERR_CUDA;
}

ieti_status ieti_mlp_forward_combine(ieti_mlp* m, const float* x_dev, const double* coef_dev, int ncoef,
                                     double* lam_dev, int batch, void* stream) {
  if (!m || !x_dev || !coef_dev || !lam_dev || batch < 1 || batch > m->max_batch || ncoef < 1 ||
      m->n_out % ncoef != 0)
    return IETI_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  MLP_TRY(forward_impl(m, x_dev, batch, st));
  const int mm = m->n_out / ncoef;
  k_combine<<<512, 256, 0, st>>>(m->Y, coef_dev, batch, ncoef, mm, m->out_scale, lam_dev);
  return cudaGetLastError() == cudaSuccess ? IETI_OK : IETI_ERR_CUDA;
}

ieti_status ieti_mlp_fit(ieti_mlp* m, const float* X_dev, const float* T_dev, int n_samples, int batch,
                         int epochs, float lr, float decay, unsigned long long seed, int normalise,
                         float* loss_host, void* stream) {
  if (!m || !X_dev || !T_dev || n_samples < 1 || batch < 1 || batch > m->max_batch || epochs < 1 || !(lr > 0) ||
      !(decay > 0) || decay > 1)
    return IETI_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (normalise) {
    k_feature_stats<<<(m->n_in + 127) / 128, 128, 0, st>>>(X_dev, n_samples, m->n_in, m->shift, m->scale);
    k_rms<<<1, 1024, 0, st>>>(T_dev, (int64_t)n_samples * m->n_out, m->loss_acc);
    float rms = 0.f;
    if (cudaMemcpyAsync(&rms, m->loss_acc, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return IETI_ERR_CUDA;
    m->out_scale = rms > 0.f && std::isfinite(rms) ? rms : 1.0f;
  }
  // every epoch's sample order: Fisher-Yates driven by splitmix64(seed, epoch)
  const int64_t total = (int64_t)epochs * n_samples;
  if (total > m->perm_cap) {
    int* p = nullptr;
    if (cudaMalloc(&p, sizeof(int) * total) != cudaSuccess) {
      cudaGetLastError();
      m->err = "cudaMalloc failed (sample order)";
      return IETI_ERR_OOM;
    }
    m->allocs.push_back(p);
    m->perm = p;
    m->perm_cap = total;
  }
  std::vector<int> order((size_t)total);
  for (int e = 0; e < epochs; ++e) {
    int* o = order.data() + (int64_t)e * n_samples;
    for (int i = 0; i < n_samples; ++i) o[i] = i;
    uint64_t state = seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(e + 1));
    for (int i = n_samples - 1; i > 0; --i) {
      const int j = (int)(splitmix64(state) % (uint64_t)(i + 1));
      const int t = o[i];
      o[i] = o[j];
      o[j] = t;
    }
  }
  if (cudaMemcpyAsync(m->perm, order.data(), sizeof(int) * total, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return IETI_ERR_CUDA;
  cudaMemsetAsync(m->loss_acc, 0, sizeof(float), st);
  int nbatch_last = 0;
  float lr_e = lr;
  for (int e = 0; e < epochs; ++e, lr_e *= decay) {
    for (int b0 = 0; b0 < n_samples; b0 += batch) {
      const int nb = n_samples - b0 < batch ? n_samples - b0 : batch;
      const int* idx = m->perm + (int64_t)e * n_samples + b0;
      k_gather_rows<<<128, 256, 0, st>>>(X_dev, idx, nb, m->n_in, m->Xg);
      k_gather_rows<<<256, 256, 0, st>>>(T_dev, idx, nb, m->n_out, m->Tg);
      MLP_TRY(backward_impl(m, m->Xg, m->Tg, nb, st));
      if (e == epochs - 1) {
        k_accumulate<<<1, 32, 0, st>>>(m->loss_dev, m->loss_acc);
        ++nbatch_last;
      }
      MLP_TRY(adam_impl(m, lr_e, st));
    }
  }
  if (cudaGetLastError() != cudaSuccess) return IETI_ERR_CUDA;
  if (loss_host) {
    float acc = 0.f;
    if (cudaMemcpyAsync(&acc, m->loss_acc, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return IETI_ERR_CUDA;
    *loss_host = acc / (float)nbatch_last;
  }
  return IETI_OK;
}

const char* ieti_mlp_last_error(const ieti_mlp* m) { return m ? m->err.c_str() : ""; }

void ieti_mlp_destroy(ieti_mlp* m) {
  if (!m) return;
  for (void* p : m->allocs) cudaFree(p);
  delete m;
}

}  // extern "C"
