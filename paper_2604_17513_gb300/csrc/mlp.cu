// Warm-start network kernels: a 3-layer perceptron 10 -> 128 -> 128 -> 6 with
// ReLU, evaluated per contact.  Weights are kept as FP32 master copies and
// rounded to bf16 when staged into shared memory; every product accumulates
// in FP32.  Parameter layout (flat): W1[128][10] b1[128] W2[128][128] b2[128]
// W3[6][128] b3[6].
//
//   k_mlp_forward   y = f(x) for a batch (inference inside the step)
//   k_mlp_fwd_bwd   per-sample forward and backward of L = (1/B) sum 0.5|y - t|^2,
//                   keeping the activations and the pre-activation gradients
//   k_mlp_wgrad     weight gradients as batch sums of outer products
//   k_mlp_adam      Adam update of the FP32 master weights
#include <cuda_bf16.h>

#include <algorithm>

#include "flash_internal.cuh"

namespace flash {
namespace {

constexpr int NI = 10, NH = 128, NO = 6;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH, NPARAM = OFF_B3 + NO;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// stage the (bf16-rounded weights, FP32 biases) into shared memory
__device__ void stage_params(const float *p, float *w) {
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) {
    const bool bias = (i >= OFF_B1 && i < OFF_W2) || (i >= OFF_B2 && i < OFF_W3) || i >= OFF_B3;
    w[i] = bias ? p[i] : bf16r(p[i]);
  }
}

// ---------------------------------------------------------------- inference
// One sample per thread.  The layer-1 activations stay in registers; W2 is
// staged transposed (W2t[j][i]), so the weights of eight consecutive output
// neurons for input j are two 16-byte broadcast loads.  Blocks stage the
// weights once and loop over 128-sample tiles.  Every output neuron sums its
// inputs in ascending order from its bias, as the training kernel does.
constexpr int FWD_T = 128;    // samples (= threads) per tile
constexpr int FWD_MIN_BLOCKS = 2;

__device__ void stage_params_fwd(const float *p, float *w) {
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) {
    const bool bias = (i >= OFF_B1 && i < OFF_W2) || (i >= OFF_B2 && i < OFF_W3) || i >= OFF_B3;
    int d = i;
    if (i >= OFF_W2 && i < OFF_B2) {   // W2[r][c] -> W2t[c][r]
      const int r = (i - OFF_W2) / NH, c = (i - OFF_W2) % NH;
      d = OFF_W2 + c * NH + r;
    }
    w[d] = bias ? p[i] : bf16r(p[i]);
  }
}

__global__ void __launch_bounds__(FWD_T, FWD_MIN_BLOCKS) k_mlp_forward(const float *__restrict__ params,
                                                                      const float *__restrict__ X,
                                                                      float *__restrict__ Y,
                                                                      const int64_t *__restrict__ n_rows_dev,
                                                                      int64_t n_rows_host) {
  extern __shared__ __align__(16) float sm[];
  float *w = sm;   // NPARAM (W2 transposed)
  const int64_t n_rows = n_rows_dev ? *n_rows_dev : n_rows_host;
  const int64_t tiles = (n_rows + FWD_T - 1) / FWD_T;
  if (blockIdx.x >= tiles) return;
  stage_params_fwd(params, w);
  __syncthreads();
  const float4 *w2t = reinterpret_cast<const float4 *>(w + OFF_W2);   // OFF_W2 is a multiple of 4
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t row = tile * FWD_T + threadIdx.x;
    const bool live = row < n_rows;
    float x[NI];
#pragma unroll
    for (int j = 0; j < NI; j++) x[j] = live ? X[row * NI + j] : 0.f;
    float h1[NH];
#pragma unroll
    for (int i = 0; i < NH; i++) {
      float s = w[OFF_B1 + i];
#pragma unroll
      for (int j = 0; j < NI; j++) s = fmaf(w[OFF_W1 + i * NI + j], x[j], s);
      h1[i] = fmaxf(s, 0.f);
    }
    // layer 2 fused with layer 3: y += W3[:, i] * relu(W2[i, :] h1 + b2[i])
    float y[NO];
#pragma unroll
    for (int k = 0; k < NO; k++) y[k] = w[OFF_B3 + k];
    for (int i = 0; i < NH; i += 8) {
      float s[8];
#pragma unroll
      for (int u = 0; u < 8; u++) s[u] = w[OFF_B2 + i + u];
#pragma unroll
      for (int j = 0; j < NH; j++) {
        const float4 a = w2t[(j * NH + i) >> 2], b = w2t[((j * NH + i) >> 2) + 1];
        const float h = h1[j];
        s[0] = fmaf(a.x, h, s[0]); s[1] = fmaf(a.y, h, s[1]); s[2] = fmaf(a.z, h, s[2]); s[3] = fmaf(a.w, h, s[3]);
        s[4] = fmaf(b.x, h, s[4]); s[5] = fmaf(b.y, h, s[5]); s[6] = fmaf(b.z, h, s[6]); s[7] = fmaf(b.w, h, s[7]);
      }
#pragma unroll
      for (int u = 0; u < 8; u++) s[u] = fmaxf(s[u], 0.f);
#pragma unroll
      for (int g = 0; g < 8; g += 4)
#pragma unroll
        for (int k = 0; k < NO; k++)
          y[k] += w[OFF_W3 + k * NH + i + g] * s[g] + w[OFF_W3 + k * NH + i + g + 1] * s[g + 1] +
                  w[OFF_W3 + k * NH + i + g + 2] * s[g + 2] + w[OFF_W3 + k * NH + i + g + 3] * s[g + 3];
    }
    if (live)
#pragma unroll
      for (int k = 0; k < NO; k++) Y[row * NO + k] = y[k];
  }
}

// ---------------------------------------------------------------- training
constexpr int BWD_T = 64;    // samples (= threads) per block

// Per-sample forward + backward.  Outputs (row-major, per sample):
//   H1, H2 [B][NH] post-ReLU activations, DZ1, DZ2 [B][NH] gradients of the
//   loss w.r.t. the pre-activations, DY [B][NO] = (y - t)/B, SE [B] = |y - t|^2
__global__ void __launch_bounds__(BWD_T) k_mlp_fwd_bwd(const float *__restrict__ params, const float *__restrict__ X,
                                                       const float *__restrict__ T, int B, float *H1, float *H2,
                                                       float *DZ1, float *DZ2, float *DY, float *SE) {
  extern __shared__ float sm[];
  float *w = sm;
  float *h1 = sm + NPARAM + (NPARAM & 1);   // [NH][BWD_T]
  float *h2 = h1 + NH * BWD_T;              // [NH][BWD_T]
  float *dz = h2 + NH * BWD_T;              // [NH][BWD_T]
  stage_params(params, w);
  __syncthreads();
  const int t = threadIdx.x;
  const int row = blockIdx.x * BWD_T + t;
  const bool live = row < B;
  float x[NI];
#pragma unroll
  for (int j = 0; j < NI; j++) x[j] = live ? X[(size_t)row * NI + j] : 0.f;
  for (int i = 0; i < NH; i++) {
    float s = w[OFF_B1 + i];
#pragma unroll
    for (int j = 0; j < NI; j++) s = fmaf(w[OFF_W1 + i * NI + j], x[j], s);
    h1[i * BWD_T + t] = fmaxf(s, 0.f);
  }
  for (int i = 0; i < NH; i++) {
    float s = w[OFF_B2 + i];
#pragma unroll 8
    for (int j = 0; j < NH; j++) s = fmaf(w[OFF_W2 + i * NH + j], h1[j * BWD_T + t], s);
    h2[i * BWD_T + t] = fmaxf(s, 0.f);
  }
  float dy[NO], se = 0.f;
#pragma unroll
  for (int k = 0; k < NO; k++) {
    float s = w[OFF_B3 + k];
    for (int j = 0; j < NH; j++) s = fmaf(w[OFF_W3 + k * NH + j], h2[j * BWD_T + t], s);
    const float e = live ? s - T[(size_t)row * NO + k] : 0.f;
    se += e * e;
    dy[k] = e / (float)B;
  }
  // dz2 = (W3^T dy) * [z2 > 0]
  for (int i = 0; i < NH; i++) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NO; k++) s = fmaf(w[OFF_W3 + k * NH + i], dy[k], s);
    dz[i * BWD_T + t] = h2[i * BWD_T + t] > 0.f ? s : 0.f;
  }
  if (live) {
    for (int i = 0; i < NH; i++) {
      H1[(size_t)row * NH + i] = h1[i * BWD_T + t];
      H2[(size_t)row * NH + i] = h2[i * BWD_T + t];
      DZ2[(size_t)row * NH + i] = dz[i * BWD_T + t];
    }
#pragma unroll
    for (int k = 0; k < NO; k++) DY[(size_t)row * NO + k] = dy[k];
    SE[row] = se;
  }
  // dz1 = (W2^T dz2) * [z1 > 0]
  for (int j = 0; j < NH; j++) {
    float s = 0.f;
#pragma unroll 8
    for (int i = 0; i < NH; i++) s = fmaf(w[OFF_W2 + i * NH + j], dz[i * BWD_T + t], s);
    if (live) DZ1[(size_t)row * NH + j] = h1[j * BWD_T + t] > 0.f ? s : 0.f;
  }
}

// One thread per parameter: gradient = sum over the batch of an outer-product
// entry (weights) or of the pre-activation gradient (biases).
__global__ void k_mlp_wgrad(const float *__restrict__ X, const float *__restrict__ H1, const float *__restrict__ H2,
                            const float *__restrict__ DZ1, const float *__restrict__ DZ2, const float *__restrict__ DY,
                            int B, float *__restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  float s = 0.f;
  if (p < OFF_B1) {
    const int i = p / NI, j = p % NI;
    for (int b = 0; b < B; b++) s = fmaf(DZ1[(size_t)b * NH + i], X[(size_t)b * NI + j], s);
  } else if (p < OFF_W2) {
    const int i = p - OFF_B1;
    for (int b = 0; b < B; b++) s += DZ1[(size_t)b * NH + i];
  } else if (p < OFF_B2) {
    const int i = (p - OFF_W2) / NH, j = (p - OFF_W2) % NH;
    for (int b = 0; b < B; b++) s = fmaf(DZ2[(size_t)b * NH + i], H1[(size_t)b * NH + j], s);
  } else if (p < OFF_W3) {
    const int i = p - OFF_B2;
    for (int b = 0; b < B; b++) s += DZ2[(size_t)b * NH + i];
  } else if (p < OFF_B3) {
    const int k = (p - OFF_W3) / NH, j = (p - OFF_W3) % NH;
    for (int b = 0; b < B; b++) s = fmaf(DY[(size_t)b * NO + k], H2[(size_t)b * NH + j], s);
  } else {
    const int k = p - OFF_B3;
    for (int b = 0; b < B; b++) s += DY[(size_t)b * NO + k];
  }
  grad[p] = s;
}

__global__ void k_mlp_adam(float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_sum(const float *x, int n, float *out) {
  __shared__ float sh[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

size_t fwd_smem() { return sizeof(float) * NPARAM; }
size_t bwd_smem() { return sizeof(float) * (NPARAM + (NPARAM & 1) + 3 * NH * BWD_T); }

cudaError_t configure_mlp() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem());
  if (e == cudaSuccess) done = true;
  return e;
}

}  // namespace

int mlp_num_params() { return NPARAM; }

cudaError_t mlp_forward(const float *params, const float *X, float *Y, const int64_t *n_rows_dev, int64_t max_rows,
                        cudaStream_t st) {
  cudaError_t e = configure_mlp();
  if (e != cudaSuccess) return e;
  if (max_rows <= 0) return cudaSuccess;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  }
  // enough blocks to fill every SM at the resident count; each loops over tiles
  const int64_t tiles = (max_rows + FWD_T - 1) / FWD_T;
  const int64_t blocks = std::min<int64_t>(tiles, (int64_t)sms * FWD_MIN_BLOCKS);
  k_mlp_forward<<<(unsigned)blocks, FWD_T, fwd_smem(), st>>>(params, X, Y, n_rows_dev, max_rows);
  return cudaGetLastError();
}

}  // namespace flash

using namespace flash;

extern "C" {

int32_t flash_mlp_num_params(void) { return NPARAM; }

flash_status flash_mlp_forward(const float *params, const float *x, float *y, int64_t rows, void *stream) {
  if (!params || !x || !y || rows < 0) {
    set_error("flash_mlp_forward: invalid arguments");
    return FLASH_EINVAL;
  }
  FLASH_CUDA_TRY(mlp_forward(params, x, y, nullptr, rows, (cudaStream_t)stream));
  return FLASH_OK;
}

flash_status flash_mlp_loss_grad(const float *params, const float *x, const float *t, int32_t rows, float *grad,
                                 float *loss, float *work, void *stream) {
  if (!params || !x || !t || !grad || !loss || !work || rows <= 0) {
    set_error("flash_mlp_loss_grad: invalid arguments");
    return FLASH_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  FLASH_CUDA_TRY(configure_mlp());
  float *H1 = work, *H2 = H1 + (size_t)rows * NH, *DZ1 = H2 + (size_t)rows * NH, *DZ2 = DZ1 + (size_t)rows * NH;
  float *DY = DZ2 + (size_t)rows * NH, *SE = DY + (size_t)rows * NO;
  k_mlp_fwd_bwd<<<(rows + BWD_T - 1) / BWD_T, BWD_T, bwd_smem(), st>>>(params, x, t, rows, H1, H2, DZ1, DZ2, DY, SE);
  FLASH_CUDA_TRY(cudaGetLastError());
  k_mlp_wgrad<<<(NPARAM + 255) / 256, 256, 0, st>>>(x, H1, H2, DZ1, DZ2, DY, rows, grad);
  FLASH_CUDA_TRY(cudaGetLastError());
  k_sum<<<1, 256, 0, st>>>(SE, rows, loss);
  FLASH_CUDA_TRY(cudaGetLastError());
  return FLASH_OK;
}

int64_t flash_mlp_work_floats(int32_t rows) { return (int64_t)rows * (4 * NH + NO + 1); }

flash_status flash_mlp_adam(float *params, const float *grad, float *m, float *v, int32_t step, float lr,
                            void *stream) {
  if (!params || !grad || !m || !v || step < 1) {
    set_error("flash_mlp_adam: invalid arguments");
    return FLASH_EINVAL;
  }
  const float b1 = 0.9f, b2 = 0.999f;
  k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      params, grad, m, v, lr, b1, b2, 1e-8f, 1.f - powf(b1, (float)step), 1.f - powf(b2, (float)step));
  FLASH_CUDA_TRY(cudaGetLastError());
  return FLASH_OK;
}

}  // extern "C"
