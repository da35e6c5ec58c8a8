// One-time setup on the device (Algorithm 1 lines 1-2: factorise the
// constant system matrix once).  A is SPD, so Gauss-Jordan elimination
// without pivoting is stable; it is run in FP64 in place, a batch of
// matrices of equal size at once (one launch pair per pivot), and the result
// is cast to the FP32 copy and the scaled f16 hi/lo split used by the
// per-iteration global solves.
#include "flash_internal.cuh"

namespace flash {
namespace {

__global__ void k_gj_prep(const double *A, int n_pad, int k, double *rowk, double *colk) {
  const int b = blockIdx.y;
  const double *M = A + (size_t)b * n_pad * n_pad;
  const double p = M[(size_t)k * n_pad + k];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_pad; j += gridDim.x * blockDim.x) {
    rowk[(size_t)b * n_pad + j] = (j == k ? 1.0 : M[(size_t)k * n_pad + j]) / p;
    colk[(size_t)b * n_pad + j] = M[(size_t)j * n_pad + k];
  }
}

__global__ void k_gj_update(double *A, int n_pad, int k, const double *rowk, const double *colk) {
  const int b = blockIdx.z;
  double *M = A + (size_t)b * n_pad * n_pad;
  const int i = blockIdx.y;
  const double ci = colk[(size_t)b * n_pad + i];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_pad; j += gridDim.x * blockDim.x) {
    double rj = rowk[(size_t)b * n_pad + j];
    if (i == k) M[(size_t)i * n_pad + j] = rj;
    else M[(size_t)i * n_pad + j] = (j == k ? 0.0 : M[(size_t)i * n_pad + j]) - ci * rj;
  }
}

__global__ void k_cast(const double *A, size_t count, float *A32, __half *hi, __half *lo, __nv_bfloat16 *bf,
                       float scale) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    double x = A[i];
    A32[i] = (float)x;
    if (bf) bf[i] = __float2bfloat16_rn((float)(x * scale));
    if (hi) {
      float xs = (float)(x * scale);
      __half h = __float2half_rn(xs);
      hi[i] = h;
      lo[i] = __float2half_rn(xs - __half2float(h));
    }
  }
}

}  // namespace

cudaError_t invert_spd_f64(double *A, int n, int n_pad, int batch, cudaStream_t st) {
  (void)n;
  double *rowk = nullptr, *colk = nullptr;
  cudaError_t err = cudaMallocAsync(&rowk, sizeof(double) * n_pad * batch, st);
  if (err != cudaSuccess) return err;
  err = cudaMallocAsync(&colk, sizeof(double) * n_pad * batch, st);
  if (err != cudaSuccess) return err;
  int tpb = 256;
  int bx = (n_pad + tpb - 1) / tpb;
  for (int k = 0; k < n_pad; k++) {
    k_gj_prep<<<dim3(bx, batch), tpb, 0, st>>>(A, n_pad, k, rowk, colk);
    k_gj_update<<<dim3(bx, n_pad, batch), tpb, 0, st>>>(A, n_pad, k, rowk, colk);
  }
  err = cudaGetLastError();
  cudaFreeAsync(rowk, st);
  cudaFreeAsync(colk, st);
  return err;
}

cudaError_t cast_inverse(const double *A64, int n_pad, float *A32, __half *hi, __half *lo, int a_exp,
                         cudaStream_t st, __nv_bfloat16 *bf) {
  size_t count = (size_t)n_pad * n_pad;
  k_cast<<<1024, 256, 0, st>>>(A64, count, A32, hi, lo, bf, ldexpf(1.f, a_exp));
  return cudaGetLastError();
}

}  // namespace flash
