// FP32 dense global solve on the CUDA cores (baseline path and reference for
// the tensor-core path):  OUT[:, j] = A^-1 * RHS[:, j] for every column j of
// a group (one column per environment and coordinate), i.e. the
// "S^T S g" applies of Algorithm 1 done with the explicit dense inverse.
//
// Tiles: 128 rows x 128 columns x 16 k per CTA, 256 threads, 8x8 outputs per
// thread.  The matrix tile is read along its rows (coalesced), so the kernel
// computes M^T * RHS: equal to M * RHS for the symmetric A^-1; the eigen-form
// solve passes V to get V^T * RHS and V^T to get V * RHS.
// Epilogue mode 1 adds the previous iterate and the first solve:
//   q^k = q^{k-1} + w + A^-1 J^T dgamma   (Eq. correction in correction form).
#include "flash_internal.cuh"

namespace flash {
namespace {

constexpr int BM = 128, BN = 128, BK = 16;

__global__ void __launch_bounds__(256) k_gemm_f32(const float *__restrict__ A, const float *__restrict__ B,
                                                  float *__restrict__ C, const float *__restrict__ W,
                                                  const int *__restrict__ done, const int *__restrict__ genv,
                                                  int n_pad, int c0, int cols, int mode,
                                                  const float *__restrict__ lam, const float *__restrict__ kenv) {
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  // columns [c0, cols) of the buffers; tiles past `cols` read zeros
  const int m0 = blockIdx.y * BM, j0 = c0 + blockIdx.x * BN;
  const int tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; i++)
#pragma unroll
    for (int j = 0; j < 8; j++) acc[i][j] = 0.f;

  // loader mapping: A tile 16 x 128 floats = 512 float4, 2 per thread
  //                 B tile 128 cols x 16 k = 512 float4, 2 per thread
  auto load = [&](int buf, int k0) {
#pragma unroll
    for (int t = 0; t < 2; t++) {
      int idx = tid + t * 256;
      int kr = idx >> 5, mc = (idx & 31) * 4;
      float4 va = *reinterpret_cast<const float4 *>(A + (size_t)(k0 + kr) * n_pad + m0 + mc);
      *reinterpret_cast<float4 *>(&As[buf][kr][mc]) = va;
      int jc = idx >> 2, kq = (idx & 3) * 4;
      const float4 vb = j0 + jc < cols ? *reinterpret_cast<const float4 *>(B + (size_t)(j0 + jc) * n_pad + k0 + kq)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
      Bs[buf][kq + 0][jc] = vb.x;
      Bs[buf][kq + 1][jc] = vb.y;
      Bs[buf][kq + 2][jc] = vb.z;
      Bs[buf][kq + 3][jc] = vb.w;
    }
  };
  load(0, 0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < n_pad; k0 += BK) {
    if (k0 + BK < n_pad) load(buf ^ 1, k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; kk++) {
      float a[8], b[8];
      float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
      b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int j = 0; j < 8; j++) {
    int col = j0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
    if (col >= cols) continue;
    if (done && done[genv[col / 3]]) continue;
    float *c = C + (size_t)col * n_pad;
    const float *w = W + (size_t)col * n_pad;
    const float ke = mode == 2 ? kenv[col / 3] : 0.f;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      int row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
      if (mode == 0) c[row] = acc[i][j];
      else if (mode == 2) c[row] = acc[i][j] / (1.f + ke * lam[row]);
      else c[row] = c[row] + w[row] + acc[i][j];
    }
  }
}

}  // namespace

cudaError_t gemm_simt(const Group &g, const SolveMat &M, const float *rhs, float *out, const float *w,
                      const int *done, int mode, const float *lam, const float *kenv, cudaStream_t st, int c0, int c1) {
  if (c1 < 0) c1 = g.cols;
  if (c0 < 0 || c1 > g.cols || c0 >= c1) return c0 == c1 ? cudaSuccess : cudaErrorInvalidValue;
  dim3 grid((c1 - c0 + BN - 1) / BN, g.n_pad / BM);
  k_gemm_f32<<<grid, 256, 0, st>>>(M.f32, rhs, out, w, done, g.genv, g.n_pad, c0, c1, mode, lam, kenv);
  return cudaGetLastError();
}

// Plain launch of the FP32 apply on caller-provided, already padded buffers
// (A^-1 [n_pad][n_pad], B and C [cols rounded up to 128][n_pad]).
cudaError_t gemm_simt_raw(const float *Ainv, const float *rhs, float *out, int n_pad, int cols, cudaStream_t st) {
  dim3 grid((cols + BN - 1) / BN, n_pad / BM);
  k_gemm_f32<<<grid, 256, 0, st>>>(Ainv, rhs, out, nullptr, nullptr, nullptr, n_pad, 0, cols, 0, nullptr, nullptr);
  return cudaGetLastError();
}

}  // namespace flash
