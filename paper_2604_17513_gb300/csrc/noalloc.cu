// Allocation-free dense apply out = A^-1 * rhs for callers that cannot call
// cudaMalloc.  Its scratch (padded copy of A^-1, column-layout right-hand
// sides and results) lives in one file-scope __device__ array of fixed size,
// which every GPU that loads this library holds until the process exits.
// All calls share that array; calls that overlap on the GPU (different
// streams, or different host threads on the same device) race on it.
#include <mutex>

#include "flash_internal.cuh"

namespace flash {
namespace {

constexpr int kNaMaxNPad = 512;    // largest vertex count, padded to 128
constexpr int kNaMaxCols = 768;    // largest 3 * environments (256 environments)
constexpr size_t kNaA = (size_t)kNaMaxNPad * kNaMaxNPad;
constexpr size_t kNaCols = (size_t)kNaMaxCols * kNaMaxNPad;

// 4 MiB: [A^-1 padded | rhs columns | result columns]
static __device__ __align__(256) float g_noalloc_scratch[kNaA + 2 * kNaCols];

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
float *g_na_ptr[kMaxDevices] = {nullptr};
unsigned long long g_na_ctx[kMaxDevices] = {0};   // context the cached address belongs to

// Unique id of the calling thread's current CUDA context (0 when none is
// current or the driver cannot say).  A device reset destroys the primary
// context and a new one loads this library's module at a new address, so the
// cached symbol address is keyed on this id.  The driver calls are resolved
// through the runtime, so the library still links no libcuda.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q1, q2;
    void *f1 = nullptr, *f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_cur = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
  });
  if (!get_cur || !get_id) return 0;
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// device address of the scratch array for the current device, looked up with
// that device current on its first use and again whenever its context has
// changed since (after a device reset); with no context id available it is
// looked up on every call
cudaError_t scratch_for_current_device(float **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_na_ptr[dev] || ctx == 0 || ctx != g_na_ctx[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<float *>(p);
    g_na_ctx[dev] = current_context_id();   // the lookup made the primary context current
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

// copy the transpose of A^-1 [n][n] (row-major) into the zero-padded
// [n_pad][n_pad] block: the CUDA-core contraction reads its matrix operand
// along rows and forms M^T * RHS, so it is given M = (A^-1)^T and returns
// A^-1 * RHS for any square matrix, symmetric or not
__global__ void k_na_pad_matrix(const float *A, int n, int n_pad, float *Ap) {
  const size_t total = (size_t)n_pad * n_pad;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n_pad), j = (int)(t % n_pad);
    Ap[t] = (i < n && j < n) ? A[(size_t)j * n + i] : 0.f;
  }
}

// user [m][n][3] -> columns [cols_pad][n_pad]; padding rows and columns zeroed
__global__ void k_na_to_cols(const float *rhs, int n, int m, int n_pad, int cols_pad, float *cols) {
  const size_t total = (size_t)cols_pad * n_pad;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int col = (int)(t / n_pad), i = (int)(t % n_pad);
    const int env = col / 3, c = col % 3;
    cols[t] = (env < m && i < n) ? rhs[((size_t)env * n + i) * 3 + c] : 0.f;
  }
}

// columns [cols][n_pad] -> user [m][n][3]
__global__ void k_na_from_cols(const float *cols, int n, int m, int n_pad, float *out) {
  const size_t total = (size_t)m * n * 3;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % 3);
    const size_t vi = t / 3;
    const int i = (int)(vi % n), env = (int)(vi / n);
    out[t] = cols[(size_t)(env * 3 + c) * n_pad + i];
  }
}

}  // namespace
}  // namespace flash

extern "C" flash_status flash_dense_apply_noalloc(const float *Ainv, int32_t n, int32_t m, const float *rhs, float *out,
                                                  void *stream) {
  using namespace flash;
  if (!Ainv || !rhs || !out || n <= 0 || m <= 0) {
    set_error("flash_dense_apply_noalloc: null pointer or non-positive size");
    return FLASH_EINVAL;
  }
  const int n_pad = (n + 127) / 128 * 128;
  const int cols = 3 * m;
  const int cols_pad = (cols + 127) / 128 * 128;
  if (n_pad > kNaMaxNPad || cols_pad > kNaMaxCols) {
    set_error("flash_dense_apply_noalloc: size beyond the fixed scratch (at most 512 vertices and 256 "
              "environments per call)");
    return FLASH_EINVAL;
  }
  float *base = nullptr;
  FLASH_CUDA_TRY(scratch_for_current_device(&base));
  float *Ap = base, *B = base + kNaA, *C = base + kNaA + kNaCols;
  cudaStream_t st = (cudaStream_t)stream;
  k_na_pad_matrix<<<256, 256, 0, st>>>(Ainv, n, n_pad, Ap);
  FLASH_CUDA_TRY(cudaGetLastError());
  k_na_to_cols<<<256, 256, 0, st>>>(rhs, n, m, n_pad, cols_pad, B);
  FLASH_CUDA_TRY(cudaGetLastError());
  FLASH_CUDA_TRY(gemm_simt_raw(Ap, B, C, n_pad, cols, st));
  k_na_from_cols<<<256, 256, 0, st>>>(C, n, m, n_pad, out);
  FLASH_CUDA_TRY(cudaGetLastError());
  return FLASH_OK;
}
