// Tensor-core global solve for sm_103a: the dense multi-RHS apply
//   OUT[:, j] = A^-1 * RHS[:, j]   over all columns j = (environment, coord)
// of a group -- the "S^T S g" applies of Algorithm 1 done with the explicit
// inverse of the constant system matrix shared by every environment.
//
// Precision: A^-1 and every RHS column are split into f16 hi + lo parts with
// power-of-two scales (A^-1 by 2^a_exp once at setup, each RHS column by its
// own scale), and three tcgen05.mma products hi*hi + hi*lo + lo*hi accumulate
// in FP32 in tensor memory, which keeps ~21 significant bits: enough for the
// correction form q^k = q^{k-1} + A^-1 r, whose error against the FP64
// oracle must stay below 1e-5 m.
//
// K halves: every apply sums k < n/2 and k >= n/2 into two separate FP32
// accumulators and adds the two in the epilogue.  A tile runs either on one
// CTA (both accumulators in its TMEM) or on two CTAs, one half each
// (split-K): each writes its accumulator to a global scratch tile and counts
// itself in the tile's arrival counter, and the second to arrive adds the
// first's partial to its own.  FP32 addition of two values is commutative,
// so both forms give bit-identical results and the choice can be timed.
//
// Structure (one 128 x BN output tile per CTA or CTA pair, 128 threads;
// BN = 64, 128, 176 or 256 columns and the split, chosen per column range
// by timing the candidates on the group's own matrix when the scene is
// finalised):
//   warp 0 lane 0  TMA producer: 4 tiles (A hi/lo 128 x 64, B hi/lo BN x 64
//                  f16) per k-block into a 2..4-stage ring, 128B swizzle; the
//                  last column tile may run past the matrix (zero fill)
//   warp 1 lane 0  MMA issuer: 4 k-slices x 3 products of M128 N(BN) K16,
//                  tcgen05.commit frees the stage / signals the epilogue
//   warp 2         allocates / frees the TMEM columns
//   all 4 warps    epilogue: tcgen05.ld 32 lanes x 32 (or 16) columns at a
//                  time, rescale, coalesced column stores of live columns
// Every mbarrier wait is bounded; on timeout the CTA raises an error flag,
// drains what it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "flash_internal.cuh"

namespace flash {
namespace {

constexpr int BM = 128, BK = 64;
constexpr int TILE_A = BM * BK * 2;   // bytes of one f16 A tile (16 KiB)
constexpr long long WAIT_CYCLES = 4000000000ll;  // ~2 s of SM clock before a wait is declared hung

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// bounded wait on the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit = WAIT_CYCLES) {
  uint32_t addr = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, uint64_t *bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)2 << 61;                        // 128B swizzle
  return d;
}

// instruction descriptor: kind::f16, A = B = f16 (or both bf16), D = f32,
// both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool bf16 = false) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// tile configuration: B tile bytes, ring depth that fits 227 KB, TMEM columns
template <int BN> struct TileCfg {
  static constexpr int TILE_B = BN * BK * 2;
  static constexpr int STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;
  static constexpr int STAGES = (227 * 1024 - 2048) / STAGE_BYTES > 4 ? 4 : (227 * 1024 - 2048) / STAGE_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
  static constexpr int TMEM_COLS = BN <= 64 ? 64 : BN <= 128 ? 128 : 256;          // one accumulator
  static constexpr int TMEM_COLS2 = 2 * BN <= 128 ? 128 : 2 * BN <= 256 ? 256 : 512;  // both K halves
  static_assert(BN % 16 == 0 && BN >= 64 && BN <= 256, "tcgen05 M128 needs N in [16, 256], multiple of 16");
  static_assert(TILE_B % 1024 == 0, "128B-swizzled tiles start on 1 KiB boundaries");
  static_assert(STAGES >= 2, "ring needs two stages");
};

// 32 lanes x 32 (X = 32) or 16 (X = 16) consecutive TMEM columns into registers
template <int X> __device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t *v);
template <> __device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, uint32_t *v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
        "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
        "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
template <> __device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, uint32_t *v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// epilogue of X accumulated columns starting at tile column c0: rescale and
// store the live ones
template <int X>
__device__ __forceinline__ void store_cols(const float *v, float *o, const float *wv, int n_pad, int mode, float lr,
                                           const float *col_scale, const float *col_k, const int *col_live, int c0) {
  if (mode == 2) {
#pragma unroll
    for (int j = 0; j < X; j++)
      if (col_live[c0 + j]) o[(size_t)j * n_pad] = v[j] * col_scale[c0 + j] / (1.f + col_k[c0 + j] * lr);
  } else if (mode == 0) {
#pragma unroll
    for (int j = 0; j < X; j++)
      if (col_live[c0 + j]) o[(size_t)j * n_pad] = v[j] * col_scale[c0 + j];
  } else if (mode == 3) {   // accumulate: a refinement step's correction
#pragma unroll
    for (int j = 0; j < X; j++)
      if (col_live[c0 + j]) o[(size_t)j * n_pad] += v[j] * col_scale[c0 + j];
  } else {
    float prev[X];
#pragma unroll
    for (int j = 0; j < X; j++) prev[j] = col_live[c0 + j] ? o[(size_t)j * n_pad] + wv[(size_t)j * n_pad] : 0.f;
#pragma unroll
    for (int j = 0; j < X; j++)
      if (col_live[c0 + j]) o[(size_t)j * n_pad] = prev[j] + v[j] * col_scale[c0 + j];
  }
}

// The tile's sum of both K halves for X columns at tile column c0 of this
// thread's row: both TMEM accumulators (one CTA), or this CTA's accumulator
// plus the other CTA's partial from the scratch tile (split-K, last arrival).
template <int X>
__device__ __forceinline__ void tile_sum(uint32_t tbase, int two_acc, int bn, const float *other, float *v) {
  uint32_t a[X];
  tmem_ld<X>(tbase, a);
  if (two_acc) {
    uint32_t b[X];
    tmem_ld<X>(tbase + (uint32_t)bn, b);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < X; j++) v[j] = __uint_as_float(a[j]) + __uint_as_float(b[j]);
  } else {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < X; j++) v[j] = __uint_as_float(a[j]) + __ldcg(other + (size_t)j * BM);
  }
}

// this CTA's accumulator for X columns at tile column c0 into the scratch tile
template <int X>
__device__ __forceinline__ void tile_spill(uint32_t tbase, float *mine) {
  uint32_t a[X];
  tmem_ld<X>(tbase, a);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < X; j++) mine[(size_t)j * BM] = __uint_as_float(a[j]);
}

// One 128 x BN output tile at rows m0.., columns j0.. (tensor maps in
// parameter or global memory).  nsplit = 1: both K halves on this CTA;
// nsplit = 2: half ksplit only, with the scratch tiles part (two per tile,
// [2][BN][128] floats) and the arrival counter sem of tile tile_id.
template <int BN, bool BF = false>
__device__ __forceinline__ void gemm_tile(const CUtensorMap *pAh, const CUtensorMap *pAl, const CUtensorMap *pBh,
                                          const CUtensorMap *pBl, float *__restrict__ out,
                                          const float *__restrict__ W, const float *__restrict__ rscale,
                                          const int *__restrict__ done, const int *__restrict__ genv, int *status,
                                          int n_pad, int m0, int j0, int cols, float a_unscale, int mode,
                                          const float *__restrict__ lam, const float *__restrict__ kenv,
                                          int nsplit = 1, int ksplit = 0, float *part = nullptr, int *sem = nullptr,
                                          int tile_id = 0) {
  using Cfg = TileCfg<BN>;
  constexpr int STAGES = Cfg::STAGES, STAGE_BYTES = Cfg::STAGE_BYTES, TILE_B = Cfg::TILE_B;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int fail_sh, last_sh;
  __shared__ float col_scale[BN];
  __shared__ float col_k[BN];
  __shared__ int col_live[BN];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KB = n_pad / BK, KH = KB / 2;   // n_pad is a multiple of 128: KB is even
  const int kb0 = nsplit == 2 ? ksplit * KH : 0, kb1 = nsplit == 2 ? kb0 + KH : KB;
  const uint32_t tmem_cols = nsplit == 2 ? Cfg::TMEM_COLS : Cfg::TMEM_COLS2;
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

  // skip tiles whose environments have all converged (their columns are
  // never read again in this step)
  {
    int live = 0;
    for (int c = j0 + threadIdx.x; c < min(j0 + BN, cols); c += blockDim.x) live |= !done[genv[c / 3]];
    if (!__syncthreads_or(live)) return;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fail_sh = 0;
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int i = 0;   // k-blocks issued
    for (; kb0 + i < kb1; i++) {
      const int s = i % STAGES;
      if (!mbar_wait(&empty_bar[s], ((i / STAGES) & 1) ^ 1)) { atomicExch(&fail_sh, 1); break; }
      uint8_t *st = smem + s * STAGE_BYTES;
      const int k0 = (kb0 + i) * BK;
      if constexpr (BF) {   // one bf16 product: the hi slots of the stage only
        mbar_expect_tx(&full_bar[s], TILE_A + TILE_B);
        tma_load_2d(st, pAh, &full_bar[s], k0, m0);
        tma_load_2d(st + 2 * TILE_A, pBh, &full_bar[s], k0, j0);
      } else {
        mbar_expect_tx(&full_bar[s], STAGE_BYTES);
        tma_load_2d(st, pAh, &full_bar[s], k0, m0);
        tma_load_2d(st + TILE_A, pAl, &full_bar[s], k0, m0);
        tma_load_2d(st + 2 * TILE_A, pBh, &full_bar[s], k0, j0);
        tma_load_2d(st + 2 * TILE_A + TILE_B, pBl, &full_bar[s], k0, j0);
      }
    }
    // drain: wait until every stage this thread armed has landed (bounded)
    for (int t = max(0, i - STAGES); t < i; t++) mbar_wait(&full_bar[t % STAGES], (t / STAGES) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: k-blocks below KH into the first
    // accumulator, the others into the second (one CTA), or this CTA's half
    // into its only accumulator (split-K)
    constexpr uint32_t idesc = idesc_f16(BM, BN, BF);
    bool ok = true;
    for (int i = 0; kb0 + i < kb1; i++) {
      const int s = i % STAGES, kb = kb0 + i;
      if (!mbar_wait(&full_bar[s], (i / STAGES) & 1)) { atomicExch(&fail_sh, 1); ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
      const uint32_t ah = base, al = base + TILE_A, bh = base + 2 * TILE_A, bl = base + 2 * TILE_A + TILE_B;
      const uint32_t acc = tmem + ((nsplit == 1 && kb >= KH) ? (uint32_t)BN : 0u);
      const bool first = kb == kb0 || (nsplit == 1 && kb == KH);
#pragma unroll
      for (int ks = 0; ks < BK / 16; ks++) {
        const uint32_t off = ks * 32;   // 16 f16 / bf16 along K inside the 128-byte swizzle row
        mma_f16(acc, smem_desc(ah + off), smem_desc(bh + off), idesc, (first && ks == 0) ? 0u : 1u);
        if constexpr (!BF) {
          mma_f16(acc, smem_desc(ah + off), smem_desc(bl + off), idesc, 1u);
          mma_f16(acc, smem_desc(al + off), smem_desc(bh + off), idesc, 1u);
        }
      }
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&done_bar);
    (void)ok;
  }
  __syncwarp();
  // ---------------- epilogue (all 4 warps; warp w owns TMEM lanes 32w..32w+31)
  // per-column scale (A and RHS unscaling) and liveness, staged once per tile
  for (int c = threadIdx.x; c < BN; c += blockDim.x) {
    const int col = j0 + c;
    const bool in = col < cols;
    col_scale[c] = in ? a_unscale * rscale[col] : 0.f;
    col_k[c] = (in && mode == 2) ? kenv[col / 3] : 0.f;
    col_live[c] = in && (mode != 1 || !done[genv[col / 3]]);
  }
  bool ok = mbar_wait(&done_bar, 0);
  if (!ok) atomicExch(&fail_sh, 1);
  __syncthreads();
  const int rl = warp * 32 + lane;   // this thread's row of the tile (its TMEM lane)
  const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
  const float *other = nullptr;
  bool write_out = true;
  if (nsplit == 2) {
    // split-K: spill this half, count the arrival; the second CTA to arrive
    // owns the output.  A CTA that failed still counts itself, so the
    // counter is back at zero for the next launch.
    float *mine = part + ((size_t)(2 * tile_id + ksplit) * BN) * BM + rl;
    if (!fail_sh) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
      for (int c0 = 0; c0 + 32 <= BN; c0 += 32) tile_spill<32>(tbase + (uint32_t)c0, mine + (size_t)c0 * BM);
      if constexpr (BN % 32 == 16) tile_spill<16>(tbase + (uint32_t)(BN - 16), mine + (size_t)(BN - 16) * BM);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const int old = atomicAdd(sem + tile_id, 1);
      last_sh = old == 1;
      if (old == 1) sem[tile_id] = 0;
    }
    __syncthreads();
    write_out = last_sh != 0;
    if (write_out) __threadfence();
    other = part + ((size_t)(2 * tile_id + 1 - ksplit) * BN) * BM + rl;
  }
  if (fail_sh) {
    if (threadIdx.x == 0) atomicOr(status, 1 << 11);
  } else if (write_out) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int row = m0 + rl;
    const float lr = mode == 2 ? lam[row] : 0.f;
    const int two = nsplit == 1;
    float v[32];
#pragma unroll 1
    for (int c0 = 0; c0 + 32 <= BN; c0 += 32) {
      tile_sum<32>(tbase + (uint32_t)c0, two, BN, other ? other + (size_t)c0 * BM : nullptr, v);
      store_cols<32>(v, out + (size_t)(j0 + c0) * n_pad + row, W ? W + (size_t)(j0 + c0) * n_pad + row : nullptr,
                     n_pad, mode, lr, col_scale, col_k, col_live, c0);
    }
    if constexpr (BN % 32 == 16) {
      constexpr int c0 = BN - 16;
      tile_sum<16>(tbase + (uint32_t)c0, two, BN, other ? other + (size_t)c0 * BM : nullptr, v);
      store_cols<16>(v, out + (size_t)(j0 + c0) * n_pad + row, W ? W + (size_t)(j0 + c0) * n_pad + row : nullptr,
                     n_pad, mode, lr, col_scale, col_k, col_live, c0);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
  }
}

// One group's apply: tile (x, y) covers rows 128 y.. and columns
// c_begin + BN x .. of [c_begin, cols); z is the K half with gridDim.z = 2.
template <int BN, bool BF = false>
__global__ void __launch_bounds__(128, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
              const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
              float *__restrict__ out, const float *__restrict__ W, const float *__restrict__ rscale,
              const int *__restrict__ done, const int *__restrict__ genv, int *status, int n_pad, int c_begin,
              int cols, float a_unscale, int mode, const float *__restrict__ lam, const float *__restrict__ kenv,
              float *part, int *sem) {
  gemm_tile<BN, BF>(&tmAh, &tmAl, &tmBh, &tmBl, out, W, rscale, done, genv, status, n_pad, blockIdx.y * BM,
                    c_begin + blockIdx.x * BN, cols, a_unscale, mode, lam, kenv, (int)gridDim.z, (int)blockIdx.z, part,
                    sem, (int)(blockIdx.y * gridDim.x + blockIdx.x));
}

// One apply of several groups in one launch (uneven batches: every mesh
// template of a lane at once).  Problem p owns tiles [tile0_p, tile0_{p+1});
// its tensor maps live in global memory, encoded once when the scene is
// finalised.  Plain A^-1 applies only (epilogue mode 0).
struct GemmProblem {
  CUtensorMap ah, al, bh, bl;   // 64-byte aligned, 128 bytes each
  const float *rscale;
  const int *genv;
  int n_pad, c_begin, cols, tiles_x, tile0;
  float a_unscale;
};

template <int BN>
__global__ void __launch_bounds__(128, 1)
    k_gemm_tc_grouped(const GemmProblem *__restrict__ P, int nprob, float *const *__restrict__ outs,
                      const int *__restrict__ done, int *status) {
  const int t = blockIdx.x;
  int p = 0;
  while (p + 1 < nprob && P[p + 1].tile0 <= t) p++;
  const GemmProblem &pr = P[p];
  const int local = t - pr.tile0;
  const int tx = local % pr.tiles_x, ty = local / pr.tiles_x;
  gemm_tile<BN>(&pr.ah, &pr.al, &pr.bh, &pr.bl, outs[p], nullptr, pr.rscale, done, pr.genv, status, pr.n_pad,
                ty * BM, pr.c_begin + tx * BN, pr.cols, pr.a_unscale, 0, nullptr, nullptr);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2D f16 tensor [outer][inner] (inner contiguous), box 64 x rows, 128B swizzle
bool make_map(CUtensorMap *tm, const void *ptr, uint64_t inner, uint64_t outer, uint32_t box_rows,
              bool bf16 = false) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {BK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(tm, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && get_encode() != nullptr;
}

namespace {

template <int BN, bool BF>
cudaError_t launch_tile(const Group &g, const SolveMat &M, float *out, const float *w, const int *done, int mode,
                        const float *lam, const float *kenv, cudaStream_t st, int c0, int c1, const SplitK &sk) {
  using Cfg = TileCfg<BN>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(k_gemm_tc<BN, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (g.n_pad % BM != 0 || g.n_pad % BK != 0) return cudaErrorInvalidValue;
  CUtensorMap tmAh, tmAl, tmBh, tmBl;
  if (BF) {   // bf16 matrix and right-hand sides (the rh buffer holds bf16 in this mode)
    if (!M.bf || !make_map(&tmAh, M.bf, g.n_pad, g.n_pad, BM, true) ||
        !make_map(&tmBh, g.rh, g.n_pad, g.cols_pad, BN, true))
      return cudaErrorInvalidValue;
    tmAl = tmAh;
    tmBl = tmBh;
  } else if (!make_map(&tmAh, M.hi, g.n_pad, g.n_pad, BM) || !make_map(&tmAl, M.lo, g.n_pad, g.n_pad, BM) ||
             !make_map(&tmBh, g.rh, g.n_pad, g.cols_pad, BN) || !make_map(&tmBl, g.rl, g.n_pad, g.cols_pad, BN)) {
    return cudaErrorInvalidValue;
  }
  // column tiles cover the live columns; the last may run past the
  // matrix (TMA fills zeros, the epilogue stores only columns < cols)
  const int split = sk.split == 2 ? 2 : 1;
  dim3 grid((c1 - c0 + BN - 1) / BN, g.n_pad / BM, split);
  if (split == 2 && (!sk.part || !sk.sem || (size_t)grid.x * grid.y > sk.tiles ||
                     (size_t)grid.x * grid.y * 2 * BN * BM > sk.part_floats))
    return cudaErrorInvalidValue;
  k_gemm_tc<BN, BF><<<grid, 128, Cfg::SMEM_BYTES, st>>>(tmAh, tmAl, tmBh, tmBl, out, w, g.rscale, done, g.genv,
                                                         g.status, g.n_pad, c0, c1, ldexpf(1.f, -M.exp), mode, lam,
                                                         kenv, sk.part, sk.sem);
  return cudaGetLastError();
}

cudaError_t launch_bn(int bn, const Group &g, const SolveMat &M, float *out, const float *w, const int *done,
                      int mode, const float *lam, const float *kenv, cudaStream_t st, int c0, int c1,
                      bool bf = false, const SplitK &sk = SplitK()) {
  if (c1 < 0) c1 = g.cols;
  if (c0 < 0 || c1 > g.cols || c0 >= c1) return c0 == c1 ? cudaSuccess : cudaErrorInvalidValue;
  if (bf) {
    switch (bn) {
      case 64: return launch_tile<64, true>(g, M, out, w, done, mode, lam, kenv, st, c0, c1, sk);
      case 176: return launch_tile<176, true>(g, M, out, w, done, mode, lam, kenv, st, c0, c1, sk);
      case 256: return launch_tile<256, true>(g, M, out, w, done, mode, lam, kenv, st, c0, c1, sk);
      default: return launch_tile<128, true>(g, M, out, w, done, mode, lam, kenv, st, c0, c1, sk);
    }
  }
  switch (bn) {
    case 64: return launch_tile<64, false>(g, M, out, w, done, mode, lam, kenv, st, c0, c1, sk);
    case 176: return launch_tile<176, false>(g, M, out, w, done, mode, lam, kenv, st, c0, c1, sk);
    case 256: return launch_tile<256, false>(g, M, out, w, done, mode, lam, kenv, st, c0, c1, sk);
    default: return launch_tile<128, false>(g, M, out, w, done, mode, lam, kenv, st, c0, c1, sk);
  }
}

}  // namespace

size_t gemm_problem_bytes() { return sizeof(GemmProblem); }

// Fill one grouped-apply problem (host memory of gemm_problem_bytes()) for
// columns [c0, c1) of group g with matrix M; its tiles start at tile0.
// Returns the problem's tile count, or -1 if the tensor maps cannot be made.
int gemm_problem(void *dst, const Group &g, const SolveMat &M, int c0, int c1, int tile0) {
  if (g.n_pad % BM != 0 || g.n_pad % BK != 0 || c1 <= c0) return -1;
  GemmProblem pr;
  std::memset(&pr, 0, sizeof(pr));
  if (!make_map(&pr.ah, M.hi, g.n_pad, g.n_pad, BM) || !make_map(&pr.al, M.lo, g.n_pad, g.n_pad, BM) ||
      !make_map(&pr.bh, g.rh, g.n_pad, g.cols_pad, kGroupedBN) || !make_map(&pr.bl, g.rl, g.n_pad, g.cols_pad, kGroupedBN))
    return -1;
  pr.rscale = g.rscale;
  pr.genv = g.genv;
  pr.n_pad = g.n_pad;
  pr.c_begin = c0;
  pr.cols = c1;
  pr.tiles_x = (c1 - c0 + kGroupedBN - 1) / kGroupedBN;
  pr.tile0 = tile0;
  pr.a_unscale = ldexpf(1.f, -M.exp);
  std::memcpy(dst, &pr, sizeof(pr));
  return pr.tiles_x * (g.n_pad / BM);
}

namespace {
// The failure path of the bounded waits, run on purpose: one thread waits,
// with the solve's own wait routine and a given cycle limit, on an mbarrier
// that nothing arrives at; the wait runs out and the timeout bit is set, as
// a tensor-core tile does when its wait runs out.
__global__ void k_wait_probe(int *status, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0, limit)) atomicOr(status, 1 << 11);
  }
}
}  // namespace

cudaError_t launch_wait_probe(int *status, long long limit, cudaStream_t st) {
  if (limit <= 0 || limit > WAIT_CYCLES) return cudaErrorInvalidValue;
  k_wait_probe<<<1, 32, 0, st>>>(status, limit);
  return cudaGetLastError();
}

cudaError_t gemm_tc_grouped(const void *probs, int nprob, int tiles, float *const *outs, const int *done, int *status,
                            cudaStream_t st) {
  using Cfg = TileCfg<kGroupedBN>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc_grouped<kGroupedBN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (nprob <= 0 || tiles <= 0) return cudaSuccess;
  k_gemm_tc_grouped<kGroupedBN><<<tiles, 128, Cfg::SMEM_BYTES, st>>>(static_cast<const GemmProblem *>(probs), nprob,
                                                                      outs, done, status);
  return cudaGetLastError();
}

cudaError_t gemm_tc(const Group &g, const SolveMat &M, float *out, const float *w, const int *done, int mode,
                    const float *lam, const float *kenv, cudaStream_t st, int c0, int c1, int bn, bool bf,
                    const SplitK &sk) {
  return launch_bn(bn > 0 ? bn : g.tc_bn, g, M, out, w, done, mode, lam, kenv, st, c0, c1, bf, sk);
}

// Scratch of a split-K apply of columns [c0, c1) of group g, any tile width:
// two [BN][128] partial tiles and one arrival counter per tile.
void splitk_need(const Group &g, int c0, int c1, size_t *tiles, size_t *part_floats) {
  const size_t ty = (size_t)g.n_pad / BM, cols = (size_t)(c1 - c0);
  *tiles = ((cols + 63) / 64) * ty;
  *part_floats = 2 * (cols + 255) * ty * BM;
}

// Tile autotuner: time each candidate tile width (and, with split-K scratch,
// each width run as two K halves on two CTAs) on the group's own matrix and
// column count (the right-hand side is whatever the group holds, zeros at
// setup) and keep the fastest.  Which wins depends on how the tiles of the
// group fill the SMs.
cudaError_t tune_gemm_tc(const Group &g, const int *done, cudaStream_t st, int c0, int c1, int *bn_out,
                         int *split_out, const SplitK &sk) {
  const SolveMat &M = g.eig ? g.Vt : g.inv;
  const int cand[] = {64, 128, 176, 256};
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  float best = 1e30f;
  int best_bn = 128, best_split = 1;
  // sk.split: 0 times both forms, 2 split-K only; no scratch: one CTA per tile
  const int min_split = sk.part && sk.sem && sk.split == 2 ? 2 : 1;
  const int max_split = sk.part && sk.sem ? 2 : 1;
  for (int split = min_split; split <= max_split && e == cudaSuccess; split++)
    for (int bn : cand) {
      SplitK k = sk;
      k.split = split;
      if ((e = launch_bn(bn, g, M, g.w, nullptr, done, 0, nullptr, nullptr, st, c0, c1, false, k)) != cudaSuccess)
        break;
      float t_min = 1e30f;
      for (int r = 0; r < 5 && e == cudaSuccess; r++) {
        // one launch per measurement; the minimum is the least disturbed
        cudaEventRecord(e0, st);
        e = launch_bn(bn, g, M, g.w, nullptr, done, 0, nullptr, nullptr, st, c0, c1, false, k);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        t_min = fminf(t_min, ms);
      }
      if (e != cudaSuccess) break;
      if (t_min < best) { best = t_min; best_bn = bn; best_split = split; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *bn_out = best_bn;
  if (split_out) *split_out = best_split;
  return e;
}

}  // namespace flash
