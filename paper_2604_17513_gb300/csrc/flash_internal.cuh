// Internal declarations of the FLASH CUDA library (not part of the C ABI).
//
// Device layout, per group of environments sharing one system matrix
// (same mesh, same stiffness scale):
//   state      float [N_g][3][n_pad]   one contiguous column per (env, coord),
//                                      so the global solve is a multi-RHS
//                                      product  A^-1 [n_pad x n_pad] * R [n_pad x 3N_g]
//   elements   int   [E][4], float D[E][12] (F[c][j] = sum_a x_a[c] D[a][j]),
//              float wt[E] = h^2 * w_i
//   hinges     int   [H][4], float hc[H][4]  (bending stencil scaled by h sqrt(w_b s))
//   incidence  CSR vertex -> element slot (4e + a) and vertex -> hinge slot
//   contacts   per env, sorted by (vertex, obstacle): vert, obs, gamma[4]
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/flash.h"

namespace flash {

constexpr int kMaxPerVertex = 4; // contacts solved jointly on one vertex
constexpr int kMaxBeginSmem = 160 * 1024;   // self-contact triangle and edge boxes in the begin kernel
constexpr int kFmW = 8;          // floats per self-contact row of the full metric's fm_w
constexpr float kDamp = 1e-6f;   // Newton-step damping of the per-vertex block
constexpr int kBigMesh = 2048;   // meshes with more vertices get 1024-thread local-pass CTAs

struct MeshTemplate {
  int type = 0, n = 0, E = 0;
  std::vector<double> rest, mass;
  std::vector<int> elems;
  double w_stretch = 0, w_bend = 0;
  double thickness = -1;
};

// a matrix the global solve applies: FP32 copy for the CUDA-core path and
// f16 hi/lo split scaled by 2^exp for the tensor-core path ([n_pad][n_pad])
struct SolveMat {
  float *f32 = nullptr;
  __half *hi = nullptr, *lo = nullptr;
  __nv_bfloat16 *bf = nullptr;   // bf16 copy scaled by 2^exp (FLASH_SOLVE_BF16R)
  int exp = 0;
};

struct Group {
  int mesh = 0;
  float stiff = 1.f;
  float tau = 0.f;     // contact thickness of this group's mesh
  int n = 0, n_pad = 0, E = 0, H = 0, vpe = 3, nc = 2, type = 0;
  int N = 0;           // environments in the group
  int cols = 0;        // 3 * N
  int cols_pad = 0;    // columns allocated (multiple of 128)
  std::vector<int> env_ids;   // group-local -> global env
  // mesh data (device)
  int *genv = nullptr;        // [N] global env index
  int *elems = nullptr;       // [E][4]
  float *D = nullptr;         // [E][12]
  float *wt = nullptr;        // [E]
  // triangle meshes: one 32-byte record per element for the local pass,
  // {v0, v1, v2 (int bits), weight}, {D[1][0], D[1][1], D[2][0], D[2][1]}
  // (row 0 of the operator is -(row 1 + row 2): it annihilates translations)
  float4 *erec = nullptr;     // [E][2]
  // element -> vertex forces are summed per vertex through CSR tables over
  // the slots e * vpe + a (element e, local vertex a), in incidence order
  uint16_t *coff = nullptr;   // [n + 1, padded to even] slot offsets
  uint16_t *cidx = nullptr;   // [E * vpe, padded to even] slots
  int ev = 0;                 // E * vpe
  // bending as a constant operator K_b (rows sum to zero), off-diagonal
  // entries in pairs, pair-major: entries 2p and 2p + 1 of vertex i at
  // [p * n_pad + i] = {j, K_ij bits, j', K_ij' bits}; empty entries are {i, 0}
  int4 *kb = nullptr;
  int deg_b = 0;
  float *mass = nullptr;      // [n]
  // explicit inverse (groups with one stiffness) ...
  SolveMat inv;
  // ... or, for per-environment stiffness k_e on a mesh without bending, the
  // eigenbasis of (L, M): A_e^-1 = V diag(1 / (1 + k_e lambda)) V^T
  bool eig = false;
  SolveMat V, Vt;
  float *lam = nullptr;                   // [n_pad] eigenvalues (0 in the padding)
  float *kenv = nullptr;                  // [N] stiffness scale of each environment
  float *y = nullptr;                     // [cols_pad][n_pad] eigen-coordinates (intermediate)
  // state (device) [cols_pad][n_pad]
  float *q = nullptr, *v = nullptr, *qt = nullptr, *qp = nullptr;
  float *r = nullptr, *w = nullptr, *f = nullptr;
  float *dq = nullptr;                    // A^-1 J^T dgamma (second global solve)
  __half *rh = nullptr, *rl = nullptr;    // split RHS for the tensor-core path
  float *rscale = nullptr;                // [cols_pad] power-of-two column scale
  // contacts (device)
  int *ccount = nullptr, *cvert = nullptr, *cobs = nullptr;
  float *cgam = nullptr;
  int *pcount = nullptr, *pvert = nullptr, *pobs = nullptr;
  float *pgam = nullptr;
  uint8_t *gflag = nullptr;               // [N][n_pad] grasped vertices (S_grip)
  // cloth self-collision (triangle meshes of a scene with self_collide)
  int self = 0;                           // multi-vertex rows possible (self contacts or box features)
  int selfc = 0, ofeat = 0;               // detection of self contacts / of box-feature rows
  int *ctri = nullptr, *pctri = nullptr;  // [N][cap] feature of each multi-vertex row, -1 otherwise
  float *fm_w = nullptr;                  // [N][cap][8] full metric: weights, effective mass, vertices 1..3
  int ned = 0;                            // unique edges (a < b) in (a, b) order
  int2 *edges = nullptr;                  // [ned]
  int *eoff = nullptr;                    // [n + 1] edges owned by vertex a: eoff[a] .. eoff[a + 1]
  int3 *rtris = nullptr;                  // [rT] surface triangles for ray casting
  int rT = 0;
  int tc_bn = 128;                        // tensor-core tile width (columns), set by the tile autotuner
  // full contact metric (flash_scene_desc.metric = FLASH_METRIC_FULL)
  float *fm_lin = nullptr, *fm_V = nullptr, *fm_H = nullptr, *fm_cs = nullptr, *fm_sn = nullptr, *fm_g = nullptr;
  float *fm_beta = nullptr, *fm_adiag = nullptr, *fm_u = nullptr;
  int *fm_jm = nullptr;
  int fm_m = 0, fm_adiag_stride = 0;
  size_t smem_local = 0;
  bool c_in_smem = true;                  // element forces and CSR tables in shared memory
  float *cscratch = nullptr;              // element forces [N][ev + 1][3] when they do not fit
  int *status = nullptr;                  // scene status word (device)
  // learned warm start / recording (allocated on first use)
  int64_t *row_off = nullptr;             // [N + 1] compact contact rows
  float *feat = nullptr, *pred = nullptr, *targ = nullptr;   // [N * cap][10|6|6]
};

}  // namespace flash

namespace flash {
// Split-K launch of a tensor-core apply: split 2 runs the two K halves of
// each tile on two CTAs, which meet through the scratch partial tiles and
// per-tile arrival counters (zero between launches); split 1 needs none.
struct SplitK {
  int split = 1;
  float *part = nullptr;   // [tiles][2][BN][128]
  int *sem = nullptr;      // [tiles]
  size_t tiles = 0, part_floats = 0;
};
// One table launch over the environments of several groups: CTA b works on
// environment map[b].y of group map[b].x (a row of the scene's group table).
struct Batch {
  int vpe = 0;            // vertices per element of its groups (local pass only)
  int threads = 512;      // local pass: threads per CTA, one environment each (256, 512 or 1024)
  int blocks = 0;         // CTAs, one per environment
  size_t smem = 0;        // dynamic shared memory per CTA: the largest need of its groups
  int2 *map = nullptr;    // device [blocks]
};
// Environments [l0, l1) of one group: columns 3 l0 .. 3 l1 of its solves.
struct LaneRange {
  int group = 0, l0 = 0, l1 = 0;
  int tc_bn = 128;        // tensor-core tile width for this column range (autotuned)
  int tc_split = 1;       // 2: each tile's K halves on two CTAs (autotuned)
};
// A lane: a partition of the environments stepped on its own stream, so
// that the wave tails of one lane's kernels overlap other lanes' work.
// Results do not depend on the partition.
// Every dense-inverse apply of a lane in one tensor-core launch (grouped
// apply): problem table (device) and, per output kind (0: w, 1: dq, 2: the
// full metric's fm_u), the output buffer of each problem (device).
struct GroupedApply {
  void *probs = nullptr;
  int n = 0, tiles = 0;
  float **outs[3] = {nullptr, nullptr, nullptr};
  std::vector<int> ranges;      // the lane's ranges it covers
};
struct Lane {
  cudaStream_t st = nullptr;    // null: the caller's stream (single-lane scenes)
  cudaEvent_t done = nullptr;   // join event
  cudaStream_t body_st = nullptr;   // the lane's stream while the tolerance loop's body is captured
  std::vector<LaneRange> ranges;
  Batch all;                    // begin / NCP / end over the lane's environments
  std::vector<Batch> local;     // local pass, by element type and shared-memory class
  size_t ncp_smem_tc = 0;
  int ncp_threads = 256;        // lite NCP pass: threads per CTA, one environment each (128, 256 or 512)
  SplitK sk;                    // split-K scratch of the lane's applies (they run in stream order)
  GroupedApply ga;
};
}  // namespace flash

struct flash_scene {
  flash_scene_desc d{};
  std::vector<flash::MeshTemplate> meshes;
  std::vector<flash_env_desc> envs;
  std::vector<int> env_mesh;
  std::vector<flash::Group> groups;
  std::vector<int> env_group, env_local;
  std::vector<int64_t> voff;   // host [N+1]
  int N = 0, K = 0, cap = 0;
  bool finalized = false;
  // env-level device arrays
  float *mu = nullptr;
  int *otype = nullptr;
  float *odims = nullptr, *ocomp = nullptr;
  float *pose_t = nullptr, *pose_th = nullptr;   // [N][FLASH_MAX_OBS][7]
  int *iters = nullptr, *done = nullptr;
  float *rncp = nullptr;
  // bilateral grasp per environment: state 0 none, 1 activate at the next
  // step's start, 2 held, 3 release at the next step's start; the obstacle
  // carrying the anchor (-1 none); anchor xyz and activation radius
  int *gstate = nullptr, *gobs = nullptr, *greq = nullptr;
  float *ganchor = nullptr;   // [N][4]
  unsigned long long *rc_keys = nullptr;   // ray casting work buffer
  size_t rc_keys_n = 0;
  int rc_tag = 0;                          // frame tag of the next render
  size_t begin_smem = 0;                   // begin kernel's triangle boxes (self-collision scenes)
  void *rc_prep = nullptr;                 // per-environment view constants
  int *status = nullptr;      // device status word
  int *active = nullptr;      // device counter of environments still iterating
  int *h_active = nullptr;    // pinned host mirror
  int *kit = nullptr;         // device iteration index of the graphed tolerance loop
  unsigned long long *trips = nullptr;   // device count of that loop's body runs (launch accounting)
  int64_t *d_voff = nullptr;
  std::vector<void *> allocs;
  // launch accounting
  int64_t launches = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<int> ev_kind;   // kind of each recorded pair
  float *mlp_params = nullptr;   // warm-start network (device, flat)
  float *ws_bounds = nullptr;    // warm-start input range [lo 10][hi 10] (device)
  int use_dq = 0;
  bool record = false;
  double prof_ms[FLASH_NUM_KINDS] = {0};
  int64_t prof_n[FLASH_NUM_KINDS] = {0};
  // per-environment kernels run as table launches (CTA -> group, environment)
  // over the environments of a lane; lanes step concurrently on their streams
  void *gtab = nullptr;                        // device table of group views
  std::vector<flash::Lane> lanes;
  cudaEvent_t fork_ev = nullptr;
  // captured FLASH_MODE_FIXED step, replayed by flash_step
  cudaStream_t cap_st = nullptr;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_launches = 0;   // kernels in one replay (outside a tolerance loop's body)
  int64_t body_launches = 0;    // kernels in one run of the tolerance loop's body
  cudaStream_t body_st = nullptr;   // captures the tolerance loop's body
  bool capturing = false;       // step_once is being captured
  bool tune_pending = false;    // threads per environment still to be timed (first step)
  bool graph_stale = true;      // a setting that changes the step's launches has changed
  bool grouped = false;         // lanes apply their dense inverses in one grouped launch (chosen at finalize)
};

namespace flash {

// error handling ---------------------------------------------------------
void set_error(const std::string &msg);
#define FLASH_CUDA_TRY(expr)                                                     \
  do {                                                                           \
    cudaError_t e_ = (expr);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      ::flash::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));    \
      return FLASH_ECUDA;                                                        \
    }                                                                            \
  } while (0)

// kernel launchers (step_kernels.cu) ---------------------------------------
struct StepArgs {
  float h, gx, gy, gz, tol, gmax, tau, margin;
  int k_min, k_cap, mode, warm, K, cap;
};
cudaError_t configure_kernels();
cudaError_t launch_row_offsets(const Group &g, int64_t *off, cudaStream_t st);
cudaError_t launch_features(const flash_scene *s, const Group &g, const StepArgs &a, const int64_t *off, float *X,
                            cudaStream_t st);
cudaError_t launch_apply_learned(const flash_scene *s, const Group &g, const StepArgs &a, const int64_t *off,
                                 const float *X, const float *Y, const float *bounds, int flags, cudaStream_t st);
cudaError_t launch_targets(const flash_scene *s, const Group &g, const StepArgs &a, const int64_t *off, float *T,
                           cudaStream_t st);
int mlp_num_params();
cudaError_t mlp_forward(const float *params, const float *X, float *Y, const int64_t *n_rows_dev, int64_t max_rows,
                        cudaStream_t st);
cudaError_t launch_state_io(const flash_scene *s, const Group &g, const float *q_user, const float *v_user,
                            float *q_out, float *v_out, int to_user, cudaStream_t st);
cudaError_t launch_rhs_io(const Group &g, const int64_t *voff, int first_env, const float *user, float *cols,
                          int to_user, cudaStream_t st);
// f16 hi/lo split of the columns of environments [l0, l1) of src (l1 < 0: all)
cudaError_t launch_split_rhs(const Group &g, const float *src, cudaStream_t st, int l0 = 0, int l1 = -1,
                             bool bf16 = false);
// bf16 solve with refinement: for environments [l0, l1) of a tet group, the
// residual rhs32 - A w in FP32 from the element operators, written as the
// next apply's bf16 right-hand sides (rh) with their column scales
cudaError_t launch_refine(const flash_scene *s, const Group &g, const float *rhs32, const float *w, int l0, int l1,
                          cudaStream_t st);
// lanes and their table launches (build_lanes at finalize)
cudaError_t build_lanes(flash_scene *s, int n_lanes);
cudaError_t launch_begin_lane(const flash_scene *s, const Lane &L, const StepArgs &a, cudaStream_t st);
// ray casting (raycast.cu) -------------------------------------------------
struct RcCam {
  int W, H;
  float fx, fy, cx, cy, zn, zf;
};
// vertex positions of the environments of one mesh: vertex i, coordinate c
// of source environment l at x[l * env_stride + c * coord_stride + i * vert_stride]
struct RcMesh {
  const float *x;
  long long env_stride;
  int coord_stride, vert_stride;
  const int *genv;   // source environment -> output environment (nullptr: first_env + l)
  int first_env;
  const int3 *tris;
  int T;
};
// obstacles of output environment e: k < K at [e * stride + k]
struct RcObs {
  const int *type;
  const float *dims, *pose;
  int K, stride;
};
// keys: per-pixel work buffer; tag: the frame's tag (kFirstTag down to 0,
// then rc_next_tag refills the buffer); triangles per mesh < kMaxRcTris
constexpr int kFirstTag = 254;
constexpr int kMaxRcTris = (1 << 25) - 1;
cudaError_t rc_next_tag(unsigned long long *keys, size_t n_keys, int *tag, cudaStream_t st);
cudaError_t rc_launch_tri(const RcMesh &M, int n_envs, const float *cam_poses, const RcCam &C,
                          unsigned long long *keys, unsigned tag, cudaStream_t st);
// prep: device workspace of rc_prep_bytes(n_envs) (per-environment view constants)
size_t rc_prep_bytes(int n_envs);
cudaError_t rc_launch_resolve(const RcObs &O, const float *cam_poses, const RcCam &C, int first_env, int n_envs,
                              const unsigned long long *keys, unsigned tag, void *prep, float *depth, uint8_t *seg,
                              float *pts, cudaStream_t st);
flash_status rc_check_camera(const flash_camera *cam, int64_t n_envs, RcCam *out);

// grasp requests s->greq[first_env, first_env + count) -> per-environment grasp state
cudaError_t launch_grasp_set(const flash_scene *s, int first_env, int count, int obstacle, float ax, float ay,
                             float az, float radius, cudaStream_t st);
cudaError_t launch_local_lane(const flash_scene *s, const Lane &L, const StepArgs &a, int k, int residual_only, int tc,
                              cudaStream_t st, int *launched);
cudaError_t launch_local_batch(const flash_scene *s, const Batch &b, int threads, const StepArgs &a, int k,
                               int residual_only, int tc, cudaStream_t st);
cudaError_t launch_ncp_lane(const flash_scene *s, const Lane &L, const StepArgs &a, int tc, cudaStream_t st,
                            int threads = 0);
cudaError_t launch_tol_next(cudaGraphConditionalHandle h, int *active, int *kit, unsigned long long *trips, int last,
                            int first, cudaStream_t st);
cudaError_t launch_end_lane(const flash_scene *s, const Lane &L, const StepArgs &a, cudaStream_t st);
// full contact metric: Newton step with preconditioned GMRES on Z = J A^-1 J^T + E
cudaError_t launch_fm_setup_lane(const flash_scene *s, const Lane &L, const StepArgs &a, cudaStream_t st);
cudaError_t launch_fm_scatter_lane(const flash_scene *s, const Lane &L, const StepArgs &a, int j, int tc,
                                   cudaStream_t st);
cudaError_t launch_fm_gather_lane(const flash_scene *s, const Lane &L, const StepArgs &a, int j, cudaStream_t st);
cudaError_t launch_fm_finish_lane(const flash_scene *s, const Lane &L, const StepArgs &a, int tc, cudaStream_t st);
// diag(A_e^-1) of every environment of an eigen-form group, and of a dense inverse
cudaError_t launch_fm_adiag(const Group &g, cudaStream_t st);

// global solve (gemm_simt.cu / gemm_tc.cu) -----------------------------------
// out = M * rhs over columns [c0, c1) of a group (c1 < 0: all), M = A^-1, V or V^T (the CUDA-core
// kernel computes M^T * rhs: callers pass the transposed matrix).  Epilogue
// mode 0: out = acc (tiles whose environments are all done are skipped)
// mode 1: q  = q + w + acc (skips environments whose done flag is set)
// mode 2: out = acc / (1 + kenv[env] * lam[row])  (eigen-coordinate scaling)
cudaError_t gemm_simt(const Group &g, const SolveMat &M, const float *rhs, float *out, const float *w,
                      const int *done, int mode, const float *lam, const float *kenv, cudaStream_t st, int c0 = 0,
                      int c1 = -1);
// bn: tile width (0: the group's autotuned width)
// bf: one bf16 product (matrix M.bf, right-hand sides bf16 in rh) instead of the f16 hi/lo split;
// epilogue mode 3: out += acc (a refinement step's correction)
cudaError_t gemm_tc(const Group &g, const SolveMat &M, float *out, const float *w, const int *done, int mode,
                    const float *lam, const float *kenv, cudaStream_t st, int c0 = 0, int c1 = -1, int bn = 0,
                    bool bf = false, const SplitK &sk = SplitK());
// one bounded mbarrier wait that nothing completes (limit in SM cycles, at
// most the solve's own limit): sets the status word's timeout bit
cudaError_t launch_wait_probe(int *status, long long limit, cudaStream_t st);
// scratch a split-K apply of columns [c0, c1) of g needs at any tile width
void splitk_need(const Group &g, int c0, int c1, size_t *tiles, size_t *part_floats);
bool tc_available();
// grouped apply (one launch over several groups' dense applies, tile width kGroupedBN)
constexpr int kGroupedBN = 64;
size_t gemm_problem_bytes();
int gemm_problem(void *dst, const Group &g, const SolveMat &M, int c0, int c1, int tile0);
cudaError_t gemm_tc_grouped(const void *probs, int nprob, int tiles, float *const *outs, const int *done, int *status,
                            cudaStream_t st);
// time the tile widths (and, given scratch, split-K) on columns [c0, c1) of
// the group; fastest in *bn and *split
cudaError_t tune_gemm_tc(const Group &g, const int *done, cudaStream_t st, int c0, int c1, int *bn, int *split,
                         const SplitK &sk = SplitK());
cudaError_t gemm_simt_raw(const float *Ainv, const float *rhs, float *out, int n_pad, int cols, cudaStream_t st);

// setup (setup_kernels.cu) ---------------------------------------------------
cudaError_t invert_spd_f64(double *A, int n, int n_pad, int batch, cudaStream_t st);
cudaError_t cast_inverse(const double *A64, int n_pad, float *A32, __half *hi, __half *lo, int a_exp,
                         cudaStream_t st, __nv_bfloat16 *bf = nullptr);
// symmetric eigen-decomposition by cyclic Jacobi rotations (host, FP64):
// B (n x n, destroyed) = W diag(lam) W^T, W row-major with eigenvectors as columns
void jacobi_eigen(int n, std::vector<double> &B, std::vector<double> &W, std::vector<double> &lam);

}  // namespace flash
