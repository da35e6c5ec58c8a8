/* flash.h — C ABI of the GB300-native batched deformable + frictional-contact
 * time step (FLASH, arxiv 2604.17513, Sec. III "Preliminary" and Sec. IV-B
 * "Simulation Core", Algorithm 1 "Multi-Env GPU-based Pipeline").
 *
 * One process, one GPU.  All environments that share a mesh (and a stiffness
 * scale) share one constant system matrix A = M + h^2 sum_i w_i G_i^T G_i
 * (Sec. III-B); every step of every environment runs in this library's CUDA
 * kernels.  Calls are stream-ordered: nothing synchronises the host except
 * flash_scene_finalize, the *_host getters, flash_launch_count and the
 * eager tolerance mode of flash_step, which reads a device count every few
 * iterations (the graphed tolerance mode decides on the device).
 *
 * Conventions
 *   - z is up; positions in metres; obstacle pose = (px,py,pz, qw,qx,qy,qz).
 *   - State layout seen by callers: float32 [sum_e n_e][3], environments in
 *     the order they were added, vertices in mesh order (xyz interleaved).
 *   - Contact multipliers gamma = h^2 * lambda (kg m), stored per contact as
 *     (gamma_n, gamma_t world x, y, z); the contact impulse is gamma / h.
 *   - Pointers marked "device" must be device memory of the current CUDA
 *     device; "host" pointers are read during the call only.  The library
 *     owns every allocation it makes and frees it in flash_scene_destroy.
 *   - Every call returns a flash_status; on error a thread-local message is
 *     available from flash_last_error().  Kernels never trap: device-side
 *     problems (non-finite state, contact overflow) set a per-scene status
 *     word that the next call reports.
 */
#ifndef FLASH_H
#define FLASH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t flash_status;
#define FLASH_OK 0
#define FLASH_EINVAL (-1)   /* bad argument or descriptor */
#define FLASH_ENOMEM (-2)   /* device or host allocation failed */
#define FLASH_ECUDA (-3)    /* a CUDA runtime call failed */
#define FLASH_ETIMEOUT (-4) /* a bounded device wait ran out */
#define FLASH_ENOTIMPL (-5) /* feature not available in this build */
#define FLASH_ESTATE (-6)   /* call out of order (e.g. step before finalize) */
#define FLASH_ENUMERIC (-7) /* setup matrix not positive definite, NaN state */
#define FLASH_EINDEX (-8)   /* checked build: a kernel read an index out of its range */
#define FLASH_WOVERFLOW 1   /* warning: contacts beyond capacity were dropped */

#define FLASH_TRI 0
#define FLASH_TET 1

#define FLASH_OBS_NONE 0
#define FLASH_OBS_PLANE 1  /* plane through the pose origin, normal = body +z */
#define FLASH_OBS_SPHERE 2 /* dims[0] = radius */
#define FLASH_OBS_BOX 3    /* dims = half extents */
#define FLASH_MAX_OBS 8
#define FLASH_GRASP_SLOT FLASH_MAX_OBS /* contact-list obstacle slot of grasp rows */
#define FLASH_SELF_SLOT (FLASH_MAX_OBS + 1) /* contact-list slot of cloth self contacts */
#define FLASH_SELF_MAX 4 /* vertex-triangle self contacts per vertex at most */
#define FLASH_EE_SLOT (FLASH_MAX_OBS + 2) /* contact-list slot of cloth edge-edge contacts */
#define FLASH_EE_MAX 4 /* edge-edge contacts per vertex at most */
#define FLASH_OVT_SLOT (FLASH_MAX_OBS + 3) /* contact-list slot of box corners against cloth triangles */
#define FLASH_OEE_SLOT (FLASH_MAX_OBS + 4) /* contact-list slot of box edges against cloth edges */
#define FLASH_OFEAT_MAX 4 /* rows of each box-feature kind per vertex at most */

#define FLASH_MODE_FIXED 0 /* exactly k_max local-global iterations per step */
#define FLASH_MODE_TOL 1   /* iterate until r_ncp <= tol_ncp (k >= k_min) or k_cap */

#define FLASH_SOLVE_F32 0    /* global solve: FP32 dense apply on the CUDA cores */
#define FLASH_SOLVE_F16X3 1  /* global solve: tcgen05 f16 hi/lo split, FP32 accumulate */
#define FLASH_SOLVE_BF16R 2  /* global solve: tcgen05 bf16, FP32 accumulate, refine_steps steps of
                                iterative refinement with the residual rhs - A w in FP32 (tet meshes) */

#define FLASH_METRIC_LITE 0  /* contact metric Z = J M^-1 J^T + E (Sec. IV-B.1), per-vertex blocks */
#define FLASH_METRIC_FULL 1  /* Z = J A^-1 J^T + E (Sec. III-C), lin_iters steps of GMRES per Newton step */

#define FLASH_WARM_COLD 0    /* gamma^0 = 0, q^0 = q~ (the paper's start) */
#define FLASH_WARM_PREV 1    /* gamma^0 = previous step's gamma of the same contact */
#define FLASH_WARM_LEARNED 2 /* gamma^0, q^0 from the warm-start network */

/* Scene-wide solver settings (Sec. III; Algorithm 1; appendix scene config).
 * h: timestep (s).  gravity: m/s^2.  tol_ncp: NCP residual tolerance (m) of
 * FLASH_MODE_TOL.  maxforce: clamp on the normal force (N).  thickness: the
 * default contact thickness tau (m) of meshes that give none.  margin:
 * detection margin delta (m).  k_max: iterations of FLASH_MODE_FIXED.
 * k_min/k_cap: bounds of FLASH_MODE_TOL.  contact_cap: contacts per
 * environment.  solve: FLASH_SOLVE_*.  warm: FLASH_WARM_*.  lanes: number of
 * independent environment partitions stepped concurrently on their own
 * streams (0 = chosen from the batch size; results do not depend on it).
 * eager: 0 = a step is captured once in a CUDA graph and replayed (not
 * while profiling; the learned warm start and contact recording are part
 * of the graph);
 * in FLASH_MODE_TOL the graph holds the iteration loop as a while-node that
 * the device keeps running while an environment is still iterating (at
 * most k_cap runs), so a step needs no host round trip; 1 = every step
 * launches its kernels one by one and the host stops the tolerance loop.
 * Both give the same results.
 * metric: FLASH_METRIC_*.  lin_iters: linear-solver iterations of the full
 * metric, 1..32 (0 = 10, the paper's parameter table): each Newton step runs
 * that many GMRES steps on Z dy = rhs over all contacts of an environment,
 * preconditioned by Z's 3x3 diagonal blocks; every GMRES step costs one
 * application of A^-1 to all environments.
 * self_collide: 1 turns on cloth self-collision for triangle meshes (needs
 * FLASH_METRIC_FULL): a vertex p and a triangle f of the same mesh that
 * touches none of p's own triangles are in contact when p lies within
 * thickness + margin of f's plane with its projection inside f up to 0.1 in
 * barycentric terms (at q_t or q~); the first FLASH_SELF_MAX such triangles
 * (in index order) per vertex get a row (slot FLASH_SELF_SLOT) whose normal
 * is f's, oriented towards the side p was on at the step start, gap =
 * distance to the plane - thickness, the contact point moving as p minus
 * the barycentric combination of f's corners.  Edge-edge contacts: the
 * mesh's unique edges (a, b), a < b, numbered in (a, b) order; edges e1 =
 * (a, b) and e2 = (c, d), e1 < e2 (each pair once), with no common vertex
 * and no triangle holding a or b together with c or d are in contact when the closest points of their
 * lines lie inside both edges, nearer than thickness + margin (at q_t or
 * q~); vertex a gets a row (slot FLASH_EE_SLOT, feature e1 * n_edges + e2)
 * for each of the first FLASH_EE_MAX such pairs of its edges (e1, then e2
 * ascending).  Its normal is that of both edges, oriented by the side
 * (a, b) was on at the step start, gap = distance between the lines -
 * thickness, the contact point moving as (1 - s) x_a + s x_b - (1 - t) x_c
 * - t x_d.  Rows of a vertex: obstacles, grasp, vertex-triangle, edge-edge,
 * then the box-feature rows below.
 * The paper disables self-collision and describes no method; this is the
 * library's reading.
 * obstacle_features: 1 adds contact rows between the corners and edges of
 * box obstacles and a cloth (triangle meshes; needs FLASH_METRIC_FULL), so
 * that a box narrower than the cloth's cells cannot pass between its
 * vertices.  Box corner k (0..7; bit i of k set: +half extent on axis i,
 * clear: -) of obstacle o against triangle f: a row of f's first vertex
 * (slot FLASH_OVT_SLOT, feature (f * FLASH_MAX_OBS + o) * 8 + k) when the
 * corner, at the obstacle's pose at t+h, lies within thickness + margin of
 * f's plane with its projection inside f up to 0.1 in barycentric terms,
 * at q_t or q~.  The contact point moves as the barycentric combination of
 * f's corners; normal = f's, oriented towards the side the cloth was on,
 * seen from the box corner, at the step start; gap = distance from the box
 * corner to the plane - thickness.  Box edge j (0..11: along axis j / 4,
 * on the + side of the other two axes, in increasing order, where bits 0
 * and 1 of j % 4 are set) of obstacle o against the cloth edge e = (a, b):
 * a row of a (slot FLASH_OEE_SLOT, feature (e * FLASH_MAX_OBS + o) * 12 +
 * j) when the closest points of the two lines lie inside both and nearer
 * than thickness + margin, at q_t or q~; the contact point moves as
 * (1 - s) x_a + s x_b; normal = that of both lines, oriented by the side the
 * cloth edge was on at the step start; gap = distance between the lines -
 * thickness.  The first FLASH_OFEAT_MAX rows of each kind per vertex are
 * kept, in feature order.  The paper describes none; this is the library's
 * reading.
 * grouped_solve (tensor-core solve, scenes of several mesh templates and
 * lanes): a lane applies the dense inverses of all its templates in one
 * launch (FLASH_GROUPED_ON), one launch per template (FLASH_GROUPED_OFF), or
 * whichever of the two is faster when the scene is finalised
 * (FLASH_GROUPED_AUTO, 0).  Results do not depend on it.
 * refine_steps (FLASH_SOLVE_BF16R): steps of iterative refinement after the
 * bf16 apply, 0..4: each computes rhs - A w in FP32 from the element
 * operators and adds the bf16 apply of it.  BF16R needs a well-conditioned
 * A: it is refused (FLASH_ENOTIMPL) for triangle meshes, whose systems (cond
 * ~1e7 for the 32x32 cloth) make each step grow the error.
 * local_threads, ncp_threads: threads per environment (one CTA each) of the
 * local pass (0, 256, 512 or 1024) and of the lite NCP pass (0, 128, 256 or
 * 512).  0 takes the library's choice (local: 1024 for meshes above 2048
 * vertices, else 512; NCP: 256); FLASH_THREADS_TUNE (-1) times the
 * candidates on the scene's first step and keeps the fastest (see
 * flash_scene_threads).  Fewer threads per environment put more
 * environments on each SM; more shorten each environment's dependent chain.
 * Results do not depend on either (each vertex and contact row is handled
 * by one thread in a fixed order; the block reductions are maxima), except
 * with self or box-feature rows, whose forces are summed with atomics.
 * split_k (tensor-core solve): each output tile of a lane's apply sums its
 * two K halves on one CTA (FLASH_SPLITK_OFF) or on two CTAs that meet
 * through a scratch tile (FLASH_SPLITK_ON), or whichever the autotuner
 * times faster for each column range (FLASH_SPLITK_AUTO, 0); results do not
 * depend on it (see flash_tile_splits). */
#define FLASH_SPLITK_AUTO 0
#define FLASH_SPLITK_OFF 1
#define FLASH_SPLITK_ON 2
#define FLASH_THREADS_TUNE (-1)
#define FLASH_GROUPED_AUTO 0
#define FLASH_GROUPED_OFF 1
#define FLASH_GROUPED_ON 2
typedef struct {
  double h;
  double gravity[3];
  double tol_ncp;
  double maxforce;
  double thickness;
  double margin;
  int32_t k_max, k_min, k_cap, mode;
  int32_t contact_cap;
  int32_t solve;
  int32_t warm;
  int32_t lanes;
  int32_t eager;
  int32_t metric;
  int32_t lin_iters;
  int32_t self_collide;
  int32_t obstacle_features;
  int32_t grouped_solve;
  int32_t refine_steps;
  int32_t local_threads;
  int32_t ncp_threads;
  int32_t split_k;
} flash_scene_desc;

/* A mesh template (asset).  type: FLASH_TRI (TRI_ARAP stretch + flat-rest
 * bending on interior edges) or FLASH_TET (corotational strain).  rest: host
 * float64 [n][3]; elems: host int32 [E][3|4]; mass: host float64 [n] (kg).
 * w_stretch: weight per unit rest area (TRI) or volume (TET); w_bend: bending
 * weight (TRI only); thickness: contact thickness tau (m) subtracted from the
 * signed distances of this mesh's vertices (a negative value takes the
 * scene's default). */
typedef struct {
  int32_t type;
  int32_t n_verts, n_elems;
  const double *rest;
  const int32_t *elems;
  const double *mass;
  double w_stretch, w_bend;
  double thickness;
} flash_mesh_desc;

/* Per-environment parameters.  mu: Coulomb coefficient.  stiffness: scale on
 * the mesh's w_stretch (environments with equal scale share A).  Obstacles:
 * kinematic planes, spheres and boxes (ground, fingers, props); compliance is
 * the normal compliance in m/N (0 = rigid). */
typedef struct {
  float mu;
  float stiffness;
  int32_t n_obs;
  int32_t obs_type[FLASH_MAX_OBS];
  float obs_dims[FLASH_MAX_OBS][3];
  float obs_compliance[FLASH_MAX_OBS];
} flash_env_desc;

typedef struct flash_scene flash_scene;

/* Creation / setup (the paper's load_config / set_envs / initialize). */
flash_status flash_scene_create(const flash_scene_desc *desc, flash_scene **out);
flash_status flash_mesh_add(flash_scene *s, const flash_mesh_desc *mesh, int32_t *mesh_id);
flash_status flash_envs_add(flash_scene *s, int32_t mesh_id, int32_t n, const flash_env_desc *envs,
                            int32_t *first_env);
/* Builds A per (mesh, stiffness), inverts it once in FP64 on the device
 * (Algorithm 1 setup: Cholesky / explicit inverse), allocates all state.
 * Synchronises the stream. */
flash_status flash_scene_finalize(flash_scene *s, void *stream);
void flash_scene_destroy(flash_scene *s);

int32_t flash_num_envs(const flash_scene *s);
int64_t flash_num_verts(const flash_scene *s);                       /* sum_e n_e */
flash_status flash_env_offsets(const flash_scene *s, int64_t *off); /* host [N+1] */

/* State I/O: q, v device float32 [sum n_e][3] (either may be NULL). */
flash_status flash_set_state(flash_scene *s, const float *q, const float *v, void *stream);
flash_status flash_get_state(const flash_scene *s, float *q, float *v, void *stream);

/* Kinematic obstacle targets (the paper's move_ee): device float32
 * [N][FLASH_MAX_OBS][7].  which = 0 sets the current and next pose (reset),
 * which = 1 sets the pose the next step moves to.  After a step the next
 * pose becomes the current one. */
flash_status flash_set_obstacle_poses(flash_scene *s, const float *poses, int32_t which, void *stream);

/* Bilateral grasp (the paper's grasp_ee; appendix "Bilateral Constraint for
 * Cloth Control"): every vertex i of the grasped set S_grip of an environment
 * carries the equality constraint C = x_i - p_grip(t+h) = 0, with p_grip the
 * point `anchor` (body frame of obstacle `obstacle`) at that obstacle's pose
 * at the end of the step.  The constraint is one more row of the
 * environment's contact list (obstacle slot FLASH_GRASP_SLOT, after the
 * vertex's obstacle rows; frame = world axes, gamma = its multiplier) solved
 * by the same Newton/NCP iterations; use the full metric to hold it tightly.
 *
 * For environments [first_env, first_env + count): request host int32
 * [count], per environment
 *    1  activate: at the start of the next step, S_grip becomes the vertices
 *       whose position lies within `radius` (metres, Euclidean, FP32) of the
 *       anchor at the obstacle's current pose;
 *    0  release: S_grip becomes empty at the start of the next step;
 *   -1  leave the environment's grasp unchanged.
 * obstacle in [0, FLASH_MAX_OBS) (typically a FLASH_OBS_NONE pose carrier,
 * moved by flash_set_obstacle_poses like any obstacle); anchor host float [3]
 * (NULL: the obstacle's origin); radius >= 0.  One gripper per environment:
 * a new activation replaces S_grip.  Stream-ordered with flash_step; the
 * grasp set is kept across steps and is not changed by flash_set_state.
 * FLASH_EINVAL for a bad range, obstacle, radius or request value. */
flash_status flash_grasp(flash_scene *s, int32_t first_env, int32_t count, const int32_t *request,
                         int32_t obstacle, const float *anchor, float radius, void *stream);

/* ---------------------------------------------------------------------------
 * Depth ray casting (appendix, depth rendering: depth maps, instance
 * segmentation masks and point clouds cast directly from the simulation
 * state).
 *
 * Camera model: pinhole with the intrinsics below and a pose per
 * environment, camera-to-world (px,py,pz, qw,qx,qy,qz); camera axes x right,
 * y down, z along the view.  Pixel (u, v) (u the column; images row-major
 * [H][W]) casts the ray from the camera centre through image point
 * (u + 1/2, v + 1/2), direction d = ((u + 1/2 - cx)/fx, (v + 1/2 - cy)/fy, 1)
 * in camera axes, so a hit's ray parameter is its depth.  A pixel sees the
 * nearest hit with depth in [z_near, z_far] over the environment's surface
 * triangles (instance 1; tetrahedral meshes show their boundary faces) and
 * its obstacles (instance 2 + k for obstacle k; FLASH_OBS_NONE is
 * invisible); every surface is two-sided; equal depths go to the smaller
 * instance.  Mesh edge tests are watertight: a ray never passes between two
 * triangles that share an edge.
 *
 * Outputs (device; seg and points may be NULL): depth float32 [N][H][W]
 * (0: no hit), seg uint8 [N][H][W] (0: no hit), points float32
 * [N][H][W][3] world hit points (NaN: no hit).  Two kernel launches per
 * call, stream-ordered; the caller keeps the output buffers.
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t width, height; /* pixels; 1 <= width*height <= 2^26, height <= 524280 */
  float fx, fy, cx, cy;  /* intrinsics in pixels; fx, fy > 0 */
  float z_near, z_far;   /* depth range (m); 0 < z_near < z_far */
} flash_camera;

/* Renders every environment of a finalized scene from its current state:
 * positions as left by the last step or flash_set_state, obstacle poses of
 * the current time (after a step: the pose it moved to).  cam_poses: device
 * float32 [N][7].  The scene keeps a per-pixel work buffer of N*W*H*8 bytes,
 * allocated on the first call (and again when the image grows). */
flash_status flash_render(flash_scene *s, const flash_camera *cam, const float *cam_poses, float *depth,
                          uint8_t *seg, float *points, void *stream);

/* Standalone batched ray caster for N environments that share one triangle
 * mesh (n_verts vertices, tris host int32 [n_tris][3], indices checked),
 * independent of a scene.  Owns the triangle list and the N*W*H*8-byte work
 * buffer; synchronous allocation in create. */
typedef struct flash_raycaster flash_raycaster;
flash_status flash_raycaster_create(const flash_camera *cam, int32_t n_envs, int32_t n_verts, int32_t n_tris,
                                    const int32_t *tris, flash_raycaster **out);
/* verts device float32 [N][n_verts][3]; obstacles per environment: n_obs
 * (0..FLASH_MAX_OBS), obs_type device int32 [N][n_obs], obs_dims device
 * float32 [N][n_obs][3], obs_poses device float32 [N][n_obs][7] (pose as
 * in flash_set_obstacle_poses); cam_poses device float32 [N][7]. */
flash_status flash_raycast(flash_raycaster *rc, const float *verts, int32_t n_obs, const int32_t *obs_type,
                           const float *obs_dims, const float *obs_poses, const float *cam_poses, float *depth,
                           uint8_t *seg, float *points, void *stream);
void flash_raycaster_destroy(flash_raycaster *rc);
/* Per-kernel device time of later flash_raycast calls: enable != 0 brackets
 * the two launches with CUDA events on the call's stream and waits for them
 * at the end of each call (for measurement only); the totals restart at
 * every flash_raycaster_profile call.  profile_read: ms host double [2] and
 * launches host int64 [2], index 0 the triangle pass, 1 the per-pixel
 * resolve. */
flash_status flash_raycaster_profile(flash_raycaster *rc, int32_t enable);
flash_status flash_raycaster_profile_read(const flash_raycaster *rc, double *ms, int64_t *launches);

/* Advance every environment by n_steps (Algorithm 1 body). */
flash_status flash_step(flash_scene *s, int32_t n_steps, void *stream);

/* Contacts of the last step: count device int32 [N]; vert, obs device int32
 * [N][cap] (obs = FLASH_GRASP_SLOT for a grasp row); gamma device float32
 * [N][cap][4] (any may be NULL).  A vertex holds at most one row per
 * obstacle plus one grasp row, FLASH_SELF_MAX vertex-triangle,
 * FLASH_EE_MAX edge-edge and 2 FLASH_OFEAT_MAX box-feature rows, so cap =
 * n_verts * (n_obs + 1 + FLASH_SELF_MAX + FLASH_EE_MAX + 2 FLASH_OFEAT_MAX)
 * never overflows. */
flash_status flash_get_contacts(const flash_scene *s, int32_t *count, int32_t *vert, int32_t *obs,
                                float *gamma, void *stream);
int32_t flash_contact_cap(const flash_scene *s);
/* Feature of each row of the last step's contact lists: device int32
 * [N][cap]; the triangle of a vertex-triangle self contact, e1 * n_edges +
 * e2 for an edge-edge contact, the box-feature index of a FLASH_OVT_SLOT or
 * FLASH_OEE_SLOT row, -1 for the other rows. */
flash_status flash_get_contact_tris(const flash_scene *s, int32_t *tri, void *stream);

/* Per-environment statistics of the last step: iterations used and the NCP
 * residual max_j |phi_j| (m) of the final iterate; device int32/float32 [N]. */
flash_status flash_get_stats(const flash_scene *s, int32_t *iters, float *rncp, void *stream);
/* Device status word of the steps since the last flash_set_state (which
 * clears it), as a flash_status; synchronises the stream.  The kernels set
 * bits and never trap; this call turns them into, by priority:
 *   FLASH_ETIMEOUT  a bounded mbarrier wait of the tensor-core solve ran out
 *                   (its results are not valid);
 *   FLASH_EINDEX    (checked build only, see flash_checked_build) a step
 *                   kernel read a vertex, element-slot or contact index
 *                   outside its range; it used index 0 instead, so the
 *                   step's results are not valid;
 *   FLASH_ENUMERIC  a non-finite position or NCP residual (the environment
 *                   holding it stops iterating; other environments are not
 *                   affected, they share no data);
 *   FLASH_WOVERFLOW a contact list exceeded the scene's contact_cap (the
 *                   rows past it were dropped), or a vertex held more rows
 *                   than the lite metric's per-vertex block (4; the extra
 *                   rows were left unsolved).
 * flash_last_error() names the cause. */
flash_status flash_status_word(flash_scene *s, void *stream);

/* The global solve alone (Eq. correction's A^-1 apply) on the environments of
 * one group [first_env, first_env + n): rhs, out device float32 [n][n_v][3].
 * For parity tests of the dense contraction. */
flash_status flash_global_apply(flash_scene *s, int32_t first_env, int32_t n, const float *rhs,
                                float *out, void *stream);

/* Kernel accounting for measurement.  Kinds: 0 begin-of-step (detection,
 * prediction), 1 local step + residual, 2 global solve (dense apply), 3 NCP
 * blocks, 4 end-of-step.  flash_profile_enable(s, 1) brackets every launch
 * with CUDA events on the launching stream, 5 the learned warm start;
 * flash_profile_read synchronises
 * and returns the summed device time (ms) and launch count of one kind since
 * the last enable.  flash_launch_count returns the number of kernels this
 * scene has launched since creation; the iterations of a graphed tolerance
 * loop are counted on the device, so it synchronises the device. */
#define FLASH_KIND_BEGIN 0
#define FLASH_KIND_LOCAL 1
#define FLASH_KIND_SOLVE 2
#define FLASH_KIND_NCP 3
#define FLASH_KIND_END 4
#define FLASH_KIND_WARM 5 /* learned warm start: features, network, apply */
#define FLASH_NUM_KINDS 6
flash_status flash_profile_enable(flash_scene *s, int32_t enable);
flash_status flash_profile_read(flash_scene *s, int32_t kind, double *total_ms, int64_t *launches);
int64_t flash_launch_count(const flash_scene *s);
/* Number of lanes the scene steps concurrently (flash_scene_desc.lanes, or
 * the count chosen from the batch size); 0 before finalize. */
int32_t flash_lane_count(const flash_scene *s);
/* Tensor-core tile width (output columns per CTA) the autotuner chose for
 * each lane's column range of each group, lane by lane: up to max_out values
 * into the host array out; returns how many ranges there are (0 on the
 * CUDA-core path or before finalize). */
int32_t flash_tile_widths(const flash_scene *s, int32_t *out, int32_t max_out);
/* For the same ranges, in the same order: 2 where the autotuner runs each
 * output tile's two K halves on two CTAs (split-K), else 1.  Every apply
 * sums the two K halves separately and adds them last, so results do not
 * depend on this choice. */
int32_t flash_tile_splits(const flash_scene *s, int32_t *out, int32_t max_out);
/* 1 if the scene's lanes apply their dense inverses in one grouped launch
 * (flash_scene_desc.grouped_solve), else 0; 0 before finalize. */
int32_t flash_grouped_solve(const flash_scene *s);
/* Threads per environment in use: kind 0, the local pass's launches (one
 * per batch of environments with the same element type and shared-memory
 * need, lane by lane); kind 1, the lite NCP pass's (one per lane).  Writes
 * up to max_out values into the host array out and returns how many there
 * are (0 before finalize or for another kind).  With FLASH_THREADS_TUNE the
 * values are the library's choice until the first step has timed the
 * candidates, and the timed choice after it. */
int32_t flash_scene_threads(const flash_scene *s, int32_t kind, int32_t *out, int32_t max_out);

/* The bounded-wait failure path, run on purpose (a test hook, both builds):
 * one GPU thread waits, with the tensor-core solve's wait routine and a
 * limit of limit_cycles SM cycles (1..4e9; the solve itself uses 4e9,
 * about 2 s), on an mbarrier that nothing arrives at.  The wait runs out,
 * the status word's timeout bit is set and the thread returns, so the next
 * flash_status_word reports FLASH_ETIMEOUT and flash_set_state clears it;
 * the context stays usable.  Asynchronous on stream. */
flash_status flash_test_bounded_wait(flash_scene *s, int64_t limit_cycles, void *stream);
/* 1 in the checked build (libflash_check.so, compiled with FLASH_CHECK):
 * the step kernels range-check every vertex, element-slot and contact index
 * they read, replace an index out of range by 0 and report FLASH_EINDEX
 * through flash_status_word, instead of reading or writing out of bounds.
 * 0 in the regular build. */
int32_t flash_checked_build(void);
/* Fault injection for the checked build (the paper describes no failure
 * handling; this is the library's own test hook): sets corner `corner` of
 * element `element` of the mesh that environment `env` uses to vertex index
 * `value` in the device element table the step kernels read (shared by the
 * environments of that mesh group), and returns the previous index in *old.
 * Returns FLASH_ENOTIMPL in the regular build, FLASH_EINVAL for an env,
 * element or corner out of range; `value` itself is not checked (that is
 * its purpose).  Synchronous. */
flash_status flash_check_poke_element(flash_scene *s, int32_t env, int32_t element, int32_t corner, int32_t value,
                                      int32_t *old);

/* Learned warm start (the paper has no learned component; the network
 * predicts the initial multipliers gamma^0 and the first iterate at each
 * contact vertex from per-contact features).  Network: 10 -> 128 -> 128 -> 6
 * perceptron with ReLU, flat float32 parameters W1[128][10] b1[128]
 * W2[128][128] b2[128] W3[6][128] b3[6]; weights are rounded to bf16 when
 * used, products accumulate in FP32.  Features per contact (frame n, t1, t2
 * and gap at the predicted position q~): gap [mm], relative velocity in the
 * frame [0.1 m/s], n, previous step's multipliers y = gamma/m_v in the frame
 * [mm].  Outputs: y^0 in the frame [mm] (normal part clamped at 0) and
 * q^0 - q~ at the vertex [mm].
 *
 * flash_warmstart_set: mode = FLASH_WARM_*; params (device, copied) are
 * required for FLASH_WARM_LEARNED; flags (use_dq): bit 0 also moves contact
 * vertices to the predicted first iterate, bit 1 keeps only the normal
 * multiplier.  A contact whose features leave the trained input range
 * starts cold: flash_warmstart_bounds sets that range per feature (host
 * arrays lo[10], hi[10], lo <= hi, copied; default -100..100).
 * flash_record_contacts: while enabled every step stores features (at the
 * start) and targets (converged multipliers and q - q~, same units) of all
 * contacts; flash_get_recorded copies the last step's rows (environments in
 * group order) into device X [rows][10] and T [rows][6], synchronising.
 * Targets of environments whose final residual exceeds tol_ncp are NaN. */
flash_status flash_warmstart_set(flash_scene *s, const float *params, int32_t mode, int32_t use_dq);
flash_status flash_warmstart_bounds(flash_scene *s, const float *lo, const float *hi);
flash_status flash_record_contacts(flash_scene *s, int32_t enable);
flash_status flash_get_recorded(flash_scene *s, float *X, float *T, int64_t max_rows, int64_t *rows, void *stream);

/* Network kernels used for inference and training (device pointers).
 * flash_mlp_loss_grad: grad = d/dparams of (1/rows) sum_b 0.5 |f(x_b) - t_b|^2,
 * loss = sum_b |f(x_b) - t_b|^2 (device scalar); work needs
 * flash_mlp_work_floats(rows) floats.  flash_mlp_adam: one Adam step
 * (beta 0.9, 0.999, eps 1e-8) of the master weights, step counted from 1. */
int32_t flash_mlp_num_params(void);
flash_status flash_mlp_forward(const float *params, const float *x, float *y, int64_t rows, void *stream);
flash_status flash_mlp_loss_grad(const float *params, const float *x, const float *t, int32_t rows, float *grad,
                                 float *loss, float *work, void *stream);
int64_t flash_mlp_work_floats(int32_t rows);
flash_status flash_mlp_adam(float *params, const float *grad, float *m, float *v, int32_t step, float lr,
                            void *stream);

/* Allocation-free dense apply out = Ainv * rhs, for callers that must not
 * call cudaMalloc: real-time control loops and plugin hosts that reserve all
 * device memory up front, where an allocation can implicitly synchronise the
 * device and stall the loop or exceed the host's memory budget.  The paper
 * has no counterpart; it is the global solve's FP32 apply as a standalone
 * call.  Ainv: device float32 [n][n], row-major, any square matrix (e.g. the
 * explicit inverse of a mesh's system matrix; it need not be symmetric):
 * out[e][i][c] = sum_j Ainv[i][j] rhs[e][j][c].  rhs, out: device float32
 * [m][n][3], caller-owned.  Limits: n <= 512 vertices and m <= 256
 * environments per call; larger sizes return FLASH_EINVAL.  Scratch is a
 * fixed 4 MiB __device__ array that every GPU loading the library holds
 * until exit; a device's first call looks up its address (make that first
 * call before any stream capture), and a call looks it up again when the
 * device's context has changed since (after cudaDeviceReset).  Calls share
 * the array: calls that overlap on the GPU race. */
flash_status flash_dense_apply_noalloc(const float *Ainv, int32_t n, int32_t m, const float *rhs, float *out,
                                       void *stream);

const char *flash_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FLASH_H */
