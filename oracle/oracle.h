/* FP64 CPU oracle for the batched FLASH time step (arxiv 2604.17513).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline arm may load this library.  It shares no code,
 * header, table or constant with the CUDA library; both sides read the same
 * seeded scene arrays and nothing else.
 *
 * What it computes, in the paper's order (Algorithm 1, "Multi-Env GPU-based
 * Pipeline"; Sec. III "Preliminary" and Sec. IV-B):
 *   setup   A = M + h^2 sum_i w_i G_i^T G_i  (Sec. III-B), dense Cholesky
 *   step    collision detection, q~ = q_t + h v_t + h^2 g, then k iterations of
 *             p_i = project(G_i q^{k-1})                      (Eq. internal)
 *             b = M q~ + h^2 sum w_i G_i^T p_i               (Sec. III-B)
 *             J, E, g = b + J^T gamma^{k-1}, h = -phi + J q^{k-1} (Sec. III-C)
 *             Z = J M^-1 J^T + E  (lite metric, Sec. IV-B.1) or J A^-1 J^T + E
 *             dgamma = Z^-1 (h - J A^-1 g)                    (Algorithm 1)
 *             q^k = A^-1 (b + J^T gamma^k)                    (Eq. correction)
 *           then v = (q - q_t)/h.
 * gamma = h^2 * lambda throughout (kg m); impulses are gamma/h.
 *
 * Readings of the paper where it is silent are listed in the design notes
 * and restated beside the code that takes them.
 */
#ifndef FLASH_ORACLE_H
#define FLASH_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct OrMesh OrMesh;

/* element types */
#define OR_TRI 0
#define OR_TET 1
/* obstacle types */
#define OR_PLANE 1
#define OR_SPHERE 2
#define OR_BOX 3

/* dp[] (double parameters) */
#define OR_DP_H 0
#define OR_DP_GX 1
#define OR_DP_GY 2
#define OR_DP_GZ 3
#define OR_DP_TOL 4
#define OR_DP_MAXFORCE 5
#define OR_DP_TAU 6
#define OR_DP_MARGIN 7
#define OR_DP_MU 8
#define OR_DP_GRASP_OBS 9 /* obstacle carrying the grasp anchor (as a double), -1: no grasp */
#define OR_DP_ANCHOR 10   /* 10..12: anchor point in that obstacle's frame */
#define OR_DP_SELF 13 /* nonzero: cloth self-collision (vertex against triangle) */
#define OR_DP_OFEAT 14 /* nonzero: box corners and edges against cloth triangles and edges */
#define OR_DP_SIZE 15

/* Bilateral grasp (appendix, Bilateral Constraint for Cloth Control): a
 * grasped vertex i carries the equality C = x_i - p_grip = 0 with p_grip the
 * anchor at the gripper's pose at t+h.  It sits in the contact list with the
 * obstacle slot OR_GRASP_SLOT (after every obstacle, so lists stay sorted). */
#define OR_GRASP_SLOT 8
/* Self contact of a cloth vertex with a triangle of the same cloth (contact
 * list slot OR_SELF_SLOT, triangle in ctri): at most OR_SELF_MAX per vertex,
 * projections inside the triangle up to OR_SELF_BARY (barycentric). */
#define OR_SELF_SLOT 9
#define OR_SELF_MAX 4
#define OR_SELF_BARY 0.1
/* Edge-edge self contact of an edge e1 = (i, b), b > i, with an edge e2 > e1
 * (slot OR_EE_SLOT, feature e1 * n_edges + e2 in ctri, edges (a < b)
 * sorted; each unordered pair once): at most OR_EE_MAX per vertex i. */
#define OR_EE_SLOT 10
#define OR_EE_MAX 4
/* Contacts of box obstacle features with a cloth (a reading: the paper
 * describes none; a vertex row cannot see a box corner or edge that passes
 * between the cloth's vertices).  Box corner k (0..7) of obstacle o against
 * triangle f: slot OR_OVT_SLOT, feature (f * OR_MAX_OBS + o) * 8 + k,
 * listed under f's first vertex.  Box edge j (0..11) of obstacle o against
 * the cloth edge e = (a, b): slot OR_OEE_SLOT, feature (e * OR_MAX_OBS + o)
 * * 12 + j, listed under a.  At most OR_OFEAT_MAX of each per vertex, in
 * feature order. */
#define OR_OVT_SLOT 11
#define OR_OEE_SLOT 12
#define OR_OFEAT_MAX 4
#define OR_MAX_OBS 8
#define OR_NDP 9
/* ip[] (integer parameters) */
#define OR_IP_KMAX 0
#define OR_IP_KMIN 1
#define OR_IP_KCAP 2
#define OR_IP_MODE 3   /* 0: exactly k_max iterations; 1: until r_ncp <= tol */
#define OR_IP_METRIC 4 /* 0: lite  J M^-1 J^T + E;  1: full  J A^-1 J^T + E (exact solve);
                          2: full, Z solved by OR_IP_LINIT steps of preconditioned GMRES */
#define OR_IP_LINIT 5  /* linear-solver iterations of metric 2 */
#define OR_NIP 5

OrMesh *or_mesh_new(int type, int n, const double *rest, int ne, const int *elems,
                    const double *mass, double w_stretch, double w_bend, double h);
void or_mesh_free(OrMesh *m);
int or_mesh_hinges(const OrMesh *m);
/* unique edges (a < b) of a triangle mesh in (a, b) order: count, and the
 * pairs into out [count][2] when out is not NULL */
int or_mesh_edges(const OrMesh *m, int *out);
void or_mesh_matrix(const OrMesh *m, double *A_out);             /* dense n x n */
void or_solve(const OrMesh *m, const double *rhs, double *out);  /* A^-1 rhs, [n][3] */
void or_project(const OrMesh *m, const double *q, double *p);    /* [ne][9] row-major 3x2|3x3 */
void or_assemble_b(const OrMesh *m, const double *qt, const double *p, double *b);
double or_pd_energy(const OrMesh *m, const double *q, const double *qt, const double *p);
void or_closest_rotation(int cols, const double *F, double *R); /* 3x2 or 3x3, row-major */

/* signed distance, unit normal and (optionally) obstacle point displacement
 * over the step for one point; pose = (p, qw, qx, qy, qz) */
double or_sdf(int type, const double *dims, const double *pose, const double *x, double *nrm);

/* attached: [n] grasp flags (or NULL); a flagged vertex gets an OR_GRASP_SLOT
 * entry after its obstacle contacts, then its self contacts (OR_SELF_SLOT,
 * triangle in ctri; OR_EE_SLOT, edge pair in ctri; -1 for the other rows;
 * ctri may be NULL) when dp[OR_DP_SELF] is set, then its box-feature rows
 * (OR_OVT_SLOT, OR_OEE_SLOT) when dp[OR_DP_OFEAT] is set */
int or_detect(const OrMesh *m, const double *dp, int K, const int *otype, const double *odims,
              const double *pose_th, const double *q, const double *v, const unsigned char *attached,
              int cap, int *cvert, int *cobs, int *ctri);

int or_solve_step(const OrMesh *m, const double *dp, const int *ip, int K, const int *otype,
                  const double *odims, const double *ocomp, const double *pose_t,
                  const double *pose_th, double *q, double *v, const double *q_init, int count,
                  const int *cvert, const int *cobs, const int *ctri, double *cgamma, int *iters,
                  double *rncp, double *trace);

/* NCP residual of (q, gamma) for a given contact list (max-norm, metres) */
double or_residual(const OrMesh *m, const double *dp, int K, const int *otype, const double *odims,
                   const double *ocomp, const double *pose_t, const double *pose_th,
                   const double *q_t, const double *q, int count, const int *cvert, const int *cobs,
                   const int *ctri, const double *cgamma);

/* fischer-burmeister value, exported for the closed-form pins */
double or_fb(double a, double b);

/* Depth ray casting of one environment (raycast.c; appendix, depth
 * rendering).  x [n][3] world vertex positions, tris [T][3] (instance 1);
 * obstacles k < K of type otype[k], dims odims[k][3], pose opose[k][7]
 * (instance 2 + k; type 0 invisible).  cam[7] camera-to-world pose; intr =
 * (fx, fy, cx, cy, z_near, z_far).  Pixel (u, v): ray through image point
 * (u + 1/2, v + 1/2), d_cam = ((u + 1/2 - cx)/fx, (v + 1/2 - cy)/fy, 1), so
 * t = depth.  Hit = smallest t in [z_near, z_far] (ties: smaller instance,
 * then smaller triangle index).  dil grows (> 0) or shrinks (< 0) every
 * primitive: triangles by |dil| in barycentric coordinates, spheres by
 * |dil| r, boxes by |dil| times the largest half extent; planes unchanged.
 * Outputs depth [H][W] (0: no hit), seg [H][W] (0: no hit), pts [H][W][3]
 * world hit points (NaN: no hit). */
void or_raycast(int n, const double *x, int T, const int *tris, int K, const int *otype, const double *odims,
                const double *opose, const double *cam, const double *intr, int W, int H, double dil,
                double *depth, int *seg, double *pts);
/* the same for a list of pixels uv [npix][2] = (u, v); outputs [npix] */
void or_raycast_pixels(int n, const double *x, int T, const int *tris, int K, const int *otype,
                       const double *odims, const double *opose, const double *cam, const double *intr, int npix,
                       const int *uv, double dil, double *depth, int *seg, double *pts);

#ifdef __cplusplus
}
#endif
#endif
