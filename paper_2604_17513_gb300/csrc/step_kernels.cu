// Per-step kernels of the batched FLASH time step (Algorithm 1 body):
//   k_begin  collision detection + predicted state q~ (Algorithm 1 lines
//            "Collision detection", "q~ = q_t + h v_t + h^2 M^-1 f_ext")
//   k_local  contact linearisation at q^{k-1} and NCP residual, local
//            projection p_i = project(G_i q^{k-1}) (Eq. internal), and the
//            residual r = g - A q^{k-1} (Sec. III-B, III-C) in correction form
//   k_ncp    lite Schur blocks Z = J M^-1 J^T + E per vertex (Sec. IV-B.1)
//            and dgamma = Z^-1 (h - J A^-1 g); writes J^T dgamma
//   k_end    v = (q - q_t)/h, contact list kept for warm starts
// One CTA per environment; the whole environment state stays in shared
// memory inside a kernel, so element projections never reach HBM unless
// the mesh is too large for shared memory.
#include "device_math.cuh"
#include "flash_internal.cuh"

#include <algorithm>

namespace flash {

namespace {

struct GroupView {
  int n, n_pad, E, H, vpe, nc, type, cap;
  const int *genv, *elems;
  const float *D, *wt, *mass;
  const float4 *erec;            // triangle meshes: packed element records [E][2]
  float *q, *v, *qt, *qp, *r, *f, *w, *dq;
  __half *rh, *rl;
  float *rscale;
  int *ccount, *cvert, *cobs, *pcount, *pvert, *pobs;
  uint8_t *gflag;                // [N][n_pad] grasped vertices
  int self;                      // multi-vertex rows possible (self contacts or box features)
  int selfc, ofeat;              // detection of cloth self contacts / of box-feature rows
  int *ctri, *pctri;             // [N][cap] feature of self-contact rows (triangle, or e1 * ned + e2)
  float *fm_w;                   // [N][cap][kFmW] full metric: weights, effective mass, vertices 1..3
  int ned;                       // unique edges (a < b), (a, b) order
  const int2 *edges;             // [ned]
  const int *eoff;               // [n + 1] edges owned by vertex a
  const uint16_t *coff, *cidx;   // CSR vertex -> element slots e * vpe + a
  const int4 *kb;                // bending operator, off-diagonal entries in pairs, pair-major
  int ev, deg_b;
  const float *kenv;   // per-environment stiffness scale (eigen-form groups), else null
  int bf16;            // right-hand sides as bf16 + an FP32 copy (FLASH_SOLVE_BF16R)
  float *cgam, *pgam, *cscratch;
  int c_in_smem;
  float tau;           // contact thickness of the group's mesh
  // full contact metric (iterative Z solve); null unless the scene uses it
  float *fm_lin;       // [N][cap][kFmLin] per contact: R, cn, Ct, dn, dtn, Dtt, preconditioner scale s
  float *fm_V;         // [N][m + 1][3 cap] Krylov basis
  float *fm_H;         // [N][(m + 1) m] Hessenberg matrix after the rotations, H[i][j] at i m + j
  float *fm_cs, *fm_sn, *fm_g;   // [N][m], [N][m], [N][m + 1] Givens rotations and rotated right side
  float *fm_beta;      // [N] norm of the right side
  int *fm_jm;          // [N] Arnoldi columns built; negative once the basis stopped early
  const float *fm_adiag;   // [N or 1][n_pad] diagonal of A^-1 (fm_adiag_stride 0: shared)
  float *fm_u;         // [cols_pad][n_pad] A^-1 applied to the Krylov forces
  int fm_m, fm_adiag_stride;
  int *status;         // the scene's status word (checked build: index range errors)
};

struct EnvView {
  const float *mu, *odims, *ocomp, *pose_t, *pose_th;
  const int *otype;
  int *iters, *done, *status, *active;
  const int *kit;
  float *rncp;
  int *gstate;
  const int *gobs;
  const float *ganchor;
};

GroupView view(const flash_scene *s, const Group &g) {
  GroupView v;
  v.n = g.n; v.n_pad = g.n_pad; v.E = g.E; v.H = g.H; v.vpe = g.vpe; v.nc = g.nc; v.type = g.type; v.cap = s->cap;
  v.genv = g.genv; v.elems = g.elems; v.D = g.D; v.wt = g.wt; v.mass = g.mass; v.erec = g.erec;
  v.q = g.q; v.v = g.v; v.qt = g.qt; v.qp = g.qp; v.r = g.r; v.f = g.f; v.w = g.w; v.dq = g.dq;
  v.rh = g.rh; v.rl = g.rl; v.rscale = g.rscale;
  v.ccount = g.ccount; v.cvert = g.cvert; v.cobs = g.cobs; v.pcount = g.pcount; v.pvert = g.pvert;
  v.pobs = g.pobs; v.cgam = g.cgam; v.pgam = g.pgam; v.cscratch = g.cscratch; v.gflag = g.gflag;
  v.self = g.self; v.selfc = g.selfc; v.ofeat = g.ofeat; v.ctri = g.ctri; v.pctri = g.pctri; v.fm_w = g.fm_w;
  v.ned = g.ned; v.edges = g.edges; v.eoff = g.eoff;
  v.c_in_smem = g.c_in_smem ? 1 : 0;
  v.coff = g.coff; v.cidx = g.cidx; v.kb = g.kb; v.ev = g.ev; v.deg_b = g.deg_b;
  v.fm_lin = g.fm_lin; v.fm_V = g.fm_V; v.fm_H = g.fm_H; v.fm_cs = g.fm_cs; v.fm_sn = g.fm_sn; v.fm_g = g.fm_g;
  v.fm_beta = g.fm_beta; v.fm_jm = g.fm_jm; v.fm_adiag = g.fm_adiag; v.fm_u = g.fm_u; v.fm_m = g.fm_m;
  v.fm_adiag_stride = g.fm_adiag_stride;
  v.kenv = g.eig ? g.kenv : nullptr;
  v.bf16 = s->d.solve == FLASH_SOLVE_BF16R ? 1 : 0;
  v.tau = (float)g.tau;
  v.status = s->status;
  return v;
}

EnvView eview(const flash_scene *s) {
  EnvView e;
  e.mu = s->mu; e.odims = s->odims; e.ocomp = s->ocomp; e.pose_t = s->pose_t; e.pose_th = s->pose_th;
  e.otype = s->otype; e.iters = s->iters; e.done = s->done; e.status = s->status; e.active = s->active;
  e.kit = s->kit;
  e.rncp = s->rncp;
  e.gstate = s->gstate; e.gobs = s->gobs; e.ganchor = s->ganchor;
  return e;
}

// Index range check of the checked build (FLASH_CHECK): an index outside
// [0, n) sets bit 12 of the status word and reads as 0, so no access leaves
// its array.  The regular build passes every index through unchanged.
__device__ __forceinline__ int chk(int i, int n, int *status) {
#ifdef FLASH_CHECK
  if ((unsigned)i >= (unsigned)n) {
    atomicOr(status, 1 << 12);
    return 0;
  }
#else
  (void)n;
  (void)status;
#endif
  return i;
}
// corner k of element f, a vertex of the group's mesh
__device__ __forceinline__ int elem_v(const GroupView &G, int f, int k) {
  return chk(G.elems[4 * f + k], G.n, G.status);
}
// the CSR tables: slot offsets of vertex p, and the element slot at sl
__device__ __forceinline__ int csr_off(const GroupView &G, int p) { return chk(G.coff[p], G.ev + 1, G.status); }
__device__ __forceinline__ int csr_slot(const GroupView &G, int sl) { return chk(G.cidx[sl], G.ev, G.status); }
__device__ __forceinline__ int2 edge_v(const GroupView &G, int e) {
  const int2 E = G.edges[e];
  return make_int2(chk(E.x, G.n, G.status), chk(E.y, G.n, G.status));
}

// block-wide exclusive scan of one int per thread (blockDim <= 1024)
__device__ int block_exclusive_scan(int x, int *total, int *sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int inc = x;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int t = lane < nw ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sh[lane] = t;  // inclusive warp totals
  }
  __syncthreads();
  int base = wid > 0 ? sh[wid - 1] : 0;
  *total = sh[nw - 1];
  __syncthreads();
  return base + inc - x;
}

__device__ float block_max(float x, float *sh) {
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  float t = lane < nw ? sh[lane] : 0.f;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  float r = sh[0];
  __syncthreads();
  return r;
}

// block-wide max of three values at once (2 barriers)
__device__ void block_max3(float &x0, float &x1, float &x2, float (*sh)[3]) {
  for (int o = 16; o > 0; o >>= 1) {
    x0 = fmaxf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
    x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
    x2 = fmaxf(x2, __shfl_xor_sync(0xffffffffu, x2, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) { sh[wid][0] = x0; sh[wid][1] = x1; sh[wid][2] = x2; }
  __syncthreads();
  float m0 = 0.f, m1 = 0.f, m2 = 0.f;
  for (int w = 0; w < nw; w++) { m0 = fmaxf(m0, sh[w][0]); m1 = fmaxf(m1, sh[w][1]); m2 = fmaxf(m2, sh[w][2]); }
  x0 = m0; x1 = m1; x2 = m2;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// begin of step: q_t, q~, detection, gamma^0
// ---------------------------------------------------------------------------
// Self-contact candidate (cloth self-collision, the library's reading; the
// paper disables it): vertex p and triangle f (not touching a triangle of
// p), p within `reach` of f's plane with its projection inside f up to
// kSelfBary (barycentric), at q_t or at q~.
constexpr float kSelfBary = 0.1f;
constexpr int kSlots = FLASH_OEE_SLOT + 1;   // contact-list slots: obstacles, grasp, self, edge-edge, box features

__device__ __forceinline__ bool self_candidate(const GroupView &G, int p, int f, float reach, const float *x0,
                                               const float *x1) {
  const int np = G.n_pad;
  const int t0 = elem_v(G, f, 0), t1 = elem_v(G, f, 1), t2 = elem_v(G, f, 2);
  if (t0 == p || t1 == p || t2 == p) return false;
  bool hit = false;
  for (int k = 0; k < 2 && !hit; k++) {
    const float *x = k == 0 ? x0 : x1;
    const V3 A = v3(x[t0], x[np + t0], x[2 * np + t0]), B = v3(x[t1], x[np + t1], x[2 * np + t1]);
    const V3 Cc = v3(x[t2], x[np + t2], x[2 * np + t2]), P = v3(x[p], x[np + p], x[2 * np + p]);
    const V3 nf = cross(B - A, Cc - A);
    const float ar = norm(nf);
    if (!(ar > 0.f)) continue;
    const V3 nh = (1.f / ar) * nf;
    const float d = dot(nh, P - A);
    const V3 y = P - d * nh;
    const float wa = dot(nh, cross(B - y, Cc - y)) / ar, wb = dot(nh, cross(Cc - y, A - y)) / ar;
    const float wc = 1.f - wa - wb;
    hit = fabsf(d) < reach && wa >= -kSelfBary && wb >= -kSelfBary && wc >= -kSelfBary;
  }
  if (!hit) return false;
  // f must not touch a triangle of p (topological neighbours never collide)
  for (int sl = csr_off(G, p); sl < csr_off(G, p + 1); sl++) {
    const int g = csr_slot(G, sl) / 3;
    for (int c = 0; c < 3; c++) {
      const int u = elem_v(G, g, c);
      if (u == t0 || u == t1 || u == t2) return false;
    }
  }
  return true;
}

// Closest points of the lines through (A, B) and (C, D): A + s (B - A) and
// C + t (D - C).  With nn = (B - A) x (D - C): s = ((C - A) x (D - C)).nn /
// |nn|^2 and t = ((C - A) x (B - A)).nn / |nn|^2, which keeps the
// cancellation of |d1|^2 |d2|^2 - (d1.d2)^2 out of near-parallel pairs;
// false when the lines are parallel to rounding.
__device__ __forceinline__ bool line_params(V3 A, V3 B, V3 C, V3 D, float &s, float &t) {
  const V3 d1 = B - A, d2 = D - C, r = C - A;
  const V3 nn = cross(d1, d2);
  const float n2 = dot(nn, nn);
  if (!(n2 > 1e-12f * dot(d1, d1) * dot(d2, d2))) return false;
  s = dot(cross(r, d2), nn) / n2;
  t = dot(cross(r, d1), nn) / n2;
  return true;
}

__device__ __forceinline__ V3 col3(const float *x, int ld, int i) { return v3(x[i], x[ld + i], x[2 * ld + i]); }

// Edge-edge candidate (the library's reading, like the vertex-triangle one):
// edges e1 = (a, b) and e2 = (c, d) with no common vertex and no triangle
// holding a or b together with c or d, whose lines' closest points lie
// inside both edges and nearer than `reach`, at q_t or at q~.
__device__ __forceinline__ bool ee_candidate(const GroupView &G, int e1, int e2, float reach, const float *x0,
                                             const float *x1) {
  const int np = G.n_pad;
  const int2 E1 = edge_v(G, e1), E2 = edge_v(G, e2);
  const int a = E1.x, b = E1.y, c = E2.x, d = E2.y;
  if (a == c || a == d || b == c || b == d) return false;
  bool hit = false;
  for (int k = 0; k < 2 && !hit; k++) {
    const float *x = k == 0 ? x0 : x1;
    const V3 A = col3(x, np, a), B = col3(x, np, b), C = col3(x, np, c), D = col3(x, np, d);
    float s, t;
    if (!line_params(A, B, C, D, s, t)) continue;
    if (!(s > 0.f && s < 1.f && t > 0.f && t < 1.f)) continue;
    const V3 dd = (A - C) + s * (B - A) - t * (D - C);
    hit = norm(dd) < reach;
  }
  if (!hit) return false;
  for (int k = 0; k < 2; k++) {
    const int p = k == 0 ? a : b;
    for (int sl = csr_off(G, p); sl < csr_off(G, p + 1); sl++) {
      const int g = csr_slot(G, sl) / 3;
      for (int j = 0; j < 3; j++) {
        const int u = elem_v(G, g, j);
        if (u == c || u == d) return false;
      }
    }
  }
  return true;
}

// Box features (the library's reading; the paper describes none).  Corner
// k of a box: bit i of k set = +half extent on axis i.  Edge j: along axis
// j / 4, on the sides of the other two axes (in increasing order) given by
// bits 0 and 1 of j % 4.
__device__ __forceinline__ V3 box_corner_body(const float *d, int k) {
  return v3((k & 1) ? d[0] : -d[0], (k & 2) ? d[1] : -d[1], (k & 4) ? d[2] : -d[2]);
}
__device__ __forceinline__ void box_edge_body(const float *d, int j, V3 &p0, V3 &p1) {
  const int ax = j >> 2, m = j & 3;
  const float sb = (m & 1) ? 1.f : -1.f, sc = (m & 2) ? 1.f : -1.f;
  if (ax == 0) { p0 = v3(-d[0], sb * d[1], sc * d[2]); p1 = v3(d[0], sb * d[1], sc * d[2]); }
  else if (ax == 1) { p0 = v3(sb * d[0], -d[1], sc * d[2]); p1 = v3(sb * d[0], d[1], sc * d[2]); }
  else { p0 = v3(sb * d[0], sc * d[1], -d[2]); p1 = v3(sb * d[0], sc * d[1], d[2]); }
}
__device__ __forceinline__ V3 pose_point(const float *pose, V3 pb) {
  return qrot(pose + 3, pb, false) + v3(pose[0], pose[1], pose[2]);
}

// Box-corner candidate: the corner C within `reach` of triangle f's plane,
// its projection inside f up to kSelfBary (barycentric), at q_t or at q~.
__device__ __forceinline__ bool ovt_candidate(const GroupView &G, int f, V3 C, float reach, const float *x0,
                                              const float *x1) {
  const int np = G.n_pad;
  const int t0 = elem_v(G, f, 0), t1 = elem_v(G, f, 1), t2 = elem_v(G, f, 2);
  for (int k = 0; k < 2; k++) {
    const float *x = k == 0 ? x0 : x1;
    const V3 A = col3(x, np, t0), B = col3(x, np, t1), Cc = col3(x, np, t2);
    const V3 nf = cross(B - A, Cc - A);
    const float ar = norm(nf);
    if (!(ar > 0.f)) continue;
    const V3 nh = (1.f / ar) * nf;
    const float d = dot(nh, C - A);
    const V3 y = C - d * nh;
    const float wa = dot(nh, cross(B - y, Cc - y)) / ar, wb = dot(nh, cross(Cc - y, A - y)) / ar;
    const float wc = 1.f - wa - wb;
    if (fabsf(d) < reach && wa >= -kSelfBary && wb >= -kSelfBary && wc >= -kSelfBary) return true;
  }
  return false;
}

// Box-edge candidate: the box edge (C, D) and the cloth edge e, whose lines'
// closest points lie inside both and nearer than `reach`, at q_t or at q~.
__device__ __forceinline__ bool oee_candidate(const GroupView &G, int e, V3 C, V3 D, float reach, const float *x0,
                                              const float *x1) {
  const int np = G.n_pad;
  const int2 E = edge_v(G, e);
  for (int k = 0; k < 2; k++) {
    const float *x = k == 0 ? x0 : x1;
    const V3 A = col3(x, np, E.x), B = col3(x, np, E.y);
    float s, t;
    if (!line_params(A, B, C, D, s, t)) continue;
    if (!(s > 0.f && s < 1.f && t > 0.f && t < 1.f)) continue;
    if (norm((A - C) + s * (B - A) - t * (D - C)) < reach) return true;
  }
  return false;
}

// SELF: the group detects cloth self contacts (a compile-time switch, so the
// kernels of scenes without self-collision carry none of its code)
template <bool SELF>
__device__ __forceinline__ void begin_body(const GroupView &G, const int l, const EnvView &V, StepArgs a, int boxes) {
  __shared__ int sh_scan[32];
  __shared__ int s_type[FLASH_MAX_OBS];
  __shared__ float s_dims[FLASH_MAX_OBS][3], s_pose[FLASH_MAX_OBS][7];
  a.tau = G.tau;
  const bool self = SELF && G.self;   // tetrahedral groups of a self-collision scene have none
  const bool selfc = self && G.selfc, ofeat = self && G.ofeat;
  const int e = G.genv[l];
  const int n = G.n, np = G.n_pad;
  float *q = G.q + (size_t)l * 3 * np, *v = G.v + (size_t)l * 3 * np;
  float *qt = G.qt + (size_t)l * 3 * np, *qp = G.qp + (size_t)l * 3 * np, *f = G.f + (size_t)l * 3 * np;
  if (threadIdx.x < a.K) {
    int o = threadIdx.x;
    s_type[o] = V.otype[e * FLASH_MAX_OBS + o];
    for (int c = 0; c < 3; c++) s_dims[o][c] = V.odims[(e * FLASH_MAX_OBS + o) * 3 + c];
    for (int c = 0; c < 7; c++) s_pose[o][c] = V.pose_th[(e * FLASH_MAX_OBS + o) * 7 + c];
  }
  if (threadIdx.x == 0) V.done[e] = 0;
  // bilateral grasp: a pending activation takes the vertices within the
  // radius of the anchor at the carrying obstacle's current pose; a pending
  // release empties the set (appendix, Bilateral Constraint for Cloth Control)
  const int gst = V.gstate[e];
  V3 gp = v3(0.f, 0.f, 0.f);
  float grad2 = -1.f;
  if (gst == 1) {
    const float *ps = V.pose_t + (e * FLASH_MAX_OBS + V.gobs[e]) * 7;
    const float *an = V.ganchor + 4 * e;
    gp = qrot(ps + 3, v3(an[0], an[1], an[2]), false) + v3(ps[0], ps[1], ps[2]);
    grad2 = an[3] * an[3];
  }
  uint8_t *gflag = G.gflag + (size_t)l * np;
  const float h = a.h, h2 = a.h * a.h;
  const float gv[3] = {a.gx, a.gy, a.gz};
  if (self) {
    // self contacts test triangles against q_t and q~ of every vertex: both
    // are written first
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      for (int c = 0; c < 3; c++) {
        const float qq = q[c * np + i], pp = qq + h * v[c * np + i] + h2 * gv[c];
        qt[c * np + i] = qq;
        qp[c * np + i] = pp;
        q[c * np + i] = pp;   // q^0 = q~
        f[c * np + i] = 0.f;
      }
  }
  __syncthreads();
  // per-triangle boxes over q_t and q~, grown by the reach plus a fifth of the
  // longest edge (a projection may lie a tenth outside in barycentric terms):
  // a vertex whose own box misses a triangle's cannot be its candidate.
  // Per-edge boxes over q_t and q~ grown by the reach: two edges whose
  // boxes miss each other cannot come within reach.
  extern __shared__ float sbox[];   // [E][6] then [ned][6] when boxes
  const float reach = a.tau + a.margin;
  if (selfc && boxes) {
    for (int t = threadIdx.x; t < G.E; t += blockDim.x) {
      float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, el = 0.f;
      int tv[3];
      for (int k = 0; k < 3; k++) tv[k] = elem_v(G, t, k);
      for (int k = 0; k < 3; k++)
        for (int c = 0; c < 3; c++) {
          const float x0 = qt[c * np + tv[k]], x1 = qp[c * np + tv[k]];
          lo[c] = fminf(lo[c], fminf(x0, x1));
          hi[c] = fmaxf(hi[c], fmaxf(x0, x1));
        }
      for (int c = 0; c < 3; c++) el = fmaxf(el, hi[c] - lo[c]);
      const float g = reach + 0.2f * 1.7320508f * el;   // longest edge <= sqrt(3) x the box's largest side
      for (int c = 0; c < 3; c++) { sbox[6 * t + c] = lo[c] - g; sbox[6 * t + 3 + c] = hi[c] + g; }
    }
    float *ebox = sbox + 6 * G.E;
    for (int k = threadIdx.x; k < G.ned; k += blockDim.x) {
      const int2 ev = edge_v(G, k);
      for (int c = 0; c < 3; c++) {
        const float a0 = qt[c * np + ev.x], a1 = qp[c * np + ev.x], b0 = qt[c * np + ev.y], b1 = qp[c * np + ev.y];
        ebox[6 * k + c] = fminf(fminf(a0, a1), fminf(b0, b1)) - reach;
        ebox[6 * k + 3 + c] = fmaxf(fmaxf(a0, a1), fmaxf(b0, b1)) + reach;
      }
    }
    __syncthreads();
  }
  int base = 0;
  int *cvert = G.cvert + (size_t)l * G.cap, *cobs = G.cobs + (size_t)l * G.cap;
  int *ctri = self ? G.ctri + (size_t)l * G.cap : nullptr;
  for (int i0 = 0; i0 < n; i0 += blockDim.x) {
    int i = i0 + threadIdx.x;
    unsigned mask = 0;
    int sf[FLASH_SELF_MAX], se[FLASH_EE_MAX], sv[FLASH_OFEAT_MAX], sb[FLASH_OFEAT_MAX];
    int ns = 0, ne = 0, nv = 0, nb = 0;
    if (i < n) {
      float x0[3], x1[3];
      if (self) {
        for (int c = 0; c < 3; c++) { x0[c] = qt[c * np + i]; x1[c] = qp[c * np + i]; }
      } else {
        for (int c = 0; c < 3; c++) {
          float qq = q[c * np + i], vv = v[c * np + i];
          float pp = qq + h * vv + h2 * gv[c];
          qt[c * np + i] = qq;
          qp[c * np + i] = pp;
          q[c * np + i] = pp;   // q^0 = q~
          f[c * np + i] = 0.f;
          x0[c] = qq;
          x1[c] = pp;
        }
      }
      if (gst == 1) {
        const V3 d = v3(x0[0], x0[1], x0[2]) - gp;
        gflag[i] = dot(d, d) <= grad2 ? 1 : 0;
      } else if (gst == 3) {
        gflag[i] = 0;
      }
      if (gflag[i]) mask |= 1u << FLASH_GRASP_SLOT;
      // box features: a box can reach a triangle or edge of i only if it
      // comes within reach + 1.3 L of i, L the longest edge at i at q_t or
      // q~ (a projection inside the triangle up to 0.1 lies within 1.3 L of
      // its first corner)
      float cull = -INFINITY;
      if (ofeat) {
        float L2 = 0.f;
        for (int sl = csr_off(G, i); sl < csr_off(G, i + 1); sl++) {
          const int t = csr_slot(G, sl) / 3;
          for (int c = 0; c < 3; c++) {
            const int u = elem_v(G, t, c);
            const V3 d0 = col3(qt, np, u) - v3(x0[0], x0[1], x0[2]), d1 = col3(qp, np, u) - v3(x1[0], x1[1], x1[2]);
            L2 = fmaxf(L2, fmaxf(dot(d0, d0), dot(d1, d1)));
          }
        }
        cull = a.tau + a.margin + 1.3f * sqrtf(L2) + 1e-4f;
      }
      unsigned near = 0;
      for (int o = 0; o < a.K; o++) {
        if (s_type[o] == FLASH_OBS_NONE) continue;
        V3 nn;
        float s0 = obstacle_sdf(s_type[o], s_dims[o], s_pose[o], v3(x0[0], x0[1], x0[2]), nn);
        float s1 = obstacle_sdf(s_type[o], s_dims[o], s_pose[o], v3(x1[0], x1[1], x1[2]), nn);
        if (fminf(s0, s1) < a.tau + a.margin) mask |= 1u << o;
        if (s_type[o] == FLASH_OBS_BOX && fminf(s0, s1) < cull) near |= 1u << o;
      }
      if (near) {
        // corners against the triangles whose first vertex is i (element
        // slots 3 f + 0 of i, f ascending), then box edges against the
        // edges (i, b), each in feature order
        for (int sl = csr_off(G, i); sl < csr_off(G, i + 1) && nv < FLASH_OFEAT_MAX; sl++) {
          const int cs = csr_slot(G, sl);
          if (cs % 3 != 0) continue;
          const int f = cs / 3;
          for (int o = 0; o < a.K && nv < FLASH_OFEAT_MAX; o++) {
            if (!((near >> o) & 1u)) continue;
            for (int k = 0; k < 8 && nv < FLASH_OFEAT_MAX; k++)
              if (ovt_candidate(G, f, pose_point(s_pose[o], box_corner_body(s_dims[o], k)), reach, qt, qp))
                sv[nv++] = (f * FLASH_MAX_OBS + o) * 8 + k;
          }
        }
        for (int e1 = chk(G.eoff[i], G.ned + 1, G.status); e1 < chk(G.eoff[i + 1], G.ned + 1, G.status) && nb < FLASH_OFEAT_MAX; e1++)
          for (int o = 0; o < a.K && nb < FLASH_OFEAT_MAX; o++) {
            if (!((near >> o) & 1u)) continue;
            for (int j = 0; j < 12 && nb < FLASH_OFEAT_MAX; j++) {
              V3 p0, p1;
              box_edge_body(s_dims[o], j, p0, p1);
              if (oee_candidate(G, e1, pose_point(s_pose[o], p0), pose_point(s_pose[o], p1), reach, qt, qp))
                sb[nb++] = (e1 * FLASH_MAX_OBS + o) * 12 + j;
            }
          }
      }
      if (selfc) {   // the first FLASH_SELF_MAX candidate triangles in index order
        const float vlo[3] = {fminf(x0[0], x1[0]), fminf(x0[1], x1[1]), fminf(x0[2], x1[2])};
        const float vhi[3] = {fmaxf(x0[0], x1[0]), fmaxf(x0[1], x1[1]), fmaxf(x0[2], x1[2])};
        for (int t = 0; t < G.E && ns < FLASH_SELF_MAX; t++) {
          if (boxes) {
            const float *b = sbox + 6 * t;
            if (vhi[0] < b[0] || vlo[0] > b[3] || vhi[1] < b[1] || vlo[1] > b[4] || vhi[2] < b[2] || vlo[2] > b[5])
              continue;
          }
          if (self_candidate(G, i, t, reach, qt, qp)) sf[ns++] = t;
        }
        // edge-edge: the first FLASH_EE_MAX pairs (e1, e2 > e1) of the edges
        // i owns (e1, then e2 ascending); the pair (e2, e1) would repeat the
        // same constraint
        const float *ebox = sbox + 6 * G.E;
        for (int e1 = chk(G.eoff[i], G.ned + 1, G.status); e1 < chk(G.eoff[i + 1], G.ned + 1, G.status) && ne < FLASH_EE_MAX; e1++) {
          float b1[6];
          if (boxes)
            for (int c = 0; c < 6; c++) b1[c] = ebox[6 * e1 + c];
          for (int e2 = e1 + 1; e2 < G.ned && ne < FLASH_EE_MAX; e2++) {
            if (boxes) {
              const float *b = ebox + 6 * e2;
              if (b1[3] < b[0] || b1[0] > b[3] || b1[4] < b[1] || b1[1] > b[4] || b1[5] < b[2] || b1[2] > b[5])
                continue;
            }
            if (ee_candidate(G, e1, e2, reach, qt, qp)) se[ne++] = e1 * G.ned + e2;
          }
        }
      }
    }
    int cnt = __popc(mask) + ns + ne + nv + nb, total;
    int off = block_exclusive_scan(cnt, &total, sh_scan);
    int pos = base + off;
    for (int o = 0; o < a.K; o++)
      if (mask & (1u << o)) {
        if (pos < G.cap) { cvert[pos] = i; cobs[pos] = o; if (ctri) ctri[pos] = -1; }
        pos++;
      }
    if (mask & (1u << FLASH_GRASP_SLOT)) {   // the grasp row follows the obstacle rows
      if (pos < G.cap) { cvert[pos] = i; cobs[pos] = FLASH_GRASP_SLOT; if (ctri) ctri[pos] = -1; }
      pos++;
    }
    for (int k = 0; k < ns; k++) {           // then the self contacts
      if (pos < G.cap) { cvert[pos] = i; cobs[pos] = FLASH_SELF_SLOT; ctri[pos] = sf[k]; }
      pos++;
    }
    for (int k = 0; k < ne; k++) {
      if (pos < G.cap) { cvert[pos] = i; cobs[pos] = FLASH_EE_SLOT; ctri[pos] = se[k]; }
      pos++;
    }
    for (int k = 0; k < nv; k++) {           // then the box features
      if (pos < G.cap) { cvert[pos] = i; cobs[pos] = FLASH_OVT_SLOT; ctri[pos] = sv[k]; }
      pos++;
    }
    for (int k = 0; k < nb; k++) {
      if (pos < G.cap) { cvert[pos] = i; cobs[pos] = FLASH_OEE_SLOT; ctri[pos] = sb[k]; }
      pos++;
    }
    base += total;
  }
  if (threadIdx.x == 0) {
    G.ccount[l] = min(base, G.cap);
    if (base > G.cap) atomicOr(V.status, 1 << 8);
    if (gst == 1) V.gstate[e] = 2;
    if (gst == 3) V.gstate[e] = 0;
  }
  __syncthreads();
  int cnt = min(base, G.cap);
  float *gam = G.cgam + (size_t)l * G.cap * 4;
  const int pc = G.pcount[l];
  const int *pv = G.pvert + (size_t)l * G.cap, *po = G.pobs + (size_t)l * G.cap;
  const int *pt = self ? G.pctri + (size_t)l * G.cap : nullptr;
  const float *pg = G.pgam + (size_t)l * G.cap * 4;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    float g4[4] = {0.f, 0.f, 0.f, 0.f};
    if (a.warm == FLASH_WARM_PREV && pc > 0) {
      // previous list sorted by (vertex, slot, feature)
      const long long key = (long long)(cvert[j] * kSlots + cobs[j]) * 0x100000000LL + (ctri ? ctri[j] + 1 : 0);
      int lo = 0, hi = pc - 1;
      while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        const long long km = (long long)(pv[mid] * kSlots + po[mid]) * 0x100000000LL + (pt ? pt[mid] + 1 : 0);
        if (km == key) {
          for (int c = 0; c < 4; c++) g4[c] = pg[mid * 4 + c];
          break;
        }
        if (km < key) lo = mid + 1; else hi = mid - 1;
      }
    }
    for (int c = 0; c < 4; c++) gam[j * 4 + c] = g4[c];
  }
}

// ---------------------------------------------------------------------------
// local step + residual
// ---------------------------------------------------------------------------
// Write one environment's three columns in f16 hi/lo with a power-of-two
// scale per column (tensor-core RHS); vals in shared memory [3][ld].  Each
// thread passes the maxima of |vals| it already knows (or 0); the kernel
// completes them over the rows this thread owns and reduces once.
__device__ void write_split_columns(const GroupView &G, int l, const float *vals, int ld, float (*sh3)[3], bool scan,
                                    float m0 = 0.f, float m1 = 0.f, float m2 = 0.f, float *fp32 = nullptr) {
  const int n = G.n, np = G.n_pad;
  float m[3] = {m0, m1, m2};
  if (scan)
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      for (int c = 0; c < 3; c++) m[c] = fmaxf(m[c], fabsf(vals[c * ld + i]));
  block_max3(m[0], m[1], m[2], sh3);
  for (int c = 0; c < 3; c++) {
    int ex = 0;
    if (m[c] > 0.f) {
      frexpf(m[c], &ex);   // m = f * 2^ex, f in [0.5, 1)
      // scaled max in [2^13, 2^14); the cap keeps 2^ex finite and 2^-ex a
      // normal float for columns below 2^-112 (a contact update that has
      // converged to rounding level), which then scale to less than 2^14.
      ex = min(14 - ex, 126);
    }
    const float sc = ldexpf(1.f, ex);
    const size_t col = (size_t)(l * 3 + c);
    if (threadIdx.x == 0) G.rscale[col] = ldexpf(1.f, -ex);
    if (G.bf16) {
      // one bf16 column with the same power-of-two scale, and the FP32
      // values the refinement's residual starts from
      __nv_bfloat162 *hb = reinterpret_cast<__nv_bfloat162 *>(G.rh + col * np);
      for (int i = threadIdx.x; i < np / 2; i += blockDim.x) {
        const float x0 = 2 * i < n ? vals[c * ld + 2 * i] : 0.f, x1 = 2 * i + 1 < n ? vals[c * ld + 2 * i + 1] : 0.f;
        hb[i] = __floats2bfloat162_rn(x0 * sc, x1 * sc);
        if (fp32) *reinterpret_cast<float2 *>(fp32 + col * np + 2 * i) = make_float2(x0, x1);
      }
      continue;
    }
    __half2 *hh = reinterpret_cast<__half2 *>(G.rh + col * np), *hl = reinterpret_cast<__half2 *>(G.rl + col * np);
    for (int i = threadIdx.x; i < np / 2; i += blockDim.x) {
      const float x0 = 2 * i < n ? vals[c * ld + 2 * i] * sc : 0.f;
      const float x1 = 2 * i + 1 < n ? vals[c * ld + 2 * i + 1] * sc : 0.f;
      const __half2 xh = __floats2half2_rn(x0, x1);
      hh[i] = xh;
      const float2 back = __half22float2(xh);
      hl[i] = __floats2half2_rn(x0 - back.x, x1 - back.y);
    }
  }
}

struct ObsShared {
  int type[FLASH_MAX_OBS];
  float dims[FLASH_MAX_OBS][3], pose[FLASH_MAX_OBS][7], poset[FLASH_MAX_OBS][7], comp[FLASH_MAX_OBS];
  PoseM pm[FLASH_MAX_OBS];
  float gp[3];   // grasp target p_grip(t+h)
};

__device__ __forceinline__ void load_obstacles(const EnvView &V, int e, int K, ObsShared &O) {
  if (threadIdx.x < K) {
    int o = threadIdx.x;
    O.type[o] = V.otype[e * FLASH_MAX_OBS + o];
    O.comp[o] = V.ocomp[e * FLASH_MAX_OBS + o];
    for (int c = 0; c < 3; c++) O.dims[o][c] = V.odims[(e * FLASH_MAX_OBS + o) * 3 + c];
    for (int c = 0; c < 7; c++) {
      O.pose[o][c] = V.pose_th[(e * FLASH_MAX_OBS + o) * 7 + c];
      O.poset[o][c] = V.pose_t[(e * FLASH_MAX_OBS + o) * 7 + c];
    }
    make_posem(O.poset[o], O.pose[o], O.pm[o]);
  }
  if (threadIdx.x == 0) {
    const int go = V.gobs[e];
    if (go >= 0) {
      const float *ps = V.pose_th + (e * FLASH_MAX_OBS + go) * 7;
      const float *an = V.ganchor + 4 * e;
      const V3 p = qrot(ps + 3, v3(an[0], an[1], an[2]), false) + v3(ps[0], ps[1], ps[2]);
      O.gp[0] = p.x; O.gp[1] = p.y; O.gp[2] = p.z;
    } else {
      O.gp[0] = 0.f; O.gp[1] = 0.f; O.gp[2] = 0.f;
    }
  }
}

// Grasp row: the frame is the world axes, phi = x - p_grip(t+h) (the
// constraint itself), D_C = I (phi moves one to one with x) and D_y = 0 (a
// rigid, zero-length link); never "separated".
__device__ __forceinline__ void linearize_grasp(const float *gp, V3 x, ContactLin &L) {
#pragma unroll
  for (int t = 0; t < 9; t++) L.R[t] = (t % 4 == 0) ? 1.f : 0.f;
  L.phi[0] = x.x - gp[0]; L.phi[1] = x.y - gp[1]; L.phi[2] = x.z - gp[2];
  L.cn = 1.f;
  L.Ct[0] = 1.f; L.Ct[1] = 0.f; L.Ct[2] = 0.f; L.Ct[3] = 1.f;
  L.dn = 0.f; L.dtn[0] = 0.f; L.dtn[1] = 0.f;
  L.Dtt[0] = 0.f; L.Dtt[1] = 0.f; L.Dtt[2] = 0.f; L.Dtt[3] = 0.f;
  L.gap = -1.f;
}

__device__ __forceinline__ void lin_at(const ObsShared &O, int o, const StepArgs &a, float mu, float mv, V3 x, V3 xt,
                                       const float *g, ContactLin &L) {
  if (o == FLASH_GRASP_SLOT) {
    linearize_grasp(O.gp, x, L);
    return;
  }
  linearize_contact_m(O.type[o], O.dims[o], O.comp[o], O.pm[o], a.tau, mu, a.h, mv, x, xt, g, L);
}

// A self-contact row moves the contact point as sum_k w_k x_{v_k} over four
// vertices (v_0 the row's own vertex); its multipliers scale with the
// effective mass meff = 1 / sum_k w_k^2 / m_{v_k}.
struct SelfRow {
  int v[4];
  float w[4];
  float meff;
};

// Self contact of vertex p with triangle f (cloth self-collision, the
// library's reading): positions x of the iterate ([3][ld]) and xt of the step
// start ([3][n_pad]).  Frame normal = f's unit normal, oriented towards the
// side p was on at q_t; gap = distance to the plane - tau; the contact point
// moves as p minus the barycentric combination w of f's corners (p's
// projection): weights (1, -w); slip = displacement of p relative to that
// point over the step.
__device__ __noinline__ void lin_self(const GroupView &G, int p, int f, const float *x, int ld, const float *xt,
                                      float mu, float h, float tau, const float *g, ContactLin &L, SelfRow &S) {
  const int np = G.n_pad;
  const int t[3] = {elem_v(G, f, 0), elem_v(G, f, 1), elem_v(G, f, 2)};
  V3 X[3], Xt[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    X[k] = col3(x, ld, t[k]);
    Xt[k] = col3(xt, np, t[k]);
  }
  const V3 P = col3(x, ld, p), Pt = col3(xt, np, p);
  const V3 nf = cross(X[1] - X[0], X[2] - X[0]);
  const float ar = norm(nf);
  V3 nh = v3(0.f, 0.f, 1.f);
  float d = 0.f;
  float w[3] = {1.f / 3.f, 1.f / 3.f, 1.f / 3.f};
  if (ar > 0.f) {
    nh = (1.f / ar) * nf;
    d = dot(nh, P - X[0]);
    const V3 y = P - d * nh;
    w[0] = dot(nh, cross(X[1] - y, X[2] - y)) / ar;
    w[1] = dot(nh, cross(X[2] - y, X[0] - y)) / ar;
    w[2] = 1.f - w[0] - w[1];
  }
  const float side = dot(cross(Xt[1] - Xt[0], Xt[2] - Xt[0]), Pt - Xt[0]) < 0.f ? -1.f : 1.f;
  const V3 n = side * nh;
  float inv = 1.f / __ldg(G.mass + p);
  V3 rel = P - Pt;
  S.v[0] = p;
  S.w[0] = 1.f;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    inv += w[k] * w[k] / __ldg(G.mass + t[k]);
    rel = rel - w[k] * (X[k] - Xt[k]);
    S.v[1 + k] = t[k];
    S.w[1 + k] = -w[k];
  }
  S.meff = 1.f / inv;
  V3 t1, t2;
  tangent_basis(n, t1, t2);
  contact_law(n, t1, t2, side * d - tau, rel, 0.f, mu, h, S.meff, g, L);
}

// Edge-edge contact of e1 = (a, b) with e2 = (c, d) (the library's reading):
// (s, t) = closest points of the two lines at x (1/2 when parallel), weights
// (1 - s, s, -(1 - t), -t); frame normal = the unit normal of both edges at
// x, oriented by the side e1 was on at q_t; gap = n.(point on e1 - point on
// e2) - tau; slip = that difference's displacement over the step.
__device__ __noinline__ void lin_ee(const GroupView &G, int e1, int e2, const float *x, int ld, const float *xt,
                                    float mu, float h, float tau, const float *g, ContactLin &L, SelfRow &S) {
  const int np = G.n_pad;
  const int2 E1 = edge_v(G, e1), E2 = edge_v(G, e2);
  const int v[4] = {E1.x, E1.y, E2.x, E2.y};
  V3 X[4], Dx[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    X[k] = col3(x, ld, v[k]);
    Dx[k] = X[k] - col3(xt, np, v[k]);
  }
  float s = 0.5f, t = 0.5f;
  line_params(X[0], X[1], X[2], X[3], s, t);
  const V3 nc = cross(X[1] - X[0], X[3] - X[2]);
  const float nl = norm(nc);
  const V3 nr = nl > 0.f ? (1.f / nl) * nc : v3(0.f, 0.f, 1.f);
  // the side at q_t: n_t.(a - c) (n_t is normal to both edges, so any pair of
  // points on them gives the same value)
  const V3 At = col3(xt, np, v[0]), Ct = col3(xt, np, v[2]);
  const V3 nt = cross(col3(xt, np, v[1]) - At, col3(xt, np, v[3]) - Ct);
  const float side = dot(nt, At - Ct) < 0.f ? -1.f : 1.f;
  const float w[4] = {1.f - s, s, -(1.f - t), -t};
  float inv = 0.f;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    inv += w[k] * w[k] / __ldg(G.mass + v[k]);
    S.v[k] = v[k];
    S.w[k] = w[k];
  }
  S.meff = 1.f / inv;
  const V3 dd = (X[0] - X[2]) + s * (X[1] - X[0]) - t * (X[3] - X[2]);
  const V3 rel = (Dx[0] - Dx[2]) + s * (Dx[1] - Dx[0]) - t * (Dx[3] - Dx[2]);
  const V3 n = side * nr;
  V3 t1, t2;
  tangent_basis(n, t1, t2);
  contact_law(n, t1, t2, dot(n, dd) - tau, rel, 0.f, mu, h, S.meff, g, L);
}

// Box corner k of obstacle o against triangle f (feature (f * FLASH_MAX_OBS
// + o) * 8 + k; the library's reading): weights w = barycentric weights of
// the box corner's projection on f's plane at x (row vertices f's corners,
// the first one the row's own); frame normal = f's unit normal, oriented
// towards the side the cloth was on, seen from the box corner, at q_t; gap
// = n.(sum w x - C) - tau, C the box corner at t+h; slip = that point's
// displacement relative to the box corner over the step.
__device__ __noinline__ void lin_ovt(const GroupView &G, const ObsShared &O, int feat, const float *x, int ld,
                                     const float *xt, float mu, float h, float tau, const float *g, ContactLin &L,
                                     SelfRow &S) {
  const int np = G.n_pad;
  const int f = feat / (8 * FLASH_MAX_OBS), o = feat / 8 % FLASH_MAX_OBS, kc = feat % 8;
  const int t[3] = {elem_v(G, f, 0), elem_v(G, f, 1), elem_v(G, f, 2)};
  const V3 cb = box_corner_body(O.dims[o], kc);
  const V3 C = pose_point(O.pose[o], cb), Ct = pose_point(O.poset[o], cb);
  V3 X[3], Xt[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    X[k] = col3(x, ld, t[k]);
    Xt[k] = col3(xt, np, t[k]);
  }
  const V3 nf = cross(X[1] - X[0], X[2] - X[0]);
  const float ar = norm(nf);
  V3 nh = v3(0.f, 0.f, 1.f);
  float d = 0.f;
  float w[3] = {1.f / 3.f, 1.f / 3.f, 1.f / 3.f};
  if (ar > 0.f) {
    nh = (1.f / ar) * nf;
    d = dot(nh, C - X[0]);
    const V3 y = C - d * nh;
    w[0] = dot(nh, cross(X[1] - y, X[2] - y)) / ar;
    w[1] = dot(nh, cross(X[2] - y, X[0] - y)) / ar;
    w[2] = 1.f - w[0] - w[1];
  }
  // the cloth lies on the -n_t side of the corner when the corner is on its + side
  const float side = dot(cross(Xt[1] - Xt[0], Xt[2] - Xt[0]), Ct - Xt[0]) > 0.f ? -1.f : 1.f;
  const V3 n = side * nh;
  float inv = 0.f;
  V3 rel = Ct - C;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    inv += w[k] * w[k] / __ldg(G.mass + t[k]);
    rel = rel + w[k] * (X[k] - Xt[k]);
    S.v[k] = t[k];
    S.w[k] = w[k];
  }
  S.v[3] = t[0];
  S.w[3] = 0.f;
  S.meff = 1.f / inv;
  V3 t1, t2;
  tangent_basis(n, t1, t2);
  contact_law(n, t1, t2, -side * d - tau, rel, 0.f, mu, h, S.meff, g, L);   // n.(sum w x - C) = -side d
}

// Box edge j of obstacle o against the cloth edge e = (a, b) (feature (e *
// FLASH_MAX_OBS + o) * 12 + j; the library's reading): (s, t) = closest
// points of the cloth edge's line and the box edge's line (C, D at t+h) at
// x (1/2 when parallel); weights (1 - s, s) on (a, b); frame normal = the
// unit normal of both lines, oriented by the side the cloth edge was on at
// q_t; gap = n.((1 - s) x_a + s x_b - (1 - t) C - t D) - tau; slip = that
// difference's displacement over the step.
__device__ __noinline__ void lin_oee(const GroupView &G, const ObsShared &O, int feat, const float *x, int ld,
                                     const float *xt, float mu, float h, float tau, const float *g, ContactLin &L,
                                     SelfRow &S) {
  const int np = G.n_pad;
  const int e = feat / (12 * FLASH_MAX_OBS), o = feat / 12 % FLASH_MAX_OBS, j = feat % 12;
  const int2 E = edge_v(G, e);
  V3 p0, p1;
  box_edge_body(O.dims[o], j, p0, p1);
  const V3 C = pose_point(O.pose[o], p0), D = pose_point(O.pose[o], p1);
  const V3 Ct = pose_point(O.poset[o], p0), Dt = pose_point(O.poset[o], p1);
  const V3 A = col3(x, ld, E.x), B = col3(x, ld, E.y), At = col3(xt, np, E.x), Bt = col3(xt, np, E.y);
  float s = 0.5f, t = 0.5f;
  line_params(A, B, C, D, s, t);
  const V3 nc = cross(B - A, D - C);
  const float nl = norm(nc);
  const V3 nr = nl > 0.f ? (1.f / nl) * nc : v3(0.f, 0.f, 1.f);
  // n_t is normal to both lines at q_t, so n_t.(a - C) is the side for any pair of points on them
  const float side = dot(cross(Bt - At, Dt - Ct), At - Ct) < 0.f ? -1.f : 1.f;
  const float ma = __ldg(G.mass + E.x), mb = __ldg(G.mass + E.y);
  S.v[0] = E.x; S.v[1] = E.y; S.v[2] = E.x; S.v[3] = E.x;
  S.w[0] = 1.f - s; S.w[1] = s; S.w[2] = 0.f; S.w[3] = 0.f;
  S.meff = 1.f / ((1.f - s) * (1.f - s) / ma + s * s / mb);
  const V3 dd = (A - C) + s * (B - A) - t * (D - C);
  const V3 rel = (1.f - s) * (A - At) + s * (B - Bt) - (1.f - t) * (C - Ct) - t * (D - Dt);
  const V3 n = side * nr;
  V3 t1, t2;
  tangent_basis(n, t1, t2);
  contact_law(n, t1, t2, dot(n, dd) - tau, rel, 0.f, mu, h, S.meff, g, L);
}

// a multi-vertex row (slot FLASH_SELF_SLOT, FLASH_EE_SLOT, FLASH_OVT_SLOT or
// FLASH_OEE_SLOT) of vertex vtx
__device__ __forceinline__ void lin_row(const GroupView &G, const ObsShared &O, int o, int vtx, int feat,
                                        const float *x, int ld, const float *xt, float mu, float h, float tau,
                                        const float *g, ContactLin &L, SelfRow &S) {
  if (o == FLASH_SELF_SLOT) lin_self(G, vtx, feat, x, ld, xt, mu, h, tau, g, L, S);
  else if (o == FLASH_EE_SLOT) lin_ee(G, feat / G.ned, feat % G.ned, x, ld, xt, mu, h, tau, g, L, S);
  else if (o == FLASH_OVT_SLOT) lin_ovt(G, O, feat, x, ld, xt, mu, h, tau, g, L, S);
  else lin_oee(G, O, feat, x, ld, xt, mu, h, tau, g, L, S);
}

// world force R^T gamma of a contact (gamma = (g_n, g_t world))
__device__ __forceinline__ V3 contact_force(const ContactLin &L, const float *g) {
  const float y1 = L.R[3] * g[1] + L.R[4] * g[2] + L.R[5] * g[3];
  const float y2 = L.R[6] * g[1] + L.R[7] * g[2] + L.R[8] * g[3];
  return v3(L.R[0] * g[0] + L.R[3] * y1 + L.R[6] * y2, L.R[1] * g[0] + L.R[4] * y1 + L.R[7] * y2,
            L.R[2] * g[0] + L.R[5] * y1 + L.R[8] * y2);
}

// w_k F added to the row's four vertices ([3][ld] columns)
__device__ __forceinline__ void scatter_row(const int v[4], const float w[4], V3 F, float *col, int ld) {
#pragma unroll
  for (int k = 0; k < 4; k++) {
    atomicAdd(col + v[k], w[k] * F.x);
    atomicAdd(col + ld + v[k], w[k] * F.y);
    atomicAdd(col + 2 * ld + v[k], w[k] * F.z);
  }
}

// full metric: a self row's weights, effective mass and vertices 1..3 (vertex
// 0 is the row's own) as stored by the setup kernel
__device__ __forceinline__ void fm_row_store(float *fw, const SelfRow &S) {
  *reinterpret_cast<float4 *>(fw) = make_float4(S.w[0], S.w[1], S.w[2], S.w[3]);
  *reinterpret_cast<float4 *>(fw + 4) =
      make_float4(S.meff, __int_as_float(S.v[1]), __int_as_float(S.v[2]), __int_as_float(S.v[3]));
}
__device__ __forceinline__ void fm_row_load(const float *fw, int vtx, SelfRow &S, int n, int *status) {
  const float4 a = *reinterpret_cast<const float4 *>(fw), b = *reinterpret_cast<const float4 *>(fw + 4);
  S.w[0] = a.x; S.w[1] = a.y; S.w[2] = a.z; S.w[3] = a.w;
  S.meff = b.x;
  S.v[0] = vtx;
  S.v[1] = chk(__float_as_int(b.y), n, status);
  S.v[2] = chk(__float_as_int(b.z), n, status);
  S.v[3] = chk(__float_as_int(b.w), n, status);
}

template <int VPE, bool SELF>
__device__ __forceinline__ void local_body(const GroupView &G, const int l, const EnvView &V, StepArgs a, int k,
                                           int residual_only, int tc, int pending) {
  // VPE = vertices per element: 3 (triangle, F is 3x2) or 4 (tet, F is 3x3)
  constexpr int nc = VPE - 1, vpe = VPE;
  extern __shared__ float smem[];
  __shared__ float sh_red[32];
  __shared__ float sh3[32][3];
  __shared__ int s_done;
  __shared__ ObsShared O;
  a.tau = G.tau;
  const int e = G.genv[l];
  const int n = G.n, np = G.n_pad, ns = (n + 3) & ~3;
  if (V.done[e]) return;
  float *qs = smem;             // [3][ns]
  float *rs = qs + 3 * ns;      // [3][ns]
  float *Fs;                    // element forces on their vertices [ev][3]
  const uint16_t *coff, *cidx;  // CSR vertex -> slots of Fs
  if (G.c_in_smem) {
    Fs = rs + 3 * ns;
    uint32_t *t = reinterpret_cast<uint32_t *>(Fs + 3 * (G.ev + 1));
    const int w_off = (n + 2) >> 1, w_idx = (G.ev + 1) >> 1;   // table sizes in 4-byte words
    const uint32_t *src_off = reinterpret_cast<const uint32_t *>(G.coff);
    const uint32_t *src_idx = reinterpret_cast<const uint32_t *>(G.cidx);
    for (int i = threadIdx.x; i < w_off; i += blockDim.x) t[i] = __ldg(src_off + i);
    for (int i = threadIdx.x; i < w_idx; i += blockDim.x) t[w_off + i] = __ldg(src_idx + i);
    coff = reinterpret_cast<const uint16_t *>(t);
    cidx = coff + 2 * w_off;
  } else {
    Fs = G.cscratch + (size_t)l * 3 * (G.ev + 1);
    coff = G.coff;
    cidx = G.cidx;
  }
  // q^{k-1} = q^{k-2} + w + A^-1 J^T dgamma: the previous iteration's position
  // update (correction form) is applied here, while the state is loaded, so
  // both global solves keep a store-only epilogue.  Columns are 16-byte
  // aligned (n_pad is a multiple of 128); the padding reads as zero.
  float *q = G.q + (size_t)l * 3 * np;
  const int n4 = ns >> 2;
  if (pending) {
    const float *w = G.w + (size_t)l * 3 * np, *dq = G.dq + (size_t)l * 3 * np;
    for (int i = threadIdx.x; i < 3 * n4; i += blockDim.x) {
      const int c = i / n4, j = (i - c * n4) * 4;
      float4 x = *reinterpret_cast<const float4 *>(q + c * np + j);
      const float4 u = *reinterpret_cast<const float4 *>(w + c * np + j);
      const float4 d = *reinterpret_cast<const float4 *>(dq + c * np + j);
      x.x = x.x + u.x + d.x; x.y = x.y + u.y + d.y; x.z = x.z + u.z + d.z; x.w = x.w + u.w + d.w;
      *reinterpret_cast<float4 *>(q + c * np + j) = x;
      *reinterpret_cast<float4 *>(qs + c * ns + j) = x;
    }
  } else {
    for (int i = threadIdx.x; i < 3 * n4; i += blockDim.x) {
      const int c = i / n4, j = (i - c * n4) * 4;
      *reinterpret_cast<float4 *>(qs + c * ns + j) = *reinterpret_cast<const float4 *>(q + c * np + j);
    }
  }
  load_obstacles(V, e, a.K, O);
  __syncthreads();
  if (!residual_only) {
    const float ks = G.kenv ? G.kenv[l] : 1.f;
    // ---- local projection p_i = closest rotation to F_i = G_i q, and the
    //      element's forces w~ D_a^T (p - F) on each of its vertices a.
    //      F is formed from edge differences (the operator annihilates
    //      translations), which keeps |q| out of its rounding.
    if constexpr (VPE == 3) {
      // triangles: one packed record per element (two 16-byte loads); the
      // force on the first vertex is minus the other two, so every element's
      // forces sum to zero as the operator's rows do
#pragma unroll 2
      for (int el = threadIdx.x; el < G.E; el += blockDim.x) {
        const float4 r0 = __ldg(G.erec + 2 * el), r1 = __ldg(G.erec + 2 * el + 1);
        const int v0 = chk(__float_as_int(r0.x), n, G.status), v1 = chk(__float_as_int(r0.y), n, G.status),
                  v2 = chk(__float_as_int(r0.z), n, G.status);
        float F[6], R[6], P[6];
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const float x0 = qs[c * ns + v0];
          const float d1 = qs[c * ns + v1] - x0, d2 = qs[c * ns + v2] - x0;
          F[2 * c] = d1 * r1.x + d2 * r1.z;
          F[2 * c + 1] = d1 * r1.y + d2 * r1.w;
        }
        closest_rot32(F, R);
        const float wt = r0.w * ks;
#pragma unroll
        for (int t = 0; t < 6; t++) P[t] = wt * (R[t] - F[t]);
        float *Fe = Fs + (size_t)el * 9;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const float f1 = r1.x * P[2 * c] + r1.y * P[2 * c + 1];
          const float f2 = r1.z * P[2 * c] + r1.w * P[2 * c + 1];
          Fe[3 + c] = f1;
          Fe[6 + c] = f2;
          Fe[c] = -(f1 + f2);
        }
      }
    } else {
    const bool fs16 = (reinterpret_cast<uintptr_t>(Fs) & 15) == 0;   // shared memory; the global scratch may not be
    for (int el = threadIdx.x; el < G.E; el += blockDim.x) {
      const int4 vi = *reinterpret_cast<const int4 *>(G.elems + 4 * el);
      const int vv[4] = {chk(vi.x, n, G.status), chk(vi.y, n, G.status), chk(vi.z, n, G.status),
                          chk(vi.w, n, G.status)};
      // the element's 4 x 3 operator rows: three 16-byte loads (48 B a record)
      const float4 *D4 = reinterpret_cast<const float4 *>(G.D + 12 * el);
      float F[9], R[9], P[9], Dl[12];
#pragma unroll
      for (int t = 0; t < 3; t++) {
        const float4 d = __ldg(D4 + t);
        Dl[4 * t] = d.x; Dl[4 * t + 1] = d.y; Dl[4 * t + 2] = d.z; Dl[4 * t + 3] = d.w;
      }
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const float x0 = qs[c * ns + vv[0]];
        float dx[vpe - 1];
#pragma unroll
        for (int aa = 1; aa < vpe; aa++) dx[aa - 1] = qs[c * ns + vv[aa]] - x0;
#pragma unroll
        for (int j = 0; j < nc; j++) {
          float s = 0.f;
#pragma unroll
          for (int aa = 1; aa < vpe; aa++) s += dx[aa - 1] * Dl[aa * 3 + j];
          F[nc * c + j] = s;
        }
      }
      if constexpr (nc == 2) closest_rot32(F, R);
      else closest_rot33(F, R);
      const float wt = __ldg(G.wt + el) * ks;
#pragma unroll
      for (int t = 0; t < 3 * nc; t++) P[t] = wt * (R[t] - F[t]);
      float *Fe = Fs + (size_t)el * vpe * 3;
      float fe[3 * vpe];
#pragma unroll
      for (int aa = 0; aa < vpe; aa++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
          float s = 0.f;
#pragma unroll
          for (int j = 0; j < nc; j++) s += Dl[aa * 3 + j] * P[nc * c + j];
          fe[aa * 3 + c] = s;
        }
      if (fs16) {   // 48-byte records: three 16-byte stores
#pragma unroll
        for (int t = 0; t < 3; t++)
          reinterpret_cast<float4 *>(Fe)[t] = make_float4(fe[4 * t], fe[4 * t + 1], fe[4 * t + 2], fe[4 * t + 3]);
      } else {
#pragma unroll
        for (int t = 0; t < 3 * vpe; t++) Fe[t] = fe[t];
      }
    }
    }
    // ---- per vertex: inertia M (q~ - q) and bending - sum_j K_ij (q_j - q_i).
    //      The operator's rows sum to zero; the terms are large and cancel.
    //      Summed naively, each vertex's rounding errors would add up to a net
    //      force over the mesh that the rigid modes of A^-1 amplify, so the
    //      products and sums use error-free transforms (the row is rounded
    //      once); the operations are explicitly rounded, out of FMA contraction.
    const float *qp = G.qp + (size_t)l * 3 * np;
    // two vertices per pass of a thread (i and i + blockDim), their sums
    // interleaved entry by entry: six independent chains and two operator
    // loads in flight; each vertex's own sum keeps its order
    for (int i = threadIdx.x; i < n; i += 2 * blockDim.x) {
      const int i2 = i + blockDim.x;
      const bool two = i2 < n;
      const int j2 = two ? i2 : i;
      float x[2][3], sum[2][3], err[2][3];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        x[0][c] = qs[c * ns + i];
        x[1][c] = qs[c * ns + j2];
        sum[0][c] = sum[1][c] = err[0][c] = err[1][c] = 0.f;
      }
      // entries in pairs: one 16-byte load holds two (index, weight) entries
      const int pairs = (G.deg_b + 1) >> 1;
      for (int p = 0; p < pairs; p++) {
        const int4 ra = __ldg(G.kb + (size_t)p * np + i), rb = __ldg(G.kb + (size_t)p * np + j2);
#pragma unroll
        for (int h = 0; h < 2; h++) {
          if (h == 1 && 2 * p + 1 >= G.deg_b) break;   // the filler of an odd count
          const int ka[2] = {chk(h ? ra.z : ra.x, n, G.status), chk(h ? rb.z : rb.x, n, G.status)};
          const float kv[2] = {__int_as_float(h ? ra.w : ra.y), __int_as_float(h ? rb.w : rb.y)};
#pragma unroll
          for (int u = 0; u < 2; u++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
              const float kk = kv[u];
              const float d = __fsub_rn(qs[c * ns + ka[u]], x[u][c]);
              const float pr = __fmul_rn(kk, d), pe = __fmaf_rn(kk, d, -pr);   // kk d = pr + pe exactly
              const float s1 = __fadd_rn(sum[u][c], pr), bp = __fsub_rn(s1, sum[u][c]);
              const float se = __fadd_rn(__fsub_rn(sum[u][c], __fsub_rn(s1, bp)), __fsub_rn(pr, bp));   // sum + pr = s1 + se
              sum[u][c] = s1;
              err[u][c] = __fadd_rn(err[u][c], __fadd_rn(se, pe));
            }
        }
      }
      const float m0 = __ldg(G.mass + i);
#pragma unroll
      for (int c = 0; c < 3; c++) rs[c * ns + i] = m0 * (qp[c * np + i] - x[0][c]) - (sum[0][c] + err[0][c]);
      if (two) {
        const float m1 = __ldg(G.mass + i2);
#pragma unroll
        for (int c = 0; c < 3; c++) rs[c * ns + i2] = m1 * (qp[c * np + i2] - x[1][c]) - (sum[1][c] + err[1][c]);
      }
    }
    __syncthreads();
    // ---- residual r = M (q~ - q) + sum_e D_a^T w~ (p_e - F_e) - bending.
    //      Triangle meshes (about six slots a vertex): a thread's two
    //      vertices gathered in one loop, each in its own slot order (six
    //      independent chains); tet meshes (about twenty, more uneven) one
    //      vertex at a time, which measured faster for them.
    if constexpr (VPE == 3) {
    for (int i = threadIdx.x; i < n; i += 2 * blockDim.x) {
      const int i2 = i + blockDim.x;
      const bool two = i2 < n;
      float acc[2][3];
      int t[2], t1[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int iv = u == 0 ? i : (two ? i2 : i);
        acc[u][0] = rs[iv]; acc[u][1] = rs[ns + iv]; acc[u][2] = rs[2 * ns + iv];
        t[u] = chk(coff[iv], G.ev + 1, G.status);
        t1[u] = u == 1 && !two ? t[u] : chk(coff[iv + 1], G.ev + 1, G.status);
      }
      while (t[0] < t1[0] || t[1] < t1[1]) {
#pragma unroll
        for (int u = 0; u < 2; u++)
          if (t[u] < t1[u]) {
            const float *f = Fs + 3 * chk(cidx[t[u]], G.ev, G.status);
            acc[u][0] += f[0];
            acc[u][1] += f[1];
            acc[u][2] += f[2];
            t[u]++;
          }
      }
      rs[i] = acc[0][0];
      rs[ns + i] = acc[0][1];
      rs[2 * ns + i] = acc[0][2];
      if (two) {
        rs[i2] = acc[1][0];
        rs[ns + i2] = acc[1][1];
        rs[2 * ns + i2] = acc[1][2];
      }
    }
    } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      float acc0 = rs[i], acc1 = rs[ns + i], acc2 = rs[2 * ns + i];
      const int t1 = chk(coff[i + 1], G.ev + 1, G.status);
      for (int t = chk(coff[i], G.ev + 1, G.status); t < t1; t++) {
        const float *f = Fs + 3 * chk(cidx[t], G.ev, G.status);
        acc0 += f[0];
        acc1 += f[1];
        acc2 += f[2];
      }
      rs[i] = acc0;
      rs[ns + i] = acc1;
      rs[2 * ns + i] = acc2;
    }
    }
  }
  __syncthreads();
  // ---- contacts: linearise at (q^{k-1}, gamma^{k-1}), NCP residual of that
  //      iterate, and + J^T gamma^{k-1} (one thread per vertex run)
  const int cnt = G.ccount[l];
  const int *cvert = G.cvert + (size_t)l * G.cap, *cobs = G.cobs + (size_t)l * G.cap;
  const float *gam = G.cgam + (size_t)l * G.cap * 4;
  const float *qt = G.qt + (size_t)l * 3 * np;
  const float mu = V.mu[e];
  float rmax = 0.f;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const int vtx = chk(cvert[j], G.n, G.status);
    if (j > 0 && cvert[j - 1] == vtx) continue;
    const V3 x = v3(qs[vtx], qs[ns + vtx], qs[2 * ns + vtx]);
    const V3 xt = v3(qt[vtx], qt[np + vtx], qt[2 * np + vtx]);
    const float mv = __ldg(G.mass + vtx);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int jj = j; jj < cnt && cvert[jj] == vtx; jj++) {
      ContactLin L;
      const float4 g4 = *reinterpret_cast<const float4 *>(gam + 4 * jj);
      const float g[4] = {g4.x, g4.y, g4.z, g4.w};
      if (SELF && cobs[jj] >= FLASH_SELF_SLOT) continue;   // second pass below
      lin_at(O, chk(cobs[jj], kSlots, G.status), a, mu, mv, x, xt, g, L);
      rmax = fmaxf(rmax, fmaxf(fabsf(L.phi[0]), fmaxf(fabsf(L.phi[1]), fabsf(L.phi[2]))));
      const float y1 = L.R[3] * g[1] + L.R[4] * g[2] + L.R[5] * g[3];
      const float y2 = L.R[6] * g[1] + L.R[7] * g[2] + L.R[8] * g[3];
      fx += L.R[0] * g[0] + L.R[3] * y1 + L.R[6] * y2;
      fy += L.R[1] * g[0] + L.R[4] * y1 + L.R[7] * y2;
      fz += L.R[2] * g[0] + L.R[5] * y1 + L.R[8] * y2;
    }
    if (!residual_only) {
      if (SELF) {   // other threads' self contacts may reach this vertex
        atomicAdd(rs + vtx, fx);
        atomicAdd(rs + ns + vtx, fy);
        atomicAdd(rs + 2 * ns + vtx, fz);
      } else {
        rs[vtx] += fx;
        rs[ns + vtx] += fy;
        rs[2 * ns + vtx] += fz;
      }
    }
  }
  if (SELF) {
    // self contacts (vertex-triangle, edge-edge): w_k F on the row's vertices
    const int *ctri = G.ctri + (size_t)l * G.cap;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      if (cobs[j] < FLASH_SELF_SLOT) continue;
      ContactLin L;
      SelfRow S;
      lin_row(G, O, chk(cobs[j], kSlots, G.status), chk(cvert[j], G.n, G.status), ctri[j], qs, ns, qt, mu, a.h, a.tau, gam + 4 * j, L, S);
      rmax = fmaxf(rmax, fmaxf(fabsf(L.phi[0]), fmaxf(fabsf(L.phi[1]), fabsf(L.phi[2]))));
      if (!residual_only) scatter_row(S.v, S.w, contact_force(L, gam + 4 * j), rs, ns);
    }
  }
  rmax = block_max(rmax, sh_red);
  if (threadIdx.x == 0) {
    const int it = k - 1;
    int stop;
    if (a.mode == FLASH_MODE_FIXED) stop = residual_only;
    else stop = (it >= a.k_min && rmax <= a.tol) || it >= a.k_cap || residual_only;
    if (!isfinite(rmax)) { atomicOr(V.status, 1 << 9); stop = 1; }
    if (stop) {
      V.done[e] = 1;
      V.iters[e] = it;
      V.rncp[e] = rmax;
    } else if (a.mode == FLASH_MODE_TOL) {
      atomicAdd(V.active, 1);
    }
    s_done = stop;
  }
  __syncthreads();
  if (s_done) return;
  if (tc) {
    write_split_columns(G, l, rs, ns, sh3, true, 0.f, 0.f, 0.f, G.r);
  } else {
    float *r = G.r + (size_t)l * 3 * np;
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
      int c = i / n, j = i - c * n;
      r[c * np + j] = rs[c * ns + j];
    }
  }
}

// Iterative refinement of the bf16 solve (tet meshes): the residual
// rhs - A w of the current solution w in FP32, with A w = M w + sum_e
// w~_e k_e D_e^T (D_e w) from the element operators (the local pass's
// operators without the projection), summed per vertex through the same CSR
// table; the result becomes the next bf16 apply's right-hand side.
__device__ __forceinline__ void refine_body(const GroupView &G, const int l, const EnvView &V, const float *rhs32,
                                            const float *wv) {
  constexpr int vpe = 4, nc = 3;
  extern __shared__ float smem[];
  __shared__ float sh3[32][3];
  const int e = G.genv[l];
  const int n = G.n, np = G.n_pad, ns = (n + 3) & ~3;
  if (V.done[e]) return;
  float *ws = smem, *rs = ws + 3 * ns, *Fs;
  const uint16_t *coff, *cidx;
  if (G.c_in_smem) {
    Fs = rs + 3 * ns;
    uint32_t *t = reinterpret_cast<uint32_t *>(Fs + 3 * (G.ev + 1));
    const int w_off = (n + 2) >> 1, w_idx = (G.ev + 1) >> 1;
    const uint32_t *src_off = reinterpret_cast<const uint32_t *>(G.coff);
    const uint32_t *src_idx = reinterpret_cast<const uint32_t *>(G.cidx);
    for (int i = threadIdx.x; i < w_off; i += blockDim.x) t[i] = __ldg(src_off + i);
    for (int i = threadIdx.x; i < w_idx; i += blockDim.x) t[w_off + i] = __ldg(src_idx + i);
    coff = reinterpret_cast<const uint16_t *>(t);
    cidx = coff + 2 * w_off;
  } else {
    Fs = G.cscratch + (size_t)l * 3 * (G.ev + 1);
    coff = G.coff;
    cidx = G.cidx;
  }
  const float *w = wv + (size_t)l * 3 * np, *b = rhs32 + (size_t)l * 3 * np;
  for (int i = threadIdx.x; i < 3 * ns; i += blockDim.x) {
    const int c = i / ns, j = i - c * ns;
    const float x = j < n ? w[c * np + j] : 0.f;
    ws[i] = x;
    rs[i] = j < n ? b[c * np + j] - __ldg(G.mass + j) * x : 0.f;
  }
  __syncthreads();
  const float ks = G.kenv ? G.kenv[l] : 1.f;
  for (int el = threadIdx.x; el < G.E; el += blockDim.x) {
    const int4 vi = *reinterpret_cast<const int4 *>(G.elems + 4 * el);
    const int vv[4] = {chk(vi.x, n, G.status), chk(vi.y, n, G.status), chk(vi.z, n, G.status),
                          chk(vi.w, n, G.status)};
    const float4 *D4 = reinterpret_cast<const float4 *>(G.D + 12 * el);
    float F[9], Dl[12];
#pragma unroll
    for (int t = 0; t < 3; t++) {
      const float4 d = __ldg(D4 + t);
      Dl[4 * t] = d.x; Dl[4 * t + 1] = d.y; Dl[4 * t + 2] = d.z; Dl[4 * t + 3] = d.w;
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const float x0 = ws[c * ns + vv[0]];
#pragma unroll
      for (int j = 0; j < nc; j++) {
        float sm = 0.f;
#pragma unroll
        for (int aa = 1; aa < vpe; aa++) sm += (ws[c * ns + vv[aa]] - x0) * Dl[aa * 3 + j];
        F[nc * c + j] = sm;
      }
    }
    const float wt = __ldg(G.wt + el) * ks;
    float *Fe = Fs + (size_t)el * vpe * 3;
#pragma unroll
    for (int aa = 0; aa < vpe; aa++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        float sm = 0.f;
#pragma unroll
        for (int j = 0; j < nc; j++) sm += Dl[aa * 3 + j] * F[nc * c + j];
        Fe[aa * 3 + c] = wt * sm;
      }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float a0 = rs[i], a1 = rs[ns + i], a2 = rs[2 * ns + i];
    const int t1 = chk(coff[i + 1], G.ev + 1, G.status);
    for (int t = chk(coff[i], G.ev + 1, G.status); t < t1; t++) {
      const float *f = Fs + 3 * chk(cidx[t], G.ev, G.status);
      a0 -= f[0];
      a1 -= f[1];
      a2 -= f[2];
    }
    rs[i] = a0;
    rs[ns + i] = a1;
    rs[2 * ns + i] = a2;
  }
  __syncthreads();
  write_split_columns(G, l, rs, ns, sh3, true);
}

// ---------------------------------------------------------------------------
// NCP update on the lite metric: per-vertex blocks
// ---------------------------------------------------------------------------
__device__ void solve_dense(int N, float *A, float *b) {
  for (int c = 0; c < N; c++) {
    int piv = c;
    for (int r = c + 1; r < N; r++)
      if (fabsf(A[r * N + c]) > fabsf(A[piv * N + c])) piv = r;
    if (piv != c) {
      for (int j = 0; j < N; j++) { float t = A[c * N + j]; A[c * N + j] = A[piv * N + j]; A[piv * N + j] = t; }
      float t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    float d = A[c * N + c];
    if (fabsf(d) < 1e-30f) d = copysignf(1e-30f, d);
    for (int r = c + 1; r < N; r++) {
      float fct = A[r * N + c] / d;
      for (int j = c; j < N; j++) A[r * N + j] -= fct * A[c * N + j];
      b[r] -= fct * b[c];
    }
  }
  for (int c = N - 1; c >= 0; c--) {
    float s = b[c];
    for (int j = c + 1; j < N; j++) s -= A[c * N + j] * b[j];
    float d = A[c * N + c];
    if (fabsf(d) < 1e-30f) d = copysignf(1e-30f, d);
    b[c] = s / d;
  }
}

// A contact that is separated (gap > 0) and carries no force has D_C = 0 and
// D_y = I, so its Newton row gives dy = 0 and it does not couple to the other
// contacts of the vertex: it can be left out of the block exactly.
__device__ __forceinline__ bool separated_free(const ContactLin &L, const float *g) {
  return L.gap > 0.f && g[0] == 0.f && g[1] == 0.f && g[2] == 0.f && g[3] == 0.f;
}

// D_C (3x3) and D_y (3x3) of one contact
__device__ __forceinline__ void lin_mats(const ContactLin &L, float DC[9], float Dy[9]) {
  DC[0] = L.cn; DC[1] = 0.f; DC[2] = 0.f;
  DC[3] = 0.f; DC[4] = L.Ct[0]; DC[5] = L.Ct[1];
  DC[6] = 0.f; DC[7] = L.Ct[2]; DC[8] = L.Ct[3];
  Dy[0] = L.dn; Dy[1] = 0.f; Dy[2] = 0.f;
  Dy[3] = L.dtn[0]; Dy[4] = L.Dtt[0]; Dy[5] = L.Dtt[1];
  Dy[6] = L.dtn[1]; Dy[7] = L.Dtt[2]; Dy[8] = L.Dtt[3];
}

// gamma^k = gamma^{k-1} + m dy (normal clamped at h^2 maxforce); returns J^T dgamma
__device__ __forceinline__ V3 apply_update(const ContactLin &L, float mv, float gmax, const float *dy, float *g) {
  float dgn = mv * dy[0], dg1 = mv * dy[1], dg2 = mv * dy[2];
  const float gn_old = g[0];
  const float gn = fminf(gn_old + dgn, gmax);
  dgn = gn - gn_old;
  const float y1 = L.R[3] * g[1] + L.R[4] * g[2] + L.R[5] * g[3] + dg1;
  const float y2 = L.R[6] * g[1] + L.R[7] * g[2] + L.R[8] * g[3] + dg2;
  g[0] = gn;
  g[1] = L.R[3] * y1 + L.R[6] * y2;
  g[2] = L.R[4] * y1 + L.R[7] * y2;
  g[3] = L.R[5] * y1 + L.R[8] * y2;
  return v3(L.R[0] * dgn + L.R[3] * dg1 + L.R[6] * dg2, L.R[1] * dgn + L.R[4] * dg1 + L.R[7] * dg2,
            L.R[2] * dgn + L.R[5] * dg1 + L.R[8] * dg2);
}

// Two contacts on one vertex (e.g. a cloth point squeezed between a finger and
// the ground): 6x6 lite block solved by block elimination in registers,
//   S = Z22 - Z21 Z11^-1 Z12,  x2 = S^-1 (b2 - Z21 Z11^-1 b1),  x1 = Z11^-1 (b1 - Z12 x2)
// where Z11, Z22 are the single-contact blocks (normal row, then 2x2 tangential).
__device__ __forceinline__ void solve_single_block(const ContactLin &L, const float b[3], float x[3]) {
  x[0] = b[0] / (L.cn + L.dn + kDamp);
  const float b1 = b[1] - L.dtn[0] * x[0], b2 = b[2] - L.dtn[1] * x[0];
  const float m00 = L.Ct[0] + L.Dtt[0] + kDamp, m01 = L.Ct[1] + L.Dtt[1];
  const float m10 = L.Ct[2] + L.Dtt[2], m11 = L.Ct[3] + L.Dtt[3] + kDamp;
  const float inv = 1.f / (m00 * m11 - m01 * m10);
  x[1] = (m11 * b1 - m01 * b2) * inv;
  x[2] = (m00 * b2 - m10 * b1) * inv;
}

__device__ __forceinline__ void dc_times(const ContactLin &L, const float v[3], float out[3]) {
  out[0] = L.cn * v[0];
  out[1] = L.Ct[0] * v[1] + L.Ct[1] * v[2];
  out[2] = L.Ct[2] * v[1] + L.Ct[3] * v[2];
}

__device__ __noinline__ V3 solve_two(const ContactLin &L1, const ContactLin &L2, const StepArgs &a, float mv, V3 du,
                                     float *g1, float *g2) {
  float RR12[9];   // R1 R2^T
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++)
      RR12[3 * r + c] = L1.R[3 * r] * L2.R[3 * c] + L1.R[3 * r + 1] * L2.R[3 * c + 1] + L1.R[3 * r + 2] * L2.R[3 * c + 2];
  float b1[3], b2[3], t[3];
  {
    const float r1[3] = {L1.R[0] * du.x + L1.R[1] * du.y + L1.R[2] * du.z, L1.R[3] * du.x + L1.R[4] * du.y + L1.R[5] * du.z,
                         L1.R[6] * du.x + L1.R[7] * du.y + L1.R[8] * du.z};
    const float r2[3] = {L2.R[0] * du.x + L2.R[1] * du.y + L2.R[2] * du.z, L2.R[3] * du.x + L2.R[4] * du.y + L2.R[5] * du.z,
                         L2.R[6] * du.x + L2.R[7] * du.y + L2.R[8] * du.z};
    dc_times(L1, r1, t);
    for (int i = 0; i < 3; i++) b1[i] = -L1.phi[i] - t[i];
    dc_times(L2, r2, t);
    for (int i = 0; i < 3; i++) b2[i] = -L2.phi[i] - t[i];
  }
  // Z12 = D_C1 R1 R2^T, Z21 = D_C2 R2 R1^T; X = Z11^-1 Z12 (column by column)
  float X[9], S[9];
  for (int c = 0; c < 3; c++) {
    const float col[3] = {RR12[c], RR12[3 + c], RR12[6 + c]};
    float z[3], xx[3];
    dc_times(L1, col, z);
    solve_single_block(L1, z, xx);
    X[c] = xx[0]; X[3 + c] = xx[1]; X[6 + c] = xx[2];
  }
  // S = Z22 - Z21 X, with Z22 = D_C2 + D_y2 + damp I
  for (int c = 0; c < 3; c++) {
    // (R2 R1^T) X[:, c]
    float v[3];
    for (int r = 0; r < 3; r++) v[r] = RR12[r] * X[c] + RR12[3 + r] * X[3 + c] + RR12[6 + r] * X[6 + c];
    float z[3];
    dc_times(L2, v, z);
    for (int r = 0; r < 3; r++) S[3 * r + c] = -z[r];
  }
  S[0] += L2.cn + L2.dn + kDamp;
  S[3] += L2.dtn[0]; S[4] += L2.Ct[0] + L2.Dtt[0] + kDamp; S[5] += L2.Ct[1] + L2.Dtt[1];
  S[6] += L2.dtn[1]; S[7] += L2.Ct[2] + L2.Dtt[2]; S[8] += L2.Ct[3] + L2.Dtt[3] + kDamp;
  // rhs2 = b2 - Z21 Z11^-1 b1
  float y1[3];
  solve_single_block(L1, b1, y1);
  {
    float v[3], z[3];
    for (int r = 0; r < 3; r++) v[r] = RR12[r] * y1[0] + RR12[3 + r] * y1[1] + RR12[6 + r] * y1[2];
    dc_times(L2, v, z);
    for (int r = 0; r < 3; r++) b2[r] -= z[r];
  }
  // x2 = S^-1 rhs2 (adjugate)
  const float c00 = S[4] * S[8] - S[5] * S[7], c01 = S[5] * S[6] - S[3] * S[8], c02 = S[3] * S[7] - S[4] * S[6];
  const float det = S[0] * c00 + S[1] * c01 + S[2] * c02;
  const float id = 1.f / det;
  float x2[3];
  x2[0] = (c00 * b2[0] + (S[2] * S[7] - S[1] * S[8]) * b2[1] + (S[1] * S[5] - S[2] * S[4]) * b2[2]) * id;
  x2[1] = (c01 * b2[0] + (S[0] * S[8] - S[2] * S[6]) * b2[1] + (S[2] * S[3] - S[0] * S[5]) * b2[2]) * id;
  x2[2] = (c02 * b2[0] + (S[1] * S[6] - S[0] * S[7]) * b2[1] + (S[0] * S[4] - S[1] * S[3]) * b2[2]) * id;
  // x1 = Z11^-1 (b1 - Z12 x2)
  {
    float v[3], z[3];
    for (int r = 0; r < 3; r++) v[r] = RR12[3 * r] * x2[0] + RR12[3 * r + 1] * x2[1] + RR12[3 * r + 2] * x2[2];
    dc_times(L1, v, z);
    for (int r = 0; r < 3; r++) b1[r] -= z[r];
  }
  float x1[3];
  solve_single_block(L1, b1, x1);
  return apply_update(L1, mv, a.gmax, x1, g1) + apply_update(L2, mv, a.gmax, x2, g2);
}

// several contacts on one vertex: dense (3c x 3c) block of the lite metric,
// kept out of line so the common single-contact path stays in registers
__device__ __noinline__ V3 solve_multi(const ContactLin *Ls, const StepArgs &a, float mv, V3 du, int c, float *gam,
                                       const int *idx) {
  const int N3 = 3 * c;
  float Z[12 * 12], rhs[12];
  for (int aa = 0; aa < c; aa++) {
    float DC[9], Dy[9];
    lin_mats(Ls[aa], DC, Dy);
    const float *Ra = Ls[aa].R;
    float Rdu[3] = {Ra[0] * du.x + Ra[1] * du.y + Ra[2] * du.z, Ra[3] * du.x + Ra[4] * du.y + Ra[5] * du.z,
                    Ra[6] * du.x + Ra[7] * du.y + Ra[8] * du.z};
    for (int r = 0; r < 3; r++)
      rhs[3 * aa + r] = -Ls[aa].phi[r] - (DC[3 * r] * Rdu[0] + DC[3 * r + 1] * Rdu[1] + DC[3 * r + 2] * Rdu[2]);
    for (int bb = 0; bb < c; bb++) {
      const float *Rb = Ls[bb].R;
      float RR[9];
      for (int r = 0; r < 3; r++)
        for (int cc = 0; cc < 3; cc++)
          RR[3 * r + cc] = Ra[3 * r] * Rb[3 * cc] + Ra[3 * r + 1] * Rb[3 * cc + 1] + Ra[3 * r + 2] * Rb[3 * cc + 2];
      for (int r = 0; r < 3; r++)
        for (int cc = 0; cc < 3; cc++) {
          float sum = DC[3 * r] * RR[cc] + DC[3 * r + 1] * RR[3 + cc] + DC[3 * r + 2] * RR[6 + cc];
          if (aa == bb) sum += Dy[3 * r + cc] + (r == cc ? kDamp : 0.f);
          Z[(3 * aa + r) * N3 + 3 * bb + cc] = sum;
        }
    }
  }
  solve_dense(N3, Z, rhs);
  V3 fsum = v3(0.f, 0.f, 0.f);
  for (int aa = 0; aa < c; aa++) fsum = fsum + apply_update(Ls[aa], mv, a.gmax, rhs + 3 * aa, gam + 4 * idx[aa]);
  return fsum;
}

__device__ __forceinline__ void ncp_body(const GroupView &G, const int l, const EnvView &V, StepArgs a, int tc) {
  extern __shared__ float fs[];   // [3][n] contact force (tc path)
  __shared__ float sh3[32][3];
  __shared__ ObsShared O;
  a.tau = G.tau;
  const int e = G.genv[l];
  const int n = G.n, np = G.n_pad;
  if (V.done[e]) return;
  const int cnt = G.ccount[l];
  const int *cvert = G.cvert + (size_t)l * G.cap, *cobs = G.cobs + (size_t)l * G.cap;
  float *gam = G.cgam + (size_t)l * G.cap * 4;
  const float *q = G.q + (size_t)l * 3 * np, *w = G.w + (size_t)l * 3 * np, *qt = G.qt + (size_t)l * 3 * np;
  float *f = G.f + (size_t)l * 3 * np;
  const float mu = V.mu[e];
  load_obstacles(V, e, a.K, O);
  if (tc)
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) fs[i] = 0.f;
  __syncthreads();
  float fm0 = 0.f, fm1 = 0.f, fm2 = 0.f;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const int vtx = chk(cvert[j], G.n, G.status);
    if (j > 0 && cvert[j - 1] == vtx) continue;
    int c = 1;
    while (j + c < cnt && cvert[j + c] == vtx) c++;
    if (c > kMaxPerVertex) {
      atomicOr(V.status, 1 << 10);
      c = kMaxPerVertex;
    }
    const float mv = __ldg(G.mass + vtx);
    const V3 x = v3(q[vtx], q[np + vtx], q[2 * np + vtx]);
    const V3 xt = v3(qt[vtx], qt[np + vtx], qt[2 * np + vtx]);
    const V3 du = v3(w[vtx], w[np + vtx], w[2 * np + vtx]);   // u - q^{k-1} = A^-1 r
    V3 fsum = v3(0.f, 0.f, 0.f);
    if (c == 1) {
      // single contact: R R^T = I, Z = D_C + D_y + damp I is block lower
      // triangular (normal row first, then the 2x2 tangential block)
      ContactLin L;
      float *g = gam + 4 * j;
      lin_at(O, chk(cobs[j], kSlots, G.status), a, mu, mv, x, xt, g, L);
      if (!separated_free(L, g)) {
        const float Rdu0 = L.R[0] * du.x + L.R[1] * du.y + L.R[2] * du.z;
        const float Rdu1 = L.R[3] * du.x + L.R[4] * du.y + L.R[5] * du.z;
        const float Rdu2 = L.R[6] * du.x + L.R[7] * du.y + L.R[8] * du.z;
        float dy[3];
        dy[0] = (-L.phi[0] - L.cn * Rdu0) / (L.cn + L.dn + kDamp);
        const float b1 = -L.phi[1] - (L.Ct[0] * Rdu1 + L.Ct[1] * Rdu2) - L.dtn[0] * dy[0];
        const float b2 = -L.phi[2] - (L.Ct[2] * Rdu1 + L.Ct[3] * Rdu2) - L.dtn[1] * dy[0];
        const float m00 = L.Ct[0] + L.Dtt[0] + kDamp, m01 = L.Ct[1] + L.Dtt[1];
        const float m10 = L.Ct[2] + L.Dtt[2], m11 = L.Ct[3] + L.Dtt[3] + kDamp;
        const float inv = 1.f / (m00 * m11 - m01 * m10);
        dy[1] = (m11 * b1 - m01 * b2) * inv;
        dy[2] = (m00 * b2 - m10 * b1) * inv;
        fsum = apply_update(L, mv, a.gmax, dy, g);
      }
    } else {
      // several contacts: linearise all, keep those that are not separated
      // and force-free (those have dy = 0 exactly and do not couple)
      ContactLin Ls[kMaxPerVertex];
      int idx[kMaxPerVertex];
      int na = 0;
      for (int aa = 0; aa < c; aa++) {
        lin_at(O, chk(cobs[j + aa], kSlots, G.status), a, mu, mv, x, xt, gam + 4 * (j + aa), Ls[na]);
        if (!separated_free(Ls[na], gam + 4 * (j + aa))) idx[na++] = j + aa;
      }
      if (na == 1) {
        const ContactLin &L = Ls[0];
        float *g = gam + 4 * idx[0];
        const float Rdu0 = L.R[0] * du.x + L.R[1] * du.y + L.R[2] * du.z;
        const float Rdu1 = L.R[3] * du.x + L.R[4] * du.y + L.R[5] * du.z;
        const float Rdu2 = L.R[6] * du.x + L.R[7] * du.y + L.R[8] * du.z;
        float b[3] = {-L.phi[0] - L.cn * Rdu0, -L.phi[1] - (L.Ct[0] * Rdu1 + L.Ct[1] * Rdu2),
                      -L.phi[2] - (L.Ct[2] * Rdu1 + L.Ct[3] * Rdu2)};
        float dy[3];
        solve_single_block(L, b, dy);
        fsum = apply_update(L, mv, a.gmax, dy, g);
      } else if (na == 2) {
        fsum = solve_two(Ls[0], Ls[1], a, mv, du, gam + 4 * idx[0], gam + 4 * idx[1]);
      } else if (na > 2) {
        fsum = solve_multi(Ls, a, mv, du, na, gam, idx);
      }
    }
    fm0 = fmaxf(fm0, fabsf(fsum.x)); fm1 = fmaxf(fm1, fabsf(fsum.y)); fm2 = fmaxf(fm2, fabsf(fsum.z));
    if (tc) {
      fs[vtx] = fsum.x; fs[n + vtx] = fsum.y; fs[2 * n + vtx] = fsum.z;
    } else {
      f[vtx] = fsum.x; f[np + vtx] = fsum.y; f[2 * np + vtx] = fsum.z;
    }
  }
  if (tc) {
    __syncthreads();
    // every nonzero row of fs was written by this block with its max tracked
    write_split_columns(G, l, fs, n, sh3, false, fm0, fm1, fm2, G.f);
  }
}

// ---------------------------------------------------------------------------
// Full contact metric (Sec. III-C, Eq. schur): Z = J A^-1 J^T + E instead of
// the lite J M^-1 J^T + E.  Per environment and local-global iteration the
// Newton system Z dy = rhs over all its contacts is solved by m steps of
// GMRES (the paper's "linear-solver iterations") from dy = 0,
// right-preconditioned by the inverses of Z's 3x3 diagonal blocks
// D_C a_vv m_v + D_y (+ damping), Arnoldi with classical Gram-Schmidt and
// one reorthogonalisation, Givens rotations for the least-squares problem;
// the basis stops early once a new Arnoldi vector's norm is below 1e-6 |rhs|.
// Z is applied matrix-free: forces m_v R^T x on the contact vertices
// (fm_scatter), one A^-1 contraction over all environments (the group's
// global solve), then D_C R u + (D_y + damping) x at each contact
// (fm_gather).  fm_finish forms dy, updates the multipliers and writes
// J^T dgamma like the lite NCP kernel.
// ---------------------------------------------------------------------------
constexpr int kFmLin = 22;   // floats per contact: R[9], cn, Ct[4], dn, dtn[2], Dtt[4], s
constexpr int kFmMax = 32;   // most linear-solver iterations

__device__ __forceinline__ void fm_store(float *d, const ContactLin &L, float sc) {
#pragma unroll
  for (int t = 0; t < 9; t++) d[t] = L.R[t];
  d[9] = L.cn;
#pragma unroll
  for (int t = 0; t < 4; t++) d[10 + t] = L.Ct[t];
  d[14] = L.dn; d[15] = L.dtn[0]; d[16] = L.dtn[1];
#pragma unroll
  for (int t = 0; t < 4; t++) d[17 + t] = L.Dtt[t];
  d[21] = sc;
}

__device__ __forceinline__ float fm_load(const float *d, ContactLin &L) {
#pragma unroll
  for (int t = 0; t < 9; t++) L.R[t] = d[t];
  L.cn = d[9];
#pragma unroll
  for (int t = 0; t < 4; t++) L.Ct[t] = d[10 + t];
  L.dn = d[14]; L.dtn[0] = d[15]; L.dtn[1] = d[16];
#pragma unroll
  for (int t = 0; t < 4; t++) L.Dtt[t] = d[17 + t];
  return d[21];
}

// x = P^-1 v with P = D_C s + D_y + damping (s = a_vv m_v): the lite block
// with the D_C rows scaled by s
__device__ __forceinline__ void fm_pinv(const ContactLin &L, float sc, const float v[3], float x[3]) {
  ContactLin Ls = L;
  Ls.cn *= sc;
#pragma unroll
  for (int t = 0; t < 4; t++) Ls.Ct[t] *= sc;
  solve_single_block(Ls, v, x);
}

__device__ float block_sum(float v, float *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < nw; w++) t += sh[w];
  __syncthreads();
  return t;
}

// block-wide sums of cnt (<= kFmMax + 1) values per thread, in place
__device__ void block_sum_n(float *v, int cnt, float (*sh)[kFmMax + 1]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int i = 0; i < cnt; i++) {
    float x = v[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[wid][i] = x;
  }
  __syncthreads();
  for (int i = 0; i < cnt; i++) {
    float t = 0.f;
    for (int w = 0; w < nw; w++) t += sh[w][i];
    v[i] = t;
  }
  __syncthreads();
}

// right side, stored linearisation and first Arnoldi vector
__device__ __forceinline__ void fm_setup_body(const GroupView &G, const int l, const EnvView &V, StepArgs a) {
  __shared__ ObsShared O;
  __shared__ float sh[32];
  a.tau = G.tau;
  const int e = G.genv[l];
  if (V.done[e]) return;
  const int np = G.n_pad, cap = G.cap, m = G.fm_m;
  const size_t N3 = 3 * (size_t)cap;
  const int cnt = G.ccount[l];
  const int *cvert = G.cvert + (size_t)l * cap, *cobs = G.cobs + (size_t)l * cap;
  const float *gam = G.cgam + (size_t)l * cap * 4;
  const float *q = G.q + (size_t)l * 3 * np, *w = G.w + (size_t)l * 3 * np, *qt = G.qt + (size_t)l * 3 * np;
  const float *ad = G.fm_adiag + (size_t)l * G.fm_adiag_stride;
  float *lin = G.fm_lin + (size_t)l * cap * kFmLin;
  float *V0 = G.fm_V + (size_t)l * (m + 1) * N3;
  const float mu = V.mu[e];
  load_obstacles(V, e, a.K, O);
  __syncthreads();
  float ss = 0.f;
  for (int c = threadIdx.x; c < cnt; c += blockDim.x) {
    const int vtx = chk(cvert[c], G.n, G.status);
    const float mv = __ldg(G.mass + vtx);
    const V3 x = v3(q[vtx], q[np + vtx], q[2 * np + vtx]);
    const V3 xt = v3(qt[vtx], qt[np + vtx], qt[2 * np + vtx]);
    const V3 du = v3(w[vtx], w[np + vtx], w[2 * np + vtx]);   // u - q^{k-1} = A^-1 r
    ContactLin L;
    V3 du_c = du;
    float sc;
    if (G.self && cobs[c] >= FLASH_SELF_SLOT) {
      // J du = sum w_k du_k; preconditioner scale (sum w_k^2 a_kk) meff
      SelfRow S;
      lin_row(G, O, chk(cobs[c], kSlots, G.status), vtx, G.ctri[(size_t)l * cap + c], q, np, qt, mu, a.h, a.tau, gam + 4 * c, L, S);
      float av = 0.f;
      du_c = v3(0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        du_c = du_c + S.w[k] * col3(w, np, S.v[k]);
        av += S.w[k] * S.w[k] * ad[S.v[k]];
      }
      sc = av * S.meff;
      fm_row_store(G.fm_w + ((size_t)l * cap + c) * kFmW, S);
    } else {
      lin_at(O, chk(cobs[c], kSlots, G.status), a, mu, mv, x, xt, gam + 4 * c, L);
      sc = ad[vtx] * mv;
    }
    const float Rdu0 = L.R[0] * du_c.x + L.R[1] * du_c.y + L.R[2] * du_c.z;
    const float Rdu1 = L.R[3] * du_c.x + L.R[4] * du_c.y + L.R[5] * du_c.z;
    const float Rdu2 = L.R[6] * du_c.x + L.R[7] * du_c.y + L.R[8] * du_c.z;
    const float b0 = -L.phi[0] - L.cn * Rdu0;
    const float b1 = -L.phi[1] - (L.Ct[0] * Rdu1 + L.Ct[1] * Rdu2);
    const float b2 = -L.phi[2] - (L.Ct[2] * Rdu1 + L.Ct[3] * Rdu2);
    fm_store(lin + (size_t)c * kFmLin, L, sc);
    V0[3 * c] = b0; V0[3 * c + 1] = b1; V0[3 * c + 2] = b2;
    ss += b0 * b0 + b1 * b1 + b2 * b2;
  }
  const float beta = sqrtf(block_sum(ss, sh));
  if (threadIdx.x == 0) {
    G.fm_beta[l] = beta;
    G.fm_g[(size_t)l * (m + 1)] = beta;
    G.fm_jm[l] = beta > 0.f ? 0 : -1;    // -1: stopped with no column
  }
  if (beta > 0.f)
    for (int c = threadIdx.x; c < cnt; c += blockDim.x)
      for (int r = 0; r < 3; r++) V0[3 * c + r] = V0[3 * c + r] / beta;
}

// forces m_v R^T P^-1 v_j on the contact vertices, written as the group's
// right-hand columns (f16 split on the tensor-core path)
__device__ __forceinline__ void fm_scatter_body(const GroupView &G, const int l, const EnvView &V, int j, int tc) {
  extern __shared__ float fs[];   // [3][n]
  __shared__ float sh3[32][3];
  const int e = G.genv[l];
  if (V.done[e] || G.fm_jm[l] < 0) return;
  const int n = G.n, np = G.n_pad, cap = G.cap, m = G.fm_m;
  const size_t N3 = 3 * (size_t)cap;
  const int cnt = G.ccount[l];
  const int *cvert = G.cvert + (size_t)l * cap;
  const float *lin = G.fm_lin + (size_t)l * cap * kFmLin;
  const float *Vj = G.fm_V + ((size_t)l * (m + 1) + j) * N3;
  for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) fs[i] = 0.f;
  __syncthreads();
  float fm0 = 0.f, fm1 = 0.f, fm2 = 0.f;
  for (int c = threadIdx.x; c < cnt; c += blockDim.x) {
    const int vtx = chk(cvert[c], G.n, G.status);
    if (c > 0 && cvert[c - 1] == vtx) continue;
    const float mv = __ldg(G.mass + vtx);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int cc = c; cc < cnt && cvert[cc] == vtx; cc++) {
      ContactLin L;
      const float sc = fm_load(lin + (size_t)cc * kFmLin, L);
      const float v[3] = {Vj[3 * cc], Vj[3 * cc + 1], Vj[3 * cc + 2]};
      float t[3];
      fm_pinv(L, sc, v, t);
      const bool selfrow = G.self && G.cobs[(size_t)l * cap + cc] >= FLASH_SELF_SLOT;
      SelfRow S;
      if (selfrow) fm_row_load(G.fm_w + ((size_t)l * cap + cc) * kFmW, vtx, S, G.n, G.status);
      const float me = selfrow ? S.meff : mv;
      const V3 F = v3(me * (L.R[0] * t[0] + L.R[3] * t[1] + L.R[6] * t[2]),
                      me * (L.R[1] * t[0] + L.R[4] * t[1] + L.R[7] * t[2]),
                      me * (L.R[2] * t[0] + L.R[5] * t[1] + L.R[8] * t[2]));
      if (selfrow) {
        scatter_row(S.v, S.w, F, fs, n);
      } else {
        fx += F.x; fy += F.y; fz += F.z;
      }
    }
    if (G.self) {
      atomicAdd(fs + vtx, fx); atomicAdd(fs + n + vtx, fy); atomicAdd(fs + 2 * n + vtx, fz);
    } else {
      fs[vtx] = fx; fs[n + vtx] = fy; fs[2 * n + vtx] = fz;
    }
    fm0 = fmaxf(fm0, fabsf(fx)); fm1 = fmaxf(fm1, fabsf(fy)); fm2 = fmaxf(fm2, fabsf(fz));
  }
  __syncthreads();
  if (tc) {
    // with self contacts the column maxima are known only after the sums
    write_split_columns(G, l, fs, n, sh3, G.self != 0, fm0, fm1, fm2, G.f);
  } else {
    float *f = G.f + (size_t)l * 3 * np;
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
      const int c = i / n, jj = i - c * n;
      f[c * np + jj] = fs[i];
    }
  }
}

// w = Z P^-1 v_j from u = A^-1 f, orthogonalised against v_0..v_j (two
// classical Gram-Schmidt passes), rotated column j of H, next basis vector
__device__ __forceinline__ void fm_gather_body(const GroupView &G, const int l, const EnvView &V, int j) {
  __shared__ float shn[32][kFmMax + 1];
  __shared__ float sh[32];
  __shared__ float s_hn;
  __shared__ int s_stop;
  const int e = G.genv[l];
  if (V.done[e] || G.fm_jm[l] < 0) return;
  const int np = G.n_pad, cap = G.cap, m = G.fm_m;
  const size_t N3 = 3 * (size_t)cap;
  const int cnt = G.ccount[l];
  const int *cvert = G.cvert + (size_t)l * cap;
  const float *lin = G.fm_lin + (size_t)l * cap * kFmLin;
  const float *u = G.fm_u + (size_t)l * 3 * np;
  float *Vb = G.fm_V + (size_t)l * (m + 1) * N3;
  const float *Vj = Vb + (size_t)j * N3;
  float *Vn = Vb + (size_t)(j + 1) * N3;   // w, then v_{j+1}
  float d[kFmMax + 1];
  for (int i = 0; i <= j; i++) d[i] = 0.f;
  for (int c = threadIdx.x; c < cnt; c += blockDim.x) {
    ContactLin L;
    const float sc = fm_load(lin + (size_t)c * kFmLin, L);
    const float v[3] = {Vj[3 * c], Vj[3 * c + 1], Vj[3 * c + 2]};
    float t[3];
    fm_pinv(L, sc, v, t);
    const int vtx = chk(cvert[c], G.n, G.status);
    float ux = u[vtx], uy = u[np + vtx], uz = u[2 * np + vtx];
    if (G.self && G.cobs[(size_t)l * cap + c] >= FLASH_SELF_SLOT) {   // J u = sum w_k u_k
      SelfRow S;
      fm_row_load(G.fm_w + ((size_t)l * cap + c) * kFmW, vtx, S, G.n, G.status);
      ux = 0.f; uy = 0.f; uz = 0.f;
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const int t = S.v[k];
        ux += S.w[k] * u[t]; uy += S.w[k] * u[np + t]; uz += S.w[k] * u[2 * np + t];
      }
    }
    const float Ru0 = L.R[0] * ux + L.R[1] * uy + L.R[2] * uz;
    const float Ru1 = L.R[3] * ux + L.R[4] * uy + L.R[5] * uz;
    const float Ru2 = L.R[6] * ux + L.R[7] * uy + L.R[8] * uz;
    const float z0 = L.cn * Ru0 + (L.dn + kDamp) * t[0];
    const float z1 = L.Ct[0] * Ru1 + L.Ct[1] * Ru2 + L.dtn[0] * t[0] + (L.Dtt[0] + kDamp) * t[1] + L.Dtt[1] * t[2];
    const float z2 = L.Ct[2] * Ru1 + L.Ct[3] * Ru2 + L.dtn[1] * t[0] + L.Dtt[2] * t[1] + (L.Dtt[3] + kDamp) * t[2];
    Vn[3 * c] = z0; Vn[3 * c + 1] = z1; Vn[3 * c + 2] = z2;
    for (int i = 0; i <= j; i++) {
      const float *vi = Vb + (size_t)i * N3 + 3 * c;
      d[i] += z0 * vi[0] + z1 * vi[1] + z2 * vi[2];
    }
  }
  block_sum_n(d, j + 1, shn);
  float d2[kFmMax + 1];
  for (int i = 0; i <= j; i++) d2[i] = 0.f;
  for (int c = threadIdx.x; c < cnt; c += blockDim.x)
    for (int r = 0; r < 3; r++) {
      float z = Vn[3 * c + r];
      for (int i = 0; i <= j; i++) z -= d[i] * Vb[(size_t)i * N3 + 3 * c + r];
      Vn[3 * c + r] = z;
      for (int i = 0; i <= j; i++) d2[i] += z * Vb[(size_t)i * N3 + 3 * c + r];
    }
  block_sum_n(d2, j + 1, shn);
  float hs = 0.f;
  for (int c = threadIdx.x; c < cnt; c += blockDim.x)
    for (int r = 0; r < 3; r++) {
      float z = Vn[3 * c + r];
      for (int i = 0; i <= j; i++) z -= d2[i] * Vb[(size_t)i * N3 + 3 * c + r];
      Vn[3 * c + r] = z;
      hs += z * z;
    }
  const float hn = sqrtf(block_sum(hs, sh));
  if (threadIdx.x == 0) {
    float *H = G.fm_H + (size_t)l * (m + 1) * m;
    float *cs = G.fm_cs + (size_t)l * m, *sn = G.fm_sn + (size_t)l * m, *g = G.fm_g + (size_t)l * (m + 1);
    float h[kFmMax + 1];
    for (int i = 0; i <= j; i++) h[i] = d[i] + d2[i];
    h[j + 1] = hn;
    for (int i = 0; i < j; i++) {   // earlier rotations on column j
      const float a0 = h[i], a1 = h[i + 1];
      h[i] = cs[i] * a0 + sn[i] * a1;
      h[i + 1] = -sn[i] * a0 + cs[i] * a1;
    }
    const float a0 = h[j], a1 = h[j + 1], rr = sqrtf(a0 * a0 + a1 * a1);
    cs[j] = rr > 0.f ? a0 / rr : 1.f;
    sn[j] = rr > 0.f ? a1 / rr : 0.f;
    h[j] = rr;
    for (int i = 0; i <= j; i++) H[(size_t)i * m + j] = h[i];
    H[(size_t)(j + 1) * m + j] = 0.f;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    const int stop = hn <= 1e-6f * G.fm_beta[l];
    G.fm_jm[l] = stop ? -(j + 1) - 1 : j + 1;
    s_hn = hn;
    s_stop = stop;
  }
  __syncthreads();
  if (!s_stop)
    for (int c = threadIdx.x; c < cnt; c += blockDim.x)
      for (int r = 0; r < 3; r++) Vn[3 * c + r] = Vn[3 * c + r] / s_hn;
}

// dy = P^-1 V y from the triangular system, multiplier update and J^T dgamma
__device__ __forceinline__ void fm_finish_body(const GroupView &G, const int l, const EnvView &V, const StepArgs &a,
                                               int tc) {
  extern __shared__ float fs[];   // [3][n]
  __shared__ float sh3[32][3];
  __shared__ float ys[kFmMax];
  const int e = G.genv[l];
  if (V.done[e]) return;
  const int n = G.n, np = G.n_pad, cap = G.cap, m = G.fm_m;
  const size_t N3 = 3 * (size_t)cap;
  const int jv = G.fm_jm[l], jm = jv < 0 ? -jv - 1 : jv;
  if (threadIdx.x == 0) {
    const float *H = G.fm_H + (size_t)l * (m + 1) * m, *g = G.fm_g + (size_t)l * (m + 1);
    for (int i = jm - 1; i >= 0; i--) {
      float sacc = g[i];
      for (int c = i + 1; c < jm; c++) sacc -= H[(size_t)i * m + c] * ys[c];
      const float hii = H[(size_t)i * m + i];
      ys[i] = hii != 0.f ? sacc / hii : 0.f;
    }
  }
  for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) fs[i] = 0.f;
  __syncthreads();
  const int cnt = G.ccount[l];
  const int *cvert = G.cvert + (size_t)l * cap;
  const float *lin = G.fm_lin + (size_t)l * cap * kFmLin;
  const float *Vb = G.fm_V + (size_t)l * (m + 1) * N3;
  float *gam = G.cgam + (size_t)l * cap * 4;
  float fm0 = 0.f, fm1 = 0.f, fm2 = 0.f;
  for (int c = threadIdx.x; c < cnt; c += blockDim.x) {
    const int vtx = chk(cvert[c], G.n, G.status);
    if (c > 0 && cvert[c - 1] == vtx) continue;
    const float mv = __ldg(G.mass + vtx);
    V3 fsum = v3(0.f, 0.f, 0.f);
    for (int cc = c; cc < cnt && cvert[cc] == vtx; cc++) {
      ContactLin L;
      const float sc = fm_load(lin + (size_t)cc * kFmLin, L);
      float z[3] = {0.f, 0.f, 0.f};
      for (int i = 0; i < jm; i++)
        for (int r = 0; r < 3; r++) z[r] += ys[i] * Vb[(size_t)i * N3 + 3 * cc + r];
      float dy[3];
      fm_pinv(L, sc, z, dy);
      const bool selfrow = G.self && G.cobs[(size_t)l * cap + cc] >= FLASH_SELF_SLOT;
      SelfRow S;
      if (selfrow) fm_row_load(G.fm_w + ((size_t)l * cap + cc) * kFmW, vtx, S, G.n, G.status);
      const V3 F = apply_update(L, selfrow ? S.meff : mv, a.gmax, dy, gam + 4 * cc);
      if (selfrow) scatter_row(S.v, S.w, F, fs, n);
      else fsum = fsum + F;
    }
    if (G.self) {
      atomicAdd(fs + vtx, fsum.x); atomicAdd(fs + n + vtx, fsum.y); atomicAdd(fs + 2 * n + vtx, fsum.z);
    } else {
      fs[vtx] = fsum.x; fs[n + vtx] = fsum.y; fs[2 * n + vtx] = fsum.z;
    }
    fm0 = fmaxf(fm0, fabsf(fsum.x)); fm1 = fmaxf(fm1, fabsf(fsum.y)); fm2 = fmaxf(fm2, fabsf(fsum.z));
  }
  __syncthreads();
  if (tc) {
    write_split_columns(G, l, fs, n, sh3, G.self != 0, fm0, fm1, fm2, G.f);
  } else {
    float *f = G.f + (size_t)l * 3 * np;
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
      const int c = i / n, jj = i - c * n;
      f[c * np + jj] = fs[i];
    }
  }
}

// diag(A^-1): dense inverse (shared by the group's environments) or, for the
// eigen form, sum_k V[v][k]^2 / (1 + k_e lam_k) per environment
__global__ void k_fm_adiag(const float *Ainv, const float *Vm, const float *lam, const float *kenv, int n, int np,
                           float *out) {
  const int l = blockIdx.y;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    if (Ainv) {
      out[v] = Ainv[(size_t)v * np + v];
    } else {
      const float ke = kenv[l];
      float s = 0.f;
      for (int k = 0; k < n; k++) {
        const float x = Vm[(size_t)v * np + k];
        s += x * x / (1.f + ke * lam[k]);
      }
      out[(size_t)l * np + v] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// end of step: velocity, keep the contact list for warm starts
// ---------------------------------------------------------------------------
__device__ __forceinline__ void end_body(const GroupView &G, const int l, const EnvView &V, const StepArgs &a) {
  const int n = G.n, np = G.n_pad;
  const float inv_h = 1.f / a.h;
  float *q = G.q + (size_t)l * 3 * np, *v = G.v + (size_t)l * 3 * np;
  const float *qt = G.qt + (size_t)l * 3 * np;
  // 16-byte columns (n_pad is a multiple of 128); q and q_t are zero in the
  // padding, so the velocity there is zero too
  const int n4 = (n + 3) >> 2;
  for (int i = threadIdx.x; i < 3 * n4; i += blockDim.x) {
    const int c = i / n4, j = (i - c * n4) * 4;
    const float4 qq = *reinterpret_cast<const float4 *>(q + c * np + j);
    const float4 tt = *reinterpret_cast<const float4 *>(qt + c * np + j);
    const float4 vv = make_float4((qq.x - tt.x) * inv_h, (qq.y - tt.y) * inv_h, (qq.z - tt.z) * inv_h,
                                  (qq.w - tt.w) * inv_h);
    *reinterpret_cast<float4 *>(v + c * np + j) = vv;
    if (!(isfinite(qq.x) && isfinite(qq.y) && isfinite(qq.z) && isfinite(qq.w))) atomicOr(V.status, 1 << 9);
  }
  const int cnt = G.ccount[l];
  if (threadIdx.x == 0) G.pcount[l] = cnt;
  const float4 *cg = reinterpret_cast<const float4 *>(G.cgam + (size_t)l * G.cap * 4);
  float4 *pg = reinterpret_cast<float4 *>(G.pgam + (size_t)l * G.cap * 4);
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    G.pvert[(size_t)l * G.cap + j] = G.cvert[(size_t)l * G.cap + j];
    G.pobs[(size_t)l * G.cap + j] = G.cobs[(size_t)l * G.cap + j];
    if (G.self) G.pctri[(size_t)l * G.cap + j] = G.ctri[(size_t)l * G.cap + j];
    pg[j] = cg[j];
  }
}

// grasp requests (1 activate, 0 release, -1 keep) -> per-environment grasp
// state; the activation itself runs in the next step's begin kernel
__global__ void k_grasp_set(int *gstate, int *gobs, float *ganchor, const int *req, int first, int count, int obstacle,
                            float4 anchor_radius) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int e = first + i, r = req[e];
  if (r == 1) {
    gstate[e] = 1;
    gobs[e] = obstacle;
    ganchor[4 * e] = anchor_radius.x; ganchor[4 * e + 1] = anchor_radius.y;
    ganchor[4 * e + 2] = anchor_radius.z; ganchor[4 * e + 3] = anchor_radius.w;
  } else if (r == 0) {
    gstate[e] = gstate[e] == 0 ? 0 : 3;
  }
}

// Entry points: table launches over the environments of one or more groups,
// CTA b = (group map[b].x, environment map[b].y).  Every scene, one group or
// many, runs these same kernels.
template <bool SELF>
__global__ void __launch_bounds__(256) k_begin_tab(const GroupView *__restrict__ tab, const int2 *__restrict__ map,
                                                   EnvView V, StepArgs a, int boxes) {
  const int2 b = map[blockIdx.x];
  begin_body<SELF>(tab[b.x], b.y, V, a, boxes);
}
template <int VPE, bool SELF, int NT = 512>
__global__ void __launch_bounds__(NT, 1024 / NT) k_local_tab(const GroupView *__restrict__ tab, const int2 *__restrict__ map,
                                                      EnvView V, StepArgs a, int k, int residual_only, int tc,
                                                      int pending) {
  const int2 b = map[blockIdx.x];
  if (k == 0) {   // inside the graphed tolerance loop: the iteration index is on the device
    k = *V.kit;
    pending = k > 1;
  }
  local_body<VPE, SELF>(tab[b.x], b.y, V, a, k, residual_only, tc, pending);
}
__global__ void __launch_bounds__(512, 2) k_refine(GroupView G, EnvView V, const float *rhs32, const float *w, int l0) {
  refine_body(G, l0 + blockIdx.x, V, rhs32, w);
}
// End of one iteration of the graphed tolerance loop (Mode B): the loop runs
// again while some environment is still iterating and the cap allows; the
// index only grows, so the loop ends after at most `last` - 1 runs whatever
// the kernels computed.  first = 1 after the loop's first iteration, which
// runs ahead of the loop with a literal index.
__global__ void k_tol_next(cudaGraphConditionalHandle h, int *active, int *kit, unsigned long long *trips, int last,
                           int first) {
  const int k = first ? 1 : *kit;
  cudaGraphSetConditional(h, (*active > 0 && k < last) ? 1u : 0u);
  *active = 0;
  *kit = k + 1;
  if (!first) *trips += 1;
}
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_ncp_tab(const GroupView *__restrict__ tab,
                                                          const int2 *__restrict__ map, EnvView V, StepArgs a, int tc) {
  const int2 b = map[blockIdx.x];
  ncp_body(tab[b.x], b.y, V, a, tc);
}
__global__ void __launch_bounds__(256) k_end_tab(const GroupView *__restrict__ tab, const int2 *__restrict__ map,
                                                 EnvView V, StepArgs a) {
  const int2 b = map[blockIdx.x];
  end_body(tab[b.x], b.y, V, a);
}

__global__ void __launch_bounds__(256) k_fm_setup_tab(const GroupView *__restrict__ tab, const int2 *__restrict__ map,
                                                      EnvView V, StepArgs a) {
  const int2 b = map[blockIdx.x];
  fm_setup_body(tab[b.x], b.y, V, a);
}
__global__ void __launch_bounds__(256) k_fm_scatter_tab(const GroupView *__restrict__ tab, const int2 *__restrict__ map,
                                                        EnvView V, int j, int tc) {
  const int2 b = map[blockIdx.x];
  fm_scatter_body(tab[b.x], b.y, V, j, tc);
}
__global__ void __launch_bounds__(256) k_fm_gather_tab(const GroupView *__restrict__ tab, const int2 *__restrict__ map,
                                                       EnvView V, int j) {
  const int2 b = map[blockIdx.x];
  fm_gather_body(tab[b.x], b.y, V, j);
}
__global__ void __launch_bounds__(256) k_fm_finish_tab(const GroupView *__restrict__ tab, const int2 *__restrict__ map,
                                                       EnvView V, StepArgs a, int tc) {
  const int2 b = map[blockIdx.x];
  fm_finish_body(tab[b.x], b.y, V, a, tc);
}

// user layout [sum n_e][3] <-> group columns [N_g][3][n_pad]
__global__ void k_state_io(GroupView G, const int64_t *voff, const float *qu, const float *vu, float *qo, float *vo,
                           int to_user) {
  const int l = blockIdx.y, e = G.genv[l];
  const int n = G.n, np = G.n_pad;
  const int64_t base = voff[e];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int c = 0; c < 3; c++) {
      size_t gi = (size_t)l * 3 * np + (size_t)c * np + i;
      size_t ui = (size_t)(base + i) * 3 + c;
      if (to_user) {
        if (qo) qo[ui] = G.q[gi];
        if (vo) vo[ui] = G.v[gi];
      } else {
        if (qu) G.q[gi] = qu[ui];
        if (vu) G.v[gi] = vu[ui];
      }
    }
}

__global__ void k_rhs_io(int n, int np, const int *genv, const int64_t *voff, int first_env, const float *user,
                         float *cols, int to_user) {
  const int l = blockIdx.y;
  const int64_t base = voff[genv[l]] - voff[first_env];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int c = 0; c < 3; c++) {
      size_t gi = (size_t)l * 3 * np + (size_t)c * np + i;
      size_t ui = (size_t)(base + i) * 3 + c;
      if (to_user) ((float *)user)[ui] = cols[gi];
      else cols[gi] = user[ui];
    }
}

__global__ void __launch_bounds__(256) k_split(GroupView G, const float *src, int l0) {
  __shared__ float sh3[32][3];
  extern __shared__ float vals[];
  const int l = l0 + blockIdx.x, n = G.n, np = G.n_pad;
  for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
    int c = i / n, j = i - c * n;
    vals[i] = src[(size_t)l * 3 * np + c * np + j];
  }
  __syncthreads();
  write_split_columns(G, l, vals, n, sh3, true);
}

// ---------------------------------------------------------------------------
// learned warm start: per-contact features, prediction, training targets
// ---------------------------------------------------------------------------
// Feature / output scales: gaps and scaled multipliers y = gamma / m_v in
// millimetres, velocities in units of 0.1 m/s.
constexpr float kFeatLen = 1e3f, kFeatVel = 10.f;
constexpr int kWarmDq = 1, kWarmNormalOnly = 2;

__global__ void k_row_offsets(const int *count, int N, int64_t *off) {
  __shared__ int sh[32];
  int64_t base = 0;
  for (int i0 = 0; i0 < N; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const int c = i < N ? count[i] : 0;
    int total;
    const int ex = block_exclusive_scan(c, &total, sh);
    if (i < N) off[i] = base + ex;
    base += total;
  }
  if (threadIdx.x == 0) off[N] = base;
}

// frame (n, t1, t2) and gap of a contact at the predicted position
__device__ __forceinline__ void contact_frame_at(const ObsShared &O, int o, float tau, V3 x, V3 &n, V3 &t1, V3 &t2,
                                                 float &gap) {
  gap = obstacle_sdf(O.type[o], O.dims[o], O.pose[o], x, n) - tau;
  tangent_basis(n, t1, t2);
}

__global__ void __launch_bounds__(256) k_features(GroupView G, EnvView V, StepArgs a, const int64_t *off, float *X) {
  __shared__ ObsShared O;
  const int l = blockIdx.x, e = G.genv[l];
  const int np = G.n_pad;
  load_obstacles(V, e, a.K, O);
  __syncthreads();
  const int cnt = G.ccount[l];
  const int *cvert = G.cvert + (size_t)l * G.cap, *cobs = G.cobs + (size_t)l * G.cap;
  const float *qp = G.qp + (size_t)l * 3 * np, *v = G.v + (size_t)l * 3 * np;
  const int pc = G.pcount[l];
  const int *pv = G.pvert + (size_t)l * G.cap, *po = G.pobs + (size_t)l * G.cap;
  const float *pg = G.pgam + (size_t)l * G.cap * 4;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const int vtx = chk(cvert[j], G.n, G.status), o = chk(cobs[j], kSlots, G.status);
    if (o >= FLASH_GRASP_SLOT) {   // grasp and self rows are not predicted: NaN features keep them cold
      for (int c = 0; c < 10; c++) X[(off[l] + j) * 10 + c] = __int_as_float(0x7fc00000);
      continue;
    }
    const V3 x = v3(qp[vtx], qp[np + vtx], qp[2 * np + vtx]);
    V3 n, t1, t2;
    float gap;
    contact_frame_at(O, o, a.tau, x, n, t1, t2, gap);
    // obstacle velocity at the point over the step
    const float *pt = O.poset[o], *pth = O.pose[o];
    const V3 pb = qrot(pth + 3, x - v3(pth[0], pth[1], pth[2]), true);
    const V3 xo = qrot(pt + 3, pb, false) + v3(pt[0], pt[1], pt[2]);
    const V3 vr = v3(v[vtx], v[np + vtx], v[2 * np + vtx]) - (1.f / a.h) * (x - xo);
    // previous step's multipliers of the same (vertex, obstacle)
    float g4[4] = {0.f, 0.f, 0.f, 0.f};
    const int key = vtx * kSlots + o;
    int lo = 0, hi = pc - 1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int km = pv[mid] * kSlots + po[mid];
      if (km == key) {
        for (int c = 0; c < 4; c++) g4[c] = pg[mid * 4 + c];
        break;
      }
      if (km < key) lo = mid + 1; else hi = mid - 1;
    }
    const float s = kFeatLen / __ldg(G.mass + vtx);
    const V3 gt = v3(g4[1], g4[2], g4[3]);
    float *xr = X + (off[l] + j) * 10;
    xr[0] = gap * kFeatLen;
    xr[1] = dot(n, vr) * kFeatVel; xr[2] = dot(t1, vr) * kFeatVel; xr[3] = dot(t2, vr) * kFeatVel;
    xr[4] = n.x; xr[5] = n.y; xr[6] = n.z;
    xr[7] = g4[0] * s; xr[8] = dot(t1, gt) * s; xr[9] = dot(t2, gt) * s;
  }
}

// gamma^0 (and optionally q^0 at contact vertices) from the network output
__global__ void __launch_bounds__(256) k_apply_learned(GroupView G, EnvView V, StepArgs a, const int64_t *off,
                                                       const float *X, const float *Y, const float *bounds,
                                                       int flags) {
  __shared__ ObsShared O;
  const int l = blockIdx.x, e = G.genv[l];
  const int np = G.n_pad;
  load_obstacles(V, e, a.K, O);
  __syncthreads();
  const int cnt = G.ccount[l];
  const int *cvert = G.cvert + (size_t)l * G.cap, *cobs = G.cobs + (size_t)l * G.cap;
  float *qp = G.qp + (size_t)l * 3 * np, *q = G.q + (size_t)l * 3 * np;
  float *gam = G.cgam + (size_t)l * G.cap * 4;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const int vtx = chk(cvert[j], G.n, G.status), o = chk(cobs[j], kSlots, G.status);
    if (o >= FLASH_GRASP_SLOT) continue;
    const V3 x = v3(qp[vtx], qp[np + vtx], qp[2 * np + vtx]);
    V3 n, t1, t2;
    float gap;
    contact_frame_at(O, o, a.tau, x, n, t1, t2, gap);
    const float *y = Y + (off[l] + j) * 6;
    // contacts whose features lie outside the trained range start cold
    const float *xr = X + (off[l] + j) * 10;
    bool in_range = true;
    for (int c = 0; c < 10; c++) in_range = in_range && xr[c] >= bounds[c] && xr[c] <= bounds[10 + c];
    if (!in_range) continue;
    const float mv = __ldg(G.mass + vtx) / kFeatLen;
    const float gn = fmaxf(y[0], 0.f) * mv;
    const V3 gt = (flags & kWarmNormalOnly) ? v3(0.f, 0.f, 0.f) : (y[1] * mv) * t1 + (y[2] * mv) * t2;
    float *g = gam + 4 * j;
    g[0] = fminf(gn, a.gmax); g[1] = gt.x; g[2] = gt.y; g[3] = gt.z;
    if ((flags & kWarmDq) && (j == 0 || cvert[j - 1] != vtx)) {
      q[vtx] = x.x + y[3] / kFeatLen;
      q[np + vtx] = x.y + y[4] / kFeatLen;
      q[2 * np + vtx] = x.z + y[5] / kFeatLen;
    }
  }
}

// training targets after the step: converged multipliers in the frame of the
// predicted position (scaled like the features) and q* - q~ at the vertex
__global__ void __launch_bounds__(256) k_targets(GroupView G, EnvView V, StepArgs a, const int64_t *off, float *T) {
  __shared__ ObsShared O;
  const int l = blockIdx.x, e = G.genv[l];
  const int np = G.n_pad;
  load_obstacles(V, e, a.K, O);
  __syncthreads();
  const int cnt = G.ccount[l];
  const int *cvert = G.cvert + (size_t)l * G.cap, *cobs = G.cobs + (size_t)l * G.cap;
  const float *qp = G.qp + (size_t)l * 3 * np, *q = G.q + (size_t)l * 3 * np;
  const float *gam = G.cgam + (size_t)l * G.cap * 4;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const int vtx = chk(cvert[j], G.n, G.status), o = chk(cobs[j], kSlots, G.status);
    float *t = T + (off[l] + j) * 6;
    if (o >= FLASH_GRASP_SLOT || !(V.rncp[e] <= a.tol)) {   // grasp / self row or not converged: no target
      for (int c = 0; c < 6; c++) t[c] = __int_as_float(0x7fc00000);
      continue;
    }
    const V3 x = v3(qp[vtx], qp[np + vtx], qp[2 * np + vtx]);
    V3 n, t1, t2;
    float gap;
    contact_frame_at(O, o, a.tau, x, n, t1, t2, gap);
    const float *g = gam + 4 * j;
    const float s = kFeatLen / __ldg(G.mass + vtx);
    const V3 gt = v3(g[1], g[2], g[3]);
    t[0] = g[0] * s; t[1] = dot(t1, gt) * s; t[2] = dot(t2, gt) * s;
    t[3] = (q[vtx] - x.x) * kFeatLen; t[4] = (q[np + vtx] - x.y) * kFeatLen; t[5] = (q[2 * np + vtx] - x.z) * kFeatLen;
  }
}

}  // namespace

template <int NT>
cudaError_t configure_local() {
  cudaError_t e = cudaFuncSetAttribute(k_local_tab<3, false, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       220 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_local_tab<3, true, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_local_tab<4, false, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
}

cudaError_t configure_kernels() {
  cudaError_t e = configure_local<256>();
  if (e != cudaSuccess) return e;
  e = configure_local<512>();
  if (e != cudaSuccess) return e;
  e = configure_local<1024>();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_refine, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_ncp_tab<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_ncp_tab<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_ncp_tab<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_begin_tab<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxBeginSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fm_scatter_tab, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fm_finish_tab, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_split, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
}

cudaError_t launch_row_offsets(const Group &g, int64_t *off, cudaStream_t st) {
  k_row_offsets<<<1, 1024, 0, st>>>(g.ccount, g.N, off);
  return cudaGetLastError();
}

cudaError_t launch_features(const flash_scene *s, const Group &g, const StepArgs &a, const int64_t *off, float *X,
                            cudaStream_t st) {
  k_features<<<g.N, 256, 0, st>>>(view(s, g), eview(s), a, off, X);
  return cudaGetLastError();
}

cudaError_t launch_apply_learned(const flash_scene *s, const Group &g, const StepArgs &a, const int64_t *off,
                                 const float *X, const float *Y, const float *bounds, int flags, cudaStream_t st) {
  k_apply_learned<<<g.N, 256, 0, st>>>(view(s, g), eview(s), a, off, X, Y, bounds, flags);
  return cudaGetLastError();
}

cudaError_t launch_targets(const flash_scene *s, const Group &g, const StepArgs &a, const int64_t *off, float *T,
                           cudaStream_t st) {
  k_targets<<<g.N, 256, 0, st>>>(view(s, g), eview(s), a, off, T);
  return cudaGetLastError();
}

cudaError_t launch_state_io(const flash_scene *s, const Group &g, const float *q_user, const float *v_user,
                            float *q_out, float *v_out, int to_user, cudaStream_t st) {
  dim3 grid((g.n + 255) / 256, g.N);
  k_state_io<<<grid, 256, 0, st>>>(view(s, g), s->d_voff, q_user, v_user, q_out, v_out, to_user);
  return cudaGetLastError();
}

cudaError_t launch_rhs_io(const Group &g, const int64_t *voff, int first_env, const float *user, float *cols,
                          int to_user, cudaStream_t st) {
  dim3 grid((g.n + 255) / 256, g.N);
  k_rhs_io<<<grid, 256, 0, st>>>(g.n, g.n_pad, g.genv, voff, first_env, user, cols, to_user);
  return cudaGetLastError();
}

cudaError_t launch_refine(const flash_scene *s, const Group &g, const float *rhs32, const float *w, int l0, int l1,
                          cudaStream_t st) {
  if (g.vpe != 4) return cudaErrorInvalidValue;
  if (l1 <= l0) return cudaSuccess;
  k_refine<<<l1 - l0, 512, g.smem_local, st>>>(view(s, g), eview(s), rhs32, w, l0);
  return cudaGetLastError();
}

cudaError_t launch_split_rhs(const Group &g, const float *src, cudaStream_t st, int l0, int l1, bool bf16) {
  if (l1 < 0) l1 = g.N;
  if (l0 < 0 || l1 > g.N || l0 >= l1) return l0 == l1 ? cudaSuccess : cudaErrorInvalidValue;
  GroupView v;
  memset(&v, 0, sizeof v);
  v.n = g.n; v.n_pad = g.n_pad; v.rh = g.rh; v.rl = g.rl; v.rscale = g.rscale;
  v.bf16 = bf16 ? 1 : 0;
  k_split<<<l1 - l0, 256, sizeof(float) * 3 * g.n, st>>>(v, src, l0);
  return cudaGetLastError();
}

namespace {

template <typename T>
cudaError_t upload_owned(flash_scene *s, T **p, const std::vector<T> &h) {
  void *ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(h.size(), 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  s->allocs.push_back(ptr);
  *p = (T *)ptr;
  if (!h.empty()) e = cudaMemcpy(ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

// Shared-memory class of a local-pass CTA (a batching key): how many CTAs with
// `smem` bytes of dynamic shared memory next to their static shared memory
// fit on one SM, at most 4.
int local_class(size_t smem) {
  const size_t per_sm = 228 * 1024, static_smem = sizeof(ObsShared) + 1024;
  const int c = (int)(per_sm / (smem + static_smem + 1024));
  return std::max(1, std::min(4, c));
}

}  // namespace

// Lanes: the environments are partitioned into lanes that step concurrently
// on their own streams.  A group with at least kMinLaneEnvs environments per
// lane is split into contiguous environment ranges, one per lane (each range
// still fills whole contraction tiles); smaller groups go whole to the
// least-loaded lane (work ~ environments x (vertices + elements)).  Each
// lane gets block maps for its table launches: larger
// meshes first, so their longer CTAs start in the first wave; the local
// pass split by element type and by how many of its CTAs fit on one SM.
constexpr int kMinLaneEnvs = 64;

cudaError_t build_lanes(flash_scene *s, int n_lanes) {
  const int G = (int)s->groups.size();
  std::vector<GroupView> tab(G);
  for (int i = 0; i < G; i++) tab[i] = view(s, s->groups[i]);
  GroupView *dtab = nullptr;
  cudaError_t e = upload_owned(s, &dtab, tab);
  if (e != cudaSuccess) return e;
  s->gtab = dtab;
  n_lanes = std::max(1, n_lanes);
  s->lanes.assign(n_lanes, Lane());
  std::vector<double> load(n_lanes, 0.0);
  std::vector<int> order(G);
  for (int i = 0; i < G; i++) order[i] = i;
  auto work = [&](int gi) { const Group &g = s->groups[gi]; return (double)g.N * (g.n + g.E); };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
  for (int gi : order) {
    const Group &g = s->groups[gi];
    if (g.N >= kMinLaneEnvs * n_lanes) {
      for (int k = 0; k < n_lanes; k++) {
        LaneRange r;
        r.group = gi;
        r.l0 = (int)((int64_t)g.N * k / n_lanes);
        r.l1 = (int)((int64_t)g.N * (k + 1) / n_lanes);
        s->lanes[k].ranges.push_back(r);
        load[k] += work(gi) / n_lanes;
      }
    } else {
      const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      LaneRange r;
      r.group = gi;
      r.l0 = 0;
      r.l1 = g.N;
      s->lanes[k].ranges.push_back(r);
      load[k] += work(gi);
    }
  }
  for (Lane &L : s->lanes) {
    // ranges of larger meshes first
    std::stable_sort(L.ranges.begin(), L.ranges.end(), [&](const LaneRange &x, const LaneRange &y) {
      const Group &a = s->groups[x.group], &b = s->groups[y.group];
      return (int64_t)a.E + a.n > (int64_t)b.E + b.n;
    });
    std::vector<int2> all;
    int nmax = 0;
    for (const LaneRange &r : L.ranges) {
      for (int l = r.l0; l < r.l1; l++) all.push_back(make_int2(r.group, l));
      nmax = std::max(nmax, s->groups[r.group].n);
    }
    L.all.blocks = (int)all.size();
    if ((e = upload_owned(s, &L.all.map, all)) != cudaSuccess) return e;
    L.ncp_smem_tc = sizeof(float) * 3 * (size_t)nmax;
    L.ncp_threads = s->d.ncp_threads > 0 ? s->d.ncp_threads : 256;
    for (int vpe = 3; vpe <= 4; vpe++)
      for (int big = 1; big >= 0; big--)
      for (int cls = 4; cls >= 1; cls--) {
        Batch b;
        b.vpe = vpe;
        b.threads = s->d.local_threads > 0 ? s->d.local_threads : big ? 1024 : 512;
        std::vector<int2> m;
        for (const LaneRange &r : L.ranges) {
          const Group &g = s->groups[r.group];
          if (g.vpe != vpe || local_class(g.smem_local) != cls || (g.n > kBigMesh) != (big == 1)) continue;
          for (int l = r.l0; l < r.l1; l++) m.push_back(make_int2(r.group, l));
          b.smem = std::max(b.smem, g.smem_local);
        }
        if (m.empty()) continue;
        b.blocks = (int)m.size();
        if ((e = upload_owned(s, &b.map, m)) != cudaSuccess) return e;
        L.local.push_back(b);
      }
  }
  return cudaSuccess;
}

cudaError_t launch_grasp_set(const flash_scene *s, int first_env, int count, int obstacle, float ax, float ay,
                             float az, float radius, cudaStream_t st) {
  k_grasp_set<<<(count + 255) / 256, 256, 0, st>>>(s->gstate, s->gobs, s->ganchor, s->greq, first_env, count,
                                                   obstacle, make_float4(ax, ay, az, radius));
  return cudaGetLastError();
}

cudaError_t launch_begin_lane(const flash_scene *s, const Lane &L, const StepArgs &a, cudaStream_t st) {
  if (!L.all.blocks) return cudaSuccess;
  if (s->d.self_collide || s->d.obstacle_features)
    k_begin_tab<true><<<L.all.blocks, 256, s->begin_smem, st>>>((const GroupView *)s->gtab, L.all.map, eview(s), a,
                                                               s->begin_smem > 0 ? 1 : 0);
  else
    k_begin_tab<false><<<L.all.blocks, 256, 0, st>>>((const GroupView *)s->gtab, L.all.map, eview(s), a, 0);
  return cudaGetLastError();
}

namespace {
template <int NT>
void local_launch(const flash_scene *s, const Batch &b, const StepArgs &a, int k, int residual_only, int tc,
                  cudaStream_t st) {
  const int pending = k > 1;
  const GroupView *tab = (const GroupView *)s->gtab;
  const bool self = s->d.self_collide || s->d.obstacle_features;
  if (b.vpe == 3 && self)
    k_local_tab<3, true, NT><<<b.blocks, NT, b.smem, st>>>(tab, b.map, eview(s), a, k, residual_only, tc, pending);
  else if (b.vpe == 3)
    k_local_tab<3, false, NT><<<b.blocks, NT, b.smem, st>>>(tab, b.map, eview(s), a, k, residual_only, tc, pending);
  else
    k_local_tab<4, false, NT><<<b.blocks, NT, b.smem, st>>>(tab, b.map, eview(s), a, k, residual_only, tc, pending);
}
}  // namespace

// One local-pass batch with `threads` threads per environment (0: the
// batch's own choice).
cudaError_t launch_local_batch(const flash_scene *s, const Batch &b, int threads, const StepArgs &a, int k,
                               int residual_only, int tc, cudaStream_t st) {
  switch (threads > 0 ? threads : b.threads) {
    case 256: local_launch<256>(s, b, a, k, residual_only, tc, st); break;
    case 512: local_launch<512>(s, b, a, k, residual_only, tc, st); break;
    case 1024: local_launch<1024>(s, b, a, k, residual_only, tc, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_local_lane(const flash_scene *s, const Lane &L, const StepArgs &a, int k, int residual_only, int tc,
                              cudaStream_t st, int *launched) {
  for (const Batch &b : L.local) {
    const cudaError_t e = launch_local_batch(s, b, 0, a, k, residual_only, tc, st);
    if (e != cudaSuccess) return e;
    ++*launched;
  }
  return cudaSuccess;
}

cudaError_t launch_tol_next(cudaGraphConditionalHandle h, int *active, int *kit, unsigned long long *trips, int last,
                            int first, cudaStream_t st) {
  k_tol_next<<<1, 1, 0, st>>>(h, active, kit, trips, last, first);
  return cudaGetLastError();
}

cudaError_t launch_ncp_lane(const flash_scene *s, const Lane &L, const StepArgs &a, int tc, cudaStream_t st,
                            int threads) {
  if (!L.all.blocks) return cudaSuccess;
  const GroupView *tab = (const GroupView *)s->gtab;
  const size_t smem = tc ? L.ncp_smem_tc : 0;
  switch (threads > 0 ? threads : L.ncp_threads) {
    case 128: k_ncp_tab<128><<<L.all.blocks, 128, smem, st>>>(tab, L.all.map, eview(s), a, tc); break;
    case 256: k_ncp_tab<256><<<L.all.blocks, 256, smem, st>>>(tab, L.all.map, eview(s), a, tc); break;
    case 512: k_ncp_tab<512><<<L.all.blocks, 512, smem, st>>>(tab, L.all.map, eview(s), a, tc); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_end_lane(const flash_scene *s, const Lane &L, const StepArgs &a, cudaStream_t st) {
  if (!L.all.blocks) return cudaSuccess;
  k_end_tab<<<L.all.blocks, 256, 0, st>>>((const GroupView *)s->gtab, L.all.map, eview(s), a);
  return cudaGetLastError();
}

cudaError_t launch_fm_setup_lane(const flash_scene *s, const Lane &L, const StepArgs &a, cudaStream_t st) {
  if (!L.all.blocks) return cudaSuccess;
  k_fm_setup_tab<<<L.all.blocks, 256, 0, st>>>((const GroupView *)s->gtab, L.all.map, eview(s), a);
  return cudaGetLastError();
}

cudaError_t launch_fm_scatter_lane(const flash_scene *s, const Lane &L, const StepArgs &a, int j, int tc,
                                   cudaStream_t st) {
  (void)a;
  if (!L.all.blocks) return cudaSuccess;
  k_fm_scatter_tab<<<L.all.blocks, 256, L.ncp_smem_tc, st>>>((const GroupView *)s->gtab, L.all.map, eview(s), j, tc);
  return cudaGetLastError();
}

cudaError_t launch_fm_gather_lane(const flash_scene *s, const Lane &L, const StepArgs &a, int j, cudaStream_t st) {
  (void)a;
  if (!L.all.blocks) return cudaSuccess;
  k_fm_gather_tab<<<L.all.blocks, 256, 0, st>>>((const GroupView *)s->gtab, L.all.map, eview(s), j);
  return cudaGetLastError();
}

cudaError_t launch_fm_finish_lane(const flash_scene *s, const Lane &L, const StepArgs &a, int tc, cudaStream_t st) {
  if (!L.all.blocks) return cudaSuccess;
  k_fm_finish_tab<<<L.all.blocks, 256, L.ncp_smem_tc, st>>>((const GroupView *)s->gtab, L.all.map, eview(s), a, tc);
  return cudaGetLastError();
}

cudaError_t launch_fm_adiag(const Group &g, cudaStream_t st) {
  dim3 grid((g.n + 255) / 256, g.eig ? g.N : 1);
  k_fm_adiag<<<grid, 256, 0, st>>>(g.eig ? nullptr : g.inv.f32, g.V.f32, g.lam, g.kenv, g.n, g.n_pad, g.fm_adiag);
  return cudaGetLastError();
}

}  // namespace flash
