// Device-side geometry and per-element / per-contact math of the step.
// FP32 throughout; every function is a restatement of the method's step:
//   closest rotation   -> local projection of Eq. (internal)
//   sdf / frame / law  -> contact function phi of Eq. (lagrange_b)
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "../../include/flash.h"

namespace flash {

struct V3 {
  float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float norm(V3 a) { return sqrtf(dot(a, a)); }

// rotation of v by unit quaternion q = (w, x, y, z), or by its conjugate
__device__ __forceinline__ V3 qrot(const float *q, V3 v, bool inverse) {
  float w = q[0], x = inverse ? -q[1] : q[1], y = inverse ? -q[2] : q[2], z = inverse ? -q[3] : q[3];
  // v' = v + 2w (u x v) + 2 u x (u x v),  u = (x, y, z)
  V3 u = {x, y, z};
  V3 t = 2.f * cross(u, v);
  return v + w * t + cross(u, t);
}

// Signed distance and outward unit normal of a kinematic obstacle at x.
// pose: p(3), quaternion(4).  Box: largest per-axis distance picks the face
// inside, ties resolved x < y < z.  Sphere centre maps to +z.
__device__ __forceinline__ float obstacle_sdf(int type, const float *dims, const float *pose, V3 x, V3 &n) {
  V3 p = qrot(pose + 3, x - v3(pose[0], pose[1], pose[2]), true);
  V3 nb = {0.f, 0.f, 1.f};
  float sd;
  if (type == FLASH_OBS_PLANE) {
    sd = p.z;
  } else if (type == FLASH_OBS_SPHERE) {
    float d = norm(p);
    if (d > 1e-12f) nb = (1.f / d) * p;
    sd = d - dims[0];
  } else {
    float dx = fabsf(p.x) - dims[0], dy = fabsf(p.y) - dims[1], dz = fabsf(p.z) - dims[2];
    if (dx > 0.f || dy > 0.f || dz > 0.f) {
      V3 o = {fmaxf(dx, 0.f), fmaxf(dy, 0.f), fmaxf(dz, 0.f)};
      float on = norm(o);
      nb = {copysignf(1.f, p.x) * o.x / on, copysignf(1.f, p.y) * o.y / on, copysignf(1.f, p.z) * o.z / on};
      if (p.x == 0.f) nb.x = o.x / on;
      if (p.y == 0.f) nb.y = o.y / on;
      if (p.z == 0.f) nb.z = o.z / on;
      sd = on;
    } else {
      int ax = 0;
      float dm = dx;
      if (dy > dm) { ax = 1; dm = dy; }
      if (dz > dm) { ax = 2; dm = dz; }
      float pc = ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
      float sg = pc >= 0.f ? 1.f : -1.f;
      nb = {ax == 0 ? sg : 0.f, ax == 1 ? sg : 0.f, ax == 2 ? sg : 0.f};
      sd = dm;
    }
  }
  n = qrot(pose + 3, nb, false);
  return sd;
}

// Obstacle pose as a rotation matrix (row-major, body -> world) and origin;
// `slip` maps a world point at t+h to where the same obstacle material point
// was at t: x_t = S x + s.
struct PoseM {
  float R[9], p[3];
  float S[9], s[3];
};

__device__ __forceinline__ void quat_to_mat(const float *q, float *R) {
  const float w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// pose_t, pose_th (p, quat) -> PoseM of the t+h pose plus the slip map
__device__ __forceinline__ void make_posem(const float *pose_t, const float *pose_th, PoseM &P) {
  float Rt[9];
  quat_to_mat(pose_th + 3, P.R);
  quat_to_mat(pose_t + 3, Rt);
  for (int i = 0; i < 3; i++) P.p[i] = pose_th[i];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++)
      P.S[3 * i + j] = Rt[3 * i] * P.R[3 * j] + Rt[3 * i + 1] * P.R[3 * j + 1] + Rt[3 * i + 2] * P.R[3 * j + 2];
  for (int i = 0; i < 3; i++)
    P.s[i] = pose_t[i] - (P.S[3 * i] * pose_th[0] + P.S[3 * i + 1] * pose_th[1] + P.S[3 * i + 2] * pose_th[2]);
}

// signed distance and outward unit normal with a matrix pose (same rules as obstacle_sdf)
__device__ __forceinline__ float obstacle_sdf_m(int type, const float *dims, const PoseM &P, V3 x, V3 &n) {
  const V3 d = x - v3(P.p[0], P.p[1], P.p[2]);
  const float *R = P.R;
  // body coordinates: R^T d
  const V3 p = {R[0] * d.x + R[3] * d.y + R[6] * d.z, R[1] * d.x + R[4] * d.y + R[7] * d.z,
                R[2] * d.x + R[5] * d.y + R[8] * d.z};
  V3 nb = {0.f, 0.f, 1.f};
  float sd;
  if (type == FLASH_OBS_PLANE) {
    sd = p.z;
  } else if (type == FLASH_OBS_SPHERE) {
    float dd = norm(p);
    if (dd > 1e-12f) nb = (1.f / dd) * p;
    sd = dd - dims[0];
  } else {
    float dx = fabsf(p.x) - dims[0], dy = fabsf(p.y) - dims[1], dz = fabsf(p.z) - dims[2];
    if (dx > 0.f || dy > 0.f || dz > 0.f) {
      V3 o = {fmaxf(dx, 0.f), fmaxf(dy, 0.f), fmaxf(dz, 0.f)};
      float on = norm(o);
      nb = {(p.x >= 0.f ? 1.f : -1.f) * o.x / on, (p.y >= 0.f ? 1.f : -1.f) * o.y / on,
            (p.z >= 0.f ? 1.f : -1.f) * o.z / on};
      sd = on;
    } else {
      int ax = 0;
      float dm = dx;
      if (dy > dm) { ax = 1; dm = dy; }
      if (dz > dm) { ax = 2; dm = dz; }
      float pc = ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
      float sg = pc >= 0.f ? 1.f : -1.f;
      nb = {ax == 0 ? sg : 0.f, ax == 1 ? sg : 0.f, ax == 2 ? sg : 0.f};
      sd = dm;
    }
  }
  n = {R[0] * nb.x + R[1] * nb.y + R[2] * nb.z, R[3] * nb.x + R[4] * nb.y + R[5] * nb.z,
       R[6] * nb.x + R[7] * nb.y + R[8] * nb.z};
  return sd;
}

// Branchless orthonormal basis (Duff et al. 2017): t1, t2 orthogonal to n.
__device__ __forceinline__ void tangent_basis(V3 n, V3 &t1, V3 &t2) {
  float s = n.z >= 0.f ? 1.f : -1.f;
  float a = -1.f / (s + n.z);
  float b = n.x * n.y * a;
  t1 = {1.f + s * n.x * n.x * a, s * b, -s * n.x};
  t2 = {b, s + n.y * n.y * a, -n.y};
}

// Closest 3x2 matrix with orthonormal columns to F (row-major 3x2):
// R = F (F^T F)^-1/2, with the closed-form square root of a 2x2 SPD matrix.
__device__ __forceinline__ void closest_rot32(const float *F, float *R) {
  float a = F[0] * F[0] + F[2] * F[2] + F[4] * F[4];
  float b = F[0] * F[1] + F[2] * F[3] + F[4] * F[5];
  float c = F[1] * F[1] + F[3] * F[3] + F[5] * F[5];
  float det = fmaxf(a * c - b * b, 0.f);
  float s = sqrtf(det);
  float t = sqrtf(fmaxf(a + c + 2.f * s, 0.f));
  if (s > 1e-10f * (a + c) && t > 0.f) {
    float k = 1.f / (s * t);
    float i00 = (c + s) * k, i01 = -b * k, i11 = (a + s) * k;
    for (int r = 0; r < 3; r++) {
      float f0 = F[2 * r], f1 = F[2 * r + 1];
      R[2 * r] = f0 * i00 + f1 * i01;
      R[2 * r + 1] = f0 * i01 + f1 * i11;
    }
    return;
  }
  // rank <= 1: keep the dominant column direction, complete with the axis
  // least aligned with it
  V3 c0 = {F[0], F[2], F[4]}, c1 = {F[1], F[3], F[5]};
  float n0 = norm(c0), n1 = norm(c1);
  V3 u1 = n0 >= n1 ? c0 : c1;
  float nu = fmaxf(n0, n1);
  u1 = nu > 0.f ? (1.f / nu) * u1 : v3(1.f, 0.f, 0.f);
  int k = 0;
  float m = fabsf(u1.x);
  if (fabsf(u1.y) < m) { k = 1; m = fabsf(u1.y); }
  if (fabsf(u1.z) < m) { k = 2; }
  V3 e = {k == 0 ? 1.f : 0.f, k == 1 ? 1.f : 0.f, k == 2 ? 1.f : 0.f};
  V3 u2 = e - dot(u1, e) * u1;
  u2 = (1.f / norm(u2)) * u2;
  // right singular vectors: v1 along the dominant column's weights
  float v1x = n0 >= n1 ? 1.f : 0.f, v1y = 1.f - v1x;
  if (nu > 0.f) {
    float l = sqrtf(n0 * n0 + n1 * n1);
    v1x = dot(u1, c0) / l;
    v1y = dot(u1, c1) / l;
  }
  float v2x = -v1y, v2y = v1x;
  R[0] = u1.x * v1x + u2.x * v2x; R[1] = u1.x * v1y + u2.x * v2y;
  R[2] = u1.y * v1x + u2.y * v2x; R[3] = u1.y * v1y + u2.y * v2y;
  R[4] = u1.z * v1x + u2.z * v2x; R[5] = u1.z * v1y + u2.z * v2y;
}

// Closest rotation (det +1) to the 3x3 F (row-major): Jacobi eigenvectors of
// F^T F give the two dominant right singular vectors v1, v2; then
// R = u1 v1^T + u2 v2^T + (u1 x u2)(v1 x v2)^T, which equals
// U diag(1, 1, det(U V^T)) V^T.
__device__ __forceinline__ void closest_rot33_jacobi(const float *F, float *R);

// Closest rotation to a 3x3 F.  For a well-conditioned F with det F > 0
// the closest rotation is the orthogonal polar factor, reached by the
// scaled Newton iteration X <- (z X + X^-T / z) / 2 from X = F (Higham's
// polar iteration: quadratic convergence, (1,F)-norm scaling
// z = sqrt(|X^-1|_F / |X|_F) in the first two steps); at most six steps
// take a strain of tens of percent to FP32 precision with about a third of
// the operations of the Jacobi eigen-decomposition.  From the third step on
// the iteration stops once no entry moved by more than 5e-7 (four ulps of
// a rotation's entries): the iterate is then at the rounding level, where a
// further step only moves it within that noise.  Nearly singular or
// inverted F (det F <= 1e-2 (|F|_F / sqrt 3)^3) take the Jacobi path,
// which handles rank deficiency and reflections.
__device__ __forceinline__ void closest_rot33(const float *F, float *R) {
  float X[9];
#pragma unroll
  for (int t = 0; t < 9; t++) X[t] = F[t];
  const float fn2 = X[0] * X[0] + X[1] * X[1] + X[2] * X[2] + X[3] * X[3] + X[4] * X[4] + X[5] * X[5] + X[6] * X[6] +
                    X[7] * X[7] + X[8] * X[8];
  const float c0 = X[4] * X[8] - X[5] * X[7], c1 = X[5] * X[6] - X[3] * X[8], c2 = X[3] * X[7] - X[4] * X[6];
  const float det0 = X[0] * c0 + X[1] * c1 + X[2] * c2;
  const float ref = fn2 * (1.f / 3.f);
  if (!(det0 > 1e-2f * ref * sqrtf(ref))) {
    closest_rot33_jacobi(F, R);
    return;
  }
#pragma unroll
  for (int it = 0; it < 6; it++) {
    // Y = X^-T = cof(X) / det X
    float Y[9];
    Y[0] = X[4] * X[8] - X[5] * X[7];
    Y[1] = X[5] * X[6] - X[3] * X[8];
    Y[2] = X[3] * X[7] - X[4] * X[6];
    Y[3] = X[2] * X[7] - X[1] * X[8];
    Y[4] = X[0] * X[8] - X[2] * X[6];
    Y[5] = X[1] * X[6] - X[0] * X[7];
    Y[6] = X[1] * X[5] - X[2] * X[4];
    Y[7] = X[2] * X[3] - X[0] * X[5];
    Y[8] = X[0] * X[4] - X[1] * X[3];
    const float inv_det = 1.f / (X[0] * Y[0] + X[1] * Y[1] + X[2] * Y[2]);
#pragma unroll
    for (int t = 0; t < 9; t++) Y[t] *= inv_det;
    float a = 0.5f, b = 0.5f;
    if (it < 2) {
      float nx = 0.f, ny = 0.f;
#pragma unroll
      for (int t = 0; t < 9; t++) {
        nx += X[t] * X[t];
        ny += Y[t] * Y[t];
      }
      const float z = sqrtf(sqrtf(ny / nx));   // sqrt(|X^-1|_F / |X|_F)
      a = 0.5f * z;
      b = 0.5f / z;
    }
    float dmax = 0.f;
#pragma unroll
    for (int t = 0; t < 9; t++) {
      const float xn = a * X[t] + b * Y[t];
      dmax = fmaxf(dmax, fabsf(xn - X[t]));
      X[t] = xn;
    }
    if (it >= 2 && dmax <= 5e-7f) break;
  }
#pragma unroll
  for (int t = 0; t < 9; t++) R[t] = X[t];
}

__device__ __forceinline__ void closest_rot33_jacobi(const float *F, float *R) {
  float C[3][3];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) C[i][j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
  float V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  // fully unrolled: every index is a constant, so C and V stay in registers
#pragma unroll
  for (int sweep = 0; sweep < 6; sweep++) {
#pragma unroll
    for (int pq = 0; pq < 3; pq++) {
      int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      float apq = C[p][q];
      if (fabsf(apq) < 1e-30f) continue;
      float theta = (C[q][q] - C[p][p]) / (2.f * apq);
      float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
      float c = rsqrtf(t * t + 1.f), s = t * c;
      for (int k = 0; k < 3; k++) {  // C <- C J  (columns p, q)
        float ckp = C[k][p], ckq = C[k][q];
        C[k][p] = c * ckp - s * ckq;
        C[k][q] = s * ckp + c * ckq;
      }
      for (int k = 0; k < 3; k++) {  // C <- J^T C (rows p, q)
        float cpk = C[p][k], cqk = C[q][k];
        C[p][k] = c * cpk - s * cqk;
        C[q][k] = s * cpk + c * cqk;
      }
      for (int k = 0; k < 3; k++) {
        float vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
      }
    }
  }
  // order eigenvalues descending
  int i0 = 0, i1 = 1, i2 = 2;
  float e0 = C[0][0], e1 = C[1][1], e2 = C[2][2];
  if (e1 > e0) { int t = i0; i0 = i1; i1 = t; float x = e0; e0 = e1; e1 = x; }
  if (e2 > e0) { int t = i0; i0 = i2; i2 = t; float x = e0; e0 = e2; e2 = x; }
  if (e2 > e1) { int t = i1; i1 = i2; i2 = t; }
  V3 v1 = {V[0][i0], V[1][i0], V[2][i0]}, v2 = {V[0][i1], V[1][i1], V[2][i1]};
  v2 = v2 - dot(v1, v2) * v1;
  v2 = (1.f / norm(v2)) * v2;
  V3 Fv1 = {F[0] * v1.x + F[1] * v1.y + F[2] * v1.z, F[3] * v1.x + F[4] * v1.y + F[5] * v1.z,
            F[6] * v1.x + F[7] * v1.y + F[8] * v1.z};
  V3 Fv2 = {F[0] * v2.x + F[1] * v2.y + F[2] * v2.z, F[3] * v2.x + F[4] * v2.y + F[5] * v2.z,
            F[6] * v2.x + F[7] * v2.y + F[8] * v2.z};
  float n1 = norm(Fv1);
  V3 u1 = n1 > 1e-20f ? (1.f / n1) * Fv1 : v1;
  V3 u2 = Fv2 - dot(u1, Fv2) * u1;
  float n2 = norm(u2);
  if (n2 > 1e-12f * fmaxf(n1, 1e-30f)) {
    u2 = (1.f / n2) * u2;
  } else {  // rank <= 1: complete with the least-aligned axis
    int k = 0;
    float m = fabsf(u1.x);
    if (fabsf(u1.y) < m) { k = 1; m = fabsf(u1.y); }
    if (fabsf(u1.z) < m) { k = 2; }
    V3 e = {k == 0 ? 1.f : 0.f, k == 1 ? 1.f : 0.f, k == 2 ? 1.f : 0.f};
    u2 = e - dot(u1, e) * u1;
    u2 = (1.f / norm(u2)) * u2;
  }
  V3 u3 = cross(u1, u2), v3_ = cross(v1, v2);
  const float uu[3][3] = {{u1.x, u2.x, u3.x}, {u1.y, u2.y, u3.y}, {u1.z, u2.z, u3.z}};
  const float vv[3][3] = {{v1.x, v2.x, v3_.x}, {v1.y, v2.y, v3_.y}, {v1.z, v2.z, v3_.z}};
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) R[3 * i + j] = uu[i][0] * vv[j][0] + uu[i][1] * vv[j][1] + uu[i][2] * vv[j][2];
}

// Per-contact linearisation of phi at (x, gamma) -- contact law readings:
//   normal   phi_n = FB(a + alpha y_n, y_n),  a = sd - tau, y = gamma / m_v,
//            alpha = compliance * m_v / h^2 (Fischer-Burmeister)
//   friction phi_t = y_t - Proj_{|.| <= mu max(y_n, 0)}(y_t - s),
//            s = tangential slip relative to the obstacle's material point
// Output lin[24]: R rows n,t1,t2 (9) | phi (3) | DC: cn, Ct(2x2) (5) |
//                 Dy: dn, dtn(2), Dtt(2x2) (7)
struct ContactLin {
  float R[9], phi[3], cn, Ct[4], dn, dtn[2], Dtt[4];
  float gap;   // a = sd - tau at the linearisation point
};

// The contact law at a linearisation point (unit normal n with its tangent
// basis t1, t2; gap a; slip rel over the step; normal compliance comp; mass mv
// that scales the multipliers, y = gamma / mv).
__device__ __forceinline__ void contact_law(V3 n, V3 t1, V3 t2, float a, V3 rel, float comp, float mu, float h,
                                            float mv, const float *g, ContactLin &L) {
  L.R[0] = n.x; L.R[1] = n.y; L.R[2] = n.z;
  L.R[3] = t1.x; L.R[4] = t1.y; L.R[5] = t1.z;
  L.R[6] = t2.x; L.R[7] = t2.y; L.R[8] = t2.z;
  const float inv_m = 1.f / mv;
  L.gap = a;
  const float yn = g[0] * inv_m;
  const float alpha = comp * mv / (h * h);
  const float ae = a + alpha * yn;
  const float r = sqrtf(ae * ae + yn * yn);
  float ca, cy;
  if (r < 1e-12f) {
    ca = 0.29289321881345254f;
    cy = 0.29289321881345254f;
    L.phi[0] = ae + yn - r;
  } else if (yn == 0.f) {
    // no multiplier yet: r = |ae| exactly.  Taken apart so that a separated
    // row keeps phi = 0 and D_C = 0 exactly (its multiplier stays zero); the
    // approximate square root would leave 1 - ae / r at a rounding error,
    // enough for a multiplier of ~1e-15 whose cone of that radius then turns
    // the next iteration's friction towards the direction of rounding noise
    ca = ae > 0.f ? 0.f : 2.f;
    cy = 1.f;
    L.phi[0] = ae > 0.f ? 0.f : 2.f * ae;
  } else {
    const float ir = 1.f / r;
    ca = 1.f - ae * ir;
    cy = 1.f - yn * ir;
    L.phi[0] = ae + yn - r;
  }
  L.cn = ca;
  L.dn = ca * alpha + cy;
  const float s0 = dot(t1, rel), s1 = dot(t2, rel);
  const V3 gt = {g[1], g[2], g[3]};
  const float y0 = dot(t1, gt) * inv_m, y1 = dot(t2, gt) * inv_m;
  const float rad = mu * fmaxf(yn, 0.f);
  const float d0 = y0 - s0, d1 = y1 - s1;
  const float dn = sqrtf(d0 * d0 + d1 * d1);
  if (rad == 0.f) {
    L.phi[1] = y0; L.phi[2] = y1;
    L.Ct[0] = 0.f; L.Ct[1] = 0.f; L.Ct[2] = 0.f; L.Ct[3] = 0.f;
    L.dtn[0] = 0.f; L.dtn[1] = 0.f;
    L.Dtt[0] = 1.f; L.Dtt[1] = 0.f; L.Dtt[2] = 0.f; L.Dtt[3] = 1.f;
  } else if (dn <= rad) {
    L.phi[1] = s0; L.phi[2] = s1;
    L.Ct[0] = 1.f; L.Ct[1] = 0.f; L.Ct[2] = 0.f; L.Ct[3] = 1.f;
    L.dtn[0] = 0.f; L.dtn[1] = 0.f;
    L.Dtt[0] = 0.f; L.Dtt[1] = 0.f; L.Dtt[2] = 0.f; L.Dtt[3] = 0.f;
  } else {
    const float idn = 1.f / dn;
    const float h0 = d0 * idn, h1 = d1 * idn;
    L.phi[1] = y0 - rad * h0;
    L.phi[2] = y1 - rad * h1;
    const float k = rad * idn;
    const float P00 = 1.f - h0 * h0, P01 = -h0 * h1, P11 = 1.f - h1 * h1;
    L.Ct[0] = k * P00; L.Ct[1] = k * P01; L.Ct[2] = k * P01; L.Ct[3] = k * P11;
    L.Dtt[0] = 1.f - k * P00; L.Dtt[1] = -k * P01; L.Dtt[2] = -k * P01; L.Dtt[3] = 1.f - k * P11;
    if (yn > 0.f) { L.dtn[0] = -mu * h0; L.dtn[1] = -mu * h1; }
    else { L.dtn[0] = 0.f; L.dtn[1] = 0.f; }
  }
}

__device__ __forceinline__ void linearize_contact_m(int type, const float *dims, float comp, const PoseM &P, float tau,
                                                    float mu, float h, float mv, V3 x, V3 xt, const float *g,
                                                    ContactLin &L) {
  V3 n, t1, t2;
  const float sd = obstacle_sdf_m(type, dims, P, x, n);
  tangent_basis(n, t1, t2);
  // slip relative to the obstacle's material point over the step
  const V3 xo = {P.S[0] * x.x + P.S[1] * x.y + P.S[2] * x.z + P.s[0], P.S[3] * x.x + P.S[4] * x.y + P.S[5] * x.z + P.s[1],
                 P.S[6] * x.x + P.S[7] * x.y + P.S[8] * x.z + P.s[2]};
  contact_law(n, t1, t2, sd - tau, xo - xt, comp, mu, h, mv, g, L);
}

}  // namespace flash
