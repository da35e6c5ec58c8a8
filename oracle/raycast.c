/* FP64 CPU oracle for depth ray casting of the simulation state (appendix,
 * depth rendering: depth maps, instance segmentation masks and point clouds
 * ray cast directly from the simulated meshes and obstacles).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  The plain definition, by brute
 * force: every pixel's ray is tested against every triangle and every
 * obstacle, and the nearest hit in [z_near, z_far] is kept.  No acceleration
 * structure, no culling, no ordering beyond that definition.
 *
 * Camera: pinhole, pose = camera-to-world (p, qw, qx, qy, qz); camera axes
 * x right, y down, z along the view.  Pixel (u, v) (u the column) casts the
 * ray from the camera centre through image point (u + 1/2, v + 1/2):
 * d_cam = ((u + 1/2 - cx)/fx, (v + 1/2 - cy)/fy, 1), so the ray parameter t
 * of a hit is its depth (camera z).  All surfaces are two-sided.
 */
#include <math.h>
#include <string.h>

#include "oracle.h"

static double rc_dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void rc_cross(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
/* rotation matrix of the unit quaternion (w, x, y, z), row-major */
static void rc_quat_mat(const double *q, double *R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}
static void rc_mul(const double *R, const double *v, double *o) {
  for (int i = 0; i < 3; i++) o[i] = R[3 * i] * v[0] + R[3 * i + 1] * v[1] + R[3 * i + 2] * v[2];
}
static void rc_mul_t(const double *R, const double *v, double *o) {
  for (int i = 0; i < 3; i++) o[i] = R[i] * v[0] + R[3 + i] * v[1] + R[6 + i] * v[2];
}

/* Ray o + t d against triangle (a, b, c): solve o + t d = a + b1 (b - a) + b2 (c - a)
 * by Cramer's rule; inside when every barycentric coordinate is >= -dil. */
static int ray_triangle(const double *o, const double *d, const double *a, const double *b, const double *c,
                        double dil, double *t) {
  double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  double s[3] = {o[0] - a[0], o[1] - a[1], o[2] - a[2]};
  double p[3], qv[3];
  rc_cross(d, e2, p);
  double det = rc_dot(e1, p);
  if (fabs(det) <= 1e-300) return 0;
  double b1 = rc_dot(s, p) / det;
  rc_cross(s, e1, qv);
  double b2 = rc_dot(d, qv) / det;
  double b0 = 1.0 - b1 - b2;
  if (b0 < -dil || b1 < -dil || b2 < -dil) return 0;
  *t = rc_dot(e2, qv) / det;
  return 1;
}

/* Ray against obstacle k (plane through the pose origin with normal body +z,
 * sphere of radius dims[0], box of half extents dims); nearest t >= t_lo. */
static int ray_obstacle(int type, const double *dims, const double *pose, const double *o, const double *d,
                        double dil, double t_lo, double *t) {
  double R[9];
  rc_quat_mat(pose + 3, R);
  if (type == OR_PLANE) {
    double n[3] = {R[2], R[5], R[8]};
    double dn = rc_dot(n, d);
    if (fabs(dn) <= 1e-300) return 0;
    double w[3] = {pose[0] - o[0], pose[1] - o[1], pose[2] - o[2]};
    *t = rc_dot(n, w) / dn;
    return *t >= t_lo;
  }
  if (type == OR_SPHERE) {
    double r = dims[0] * (1.0 + dil);
    double oc[3] = {o[0] - pose[0], o[1] - pose[1], o[2] - pose[2]};
    double a = rc_dot(d, d), b = rc_dot(d, oc), c = rc_dot(oc, oc) - r * r;
    double disc = b * b - a * c;
    if (disc < 0) return 0;
    double sq = sqrt(disc);
    double t1 = (-b - sq) / a, t2 = (-b + sq) / a;
    if (t1 >= t_lo) { *t = t1; return 1; }
    if (t2 >= t_lo) { *t = t2; return 1; }
    return 0;
  }
  if (type == OR_BOX) {
    double hm = fmax(dims[0], fmax(dims[1], dims[2]));
    double w[3] = {o[0] - pose[0], o[1] - pose[1], o[2] - pose[2]};
    double ob[3], db[3];
    rc_mul_t(R, w, ob);
    rc_mul_t(R, d, db);
    double tmin = -INFINITY, tmax = INFINITY;
    for (int i = 0; i < 3; i++) {
      double h = dims[i] + dil * hm;
      if (fabs(db[i]) <= 1e-300) {
        if (fabs(ob[i]) > h) return 0;
        continue;
      }
      double ta = (-h - ob[i]) / db[i], tb = (h - ob[i]) / db[i];
      if (ta > tb) { double x = ta; ta = tb; tb = x; }
      if (ta > tmin) tmin = ta;
      if (tb < tmax) tmax = tb;
    }
    if (tmin > tmax) return 0;
    if (tmin >= t_lo) { *t = tmin; return 1; }
    if (tmax >= t_lo) { *t = tmax; return 1; }
    return 0;
  }
  return 0;
}

/* the nearest hit of pixel (u, v) */
static void cast_pixel(const double *x, int T, const int *tris, int K, const int *otype, const double *odims,
                       const double *opose, const double *cam, const double *Rc, const double *intr, int u, int v,
                       double dil, double *depth, int *seg, double *pt) {
  const double fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3], zn = intr[4], zf = intr[5];
  const double dc[3] = {(u + 0.5 - cx) / fx, (v + 0.5 - cy) / fy, 1.0};
  double d[3];
  rc_mul(Rc, dc, d);
  double best = INFINITY;
  int inst = 0;
  /* triangles: instance 1, in index order (strict < keeps the smaller index) */
  for (int f = 0; f < T; f++) {
    double t;
    if (ray_triangle(cam, d, x + 3 * tris[3 * f], x + 3 * tris[3 * f + 1], x + 3 * tris[3 * f + 2], dil, &t) &&
        t >= zn && t <= zf && t < best) {
      best = t;
      inst = 1;
    }
  }
  /* obstacles: instance 2 + k; on a tie the smaller instance keeps the pixel */
  for (int k = 0; k < K; k++) {
    double t;
    if (otype[k] == 0) continue;
    if (ray_obstacle(otype[k], odims + 3 * k, opose + 7 * k, cam, d, dil, zn, &t) && t <= zf && t < best) {
      best = t;
      inst = 2 + k;
    }
  }
  if (inst) {
    *depth = best;
    *seg = inst;
    for (int c = 0; c < 3; c++) pt[c] = cam[c] + best * d[c];
  } else {
    *depth = 0.0;
    *seg = 0;
    for (int c = 0; c < 3; c++) pt[c] = NAN;
  }
}

void or_raycast(int n, const double *x, int T, const int *tris, int K, const int *otype, const double *odims,
                const double *opose, const double *cam, const double *intr, int W, int H, double dil,
                double *depth, int *seg, double *pts) {
  (void)n;
  double Rc[9];
  rc_quat_mat(cam + 3, Rc);
  for (int v = 0; v < H; v++)
    for (int u = 0; u < W; u++) {
      const size_t p = (size_t)v * W + u;
      cast_pixel(x, T, tris, K, otype, odims, opose, cam, Rc, intr, u, v, dil, depth + p, seg + p, pts + 3 * p);
    }
}

void or_raycast_pixels(int n, const double *x, int T, const int *tris, int K, const int *otype,
                       const double *odims, const double *opose, const double *cam, const double *intr, int npix,
                       const int *uv, double dil, double *depth, int *seg, double *pts) {
  (void)n;
  double Rc[9];
  rc_quat_mat(cam + 3, Rc);
  for (int i = 0; i < npix; i++)
    cast_pixel(x, T, tris, K, otype, odims, opose, cam, Rc, intr, uv[2 * i], uv[2 * i + 1], dil, depth + i,
               seg + i, pts + 3 * i);
}
