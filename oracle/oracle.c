/* FP64 CPU oracle for the batched FLASH time step (arxiv 2604.17513).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline arm, never by the product path.  Plain, slow and
 * written to be checked against the paper by eye: dense matrices, textbook
 * Cholesky, one-sided Jacobi SVD, Gaussian elimination with partial pivoting.
 * Shares no code with the CUDA library.
 *
 * Parity status per function (pins live in tests/test_oracle_*.py):
 *   closest rotation ........ pinned (rest shape, rotation equivariance, SVD identity)
 *   system matrix / solve ... pinned (residual of A x = b, SPD, null space of G)
 *   local-global energy ..... pinned (monotone decrease without contact)
 *   free fall / rest ........ pinned (closed forms of implicit Euler)
 *   normal contact .......... pinned (resting particle: gamma_n = m g h^2)
 *   Coulomb friction ........ pinned (incline stick/slide vs tan(theta) <= mu)
 *   complementarity ......... pinned (lambda >= 0, gap >= 0, cone, at Mode-B convergence)
 *   brute force ............. pinned (2^C active-set enumeration, frictionless)
 *   lite vs full metric ..... pinned (same converged fixed point)
 *   Mode-A iterates ......... parity unpinned: the paper prints no iterate values
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_DAMP 1e-6

/* ------------------------------------------------------------------------ */
/* small helpers                                                            */
/* ------------------------------------------------------------------------ */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* rotate v by unit quaternion (w, x, y, z): v' = q v q* */
static void quat_rot(const double *q, const double *v, double *out) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                 2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                 2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
  for (int i = 0; i < 3; i++) out[i] = R[3 * i] * v[0] + R[3 * i + 1] * v[1] + R[3 * i + 2] * v[2];
}
static void quat_rot_inv(const double *q, const double *v, double *out) {
  double qc[4] = {q[0], -q[1], -q[2], -q[3]};
  quat_rot(qc, v, out);
}
/* world point -> body frame of pose (p, quat) */
static void to_body(const double *pose, const double *x, double *pb) {
  double d[3] = {x[0] - pose[0], x[1] - pose[1], x[2] - pose[2]};
  quat_rot_inv(pose + 3, d, pb);
}
static void to_world(const double *pose, const double *pb, double *x) {
  quat_rot(pose + 3, pb, x);
  for (int i = 0; i < 3; i++) x[i] += pose[i];
}

/* ------------------------------------------------------------------------ */
/* mesh and system matrix  (Sec. III-B: A = M + h^2 sum w_i G_i^T G_i)       */
/* ------------------------------------------------------------------------ */
struct OrMesh {
  int type, n, ne, nh;
  double h, w_bend;
  double *mass;  /* [n] */
  int *elems;    /* [ne][3|4] */
  double *D;     /* [ne][4][3]: F[c][j] = sum_a x[v_a][c] D[a][j] */
  double *w;     /* [ne] element weight = w_stretch * rest area|volume */
  int *hv;       /* [nh][4] hinge vertices (edge x0 x1, opposite x2 x3) */
  double *hk;    /* [nh][4] hinge stencil k */
  double *hs;    /* [nh] hinge scale 3 / (A0 + A1) */
  double *A;     /* [n][n] dense system matrix (scalar block, A = A_s (x) I3) */
  double *L;     /* [n][n] Cholesky factor, lower */
  double *Adiag; /* [n] diagonal of A^-1 (computed on first use) */
  int ned;       /* triangle meshes: unique edges (a < b), sorted by (a, b) */
  int *ed;       /* [ned][2] */
};

static int ncols(const OrMesh *m) { return m->type == OR_TRI ? 2 : 3; }
static int nvpe(const OrMesh *m) { return m->type == OR_TRI ? 3 : 4; }

/* 2x2 / 3x3 inverse */
static void inv2(const double *a, double *o) {
  double det = a[0] * a[3] - a[1] * a[2];
  o[0] = a[3] / det; o[1] = -a[1] / det; o[2] = -a[2] / det; o[3] = a[0] / det;
}
static double det3(const double *a) {
  return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
         a[2] * (a[3] * a[7] - a[4] * a[6]);
}
static void inv3(const double *a, double *o) {
  double d = det3(a);
  o[0] = (a[4] * a[8] - a[5] * a[7]) / d; o[1] = (a[2] * a[7] - a[1] * a[8]) / d;
  o[2] = (a[1] * a[5] - a[2] * a[4]) / d; o[3] = (a[5] * a[6] - a[3] * a[8]) / d;
  o[4] = (a[0] * a[8] - a[2] * a[6]) / d; o[5] = (a[2] * a[3] - a[0] * a[5]) / d;
  o[6] = (a[3] * a[7] - a[4] * a[6]) / d; o[7] = (a[1] * a[6] - a[0] * a[7]) / d;
  o[8] = (a[0] * a[4] - a[1] * a[3]) / d;
}

/* Triangle: rest edges expressed in the triangle's own 2D frame give Dm (2x2);
 * F = Ds Dm^-1 with Ds = [x1-x0, x2-x0].  Tet: Dm = [X1-X0, X2-X0, X3-X0]. */
static void build_element(OrMesh *m, int e, const double *rest) {
  const int *v = m->elems + e * nvpe(m);
  double *D = m->D + e * 12;
  memset(D, 0, 12 * sizeof(double));
  if (m->type == OR_TRI) {
    double e1[3], e2[3], nn[3], u[3], wv[3];
    for (int c = 0; c < 3; c++) {
      e1[c] = rest[3 * v[1] + c] - rest[3 * v[0] + c];
      e2[c] = rest[3 * v[2] + c] - rest[3 * v[0] + c];
    }
    cross3(e1, e2, nn);
    double area = 0.5 * norm3(nn);
    double l1 = norm3(e1);
    for (int c = 0; c < 3; c++) u[c] = e1[c] / l1;
    double nl = norm3(nn);
    for (int c = 0; c < 3; c++) nn[c] /= nl;
    cross3(nn, u, wv);
    double Dm[4] = {dot3(e1, u), dot3(e2, u), dot3(e1, wv), dot3(e2, wv)}, Di[4];
    inv2(Dm, Di);
    /* D = [[-1,-1],[1,0],[0,1]] * Dm^-1 */
    for (int j = 0; j < 2; j++) {
      D[0 * 3 + j] = -Di[0 * 2 + j] - Di[1 * 2 + j];
      D[1 * 3 + j] = Di[0 * 2 + j];
      D[2 * 3 + j] = Di[1 * 2 + j];
    }
    m->w[e] *= area;
  } else {
    double Dm[9], Di[9];
    for (int c = 0; c < 3; c++)
      for (int j = 0; j < 3; j++) Dm[3 * c + j] = rest[3 * v[j + 1] + c] - rest[3 * v[0] + c];
    double vol = fabs(det3(Dm)) / 6.0;
    inv3(Dm, Di);
    for (int j = 0; j < 3; j++) {
      D[0 * 3 + j] = -Di[0 * 3 + j] - Di[1 * 3 + j] - Di[2 * 3 + j];
      for (int a = 1; a < 4; a++) D[a * 3 + j] = Di[(a - 1) * 3 + j];
    }
    m->w[e] *= vol;
  }
}

/* Quadratic flat-rest bending on interior edges (reading: the paper gives only a
 * scalar bending weight).  For edge (x0,x1) with opposite vertices x2, x3 the
 * stencil k annihilates constants and the rest positions (so flat rest shapes
 * carry no bending energy); k2 = |e|/h2, k3 = |e|/h3 with h2, h3 the heights of
 * the opposite vertices over the edge.  Energy (w_b/2) * 3/(A0+A1) * |sum k_i x_i|^2. */
static int cmp_edge(const void *a, const void *b) {
  const int *x = (const int *)a, *y = (const int *)b;
  if (x[0] != y[0]) return x[0] - y[0];
  if (x[1] != y[1]) return x[1] - y[1];
  return x[2] - y[2];
}
static void build_hinges(OrMesh *m, const double *rest) {
  m->nh = 0;
  if (m->type != OR_TRI || m->ne == 0) return;
  size_t ne3 = (size_t)3 * (size_t)m->ne;
  int *ed = (int *)malloc(sizeof(int) * 4 * ne3); /* (lo, hi, tri, opposite) */
  for (int t = 0; t < m->ne; t++) {
    const int *v = m->elems + 3 * t;
    for (int k = 0; k < 3; k++) {
      int a = v[k], b = v[(k + 1) % 3], o = v[(k + 2) % 3];
      int *r = ed + 4 * (3 * t + k);
      r[0] = a < b ? a : b; r[1] = a < b ? b : a; r[2] = t; r[3] = o;
    }
  }
  qsort(ed, ne3, 4 * sizeof(int), cmp_edge);
  m->hv = (int *)malloc(sizeof(int) * 4 * ne3);
  m->hk = (double *)malloc(sizeof(double) * 4 * ne3);
  m->hs = (double *)malloc(sizeof(double) * ne3);
  for (size_t i = 0; i + 1 < ne3; i++) {
    int *r0 = ed + 4 * i, *r1 = ed + 4 * (i + 1);
    if (r0[0] != r1[0] || r0[1] != r1[1]) continue;
    int x[4] = {r0[0], r0[1], r0[3], r1[3]};
    const double *X0 = rest + 3 * x[0], *X1 = rest + 3 * x[1], *X2 = rest + 3 * x[2], *X3 = rest + 3 * x[3];
    double e[3], d2[3], d3[3], c2[3], c3[3];
    for (int c = 0; c < 3; c++) { e[c] = X1[c] - X0[c]; d2[c] = X2[c] - X0[c]; d3[c] = X3[c] - X0[c]; }
    double le = norm3(e);
    cross3(e, d2, c2); cross3(e, d3, c3);
    double A0 = 0.5 * norm3(c2), A1 = 0.5 * norm3(c3);
    double h2 = 2 * A0 / le, h3 = 2 * A1 / le;
    double k2 = le / h2, k3 = le / h3;
    double s2 = dot3(d2, e) / le, s3 = dot3(d3, e) / le;
    double k1 = -(k2 * s2 + k3 * s3) / le;
    double k0 = -(k1 + k2 + k3);
    int h = m->nh++;
    memcpy(m->hv + 4 * h, x, sizeof x);
    m->hk[4 * h + 0] = k0; m->hk[4 * h + 1] = k1; m->hk[4 * h + 2] = k2; m->hk[4 * h + 3] = k3;
    m->hs[h] = 3.0 / (A0 + A1);
    i++;
  }
  free(ed);
}

/* textbook dense Cholesky A = L L^T (lower), returns 0 on success */
static int cholesky(int n, const double *A, double *L) {
  memset(L, 0, sizeof(double) * (size_t)n * n);
  for (int j = 0; j < n; j++) {
    double s = A[(size_t)j * n + j];
    for (int k = 0; k < j; k++) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (s <= 0) return -1;
    double d = sqrt(s);
    L[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; i++) {
      double t = A[(size_t)i * n + j];
      for (int k = 0; k < j; k++) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = t / d;
    }
  }
  return 0;
}

static int edge_cmp(const void *x, const void *y) {
  const int *a = (const int *)x, *b = (const int *)y;
  return a[0] != b[0] ? (a[0] > b[0]) - (a[0] < b[0]) : (a[1] > b[1]) - (a[1] < b[1]);
}

/* unique edges of a triangle mesh, (a < b), sorted */
static void build_edges(OrMesh *m) {
  m->ned = 0;
  m->ed = NULL;
  if (m->type != OR_TRI || m->ne == 0) return;
  int *all = (int *)malloc(sizeof(int) * 6 * m->ne);
  for (int e = 0; e < m->ne; e++)
    for (int k = 0; k < 3; k++) {
      int a = m->elems[3 * e + k], b = m->elems[3 * e + (k + 1) % 3];
      all[6 * e + 2 * k] = a < b ? a : b;
      all[6 * e + 2 * k + 1] = a < b ? b : a;
    }
  qsort(all, 3 * m->ne, 2 * sizeof(int), edge_cmp);
  m->ed = (int *)malloc(sizeof(int) * 6 * m->ne);
  for (int k = 0; k < 3 * m->ne; k++)
    if (k == 0 || all[2 * k] != all[2 * k - 2] || all[2 * k + 1] != all[2 * k - 1]) {
      m->ed[2 * m->ned] = all[2 * k];
      m->ed[2 * m->ned + 1] = all[2 * k + 1];
      m->ned++;
    }
  free(all);
}

OrMesh *or_mesh_new(int type, int n, const double *rest, int ne, const int *elems,
                    const double *mass, double w_stretch, double w_bend, double h) {
  OrMesh *m = (OrMesh *)calloc(1, sizeof(OrMesh));
  m->type = type; m->n = n; m->ne = ne; m->h = h; m->w_bend = w_bend;
  int vp = type == OR_TRI ? 3 : 4;
  m->mass = (double *)malloc(sizeof(double) * n);
  memcpy(m->mass, mass, sizeof(double) * n);
  m->elems = (int *)malloc(sizeof(int) * vp * (ne > 0 ? ne : 1));
  if (ne) memcpy(m->elems, elems, sizeof(int) * vp * ne);
  m->D = (double *)malloc(sizeof(double) * 12 * (ne > 0 ? ne : 1));
  m->w = (double *)malloc(sizeof(double) * (ne > 0 ? ne : 1));
  for (int e = 0; e < ne; e++) { m->w[e] = w_stretch; build_element(m, e, rest); }
  build_hinges(m, rest);
  if (w_bend == 0.0) m->nh = 0;
  build_edges(m);
  /* assemble A (scalar n x n) */
  m->A = (double *)calloc((size_t)n * n, sizeof(double));
  m->L = (double *)malloc(sizeof(double) * (size_t)n * n);
  for (int i = 0; i < n; i++) m->A[(size_t)i * n + i] = mass[i];
  int nc = ncols(m);
  for (int e = 0; e < ne; e++) {
    const int *v = m->elems + e * vp;
    const double *D = m->D + e * 12;
    for (int a = 0; a < vp; a++)
      for (int b = 0; b < vp; b++) {
        double s = 0;
        for (int j = 0; j < nc; j++) s += D[a * 3 + j] * D[b * 3 + j];
        m->A[(size_t)v[a] * n + v[b]] += h * h * m->w[e] * s;
      }
  }
  for (int k = 0; k < m->nh; k++) {
    const int *v = m->hv + 4 * k;
    const double *kk = m->hk + 4 * k;
    for (int a = 0; a < 4; a++)
      for (int b = 0; b < 4; b++) m->A[(size_t)v[a] * n + v[b]] += h * h * w_bend * m->hs[k] * kk[a] * kk[b];
  }
  if (cholesky(n, m->A, m->L) != 0) { or_mesh_free(m); return NULL; }
  return m;
}

void or_mesh_free(OrMesh *m) {
  if (!m) return;
  free(m->ed);
  free(m->mass); free(m->elems); free(m->D); free(m->w);
  free(m->hv); free(m->hk); free(m->hs); free(m->A); free(m->L); free(m->Adiag);
  free(m);
}
int or_mesh_hinges(const OrMesh *m) { return m->nh; }
int or_mesh_edges(const OrMesh *m, int *out) {
  if (out && m->ned) memcpy(out, m->ed, sizeof(int) * 2 * m->ned);
  return m->ned;
}
void or_mesh_matrix(const OrMesh *m, double *A_out) { memcpy(A_out, m->A, sizeof(double) * (size_t)m->n * m->n); }

/* A^-1 rhs via the Cholesky factor, per coordinate (A = A_s (x) I3) */
void or_solve(const OrMesh *m, const double *rhs, double *out) {
  int n = m->n;
  double *y = (double *)malloc(sizeof(double) * n);
  for (int c = 0; c < 3; c++) {
    for (int i = 0; i < n; i++) {
      double s = rhs[3 * i + c];
      for (int k = 0; k < i; k++) s -= m->L[(size_t)i * n + k] * y[k];
      y[i] = s / m->L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
      double s = y[i];
      for (int k = i + 1; k < n; k++) s -= m->L[(size_t)k * n + i] * out[3 * k + c];
      out[3 * i + c] = s / m->L[(size_t)i * n + i];
    }
  }
  free(y);
}

/* ------------------------------------------------------------------------ */
/* local step: closest rotation (Eq. internal, zeta_i = indicator of SO(3) / */
/* of 3x2 matrices with orthonormal columns)                               */
/* ------------------------------------------------------------------------ */
/* One-sided Jacobi SVD of the 3 x c matrix F (c = 2 or 3): returns U (3 x c,
 * columns), sigma (descending) and V (c x c) with F = U diag(sigma) V^T. */
static void jacobi_svd(int c, const double *F, double *U, double *sig, double *V) {
  double W[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < c; j++) W[3 * j + i] = F[c * i + j]; /* W column-major: column j */
  double Vc[9] = {0};
  for (int j = 0; j < c; j++) Vc[c * j + j] = 1.0;           /* Vc column-major c x c */
  for (int sweep = 0; sweep < 60; sweep++) {
    double off = 0;
    for (int p = 0; p < c - 1; p++)
      for (int q = p + 1; q < c; q++) {
        double al = dot3(W + 3 * p, W + 3 * p), be = dot3(W + 3 * q, W + 3 * q), ga = dot3(W + 3 * p, W + 3 * q);
        if (fabs(ga) <= 1e-300 || fabs(ga) <= 1e-17 * sqrt(al * be)) continue;
        off = fmax(off, fabs(ga) / sqrt(al * be));
        double ze = (be - al) / (2 * ga);
        double t = (ze >= 0 ? 1.0 : -1.0) / (fabs(ze) + sqrt(1 + ze * ze));
        double cs = 1 / sqrt(1 + t * t), sn = cs * t;
        for (int i = 0; i < 3; i++) {
          double a = W[3 * p + i], b = W[3 * q + i];
          W[3 * p + i] = cs * a - sn * b; W[3 * q + i] = sn * a + cs * b;
        }
        for (int i = 0; i < c; i++) {
          double a = Vc[c * p + i], b = Vc[c * q + i];
          Vc[c * p + i] = cs * a - sn * b; Vc[c * q + i] = sn * a + cs * b;
        }
      }
    if (off < 1e-16) break;
  }
  int ord[3] = {0, 1, 2};
  double s[3];
  for (int j = 0; j < c; j++) s[j] = norm3(W + 3 * j);
  for (int a = 0; a < c; a++)
    for (int b = a + 1; b < c; b++)
      if (s[ord[b]] > s[ord[a]]) { int t = ord[a]; ord[a] = ord[b]; ord[b] = t; }
  for (int j = 0; j < c; j++) {
    int o = ord[j];
    sig[j] = s[o];
    for (int i = 0; i < 3; i++) U[3 * j + i] = s[o] > 1e-300 ? W[3 * o + i] / s[o] : 0.0;
    for (int i = 0; i < c; i++) V[c * j + i] = Vc[c * o + i];
  }
}

/* unit vector orthogonal to u: the coordinate axis least aligned with u,
 * made orthogonal (reading: deterministic completion of a rank-deficient F) */
static void complete_axis(const double *u, double *out) {
  int k = 0;
  for (int i = 1; i < 3; i++) if (fabs(u[i]) < fabs(u[k])) k = i;
  double e[3] = {0, 0, 0};
  e[k] = 1;
  double d = dot3(u, e);
  for (int i = 0; i < 3; i++) out[i] = e[i] - d * u[i];
  double l = norm3(out);
  for (int i = 0; i < 3; i++) out[i] /= l;
}

/* R = argmin ||R - F||_F over 3x2 matrices with orthonormal columns (cols=2)
 * or over SO(3) (cols=3): R = U diag(1,..,det(U V^T)) V^T */
void or_closest_rotation(int cols, const double *F, double *R) {
  double U[9], sg[3], V[9];
  jacobi_svd(cols, F, U, sg, V);
  double tiny = 1e-12 * (sg[0] > 0 ? sg[0] : 1.0);
  if (sg[0] <= 1e-300) { U[0] = 1; U[1] = 0; U[2] = 0; }
  if (sg[1] <= tiny) complete_axis(U, U + 3);
  if (cols == 3) {
    if (sg[2] <= tiny) cross3(U, U + 3, U + 6);
    double Um[9];
    for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) Um[3 * i + j] = U[3 * j + i];
    double Vm[9];
    for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) Vm[3 * i + j] = V[3 * j + i];
    double d = det3(Um) * det3(Vm);
    for (int i = 0; i < 3; i++) U[6 + i] *= (d < 0 ? -1.0 : 1.0);
  }
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < cols; j++) {
      double s = 0;
      for (int k = 0; k < cols; k++) s += U[3 * k + i] * V[cols * k + j];
      R[cols * i + j] = s;
    }
}

static void element_F(const OrMesh *m, int e, const double *q, double *F) {
  int vp = nvpe(m), nc = ncols(m);
  const int *v = m->elems + e * vp;
  const double *D = m->D + e * 12;
  for (int c = 0; c < 3; c++)
    for (int j = 0; j < nc; j++) {
      double s = 0;
      for (int a = 0; a < vp; a++) s += q[3 * v[a] + c] * D[a * 3 + j];
      F[nc * c + j] = s;
    }
}

void or_project(const OrMesh *m, const double *q, double *p) {
  for (int e = 0; e < m->ne; e++) {
    double F[9];
    element_F(m, e, q, F);
    or_closest_rotation(ncols(m), F, p + 9 * e);
  }
}

/* b = M q~ + h^2 sum_i w_i G_i^T p_i   (Sec. III-B) */
void or_assemble_b(const OrMesh *m, const double *qt, const double *p, double *b) {
  int n = m->n, vp = nvpe(m), nc = ncols(m);
  double h2 = m->h * m->h;
  for (int i = 0; i < n; i++)
    for (int c = 0; c < 3; c++) b[3 * i + c] = m->mass[i] * qt[3 * i + c];
  for (int e = 0; e < m->ne; e++) {
    const int *v = m->elems + e * vp;
    const double *D = m->D + e * 12, *P = p + 9 * e;
    for (int a = 0; a < vp; a++)
      for (int c = 0; c < 3; c++) {
        double s = 0;
        for (int j = 0; j < nc; j++) s += D[a * 3 + j] * P[nc * c + j];
        b[3 * v[a] + c] += h2 * m->w[e] * s;
      }
  }
}

/* E(q,p) = 1/(2h^2) |M^1/2 (q - q~)|^2 + sum w_i/2 |G_i q - p_i|^2 + bending (Eq. implicit) */
double or_pd_energy(const OrMesh *m, const double *q, const double *qt, const double *p) {
  double E = 0, h2 = m->h * m->h;
  int nc = ncols(m);
  for (int i = 0; i < m->n; i++)
    for (int c = 0; c < 3; c++) {
      double d = q[3 * i + c] - qt[3 * i + c];
      E += 0.5 / h2 * m->mass[i] * d * d;
    }
  for (int e = 0; e < m->ne; e++) {
    double F[9];
    element_F(m, e, q, F);
    double s = 0;
    for (int k = 0; k < 3 * nc; k++) s += (F[k] - p[9 * e + k]) * (F[k] - p[9 * e + k]);
    E += 0.5 * m->w[e] * s;
  }
  for (int k = 0; k < m->nh; k++)
    for (int c = 0; c < 3; c++) {
      double s = 0;
      for (int a = 0; a < 4; a++) s += m->hk[4 * k + a] * q[3 * m->hv[4 * k + a] + c];
      E += 0.5 * m->w_bend * m->hs[k] * s * s;
    }
  return E;
}

/* ------------------------------------------------------------------------ */
/* obstacles and contact (Sec. III-A, Eq. lagrange; phi per the readings)   */
/* ------------------------------------------------------------------------ */
double or_sdf(int type, const double *dims, const double *pose, const double *x, double *nrm) {
  double p[3], nb[3] = {0, 0, 1}, sd = 0;
  to_body(pose, x, p);
  if (type == OR_PLANE) {
    sd = p[2];
  } else if (type == OR_SPHERE) {
    double d = norm3(p);
    if (d > 1e-12) for (int i = 0; i < 3; i++) nb[i] = p[i] / d;
    sd = d - dims[0];
  } else { /* box */
    double d[3], o[3], on = 0;
    int outside = 0;
    for (int i = 0; i < 3; i++) {
      d[i] = fabs(p[i]) - dims[i];
      o[i] = d[i] > 0 ? d[i] : 0;
      if (d[i] > 0) outside = 1;
      on += o[i] * o[i];
    }
    if (outside) {
      on = sqrt(on);
      for (int i = 0; i < 3; i++) nb[i] = (p[i] >= 0 ? 1.0 : -1.0) * o[i] / on;
      sd = on;
    } else {
      int ax = 0;
      for (int i = 1; i < 3; i++) if (d[i] > d[ax]) ax = i;
      nb[0] = nb[1] = nb[2] = 0;
      nb[ax] = p[ax] >= 0 ? 1.0 : -1.0;
      sd = d[ax];
    }
  }
  if (nrm) quat_rot(pose + 3, nb, nrm);
  return sd;
}

/* Duff et al. 2017 branchless orthonormal basis: rows t1, t2 orthogonal to n */
static void tangent_frame(const double *n, double *t1, double *t2) {
  double s = n[2] >= 0 ? 1.0 : -1.0;
  double a = -1.0 / (s + n[2]);
  double b = n[0] * n[1] * a;
  t1[0] = 1 + s * n[0] * n[0] * a; t1[1] = s * b; t1[2] = -s * n[0];
  t2[0] = b; t2[1] = s + n[1] * n[1] * a; t2[2] = -n[1];
}

double or_fb(double a, double b) { return a + b - sqrt(a * a + b * b); }

static int tri_plane(const double *a, const double *b, const double *c, const double *p, double *nh, double *d,
                     double *w);

/* triangles f and g share a vertex */
static int tri_touch(const int *f, const int *g) {
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      if (f[a] == g[b]) return 1;
  return 0;
}

/* Self-contact candidate (a reading): vertex p and triangle f of the same
 * cloth, f not touching any triangle incident to p (topological neighbours
 * are excluded), with p within tau + margin of f's plane and its projection
 * inside f up to OR_SELF_BARY in barycentric terms, at q_t or at q~. */
static int self_candidate(const OrMesh *m, double reach, int p, int f, const double *x0, const double *x1) {
  const int *t = m->elems + 3 * f;
  if (t[0] == p || t[1] == p || t[2] == p) return 0;
  int hit = 0;
  for (int k = 0; k < 2 && !hit; k++) {
    const double *x = k == 0 ? x0 : x1;
    double nh[3], d, w[3];
    if (!tri_plane(x + 3 * t[0], x + 3 * t[1], x + 3 * t[2], x + 3 * p, nh, &d, w)) continue;
    hit = fabs(d) < reach && w[0] >= -OR_SELF_BARY && w[1] >= -OR_SELF_BARY && w[2] >= -OR_SELF_BARY;
  }
  if (!hit) return 0;
  for (int g = 0; g < m->ne; g++) {
    const int *tg = m->elems + 3 * g;
    if ((tg[0] == p || tg[1] == p || tg[2] == p) && tri_touch(tg, t)) return 0;
  }
  return 1;
}

/* Closest points of the lines through segments (a, b) and (c, d): a + s (b -
 * a) and c + t (d - c); 0 if the lines are parallel to rounding. */
static int line_params(const double *a, const double *b, const double *c, const double *d, double *s, double *t) {
  double d1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, d2[3] = {d[0] - c[0], d[1] - c[1], d[2] - c[2]};
  double r[3] = {a[0] - c[0], a[1] - c[1], a[2] - c[2]};
  double A = dot3(d1, d1), B = dot3(d1, d2), C = dot3(d2, d2), D = dot3(d1, r), E = dot3(d2, r);
  double den = A * C - B * B;
  if (!(den > 1e-12 * A * C)) return 0;
  *s = (B * E - C * D) / den;
  *t = (A * E - B * D) / den;
  return 1;
}

/* Edge-edge candidate (a reading, like the vertex-triangle one): edges e1
 * = (a, b) and e2 = (c, d) of the same cloth, e2 touching no triangle of a
 * or b, whose lines' closest points lie inside both segments and within
 * reach of each other, at q_t or at q~. */
static int ee_candidate(const OrMesh *m, double reach, int e1, int e2, const double *x0, const double *x1) {
  const int a = m->ed[2 * e1], b = m->ed[2 * e1 + 1], c = m->ed[2 * e2], d = m->ed[2 * e2 + 1];
  if (a == c || a == d || b == c || b == d) return 0;
  int hit = 0;
  for (int k = 0; k < 2 && !hit; k++) {
    const double *x = k == 0 ? x0 : x1;
    double s, t;
    if (!line_params(x + 3 * a, x + 3 * b, x + 3 * c, x + 3 * d, &s, &t)) continue;
    if (!(s > 0 && s < 1 && t > 0 && t < 1)) continue;
    double dd[3];
    for (int i = 0; i < 3; i++)
      dd[i] = (1 - s) * x[3 * a + i] + s * x[3 * b + i] - (1 - t) * x[3 * c + i] - t * x[3 * d + i];
    hit = norm3(dd) < reach;
  }
  if (!hit) return 0;
  for (int g = 0; g < m->ne; g++) {
    const int *tg = m->elems + 3 * g;
    int has_ab = 0, has_cd = 0;
    for (int k = 0; k < 3; k++) {
      has_ab |= tg[k] == a || tg[k] == b;
      has_cd |= tg[k] == c || tg[k] == d;
    }
    if (has_ab && has_cd) return 0;
  }
  return 1;
}

/* Box corner k (0..7) in the box's frame: bit i of k set = +dims[i] on axis
 * i, clear = -dims[i] (dims are half extents). */
static void box_corner(const double *dims, int k, double *p) {
  for (int i = 0; i < 3; i++) p[i] = (k >> i & 1) ? dims[i] : -dims[i];
}

/* Box edge j (0..11) in the box's frame: along axis a = j / 4 from -dims[a]
 * to +dims[a], on the sides of the other two axes (b < c) given by bits 0
 * (b) and 1 (c) of j % 4. */
static void box_edge(const double *dims, int j, double *p0, double *p1) {
  const int a = j / 4, m = j % 4, b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
  p0[a] = -dims[a];
  p1[a] = dims[a];
  p0[b] = p1[b] = (m & 1) ? dims[b] : -dims[b];
  p0[c] = p1[c] = (m & 2) ? dims[c] : -dims[c];
}

/* Box-corner candidate (a reading, like the vertex-triangle self contact):
 * the corner C (at the obstacle's pose at t+h) within reach of triangle f's
 * plane with its projection inside f up to OR_SELF_BARY, at q_t or q~. */
static int ovt_candidate(const OrMesh *m, double reach, int f, const double *C, const double *x0, const double *x1) {
  const int *t = m->elems + 3 * f;
  for (int k = 0; k < 2; k++) {
    const double *x = k == 0 ? x0 : x1;
    double nh[3], d, w[3];
    if (!tri_plane(x + 3 * t[0], x + 3 * t[1], x + 3 * t[2], C, nh, &d, w)) continue;
    if (fabs(d) < reach && w[0] >= -OR_SELF_BARY && w[1] >= -OR_SELF_BARY && w[2] >= -OR_SELF_BARY) return 1;
  }
  return 0;
}

/* Box-edge candidate (a reading, like the edge-edge self contact): the box
 * edge (C, D) (at t+h) and the cloth edge e = (a, b), whose lines' closest
 * points lie inside both and nearer than reach, at q_t or q~. */
static int oee_candidate(const OrMesh *m, double reach, int e, const double *C, const double *D, const double *x0,
                         const double *x1) {
  const int a = m->ed[2 * e], b = m->ed[2 * e + 1];
  for (int k = 0; k < 2; k++) {
    const double *x = k == 0 ? x0 : x1;
    double s, t;
    if (!line_params(x + 3 * a, x + 3 * b, C, D, &s, &t)) continue;
    if (!(s > 0 && s < 1 && t > 0 && t < 1)) continue;
    double dd[3];
    for (int i = 0; i < 3; i++) dd[i] = (1 - s) * x[3 * a + i] + s * x[3 * b + i] - (1 - t) * C[i] - t * D[i];
    if (norm3(dd) < reach) return 1;
  }
  return 0;
}

int or_detect(const OrMesh *m, const double *dp, int K, const int *otype, const double *odims,
              const double *pose_th, const double *q, const double *v, const unsigned char *attached,
              int cap, int *cvert, int *cobs, int *ctri) {
  double h = dp[OR_DP_H], tau = dp[OR_DP_TAU], marg = dp[OR_DP_MARGIN];
  const int self = dp[OR_DP_SELF] != 0.0 && m->type == OR_TRI;
  const int ofeat = dp[OR_DP_OFEAT] != 0.0 && m->type == OR_TRI;
  double *xp = (double *)malloc(sizeof(double) * 3 * (m->n > 0 ? m->n : 1));
  for (int i = 0; i < m->n; i++)
    for (int c = 0; c < 3; c++) xp[3 * i + c] = q[3 * i + c] + h * v[3 * i + c] + h * h * dp[OR_DP_GX + c];
  int cnt = 0;
  for (int i = 0; i < m->n; i++) {
    for (int o = 0; o < K; o++) {
      if (otype[o] == 0) continue;
      double s0 = or_sdf(otype[o], odims + 3 * o, pose_th + 7 * o, q + 3 * i, NULL);
      double s1 = or_sdf(otype[o], odims + 3 * o, pose_th + 7 * o, xp + 3 * i, NULL);
      if (fmin(s0, s1) < tau + marg) {
        if (cnt < cap) { cvert[cnt] = i; cobs[cnt] = o; if (ctri) ctri[cnt] = -1; }
        cnt++;
      }
    }
    if (attached && attached[i]) {
      if (cnt < cap) { cvert[cnt] = i; cobs[cnt] = OR_GRASP_SLOT; if (ctri) ctri[cnt] = -1; }
      cnt++;
    }
    /* self contacts: the first OR_SELF_MAX candidate triangles in index order */
    for (int f = 0, ns = 0; self && f < m->ne && ns < OR_SELF_MAX; f++)
      if (self_candidate(m, tau + marg, i, f, q, xp)) {
        if (cnt < cap) { cvert[cnt] = i; cobs[cnt] = OR_SELF_SLOT; if (ctri) ctri[cnt] = f; }
        cnt++;
        ns++;
      }
    /* edge-edge contacts of the edges (i, b), b > i (in edge order), each
     * unordered pair once (e2 > e1: the pair (e2, e1) would be the same
     * constraint again): the first OR_EE_MAX candidate pairs, feature index
     * e1 * ned + e2 */
    int ne_i = 0;
    for (int e1 = 0; self && e1 < m->ned && ne_i < OR_EE_MAX; e1++) {
      if (m->ed[2 * e1] != i) continue;
      for (int e2 = e1 + 1; e2 < m->ned && ne_i < OR_EE_MAX; e2++)
        if (ee_candidate(m, tau + marg, e1, e2, q, xp)) {
          if (cnt < cap) { cvert[cnt] = i; cobs[cnt] = OR_EE_SLOT; if (ctri) ctri[cnt] = e1 * m->ned + e2; }
          cnt++;
          ne_i++;
        }
    }
    /* box features: corners against the triangles whose first vertex is i,
     * then box edges against the edges (i, b), each in feature order */
    int nc_i = 0;
    for (int f = 0; ofeat && f < m->ne && nc_i < OR_OFEAT_MAX; f++) {
      if (m->elems[3 * f] != i) continue;
      for (int o = 0; o < K && nc_i < OR_OFEAT_MAX; o++) {
        if (otype[o] != OR_BOX) continue;
        for (int kc = 0; kc < 8 && nc_i < OR_OFEAT_MAX; kc++) {
          double cb[3], C[3];
          box_corner(odims + 3 * o, kc, cb);
          to_world(pose_th + 7 * o, cb, C);
          if (ovt_candidate(m, tau + marg, f, C, q, xp)) {
            if (cnt < cap) { cvert[cnt] = i; cobs[cnt] = OR_OVT_SLOT; if (ctri) ctri[cnt] = (f * OR_MAX_OBS + o) * 8 + kc; }
            cnt++;
            nc_i++;
          }
        }
      }
    }
    int nb_i = 0;
    for (int e = 0; ofeat && e < m->ned && nb_i < OR_OFEAT_MAX; e++) {
      if (m->ed[2 * e] != i) continue;
      for (int o = 0; o < K && nb_i < OR_OFEAT_MAX; o++) {
        if (otype[o] != OR_BOX) continue;
        for (int j = 0; j < 12 && nb_i < OR_OFEAT_MAX; j++) {
          double b0[3], b1[3], C[3], D[3];
          box_edge(odims + 3 * o, j, b0, b1);
          to_world(pose_th + 7 * o, b0, C);
          to_world(pose_th + 7 * o, b1, D);
          if (oee_candidate(m, tau + marg, e, C, D, q, xp)) {
            if (cnt < cap) { cvert[cnt] = i; cobs[cnt] = OR_OEE_SLOT; if (ctri) ctri[cnt] = (e * OR_MAX_OBS + o) * 12 + j; }
            cnt++;
            nb_i++;
          }
        }
      }
    }
  }
  free(xp);
  return cnt;
}

/* Linearisation of one contact at (x, gamma).  gamma = (g_n, g_t world[3]).
 * Multipliers are scaled to metres, y = gamma / m_v, so that the
 * Fischer-Burmeister normal law phi_n = FB(a + alpha y_n, y_n) (alpha = normal
 * compliance * m_v / h^2) and the proximal friction law
 * phi_t = y_t - Proj_{|.|<=mu max(y_n,0)}(y_t - s) are in metres.  D_C is the
 * derivative of phi with respect to the contact-space coordinates (gap, slip),
 * D_y its derivative with respect to y. */
typedef struct {
  double R[9];      /* rows: n, t1, t2 */
  double phi[3];
  double DC[9];     /* 3x3 */
  double Dy[9];     /* 3x3 */
  /* the contact point moves as sum_i w[i] x[vi[i]] (vertex contacts: the
   * vertex alone; self contacts: +1 on the vertex, minus the barycentric
   * weights of its closest point on the triangle); meff = 1 / sum w^2 / m */
  int nv, vi[4];
  double w[4], meff;
} Lin;

/* The contact law at a linearisation point: unit normal n, gap a (metres),
 * tangential slip rel over the step (world vector), normal compliance comp,
 * mass mv that scales the multipliers (y = gamma / mv). */
static void contact_law(const double *n, double a, const double *rel, double comp, double mu, double h, double mv,
                        const double *g, Lin *L) {
  double t1[3], t2[3];
  tangent_frame(n, t1, t2);
  for (int i = 0; i < 3; i++) { L->R[i] = n[i]; L->R[3 + i] = t1[i]; L->R[6 + i] = t2[i]; }
  memset(L->DC, 0, sizeof L->DC);
  memset(L->Dy, 0, sizeof L->Dy);
  /* normal: FB with compliance */
  double yn = g[0] / mv;
  double alpha = comp * mv / (h * h);
  double ae = a + alpha * yn;
  double r = sqrt(ae * ae + yn * yn);
  double ca, cy;
  if (r < 1e-12) { ca = 1 - 1 / sqrt(2.0); cy = 1 - 1 / sqrt(2.0); }
  else { ca = 1 - ae / r; cy = 1 - yn / r; }
  L->phi[0] = ae + yn - r;
  L->DC[0] = ca;
  L->Dy[0] = ca * alpha + cy;
  double s[2] = {dot3(t1, rel), dot3(t2, rel)};
  double yt[2] = {dot3(t1, g + 1) / mv, dot3(t2, g + 1) / mv};
  double rad = mu * (yn > 0 ? yn : 0);
  double d[2] = {yt[0] - s[0], yt[1] - s[1]};
  double dn = sqrt(d[0] * d[0] + d[1] * d[1]);
  if (rad == 0.0) {
    /* cone of zero radius (no normal force): the proximal map is the zero
     * map, phi_t = y_t whatever the slip */
    L->phi[1] = yt[0]; L->phi[2] = yt[1];
    L->Dy[4] = 1; L->Dy[8] = 1;
  } else if (dn <= rad) { /* stick (ties included) */
    L->phi[1] = s[0]; L->phi[2] = s[1];
    L->DC[4] = 1; L->DC[8] = 1;
  } else {
    double dh[2] = {d[0] / dn, d[1] / dn};
    L->phi[1] = yt[0] - rad * dh[0];
    L->phi[2] = yt[1] - rad * dh[1];
    double P[4] = {1 - dh[0] * dh[0], -dh[0] * dh[1], -dh[1] * dh[0], 1 - dh[1] * dh[1]};
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++) {
        L->DC[3 * (1 + i) + 1 + j] = rad * P[2 * i + j] / dn;
        L->Dy[3 * (1 + i) + 1 + j] = (i == j ? 1.0 : 0.0) - rad * P[2 * i + j] / dn;
      }
    if (yn > 0) { L->Dy[3] = -mu * dh[0]; L->Dy[6] = -mu * dh[1]; }
  }
}

/* vertex against a kinematic obstacle */
static void linearize(int type, const double *dims, double comp, const double *pose_t,
                      const double *pose_th, double tau, double mu, double h, double mv,
                      const double *x, const double *xt, const double *g, Lin *L) {
  double n[3];
  double sd = or_sdf(type, dims, pose_th, x, n);
  /* tangential slip: displacement relative to the obstacle's material point */
  double pb[3], xo[3];
  to_body(pose_th, x, pb);
  to_world(pose_t, pb, xo);               /* where that material point was at t */
  double dc[3] = {x[0] - xo[0], x[1] - xo[1], x[2] - xo[2]};
  double rel[3] = {x[0] - xt[0] - dc[0], x[1] - xt[1] - dc[1], x[2] - xt[2] - dc[2]};
  contact_law(n, sd - tau, rel, comp, mu, h, mv, g, L);
}

/* Plane of triangle (a, b, c) at x: unit normal nh, signed distance d of the
 * point p and the barycentric weights w of its projection; 0 if degenerate. */
static int tri_plane(const double *a, const double *b, const double *c, const double *p, double *nh, double *d,
                     double *w) {
  double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  double nf[3];
  cross3(e1, e2, nf);
  double ar = norm3(nf);
  if (ar <= 1e-300) return 0;
  for (int i = 0; i < 3; i++) nh[i] = nf[i] / ar;
  double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
  *d = dot3(nh, ap);
  double y[3] = {p[0] - *d * nh[0], p[1] - *d * nh[1], p[2] - *d * nh[2]};
  double ya[3] = {a[0] - y[0], a[1] - y[1], a[2] - y[2]}, yb[3] = {b[0] - y[0], b[1] - y[1], b[2] - y[2]},
         yc[3] = {c[0] - y[0], c[1] - y[1], c[2] - y[2]}, t[3];
  cross3(yb, yc, t);
  w[0] = dot3(nh, t) / ar;
  cross3(yc, ya, t);
  w[1] = dot3(nh, t) / ar;
  w[2] = 1.0 - w[0] - w[1];
  return 1;
}

/* Self contact of vertex p with triangle f (a reading: the paper disables
 * self-collision and describes none).  Frame normal n = the triangle's unit
 * normal at x, oriented towards the side p was on at t; gap = n.(x_p - c) -
 * tau with c the projection of p on the triangle's plane, barycentric
 * weights w; slip = displacement of p relative to the triangle point c over
 * the step; the multipliers scale with the contact's effective mass
 * meff = 1 / (1/m_p + sum w_i^2 / m_i). */
static void linearize_self(const OrMesh *m, double tau, double mu, double h, int p, int f, const double *q,
                           const double *qt, const double *g, Lin *L) {
  const int *t = m->elems + 3 * f;
  double nh[3], d, w[3], nt[3], dt, wt[3];
  L->nv = 4;
  L->vi[0] = p;
  for (int i = 0; i < 3; i++) L->vi[1 + i] = t[i];
  if (!tri_plane(q + 3 * t[0], q + 3 * t[1], q + 3 * t[2], q + 3 * p, nh, &d, w)) {
    nh[0] = 0; nh[1] = 0; nh[2] = 1; d = 0; w[0] = w[1] = w[2] = 1.0 / 3.0;
  }
  double side = 1.0;
  if (tri_plane(qt + 3 * t[0], qt + 3 * t[1], qt + 3 * t[2], qt + 3 * p, nt, &dt, wt) && dt < 0) side = -1.0;
  double n[3] = {side * nh[0], side * nh[1], side * nh[2]};
  double inv = 1.0 / m->mass[p];
  L->w[0] = 1.0;
  for (int i = 0; i < 3; i++) {
    L->w[1 + i] = -w[i];
    inv += w[i] * w[i] / m->mass[t[i]];
  }
  L->meff = 1.0 / inv;
  double rel[3];
  for (int c = 0; c < 3; c++) {
    rel[c] = q[3 * p + c] - qt[3 * p + c];
    for (int i = 0; i < 3; i++) rel[c] -= w[i] * (q[3 * t[i] + c] - qt[3 * t[i] + c]);
  }
  contact_law(n, side * d - tau, rel, 0.0, mu, h, L->meff, g, L);
}

/* Edge-edge self contact of e1 = (a, b) and e2 = (c, d): the contact point
 * moves as (1 - s) x_a + s x_b - (1 - t) x_c - t x_d with (s, t) the closest
 * points of the two lines at x; frame normal = the unit normal of both
 * edges, oriented by the side the first edge was on at t; gap = distance
 * between the lines along it - tau. */
static void linearize_ee(const OrMesh *m, double tau, double mu, double h, int e1, int e2, const double *q,
                         const double *qt, const double *g, Lin *L) {
  const int v[4] = {m->ed[2 * e1], m->ed[2 * e1 + 1], m->ed[2 * e2], m->ed[2 * e2 + 1]};
  double s = 0.5, t = 0.5, st = 0.5, tt = 0.5;
  line_params(q + 3 * v[0], q + 3 * v[1], q + 3 * v[2], q + 3 * v[3], &s, &t);
  double d1[3], d2[3], nr[3], dd[3];
  for (int i = 0; i < 3; i++) {
    d1[i] = q[3 * v[1] + i] - q[3 * v[0] + i];
    d2[i] = q[3 * v[3] + i] - q[3 * v[2] + i];
  }
  cross3(d1, d2, nr);
  double nn = norm3(nr);
  if (nn > 0) for (int i = 0; i < 3; i++) nr[i] /= nn;
  else { nr[0] = 0; nr[1] = 0; nr[2] = 1; }
  /* side at the step start */
  line_params(qt + 3 * v[0], qt + 3 * v[1], qt + 3 * v[2], qt + 3 * v[3], &st, &tt);
  double e1t[3], e2t[3], nt[3], dt[3];
  for (int i = 0; i < 3; i++) {
    e1t[i] = qt[3 * v[1] + i] - qt[3 * v[0] + i];
    e2t[i] = qt[3 * v[3] + i] - qt[3 * v[2] + i];
    dt[i] = (1 - st) * qt[3 * v[0] + i] + st * qt[3 * v[1] + i] - (1 - tt) * qt[3 * v[2] + i] - tt * qt[3 * v[3] + i];
  }
  cross3(e1t, e2t, nt);
  const double side = dot3(nt, dt) < 0 ? -1.0 : 1.0;
  const double w[4] = {1 - s, s, -(1 - t), -t};
  double inv = 0;
  L->nv = 4;
  for (int k = 0; k < 4; k++) {
    L->vi[k] = v[k];
    L->w[k] = w[k];
    inv += w[k] * w[k] / m->mass[v[k]];
  }
  L->meff = 1.0 / inv;
  double rel[3];
  for (int i = 0; i < 3; i++) {
    dd[i] = 0;
    rel[i] = 0;
    for (int k = 0; k < 4; k++) {
      dd[i] += w[k] * q[3 * v[k] + i];
      rel[i] += w[k] * (q[3 * v[k] + i] - qt[3 * v[k] + i]);
    }
  }
  double n[3] = {side * nr[0], side * nr[1], side * nr[2]};
  contact_law(n, dot3(n, dd) - tau, rel, 0.0, mu, h, L->meff, g, L);
}

/* Box corner k of obstacle o against triangle f (a reading; feature
 * (f * OR_MAX_OBS + o) * 8 + k).  The contact point moves as sum_i w_i x_i
 * over f's corners, w the barycentric weights of the box corner's
 * projection on f's plane at x; frame normal n = f's unit normal, oriented
 * towards the side the cloth was on, seen from the box corner, at t; gap =
 * n.(sum_i w_i x_i - C) - tau with C the box corner at t+h; slip = that
 * point's displacement relative to the box corner over the step. */
static void linearize_ovt(const OrMesh *m, const double *odims, const double *pose_t, const double *pose_th,
                          double tau, double mu, double h, int feat, const double *q, const double *qt,
                          const double *g, Lin *L) {
  const int f = feat / (8 * OR_MAX_OBS), o = feat / 8 % OR_MAX_OBS, kc = feat % 8;
  const int *t = m->elems + 3 * f;
  double cb[3], C[3], Ct[3];
  box_corner(odims + 3 * o, kc, cb);
  to_world(pose_th + 7 * o, cb, C);
  to_world(pose_t + 7 * o, cb, Ct);
  double nh[3], d, w[3], nt[3], dt, wt[3];
  if (!tri_plane(q + 3 * t[0], q + 3 * t[1], q + 3 * t[2], C, nh, &d, w)) {
    nh[0] = 0; nh[1] = 0; nh[2] = 1; d = 0; w[0] = w[1] = w[2] = 1.0 / 3.0;
  }
  /* the cloth lies on the -nt side of the corner when the corner is on its +nt side */
  double side = 1.0;
  if (tri_plane(qt + 3 * t[0], qt + 3 * t[1], qt + 3 * t[2], Ct, nt, &dt, wt) && dt > 0) side = -1.0;
  double n[3] = {side * nh[0], side * nh[1], side * nh[2]};
  double inv = 0, rel[3];
  L->nv = 3;
  for (int i = 0; i < 3; i++) {
    L->vi[i] = t[i];
    L->w[i] = w[i];
    inv += w[i] * w[i] / m->mass[t[i]];
  }
  L->meff = 1.0 / inv;
  for (int c = 0; c < 3; c++) {
    rel[c] = -(C[c] - Ct[c]);
    for (int i = 0; i < 3; i++) rel[c] += w[i] * (q[3 * t[i] + c] - qt[3 * t[i] + c]);
  }
  /* n.(sum w x - C) = n.(-d nh) */
  contact_law(n, -side * d - tau, rel, 0.0, mu, h, L->meff, g, L);
}

/* Box edge j of obstacle o against the cloth edge e = (a, b) (a reading;
 * feature (e * OR_MAX_OBS + o) * 12 + j).  (s, t) = closest points of the
 * cloth edge's line and the box edge's line (C, D at t+h) at x (1/2 when
 * parallel); the contact point moves as (1 - s) x_a + s x_b; frame normal =
 * the unit normal of both lines at x, oriented by the side the cloth edge
 * was on at t; gap = n.((1 - s) x_a + s x_b - (1 - t) C - t D) - tau; slip
 * = that difference's displacement over the step. */
static void linearize_oee(const OrMesh *m, const double *odims, const double *pose_t, const double *pose_th,
                          double tau, double mu, double h, int feat, const double *q, const double *qt,
                          const double *g, Lin *L) {
  const int e = feat / (12 * OR_MAX_OBS), o = feat / 12 % OR_MAX_OBS, j = feat % 12;
  const int a = m->ed[2 * e], b = m->ed[2 * e + 1];
  double b0[3], b1[3], C[3], D[3], Ct[3], Dt[3];
  box_edge(odims + 3 * o, j, b0, b1);
  to_world(pose_th + 7 * o, b0, C);
  to_world(pose_th + 7 * o, b1, D);
  to_world(pose_t + 7 * o, b0, Ct);
  to_world(pose_t + 7 * o, b1, Dt);
  double s = 0.5, t = 0.5;
  line_params(q + 3 * a, q + 3 * b, C, D, &s, &t);
  double d1[3], d2[3], nr[3], e1t[3], e2t[3], nt[3], at[3];
  for (int i = 0; i < 3; i++) {
    d1[i] = q[3 * b + i] - q[3 * a + i];
    d2[i] = D[i] - C[i];
    e1t[i] = qt[3 * b + i] - qt[3 * a + i];
    e2t[i] = Dt[i] - Ct[i];
    at[i] = qt[3 * a + i] - Ct[i];
  }
  cross3(d1, d2, nr);
  double nn = norm3(nr);
  if (nn > 0) for (int i = 0; i < 3; i++) nr[i] /= nn;
  else { nr[0] = 0; nr[1] = 0; nr[2] = 1; }
  /* side at the step start: nt is normal to both lines, so nt.(a - C) is
   * the same for any pair of points on them */
  cross3(e1t, e2t, nt);
  const double side = dot3(nt, at) < 0 ? -1.0 : 1.0;
  double n[3] = {side * nr[0], side * nr[1], side * nr[2]}, dd[3], rel[3];
  L->nv = 2;
  L->vi[0] = a; L->vi[1] = b;
  L->w[0] = 1 - s; L->w[1] = s;
  L->meff = 1.0 / ((1 - s) * (1 - s) / m->mass[a] + s * s / m->mass[b]);
  for (int i = 0; i < 3; i++) {
    dd[i] = (1 - s) * q[3 * a + i] + s * q[3 * b + i] - (1 - t) * C[i] - t * D[i];
    rel[i] = (1 - s) * (q[3 * a + i] - qt[3 * a + i]) + s * (q[3 * b + i] - qt[3 * b + i]) -
             (1 - t) * (C[i] - Ct[i]) - t * (D[i] - Dt[i]);
  }
  contact_law(n, dot3(n, dd) - tau, rel, 0.0, mu, h, L->meff, g, L);
}

/* Gaussian elimination with partial pivoting, in place; x = A^-1 b (size k) */
static void gauss_solve(int k, double *A, double *b) {
  for (int c = 0; c < k; c++) {
    int piv = c;
    for (int r = c + 1; r < k; r++) if (fabs(A[r * k + c]) > fabs(A[piv * k + c])) piv = r;
    if (piv != c) {
      for (int j = 0; j < k; j++) { double t = A[c * k + j]; A[c * k + j] = A[piv * k + j]; A[piv * k + j] = t; }
      double t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    double d = A[c * k + c];
    if (fabs(d) < 1e-300) d = 1e-300;
    for (int r = c + 1; r < k; r++) {
      double f = A[r * k + c] / d;
      if (f == 0) continue;
      for (int j = c; j < k; j++) A[r * k + j] -= f * A[c * k + j];
      b[r] -= f * b[c];
    }
  }
  for (int c = k - 1; c >= 0; c--) {
    double s = b[c];
    for (int j = c + 1; j < k; j++) s -= A[c * k + j] * b[j];
    double d = A[c * k + c];
    b[c] = s / (fabs(d) < 1e-300 ? 1e-300 : d);
  }
}

/* Bilateral grasp row: world axes as the frame, phi = x - p_grip (t+h),
 * D_C = I (phi moves with the vertex one to one), D_y = 0 (rigid link). */
static void linearize_grasp(const double *dp, const double *pose_th, const double *x, Lin *L) {
  double p[3];
  to_world(pose_th + 7 * (int)dp[OR_DP_GRASP_OBS], dp + OR_DP_ANCHOR, p);
  memset(L, 0, sizeof *L);
  for (int r = 0; r < 3; r++) {
    L->R[4 * r] = 1.0;
    L->DC[4 * r] = 1.0;
    L->phi[r] = x[r] - p[r];
  }
}

static void contact_lin_all(const OrMesh *m, const double *dp, const int *otype, const double *odims,
                            const double *ocomp, const double *pose_t, const double *pose_th,
                            const double *qt, const double *q, int count, const int *cvert,
                            const int *cobs, const int *ctri, const double *cg, Lin *lin) {
  for (int i = 0; i < count; i++) {
    int v = cvert[i], o = cobs[i];
    Lin *L = lin + i;
    if (o == OR_SELF_SLOT) {
      linearize_self(m, dp[OR_DP_TAU], dp[OR_DP_MU], dp[OR_DP_H], v, ctri[i], q, qt, cg + 4 * i, L);
      continue;
    }
    if (o == OR_EE_SLOT) {
      linearize_ee(m, dp[OR_DP_TAU], dp[OR_DP_MU], dp[OR_DP_H], ctri[i] / m->ned, ctri[i] % m->ned, q, qt,
                   cg + 4 * i, L);
      continue;
    }
    if (o == OR_OVT_SLOT || o == OR_OEE_SLOT) {
      (o == OR_OVT_SLOT ? linearize_ovt : linearize_oee)(m, odims, pose_t, pose_th, dp[OR_DP_TAU], dp[OR_DP_MU],
                                                         dp[OR_DP_H], ctri[i], q, qt, cg + 4 * i, L);
      continue;
    }
    if (o == OR_GRASP_SLOT) linearize_grasp(dp, pose_th, q + 3 * v, L);
    else
      linearize(otype[o], odims + 3 * o, ocomp[o], pose_t + 7 * o, pose_th + 7 * o, dp[OR_DP_TAU],
                dp[OR_DP_MU], dp[OR_DP_H], m->mass[v], q + 3 * v, qt + 3 * v, cg + 4 * i, L);
    L->nv = 1;
    L->vi[0] = v;
    L->w[0] = 1.0;
    L->meff = m->mass[v];
  }
}

static double max_abs_phi(int count, const Lin *lin) {
  double r = 0;
  for (int i = 0; i < count; i++)
    for (int j = 0; j < 3; j++) r = fmax(r, fabs(lin[i].phi[j]));
  return r;
}

double or_residual(const OrMesh *m, const double *dp, int K, const int *otype, const double *odims,
                   const double *ocomp, const double *pose_t, const double *pose_th,
                   const double *q_t, const double *q, int count, const int *cvert, const int *cobs,
                   const int *ctri, const double *cgamma) {
  (void)K;
  Lin *lin = (Lin *)malloc(sizeof(Lin) * (count > 0 ? count : 1));
  contact_lin_all(m, dp, otype, odims, ocomp, pose_t, pose_th, q_t, q, count, cvert, cobs, ctri, cgamma, lin);
  double r = max_abs_phi(count, lin);
  free(lin);
  return r;
}

/* J^T gamma for every contact added into f [n][3]: n g_n + P_t g_t (the
 * tangential multiplier is kept as a world vector in the tangent plane) */
static void add_contact_force(int count, const Lin *lin, const double *cg, double *f) {
  for (int i = 0; i < count; i++) {
    const Lin *L = lin + i;
    const double *R = L->R, *g = cg + 4 * i;
    double yt1 = dot3(R + 3, g + 1), yt2 = dot3(R + 6, g + 1);
    for (int c = 0; c < 3; c++) {
      double F = R[c] * g[0] + R[3 + c] * yt1 + R[6 + c] * yt2;
      for (int a = 0; a < L->nv; a++) f[3 * L->vi[a] + c] += L->w[a] * F;
    }
  }
}

/* J du at contact L: the contact point's share of du [n][3] */
static void contact_gather(const Lin *L, const double *du, double *out) {
  for (int c = 0; c < 3; c++) {
    out[c] = 0;
    for (int a = 0; a < L->nv; a++) out[c] += L->w[a] * du[3 * L->vi[a] + c];
  }
}

/* Solve the Newton system for the contacts listed in idx[0..k) jointly:
 *   (D_C R_i R_j^T X_ij m_j + delta_ij D_y,i) dy_j = -phi_i - D_C,i R_i (u - q)_{v_i}
 * with X = M^-1 (lite metric, Sec. IV-B.1) or A^-1 (full metric, Eq. schur),
 * then gamma += m dy (Algorithm 1: lambda^k = lambda^{k-1} + dlambda). */
static void newton_block(const OrMesh *m, int metric, const double *Ainv, int k, const int *idx,
                         const Lin *lin, const double *u, const double *q, double *cg, double gmax) {
  int N = 3 * k;
  double *Z = (double *)calloc((size_t)N * N, sizeof(double));
  double *rhs = (double *)malloc(sizeof(double) * N);
  double *dd = (double *)malloc(sizeof(double) * 3 * m->n);
  for (int i = 0; i < 3 * m->n; i++) dd[i] = u[i] - q[i];
  for (int a = 0; a < k; a++) {
    int i = idx[a];
    const Lin *Li = lin + i;
    double du[3];
    contact_gather(Li, dd, du);
    double Rdu[3] = {dot3(Li->R, du), dot3(Li->R + 3, du), dot3(Li->R + 6, du)};
    for (int r = 0; r < 3; r++) {
      double s = 0;
      for (int c = 0; c < 3; c++) s += Li->DC[3 * r + c] * Rdu[c];
      rhs[3 * a + r] = -Li->phi[r] - s;
    }
    for (int b = 0; b < k; b++) {
      int j = idx[b];
      const Lin *Lj = lin + j;
      /* X = J_a X J_b^T with X = M^-1 (lite) or A^-1 (full), both scalar per vertex pair */
      double X = 0;
      for (int s1 = 0; s1 < Li->nv; s1++)
        for (int s2 = 0; s2 < Lj->nv; s2++) {
          int va = Li->vi[s1], vb = Lj->vi[s2];
          double x = metric == 0 ? (va == vb ? 1.0 / m->mass[va] : 0.0) : Ainv[(size_t)va * m->n + vb];
          X += Li->w[s1] * Lj->w[s2] * x;
        }
      if (X == 0.0 && a != b) continue;
      double RR[9];
      for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) RR[3 * r + c] = dot3(Li->R + 3 * r, Lj->R + 3 * c) * X * Lj->meff;
      for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
          double s = 0;
          for (int t = 0; t < 3; t++) s += Li->DC[3 * r + t] * RR[3 * t + c];
          Z[(3 * a + r) * N + 3 * b + c] += s;
        }
      if (a == b)
        for (int r = 0; r < 3; r++) {
          for (int c = 0; c < 3; c++) Z[(3 * a + r) * N + 3 * b + c] += Li->Dy[3 * r + c];
          /* reading: a tiny damping of the Newton step keeps blocks of
           * redundant contacts on one vertex (e.g. two sticking contacts)
           * solvable; it leaves every fixed point unchanged */
          Z[(3 * a + r) * N + 3 * b + r] += OR_DAMP;
        }
    }
  }
  gauss_solve(N, Z, rhs);
  for (int a = 0; a < k; a++) {
    int i = idx[a];
    double mv = lin[i].meff;
    const double *R = lin[i].R;
    double *g = cg + 4 * i;
    g[0] += mv * rhs[3 * a];
    if (g[0] > gmax) g[0] = gmax;
    double yt1 = dot3(R + 3, g + 1) + mv * rhs[3 * a + 1];
    double yt2 = dot3(R + 6, g + 1) + mv * rhs[3 * a + 2];
    for (int c = 0; c < 3; c++) g[1 + c] = R[3 + c] * yt1 + R[6 + c] * yt2;
  }
  free(Z);
  free(rhs);
  free(dd);
}

/* diag(A^-1), one solve per vertex on first use */
static const double *ainv_diag(OrMesh *m) {
  if (m->Adiag) return m->Adiag;
  int n = m->n;
  m->Adiag = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  double *e = (double *)calloc(3 * (size_t)n, sizeof(double)), *col = (double *)malloc(sizeof(double) * 3 * n);
  for (int j = 0; j < n; j++) {
    e[3 * j] = 1.0;
    or_solve(m, e, col);
    m->Adiag[j] = col[3 * j];
    e[3 * j] = 0.0;
  }
  free(e); free(col);
  return m->Adiag;
}

/* z = Z x for the full metric, matrix-free: forces m_b R_b^T x_b on the
 * contact vertices, one solve with A, then at each contact a
 * D_C(a) R_a (A^-1 f)_{v_a} + (D_y(a) + damping) x_a. */
static void full_z_apply(const OrMesh *m, int k, const Lin *lin, const double *x, double *f, double *u,
                         double *z) {
  memset(f, 0, sizeof(double) * 3 * m->n);
  for (int b = 0; b < k; b++) {
    const Lin *L = lin + b;
    for (int c = 0; c < 3; c++) {
      double F = L->meff * (L->R[c] * x[3 * b] + L->R[3 + c] * x[3 * b + 1] + L->R[6 + c] * x[3 * b + 2]);
      for (int s2 = 0; s2 < L->nv; s2++) f[3 * L->vi[s2] + c] += L->w[s2] * F;
    }
  }
  or_solve(m, f, u);
  for (int a = 0; a < k; a++) {
    const Lin *L = lin + a;
    double ua[3];
    contact_gather(L, u, ua);
    double Ru[3] = {dot3(L->R, ua), dot3(L->R + 3, ua), dot3(L->R + 6, ua)};
    for (int r = 0; r < 3; r++) {
      double s = OR_DAMP * x[3 * a + r];
      for (int c = 0; c < 3; c++) s += L->DC[3 * r + c] * Ru[c] + L->Dy[3 * r + c] * x[3 * a + c];
      z[3 * a + r] = s;
    }
  }
}

/* Full-metric Newton step with an iterative Z solve (the "linear-solver
 * iterations" of the paper's parameter table): mlin steps of GMRES (Saad and
 * Schultz 1986) on Z dy = rhs from dy = 0, right-preconditioned by the
 * inverses of Z's 3x3 diagonal blocks, Arnoldi with modified Gram-Schmidt,
 * Givens rotations for the small least-squares problem; stops early when
 * the new Arnoldi vector's norm falls below 1e-6 |rhs| (the Krylov space is
 * exhausted to rounding).  Contacts: the whole list of the environment.
 * The multiplier update is the one of newton_block. */
static void newton_gmres(OrMesh *m, int k, const Lin *lin, const double *u, const double *q, double *cg,
                         double gmax, int mlin) {
  int N = 3 * k;
  if (k == 0 || mlin < 1) return;
  const double *ad = ainv_diag(m);
  double *rhs = (double *)malloc(sizeof(double) * N);
  double *Pinv = (double *)malloc(sizeof(double) * 9 * k);
  double *dd = (double *)malloc(sizeof(double) * 3 * m->n);
  for (int i = 0; i < 3 * m->n; i++) dd[i] = u[i] - q[i];
  for (int a = 0; a < k; a++) {
    const Lin *L = lin + a;
    double du[3];
    contact_gather(L, dd, du);
    double Rdu[3] = {dot3(L->R, du), dot3(L->R + 3, du), dot3(L->R + 6, du)};
    for (int r = 0; r < 3; r++) {
      double s = 0;
      for (int c = 0; c < 3; c++) s += L->DC[3 * r + c] * Rdu[c];
      rhs[3 * a + r] = -L->phi[r] - s;
    }
    /* diagonal block D_C (sum_i w_i^2 a_{v_i v_i}) meff + D_y + damping (R R^T
     * = I; a reading for contacts over several vertices: the diagonal of
     * A^-1 only) and its inverse */
    double av = 0;
    for (int s2 = 0; s2 < L->nv; s2++) av += L->w[s2] * L->w[s2] * ad[L->vi[s2]];
    double B[9], I[9];
    for (int t = 0; t < 9; t++) B[t] = L->DC[t] * av * L->meff + L->Dy[t];
    for (int r = 0; r < 3; r++) B[4 * r] += OR_DAMP;
    for (int c = 0; c < 3; c++) {
      double e3[3] = {0, 0, 0}, A3[9];
      e3[c] = 1.0;
      memcpy(A3, B, sizeof A3);
      gauss_solve(3, A3, e3);
      for (int r = 0; r < 3; r++) I[3 * r + c] = e3[r];
    }
    memcpy(Pinv + 9 * a, I, sizeof I);
  }
  double beta = 0;
  for (int i = 0; i < N; i++) beta += rhs[i] * rhs[i];
  beta = sqrt(beta);
  double *dy = (double *)calloc(N, sizeof(double));
  if (beta > 0) {
    double *V = (double *)calloc((size_t)(mlin + 1) * N, sizeof(double));
    double *H = (double *)calloc((size_t)(mlin + 1) * mlin, sizeof(double));  /* H[i][j] at i * mlin + j */
    double *cs = (double *)calloc(mlin, sizeof(double)), *sn = (double *)calloc(mlin, sizeof(double));
    double *gv = (double *)calloc(mlin + 1, sizeof(double));
    double *t = (double *)malloc(sizeof(double) * N), *w = (double *)malloc(sizeof(double) * N);
    double *f = (double *)malloc(sizeof(double) * 3 * m->n), *uu = (double *)malloc(sizeof(double) * 3 * m->n);
    for (int i = 0; i < N; i++) V[i] = rhs[i] / beta;
    gv[0] = beta;
    int jm = 0;
    for (int j = 0; j < mlin; j++) {
      const double *vj = V + (size_t)j * N;
      for (int a = 0; a < k; a++)
        for (int r = 0; r < 3; r++) t[3 * a + r] = dot3(Pinv + 9 * a + 3 * r, vj + 3 * a);
      full_z_apply(m, k, lin, t, f, uu, w);
      for (int i = 0; i <= j; i++) {
        const double *vi = V + (size_t)i * N;
        double h = 0;
        for (int e = 0; e < N; e++) h += w[e] * vi[e];
        H[i * mlin + j] = h;
        for (int e = 0; e < N; e++) w[e] -= h * vi[e];
      }
      double hn = 0;
      for (int e = 0; e < N; e++) hn += w[e] * w[e];
      hn = sqrt(hn);
      H[(j + 1) * mlin + j] = hn;
      for (int i = 0; i < j; i++) {  /* previous rotations on column j */
        double a0 = H[i * mlin + j], a1 = H[(i + 1) * mlin + j];
        H[i * mlin + j] = cs[i] * a0 + sn[i] * a1;
        H[(i + 1) * mlin + j] = -sn[i] * a0 + cs[i] * a1;
      }
      double a0 = H[j * mlin + j], a1 = H[(j + 1) * mlin + j], rr = sqrt(a0 * a0 + a1 * a1);
      cs[j] = rr > 0 ? a0 / rr : 1.0;
      sn[j] = rr > 0 ? a1 / rr : 0.0;
      H[j * mlin + j] = rr;
      H[(j + 1) * mlin + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      jm = j + 1;
      if (hn <= 1e-6 * beta) break;
      for (int e = 0; e < N; e++) V[(size_t)(j + 1) * N + e] = w[e] / hn;
    }
    /* H[0..jm)[0..jm) y = g, back substitution; z = V y; dy = P^-1 z */
    double *y = (double *)calloc(jm > 0 ? jm : 1, sizeof(double));
    for (int i = jm - 1; i >= 0; i--) {
      double s = gv[i];
      for (int c = i + 1; c < jm; c++) s -= H[i * mlin + c] * y[c];
      y[i] = H[i * mlin + i] != 0 ? s / H[i * mlin + i] : 0.0;
    }
    for (int e = 0; e < N; e++) {
      double s = 0;
      for (int i = 0; i < jm; i++) s += V[(size_t)i * N + e] * y[i];
      w[e] = s;
    }
    for (int a = 0; a < k; a++)
      for (int r = 0; r < 3; r++) dy[3 * a + r] = dot3(Pinv + 9 * a + 3 * r, w + 3 * a);
    free(y); free(V); free(H); free(cs); free(sn); free(gv); free(t); free(w); free(f); free(uu);
  }
  for (int a = 0; a < k; a++) {
    double mv = lin[a].meff;
    const double *R = lin[a].R;
    double *g = cg + 4 * a;
    g[0] += mv * dy[3 * a];
    if (g[0] > gmax) g[0] = gmax;
    double yt1 = dot3(R + 3, g + 1) + mv * dy[3 * a + 1];
    double yt2 = dot3(R + 6, g + 1) + mv * dy[3 * a + 2];
    for (int c = 0; c < 3; c++) g[1 + c] = R[3 + c] * yt1 + R[6 + c] * yt2;
  }
  free(dy); free(rhs); free(Pinv); free(dd);
}

int or_solve_step(const OrMesh *m, const double *dp, const int *ip, int K, const int *otype,
                  const double *odims, const double *ocomp, const double *pose_t,
                  const double *pose_th, double *q, double *v, const double *q_init, int count,
                  const int *cvert, const int *cobs, const int *ctri, double *cgamma, int *iters, double *rncp,
                  double *trace) {
  (void)K;
  int n = m->n;
  double h = dp[OR_DP_H], h2 = h * h;
  double gmax = h2 * dp[OR_DP_MAXFORCE];
  int kmax = ip[OR_IP_KMAX], kmin = ip[OR_IP_KMIN], kcap = ip[OR_IP_KCAP], mode = ip[OR_IP_MODE];
  int metric = ip[OR_IP_METRIC];
  size_t vb = sizeof(double) * 3 * n;
  double *qt = (double *)malloc(vb), *qp = (double *)malloc(vb), *qc = (double *)malloc(vb);
  double *b = (double *)malloc(vb), *g = (double *)malloc(vb), *u = (double *)malloc(vb);
  double *p = (double *)malloc(sizeof(double) * 9 * (m->ne > 0 ? m->ne : 1));
  Lin *lin = (Lin *)malloc(sizeof(Lin) * (count > 0 ? count : 1));
  double *Ainv = NULL;
  if (metric == 1 && count > 0) {
    Ainv = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *e = (double *)calloc(3 * n, sizeof(double)), *col = (double *)malloc(vb);
    for (int j = 0; j < n; j++) {
      e[3 * j] = 1.0;
      or_solve(m, e, col);
      for (int i = 0; i < n; i++) Ainv[(size_t)i * n + j] = col[3 * i];
      e[3 * j] = 0.0;
    }
    free(e); free(col);
  }
  /* predicted state q~ = q_t + h v_t + h^2 M^-1 f_ext (f_ext = M g) */
  memcpy(qt, q, vb);
  for (int i = 0; i < n; i++)
    for (int c = 0; c < 3; c++) qp[3 * i + c] = qt[3 * i + c] + h * v[3 * i + c] + h2 * dp[OR_DP_GX + c];
  memcpy(qc, q_init ? q_init : qp, vb);
  /* group contacts by vertex (the list is sorted by vertex) */
  int *grp = (int *)malloc(sizeof(int) * (count + 1));
  int ngrp = 0;
  for (int i = 0; i < count; i++) if (i == 0 || cvert[i] != cvert[i - 1]) grp[ngrp++] = i;
  grp[ngrp] = count;
  int *all = (int *)malloc(sizeof(int) * (count > 0 ? count : 1));
  for (int i = 0; i < count; i++) all[i] = i;
  int k = 0;
  double r = 0;
  for (;;) {
    contact_lin_all(m, dp, otype, odims, ocomp, pose_t, pose_th, qt, qc, count, cvert, cobs, ctri, cgamma, lin);
    r = max_abs_phi(count, lin);
    if (trace) trace[k] = r;
    if (mode == 0) { if (k >= kmax) break; }
    else if ((k >= kmin && r <= dp[OR_DP_TOL]) || k >= kcap) break;
    /* local projection, then b */
    or_project(m, qc, p);
    or_assemble_b(m, qp, p, b);
    /* g = b + J^T gamma^{k-1};  u = A^-1 g */
    memcpy(g, b, vb);
    add_contact_force(count, lin, cgamma, g);
    or_solve(m, g, u);
    /* dgamma = Z^-1 (h - J u),  gamma^k = gamma^{k-1} + dgamma */
    if (metric == 0) {
      for (int t = 0; t < ngrp; t++)
        newton_block(m, 0, NULL, grp[t + 1] - grp[t], all + grp[t], lin, u, qc, cgamma, gmax);
    } else if (metric == 1 && count > 0) {
      newton_block(m, 1, Ainv, count, all, lin, u, qc, cgamma, gmax);
    } else if (metric == 2) {
      newton_gmres((OrMesh *)m, count, lin, u, qc, cgamma, gmax, ip[OR_IP_LINIT]);
    }
    /* q^k = A^-1 (b + J^T gamma^k) */
    memcpy(g, b, vb);
    add_contact_force(count, lin, cgamma, g);
    or_solve(m, g, qc);
    k++;
  }
  for (int i = 0; i < 3 * n; i++) {
    v[i] = (qc[i] - qt[i]) / h;
    q[i] = qc[i];
  }
  if (iters) *iters = k;
  if (rncp) *rncp = r;
  free(qt); free(qp); free(qc); free(b); free(g); free(u); free(p); free(lin);
  free(grp); free(all); free(Ainv);
  return 0;
}
