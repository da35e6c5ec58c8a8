// Batched depth ray casting of the simulation state (appendix, depth
// rendering: depth maps, instance segmentation masks and point clouds cast
// directly from the simulated meshes and obstacles).
//
// Every pixel sees the nearest hit along its ray.  The mesh part runs in
// object order, which suits the many small triangles of a cloth (a triangle
// covers a few pixels): one thread per (environment, triangle) transforms its
// three vertices into the camera frame, walks the pixels of its projected
// bounding box, tests each pixel's ray exactly and keeps the nearest hit per
// pixel with a 64-bit atomic min of (depth bits, triangle index): the result
// is the nearest triangle hit of every pixel, the same answer as a ray-first
// traversal, without building or refitting an acceleration structure for
// the per-step geometry.  A second pass per pixel intersects the analytic
// obstacles, picks the nearest surface and writes depth, instance and the
// world point.
//
// Watertight coverage: for a triangle in front of the camera, a pixel's ray
// meets it iff the pixel centre lies in its projection; projections are
// snapped to 1/4096 pixel per vertex and the 2D edge functions evaluated
// exactly in integers, so no ray slips between triangles that share an edge
// or a vertex (the snap moves a decision by at most 1/4096 pixel).
// Triangles reaching behind the camera use the 3D cone test (the three
// triple products d.(a x b) share a sign).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "flash_internal.cuh"

namespace flash {

namespace {

// Per-pixel keys are not cleared between frames.  A key packs an 8-bit frame
// tag, the depth's bits without the sign (depth > 0) and the triangle index:
// tag << 56 | depth_bits << 25 | triangle.  Frames count their tag down
// (254, 253, ..., 0), so with atomicMin any hit of the current frame beats
// whatever an older frame left, and the resolve pass reads a key as a hit
// only when its tag is the current one.  After tag 0 the buffer is refilled
// with all ones (tag 255: never current) and the count restarts at 254.
__device__ __forceinline__ void store_key(unsigned long long *k, float depth, int f, unsigned tag) {
  const unsigned long long key = ((unsigned long long)tag << 56) |
                                 ((unsigned long long)(__float_as_uint(depth) & 0x7fffffffu) << 25) | (unsigned)f;
  atomicMin(k, key);
}
// fixed-point image coordinates: 1/4096 pixel; projections beyond 2^17
// pixels take the 3D path, so every edge-function product fits in 62 bits
constexpr int kSubBits = 12;
constexpr long long kSub = 1LL << kSubBits;
constexpr float kMaxProj = 131072.f;

__device__ __forceinline__ void rc_quat_mat(const float *q, float *R) {
  const float w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// a x b with every product and sum rounded explicitly (no contraction
// choices left to the compiler), so equal operands give equal bits anywhere
__device__ __forceinline__ float3 cross_rn(float3 a, float3 b) {
  return make_float3(__fmaf_rn(a.y, b.z, -__fmul_rn(a.z, b.y)), __fmaf_rn(a.z, b.x, -__fmul_rn(a.x, b.z)),
                     __fmaf_rn(a.x, b.y, -__fmul_rn(a.y, b.x)));
}
// d.c with d = (dx, dy, 1)
__device__ __forceinline__ float edge_rn(float3 c, float dx, float dy) {
  return __fmaf_rn(dx, c.x, __fmaf_rn(dy, c.y, c.z));
}
// ray direction of pixel (u, v) in camera axes (z component 1)
__device__ __forceinline__ float ray_dx(int u, const RcCam &C) { return __fdiv_rn(__fadd_rn(u + 0.5f, -C.cx), C.fx); }
__device__ __forceinline__ float ray_dy(int v, const RcCam &C) { return __fdiv_rn(__fadd_rn(v + 0.5f, -C.cy), C.fy); }

__global__ void __launch_bounds__(256) k_rc_tri(RcMesh M, const float *__restrict__ cam_poses, RcCam C,
                                                unsigned long long *__restrict__ keys, unsigned tag) {
  __shared__ float sR[9], sp[3];
  const int l = blockIdx.y;
  const int e = M.genv ? M.genv[l] : M.first_env + l;
  if (threadIdx.x == 0) {
    const float *cp = cam_poses + 7 * (size_t)e;
    rc_quat_mat(cp + 3, sR);
    sp[0] = cp[0]; sp[1] = cp[1]; sp[2] = cp[2];
  }
  __syncthreads();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= M.T) return;
  const int3 t = M.tris[f];
  const int vi[3] = {t.x, t.y, t.z};
  const float *xe = M.x + (size_t)l * M.env_stride;
  float3 y[3];
  float zmin = INFINITY, zmax = -INFINITY;
  bool finite = true;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const float *xv = xe + (size_t)vi[k] * M.vert_stride;
    const float w0 = __fsub_rn(xv[0], sp[0]), w1 = __fsub_rn(xv[M.coord_stride], sp[1]),
                w2 = __fsub_rn(xv[2 * M.coord_stride], sp[2]);
    // camera coordinates y = R^T (x - p)
    y[k] = make_float3(__fmaf_rn(sR[6], w2, __fmaf_rn(sR[3], w1, __fmul_rn(sR[0], w0))),
                       __fmaf_rn(sR[7], w2, __fmaf_rn(sR[4], w1, __fmul_rn(sR[1], w0))),
                       __fmaf_rn(sR[8], w2, __fmaf_rn(sR[5], w1, __fmul_rn(sR[2], w0))));
    finite = finite && isfinite(y[k].x) && isfinite(y[k].y) && isfinite(y[k].z);
    zmin = fminf(zmin, y[k].z);
    zmax = fmaxf(zmax, y[k].z);
  }
  // no point of the triangle can lie in the depth range
  if (!finite || zmax < C.zn || zmin > C.zf) return;
  // supporting plane n.x = n.y0 (edge vectors are short and accurate)
  const float3 e1 = make_float3(y[1].x - y[0].x, y[1].y - y[0].y, y[1].z - y[0].z);
  const float3 e2 = make_float3(y[2].x - y[0].x, y[2].y - y[0].y, y[2].z - y[0].z);
  const float3 n = make_float3(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x);
  const float num = n.x * y[0].x + n.y * y[0].y + n.z * y[0].z;
  unsigned long long *ke = keys + (size_t)e * C.W * C.H;
  // Coverage.  With every vertex in front of the camera the ray of a pixel
  // meets the triangle iff the pixel centre lies in the projected triangle:
  // vertices are projected and snapped to 1/4096 pixel (per vertex, the same
  // bits in every triangle that uses it) and the 2D edge functions are
  // evaluated exactly in 64-bit integers, so shared edges and vertices leave
  // no gap.  Pixel centres sit on integer coordinates.
  int X[3], Y[3];   // |X|, |Y| < 2^29
  bool fixed_point = zmin > 0.5f * C.zn;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    if (!fixed_point) break;
    const float iz = __fdividef(1.f, y[k].z);
    const float uc = __fmaf_rn(C.fx, __fmul_rn(y[k].x, iz), C.cx - 0.5f);
    const float vc = __fmaf_rn(C.fy, __fmul_rn(y[k].y, iz), C.cy - 0.5f);
    if (!(fabsf(uc) < kMaxProj && fabsf(vc) < kMaxProj)) fixed_point = false;
    X[k] = __float2int_rn(__fmul_rn(uc, (float)kSub));
    Y[k] = __float2int_rn(__fmul_rn(vc, (float)kSub));
  }
  if (fixed_point) {
    const int xmin = min(X[0], min(X[1], X[2])), xmax = max(X[0], max(X[1], X[2]));
    const int ymin = min(Y[0], min(Y[1], Y[2])), ymax = max(Y[0], max(Y[1], Y[2]));
    // pixels with centres inside the bounding box (ceil / floor of the scaled
    // range; >> of a negative value rounds towards minus infinity)
    const int u0 = max(0, -((-xmin) >> kSubBits)), u1 = min(C.W - 1, xmax >> kSubBits);
    const int v0 = max(0, -((-ymin) >> kSubBits)), v1 = min(C.H - 1, ymax >> kSubBits);
    const long long area = (long long)(X[1] - X[0]) * (Y[2] - Y[0]) - (long long)(Y[1] - Y[0]) * (X[2] - X[0]);
    if (area == 0 || u0 > u1 || v0 > v1) return;   // seen edge-on, or between pixel centres
    const float ifx = 1.f / C.fx, ify = 1.f / C.fy;
    if (u1 - u0 < 4 && v1 - v0 < 4) {
      // Small triangle (at most 4 x 4 pixel centres): coordinates relative to
      // the first pixel centre are below 5 pixels = 20480 units, so every
      // edge-function product stays below 2^29 and 32-bit integers are exact.
      const int bx = u0 * (int)kSub, by = v0 * (int)kSub;
      int x[3], yy[3];
#pragma unroll
      for (int k = 0; k < 3; k++) { x[k] = X[k] - bx; yy[k] = Y[k] - by; }
      const int t0 = yy[1] - yy[2], t1 = yy[2] - yy[0], t2 = yy[0] - yy[1];   // change per pixel / kSub
      const int nu = u1 - u0, nv = v1 - v0;
      for (int j = 0; j <= nv; j++) {
        const int py = j * (int)kSub;
        int E0 = (x[2] - x[1]) * (py - yy[1]) + t0 * (0 - x[1]);
        int E1 = (x[0] - x[2]) * (py - yy[2]) + t1 * (0 - x[2]);
        int E2 = (x[1] - x[0]) * (py - yy[0]) + t2 * (0 - x[0]);
        const float rowc = n.y * ((v0 + j + 0.5f - C.cy) * ify) + n.z;
        for (int i = 0; i <= nu; i++, E0 += t0 * (int)kSub, E1 += t1 * (int)kSub, E2 += t2 * (int)kSub) {
          const bool in = (E0 >= 0 && E1 >= 0 && E2 >= 0) || (E0 <= 0 && E1 <= 0 && E2 <= 0);
          if (!in) continue;
          const int u = u0 + i;
          const float nd = n.x * ((u + 0.5f - C.cx) * ifx) + rowc;
          if (nd == 0.f) continue;
          const float depth = __fdividef(num, nd);
          if (!(depth >= C.zn && depth <= C.zf)) continue;
          store_key(ke + (size_t)(v0 + j) * C.W + u, depth, f, tag);
        }
      }
      return;
    }
    // edge functions at the row's first pixel, then stepped exactly by
    // their (integer) change per pixel
    const long long s0 = (long long)(Y[1] - Y[2]) * kSub, s1 = (long long)(Y[2] - Y[0]) * kSub,
                    s2 = (long long)(Y[0] - Y[1]) * kSub;
    for (int v = v0; v <= v1; v++) {
      const long long py = (long long)v * kSub, px = (long long)u0 * kSub;
      long long E0 = (long long)(X[2] - X[1]) * (py - Y[1]) - (long long)(Y[2] - Y[1]) * (px - X[1]);
      long long E1 = (long long)(X[0] - X[2]) * (py - Y[2]) - (long long)(Y[0] - Y[2]) * (px - X[2]);
      long long E2 = (long long)(X[1] - X[0]) * (py - Y[0]) - (long long)(Y[1] - Y[0]) * (px - X[0]);
      const float rowc = n.y * ((v + 0.5f - C.cy) * ify) + n.z;
      for (int u = u0; u <= u1; u++, E0 += s0, E1 += s1, E2 += s2) {
        const bool in = (E0 >= 0 && E1 >= 0 && E2 >= 0) || (E0 <= 0 && E1 <= 0 && E2 <= 0);
        if (!in) continue;
        const float nd = n.x * ((u + 0.5f - C.cx) * ifx) + rowc;
        if (nd == 0.f) continue;
        const float depth = __fdividef(num, nd);
        if (!(depth >= C.zn && depth <= C.zf)) continue;
        store_key(ke + (size_t)v * C.W + u, depth, f, tag);
      }
    }
    return;
  }
  // A triangle reaching behind the camera (or projecting absurdly far): the
  // 3D test over the whole image, d inside the cone of the three vertices
  // (edge normals formed in ascending vertex order, so shared edges agree).
  float3 ce[3];
  float sg[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    if (vi[a] < vi[b]) { ce[k] = cross_rn(y[a], y[b]); sg[k] = 1.f; }
    else { ce[k] = cross_rn(y[b], y[a]); sg[k] = -1.f; }
  }
  for (int v = 0; v < C.H; v++) {
    const float dy = ray_dy(v, C);
    for (int u = 0; u < C.W; u++) {
      const float dx = ray_dx(u, C);
      const float s0 = sg[0] * edge_rn(ce[0], dx, dy);
      const float s1 = sg[1] * edge_rn(ce[1], dx, dy);
      const float s2 = sg[2] * edge_rn(ce[2], dx, dy);
      const bool in = (s0 >= 0.f && s1 >= 0.f && s2 >= 0.f) || (s0 <= 0.f && s1 <= 0.f && s2 <= 0.f);
      if (!in) continue;
      const float nd = n.x * dx + n.y * dy + n.z;
      if (nd == 0.f) continue;
      const float depth = num / nd;
      if (!(depth >= C.zn && depth <= C.zf)) continue;
      store_key(ke + (size_t)v * C.W + u, depth, f, tag);
    }
  }
}

// Obstacles in the frame of one camera: what every pixel's test shares.
struct ObsRay {
  int type;
  float a[3];   // plane: world normal; sphere: centre - camera; box: camera in box axes
  float b;      // plane: n.(p - o); sphere: r^2
  float R[9];   // box: rotation body -> world (rows), so R^T d is the ray in box axes
  float h[3];   // box: half extents
};

// nearest hit t >= zn of the ray o + t d with an obstacle (INFINITY: none)
__device__ __forceinline__ float ray_obstacle(const ObsRay &Q, float3 d, float zn) {
  if (Q.type == FLASH_OBS_PLANE) {
    const float dn = Q.a[0] * d.x + Q.a[1] * d.y + Q.a[2] * d.z;
    const float t = __fdividef(Q.b, dn);
    return (dn != 0.f && t >= zn) ? t : INFINITY;
  }
  if (Q.type == FLASH_OBS_SPHERE) {
    // closest approach along the unit direction, then the chord: no
    // cancellation between |c - o|^2 and r^2 near the silhouette
    const float il = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
    const float3 u = make_float3(d.x * il, d.y * il, d.z * il);
    const float tc = u.x * Q.a[0] + u.y * Q.a[1] + u.z * Q.a[2];
    const float3 q = make_float3(Q.a[0] - tc * u.x, Q.a[1] - tc * u.y, Q.a[2] - tc * u.z);
    const float h2 = q.x * q.x + q.y * q.y + q.z * q.z;
    if (h2 > Q.b) return INFINITY;
    const float sq = sqrtf(Q.b - h2);
    const float t1 = (tc - sq) * il, t2 = (tc + sq) * il;
    return t1 >= zn ? t1 : (t2 >= zn ? t2 : INFINITY);
  }
  if (Q.type == FLASH_OBS_BOX) {
    float tmin = -INFINITY, tmax = INFINITY;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const float db = Q.R[i] * d.x + Q.R[3 + i] * d.y + Q.R[6 + i] * d.z;
      if (db == 0.f) {
        if (fabsf(Q.a[i]) > Q.h[i]) return INFINITY;
        continue;
      }
      const float inv = __frcp_rn(db);
      float ta = (-Q.h[i] - Q.a[i]) * inv, tb = (Q.h[i] - Q.a[i]) * inv;
      if (ta > tb) { const float x = ta; ta = tb; tb = x; }
      tmin = fmaxf(tmin, ta);
      tmax = fminf(tmax, tb);
    }
    if (tmin > tmax) return INFINITY;
    return tmin >= zn ? tmin : (tmax >= zn ? tmax : INFINITY);
  }
  return INFINITY;
}

// What every pixel of one environment's view shares: the camera and, per
// obstacle, its ray-test constants and the bounds of its projection.
struct EnvPrep {
  float Rc[9], p[3], ifx, ify;
  ObsRay Q[FLASH_MAX_OBS];
  float bounds[FLASH_MAX_OBS][4];   // projected corners, pixel-centre units: umin, umax, vmin, vmax
  int act[FLASH_MAX_OBS];           // 0: invisible; 1: test where the bounds reach; 2: test everywhere
};

__global__ void __launch_bounds__(32) k_rc_prep(RcObs O, const float *__restrict__ cam_poses, RcCam C,
                                                int first_env, EnvPrep *__restrict__ prep) {
  const int e = first_env + blockIdx.x;
  EnvPrep &P = prep[blockIdx.x];
  const float *cp = cam_poses + 7 * (size_t)e;
  if (threadIdx.x == 31) {
    rc_quat_mat(cp + 3, P.Rc);
    P.p[0] = cp[0]; P.p[1] = cp[1]; P.p[2] = cp[2];
    P.ifx = 1.f / C.fx;
    P.ify = 1.f / C.fy;
  }
  if (threadIdx.x >= O.K) return;
  const int k = threadIdx.x;
  const size_t b = (size_t)e * O.stride + k;
  const float *pose = O.pose + 7 * b, *dims = O.dims + 3 * b;
  ObsRay &Q = P.Q[k];
  Q.type = O.type[b];
  float R[9];
  rc_quat_mat(pose + 3, R);
  const float w[3] = {pose[0] - cp[0], pose[1] - cp[1], pose[2] - cp[2]};   // obstacle origin - camera
  if (Q.type == FLASH_OBS_PLANE) {
    Q.a[0] = R[2]; Q.a[1] = R[5]; Q.a[2] = R[8];
    Q.b = R[2] * w[0] + R[5] * w[1] + R[8] * w[2];
  } else if (Q.type == FLASH_OBS_SPHERE) {
    Q.a[0] = w[0]; Q.a[1] = w[1]; Q.a[2] = w[2];
    Q.b = dims[0] * dims[0];
  } else {
    for (int i = 0; i < 3; i++) Q.a[i] = -(R[i] * w[0] + R[3 + i] * w[1] + R[6 + i] * w[2]);
    for (int i = 0; i < 9; i++) Q.R[i] = R[i];
    for (int i = 0; i < 3; i++) Q.h[i] = dims[i];
  }
  // A sphere or box is tested only near its projection, bounded by the
  // projected corners of the box (of the sphere's bounding cube); a shape
  // reaching behind the camera is tested everywhere.
  int act = Q.type == FLASH_OBS_NONE ? 0 : 2;
  if (Q.type == FLASH_OBS_SPHERE || Q.type == FLASH_OBS_BOX) {
    float Rc[9];
    rc_quat_mat(cp + 3, Rc);
    const bool sph = Q.type == FLASH_OBS_SPHERE;
    const float hx = dims[0], hy = sph ? dims[0] : dims[1], hz = sph ? dims[0] : dims[2];
    bool front = true;
    float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    for (int c = 0; c < 8 && front; c++) {
      const float bx = (c & 1) ? hx : -hx, by = (c & 2) ? hy : -hy, bz = (c & 4) ? hz : -hz;
      float x[3];
      for (int i = 0; i < 3; i++)
        x[i] = w[i] + (sph ? (i == 0 ? bx : i == 1 ? by : bz) : R[3 * i] * bx + R[3 * i + 1] * by + R[3 * i + 2] * bz);
      const float yx = Rc[0] * x[0] + Rc[3] * x[1] + Rc[6] * x[2];
      const float yy = Rc[1] * x[0] + Rc[4] * x[1] + Rc[7] * x[2];
      const float yz = Rc[2] * x[0] + Rc[5] * x[1] + Rc[8] * x[2];
      if (!(yz > 0.5f * C.zn)) { front = false; break; }
      const float uc = C.fx * yx / yz + C.cx - 0.5f, vc = C.fy * yy / yz + C.cy - 0.5f;
      umin = fminf(umin, uc); umax = fmaxf(umax, uc);
      vmin = fminf(vmin, vc); vmax = fmaxf(vmax, vc);
    }
    if (front) {
      act = 1;
      P.bounds[k][0] = umin - 1.f; P.bounds[k][1] = umax + 1.f;   // a pixel of slack each way
      P.bounds[k][2] = vmin - 1.f; P.bounds[k][3] = vmax + 1.f;
    }
  }
  P.act[k] = act;
}

__global__ void __launch_bounds__(256) k_rc_resolve(int K, const EnvPrep *__restrict__ prep, RcCam C, int first_env,
                                                    const unsigned long long *__restrict__ keys, unsigned tag,
                                                    float *__restrict__ depth, uint8_t *__restrict__ seg,
                                                    float *__restrict__ pts) {
  // block = a 32 x 8 pixel tile of environment blockIdx.z
  __shared__ EnvPrep P;
  __shared__ int sact[FLASH_MAX_OBS];
  const int e = first_env + blockIdx.z;
  const int WH = C.W * C.H;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  {
    const int *src = reinterpret_cast<const int *>(prep + blockIdx.z);
    int *dst = reinterpret_cast<int *>(&P);
    for (int i = tid; i < (int)(sizeof(EnvPrep) / 4); i += 256) dst[i] = src[i];
  }
  __syncthreads();
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 8;
  if (tid < K) {   // obstacles whose projection reaches this tile
    int act = P.act[tid];
    if (act == 1)
      act = P.bounds[tid][1] >= c0 && P.bounds[tid][0] <= c0 + 31 && P.bounds[tid][3] >= r0 && P.bounds[tid][2] <= r0 + 7;
    sact[tid] = act;
  }
  __syncthreads();
  const int u = c0 + threadIdx.x, v = r0 + threadIdx.y;
  if (u >= C.W || v >= C.H) return;
  const int pix = v * C.W + u;
  const float dx = (u + 0.5f - C.cx) * P.ifx, dy = (v + 0.5f - C.cy) * P.ify;
  const float3 d = make_float3(P.Rc[0] * dx + P.Rc[1] * dy + P.Rc[2], P.Rc[3] * dx + P.Rc[4] * dy + P.Rc[5],
                               P.Rc[6] * dx + P.Rc[7] * dy + P.Rc[8]);
  const size_t pe = (size_t)e * WH + pix;
  const unsigned long long key = keys[pe];
  float best = INFINITY;
  int inst = 0;
  if ((unsigned)(key >> 56) == tag) {   // a hit of this frame
    best = __uint_as_float((unsigned)(key >> 25) & 0x7fffffffu);
    inst = 1;
  }
  for (int k = 0; k < K; k++) {   // ties keep the smaller instance
    if (!sact[k]) continue;
    const float t = ray_obstacle(P.Q[k], d, C.zn);
    if (t <= C.zf && t < best) {
      best = t;
      inst = 2 + k;
    }
  }
  depth[pe] = inst ? best : 0.f;
  if (seg) seg[pe] = (uint8_t)inst;
  if (pts) {
    const float nan = __int_as_float(0x7fc00000);
    pts[3 * pe] = inst ? P.p[0] + best * d.x : nan;
    pts[3 * pe + 1] = inst ? P.p[1] + best * d.y : nan;
    pts[3 * pe + 2] = inst ? P.p[2] + best * d.z : nan;
  }
}

}  // namespace

cudaError_t rc_launch_tri(const RcMesh &M, int n_envs, const float *cam_poses, const RcCam &C,
                          unsigned long long *keys, unsigned tag, cudaStream_t st) {
  if (M.T <= 0 || n_envs <= 0) return cudaSuccess;
  k_rc_tri<<<dim3((M.T + 255) / 256, n_envs), 256, 0, st>>>(M, cam_poses, C, keys, tag);
  return cudaGetLastError();
}

size_t rc_prep_bytes(int n_envs) { return sizeof(EnvPrep) * (size_t)std::max(n_envs, 1); }

cudaError_t rc_launch_resolve(const RcObs &O, const float *cam_poses, const RcCam &C, int first_env, int n_envs,
                              const unsigned long long *keys, unsigned tag, void *prep, float *depth, uint8_t *seg,
                              float *pts, cudaStream_t st) {
  if (n_envs <= 0) return cudaSuccess;
  EnvPrep *P = reinterpret_cast<EnvPrep *>(prep);
  k_rc_prep<<<n_envs, 32, 0, st>>>(O, cam_poses, C, first_env, P);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_rc_resolve<<<dim3((C.W + 31) / 32, (C.H + 7) / 8, n_envs), dim3(32, 8), 0, st>>>(O.K, P, C, first_env, keys, tag,
                                                                                      depth, seg, pts);
  return cudaGetLastError();
}

cudaError_t rc_next_tag(unsigned long long *keys, size_t n_keys, int *tag, cudaStream_t st) {
  if (*tag < 0) {   // tags used up: refill with all ones (tag 255) and restart
    const cudaError_t e = cudaMemsetAsync(keys, 0xff, n_keys * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    *tag = kFirstTag;
  }
  return cudaSuccess;
}

flash_status rc_check_camera(const flash_camera *cam, int64_t n_envs, RcCam *out) {
  if (!cam) { set_error("camera is NULL"); return FLASH_EINVAL; }
  const int64_t W = cam->width, H = cam->height;
  if (W < 1 || H < 1 || W * H > (1 << 26) || H > 8 * 65535 || n_envs * W * H > ((int64_t)1 << 34)) {
    set_error("camera size out of range (1 <= W*H <= 2^26 pixels, H <= 524280, N*W*H <= 2^34)");
    return FLASH_EINVAL;
  }
  const float v[6] = {cam->fx, cam->fy, cam->cx, cam->cy, cam->z_near, cam->z_far};
  for (float x : v)
    if (!std::isfinite(x)) { set_error("camera parameters must be finite"); return FLASH_EINVAL; }
  if (!(cam->fx > 0.f && cam->fy > 0.f) || !(cam->z_near > 0.f && cam->z_near < cam->z_far)) {
    set_error("camera needs fx, fy > 0 and 0 < z_near < z_far");
    return FLASH_EINVAL;
  }
  *out = RcCam{(int)W, (int)H, cam->fx, cam->fy, cam->cx, cam->cy, cam->z_near, cam->z_far};
  return FLASH_OK;
}

}  // namespace flash

struct flash_raycaster {
  flash::RcCam cam{};
  int N = 0, n = 0, T = 0;
  int3 *tris = nullptr;
  unsigned long long *keys = nullptr;
  void *prep = nullptr;   // per-environment view constants
  int tag = flash::kFirstTag;   // frame tag of the next cast
  // per-kernel device time while profiling (0: triangles, 1: resolve)
  bool profiling = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  double prof_ms[2] = {0, 0};
  int64_t prof_n[2] = {0, 0};
};

using flash::set_error;

flash_status flash_raycaster_create(const flash_camera *cam, int32_t n_envs, int32_t n_verts, int32_t n_tris,
                                    const int32_t *tris, flash_raycaster **out) {
  if (!out) { set_error("out is NULL"); return FLASH_EINVAL; }
  *out = nullptr;
  if (n_envs < 1 || n_envs > 65535 || n_verts < 0 || n_tris < 0 || n_tris > flash::kMaxRcTris ||
      (n_tris > 0 && !tris)) {
    set_error("invalid ray caster sizes (1 <= n_envs <= 65535, n_verts >= 0, 0 <= n_tris < 2^25)");
    return FLASH_EINVAL;
  }
  flash::RcCam C;
  flash_status r = flash::rc_check_camera(cam, n_envs, &C);
  if (r != FLASH_OK) return r;
  for (int64_t i = 0; i < 3 * (int64_t)n_tris; i++)
    if (tris[i] < 0 || tris[i] >= n_verts) { set_error("triangle vertex index out of range"); return FLASH_EINVAL; }
  flash_raycaster *rc = new flash_raycaster;
  rc->cam = C;
  rc->N = n_envs; rc->n = n_verts; rc->T = n_tris;
  const size_t keys = (size_t)n_envs * C.W * C.H;
  cudaError_t e = cudaMalloc(&rc->keys, keys * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(rc->keys, 0xff, keys * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();   // the buffer is ready for any stream
  if (e == cudaSuccess) e = cudaMalloc(&rc->prep, flash::rc_prep_bytes(n_envs));
  if (e == cudaSuccess && n_tris > 0) {
    e = cudaMalloc(&rc->tris, sizeof(int3) * n_tris);
    if (e == cudaSuccess) e = cudaMemcpy(rc->tris, tris, sizeof(int3) * n_tris, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    set_error(std::string("ray caster allocation: ") + cudaGetErrorString(e));
    flash_raycaster_destroy(rc);
    return e == cudaErrorMemoryAllocation ? FLASH_ENOMEM : FLASH_ECUDA;
  }
  *out = rc;
  return FLASH_OK;
}

void flash_raycaster_destroy(flash_raycaster *rc) {
  if (!rc) return;
  for (cudaEvent_t e : rc->ev)
    if (e) cudaEventDestroy(e);
  if (rc->tris) cudaFree(rc->tris);
  if (rc->keys) cudaFree(rc->keys);
  if (rc->prep) cudaFree(rc->prep);
  delete rc;
}

flash_status flash_raycast(flash_raycaster *rc, const float *verts, int32_t n_obs, const int32_t *obs_type,
                           const float *obs_dims, const float *obs_poses, const float *cam_poses, float *depth,
                           uint8_t *seg, float *points, void *stream) {
  if (!rc || !depth || !cam_poses || (rc->T > 0 && !verts)) { set_error("invalid arguments"); return FLASH_EINVAL; }
  if (n_obs < 0 || n_obs > FLASH_MAX_OBS || (n_obs > 0 && (!obs_type || !obs_dims || !obs_poses))) {
    set_error("obstacles: 0 <= n_obs <= FLASH_MAX_OBS with type, dims and poses");
    return FLASH_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool prof = rc->profiling;
  if (prof) FLASH_CUDA_TRY(cudaEventRecord(rc->ev[0], st));
  flash::RcMesh M{verts, 3LL * rc->n, 1, 3, nullptr, 0, rc->tris, rc->T};
  FLASH_CUDA_TRY(flash::rc_next_tag(rc->keys, (size_t)rc->N * rc->cam.W * rc->cam.H, &rc->tag, st));
  const unsigned tag = (unsigned)rc->tag;
  FLASH_CUDA_TRY(flash::rc_launch_tri(M, rc->N, cam_poses, rc->cam, rc->keys, tag, st));
  if (prof) FLASH_CUDA_TRY(cudaEventRecord(rc->ev[1], st));
  flash::RcObs O{obs_type, obs_dims, obs_poses, n_obs, n_obs};
  FLASH_CUDA_TRY(
      flash::rc_launch_resolve(O, cam_poses, rc->cam, 0, rc->N, rc->keys, tag, rc->prep, depth, seg, points, st));
  rc->tag--;
  if (prof) {
    FLASH_CUDA_TRY(cudaEventRecord(rc->ev[2], st));
    FLASH_CUDA_TRY(cudaEventSynchronize(rc->ev[2]));
    float a = 0.f, b = 0.f;
    FLASH_CUDA_TRY(cudaEventElapsedTime(&a, rc->ev[0], rc->ev[1]));
    FLASH_CUDA_TRY(cudaEventElapsedTime(&b, rc->ev[1], rc->ev[2]));
    if (rc->T > 0) { rc->prof_ms[0] += a; rc->prof_n[0]++; }
    rc->prof_ms[1] += b;
    rc->prof_n[1]++;
  }
  return FLASH_OK;
}

flash_status flash_raycaster_profile(flash_raycaster *rc, int32_t enable) {
  if (!rc) { set_error("ray caster is NULL"); return FLASH_EINVAL; }
  if (enable && !rc->ev[0])
    for (cudaEvent_t &e : rc->ev) FLASH_CUDA_TRY(cudaEventCreate(&e));
  rc->profiling = enable != 0;
  rc->prof_ms[0] = rc->prof_ms[1] = 0.0;
  rc->prof_n[0] = rc->prof_n[1] = 0;
  return FLASH_OK;
}

flash_status flash_raycaster_profile_read(const flash_raycaster *rc, double *ms, int64_t *launches) {
  if (!rc || !ms || !launches) { set_error("invalid arguments"); return FLASH_EINVAL; }
  for (int k = 0; k < 2; k++) { ms[k] = rc->prof_ms[k]; launches[k] = rc->prof_n[k]; }
  return FLASH_OK;
}
