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

namespace flash {

namespace {

struct GroupView {
  int n, n_pad, E, H, vpe, nc, type, cap;
  const int *genv, *elems, *hv, *v2e_off, *v2e, *v2h_off, *v2h;
  const float *D, *wt, *hc, *mass;
  float *q, *v, *qt, *qp, *r, *f, *w;
  __half *rh, *rl;
  float *rscale;
  int *ccount, *cvert, *cobs, *pcount, *pvert, *pobs;
  float *cgam, *clin, *pgam, *pscratch;
  int p_in_smem;
};

struct EnvView {
  const float *mu, *odims, *ocomp, *pose_t, *pose_th;
  const int *otype;
  int *iters, *done, *status, *active;
  float *rncp;
};

GroupView view(const flash_scene *s, const Group &g) {
  GroupView v;
  v.n = g.n; v.n_pad = g.n_pad; v.E = g.E; v.H = g.H; v.vpe = g.vpe; v.nc = g.nc; v.type = g.type; v.cap = s->cap;
  v.genv = g.genv; v.elems = g.elems; v.hv = g.hv; v.v2e_off = g.v2e_off; v.v2e = g.v2e;
  v.v2h_off = g.v2h_off; v.v2h = g.v2h; v.D = g.D; v.wt = g.wt; v.hc = g.hc; v.mass = g.mass;
  v.q = g.q; v.v = g.v; v.qt = g.qt; v.qp = g.qp; v.r = g.r; v.f = g.f; v.w = g.w;
  v.rh = g.rh; v.rl = g.rl; v.rscale = g.rscale;
  v.ccount = g.ccount; v.cvert = g.cvert; v.cobs = g.cobs; v.pcount = g.pcount; v.pvert = g.pvert;
  v.pobs = g.pobs; v.cgam = g.cgam; v.clin = g.clin; v.pgam = g.pgam; v.pscratch = g.pscratch;
  v.p_in_smem = g.p_in_smem ? 1 : 0;
  return v;
}

EnvView eview(const flash_scene *s) {
  EnvView e;
  e.mu = s->mu; e.odims = s->odims; e.ocomp = s->ocomp; e.pose_t = s->pose_t; e.pose_th = s->pose_th;
  e.otype = s->otype; e.iters = s->iters; e.done = s->done; e.status = s->status; e.active = s->active;
  e.rncp = s->rncp;
  return e;
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

// ---------------------------------------------------------------------------
// begin of step: q_t, q~, detection, gamma^0
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_begin(GroupView G, EnvView V, StepArgs a) {
  __shared__ int sh_scan[32];
  __shared__ int s_type[FLASH_MAX_OBS];
  __shared__ float s_dims[FLASH_MAX_OBS][3], s_pose[FLASH_MAX_OBS][7];
  const int l = blockIdx.x, e = G.genv[l];
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
  __syncthreads();
  const float h = a.h, h2 = a.h * a.h;
  const float gv[3] = {a.gx, a.gy, a.gz};
  int base = 0;
  int *cvert = G.cvert + (size_t)l * G.cap, *cobs = G.cobs + (size_t)l * G.cap;
  for (int i0 = 0; i0 < n; i0 += blockDim.x) {
    int i = i0 + threadIdx.x;
    unsigned mask = 0;
    if (i < n) {
      float x0[3], x1[3];
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
      for (int o = 0; o < a.K; o++) {
        if (s_type[o] == FLASH_OBS_NONE) continue;
        V3 nn;
        float s0 = obstacle_sdf(s_type[o], s_dims[o], s_pose[o], v3(x0[0], x0[1], x0[2]), nn);
        float s1 = obstacle_sdf(s_type[o], s_dims[o], s_pose[o], v3(x1[0], x1[1], x1[2]), nn);
        if (fminf(s0, s1) < a.tau + a.margin) mask |= 1u << o;
      }
    }
    int cnt = __popc(mask), total;
    int off = block_exclusive_scan(cnt, &total, sh_scan);
    int pos = base + off;
    for (int o = 0; o < a.K; o++)
      if (mask & (1u << o)) {
        if (pos < G.cap) { cvert[pos] = i; cobs[pos] = o; }
        pos++;
      }
    base += total;
  }
  if (threadIdx.x == 0) {
    G.ccount[l] = min(base, G.cap);
    if (base > G.cap) atomicOr(V.status, 1 << 8);
  }
  __syncthreads();
  int cnt = min(base, G.cap);
  float *gam = G.cgam + (size_t)l * G.cap * 4;
  const int pc = G.pcount[l];
  const int *pv = G.pvert + (size_t)l * G.cap, *po = G.pobs + (size_t)l * G.cap;
  const float *pg = G.pgam + (size_t)l * G.cap * 4;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    float g4[4] = {0.f, 0.f, 0.f, 0.f};
    if (a.warm == FLASH_WARM_PREV && pc > 0) {
      int key = cvert[j] * FLASH_MAX_OBS + cobs[j];
      int lo = 0, hi = pc - 1;
      while (lo <= hi) {  // previous list is sorted by (vertex, obstacle)
        int mid = (lo + hi) >> 1;
        int km = pv[mid] * FLASH_MAX_OBS + po[mid];
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
__device__ __forceinline__ void store_lin(float *dst, const ContactLin &L) {
  for (int i = 0; i < 9; i++) dst[i] = L.R[i];
  dst[9] = L.phi[0]; dst[10] = L.phi[1]; dst[11] = L.phi[2];
  dst[12] = L.cn;
  for (int i = 0; i < 4; i++) dst[13 + i] = L.Ct[i];
  dst[17] = L.dn; dst[18] = L.dtn[0]; dst[19] = L.dtn[1];
  for (int i = 0; i < 4; i++) dst[20 + i] = L.Dtt[i];
}

// write one environment's three columns in f16 hi/lo with a power-of-two
// scale per column (tensor-core RHS); vals in shared memory [3][n]
__device__ void write_split_columns(const GroupView &G, int l, const float *vals, float *sh_red) {
  const int n = G.n, np = G.n_pad;
  for (int c = 0; c < 3; c++) {
    float m = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, fabsf(vals[c * n + i]));
    m = block_max(m, sh_red);
    int ex = 0;
    if (m > 0.f) {
      frexpf(m, &ex);      // m = f * 2^ex, f in [0.5, 1)
      ex = 14 - ex;        // scaled max in [2^13, 2^14)
    }
    float sc = ldexpf(1.f, ex);
    size_t col = (size_t)(l * 3 + c);
    if (threadIdx.x == 0) G.rscale[col] = ldexpf(1.f, -ex);
    __half *hh = G.rh + col * np, *hl = G.rl + col * np;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
      float x = i < n ? vals[c * n + i] * sc : 0.f;
      __half xh = __float2half_rn(x);
      hh[i] = xh;
      hl[i] = __float2half_rn(x - __half2float(xh));
    }
  }
}

__global__ void __launch_bounds__(512) k_local(GroupView G, EnvView V, StepArgs a, int k, int residual_only,
                                               int tc) {
  extern __shared__ float smem[];
  __shared__ float sh_red[32];
  __shared__ int s_done;
  __shared__ int s_type[FLASH_MAX_OBS];
  __shared__ float s_dims[FLASH_MAX_OBS][3], s_pose[FLASH_MAX_OBS][7], s_poset[FLASH_MAX_OBS][7],
      s_comp[FLASH_MAX_OBS];
  const int l = blockIdx.x, e = G.genv[l];
  const int n = G.n, np = G.n_pad, nc = G.nc, vpe = G.vpe;
  if (V.done[e]) return;
  float *qs = smem;           // [3][n]
  float *rs = qs + 3 * n;     // [3][n]
  float *Ps, *Ss;
  if (G.p_in_smem) {
    Ps = rs + 3 * n;          // [E][nc*3]
    Ss = Ps + (size_t)G.E * nc * 3;  // [H][3]
  } else {
    Ps = G.pscratch + (size_t)l * ((size_t)G.E * nc * 3 + (size_t)G.H * 3);
    Ss = Ps + (size_t)G.E * nc * 3;
  }
  const float *q = G.q + (size_t)l * 3 * np;
  for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
    int c = i / n, j = i - c * n;
    qs[i] = q[c * np + j];
  }
  if (threadIdx.x < a.K) {
    int o = threadIdx.x;
    s_type[o] = V.otype[e * FLASH_MAX_OBS + o];
    s_comp[o] = V.ocomp[e * FLASH_MAX_OBS + o];
    for (int c = 0; c < 3; c++) s_dims[o][c] = V.odims[(e * FLASH_MAX_OBS + o) * 3 + c];
    for (int c = 0; c < 7; c++) {
      s_pose[o][c] = V.pose_th[(e * FLASH_MAX_OBS + o) * 7 + c];
      s_poset[o][c] = V.pose_t[(e * FLASH_MAX_OBS + o) * 7 + c];
    }
  }
  __syncthreads();
  // ---- contacts: linearise at (q^{k-1}, gamma^{k-1}); residual of that iterate
  const int cnt = G.ccount[l];
  const int *cvert = G.cvert + (size_t)l * G.cap, *cobs = G.cobs + (size_t)l * G.cap;
  const float *gam = G.cgam + (size_t)l * G.cap * 4;
  float *lin = G.clin + (size_t)l * G.cap * kLin;
  const float *qt = G.qt + (size_t)l * 3 * np;
  const float mu = V.mu[e];
  float rmax = 0.f;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    int vtx = cvert[j], o = cobs[j];
    ContactLin L;
    linearize_contact(s_type[o], s_dims[o], s_comp[o], s_poset[o], s_pose[o], a.tau, mu, a.h, G.mass[vtx],
                      v3(qs[vtx], qs[n + vtx], qs[2 * n + vtx]), v3(qt[vtx], qt[np + vtx], qt[2 * np + vtx]),
                      gam + 4 * j, L);
    store_lin(lin + (size_t)j * kLin, L);
    rmax = fmaxf(rmax, fmaxf(fabsf(L.phi[0]), fmaxf(fabsf(L.phi[1]), fabsf(L.phi[2]))));
  }
  rmax = block_max(rmax, sh_red);
  if (threadIdx.x == 0) {
    int it = k - 1;
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
  // ---- local projection p_i = closest rotation to F_i = G_i q; store w~(p - F)
  const float h2w = 1.f;  // wt already holds h^2 w_i
  (void)h2w;
  for (int el = threadIdx.x; el < G.E; el += blockDim.x) {
    const int *vi = G.elems + 4 * el;
    const float *D = G.D + 12 * el;
    float F[9], R[9];
    for (int c = 0; c < 3; c++)
      for (int j = 0; j < nc; j++) {
        float s = 0.f;
        for (int aa = 0; aa < vpe; aa++) s += qs[c * n + vi[aa]] * D[aa * 3 + j];
        F[nc * c + j] = s;
      }
    if (nc == 2) closest_rot32(F, R);
    else closest_rot33(F, R);
    float wt = G.wt[el];
    float *P = Ps + (size_t)el * nc * 3;
    for (int t = 0; t < 3 * nc; t++) P[t] = wt * (R[t] - F[t]);
  }
  for (int hh = threadIdx.x; hh < G.H; hh += blockDim.x) {
    const int *vi = G.hv + 4 * hh;
    const float *cc = G.hc + 4 * hh;
    for (int c = 0; c < 3; c++) {
      float s = 0.f;
      for (int aa = 0; aa < 4; aa++) s += cc[aa] * qs[c * n + vi[aa]];
      Ss[hh * 3 + c] = s;
    }
  }
  __syncthreads();
  // ---- residual r = M (q~ - q) + sum G^T w~ (p - G q) - bending
  const float *qp = G.qp + (size_t)l * 3 * np;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float m = G.mass[i];
    float acc[3];
    for (int c = 0; c < 3; c++) acc[c] = m * (qp[c * np + i] - qs[c * n + i]);
    for (int t = G.v2e_off[i]; t < G.v2e_off[i + 1]; t++) {
      int slot = G.v2e[t];
      int el = slot >> 2, aa = slot & 3;
      const float *D = G.D + 12 * el + 3 * aa;
      const float *P = Ps + (size_t)el * nc * 3;
      for (int c = 0; c < 3; c++) {
        float s = 0.f;
        for (int j = 0; j < nc; j++) s += D[j] * P[nc * c + j];
        acc[c] += s;
      }
    }
    for (int t = G.v2h_off[i]; t < G.v2h_off[i + 1]; t++) {
      int slot = G.v2h[t];
      int hh = slot >> 2, aa = slot & 3;
      float cc = G.hc[4 * hh + aa];
      for (int c = 0; c < 3; c++) acc[c] -= cc * Ss[hh * 3 + c];
    }
    for (int c = 0; c < 3; c++) rs[c * n + i] = acc[c];
  }
  __syncthreads();
  // ---- + J^T gamma^{k-1} (frame of q^{k-1}); one thread per vertex run
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    if (j > 0 && cvert[j - 1] == cvert[j]) continue;
    int vtx = cvert[j];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int jj = j; jj < cnt && cvert[jj] == vtx; jj++) {
      const float *L = lin + (size_t)jj * kLin;
      const float *g = gam + 4 * jj;
      float gn = g[0];
      float y1 = L[3] * g[1] + L[4] * g[2] + L[5] * g[3];
      float y2 = L[6] * g[1] + L[7] * g[2] + L[8] * g[3];
      fx += L[0] * gn + L[3] * y1 + L[6] * y2;
      fy += L[1] * gn + L[4] * y1 + L[7] * y2;
      fz += L[2] * gn + L[5] * y1 + L[8] * y2;
    }
    rs[vtx] += fx;
    rs[n + vtx] += fy;
    rs[2 * n + vtx] += fz;
  }
  __syncthreads();
  if (tc) {
    write_split_columns(G, l, rs, sh_red);
  } else {
    float *r = G.r + (size_t)l * 3 * np;
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
      int c = i / n, j = i - c * n;
      r[c * np + j] = rs[i];
    }
  }
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

// rows of D_C (3x3) and D_y (3x3) of one contact from its linearisation
__device__ __forceinline__ void lin_mats(const float *L, float DC[9], float Dy[9]) {
  DC[0] = L[12]; DC[1] = 0.f; DC[2] = 0.f;
  DC[3] = 0.f; DC[4] = L[13]; DC[5] = L[14];
  DC[6] = 0.f; DC[7] = L[15]; DC[8] = L[16];
  Dy[0] = L[17]; Dy[1] = 0.f; Dy[2] = 0.f;
  Dy[3] = L[18]; Dy[4] = L[20]; Dy[5] = L[21];
  Dy[6] = L[19]; Dy[7] = L[22]; Dy[8] = L[23];
}

__global__ void __launch_bounds__(256) k_ncp(GroupView G, EnvView V, StepArgs a, int tc) {
  extern __shared__ float fs[];   // [3][n] contact force (tc path)
  __shared__ float sh_red[32];
  const int l = blockIdx.x, e = G.genv[l];
  const int n = G.n, np = G.n_pad;
  if (V.done[e]) return;
  const int cnt = G.ccount[l];
  const int *cvert = G.cvert + (size_t)l * G.cap;
  float *gam = G.cgam + (size_t)l * G.cap * 4;
  const float *lin = G.clin + (size_t)l * G.cap * kLin;
  const float *q = G.q + (size_t)l * 3 * np, *w = G.w + (size_t)l * 3 * np;
  float *f = G.f + (size_t)l * 3 * np;
  if (tc)
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) fs[i] = 0.f;
  __syncthreads();
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    if (j > 0 && cvert[j - 1] == cvert[j]) continue;
    const int vtx = cvert[j];
    int c = 1;
    while (j + c < cnt && cvert[j + c] == vtx) c++;
    if (c > kMaxPerVertex) {
      atomicOr(V.status, 1 << 10);
      c = kMaxPerVertex;
    }
    const float mv = G.mass[vtx];
    const V3 du = {w[vtx], w[np + vtx], w[2 * np + vtx]};  // u - q^{k-1} = A^-1 r
    const int N3 = 3 * c;
    float Z[12 * 12], rhs[12];
    for (int aa = 0; aa < c; aa++) {
      const float *La = lin + (size_t)(j + aa) * kLin;
      float DC[9], Dy[9];
      lin_mats(La, DC, Dy);
      float Rdu[3] = {La[0] * du.x + La[1] * du.y + La[2] * du.z, La[3] * du.x + La[4] * du.y + La[5] * du.z,
                      La[6] * du.x + La[7] * du.y + La[8] * du.z};
      for (int r = 0; r < 3; r++)
        rhs[3 * aa + r] = -La[9 + r] - (DC[3 * r] * Rdu[0] + DC[3 * r + 1] * Rdu[1] + DC[3 * r + 2] * Rdu[2]);
      for (int bb = 0; bb < c; bb++) {
        const float *Lb = lin + (size_t)(j + bb) * kLin;
        float RR[9];
        for (int r = 0; r < 3; r++)
          for (int cc = 0; cc < 3; cc++)
            RR[3 * r + cc] = La[3 * r] * Lb[3 * cc] + La[3 * r + 1] * Lb[3 * cc + 1] + La[3 * r + 2] * Lb[3 * cc + 2];
        for (int r = 0; r < 3; r++)
          for (int cc = 0; cc < 3; cc++) {
            float s = DC[3 * r] * RR[cc] + DC[3 * r + 1] * RR[3 + cc] + DC[3 * r + 2] * RR[6 + cc];
            if (aa == bb) s += Dy[3 * r + cc] + (r == cc ? kDamp : 0.f);
            Z[(3 * aa + r) * N3 + 3 * bb + cc] = s;
          }
      }
    }
    solve_dense(N3, Z, rhs);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int aa = 0; aa < c; aa++) {
      const float *La = lin + (size_t)(j + aa) * kLin;
      float *g = gam + 4 * (j + aa);
      float dgn = mv * rhs[3 * aa], dg1 = mv * rhs[3 * aa + 1], dg2 = mv * rhs[3 * aa + 2];
      float gn_old = g[0];
      float gn = fminf(gn_old + dgn, a.gmax);
      dgn = gn - gn_old;
      float y1 = La[3] * g[1] + La[4] * g[2] + La[5] * g[3] + dg1;
      float y2 = La[6] * g[1] + La[7] * g[2] + La[8] * g[3] + dg2;
      g[0] = gn;
      g[1] = La[3] * y1 + La[6] * y2;
      g[2] = La[4] * y1 + La[7] * y2;
      g[3] = La[5] * y1 + La[8] * y2;
      // J^T dgamma in the frame of q^{k-1}; the tangential part of gamma^{k-1}
      // was already projected onto that frame in the residual
      fx += La[0] * dgn + La[3] * dg1 + La[6] * dg2;
      fy += La[1] * dgn + La[4] * dg1 + La[7] * dg2;
      fz += La[2] * dgn + La[5] * dg1 + La[8] * dg2;
    }
    if (tc) {
      fs[vtx] = fx; fs[n + vtx] = fy; fs[2 * n + vtx] = fz;
    } else {
      f[vtx] = fx; f[np + vtx] = fy; f[2 * np + vtx] = fz;
    }
  }
  if (tc) {
    __syncthreads();
    write_split_columns(G, l, fs, sh_red);
  }
}

// ---------------------------------------------------------------------------
// end of step: velocity, keep the contact list for warm starts
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_end(GroupView G, EnvView V, StepArgs a) {
  const int l = blockIdx.x, e = G.genv[l];
  const int n = G.n, np = G.n_pad;
  (void)e;
  const float inv_h = 1.f / a.h;
  float *q = G.q + (size_t)l * 3 * np, *v = G.v + (size_t)l * 3 * np;
  const float *qt = G.qt + (size_t)l * 3 * np;
  for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
    int c = i / n, j = i - c * n;
    float qq = q[c * np + j];
    v[c * np + j] = (qq - qt[c * np + j]) * inv_h;
    if (!isfinite(qq)) atomicOr(V.status, 1 << 9);
  }
  const int cnt = G.ccount[l];
  if (threadIdx.x == 0) G.pcount[l] = cnt;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    G.pvert[(size_t)l * G.cap + j] = G.cvert[(size_t)l * G.cap + j];
    G.pobs[(size_t)l * G.cap + j] = G.cobs[(size_t)l * G.cap + j];
    for (int c = 0; c < 4; c++) G.pgam[((size_t)l * G.cap + j) * 4 + c] = G.cgam[((size_t)l * G.cap + j) * 4 + c];
  }
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

__global__ void __launch_bounds__(256) k_split(GroupView G, const float *src) {
  __shared__ float sh_red[32];
  extern __shared__ float vals[];
  const int l = blockIdx.x, n = G.n, np = G.n_pad;
  for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
    int c = i / n, j = i - c * n;
    vals[i] = src[(size_t)l * 3 * np + c * np + j];
  }
  __syncthreads();
  write_split_columns(G, l, vals, sh_red);
}

}  // namespace

cudaError_t configure_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_local, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_ncp, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_split, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
}

cudaError_t launch_begin(const flash_scene *s, const Group &g, const StepArgs &a, cudaStream_t st) {
  k_begin<<<g.N, 256, 0, st>>>(view(s, g), eview(s), a);
  return cudaGetLastError();
}

cudaError_t launch_local(const flash_scene *s, const Group &g, const StepArgs &a, int k, int residual_only, int tc,
                         cudaStream_t st) {
  k_local<<<g.N, 512, g.smem_local, st>>>(view(s, g), eview(s), a, k, residual_only, tc);
  return cudaGetLastError();
}

cudaError_t launch_ncp(const flash_scene *s, const Group &g, const StepArgs &a, int tc, cudaStream_t st) {
  size_t sm = tc ? sizeof(float) * 3 * g.n : 0;
  k_ncp<<<g.N, 256, sm, st>>>(view(s, g), eview(s), a, tc);
  return cudaGetLastError();
}

cudaError_t launch_end(const flash_scene *s, const Group &g, const StepArgs &a, cudaStream_t st) {
  k_end<<<g.N, 256, 0, st>>>(view(s, g), eview(s), a);
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

cudaError_t launch_split_rhs(const Group &g, const float *src, const int *done, cudaStream_t st) {
  (void)done;
  GroupView v;
  memset(&v, 0, sizeof v);
  v.n = g.n; v.n_pad = g.n_pad; v.rh = g.rh; v.rl = g.rl; v.rscale = g.rscale;
  k_split<<<g.N, 256, sizeof(float) * 3 * g.n, st>>>(v, src);
  return cudaGetLastError();
}

}  // namespace flash
