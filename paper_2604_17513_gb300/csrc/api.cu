// Host side of the C ABI: scene description, one-time setup (element data,
// bending stencils, the constant system matrix A = M + h^2 sum w_i G_i^T G_i
// of Sec. III-B and its explicit inverse), state I/O and the per-step
// launch sequence of Algorithm 1.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <tuple>
#include <utility>

#include <nvtx3/nvToolsExt.h>

#include "flash_internal.cuh"

namespace flash {

// NVTX range over a host call (finalize, step, render, ...): profilers can
// select or leave out its launches (e.g. the autotuner's timing launches
// inside "flash.finalize"); a no-op unless a tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

static thread_local std::string g_error;
void set_error(const std::string &msg) { g_error = msg; }

namespace {

flash_status fail(flash_status code, const std::string &msg) {
  set_error(msg);
  return code;
}

template <typename T>
cudaError_t dalloc(flash_scene *s, T **p, size_t count) {
  void *ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  e = cudaMemset(ptr, 0, std::max<size_t>(count, 1) * sizeof(T));
  s->allocs.push_back(ptr);
  *p = (T *)ptr;
  return e;
}

template <typename T>
cudaError_t upload(flash_scene *s, T **p, const std::vector<T> &h) {
  cudaError_t e = dalloc(s, p, h.size());
  if (e != cudaSuccess) return e;
  if (!h.empty()) e = cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// most lanes chosen automatically
constexpr int kMaxAutoLanes = 4, kMaxAutoLanesGroups = 8;
// tolerance mode: iterations between the host's reads of the active count
constexpr int kTolCheck = 4;
// most linear-solver iterations of the full contact metric (the kernels' bound)
constexpr int kMaxLinIters = 32;
constexpr int kFmLinFloats = 22;   // per-contact linearisation record of the full metric

// ---------------------------------------------------------------------------
// element operators: F = Ds Dm^-1 written as F[c][j] = sum_a x_a[c] D[a][j]
// ---------------------------------------------------------------------------
struct ElemData {
  std::vector<double> D;    // [E][12]
  std::vector<double> size; // rest area or volume
};

ElemData element_operators(const MeshTemplate &m) {
  ElemData out;
  out.D.assign((size_t)m.E * 12, 0.0);
  out.size.assign(m.E, 0.0);
  const int vpe = m.type == FLASH_TRI ? 3 : 4;
  for (int e = 0; e < m.E; e++) {
    const int *v = &m.elems[(size_t)e * vpe];
    auto X = [&](int a, int c) { return m.rest[3 * (size_t)v[a] + c]; };
    double *D = &out.D[(size_t)e * 12];
    if (m.type == FLASH_TRI) {
      double e1[3], e2[3];
      for (int c = 0; c < 3; c++) { e1[c] = X(1, c) - X(0, c); e2[c] = X(2, c) - X(0, c); }
      double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
      double b1[3] = {e1[0] / l1, e1[1] / l1, e1[2] / l1};
      double p = e2[0] * b1[0] + e2[1] * b1[1] + e2[2] * b1[2];
      double o[3] = {e2[0] - p * b1[0], e2[1] - p * b1[1], e2[2] - p * b1[2]};
      double lo = std::sqrt(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]);
      // rest edges in the triangle's plane: Dm = [[l1, p], [0, lo]]
      double i00 = 1.0 / l1, i01 = -p / (l1 * lo), i11 = 1.0 / lo;
      double Di[2][2] = {{i00, i01}, {0.0, i11}};
      for (int j = 0; j < 2; j++) {
        D[0 * 3 + j] = -(Di[0][j] + Di[1][j]);
        D[1 * 3 + j] = Di[0][j];
        D[2 * 3 + j] = Di[1][j];
      }
      out.size[e] = 0.5 * l1 * lo;
    } else {
      double M[3][3];
      for (int c = 0; c < 3; c++)
        for (int j = 0; j < 3; j++) M[c][j] = X(j + 1, c) - X(0, c);
      double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                   M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                   M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
      double I[3][3];
      I[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / det;
      I[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
      I[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
      I[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / det;
      I[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
      I[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
      I[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / det;
      I[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
      I[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
      for (int j = 0; j < 3; j++) {
        D[0 * 3 + j] = -(I[0][j] + I[1][j] + I[2][j]);
        for (int a = 0; a < 3; a++) D[(a + 1) * 3 + j] = I[a][j];
      }
      out.size[e] = std::fabs(det) / 6.0;
    }
  }
  return out;
}

// Flat-rest quadratic bending on interior edges.  For the hinge (x0,x1 | x2,
// x3) the stencil k has k2 = |e|^2 / (2 A0), k3 = |e|^2 / (2 A1) and k0, k1
// fixed by annihilating constants and the rest positions along the edge; the
// energy is (w_b / 2) * 3 / (A0 + A1) * |sum_a k_a x_a|^2.
struct Hinges {
  std::vector<int> v;      // [H][4]
  std::vector<double> k;   // [H][4]
  std::vector<double> s;   // [H] 3 / (A0 + A1)
};

Hinges bending_hinges(const MeshTemplate &m) {
  Hinges out;
  if (m.type != FLASH_TRI) return out;
  std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> edges;  // edge -> (tri, opposite)
  for (int t = 0; t < m.E; t++)
    for (int k = 0; k < 3; k++) {
      int a = m.elems[3 * t + k], b = m.elems[3 * t + (k + 1) % 3], o = m.elems[3 * t + (k + 2) % 3];
      edges[{std::min(a, b), std::max(a, b)}].push_back({t, o});
    }
  for (auto &kv : edges) {
    if (kv.second.size() != 2) continue;
    int x[4] = {kv.first.first, kv.first.second, kv.second[0].second, kv.second[1].second};
    auto P = [&](int i, int c) { return m.rest[3 * (size_t)x[i] + c]; };
    double e[3], d2[3], d3[3];
    for (int c = 0; c < 3; c++) { e[c] = P(1, c) - P(0, c); d2[c] = P(2, c) - P(0, c); d3[c] = P(3, c) - P(0, c); }
    double le2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2], le = std::sqrt(le2);
    auto area = [&](const double *d) {
      double c0 = e[1] * d[2] - e[2] * d[1], c1 = e[2] * d[0] - e[0] * d[2], c2 = e[0] * d[1] - e[1] * d[0];
      return 0.5 * std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    };
    double A0 = area(d2), A1 = area(d3);
    double k2 = le2 / (2 * A0), k3 = le2 / (2 * A1);
    double s2 = (d2[0] * e[0] + d2[1] * e[1] + d2[2] * e[2]) / le;
    double s3 = (d3[0] * e[0] + d3[1] * e[1] + d3[2] * e[2]) / le;
    double k1 = -(k2 * s2 + k3 * s3) / le;
    double k0 = -(k1 + k2 + k3);
    for (int i = 0; i < 4; i++) out.v.push_back(x[i]);
    out.k.insert(out.k.end(), {k0, k1, k2, k3});
    out.s.push_back(3.0 / (A0 + A1));
  }
  return out;
}

flash_status build_group(flash_scene *s, Group &g, cudaStream_t st) {
  const MeshTemplate &m = s->meshes[g.mesh];
  const double h = s->d.h, h2 = h * h;
  g.type = m.type; g.n = m.n; g.E = m.E;
  g.tau = (float)(m.thickness >= 0 ? m.thickness : s->d.thickness);
  g.vpe = m.type == FLASH_TRI ? 3 : 4;
  g.nc = m.type == FLASH_TRI ? 2 : 3;
  g.n_pad = round_up(std::max(m.n, 1), 128);
  g.N = (int)g.env_ids.size();
  g.cols = 3 * g.N;
  g.cols_pad = round_up(g.cols, 128);
  const int n = g.n, np = g.n_pad;
  ElemData ed = element_operators(m);
  Hinges hg = bending_hinges(m);
  if (m.w_bend == 0.0) hg = Hinges{};
  g.H = (int)hg.s.size();
  // element arrays
  std::vector<int> el((size_t)m.E * 4, 0);
  std::vector<float> Df((size_t)m.E * 12), wt(m.E);
  for (int e = 0; e < m.E; e++) {
    for (int a = 0; a < g.vpe; a++) el[(size_t)e * 4 + a] = m.elems[(size_t)e * g.vpe + a];
    for (int t = 0; t < 12; t++) Df[(size_t)e * 12 + t] = (float)ed.D[(size_t)e * 12 + t];
    wt[e] = (float)(h2 * m.w_stretch * (g.eig ? 1.0 : g.stiff) * ed.size[e]);
  }
  std::vector<float> massf(np, 0.f);
  for (int i = 0; i < n; i++) massf[i] = (float)m.mass[i];
  std::vector<int> genv(g.env_ids.begin(), g.env_ids.end());
  FLASH_CUDA_TRY(upload(s, &g.genv, genv));
  FLASH_CUDA_TRY(upload(s, &g.elems, el));
  FLASH_CUDA_TRY(upload(s, &g.D, Df));
  FLASH_CUDA_TRY(upload(s, &g.wt, wt));
  if (m.type == FLASH_TRI) {
    std::vector<float> rec((size_t)m.E * 8);
    for (int e = 0; e < m.E; e++) {
      float *r = rec.data() + (size_t)e * 8;
      for (int a = 0; a < 3; a++) std::memcpy(r + a, &el[(size_t)e * 4 + a], sizeof(int));
      r[3] = wt[e];
      r[4] = Df[(size_t)e * 12 + 3]; r[5] = Df[(size_t)e * 12 + 4];
      r[6] = Df[(size_t)e * 12 + 6]; r[7] = Df[(size_t)e * 12 + 7];
    }
    float *d = nullptr;
    FLASH_CUDA_TRY(upload(s, &d, rec));
    g.erec = reinterpret_cast<float4 *>(d);
  }
  FLASH_CUDA_TRY(upload(s, &g.mass, massf));
  {
    // surface triangles for ray casting: the triangles themselves, or the
    // faces that belong to one tetrahedron only (in tetrahedron order)
    std::vector<int> rt;
    if (m.type == FLASH_TRI) {
      rt.assign(m.elems.begin(), m.elems.begin() + (size_t)3 * m.E);
    } else {
      std::map<std::array<int, 3>, int> count;
      auto face = [&](int e, int k) {
        std::array<int, 3> f;
        for (int a = 0, j = 0; a < 4; a++)
          if (a != k) f[j++] = m.elems[(size_t)e * 4 + a];
        return f;
      };
      auto key = [](std::array<int, 3> f) { std::sort(f.begin(), f.end()); return f; };
      for (int e = 0; e < m.E; e++)
        for (int k = 0; k < 4; k++) count[key(face(e, k))]++;
      for (int e = 0; e < m.E; e++)
        for (int k = 0; k < 4; k++) {
          const std::array<int, 3> f = face(e, k);
          if (count[key(f)] == 1) rt.insert(rt.end(), f.begin(), f.end());
        }
    }
    g.rT = (int)(rt.size() / 3);
    if (g.rT > kMaxRcTris) return fail(FLASH_EINVAL, "mesh has too many surface triangles for ray casting");
    if (g.rT > 0) {
      int *d = nullptr;
      FLASH_CUDA_TRY(upload(s, &d, rt));
      g.rtris = reinterpret_cast<int3 *>(d);
    }
  }
  {
    // CSR vertex -> element slots (e * vpe + a), incidence order
    g.ev = m.E * g.vpe;
    if (g.ev > 65534) return fail(FLASH_EINVAL, "mesh has more than 65534 element-vertex slots");
    std::vector<uint16_t> coff((size_t)n + 2, 0), cidx((size_t)g.ev + 1, 0);
    for (int e = 0; e < m.E; e++)
      for (int a = 0; a < g.vpe; a++) coff[el[(size_t)e * 4 + a] + 1]++;
    for (int i = 0; i < n; i++) coff[i + 1] += coff[i];
    std::vector<int> fill(coff.begin(), coff.begin() + n);
    for (int e = 0; e < m.E; e++)
      for (int a = 0; a < g.vpe; a++) cidx[fill[el[(size_t)e * 4 + a]]++] = (uint16_t)(e * g.vpe + a);
    coff.resize(((size_t)n + 2) & ~(size_t)1);      // even length: copied as 4-byte words
    cidx.resize(((size_t)g.ev + 1) & ~(size_t)1);
    FLASH_CUDA_TRY(upload(s, &g.coff, coff));
    FLASH_CUDA_TRY(upload(s, &g.cidx, cidx));
    // bending operator K_b = sum_h c_h k_h k_h^T (c_h = h^2 w_b 3 / (A0 + A1));
    // its rows sum to zero, so the residual uses sum_{j != i} K_ij (q_j - q_i)
    std::vector<std::map<int, double>> rows(n);
    for (int t = 0; t < g.H; t++) {
      const double c = h2 * m.w_bend * hg.s[t];
      for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++)
          if (hg.v[4 * t + a] != hg.v[4 * t + b])
            rows[hg.v[4 * t + a]][hg.v[4 * t + b]] += c * hg.k[4 * t + a] * hg.k[4 * t + b];
    }
    g.deg_b = 0;
    for (int i = 0; i < n; i++) g.deg_b = std::max(g.deg_b, (int)rows[i].size());
    // entries in pairs (2p, 2p + 1) per 16-byte record, pair-major
    // [pairs][n_pad]; unused entries are (i, 0)
    const int pairs = (std::max(g.deg_b, 1) + 1) / 2;
    std::vector<int4> kb((size_t)pairs * np);
    auto bits = [](float f) { int b; std::memcpy(&b, &f, 4); return b; };
    for (int i = 0; i < np; i++)
      for (int p = 0; p < pairs; p++) kb[(size_t)p * np + i] = int4{i < n ? i : 0, 0, i < n ? i : 0, 0};
    for (int i = 0; i < n; i++) {
      int t = 0;
      for (auto &kv : rows[i]) {
        int4 &r = kb[(size_t)(t / 2) * np + i];
        if (t % 2 == 0) { r.x = kv.first; r.y = bits((float)kv.second); }
        else { r.z = kv.first; r.w = bits((float)kv.second); }
        t++;
      }
    }
    FLASH_CUDA_TRY(upload(s, &g.kb, kb));
  }
  if (g.eig) {
    // per-environment stiffness: A_e = M + k_e L with L = h^2 w sum vol D D^T.
    // With B = M^-1/2 L M^-1/2 = W diag(lam) W^T and V = M^-1/2 W,
    // A_e^-1 = V diag(1 / (1 + k_e lam)) V^T.
    std::vector<double> B((size_t)n * n, 0.0);
    for (int e = 0; e < m.E; e++) {
      const double w = h2 * m.w_stretch * ed.size[e];
      const double *D = &ed.D[(size_t)e * 12];
      for (int a = 0; a < g.vpe; a++)
        for (int b = 0; b < g.vpe; b++) {
          double dd = 0;
          for (int j = 0; j < g.nc; j++) dd += D[a * 3 + j] * D[b * 3 + j];
          const int va = el[(size_t)e * 4 + a], vb = el[(size_t)e * 4 + b];
          B[(size_t)va * n + vb] += w * dd / std::sqrt(m.mass[va] * m.mass[vb]);
        }
    }
    std::vector<double> W, lam;
    jacobi_eigen(n, B, W, lam);
    std::vector<double> Vp((size_t)np * np, 0.0), Vtp((size_t)np * np, 0.0);
    std::vector<float> lamf(np, 0.f);
    double vmax = 0;
    for (int i = 0; i < n; i++) {
      const double is = 1.0 / std::sqrt(m.mass[i]);
      for (int j = 0; j < n; j++) {
        const double v = W[(size_t)i * n + j] * is;
        Vp[(size_t)i * np + j] = v;
        Vtp[(size_t)j * np + i] = v;
        vmax = std::max(vmax, std::fabs(v));
      }
    }
    for (int j = 0; j < n; j++) lamf[j] = (float)std::max(lam[j], 0.0);
    int vex = 0;
    std::frexp(vmax, &vex);
    for (SolveMat *Mx : {&g.V, &g.Vt}) {
      Mx->exp = 14 - vex;
      FLASH_CUDA_TRY(dalloc(s, &Mx->f32, (size_t)np * np));
      FLASH_CUDA_TRY(dalloc(s, &Mx->hi, (size_t)np * np));
      FLASH_CUDA_TRY(dalloc(s, &Mx->lo, (size_t)np * np));
      if (s->d.solve == FLASH_SOLVE_BF16R) FLASH_CUDA_TRY(dalloc(s, &Mx->bf, (size_t)np * np));
    }
    double *dV = nullptr;
    FLASH_CUDA_TRY(cudaMalloc(&dV, sizeof(double) * Vp.size()));
    FLASH_CUDA_TRY(cudaMemcpy(dV, Vp.data(), sizeof(double) * Vp.size(), cudaMemcpyHostToDevice));
    FLASH_CUDA_TRY(cast_inverse(dV, np, g.V.f32, g.V.hi, g.V.lo, g.V.exp, st, g.V.bf));
    FLASH_CUDA_TRY(cudaStreamSynchronize(st));
    FLASH_CUDA_TRY(cudaMemcpy(dV, Vtp.data(), sizeof(double) * Vtp.size(), cudaMemcpyHostToDevice));
    FLASH_CUDA_TRY(cast_inverse(dV, np, g.Vt.f32, g.Vt.hi, g.Vt.lo, g.Vt.exp, st, g.Vt.bf));
    FLASH_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(dV);
    FLASH_CUDA_TRY(upload(s, &g.lam, lamf));
    std::vector<float> ke(g.N);
    for (int l = 0; l < g.N; l++) ke[l] = s->envs[g.env_ids[l]].stiffness;
    FLASH_CUDA_TRY(upload(s, &g.kenv, ke));
    FLASH_CUDA_TRY(dalloc(s, &g.y, (size_t)g.cols_pad * np));
  } else {
  // system matrix A (scalar n x n block of A = A_s (x) I3), padded with I
  std::vector<double> A((size_t)np * np, 0.0);
  for (int i = 0; i < np; i++) A[(size_t)i * np + i] = i < n ? m.mass[i] : 1.0;
  for (int e = 0; e < m.E; e++) {
    const double w = h2 * m.w_stretch * g.stiff * ed.size[e];
    const double *D = &ed.D[(size_t)e * 12];
    for (int a = 0; a < g.vpe; a++)
      for (int b = 0; b < g.vpe; b++) {
        double dd = 0;
        for (int j = 0; j < g.nc; j++) dd += D[a * 3 + j] * D[b * 3 + j];
        A[(size_t)el[(size_t)e * 4 + a] * np + el[(size_t)e * 4 + b]] += w * dd;
      }
  }
  for (int t = 0; t < g.H; t++) {
    double c = h2 * m.w_bend * hg.s[t];
    for (int a = 0; a < 4; a++)
      for (int b = 0; b < 4; b++) A[(size_t)hg.v[4 * t + a] * np + hg.v[4 * t + b]] += c * hg.k[4 * t + a] * hg.k[4 * t + b];
  }
  for (int i = 0; i < n; i++)
    if (!(A[(size_t)i * np + i] > 0.0)) return fail(FLASH_ENUMERIC, "system matrix has a non-positive diagonal");
  double *dA = nullptr;
  FLASH_CUDA_TRY(cudaMalloc(&dA, sizeof(double) * A.size()));
  FLASH_CUDA_TRY(cudaMemcpy(dA, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice));
  FLASH_CUDA_TRY(invert_spd_f64(dA, n, np, 1, st));
  FLASH_CUDA_TRY(cudaMemcpyAsync(A.data(), dA, sizeof(double) * A.size(), cudaMemcpyDeviceToHost, st));
  FLASH_CUDA_TRY(cudaStreamSynchronize(st));
  double amax = 0;
  for (double x : A) {
    if (!std::isfinite(x)) { cudaFree(dA); return fail(FLASH_ENUMERIC, "system matrix inverse is not finite"); }
    amax = std::max(amax, std::fabs(x));
  }
  int ex = 0;
  std::frexp(amax, &ex);
  g.inv.exp = 14 - ex;
  FLASH_CUDA_TRY(dalloc(s, &g.inv.f32, (size_t)np * np));
  FLASH_CUDA_TRY(dalloc(s, &g.inv.hi, (size_t)np * np));
  FLASH_CUDA_TRY(dalloc(s, &g.inv.lo, (size_t)np * np));
  if (s->d.solve == FLASH_SOLVE_BF16R) FLASH_CUDA_TRY(dalloc(s, &g.inv.bf, (size_t)np * np));
  FLASH_CUDA_TRY(cast_inverse(dA, np, g.inv.f32, g.inv.hi, g.inv.lo, g.inv.exp, st, g.inv.bf));
  FLASH_CUDA_TRY(cudaStreamSynchronize(st));
  cudaFree(dA);
  }
  // state and contact buffers
  size_t sz = (size_t)g.cols_pad * np;
  FLASH_CUDA_TRY(dalloc(s, &g.q, sz));
  FLASH_CUDA_TRY(dalloc(s, &g.v, sz));
  FLASH_CUDA_TRY(dalloc(s, &g.qt, sz));
  FLASH_CUDA_TRY(dalloc(s, &g.qp, sz));
  FLASH_CUDA_TRY(dalloc(s, &g.r, sz));
  FLASH_CUDA_TRY(dalloc(s, &g.w, sz));
  FLASH_CUDA_TRY(dalloc(s, &g.f, sz));
  FLASH_CUDA_TRY(dalloc(s, &g.dq, sz));
  FLASH_CUDA_TRY(dalloc(s, &g.rh, sz));
  FLASH_CUDA_TRY(dalloc(s, &g.rl, sz));
  FLASH_CUDA_TRY(dalloc(s, &g.rscale, (size_t)g.cols_pad));
  size_t cc = (size_t)g.N * s->cap;
  FLASH_CUDA_TRY(dalloc(s, &g.ccount, (size_t)g.N));
  FLASH_CUDA_TRY(dalloc(s, &g.cvert, cc));
  FLASH_CUDA_TRY(dalloc(s, &g.cobs, cc));
  FLASH_CUDA_TRY(dalloc(s, &g.cgam, cc * 4));
  FLASH_CUDA_TRY(dalloc(s, &g.pcount, (size_t)g.N));
  FLASH_CUDA_TRY(dalloc(s, &g.pvert, cc));
  FLASH_CUDA_TRY(dalloc(s, &g.pobs, cc));
  FLASH_CUDA_TRY(dalloc(s, &g.pgam, cc * 4));
  FLASH_CUDA_TRY(dalloc(s, &g.gflag, (size_t)g.N * np));
  g.selfc = s->d.self_collide && m.type == FLASH_TRI ? 1 : 0;
  g.ofeat = s->d.obstacle_features && m.type == FLASH_TRI ? 1 : 0;
  g.self = g.selfc || g.ofeat ? 1 : 0;
  if (g.self) {
    FLASH_CUDA_TRY(dalloc(s, &g.ctri, cc));
    FLASH_CUDA_TRY(dalloc(s, &g.pctri, cc));
    // unique edges (a < b) in (a, b) order and the range owned by each a
    std::vector<std::pair<int, int>> all;
    all.reserve((size_t)3 * m.E);
    for (int e = 0; e < m.E; e++)
      for (int k = 0; k < 3; k++) {
        const int a = m.elems[(size_t)3 * e + k], b = m.elems[(size_t)3 * e + (k + 1) % 3];
        all.emplace_back(std::min(a, b), std::max(a, b));
      }
    std::sort(all.begin(), all.end());
    all.erase(std::unique(all.begin(), all.end()), all.end());
    g.ned = (int)all.size();
    if ((long long)g.ned * g.ned > 0x7fffffffLL)
      return fail(FLASH_EINVAL, "too many edges for edge-edge self contacts (n_edges^2 must fit in int32)");
    std::vector<int> ed((size_t)2 * std::max(g.ned, 1), 0), eoff((size_t)n + 1, 0);
    for (int k = 0; k < g.ned; k++) {
      ed[2 * k] = all[k].first;
      ed[2 * k + 1] = all[k].second;
      eoff[all[k].first + 1]++;
    }
    for (int i = 0; i < n; i++) eoff[i + 1] += eoff[i];
    int *d = nullptr;
    FLASH_CUDA_TRY(upload(s, &d, ed));
    g.edges = reinterpret_cast<int2 *>(d);
    FLASH_CUDA_TRY(upload(s, &g.eoff, eoff));
  }
  // local pass shared memory: q and r ([3][ns] each, ns = n rounded up to 4),
  // then the element forces [ev + 1][3] (last row zero) and the CSR tables
  const size_t ns = ((size_t)n + 3) & ~(size_t)3;
  const size_t base = sizeof(float) * 6 * ns;
  const size_t forces = sizeof(float) * 3 * ((size_t)g.ev + 1);
  const size_t tables = sizeof(uint16_t) * ((((size_t)n + 2) & ~(size_t)1) + (((size_t)g.ev + 1) & ~(size_t)1));
  if (base + forces + tables <= 200 * 1024) {
    g.c_in_smem = true;
    g.smem_local = base + forces + tables;
  } else {
    g.c_in_smem = false;
    g.smem_local = base;
    if (g.smem_local > 200 * 1024) return fail(FLASH_EINVAL, "mesh too large for one CTA per environment");
    FLASH_CUDA_TRY(dalloc(s, &g.cscratch, 3 * ((size_t)g.ev + 1) * g.N));
  }
  return FLASH_OK;
}

// default input range of the warm-start network: |feature| <= 100
constexpr float kDefaultFeatureBound = 100.f;

cudaError_t ensure_learn_buffers(flash_scene *s) {
  if (!s->ws_bounds) {
    std::vector<float> b(20);
    for (int c = 0; c < 10; c++) { b[c] = -kDefaultFeatureBound; b[10 + c] = kDefaultFeatureBound; }
    cudaError_t e = upload(s, &s->ws_bounds, b);
    if (e != cudaSuccess) return e;
  }
  for (auto &g : s->groups) {
    if (g.row_off) continue;
    size_t rows = (size_t)g.N * s->cap;
    cudaError_t e = dalloc(s, &g.row_off, (size_t)g.N + 1);
    if (e != cudaSuccess) return e;
    if ((e = dalloc(s, &g.feat, rows * 10)) != cudaSuccess) return e;
    if ((e = dalloc(s, &g.pred, rows * 6)) != cudaSuccess) return e;
    if ((e = dalloc(s, &g.targ, rows * 6)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

StepArgs step_args(const flash_scene *s) {
  StepArgs a;
  a.h = (float)s->d.h;
  a.gx = (float)s->d.gravity[0]; a.gy = (float)s->d.gravity[1]; a.gz = (float)s->d.gravity[2];
  a.tol = (float)s->d.tol_ncp;
  a.gmax = (float)(s->d.h * s->d.h * s->d.maxforce);
  a.tau = (float)s->d.thickness;
  a.margin = (float)s->d.margin;
  a.k_min = s->d.k_min; a.k_cap = s->d.k_cap; a.mode = s->d.mode; a.warm = s->d.warm;
  a.K = s->K; a.cap = s->cap;
  return a;
}

bool use_tc(const flash_scene *s) { return s->d.solve == FLASH_SOLVE_F16X3 || s->d.solve == FLASH_SOLVE_BF16R; }

// step arguments of one group (contact thickness is a property of the mesh)
StepArgs group_args(const StepArgs &a, const Group &g) {
  StepArgs ga = a;
  ga.tau = g.tau;
  return ga;
}

cudaEvent_t pool_event(flash_scene *s) {
  if (s->ev_used == s->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    s->ev_pool.push_back(e);
  }
  return s->ev_pool[s->ev_used++];
}

// Launch accounting: counts kernels and, while profiling, brackets the launch
// with a pair of events on the launching stream.
template <typename F>
cudaError_t timed(flash_scene *s, int kind, cudaStream_t st, F &&f) {
  s->launches += 1;
  if (!s->profiling) return f();
  cudaEvent_t e0 = pool_event(s), e1 = pool_event(s);
  if (!e0 || !e1) return cudaErrorMemoryAllocation;
  cudaEventRecord(e0, st);
  cudaError_t r = f();
  cudaEventRecord(e1, st);
  s->ev_kind.push_back(kind);
  return r;
}

cudaError_t flush_profile(flash_scene *s) {
  if (s->ev_kind.empty()) return cudaSuccess;
  cudaError_t e;
  for (size_t i = 0; i < s->ev_kind.size(); i++) {
    float ms = 0.f;
    // pairs may sit on different streams (the lanes of a scene)
    if ((e = cudaEventSynchronize(s->ev_pool[2 * i + 1])) != cudaSuccess) return e;
    e = cudaEventElapsedTime(&ms, s->ev_pool[2 * i], s->ev_pool[2 * i + 1]);
    if (e != cudaSuccess) return e;
    s->prof_ms[s->ev_kind[i]] += ms;
    s->prof_n[s->ev_kind[i]] += 1;
  }
  s->ev_kind.clear();
  s->ev_used = 0;
  return cudaSuccess;
}

// out = A^-1 * (the group's current right-hand side) for environments
// [l0, l1) (l1 < 0: all): r in FP32 (CUDA-core path) or its f16 split
// (tensor-core path); bn is the tile width for that column range
cudaError_t apply_inverse(flash_scene *s, const Group &g, const float *rhs32, float *out, cudaStream_t st, int l0 = 0,
                          int l1 = -1, int bn = 0, const SplitK &sk = SplitK()) {
  const bool tc = use_tc(s);
  if (l1 < 0) l1 = g.N;
  const int c0 = 3 * l0, c1 = 3 * l1;
  if (s->d.solve == FLASH_SOLVE_BF16R) {
    // one bf16 product per contraction (FP32 accumulation), then
    // refine_steps corrections: out += A^-1 (rhs - A out), the residual in
    // FP32 from the element operators (launch_refine)
    auto bf_apply = [&](int mode) -> cudaError_t {   // mode 0: out = A^-1 rh; 3: out += A^-1 rh
      if (!g.eig) return gemm_tc(g, g.inv, out, nullptr, s->done, mode, nullptr, nullptr, st, c0, c1, bn, true, sk);
      cudaError_t e = gemm_tc(g, g.Vt, g.y, nullptr, s->done, 2, g.lam, g.kenv, st, c0, c1, bn, true, sk);
      if (e == cudaSuccess) e = launch_split_rhs(g, g.y, st, l0, l1, true);
      if (e == cudaSuccess) e = gemm_tc(g, g.V, out, nullptr, s->done, mode, nullptr, nullptr, st, c0, c1, bn, true, sk);
      return e;
    };
    cudaError_t e = timed(s, FLASH_KIND_SOLVE, st, [&] { return bf_apply(0); });
    for (int it = 0; it < s->d.refine_steps && e == cudaSuccess; it++) {
      e = timed(s, FLASH_KIND_SOLVE, st, [&] { return launch_refine(s, g, rhs32, out, l0, l1, st); });
      if (e == cudaSuccess) e = timed(s, FLASH_KIND_SOLVE, st, [&] { return bf_apply(3); });
    }
    return e;
  }
  if (!g.eig) {
    return timed(s, FLASH_KIND_SOLVE, st, [&] {
      return tc ? gemm_tc(g, g.inv, out, nullptr, s->done, 0, nullptr, nullptr, st, c0, c1, bn, false, sk)
                : gemm_simt(g, g.inv, rhs32, out, nullptr, s->done, 0, nullptr, nullptr, st, c0, c1);
    });
  }
  // eigen form: y = diag(1/(1 + k_e lam)) V^T rhs, out = V y
  // (the CUDA-core kernel reads its matrix transposed, so it is given V for V^T and V^T for V)
  cudaError_t e = timed(s, FLASH_KIND_SOLVE, st, [&] {
    return tc ? gemm_tc(g, g.Vt, g.y, nullptr, s->done, 2, g.lam, g.kenv, st, c0, c1, bn, false, sk)
              : gemm_simt(g, g.V, rhs32, g.y, nullptr, s->done, 2, g.lam, g.kenv, st, c0, c1);
  });
  if (e != cudaSuccess) return e;
  if (tc) {
    e = timed(s, FLASH_KIND_SOLVE, st, [&] { return launch_split_rhs(g, g.y, st, l0, l1); });
    if (e != cudaSuccess) return e;
  }
  return timed(s, FLASH_KIND_SOLVE, st, [&] {
    return tc ? gemm_tc(g, g.V, out, nullptr, s->done, 0, nullptr, nullptr, st, c0, c1, bn, false, sk)
              : gemm_simt(g, g.Vt, g.y, out, nullptr, s->done, 0, nullptr, nullptr, st, c0, c1);
  });
}

// Lanes: every lane's work of a phase is ordered after everything already on
// the caller's stream (fork) and before anything issued to it next (join).
// A single-lane scene runs on the caller's stream directly.
cudaStream_t lane_stream(const Lane &L, cudaStream_t st) { return L.st ? L.st : st; }

cudaError_t fork(flash_scene *s, cudaStream_t st) {
  if (s->lanes.size() < 2) return cudaSuccess;
  cudaError_t e = cudaEventRecord(s->fork_ev, st);
  for (size_t i = 0; i < s->lanes.size() && e == cudaSuccess; i++) e = cudaStreamWaitEvent(s->lanes[i].st, s->fork_ev, 0);
  return e;
}

cudaError_t join(flash_scene *s, cudaStream_t st) {
  if (s->lanes.size() < 2) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < s->lanes.size() && e == cudaSuccess; i++) {
    e = cudaEventRecord(s->lanes[i].done, s->lanes[i].st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->lanes[i].done, 0);
  }
  return e;
}

// One lane's global applies of a phase, out_g = A_g^-1 in_g over its ranges;
// kind names the output (0: w, 1: dq, 2: fm_u) for the grouped launch, which
// covers the lane's dense-inverse ranges when the scene chose it.
template <typename In, typename Out>
cudaError_t apply_lane(flash_scene *s, const Lane &L, cudaStream_t st, In in, Out out, int kind) {
  cudaError_t e = cudaSuccess;
  const bool grouped = s->grouped && L.ga.n > 0 && use_tc(s);
  if (grouped)
    e = timed(s, FLASH_KIND_SOLVE, st, [&] {
      return gemm_tc_grouped(L.ga.probs, L.ga.n, L.ga.tiles, L.ga.outs[kind], s->done, s->status, st);
    });
  for (size_t i = 0; i < L.ranges.size() && e == cudaSuccess; i++) {
    if (grouped && std::find(L.ga.ranges.begin(), L.ga.ranges.end(), (int)i) != L.ga.ranges.end()) continue;
    const LaneRange &r = L.ranges[i];
    Group &g = s->groups[r.group];
    SplitK sk = L.sk;
    sk.split = r.tc_split;
    e = apply_inverse(s, g, in(g), out(g), st, r.l0, r.l1, r.tc_bn, sk);
  }
  return e;
}

// The grouped apply of every lane with two or more dense-inverse ranges:
// problem tables (tensor maps encoded once) and per-kind output tables.
flash_status build_grouped(flash_scene *s) {
  for (Lane &L : s->lanes) {
    std::vector<int> idx;
    for (size_t i = 0; i < L.ranges.size(); i++)
      if (!s->groups[L.ranges[i].group].eig) idx.push_back((int)i);
    if (idx.size() < 2) continue;
    const size_t pb = gemm_problem_bytes();
    std::vector<unsigned char> host(pb * idx.size());
    std::vector<float *> outs[3];
    int tiles = 0;
    for (size_t k = 0; k < idx.size(); k++) {
      const LaneRange &r = L.ranges[idx[k]];
      Group &g = s->groups[r.group];
      const int t = gemm_problem(host.data() + k * pb, g, g.inv, 3 * r.l0, 3 * r.l1, tiles);
      if (t < 0) return fail(FLASH_ECUDA, "grouped apply: tensor map encoding failed");
      tiles += t;
      outs[0].push_back(g.w);
      outs[1].push_back(g.dq);
      outs[2].push_back(g.fm_u);
    }
    unsigned char *d = nullptr;
    FLASH_CUDA_TRY(upload(s, &d, host));
    L.ga.probs = d;
    for (int kd = 0; kd < 3; kd++) FLASH_CUDA_TRY(upload(s, &L.ga.outs[kd], outs[kd]));
    L.ga.n = (int)idx.size();
    L.ga.tiles = tiles;
    L.ga.ranges = idx;
  }
  return FLASH_OK;
}

// Device time of one phase of every lane's applies running concurrently
// (the best of three runs after a warm-up run).
cudaError_t apply_phase_ms(flash_scene *s, cudaStream_t st, float *best_ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  float t = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = fork(s, st);
    for (const Lane &L : s->lanes)
      if (e == cudaSuccess)
        e = apply_lane(s, L, lane_stream(L, st), [](Group &g) { return g.r; }, [](Group &g) { return g.w; }, 0);
    if (e == cudaSuccess) e = join(s, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) t = std::min(t, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_ms = t;
  return e;
}

}  // namespace

// Cyclic Jacobi eigenvalue iteration: rotate away each off-diagonal entry in
// turn until the off-diagonal mass is negligible; W accumulates the rotations.
void jacobi_eigen(int n, std::vector<double> &B, std::vector<double> &W, std::vector<double> &lam) {
  W.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; i++) W[(size_t)i * n + i] = 1.0;
  double total = 0;
  for (double x : B) total += x * x;
  for (int sweep = 0; sweep < 50; sweep++) {
    double off = 0;
    for (int p = 0; p < n; p++)
      for (int q = p + 1; q < n; q++) off += B[(size_t)p * n + q] * B[(size_t)p * n + q];
    if (off <= 1e-30 * total) break;
    for (int p = 0; p < n - 1; p++)
      for (int q = p + 1; q < n; q++) {
        const double bpq = B[(size_t)p * n + q];
        if (std::fabs(bpq) < 1e-300) continue;
        const double theta = (B[(size_t)q * n + q] - B[(size_t)p * n + p]) / (2.0 * bpq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; k++) {   // columns p, q
          const double bkp = B[(size_t)k * n + p], bkq = B[(size_t)k * n + q];
          B[(size_t)k * n + p] = c * bkp - sn * bkq;
          B[(size_t)k * n + q] = sn * bkp + c * bkq;
        }
        for (int k = 0; k < n; k++) {   // rows p, q
          const double bpk = B[(size_t)p * n + k], bqk = B[(size_t)q * n + k];
          B[(size_t)p * n + k] = c * bpk - sn * bqk;
          B[(size_t)q * n + k] = sn * bpk + c * bqk;
        }
        for (int k = 0; k < n; k++) {
          const double wkp = W[(size_t)k * n + p], wkq = W[(size_t)k * n + q];
          W[(size_t)k * n + p] = c * wkp - sn * wkq;
          W[(size_t)k * n + q] = sn * wkp + c * wkq;
        }
      }
  }
  lam.resize(n);
  for (int i = 0; i < n; i++) lam[i] = B[(size_t)i * n + i];
}

}  // namespace flash

using namespace flash;

extern "C" {

const char *flash_last_error(void) { return g_error.c_str(); }

flash_status flash_scene_create(const flash_scene_desc *desc, flash_scene **out) {
  if (!desc || !out) return fail(FLASH_EINVAL, "null argument");
  if (!(desc->h > 0) || desc->k_max < 0 || desc->k_cap < 0 || desc->k_min < 0 || desc->contact_cap < 0 ||
      desc->grouped_solve < FLASH_GROUPED_AUTO || desc->grouped_solve > FLASH_GROUPED_ON)
    return fail(FLASH_EINVAL, "invalid scene descriptor");
  if (desc->mode != FLASH_MODE_FIXED && desc->mode != FLASH_MODE_TOL) return fail(FLASH_EINVAL, "invalid mode");
  if (desc->solve != FLASH_SOLVE_F32 && desc->solve != FLASH_SOLVE_F16X3 && desc->solve != FLASH_SOLVE_BF16R)
    return fail(FLASH_EINVAL, "invalid solve");
  if (desc->refine_steps < 0 || desc->refine_steps > 4) return fail(FLASH_EINVAL, "refine_steps must be in 0..4");
  if (desc->local_threads != 0 && desc->local_threads != FLASH_THREADS_TUNE && desc->local_threads != 256 &&
      desc->local_threads != 512 && desc->local_threads != 1024)
    return fail(FLASH_EINVAL, "local_threads must be 0, -1 (tune), 256, 512 or 1024");
  if (desc->ncp_threads != 0 && desc->ncp_threads != FLASH_THREADS_TUNE && desc->ncp_threads != 128 &&
      desc->ncp_threads != 256 && desc->ncp_threads != 512)
    return fail(FLASH_EINVAL, "ncp_threads must be 0, -1 (tune), 128, 256 or 512");
  if (desc->split_k < FLASH_SPLITK_AUTO || desc->split_k > FLASH_SPLITK_ON)
    return fail(FLASH_EINVAL, "split_k must be 0 (auto), 1 (off) or 2 (on)");
  if (desc->warm < FLASH_WARM_COLD || desc->warm > FLASH_WARM_LEARNED) return fail(FLASH_EINVAL, "invalid warm start");
  if (desc->metric != FLASH_METRIC_LITE && desc->metric != FLASH_METRIC_FULL) return fail(FLASH_EINVAL, "invalid metric");
  if (desc->lin_iters < 0 || desc->lin_iters > kMaxLinIters) return fail(FLASH_EINVAL, "lin_iters must be 0..32");
  if (desc->self_collide != 0 && desc->self_collide != 1) return fail(FLASH_EINVAL, "self_collide must be 0 or 1");
  if (desc->self_collide && desc->metric != FLASH_METRIC_FULL)
    return fail(FLASH_EINVAL, "cloth self-collision needs the full metric (FLASH_METRIC_FULL)");
  if (desc->obstacle_features != 0 && desc->obstacle_features != 1)
    return fail(FLASH_EINVAL, "obstacle_features must be 0 or 1");
  if (desc->obstacle_features && desc->metric != FLASH_METRIC_FULL)
    return fail(FLASH_EINVAL, "box-feature contacts need the full metric (FLASH_METRIC_FULL)");
  flash_scene *s = new flash_scene();
  s->d = *desc;
  if (s->d.lin_iters == 0) s->d.lin_iters = 10;
  s->cap = desc->contact_cap;
  *out = s;
  return FLASH_OK;
}

flash_status flash_mesh_add(flash_scene *s, const flash_mesh_desc *m, int32_t *mesh_id) {
  if (!s || !m) return fail(FLASH_EINVAL, "null argument");
  if (s->finalized) return fail(FLASH_ESTATE, "scene already finalized");
  if ((m->type != FLASH_TRI && m->type != FLASH_TET) || m->n_verts <= 0 || m->n_elems < 0 || !m->rest || !m->mass ||
      (m->n_elems > 0 && !m->elems))
    return fail(FLASH_EINVAL, "invalid mesh descriptor");
  MeshTemplate t;
  t.type = m->type; t.n = m->n_verts; t.E = m->n_elems;
  t.rest.assign(m->rest, m->rest + 3 * (size_t)m->n_verts);
  t.mass.assign(m->mass, m->mass + m->n_verts);
  int vpe = m->type == FLASH_TRI ? 3 : 4;
  t.elems.assign(m->elems, m->elems + (size_t)vpe * m->n_elems);
  for (int x : t.elems)
    if (x < 0 || x >= t.n) return fail(FLASH_EINVAL, "element index out of range");
  for (double x : t.mass)
    if (!(x > 0)) return fail(FLASH_EINVAL, "vertex mass must be positive");
  t.w_stretch = m->w_stretch; t.w_bend = m->w_bend;
  t.thickness = m->thickness;
  s->meshes.push_back(std::move(t));
  if (mesh_id) *mesh_id = (int32_t)s->meshes.size() - 1;
  return FLASH_OK;
}

flash_status flash_envs_add(flash_scene *s, int32_t mesh_id, int32_t n, const flash_env_desc *envs,
                            int32_t *first_env) {
  if (!s || !envs || n <= 0) return fail(FLASH_EINVAL, "invalid arguments");
  if (s->finalized) return fail(FLASH_ESTATE, "scene already finalized");
  if (mesh_id < 0 || mesh_id >= (int)s->meshes.size()) return fail(FLASH_EINVAL, "unknown mesh");
  for (int i = 0; i < n; i++) {
    if (envs[i].n_obs < 0 || envs[i].n_obs > FLASH_MAX_OBS) return fail(FLASH_EINVAL, "too many obstacles");
    for (int o = 0; o < envs[i].n_obs; o++)
      if (envs[i].obs_type[o] < FLASH_OBS_NONE || envs[i].obs_type[o] > FLASH_OBS_BOX)
        return fail(FLASH_EINVAL, "unknown obstacle type");
  }
  if (first_env) *first_env = (int32_t)s->envs.size();
  for (int i = 0; i < n; i++) {
    s->envs.push_back(envs[i]);
    s->env_mesh.push_back(mesh_id);
  }
  return FLASH_OK;
}

flash_status flash_scene_finalize(flash_scene *s, void *stream) {
  NvtxRange range("flash.finalize");
  if (!s) return fail(FLASH_EINVAL, "null scene");
  if (s->finalized) return fail(FLASH_ESTATE, "scene already finalized");
  if (s->envs.empty()) return fail(FLASH_EINVAL, "no environments");
  cudaStream_t st = (cudaStream_t)stream;
  FLASH_CUDA_TRY(configure_kernels());
  s->N = (int)s->envs.size();
  s->K = 0;
  for (auto &e : s->envs) s->K = std::max(s->K, (int)e.n_obs);
  // groups: one per (mesh, stiffness); a mesh without bending whose
  // environments use several stiffness scales gets one eigen-form group
  std::map<int, std::vector<float>> mesh_stiff;
  for (int e = 0; e < s->N; e++) {
    auto &v = mesh_stiff[s->env_mesh[e]];
    if (std::find(v.begin(), v.end(), s->envs[e].stiffness) == v.end()) v.push_back(s->envs[e].stiffness);
  }
  auto use_eig = [&](int mesh) {
    const MeshTemplate &m = s->meshes[mesh];
    return m.w_bend == 0.0 && mesh_stiff[mesh].size() > 1 && m.n <= 2048;
  };
  std::map<std::pair<int, float>, int> key;
  s->env_group.resize(s->N);
  s->env_local.resize(s->N);
  for (int e = 0; e < s->N; e++) {
    const int mesh = s->env_mesh[e];
    const bool eig = use_eig(mesh);
    auto k = std::make_pair(mesh, eig ? -1.f : s->envs[e].stiffness);
    auto it = key.find(k);
    int gi;
    if (it == key.end()) {
      gi = (int)s->groups.size();
      key[k] = gi;
      Group g;
      g.mesh = mesh;
      g.stiff = k.second;
      g.eig = eig;
      s->groups.push_back(g);
    } else {
      gi = it->second;
    }
    s->env_group[e] = gi;
    s->env_local[e] = (int)s->groups[gi].env_ids.size();
    s->groups[gi].env_ids.push_back(e);
  }
  if (use_tc(s) && !tc_available())
    return fail(FLASH_ENOTIMPL, "tensor-core solve needs an sm_103 device and the TMA driver entry point");
  if (s->d.solve == FLASH_SOLVE_BF16R)
    for (const auto &m : s->meshes)
      if (m.type != FLASH_TET)
        return fail(FLASH_ENOTIMPL, "the bf16 solve with refinement needs a well-conditioned system matrix (tet "
                                    "meshes); a cloth's (condition ~1e7) makes every refinement step grow the error");
  FLASH_CUDA_TRY(dalloc(s, &s->status, 1));
  s->voff.assign(s->N + 1, 0);
  for (int e = 0; e < s->N; e++) s->voff[e + 1] = s->voff[e] + s->meshes[s->env_mesh[e]].n;
  for (auto &g : s->groups) {
    g.status = s->status;
    flash_status r = build_group(s, g, st);
    if (r != FLASH_OK) return r;
    if (s->d.metric == FLASH_METRIC_FULL) {
      // full metric: per-contact linearisation, Krylov basis, Hessenberg
      // matrix, rotations, diag(A^-1), and the output of the Krylov applies
      const int m = s->d.lin_iters;
      const size_t cc = (size_t)g.N * s->cap;
      g.fm_m = m;
      FLASH_CUDA_TRY(dalloc(s, &g.fm_lin, cc * kFmLinFloats));
      if (g.self) FLASH_CUDA_TRY(dalloc(s, &g.fm_w, cc * kFmW));
      FLASH_CUDA_TRY(dalloc(s, &g.fm_V, (size_t)(m + 1) * 3 * cc));
      FLASH_CUDA_TRY(dalloc(s, &g.fm_H, (size_t)g.N * (m + 1) * m));
      FLASH_CUDA_TRY(dalloc(s, &g.fm_cs, (size_t)g.N * m));
      FLASH_CUDA_TRY(dalloc(s, &g.fm_sn, (size_t)g.N * m));
      FLASH_CUDA_TRY(dalloc(s, &g.fm_g, (size_t)g.N * (m + 1)));
      FLASH_CUDA_TRY(dalloc(s, &g.fm_beta, (size_t)g.N));
      FLASH_CUDA_TRY(dalloc(s, &g.fm_jm, (size_t)g.N));
      FLASH_CUDA_TRY(dalloc(s, &g.fm_u, (size_t)g.cols_pad * g.n_pad));
      g.fm_adiag_stride = g.eig ? g.n_pad : 0;
      FLASH_CUDA_TRY(dalloc(s, &g.fm_adiag, g.eig ? (size_t)g.N * g.n_pad : (size_t)g.n_pad));
      FLASH_CUDA_TRY(launch_fm_adiag(g, st));
    }
  }
  // self-collision: the begin kernel keeps every triangle's and edge's box
  // in shared memory when the largest triangle mesh fits (else it tests
  // every pair)
  if (s->d.self_collide) {
    size_t need = 0;
    for (const Group &g : s->groups)
      if (g.selfc) need = std::max(need, sizeof(float) * 6 * ((size_t)g.E + g.ned));
    s->begin_smem = need <= (size_t)kMaxBeginSmem ? need : 0;
  }
  // env-level arrays
  std::vector<float> mu(s->N), odims((size_t)s->N * FLASH_MAX_OBS * 3, 0.f), ocomp((size_t)s->N * FLASH_MAX_OBS, 0.f);
  std::vector<int> otype((size_t)s->N * FLASH_MAX_OBS, 0);
  std::vector<float> pose((size_t)s->N * FLASH_MAX_OBS * 7, 0.f);
  for (int e = 0; e < s->N; e++) {
    const flash_env_desc &d = s->envs[e];
    mu[e] = d.mu;
    for (int o = 0; o < d.n_obs; o++) {
      otype[e * FLASH_MAX_OBS + o] = d.obs_type[o];
      ocomp[e * FLASH_MAX_OBS + o] = d.obs_compliance[o];
      for (int c = 0; c < 3; c++) odims[(e * FLASH_MAX_OBS + o) * 3 + c] = d.obs_dims[o][c];
    }
    for (int o = 0; o < FLASH_MAX_OBS; o++) pose[(e * FLASH_MAX_OBS + o) * 7 + 3] = 1.f;
  }
  FLASH_CUDA_TRY(upload(s, &s->mu, mu));
  FLASH_CUDA_TRY(upload(s, &s->otype, otype));
  FLASH_CUDA_TRY(upload(s, &s->odims, odims));
  FLASH_CUDA_TRY(upload(s, &s->ocomp, ocomp));
  FLASH_CUDA_TRY(upload(s, &s->pose_t, pose));
  FLASH_CUDA_TRY(upload(s, &s->pose_th, pose));
  FLASH_CUDA_TRY(dalloc(s, &s->iters, (size_t)s->N));
  FLASH_CUDA_TRY(dalloc(s, &s->done, (size_t)s->N));
  FLASH_CUDA_TRY(dalloc(s, &s->rncp, (size_t)s->N));
  FLASH_CUDA_TRY(dalloc(s, &s->active, 1));
  FLASH_CUDA_TRY(dalloc(s, &s->kit, 1));
  FLASH_CUDA_TRY(dalloc(s, &s->trips, 1));
  FLASH_CUDA_TRY(dalloc(s, &s->gstate, (size_t)s->N));
  FLASH_CUDA_TRY(upload(s, &s->gobs, std::vector<int>(s->N, -1)));
  FLASH_CUDA_TRY(dalloc(s, &s->greq, (size_t)s->N));
  FLASH_CUDA_TRY(dalloc(s, &s->ganchor, (size_t)s->N * 4));
  FLASH_CUDA_TRY(upload(s, &s->d_voff, s->voff));
  FLASH_CUDA_TRY(cudaMallocHost(&s->h_active, sizeof(int)));
  // lanes: explicit count, or about one per 256 environments (at most 4):
  // a lane needs enough CTAs to fill a good part of the GPU by itself;
  // several mesh groups: one lane per group up to kMaxAutoLanesGroups (the
  // lanes are what runs the groups' small contractions concurrently)
  int n_lanes = s->d.lanes > 0 ? s->d.lanes
                : s->groups.size() > 1 ? std::min<int>(kMaxAutoLanesGroups, (int)s->groups.size())
                                       : std::max(1, std::min(kMaxAutoLanes, s->N / 256));
  FLASH_CUDA_TRY(build_lanes(s, n_lanes));
  if (s->lanes.size() > 1) {
    FLASH_CUDA_TRY(cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming));
    for (Lane &L : s->lanes) {
      FLASH_CUDA_TRY(cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking));
      FLASH_CUDA_TRY(cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming));
    }
  }
  if (use_tc(s)) {
    // split-K scratch per lane, for the largest of its column ranges
    for (Lane &L : s->lanes) {
      if (s->d.split_k == FLASH_SPLITK_OFF) break;
      size_t tiles = 0, part = 0;
      for (const LaneRange &r : L.ranges) {
        size_t t = 0, p = 0;
        splitk_need(s->groups[r.group], 3 * r.l0, 3 * r.l1, &t, &p);
        tiles = std::max(tiles, t);
        part = std::max(part, p);
      }
      if (!tiles) continue;
      FLASH_CUDA_TRY(dalloc(s, &L.sk.part, part));
      FLASH_CUDA_TRY(dalloc(s, &L.sk.sem, tiles));
      FLASH_CUDA_TRY(cudaMemset(L.sk.sem, 0, tiles * sizeof(int)));
      L.sk.tiles = tiles;
      L.sk.part_floats = part;
    }
    // tile autotuner: each group's full column range (global applies, one
    // CTA per tile) and each lane's range (the step, split-K as well), timed
    // once per distinct column count
    std::map<std::tuple<int, int, int>, std::pair<int, int>> tuned;
    auto tune = [&](int gi, int l0, int l1, const SplitK &sk) -> std::pair<int, int> {
      const auto key = std::make_tuple(gi, l1 - l0, sk.part ? sk.split : -1);
      auto it = tuned.find(key);
      if (it != tuned.end()) return it->second;
      int bn = 128, split = 1;
      if (tune_gemm_tc(s->groups[gi], s->done, st, 3 * l0, 3 * l1, &bn, &split, sk) != cudaSuccess) bn = -1;
      tuned[key] = std::make_pair(bn, split);
      return tuned[key];
    };
    for (size_t gi = 0; gi < s->groups.size(); gi++) {
      const int bn = tune((int)gi, 0, s->groups[gi].N, SplitK()).first;
      if (bn < 0) return fail(FLASH_ECUDA, "tile autotuner failed");
      s->groups[gi].tc_bn = bn;
    }
    for (Lane &L : s->lanes)
      for (LaneRange &r : L.ranges) {
        // FLASH_SPLITK_ON times the widths as split-K only
        SplitK sk = L.sk;
        sk.split = s->d.split_k == FLASH_SPLITK_ON ? 2 : 0;
        const auto c = tune(r.group, r.l0, r.l1, sk);
        if (c.first < 0) return fail(FLASH_ECUDA, "tile autotuner failed");
        r.tc_bn = c.first;
        r.tc_split = c.second;
      }
    if (s->lanes.size() > 1) {
      // lanes run their contractions at the same time, which the per-range
      // timings above do not see: time one phase of every lane's applies
      // running concurrently for those choices and for each uniform width,
      // and keep the fastest configuration
      const int64_t launches0 = s->launches;
      cudaEvent_t e0, e1;
      FLASH_CUDA_TRY(cudaEventCreate(&e0));
      FLASH_CUDA_TRY(cudaEventCreate(&e1));
      auto phase_ms = [&](float *best_ms) -> cudaError_t {
        float t = 1e30f;
        for (int rep = 0; rep < 4; rep++) {
          cudaError_t e = cudaEventRecord(e0, st);
          if (e == cudaSuccess) e = fork(s, st);
          for (const Lane &L : s->lanes)
            if (e == cudaSuccess)
              e = apply_lane(s, L, lane_stream(L, st), [](Group &g) { return g.r; }, [](Group &g) { return g.w; }, 0);
          if (e == cudaSuccess) e = join(s, st);
          if (e == cudaSuccess) e = cudaEventRecord(e1, st);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          if (e != cudaSuccess) return e;
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) t = std::min(t, ms);     // the first run warms up
        }
        *best_ms = t;
        return cudaSuccess;
      };
      std::vector<std::pair<int, int>> chosen;
      for (const Lane &L : s->lanes)
        for (const LaneRange &r : L.ranges) chosen.push_back(std::make_pair(r.tc_bn, r.tc_split));
      float best = 0.f;
      FLASH_CUDA_TRY(phase_ms(&best));
      const int split0 = s->d.split_k == FLASH_SPLITK_ON ? 2 : 1, split1 = s->d.split_k == FLASH_SPLITK_AUTO ? 2 : split0;
      for (int split = split0; split <= split1; split++)
        for (int bn : {64, 128, 176, 256}) {
          for (Lane &L : s->lanes)
            for (LaneRange &r : L.ranges) {
              r.tc_bn = bn;
              r.tc_split = split;
            }
          float t = 0.f;
          FLASH_CUDA_TRY(phase_ms(&t));
          if (t < best) {
            best = t;
            chosen.assign(chosen.size(), std::make_pair(bn, split));
          }
        }
      size_t k = 0;
      for (Lane &L : s->lanes)
        for (LaneRange &r : L.ranges) {
          r.tc_bn = chosen[k].first;
          r.tc_split = chosen[k++].second;
        }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      s->launches = launches0;
    }
    // lanes of several mesh templates: one grouped launch for all their
    // dense applies (f16 hi/lo solve), kept if it beats the per-range launches
    const flash_status gs = s->d.solve == FLASH_SOLVE_F16X3 ? build_grouped(s) : FLASH_OK;
    if (gs != FLASH_OK) return gs;
    bool any = false;
    for (const Lane &L : s->lanes) any = any || L.ga.n > 0;
    if (any && s->d.grouped_solve == FLASH_GROUPED_ON) {
      s->grouped = true;
    } else if (any && s->d.grouped_solve == FLASH_GROUPED_AUTO) {
      const int64_t launches0 = s->launches;
      float t_off = 0.f, t_on = 0.f;
      s->grouped = false;
      FLASH_CUDA_TRY(apply_phase_ms(s, st, &t_off));
      s->grouped = true;
      FLASH_CUDA_TRY(apply_phase_ms(s, st, &t_on));
      s->grouped = t_on < t_off;
      s->launches = launches0;
    }
  }
  FLASH_CUDA_TRY(cudaStreamSynchronize(st));
  s->tune_pending = s->d.local_threads == FLASH_THREADS_TUNE ||
                    (s->d.ncp_threads == FLASH_THREADS_TUNE && s->d.metric == FLASH_METRIC_LITE);
  s->finalized = true;
  return FLASH_OK;
}

void flash_scene_destroy(flash_scene *s) {
  if (!s) return;
  cudaDeviceSynchronize();
  for (void *p : s->allocs) cudaFree(p);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->cap_st) cudaStreamDestroy(s->cap_st);
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  if (s->body_st) cudaStreamDestroy(s->body_st);
  for (flash::Lane &L : s->lanes) {
    if (L.done) cudaEventDestroy(L.done);
    if (L.st) cudaStreamDestroy(L.st);
    if (L.body_st) cudaStreamDestroy(L.body_st);
  }
  if (s->fork_ev) cudaEventDestroy(s->fork_ev);
  if (s->h_active) cudaFreeHost(s->h_active);
  if (s->rc_keys) cudaFree(s->rc_keys);
  if (s->rc_prep) cudaFree(s->rc_prep);
  delete s;
}

int32_t flash_num_envs(const flash_scene *s) { return s ? (int32_t)s->envs.size() : 0; }

int64_t flash_num_verts(const flash_scene *s) {
  if (!s) return 0;
  int64_t t = 0;
  for (size_t e = 0; e < s->envs.size(); e++) t += s->meshes[s->env_mesh[e]].n;
  return t;
}

flash_status flash_env_offsets(const flash_scene *s, int64_t *off) {
  if (!s || !off) return fail(FLASH_EINVAL, "null argument");
  int64_t t = 0;
  off[0] = 0;
  for (size_t e = 0; e < s->envs.size(); e++) {
    t += s->meshes[s->env_mesh[e]].n;
    off[e + 1] = t;
  }
  return FLASH_OK;
}

int32_t flash_contact_cap(const flash_scene *s) { return s ? s->cap : 0; }

flash_status flash_set_state(flash_scene *s, const float *q, const float *v, void *stream) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  for (auto &g : s->groups) FLASH_CUDA_TRY(launch_state_io(s, g, q, v, nullptr, nullptr, 0, (cudaStream_t)stream));
  // a new state starts a new history: the status word reports only what the
  // steps taken from it find
  FLASH_CUDA_TRY(cudaMemsetAsync(s->status, 0, sizeof(int), (cudaStream_t)stream));
  return FLASH_OK;
}

flash_status flash_get_state(const flash_scene *s, float *q, float *v, void *stream) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  for (auto &g : s->groups) FLASH_CUDA_TRY(launch_state_io(s, g, nullptr, nullptr, q, v, 1, (cudaStream_t)stream));
  return FLASH_OK;
}

flash_status flash_set_obstacle_poses(flash_scene *s, const float *poses, int32_t which, void *stream) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  if (!poses || (which != 0 && which != 1)) return fail(FLASH_EINVAL, "invalid arguments");
  size_t bytes = sizeof(float) * s->N * FLASH_MAX_OBS * 7;
  cudaStream_t st = (cudaStream_t)stream;
  FLASH_CUDA_TRY(cudaMemcpyAsync(s->pose_th, poses, bytes, cudaMemcpyDeviceToDevice, st));
  if (which == 0) FLASH_CUDA_TRY(cudaMemcpyAsync(s->pose_t, poses, bytes, cudaMemcpyDeviceToDevice, st));
  return FLASH_OK;
}

flash_status flash_grasp(flash_scene *s, int32_t first_env, int32_t count, const int32_t *request,
                         int32_t obstacle, const float *anchor, float radius, void *stream) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  if (count == 0) return FLASH_OK;
  if (!request || first_env < 0 || count < 0 || first_env > s->N - count)
    return fail(FLASH_EINVAL, "invalid environment range");
  if (obstacle < 0 || obstacle >= FLASH_MAX_OBS) return fail(FLASH_EINVAL, "grasp obstacle out of range");
  if (!(radius >= 0.f) || !std::isfinite(radius)) return fail(FLASH_EINVAL, "grasp radius must be finite and >= 0");
  float an[3] = {0.f, 0.f, 0.f};
  if (anchor)
    for (int c = 0; c < 3; c++) {
      if (!std::isfinite(anchor[c])) return fail(FLASH_EINVAL, "grasp anchor is not finite");
      an[c] = anchor[c];
    }
  for (int i = 0; i < count; i++)
    if (request[i] < -1 || request[i] > 1) return fail(FLASH_EINVAL, "grasp request must be -1, 0 or 1");
  cudaStream_t st = (cudaStream_t)stream;
  FLASH_CUDA_TRY(cudaMemcpyAsync(s->greq + first_env, request, sizeof(int32_t) * count, cudaMemcpyHostToDevice, st));
  FLASH_CUDA_TRY(launch_grasp_set(s, first_env, count, obstacle, an[0], an[1], an[2], radius, st));
  s->launches++;
  return FLASH_OK;
}

flash_status flash_render(flash_scene *s, const flash_camera *cam, const float *cam_poses, float *depth,
                          uint8_t *seg, float *points, void *stream) {
  NvtxRange range("flash.render");
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  if (!cam_poses || !depth) return fail(FLASH_EINVAL, "cam_poses and depth are required");
  if (s->N > 65535) return fail(FLASH_EINVAL, "ray casting takes at most 65535 environments");
  RcCam C;
  const flash_status r = rc_check_camera(cam, s->N, &C);
  if (r != FLASH_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t need = (size_t)s->N * C.W * C.H;
  if (need > s->rc_keys_n) {
    if (s->rc_keys) {
      FLASH_CUDA_TRY(cudaStreamSynchronize(st));
      FLASH_CUDA_TRY(cudaFree(s->rc_keys));
      s->rc_keys = nullptr;
      s->rc_keys_n = 0;
    }
    FLASH_CUDA_TRY(cudaMalloc(&s->rc_keys, need * sizeof(unsigned long long)));
    s->rc_keys_n = need;
    if (!s->rc_prep) FLASH_CUDA_TRY(cudaMalloc(&s->rc_prep, rc_prep_bytes(s->N)));
    s->rc_tag = -1;   // the first render fills the buffer
  }
  FLASH_CUDA_TRY(rc_next_tag(s->rc_keys, s->rc_keys_n, &s->rc_tag, st));
  const unsigned tag = (unsigned)s->rc_tag;
  for (const Group &g : s->groups) {
    const RcMesh M{g.q, 3LL * g.n_pad, g.n_pad, 1, g.genv, 0, g.rtris, g.rT};
    FLASH_CUDA_TRY(rc_launch_tri(M, g.N, cam_poses, C, s->rc_keys, tag, st));
    if (g.rT > 0) s->launches++;
  }
  const RcObs O{s->otype, s->odims, s->pose_t, s->K, FLASH_MAX_OBS};
  FLASH_CUDA_TRY(rc_launch_resolve(O, cam_poses, C, 0, s->N, s->rc_keys, tag, s->rc_prep, depth, seg, points, st));
  s->launches += 2;
  s->rc_tag--;
  return FLASH_OK;
}

namespace {

// Threads per environment of the local and lite NCP passes, timed on the
// scene's first step (FLASH_THREADS_TUNE), between its begin kernels and its
// first iteration, with the lanes joined on st.  Each candidate runs the
// first iteration's pass (k = 1: no pending update, outputs overwritten) from
// the same saved stop flags, iteration counts and residuals, and each NCP
// candidate from the same saved multipliers; everything is restored after the
// last candidate, so the step that follows is the one an untuned scene takes.
// The fastest of three runs of each candidate is compared, per local batch and
// per lane.
flash_status tune_threads(flash_scene *s, const StepArgs &a, int tc, cudaStream_t st) {
  NvtxRange range("flash.tune_threads");
  s->tune_pending = false;
  s->graph_stale = true;
  const bool profiling = s->profiling;   // the candidates' launches stay out of the kernel profile
  s->profiling = false;
  constexpr int kReps = 3;
  const size_t N = (size_t)s->N;
  std::vector<void *> tmp;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&] {
    cudaStreamSynchronize(st);
    for (void *p : tmp) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  auto run = [&]() -> cudaError_t {
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // saved per-environment stop state: done, iters, rncp
    void *sv = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&sv, N * (2 * sizeof(int) + sizeof(float)));
    if (e != cudaSuccess) return e;
    tmp.push_back(sv);
    int *sdone = (int *)sv, *siters = sdone + N;
    float *srncp = (float *)(siters + N);
    e = cudaMemcpyAsync(sdone, s->done, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(siters, s->iters, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(srncp, s->rncp, N * sizeof(float), cudaMemcpyDeviceToDevice, st);
    auto restore = [&]() -> cudaError_t {
      cudaError_t r = cudaMemcpyAsync(s->done, sdone, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
      if (r == cudaSuccess) r = cudaMemcpyAsync(s->iters, siters, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
      if (r == cudaSuccess) r = cudaMemcpyAsync(s->rncp, srncp, N * sizeof(float), cudaMemcpyDeviceToDevice, st);
      return r;
    };
    auto time_ms = [&](const std::function<cudaError_t()> &f, float *ms) -> cudaError_t {
      cudaError_t r = cudaEventRecord(e0, st);
      if (r == cudaSuccess) r = f();
      if (r == cudaSuccess) r = cudaEventRecord(e1, st);
      if (r == cudaSuccess) r = cudaEventSynchronize(e1);
      if (r == cudaSuccess) r = cudaEventElapsedTime(ms, e0, e1);
      s->launches++;
      return r;
    };
    if (s->d.local_threads == FLASH_THREADS_TUNE) {
      static const int cand[3] = {256, 512, 1024};
      for (Lane &L : s->lanes)
        for (Batch &b : L.local) {
          float best[3] = {1e30f, 1e30f, 1e30f};
          for (int rep = 0; rep < kReps && e == cudaSuccess; rep++)
            for (int c = 0; c < 3 && e == cudaSuccess; c++) {
              float ms = 0.f;
              e = restore();
              if (e == cudaSuccess)
                e = time_ms([&] { return launch_local_batch(s, b, cand[c], a, 1, 0, tc, st); }, &ms);
              best[c] = std::min(best[c], ms);
            }
          int k = 0;
          for (int c = 1; c < 3; c++)
            if (best[c] < best[k]) k = c;
          b.threads = cand[k];
        }
    }
    if (e == cudaSuccess && s->d.ncp_threads == FLASH_THREADS_TUNE && s->d.metric == FLASH_METRIC_LITE) {
      // the first iteration's residual and w = A^-1 r, then the NCP candidates
      // from the saved multipliers
      e = restore();
      for (Lane &L : s->lanes) {
        int launched = 0;
        if (e == cudaSuccess) e = launch_local_lane(s, L, a, 1, 0, tc, st, &launched);
        s->launches += launched;
        if (e == cudaSuccess) e = apply_lane(s, L, st, [](Group &g) { return g.r; }, [](Group &g) { return g.w; }, 0);
      }
      std::vector<float *> saved(s->groups.size(), nullptr);
      for (size_t gi = 0; gi < s->groups.size() && e == cudaSuccess; gi++) {
        const Group &g = s->groups[gi];
        const size_t bytes = (size_t)g.N * s->cap * 4 * sizeof(float);
        void *p = nullptr;
        e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) break;
        tmp.push_back(p);
        saved[gi] = (float *)p;
        e = cudaMemcpyAsync(p, g.cgam, bytes, cudaMemcpyDeviceToDevice, st);
      }
      auto restore_gamma = [&]() -> cudaError_t {
        cudaError_t r = cudaSuccess;
        for (size_t gi = 0; gi < s->groups.size() && r == cudaSuccess; gi++) {
          const Group &g = s->groups[gi];
          r = cudaMemcpyAsync(g.cgam, saved[gi], (size_t)g.N * s->cap * 4 * sizeof(float), cudaMemcpyDeviceToDevice,
                              st);
        }
        return r;
      };
      static const int cand[3] = {128, 256, 512};
      for (Lane &L : s->lanes) {
        float best[3] = {1e30f, 1e30f, 1e30f};
        for (int rep = 0; rep < kReps && e == cudaSuccess; rep++)
          for (int c = 0; c < 3 && e == cudaSuccess; c++) {
            float ms = 0.f;
            e = restore_gamma();
            if (e == cudaSuccess) e = time_ms([&] { return launch_ncp_lane(s, L, a, tc, st, cand[c]); }, &ms);
            best[c] = std::min(best[c], ms);
          }
        int k = 0;
        for (int c = 1; c < 3; c++)
          if (best[c] < best[k]) k = c;
        L.ncp_threads = cand[k];
      }
      if (e == cudaSuccess) e = restore_gamma();
    }
    if (e == cudaSuccess) e = restore();
    return e;
  };
  const cudaError_t e = run();
  cleanup();
  s->profiling = profiling;
  FLASH_CUDA_TRY(e);
  return FLASH_OK;
}

// One time step (Algorithm 1 body) issued on st and the lanes' streams.
flash_status tol_loop_graphed(flash_scene *s, cudaStream_t st, const std::function<cudaError_t(int, int)> &local,
                              const std::function<cudaError_t(cudaStream_t)> &solves);

flash_status step_once(flash_scene *s, cudaStream_t st) {
  NvtxRange range(s->capturing ? "flash.capture_step" : "flash.step_once");
  const bool learned = s->d.warm == FLASH_WARM_LEARNED;
  const StepArgs a = step_args(s);
  const int tc = use_tc(s) ? 1 : 0;
  const size_t pose_bytes = sizeof(float) * s->N * FLASH_MAX_OBS * 7;
  // Every phase is issued lane by lane; each lane's kernels run in order on
  // its own stream, so lanes only meet at the forks and joins below.
  auto begin = [&]() -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (const Lane &L : s->lanes)
      if (e == cudaSuccess)
        e = timed(s, FLASH_KIND_BEGIN, lane_stream(L, st), [&] { return launch_begin_lane(s, L, a, lane_stream(L, st)); });
    return e;
  };
  auto local = [&](int k, int residual_only) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (const Lane &L : s->lanes) {
      if (e != cudaSuccess) break;
      const cudaStream_t ls = lane_stream(L, st);
      int launched = 0;
      e = timed(s, FLASH_KIND_LOCAL, ls, [&] { return launch_local_lane(s, L, a, k, residual_only, tc, ls, &launched); });
      s->launches += launched - 1;
    }
    return e;
  };
  auto solves = [&]() -> cudaError_t {
    // w = A^-1 r ;  NCP ;  dq = A^-1 J^T dgamma  (q^k = q^{k-1} + w + dq, applied by the next local pass)
    cudaError_t e = cudaSuccess;
    for (const Lane &L : s->lanes)
      if (e == cudaSuccess) e = apply_lane(s, L, lane_stream(L, st), [](Group &g) { return g.r; }, [](Group &g) { return g.w; }, 0);
    if (s->d.metric == FLASH_METRIC_FULL) {
      // Newton step on the full metric: GMRES, one A^-1 application per step
      for (const Lane &L : s->lanes)
        if (e == cudaSuccess)
          e = timed(s, FLASH_KIND_NCP, lane_stream(L, st), [&] { return launch_fm_setup_lane(s, L, a, lane_stream(L, st)); });
      for (int j = 0; j < s->d.lin_iters && e == cudaSuccess; j++) {
        for (const Lane &L : s->lanes)
          if (e == cudaSuccess)
            e = timed(s, FLASH_KIND_NCP, lane_stream(L, st),
                      [&] { return launch_fm_scatter_lane(s, L, a, j, tc, lane_stream(L, st)); });
        for (const Lane &L : s->lanes)
          if (e == cudaSuccess)
            e = apply_lane(s, L, lane_stream(L, st), [](Group &g) { return g.f; }, [](Group &g) { return g.fm_u; }, 2);
        for (const Lane &L : s->lanes)
          if (e == cudaSuccess)
            e = timed(s, FLASH_KIND_NCP, lane_stream(L, st), [&] { return launch_fm_gather_lane(s, L, a, j, lane_stream(L, st)); });
      }
      for (const Lane &L : s->lanes)
        if (e == cudaSuccess)
          e = timed(s, FLASH_KIND_NCP, lane_stream(L, st), [&] { return launch_fm_finish_lane(s, L, a, tc, lane_stream(L, st)); });
    } else {
    for (const Lane &L : s->lanes)
      if (e == cudaSuccess)
        e = timed(s, FLASH_KIND_NCP, lane_stream(L, st), [&] { return launch_ncp_lane(s, L, a, tc, lane_stream(L, st)); });
    }
    for (const Lane &L : s->lanes)
      if (e == cudaSuccess) e = apply_lane(s, L, lane_stream(L, st), [](Group &g) { return g.f; }, [](Group &g) { return g.dq; }, 1);
    return e;
  };
  auto end = [&]() -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (const Lane &L : s->lanes)
      if (e == cudaSuccess)
        e = timed(s, FLASH_KIND_END, lane_stream(L, st), [&] { return launch_end_lane(s, L, a, lane_stream(L, st)); });
    return e;
  };
  {
    FLASH_CUDA_TRY(fork(s, st));
    FLASH_CUDA_TRY(begin());
    if (learned || s->record) {
      // per-group warm-start work on the caller's stream, between the lanes' phases
      FLASH_CUDA_TRY(join(s, st));
      for (auto &g : s->groups) {
        FLASH_CUDA_TRY(timed(s, FLASH_KIND_WARM, st, [&] { return launch_row_offsets(g, g.row_off, st); }));
        FLASH_CUDA_TRY(timed(s, FLASH_KIND_WARM, st, [&] { return launch_features(s, g, group_args(a, g), g.row_off, g.feat, st); }));
        if (learned) {
          FLASH_CUDA_TRY(timed(s, FLASH_KIND_WARM, st, [&] {
            return mlp_forward(s->mlp_params, g.feat, g.pred, g.row_off + g.N, (int64_t)g.N * s->cap, st);
          }));
          FLASH_CUDA_TRY(timed(s, FLASH_KIND_WARM, st, [&] {
            return launch_apply_learned(s, g, group_args(a, g), g.row_off, g.feat, g.pred, s->ws_bounds, s->use_dq, st);
          }));
        }
      }
      FLASH_CUDA_TRY(fork(s, st));
    }
    if (s->tune_pending && !s->capturing) {
      FLASH_CUDA_TRY(join(s, st));
      const flash_status r = tune_threads(s, a, tc, st);
      if (r != FLASH_OK) return r;
      FLASH_CUDA_TRY(fork(s, st));
    }
    if (s->d.mode == FLASH_MODE_FIXED) {
      for (int k = 1; k <= s->d.k_max; k++) {
        FLASH_CUDA_TRY(local(k, 0));
        FLASH_CUDA_TRY(solves());
      }
      FLASH_CUDA_TRY(local(s->d.k_max + 1, 1));
      FLASH_CUDA_TRY(join(s, st));
    } else if (s->capturing) {
      // captured: the loop runs on the device (a graph while-node)
      FLASH_CUDA_TRY(join(s, st));
      const flash_status r = tol_loop_graphed(s, st, local, [&](cudaStream_t body) {
        const cudaStream_t outer = st;
        st = body;   // the phase lambdas issue on st and the lanes' streams
        cudaError_t e = fork(s, st);
        if (e == cudaSuccess) e = solves();
        if (e == cudaSuccess) e = local(0, 0);
        if (e == cudaSuccess) e = join(s, st);
        st = outer;
        return e;
      });
      if (r != FLASH_OK) return r;
    } else {
      // Every environment stops on the device (its local pass sets its done
      // flag; later passes skip it), so the host only needs to learn when all
      // have stopped: it reads the count of environments still iterating
      // every kTolCheck iterations, and the launches in between queue ahead
      // of the GPU.  Iterations after the last environment stopped change
      // nothing.
      FLASH_CUDA_TRY(join(s, st));
      const int last = s->d.k_cap + 1;
      for (int k = 1; k <= last; k++) {
        const bool check = k % kTolCheck == 0 || k == last;
        if (check) FLASH_CUDA_TRY(cudaMemsetAsync(s->active, 0, sizeof(int), st));
        FLASH_CUDA_TRY(fork(s, st));
        FLASH_CUDA_TRY(local(k, 0));
        if (check) {
          FLASH_CUDA_TRY(join(s, st));
          FLASH_CUDA_TRY(cudaMemcpyAsync(s->h_active, s->active, sizeof(int), cudaMemcpyDeviceToHost, st));
          FLASH_CUDA_TRY(cudaStreamSynchronize(st));
          if (*s->h_active == 0) break;
          FLASH_CUDA_TRY(fork(s, st));
        }
        FLASH_CUDA_TRY(solves());
        FLASH_CUDA_TRY(join(s, st));
      }
    }
    if (s->record)
      for (auto &g : s->groups)
        FLASH_CUDA_TRY(timed(s, FLASH_KIND_WARM, st, [&] { return launch_targets(s, g, group_args(a, g), g.row_off, g.targ, st); }));
    FLASH_CUDA_TRY(fork(s, st));
    FLASH_CUDA_TRY(end());
    FLASH_CUDA_TRY(join(s, st));
    FLASH_CUDA_TRY(cudaMemcpyAsync(s->pose_t, s->pose_th, pose_bytes, cudaMemcpyDeviceToDevice, st));
  }
  return FLASH_OK;
}

// The tolerance mode's iterations (Algorithm 1's loop, stopped per
// environment on r_ncp <= tol, Mode B) inside a captured step.  The first
// iteration's local pass is issued ahead of a graph while-node; each run of
// the node's body is {global solves, NCP, next local pass, k_tol_next}, and
// k_tol_next keeps the node running while an environment is still iterating.
// This is the host loop of the eager path with the host's reads of the
// active count replaced by the device deciding: the iterations each
// environment runs, and so the results, are the same.  The body is
// captured into the node's own graph on separate streams (a stream that has
// joined one capture cannot join another).
flash_status tol_loop_graphed(flash_scene *s, cudaStream_t st, const std::function<cudaError_t(int, int)> &local,
                              const std::function<cudaError_t(cudaStream_t)> &body_phases) {
  const int last = s->d.k_cap + 1;
  FLASH_CUDA_TRY(cudaMemsetAsync(s->active, 0, sizeof(int), st));
  FLASH_CUDA_TRY(fork(s, st));
  FLASH_CUDA_TRY(local(1, 0));
  FLASH_CUDA_TRY(join(s, st));
  cudaStreamCaptureStatus cs;
  cudaGraph_t graph = nullptr;
  FLASH_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, nullptr, nullptr, nullptr));
  cudaGraphConditionalHandle h;
  FLASH_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, graph, 0, 0));
  FLASH_CUDA_TRY(launch_tol_next(h, s->active, s->kit, s->trips, last, 1, st));
  s->launches++;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  FLASH_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, nullptr, &nd));
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  FLASH_CUDA_TRY(cudaGraphAddNode(&node, graph, deps, nullptr, nd, &p));
  if (!s->body_st) FLASH_CUDA_TRY(cudaStreamCreateWithFlags(&s->body_st, cudaStreamNonBlocking));
  if (s->lanes.size() > 1)
    for (Lane &L : s->lanes)
      if (!L.body_st) FLASH_CUDA_TRY(cudaStreamCreateWithFlags(&L.body_st, cudaStreamNonBlocking));
  FLASH_CUDA_TRY(cudaStreamBeginCaptureToGraph(s->body_st, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
  auto swap_lanes = [&] {
    if (s->lanes.size() > 1)
      for (Lane &L : s->lanes) std::swap(L.st, L.body_st);
  };
  swap_lanes();
  const int64_t l0 = s->launches;
  cudaError_t e = body_phases(s->body_st);
  if (e == cudaSuccess) e = launch_tol_next(h, s->active, s->kit, s->trips, last, 0, s->body_st);
  s->body_launches = s->launches - l0 + 1;
  s->launches = l0;
  swap_lanes();
  cudaGraph_t body = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(s->body_st, &body);
  FLASH_CUDA_TRY(e);
  FLASH_CUDA_TRY(ee);
  FLASH_CUDA_TRY(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return FLASH_OK;
}

// Capture one step into a graph on an internal stream (the caller's stream
// may be the legacy default stream, which cannot capture).
flash_status capture_step(flash_scene *s) {
  if (s->body_launches) {
    // fold the previous graph's loop runs into the host count
    unsigned long long trips = 0;
    FLASH_CUDA_TRY(cudaMemcpy(&trips, s->trips, sizeof(trips), cudaMemcpyDeviceToHost));
    FLASH_CUDA_TRY(cudaMemset(s->trips, 0, sizeof(trips)));
    s->launches += (int64_t)trips * s->body_launches;
    s->body_launches = 0;
  }
  if (s->graph) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  if (!s->cap_st) FLASH_CUDA_TRY(cudaStreamCreateWithFlags(&s->cap_st, cudaStreamNonBlocking));
  FLASH_CUDA_TRY(cudaStreamBeginCapture(s->cap_st, cudaStreamCaptureModeThreadLocal));
  const int64_t l0 = s->launches;
  s->capturing = true;
  const flash_status r = step_once(s, s->cap_st);
  s->capturing = false;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s->cap_st, &g);
  s->graph_launches = s->launches - l0;
  s->launches = l0;
  if (r != FLASH_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  FLASH_CUDA_TRY(e);
  const cudaError_t ei = cudaGraphInstantiate(&s->graph, g, 0);
  cudaGraphDestroy(g);
  FLASH_CUDA_TRY(ei);
  s->graph_stale = false;
  return FLASH_OK;
}

}  // namespace

flash_status flash_step(flash_scene *s, int32_t n_steps, void *stream) {
  NvtxRange range("flash.step");
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  if (n_steps < 0) return fail(FLASH_EINVAL, "negative step count");
  const bool learned = s->d.warm == FLASH_WARM_LEARNED;
  if (learned && !s->mlp_params) return fail(FLASH_ESTATE, "learned warm start needs weights (flash_warmstart_set)");
  cudaStream_t st = (cudaStream_t)stream;
  const bool graphed = !s->d.eager && !s->profiling;
  if (graphed) {
    if (s->tune_pending && n_steps > 0) {
      // the first step runs eagerly: it times the thread counts the graph uses
      const flash_status r = step_once(s, st);
      if (r != FLASH_OK) return r;
      n_steps--;
    }
    if (!s->graph || s->graph_stale) {
      const flash_status r = capture_step(s);
      if (r != FLASH_OK) return r;
    }
    for (int step = 0; step < n_steps; step++) {
      FLASH_CUDA_TRY(cudaGraphLaunch(s->graph, st));
      s->launches += s->graph_launches;
    }
    return FLASH_OK;
  }
  for (int step = 0; step < n_steps; step++) {
    const flash_status r = step_once(s, st);
    if (r != FLASH_OK) return r;
  }
  return FLASH_OK;
}

flash_status flash_warmstart_set(flash_scene *s, const float *params, int32_t mode, int32_t use_dq) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  if (mode < FLASH_WARM_COLD || mode > FLASH_WARM_LEARNED) return fail(FLASH_EINVAL, "invalid warm-start mode");
  if (params) {
    if (!s->mlp_params) FLASH_CUDA_TRY(dalloc(s, &s->mlp_params, (size_t)mlp_num_params()));
    FLASH_CUDA_TRY(cudaMemcpy(s->mlp_params, params, sizeof(float) * mlp_num_params(), cudaMemcpyDeviceToDevice));
  }
  if (mode == FLASH_WARM_LEARNED) {
    if (!s->mlp_params) return fail(FLASH_EINVAL, "learned warm start needs parameters");
    FLASH_CUDA_TRY(ensure_learn_buffers(s));
  }
  s->d.warm = mode;
  s->use_dq = use_dq;
  s->graph_stale = true;
  return FLASH_OK;
}

flash_status flash_warmstart_bounds(flash_scene *s, const float *lo, const float *hi) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  if (!lo || !hi) return fail(FLASH_EINVAL, "null bounds");
  std::vector<float> b(20);
  for (int c = 0; c < 10; c++) {
    if (!(lo[c] <= hi[c])) return fail(FLASH_EINVAL, "warm-start bounds need lo <= hi");
    b[c] = lo[c];
    b[10 + c] = hi[c];
  }
  FLASH_CUDA_TRY(ensure_learn_buffers(s));
  FLASH_CUDA_TRY(cudaMemcpy(s->ws_bounds, b.data(), sizeof(float) * 20, cudaMemcpyHostToDevice));
  return FLASH_OK;
}

flash_status flash_record_contacts(flash_scene *s, int32_t enable) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  if (enable) FLASH_CUDA_TRY(ensure_learn_buffers(s));
  s->record = enable != 0;
  s->graph_stale = true;
  return FLASH_OK;
}

flash_status flash_get_recorded(flash_scene *s, float *X, float *T, int64_t max_rows, int64_t *rows, void *stream) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  if (!s->groups.front().row_off) return fail(FLASH_ESTATE, "recording was never enabled");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t pos = 0;
  for (auto &g : s->groups) {
    int64_t n = 0;
    FLASH_CUDA_TRY(cudaMemcpyAsync(&n, g.row_off + g.N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    FLASH_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t take = std::max<int64_t>(0, std::min(n, max_rows - pos));
    if (take > 0) {
      if (X) FLASH_CUDA_TRY(cudaMemcpyAsync(X + pos * 10, g.feat, sizeof(float) * 10 * take, cudaMemcpyDeviceToDevice, st));
      if (T) FLASH_CUDA_TRY(cudaMemcpyAsync(T + pos * 6, g.targ, sizeof(float) * 6 * take, cudaMemcpyDeviceToDevice, st));
    }
    pos += n;
  }
  if (rows) *rows = pos;
  return FLASH_OK;
}

flash_status flash_profile_enable(flash_scene *s, int32_t enable) {
  if (!s) return fail(FLASH_EINVAL, "null scene");
  FLASH_CUDA_TRY(flush_profile(s));
  s->profiling = enable != 0;
  for (int k = 0; k < FLASH_NUM_KINDS; k++) { s->prof_ms[k] = 0; s->prof_n[k] = 0; }
  return FLASH_OK;
}

flash_status flash_profile_read(flash_scene *s, int32_t kind, double *total_ms, int64_t *launches) {
  if (!s || kind < 0 || kind >= FLASH_NUM_KINDS) return fail(FLASH_EINVAL, "invalid arguments");
  FLASH_CUDA_TRY(flush_profile(s));
  if (total_ms) *total_ms = s->prof_ms[kind];
  if (launches) *launches = s->prof_n[kind];
  return FLASH_OK;
}

int64_t flash_launch_count(const flash_scene *s) {
  if (!s) return 0;
  if (!s->trips || !s->body_launches) return s->launches;
  // kernels of the graphed tolerance loop: known on the device only
  unsigned long long trips = 0;
  if (cudaMemcpy(&trips, s->trips, sizeof(trips), cudaMemcpyDeviceToHost) != cudaSuccess) return s->launches;
  return s->launches + (int64_t)trips * s->body_launches;
}

int32_t flash_lane_count(const flash_scene *s) { return s && s->finalized ? (int32_t)s->lanes.size() : 0; }

int32_t flash_grouped_solve(const flash_scene *s) { return s && s->finalized && s->grouped ? 1 : 0; }

flash_status flash_test_bounded_wait(flash_scene *s, int64_t limit_cycles, void *stream) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  if (limit_cycles <= 0 || limit_cycles > 4000000000LL)
    return fail(FLASH_EINVAL, "limit_cycles must be in 1..4e9");
  FLASH_CUDA_TRY(launch_wait_probe(s->status, (long long)limit_cycles, (cudaStream_t)stream));
  s->launches++;
  return FLASH_OK;
}

int32_t flash_checked_build(void) {
#ifdef FLASH_CHECK
  return 1;
#else
  return 0;
#endif
}

flash_status flash_check_poke_element(flash_scene *s, int32_t env, int32_t element, int32_t corner, int32_t value,
                                      int32_t *old) {
#ifndef FLASH_CHECK
  (void)s; (void)env; (void)element; (void)corner; (void)value; (void)old;
  return fail(FLASH_ENOTIMPL, "element poking exists in the checked build only");
#else
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  if (env < 0 || env >= s->N) return fail(FLASH_EINVAL, "environment out of range");
  Group &g = s->groups[s->env_group[env]];
  if (element < 0 || element >= g.E || corner < 0 || corner >= g.vpe)
    return fail(FLASH_EINVAL, "element or corner out of range");
  int prev = 0;
  FLASH_CUDA_TRY(cudaDeviceSynchronize());
  FLASH_CUDA_TRY(cudaMemcpy(&prev, g.elems + (size_t)4 * element + corner, sizeof(int), cudaMemcpyDeviceToHost));
  FLASH_CUDA_TRY(cudaMemcpy(g.elems + (size_t)4 * element + corner, &value, sizeof(int), cudaMemcpyHostToDevice));
  if (g.erec)   // the triangle records carry the same vertex ids as float bits
    FLASH_CUDA_TRY(cudaMemcpy(reinterpret_cast<float *>(g.erec) + (size_t)8 * element + corner, &value, sizeof(int),
                              cudaMemcpyHostToDevice));
  if (old) *old = prev;
  return FLASH_OK;
#endif
}

int32_t flash_scene_threads(const flash_scene *s, int32_t kind, int32_t *out, int32_t max_out) {
  if (!s || !s->finalized || (kind != 0 && kind != 1)) return 0;
  int32_t k = 0;
  for (const Lane &L : s->lanes) {
    if (kind == 1) {
      if (out && k < max_out) out[k] = L.ncp_threads;
      k++;
      continue;
    }
    for (const Batch &b : L.local) {
      if (out && k < max_out) out[k] = b.threads;
      k++;
    }
  }
  return k;
}

int32_t flash_tile_splits(const flash_scene *s, int32_t *out, int32_t max_out) {
  if (!s || !s->finalized || !use_tc(s)) return 0;
  int32_t k = 0;
  for (const Lane &L : s->lanes)
    for (const LaneRange &r : L.ranges) {
      if (out && k < max_out) out[k] = r.tc_split;
      k++;
    }
  return k;
}

int32_t flash_tile_widths(const flash_scene *s, int32_t *out, int32_t max_out) {
  if (!s || !s->finalized || !use_tc(s)) return 0;
  int32_t k = 0;
  for (const Lane &L : s->lanes)
    for (const LaneRange &r : L.ranges) {
      if (out && k < max_out) out[k] = r.tc_bn;
      k++;
    }
  return k;
}

flash_status flash_get_contacts(const flash_scene *s, int32_t *count, int32_t *vert, int32_t *obs, float *gamma,
                                void *stream) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  cudaStream_t st = (cudaStream_t)stream;
  for (auto &g : s->groups)
    for (int l = 0; l < g.N; l++) {
      int e = g.env_ids[l];
      size_t cs = (size_t)s->cap;
      if (count) FLASH_CUDA_TRY(cudaMemcpyAsync(count + e, g.pcount + l, sizeof(int), cudaMemcpyDeviceToDevice, st));
      if (vert) FLASH_CUDA_TRY(cudaMemcpyAsync(vert + e * cs, g.pvert + l * cs, sizeof(int) * cs, cudaMemcpyDeviceToDevice, st));
      if (obs) FLASH_CUDA_TRY(cudaMemcpyAsync(obs + e * cs, g.pobs + l * cs, sizeof(int) * cs, cudaMemcpyDeviceToDevice, st));
      if (gamma)
        FLASH_CUDA_TRY(cudaMemcpyAsync(gamma + e * cs * 4, g.pgam + l * cs * 4, sizeof(float) * cs * 4,
                                       cudaMemcpyDeviceToDevice, st));
    }
  return FLASH_OK;
}

flash_status flash_get_contact_tris(const flash_scene *s, int32_t *tri, void *stream) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  if (!tri) return fail(FLASH_EINVAL, "tri is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t cs = (size_t)s->cap;
  for (auto &g : s->groups)
    for (int l = 0; l < g.N; l++) {
      const int e = g.env_ids[l];
      if (g.self)
        FLASH_CUDA_TRY(cudaMemcpyAsync(tri + e * cs, g.pctri + l * cs, sizeof(int) * cs, cudaMemcpyDeviceToDevice, st));
      else
        FLASH_CUDA_TRY(cudaMemsetAsync(tri + e * cs, 0xff, sizeof(int) * cs, st));
    }
  return FLASH_OK;
}

flash_status flash_get_stats(const flash_scene *s, int32_t *iters, float *rncp, void *stream) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  cudaStream_t st = (cudaStream_t)stream;
  if (iters) FLASH_CUDA_TRY(cudaMemcpyAsync(iters, s->iters, sizeof(int) * s->N, cudaMemcpyDeviceToDevice, st));
  if (rncp) FLASH_CUDA_TRY(cudaMemcpyAsync(rncp, s->rncp, sizeof(float) * s->N, cudaMemcpyDeviceToDevice, st));
  return FLASH_OK;
}

flash_status flash_status_word(flash_scene *s, void *stream) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  int w = 0;
  cudaStream_t st = (cudaStream_t)stream;
  FLASH_CUDA_TRY(cudaMemcpyAsync(&w, s->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  FLASH_CUDA_TRY(cudaStreamSynchronize(st));
  if (w & (1 << 11)) return fail(FLASH_ETIMEOUT, "a bounded wait of the tensor-core solve ran out");
  if (w & (1 << 12)) return fail(FLASH_EINDEX, "a step kernel read an index out of its range (checked build)");
  if (w & (1 << 9)) return fail(FLASH_ENUMERIC, "non-finite state or residual");
  if (w & (1 << 8)) {
    set_error("contacts beyond the scene's contact capacity were dropped");
    return FLASH_WOVERFLOW;
  }
  if (w & (1 << 10)) {
    set_error("a vertex had more contacts than the per-vertex NCP block holds; the extra rows were not solved");
    return FLASH_WOVERFLOW;
  }
  return FLASH_OK;
}

flash_status flash_global_apply(flash_scene *s, int32_t first_env, int32_t n, const float *rhs, float *out,
                                void *stream) {
  if (!s || !s->finalized) return fail(FLASH_ESTATE, "scene not finalized");
  if (first_env < 0 || first_env >= s->N || !rhs || !out) return fail(FLASH_EINVAL, "invalid arguments");
  Group &g = s->groups[s->env_group[first_env]];
  if (g.env_ids.front() != first_env || (int)g.env_ids.size() != n)
    return fail(FLASH_EINVAL, "range must be exactly one group of environments");
  for (int l = 0; l < n; l++)
    if (g.env_ids[l] != first_env + l) return fail(FLASH_EINVAL, "group environments are not contiguous");
  cudaStream_t st = (cudaStream_t)stream;
  FLASH_CUDA_TRY(cudaMemsetAsync(s->done, 0, sizeof(int) * s->N, st));
  FLASH_CUDA_TRY(launch_rhs_io(g, s->d_voff, first_env, rhs, g.r, 0, st));
  if (use_tc(s)) FLASH_CUDA_TRY(launch_split_rhs(g, g.r, st, 0, -1, s->d.solve == FLASH_SOLVE_BF16R));
  FLASH_CUDA_TRY(apply_inverse(s, g, g.r, g.w, st));
  FLASH_CUDA_TRY(launch_rhs_io(g, s->d_voff, first_env, out, g.w, 1, st));
  return FLASH_OK;
}

}  // extern "C"
