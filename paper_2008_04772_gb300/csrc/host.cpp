// Host-side construction of meshes, RWG / Buffa–Christiansen slot tables,
// singular pair lists, sparsity patterns and quadrature tables.
//
// Section 2 (M disjoint closed surfaces, outward normals) and Section 3.2
// (RWG on the primal mesh, BC on its barycentric refinement) of
// arXiv 2008.04772. All O(N) setup; the O(N^2) numerics run on the GPU.
#include <algorithm>
#include <array>
#include <thread>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <tuple>
#include <unordered_map>

#include "internal.h"

namespace cal {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

const char* last_error() { return g_err; }

// ---------------------------------------------------------------------------
// instrumentation
// ---------------------------------------------------------------------------
static std::atomic<int64_t> g_launches{0};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
struct ProfRec {
  std::string name;
  double units;
  cudaEvent_t a, b;
  unsigned long long* counter;  // device-counted units (replaces `units` when set)
};
static std::vector<ProfRec> g_prof;

void note_launch(int n) { g_launches += n; }
int64_t launches() { return g_launches.load(); }

int prof_begin(cudaStream_t st, const char* name, double units) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return -1;
  ProfRec r{name, units, nullptr, nullptr, nullptr};
  if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return -1;
  cudaEventRecord(r.a, st);
  g_prof.push_back(r);
  return (int)g_prof.size() - 1;
}

void prof_end(cudaStream_t st, int token) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (token < 0 || token >= (int)g_prof.size()) return;
  cudaEventRecord(g_prof[token].b, st);
}

unsigned long long* prof_counter(int token, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (token < 0 || token >= (int)g_prof.size()) return nullptr;
  ProfRec& r = g_prof[token];
  if (!r.counter) {
    if (cudaMallocAsync((void**)&r.counter, sizeof(unsigned long long), st) != cudaSuccess) {
      r.counter = nullptr;
      return nullptr;
    }
    cudaMemsetAsync(r.counter, 0, sizeof(unsigned long long), st);
  }
  return r.counter;
}

int prof_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& r : g_prof) {
    cudaEventSynchronize(r.b);
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
    if (r.counter) cudaFree(r.counter);
  }
  g_prof.clear();
  g_prof_on = on != 0;
  return CAL_OK;
}

int prof_read(const char* name, int64_t* n, double* ms, double* units) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  int64_t cnt = 0;
  double tot = 0.0, u = 0.0;
  for (auto& r : g_prof) {
    if (r.name != name) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return fail(CAL_ECUDA, "profile: event wait failed");
    float t = 0.0f;
    cudaEventElapsedTime(&t, r.a, r.b);
    ++cnt;
    tot += t;
    if (r.counter) {
      unsigned long long c = 0;
      if (cudaMemcpy(&c, r.counter, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(CAL_ECUDA, "profile: counter read failed");
      u += (double)c;
    } else {
      u += r.units;
    }
  }
  if (n) *n = cnt;
  if (ms) *ms = tot;
  if (units) *units = u;
  return CAL_OK;
}

// ---------------------------------------------------------------------------
// quadrature tables
// ---------------------------------------------------------------------------
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    // Newton iteration on P_n from the Chebyshev-like initial guess
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? t : p1;
      double pnm1 = (n == 1) ? 1.0 : p0;
      dp = n * (t * pn - pnm1) / (t * t - 1.0);
      double dt = pn / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    // weights from the converged node
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double pn = (n == 1) ? t : p1, pnm1 = (n == 1) ? 1.0 : p0;
    dp = n * (t * pn - pnm1) / (t * t - 1.0);
    x[i] = 0.5 * (1.0 - t);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2/((1-t^2) P'^2) mapped to [0,1]
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return x[a] < x[b]; });
  std::vector<double> xs(n), ws(n);
  for (int i = 0; i < n; ++i) { xs[i] = x[idx[i]]; ws[i] = w[idx[i]]; }
  x.swap(xs);
  w.swap(ws);
}

void triangle_rule(int npts, std::vector<double>& bary, std::vector<double>& w) {
  bary.clear();
  w.clear();
  if (npts == 1) {
    bary = {1.0 / 3, 1.0 / 3, 1.0 / 3};
    w = {1.0};
    return;
  }
  if (npts == 3) {  // degree 2 (Strang–Fix): (2/3, 1/6, 1/6) and permutations, equal weights
    bary = {2.0 / 3, 1.0 / 6, 1.0 / 6, 1.0 / 6, 2.0 / 3, 1.0 / 6, 1.0 / 6, 1.0 / 6, 2.0 / 3};
    w = {1.0 / 3, 1.0 / 3, 1.0 / 3};
    return;
  }
  if (npts == 4) {  // degree 3 (Strang–Fix): centroid -27/48, (3/5, 1/5, 1/5) and permutations 25/48
    bary = {1.0 / 3, 1.0 / 3, 1.0 / 3, 0.6, 0.2, 0.2, 0.2, 0.6, 0.2, 0.2, 0.2, 0.6};
    w = {-27.0 / 48, 25.0 / 48, 25.0 / 48, 25.0 / 48};
    return;
  }
  // symmetric degree-4 rule with 6 points (Strang–Fix, Dunavant), closed form
  const double s10 = std::sqrt(10.0), s25 = std::sqrt(0.4);
  const double a = (8.0 - s10 + std::sqrt(38.0 - 44.0 * s25)) / 18.0;
  const double b = (8.0 - s10 - std::sqrt(38.0 - 44.0 * s25)) / 18.0;
  const double root = std::sqrt(213125.0 - 53320.0 * s10);
  const double wa = (620.0 + root) / 3720.0, wb = (620.0 - root) / 3720.0;
  for (auto [p, wp] : {std::pair<double, double>{a, wa}, {b, wb}}) {
    double c = 1.0 - 2.0 * p;
    double pts[3][3] = {{c, p, p}, {p, c, p}, {p, p, c}};
    for (auto& q : pts) {
      bary.insert(bary.end(), q, q + 3);
      w.push_back(wp);
    }
  }
}

// ---------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------
int build_mesh(Mesh& m, const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
               const int32_t* domain) {
  if (!verts || !tris || nv < 3 || nt < 4 || nv > (1LL << 30) || nt > (1LL << 30))
    return fail(CAL_EINVAL, "mesh_create: bad sizes or NULL arrays (nv=%lld nt=%lld)",
                (long long)nv, (long long)nt);
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!std::isfinite(verts[i])) return fail(CAL_EINVAL, "mesh_create: non-finite vertex coordinate");
  int maxdom = 0;
  for (int64_t t = 0; t < nt; ++t) {
    for (int a = 0; a < 3; ++a)
      if (tris[3 * t + a] < 0 || tris[3 * t + a] >= nv)
        return fail(CAL_EINVAL, "mesh_create: triangle %lld has vertex id out of range", (long long)t);
    if (tris[3 * t] == tris[3 * t + 1] || tris[3 * t + 1] == tris[3 * t + 2] ||
        tris[3 * t] == tris[3 * t + 2])
      return fail(CAL_EMESH, "mesh_create: degenerate triangle %lld", (long long)t);
    int d = domain ? domain[t] : 0;
    if (d < 0 || d > (1 << 20)) return fail(CAL_EINVAL, "mesh_create: bad scatterer id");
    maxdom = std::max(maxdom, d);
  }
  m.nv = nv;
  m.M = maxdom + 1;
  m.X.assign(verts, verts + 3 * nv);
  // group triangles by scatterer (stable), keeping each vertex order
  std::vector<int64_t> order(nt);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return (domain ? domain[a] : 0) < (domain ? domain[b] : 0);
  });
  m.nt = nt;
  m.T.resize(3 * nt);
  m.dom.resize(nt);
  for (int64_t i = 0; i < nt; ++i) {
    for (int a = 0; a < 3; ++a) m.T[3 * i + a] = tris[3 * order[i] + a];
    m.dom[i] = domain ? domain[order[i]] : 0;
  }
  // scatterers must not share vertices
  std::vector<int> vdom(nv, -1);
  for (int64_t t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a) {
      int v = m.T[3 * t + a];
      if (vdom[v] >= 0 && vdom[v] != m.dom[t])
        return fail(CAL_EMESH, "mesh_create: scatterers %d and %d share vertex %d", vdom[v], m.dom[t], v);
      vdom[v] = m.dom[t];
    }
  m.tri_off.assign(m.M + 1, 0);
  for (int64_t t = 0; t < nt; ++t) m.tri_off[m.dom[t] + 1]++;
  for (int64_t d = 0; d < m.M; ++d) {
    if (m.tri_off[d + 1] == 0) return fail(CAL_EINVAL, "mesh_create: scatterer %lld has no triangles", (long long)d);
    m.tri_off[d + 1] += m.tri_off[d];
  }
  // edges: key (dom, lo, hi) -> (T+, a+) and (T-, a-)
  struct Slot { int tp = -1, ap = -1, tm = -1, am = -1; };
  std::map<std::tuple<int, int, int>, Slot> edges;
  for (int64_t t = 0; t < nt; ++t)
    for (int i = 0; i < 3; ++i) {
      int a = m.T[3 * t + i], b = m.T[3 * t + (i + 1) % 3];
      int opp = (i + 2) % 3;
      auto& s = edges[{m.dom[t], std::min(a, b), std::max(a, b)}];
      if (a < b) {
        if (s.tp >= 0) return fail(CAL_EMESH, "mesh_create: edge (%d,%d) traversed twice the same way: not an oriented manifold", a, b);
        s.tp = (int)t; s.ap = opp;
      } else {
        if (s.tm >= 0) return fail(CAL_EMESH, "mesh_create: edge (%d,%d) traversed twice the same way: not an oriented manifold", a, b);
        s.tm = (int)t; s.am = opp;
      }
    }
  m.ne = (int64_t)edges.size();
  m.e_lo.resize(m.ne); m.e_hi.resize(m.ne); m.e_dom.resize(m.ne);
  m.e_tp.resize(m.ne); m.e_ap.resize(m.ne); m.e_tm.resize(m.ne); m.e_am.resize(m.ne);
  m.e_len.resize(m.ne);
  m.tri_edge.assign(3 * nt, -1);
  m.tri_sign.assign(3 * nt, 0);
  m.edge_off.assign(m.M + 1, 0);
  m.valence.assign(nv, 0);
  int64_t e = 0;
  m.h = 0.0;
  for (auto& [key, s] : edges) {
    if (s.tp < 0 || s.tm < 0)
      return fail(CAL_EMESH, "mesh_create: open edge (%d,%d): surface not closed", std::get<1>(key), std::get<2>(key));
    m.e_dom[e] = std::get<0>(key);
    m.e_lo[e] = std::get<1>(key);
    m.e_hi[e] = std::get<2>(key);
    m.e_tp[e] = s.tp; m.e_ap[e] = s.ap; m.e_tm[e] = s.tm; m.e_am[e] = s.am;
    double d2 = 0;
    for (int c = 0; c < 3; ++c) {
      double d = m.X[3 * m.e_hi[e] + c] - m.X[3 * m.e_lo[e] + c];
      d2 += d * d;
    }
    m.e_len[e] = std::sqrt(d2);
    m.h = std::max(m.h, m.e_len[e]);
    m.tri_edge[3 * s.tp + s.ap] = (int)e; m.tri_sign[3 * s.tp + s.ap] = +1;
    m.tri_edge[3 * s.tm + s.am] = (int)e; m.tri_sign[3 * s.tm + s.am] = -1;
    m.edge_off[m.e_dom[e] + 1]++;
    m.valence[m.e_lo[e]]++;
    m.valence[m.e_hi[e]]++;
    ++e;
  }
  for (int64_t d = 0; d < m.M; ++d) m.edge_off[d + 1] += m.edge_off[d];
  m.max_valence = *std::max_element(m.valence.begin(), m.valence.end());
  for (int64_t t = 0; t < nt; ++t) {
    double u[3], v[3];
    for (int c = 0; c < 3; ++c) {
      u[c] = m.X[3 * m.T[3 * t + 1] + c] - m.X[3 * m.T[3 * t] + c];
      v[c] = m.X[3 * m.T[3 * t + 2] + c] - m.X[3 * m.T[3 * t] + c];
    }
    double n0 = u[1] * v[2] - u[2] * v[1], n1 = u[2] * v[0] - u[0] * v[2], n2 = u[0] * v[1] - u[1] * v[0];
    if (!(n0 * n0 + n1 * n1 + n2 * n2 > 0.0))
      return fail(CAL_EMESH, "mesh_create: zero-area triangle %lld", (long long)t);
  }
  return CAL_OK;
}

// ---------------------------------------------------------------------------
// spaces
// ---------------------------------------------------------------------------
static TriD make_tri(const double* P0, const double* P1, const double* P2, int v0, int v1, int v2) {
  TriD t{};
  const double* P[3] = {P0, P1, P2};
  for (int c = 0; c < 3; ++c) t.c[c] = (P0[c] + P1[c] + P2[c]) / 3.0;
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) t.off[a][c] = P[a][c] - t.c[c];
  double u[3], v[3];
  for (int c = 0; c < 3; ++c) { u[c] = P1[c] - P0[c]; v[c] = P2[c] - P0[c]; }
  double n0 = u[1] * v[2] - u[2] * v[1], n1 = u[2] * v[0] - u[0] * v[2], n2 = u[0] * v[1] - u[1] * v[0];
  t.area = 0.5 * std::sqrt(n0 * n0 + n1 * n1 + n2 * n2);
  t.vid[0] = v0; t.vid[1] = v1; t.vid[2] = v2;
  double d2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    double q = 0.0;
    for (int c = 0; c < 3; ++c) q += (P[(a + 1) % 3][c] - P[a][c]) * (P[(a + 1) % 3][c] - P[a][c]);
    d2 = std::max(d2, q);
  }
  t.diam = std::sqrt(d2);
  return t;
}

static void box_add(std::vector<double>& lo, std::vector<double>& hi, int64_t i, const double* p) {
  for (int c = 0; c < 3; ++c) {
    lo[3 * i + c] = std::min(lo[3 * i + c], p[c]);
    hi[3 * i + c] = std::max(hi[3 * i + c], p[c]);
  }
}

int build_rwg(Space& s, Mesh& m) {
  s.mesh = &m;
  s.kind = CAL_RWG;
  s.ntri = m.nt;
  s.nbasis = m.ne;
  s.nslot = 3;
  s.triD.resize(m.nt);
  s.slot_edge.assign(3 * m.nt, -1);
  s.slot_sw.assign(12 * m.nt, 0.0);
  for (int64_t t = 0; t < m.nt; ++t) {
    const int* v = &m.T[3 * t];
    s.triD[t] = make_tri(&m.X[3 * v[0]], &m.X[3 * v[1]], &m.X[3 * v[2]], v[0], v[1], v[2]);
    for (int a = 0; a < 3; ++a) {
      // RWG on T: sign l/(2|T|) (x - P_a) = sigma (x - c) - sigma (P_a - c)
      int e = m.tri_edge[3 * t + a];
      double sig = m.tri_sign[3 * t + a] * m.e_len[e] / (2.0 * s.triD[t].area);
      s.slot_edge[3 * t + a] = e;
      s.slot_sw[12 * t + 4 * a] = sig;
      for (int c = 0; c < 3; ++c) s.slot_sw[12 * t + 4 * a + 1 + c] = -sig * s.triD[t].off[a][c];
    }
  }
  s.tri_off = m.tri_off;
  s.box_lo.assign(3 * m.ne, 1e300);
  s.box_hi.assign(3 * m.ne, -1e300);
  for (int64_t e = 0; e < m.ne; ++e)
    for (int t : {m.e_tp[e], m.e_tm[e]})
      for (int a = 0; a < 3; ++a) box_add(s.box_lo, s.box_hi, e, &m.X[3 * m.T[3 * t + a]]);
  build_singular_pairs(s);
  return CAL_OK;
}

// BC: sigma_{b,tau} |tau| per cell slot (cell_slot_s), and whether it is one
// constant over each cell (sigma_factors), to 1e-9
static void bc_sigma_factors(Space& s) {
  const int64_t nv = (int64_t)s.cell_tri_ptr.size() - 1;
  s.cell_slot_s.assign(s.cell_edge.size(), 0.0f);
  bool ok = true;
  for (int64_t v = 0; v < nv && ok; ++v) {
    const int t0 = s.cell_tri_ptr[v], t1 = s.cell_tri_ptr[v + 1];
    const int e0 = s.cell_edge_ptr[v], ns = s.cell_edge_ptr[v + 1] - e0;
    if (t1 == t0) continue;
    for (int sl = 0; sl < ns && ok; ++sl) {
      const int tau0 = s.cell_tri[t0];
      const double sb = s.slot_sw[((size_t)tau0 * s.nslot + sl) * 4] * s.triD[tau0].area;
      for (int q = t0; q < t1 && ok; ++q) {
        const int tau = s.cell_tri[q];
        const double v2 = s.slot_sw[((size_t)tau * s.nslot + sl) * 4] * s.triD[tau].area;
        ok = std::abs(v2 - sb) <= 1e-9 * std::abs(sb) + 1e-300;
      }
      s.cell_slot_s[e0 + sl] = (float)sb;
    }
  }
  s.sigma_factors = ok;
}

int build_bc(Space& s, Mesh& m) {
  s.mesh = &m;
  s.kind = CAL_BC;
  const int64_t nv = m.nv, ne = m.ne, nt = m.nt;
  s.ntri = 6 * nt;
  s.nbasis = ne;
  s.nslot = m.max_valence;
  // barycentric vertices: primal v, edge midpoints nv + e, barycentres nv + ne + t
  std::vector<double> Xb(3 * (nv + ne + nt));
  std::copy(m.X.begin(), m.X.end(), Xb.begin());
  for (int64_t e = 0; e < ne; ++e)
    for (int c = 0; c < 3; ++c)
      Xb[3 * (nv + e) + c] = 0.5 * (m.X[3 * m.e_lo[e] + c] + m.X[3 * m.e_hi[e] + c]);
  for (int64_t t = 0; t < nt; ++t)
    for (int c = 0; c < 3; ++c)
      Xb[3 * (nv + ne + t) + c] =
          (m.X[3 * m.T[3 * t] + c] + m.X[3 * m.T[3 * t + 1] + c] + m.X[3 * m.T[3 * t + 2] + c]) / 3.0;
  s.triD.resize(s.ntri);
  s.parent.resize(s.ntri);
  std::vector<int> ids(3 * s.ntri);
  parallel_for((int)nt, [&](int t) {
    int v0 = m.T[3 * t], v1 = m.T[3 * t + 1], v2 = m.T[3 * t + 2];
    // edges opposite local vertices: a=2 -> (v0,v1), a=0 -> (v1,v2), a=1 -> (v2,v0)
    int m01 = (int)nv + m.tri_edge[3 * t + 2];
    int m12 = (int)nv + m.tri_edge[3 * t + 0];
    int m20 = (int)nv + m.tri_edge[3 * t + 1];
    int c = (int)(nv + ne + t);
    int sub[6][3] = {{v0, m01, c}, {m01, v1, c}, {v1, m12, c}, {m12, v2, c}, {v2, m20, c}, {m20, v0, c}};
    for (int k = 0; k < 6; ++k) {
      int64_t tau = 6 * t + k;
      for (int a = 0; a < 3; ++a) ids[3 * tau + a] = sub[k][a];
      s.triD[tau] = make_tri(&Xb[3 * sub[k][0]], &Xb[3 * sub[k][1]], &Xb[3 * sub[k][2]], sub[k][0],
                             sub[k][1], sub[k][2]);
      s.parent[tau] = (int)t;
    }
  });
  // dual cells: barycentric triangles touching each primal vertex
  s.cell_tri_ptr.assign(nv + 1, 0);
  for (int64_t tau = 0; tau < s.ntri; ++tau)
    for (int a = 0; a < 3; ++a)
      if (ids[3 * tau + a] < nv) s.cell_tri_ptr[ids[3 * tau + a] + 1]++;
  for (int64_t v = 0; v < nv; ++v) s.cell_tri_ptr[v + 1] += s.cell_tri_ptr[v];
  s.cell_tri.resize(s.cell_tri_ptr[nv]);
  {
    std::vector<int> fill(s.cell_tri_ptr.begin(), s.cell_tri_ptr.end() - 1);
    for (int64_t tau = 0; tau < s.ntri; ++tau)
      for (int a = 0; a < 3; ++a)
        if (ids[3 * tau + a] < nv) s.cell_tri[fill[ids[3 * tau + a]]++] = (int)tau;
  }
  // edges of each cell (slot order = ascending edge index)
  s.cell_edge_ptr.assign(nv + 1, 0);
  for (int64_t e = 0; e < ne; ++e) { s.cell_edge_ptr[m.e_lo[e] + 1]++; s.cell_edge_ptr[m.e_hi[e] + 1]++; }
  for (int64_t v = 0; v < nv; ++v) s.cell_edge_ptr[v + 1] += s.cell_edge_ptr[v];
  s.cell_edge.resize(s.cell_edge_ptr[nv]);
  {
    std::vector<int> fill(s.cell_edge_ptr.begin(), s.cell_edge_ptr.end() - 1);
    for (int64_t e = 0; e < ne; ++e) {
      s.cell_edge[fill[m.e_lo[e]]++] = (int)e;
      s.cell_edge[fill[m.e_hi[e]]++] = (int)e;
    }
  }
  s.slot_edge.assign((size_t)s.ntri * s.nslot, -1);
  s.slot_sw.assign((size_t)s.ntri * s.nslot * 4, 0.0);
  parallel_for((int)s.ntri, [&](int tau) {
    int v = -1;
    for (int a = 0; a < 3; ++a)
      if (ids[3 * tau + a] < nv) v = ids[3 * tau + a];
    for (int q = s.cell_edge_ptr[v], sl = 0; q < s.cell_edge_ptr[v + 1]; ++q, ++sl)
      s.slot_edge[(size_t)tau * s.nslot + sl] = s.cell_edge[q];
  });
  // BC_e on each dual cell: walk counter-clockwise around v from the spoke
  // (v, mid(e)); spoke j carries flux F_j = sgn l (j/2N - 1/2) (F_0 = 0), the
  // two triangles at mid(e) carry sgn l/2 through the dual edge, and every
  // small triangle gets divergence integral sgn l/(2N).
  // cells are independent (each writes the slots of its own triangles); the
  // first cell that is not a closed fan is reported
  std::atomic<int64_t> bad_fan(-1), bad_walk(-1);
  parallel_for((int)nv, [&](int v) {
    std::vector<std::pair<int, int>> succ;  // s -> (tau, s')
    std::vector<int> succ_key;
    int b0 = s.cell_tri_ptr[v], b1 = s.cell_tri_ptr[v + 1];
    int twoN = b1 - b0;
    if (twoN == 0) return;
    for (int q = b0; q < b1; ++q) {
      int tau = s.cell_tri[q];
      int k = 0;
      while (ids[3 * tau + k] != v) ++k;
      succ_key.push_back(ids[3 * tau + (k + 1) % 3]);
      succ.push_back({tau, ids[3 * tau + (k + 2) % 3]});
    }
    for (int q = s.cell_edge_ptr[v], sl = 0; q < s.cell_edge_ptr[v + 1]; ++q, ++sl) {
      int e = s.cell_edge[q];
      double sgn = (m.e_lo[e] == v) ? 1.0 : -1.0;
      double l = m.e_len[e];
      auto flux = [&](int j) { return (j % twoN == 0) ? 0.0 : sgn * l * ((double)j / twoN - 0.5); };
      int sp = (int)nv + e;
      for (int j = 0; j < twoN; ++j) {
        int pos = (int)(std::find(succ_key.begin(), succ_key.end(), sp) - succ_key.begin());
        if (pos >= twoN) {
          int64_t none = -1;
          bad_fan.compare_exchange_strong(none, v);
          return;
        }
        int tau = succ[pos].first, sn = succ[pos].second;
        double beta[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) {
          int id = ids[3 * tau + a];
          if (id == v) beta[a] = (j == 0 || j == twoN - 1) ? sgn * l * 0.5 : 0.0;
          else if (id == sp) beta[a] = flux(j + 1);
          else if (id == sn) beta[a] = -flux(j);
        }
        const TriD& T = s.triD[tau];
        double sig = (beta[0] + beta[1] + beta[2]) / (2.0 * T.area);
        double* sw = &s.slot_sw[((size_t)tau * s.nslot + sl) * 4];
        sw[0] = sig;
        for (int c = 0; c < 3; ++c)
          sw[1 + c] = -(beta[0] * T.off[0][c] + beta[1] * T.off[1][c] + beta[2] * T.off[2][c]) / (2.0 * T.area);
        sp = sn;
      }
      if (sp != (int)nv + e) {
        int64_t none = -1;
        bad_walk.compare_exchange_strong(none, v);
        return;
      }
    }
  });
  if (bad_fan >= 0)
    return fail(CAL_EMESH, "space_create(BC): dual cell of vertex %lld is not a closed fan", (long long)bad_fan.load());
  if (bad_walk >= 0)
    return fail(CAL_EMESH, "space_create(BC): dual cell walk did not close at vertex %lld", (long long)bad_walk.load());
  // support boxes: union of both dual cells
  s.box_lo.assign(3 * ne, 1e300);
  s.box_hi.assign(3 * ne, -1e300);
  parallel_for((int)ne, [&](int e) {
    for (int v : {m.e_lo[e], m.e_hi[e]})
      for (int q = s.cell_tri_ptr[v]; q < s.cell_tri_ptr[v + 1]; ++q)
        for (int a = 0; a < 3; ++a) box_add(s.box_lo, s.box_hi, e, &Xb[3 * ids[3 * s.cell_tri[q] + a]]);
  });
  s.tri_off.resize(m.M + 1);
  for (int64_t d = 0; d <= m.M; ++d) s.tri_off[d] = 6 * m.tri_off[d];
  bc_sigma_factors(s);
  build_singular_pairs(s);
  return CAL_OK;
}

// Touching triangle pairs per scatterer. Triangles are split into contiguous
// ranges over a few host threads; each range lists its pairs in (t, u) order
// and the ranges are concatenated, so the list is the same for any thread count.
void build_singular_pairs(Space& s) {
  const Mesh& m = *s.mesh;
  s.sing.assign(m.M, {});
  // vertex -> triangles (CSR over the vertex ids of the space's triangles)
  int maxid = 0;
  for (int64_t t = 0; t < s.ntri; ++t)
    for (int a = 0; a < 3; ++a) maxid = std::max(maxid, s.triD[t].vid[a]);
  std::vector<int> vptr(maxid + 2, 0), vtri;
  for (int64_t t = 0; t < s.ntri; ++t)
    for (int a = 0; a < 3; ++a) ++vptr[s.triD[t].vid[a] + 1];
  for (int v = 0; v <= maxid; ++v) vptr[v + 1] += vptr[v];
  vtri.resize(vptr[maxid + 1]);
  {
    std::vector<int> fill(vptr.begin(), vptr.end() - 1);
    for (int64_t t = 0; t < s.ntri; ++t)
      for (int a = 0; a < 3; ++a) vtri[fill[s.triD[t].vid[a]]++] = (int)t;
  }
  for (int64_t d = 0; d < m.M; ++d) {
    const int64_t t0 = s.tri_off[d], t1 = s.tri_off[d + 1];
    const int nth = (int)std::max<int64_t>(
        1, std::min<int64_t>({16, (int64_t)std::thread::hardware_concurrency(), (t1 - t0) / 1024}));
    std::vector<std::vector<SingPair>> part(nth);
    auto work = [&](int w) {
      const int64_t a0 = t0 + (t1 - t0) * w / nth, a1 = t0 + (t1 - t0) * (w + 1) / nth;
      auto& out = part[w];
      out.reserve((size_t)(a1 - a0) * 12);
      std::vector<int> stamp(s.ntri, -1), nb;
      for (int64_t t = a0; t < a1; ++t) {
        nb.clear();
        const int* i1 = s.triD[t].vid;
        for (int a = 0; a < 3; ++a)
          for (int q = vptr[i1[a]]; q < vptr[i1[a] + 1]; ++q) {
            const int u = vtri[q];
            if (stamp[u] != (int)t) {
              stamp[u] = (int)t;
              nb.push_back(u);
            }
          }
        std::sort(nb.begin(), nb.end());
        for (int u : nb) {
          if (u < t0 || u >= t1) continue;  // touching triangles of one scatterer only
          const int* i2 = s.triD[u].vid;
          int shared = 0;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) shared += i1[a] == i2[b];
          // vertex-sharing pairs: keep one order, the kernel adds the transpose
          if (shared == 1 && u < t) continue;
          SingPair p{};
          p.t1 = (int)t;
          p.t2 = u;
          int ns = 0;
          int sh1[3], sh2[3];
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
              if (i1[a] == i2[b]) { sh1[ns] = a; sh2[ns] = b; ++ns; }
          p.cls = (signed char)ns;
          int n1 = 0, n2 = 0;
          for (int q = 0; q < ns; ++q) { p.o1[n1++] = (signed char)sh1[q]; p.o2[n2++] = (signed char)sh2[q]; }
          for (int a = 0; a < 3; ++a) {
            bool u1 = false, u2 = false;
            for (int q = 0; q < ns; ++q) { u1 |= sh1[q] == a; u2 |= sh2[q] == a; }
            if (!u1) p.o1[n1++] = (signed char)a;
            if (!u2) p.o2[n2++] = (signed char)a;
          }
          out.push_back(p);
        }
      }
    };
    if (nth == 1) {
      work(0);
    } else {
      std::vector<std::thread> th;
      for (int w = 0; w < nth; ++w) th.emplace_back(work, w);
      for (auto& x : th) x.join();
    }
    // grouped by class, costliest rules first: lanes of one warp then run the
    // same rule (the float32-output kernel takes one pair per lane)
    // (each range's pairs of a class go after those of the earlier ranges, so
    // the order does not depend on the thread count; the ranges copy in parallel)
    auto rank = [](const SingPair& q) { return q.cls == 2 ? 0 : (q.cls == 3 ? 1 : 2); };
    std::vector<std::array<size_t, 3>> cnt(nth, {0, 0, 0});
    parallel_for(nth, [&](int w) {
      for (const SingPair& q : part[w]) ++cnt[w][rank(q)];
    });
    std::vector<std::array<size_t, 3>> off(nth);
    size_t pos = 0;
    for (int c = 0; c < 3; ++c)
      for (int w = 0; w < nth; ++w) {
        off[w][c] = pos;
        pos += cnt[w][c];
      }
    auto& out = s.sing[d];
    out.resize(pos);
    auto copy = [&](int w) {
      std::array<size_t, 3> o = off[w];
      for (const SingPair& q : part[w]) out[o[rank(q)]++] = q;
    };
    if (nth == 1) {
      copy(0);
    } else {
      std::vector<std::thread> th;
      for (int w = 0; w < nth; ++w) th.emplace_back(copy, w);
      for (auto& x : th) x.join();
    }
  }
}

// Support-box pattern: (i, j) kept iff the boxes are <= chi apart. Box
// centres are binned on a uniform grid of cell size >= (largest box extent +
// chi) / 2, so every partner of i lies within two cells of i's cell; the
// boxes are copied in cell order for contiguous scans, and rows are
// independent and are built by a few host threads.
void near_pattern(const Space& s, int scat, double chi, std::vector<int64_t>& rowptr,
                  std::vector<int>& col) {
  const Mesh& m = *s.mesh;
  const int64_t e0 = scat < 0 ? 0 : m.edge_off[scat];
  const int64_t e1 = scat < 0 ? m.ne : m.edge_off[scat + 1];
  const int64_t n = e1 - e0;
  rowptr.assign(n + 1, 0);
  col.clear();
  if (n == 0) return;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, ext = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) {
      const double a = s.box_lo[3 * (e0 + i) + c], b = s.box_hi[3 * (e0 + i) + c];
      lo[c] = std::min(lo[c], 0.5 * (a + b));
      hi[c] = std::max(hi[c], 0.5 * (a + b));
      ext = std::max(ext, b - a);
    }
  // centres of partners differ by at most ext + chi per coordinate
  double cell = std::max(0.5 * (ext + chi), 1e-300);
  int dim[3];
  for (int c = 0; c < 3; ++c) dim[c] = (int)std::min<double>(std::floor((hi[c] - lo[c]) / cell) + 1, 1 << 20);
  while ((double)dim[0] * dim[1] * dim[2] > 8.0 * (double)n + 64) {  // bounded grid size
    cell *= 1.25;
    for (int c = 0; c < 3; ++c) dim[c] = (int)std::floor((hi[c] - lo[c]) / cell) + 1;
  }
  const int reach = (int)std::ceil((ext + chi) / cell - 1e-12);
  auto cidx = [&](int64_t i, int* g) {
    for (int c = 0; c < 3; ++c) {
      const double x = 0.5 * (s.box_lo[3 * (e0 + i) + c] + s.box_hi[3 * (e0 + i) + c]);
      g[c] = std::min(dim[c] - 1, std::max(0, (int)((x - lo[c]) / cell)));
    }
  };
  const int64_t ncell = (int64_t)dim[0] * dim[1] * dim[2];
  std::vector<int64_t> cptr(ncell + 1, 0);
  std::vector<int> cell_of(n), citems(n);
  for (int64_t i = 0; i < n; ++i) {
    int g[3];
    cidx(i, g);
    cell_of[i] = (int)(((int64_t)g[2] * dim[1] + g[1]) * dim[0] + g[0]);
    ++cptr[cell_of[i] + 1];
  }
  for (int64_t c = 0; c < ncell; ++c) cptr[c + 1] += cptr[c];
  {
    std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
    for (int64_t i = 0; i < n; ++i) citems[fill[cell_of[i]]++] = (int)i;
  }
  // boxes in cell order: bx[6 q .. 6 q + 5] = lo, hi of citems[q]
  std::vector<double> bx(6 * (size_t)n);
  for (int64_t q = 0; q < n; ++q)
    for (int c = 0; c < 3; ++c) {
      bx[6 * q + c] = s.box_lo[3 * (e0 + citems[q]) + c];
      bx[6 * q + 3 + c] = s.box_hi[3 * (e0 + citems[q]) + c];
    }
  const double chi2 = chi * chi;
  const int nth = (int)std::max<int64_t>(1, std::min<int64_t>({16, (int64_t)std::thread::hardware_concurrency(),
                                                                 n / 256 + 1}));
  std::vector<std::vector<int>> cols(nth);
  std::vector<std::vector<int64_t>> counts(nth);
  auto work = [&](int w) {
    const int64_t r0 = n * w / nth, r1 = n * (w + 1) / nth;
    auto& cw = cols[w];
    auto& nw = counts[w];
    nw.assign(r1 - r0, 0);
    std::vector<int> row;
    for (int64_t i = r0; i < r1; ++i) {
      row.clear();
      const double* li = &s.box_lo[3 * (e0 + i)];
      const double* hi_ = &s.box_hi[3 * (e0 + i)];
      int g[3];
      cidx(i, g);
      for (int z = std::max(0, g[2] - reach); z <= std::min(dim[2] - 1, g[2] + reach); ++z)
        for (int y = std::max(0, g[1] - reach); y <= std::min(dim[1] - 1, g[1] + reach); ++y) {
          // cells x0..x1 of this (y, z) line are contiguous in cell order
          const int x0 = std::max(0, g[0] - reach), x1 = std::min(dim[0] - 1, g[0] + reach);
          const int64_t c0 = ((int64_t)z * dim[1] + y) * dim[0];
          for (int64_t q = cptr[c0 + x0]; q < cptr[c0 + x1 + 1]; ++q) {
            const double* b = &bx[6 * q];
            double g2 = 0;
            for (int k = 0; k < 3; ++k) {
              const double gap = std::max(0.0, std::max(b[k] - hi_[k], li[k] - b[3 + k]));
              g2 += gap * gap;
            }
            if (g2 <= chi2) row.push_back(citems[q]);
          }
        }
      std::sort(row.begin(), row.end());
      cw.insert(cw.end(), row.begin(), row.end());
      nw[i - r0] = (int64_t)row.size();
    }
  };
  if (nth == 1) {
    work(0);
  } else {
    std::vector<std::thread> th;
    for (int w = 0; w < nth; ++w) th.emplace_back(work, w);
    for (auto& t : th) t.join();
  }
  int64_t k = 0;
  for (int w = 0; w < nth; ++w) {
    const int64_t r0 = n * w / nth;
    for (size_t q = 0; q < counts[w].size(); ++q) rowptr[r0 + q + 1] = (k += counts[w][q]);
  }
  col.reserve(k);
  for (int w = 0; w < nth; ++w) col.insert(col.end(), cols[w].begin(), cols[w].end());
}

void gram_pattern(const Space& bc, std::vector<int64_t>& rowptr, std::vector<int>& col) {
  const Mesh& m = *bc.mesh;
  std::vector<std::vector<int>> rows(m.ne);
  for (int64_t tau = 0; tau < bc.ntri; ++tau) {
    int t = bc.parent[tau];
    for (int a = 0; a < 3; ++a) {
      int i = m.tri_edge[3 * t + a];
      for (int sl = 0; sl < bc.nslot; ++sl) {
        int j = bc.slot_edge[(size_t)tau * bc.nslot + sl];
        if (j >= 0) rows[i].push_back(j);
      }
    }
  }
  rowptr.assign(m.ne + 1, 0);
  col.clear();
  for (int64_t i = 0; i < m.ne; ++i) {
    auto& r = rows[i];
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    col.insert(col.end(), r.begin(), r.end());
    rowptr[i + 1] = (int64_t)col.size();
  }
}

// ---------------------------------------------------------------------------
// device upload
// ---------------------------------------------------------------------------
template <typename T>
static int upload(T** dst, const T* src, size_t n, cudaStream_t st) {
  if (n == 0) { *dst = nullptr; return CAL_OK; }
  if (dalloc((void**)dst, n * sizeof(T), st) != cudaSuccess)
    return fail(CAL_ENOMEM, "device allocation of %zu bytes failed", n * sizeof(T));
  CAL_TRY_CUDA(cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, st));
  return CAL_OK;
}

int upload_space(Space& s, cudaStream_t st) {
  std::vector<TriF> tf(s.ntri);
  for (int64_t t = 0; t < s.ntri; ++t) {
    const TriD& d = s.triD[t];
    TriF f{};
    for (int c = 0; c < 3; ++c) {
      f.chi[c] = (float)d.c[c];
      f.clo[c] = (float)(d.c[c] - (double)f.chi[c]);
      for (int a = 0; a < 3; ++a) f.off[a][c] = (float)d.off[a][c];
    }
    f.area = (float)d.area;
    f.diam = (float)d.diam;
    for (int a = 0; a < 3; ++a) f.vid[a] = d.vid[a];
    tf[t] = f;
  }
  std::vector<float> swf(s.slot_sw.begin(), s.slot_sw.end());
  int rc;
  if ((rc = upload(&s.d_triF, tf.data(), tf.size(), st))) return rc;
  if ((rc = upload(&s.d_triD, s.triD.data(), s.triD.size(), st))) return rc;
  if ((rc = upload(&s.d_slot_edge, s.slot_edge.data(), s.slot_edge.size(), st))) return rc;
  if ((rc = upload(&s.d_slot_swf, swf.data(), swf.size(), st))) return rc;
  if ((rc = upload(&s.d_slot_swd, s.slot_sw.data(), s.slot_sw.size(), st))) return rc;
  if (s.kind == CAL_BC) {
    if ((rc = upload(&s.d_cell_slot_s, s.cell_slot_s.data(), std::max<size_t>(s.cell_slot_s.size(), 1), st)))
      return rc;
    if ((rc = upload(&s.d_cell_tri_ptr, s.cell_tri_ptr.data(), s.cell_tri_ptr.size(), st))) return rc;
    if ((rc = upload(&s.d_cell_tri, s.cell_tri.data(), s.cell_tri.size(), st))) return rc;
    if ((rc = upload(&s.d_cell_edge_ptr, s.cell_edge_ptr.data(), s.cell_edge_ptr.size(), st))) return rc;
    if ((rc = upload(&s.d_cell_edge, s.cell_edge.data(), s.cell_edge.size(), st))) return rc;
  }
  s.d_sing.assign(s.sing.size(), nullptr);
  for (size_t d = 0; d < s.sing.size(); ++d)
    if ((rc = upload(&s.d_sing[d], s.sing[d].data(), s.sing[d].size(), st))) return rc;
  // the host arrays are pageable and some are locals: wait until the copies have read them
  CAL_TRY_CUDA(cudaStreamSynchronize(st));
  return CAL_OK;
}

// Long-lived objects are used only by calls that return after their GPU work
// has completed, so their memory is released in order on the legacy stream: no
// context (whose stream might already be destroyed) is needed at that point.
Space::~Space() {
  for (void* p : {(void*)d_triF, (void*)d_triD, (void*)d_slot_edge, (void*)d_slot_swf, (void*)d_slot_swd,
                  (void*)d_cell_tri_ptr, (void*)d_cell_tri, (void*)d_cell_edge_ptr, (void*)d_cell_edge,
                  (void*)d_cell_slot_s})
    dfree(p, nullptr);
  for (auto p : d_sing) dfree(p, nullptr);
  for (auto& e : sing_static) {
    dfree(e.buf, nullptr);
    if (e.done) cudaEventDestroy(e.done);
  }
  for (auto& u : unit_lists) {
    dfree(u->d_units, nullptr);
    dfree(u->d_wlist, nullptr);
    if (u->done) cudaEventDestroy(u->done);
  }
}

HMat::~HMat() {
  dfree(d_idx, nullptr);
  dfree(d_near_tab, nullptr);
  dfree(d_roff_near, nullptr);
  dfree(d_roff_far, nullptr);
  for (int q = 0; q < 2; ++q)
    for (void* p : {d_near[q], d_U[q], d_V[q], (void*)d_far_tab[q], (void*)d_koff[q]}) dfree(p, nullptr);
}

Op::~Op() {
  delete hmat;
  dfree(d_S, nullptr);
  dfree(d_C, nullptr);
  dfree(d_rowptr, nullptr);
  dfree(d_col, nullptr);
}

}  // namespace cal
