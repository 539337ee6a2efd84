// Galerkin assembly of the Maxwell operators S and C on sm_103a.
//
// arXiv 2008.04772, Section 2 (operators, G = e^{ikr}/(4 pi r)) and Section 3.3
// (tensor Gauss rules on regular triangle pairs, Sauter–Schwab rules on pairs
// sharing a vertex, an edge or the whole triangle).
//
// Every basis piece on a triangle is phi = sigma (x - c) + w (see internal.h).
// For a triangle pair with centroids c1, c2, Delta = c1 - c2, local points
// xi = x - c1, eta = y - c2, the kernel sums eighteen complex moments
//   S: G0 = sum G,  Gx = sum G xi,  Gy = sum G eta,  Gxy = sum G xi.eta
//   C: g0 = sum g,  gx = sum g xi,  gy = sum g eta,  gxy = sum g xi x eta
// (weights w_p |T1| w_q |T2| folded in; grad_x G = g (x - y)), turns them into
// "pair coefficients"
//   s = Delta.gxy, X1 = Delta x gx + gxy, X2 = gy x Delta - gxy,
//   V = Delta g0 + gx - gy,
// and every (test piece a, trial piece b) entry follows in closed form:
//   S_ab = -ik [sa sb Gxy + sa wb.Gx + sb wa.Gy + (wa.wb) G0] + (4i/k) sa sb G0
//   C_ab = sa sb s + sa wb.X1 + sb wa.X2 + wa.(wb x V).
// Local coordinates relative to the centroids keep float32 free of
// cancellation; Delta is formed from hi+lo float centroids.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "internal.h"

namespace cal {

// ---------------------------------------------------------------------------
// rules passed by value
// ---------------------------------------------------------------------------
// Regular rules: nreg = 6 or 1 applies that rule to every regular pair (table
// entries 0 .. nreg-1). nreg = 0 selects by the pair's class (Section 3.3,
// default orders q_near, q_medium, q_far = 4, 3, 2): the near rule (6 points)
// at entries 0..5, the medium rule (4 points) at 6..9, the far rule (3 points)
// at 10..12. A pair is near if |c1 - c2| <= 2 max(d1, d2), medium if <= 4 max,
// far otherwise (c centroids, d longest edges; the paper states no bounds), the
// bounds with a relative margin of 2^-20 (pair_class).
struct Rules {
  float rbf[39], rwf[13];
  double rbd[39], rwd[13];
  double gx[16], gw[16];
  int nreg, ng;
};
constexpr int RULE_OFF_MEDIUM = 6, RULE_OFF_FAR = 10, RULE_POINTS_ALL = 13;

// per host thread: request streams driven from several threads may use different rules
static thread_local Rules g_rules;

int set_quadrature_tables(int nreg, int nsing) {
  if (nreg != 6 && nreg != 1 && nreg != 0)
    return fail(CAL_EINVAL, "q_regular must be 6, 1 or 0 (classes) (got %d)", nreg);
  if (nsing < 1 || nsing > 16) return fail(CAL_EINVAL, "q_singular must be in 1..16 (got %d)", nsing);
  std::vector<double> x, gw;
  gauss_legendre01(nsing, x, gw);
  Rules r{};
  int at = 0;
  for (int n : (nreg == 0 ? std::vector<int>{6, 4, 3} : std::vector<int>{nreg})) {
    std::vector<double> b, w;
    triangle_rule(n, b, w);
    for (int i = 0; i < 3 * n; ++i) { r.rbd[3 * at + i] = b[i]; r.rbf[3 * at + i] = (float)b[i]; }
    for (int i = 0; i < n; ++i) { r.rwd[at + i] = w[i]; r.rwf[at + i] = (float)w[i]; }
    at += n;
  }
  for (int i = 0; i < nsing; ++i) { r.gx[i] = x[i]; r.gw[i] = gw[i]; }
  r.nreg = nreg;
  r.ng = nsing;
  g_rules = r;
  return CAL_OK;
}

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
template <typename R>
struct V3 { R x, y, z; };

template <typename R>
__device__ __forceinline__ V3<R> v3(R a, R b, R c) { return {a, b, c}; }

template <typename R>
__device__ __forceinline__ R dot3(const V3<R>& a, const V3<R>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename R>
__device__ __forceinline__ V3<R> cross3(const V3<R>& a, const V3<R>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// ---------------------------------------------------------------------------
// kernel values G = e^{ikr}/(4 pi r) and g = (ikr - 1) e^{ikr}/(4 pi r^3)
// ---------------------------------------------------------------------------
// w4: quadrature weight over 4 pi, folded into the amplitude
__device__ __forceinline__ void green4(float r2, float kr, float ki, float& Gr, float& Gi,
                                       float& gr, float& gi, float w4) {
  const float rinv = rsqrtf(r2);
  const float r = r2 * rinv;
  const float ph = kr * r;
  // Cody–Waite reduction of the phase to [-pi, pi] with 2 pi split in two
  // floats (hi exact in 24 bits, lo the float32 remainder of the float64 value)
  constexpr double TWO_PI = 6.283185307179586476925286766559;
  constexpr float TP_HI = (float)TWO_PI;
  constexpr float TP_LO = (float)(TWO_PI - (double)(float)TWO_PI);
  constexpr float INV_TP = (float)(1.0 / TWO_PI);
  const float n = rintf(ph * INV_TP);
  float th = fmaf(-n, TP_HI, ph);
  th = fmaf(-n, TP_LO, th);
  float s, c;
  __sincosf(th, &s, &c);
  float amp = rinv * w4;
  if (ki != 0.0f) amp *= __expf(-ki * r);
  Gr = amp * c;
  Gi = amp * s;
  const float fr = (-ki * r - 1.0f) * rinv * rinv;
  const float fi = kr * rinv;
  gr = Gr * fr - Gi * fi;
  gi = Gr * fi + Gi * fr;
}

constexpr float INV_4PI_F = (float)(0.25 / 3.14159265358979323846);

// w: quadrature weight folded into the amplitude (pass 1 for none)
__device__ __forceinline__ void green(float r2, float kr, float ki, float& Gr, float& Gi,
                                      float& gr, float& gi, float w = 1.0f) {
  green4(r2, kr, ki, Gr, Gi, gr, gi, w * INV_4PI_F);
}

__device__ __forceinline__ void green(double r2, double kr, double ki, double& Gr, double& Gi,
                                      double& gr, double& gi, double w = 1.0) {
  const double r = sqrt(r2);
  const double rinv = 1.0 / r;
  double s, c;
  sincos(kr * r, &s, &c);
  double amp = rinv * (w * (0.25 / 3.14159265358979323846));
  if (ki != 0.0) amp *= exp(-ki * r);
  Gr = amp * c;
  Gi = amp * s;
  const double fr = (-ki * r - 1.0) * rinv * rinv;
  const double fi = kr * rinv;
  gr = Gr * fr - Gi * fi;
  gi = Gr * fi + Gi * fr;
}

// ---------------------------------------------------------------------------
// moments -> pair coefficients
// ---------------------------------------------------------------------------
template <typename R>
struct Mom {
  // S moments
  R G0r, G0i, Gxyr, Gxyi;
  V3<R> Gxr, Gxi, Gyr, Gyi;
  // C moments
  R g0r, g0i;
  V3<R> gxr, gxi, gyr, gyi, gxyr, gxyi;
  __device__ void zero() {
    G0r = G0i = Gxyr = Gxyi = g0r = g0i = R(0);
    Gxr = Gxi = Gyr = Gyi = gxr = gxi = gyr = gyi = gxyr = gxyi = {R(0), R(0), R(0)};
  }
};

// 18 complex pair coefficients, as 36 reals in a fixed order:
//  0..1 G0, 2..7 Gx, 8..13 Gy, 14..15 Gxy, 16..17 s, 18..23 X1, 24..29 X2, 30..35 V
// complex vectors are stored (re x, re y, re z, im x, im y, im z)
template <typename R>
__device__ __forceinline__ void pair_coeffs(const Mom<R>& m, const V3<R>& D, R* pc) {
  pc[0] = m.G0r; pc[1] = m.G0i;
  pc[2] = m.Gxr.x; pc[3] = m.Gxr.y; pc[4] = m.Gxr.z; pc[5] = m.Gxi.x; pc[6] = m.Gxi.y; pc[7] = m.Gxi.z;
  pc[8] = m.Gyr.x; pc[9] = m.Gyr.y; pc[10] = m.Gyr.z; pc[11] = m.Gyi.x; pc[12] = m.Gyi.y; pc[13] = m.Gyi.z;
  pc[14] = m.Gxyr; pc[15] = m.Gxyi;
  pc[16] = dot3(D, m.gxyr);
  pc[17] = dot3(D, m.gxyi);
  V3<R> a = cross3(D, m.gxr), b = cross3(D, m.gxi);
  pc[18] = a.x + m.gxyr.x; pc[19] = a.y + m.gxyr.y; pc[20] = a.z + m.gxyr.z;
  pc[21] = b.x + m.gxyi.x; pc[22] = b.y + m.gxyi.y; pc[23] = b.z + m.gxyi.z;
  a = cross3(m.gyr, D); b = cross3(m.gyi, D);
  pc[24] = a.x - m.gxyr.x; pc[25] = a.y - m.gxyr.y; pc[26] = a.z - m.gxyr.z;
  pc[27] = b.x - m.gxyi.x; pc[28] = b.y - m.gxyi.y; pc[29] = b.z - m.gxyi.z;
  pc[30] = D.x * m.g0r + m.gxr.x - m.gyr.x;
  pc[31] = D.y * m.g0r + m.gxr.y - m.gyr.y;
  pc[32] = D.z * m.g0r + m.gxr.z - m.gyr.z;
  pc[33] = D.x * m.g0i + m.gxi.x - m.gyi.x;
  pc[34] = D.y * m.g0i + m.gxi.y - m.gyi.y;
  pc[35] = D.z * m.g0i + m.gxi.z - m.gyi.z;
}

// entry of one (test piece a, trial piece b) combination from pair coefficients
template <typename R>
__device__ __forceinline__ void entry_from_pc(const R* pc, R sa, const V3<R>& wa, R sb,
                                              const V3<R>& wb, R mikr, R miki, R c4r, R c4i,
                                              bool wantS, bool wantC, R& Sr, R& Si, R& Cr,
                                              R& Ci) {
  if (wantS) {
    const R ss = sa * sb;
    const V3<R> Gxr = {pc[2], pc[3], pc[4]}, Gxi = {pc[5], pc[6], pc[7]};
    const V3<R> Gyr = {pc[8], pc[9], pc[10]}, Gyi = {pc[11], pc[12], pc[13]};
    const R ww = dot3(wa, wb);
    const R br = ss * pc[14] + sa * dot3(wb, Gxr) + sb * dot3(wa, Gyr) + ww * pc[0];
    const R bi = ss * pc[15] + sa * dot3(wb, Gxi) + sb * dot3(wa, Gyi) + ww * pc[1];
    Sr = mikr * br - miki * bi + ss * (c4r * pc[0] - c4i * pc[1]);
    Si = mikr * bi + miki * br + ss * (c4r * pc[1] + c4i * pc[0]);
  }
  if (wantC) {
    const R ss = sa * sb;
    const V3<R> X1r = {pc[18], pc[19], pc[20]}, X1i = {pc[21], pc[22], pc[23]};
    const V3<R> X2r = {pc[24], pc[25], pc[26]}, X2i = {pc[27], pc[28], pc[29]};
    const V3<R> Vr = {pc[30], pc[31], pc[32]}, Vi = {pc[33], pc[34], pc[35]};
    const V3<R> wxw = cross3(wa, wb);
    Cr = ss * pc[16] + sa * dot3(wb, X1r) + sb * dot3(wa, X2r) + dot3(wxw, Vr);
    Ci = ss * pc[17] + sa * dot3(wb, X1i) + sb * dot3(wa, X2i) + dot3(wxw, Vi);
  }
}

// ---------------------------------------------------------------------------
// output sinks: dense (atomics into a row-major block) or CSR (row search)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void atomic_add_c(float* base, int64_t idx, float re, float im) {
  atomicAdd(reinterpret_cast<float2*>(base) + idx, make_float2(re, im));
}
__device__ __forceinline__ void atomic_add_c(double* base, int64_t idx, double re, double im) {
  atomicAdd(base + 2 * idx, re);
  atomicAdd(base + 2 * idx + 1, im);
}

template <typename RO>
struct Sink {
  RO* S;
  RO* C;
  int64_t off;           // first basis index of the block
  int64_t ld;            // dense leading dimension; 0 for CSR
  const int64_t* rowptr; // CSR
  const int* col;
  __device__ __forceinline__ int64_t index(int i, int j) const {
    const int64_t li = i - off, lj = j - off;
    if (ld) return li * ld + lj;
    int64_t lo = rowptr[li], hi = rowptr[li + 1] - 1;
    while (lo <= hi) {
      int64_t mid = (lo + hi) >> 1;
      int c = col[mid];
      if (c == lj) return mid;
      if (c < lj) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
  }
  template <typename V>
  __device__ __forceinline__ void add(int i, int j, bool wS, bool wC, V Sr, V Si, V Cr, V Ci) const {
    const int64_t k = index(i, j);
    if (k < 0) return;
    if (wS) atomic_add_c(S, k, (RO)Sr, (RO)Si);
    if (wC) atomic_add_c(C, k, (RO)Cr, (RO)Ci);
  }
};

// ---------------------------------------------------------------------------
// regular-pair quadrature over the tensor rule (NREG points per triangle)
// ---------------------------------------------------------------------------
template <typename R, int NREG>
__device__ __forceinline__ void regular_moments(const V3<R>* xi, const R* wx, const V3<R>* eta,
                                                const R* wy, const V3<R>& D, R kr, R ki,
                                                bool wantC, Mom<R>& m) {
  m.zero();
#pragma unroll
  for (int p = 0; p < NREG; ++p) {
    R s0r = 0, s0i = 0, t0r = 0, t0i = 0;
    V3<R> ser = {0, 0, 0}, sei = {0, 0, 0}, ter = {0, 0, 0}, tei = {0, 0, 0};
    const V3<R> dp = {D.x + xi[p].x, D.y + xi[p].y, D.z + xi[p].z};
#pragma unroll
    for (int q = 0; q < NREG; ++q) {
      const R dx = dp.x - eta[q].x, dy = dp.y - eta[q].y, dz = dp.z - eta[q].z;
      R Gr, Gi, gr, gi;
      green(dx * dx + dy * dy + dz * dz, kr, ki, Gr, Gi, gr, gi);
      Gr *= wy[q]; Gi *= wy[q]; gr *= wy[q]; gi *= wy[q];
      s0r += Gr; s0i += Gi;
      ser.x += Gr * eta[q].x; ser.y += Gr * eta[q].y; ser.z += Gr * eta[q].z;
      sei.x += Gi * eta[q].x; sei.y += Gi * eta[q].y; sei.z += Gi * eta[q].z;
      if (wantC) {
        t0r += gr; t0i += gi;
        ter.x += gr * eta[q].x; ter.y += gr * eta[q].y; ter.z += gr * eta[q].z;
        tei.x += gi * eta[q].x; tei.y += gi * eta[q].y; tei.z += gi * eta[q].z;
      }
    }
    const R w = wx[p];
    const V3<R> x = xi[p];
    m.G0r += w * s0r; m.G0i += w * s0i;
    m.Gxr.x += w * x.x * s0r; m.Gxr.y += w * x.y * s0r; m.Gxr.z += w * x.z * s0r;
    m.Gxi.x += w * x.x * s0i; m.Gxi.y += w * x.y * s0i; m.Gxi.z += w * x.z * s0i;
    m.Gyr.x += w * ser.x; m.Gyr.y += w * ser.y; m.Gyr.z += w * ser.z;
    m.Gyi.x += w * sei.x; m.Gyi.y += w * sei.y; m.Gyi.z += w * sei.z;
    m.Gxyr += w * dot3(x, ser); m.Gxyi += w * dot3(x, sei);
    if (wantC) {
      m.g0r += w * t0r; m.g0i += w * t0i;
      m.gxr.x += w * x.x * t0r; m.gxr.y += w * x.y * t0r; m.gxr.z += w * x.z * t0r;
      m.gxi.x += w * x.x * t0i; m.gxi.y += w * x.y * t0i; m.gxi.z += w * x.z * t0i;
      m.gyr.x += w * ter.x; m.gyr.y += w * ter.y; m.gyr.z += w * ter.z;
      m.gyi.x += w * tei.x; m.gyi.y += w * tei.y; m.gyi.z += w * tei.z;
      const V3<R> cr = cross3(x, ter), ci = cross3(x, tei);
      m.gxyr.x += w * cr.x; m.gxyr.y += w * cr.y; m.gxyr.z += w * cr.z;
      m.gxyi.x += w * ci.x; m.gxyi.y += w * ci.y; m.gxyi.z += w * ci.z;
    }
  }
}

// same sums with both point sets staged as (x, y, z, weight) quadruples
template <typename R> struct __align__(4 * sizeof(R)) P4 { R x, y, z, w; };

template <typename R, int NREG>
__device__ __forceinline__ void regular_moments_staged(const P4<R>* __restrict__ X,
                                                       const P4<R>* __restrict__ Y, const V3<R>& D,
                                                       R kr, R ki, bool wantC, Mom<R>& m) {
  m.zero();
#pragma unroll 2
  for (int p = 0; p < NREG; ++p) {
    const P4<R> xp = X[p];
    R s0r = 0, s0i = 0, t0r = 0, t0i = 0;
    V3<R> ser = {0, 0, 0}, sei = {0, 0, 0}, ter = {0, 0, 0}, tei = {0, 0, 0};
    const V3<R> dp = {D.x + xp.x, D.y + xp.y, D.z + xp.z};
#pragma unroll
    for (int q = 0; q < NREG; ++q) {
      const P4<R> yq = Y[q];
      const R dx = dp.x - yq.x, dy = dp.y - yq.y, dz = dp.z - yq.z;
      R Gr, Gi, gr, gi;
      green(dx * dx + dy * dy + dz * dz, kr, ki, Gr, Gi, gr, gi, yq.w);
      s0r += Gr; s0i += Gi;
      ser.x += Gr * yq.x; ser.y += Gr * yq.y; ser.z += Gr * yq.z;
      sei.x += Gi * yq.x; sei.y += Gi * yq.y; sei.z += Gi * yq.z;
      if (wantC) {
        t0r += gr; t0i += gi;
        ter.x += gr * yq.x; ter.y += gr * yq.y; ter.z += gr * yq.z;
        tei.x += gi * yq.x; tei.y += gi * yq.y; tei.z += gi * yq.z;
      }
    }
    const R w = xp.w;
    const V3<R> x = {xp.x, xp.y, xp.z};
    m.G0r += w * s0r; m.G0i += w * s0i;
    m.Gxr.x += w * x.x * s0r; m.Gxr.y += w * x.y * s0r; m.Gxr.z += w * x.z * s0r;
    m.Gxi.x += w * x.x * s0i; m.Gxi.y += w * x.y * s0i; m.Gxi.z += w * x.z * s0i;
    m.Gyr.x += w * ser.x; m.Gyr.y += w * ser.y; m.Gyr.z += w * ser.z;
    m.Gyi.x += w * sei.x; m.Gyi.y += w * sei.y; m.Gyi.z += w * sei.z;
    m.Gxyr += w * dot3(x, ser); m.Gxyi += w * dot3(x, sei);
    if (wantC) {
      m.g0r += w * t0r; m.g0i += w * t0i;
      m.gxr.x += w * x.x * t0r; m.gxr.y += w * x.y * t0r; m.gxr.z += w * x.z * t0r;
      m.gxi.x += w * x.x * t0i; m.gxi.y += w * x.y * t0i; m.gxi.z += w * x.z * t0i;
      m.gyr.x += w * ter.x; m.gyr.y += w * ter.y; m.gyr.z += w * ter.z;
      m.gyi.x += w * tei.x; m.gyi.y += w * tei.y; m.gyi.z += w * tei.z;
      const V3<R> cr = cross3(x, ter), ci = cross3(x, tei);
      m.gxyr.x += w * cr.x; m.gxyr.y += w * cr.y; m.gxyr.z += w * cr.z;
      m.gxyi.x += w * ci.x; m.gxyi.y += w * ci.y; m.gxyi.z += w * ci.z;
    }
  }
}

// one quadrature point of a triangle (relative to its centroid) and its weight
__device__ __forceinline__ P4<float> staged_point(const TriF& t, const Rules& rl, int q) {
  const float b0 = rl.rbf[3 * q], b1 = rl.rbf[3 * q + 1], b2 = rl.rbf[3 * q + 2];
  return {b0 * t.off[0][0] + b1 * t.off[1][0] + b2 * t.off[2][0],
          b0 * t.off[0][1] + b1 * t.off[1][1] + b2 * t.off[2][1],
          b0 * t.off[0][2] + b1 * t.off[1][2] + b2 * t.off[2][2], rl.rwf[q] * t.area};
}
__device__ __forceinline__ P4<double> staged_point(const TriD& t, const Rules& rl, int q) {
  const double b0 = rl.rbd[3 * q], b1 = rl.rbd[3 * q + 1], b2 = rl.rbd[3 * q + 2];
  return {b0 * t.off[0][0] + b1 * t.off[1][0] + b2 * t.off[2][0],
          b0 * t.off[0][1] + b1 * t.off[1][1] + b2 * t.off[2][1],
          b0 * t.off[0][2] + b1 * t.off[1][2] + b2 * t.off[2][2], rl.rwd[q] * t.area};
}

// centroid difference from staged centroids: float keeps hi + lo parts
template <typename R> struct Cent;
template <> struct Cent<float> {
  float hi[3], lo[3], d;  // d: longest edge
  __device__ void set(const TriF& t) {
    for (int c = 0; c < 3; ++c) { hi[c] = t.chi[c]; lo[c] = t.clo[c]; }
    d = t.diam;
  }
  __device__ V3<float> minus(const Cent& b) const {
    return {(hi[0] - b.hi[0]) + (lo[0] - b.lo[0]), (hi[1] - b.hi[1]) + (lo[1] - b.lo[1]),
            (hi[2] - b.hi[2]) + (lo[2] - b.lo[2])};
  }
};
template <> struct Cent<double> {
  double c[3], d;  // d: longest edge
  __device__ void set(const TriD& t) {
    for (int q = 0; q < 3; ++q) c[q] = t.c[q];
    d = t.diam;
  }
  __device__ V3<double> minus(const Cent& b) const { return {c[0] - b.c[0], c[1] - b.c[1], c[2] - b.c[2]}; }
};

// triangle loaders: quadrature points relative to the centroid and weights
template <int NREG>
__device__ __forceinline__ void load_points(const TriF& t, const Rules& rl, V3<float>* p, float* w, int off = 0) {
#pragma unroll
  for (int q = 0; q < NREG; ++q) {
    const float b0 = rl.rbf[3 * (off + q)], b1 = rl.rbf[3 * (off + q) + 1], b2 = rl.rbf[3 * (off + q) + 2];
    p[q] = {b0 * t.off[0][0] + b1 * t.off[1][0] + b2 * t.off[2][0],
            b0 * t.off[0][1] + b1 * t.off[1][1] + b2 * t.off[2][1],
            b0 * t.off[0][2] + b1 * t.off[1][2] + b2 * t.off[2][2]};
    w[q] = rl.rwf[off + q] * t.area;
  }
}
template <int NREG>
__device__ __forceinline__ void load_points(const TriD& t, const Rules& rl, V3<double>* p, double* w, int off = 0) {
#pragma unroll
  for (int q = 0; q < NREG; ++q) {
    const double b0 = rl.rbd[3 * (off + q)], b1 = rl.rbd[3 * (off + q) + 1], b2 = rl.rbd[3 * (off + q) + 2];
    p[q] = {b0 * t.off[0][0] + b1 * t.off[1][0] + b2 * t.off[2][0],
            b0 * t.off[0][1] + b1 * t.off[1][1] + b2 * t.off[2][1],
            b0 * t.off[0][2] + b1 * t.off[1][2] + b2 * t.off[2][2]};
    w[q] = rl.rwd[off + q] * t.area;
  }
}
__device__ __forceinline__ V3<float> centroid_delta(const TriF& a, const TriF& b) {
  return {(a.chi[0] - b.chi[0]) + (a.clo[0] - b.clo[0]), (a.chi[1] - b.chi[1]) + (a.clo[1] - b.clo[1]),
          (a.chi[2] - b.chi[2]) + (a.clo[2] - b.clo[2])};
}
__device__ __forceinline__ V3<double> centroid_delta(const TriD& a, const TriD& b) {
  return {a.c[0] - b.c[0], a.c[1] - b.c[1], a.c[2] - b.c[2]};
}
template <typename TRI>
__device__ __forceinline__ bool touching(const TRI& a, const TRI& b) {
  bool t = false;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) t |= (a.vid[i] == b.vid[j]);
  return t;
}

// class of a regular pair: 0 near, 1 medium, 2 far: |D|^2 against (2 b dmax)^2
// and (4 b dmax)^2 with b = 1 + 2^-20 (a margin far above float32 rounding of
// the distance, so that ties exactly at 2 or 4 are near / medium on every path)
template <typename R>
__device__ __forceinline__ int pair_class(const V3<R>& D, R d1, R d2) {
  constexpr double B = 1.0 + 1.0 / 1048576.0;
  const R dm = d1 > d2 ? d1 : d2;
  const R r2 = D.x * D.x + D.y * D.y + D.z * D.z, m2 = dm * dm;
  return r2 <= R(4.0 * B * B) * m2 ? 0 : (r2 <= R(16.0 * B * B) * m2 ? 1 : 2);
}

template <typename R, int N, typename TRI>
__device__ __forceinline__ void pair_moments_n(const TRI& A, const TRI& B, const Rules& rl, int off, const V3<R>& D,
                                               R kr, R ki, bool wantC, Mom<R>& m) {
  V3<R> xi[N], eta[N];
  R wx[N], wy[N];
  load_points<N>(A, rl, xi, wx, off);
  load_points<N>(B, rl, eta, wy, off);
  regular_moments<R, N>(xi, wx, eta, wy, D, kr, ki, wantC, m);
}

// moments of a regular pair with the rule NREG (6 or 1), or by class (NREG 0);
// returns the integrand evaluations
template <typename R, int NREG, typename TRI>
__device__ __forceinline__ int pair_moments(const TRI& A, const TRI& B, const Rules& rl, const V3<R>& D, R kr, R ki,
                                            bool wantC, Mom<R>& m) {
  if constexpr (NREG > 0) {
    pair_moments_n<R, NREG>(A, B, rl, 0, D, kr, ki, wantC, m);
    return NREG * NREG;
  } else {
    const int c = pair_class<R>(D, (R)A.diam, (R)B.diam);
    if (c == 2) { pair_moments_n<R, 3>(A, B, rl, RULE_OFF_FAR, D, kr, ki, wantC, m); return 9; }
    if (c == 1) { pair_moments_n<R, 4>(A, B, rl, RULE_OFF_MEDIUM, D, kr, ki, wantC, m); return 16; }
    pair_moments_n<R, 6>(A, B, rl, 0, D, kr, ki, wantC, m);
    return 36;
  }
}

// adds a per-thread count to *cnt with one atomic per converged group of lanes
__device__ __forceinline__ void count_add(unsigned long long* cnt, unsigned v) {
  if (!cnt) return;
  unsigned lane;
  asm volatile("mov.u32 %0, %%laneid;" : "=r"(lane));
  const unsigned mask = __activemask();
  const unsigned tot = __reduce_add_sync(mask, v);
  if (lane == (unsigned)(__ffs(mask) - 1) && tot) atomicAdd(cnt, (unsigned long long)tot);
}

template <typename R> struct TriOf;
template <> struct TriOf<float> { using T = TriF; };
template <> struct TriOf<double> { using T = TriD; };

// ---------------------------------------------------------------------------
// A3: regular RWG pairs, one thread per unordered pair t1 < t2 (the rule is
// symmetric in the two triangles and both operators are symmetric, so each
// result is added at (i, j) and (j, i)); touching pairs are left to the
// singular kernel.
// ---------------------------------------------------------------------------
template <typename R, int NREG>
__global__ void __launch_bounds__(256) rwg_regular_kernel(
    const typename TriOf<R>::T* __restrict__ tri, const int* __restrict__ slot_edge,
    const R* __restrict__ slot_sw, int64_t t0, int64_t ntr, R kr, R ki, R mikr, R miki, R c4r,
    R c4i, bool wantS, bool wantC, Rules rl, Sink<R> out, unsigned long long* cnt) {
  using TRI = typename TriOf<R>::T;
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bi > bj) return;
  const int64_t i1 = (int64_t)bi * 16 + threadIdx.y;
  const int64_t i2 = (int64_t)bj * 16 + threadIdx.x;
  if (i1 >= ntr || i2 >= ntr || i1 >= i2) return;
  const int64_t t1 = t0 + i1, t2 = t0 + i2;
  const TRI A = tri[t1];
  const TRI B = tri[t2];
  if (touching(A, B)) return;
  const V3<R> D = centroid_delta(A, B);
  Mom<R> m;
  const int ev = pair_moments<R, NREG>(A, B, rl, D, kr, ki, wantC, m);
  count_add(cnt, (unsigned)ev);
  R pc[36];
  pair_coeffs(m, D, pc);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int ea = slot_edge[3 * t1 + a];
    const R sa = slot_sw[12 * t1 + 4 * a];
    const V3<R> wa = {slot_sw[12 * t1 + 4 * a + 1], slot_sw[12 * t1 + 4 * a + 2], slot_sw[12 * t1 + 4 * a + 3]};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int eb = slot_edge[3 * t2 + b];
      const R sb = slot_sw[12 * t2 + 4 * b];
      const V3<R> wb = {slot_sw[12 * t2 + 4 * b + 1], slot_sw[12 * t2 + 4 * b + 2], slot_sw[12 * t2 + 4 * b + 3]};
      R Sr = 0, Si = 0, Cr = 0, Ci = 0;
      entry_from_pc(pc, sa, wa, sb, wb, mikr, miki, c4r, c4i, wantS, wantC, Sr, Si, Cr, Ci);
      out.add(ea, eb, wantS, wantC, Sr, Si, Cr, Ci);
      out.add(eb, ea, wantS, wantC, Sr, Si, Cr, Ci);
    }
  }
}

// ---------------------------------------------------------------------------
// A8: matrix-free application of the regular part of a PMCHWT block. Every
// non-touching pair t1 < t2 forms its 3 x 3 local S and C entries exactly as
// the stored assembly does and applies them at once,
//   y1 += C x1 + alpha S x2,  y2 += C x2 + beta S x1,
// at the rows of t1 and, mirrored (both operators are symmetric), at the rows
// of t2. A 16 x 16 tile of pairs is reduced with warp shuffles and shared
// memory and added to y with one atomic per (triangle, slot, half, rhs).
// Touching pairs are left to the stored sparse singular block.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_c(const float2* p, float& re, float& im) { const float2 v = *p; re = v.x; im = v.y; }
__device__ __forceinline__ void load_c(const float2* p, double& re, double& im) { const float2 v = *p; re = v.x; im = v.y; }
__device__ __forceinline__ void load_c(const double2* p, float& re, float& im) { const double2 v = *p; re = (float)v.x; im = (float)v.y; }
__device__ __forceinline__ void load_c(const double2* p, double& re, double& im) { const double2 v = *p; re = v.x; im = v.y; }
__device__ __forceinline__ void atomic_add_v(float2* p, float re, float im) { atomicAdd(p, make_float2(re, im)); }
__device__ __forceinline__ void atomic_add_v(double2* p, float re, float im) {
  atomicAdd(&p->x, (double)re);
  atomicAdd(&p->y, (double)im);
}
__device__ __forceinline__ void atomic_add_v(double2* p, double re, double im) {
  atomicAdd(&p->x, re);
  atomicAdd(&p->y, im);
}

// AT: arithmetic of the application (float64 for float64 vectors, so that a
// refinement residual gets exact products of the float32 entries)
template <typename R, int NREG, typename VT, typename AT>
__global__ void __launch_bounds__(256) rwg_free_kernel(
    const typename TriOf<R>::T* __restrict__ tri, const int* __restrict__ slot_edge,
    const R* __restrict__ slot_sw, int64_t t0, int64_t ntr, R kr, R ki, R mikr, R miki, R c4r, R c4i,
    Rules rl, const VT* __restrict__ x, VT* __restrict__ y, int64_t n, int nrhs, AT ar, AT ai, AT br, AT bi,
    unsigned long long* cnt) {
  using TRI = typename TriOf<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // acc[((((side * 16 + t) * 3 + slot) * 2 + half) * nrhs + rhs) * 2 + (re, im)]
  AT* acc = reinterpret_cast<AT*>(smem_raw);
  const int tbi = blockIdx.y, tbj = blockIdx.x;
  if (tbi > tbj) return;  // the whole block: the tile lies below the diagonal
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 16 + tx;
  const int nacc = 2 * 16 * 3 * 2 * nrhs * 2;
  for (int q = tid; q < nacc; q += 256) acc[q] = AT(0);
  __syncthreads();
  const int64_t i1 = (int64_t)tbi * 16 + ty, i2 = (int64_t)tbj * 16 + tx;
  bool active = i1 < ntr && i2 < ntr && i1 < i2;
  const int64_t t1 = t0 + (active ? i1 : 0), t2 = t0 + (active ? i2 : 0);
  AT Sr[9], Si[9], Cr[9], Ci[9];
  int ea[3], eb[3];
#pragma unroll
  for (int q = 0; q < 9; ++q) Sr[q] = Si[q] = Cr[q] = Ci[q] = AT(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) ea[a] = eb[a] = 0;
  if (active) {
    const TRI A = tri[t1];
    const TRI B = tri[t2];
    active = !touching(A, B);
    if (active) {
      const V3<R> D = centroid_delta(A, B);
      Mom<R> m;
      const int ev = pair_moments<R, NREG>(A, B, rl, D, kr, ki, true, m);
      count_add(cnt, (unsigned)(ev * nrhs));
      R pc[36];
      pair_coeffs(m, D, pc);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        ea[a] = slot_edge[3 * t1 + a];
        eb[a] = slot_edge[3 * t2 + a];
        const R sa = slot_sw[12 * t1 + 4 * a];
        const V3<R> wa = {slot_sw[12 * t1 + 4 * a + 1], slot_sw[12 * t1 + 4 * a + 2], slot_sw[12 * t1 + 4 * a + 3]};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const R sb = slot_sw[12 * t2 + 4 * b];
          const V3<R> wb = {slot_sw[12 * t2 + 4 * b + 1], slot_sw[12 * t2 + 4 * b + 2],
                            slot_sw[12 * t2 + 4 * b + 3]};
          R er = 0, ei = 0, fr = 0, fi = 0;
          entry_from_pc(pc, sa, wa, sb, wb, mikr, miki, c4r, c4i, true, true, er, ei, fr, fi);
          Sr[3 * a + b] = er; Si[3 * a + b] = ei; Cr[3 * a + b] = fr; Ci[3 * a + b] = fi;
        }
      }
    }
  }
  for (int r = 0; r < nrhs; ++r) {
    const VT* x1 = x + (int64_t)r * 2 * n;
    const VT* x2 = x1 + n;
    AT u1r[3], u1i[3], u2r[3], u2i[3], v1r[3], v1i[3], v2r[3], v2i[3];  // x at t1 (u) and t2 (v)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      u1r[a] = u1i[a] = u2r[a] = u2i[a] = v1r[a] = v1i[a] = v2r[a] = v2i[a] = AT(0);
      if (active) {
        load_c(x1 + ea[a], u1r[a], u1i[a]);
        load_c(x2 + ea[a], u2r[a], u2i[a]);
        load_c(x1 + eb[a], v1r[a], v1i[a]);
        load_c(x2 + eb[a], v2r[a], v2i[a]);
      }
    }
    // row side (t1): 3 slots x 2 halves, complex; col side (t2) the same
    AT row[12], col[12];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      AT c1r = 0, c1i = 0, c2r = 0, c2i = 0, s1r = 0, s1i = 0, s2r = 0, s2i = 0;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int k = 3 * a + b;
        c1r += Cr[k] * v1r[b] - Ci[k] * v1i[b]; c1i += Cr[k] * v1i[b] + Ci[k] * v1r[b];
        c2r += Cr[k] * v2r[b] - Ci[k] * v2i[b]; c2i += Cr[k] * v2i[b] + Ci[k] * v2r[b];
        s2r += Sr[k] * v2r[b] - Si[k] * v2i[b]; s2i += Sr[k] * v2i[b] + Si[k] * v2r[b];
        s1r += Sr[k] * v1r[b] - Si[k] * v1i[b]; s1i += Sr[k] * v1i[b] + Si[k] * v1r[b];
      }
      row[4 * a + 0] = c1r + ar * s2r - ai * s2i;
      row[4 * a + 1] = c1i + ar * s2i + ai * s2r;
      row[4 * a + 2] = c2r + br * s1r - bi * s1i;
      row[4 * a + 3] = c2i + br * s1i + bi * s1r;
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      AT c1r = 0, c1i = 0, c2r = 0, c2i = 0, s1r = 0, s1i = 0, s2r = 0, s2i = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int k = 3 * a + b;
        c1r += Cr[k] * u1r[a] - Ci[k] * u1i[a]; c1i += Cr[k] * u1i[a] + Ci[k] * u1r[a];
        c2r += Cr[k] * u2r[a] - Ci[k] * u2i[a]; c2i += Cr[k] * u2i[a] + Ci[k] * u2r[a];
        s2r += Sr[k] * u2r[a] - Si[k] * u2i[a]; s2i += Sr[k] * u2i[a] + Si[k] * u2r[a];
        s1r += Sr[k] * u1r[a] - Si[k] * u1i[a]; s1i += Sr[k] * u1i[a] + Si[k] * u1r[a];
      }
      col[4 * b + 0] = c1r + ar * s2r - ai * s2i;
      col[4 * b + 1] = c1i + ar * s2i + ai * s2r;
      col[4 * b + 2] = c2r + br * s1r - bi * s1i;
      col[4 * b + 3] = c2i + br * s1i + bi * s1r;
    }
    // rows share t1 across the 16 lanes of a half warp; columns share t2
    // across the two half warps
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      AT v = row[q];
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      row[q] = v;
      col[q] += __shfl_xor_sync(0xffffffffu, col[q], 16);
    }
    if (tx == 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          AT* o = acc + ((((0 * 16 + ty) * 3 + a) * 2 + h) * nrhs + r) * 2;
          o[0] += row[4 * a + 2 * h];
          o[1] += row[4 * a + 2 * h + 1];
        }
    }
    if ((ty & 1) == 0) {
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          AT* o = acc + ((((1 * 16 + tx) * 3 + b) * 2 + h) * nrhs + r) * 2;
          atomicAdd(o, col[4 * b + 2 * h]);
          atomicAdd(o + 1, col[4 * b + 2 * h + 1]);
        }
    }
  }
  __syncthreads();
  // flush: one atomic per (side, triangle, slot, half, rhs)
  for (int q = tid; q < nacc / 2; q += 256) {
    const int r = q % nrhs;
    int rest = q / nrhs;
    const int h = rest % 2;
    rest /= 2;
    const int slot = rest % 3;
    rest /= 3;
    const int t = rest % 16, side = rest / 16;
    const int64_t tt = (int64_t)(side == 0 ? tbi : tbj) * 16 + t;
    if (tt >= ntr) continue;
    const AT vr = acc[2 * q], vi = acc[2 * q + 1];
    if (vr == AT(0) && vi == AT(0)) continue;
    const int e = slot_edge[3 * (t0 + tt) + slot];
    if (e < 0) continue;
    atomic_add_v(y + (int64_t)r * 2 * n + (int64_t)h * n + e, vr, vi);
  }
}

// ---------------------------------------------------------------------------
// A5: BC assembly by dual-cell tiles (v, w), v <= w. A block takes a "unit":
// one test cell v and up to 16 trial cells w (a run of the tile list); v's
// quadrature points, centroids, vertex ids and slot coefficients are staged
// in shared memory once per unit, w's once per tile. Per tile, stage 1 forms
// the pair coefficients of every (tau1 in D(v), tau2 in D(w)) in shared
// memory (pair-major, 36 reals, vector stores); stage 2 contracts the trial
// side per (tau1, trial slot) and stage 3 the test side per (test slot, trial
// slot), S and C as separate work items; the result is added to the output
// and to the mirrored entry when v != w.
// ---------------------------------------------------------------------------
struct BcUnit {
  int v;      // test cell (vertex id)
  int begin;  // first trial cell in the w list
  int count;  // trial cells
  int flag;   // -1: classify each pair; >= 0 (class rules, bc_owner_kernel):
              // every pair is far, and bit j drops trial cell j
};

template <typename R> struct Vec4Of;
template <> struct Vec4Of<float> { using T = float4; static constexpr int N = 4; };
template <> struct Vec4Of<double> { using T = double2; static constexpr int N = 2; };

// copy n reals (n a multiple of 4, both pointers 16-byte aligned) with vector moves
template <typename R>
__device__ __forceinline__ void vcopy(R* __restrict__ dst, const R* __restrict__ src, int n) {
  using V = typename Vec4Of<R>::T;
  constexpr int K = Vec4Of<R>::N;
  const V* s = reinterpret_cast<const V*>(src);
  V* d = reinterpret_cast<V*>(dst);
  for (int q = 0; q < n / K; ++q) d[q] = s[q];
}

constexpr int BC_RED = 20;  // stage-2 record: S part [0, 12), C part [12, 20)

// Per-launch copies of what a tile stages, in cell order (cell_tri order), so
// that staging a cell is a few contiguous, coalesced copies.
template <typename R>
struct CellData {
  P4<R>* pts;    // [ncelltri][NREG] quadrature points relative to the centroid, with weights
  P4<R>* sw;     // [ncelltri][nslot] slot coefficients (sigma, w)
  Cent<R>* cen;  // [ncelltri]
  int* vid;      // [ncelltri][3]
};

// staged points per triangle: the rule's, or all three class rules (13)
template <int NREG> __host__ __device__ constexpr int staged_points() { return NREG > 0 ? NREG : RULE_POINTS_ALL; }

template <typename R, int NREG>
__global__ void bc_cell_prep_kernel(const typename TriOf<R>::T* __restrict__ tri, const R* __restrict__ slot_sw,
                                    int nslot, const int* __restrict__ cell_tri, int64_t ncelltri, Rules rl,
                                    CellData<R> cd) {
  constexpr int NS = staged_points<NREG>();
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ncelltri * NS) return;
  const int64_t t = q / NS;
  const int u = (int)(q % NS);
  const int tau = cell_tri[t];
  const typename TriOf<R>::T T = tri[tau];
  cd.pts[q] = staged_point(T, rl, u);
  if (u == 0) {
    cd.cen[t].set(T);
    cd.vid[3 * t] = T.vid[0];
    cd.vid[3 * t + 1] = T.vid[1];
    cd.vid[3 * t + 2] = T.vid[2];
    const P4<R>* src = reinterpret_cast<const P4<R>*>(slot_sw) + (size_t)tau * nslot;
    for (int sl = 0; sl < nslot; ++sl) cd.sw[t * nslot + sl] = src[sl];
  }
}

template <typename R, int NREG, int TT>
__global__ void __launch_bounds__(TT, sizeof(R) == 4 ? 4 : 2) bc_tile_kernel(
    CellData<R> cd, int nslot, const int* __restrict__ cell_ptr, const int* __restrict__ cell_edge_ptr,
    const int* __restrict__ cell_edge, const BcUnit* __restrict__ units, int64_t nunits,
    const int* __restrict__ wlist, R kr, R ki, R mikr, R miki, R c4r, R c4i, bool wantS, bool wantC,
    Sink<R> out, int max_cell, int chunk, unsigned long long* cnt) {
  constexpr int NS = staged_points<NREG>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* pcs = reinterpret_cast<R*>(smem_raw);                        // [chunk * max_cell][36]
  R* red = pcs + (size_t)chunk * max_cell * 36;                   // [chunk][nslot][BC_RED]
  R* acc = red + (size_t)chunk * nslot * BC_RED;                  // [nslot][nslot][4]
  const size_t staged_off =
      ((((size_t)chunk * max_cell * 36 + (size_t)chunk * nslot * BC_RED + (size_t)nslot * nslot * 4) *
            sizeof(R) + 15) / 16) * 16;
  P4<R>* ptsA = reinterpret_cast<P4<R>*>(smem_raw + staged_off);  // [max_cell][NS]
  P4<R>* ptsB = ptsA + (size_t)max_cell * NS;
  P4<R>* swA = ptsB + (size_t)max_cell * NS;                      // [max_cell][nslot] (s, w)
  P4<R>* swB = swA + (size_t)max_cell * nslot;
  Cent<R>* cA = reinterpret_cast<Cent<R>*>(swB + (size_t)max_cell * nslot);
  Cent<R>* cB = cA + max_cell;
  int* vidA = reinterpret_cast<int*>(cB + max_cell);              // [max_cell][3]
  int* vidB = vidA + 3 * max_cell;
  // stage one cell's quadrature points, centroids, vertex ids and slot
  // coefficients: contiguous copies of the cell-ordered arrays
  auto stage_cell = [&](int cell, P4<R>* pts, Cent<R>* cen, int* vid, P4<R>* swc) {
    const int b0 = cell_ptr[cell], n = cell_ptr[cell + 1] - b0;
    const P4<R>* sp = cd.pts + (size_t)b0 * NS;
    const P4<R>* ss = cd.sw + (size_t)b0 * nslot;
    for (int q = threadIdx.x; q < n * NS; q += TT) pts[q] = sp[q];
    for (int q = threadIdx.x; q < n * nslot; q += TT) swc[q] = ss[q];
    const int* sc = reinterpret_cast<const int*>(cd.cen + b0);
    int* dc = reinterpret_cast<int*>(cen);
    constexpr int CW = (int)(sizeof(Cent<R>) / sizeof(int));
    for (int q = threadIdx.x; q < n * CW; q += TT) dc[q] = sc[q];
    for (int q = threadIdx.x; q < n * 3; q += TT) vid[q] = cd.vid[(size_t)b0 * 3 + q];
  };
  // the slots of every triangle of a cell are the cell's edges, in one order
  auto nvalid = [&](int cell) { return cell_edge_ptr[cell + 1] - cell_edge_ptr[cell]; };
  unsigned evals = 0;  // integrand evaluations of this thread (profiling count)
  for (int64_t uidx = blockIdx.x; uidx < nunits; uidx += gridDim.x) {
    const BcUnit U = units[uidx];
    const int v = U.v;
    const int b1 = cell_ptr[v], n1 = cell_ptr[v + 1] - b1;
    const int ns1 = nvalid(v);
    __syncthreads();  // the previous unit is done with the A side
    stage_cell(v, ptsA, cA, vidA, swA);
    for (int wi = 0; wi < U.count; ++wi) {
      const int w = wlist[U.begin + wi];
      const int b2 = cell_ptr[w], n2 = cell_ptr[w + 1] - b2;
      const int ns2 = nvalid(w);
      __syncthreads();  // the previous tile is done with the B side and acc
      stage_cell(w, ptsB, cB, vidB, swB);
      for (int q = threadIdx.x; q < ns1 * ns2 * 4; q += TT) acc[q] = R(0);
      __syncthreads();
      for (int c0 = 0; c0 < n1; c0 += chunk) {
        const int nc = min(chunk, n1 - c0);
        // stage 1: pair coefficients of (tau1 in the chunk) x (tau2 in D(w))
        for (int p = threadIdx.x; p < nc * n2; p += TT) {
          const int i1 = c0 + p / n2, i2 = p % n2;
          const int* va = vidA + 3 * i1;
          const int* vb = vidB + 3 * i2;
          bool touch = false;
#pragma unroll
          for (int x = 0; x < 3; ++x)
#pragma unroll
            for (int y = 0; y < 3; ++y) touch |= va[x] == vb[y];
          __align__(16) R tmp[36];
          if (touch) {
#pragma unroll
            for (int q = 0; q < 36; ++q) tmp[q] = R(0);
          } else {
            const V3<R> D = cA[i1].minus(cB[i2]);
            Mom<R> m;
            const P4<R>* X = ptsA + i1 * NS;
            const P4<R>* Y = ptsB + i2 * NS;
            if constexpr (NREG > 0) {
              regular_moments_staged<R, NREG>(X, Y, D, kr, ki, wantC, m);
              evals += NREG * NREG;
            } else {
              const int c = pair_class<R>(D, cA[i1].d, cB[i2].d);
              if (c == 2) {
                regular_moments_staged<R, 3>(X + RULE_OFF_FAR, Y + RULE_OFF_FAR, D, kr, ki, wantC, m);
                evals += 9;
              } else if (c == 1) {
                regular_moments_staged<R, 4>(X + RULE_OFF_MEDIUM, Y + RULE_OFF_MEDIUM, D, kr, ki, wantC, m);
                evals += 16;
              } else {
                regular_moments_staged<R, 6>(X, Y, D, kr, ki, wantC, m);
                evals += 36;
              }
            }
            pair_coeffs(m, D, tmp);
          }
          vcopy(pcs + (size_t)p * 36, tmp, 36);
        }
        __syncthreads();
        // stage 2: per (tau1, trial slot b), sum over tau2 of the trial-side factors
        const int nS2 = wantS ? nc * ns2 : 0, nC2 = wantC ? nc * ns2 : 0;
        for (int q = threadIdx.x; q < nS2 + nC2; q += TT) {
          const bool isS = q < nS2;
          const int it = isS ? q : q - nS2;
          const int i1 = it / ns2, sb_i = it % ns2;
          R* o = red + (size_t)(i1 * nslot + sb_i) * BC_RED;
          if (isS) {
            R AS_r = 0, AS_i = 0, BS_r = 0, BS_i = 0;
            V3<R> WS_r = {0, 0, 0}, WS_i = {0, 0, 0};
#pragma unroll 4
            for (int i2 = 0; i2 < n2; ++i2) {
              const P4<R> u = swB[i2 * nslot + sb_i];
              const R sb = u.x;
              const V3<R> wb = {u.y, u.z, u.w};
              __align__(16) R pc[16];
              vcopy(pc, pcs + (size_t)(i1 * n2 + i2) * 36, 16);
              AS_r += sb * pc[14] + wb.x * pc[2] + wb.y * pc[3] + wb.z * pc[4];
              AS_i += sb * pc[15] + wb.x * pc[5] + wb.y * pc[6] + wb.z * pc[7];
              BS_r += sb * pc[0];
              BS_i += sb * pc[1];
              WS_r.x += sb * pc[8] + wb.x * pc[0]; WS_r.y += sb * pc[9] + wb.y * pc[0]; WS_r.z += sb * pc[10] + wb.z * pc[0];
              WS_i.x += sb * pc[11] + wb.x * pc[1]; WS_i.y += sb * pc[12] + wb.y * pc[1]; WS_i.z += sb * pc[13] + wb.z * pc[1];
            }
            __align__(16) R rec[12] = {AS_r, AS_i, BS_r, BS_i, WS_r.x, WS_r.y, WS_r.z, WS_i.x, WS_i.y, WS_i.z, R(0), R(0)};
            vcopy(o, rec, 12);
          } else {
            R AC_r = 0, AC_i = 0;
            V3<R> WC_r = {0, 0, 0}, WC_i = {0, 0, 0};
#pragma unroll 4
            for (int i2 = 0; i2 < n2; ++i2) {
              const P4<R> u = swB[i2 * nslot + sb_i];
              const R sb = u.x;
              const V3<R> wb = {u.y, u.z, u.w};
              __align__(16) R pc[20];
              vcopy(pc, pcs + (size_t)(i1 * n2 + i2) * 36 + 16, 20);  // components 16..35
              AC_r += sb * pc[0] + wb.x * pc[2] + wb.y * pc[3] + wb.z * pc[4];
              AC_i += sb * pc[1] + wb.x * pc[5] + wb.y * pc[6] + wb.z * pc[7];
              const V3<R> Vr = {pc[14], pc[15], pc[16]}, Vi = {pc[17], pc[18], pc[19]};
              const V3<R> cr = cross3(wb, Vr), ci = cross3(wb, Vi);
              WC_r.x += sb * pc[8] + cr.x; WC_r.y += sb * pc[9] + cr.y; WC_r.z += sb * pc[10] + cr.z;
              WC_i.x += sb * pc[11] + ci.x; WC_i.y += sb * pc[12] + ci.y; WC_i.z += sb * pc[13] + ci.z;
            }
            __align__(16) R rec[8] = {AC_r, AC_i, WC_r.x, WC_r.y, WC_r.z, WC_i.x, WC_i.y, WC_i.z};
            vcopy(o + 12, rec, 8);
          }
        }
        __syncthreads();
        // stage 3: per (test slot a, trial slot b), sum over the chunk's tau1
        const int nS3 = wantS ? ns1 * ns2 : 0, nC3 = wantC ? ns1 * ns2 : 0;
        for (int q = threadIdx.x; q < nS3 + nC3; q += TT) {
          const bool isS = q < nS3;
          const int it = isS ? q : q - nS3;
          const int sa_i = it / ns2, sb_i = it % ns2;
          R vr = 0, vi = 0;
#pragma unroll 4
          for (int i1 = 0; i1 < nc; ++i1) {
            const P4<R> u = swA[(c0 + i1) * nslot + sa_i];
            const R sa = u.x;
            const V3<R> wa = {u.y, u.z, u.w};
            const R* orec = red + (size_t)(i1 * nslot + sb_i) * BC_RED;
            if (isS) {
              __align__(16) R o[12];
              vcopy(o, orec, 12);
              // sa (mik AS + c4 BS) + mik (wa . WS)
              const R pr = sa * o[0] + wa.x * o[4] + wa.y * o[5] + wa.z * o[6];
              const R pi = sa * o[1] + wa.x * o[7] + wa.y * o[8] + wa.z * o[9];
              vr += mikr * pr - miki * pi + sa * (c4r * o[2] - c4i * o[3]);
              vi += mikr * pi + miki * pr + sa * (c4r * o[3] + c4i * o[2]);
            } else {
              __align__(16) R o[8];
              vcopy(o, orec + 12, 8);
              vr += sa * o[0] + wa.x * o[2] + wa.y * o[3] + wa.z * o[4];
              vi += sa * o[1] + wa.x * o[5] + wa.y * o[6] + wa.z * o[7];
            }
          }
          R* a4 = acc + (size_t)it * 4 + (isS ? 0 : 2);
          a4[0] += vr;
          a4[1] += vi;
        }
        __syncthreads();
      }
      for (int q = threadIdx.x; q < ns1 * ns2; q += TT) {
        const int sa_i = q / ns2, sb_i = q % ns2;
        const R* a4 = acc + (size_t)q * 4;
        const int ea = cell_edge[cell_edge_ptr[v] + sa_i];
        const int eb = cell_edge[cell_edge_ptr[w] + sb_i];
        out.add(ea, eb, wantS, wantC, a4[0], a4[1], a4[2], a4[3]);
        if (v != w) out.add(eb, ea, wantS, wantC, a4[0], a4[1], a4[2], a4[3]);
      }
    }
  }
  count_add(cnt, evals);
}

// ---------------------------------------------------------------------------
// A5, float32, cells of at most BC_OWN_SLOTS edges: one thread per (test
// triangle tau1 of v, trial cell w_j) of a unit. The thread walks the
// triangles tau2 of w_j, forms each pair's moments and pair coefficients and
// contracts them with w_j's trial slots at once into register sums (the
// stage-2 records of bc_tile_kernel), so pair coefficients never go through
// shared memory and the pair loop has no barrier. The divergence parts of the
// slots factor as s_b / |tau2| over a cell, so their terms are one sum per
// thread rather than one per slot. The records are then written
// to shared memory once and contracted with the test slots per (j, a, b).
// Units hold up to floor(TT / n1) trial cells so that the items fill the
// block. The trial triangles of a unit are staged in shared memory first, as
// packed records (owner_rec_words float4 each), so the pair loop reads no
// global memory except the points of the rare near and medium pairs.
// ---------------------------------------------------------------------------
constexpr int BC_OWN_SLOTS = 6;
constexpr int BC_OWN_REC = 20;    // S record [0, 10), C record [10, 18), padding
constexpr int BC_OWN_STAGE = 160;  // staged trial triangle rows per unit (count x max_cell)

// packed trial record, in float4 words: the trial rule points (the far rule's
// 3 in class mode) with their weights over 4 pi, BC_OWN_SLOTS slot quadruples (zero past nslot), then
// (hi.x, hi.y, hi.z, lo.x), (lo.y, lo.z, d, vid0), (vid1, vid2, 1/|tau|, 0) with the
// vertex ids stored as int bits
template <int NREG> __host__ __device__ constexpr int owner_trial_pts() { return NREG > 0 ? NREG : 3; }
template <int NREG> __host__ __device__ constexpr int owner_rec_words() {
  return owner_trial_pts<NREG>() + BC_OWN_SLOTS + 3;
}

template <int NREG>
__global__ void bc_trial_pack_kernel(CellData<float> cd, int nslot, int64_t nct, const TriF* __restrict__ tri,
                                     const int* __restrict__ cell_tri, float4* __restrict__ rec) {
  constexpr int NP = owner_trial_pts<NREG>(), RW = owner_rec_words<NREG>(), NS = staged_points<NREG>();
  constexpr int OFF = NREG > 0 ? 0 : RULE_OFF_FAR;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nct * RW) return;
  const int64_t t = q / RW;
  const int u = (int)(q - t * RW);
  float4 o = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (u < NP) {
    const P4<float> p = cd.pts[t * NS + OFF + u];
    o = make_float4(p.x, p.y, p.z, p.w * INV_4PI_F);
  } else if (u < NP + BC_OWN_SLOTS) {
    const int sl = u - NP;
    if (sl < nslot) {
      const P4<float> p = cd.sw[t * nslot + sl];
      o = make_float4(p.x, p.y, p.z, p.w);
    }
  } else {
    const Cent<float>& c = cd.cen[t];
    const int* v = cd.vid + 3 * t;
    const int k = u - NP - BC_OWN_SLOTS;
    if (k == 0) o = make_float4(c.hi[0], c.hi[1], c.hi[2], c.lo[0]);
    else if (k == 1) o = make_float4(c.lo[1], c.lo[2], c.d, __int_as_float(v[0]));
    else o = make_float4(__int_as_float(v[1]), __int_as_float(v[2]), 1.0f / tri[cell_tri[t]].area, 0.0f);
  }
  rec[q] = o;
}

// Packed float32 pairs: one FFMA2 / FADD2 / FMUL2 does two round-to-nearest
// float32 operations, here the real and imaginary parts of one complex
// quantity (or of its three components), so the owner kernel's arithmetic is
// that of plain float32 at about half the issued instructions.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// moments of one regular pair, each complex value a (re, im) pair: S needs
// int G, int G x, int G y and int G x.y; C the same of the gradient factor g,
// with int g x cross y in place of the dot product (x, y relative to the
// centroids)
struct Mom2 {
  float2 G0, Gx[3], Gy[3], Gxy;
  float2 g0, gx[3], gy[3], gxy[3];
};

// Moments of one regular pair for the owner kernel: test points X = (x, y, z,
// w) with XW = (w x, w y, w z, w); trial points Y with weights over 4 pi when
// PRE (the packed records), plain weights otherwise.
template <int NP, bool PRE, bool FULL>
__device__ __forceinline__ void owner_moments(const P4<float>* __restrict__ X, const P4<float>* __restrict__ XW,
                                              const P4<float>* __restrict__ Y, const V3<float>& D, float kr,
                                              float ki, bool wantC, Mom2& m) {
  const float2 z0 = make_float2(0.f, 0.f);
  m.G0 = m.Gxy = m.g0 = z0;
#pragma unroll
  for (int c = 0; c < 3; ++c) m.Gx[c] = m.Gy[c] = m.gx[c] = m.gy[c] = m.gxy[c] = z0;
  // FULL (S and C fixed at compile time): all test points unrolled; otherwise
  // two at a time
#pragma unroll(FULL ? NP : 2)
  for (int p = 0; p < NP; ++p) {
    const P4<float> xp = X[p], xw = XW[p];
    float2 s0 = z0, t0 = z0, se[3] = {z0, z0, z0}, te[3] = {z0, z0, z0};
    const V3<float> dp = {D.x + xp.x, D.y + xp.y, D.z + xp.z};
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const P4<float> yq = Y[q];
      const float dx = dp.x - yq.x, dy = dp.y - yq.y, dz = dp.z - yq.z;
      float Gr, Gi, gr, gi;
      green4(dx * dx + dy * dy + dz * dz, kr, ki, Gr, Gi, gr, gi, PRE ? yq.w : yq.w * INV_4PI_F);
      const float2 G = make_float2(Gr, Gi);
      s0 = add2(s0, G);
      se[0] = fma2(G, dup2(yq.x), se[0]);
      se[1] = fma2(G, dup2(yq.y), se[1]);
      se[2] = fma2(G, dup2(yq.z), se[2]);
      if (wantC) {
        const float2 g = make_float2(gr, gi);
        t0 = add2(t0, g);
        te[0] = fma2(g, dup2(yq.x), te[0]);
        te[1] = fma2(g, dup2(yq.y), te[1]);
        te[2] = fma2(g, dup2(yq.z), te[2]);
      }
    }
    const float2 w2 = dup2(xw.w), x2 = dup2(xw.x), y2 = dup2(xw.y), z2 = dup2(xw.z);
    m.G0 = fma2(w2, s0, m.G0);
    m.Gx[0] = fma2(x2, s0, m.Gx[0]);
    m.Gx[1] = fma2(y2, s0, m.Gx[1]);
    m.Gx[2] = fma2(z2, s0, m.Gx[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) m.Gy[c] = fma2(w2, se[c], m.Gy[c]);
    m.Gxy = fma2(z2, se[2], fma2(y2, se[1], fma2(x2, se[0], m.Gxy)));
    if (wantC) {
      m.g0 = fma2(w2, t0, m.g0);
      m.gx[0] = fma2(x2, t0, m.gx[0]);
      m.gx[1] = fma2(y2, t0, m.gx[1]);
      m.gx[2] = fma2(z2, t0, m.gx[2]);
#pragma unroll
      for (int c = 0; c < 3; ++c) m.gy[c] = fma2(w2, te[c], m.gy[c]);
      // gxy += (w x) cross te
      m.gxy[0] = fma2(y2, te[2], fma2(dup2(-xw.z), te[1], m.gxy[0]));
      m.gxy[1] = fma2(z2, te[0], fma2(dup2(-xw.x), te[2], m.gxy[1]));
      m.gxy[2] = fma2(x2, te[1], fma2(dup2(-xw.y), te[0], m.gxy[2]));
    }
  }
}

// the C pair coefficients from the moments (D = c1 - c2): D . gxy; X1 = D x gx
// + gxy; Y2 = gxy - gy x D (the coefficient gy x D - gxy with its sign
// flipped); V = D g0 + gx - gy and nV = -V
struct PairC2 {
  float2 Dgxy, X1[3], Y2[3], V[3], nV[3];
};

__device__ __forceinline__ void pair_c_coeffs(const Mom2& m, const V3<float>& D, PairC2& pc) {
  const float2 dx = dup2(D.x), dy = dup2(D.y), dz = dup2(D.z);
  const float2 ndx = dup2(-D.x), ndy = dup2(-D.y), ndz = dup2(-D.z), mone = dup2(-1.f);
  pc.Dgxy = fma2(dz, m.gxy[2], fma2(dy, m.gxy[1], mul2(dx, m.gxy[0])));
  pc.X1[0] = fma2(dy, m.gx[2], fma2(ndz, m.gx[1], m.gxy[0]));
  pc.X1[1] = fma2(dz, m.gx[0], fma2(ndx, m.gx[2], m.gxy[1]));
  pc.X1[2] = fma2(dx, m.gx[1], fma2(ndy, m.gx[0], m.gxy[2]));
  pc.Y2[0] = fma2(m.gy[2], dy, fma2(m.gy[1], ndz, m.gxy[0]));
  pc.Y2[1] = fma2(m.gy[0], dz, fma2(m.gy[2], ndx, m.gxy[1]));
  pc.Y2[2] = fma2(m.gy[1], dx, fma2(m.gy[0], ndy, m.gxy[2]));
  pc.V[0] = fma2(dx, m.g0, fma2(mone, m.gy[0], m.gx[0]));
  pc.V[1] = fma2(dy, m.g0, fma2(mone, m.gy[1], m.gx[1]));
  pc.V[2] = fma2(dz, m.g0, fma2(mone, m.gy[2], m.gx[2]));
  pc.nV[0] = fma2(ndx, m.g0, fma2(mone, m.gx[0], m.gy[0]));
  pc.nV[1] = fma2(ndy, m.g0, fma2(mone, m.gx[1], m.gy[1]));
  pc.nV[2] = fma2(ndz, m.g0, fma2(mone, m.gx[2], m.gy[2]));
}

// asynchronous global -> shared copies (complete at cp.async.wait_all of the
// issuing thread; a barrier after that makes them visible to the block)
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Tensor memory as per-thread scratch rows (tcgen05): in a CTA of 128
// threads, warp w may reach TMEM lanes 32w .. 32w + 31, so thread t owns lane
// t; a load or store moves 16 or 32 consecutive 32-bit columns of that lane.
// These are warp-collective (.sync.aligned): every lane of the warp executes
// them together. tcgen05.ld results are valid after tm_wait_ld; a load of
// columns written by tcgen05.st sees them after tm_wait_st.
__device__ __forceinline__ uint32_t tm_lane_addr(uint32_t base) {
  return base + ((uint32_t)(threadIdx.x & ~31u) << 16);
}
__device__ __forceinline__ void tm_ld16(uint32_t ta, float* v) {
  uint32_t u[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
               : "r"(ta));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(u[i]);
}
__device__ __forceinline__ void tm_ld32(uint32_t ta, float* v) {
  uint32_t u[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]), "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
               : "r"(ta));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(u[i]);
}
__device__ __forceinline__ void tm_st16(uint32_t ta, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
               :: "r"(ta), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
               : "memory");
}
__device__ __forceinline__ void tm_st32(uint32_t ta, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
               :: "r"(ta), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])), "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])), "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])), "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])), "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])), "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
               : "memory");
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

constexpr int BC_OWN_TMEM_COLS = 128;  // tensor-memory columns per CTA (96 used: six slots x 16)

// bytes of the shared region that holds the staged trial records and test
// points, then the per-thread records (16-byte multiple)
__host__ __device__ inline size_t owner_region_bytes(int tt, int rw, int ns, int max_cell) {
  const size_t staging = (size_t)BC_OWN_STAGE * rw * 16 + 2 * (size_t)max_cell * ns * 16;
  const size_t records = (size_t)tt * BC_OWN_SLOTS * BC_OWN_REC * sizeof(float);
  return staging > records ? staging : records;
}

// the w_b terms of one pair for one trial slot, added to its 8 complex sums
// f[0..16): S: AS = w_b . Gx, WS = w_b G0; C: AC = w_b . X1, WC = w_b x V
__device__ __forceinline__ void owner_slot_update(float* f, float2 bx, float2 by, float2 bz, const Mom2& m,
                                                  const PairC2& pc) {
  float2 o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) o[k] = make_float2(f[2 * k], f[2 * k + 1]);
  o[0] = fma2(bz, m.Gx[2], fma2(by, m.Gx[1], fma2(bx, m.Gx[0], o[0])));
  o[1] = fma2(bx, m.G0, o[1]);
  o[2] = fma2(by, m.G0, o[2]);
  o[3] = fma2(bz, m.G0, o[3]);
  o[4] = fma2(bz, pc.X1[2], fma2(by, pc.X1[1], fma2(bx, pc.X1[0], o[4])));
  o[5] = fma2(by, pc.V[2], fma2(bz, pc.nV[1], o[5]));
  o[6] = fma2(bz, pc.V[0], fma2(bx, pc.nV[2], o[6]));
  o[7] = fma2(bx, pc.V[1], fma2(by, pc.nV[0], o[7]));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    f[2 * k] = o[k].x;
    f[2 * k + 1] = o[k].y;
  }
}

template <int NREG, int TT, bool BOTH>
__global__ void __launch_bounds__(TT, 3) bc_owner_kernel(
    CellData<float> cd, int nslot, const int* __restrict__ cell_ptr, const int* __restrict__ cell_edge_ptr,
    const int* __restrict__ cell_edge, const BcUnit* __restrict__ units, int64_t nunits,
    const int* __restrict__ wlist, const float4* __restrict__ trec, const float* __restrict__ cell_slot_s, float kr,
    float ki, float mikr, float miki, float c4r, float c4i, bool wantS, bool wantC, Sink<float> out, int max_cell,
    unsigned long long* cnt) {
  constexpr int NS = staged_points<NREG>();
  constexpr int NSL = BC_OWN_SLOTS;
  constexpr int NP = owner_trial_pts<NREG>(), RW = owner_rec_words<NREG>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // one region holds the staged trial records and test points during the pair
  // loop, and the per-thread records after it (a barrier in between)
  float4* trial = reinterpret_cast<float4*>(smem_raw);                             // [BC_OWN_STAGE][RW]
  P4<float>* ptsA = reinterpret_cast<P4<float>*>(trial + (size_t)BC_OWN_STAGE * RW);  // [max_cell][NS]
  P4<float>* ptsW = ptsA + (size_t)max_cell * NS;                                   // [max_cell][NS] w (x, y, z), w
  float* rec = reinterpret_cast<float*>(smem_raw);                                  // [TT][NSL][BC_OWN_REC]
  const size_t region = owner_region_bytes(TT, RW, NS, max_cell);
  P4<float>* swA = reinterpret_cast<P4<float>*>(smem_raw + region);                 // [max_cell][nslot]
  Cent<float>* cA = reinterpret_cast<Cent<float>*>(swA + (size_t)max_cell * nslot);
  int* vidA = reinterpret_cast<int*>(cA + max_cell);                                // [max_cell][3]
  int* jb = vidA + 3 * max_cell;                                                    // [TT] first trial triangle
  int* jn = jb + TT;                                                                // [TT] trial triangles
  int* jw = jn + TT;                                                                // [TT] trial cell
  float* js = reinterpret_cast<float*>(jw + TT);                                    // [TT][NSL] s_b of cell j
  int* jns = reinterpret_cast<int*>(js + TT * NSL);                                 // [TT] slots of cell j
  int* jeb = jns + TT;                                                              // [TT][NSL] edge of slot b
  int* eaS = jeb + TT * NSL;                                                        // [NSL] edge of test slot a
  int* wnext = eaS + NSL;                                                           // [TT] next unit's trial cells
  BcUnit* nextU = reinterpret_cast<BcUnit*>((reinterpret_cast<uintptr_t>(wnext + TT) + 15) & ~uintptr_t(15));
  uint32_t* tm_base = reinterpret_cast<uint32_t*>(nextU + 1);
  if (BOTH) wantS = wantC = true;  // S and C: the branches on them fold away
  unsigned evals = 0;
  // the trial-slot sums of each thread live in its tensor-memory lane (96 of
  // 128 columns), so that they hold no registers during the evaluations
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(tm_base)),
                 "r"(BC_OWN_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmr = tm_lane_addr(*tm_base);
  // The next unit's descriptor and trial-cell list are copied into shared
  // memory while the current unit computes (cp.async), so a unit starts two
  // dependent global loads closer to its data.
  if (threadIdx.x == 0 && (int64_t)blockIdx.x < nunits) cp_async16(nextU, units + blockIdx.x);
  cp_async_wait_all();
  __syncthreads();
  if ((int64_t)blockIdx.x < nunits && (int)threadIdx.x < nextU->count)
    cp_async4(wnext + threadIdx.x, wlist + nextU->begin + threadIdx.x);
  cp_async_wait_all();
  for (int64_t uidx = blockIdx.x; uidx < nunits; uidx += gridDim.x) {
    __syncthreads();  // the previous unit is done with every buffer; nextU and wnext have landed
    const BcUnit U = *nextU;
    const int v = U.v;
    // class rules: a unit whose pairs are all far (decided per cell pair on the
    // host, with a margin over this kernel's own test) skips the per-pair class
    // test, so its warps never split between rules; uniform over the block
    const bool all_far = NREG == 0 && U.flag >= 0;
    const int drop = U.flag > 0 ? U.flag : 0;
    const int b1 = cell_ptr[v], n1 = cell_ptr[v + 1] - b1;
    const int ea0 = cell_edge_ptr[v], ns1 = cell_edge_ptr[v + 1] - ea0;
    for (int q = threadIdx.x; q < ns1; q += TT) eaS[q] = cell_edge[ea0 + q];
    for (int q = threadIdx.x; q < n1 * NS; q += TT) {
      const P4<float> x = cd.pts[(size_t)b1 * NS + q];
      ptsA[q] = x;
      ptsW[q] = {x.w * x.x, x.w * x.y, x.w * x.z, x.w};
    }
    for (int q = threadIdx.x; q < n1 * nslot; q += TT) swA[q] = cd.sw[(size_t)b1 * nslot + q];
    for (int q = threadIdx.x; q < n1; q += TT) {
      cA[q] = cd.cen[b1 + q];
      for (int c = 0; c < 3; ++c) vidA[3 * q + c] = cd.vid[(size_t)(b1 + q) * 3 + c];
    }
    for (int j = threadIdx.x; j < U.count; j += TT) {
      const int w = wnext[j];
      const int b = cell_ptr[w];
      jw[j] = w;
      jb[j] = b;
      jn[j] = (drop >> j) & 1 ? 0 : cell_ptr[w + 1] - b;  // a dropped cell has no pairs here
      const int e0 = cell_edge_ptr[w], ns = cell_edge_ptr[w + 1] - e0;
      jns[j] = ns;
#pragma unroll
      for (int sl = 0; sl < NSL; ++sl) {
        js[j * NSL + sl] = sl < ns ? cell_slot_s[e0 + sl] : 0.0f;
        jeb[j * NSL + sl] = sl < ns ? cell_edge[e0 + sl] : -1;
      }
    }
    __syncthreads();
    // trial records: cell j at rows [j max_cell, j max_cell + n2); the host
    // keeps count x max_cell <= BC_OWN_STAGE
    // (asynchronous copies: all of a thread's rows are in flight at once)
    for (int q = threadIdx.x; q < U.count * max_cell * RW; q += TT) {
      const int row = q / RW, u = q - row * RW;
      const int j = row / max_cell, i2 = row - j * max_cell;
      if (i2 < jn[j]) cp_async16(trial + q, trec + (size_t)(jb[j] + i2) * RW + u);
    }
    cp_async_wait_all();
    __syncthreads();
    // every thread has read nextU and wnext: copy the next unit's descriptor
    const bool more = uidx + gridDim.x < nunits;
    if (threadIdx.x == 0 && more) cp_async16(nextU, units + uidx + gridDim.x);
    const int items = n1 * U.count;
    // pair loop: thread t = j n1 + i1. Every lane of a warp runs the warp's
    // largest trip count (the tensor-memory moves are warp-collective); a lane
    // past its own pairs, or a thread with no item, only takes part in them.
    const bool item = (int)threadIdx.x < items;
    const int j = item ? (int)threadIdx.x / n1 : 0, i1 = item ? (int)threadIdx.x - j * n1 : 0;
    const int b2 = jb[j], n2 = item ? jn[j] : 0;
    const int ns2 = jns[j];
    const float4* R2 = trial + (size_t)j * max_cell * RW;
    const Cent<float> ca = cA[i1];
    const int va0 = vidA[3 * i1], va1 = vidA[3 * i1 + 1], va2 = vidA[3 * i1 + 2];
    const P4<float>* X = ptsA + i1 * NS;
    const P4<float>* XW = ptsW + i1 * NS;
    // slot b on tau2 is sigma_b (y - c2) + w_b with sigma_b = s_b / |tau2| (s_b
    // constant over the cell): the sigma terms of all slots are one sum a[]
    // over tau2 of the pair coefficients times 1/|tau2|, scaled by s_b at the
    // end; the w_b terms of slot b are 8 complex sums in tensor-memory columns
    // 16 b .. 16 b + 15. Record layout, complex (re, im) pairs: S: AS, BS,
    // WS[3]; C: AC, WC[3] (BS has no w_b term).
    const float2 z0 = make_float2(0.f, 0.f);
    float2 a[9];
#pragma unroll
    for (int f = 0; f < 9; ++f) a[f] = z0;
    {
      float zz[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) zz[q] = 0.f;
      tm_wait_st();  // the previous unit's stores (read back below) are complete
      tm_st32(tmr, zz);
      tm_st32(tmr + 32, zz);
      tm_st32(tmr + 64, zz);
    }
    const int n2w = __reduce_max_sync(0xffffffffu, n2);
    for (int i2 = 0; i2 < n2w; ++i2) {
      bool act = i2 < n2;
      const float4* rr = R2 + i2 * RW;
      const P4<float>* Ys = reinterpret_cast<const P4<float>*>(rr);
      Mom2 m;
      PairC2 pc;
      if (act) {
        const float4 k0 = rr[NP + NSL], k1 = rr[NP + NSL + 1], k2 = rr[NP + NSL + 2];
        const int vb0 = __float_as_int(k1.w), vb1 = __float_as_int(k2.x), vb2 = __float_as_int(k2.y);
        Cent<float> cb;
        cb.hi[0] = k0.x; cb.hi[1] = k0.y; cb.hi[2] = k0.z;
        cb.lo[0] = k0.w; cb.lo[1] = k1.x; cb.lo[2] = k1.y;
        cb.d = k1.z;
        const V3<float> D = ca.minus(cb);
        // Sauter–Schwab pairs (a shared vertex) are the singular kernel's; such
        // pairs are always near: |c1 - c2| <= 2/3 (d1 + d2)
        auto touch = [&]() {
          return va0 == vb0 || va0 == vb1 || va0 == vb2 || va1 == vb0 || va1 == vb1 || va1 == vb2 || va2 == vb0 ||
                 va2 == vb1 || va2 == vb2;
        };
        if constexpr (NREG > 0) {
          if (touch()) {
            act = false;
          } else {
            owner_moments<NREG, true, BOTH>(X, XW, Ys, D, kr, ki, wantC, m);
            evals += NREG * NREG;
          }
        } else if (all_far) {
          owner_moments<3, true, BOTH>(X + RULE_OFF_FAR, XW + RULE_OFF_FAR, Ys, D, kr, ki, wantC, m);
          evals += 9;
        } else {
          const int c = pair_class<float>(D, ca.d, cb.d);
          if (c == 2) {
            owner_moments<3, true, BOTH>(X + RULE_OFF_FAR, XW + RULE_OFF_FAR, Ys, D, kr, ki, wantC, m);
            evals += 9;
          } else if (c == 0 && touch()) {
            act = false;
          } else {
            // near and medium pairs (under 1%): points from global memory
            const P4<float>* Y = cd.pts + (size_t)(b2 + i2) * NS;
            if (c == 1) {
              owner_moments<4, false, BOTH>(X + RULE_OFF_MEDIUM, XW + RULE_OFF_MEDIUM, Y + RULE_OFF_MEDIUM, D, kr,
                                            ki, wantC, m);
              evals += 16;
            } else {
              owner_moments<6, false, BOTH>(X, XW, Y, D, kr, ki, wantC, m);
              evals += 36;
            }
          }
        }
        if (act) {
          pair_c_coeffs(m, D, pc);
          // sigma terms: the pair coefficients that multiply sigma_b, times 1/|tau2|
          const float2 beta = dup2(k2.z), nbeta = dup2(-k2.z);
          a[0] = fma2(beta, m.Gxy, a[0]);
          a[1] = fma2(beta, m.G0, a[1]);
#pragma unroll
          for (int c = 0; c < 3; ++c) a[2 + c] = fma2(beta, m.Gy[c], a[2 + c]);
          a[5] = fma2(beta, pc.Dgxy, a[5]);
#pragma unroll
          for (int c = 0; c < 3; ++c) a[6 + c] = fma2(nbeta, pc.Y2[c], a[6 + c]);
        }
      }
      // the w_b terms, three slots at a time through registers
      const P4<float>* swb = Ys + NP;
      __syncwarp();
      tm_wait_st();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float rf[48];
        tm_ld32(tmr + 48 * h, rf);
        tm_ld16(tmr + 48 * h + 32, rf + 32);
        tm_wait_ld();
        if (act) {
          // every slot: past the cell's own, the records hold w_b = 0, so those
          // sums stay zero (and are never written out) without a branch here
#pragma unroll
          for (int bb = 0; bb < 3; ++bb) {
            const P4<float> u = swb[3 * h + bb];
            owner_slot_update(rf + 16 * bb, dup2(u.y), dup2(u.z), dup2(u.w), m, pc);
          }
        }
        __syncwarp();
        tm_st32(tmr + 48 * h, rf);
        tm_st16(tmr + 48 * h + 32, rf + 32);
      }
    }
    __syncthreads();  // every thread is done with the staged trial records: the records overwrite them
    tm_wait_st();
    {
      float* dst = rec + (size_t)threadIdx.x * NSL * BC_OWN_REC;
#pragma unroll
      for (int b = 0; b < NSL; ++b) {
        float f[16];
        tm_ld16(tmr + 16 * b, f);
        tm_wait_ld();
        if (item && b < ns2) {
          const float2 sb = dup2(js[j * NSL + b]);
          __align__(16) float2 tmp[BC_OWN_REC / 2];
          tmp[0] = fma2(sb, a[0], make_float2(f[0], f[1]));  // AS
          tmp[1] = mul2(sb, a[1]);                           // BS
#pragma unroll
          for (int c = 0; c < 3; ++c) tmp[2 + c] = fma2(sb, a[2 + c], make_float2(f[2 + 2 * c], f[3 + 2 * c]));  // WS
          tmp[5] = fma2(sb, a[5], make_float2(f[8], f[9]));  // AC
#pragma unroll
          for (int c = 0; c < 3; ++c) tmp[6 + c] = fma2(sb, a[6 + c], make_float2(f[10 + 2 * c], f[11 + 2 * c]));  // WC
          tmp[9] = z0;
          vcopy(dst + b * BC_OWN_REC, reinterpret_cast<const float*>(tmp), BC_OWN_REC);
        }
      }
    }
    if (threadIdx.x == 0) cp_async_wait_all();
    __syncthreads();  // records written; the next descriptor has landed
    // the next unit's trial-cell list (wnext was read in this unit's staging)
    if (more && (int)threadIdx.x < nextU->count) cp_async4(wnext + threadIdx.x, wlist + nextU->begin + threadIdx.x);
    // test-side contraction per (j, a, b), S and C together, summed over tau1;
    // the constants -ik and c4 of the S entry factor out of the sum
    for (int q = threadIdx.x; q < U.count * ns1 * NSL; q += TT) {
      const int j = q / (ns1 * NSL);
      const int rest = q - j * ns1 * NSL;
      const int sa_i = rest / NSL, sb_i = rest - (rest / NSL) * NSL;
      const int w = jw[j];
      if (sb_i >= jns[j] || jn[j] == 0) continue;
      float2 P = make_float2(0.f, 0.f), Q = P, Cs = P;
      for (int i1 = 0; i1 < n1; ++i1) {
        const P4<float> u = swA[i1 * nslot + sa_i];
        const float2 sa = dup2(u.x), wx = dup2(u.y), wy = dup2(u.z), wz = dup2(u.w);
        __align__(16) float2 o[BC_OWN_REC / 2];
        vcopy(reinterpret_cast<float*>(o), rec + ((size_t)(j * n1 + i1) * NSL + sb_i) * BC_OWN_REC, BC_OWN_REC);
        // S: sa AS + wa . WS (times -ik), sa BS (times c4); C: sa AC + wa . WC
        P = fma2(wz, o[4], fma2(wy, o[3], fma2(wx, o[2], fma2(sa, o[0], P))));
        Q = fma2(sa, o[1], Q);
        Cs = fma2(wz, o[8], fma2(wy, o[7], fma2(wx, o[6], fma2(sa, o[5], Cs))));
      }
      const float sr = mikr * P.x - miki * P.y + c4r * Q.x - c4i * Q.y;
      const float si = mikr * P.y + miki * P.x + c4r * Q.y + c4i * Q.x;
      const int ea = eaS[sa_i];
      const int eb = jeb[j * NSL + sb_i];
      out.add(ea, eb, wantS, wantC, sr, si, Cs.x, Cs.y);
      if (v != w) out.add(eb, ea, wantS, wantC, sr, si, Cs.x, Cs.y);
    }
    cp_async_wait_all();  // this thread's copies of the next trial-cell list
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tm_base), "r"(BC_OWN_TMEM_COLS)
                 : "memory");
  count_add(cnt, evals);
}

// ---------------------------------------------------------------------------
// Float32 RWG pairs in 16 x 16 tiles (rows: triangles tbi 16 + t, columns
// tbj 16 + t): the tile's triangles staged in shared memory once (rule points
// with the test weights folded in and the trial weights over 4 pi, centroids,
// vertex ids, slots and their edges), and each pair's moments, pair
// coefficients and 3 x 3 local S and C on packed (re, im) float32 pairs
// (FFMA2 / FADD2 / FMUL2). Used by the matrix-free product and by the stored
// assembly.
// ---------------------------------------------------------------------------
template <int NS>
struct RwgTile {
  P4<float> X[16 * NS];   // test points (rows)
  P4<float> XW[16 * NS];  // w (x, y, z), w
  P4<float> Y[16 * NS];   // trial points, w / 4 pi (columns)
  P4<float> SWR[48], SWC[48];  // slots (sigma, w) of rows and columns
  Cent<float> CR[16], CC[16];
  int VR[48], VC[48];  // vertex ids
  int ER[48], EC[48];  // slot edges
};

template <int NS>
__device__ __forceinline__ void rwg_tile_stage(RwgTile<NS>& T, const TriF* __restrict__ tri,
                                               const int* __restrict__ slot_edge, const float* __restrict__ slot_sw,
                                               int64_t t0, int64_t ntr, int tbi, int tbj, const Rules& rl, int tid) {
  for (int q = tid; q < 2 * 16 * NS; q += 256) {
    const int side = q / (16 * NS), rest = q - side * 16 * NS, t = rest / NS, u = rest - t * NS;
    const int64_t it = (int64_t)(side == 0 ? tbi : tbj) * 16 + t;
    if (it >= ntr) continue;
    const TriF tr = tri[t0 + it];
    const P4<float> p = staged_point(tr, rl, u);
    if (side == 0) {
      T.X[t * NS + u] = p;
      T.XW[t * NS + u] = {p.w * p.x, p.w * p.y, p.w * p.z, p.w};
    } else {
      T.Y[t * NS + u] = {p.x, p.y, p.z, p.w * INV_4PI_F};
    }
    if (u == 0) {
      (side == 0 ? T.CR : T.CC)[t].set(tr);
      int* v = (side == 0 ? T.VR : T.VC) + 3 * t;
      int* e = (side == 0 ? T.ER : T.EC) + 3 * t;
      P4<float>* w = (side == 0 ? T.SWR : T.SWC) + 3 * t;
      for (int a = 0; a < 3; ++a) {
        v[a] = tr.vid[a];
        e[a] = slot_edge[3 * (t0 + it) + a];
        w[a] = reinterpret_cast<const P4<float>*>(slot_sw)[3 * (t0 + it) + a];
      }
    }
  }
}

// The 3 x 3 local S and C of the pair (row ty, column tx) of a staged tile;
// false (and nothing formed) for touching pairs, whose entries are the
// singular kernel's. ev: the point-pair evaluations.
template <int NREG, int NS>
__device__ __forceinline__ bool rwg_tile_entries(const RwgTile<NS>& T, int ty, int tx, float kr, float ki, float mikr,
                                                 float miki, float c4r, float c4i, float2* S, float2* C,
                                                 unsigned& ev) {
  const int* va = T.VR + 3 * ty;
  const int* vb = T.VC + 3 * tx;
  bool touch = false;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) touch |= va[a] == vb[b];
  if (touch) return false;
  const Cent<float> ca = T.CR[ty], cb = T.CC[tx];
  const V3<float> D = ca.minus(cb);
  const P4<float>* Xa = T.X + ty * NS;
  const P4<float>* XWa = T.XW + ty * NS;
  const P4<float>* Yb = T.Y + tx * NS;
  Mom2 m;
  if constexpr (NREG > 0) {
    owner_moments<NREG, true, true>(Xa, XWa, Yb, D, kr, ki, true, m);
    ev = NREG * NREG;
  } else {
    const int c = pair_class<float>(D, ca.d, cb.d);
    if (c == 2) {
      owner_moments<3, true, true>(Xa + RULE_OFF_FAR, XWa + RULE_OFF_FAR, Yb + RULE_OFF_FAR, D, kr, ki, true, m);
      ev = 9;
    } else if (c == 1) {
      owner_moments<4, true, true>(Xa + RULE_OFF_MEDIUM, XWa + RULE_OFF_MEDIUM, Yb + RULE_OFF_MEDIUM, D, kr, ki, true,
                                   m);
      ev = 16;
    } else {
      owner_moments<6, true, true>(Xa, XWa, Yb, D, kr, ki, true, m);
      ev = 36;
    }
  }
  PairC2 pc;
  pair_c_coeffs(m, D, pc);
  // S_ab = -ik [s_a s_b Gxy + s_a w_b.Gx + s_b w_a.Gy + w_a.w_b G0] + c4 s_a s_b G0
  // C_ab = s_a s_b D.gxy + s_a w_b.X1 + s_b w_a.X2 + (w_a x w_b).V, X2 = -Y2
  const float2 c4G0 = make_float2(c4r * m.G0.x - c4i * m.G0.y, c4r * m.G0.y + c4i * m.G0.x);
  float2 wbGx[3], wbX1[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const P4<float> u = T.SWC[3 * tx + b];
    wbGx[b] = fma2(dup2(u.w), m.Gx[2], fma2(dup2(u.z), m.Gx[1], mul2(dup2(u.y), m.Gx[0])));
    wbX1[b] = fma2(dup2(u.w), pc.X1[2], fma2(dup2(u.z), pc.X1[1], mul2(dup2(u.y), pc.X1[0])));
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const P4<float> ua = T.SWR[3 * ty + a];
    const float2 waGy = fma2(dup2(ua.w), m.Gy[2], fma2(dup2(ua.z), m.Gy[1], mul2(dup2(ua.y), m.Gy[0])));
    const float2 waY2 = fma2(dup2(ua.w), pc.Y2[2], fma2(dup2(ua.z), pc.Y2[1], mul2(dup2(ua.y), pc.Y2[0])));
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const P4<float> ub = T.SWC[3 * tx + b];
      const float ss = ua.x * ub.x;
      const float ww = ua.y * ub.y + ua.z * ub.z + ua.w * ub.w;
      const float2 B = fma2(dup2(ss), m.Gxy, fma2(dup2(ua.x), wbGx[b], fma2(dup2(ub.x), waGy, mul2(dup2(ww), m.G0))));
      S[3 * a + b] = make_float2(mikr * B.x - miki * B.y + ss * c4G0.x, mikr * B.y + miki * B.x + ss * c4G0.y);
      const float cx = ua.z * ub.w - ua.w * ub.z, cy = ua.w * ub.y - ua.y * ub.w, cz = ua.y * ub.z - ua.z * ub.y;
      const float2 VW = fma2(dup2(cz), pc.V[2], fma2(dup2(cy), pc.V[1], mul2(dup2(cx), pc.V[0])));
      C[3 * a + b] = fma2(dup2(ss), pc.Dgxy, fma2(dup2(ua.x), wbX1[b], fma2(dup2(-ub.x), waY2, VW)));
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// A8, float32 operator and float32 vectors: the product of rwg_free_kernel on
// a staged tile with packed-pair arithmetic.
// ---------------------------------------------------------------------------
template <int NREG>
__global__ void __launch_bounds__(256) rwg_free_f32_kernel(
    const TriF* __restrict__ tri, const int* __restrict__ slot_edge, const float* __restrict__ slot_sw, int64_t t0,
    int64_t ntr, float kr, float ki, float mikr, float miki, float c4r, float c4i, Rules rl,
    const float2* __restrict__ x, float2* __restrict__ y, int64_t n, int nrhs, float ar, float ai, float br,
    float bi, unsigned long long* cnt) {
  constexpr int NS = staged_points<NREG>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RwgTile<NS>& T = *reinterpret_cast<RwgTile<NS>*>(smem_raw);
  float* acc = reinterpret_cast<float*>(&T + 1);  // as rwg_free_kernel
  const int* ER = T.ER;
  const int* EC = T.EC;
  const int tbi = blockIdx.y, tbj = blockIdx.x;
  if (tbi > tbj) return;  // the whole block: the tile lies below the diagonal
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 16 + tx;
  const int nacc = 2 * 16 * 3 * 2 * nrhs * 2;
  for (int q = tid; q < nacc; q += 256) acc[q] = 0.f;
  rwg_tile_stage<NS>(T, tri, slot_edge, slot_sw, t0, ntr, tbi, tbj, rl, tid);
  __syncthreads();
  const int64_t i1 = (int64_t)tbi * 16 + ty, i2 = (int64_t)tbj * 16 + tx;
  bool active = i1 < ntr && i2 < ntr && i1 < i2;
  const float2 z0 = make_float2(0.f, 0.f);
  float2 S[9], C[9];  // entries (a, b) of the pair, complex
#pragma unroll
  for (int q = 0; q < 9; ++q) S[q] = C[q] = z0;
  if (active) {
    unsigned ev = 0;
    active = rwg_tile_entries<NREG, NS>(T, ty, tx, kr, ki, mikr, miki, c4r, c4i, S, C, ev);
    if (active) count_add(cnt, ev * (unsigned)nrhs);
  }
  int ea[3], eb[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ea[a] = ER[3 * ty + a];
    eb[a] = EC[3 * tx + a];
  }
  // complex product e v accumulated into acc: (er v + ei (-v.y, v.x))
  auto cmac = [](float2 e, float2 v, float2 vs, float2 a) { return fma2(dup2(e.y), vs, fma2(dup2(e.x), v, a)); };
  for (int r = 0; r < nrhs; ++r) {
    const float2* x1 = x + (int64_t)r * 2 * n;
    const float2* x2 = x1 + n;
    float2 u1[3], u2[3], v1[3], v2[3], u1s[3], u2s[3], v1s[3], v2s[3];  // x at t1 (u) and t2 (v); swapped
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      u1[a] = u2[a] = v1[a] = v2[a] = z0;
      if (active) {
        u1[a] = x1[ea[a]];
        u2[a] = x2[ea[a]];
        v1[a] = x1[eb[a]];
        v2[a] = x2[eb[a]];
      }
      u1s[a] = make_float2(-u1[a].y, u1[a].x);
      u2s[a] = make_float2(-u2[a].y, u2[a].x);
      v1s[a] = make_float2(-v1[a].y, v1[a].x);
      v2s[a] = make_float2(-v2[a].y, v2[a].x);
    }
    float row[12], col[12];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2 c1 = z0, c2 = z0, s1 = z0, s2 = z0;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int k = 3 * a + b;
        c1 = cmac(C[k], v1[b], v1s[b], c1);
        c2 = cmac(C[k], v2[b], v2s[b], c2);
        s1 = cmac(S[k], v1[b], v1s[b], s1);
        s2 = cmac(S[k], v2[b], v2s[b], s2);
      }
      row[4 * a + 0] = c1.x + ar * s2.x - ai * s2.y;
      row[4 * a + 1] = c1.y + ar * s2.y + ai * s2.x;
      row[4 * a + 2] = c2.x + br * s1.x - bi * s1.y;
      row[4 * a + 3] = c2.y + br * s1.y + bi * s1.x;
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      float2 c1 = z0, c2 = z0, s1 = z0, s2 = z0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int k = 3 * a + b;
        c1 = cmac(C[k], u1[a], u1s[a], c1);
        c2 = cmac(C[k], u2[a], u2s[a], c2);
        s1 = cmac(S[k], u1[a], u1s[a], s1);
        s2 = cmac(S[k], u2[a], u2s[a], s2);
      }
      col[4 * b + 0] = c1.x + ar * s2.x - ai * s2.y;
      col[4 * b + 1] = c1.y + ar * s2.y + ai * s2.x;
      col[4 * b + 2] = c2.x + br * s1.x - bi * s1.y;
      col[4 * b + 3] = c2.y + br * s1.y + bi * s1.x;
    }
    // rows share t1 across the 16 lanes of a half warp; columns share t2
    // across the two half warps
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      float v = row[q];
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      row[q] = v;
      col[q] += __shfl_xor_sync(0xffffffffu, col[q], 16);
    }
    if (tx == 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float* o = acc + ((((0 * 16 + ty) * 3 + a) * 2 + h) * nrhs + r) * 2;
          o[0] += row[4 * a + 2 * h];
          o[1] += row[4 * a + 2 * h + 1];
        }
    }
    if ((ty & 1) == 0) {
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float* o = acc + ((((1 * 16 + tx) * 3 + b) * 2 + h) * nrhs + r) * 2;
          atomicAdd(o, col[4 * b + 2 * h]);
          atomicAdd(o + 1, col[4 * b + 2 * h + 1]);
        }
    }
  }
  __syncthreads();
  // flush: one atomic per (side, triangle, slot, half, rhs)
  for (int q = tid; q < nacc / 2; q += 256) {
    const int r = q % nrhs;
    int rest = q / nrhs;
    const int h = rest % 2;
    rest /= 2;
    const int slot = rest % 3;
    rest /= 3;
    const int t = rest % 16, side = rest / 16;
    const int64_t tt = (int64_t)(side == 0 ? tbi : tbj) * 16 + t;
    if (tt >= ntr) continue;
    const float vr = acc[2 * q], vi = acc[2 * q + 1];
    if (vr == 0.f && vi == 0.f) continue;
    const int e = (side == 0 ? ER : EC)[3 * t + slot];
    if (e < 0) continue;
    atomicAdd(y + (int64_t)r * 2 * n + (int64_t)h * n + e, make_float2(vr, vi));
  }
}

// ---------------------------------------------------------------------------
// A3, float32: the stored regular RWG pairs on a staged tile with packed-pair
// arithmetic. The tile's 48 row slots and 48 column slots map to their
// distinct edges (neighbouring triangles share edges); each pair adds its
// 3 x 3 S and C into a shared edge x edge accumulator, and each non-zero
// cell goes to the block once, with its mirror (both operators are
// symmetric on regular pairs).
// ---------------------------------------------------------------------------
constexpr int RWG_TILE_SLOTS = 48;

template <int NREG>
__global__ void __launch_bounds__(256) rwg_regular_f32_kernel(
    const TriF* __restrict__ tri, const int* __restrict__ slot_edge, const float* __restrict__ slot_sw, int64_t t0,
    int64_t ntr, float kr, float ki, float mikr, float miki, float c4r, float c4i, bool wantS, bool wantC, Rules rl,
    Sink<float> out, unsigned long long* cnt) {
  constexpr int NS = staged_points<NREG>();
  constexpr int NE = RWG_TILE_SLOTS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RwgTile<NS>& T = *reinterpret_cast<RwgTile<NS>*>(smem_raw);
  float* accS = reinterpret_cast<float*>(&T + 1);  // [NE][NE] complex
  float* accC = accS + 2 * NE * NE;
  int* UR = reinterpret_cast<int*>(accC + 2 * NE * NE);  // slot -> distinct row edge (or -1)
  int* UC = UR + NE;
  int* firstR = UC + NE;  // 1 where a slot holds the first occurrence of its edge
  int* firstC = firstR + NE;
  int* uER = firstC + NE;  // the distinct row edges, in slot order of first occurrence
  int* uEC = uER + NE;
  int* nU = uEC + NE;     // distinct row and column edges
  const int tbi = blockIdx.y, tbj = blockIdx.x;
  if (tbi > tbj) return;  // the whole block: the tile lies below the diagonal
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 16 + tx;
  for (int q = tid; q < 4 * NE * NE; q += 256) accS[q] = 0.f;  // accS and accC
  rwg_tile_stage<NS>(T, tri, slot_edge, slot_sw, t0, ntr, tbi, tbj, rl, tid);
  __syncthreads();
  // distinct edges: slot q (rows: threads 0..47, columns: 64..111) is a first
  // occurrence when no earlier slot of its side has its edge; its index is
  // the count of first occurrences before its first occurrence
  const int side = tid < 64 ? 0 : 1, q = tid - 64 * side;
  const int* E = side == 0 ? T.ER : T.EC;
  const int64_t base = (int64_t)(side == 0 ? tbi : tbj) * 16;
  int first = -1;
  if (tid < 128 && q < NE && base + q / 3 < ntr && E[q] >= 0) {
    first = q;
    for (int r = 0; r < q; ++r)
      if (base + r / 3 < ntr && E[r] == E[q]) {
        first = r;
        break;
      }
    (side == 0 ? firstR : firstC)[q] = first == q;
  } else if (tid < 128 && q < NE) {
    (side == 0 ? firstR : firstC)[q] = 0;
  }
  __syncthreads();
  if (tid < 128 && q < NE) {
    const int* F = side == 0 ? firstR : firstC;
    int u = -1;
    if (first >= 0) {
      u = 0;
      for (int r = 0; r < first; ++r) u += F[r];
    }
    (side == 0 ? UR : UC)[q] = u;
    if (first == q) (side == 0 ? uER : uEC)[u] = E[q];
    if (q == NE - 1) {
      int n = 0;
      for (int r = 0; r < NE; ++r) n += F[r];
      nU[side] = n;
    }
  }
  __syncthreads();
  const int64_t i1 = (int64_t)tbi * 16 + ty, i2 = (int64_t)tbj * 16 + tx;
  if (i1 < ntr && i2 < ntr && i1 < i2) {
    float2 S[9], C[9];
    unsigned ev = 0;
    if (rwg_tile_entries<NREG, NS>(T, ty, tx, kr, ki, mikr, miki, c4r, c4i, S, C, ev)) {
      count_add(cnt, ev);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int ur = UR[3 * ty + a];
        if (ur < 0) continue;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const int uc = UC[3 * tx + b];
          if (uc < 0) continue;
          const int k = 2 * (ur * NE + uc);
          atomicAdd(accS + k, S[3 * a + b].x);
          atomicAdd(accS + k + 1, S[3 * a + b].y);
          atomicAdd(accC + k, C[3 * a + b].x);
          atomicAdd(accC + k + 1, C[3 * a + b].y);
        }
      }
    }
  }
  __syncthreads();
  // flush: the distinct edges of each side (slot order of first occurrences)
  const int nr = nU[0], nc = nU[1];
  for (int q2 = tid; q2 < nr * nc; q2 += 256) {
    const int ur = q2 / nc, uc = q2 - ur * nc;
    const int k = 2 * (ur * NE + uc);
    const float sr = accS[k], si = accS[k + 1], cr = accC[k], ci = accC[k + 1];
    if (sr == 0.f && si == 0.f && cr == 0.f && ci == 0.f) continue;
    const int er = uER[ur], ec = uEC[uc];
    out.add(er, ec, wantS, wantC, sr, si, cr, ci);
    out.add(ec, er, wantS, wantC, sr, si, cr, ci);
  }
}

constexpr int BC_OWNER_TT = 128;

// trial cells per unit for the one-thread-per-(test triangle, trial cell)
// kernel with a test cell of n1 triangles and at most max_cell triangles per
// cell; 0 when that kernel does not apply (float64, cells with more than
// BC_OWN_SLOTS edges or more than BC_OWN_STAGE triangles)
int bc_owner_width(const Space& s, int precision, int n1, int max_cell) {
  if (precision != CAL_FP32 || s.nslot > BC_OWN_SLOTS || !s.sigma_factors || n1 < 1 || n1 > BC_OWNER_TT ||
      max_cell < n1 || max_cell > BC_OWN_STAGE)
    return 0;
  return std::max(1, std::min(BC_OWNER_TT / n1, BC_OWN_STAGE / max_cell));
}

// ---------------------------------------------------------------------------
// A4: singular pairs by Sauter–Schwab rules in float64, one warp per ordered
// pair; the q^4 Gauss points of all sub-regions are spread over the lanes.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ void ss_map(int cls, int r, double xi, double e1, double e2, double e3,
                                       double* xh, double* yh, double& jac) {
  // maps of [0,1]^4 onto pairs of points of the reference triangle
  // {0 <= s2 <= s1 <= 1}; shared vertex at (0,0), shared edge (0,0)-(1,0)
  if (cls == 3) {
    jac = xi * xi * xi * e1 * e1 * e2;
    switch (r) {
      case 0: xh[0] = xi; xh[1] = xi * (1 - e1 + e1 * e2); yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * (1 - e1); break;
      case 1: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * (1 - e1); yh[0] = xi; yh[1] = xi * (1 - e1 + e1 * e2); break;
      case 2: xh[0] = xi; xh[1] = xi * e1 * (1 - e2 + e2 * e3); yh[0] = xi * (1 - e1 * e2); yh[1] = xi * e1 * (1 - e2); break;
      case 3: xh[0] = xi * (1 - e1 * e2); xh[1] = xi * e1 * (1 - e2); yh[0] = xi; yh[1] = xi * e1 * (1 - e2 + e2 * e3); break;
      case 4: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * (1 - e2 * e3); yh[0] = xi; yh[1] = xi * e1 * (1 - e2); break;
      default: xh[0] = xi; xh[1] = xi * e1 * (1 - e2); yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * e1 * (1 - e2 * e3); break;
    }
  } else if (cls == 2) {
    jac = xi * xi * xi * e1 * e1 * (r == 0 ? 1.0 : e2);
    switch (r) {
      case 0: xh[0] = xi; xh[1] = xi * e1 * e3; yh[0] = xi * (1 - e1 * e2); yh[1] = xi * e1 * (1 - e2); break;
      case 1: xh[0] = xi; xh[1] = xi * e1; yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * e1 * e2 * (1 - e3); break;
      case 2: xh[0] = xi * (1 - e1 * e2); xh[1] = xi * e1 * (1 - e2); yh[0] = xi; yh[1] = xi * e1 * e2 * e3; break;
      case 3: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * e2 * (1 - e3); yh[0] = xi; yh[1] = xi * e1; break;
      default: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * (1 - e2 * e3); yh[0] = xi; yh[1] = xi * e1 * e2; break;
    }
  } else {
    jac = xi * xi * xi * e2;
    if (r == 0) { xh[0] = xi; xh[1] = xi * e1; yh[0] = xi * e2; yh[1] = xi * e2 * e3; }
    else { xh[0] = xi * e2; xh[1] = xi * e2 * e3; yh[0] = xi; yh[1] = xi * e1; }
  }
}

// Float32 variant of the singular rules. Near the singularity x - y is small
// while x and y are not, so instead of subtracting mapped points the
// difference is assembled from reference-coordinate differences that each
// map yields in closed form (e.g. x1 - y1 = xi e1 e2 in the first identical
// sub-region) times the panel edge vectors; shared vertices cancel exactly.
__device__ __forceinline__ void ss_map_f32(int cls, int r, float xi, float e1, float e2, float e3,
                                           float* xh, float* yh, float* dh, float& jac) {
  if (cls == 3) {
    jac = xi * xi * xi * e1 * e1 * e2;
    const float a = xi * e1 * e2, b = a * e3;  // xi e1 e2, xi e1 e2 e3
    switch (r) {
      case 0: xh[0] = xi; xh[1] = xi * (1 - e1 + e1 * e2); yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * (1 - e1);
              dh[0] = b; dh[1] = a; break;
      case 1: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * (1 - e1); yh[0] = xi; yh[1] = xi * (1 - e1 + e1 * e2);
              dh[0] = -b; dh[1] = -a; break;
      case 2: xh[0] = xi; xh[1] = xi * e1 * (1 - e2 + e2 * e3); yh[0] = xi * (1 - e1 * e2); yh[1] = xi * e1 * (1 - e2);
              dh[0] = a; dh[1] = b; break;
      case 3: xh[0] = xi * (1 - e1 * e2); xh[1] = xi * e1 * (1 - e2); yh[0] = xi; yh[1] = xi * e1 * (1 - e2 + e2 * e3);
              dh[0] = -a; dh[1] = -b; break;
      case 4: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * (1 - e2 * e3); yh[0] = xi; yh[1] = xi * e1 * (1 - e2);
              dh[0] = -b; dh[1] = a * (1 - e3); break;
      default: xh[0] = xi; xh[1] = xi * e1 * (1 - e2); yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * e1 * (1 - e2 * e3);
               dh[0] = b; dh[1] = -a * (1 - e3); break;
    }
  } else if (cls == 2) {
    jac = xi * xi * xi * e1 * e1 * (r == 0 ? 1.0f : e2);
    switch (r) {
      case 0: xh[0] = xi; xh[1] = xi * e1 * e3; yh[0] = xi * (1 - e1 * e2); yh[1] = xi * e1 * (1 - e2);
              dh[0] = xi * e1 * e2; break;
      case 1: xh[0] = xi; xh[1] = xi * e1; yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * e1 * e2 * (1 - e3);
              dh[0] = xi * e1 * e2 * e3; break;
      case 2: xh[0] = xi * (1 - e1 * e2); xh[1] = xi * e1 * (1 - e2); yh[0] = xi; yh[1] = xi * e1 * e2 * e3;
              dh[0] = -xi * e1 * e2; break;
      case 3: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * e2 * (1 - e3); yh[0] = xi; yh[1] = xi * e1;
              dh[0] = -xi * e1 * e2 * e3; break;
      default: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * (1 - e2 * e3); yh[0] = xi; yh[1] = xi * e1 * e2;
               dh[0] = -xi * e1 * e2 * e3; break;
    }
    dh[1] = 0.0f;  // unused: the second coordinates lie on different panels
  } else {
    jac = xi * xi * xi * e2;
    if (r == 0) { xh[0] = xi; xh[1] = xi * e1; yh[0] = xi * e2; yh[1] = xi * e2 * e3; }
    else { xh[0] = xi * e2; xh[1] = xi * e2 * e3; yh[0] = xi; yh[1] = xi * e1; }
    dh[0] = dh[1] = 0.0f;
  }
}

struct RulesF { float gx[16], gw[16]; int ng; };

__global__ void __launch_bounds__(128) singular_kernel_f32(
    const TriF* __restrict__ tri, const SingPair* __restrict__ pairs, int64_t np,
    const int* __restrict__ slot_edge, const float* __restrict__ slot_sw, int nslot, float kr,
    float ki, float mikr, float miki, float c4r, float c4i, bool wantS, bool wantC, RulesF rl,
    Sink<float> out) {
  const int lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (p >= np) return;
  const SingPair sp = pairs[p];
  const TriF A = tri[sp.t1];
  const TriF B = tri[sp.t2];
  const int cls = sp.cls;
  const bool doC = wantC && cls != 3;
  V3<float> Q1[3], Q2[3];
  for (int a = 0; a < 3; ++a) {
    Q1[a] = {A.off[sp.o1[a]][0], A.off[sp.o1[a]][1], A.off[sp.o1[a]][2]};
    Q2[a] = {B.off[sp.o2[a]][0], B.off[sp.o2[a]][1], B.off[sp.o2[a]][2]};
  }
  const V3<float> E1 = {Q1[1].x - Q1[0].x, Q1[1].y - Q1[0].y, Q1[1].z - Q1[0].z};
  const V3<float> F1 = {Q1[2].x - Q1[1].x, Q1[2].y - Q1[1].y, Q1[2].z - Q1[1].z};
  const V3<float> E2 = {Q2[1].x - Q2[0].x, Q2[1].y - Q2[0].y, Q2[1].z - Q2[0].z};
  const V3<float> F2 = {Q2[2].x - Q2[1].x, Q2[2].y - Q2[1].y, Q2[2].z - Q2[1].z};
  const V3<float> D = centroid_delta(A, B);
  const float scale = 4.0f * A.area * B.area;
  const int ng = rl.ng, nreg = (cls == 3 ? 6 : (cls == 2 ? 5 : 2));
  const int ng2 = ng * ng, ng4 = ng2 * ng2;
  Mom<float> m;
  m.zero();
  for (int idx = lane; idx < nreg * ng4; idx += 32) {
    const int r = idx / ng4;
    int rem = idx - r * ng4;
    const int a0 = rem / (ng2 * ng);
    rem -= a0 * ng2 * ng;
    const int a1 = rem / ng2;
    rem -= a1 * ng2;
    const int a2 = rem / ng, a3 = rem - a2 * ng;
    float xh[2], yh[2], dh[2], jac;
    ss_map_f32(cls, r, rl.gx[a0], rl.gx[a1], rl.gx[a2], rl.gx[a3], xh, yh, dh, jac);
    const float w = rl.gw[a0] * rl.gw[a1] * rl.gw[a2] * rl.gw[a3] * jac * scale;
    const V3<float> x = {Q1[0].x + xh[0] * E1.x + xh[1] * F1.x, Q1[0].y + xh[0] * E1.y + xh[1] * F1.y,
                         Q1[0].z + xh[0] * E1.z + xh[1] * F1.z};
    const V3<float> y = {Q2[0].x + yh[0] * E2.x + yh[1] * F2.x, Q2[0].y + yh[0] * E2.y + yh[1] * F2.y,
                         Q2[0].z + yh[0] * E2.z + yh[1] * F2.z};
    V3<float> d;  // x - y without cancellation
    if (cls == 3) {
      d = {dh[0] * E1.x + dh[1] * F1.x, dh[0] * E1.y + dh[1] * F1.y, dh[0] * E1.z + dh[1] * F1.z};
    } else if (cls == 2) {
      d = {dh[0] * E1.x + xh[1] * F1.x - yh[1] * F2.x, dh[0] * E1.y + xh[1] * F1.y - yh[1] * F2.y,
           dh[0] * E1.z + xh[1] * F1.z - yh[1] * F2.z};
    } else {
      d = {xh[0] * E1.x + xh[1] * F1.x - yh[0] * E2.x - yh[1] * F2.x,
           xh[0] * E1.y + xh[1] * F1.y - yh[0] * E2.y - yh[1] * F2.y,
           xh[0] * E1.z + xh[1] * F1.z - yh[0] * E2.z - yh[1] * F2.z};
    }
    float Gr, Gi, gr, gi;
    green(d.x * d.x + d.y * d.y + d.z * d.z, kr, ki, Gr, Gi, gr, gi);
    Gr *= w; Gi *= w; gr *= w; gi *= w;
    m.G0r += Gr; m.G0i += Gi;
    m.Gxr.x += Gr * x.x; m.Gxr.y += Gr * x.y; m.Gxr.z += Gr * x.z;
    m.Gxi.x += Gi * x.x; m.Gxi.y += Gi * x.y; m.Gxi.z += Gi * x.z;
    m.Gyr.x += Gr * y.x; m.Gyr.y += Gr * y.y; m.Gyr.z += Gr * y.z;
    m.Gyi.x += Gi * y.x; m.Gyi.y += Gi * y.y; m.Gyi.z += Gi * y.z;
    const float xy = dot3(x, y);
    m.Gxyr += Gr * xy; m.Gxyi += Gi * xy;
    if (doC) {
      const V3<float> xy3 = cross3(x, y);
      m.g0r += gr; m.g0i += gi;
      m.gxr.x += gr * x.x; m.gxr.y += gr * x.y; m.gxr.z += gr * x.z;
      m.gxi.x += gi * x.x; m.gxi.y += gi * x.y; m.gxi.z += gi * x.z;
      m.gyr.x += gr * y.x; m.gyr.y += gr * y.y; m.gyr.z += gr * y.z;
      m.gyi.x += gi * y.x; m.gyi.y += gi * y.y; m.gyi.z += gi * y.z;
      m.gxyr.x += gr * xy3.x; m.gxyr.y += gr * xy3.y; m.gxyr.z += gr * xy3.z;
      m.gxyi.x += gi * xy3.x; m.gxyi.y += gi * xy3.y; m.gxyi.z += gi * xy3.z;
    }
  }
  float* mv = reinterpret_cast<float*>(&m);
  constexpr int NM = sizeof(Mom<float>) / sizeof(float);
#pragma unroll
  for (int q = 0; q < NM; ++q) {
    float v = mv[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    mv[q] = v;
  }
  float pc[36];
  pair_coeffs(m, D, pc);
  for (int q = lane; q < nslot * nslot; q += 32) {
    const int a = q / nslot, b = q % nslot;
    const int ea = slot_edge[(size_t)sp.t1 * nslot + a];
    const int eb = slot_edge[(size_t)sp.t2 * nslot + b];
    if (ea < 0 || eb < 0) continue;
    const float* swa = slot_sw + ((size_t)sp.t1 * nslot + a) * 4;
    const float* swb = slot_sw + ((size_t)sp.t2 * nslot + b) * 4;
    const V3<float> wa = {swa[1], swa[2], swa[3]}, wb = {swb[1], swb[2], swb[3]};
    float Sr = 0, Si = 0, Cr = 0, Ci = 0;
    entry_from_pc(pc, swa[0], wa, swb[0], wb, mikr, miki, c4r, c4i, wantS, doC, Sr, Si, Cr, Ci);
    out.add(ea, eb, wantS, doC, Sr, Si, Cr, Ci);
    if (cls == 1) out.add(eb, ea, wantS, doC, Sr, Si, Cr, Ci);
  }
}

// ---------------------------------------------------------------------------
// Double-precision e^{i theta} and e^{z} for the singular-pair kernel. Argument
// reduction after Cody and Waite (pi/2 split into three parts and ln 2 into
// two, each leading part short enough that n * part is exact), then truncated
// Taylor series on the reduced interval: |t| <= pi/4 with terms up to t^17
// (the first omitted term is below 1e-19) and |t| <= ln(2)/2 with terms up to
// t^13 (below 5e-18). Arguments outside the reduction's range go to the CUDA
// library. The split constants are the binary expansions of pi/2 and ln 2.
// ---------------------------------------------------------------------------
namespace dm {
constexpr double PIO2_A = 1.5707963267341256, PIO2_B = 6.077100506303966e-11, PIO2_C = 2.0222662487959506e-21;
constexpr double TWO_OVER_PI = 0.6366197723675814;
constexpr double LN2_A = 0.6931471805598903, LN2_B = 5.497923018708371e-14;
constexpr double LOG2E = 1.4426950408889634;
}  // namespace dm

__device__ __forceinline__ void cis_f64(double th, double& c, double& s) {
  if (!(fabs(th) < 1.0e6)) {
    sincos(th, &s, &c);
    return;
  }
  const double n = rint(th * dm::TWO_OVER_PI);
  double t = fma(-n, dm::PIO2_A, th);
  t = fma(-n, dm::PIO2_B, t);
  t = fma(-n, dm::PIO2_C, t);
  const double u = -t * t;
  // cos t = sum_k u^k / (2k)!,  sin t = t sum_k u^k / (2k+1)!,  k = 0..8
  double pc = 1.0 / 20922789888000.0;
  pc = fma(pc, u, 1.0 / 87178291200.0);
  pc = fma(pc, u, 1.0 / 479001600.0);
  pc = fma(pc, u, 1.0 / 3628800.0);
  pc = fma(pc, u, 1.0 / 40320.0);
  pc = fma(pc, u, 1.0 / 720.0);
  pc = fma(pc, u, 1.0 / 24.0);
  pc = fma(pc, u, 0.5);
  pc = fma(pc, u, 1.0);
  double ps = 1.0 / 355687428096000.0;
  ps = fma(ps, u, 1.0 / 1307674368000.0);
  ps = fma(ps, u, 1.0 / 6227020800.0);
  ps = fma(ps, u, 1.0 / 39916800.0);
  ps = fma(ps, u, 1.0 / 362880.0);
  ps = fma(ps, u, 1.0 / 5040.0);
  ps = fma(ps, u, 1.0 / 120.0);
  ps = fma(ps, u, 1.0 / 6.0);
  ps = fma(ps, u, 1.0);
  ps *= t;
  // e^{i theta} = e^{i t} i^q
  const int q = (int)n & 3;
  c = q == 0 ? pc : (q == 1 ? -ps : (q == 2 ? -pc : ps));
  s = q == 0 ? ps : (q == 1 ? pc : (q == 2 ? -ps : -pc));
}

__device__ __forceinline__ double exp_f64(double z) {
  if (!(fabs(z) < 700.0)) return exp(z);
  const double n = rint(z * dm::LOG2E);
  double t = fma(-n, dm::LN2_A, z);
  t = fma(-n, dm::LN2_B, t);
  double p = 1.0 / 6227020800.0;
  p = fma(p, t, 1.0 / 479001600.0);
  p = fma(p, t, 1.0 / 39916800.0);
  p = fma(p, t, 1.0 / 3628800.0);
  p = fma(p, t, 1.0 / 362880.0);
  p = fma(p, t, 1.0 / 40320.0);
  p = fma(p, t, 1.0 / 5040.0);
  p = fma(p, t, 1.0 / 720.0);
  p = fma(p, t, 1.0 / 120.0);
  p = fma(p, t, 1.0 / 24.0);
  p = fma(p, t, 1.0 / 6.0);
  p = fma(p, t, 0.5);
  p = fma(p, t, 1.0);
  p = fma(p, t, 1.0);
  return p * __longlong_as_double((long long)((int)n + 1023) << 52);
}

// max |cis_f64 - (cos, sin)| and max relative |exp_f64 - exp| over n points
// spread evenly on [lo, hi] (the library functions as the yardstick)
__global__ void elementary_check_kernel(int64_t n, double lo, double hi, unsigned long long* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = lo + (hi - lo) * ((double)i / (double)(n > 1 ? n - 1 : 1));
  double c, s, c0, s0;
  cis_f64(x, c, s);
  sincos(x, &s0, &c0);
  const double ec = fmax(fabs(c - c0), fabs(s - s0));
  const double e0 = exp(-fabs(x));
  const double ee = e0 > 0 ? fabs(exp_f64(-fabs(x)) - e0) / e0 : 0.0;
  // non-negative doubles order like their bit patterns
  atomicMax(err, (unsigned long long)__double_as_longlong(ec));
  atomicMax(err + 1, (unsigned long long)__double_as_longlong(ee));
}

int check_elementary(int64_t n, double lo, double hi, double* err_cis, double* err_exp) {
  if (n < 1 || !(hi >= lo) || !err_cis || !err_exp) return fail(CAL_EINVAL, "elementary check: bad arguments");
  unsigned long long* d = nullptr;
  CAL_TRY_CUDA(cudaMalloc((void**)&d, 2 * sizeof(unsigned long long)));
  cudaMemset(d, 0, 2 * sizeof(unsigned long long));
  elementary_check_kernel<<<(unsigned)((n + 255) / 256), 256>>>(n, lo, hi, d);
  note_launch();
  unsigned long long h[2] = {0, 0};
  const cudaError_t e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  CAL_TRY_CUDA(e);
  double v[2];
  std::memcpy(v, h, sizeof(v));
  *err_cis = v[0];
  *err_exp = v[1];
  return CAL_OK;
}

// Radial sums of one (region, e) direction: over the Gauss nodes xi_j of the
// radial variable, with r = xi_j rho,
//   SG_d += e^{ikr} w_j xi_j^2 xi_j^d,  Sg_d += (ikr - 1) e^{ikr} w_j xi_j^d,  d = 0, 1, 2,
// as (re, im) pairs. NG > 0 fixes the node count at compile time (unrolled).
template <int NG>
__device__ __forceinline__ void radial_sums(const double* gx, const double* gw, int ng, double rho, double kr,
                                            double ki, bool doC, double* SG, double* Sg) {
  const int nn = NG > 0 ? NG : ng;
#pragma unroll
  for (int j = 0; j < (NG > 0 ? NG : 16); ++j) {
    if (NG == 0 && j >= nn) break;
    const double xi = gx[j], wj = gw[j];
    const double rr = xi * rho;
    double cth, sth;
    cis_f64(kr * rr, cth, sth);
    if (ki != 0.0) {
      const double e = exp_f64(-ki * rr);
      cth *= e;
      sth *= e;
    }
    const double tg = wj * xi * xi;
    const double Tr = cth * tg, Ti = sth * tg;
    SG[0] += Tr; SG[1] += Ti;
    SG[2] = fma(Tr, xi, SG[2]); SG[3] = fma(Ti, xi, SG[3]);
    SG[4] = fma(Tr, xi * xi, SG[4]); SG[5] = fma(Ti, xi * xi, SG[5]);
    if (doC) {
      const double fr = -ki * rr - 1.0, fi = kr * rr;
      const double Ur = (fr * cth - fi * sth) * wj, Ui = (fr * sth + fi * cth) * wj;
      Sg[0] += Ur; Sg[1] += Ui;
      Sg[2] = fma(Ur, xi, Sg[2]); Sg[3] = fma(Ui, xi, Sg[3]);
      Sg[4] = fma(Ur, xi * xi, Sg[4]); Sg[5] = fma(Ui, xi * xi, Sg[5]);
    }
  }
}

// Reference-coordinate moments MG, Mg (18 reals each: (re, im) of the nine
// monomials) -> centroid-relative moments -> pair coefficients -> entries of
// the (test slot, trial slot) combinations q = first, first + step, ...
// pair coefficients (the layout of pair_coeffs) of a touching pair from its
// float64 monomial moments and parametrisation
__device__ __forceinline__ void sing_pair_coeffs(const double* MG, const double* Mg, const V3<double>* Q1,
                                                 const V3<double>* Q2, const V3<double>& ea, const V3<double>& eb,
                                                 const V3<double>& ec, const V3<double>& ed, const V3<double>& D,
                                                 double* pc) {
  // x = q0 + x0 a + x1 b, y = p0 + y0 c + y1 d
  const V3<double> q0 = Q1[0], p0 = Q2[0];
  const V3<double> vx[3] = {q0, ea, eb};  // factors of 1, x0, x1
  const V3<double> vy[3] = {p0, ec, ed};  // factors of 1, y0, y1
  // monomial index of (i, j): i, j in {0: 1, 1: first, 2: second}
  auto mix = [](int i, int j) { return i == 0 ? (j == 0 ? 0 : 2 + j) : (j == 0 ? i : 2 * i + j + 2); };
  Mom<double> m;
  m.zero();
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // re, im (unrolled: the moment arrays stay in registers)
    double G0 = MG[h], g0 = Mg[h];
    V3<double> Gx = {0, 0, 0}, Gy = {0, 0, 0}, gx = {0, 0, 0}, gy = {0, 0, 0}, gxy = {0, 0, 0};
    double Gxy = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double Mxi = MG[2 * mix(i, 0) + h], mxi = Mg[2 * mix(i, 0) + h];
      Gx = {Gx.x + vx[i].x * Mxi, Gx.y + vx[i].y * Mxi, Gx.z + vx[i].z * Mxi};
      gx = {gx.x + vx[i].x * mxi, gx.y + vx[i].y * mxi, gx.z + vx[i].z * mxi};
      const double Myi = MG[2 * mix(0, i) + h], myi = Mg[2 * mix(0, i) + h];
      Gy = {Gy.x + vy[i].x * Myi, Gy.y + vy[i].y * Myi, Gy.z + vy[i].z * Myi};
      gy = {gy.x + vy[i].x * myi, gy.y + vy[i].y * myi, gy.z + vy[i].z * myi};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double Mij = MG[2 * mix(i, j) + h], mij = Mg[2 * mix(i, j) + h];
        Gxy += dot3(vx[i], vy[j]) * Mij;
        const V3<double> cxy = cross3(vx[i], vy[j]);
        gxy = {gxy.x + cxy.x * mij, gxy.y + cxy.y * mij, gxy.z + cxy.z * mij};
      }
    }
    if (h == 0) {
      m.G0r = G0; m.Gxr = Gx; m.Gyr = Gy; m.Gxyr = Gxy;
      m.g0r = g0; m.gxr = gx; m.gyr = gy; m.gxyr = gxy;
    } else {
      m.G0i = G0; m.Gxi = Gx; m.Gyi = Gy; m.Gxyi = Gxy;
      m.g0i = g0; m.gxi = gx; m.gyi = gy; m.gxyi = gxy;
    }
  }
  pair_coeffs(m, D, pc);
}

template <typename RO>
__device__ __forceinline__ void sing_emit(const double* MG, const double* Mg, const V3<double>* Q1,
                                          const V3<double>* Q2, const V3<double>& ea, const V3<double>& eb,
                                          const V3<double>& ec, const V3<double>& ed, const V3<double>& D,
                                          const SingPair& sp, const int* __restrict__ slot_edge,
                                          const double* __restrict__ slot_sw, int nslot, double mikr, double miki,
                                          double c4r, double c4i, bool wantS, bool doC, int first, int step,
                                          const Sink<RO>& out) {
  const int cls = sp.cls;
  double pc[36];
  sing_pair_coeffs(MG, Mg, Q1, Q2, ea, eb, ec, ed, D, pc);
  for (int q = first; q < nslot * nslot; q += step) {
    const int a = q / nslot, b = q % nslot;
    const int e1 = slot_edge[(size_t)sp.t1 * nslot + a];
    const int e2 = slot_edge[(size_t)sp.t2 * nslot + b];
    if (e1 < 0 || e2 < 0) continue;
    const double* swa = slot_sw + ((size_t)sp.t1 * nslot + a) * 4;
    const double* swb = slot_sw + ((size_t)sp.t2 * nslot + b) * 4;
    const V3<double> wa = {swa[1], swa[2], swa[3]}, wb = {swb[1], swb[2], swb[3]};
    double Sr = 0, Si = 0, Cr = 0, Ci = 0;
    entry_from_pc(pc, swa[0], wa, swb[0], wb, mikr, miki, c4r, c4i, wantS, doC, Sr, Si, Cr, Ci);
    out.add(e1, e2, wantS, doC, Sr, Si, Cr, Ci);
    // vertex-sharing pairs are stored once (t1 < t2): the two-region rule maps
    // onto itself when the triangles swap roles, so (t2, t1) gives the transpose
    if (cls == 1) out.add(e2, e1, wantS, doC, Sr, Si, Cr, Ci);
  }
}

// Every Sauter–Schwab map is x = xi f(e), y = xi g(e) in the reference
// coordinates of the two triangles (shared vertex at the origin of both), and
// its jacobian is xi^3 J(e). So x - y = xi rho(e), the 1/r of G cancels two
// powers of xi, and a basis monomial m(x, y) of degree d carries xi^d. For
// each (region, e1, e2, e3) a lane therefore forms rho and the monomials once
// and sums the kernel over the Gauss nodes of xi in three radial sums (xi^0,
// xi^1, xi^2); the same quadrature points and weights as the direct form.
// The float64 monomial moments of one ordered touching pair, summed over the
// warp (every lane gets them), with the pair's parametrisation: corners Q1, Q2
// relative to each centroid (shared vertices first), edge vectors and D.
struct SingGeom {
  V3<double> Q1[3], Q2[3], ea, eb, ec, ed, D;
};

__device__ __forceinline__ void sing_pair_moments(const TriD& A, const TriD& B, const SingPair& sp, double kr,
                                                  double ki, bool doC, const Rules& rl, int lane, SingGeom& gm,
                                                  double* MG, double* Mg) {
  const int cls = sp.cls;
  V3<double>* Q1 = gm.Q1;
  V3<double>* Q2 = gm.Q2;
  for (int a = 0; a < 3; ++a) {
    Q1[a] = {A.off[sp.o1[a]][0], A.off[sp.o1[a]][1], A.off[sp.o1[a]][2]};
    Q2[a] = {B.off[sp.o2[a]][0], B.off[sp.o2[a]][1], B.off[sp.o2[a]][2]};
  }
  gm.ea = {Q1[1].x - Q1[0].x, Q1[1].y - Q1[0].y, Q1[1].z - Q1[0].z};
  gm.eb = {Q1[2].x - Q1[1].x, Q1[2].y - Q1[1].y, Q1[2].z - Q1[1].z};
  gm.ec = {Q2[1].x - Q2[0].x, Q2[1].y - Q2[0].y, Q2[1].z - Q2[0].z};
  gm.ed = {Q2[2].x - Q2[1].x, Q2[2].y - Q2[1].y, Q2[2].z - Q2[1].z};
  gm.D = {A.c[0] - B.c[0], A.c[1] - B.c[1], A.c[2] - B.c[2]};
  const V3<double> ea = gm.ea, eb = gm.eb, ec = gm.ec, ed = gm.ed;
  const double scale = 4.0 * A.area * B.area;
  const int ng = rl.ng, nreg = (cls == 3 ? 6 : (cls == 2 ? 5 : 2));
  const int ng2 = ng * ng, ng3 = ng2 * ng;
  constexpr double INV_4PI = 0.25 / 3.14159265358979323846;
  // monomial moments sum K w m(x, y), m in {1, x0, x1, y0, y1, x0 y0, x0 y1,
  // x1 y0, x1 y1} (reference coordinates), K = G and g; (re, im) pairs
#pragma unroll
  for (int q = 0; q < 18; ++q) MG[q] = Mg[q] = 0.0;
  for (int idx = lane; idx < nreg * ng3; idx += 32) {
    const int r = idx / ng3;
    int rem = idx - r * ng3;
    const int a1 = rem / ng2;
    rem -= a1 * ng2;
    const int a2 = rem / ng, a3 = rem - a2 * ng;
    double xh[2], yh[2], jac;
    ss_map(cls, r, 1.0, rl.gx[a1], rl.gx[a2], rl.gx[a3], xh, yh, jac);
    // x - y at xi = 1; the shared vertex cancels exactly
    const V3<double> dr = {xh[0] * ea.x + xh[1] * eb.x - yh[0] * ec.x - yh[1] * ed.x,
                           xh[0] * ea.y + xh[1] * eb.y - yh[0] * ec.y - yh[1] * ed.y,
                           xh[0] * ea.z + xh[1] * eb.z - yh[0] * ec.z - yh[1] * ed.z};
    const double rho = sqrt(dot3(dr, dr));
    const double irho = 1.0 / rho;
    const double We = rl.gw[a1] * rl.gw[a2] * rl.gw[a3] * jac * scale;
    double SG[6] = {0, 0, 0, 0, 0, 0}, Sg[6] = {0, 0, 0, 0, 0, 0};  // (re, im) for xi^0, xi^1, xi^2
    if (ng == 4)
      radial_sums<4>(rl.gx, rl.gw, 4, rho, kr, ki, doC, SG, Sg);  // unrolled: four independent chains
    else
      radial_sums<0>(rl.gx, rl.gw, ng, rho, kr, ki, doC, SG, Sg);
    const double cG = We * irho * INV_4PI, cg = cG * irho * irho;
    const double mono[9] = {1.0, xh[0], xh[1], yh[0], yh[1], xh[0] * yh[0], xh[0] * yh[1], xh[1] * yh[0],
                            xh[1] * yh[1]};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int d = k == 0 ? 0 : (k < 5 ? 2 : 4);  // radial sum of the monomial's degree
      const double fG = cG * mono[k], fg = cg * mono[k];
      MG[2 * k] = fma(fG, SG[d], MG[2 * k]);
      MG[2 * k + 1] = fma(fG, SG[d + 1], MG[2 * k + 1]);
      if (doC) {
        Mg[2 * k] = fma(fg, Sg[d], Mg[2 * k]);
        Mg[2 * k + 1] = fma(fg, Sg[d + 1], Mg[2 * k + 1]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 18; ++q) {
    double v = MG[q], u = Mg[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v += __shfl_xor_sync(0xffffffffu, v, o);
      u += __shfl_xor_sync(0xffffffffu, u, o);
    }
    MG[q] = v;
    Mg[q] = u;
  }
}

template <typename RO>
__global__ void __launch_bounds__(128) singular_kernel(
    const TriD* __restrict__ tri, const SingPair* __restrict__ pairs, int64_t np,
    const int* __restrict__ slot_edge, const double* __restrict__ slot_sw, int nslot, double kr,
    double ki, double mikr, double miki, double c4r, double c4i, bool wantS, bool wantC,
    Rules rl, Sink<RO> out) {
  const int lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (p >= np) return;
  const SingPair sp = pairs[p];
  const TriD A = tri[sp.t1];
  const TriD B = tri[sp.t2];
  const bool doC = wantC && sp.cls != 3;  // flat identical panels: C vanishes
  SingGeom gm;
  double MG[18], Mg[18];
  sing_pair_moments(A, B, sp, kr, ki, doC, rl, lane, gm, MG, Mg);
  sing_emit(MG, Mg, gm.Q1, gm.Q2, gm.ea, gm.eb, gm.ec, gm.ed, gm.D, sp, slot_edge, slot_sw, nslot, mikr, miki, c4r,
            c4i, wantS, doC, lane, 32, out);
}

// ---------------------------------------------------------------------------
// A4 with float32 output: one lane per pair, and the kernel split into a
// static and a dynamic part,
//   G = 1/(4 pi r) + (e^{ikr} - 1)/(4 pi r),
//   g = -1/(4 pi r^3) + ((ikr - 1) e^{ikr} + 1)/(4 pi r^3).
// The static parts carry the singularity and, for g, the large moments that
// cancel when they are combined into entries: they are summed in float64, and
// their radial sums are the rule's own sums of xi^d (no transcendental
// function). The dynamic parts are smooth (O(kr) and O((kr)^2) relative to
// the static ones); they are evaluated in float32 with relative accuracy
// (series of e^z - 1 - z for |z| <= 2) and summed in float32 per region, then
// in float64. Both use the same quadrature points and weights as the float64
// kernel, whose result this reproduces to float32 output accuracy.
// ---------------------------------------------------------------------------
struct SsPt {                      // one (region, e1, e2, e3) direction at xi = 1, float pairs hi + lo
  float x0h, x0l, x1h, x1l;        // reference coordinates of x
  float y0h, y0l, y1h, y1l;        // and of y
  float mh[4], ml[4];              // x0 y0, x0 y1, x1 y0, x1 y1
  float wh, wl;                    // gw(e1) gw(e2) gw(e3) J(e)
};

// Double-float arithmetic (a value is h + l, |l| <= ulp(h) / 2) on the float32
// pipes, from the error-free transformations: TwoProd by fused multiply-add
// and Knuth's TwoSum. The rounded intrinsics keep the compiler from contracting
// or reassociating them.
struct DF { float h, l; };
__device__ __forceinline__ DF df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_quick(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  DF p = df_two_prod(a.h, b.h);
  p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
  return df_quick(p.h, p.l);
}
// the low parts added without a second TwoSum: relative error about 2^-46 of
// |a| + |b| (the terms summed here are of one sign, or their cancellation is
// bounded by the quadrature geometry)
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = df_two_sum(a.h, b.h);
  s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return df_quick(s.h, s.l);
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.h, -a.l}; }
__device__ __forceinline__ DF df_of(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_val(DF a) { return (double)a.h + (double)a.l; }

struct SsRadial {
  double sG[3], sg[3];             // sum_j w_j xi_j^{2+d}, -sum_j w_j xi_j^d (d = 0, 1, 2)
  float xi[16], wG[16][3], wg[16][3];
  int ng;
};

// v = e^z - 1 - z in float32 with relative accuracy. |z| <= 2: Taylor series
// z^2 sum_{m=0..12} z^m / (m + 2)!, the first omitted term below 2e-8 |v|;
// otherwise e^z from expf and sincosf (|v| > 1 there).
__device__ __forceinline__ void expm1mz_f32(float zr, float zi, float& vr, float& vi) {
  if (zr * zr + zi * zi <= 4.0f) {
    constexpr float c[13] = {1.0f / 2, 1.0f / 6, 1.0f / 24, 1.0f / 120, 1.0f / 720, 1.0f / 5040, 1.0f / 40320,
                             1.0f / 362880, 1.0f / 3628800, 1.0f / 39916800, 1.0f / 479001600,
                             1.0f / 6227020800.0f, 1.0f / 87178291200.0f};
    float pr = c[12], pi = 0.0f;
#pragma unroll
    for (int m = 11; m >= 0; --m) {
      const float tr = fmaf(pr, zr, fmaf(-pi, zi, c[m]));
      pi = fmaf(pr, zi, pi * zr);
      pr = tr;
    }
    const float z2r = (zr - zi) * (zr + zi), z2i = 2.0f * zr * zi;
    vr = fmaf(z2r, pr, -z2i * pi);
    vi = fmaf(z2r, pi, z2i * pr);
  } else {
    const float e = expf(zr);
    float sn, cs;
    sincosf(zi, &sn, &cs);
    vr = fmaf(e, cs, -1.0f) - zr;
    vi = fmaf(e, sn, -zi);
  }
}

// dynamic radial sums over the Gauss nodes xi_j (r = xi_j rho, z = ikr):
//   SG_d += w_j xi_j^{2+d} (e^z - 1),  Sg_d += w_j xi_j^d ((z - 1) e^z + 1)
template <int NG>
__device__ __forceinline__ void dyn_radial(const SsRadial& rs, float rho, float kr, float ki, bool doC, float* SG,
                                           float* Sg) {
#pragma unroll
  for (int j = 0; j < (NG > 0 ? NG : 16); ++j) {
    if (NG == 0 && j >= rs.ng) break;
    const float t = rho * rs.xi[j];
    const float zr = -ki * t, zi = kr * t;
    float vr, vi;
    expm1mz_f32(zr, zi, vr, vi);
    const float ur = vr + zr, ui = vi + zi;  // e^z - 1
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      SG[2 * d] = fmaf(rs.wG[j][d], ur, SG[2 * d]);
      SG[2 * d + 1] = fmaf(rs.wG[j][d], ui, SG[2 * d + 1]);
    }
    if (doC) {
      // (z - 1) e^z + 1 = z (e^z - 1) - (e^z - 1 - z)
      const float fr = fmaf(zr, ur, -fmaf(zi, ui, vr)), fi = fmaf(zr, ui, fmaf(zi, ur, -vi));
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        Sg[2 * d] = fmaf(rs.wg[j][d], fr, Sg[2 * d]);
        Sg[2 * d + 1] = fmaf(rs.wg[j][d], fi, Sg[2 * d + 1]);
      }
    }
  }
}

template <int NG>
__global__ void __launch_bounds__(128) singular_split_kernel(
    const TriD* __restrict__ tri, const SingPair* __restrict__ pairs, int64_t np,
    const int* __restrict__ slot_edge, const double* __restrict__ slot_sw, int nslot, double kr,
    double ki, double mikr, double miki, double c4r, double c4i, bool wantS, bool wantC,
    const SsPt* __restrict__ tab, SsRadial rs, Sink<float> out, double* __restrict__ stat_out,
    const double* __restrict__ stat_in) {
  // stat_out: store this pair's static sums (TG, Tg) for the space's next
  // wavenumber; stat_in: read them and run the float32 remainder only
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const SingPair sp = pairs[p];
  const int cls = sp.cls;
  const bool doC = wantC && cls != 3;  // flat identical panels: C vanishes
  V3<double> ea, eb, ec, ed;
  {
    const TriD& A = tri[sp.t1];
    const TriD& B = tri[sp.t2];
    const int a0 = sp.o1[0], a1 = sp.o1[1], a2 = sp.o1[2], b0 = sp.o2[0], b1 = sp.o2[1], b2 = sp.o2[2];
    ea = {A.off[a1][0] - A.off[a0][0], A.off[a1][1] - A.off[a0][1], A.off[a1][2] - A.off[a0][2]};
    eb = {A.off[a2][0] - A.off[a1][0], A.off[a2][1] - A.off[a1][1], A.off[a2][2] - A.off[a1][2]};
    ec = {B.off[b1][0] - B.off[b0][0], B.off[b1][1] - B.off[b0][1], B.off[b1][2] - B.off[b0][2]};
    ed = {B.off[b2][0] - B.off[b1][0], B.off[b2][1] - B.off[b1][1], B.off[b2][2] - B.off[b1][2]};
  }
  const int ng = NG > 0 ? NG : rs.ng, ng3 = ng * ng * ng;
  const int nreg = cls == 3 ? 6 : (cls == 2 ? 5 : 2);
  const SsPt* T = tab + (cls == 1 ? 0 : (cls == 2 ? 2 : 7)) * ng3;
  const float fkr = (float)kr, fki = (float)ki;
  // static moments (real: summed in double-float, held in float64) and dynamic
  // moments ((re, im), float32 per region, float64 over regions)
  DF STG[9], STg[9], DG[18], Dg[18];
#pragma unroll
  for (int q = 0; q < 9; ++q) STG[q] = STg[q] = DF{0.0f, 0.0f};
#pragma unroll
  for (int q = 0; q < 18; ++q) DG[q] = Dg[q] = DF{0.0f, 0.0f};
  const V3<float> fa = {(float)ea.x, (float)ea.y, (float)ea.z}, fb = {(float)eb.x, (float)eb.y, (float)eb.z};
  const V3<float> fc = {(float)ec.x, (float)ec.y, (float)ec.z}, fd = {(float)ed.x, (float)ed.y, (float)ed.z};
  // the edge vectors in double-float for the static sums
  DF EA[3], EB[3], EC[3], ED[3];
  if (!stat_in) {
    EA[0] = df_of(ea.x); EA[1] = df_of(ea.y); EA[2] = df_of(ea.z);
    EB[0] = df_of(eb.x); EB[1] = df_of(eb.y); EB[2] = df_of(eb.z);
    EC[0] = df_of(ec.x); EC[1] = df_of(ec.y); EC[2] = df_of(ec.z);
    ED[0] = df_of(ed.x); ED[1] = df_of(ed.y); ED[2] = df_of(ed.z);
  }
  for (int r = 0; r < nreg; ++r) {
    float dG[18], dg[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) dG[q] = dg[q] = 0.0f;
    if (stat_in) {
      // the static sums are known: only the float32 remainder, with x - y in
      // float32 (its rounding near the singular set touches only O((kr)^2) terms)
      for (int q = 0; q < ng3; ++q) {
        const SsPt& e = T[r * ng3 + q];
        const float fx0 = e.x0h, fx1 = e.x1h, fy0 = e.y0h, fy1 = e.y1h;
        const V3<float> dr = {fx0 * fa.x + fx1 * fb.x - fy0 * fc.x - fy1 * fd.x,
                              fx0 * fa.y + fx1 * fb.y - fy0 * fc.y - fy1 * fd.y,
                              fx0 * fa.z + fx1 * fb.z - fy0 * fc.z - fy1 * fd.z};
        const float r2f = dr.x * dr.x + dr.y * dr.y + dr.z * dr.z;
        const float yf = rsqrtf(r2f);
        float SG[6] = {0, 0, 0, 0, 0, 0}, Sg[6] = {0, 0, 0, 0, 0, 0};
        dyn_radial<NG>(rs, r2f * yf, fkr, fki, doC, SG, Sg);
        const float cGf = e.wh * yf, cgf = cGf * yf * yf;
        const float fm[9] = {1.0f, fx0, fx1, fy0, fy1, fx0 * fy0, fx0 * fy1, fx1 * fy0, fx1 * fy1};
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const int d = k == 0 ? 0 : (k < 5 ? 2 : 4);
          const float a = cGf * fm[k];
          dG[2 * k] = fmaf(a, SG[d], dG[2 * k]);
          dG[2 * k + 1] = fmaf(a, SG[d + 1], dG[2 * k + 1]);
          if (doC) {
            const float b = cgf * fm[k];
            dg[2 * k] = fmaf(b, Sg[d], dg[2 * k]);
            dg[2 * k + 1] = fmaf(b, Sg[d + 1], dg[2 * k + 1]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 18; ++q) {
        DG[q] = df_add(DG[q], DF{dG[q], 0.0f});
        if (doC) Dg[q] = df_add(Dg[q], DF{dg[q], 0.0f});
      }
      continue;
    }
    for (int q = 0; q < ng3; ++q) {
      const SsPt& e = T[r * ng3 + q];
      const DF X0{e.x0h, e.x0l}, X1{e.x1h, e.x1l}, Y0{e.y0h, e.y0l}, Y1{e.y1h, e.y1l};
      // x - y at xi = 1 in double-float; the shared vertex cancels exactly
      DF dr[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        DF s = df_mul(X0, EA[c]);
        s = df_add(s, df_mul(X1, EB[c]));
        s = df_add(s, df_neg(df_mul(Y0, EC[c])));
        dr[c] = df_add(s, df_neg(df_mul(Y1, ED[c])));
      }
      const DF r2 = df_add(df_add(df_mul(dr[0], dr[0]), df_mul(dr[1], dr[1])), df_mul(dr[2], dr[2]));
      const float r2f = r2.h;
      float yf;
      DF y;
      if (r2f > 1e-30f && r2f < 1e30f) {
        // float32 seed and one double-float Newton step y <- y + y (1 - r2 y^2) / 2
        // for r2^{-1/2}: relative error about 1.5 e0^2 plus the double-float rounding
        yf = rsqrtf(r2f);
        const DF hh = df_add(DF{1.0f, 0.0f}, df_neg(df_mul(r2, df_two_prod(yf, yf))));
        y = df_add(DF{yf, 0.0f}, df_two_prod(yf, 0.5f * hh.h));
      } else {
        const double yd = 1.0 / sqrt(df_val(r2));
        y = df_of(yd);
        yf = y.h;
      }
      const DF cG = df_mul(DF{e.wh, e.wl}, y);
      const DF mono[9] = {DF{1.0f, 0.0f}, X0, X1, Y0, Y1, DF{e.mh[0], e.ml[0]}, DF{e.mh[1], e.ml[1]},
                          DF{e.mh[2], e.ml[2]}, DF{e.mh[3], e.ml[3]}};
#pragma unroll
      for (int k = 0; k < 9; ++k) STG[k] = df_add(STG[k], df_mul(cG, mono[k]));
      if (doC) {
        const DF cg = df_mul(cG, df_mul(y, y));
#pragma unroll
        for (int k = 0; k < 9; ++k) STg[k] = df_add(STg[k], df_mul(cg, mono[k]));
      }
      // dynamic part in float32
      float SG[6] = {0, 0, 0, 0, 0, 0}, Sg[6] = {0, 0, 0, 0, 0, 0};
      dyn_radial<NG>(rs, r2f * yf, fkr, fki, doC, SG, Sg);
      const float cGf = e.wh * yf, cgf = cGf * yf * yf;
      const float fx0 = e.x0h, fx1 = e.x1h, fy0 = e.y0h, fy1 = e.y1h;
      const float fm[9] = {1.0f, fx0, fx1, fy0, fy1, fx0 * fy0, fx0 * fy1, fx1 * fy0, fx1 * fy1};
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int d = k == 0 ? 0 : (k < 5 ? 2 : 4);
        const float a = cGf * fm[k];
        dG[2 * k] = fmaf(a, SG[d], dG[2 * k]);
        dG[2 * k + 1] = fmaf(a, SG[d + 1], dG[2 * k + 1]);
        if (doC) {
          const float b = cgf * fm[k];
          dg[2 * k] = fmaf(b, Sg[d], dg[2 * k]);
          dg[2 * k + 1] = fmaf(b, Sg[d + 1], dg[2 * k + 1]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 18; ++q) {
      DG[q] = df_add(DG[q], DF{dG[q], 0.0f});
      if (doC) Dg[q] = df_add(Dg[q], DF{dg[q], 0.0f});
    }
  }
  double TG[9], Tg[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    TG[k] = stat_in ? stat_in[p * 18 + k] : df_val(STG[k]);
    Tg[k] = stat_in ? stat_in[p * 18 + 9 + k] : df_val(STg[k]);
  }
  if (stat_out) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      stat_out[p * 18 + k] = TG[k];
      stat_out[p * 18 + 9 + k] = Tg[k];
    }
  }
  const TriD& A = tri[sp.t1];
  const TriD& B = tri[sp.t2];
  V3<double> Q1[3], Q2[3];
  for (int a = 0; a < 3; ++a) {
    Q1[a] = {A.off[sp.o1[a]][0], A.off[sp.o1[a]][1], A.off[sp.o1[a]][2]};
    Q2[a] = {B.off[sp.o2[a]][0], B.off[sp.o2[a]][1], B.off[sp.o2[a]][2]};
  }
  const V3<double> D = {A.c[0] - B.c[0], A.c[1] - B.c[1], A.c[2] - B.c[2]};
  constexpr double INV_4PI = 0.25 / 3.14159265358979323846;
  const double sc = 4.0 * A.area * B.area * INV_4PI;
  double MG[18], Mg[18];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int d = k == 0 ? 0 : (k < 5 ? 1 : 2);
    MG[2 * k] = sc * fma(rs.sG[d], TG[k], df_val(DG[2 * k]));
    MG[2 * k + 1] = sc * df_val(DG[2 * k + 1]);
    Mg[2 * k] = sc * fma(rs.sg[d], Tg[k], df_val(Dg[2 * k]));
    Mg[2 * k + 1] = sc * df_val(Dg[2 * k + 1]);
  }
  sing_emit(MG, Mg, Q1, Q2, ea, eb, ec, ed, D, sp, slot_edge, slot_sw, nslot, mikr, miki, c4r, c4i, wantS, doC, 0,
            1, out);
}

// Host-built table of the Sauter–Schwab directions for ng Gauss points per
// dimension: classes 1, 2, 3 (vertex, edge, identical) at offsets 0, 2 ng^3,
// 7 ng^3, region-major. One copy per (device, ng), kept for the process.
static const SsPt* ss_table(int ng, const double* gx, const double* gw, cudaStream_t st) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, SsPt*> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find({dev, ng});
  if (it != cache.end()) return it->second;
  const int ng3 = ng * ng * ng;
  std::vector<SsPt> h((size_t)13 * ng3);
  const int cls_of[3] = {1, 2, 3}, nreg_of[3] = {2, 5, 6}, off_of[3] = {0, 2, 7};
  for (int c = 0; c < 3; ++c)
    for (int idx = 0; idx < nreg_of[c] * ng3; ++idx) {
      const int r = idx / ng3, a1 = (idx / (ng * ng)) % ng, a2 = (idx / ng) % ng, a3 = idx % ng;
      double xh[2], yh[2], jac;
      ss_map(cls_of[c], r, 1.0, gx[a1], gx[a2], gx[a3], xh, yh, jac);
      SsPt& e = h[(size_t)off_of[c] * ng3 + idx];
      auto split = [](double x, float& hi, float& lo) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
      };
      split(xh[0], e.x0h, e.x0l);
      split(xh[1], e.x1h, e.x1l);
      split(yh[0], e.y0h, e.y0l);
      split(yh[1], e.y1h, e.y1l);
      const double m[4] = {xh[0] * yh[0], xh[0] * yh[1], xh[1] * yh[0], xh[1] * yh[1]};
      for (int k = 0; k < 4; ++k) split(m[k], e.mh[k], e.ml[k]);
      split(gw[a1] * gw[a2] * gw[a3] * jac, e.wh, e.wl);
    }
  SsPt* d = nullptr;
  if (cudaMalloc((void**)&d, h.size() * sizeof(SsPt)) != cudaSuccess) return nullptr;
  if (cudaMemcpyAsync(d, h.data(), h.size() * sizeof(SsPt), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  cache[{dev, ng}] = d;
  return d;
}

static SsRadial ss_radial(const Rules& rl) {
  SsRadial rs{};
  rs.ng = rl.ng;
  for (int j = 0; j < rl.ng; ++j) {
    const double x = rl.gx[j], w = rl.gw[j];
    rs.xi[j] = (float)x;
    for (int d = 0; d < 3; ++d) {
      const double xd = d == 0 ? 1.0 : (d == 1 ? x : x * x);
      rs.sG[d] += w * x * x * xd;
      rs.sg[d] -= w * xd;
      rs.wG[j][d] = (float)(w * x * x * xd);
      rs.wg[j][d] = (float)(w * xd);
    }
  }
  return rs;
}

// ---------------------------------------------------------------------------
// A6: Gram matrix G_ij = <BC_j, RWG_i> = int BC_j . (n x RWG_i). On a
// barycentric triangle tau both are sigma (x - c_tau) + w with constant
// sigma, w; since int_tau (x - c_tau) = 0 and (x-c).(n x (x-c)) = 0, the
// integral is exactly |tau| w_BC . (n x w_RWG).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t csr_find(const int64_t* rowptr, const int* col, int row, int c) {
  int64_t lo = rowptr[row], hi = rowptr[row + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) >> 1;
    if (col[mid] == c) return mid;
    if (col[mid] < c) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

__global__ void gram_kernel(const TriD* __restrict__ btri, const int* __restrict__ bslot_edge,
                            const double* __restrict__ bslot_sw, int nslot,
                            const int* __restrict__ parent, const TriD* __restrict__ ptri,
                            const int* __restrict__ pslot_edge, const double* __restrict__ pslot_sw,
                            int64_t ntau, const int64_t* rowptr, const int* col,
                            const int64_t* rowptrT, const int* colT, double* vals, double* valsT) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ntau * nslot) return;
  const int64_t tau = q / nslot;
  const int sl = (int)(q % nslot);
  const int j = bslot_edge[q];
  if (j < 0) return;
  const TriD T = btri[tau];
  const double* swj = bslot_sw + q * 4;
  const V3<double> wj = {swj[1], swj[2], swj[3]};
  V3<double> u = {T.off[1][0] - T.off[0][0], T.off[1][1] - T.off[0][1], T.off[1][2] - T.off[0][2]};
  V3<double> v = {T.off[2][0] - T.off[0][0], T.off[2][1] - T.off[0][1], T.off[2][2] - T.off[0][2]};
  V3<double> n = cross3(u, v);
  const double nn = sqrt(dot3(n, n));
  n = {n.x / nn, n.y / nn, n.z / nn};
  const int t = parent[tau];
  const TriD P = ptri[t];
  const V3<double> dc = {T.c[0] - P.c[0], T.c[1] - P.c[1], T.c[2] - P.c[2]};
  for (int a = 0; a < 3; ++a) {
    const int i = pslot_edge[3 * t + a];
    const double* swi = pslot_sw + (3 * t + a) * 4;
    const V3<double> wi = {swi[1] + swi[0] * dc.x, swi[2] + swi[0] * dc.y, swi[3] + swi[0] * dc.z};
    const double val = T.area * dot3(wj, cross3(n, wi));
    const int64_t k = csr_find(rowptr, col, i, j);
    if (k >= 0) atomicAdd(vals + k, val);
    const int64_t kt = csr_find(rowptrT, colT, j, i);
    if (kt >= 0) atomicAdd(valsT + kt, val);
  }
  (void)sl;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename R>
static void wave_scalars(double kr, double ki, R& mikr, R& miki, R& c4r, R& c4i) {
  // -ik and 4i/k
  mikr = (R)ki;
  miki = (R)(-kr);
  const double k2 = kr * kr + ki * ki;
  c4r = (R)(4.0 * ki / k2);
  c4i = (R)(4.0 * kr / k2);
}

template <typename R>
static Sink<R> make_sink(const AssembleArgs& a) {
  Sink<R> s;
  s.S = reinterpret_cast<R*>(a.S);
  s.C = reinterpret_cast<R*>(a.C);
  s.off = a.row_off;
  s.ld = (a.format == CAL_DENSE) ? a.ld : 0;
  s.rowptr = a.rowptr;
  s.col = a.col;
  return s;
}

template <typename R>
static int rwg_regular_t(const AssembleArgs& a) {
  const Space& s = *a.sp;
  const int64_t t0 = a.scat < 0 ? 0 : s.tri_off[a.scat];
  const int64_t ntr = (a.scat < 0 ? s.ntri : s.tri_off[a.scat + 1]) - t0;
  const int64_t nb = (ntr + 15) / 16;
  if (nb > 65535) return fail(CAL_EINVAL, "too many triangles for the regular-pair grid (%lld)", (long long)ntr);
  R mikr, miki, c4r, c4i;
  wave_scalars(a.kr, a.ki, mikr, miki, c4r, c4i);
  dim3 grid((unsigned)nb, (unsigned)nb), block(16, 16);
  const Sink<R> out = make_sink<R>(a);
  const bool wS = a.want & 1, wC = a.want & 2;
  const typename TriOf<R>::T* tri;
  const R* sw;
  if constexpr (sizeof(R) == 4) { tri = s.d_triF; sw = s.d_slot_swf; }
  else { tri = s.d_triD; sw = s.d_slot_swd; }
  // algorithmic work: unordered non-touching pairs x rule points squared
  int64_t nsing = 0;  // ordered touching pairs (vertex pairs are listed once)
  for (int d = (a.scat < 0 ? 0 : a.scat); d < (a.scat < 0 ? (int)s.sing.size() : a.scat + 1); ++d)
    for (const SingPair& q : s.sing[d]) nsing += q.cls == 1 ? 2 : 1;
  const double units = ((double)ntr * (ntr - 1) / 2 - (double)(nsing - ntr) / 2) * a.nreg * a.nreg;
  const int tok = prof_begin(a.stream, "rwg_regular", units);
  // by class the evaluations depend on the geometry: counted on the device
  unsigned long long* cnt = a.nreg == 0 ? prof_counter(tok, a.stream) : nullptr;
  if constexpr (sizeof(R) == 4) {
    // float32: the staged tile with a shared edge x edge accumulator
    constexpr int NSP = RULE_POINTS_ALL;
    const int tile = a.nreg == 6 ? (int)sizeof(RwgTile<6>) : (a.nreg == 1 ? (int)sizeof(RwgTile<1>) : (int)sizeof(RwgTile<NSP>));
    const int smem = tile + 4 * RWG_TILE_SLOTS * RWG_TILE_SLOTS * (int)sizeof(float) + (6 * RWG_TILE_SLOTS + 2) * (int)sizeof(int);
    auto fk = a.nreg == 6 ? rwg_regular_f32_kernel<6> : (a.nreg == 1 ? rwg_regular_f32_kernel<1> : rwg_regular_f32_kernel<0>);
    if (int rc = ensure_dyn_smem((const void*)fk, smem)) {
      prof_end(a.stream, tok);
      return rc;
    }
    fk<<<grid, block, smem, a.stream>>>(tri, s.d_slot_edge, sw, t0, ntr, (float)a.kr, (float)a.ki, mikr, miki, c4r,
                                        c4i, wS, wC, g_rules, out, cnt);
  } else {
    auto kern = a.nreg == 6 ? rwg_regular_kernel<R, 6> : (a.nreg == 1 ? rwg_regular_kernel<R, 1> : rwg_regular_kernel<R, 0>);
    kern<<<grid, block, 0, a.stream>>>(tri, s.d_slot_edge, sw, t0, ntr, (R)a.kr, (R)a.ki, mikr, miki, c4r, c4i, wS, wC,
                                       g_rules, out, cnt);
  }
  prof_end(a.stream, tok);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

int launch_rwg_regular(const AssembleArgs& a) {
  return a.precision == CAL_FP32 ? rwg_regular_t<float>(a) : rwg_regular_t<double>(a);
}

struct BcTiles {
  int* d_cells = nullptr;
  int2* d_tiles = nullptr;
};

template <typename R>
static int bc_regular_t(const AssembleArgs& a, const BcUnit* units, int64_t nunits, const int* wlist, int max_cell,
                        int n_sm, double work) {
  const Space& s = *a.sp;
  R mikr, miki, c4r, c4i;
  wave_scalars(a.kr, a.ki, mikr, miki, c4r, c4i);
  const Sink<R> out = make_sink<R>(a);
  const bool wS = a.want & 1, wC = a.want & 2;
  if (nunits == 0) return CAL_OK;
  // test-cell triangles are processed in chunks so that any valence fits
  auto smem_for = [&](int ch) {
    const size_t reals = (size_t)ch * max_cell * 36 + (size_t)ch * s.nslot * BC_RED + (size_t)s.nslot * s.nslot * 4;
    const size_t ns = a.nreg > 0 ? (size_t)a.nreg : (size_t)RULE_POINTS_ALL;
    const size_t staged = 2 * (size_t)max_cell * ns * 4 * sizeof(R) +           // points
                          2 * (size_t)max_cell * s.nslot * 4 * sizeof(R) +     // slot coefficients
                          2 * (size_t)max_cell * sizeof(Cent<R>) +             // centroids
                          2 * (size_t)max_cell * 3 * sizeof(int);              // vertex ids
    return ((reals * sizeof(R) + 15) / 16) * 16 + staged + 64;
  };
  int chunk = max_cell;
  while (chunk > 1 && smem_for(chunk) > 56 * 1024) --chunk;
  const size_t smem = smem_for(chunk);
  if (smem > 227 * 1024) return fail(CAL_EINVAL, "dual cell too large for the tile kernel (%d triangles)", max_cell);
  const typename TriOf<R>::T* tri;
  const R* sw;
  if constexpr (sizeof(R) == 4) { tri = s.d_triF; sw = s.d_slot_swf; }
  else { tri = s.d_triD; sw = s.d_slot_swd; }
  // cell-ordered copies of the staged data (per launch: the points depend on the rule)
  const int64_t nct = (int64_t)s.cell_tri.size();
  const int nreg = a.nreg;
  CellData<R> cd{};
  const int nsp = nreg > 0 ? nreg : RULE_POINTS_ALL;  // staged points per triangle
  const size_t b_pts = (size_t)nct * nsp * sizeof(P4<R>), b_sw = (size_t)nct * s.nslot * sizeof(P4<R>);
  const size_t b_cen = (size_t)nct * sizeof(Cent<R>), b_vid = (size_t)nct * 3 * sizeof(int);
  auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
  unsigned char* buf = nullptr;
  CAL_TRY_CUDA(cudaMallocAsync((void**)&buf, r256(b_pts) + r256(b_sw) + r256(b_cen) + r256(b_vid), a.stream));
  cd.pts = reinterpret_cast<P4<R>*>(buf);
  cd.sw = reinterpret_cast<P4<R>*>(buf + r256(b_pts));
  cd.cen = reinterpret_cast<Cent<R>*>(buf + r256(b_pts) + r256(b_sw));
  cd.vid = reinterpret_cast<int*>(buf + r256(b_pts) + r256(b_sw) + r256(b_cen));
  auto prep = nreg == 6 ? bc_cell_prep_kernel<R, 6> : (nreg == 1 ? bc_cell_prep_kernel<R, 1> : bc_cell_prep_kernel<R, 0>);
  prep<<<(unsigned)((nct * nsp + 255) / 256), 256, 0, a.stream>>>(tri, sw, s.nslot, s.d_cell_tri, nct, g_rules, cd);
  note_launch();
  if constexpr (sizeof(R) == 4) {
    if (bc_owner_width(s, a.precision, max_cell, max_cell) > 0) {
      // one thread per (test triangle, trial cell); units sized by bc_owner_width
      constexpr int OT = BC_OWNER_TT;
      auto okern = (wS && wC) ? (nreg == 6 ? bc_owner_kernel<6, OT, true>
                                           : (nreg == 1 ? bc_owner_kernel<1, OT, true> : bc_owner_kernel<0, OT, true>))
                              : (nreg == 6 ? bc_owner_kernel<6, OT, false>
                                           : (nreg == 1 ? bc_owner_kernel<1, OT, false> : bc_owner_kernel<0, OT, false>));
      auto pack = nreg == 6 ? bc_trial_pack_kernel<6> : (nreg == 1 ? bc_trial_pack_kernel<1> : bc_trial_pack_kernel<0>);
      const int rw = nreg == 6 ? owner_rec_words<6>() : (nreg == 1 ? owner_rec_words<1>() : owner_rec_words<0>());
      float4* trec = nullptr;
      if (cudaMallocAsync((void**)&trec, (size_t)std::max<int64_t>(nct, 1) * rw * sizeof(float4), a.stream) !=
          cudaSuccess) {
        cudaFreeAsync(buf, a.stream);
        return fail(CAL_ENOMEM, "bc owner kernel: cannot allocate the trial records");
      }
      pack<<<(unsigned)((nct * rw + 255) / 256), 256, 0, a.stream>>>(cd, s.nslot, nct, s.d_triF, s.d_cell_tri, trec);
      note_launch();
      const int nsp_o = nreg > 0 ? nreg : RULE_POINTS_ALL;
      const size_t osmem = owner_region_bytes(OT, rw, nsp_o, max_cell) +
                           (size_t)max_cell * s.nslot * sizeof(P4<float>) + (size_t)max_cell * sizeof(Cent<float>) +
                           (size_t)max_cell * 3 * sizeof(int) + 3 * (size_t)OT * sizeof(int) +
                           (size_t)OT * BC_OWN_SLOTS * sizeof(float) +
                           // slot counts, slot edges, test edges, next trial cells, next descriptor
                           (size_t)OT * sizeof(int) + (size_t)OT * BC_OWN_SLOTS * sizeof(int) +
                           BC_OWN_SLOTS * sizeof(int) + (size_t)OT * sizeof(int) + 2 * sizeof(BcUnit) + 16 + 64;
      int rc = ensure_dyn_smem((const void*)okern, (int)osmem);
      // three CTAs of ~72 KB need the largest shared-memory carveout
      if (!rc && cudaFuncSetAttribute((const void*)okern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        rc = fail(CAL_ECUDA, "bc owner kernel: carveout preference failed");
      // CTAs per SM from the kernel's registers, shared memory and tensor-memory
      // columns. The runtime's occupancy query answers 1 for this kernel
      // (measured, with 3 fitting), which would leave a third of the SM idle.
      int per_sm = 0;
      if (!rc) {
        cudaFuncAttributes fa{};
        int dev = 0, regs_sm = 0, smem_sm = 0, smem_res = 0;
        if (cudaFuncGetAttributes(&fa, (const void*)okern) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_res, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
          rc = fail(CAL_ECUDA, "bc owner kernel: attribute query failed");
        } else {
          const int regs_cta = ((fa.numRegs + 7) / 8) * 8 * OT;  // allocated per warp in units of 8 x 32
          const size_t smem_cta = osmem + fa.sharedSizeBytes + smem_res;
          per_sm = std::min({regs_sm / std::max(1, regs_cta), (int)(smem_sm / smem_cta), 512 / BC_OWN_TMEM_COLS});
        }
      }
      if (!rc) {
        const int64_t grid = std::min<int64_t>(nunits, (int64_t)std::max(1, per_sm) * n_sm * 2);
        const int tok = prof_begin(a.stream, "bc_tile", work);
        unsigned long long* cnt = nreg == 0 ? prof_counter(tok, a.stream) : nullptr;
        okern<<<(unsigned)grid, OT, osmem, a.stream>>>(cd, s.nslot, s.d_cell_tri_ptr, s.d_cell_edge_ptr, s.d_cell_edge,
                                                      units, nunits, wlist, trec, s.d_cell_slot_s, (float)a.kr,
                                                      (float)a.ki, mikr, miki, c4r, c4i, wS, wC, out, max_cell, cnt);
        prof_end(a.stream, tok);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) rc = fail(CAL_ECUDA, "bc owner kernel launch failed");
      }
      cudaFreeAsync(trec, a.stream);
      cudaFreeAsync(buf, a.stream);
      return rc;
    }
  }
  constexpr int TT = 128;
  auto kern = nreg == 6 ? bc_tile_kernel<R, 6, TT> : (nreg == 1 ? bc_tile_kernel<R, 1, TT> : bc_tile_kernel<R, 0, TT>);
  int rc = ensure_dyn_smem((const void*)kern, (int)smem);
  int per_sm = 0;
  if (!rc && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TT, smem) != cudaSuccess)
    rc = fail(CAL_ECUDA, "bc tile kernel: occupancy query failed");
  if (!rc) {
    const int64_t grid = std::min<int64_t>(nunits, (int64_t)std::max(1, per_sm) * n_sm * 2);
    const int tok = prof_begin(a.stream, "bc_tile", work);
    unsigned long long* cnt = nreg == 0 ? prof_counter(tok, a.stream) : nullptr;
    kern<<<(unsigned)grid, TT, smem, a.stream>>>(cd, s.nslot, s.d_cell_tri_ptr, s.d_cell_edge_ptr, s.d_cell_edge,
                                                units, nunits, wlist, (R)a.kr, (R)a.ki, mikr, miki, c4r, c4i, wS, wC,
                                                out, max_cell, chunk, cnt);
    prof_end(a.stream, tok);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) rc = fail(CAL_ECUDA, "bc tile kernel launch failed");
  }
  cudaFreeAsync(buf, a.stream);  // stream-ordered: after the kernel
  return rc;
}

int launch_bc_regular_units(const AssembleArgs& a, const void* units, int64_t nunits, const int* wlist, int max_cell,
                            int n_sm, double work) {
  const BcUnit* u = reinterpret_cast<const BcUnit*>(units);
  return a.precision == CAL_FP32 ? bc_regular_t<float>(a, u, nunits, wlist, max_cell, n_sm, work)
                                 : bc_regular_t<double>(a, u, nunits, wlist, max_cell, n_sm, work);
}

int launch_singular(const AssembleArgs& a) {
  const Space& s = *a.sp;
  double mikr, miki, c4r, c4i;
  wave_scalars(a.kr, a.ki, mikr, miki, c4r, c4i);
  const bool wS = a.want & 1, wC = a.want & 2;
  const int d0 = a.scat < 0 ? 0 : a.scat;
  const int d1 = a.scat < 0 ? (int)s.sing.size() : a.scat + 1;
  for (int d = d0; d < d1; ++d) {
    const int64_t np = (int64_t)s.sing[d].size();
    if (np == 0) continue;
    const unsigned grid = (unsigned)((np + 3) / 4);
    double regions = 0;
    for (const SingPair& q : s.sing[d]) regions += (q.cls == 3 ? 6 : (q.cls == 2 ? 5 : 2));
    const double ng2 = (double)a.nsing * a.nsing;
    const int tok = prof_begin(a.stream, "singular", regions * ng2 * ng2);
    if (a.sing32) {
      RulesF rf{};
      for (int q = 0; q < 16; ++q) { rf.gx[q] = (float)g_rules.gx[q]; rf.gw[q] = (float)g_rules.gw[q]; }
      rf.ng = g_rules.ng;
      float fmr, fmi, f4r, f4i;
      wave_scalars(a.kr, a.ki, fmr, fmi, f4r, f4i);
      singular_kernel_f32<<<grid, 128, 0, a.stream>>>(s.d_triF, s.d_sing[d], np, s.d_slot_edge, s.d_slot_swf,
                                                      s.nslot, (float)a.kr, (float)a.ki, fmr, fmi, f4r, f4i,
                                                      wS, wC, rf, make_sink<float>(a));
    } else if (a.precision == CAL_FP32) {
      const SsPt* tab = ss_table(g_rules.ng, g_rules.gx, g_rules.gw, a.stream);
      if (!tab) {
        prof_end(a.stream, tok);
        return fail(CAL_ECUDA, "singular rule table: device allocation failed");
      }
      const SsRadial rs = ss_radial(g_rules);
      const unsigned g1 = (unsigned)((np + 127) / 128);
      // the static sums depend on the geometry and the Gauss order only: the
      // first launch that computes all of them keeps them, later ones read them
      std::lock_guard<std::mutex> lk(s.static_mu);
      if (s.sing_static.size() != s.sing.size()) s.sing_static.resize(s.sing.size());
      Space::StaticSums& st = s.sing_static[d];
      double* sout = nullptr;
      const double* sin = nullptr;
      if (st.ready && st.ng == g_rules.ng) {
        if (cudaStreamWaitEvent(a.stream, st.done, 0) != cudaSuccess) {
          prof_end(a.stream, tok);
          return fail(CAL_ECUDA, "singular static sums: stream wait failed");
        }
        sin = st.buf;
      } else if (!st.buf && wC) {
        if (dalloc((void**)&st.buf, (size_t)np * 18 * sizeof(double), a.stream) == cudaSuccess &&
            cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming) == cudaSuccess) {
          st.ng = g_rules.ng;
          sout = st.buf;
        } else {
          cudaGetLastError();  // no cache: this launch runs in full
        }
      }
      if (g_rules.ng == 4)
        singular_split_kernel<4><<<g1, 128, 0, a.stream>>>(s.d_triD, s.d_sing[d], np, s.d_slot_edge, s.d_slot_swd,
                                                           s.nslot, a.kr, a.ki, mikr, miki, c4r, c4i, wS, wC, tab,
                                                           rs, make_sink<float>(a), sout, sin);
      else
        singular_split_kernel<0><<<g1, 128, 0, a.stream>>>(s.d_triD, s.d_sing[d], np, s.d_slot_edge, s.d_slot_swd,
                                                           s.nslot, a.kr, a.ki, mikr, miki, c4r, c4i, wS, wC, tab,
                                                           rs, make_sink<float>(a), sout, sin);
      if (sout && cudaPeekAtLastError() == cudaSuccess && cudaEventRecord(st.done, a.stream) == cudaSuccess)
        st.ready = true;
    } else {
      singular_kernel<double><<<grid, 128, 0, a.stream>>>(s.d_triD, s.d_sing[d], np, s.d_slot_edge,
                                                          s.d_slot_swd, s.nslot, a.kr, a.ki, mikr, miki,
                                                          c4r, c4i, wS, wC, g_rules, make_sink<double>(a));
    }
    prof_end(a.stream, tok);
    note_launch();
    CAL_TRY_CUDA(cudaGetLastError());
  }
  return CAL_OK;
}

int launch_gram(const Space& rwg, const Space& bc, const int64_t* rowptr, const int* col,
                const int64_t* rowptrT, const int* colT, double* vals, double* valsT,
                cudaStream_t stream) {
  int* d_parent = nullptr;
  CAL_TRY_CUDA(cudaMallocAsync((void**)&d_parent, bc.parent.size() * sizeof(int), stream));
  CAL_TRY_CUDA(cudaMemcpyAsync(d_parent, bc.parent.data(), bc.parent.size() * sizeof(int),
                               cudaMemcpyHostToDevice, stream));
  const int64_t n = bc.ntri * bc.nslot;
  gram_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(
      bc.d_triD, bc.d_slot_edge, bc.d_slot_swd, bc.nslot, d_parent, rwg.d_triD, rwg.d_slot_edge,
      rwg.d_slot_swd, bc.ntri, rowptr, col, rowptrT, colT, vals, valsT);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  CAL_TRY_CUDA(cudaFreeAsync(d_parent, stream));
  return CAL_OK;
}

template <typename R, typename VT, typename AT>
static int rwg_free_t(const Space& s, int scat, double kr, double ki, int nreg, const VT* x, VT* y, int64_t n,
                      int nrhs, double ar, double ai, double br, double bi, cudaStream_t st) {
  const int64_t t0 = scat < 0 ? 0 : s.tri_off[scat];
  const int64_t ntr = (scat < 0 ? s.ntri : s.tri_off[scat + 1]) - t0;
  const int64_t nb = (ntr + 15) / 16;
  if (nb > 65535) return fail(CAL_EINVAL, "too many triangles for the regular-pair grid (%lld)", (long long)ntr);
  if (ntr < 2) return CAL_OK;
  R mikr, miki, c4r, c4i;
  wave_scalars(kr, ki, mikr, miki, c4r, c4i);
  const typename TriOf<R>::T* tri;
  const R* sw;
  if constexpr (sizeof(R) == 4) { tri = s.d_triF; sw = s.d_slot_swf; }
  else { tri = s.d_triD; sw = s.d_slot_swd; }
  int64_t nsing = 0;
  for (int d = (scat < 0 ? 0 : scat); d < (scat < 0 ? (int)s.sing.size() : scat + 1); ++d)
    for (const SingPair& q : s.sing[d]) nsing += q.cls == 1 ? 2 : 1;
  const double units = ((double)ntr * (ntr - 1) / 2 - (double)(nsing - ntr) / 2) * nreg * nreg;
  dim3 grid((unsigned)nb, (unsigned)nb), block(16, 16);
  if constexpr (sizeof(R) == 4 && sizeof(VT) == 8) {
    // float32 vectors: the staged, packed-pair kernel
    constexpr int NSP = RULE_POINTS_ALL;  // the largest staging (class rules)
    for (int r0 = 0; r0 < nrhs; r0 += 32) {
      const int nr = std::min(32, nrhs - r0);
      const int tile = nreg == 6 ? (int)sizeof(RwgTile<6>) : (nreg == 1 ? (int)sizeof(RwgTile<1>) : (int)sizeof(RwgTile<NSP>));
      const int smem = tile + 2 * 16 * 3 * 2 * nr * 2 * 4;
      auto kern = nreg == 6 ? rwg_free_f32_kernel<6> : (nreg == 1 ? rwg_free_f32_kernel<1> : rwg_free_f32_kernel<0>);
      if (int rc = ensure_dyn_smem((const void*)kern, smem)) return rc;
      const int tok = prof_begin(st, "rwg_free", units * nr);
      unsigned long long* cnt = nreg == 0 ? prof_counter(tok, st) : nullptr;
      kern<<<grid, block, smem, st>>>(tri, s.d_slot_edge, sw, t0, ntr, (float)kr, (float)ki, (float)mikr,
                                      (float)miki, (float)c4r, (float)c4i, g_rules,
                                      reinterpret_cast<const float2*>(x) + (int64_t)r0 * 2 * n,
                                      reinterpret_cast<float2*>(y) + (int64_t)r0 * 2 * n, n, nr, (float)ar,
                                      (float)ai, (float)br, (float)bi, cnt);
      prof_end(st, tok);
      note_launch();
      CAL_TRY_CUDA(cudaGetLastError());
    }
    return CAL_OK;
  } else {
    for (int r0 = 0; r0 < nrhs; r0 += 32) {
      const int nr = std::min(32, nrhs - r0);
      const int smem = 2 * 16 * 3 * 2 * nr * 2 * (int)sizeof(AT);
      auto kern = nreg == 6 ? rwg_free_kernel<R, 6, VT, AT>
                            : (nreg == 1 ? rwg_free_kernel<R, 1, VT, AT> : rwg_free_kernel<R, 0, VT, AT>);
      if (int rc = ensure_dyn_smem((const void*)kern, smem)) return rc;
      const int tok = prof_begin(st, "rwg_free", units * nr);
      unsigned long long* cnt = nreg == 0 ? prof_counter(tok, st) : nullptr;
      kern<<<grid, block, smem, st>>>(tri, s.d_slot_edge, sw, t0, ntr, (R)kr, (R)ki, mikr, miki, c4r, c4i, g_rules,
                                      x + (int64_t)r0 * 2 * n, y + (int64_t)r0 * 2 * n, n, nr, (AT)ar, (AT)ai,
                                      (AT)br, (AT)bi, cnt);
      prof_end(st, tok);
      note_launch();
      CAL_TRY_CUDA(cudaGetLastError());
    }
    return CAL_OK;
  }
}

int launch_rwg_free(const Space& s, int scat, double kr, double ki, int nreg, int precision, int vec_prec,
                    const void* x, void* y, int64_t n, int nrhs, double ar, double ai, double br, double bi,
                    cudaStream_t st) {
  if (int rc = set_quadrature_tables(nreg, 1)) return rc;
  if (precision == CAL_FP64)
    return rwg_free_t<double, double2, double>(s, scat, kr, ki, nreg, (const double2*)x, (double2*)y, n, nrhs, ar,
                                               ai, br, bi, st);
  if (vec_prec == CAL_FP64)
    return rwg_free_t<float, double2, double>(s, scat, kr, ki, nreg, (const double2*)x, (double2*)y, n, nrhs, ar,
                                              ai, br, bi, st);
  return rwg_free_t<float, float2, float>(s, scat, kr, ki, nreg, (const float2*)x, (float2*)y, n, nrhs, ar, ai, br,
                                          bi, st);
}

// ---------------------------------------------------------------------------
// The mixed discretisation (eq. mixed_discretisation): C between RWG written
// on the barycentric refinement (RWG_b: the three RWG pieces of a primal
// triangle restricted to each of its six children) and BC, float64. The
// regular pairs tau1 < tau2 of the block's barycentric triangles are formed
// once and give, by the symmetry of the bilinear form and of the tensor rule,
// both orientations and both blocks: C(RWG_b, BC) and C(BC, RWG_b) = its
// transpose there. The touching pairs take the float64 Sauter–Schwab rules in
// their listed orders (vertex pairs, listed once, also in the swapped order),
// each order contracted separately for the two blocks.
// ---------------------------------------------------------------------------
struct CrossSlots {
  const int* redge;      // [ntri][3] RWG_b edges
  const double* rsw;     // [ntri][3][4]
  const int* bedge;      // [ntri][nslot] BC edges
  const double* bsw;     // [ntri][nslot][4]
  int nslot;
};

__device__ __forceinline__ void cross_add(const double* pc, const double* swa, const double* swb, int ea, int eb,
                                          const Sink<double>& out) {
  double Sr = 0, Si = 0, Cr = 0, Ci = 0;
  const V3<double> wa = {swa[1], swa[2], swa[3]}, wb = {swb[1], swb[2], swb[3]};
  entry_from_pc(pc, swa[0], wa, swb[0], wb, 0.0, 0.0, 0.0, 0.0, false, true, Sr, Si, Cr, Ci);
  out.add(ea, eb, false, true, Sr, Si, Cr, Ci);
}

template <int NREG>
__global__ void __launch_bounds__(256) cross_regular_kernel(const TriD* __restrict__ tri, CrossSlots cs, int64_t t0,
                                                            int64_t ntr, double kr, double ki, Rules rl,
                                                            Sink<double> rb, Sink<double> br) {
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bi > bj) return;
  const int64_t i1 = (int64_t)bi * 16 + threadIdx.y;
  const int64_t i2 = (int64_t)bj * 16 + threadIdx.x;
  if (i1 >= ntr || i2 >= ntr || i1 >= i2) return;
  const int64_t t1 = t0 + i1, t2 = t0 + i2;
  const TriD A = tri[t1];
  const TriD B = tri[t2];
  if (touching(A, B)) return;
  const V3<double> D = centroid_delta(A, B);
  Mom<double> m;
  pair_moments<double, NREG>(A, B, rl, D, kr, ki, true, m);
  double pc[36];
  pair_coeffs(m, D, pc);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < cs.nslot; ++b) {
      // RWG_b on t1 (test) with BC on t2 (trial), and BC on t1 with RWG_b on t2
      const int r1 = cs.redge[3 * t1 + a], c2 = cs.bedge[(size_t)t2 * cs.nslot + b];
      if (r1 >= 0 && c2 >= 0) {
        double Sr = 0, Si = 0, Cr = 0, Ci = 0;
        const double* swa = cs.rsw + (3 * t1 + a) * 4;
        const double* swb = cs.bsw + ((size_t)t2 * cs.nslot + b) * 4;
        entry_from_pc(pc, swa[0], V3<double>{swa[1], swa[2], swa[3]}, swb[0], V3<double>{swb[1], swb[2], swb[3]},
                      0.0, 0.0, 0.0, 0.0, false, true, Sr, Si, Cr, Ci);
        rb.add(r1, c2, false, true, Sr, Si, Cr, Ci);
        br.add(c2, r1, false, true, Sr, Si, Cr, Ci);
      }
      const int c1 = cs.bedge[(size_t)t1 * cs.nslot + b], r2 = cs.redge[3 * t2 + a];
      if (c1 >= 0 && r2 >= 0) {
        double Sr = 0, Si = 0, Cr = 0, Ci = 0;
        const double* swa = cs.bsw + ((size_t)t1 * cs.nslot + b) * 4;
        const double* swb = cs.rsw + (3 * t2 + a) * 4;
        entry_from_pc(pc, swa[0], V3<double>{swa[1], swa[2], swa[3]}, swb[0], V3<double>{swb[1], swb[2], swb[3]},
                      0.0, 0.0, 0.0, 0.0, false, true, Sr, Si, Cr, Ci);
        br.add(c1, r2, false, true, Sr, Si, Cr, Ci);
        rb.add(r2, c1, false, true, Sr, Si, Cr, Ci);
      }
    }
}

__global__ void __launch_bounds__(128) cross_singular_kernel(const TriD* __restrict__ tri,
                                                             const SingPair* __restrict__ pairs, int64_t np,
                                                             CrossSlots cs, double kr, double ki, Rules rl,
                                                             Sink<double> rb, Sink<double> br) {
  const int lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (p >= np) return;
  const SingPair sp = pairs[p];
  if (sp.cls == 3) return;  // flat identical panels: C vanishes
  const TriD A = tri[sp.t1];
  const TriD B = tri[sp.t2];
  SingGeom gm;
  double MG[18], Mg[18];
  sing_pair_moments(A, B, sp, kr, ki, true, rl, lane, gm, MG, Mg);
  double pc[36];
  sing_pair_coeffs(MG, Mg, gm.Q1, gm.Q2, gm.ea, gm.eb, gm.ec, gm.ed, gm.D, pc);
  const int ns = cs.nslot;
  for (int q = lane; q < 3 * ns; q += 32) {
    const int a = q / ns, b = q - a * ns;
    // test RWG_b on t1, trial BC on t2 -> C(RWG_b, BC); test BC on t1, trial RWG_b on t2 -> C(BC, RWG_b)
    const int r1 = cs.redge[3 * sp.t1 + a], c2 = cs.bedge[(size_t)sp.t2 * ns + b];
    const int c1 = cs.bedge[(size_t)sp.t1 * ns + b], r2 = cs.redge[3 * sp.t2 + a];
    const double* rs1 = cs.rsw + (3 * sp.t1 + a) * 4;
    const double* bs2 = cs.bsw + ((size_t)sp.t2 * ns + b) * 4;
    const double* bs1 = cs.bsw + ((size_t)sp.t1 * ns + b) * 4;
    const double* rs2 = cs.rsw + (3 * sp.t2 + a) * 4;
    if (r1 >= 0 && c2 >= 0) {
      cross_add(pc, rs1, bs2, r1, c2, rb);
      // a vertex pair's rule maps onto itself with the triangles swapped: the
      // (t2, t1) order, BC on t2 tested against RWG_b on t1, is the same value
      if (sp.cls == 1) cross_add(pc, rs1, bs2, c2, r1, br);
    }
    if (c1 >= 0 && r2 >= 0) {
      cross_add(pc, bs1, rs2, c1, r2, br);
      if (sp.cls == 1) cross_add(pc, bs1, rs2, r2, c1, rb);
    }
  }
}

int launch_cross_c(const Space& bc, const int* d_redge, const double* d_rsw, int scat, double kr, double ki, int nreg,
                   int nsing, int64_t row_off, int64_t ld, double* Crb, double* Cbr, cudaStream_t st) {
  int rc = set_quadrature_tables(nreg, nsing);
  if (rc) return rc;
  const int64_t t0 = scat < 0 ? 0 : bc.tri_off[scat];
  const int64_t ntr = (scat < 0 ? bc.ntri : bc.tri_off[scat + 1]) - t0;
  const int64_t nb = (ntr + 15) / 16;
  if (nb > 65535) return fail(CAL_EINVAL, "too many triangles for the regular-pair grid (%lld)", (long long)ntr);
  CrossSlots cs{d_redge, d_rsw, bc.d_slot_edge, bc.d_slot_swd, bc.nslot};
  Sink<double> rb{nullptr, Crb, row_off, ld, nullptr, nullptr};
  Sink<double> br{nullptr, Cbr, row_off, ld, nullptr, nullptr};
  const int tok = prof_begin(st, "cross", 0.0);
  auto kern = nreg == 6 ? cross_regular_kernel<6> : (nreg == 1 ? cross_regular_kernel<1> : cross_regular_kernel<0>);
  if (ntr > 1) {
    kern<<<dim3((unsigned)nb, (unsigned)nb), dim3(16, 16), 0, st>>>(bc.d_triD, cs, t0, ntr, kr, ki, g_rules, rb, br);
    note_launch();
  }
  const int d0 = scat < 0 ? 0 : scat, d1 = scat < 0 ? (int)bc.sing.size() : scat + 1;
  for (int d = d0; d < d1; ++d) {
    const int64_t np = (int64_t)bc.sing[d].size();
    if (np == 0) continue;
    cross_singular_kernel<<<(unsigned)((np + 3) / 4), 128, 0, st>>>(bc.d_triD, bc.d_sing[d], np, cs, kr, ki, g_rules,
                                                                    rb, br);
    note_launch();
  }
  prof_end(st, tok);
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

}  // namespace cal
