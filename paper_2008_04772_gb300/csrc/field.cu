// Electric field at points off the surface (the |E|^2 maps of Section 5).
//
// The Stratton–Chu representations (eqs. StrattonChu_int, StrattonChu_ext) with
// the potential operators of Section 2,
//   E_k v(x) = ik int v G - (1/(ik)) grad_x int div v G,   H_k v(x) = curl_x int v G,
// G = e^{ik|x-y|}/(4 pi |x-y|), so that with grad_x G = (x - y) g,
// g = (ik r - 1) e^{ikr}/(4 pi r^3):
//   E_k v(x) = sum w [ik G v - (1/(ik)) g div v (x - y)],  H_k v(x) = sum w g (x - y) x v.
// From the solved traces u_1 = sum c_e RWG_e = gamma_D E and u_2 = sum d_e RWG_e:
//   exterior:        E = E^inc - [H_ke(u_1) + E_ke((mu_e/k_e) u_2)]   (union surface)
//   inside Gamma_m:  E = H_km(u_1) + E_km((mu_m/k_m) u_2)             (Gamma_m only)
// The region of a point is the scatterer whose closed mesh winds around it
// (winding number = solid angle / 4 pi, Van Oosterom–Strackee formula per
// triangle), or the exterior. Surface integrals use the 6-point rule on the
// 4^levels congruent sub-triangles of each triangle.
//
// Three kernels: regions (thread per point, all triangles), source points
// (thread per triangle: positions, weights and the currents u_1, u_2, div u_2
// at every composite-rule point), and the potentials: one thread per field
// point of a region, sources streamed through shared memory in tiles, float32
// arithmetic for float32-bulk solutions and float64 for CAL_FP64 ones.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"
#include "solve.h"

namespace cal {
namespace {

inline unsigned blocks_of(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// region of each point: m if the winding number of scatterer m's triangles
// exceeds 1/2, else -1. Triangles are grouped by scatterer (tri_off).
__global__ void winding_kernel(const TriD* __restrict__ tri, const int64_t* __restrict__ tri_off, int M,
                               const double* __restrict__ pts, int64_t npt, int32_t* __restrict__ region) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npt) return;
  const double x[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
  int reg = -1;
  for (int m = 0; m < M; ++m) {
    double omega = 0.0;
    for (int64_t t = tri_off[m]; t < tri_off[m + 1]; ++t) {
      const TriD T = tri[t];
      double v[3][3], l[3];
      for (int a = 0; a < 3; ++a) {
        for (int c = 0; c < 3; ++c) v[a][c] = T.c[c] + T.off[a][c] - x[c];
        l[a] = sqrt(v[a][0] * v[a][0] + v[a][1] * v[a][1] + v[a][2] * v[a][2]);
      }
      auto dot = [](const double* p, const double* q) { return p[0] * q[0] + p[1] * q[1] + p[2] * q[2]; };
      const double bxc[3] = {v[1][1] * v[2][2] - v[1][2] * v[2][1], v[1][2] * v[2][0] - v[1][0] * v[2][2],
                             v[1][0] * v[2][1] - v[1][1] * v[2][0]};
      const double num = dot(v[0], bxc);
      const double den = l[0] * l[1] * l[2] + dot(v[0], v[1]) * l[2] + dot(v[1], v[2]) * l[0] + dot(v[2], v[0]) * l[1];
      omega += 2.0 * atan2(num, den);
    }
    if (omega > 2.0 * M_PI) reg = m;  // winding number omega / 4 pi > 1/2
  }
  region[i] = reg;
}

template <typename AT>
struct __align__(16) Src {
  AT y[3], w;
  AT a[6];   // u_1 (3 complex)
  AT d[6];   // u_2 (3 complex)
  AT dd[2];  // div u_2
};

// sources of every triangle t at the Q composite-rule points, for right-hand side q
template <typename AT>
__global__ void field_sources_kernel(const TriD* __restrict__ tri, const int* __restrict__ slot_edge,
                                     const double* __restrict__ slot_sw, int64_t nt, const double2* __restrict__ x,
                                     const double2* __restrict__ xinc, int64_t ne, const double* __restrict__ bary,
                                     const double* __restrict__ wq, int Q, Src<AT>* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (t >= nt) return;
  const TriD T = tri[t];
  const double2* xq = x + (size_t)q * 2 * ne;
  const double2* iq = xinc ? xinc + (size_t)q * 2 * ne : nullptr;
  double ca[3][2], cd[3][2], sg[3], wv[3][3];
  for (int a = 0; a < 3; ++a) {
    const int e = slot_edge[3 * t + a];
    double2 c1 = xq[e], c2 = xq[ne + e];
    if (iq) {
      c1.x += iq[e].x; c1.y += iq[e].y;
      c2.x += iq[ne + e].x; c2.y += iq[ne + e].y;
    }
    ca[a][0] = c1.x; ca[a][1] = c1.y;
    cd[a][0] = c2.x; cd[a][1] = c2.y;
    const double* sw = slot_sw + (3 * t + a) * 4;
    sg[a] = sw[0];
    for (int c = 0; c < 3; ++c) wv[a][c] = sw[1 + c];
  }
  double dd[2] = {0.0, 0.0};
  for (int a = 0; a < 3; ++a) {
    dd[0] += 2.0 * sg[a] * cd[a][0];
    dd[1] += 2.0 * sg[a] * cd[a][1];
  }
  for (int u = 0; u < Q; ++u) {
    double xi[3];
    for (int c = 0; c < 3; ++c)
      xi[c] = bary[3 * u] * T.off[0][c] + bary[3 * u + 1] * T.off[1][c] + bary[3 * u + 2] * T.off[2][c];
    Src<AT> s;
    for (int c = 0; c < 3; ++c) s.y[c] = (AT)(T.c[c] + xi[c]);
    s.w = (AT)(wq[u] * T.area);
    for (int c = 0; c < 3; ++c) {
      double ar = 0, ai = 0, dr = 0, di = 0;
      for (int a = 0; a < 3; ++a) {
        const double phi = sg[a] * xi[c] + wv[a][c];
        ar += ca[a][0] * phi; ai += ca[a][1] * phi;
        dr += cd[a][0] * phi; di += cd[a][1] * phi;
      }
      s.a[2 * c] = (AT)ar; s.a[2 * c + 1] = (AT)ai;
      s.d[2 * c] = (AT)dr; s.d[2 * c + 1] = (AT)di;
    }
    s.dd[0] = (AT)dd[0];
    s.dd[1] = (AT)dd[1];
    out[((size_t)q * nt + t) * Q + u] = s;
  }
}

__device__ __forceinline__ void cis_exp(float kr, float ki, float r, float& c, float& s, float& amp) {
  // phase reduced to [-pi, pi] by Cody–Waite with 2 pi split in two floats (kr r
  // reaches ~100 on the aggregates), then the hardware sine and cosine
  constexpr double TWO_PI = 6.283185307179586476925286766559;
  constexpr float TP_HI = (float)TWO_PI;
  constexpr float TP_LO = (float)(TWO_PI - (double)(float)TWO_PI);
  constexpr float INV_TP = (float)(1.0 / TWO_PI);
  const float ph = kr * r;
  const float n = rintf(ph * INV_TP);
  float th = fmaf(-n, TP_HI, ph);
  th = fmaf(-n, TP_LO, th);
  __sincosf(th, &s, &c);
  amp = ki != 0.0f ? __expf(-ki * r) : 1.0f;
}
__device__ __forceinline__ void cis_exp(double kr, double ki, double r, double& c, double& s, double& amp) {
  sincos(kr * r, &s, &c);
  amp = exp(-ki * r);
}
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

constexpr int FIELD_THREADS = 128;

// E at the points idx[0..np) of one region, for right-hand side blockIdx.y:
// sources [s0, s1) of that right-hand side at wavenumber k;
// out = sgn [H_k(u_1) + scale E_k(u_2)] (+ E^inc at k_e when add_inc)
template <typename AT>
__global__ void __launch_bounds__(FIELD_THREADS) field_eval_kernel(
    const Src<AT>* __restrict__ src, int64_t nsrc_total, int64_t s0, int64_t s1, int64_t chunk,
    const int* __restrict__ idx, int64_t np, const double* __restrict__ pts, double kr, double ki,
    AT* __restrict__ part) {
  __shared__ Src<AT> tile[FIELD_THREADS];
  const int q = blockIdx.y;
  // this block's chunk of the source points (blockIdx.z of the split)
  const int64_t a0 = s0 + (int64_t)blockIdx.z * chunk;
  const int64_t a1 = a0 + chunk < s1 ? a0 + chunk : s1;
  const int64_t p = (int64_t)blockIdx.x * FIELD_THREADS + threadIdx.x;
  const bool live = p < np;
  const int i = live ? idx[p] : 0;
  const AT x[3] = {(AT)pts[3 * i], (AT)pts[3 * i + 1], (AT)pts[3 * i + 2]};
  const AT kre = (AT)kr, kim = (AT)ki;
  const AT inv4pi = (AT)(0.25 / M_PI);
  // S1 = sum w G u_2, S2 = sum w g div u_2 (x - y), H = sum w g (x - y) x u_1
  AT S1[6] = {}, S2[6] = {}, H[6] = {};
  const Src<AT>* sq = src + (size_t)q * nsrc_total;
  for (int64_t b0 = a0; b0 < a1; b0 += FIELD_THREADS) {
    const int nb = (int)(a1 - b0 < FIELD_THREADS ? a1 - b0 : FIELD_THREADS);
    __syncthreads();
    if (threadIdx.x < nb) tile[threadIdx.x] = sq[b0 + threadIdx.x];
    __syncthreads();
    if (!live) continue;
    for (int j = 0; j < nb; ++j) {
      const Src<AT>& s = tile[j];
      const AT dx = x[0] - s.y[0], dy = x[1] - s.y[1], dz = x[2] - s.y[2];
      const AT r2 = dx * dx + dy * dy + dz * dz;
      const AT ir = rsqrt_t(r2);
      const AT r = r2 * ir;
      AT c, sn, amp;
      cis_exp(kre, kim, r, c, sn, amp);
      const AT a0 = amp * ir * inv4pi * s.w;  // w |G|
      const AT Gr = a0 * c, Gi = a0 * sn;       // w G
      // w g = w G (ik r - 1) / r^2, ik r = (i kre - kim) r
      const AT fr = (-kim * r - (AT)1) * ir * ir, fi = kre * r * ir * ir;
      const AT gr = Gr * fr - Gi * fi, gi = Gr * fi + Gi * fr;
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        S1[2 * cc] += Gr * s.d[2 * cc] - Gi * s.d[2 * cc + 1];
        S1[2 * cc + 1] += Gr * s.d[2 * cc + 1] + Gi * s.d[2 * cc];
      }
      const AT hr = gr * s.dd[0] - gi * s.dd[1], hi = gr * s.dd[1] + gi * s.dd[0];
      S2[0] += hr * dx; S2[1] += hi * dx;
      S2[2] += hr * dy; S2[3] += hi * dy;
      S2[4] += hr * dz; S2[5] += hi * dz;
      // (x - y) x u_1, complex components
      const AT cxr = dy * s.a[4] - dz * s.a[2], cxi = dy * s.a[5] - dz * s.a[3];
      const AT cyr = dz * s.a[0] - dx * s.a[4], cyi = dz * s.a[1] - dx * s.a[5];
      const AT czr = dx * s.a[2] - dy * s.a[0], czi = dx * s.a[3] - dy * s.a[1];
      H[0] += gr * cxr - gi * cxi; H[1] += gr * cxi + gi * cxr;
      H[2] += gr * cyr - gi * cyi; H[3] += gr * cyi + gi * cyr;
      H[4] += gr * czr - gi * czi; H[5] += gr * czi + gi * czr;
    }
  }
  if (!live) return;
  // partial sums of this chunk: part[((split * nrhs + q) * np + p) * 18 + k]
  AT* o = part + (((size_t)blockIdx.z * gridDim.y + q) * np + p) * 18;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    o[k] = S1[k];
    o[6 + k] = S2[k];
    o[12 + k] = H[k];
  }
}

// the field at each point of a region from the chunks' partial sums (added in
// float64): E_k(u_2) = ik S1 - (1/(ik)) S2, then the representation's sign,
// scale and, outside, the incident field
template <typename AT>
__global__ void field_finish_kernel(const AT* __restrict__ part, int nsplit, int nrhs, const int* __restrict__ idx,
                                    int64_t np, const double* __restrict__ pts, double kr, double ki, double sgn,
                                    double scr, double sci, int add_inc, double ke, const double* __restrict__ inc,
                                    double2* __restrict__ out, int64_t npt_total) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (p >= np) return;
  const int i = idx[p];
  double S[18];
  for (int k = 0; k < 18; ++k) S[k] = 0.0;
  for (int c = 0; c < nsplit; ++c) {
    const AT* o = part + (((size_t)c * nrhs + q) * np + p) * 18;
    for (int k = 0; k < 18; ++k) S[k] += (double)o[k];
  }
  const double* S1 = S;
  const double* S2 = S + 6;
  const double* H = S + 12;
  // E_k(u_2) = ik S1 - (1/(ik)) S2; ik = i kr - ki
  const double ikr = -ki, iki = kr;
  const double den = ikr * ikr + iki * iki;
  const double jr = ikr / den, ji = -iki / den;  // 1/(ik)
  double2* ot = out + ((size_t)q * npt_total + i) * 3;
  double einc[3][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
  if (add_inc) {
    const double* dq = inc + 6 * q;
    const double ph = ke * (dq[0] * pts[3 * i] + dq[1] * pts[3 * i + 1] + dq[2] * pts[3 * i + 2]);
    double sp, cp;
    sincos(ph, &sp, &cp);
    for (int cc = 0; cc < 3; ++cc) {
      einc[cc][0] = cp * dq[3 + cc];
      einc[cc][1] = sp * dq[3 + cc];
    }
  }
  for (int cc = 0; cc < 3; ++cc) {
    const double s1r = S1[2 * cc], s1i = S1[2 * cc + 1];
    const double s2r = S2[2 * cc], s2i = S2[2 * cc + 1];
    const double er = (ikr * s1r - iki * s1i) - (jr * s2r - ji * s2i);
    const double ei = (ikr * s1i + iki * s1r) - (jr * s2i + ji * s2r);
    const double tr = H[2 * cc] + (scr * er - sci * ei);
    const double ti = H[2 * cc + 1] + (scr * ei + sci * er);
    ot[cc] = make_double2(einc[cc][0] + sgn * tr, einc[cc][1] + sgn * ti);
  }
}

// barycentric points and weights (sum 1) of the 6-point rule on the 4^levels
// sub-triangles of a uniform midpoint subdivision
void composite_table(int levels, std::vector<double>& bary, std::vector<double>& w) {
  std::vector<double> b6, w6;
  triangle_rule(6, b6, w6);
  std::vector<std::array<double, 9>> tris = {{1, 0, 0, 0, 1, 0, 0, 0, 1}};
  for (int l = 0; l < levels; ++l) {
    std::vector<std::array<double, 9>> nxt;
    for (const auto& T : tris) {
      double v[3][3], m[3][3];
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) v[a][c] = T[3 * a + c];
      for (int c = 0; c < 3; ++c) {
        m[0][c] = 0.5 * (v[0][c] + v[1][c]);
        m[1][c] = 0.5 * (v[1][c] + v[2][c]);
        m[2][c] = 0.5 * (v[2][c] + v[0][c]);
      }
      auto mk = [](const double* a, const double* b, const double* c) {
        return std::array<double, 9>{a[0], a[1], a[2], b[0], b[1], b[2], c[0], c[1], c[2]};
      };
      nxt.push_back(mk(v[0], m[0], m[2]));
      nxt.push_back(mk(m[0], v[1], m[1]));
      nxt.push_back(mk(m[2], m[1], v[2]));
      nxt.push_back(mk(m[0], m[1], m[2]));
    }
    tris.swap(nxt);
  }
  bary.clear();
  w.clear();
  for (const auto& T : tris)
    for (int u = 0; u < 6; ++u) {
      for (int c = 0; c < 3; ++c)
        bary.push_back(b6[3 * u] * T[c] + b6[3 * u + 1] * T[3 + c] + b6[3 * u + 2] * T[6 + c]);
      w.push_back(w6[u] / (double)tris.size());
    }
}

template <typename AT>
int near_field_t(const FieldArgs& f, const std::vector<int>& reg_h, cudaStream_t st) {
  const Space& sp = *f.rwg;
  const int64_t nt = sp.ntri, ne = sp.nbasis;
  std::vector<double> bary, wq;
  composite_table(f.levels, bary, wq);
  const int Q = (int)wq.size();
  const int64_t nsrc = nt * Q;
  double *d_bary = nullptr, *d_wq = nullptr;
  Src<AT>* d_src = nullptr;
  int* d_idx = nullptr;
  auto cleanup = [&]() {
    dfree(d_bary, st);
    dfree(d_wq, st);
    dfree(d_src, st);
    dfree(d_idx, st);
  };
  if (dalloc((void**)&d_bary, bary.size() * sizeof(double), st) != cudaSuccess ||
      dalloc((void**)&d_wq, wq.size() * sizeof(double), st) != cudaSuccess ||
      dalloc((void**)&d_src, (size_t)f.nrhs * nsrc * sizeof(Src<AT>), st) != cudaSuccess ||
      dalloc((void**)&d_idx, std::max<size_t>(reg_h.size(), 1) * sizeof(int), st) != cudaSuccess) {
    cleanup();
    return fail(CAL_ENOMEM, "near field: cannot allocate %lld source points",
                (long long)(f.nrhs * nsrc));
  }
  CAL_TRY_CUDA(cudaMemcpyAsync(d_bary, bary.data(), bary.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  CAL_TRY_CUDA(cudaMemcpyAsync(d_wq, wq.data(), wq.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  field_sources_kernel<AT><<<dim3(blocks_of(nt, 128), f.nrhs), 128, 0, st>>>(
      sp.d_triD, sp.d_slot_edge, sp.d_slot_swd, nt, f.x, f.xinc, ne, d_bary, d_wq, Q, d_src);
  note_launch();
  // points grouped by region: the exterior (-1) then each scatterer
  std::vector<int> order;
  std::vector<int64_t> start(f.M + 3, 0);
  for (int r = -1; r < f.M; ++r) {
    start[r + 1] = (int64_t)order.size();
    for (int64_t i = 0; i < f.npt; ++i)
      if (reg_h[i] == r) order.push_back((int)i);
  }
  start[f.M + 1] = (int64_t)order.size();
  if (!order.empty())
    CAL_TRY_CUDA(cudaMemcpyAsync(d_idx, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  const int tok = prof_begin(st, "near_field", 0.0);
  for (int r = -1; r < f.M; ++r) {
    const int64_t np = start[r + 2] - start[r + 1];
    if (np == 0) continue;
    std::complex<double> k, scale;
    int64_t s0, s1;
    if (r < 0) {
      k = f.k_e;
      scale = f.mu_e / f.k_e;
      s0 = 0;
      s1 = nsrc;
    } else {
      k = f.k_m[r];
      scale = f.mu_m[r] / f.k_m[r];
      s0 = sp.tri_off[r] * Q;
      s1 = sp.tri_off[r + 1] * Q;
    }
    const double sgn = r < 0 ? -1.0 : 1.0;
    // the sources are split into chunks so that the grid fills the GPU (a
    // region may hold only a few thousand points): about 8 blocks per SM,
    // each chunk at least 8 tiles of sources, the partial sums within 256 MB
    const int64_t tiles = (int64_t)blocks_of(np, FIELD_THREADS) * f.nrhs;
    const int64_t ns = s1 - s0;
    int64_t nsplit = std::max<int64_t>(1, (8LL * std::max(1, f.n_sm) + tiles - 1) / tiles);
    nsplit = std::min<int64_t>(nsplit, std::max<int64_t>(1, ns / (8 * FIELD_THREADS)));
    nsplit = std::min<int64_t>(nsplit, std::max<int64_t>(1, (256LL << 20) / ((int64_t)f.nrhs * np * 18 * sizeof(AT))));
    nsplit = std::min<int64_t>(nsplit, 65535);
    const int64_t chunk = (ns + nsplit - 1) / nsplit;
    AT* d_part = nullptr;
    if (dalloc((void**)&d_part, (size_t)nsplit * f.nrhs * np * 18 * sizeof(AT), st) != cudaSuccess) {
      prof_end(st, tok);
      cleanup();
      return fail(CAL_ENOMEM, "near field: cannot allocate the partial sums");
    }
    field_eval_kernel<AT><<<dim3(blocks_of(np, FIELD_THREADS), f.nrhs, (unsigned)nsplit), FIELD_THREADS, 0, st>>>(
        d_src, nsrc, s0, s1, chunk, d_idx + start[r + 1], np, f.d_pts, k.real(), k.imag(), d_part);
    note_launch();
    field_finish_kernel<AT><<<dim3(blocks_of(np, 128), f.nrhs), 128, 0, st>>>(
        d_part, (int)nsplit, f.nrhs, d_idx + start[r + 1], np, f.d_pts, k.real(), k.imag(), sgn, scale.real(),
        scale.imag(), r < 0 ? 1 : 0, f.k_e, f.d_inc, f.d_out, f.npt);
    note_launch();
    dfree(d_part, st);
  }
  prof_end(st, tok);
  cudaError_t e = cudaGetLastError();
  cleanup();
  if (e != cudaSuccess) return fail(CAL_ECUDA, "near field: %s", cudaGetErrorString(e));
  return CAL_OK;
}

}  // namespace

int launch_regions(const Space& rwg, int M, const double* d_pts, int64_t npt, int32_t* d_region, cudaStream_t st) {
  int64_t* d_off = nullptr;
  CAL_TRY_CUDA(dalloc((void**)&d_off, (M + 1) * sizeof(int64_t), st));
  CAL_TRY_CUDA(cudaMemcpyAsync(d_off, rwg.tri_off.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  winding_kernel<<<blocks_of(npt, 128), 128, 0, st>>>(rwg.d_triD, d_off, M, d_pts, npt, d_region);
  note_launch();
  cudaError_t e = cudaGetLastError();
  CAL_TRY_CUDA(cudaStreamSynchronize(st));  // the host offsets are read by the copy
  dfree(d_off, st);
  if (e != cudaSuccess) return fail(CAL_ECUDA, "regions: %s", cudaGetErrorString(e));
  return CAL_OK;
}

int launch_near_field(const FieldArgs& f, const std::vector<int>& region, cudaStream_t st) {
  return f.precision == CAL_FP64 ? near_field_t<double>(f, region, st) : near_field_t<float>(f, region, st);
}

}  // namespace cal
