// Operator application, Gram solves, GMRES, right-hand side and far field.
//
// arXiv 2008.04772: the block operator of eqs. multiple_operator / AimAem, the
// strong form M_P^-1 P M_A^-1 A of Section 3.2 (eqs. GalA-MassP), restarted
// GMRES of Section 4, the incident traces of eq. boundary_conditions_traces and
// the far field of the Stratton–Chu representation (eq. StrattonChu_ext).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <type_traits>

#include "solve.h"

namespace cal {

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

template <typename A, typename B>
__device__ __forceinline__ void cfma(A& acc, const B& a, const B& b) {
  acc.x += (decltype(acc.x))a.x * b.x - (decltype(acc.x))a.y * b.y;
  acc.y += (decltype(acc.x))a.x * b.y + (decltype(acc.x))a.y * b.x;
}

// ---------------------------------------------------------------------------
// A7: one (S, C) block of the PMCHWT operator applied to both halves of x:
//   y1[r] += sum C x1 + alpha sum S x2,  y2[r] += sum C x2 + beta sum S x1
// with x, y component-major. Each matrix element is read once per
// application; a warp owns ROWS rows and its lanes stride over columns.
// ---------------------------------------------------------------------------
template <typename MT, typename VT, typename AT, int ROWS>
__global__ void __launch_bounds__(256) pair_gemv_kernel(
    const MT* __restrict__ S, const MT* __restrict__ C, int64_t nr, int64_t nc, int64_t ld,
    const VT* __restrict__ x1, const VT* __restrict__ x2, VT* __restrict__ y1,
    VT* __restrict__ y2, double ar, double ai, double br, double bi) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t r0 = warp * ROWS;
  if (r0 >= nr) return;
  AT cx1[ROWS], cx2[ROWS], sx1[ROWS], sx2[ROWS];
#pragma unroll
  for (int q = 0; q < ROWS; ++q) cx1[q] = cx2[q] = sx1[q] = sx2[q] = AT{0, 0};
  for (int64_t c = lane; c < nc; c += 32) {
    const VT u = x1[c], v = x2[c];
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      const int64_t r = r0 + q;
      if (r < nr) {
        if (C) {
          const MT m = C[r * ld + c];
          cfma(cx1[q], m, MT{(decltype(m.x))u.x, (decltype(m.x))u.y});
          cfma(cx2[q], m, MT{(decltype(m.x))v.x, (decltype(m.x))v.y});
        }
        if (S) {
          const MT m = S[r * ld + c];
          cfma(sx1[q], m, MT{(decltype(m.x))u.x, (decltype(m.x))u.y});
          cfma(sx2[q], m, MT{(decltype(m.x))v.x, (decltype(m.x))v.y});
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < ROWS; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cx1[q].x += __shfl_xor_sync(0xffffffffu, cx1[q].x, o);
      cx1[q].y += __shfl_xor_sync(0xffffffffu, cx1[q].y, o);
      cx2[q].x += __shfl_xor_sync(0xffffffffu, cx2[q].x, o);
      cx2[q].y += __shfl_xor_sync(0xffffffffu, cx2[q].y, o);
      sx1[q].x += __shfl_xor_sync(0xffffffffu, sx1[q].x, o);
      sx1[q].y += __shfl_xor_sync(0xffffffffu, sx1[q].y, o);
      sx2[q].x += __shfl_xor_sync(0xffffffffu, sx2[q].x, o);
      sx2[q].y += __shfl_xor_sync(0xffffffffu, sx2[q].y, o);
    }
    const int64_t r = r0 + q;
    if (lane == 0 && r < nr) {
      // y1 += C x1 + alpha S x2 ; y2 += C x2 + beta S x1
      VT a = y1[r], b = y2[r];
      a.x += cx1[q].x + ar * sx2[q].x - ai * sx2[q].y;
      a.y += cx1[q].y + ar * sx2[q].y + ai * sx2[q].x;
      b.x += cx2[q].x + br * sx1[q].x - bi * sx1[q].y;
      b.y += cx2[q].y + br * sx1[q].y + bi * sx1[q].x;
      y1[r] = a;
      y2[r] = b;
    }
  }
}

// Vectorised variant for complex64 matrices with an even leading dimension:
// every lane streams 16-byte words (two complex entries) of ROWS rows of S
// and C, with two column steps in flight, so that enough bytes are
// outstanding per SM to run at HBM bandwidth. x is read through L1/L2.
template <typename VT> struct Pair2;
template <> struct Pair2<float2> {
  __device__ static void load(const float2* x, int64_t c2, float2& a, float2& b) {
    const float4 q = reinterpret_cast<const float4*>(x)[c2];
    a = {q.x, q.y};
    b = {q.z, q.w};
  }
};
template <> struct Pair2<double2> {
  __device__ static void load(const double2* x, int64_t c2, double2& a, double2& b) {
    a = x[2 * c2];
    b = x[2 * c2 + 1];
  }
};

// Float64 vectors applied to float32 operators without float64 arithmetic
// (float64 runs at 1/64 of the float32 rate here). Each float32 entry a times
// a float64 value x = xh + xl (two floats, |xl| <= ulp(xh)/2) is
//   a xh = p + e exactly (p = fl(a xh), e = fma(a, xh, -p)), plus fl(a xl),
// and the sums are double-float (hi, lo) pairs: TwoSum (Knuth) carries the
// rounding error of every hi addition into lo. Relative error of each sum
// about 2^-48 per term, far below the float32 operator it applies.
// (explicitly rounded operations: no contraction of the product into the sums)
__device__ __forceinline__ void df_mac(float& hi, float& lo, float a, float xh, float xl) {
  const float p = __fmul_rn(a, xh);
  const float e = fmaf(a, xh, -p);
  const float c = fmaf(a, xl, e);
  const float s = __fadd_rn(hi, p);
  const float v = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(p, v));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, c));
}

// (hi, lo) += (hi2, lo2), TwoSum on the high parts
__device__ __forceinline__ void df_add(float& hi, float& lo, float hi2, float lo2) {
  const float s = __fadd_rn(hi, hi2);
  const float v = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(hi2, v));
  hi = s;
  lo = __fadd_rn(__fadd_rn(lo, lo2), err);
}

// complex (hr + i hi) += (mr + i mi)(x), x = (re hi, re lo, im hi, im lo)
__device__ __forceinline__ void df_cmac(float& hr, float& lr, float& hi, float& li, float mr, float mi,
                                        const float4& x) {
  df_mac(hr, lr, mr, x.x, x.y);
  df_mac(hr, lr, -mi, x.z, x.w);
  df_mac(hi, li, mr, x.z, x.w);
  df_mac(hi, li, mi, x.x, x.y);
}

// x [q][2n] (float64 complex), columns [off, off + cols) of both halves ->
// xs [q][h][cols] as (re hi, re lo, im hi, im lo)
__global__ void split_df_multi_kernel(const double2* __restrict__ x, int64_t n, int64_t off, int64_t cols,
                                      int nrhs, float4* __restrict__ xs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * cols * nrhs) return;
  const int64_t c = t % cols, qh = t / cols;
  const int h = (int)(qh & 1);
  const int64_t q = qh >> 1;
  const double2 v = x[q * 2 * n + h * n + off + c];
  const float rh = (float)v.x, ih = (float)v.y;
  xs[t] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}

// x (float64 complex) -> (re hi, re lo, im hi, im lo)
__global__ void split_df_kernel(const double2* __restrict__ x, float4* __restrict__ xs, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = x[i];
  const float rh = (float)v.x, ih = (float)v.y;
  xs[i] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}

template <typename VT, typename AT, int ROWS>
__global__ void __launch_bounds__(256, 2) pair_gemv_vec_kernel(
    const float4* __restrict__ S, const float4* __restrict__ C, int64_t nr, int64_t nc,
    int64_t ld2, const VT* __restrict__ x1, const VT* __restrict__ x2, VT* __restrict__ y1,
    VT* __restrict__ y2, double ar, double ai, double br, double bi) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t r0 = warp * ROWS;
  if (r0 >= nr) return;
  const int64_t nc2 = nc >> 1;
  AT cx1[ROWS], cx2[ROWS], sx1[ROWS], sx2[ROWS];
#pragma unroll
  for (int q = 0; q < ROWS; ++q) cx1[q] = cx2[q] = sx1[q] = sx2[q] = AT{0, 0};
  const bool hasC = C != nullptr, hasS = S != nullptr;
  // U column steps are loaded before any is consumed: U * ROWS * 2 16-byte words
  // per lane in flight
  constexpr int U = 4;
  int64_t rr[ROWS];
#pragma unroll
  for (int q = 0; q < ROWS; ++q) rr[q] = min(r0 + q, nr - 1) * ld2;
  auto consume = [&](const float4* mc, const float4* ms, int64_t c2) {
    VT u0, u1, v0, v1;
    Pair2<VT>::load(x1, c2, u0, u1);
    Pair2<VT>::load(x2, c2, v0, v1);
    const float2 fu0 = {(float)u0.x, (float)u0.y}, fu1 = {(float)u1.x, (float)u1.y};
    const float2 fv0 = {(float)v0.x, (float)v0.y}, fv1 = {(float)v1.x, (float)v1.y};
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      if (hasC) {
        const float2 m0 = {mc[q].x, mc[q].y}, m1 = {mc[q].z, mc[q].w};
        cfma(cx1[q], m0, fu0); cfma(cx1[q], m1, fu1);
        cfma(cx2[q], m0, fv0); cfma(cx2[q], m1, fv1);
      }
      if (hasS) {
        const float2 m0 = {ms[q].x, ms[q].y}, m1 = {ms[q].z, ms[q].w};
        cfma(sx1[q], m0, fu0); cfma(sx1[q], m1, fu1);
        cfma(sx2[q], m0, fv0); cfma(sx2[q], m1, fv1);
      }
    }
  };
  int64_t c2 = lane;
  for (; c2 + 32 * (U - 1) < nc2; c2 += 32 * U) {
    float4 mc[U][ROWS], ms[U][ROWS];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int q = 0; q < ROWS; ++q) {
        if (hasC) mc[u][q] = __ldcs(C + rr[q] + c2 + 32 * u);
        if (hasS) ms[u][q] = __ldcs(S + rr[q] + c2 + 32 * u);
      }
#pragma unroll
    for (int u = 0; u < U; ++u) consume(mc[u], ms[u], c2 + 32 * u);
  }
  for (; c2 < nc2; c2 += 32) {
    float4 mc[ROWS], ms[ROWS];
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      if (hasC) mc[q] = __ldcs(C + rr[q] + c2);
      if (hasS) ms[q] = __ldcs(S + rr[q] + c2);
    }
    consume(mc, ms, c2);
  }
#pragma unroll
  for (int q = 0; q < ROWS; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cx1[q].x += __shfl_xor_sync(0xffffffffu, cx1[q].x, o);
      cx1[q].y += __shfl_xor_sync(0xffffffffu, cx1[q].y, o);
      cx2[q].x += __shfl_xor_sync(0xffffffffu, cx2[q].x, o);
      cx2[q].y += __shfl_xor_sync(0xffffffffu, cx2[q].y, o);
      sx1[q].x += __shfl_xor_sync(0xffffffffu, sx1[q].x, o);
      sx1[q].y += __shfl_xor_sync(0xffffffffu, sx1[q].y, o);
      sx2[q].x += __shfl_xor_sync(0xffffffffu, sx2[q].x, o);
      sx2[q].y += __shfl_xor_sync(0xffffffffu, sx2[q].y, o);
    }
    const int64_t r = r0 + q;
    if (lane == 0 && r < nr) {
      // odd column count: the last column of this row
      if (nc & 1) {
        const int64_t c = nc - 1;
        const float2* Cr = reinterpret_cast<const float2*>(C);
        const float2* Sr = reinterpret_cast<const float2*>(S);
        const float2 u = {(float)x1[c].x, (float)x1[c].y}, v = {(float)x2[c].x, (float)x2[c].y};
        if (hasC) { cfma(cx1[q], Cr[r * 2 * ld2 + c], u); cfma(cx2[q], Cr[r * 2 * ld2 + c], v); }
        if (hasS) { cfma(sx1[q], Sr[r * 2 * ld2 + c], u); cfma(sx2[q], Sr[r * 2 * ld2 + c], v); }
      }
      VT a = y1[r], b = y2[r];
      a.x += cx1[q].x + ar * sx2[q].x - ai * sx2[q].y;
      a.y += cx1[q].y + ar * sx2[q].y + ai * sx2[q].x;
      b.x += cx2[q].x + br * sx1[q].x - bi * sx1[q].y;
      b.y += cx2[q].y + br * sx1[q].y + bi * sx1[q].x;
      y1[r] = a;
      y2[r] = b;
    }
  }
}

// Work units of one row and a chunk of CHUNK2 16-byte column words; a grid of
// a few CTAs per SM strides over the units, so no partial last wave idles
// SMs, and every unit adds its partial row sums with atomics (y is zeroed by
// the caller before the operator is applied).
__device__ __forceinline__ void atomic_add_v(float2* p, float x, float y) {
  atomicAdd(p, make_float2(x, y));
}
__device__ __forceinline__ void atomic_add_v(double2* p, double x, double y) {
  atomicAdd(&p->x, x);
  atomicAdd(&p->y, y);
}

// TWO_S: a combined block (reading 18) with separate S matrices for the two
// halves, y1 += C x1 + S x2 and y2 += C x2 + S2 x1 (the caller passes
// alpha = beta = 1); three matrices are read instead of two per block pair.
template <typename VT, typename AT, bool TWO_S = false>
__global__ void __launch_bounds__(256, TWO_S ? 2 : 3) pair_gemv_units_kernel(
    const float4* __restrict__ S, const float4* __restrict__ C, int64_t nr, int64_t nc2,
    int64_t ld2, int64_t chunk2, const VT* __restrict__ x1, const VT* __restrict__ x2,
    VT* __restrict__ y1, VT* __restrict__ y2, double ar, double ai, double br, double bi,
    const float4* __restrict__ S2 = nullptr) {
  const int lane = threadIdx.x & 31;
  const int64_t nsplit = (nc2 + chunk2 - 1) / chunk2;
  const int64_t nunits = nr * nsplit;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool hasC = C != nullptr, hasS = S != nullptr;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < nunits; u += wstride) {
    const int64_t r = u / nsplit;
    const int64_t c_lo = (u % nsplit) * chunk2, c_hi = min(c_lo + chunk2, nc2);
    const float4* Cr = C + r * ld2;
    const float4* Sr = S + r * ld2;
    const float4* S2r = TWO_S ? S2 + r * ld2 : nullptr;
    AT cx1 = {0, 0}, cx2 = {0, 0}, sx1 = {0, 0}, sx2 = {0, 0};
    constexpr int U = 4;
    int64_t c2 = c_lo + lane;
    auto consume = [&](float4 mc, float4 ms, float4 ms2, int64_t c) {
      VT u0, u1, v0, v1;
      Pair2<VT>::load(x1, c, u0, u1);
      Pair2<VT>::load(x2, c, v0, v1);
      using E = decltype(cx1.x);
      const AT fu0 = {(E)u0.x, (E)u0.y}, fu1 = {(E)u1.x, (E)u1.y};
      const AT fv0 = {(E)v0.x, (E)v0.y}, fv1 = {(E)v1.x, (E)v1.y};
      if (hasC) {
        const AT m0 = {(E)mc.x, (E)mc.y}, m1 = {(E)mc.z, (E)mc.w};
        cfma(cx1, m0, fu0); cfma(cx1, m1, fu1);
        cfma(cx2, m0, fv0); cfma(cx2, m1, fv1);
      }
      if (hasS) {
        const AT m0 = {(E)ms.x, (E)ms.y}, m1 = {(E)ms.z, (E)ms.w};
        if (TWO_S) {
          const AT n0 = {(E)ms2.x, (E)ms2.y}, n1 = {(E)ms2.z, (E)ms2.w};
          cfma(sx1, n0, fu0); cfma(sx1, n1, fu1);
        } else {
          cfma(sx1, m0, fu0); cfma(sx1, m1, fu1);
        }
        cfma(sx2, m0, fv0); cfma(sx2, m1, fv1);
      }
    };
    for (; c2 + 32 * (U - 1) < c_hi; c2 += 32 * U) {
      float4 mc[U], ms[U], ms2[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        if (hasC) mc[k] = __ldcs(Cr + c2 + 32 * k);
        if (hasS) ms[k] = __ldcs(Sr + c2 + 32 * k);
        if (TWO_S) ms2[k] = __ldcs(S2r + c2 + 32 * k);
      }
#pragma unroll
      for (int k = 0; k < U; ++k) consume(mc[k], ms[k], TWO_S ? ms2[k] : ms[k], c2 + 32 * k);
    }
    for (; c2 < c_hi; c2 += 32) {
      float4 mc = {0, 0, 0, 0}, ms = {0, 0, 0, 0}, ms2 = {0, 0, 0, 0};
      if (hasC) mc = __ldcs(Cr + c2);
      if (hasS) ms = __ldcs(Sr + c2);
      if (TWO_S) ms2 = __ldcs(S2r + c2);
      consume(mc, ms, ms2, c2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cx1.x += __shfl_xor_sync(0xffffffffu, cx1.x, o); cx1.y += __shfl_xor_sync(0xffffffffu, cx1.y, o);
      cx2.x += __shfl_xor_sync(0xffffffffu, cx2.x, o); cx2.y += __shfl_xor_sync(0xffffffffu, cx2.y, o);
      sx1.x += __shfl_xor_sync(0xffffffffu, sx1.x, o); sx1.y += __shfl_xor_sync(0xffffffffu, sx1.y, o);
      sx2.x += __shfl_xor_sync(0xffffffffu, sx2.x, o); sx2.y += __shfl_xor_sync(0xffffffffu, sx2.y, o);
    }
    if (lane == 0) {
      using E = decltype(y1->x);
      atomic_add_v(y1 + r, (E)(cx1.x + ar * sx2.x - ai * sx2.y), (E)(cx1.y + ar * sx2.y + ai * sx2.x));
      atomic_add_v(y2 + r, (E)(cx2.x + br * sx1.x - bi * sx1.y), (E)(cx2.y + br * sx1.y + bi * sx1.x));
    }
  }
}

// Combined block of two operator pairs on one set of unknowns (reading 18):
// C' = C_a + C_b, S1 = alpha_a S_a + alpha_b S_b, S2 = beta_a S_a + beta_b S_b.
// The first pair covers the whole [rows][ld] block; the second, of side nb,
// sits on its diagonal at (off, off) (an interior block inside the union, or
// the same rows when off = 0 and nb = rows). Float32 fused multiply-adds: the
// pass streams five matrices in and three out at HBM speed.
__device__ __forceinline__ float2 cmul_f(float ar, float ai, float2 s) {
  return make_float2(fmaf(ar, s.x, -ai * s.y), fmaf(ar, s.y, ai * s.x));
}
__device__ __forceinline__ float2 cmul2_f(float ar, float ai, float2 s, float br, float bi, float2 u) {
  return make_float2(fmaf(ar, s.x, fmaf(-ai, s.y, fmaf(br, u.x, -bi * u.y))),
                     fmaf(ar, s.y, fmaf(ai, s.x, fmaf(br, u.y, bi * u.x))));
}

__global__ void combine_init_kernel(const float2* __restrict__ S, const float2* __restrict__ C, int64_t n,
                                    float ar, float ai, float br, float bi, float2* __restrict__ Co,
                                    float2* __restrict__ S1, float2* __restrict__ S2) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const float2 s = __ldcs(S + q);
    Co[q] = __ldcs(C + q);
    S1[q] = cmul_f(ar, ai, s);
    S2[q] = cmul_f(br, bi, s);
  }
}

// rows by blockIdx.y (grid-stride), columns by the x dimension
__global__ void combine_add_kernel(const float2* __restrict__ Sa, const float2* __restrict__ Ca,
                                   const float2* __restrict__ Sb, const float2* __restrict__ Cb, int64_t nb,
                                   int64_t ld, int64_t off, float a1r, float a1i, float b1r, float b1i, float a2r,
                                   float a2i, float b2r, float b2i, float2* __restrict__ Co,
                                   float2* __restrict__ S1, float2* __restrict__ S2) {
  for (int64_t i = blockIdx.y; i < nb; i += gridDim.y)
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nb; j += (int64_t)gridDim.x * blockDim.x) {
      const int64_t at = (off + i) * ld + off + j, q = i * nb + j;
      const float2 sa = __ldcs(Sa + at), ca = __ldcs(Ca + at), sb = __ldcs(Sb + q), cb = __ldcs(Cb + q);
      Co[at] = make_float2(ca.x + cb.x, ca.y + cb.y);
      S1[at] = cmul2_f(a1r, a1i, sa, a2r, a2i, sb);
      S2[at] = cmul2_f(b1r, b1i, sa, b2r, b2i, sb);
    }
}

int combine_blocks(const void* Sa, const void* Ca, int64_t rows, std::complex<double> aa, std::complex<double> ba,
                   const void* Sb, const void* Cb, int64_t nb, int64_t off, std::complex<double> ab,
                   std::complex<double> bb, void* Co, void* S1, void* S2, bool init, int n_sm, cudaStream_t st) {
  if (init) {
    combine_init_kernel<<<(unsigned)std::max(1, n_sm * 8), 256, 0, st>>>(
        (const float2*)Sa, (const float2*)Ca, rows * rows, (float)aa.real(), (float)aa.imag(), (float)ba.real(),
        (float)ba.imag(), (float2*)Co, (float2*)S1, (float2*)S2);
    note_launch();
  }
  if (Sb) {
    if (off < 0 || off + nb > rows) return fail(CAL_EINVAL, "combined block: inner block out of range");
    const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((nb + 255) / 256, 8)),
                    (unsigned)std::max<int64_t>(1, std::min<int64_t>(nb, 65535)));
    combine_add_kernel<<<grid, 256, 0, st>>>(
        (const float2*)Sa, (const float2*)Ca, (const float2*)Sb, (const float2*)Cb, nb, rows, off,
        (float)aa.real(), (float)aa.imag(), (float)ba.real(), (float)ba.imag(), (float)ab.real(), (float)ab.imag(),
        (float)bb.real(), (float)bb.imag(), (float2*)Co, (float2*)S1, (float2*)S2);
    note_launch();
  }
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

// pair_gemv_units_kernel for one float64 vector on float32 blocks, in
// double-float arithmetic: x pre-split into (hi, lo) floats, per-lane
// (hi, lo) sums, a double-float warp reduction and one float64 atomic per row.
__global__ void __launch_bounds__(256, 3) pair_gemv_df_kernel(
    const float4* __restrict__ S, const float4* __restrict__ C, int64_t nr, int64_t nc2, int64_t ld2,
    int64_t chunk2, const float4* __restrict__ xs1, const float4* __restrict__ xs2, double2* __restrict__ y1,
    double2* __restrict__ y2, double ar, double ai, double br, double bi) {
  const int lane = threadIdx.x & 31;
  const int64_t nsplit = (nc2 + chunk2 - 1) / chunk2;
  const int64_t nunits = nr * nsplit;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool hasC = C != nullptr, hasS = S != nullptr;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < nunits; u += wstride) {
    const int64_t r = u / nsplit;
    const int64_t c_lo = (u % nsplit) * chunk2, c_hi = min(c_lo + chunk2, nc2);
    const float4* Cr = C + r * ld2;
    const float4* Sr = S + r * ld2;
    // (hi, lo) of: C x1 (re, im), C x2, S x1, S x2
    float h[8], l[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = l[k] = 0.0f;
    for (int64_t c2 = c_lo + lane; c2 < c_hi; c2 += 32) {
      const float4 u0 = xs1[2 * c2], u1 = xs1[2 * c2 + 1], v0 = xs2[2 * c2], v1 = xs2[2 * c2 + 1];
      if (hasC) {
        const float4 m = __ldcs(Cr + c2);
        df_cmac(h[0], l[0], h[1], l[1], m.x, m.y, u0); df_cmac(h[0], l[0], h[1], l[1], m.z, m.w, u1);
        df_cmac(h[2], l[2], h[3], l[3], m.x, m.y, v0); df_cmac(h[2], l[2], h[3], l[3], m.z, m.w, v1);
      }
      if (hasS) {
        const float4 m = __ldcs(Sr + c2);
        df_cmac(h[4], l[4], h[5], l[5], m.x, m.y, u0); df_cmac(h[4], l[4], h[5], l[5], m.z, m.w, u1);
        df_cmac(h[6], l[6], h[7], l[7], m.x, m.y, v0); df_cmac(h[6], l[6], h[7], l[7], m.z, m.w, v1);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float h2 = __shfl_xor_sync(0xffffffffu, h[k], o), l2 = __shfl_xor_sync(0xffffffffu, l[k], o);
        df_add(h[k], l[k], h2, l2);
      }
    if (lane == 0) {
      double d[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) d[k] = (double)h[k] + (double)l[k];
      // d: C x1 = (d0, d1), C x2 = (d2, d3), S x1 = (d4, d5), S x2 = (d6, d7)
      atomic_add_v(y1 + r, d[0] + ar * d[6] - ai * d[7], d[1] + ar * d[7] + ai * d[6]);
      atomic_add_v(y2 + r, d[2] + br * d[4] - bi * d[5], d[3] + br * d[5] + bi * d[4]);
    }
  }
}

// CSR variant (near-field P): S and C share the pattern; warp per row
template <typename MT, typename VT, typename AT>
__global__ void pair_spmv_kernel(const MT* __restrict__ S, const MT* __restrict__ C,
                                 const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                                 int64_t nr, const VT* __restrict__ x1, const VT* __restrict__ x2,
                                 VT* __restrict__ y1, VT* __restrict__ y2, double ar, double ai,
                                 double br, double bi) {
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= nr) return;
  AT cx1{0, 0}, cx2{0, 0}, sx1{0, 0}, sx2{0, 0};
  for (int64_t k = rowptr[r] + lane; k < rowptr[r + 1]; k += 32) {
    const int c = col[k];
    const VT u = x1[c], v = x2[c];
    if (C) {
      const MT m = C[k];
      cfma(cx1, m, MT{(decltype(m.x))u.x, (decltype(m.x))u.y});
      cfma(cx2, m, MT{(decltype(m.x))v.x, (decltype(m.x))v.y});
    }
    if (S) {
      const MT m = S[k];
      cfma(sx1, m, MT{(decltype(m.x))u.x, (decltype(m.x))u.y});
      cfma(sx2, m, MT{(decltype(m.x))v.x, (decltype(m.x))v.y});
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cx1.x += __shfl_xor_sync(0xffffffffu, cx1.x, o); cx1.y += __shfl_xor_sync(0xffffffffu, cx1.y, o);
    cx2.x += __shfl_xor_sync(0xffffffffu, cx2.x, o); cx2.y += __shfl_xor_sync(0xffffffffu, cx2.y, o);
    sx1.x += __shfl_xor_sync(0xffffffffu, sx1.x, o); sx1.y += __shfl_xor_sync(0xffffffffu, sx1.y, o);
    sx2.x += __shfl_xor_sync(0xffffffffu, sx2.x, o); sx2.y += __shfl_xor_sync(0xffffffffu, sx2.y, o);
  }
  if (lane == 0) {
    VT a = y1[r], b = y2[r];
    a.x += cx1.x + ar * sx2.x - ai * sx2.y;
    a.y += cx1.y + ar * sx2.y + ai * sx2.x;
    b.x += cx2.x + br * sx1.x - bi * sx1.y;
    b.y += cx2.y + br * sx1.y + bi * sx1.x;
    y1[r] = a;
    y2[r] = b;
  }
}

// The CSR variant for nrhs vectors at once. The block's columns of x are
// first copied right-hand-side-interleaved (xt[h][c][q]); a warp takes one row
// and qw right-hand sides (qw a power of two <= 32), its lanes split the
// row's entries into 32 / qw parts, so each matrix entry is read once per
// row and group and the gathered x values of a column are contiguous.
template <typename VT>
__global__ void interleave_rhs_kernel(const VT* __restrict__ x, int64_t n, int64_t col_off, int64_t cols,
                                      int nrhs, VT* __restrict__ xt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * cols * nrhs) return;
  const int q = (int)(t % nrhs);
  const int64_t rest = t / nrhs;
  const int64_t c = rest % cols;
  const int h = (int)(rest / cols);
  xt[t] = x[(int64_t)q * 2 * n + h * n + col_off + c];
}

template <typename MT, typename VT, typename AT>
__global__ void pair_spmv_multi_kernel(const MT* __restrict__ S, const MT* __restrict__ C,
                                       const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                                       int64_t nr, const VT* __restrict__ xt, int64_t cols, int nrhs, int qw,
                                       VT* __restrict__ y, int64_t n, int64_t row_off, double ar, double ai,
                                       double br, double bi) {
  const int lane = threadIdx.x & 31;
  const int ngr = (nrhs + qw - 1) / qw;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t r = w / ngr;
  if (r >= nr) return;
  const int g = (int)(w % ngr);
  const int ql = lane % qw, part = lane / qw, parts = 32 / qw;
  const int q = g * qw + ql;
  const bool on = q < nrhs;
  const VT* x1t = xt;
  const VT* x2t = xt + cols * nrhs;
  AT cx1{0, 0}, cx2{0, 0}, sx1{0, 0}, sx2{0, 0};
  for (int64_t k = rowptr[r] + part; k < rowptr[r + 1]; k += parts) {
    const int c = col[k];
    VT u{0, 0}, v{0, 0};
    if (on) {
      u = x1t[(int64_t)c * nrhs + q];
      v = x2t[(int64_t)c * nrhs + q];
    }
    if (C) {
      const MT m = C[k];
      cfma(cx1, m, MT{(decltype(m.x))u.x, (decltype(m.x))u.y});
      cfma(cx2, m, MT{(decltype(m.x))v.x, (decltype(m.x))v.y});
    }
    if (S) {
      const MT m = S[k];
      cfma(sx1, m, MT{(decltype(m.x))u.x, (decltype(m.x))u.y});
      cfma(sx2, m, MT{(decltype(m.x))v.x, (decltype(m.x))v.y});
    }
  }
  for (int o = 16; o >= qw; o >>= 1) {
    cx1.x += __shfl_xor_sync(0xffffffffu, cx1.x, o); cx1.y += __shfl_xor_sync(0xffffffffu, cx1.y, o);
    cx2.x += __shfl_xor_sync(0xffffffffu, cx2.x, o); cx2.y += __shfl_xor_sync(0xffffffffu, cx2.y, o);
    sx1.x += __shfl_xor_sync(0xffffffffu, sx1.x, o); sx1.y += __shfl_xor_sync(0xffffffffu, sx1.y, o);
    sx2.x += __shfl_xor_sync(0xffffffffu, sx2.x, o); sx2.y += __shfl_xor_sync(0xffffffffu, sx2.y, o);
  }
  if (part == 0 && on) {
    VT* y1 = y + (int64_t)q * 2 * n + row_off + r;
    VT* y2 = y1 + n;
    VT a = *y1, b = *y2;
    a.x += cx1.x + ar * sx2.x - ai * sx2.y;
    a.y += cx1.y + ar * sx2.y + ai * sx2.x;
    b.x += cx2.x + br * sx1.x - bi * sx1.y;
    b.y += cx2.y + br * sx1.y + bi * sx1.x;
    *y1 = a;
    *y2 = b;
  }
}

template <typename MT, typename VT, typename AT>
static int pair_spmv_multi_t(const BlockRef& b, const VT* x, VT* y, int64_t n, int nrhs, double ar, double ai,
                             double br, double bi, VT* xt, cudaStream_t st) {
  const int64_t tot = 2 * b.cols * nrhs;
  if (tot > 0) {
    interleave_rhs_kernel<VT><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(x, n, b.col_off, b.cols, nrhs, xt);
    note_launch();
  }
  int qw = 1;
  while (qw < nrhs && qw < 32) qw <<= 1;
  const int64_t warps = b.rows * ((nrhs + qw - 1) / qw);
  const int tok = prof_begin(st, "pair_spmv", 0.0);
  pair_spmv_multi_kernel<MT, VT, AT><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<const MT*>(b.S), reinterpret_cast<const MT*>(b.C), b.rowptr, b.col, b.rows, xt, b.cols,
      nrhs, qw, y, n, b.row_off, ar, ai, br, bi);
  prof_end(st, tok);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

int pair_spmv_multi(const BlockRef& b, int vec_prec, const void* x, void* y, int64_t n, int nrhs, double ar,
                    double ai, double br, double bi, void* scratch, cudaStream_t st) {
  if (!b.rowptr) return fail(CAL_EINVAL, "multi-vector SpMV: CSR blocks only");
  if (b.precision == CAL_FP64)
    return pair_spmv_multi_t<double2, double2, double2>(b, (const double2*)x, (double2*)y, n, nrhs, ar, ai, br, bi,
                                                        (double2*)scratch, st);
  if (vec_prec == CAL_FP64)
    return pair_spmv_multi_t<float2, double2, double2>(b, (const double2*)x, (double2*)y, n, nrhs, ar, ai, br, bi,
                                                       (double2*)scratch, st);
  return pair_spmv_multi_t<float2, float2, float2>(b, (const float2*)x, (float2*)y, n, nrhs, ar, ai, br, bi,
                                                   (float2*)scratch, st);
}

// plain y = X x for one dense operator (C-ABI cal_matvec)
template <typename MT>
__global__ void gemv_kernel(const MT* __restrict__ X, int64_t nr, int64_t nc, const MT* __restrict__ x,
                            MT* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= nr) return;
  double2 acc{0, 0};
  for (int64_t c = lane; c < nc; c += 32) cfma(acc, X[r * nc + c], x[c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) y[r] = MT{(decltype(y[r].x))acc.x, (decltype(y[r].x))acc.y};
}

template <typename MT>
__global__ void spmv_kernel(const MT* __restrict__ X, const int64_t* __restrict__ rowptr,
                            const int* __restrict__ col, int64_t nr, const MT* __restrict__ x,
                            MT* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= nr) return;
  double2 acc{0, 0};
  for (int64_t k = rowptr[r] + lane; k < rowptr[r + 1]; k += 32) cfma(acc, X[k], x[col[k]]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) y[r] = MT{(decltype(y[r].x))acc.x, (decltype(y[r].x))acc.y};
}

// ---------------------------------------------------------------------------
// elementwise helpers
// ---------------------------------------------------------------------------
template <typename A, typename B>
__global__ void convert_kernel(const A* __restrict__ a, B* __restrict__ b, int64_t n, double scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = B{(decltype(b[i].x))(a[i].x * scale), (decltype(b[i].x))(a[i].y * scale)};
}

template <typename T>
__global__ void zero_kernel(T* a, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = T{0, 0};
}

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// A6: BiCGStab on the real sparse Gram matrix for nsys complex systems that
// share it (x, b: [nsys][n]). Two phases per iteration k: K1 finishes step
// k-1 (s = r - alpha v, r = s - omega t, x += alpha p + omega s, row by row)
// and forms p_k and v_k = G p_k; K2 forms s_k and t_k = G s_k. rho_k comes
// from the K2 sums by r0^H r_k = r0^H s - omega r0^H t, so no third pass over
// the rows is needed. Float64 sums double-buffered by iteration parity; every
// block rebuilds the step scalars from them and keeps rho, alpha, omega of
// the previous step in shared memory (all blocks compute the same values).
// acc layout per (parity, bank, system): 0-1 r0^H v_k, 2 |r_k|^2 (K1);
// 3-4 t^H s, 5 t^H t, 6-7 r0^H s, 8-9 r0^H t (K2).
// ---------------------------------------------------------------------------
constexpr int BI_ACC = 10;

template <typename R>
struct BiArgs {
  const int64_t* rowptr;
  const int* col;
  const R* val;
  int64_t n;
  int nsys;
  double neg;        // multiply the solution by this (M_P = -G^T)
  // x, r (by parity: r_k in rr[k & 1]), the shadow residual r0, p and v (by
  // parity), t
  typename CT<R>::T *x, *rr0, *rr1, *rh, *p0, *p1, *v0, *v1, *t;
  double* acc;       // [2][BI_BANKS][nsys][BI_ACC]
  double tol2;       // tol^2
  double* bnorm2;    // [nsys]
  int lpr;           // lanes per (row, system)
  int three;         // three passes per iteration (many systems): p_k stored before v_k = G p_k
  GridBar* bar;      // barrier state of the cooperative launch
  int* err;          // sticky: set when a barrier wait gave up
};

// The per-system sums go to BI_BANKS copies (block b adds into bank b mod
// BI_BANKS); readers add the banks in a fixed order. One bank measured best
// on the 7680-unknown Gram systems: the reads of more banks sit on the
// critical path of every phase, same-address atomics of a few hundred blocks
// do not. Gathered columns are fetched BI_W at a time per lane.
#ifndef BI_BANKS
#define BI_BANKS 1
#endif
#ifndef BI_W
#define BI_W 8
#endif
#ifndef BI_LPR
#define BI_LPR 4
#endif
__device__ __forceinline__ double* ACC(double* acc, int nsys, int par, int bank, int s) {
  return acc + (((size_t)par * BI_BANKS + bank) * nsys + s) * BI_ACC;
}
__device__ __forceinline__ void acc_read(double* acc, int nsys, int par, int s, double (&v)[BI_ACC]) {
#pragma unroll
  for (int q = 0; q < BI_ACC; ++q) v[q] = 0.0;
#pragma unroll
  for (int b = 0; b < BI_BANKS; ++b) {
    const double* a = ACC(acc, nsys, par, b, s);
#pragma unroll
    for (int q = 0; q < BI_ACC; ++q) v[q] += a[q];
  }
}
__device__ __forceinline__ void acc_zero(double* acc, int nsys, int par, int s) {
  for (int b = 0; b < BI_BANKS; ++b)
    for (int q = 0; q < BI_ACC; ++q) ACC(acc, nsys, par, b, s)[q] = 0.0;
}

__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi, double& cr, double& ci) {
  const double d = br * br + bi * bi;
  cr = (ar * br + ai * bi) / d;
  ci = (ai * br - ar * bi) / d;
}

// The step scalars in the storage precision R: float32 on the FP32 path, where
// the vectors they scale are float32 (float64 division is slow here); the
// sums they come from stay float64.
template <typename R>
__device__ __forceinline__ void cdiv_r(double ar, double ai, double br, double bi, double& cr, double& ci) {
  if constexpr (sizeof(R) == 4) {
    // scale by a power of two near the larger part of b (exact; no float64
    // division) so that |b|^2 stays in float range
    const double sb = fmax(fabs(br), fabs(bi));
    const int e = ((__double2hiint(sb) >> 20) & 0x7ff) - 1023;
    const double sc = __hiloint2double((1023 - max(-1000, min(1000, e))) << 20, 0);  // 2^-e
    const float xr = (float)(ar * sc), xi = (float)(ai * sc), yr = (float)(br * sc), yi = (float)(bi * sc);
    const float inv = 1.0f / (yr * yr + yi * yi);
    cr = (double)((xr * yr + xi * yi) * inv);
    ci = (double)((xi * yr - xr * yi) * inv);
  } else {
    cdiv(ar, ai, br, bi, cr, ci);
  }
}

template <int NV>
__device__ __forceinline__ void block_accumulate(double (&v)[NV], double* dst) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double a = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) sh[q][wid] = a;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double a = lane < nw ? sh[q][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0 && a != 0.0) atomicAdd(dst + q, a);
    }
  }
  __syncthreads();
}

// Vectors are stored system-interleaved, element (i, s) at i * nsys + s, so
// that the lanes of a warp (consecutive systems of one row, or consecutive
// rows of few systems) read the entries of a gathered column contiguously and
// load each matrix entry once. A block is nsys x lpr x rpb threads: lpr lanes
// share one (row, system) and split its gathered columns (their sums meet by
// shuffles), rpb rows per pass, grid-stride over rows. The first nsys threads
// of a block form the per-system scalars of the step once, in float64, from
// the sums of the previous step.
struct BiLayout {
  int ns, lpr, rpb, s, sub, r0;
  __device__ BiLayout(int nsys, int lanes)
      : ns(nsys), lpr(lanes), rpb(blockDim.x / (nsys * lanes)), s(threadIdx.x % nsys),
        sub((threadIdx.x / nsys) % lanes), r0(threadIdx.x / (nsys * lanes)) {}
  // first row of this block's pass (uniform in the block) and the stride
  __device__ int64_t base() const { return (int64_t)blockIdx.x * rpb; }
  __device__ int64_t step() const { return (int64_t)gridDim.x * rpb; }
};

// sum over the lpr lanes of one (row, system): lane bits [log2 ns, log2 ns +
// log2 lpr) (ns and lpr powers of two with ns lpr dividing 32 whenever lpr > 1)
template <typename R>
__device__ __forceinline__ R lane_group_sum(const BiLayout& L, R v) {
  for (int o = L.ns; o < L.ns * L.lpr; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// per-system sums of the block's partials (NV per thread of type T), returned
// in v of the first nsys threads as float64 (nsys dividing 32: lanes of one
// system are nsys apart in a warp, summed by shuffles in T first; otherwise
// each system's partials are summed directly in float64)
template <int NV, typename T>
__device__ __forceinline__ void system_sums(const BiLayout& L, const T (&p)[NV], double (&v)[NV], double* red) {
  const int ns = L.ns, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((32 % ns) == 0 && (blockDim.x & 31) == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      T a = p[q];
      for (int o = 16; o >= ns; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane < ns) red[(q * nw + wid) * ns + lane] = (double)a;
    }
    __syncthreads();
    if (threadIdx.x < ns)
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        double a = 0.0;
        for (int w = 0; w < nw; ++w) a += red[(q * nw + w) * ns + threadIdx.x];
        v[q] = a;
      }
  } else {
#pragma unroll
    for (int q = 0; q < NV; ++q) red[q * blockDim.x + threadIdx.x] = (double)p[q];
    __syncthreads();
    const int groups = blockDim.x / ns;
    if (threadIdx.x < ns)
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        double a = 0.0;
        for (int r = 0; r < groups; ++r) a += red[q * blockDim.x + r * ns + threadIdx.x];
        v[q] = a;
      }
  }
}

template <int NV, typename T>
__device__ __forceinline__ void system_accumulate(const BiLayout& L, const T (&p)[NV], double* red, double* acc,
                                                  int nsys, int par, int off) {
  double w[NV];
  system_sums<NV, T>(L, p, w, red);
  if (threadIdx.x < L.ns)
#pragma unroll
    for (int q = 0; q < NV; ++q)
      if (w[q] != 0.0) atomicAdd(ACC(acc, nsys, par, blockIdx.x % BI_BANKS, threadIdx.x) + off + q, w[q]);
}

// Row partials of the dot products: float32 for float32 vectors (one row per
// thread, a few terms per lane; float64 adds run at 1/64 of the float32 rate
// here and were a third of the solve's time), float64 for float64 vectors;
// the sums across warps and blocks are float64.
template <typename R> struct DotT { using T = double; };
template <> struct DotT<float> { using T = float; };

// The Gram matrix does not change during a solve: when one sweep of the grid
// covers every row (each thread has at most one row) and the row has at most
// BI_W entries per lane, the lane keeps its entries in registers for the whole
// solve, and no pass reloads the row pointers, columns and values. The kernel
// with the cache is a separate instance (more registers, two blocks per SM);
// the float32 one without keeps three blocks per SM for solves of many rows.
template <typename R>
struct RowCache {
  int cj[BI_W];
  R gv[BI_W];
  bool ok;
};

template <typename R>
__device__ __forceinline__ void row_cache_load(const BiArgs<R>& A, RowCache<R>& rc) {
  const BiLayout L(A.nsys, A.lpr);
  const int64_t i = L.base() + L.r0;
  rc.ok = false;
#pragma unroll
  for (int u = 0; u < BI_W; ++u) {
    rc.cj[u] = -1;
    rc.gv[u] = R(0);
  }
  if (L.step() < A.n || i >= A.n) return;
  const int64_t q0 = A.rowptr[i], q1 = A.rowptr[i + 1];
  if (q1 - q0 > (int64_t)BI_W * L.lpr) return;
#pragma unroll
  for (int u = 0; u < BI_W; ++u) {
    const int64_t q = q0 + L.sub + (int64_t)u * L.lpr;
    if (q < q1) {
      rc.cj[u] = A.col[q];
      rc.gv[u] = A.val[q];
    }
  }
  rc.ok = true;
}

// (vr, vi) += this lane's share of sum_j g_ij f(j) over row i: from the
// register cache when it holds the row, else loaded BI_W entries at a time
template <typename R, typename F>
__device__ __forceinline__ void row_gather(const BiArgs<R>& A, const BiLayout& L, const RowCache<R>& rc, int64_t i,
                                           F f, R& vr, R& vi) {
  auto take = [&](const int (&cj)[BI_W], const R (&gv)[BI_W]) {
#pragma unroll
    for (int u = 0; u < BI_W; ++u)
      if (cj[u] >= 0) {
        const auto w = f(cj[u]);
        vr += gv[u] * w.x;
        vi += gv[u] * w.y;
      }
  };
  if (rc.ok) {
    take(rc.cj, rc.gv);
    return;
  }
  const int64_t q1 = A.rowptr[i + 1];
  for (int64_t qb = A.rowptr[i] + L.sub; qb < q1; qb += (int64_t)BI_W * L.lpr) {
    int cj[BI_W];
    R gv[BI_W];
#pragma unroll
    for (int u = 0; u < BI_W; ++u) {
      const int64_t q = qb + (int64_t)u * L.lpr;
      cj[u] = q < q1 ? A.col[q] : -1;
      gv[u] = q < q1 ? A.val[q] : R(0);
    }
    take(cj, gv);
  }
}

// per-block step state of each system (shared memory; the same in every block)
struct BiState {
  double rho_r, rho_i;  // rho_k = r0^H r_k
  double al_r, al_i;    // alpha_k
  double om_r, om_i;    // omega_k
  double beta_r, beta_i;
  int act;              // system still iterating
};

template <typename R>
__device__ __forceinline__ void bicg_phase_init(const BiArgs<R>& A, const typename CT<R>::T* __restrict__ b,
                                                double* red) {
  // x = 0; r_{-1} (parity 1) = r0 = b; p_{-1} = v_{-1} = t = 0; |b|^2 per system
  const BiLayout L(A.nsys, A.lpr);
  double part[1] = {0.0}, sum[1];
  if (L.sub == 0)
    for (int64_t i = L.base() + L.r0; i < A.n; i += L.step()) {
      const int64_t k = i * L.ns + L.s;
      const auto bv = b[(int64_t)L.s * A.n + i];
      A.x[k] = {0, 0};
      A.rr1[k] = bv;
      A.rh[k] = bv;
      A.p1[k] = A.v1[k] = A.t[k] = {0, 0};
      part[0] += (double)bv.x * bv.x + (double)bv.y * bv.y;
    }
  system_sums<1, double>(L, part, sum, red);
  if (threadIdx.x < L.ns && sum[0] != 0.0) atomicAdd(A.bnorm2 + threadIdx.x, sum[0]);
}

// K1 of iteration k (parity P = k & 1): finish step k-1 row by row (s = r -
// alpha v, r_k = s - omega t, x += alpha p + omega s) and form p_k = r_k +
// beta (p_{k-1} - omega v_{k-1}) and v_k = G p_k, the gathered p_k rebuilt
// from the step k-1 vectors; sums r0^H v_k and |r_k|^2 (mode 0). With many
// systems the rebuild (four loads per gathered entry and system) costs more
// than a grid barrier, so the phase runs in two passes: mode 1 does the row
// updates and stores p_k (sum |r_k|^2), mode 2, after a barrier, forms v_k =
// G p_k from the stored p_k (sum r0^H v_k).
template <typename R>
__device__ __forceinline__ void bicg_phase_k1(const BiArgs<R>& A, const RowCache<R>& rc, int k, BiState* st,
                                              double* red, int mode) {
  const BiLayout L(A.nsys, A.lpr);
  const int P = k & 1, ns = L.ns;
  if (threadIdx.x < ns && mode != 2) {
    const int s = threadIdx.x;
    BiState& z = st[s];
    if (k == 0) {
      z = BiState{};
      z.rho_r = A.bnorm2[s];  // r0^H r_0 = |b|^2
      z.om_r = 1.0;
      z.act = A.bnorm2[s] > 0.0;
    } else if (z.act) {
      double a[BI_ACC];
      acc_read(A.acc, A.nsys, P ^ 1, s, a);  // the K2 sums of step k-1
      if (a[5] == 0.0) {
        z.act = 0;  // t = 0: breakdown, x stays x_{k-1}
      } else {
        double omr, omi, rn_r, rn_i, tr, ti, br, bi;
        cdiv_r<R>(a[3], a[4], a[5], 0.0, omr, omi);                        // omega_{k-1}
        rn_r = a[6] - (omr * a[8] - omi * a[9]);                           // rho_k
        rn_i = a[7] - (omr * a[9] + omi * a[8]);
        cdiv_r<R>(rn_r, rn_i, z.rho_r, z.rho_i, br, bi);                  // rho_k / rho_{k-1}
        cdiv_r<R>(z.al_r, z.al_i, omr, omi, tr, ti);                      // alpha_{k-1} / omega_{k-1}
        z.beta_r = br * tr - bi * ti;
        z.beta_i = br * ti + bi * tr;
        z.om_r = omr;
        z.om_i = omi;
        z.rho_r = rn_r;
        z.rho_i = rn_i;
      }
    }
  }
  __syncthreads();
  bool any = false;
  for (int q = 0; q < ns; ++q) any |= st[q].act != 0;
  if (!any) return;
  const int s = L.s;
  const BiState& z = st[s];
  const bool act = z.act != 0;
  const bool first = k == 0;
  // the scalars of step k-1 (zero at k = 0: r_{-1} = b gives r_0 = b, p_0 = b)
  const R aR = first ? R(0) : (R)z.al_r, aI = first ? R(0) : (R)z.al_i;
  const R oR = first ? R(0) : (R)z.om_r, oI = first ? R(0) : (R)z.om_i;
  const R bR = first ? R(0) : (R)z.beta_r, bI = first ? R(0) : (R)z.beta_i;
  const auto* rprev = P ? A.rr0 : A.rr1;
  auto* rcur = P ? A.rr1 : A.rr0;
  const auto* pprev = P ? A.p0 : A.p1;
  auto* pcur = P ? A.p1 : A.p0;
  const auto* vprev = P ? A.v0 : A.v1;
  auto* vcur = P ? A.v1 : A.v0;
  using V = typename CT<R>::T;
  // r_k and p_k from the step k-1 entries r, v, t, p of one row
  auto rp_of = [&](V r1, V v1, V t1, V p1, V& rk, V& pk, V& sk) {
    sk = {r1.x - (aR * v1.x - aI * v1.y), r1.y - (aR * v1.y + aI * v1.x)};
    rk = {sk.x - (oR * t1.x - oI * t1.y), sk.y - (oR * t1.y + oI * t1.x)};
    const R dx = p1.x - (oR * v1.x - oI * v1.y), dy = p1.y - (oR * v1.y + oI * v1.x);
    pk = {rk.x + bR * dx - bI * dy, rk.y + bR * dy + bI * dx};
  };
  auto rp = [&](int64_t j, V& rk, V& pk, V& sk) {
    const int64_t kk = j * ns + s;
    rp_of(rprev[kk], vprev[kk], A.t[kk], pprev[kk], rk, pk, sk);
  };
  using D = typename DotT<R>::T;
  D part[3] = {0, 0, 0};
  if (mode == 1) {
    // row updates only: x, r_k and p_k of this thread's own rows
    if (act && L.sub == 0)
      for (int64_t i = L.base() + L.r0; i < A.n; i += L.step()) {
        const int64_t kk = i * ns + s;
        typename CT<R>::T rk, pk, sk;
        rp(i, rk, pk, sk);
        const auto p1 = pprev[kk], xi = A.x[kk];
        A.x[kk] = {xi.x + (aR * p1.x - aI * p1.y) + (oR * sk.x - oI * sk.y),
                   xi.y + (aR * p1.y + aI * p1.x) + (oR * sk.y + oI * sk.x)};
        rcur[kk] = rk;
        pcur[kk] = pk;
        part[2] += (D)rk.x * rk.x + (D)rk.y * rk.y;
      }
    system_accumulate<3, D>(L, part, red, A.acc, A.nsys, P, 0);
    return;
  }
  for (int64_t i0 = L.base(); i0 < A.n; i0 += L.step()) {
    const int64_t i = i0 + L.r0;
    const bool live = act && i < A.n;
    const bool own = live && L.sub == 0;
    const int64_t kk = i * ns + s;
    // the row's own entries, loaded before the gathers so that both are in flight
    V r1{}, v1{}, t1{}, p1{}, xi{}, h{};
    if (own) {
      h = A.rh[kk];
      if (mode != 2) {
        r1 = rprev[kk];
        v1 = vprev[kk];
        t1 = A.t[kk];
        p1 = pprev[kk];
        xi = A.x[kk];
      }
    }
    R vr = 0, vi = 0;
    if (live) {
      if (mode == 2)
        row_gather<R>(A, L, rc, i, [&](int j) { return pcur[(int64_t)j * ns + s]; }, vr, vi);
      else
        row_gather<R>(A, L, rc, i, [&](int j) {
          V rk, pk, sk;
          rp(j, rk, pk, sk);
          return pk;
        }, vr, vi);
    }
    vr = lane_group_sum(L, vr);
    vi = lane_group_sum(L, vi);
    if (own && mode == 2) {
      vcur[kk] = {vr, vi};
      part[0] += (D)(h.x * vr + h.y * vi);   // conj(r0) v
      part[1] += (D)(h.x * vi - h.y * vr);
    } else if (own) {
      V rk, pk, sk;
      rp_of(r1, v1, t1, p1, rk, pk, sk);
      A.x[kk] = {xi.x + (aR * p1.x - aI * p1.y) + (oR * sk.x - oI * sk.y),
                 xi.y + (aR * p1.y + aI * p1.x) + (oR * sk.y + oI * sk.x)};
      rcur[kk] = rk;
      pcur[kk] = pk;
      vcur[kk] = {vr, vi};
      part[0] += (D)(h.x * vr + h.y * vi);   // conj(r0) v
      part[1] += (D)(h.x * vi - h.y * vr);
      part[2] += (D)rk.x * rk.x + (D)rk.y * rk.y;
    }
  }
  system_accumulate<3, D>(L, part, red, A.acc, A.nsys, P, 0);
}

// K2 of iteration k: convergence of r_k; alpha_k = rho_k / (r0^H v_k);
// s = r_k - alpha v_k, t = G s (gathered s rebuilt); sums t^H s, t^H t,
// r0^H s, r0^H t. Returns false (in every block alike) when no system is
// active any more.
template <typename R>
__device__ __forceinline__ bool bicg_phase_k2(const BiArgs<R>& A, const RowCache<R>& rc, int k, BiState* st,
                                              double* red) {
  const BiLayout L(A.nsys, A.lpr);
  const int P = k & 1, ns = L.ns;
  if (threadIdx.x < ns) {
    const int s = threadIdx.x;
    BiState& z = st[s];
    if (blockIdx.x == 0) acc_zero(A.acc, A.nsys, P ^ 1, s);  // read by this step's K1; K1 of k+1 adds there
    if (z.act) {
      double a[BI_ACC];
      acc_read(A.acc, A.nsys, P, s, a);
      if (a[2] <= A.tol2 * A.bnorm2[s] || (a[0] == 0.0 && a[1] == 0.0)) {
        z.act = 0;  // converged (or breakdown): x_k is the solution
      } else {
        cdiv_r<R>(z.rho_r, z.rho_i, a[0], a[1], z.al_r, z.al_i);
      }
    }
  }
  __syncthreads();
  bool any = false;
  for (int q = 0; q < ns; ++q) any |= st[q].act != 0;
  if (!any) return false;
  const int s = L.s;
  const BiState& z = st[s];
  const bool act = z.act != 0;
  const R aR = (R)z.al_r, aI = (R)z.al_i;
  const auto* rcur = P ? A.rr1 : A.rr0;
  const auto* vcur = P ? A.v1 : A.v0;
  auto sj = [&](int64_t j) {
    const int64_t kk = j * ns + s;
    const auto vv = vcur[kk], rj = rcur[kk];
    return typename CT<R>::T{rj.x - (aR * vv.x - aI * vv.y), rj.y - (aR * vv.y + aI * vv.x)};
  };
  using D = typename DotT<R>::T;
  D part[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t i0 = L.base(); i0 < A.n; i0 += L.step()) {
    const int64_t i = i0 + L.r0;
    const bool live = act && i < A.n;
    const bool own = live && L.sub == 0;
    const int64_t kk = i * ns + s;
    // the row's own entries, loaded before the gathers so that both are in flight
    typename CT<R>::T vo{}, ro{}, h{};
    if (own) {
      vo = vcur[kk];
      ro = rcur[kk];
      h = A.rh[kk];
    }
    R tr = 0, ti = 0;
    if (live) row_gather<R>(A, L, rc, i, sj, tr, ti);
    tr = lane_group_sum(L, tr);
    ti = lane_group_sum(L, ti);
    if (own) {
      A.t[kk] = {tr, ti};
      const typename CT<R>::T si{ro.x - (aR * vo.x - aI * vo.y), ro.y - (aR * vo.y + aI * vo.x)};
      part[0] += (D)(tr * si.x + ti * si.y);   // conj(t) s
      part[1] += (D)(tr * si.y - ti * si.x);
      part[2] += (D)(tr * tr + ti * ti);
      part[3] += (D)(h.x * si.x + h.y * si.y); // conj(r0) s
      part[4] += (D)(h.x * si.y - h.y * si.x);
      part[5] += (D)(h.x * tr + h.y * ti);     // conj(r0) t
      part[6] += (D)(h.x * ti - h.y * tr);
    }
  }
  system_accumulate<7, D>(L, part, red, A.acc, A.nsys, P, 3);
  return true;
}

// After the last iteration (maxit reached) the systems still active take the
// update of step k: x += alpha p_k + omega s with omega from the K2 sums.
template <typename R>
__device__ __forceinline__ void bicg_phase_last(const BiArgs<R>& A, int k, BiState* st) {
  const BiLayout L(A.nsys, A.lpr);
  const int P = k & 1, ns = L.ns;
  if (threadIdx.x < ns) {
    const int s = threadIdx.x;
    BiState& z = st[s];
    if (z.act) {
      double a[BI_ACC];
      acc_read(A.acc, A.nsys, P, s, a);
      if (a[5] == 0.0) z.act = 0;
      else cdiv_r<R>(a[3], a[4], a[5], 0.0, z.om_r, z.om_i);
    }
  }
  __syncthreads();
  const int s = L.s;
  const BiState& z = st[s];
  if (!z.act || L.sub != 0) return;
  const R aR = (R)z.al_r, aI = (R)z.al_i, oR = (R)z.om_r, oI = (R)z.om_i;
  const auto* rcur = P ? A.rr1 : A.rr0;
  const auto* vcur = P ? A.v1 : A.v0;
  const auto* pcur = P ? A.p1 : A.p0;
  for (int64_t i = L.base() + L.r0; i < A.n; i += L.step()) {
    const int64_t kk = i * ns + s;
    const auto rk = rcur[kk], vv = vcur[kk], pp = pcur[kk], xi = A.x[kk];
    const R sx = rk.x - (aR * vv.x - aI * vv.y), sy = rk.y - (aR * vv.y + aI * vv.x);
    A.x[kk] = {xi.x + (aR * pp.x - aI * pp.y) + (oR * sx - oI * sy),
               xi.y + (aR * pp.y + aI * pp.x) + (oR * sy + oI * sx)};
  }
}

template <typename R>
__device__ __forceinline__ void bicg_phase_finish(const BiArgs<R>& A, typename CT<R>::T* __restrict__ out) {
  const BiLayout L(A.nsys, A.lpr);
  if (L.sub != 0) return;
  for (int64_t i = L.base() + L.r0; i < A.n; i += L.step()) {
    const auto v = A.x[i * L.ns + L.s];
    out[(size_t)L.s * A.n + i] = {(R)(A.neg * v.x), (R)(A.neg * v.y)};
  }
}

template <typename R>
__global__ void real_convert_kernel(const double* __restrict__ a, R* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (R)a[i];
}

// Grid-wide barrier of a cooperative launch (every block resident). The
// barrier state is zeroed before the launch; count only grows, so barrier g
// (1-based) is passed once count reaches g x gridDim.x. Thread 0 of each block
// arrives with an acquire-release add (its block's writes, ordered before it
// by the block barrier, are released; the last arrival acquires everyone
// else's) and polls with acquire loads: no reset and no second word on the
// critical path. Every wait is bounded: after GRID_BAR_SPINS polls the block
// raises the error word (and the solver's sticky error) and leaves; a block
// that sees the error word while it waits leaves too.
constexpr long long GRID_BAR_SPINS = 1LL << 22;

__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool grid_sync(GridBar* gb, int* sticky, unsigned& gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned want = (gen + 1) * gridDim.x;
    unsigned c = atom_add_acq_rel_gpu(&gb->count, 1u) + 1u;
    long long spins = 0;
    while (c < want) {
      if (((++spins & 255) == 0 && ld_relaxed_gpu(&gb->err)) || spins > GRID_BAR_SPINS) {
        atomicExch(&gb->err, 1);
        atomicExch(sticky, 1);
        ok = 0;
        break;
      }
      c = ld_acquire_gpu(&gb->count);
    }
    s_ok = ok;
  }
  __syncthreads();
  ++gen;
  return s_ok != 0;
}

// A6, the whole BiCGStab solve in one cooperative launch: the phases (init,
// then K1 and K2 per iteration) separated by grid barriers instead of kernel
// boundaries, and the loop left as soon as every system has converged. The
// dynamic shared memory holds the reduction scratch and the BiState array.
template <typename R, bool CACHE>
__global__ void __launch_bounds__(256, (CACHE || sizeof(R) == 8) ? 2 : 3)
    bicg_persistent(BiArgs<R> A, const typename CT<R>::T* __restrict__ b, typename CT<R>::T* __restrict__ out,
                    int maxit) {
  extern __shared__ double red[];
  BiState* st = reinterpret_cast<BiState*>(red + 7 * blockDim.x);
  unsigned gen = 0;
  RowCache<R> rc;
  if constexpr (CACHE) row_cache_load<R>(A, rc);
  else rc.ok = false;
  bicg_phase_init<R>(A, b, red);
  if (!grid_sync(A.bar, A.err, gen)) return;
  int k = 0;
  bool running = true;
  for (; k < maxit; ++k) {
    if (A.three) {
      bicg_phase_k1<R>(A, rc, k, st, red, 1);
      if (!grid_sync(A.bar, A.err, gen)) return;
      bicg_phase_k1<R>(A, rc, k, st, red, 2);
    } else {
      bicg_phase_k1<R>(A, rc, k, st, red, 0);
    }
    if (!grid_sync(A.bar, A.err, gen)) return;
    if (!bicg_phase_k2<R>(A, rc, k, st, red)) { running = false; break; }
    if (!grid_sync(A.bar, A.err, gen)) return;
  }
  if (running && k > 0) bicg_phase_last<R>(A, k - 1, st);
  // x rows are this thread's own (same layout in every phase): no barrier
  bicg_phase_finish<R>(A, out);
}

// Check of the bounded barrier: 4 blocks pass 3 barriers; block skip_block
// (if in range) leaves at once, so the others give up after their bounded
// wait. *status: 0 when every block passed every barrier, 1 when a wait gave up.
__global__ void grid_barrier_check_kernel(GridBar* gb, int* sticky, int skip_block, int* passed) {
  if ((int)blockIdx.x == skip_block) return;
  unsigned gen = 0;
  for (int i = 0; i < 3; ++i)
    if (!grid_sync(gb, sticky, gen)) return;
  if (threadIdx.x == 0) atomicAdd(passed, 1);
}

int grid_barrier_check(int skip_block, int* status, cudaStream_t st) {
  constexpr unsigned nb = 4;
  int* buf = nullptr;  // GridBar (4 ints), sticky, passed
  CAL_TRY_CUDA(dalloc((void**)&buf, 8 * sizeof(int), st));
  CAL_TRY_CUDA(cudaMemsetAsync(buf, 0, 8 * sizeof(int), st));
  GridBar* gb = reinterpret_cast<GridBar*>(buf);
  int* sticky = buf + 4;
  int* passed = buf + 5;
  void* args[] = {(void*)&gb, (void*)&sticky, (void*)&skip_block, (void*)&passed};
  const cudaError_t e =
      cudaLaunchCooperativeKernel((const void*)grid_barrier_check_kernel, dim3(nb), dim3(64), args, 0, st);
  note_launch();
  int h[2] = {0, 0};
  if (e == cudaSuccess) CAL_TRY_CUDA(cudaMemcpyAsync(h, sticky, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CAL_TRY_CUDA(cudaStreamSynchronize(st));
  dfree(buf, st);
  if (e != cudaSuccess) return fail(CAL_ECUDA, "barrier check launch: %s", cudaGetErrorString(e));
  const unsigned expect = (skip_block >= 0 && skip_block < (int)nb) ? 0u : nb;
  *status = h[0] ? 1 : 0;
  if (!h[0] && (unsigned)h[1] != expect) return fail(CAL_ECUDA, "barrier check: %d blocks passed", h[1]);
  return CAL_OK;
}

template <typename R>
int GramSolver<R>::init(const int64_t* rowptr, const int* col, const double* vals_dev, int64_t n_,
                        int nsys_, int64_t nnz, double neg_, double tol_, int maxit_, cudaStream_t st) {
  n = n_;
  nsys = nsys_;
  neg = neg_;
  tol = tol_;
  maxit = maxit_;
  d_rowptr = rowptr;
  d_col = col;
  if (nsys < 1 || nsys > 256) return fail(CAL_EINVAL, "Gram solve: %d systems (1..256)", nsys);
  const size_t vb = (size_t)n * nsys * sizeof(C);
  CAL_TRY_CUDA(dalloc((void**)&d_val, nnz * sizeof(R), st));
  if (nnz > 0) {
    real_convert_kernel<R><<<(unsigned)((nnz + 255) / 256), 256, 0, st>>>(vals_dev, d_val, nnz);
    note_launch();
    CAL_TRY_CUDA(cudaGetLastError());
  }
  CAL_TRY_CUDA(dalloc((void**)&d_work, 9 * vb, st));
  // per solve: [2][BI_BANKS][nsys][BI_ACC] sums, [nsys] |b|^2, then the barrier state
  CAL_TRY_CUDA(dalloc((void**)&d_acc, acc_bytes(), st));
  CAL_TRY_CUDA(dalloc((void**)&d_err, sizeof(int), st));
  CAL_TRY_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
  // nsys x rpb threads per block, rows grid-strided over as many blocks as
  // can be resident at once (the cooperative launch requires all of them)
  // lanes per (row, system): several for few systems (their gathers split a
  // row's columns), one when the systems alone fill the warps
  const bool pow2 = (nsys & (nsys - 1)) == 0;
  lpr = (pow2 && nsys <= 16) ? std::min(BI_LPR, 32 / nsys) : 1;
  rpb = std::max(1, 256 / (nsys * lpr));
  threads = nsys * lpr * rpb;
  smem = 7 * (size_t)threads * sizeof(double) + (size_t)nsys * sizeof(BiState);  // reduction scratch, step state
  int dev = 0, n_sm = 0, per_sm = 0;
  CAL_TRY_CUDA(cudaGetDevice(&dev));
  CAL_TRY_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t row_blocks = (n + rpb - 1) / rpb;
  // the instance that keeps the row entries in registers when its resident
  // blocks cover every row in one sweep, else the one with more blocks
  CAL_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bicg_persistent<R, true>, threads, smem));
  cached = per_sm >= 1 && row_blocks <= (int64_t)n_sm * std::min(per_sm, 8);
  if (!cached)
    CAL_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bicg_persistent<R, false>, threads, smem));
  if (per_sm < 1) return fail(CAL_ECUDA, "Gram solve: the persistent kernel does not fit on an SM");
  grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(row_blocks, (int64_t)n_sm * std::min(per_sm, 8)));
  return CAL_OK;
}

template <typename R>
GramSolver<R>::~GramSolver() {
  // every solve has completed when the solver is destroyed: release on the legacy stream
  for (void* p : {(void*)d_val, (void*)d_work, (void*)d_acc, (void*)d_err}) dfree(p, nullptr);
}

template <typename R>
size_t GramSolver<R>::acc_bytes() const {
  return (2 * (size_t)BI_BANKS * nsys * BI_ACC + nsys) * sizeof(double) + sizeof(GridBar);
}

// One solve: clear the sums and the barrier, one cooperative launch.
template <typename R>
int GramSolver<R>::solve(const C* b, C* out, cudaStream_t st) {
  BiArgs<R> A;
  A.rowptr = d_rowptr;
  A.col = d_col;
  A.val = d_val;
  A.n = n;
  A.nsys = nsys;
  A.neg = neg;
  const size_t nv = (size_t)n * nsys;
  A.x = d_work; A.rr0 = d_work + nv; A.rr1 = d_work + 2 * nv; A.rh = d_work + 3 * nv; A.p0 = d_work + 4 * nv;
  A.p1 = d_work + 5 * nv; A.v0 = d_work + 6 * nv; A.v1 = d_work + 7 * nv; A.t = d_work + 8 * nv;
  A.acc = d_acc;
  A.bnorm2 = d_acc + 2 * BI_BANKS * nsys * BI_ACC;
  A.bar = reinterpret_cast<GridBar*>(d_acc + 2 * BI_BANKS * nsys * BI_ACC + nsys);
  A.err = d_err;
  A.tol2 = tol * tol;
  A.lpr = lpr;
  A.three = nsys >= 16 ? 1 : 0;
  const int tok = prof_begin(st, "bicgstab", 0.0);
  CAL_TRY_CUDA(cudaMemsetAsync(d_acc, 0, acc_bytes(), st));
  int mi = maxit;
  void* args[] = {(void*)&A, (void*)&b, (void*)&out, (void*)&mi};
  const void* kern = cached ? (const void*)bicg_persistent<R, true> : (const void*)bicg_persistent<R, false>;
  const cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(threads), args, smem, st);
  prof_end(st, tok);
  note_launch();
  if (e != cudaSuccess) return fail(CAL_ECUDA, "Gram solve launch: %s", cudaGetErrorString(e));
  return CAL_OK;
}

template <typename R>
int GramSolver<R>::check(cudaStream_t st) const {
  int h = 0;
  CAL_TRY_CUDA(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CAL_TRY_CUDA(cudaStreamSynchronize(st));
  if (h) return fail(CAL_ETIMEOUT, "Gram solve: a bounded grid barrier gave up");
  return CAL_OK;
}

template struct GramSolver<float>;
template struct GramSolver<double>;

// ---------------------------------------------------------------------------
// launch wrappers for the operator application
// ---------------------------------------------------------------------------
template <typename MT, typename VT, typename AT>
static int pair_apply_t(const BlockRef& b, const VT* x, VT* y, int64_t n, double ar, double ai,
                        double br, double bi, cudaStream_t st) {
  const VT* x1 = x + b.col_off;
  const VT* x2 = x + n + b.col_off;
  VT* y1 = y + b.row_off;
  VT* y2 = y + n + b.row_off;
  const MT* S = reinterpret_cast<const MT*>(b.S);
  const MT* C = reinterpret_cast<const MT*>(b.C);
  if (b.rowptr) {
    if (b.S2) return fail(CAL_EINVAL, "combined block: dense blocks only");
    const int tok = prof_begin(st, "pair_spmv", 0.0);
    pair_spmv_kernel<MT, VT, AT><<<blocks_for(b.rows * 32, 256), 256, 0, st>>>(
        S, C, b.rowptr, b.col, b.rows, x1, x2, y1, y2, ar, ai, br, bi);
    prof_end(st, tok);
    note_launch();
  } else {
    // a combined block (S2 set) runs only on the float32-vector streaming kernel
    const bool s2_ok = std::is_same<MT, float2>::value && std::is_same<VT, float2>::value && S && C &&
                       b.cols % 2 == 0 && (uintptr_t)S % 16 == 0 && (uintptr_t)C % 16 == 0 &&
                       (uintptr_t)b.S2 % 16 == 0 && (uintptr_t)x1 % 16 == 0 && (uintptr_t)x2 % 16 == 0;
    if (b.S2 && !s2_ok) return fail(CAL_EINVAL, "combined block: float32 dense blocks and vectors only");
    const double bytes = (double)b.rows * b.cols * sizeof(MT) * ((S ? 1 : 0) + (C ? 1 : 0) + (b.S2 ? 1 : 0));
    const int tok = prof_begin(st, "pair_gemv", bytes);
    const bool aligned16 = ((uintptr_t)S % 16 == 0) && ((uintptr_t)C % 16 == 0) &&
                           ((uintptr_t)x1 % 16 == 0) && ((uintptr_t)x2 % 16 == 0);
    if constexpr (sizeof(MT) == 8 && std::is_same<VT, double2>::value) {
      if (b.cols % 2 == 0 && aligned16) {
        int nsm = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        // x split once into (hi, lo) floats; stream-ordered scratch
        float4* xs = nullptr;
        if (dalloc((void**)&xs, 2 * (size_t)b.cols * sizeof(float4), st) != cudaSuccess) {
          prof_end(st, tok);
          return fail(CAL_ENOMEM, "float64-vector product: scratch allocation failed");
        }
        split_df_kernel<<<blocks_for(b.cols, 256), 256, 0, st>>>(x1, xs, b.cols);
        split_df_kernel<<<blocks_for(b.cols, 256), 256, 0, st>>>(x2, xs + b.cols, b.cols);
        const int64_t nc2 = b.cols / 2;
        const int64_t chunk2 = std::min<int64_t>(nc2, 1024);
        const int64_t units = b.rows * ((nc2 + chunk2 - 1) / chunk2);
        const int64_t grid = std::min<int64_t>((units + 7) / 8, (int64_t)nsm * 3);
        pair_gemv_df_kernel<<<(unsigned)grid, 256, 0, st>>>(reinterpret_cast<const float4*>(S),
                                                           reinterpret_cast<const float4*>(C), b.rows, nc2,
                                                           b.cols / 2, chunk2, xs, xs + b.cols, y1, y2, ar, ai, br,
                                                           bi);
        dfree(xs, st);
        prof_end(st, tok);
        note_launch(3);
        CAL_TRY_CUDA(cudaGetLastError());
        return CAL_OK;
      }
    } else if constexpr (sizeof(MT) == 8) {
      if (b.cols % 2 == 0 && aligned16) {
        int nsm = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int64_t nc2 = b.cols / 2;
        const int64_t chunk2 = std::min<int64_t>(nc2, 1024);
        const int64_t units = b.rows * ((nc2 + chunk2 - 1) / chunk2);
        const int64_t grid = std::min<int64_t>((units + 7) / 8, (int64_t)nsm * 3);
        if (b.S2 && S && C)
          pair_gemv_units_kernel<VT, AT, true><<<(unsigned)std::min<int64_t>(grid, (int64_t)nsm * 2), 256, 0, st>>>(
              reinterpret_cast<const float4*>(S), reinterpret_cast<const float4*>(C), b.rows, nc2, b.cols / 2,
              chunk2, x1, x2, y1, y2, ar, ai, br, bi, reinterpret_cast<const float4*>(b.S2));
        else
          pair_gemv_units_kernel<VT, AT><<<(unsigned)grid, 256, 0, st>>>(
              reinterpret_cast<const float4*>(S), reinterpret_cast<const float4*>(C), b.rows, nc2,
              b.cols / 2, chunk2, x1, x2, y1, y2, ar, ai, br, bi);
        prof_end(st, tok);
        note_launch();
        CAL_TRY_CUDA(cudaGetLastError());
        return CAL_OK;
      }
    }
    constexpr int ROWS = 4;
    const int64_t warps = (b.rows + ROWS - 1) / ROWS;
    pair_gemv_kernel<MT, VT, AT, ROWS><<<blocks_for(warps * 32, 256), 256, 0, st>>>(
        S, C, b.rows, b.cols, b.cols, x1, x2, y1, y2, ar, ai, br, bi);
    prof_end(st, tok);
    note_launch();
  }
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

// ---------------------------------------------------------------------------
// Several right-hand sides on a dense complex64 block pair at once:
//   y1_q += C x1_q + alpha S x2_q,  y2_q += C x2_q + beta S x1_q,  q < nrhs.
// One thread per row walks a 64-column chunk; the chunk of x for G right-hand
// sides is staged in shared memory and read by broadcast, so each matrix entry
// is read once per group of G vectors. AT is the arithmetic: float32 for
// float32 vectors (G = 8), float64 products and sums for float64 vectors
// (G = 4), so that the refinement residual b - A x is exact up to float64
// rounding for the stored complex64 A.
// ---------------------------------------------------------------------------
constexpr int MV_W = 64;

template <typename VT, typename AT, int G>
__global__ void __launch_bounds__(256) pair_gemv_multi_kernel(
    const float2* __restrict__ S, const float2* __restrict__ C, int64_t rows, int64_t cols, int64_t ld,
    const VT* __restrict__ x1, const VT* __restrict__ x2, int64_t xstride, VT* __restrict__ y1,
    VT* __restrict__ y2, int nrhs, AT ar, AT ai, AT br, AT bi) {
  using AT2 = typename std::conditional<sizeof(AT) == 4, float2, double2>::type;
  __shared__ AT2 xsh[2][G][MV_W];
  const int64_t nrb = (rows + 255) / 256;
  const int64_t nch = (cols + MV_W - 1) / MV_W;
  const int ngr = (nrhs + G - 1) / G;
  const int64_t units = nrb * nch * ngr;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int g = (int)(u % ngr);
    const int64_t rest = u / ngr;
    const int64_t ch = rest % nch, rb = rest / nch;
    const int64_t c0 = ch * MV_W;
    const int q0 = g * G;
    const int nc = (int)(cols - c0 < MV_W ? cols - c0 : MV_W);
    __syncthreads();  // the previous unit's readers are done with xsh
    for (int t = threadIdx.x; t < 2 * G * MV_W; t += 256) {
      const int c = t % MV_W, q = (t / MV_W) % G, h = t / (MV_W * G);
      AT2 v = {AT(0), AT(0)};
      if (c < nc && q0 + q < nrhs) {
        const VT xv = (h ? x2 : x1)[(int64_t)(q0 + q) * xstride + c0 + c];
        v = {(AT)xv.x, (AT)xv.y};
      }
      xsh[h][q][c] = v;
    }
    __syncthreads();
    const int64_t row = rb * 256 + threadIdx.x;
    if (row >= rows) continue;
    AT acc[G][8];
#pragma unroll
    for (int q = 0; q < G; ++q)
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[q][k] = AT(0);
    const float2* Sr = S + row * ld + c0;
    const float2* Cr = C + row * ld + c0;
    for (int c = 0; c < nc; ++c) {
      const float2 sf = S ? Sr[c] : make_float2(0.f, 0.f);
      const float2 cf = C ? Cr[c] : make_float2(0.f, 0.f);
      const AT svx = sf.x, svy = sf.y, cvx = cf.x, cvy = cf.y;
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const AT2 a1 = xsh[0][q][c], a2 = xsh[1][q][c];
        acc[q][0] = fma(cvx, a1.x, fma(-cvy, a1.y, acc[q][0]));
        acc[q][1] = fma(cvx, a1.y, fma(cvy, a1.x, acc[q][1]));
        acc[q][2] = fma(svx, a2.x, fma(-svy, a2.y, acc[q][2]));
        acc[q][3] = fma(svx, a2.y, fma(svy, a2.x, acc[q][3]));
        acc[q][4] = fma(cvx, a2.x, fma(-cvy, a2.y, acc[q][4]));
        acc[q][5] = fma(cvx, a2.y, fma(cvy, a2.x, acc[q][5]));
        acc[q][6] = fma(svx, a1.x, fma(-svy, a1.y, acc[q][6]));
        acc[q][7] = fma(svx, a1.y, fma(svy, a1.x, acc[q][7]));
      }
    }
#pragma unroll
    for (int q = 0; q < G; ++q) {
      if (q0 + q >= nrhs) break;
      const AT r1 = acc[q][0] + ar * acc[q][2] - ai * acc[q][3];
      const AT i1 = acc[q][1] + ar * acc[q][3] + ai * acc[q][2];
      const AT r2 = acc[q][4] + br * acc[q][6] - bi * acc[q][7];
      const AT i2 = acc[q][5] + br * acc[q][7] + bi * acc[q][6];
      VT* o1 = y1 + (int64_t)(q0 + q) * xstride + row;
      VT* o2 = y2 + (int64_t)(q0 + q) * xstride + row;
      atomicAdd(&o1->x, (decltype(o1->x))r1);
      atomicAdd(&o1->y, (decltype(o1->y))i1);
      atomicAdd(&o2->x, (decltype(o2->x))r2);
      atomicAdd(&o2->y, (decltype(o2->y))i2);
    }
  }
}

// The same product for float64 vectors in double-float arithmetic (df_mac).
template <int G>
__global__ void __launch_bounds__(256) pair_gemv_multi_df_kernel(
    const float2* __restrict__ S, const float2* __restrict__ C, int64_t rows, int64_t cols, int64_t ld,
    const float4* __restrict__ xs, int64_t xstride, double2* __restrict__ y1, double2* __restrict__ y2, int nrhs,
    double ar, double ai, double br, double bi) {
  // xs: x split into (re hi, re lo, im hi, im lo), [q][h][cols]; y stride xstride
  __shared__ float4 xsh[2][G][MV_W];
  const int64_t nrb = (rows + 255) / 256;
  const int64_t nch = (cols + MV_W - 1) / MV_W;
  const int ngr = (nrhs + G - 1) / G;
  const int64_t units = nrb * nch * ngr;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int g = (int)(u % ngr);
    const int64_t rest = u / ngr;
    const int64_t ch = rest % nch, rb = rest / nch;
    const int64_t c0 = ch * MV_W;
    const int q0 = g * G;
    const int nc = (int)(cols - c0 < MV_W ? cols - c0 : MV_W);
    __syncthreads();  // the previous unit's readers are done with xsh
    for (int t = threadIdx.x; t < 2 * G * MV_W; t += 256) {
      const int c = t % MV_W, q = (t / MV_W) % G, h = t / (MV_W * G);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (c < nc && q0 + q < nrhs) v = xs[((int64_t)(q0 + q) * 2 + h) * cols + c0 + c];
      xsh[h][q][c] = v;
    }
    __syncthreads();
    const int64_t row = rb * 256 + threadIdx.x;
    if (row >= rows) continue;
    float hi[G][8], lo[G][8];
#pragma unroll
    for (int q = 0; q < G; ++q)
#pragma unroll
      for (int k = 0; k < 8; ++k) hi[q][k] = lo[q][k] = 0.0f;
    const float2* Sr = S + row * ld + c0;
    const float2* Cr = C + row * ld + c0;
    for (int c = 0; c < nc; ++c) {
      const float2 sf = S ? Sr[c] : make_float2(0.f, 0.f);
      const float2 cf = C ? Cr[c] : make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const float4 a1 = xsh[0][q][c], a2 = xsh[1][q][c];
        // C x1
        df_mac(hi[q][0], lo[q][0], cf.x, a1.x, a1.y); df_mac(hi[q][0], lo[q][0], -cf.y, a1.z, a1.w);
        df_mac(hi[q][1], lo[q][1], cf.x, a1.z, a1.w); df_mac(hi[q][1], lo[q][1], cf.y, a1.x, a1.y);
        // S x2
        df_mac(hi[q][2], lo[q][2], sf.x, a2.x, a2.y); df_mac(hi[q][2], lo[q][2], -sf.y, a2.z, a2.w);
        df_mac(hi[q][3], lo[q][3], sf.x, a2.z, a2.w); df_mac(hi[q][3], lo[q][3], sf.y, a2.x, a2.y);
        // C x2
        df_mac(hi[q][4], lo[q][4], cf.x, a2.x, a2.y); df_mac(hi[q][4], lo[q][4], -cf.y, a2.z, a2.w);
        df_mac(hi[q][5], lo[q][5], cf.x, a2.z, a2.w); df_mac(hi[q][5], lo[q][5], cf.y, a2.x, a2.y);
        // S x1
        df_mac(hi[q][6], lo[q][6], sf.x, a1.x, a1.y); df_mac(hi[q][6], lo[q][6], -sf.y, a1.z, a1.w);
        df_mac(hi[q][7], lo[q][7], sf.x, a1.z, a1.w); df_mac(hi[q][7], lo[q][7], sf.y, a1.x, a1.y);
      }
    }
#pragma unroll
    for (int q = 0; q < G; ++q) {
      if (q0 + q >= nrhs) break;
      double acc[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = (double)hi[q][k] + (double)lo[q][k];
      const double r1 = acc[0] + ar * acc[2] - ai * acc[3];
      const double i1 = acc[1] + ar * acc[3] + ai * acc[2];
      const double r2 = acc[4] + br * acc[6] - bi * acc[7];
      const double i2 = acc[5] + br * acc[7] + bi * acc[6];
      double2* o1 = y1 + (int64_t)(q0 + q) * xstride + row;
      double2* o2 = y2 + (int64_t)(q0 + q) * xstride + row;
      atomicAdd(&o1->x, r1);
      atomicAdd(&o1->y, i1);
      atomicAdd(&o2->x, r2);
      atomicAdd(&o2->y, i2);
    }
  }
}

int pair_apply_multi(const BlockRef& b, int vec_prec, const void* x, void* y, int64_t n, int nrhs, double ar,
                     double ai, double br, double bi, int n_sm, cudaStream_t st) {
  if (b.precision != CAL_FP32 || b.rowptr) return fail(CAL_EINVAL, "multi-vector GEMV: dense float32 blocks only");
  const int G = vec_prec == CAL_FP64 ? 4 : 8;
  const int64_t units = ((b.rows + 255) / 256) * ((b.cols + MV_W - 1) / MV_W) * ((nrhs + G - 1) / G);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(units, (int64_t)n_sm * 8));
  const double bytes = (double)b.rows * b.cols * 8.0 * ((b.S ? 1 : 0) + (b.C ? 1 : 0));
  const int tok = prof_begin(st, "pair_gemv", bytes * ((nrhs + G - 1) / G));
  const float2* S = reinterpret_cast<const float2*>(b.S);
  const float2* C = reinterpret_cast<const float2*>(b.C);
  if (vec_prec == CAL_FP64) {
    const double2* xx = (const double2*)x;
    double2* yy = (double2*)y;
    // x split once into (hi, lo) floats; stream-ordered scratch
    float4* xs = nullptr;
    const int64_t nxs = 2 * b.cols * nrhs;
    if (dalloc((void**)&xs, std::max<int64_t>(nxs, 1) * sizeof(float4), st) != cudaSuccess) {
      prof_end(st, tok);
      return fail(CAL_ENOMEM, "multi-vector GEMV: scratch allocation failed");
    }
    split_df_multi_kernel<<<(unsigned)((nxs + 255) / 256), 256, 0, st>>>(xx, n, b.col_off, b.cols, nrhs, xs);
    note_launch();
    pair_gemv_multi_df_kernel<4><<<grid, 256, 0, st>>>(S, C, b.rows, b.cols, b.cols, xs, 2 * n, yy + b.row_off,
                                                      yy + n + b.row_off, nrhs, ar, ai, br, bi);
    dfree(xs, st);
  } else {
    const float2* xx = (const float2*)x;
    float2* yy = (float2*)y;
    pair_gemv_multi_kernel<float2, float, 8><<<grid, 256, 0, st>>>(
        S, C, b.rows, b.cols, b.cols, xx + b.col_off, xx + n + b.col_off, 2 * n, yy + b.row_off,
        yy + n + b.row_off, nrhs, (float)ar, (float)ai, (float)br, (float)bi);
  }
  prof_end(st, tok);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

int pair_apply(const BlockRef& b, int vec_prec, const void* x, void* y, int64_t n, double ar,
               double ai, double br, double bi, cudaStream_t st) {
  if (b.precision == CAL_FP64)
    return pair_apply_t<double2, double2, double2>(b, (const double2*)x, (double2*)y, n, ar, ai, br, bi, st);
  if (vec_prec == CAL_FP64)
    return pair_apply_t<float2, double2, double2>(b, (const double2*)x, (double2*)y, n, ar, ai, br, bi, st);
  return pair_apply_t<float2, float2, float2>(b, (const float2*)x, (float2*)y, n, ar, ai, br, bi, st);
}

int zero_vec(void* y, int prec, int64_t n, cudaStream_t st) {
  note_launch();
  if (prec == CAL_FP64) zero_kernel<double2><<<blocks_for(n, 256), 256, 0, st>>>((double2*)y, n);
  else zero_kernel<float2><<<blocks_for(n, 256), 256, 0, st>>>((float2*)y, n);
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

int convert_vec(const void* a, int pa, void* b, int pb, int64_t n, double scale, cudaStream_t st) {
  note_launch();
  const unsigned g = blocks_for(n, 256);
  if (pa == CAL_FP64 && pb == CAL_FP32) convert_kernel<double2, float2><<<g, 256, 0, st>>>((const double2*)a, (float2*)b, n, scale);
  else if (pa == CAL_FP32 && pb == CAL_FP64) convert_kernel<float2, double2><<<g, 256, 0, st>>>((const float2*)a, (double2*)b, n, scale);
  else if (pa == CAL_FP64) convert_kernel<double2, double2><<<g, 256, 0, st>>>((const double2*)a, (double2*)b, n, scale);
  else convert_kernel<float2, float2><<<g, 256, 0, st>>>((const float2*)a, (float2*)b, n, scale);
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

// y[i] += alpha sum_j X[i ld + j] x[j], i < rows, j < cols (float64, warp per row)
__global__ void gemv_acc_kernel(const double2* __restrict__ X, int64_t ld, int64_t rows, int64_t cols,
                                const double2* __restrict__ x, double2* __restrict__ y, double ar, double ai) {
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= rows) return;
  const double2* Xr = X + r * ld;
  double sr = 0, si = 0;
  for (int64_t j = lane; j < cols; j += 32) {
    const double2 m = Xr[j], v = x[j];
    sr += m.x * v.x - m.y * v.y;
    si += m.x * v.y + m.y * v.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) {
    y[r].x += ar * sr - ai * si;
    y[r].y += ar * si + ai * sr;
  }
}

int gemv_acc(const double2* X, int64_t ld, int64_t rows, int64_t cols, const double2* x, double2* y,
             std::complex<double> alpha, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return CAL_OK;
  const int tok = prof_begin(st, "pair_gemv", (double)rows * cols * 16.0);
  gemv_acc_kernel<<<blocks_for(rows * 32, 256), 256, 0, st>>>(X, ld, rows, cols, x, y, alpha.real(), alpha.imag());
  prof_end(st, tok);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

int single_apply(const Op& op, const void* X, const void* x, void* y, int64_t nrhs, cudaStream_t st) {
  for (int64_t q = 0; q < nrhs; ++q) {
    note_launch();
    const unsigned g = blocks_for(op.rows * 32, 256);
    if (op.precision == CAL_FP64) {
      const double2* xx = (const double2*)x + q * op.cols;
      double2* yy = (double2*)y + q * op.rows;
      if (op.format == CAL_DENSE) gemv_kernel<double2><<<g, 256, 0, st>>>((const double2*)X, op.rows, op.cols, xx, yy);
      else spmv_kernel<double2><<<g, 256, 0, st>>>((const double2*)X, op.d_rowptr, op.d_col, op.rows, xx, yy);
    } else {
      const float2* xx = (const float2*)x + q * op.cols;
      float2* yy = (float2*)y + q * op.rows;
      if (op.format == CAL_DENSE) gemv_kernel<float2><<<g, 256, 0, st>>>((const float2*)X, op.rows, op.cols, xx, yy);
      else spmv_kernel<float2><<<g, 256, 0, st>>>((const float2*)X, op.d_rowptr, op.d_col, op.rows, xx, yy);
    }
  }
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

// ---------------------------------------------------------------------------
// GMRES helpers (float64), batched over right-hand sides (blockIdx.y = q):
// classical Gram–Schmidt with one reorthogonalisation, Givens rotations and
// the triangular solve on the device.
// ---------------------------------------------------------------------------
// h[q][i] += V_q,i^H w_q for i < m. Each thread takes E elements of the column
// (blockDim.x apart) and sums their products before the warp reduction: the
// float64 shuffle adds, not the products, dominated at one element per thread
// (float64 runs at 1/64 of the float32 rate here). Per basis vector the
// block's sum goes to h with one atomic.
template <int E>
__global__ void __launch_bounds__(256) multi_dot_kernel(const double2* __restrict__ V, int64_t bV, int m,
                                                        const double2* __restrict__ w, int64_t n, double2* h,
                                                        int64_t bh) {
  __shared__ double sr[8][32], si[8][32];
  const int q = blockIdx.y;
  V += q * bV;
  w += q * n;
  h += q * bh;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t k0 = (int64_t)blockIdx.x * blockDim.x * E + threadIdx.x;
  double2 wk[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int64_t k = k0 + (int64_t)e * blockDim.x;
    wk[e] = k < n ? w[k] : double2{0, 0};
  }
  for (int i = 0; i < m; ++i) {
    const double2* Vi = V + (size_t)i * n;
    double ar = 0, ai = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int64_t k = k0 + (int64_t)e * blockDim.x;
      if (k < n) {
        const double2 v = Vi[k];
        ar = fma(v.x, wk[e].x, ar);
        ar = fma(v.y, wk[e].y, ar);
        ai = fma(v.x, wk[e].y, ai);
        ai = fma(-v.y, wk[e].x, ai);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) { sr[wid][i & 31] = ar; si[wid][i & 31] = ai; }
    if ((i & 31) == 31 || i == m - 1) {
      __syncthreads();
      const int base = i & ~31;
      const int cnt = i - base + 1;
      if (threadIdx.x < cnt) {
        double tr = 0, ti = 0;
        for (int qq = 0; qq < (int)(blockDim.x >> 5); ++qq) { tr += sr[qq][threadIdx.x]; ti += si[qq][threadIdx.x]; }
        atomicAdd(&h[base + threadIdx.x].x, tr);
        atomicAdd(&h[base + threadIdx.x].y, ti);
      }
      __syncthreads();
    }
  }
}

__global__ void multi_axpy_kernel(const double2* __restrict__ V, int64_t bV, int m,
                                  const double2* __restrict__ h, int64_t bh, double2* __restrict__ w, int64_t n) {
  // w_q -= sum_i h_q,i V_q,i
  const int q = blockIdx.y;
  V += q * bV;
  h += q * bh;
  w += q * n;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double2 acc = w[k];
  for (int i = 0; i < m; ++i) {
    const double2 v = V[(size_t)i * n + k], c = h[i];
    acc.x -= c.x * v.x - c.y * v.y;
    acc.y -= c.x * v.y + c.y * v.x;
  }
  w[k] = acc;
}

__global__ void norm2_kernel(const double2* __restrict__ w, int64_t n, double* out, int64_t bout) {
  const int q = blockIdx.y;
  w += q * n;
  double part[1] = {0.0};
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) part[0] = w[k].x * w[k].x + w[k].y * w[k].y;
  block_accumulate<1>(part, out + q * bout);
}

__global__ void scale_kernel(const double2* __restrict__ w, int64_t bw, int64_t n, const double* nrm2,
                             int64_t bn, double2* __restrict__ out, int64_t bout) {
  const int q = blockIdx.y;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double nn = nrm2[q * bn];
  const double s = nn > 0 ? 1.0 / sqrt(nn) : 0.0;
  const double2 v = w[q * bw + k];
  out[q * bout + k] = {v.x * s, v.y * s};
}

// Arnoldi column j finished for every q: H[0..j][j] = h1 + h2, H[j+1][j] = ||w||;
// apply the previous rotations, build the new one, update g, report |g_{j+1}|.
__global__ void givens_kernel(double2* H, int ldh, int64_t bH, int j, const double2* h1, const double2* h2,
                              int64_t bh, const double* wn2, int64_t bwn, double2* cs, double2* sn, int64_t bcs,
                              double2* g, int64_t bg, double* res_out, int64_t bres, int nrhs) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nrhs) return;
  double2* col = H + q * bH + (size_t)j * ldh;
  h1 += q * bh;
  h2 += q * bh;
  cs += q * bcs;
  sn += q * bcs;
  g += q * bg;
  for (int i = 0; i <= j; ++i) col[i] = {h1[i].x + h2[i].x, h1[i].y + h2[i].y};
  col[j + 1] = {sqrt(wn2[q * bwn]), 0.0};
  for (int i = 0; i < j; ++i) {
    // [c s; -conj(s) c] with real c
    const double c = cs[i].x;
    const double2 s = sn[i];
    const double2 a = col[i], b = col[i + 1];
    col[i] = {c * a.x + (s.x * b.x - s.y * b.y), c * a.y + (s.x * b.y + s.y * b.x)};
    col[i + 1] = {-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y};
  }
  const double2 a = col[j], b = col[j + 1];
  const double na = sqrt(a.x * a.x + a.y * a.y), nb = sqrt(b.x * b.x + b.y * b.y);
  const double den = sqrt(na * na + nb * nb);
  double c;
  double2 s;
  if (na == 0.0) { c = 0.0; s = {1.0, 0.0}; }
  else {
    c = na / den;
    // s = (a/|a|) conj(b) / den
    const double ux = a.x / na, uy = a.y / na;
    s = {(ux * b.x + uy * b.y) / den, (uy * b.x - ux * b.y) / den};
  }
  cs[j] = {c, 0.0};
  sn[j] = s;
  col[j] = {c * a.x + (s.x * b.x - s.y * b.y), c * a.y + (s.x * b.y + s.y * b.x)};
  col[j + 1] = {0.0, 0.0};
  const double2 gj = g[j];
  g[j + 1] = {-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x)};
  g[j] = {c * gj.x, c * gj.y};
  res_out[q * bres] = sqrt(g[j + 1].x * g[j + 1].x + g[j + 1].y * g[j + 1].y);
}

// y = H[0..m)[0..m)^-1 g (upper triangular), then x += V y (one right-hand side)
__global__ void backsolve_kernel(const double2* H, int ldh, int m, const double2* g, double2* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = m - 1; i >= 0; --i) {
    double2 acc = g[i];
    for (int q = i + 1; q < m; ++q) {
      const double2 h = H[(size_t)q * ldh + i], v = y[q];
      acc.x -= h.x * v.x - h.y * v.y;
      acc.y -= h.x * v.y + h.y * v.x;
    }
    const double2 d = H[(size_t)i * ldh + i];
    const double dd = d.x * d.x + d.y * d.y;
    y[i] = {(acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd};
  }
}

__global__ void combine_kernel(const double2* __restrict__ V, int64_t ldv, int m,
                               const double2* __restrict__ y, double2* __restrict__ x, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double2 acc = x[k];
  for (int i = 0; i < m; ++i) {
    const double2 v = V[(size_t)i * ldv + k], c = y[i];
    acc.x += c.x * v.x - c.y * v.y;
    acc.y += c.x * v.y + c.y * v.x;
  }
  x[k] = acc;
}

__global__ void axpby_kernel(const double2* a, double sa, const double2* b, double sb, double2* out,
                             int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = {sa * a[k].x + sb * b[k].x, sa * a[k].y + sb * b[k].y};
}

__global__ void gather_kernel(const double2* __restrict__ src, int64_t bsrc, double2* __restrict__ dst, int64_t n) {
  const int q = blockIdx.y;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) dst[q * n + k] = src[q * bsrc + k];
}

int gmres_cgs_step(const double2* V, int64_t bV, int64_t n, int j, double2* w, double2* h1, double2* h2,
                   int64_t bh, double* wn2, int64_t bwn, int nrhs, cudaStream_t st) {
  const dim3 g(blocks_for(n, 256), nrhs);
  // two dot/axpy passes over the j+1 basis vectors of every column
  const int tok = prof_begin(st, "gmres_cgs", 4.0 * (j + 1) * (double)n * sizeof(double2) * nrhs);
  CAL_TRY_CUDA(cudaMemsetAsync(h1, 0, nrhs * bh * sizeof(double2), st));
  CAL_TRY_CUDA(cudaMemsetAsync(h2, 0, nrhs * bh * sizeof(double2), st));
  for (int q = 0; q < nrhs; ++q) CAL_TRY_CUDA(cudaMemsetAsync(wn2 + q * bwn, 0, sizeof(double), st));
  // elements per thread of the dot products: as many as keep about four
  // blocks per SM busy (one for short columns of a single right-hand side)
  int dev = 0, n_sm = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(CAL_ECUDA, "gmres: device query failed");
  int E = 8;
  while (E > 1 && (int64_t)blocks_for(n, 256 * E) * nrhs < 4LL * n_sm) E >>= 1;
  const dim3 gd(blocks_for(n, 256 * E), nrhs);
  auto dot = E == 8 ? multi_dot_kernel<8> : E == 4 ? multi_dot_kernel<4> : E == 2 ? multi_dot_kernel<2> : multi_dot_kernel<1>;
  dot<<<gd, 256, 0, st>>>(V, bV, j + 1, w, n, h1, bh);
  multi_axpy_kernel<<<g, 256, 0, st>>>(V, bV, j + 1, h1, bh, w, n);
  dot<<<gd, 256, 0, st>>>(V, bV, j + 1, w, n, h2, bh);
  multi_axpy_kernel<<<g, 256, 0, st>>>(V, bV, j + 1, h2, bh, w, n);
  norm2_kernel<<<g, 256, 0, st>>>(w, n, wn2, bwn);
  prof_end(st, tok);
  note_launch(5);
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

int gmres_givens(double2* H, int ldh, int64_t bH, int j, const double2* h1, const double2* h2, int64_t bh,
                 const double* wn2, int64_t bwn, double2* cs, double2* sn, int64_t bcs, double2* g, int64_t bg,
                 double* res, int64_t bres, int nrhs, cudaStream_t st) {
  givens_kernel<<<(nrhs + 31) / 32, 32, 0, st>>>(H, ldh, bH, j, h1, h2, bh, wn2, bwn, cs, sn, bcs, g, bg, res,
                                                 bres, nrhs);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

int gmres_scale(const double2* w, int64_t bw, int64_t n, const double* nrm2, int64_t bn, double2* out,
                int64_t bout, int nrhs, cudaStream_t st) {
  scale_kernel<<<dim3(blocks_for(n, 256), nrhs), 256, 0, st>>>(w, bw, n, nrm2, bn, out, bout);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

int gmres_update(const double2* H, int ldh, int m, const double2* g, double2* y, const double2* V,
                 int64_t n, double2* x, cudaStream_t st) {
  backsolve_kernel<<<1, 32, 0, st>>>(H, ldh, m, g, y);
  combine_kernel<<<blocks_for(n, 256), 256, 0, st>>>(V, n, m, y, x, n);
  note_launch(2);
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

int vec_norm2(const double2* w, int64_t n, double* out, int64_t bout, int nrhs, cudaStream_t st) {
  for (int q = 0; q < nrhs; ++q) CAL_TRY_CUDA(cudaMemsetAsync(out + q * bout, 0, sizeof(double), st));
  norm2_kernel<<<dim3(blocks_for(n, 256), nrhs), 256, 0, st>>>(w, n, out, bout);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

int vec_axpby(const double2* a, double sa, const double2* b, double sb, double2* out, int64_t n,
              cudaStream_t st) {
  axpby_kernel<<<blocks_for(n, 256), 256, 0, st>>>(a, sa, b, sb, out, n);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

int vec_gather(const double2* src, int64_t bsrc, double2* dst, int64_t n, int nrhs, cudaStream_t st) {
  gather_kernel<<<dim3(blocks_for(n, 256), nrhs), 256, 0, st>>>(src, bsrc, dst, n);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

// ---------------------------------------------------------------------------
// A11: right-hand side b = [<u1, RWG_i>; <u2, RWG_i>] with
// u1 = E x n, u2 = (k/mu) (d x p) e^{ik d.x} x n, <a x n, phi> = -int a.phi,
// 6-point rule per triangle, float64.
// ---------------------------------------------------------------------------
// mode 0: the tested incident traces b = (-int phi.E, -(k/mu) int phi.(d x p) e^{ik d.x})
// (the identity pairing of eq. dualpairingGammam with tangential test functions);
// mode 1: the L2 loads (int phi.(E x n), (k/mu) int phi.((d x p) e^{ik d.x} x n)) of the
// projection of u^inc onto RWG, written as F.(n x phi)
__global__ void rhs_kernel(const TriD* __restrict__ tri, const int* __restrict__ slot_edge,
                           const double* __restrict__ slot_sw, int nslot, int64_t nt, const double* inc,
                           int nrhs, double k, double mu, Rules6 rl, int64_t ne,
                           double2* __restrict__ b, int mode) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (t >= nt || q >= nrhs) return;
  const TriD T = tri[t];
  const double d[3] = {inc[6 * q], inc[6 * q + 1], inc[6 * q + 2]};
  const double p[3] = {inc[6 * q + 3], inc[6 * q + 4], inc[6 * q + 5]};
  const double dxp[3] = {d[1] * p[2] - d[2] * p[1], d[2] * p[0] - d[0] * p[2], d[0] * p[1] - d[1] * p[0]};
  // unit outward normal (vertices counter-clockwise seen from outside)
  double nrm[3];
  {
    double e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
      e1[c] = T.off[1][c] - T.off[0][c];
      e2[c] = T.off[2][c] - T.off[0][c];
    }
    nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
    nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
    nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double il = 1.0 / sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    for (int c = 0; c < 3; ++c) nrm[c] *= il;
  }
  const double sgn = mode == 0 ? -1.0 : 1.0;
  constexpr int MAXS = 16;  // slots per triangle (BC: the valence)
  double acc1[MAXS][2] = {}, acc2[MAXS][2] = {};
  for (int u = 0; u < 6; ++u) {
    double xi[3];
    for (int c = 0; c < 3; ++c)
      xi[c] = rl.b[3 * u] * T.off[0][c] + rl.b[3 * u + 1] * T.off[1][c] + rl.b[3 * u + 2] * T.off[2][c];
    double ph = 0;
    for (int c = 0; c < 3; ++c) ph += d[c] * (T.c[c] + xi[c]);
    double s, co;
    sincos(k * ph, &s, &co);
    const double w = rl.w[u] * T.area;
    for (int a = 0; a < nslot; ++a) {
      const double* sw = slot_sw + ((size_t)t * nslot + a) * 4;
      double phi[3];
      for (int c = 0; c < 3; ++c) phi[c] = sw[0] * xi[c] + sw[1 + c];
      if (mode == 1) {  // n x phi
        const double v[3] = {nrm[1] * phi[2] - nrm[2] * phi[1], nrm[2] * phi[0] - nrm[0] * phi[2],
                             nrm[0] * phi[1] - nrm[1] * phi[0]};
        for (int c = 0; c < 3; ++c) phi[c] = v[c];
      }
      const double e1 = p[0] * phi[0] + p[1] * phi[1] + p[2] * phi[2];
      const double e2 = dxp[0] * phi[0] + dxp[1] * phi[1] + dxp[2] * phi[2];
      acc1[a][0] += sgn * w * co * e1;
      acc1[a][1] += sgn * w * s * e1;
      acc2[a][0] += sgn * (k / mu) * w * co * e2;
      acc2[a][1] += sgn * (k / mu) * w * s * e2;
    }
  }
  for (int a = 0; a < nslot; ++a) {
    const int e = slot_edge[(size_t)t * nslot + a];
    if (e < 0) continue;
    double2* bq = b + (size_t)q * 2 * ne;
    atomicAdd(&bq[e].x, acc1[a][0]);
    atomicAdd(&bq[e].y, acc1[a][1]);
    atomicAdd(&bq[ne + e].x, acc2[a][0]);
    atomicAdd(&bq[ne + e].y, acc2[a][1]);
  }
}

// Far field E_inf(xh) = -(ik/4pi) [xh x Ja - xh x (xh x Jb)],
// Ja = int a e^{-ik xh.y}, Jb = (mu/k) int (sum d_e RWG_e) e^{-ik xh.y}.
int launch_rhs(const Space& rwg, const double* d_inc, int nrhs, double k, double mu, double2* d_b,
               cudaStream_t st, int mode) {
  Rules6 rl = rules6();
  CAL_TRY_CUDA(cudaMemsetAsync(d_b, 0, (size_t)nrhs * 2 * rwg.nbasis * sizeof(double2), st));
  dim3 grid(blocks_for(rwg.ntri, 128), nrhs);
  if (rwg.nslot > 16) return fail(CAL_EINVAL, "right-hand side: %d slots per triangle (at most 16)", rwg.nslot);
  rhs_kernel<<<grid, 128, 0, st>>>(rwg.d_triD, rwg.d_slot_edge, rwg.d_slot_swd, rwg.nslot, rwg.ntri, d_inc, nrhs,
                                   k, mu, rl, rwg.nbasis, d_b, mode);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

// RWG mass matrix M_ij = int phi_i . phi_j (degree-2 integrand: the 6-point rule
// is exact), accumulated per triangle into a CSR pattern that holds every pair
// of edges of one triangle; the column of an entry is found by a scan of its row
__global__ void rwg_mass_kernel(const TriD* __restrict__ tri, const int* __restrict__ slot_edge,
                                const double* __restrict__ slot_sw, int64_t nt, Rules6 rl,
                                const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                                double* __restrict__ val) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const TriD T = tri[t];
  for (int a = 0; a < 3; ++a) {
    const int ea = slot_edge[3 * t + a];
    if (ea < 0) continue;
    const double* sa = slot_sw + (3 * t + a) * 4;
    for (int b = 0; b < 3; ++b) {
      const int eb = slot_edge[3 * t + b];
      if (eb < 0) continue;
      const double* sb = slot_sw + (3 * t + b) * 4;
      double m = 0.0;
      for (int u = 0; u < 6; ++u) {
        double dot = 0.0;
        for (int c = 0; c < 3; ++c) {
          const double xi = rl.b[3 * u] * T.off[0][c] + rl.b[3 * u + 1] * T.off[1][c] + rl.b[3 * u + 2] * T.off[2][c];
          dot += (sa[0] * xi + sa[1 + c]) * (sb[0] * xi + sb[1 + c]);
        }
        m += rl.w[u] * dot;
      }
      m *= T.area;
      for (int64_t q = rowptr[ea]; q < rowptr[ea + 1]; ++q)
        if (col[q] == eb) {
          atomicAdd(val + q, m);
          break;
        }
    }
  }
}

int launch_rwg_mass(const Space& rwg, const int64_t* rowptr, const int* col, double* val, cudaStream_t st) {
  Rules6 rl = rules6();
  rwg_mass_kernel<<<blocks_for(rwg.ntri, 128), 128, 0, st>>>(rwg.d_triD, rwg.d_slot_edge, rwg.d_slot_swd,
                                                             rwg.ntri, rl, rowptr, col, val);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

// Far field in two passes: the surface currents at the 6 points of every
// triangle, J_a = sum_slots x1 phi and J_b = (mu/k) sum_slots x2 phi times the
// rule weight and area (independent of the direction), then per direction one
// sum of J e^{-ik xhat . x} over all points. AT: float64, or float32 for a
// float32-bulk solution (phases |k xhat . x| stay small for the meshes here;
// the far field is compared at 1e-4).
template <typename AT>
struct FfPoint {
  AT x[3];
  AT j[12];  // J_a (re, im) per component, then J_b
};

// comps: bit 1 takes J_a from the first half of x, bit 2 J_b from the second
// (the mixed discretisation expands the two traces in different spaces);
// points of right-hand side q at pts + q * stride
template <typename AT>
__global__ void ff_points_kernel(const TriD* __restrict__ tri, const int* __restrict__ slot_edge,
                                 const double* __restrict__ slot_sw, int nslot, int64_t nt,
                                 const double2* __restrict__ x, int64_t ne, double k, double mu, Rules6 rl, int comps,
                                 int64_t stride, FfPoint<AT>* __restrict__ pts) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (t >= nt) return;
  const TriD T = tri[t];
  const double2* xq = x + (size_t)q * 2 * ne;
  constexpr int MAXS = 16;
  double ca[MAXS][2], cb[MAXS][2];
  for (int a = 0; a < nslot; ++a) {
    const int e = slot_edge[(size_t)t * nslot + a];
    const bool ok = e >= 0;
    ca[a][0] = ok && (comps & 1) ? xq[e].x : 0.0; ca[a][1] = ok && (comps & 1) ? xq[e].y : 0.0;
    cb[a][0] = ok && (comps & 2) ? xq[ne + e].x * (mu / k) : 0.0;
    cb[a][1] = ok && (comps & 2) ? xq[ne + e].y * (mu / k) : 0.0;
  }
  for (int u = 0; u < 6; ++u) {
    double xi[3];
    for (int c = 0; c < 3; ++c)
      xi[c] = rl.b[3 * u] * T.off[0][c] + rl.b[3 * u + 1] * T.off[1][c] + rl.b[3 * u + 2] * T.off[2][c];
    const double w = rl.w[u] * T.area;
    double J[12] = {};
    for (int a = 0; a < nslot; ++a) {
      const double* sw = slot_sw + ((size_t)t * nslot + a) * 4;
      for (int c = 0; c < 3; ++c) {
        const double phi = w * (sw[0] * xi[c] + sw[1 + c]);
        J[2 * c] += ca[a][0] * phi; J[2 * c + 1] += ca[a][1] * phi;
        J[6 + 2 * c] += cb[a][0] * phi; J[6 + 2 * c + 1] += cb[a][1] * phi;
      }
    }
    FfPoint<AT>& o = pts[(size_t)q * stride + t * 6 + u];
    for (int c = 0; c < 3; ++c) o.x[c] = (AT)(T.c[c] + xi[c]);
    for (int c = 0; c < 12; ++c) o.j[c] = (AT)J[c];
  }
}

template <typename AT>
__global__ void ff_sum_kernel(const FfPoint<AT>* __restrict__ pts, int64_t npts, const double* dirs, int64_t ndir,
                              double k, double2* out) {
  const int64_t dq = blockIdx.x;  // direction
  const int q = blockIdx.y;       // right-hand side
  const double xh[3] = {dirs[3 * dq], dirs[3 * dq + 1], dirs[3 * dq + 2]};
  const AT kx[3] = {(AT)(-k * xh[0]), (AT)(-k * xh[1]), (AT)(-k * xh[2])};
  const FfPoint<AT>* P = pts + (size_t)q * npts;
  AT acc[12] = {};
  for (int64_t p = threadIdx.x; p < npts; p += blockDim.x) {
    const FfPoint<AT>& o = P[p];
    const AT ph = kx[0] * o.x[0] + kx[1] * o.x[1] + kx[2] * o.x[2];
    AT s, c;
    if constexpr (sizeof(AT) == 4) sincosf(ph, &s, &c);
    else sincos(ph, &s, &c);
#pragma unroll
    for (int m = 0; m < 6; ++m) {  // (J_re + i J_im)(c + i s)
      acc[2 * m] += o.j[2 * m] * c - o.j[2 * m + 1] * s;
      acc[2 * m + 1] += o.j[2 * m] * s + o.j[2 * m + 1] * c;
    }
  }
  __shared__ double sh[12][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = 0; c < 12; ++c) {
    double v = (double)acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[c][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double J[12];
    for (int c = 0; c < 12; ++c) {
      J[c] = 0;
      for (int q2 = 0; q2 < (int)(blockDim.x >> 5); ++q2) J[c] += sh[c][q2];
    }
    double Ja[3][2], Jb[3][2], A[3][2], B1[3][2], B[3][2];
    for (int c = 0; c < 3; ++c) {
      Ja[c][0] = J[2 * c]; Ja[c][1] = J[2 * c + 1];
      Jb[c][0] = J[6 + 2 * c]; Jb[c][1] = J[6 + 2 * c + 1];
    }
    for (int z = 0; z < 2; ++z) {
      // A = xh x Ja ; B1 = xh x Jb ; B = xh x B1
      A[0][z] = xh[1] * Ja[2][z] - xh[2] * Ja[1][z];
      A[1][z] = xh[2] * Ja[0][z] - xh[0] * Ja[2][z];
      A[2][z] = xh[0] * Ja[1][z] - xh[1] * Ja[0][z];
      B1[0][z] = xh[1] * Jb[2][z] - xh[2] * Jb[1][z];
      B1[1][z] = xh[2] * Jb[0][z] - xh[0] * Jb[2][z];
      B1[2][z] = xh[0] * Jb[1][z] - xh[1] * Jb[0][z];
    }
    for (int z = 0; z < 2; ++z) {
      B[0][z] = xh[1] * B1[2][z] - xh[2] * B1[1][z];
      B[1][z] = xh[2] * B1[0][z] - xh[0] * B1[2][z];
      B[2][z] = xh[0] * B1[1][z] - xh[1] * B1[0][z];
    }
    const double f = k / (4.0 * 3.14159265358979323846);
    for (int c = 0; c < 3; ++c) {
      const double vr = A[c][0] - B[c][0], vi = A[c][1] - B[c][1];
      // -(i f) (vr + i vi) = f vi - i f vr
      out[((size_t)q * ndir + dq) * 3 + c] = {f * vi, -f * vr};
    }
  }
}

template <typename AT>
static int farfield_t(const Space& rwg, const double2* d_x, int nrhs, const double* d_dirs, int64_t ndir, double k,
                      double mu, double2* d_out, cudaStream_t st) {
  Rules6 rl = rules6();
  const int64_t npts = rwg.ntri * 6;
  FfPoint<AT>* pts = nullptr;
  if (dalloc((void**)&pts, (size_t)nrhs * npts * sizeof(FfPoint<AT>), st) != cudaSuccess)
    return fail(CAL_ENOMEM, "far field: scratch allocation failed");
  ff_points_kernel<AT><<<dim3(blocks_for(rwg.ntri, 128), nrhs), 128, 0, st>>>(
      rwg.d_triD, rwg.d_slot_edge, rwg.d_slot_swd, rwg.nslot, rwg.ntri, d_x, rwg.nbasis, k, mu, rl, 3, npts, pts);
  ff_sum_kernel<AT><<<dim3((unsigned)ndir, nrhs), 256, 0, st>>>(pts, npts, d_dirs, ndir, k, d_out);
  note_launch(2);
  dfree(pts, st);
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

// the mixed discretisation: u_1 in RWG (the primal space), u_2 in BC
static int farfield_mixed_t(const Space& rwg, const Space& bc, const double2* d_x, int nrhs, const double* d_dirs,
                            int64_t ndir, double k, double mu, double2* d_out, cudaStream_t st) {
  if (bc.nslot > 16) return fail(CAL_EINVAL, "far field: %d slots per triangle (at most 16)", bc.nslot);
  Rules6 rl = rules6();
  const int64_t n1 = rwg.ntri * 6, npts = n1 + bc.ntri * 6;
  FfPoint<double>* pts = nullptr;
  if (dalloc((void**)&pts, (size_t)nrhs * npts * sizeof(FfPoint<double>), st) != cudaSuccess)
    return fail(CAL_ENOMEM, "far field: scratch allocation failed");
  ff_points_kernel<double><<<dim3(blocks_for(rwg.ntri, 128), nrhs), 128, 0, st>>>(
      rwg.d_triD, rwg.d_slot_edge, rwg.d_slot_swd, rwg.nslot, rwg.ntri, d_x, rwg.nbasis, k, mu, rl, 1, npts, pts);
  ff_points_kernel<double><<<dim3(blocks_for(bc.ntri, 128), nrhs), 128, 0, st>>>(
      bc.d_triD, bc.d_slot_edge, bc.d_slot_swd, bc.nslot, bc.ntri, d_x, bc.nbasis, k, mu, rl, 2, npts, pts + n1);
  ff_sum_kernel<double><<<dim3((unsigned)ndir, nrhs), 256, 0, st>>>(pts, npts, d_dirs, ndir, k, d_out);
  note_launch(3);
  dfree(pts, st);
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

int launch_farfield_mixed(const Space& rwg, const Space& bc, const double2* d_x, int nrhs, const double* d_dirs,
                          int64_t ndir, double k, double mu, double2* d_out, cudaStream_t st) {
  return farfield_mixed_t(rwg, bc, d_x, nrhs, d_dirs, ndir, k, mu, d_out, st);
}

int launch_farfield(const Space& rwg, const double2* d_x, int nrhs, const double* d_dirs, int64_t ndir,
                    double k, double mu, double2* d_out, int precision, cudaStream_t st) {
  return precision == CAL_FP64 ? farfield_t<double>(rwg, d_x, nrhs, d_dirs, ndir, k, mu, d_out, st)
                               : farfield_t<float>(rwg, d_x, nrhs, d_dirs, ndir, k, mu, d_out, st);
}

Rules6 rules6() {
  std::vector<double> b, w;
  triangle_rule(6, b, w);
  Rules6 r;
  for (int i = 0; i < 18; ++i) r.b[i] = b[i];
  for (int i = 0; i < 6; ++i) r.w[i] = w[i];
  return r;
}

}  // namespace cal
