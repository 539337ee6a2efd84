// H-matrix form of an operator block with ACA (Section 3.3).
//
// The paper's software assembles the preconditioner as an H-matrix: cluster
// trees of the dofs by repeated geometric subdivision; a block of two clusters
// is admissible when the bounding boxes of their supports are disjoint (eq.
// admissibility with dist > 0), otherwise it is split until its parts are
// admissible or below a minimum size, and then stored dense (inadmissible).
// Admissible blocks are approximated by adaptive cross approximation to the
// tolerance nu, and only those within chi of each other are kept (eq.
// nf_condition, the bi-parametric cutoff); the rest are dropped.
//
// Here the clusters and leaves are built on the host from the supports'
// bounding boxes (median split of the box centres along the longest side of
// the cluster's box, minimum size 16, stable order); the entries come from the
// dense block on the device. One CTA per admissible leaf runs partially
// pivoted ACA (the next row pivot is the largest entry of the newest column
// among unused rows; the stopping test |u_r| |v_r| <= nu |sum_k u_k v_k^T|_F
// uses the running Frobenius norm), in the block's precision, and the ranks
// and factors are then packed. The product applies the dense leaves and the
// factors (V^T x, then U times that) with atomics into y.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

#include "internal.h"
#include "solve.h"

namespace cal {
namespace {

constexpr int HM_NMIN = 16;       // minimum cluster size
constexpr int ACA_THREADS = 256;

inline unsigned nblocks(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// ---- host: cluster tree and block tree ---------------------------------------
struct Cluster {
  std::vector<int> idx;
  double lo[3], hi[3];
  int child[2] = {-1, -1};
};

int build_cluster(std::vector<Cluster>& T, const double* blo, const double* bhi, std::vector<int> idx) {
  Cluster c;
  for (int a = 0; a < 3; ++a) {
    c.lo[a] = 1e300;
    c.hi[a] = -1e300;
  }
  for (int i : idx)
    for (int a = 0; a < 3; ++a) {
      c.lo[a] = std::min(c.lo[a], blo[3 * i + a]);
      c.hi[a] = std::max(c.hi[a], bhi[3 * i + a]);
    }
  const int me = (int)T.size();
  c.idx = idx;
  T.push_back(c);
  if ((int)idx.size() <= HM_NMIN) return me;
  int ax = 0;
  for (int a = 1; a < 3; ++a)
    if (T[me].hi[a] - T[me].lo[a] > T[me].hi[ax] - T[me].lo[ax]) ax = a;
  std::stable_sort(idx.begin(), idx.end(), [&](int p, int q) {
    return 0.5 * (blo[3 * p + ax] + bhi[3 * p + ax]) < 0.5 * (blo[3 * q + ax] + bhi[3 * q + ax]);
  });
  const size_t h = idx.size() / 2;
  const int c0 = build_cluster(T, blo, bhi, std::vector<int>(idx.begin(), idx.begin() + h));
  const int c1 = build_cluster(T, blo, bhi, std::vector<int>(idx.begin() + h, idx.end()));
  T[me].child[0] = c0;
  T[me].child[1] = c1;
  return me;
}

double box_distance(const Cluster& a, const Cluster& b) {
  double s = 0.0;
  for (int q = 0; q < 3; ++q) {
    const double g = std::max(0.0, std::max(b.lo[q] - a.hi[q], a.lo[q] - b.hi[q]));
    s += g * g;
  }
  return std::sqrt(s);
}

struct LeafH {
  int a, b;
  bool adm;
  double dist;
};

void block_tree(const std::vector<Cluster>& T, int a, int b, std::vector<LeafH>& out) {
  const double d = box_distance(T[a], T[b]);
  if (d > 0.0) {
    out.push_back({a, b, true, d});
  } else if ((int)T[a].idx.size() <= HM_NMIN || (int)T[b].idx.size() <= HM_NMIN || T[a].child[0] < 0 ||
             T[b].child[0] < 0) {
    out.push_back({a, b, false, d});
  } else {
    for (int ca : T[a].child)
      for (int cb : T[b].child) block_tree(T, ca, cb, out);
  }
}

// ---- device helpers ------------------------------------------------------------
template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

template <typename R>
struct ArgMax {
  R v;
  int i;
};

// block-wide (value, index) maximum, the smaller index on ties; all threads get it
template <typename R>
__device__ ArgMax<R> block_argmax(R v, int i, ArgMax<R>* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    const R v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = {v, i};
  __syncthreads();
  if (w == 0) {
    ArgMax<R> x = lane < (int)(blockDim.x >> 5) ? sh[lane] : ArgMax<R>{R(-2), 0x7fffffff};
    for (int o = 16; o > 0; o >>= 1) {
      const R v2 = __shfl_xor_sync(0xffffffffu, x.v, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, x.i, o);
      if (v2 > x.v || (v2 == x.v && i2 < x.i)) { x.v = v2; x.i = i2; }
    }
    if (lane == 0) sh[32] = x;
  }
  __syncthreads();
  return sh[32];
}

// block-wide sum of K values per thread; all threads get the sums
template <typename R, int K>
__device__ void block_sum(R* v, R* sh) {
  for (int k = 0; k < K; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0)
    for (int k = 0; k < K; ++k) sh[w * K + k] = v[k];
  __syncthreads();
  for (int k = 0; k < K; ++k) {
    R s = 0;
    for (int q = 0; q < nw; ++q) s += sh[q * K + k];
    v[k] = s;
  }
  __syncthreads();
}

// Partially pivoted ACA of the leaf B = A[rows, cols] (A dense, leading dimension
// ld, local indices), one CTA per leaf. U [maxr][nr] and V [maxr][nc] are the
// leaf's scratch; rowbuf [nc], used [nr] as well. Writes the rank.
template <typename R>
__global__ void __launch_bounds__(ACA_THREADS) aca_kernel(const typename C2<R>::T* __restrict__ A, int64_t ld,
                                                          const int* __restrict__ idx, const HLeafD* __restrict__ tab,
                                                          int nleaf, R nu, int maxr_cap,
                                                          typename C2<R>::T* __restrict__ Upool,
                                                          typename C2<R>::T* __restrict__ Vpool,
                                                          unsigned char* __restrict__ usedpool,
                                                          const int64_t* __restrict__ usedoff, int* __restrict__ ranks) {
  using T = typename C2<R>::T;
  __shared__ ArgMax<R> sh_am[33];
  __shared__ R sh_sum[8 * 4];
  __shared__ int sh_i;
  for (int f = blockIdx.x; f < nleaf; f += gridDim.x) {
    const HLeafD L = tab[f];
    const int* rows = idx + L.r0;
    const int* cols = idx + L.c0;
    T* U = Upool + L.uoff;  // [k][nr]
    T* V = Vpool + L.voff;  // [k][nc]
    unsigned char* used = usedpool + usedoff[f];
    const int nr = L.nr, nc = L.nc;
    const int maxr = min(min(nr, nc), maxr_cap);
    for (int a = threadIdx.x; a < nr; a += blockDim.x) used[a] = 0;
    int i = 0, rank = 0;
    R norm2 = 0;
    __syncthreads();
    while (rank < maxr) {
      if (threadIdx.x == 0) used[i] = 1;
      // residual row i, kept in V[rank] for now; its largest entry (first on ties)
      R best = R(-1);
      int bj = 0x7fffffff;
      const int64_t ri = rows[i];
      for (int j = threadIdx.x; j < nc; j += blockDim.x) {
        T r = A[ri * ld + cols[j]];
        for (int k = 0; k < rank; ++k) {
          const T u = U[(int64_t)k * nr + i], v = V[(int64_t)k * nc + j];
          r.x -= u.x * v.x - u.y * v.y;
          r.y -= u.x * v.y + u.y * v.x;
        }
        V[(int64_t)rank * nc + j] = r;
        const R m = sqrt(r.x * r.x + r.y * r.y);
        if (m > best) { best = m; bj = j; }
      }
      const ArgMax<R> am = block_argmax<R>(best, bj, sh_am);
      if (!(am.v > R(0)) || am.i >= nc) {
        // a zero residual row: take the first unused row
        if (threadIdx.x == 0) {
          int nxt = -1;
          for (int a = 0; a < nr; ++a)
            if (!used[a]) { nxt = a; break; }
          sh_i = nxt;
        }
        __syncthreads();
        if (sh_i < 0) break;
        i = sh_i;
        __syncthreads();
        continue;
      }
      const int j = am.i;
      const T piv = V[(int64_t)rank * nc + j];
      __syncthreads();
      const R pd = piv.x * piv.x + piv.y * piv.y;
      // v = r / r_j
      for (int q = threadIdx.x; q < nc; q += blockDim.x) {
        const T r = V[(int64_t)rank * nc + q];
        V[(int64_t)rank * nc + q] = {(r.x * piv.x + r.y * piv.y) / pd, (r.y * piv.x - r.x * piv.y) / pd};
      }
      // residual column j: u = A[:, j] - sum_k V_k[j] U_k
      const int64_t cj = cols[j];
      for (int a = threadIdx.x; a < nr; a += blockDim.x) {
        T u = A[(int64_t)rows[a] * ld + cj];
        for (int k = 0; k < rank; ++k) {
          const T uu = U[(int64_t)k * nr + a], vv = V[(int64_t)k * nc + j];
          u.x -= vv.x * uu.x - vv.y * uu.y;
          u.y -= vv.x * uu.y + vv.y * uu.x;
        }
        U[(int64_t)rank * nr + a] = u;
      }
      __syncthreads();
      // |u|^2 |v|^2 and the cross terms 2 Re((U_k^H u)(V_k^H v)) of the running norm
      R s[4] = {0, 0, 0, 0};
      for (int a = threadIdx.x; a < nr; a += blockDim.x) {
        const T u = U[(int64_t)rank * nr + a];
        s[0] += u.x * u.x + u.y * u.y;
      }
      for (int q = threadIdx.x; q < nc; q += blockDim.x) {
        const T v = V[(int64_t)rank * nc + q];
        s[1] += v.x * v.x + v.y * v.y;
      }
      block_sum<R, 2>(s, sh_sum);
      const R nu2 = s[0] * s[1];
      R cross = 0;
      for (int k = 0; k < rank; ++k) {
        R d[4] = {0, 0, 0, 0};  // U_k^H u (re, im), V_k^H v (re, im)
        for (int a = threadIdx.x; a < nr; a += blockDim.x) {
          const T p = U[(int64_t)k * nr + a], u = U[(int64_t)rank * nr + a];
          d[0] += p.x * u.x + p.y * u.y;
          d[1] += p.x * u.y - p.y * u.x;
        }
        for (int q = threadIdx.x; q < nc; q += blockDim.x) {
          const T p = V[(int64_t)k * nc + q], v = V[(int64_t)rank * nc + q];
          d[2] += p.x * v.x + p.y * v.y;
          d[3] += p.x * v.y - p.y * v.x;
        }
        block_sum<R, 4>(d, sh_sum);
        cross += 2 * (d[0] * d[2] - d[1] * d[3]);
      }
      norm2 += nu2 + cross;
      ++rank;
      if (sqrt(nu2) <= nu * sqrt(max(norm2, R(0)))) break;
      // next row: the largest |u| among unused rows
      R cb = R(-1);
      int ci = 0x7fffffff;
      for (int a = threadIdx.x; a < nr; a += blockDim.x) {
        const T u = U[(int64_t)(rank - 1) * nr + a];
        const R m = used[a] ? R(-1) : sqrt(u.x * u.x + u.y * u.y);
        if (m > cb) { cb = m; ci = a; }
      }
      const ArgMax<R> nx = block_argmax<R>(cb, ci, sh_am);
      if (nx.v < R(0)) break;
      i = nx.i;
    }
    if (threadIdx.x == 0) ranks[f] = rank;
    __syncthreads();
  }
}

// dense leaves: values gathered from the dense block
template <typename T>
__global__ void gather_near_kernel(const T* __restrict__ A, int64_t ld, const int* __restrict__ idx,
                                   const HNearD* __restrict__ tab, int nleaf, T* __restrict__ out) {
  for (int f = blockIdx.x; f < nleaf; f += gridDim.x) {
    const HNearD L = tab[f];
    for (int q = threadIdx.x; q < L.nr * L.nc; q += blockDim.x) {
      const int a = q / L.nc, b = q - a * L.nc;
      out[L.off + q] = A[(int64_t)idx[L.r0 + a] * ld + idx[L.c0 + b]];
    }
  }
}

// pack the factors of rank r from the scratch (capacity min(nr, nc, cap)) to offsets
template <typename T>
__global__ void pack_factors_kernel(const T* __restrict__ Us, const T* __restrict__ Vs, const HLeafD* __restrict__ st,
                                    const HLeafD* __restrict__ dt, int nleaf, T* __restrict__ U, T* __restrict__ V) {
  for (int f = blockIdx.x; f < nleaf; f += gridDim.x) {
    const HLeafD s = st[f], d = dt[f];
    for (int q = threadIdx.x; q < d.rank * d.nr; q += blockDim.x) U[d.uoff + q] = Us[s.uoff + q];
    for (int q = threadIdx.x; q < d.rank * d.nc; q += blockDim.x) V[d.voff + q] = Vs[s.voff + q];
  }
}

// reconstruct the dense block [n][n] (zeroed by the caller) from the leaves
template <typename T>
__global__ void expand_kernel(const int* __restrict__ idx, const HNearD* __restrict__ nt, int nnear,
                              const T* __restrict__ nearv, const HLeafD* __restrict__ ft, int nfar,
                              const T* __restrict__ U, const T* __restrict__ V, int64_t n, T* __restrict__ out) {
  const int f = blockIdx.x;
  if (f < nnear) {
    const HNearD L = nt[f];
    for (int q = threadIdx.x; q < L.nr * L.nc; q += blockDim.x) {
      const int a = q / L.nc, b = q - a * L.nc;
      out[(int64_t)idx[L.r0 + a] * n + idx[L.c0 + b]] = nearv[L.off + q];
    }
  } else if (f - nnear < nfar) {
    const HLeafD L = ft[f - nnear];
    for (int q = threadIdx.x; q < L.nr * L.nc; q += blockDim.x) {
      const int a = q / L.nc, b = q - a * L.nc;
      T s = {0, 0};
      for (int k = 0; k < L.rank; ++k) {
        const T u = U[L.uoff + (int64_t)k * L.nr + a], v = V[L.voff + (int64_t)k * L.nc + b];
        s.x += u.x * v.x - u.y * v.y;
        s.y += u.x * v.y + u.y * v.x;
      }
      out[(int64_t)idx[L.r0 + a] * n + idx[L.c0 + b]] = s;
    }
  }
}

// ---- product -------------------------------------------------------------------
__device__ __forceinline__ void addc(float2* p, double re, double im) {
  atomicAdd(&p->x, (float)re);
  atomicAdd(&p->y, (float)im);
}
__device__ __forceinline__ void addc(double2* p, double re, double im) {
  atomicAdd(&p->x, re);
  atomicAdd(&p->y, im);
}

// dense leaves, warp per (leaf, row): y1 += C x1 + alpha S x2, y2 += C x2 + beta S x1
// (S or C may be absent); x, y the block's rows/cols halves (offset applied);
// roff: prefix sums of the leaves' row counts
__device__ __forceinline__ int find_leaf(const int64_t* __restrict__ off, int n, int64_t g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename MT, typename VT>
__global__ void hmat_near_kernel(const int* __restrict__ idx, const HNearD* __restrict__ tab, int nleaf,
                                 const int64_t* __restrict__ roff, const MT* __restrict__ S, const MT* __restrict__ C,
                                 const VT* __restrict__ x1, const VT* __restrict__ x2, VT* __restrict__ y1,
                                 VT* __restrict__ y2, double ar, double ai, double br, double bi) {
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (nleaf == 0 || w >= roff[nleaf]) return;
  const int f = find_leaf(roff, nleaf, w);
  const HNearD L = tab[f];
  const int a = (int)(w - roff[f]);
  double c1r = 0, c1i = 0, c2r = 0, c2i = 0, s1r = 0, s1i = 0, s2r = 0, s2i = 0;
  for (int b = lane; b < L.nc; b += 32) {
    const int col = idx[L.c0 + b];
    const VT u = x1[col], v = x2[col];
    const int64_t q = L.off + (int64_t)a * L.nc + b;
    if (C) {
      const MT m = C[q];
      c1r += (double)m.x * u.x - (double)m.y * u.y; c1i += (double)m.x * u.y + (double)m.y * u.x;
      c2r += (double)m.x * v.x - (double)m.y * v.y; c2i += (double)m.x * v.y + (double)m.y * v.x;
    }
    if (S) {
      const MT m = S[q];
      s1r += (double)m.x * u.x - (double)m.y * u.y; s1i += (double)m.x * u.y + (double)m.y * u.x;
      s2r += (double)m.x * v.x - (double)m.y * v.y; s2i += (double)m.x * v.y + (double)m.y * v.x;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    c1r += __shfl_xor_sync(0xffffffffu, c1r, o); c1i += __shfl_xor_sync(0xffffffffu, c1i, o);
    c2r += __shfl_xor_sync(0xffffffffu, c2r, o); c2i += __shfl_xor_sync(0xffffffffu, c2i, o);
    s1r += __shfl_xor_sync(0xffffffffu, s1r, o); s1i += __shfl_xor_sync(0xffffffffu, s1i, o);
    s2r += __shfl_xor_sync(0xffffffffu, s2r, o); s2i += __shfl_xor_sync(0xffffffffu, s2i, o);
  }
  if (lane == 0) {
    const int row = idx[L.r0 + a];
    addc(y1 + row, c1r + ar * s2r - ai * s2i, c1i + ar * s2i + ai * s2r);
    addc(y2 + row, c2r + br * s1r - bi * s1i, c2i + br * s1i + bi * s1r);
  }
}

// low-rank leaves, phase 1: t[f][k] = (V_S,k^T x1, V_S,k^T x2, V_C,k^T x1, V_C,k^T x2),
// warp per (leaf, k) of each operator
template <typename MT, typename VT>
__global__ void hmat_vt_kernel(const int* __restrict__ idx, const HLeafD* __restrict__ tab, int nleaf,
                               const int64_t* __restrict__ koff, const MT* __restrict__ V, const VT* __restrict__ x1,
                               const VT* __restrict__ x2, double2* __restrict__ t) {
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  // binary search of the leaf whose k range holds w
  int lo = 0, hi = nleaf - 1;
  if (nleaf == 0 || w >= koff[nleaf]) return;
  lo = find_leaf(koff, nleaf, w);
  (void)hi;
  const HLeafD L = tab[lo];
  const int k = (int)(w - koff[lo]);
  double ar = 0, ai = 0, br = 0, bi = 0;
  for (int b = lane; b < L.nc; b += 32) {
    const MT v = V[L.voff + (int64_t)k * L.nc + b];
    const int col = idx[L.c0 + b];
    const VT u = x1[col], z = x2[col];
    ar += (double)v.x * u.x - (double)v.y * u.y; ai += (double)v.x * u.y + (double)v.y * u.x;
    br += (double)v.x * z.x - (double)v.y * z.y; bi += (double)v.x * z.y + (double)v.y * z.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, o); ai += __shfl_xor_sync(0xffffffffu, ai, o);
    br += __shfl_xor_sync(0xffffffffu, br, o); bi += __shfl_xor_sync(0xffffffffu, bi, o);
  }
  if (lane == 0) {
    t[2 * w] = make_double2(ar, ai);
    t[2 * w + 1] = make_double2(br, bi);
  }
}

// low-rank leaves, phase 2: thread per (leaf, row): y1 += U_C tC1 + alpha U_S tS2,
// y2 += U_C tC2 + beta U_S tS1 (tX1 = V_X^T x1, tX2 = V_X^T x2)
template <typename MT, typename VT>
__global__ void hmat_u_kernel(const int* __restrict__ idx, const HLeafD* __restrict__ tabS,
                              const HLeafD* __restrict__ tabC, int nleaf, const int64_t* __restrict__ roff,
                              const int64_t* __restrict__ koffS, const int64_t* __restrict__ koffC,
                              const MT* __restrict__ US, const MT* __restrict__ UC, const double2* __restrict__ tS,
                              const double2* __restrict__ tC, VT* __restrict__ y1, VT* __restrict__ y2, double ar,
                              double ai, double br, double bi) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (nleaf == 0 || g >= roff[nleaf]) return;
  const int lo = find_leaf(roff, nleaf, g);
  const int a = (int)(g - roff[lo]);
  double o1r = 0, o1i = 0, o2r = 0, o2i = 0;
  if (tabC) {
    const HLeafD L = tabC[lo];
    for (int k = 0; k < L.rank; ++k) {
      const MT u = UC[L.uoff + (int64_t)k * L.nr + a];
      const double2 t1 = tC[2 * (koffC[lo] + k)], t2 = tC[2 * (koffC[lo] + k) + 1];
      o1r += (double)u.x * t1.x - (double)u.y * t1.y; o1i += (double)u.x * t1.y + (double)u.y * t1.x;
      o2r += (double)u.x * t2.x - (double)u.y * t2.y; o2i += (double)u.x * t2.y + (double)u.y * t2.x;
    }
  }
  if (tabS) {
    const HLeafD L = tabS[lo];
    double s1r = 0, s1i = 0, s2r = 0, s2i = 0;  // U_S tS1, U_S tS2
    for (int k = 0; k < L.rank; ++k) {
      const MT u = US[L.uoff + (int64_t)k * L.nr + a];
      const double2 t1 = tS[2 * (koffS[lo] + k)], t2 = tS[2 * (koffS[lo] + k) + 1];
      s1r += (double)u.x * t1.x - (double)u.y * t1.y; s1i += (double)u.x * t1.y + (double)u.y * t1.x;
      s2r += (double)u.x * t2.x - (double)u.y * t2.y; s2i += (double)u.x * t2.y + (double)u.y * t2.x;
    }
    o1r += ar * s2r - ai * s2i; o1i += ar * s2i + ai * s2r;
    o2r += br * s1r - bi * s1i; o2i += br * s1i + bi * s1r;
  }
  const HLeafD L = tabS ? tabS[lo] : tabC[lo];
  const int row = idx[L.r0 + a];
  addc(y1 + row, o1r, o1i);
  addc(y2 + row, o2r, o2i);
}

template <typename R>
int compress_t(const Op& dense, const Space& sp, double nu, double chi, int max_rank, Op& out, cudaStream_t st) {
  using T = typename C2<R>::T;
  const int64_t n = dense.rows, off = dense.row_offset;
  auto* h = new HMat();
  out.hmat = h;
  h->n = n;
  h->precision = dense.precision;
  // clusters over the block's dofs (local indices) and the leaves of the block tree
  std::vector<Cluster> tree;
  std::vector<int> all(n);
  std::iota(all.begin(), all.end(), 0);
  std::vector<double> blo(3 * n), bhi(3 * n);
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      blo[3 * i + a] = sp.box_lo[3 * (off + i) + a];
      bhi[3 * i + a] = sp.box_hi[3 * (off + i) + a];
    }
  const int root = build_cluster(tree, blo.data(), bhi.data(), all);
  std::vector<LeafH> leaves;
  block_tree(tree, root, root, leaves);
  for (const LeafH& l : leaves) {
    if (l.adm && !(l.dist <= chi)) continue;  // beyond the cutoff: dropped
    HMat::Leaf L;
    L.r0 = (int64_t)h->idx.size();
    h->idx.insert(h->idx.end(), tree[l.a].idx.begin(), tree[l.a].idx.end());
    L.c0 = (int64_t)h->idx.size();
    h->idx.insert(h->idx.end(), tree[l.b].idx.begin(), tree[l.b].idx.end());
    L.nr = (int)tree[l.a].idx.size();
    L.nc = (int)tree[l.b].idx.size();
    L.dist = l.dist;
    (l.adm ? h->far : h->near).push_back(L);
  }
  const int nops = (dense.d_S ? 1 : 0) + (dense.d_C ? 1 : 0);
  CAL_TRY_CUDA(dalloc((void**)&h->d_idx, std::max<size_t>(h->idx.size(), 1) * sizeof(int), st));
  CAL_TRY_CUDA(cudaMemcpyAsync(h->d_idx, h->idx.data(), h->idx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  // dense leaves
  std::vector<HNearD> nt(h->near.size());
  int64_t ne = 0;
  for (size_t f = 0; f < h->near.size(); ++f) {
    const HMat::Leaf& L = h->near[f];
    nt[f] = {L.r0, L.c0, ne, L.nr, L.nc};
    ne += (int64_t)L.nr * L.nc;
  }
  h->near_entries = ne;
  CAL_TRY_CUDA(dalloc((void**)&h->d_near_tab, std::max<size_t>(nt.size(), 1) * sizeof(HNearD), st));
  CAL_TRY_CUDA(cudaMemcpyAsync(h->d_near_tab, nt.data(), nt.size() * sizeof(HNearD), cudaMemcpyHostToDevice, st));
  // low-rank leaves: scratch of capacity min(nr, nc, max_rank) per leaf
  const int nf = (int)h->far.size();
  std::vector<HLeafD> ft(nf);
  std::vector<int64_t> uoff_used(nf + 1, 0);
  int64_t ucap = 0, vcap = 0;
  for (int f = 0; f < nf; ++f) {
    const HMat::Leaf& L = h->far[f];
    const int cap = std::min(std::min(L.nr, L.nc), max_rank);
    ft[f] = {L.r0, L.c0, ucap, vcap, L.nr, L.nc, 0, 0};
    ucap += (int64_t)cap * L.nr;
    vcap += (int64_t)cap * L.nc;
    uoff_used[f + 1] = uoff_used[f] + L.nr;
  }
  HLeafD* d_ft = nullptr;
  T *Us = nullptr, *Vs = nullptr;
  unsigned char* used = nullptr;
  int64_t* d_usedoff = nullptr;
  int* d_ranks = nullptr;
  struct Tmp {
    std::vector<void*> p;
    cudaStream_t s;
    ~Tmp() { for (void* q : p) dfree(q, s); }
  } tmp{{}, st};
  if (nf > 0) {
    CAL_TRY_CUDA(dalloc((void**)&d_ft, nf * sizeof(HLeafD), st));
    tmp.p.push_back(d_ft);
    CAL_TRY_CUDA(dalloc((void**)&Us, std::max<int64_t>(ucap, 1) * sizeof(T), st));
    tmp.p.push_back(Us);
    CAL_TRY_CUDA(dalloc((void**)&Vs, std::max<int64_t>(vcap, 1) * sizeof(T), st));
    tmp.p.push_back(Vs);
    CAL_TRY_CUDA(dalloc((void**)&used, std::max<int64_t>(uoff_used[nf], 1), st));
    tmp.p.push_back(used);
    CAL_TRY_CUDA(dalloc((void**)&d_usedoff, (nf + 1) * sizeof(int64_t), st));
    tmp.p.push_back(d_usedoff);
    CAL_TRY_CUDA(dalloc((void**)&d_ranks, nf * sizeof(int), st));
    tmp.p.push_back(d_ranks);
    CAL_TRY_CUDA(cudaMemcpyAsync(d_ft, ft.data(), nf * sizeof(HLeafD), cudaMemcpyHostToDevice, st));
    CAL_TRY_CUDA(cudaMemcpyAsync(d_usedoff, uoff_used.data(), (nf + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  }
  h->stored = 0;
  for (int q = 0, op = 0; q < 2; ++q) {
    const void* src = q == 0 ? dense.d_S : dense.d_C;
    if (!src) continue;
    const T* A = (const T*)src;
    // dense leaves
    CAL_TRY_CUDA(dalloc(&h->d_near[q], std::max<int64_t>(ne, 1) * sizeof(T), st));
    if (!nt.empty()) {
      gather_near_kernel<T><<<nblocks((int64_t)nt.size(), 1), 256, 0, st>>>(A, n, h->d_idx, h->d_near_tab,
                                                                             (int)nt.size(), (T*)h->d_near[q]);
      note_launch();
    }
    h->stored += ne;
    // ACA per admissible leaf
    std::vector<HLeafD> packed(nf);
    int64_t uo = 0, vo = 0;
    h->rank[q].assign(nf, 0);
    if (nf > 0) {
      const int tok = prof_begin(st, "aca", 0.0);
      aca_kernel<R><<<(unsigned)std::min(nf, 65535), ACA_THREADS, 0, st>>>(
          A, n, h->d_idx, d_ft, nf, (R)nu, max_rank, Us, Vs, used, d_usedoff, d_ranks);
      prof_end(st, tok);
      note_launch();
      CAL_TRY_CUDA(cudaGetLastError());
      CAL_TRY_CUDA(cudaMemcpyAsync(h->rank[q].data(), d_ranks, nf * sizeof(int), cudaMemcpyDeviceToHost, st));
      CAL_TRY_CUDA(cudaStreamSynchronize(st));
      for (int f = 0; f < nf; ++f) {
        packed[f] = ft[f];
        packed[f].uoff = uo;
        packed[f].voff = vo;
        packed[f].rank = h->rank[q][f];
        uo += (int64_t)packed[f].rank * ft[f].nr;
        vo += (int64_t)packed[f].rank * ft[f].nc;
        h->max_rank_seen = std::max(h->max_rank_seen, packed[f].rank);
      }
      std::vector<HLeafD> srcs = ft;
      for (int f = 0; f < nf; ++f) srcs[f].rank = packed[f].rank;
      CAL_TRY_CUDA(dalloc(&h->d_U[q], std::max<int64_t>(uo, 1) * sizeof(T), st));
      CAL_TRY_CUDA(dalloc(&h->d_V[q], std::max<int64_t>(vo, 1) * sizeof(T), st));
      CAL_TRY_CUDA(dalloc((void**)&h->d_far_tab[q], nf * sizeof(HLeafD), st));
      HLeafD* d_src = nullptr;
      CAL_TRY_CUDA(dalloc((void**)&d_src, nf * sizeof(HLeafD), st));
      tmp.p.push_back(d_src);
      CAL_TRY_CUDA(cudaMemcpyAsync(d_src, srcs.data(), nf * sizeof(HLeafD), cudaMemcpyHostToDevice, st));
      CAL_TRY_CUDA(cudaMemcpyAsync(h->d_far_tab[q], packed.data(), nf * sizeof(HLeafD), cudaMemcpyHostToDevice, st));
      pack_factors_kernel<T><<<(unsigned)std::min(nf, 65535), 256, 0, st>>>(Us, Vs, d_src, h->d_far_tab[q], nf,
                                                                            (T*)h->d_U[q], (T*)h->d_V[q]);
      note_launch();
      CAL_TRY_CUDA(cudaGetLastError());
    }
    h->stored += uo + vo;
    // rank prefix sums of this operator
    std::vector<int64_t> ko(nf + 1, 0);
    for (int f = 0; f < nf; ++f) ko[f + 1] = ko[f] + h->rank[q][f];
    h->ktot[q] = ko[nf];
    CAL_TRY_CUDA(dalloc((void**)&h->d_koff[q], (nf + 1) * sizeof(int64_t), st));
    CAL_TRY_CUDA(cudaMemcpyAsync(h->d_koff[q], ko.data(), (nf + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CAL_TRY_CUDA(cudaStreamSynchronize(st));  // ko is read by the copy
    ++op;
  }
  // row prefix sums of the dense and the low-rank leaves
  std::vector<int64_t> rn(h->near.size() + 1, 0), rf(nf + 1, 0);
  for (size_t f = 0; f < h->near.size(); ++f) rn[f + 1] = rn[f] + h->near[f].nr;
  for (int f = 0; f < nf; ++f) rf[f + 1] = rf[f] + h->far[f].nr;
  h->near_rows = rn.back();
  h->far_rows = rf.back();
  CAL_TRY_CUDA(dalloc((void**)&h->d_roff_near, rn.size() * sizeof(int64_t), st));
  CAL_TRY_CUDA(dalloc((void**)&h->d_roff_far, rf.size() * sizeof(int64_t), st));
  CAL_TRY_CUDA(cudaMemcpyAsync(h->d_roff_near, rn.data(), rn.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  CAL_TRY_CUDA(cudaMemcpyAsync(h->d_roff_far, rf.data(), rf.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  CAL_TRY_CUDA(cudaStreamSynchronize(st));  // host tables are read by the copies; the scratch goes
  (void)nops;
  return CAL_OK;
}

template <typename MT, typename VT>
int hmat_apply_t(const HMat& h, bool withS, bool withC, const VT* x1, const VT* x2, VT* y1, VT* y2, double ar,
                 double ai, double br, double bi, cudaStream_t st) {
  withS = withS && h.d_near[0];
  withC = withC && h.d_near[1];
  const MT* S = withS ? (const MT*)h.d_near[0] : nullptr;
  const MT* C = withC ? (const MT*)h.d_near[1] : nullptr;
  const int nn = (int)h.near.size(), nf = (int)h.far.size();
  const int tok = prof_begin(st, "hmat", 0.0);
  if (nn > 0 && (S || C)) {
    hmat_near_kernel<MT, VT><<<nblocks(h.near_rows * 32, 256), 256, 0, st>>>(h.d_idx, h.d_near_tab, nn, h.d_roff_near,
                                                                             S, C, x1, x2, y1, y2, ar, ai, br, bi);
    note_launch();
  }
  const int64_t kS = withS ? h.ktot[0] : 0, kC = withC ? h.ktot[1] : 0;
  if (nf > 0 && kS + kC > 0) {
    double2* t = nullptr;
    if (dalloc((void**)&t, 2 * (size_t)(kS + kC) * sizeof(double2), st) != cudaSuccess) {
      prof_end(st, tok);
      return fail(CAL_ENOMEM, "H-matrix product: cannot allocate the rank sums");
    }
    double2* tS = t;
    double2* tC = t + 2 * kS;
    if (kS > 0) {
      hmat_vt_kernel<MT, VT><<<nblocks(kS * 32, 256), 256, 0, st>>>(h.d_idx, h.d_far_tab[0], nf, h.d_koff[0],
                                                                    (const MT*)h.d_V[0], x1, x2, tS);
      note_launch();
    }
    if (kC > 0) {
      hmat_vt_kernel<MT, VT><<<nblocks(kC * 32, 256), 256, 0, st>>>(h.d_idx, h.d_far_tab[1], nf, h.d_koff[1],
                                                                    (const MT*)h.d_V[1], x1, x2, tC);
      note_launch();
    }
    hmat_u_kernel<MT, VT><<<nblocks(h.far_rows, 256), 256, 0, st>>>(
        h.d_idx, kS > 0 ? h.d_far_tab[0] : nullptr, kC > 0 ? h.d_far_tab[1] : nullptr, nf, h.d_roff_far, h.d_koff[0],
        h.d_koff[1], (const MT*)h.d_U[0], (const MT*)h.d_U[1], tS, tC, y1, y2, ar, ai, br, bi);
    note_launch();
    dfree(t, st);
  }
  prof_end(st, tok);
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

}  // namespace

int hmat_compress(const Op& dense, const Space& sp, double nu, double chi, int max_rank, Op& out,
                  cudaStream_t st) {
  if (dense.format != CAL_DENSE || dense.rows != dense.cols)
    return fail(CAL_EINVAL, "H-matrix: needs a dense square block");
  if (!(nu > 0) || !(chi >= 0)) return fail(CAL_EINVAL, "H-matrix: nu must be > 0 and chi >= 0");
  out.ctx = dense.ctx;
  out.op_mask = dense.op_mask;
  out.precision = dense.precision;
  out.format = CAL_HMAT;
  out.rows = dense.rows;
  out.cols = dense.cols;
  out.row_offset = dense.row_offset;
  int rc = dense.precision == CAL_FP64 ? compress_t<double>(dense, sp, nu, chi, max_rank, out, st)
                                       : compress_t<float>(dense, sp, nu, chi, max_rank, out, st);
  if (!rc) out.nnz = out.hmat->stored;  // stored complex entries of all its operators
  return rc;
}

// y1 += C x1 + alpha S x2, y2 += C x2 + beta S x1 with separate halves (local indices)
int hmat_apply_halves(const HMat& h, bool withS, bool withC, int vec_prec, const void* x1, const void* x2, void* y1,
                      void* y2, double ar, double ai, double br, double bi, cudaStream_t st) {
  if (h.precision == CAL_FP64)
    return hmat_apply_t<double2, double2>(h, withS, withC, (const double2*)x1, (const double2*)x2, (double2*)y1,
                                          (double2*)y2, ar, ai, br, bi, st);
  if (vec_prec == CAL_FP64)
    return hmat_apply_t<float2, double2>(h, withS, withC, (const double2*)x1, (const double2*)x2, (double2*)y1,
                                         (double2*)y2, ar, ai, br, bi, st);
  return hmat_apply_t<float2, float2>(h, withS, withC, (const float2*)x1, (const float2*)x2, (float2*)y1,
                                      (float2*)y2, ar, ai, br, bi, st);
}

// y1 += C x1 + alpha S x2, y2 += C x2 + beta S x1 on the H block (x, y component-major
// of length 2 ntot, the block at row/col offset off)
int hmat_pair_apply(const HMat& h, bool withS, bool withC, int vec_prec, const void* x, void* y, int64_t ntot,
                    int64_t off, double ar, double ai, double br, double bi, cudaStream_t st) {
  if (h.precision == CAL_FP64) {
    const double2* xx = (const double2*)x;
    double2* yy = (double2*)y;
    return hmat_apply_t<double2, double2>(h, withS, withC, xx + off, xx + ntot + off, yy + off, yy + ntot + off, ar,
                                          ai, br, bi, st);
  }
  if (vec_prec == CAL_FP64) {
    const double2* xx = (const double2*)x;
    double2* yy = (double2*)y;
    return hmat_apply_t<float2, double2>(h, withS, withC, xx + off, xx + ntot + off, yy + off, yy + ntot + off, ar, ai,
                                         br, bi, st);
  }
  const float2* xx = (const float2*)x;
  float2* yy = (float2*)y;
  return hmat_apply_t<float2, float2>(h, withS, withC, xx + off, xx + ntot + off, yy + off, yy + ntot + off, ar, ai,
                                      br, bi, st);
}

// operator `which` (0 = S, 1 = C) reconstructed densely into dst [n][n] (device)
int hmat_expand(const HMat& h, int which, void* dst, cudaStream_t st) {
  const size_t es = h.precision == CAL_FP64 ? 16 : 8;
  CAL_TRY_CUDA(cudaMemsetAsync(dst, 0, (size_t)h.n * h.n * es, st));
  const int nn = (int)h.near.size(), nf = (int)h.far.size();
  if (nn + nf == 0) return CAL_OK;
  if (h.precision == CAL_FP64)
    expand_kernel<double2><<<(unsigned)(nn + nf), 256, 0, st>>>(h.d_idx, h.d_near_tab, nn, (const double2*)h.d_near[which],
                                                            h.d_far_tab[which], nf, (const double2*)h.d_U[which],
                                                            (const double2*)h.d_V[which], h.n, (double2*)dst);
  else
    expand_kernel<float2><<<(unsigned)(nn + nf), 256, 0, st>>>(h.d_idx, h.d_near_tab, nn, (const float2*)h.d_near[which],
                                                           h.d_far_tab[which], nf, (const float2*)h.d_U[which],
                                                           (const float2*)h.d_V[which], h.n, (float2*)dst);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

}  // namespace cal
