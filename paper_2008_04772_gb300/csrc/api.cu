// C ABI of the library (include/cal.h) and the PMCHWT solve pipeline.
//
// arXiv 2008.04772: assembly of A on RWG x RWG and of P on BC x BC
// (eq. RWG_discretisation1), identical blocks assembled once (Section 3.2:
// S and C per wavenumber serve both block rows), the strong form
// M_P^-1 P M_A^-1 A solved by restarted GMRES (Section 4), the incident traces
// and the far field of the exterior representation.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <condition_variable>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "solve.h"

namespace cal {
const char* last_error();
int64_t launches();
int prof_enable(int on);
int prof_read(const char* name, int64_t* n, double* ms, double* units);
}

using namespace cal;

namespace {

double now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// vertices of one scatterer (or all) that own a non-empty dual cell
std::vector<int> cell_list(const Space& s, int scat) {
  const Mesh& m = *s.mesh;
  std::vector<char> used(m.nv, 0);
  const int64_t t0 = scat < 0 ? 0 : m.tri_off[scat], t1 = scat < 0 ? m.nt : m.tri_off[scat + 1];
  for (int64_t t = t0; t < t1; ++t)
    for (int a = 0; a < 3; ++a) used[m.T[3 * t + a]] = 1;
  std::vector<int> out;
  for (int64_t v = 0; v < m.nv; ++v)
    if (used[v]) out.push_back((int)v);
  return out;
}

// Bounding ball of a dual cell for the class rules (Section 3.3): C the mean of
// its triangle centroids, rho the largest distance of one of them from C, dm
// the longest edge of its triangles.
struct CellBall {
  double c[3] = {0, 0, 0}, rho = 0, dm = 0;
};

std::vector<CellBall> cell_balls(const Space& sp, const std::vector<int>& cells, int nv) {
  std::vector<CellBall> B(nv);
  for (int v : cells) {
    CellBall& b = B[v];
    const int t0 = sp.cell_tri_ptr[v], t1 = sp.cell_tri_ptr[v + 1];
    for (int q = t0; q < t1; ++q)
      for (int c = 0; c < 3; ++c) b.c[c] += sp.triD[sp.cell_tri[q]].c[c] / (t1 - t0);
    for (int q = t0; q < t1; ++q) {
      const TriD& t = sp.triD[sp.cell_tri[q]];
      double d2 = 0;
      for (int c = 0; c < 3; ++c) d2 += (t.c[c] - b.c[c]) * (t.c[c] - b.c[c]);
      b.rho = std::max(b.rho, std::sqrt(d2));
      b.dm = std::max(b.dm, t.diam);
    }
  }
  return B;
}

// Every triangle pair of cells v and w takes the far rule: the pair's centroid
// distance is at least |C_v - C_w| - rho_v - rho_w, and the far class asks for
// more than 4 max(d1, d2). The relative margin 1e-4 covers the float32
// rounding of the kernels' own per-pair test, so a pair in such a cell pair is
// classed far there too and its arithmetic is the same either way.
constexpr double FAR_MARGIN = 1.0 + 1e-4;
double far_reach(const CellBall& b) { return b.rho + 4.0 * FAR_MARGIN * b.dm; }
bool cells_far(const CellBall& a, const CellBall& b) {
  double d2 = 0;
  for (int c = 0; c < 3; ++c) d2 += (a.c[c] - b.c[c]) * (a.c[c] - b.c[c]);
  const double t = a.rho + b.rho + 4.0 * FAR_MARGIN * std::max(a.dm, b.dm);  // |C_v - C_w| > t
  return d2 > t * t;
}

// cells in Morton order of their centres: the cells of one edge's two ends come
// close together in the unit order, so the rows of the output they accumulate
// into stay in L2 while they are written
void spatial_order(std::vector<int>& cells, const std::vector<CellBall>& B) {
  if (cells.size() < 2) return;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int v : cells)
    for (int c = 0; c < 3; ++c) { lo[c] = std::min(lo[c], B[v].c[c]); hi[c] = std::max(hi[c], B[v].c[c]); }
  double ext = 0;
  for (int c = 0; c < 3; ++c) ext = std::max(ext, hi[c] - lo[c]);
  if (!(ext > 0)) return;
  auto spread = [](uint64_t x) {  // 21 bits -> every third bit
    x &= 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
  };
  std::vector<std::pair<uint64_t, int>> key;
  key.reserve(cells.size());
  for (int v : cells) {
    uint64_t code = 0;
    for (int c = 0; c < 3; ++c) {
      const double f = (B[v].c[c] - lo[c]) / ext;
      code |= spread((uint64_t)std::min(2097151.0, std::max(0.0, f * 2097151.0))) << c;
    }
    key.push_back({code, v});
  }
  std::sort(key.begin(), key.end());
  for (size_t q = 0; q < key.size(); ++q) cells[q] = key[q].second;
}

// per position i of cells, the positions j >= i whose cell pair is not all
// far (sorted), found through a uniform grid of buckets: a pair that is not
// all far is closer than R_v = rho_v + rho_max + 4 margin max(dm_v, dm_max),
// so it lies within ceil(R_v / b) buckets per axis of bucket size b; a bucket
// lists its cells in increasing position and is scanned from position i on
std::vector<std::vector<int>> near_cells(const std::vector<int>& cells, const std::vector<CellBall>& B) {
  const int nc = (int)cells.size();
  std::vector<std::vector<int>> out(nc);
  if (nc == 0) return out;
  double rho_max = 0, dm_max = 0, lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int v : cells) {
    rho_max = std::max(rho_max, B[v].rho);
    dm_max = std::max(dm_max, B[v].dm);
    for (int c = 0; c < 3; ++c) { lo[c] = std::min(lo[c], B[v].c[c]); hi[c] = std::max(hi[c], B[v].c[c]); }
  }
  auto reach = [&](const CellBall& a) { return a.rho + rho_max + 4.0 * FAR_MARGIN * std::max(a.dm, dm_max); };
  const double g = 2.0 * rho_max + 4.0 * FAR_MARGIN * dm_max;  // the largest R_v
  // bucket size g / 2, grown until there are at most 8 buckets per cell
  double b = std::max(0.5 * g, 1e-300);
  int64_t nb[3];
  for (;;) {
    for (int c = 0; c < 3; ++c) nb[c] = (int64_t)((hi[c] - lo[c]) / b) + 1;
    if (nb[0] * nb[1] * nb[2] <= 8 * (int64_t)nc + 64) break;
    b *= 1.5;
  }
  auto coord = [&](int v, int c) { return std::min<int64_t>(nb[c] - 1, (int64_t)((B[v].c[c] - lo[c]) / b)); };
  const int64_t nbt = nb[0] * nb[1] * nb[2];
  std::vector<int> start(nbt + 1, 0), ent(nc);
  std::vector<int64_t> bid(nc);
  for (int j = 0; j < nc; ++j) {
    const int v = cells[j];
    bid[j] = (coord(v, 2) * nb[1] + coord(v, 1)) * nb[0] + coord(v, 0);
    ++start[bid[j] + 1];
  }
  for (int64_t q = 0; q < nbt; ++q) start[q + 1] += start[q];
  {
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (int j = 0; j < nc; ++j) ent[fill[bid[j]]++] = j;  // increasing j within a bucket
  }
  parallel_for(nc, [&](int i) {
    const int v = cells[i];
    const CellBall& bv = B[v];
    const int64_t x0 = coord(v, 0), y0 = coord(v, 1), z0 = coord(v, 2);
    const int r = (int)std::ceil(reach(bv) / b);
    for (int64_t z = std::max<int64_t>(0, z0 - r); z <= std::min(nb[2] - 1, z0 + r); ++z)
      for (int64_t y = std::max<int64_t>(0, y0 - r); y <= std::min(nb[1] - 1, y0 + r); ++y)
        for (int64_t x = std::max<int64_t>(0, x0 - r); x <= std::min(nb[0] - 1, x0 + r); ++x) {
          const int64_t q = (z * nb[1] + y) * nb[0] + x;
          for (const int* e = std::lower_bound(ent.data() + start[q], ent.data() + start[q + 1], i);
               e < ent.data() + start[q + 1]; ++e)
            if (!cells_far(bv, B[cells[*e]])) out[i].push_back(*e);
        }
    std::sort(out[i].begin(), out[i].end());
  });
  return out;
}

// Work units of the BC regular-pair kernels for one scatterer: tiles (v, w),
// v <= w, of dual cells, grouped into units of one test cell and up to 16
// trial cells (or as many as fill the block of the float32 per-thread kernel).
// Dense blocks take every cell pair; near-field blocks the cell pairs that
// hold a kept entry of the CSR pattern np.
int build_units(const Space& sp, int scat, bool dense, int64_t rows, int64_t row_offset,
                const Space::NearPattern* np, int precision, int nreg, Space::UnitLists& L, cudaStream_t st) {
  const Mesh& m = *sp.mesh;
  std::vector<int> cells = cell_list(sp, scat);
  int max_cell = 0;
  for (int v : cells) max_cell = std::max(max_cell, sp.cell_tri_ptr[v + 1] - sp.cell_tri_ptr[v]);
  // tiles (v, w), v <= w, grouped into units of one test cell and up to 16 trial
  // cells (or as many as fill the block of the float32 per-thread kernel)
  const bool owner = bc_owner_width(sp, precision, max_cell, max_cell) > 0;
  auto unit_of = [&](int v) {
    if (!owner) return 16;
    return bc_owner_width(sp, precision, std::max(1, sp.cell_tri_ptr[v + 1] - sp.cell_tri_ptr[v]), max_cell);
  };
  // {v, begin, count, flag} per unit; flag -1: per-pair class test; flag >= 0
  // (class rules, per-thread kernel): every pair of the unit is far, and bit j
  // of flag drops trial cell j (a cell pair left to a flag -1 unit)
  std::vector<int> units;
  std::vector<int> wlist;
  std::vector<int2> tiles;
  const bool split_far = owner && nreg == 0;
  std::vector<CellBall> balls;
  if (split_far) balls = cell_balls(sp, cells, (int)m.nv);
  if (!dense) {
    // tiles (v, w), v <= w, of the cell pairs that hold a kept entry (i, j):
    // v and w end cells of i and j; per test cell a stamp array deduplicates
    const int64_t off = row_offset;
    std::vector<int> cell_rows_ptr(m.nv + 1, 0), cell_rows;
    for (int64_t i = 0; i < rows; ++i) {
      ++cell_rows_ptr[m.e_lo[off + i] + 1];
      ++cell_rows_ptr[m.e_hi[off + i] + 1];
    }
    for (int64_t v = 0; v < m.nv; ++v) cell_rows_ptr[v + 1] += cell_rows_ptr[v];
    cell_rows.resize(cell_rows_ptr[m.nv]);
    {
      std::vector<int> fill(cell_rows_ptr.begin(), cell_rows_ptr.end() - 1);
      for (int64_t i = 0; i < rows; ++i) {
        cell_rows[fill[m.e_lo[off + i]]++] = (int)i;
        cell_rows[fill[m.e_hi[off + i]]++] = (int)i;
      }
    }
    std::vector<int> stamp(m.nv, -1), ws;
    for (int v : cells) {
      ws.clear();
      for (int r = cell_rows_ptr[v]; r < cell_rows_ptr[v + 1]; ++r) {
        const int64_t i = cell_rows[r];
        for (int64_t q = np->rowptr[i]; q < np->rowptr[i + 1]; ++q) {
          const int64_t j = off + np->col[q];
          for (int w : {m.e_lo[j], m.e_hi[j]})
            if (w >= v && stamp[w] != v) {
              stamp[w] = v;
              ws.push_back(w);
            }
        }
      }
      std::sort(ws.begin(), ws.end());
      // with class rules: the cell pairs that are not all far first
      if (split_far)
        std::stable_partition(ws.begin(), ws.end(), [&](int w) { return !cells_far(balls[v], balls[w]); });
      for (int w : ws) tiles.push_back(make_int2(v, w));
    }
    wlist.resize(tiles.size());
    for (size_t q = 0; q < tiles.size(); ++q) wlist[q] = tiles[q].y;
    for (size_t q = 0; q < tiles.size();) {
      size_t e = q;
      const size_t unit = (size_t)unit_of(tiles[q].x);
      const bool far = split_far && cells_far(balls[tiles[q].x], balls[tiles[q].y]);
      while (e < tiles.size() && tiles[e].x == tiles[q].x && e - q < unit &&
             (!split_far || cells_far(balls[tiles[e].x], balls[tiles[e].y]) == far))
        ++e;
      units.insert(units.end(), {tiles[q].x, (int)q, (int)(e - q), far ? 0 : -1});
      q = e;
    }
  } else if (split_far) {
    // all trial ranges are runs of cells; the cell pairs that are not all far
    // also get units of their own, listed after the cells in wlist
    spatial_order(cells, balls);
    wlist = cells;
    const int nc = (int)cells.size();
    const std::vector<std::vector<int>> nearj = near_cells(cells, balls);
    // per test cell: its units (mixed first, then the runs with drop masks),
    // counted, placed by prefix sums and written in parallel
    std::vector<int64_t> uoff(nc + 1, 0), woff(nc + 1, 0);
    auto far_mask = [&](const std::vector<int>& nj, size_t& p, int j0, int cnt) {
      int mask = 0;
      while (p < nj.size() && nj[p] < j0 + cnt) mask |= 1 << (nj[p++] - j0);
      return mask;
    };
    parallel_for(nc, [&](int i) {
      const int unit = std::min(31, unit_of(cells[i]));  // the drop mask has 31 bits
      const std::vector<int>& nj = nearj[i];
      int64_t nu = (int64_t)((nj.size() + unit - 1) / unit);
      size_t p = 0;
      for (int j0 = i; j0 < nc; j0 += unit) {
        const int cnt = std::min(unit, nc - j0);
        if (far_mask(nj, p, j0, cnt) != (int)((1u << cnt) - 1)) ++nu;
      }
      uoff[i + 1] = nu;
      woff[i + 1] = (int64_t)nj.size();
    });
    for (int i = 0; i < nc; ++i) {
      uoff[i + 1] += uoff[i];
      woff[i + 1] += woff[i];
    }
    units.resize((size_t)4 * uoff[nc]);
    wlist.resize((size_t)nc + woff[nc]);
    parallel_for(nc, [&](int i) {
      const int unit = std::min(31, unit_of(cells[i]));
      const std::vector<int>& nj = nearj[i];
      int* u = units.data() + 4 * uoff[i];
      int64_t w = nc + woff[i];
      for (size_t q = 0; q < nj.size(); q += unit) {
        const int cnt = (int)std::min<size_t>(unit, nj.size() - q);
        *u++ = cells[i];
        *u++ = (int)w;
        *u++ = cnt;
        *u++ = -1;
        for (int k = 0; k < cnt; ++k) wlist[w++] = cells[nj[q + k]];
      }
      size_t p = 0;
      for (int j0 = i; j0 < nc; j0 += unit) {
        const int cnt = std::min(unit, nc - j0);
        const int mask = far_mask(nj, p, j0, cnt);
        if (mask != (int)((1u << cnt) - 1)) {
          *u++ = cells[i];
          *u++ = j0;
          *u++ = cnt;
          *u++ = mask;
        }
      }
    });
  } else {
    wlist = cells;
    const int nc = (int)cells.size();
    units.reserve((size_t)4 * nc * (nc / std::max(1, unit_of(cells[0])) + 2));
    for (int i = 0; i < nc; ++i) {
      const int unit = unit_of(cells[i]);
      for (int j0 = i; j0 < nc; j0 += unit) units.insert(units.end(), {cells[i], j0, std::min(unit, nc - j0), -1});
    }
  }
  L.nunits = (int64_t)units.size() / 4;
  L.max_cell = max_cell;
  if (L.nunits > 0) {
    // pageable sources: the copies have read them when they return
    CAL_TRY_CUDA(dalloc((void**)&L.d_units, units.size() * sizeof(int), st));
    CAL_TRY_CUDA(dalloc((void**)&L.d_wlist, std::max<size_t>(wlist.size(), 1) * sizeof(int), st));
    CAL_TRY_CUDA(cudaMemcpyAsync(L.d_units, units.data(), units.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CAL_TRY_CUDA(cudaMemcpyAsync(L.d_wlist, wlist.data(), wlist.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  CAL_TRY_CUDA(cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming));
  CAL_TRY_CUDA(cudaEventRecord(L.done, st));
  // algorithmic work: cell-pair triangle pairs minus touching ones, times rule points squared
  double pairs = 0.0;
  if (dense) {
    double s1 = 0, s2 = 0;
    for (int v : cells) { const double n = sp.cell_tri_ptr[v + 1] - sp.cell_tri_ptr[v]; s1 += n; s2 += n * n; }
    pairs = 0.5 * (s1 * s1 + s2);
  } else {
    for (const int2& t : tiles)
      pairs += (double)(sp.cell_tri_ptr[t.x + 1] - sp.cell_tri_ptr[t.x]) * (sp.cell_tri_ptr[t.y + 1] - sp.cell_tri_ptr[t.y]);
  }
  {
    // dual cell of each small triangle of the listed cells
    std::vector<int> tri_cell(sp.triD.size(), -1);
    for (int v : cells)
      for (int q = sp.cell_tri_ptr[v]; q < sp.cell_tri_ptr[v + 1]; ++q) tri_cell[sp.cell_tri[q]] = v;
    const int d0 = scat < 0 ? 0 : scat, d1 = scat < 0 ? (int)sp.sing.size() : scat + 1;
    for (int d = d0; d < d1; ++d)
      for (const SingPair& q : sp.sing[d]) {
        const double mult = q.cls == 1 ? 2.0 : 1.0;  // vertex pairs are listed once
        pairs -= mult * (tri_cell[q.t1] == tri_cell[q.t2] ? 1.0 : 0.5);
      }
  }
  L.pairs = pairs;
  return CAL_OK;
}

// the near-field pattern of (scatterer, cutoff), built once per space
const Space::NearPattern& cached_near_pattern(const Space& sp, int scat, double chi) {
  std::lock_guard<std::mutex> lk(sp.static_mu);
  for (auto& q : sp.near_patterns)
    if (q->scat == scat && q->chi == chi) return *q;
  auto q = std::make_unique<Space::NearPattern>();
  q->scat = scat;
  q->chi = chi;
  near_pattern(sp, scat, chi, q->rowptr, q->col);
  sp.near_patterns.push_back(std::move(q));
  return *sp.near_patterns.back();
}

// the BC work units of (scatterer, cutoff, rule, kernel), built and uploaded
// once per space; a caller on another stream waits for the upload
int cached_unit_lists(const Space& sp, int scat, double chi, int nreg, int precision, cudaStream_t st,
                      Space::UnitLists** out) {
  const Mesh& m = *sp.mesh;
  const bool dense = std::isinf(chi);
  const Space::NearPattern* np = dense ? nullptr : &cached_near_pattern(sp, scat, chi);
  const bool fp32 = precision == CAL_FP32;
  std::lock_guard<std::mutex> lk(sp.unit_mu);
  for (auto& u : sp.unit_lists)
    if (u->scat == scat && u->chi == chi && u->nreg == nreg && u->owner == fp32) {
      CAL_TRY_CUDA(cudaStreamWaitEvent(st, u->done, 0));
      if (out) *out = u.get();
      return CAL_OK;
    }
  auto u = std::make_unique<Space::UnitLists>();
  u->scat = scat;
  u->chi = chi;
  u->nreg = nreg;
  u->owner = fp32;
  const int64_t off = scat < 0 ? 0 : m.edge_off[scat];
  const int64_t rows = (scat < 0 ? m.ne : m.edge_off[scat + 1]) - off;
  if (int rc = build_units(sp, scat, dense, rows, off, np, precision, nreg, *u, st)) return rc;
  if (out) *out = u.get();
  sp.unit_lists.push_back(std::move(u));
  return CAL_OK;
}

// Kernel arguments of one allocated block.
static AssembleArgs block_args(const Op& op, double kr, double ki, const Space& sp, int scat, int nreg, int nsing,
                               int precision, bool sing32) {
  AssembleArgs a{};
  a.sp = &sp;
  a.scat = scat;
  a.kr = kr;
  a.ki = ki;
  a.want = op.op_mask;
  a.nreg = nreg;
  a.nsing = nsing;
  a.precision = precision;
  a.sing32 = sing32;
  a.format = op.format;
  a.row_off = op.row_offset;
  a.ld = op.cols;
  a.rowptr = op.d_rowptr;
  a.col = op.d_col;
  a.S = op.d_S;
  a.C = op.d_C;
  a.stream = op.ctx->stream;
  return a;
}

// The regular (non-touching) pairs of an allocated block.
static int assemble_regular(Ctx& ctx, const Op& op, double kr, double ki, const Space& sp, int scat, double chi,
                            int nreg, int nsing, int precision, bool sing32) {
  const AssembleArgs a = block_args(op, kr, ki, sp, scat, nreg, nsing, precision, sing32);
  int rc = CAL_OK;
  if (sp.kind == CAL_RWG) {
    rc = launch_rwg_regular(a);
  } else {
    // the work units are the same for every wavenumber: built once per space
    Space::UnitLists* L = nullptr;
    if ((rc = cached_unit_lists(sp, scat, chi, nreg, precision, a.stream, &L))) return rc;
    if (L->nunits > 0)
      rc = launch_bc_regular_units(a, L->d_units, L->nunits, L->d_wlist, L->max_cell, ctx.n_sm,
                                   L->pairs * nreg * nreg);
  }
  if (rc) return rc;
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

// Assemble S and/or C of one block (scat = -1: union; else scatterer scat).
// parts: 1 allocates the zeroed block and enqueues its touching (singular)
// pairs; 2 enqueues the regular pairs of the block that part 1 left in out,
// given the same arguments; 3 does both. Every kernel adds into the zeroed
// block, so the parts may run in either order: a caller can enqueue part 1
// of several blocks while the work units of part 2 are still being built.
int assemble_block(Ctx& ctx, int want, double kr, double ki, const Space& sp, int scat, double chi,
                   int nreg, int nsing, int precision, std::unique_ptr<Op>& out, int parts = 3) {
  const Mesh& m = *sp.mesh;
  if (scat >= m.M) return fail(CAL_EINVAL, "assemble: scatterer %d out of range", scat);
  if (!(want & 3)) return fail(CAL_EINVAL, "assemble: op_mask must contain CAL_OP_S or CAL_OP_C");
  if (precision != CAL_FP32 && precision != CAL_FP64 && precision != CAL_FP32_ALL)
    return fail(CAL_EINVAL, "assemble: bad precision");
  const bool sing32 = precision == CAL_FP32_ALL;
  if (sing32) precision = CAL_FP32;
  if (!std::isfinite(kr) || !std::isfinite(ki) || (kr == 0 && ki == 0))
    return fail(CAL_EINVAL, "assemble: wavenumber must be finite and non-zero");
  int rc = set_quadrature_tables(nreg, nsing);
  if (rc) return rc;
  if (!(parts & 1)) {
    if (!out || out->op_mask != want) return fail(CAL_EINVAL, "assemble: no block from the first part");
    return assemble_regular(ctx, *out, kr, ki, sp, scat, chi, nreg, nsing, precision, sing32);
  }
  auto op = std::make_unique<Op>();
  op->ctx = &ctx;
  op->op_mask = want;
  op->precision = precision;
  op->row_offset = scat < 0 ? 0 : m.edge_off[scat];
  op->rows = op->cols = (scat < 0 ? m.ne : m.edge_off[scat + 1] - m.edge_off[scat]);
  const bool dense = std::isinf(chi);
  op->format = dense ? CAL_DENSE : CAL_CSR;
  if (!dense) {
    if (!(chi >= 0)) return fail(CAL_EINVAL, "assemble: near_cutoff must be >= 0 or INFINITY");
    {
      // the pattern depends on the geometry and the cutoff only: built once per space
      const Space::NearPattern& np = cached_near_pattern(sp, scat, chi);
      op->h_rowptr = np.rowptr;
      op->h_col = np.col;
    }
    op->nnz = op->h_rowptr.back();
  } else {
    op->nnz = op->rows * op->cols;
  }
  const size_t esz = precision == CAL_FP32 ? 8 : 16;
  const size_t bytes = (size_t)op->nnz * esz;
  cudaStream_t st = ctx.stream;
  if (want & 1) {
    if (dalloc(&op->d_S, std::max<size_t>(bytes, 16), st) != cudaSuccess)
      return fail(CAL_ENOMEM, "assemble: cannot allocate %zu bytes for S", bytes);
    CAL_TRY_CUDA(cudaMemsetAsync(op->d_S, 0, bytes, st));
  }
  if (want & 2) {
    if (dalloc(&op->d_C, std::max<size_t>(bytes, 16), st) != cudaSuccess)
      return fail(CAL_ENOMEM, "assemble: cannot allocate %zu bytes for C", bytes);
    CAL_TRY_CUDA(cudaMemsetAsync(op->d_C, 0, bytes, st));
  }
  if (!dense) {
    CAL_TRY_CUDA(dalloc((void**)&op->d_rowptr, op->h_rowptr.size() * sizeof(int64_t), st));
    CAL_TRY_CUDA(dalloc((void**)&op->d_col, std::max<size_t>(op->h_col.size(), 1) * sizeof(int), st));
    CAL_TRY_CUDA(cudaMemcpyAsync(op->d_rowptr, op->h_rowptr.data(), op->h_rowptr.size() * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, st));
    if (!op->h_col.empty())
      CAL_TRY_CUDA(cudaMemcpyAsync(op->d_col, op->h_col.data(), op->h_col.size() * sizeof(int),
                                   cudaMemcpyHostToDevice, st));
  }
  if ((rc = launch_singular(block_args(*op, kr, ki, sp, scat, nreg, nsing, precision, sing32)))) return rc;
  CAL_TRY_CUDA(cudaGetLastError());
  if ((parts & 2) && (rc = assemble_regular(ctx, *op, kr, ki, sp, scat, chi, nreg, nsing, precision, sing32)))
    return rc;
  out = std::move(op);
  return CAL_OK;
}

// Sparse block holding only the touching-pair (Sauter–Schwab) entries of S and C
// on an RWG space: the stored part of a matrix-free operator. Its pattern is
// every (i, j) whose supports share a triangle pair of the singular list.
int assemble_singular_block(Ctx& ctx, double kr, double ki, const Space& sp, int scat, int nsing, int precision,
                            std::unique_ptr<Op>& out) {
  const Mesh& m = *sp.mesh;
  const bool sing32 = precision == CAL_FP32_ALL;
  if (sing32) precision = CAL_FP32;
  int rc = set_quadrature_tables(6, nsing);
  if (rc) return rc;
  auto op = std::make_unique<Op>();
  op->ctx = &ctx;
  op->op_mask = 3;
  op->precision = precision;
  op->row_offset = scat < 0 ? 0 : m.edge_off[scat];
  op->rows = op->cols = (scat < 0 ? m.ne : m.edge_off[scat + 1] - m.edge_off[scat]);
  op->format = CAL_CSR;
  const int64_t off = op->row_offset;
  std::vector<std::vector<int>> rows(op->rows);
  const int d0 = scat < 0 ? 0 : scat, d1 = scat < 0 ? (int)sp.sing.size() : scat + 1;
  for (int d = d0; d < d1; ++d)
    for (const SingPair& q : sp.sing[d])
      for (int a = 0; a < sp.nslot; ++a)
        for (int b = 0; b < sp.nslot; ++b) {
          const int ea = sp.slot_edge[(size_t)q.t1 * sp.nslot + a], eb = sp.slot_edge[(size_t)q.t2 * sp.nslot + b];
          if (ea < 0 || eb < 0) continue;
          rows[ea - off].push_back((int)(eb - off));
          rows[eb - off].push_back((int)(ea - off));
        }
  op->h_rowptr.assign(op->rows + 1, 0);
  for (int64_t i = 0; i < op->rows; ++i) {
    std::sort(rows[i].begin(), rows[i].end());
    rows[i].erase(std::unique(rows[i].begin(), rows[i].end()), rows[i].end());
    op->h_col.insert(op->h_col.end(), rows[i].begin(), rows[i].end());
    op->h_rowptr[i + 1] = (int64_t)op->h_col.size();
  }
  op->nnz = op->h_rowptr.back();
  const size_t bytes = (size_t)op->nnz * (precision == CAL_FP32 ? 8 : 16);
  cudaStream_t st = ctx.stream;
  CAL_TRY_CUDA(dalloc(&op->d_S, std::max<size_t>(bytes, 16), st));
  CAL_TRY_CUDA(dalloc(&op->d_C, std::max<size_t>(bytes, 16), st));
  CAL_TRY_CUDA(cudaMemsetAsync(op->d_S, 0, bytes, st));
  CAL_TRY_CUDA(cudaMemsetAsync(op->d_C, 0, bytes, st));
  CAL_TRY_CUDA(dalloc((void**)&op->d_rowptr, op->h_rowptr.size() * sizeof(int64_t), st));
  CAL_TRY_CUDA(dalloc((void**)&op->d_col, std::max<size_t>(op->h_col.size(), 1) * sizeof(int), st));
  CAL_TRY_CUDA(cudaMemcpyAsync(op->d_rowptr, op->h_rowptr.data(), op->h_rowptr.size() * sizeof(int64_t),
                               cudaMemcpyHostToDevice, st));
  if (!op->h_col.empty())
    CAL_TRY_CUDA(cudaMemcpyAsync(op->d_col, op->h_col.data(), op->h_col.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 st));
  AssembleArgs a{};
  a.sp = &sp;
  a.scat = scat;
  a.kr = kr;
  a.ki = ki;
  a.want = 3;
  a.nreg = 6;
  a.nsing = nsing;
  a.precision = precision;
  a.sing32 = sing32;
  a.format = CAL_CSR;
  a.row_off = off;
  a.ld = 0;
  a.rowptr = op->d_rowptr;
  a.col = op->d_col;
  a.S = op->d_S;
  a.C = op->d_C;
  a.stream = st;
  if ((rc = launch_singular(a))) return rc;
  // the host pattern must outlive the copies
  CAL_TRY_CUDA(cudaStreamSynchronize(st));
  out = std::move(op);
  return CAL_OK;
}

std::complex<double> interior_k(double k_e, std::complex<double> eps, std::complex<double> mu) {
  std::complex<double> km = k_e * std::sqrt(eps * mu);
  if (km.imag() < 0) km = -km;
  return km;
}

}  // namespace

// =============================================================================
// solution object
// =============================================================================
struct cal_solution {
  Ctx* ctx = nullptr;
  std::shared_ptr<Space> rwg;  // shared with the problem it came from
  std::shared_ptr<Space> bc;   // the mixed discretisation: the space of the second trace
  double2* d_x = nullptr;  // [nrhs][2N]
  // rhs_mode 1: the L2 projection of u^inc onto RWG [nrhs][2N], so that the total
  // trace is d_x + d_cinc (the interior representation needs total traces)
  double2* d_cinc = nullptr;
  int64_t nrhs = 0, ne = 0;
  double k_e = 0.0, mu_e = 1.0;
  std::vector<std::complex<double>> k_m, mu_m;  // per scatterer
  std::vector<double> inc;                      // [nrhs][6] incident plane waves
  int rhs_mode = 0;
  int precision = CAL_FP64;  // of the solve: float32 bulk evaluates its far field in float32
  cal_solve_info info{};
  ~cal_solution() {  // far-field and copy calls are synchronous
    dfree(d_x, nullptr);
    dfree(d_cinc, nullptr);
  }
};

namespace {

struct Pmchwt {
  Ctx* ctx = nullptr;    // context of the call in progress (create or solve)
  Mesh* mesh = nullptr;  // only during create
  int M;
  int64_t N;  // basis count
  double k_e;
  std::vector<std::complex<double>> k_m, mu_m;
  cal_solve_opts o;
  std::shared_ptr<Space> rwg, bc;
  std::unique_ptr<Op> A_ext;
  std::vector<std::unique_ptr<Op>> A_int, P_ext, P_int;
  // Gram
  int64_t* d_grp = nullptr;
  int* d_gcol = nullptr;
  int64_t* d_grpT = nullptr;
  int* d_gcolT = nullptr;
  double* d_gval = nullptr;
  double* d_gvalT = nullptr;
  int64_t gnnz = 0;
  std::unique_ptr<GramSolver<float>> gsA32, gsP32;
  std::unique_ptr<GramSolver<double>> gsA64, gsP64;
  // RWG mass matrix (int phi_i . phi_j) and its solver, for the L2 projection of
  // u^inc in the scattered-trace right-hand side; built on first use
  int64_t* d_mrp = nullptr;
  int* d_mcol = nullptr;
  double* d_mval = nullptr;
  int64_t mnnz = 0;
  std::unique_ptr<GramSolver<double>> gsM;
  // the mixed discretisation (eq. mixed_discretisation, float64): S on RWG (A_ext,
  // A_int), S on BC (Sb_ext on the union, Sb_int per scatterer), C between RWG on
  // the barycentric refinement and BC (dense, rows first: Crb = <C BC, RWG>,
  // Cbr = <C RWG, BC>), the RWG slots on the barycentric triangles, and one Gram
  // solver per half
  bool mixed = false;
  std::unique_ptr<Op> Sb_ext;
  std::vector<std::unique_ptr<Op>> Sb_int;
  double2* Crb_ext = nullptr;
  double2* Cbr_ext = nullptr;
  std::vector<double2*> Crb_int, Cbr_int;
  int* d_redge = nullptr;
  double* d_rsw = nullptr;
  std::unique_ptr<GramSolver<double>> gmA, gmP;
  // batch of right-hand sides advanced in lockstep
  int nb = 1;
  // work vectors [nb][2N] (complex128-sized)
  void* t1 = nullptr;
  void* t2 = nullptr;
  double2* d_gath = nullptr;
  void* d_xt = nullptr;  // right-hand-side-interleaved copy of x for the CSR blocks
  // tensor-core product buffers
  int NB = 0;
  float* d_Bt = nullptr;
  float* d_Bh = nullptr;  // TF32 part and remainder of d_Bt
  float* d_Bl = nullptr;
  float* d_ZS = nullptr;
  float* d_ZC = nullptr;
  int* d_gemm_err = nullptr;
  int64_t matvecs = 0;
  // float32 combined blocks for the one-vector float32 product (reading 18):
  // C = C_e + C_i, S1 = alpha_e S_e + alpha_i S_i, S2 = beta_e S_e + beta_i S_i
  struct Combo {
    void* C = nullptr;
    void* S1 = nullptr;
    void* S2 = nullptr;
    int64_t rows = 0, off = 0;
  };
  Combo cA;
  std::vector<Combo> cP;
  ~Pmchwt() {
    cudaStream_t st = nullptr;  // every solve has completed: the legacy stream orders the release
    for (void* p : {(void*)d_grp, (void*)d_gcol, (void*)d_grpT, (void*)d_gcolT, (void*)d_gval, (void*)d_gvalT, t1,
                    t2, (void*)d_gath, d_xt, (void*)d_Bt, (void*)d_Bh, (void*)d_Bl, (void*)d_ZS, (void*)d_ZC,
                    (void*)d_gemm_err, (void*)d_mrp, (void*)d_mcol, (void*)d_mval})
      dfree(p, st);
    free_combo(cA);
    for (auto& c : cP) free_combo(c);
    for (void* p : {(void*)Crb_ext, (void*)Cbr_ext, (void*)d_redge, (void*)d_rsw}) dfree(p, st);
    for (auto* v : {&Crb_int, &Cbr_int})
      for (double2* p : *v) dfree(p, st);
  }
  static void free_combo(Combo& c) {
    for (void* p : {c.C, c.S1, c.S2}) dfree(p, nullptr);
    c = Combo{};
  }
  int alloc_combo(Combo& c, int64_t rows, int64_t off, cudaStream_t st) {
    c.rows = rows;
    c.off = off;
    const size_t bytes = (size_t)rows * rows * sizeof(float2);
    for (void** p : {&c.C, &c.S1, &c.S2})
      if (dalloc(p, std::max<size_t>(bytes, 16), st) != cudaSuccess) {
        free_combo(c);
        cudaGetLastError();
        return fail(CAL_ENOMEM, "combined block: cannot allocate %zu bytes", bytes);
      }
    return CAL_OK;
  }
  // A: the exterior pair on the union with every interior pair on its diagonal
  int build_combo_A(cudaStream_t st) {
    if (o.precision != CAL_FP32 || o.matrix_free || !A_ext || A_ext->format != CAL_DENSE || !A_ext->d_S ||
        !A_ext->d_C || A_ext->rows % 2)
      return CAL_OK;
    for (auto& a : A_int)
      if (!a || a->format != CAL_DENSE || !a->d_S || !a->d_C) return CAL_OK;
    int rc = alloc_combo(cA, N, 0, st);
    if (rc) return rc;
    const std::complex<double> ae = 1.0 / k_e, be = -k_e;
    const bool whole = M == 1 && A_int[0]->rows == N;
    if (!whole && (rc = combine_blocks(A_ext->d_S, A_ext->d_C, N, ae, be, nullptr, nullptr, 0, 0, 0.0, 0.0, cA.C,
                                       cA.S1, cA.S2, true, ctx->n_sm, st)))
      return rc;
    for (int m = 0; m < M; ++m) {
      const std::complex<double> am = mu_m[m] / k_m[m], bm = -k_m[m] / mu_m[m];
      if ((rc = combine_blocks(A_ext->d_S, A_ext->d_C, N, ae, be, A_int[m]->d_S, A_int[m]->d_C, A_int[m]->rows,
                               A_int[m]->row_offset, am, bm, cA.C, cA.S1, cA.S2, false, ctx->n_sm, st)))
        return rc;
    }
    return CAL_OK;
  }
  // P = D: the exterior and interior pairs of each scatterer
  int build_combo_P(cudaStream_t st) {
    if (o.precision != CAL_FP32 || o.precond != CAL_PRECOND_D || (int)P_ext.size() != M || (int)P_int.size() != M)
      return CAL_OK;
    // the streaming kernel reads x in 16-byte words: even offsets and N
    for (int m = 0; m < M; ++m)
      for (Op* a : {P_ext[m].get(), P_int[m].get()})
        if (!a || a->format != CAL_DENSE || !a->d_S || !a->d_C || a->rows % 2 || a->row_offset % 2 || N % 2)
          return CAL_OK;
    cP.resize(M);
    for (int m = 0; m < M; ++m) {
      const int64_t n = P_ext[m]->rows;
      int rc = alloc_combo(cP[m], n, P_ext[m]->row_offset, st);
      if (!rc)
        rc = combine_blocks(P_ext[m]->d_S, P_ext[m]->d_C, n, 1.0 / k_e, -k_e, P_int[m]->d_S, P_int[m]->d_C, n, 0,
                            mu_m[m] / k_m[m], -k_m[m] / mu_m[m], cP[m].C, cP[m].S1, cP[m].S2, false, ctx->n_sm,
                            st);
      if (rc) {
        for (auto& c : cP) free_combo(c);
        cP.clear();
        return rc;
      }
    }
    return CAL_OK;
  }
  // one float32 vector through a combined block: y += (C x1 + S1 x2, C x2 + S2 x1)
  int apply_combo(const Combo& c, const void* x, void* y) {
    BlockRef b;
    b.C = c.C;
    b.S = c.S1;
    b.S2 = c.S2;
    b.rows = b.cols = c.rows;
    b.row_off = b.col_off = c.off;
    b.precision = CAL_FP32;
    return pair_apply(b, CAL_FP32, x, y, N, 1.0, 0.0, 1.0, 0.0, ctx->stream);
  }

  BlockRef ref(const Op& op, bool withS = true, bool withC = true) const {
    BlockRef b;
    b.S = withS ? op.d_S : nullptr;
    b.C = withC ? op.d_C : nullptr;
    b.rows = op.rows;
    b.cols = op.cols;
    b.row_off = b.col_off = op.row_offset;
    b.precision = op.precision;
    b.rowptr = op.format == CAL_CSR ? op.d_rowptr : nullptr;
    b.col = op.format == CAL_CSR ? op.d_col : nullptr;
    if (op.hmat) {
      b.hmat = op.hmat;
      b.hmask = (withS ? 1 : 0) | (withC ? 2 : 0);
    }
    return b;
  }

  // Batch state for nbatch right-hand sides in lockstep: work vectors,
  // tensor-core product buffers and the Gram solvers (2 nbatch systems).
  // Kept between solves of the same batch width.
  int setup_batch(int nbatch) {
    if (nbatch == nb && t1) return CAL_OK;
    for (void* p : {t1, t2, (void*)d_gath, d_xt, (void*)d_Bt, (void*)d_Bh, (void*)d_Bl, (void*)d_ZS, (void*)d_ZC,
                    (void*)d_gemm_err})
      dfree(p, nullptr);  // the previous solve has completed
    t1 = t2 = nullptr;
    d_gath = nullptr;
    d_xt = nullptr;
    d_Bt = d_Bh = d_Bl = d_ZS = d_ZC = nullptr;
    d_gemm_err = nullptr;
    NB = 0;
    gsA32.reset();
    gsP32.reset();
    gsA64.reset();
    gsP64.reset();
    cudaStream_t st = ctx->stream;
    int rc;
    if (mixed) {
      gmA.reset();
      gmP.reset();
      gmA = std::make_unique<GramSolver<double>>();
      gmP = std::make_unique<GramSolver<double>>();
      if ((rc = gmA->init(d_grp, d_gcol, d_gval, N, 1, gnnz, 1.0, 1e-13, 30, st))) return rc;
      if ((rc = gmP->init(d_grpT, d_gcolT, d_gvalT, N, 1, gnnz, -1.0, 1e-13, 30, st))) return rc;
    } else if (o.precond != CAL_PRECOND_NONE) {
      // M_A = diag(G, G); M_P = diag(-G^T, -G^T): two component systems per vector
      if (o.precision == CAL_FP64) {
        gsA64 = std::make_unique<GramSolver<double>>();
        gsP64 = std::make_unique<GramSolver<double>>();
        if ((rc = gsA64->init(d_grp, d_gcol, d_gval, N, 2 * nbatch, gnnz, 1.0, 1e-13, 30, st))) return rc;
        if ((rc = gsP64->init(d_grpT, d_gcolT, d_gvalT, N, 2 * nbatch, gnnz, -1.0, 1e-13, 30, st))) return rc;
      } else {
        gsA32 = std::make_unique<GramSolver<float>>();
        gsP32 = std::make_unique<GramSolver<float>>();
        if ((rc = gsA32->init(d_grp, d_gcol, d_gval, N, 2 * nbatch, gnnz, 1.0, 1e-6, 14, st))) return rc;
        if ((rc = gsP32->init(d_grpT, d_gcolT, d_gvalT, N, 2 * nbatch, gnnz, -1.0, 1e-6, 14, st))) return rc;
      }
    }
    return alloc_batch(nbatch);
  }

  int alloc_batch(int nrhs) {
    nb = nrhs;
    const size_t vbytes = (size_t)nb * 2 * N * sizeof(double2);
    cudaStream_t st = ctx->stream;
    CAL_TRY_CUDA(dalloc(&t1, vbytes, st));
    CAL_TRY_CUDA(dalloc(&t2, vbytes, st));
    CAL_TRY_CUDA(dalloc((void**)&d_gath, vbytes, st));
    CAL_TRY_CUDA(dalloc(&d_xt, vbytes, st));
    if (o.precision == CAL_FP32 && nb >= 4 && gemm_tc_supported(2, nb)) {
      NB = ((4 * nb + 15) / 16) * 16;
      int64_t maxrows = A_ext->rows;
      CAL_TRY_CUDA(dalloc((void**)&d_Bt, (size_t)NB * 2 * maxrows * sizeof(float), st));
      CAL_TRY_CUDA(dalloc((void**)&d_Bh, (size_t)NB * 2 * maxrows * sizeof(float), st));
      CAL_TRY_CUDA(dalloc((void**)&d_Bl, (size_t)NB * 2 * maxrows * sizeof(float), st));
      CAL_TRY_CUDA(dalloc((void**)&d_ZS, (size_t)maxrows * NB * sizeof(float), st));
      CAL_TRY_CUDA(dalloc((void**)&d_ZC, (size_t)maxrows * NB * sizeof(float), st));
      CAL_TRY_CUDA(dalloc((void**)&d_gemm_err, sizeof(int), st));
      CAL_TRY_CUDA(cudaMemsetAsync(d_gemm_err, 0, sizeof(int), st));
    }
    return CAL_OK;
  }

  // y += block applied to x for nrhs right-hand sides ([nrhs][2N] each)
  int apply_block(const BlockRef& b, const void* x, void* y, int vec_prec, int nrhs, std::complex<double> al,
                  std::complex<double> be) {
    cudaStream_t st = ctx->stream;
    if (b.hmat) {
      const size_t vsz = vec_prec == CAL_FP64 ? sizeof(double2) : sizeof(float2);
      for (int q = 0; q < nrhs; ++q) {
        int rc = hmat_pair_apply(*b.hmat, b.hmask & 1, b.hmask & 2, vec_prec, (const char*)x + q * 2 * N * vsz,
                                 (char*)y + q * 2 * N * vsz, N, b.row_off, al.real(), al.imag(), be.real(), be.imag(),
                                 st);
        if (rc) return rc;
      }
      return CAL_OK;
    }
    const bool dense32 = b.precision == CAL_FP32 && !b.rowptr && vec_prec == CAL_FP32;
    if (dense32 && d_Bt && nrhs == nb && gemm_tc_supported(b.cols, nrhs)) {
      int rc;
      const float2* X = (const float2*)x;
      if ((rc = embed_rhs<float2>(X, nrhs, N, b.col_off, b.cols, d_Bt, NB, st))) return rc;
      const int64_t K = 2 * b.cols;
      // the vectors are split into TF32 parts once per product; the operator is
      // read as float32 and split in the kernel
      if ((rc = split_tf32(d_Bt, d_Bh, d_Bl, (int64_t)NB * K, st))) return rc;
      const float* ZS = nullptr;
      const float* ZC = nullptr;
      if (b.S) {
        if ((rc = gemm_tf32x3_bsplit((const float*)b.S, b.rows, K, d_Bh, d_Bl, NB, d_ZS, d_gemm_err, ctx->n_sm, st)))
          return rc;
        ZS = d_ZS;
      }
      if (b.C) {
        if ((rc = gemm_tf32x3_bsplit((const float*)b.C, b.rows, K, d_Bh, d_Bl, NB, d_ZC, d_gemm_err, ctx->n_sm, st)))
          return rc;
        ZC = d_ZC;
      }
      return combine_rhs<float2>(ZS, ZC, b.rows, NB, nrhs, N, b.row_off, (float2*)y, al.real(), al.imag(),
                                 be.real(), be.imag(), st);
    }
    if (b.precision == CAL_FP32 && !b.rowptr && nrhs >= 2)
      return pair_apply_multi(b, vec_prec, x, y, N, nrhs, al.real(), al.imag(), be.real(), be.imag(), ctx->n_sm,
                              st);
    if (b.rowptr && nrhs >= 2 && d_xt && nrhs <= nb)
      return pair_spmv_multi(b, vec_prec, x, y, N, nrhs, al.real(), al.imag(), be.real(), be.imag(), d_xt, st);
    const size_t vsz = vec_prec == CAL_FP64 ? sizeof(double2) : sizeof(float2);
    for (int q = 0; q < nrhs; ++q) {
      int rc = pair_apply(b, vec_prec, (const char*)x + q * 2 * N * vsz, (char*)y + q * 2 * N * vsz, N, al.real(),
                          al.imag(), be.real(), be.imag(), st);
      if (rc) return rc;
    }
    return CAL_OK;
  }

  // y = A x (y overwritten); vec_prec = precision of x, y
  int apply_A(const void* x, void* y, int vec_prec, int nrhs) {
    cudaStream_t st = ctx->stream;
    int rc = zero_vec(y, vec_prec, 2 * N * nrhs, st);
    if (rc) return rc;
    if (vec_prec == CAL_FP32 && nrhs == 1 && cA.C) {
      if ((rc = apply_combo(cA, x, y))) return rc;
      matvecs += 4LL * M * M + 4LL * M;
      return CAL_OK;
    }
    const std::complex<double> ae = 1.0 / k_e, be = -k_e;  // mu_e = 1
    if ((rc = apply_block(ref(*A_ext), x, y, vec_prec, nrhs, ae, be))) return rc;
    if (o.matrix_free &&
        (rc = launch_rwg_free(*rwg, -1, k_e, 0.0, o.q_regular_A, o.precision, vec_prec, x, y, N, nrhs, ae.real(),
                              ae.imag(), be.real(), be.imag(), st)))
      return rc;
    for (int m = 0; m < M; ++m) {
      const std::complex<double> am = mu_m[m] / k_m[m], bm = -k_m[m] / mu_m[m];
      if ((rc = apply_block(ref(*A_int[m]), x, y, vec_prec, nrhs, am, bm))) return rc;
      if (o.matrix_free &&
          (rc = launch_rwg_free(*rwg, m, k_m[m].real(), k_m[m].imag(), o.q_regular_A, o.precision, vec_prec, x, y,
                                N, nrhs, am.real(), am.imag(), bm.real(), bm.imag(), st)))
        return rc;
    }
    matvecs += (4LL * M * M + 4LL * M) * nrhs;
    return CAL_OK;
  }

  // ---- the mixed discretisation ------------------------------------------
  // RWG on the barycentric refinement: on a child tau of primal triangle t the
  // piece sigma (x - c_t) + w_t is sigma (x - c_tau) + (w_t + sigma (c_tau - c_t))
  int build_rwgb(cudaStream_t st) {
    const Space& R = *rwg;
    const Space& B = *bc;
    std::vector<int> edge(3 * B.ntri);
    std::vector<double> sw(12 * B.ntri);
    for (int64_t tau = 0; tau < B.ntri; ++tau) {
      const int t = B.parent[tau];
      for (int a = 0; a < 3; ++a) {
        edge[3 * tau + a] = R.slot_edge[3 * t + a];
        const double* ps = &R.slot_sw[(3 * (size_t)t + a) * 4];
        double* q = &sw[(3 * (size_t)tau + a) * 4];
        q[0] = ps[0];
        for (int c = 0; c < 3; ++c) q[1 + c] = ps[1 + c] + ps[0] * (B.triD[tau].c[c] - R.triD[t].c[c]);
      }
    }
    CAL_TRY_CUDA(dalloc((void**)&d_redge, edge.size() * sizeof(int), st));
    CAL_TRY_CUDA(dalloc((void**)&d_rsw, sw.size() * sizeof(double), st));
    CAL_TRY_CUDA(cudaMemcpyAsync(d_redge, edge.data(), edge.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CAL_TRY_CUDA(cudaMemcpyAsync(d_rsw, sw.data(), sw.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CAL_TRY_CUDA(cudaStreamSynchronize(st));  // the host tables are read by the copies
    return CAL_OK;
  }

  // y += the mixed block of one wavenumber on rows/cols [off, off + n):
  // y1 += -(k/mu) Srr x1 + Crb x2, y2 += Cbr x1 + (mu/k) Sbb x2, the four
  // matrices at (r0, r0) of their storage with leading dimension ld
  int mixed_block(const double2* Srr, const double2* Sbb, const double2* Crb, const double2* Cbr, int64_t ld,
                  int64_t r0, int64_t off, int64_t n, std::complex<double> k, std::complex<double> mu,
                  const double2* x, double2* y) {
    cudaStream_t st = ctx->stream;
    const int64_t at = r0 * ld + r0;
    const double2 *x1 = x + off, *x2 = x + N + off;
    double2 *y1 = y + off, *y2 = y + N + off;
    int rc;
    if ((rc = gemv_acc(Srr + at, ld, n, n, x1, y1, -k / mu, st)) || (rc = gemv_acc(Crb + at, ld, n, n, x2, y1, 1.0, st)) ||
        (rc = gemv_acc(Cbr + at, ld, n, n, x1, y2, 1.0, st)) || (rc = gemv_acc(Sbb + at, ld, n, n, x2, y2, mu / k, st)))
      return rc;
    return CAL_OK;
  }

  // y = A x (diag_only: the diagonal blocks, P = D), float64, one vector
  int mixed_apply(const double2* x, double2* y, bool diag_only) {
    cudaStream_t st = ctx->stream;
    int rc = zero_vec(y, CAL_FP64, 2 * N, st);
    if (rc) return rc;
    const double2* SeR = (const double2*)A_ext->d_S;
    const double2* SeB = (const double2*)Sb_ext->d_S;
    if (!diag_only) {
      if ((rc = mixed_block(SeR, SeB, Crb_ext, Cbr_ext, N, 0, 0, N, k_e, 1.0, x, y))) return rc;
    }
    for (int m = 0; m < M; ++m) {
      const int64_t off = A_int[m]->row_offset, n = A_int[m]->rows;
      if (diag_only && (rc = mixed_block(SeR, SeB, Crb_ext, Cbr_ext, N, off, off, n, k_e, 1.0, x, y))) return rc;
      if ((rc = mixed_block((const double2*)A_int[m]->d_S, (const double2*)Sb_int[m]->d_S, Crb_int[m], Cbr_int[m], n,
                            0, off, n, k_m[m], mu_m[m], x, y)))
        return rc;
    }
    matvecs += diag_only ? 8LL * M : 4LL * M * M + 4LL * M;
    return CAL_OK;
  }

  // w = M^-1 y with M = [[0, G], [-G^T, 0]]: w2 = G^-1 y1, w1 = -G^-T y2
  int mixed_minv(const double2* y, double2* w) {
    cudaStream_t st = ctx->stream;
    int rc;
    if ((rc = gmA->solve(y, w + N, st))) return rc;
    return gmP->solve(y + N, w, st);
  }

  // y = A^i x = diag(A^i_m) x, the interior blocks only (y overwritten)
  int apply_Ai(const void* x, void* y, int vec_prec, int nrhs) {
    cudaStream_t st = ctx->stream;
    int rc = zero_vec(y, vec_prec, 2 * N * nrhs, st);
    if (rc) return rc;
    for (int m = 0; m < M; ++m) {
      const std::complex<double> am = mu_m[m] / k_m[m], bm = -k_m[m] / mu_m[m];
      if ((rc = apply_block(ref(*A_int[m]), x, y, vec_prec, nrhs, am, bm))) return rc;
      if (o.matrix_free &&
          (rc = launch_rwg_free(*rwg, m, k_m[m].real(), k_m[m].imag(), o.q_regular_A, o.precision, vec_prec, x, y,
                                N, nrhs, am.real(), am.imag(), bm.real(), bm.imag(), st)))
        return rc;
    }
    return CAL_OK;
  }

  // RWG mass matrix on the device: the pattern holds every pair of edges of one
  // triangle, the values come from one kernel
  int build_mass() {
    if (d_mval) return CAL_OK;
    cudaStream_t st = ctx->stream;
    const Space& sp = *rwg;
    std::vector<std::vector<int>> rows(N);
    for (int64_t t = 0; t < sp.ntri; ++t)
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          const int ea = sp.slot_edge[3 * t + a], eb = sp.slot_edge[3 * t + b];
          if (ea >= 0 && eb >= 0) rows[ea].push_back(eb);
        }
    std::vector<int64_t> rp(N + 1, 0);
    std::vector<int> col;
    for (int64_t i = 0; i < N; ++i) {
      std::sort(rows[i].begin(), rows[i].end());
      rows[i].erase(std::unique(rows[i].begin(), rows[i].end()), rows[i].end());
      col.insert(col.end(), rows[i].begin(), rows[i].end());
      rp[i + 1] = (int64_t)col.size();
    }
    mnnz = (int64_t)col.size();
    CAL_TRY_CUDA(dalloc((void**)&d_mrp, (N + 1) * sizeof(int64_t), st));
    CAL_TRY_CUDA(dalloc((void**)&d_mcol, std::max<int64_t>(mnnz, 1) * sizeof(int), st));
    CAL_TRY_CUDA(dalloc((void**)&d_mval, std::max<int64_t>(mnnz, 1) * sizeof(double), st));
    CAL_TRY_CUDA(cudaMemcpyAsync(d_mrp, rp.data(), (N + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CAL_TRY_CUDA(cudaMemcpyAsync(d_mcol, col.data(), mnnz * sizeof(int), cudaMemcpyHostToDevice, st));
    CAL_TRY_CUDA(cudaMemsetAsync(d_mval, 0, mnnz * sizeof(double), st));
    int rc = launch_rwg_mass(sp, d_mrp, d_mcol, d_mval, st);
    CAL_TRY_CUDA(cudaStreamSynchronize(st));  // the host pattern is read by the copies
    return rc;
  }

  // The paper's scattered-trace right-hand side (eq. PMCHWT_multiple_scatterers):
  // b = (1/2 I - D^i) u^inc tested, D^i = diag(A^i_m). The identity term is the
  // exactly tested incident trace (b_tot, the total-trace right-hand side, on
  // entry); D^i acts on the L2 projection c of u^inc onto RWG (mass matrix
  // int phi_i . phi_j, loads int phi_i . (field x n)). b [nrhs][2N] is replaced by
  // b_tot / 2 - A^i c; c [nrhs][2N] is kept (the incident part of the total
  // trace). Batches of nb right-hand sides.
  int scattered_rhs(const double* d_inc, int64_t nrhs, double2* b, double2* c) {
    cudaStream_t st = ctx->stream;
    int rc;
    if ((rc = build_mass())) return rc;
    const int64_t n2 = 2 * N;
    double2* load = nullptr;
    double2* y = nullptr;
    CAL_TRY_CUDA(dalloc((void**)&load, (size_t)nb * n2 * sizeof(double2), st));
    if (dalloc((void**)&y, (size_t)nb * n2 * sizeof(double2), st) != cudaSuccess) {
      dfree(load, st);
      return fail(CAL_ENOMEM, "scattered right-hand side: cannot allocate work vectors");
    }
    for (int64_t q0 = 0; q0 < nrhs && !rc; q0 += nb) {
      const int nq = (int)std::min<int64_t>(nb, nrhs - q0);
      if (!gsM || gsM->nsys != 2 * nq) {
        gsM = std::make_unique<GramSolver<double>>();
        if ((rc = gsM->init(d_mrp, d_mcol, d_mval, N, 2 * nq, mnnz, 1.0, 1e-13, 200, st))) break;
      }
      if ((rc = launch_rhs(*rwg, d_inc + 6 * q0, nq, k_e, 1.0, load, st, 1))) break;
      if ((rc = gsM->solve(load, c + q0 * n2, st))) break;
      if ((rc = apply_Ai(c + q0 * n2, y, CAL_FP64, nq))) break;
      if ((rc = vec_axpby(b + q0 * n2, 0.5, y, -1.0, b + q0 * n2, nq * n2, st))) break;
    }
    dfree(load, st);
    dfree(y, st);
    if (!rc && gsM) rc = gsM->check(st);
    return rc;
  }

  // y = P x on BC coefficients (y overwritten)
  int apply_P(const void* x, void* y, int vec_prec, int nrhs) {
    cudaStream_t st = ctx->stream;
    int rc = zero_vec(y, vec_prec, 2 * N * nrhs, st);
    if (rc) return rc;
    const int pc = o.precond;
    const bool ext = pc == CAL_PRECOND_D || pc == CAL_PRECOND_DE || pc == CAL_PRECOND_SE;
    const bool in = pc == CAL_PRECOND_D || pc == CAL_PRECOND_DI || pc == CAL_PRECOND_SI;
    const bool onlyS = pc == CAL_PRECOND_SE || pc == CAL_PRECOND_SI;
    if (vec_prec == CAL_FP32 && nrhs == 1 && !cP.empty()) {
      for (const Combo& c : cP)
        if ((rc = apply_combo(c, x, y))) return rc;
      matvecs += 8LL * M;
      return CAL_OK;
    }
    for (int m = 0; m < M; ++m) {
      if (ext && (rc = apply_block(ref(*P_ext[m], true, !onlyS), x, y, vec_prec, nrhs, 1.0 / k_e, -k_e))) return rc;
      if (in && (rc = apply_block(ref(*P_int[m], true, !onlyS), x, y, vec_prec, nrhs, mu_m[m] / k_m[m],
                                  -k_m[m] / mu_m[m])))
        return rc;
    }
    matvecs += ((ext ? (onlyS ? 2 : 4) : 0) + (in ? (onlyS ? 2 : 4) : 0)) * (int64_t)M * nrhs;
    return CAL_OK;
  }

  // w = M_P^-1 P M_A^-1 y for nrhs vectors; y, w float64 [nrhs][2N]
  int apply_precond(const double2* y, double2* w, int nrhs) {
    cudaStream_t st = ctx->stream;
    int rc;
    const int64_t n2 = 2 * N * nrhs;
    if (mixed) {  // w = M^-1 D M^-1 y (one vector)
      double2* a = (double2*)t1;
      double2* b = (double2*)t2;
      if ((rc = mixed_minv(y, a)) || (rc = mixed_apply(a, b, true))) return rc;
      return mixed_minv(b, w);
    }
    if (o.precond == CAL_PRECOND_NONE) {
      CAL_TRY_CUDA(cudaMemcpyAsync(w, y, n2 * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      return CAL_OK;
    }
    if (o.precision == CAL_FP64) {
      double2* a = (double2*)t1;
      double2* b = (double2*)t2;
      if ((rc = gsA64->solve(y, a, st))) return rc;
      if ((rc = apply_P(a, b, CAL_FP64, nrhs))) return rc;
      return gsP64->solve(b, w, st);
    }
    float2* a = (float2*)t1;
    float2* b = (float2*)t2;
    if ((rc = convert_vec(y, CAL_FP64, b, CAL_FP32, n2, 1.0, st))) return rc;
    if ((rc = gsA32->solve(b, a, st))) return rc;
    if ((rc = apply_P(a, b, CAL_FP32, nrhs))) return rc;
    if ((rc = gsP32->solve(b, a, st))) return rc;
    return convert_vec(a, CAL_FP32, w, CAL_FP64, n2, 1.0, st);
  }

  // w = B v, B = M_P^-1 P M_A^-1 A ; v, w float64 [nb][2N]
  int apply_B(const double2* v, double2* w, double2* scratch) {
    int rc;
    cudaStream_t st = ctx->stream;
    const int64_t n2 = 2 * N * nb;
    if (mixed) {
      if ((rc = mixed_apply(v, scratch, false))) return rc;
      return apply_precond(scratch, w, 1);
    }
    if (o.precision == CAL_FP64) {
      if ((rc = apply_A(v, scratch, CAL_FP64, nb))) return rc;
      return apply_precond(scratch, w, nb);
    }
    float2* a = (float2*)t1;
    float2* b = (float2*)t2;
    if ((rc = convert_vec(v, CAL_FP64, a, CAL_FP32, n2, 1.0, st))) return rc;
    if ((rc = apply_A(a, b, CAL_FP32, nb))) return rc;
    if (o.precond == CAL_PRECOND_NONE) return convert_vec(b, CAL_FP32, w, CAL_FP64, n2, 1.0, st);
    if ((rc = gsA32->solve(b, a, st))) return rc;
    if ((rc = apply_P(a, b, CAL_FP32, nb))) return rc;
    if ((rc = gsP32->solve(b, a, st))) return rc;
    return convert_vec(a, CAL_FP32, w, CAL_FP64, n2, 1.0, st);
  }

  // Restarted GMRES on B d_q = rhs_q for the nb right-hand sides in lockstep,
  // d_q0 = 0, added into x_q. Per-column relative targets tol[q]; a column
  // stops when its Givens residual (or explicit residual after a complete
  // cycle) meets its target, and its iterate is updated at that point.
  int gmres(const double2* rhs, double2* x, const std::vector<double>& tol, std::vector<int>& iters,
            std::vector<double>& rel_res, int maxit) {
    cudaStream_t st = ctx->stream;
    const int64_t n = 2 * N;
    const int m = std::max(1, std::min<int>(o.restart, maxit));
    const int q_n = nb;
    double2 *V, *w, *scr, *H, *cs, *sn, *g, *h1, *h2, *y, *r;
    double *dscal, *hres;
    const size_t vb = n * sizeof(double2);
    const int64_t bV = (int64_t)(m + 1) * n, bH = (int64_t)(m + 1) * m, bh = m + 2;
    CAL_TRY_CUDA(cudaMallocAsync((void**)&V, q_n * bV * sizeof(double2), st));
    CAL_TRY_CUDA(cudaMallocAsync((void**)&w, q_n * vb, st));
    CAL_TRY_CUDA(cudaMallocAsync((void**)&scr, q_n * vb, st));
    CAL_TRY_CUDA(cudaMallocAsync((void**)&r, q_n * vb, st));
    CAL_TRY_CUDA(cudaMallocAsync((void**)&H, q_n * bH * sizeof(double2), st));
    CAL_TRY_CUDA(cudaMallocAsync((void**)&cs, q_n * bh * sizeof(double2), st));
    CAL_TRY_CUDA(cudaMallocAsync((void**)&sn, q_n * bh * sizeof(double2), st));
    CAL_TRY_CUDA(cudaMallocAsync((void**)&g, q_n * bh * sizeof(double2), st));
    CAL_TRY_CUDA(cudaMallocAsync((void**)&h1, q_n * bh * sizeof(double2), st));
    CAL_TRY_CUDA(cudaMallocAsync((void**)&h2, q_n * bh * sizeof(double2), st));
    CAL_TRY_CUDA(cudaMallocAsync((void**)&y, q_n * bh * sizeof(double2), st));
    CAL_TRY_CUDA(cudaMallocAsync((void**)&dscal, q_n * 4 * sizeof(double), st));
    hres = ctx->pinned;  // 4 doubles per right-hand side; q_n <= 32
    std::vector<double2> gh(q_n * bh);
    int rc = CAL_OK;
    auto cleanup = [&]() {
      cudaFreeAsync(V, st); cudaFreeAsync(w, st); cudaFreeAsync(scr, st); cudaFreeAsync(r, st);
      cudaFreeAsync(H, st); cudaFreeAsync(cs, st); cudaFreeAsync(sn, st); cudaFreeAsync(g, st);
      cudaFreeAsync(h1, st); cudaFreeAsync(h2, st); cudaFreeAsync(y, st); cudaFreeAsync(dscal, st);
      cudaStreamSynchronize(st);
    };
    iters.assign(q_n, 0);
    rel_res.assign(q_n, 0.0);
    // ||rhs_q||
    if ((rc = vec_norm2(rhs, n, dscal, 4, q_n, st))) { cleanup(); return rc; }
    CAL_TRY_CUDA(cudaMemcpyAsync(hres, dscal, q_n * 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CAL_TRY_CUDA(cudaStreamSynchronize(st));
    std::vector<double> bnorm(q_n), beta(q_n);
    std::vector<char> active(q_n);
    int n_active = 0;
    for (int q = 0; q < q_n; ++q) {
      bnorm[q] = std::sqrt(hres[4 * q]);
      beta[q] = bnorm[q];
      active[q] = bnorm[q] > 0.0;
      n_active += active[q];
    }
    CAL_TRY_CUDA(cudaMemcpyAsync(r, rhs, q_n * vb, cudaMemcpyDeviceToDevice, st));
    int it = 0;
    while (n_active > 0 && it < maxit) {
      // V0 = r / beta, g = (beta, 0, ...)
      std::fill(gh.begin(), gh.end(), double2{0.0, 0.0});
      for (int q = 0; q < q_n; ++q) {
        gh[q * bh] = {beta[q], 0.0};
        hres[4 * q + 1] = beta[q] * beta[q];
      }
      CAL_TRY_CUDA(cudaMemcpyAsync(g, gh.data(), gh.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
      for (int q = 0; q < q_n; ++q)
        CAL_TRY_CUDA(cudaMemcpyAsync(dscal + 4 * q + 1, hres + 4 * q + 1, sizeof(double), cudaMemcpyHostToDevice, st));
      if ((rc = gmres_scale(r, n, n, dscal + 1, 4, V, bV, q_n, st))) break;
      std::vector<char> cycle_active = active;
      int j = 0;
      for (; j < m && it < maxit; ++j) {
        if ((rc = vec_gather(V + (size_t)j * n, bV, d_gath, n, q_n, st))) break;
        if ((rc = apply_B(d_gath, w, scr))) break;
        ++it;
        if ((rc = gmres_cgs_step(V, bV, n, j, w, h1, h2, bh, dscal + 2, 4, q_n, st))) break;
        if ((rc = gmres_givens(H, m + 1, bH, j, h1, h2, bh, dscal + 2, 4, cs, sn, bh, g, bh, dscal + 3, 4, q_n, st)))
          break;
        if ((rc = gmres_scale(w, n, n, dscal + 2, 4, V + (size_t)(j + 1) * n, bV, q_n, st))) break;
        CAL_TRY_CUDA(cudaMemcpyAsync(hres, dscal, q_n * 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CAL_TRY_CUDA(cudaStreamSynchronize(st));
        for (int q = 0; q < q_n; ++q) {
          if (!cycle_active[q]) continue;
          ++iters[q];
          rel_res[q] = hres[4 * q + 3] / bnorm[q];
          if (!std::isfinite(rel_res[q])) { rc = fail(CAL_ECUDA, "GMRES: non-finite residual"); break; }
          if (rel_res[q] <= tol[q] && j < m - 1) {
            // this column has converged inside the cycle: update it now
            if ((rc = gmres_update(H + q * bH, m + 1, j + 1, g + q * bh, y + q * bh, V + q * bV, n, x + q * n, st)))
              break;
            cycle_active[q] = 0;
            active[q] = 0;
            --n_active;
          }
        }
        if (rc || n_active == 0) { ++j; break; }
      }
      if (rc) break;
      const int ncol = std::min(j, m);
      for (int q = 0; q < q_n; ++q)
        if (cycle_active[q] && (rc = gmres_update(H + q * bH, m + 1, ncol, g + q * bh, y + q * bh, V + q * bV, n,
                                                  x + q * n, st)))
          break;
      if (rc || n_active == 0 || it >= maxit) break;
      // end of a full cycle: explicit residual r = rhs - B x
      if ((rc = apply_B(x, w, scr))) break;
      if ((rc = vec_axpby(rhs, 1.0, w, -1.0, r, n * q_n, st))) break;
      if ((rc = vec_norm2(r, n, dscal, 4, q_n, st))) break;
      CAL_TRY_CUDA(cudaMemcpyAsync(hres, dscal, q_n * 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
      CAL_TRY_CUDA(cudaStreamSynchronize(st));
      for (int q = 0; q < q_n; ++q) {
        if (!active[q]) continue;
        beta[q] = std::sqrt(hres[4 * q]);
        rel_res[q] = beta[q] / bnorm[q];
        if (rel_res[q] <= tol[q]) { active[q] = 0; --n_active; }
      }
    }
    cleanup();
    return rc;
  }

  // relative 2-norms of the nb columns of a [nb][2N] float64 block
  int norms(const double2* v, std::vector<double>& out) {
    cudaStream_t st = ctx->stream;
    double* dn;
    std::vector<double> h(4 * nb);
    CAL_TRY_CUDA(cudaMallocAsync((void**)&dn, 4 * nb * sizeof(double), st));
    int rc = vec_norm2(v, 2 * N, dn, 4, nb, st);
    CAL_TRY_CUDA(cudaMemcpyAsync(h.data(), dn, 4 * nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    CAL_TRY_CUDA(cudaFreeAsync(dn, st));
    CAL_TRY_CUDA(cudaStreamSynchronize(st));
    out.resize(nb);
    for (int q = 0; q < nb; ++q) out[q] = std::sqrt(h[4 * q]);
    return rc;
  }
};

void opts_default(cal_solve_opts* o) {
  o->precond = CAL_PRECOND_D;
  o->precision = CAL_FP32;
  o->q_regular_A = 6;
  o->q_singular_A = 4;
  o->q_regular_P = 6;
  o->q_singular_P = 4;
  o->near_cutoff_P = INFINITY;
  o->tol = 1e-5;
  o->restart = 200;
  o->maxit = 1000;
  o->refine = 3;
  o->rhs_mode = 0;
  o->matrix_free = 0;
  o->aca_nu_P = 0.0;
  o->discretisation = 0;
}

}  // namespace

// A problem: the assembled A and P blocks, the Gram matrices and the spaces of
// one (mesh, k, material, options), resident on the device between solves.
struct cal_problem {
  int device = 0;
  Pmchwt P;
  double t_setup = 0, t_assemble_A = 0, t_assemble_P = 0;  // seconds, at creation
  int64_t bytes_A = 0, bytes_P = 0, bytes_G = 0;
  int64_t batch_bytes() const {
    if (!P.t1) return 0;
    const int64_t n2 = 2 * P.N;
    int64_t b = 3 * (int64_t)P.nb * n2 * 16;
    if (P.d_Bt) {
      b += 3 * (int64_t)P.NB * 2 * P.A_ext->rows * 4 + 2 * (int64_t)P.A_ext->rows * P.NB * 4;
    }
    const int64_t csz = P.o.precision == CAL_FP64 ? 16 : 8, rsz = csz / 2;
    if (P.o.precond != CAL_PRECOND_NONE) b += 2 * (P.gnnz * rsz + 10 * (int64_t)P.nb * P.N * csz);
    return b;
  }
};

// =============================================================================
// C ABI
// =============================================================================
extern "C" {

const char* cal_last_error(void) { return cal::last_error(); }

int cal_init(cal_ctx** out, int device) {
  if (!out) return fail(CAL_EINVAL, "cal_init: out is NULL");
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    return fail(CAL_ECUDA, "cal_init: no CUDA device available");
  }
  if (device < 0 || device >= n) return fail(CAL_EINVAL, "cal_init: device %d out of range", device);
  CAL_TRY_CUDA(cudaSetDevice(device));
  auto* c = new cal_ctx;
  c->impl.device = device;
  if (cudaStreamCreateWithFlags(&c->impl.stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return fail(CAL_ECUDA, "cal_init: cannot create stream");
  }
  cudaDeviceGetAttribute(&c->impl.n_sm, cudaDevAttrMultiProcessorCount, device);
  if (cudaMallocHost((void**)&c->impl.pinned, 4096 * sizeof(double)) != cudaSuccess) {
    cudaStreamDestroy(c->impl.stream);
    delete c;
    return fail(CAL_ENOMEM, "cal_init: cannot allocate pinned scratch");
  }
  // keep freed blocks in the stream-ordered pool: repeated solves reuse them
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  *out = c;
  return CAL_OK;
}

void cal_ctx_destroy(cal_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->impl.stream);
  cudaStreamDestroy(ctx->impl.stream);
  cudaFreeHost(ctx->impl.pinned);
  delete ctx;
}

void* cal_ctx_stream(cal_ctx* ctx) { return ctx ? (void*)ctx->impl.stream : nullptr; }

int cal_mesh_create(cal_ctx* ctx, const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                    const int32_t* domain, cal_mesh** out) {
  if (!ctx || !out) return fail(CAL_EINVAL, "cal_mesh_create: NULL argument");
  auto* m = new cal_mesh;
  m->impl.ctx = &ctx->impl;
  int rc = build_mesh(m->impl, verts, nv, tris, nt, domain);
  if (rc) { delete m; return rc; }
  *out = m;
  return CAL_OK;
}

void cal_mesh_destroy(cal_mesh* mesh) { delete mesh; }

int cal_mesh_get_info(const cal_mesh* mesh, cal_mesh_info* info) {
  if (!mesh || !info) return fail(CAL_EINVAL, "cal_mesh_get_info: NULL argument");
  const Mesh& m = mesh->impl;
  info->n_vertices = m.nv;
  info->n_triangles = m.nt;
  info->n_edges = m.ne;
  info->n_scatterers = m.M;
  info->h = m.h;
  info->max_valence = m.max_valence;
  return CAL_OK;
}

int cal_space_create(cal_mesh* mesh, int kind, cal_space** out) {
  if (!mesh || !out) return fail(CAL_EINVAL, "cal_space_create: NULL argument");
  if (kind != CAL_RWG && kind != CAL_BC) return fail(CAL_EINVAL, "cal_space_create: kind must be CAL_RWG or CAL_BC");
  CAL_TRY_CUDA(cudaSetDevice(mesh->impl.ctx->device));
  auto* s = new cal_space;
  int rc = kind == CAL_RWG ? build_rwg(s->impl, mesh->impl) : build_bc(s->impl, mesh->impl);
  if (!rc) rc = upload_space(s->impl, mesh->impl.ctx->stream);
  if (rc) { delete s; return rc; }
  *out = s;
  return CAL_OK;
}

void cal_space_destroy(cal_space* space) { delete space; }  // every call that reads it is synchronous

int cal_assemble(cal_ctx* ctx, int op_mask, double k_re, double k_im, cal_space* test,
                 cal_space* trial, int scatterer, double near_cutoff, int q_regular, int q_singular,
                 int precision, cal_op** out) {
  if (!ctx || !test || !trial || !out) return fail(CAL_EINVAL, "cal_assemble: NULL argument");
  if (test != trial) return fail(CAL_EINVAL, "cal_assemble: test and trial must be the same space");
  CAL_TRY_CUDA(cudaSetDevice(ctx->impl.device));
  std::unique_ptr<Op> op;
  int rc = assemble_block(ctx->impl, op_mask & 3, k_re, k_im, test->impl, scatterer, near_cutoff,
                          q_regular, q_singular, precision, op);
  if (rc) return rc;
  CAL_TRY_CUDA(cudaStreamSynchronize(ctx->impl.stream));
  auto* o = new cal_op;
  o->impl = std::move(*op);  // a member-wise copy: the source gives up every device pointer
  op->d_S = op->d_C = nullptr;
  op->d_rowptr = nullptr;
  op->d_col = nullptr;
  op->hmat = nullptr;
  *out = o;
  return CAL_OK;
}

void cal_op_destroy(cal_op* op) {
  if (!op) return;
  // a matvec on a caller stream may still read the operator: wait for the device
  cudaDeviceSynchronize();
  delete op;
}

int cal_op_get_info(const cal_op* op, cal_op_info* info) {
  if (!op || !info) return fail(CAL_EINVAL, "cal_op_get_info: NULL argument");
  info->rows = op->impl.rows;
  info->cols = op->impl.cols;
  info->nnz = op->impl.nnz;
  info->format = op->impl.format;
  info->precision = op->impl.precision;
  info->op_mask = op->impl.op_mask;
  info->row_offset = (int32_t)op->impl.row_offset;
  return CAL_OK;
}

int cal_op_export(const cal_op* op, int which, void* dst, int64_t* row_ptr, int64_t* col_idx) {
  if (!op || !dst) return fail(CAL_EINVAL, "cal_op_export: NULL argument");
  const Op& o = op->impl;
  if (o.hmat) {
    const int q = which == CAL_OP_S ? 0 : (which == CAL_OP_C ? 1 : -1);
    if (q < 0 || !o.hmat->d_near[q]) return fail(CAL_EINVAL, "cal_op_export: operator %d was not assembled", which);
    const size_t bytes = (size_t)o.rows * o.cols * (o.precision == CAL_FP32 ? 8 : 16);
    cudaStream_t st = o.ctx->stream;
    void* tmp = nullptr;
    CAL_TRY_CUDA(dalloc(&tmp, bytes, st));
    int rc = hmat_expand(*o.hmat, q, tmp, st);
    if (!rc && cudaMemcpyAsync(dst, tmp, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               st) != cudaSuccess)
      rc = fail(CAL_ECUDA, "cal_op_export: copy failed");
    dfree(tmp, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = fail(CAL_ECUDA, "cal_op_export: stream failed");
    return rc;
  }
  const void* src = which == CAL_OP_S ? o.d_S : (which == CAL_OP_C ? o.d_C : nullptr);
  if (!src) return fail(CAL_EINVAL, "cal_op_export: operator %d was not assembled", which);
  const size_t bytes = (size_t)o.nnz * (o.precision == CAL_FP32 ? 8 : 16);
  CAL_TRY_CUDA(cudaMemcpy(dst, src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  if (o.format == CAL_CSR) {
    if (row_ptr) std::copy(o.h_rowptr.begin(), o.h_rowptr.end(), row_ptr);
    if (col_idx)
      for (size_t q = 0; q < o.h_col.size(); ++q) col_idx[q] = o.h_col[q];
  }
  return CAL_OK;
}

int cal_matvec(const cal_op* op, int which, const void* x, void* y, int64_t nrhs, void* stream) {
  if (!op || !x || !y || nrhs < 1) return fail(CAL_EINVAL, "cal_matvec: bad argument");
  const Op& o = op->impl;
  if (o.hmat) {
    const int q = which == CAL_OP_S ? 0 : (which == CAL_OP_C ? 1 : -1);
    if (q < 0 || !o.hmat->d_near[q]) return fail(CAL_EINVAL, "cal_matvec: operator %d was not assembled", which);
    if (!is_device_ptr(x) || !is_device_ptr(y)) return fail(CAL_EINVAL, "cal_matvec: x and y must be device pointers");
    cudaStream_t st = stream ? (cudaStream_t)stream : o.ctx->stream;
    const size_t vsz = o.precision == CAL_FP64 ? sizeof(double2) : sizeof(float2);
    void* junk = nullptr;  // the second half of the pair form, discarded
    CAL_TRY_CUDA(dalloc(&junk, o.rows * vsz, st));
    int rc = CAL_OK;
    for (int64_t v = 0; v < nrhs && !rc; ++v) {
      const char* xv = (const char*)x + v * o.cols * vsz;
      char* yv = (char*)y + v * o.rows * vsz;
      CAL_TRY_CUDA(cudaMemsetAsync(yv, 0, o.rows * vsz, st));
      // S: y1 += 1 * S x2 (x2 = x); C: y1 += C x1 (x1 = x)
      rc = hmat_apply_halves(*o.hmat, q == 0, q == 1, o.precision, xv, xv, yv, junk, 1.0, 0.0, 0.0, 0.0, st);
    }
    dfree(junk, st);
    return rc;
  }
  const void* X = which == CAL_OP_S ? o.d_S : (which == CAL_OP_C ? o.d_C : nullptr);
  if (!X) return fail(CAL_EINVAL, "cal_matvec: operator %d was not assembled", which);
  if (!is_device_ptr(x) || !is_device_ptr(y)) return fail(CAL_EINVAL, "cal_matvec: x and y must be device pointers");
  cudaStream_t st = stream ? (cudaStream_t)stream : o.ctx->stream;
  // several vectors on a float32 dense operator: the tensor-core 3xTF32 product
  if (o.precision == CAL_FP32 && o.format == CAL_DENSE && nrhs >= 4 && (nrhs + 1) / 2 * 4 <= 256 && o.cols % 2 == 0)
  {
    return multi_matvec_tc((const float2*)X, o.rows, o.cols, (const float2*)x, (float2*)y, (int)nrhs, o.ctx->n_sm, st);
  }
  return single_apply(o, X, x, y, nrhs, st);
}

int cal_op_compress(cal_ctx* ctx, const cal_op* dense, const cal_space* space, double nu, double chi,
                    cal_op** out) {
  if (!ctx || !dense || !space || !out) return fail(CAL_EINVAL, "cal_op_compress: NULL argument");
  const Op& d = dense->impl;
  if (d.format != CAL_DENSE || d.rows != d.cols) return fail(CAL_EINVAL, "cal_op_compress: needs a dense square operator");
  if (d.row_offset + d.rows > space->impl.nbasis)
    return fail(CAL_EINVAL, "cal_op_compress: the operator's rows lie outside the space");
  if (!(nu > 0) || !(chi >= 0)) return fail(CAL_EINVAL, "cal_op_compress: nu must be > 0 and chi >= 0");
  CAL_TRY_CUDA(cudaSetDevice(ctx->impl.device));
  auto* o = new cal_op;
  int rc = hmat_compress(d, space->impl, nu, chi, 512, o->impl, ctx->impl.stream);
  if (!rc && cudaStreamSynchronize(ctx->impl.stream) != cudaSuccess) rc = fail(CAL_ECUDA, "cal_op_compress: stream failed");
  if (rc) {
    delete o;
    return rc;
  }
  *out = o;
  return CAL_OK;
}

int cal_gram_export(cal_space* rwg, cal_space* bc, double* dst_host) {
  if (!rwg || !bc || !dst_host || rwg->impl.kind != CAL_RWG || bc->impl.kind != CAL_BC ||
      rwg->impl.mesh != bc->impl.mesh)
    return fail(CAL_EINVAL, "cal_gram_export: need an RWG and a BC space of the same mesh");
  const Space& B = bc->impl;
  const int64_t n = B.nbasis;
  std::vector<int64_t> rp, rpT;
  std::vector<int> col, colT;
  gram_pattern(B, rp, col);
  // transpose pattern
  rpT.assign(n + 1, 0);
  for (int c : col) rpT[c + 1]++;
  for (int64_t i = 0; i < n; ++i) rpT[i + 1] += rpT[i];
  colT.resize(col.size());
  {
    std::vector<int64_t> fill(rpT.begin(), rpT.end() - 1);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t q = rp[i]; q < rp[i + 1]; ++q) colT[fill[col[q]]++] = (int)i;
  }
  int64_t *drp, *drpT;
  int *dc, *dcT;
  double *dv, *dvT;
  const size_t nnz = col.size();
  CAL_TRY_CUDA(cudaMalloc((void**)&drp, (n + 1) * sizeof(int64_t)));
  CAL_TRY_CUDA(cudaMalloc((void**)&drpT, (n + 1) * sizeof(int64_t)));
  CAL_TRY_CUDA(cudaMalloc((void**)&dc, nnz * sizeof(int)));
  CAL_TRY_CUDA(cudaMalloc((void**)&dcT, nnz * sizeof(int)));
  CAL_TRY_CUDA(cudaMalloc((void**)&dv, nnz * sizeof(double)));
  CAL_TRY_CUDA(cudaMalloc((void**)&dvT, nnz * sizeof(double)));
  CAL_TRY_CUDA(cudaMemcpy(drp, rp.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
  CAL_TRY_CUDA(cudaMemcpy(drpT, rpT.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
  CAL_TRY_CUDA(cudaMemcpy(dc, col.data(), nnz * sizeof(int), cudaMemcpyHostToDevice));
  CAL_TRY_CUDA(cudaMemcpy(dcT, colT.data(), nnz * sizeof(int), cudaMemcpyHostToDevice));
  CAL_TRY_CUDA(cudaMemset(dv, 0, nnz * sizeof(double)));
  CAL_TRY_CUDA(cudaMemset(dvT, 0, nnz * sizeof(double)));
  int rc = launch_gram(rwg->impl, B, drp, dc, drpT, dcT, dv, dvT, 0);
  std::vector<double> v(nnz);
  if (!rc) {
    CAL_TRY_CUDA(cudaDeviceSynchronize());
    CAL_TRY_CUDA(cudaMemcpy(v.data(), dv, nnz * sizeof(double), cudaMemcpyDeviceToHost));
    std::fill(dst_host, dst_host + n * n, 0.0);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t q = rp[i]; q < rp[i + 1]; ++q) dst_host[i * n + col[q]] = v[q];
  }
  cudaFree(drp); cudaFree(drpT); cudaFree(dc); cudaFree(dcT); cudaFree(dv); cudaFree(dvT);
  return rc;
}

void cal_solve_opts_default(cal_solve_opts* opts) {
  if (opts) opts_default(opts);
}

int cal_problem_create(cal_ctx* ctx, cal_mesh* mesh, double k_ext, const double* eps_r, const double* mu_r,
                       const cal_solve_opts* opts, cal_problem** out) {
  if (!ctx || !mesh || !eps_r || !out) return fail(CAL_EINVAL, "cal_problem_create: bad argument");
  if (!(k_ext > 0) || !std::isfinite(k_ext)) return fail(CAL_EINVAL, "cal_problem_create: k_ext must be positive");
  CAL_TRY_CUDA(cudaSetDevice(ctx->impl.device));
  const double t_start = now();
  auto prob = std::make_unique<cal_problem>();
  prob->device = ctx->impl.device;
  Pmchwt& P = prob->P;
  P.ctx = &ctx->impl;
  P.mesh = &mesh->impl;
  P.M = (int)mesh->impl.M;
  P.N = mesh->impl.ne;
  P.k_e = k_ext;
  if (opts) P.o = *opts; else opts_default(&P.o);
  const cal_solve_opts& o = P.o;
  if (o.precision != CAL_FP32 && o.precision != CAL_FP64 && o.precision != CAL_FP32_ALL)
    return fail(CAL_EINVAL, "solve: bad precision");
  if (o.precond < CAL_PRECOND_NONE || o.precond > CAL_PRECOND_SI) return fail(CAL_EINVAL, "solve: bad preconditioner");
  if (!(o.tol > 0) || o.restart < 1 || o.maxit < 1) return fail(CAL_EINVAL, "solve: bad tolerance/restart/maxit");
  if (!(o.aca_nu_P >= 0) || !std::isfinite(o.aca_nu_P)) return fail(CAL_EINVAL, "solve: aca_nu_P must be >= 0");
  if (o.discretisation != 0 && o.discretisation != 1) return fail(CAL_EINVAL, "solve: discretisation must be 0 or 1");
  if (o.discretisation == 1 && (o.precision != CAL_FP64 || o.precond != CAL_PRECOND_D || o.matrix_free ||
                                o.rhs_mode != 0 || o.aca_nu_P > 0))
    return fail(CAL_EINVAL,
                "solve: the mixed discretisation needs CAL_FP64, CAL_PRECOND_D, stored A, rhs_mode 0 and no ACA");
  if (o.rhs_mode != 0 && o.rhs_mode != 1)
    return fail(CAL_EINVAL, "solve: rhs_mode must be 0 (total traces) or 1 (the paper's scattered traces)");
  for (int m = 0; m < P.M; ++m) {
    std::complex<double> e(eps_r[2 * m], eps_r[2 * m + 1]);
    std::complex<double> u = mu_r ? std::complex<double>(mu_r[2 * m], mu_r[2 * m + 1]) : 1.0;
    if (!std::isfinite(e.real()) || !std::isfinite(e.imag()) || !std::isfinite(u.real()) ||
        !std::isfinite(u.imag()) || std::abs(e) == 0.0 || std::abs(u) == 0.0)
      return fail(CAL_EINVAL, "solve: bad eps_r/mu_r for scatterer %d", m);
    P.k_m.push_back(interior_k(k_ext, e, u));
    P.mu_m.push_back(u);
  }
  cudaStream_t st = ctx->impl.stream;
  int rc;
  // spaces: the BC space is built by a host thread while this thread builds
  // the RWG space and enqueues A's assembly (the launches are asynchronous);
  // both only read the mesh
  const bool need_bc = o.precond != CAL_PRECOND_NONE;
  struct BcBuild {
    std::thread th;
    int rc = CAL_OK;
    std::string msg;
    double seconds = 0.0;
    std::mutex mu;
    std::condition_variable cv;
    bool built = false;  // the space is built (its work units may still be in progress)
    ~BcBuild() { if (th.joinable()) th.join(); }
    void set_built() {
      {
        std::lock_guard<std::mutex> lk(mu);
        built = true;
      }
      cv.notify_all();
    }
    int wait_built() {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [this] { return built; });
      return rc ? fail(rc, "%s", msg.c_str()) : CAL_OK;
    }
    int join() {
      if (th.joinable()) th.join();
      return rc ? fail(rc, "%s", msg.c_str()) : CAL_OK;
    }
  } bcb;
  if (need_bc) {
    P.bc = std::make_shared<Space>();
    Space* bcs = P.bc.get();
    Mesh* mh = &mesh->impl;
    // P's blocks (one per scatterer, exterior and interior alike) need the work
    // units of the BC regular-pair kernels: once the space is built, the same
    // thread builds them, on a stream of its own, while the device runs A and
    // the touching pairs of P that this thread enqueues meanwhile
    const bool prebuild = o.discretisation == 0;
    const double chi_units =
        (o.aca_nu_P > 0 || std::isinf(o.near_cutoff_P)) ? INFINITY : o.near_cutoff_P * mesh->impl.h;
    const int prec_units = o.precision == CAL_FP64 ? CAL_FP64 : CAL_FP32;
    const int nreg_units = o.q_regular_P, dev = ctx->impl.device, M = P.M;
    bcb.th = std::thread([&bcb, bcs, mh, prebuild, chi_units, prec_units, nreg_units, dev, M]() {
      const double tb = now();
      bcb.rc = build_bc(*bcs, *mh);
      if (bcb.rc) bcb.msg = last_error();
      bcb.set_built();
      if (!bcb.rc && prebuild && set_quadrature_tables(nreg_units, 1) == CAL_OK) {
        // a failure here only leaves the lists to the assembly itself
        cudaStream_t ps = nullptr;
        if (cudaSetDevice(dev) == cudaSuccess && cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) == cudaSuccess) {
          for (int m = 0; m < M; ++m)
            if (cached_unit_lists(*bcs, m, chi_units, nreg_units, prec_units, ps, nullptr) != CAL_OK) break;
          cudaStreamDestroy(ps);
        }
        cudaGetLastError();
      }
      bcb.seconds = now() - tb;
    });
  }
  P.rwg = std::make_shared<Space>();
  if ((rc = build_rwg(*P.rwg, mesh->impl)) || (rc = upload_space(*P.rwg, st))) return rc;
  double t_setup_host = now() - t_start;
  // device phase times from events on the stream (the host does not wait in between)
  struct Ev {
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
    ~Ev() { for (auto x : e) if (x) cudaEventDestroy(x); }
  } ev;
  for (auto& x : ev.e) CAL_TRY_CUDA(cudaEventCreate(&x));
  CAL_TRY_CUDA(cudaEventRecord(ev.e[0], st));
  // A: S, C at k_e on the union; S, C at k_m on each scatterer
  const int aprec = o.precision;  // assembly mode (CAL_FP32_ALL: float32 singular pairs)
  const int prec = aprec == CAL_FP64 ? CAL_FP64 : CAL_FP32;  // storage and vector precision
  P.o.precision = prec;
  P.A_int.resize(P.M);
  if (o.matrix_free) {
    // only the touching-pair entries are stored; the rest is recomputed per application
    if (o.q_regular_A != 6 && o.q_regular_A != 1 && o.q_regular_A != 0)
      return fail(CAL_EINVAL, "q_regular must be 6, 1 or 0 (classes)");
    if ((rc = assemble_singular_block(ctx->impl, k_ext, 0.0, *P.rwg, -1, o.q_singular_A, aprec, P.A_ext)))
      return rc;
    for (int m = 0; m < P.M; ++m)
      if ((rc = assemble_singular_block(ctx->impl, P.k_m[m].real(), P.k_m[m].imag(), *P.rwg, m, o.q_singular_A,
                                        aprec, P.A_int[m])))
        return rc;
  } else {
    P.mixed = o.discretisation == 1;
    const int wantA = P.mixed ? 1 : 3;  // the mixed form takes C between RWG and BC instead
    if ((rc = assemble_block(ctx->impl, wantA, k_ext, 0.0, *P.rwg, -1, INFINITY, o.q_regular_A, o.q_singular_A,
                             aprec, P.A_ext)))
      return rc;
    for (int m = 0; m < P.M; ++m)
      if ((rc = assemble_block(ctx->impl, wantA, P.k_m[m].real(), P.k_m[m].imag(), *P.rwg, m, INFINITY,
                               o.q_regular_A, o.q_singular_A, aprec, P.A_int[m])))
        return rc;
  }
  if ((rc = P.build_combo_A(st))) return rc;
  CAL_TRY_CUDA(cudaEventRecord(ev.e[1], st));
  if (need_bc) {
    const double tb = now();
    if ((rc = bcb.wait_built()) || (rc = upload_space(*P.bc, st))) return rc;
    t_setup_host += now() - tb;  // the part of the BC build A's enqueue did not hide
  }
  CAL_TRY_CUDA(cudaEventRecord(ev.e[2], st));
  int64_t bytes_A = 0, bytes_P = 0, bytes_G = 0;
  const size_t esz = prec == CAL_FP32 ? 8 : 16;
  for (auto* a : {P.A_ext.get()}) bytes_A += a->nnz * esz * 2;
  for (auto& a : P.A_int) bytes_A += a->nnz * esz * 2;
  // P on BC: block diagonal per scatterer
  if (need_bc) {
    const int pc = o.precond;
    const bool ext = pc == CAL_PRECOND_D || pc == CAL_PRECOND_DE || pc == CAL_PRECOND_SE;
    const bool in = pc == CAL_PRECOND_D || pc == CAL_PRECOND_DI || pc == CAL_PRECOND_SI;
    const int want = (pc == CAL_PRECOND_SE || pc == CAL_PRECOND_SI) ? 1 : 3;
    const double chi_abs = std::isinf(o.near_cutoff_P) ? INFINITY : o.near_cutoff_P * mesh->impl.h;
    const bool aca = o.aca_nu_P > 0;
    // with ACA the cutoff acts on admissible H-matrix leaves, not on entries
    const double chi = aca ? INFINITY : chi_abs;
    P.P_ext.resize(P.M);
    P.P_int.resize(P.M);
    auto to_hmat = [&](std::unique_ptr<Op>& op) -> int {
      if (!aca || !op) return CAL_OK;
      auto h = std::make_unique<Op>();
      int r = hmat_compress(*op, *P.bc, o.aca_nu_P, chi_abs, 512, *h, st);
      if (r) return r;
      op = std::move(h);  // the dense block is released in stream order
      return CAL_OK;
    };
    if (P.mixed) {
      // S on BC (union and per scatterer) and C between RWG and BC, A's rules
      if ((rc = bcb.join()) || (rc = P.build_rwgb(st))) return rc;
      if ((rc = assemble_block(ctx->impl, 1, k_ext, 0.0, *P.bc, -1, INFINITY, o.q_regular_A, o.q_singular_A,
                               CAL_FP64, P.Sb_ext)))
        return rc;
      const size_t b2 = (size_t)P.N * P.N * sizeof(double2);
      CAL_TRY_CUDA(dalloc((void**)&P.Crb_ext, b2, st));
      CAL_TRY_CUDA(dalloc((void**)&P.Cbr_ext, b2, st));
      CAL_TRY_CUDA(cudaMemsetAsync(P.Crb_ext, 0, b2, st));
      CAL_TRY_CUDA(cudaMemsetAsync(P.Cbr_ext, 0, b2, st));
      if ((rc = launch_cross_c(*P.bc, P.d_redge, P.d_rsw, -1, k_ext, 0.0, o.q_regular_A, o.q_singular_A, 0, P.N,
                               (double*)P.Crb_ext, (double*)P.Cbr_ext, st)))
        return rc;
      bytes_P += (int64_t)(b2 * 2 + P.Sb_ext->nnz * 16);
      P.Sb_int.resize(P.M);
      P.Crb_int.assign(P.M, nullptr);
      P.Cbr_int.assign(P.M, nullptr);
      for (int m = 0; m < P.M; ++m) {
        if ((rc = assemble_block(ctx->impl, 1, P.k_m[m].real(), P.k_m[m].imag(), *P.bc, m, INFINITY, o.q_regular_A,
                                 o.q_singular_A, CAL_FP64, P.Sb_int[m])))
          return rc;
        const int64_t nm = P.Sb_int[m]->rows;
        const size_t bm = (size_t)nm * nm * sizeof(double2);
        CAL_TRY_CUDA(dalloc((void**)&P.Crb_int[m], bm, st));
        CAL_TRY_CUDA(dalloc((void**)&P.Cbr_int[m], bm, st));
        CAL_TRY_CUDA(cudaMemsetAsync(P.Crb_int[m], 0, bm, st));
        CAL_TRY_CUDA(cudaMemsetAsync(P.Cbr_int[m], 0, bm, st));
        if ((rc = launch_cross_c(*P.bc, P.d_redge, P.d_rsw, m, P.k_m[m].real(), P.k_m[m].imag(), o.q_regular_A,
                                 o.q_singular_A, P.Sb_int[m]->row_offset, nm, (double*)P.Crb_int[m],
                                 (double*)P.Cbr_int[m], st)))
          return rc;
        bytes_P += (int64_t)(bm * 2 + P.Sb_int[m]->nnz * 16);
      }
    }
    // the touching pairs of every block and the Gram matrix need the space
    // only: the device runs them while the other thread finishes the work units
    auto assemble_P = [&](int m, int parts) -> int {
      int r = CAL_OK;
      if (ext && (r = assemble_block(ctx->impl, want, k_ext, 0.0, *P.bc, m, chi, o.q_regular_P, o.q_singular_P,
                                     aprec, P.P_ext[m], parts)))
        return r;
      if (in && (r = assemble_block(ctx->impl, want, P.k_m[m].real(), P.k_m[m].imag(), *P.bc, m, chi,
                                    o.q_regular_P, o.q_singular_P, aprec, P.P_int[m], parts)))
        return r;
      return CAL_OK;
    };
    for (int m = 0; m < P.M && !P.mixed; ++m)
      if ((rc = assemble_P(m, 1))) return rc;
    // Gram G (rows RWG, cols BC) and its transpose
    std::vector<int64_t> rp, rpT;
    std::vector<int> col, colT;
    gram_pattern(*P.bc, rp, col);
    const int64_t n = P.N;
    rpT.assign(n + 1, 0);
    for (int c : col) rpT[c + 1]++;
    for (int64_t i = 0; i < n; ++i) rpT[i + 1] += rpT[i];
    colT.resize(col.size());
    {
      std::vector<int64_t> fill(rpT.begin(), rpT.end() - 1);
      for (int64_t i = 0; i < n; ++i)
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) colT[fill[col[q]]++] = (int)i;
    }
    P.gnnz = (int64_t)col.size();
    CAL_TRY_CUDA(dalloc((void**)&P.d_grp, (n + 1) * sizeof(int64_t), st));
    CAL_TRY_CUDA(dalloc((void**)&P.d_grpT, (n + 1) * sizeof(int64_t), st));
    CAL_TRY_CUDA(dalloc((void**)&P.d_gcol, P.gnnz * sizeof(int), st));
    CAL_TRY_CUDA(dalloc((void**)&P.d_gcolT, P.gnnz * sizeof(int), st));
    CAL_TRY_CUDA(dalloc((void**)&P.d_gval, P.gnnz * sizeof(double), st));
    CAL_TRY_CUDA(dalloc((void**)&P.d_gvalT, P.gnnz * sizeof(double), st));
    CAL_TRY_CUDA(cudaMemcpyAsync(P.d_grp, rp.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CAL_TRY_CUDA(cudaMemcpyAsync(P.d_grpT, rpT.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CAL_TRY_CUDA(cudaMemcpyAsync(P.d_gcol, col.data(), P.gnnz * sizeof(int), cudaMemcpyHostToDevice, st));
    CAL_TRY_CUDA(cudaMemcpyAsync(P.d_gcolT, colT.data(), P.gnnz * sizeof(int), cudaMemcpyHostToDevice, st));
    CAL_TRY_CUDA(cudaMemsetAsync(P.d_gval, 0, P.gnnz * sizeof(double), st));
    CAL_TRY_CUDA(cudaMemsetAsync(P.d_gvalT, 0, P.gnnz * sizeof(double), st));
    if ((rc = launch_gram(*P.rwg, *P.bc, P.d_grp, P.d_gcol, P.d_grpT, P.d_gcolT, P.d_gval, P.d_gvalT, st)))
      return rc;
    bytes_G = 2 * ((n + 1) * 8 + P.gnnz * (4 + 8));
    if ((rc = bcb.join())) return rc;
    for (int m = 0; m < P.M && !P.mixed; ++m) {
      if ((rc = assemble_P(m, 2)) || (rc = to_hmat(P.P_ext[m])) || (rc = to_hmat(P.P_int[m]))) return rc;
      for (auto* op : {P.P_ext[m].get(), P.P_int[m].get()})
        if (op)
          bytes_P += op->hmat ? op->hmat->stored * (int64_t)esz
                              : op->nnz * esz * ((want & 2) ? 2 : 1) +
                                    (op->format == CAL_CSR ? (int64_t)(op->h_rowptr.size() * 8 + op->h_col.size() * 4)
                                                           : 0);
    }
  }
  if ((rc = P.build_combo_P(st))) return rc;
  if (P.cA.C) bytes_A += 3 * P.cA.rows * P.cA.rows * 8;
  for (const auto& c : P.cP) bytes_P += 3 * c.rows * c.rows * 8;
  CAL_TRY_CUDA(cudaEventRecord(ev.e[3], st));
  CAL_TRY_CUDA(cudaStreamSynchronize(st));
  float ms_A = 0.0f, ms_P = 0.0f;
  cudaEventElapsedTime(&ms_A, ev.e[0], ev.e[1]);
  cudaEventElapsedTime(&ms_P, ev.e[2], ev.e[3]);
  prob->t_setup = t_setup_host;       // host: spaces (the BC space overlaps A's assembly)
  prob->t_assemble_A = 1e-3 * ms_A;   // device time of A's launches
  prob->t_assemble_P = 1e-3 * ms_P;   // device time of P's launches and the Gram matrix
  prob->bytes_A = bytes_A;
  prob->bytes_P = bytes_P;
  prob->bytes_G = bytes_G;
  P.mesh = nullptr;  // the mesh may go: the solves need only the spaces and blocks
  P.ctx = nullptr;
  *out = prob.release();
  return CAL_OK;
}

int cal_problem_apply(cal_ctx* ctx, cal_problem* prob, const double* x, double* y, int64_t nrhs) {
  if (!ctx || !prob || !x || !y || nrhs < 1) return fail(CAL_EINVAL, "cal_problem_apply: bad argument");
  if (ctx->impl.device != prob->device)
    return fail(CAL_EINVAL, "cal_problem_apply: the problem lives on device %d", prob->device);
  CAL_TRY_CUDA(cudaSetDevice(ctx->impl.device));
  Pmchwt& P = prob->P;
  struct Bind {
    Pmchwt& P;
    ~Bind() { P.ctx = nullptr; }
  } bind{P};
  P.ctx = &ctx->impl;
  cudaStream_t st = ctx->impl.stream;
  const size_t bytes = (size_t)nrhs * 2 * P.N * sizeof(double2);
  void *dx = nullptr, *dy = nullptr;
  CAL_TRY_CUDA(dalloc(&dx, bytes, st));
  if (dalloc(&dy, bytes, st) != cudaSuccess) {
    dfree(dx, st);
    return fail(CAL_ENOMEM, "cal_problem_apply: device allocation failed");
  }
  int rc = CAL_OK;
  if (cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = fail(CAL_ECUDA, "copy failed");
  if (!rc && P.mixed) {
    for (int64_t q = 0; q < nrhs && !rc; ++q)
      rc = P.mixed_apply((const double2*)dx + q * 2 * P.N, (double2*)dy + q * 2 * P.N, false);
  } else if (!rc) {
    rc = P.apply_A(dx, dy, CAL_FP64, (int)nrhs);
  }
  if (!rc && cudaMemcpyAsync(y, dy, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = fail(CAL_ECUDA, "copy failed");
  dfree(dx, st);
  dfree(dy, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = fail(CAL_ECUDA, "cal_problem_apply: stream failed");
  return rc;
}

void cal_problem_destroy(cal_problem* prob) { delete prob; }  // its solves are synchronous

int cal_problem_get_info(const cal_problem* prob, cal_problem_info* info) {
  if (!prob || !info) return fail(CAL_EINVAL, "cal_problem_get_info: NULL argument");
  const Pmchwt& P = prob->P;
  info->n_unknowns = 2 * P.N;
  info->n_scatterers = P.M;
  info->precision = P.o.precision;
  info->precond = P.o.precond;
  info->bytes_A = prob->bytes_A;
  info->bytes_P = prob->bytes_P;
  info->bytes_G = prob->bytes_G;
  info->bytes_batch = prob->batch_bytes();
  info->batch_width = P.t1 ? P.nb : 0;
  info->t_setup = prob->t_setup;
  info->t_assemble_A = prob->t_assemble_A;
  info->t_assemble_P = prob->t_assemble_P;
  return CAL_OK;
}

int cal_problem_solve(cal_ctx* ctx, cal_problem* prob, const double* inc, int64_t nrhs,
                      const cal_solve_opts* solver, cal_solution** out) {
  if (!ctx || !prob || !inc || nrhs < 1 || !out) return fail(CAL_EINVAL, "cal_problem_solve: bad argument");
  if (solver && (!(solver->tol > 0) || solver->restart < 1 || solver->maxit < 1 || solver->refine < 0))
    return fail(CAL_EINVAL, "cal_problem_solve: bad tolerance/restart/maxit/refine");
  if (solver && solver->rhs_mode != 0 && solver->rhs_mode != 1)
    return fail(CAL_EINVAL, "solve: rhs_mode must be 0 (total traces) or 1 (the paper's scattered traces)");
  if (ctx->impl.device != prob->device)
    return fail(CAL_EINVAL, "cal_problem_solve: the problem lives on device %d", prob->device);
  for (int64_t q = 0; q < 6 * nrhs; ++q)
    if (!std::isfinite(inc[q])) return fail(CAL_EINVAL, "solve: non-finite incident field");
  CAL_TRY_CUDA(cudaSetDevice(ctx->impl.device));
  Pmchwt& P = prob->P;
  // the problem runs on this call's context, with this call's solver
  // settings, until it returns
  struct Bind {
    Pmchwt& P;
    cal_solve_opts saved;
    ~Bind() {
      P.ctx = nullptr;
      P.o = saved;
    }
  } bind{P, P.o};
  P.ctx = &ctx->impl;
  if (solver) {
    P.o.tol = solver->tol;
    P.o.restart = solver->restart;
    P.o.maxit = solver->maxit;
    P.o.refine = solver->refine;
    P.o.rhs_mode = solver->rhs_mode;
  }
  const cal_solve_opts& o = P.o;
  const int prec = o.precision;
  cudaStream_t st = ctx->impl.stream;
  const double t0 = now();
  int rc;
  const int nbatch = P.mixed ? 1 : (int)std::min<int64_t>(nrhs, 32);
  if (P.mixed && P.o.rhs_mode != 0) return fail(CAL_EINVAL, "solve: the mixed discretisation takes rhs_mode 0");
  if ((rc = P.setup_batch(nbatch))) return rc;
  if (P.d_gemm_err) CAL_TRY_CUDA(cudaMemsetAsync(P.d_gemm_err, 0, sizeof(int), st));
  // right-hand sides and solves
  auto sol = std::make_unique<cal_solution>();
  sol->ctx = &ctx->impl;
  sol->nrhs = nrhs;
  sol->ne = P.N;
  sol->k_e = P.k_e;
  sol->precision = P.o.precision == CAL_FP64 ? CAL_FP64 : CAL_FP32;
  sol->k_m = P.k_m;
  sol->mu_m = P.mu_m;
  sol->inc.assign(inc, inc + 6 * nrhs);
  sol->rhs_mode = o.rhs_mode;
  const int64_t n2 = 2 * P.N;
  double* d_inc;
  double2 *d_b, *d_rhs, *d_r;
  CAL_TRY_CUDA(dalloc((void**)&d_inc, 6 * nrhs * sizeof(double), st));
  CAL_TRY_CUDA(dalloc((void**)&d_b, nrhs * n2 * sizeof(double2), st));
  CAL_TRY_CUDA(dalloc((void**)&d_rhs, nbatch * n2 * sizeof(double2), st));
  CAL_TRY_CUDA(dalloc((void**)&d_r, nbatch * n2 * sizeof(double2), st));
  CAL_TRY_CUDA(dalloc((void**)&sol->d_x, nrhs * n2 * sizeof(double2), st));
  CAL_TRY_CUDA(cudaMemsetAsync(sol->d_x, 0, nrhs * n2 * sizeof(double2), st));
  CAL_TRY_CUDA(cudaMemcpyAsync(d_inc, inc, 6 * nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
  struct Guard {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    ~Guard() { dfree(p, s); }
  };
  Guard g1{d_b, st}, g2{d_rhs, st}, g3{d_r, st}, g4{d_inc, st};
  if ((rc = launch_rhs(*P.rwg, d_inc, (int)nrhs, P.k_e, 1.0, d_b, st))) return rc;
  if (P.mixed) {
    // rows tested with RWG take the second trace component, rows tested with BC
    // the first: b = (b_RWG second half, b_BC first half)
    double2* d_bb = nullptr;
    CAL_TRY_CUDA(dalloc((void**)&d_bb, nrhs * n2 * sizeof(double2), st));
    Guard gbb{d_bb, st};
    if ((rc = launch_rhs(*P.bc, d_inc, (int)nrhs, P.k_e, 1.0, d_bb, st))) return rc;
    for (int64_t q = 0; q < nrhs; ++q) {
      CAL_TRY_CUDA(cudaMemcpyAsync(d_b + q * n2, d_b + q * n2 + P.N, P.N * sizeof(double2), cudaMemcpyDeviceToDevice,
                                   st));
      CAL_TRY_CUDA(cudaMemcpyAsync(d_b + q * n2 + P.N, d_bb + q * n2, P.N * sizeof(double2), cudaMemcpyDeviceToDevice,
                                   st));
    }
    CAL_TRY_CUDA(cudaStreamSynchronize(st));
  }
  if (o.rhs_mode == 1) {
    CAL_TRY_CUDA(dalloc((void**)&sol->d_cinc, nrhs * n2 * sizeof(double2), st));
    if ((rc = P.scattered_rhs(d_inc, nrhs, d_b, sol->d_cinc))) return rc;
  }
  P.matvecs = 0;
  int total_it = 0;
  double worst_res = 0.0;
  bool all_conv = true;
  for (int64_t q0 = 0; q0 < nrhs; q0 += nbatch) {
    // the last batch may be short: pad it with zero right-hand sides
    const int nq = (int)std::min<int64_t>(nbatch, nrhs - q0);
    double2* b = d_b + q0 * n2;
    std::vector<double2*> xs;
    double2* x = nullptr;
    Guard gx{nullptr, st}, gbb{nullptr, st};
    if (nq == nbatch) {
      x = sol->d_x + q0 * n2;
    } else {
      double2 *xb, *bb;
      CAL_TRY_CUDA(dalloc((void**)&xb, nbatch * n2 * sizeof(double2), st));
      CAL_TRY_CUDA(dalloc((void**)&bb, nbatch * n2 * sizeof(double2), st));
      gx.p = xb;
      gbb.p = bb;
      CAL_TRY_CUDA(cudaMemsetAsync(xb, 0, nbatch * n2 * sizeof(double2), st));
      CAL_TRY_CUDA(cudaMemsetAsync(bb, 0, nbatch * n2 * sizeof(double2), st));
      CAL_TRY_CUDA(cudaMemcpyAsync(bb, b, nq * n2 * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      x = xb;
      b = bb;
    }
    std::vector<int> its(nbatch, 0);
    std::vector<double> res(nbatch, 0.0);
    if (prec == CAL_FP64 || o.refine <= 0) {
      // d = GMRES(B, M^-1 b)
      if ((rc = P.apply_precond(b, d_rhs, nbatch))) return rc;
      std::vector<double> tol(nbatch, o.tol);
      if ((rc = P.gmres(d_rhs, x, tol, its, res, o.maxit))) return rc;
    } else {
      // FP64 iterative refinement around FP32-bulk GMRES: r = b - A x in
      // float64 accumulation, correction from the preconditioned system.
      std::vector<double> r0, rn;
      std::vector<char> done(nbatch, 0);
      int budget = o.maxit;
      for (int step = 0; step <= o.refine; ++step) {
        if (step == 0) {
          CAL_TRY_CUDA(cudaMemcpyAsync(d_r, b, nbatch * n2 * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        } else {
          if ((rc = P.apply_A(x, d_r, CAL_FP64, nbatch))) return rc;  // float64 vectors, complex64 matrices
          if ((rc = vec_axpby(b, 1.0, d_r, -1.0, d_r, nbatch * n2, st))) return rc;
        }
        if ((rc = P.apply_precond(d_r, d_rhs, nbatch))) return rc;
        if ((rc = P.norms(d_rhs, rn))) return rc;
        if (step == 0) r0 = rn;
        bool all = true;
        std::vector<double> tol(nbatch, 1.0);
        for (int q = 0; q < nbatch; ++q) {
          res[q] = r0[q] > 0 ? rn[q] / r0[q] : 0.0;
          if (r0[q] == 0.0 || (step > 0 && res[q] <= o.tol)) done[q] = 1;
          // columns that are done get an unreachable-to-miss target of 1 (no iteration)
          // the float32 GMRES's own residual runs ahead of the float64 one, so
          // it aims at half the target: the float64 check then usually passes
          // at once, without a second residual pass and a correction solve
          tol[q] = done[q] ? 2.0 : std::min(0.5, std::max(0.5 * o.tol * r0[q] / rn[q], 2e-6));
          all = all && done[q];
        }
        if (all || step == o.refine || budget <= 0) break;
        std::vector<int> it_s;
        std::vector<double> res_s;
        if ((rc = P.gmres(d_rhs, x, tol, it_s, res_s, budget))) return rc;
        int mx = 0;
        for (int q = 0; q < nbatch; ++q) { its[q] += it_s[q]; mx = std::max(mx, it_s[q]); }
        budget -= mx;
        if (budget <= 0) {
          if ((rc = P.apply_A(x, d_r, CAL_FP64, nbatch)) || (rc = vec_axpby(b, 1.0, d_r, -1.0, d_r, nbatch * n2, st)) ||
              (rc = P.apply_precond(d_r, d_rhs, nbatch)) || (rc = P.norms(d_rhs, rn)))
            return rc;
          for (int q = 0; q < nbatch; ++q) res[q] = r0[q] > 0 ? rn[q] / r0[q] : 0.0;
          break;
        }
      }
    }
    if (nq != nbatch)
      CAL_TRY_CUDA(cudaMemcpyAsync(sol->d_x + q0 * n2, x, nq * n2 * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    for (int q = 0; q < nq; ++q) {
      total_it = std::max(total_it, its[q]);
      worst_res = std::max(worst_res, res[q]);
      if (!(res[q] <= o.tol)) all_conv = false;
    }
    CAL_TRY_CUDA(cudaStreamSynchronize(st));
  }
  if (P.d_gemm_err) {
    int herr = 0;
    CAL_TRY_CUDA(cudaMemcpyAsync(&herr, P.d_gemm_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CAL_TRY_CUDA(cudaStreamSynchronize(st));
    if (herr) return fail(CAL_ETIMEOUT, "tensor-core product: a bounded wait gave up");
  }
  if (P.gsA32 && (rc = P.gsA32->check(st))) return rc;
  if (P.gsP32 && (rc = P.gsP32->check(st))) return rc;
  if (P.gsA64 && (rc = P.gsA64->check(st))) return rc;
  if (P.gsP64 && (rc = P.gsP64->check(st))) return rc;
  if (P.gmA && (rc = P.gmA->check(st))) return rc;
  if (P.gmP && (rc = P.gmP->check(st))) return rc;
  CAL_TRY_CUDA(cudaStreamSynchronize(st));
  const double t_end = now();
  sol->rwg = P.rwg;
  if (P.mixed) sol->bc = P.bc;  // the second trace is expanded in BC
  cal_solve_info& info = sol->info;
  info.iterations = total_it;
  info.converged = all_conv;
  info.matvecs = P.matvecs;
  info.residual = worst_res;
  info.t_setup = prob->t_setup;
  info.t_assemble_A = prob->t_assemble_A;
  info.t_assemble_P = prob->t_assemble_P;
  info.t_solve = t_end - t0;
  info.bytes_A = prob->bytes_A;
  info.bytes_P = prob->bytes_P;
  info.n_unknowns = 2 * P.N;
  *out = sol.release();
  if (!all_conv) return fail(CAL_ENOTCONV, "GMRES reached maxit (residual %.3e > tol %.1e)", worst_res, o.tol);
  return CAL_OK;
}

int cal_pmchwt_solve(cal_ctx* ctx, cal_mesh* mesh, double k_ext, const double* eps_r,
                     const double* mu_r, const double* inc, int64_t nrhs,
                     const cal_solve_opts* opts, cal_solution** out) {
  if (!ctx || !mesh || !eps_r || !inc || nrhs < 1 || !out) return fail(CAL_EINVAL, "cal_pmchwt_solve: bad argument");
  for (int64_t q = 0; q < 6 * nrhs; ++q)
    if (!std::isfinite(inc[q])) return fail(CAL_EINVAL, "solve: non-finite incident field");
  cal_problem* prob = nullptr;
  int rc = cal_problem_create(ctx, mesh, k_ext, eps_r, mu_r, opts, &prob);
  if (rc) return rc;
  rc = cal_problem_solve(ctx, prob, inc, nrhs, nullptr, out);
  cal_problem_destroy(prob);
  return rc;
}

int cal_solution_get_info(const cal_solution* sol, cal_solve_info* info) {
  if (!sol || !info) return fail(CAL_EINVAL, "cal_solution_get_info: NULL argument");
  *info = sol->info;
  return CAL_OK;
}

int cal_solution_coefficients(const cal_solution* sol, double* dst_host) {
  if (!sol || !dst_host) return fail(CAL_EINVAL, "cal_solution_coefficients: NULL argument");
  CAL_TRY_CUDA(cudaMemcpyAsync(dst_host, sol->d_x, sol->nrhs * 2 * sol->ne * sizeof(double2), cudaMemcpyDeviceToHost,
                               sol->ctx->stream));
  CAL_TRY_CUDA(cudaStreamSynchronize(sol->ctx->stream));
  return CAL_OK;
}

int cal_farfield(const cal_solution* sol, const double* dirs, int64_t ndir, double* out) {
  if (!sol || !dirs || !out || ndir < 1) return fail(CAL_EINVAL, "cal_farfield: bad argument");
  for (int64_t q = 0; q < 3 * ndir; ++q)
    if (!std::isfinite(dirs[q])) return fail(CAL_EINVAL, "cal_farfield: non-finite direction");
  cudaStream_t st = sol->ctx->stream;
  double* d_dirs;
  double2* d_out;
  CAL_TRY_CUDA(dalloc((void**)&d_dirs, 3 * ndir * sizeof(double), st));
  CAL_TRY_CUDA(dalloc((void**)&d_out, sol->nrhs * ndir * 3 * sizeof(double2), st));
  CAL_TRY_CUDA(cudaMemcpyAsync(d_dirs, dirs, 3 * ndir * sizeof(double), cudaMemcpyHostToDevice, st));
  int rc = sol->bc ? launch_farfield_mixed(*sol->rwg, *sol->bc, sol->d_x, (int)sol->nrhs, d_dirs, ndir, sol->k_e,
                                           sol->mu_e, d_out, st)
                   : launch_farfield(*sol->rwg, sol->d_x, (int)sol->nrhs, d_dirs, ndir, sol->k_e, sol->mu_e, d_out,
                                     sol->precision, st);
  if (!rc) {
    CAL_TRY_CUDA(cudaMemcpyAsync(out, d_out, sol->nrhs * ndir * 3 * sizeof(double2), cudaMemcpyDeviceToHost, st));
    CAL_TRY_CUDA(cudaStreamSynchronize(st));
  }
  dfree(d_dirs, st);
  dfree(d_out, st);
  return rc;
}

int cal_near_field(const cal_solution* sol, const double* points, int64_t npt, int levels,
                   const int32_t* region_in, int32_t* region_out, double* out) {
  if (!sol || !points || !out || npt < 1) return fail(CAL_EINVAL, "cal_near_field: bad argument");
  if (levels < 0 || levels > 4) return fail(CAL_EINVAL, "cal_near_field: levels must be in [0, 4]");
  for (int64_t q = 0; q < 3 * npt; ++q)
    if (!std::isfinite(points[q])) return fail(CAL_EINVAL, "cal_near_field: non-finite point");
  const Space& sp = *sol->rwg;
  const int M = (int)sp.tri_off.size() - 1;
  if (region_in)
    for (int64_t i = 0; i < npt; ++i)
      if (region_in[i] < -1 || region_in[i] >= M)
        return fail(CAL_EINVAL, "cal_near_field: region %d of point %lld outside [-1, %d)", region_in[i],
                    (long long)i, M);
  if ((int)sol->k_m.size() != M) return fail(CAL_EINVAL, "cal_near_field: solution without material data");
  if (sol->bc) return fail(CAL_EINVAL, "cal_near_field: not available for the mixed discretisation");
  CAL_TRY_CUDA(cudaSetDevice(sol->ctx->device));
  cudaStream_t st = sol->ctx->stream;
  double* d_pts = nullptr;
  double* d_inc = nullptr;
  double2* d_out = nullptr;
  int32_t* d_reg = nullptr;
  struct Free {
    std::vector<void*> p;
    cudaStream_t s;
    ~Free() { for (void* q : p) dfree(q, s); }
  } fr{{}, st};
  const size_t out_bytes = (size_t)sol->nrhs * npt * 3 * sizeof(double2);
  CAL_TRY_CUDA(dalloc((void**)&d_pts, 3 * npt * sizeof(double), st));
  fr.p.push_back(d_pts);
  CAL_TRY_CUDA(dalloc((void**)&d_inc, sol->inc.size() * sizeof(double), st));
  fr.p.push_back(d_inc);
  CAL_TRY_CUDA(dalloc((void**)&d_out, out_bytes, st));
  fr.p.push_back(d_out);
  CAL_TRY_CUDA(cudaMemcpyAsync(d_pts, points, 3 * npt * sizeof(double), cudaMemcpyHostToDevice, st));
  CAL_TRY_CUDA(cudaMemcpyAsync(d_inc, sol->inc.data(), sol->inc.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  std::vector<int> reg(npt);
  if (region_in) {
    std::copy(region_in, region_in + npt, reg.begin());
  } else {
    CAL_TRY_CUDA(dalloc((void**)&d_reg, npt * sizeof(int32_t), st));
    fr.p.push_back(d_reg);
    int rc = launch_regions(sp, M, d_pts, npt, d_reg, st);
    if (rc) return rc;
    CAL_TRY_CUDA(cudaMemcpyAsync(reg.data(), d_reg, npt * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CAL_TRY_CUDA(cudaStreamSynchronize(st));
  }
  FieldArgs f;
  f.rwg = &sp;
  f.M = M;
  f.levels = levels;
  f.precision = sol->precision;
  f.nrhs = (int)sol->nrhs;
  f.x = sol->d_x;
  f.xinc = sol->d_cinc;  // scattered-trace solutions: total trace = u^s + projected u^inc
  f.d_pts = d_pts;
  f.npt = npt;
  f.d_inc = d_inc;
  f.d_out = d_out;
  f.k_e = sol->k_e;
  f.mu_e = sol->mu_e;
  f.k_m = sol->k_m;
  f.mu_m = sol->mu_m;
  f.n_sm = sol->ctx->n_sm;
  int rc = launch_near_field(f, reg, st);
  if (rc) return rc;
  CAL_TRY_CUDA(cudaMemcpyAsync(out, d_out, out_bytes, cudaMemcpyDeviceToHost, st));
  CAL_TRY_CUDA(cudaStreamSynchronize(st));
  if (region_out) std::copy(reg.begin(), reg.end(), region_out);
  return CAL_OK;
}

void cal_solution_destroy(cal_solution* sol) { delete sol; }

int cal_check_elementary(int64_t n, double lo, double hi, double* err_cis, double* err_exp) {
  return cal::check_elementary(n, lo, hi, err_cis, err_exp);
}

int cal_check_grid_barrier(cal_ctx* ctx, int skip_block, int* status) {
  if (!ctx || !status) return fail(CAL_EINVAL, "cal_check_grid_barrier: NULL argument");
  return cal::grid_barrier_check(skip_block, status, ctx->impl.stream);
}

int64_t cal_kernel_launches(void) { return cal::launches(); }

int cal_profile_enable(int on) { return cal::prof_enable(on); }

int cal_profile_read(const char* name, int64_t* launches, double* total_ms, double* units) {
  if (!name) return fail(CAL_EINVAL, "cal_profile_read: NULL name");
  return cal::prof_read(name, launches, total_ms, units);
}

}  // extern "C"
