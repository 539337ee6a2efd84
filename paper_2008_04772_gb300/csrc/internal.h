// Internal declarations of the GB300 PMCHWT library (not part of the C ABI).
//
// Every basis function (RWG on primal triangles, BC on barycentric ones) is
// stored per triangle tau as "slots": on tau it equals sigma * (x - c_tau) + w,
// with c_tau the centroid, so div = 2 sigma (Section 3.2 spaces, lowest-order
// Raviart–Thomas pieces). A triangle carries up to `nslot` such pieces, each
// tagged with its global basis (edge) index, or -1 for an empty slot.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "cal.h"

namespace cal {

// ---- errors ----------------------------------------------------------------
void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);
#define CAL_TRY_CUDA(expr)                                                    \
  do {                                                                        \
    cudaError_t _e = (expr);                                                  \
    if (_e != cudaSuccess)                                                    \
      return ::cal::fail(CAL_ECUDA, "%s: %s (%s:%d)", #expr,                  \
                         cudaGetErrorString(_e), __FILE__, __LINE__);         \
  } while (0)

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device. The limit only grows, so a launch from another host thread
// that was sized for less stays valid (setting it per launch would race).
inline int ensure_dyn_smem(const void* kern, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> limit;
  int dev = 0;
  CAL_TRY_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  int& cur = limit[{dev, kern}];
  if (bytes > cur) {
    CAL_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    cur = bytes;
  }
  return CAL_OK;
}

// ---- instrumentation (host.cpp) ------------------------------------------------
void note_launch(int n = 1);
// events around one launch of kernel family `name` doing `units` of work
int prof_begin(cudaStream_t st, const char* name, double units);
void prof_end(cudaStream_t st, int token);
// a zeroed device counter whose value (read after the launch) replaces the
// token's units; nullptr when profiling is off or the token is invalid
unsigned long long* prof_counter(int token, cudaStream_t st);

// ---- device records ----------------------------------------------------------
// float32 triangle: centroid as hi + lo float pair, vertex offsets from it.
// diam: longest edge (the size in the near / medium / far class of a pair)
struct __align__(16) TriF {
  float chi[3], clo[3];
  float off[3][3];
  float area;
  int vid[3];
  float diam;
};
struct __align__(16) TriD {
  double c[3];
  double off[3][3];
  double area;
  int vid[3];
  int pad;
  double diam;
};

// ordered singular pair (shares >= 1 vertex id) with Sauter–Schwab vertex orders:
// shared vertices first (in the test triangle's storage order), the rest after
struct SingPair {
  int t1, t2;
  signed char cls;      // 1 vertex, 2 edge, 3 identical
  signed char o1[3], o2[3];
  signed char pad;
};

// f(i) for i in [0, n) on up to 16 host threads (chunks of 32 taken in turn);
// f must only write what belongs to its own i
template <class F>
inline void parallel_for(int n, const F& f) {
  const int nt = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), 16));
  if (nt == 1 || n < 512) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int> next(0);
  auto work = [&]() {
    for (;;) {
      const int i0 = next.fetch_add(32);
      if (i0 >= n) return;
      for (int i = i0; i < std::min(n, i0 + 32); ++i) f(i);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(work);
  work();
  for (auto& x : th) x.join();
}

// ---- host objects --------------------------------------------------------------
struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int n_sm = 0;
  double* pinned = nullptr;  // small page-locked scratch for residual read-backs
};

// stream-ordered device memory: no device-wide synchronisation, so requests on
// different streams overlap (a plain cudaFree waits for the whole device)
inline cudaError_t dalloc(void** p, size_t n, cudaStream_t s) { return cudaMallocAsync(p, n ? n : 16, s); }
inline void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

struct Mesh {
  Ctx* ctx = nullptr;
  int64_t nv = 0, nt = 0, ne = 0, M = 0;
  std::vector<double> X;         // [nv][3]
  std::vector<int> T;            // [nt][3], triangles grouped by scatterer
  std::vector<int> dom;          // [nt]
  std::vector<int> e_lo, e_hi, e_dom, e_tp, e_ap, e_tm, e_am;
  std::vector<double> e_len;
  std::vector<int> tri_edge;     // [nt][3]: edge opposite local vertex a
  std::vector<int> tri_sign;     // [nt][3]: +1 if the triangle is T+ of that edge
  std::vector<int64_t> tri_off, edge_off, vert_lo, vert_hi;  // per scatterer ranges
  std::vector<int> valence;      // edges per vertex
  double h = 0.0;
  int max_valence = 0;
};

struct Space {
  Mesh* mesh = nullptr;
  int kind = 0;
  int64_t ntri = 0, nbasis = 0;
  int nslot = 0;
  std::vector<TriD> triD;        // host master copy
  std::vector<int> slot_edge;    // [ntri][nslot]
  std::vector<double> slot_sw;   // [ntri][nslot][4] = sigma, w
  std::vector<int> parent;       // BC: primal parent triangle of each tau
  // dual cells (BC): barycentric triangles and edges of each primal vertex
  std::vector<int> cell_tri_ptr, cell_tri, cell_edge_ptr, cell_edge;
  // support bounding boxes per basis
  std::vector<double> box_lo, box_hi;  // [nbasis][3]
  // triangle ranges per scatterer
  std::vector<int64_t> tri_off;
  // singular ordered pairs per scatterer
  std::vector<std::vector<SingPair>> sing;
  // device copies
  TriF* d_triF = nullptr;
  TriD* d_triD = nullptr;
  int* d_slot_edge = nullptr;
  float* d_slot_swf = nullptr;
  double* d_slot_swd = nullptr;
  int* d_cell_tri_ptr = nullptr;
  int* d_cell_tri = nullptr;
  int* d_cell_edge_ptr = nullptr;  // BC: slot sl of every triangle of cell v is cell_edge[cell_edge_ptr[v] + sl]
  int* d_cell_edge = nullptr;
  std::vector<SingPair*> d_sing;
  // BC: on every small triangle tau of a dual cell the divergence of each of the
  // cell's functions is +-l_e/(2N_v)/|tau|, so sigma_{b,tau} = s_b / |tau| with s_b
  // constant over the cell: cell_slot_s[cell_edge_ptr[v] + sl] = s_b (float), and
  // sigma_factors records that the slot table satisfies this to 1e-9
  std::vector<float> cell_slot_s;
  float* d_cell_slot_s = nullptr;
  bool sigma_factors = false;
  // k-independent float64 sums of the touching pairs (18 doubles per pair),
  // per scatterer: filled by its first float32 singular launch that asks for
  // C, read by later float32 launches with the same Gauss order
  struct StaticSums {
    double* buf = nullptr;
    int ng = 0;
    bool ready = false;
    cudaEvent_t done = nullptr;  // recorded on the filling stream after the launch
  };
  mutable std::mutex static_mu;
  mutable std::vector<StaticSums> sing_static;
  // BC regular-pair work units (a test cell and a run of trial cells) of one
  // scatterer, cutoff, rule and kernel: built and uploaded by the first
  // assembly that asks, read by the later ones (a problem's exterior and
  // interior blocks take the same lists); guarded by unit_mu, which is held
  // while a list is built (the singular launches' static_mu is not)
  mutable std::mutex unit_mu;
  struct UnitLists {
    int scat = 0, nreg = 0;
    double chi = 0;
    bool owner = false;
    int max_cell = 0;
    int64_t nunits = 0;
    double pairs = 0;  // regular triangle pairs (the work count)
    int* d_units = nullptr;
    int* d_wlist = nullptr;
    cudaEvent_t done = nullptr;  // the uploads, recorded on the stream that made them
  };
  mutable std::vector<std::unique_ptr<UnitLists>> unit_lists;
  // near-field patterns (CSR over the scatterer's edges) per (scatterer,
  // cutoff); guarded by static_mu
  struct NearPattern {
    int scat = 0;
    double chi = 0;
    std::vector<int64_t> rowptr;
    std::vector<int> col;
  };
  mutable std::vector<std::unique_ptr<NearPattern>> near_patterns;
  ~Space();
};

// H-matrix form of a square operator block (Section 3.3): the leaves of a block
// cluster tree over the supports' bounding boxes; inadmissible leaves are kept
// dense, admissible ones within the cutoff as U V^T from ACA, the rest dropped.
// Up to two operators (S, C) share the leaves; each has its own ranks.
struct HLeafD {  // device record of a low-rank leaf
  int64_t r0, c0, uoff, voff;  // index-list offsets; offsets of U [rank][nr] and V [rank][nc]
  int nr, nc, rank, pad;
};
struct HNearD {  // device record of a dense leaf
  int64_t r0, c0, off;  // index-list offsets; offset of its [nr][nc] values
  int nr, nc;
};
struct HMat {
  int64_t n = 0;                 // dofs of the (square) block
  int precision = CAL_FP64;
  std::vector<int> idx;          // local dof lists of the leaves, concatenated
  struct Leaf {
    int64_t r0, c0;              // offsets into idx
    int nr, nc;
    double dist;                 // distance of the cluster boxes
  };
  std::vector<Leaf> near, far;   // inadmissible; admissible within the cutoff
  int64_t near_entries = 0;
  int* d_idx = nullptr;
  HNearD* d_near_tab = nullptr;
  void* d_near[2] = {nullptr, nullptr};     // per operator (0 = S, 1 = C)
  void* d_U[2] = {nullptr, nullptr};
  void* d_V[2] = {nullptr, nullptr};
  HLeafD* d_far_tab[2] = {nullptr, nullptr};
  std::vector<int> rank[2];
  // prefix sums for the product: rows of the dense and of the low-rank leaves,
  // ranks per operator (device copies)
  int64_t* d_roff_near = nullptr;
  int64_t* d_roff_far = nullptr;
  int64_t* d_koff[2] = {nullptr, nullptr};
  int64_t near_rows = 0, far_rows = 0, ktot[2] = {0, 0};
  int64_t stored = 0;            // stored complex entries, all operators
  int max_rank_seen = 0;
  ~HMat();
};

struct Op {
  Ctx* ctx = nullptr;
  int op_mask = 0, precision = 0, format = 0;
  int64_t rows = 0, cols = 0, nnz = 0;
  int64_t row_offset = 0;
  void* d_S = nullptr;           // dense [rows][cols] or CSR values
  void* d_C = nullptr;
  int64_t* d_rowptr = nullptr;   // CSR
  int* d_col = nullptr;
  std::vector<int64_t> h_rowptr; // CSR pattern on the host
  std::vector<int> h_col;
  HMat* hmat = nullptr;          // CAL_HMAT: the H-matrix form (owned)
  ~Op();
};

// ---- host construction (host.cpp) ----------------------------------------------
int build_mesh(Mesh& m, const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
               const int32_t* domain);
int build_rwg(Space& s, Mesh& m);
int build_bc(Space& s, Mesh& m);
void build_singular_pairs(Space& s);
// near-field CSR pattern within one scatterer block: keep (i,j) iff the
// support boxes are at most chi apart; local indices (edge - edge_off)
void near_pattern(const Space& s, int scat, double chi, std::vector<int64_t>& rowptr,
                  std::vector<int>& col);
// Gram pattern (rows RWG edges, cols BC edges), CSR
void gram_pattern(const Space& bc, std::vector<int64_t>& rowptr, std::vector<int>& col);
int upload_space(Space& s, cudaStream_t st);  // stream-ordered; returns after the copies

// quadrature tables (host.cpp): Gauss–Legendre on [0,1] by Newton iteration on
// Legendre polynomials; the symmetric degree-4 six-point triangle rule from its
// closed form; the centroid rule.
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);
void triangle_rule(int npts, std::vector<double>& bary, std::vector<double>& w);

// ---- device launches (assemble.cu) --------------------------------------------
struct AssembleArgs {
  const Space* sp;
  int scat;             // -1 = union
  double kr, ki;
  int want;             // bit 1 S, bit 2 C
  int nreg, nsing;      // regular points per triangle, GL points per dimension
  int precision;         // storage/regular-pair precision: CAL_FP32 or CAL_FP64
  int sing32;            // singular pairs in float32 (CAL_FP32_ALL)
  int format;
  // dense output
  int64_t row_off, ld;
  // CSR output (local indices)
  const int64_t* rowptr;
  const int* col;
  void* S;
  void* C;
  cudaStream_t stream;
};
int set_quadrature_tables(int nreg, int nsing);
int launch_rwg_regular(const AssembleArgs& a);
// max errors of the singular kernel's own double cis/exp against the CUDA library
int check_elementary(int64_t n, double lo, double hi, double* err_cis, double* err_exp);
int launch_singular(const AssembleArgs& a);
// A8: y += the regular (non-touching) part of the PMCHWT block of space s
// restricted to scatterer scat (-1: union) at wavenumber k, computed on the
// fly: y1 += C x1 + alpha S x2, y2 += C x2 + beta S x1 for nrhs vectors
// [nrhs][2n]; precision CAL_FP32 or CAL_FP64 (kernel), vec_prec of x and y
int launch_rwg_free(const Space& s, int scat, double kr, double ki, int nreg, int precision, int vec_prec,
                    const void* x, void* y, int64_t n, int nrhs, double ar, double ai, double br, double bi,
                    cudaStream_t st);
// C of the mixed discretisation in float64: Crb [rows][ld] = <C BC_j, RWG_i> with
// RWG written on the barycentric refinement (d_redge [ntri][3], d_rsw
// [ntri][3][4] on the BC space's triangles) and Cbr = <C RWG_j, BC_i>, dense,
// block of scatterer scat (-1: union) at row/col offset row_off; zeroed by the
// caller; nreg: 6, 1 or 0 (classes)
int launch_cross_c(const Space& bc, const int* d_redge, const double* d_rsw, int scat, double kr, double ki, int nreg,
                   int nsing, int64_t row_off, int64_t ld, double* Crb, double* Cbr, cudaStream_t st);
int launch_gram(const Space& rwg, const Space& bc, const int64_t* rowptr, const int* col,
                const int64_t* rowptrT, const int* colT, double* vals, double* valsT,
                cudaStream_t stream);

}  // namespace cal

struct cal_ctx { cal::Ctx impl; };
struct cal_mesh { cal::Mesh impl; };
struct cal_space { cal::Space impl; };
struct cal_op { cal::Op impl; };
