// Solver-side internal interfaces (operator application, Gram solves, GMRES).
#pragma once

#include <complex>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace cal {

struct Rules6 {
  double b[18];
  double w[6];
};
Rules6 rules6();

// one stored (S, C) block of a PMCHWT-structured operator
struct BlockRef {
  const void* S = nullptr;      // may be null (operator absent)
  const void* C = nullptr;
  int64_t rows = 0, cols = 0;
  int64_t row_off = 0, col_off = 0;
  int precision = CAL_FP64;
  const int64_t* rowptr = nullptr;  // CSR when non-null
  const int* col = nullptr;
  // combined block (float32 dense, one vector): y1 += C x1 + S x2, y2 += C x2 + S2 x1
  const void* S2 = nullptr;
  const HMat* hmat = nullptr;  // CAL_HMAT block: S and C in H-matrix form
  int hmask = 0;               // with hmat: bit 1 apply S, bit 2 apply C
};

// y1 += C x1 + alpha S x2, y2 += C x2 + beta S x1 on the block's rows/cols;
// x, y component-major of length 2n (n = total basis count)
int pair_apply(const BlockRef& b, int vec_prec, const void* x, void* y, int64_t n, double ar,
               double ai, double br, double bi, cudaStream_t st);
// the same for nrhs vectors [nrhs][2n] at once (dense float32 blocks; float32
// arithmetic for float32 vectors, float64 products and sums for float64 ones)
int pair_apply_multi(const BlockRef& b, int vec_prec, const void* x, void* y, int64_t n, int nrhs, double ar,
                     double ai, double br, double bi, int n_sm, cudaStream_t st);
// the same for a CSR block (near-field P, touching-pair blocks); scratch holds
// 2 * cols * nrhs vector elements (the interleaved copy of x)
int pair_spmv_multi(const BlockRef& b, int vec_prec, const void* x, void* y, int64_t n, int nrhs, double ar,
                    double ai, double br, double bi, void* scratch, cudaStream_t st);
int zero_vec(void* y, int prec, int64_t n, cudaStream_t st);
int convert_vec(const void* a, int pa, void* b, int pb, int64_t n, double scale, cudaStream_t st);
int single_apply(const Op& op, const void* X, const void* x, void* y, int64_t nrhs, cudaStream_t st);

// Combined float32 block of two operator pairs on one set of unknowns:
// C = Ca + Cb, S1 = aa Sa + ab Sb, S2 = ba Sa + bb Sb, with (Sa, Ca) dense
// [rows][rows] and (Sb, Cb) [nb][nb] on its diagonal at (off, off). init:
// first fill C, S1, S2 from (Sa, Ca) alone; Sb == nullptr: no inner block.
int combine_blocks(const void* Sa, const void* Ca, int64_t rows, std::complex<double> aa, std::complex<double> ba,
                   const void* Sb, const void* Cb, int64_t nb, int64_t off, std::complex<double> ab,
                   std::complex<double> bb, void* Co, void* S1, void* S2, bool init, int n_sm, cudaStream_t st);

// check of the bounded grid barrier (see cal_check_grid_barrier)
int grid_barrier_check(int skip_block, int* status, cudaStream_t st);

// BiCGStab on the real sparse Gram matrix, nsys complex systems sharing it
// grid-wide barrier state of a cooperative launch (zeroed before the launch):
// count of arrivals since the launch, the error word of a wait that gave up
struct GridBar {
  unsigned count, pad0;
  int err, pad1;
};

template <typename R>
struct GramSolver {
  using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
  const int64_t* d_rowptr = nullptr;
  const int* d_col = nullptr;
  R* d_val = nullptr;
  int64_t n = 0;
  int nsys = 0;
  double neg = 1.0, tol = 1e-10;
  int maxit = 30;
  C* d_work = nullptr;
  double* d_acc = nullptr;   // per-solve sums, |b|^2 and the grid barrier state
  int* d_err = nullptr;      // sticky: a bounded barrier wait gave up
  int lpr = 1, rpb = 1, threads = 0;
  unsigned grid = 0;
  size_t smem = 0;
  bool cached = false;  // one sweep covers the rows: the row entries stay in registers
  int init(const int64_t* rowptr, const int* col, const double* vals_dev, int64_t n, int nsys,
           int64_t nnz, double neg, double tol, int maxit, cudaStream_t st);
  // x = neg G^{-1} b for the nsys systems (b, out: [nsys][n]), one cooperative launch
  int solve(const C* b, C* out, cudaStream_t st);
  // CAL_ETIMEOUT if any solve since init gave up at a barrier (synchronises st)
  int check(cudaStream_t st) const;
  size_t acc_bytes() const;
  ~GramSolver();
};

int gmres_cgs_step(const double2* V, int64_t bV, int64_t n, int j, double2* w, double2* h1, double2* h2,
                   int64_t bh, double* wn2, int64_t bwn, int nrhs, cudaStream_t st);
int gmres_givens(double2* H, int ldh, int64_t bH, int j, const double2* h1, const double2* h2, int64_t bh,
                 const double* wn2, int64_t bwn, double2* cs, double2* sn, int64_t bcs, double2* g, int64_t bg,
                 double* res, int64_t bres, int nrhs, cudaStream_t st);
int gmres_scale(const double2* w, int64_t bw, int64_t n, const double* nrm2, int64_t bn, double2* out,
                int64_t bout, int nrhs, cudaStream_t st);
int gmres_update(const double2* H, int ldh, int m, const double2* g, double2* y, const double2* V,
                 int64_t n, double2* x, cudaStream_t st);
int vec_norm2(const double2* w, int64_t n, double* out, int64_t bout, int nrhs, cudaStream_t st);
int vec_axpby(const double2* a, double sa, const double2* b, double sb, double2* out, int64_t n,
              cudaStream_t st);
int vec_gather(const double2* src, int64_t bsrc, double2* dst, int64_t n, int nrhs, cudaStream_t st);

// A10 (gemm_tc.cu): tensor-core 3xTF32 product and the right-hand-side embedding
bool gemm_tc_supported(int64_t cols, int nrhs);
int multi_matvec_tc(const float2* Xop, int64_t rows, int64_t cols, const float2* x, float2* y, int nrhs, int n_sm,
                    cudaStream_t st);
int split_tf32(const float* x, float* hi, float* lo, int64_t n, cudaStream_t st);
int gemm_tf32x3(const float* A, int64_t M, int64_t K, const float* Bt, int NB, float* Z, int* d_err,
                int n_sm, cudaStream_t st);
int gemm_tf32x3_bsplit(const float* A, int64_t M, int64_t K, const float* Bh, const float* Bl, int NB, float* Z,
                       int* d_err, int n_sm, cudaStream_t st);
template <typename VT>
int embed_rhs(const VT* X, int nrhs, int64_t n_total, int64_t col_off, int64_t ncols, float* Bt, int NB,
              cudaStream_t st);
template <typename VT>
int combine_rhs(const float* ZS, const float* ZC, int64_t rows, int NB, int nrhs, int64_t n_total, int64_t row_off,
                VT* Y, double ar, double ai, double br, double bi, cudaStream_t st);

// mode 0: tested incident traces (the total-trace right-hand side); mode 1: the
// loads int phi.(field x n) of the L2 projection of u^inc onto RWG
int launch_rhs(const Space& rwg, const double* d_inc, int nrhs, double k, double mu, double2* d_b,
               cudaStream_t st, int mode = 0);
// values of the RWG mass matrix int phi_i . phi_j on a CSR pattern holding every
// pair of edges of a triangle (values zeroed by the caller)
int launch_rwg_mass(const Space& rwg, const int64_t* rowptr, const int* col, double* val, cudaStream_t st);
int launch_farfield(const Space& rwg, const double2* d_x, int nrhs, const double* d_dirs, int64_t ndir,
                    double k, double mu, double2* d_out, int precision, cudaStream_t st);
// the mixed discretisation's far field: u_1 in RWG, u_2 in BC (float64)
int launch_farfield_mixed(const Space& rwg, const Space& bc, const double2* d_x, int nrhs, const double* d_dirs,
                          int64_t ndir, double k, double mu, double2* d_out, cudaStream_t st);
// y += alpha X x for a dense float64 block X [rows][ld] (rows x cols used)
int gemv_acc(const double2* X, int64_t ld, int64_t rows, int64_t cols, const double2* x, double2* y,
             std::complex<double> alpha, cudaStream_t st);

// H-matrix form with ACA (hmat.cu, Section 3.3): out gets the CAL_HMAT form of the
// dense square block (S and/or C) on the space's supports; leaves within chi
// kept (ACA to nu, at most max_rank), inadmissible leaves dense
int hmat_compress(const Op& dense, const Space& sp, double nu, double chi, int max_rank, Op& out, cudaStream_t st);
int hmat_pair_apply(const HMat& h, bool withS, bool withC, int vec_prec, const void* x, void* y, int64_t ntot,
                    int64_t off, double ar, double ai, double br, double bi, cudaStream_t st);
int hmat_apply_halves(const HMat& h, bool withS, bool withC, int vec_prec, const void* x1, const void* x2, void* y1,
                      void* y2, double ar, double ai, double br, double bi, cudaStream_t st);
int hmat_expand(const HMat& h, int which, void* dst, cudaStream_t st);

// Near field (field.cu): the Stratton–Chu representations of the solved traces
// at points off the surface
struct FieldArgs {
  const Space* rwg = nullptr;
  int M = 1, levels = 2, precision = CAL_FP64, nrhs = 1;
  int n_sm = 0;                   // SMs of the device (grid sizing)
  const double2* x = nullptr;     // [nrhs][2N] coefficients (c, d)
  const double2* xinc = nullptr;  // optional [nrhs][2N] added to x (total traces)
  const double* d_pts = nullptr;  // [npt][3]
  int64_t npt = 0;
  const double* d_inc = nullptr;  // [nrhs][6] incident plane waves
  double2* d_out = nullptr;       // [nrhs][npt][3]
  double k_e = 1.0, mu_e = 1.0;
  std::vector<std::complex<double>> k_m, mu_m;
};
// region of each point: the scatterer m whose mesh winds around it, or -1
int launch_regions(const Space& rwg, int M, const double* d_pts, int64_t npt, int32_t* d_region, cudaStream_t st);
int launch_near_field(const FieldArgs& f, const std::vector<int>& region, cudaStream_t st);

// BC tile launcher (assemble.cu)
// A5 over units: units [nunits] of {v, begin, count, flag} ints, each a test
// cell v with the trial cells wlist[begin .. begin + count)
int launch_bc_regular_units(const AssembleArgs& a, const void* units, int64_t nunits, const int* wlist, int max_cell,
                            int n_sm, double work);
// trial cells per unit for a test cell of n1 triangles when the float32
// one-thread-per-(test triangle, trial cell) kernel applies, else 0
int bc_owner_width(const Space& s, int precision, int n1, int max_cell);

}  // namespace cal
