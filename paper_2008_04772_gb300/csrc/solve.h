// Solver-side internal interfaces (operator application, Gram solves, GMRES).
#pragma once

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
};

// y1 += C x1 + alpha S x2, y2 += C x2 + beta S x1 on the block's rows/cols;
// x, y component-major of length 2n (n = total basis count)
int pair_apply(const BlockRef& b, int vec_prec, const void* x, void* y, int64_t n, double ar,
               double ai, double br, double bi, cudaStream_t st);
int zero_vec(void* y, int prec, int64_t n, cudaStream_t st);
int convert_vec(const void* a, int pa, void* b, int pb, int64_t n, double scale, cudaStream_t st);
int single_apply(const Op& op, const void* X, const void* x, void* y, int64_t nrhs, cudaStream_t st);

// BiCGStab on the real sparse Gram matrix, nsys complex systems sharing it
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
  C* d_in = nullptr;
  C* d_out = nullptr;
  double* d_acc = nullptr;
  int* d_done = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int enqueue(const C* b, C* out, cudaStream_t st);
  int init(const int64_t* rowptr, const int* col, const double* vals_dev, int64_t n, int nsys,
           int64_t nnz, double neg, double tol, int maxit);
  int solve(const C* b, C* out, cudaStream_t st);
  ~GramSolver();
};

int gmres_cgs_step(const double2* V, int64_t n, int j, double2* w, double2* h1, double2* h2,
                   double* wn2, cudaStream_t st);
int gmres_givens(double2* H, int ldh, int j, const double2* h1, const double2* h2, const double* wn2,
                 double2* cs, double2* sn, double2* g, double* res, cudaStream_t st);
int gmres_scale(const double2* w, int64_t n, const double* nrm2, double2* out, cudaStream_t st);
int gmres_update(const double2* H, int ldh, int m, const double2* g, double2* y, const double2* V,
                 int64_t n, double2* x, cudaStream_t st);
int vec_norm2(const double2* w, int64_t n, double* out, cudaStream_t st);
int vec_axpby(const double2* a, double sa, const double2* b, double sb, double2* out, int64_t n,
              cudaStream_t st);

int launch_rhs(const Space& rwg, const double* d_inc, int nrhs, double k, double mu, double2* d_b,
               cudaStream_t st);
int launch_farfield(const Space& rwg, const double2* d_x, int nrhs, const double* d_dirs, int64_t ndir,
                    double k, double mu, double2* d_out, cudaStream_t st);

// BC tile launcher (assemble.cu)
int launch_bc_regular_tiles(const AssembleArgs& a, const int* cells, int64_t ncell, const int2* tiles,
                            int64_t ntile, int max_cell, int n_sm, double units);

}  // namespace cal
