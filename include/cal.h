/*
 * cal.h — C ABI of the GB300 (sm_103a) Calderón-preconditioned PMCHWT library.
 *
 * Method: Kleanthous, Betcke, Hewett, Escapil-Inchauspé, Jerez-Hanckes,
 * Baran, "Accelerated Calderón preconditioning for Maxwell transmission
 * problems", arXiv 2008.04772. Section and equation names below refer to it.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: 0 on success, a negative CAL_E* code on failure; the
 *   calling thread's message is then available from cal_last_error().
 *   No entry point aborts the process or traps the device.
 * - Ownership: every input array is copied at the call; the caller may free
 *   it on return. Handles (cal_ctx, cal_mesh, cal_space, cal_op,
 *   cal_solution, cal_queue) are owned by the library and freed by the
 *   matching *_destroy, which accepts NULL. Objects created from a context
 *   must be destroyed before the context.
 * - Output buffers are allocated by the caller. Where an argument is marked
 *   "host or device", the library inspects the pointer and copies accordingly.
 * - Complex numbers are interleaved (re, im); complex64 = 2 x float32,
 *   complex128 = 2 x float64. Dense matrices are row-major.
 * - Time convention e^{-i omega t}; relative permittivity/permeability,
 *   exterior medium eps = mu = 1 (Section 2).
 * - Basis numbering: primal edges sorted by (scatterer id, lower vertex id,
 *   higher vertex id); RWG_e and BC_e share the index e (Section 3.2).
 * - PMCHWT unknowns are component-major: x = [c_0..c_{N-1}, d_0..d_{N-1}],
 *   u_1 = sum c_e RWG_e = gamma_D E, u_2 = sum d_e RWG_e = (k/mu) gamma_N E
 *   (eq. boundary_conditions_traces), N = number of primal edges.
 */
#ifndef CAL_H
#define CAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes --------------------------------------------------------- */
#define CAL_OK 0
#define CAL_EINVAL (-1)    /* bad argument (NULL, size, NaN, unsupported option) */
#define CAL_EMESH (-2)     /* not a closed, consistently oriented 2-manifold, or
                              scatterers share vertices */
#define CAL_ENOMEM (-3)    /* device/host allocation or HBM admission refused;
                              nothing is left partially allocated */
#define CAL_ENOTCONV (-4)  /* GMRES reached maxit; the solution is still returned */
#define CAL_ETIMEOUT (-5)  /* a bounded wait gave up (queue) */
#define CAL_ECUDA (-6)     /* a CUDA runtime call failed */

/* ---- enumerations -------------------------------------------------------- */
#define CAL_RWG 1          /* Rao–Wilton–Glisson on the primal mesh (Section 3.2) */
#define CAL_BC 2           /* Buffa–Christiansen on the barycentric refinement    */

#define CAL_OP_S 1         /* electric operator S = gamma_D E (Section 2)          */
#define CAL_OP_C 2         /* magnetic operator C = gamma_D H (Section 2)          */

#define CAL_FP64 1         /* all assembly and storage in float64 (complex128)    */
#define CAL_FP32 2         /* "FP32 bulk": regular pairs in float32; singular
                              (Sauter-Schwab) pairs split into the static kernel
                              parts 1/(4 pi r), -1/(4 pi r^3), summed in
                              double-float (pairs of floats, ~2^-46 relative),
                              and the smooth remainder in float32; storage
                              complex64                                          */
#define CAL_FP32_ALL 3     /* regular and singular pairs in float32 (singular point
                              differences formed in reference coordinates, so no
                              cancellation), storage complex64                     */

#define CAL_DENSE 1
#define CAL_CSR 2
#define CAL_HMAT 3         /* H-matrix: dense and low-rank (ACA) leaves, Section 3.3 */

/* preconditioners of Section 3.1 (P = A is available for one scatterer, where
   it equals D) */
#define CAL_PRECOND_NONE 0
#define CAL_PRECOND_D 1
#define CAL_PRECOND_DE 2
#define CAL_PRECOND_DI 3
#define CAL_PRECOND_SE 4
#define CAL_PRECOND_SI 5

/* ---- opaque handles ------------------------------------------------------ */
typedef struct cal_ctx cal_ctx;
typedef struct cal_mesh cal_mesh;
typedef struct cal_space cal_space;
typedef struct cal_op cal_op;
typedef struct cal_solution cal_solution;
typedef struct cal_problem cal_problem;
typedef struct cal_queue cal_queue;

/* ---- context ------------------------------------------------------------- */
/* Bind a context to CUDA device `device` and create its stream. */
int cal_init(cal_ctx** out, int device);
void cal_ctx_destroy(cal_ctx* ctx);
/* Message of the last failed call on this thread ("" if none). */
const char* cal_last_error(void);
/* The context's CUDA stream (cudaStream_t), for callers that order their own work. */
void* cal_ctx_stream(cal_ctx* ctx);

/* ---- mesh (Section 2: M disjoint closed surfaces Gamma_m) --------------- */
/* verts [nv][3] float64; tris [nt][3] int32 vertex ids, counter-clockwise seen
   from outside (normal into the exterior, Section 2); domain [nt] int32
   scatterer ids 0..M-1, or NULL for M = 1. Validates that every edge is used
   exactly twice in opposite directions and that scatterers share no vertex
   (CAL_EMESH otherwise). */
int cal_mesh_create(cal_ctx* ctx, const double* verts, int64_t nv, const int32_t* tris,
                    int64_t nt, const int32_t* domain, cal_mesh** out);
void cal_mesh_destroy(cal_mesh* mesh);

typedef struct {
  int64_t n_vertices, n_triangles, n_edges, n_scatterers;
  double h;                 /* maximum primal edge length */
  int32_t max_valence;      /* maximum number of edges at a vertex */
} cal_mesh_info;
int cal_mesh_get_info(const cal_mesh* mesh, cal_mesh_info* info);

/* ---- spaces (Section 3.2, eq. RWG_discretisation1) ----------------------- */
/* kind CAL_RWG: RWG_e = +l_e f on T+ (the triangle whose counter-clockwise
   cycle runs lower -> higher vertex along e) and -l_e f on T-, with
   f(x) = (x - p)/(2|T|), p the vertex opposite e.
   kind CAL_BC: Buffa–Christiansen function of edge e on the barycentric
   refinement: flux l_e crosses the dual edge of e from the dual cell of the
   lower vertex to that of the higher one; divergence integral +-l_e/(2N_v)
   on each of the 2N_v small triangles of a cell; circulation fixed by mirror
   symmetry about the half-edge, which carries zero flux. */
int cal_space_create(cal_mesh* mesh, int kind, cal_space** out);
void cal_space_destroy(cal_space* space);

/* ---- Galerkin assembly (Sections 2, 3.3) --------------------------------- */
/* Assembles <S phi_j, phi_i> and/or <C phi_j, phi_i> (op_mask = CAL_OP_S |
   CAL_OP_C) at wavenumber k = k_re + i k_im over test x trial, both RWG or
   both BC on the same mesh, with the pairing <a,b> = int a.(n x b)
   (eq. dualpairingGammam):
     S_ij = -ik II G phi_i.phi_j + (i/k) II G div phi_i div phi_j,
     C_ij =     II grad_x G . (phi_i(x) x phi_j(y)),  G = e^{ikr}/(4 pi r).
   scatterer = -1 assembles the union surface (all pairs, "exterior" use);
   scatterer = m restricts test and trial to Gamma_m (interior use).
   near_cutoff: INFINITY = dense; otherwise entry (i,j) is kept iff the
   bounding boxes of the supports are <= near_cutoff apart (eq. nf_condition
   read at entry level) and the result is CSR (BC spaces only).
   q_regular: points per triangle of the regular tensor rule, 6 (degree 4,
   36 evaluations per pair) or 1 (centroid) for every regular pair; or 0: by
   the pair's class (Section 3.3, default orders q_near, q_medium, q_far =
   4, 3, 2): 6, 4 or 3 points (36 / 16 / 9 evaluations) for a pair whose
   centroid distance is <= 2, <= 4 or > 4 times the longer of the two
   longest edges (the paper names the classes, not these bounds); q_singular: Gauss–Legendre
   points per dimension of the Sauter–Schwab rules, 1..16 (4 gives the
   paper's 512/1280/1536 evaluations). precision: CAL_FP64, CAL_FP32 or
   CAL_FP32_ALL. */
int cal_assemble(cal_ctx* ctx, int op_mask, double k_re, double k_im, cal_space* test,
                 cal_space* trial, int scatterer, double near_cutoff, int q_regular,
                 int q_singular, int precision, cal_op** out);
void cal_op_destroy(cal_op* op);

typedef struct {
  int64_t rows, cols, nnz;  /* nnz = rows*cols for dense */
  int32_t format;           /* CAL_DENSE or CAL_CSR */
  int32_t precision;        /* CAL_FP64 (complex128 values) or CAL_FP32 (complex64) */
  int32_t op_mask;
  int32_t row_offset;       /* first basis index of the block (scatterer restriction) */
} cal_op_info;
int cal_op_get_info(const cal_op* op, cal_op_info* info);

/* Copies operator `which` (CAL_OP_S or CAL_OP_C) to dst (host or device):
   dense: rows*cols complex values of the op's precision; CSR: nnz values, and
   when row_ptr/col_idx are non-NULL also rows+1 and nnz int64 indices (host). */
int cal_op_export(const cal_op* op, int which, void* dst, int64_t* row_ptr, int64_t* col_idx);

/* y = X x for X = operator `which`; x [nrhs][cols], y [nrhs][rows] complex of
   the op's precision, both device pointers; enqueued on `stream`
   (cudaStream_t, NULL = the context stream). For a float32 dense operator and
   4 <= nrhs <= 128 vectors (even cols) the product runs on the tensor cores
   as a 3xTF32 GEMM (float32 accuracy: each 32-wide K tile's partial product is
   summed in registers with round-to-nearest; the operator is read once, as
   float32, and split into its TF32 parts in shared memory, so no copy of it is
   kept); otherwise one GEMV/SpMV per vector. */
int cal_matvec(const cal_op* op, int which, const void* x, void* y, int64_t nrhs, void* stream);

/* The paper has no counterpart to this entry point: it serves callers that
   may not allocate device memory. Same product and arguments as cal_matvec's
   tensor-core branch (float32 dense operator, even cols, 3xTF32), for
   1 <= nrhs <= CAL_MATVEC_STATIC_MAX_NRHS, but every temporary lives in one
   fixed device array of CAL_MATVEC_STATIC_SCRATCH_BYTES per device; the call
   allocates nothing (no cudaMalloc/cudaFree, no allocating library routine).
   The scratch needed is 4*NB*(2*cols + rows) bytes with NB =
   16*ceil(ceil(nrhs/2)/4), plus (nrhs+1)*cols*8 for odd nrhs, plus a flag
   (each part rounded up to 256 bytes): a 7680 x 7680 block fits every nrhs up
   to 128. Larger requests return CAL_EINVAL, with the sizes in
   cal_last_error(), before any GPU work. x and y must be device memory of the
   operator's device (CAL_EINVAL otherwise). All calls share the array: calls
   whose GPU work overlaps (other streams, other host threads) race on it and
   must be serialised by the caller. The first call on a device looks up the
   array's device address (cudaGetSymbolAddress) and keeps it, so make that
   first call before any stream capture, and do not use the library across a
   cudaDeviceReset. The caller's current device is unchanged on return.
   Returns after the product has completed on `stream`; CAL_ETIMEOUT if a
   bounded wait of the product gave up. */
#define CAL_MATVEC_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
#define CAL_MATVEC_STATIC_MAX_NRHS 128
int cal_matvec_static(const cal_op* op, int which, const void* x, void* y, int64_t nrhs, void* stream);

/* H-matrix form of a dense square operator (Section 3.3; the assembly of the
   paper's software, approximated from the assembled entries): a cluster tree
   of the basis functions of `space` in the block (median split of the support
   boxes' centres along the longest side of the cluster box, at most 16 per
   leaf cluster); a block of two clusters is admissible when their support
   boxes are disjoint (eq. admissibility), otherwise split down to leaf
   clusters and kept dense. Admissible leaves within chi of each other are
   approximated by partially pivoted ACA to the relative tolerance nu (stop when
   |u_r||v_r| <= nu |sum u_k v_k^T|_F), the others dropped (eq. nf_condition,
   chi = INFINITY keeps all). The result (format CAL_HMAT) can be exported
   (densely expanded), applied with cal_matvec, and its info's nnz is the number
   of stored complex entries of all its operators (S and C together). */
int cal_op_compress(cal_ctx* ctx, const cal_op* dense, const cal_space* space, double nu, double chi,
                    cal_op** out);

/* Gram matrix G_ij = <BC_j, RWG_i> = int BC_j . (n x RWG_i) (eqs. MassA,
   MassP: M_A = diag(G, G), M_P = diag(-G^T, -G^T) in the unknown ordering above)
   written densely to dst_host [N][N] float64. For tests of small meshes. */
int cal_gram_export(cal_space* rwg, cal_space* bc, double* dst_host);

/* ---- PMCHWT solve (eqs. PMCHWT_multiple_scatterers, GalA-MassP) --------- */
typedef struct {
  int32_t precond;          /* CAL_PRECOND_*                                   */
  int32_t precision;        /* CAL_FP64, CAL_FP32 (FP32 bulk) or CAL_FP32_ALL  */
  int32_t q_regular_A, q_singular_A;   /* A's rules (6 / 1 / 0 = by class, 4)  */
  int32_t q_regular_P, q_singular_P;   /* P's rules (bi-parametric: 1, 1)      */
  double near_cutoff_P;     /* chi_P in units of h; INFINITY = dense P          */
  double tol;               /* GMRES relative preconditioned residual           */
  int32_t restart;          /* GMRES restart (paper: 200)                       */
  int32_t maxit;            /* iteration cap                                    */
  int32_t refine;           /* FP32 path: outer FP64 iterative refinement steps */
  int32_t rhs_mode;         /* 0 = total traces (A^e + A^i) u = u^inc; 1 = the
                               paper's scattered traces (eq.
                               PMCHWT_multiple_scatterers): (A^e + A^i) u^s =
                               (1/2 I - D^i) u^inc, D^i = diag(A^i_m) applied to
                               the L2 projection of u^inc onto RWG (mass matrix
                               int phi_i.phi_j, loads int phi_i.(field x n)); the
                               solution holds u^s, with the same far field        */
  int32_t matrix_free;      /* 1: A is not stored; its regular pairs are
                               recomputed in every application (only the
                               touching-pair entries are kept, sparse)          */
  double aca_nu_P;          /* > 0: P's blocks as H-matrices (Section 3.3):
                               admissible leaves (disjoint support boxes)
                               within chi_P = near_cutoff_P * h of each other by
                               ACA to this tolerance, the others dropped,
                               inadmissible leaves dense (the block-level reading
                               of eq. nf_condition); 0: dense or entry-level
                               near-field P                                     */
  int32_t discretisation;   /* 0: eq. RWG_discretisation1 (RWG for A, BC for P);
                               1: the mixed discretisation of eq.
                               mixed_discretisation: each scatterer's traces in
                               (RWG_m, BC_m) for trial and test alike, RWG
                               written on the barycentric refinement for the
                               blocks C(RWG, BC), C(BC, RWG); P = D reuses A's
                               diagonal blocks; float64 (CAL_FP64) only, precond
                               CAL_PRECOND_D, total-trace right-hand side       */
} cal_solve_opts;
void cal_solve_opts_default(cal_solve_opts* opts);

typedef struct {
  int32_t iterations;       /* GMRES iterations (sum over refinement steps)     */
  int32_t converged;
  int64_t matvecs;          /* boundary-operator applications, Table tab:matvecs */
  double residual;          /* final relative preconditioned residual           */
  double t_setup, t_assemble_A, t_assemble_P, t_solve;  /* seconds: host time of the
                            spaces (the BC space is built while A is assembled), device time of
                            A's and P's assembly, wall time of the solve                       */
  int64_t bytes_A, bytes_P; /* device bytes of the stored operators (with the
                               combined float32 blocks of the one-vector product) */
  int64_t n_unknowns;       /* 2N                                               */
} cal_solve_info;

/* Solves for nrhs incident plane waves inc [nrhs][6] = (direction, polarisation),
   E^inc = p e^{i k_ext d.x}; eps_r, mu_r [M][2] (re, im) per scatterer (mu_r may
   be NULL for 1). The returned solution keeps the total boundary traces on the
   device. Returns CAL_ENOTCONV (with a usable solution) if maxit was reached. */
int cal_pmchwt_solve(cal_ctx* ctx, cal_mesh* mesh, double k_ext, const double* eps_r,
                     const double* mu_r, const double* inc, int64_t nrhs,
                     const cal_solve_opts* opts, cal_solution** out);
int cal_solution_get_info(const cal_solution* sol, cal_solve_info* info);
/* Coefficients x [nrhs][2N] complex128 to host memory (component-major, see top). */
int cal_solution_coefficients(const cal_solution* sol, double* dst_host);
/* Far-field pattern E_inf(x_hat), E^s ~ E_inf e^{ik r}/r, for unit directions
   dirs [ndir][3]: out [nrhs][ndir][3] complex128 (host). */
int cal_farfield(const cal_solution* sol, const double* dirs, int64_t ndir, double* out);
/* Total electric field at points off the surface (the |E|^2 maps of Section 5),
   from the Stratton–Chu representations (eqs. StrattonChu_int, StrattonChu_ext)
   with the potential operators E_k, H_k of Section 2:
     exterior:       E = E^inc - [H_ke(u_1) + E_ke((mu_e/k_e) u_2)] over all surfaces,
     inside Gamma_m: E = H_km(u_1) + E_km((mu_m/k_m) u_2) over Gamma_m,
   with the solution's total traces (a scattered-trace solution, rhs_mode 1,
   adds the L2 projection of u^inc it was built from). points [npt][3];
   levels 0..4: each triangle is split into 4^levels congruent sub-triangles
   with the 6-point rule on each (points should stay a few sub-triangle sizes
   away from the surface); region_in [npt] (-1 exterior, m inside Gamma_m) or
   NULL to take each point's region from the winding numbers of the closed
   meshes; region_out [npt] (may be NULL) receives the regions used.
   out [nrhs][npt][3] complex128 (host). Evaluated in float32 for float32-bulk
   solutions, float64 for CAL_FP64 ones. */
int cal_near_field(const cal_solution* sol, const double* points, int64_t npt, int levels,
                   const int32_t* region_in, int32_t* region_out, double* out);
void cal_solution_destroy(cal_solution* sol);

/* ---- resident problems --------------------------------------------------- */
/* cal_pmchwt_solve is cal_problem_create + cal_problem_solve +
   cal_problem_destroy. A problem keeps everything that depends only on
   (mesh, k_ext, materials, options) on the device: the spaces, the stored A
   blocks (eq. multiple_operator), the P blocks (§3.1) and the Gram matrices
   (eqs. MassA, MassP), so that further incident fields (the orientation
   averages of §5) cost only GMRES. The mesh may be destroyed once create has
   returned. Solves of one problem must not overlap in time; any context on the
   problem's device may run them (the work goes on that context's stream). */
int cal_problem_create(cal_ctx* ctx, cal_mesh* mesh, double k_ext, const double* eps_r,
                       const double* mu_r, const cal_solve_opts* opts, cal_problem** out);
/* Same contract and result as cal_pmchwt_solve for the problem's operators;
   info.t_setup/t_assemble_* are the problem's creation times. `solver` (may be
   NULL: the options given at creation) supplies tol, restart, maxit and refine
   for this solve; its assembly fields are ignored. */
int cal_problem_solve(cal_ctx* ctx, cal_problem* prob, const double* inc, int64_t nrhs,
                      const cal_solve_opts* solver, cal_solution** out);
typedef struct {
  int64_t n_unknowns;                 /* 2N                                        */
  int32_t n_scatterers, precision, precond;
  int64_t bytes_A, bytes_P, bytes_G;  /* stored blocks (with the combined float32
                                         blocks) and Gram CSR (device bytes)      */
  int64_t bytes_batch;                /* work vectors and Gram-solver state kept for
                                         the last batch width (0 before a solve)  */
  int32_t batch_width;                /* right-hand sides per lockstep batch       */
  double t_setup, t_assemble_A, t_assemble_P;
} cal_problem_info;
/* y = A x with the problem's PMCHWT operator A (eqs. multiple_operator,
   AimAem: the exterior blocks on the union plus each scatterer's interior
   blocks), stored or matrix-free as it was created; x, y [nrhs][2N] complex128
   host arrays in the unknown ordering above. Vectors are applied in float64
   (the operator's entries keep the problem's precision). */
int cal_problem_apply(cal_ctx* ctx, cal_problem* prob, const double* x, double* y, int64_t nrhs);
int cal_problem_get_info(const cal_problem* prob, cal_problem_info* info);
void cal_problem_destroy(cal_problem* prob);

/* ---- request queue (serving loop) ------------------------------------------
   Continuous batching of scattering solves: requests of different meshes,
   wavenumbers, materials and incident fields are submitted at any time and
   run on `slots` worker streams of one device, so their GPU work overlaps.
   Admission is by HBM footprint: a request starts once its estimated bytes
   (stored A and P blocks, Gram matrices, Krylov basis and vectors; reconciled
   with the real sizes once its operators exist) fit in the budget next to what
   is running and resident. Operators stay resident after a solve (LRU, evicted
   when admission needs the room), so a later request of the same problem
   (same mesh, k_ext, materials and assembly options) goes straight to GMRES,
   and pending requests of one problem with equal solver options are merged
   into one lockstep multi-right-hand-side batch (up to 32 columns). The paper
   motivates many solves of one scatterer by orientation averaging (§5). */
typedef struct {
  const double* verts; int64_t nv;     /* as cal_mesh_create                     */
  const int32_t* tris; int64_t nt;
  const int32_t* domain;               /* may be NULL (one scatterer)            */
  double k_ext;
  const double* eps_r;                 /* [M][2]                                 */
  const double* mu_r;                  /* [M][2] or NULL                         */
  const double* inc; int64_t nrhs;     /* [nrhs][6] as cal_pmchwt_solve          */
  const double* dirs; int64_t ndir;    /* far-field directions [ndir][3]         */
  cal_solve_opts opts;
} cal_request;

typedef struct {
  int32_t status;        /* the request's own result: CAL_OK, CAL_ENOTCONV (far
                            field still valid), or the error of its solve      */
  int32_t iterations;
  double residual;
  double t_submit, t_start, t_done;  /* seconds on the queue's clock; latency =
                                        t_done - t_submit (far field ready)     */
  int64_t footprint_bytes;           /* bytes reserved at admission             */
  int32_t batch_rhs;                 /* columns of the lockstep batch it ran in */
  int32_t reused;                    /* 1: operators were already resident      */
} cal_request_result;

typedef struct {
  int64_t submitted, completed, rejected;
  int64_t batches;            /* problem solves run (a merged batch counts once)   */
  int64_t merged;             /* requests that joined another request's batch     */
  int64_t problems_created, problem_hits, evictions;
  int64_t budget_bytes, reserved_bytes, peak_reserved_bytes;
  int32_t slots, running, peak_running, pending;
} cal_queue_stats;

/* One queue per device; hbm_budget_bytes = 0 takes 85% of the free device
   memory at creation. slots >= 1 worker threads, each with its own context
   and stream. */
int cal_queue_create(int device, size_t hbm_budget_bytes, int slots, cal_queue** out);
/* Copies every input (the caller's arrays may be reused at once), checks the
   mesh (CAL_EMESH) and the footprint: CAL_ENOMEM if the request alone cannot
   fit the budget. On success *ticket identifies the request. */
int cal_queue_submit(cal_queue* q, const cal_request* req, int64_t* ticket);
/* Waits up to timeout_s seconds (< 0: no limit) for the request. CAL_OK when it
   has completed (its own status in res->status; farfield, if not NULL, receives
   [nrhs][ndir][3] complex128) and the ticket is released; CAL_ETIMEOUT if it
   is still pending or running; CAL_EINVAL for an unknown ticket. */
int cal_queue_wait(cal_queue* q, int64_t ticket, double timeout_s, cal_request_result* res,
                   double* farfield);
/* Request states of cal_queue_poll */
#define CAL_REQ_PENDING 0  /* queued: not yet admitted (waits for HBM budget or a slot) */
#define CAL_REQ_RUNNING 1  /* admitted: its batch is being assembled or solved        */
#define CAL_REQ_DONE    2  /* finished: cal_queue_wait returns at once                */
/* Non-blocking: *state = CAL_REQ_PENDING, CAL_REQ_RUNNING or CAL_REQ_DONE. The
   ticket stays valid (only cal_queue_wait releases it); CAL_EINVAL for an
   unknown or already released ticket. */
int cal_queue_poll(cal_queue* q, int64_t ticket, int* state);
int cal_queue_get_stats(cal_queue* q, cal_queue_stats* stats);
/* Finishes the batches that are running, drops pending requests, frees the
   resident operators and the worker contexts. */
void cal_queue_destroy(cal_queue* q);
/* Estimated device bytes of a request (host only, no GPU needed): the
   resident part (spaces, A, P, Gram) and the per-solve part. */
int cal_request_footprint(const cal_request* req, int64_t* resident_bytes, int64_t* solve_bytes);

/* ---- instrumentation ------------------------------------------------------ */
/* The paper has no counterpart: a check of the double-precision e^{i x} and
   e^{-|x|} that the singular-pair kernel evaluates itself (Cody–Waite
   reduction, Taylor series), against the CUDA library's sincos and exp, on n
   points evenly spread over [lo, hi] on the current device. Writes the max
   absolute error of (cos, sin) and the max relative error of exp. */
int cal_check_elementary(int64_t n, double lo, double hi, double* err_cis, double* err_exp);
/* The paper has no counterpart: a check of the bounded grid-wide barrier of
   the Gram solver's cooperative kernel, on ctx's device. Four blocks pass
   three barriers; when skip_block is in [0, 4) that block leaves before the
   first one, so the others give up after their bounded wait (about a second
   or two) and report it. *status = 0 when every block passed every barrier,
   1 when a wait gave up. Returns CAL_OK unless the launch or a copy failed;
   the context stays usable either way. */
int cal_check_grid_barrier(cal_ctx* ctx, int skip_block, int* status);
/* Number of kernels this library has launched since load (all contexts). */
int64_t cal_kernel_launches(void);
/* on != 0: bracket every assembly kernel launch with CUDA events on its own
   stream; off clears the records. */
int cal_profile_enable(int on);
/* Sum over recorded launches of kernel family `name` ("rwg_regular",
   "bc_tile", "singular", "gram", "pair_gemv", "bicgstab"): launches,
   total device milliseconds, and algorithmic work units (point-pair
   integrand evaluations for assembly kernels, matrix bytes for GEMVs).
   Waits for the recorded events. */
int cal_profile_read(const char* name, int64_t* launches, double* total_ms, double* units);

#ifdef __cplusplus
}
#endif
#endif /* CAL_H */
