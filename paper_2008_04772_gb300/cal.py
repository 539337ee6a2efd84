"""Thin ctypes binding of the C ABI in include/cal.h (argument marshalling only).

Every computation happens in libcal.so; this module converts numpy arrays to
pointers, checks return codes and turns them into exceptions. Importing it
does not load the library; the first call does, and fails loudly when the
library has not been built (``python -m paper_2008_04772_gb300.build``).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcal.so")

# constants of include/cal.h
OK, EINVAL, EMESH, ENOMEM, ENOTCONV, ETIMEOUT, ECUDA = 0, -1, -2, -3, -4, -5, -6
RWG, BC = 1, 2
OP_S, OP_C = 1, 2
FP64, FP32, FP32_ALL = 1, 2, 3
DENSE, CSR, HMAT = 1, 2, 3
PRECOND = {"none": 0, "D": 1, "De": 2, "Di": 3, "Se": 4, "Si": 5}
REQ_PENDING, REQ_RUNNING, REQ_DONE = 0, 1, 2

_lib = None


class CalError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cal error {code}: {msg}")
        self.code = code


class MeshInfo(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("n_edges", ctypes.c_int64), ("n_scatterers", ctypes.c_int64),
                ("h", ctypes.c_double), ("max_valence", ctypes.c_int32)]


class OpInfo(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("format", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("op_mask", ctypes.c_int32), ("row_offset", ctypes.c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("precond", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("q_regular_A", ctypes.c_int32), ("q_singular_A", ctypes.c_int32),
                ("q_regular_P", ctypes.c_int32), ("q_singular_P", ctypes.c_int32),
                ("near_cutoff_P", ctypes.c_double), ("tol", ctypes.c_double),
                ("restart", ctypes.c_int32), ("maxit", ctypes.c_int32),
                ("refine", ctypes.c_int32), ("rhs_mode", ctypes.c_int32),
                ("matrix_free", ctypes.c_int32), ("aca_nu_P", ctypes.c_double),
                ("discretisation", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("matvecs", ctypes.c_int64), ("residual", ctypes.c_double),
                ("t_setup", ctypes.c_double), ("t_assemble_A", ctypes.c_double),
                ("t_assemble_P", ctypes.c_double), ("t_solve", ctypes.c_double),
                ("bytes_A", ctypes.c_int64), ("bytes_P", ctypes.c_int64),
                ("n_unknowns", ctypes.c_int64)]


class ProblemInfo(ctypes.Structure):
    _fields_ = [("n_unknowns", ctypes.c_int64), ("n_scatterers", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("bytes_A", ctypes.c_int64), ("bytes_P", ctypes.c_int64), ("bytes_G", ctypes.c_int64),
                ("bytes_batch", ctypes.c_int64), ("batch_width", ctypes.c_int32),
                ("t_setup", ctypes.c_double), ("t_assemble_A", ctypes.c_double),
                ("t_assemble_P", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("nv", ctypes.c_int64),
                ("tris", ctypes.c_void_p), ("nt", ctypes.c_int64),
                ("domain", ctypes.c_void_p), ("k_ext", ctypes.c_double),
                ("eps_r", ctypes.c_void_p), ("mu_r", ctypes.c_void_p),
                ("inc", ctypes.c_void_p), ("nrhs", ctypes.c_int64),
                ("dirs", ctypes.c_void_p), ("ndir", ctypes.c_int64),
                ("opts", SolveOpts)]


class RequestResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("residual", ctypes.c_double), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("footprint_bytes", ctypes.c_int64), ("batch_rhs", ctypes.c_int32),
                ("reused", ctypes.c_int32)]


class QueueStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("merged", ctypes.c_int64), ("problems_created", ctypes.c_int64),
                ("problem_hits", ctypes.c_int64), ("evictions", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64), ("reserved_bytes", ctypes.c_int64),
                ("peak_reserved_bytes", ctypes.c_int64), ("slots", ctypes.c_int32),
                ("running", ctypes.c_int32), ("peak_running", ctypes.c_int32),
                ("pending", ctypes.c_int32)]


def declared_symbols(header=None):
    """Function names declared in include/cal.h."""
    import re
    header = header or os.path.join(os.path.dirname(_HERE), "include", "cal.h")
    text = open(header).read()
    return sorted(set(re.findall(r"\b(cal_[a-z_0-9]+)\s*\(", text)))


def lib():
    """Load libcal.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2008_04772_gb300.build` (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "cal_init": ([ctypes.POINTER(P), ctypes.c_int], ctypes.c_int),
        "cal_ctx_destroy": ([P], None),
        "cal_last_error": ([], ctypes.c_char_p),
        "cal_ctx_stream": ([P], P),
        "cal_mesh_create": ([P, P, i64, P, i64, P, ctypes.POINTER(P)], ctypes.c_int),
        "cal_mesh_destroy": ([P], None),
        "cal_mesh_get_info": ([P, ctypes.POINTER(MeshInfo)], ctypes.c_int),
        "cal_space_create": ([P, ctypes.c_int, ctypes.POINTER(P)], ctypes.c_int),
        "cal_space_destroy": ([P], None),
        "cal_assemble": ([P, ctypes.c_int, d, d, P, P, ctypes.c_int, d, ctypes.c_int, ctypes.c_int,
                          ctypes.c_int, ctypes.POINTER(P)], ctypes.c_int),
        "cal_op_destroy": ([P], None),
        "cal_op_get_info": ([P, ctypes.POINTER(OpInfo)], ctypes.c_int),
        "cal_op_export": ([P, ctypes.c_int, P, P, P], ctypes.c_int),
        "cal_matvec": ([P, ctypes.c_int, P, P, i64, P], ctypes.c_int),
        "cal_matvec_static": ([P, ctypes.c_int, P, P, i64, P], ctypes.c_int),
        "cal_near_field": ([P, P, i64, ctypes.c_int, P, P, P], ctypes.c_int),
        "cal_op_compress": ([P, P, P, ctypes.c_double, ctypes.c_double, P], ctypes.c_int),
        "cal_gram_export": ([P, P, P], ctypes.c_int),
        "cal_solve_opts_default": ([ctypes.POINTER(SolveOpts)], None),
        "cal_pmchwt_solve": ([P, P, d, P, P, P, i64, ctypes.POINTER(SolveOpts), ctypes.POINTER(P)],
                             ctypes.c_int),
        "cal_solution_get_info": ([P, ctypes.POINTER(SolveInfo)], ctypes.c_int),
        "cal_solution_coefficients": ([P, P], ctypes.c_int),
        "cal_farfield": ([P, P, i64, P], ctypes.c_int),
        "cal_solution_destroy": ([P], None),
        "cal_problem_create": ([P, P, d, P, P, ctypes.POINTER(SolveOpts), ctypes.POINTER(P)], ctypes.c_int),
        "cal_problem_solve": ([P, P, P, i64, ctypes.POINTER(SolveOpts), ctypes.POINTER(P)], ctypes.c_int),
        "cal_problem_get_info": ([P, ctypes.POINTER(ProblemInfo)], ctypes.c_int),
        "cal_problem_apply": ([P, P, P, P, i64], ctypes.c_int),
        "cal_problem_destroy": ([P], None),
        "cal_queue_create": ([ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(P)], ctypes.c_int),
        "cal_queue_submit": ([P, ctypes.POINTER(Request), ctypes.POINTER(i64)], ctypes.c_int),
        "cal_queue_wait": ([P, i64, d, ctypes.POINTER(RequestResult), P], ctypes.c_int),
        "cal_queue_poll": ([P, i64, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cal_queue_get_stats": ([P, ctypes.POINTER(QueueStats)], ctypes.c_int),
        "cal_queue_destroy": ([P], None),
        "cal_request_footprint": ([ctypes.POINTER(Request), ctypes.POINTER(i64), ctypes.POINTER(i64)],
                                  ctypes.c_int),
        "cal_kernel_launches": ([], i64),
        "cal_check_elementary": ([i64, d, d, ctypes.POINTER(d), ctypes.POINTER(d)], ctypes.c_int),
        "cal_check_grid_barrier": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cal_profile_enable": ([ctypes.c_int], ctypes.c_int),
        "cal_profile_read": ([ctypes.c_char_p, ctypes.POINTER(i64), ctypes.POINTER(d),
                              ctypes.POINTER(d)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(rc, allow=()):
    if rc != OK and rc not in allow:
        raise CalError(rc, lib().cal_last_error().decode())
    return rc


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class Context:
    def __init__(self, device: int = 0):
        self.h = ctypes.c_void_p()
        _check(lib().cal_init(ctypes.byref(self.h), device))

    @property
    def stream(self):
        return lib().cal_ctx_stream(self.h)

    def check_grid_barrier(self, skip_block: int = -1) -> int:
        """Bounded grid-barrier check (cal_check_grid_barrier): 0 when every
        block passed, 1 when a wait gave up (skip_block in 0..3 makes one block
        leave early)."""
        st = ctypes.c_int(-1)
        _check(lib().cal_check_grid_barrier(self.h, skip_block, ctypes.byref(st)))
        return st.value

    def close(self):
        if self.h:
            lib().cal_ctx_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    def __init__(self, ctx: Context, verts, tris, domain=None):
        self.ctx = ctx
        v = np.ascontiguousarray(verts, dtype=np.float64)
        t = np.ascontiguousarray(tris, dtype=np.int32)
        dm = None if domain is None else np.ascontiguousarray(domain, dtype=np.int32)
        self.h = ctypes.c_void_p()
        _check(lib().cal_mesh_create(ctx.h, _ptr(v), len(v), _ptr(t), len(t), _ptr(dm),
                                     ctypes.byref(self.h)))

    def info(self) -> MeshInfo:
        out = MeshInfo()
        _check(lib().cal_mesh_get_info(self.h, ctypes.byref(out)))
        return out

    def __del__(self):
        if getattr(self, "h", None):
            lib().cal_mesh_destroy(self.h)


class Space:
    def __init__(self, mesh: Mesh, kind: int):
        self.mesh = mesh
        self.kind = kind
        self.h = ctypes.c_void_p()
        _check(lib().cal_space_create(mesh.h, kind, ctypes.byref(self.h)))

    def __del__(self):
        if getattr(self, "h", None):
            lib().cal_space_destroy(self.h)


class Operator:
    def __init__(self, h, ctx=None):
        self.h = h
        self.ctx = ctx  # keeps the context alive while the operator is

    def info(self) -> OpInfo:
        out = OpInfo()
        _check(lib().cal_op_get_info(self.h, ctypes.byref(out)))
        return out

    def export(self, which: int):
        """Dense [rows, cols] complex array, or (values, row_ptr, col_idx) for CSR."""
        inf = self.info()
        dt = np.complex64 if inf.precision == FP32 else np.complex128
        if inf.format == HMAT:  # expanded densely
            vals = np.zeros(inf.rows * inf.cols, dtype=dt)
            _check(lib().cal_op_export(self.h, which, _ptr(vals), None, None))
            return vals.reshape(inf.rows, inf.cols)
        vals = np.zeros(inf.nnz, dtype=dt)
        if inf.format == DENSE:
            _check(lib().cal_op_export(self.h, which, _ptr(vals), None, None))
            return vals.reshape(inf.rows, inf.cols)
        rp = np.zeros(inf.rows + 1, dtype=np.int64)
        ci = np.zeros(max(inf.nnz, 1), dtype=np.int64)
        _check(lib().cal_op_export(self.h, which, _ptr(vals), _ptr(rp), _ptr(ci)))
        return vals, rp, ci[:inf.nnz]

    def matvec(self, which: int, x_ptr: int, y_ptr: int, nrhs: int = 1, stream=None):
        """y = X x on device pointers (e.g. torch CUDA tensors' data_ptr())."""
        _check(lib().cal_matvec(self.h, which, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr),
                                nrhs, stream))

    def matvec_static(self, which: int, x_ptr: int, y_ptr: int, nrhs: int = 1, stream=None):
        """y = X x like matvec's tensor-core branch, with no device allocation:
        the temporaries live in one fixed per-device array shared by all calls."""
        _check(lib().cal_matvec_static(self.h, which, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr),
                                       nrhs, stream))

    def __del__(self):
        if getattr(self, "h", None):
            lib().cal_op_destroy(self.h)


def compress(ctx: Context, op: Operator, space: Space, nu: float, chi: float = math.inf) -> Operator:
    """H-matrix form of a dense square operator (ACA to nu, admissible leaves
    within chi kept)."""
    h = ctypes.c_void_p()
    _check(lib().cal_op_compress(ctx.h, op.h, space.h, float(nu), float(chi), ctypes.byref(h)))
    return Operator(h, ctx)


def assemble(ctx: Context, op_mask: int, k: complex, space: Space, scatterer: int = -1,
             near_cutoff: float = math.inf, q_regular: int = 6, q_singular: int = 4,
             precision: int = FP64) -> Operator:
    h = ctypes.c_void_p()
    k = complex(k)
    _check(lib().cal_assemble(ctx.h, op_mask, k.real, k.imag, space.h, space.h, scatterer,
                              near_cutoff, q_regular, q_singular, precision, ctypes.byref(h)))
    return Operator(h, ctx)


def gram(rwg: Space, bc: Space):
    n = rwg.mesh.info().n_edges
    out = np.zeros((n, n), dtype=np.float64)
    _check(lib().cal_gram_export(rwg.h, bc.h, _ptr(out)))
    return out


def solve_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib().cal_solve_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precond" and isinstance(v, str):
            v = PRECOND[v]
        setattr(o, k, v)
    return o


class Solution:
    def __init__(self, h, nrhs, n_edges, rc, ctx=None):
        self.h = h
        self.ctx = ctx
        self.nrhs = nrhs
        self.n_edges = n_edges
        self.rc = rc

    def info(self) -> SolveInfo:
        out = SolveInfo()
        _check(lib().cal_solution_get_info(self.h, ctypes.byref(out)))
        return out

    def coefficients(self):
        out = np.zeros((self.nrhs, 2 * self.n_edges), dtype=np.complex128)
        _check(lib().cal_solution_coefficients(self.h, _ptr(out)))
        return out

    def far_field(self, dirs):
        d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
        out = np.zeros((self.nrhs, len(d), 3), dtype=np.complex128)
        _check(lib().cal_farfield(self.h, _ptr(d), len(d), _ptr(out)))
        return out

    def near_field(self, points, levels: int = 2, region=None):
        """Total E at points off the surface: ([nrhs][npt][3] complex, regions [npt])."""
        p = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
        out = np.zeros((self.nrhs, len(p), 3), dtype=np.complex128)
        reg_out = np.zeros(len(p), dtype=np.int32)
        reg_in = None if region is None else np.ascontiguousarray(region, dtype=np.int32)
        _check(lib().cal_near_field(self.h, _ptr(p), len(p), int(levels),
                                    None if reg_in is None else _ptr(reg_in), _ptr(reg_out), _ptr(out)))
        return out, reg_out

    def __del__(self):
        if getattr(self, "h", None):
            lib().cal_solution_destroy(self.h)


def _materials(M, eps_r, mu_r):
    """(re, im) arrays [M][2] for eps_r and mu_r (a scalar applies to every scatterer)."""
    e = np.asarray(eps_r, dtype=np.complex128).reshape(-1)
    if len(e) == 1:
        e = np.repeat(e, M)
    ea = np.ascontiguousarray(np.stack([e.real, e.imag], 1))
    ma = None
    if mu_r is not None:
        mu = np.asarray(mu_r, dtype=np.complex128).reshape(-1)
        if len(mu) == 1:
            mu = np.repeat(mu, M)
        ma = np.ascontiguousarray(np.stack([mu.real, mu.imag], 1))
    return ea, ma


def pmchwt_solve(ctx: Context, mesh: Mesh, k_ext: float, eps_r, inc, mu_r=None,
                 opts: SolveOpts | None = None, allow_not_converged: bool = False) -> Solution:
    ea, ma = _materials(mesh.info().n_scatterers, eps_r, mu_r)
    inc = np.ascontiguousarray(np.atleast_2d(inc), dtype=np.float64)
    h = ctypes.c_void_p()
    o = opts or solve_opts()
    rc = lib().cal_pmchwt_solve(ctx.h, mesh.h, float(k_ext), _ptr(ea), _ptr(ma), _ptr(inc),
                                len(inc), ctypes.byref(o), ctypes.byref(h))
    _check(rc, allow=(ENOTCONV,) if allow_not_converged else ())
    return Solution(h, len(inc), mesh.info().n_edges, rc, ctx)


class Problem:
    """Assembled operators of one (mesh, k_ext, materials, options), resident on the device."""

    def __init__(self, ctx: Context, mesh: Mesh, k_ext: float, eps_r, mu_r=None,
                 opts: SolveOpts | None = None):
        ea, ma = _materials(mesh.info().n_scatterers, eps_r, mu_r)
        self.ctx = ctx
        self.n_edges = mesh.info().n_edges
        self.h = ctypes.c_void_p()
        o = opts or solve_opts()
        _check(lib().cal_problem_create(ctx.h, mesh.h, float(k_ext), _ptr(ea), _ptr(ma), ctypes.byref(o),
                                        ctypes.byref(self.h)))

    def info(self) -> ProblemInfo:
        out = ProblemInfo()
        _check(lib().cal_problem_get_info(self.h, ctypes.byref(out)))
        return out

    def solve(self, inc, ctx: Context | None = None, solver: SolveOpts | None = None,
              allow_not_converged: bool = False) -> Solution:
        """solver: tol/restart/maxit/refine for this solve (None: those given at creation)."""
        c = ctx or self.ctx
        inc = np.ascontiguousarray(np.atleast_2d(inc), dtype=np.float64)
        h = ctypes.c_void_p()
        rc = lib().cal_problem_solve(c.h, self.h, _ptr(inc), len(inc),
                                     ctypes.byref(solver) if solver is not None else None, ctypes.byref(h))
        _check(rc, allow=(ENOTCONV,) if allow_not_converged else ())
        return Solution(h, len(inc), self.n_edges, rc, c)

    def apply(self, x, ctx: Context | None = None):
        """y = A x for x [nrhs][2N] complex (the PMCHWT operator of the problem)."""
        c = ctx or self.ctx
        xx = np.ascontiguousarray(np.atleast_2d(x), dtype=np.complex128)
        y = np.zeros_like(xx)
        _check(lib().cal_problem_apply(c.h, self.h, _ptr(xx), _ptr(y), len(xx)))
        return y

    def __del__(self):
        if getattr(self, "h", None):
            lib().cal_problem_destroy(self.h)


def make_request(verts, tris, domain, k_ext, eps_r, inc, dirs, mu_r=None, opts: SolveOpts | None = None):
    """A cal_request and the arrays it points to (keep both alive until submitted)."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    dm = None if domain is None else np.ascontiguousarray(domain, dtype=np.int32)
    M = 1 if dm is None else int(dm.max()) + 1
    ea, ma = _materials(M, eps_r, mu_r)
    inc = np.ascontiguousarray(np.atleast_2d(inc), dtype=np.float64)
    d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    r = Request()
    r.verts, r.nv = v.ctypes.data, len(v)
    r.tris, r.nt = t.ctypes.data, len(t)
    r.domain = None if dm is None else dm.ctypes.data
    r.k_ext = float(k_ext)
    r.eps_r = ea.ctypes.data
    r.mu_r = None if ma is None else ma.ctypes.data
    r.inc, r.nrhs = inc.ctypes.data, len(inc)
    r.dirs, r.ndir = d.ctypes.data, len(d)
    r.opts = opts or solve_opts()
    return r, (v, t, dm, ea, ma, inc, d)


def request_footprint(req: Request):
    """(resident bytes, per-solve bytes) the queue reserves for a request (host only)."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().cal_request_footprint(ctypes.byref(req), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


class Queue:
    """Serving loop: continuous batching of solve requests on one device."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, slots: int = 4):
        self.h = ctypes.c_void_p()
        _check(lib().cal_queue_create(device, budget_bytes, slots, ctypes.byref(self.h)))
        self._shape = {}

    def submit(self, verts, tris, domain, k_ext, eps_r, inc, dirs, mu_r=None,
               opts: SolveOpts | None = None) -> int:
        r, keep = make_request(verts, tris, domain, k_ext, eps_r, inc, dirs, mu_r, opts)
        t = ctypes.c_int64()
        _check(lib().cal_queue_submit(self.h, ctypes.byref(r), ctypes.byref(t)))
        del keep  # the queue copied every input
        self._shape[t.value] = (r.nrhs, r.ndir)
        return t.value

    def wait(self, ticket: int, timeout: float = -1.0):
        """(RequestResult, far field [nrhs][ndir][3] complex128 or None if it failed)."""
        nrhs, ndir = self._shape.get(ticket, (0, 0))
        res = RequestResult()
        far = np.zeros((nrhs, ndir, 3), dtype=np.complex128) if nrhs else None
        _check(lib().cal_queue_wait(self.h, ticket, float(timeout), ctypes.byref(res), _ptr(far)))
        self._shape.pop(ticket, None)
        ok = res.status in (OK, ENOTCONV)
        return res, (far if ok else None)

    def poll(self, ticket: int) -> int:
        """REQ_PENDING, REQ_RUNNING or REQ_DONE, without waiting."""
        st = ctypes.c_int()
        _check(lib().cal_queue_poll(self.h, ticket, ctypes.byref(st)))
        return st.value

    def stats(self) -> QueueStats:
        out = QueueStats()
        _check(lib().cal_queue_get_stats(self.h, ctypes.byref(out)))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().cal_queue_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        self.close()
