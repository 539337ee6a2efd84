"""Dense Galerkin assembly of S and C on RWG / BC spaces (test infrastructure).

Section 3.2-3.3 of the paper. A Galerkin entry between basis functions
phi_i = sum beta f_{tau1,a} and phi_j = sum beta' f_{tau2,b} is
sum beta beta' L(tau1, tau2)[a, b], with L the local blocks of
``orc_bem.c``; in matrix form  M = B_test L B_trial^T  (a library matmul).

Near-field cutoff chi (eq. nf_condition): the paper applies it to
admissible cluster blocks of an H-matrix; reading taken here, at entry
level: entry (i, j) is kept iff the bounding boxes of the supports of phi_i
and phi_j are at most chi apart; kept entries are computed completely.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

from .quadrature import CLASS_BOUNDS, CLASS_POINTS, gauss_legendre_01, triangle_rule
from .spaces import aabb_distance

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = None


def build(force: bool = False) -> str:
    """Compile orc_bem.c with gcc -O2 -fopenmp into oracle/_lib/liborc.so."""
    os.makedirs(_LIBDIR, exist_ok=True)
    src = os.path.join(_HERE, "orc_bem.c")
    out = os.path.join(_LIBDIR, "liborc.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu99",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


def lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(build())
        d, l, i = ctypes.c_double, ctypes.c_long, ctypes.c_int
        P = ctypes.c_void_p
        _LIB.orc_blocks.argtypes = [P, P, P, l, P, l, d, d, i, P, P, P, d, d, i, P, P, P, P, P]
        _LIB.orc_blocks.restype = None
        _LIB.orc_ss_polynomial.argtypes = [P, P, i, P, P, P, P, i, P, P]
        _LIB.orc_ss_polynomial.restype = d
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Rules:
    """Quadrature choice: regular points per triangle and Gauss points per dimension.

    n_regular = 6 or 1: that rule for every regular pair. n_regular = 0: the
    near / medium / far classes with 6 / 4 / 3 points (orders 4 / 3 / 2, the
    paper's defaults), bounds in ``quadrature.CLASS_BOUNDS``.
    """

    def __init__(self, n_regular: int = 6, n_gauss: int = 4):
        self.n_regular = n_regular
        self.n_gauss = n_gauss
        pts = CLASS_POINTS if n_regular == 0 else (n_regular,) * 3
        rules = [triangle_rule(n) for n in pts]
        self.class_points = np.array(pts, dtype=np.int32)
        self.class_rb = np.concatenate([r[0].reshape(-1) for r in rules])
        self.class_rw = np.concatenate([r[1] for r in rules])
        self.bounds = CLASS_BOUNDS
        self.rb, self.rw = rules[0]
        self.gx, self.gw = gauss_legendre_01(n_gauss)


def local_blocks(X, ids, test, trial, k, rules: Rules, want=3, counts=None):
    """Local 3x3 blocks of S and C: two complex arrays [n1, n2, 3, 3]."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    test = np.ascontiguousarray(test, dtype=np.int64)
    trial = np.ascontiguousarray(trial, dtype=np.int64)
    n1, n2 = len(test), len(trial)
    S = np.zeros((n1, n2, 3, 3), dtype=np.complex128)
    C = np.zeros((n1, n2, 3, 3), dtype=np.complex128)
    npts = np.ascontiguousarray(rules.class_points, dtype=np.int32)
    rb = np.ascontiguousarray(rules.class_rb, dtype=np.float64)
    rw = np.ascontiguousarray(rules.class_rw, dtype=np.float64)
    gx = np.ascontiguousarray(rules.gx, dtype=np.float64)
    gw = np.ascontiguousarray(rules.gw, dtype=np.float64)
    cnt = np.zeros(4, dtype=np.int64)
    k = complex(k)
    lib().orc_blocks(_ptr(X), _ptr(ids), _ptr(test), n1, _ptr(trial), n2, k.real, k.imag,
                     int(want), _ptr(npts), _ptr(rb), _ptr(rw), rules.bounds[0], rules.bounds[1],
                     rules.n_gauss, _ptr(gx), _ptr(gw), _ptr(S), _ptr(C), _ptr(cnt))
    if counts is not None:
        counts += cnt
    return S, C


def _space_tri_arrays(space):
    """Vertex coordinate array and triangle ids of the triangle set of a space."""
    # tri_xyz is [n, 3, 3]; build a flat vertex table indexed by the global ids
    ids = space.tri_ids
    nid = int(ids.max()) + 1
    X = np.zeros((nid, 3))
    X[ids.reshape(-1)] = space.tri_xyz.reshape(-1, 3)
    return X, ids


def assemble(test_space, trial_space, k, rules: Rules, want=3, rows=None, cols=None,
             counts=None, max_block_entries=2e7):
    """Dense S and C Galerkin matrices restricted to test ``rows`` x trial ``cols``.

    Returns (S, C), complex [n_rows, n_cols]. Test and trial spaces must live
    on the same triangle set (both primal or both barycentric).
    """
    X, ids = _space_tri_arrays(trial_space)
    rows = np.arange(test_space.N) if rows is None else np.asarray(rows)
    cols = np.arange(trial_space.N) if cols is None else np.asarray(cols)
    Brow = test_space.B.tocsr()[rows]
    Bcol = trial_space.B.tocsr()[cols]
    test_tris = np.unique(Brow.nonzero()[1] // 3)
    trial_tris = np.unique(Bcol.nonzero()[1] // 3)
    tcols = (3 * trial_tris[:, None] + np.arange(3)[None, :]).reshape(-1)
    BcolT = Bcol[:, tcols].T.tocsr()                  # [3 n_trial_tris, n_cols]
    S = np.zeros((len(rows), len(cols)), dtype=np.complex128)
    C = np.zeros_like(S)
    nb = max(1, int(max_block_entries // (9 * max(1, len(trial_tris)))))
    for s in range(0, len(test_tris), nb):
        tb = test_tris[s:s + nb]
        Ls, Lc = local_blocks(X, ids, tb, trial_tris, k, rules, want, counts)
        rcols = (3 * tb[:, None] + np.arange(3)[None, :]).reshape(-1)
        Bsub = Brow[:, rcols]                          # [n_rows, 3 nb]
        for L, out in ((Ls, S), (Lc, C)):
            Lm = L.transpose(0, 2, 1, 3).reshape(3 * len(tb), 3 * len(trial_tris))
            out += Bsub @ np.asarray(BcolT.T.dot(Lm.T).T)
    return S, C


def near_field_mask(test_space, trial_space, chi):
    """Entry (i, j) kept iff dist(AABB(supp phi_i), AABB(supp phi_j)) <= chi."""
    if np.isinf(chi):
        return np.ones((test_space.N, trial_space.N), dtype=bool)
    return aabb_distance(test_space, trial_space) <= chi


def gram_bc_rwg(rwg, bc):
    """G_ij = <BC_j, RWG_i> = int BC_j . (n x RWG_i) (eqs. MassA / dualpairingGammam).

    Integrated on the barycentric triangles with the degree-2 three-point rule,
    which is exact for this piecewise-quadratic integrand.
    """
    bary, w = triangle_rule(3)
    ntau = bc.tri_xyz.shape[0]
    tau = np.arange(ntau)
    par = bc.parent
    Lg = np.zeros((ntau, 3, 3))                 # [tau, a (bc local), b (primal local)]
    Pp = rwg.tri_xyz[par]                       # parent primal triangles [ntau, 3, 3]
    Ap = rwg.area[par]
    nrm = bc.normal
    for q in range(len(w)):
        x, fbc = bc.values(tau, bary[q:q + 1])  # x [ntau,1,3], fbc [ntau,1,3,3]
        x = x[:, 0]
        fbc = fbc[:, 0]
        fpr = (x[:, None, :] - Pp) / (2.0 * Ap)[:, None, None]      # [ntau, 3(b), 3]
        rot = np.cross(nrm[:, None, :], fpr)                         # n x f
        Lg += w[q] * bc.area[:, None, None] * np.einsum("tac,tbc->tab", fbc, rot)
    rows = (3 * par[:, None, None] + np.arange(3)[None, None, :]).repeat(3, 1)  # b index
    cols = (3 * tau[:, None, None] + np.arange(3)[None, :, None]).repeat(3, 2)  # a index
    Lbig = sp.csr_matrix((Lg.reshape(-1), (rows.reshape(-1), cols.reshape(-1))),
                         shape=(rwg.B.shape[1], bc.B.shape[1]))
    G = rwg.B @ Lbig @ bc.B.T
    return np.asarray(G.todense())


def identity_rwg(rwg):
    """I_ij = <RWG_j, RWG_i> = int RWG_j . (n x RWG_i) on the primal mesh (degree-2, exact)."""
    bary, w = triangle_rule(3)
    nt = rwg.tri_xyz.shape[0]
    t = np.arange(nt)
    L = np.zeros((nt, 3, 3))
    for q in range(len(w)):
        x, f = rwg.values(t, bary[q:q + 1])
        f = f[:, 0]
        rot = np.cross(rwg.normal[:, None, :], f)
        L += w[q] * rwg.area[:, None, None] * np.einsum("tac,tbc->tba", f, rot)
    rows = (3 * t[:, None, None] + np.arange(3)[None, :, None]).repeat(3, 2)
    cols = (3 * t[:, None, None] + np.arange(3)[None, None, :]).repeat(3, 1)
    Lbig = sp.csr_matrix((L.reshape(-1), (rows.reshape(-1), cols.reshape(-1))),
                         shape=(rwg.B.shape[1], rwg.B.shape[1]))
    return np.asarray((rwg.B @ Lbig @ rwg.B.T).todense())
