"""The mixed (RWG, BC) discretisation, eq. mixed_discretisation (test infrastructure).

Section 3.2 notes that, besides the choice of this paper (RWG for A's domain,
dual and P's range; BC for P's domain, dual and A's range, eq.
RWG_discretisation1), the earlier work uses one space for everything: each
scatterer's pair of traces in (RWG_m, BC_m), for A and for P alike, so that P
reuses A's blocks. This module builds that discretisation on the barycentric
mesh, where both spaces live: RWG functions are written there as combinations
of the local RT0 functions of the six sub-triangles of each primal triangle.

With the swapped pairing <(a1, a2), (b1, b2)> = <a1, b2> + <a2, b1> and trial
(u1, u2) in (RWG, BC), test (v1, v2) in (RWG, BC), a block [[C, (mu/k) S],
[-(k/mu) S, C]] is tested as

    rows (v1, 0):  [-(k/mu) S(RWG, RWG),  C(RWG, BC)]
    rows (0, v2):  [ C(BC, RWG),         (mu/k) S(BC, BC)]

(test space first), and the identity as [[0, G], [-G^T, 0]] with the Gram
G_ij = <BC_j, RWG_i> of eq. MassA.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import bem
from .pmchwt import PMCHWT, gmres
from .quadrature import triangle_rule
from .spaces import Space, barycentric_refinement, bc_space, rwg_space


def refined_rwg(topo) -> Space:
    """RWG on the barycentric refinement: on a sub-triangle tau of primal t,
    f_{t,a} = (x - P_a)/(2|t|) equals sum_b beta_b (x - Q_b)/(2|tau|) with
    sum_b beta_b = |tau|/|t| and sum_b beta_b Q_b = (|tau|/|t|) P_a, i.e. beta =
    (|tau|/|t|) times the barycentric coordinates of P_a in tau (its plane)."""
    coarse = rwg_space(topo)
    X, ids, parent = barycentric_refinement(topo)
    Q = X[ids]                                       # [6 nt, 3, 3]
    P = coarse.tri_xyz                               # [nt, 3, 3]
    area_t = coarse.area
    c = np.cross(Q[:, 1] - Q[:, 0], Q[:, 2] - Q[:, 0])
    area_tau = 0.5 * np.linalg.norm(c, axis=1)
    ntau = len(ids)
    # R[3 t + a, 3 tau + b] = beta_b of f_{t,a} on tau
    rows, cols, vals = [], [], []
    for tau in range(ntau):
        t = parent[tau]
        M = np.vstack([Q[tau].T, np.ones(3)])        # [4, 3]: sum_b lam_b (Q_b, 1)
        for a in range(3):
            lam = np.linalg.lstsq(M, np.append(P[t, a], 1.0), rcond=None)[0]
            for b in range(3):
                rows.append(3 * t + a)
                cols.append(3 * tau + b)
                vals.append(area_tau[tau] / area_t[t] * lam[b])
    R = sp.csr_matrix((vals, (rows, cols)), shape=(3 * len(P), 3 * ntau))
    return Space("RWG_bary", topo, Q, ids, parent, coarse.B @ R)


def _tested(space, inc, k, which):
    """-int field . phi_i over the space's triangles for the incident trace
    component `which` (1: E, 2: (k/mu_e)(d x p) e^{ik d.x}, mu_e = 1); with
    <a x n, phi> = -int a . phi (see pmchwt)."""
    d = np.asarray(inc[:3], dtype=np.float64)
    p = np.asarray(inc[3:6], dtype=np.float64)
    vec = p if which == 1 else k * np.cross(d, p)
    bary, w = triangle_rule(6)
    nt = space.tri_xyz.shape[0]
    x, f = space.values(np.arange(nt), bary)
    ph = np.exp(1j * k * (x @ d))
    wA = w[None, :] * space.area[:, None]
    loc = -np.einsum("tq,tq,tqac,c->ta", wA, ph, f, vec)
    return space.B @ loc.reshape(-1)


def _current_integral(space, coeffs, k, xh):
    """J = int v(y) e^{-ik xh.y} of the expansion sum_j coeffs_j phi_j."""
    bary, w = triangle_rule(6)
    nt = space.tri_xyz.shape[0]
    y, f = space.values(np.arange(nt), bary)
    wA = w[None, :] * space.area[:, None]
    beta = (space.B.T @ coeffs).reshape(nt, 3)
    v = np.einsum("ta,tqac->tqc", beta, f)
    ph = np.exp(-1j * k * (y @ xh)) * wA
    return np.einsum("tq,tqc->c", ph, v)


class MixedPMCHWT:
    """PMCHWT with P = D on the mixed discretisation (trial and test (RWG_m, BC_m))."""

    def __init__(self, verts, tris, domain, k_ext, eps_r, mu_r=None, rules=(6, 4)):
        self.base = PMCHWT(verts, tris, domain, k_ext, eps_r, mu_r, rules_A=rules, rules_P=rules, precond="I")
        self.rules = bem.Rules(*rules)
        b = self.base
        self.M, self.N_e, self.edge_ranges = b.M, b.N_e, b.edge_ranges
        self.k_e, self.mu_e, self.k_m, self.mu_r = b.k_e, b.mu_e, b.k_m, b.mu_r
        self.rwg = b.rwg
        self.rwg_b = refined_rwg(b.topo)
        self.bc = bc_space(b.topo)

    def _ops(self, k, idx=None):
        """S(RWG,RWG), C(RWG,BC), C(BC,RWG), S(BC,BC) at wavenumber k (test first)."""
        r = self.rules
        S_rr, _ = bem.assemble(self.rwg, self.rwg, k, r, want=1, rows=idx, cols=idx)
        _, C_rb = bem.assemble(self.rwg_b, self.bc, k, r, want=2, rows=idx, cols=idx)
        _, C_br = bem.assemble(self.bc, self.rwg_b, k, r, want=2, rows=idx, cols=idx)
        S_bb, _ = bem.assemble(self.bc, self.bc, k, r, want=1, rows=idx, cols=idx)
        return S_rr, C_rb, C_br, S_bb

    def assemble(self):
        self.ext = self._ops(self.k_e)
        self.int = [self._ops(self.k_m[m], np.arange(a, b)) for m, (a, b) in enumerate(self.edge_ranges)]
        self.G = bem.gram_bc_rwg(self.rwg, self.bc)

    @staticmethod
    def _block(ops, k, mu, sl=None):
        S_rr, C_rb, C_br, S_bb = (o if sl is None else o[sl] for o in ops)
        return np.block([[-(k / mu) * S_rr, C_rb], [C_br, (mu / k) * S_bb]])

    def matrix_A(self, diagonal_only=False):
        n = 2 * self.N_e
        A = np.zeros((n, n), dtype=np.complex128)
        R = self.edge_ranges
        for m, (a, b) in enumerate(R):
            for l, (c, d) in enumerate(R):
                if diagonal_only and m != l:
                    continue
                blk = self._block(self.ext, self.k_e, self.mu_e, np.s_[a:b, c:d])
                if m == l:
                    blk = blk + self._block(self.int[m], self.k_m[m], self.mu_r[m])
                A[2 * a:2 * b, 2 * c:2 * d] = blk
        return A

    def mass(self):
        """Identity in the swapped pairing: [[0, G], [-G^T, 0]] per scatterer."""
        n = 2 * self.N_e
        Mm = np.zeros((n, n))
        for (a, b) in self.edge_ranges:
            G = self.G[a:b, a:b]
            nb = b - a
            Mm[2 * a:2 * a + nb, 2 * a + nb:2 * b] = G
            Mm[2 * a + nb:2 * b, 2 * a:2 * a + nb] = -G.T
        return Mm

    def rhs(self, inc):
        """Rows (RWG, 0) take trace component 2 tested with RWG, rows (0, BC)
        component 1 tested with BC."""
        b2 = _tested(self.rwg, inc, self.k_e, 2)
        b1 = _tested(self.bc, inc, self.k_e, 1)
        return self.base._paper_order(b2, b1)

    def solve(self, inc, tol=1e-5, restart=200, maxit=2000):
        """GMRES on M^-1 D M^-1 A x = M^-1 D M^-1 b, D = the diagonal blocks of A."""
        A = self.matrix_A()
        D = self.matrix_A(diagonal_only=True)
        lu = sla.lu_factor(self.mass())
        apply = lambda v: sla.lu_solve(lu, D @ sla.lu_solve(lu, A @ v))
        rhs = sla.lu_solve(lu, D @ sla.lu_solve(lu, self.rhs(inc)))
        x, it, hist = gmres(apply, rhs, tol, restart, maxit)
        return x, {"iterations": it, "residuals": hist}

    def far_field(self, x, dirs):
        """As pmchwt.PMCHWT.far_field, the second trace expanded in BC."""
        c, d = self.base.split(x)
        dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
        out = np.zeros((len(dirs), 3), dtype=np.complex128)
        for n_, xh in enumerate(dirs):
            Ja = _current_integral(self.rwg, c, self.k_e, xh)
            Jb = _current_integral(self.bc, (self.mu_e / self.k_e) * d, self.k_e, xh)
            out[n_] = -(1j * self.k_e / (4 * np.pi)) * (np.cross(xh, Ja) - np.cross(xh, np.cross(xh, Jb)))
        return out
