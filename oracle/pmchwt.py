"""PMCHWT block system, Calderón preconditioners, GMRES, far field (test infrastructure).

Paper sections and equations followed, in the paper's own conventions:

* eq. PMCHWT_multiple_scatterers / multiple_operator / AimAem: A is the
  M x M block operator with diagonal blocks A^e_m + A^i_m and off-diagonal
  blocks A_{ml}; each block is [[C, (mu/k) S], [-(k/mu) S, C]].
* Section 3.1: preconditioners P in {A, D, D^e, D^i, S^e, S^i, I}.
* eqs. dualdef, GalA, GalP, MassA, MassP, RWG_discretisation1: A and its
  dual space on RWG x RWG, P and its dual on BC x BC; the dual pairing of
  X pairs (c, d) with (e, f) as <c, f> + <d, e>, so every test row block is
  component-swapped; the solved system is M_P^-1 P M_A^-1 A x = M_P^-1 P M_A^-1 b.
* Section 4: restarted GMRES, x0 = 0, stop on the relative residual of the
  preconditioned system (reading: the paper does not say which residual).
* Table tab:matvecs: one "matvec" is one application of one discretised
  boundary operator; the counter below charges 4M^2+4M per application of A
  and 8M / 4M / 2M per application of D / D^{e,i} / S^{e,i}.

Unknown ordering follows eq. multiple_operator: per scatterer m the pair
(u_m1 = gamma_D E, u_m2 = (k/mu) gamma_N E), each expanded in RWG_m.

Right-hand side (reading; the paper writes (1/2 I - D^i) u^inc for the
scattered traces): the jump relations (eq. BIOrelns) give A^i u^i = u^i / 2
for interior traces and A^e u^inc = u^inc / 2 for the entire incident field,
so the total traces u^i = u^s + u^inc solve (A^e + A^i) u^i = u^inc. The
default system therefore uses b = <u^inc, dual>, and the solution is the
total (= interior) trace. The paper's scattered-trace form is
``rhs_mode='scattered'`` (D^i applied to the L2 projection of u^inc onto
RWG); its solution is u^s, and the far field of either trace is the same
(the incident traces radiate nothing outside).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import bem
from .quadrature import triangle_rule
from .spaces import Topology, bc_space, rwg_space

PRECONDITIONERS = ("I", "A", "D", "De", "Di", "Se", "Si")


def interior_wavenumber(k_e, eps_r, mu_r):
    """k_m = k_e sqrt(eps_r mu_r), principal branch (Im >= 0 for e^{-i omega t})."""
    km = complex(k_e) * np.sqrt(complex(eps_r) * complex(mu_r))
    if km.imag < 0:
        km = -km
    return km


def matvec_units(precond: str, M: int):
    """Per-iteration and initial BIO applications of Table tab:matvecs."""
    a = 4 * M * M + 4 * M
    p = {"I": 0, "A": 4 * M * M + 4 * M, "D": 8 * M, "De": 4 * M, "Di": 4 * M,
         "Se": 2 * M, "Si": 2 * M}[precond]
    return a + p, p


def gmres(apply, b, tol, restart, maxit, on_apply=None):
    """Restarted GMRES (Saad & Schultz) with modified Gram–Schmidt and Givens rotations.

    x0 = 0; stops when ||b - apply(x)|| / ||b|| <= tol (estimated by the
    Givens residual inside a cycle, recomputed explicitly after each complete
    cycle) or after ``maxit`` iterations. Returns x, iterations, residual history.
    """
    n = len(b)
    bnorm = np.linalg.norm(b)
    x = np.zeros(n, dtype=np.complex128)
    if bnorm == 0.0:
        return x, 0, [0.0]
    r = b.copy()
    beta = bnorm
    hist = [1.0]
    it = 0
    while True:
        m = restart
        V = np.zeros((m + 1, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        done = False
        j_last = -1
        for j in range(m):
            w = apply(V[j])
            it += 1
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            a, c = H[j, j], H[j + 1, j]
            den = math.sqrt(abs(a) ** 2 + abs(c) ** 2)
            if abs(a) == 0.0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a) / den
                sn[j] = (a / abs(a)) * np.conj(c) / den
            H[j, j] = cs[j] * a + sn[j] * c
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            res = abs(g[j + 1]) / bnorm
            hist.append(res)
            j_last = j
            if (res <= tol and j < m - 1) or it >= maxit:
                done = True
                break
        k = j_last + 1
        y = sla.solve_triangular(H[:k, :k], g[:k])
        x = x + V[:k].T @ y
        if done:
            return x, it, hist
        r = b - apply(x)
        beta = np.linalg.norm(r)
        hist[-1] = beta / bnorm
        if beta / bnorm <= tol:
            return x, it, hist


class PMCHWT:
    """Oracle of one multi-scatterer PMCHWT problem on a closed mesh."""

    def __init__(self, verts, tris, domain, k_ext, eps_r, mu_r=None,
                 rules_A=(6, 4), rules_P=(6, 4), precond="D", chi_P=math.inf,
                 rhs_mode="total", aca_P=None):
        self.topo = Topology(verts, tris, domain)
        self.M = int(np.max(domain)) + 1
        eps_r = np.atleast_1d(np.asarray(eps_r, dtype=np.complex128))
        if len(eps_r) == 1:
            eps_r = np.repeat(eps_r, self.M)
        mu_r = np.ones(self.M, dtype=np.complex128) if mu_r is None else \
            np.atleast_1d(np.asarray(mu_r, dtype=np.complex128))
        if len(mu_r) == 1:
            mu_r = np.repeat(mu_r, self.M)
        self.k_e = complex(k_ext)
        self.mu_e = 1.0
        self.eps_r, self.mu_r = eps_r, mu_r
        self.k_m = np.array([interior_wavenumber(k_ext, e, m) for e, m in zip(eps_r, mu_r)])
        self.rules_A = bem.Rules(*rules_A)
        self.rules_P = bem.Rules(*rules_P)
        if precond not in PRECONDITIONERS:
            raise ValueError(precond)
        self.precond = precond
        self.chi_P = chi_P
        # aca_P = (nu_P, chi_P): P's blocks as H-matrices (hmatrix.compress: ACA to
        # nu_P on admissible blocks within chi_P, Section 3.3) instead of the
        # entry-level cutoff chi_P
        self.aca_P = aca_P
        self.P_stored = None
        self.rhs_mode = rhs_mode
        self.rwg = rwg_space(self.topo)
        self.N_e = self.topo.n_edges
        self.edge_ranges = []
        for m in range(self.M):
            idx = np.nonzero(self.topo.edge_domain == m)[0]
            self.edge_ranges.append((int(idx[0]), int(idx[-1]) + 1))
        self.matvecs = 0
        self._assembled = False

    # ------------------------------------------------------------------
    def assemble(self, need_bc=True):
        """A blocks (S, C at k_e on the union, at k_m per scatterer), P blocks, Grams."""
        rwg = self.rwg
        self.S_e, self.C_e = bem.assemble(rwg, rwg, self.k_e, self.rules_A)
        self.S_i, self.C_i = [], []
        for m, (a, b) in enumerate(self.edge_ranges):
            idx = np.arange(a, b)
            S, C = bem.assemble(rwg, rwg, self.k_m[m], self.rules_A, rows=idx, cols=idx)
            self.S_i.append(S)
            self.C_i.append(C)
        if need_bc and self.precond != "I":
            self.bc = bc_space(self.topo)
            self.G = bem.gram_bc_rwg(rwg, self.bc)
            self._assemble_P()
        self._assembled = True

    def _assemble_P(self):
        bc = self.bc
        self.P_blocks = []
        mask = bem.near_field_mask(bc, bc, math.inf if self.aca_P else self.chi_P)
        pc = self.precond
        for m, (a, b) in enumerate(self.edge_ranges):
            idx = np.arange(a, b)
            blk = {}
            msk = mask[np.ix_(idx, idx)]
            if pc in ("A", "D", "De", "Se"):
                want = 1 if pc == "Se" else 3
                S, C = bem.assemble(bc, bc, self.k_e, self.rules_P, want=want, rows=idx, cols=idx)
                blk["S_e"], blk["C_e"] = S * msk, C * msk
            if pc in ("A", "D", "Di", "Si"):
                want = 1 if pc == "Si" else 3
                S, C = bem.assemble(bc, bc, self.k_m[m], self.rules_P, want=want, rows=idx, cols=idx)
                blk["S_i"], blk["C_i"] = S * msk, C * msk
            if self.aca_P:
                from . import hmatrix
                nu, chi = self.aca_P
                keys = sorted(blk)
                comp, stored = hmatrix.compress([blk[q] for q in keys], bc.aabb_lo[idx], bc.aabb_hi[idx], nu, chi)
                blk = dict(zip(keys, comp))
                self.P_stored = (self.P_stored or 0) + stored
            self.P_blocks.append(blk)
        if pc == "A":
            S, C = bem.assemble(bc, bc, self.k_e, self.rules_P)
            self.P_offdiag = (S * mask, C * mask)

    # ------------------------------------------------------------------
    def _block(self, C, S, k, mu):
        """Operator block [[C, (mu/k) S], [-(k/mu) S, C]] tested with the swapped pairing."""
        return np.block([[-(k / mu) * S, C], [C, (mu / k) * S]])

    def matrix_A(self):
        """Dense Galerkin matrix of A (paper's ordering and swapped test rows)."""
        n = 2 * self.N_e
        A = np.zeros((n, n), dtype=np.complex128)
        R = self.edge_ranges
        for m, (a, b) in enumerate(R):
            for l, (c, d) in enumerate(R):
                Se = self.S_e[a:b, c:d]
                Ce = self.C_e[a:b, c:d]
                blk = self._block(Ce, Se, self.k_e, self.mu_e)
                if m == l:
                    blk = blk + self._block(self.C_i[m], self.S_i[m], self.k_m[m], self.mu_r[m])
                A[2 * a:2 * b, 2 * c:2 * d] = blk
        return A

    def matrix_P(self):
        """Dense Galerkin matrix of the chosen preconditioner on BC x BC."""
        n = 2 * self.N_e
        P = np.zeros((n, n), dtype=np.complex128)
        R = self.edge_ranges
        z = lambda a, b: np.zeros((b - a, b - a), dtype=np.complex128)
        for m, (a, b) in enumerate(R):
            blk = self.P_blocks[m]
            tot = np.zeros((2 * (b - a), 2 * (b - a)), dtype=np.complex128)
            if "S_e" in blk:
                C = blk["C_e"] if self.precond != "Se" else z(a, b)
                tot += self._block(C, blk["S_e"], self.k_e, self.mu_e)
            if "S_i" in blk:
                C = blk["C_i"] if self.precond != "Si" else z(a, b)
                tot += self._block(C, blk["S_i"], self.k_m[m], self.mu_r[m])
            P[2 * a:2 * b, 2 * a:2 * b] = tot
        if self.precond == "A":
            Soff, Coff = self.P_offdiag
            for m, (a, b) in enumerate(R):
                for l, (c, d) in enumerate(R):
                    if m != l:
                        P[2 * a:2 * b, 2 * c:2 * d] = self._block(
                            Coff[a:b, c:d], Soff[a:b, c:d], self.k_e, self.mu_e)
        return P

    def mass_A(self):
        """M_A: dual (RWG), range (BC): per scatterer [[0, G], [G, 0]], G_ij = <BC_j, RWG_i>."""
        n = 2 * self.N_e
        MA = np.zeros((n, n))
        for (a, b) in self.edge_ranges:
            G = self.G[a:b, a:b]
            nb = b - a
            MA[2 * a:2 * a + nb, 2 * a + nb:2 * b] = G
            MA[2 * a + nb:2 * b, 2 * a:2 * a + nb] = G
        return MA

    def mass_P(self):
        """M_P: dual (BC), range (RWG): G'_ij = <RWG_j, BC_i> = -G_ji."""
        n = 2 * self.N_e
        MP = np.zeros((n, n))
        for (a, b) in self.edge_ranges:
            Gp = -self.G[a:b, a:b].T
            nb = b - a
            MP[2 * a:2 * a + nb, 2 * a + nb:2 * b] = Gp
            MP[2 * a + nb:2 * b, 2 * a:2 * a + nb] = Gp
        return MP

    # ------------------------------------------------------------------
    def _incident_fields(self, inc):
        """Rule points of every primal triangle and the two incident traces there.

        u^inc = (E x n, (k_e/mu_e) gamma_N E) with E = p e^{ik_e d.x}: gamma_N E =
        (1/(ik)) (curl E) x n = (d x p) e^{ik_e d.x} x n.
        Returns x [nt,q,3], f [nt,q,3,3] (RWG-local functions), weights w |T| [nt,q],
        E [nt,q,3] and (k_e/mu_e)(d x p) e^{ik_e d.x} [nt,q,3] (fields, not yet crossed
        with n).
        """
        d = np.asarray(inc[:3], dtype=np.float64)
        p = np.asarray(inc[3:6], dtype=np.float64)
        dxp = np.cross(d, p)
        bary, w = triangle_rule(6)
        rwg = self.rwg
        nt = rwg.tri_xyz.shape[0]
        x, f = rwg.values(np.arange(nt), bary)             # x [nt,q,3], f [nt,q,3,3]
        ph = np.exp(1j * self.k_e * (x @ d))               # [nt, q]
        wA = w[None, :] * rwg.area[:, None]
        E1 = ph[:, :, None] * p[None, None, :]
        E2 = (self.k_e / self.mu_e) * ph[:, :, None] * dxp[None, None, :]
        return x, f, wA, E1, E2

    def _paper_order(self, v1, v2):
        """Per scatterer [v1_m; v2_m] from two edge-indexed vectors."""
        out = np.zeros(2 * self.N_e, dtype=np.complex128)
        for (a, c) in self.edge_ranges:
            nb = c - a
            out[2 * a:2 * a + nb] = v1[a:c]
            out[2 * a + nb:2 * c] = v2[a:c]
        return out

    def _tested_incident(self, inc):
        """<u^inc, dual> in the swapped pairing (paper ordering of the test rows).

        With <a x n, phi> = -int a . phi for tangential phi, the row (phi_i, 0)
        takes component 2 and (0, phi_i) component 1.
        """
        _, f, wA, E1, E2 = self._incident_fields(inc)
        loc1 = -np.einsum("tq,tqac,tqc->ta", wA, f, E1)
        loc2 = -np.einsum("tq,tqac,tqc->ta", wA, f, E2)
        b1 = self.rwg.B @ loc1.reshape(-1)
        b2 = self.rwg.B @ loc2.reshape(-1)
        return self._paper_order(b2, b1)

    def incident_coefficients(self, inc):
        """L2 projection of u^inc onto RWG: paper-ordered coefficients c (reading:
        the paper applies D^i to u^inc without saying how u^inc enters the
        discrete space; here it is the L2-orthogonal projection, the Gram matrix
        being int phi_i . phi_j and the load int phi_i . (field x n))."""
        rwg = self.rwg
        _, f, wA, E1, E2 = self._incident_fields(inc)
        nrm = rwg.normal                                   # [nt, 3]
        T1 = np.cross(E1, nrm[:, None, :])                 # E x n
        T2 = np.cross(E2, nrm[:, None, :])
        l1 = np.einsum("tq,tqac,tqc->ta", wA, f, T1)
        l2 = np.einsum("tq,tqac,tqc->ta", wA, f, T2)
        loc = np.einsum("tq,tqac,tqbc->tab", wA, f, f)    # local RT0 mass, exact (degree 2)
        nt = loc.shape[0]
        import scipy.sparse as sp
        rows = np.repeat(np.arange(3 * nt), 3)
        cols = (3 * np.arange(nt)[:, None, None] + np.arange(3)[None, None, :]).repeat(3, 1).reshape(-1)
        Lm = sp.csr_matrix((loc.reshape(-1), (rows, cols)), shape=(3 * nt, 3 * nt))
        Mass = (rwg.B @ Lm @ rwg.B.T).toarray()
        c1 = np.linalg.solve(Mass, rwg.B @ l1.reshape(-1))
        c2 = np.linalg.solve(Mass, rwg.B @ l2.reshape(-1))
        return self._paper_order(c1, c2)

    def rhs(self, inc):
        """b for one incident plane wave inc = (d_hat, p_hat) (6 numbers).

        total (default): b = <u^inc, dual>; the solution is the total trace.
        scattered (eq. PMCHWT_multiple_scatterers): b = <(1/2 I - D^i) u^inc, dual>
        with D^i = diag(A^i_m): the identity term tested exactly, D^i applied to the
        L2 projection of u^inc onto RWG (``incident_coefficients``); the solution
        is the scattered trace u^s.
        """
        b = self._tested_incident(inc)
        if self.rhs_mode == "total":
            return b
        if self.rhs_mode != "scattered":
            raise ValueError(self.rhs_mode)
        if not self._assembled:
            self.assemble()
        c = self.incident_coefficients(inc)
        out = 0.5 * b
        for m, (a, e) in enumerate(self.edge_ranges):
            blk = self._block(self.C_i[m], self.S_i[m], self.k_m[m], self.mu_r[m])
            out[2 * a:2 * e] -= blk @ c[2 * a:2 * e]
        return out

    def solve(self, inc, tol=1e-6, restart=200, maxit=2000):
        """Solve M_P^-1 P M_A^-1 A x = M_P^-1 P M_A^-1 b by GMRES; returns x, info."""
        if not self._assembled:
            self.assemble()
        A = self.matrix_A()
        b = self.rhs(inc)
        per_it, init = matvec_units(self.precond, self.M)
        if self.precond == "I":
            apply = lambda v: A @ v
            rhs = b
        else:
            P = self.matrix_P()
            luA = sla.lu_factor(self.mass_A())
            luP = sla.lu_factor(self.mass_P())
            apply = lambda v: sla.lu_solve(luP, P @ sla.lu_solve(luA, A @ v))
            rhs = sla.lu_solve(luP, P @ sla.lu_solve(luA, b))
        self.matvecs = init
        counter = {"n": 0}

        def counted(v):
            counter["n"] += 1
            return apply(v)

        x, it, hist = gmres(counted, rhs, tol, restart, maxit)
        self.matvecs += per_it * counter["n"]
        return x, {"iterations": it, "applications": counter["n"], "matvecs": self.matvecs,
                   "residuals": hist}

    # ------------------------------------------------------------------
    def split(self, x):
        """Paper-ordered x -> (c, d) coefficient vectors over all edges (component-major)."""
        c = np.zeros(self.N_e, dtype=np.complex128)
        d = np.zeros(self.N_e, dtype=np.complex128)
        for (a, b) in self.edge_ranges:
            nb = b - a
            c[a:b] = x[2 * a:2 * a + nb]
            d[a:b] = x[2 * a + nb:2 * b]
        return c, d

    def far_field(self, x, dirs):
        """E^inf(x_hat) = -(ik_e/4pi) [x_hat x J_a - x_hat x (x_hat x J_b)].

        Derived from the exterior Stratton–Chu formula (eq. StrattonChu_ext)
        with G ~ e^{ikr}/(4 pi r) e^{-ik x_hat.y}: a = gamma_D E (first trace),
        b = gamma_N E = (mu_e/k_e) (second trace); J_v = int v e^{-ik_e x_hat.y}.
        Total traces may replace scattered ones because the entire incident
        field has a zero exterior representation. Integrals use the 6-point rule.
        """
        c, d = self.split(x)
        dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
        bary, w = triangle_rule(6)
        rwg = self.rwg
        nt = rwg.tri_xyz.shape[0]
        y, f = rwg.values(np.arange(nt), bary)              # y [nt,q,3], f [nt,q,3,3]
        wA = w[None, :] * rwg.area[:, None]
        # basis values: phi_i(y) = sum_a B[i, 3t+a] f_{t,a}(y)  -> coefficient field per (t, a)
        ca = (rwg.B.T @ c).reshape(nt, 3)
        da = (rwg.B.T @ d).reshape(nt, 3) * (self.mu_e / self.k_e)
        va = np.einsum("ta,tqac->tqc", ca, f)               # a(y) at points
        vb = np.einsum("ta,tqac->tqc", da, f)
        out = np.zeros((len(dirs), 3), dtype=np.complex128)
        for n_, xh in enumerate(dirs):
            ph = np.exp(-1j * self.k_e * (y @ xh)) * wA
            Ja = np.einsum("tq,tqc->c", ph, va)
            Jb = np.einsum("tq,tqc->c", ph, vb)
            out[n_] = -(1j * self.k_e / (4 * np.pi)) * (np.cross(xh, Ja) - np.cross(xh, np.cross(xh, Jb)))
        return out
