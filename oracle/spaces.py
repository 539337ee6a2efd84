"""Primal edges, RWG and Buffa–Christiansen spaces (test infrastructure).

Section 3.2 of the paper: RWG_m is spanned by the Rao–Wilton–Glisson
functions of the primal mesh of Gamma_m, BC_m by the Buffa–Christiansen
functions on its barycentric refinement (six triangles per primal triangle);
both have one function per primal edge, and BC_m is dual to RWG_m under the
pairing <a, b> = int a . (n x b) (eq. dualpairingGammam).

Every basis function here is stored in one uniform form: on each triangle tau
of its support it is a sum over the three local vertices a of
beta * f_{tau,a}, where f_{tau,a}(x) = (x - P_a) / (2 |tau|) is the
lowest-order Raviart–Thomas shape function with unit outward flux through
the edge opposite P_a and zero flux through the other two edges. So beta is
exactly the outward flux of the function through that edge.

Conventions (readings where the paper is silent):
* edges are numbered by sorted (scatterer id, lower vertex id, higher vertex
  id); edge e is oriented from its lower to its higher vertex id;
* T+ of an edge is the triangle whose counter-clockwise vertex cycle runs
  lower -> higher along the edge, T- the other one; RWG_e = +l_e f on T+ and
  -l_e f on T-, i.e. flux l_e from T+ to T-;
* BC_e (reading of buffa2007dual, which the paper cites without giving
  coefficients): total flux l_e crossing the dual edge of e from the dual
  cell D(lo) to D(hi); the divergence integral is +l_e/(2N) on each of the
  2N small triangles of D(lo) (N = primal edges at the vertex) and
  -l_e/(2N) on each small triangle of D(hi); the free circulation is fixed by
  mirror symmetry about the spoke (v, mid(e)), which carries zero flux. The
  spoke fluxes follow from flux balance triangle by triangle.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class Topology:
    """Primal edges of a closed, consistently oriented triangulation."""

    def __init__(self, verts, tris, domain):
        self.verts = np.asarray(verts, dtype=np.float64)
        self.tris = np.asarray(tris, dtype=np.int64)
        self.domain = np.asarray(domain, dtype=np.int64)
        nt = len(self.tris)
        slots = {}
        for t in range(nt):
            for i in range(3):
                a, b = self.tris[t, i], self.tris[t, (i + 1) % 3]
                opp = (i + 2) % 3
                key = (int(self.domain[t]), int(min(a, b)), int(max(a, b)))
                entry = slots.setdefault(key, [None, None])
                s = 0 if a < b else 1
                if entry[s] is not None:
                    raise ValueError("edge used twice in the same direction: not an oriented 2-manifold")
                entry[s] = (t, opp)
        keys = sorted(slots)
        for k in keys:
            if slots[k][0] is None or slots[k][1] is None:
                raise ValueError("open edge: surface is not closed")
        self.edge_key = {k: i for i, k in enumerate(keys)}
        self.edges = np.array([[k[1], k[2]] for k in keys], dtype=np.int64)
        self.edge_domain = np.array([k[0] for k in keys], dtype=np.int64)
        self.tplus = np.array([slots[k][0][0] for k in keys], dtype=np.int64)
        self.aplus = np.array([slots[k][0][1] for k in keys], dtype=np.int64)
        self.tminus = np.array([slots[k][1][0] for k in keys], dtype=np.int64)
        self.aminus = np.array([slots[k][1][1] for k in keys], dtype=np.int64)
        d = self.verts[self.edges[:, 1]] - self.verts[self.edges[:, 0]]
        self.length = np.sqrt((d * d).sum(1))
        self.n_edges = len(keys)
        self.h = float(self.length.max())

    def edge_of(self, t, a, b):
        return self.edge_key[(int(self.domain[t]), int(min(a, b)), int(max(a, b)))]


def _tri_geometry(P):
    """Areas and unit normals of triangles P [n, 3, 3] (vertex order gives the normal)."""
    c = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    nrm = np.sqrt((c * c).sum(1))
    return 0.5 * nrm, c / nrm[:, None]


class Space:
    """A div-conforming space stored as local RT0 fluxes on a triangle set.

    ``B`` is the sparse [N, 3*n_tri] matrix of fluxes beta: basis i equals
    sum over (tau, a) of B[i, 3 tau + a] * f_{tau,a}.
    """

    def __init__(self, kind, topo, tri_xyz, tri_ids, parent, B):
        self.kind = kind
        self.topo = topo
        self.tri_xyz = tri_xyz
        self.tri_ids = tri_ids
        self.parent = parent
        self.area, self.normal = _tri_geometry(tri_xyz)
        self.B = sp.csr_matrix(B)
        self.N = self.B.shape[0]
        self.domain = topo.edge_domain
        # bounding box of each support
        lo = np.full((self.N, 3), np.inf)
        hi = np.full((self.N, 3), -np.inf)
        coo = self.B.tocoo()
        tmin = tri_xyz.min(1)
        tmax = tri_xyz.max(1)
        for i, col in zip(coo.row, coo.col):
            tau = col // 3
            lo[i] = np.minimum(lo[i], tmin[tau])
            hi[i] = np.maximum(hi[i], tmax[tau])
        self.aabb_lo, self.aabb_hi = lo, hi

    def values(self, tau, bary):
        """f_{tau,a}(x) for the local functions at barycentric points: [n_tau, npts, 3(a), 3]."""
        P = self.tri_xyz[tau]                       # [n, 3, 3]
        x = np.einsum("qa,nac->nqc", bary, P)       # [n, q, 3]
        f = (x[:, :, None, :] - P[:, None, :, :]) / (2.0 * self.area[tau])[:, None, None, None]
        return x, f


def rwg_space(topo: Topology) -> Space:
    """RWG_e = +l_e f_{T+, a+} - l_e f_{T-, a-} (Section 3.2, rao1982electromagnetic)."""
    nt = len(topo.tris)
    P = topo.verts[topo.tris]
    ne = topo.n_edges
    rows = np.concatenate([np.arange(ne), np.arange(ne)])
    cols = np.concatenate([3 * topo.tplus + topo.aplus, 3 * topo.tminus + topo.aminus])
    vals = np.concatenate([topo.length, -topo.length])
    B = sp.csr_matrix((vals, (rows, cols)), shape=(ne, 3 * nt))
    return Space("RWG", topo, P, topo.tris.copy(), np.arange(nt), B)


def barycentric_refinement(topo: Topology):
    """Six triangles per primal triangle (v0,m01,c),(m01,v1,c),(v1,m12,c),(m12,v2,c),(v2,m20,c),(m20,v0,c).

    Vertex ids: primal v -> v, midpoint of edge e -> nv + e, barycentre of t -> nv + ne + t.
    """
    nv, ne, nt = len(topo.verts), topo.n_edges, len(topo.tris)
    mids = 0.5 * (topo.verts[topo.edges[:, 0]] + topo.verts[topo.edges[:, 1]])
    bary = topo.verts[topo.tris].mean(1)
    X = np.concatenate([topo.verts, mids, bary])
    ids = np.empty((6 * nt, 3), dtype=np.int64)
    for t in range(nt):
        v0, v1, v2 = topo.tris[t]
        m01 = nv + topo.edge_of(t, v0, v1)
        m12 = nv + topo.edge_of(t, v1, v2)
        m20 = nv + topo.edge_of(t, v2, v0)
        c = nv + ne + t
        ids[6 * t:6 * t + 6] = [(v0, m01, c), (m01, v1, c), (v1, m12, c),
                                (m12, v2, c), (v2, m20, c), (m20, v0, c)]
    parent = np.repeat(np.arange(nt), 6)
    return X, ids, parent


def bc_space(topo: Topology) -> Space:
    """Buffa–Christiansen functions on the barycentric refinement (reading in module doc)."""
    nv, ne = len(topo.verts), topo.n_edges
    X, ids, parent = barycentric_refinement(topo)
    # dual cells: barycentric triangles touching each primal vertex, with the
    # counter-clockwise successor map  s -> (tau, s') for tau = (v, s, s')
    succ = [dict() for _ in range(nv)]
    for tau in range(len(ids)):
        for k in range(3):
            v = ids[tau, k]
            if v < nv:
                s, s2 = ids[tau, (k + 1) % 3], ids[tau, (k + 2) % 3]
                succ[v][s] = (tau, s2)
    rows, cols, vals = [], [], []
    for e in range(ne):
        lo, hi = topo.edges[e]
        l = topo.length[e]
        for v, sgn in ((lo, 1.0), (hi, -1.0)):
            cell = succ[v]
            twoN = len(cell)
            s = nv + e
            flux = lambda j: 0.0 if j % twoN == 0 else sgn * l * (j / twoN - 0.5)
            for j in range(twoN):
                tau, s_next = cell[s]
                loc = {int(ids[tau, q]): q for q in range(3)}
                outer = sgn * l * 0.5 if j in (0, twoN - 1) else 0.0
                beta = {loc[v]: outer, loc[s]: flux(j + 1), loc[s_next]: -flux(j)}
                for a in range(3):
                    if beta[a] != 0.0:
                        rows.append(e)
                        cols.append(3 * tau + a)
                        vals.append(beta[a])
                s = s_next
            if s != nv + e:
                raise ValueError("dual cell walk did not close")
    B = sp.csr_matrix((vals, (rows, cols)), shape=(ne, 3 * len(ids)))
    return Space("BC", topo, X[ids], ids, parent, B)


def aabb_distance(sp_a: Space, sp_b: Space):
    """Dense [N_a, N_b] distance between support bounding boxes."""
    lo_a, hi_a = sp_a.aabb_lo[:, None, :], sp_a.aabb_hi[:, None, :]
    lo_b, hi_b = sp_b.aabb_lo[None, :, :], sp_b.aabb_hi[None, :, :]
    gap = np.maximum(0.0, np.maximum(lo_b - hi_a, lo_a - hi_b))
    return np.sqrt((gap * gap).sum(-1))
