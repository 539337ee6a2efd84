"""Pins of the oracle's S and C integrals and of its RWG / BC spaces (CPU only)."""
import math

import numpy as np
import pytest

from oracle import bem, spaces
from paper_2008_04772_gb300 import meshgen


# ---------------------------------------------------------------------------
# analytic potential of a uniform triangle at an in-plane point
# ---------------------------------------------------------------------------
def _inplane_potential(x, P):
    """int_T 1/|x-y| dy for x in the plane of T (signed decomposition into 3 triangles).

    For each edge A->B (counter-clockwise about the normal), the triangle
    (x, A, B) contributes h (asinh(s_B/|h|) - asinh(s_A/|h|)), with h the signed
    distance from x to the edge line (positive inside) and s the coordinate
    along the edge from the foot of x.
    """
    n = np.cross(P[1] - P[0], P[2] - P[0])
    n /= np.linalg.norm(n)
    tot = 0.0
    for i in range(3):
        A, B = P[i], P[(i + 1) % 3]
        u = (B - A) / np.linalg.norm(B - A)
        inward = np.cross(n, u)
        h = np.dot(x - A, inward)
        if abs(h) < 1e-14:
            continue
        sA = np.dot(A - x, u)
        sB = np.dot(B - x, u)
        tot += h * (math.asinh(sB / abs(h)) - math.asinh(sA / abs(h)))
    return tot


def _composite_points(P, level):
    """Points and weights of the 6-point rule on 4**level congruent sub-triangles of P."""
    from oracle.quadrature import triangle_rule
    tris = [np.array(P, dtype=np.float64)]
    for _ in range(level):
        nt = []
        for T in tris:
            a, b, c = T
            ab, bc, ca = 0.5 * (a + b), 0.5 * (b + c), 0.5 * (c + a)
            nt += [np.array([a, ab, ca]), np.array([ab, b, bc]), np.array([ca, bc, c]),
                   np.array([ab, bc, ca])]
        tris = nt
    bary, w = triangle_rule(6)
    pts, wts = [], []
    for T in tris:
        area = 0.5 * np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0]))
        pts.append(bary @ T)
        wts.append(w * area)
    return np.concatenate(pts), np.concatenate(wts)


def _static_double_integral(P1, P2, level=5):
    x, w = _composite_points(P1, level)
    return sum(wi * _inplane_potential(xi, P2) for xi, wi in zip(x, w))


@pytest.mark.parametrize("case", ["identical", "edge", "vertex"])
def test_singular_static_part_matches_analytic_potential(oracle_lib, case):
    # Coplanar pairs in z = 0. At k -> 0, Im S_loc[a][b] * k * |T1||T2| * 4 pi
    # tends to II 1/|x-y| (the divergence term dominates); the reference value
    # integrates the closed-form inner potential with a fine composite rule.
    X = np.array([[0, 0, 0], [1, 0, 0], [0.3, 0.9, 0], [0.8, -0.7, 0], [-0.6, -0.4, 0]],
                 dtype=np.float64)
    ids = {"identical": ([0, 1, 2], [0, 1, 2]),
           "edge": ([0, 1, 2], [1, 0, 3]),
           "vertex": ([0, 1, 2], [0, 4, 3])}[case]
    tri_ids = np.array(ids)
    k = 1e-6
    S, C = bem.local_blocks(X, tri_ids, [0], [1], k, bem.Rules(6, 8))
    A1 = 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
    A2 = 0.5 * np.linalg.norm(np.cross(X[tri_ids[1][1]] - X[tri_ids[1][0]],
                                       X[tri_ids[1][2]] - X[tri_ids[1][0]]))
    got = S[0, 0, 0, 0].imag * k * A1 * A2 * 4 * math.pi
    ref = _static_double_integral(X[tri_ids[0]], X[tri_ids[1]])
    assert abs(got - ref) < 2e-5 * abs(ref), (got, ref)
    # coplanar -> C vanishes identically
    assert np.abs(C).max() < 1e-12 * np.abs(S).max()


def _pair(cls, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(6, 3))
    ids = {3: ([0, 1, 2], [0, 1, 2]), 2: ([0, 1, 2], [1, 0, 3]), 1: ([0, 1, 2], [0, 4, 5]),
           0: ([0, 1, 2], [3, 4, 5])}[cls]
    if cls == 0:
        X[3:] += 4.0
    return X, np.array(ids)


@pytest.mark.parametrize("cls", [1, 2, 3])
def test_singular_rule_converges_and_is_symmetric(oracle_lib, cls):
    # Sauter–Schwab order 4 (the paper's q_singular = 6) against orders 8 and 12
    # on a non-coplanar pair; both operators are symmetric, so the blocks of
    # (T2, T1) must be the transposes of those of (T1, T2) to quadrature accuracy.
    X, ids = _pair(cls, seed=10 + cls)
    k = 2.0 + 0.3j
    S4, C4 = bem.local_blocks(X, ids, [0], [1], k, bem.Rules(6, 4))
    S8, C8 = bem.local_blocks(X, ids, [0], [1], k, bem.Rules(6, 8))
    S16, C16 = bem.local_blocks(X, ids, [0], [1], k, bem.Rules(6, 16))
    Sr, Cr = bem.local_blocks(X, ids, [1], [0], k, bem.Rules(6, 16))
    nS, nC = np.abs(S16).max(), max(np.abs(C16).max(), 1e-300)
    # spectral convergence in the Gauss order (measured: ~1e-3, ~1e-6 at 4, 8)
    assert np.abs(S8 - S16).max() < 2e-5 * nS
    assert np.abs(S4 - S16).max() < 5e-3 * nS
    assert np.abs(Sr[0, 0].T - S16[0, 0]).max() < 1e-8 * nS
    if cls != 3:
        assert np.abs(C8 - C16).max() < 1e-4 * nC
        assert np.abs(C4 - C16).max() < 2e-2 * nC
        assert np.abs(Cr[0, 0].T - C16[0, 0]).max() < 1e-7 * nC
    else:
        assert nC < 1e-12 * nS   # flat identical panels: C = 0


def test_regular_pair_dipole_limit(oracle_lib):
    # Two small triangles (size eps) a distance R apart: the Galerkin integrals
    # reduce to point interactions of the integrated local functions
    # F_a = int f_a = (c - P_a)/2 and of the unit divergence integrals:
    #   S -> -ik G F_a.F'_b + (i/k) G,   C -> grad_x G(c1, c2) . (F_a x F'_b).
    rng = np.random.default_rng(3)
    eps, R = 1e-3, 1.3
    P1 = rng.normal(size=(3, 3)) * eps
    P2 = rng.normal(size=(3, 3)) * eps + np.array([R, 0.4, -0.2])
    X = np.concatenate([P1, P2])
    ids = np.array([[0, 1, 2], [3, 4, 5]])
    k = 3.0 + 0.2j
    S, C = bem.local_blocks(X, ids, [0], [1], k, bem.Rules(6, 4))
    c1, c2 = P1.mean(0), P2.mean(0)
    d = c1 - c2
    r = np.linalg.norm(d)
    G = np.exp(1j * k * r) / (4 * math.pi * r)
    gradG = d * (1j * k * r - 1) * np.exp(1j * k * r) / (4 * math.pi * r ** 3)
    for a in range(3):
        for b in range(3):
            Fa, Fb = 0.5 * (c1 - P1[a]), 0.5 * (c2 - P2[b])
            s_ref = -1j * k * G * np.dot(Fa, Fb) + (1j / k) * G
            c_ref = np.dot(gradG, np.cross(Fa, Fb))
            assert abs(S[0, 0, a, b] - s_ref) < 1e-5 * abs(s_ref)
            assert abs(C[0, 0, a, b] - c_ref) < 1e-2 * abs(c_ref) + 1e-12 * abs(s_ref)


def test_operators_complex_symmetric_on_sphere(oracle_lib):
    m = meshgen.icosphere(1)
    topo = spaces.Topology(m.verts, m.tris, m.domain)
    rwg = spaces.rwg_space(topo)
    S, C = bem.assemble(rwg, rwg, 2.0 + 0.1j, bem.Rules(6, 4))
    assert np.linalg.norm(S - S.T) < 1e-4 * np.linalg.norm(S)
    assert np.linalg.norm(C - C.T) < 1e-4 * np.linalg.norm(C)
    # with exact tensor rules on all pairs the asymmetry comes only from the
    # singular rules; raising their order shrinks it
    S8, C8 = bem.assemble(rwg, rwg, 2.0 + 0.1j, bem.Rules(6, 8))
    assert np.linalg.norm(S8 - S8.T) < 0.2 * np.linalg.norm(S - S.T)


# ---------------------------------------------------------------------------
# spaces
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def sphere_spaces():
    m = meshgen.icosphere(2)
    topo = spaces.Topology(m.verts, m.tris, m.domain)
    return topo, spaces.rwg_space(topo), spaces.bc_space(topo)


def _edge_flux_balance(space):
    """Max over shared triangle edges of |outflux from one side + outflux from the other|."""
    ids = space.tri_ids
    owner = {}
    B = space.B.tocsr()
    worst = 0.0
    for i in range(space.N):
        row = B.getrow(i)
        flux = {}
        for col, val in zip(row.indices, row.data):
            tau, a = divmod(col, 3)
            e = tuple(sorted((ids[tau, (a + 1) % 3], ids[tau, (a + 2) % 3])))
            flux[e] = flux.get(e, 0.0) + val
        # every edge seen from both sides sums to zero except the support boundary,
        # where the single side carries zero flux
        worst = max(worst, max(abs(v) for v in flux.values()))
    return worst


def test_rwg_and_bc_are_div_conforming(sphere_spaces):
    topo, rwg, bc = sphere_spaces
    assert _edge_flux_balance(rwg) < 1e-13
    assert _edge_flux_balance(bc) < 1e-13


def test_bc_divergence_and_flux(sphere_spaces):
    # Divergence integral l_e/(2N) on each small triangle of D(lo), -l_e/(2N) on
    # D(hi); total flux l_e crosses the dual edge of e; support D(lo) u D(hi).
    topo, rwg, bc = sphere_spaces
    nv = len(topo.verts)
    B = bc.B.tocsr()
    valence = np.bincount(topo.edges.reshape(-1), minlength=nv)
    for e in range(0, topo.n_edges, 7):
        lo, hi = topo.edges[e]
        l = topo.length[e]
        row = B.getrow(e)
        div = {}
        for col, val in zip(row.indices, row.data):
            tau = col // 3
            div[tau] = div.get(tau, 0.0) + val
        cells = {lo: [], hi: []}
        for tau, dv in div.items():
            v = [x for x in bc.tri_ids[tau] if x < nv][0]
            assert v in (lo, hi)
            cells[v].append(dv)
        assert len(cells[lo]) == 2 * valence[lo] and len(cells[hi]) == 2 * valence[hi]
        assert np.allclose(cells[lo], l / (2 * valence[lo]), atol=1e-14)
        assert np.allclose(cells[hi], -l / (2 * valence[hi]), atol=1e-14)


def test_gram_is_well_conditioned_under_refinement():
    # BC is dual to RWG (Section 3.2): cond(<BC_j, RWG_i>) stays bounded as h -> 0,
    # while the RWG-RWG pairing matrix is singular.
    conds = []
    for level in (1, 2, 3):
        m = meshgen.icosphere(level)
        topo = spaces.Topology(m.verts, m.tris, m.domain)
        rwg, bc = spaces.rwg_space(topo), spaces.bc_space(topo)
        G = bem.gram_bc_rwg(rwg, bc)
        conds.append(np.linalg.cond(G))
        if level == 2:
            Irr = bem.identity_rwg(rwg)
            sv = np.linalg.svd(Irr, compute_uv=False)
            assert sv[-1] < 1e-10 * sv[0]
    assert max(conds) < 10.0
    assert conds[2] < 1.2 * conds[1]


def test_gram_entries_by_brute_force():
    # <BC_j, RWG_i> integrated by a 4**3-fold composite degree-4 rule on each
    # barycentric triangle, evaluating both functions pointwise.
    m = meshgen.icosphere(1)
    topo = spaces.Topology(m.verts, m.tris, m.domain)
    rwg, bc = spaces.rwg_space(topo), spaces.bc_space(topo)
    G = bem.gram_bc_rwg(rwg, bc)

    def field(space, i, tau_set, pts_of):
        row = space.B.getrow(i)
        val = {}
        for col, beta in zip(row.indices, row.data):
            tau, a = divmod(col, 3)
            if tau in tau_set:
                x = pts_of[tau]
                val[tau] = val.get(tau, 0) + beta * (x - space.tri_xyz[tau, a]) / (2 * space.area[tau])
        return val

    rng = np.random.default_rng(0)
    for _ in range(6):
        i, j = rng.integers(0, topo.n_edges, 2)
        i = j if rng.random() < 0.5 else i
        taus = set(np.unique(bc.B.getrow(j).indices // 3))
        pts, wts = {}, {}
        for tau in taus:
            pts[tau], wts[tau] = _composite_points(bc.tri_xyz[tau], 3)
        vb = field(bc, j, taus, pts)
        ref = 0.0
        for tau in taus:
            t = bc.parent[tau]
            x = pts[tau]
            row = rwg.B.getrow(i)
            vr = np.zeros_like(x)
            for col, beta in zip(row.indices, row.data):
                tt, a = divmod(col, 3)
                if tt == t:
                    vr += beta * (x - rwg.tri_xyz[tt, a]) / (2 * rwg.area[tt])
            rot = np.cross(bc.normal[tau], vr)
            ref += np.sum(wts[tau] * np.einsum("qc,qc->q", vb.get(tau, np.zeros_like(x)), rot))
        assert abs(G[i, j] - ref) < 1e-12 * max(1.0, np.abs(G).max())
