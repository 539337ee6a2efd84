"""Pins of the oracle's system, solver, far field and Mie series (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import bem, mie, pmchwt, spaces
from paper_2008_04772_gb300 import meshgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = 3.17 + 0.01j
INC = np.array([0.0, 0.0, 1.0, 1.0, 0.0, 0.0])


# ---------------------------------------------------------------------------
# Mie series
# ---------------------------------------------------------------------------
def test_mie_matches_bohren_huffman_example():
    r, lam, mre, mim, qsca, qext, qback = np.loadtxt(os.path.join(GOLDEN, "bhmie_example.txt"))
    x = 2 * math.pi * r / lam
    qe, qs = mie.efficiencies(x, complex(mre, mim))
    a, b = mie.coefficients(x, complex(mre, mim))
    n = np.arange(1, len(a) + 1)
    qb = abs(np.sum((2 * n + 1) * (-1) ** n * (a - b))) ** 2 / x ** 2
    assert abs(qs - qsca) < 6e-6 and abs(qe - qext) < 6e-6 and abs(qb - qback) < 6e-6


def test_mie_rayleigh_limit():
    # x << 1: S1 = -i x^3 (m^2-1)/(m^2+2), S2 = S1 cos(theta) (Bohren & Huffman Sec. 5.2)
    x, m = 1e-3, np.sqrt(EPS)
    th = np.linspace(0, math.pi, 7)
    S1, S2 = mie.amplitudes(x, m, th)
    ref = -1j * x ** 3 * (m * m - 1) / (m * m + 2)
    assert np.allclose(S1, ref, rtol=1e-5)
    assert np.allclose(S2, ref * np.cos(th), rtol=1e-5, atol=1e-5 * abs(ref))


def test_mie_far_field_optical_theorem_and_energy():
    # sigma_ext = (4 pi / k) Im(p . E_inf(d)), sigma_sca = int |E_inf|^2 dOmega
    k, a = 2.0, 1.0
    qe, qs = mie.efficiencies(k * a, np.sqrt(EPS))
    fwd = mie.far_field(k, a, EPS, np.array([[0.0, 0.0, 1.0]]))[0]
    assert abs(4 * math.pi / k * fwd[0].imag - qe * math.pi * a * a) < 1e-10
    # Gauss–Legendre in cos(theta) x trapezoid in phi
    from oracle.quadrature import gauss_legendre_01
    u, wu = gauss_legendre_01(60)
    ct = 2 * u - 1
    ph = np.linspace(0, 2 * math.pi, 64, endpoint=False)
    C, P = np.meshgrid(ct, ph, indexing="ij")
    S = np.sqrt(1 - C ** 2)
    dirs = np.stack([S * np.cos(P), S * np.sin(P), C], -1).reshape(-1, 3)
    E = mie.far_field(k, a, EPS, dirs)
    w = (2 * wu)[:, None].repeat(len(ph), 1).reshape(-1) * (2 * math.pi / len(ph))
    sca = np.sum(w * np.sum(abs(E) ** 2, 1))
    assert abs(sca - qs * math.pi * a * a) < 1e-9 * sca
    assert qe > qs   # absorbing sphere


# ---------------------------------------------------------------------------
# full discretisation against Mie
# ---------------------------------------------------------------------------
def _direct_far_field(level, k=2.0, eps=EPS):
    m = meshgen.icosphere(level)
    pb = pmchwt.PMCHWT(m.verts, m.tris, m.domain, k, eps, precond="I")
    pb.assemble(need_bc=False)
    x = np.linalg.solve(pb.matrix_A(), pb.rhs(INC))
    dirs = meshgen.sphere_cut_directions(37)
    return pb, x, pb.far_field(x, dirs), mie.far_field(k, 1.0, eps, dirs)


def test_far_field_converges_to_mie():
    errs = []
    for level in (1, 2, 3):
        _, _, F, Fm = _direct_far_field(level)
        errs.append(np.linalg.norm(F - Fm) / np.linalg.norm(Fm))
    # flat-triangle geometry error O(h): a few % at 320 triangles, falling with h
    assert errs[1] < 0.05
    assert errs[0] > errs[1] > errs[2]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 1.0, (errs, orders)


def test_energy_balance_lossless_sphere():
    # real eps_r: no absorption, sigma_ext = sigma_sca up to discretisation error
    pb, x, _, _ = _direct_far_field(2, eps=3.17)
    k = 2.0
    fwd = pb.far_field(x, np.array([[0.0, 0.0, 1.0]]))[0]
    sig_ext = 4 * math.pi / k * fwd[0].imag
    from oracle.quadrature import gauss_legendre_01
    u, wu = gauss_legendre_01(40)
    ct = 2 * u - 1
    ph = np.linspace(0, 2 * math.pi, 40, endpoint=False)
    C, P = np.meshgrid(ct, ph, indexing="ij")
    S = np.sqrt(1 - C ** 2)
    dirs = np.stack([S * np.cos(P), S * np.sin(P), C], -1).reshape(-1, 3)
    E = pb.far_field(x, dirs)
    w = (2 * wu)[:, None].repeat(len(ph), 1).reshape(-1) * (2 * math.pi / len(ph))
    sig_sca = np.sum(w * np.sum(abs(E) ** 2, 1))
    assert abs(sig_ext - sig_sca) < 0.02 * sig_sca


# ---------------------------------------------------------------------------
# GMRES, preconditioning, matvec counts
# ---------------------------------------------------------------------------
def test_gmres_matches_direct_solve():
    rng = np.random.default_rng(0)
    n = 60
    A = np.eye(n) * 3 + rng.normal(size=(n, n)) / math.sqrt(n) + 1j * rng.normal(size=(n, n)) / math.sqrt(n)
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    for restart in (200, 7):
        x, it, hist = pmchwt.gmres(lambda v: A @ v, b, 1e-12, restart, 1000)
        assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x)
        assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-11


def test_matvec_formula_reproduces_table2():
    # Table table:multiple_particle: P = D, M = 3, rho = 200
    rows = np.loadtxt(os.path.join(GOLDEN, "table2_matvecs.txt"), dtype=np.int64)
    per_it, init = pmchwt.matvec_units("D", 3)
    for R, mv in rows:
        assert per_it * (R + R // 200) + init == mv


@pytest.fixture(scope="module")
def sphere1_D():
    m = meshgen.icosphere(1)
    pb = pmchwt.PMCHWT(m.verts, m.tris, m.domain, 2.0, EPS, precond="D")
    pb.assemble()
    return pb


def test_calderon_gmres_solution_and_counter(sphere1_D):
    pb = sphere1_D
    x, info = pb.solve(INC, tol=1e-10, restart=200)
    xd = np.linalg.solve(pb.matrix_A(), pb.rhs(INC))
    assert np.linalg.norm(x - xd) < 1e-8 * np.linalg.norm(xd)
    # restarted: the counter follows Table tab:matvecs exactly
    for rho in (3, 5):
        x2, info2 = pb.solve(INC, tol=1e-6, restart=rho, maxit=500)
        R = info2["iterations"]
        assert info2["matvecs"] == 16 * (R + R // rho) + 8
        assert np.linalg.norm(x2 - xd) < 1e-4 * np.linalg.norm(xd)


def test_preconditioned_iterations_bounded_under_refinement(sphere1_D):
    # Calderón preconditioning: iteration counts do not grow with 1/h.
    it1 = sphere1_D.solve(INC, tol=1e-6)[1]["iterations"]
    m = meshgen.icosphere(2)
    pb2 = pmchwt.PMCHWT(m.verts, m.tris, m.domain, 2.0, EPS, precond="D")
    pb2.assemble()
    it2 = pb2.solve(INC, tol=1e-6)[1]["iterations"]
    pbI = pmchwt.PMCHWT(m.verts, m.tris, m.domain, 2.0, EPS, precond="I")
    pbI.assemble(need_bc=False)
    itI = pbI.solve(INC, tol=1e-6, maxit=3000)[1]["iterations"]
    assert it2 <= it1 + 3 and it2 <= 20
    assert itI > 3 * it2


def test_reduced_preconditioners_same_solution(sphere1_D):
    xd = np.linalg.solve(sphere1_D.matrix_A(), sphere1_D.rhs(INC))
    m = meshgen.icosphere(1)
    for pc, chi in (("Di", math.inf), ("Si", math.inf), ("Si", 0.4)):
        pb = pmchwt.PMCHWT(m.verts, m.tris, m.domain, 2.0, EPS, precond=pc, chi_P=chi,
                           rules_P=(1, 1) if chi < math.inf else (6, 4))
        pb.assemble()
        x, info = pb.solve(INC, tol=1e-9, maxit=400)
        assert np.linalg.norm(x - xd) < 1e-7 * np.linalg.norm(xd), pc
        per_it, init = pmchwt.matvec_units(pc, 1)
        assert info["matvecs"] == per_it * info["iterations"] + init


# ---------------------------------------------------------------------------
# discrete Calderón identities (eq. calderon_identities)
# ---------------------------------------------------------------------------
def _calderon_residuals(level, k=2.0):
    m = meshgen.icosphere(level)
    topo = spaces.Topology(m.verts, m.tris, m.domain)
    rwg, bc = spaces.rwg_space(topo), spaces.bc_space(topo)
    r = bem.Rules(6, 4)
    SR, CR = bem.assemble(rwg, rwg, k, r)
    SB, CB = bem.assemble(bc, bc, k, r)
    G = bem.gram_bc_rwg(rwg, bc)          # range BC, dual RWG
    Gp = -G.T                             # range RWG, dual BC
    # RWG interpolant of the tangential trace n x (x_hat e^{ikz}) at edge midpoints
    mid = 0.5 * (topo.verts[topo.edges[:, 0]] + topo.verts[topo.edges[:, 1]])
    t = topo.verts[topo.edges[:, 1]] - topo.verts[topo.edges[:, 0]]
    nrm = mid / np.linalg.norm(mid, axis=1)[:, None]
    mhat = np.cross(t, nrm)
    mhat /= np.linalg.norm(mhat, axis=1)[:, None]
    E = np.zeros((len(mid), 3), dtype=np.complex128)
    E[:, 0] = np.exp(1j * k * mid[:, 2])
    v = np.cross(nrm, E)
    # sign so that the flux runs from T+ to T-: m_hat points away from T+
    cp = topo.verts[topo.tris[topo.tplus]].mean(1)
    sgn = np.sign(np.einsum("ec,ec->e", mhat, mid - cp))
    x = np.einsum("ec,ec->e", v, mhat * sgn[:, None])
    ssx = np.linalg.solve(Gp, SB @ np.linalg.solve(G, SR @ x))
    ccx = np.linalg.solve(Gp, CB @ np.linalg.solve(G, CR @ x))
    csx = np.linalg.solve(Gp, CB @ np.linalg.solve(G, SR @ x))
    scx = np.linalg.solve(Gp, SB @ np.linalg.solve(G, CR @ x))
    nx = np.linalg.norm(x)
    return (np.linalg.norm(ssx - ccx + 0.25 * x) / nx, np.linalg.norm(csx + scx) / nx,
            np.linalg.norm(ssx) / nx)


@pytest.mark.slow
def test_discrete_calderon_identities_improve_with_h():
    r1 = _calderon_residuals(1)
    r2 = _calderon_residuals(2)
    # S^2 + 1/4 I - C^2 and CS + SC shrink under refinement (measured on levels
    # 1 -> 2: 5.3e-3 -> 2.3e-3 and 2.2e-3 -> 1.7e-3), while S^2 itself is O(1)
    assert r2[0] < 0.6 * r1[0] and r2[1] < 0.9 * r1[1]
    assert r2[0] < 0.02 * r2[2] and r2[1] < 0.02 * r2[2]


# ---------------------------------------------------------------------------
# the paper's scattered-trace right-hand side (1/2 I - D^i) u^inc
# ---------------------------------------------------------------------------
def test_scattered_rhs_vanishes_without_contrast():
    """With eps = mu = 1 the incident field is also an interior solution, so the
    interior Calderon projector reproduces its traces (A^i u^inc = u^inc / 2) and
    the scattered-trace right-hand side tends to zero under refinement (measured
    3.9e-2, 2.1e-2 of |<u^inc, dual>| at 80 and 320 triangles). A dropped 1/2,
    a sign error in D^i or a wrong projection of u^inc leaves an O(1) ratio."""
    ratios = []
    for level in (1, 2):
        m = meshgen.icosphere(level)
        pb = pmchwt.PMCHWT(m.verts, m.tris, m.domain, 2.0, 1.0, precond="I", rhs_mode="scattered")
        pb.assemble(need_bc=False)
        ratios.append(np.linalg.norm(pb.rhs(INC)) / np.linalg.norm(pb._tested_incident(INC)))
    assert ratios[1] < 0.03 and ratios[1] < 0.7 * ratios[0], ratios


def test_scattered_and_total_trace_far_fields_agree():
    """Solving for u^s with (1/2 I - D^i) u^inc and for the total trace with
    <u^inc, dual> gives the same far field up to the discretisation (measured
    1.3e-2 and 4.0e-3 at 80 and 320 triangles), and the scattered form also
    approaches Mie."""
    dirs = meshgen.sphere_cut_directions(37)
    diffs = []
    for level in (1, 2):
        m = meshgen.icosphere(level)
        F = {}
        for mode in ("total", "scattered"):
            pb = pmchwt.PMCHWT(m.verts, m.tris, m.domain, 2.0, EPS, precond="I", rhs_mode=mode)
            pb.assemble(need_bc=False)
            x = np.linalg.solve(pb.matrix_A(), pb.rhs(INC))
            F[mode] = pb.far_field(x, dirs)
        diffs.append(np.linalg.norm(F["total"] - F["scattered"]) / np.linalg.norm(F["total"]))
    assert diffs[1] < 1e-2 and diffs[1] < 0.5 * diffs[0], diffs
    Fm = mie.far_field(2.0, 1.0, EPS, dirs)
    assert np.linalg.norm(F["scattered"] - Fm) / np.linalg.norm(Fm) < 0.05


def test_three_cube_iterations_near_table2():
    """The three-cube benchmark of Section 4 at k_e = 2.1 (cube side 0.4, corners
    at x = -1, 0, 1, n = 1.311 + 2.289e-9 i, E^inc = z e^{ik_e x}, h = 2 pi/(10 k_e),
    GMRES tol 1e-5, restart 200) with P = D. The paper's mesh has N = 378, ours
    N = 216, so the comparison with Table 2 is soft: its first rows print 6
    iterations for q_P = (4,3,2,6) and 7 for (1,1,1,1); the oracle gives 6 and 8."""
    k = 2.1
    eps = (1.311 + 2.289e-9j) ** 2
    inc = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    m = meshgen.three_cubes(2 * math.pi / (10 * k))
    its = {}
    for rules_P in ((6, 4), (1, 1)):
        pb = pmchwt.PMCHWT(m.verts, m.tris, m.domain, k, eps, precond="D", rules_P=rules_P)
        pb.assemble()
        _, info = pb.solve(inc, tol=1e-5, restart=200, maxit=2000)
        its[rules_P] = info["iterations"]
    assert 5 <= its[(6, 4)] <= 8 and 6 <= its[(1, 1)] <= 10, its
    assert its[(1, 1)] >= its[(6, 4)]
