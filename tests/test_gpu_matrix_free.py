"""PMCHWT operator application: stored and matrix-free, against the oracle.

cal_problem_apply gives y = A x with the problem's operator (eqs.
multiple_operator, AimAem). The oracle's dense A uses per-scatterer
(x1, x2) ordering and the swapped test rows of the paper's block form; the
permutation between the two is a relabelling only.
"""
import numpy as np
import pytest

from gpu_common import EPS, mesh, rel
from oracle import pmchwt
from paper_2008_04772_gb300 import cal, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2008_04772_gb300 import build
    build.build()
    return cal.Context(0)


def _oracle_to_gpu(P, xo):
    """Oracle unknowns (per scatterer: x1 block, x2 block) -> [x1 (all), x2 (all)]."""
    N = P.N_e
    x = np.zeros(2 * N, dtype=np.complex128)
    for a, b in P.edge_ranges:
        n = b - a
        x[a:b] = xo[2 * a:2 * a + n]
        x[N + a:N + b] = xo[2 * a + n:2 * b]
    return x


def _oracle_rows_to_gpu(P, yo):
    """Oracle rows ((-k/mu) S x1 + C x2; C x1 + (mu/k) S x2) -> GPU (y1, y2)."""
    N = P.N_e
    y = np.zeros(2 * N, dtype=np.complex128)
    for a, b in P.edge_ranges:
        n = b - a
        y[N + a:N + b] = yo[2 * a:2 * a + n]
        y[a:b] = yo[2 * a + n:2 * b]
    return y


def _oracle_apply(name, k, nreg=6):
    m = mesh(name)
    P = pmchwt.PMCHWT(m.verts, m.tris, m.domain, k, EPS, rules_A=(nreg, 4))
    P.assemble(need_bc=False)
    A = P.matrix_A()
    rng = np.random.default_rng(5)
    xo = rng.normal(size=(2, A.shape[0])) + 1j * rng.normal(size=(2, A.shape[0]))
    yo = xo @ A.T
    X = np.stack([_oracle_to_gpu(P, v) for v in xo])
    Y = np.stack([_oracle_rows_to_gpu(P, v) for v in yo])
    return m, X, Y


@pytest.mark.parametrize("name,k", [("sphere2", 2.0), ("prisms2", 3.0)])
@pytest.mark.parametrize("free", [0, 1])
@pytest.mark.parametrize("nreg", [6, 0])
def test_operator_fp64_matches_oracle(ctx, name, k, free, nreg):
    m, X, Y = _oracle_apply(name, k, nreg)
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    prob = cal.Problem(ctx, gm, k, EPS, opts=cal.solve_opts(precond="none", precision=cal.FP64, matrix_free=free,
                                                            q_regular_A=nreg))
    Yg = prob.apply(X)
    assert rel(Yg, Y) < 1e-11, rel(Yg, Y)
    if free:
        # only the touching-pair entries are stored
        assert prob.info().bytes_A < 0.2 * 2 * (len(m.tris) * 1.5) ** 2 * 16 * 2


@pytest.mark.parametrize("name,k", [("sphere3", 4.0), ("prisms2", 3.0), ("cubes", 2.0)])
def test_matrix_free_fp32_equals_stored(ctx, name, k):
    m = mesh(name)
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    N = gm.info().n_edges
    rng = np.random.default_rng(7)
    X = rng.normal(size=(3, 2 * N)) + 1j * rng.normal(size=(3, 2 * N))
    o = dict(precond="none", precision=cal.FP32)
    ys = cal.Problem(ctx, gm, k, EPS, opts=cal.solve_opts(**o)).apply(X)
    yf = cal.Problem(ctx, gm, k, EPS, opts=cal.solve_opts(matrix_free=1, **o)).apply(X)
    # the same float32 entries, summed in another order
    assert rel(yf, ys) < 2e-6, rel(yf, ys)
    for j in range(3):
        assert rel(yf[j], ys[j]) < 2e-6


def test_matrix_free_solve_equals_stored_solve(ctx):
    m = mesh("prisms2")
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    d = meshgen.fibonacci_directions(3)
    inc = np.concatenate([d, meshgen.perpendicular_polarisation(d)], 1)
    dirs = meshgen.fibonacci_directions(32)
    F = {}
    for free in (0, 1):
        o = cal.solve_opts(precond="Di", near_cutoff_P=2.0, precision=cal.FP32, tol=1e-7, matrix_free=free)
        s = cal.pmchwt_solve(ctx, gm, 3.0, EPS, inc, opts=o)
        assert s.info().converged == 1
        F[free] = s.far_field(dirs)
    assert rel(F[1], F[0]) < 1e-5


def test_matrix_free_fp64_solve_matches_oracle(ctx):
    m = mesh("sphere2")
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    inc = meshgen.plane_wave_x_along_z()
    dirs = meshgen.fibonacci_directions(16)
    P = pmchwt.PMCHWT(m.verts, m.tris, m.domain, 2.0, EPS, precond="I")
    P.assemble(need_bc=False)
    xo = np.linalg.solve(P.matrix_A(), P.rhs(inc[0]))
    Fo = P.far_field(xo, dirs)
    o = cal.solve_opts(precond="D", precision=cal.FP64, tol=1e-11, matrix_free=1)
    Fg = cal.pmchwt_solve(ctx, gm, 2.0, EPS, inc, opts=o).far_field(dirs)[0]
    assert rel(Fg, Fo) < 1e-8, rel(Fg, Fo)


@pytest.mark.parametrize("name,k", [("sphere3", 4.0), ("prisms2", 3.0)])
def test_fp32_operator_fp64_vectors_multi_equals_single(ctx, name, k):
    """Float64 vectors on a float32 operator: several vectors at once (thread
    per row, vectors staged in shared memory) and one vector at a time (warp
    per row chunk, warp reduction) are two double-float (float32 pair)
    implementations of the exact product of the float32 entries; they agree
    far below float32 rounding: bar 1e-12 relative (~2^-48 per term)."""
    m = mesh(name)
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    N = gm.info().n_edges
    rng = np.random.default_rng(11)
    X = rng.normal(size=(5, 2 * N)) + 1j * rng.normal(size=(5, 2 * N))
    prob = cal.Problem(ctx, gm, k, EPS, opts=cal.solve_opts(precond="none", precision=cal.FP32))
    Ym = prob.apply(X)
    for j in range(5):
        y1 = prob.apply(X[j:j + 1])[0]
        assert rel(Ym[j], y1) < 1e-12, (j, rel(Ym[j], y1))
