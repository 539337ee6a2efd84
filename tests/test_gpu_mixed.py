"""The mixed (RWG, BC) discretisation on the GPU (eq. mixed_discretisation).

Each scatterer's traces in (RWG_m, BC_m) for trial and test alike, RWG written
on the barycentric refinement for the blocks C(RWG, BC) and C(BC, RWG), P = D
reusing A's diagonal blocks. Against the oracle (``oracle/mixed.py``):
the operator applied to random vectors (every block at once), the solution
coefficients and far field (float64, 1e-8), and Table 2's last row on the three
cubes (5 iterations at k_e = 2.1).
"""
import math

import numpy as np
import pytest

from gpu_common import EPS, mesh, rel
from oracle import mixed
from paper_2008_04772_gb300 import cal, meshgen

pytestmark = pytest.mark.gpu
INC = meshgen.plane_wave_x_along_z()


@pytest.fixture(scope="module")
def ctx():
    from paper_2008_04772_gb300 import build
    build.build()
    return cal.Context(0)


_cache = {}


def oracle(name, k, eps=EPS):
    key = (name, k, eps)
    if key not in _cache:
        m = mesh(name)
        mp = mixed.MixedPMCHWT(m.verts, m.tris, m.domain, k, eps)
        mp.assemble()
        _cache[key] = mp
    return _cache[key]


def opts_mixed(**kw):
    return cal.solve_opts(precond="D", precision=cal.FP64, discretisation=1, **kw)


@pytest.mark.parametrize("name,k", [("sphere1", 2.0), ("cubes", 2.1)])
def test_mixed_operator_matches_oracle(ctx, name, k):
    mp = oracle(name, k)
    m = mesh(name)
    prob = cal.Problem(ctx, cal.Mesh(ctx, m.verts, m.tris, m.domain), k, EPS, opts=opts_mixed())
    n = mp.N_e
    rng = np.random.default_rng(3)
    c = rng.normal(size=n) + 1j * rng.normal(size=n)
    d = rng.normal(size=n) + 1j * rng.normal(size=n)
    y = prob.apply(np.concatenate([c, d])[None, :])[0]
    y1, y2 = mp.base.split(mp.matrix_A() @ mp.base._paper_order(c, d))
    assert rel(y, np.concatenate([y1, y2])) < 1e-10, rel(y, np.concatenate([y1, y2]))


@pytest.mark.parametrize("name,k", [("sphere1", 2.0), ("sphere2", 2.0), ("cubes", 2.1)])
def test_mixed_solution_matches_oracle(ctx, name, k):
    mp = oracle(name, k)
    m = mesh(name)
    xo = np.linalg.solve(mp.matrix_A(), mp.rhs(INC[0]))
    sol = cal.pmchwt_solve(ctx, cal.Mesh(ctx, m.verts, m.tris, m.domain), k, EPS, INC, opts=opts_mixed(tol=1e-11))
    c, d = mp.base.split(xo)
    assert rel(sol.coefficients()[0], np.concatenate([c, d])) < 1e-8
    dirs = meshgen.sphere_cut_directions(19)
    assert rel(sol.far_field(dirs)[0], mp.far_field(xo, dirs)) < 1e-8


def test_mixed_three_cubes_iterations():
    """Table 2's last row (mixed discretisation, P = D, k_e = 2.1): 5 iterations;
    the oracle on this mesh: 5."""
    from paper_2008_04772_gb300 import build
    build.build()
    ctx = cal.Context(0)
    k = 2.1
    eps = (1.311 + 2.289e-9j) ** 2
    inc = np.array([[1.0, 0.0, 0.0, 0.0, 0.0, 1.0]])
    m = meshgen.three_cubes(2 * math.pi / (10 * k))
    info = cal.pmchwt_solve(ctx, cal.Mesh(ctx, m.verts, m.tris, m.domain), k, eps, inc,
                            opts=opts_mixed(tol=1e-5, restart=200)).info()
    assert 4 <= info.iterations <= 6, info.iterations
    assert info.matvecs == 72 * info.iterations + 24


def test_mixed_rejects_unsupported_options(ctx):
    m = mesh("sphere1")
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    for bad in (dict(precision=cal.FP32), dict(precond="Di"), dict(rhs_mode=1)):
        o = dict(precond="D", precision=cal.FP64, discretisation=1)
        o.update(bad)
        with pytest.raises(cal.CalError):
            cal.pmchwt_solve(ctx, gm, 2.0, EPS, INC, opts=cal.solve_opts(**o))
