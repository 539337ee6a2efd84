"""Near field on the GPU (cal_near_field) against the oracle (``oracle/field.py``).

The total field at points off the surface from the Stratton–Chu representations
with the potential operators E_k, H_k (Section 2; the |E|^2 maps of Section 5).
Element-by-element parity with the oracle on the same traces and the same
composite rule: float64 to 1e-8, float32-bulk solutions to 1e-4; the regions
from the winding numbers equal the oracle's exactly.
"""
import numpy as np
import pytest

from gpu_common import EPS, mesh, rel
from oracle import field, pmchwt
from paper_2008_04772_gb300 import cal, meshgen

pytestmark = pytest.mark.gpu
INC = meshgen.plane_wave_x_along_z()

SPHERE_PTS = np.array([[0.0, 0.0, 0.0], [0.3, 0.1, -0.2], [-0.2, 0.4, 0.1], [0.1, -0.5, 0.3],
                       [2.0, 0.0, 0.0], [0.0, 1.6, 0.5], [-1.2, -1.3, 0.4], [0.3, 0.2, 3.0]])
# the cubes span [x0, x0 + 0.4] x [0, 0.4] x [0, 0.4], x0 = -1, 0, 1
CUBE_PTS = np.array([[-0.8, 0.2, 0.2], [0.2, 0.15, 0.25], [1.2, 0.22, 0.18], [0.25, 0.2, 0.15],
                     [0.7, 0.2, 0.2], [0.2, 1.0, 0.2], [-2.0, 0.5, 0.5], [1.5, -0.4, 0.6]])


@pytest.fixture(scope="module")
def ctx():
    from paper_2008_04772_gb300 import build
    build.build()
    return cal.Context(0)


_cache = {}


def oracle(name, k):
    if (name, k) not in _cache:
        m = mesh(name)
        pb = pmchwt.PMCHWT(m.verts, m.tris, m.domain, k, EPS, precond="I")
        pb.assemble(need_bc=False)
        _cache[(name, k)] = (pb, np.linalg.solve(pb.matrix_A(), pb.rhs(INC[0])))
    return _cache[(name, k)]


def gpu_solution(ctx, name, k, precision, tol):
    m = mesh(name)
    return cal.pmchwt_solve(ctx, cal.Mesh(ctx, m.verts, m.tris, m.domain), k, EPS, INC,
                            opts=cal.solve_opts(precond="D", precision=precision, tol=tol))


@pytest.mark.parametrize("name,k,pts", [("sphere2", 2.0, SPHERE_PTS), ("cubes", 2.1, CUBE_PTS)])
def test_fp64_near_field_matches_oracle(ctx, name, k, pts):
    pb, xd = oracle(name, k)
    sol = gpu_solution(ctx, name, k, cal.FP64, 1e-12)
    E, reg = sol.near_field(pts, levels=2)
    # regions: the oracle's winding numbers, exactly
    ref_reg = -np.ones(len(pts), dtype=int)
    for mm in range(pb.M):
        sel = np.nonzero(np.asarray(pb.topo.domain) == mm)[0]
        ref_reg[field.winding_number(pb.topo.verts, pb.topo.tris[sel], pts) > 0.5] = mm
    assert np.array_equal(reg, ref_reg), (reg, ref_reg)
    Eo = field.electric_field(pb, xd, INC[0], pts, levels=2)
    assert rel(E[0], Eo) < 1e-8, rel(E[0], Eo)
    for i in range(len(pts)):
        assert rel(E[0, i], Eo[i]) < 1e-7, i


def test_fp32_near_field_within_1e4(ctx):
    pb, xd = oracle("sphere2", 2.0)
    sol = gpu_solution(ctx, "sphere2", 2.0, cal.FP32, 1e-7)
    E, _ = sol.near_field(SPHERE_PTS, levels=2)
    Eo = field.electric_field(pb, xd, INC[0], SPHERE_PTS, levels=2)
    assert rel(E[0], Eo) < 1e-4, rel(E[0], Eo)


def test_given_regions_and_levels(ctx):
    # the exterior formula evaluated at interior points (extinction theorem) and
    # another composite level, both against the oracle with the same regions
    pb, xd = oracle("sphere2", 2.0)
    sol = gpu_solution(ctx, "sphere2", 2.0, cal.FP64, 1e-12)
    pts = SPHERE_PTS[:4]
    E, reg = sol.near_field(pts, levels=1, region=-np.ones(4, dtype=np.int32))
    assert np.all(reg == -1)
    Eo = field.electric_field(pb, xd, INC[0], pts, levels=1, region=-np.ones(4, int))
    assert rel(E[0], Eo) < 1e-8
    # the total field there nearly vanishes (extinction, discretisation level)
    assert np.linalg.norm(E[0]) < 2e-2 * np.linalg.norm(field.incident_field(2.0, INC[0], pts))


def test_scattered_trace_solution_near_field(ctx):
    # rhs_mode 1 keeps the projected incident coefficients, so its total traces
    # give the same near field as the total-trace solve to discretisation level
    m = mesh("sphere2")
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    E = {}
    for mode in (0, 1):
        sol = cal.pmchwt_solve(ctx, gm, 2.0, EPS, INC, opts=cal.solve_opts(
            precond="D", precision=cal.FP64, tol=1e-10, rhs_mode=mode))
        E[mode] = sol.near_field(SPHERE_PTS, levels=2)[0][0]
    assert rel(E[1], E[0]) < 2e-2, rel(E[1], E[0])


def test_bad_arguments(ctx):
    sol = gpu_solution(ctx, "sphere1", 2.0, cal.FP32, 1e-5)
    with pytest.raises(cal.CalError):
        sol.near_field(SPHERE_PTS[:2], levels=5)
    with pytest.raises(cal.CalError):
        sol.near_field(SPHERE_PTS[:2], region=np.array([0, 3], dtype=np.int32))
