"""Pins of the oracle's near-field evaluation (the paper's |E|^2 plots, Section 5).

The field at points off the surface comes from the Stratton–Chu representations
with the potential operators E_k and H_k (``oracle/field.py``). It is pinned by
(1) the winding number of a closed mesh, (2) the far field: R e^{-ikR} E^s(R x)
tends to the oracle's separately derived far field like 1/R, and (3) the
extinction theorem: the exterior representation vanishes inside the scatterer
and the interior one outside, to discretisation level falling with h. A wrong
scaling of the second trace or a flipped H term leaves O(1) residues.
"""
import numpy as np
import pytest

from oracle import field, pmchwt
from paper_2008_04772_gb300 import meshgen

INC = meshgen.plane_wave_x_along_z()[0]
EPS = 3.17 + 0.01j
PTS_IN = np.array([[0.0, 0.0, 0.0], [0.3, 0.1, -0.2], [-0.2, 0.4, 0.1]])
PTS_OUT = np.array([[2.0, 0.0, 0.0], [0.0, 1.6, 0.5], [-1.2, -1.3, 0.4]])


def _solved(level):
    m = meshgen.icosphere(level)
    pb = pmchwt.PMCHWT(m.verts, m.tris, m.domain, 2.0, EPS, precond="I")
    pb.assemble(need_bc=False)
    return m, pb, np.linalg.solve(pb.matrix_A(), pb.rhs(INC))


@pytest.fixture(scope="module")
def solved():
    return {lvl: _solved(lvl) for lvl in (1, 2)}


def test_winding_number_of_closed_sphere():
    m = meshgen.icosphere(2)
    assert np.allclose(field.winding_number(m.verts, m.tris, PTS_IN), 1.0, atol=1e-12)
    assert np.allclose(field.winding_number(m.verts, m.tris, PTS_OUT), 0.0, atol=1e-12)


def test_composite_rule_integrates_exactly():
    """4^s sub-triangles, 6-point rule each: weights sum to 1, degree 4 exact."""
    for s in (0, 1, 2):
        b, w = field.composite_rule(s)
        assert abs(w.sum() - 1.0) < 1e-14
        # mean over a triangle of l1^a l2^b l3^c = 2 a! b! c! / (a + b + c + 2)!:
        # l1^2 l2^2 gives 8/720
        assert abs(np.sum(w * b[:, 0] ** 2 * b[:, 1] ** 2) - 8 / 720) < 1e-13


def test_far_field_limit(solved):
    _, pb, x = solved[2]
    dirs = meshgen.fibonacci_directions(8)
    Finf = pb.far_field(x, dirs)
    errs = []
    for R in (250.0, 1000.0):
        P = R * dirs
        Es = field.electric_field(pb, x, INC, P, levels=0, region=-np.ones(len(P), int)) \
            - field.incident_field(pb.k_e, INC, P)
        errs.append(np.linalg.norm(Es * R * np.exp(-1j * pb.k_e * R) - Finf) / np.linalg.norm(Finf))
    # measured 4.0e-3 and 9.9e-4: the 1/R term of the expansion
    assert errs[1] < 2e-3 and 3.0 < errs[0] / errs[1] < 5.0, errs


def test_extinction_inside_and_outside(solved):
    """Exterior formula at interior points and interior formula at exterior
    points: measured 3.2e-3 / 3.3e-3 at 80 triangles, 3.7e-4 / 3.4e-4 at 320."""
    res = []
    for lvl in (1, 2):
        _, pb, x = solved[lvl]
        e_in = field.electric_field(pb, x, INC, PTS_IN, levels=2, region=-np.ones(3, int))
        i_out = field.electric_field(pb, x, INC, PTS_OUT, levels=2, region=np.zeros(3, int))
        E_out = field.electric_field(pb, x, INC, PTS_OUT, levels=2)
        Einc = field.incident_field(pb.k_e, INC, PTS_IN)
        res.append((np.linalg.norm(e_in) / np.linalg.norm(Einc), np.linalg.norm(i_out) / np.linalg.norm(E_out)))
    assert max(res[1]) < 2e-3, res
    assert res[1][0] < 0.3 * res[0][0] and res[1][1] < 0.3 * res[0][1], res
