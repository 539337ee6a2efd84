"""Pins of the oracle's quadrature rules and Sauter–Schwab maps (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import bem
from oracle.quadrature import gauss_legendre_01, triangle_rule

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n", [1, 2, 4, 8])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = gauss_legendre_01(n)
    for p in range(2 * n):
        assert abs(np.dot(w, x ** p) - 1.0 / (p + 1)) < 1e-14
    # and not exact one degree higher (so a wrong rule cannot pass by accident)
    assert abs(np.dot(w, x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-12


@pytest.mark.parametrize("npts,degree", [(1, 1), (3, 2), (4, 3), (6, 4)])
def test_triangle_rule_exact_monomials(npts, degree):
    # int over the unit triangle of l1^a l2^b l3^c, normalised by area:
    # 2 a! b! c! / (a+b+c+2)!
    bary, w = triangle_rule(npts)
    assert abs(w.sum() - 1.0) < 1e-14
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            for c in range(degree + 1 - a - b):
                exact = 2.0 * math.factorial(a) * math.factorial(b) * math.factorial(c) / \
                    math.factorial(a + b + c + 2)
                got = np.sum(w * bary[:, 0] ** a * bary[:, 1] ** b * bary[:, 2] ** c)
                assert abs(got - exact) < 1e-14, (a, b, c)


def test_dunavant_table_matches_closed_form():
    # Closed form of the degree-4 six-point rule (Strang–Fix / Dunavant).
    s10, s25 = math.sqrt(10.0), math.sqrt(0.4)
    a = (8 - s10 + math.sqrt(38 - 44 * s25)) / 18
    b = (8 - s10 - math.sqrt(38 - 44 * s25)) / 18
    wa = (620 + math.sqrt(213125 - 53320 * s10)) / 3720
    wb = (620 - math.sqrt(213125 - 53320 * s10)) / 3720
    bary, w = triangle_rule(6)
    assert np.allclose(sorted(set(np.round(bary[:, 1], 15))), sorted([a, 1 - 2 * a, b, 1 - 2 * b]),
                       atol=1e-14)
    assert np.allclose(sorted(set(np.round(w, 15))), sorted([wb, wa]), atol=1e-14)


def _tri_pair(cls, seed=0):
    """Non-coplanar triangle pair sharing 3/2/1 vertices, with canonical orders."""
    rng = np.random.default_rng(seed)
    A, B, C1, C2, D = rng.normal(size=(5, 3))
    if cls == 3:
        P1 = np.array([A, B, C1]); P2 = P1.copy()
        return P1, P2, [0, 1, 2], [0, 1, 2]
    if cls == 2:
        P1 = np.array([A, B, C1]); P2 = np.array([B, A, C2])
        return P1, P2, [0, 1, 2], [1, 0, 2]
    P1 = np.array([A, B, C1]); P2 = np.array([C2, D, A])
    return P1, P2, [0, 1, 2], [2, 0, 1]


def _poly_tri_integral(P, pw):
    """int_T prod_c (1 + x_c)^pw_c by the degree-4 rule (exact for total degree <= 4)."""
    bary, w = triangle_rule(6)
    area = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
    x = bary @ P
    return area * np.sum(w * np.prod((1 + x) ** np.asarray(pw)[None, :], axis=1))


@pytest.mark.parametrize("cls", [1, 2, 3])
def test_sauter_schwab_maps_integrate_polynomials_exactly(oracle_lib, cls):
    # The sub-region maps must carry the product measure of T1 x T2: for a
    # separable polynomial kernel the result is the product of two plain
    # triangle integrals. A wrong region, Jacobian or vertex order fails this.
    P1, P2, o1, o2 = _tri_pair(cls, seed=cls)
    gx, gw = gauss_legendre_01(8)
    import ctypes
    for px, py in [((0, 0, 0), (0, 0, 0)), ((1, 0, 0), (0, 1, 0)), ((2, 1, 0), (0, 0, 2)),
                   ((0, 2, 2), (1, 1, 1)), ((1, 1, 2), (3, 0, 1))]:
        args = [np.ascontiguousarray(a, dtype=t) for a, t in
                ((P1, np.float64), (P2, np.float64), (o1, np.int32), (o2, np.int32),
                 (px, np.int32), (py, np.int32), (gx, np.float64), (gw, np.float64))]
        ptr = [a.ctypes.data_as(ctypes.c_void_p) for a in args]
        got = oracle_lib.orc_ss_polynomial(ptr[0], ptr[1], cls, ptr[2], ptr[3], ptr[4], ptr[5],
                                           8, ptr[6], ptr[7])
        exact = _poly_tri_integral(P1, px) * _poly_tri_integral(P2, py)
        assert abs(got - exact) < 1e-12 * max(1.0, abs(exact)), (px, py, got, exact)


def test_evaluation_counts_match_paper(oracle_lib):
    # Section 3.3: 36 / 1 regular evaluations; 512/1280/1536 and 2/5/6 singular.
    rows = np.loadtxt(os.path.join(GOLDEN, "quadrature_counts.txt"), dtype=np.int64)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0.3], [-1, 0.2, 0.1],
                  [5, 5, 5], [6, 5, 5], [5, 6, 5]], dtype=np.float64)
    ids = np.array([[0, 1, 2], [1, 3, 2], [0, 2, 4], [5, 6, 7], [3, 1, 0]])
    # pairs: (0,0) identical, (0,1) edge, (0,2) edge, (0,3) regular, (1,2) vertex
    for nreg, ng, reg, vtx, edg, idn in rows:
        rules = bem.Rules(int(nreg), int(ng))
        for test, trial, col, expect in [([0], [0], 3, idn), ([0], [1], 2, edg), ([0], [3], 0, reg),
                                         ([1], [2], 1, vtx)]:
            cnt = np.zeros(4, dtype=np.int64)
            bem.local_blocks(X, ids, test, trial, 1.0, rules, 3, cnt)
            assert cnt[col] == expect and cnt.sum() == expect


@pytest.mark.parametrize("rel,expect", [(1.5, 36), (3.0, 16), (6.0, 9)])
def test_regular_class_by_relative_distance(oracle_lib, rel, expect):
    # Section 3.3: the default orders (4, 3, 2) give 36 / 16 / 9 evaluations for
    # near / medium / far pairs; the class follows |c1 - c2| / max(d1, d2)
    # (bounds 2 and 4). Two copies of a right triangle (longest edge sqrt 2).
    T = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    L = rel * math.sqrt(2.0)
    X = np.concatenate([T, T + np.array([0.0, 0.0, L])])
    ids = np.array([[0, 1, 2], [3, 4, 5]])
    cnt = np.zeros(4, dtype=np.int64)
    bem.local_blocks(X, ids, [0], [1], 1.5, bem.Rules(0, 4), 3, cnt)
    assert cnt[0] == expect and cnt.sum() == expect


@pytest.mark.parametrize("rel", [3.0, 6.0, 12.0])
def test_medium_and_far_rules_approach_the_near_rule(oracle_lib, rel):
    # The cheaper rules integrate the same smooth integrand: the classed blocks
    # of a medium or far pair stay within the low-order rules' error of the
    # 36-point ones (about (k d)^3 for the oscillatory factor, d the element size).
    rng = np.random.default_rng(int(rel))
    T1 = rng.normal(size=(3, 3)) * 0.5
    T2 = rng.normal(size=(3, 3)) * 0.5
    d = max(np.linalg.norm(T1[(a + 1) % 3] - T1[a]) for a in range(3))
    d = max(d, max(np.linalg.norm(T2[(a + 1) % 3] - T2[a]) for a in range(3)))
    shift = np.array([1.0, 0.3, -0.2]) / np.linalg.norm([1.0, 0.3, -0.2])
    c1, c2 = T1.mean(0), T2.mean(0)
    T2 = T2 - c2 + c1 + shift * rel * d * 1.01
    X = np.concatenate([T1, T2])
    ids = np.array([[0, 1, 2], [3, 4, 5]])
    errs = []
    # wavenumbers with k d about 0.5 and 0.25, as on a mesh of several elements per wavelength
    for k in (0.5 / d, 0.25 / d * (1.0 + 0.02j)):
        Sc, Cc = bem.local_blocks(X, ids, [0], [1], k, bem.Rules(0, 4))
        Sn, Cn = bem.local_blocks(X, ids, [0], [1], k, bem.Rules(6, 4))
        errs.append(max(np.abs(Sc - Sn).max() / np.abs(Sn).max(), np.abs(Cc - Cn).max() / np.abs(Cn).max()))
        assert not np.allclose(Sc, Sn, rtol=1e-14, atol=0)  # a different rule was used
    assert max(errs) < {3.0: 1e-3, 6.0: 5e-4, 12.0: 5e-4}[rel], errs
