"""Quadrature rules of the oracle (test infrastructure; see ``oracle/__init__``).

Section 3.3 of the paper: regular pairs use a tensor product of symmetric
triangle rules — order 4 -> 6 points per triangle (36 evaluations per pair),
order 3 -> 4 points (16), order 2 -> 3 points (9), order 1 -> 1 point; the
order of a pair follows its near / medium / far class (defaults q_near,
q_medium, q_far = 4, 3, 2). Singular pairs use Sauter–Schwab rules whose 4D
Gauss product has q**4 points per sub-region (q = 4: 1536/1280/512
evaluations for coincident/edge/vertex pairs, q = 1: 6/5/2).

Near / medium / far (the paper names the classes, not their bounds): a pair
is near if |c1 - c2| <= 2 max(d1, d2), medium if <= 4 max(d1, d2), far
otherwise, with c the centroids and d the longest edges of the triangles.
The bounds carry a relative margin of 2^-20, so that pairs exactly at 2 or 4
(common on structured meshes) fall on the same side in every precision.
"""
import numpy as np


def gauss_legendre_01(n: int):
    """n-point Gauss–Legendre rule on [0, 1] by the Golub–Welsch eigenvalue method."""
    if n == 1:
        return np.array([0.5]), np.array([1.0])
    k = np.arange(1, n, dtype=np.float64)
    beta = k / np.sqrt(4.0 * k * k - 1.0)
    J = np.diag(beta, 1) + np.diag(beta, -1)
    t, V = np.linalg.eigh(J)
    w = 2.0 * V[0, :] ** 2
    return 0.5 * (t + 1.0), 0.5 * w


# Dunavant (1985), degree-4 six-point symmetric rule on the triangle, from
# the published table: barycentric (a, a, 1-2a) and (b, b, 1-2b), weights
# normalised to sum to 1.
_DUNAVANT6 = ((0.445948490915965, 0.223381589678011),
              (0.091576213509771, 0.109951743655322))


# relative distance bounds of the near and medium classes (see the module note)
CLASS_BOUNDS = (2.0 * (1.0 + 2.0 ** -20), 4.0 * (1.0 + 2.0 ** -20))
# points per triangle of the near, medium and far rules at the default orders
CLASS_POINTS = (6, 4, 3)


def triangle_rule(npts: int):
    """Symmetric triangle rule: barycentric points [n, 3] and weights [n] summing to 1.

    npts = 6: degree 4 (Dunavant); npts = 4: degree 3 (Strang–Fix: centroid
    with weight -27/48 and the three points (3/5, 1/5, 1/5) with 25/48);
    npts = 3: degree 2 (Strang–Fix, (2/3, 1/6, 1/6)); npts = 1: centroid.
    """
    if npts == 1:
        return np.array([[1 / 3, 1 / 3, 1 / 3]]), np.array([1.0])
    if npts == 4:
        b = np.array([[1 / 3, 1 / 3, 1 / 3], [3 / 5, 1 / 5, 1 / 5], [1 / 5, 3 / 5, 1 / 5],
                      [1 / 5, 1 / 5, 3 / 5]])
        return b, np.array([-27 / 48, 25 / 48, 25 / 48, 25 / 48])
    if npts == 3:
        b = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])
        return b, np.full(3, 1.0 / 3.0)
    if npts == 6:
        pts, wts = [], []
        for a, w in _DUNAVANT6:
            c = 1.0 - 2.0 * a
            for p in ((c, a, a), (a, c, a), (a, a, c)):
                pts.append(p)
                wts.append(w)
        return np.array(pts), np.array(wts)
    raise ValueError(f"no {npts}-point triangle rule")


def regular_points_for_order(q: int) -> int:
    """Paper's regular order -> points per triangle (Section 3.3): 4 -> 6, 3 -> 4, 2 -> 3, 1 -> 1."""
    return {4: 6, 3: 4, 2: 3, 1: 1}[q]


def singular_gauss_for_order(q: int) -> int:
    """Paper's q_singular -> Gauss points per dimension: 6 -> 4 (4**4*{6,5,2}), 1 -> 1."""
    return {6: 4, 1: 1}[q]
