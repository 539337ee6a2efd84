"""Electric field at points off the surface (test infrastructure; see ``oracle``).

The paper's |E|^2 plots on a plane (Section 5, the figure of the 8-branch
aggregate) evaluate the Stratton–Chu representations, eqs. StrattonChu_int and
StrattonChu_ext, with the electric and magnetic potential operators of
Section 2:

    E_k v(x) = ik int v G - (1/(ik)) grad_x int div v G,
    H_k v(x) = curl_x int v G,         G = e^{ik|x-y|} / (4 pi |x-y|),

so that with grad_x G = (x - y) g, g = (ik r - 1) e^{ikr} / (4 pi r^3),

    E_k v(x) = sum w [ik v G - (1/(ik)) div v (x - y) g],
    H_k v(x) = sum w g (x - y) x v.

Fields from the solved traces (paper ordering, second component scaled by
k/mu, see ``pmchwt``):

    x in Omega_e:    E = E^inc - sum_m [H^e(gamma_D E) + E^e(gamma_N^+ E)]
    x in Omega^i_m:  E = H^i_m(gamma_D E) + E^i_m(gamma_N^- E)

with gamma_N^+ E = (mu_e/k_e) d and gamma_N^- E = (mu_m/k_m) d for the second
trace component d. Total traces may stand in the exterior formula because the
incident field radiates nothing outside. Which region a point lies in comes
from the winding number of each scatterer's closed triangle mesh (the solid
angle of Van Oosterom and Strackee, IEEE Trans. Biomed. Eng. 30, 1983).

Quadrature: each triangle split into 4^s congruent sub-triangles with the
6-point rule on each; points should keep a distance of a few sub-triangle
sizes from the surface.
"""
from __future__ import annotations

import numpy as np

from .quadrature import triangle_rule


def composite_rule(levels: int):
    """Barycentric points [q, 3] and weights [q] (sum 1): the 6-point rule on the
    4^levels sub-triangles of a uniform midpoint subdivision."""
    tris = [np.eye(3)]                           # rows: barycentric vertices
    for _ in range(levels):
        nxt = []
        for T in tris:
            a, b, c = T
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array([a, ab, ca]), np.array([ab, b, bc]), np.array([ca, bc, c]),
                    np.array([ab, bc, ca])]
        tris = nxt
    b6, w6 = triangle_rule(6)
    pts = np.concatenate([b6 @ T for T in tris])
    wts = np.concatenate([w6 / len(tris) for _ in tris])
    return pts, wts


def winding_number(verts, tris, points):
    """Solid angle of the closed oriented mesh seen from each point / 4 pi:
    1 inside (outward normals), 0 outside."""
    P = np.asarray(points, dtype=np.float64)
    V = np.asarray(verts, dtype=np.float64)
    T = np.asarray(tris)
    out = np.zeros(len(P))
    for i, x in enumerate(P):
        a = V[T[:, 0]] - x
        b = V[T[:, 1]] - x
        c = V[T[:, 2]] - x
        la, lb, lc = (np.linalg.norm(v, axis=1) for v in (a, b, c))
        num = np.einsum("ij,ij->i", a, np.cross(b, c))
        den = la * lb * lc + np.einsum("ij,ij->i", a, b) * lc + np.einsum("ij,ij->i", b, c) * la \
            + np.einsum("ij,ij->i", c, a) * lb
        out[i] = np.sum(2.0 * np.arctan2(num, den)) / (4.0 * np.pi)
    return out


def surface_sources(space, coeffs, tri_idx, levels):
    """Quadrature points y [n, 3], weights w |T| [n], current v(y) [n, 3] and
    div v [n] of the RWG expansion sum_j coeffs_j phi_j on the triangles tri_idx."""
    bary, w = composite_rule(levels)
    x, f = space.values(tri_idx, bary)           # [nt, q, 3], [nt, q, 3(a), 3]
    beta = (space.B.T @ coeffs).reshape(-1, 3)[tri_idx]   # local fluxes [nt, 3]
    v = np.einsum("ta,tqac->tqc", beta, f)
    area = space.area[tri_idx]
    div = beta.sum(1) / area                     # div f_{tau,a} = 1 / |tau|
    wA = w[None, :] * area[:, None]
    q = len(w)
    return (x.reshape(-1, 3), wA.reshape(-1), v.reshape(-1, 3),
            np.repeat(div, q))


def potentials(k, src_a, src_b, points, chunk=64):
    """H_k(a)(x) + E_k(b)(x) at the points, for currents a, b given as
    surface_sources tuples on the same quadrature points."""
    y, w, va, _ = src_a
    _, _, vb, db = src_b
    k = complex(k)
    P = np.asarray(points, dtype=np.float64)
    out = np.zeros((len(P), 3), dtype=np.complex128)
    for s in range(0, len(P), chunk):
        X = P[s:s + chunk]
        d = X[:, None, :] - y[None, :, :]        # x - y
        r = np.sqrt(np.einsum("pqc,pqc->pq", d, d))
        G = np.exp(1j * k * r) / (4.0 * np.pi * r)
        g = (1j * k * r - 1.0) * G / (r * r)
        wG = w[None, :] * G
        wg = w[None, :] * g
        Eb = 1j * k * np.einsum("pq,qc->pc", wG, vb) \
            - (1.0 / (1j * k)) * np.einsum("pq,q,pqc->pc", wg, db, d)
        Ha = np.einsum("pq,pqc->pc", wg, np.cross(d, va[None, :, :]))
        out[s:s + chunk] = Ha + Eb
    return out


def incident_field(k, inc, points):
    """E^inc = p e^{ik d.x} for inc = (d, p)."""
    d = np.asarray(inc[:3], dtype=np.float64)
    p = np.asarray(inc[3:6], dtype=np.float64)
    P = np.asarray(points, dtype=np.float64)
    return np.exp(1j * complex(k) * (P @ d))[:, None] * p[None, :]


def electric_field(pb, x, inc, points, levels=2, region=None):
    """Total electric field at the points from the solved total traces x of the
    oracle problem pb (paper ordering), following the module formulas. region
    (optional): -1 exterior or m for scatterer m per point; by default from
    the winding numbers."""
    P = np.asarray(points, dtype=np.float64)
    c, d = pb.split(x)
    topo, rwg = pb.topo, pb.rwg
    nt = len(topo.tris)
    tri_dom = np.asarray(topo.domain)
    if region is None:
        region = -np.ones(len(P), dtype=int)
        for m in range(pb.M):
            sel = np.nonzero(tri_dom == m)[0]
            wn = winding_number(topo.verts, topo.tris[sel], P)
            region[wn > 0.5] = m
    E = np.zeros((len(P), 3), dtype=np.complex128)
    ext = np.nonzero(region < 0)[0]
    all_t = np.arange(nt)
    if len(ext):
        a = surface_sources(rwg, c, all_t, levels)
        b = surface_sources(rwg, (pb.mu_e / pb.k_e) * d, all_t, levels)
        E[ext] = incident_field(pb.k_e, inc, P[ext]) - potentials(pb.k_e, a, b, P[ext])
    for m in range(pb.M):
        sel = np.nonzero(region == m)[0]
        if not len(sel):
            continue
        tm = np.nonzero(tri_dom == m)[0]
        a = surface_sources(rwg, c, tm, levels)
        b = surface_sources(rwg, (pb.mu_r[m] / pb.k_m[m]) * d, tm, levels)
        E[sel] = potentials(pb.k_m[m], a, b, P[sel])
    return E
