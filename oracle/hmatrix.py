"""H-matrix blocks with ACA and the near-field cutoff of Section 3.3 (test infrastructure).

Section 3.3 describes the bi-parametric H-matrix assembly of the paper's
software: cluster trees of the test and trial dofs by repeated geometric
subdivision; a block of two clusters is admissible if the bounding boxes of
their supports are disjoint (eq. admissibility: dist > 0); otherwise it is
split until its parts are admissible or smaller than a minimum block size, in
which case it is inadmissible and assembled densely. Admissible blocks are
approximated by adaptive cross approximation (ACA, Bebendorf 2000) to a
tolerance nu, and only those with dist(X, Y) <= chi (eq. nf_condition) are
kept; the others are set to zero.

Readings (the paper leaves these to the software): clusters are split at the
median of the support-box centres along the longest side of the cluster's box;
the minimum block size is 16 dofs; ACA uses partial pivoting and stops when
|u_r| |v_r| <= nu |B_r|_F with the running Frobenius norm of the approximation.
Entries come from a dense matrix (this is a model of the approximation, not of
the assembly cost).
"""
from __future__ import annotations

import numpy as np

N_MIN = 16


def cluster_tree(lo, hi, idx=None, n_min=N_MIN):
    """Binary tree over the dofs: node = (idx, box_lo, box_hi, children)."""
    if idx is None:
        idx = np.arange(len(lo))
    blo, bhi = lo[idx].min(0), hi[idx].max(0)
    if len(idx) <= n_min:
        return (idx, blo, bhi, ())
    c = 0.5 * (lo[idx] + hi[idx])
    ax = int(np.argmax(bhi - blo))
    order = idx[np.argsort(c[:, ax], kind="stable")]
    h = len(order) // 2
    return (idx, blo, bhi, (cluster_tree(lo, hi, order[:h], n_min), cluster_tree(lo, hi, order[h:], n_min)))


def box_distance(a_lo, a_hi, b_lo, b_hi):
    gap = np.maximum(0.0, np.maximum(b_lo - a_hi, a_lo - b_hi))
    return float(np.sqrt((gap * gap).sum()))


def block_tree(t, s, n_min=N_MIN):
    """Leaves (rows, cols, admissible, dist) of the block cluster tree of t x s."""
    out = []

    def rec(a, b):
        d = box_distance(a[1], a[2], b[1], b[2])
        if d > 0.0:
            out.append((a[0], b[0], True, d))
        elif len(a[0]) <= n_min or len(b[0]) <= n_min or not a[3] or not b[3]:
            out.append((a[0], b[0], False, d))
        else:
            for ca in a[3]:
                for cb in b[3]:
                    rec(ca, cb)

    rec(t, s)
    return out


def aca(B, nu, max_rank=None):
    """Partially pivoted ACA of B: U [m, r], V [n, r] with B ~ U V^T."""
    m, n = B.shape
    max_rank = min(m, n) if max_rank is None else max_rank
    U, V = [], []
    used = np.zeros(m, dtype=bool)
    i = 0
    norm2 = 0.0
    while len(U) < max_rank:
        used[i] = True
        r = B[i, :].astype(np.complex128)
        for u, v in zip(U, V):
            r = r - u[i] * v
        j = int(np.argmax(np.abs(r)))
        if abs(r[j]) == 0.0:
            free = np.nonzero(~used)[0]
            if not len(free):
                break
            i = int(free[0])
            continue
        v = r / r[j]
        u = B[:, j].astype(np.complex128)
        for uu, vv in zip(U, V):
            u = u - vv[j] * uu
        # running |sum u_k v_k^T|_F^2
        cross = sum(2.0 * np.real(np.vdot(uu, u) * np.vdot(vv, v)) for uu, vv in zip(U, V))
        nu2 = np.vdot(u, u).real * np.vdot(v, v).real
        norm2 += nu2 + cross
        U.append(u)
        V.append(v)
        if np.sqrt(nu2) <= nu * np.sqrt(max(norm2, 0.0)):
            break
        cand = np.abs(u)
        cand[used] = -1.0
        i = int(np.argmax(cand))
        if cand[i] < 0:
            break
    if not U:
        return np.zeros((m, 0), complex), np.zeros((n, 0), complex)
    return np.array(U).T, np.array(V).T


def compress(matrices, lo, hi, nu, chi, n_min=N_MIN):
    """H-matrix version of one or more dense [n, n] blocks on the same dofs:
    inadmissible leaves exact, admissible leaves with dist <= chi by ACA to nu,
    the rest zero. Returns the approximations and the stored entry count."""
    t = cluster_tree(lo, hi, n_min=n_min)
    leaves = block_tree(t, t, n_min)
    outs = [np.zeros_like(M) for M in matrices]
    stored = 0
    for rows, cols, adm, d in leaves:
        ix = np.ix_(rows, cols)
        if not adm:
            for M, O in zip(matrices, outs):
                O[ix] = M[ix]
            stored += len(rows) * len(cols) * len(matrices)
        elif d <= chi:
            for M, O in zip(matrices, outs):
                U, V = aca(M[ix], nu)
                O[ix] = U @ V.T
                stored += U.shape[1] * (len(rows) + len(cols))
    return outs, stored
