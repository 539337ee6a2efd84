"""Pins of the oracle's H-matrix model of Section 3.3 (ACA to nu, block cutoff chi).

ACA meets its stopping criterion as a norm bound on admissible blocks, the block
cluster tree partitions the matrix, a small tolerance reproduces the dense
matrix, and on the three cubes the preconditioner keeps its effect as nu grows
while a block-level cutoff chi_P -> 0 makes GMRES much slower (Table 2's trend:
rows with nu_P from 0.001 to 0.5 stay near 7 iterations; chi_P = 0.1 gives 84).
"""
import math

import numpy as np
import pytest

from oracle import bem, hmatrix, pmchwt
from oracle.spaces import Topology, bc_space
from paper_2008_04772_gb300 import meshgen


@pytest.fixture(scope="module")
def bc_ops():
    m = meshgen.icosphere(2)
    bc = bc_space(Topology(m.verts, m.tris, m.domain))
    S, C = bem.assemble(bc, bc, 2.0, bem.Rules(1, 1))
    return bc, S, C


def test_block_tree_partitions_the_matrix(bc_ops):
    bc, S, _ = bc_ops
    t = hmatrix.cluster_tree(bc.aabb_lo, bc.aabb_hi)
    cover = np.zeros(S.shape, dtype=int)
    for rows, cols, adm, d in hmatrix.block_tree(t, t):
        cover[np.ix_(rows, cols)] += 1
        assert adm == (d > 0.0)
    assert (cover == 1).all()


def test_aca_meets_its_tolerance(bc_ops):
    """On the largest admissible block of S: |B - U V^T|_2 / |B|_F <= nu, rank
    growing as nu falls (measured 9.3e-2, 8.9e-3, 4.8e-4 at ranks 7, 11, 17)."""
    bc, S, _ = bc_ops
    t = hmatrix.cluster_tree(bc.aabb_lo, bc.aabb_hi)
    adm = [l for l in hmatrix.block_tree(t, t) if l[2]]
    rows, cols, _, _ = max(adm, key=lambda l: len(l[0]) * len(l[1]))
    B = S[np.ix_(rows, cols)]
    ranks = []
    for nu in (1e-1, 1e-2, 1e-3):
        U, V = hmatrix.aca(B, nu)
        assert np.linalg.norm(B - U @ V.T, 2) <= nu * np.linalg.norm(B)
        ranks.append(U.shape[1])
    assert ranks[0] < ranks[1] < ranks[2]


def test_small_tolerance_reproduces_dense(bc_ops):
    bc, S, C = bc_ops
    (Sa, Ca), _ = hmatrix.compress([S, C], bc.aabb_lo, bc.aabb_hi, 1e-3, math.inf)
    assert np.linalg.norm(Sa - S) < 1e-3 * np.linalg.norm(S)
    assert np.linalg.norm(Ca - C) < 1e-2 * np.linalg.norm(C)


def test_three_cubes_tolerance_and_block_cutoff():
    """Three cubes at k_e = 2.1 meshed at h = 0.1 (576 triangles; at the paper's
    h no cluster pair inside one cube is admissible), P = D with q_P = (1,1,1,1):
    nu_P = 0.001 and 0.1 measured 18 and 23 iterations; chi_P = 0.1 at nu_P = 0.1
    measured 70 (chi_P = 0: 759)."""
    k = 2.1
    eps = (1.311 + 2.289e-9j) ** 2
    inc = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    m = meshgen.three_cubes(0.1)
    its = {}
    for nu, chi in ((1e-3, math.inf), (0.1, math.inf), (0.1, 0.1)):
        pb = pmchwt.PMCHWT(m.verts, m.tris, m.domain, k, eps, precond="D", rules_P=(1, 1), aca_P=(nu, chi))
        pb.assemble()
        _, info = pb.solve(inc, tol=1e-5, restart=200, maxit=2000)
        its[(nu, chi)] = info["iterations"]
    assert its[(0.1, math.inf)] <= 1.5 * its[(1e-3, math.inf)], its
    assert its[(0.1, 0.1)] >= 2 * its[(0.1, math.inf)], its
