"""Shared helpers for the GPU parity tests (seeded inputs, oracle caches)."""
import functools

import numpy as np

from oracle import bem, pmchwt, spaces
from paper_2008_04772_gb300 import meshgen

EPS = 3.17 + 0.01j


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@functools.lru_cache(maxsize=None)
def mesh(name):
    if name.startswith("sphere"):
        return meshgen.icosphere(int(name[len("sphere"):]))
    if name == "bipyr14":
        # two apex vertices of valence 14: dual cells of 28 triangles
        return meshgen.bipyramid(14)
    if name == "cubes":
        # the three cubes of Section 4 (M = 3)
        return meshgen.three_cubes(0.2)
    if name == "prisms2":
        # two disjoint prisms, ~130 triangles each: ragged tile tails, valence 3..8
        return meshgen.prism_aggregate(2, 130, seed=1, diameter=1.0, gap=0.05)
    raise KeyError(name)


@functools.lru_cache(maxsize=None)
def oracle_spaces(name):
    m = mesh(name)
    topo = spaces.Topology(m.verts, m.tris, m.domain)
    return topo, spaces.rwg_space(topo), spaces.bc_space(topo)


@functools.lru_cache(maxsize=None)
def oracle_ops(name, kind, k, nreg=6, ng=4, scat=-1):
    topo, rwg, bc = oracle_spaces(name)
    sp = rwg if kind == "RWG" else bc
    idx = None
    if scat >= 0:
        idx = np.nonzero(topo.edge_domain == scat)[0]
    return bem.assemble(sp, sp, k, bem.Rules(nreg, ng), rows=idx, cols=idx)
