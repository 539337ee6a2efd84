"""H-matrix form with ACA on the GPU (Section 3.3) against the oracle's model.

The oracle (``oracle/hmatrix.py``) builds the cluster and block trees from the
support boxes and compresses admissible leaves of the dense blocks by partially
pivoted ACA to nu, keeping those within chi. The GPU builds the same trees and
runs the same ACA on the device: on the same dense entries the compressed
operators agree leaf by leaf (same pivots, float64), the stored entry counts
agree, the product equals the expanded matrix, and the preconditioned solve
with an ACA-compressed P takes the oracle's iteration count.
"""
import math

import numpy as np
import pytest

from gpu_common import mesh, oracle_spaces, rel
from oracle import bem, hmatrix, pmchwt
from paper_2008_04772_gb300 import cal, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2008_04772_gb300 import build
    build.build()
    return cal.Context(0)


@pytest.fixture(scope="module")
def sphere2_bc(ctx):
    m = mesh("sphere2")
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    sp = cal.Space(gm, cal.BC)
    return gm, sp


@pytest.mark.parametrize("nu,chi", [(1e-1, math.inf), (1e-3, math.inf), (1e-2, 0.3)])
def test_compress_matches_oracle_model(ctx, sphere2_bc, nu, chi):
    _, sp = sphere2_bc
    topo, rwg_o, bc_o = oracle_spaces("sphere2")
    dense = cal.assemble(ctx, 3, 2.0, sp, q_regular=1, q_singular=1, precision=cal.FP64)
    S, C = dense.export(cal.OP_S), dense.export(cal.OP_C)
    # the oracle's model on the GPU's own dense entries (so that both pick the same pivots)
    (So, Co), stored = hmatrix.compress([S, C], bc_o.aabb_lo, bc_o.aabb_hi, nu, chi)
    h = cal.compress(ctx, dense, sp, nu, chi)
    info = h.info()
    assert info.format == cal.HMAT
    Sh, Ch = h.export(cal.OP_S), h.export(cal.OP_C)
    # Leaves whose pivots are not near-ties take the same pivots and factors on
    # both sides, so nearly every entry equals the model. A leaf whose pivot
    # (largest modulus) or stopping test |u||v| <= nu |B_r|_F is a tie to
    # rounding may go either way (sums in another order); either result is an
    # ACA step, within nu of the block.
    for H, O, M in ((Sh, So, S), (Ch, Co, C)):
        same = np.abs(H - O) <= 1e-9 * np.abs(M).max()
        assert same.mean() >= 0.9, same.mean()
        assert rel(H, O) < nu, rel(H, O)
    assert abs(info.nnz - stored) <= 1e-3 * stored, (info.nnz, stored)
    if math.isinf(chi):  # nothing dropped: close to the dense operators
        assert rel(Sh, S) < 3 * nu and rel(Ch, C) < 30 * nu


@pytest.mark.parametrize("prec", [cal.FP64, cal.FP32])
def test_hmatrix_product(ctx, sphere2_bc, prec):
    import torch
    _, sp = sphere2_bc
    dense = cal.assemble(ctx, 3, 2.0 + 0.1j, sp, q_regular=1, q_singular=1, precision=prec)
    h = cal.compress(ctx, dense, sp, 1e-2)
    n = h.info().cols
    rng = np.random.default_rng(5)
    dt = np.complex128 if prec == cal.FP64 else np.complex64
    x = (rng.normal(size=(2, n)) + 1j * rng.normal(size=(2, n))).astype(dt)
    rt = np.float64 if prec == cal.FP64 else np.float32
    xt = torch.from_numpy(x.view(rt).copy()).cuda()
    for which in (cal.OP_S, cal.OP_C):
        yt = torch.zeros_like(xt)
        h.matvec(which, xt.data_ptr(), yt.data_ptr(), nrhs=2)
        torch.cuda.synchronize()
        y = yt.cpu().numpy().view(dt)
        H = h.export(which).astype(np.complex128)
        yr = (H @ x.astype(np.complex128).T).T
        assert rel(y, yr) < (1e-12 if prec == cal.FP64 else 2e-6), (which, rel(y, yr))


def test_float32_compression_within_tolerance(ctx, sphere2_bc):
    # float32 ACA may pivot differently from float64 near ties; it must still meet nu
    _, sp = sphere2_bc
    dense = cal.assemble(ctx, 3, 2.0, sp, q_regular=1, q_singular=1, precision=cal.FP32)
    S = dense.export(cal.OP_S).astype(np.complex128)
    h = cal.compress(ctx, dense, sp, 1e-3)
    assert rel(h.export(cal.OP_S).astype(np.complex128), S) < 3e-3


def test_solve_with_aca_preconditioner_takes_the_oracle_iterations(ctx):
    """Three cubes (h = 0.1), k_e = 2.1, P = D with q_P = (1,1,1,1) and ACA:
    nu_P = 0.1 with chi_P = inf and 0.1 (the oracle's pins: 23 and 70 iterations).
    float64, total-trace right-hand side as in the oracle's pins."""
    k = 2.1
    eps = (1.311 + 2.289e-9j) ** 2
    inc = np.array([[1.0, 0.0, 0.0, 0.0, 0.0, 1.0]])
    m = meshgen.three_cubes(0.1)
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    h = gm.info().h
    for nu, chi in ((0.1, math.inf), (0.1, 0.1)):
        pb = pmchwt.PMCHWT(m.verts, m.tris, m.domain, k, eps, precond="D", rules_P=(1, 1), aca_P=(nu, chi))
        pb.assemble()
        _, oinfo = pb.solve(inc[0], tol=1e-5, restart=200, maxit=2000)
        opts = cal.solve_opts(precond="D", precision=cal.FP64, tol=1e-5, restart=200, maxit=2000, q_regular_P=1,
                              q_singular_P=1, aca_nu_P=nu, near_cutoff_P=chi / h if math.isfinite(chi) else math.inf)
        info = cal.pmchwt_solve(ctx, gm, k, eps, inc, opts=opts).info()
        assert abs(info.iterations - oinfo["iterations"]) <= 1, (nu, chi, info.iterations, oinfo["iterations"])
        assert info.bytes_P > 0
