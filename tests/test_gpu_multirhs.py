"""Multi-right-hand-side path: tensor-core 3xTF32 product and lockstep GMRES."""
import numpy as np
import pytest

from gpu_common import EPS, mesh, oracle_ops, rel
from paper_2008_04772_gb300 import cal, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2008_04772_gb300 import build
    build.build()
    return cal.Context(0)


def _product(ctx, name, nrhs, which, seed=0, with_f32=False):
    import torch
    m = mesh(name)
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    sp = cal.Space(gm, cal.RWG)
    op = cal.assemble(ctx, 3, 2.0 + 0.1j, sp, precision=cal.FP32)
    X = op.export(which).astype(np.complex128)
    n = X.shape[1]
    rng = np.random.default_rng(seed)
    x = (rng.normal(size=(nrhs, n)) + 1j * rng.normal(size=(nrhs, n))).astype(np.complex64)
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    yt = torch.zeros((nrhs, 2 * X.shape[0]), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    op.matvec(which, xt.data_ptr(), yt.data_ptr(), nrhs=nrhs)
    torch.cuda.synchronize()
    y = yt.cpu().numpy().view(np.complex64)
    yr = (X @ x.astype(np.complex128).T).T
    if with_f32:
        return y, yr, (X.astype(np.complex64) @ x.T).T
    return y, yr


@pytest.mark.parametrize("nrhs", [4, 5, 8, 32, 64, 127])
@pytest.mark.parametrize("which", [cal.OP_S, cal.OP_C])
def test_tensor_core_product_matches_float64(ctx, nrhs, which):
    # 3xTF32 with round-to-nearest sums of the per-K-tile partial products keeps
    # float32 accuracy: within 3x the error of a float32 GEMM of the same data
    y, yr, y32 = _product(ctx, "sphere2", nrhs, which, with_f32=True)
    floor = rel(y32, yr)
    assert rel(y, yr) < max(3 * floor, 1e-6), (rel(y, yr), floor)
    # every column, not only the aggregate
    for j in range(nrhs):
        assert rel(y[j], yr[j]) < max(3 * rel(y32[j], yr[j]), 2e-6), j


def test_tensor_core_product_full_size(ctx):
    # 7680 x 7680 block, 32 vectors (the multi-RHS shape of the solve): each
    # entry is a 15360-term sum. The tensor core adds MMA products into its
    # float32 accumulator without rounding to nearest, so the kernel starts a
    # fresh accumulator every K tile and sums the tiles in registers; the
    # product must stay within 3x the error of a float32 GEMM of the same data.
    y, yr, y32 = _product(ctx, "sphere4", 32, cal.OP_S, seed=3, with_f32=True)
    floor = rel(y32, yr)
    assert floor < 2e-6
    assert rel(y, yr) < max(3 * floor, 1e-6), (rel(y, yr), floor)


def test_tensor_core_product_full_size_wide(ctx):
    # 128 vectors: 256 real columns, two column blocks of the kernel
    y, yr, y32 = _product(ctx, "sphere4", 128, cal.OP_C, seed=4, with_f32=True)
    floor = rel(y32, yr)
    assert rel(y, yr) < max(3 * floor, 1e-6), (rel(y, yr), floor)


def test_lockstep_solve_equals_solo_solves(ctx):
    d = meshgen.fibonacci_directions(8)
    inc = np.concatenate([d, meshgen.perpendicular_polarisation(d)], 1)
    m = mesh("sphere2")
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    opts = cal.solve_opts(precond="D", precision=cal.FP32, tol=1e-7)
    dirs = meshgen.fibonacci_directions(32)
    multi = cal.pmchwt_solve(ctx, gm, 2.0, EPS, inc, opts=opts)
    Fm = multi.far_field(dirs)
    info = multi.info()
    assert info.converged == 1
    for q in (0, 3, 7):
        solo = cal.pmchwt_solve(ctx, gm, 2.0, EPS, inc[q:q + 1], opts=opts).far_field(dirs)[0]
        assert rel(Fm[q], solo) < 2e-5
    # matvec accounting covers every column
    assert info.matvecs >= 8 * 16 * 5


def test_lockstep_solve_of_32_columns_on_the_5120_sphere(ctx):
    """32 columns of 15,360 unknowns: the Arnoldi dot products sum two elements
    per thread ahead of their float64 warp reduction (a single column, and the
    small meshes above, take one); the batch must equal solo solves of its
    first and last columns."""
    d = meshgen.fibonacci_directions(32)
    inc = np.concatenate([d, meshgen.perpendicular_polarisation(d)], 1)
    m = mesh("sphere4")
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    opts = cal.solve_opts(precond="D", precision=cal.FP32, tol=1e-7)
    dirs = meshgen.fibonacci_directions(32)
    multi = cal.pmchwt_solve(ctx, gm, 2.0, EPS, inc, opts=opts)
    Fm = multi.far_field(dirs)
    assert multi.info().converged == 1
    for q in (0, 31):
        solo = cal.pmchwt_solve(ctx, gm, 2.0, EPS, inc[q:q + 1], opts=opts).far_field(dirs)[0]
        assert rel(Fm[q], solo) < 2e-5, (q, rel(Fm[q], solo))
