"""cal_matvec_static: the tensor-core product with fixed scratch, no allocation.

Its result must match cal_matvec's (same 3xTF32 product, split-K sums in a
different order) within the float32 bar of the multi-vector tests, on two
calls in a row (the second call reuses the shared scratch the first left).
Collected last so that it also runs after every other GPU test.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import mesh, rel
from paper_2008_04772_gb300 import cal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2008_04772_gb300 import build
    build.build()
    ctx = cal.Context(0)
    m = mesh("sphere4")
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    sp = cal.Space(gm, cal.RWG)
    op = cal.assemble(ctx, 3, 2.0 + 0.1j, sp, precision=cal.FP32)
    return ctx, gm, sp, op


def _vectors(op, nrhs, seed):
    import torch
    n = op.info().cols
    rng = np.random.default_rng(seed)
    x = (rng.normal(size=(nrhs, n)) + 1j * rng.normal(size=(nrhs, n))).astype(np.complex64)
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    return x, xt


@pytest.mark.parametrize("nrhs", [8, 5])
@pytest.mark.parametrize("which", [cal.OP_S, cal.OP_C])
def test_static_scratch_matches_matvec(setup, nrhs, which):
    import torch
    _, _, _, op = setup
    rows = op.info().rows
    for call, seed in enumerate((11, 12)):  # two calls in a row on the shared scratch
        x, xt = _vectors(op, nrhs, seed + nrhs)
        y_ref = torch.zeros((nrhs, 2 * rows), dtype=torch.float32, device="cuda")
        y_new = torch.full((nrhs, 2 * rows), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        op.matvec(which, xt.data_ptr(), y_ref.data_ptr(), nrhs=nrhs)
        torch.cuda.synchronize()
        op.matvec_static(which, xt.data_ptr(), y_new.data_ptr(), nrhs=nrhs)
        torch.cuda.synchronize()
        a = y_new.cpu().numpy().view(np.complex64)
        b = y_ref.cpu().numpy().view(np.complex64)
        assert np.all(np.isfinite(a)), call
        assert rel(a, b) < 1e-5, (call, rel(a, b))
        for j in range(nrhs):
            assert rel(a[j], b[j]) < 2e-5, (call, j)


def test_static_scratch_rejects_oversize(setup):
    import torch
    ctx, _, _, op = setup
    cols = op.info().cols
    xt = torch.zeros((2, 2 * cols), dtype=torch.float32, device="cuda")
    with pytest.raises(cal.CalError) as e:
        op.matvec_static(cal.OP_S, xt.data_ptr(), xt.data_ptr(), nrhs=129)
    assert "outside" in str(e.value)
    # 30720 x 30720 block with 64 vectors: 4 * 128 * 3 * 30720 bytes > 32 MiB
    m = mesh("sphere5")
    big = cal.assemble(ctx, cal.OP_S, 2.0, cal.Space(cal.Mesh(ctx, m.verts, m.tris, m.domain), cal.RWG),
                       q_regular=1, q_singular=1, precision=cal.FP32)
    xb = torch.zeros((64, 2 * big.info().cols), dtype=torch.float32, device="cuda")
    with pytest.raises(cal.CalError) as e:
        big.matvec_static(cal.OP_S, xb.data_ptr(), xb.data_ptr(), nrhs=64)
    assert "fixed maximum" in str(e.value)
    del big
    # a float64 operator is not a tensor-core operand
    s = mesh("sphere1")
    op64 = cal.assemble(ctx, cal.OP_S, 2.0, cal.Space(cal.Mesh(ctx, s.verts, s.tris, s.domain), cal.RWG),
                        q_regular=1, q_singular=1, precision=cal.FP64)
    with pytest.raises(cal.CalError) as e:
        op64.matvec_static(cal.OP_S, xt.data_ptr(), xt.data_ptr(), nrhs=2)
    assert "float32 dense" in str(e.value)
