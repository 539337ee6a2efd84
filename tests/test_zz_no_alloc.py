"""cal_matvec_static: the tensor-core product with fixed scratch, no allocation.

Some callers cannot allocate device memory: a process whose HBM is owned by
another allocator (PyTorch's caching allocator, or a serving loop that has
reserved its budget up front), where a library-internal cudaMalloc would fail
or escape that allocator's accounting. Its result must match cal_matvec's (the
same 3xTF32 product with the split done in the kernel) and the float64 product
within the float32 bar of the multi-vector tests, on two calls in a row (the
second call reuses the shared scratch the first left), and the call must not
change the device's free memory, PyTorch's allocator or the stream-ordered
pool's high-water mark. Collected last so that it also runs after every other
GPU test.
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


class _PoolWatch:
    """Used-memory high-water mark of the device's default stream-ordered pool
    (driver API, the pool every cudaMallocAsync of the library draws from),
    plus PyTorch's allocator and the device's free memory."""

    USED_CURRENT, USED_HIGH = 7, 8  # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH

    def __init__(self, device=0):
        import torch
        self.torch = torch
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), device) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def _attr(self, a):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, a, ctypes.byref(v)) == 0
        return v.value

    def start(self):
        self.torch.cuda.synchronize()
        zero = ctypes.c_uint64(0)  # resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_HIGH, ctypes.byref(zero)) == 0
        self.used0 = self._attr(self.USED_CURRENT)
        self.torch0 = self.torch.cuda.memory_allocated()
        self.free0 = self.torch.cuda.mem_get_info()[0]

    def check(self):
        self.torch.cuda.synchronize()
        # the mark was reset to zero; any allocation during the call lifts it above the use before it
        assert self._attr(self.USED_HIGH) <= self.used0, "the call drew memory from the stream-ordered pool"
        assert self.torch.cuda.memory_allocated() == self.torch0
        assert self.torch.cuda.mem_get_info()[0] == self.free0, "device free memory changed across the call"


@pytest.mark.parametrize("nrhs", [8, 5, 127])
@pytest.mark.parametrize("which", [cal.OP_S, cal.OP_C])
def test_static_scratch_matches_matvec(setup, nrhs, which):
    import torch
    _, _, _, op = setup
    rows = op.info().rows
    watch = _PoolWatch()
    # set-up call: the first call on a device looks up the scratch array's
    # address, and the driver loads the library's kernels on first use
    x0, xt0 = _vectors(op, nrhs, 7)
    y0 = torch.zeros((nrhs, 2 * rows), dtype=torch.float32, device="cuda")
    op.matvec_static(which, xt0.data_ptr(), y0.data_ptr(), nrhs=nrhs)
    for call, seed in enumerate((11, 12)):  # two calls in a row on the shared scratch
        x, xt = _vectors(op, nrhs, seed + nrhs)
        y_ref = torch.zeros((nrhs, 2 * rows), dtype=torch.float32, device="cuda")
        y_new = torch.full((nrhs, 2 * rows), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        op.matvec(which, xt.data_ptr(), y_ref.data_ptr(), nrhs=nrhs)
        torch.cuda.synchronize()
        dev_before = torch.cuda.current_device()
        watch.start()
        op.matvec_static(which, xt.data_ptr(), y_new.data_ptr(), nrhs=nrhs)
        watch.check()  # nothing allocated by the call, on any allocator
        assert torch.cuda.current_device() == dev_before
        a = y_new.cpu().numpy().view(np.complex64)
        b = y_ref.cpu().numpy().view(np.complex64)
        assert np.all(np.isfinite(a)), call
        assert rel(a, b) < 1e-6, (call, rel(a, b))
        for j in range(nrhs):
            assert rel(a[j], b[j]) < 2e-6, (call, j)


def test_static_scratch_matches_float64_product(setup):
    # against the exact (float64) product of the stored float32 operator: within
    # 3x the error of a float32 GEMM of the same data
    import torch
    _, _, _, op = setup
    rows = op.info().rows
    X = op.export(cal.OP_S).astype(np.complex128)
    x, xt = _vectors(op, 6, 21)
    y = torch.zeros((6, 2 * rows), dtype=torch.float32, device="cuda")
    op.matvec_static(cal.OP_S, xt.data_ptr(), y.data_ptr(), nrhs=6)
    torch.cuda.synchronize()
    got = y.cpu().numpy().view(np.complex64)
    ref = (X @ x.astype(np.complex128).T).T
    floor = rel((X.astype(np.complex64) @ x.T).T, ref)
    assert rel(got, ref) < max(3 * floor, 1e-6), (rel(got, ref), floor)


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
