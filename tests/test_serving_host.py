"""Host-side parts of the serving loop (no GPU): footprint estimates, request checks."""
import ctypes
import math

import numpy as np
import pytest

from paper_2008_04772_gb300 import build as libbuild
from paper_2008_04772_gb300 import cal, meshgen


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return cal.lib()


def _fp(m, nrhs=1, ndir=8, **opts):
    d = meshgen.fibonacci_directions(nrhs)
    inc = np.concatenate([d, meshgen.perpendicular_polarisation(d)], 1)
    r, keep = cal.make_request(m.verts, m.tris, m.domain, 2.0, 3.17 + 0.01j, inc,
                               meshgen.fibonacci_directions(ndir), opts=cal.solve_opts(**opts))
    return cal.request_footprint(r)


def test_footprint_counts_the_stored_blocks(L):
    m = meshgen.icosphere(2)  # 320 triangles, 480 edges, one scatterer
    N = 480
    res_none, _ = _fp(m, precond="none")
    # S and C on the union and on the one scatterer, complex64, the combined
    # float32 blocks (C, S1, S2) of the one-vector product, plus space records
    assert 7 * N * N * 8 <= res_none <= 7 * N * N * 8 + 320 * 256
    res64, _ = _fp(m, precond="none", precision=cal.FP64)
    assert 4 * N * N * 16 <= res64 <= 4 * N * N * 16 + 320 * 256
    # full Calderon adds S and C on both sides of the one scatterer, dense, and
    # their combined blocks
    res_d, _ = _fp(m, precond="D")
    assert res_d - res_none >= 7 * N * N * 8
    # reduced S^i stores one block: less than D
    res_si, _ = _fp(m, precond="Si")
    assert res_none + N * N * 8 <= res_si < res_d


def test_near_field_footprint_grows_with_cutoff(L):
    m = meshgen.prism_aggregate(1, 3000, seed=3, diameter=1.0, gap=0.05)
    dense, _ = _fp(m, precond="Di")
    sizes = [_fp(m, precond="Di", near_cutoff_P=c)[0] for c in (1.0, 2.0, 4.0)]
    assert sizes[0] <= sizes[1] <= sizes[2]
    assert sizes[0] < dense
    # a cutoff that reaches every pair costs the dense values plus CSR indices
    assert sizes[2] <= 1.5 * dense


def test_solve_footprint_scales_with_columns_and_restart(L):
    m = meshgen.icosphere(2)
    _, s1 = _fp(m, nrhs=1)
    _, s8 = _fp(m, nrhs=8)
    _, s8r = _fp(m, nrhs=8, restart=50)
    assert s1 < s8
    assert s8r < s8
    # the Krylov basis alone: 8 columns x 201 vectors x 960 unknowns x 16 B
    assert s8 - s8r >= 8 * 150 * 960 * 16


def test_footprint_rejects_bad_meshes(L):
    v = np.zeros((3, 3))
    t = np.array([[0, 1, 2]], dtype=np.int32)
    r, keep = cal.make_request(v, t, None, 2.0, 3.0, [[0, 0, 1, 1, 0, 0]], [[1, 0, 0]])
    with pytest.raises(cal.CalError) as e:
        cal.request_footprint(r)
    assert e.value.code in (cal.EMESH, cal.EINVAL)


def test_queue_without_device_fails_loudly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    rc = L.cal_queue_create(0, 1 << 30, 2, ctypes.byref(h))
    assert rc == cal.ECUDA
    assert L.cal_queue_create(0, 0, 0, ctypes.byref(h)) == cal.EINVAL
