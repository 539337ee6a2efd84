"""The C ABI library builds, loads and exports every declared symbol (CPU only)."""
import ctypes
import math
import os

import numpy as np
import pytest

from paper_2008_04772_gb300 import build as libbuild
from paper_2008_04772_gb300 import cal


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return cal.lib()


def test_every_declared_symbol_is_exported(L):
    names = cal.declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n


def test_default_options_and_null_handling(L):
    o = cal.solve_opts()
    assert o.precond == cal.PRECOND["D"] and o.restart == 200 and o.q_regular_A == 6
    assert math.isinf(o.near_cutoff_P)
    # host-side argument checks, no device work
    out = ctypes.c_void_p()
    v = np.zeros((4, 3))
    t = np.zeros((4, 3), dtype=np.int32)
    rc = L.cal_mesh_create(None, v.ctypes.data_as(ctypes.c_void_p), 4,
                           t.ctypes.data_as(ctypes.c_void_p), 4, None, ctypes.byref(out))
    assert rc == cal.EINVAL
    assert b"NULL" in L.cal_last_error()
    assert L.cal_init(None, 0) == cal.EINVAL
