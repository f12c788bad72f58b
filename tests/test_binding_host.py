"""Host-side argument checks of the ctypes binding (no device): host arrays
cross the C ABI as bare pointers, so the binding refuses arrays whose size
does not match the point sets the library reports, before any call reads
them.  A fake library stands in for libstokes_mg.so."""
import ctypes

import numpy as np
import pytest

from paper_1911_05888_gb300 import native

COUNTS = {native.PTS_VOLUME: 64, native.PTS_INTERIOR_FACE: 48, native.PTS_BOUNDARY_FACE: 16}


class FakeLib:
    def __init__(self):
        self.calls = []

    def stk_num_points(self, h, kind, out):
        out._obj.value = COUNTS[kind]
        return native.STK_OK

    def __getattr__(self, name):
        def fn(*args):
            self.calls.append(name)
            return native.STK_OK
        return fn


def ctx():
    c = object.__new__(native.Context)
    c.lib = FakeLib()
    c.h = ctypes.c_void_p(1)
    c.set_mesh(2, (2, 2), (0, 0), (1, 1), (1, 2, 1, 1))
    return c


def test_set_mesh_checks_lengths_and_records_size():
    c = ctx()
    assert c.d == 2 and c.ne == 4
    with pytest.raises(ValueError):
        c.set_mesh(2, (2, 2, 2), (0, 0), (1, 1), (1, 1, 1, 1))


def test_viscosity_and_density_sizes():
    c = ctx()
    c.set_viscosity(np.ones(64), np.ones(48), np.ones(16))
    assert c.lib.calls[-1] == "stk_set_viscosity"
    for bad in [(np.ones(63), np.ones(48), np.ones(16)), (np.ones(64), np.ones(47), np.ones(16)),
                (np.ones(64), np.ones(48), np.ones(0))]:
        n = len(c.lib.calls)
        with pytest.raises(ValueError):
            c.set_viscosity(*bad)
        assert len(c.lib.calls) == n                     # the library was not called
    c.set_density(np.ones(64), np.ones(48), 0.1)
    with pytest.raises(ValueError):
        c.set_density(np.ones(64), np.ones(49), 0.1)


def test_rhs_data_shapes():
    c = ctx()
    c.assemble_rhs(np.zeros((64, 3)), np.zeros((16, 2)), 4, 27)
    c.assemble_rhs2(np.zeros((64, 3)), np.zeros((16, 2)), np.zeros((48, 4)), 4, 27)
    with pytest.raises(ValueError):
        c.assemble_rhs(np.zeros((64, 2)), np.zeros((16, 2)), 4, 27)      # f_vol needs d+1 columns
    with pytest.raises(ValueError):
        c.assemble_rhs(np.zeros((64, 3)), np.zeros((16, 2)), 5, 27)      # wrong element count
    with pytest.raises(ValueError):
        c.assemble_rhs2(np.zeros((64, 3)), np.zeros((16, 2)), np.zeros((48, 2)), 4, 27)


def test_phase_array():
    c = ctx()
    c.set_phases([1, 2, 2, 1], [1.0, 1e3])
    with pytest.raises(ValueError):
        c.set_phases([1, 2, 2], [1.0, 1e3])
    with pytest.raises(ValueError):
        c.set_phases([1, 3, 2, 1], [1.0, 1e3])
    with pytest.raises(ValueError):
        c.set_phases([0, 1, 1, 1], [1.0, 1e3])
