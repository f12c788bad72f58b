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


class FakeTensor:
    """Stands in for a torch CUDA tensor: dtype width, entry count, layout."""

    def __init__(self, numel, itemsize=8, floating=True, cuda=True, contiguous=True):
        self._n, self._es, self._fp, self.is_cuda, self._c = numel, itemsize, floating, cuda, contiguous

    def numel(self):
        return self._n

    def element_size(self):
        return self._es

    def is_floating_point(self):
        return self._fp

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        return 4096


def set_up_ctx():
    c = ctx()
    c._level_n = [4 * 27, 27]     # two levels of a 2x2 mesh, nb = 27
    c._nb = 27
    return c


def test_device_vectors_checked_before_the_call():
    """Device vectors cross the ABI as bare pointers: a float32 vector where
    float64 is read, a vector shorter or longer than the level, or a missing
    norm scalar is refused before the library runs a kernel on it."""
    c = set_up_ctx()
    n = 4 * 27
    good = FakeTensor(n)
    c.residual_norm_static(good, good, good, FakeTensor(1))
    assert c.lib.calls[-1] == "stk_residual_norm_static"
    bad_cases = [
        (FakeTensor(n, 4), good, good, FakeTensor(1)),       # float32 x
        (good, FakeTensor(n - 1), good, FakeTensor(1)),      # short b
        (good, good, FakeTensor(n + 5), FakeTensor(1)),      # long r
        (good, good, good, FakeTensor(1, 4)),                # float32 norm
        (good, good, good, FakeTensor(0)),                   # empty norm
        (good, FakeTensor(n, 8, floating=False), good, FakeTensor(1)),   # int64 b
    ]
    for args in bad_cases:
        calls = len(c.lib.calls)
        with pytest.raises(ValueError):
            c.residual_norm_static(*args)
        assert len(c.lib.calls) == calls
    with pytest.raises(ValueError):
        c.residual(good, FakeTensor(n, 4), good)
    with pytest.raises(ValueError):
        c.vcycle(FakeTensor(n - 27), good)
    with pytest.raises(ValueError):
        c.restrict(0, good, FakeTensor(n))                   # coarse vector has 27 entries
    c.restrict(0, good, FakeTensor(27))
    with pytest.raises(ValueError):
        c.gs_colour_ex(0, 0, native.FP32, good, good)        # FP32 cycle vectors are float32
    c.gs_colour_ex(0, 0, native.FP32, FakeTensor(n, 4), FakeTensor(n, 4))
    with pytest.raises(ValueError):
        c.solve_multi(FakeTensor(3 * n), FakeTensor(2 * n), 3)
    with pytest.raises(native.StkError):
        c.gs_colour(0, 0, FakeTensor(n, contiguous=False), good)


def test_vectors_need_setup():
    c = ctx()
    with pytest.raises(native.StkError):
        c.residual(FakeTensor(4), FakeTensor(4), FakeTensor(4))
