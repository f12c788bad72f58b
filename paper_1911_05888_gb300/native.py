"""ctypes binding of the C ABI in include/stokes_mg.h (argument marshalling only).

Every function here forwards to the entry point of the same name in the
in-tree shared library libstokes_mg.so and raises StkError on a negative
status.  Device vectors are torch CUDA tensors (float64, contiguous); the
library computes everything in its own CUDA kernels.  There is no fallback:
if the library is missing or no GPU is present, loading fails loudly.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstokes_mg.so")

STK_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "SINGULAR_BLOCK", -4: "TIMEOUT", -5: "DIVERGED",
          -6: "NOT_SETUP", -7: "CUDA"}
BC_PERIODIC, BC_DIRICHLET, BC_STRESS = 0, 1, 2
FP64, FP32, BF16, FP16 = 0, 1, 2, 3
RICHARDSON, FGMRES, FGMRES_IR = 0, 1, 2
PTS_VOLUME, PTS_INTERIOR_FACE, PTS_BOUNDARY_FACE, PTS_INTERFACE = 0, 1, 2, 3
INFO_BOTTOM_SOLVER, INFO_BOTTOM_UNKNOWNS, INFO_COLOURS, INFO_DEVICE_BYTES, INFO_CLUSTERS = 0, 1, 2, 3, 4
INFO_COUPLING_BLOCKS = 5
BOTTOM_JACOBI, BOTTOM_HOST_QR, BOTTOM_CUSOLVER = 0, 1, 2
COLOURS_AUTO, COLOURS_PARITY, COLOURS_CHECKERBOARD = 0, 1, 2

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)
_c_i64_p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p

# name -> argtypes (restype int unless listed in _RESTYPE)
SIGNATURES = {
    "stk_create": [ctypes.POINTER(_vp), ctypes.c_int],
    "stk_destroy": [_vp],
    "stk_last_error": [_vp],
    "stk_set_mesh": [_vp, ctypes.c_int, _c_int_p, _c_dbl_p, _c_dbl_p, _c_int_p],
    "stk_set_discretisation": [_vp, ctypes.c_int, ctypes.c_int],
    "stk_set_penalty": [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double],
    "stk_num_points": [_vp, ctypes.c_int, _c_i64_p],
    "stk_get_points": [_vp, ctypes.c_int, _c_dbl_p, _c_dbl_p],
    "stk_set_viscosity": [_vp, _c_dbl_p, _c_dbl_p, _c_dbl_p],
    "stk_set_density": [_vp, _c_dbl_p, _c_dbl_p, ctypes.c_double],
    "stk_set_cycle": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "stk_set_cycle_shape": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "stk_host_pseudo_inverse": [ctypes.c_int, _c_dbl_p, ctypes.c_double, _c_dbl_p, _c_int_p],
    "stk_gmres_rho": [_vp, _vp, ctypes.c_double, ctypes.c_int, _c_dbl_p, _c_int_p, _c_dbl_p, _c_dbl_p, _vp],
    "stk_setup": [_vp, _vp],
    "stk_get_sizes": [_vp, _c_int_p, _c_i64_p, _c_int_p, _c_int_p],
    "stk_get_block": [_vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _c_dbl_p],
    "stk_assemble_rhs": [_vp, _c_dbl_p, _c_dbl_p, _c_dbl_p],
    "stk_residual": [_vp, _vp, _vp, _vp, _c_dbl_p, _vp],
    "stk_gs_colour": [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp],
    "stk_gs_colour_ex": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp],
    "stk_residual_ex": [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp],
    "stk_vcycle": [_vp, _vp, _vp, _vp],
    "stk_restrict": [_vp, ctypes.c_int, _vp, _vp, _vp],
    "stk_prolong": [_vp, ctypes.c_int, _vp, _vp, _vp],
    "stk_bottom_solve": [_vp, _vp, _vp, _vp],
    "stk_solve": [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _c_int_p, _c_dbl_p, _vp],
    "stk_residual_norm_static": [_vp, _vp, _vp, _vp, _vp, _vp],
    "stk_set_solver": [_vp, ctypes.c_int, ctypes.c_int],
    "stk_learn_setup": [_vp, ctypes.c_int, ctypes.c_uint64],
    "stk_learn_generate": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64],
    "stk_learn_train": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, _c_dbl_p],
    "stk_learn_enable": [_vp, ctypes.c_int],
    "stk_learn_stats": [_vp, _c_i64_p, _c_i64_p],
    "stk_learn_weights": [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int64, ctypes.c_int],
    "stk_learn_sizes": [_vp, _c_int_p, _c_int_p, _c_int_p, _c_i64_p, _c_i64_p],
    "stk_learn_infer": [_vp, _vp, _vp, _vp],
    "stk_learn_state": [_vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_float)],
    "stk_learn_grad": [_vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_float), _c_dbl_p],
    "stk_solve_multi": [_vp, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, _c_int_p,
                        _c_dbl_p, _vp],
    "stk_set_tuning": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "stk_set_wide_launch": [_vp, ctypes.c_int],
    "stk_set_mrhs_tensor": [_vp, ctypes.c_int],
    "stk_set_df_matvec": [_vp, ctypes.c_int],
    "stk_set_launch_overlap": [_vp, ctypes.c_int],
    "stk_autotune": [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), _vp],
    "stk_solve_batch": [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int,
                        ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                        ctypes.POINTER(ctypes.c_int), _vp],
    "stk_set_phases": [_vp, ctypes.c_int, _c_int_p, _c_dbl_p, ctypes.c_int],
    "stk_get_interface": [_vp, _c_int_p, _c_int_p, _c_dbl_p],
    "stk_assemble_rhs2": [_vp, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p],
    "stk_get_colours": [_vp, ctypes.c_int, _c_int_p],
    "stk_get_scaling": [_vp, _c_dbl_p],
    "stk_launch_count": [_vp, _c_i64_p],
    "stk_get_info": [_vp, ctypes.c_int, _c_i64_p],
    "stk_set_colouring": [_vp, ctypes.c_int],
    "stk_fp64_fma_rate": [_vp, _c_dbl_p, _vp],
    "stk_learn_objective": [_vp, ctypes.c_int],
    "stk_learn_history": [_vp, _c_int_p, _c_dbl_p, ctypes.c_int, _c_int_p, _c_dbl_p],
    "stk_learn_error_state": [_vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_float)],
    "stk_set_persistent": [_vp, ctypes.c_int, ctypes.c_int],
    "stk_set_clusters": [_vp, ctypes.c_int],
    "stk_set_bottom": [_vp, ctypes.c_int64],
    "stk_cut_cells": [ctypes.c_int, _c_dbl_p, _c_dbl_p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                      ctypes.c_int, ctypes.c_double, _c_i64_p, _c_int_p, _c_int_p, _c_dbl_p, _c_int_p, _c_int_p,
                      _c_dbl_p],
    "stk_solve_batch_persistent": [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                   ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int), _c_dbl_p, _vp],
    "stk_barrier_selftest": [_vp, ctypes.c_int, ctypes.c_int64, _c_i64_p],
    "stk_set_levelset_circle": [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double],
    "stk_set_phase_density": [_vp, _c_dbl_p, ctypes.c_double],
    "stk_get_point_phases": [_vp, ctypes.c_int, _c_int_p],
    "stk_set_element_warps": [_vp, ctypes.c_int],
    "stk_learn_field": [_vp, ctypes.c_uint64, _vp, _vp],
}
_RESTYPE = {"stk_last_error": ctypes.c_char_p}


class StkError(RuntimeError):
    pass


_lib = None


def load(path=LIB_PATH):
    """Load libstokes_mg.so (no fallback: raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise StkError("libstokes_mg.so not built: run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, args in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = _RESTYPE.get(name, ctypes.c_int)
        _lib = lib
    return _lib


def exported_symbols(path=LIB_PATH):
    lib = ctypes.CDLL(path)
    return {name for name in SIGNATURES if hasattr(lib, name)}


def _dbl(a):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.ctypes.data_as(_c_dbl_p), a


def _ptr(t):
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise StkError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


_DTYPE_NAMES = {8: "float64", 4: "float32"}


def _vec(name, t, count, itemsize=8, at_least=False):
    """Device pointer of a vector argument after checking what the kernels
    will assume about it: a contiguous CUDA tensor of the stated element size
    (8 = float64, 4 = float32) floating dtype and exactly `count` entries (at
    least `count` with at_least).  Device vectors cross the ABI as bare
    pointers, so a short or mistyped tensor would be read or written past its
    end; it is refused here, before the call."""
    if t is None:
        raise ValueError("%s: a device tensor is required" % name)
    if not t.is_floating_point() or t.element_size() != itemsize:
        raise ValueError("%s: expected %s, got %s" % (name, _DTYPE_NAMES.get(itemsize, itemsize),
                                                         getattr(t, "dtype", "%d-byte entries" % t.element_size())))
    n = t.numel()
    if (n < count) if at_least else (n != count):
        raise ValueError("%s: %d entries, expected %s%d" % (name, n, ">= " if at_least else "", count))
    return _ptr(t)


def _stream(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Context:
    """Owner of one stk_ctx; methods mirror the C entry points."""

    def __init__(self, device=0):
        self.lib = load()
        h = _vp()
        rc = self.lib.stk_create(ctypes.byref(h), device)
        if rc != STK_OK:
            raise StkError("stk_create failed (%s)" % ERRORS.get(rc, rc))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.stk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, name):
        if rc != STK_OK:
            msg = self.lib.stk_last_error(self.h)
            raise StkError("%s: %s (%s)" % (name, msg.decode() if msg else "", ERRORS.get(rc, rc)))

    @staticmethod
    def _expect(name, a, rows, cols=1):
        """Host arrays cross the ABI as bare pointers: refuse one whose size
        is not rows x cols before the library reads it."""
        size = np.asarray(a).size
        if size != rows * cols:
            raise ValueError("%s: %d values, expected %d x %d" % (name, size, rows, cols))

    def set_mesh(self, d, n, lo, hi, bc):
        if not (len(n) == len(lo) == len(hi) == d and len(bc) == 2 * d):
            raise ValueError("set_mesh: n, lo, hi need d entries and bc 2d")
        n_ = (ctypes.c_int * d)(*n)
        lo_ = (ctypes.c_double * d)(*lo)
        hi_ = (ctypes.c_double * d)(*hi)
        bc_ = (ctypes.c_int * (2 * d))(*bc)
        self._check(self.lib.stk_set_mesh(self.h, d, n_, lo_, hi_, bc_), "stk_set_mesh")
        self.d = d
        self.ne = int(np.prod(n))

    def set_discretisation(self, p, gamma):
        self._check(self.lib.stk_set_discretisation(self.h, p, gamma), "stk_set_discretisation")

    def set_penalty(self, tau, tau0, c_bdry=10.0, c_intra=0.0):
        self._check(self.lib.stk_set_penalty(self.h, tau, tau0, c_bdry, c_intra), "stk_set_penalty")

    def num_points(self, kind):
        n = ctypes.c_int64()
        self._check(self.lib.stk_num_points(self.h, kind, ctypes.byref(n)), "stk_num_points")
        return n.value

    def get_points(self, kind, d):
        n = self.num_points(kind)
        xyz = np.zeros((n, d))
        nrm = np.zeros((n, d))
        self._check(self.lib.stk_get_points(self.h, kind, xyz.ctypes.data_as(_c_dbl_p),
                                            nrm.ctypes.data_as(_c_dbl_p)), "stk_get_points")
        return xyz, nrm

    def set_viscosity(self, mu_vol, mu_if, mu_bf):
        self._expect("mu_vol", mu_vol, self.num_points(PTS_VOLUME))
        self._expect("mu_iface", mu_if, self.num_points(PTS_INTERIOR_FACE))
        self._expect("mu_bface", mu_bf, self.num_points(PTS_BOUNDARY_FACE))
        a, b, c = _dbl(mu_vol), _dbl(mu_if), _dbl(mu_bf)
        self._check(self.lib.stk_set_viscosity(self.h, a[0], b[0], c[0]), "stk_set_viscosity")

    def set_density(self, rho_vol, rho_if, delta):
        if rho_vol is not None:
            self._expect("rho_vol", rho_vol, self.num_points(PTS_VOLUME))
        if rho_if is not None:
            self._expect("rho_iface", rho_if, self.num_points(PTS_INTERIOR_FACE))
        a = _dbl(rho_vol) if rho_vol is not None else (None, None)
        b = _dbl(rho_if) if rho_if is not None else (None, None)
        self._check(self.lib.stk_set_density(self.h, a[0], b[0], float(delta)), "stk_set_density")

    def set_cycle(self, nu1, nu2, precision=FP64):
        self._check(self.lib.stk_set_cycle(self.h, nu1, nu2, precision), "stk_set_cycle")

    def set_cycle_shape(self, gamma=1, growth=1, max_sweeps=64):
        """gamma coarse visits per level (1 V-cycle, 2 W-cycle); smoothing
        counts nu * growth^level, at most max(nu, max_sweeps)."""
        self._check(self.lib.stk_set_cycle_shape(self.h, gamma, growth, max_sweeps), "stk_set_cycle_shape")

    def set_bottom(self, max_unknowns):
        """Stop the hierarchy at the first coarse level with at most
        max_unknowns unknowns (0: full depth); takes effect at the next setup."""
        self._check(self.lib.stk_set_bottom(self.h, int(max_unknowns)), "stk_set_bottom")

    def set_clusters(self, on):
        """Smooth level 0 with 2 x 2 element clusters (2D, p = 1); takes
        effect at the next setup."""
        self._check(self.lib.stk_set_clusters(self.h, 1 if on else 0), "stk_set_clusters")

    def set_persistent(self, max_elements, ctas_per_sm=1):
        """Run the levels of at most max_elements elements (below level 0) as
        one cooperative launch per cycle (0 turns it off)."""
        self._check(self.lib.stk_set_persistent(self.h, max_elements, ctas_per_sm), "stk_set_persistent")

    def barrier_selftest(self, absent=-1, limit_ticks=2_000_000):
        """(status, passages): STK_OK or the TIMEOUT code of the bounded grid
        barrier's self-test; raises nothing for a timeout."""
        n = ctypes.c_int64()
        rc = self.lib.stk_barrier_selftest(self.h, absent, limit_ticks, ctypes.byref(n))
        if rc not in (STK_OK, -4):
            self._check(rc, "stk_barrier_selftest")
        return rc, n.value

    def set_colouring(self, mode):
        """COLOURS_AUTO (checkerboard for the single-phase standard form,
        2^d parity colours otherwise), COLOURS_PARITY or COLOURS_CHECKERBOARD;
        takes effect at the next setup."""
        self._check(self.lib.stk_set_colouring(self.h, mode), "stk_set_colouring")

    def setup(self, stream=None):
        self._check(self.lib.stk_setup(self.h, _stream(stream)), "stk_setup")
        nl, ne, nb, _ = self.sizes()
        if getattr(self, "cut", False):
            self.ne = int(ne[0])   # merged cut-cell elements
        self._level_n = [int(v) * nb for v in ne]   # unknowns per level, for the vector checks
        self._nb = nb

    def _n(self, level=0):
        """Unknowns of a level (known after setup; the library itself rejects
        calls before setup)."""
        sizes = getattr(self, "_level_n", None)
        if sizes is None:
            raise StkError("call setup first")
        if not 0 <= level < len(sizes):
            raise ValueError("level %d outside 0..%d" % (level, len(sizes) - 1))
        return sizes[level]

    def sizes(self):
        nl = ctypes.c_int()
        nb = ctypes.c_int()
        sn = ctypes.c_int()
        self._check(self.lib.stk_get_sizes(self.h, ctypes.byref(nl), None, ctypes.byref(nb),
                                           ctypes.byref(sn)), "stk_get_sizes")
        ne = np.zeros(nl.value, dtype=np.int64)
        self._check(self.lib.stk_get_sizes(self.h, None, ne.ctypes.data_as(_c_i64_p), None, None),
                    "stk_get_sizes")
        return nl.value, ne, nb.value, sn.value

    def get_block(self, level, i, j, nb):
        out = np.zeros((nb, nb))
        self._check(self.lib.stk_get_block(self.h, level, i, j, out.ctypes.data_as(_c_dbl_p)),
                    "stk_get_block")
        return out

    def _check_rhs_data(self, f_vol, bdata, ne, idata=None):
        d = self.d
        if ne != self.ne:
            raise ValueError("assemble_rhs: ne = %d, the mesh has %d elements" % (ne, self.ne))
        self._expect("f_vol", f_vol, self.num_points(PTS_VOLUME), d + 1)
        if bdata is not None:
            self._expect("bdata", bdata, self.num_points(PTS_BOUNDARY_FACE), d)
        if idata is not None:
            kind = PTS_INTERFACE if getattr(self, "cut", False) else PTS_INTERIOR_FACE
            self._expect("idata", idata, self.num_points(kind), 2 * d)

    def assemble_rhs(self, f_vol, bdata, ne, nb):
        self._check_rhs_data(f_vol, bdata, ne)
        b = np.zeros((ne, nb))
        f = _dbl(f_vol)
        bd = _dbl(bdata) if bdata is not None else (None, None)
        self._check(self.lib.stk_assemble_rhs(self.h, f[0], bd[0], b.ctypes.data_as(_c_dbl_p)),
                    "stk_assemble_rhs")
        return b

    def residual(self, x, b, r, want_norm=False, stream=None):
        nrm = ctypes.c_double()
        n = self._n()
        self._check(self.lib.stk_residual(self.h, _vec("x", x, n), _vec("b", b, n), _vec("r", r, n),
                                          ctypes.byref(nrm) if want_norm else None, _stream(stream)),
                    "stk_residual")
        return nrm.value if want_norm else None

    def gs_colour(self, level, colour, x, b, stream=None):
        n = self._n(level)
        self._check(self.lib.stk_gs_colour(self.h, level, colour, _vec("x", x, n), _vec("b", b, n),
                                           _stream(stream)),
                    "stk_gs_colour")

    def gs_colour_ex(self, level, colour, precision, x, b, stream=None):
        n, es = self._n(level), 8 if precision == FP64 else 4
        self._check(self.lib.stk_gs_colour_ex(self.h, level, colour, precision, _vec("x", x, n, es),
                                              _vec("b", b, n, es), _stream(stream)), "stk_gs_colour_ex")

    def residual_ex(self, level, precision, x, b, r, stream=None):
        n, es = self._n(level), 8 if precision == FP64 else 4
        self._check(self.lib.stk_residual_ex(self.h, level, precision, _vec("x", x, n, es), _vec("b", b, n, es),
                                             _vec("r", r, n, es), _stream(stream)), "stk_residual_ex")

    def vcycle(self, x, b, stream=None):
        n = self._n()
        self._check(self.lib.stk_vcycle(self.h, _vec("x", x, n), _vec("b", b, n), _stream(stream)), "stk_vcycle")

    def restrict(self, level, r, rc, stream=None):
        self._check(self.lib.stk_restrict(self.h, level, _vec("r", r, self._n(level)),
                                          _vec("rc", rc, self._n(level + 1)), _stream(stream)), "stk_restrict")

    def prolong(self, level, xc, x, stream=None):
        self._check(self.lib.stk_prolong(self.h, level, _vec("xc", xc, self._n(level + 1)),
                                         _vec("x", x, self._n(level)), _stream(stream)), "stk_prolong")

    def bottom_solve(self, b, x, stream=None):
        sizes = getattr(self, "_level_n", None)
        n = self._n(len(sizes) - 1 if sizes else 0)
        self._check(self.lib.stk_bottom_solve(self.h, _vec("b", b, n), _vec("x", x, n), _stream(stream)),
                    "stk_bottom_solve")

    def solve(self, x, b, rtol=1e-10, maxit=100, stream=None):
        it = ctypes.c_int()
        hist = np.zeros(maxit + 1)
        n = self._n()
        rc = self.lib.stk_solve(self.h, _vec("x", x, n), _vec("b", b, n), rtol, maxit, ctypes.byref(it),
                                hist.ctypes.data_as(_c_dbl_p), _stream(stream))
        self._check(rc, "stk_solve")
        return it.value, hist[: it.value + 1]

    def gmres_rho(self, x0, reduction=1e-8, maxit=100, stream=None):
        """eq. (rho): (rho, iterations, relative preconditioned residual
        history, Arnoldi matrix (maxit+1) x maxit) of left-preconditioned
        GMRES on V A x = 0 from the device vector x0."""
        rho = ctypes.c_double()
        it = ctypes.c_int()
        hist = np.zeros(maxit + 1)
        hess = np.zeros((maxit + 1, maxit))
        self._check(self.lib.stk_gmres_rho(self.h, _vec("x0", x0, self._n()), reduction, maxit, ctypes.byref(rho), ctypes.byref(it),
                                           hist.ctypes.data_as(_c_dbl_p), hess.ctypes.data_as(_c_dbl_p),
                                           _stream(stream)), "stk_gmres_rho")
        n = it.value
        return rho.value, n, hist[: n + 1], hess

    def residual_norm_static(self, x, b, r, norm2, stream=None):
        """stk_residual_norm_static: r = b - A x and ||r||^2 into the device
        scalar norm2, using only the library's fixed static scratch."""
        n = self._n()
        self._check(self.lib.stk_residual_norm_static(self.h, _vec("x", x, n), _vec("b", b, n), _vec("r", r, n),
                                                      _vec("norm2", norm2, 1, at_least=True), _stream(stream)),
                    "stk_residual_norm_static")

    def solve_multi(self, X, B, nrhs, rtol=1e-10, maxit=50, inner=1, stream=None):
        it = ctypes.c_int()
        hist = np.zeros((maxit + 1) * nrhs)
        n = self._n() * nrhs
        rc = self.lib.stk_solve_multi(self.h, _vec("X", X, n), _vec("B", B, n), nrhs, rtol, maxit, inner, ctypes.byref(it),
                                      hist.ctypes.data_as(_c_dbl_p), _stream(stream))
        self._check(rc, "stk_solve_multi")
        return it.value, hist[: (it.value + 1) * nrhs].reshape(it.value + 1, nrhs)

    def learn_setup(self, hidden=64, seed=0):
        self._check(self.lib.stk_learn_setup(self.h, hidden, seed), "stk_learn_setup")

    def learn_generate(self, nseeds, cycles, seed=0):
        self._check(self.lib.stk_learn_generate(self.h, nseeds, cycles, seed), "stk_learn_generate")

    def learn_train(self, epochs, batch=4096, lr=1e-3, seed=0):
        loss = ctypes.c_double()
        self._check(self.lib.stk_learn_train(self.h, epochs, batch, lr, seed, ctypes.byref(loss)), "stk_learn_train")
        return loss.value

    def learn_sizes(self):
        i, h, o = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        n, r = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.stk_learn_sizes(self.h, ctypes.byref(i), ctypes.byref(h), ctypes.byref(o),
                                             ctypes.byref(n), ctypes.byref(r)), "stk_learn_sizes")
        return i.value, h.value, o.value, n.value, r.value

    def learn_infer(self, r, y, nrm):
        n = self._n()
        self._check(self.lib.stk_learn_infer(self.h, _vec("r", r, n, 4), _vec("y", y, n, 4),
                                             _vec("nrm", nrm, n // self._nb, 4)), "stk_learn_infer")

    def learn_state(self, state, nvec):
        r = np.zeros(nvec, dtype=np.float32)
        self._check(self.lib.stk_learn_state(self.h, state, r.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
                    "stk_learn_state")
        return r

    def learn_error_state(self, state, nvec):
        e = np.zeros(nvec, dtype=np.float32)
        self._check(self.lib.stk_learn_error_state(self.h, state, e.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
                    "stk_learn_error_state")
        return e

    def learn_objective(self, objective):
        """0: residual objective ||r - A delta||^2 / ||r||^2; 1: supervised
        MSE against the normalised error e_i / ||r_i||."""
        self._check(self.lib.stk_learn_objective(self.h, objective), "stk_learn_objective")

    def learn_history(self, max_iters=1000):
        """(decisions, ratios, kappa) of the last solve: per outer iteration
        -1 plain, 1 kept, 0 undone; ratio ||r_new|| / (kappa ||r_old||)."""
        dec = np.zeros(max_iters, dtype=np.int32)
        rat = np.zeros(max_iters)
        n = ctypes.c_int()
        kap = ctypes.c_double()
        self._check(self.lib.stk_learn_history(self.h, dec.ctypes.data_as(_c_int_p), rat.ctypes.data_as(_c_dbl_p),
                                               max_iters, ctypes.byref(n), ctypes.byref(kap)), "stk_learn_history")
        m = min(n.value, max_iters)
        return dec[:m], rat[:m], kap.value

    def learn_grad(self, state, nparam):
        g = np.zeros(nparam, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self.lib.stk_learn_grad(self.h, state, g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                            ctypes.byref(loss)), "stk_learn_grad")
        return loss.value, g

    def learn_field(self, seed, x, stream=None):
        self._check(self.lib.stk_learn_field(self.h, int(seed), _vec("x", x, self._n(0)), _stream(stream)),
                    "stk_learn_field")

    def learn_enable(self, on):
        self._check(self.lib.stk_learn_enable(self.h, 1 if on else 0), "stk_learn_enable")

    def learn_stats(self):
        a, r = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.stk_learn_stats(self.h, ctypes.byref(a), ctypes.byref(r)), "stk_learn_stats")
        return a.value, r.value

    def learn_weights(self, count, values=None):
        """Read (values None) or write the learned smoother's weights."""
        if values is None:
            out = np.zeros(count, dtype=np.float32)
            self._check(self.lib.stk_learn_weights(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                   count, 0), "stk_learn_weights")
            return out
        v = np.ascontiguousarray(values, dtype=np.float32)
        self._check(self.lib.stk_learn_weights(self.h, v.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), count, 1),
                    "stk_learn_weights")

    def set_tuning(self, variant, precision, ctas_per_sm=0, stages=0):
        self._check(self.lib.stk_set_tuning(self.h, variant, precision, ctas_per_sm, stages), "stk_set_tuning")

    def set_launch_overlap(self, on):
        self._check(self.lib.stk_set_launch_overlap(self.h, 1 if on else 0), "stk_set_launch_overlap")

    def set_df_matvec(self, on):
        self._check(self.lib.stk_set_df_matvec(self.h, 1 if on else 0), "stk_set_df_matvec")

    def set_mrhs_tensor(self, on):
        self._check(self.lib.stk_set_mrhs_tensor(self.h, 1 if on else 0), "stk_set_mrhs_tensor")

    def set_wide_launch(self, max_positions):
        self._check(self.lib.stk_set_wide_launch(self.h, max_positions), "stk_set_wide_launch")

    def autotune(self, stream=None):
        """Time the element-kernel launch shapes and keep the fastest; returns
        ({variant, ctas_cycle, variant_fp64, ctas_fp64, wide_max, df_matvec}, (best_ms_cycle, best_ms_fp64))."""
        choice = (ctypes.c_int * 6)()
        best = (ctypes.c_double * 2)()
        self._check(self.lib.stk_autotune(self.h, choice, best, _stream(stream)), "stk_autotune")
        keys = ("variant", "ctas_cycle", "variant_fp64", "ctas_fp64", "wide_max", "df_matvec")
        return dict(zip(keys, list(choice))), (best[0], best[1])

    def set_solver(self, method, restart=30):
        self._check(self.lib.stk_set_solver(self.h, method, restart), "stk_set_solver")

    def set_phases(self, chi, mu_phase, scale=True):
        chi = np.ascontiguousarray(chi, dtype=np.int32)
        mu = np.ascontiguousarray(mu_phase, dtype=np.float64)
        self._expect("chi", chi, self.ne)
        if chi.size and (chi.min() < 1 or chi.max() > len(mu)):
            raise ValueError("set_phases: phase indices must lie in 1..%d" % len(mu))
        self._check(self.lib.stk_set_phases(self.h, len(mu), chi.ctypes.data_as(_c_int_p),
                                            mu.ctypes.data_as(_c_dbl_p), 1 if scale else 0), "stk_set_phases")

    def set_levelset_circle(self, centre, radius):
        """Embedded circle (cut-cell mesh); radius 0 returns to the Cartesian mesh."""
        self._check(self.lib.stk_set_levelset_circle(self.h, float(centre[0]), float(centre[1]), float(radius)),
                    "stk_set_levelset_circle")
        self.cut = radius > 0

    def set_cut_phases(self, mu_phase, scale=True):
        """Viscosities of the circle's inside (phase 1) and outside (phase 2),
        or one viscosity: the disc alone, Dirichlet data on the circle."""
        mu = np.ascontiguousarray(mu_phase, dtype=np.float64).ravel()
        if mu.size not in (1, 2):
            raise ValueError("mu_phase: 1 or 2 values, got %d" % mu.size)
        self._check(self.lib.stk_set_phases(self.h, int(mu.size), None, mu.ctypes.data_as(_c_dbl_p),
                                            1 if scale else 0), "stk_set_phases")
        self._cut_phases = int(mu.size)

    def set_phase_density(self, rho_phase, delta):
        if delta == 0:
            self._check(self.lib.stk_set_phase_density(self.h, None, 0.0), "stk_set_phase_density")
            return
        rho = np.ascontiguousarray(rho_phase, dtype=np.float64)
        self._expect("rho_phase", rho, getattr(self, "_cut_phases", 2))
        self._check(self.lib.stk_set_phase_density(self.h, rho.ctypes.data_as(_c_dbl_p), float(delta)),
                    "stk_set_phase_density")

    def set_element_warps(self, warps):
        self._check(self.lib.stk_set_element_warps(self.h, warps), "stk_set_element_warps")

    def get_point_phases(self, kind):
        out = np.zeros(self.num_points(kind), dtype=np.int32)
        self._check(self.lib.stk_get_point_phases(self.h, kind, out.ctypes.data_as(_c_int_p)),
                    "stk_get_point_phases")
        return out

    def get_interface(self, npts, d):
        cm = np.zeros(npts, dtype=np.int32)
        cp = np.zeros(npts, dtype=np.int32)
        nr = np.zeros((npts, d))
        self._check(self.lib.stk_get_interface(self.h, cm.ctypes.data_as(_c_int_p), cp.ctypes.data_as(_c_int_p),
                                               nr.ctypes.data_as(_c_dbl_p)), "stk_get_interface")
        return cm, cp, nr

    def assemble_rhs2(self, f_vol, bdata, idata, ne, nb):
        self._check_rhs_data(f_vol, bdata, ne, idata)
        b = np.zeros((ne, nb))
        f = _dbl(f_vol)
        bd = _dbl(bdata) if bdata is not None else (None, None)
        idd = _dbl(idata) if idata is not None else (None, None)
        self._check(self.lib.stk_assemble_rhs2(self.h, f[0], bd[0], idd[0], b.ctypes.data_as(_c_dbl_p)),
                    "stk_assemble_rhs2")
        return b

    def get_colours(self, level, ne):
        out = np.zeros(ne, dtype=np.int32)
        self._check(self.lib.stk_get_colours(self.h, level, out.ctypes.data_as(_c_int_p)), "stk_get_colours")
        return out

    def get_scaling(self, ne, nb):
        out = np.zeros((ne, nb))
        self._check(self.lib.stk_get_scaling(self.h, out.ctypes.data_as(_c_dbl_p)), "stk_get_scaling")
        return out

    def info(self, what):
        """stk_get_info: one of the INFO_* keys."""
        v = ctypes.c_int64()
        self._check(self.lib.stk_get_info(self.h, what, ctypes.byref(v)), "stk_get_info")
        return v.value

    def fp64_fma_rate(self, stream=None):
        """Measured FP64 FMA rate of the device in TFLOP/s (stk_fp64_fma_rate)."""
        v = ctypes.c_double()
        self._check(self.lib.stk_fp64_fma_rate(self.h, ctypes.byref(v), _stream(stream)), "stk_fp64_fma_rate")
        return v.value

    def launch_count(self):
        n = ctypes.c_int64()
        self._check(self.lib.stk_launch_count(self.h, ctypes.byref(n)), "stk_launch_count")
        return n.value


def solve_batch(contexts, xs, bs, rtol=1e-10, maxit=200, nrhs=1, inner=3, threads=0, stream=None):
    """stk_solve_batch over Context objects and device tensors (x, b per
    problem).  Returns (iterations, status codes); raises StkError naming the
    first failing problem."""
    n = len(contexts)
    if not (len(xs) == len(bs) == n):
        raise ValueError("one x and one b per context")
    lib = contexts[0].lib
    hs = (_vp * n)(*[c.h.value for c in contexts])
    xp = (_vp * n)(*[_vec("x", t, c._n() * nrhs).value for c, t in zip(contexts, xs)])
    bp = (_vp * n)(*[_vec("b", t, c._n() * nrhs).value for c, t in zip(contexts, bs)])
    it = (ctypes.c_int * n)()
    st = (ctypes.c_int * n)()
    rc = lib.stk_solve_batch(hs, n, xp, bp, nrhs, rtol, maxit, inner, threads, it, st, _stream(stream))
    if rc != STK_OK:
        bad = [i for i in range(n) if st[i] != STK_OK]
        i = bad[0] if bad else 0
        msg = lib.stk_last_error(contexts[i].h)
        raise StkError("stk_solve_batch: problem %d: %s (%s)" % (i, msg.decode() if msg else "",
                                                                ERRORS.get(rc, rc)))
    return list(it), list(st)


def solve_batch_persistent(contexts, xs, bs, rtol=1e-10, maxit=200, ctas_per_sm=3, stream=None):
    """stk_solve_batch_persistent: the whole batch (FP32-cycle contexts) by
    iterative refinement in one cooperative launch.  Returns (iterations,
    status codes, histories [n][maxit+1])."""
    n = len(contexts)
    if not (len(xs) == len(bs) == n):
        raise ValueError("one x and one b per context")
    lib = contexts[0].lib
    hs = (_vp * n)(*[c.h.value for c in contexts])
    xp = (_vp * n)(*[_vec("x", t, c._n()).value for c, t in zip(contexts, xs)])
    bp = (_vp * n)(*[_vec("b", t, c._n()).value for c, t in zip(contexts, bs)])
    it = (ctypes.c_int * n)()
    st = (ctypes.c_int * n)()
    hist = np.zeros((n, maxit + 1))
    rc = lib.stk_solve_batch_persistent(hs, n, xp, bp, rtol, maxit, ctas_per_sm, it, st,
                                        hist.ctypes.data_as(_c_dbl_p), _stream(stream))
    if rc != STK_OK:
        msg = lib.stk_last_error(contexts[0].h)
        raise StkError("stk_solve_batch_persistent: %s (%s)" % (msg.decode() if msg else "", ERRORS.get(rc, rc)))
    return list(it), list(st), hist


def cut_cells(n, centre, radius, q=8, merge_fraction=0.25, lo=(0.0, 0.0), hi=(1.0, 1.0)):
    """stk_cut_cells (host only): pieces of the n x n grid cut by a circle.
    Returns dict of arrays cell [np, 2], phase, area, element, colour and the
    interface length."""
    lib = load()
    lo_ = (ctypes.c_double * 2)(*lo)
    hi_ = (ctypes.c_double * 2)(*hi)
    npc = ctypes.c_int64(0)
    rc = lib.stk_cut_cells(n, lo_, hi_, centre[0], centre[1], radius, q, merge_fraction, ctypes.byref(npc),
                           None, None, None, None, None, None)
    if rc != STK_OK:
        raise StkError("stk_cut_cells: %s" % ERRORS.get(rc, rc))
    m = npc.value
    cell = np.zeros((m, 2), dtype=np.int32)
    phase = np.zeros(m, dtype=np.int32)
    area = np.zeros(m)
    elem = np.zeros(m, dtype=np.int32)
    col = np.zeros(m, dtype=np.int32)
    ilen = ctypes.c_double()
    rc = lib.stk_cut_cells(n, lo_, hi_, centre[0], centre[1], radius, q, merge_fraction, ctypes.byref(npc),
                           cell.ctypes.data_as(_c_int_p), phase.ctypes.data_as(_c_int_p), area.ctypes.data_as(_c_dbl_p),
                           elem.ctypes.data_as(_c_int_p), col.ctypes.data_as(_c_int_p), ctypes.byref(ilen))
    if rc != STK_OK:
        raise StkError("stk_cut_cells: %s" % ERRORS.get(rc, rc))
    return dict(cell=cell, phase=phase, area=area, element=elem, colour=col, interface_length=ilen.value)


def host_pseudo_inverse(A, theta=1e-10):
    """stk_host_pseudo_inverse: the bottom solver's least-squares inverse of
    the symmetric matrix A on the host (no device needed).  Returns
    (pinv, number of eigenvalues snapped to zero)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("square matrix expected")
    out = np.zeros((n, n))
    sn = ctypes.c_int()
    rc = load().stk_host_pseudo_inverse(n, A.ctypes.data_as(_c_dbl_p), theta, out.ctypes.data_as(_c_dbl_p),
                                        ctypes.byref(sn))
    if rc != STK_OK:
        raise StkError("stk_host_pseudo_inverse: %s" % ERRORS.get(rc, rc))
    return out, sn.value
