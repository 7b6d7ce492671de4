"""Python access to the plain CPU FP64 oracle (hjm_oracle.c).

TEST INFRASTRUCTURE ONLY. The oracle is the slow, obviously-correct reference
the GPU library is checked against. Only the test suite, the smoke check and
the benchmark's CPU-baseline leg may import this package; the product path
never does, and the oracle shares no code with it.

Pinned functions (what fixes each, beyond the oracle itself) are listed in the
module docstrings of tests/test_oracle_pins.py. Functions without an external
pin: none of the exported calls is unpinned, but the caplet price with
epsilon > 0 and rho != 0 has no closed form (parity of that case rests on
self-convergence and on the pinned pieces it is built from).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hjm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None


MAX_KNOTS = 32


class Curve(C.Structure):
    _fields_ = [("kind", C.c_int), ("flat_rate", C.c_double), ("beta0", C.c_double),
                ("beta1", C.c_double), ("beta2", C.c_double), ("tau", C.c_double),
                ("n_knots", C.c_int), ("knot_t", C.c_double * MAX_KNOTS), ("knot_P", C.c_double * MAX_KNOTS)]


class Model(C.Structure):
    _fields_ = [("kappa", C.c_double), ("lambda_", C.c_double), ("gamma", C.c_double),
                ("theta", C.c_double), ("epsilon", C.c_double), ("rho", C.c_double),
                ("v0", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("n_r", C.c_int), ("n_y", C.c_int), ("n_v", C.c_int), ("n_steps", C.c_int),
                ("r_min", C.c_double), ("r_max", C.c_double), ("y_max", C.c_double),
                ("v_max", C.c_double), ("alpha_r", C.c_double), ("alpha_y", C.c_double),
                ("alpha_v", C.c_double), ("k_r", C.c_double), ("k_v", C.c_double),
                ("center_r_on_strike", C.c_int), ("theta_adi", C.c_double),
                ("y_boundary_order", C.c_int), ("explicit_midpoint", C.c_int), ("scheme", C.c_int)]


class Inst(C.Structure):
    _fields_ = [("kind", C.c_int), ("T", C.c_double), ("TM", C.c_double), ("K", C.c_double),
                ("strike_atm_relative", C.c_int)]


def _fill(struct_t, d):
    s = struct_t()
    for name, typ in struct_t._fields_:
        if hasattr(typ, "_length_"):  # fixed-size array: the given values, zero-padded
            vals = [float(v) for v in d.get(name, ())]
            getattr(s, name)[:len(vals)] = vals
        elif name == "n_knots":
            setattr(s, name, int(d.get(name, 0)))
        else:
            setattr(s, name, d[name])
    return s


_LIB_OMP = os.path.join(_LIB_DIR, "liborc_omp.so")


def build(force=False, omp=False):
    """Compile the oracle into oracle/_build/liborc.so (plain gcc, -O2), or
    with omp into liborc_omp.so: the same source with its OpenMP pragmas
    active (lines of a pass shared among threads; used only to time the
    oracle on all host cores, same results as the serial build)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    out = _LIB_OMP if omp else _LIB
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)
            and os.path.getmtime(out) >= os.path.getmtime(os.path.join(_HERE, "hjm_oracle.h"))):
        return out
    tmp = out + ".tmp.%d" % os.getpid()
    flags = ["-fopenmp"] if omp else ["-Wno-unknown-pragmas"]
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared"] + flags + ["-o", tmp, _SRC, "-lm"])
    os.replace(tmp, out)
    return out


_lib_omp = None


def lib(omp=False):
    """The oracle library with argument types set; omp: the OpenMP build."""
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if omp else _lib) is None:
            L = C.CDLL(build(omp=omp))
            P = C.POINTER
            dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
            L.orc_ctx_create.argtypes = [P(Curve), P(Model), P(Grid), P(Inst), P(C.c_void_p)]
            L.orc_ctx_create.restype = C.c_int
            L.orc_ctx_destroy.argtypes = [C.c_void_p]
            L.orc_n_points.argtypes = [C.c_void_p]
            L.orc_n_points.restype = C.c_long
            for f in ("orc_strike", "orc_dt"):
                getattr(L, f).argtypes = [C.c_void_p]
                getattr(L, f).restype = C.c_double
            L.orc_axis.argtypes = [C.c_void_p, C.c_int, dp, dp, dp]
            for f in ("orc_curve_f", "orc_curve_dfdt", "orc_curve_P"):
                getattr(L, f).argtypes = [P(Curve), C.c_double]
                getattr(L, f).restype = C.c_double
            L.orc_G.argtypes = [C.c_double, C.c_double]
            L.orc_G.restype = C.c_double
            L.orc_bond.argtypes = [P(Curve), P(Model)] + [C.c_double] * 4
            L.orc_bond.restype = C.c_double
            L.orc_gauss_caplet.argtypes = [P(Curve), P(Model)] + [C.c_double] * 3
            L.orc_gauss_caplet.restype = C.c_double
            L.orc_atm_strike.argtypes = [P(Curve), C.c_double, C.c_double]
            L.orc_atm_strike.restype = C.c_double
            L.orc_terminal.argtypes = [C.c_void_p, dp]
            L.orc_explicit.argtypes = [C.c_void_p, C.c_int, dp, dp]
            L.orc_apply_F.argtypes = [C.c_void_p, C.c_double, dp, dp]
            L.orc_apply_dir.argtypes = [C.c_void_p, C.c_int, C.c_double, dp, dp]
            L.orc_solve_dir.argtypes = [C.c_void_p, C.c_int, C.c_double, dp, dp]
            L.orc_solve_dir.restype = C.c_long
            L.orc_line_matrix.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_long, dp, dp, dp]
            L.orc_step.argtypes = [C.c_void_p, C.c_int, dp]
            L.orc_march.argtypes = [C.c_void_p, dp]
            L.orc_readout.argtypes = [C.c_void_p, dp]
            L.orc_readout.restype = C.c_double
            L.orc_readout_greeks.argtypes = [C.c_void_p, dp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_readout_greeks.restype = None
            L.orc_time.argtypes = [C.c_void_p, C.c_double]
            L.orc_time.restype = C.c_double
            L.orc_dirichlet.argtypes = [C.c_void_p] + [C.c_double] * 3
            L.orc_dirichlet.restype = C.c_double
            L.orc_price.argtypes = [P(Curve), P(Model), P(Grid), P(Inst), P(C.c_double)]
            L.orc_price.restype = C.c_int
            if omp:
                _lib_omp = L
            else:
                _lib = L
    return _lib_omp if omp else _lib


class OracleError(ValueError):
    pass


class Ctx:
    """One discretised problem: an item dict (curve, model, grid, inst)."""

    def __init__(self, item, omp=False):
        self.item = item
        self._L = lib(omp)
        self._c = _fill(Curve, item["curve"])
        self._m = _fill(Model, item["model"])
        self._g = _fill(Grid, item["grid"])
        self._i = _fill(Inst, item["inst"])
        h = C.c_void_p()
        st = self._L.orc_ctx_create(C.byref(self._c), C.byref(self._m), C.byref(self._g),
                                  C.byref(self._i), C.byref(h))
        if st != 0:
            raise OracleError("oracle rejected the inputs (status %d)" % st)
        self._h = h
        g = item["grid"]
        self.shape = (g["n_y"], g["n_v"], g["n_r"])  # array order j, k, i
        self.n = {0: g["n_r"], 1: g["n_v"], 2: g["n_y"]}

    def close(self):
        if getattr(self, "_h", None):
            self._L.orc_ctx_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # scalars
    @property
    def strike(self):
        return self._L.orc_strike(self._h)

    @property
    def dt(self):
        return self._L.orc_dt(self._h)

    def time(self, n):
        return self._L.orc_time(self._h, float(n))

    def axis(self, axis):
        n = self.n[axis]
        z, J, J2 = np.empty(n), np.empty(n), np.empty(n)
        self._L.orc_axis(self._h, axis, z, J, J2)
        return z, J, J2

    def _field(self):
        return np.empty(self.shape, dtype=np.float64)

    def terminal(self):
        U = self._field()
        self._L.orc_terminal(self._h, U)
        return U

    def explicit(self, n, U):
        out = self._field()
        self._L.orc_explicit(self._h, int(n), np.ascontiguousarray(U, dtype=np.float64), out)
        return out

    def apply_F(self, t, U):
        out = self._field()
        self._L.orc_apply_F(self._h, float(t), np.ascontiguousarray(U, dtype=np.float64), out)
        return out

    def apply_dir(self, d, t, U):
        out = self._field()
        self._L.orc_apply_dir(self._h, int(d), float(t), np.ascontiguousarray(U, dtype=np.float64), out)
        return out

    def solve_dir(self, d, t, rhs, return_bad=False):
        out = self._field()
        bad = self._L.orc_solve_dir(self._h, int(d), float(t),
                                  np.ascontiguousarray(rhs, dtype=np.float64), out)
        return (out, bad) if return_bad else out

    def line_matrix(self, d, t, line):
        n = self.n[d]
        a, b, c = np.empty(n), np.empty(n), np.empty(n)
        self._L.orc_line_matrix(self._h, int(d), float(t), int(line), a, b, c)
        return a, b, c

    def step(self, n, U):
        U = np.array(U, dtype=np.float64, copy=True)
        self._L.orc_step(self._h, int(n), U)
        return U

    def march(self):
        U = self._field()
        self._L.orc_march(self._h, U)
        return U

    def readout(self, U):
        return self._L.orc_readout(self._h, np.ascontiguousarray(U, dtype=np.float64))

    def readout_greeks(self, U):
        """(dC/dr, dC/dv) at the read-out point."""
        a, b = C.c_double(), C.c_double()
        self._L.orc_readout_greeks(self._h, np.ascontiguousarray(U, dtype=np.float64), C.byref(a), C.byref(b))
        return a.value, b.value

    def dirichlet(self, t, r, y):
        return self._L.orc_dirichlet(self._h, float(t), float(r), float(y))


def price(item, omp=False):
    """Price of one item by the whole march (omp: the OpenMP build, same
    results, for the benchmark-size cases)."""
    p = C.c_double()
    st = lib(omp).orc_price(C.byref(_fill(Curve, item["curve"])), C.byref(_fill(Model, item["model"])),
                         C.byref(_fill(Grid, item["grid"])), C.byref(_fill(Inst, item["inst"])),
                         C.byref(p))
    if st != 0:
        raise OracleError("oracle rejected the inputs (status %d)" % st)
    return p.value


def curve_f(curve, t):
    return lib().orc_curve_f(C.byref(_fill(Curve, curve)), float(t))


def curve_dfdt(curve, t):
    return lib().orc_curve_dfdt(C.byref(_fill(Curve, curve)), float(t))


def curve_P(curve, t):
    return lib().orc_curve_P(C.byref(_fill(Curve, curve)), float(t))


def G(kappa, s):
    return lib().orc_G(float(kappa), float(s))


def bond(curve, model, t, S, r, y):
    return lib().orc_bond(C.byref(_fill(Curve, curve)), C.byref(_fill(Model, model)),
                          float(t), float(S), float(r), float(y))


def gauss_caplet(curve, model, T, TM, K):
    return lib().orc_gauss_caplet(C.byref(_fill(Curve, curve)), C.byref(_fill(Model, model)),
                                  float(T), float(TM), float(K))


def atm_strike(curve, T, TM):
    return lib().orc_atm_strike(C.byref(_fill(Curve, curve)), float(T), float(TM))
