"""ctypes glue for the C++ oracle (test infrastructure only).

Wraps the plain CPU restatement of the discretised right-hand side N(q) and
of the three forms of J(q0) v (Eq. frechet): the literal double-precision
epsilon-quotient, the same quotient evaluated in binary128, and the exact
tangent by the complex step.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stab_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's shared library (g++, OpenMP, binary128 math)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", _LIB + ".tmp"]
    if platform.machine() in ("x86_64", "AMD64"):
        cmd.append("-lquadmath")
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Prob(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly0", ctypes.c_double), ("ly1", ctypes.c_double),
                ("lz", ctypes.c_double), ("stretch", ctypes.c_double),
                ("gamma", ctypes.c_double), ("Ma", ctypes.c_double), ("Re", ctypes.c_double),
                ("Pr", ctypes.c_double), ("S", ctypes.c_double), ("bulk", ctypes.c_double),
                ("low_order", ctypes.c_int)]


@dataclass(frozen=True)
class Problem:
    """Grid + flow parameters (nondimensional; Re <= 0 means inviscid).
    low_order = 1 selects the reduced operator: every derivative by
    second-order explicit differences instead of the compact schemes."""
    dim: int
    nx: int
    ny: int
    nz: int
    lx: float
    ly0: float
    ly1: float
    lz: float
    stretch: float
    gamma: float
    Ma: float
    Re: float
    Pr: float
    S: float
    bulk: float = 0.0
    low_order: int = 0

    @staticmethod
    def from_inputs(grid, flow, bulk: float = 0.0, low_order: int = 0) -> "Problem":
        return Problem(grid.dim, grid.nx, grid.ny, grid.nz, grid.lx, grid.ly0, grid.ly1, grid.lz,
                       grid.stretch, flow.gamma, flow.Ma, flow.Re, flow.Pr, flow.S, bulk, low_order)

    @property
    def npts(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n(self) -> int:
        return (self.dim + 2) * self.npts

    def c(self) -> _Prob:
        return _Prob(self.dim, self.nx, self.ny, self.nz, self.lx, self.ly0, self.ly1, self.lz,
                     self.stretch, self.gamma, self.Ma, self.Re, self.Pr, self.S, self.bulk, self.low_order)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Prob)
        L.orc_deriv_line.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        L.orc_deriv_line_low.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        L.orc_deriv_field.argtypes = [pp, dp, ctypes.c_int, ctypes.c_int, dp]
        for name in ("orc_rhs", "orc_rhs_quad"):
            getattr(L, name).argtypes = [pp, dp, dp, dp]
        for name in ("orc_jv_literal", "orc_jv_quad"):
            getattr(L, name).argtypes = [pp, dp, dp, ctypes.c_double, dp]
        L.orc_jv_tangent.argtypes = [pp, dp, dp, dp]
        L.orc_dense_jacobian.argtypes = [pp, dp, dp]
        L.orc_jacobian_columns.argtypes = [pp, dp, ctypes.POINTER(ctypes.c_long), ctypes.c_long, dp]
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _cplx_view(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.complex128).reshape(-1)).view(np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def deriv_line(f, h: float, order: int = 1, periodic: bool = True, low: bool = False) -> np.ndarray:
    """Compact derivative of one line, or (low) the reduced operator's second-order explicit one."""
    f = _f64(f)
    out = np.empty_like(f)
    (lib().orc_deriv_line_low if low else lib().orc_deriv_line)(order, int(periodic), f.size, h, _dp(f), _dp(out))
    return out


def deriv_field(P: Problem, f, axis: int, order: int = 1) -> np.ndarray:
    f = _f64(f).reshape(-1)
    out = np.empty_like(f)
    pc = P.c()
    lib().orc_deriv_field(ctypes.byref(pc), _dp(f), axis, order, _dp(out))
    return out


def rhs(P: Problem, q, q0sw=None, quad: bool = False) -> np.ndarray:
    """N(q) (Eq. navier_stokes on the grid); the y-boundary wave switch is frozen on q0sw (default q)."""
    q = _f64(q).reshape(-1)
    q0sw = q if q0sw is None else _f64(q0sw).reshape(-1)
    out = np.empty_like(q)
    pc = P.c()
    (lib().orc_rhs_quad if quad else lib().orc_rhs)(ctypes.byref(pc), _dp(q0sw), _dp(q), _dp(out))
    return out


def jv(P: Problem, q0, v, mode: str = "tangent", eps: float | None = None) -> np.ndarray:
    """J(q0) v for complex v.  mode: 'tangent' (complex step), 'quad' (exact
    epsilon-quotient) or 'literal' (double epsilon-quotient)."""
    q0 = _f64(q0).reshape(-1)
    vv = _cplx_view(v)
    out = np.empty_like(vv)
    pc = P.c()
    if mode == "tangent":
        lib().orc_jv_tangent(ctypes.byref(pc), _dp(q0), _dp(vv), _dp(out))
    else:
        if eps is None:
            eps = knoll_keyes_eps(q0, v)
        fn = lib().orc_jv_quad if mode == "quad" else lib().orc_jv_literal
        fn(ctypes.byref(pc), _dp(q0), _dp(vv), float(eps), _dp(out))
    return out.view(np.complex128)


def knoll_keyes_eps(q0, v) -> float:
    """eps = sqrt(eps_m) (1 + ||q0||_2) / ||v||_2 (one eps per complex direction)."""
    nv = float(np.linalg.norm(np.asarray(v).reshape(-1)))
    return float(np.sqrt(np.finfo(np.float64).eps) * (1.0 + np.linalg.norm(np.asarray(q0).reshape(-1))) / nv)


def dense_jacobian(P: Problem, q0) -> np.ndarray:
    """Dense tangent Jacobian (n x n, row-major numpy array)."""
    q0 = _f64(q0).reshape(-1)
    n = P.n
    J = np.empty((n, n))  # filled column-major, i.e. J.T in row-major terms
    pc = P.c()
    lib().orc_dense_jacobian(ctypes.byref(pc), _dp(q0), _dp(J))
    return J.T.copy()


def jacobian_columns(P: Problem, q0, cols) -> np.ndarray:
    """Columns J[:, cols] of the tangent Jacobian, shape (n, len(cols))."""
    q0 = _f64(q0).reshape(-1)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.empty((cols.size, P.n))
    pc = P.c()
    lib().orc_jacobian_columns(ctypes.byref(pc), _dp(q0), cols.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                               cols.size, _dp(out))
    return out.T.copy()
