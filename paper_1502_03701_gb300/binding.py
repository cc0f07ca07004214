"""Thin ctypes binding of the C ABI declared in include/stab.h.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device vectors are complex128 torch tensors on the GPU (their
data_ptr() is passed through); the handle is bound to the torch stream that
is current when it is created.  The library is loaded from this package's
directory and a missing or unloadable library raises immediately.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstab.so")

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NOT_CONVERGED", 5: "BREAKDOWN",
          6: "NUMERIC", 7: "TIMEOUT", 8: "BUSY", 9: "UNSUPPORTED"}

SYMBOLS = ["stab_default_opts", "stab_create", "stab_destroy", "stab_last_error", "stab_size", "stab_apply_J",
           "stab_last_eps", "stab_solve", "stab_precond_build", "stab_precond_apply", "stab_precond_block",
           "stab_orthogonalize", "stab_eigs", "stab_get_stats", "stab_orthogonalize_noalloc", "stab_timing",
           "stab_timing_read", "stab_autotune", "stab_autotune_save", "stab_autotune_load",
           "stab_set_line_config", "stab_trim_memory", "stab_estimate_bytes", "stab_eigs_batch",
           "stab_server_create", "stab_server_submit", "stab_server_wait", "stab_server_result",
           "stab_server_stats", "stab_server_destroy", "stab_jv_batch_create", "stab_jv_batch_apply",
           "stab_jv_batch_last_error", "stab_jv_batch_destroy", "stab_jv_batch_precond_apply",
           "stab_jv_batch_orthogonalize", "stab_jv_batch_solve", "stab_jv_batch_eigs", "stab_server_set_cohort"]

# stab_phase, in enum order
PHASES = ["eps", "temperature", "line_y", "line_z", "line_x", "pointwise", "cgs2", "precond_apply"]


class StabError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly0", ctypes.c_double), ("ly1", ctypes.c_double),
                ("lz", ctypes.c_double), ("stretch", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("sutherland_S", ctypes.c_double), ("bulk_visc_ratio", ctypes.c_double),
                ("eps_mode", ctypes.c_int), ("eps", ctypes.c_double), ("gmres_m", ctypes.c_int),
                ("gmres_max_restarts", ctypes.c_int), ("gmres_tol", ctypes.c_double), ("precond", ctypes.c_int),
                ("tile", ctypes.c_int * 3), ("precond_prec", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("seed", ctypes.c_ulonglong), ("gmres_basis_prec", ctypes.c_int),
                ("stencil_prec", ctypes.c_int), ("lgmres_k", ctypes.c_int),
                ("precond_factor", ctypes.c_int), ("gmres_inner_m", ctypes.c_int),
                ("gmres_inner_tol", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("jv_calls", ctypes.c_longlong), ("gmres_iterations", ctypes.c_longlong),
                ("gmres_solves", ctypes.c_longlong), ("arnoldi_steps", ctypes.c_longlong),
                ("restarts", ctypes.c_longlong), ("precond_builds", ctypes.c_longlong),
                ("seconds_total", ctypes.c_double), ("seconds_precond", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class EigJob(ctypes.Structure):
    _fields_ = [("sigma_re", ctypes.c_double), ("sigma_im", ctypes.c_double), ("tau_re", ctypes.c_double),
                ("tau_im", ctypes.c_double), ("nev", ctypes.c_int), ("ncv", ctypes.c_int), ("tol", ctypes.c_double),
                ("v0", ctypes.c_void_p), ("lambda_", ctypes.POINTER(ctypes.c_double)), ("vecs", ctypes.c_void_p),
                ("resid", ctypes.POINTER(ctypes.c_double)), ("nconv", ctypes.c_int), ("status", ctypes.c_int),
                ("stats", Stats)]


class Request(ctypes.Structure):
    _fields_ = [("base_flow", ctypes.POINTER(ctypes.c_double)), ("grid", Grid), ("Ma", ctypes.c_double),
                ("Re", ctypes.c_double), ("Pr", ctypes.c_double), ("opts", ctypes.POINTER(Opts)),
                ("sigma_re", ctypes.c_double), ("sigma_im", ctypes.c_double), ("tau_re", ctypes.c_double),
                ("tau_im", ctypes.c_double), ("nev", ctypes.c_int), ("ncv", ctypes.c_int), ("tol", ctypes.c_double),
                ("vecs", ctypes.c_void_p)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("nconv", ctypes.c_int), ("queued_s", ctypes.c_double),
                ("run_s", ctypes.c_double), ("latency_s", ctypes.c_double), ("est_bytes", ctypes.c_longlong),
                ("stats", Stats)]


_lib = None


def load():
    """Load libstab.so (must have been built by build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} missing (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double
    L.stab_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.stab_default_opts.restype = None
    L.stab_create.argtypes = [ctypes.POINTER(vp), vp, i, ctypes.POINTER(Grid), d, d, d, ctypes.POINTER(Opts), vp]
    L.stab_destroy.argtypes = [vp]
    L.stab_destroy.restype = None
    L.stab_last_error.argtypes = [vp]
    L.stab_last_error.restype = ctypes.c_char_p
    L.stab_size.argtypes = [vp]
    L.stab_size.restype = ctypes.c_longlong
    L.stab_apply_J.argtypes = [vp, vp, vp, d, d]
    L.stab_last_eps.argtypes = [vp, dp]
    L.stab_solve.argtypes = [vp, d, d, vp, vp, ctypes.POINTER(ctypes.c_int)]
    L.stab_precond_build.argtypes = [vp, d, d]
    L.stab_precond_apply.argtypes = [vp, vp, vp]
    L.stab_precond_block.argtypes = [vp, d, d, ctypes.c_longlong, dp]
    L.stab_orthogonalize.argtypes = [vp, vp, i, vp, dp, dp]
    L.stab_eigs.argtypes = [vp, d, d, d, d, i, i, d, vp, dp, vp, dp, ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(Stats)]
    L.stab_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    L.stab_orthogonalize_noalloc.argtypes = [vp, i, ctypes.c_longlong, vp, dp, dp, vp]
    L.stab_timing.argtypes = [vp, i]
    L.stab_autotune.argtypes = [vp, i, ctypes.POINTER(ctypes.c_int), dp]
    L.stab_autotune_save.argtypes = [ctypes.c_char_p]
    L.stab_set_line_config.argtypes = [vp, i, i, i, i]
    L.stab_trim_memory.argtypes = []
    L.stab_estimate_bytes.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Opts), i, i, i]
    L.stab_estimate_bytes.restype = ctypes.c_longlong
    L.stab_eigs_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(EigJob), i, i]
    L.stab_server_create.argtypes = [ctypes.POINTER(vp), i, ctypes.c_longlong, i]
    L.stab_server_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_longlong)]
    L.stab_server_wait.argtypes = [vp, ctypes.c_longlong, d]
    L.stab_server_result.argtypes = [vp, ctypes.c_longlong, dp, dp, ctypes.POINTER(RequestInfo)]
    L.stab_server_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.stab_server_destroy.argtypes = [vp]
    L.stab_autotune_load.argtypes = [ctypes.c_char_p]
    L.stab_timing_read.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    L.stab_jv_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), i, vp]
    L.stab_jv_batch_apply.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), dp]
    L.stab_jv_batch_precond_apply.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.stab_jv_batch_orthogonalize.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(i), ctypes.POINTER(vp), dp, dp]
    L.stab_server_set_cohort.argtypes = [vp, i]
    L.stab_jv_batch_solve.argtypes = [vp, dp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i)]
    L.stab_jv_batch_eigs.argtypes = [vp, ctypes.POINTER(EigJob)]
    L.stab_jv_batch_last_error.argtypes = [vp]
    L.stab_jv_batch_last_error.restype = ctypes.c_char_p
    L.stab_jv_batch_destroy.argtypes = [vp]
    L.stab_jv_batch_destroy.restype = None
    for name in SYMBOLS:
        if name not in ("stab_default_opts", "stab_destroy", "stab_last_error", "stab_size", "stab_estimate_bytes",
                        "stab_server_destroy", "stab_jv_batch_last_error", "stab_jv_batch_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def default_opts(**kw) -> Opts:
    o = Opts()
    load().stab_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "tile":
            t = list(v) + [1] * (3 - len(v))
            o.tile[0], o.tile[1], o.tile[2] = t[:3]
        else:
            setattr(o, k, v)
    return o


def _ptr(t) -> int:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return int(t)


def _vec_ptr(t, count: int, what: str) -> int:
    """Device address of a complex128 vector of at least ``count`` entries.

    torch tensors are checked (complex128, CUDA, contiguous, long enough)
    because the library cannot see their sizes; plain integers are taken as
    raw device addresses on the caller's responsibility."""
    if t is None:
        raise ValueError(f"{what}: missing vector")
    if hasattr(t, "data_ptr"):
        import torch
        if t.dtype != torch.complex128:
            raise ValueError(f"{what}: expected complex128, got {t.dtype}")
        if not t.is_cuda:
            raise ValueError(f"{what}: expected a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"{what}: expected a contiguous tensor")
        if t.numel() < count:
            raise ValueError(f"{what}: {t.numel()} entries, need {count}")
        return t.data_ptr()
    return int(t)


def orthogonalize_noalloc(V, k: int, n: int, w, stream=None):
    """CGS2 of w against k columns of V without any device allocation (no handle)."""
    L = load()
    hc = np.zeros(2 * max(k, 1))
    nrm = ctypes.c_double()
    if 0 <= k <= 128 and 1 <= n <= (1 << 28):  # sizes the library takes: check the tensors against them
        pV = _vec_ptr(V, k * n, "orthogonalize_noalloc V") if k > 0 else _ptr(V)
        pw = _vec_ptr(w, n, "orthogonalize_noalloc w")
    else:  # the library refuses these sizes before touching memory
        pV, pw = _ptr(V), _ptr(w)
    st = L.stab_orthogonalize_noalloc(pV, k, n, pw,
                                      hc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      ctypes.byref(nrm), None if stream is None else stream.cuda_stream)
    if st != 0:
        raise StabError(st, L.stab_last_error(None).decode())
    return hc.view(np.complex128)[:k], nrm.value


@dataclass
class EigResult:
    lam: np.ndarray
    resid: np.ndarray
    nconv: int
    status: int
    stats: dict


class Stab:
    """One stability problem (grid, base state, flow parameters) on the GPU."""

    def __init__(self, base_flow, grid, Ma: float, Re: float, Pr: float = 0.71, stream=None, **opts):
        import torch
        L = load()
        self._L = L
        self.opts = default_opts(**opts)
        g = Grid(grid.dim, grid.nx, grid.ny, grid.nz, grid.lx, grid.ly0, grid.ly1, grid.lz, grid.stretch)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        if isinstance(base_flow, torch.Tensor) and base_flow.is_cuda:
            bf = base_flow.contiguous().to(torch.float64)
            st = L.stab_create(ctypes.byref(h), bf.data_ptr(), 1, ctypes.byref(g), Ma, Re, Pr,
                               ctypes.byref(self.opts), stream.cuda_stream)
        else:
            bf = np.ascontiguousarray(np.asarray(base_flow, dtype=np.float64).reshape(-1))
            st = L.stab_create(ctypes.byref(h), bf.ctypes.data, 0, ctypes.byref(g), Ma, Re, Pr,
                               ctypes.byref(self.opts), stream.cuda_stream)
        if st != 0:
            raise StabError(st, L.stab_last_error(None).decode())
        self._h = h
        self.n = int(L.stab_size(h))
        self._npts_v = grid.nx * grid.ny * grid.nz
        self._dim_v = grid.dim

    def _check(self, st: int, allow=()):
        if st != 0 and st not in allow:
            raise StabError(st, self._L.stab_last_error(self._h).decode())
        return st

    def close(self):
        if getattr(self, "_h", None):
            self._L.stab_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_J(self, v, out, shift: complex = 0.0):
        self._check(self._L.stab_apply_J(self._h, _ptr(v), _ptr(out), complex(shift).real, complex(shift).imag))
        return out

    def last_eps(self) -> float:
        e = ctypes.c_double()
        self._check(self._L.stab_last_eps(self._h, ctypes.byref(e)))
        return e.value

    def solve(self, sigma: complex, b, x) -> tuple[int, int]:
        it = ctypes.c_int()
        st = self._check(self._L.stab_solve(self._h, complex(sigma).real, complex(sigma).imag, _ptr(b), _ptr(x),
                                            ctypes.byref(it)), allow=(4,))
        return st, it.value

    def precond_build(self, sigma: complex):
        self._check(self._L.stab_precond_build(self._h, complex(sigma).real, complex(sigma).imag))

    def precond_apply(self, q, z):
        self._check(self._L.stab_precond_apply(self._h, _ptr(q), _ptr(z)))
        return z

    def precond_block(self, sigma: complex, t: int) -> np.ndarray:
        bsz = self.block_size()
        out = np.empty(2 * bsz * bsz)
        self._check(self._L.stab_precond_block(self._h, complex(sigma).real, complex(sigma).imag, t,
                                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out.view(np.complex128).reshape(bsz, bsz)

    def block_size(self) -> int:
        t = self.opts.tile
        return (self.n // self._npts()) * t[0] * t[1] * (t[2] if self._dim() == 3 else 1)

    def _npts(self):
        return self._npts_v

    def _dim(self):
        return self._dim_v

    def orthogonalize(self, V, k: int, w):
        hc = np.zeros(2 * max(k, 1))
        nrm = ctypes.c_double()
        self._check(self._L.stab_orthogonalize(self._h, _ptr(V), k, _ptr(w),
                                               hc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                               ctypes.byref(nrm)))
        return hc.view(np.complex128)[:k], nrm.value

    def eigs(self, sigma: complex, tau: complex, nev: int, ncv: int, tol: float, v0=None, vecs=None) -> EigResult:
        lam = np.zeros(2 * nev)
        res = np.zeros(nev)
        nconv = ctypes.c_int()
        stats = Stats()
        dp = ctypes.POINTER(ctypes.c_double)
        st = self._check(self._L.stab_eigs(self._h, complex(sigma).real, complex(sigma).imag, complex(tau).real,
                                           complex(tau).imag, nev, ncv, tol, _ptr(v0), lam.ctypes.data_as(dp),
                                           _ptr(vecs), res.ctypes.data_as(dp), ctypes.byref(nconv),
                                           ctypes.byref(stats)), allow=(4,))
        return EigResult(lam.view(np.complex128), res, nconv.value, st, stats.as_dict())

    def autotune(self, force: bool = False) -> dict:
        """Tune the line-pass launch shape per axis; {axis: (C, L, kinds, ms)} (ms -1: from the cache)."""
        cfg = (ctypes.c_int * 9)()
        ms = (ctypes.c_double * 3)()
        self._check(self._L.stab_autotune(self._h, int(bool(force)), cfg, ms))
        return {ax: (cfg[3 * a], cfg[3 * a + 1], cfg[3 * a + 2], ms[a]) for a, ax in enumerate("xyz") if cfg[3 * a] > 0}

    def set_line_config(self, axis: int, C: int, L: int, kinds: int):
        """Pin the line-pass shape of an axis (0 x, 1 y, 2 z); (0, 0, 0) restores the default."""
        self._check(self._L.stab_set_line_config(self._h, axis, C, L, kinds))

    def timing(self, enable: bool = True):
        """Start (discarding earlier records) or stop per-phase event timing."""
        self._check(self._L.stab_timing(self._h, int(bool(enable))))

    def timing_read(self) -> dict:
        """{phase: (summed ms, intervals)} since the last read, plus 'dropped'."""
        ms = (ctypes.c_double * len(PHASES))()
        cnt = (ctypes.c_longlong * len(PHASES))()
        dropped = ctypes.c_longlong()
        self._check(self._L.stab_timing_read(self._h, ms, cnt, ctypes.byref(dropped)))
        out = {p: (ms[i], cnt[i]) for i, p in enumerate(PHASES)}
        out["dropped"] = dropped.value
        return out

    def stats(self) -> dict:
        s = Stats()
        self._check(self._L.stab_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()


def autotune_save(path: str) -> int:
    """Write the process-wide line-pass tuning cache; returns the entry count."""
    return load().stab_autotune_save(path.encode())


def autotune_load(path: str) -> int:
    """Read a tuning cache written by autotune_save; returns the entry count (-1: unreadable)."""
    return load().stab_autotune_load(path.encode())


def _grid(grid) -> Grid:
    return Grid(grid.dim, grid.nx, grid.ny, grid.nz, grid.lx, grid.ly0, grid.ly1, grid.lz, grid.stretch)


def estimate_bytes(grid, nev: int, ncv: int, yonly: bool = True, **opts) -> int:
    """Device memory estimate of one full solve (stab_estimate_bytes)."""
    g = _grid(grid)
    o = default_opts(**opts)
    return int(load().stab_estimate_bytes(ctypes.byref(g), ctypes.byref(o), int(yonly), nev, ncv))


def eigs_batch(handles, args, concurrency: int = 0):
    """stab_eigs_batch: args[i] = (sigma, tau, nev, ncv, tol) for handles[i]; returns [EigResult]."""
    L = load()
    count = len(handles)
    hs = (ctypes.c_void_p * count)(*[h._h.value for h in handles])
    jobs = (EigJob * count)()
    keep = []
    for i, (sigma, tau, nev, ncv, tol) in enumerate(args):
        lam = np.zeros(2 * nev)
        res = np.zeros(nev)
        keep.append((lam, res))
        J = jobs[i]
        J.sigma_re, J.sigma_im = complex(sigma).real, complex(sigma).imag
        J.tau_re, J.tau_im = complex(tau).real, complex(tau).imag
        J.nev, J.ncv, J.tol = nev, ncv, tol
        J.lambda_ = lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        J.resid = res.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = L.stab_eigs_batch(hs, jobs, count, concurrency)
    out = [EigResult(lam.view(np.complex128), res, jobs[i].nconv, jobs[i].status, jobs[i].stats.as_dict())
           for i, (lam, res) in enumerate(keep)]
    if st not in (0, 4):
        raise StabError(st, "stab_eigs_batch: " + "; ".join(
            L.stab_last_error(h._h).decode() for h, r in zip(handles, out) if r.status not in (0, 4)))
    return out


class JvBatch:
    """stab_jv_batch_*: J v and block-Jacobi apply of several problems (uneven grids), one launch per phase."""

    def __init__(self, handles, stream=None):
        import torch
        self._L = load()
        self.handles = list(handles)  # keeps the problems alive while the batch exists
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        count = len(self.handles)
        hs = (ctypes.c_void_p * count)(*[h._h.value for h in self.handles])
        b = ctypes.c_void_p()
        st = self._L.stab_jv_batch_create(ctypes.byref(b), hs, count, self.stream.cuda_stream)
        if st != 0:
            raise StabError(st, "stab_jv_batch_create: handles must be distinct, on this device, with y-only base flows")
        self._b = b

    def _check_open(self):
        if getattr(self, "_b", None) is None or any(getattr(h, "_h", None) is None for h in self.handles):
            raise StabError(1, "JvBatch: the batch or one of its handles is closed")

    def apply(self, vs, outs, shifts=None):
        """outs[i] = J_i vs[i] - shifts[i] vs[i] (complex128 device tensors)."""
        self._check_open()
        count = len(self.handles)
        if len(vs) != count or len(outs) != count:
            raise ValueError("one input and one output vector per handle")
        ns = [h.n for h in self.handles]
        v = (ctypes.c_void_p * count)(*[_vec_ptr(x, n, f"JvBatch.apply v[{i}]") for i, (x, n) in enumerate(zip(vs, ns))])
        o = (ctypes.c_void_p * count)(*[_vec_ptr(x, n, f"JvBatch.apply out[{i}]")
                                        for i, (x, n) in enumerate(zip(outs, ns))])
        sh = None
        if shifts is not None:
            arr = np.zeros(2 * count)
            for i, z in enumerate(shifts):
                arr[2 * i], arr[2 * i + 1] = complex(z).real, complex(z).imag
            sh = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        st = self._L.stab_jv_batch_apply(self._b, v, o, sh)
        if st != 0:
            raise StabError(st, self._L.stab_jv_batch_last_error(self._b).decode())
        return outs

    def precond_apply(self, qs, zs):
        """zs[i] = M_i^-1 qs[i] with each handle's block-Jacobi inverses (built by precond_build)."""
        self._check_open()
        count = len(self.handles)
        if len(qs) != count or len(zs) != count:
            raise ValueError("one input and one output vector per handle")
        ns = [h.n for h in self.handles]
        q = (ctypes.c_void_p * count)(*[_vec_ptr(x, n, f"JvBatch.precond_apply q[{i}]")
                                        for i, (x, n) in enumerate(zip(qs, ns))])
        z = (ctypes.c_void_p * count)(*[_vec_ptr(x, n, f"JvBatch.precond_apply z[{i}]")
                                        for i, (x, n) in enumerate(zip(zs, ns))])
        st = self._L.stab_jv_batch_precond_apply(self._b, q, z)
        if st != 0:
            raise StabError(st, self._L.stab_jv_batch_last_error(self._b).decode())
        return zs

    def orthogonalize(self, Vs, ks, ws):
        """CGS2 of ws[i] (updated in place) against the ks[i] columns of Vs[i]; returns
        ([h_i complex coefficients], [||w_i|| after])."""
        self._check_open()
        count = len(self.handles)
        if len(Vs) != count or len(ks) != count or len(ws) != count:
            raise ValueError("one basis, column count and vector per handle")
        ns = [h.n for h in self.handles]
        V = (ctypes.c_void_p * count)(*[_vec_ptr(x, int(k) * n, f"JvBatch.orthogonalize V[{i}]")
                                        for i, (x, k, n) in enumerate(zip(Vs, ks, ns))])
        K = (ctypes.c_int * count)(*[int(x) for x in ks])
        W = (ctypes.c_void_p * count)(*[_vec_ptr(x, n, f"JvBatch.orthogonalize w[{i}]")
                                        for i, (x, n) in enumerate(zip(ws, ns))])
        hc = np.zeros(2 * sum(int(x) for x in ks))
        nr = np.zeros(count)
        st = self._L.stab_jv_batch_orthogonalize(self._b, V, K, W, hc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                 nr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if st != 0:
            raise StabError(st, self._L.stab_jv_batch_last_error(self._b).decode())
        hz = hc.view(np.complex128)
        out, off = [], 0
        for x in ks:
            out.append(hz[off:off + int(x)].copy())
            off += int(x)
        return out, list(nr)

    def solve(self, sigmas, rhs, xs):
        """Lockstep GMRES: xs[i] = (J_i - sigmas[i] I)^-1 rhs[i]; returns (status, [iterations])."""
        self._check_open()
        count = len(self.handles)
        if len(sigmas) != count or len(rhs) != count or len(xs) != count:
            raise ValueError("one shift, right-hand side and solution vector per handle")
        ns = [h.n for h in self.handles]
        sg = np.zeros(2 * count)
        for i, z in enumerate(sigmas):
            sg[2 * i], sg[2 * i + 1] = complex(z).real, complex(z).imag
        b = (ctypes.c_void_p * count)(*[_vec_ptr(x, n, f"JvBatch.solve rhs[{i}]") for i, (x, n) in enumerate(zip(rhs, ns))])
        x = (ctypes.c_void_p * count)(*[_vec_ptr(v, n, f"JvBatch.solve x[{i}]") for i, (v, n) in enumerate(zip(xs, ns))])
        it = (ctypes.c_int * count)()
        st = self._L.stab_jv_batch_solve(self._b, sg.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), b, x, it)
        if st not in (0, 4):
            raise StabError(st, self._L.stab_jv_batch_last_error(self._b).decode())
        return st, list(it)

    def eigs(self, args, vecs=None):
        """Lockstep Cayley-IRAM: args[i] = (sigma, tau, nev, ncv, tol[, v0]) for handle i; vecs: None or a
        list of device tensors (nev x n) or None per instance.  Returns [EigResult]."""
        self._check_open()
        count = len(self.handles)
        if len(args) != count:
            raise ValueError("one job per handle")
        jobs = (EigJob * count)()
        keep = []
        for i, a in enumerate(args):
            sigma, tau, nev, ncv, tol = a[:5]
            v0 = a[5] if len(a) > 5 else None
            lam = np.zeros(2 * nev)
            res = np.zeros(nev)
            keep.append((lam, res))
            J = jobs[i]
            J.sigma_re, J.sigma_im = complex(sigma).real, complex(sigma).imag
            J.tau_re, J.tau_im = complex(tau).real, complex(tau).imag
            J.nev, J.ncv, J.tol = nev, ncv, tol
            J.v0 = None if v0 is None else _vec_ptr(v0, self.handles[i].n, f"JvBatch.eigs v0[{i}]")
            J.lambda_ = lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            J.resid = res.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            if vecs is not None and vecs[i] is not None:
                J.vecs = _vec_ptr(vecs[i], nev * self.handles[i].n, f"JvBatch.eigs vecs[{i}]")
        st = self._L.stab_jv_batch_eigs(self._b, jobs)
        out = [EigResult(lam.view(np.complex128), res, jobs[i].nconv, jobs[i].status, jobs[i].stats.as_dict())
               for i, (lam, res) in enumerate(keep)]
        if st not in (0, 4):
            raise StabError(st, self._L.stab_jv_batch_last_error(self._b).decode())
        return out

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            self._L.stab_jv_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching stability server (stab_server_*) on the current CUDA device."""

    def __init__(self, slots: int, mem_budget_bytes: int, autotune: bool = False, cohort: int = 1):
        self._L = load()
        self._s = ctypes.c_void_p()
        st = self._L.stab_server_create(ctypes.byref(self._s), slots, int(mem_budget_bytes), int(autotune))
        if st != 0:
            raise StabError(st, "stab_server_create failed")
        self._nev = {}
        if cohort != 1:
            st = self._L.stab_server_set_cohort(self._s, int(cohort))
            if st != 0:
                raise StabError(st, "stab_server_set_cohort: cohort must be in [1, 4096]")

    def submit(self, base_flow, grid, Ma: float, Re: float, Pr: float, sigma: complex, tau: complex, nev: int,
               ncv: int, tol: float, vectors: bool = False, **opts) -> int:
        """Queue a request; with vectors=True result() also returns the eigenvectors (nev x n)."""
        bf = np.ascontiguousarray(np.asarray(base_flow, dtype=np.float64).reshape(-1))
        o = default_opts(**opts)
        q = Request()
        q.base_flow = bf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        q.grid = _grid(grid)
        q.Ma, q.Re, q.Pr = Ma, Re, Pr
        q.opts = ctypes.pointer(o)
        q.sigma_re, q.sigma_im = complex(sigma).real, complex(sigma).imag
        q.tau_re, q.tau_im = complex(tau).real, complex(tau).imag
        q.nev, q.ncv, q.tol = nev, ncv, tol
        vecs = None
        if vectors:
            n = (grid.dim + 2) * grid.nx * grid.ny * grid.nz
            vecs = np.zeros((nev, n), dtype=np.complex128)
            q.vecs = vecs.ctypes.data
        rid = ctypes.c_longlong()
        st = self._L.stab_server_submit(self._s, ctypes.byref(q), ctypes.byref(rid))
        if st != 0:
            raise StabError(st, "stab_server_submit failed")
        self._nev[rid.value] = (nev, vecs)
        return rid.value

    def wait(self, rid: int, timeout_s: float = -1.0) -> bool:
        st = self._L.stab_server_wait(self._s, rid, timeout_s)
        if st not in (0, 7):
            raise StabError(st, "stab_server_wait: unknown request")
        return st == 0

    def result(self, rid: int):
        """(eigenvalues, residuals, info dict) of a finished request (forgotten afterwards); info["vecs"]
        holds the eigenvectors when the request asked for them."""
        nev, vecs = self._nev.pop(rid)
        lam = np.zeros(2 * nev)
        res = np.zeros(nev)
        info = RequestInfo()
        dp = ctypes.POINTER(ctypes.c_double)
        st = self._L.stab_server_result(self._s, rid, lam.ctypes.data_as(dp), res.ctypes.data_as(dp),
                                        ctypes.byref(info))
        if st != 0:
            self._nev[rid] = (nev, vecs)
            raise StabError(st, "stab_server_result: not finished or unknown")
        d = {k: getattr(info, k) for k, _ in info._fields_ if k != "stats"}
        d["stats"] = info.stats.as_dict()
        if vecs is not None:
            d["vecs"] = vecs
        return lam.view(np.complex128), res, d

    def stats(self) -> dict:
        pb, pr, q, r = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._L.stab_server_stats(self._s, ctypes.byref(pb), ctypes.byref(pr), ctypes.byref(q), ctypes.byref(r))
        return {"peak_bytes": pb.value, "peak_running": pr.value, "queued": q.value, "running": r.value}

    def close(self):
        if getattr(self, "_s", None):
            self._L.stab_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
