"""ctypes binding of the C ABI in include/hz.h (argument marshalling only).

Every computation runs in the CUDA library libhz.so; importing this module
loads it and raises ImportError when it has not been built (call
``paper_2409_16172_gb300.build.build()``).  Device buffers are torch tensors
(complex128, contiguous, on the current CUDA device); streams are torch
streams.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhz.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "hz.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                      "(run paper_2409_16172_gb300.build.build())")
lib = C.CDLL(LIB_PATH)

HZ_OK = 0
STATUS = {0: "HZ_OK", 1: "HZ_ERR_INVALID_ARG", 2: "HZ_ERR_OOM", 3: "HZ_ERR_CUDA",
          4: "HZ_ERR_NOT_CONVERGED", 5: "HZ_ERR_BREAKDOWN", 6: "HZ_ERR_TIMEOUT",
          7: "HZ_ERR_BUSY", 8: "HZ_ERR_MEDIUM"}


class HzError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class hz_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("L", C.c_double)]


class hz_interp(C.Structure):
    _fields_ = [("M", C.c_int), ("Mt", C.c_int), ("c_o", C.c_double), ("zeta_max", C.c_double),
                ("alpha", C.c_double), ("a_node", C.c_double), ("symbol_kind", C.c_int),
                ("Ma", C.c_int), ("basis", C.c_int)]


class hz_solver_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("restart", C.c_int), ("tol", C.c_double),
                ("maxit", C.c_int), ("graphs", C.c_int), ("no_precond", C.c_int),
                ("left", C.c_int)]


class hz_solve_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("status", C.c_int),
                ("converged", C.c_int), ("rel_true_resid", C.c_double),
                ("rel_est_resid", C.c_double), ("ms_total", C.c_float),
                ("ms_precond", C.c_float), ("ms_stencil", C.c_float), ("ms_arnoldi", C.c_float),
                ("model_bytes_precond", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_vp = C.c_void_p
_dp = C.POINTER(C.c_double)


class hz_tune_report(C.Structure):
    _fields_ = [("dots_bps", C.c_int), ("dots_vc", C.c_int), ("upd_bps", C.c_int),
                ("syminv_kpb", C.c_int), ("cached", C.c_int), ("dots_us", C.c_float),
                ("dots_us_default", C.c_float), ("upd_us", C.c_float),
                ("upd_us_default", C.c_float), ("apply_us", C.c_float),
                ("apply_us_default", C.c_float), ("rowinv_mode", C.c_int),
                ("col_pair", C.c_int)]


class hz_server_opts(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_slots", C.c_int), ("max_queue", C.c_int),
                ("device", C.c_int), ("autotune", C.c_int), ("max_bypass", C.c_int),
                ("batch_slots", C.c_int), ("order", C.c_int)]


class hz_request(C.Structure):
    _fields_ = [("grid", hz_grid), ("c", _dp), ("zeta", _dp), ("a", _dp), ("omega", C.c_double),
                ("interp", hz_interp), ("opts", hz_solver_opts), ("nrhs", C.c_int), ("f", _vp)]


class hz_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong), ("failed", C.c_longlong),
                ("rejected", C.c_longlong), ("active", C.c_int), ("queued", C.c_int),
                ("max_active", C.c_int), ("hbm_in_use", C.c_size_t), ("hbm_budget", C.c_size_t),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("rhs_per_s", C.c_double), ("batch_joins", C.c_longlong)]
_SIGS = {
    "hz_last_error": (C.c_char_p, []),
    "hz_version": (C.c_char_p, []),
    "hz_set_allocator": (C.c_int, [_vp, _vp, _vp]),
    "hz_create_medium": (C.c_int, [C.POINTER(hz_grid), _dp, _dp, _dp, C.c_double,
                                   C.POINTER(hz_interp), C.POINTER(_vp)]),
    "hz_medium_info": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                 _dp, _dp, _dp, _dp, _dp]),
    "hz_destroy_medium": (C.c_int, [_vp]),
    "hz_plan_create": (C.c_int, [_vp, C.POINTER(hz_solver_opts), C.c_int, C.POINTER(_vp)]),
    "hz_plan_bytes": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "hz_destroy_plan": (C.c_int, [_vp]),
    "hz_apply_operator": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _vp]),
    "hz_apply_preconditioner": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _vp]),
    "hz_gmres_solve": (C.c_int, [_vp, _vp, _vp, C.c_int, C.POINTER(hz_solve_stats), _vp]),
    "hz_gmres_solve_history": (C.c_int, [_vp, _vp, _vp, C.c_int, C.POINTER(hz_solve_stats),
                                         C.POINTER(C.c_double), C.c_int, _vp]),
    "hz_apply_preconditioner_noalloc": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _vp]),
    "hz_request_footprint": (C.c_size_t, [C.POINTER(hz_grid), C.POINTER(hz_interp),
                                          C.POINTER(hz_solver_opts), C.c_int, C.c_int]),
    "hz_server_create": (C.c_int, [C.POINTER(hz_server_opts), C.POINTER(_vp)]),
    "hz_submit": (C.c_int, [_vp, C.POINTER(hz_request), C.POINTER(C.c_uint64)]),
    "hz_poll": (C.c_int, [_vp, C.c_uint64, C.POINTER(C.c_int), _vp, _vp]),
    "hz_server_wait": (C.c_int, [_vp, C.c_uint64, C.c_double]),
    "hz_server_get_stats": (C.c_int, [_vp, C.POINTER(hz_server_stats)]),
    "hz_server_destroy": (C.c_int, [_vp]),
    "hz_plan_autotune": (C.c_int, [_vp, _vp, C.POINTER(hz_tune_report)]),
    "hz_plan_set_tune": (C.c_int, [_vp, C.POINTER(hz_tune_report)]),
    "hz_plan_hessenberg": (C.c_int, [_vp, C.c_int, _vp, C.POINTER(C.c_int)]),
    "hz_profile_enable": (C.c_int, [C.c_int]),
    "hz_profile_read": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int), C.c_int]),
    "hz_launch_count": (C.c_ulonglong, []),
    "hz_measure_fp64_peak": (C.c_int, [_dp]),
}
for _name, (_res, _args) in _SIGS.items():
    if hasattr(lib, _name):
        _f = getattr(lib, _name)
        _f.restype = _res
        _f.argtypes = _args


def header_symbols(path: str = HEADER) -> list[str]:
    """Every function name declared in include/hz.h."""
    with open(path) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:[a-z_]+\s+)*[a-z_]+\s*\**\s*(hz_[a-z0-9_]+)\s*\(",
                                 text, re.M)))


class hz_phase_stats(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_longlong), ("ms", C.c_double),
                ("bytes", C.c_double), ("flops", C.c_double)]


def profile_enable(on: bool = True):
    check(lib.hz_profile_enable(1 if on else 0))


def profile_read(reset: bool = False) -> dict:
    """{phase: dict(launches, ms, bytes, flops)} accumulated since the last reset."""
    buf = (hz_phase_stats * 32)()
    cnt = C.c_int()
    check(lib.hz_profile_read(C.cast(buf, _vp), 32, C.byref(cnt), 1 if reset else 0))
    return {buf[i].name.decode(): dict(launches=buf[i].launches, ms=buf[i].ms, bytes=buf[i].bytes,
                                       flops=buf[i].flops) for i in range(cnt.value)}


def launch_count() -> int:
    return int(lib.hz_launch_count())


def measure_fp64_peak() -> float:
    """GFLOP/s of FP64 FMA on the current device."""
    g = C.c_double()
    check(lib.hz_measure_fp64_peak(C.byref(g)))
    return g.value


def last_error() -> str:
    return lib.hz_last_error().decode()


def version() -> str:
    return lib.hz_version().decode()


def check(status: int, ok=(HZ_OK,)):
    if status not in ok:
        raise HzError(status, last_error())
    return status


def _dptr(a):
    """double* of a C-contiguous float64 numpy array (or NULL)."""
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _check_dev(x, name):
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.complex128
            and x.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous complex128 CUDA tensor")


class Medium:
    """A medium on the GPU: node table, interpolation records, gamma^2."""

    def __init__(self, c, zeta=None, a=None, *, omega: float, M: int, Mt: int = 0,
                 c_o: float = 1.0, zeta_max: float = 0.0, alpha: float = 0.15,
                 a_node: float = 0.0, symbol_kind: int = 0, L: float = 1.0, Ma: int = 0,
                 basis: int = 0):
        c = np.ascontiguousarray(c, dtype=np.float64)
        self.shape = c.shape
        if c.ndim not in (2, 3):
            raise ValueError("c must be 2D or 3D")
        zeta = None if zeta is None else np.ascontiguousarray(zeta, dtype=np.float64)
        a = None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        for arr in (zeta, a):
            if arr is not None and arr.shape != c.shape:
                raise ValueError("zeta / a must have the shape of c")
        g = hz_grid()
        g.dim = c.ndim
        dims = list(reversed(c.shape)) + [1] * (3 - c.ndim)
        for i in range(3):
            g.n[i] = dims[i]
        g.L = L
        it = hz_interp(M, Mt, c_o, zeta_max, alpha, a_node, symbol_kind, Ma, basis)
        h = _vp()
        check(lib.hz_create_medium(C.byref(g), _dptr(c), _dptr(zeta), _dptr(a), float(omega),
                                   C.byref(it), C.byref(h)))
        self._h = h
        self.omega = float(omega)
        self.n = int(np.prod(c.shape))

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        K, M, Mt = C.c_int(), C.c_int(), C.c_int()
        cmin, cmax = C.c_double(), C.c_double()
        check(lib.hz_medium_info(self._h, C.byref(K), C.byref(M), C.byref(Mt), None, None, None,
                                 C.byref(cmin), C.byref(cmax)))
        gr = np.zeros(K.value)
        gi = np.zeros(K.value)
        ak = np.zeros(K.value)
        check(lib.hz_medium_info(self._h, None, None, None, _dptr(gr), _dptr(gi), _dptr(ak), None,
                                 None))
        return dict(K=K.value, M=M.value, Mt=Mt.value, gamma=gr + 1j * gi, a=ak,
                    c_min=cmin.value, c_max=cmax.value)

    def close(self):
        if getattr(self, "_h", None):
            lib.hz_destroy_medium(self._h)
            self._h = None

    __del__ = close


class Plan:
    """Workspace for applying and solving on one medium."""

    def __init__(self, medium: Medium, *, precision: int = 1, restart: int = 40,
                 tol: float = 1e-6, maxit: int = 4000, max_nrhs: int = 1, graphs: bool = False,
                 no_precond: bool = False, left: bool = False):
        self.medium = medium
        self.max_nrhs = max_nrhs
        self.opts = hz_solver_opts(precision, restart, tol, maxit, 1 if graphs else 0,
                                   1 if no_precond else 0, 1 if left else 0)
        h = _vp()
        check(lib.hz_plan_create(medium.handle, C.byref(self.opts), max_nrhs, C.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def autotune(self, stream=None) -> dict:
        """Time the candidate launch shapes on this plan (hz_plan_autotune)."""
        r = hz_tune_report()
        check(lib.hz_plan_autotune(self._h, _stream(stream), C.byref(r)))
        return {f: getattr(r, f) for f, _ in r._fields_}

    def set_tune(self, **shape) -> None:
        """Set launch shapes (hz_plan_set_tune); unspecified ones keep the
        defaults dots_vc=8, dots_bps=2, upd_bps=4, syminv_kpb=1, rowinv_mode=0,
        col_pair=1."""
        r = hz_tune_report()
        r.dots_vc, r.dots_bps, r.upd_bps, r.syminv_kpb, r.rowinv_mode = 8, 2, 4, 1, 0
        r.col_pair = 1
        for k, v in shape.items():
            setattr(r, k, int(v))
        check(lib.hz_plan_set_tune(self._h, C.byref(r)))

    def hessenberg(self, rhs: int = 0) -> np.ndarray:
        """Unrotated Hessenberg matrix (J + 1, J) of the last Arnoldi cycle of
        right-hand side rhs (hz_plan_hessenberg); its square part's
        eigenvalues are Ritz values of the preconditioned operator."""
        m = self.opts.restart
        buf = np.zeros((m, m + 1), np.complex128)  # column j at buf[j]
        cols = C.c_int()
        check(lib.hz_plan_hessenberg(self._h, rhs, _vp(buf.ctypes.data), C.byref(cols)))
        J = cols.value
        return np.ascontiguousarray(buf[:J, :J + 1].T)

    def nbytes(self) -> int:
        b = C.c_size_t()
        check(lib.hz_plan_bytes(self._h, C.byref(b)))
        return b.value

    def apply_operator(self, x, out=None, stream=None):
        """y = P_N x in FP64 (hz_apply_operator).  x: complex128 CUDA tensor
        (precision 0) or complex64 (precision 1, widened exactly); the result
        is complex128."""
        import torch
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.is_contiguous()
                and x.dtype in (torch.complex128, torch.complex64)):
            raise TypeError("x must be a contiguous complex128 or complex64 CUDA tensor")
        prec = 0 if x.dtype == torch.complex128 else 1
        nrhs = x.numel() // self.medium.n
        out = torch.empty(x.shape, dtype=torch.complex128, device=x.device) if out is None else out
        _check_dev(out, "out")
        check(lib.hz_apply_operator(self._h, _vp(x.data_ptr()), _vp(out.data_ptr()), nrhs, prec,
                                    _stream(stream)))
        return out

    def apply_preconditioner(self, x, precision: int = 1, out=None, stream=None):
        import torch
        _check_dev(x, "x")
        nrhs = x.numel() // self.medium.n
        out = torch.empty_like(x) if out is None else out
        _check_dev(out, "out")
        check(lib.hz_apply_preconditioner(self._h, _vp(x.data_ptr()), _vp(out.data_ptr()), nrhs,
                                          precision, _stream(stream)))
        return out

    def solve(self, f, u=None, stream=None, raise_on_fail: bool = False, history: int = 0):
        """Solve P u = f.  f, u: complex128 CUDA tensors or numpy arrays
        (host buffers are staged by the library).  Returns (u, [stats]), or
        with history > 0 (u, [stats], H): H[b, s] is the estimated relative
        residual after Arnoldi step s (hz_gmres_solve_history), NaN past the
        last step."""
        import torch
        if isinstance(f, torch.Tensor):
            _check_dev(f, "f")
            nrhs = f.numel() // self.medium.n
            u = torch.zeros_like(f) if u is None else u
            _check_dev(u, "u")
            fp, up = _vp(f.data_ptr()), _vp(u.data_ptr())
        else:
            f = np.ascontiguousarray(f, dtype=np.complex128)
            nrhs = f.size // self.medium.n
            u = np.zeros_like(f) if u is None else u
            if not (isinstance(u, np.ndarray) and u.dtype == np.complex128 and u.flags.c_contiguous):
                raise TypeError("u must be a contiguous complex128 numpy array")
            fp, up = _vp(f.ctypes.data), _vp(u.ctypes.data)
        stats = (hz_solve_stats * nrhs)()
        if history > 0:
            H = np.empty((nrhs, int(history)), np.float64)
            st = lib.hz_gmres_solve_history(self._h, fp, up, nrhs, stats,
                                            H.ctypes.data_as(C.POINTER(C.c_double)),
                                            int(history), _stream(stream))
        else:
            st = lib.hz_gmres_solve(self._h, fp, up, nrhs, stats, _stream(stream))
        ok = (HZ_OK,) if raise_on_fail else (HZ_OK, 4, 5)
        check(st, ok)
        if history > 0:
            return u, [s.as_dict() for s in stats], H
        return u, [s.as_dict() for s in stats]

    def close(self):
        if getattr(self, "_h", None):
            lib.hz_destroy_plan(self._h)
            self._h = None

    __del__ = close


def _grid_of(shape, L=1.0):
    g = hz_grid()
    g.dim = len(shape)
    dims = list(reversed(shape)) + [1] * (3 - len(shape))
    for i in range(3):
        g.n[i] = dims[i]
    g.L = L
    return g


def request_footprint(shape, M, Mt, precision=1, restart=40, nrhs=1, has_a=False, Ma=0,
                      basis=0) -> int:
    g = _grid_of(tuple(shape))
    it = hz_interp(M, Mt, 1.0, 0.0, 0.15, 0.0, 0, Ma, basis)
    o = hz_solver_opts(precision, restart, 1e-6, 4000, 0, 0, 0)
    return int(lib.hz_request_footprint(C.byref(g), C.byref(it), C.byref(o), nrhs, 1 if has_a else 0))


class Server:
    """Continuous-batching solve server (hz_server_* in the C ABI)."""

    def __init__(self, max_slots: int = 4, max_queue: int = 4096, hbm_budget: int = 0,
                 device: int = 0, autotune: int = 0, max_bypass: int = 0,
                 batch_slots: int = 0, order: int = 0):
        o = hz_server_opts(hbm_budget, max_slots, max_queue, device, autotune, max_bypass,
                           batch_slots, order)
        h = _vp()
        check(lib.hz_server_create(C.byref(o), C.byref(h)))
        self._h = h
        self._shapes = {}

    def submit(self, c, f, *, omega: float, M: int, Mt: int = 0, zeta=None, a=None,
               c_o: float = 1.0, zeta_max: float = 0.0, alpha: float = 0.15, a_node: float = 0.0,
               symbol_kind: int = 0, precision: int = 1, restart: int = 40, tol: float = 1e-6,
               maxit: int = 4000, L: float = 1.0, graphs: bool = False, Ma: int = 0,
               basis: int = 0) -> int:
        c = np.ascontiguousarray(c, dtype=np.float64)
        shape = c.shape
        f = np.ascontiguousarray(f, dtype=np.complex128)
        nrhs = f.size // c.size
        zeta = None if zeta is None else np.ascontiguousarray(zeta, dtype=np.float64)
        a = None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        r = hz_request()
        r.grid = _grid_of(shape, L)
        r.c = _dptr(c)
        r.zeta = _dptr(zeta)
        r.a = _dptr(a)
        r.omega = omega
        r.interp = hz_interp(M, Mt, c_o, zeta_max, alpha, a_node, symbol_kind, Ma, basis)
        r.opts = hz_solver_opts(precision, restart, tol, maxit, 1 if graphs else 0, 0, 0)
        r.nrhs = nrhs
        r.f = _vp(f.ctypes.data)
        t = C.c_uint64()
        check(lib.hz_submit(self._h, C.byref(r), C.byref(t)))
        self._shapes[t.value] = (nrhs,) + tuple(shape)
        return t.value

    def poll(self, ticket: int):
        """(done, u, stats, status); u and stats are None until done."""
        shape = self._shapes[ticket]
        done = C.c_int()
        u = np.empty(shape, np.complex128)
        stats = (hz_solve_stats * shape[0])()
        st = lib.hz_poll(self._h, ticket, C.byref(done), _vp(u.ctypes.data), C.cast(stats, _vp))
        if not done.value:
            check(st)
            return False, None, None, st
        del self._shapes[ticket]
        return True, u, [s.as_dict() for s in stats], st

    def wait(self, ticket: int, timeout: float = 600.0):
        check(lib.hz_server_wait(self._h, ticket, timeout))

    def result(self, ticket: int, timeout: float = 600.0):
        self.wait(ticket, timeout)
        return self.poll(ticket)

    def stats(self) -> dict:
        s = hz_server_stats()
        check(lib.hz_server_get_stats(self._h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib.hz_server_destroy(self._h)
            self._h = None

    __del__ = close
