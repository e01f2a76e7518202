"""Python binding of libsrmc (include/srmc.h): argument marshalling only.

Every function keeps the C name; every compute step runs in the library's
CUDA kernels.  Device buffers are torch tensors (device memory and streams
only); host buffers are numpy arrays.  There is no CPU fallback: if the
shared library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SRMC_LIBRARY overrides the path (e.g. to compare two builds of the library).
LIB_PATH = os.environ.get("SRMC_LIBRARY") or os.path.join(_HERE, "_build", "libsrmc.so")

SRMC_OK = 0
STATUS = {0: "SRMC_OK", 1: "SRMC_ERR_INVALID_ARG", 2: "SRMC_ERR_CUDA", 3: "SRMC_ERR_OOM",
          4: "SRMC_ERR_UNSUPPORTED", 5: "SRMC_ERR_STATE"}
MODELS = {"cos": 0, "logistic": 1, "affine": 2, "user": 3}
BASES = {"lp0": 0, "lp1": 1, "lp2": 2}
PRECISIONS = {"fp32": 0, "fp64": 1}
STRATA = {"size": 0, "prob": 1}
DYNAMICS = {"euler": 0, "exact": 1}


class SrmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class srmc_problem(C.Structure):
    _fields_ = [("d", C.c_int), ("q", C.c_int), ("N", C.c_int), ("T", C.c_double),
                ("b", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double)),
                ("model", C.c_int), ("params", C.POINTER(C.c_double)), ("n_params", C.c_int),
                ("theta", C.POINTER(C.c_double)), ("dynamics", C.c_int),
                ("user_source", C.c_char_p), ("user_dynamics", C.c_int)]


class srmc_strata(C.Structure):
    _fields_ = [("cells", C.POINTER(C.c_int)), ("lo", C.POINTER(C.c_double)),
                ("hi", C.POINTER(C.c_double)), ("mu", C.c_double), ("kind", C.c_int)]


class srmc_config(C.Structure):
    _fields_ = [("basis", C.c_int), ("prec", C.c_int), ("M", C.c_longlong),
                ("seed", C.c_ulonglong), ("instance", C.c_uint), ("Cy", C.c_double),
                ("Cz", C.c_double), ("block_threads", C.c_int),
                ("M_strata", C.POINTER(C.c_longlong))]


_lock = threading.Lock()
_lib = None


def lib():
    """Load the in-tree libsrmc.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libsrmc is not built ({LIB_PATH} missing); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            vp, ll, i_ = C.c_void_p, C.c_longlong, C.c_int
            L.srmc_create.argtypes = [C.POINTER(srmc_problem), C.POINTER(srmc_strata),
                                      C.POINTER(srmc_config), C.POINTER(vp)]
            L.srmc_destroy.argtypes = [vp]; L.srmc_destroy.restype = None
            L.srmc_solve.argtypes = [vp, vp]
            L.srmc_solve_step.argtypes = [vp, i_, vp]
            L.srmc_eval.argtypes = [vp, i_, vp, ll, vp, vp, vp]
            L.srmc_centres.argtypes = [vp, vp, vp]
            L.srmc_table.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(i_), C.POINTER(i_),
                                     C.POINTER(i_), C.POINTER(ll)]
            L.srmc_stats.argtypes = [vp, C.POINTER(C.c_ulonglong)]
            L.srmc_read_table.argtypes = [vp, vp, vp, vp]
            L.srmc_set_rows.argtypes = [vp, i_, vp, vp, vp]
            L.srmc_set_rows.restype = C.c_int
            L.srmc_closed_form_error.argtypes = [vp, vp, vp]
            L.srmc_closed_form_error_inner.argtypes = [vp, vp, vp]
            L.srmc_closed_form_error_inner.restype = C.c_int
            L.srmc_point_error.argtypes = [vp, vp, ll, vp, vp]
            L.srmc_point_error.restype = C.c_int
            L.srmc_set_control.argtypes = [vp, vp]
            L.srmc_clear_control.argtypes = [vp]
            L.srmc_set_own_control.argtypes = [vp]
            L.srmc_read_control.argtypes = [vp, vp]
            L.srmc_mlp_create.argtypes = [i_, i_, C.c_ulonglong, C.POINTER(vp)]
            L.srmc_mlp_destroy.argtypes = [vp]; L.srmc_mlp_destroy.restype = None
            L.srmc_mlp_nparams.argtypes = [vp]; L.srmc_mlp_nparams.restype = i_
            L.srmc_mlp_set_params.argtypes = [vp, vp]
            L.srmc_mlp_get_params.argtypes = [vp, vp]
            L.srmc_mlp_eval.argtypes = [vp, vp, ll, vp, vp, vp]
            L.srmc_mlp_loss_grad.argtypes = [vp, vp, vp, ll, vp, vp, vp]
            L.srmc_mlp_fit.argtypes = [vp, vp, ll, i_, i_, C.c_float, C.c_ulonglong, vp, vp]
            L.srmc_cv_tabulate.argtypes = [vp, vp, vp]
            L.srmc_mlp_fit_noalloc.argtypes = [vp, vp, ll, i_, i_, C.c_float, C.c_ulonglong, vp, vp]
            L.srmc_batch_create.argtypes = [C.POINTER(vp), i_, C.POINTER(vp)]
            L.srmc_batch_destroy.argtypes = [vp]; L.srmc_batch_destroy.restype = None
            L.srmc_batch_tune.argtypes = [vp, vp, C.POINTER(i_), i_, C.POINTER(i_)]
            L.srmc_batch_solve.argtypes = [vp, vp]
            L.srmc_batch_mode.argtypes = [vp]; L.srmc_batch_mode.restype = i_
            L.srmc_batch_set_mode.argtypes = [vp, i_]; L.srmc_batch_set_mode.restype = C.c_int
            L.srmc_batch_stats.argtypes = [vp, C.POINTER(C.c_ulonglong)]; L.srmc_batch_stats.restype = C.c_int
            L.srmc_batch_strategy_ms.argtypes = [vp, C.POINTER(C.c_float)]
            L.srmc_batch_strategy_ms.restype = C.c_int
            for name in ("srmc_batch_create", "srmc_batch_tune", "srmc_batch_solve"):
                getattr(L, name).restype = C.c_int
            for name in ("srmc_read_control", "srmc_mlp_create", "srmc_mlp_set_params",
                         "srmc_mlp_get_params", "srmc_mlp_eval", "srmc_mlp_loss_grad", "srmc_mlp_fit",
                         "srmc_cv_tabulate", "srmc_mlp_fit_noalloc"):
                getattr(L, name).restype = C.c_int
            L.srmc_philox.argtypes = [vp, C.POINTER(C.c_uint32), ll, vp, vp]
            L.srmc_normals.argtypes = [vp, ll, vp, vp, vp]
            L.srmc_locate.argtypes = [vp, vp, vp, ll, vp, vp]
            L.srmc_start_points.argtypes = [vp, i_, ll, ll, ll, vp, vp]
            L.srmc_fp32_fma_probe.argtypes = [i_, i_, i_, i_, vp, vp]
            L.srmc_fp32_fma_probe.restype = C.c_int
            L.srmc_last_error.restype = C.c_char_p
            L.srmc_version.restype = C.c_int
            for name in ("srmc_create", "srmc_solve", "srmc_solve_step", "srmc_eval", "srmc_centres",
                         "srmc_table", "srmc_read_table", "srmc_closed_form_error", "srmc_stats", "srmc_philox",
                         "srmc_normals", "srmc_locate", "srmc_set_control", "srmc_clear_control",
                         "srmc_set_own_control", "srmc_start_points"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(status):
    if status != SRMC_OK:
        raise SrmcError(status, lib().srmc_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _darr(vals):
    a = (C.c_double * max(1, len(vals)))(*[float(v) for v in vals])
    return a


def exported_symbols():
    """Names declared in include/srmc.h that the loaded library exports."""
    L = lib()
    return [n for n in ("srmc_create", "srmc_destroy", "srmc_solve", "srmc_solve_step", "srmc_eval",
                        "srmc_centres", "srmc_table", "srmc_read_table", "srmc_closed_form_error",
                        "srmc_stats", "srmc_philox",
                        "srmc_normals",
                        "srmc_locate", "srmc_start_points", "srmc_fp32_fma_probe", "srmc_last_error",
                        "srmc_version")
            if hasattr(L, n)]


class Solver:
    """One SRMC problem on the current CUDA device (wraps srmc_create)."""

    def __init__(self, w, block_threads: int = 0):
        L = lib()
        self.w = w
        d, q = w.d, w.q
        self._b = _darr(w.b)
        self._sig = _darr([w.sigma[l][r] for l in range(d) for r in range(q)])
        self._prm = _darr(w.params)
        self._cells = (C.c_int * d)(*[int(c) for c in w.cells])
        self._lo = _darr(w.lo)
        self._hi = _darr(w.hi)
        th = getattr(w, "theta", None)
        self._theta = _darr(th) if th else None
        pr = srmc_problem(d, q, int(w.N), float(w.T), self._b, self._sig, MODELS[w.model],
                          self._prm, len(w.params), self._theta,
                          DYNAMICS.get(getattr(w, "dynamics", "euler"), -1),
                          (getattr(w, "user_source", None) or "").encode() or None,
                          1 if getattr(w, "user_dynamics", False) else 0)
        sa = srmc_strata(self._cells, self._lo, self._hi, float(w.mu),
                         STRATA.get(getattr(w, "strata", "size"), -1))
        ms = getattr(w, "M_strata", None)
        self._ms = None if ms is None else (C.c_longlong * len(ms))(*[int(v) for v in ms])
        cf = srmc_config(BASES[w.basis], PRECISIONS[w.precision], int(w.M), int(w.seed),
                         int(w.instance), float(w.Cy), float(w.Cz), int(block_threads),
                         self._ms)
        h = C.c_void_p()
        _check(L.srmc_create(C.byref(pr), C.byref(sa), C.byref(cf), C.byref(h)))
        self._h = h
        self.K = int(np.prod(w.cells))

    def close(self):
        if getattr(self, "_h", None):
            lib().srmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def srmc_solve(self, stream=None):
        _check(lib().srmc_solve(self._h, _stream(stream)))

    def srmc_solve_step(self, i, stream=None):
        _check(lib().srmc_solve_step(self._h, int(i), _stream(stream)))

    def srmc_eval(self, i, x, y, z=None, stream=None):
        _check(lib().srmc_eval(self._h, int(i), _ptr(x), x.shape[0], _ptr(y), _ptr(z), _stream(stream)))

    def srmc_centres(self, x, stream=None):
        _check(lib().srmc_centres(self._h, _ptr(x), _stream(stream)))

    def srmc_table(self):
        y, z = C.c_void_p(), C.c_void_p()
        p, ry, rz, K = C.c_int(), C.c_int(), C.c_int(), C.c_longlong()
        _check(lib().srmc_table(self._h, C.byref(y), C.byref(z), C.byref(p), C.byref(ry),
                                C.byref(rz), C.byref(K)))
        return dict(y64=y.value, z64=z.value, p=p.value, ry=ry.value, rz=rz.value, K=K.value)

    def srmc_read_table(self, dst_y, dst_z, stream=None):
        """Copy the FP64 tables into caller tensors (host, pinned or device)."""
        _check(lib().srmc_read_table(self._h, _ptr(dst_y), _ptr(dst_z), _stream(stream)))

    def srmc_set_rows(self, i, src_y, src_z, stream=None):
        """Install the rows of step i from tensors [K][ry], [K][rz] (float64,
        the layout of srmc_table; host or device)."""
        _check(lib().srmc_set_rows(self._h, int(i), _ptr(src_y), _ptr(src_z), _stream(stream)))

    def srmc_set_control(self, rows):
        """rows: numpy [N][K][q][p] float64 (host) or a CUDA float64 tensor."""
        if isinstance(rows, np.ndarray):
            self._ctl = np.ascontiguousarray(rows, dtype=np.float64)
            ptr = C.c_void_p(self._ctl.ctypes.data)
        else:
            ptr = _ptr(rows)
        _check(lib().srmc_set_control(self._h, ptr))

    def srmc_set_own_control(self):
        """Control from the solver's own fitted z of the later steps."""
        _check(lib().srmc_set_own_control(self._h))

    def srmc_clear_control(self):
        _check(lib().srmc_clear_control(self._h))

    def srmc_read_control(self):
        d = self.w.d
        p = {"lp0": 1, "lp1": d + 1, "lp2": 1 + d + d * (d + 1) // 2}[self.w.basis]
        out = np.zeros((self.w.N, self.K, self.w.q, p))
        _check(lib().srmc_read_control(self._h, C.c_void_p(out.ctypes.data)))
        return out

    def srmc_point_error(self, x, out, stream=None):
        """x: CUDA float64 [N][n][d]; out: CUDA float64 [N][2] (sums of squared
        y and z errors against the closed form per step)."""
        _check(lib().srmc_point_error(self._h, _ptr(x), int(x.shape[1]), _ptr(out), _stream(stream)))

    def srmc_closed_form_error(self, out, stream=None):
        _check(lib().srmc_closed_form_error(self._h, _ptr(out), _stream(stream)))

    def closed_form_error(self, inner=False):
        """[N][4] (max|dy|, mean dy^2, max|dz|, mean |dz|^2) at the centres (of
        the inner strata only if inner), as numpy."""
        import torch
        out = torch.empty((self.w.N, 4), dtype=torch.float64, device="cuda")
        if inner:
            _check(lib().srmc_closed_form_error_inner(self._h, _ptr(out), _stream(None)))
        else:
            self.srmc_closed_form_error(out)
        return out.cpu().numpy()

    def srmc_stats(self):
        out = (C.c_ulonglong * 3)()
        _check(lib().srmc_stats(self._h, out))
        return dict(fallbacks=int(out[0]), nonfinite=int(out[1]), path_steps=int(out[2]))

    def srmc_locate(self, x, k, stream=None):
        import torch
        x64 = x if x.dtype == torch.float64 else None
        x32 = x if x.dtype == torch.float32 else None
        _check(lib().srmc_locate(self._h, _ptr(x64), _ptr(x32), x.shape[0], _ptr(k), _stream(stream)))

    def srmc_start_points(self, i, k, m0, x, stream=None):
        _check(lib().srmc_start_points(self._h, int(i), int(k), int(m0), x.shape[0], _ptr(x),
                                       _stream(stream)))

    # Convenience on top of the C calls -------------------------------------
    def centres(self):
        import torch
        x = torch.empty((self.K, self.w.d), dtype=torch.float64, device="cuda")
        self.srmc_centres(x)
        return x

    def evaluate(self, i, x):
        import torch
        y = torch.empty(x.shape[0], dtype=torch.float64, device=x.device)
        z = torch.empty((x.shape[0], self.w.q), dtype=torch.float64, device=x.device)
        self.srmc_eval(i, x, y, z)
        return y, z


def srmc_philox(ctr, key, out, stream=None):
    k = (C.c_uint32 * 2)(int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF)
    _check(lib().srmc_philox(_ptr(ctr), k, ctr.shape[0], _ptr(out), _stream(stream)))


def srmc_normals(words, out64=None, out32=None, stream=None):
    _check(lib().srmc_normals(_ptr(words), words.shape[0], _ptr(out64), _ptr(out32), _stream(stream)))


def srmc_fp32_fma_probe(grid, threads, iters, packed, out, stream=None):
    """FP32 FMA throughput probe: grid * threads * iters * 32 FLOP."""
    _check(lib().srmc_fp32_fma_probe(int(grid), int(threads), int(iters), int(bool(packed)), _ptr(out),
                                     _stream(stream)))


def srmc_version() -> int:
    return int(lib().srmc_version())


def build(force: bool = False) -> str:
    from . import build as _b
    return _b.build(force=force)


class MLP:
    """The control-variate network u_theta(t, x) (wraps srmc_mlp_create)."""

    def __init__(self, n_in: int, hidden: int = 64, seed: int = 0):
        h = C.c_void_p()
        _check(lib().srmc_mlp_create(int(n_in), int(hidden), int(seed), C.byref(h)))
        self._h = h
        self.n_in = n_in
        self.P = int(lib().srmc_mlp_nparams(h))

    def close(self):
        if getattr(self, "_h", None):
            lib().srmc_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def srmc_mlp_set_params(self, params):
        a = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().srmc_mlp_set_params(self._h, C.c_void_p(a.ctypes.data)))

    def srmc_mlp_get_params(self):
        a = np.zeros(self.P, dtype=np.float32)
        _check(lib().srmc_mlp_get_params(self._h, C.c_void_p(a.ctypes.data)))
        return a

    def srmc_mlp_eval(self, a, u, grad=None, stream=None):
        _check(lib().srmc_mlp_eval(self._h, _ptr(a), a.shape[0], _ptr(u), _ptr(grad), _stream(stream)))

    def srmc_mlp_loss_grad(self, a, y, grad, loss=None, stream=None):
        _check(lib().srmc_mlp_loss_grad(self._h, _ptr(a), _ptr(y), a.shape[0], _ptr(grad), _ptr(loss),
                                         _stream(stream)))

    def srmc_mlp_fit(self, coarse: "Solver", n_data, iters, batch, lr, seed, loss_curve=None, stream=None):
        _check(lib().srmc_mlp_fit(self._h, coarse.handle, int(n_data), int(iters), int(batch), float(lr),
                                  int(seed), _ptr(loss_curve), _stream(stream)))

    def srmc_mlp_fit_noalloc(self, coarse: "Solver", n_data, iters, batch, lr, seed, loss_curve=None,
                             stream=None):
        """srmc_mlp_fit without device allocation (scratch compiled into the library)."""
        _check(lib().srmc_mlp_fit_noalloc(self._h, coarse.handle, int(n_data), int(iters), int(batch),
                                          float(lr), int(seed), _ptr(loss_curve), _stream(stream)))

    def srmc_cv_tabulate(self, solver: "Solver", stream=None):
        _check(lib().srmc_cv_tabulate(self._h, solver.handle, _stream(stream)))


class Batch:
    """Many FP32 solvers solved together (wraps srmc_batch_create); the
    solvers must outlive the batch."""

    def __init__(self, solvers):
        self._solvers = list(solvers)
        arr = (C.c_void_p * len(self._solvers))(*[s.handle for s in self._solvers])
        h = C.c_void_p()
        _check(lib().srmc_batch_create(arr, len(self._solvers), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().srmc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def srmc_batch_tune(self, stream=None):
        out = (C.c_int * 64)()
        ng = C.c_int()
        _check(lib().srmc_batch_tune(self._h, _stream(stream), out, 64, C.byref(ng)))
        return [int(out[a]) for a in range(min(ng.value, 64))]

    def srmc_batch_solve(self, stream=None):
        _check(lib().srmc_batch_solve(self._h, _stream(stream)))

    def srmc_batch_mode(self) -> int:
        return int(lib().srmc_batch_mode(self._h))

    def srmc_batch_set_mode(self, mode: int):
        _check(lib().srmc_batch_set_mode(self._h, int(mode)))

    def srmc_batch_strategy_ms(self):
        """[rounds, branches, persistent] whole-batch ms measured by the last tune."""
        out = (C.c_float * 3)()
        _check(lib().srmc_batch_strategy_ms(self._h, out))
        return [float(v) for v in out]

    def srmc_batch_stats(self) -> int:
        """Number of waits of the persistent strategy that gave up (0 normally)."""
        out = C.c_ulonglong()
        _check(lib().srmc_batch_stats(self._h, C.byref(out)))
        return int(out.value)
