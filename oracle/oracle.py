"""ctypes binding of the FP64 CPU oracle (srmc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product path (``paper_2407_21085_gb300``) never imports this module.

The oracle follows Alg. SRMDP step by step in double precision (see the
header of srmc_oracle.c for the passage behind every function).
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "srmc_oracle.c")
_HDR = os.path.join(_HERE, "srmc_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_OUT = os.path.join(_BUILD, "libsrmc_oracle.so")
DMAX = 19
PMAX = 24
MODELS = {"cos": 0, "logistic": 1, "affine": 2, "user": 3}
BASES = {"lp0": 0, "lp1": 1, "lp2": 2}
STRATA = {"size": 0, "prob": 1}
DYNAMICS = {"euler": 0, "exact": 1}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP, no FP contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    stale = (not os.path.exists(_OUT)
             or os.path.getmtime(_OUT) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _OUT + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


_USER_G = C.CFUNCTYPE(C.c_double, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double))
_USER_F = C.CFUNCTYPE(C.c_double, C.c_double, C.POINTER(C.c_double), C.c_double, C.POINTER(C.c_double),
                      C.c_int, C.POINTER(C.c_double))
_USER_B = C.CFUNCTYPE(C.c_double, C.c_double, C.POINTER(C.c_double), C.c_int, C.c_int, C.POINTER(C.c_double))
_user_libs = {}


def user_model(source: str):
    """Compile a user model's source (srmc_user_g, srmc_user_f, optionally
    srmc_user_b and srmc_user_sigma) as plain C with srmc_real = double, and
    return its (g, f, b, sigma) function pointers (b, sigma None if absent)."""
    import hashlib
    key = hashlib.sha256(source.encode()).hexdigest()[:16]
    if key not in _user_libs:
        out = os.path.join(_BUILD, f"user_{key}.so")
        src = out[:-3] + ".c"
        os.makedirs(_BUILD, exist_ok=True)
        with open(src, "w") as fh:
            fh.write("#include <math.h>\ntypedef double srmc_real;\n#define SRMC_USER\n" + source + "\n")
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", out, src, "-lm"],
                       check=True)
        L = C.CDLL(out)
        dyn = hasattr(L, "srmc_user_b") and hasattr(L, "srmc_user_sigma")
        _user_libs[key] = (L, _USER_G(("srmc_user_g", L)), _USER_F(("srmc_user_f", L)),
                           _USER_B(("srmc_user_b", L)) if dyn else None,
                           _USER_B(("srmc_user_sigma", L)) if dyn else None)
    return _user_libs[key][1:]


class _Problem(C.Structure):
    _fields_ = [
        ("d", C.c_int), ("q", C.c_int), ("N", C.c_int), ("T", C.c_double),
        ("b", C.c_double * DMAX), ("sigma", C.c_double * (DMAX * DMAX)),
        ("model", C.c_int), ("params", C.c_double * PMAX),
        ("cells", C.c_int * DMAX), ("lo", C.c_double * DMAX), ("hi", C.c_double * DMAX),
        ("mu", C.c_double), ("basis", C.c_int), ("M", C.c_int64),
        ("seed", C.c_uint64), ("instance", C.c_uint32), ("Cy", C.c_double), ("Cz", C.c_double),
        ("strata", C.c_int), ("M_strata", C.POINTER(C.c_int64)),
        ("theta", C.c_double * DMAX), ("dynamics", C.c_int),
        ("user_g", _USER_G), ("user_f", _USER_F), ("user_b", _USER_B), ("user_sigma", _USER_B),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(C.CDLL(build()))
    return _lib


def compile_variant(source_text: str, out_path: str):
    """Compile a modified copy of the oracle source (used by tests that plant a
    mistake in the oracle to show that the pins catch it) and bind it."""
    src = out_path + ".c"
    with open(src, "w") as fh:
        fh.write(source_text)
    shutil.copy(_HDR, os.path.join(os.path.dirname(out_path), "srmc_oracle.h"))
    subprocess.run(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", "-o", out_path, src, "-lm"], check=True)
    return _bind(C.CDLL(out_path))


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _bind(L):
    P = C.POINTER(_Problem)
    u32p = C.POINTER(C.c_uint32)
    dp = C.POINTER(C.c_double)
    L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.orc_uniform.argtypes = [C.c_uint32]; L.orc_uniform.restype = C.c_double
    L.orc_norminv.argtypes = [C.c_double]; L.orc_norminv.restype = C.c_double
    L.orc_normal_from_word.argtypes = [C.c_uint32]; L.orc_normal_from_word.restype = C.c_double
    L.orc_draw_word.argtypes = [P, C.c_int, C.c_int64, C.c_int64, C.c_int64]
    L.orc_draw_word.restype = C.c_uint32
    L.orc_logistic_cdf.argtypes = [C.c_double, C.c_double]; L.orc_logistic_cdf.restype = C.c_double
    L.orc_sample_restricted.argtypes = [C.c_double] * 4; L.orc_sample_restricted.restype = C.c_double
    L.orc_locate_dim.argtypes = [P, C.c_int, C.c_double]; L.orc_locate_dim.restype = C.c_int
    L.orc_locate.argtypes = [P, dp]; L.orc_locate.restype = C.c_int64
    L.orc_locate_dim_f32.argtypes = [C.c_float, C.c_float, C.c_float, C.c_int]
    L.orc_locate_dim_f32.restype = C.c_int
    L.orc_cell_edges.argtypes = [P, C.c_int, C.c_int, dp, dp]
    L.orc_stratum_centre.argtypes = [P, C.c_int64, dp]
    L.orc_cell_scale.argtypes = [P, C.c_int, C.c_int]; L.orc_cell_scale.restype = C.c_double
    L.orc_start_point.argtypes = [P, C.c_int, C.c_int64, C.c_int64, dp]
    L.orc_g.argtypes = [P, dp]; L.orc_g.restype = C.c_double
    L.orc_f.argtypes = [P, C.c_int, dp, C.c_double, dp]; L.orc_f.restype = C.c_double
    L.orc_lstsq_householder.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp]
    L.orc_lstsq_householder.restype = C.c_int
    L.orc_create.argtypes = [P]; L.orc_create.restype = C.c_void_p
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_row_len.argtypes = [C.c_void_p]; L.orc_row_len.restype = C.c_int
    L.orc_solve_full.argtypes = [C.c_void_p, C.c_int]; L.orc_solve_full.restype = C.c_int
    L.orc_fit_lazy.argtypes = [C.c_void_p, C.c_int, C.c_int64]; L.orc_fit_lazy.restype = C.c_int
    L.orc_fit_one.argtypes = [C.c_void_p, C.c_int, C.c_int64]; L.orc_fit_one.restype = C.c_int64
    L.orc_row.argtypes = [C.c_void_p, C.c_int, C.c_int64]; L.orc_row.restype = dp
    L.orc_eval.argtypes = [C.c_void_p, C.c_int, C.c_int64, dp, dp, dp]
    L.orc_eval.restype = C.c_int64
    L.orc_fallbacks.argtypes = [C.c_void_p]; L.orc_fallbacks.restype = C.c_int64
    L.orc_path_steps.argtypes = [C.c_void_p]; L.orc_path_steps.restype = C.c_int64
    L.orc_set_control.argtypes = [C.c_void_p, dp]; L.orc_set_control.restype = C.c_int
    L.orc_set_own_control.argtypes = [C.c_void_p, C.c_int]; L.orc_set_own_control.restype = None
    L.orc_set_rows_centred.argtypes = [C.c_void_p, C.c_int, dp, C.c_int64, dp, C.c_int64]
    L.orc_set_rows_centred.restype = C.c_int
    L.orc_fit_many.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.POINTER(C.c_int64), C.c_int]
    L.orc_fit_many.restype = C.c_int64
    L.orc_set_missing_zero.argtypes = [C.c_void_p, C.c_int]; L.orc_set_missing_zero.restype = None
    fp = C.POINTER(C.c_float)
    L.orc_mlp_nparams.argtypes = [C.c_int, C.c_int]; L.orc_mlp_nparams.restype = C.c_int
    L.orc_bf16.argtypes = [C.c_double]; L.orc_bf16.restype = C.c_float
    L.orc_mlp_eval.argtypes = [fp, C.c_int, C.c_int, C.c_int, dp, dp, dp]
    L.orc_mlp_loss_grad.argtypes = [fp, C.c_int, C.c_int, C.c_int, C.c_int64, dp, dp, dp]
    L.orc_mlp_loss_grad.restype = C.c_double
    return L


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def to_struct(w) -> _Problem:
    """Fill the oracle's problem struct from a workload description (any
    object with the fields of ``paper_2407_21085_gb300.workloads.Workload``)."""
    p = _Problem()
    p.d, p.q, p.N, p.T = int(w.d), int(w.q), int(w.N), float(w.T)
    for l in range(w.d):
        p.b[l] = float(w.b[l])
        for r in range(w.q):
            p.sigma[l * w.q + r] = float(w.sigma[l][r])
    p.model = MODELS[w.model]
    for a, v in enumerate(w.params):
        p.params[a] = float(v)
    for l in range(w.d):
        p.cells[l] = int(w.cells[l]); p.lo[l] = float(w.lo[l]); p.hi[l] = float(w.hi[l])
    p.mu = float(w.mu)
    p.basis = BASES[w.basis]
    p.M = int(w.M)
    p.seed = int(w.seed)
    p.instance = int(w.instance)
    p.Cy, p.Cz = float(w.Cy), float(w.Cz)
    p.strata = STRATA[getattr(w, "strata", "size")]
    for l, v in enumerate(getattr(w, "theta", None) or []):
        p.theta[l] = float(v)
    p.dynamics = DYNAMICS[getattr(w, "dynamics", "euler")]
    if w.model == "user":
        g, f, b, s = user_model(w.user_source)
        p.user_g, p.user_f = g, f
        if getattr(w, "user_dynamics", False):
            if b is None:
                raise ValueError("user_dynamics: the source defines no srmc_user_b / srmc_user_sigma")
            p.user_b, p.user_sigma = b, s
    ms = getattr(w, "M_strata", None)
    if ms is not None:
        arr = np.ascontiguousarray(ms, dtype=np.int64)
        p._keep = arr                      # owned by the struct object
        p.M_strata = arr.ctypes.data_as(C.POINTER(C.c_int64))
    return p


# ---- primitives -------------------------------------------------------------
def philox4x32_10(ctr, key):
    L = lib()
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    L.orc_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def draw_word(w, i, k, m, n):
    return int(lib().orc_draw_word(C.byref(to_struct(w)), i, k, m, n))


def uniform(word):
    return lib().orc_uniform(int(word))


def norminv(u):
    return lib().orc_norminv(float(u))


def normal_from_word(word):
    return lib().orc_normal_from_word(int(word))


def logistic_cdf(x, mu):
    return lib().orc_logistic_cdf(float(x), float(mu))


def sample_restricted(U, xlo, xhi, mu):
    return lib().orc_sample_restricted(float(U), float(xlo), float(xhi), float(mu))


def locate_dim(w, l, x):
    return int(lib().orc_locate_dim(C.byref(to_struct(w)), l, float(x)))


def locate(w, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return int(lib().orc_locate(C.byref(to_struct(w)), _dptr(x)))


def locate_dim_f32(x, lo, r, cells):
    return int(lib().orc_locate_dim_f32(float(np.float32(x)), float(np.float32(lo)),
                                         float(np.float32(r)), int(cells)))


def cell_edges(w, l, c):
    a, b = C.c_double(), C.c_double()
    lib().orc_cell_edges(C.byref(to_struct(w)), l, c, C.byref(a), C.byref(b))
    return a.value, b.value


def stratum_centre(w, k):
    x = np.zeros(w.d)
    lib().orc_stratum_centre(C.byref(to_struct(w)), int(k), _dptr(x))
    return x


def cell_scale(w, l, c):
    """Unit of the centred basis coordinate of cell c of dimension l."""
    return float(lib().orc_cell_scale(C.byref(to_struct(w)), int(l), int(c)))


def start_point(w, i, k, m):
    x = np.zeros(w.d)
    lib().orc_start_point(C.byref(to_struct(w)), int(i), int(k), int(m), _dptr(x))
    return x


def g(w, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_g(C.byref(to_struct(w)), _dptr(x))


def f(w, j, x, y, z):
    x = np.ascontiguousarray(x, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    return lib().orc_f(C.byref(to_struct(w)), int(j), _dptr(x), float(y), _dptr(z))


def lstsq_householder(A, B):
    A = np.array(A, dtype=np.float64, order="C")
    B = np.array(B, dtype=np.float64, order="C")
    if B.ndim == 1:
        B = B[:, None]
    n, p = A.shape
    r = B.shape[1]
    X = np.zeros((p, r))
    rc = lib().orc_lstsq_householder(n, p, r, _dptr(A), _dptr(B), _dptr(X))
    return X, rc


# ---- the scheme -------------------------------------------------------------
class Oracle:
    """One oracle context: the raw-basis coefficient rows of every fitted (i,k)."""

    def __init__(self, w, library=None):
        self.w = w
        self._p = to_struct(w)
        self._L = library if library is not None else lib()
        self._ctx = self._L.orc_create(C.byref(self._p))
        if not self._ctx:
            raise ValueError("oracle: invalid problem or out of memory")
        self.K = int(np.prod(w.cells))
        self.R = self._L.orc_row_len(self._ctx)

    def close(self):
        if self._ctx:
            self._L.orc_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve_full(self, nthreads: int = 0) -> None:
        if self._L.orc_solve_full(self._ctx, int(nthreads)) != 0:
            raise RuntimeError("oracle: full solve found missing rows")

    def fit_lazy(self, i: int, k: int) -> None:
        if self._L.orc_fit_lazy(self._ctx, int(i), int(k)) != 0:
            raise RuntimeError("oracle: lazy fit failed")

    def row(self, i: int, k: int):
        ptr = self._L.orc_row(self._ctx, int(i), int(k))
        if not ptr:
            return None
        return np.ctypeslib.as_array(ptr, shape=(self.R,)).copy()

    def eval(self, i: int, x):
        x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
        n = x.shape[0]
        y = np.zeros(n)
        z = np.zeros((n, self.w.q))
        miss = self._L.orc_eval(self._ctx, int(i), n, _dptr(x), _dptr(y), _dptr(z))
        if miss:
            raise RuntimeError(f"oracle: {miss} points fall in strata not fitted at step {i}")
        return y, z

    def eval_lazy(self, i: int, x):
        """Fit every stratum the points fall in (lazily), then evaluate."""
        x = np.atleast_2d(np.asarray(x, dtype=np.float64))
        if i < self.w.N:
            for a in range(x.shape[0]):
                self.fit_lazy(i, locate(self.w, x[a]))
        return self.eval(i, x)

    def set_control(self, rows):
        """Control rows [N][K][q][p] (centred basis) or None."""
        if rows is None:
            self._L.orc_set_control(self._ctx, None)
            return
        self._control = np.ascontiguousarray(rows, dtype=np.float64)
        if self._L.orc_set_control(self._ctx, _dptr(self._control)) != 0:
            raise MemoryError("oracle: control rows")

    def set_own_control(self, on: bool = True):
        """Control from the run's own fitted z of the later steps."""
        self._control = None
        self._L.orc_set_own_control(self._ctx, 1 if on else 0)

    def set_rows_centred(self, i: int, yrows, zrows):
        """Install the rows of step i of every stratum from tables in the
        centred basis: yrows [K][>= p] (alpha), zrows [K][>= q p] (beta, row
        by row per component); extra columns (padding) are skipped."""
        y = np.ascontiguousarray(yrows, dtype=np.float64)
        z = np.ascontiguousarray(zrows, dtype=np.float64)
        if y.shape[0] != self.K or z.shape[0] != self.K:
            raise ValueError("set_rows_centred: tables need one row per stratum")
        if self._L.orc_set_rows_centred(self._ctx, int(i), _dptr(y), y.shape[1], _dptr(z), z.shape[1]) != 0:
            raise ValueError(f"set_rows_centred: invalid step {i}")

    def fit_many(self, i: int, ks, nthreads: int = 0) -> None:
        """Fit the strata ks of step i in parallel (rows of later steps must exist)."""
        ks = np.ascontiguousarray(ks, dtype=np.int64)
        miss = self._L.orc_fit_many(self._ctx, int(i), ks.shape[0], ks.ctypes.data_as(C.POINTER(C.c_int64)),
                                    int(nthreads))
        if miss != 0:
            raise RuntimeError(f"oracle: fits of step {i} were missing {miss} rows")

    def set_missing_zero(self, on: bool = True) -> None:
        """Timing aid: missing rows of later steps read as the zero function."""
        self._L.orc_set_missing_zero(self._ctx, 1 if on else 0)

    @property
    def fallbacks(self) -> int:
        return int(self._L.orc_fallbacks(self._ctx))

    @property
    def path_steps(self) -> int:
        return int(self._L.orc_path_steps(self._ctx))


# ---- the MLP of the learned control variate ---------------------------------
def mlp_nparams(nin, H):
    return int(lib().orc_mlp_nparams(nin, H))


def bf16(v):
    return float(lib().orc_bf16(float(v)))


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def mlp_eval(params, nin, H, a, bf16_round=False):
    """u and the input gradient at the rows of a (n x nin)."""
    prm = np.ascontiguousarray(params, dtype=np.float32)
    a = np.ascontiguousarray(np.atleast_2d(a), dtype=np.float64)
    n = a.shape[0]
    u = np.zeros(n)
    g = np.zeros((n, nin))
    L = lib()
    for s in range(n):
        uu = C.c_double()
        gg = np.zeros(nin)
        L.orc_mlp_eval(_fptr(prm), nin, H, int(bf16_round), _dptr(a[s]), C.byref(uu), _dptr(gg))
        u[s] = uu.value
        g[s] = gg
    return u, g


def mlp_loss_grad(params, nin, H, a, y, bf16_round=False):
    prm = np.ascontiguousarray(params, dtype=np.float32)
    a = np.ascontiguousarray(a, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    g = np.zeros(mlp_nparams(nin, H))
    loss = lib().orc_mlp_loss_grad(_fptr(prm), nin, H, int(bf16_round), a.shape[0], _dptr(a),
                                   _dptr(y), _dptr(g))
    return loss, g
