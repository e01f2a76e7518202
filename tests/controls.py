"""Test-side helpers of the control-variate tests: stratum centres and basis
units computed from a workload description, and control functions tabulated
as rows in the centred basis.  These compute the *expected* inputs and values
of tests; the library never uses them (it has its own kernels for centres and
for tabulating the network), and the oracle does not import them.
"""
import math

def _cell_index(w):
    import numpy as np
    idx = np.arange(w.K)
    out = np.zeros((w.K, w.d), dtype=np.int64)
    for l in range(w.d):
        out[:, l] = idx % w.cells[l]
        idx = idx // w.cells[l]
    return out


def _logistic_quantile(num, den, mu):
    """F^{-1}(num / (num + den)) of the logistic law with scale mu."""
    import numpy as np
    return np.log(np.asarray(num, dtype=float) / np.asarray(den, dtype=float)) / mu


def centres(w):
    """Stratum centres [K][d], k with dimension 0 fastest: the centre of the
    nominal finite cell (equal-size strata) or the median of nu restricted to
    the cell (equal-probability strata)."""
    import numpy as np
    cells = _cell_index(w)
    out = np.zeros((w.K, w.d))
    for l in range(w.d):
        c = cells[:, l]
        if w.strata == "prob":
            C = w.cells[l]
            out[:, l] = _logistic_quantile(c + 0.5, C - c - 0.5, w.mu)
        else:
            h = (w.hi[l] - w.lo[l]) / w.cells[l]
            out[:, l] = w.lo[l] + (c + 0.5) * h
    return out


def cell_units(w):
    """[K][d]: the unit of the centred basis coordinate of each stratum, h/2
    (equal size) or the width between the quantiles (c + 1/4)/C and
    (c + 3/4)/C of nu (equal probability)."""
    import numpy as np
    cells = _cell_index(w)
    out = np.zeros((w.K, w.d))
    for l in range(w.d):
        c = cells[:, l]
        if w.strata == "prob":
            C = w.cells[l]
            out[:, l] = (_logistic_quantile(c + 0.75, C - c - 0.75, w.mu)
                         - _logistic_quantile(c + 0.25, C - c - 0.25, w.mu))
        else:
            out[:, l] = 0.5 * (w.hi[l] - w.lo[l]) / w.cells[l]
    return out


def control_rows(w, fn):
    """Tabulate a control function fn(t, X[n][d]) -> [n][q] on the strata as
    rows [N][K][q][p] in the centred basis [1, (x - c_k)/s_k] (centres and
    units s_k as above): the value at the centre and, for LP1, central
    differences at c +- (s_k/2) e_m (a step of one unit of the centred
    coordinate).  LP2 rows carry the same constant and linear parts and zero
    quadratic coefficients (any fixed function is a valid control)."""
    import numpy as np
    p = {"lp0": 1, "lp1": w.d + 1, "lp2": 1 + w.d + w.d * (w.d + 1) // 2}[w.basis]
    ctr = centres(w)
    unit = cell_units(w)
    rows = np.zeros((w.N, w.K, w.q, p))
    for j in range(w.N):
        t = j * w.T / w.N
        rows[j, :, :, 0] = fn(t, ctr)
        if p > 1:
            for m in range(w.d):
                e = np.zeros((w.K, w.d))
                e[:, m] = unit[:, m] / 2
                rows[j, :, :, 1 + m] = fn(t, ctr + e) - fn(t, ctr - e)
    return rows


def closed_form_z(w):
    """z*(t, x) = s0 grad u of the cos family (-s0 e^{lam(T-t)} sin(s)/sqrt(d)
    in every component) as a function for control_rows."""
    import numpy as np
    lam, s0 = w.params[0], w.params[3]

    def fn(t, X):
        s = X.sum(axis=1) / math.sqrt(w.d)
        v = -s0 * np.exp(lam * (w.T - t)) * np.sin(s) / math.sqrt(w.d)
        return np.repeat(v[:, None], w.q, axis=1)
    return fn


def random_smooth_z(w, seed: int = 0, scale: float = 0.3):
    """A seeded smooth function R^d -> R^q (a few random Fourier modes), used as
    an arbitrary control in unbiasedness tests."""
    import numpy as np
    rng = np.random.default_rng(seed)
    F = rng.normal(size=(4, w.d))
    A = rng.normal(size=(4, w.q)) * scale
    ph = rng.uniform(0, 2 * math.pi, size=4)

    def fn(t, X):
        return np.cos(X @ F.T + ph + t) @ A
    return fn
