"""The M -> infinity limit of Alg. SRMDP in dimension one, by quadrature.

With infinitely many paths per stratum the empirical OLS problems of eq. PsiM
become the population OLS problems of eq. mc:mls under nu_k, and the
responses are replaced by their conditional expectations given X_i = x:

    W_i(x) = E[ v_{i+1}(X_{i+1}) Delta W_i | X_i = x ] / dt           (Z response)
    v_i(x) = E[ v_{i+1}(X_{i+1}) + f_i(x, y_{i+1}(X_{i+1}), z_i(x)) dt | X_i = x ]
    v_N    = g,

where y_{i+1}, z_i are the truncated population fits (Z first, then Y).  The
Euler step X_{i+1} = x + b dt + s0 sqrt(dt) xi is Gaussian, so each
conditional expectation is a one-dimensional integral against a normal
density; the fitted functions jump at the cell edges, so the integrals are
split there and done by Gauss-Legendre on short pieces.  Nothing here uses
random numbers; the Monte Carlo oracle must converge to these values at rate
M^{-1/2}.  Only the "cos" model with d = q = 1 and constant b, s0 is covered.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial.legendre import leggauss
from scipy.interpolate import CubicSpline

XMAX = 30.0          # logistic tail mass beyond |x| = 30 is below 1e-13 (mu = 1)
PIECE = 0.05
GL_X, GL_W = leggauss(8)


def _nodes(a, b, cuts=()):
    pts = sorted(set([a, b] + [c for c in cuts if a < c < b]))
    xs, ws = [], []
    for lo, hi in zip(pts[:-1], pts[1:]):
        n = max(1, int(math.ceil((hi - lo) / PIECE)))
        e = np.linspace(lo, hi, n + 1)
        mid = 0.5 * (e[1:] + e[:-1])[:, None]
        half = 0.5 * (e[1:] - e[:-1])[:, None]
        xs.append((mid + half * GL_X[None, :]).ravel())
        ws.append((half * GL_W[None, :]).ravel())
    return np.concatenate(xs), np.concatenate(ws)


def population_solve(w, grid_step=0.02):
    assert w.d == 1 and w.q == 1 and w.model == "cos"
    lam, kap, kapz, s0 = w.params[:4]
    N, T, mu = w.N, w.T, w.mu
    dt = T / N
    # Transition X' = A x + c + sd xi (xi ~ N(0,1)), and E[dW | X'] = zfac xi.
    # Euler (Alg. 2) with drift b - theta x: A = 1 - theta dt, c = b dt,
    # sd = s sqrt(dt), zfac = sqrt(dt).  Exact (Alg. 1): A = e^{-theta dt},
    # c = b B, sd = s sqrt(Var I), zfac = Cov(dW, I)/sqrt(Var I) = B/sqrt(Var I)
    # with B = (1 - A)/theta, Var I = (1 - A^2)/(2 theta).
    b0 = w.b[0]
    th = w.theta[0] if getattr(w, "theta", None) else 0.0
    if getattr(w, "dynamics", "euler") == "exact" and th != 0.0:
        A = math.exp(-th * dt)
        B = (1.0 - A) / th
        var_i = (1.0 - A * A) / (2.0 * th)
        c_shift, sd, zfac = b0 * B, w.sigma[0][0] * math.sqrt(var_i), B / math.sqrt(var_i)
    else:
        A = 1.0 - th * dt
        c_shift, sd, zfac = b0 * dt, w.sigma[0][0] * math.sqrt(dt), math.sqrt(dt)
    has_drift = b0 != 0.0 or th != 0.0

    def drift_z(xs, zs):
        # the driver's b(x).z / s0 term (cancels the drift in the PDE of u)
        return -(b0 - th * xs) * zs / s0 if has_drift else 0.0
    C = w.cells[0]
    if getattr(w, "strata", "size") == "prob":
        # equal nu-probability cells: edges at the logistic quantiles c/C
        inner = [math.log(c / (C - c)) / mu for c in range(1, C)]

        def cell(x):
            return np.searchsorted(np.array(inner), x, side="right").astype(int)
    else:
        h = (w.hi[0] - w.lo[0]) / C
        inner = [w.lo[0] + c * h for c in range(1, C)]

        def cell(x):
            return np.clip(np.floor((x - w.lo[0]) / h), 0, C - 1).astype(int)
    p = {"lp0": 1, "lp1": 2, "lp2": 3}[w.basis]

    def phi(x):
        cols = [np.ones_like(x), x, x * x][:p]
        return np.stack(cols, axis=1)

    def clamp(v, L):
        return v if L <= 0 else np.clip(v, -L, L)

    def u2(j, x):
        return (math.exp(lam * (T - j * dt)) * np.cos(x)) ** 2

    def sin2e2(j, x):
        return (s0 * math.exp(lam * (T - j * dt)) * np.sin(x)) ** 2

    # Global integration nodes for X_{i+1}, split at every cell edge.
    XN, WN = _nodes(-XMAX - 2.0, XMAX + 2.0, inner)
    grid = np.arange(-XMAX, XMAX + 1e-9, grid_step)

    # Cell quadrature of nu_k (logistic density restricted to the cell).
    cellq = []
    for c in range(C):
        a = -XMAX if c == 0 else inner[c - 1]
        b = XMAX if c == C - 1 else inner[c]
        xs, ws = _nodes(a, b)
        dens = mu * np.exp(-mu * xs) / (1 + np.exp(-mu * xs)) ** 2
        wk = ws * dens
        cellq.append((xs, wk / wk.sum()))

    def project(fun_vals, c):
        xs, wk = cellq[c]
        P = phi(xs)
        G = P.T @ (P * wk[:, None])
        r = P.T @ (wk * fun_vals)
        return np.linalg.solve(G, r)

    def gauss_mean(values_at_nodes, x):
        """E[h(A x + c + sd xi)] for every x in the array x."""
        out = np.empty((len(x),) + values_at_nodes.shape[1:])
        for s in range(0, len(x), 256):
            xx = x[s:s + 256]
            ker = np.exp(-0.5 * ((XN[None, :] - A * xx[:, None] - c_shift) / sd) ** 2) / (sd * math.sqrt(2 * math.pi))
            out[s:s + 256] = (ker * WN[None, :]) @ values_at_nodes
        return out

    def moment1(values_at_nodes, x):
        """E[h(X') xi] with xi = (X' - A x - c)/sd."""
        out = np.empty(len(x))
        for s in range(0, len(x), 256):
            xx = x[s:s + 256]
            xi = (XN[None, :] - A * xx[:, None] - c_shift) / sd
            ker = np.exp(-0.5 * xi ** 2) / (sd * math.sqrt(2 * math.pi))
            out[s:s + 256] = (ker * xi * WN[None, :]) @ values_at_nodes
        return out

    alpha = [None] * N
    beta = [None] * N
    # v_{i+1} is represented as smooth spline + exact piecewise z-part.
    v_next_smooth = None        # None means v_{N} = g
    z_next = None               # (beta of step i+1) for the piecewise part

    def v_at(xs, j, smooth, zb):
        if j == N:
            return np.cos(xs)
        val = smooth(xs)
        if kapz or has_drift:
            zj = clamp(np.sum(phi(xs) * zb[cell(xs)], axis=1), w.Cz)
            val = val + dt * (kapz * (zj ** 2 - sin2e2(j, xs)) + drift_z(xs, zj))
        return val

    def y_at(xs, j):
        if j == N:
            return np.cos(xs)
        return clamp(np.sum(phi(xs) * alpha[j][cell(xs)], axis=1), w.Cy)

    for i in range(N - 1, -1, -1):
        vN = v_at(XN, i + 1, v_next_smooth, z_next)
        yN = y_at(XN, i + 1)
        # Z fit: W_i(x) = E[v_{i+1}(X') dW] / dt = E[v_{i+1}(X') xi] zfac / dt.
        bz = np.zeros((C, p))
        for c in range(C):
            xs, _ = cellq[c]
            Wv = moment1(vN, xs) * zfac / dt
            bz[c] = project(Wv, c)
        beta[i] = bz
        # Smooth part of v_i and the Y fit.
        a_ = lam + 0.5 * s0 * s0
        hN = vN + dt * (a_ * yN + kap * yN ** 2)
        smooth_vals = gauss_mean(hN, grid) - dt * kap * u2(i, grid)
        spline = CubicSpline(grid, smooth_vals)
        ay = np.zeros((C, p))
        for c in range(C):
            xs, _ = cellq[c]
            vi = spline(xs)
            if kapz or has_drift:
                zi = clamp(np.sum(phi(xs) * bz[c], axis=1), w.Cz)
                vi = vi + dt * (kapz * (zi ** 2 - sin2e2(i, xs)) + drift_z(xs, zi))
            ay[c] = project(vi, c)
        alpha[i] = ay
        v_next_smooth, z_next = spline, bz

    def evaluate(i, xs):
        xs = np.asarray(xs, dtype=float)
        y = clamp(np.sum(phi(xs) * alpha[i][cell(xs)], axis=1), w.Cy)
        z = clamp(np.sum(phi(xs) * beta[i][cell(xs)], axis=1), w.Cz)
        return y, z

    return evaluate
