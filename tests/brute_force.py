"""A second, independent restatement of Alg. SRMDP for tiny problems.

Pure Python + numpy/scipy library routines, written straight from the paper
without looking at the C oracle's structure: its own Philox-4x32-10, the
normal quantile from scipy (Cephes ndtri), the restricted logistic quantile
through scipy's logit/expit, and numpy's lstsq for every OLS.  Used only by
tests, on problems with a handful of strata and paths.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

MASK = 0xFFFFFFFF


def philox(ctr, key, rounds=10):
    c = list(ctr)
    k = list(key)
    for r in range(rounds):
        if r:
            k = [(k[0] + 0x9E3779B9) & MASK, (k[1] + 0xBB67AE85) & MASK]
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k[0]) & MASK, p1 & MASK,
             ((p0 >> 32) ^ c[3] ^ k[1]) & MASK, p0 & MASK]
    return c


def word(w, i, k, m, n):
    key = [(w.seed & MASK) ^ w.instance, (w.seed >> 32) & MASK]
    return philox([n // 4, m, k, i], key)[n % 4]


def unif(u32):
    return (u32 + 0.5) / 2.0 ** 32


def normal(u32):
    return float(special.ndtri(unif(u32)))


def cells_of(w, k):
    out = []
    for C in w.cells:
        out.append(k % C)
        k //= C
    return out


def edges(w, l, c):
    C = w.cells[l]
    if getattr(w, "strata", "size") == "prob":
        # equal nu-probability: cut at the logistic quantiles c/C
        a = -math.inf if c == 0 else float(special.logit(c / C)) / w.mu
        b = math.inf if c == C - 1 else float(special.logit((c + 1) / C)) / w.mu
        return a, b
    h = (w.hi[l] - w.lo[l]) / C
    a = -math.inf if c == 0 else w.lo[l] + c * h
    b = math.inf if c == C - 1 else w.lo[l] + (c + 1) * h
    return a, b


def centre_and_unit(w, l, c):
    """Centre of cell c and the unit of the centred basis coordinate."""
    C = w.cells[l]
    if getattr(w, "strata", "size") == "prob":
        q = lambda u: float(special.logit(u / C)) / w.mu
        return q(c + 0.5), q(c + 0.75) - q(c + 0.25)
    h = (w.hi[l] - w.lo[l]) / C
    return w.lo[l] + (c + 0.5) * h, h / 2


def start(w, i, k, m):
    x = np.zeros(w.d)
    cs = cells_of(w, k)
    for l in range(w.d):
        a, b = edges(w, l, cs[l])
        if getattr(w, "strata", "size") == "prob":
            Fa, Fb = cs[l] / w.cells[l], (cs[l] + 1) / w.cells[l]
        else:
            Fa = 0.0 if a == -math.inf else special.expit(w.mu * a)
            Fb = 1.0 if b == math.inf else special.expit(w.mu * b)
        U = unif(word(w, i, k, m, l))
        x[l] = special.logit(Fa + U * (Fb - Fa)) / w.mu
    return x


def locate(w, x):
    k, stride = 0, 1
    for l in range(w.d):
        if getattr(w, "strata", "size") == "prob":
            c = 0
            while c < w.cells[l] - 1 and x[l] >= edges(w, l, c + 1)[0]:
                c += 1
        else:
            h = (w.hi[l] - w.lo[l]) / w.cells[l]
            c = int(min(max(math.floor((x[l] - w.lo[l]) / h), 0), w.cells[l] - 1))
        k += c * stride
        stride *= w.cells[l]
    return k


def _user(w):
    from tests.user_models import PY
    return PY[w.user_source]


def g(w, x):
    if w.model == "user":
        return _user(w)[0](x, w.params)
    if w.model == "cos":
        return math.cos(x.sum() / math.sqrt(w.d))
    if w.model == "logistic":
        e = math.exp(w.T + x.sum())
        return e / (1 + e)
    p = w.params
    return p[0] + float(np.dot(p[1:1 + w.d], x))


def f(w, j, x, y, z):
    t = j * w.T / w.N
    if w.model == "user":
        return _user(w)[1](t, x, y, z, w.params)
    if w.model == "cos":
        lam, kap, kapz, s0 = w.params[:4]
        s = x.sum() / math.sqrt(w.d)
        e = math.exp(lam * (w.T - t))
        out = (lam + s0 * s0 / 2) * y + kap * (y * y - (e * math.cos(s)) ** 2)
        drift = _drift(w, x)
        if np.any(drift != 0.0):
            # u solves the PDE whose generator has drift b(x): the driver
            # cancels b(x).grad u = b(x).z / s0
            out -= float(np.dot(drift, z)) / s0
        if kapz:
            out += kapz * (float(np.dot(z, z)) - (s0 * e * math.sin(s)) ** 2)
        return out
    if w.model == "logistic":
        return float(np.sum(z)) * (y - (2 + w.q) / (2 * w.q))
    p, d = w.params, w.d
    return p[1 + d] + float(np.dot(p[2 + d:2 + 2 * d], x)) + p[2 + 2 * d] * y


def _drift(w, x):
    th = np.array(w.theta if getattr(w, "theta", None) else [0.0] * w.d, dtype=float)
    return np.array(w.b, dtype=float) - th * x


def ou_step(w, x, dw, xi2):
    """One exact step (Alg. 1) of dX_l = (b_l - theta_l X_l) dt + s_l dW_l:
    X' = X e^{-theta dt} + (b/theta)(1 - e^{-theta dt}) + s I, I the Ito integral
    of e^{-theta(dt-u)}, which given dW is normal with mean (Cov/dt) dW and
    variance Var I - Cov^2/dt (Cov = (1 - e^{-theta dt})/theta,
    Var I = (1 - e^{-2 theta dt})/(2 theta)); theta = 0 gives X + b dt + s dW."""
    dt = w.T / w.N
    th = w.theta if getattr(w, "theta", None) else [0.0] * w.d
    out = np.empty(w.d)
    for l in range(w.d):
        t, s = th[l], w.sigma[l][l]
        if t == 0.0:
            out[l] = x[l] + w.b[l] * dt + s * dw[l]
            continue
        A = math.exp(-t * dt)
        cov = (1.0 - A) / t
        var = (1.0 - A * A) / (2.0 * t)
        cond_var = max(var - cov * cov / dt, 0.0)
        I = cov / dt * dw[l] + math.sqrt(cond_var) * xi2[l]
        out[l] = x[l] * A + w.b[l] * cov + s * I
    return out


def clamp(v, L):
    return v if L <= 0 else float(np.clip(v, -L, L))


def monomials(basis, u):
    """[1] (LP0), [1, u] (LP1) or [1, u, u_a u_b for a <= b] (LP2)."""
    v = [1.0]
    if basis != "lp0":
        v += list(u)
    if basis == "lp2":
        v += [u[a] * u[b] for a in range(len(u)) for b in range(a, len(u))]
    return np.array(v)


def control_value(w, rows, j, k, x, dw):
    """zc_j(x).dw with zc_j(x) = T_Cz(beta_{j,k} . monomials((x - c_k)/s_k)),
    c_k and s_k the basis centre and unit of stratum k (rows [N][K][q][p])."""
    cs = cells_of(w, k)
    u = []
    for l in range(w.d):
        c, unit = centre_and_unit(w, l, cs[l])
        u.append((x[l] - c) / unit)
    v = monomials(w.basis, u)
    return sum(clamp(float(rows[j, k, l] @ v), w.Cz) * dw[l] for l in range(w.q))


def solve(w, control=None):
    """All rows: rows[i][k] = (alpha[p], beta[q, p]) in the raw basis.

    control: None; an array of control rows [N][K][q][p] (centred basis),
    whose step-i term zc_i(x_i).dW_i (stratum k) leaves the Y response and
    whose later terms sum_{j>i} zc_j(X_j).dW_j (stratum of X_j) leave both
    responses; or "own": the later terms with z_j the fitted z of the run
    itself, no step-i term."""
    N, d, q, M = w.N, w.d, w.q, w.M
    dt = w.T / N
    p = len(monomials(w.basis, [0.0] * d))
    sig = np.array(w.sigma, dtype=float)
    b = np.array(w.b, dtype=float)
    rows = [dict() for _ in range(N)]

    def phi(x):
        return monomials(w.basis, x)

    def y_and_z(j, x):
        if j == N:
            return g(w, x), None
        al, be = rows[j][locate(w, x)]
        v = phi(x)
        return clamp(float(al @ v), w.Cy), np.array([clamp(float(be[l] @ v), w.Cz) for l in range(q)])

    for i in range(N - 1, -1, -1):
        for k in range(w.K):
            Mk = M if getattr(w, "M_strata", None) is None else int(w.M_strata[k])
            X0, DW, S1, Y1, CZ, CI = [], [], [], [], [], []
            for m in range(Mk):
                x = start(w, i, k, m)
                X0.append(x.copy())
                path = [x]
                incs = []
                exact = getattr(w, "dynamics", "euler") == "exact"
                nw = 2 if exact else 1
                for j in range(i, N):
                    base = d + (j - i) * nw * q
                    dw = np.array([math.sqrt(dt) * normal(word(w, i, k, m, base + l)) for l in range(q)])
                    incs.append(dw)
                    if exact:
                        xi2 = [normal(word(w, i, k, m, base + q + l)) for l in range(q)]
                        path.append(ou_step(w, path[-1], dw, xi2))
                    elif getattr(w, "user_dynamics", False):
                        _, _, ub, us = _user(w)
                        xc, t = path[-1], j * dt
                        path.append(np.array([xc[l] + ub(t, xc, l, w.params) * dt
                                              + us(t, xc, l, w.params) * dw[l] for l in range(d)]))
                    else:
                        path.append(path[-1] + _drift(w, path[-1]) * dt + sig @ dw)
                cz = ci = 0.0
                for j in range(i, N):
                    xj, dw = path[j - i], incs[j - i]
                    if isinstance(control, str) and control == "own":
                        if j > i:
                            cz += float(y_and_z(j, xj)[1] @ dw)
                    elif control is not None:
                        v = control_value(w, control, j, k if j == i else locate(w, xj), xj, dw)
                        if j == i:
                            ci = v
                        else:
                            cz += v
                CZ.append(cz)
                CI.append(ci)
                S = g(w, path[-1])
                for j in range(i + 1, N):
                    xj, xj1 = path[j - i], path[j - i + 1]
                    yj1, _ = y_and_z(j + 1, xj1)
                    _, zj = y_and_z(j, xj)
                    S += f(w, j, xj, yj1, zj) * dt
                S1.append(S)
                DW.append(incs[0])
                Y1.append(y_and_z(i + 1, path[1])[0])
            A = np.array([phi(x) for x in X0])
            Bz = np.array([(S1[m] - CZ[m]) * DW[m] / dt for m in range(Mk)])
            beta = np.linalg.lstsq(A, Bz, rcond=None)[0].T          # q x p
            zi = [np.array([clamp(float(beta[l] @ phi(X0[m])), w.Cz) for l in range(q)])
                  for m in range(Mk)]
            By = np.array([S1[m] + f(w, i, X0[m], Y1[m], zi[m]) * dt - CZ[m] - CI[m]
                           for m in range(Mk)])
            alpha = np.linalg.lstsq(A, By, rcond=None)[0]
            rows[i][k] = (alpha, beta)
    return rows, y_and_z
