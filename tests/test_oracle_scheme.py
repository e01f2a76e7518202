"""Pins of the oracle's whole scheme (Alg. SRMDP) against things other than
the oracle: exact affine solutions, brute force by a second restatement, the
M -> infinity limit computed by quadrature, and the closed-form solution."""
import math

import numpy as np
import pytest

from paper_2407_21085_gb300 import workloads as W
from tests import brute_force as bf
from tests.population_d1 import population_solve


def _affine_truth(d, N, T, g0, gv, f0, fv, a, b):
    """Exact y_i of the affine model with sigma = 0, by the backward recursion
    y_i(x) = (1 + a dt) y_{i+1}(x + b dt) + dt (f0 + fv.x), y_N = g0 + gv.x
    (the MDP of eq. MDP with a deterministic Euler chain)."""
    dt = T / N
    c0, cv = g0, np.array(gv, dtype=float)
    out = [None] * (N + 1)
    out[N] = (c0, cv.copy())
    b = np.array(b, dtype=float)
    for i in range(N - 1, -1, -1):
        # y_{i+1}(x + b dt) = c0 + cv.b dt + cv.x
        s0 = c0 + float(cv @ b) * dt
        c0, cv = (1 + a * dt) * s0 + dt * f0, (1 + a * dt) * cv + dt * np.array(fv, dtype=float)
        out[i] = (c0, cv.copy())
    return out


@pytest.mark.parametrize("basis", ["lp1", "lp0", "lp2"])
def test_exact_fit_affine_deterministic(orc, basis):
    # sigma = 0: the responses are exact affine functions of x_i, so LP1 and
    # LP2 (whose span holds the affine functions) reproduce y_i exactly; with
    # LP0 we take gv = fv = 0 (constant solution).
    d, N = 2, 5
    if basis != "lp0":
        gv, fv = [0.3, -0.7], [0.2, 0.05]
    else:
        gv, fv = [0.0, 0.0], [0.0, 0.0]
    w = W.affine(d=d, N=N, C=3, M=7, g0=0.4, gv=gv, f0=-0.3, fv=fv, a=0.6, b=[0.5, -0.25],
                 s0=0.0, basis=basis)
    o = orc.Oracle(w)
    o.solve_full(2)
    truth = _affine_truth(d, N, w.T, 0.4, gv, -0.3, fv, 0.6, [0.5, -0.25])
    rng = np.random.default_rng(0)
    x = rng.uniform(-3, 3, size=(50, d))
    for i in range(N):
        y, _ = o.eval(i, x)
        want = truth[i][0] + x @ truth[i][1]
        assert np.max(np.abs(y - want)) < 1e-12 * (1 + np.max(np.abs(want)))
    assert o.fallbacks == 0


@pytest.mark.parametrize("basis", ["lp1", "lp0", "lp2"])
def test_constant_solution_with_noise(orc, basis):
    # g = c, f = 0: S_Y = c on every path for any sigma, so y = c to rounding.
    w = W.affine(d=3, N=4, C=2, M=12 if basis == "lp2" else 9, g0=0.75, gv=[0, 0, 0], f0=0.0,
                 fv=[0, 0, 0], a=0.0, s0=0.6, basis=basis)
    o = orc.Oracle(w)
    o.solve_full(2)
    x = np.random.default_rng(1).normal(size=(40, 3)) * 2
    for i in range(w.N):
        y, _ = o.eval(i, x)
        assert np.max(np.abs(y - 0.75)) < 1e-13
    assert o.fallbacks == 0


BF_CASES = [
    dict(d=1, N=3, C=3, M=5, kapz=0.0, basis="lp1"),
    dict(d=1, N=2, C=4, M=8, kapz=0.4, basis="lp1"),
    dict(d=2, N=2, C=2, M=6, kapz=0.3, basis="lp1"),
    dict(d=2, N=3, C=2, M=4, kapz=0.0, basis="lp0"),
    dict(d=1, N=3, C=4, M=6, kapz=0.2, basis="lp1", strata="prob"),
    dict(d=2, N=2, C=3, M=6, kapz=0.0, basis="lp1", strata="prob"),
    dict(d=2, N=3, C=2, M=9, kapz=0.1, basis="lp1", M_strata=[3, 9, 5, 7]),
    dict(d=1, N=3, C=3, M=6, kapz=0.0, basis="lp1", b=[0.2], theta=[0.7]),
    dict(d=2, N=3, C=2, M=5, kapz=0.2, basis="lp1", b=[0.1, -0.3], theta=[0.5, 1.2], dynamics="exact"),
    dict(d=1, N=2, C=4, M=7, kapz=0.0, basis="lp0", b=[0.0], theta=[2.0], dynamics="exact"),
    dict(d=1, N=3, C=3, M=8, kapz=0.2, basis="lp2"),
    dict(d=2, N=2, C=2, M=12, kapz=0.1, basis="lp2", strata="prob"),
    # a non-diagonal sigma (correlated coordinates), with and without a drift
    dict(d=2, N=3, C=2, M=6, kapz=0.3, basis="lp1", sigma=[[0.5, 0.2], [-0.3, 0.4]]),
    dict(d=3, N=2, C=2, M=5, kapz=0.0, basis="lp1", sigma=[[0.5, 0.1, 0.0], [0.2, 0.4, -0.1], [0.0, 0.3, 0.6]],
         b=[0.1, 0.0, -0.2], theta=[0.3, 0.0, 0.0]),
    # q != d: fewer and more Brownian components than coordinates (d x q sigma)
    dict(d=2, N=3, C=2, M=6, kapz=0.3, basis="lp1", q=1, sigma=[[0.5], [-0.3]]),
    dict(d=1, N=3, C=3, M=5, kapz=0.2, basis="lp1", q=2, sigma=[[0.4, -0.25]]),
]
_BF = {}


def _bf_workload(case):
    w = W.cos_model("bf", d=case["d"], N=case["N"], C=case["C"], a=1.0, M=case["M"], s0=0.5,
                    lam=0.5, kap=0.4, kapz=case["kapz"], basis=case["basis"], seed=11, instance=3)
    return w.replace(Cy=1.5, Cz=1.2, strata=case.get("strata", "size"),   # active truncation somewhere
                     M_strata=case.get("M_strata"), b=case.get("b", [0.0] * case["d"]),
                     theta=case.get("theta", []), dynamics=case.get("dynamics", "euler"),
                     q=case.get("q", w.q), sigma=case.get("sigma", w.sigma))


def _brute_force_mismatch(orc, n, library=None):
    """max |oracle - brute force| over y and z at 30 points and every step."""
    case = BF_CASES[n]
    w = _bf_workload(case)
    if n not in _BF:
        _BF[n] = bf.solve(w)[1]
    y_and_z = _BF[n]
    o = orc.Oracle(w, library=library)
    o.solve_full(1)
    x = np.random.default_rng(2).uniform(-2, 2, size=(30, w.d))
    worst = 0.0
    for i in range(w.N):
        y, z = o.eval(i, x)
        for a in range(len(x)):
            yb, zb = y_and_z(i, x[a])
            worst = max(worst, abs(y[a] - yb), float(np.max(np.abs(z[a] - zb))))
    return worst


@pytest.mark.parametrize("n", range(len(BF_CASES)))
def test_brute_force_tiny(orc, n):
    # A separately written straight-line restatement on the same Philox draws.
    assert _brute_force_mismatch(orc, n) < 1e-10


def _population_case(Cy, Cz, basis, strata="size", dynamics="euler", theta=0.0, b=0.0):
    w = W.cos_model("pop", d=1, N=3, C=4, a=1.0, M=20000, s0=0.5, lam=0.5, kap=0.5,
                    kapz=0.3, basis=basis, seed=5)
    return w.replace(Cy=Cy, Cz=Cz, strata=strata, dynamics=dynamics, theta=[theta], b=[b])


_POP = {}
POP_XS = np.array([[-1.4], [-0.75], [-0.25], [0.25], [0.75], [1.4]])


def _population(case):
    if case not in _POP:
        _POP[case] = population_solve(_population_case(*case))
    return _POP[case]


def _population_discrepancy(orc, case, library=None, R=6):
    """max over steps, centres and (y, z) of |mean of R runs - limit| / tol,
    tol = 5 standard errors of the mean + 2e-4; <= 1 means agreement."""
    w = _population_case(*case)
    pop = _population(case)
    ys, zs = [], []
    for r in range(R):
        o = orc.Oracle(w.replace(seed=100 + r), library=library)
        o.solve_full(0)
        yy, zz = [], []
        for i in range(w.N):
            y, z = o.eval(i, POP_XS)
            yy.append(y); zz.append(z[:, 0])
        ys.append(yy); zs.append(zz)
    ys, zs = np.array(ys), np.array(zs)            # [R, N, points]
    worst = 0.0
    for i in range(w.N):
        yp, zp = pop(i, POP_XS[:, 0])
        for arr, ref in ((ys[:, i], yp), (zs[:, i], zp)):
            se = arr.std(0, ddof=1) / math.sqrt(R)
            worst = max(worst, float(np.max(np.abs(arr.mean(0) - ref) / (5 * se + 2e-4))))
    return worst


POP_CASES = [(3.3, 5.7, "lp1"), (0.9, 0.35, "lp1"), (3.3, 5.7, "lp0"), (3.3, 5.7, "lp1", "prob"),
             (3.3, 5.7, "lp2"), (0.9, 0.35, "lp2"),
             (3.3, 5.7, "lp1", "size", "euler", 1.5, 0.4), (3.3, 5.7, "lp1", "size", "exact", 1.5, 0.4)]


@pytest.mark.parametrize("case", POP_CASES)
def test_converges_to_population_scheme(orc, case):
    # The M -> infinity limit of the scheme by deterministic quadrature; R
    # independent oracle runs (different seeds) must agree with it within
    # 5 standard errors of their mean, at every stratum centre and step.
    # (0.9, 0.35) makes both truncations active.
    assert _population_discrepancy(orc, case) <= 1.0


# Plausible slips, planted in a patched copy of the oracle source: each must
# be caught by the population pin or by the brute-force restatement.
MUTANTS = {
    "driver_at_t_j_plus_1": ("S += orc_f(P, j, x, yn, zj) * dt;", "S += orc_f(P, j + 1, x, yn, zj) * dt;"),
    "z_response_without_1_over_dt": ("B[m * q + l] = (S1[m] - CZ[m]) * DW[m * q + l] / dt;",
                                     "B[m * q + l] = (S1[m] - CZ[m]) * DW[m * q + l];"),
    "y_response_without_f_i": ("B[m] = S1[m] + orc_f(P, i, X0 + m * d, Y1[m], zi) * dt - CZ[m] - CI[m];",
                               "B[m] = S1[m] - CZ[m] - CI[m];"),
    "no_z_truncation_in_y_response": ("zi[l] = trunc_L(w, P->Cz);", "zi[l] = w;"),
    "euler_increment_dt_not_sqrt_dt": ("dw[l] = sdt * orc_normal_from_word", "dw[l] = dt * orc_normal_from_word"),
    "y_next_not_truncated": ("*y = trunc_L(v, C->P.Cy);", "*y = v;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_population_pin_catches_planted_mistakes(orc, tmp_path, name):
    old, new = MUTANTS[name]
    src = orc.source_text()
    assert src.count(old) == 1
    lib = orc.compile_variant(src.replace(old, new), str(tmp_path / f"mut_{name}.so"))
    bf_worst = max(_brute_force_mismatch(orc, n, library=lib) for n in range(len(BF_CASES)))
    pop_worst = max(_population_discrepancy(orc, case, library=lib, R=4) for case in POP_CASES[:2])
    assert bf_worst > 1e-6 or pop_worst > 1.5, (name, bf_worst, pop_worst)


def test_closed_form_error_falls_with_dt(orc):
    # Against u = e^{lam(T-t)} cos(s): the sup error at the inner centres is
    # dominated by the O(dt) bias of the discrete scheme, so halving dt (with
    # M large enough) must shrink it.
    errs = []
    for N in (4, 8, 16):
        w = W.cfg1(N=N, M=2000, C=16)
        o = orc.Oracle(w)
        o.solve_full(0)
        xs = np.array([[orc.stratum_centre(w, k)[0]] for k in range(3, 13)])
        y, _ = o.eval(0, xs)
        u = math.exp(0.5) * np.cos(xs[:, 0])
        errs.append(np.max(np.abs(y - u)))
    assert errs[0] > 1.3 * errs[1] > 1.3 ** 2 * errs[2]
    assert errs[2] < 0.15


def test_lazy_equals_full(orc):
    w = W.cfg2(M=64, C=8, N=6, precision="fp64")
    full = orc.Oracle(w)
    full.solve_full(0)
    lazy = orc.Oracle(w)
    for (i, k) in [(0, 27), (2, 9), (5, 63), (3, 0)]:
        lazy.fit_lazy(i, k)
        assert np.array_equal(lazy.row(i, k), full.row(i, k))


def test_thread_count_does_not_change_results(orc):
    w = W.cfg2(M=50, C=6, N=5)
    a = orc.Oracle(w); a.solve_full(1)
    b = orc.Oracle(w); b.solve_full(7)
    for i in range(w.N):
        for k in range(w.K):
            assert np.array_equal(a.row(i, k), b.row(i, k))
