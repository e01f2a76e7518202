"""Pins of the oracle's primitives against things other than the oracle.

Every check here compares with a published value, a closed form, a library
routine from another code base (scipy's Cephes, numpy's LAPACK), exact
rational arithmetic, or a second restatement written separately
(tests/brute_force.py).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import special, stats

from paper_2407_21085_gb300 import workloads as W
from tests import brute_force as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            v = line.split()
            assert v[0] == "10"
            rows.append(([int(a, 16) for a in v[1:5]], [int(a, 16) for a in v[5:7]],
                         [int(a, 16) for a in v[7:11]]))
    return rows


def test_philox_known_answers(orc):
    # Published known answers of Philox-4x32-10 (Salmon et al., SC'11).
    for ctr, key, want in _kat():
        assert list(orc.philox4x32_10(ctr, key)) == want


def test_philox_matches_second_restatement(orc):
    rng = np.random.default_rng(0)
    for _ in range(300):
        ctr = [int(v) for v in rng.integers(0, 2 ** 32, 4)]
        key = [int(v) for v in rng.integers(0, 2 ** 32, 2)]
        assert list(orc.philox4x32_10(ctr, key)) == bf.philox(ctr, key)
    assert bf.philox([0, 0, 0, 0], [0, 0]) == _kat()[0][2]


def test_draw_word_counter_layout(orc):
    # key = (seed_lo ^ instance, seed_hi), counter = (n/4, m, k, i), word n mod 4
    w = W.cfg2(seed=0x123456789ABCDEF0, instance=77)
    for (i, k, m, n) in [(0, 0, 0, 0), (3, 17, 4095, 5), (19, 4095, 1, 63), (7, 1234, 99, 2)]:
        key = [(0x9ABCDEF0 ^ 77), 0x12345678]
        want = bf.philox([n // 4, m, k, i], key)[n % 4]
        assert orc.draw_word(w, i, k, m, n) == want


def test_uniform_lattice(orc):
    assert orc.uniform(0) == 0.5 * 2.0 ** -32
    assert orc.uniform(0xFFFFFFFF) == (2.0 ** 32 - 0.5) * 2.0 ** -32
    assert orc.uniform(0x7FFFFFFF) + orc.uniform(0x80000000) == 1.0


def test_norminv_textbook_values(orc):
    # Phi^{-1}(0.975) = 1.959963984540054 (standard normal table value)
    assert abs(orc.norminv(0.975) - 1.959963984540054) < 2e-15
    assert orc.norminv(0.5) == 0.0
    assert abs(orc.norminv(0.8413447460685429) - 1.0) < 1e-14   # Phi(1)


def test_norminv_vs_cephes(orc):
    # scipy.special.ndtri is Cephes' independent implementation of Phi^{-1}.
    us = np.concatenate([np.logspace(-9.7, -0.31, 400), 1 - np.logspace(-9.7, -0.31, 400),
                         np.linspace(0.01, 0.99, 199)])
    for u in us:
        a = orc.norminv(u)
        b = special.ndtri(u)
        assert abs(a - b) <= 4e-15 * max(1.0, abs(b)), (u, a, b)


def test_normal_from_word_symmetry_and_range(orc):
    for wd in [0, 1, 2, 255, 0x12345678, 0x7FFFFFFF]:
        a = orc.normal_from_word(wd)
        b = orc.normal_from_word(0xFFFFFFFF - wd)
        assert a == -b
        assert abs(a - special.ndtri((wd + 0.5) / 2 ** 32)) <= 4e-15 * max(1, abs(a))
    assert -6.5 < orc.normal_from_word(0) < -6.2


def test_restricted_logistic_whole_line_is_logistic_quantile(orc):
    # One cell covering R: F^{-1}(U) = log(U/(1-U))/mu (logistic quantile).
    for mu in (1.0, 2.5):
        for U in (1e-9, 0.1, 0.5, 0.77, 1 - 1e-9):
            x = orc.sample_restricted(U, -math.inf, math.inf, mu)
            assert abs(x - math.log(U / (1 - U)) / mu) < 1e-13 * max(1, abs(x))


def test_restricted_logistic_inverts_restricted_cdf(orc):
    # F(x(U)) = F(x-) + U (F(x+) - F(x-)), with F from scipy's expit.
    for (a, b) in [(-4.0, -3.75), (-0.125, 0.0), (3.5, math.inf), (-math.inf, -3.0), (0.3, 0.9)]:
        for U in np.linspace(0.001, 0.999, 37):
            x = orc.sample_restricted(U, a, b, 1.0)
            Fa = 0.0 if a == -math.inf else special.expit(a)
            Fb = 1.0 if b == math.inf else special.expit(b)
            assert abs(special.expit(x) - (Fa + U * (Fb - Fa))) < 1e-15
            assert a <= x <= b


def test_restricted_logistic_ks(orc):
    # Samples of the start-point draws of one outer and one inner cell follow
    # the truncated logistic law (KS test against scipy.stats.logistic).
    w = W.cfg1()
    for c in (0, 13, 31):
        a, b = orc.cell_edges(w, 0, c)
        xs = np.array([orc.start_point(w, 3, c, m)[0] for m in range(4000)])
        Fa = stats.logistic.cdf(a)
        Fb = stats.logistic.cdf(b)
        cdf = lambda x: (stats.logistic.cdf(x) - Fa) / (Fb - Fa)
        assert stats.kstest(xs, cdf).pvalue > 1e-3
        assert np.all((xs >= a) & (xs <= b))


def test_start_point_matches_second_restatement(orc):
    w = W.cfg2()
    for (i, k, m) in [(0, 0, 0), (5, 2080, 17), (19, 4095, 4095), (11, 63, 1)]:
        assert np.allclose(orc.start_point(w, i, k, m), bf.start(w, i, k, m), rtol=1e-12, atol=1e-13)


def _exact_cell(x, lo, hi, C):
    xf, lof, hf = Fraction(x), Fraction(lo), (Fraction(hi) - Fraction(lo)) / C
    c = math.floor((xf - lof) / hf)
    return min(max(c, 0), C - 1)


def test_locate_matches_exact_rational_membership(orc):
    # Away from edges the FP64 decision equals exact rational cell membership.
    rng = np.random.default_rng(1)
    for w in (W.cfg1(), W.cfg2(), W.cfg3()):
        h = (w.hi[0] - w.lo[0]) / w.cells[0]
        for x in rng.uniform(w.lo[0] - 2, w.hi[0] + 2, 3000):
            t = (x - w.lo[0]) / h
            if abs(t - round(t)) < 1e-9:
                continue
            assert orc.locate_dim(w, 0, x) == _exact_cell(x, w.lo[0], w.hi[0], w.cells[0])


def test_locate_edges_half_open(orc):
    # Inner edges that are exact binary fractions belong to the upper cell;
    # points a few ulps below belong to the lower one; outer cells clamp.
    w = W.cfg2()                               # h = 1/8 exactly
    for c in range(1, 64):
        e = -4.0 + c * 0.125
        assert orc.locate_dim(w, 0, e) == c
        # x - lo is rounded before the division, so the switch from cell c-1
        # to c happens within two ulps of the edge and is monotone.
        u = np.spacing(max(abs(e), abs(e + 4.0)))   # ulp of x and of x - lo
        xs = [e + j * u for j in range(-4, 5)]
        cs = [orc.locate_dim(w, 0, x) for x in xs]
        assert cs == sorted(cs)
        assert cs[:2] == [c - 1, c - 1] and cs[4:] == [c] * 5
    assert orc.locate_dim(w, 0, -1e300) == 0 and orc.locate_dim(w, 0, 1e300) == 63
    assert orc.locate_dim(w, 0, 4.0) == 63 and orc.locate_dim(w, 0, -4.0) == 0
    assert orc.locate_dim(w, 0, float("nan")) == 0
    # stratum index: dimension 0 fastest
    assert orc.locate(w, [-4 + 5 * 0.125 + 0.01, -4 + 7 * 0.125 + 0.01]) == 5 + 7 * 64


def test_locate_f32_matches_exact_membership_away_from_edges(orc):
    rng = np.random.default_rng(2)
    lo, hi, C = -3.5, 3.5, 12
    r = np.float32(C / (hi - lo))
    for x in rng.uniform(-5, 5, 3000).astype(np.float32):
        t = (float(x) - lo) * C / (hi - lo)
        if abs(t - round(t)) < 1e-4:
            continue
        assert orc.locate_dim_f32(x, lo, r, C) == _exact_cell(float(x), lo, hi, C)


def test_start_points_lie_in_their_stratum(orc):
    w = W.cfg3()
    rng = np.random.default_rng(3)
    for _ in range(500):
        k = int(rng.integers(0, w.K)); m = int(rng.integers(0, w.M)); i = int(rng.integers(0, w.N))
        assert orc.locate(w, orc.start_point(w, i, k, m)) == k


# ---- equal-probability strata (assumption HS, example ii) --------------------

def _prob(w, C=None):
    return w.replace(strata="prob", cells=[C or c for c in w.cells])


@pytest.mark.parametrize("C", [1, 2, 3, 7, 16])
def test_prob_strata_have_equal_nu_mass(orc, C):
    # nu(H_k) = 1/K: every cell of every axis has logistic mass 1/C (scipy's
    # logistic CDF at the oracle's edges); the edges increase; centre = the
    # median of the restricted law; the basis unit is positive and finite.
    for mu in (1.0, 0.6):
        w = _prob(W.cfg1(), C).replace(mu=mu)
        prev = -math.inf
        for c in range(C):
            a, b = orc.cell_edges(w, 0, c)
            assert a == prev and a < b
            prev = b
            mass = stats.logistic.cdf(mu * b) - stats.logistic.cdf(mu * a)
            assert abs(mass - 1.0 / C) < 1e-14
            ctr = orc.stratum_centre(w, c)[0]
            assert abs(stats.logistic.cdf(mu * ctr) - (c + 0.5) / C) < 1e-14
            q = lambda u: stats.logistic.ppf(u) / mu
            assert math.isclose(orc.cell_scale(w, 0, c), q((c + 0.75) / C) - q((c + 0.25) / C), rel_tol=1e-12)
        assert prev == math.inf


def test_prob_locate_edges_and_scan(orc):
    # Half-open cells at the oracle's own edges: the edge value belongs to the
    # upper cell, the next double below to the lower one; random points agree
    # with scipy's logistic CDF (floor(C F(x))) away from the edges.
    w = _prob(W.cfg1(), 9)
    for c in range(1, 9):
        e = orc.cell_edges(w, 0, c)[0]
        assert orc.locate_dim(w, 0, e) == c
        assert orc.locate_dim(w, 0, np.nextafter(e, -np.inf)) == c - 1
    assert orc.locate_dim(w, 0, -1e300) == 0 and orc.locate_dim(w, 0, 1e300) == 8
    assert orc.locate_dim(w, 0, float("nan")) == 0
    rng = np.random.default_rng(4)
    for x in rng.logistic(size=3000) * 1.5:
        t = 9 * stats.logistic.cdf(x)
        if abs(t - round(t)) < 1e-9:
            continue
        assert orc.locate_dim(w, 0, x) == min(int(math.floor(t)), 8)


def test_prob_start_points_follow_the_restricted_law(orc):
    # Start points of an outer and an inner cell lie in the cell and follow nu
    # restricted to it (KS against scipy's logistic law); they also match the
    # second restatement.
    w = _prob(W.cfg1(), 6)
    for c in (0, 2, 5):
        a, b = orc.cell_edges(w, 0, c)
        xs = np.array([orc.start_point(w, 3, c, m)[0] for m in range(4000)])
        assert np.all((xs >= a) & (xs < b))
        Fa, Fb = c / 6, (c + 1) / 6
        assert stats.kstest(xs, lambda x: (stats.logistic.cdf(x) - Fa) / (Fb - Fa)).pvalue > 1e-3
    w2 = _prob(W.cfg3(), 5)
    rng = np.random.default_rng(5)
    for _ in range(200):
        k = int(rng.integers(0, w2.K)); m = int(rng.integers(0, 999)); i = int(rng.integers(0, w2.N))
        x = orc.start_point(w2, i, k, m)
        assert orc.locate(w2, x) == k
        assert np.allclose(x, bf.start(w2, i, k, m), rtol=1e-12, atol=1e-13)


def test_householder_lstsq_vs_lapack(orc):
    rng = np.random.default_rng(4)
    for (n, p, r) in [(50, 3, 2), (7, 7, 1), (1000, 5, 4), (3, 1, 1)]:
        A = rng.normal(size=(n, p)) + np.array([1.0] + [0.0] * (p - 1))
        B = rng.normal(size=(n, r))
        X, rc = orc.lstsq_householder(A, B)
        assert rc == 0
        ref = np.linalg.lstsq(A, B, rcond=None)[0]
        assert np.allclose(X, ref, rtol=1e-11, atol=1e-12)
    # planted exact coefficients are recovered
    A = np.column_stack([np.ones(40), rng.uniform(3, 3.5, 40), rng.uniform(-1, 1, 40)])
    c = np.array([0.7, -2.0, 0.25])
    X, rc = orc.lstsq_householder(A, A @ c)
    assert rc == 0 and np.allclose(X[:, 0], c, rtol=0, atol=1e-12)
    # rank-deficient input is reported
    A2 = np.column_stack([np.ones(10), np.full(10, 2.0)])
    assert orc.lstsq_householder(A2, np.ones(10))[1] == 1


def _pde_residual(orc, w, t_index, x, u, grad_u, hess_diag_sum, dudt):
    """d_t u + (1/2) sum_l s_l^2 d_ll u + f(t, x, u, grad_u sigma) at one point."""
    s = np.array([w.sigma[l][l] for l in range(w.d)])
    z = grad_u * s
    return dudt + 0.5 * float(np.sum(s ** 2 * hess_diag_sum)) + orc.f(w, t_index, x, u, z)


@pytest.mark.parametrize("kapz", [0.0, 0.2])
def test_cos_model_driver_solves_its_pde(orc, kapz):
    # u = e^{lam (T-t)} cos(s) with its exact derivatives must make the PDE
    # residual vanish for the oracle's f (pins every term and sign of f).
    w = W.cos_model("t", d=3, N=10, C=4, a=2.0, M=8, s0=0.35, lam=0.4, kap=0.3, kapz=kapz)
    lam = 0.4
    rng = np.random.default_rng(5)
    for j in range(w.N):
        t = j * w.dt
        x = rng.normal(size=3)
        s = x.sum() / math.sqrt(3)
        e = math.exp(lam * (1 - t))
        u = e * math.cos(s)
        grad = np.full(3, -e * math.sin(s) / math.sqrt(3))
        hess = np.full(3, -e * math.cos(s) / 3)
        assert abs(_pde_residual(orc, w, j, x, u, grad, hess, -lam * u)) < 1e-13
    # and g = u(T, .)
    x = rng.normal(size=3)
    assert abs(orc.g(w, x) - math.cos(x.sum() / math.sqrt(3))) < 1e-15


def test_paper_logistic_model_solves_its_pde(orc):
    # Sec. 5.1: y = w/(1+w), z_k = w/(1+w)^2 with w = exp(t + sum x).
    w = W.logistic_paper(d=4, N=10, C=2, M=8)
    rng = np.random.default_rng(6)
    for j in range(w.N):
        t = j * w.dt
        x = rng.normal(scale=0.5, size=4)
        om = math.exp(t + x.sum())
        u = om / (1 + om)
        grad = np.full(4, u * (1 - u))
        hess = np.full(4, u * (1 - u) * (1 - 2 * u))
        assert abs(_pde_residual(orc, w, j, x, u, grad, hess, u * (1 - u))) < 1e-14
    x = rng.normal(size=4)
    om = math.exp(1 + x.sum())
    assert abs(orc.g(w, x) - om / (1 + om)) < 1e-15
