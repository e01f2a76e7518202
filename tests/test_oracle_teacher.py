"""Pins of the oracle's teacher-forcing entries (orc_set_rows_centred,
orc_fit_many, orc_set_missing_zero) against things other than the oracle.

- Installed rows are the functions they describe: y and z evaluated by the
  oracle at random points of each stratum equal the centred polynomial
  sum_c row_c phi_c(u), u = (x - centre)/unit, evaluated here with numpy from
  its definition (LP0, LP1, LP2; equal-size and equal-probability strata).
- A step refitted from installed later rows equals the full solve's fit of
  that step when the installed rows are the full solve's own functions,
  re-expressed in the centred basis by a numpy least-squares fit on points of
  each stratum (a route that shares nothing with the oracle's expansion).
- A planted mistake in the expansion (the sign of the centre term) fails the
  first pin.
"""
import numpy as np
import pytest

from paper_2407_21085_gb300 import workloads as W
from tests import controls as CT


def _dimb(w):
    return {"lp0": 1, "lp1": w.d + 1, "lp2": 1 + w.d + w.d * (w.d + 1) // 2}[w.basis]


def _monomials(u, p):
    """[1, u_1..u_d, u_a u_b (a <= b, row order)] truncated to p entries."""
    n, d = u.shape
    cols = [np.ones(n)]
    if p > 1:
        cols += [u[:, l] for l in range(d)]
    if p > d + 1:
        cols += [u[:, a] * u[:, b] for a in range(d) for b in range(a, d)]
    return np.stack(cols, 1)


def _points_in_strata(orc, w, n_per, rng):
    """n_per points in every stratum (uniform in the finite cell; outer
    cells reach two cell widths outwards), with their stratum index."""
    cells = np.stack(np.unravel_index(np.arange(w.K), w.cells[::-1]), 1)[:, ::-1]
    xs, ks = [], []
    for k in range(w.K):
        lo = np.zeros(w.d)
        hi = np.zeros(w.d)
        for l in range(w.d):
            a, b = orc.cell_edges(w, l, int(cells[k, l]))
            if not np.isfinite(a) and not np.isfinite(b):
                a, b = -2.0, 2.0
            elif not np.isfinite(a):
                a = b - 2.0
            elif not np.isfinite(b):
                b = a + 2.0
            lo[l], hi[l] = a, b
        x = lo + (hi - lo) * rng.uniform(0.02, 0.98, size=(n_per, w.d))
        xs.append(x)
        ks.append(np.full(n_per, k))
    x = np.concatenate(xs)
    k = np.concatenate(ks)
    assert all(orc.locate(w, x[a]) == k[a] for a in range(len(k)))
    return x, k


CASES = [
    W.cfg2(C=4, N=3, M=64),
    W.cfg2(C=3, N=3, M=64, basis="lp0"),
    W.cfg2(C=3, N=3, M=64, basis="lp2"),
    W.cfg2(C=5, N=3, M=64).replace(strata="prob"),
    W.cos_model("t3", d=3, N=3, C=3, a=2.0, M=64, s0=0.3, lam=0.2, kap=0.5).replace(cells=[2, 3, 4]),
]


def _random_tables(w, rng):
    p = _dimb(w)
    Y = rng.normal(size=(w.K, p + 1))            # one padding column, as the GPU tables have
    Z = rng.normal(size=(w.K, w.q * p + 2))
    return Y, Z


def _centred_eval(w, Y, Z, x, k):
    p = _dimb(w)
    ctr, unit = CT.centres(w)[k], CT.cell_units(w)[k]
    phi = _monomials((x - ctr) / unit, p)
    y = np.sum(Y[k, :p] * phi, 1)
    z = np.stack([np.sum(Z[k, l * p:(l + 1) * p] * phi, 1) for l in range(w.q)], 1)
    return y, z


@pytest.mark.parametrize("case", range(len(CASES)))
def test_installed_rows_are_the_centred_polynomials(orc, case):
    w = CASES[case].replace(Cy=0.0, Cz=0.0, precision="fp64")       # no truncation
    rng = np.random.default_rng(case)
    o = orc.Oracle(w)
    Y, Z = _random_tables(w, rng)
    o.set_rows_centred(1, Y, Z)
    x, k = _points_in_strata(orc, w, 6, rng)
    y, z = o.eval(1, x)
    ye, ze = _centred_eval(w, Y, Z, x, k)
    scale = 1 + np.abs(ye)
    assert np.max(np.abs(y - ye) / scale) < 1e-12
    assert np.max(np.abs(z - ze) / (1 + np.abs(ze))) < 1e-12


def _centred_fit_of(orc, o, w, i, rng):
    """The full solve's rows of step i re-expressed in the centred basis: for
    every stratum, evaluate its fitted (untruncated) functions at 4 p points
    of the stratum and solve the least-squares problem in the centred
    monomials with numpy (exact for polynomials of the basis' degree)."""
    p = _dimb(w)
    x, k = _points_in_strata(orc, w, 4 * p, rng)
    y, z = o.eval(i, x)
    ctr, unit = CT.centres(w)[k], CT.cell_units(w)[k]
    phi = _monomials((x - ctr) / unit, p)
    Y = np.zeros((w.K, p))
    Z = np.zeros((w.K, w.q * p))
    for kk in range(w.K):
        s = k == kk
        Y[kk] = np.linalg.lstsq(phi[s], y[s], rcond=None)[0]
        for l in range(w.q):
            Z[kk, l * p:(l + 1) * p] = np.linalg.lstsq(phi[s], z[s, l], rcond=None)[0]
    return Y, Z


@pytest.mark.parametrize("case", [0, 2, 3, 4])
def test_teacher_forced_refit_equals_the_full_solve(orc, case):
    # truncation off so that the evaluated functions are the polynomials
    w = CASES[case].replace(Cy=0.0, Cz=0.0, precision="fp64")
    rng = np.random.default_rng(10 + case)
    full = orc.Oracle(w)
    full.solve_full(0)
    forced = orc.Oracle(w)
    for j in range(1, w.N):
        Y, Z = _centred_fit_of(orc, full, w, j, rng)
        forced.set_rows_centred(j, Y, Z)
    xs = CT.centres(w)
    for i in range(w.N - 1, -1, -1):
        # refit step i from the installed rows of steps > i, then compare, and
        # install the full solve's rows of step i again for the next (lower) i
        ks = np.arange(w.K)
        forced.fit_many(i, ks)
        yf, zf = forced.eval(i, xs)
        yr, zr = full.eval(i, xs)
        assert np.max(np.abs(yf - yr)) < 1e-9 and np.max(np.abs(zf - zr)) < 1e-9, i
        for k in range(w.K):
            a, b = forced.row(i, k), full.row(i, k)
            assert np.allclose(a, b, rtol=1e-9, atol=1e-9), (i, k)
        if i > 0:
            Y, Z = _centred_fit_of(orc, full, w, i, rng)
            forced.set_rows_centred(i, Y, Z)


def test_fit_many_equals_fit_one(orc):
    w = W.cfg2(C=4, N=4, M=96, kapz=0.2)
    a, b = orc.Oracle(w), orc.Oracle(w)
    a.solve_full(0)
    b.solve_full(0)
    ks = np.array([0, 5, 9, 15, 3])
    # refit step 1 of the listed strata: in parallel (a) and one by one (b)
    a.fit_many(1, ks, nthreads=4)
    for k in ks:
        assert b._L.orc_fit_one(b._ctx, 1, int(k)) == 0
    for k in range(w.K):
        assert np.array_equal(a.row(1, k), b.row(1, k))


def test_missing_rows_read_as_zero_only_when_asked(orc):
    # a fit whose later rows are absent: refused by default; with the timing
    # aid it runs and equals a fit from installed zero rows
    w = W.cfg2(C=3, N=4, M=64, kapz=0.2)
    a = orc.Oracle(w)
    with pytest.raises(RuntimeError):
        a.fit_many(0, [4])
    a.set_missing_zero(True)
    a.fit_many(0, [4])
    b = orc.Oracle(w)
    p = _dimb(w)
    for j in range(1, w.N):
        b.set_rows_centred(j, np.zeros((w.K, p)), np.zeros((w.K, w.q * p)))
    b.fit_many(0, [4])
    assert np.array_equal(a.row(0, 4), b.row(0, 4))


def test_expansion_pin_catches_a_planted_sign(orc, tmp_path):
    src = orc.source_text()
    old = "raw[0] -= cen[1 + l] * ctr[l] / sc[l];"
    assert old in src
    lib = orc.compile_variant(src.replace(old, "raw[0] += cen[1 + l] * ctr[l] / sc[l];"),
                              str(tmp_path / "mut_teacher.so"))
    w = CASES[0].replace(Cy=0.0, Cz=0.0, precision="fp64")
    rng = np.random.default_rng(0)
    o = orc.Oracle(w, library=lib)
    Y, Z = _random_tables(w, rng)
    o.set_rows_centred(1, Y, Z)
    x, k = _points_in_strata(orc, w, 6, rng)
    y, _ = o.eval(1, x)
    ye, _ = _centred_eval(w, Y, Z, x, k)
    assert np.max(np.abs(y - ye)) > 1e-3
