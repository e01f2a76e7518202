"""Pins of the oracle's control-variate parts: the MLP (against finite
differences and torch's bfloat16 rounding) and the martingale control in the
scheme (against the M -> infinity limit, which a zero-mean control must leave
unchanged, and against planted mistakes)."""
import math

import numpy as np
import pytest

from paper_2407_21085_gb300 import workloads as W
from tests import controls as CT
from tests import brute_force as bf
from tests.test_oracle_scheme import BF_CASES, POP_CASES, POP_XS, _bf_workload, _population, _population_case


def _params(nin, H, seed=0, scale=0.6):
    rng = np.random.default_rng(seed)
    P = []
    P.append(rng.normal(size=(H, nin)) * scale / math.sqrt(nin))
    P.append(rng.normal(size=H) * 0.1)
    P.append(rng.normal(size=(H, H)) * scale / math.sqrt(H))
    P.append(rng.normal(size=H) * 0.1)
    P.append(rng.normal(size=H) * scale / math.sqrt(H))
    P.append(rng.normal(size=1) * 0.1)
    return np.concatenate([p.ravel() for p in P]).astype(np.float32)


def test_bf16_rounding_matches_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.normal(size=2000) * 10, [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8,
                                                         0.0, 1e-30, 65504.0, 3.1415926]])
    vals32 = vals.astype(np.float32)
    want = torch.from_numpy(vals32).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([orc.bf16(float(v)) for v in vals32], dtype=np.float32)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("nin,H", [(3, 8), (7, 64)])
def test_mlp_input_gradient_vs_finite_differences(orc, nin, H):
    prm = _params(nin, H, seed=1)
    rng = np.random.default_rng(2)
    a = rng.normal(size=(5, nin))
    u, g = orc.mlp_eval(prm, nin, H, a)
    eps = 1e-6
    for s in range(5):
        for c in range(nin):
            ap, am = a[s].copy(), a[s].copy()
            ap[c] += eps
            am[c] -= eps
            fd = (orc.mlp_eval(prm, nin, H, ap)[0][0] - orc.mlp_eval(prm, nin, H, am)[0][0]) / (2 * eps)
            assert abs(fd - g[s, c]) < 1e-7 * max(1.0, abs(fd)), (s, c, fd, g[s, c])


@pytest.mark.parametrize("nin,H", [(3, 8), (7, 64)])
def test_mlp_loss_gradient_vs_finite_differences(orc, nin, H):
    prm = _params(nin, H, seed=3)
    rng = np.random.default_rng(4)
    a = rng.normal(size=(40, nin))
    y = rng.normal(size=40)
    loss, g = orc.mlp_loss_grad(prm, nin, H, a, y)
    P = orc.mlp_nparams(nin, H)
    idx = list(range(P)) if P < 200 else list(rng.choice(P, 120, replace=False)) + [P - 1]
    for q in idx:
        # perturb in double through a float copy: use a step well above float32 rounding
        eps = 1e-3
        pp, pm = prm.astype(np.float64).copy(), prm.astype(np.float64).copy()
        pp[q] += eps
        pm[q] -= eps
        lp = orc.mlp_loss_grad(pp.astype(np.float32), nin, H, a, y)[0]
        lm = orc.mlp_loss_grad(pm.astype(np.float32), nin, H, a, y)[0]
        step = float(np.float32(pp[q])) - float(np.float32(pm[q]))
        fd = (lp - lm) / step
        assert abs(fd - g[q]) < 2e-5 * max(1.0, abs(fd)) + 1e-6, (q, fd, g[q])


def test_mlp_bf16_emulation_stays_close(orc):
    prm = _params(7, 64, seed=5)
    a = np.random.default_rng(6).normal(size=(20, 7))
    u0, g0 = orc.mlp_eval(prm, 7, 64, a)
    u1, g1 = orc.mlp_eval(prm, 7, 64, a, bf16_round=True)
    assert np.max(np.abs(u1 - u0)) < 3e-2 * (1 + np.max(np.abs(u0)))
    assert np.linalg.norm(g1 - g0) < 3e-2 * np.linalg.norm(g0)


# ---- the control in the scheme -------------------------------------------------

def _pop_disc_with_control(orc, case, control_fn, library=None, R=6):
    w = _population_case(*case)
    pop = _population(case)
    rows = CT.control_rows(w, control_fn(w))
    ys, zs = [], []
    for r in range(R):
        o = orc.Oracle(w.replace(seed=100 + r), library=library)
        o.set_control(rows)
        o.solve_full(0)
        yy, zz = [], []
        for i in range(w.N):
            y, z = o.eval(i, POP_XS)
            yy.append(y); zz.append(z[:, 0])
        ys.append(yy); zs.append(zz)
    ys, zs = np.array(ys), np.array(zs)
    worst, spread = 0.0, 0.0
    for i in range(w.N):
        yp, zp = pop(i, POP_XS[:, 0])
        for arr, ref in ((ys[:, i], yp), (zs[:, i], zp)):
            se = arr.std(0, ddof=1) / math.sqrt(R)
            worst = max(worst, float(np.max(np.abs(arr.mean(0) - ref) / (5 * se + 2e-4))))
        spread = max(spread, float(np.max(ys[:, i].std(0, ddof=1))))
    return worst, spread


@pytest.mark.parametrize("which", ["closed_form", "random"])
def test_control_leaves_the_population_limit_unchanged(orc, which):
    fn = CT.closed_form_z if which == "closed_form" else (lambda w: CT.random_smooth_z(w, seed=9))
    worst, _ = _pop_disc_with_control(orc, POP_CASES[0], fn)
    assert worst <= 1.0


def test_good_control_reduces_the_spread(orc):
    # With the exact z = s0 du/dx tabulated as the control, g(X_N) + sum f dt
    # - sum z dW is y_i(x_i) up to O(dt) terms, so the seed-to-seed spread of
    # the fitted y drops while its mean does not move.
    w = W.cos_model("v", d=1, N=10, C=8, a=2.0, M=2000, s0=0.5, lam=0.5, kap=0.5, kapz=0.0)
    xs = CT.centres(w)[2:6]
    out = {}
    for name, fn in [("plain", lambda t, X: np.zeros((len(X), 1))), ("cv", CT.closed_form_z(w))]:
        rows = CT.control_rows(w, fn)
        ys = []
        for r in range(6):
            o = orc.Oracle(w.replace(seed=100 + r))
            o.set_control(rows)
            o.solve_full(0)
            ys.append([o.eval(i, xs)[0] for i in range(w.N)])
        out[name] = np.array(ys)
    sp, sc = out["plain"].std(0, ddof=1), out["cv"].std(0, ddof=1)
    assert sc.mean() < 0.4 * sp.mean(), (sc.mean(), sp.mean())
    diff = np.abs(out["plain"].mean(0) - out["cv"].mean(0))
    assert np.all(diff < 5 * np.sqrt(sp ** 2 + sc ** 2) / math.sqrt(6) + 1e-4)


CONTROL_MUTANTS = {
    # the Z response must not see zc_i(x_i).dW_i (it correlates with dW_i)
    "z_response_includes_step_i": ("B[m * q + l] = (S1[m] - CZ[m]) * DW[m * q + l] / dt;",
                                   "B[m * q + l] = (S1[m] - CZ[m] - CI[m]) * DW[m * q + l] / dt;"),
    # the control of step j must be evaluated at X_j, not at X_{j+1}
    "control_at_next_point": ("const double cd = control_dot(C, j, j == i ? k : orc_locate(P, x), x, dw);",
                              "double xq[ORC_DMAX]; for (int l = 0; l < d; ++l) xq[l] = x[l] + P->sigma[l * q + l] * dw[l];\n"
                              "                const double cd = control_dot(C, j, orc_locate(P, xq), xq, dw);"),
}


@pytest.mark.parametrize("name", sorted(CONTROL_MUTANTS))
def test_population_pin_catches_control_mistakes(orc, tmp_path, name):
    old, new = CONTROL_MUTANTS[name]
    src = orc.source_text()
    assert src.count(old) == 1
    lib = orc.compile_variant(src.replace(old, new), str(tmp_path / f"cmut_{name}.so"))
    worst, _ = _pop_disc_with_control(orc, POP_CASES[0], CT.closed_form_z, library=lib, R=4)
    assert worst > 1.5, (name, worst)


# ---- both controls against the straight-line restatement ----------------------

def _control_mismatch(orc, n, mode):
    w = _bf_workload(BF_CASES[n])
    if mode == "own":
        control = "own"
    else:
        control = CT.control_rows(w, CT.random_smooth_z(w, seed=n + 1, scale=0.8))
    y_and_z = bf.solve(w, control)[1]
    o = orc.Oracle(w)
    if mode == "own":
        o.set_own_control()
    else:
        o.set_control(control)
    o.solve_full(1)
    x = np.random.default_rng(3).uniform(-2, 2, size=(30, w.d))
    worst = 0.0
    for i in range(w.N):
        y, z = o.eval(i, x)
        for a in range(len(x)):
            yb, zb = y_and_z(i, x[a])
            worst = max(worst, abs(y[a] - yb), float(np.max(np.abs(z[a] - zb))))
    return worst


@pytest.mark.parametrize("n", range(len(BF_CASES)))
@pytest.mark.parametrize("mode", ["rows", "own"])
def test_control_brute_force_tiny(orc, n, mode):
    # Tabulated rows (step-i term in the Y response, later terms in both) and
    # the run's own z (later terms only) on the same Philox draws as a
    # separately written restatement; with N = 2 or 3 every term is exercised.
    assert _control_mismatch(orc, n, mode) < 1e-10


def test_own_control_changes_the_fits(orc):
    # guard: the own control is not a no-op (N = 3: steps 0 and 1 see it)
    w = _bf_workload(BF_CASES[0])
    o1, o2 = orc.Oracle(w), orc.Oracle(w)
    o2.set_own_control()
    o1.solve_full(1); o2.solve_full(1)
    x = np.linspace(-1, 1, 7)[:, None]
    assert np.array_equal(o1.eval(w.N - 1, x)[0], o2.eval(w.N - 1, x)[0])   # no later step
    assert np.max(np.abs(o1.eval(0, x)[0] - o2.eval(0, x)[0])) > 1e-6


def test_own_control_leaves_the_population_limit_unchanged(orc):
    # The fitted z_j of later steps come from clouds independent of C_{i,k}, so
    # the control has zero conditional mean: the average over seeds still
    # converges to the M -> infinity limit of the plain scheme.
    w = _population_case(*POP_CASES[0])
    pop = _population(POP_CASES[0])
    R = 6
    ys, zs = [], []
    for r in range(R):
        o = orc.Oracle(w.replace(seed=200 + r))
        o.set_own_control()
        o.solve_full(0)
        ys.append([o.eval(i, POP_XS)[0] for i in range(w.N)])
        zs.append([o.eval(i, POP_XS)[1][:, 0] for i in range(w.N)])
    ys, zs = np.array(ys), np.array(zs)
    worst = 0.0
    for i in range(w.N):
        yp, zp = pop(i, POP_XS[:, 0])
        for arr, ref in ((ys[:, i], yp), (zs[:, i], zp)):
            se = arr.std(0, ddof=1) / math.sqrt(R)
            worst = max(worst, float(np.max(np.abs(arr.mean(0) - ref) / (5 * se + 2e-4))))
    assert worst <= 1.0


def test_own_control_reduces_the_spread(orc):
    # The run's fitted z approximates s0 du/dx, so subtracting its martingale
    # removes most of the response noise of the later steps: the seed-to-seed
    # spread of y_0 drops (less than with the exact z), the mean stays.
    w = W.cos_model("v", d=1, N=10, C=8, a=2.0, M=2000, s0=0.5, lam=0.5, kap=0.5, kapz=0.0)
    xs = CT.centres(w)[2:6]
    out = {}
    for name in ("plain", "own"):
        ys = []
        for r in range(6):
            o = orc.Oracle(w.replace(seed=300 + r))
            if name == "own":
                o.set_own_control()
            o.solve_full(0)
            ys.append(o.eval(0, xs)[0])
        out[name] = np.array(ys)
    sp, so = out["plain"].std(0, ddof=1), out["own"].std(0, ddof=1)
    assert so.mean() < 0.6 * sp.mean(), (so.mean(), sp.mean())
    diff = np.abs(out["plain"].mean(0) - out["own"].mean(0))
    assert np.all(diff < 5 * np.sqrt(sp ** 2 + so ** 2) / math.sqrt(6) + 1e-4)


OWN_MUTANTS = {
    # sign of the own control (still zero-mean: only the restatement sees it)
    "own_sign": ("for (int l = 0; l < q; ++l) CZ[m] += zj[l] * dw[l];",
                 "for (int l = 0; l < q; ++l) CZ[m] -= zj[l] * dw[l];"),
    # the control must leave the Z response too
    "z_response_without_control": ("for (int l = 0; l < q; ++l) B[m * q + l] = (S1[m] - CZ[m]) * DW[m * q + l] / dt;",
                                   "for (int l = 0; l < q; ++l) B[m * q + l] = S1[m] * DW[m * q + l] / dt;"),
}


@pytest.mark.parametrize("name", sorted(OWN_MUTANTS))
def test_brute_force_catches_own_control_mistakes(orc, tmp_path, name):
    old, new = OWN_MUTANTS[name]
    src = orc.source_text()
    assert src.count(old) == 1
    lib = orc.compile_variant(src.replace(old, new), str(tmp_path / f"own_{name}.so"))
    w = _bf_workload(BF_CASES[0])
    y_and_z = bf.solve(w, "own")[1]
    o = orc.Oracle(w, library=lib)
    o.set_own_control()
    o.solve_full(1)
    x = np.random.default_rng(3).uniform(-2, 2, size=(30, w.d))
    worst = 0.0
    for i in range(w.N):
        y, z = o.eval(i, x)
        for a in range(len(x)):
            yb, zb = y_and_z(i, x[a])
            worst = max(worst, abs(y[a] - yb), float(np.max(np.abs(z[a] - zb))))
    assert worst > 1e-6, (name, worst)
