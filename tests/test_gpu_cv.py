"""GPU control-variate form through the C ABI against the FP64 oracle: both
sides receive the same control rows (tabulated from a given function by the
input generator) and the same Philox streams."""
import numpy as np
import pytest

from paper_2407_21085_gb300 import workloads as W
from tests import controls as CT
from tests import teacher as T
from tests.test_gpu_parity import _check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21085_gb300 import srmc
    return torch, srmc


def _rows(w, fn):
    """Control rows for w; for the FP32 form rounded to binary16, the form in
    which that solver keeps them, so that both sides use the same control."""
    rows = CT.control_rows(w, fn)
    if w.precision == "fp32":
        rows = rows.astype(np.float16).astype(np.float64)
    return rows


def _cv_parity(dev, orc, w, fn):
    torch, srmc = dev
    rows = _rows(w, fn)
    s = srmc.Solver(w)
    s.srmc_set_control(rows)
    s.srmc_solve()
    o = orc.Oracle(w)
    o.set_control(rows)
    o.solve_full(0)
    x = s.centres()
    xn = x.cpu().numpy()
    for i in range(w.N):
        gy, gz = s.evaluate(i, x)
        ry, rz = o.eval(i, xn)
        _check(w, gy.cpu().numpy(), gz.cpu().numpy(), ry, rz, where=f"step {i}")
    return s


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cv_cos_d2(dev, orc, prec):
    w = W.cfg2(C=12, N=6, M=384, precision=prec)
    _cv_parity(dev, orc, w, CT.closed_form_z(w))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cv_cos_d4_with_z_in_driver(dev, orc, prec):
    w = W.cfg3(C=3, N=4, M=200, precision=prec)
    _cv_parity(dev, orc, w, CT.random_smooth_z(w, seed=3))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cv_paper_logistic_d3(dev, orc, prec):
    w = W.logistic_paper(d=3, N=4, C=3, M=160, precision=prec)
    _cv_parity(dev, orc, w, CT.random_smooth_z(w, seed=4, scale=0.1))


def test_cv_d6(dev, orc):
    w = W.cos_model("d6", d=6, N=3, C=2, a=2.0, M=96, s0=0.3, lam=0.2, kap=0.5, precision="fp32")
    _cv_parity(dev, orc, w, CT.closed_form_z(w))


def test_fp32_form_rounds_rows_to_binary16(dev):
    # The FP32 form stores the rows in binary16 (round to nearest even,
    # saturating at +-65504): rows given in FP64 and the same rows rounded
    # beforehand give bit-identical solves; read_control returns the rows
    # as given.
    torch, srmc = dev
    w = W.cfg3(C=3, N=3, M=128)
    rows = CT.control_rows(w, CT.random_smooth_z(w, seed=5))
    rows[0, 0, 0, 0] = 1e6                         # saturates to 65504
    r16 = np.clip(rows, -65504, 65504).astype(np.float16).astype(np.float64)
    assert not np.array_equal(rows, r16)
    out = []
    for r in (rows, r16):
        s = srmc.Solver(w)
        s.srmc_set_control(r)
        assert np.array_equal(s.srmc_read_control(), r)
        s.srmc_solve()
        out.append([t.cpu().numpy() for t in s.evaluate(0, s.centres())])
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_clear_control_restores_the_plain_scheme(dev):
    torch, srmc = dev
    w = W.cfg2(C=8, N=5, M=256)
    plain = srmc.Solver(w)
    plain.srmc_solve()
    s = srmc.Solver(w)
    s.srmc_solve()
    s.srmc_set_control(CT.control_rows(w, CT.closed_form_z(w)))
    s.srmc_solve()                                 # graph re-captured with the control
    x = s.centres()
    yc, _ = s.evaluate(0, x)
    yp, _ = plain.evaluate(0, x)
    assert not torch.equal(yc, yp)
    s.srmc_clear_control()
    s.srmc_solve()
    y2, _ = s.evaluate(0, x)
    assert torch.equal(y2, yp)


def test_control_needs_lp1(dev):
    torch, srmc = dev
    w = W.cfg2(C=4, N=3, M=64, basis="lp0")
    s = srmc.Solver(w)
    with pytest.raises(srmc.SrmcError) as e:
        s.srmc_set_control(np.zeros((3, 16, 2, 1)))
    assert e.value.status == 4


def test_exact_control_cuts_the_spread_on_gpu(dev):
    # Across seeds, the fitted y spreads less with the exact z as control
    # (and the means agree): the variance reduction the control is for.
    torch, srmc = dev
    w0 = W.cfg2(C=16, N=10, M=1024)
    rows = CT.control_rows(w0, CT.closed_form_z(w0))
    ys = {"plain": [], "cv": []}
    for seed in range(8):
        w = w0.replace(seed=seed + 10)
        for name in ("plain", "cv"):
            s = srmc.Solver(w)
            if name == "cv":
                s.srmc_set_control(rows)
            s.srmc_solve()
            y, _ = s.evaluate(0, s.centres())
            ys[name].append(y.cpu().numpy())
    sp = np.std(np.array(ys["plain"]), axis=0, ddof=1)
    sc = np.std(np.array(ys["cv"]), axis=0, ddof=1)
    # inner strata: in the semi-infinite outer cells the tabulated control is
    # extrapolated far from the centre and helps less
    cells = np.stack(np.unravel_index(np.arange(w0.K), w0.cells[::-1]), 1)[:, ::-1]
    inner = np.all((cells > 0) & (cells < np.array(w0.cells) - 1), axis=1)
    assert np.mean(sc[inner]) < 0.4 * np.mean(sp[inner]), (np.mean(sc), np.mean(sp))
    dm = np.abs(np.mean(ys["plain"], axis=0) - np.mean(ys["cv"], axis=0))[inner]
    assert np.mean(dm) < 3 * np.mean(np.sqrt(sp ** 2 + sc ** 2)[inner]) / np.sqrt(8)


# ---- the run's own control: z_j of the later steps ----------------------------

def _own_parity(dev, orc, w):
    torch, srmc = dev
    s = srmc.Solver(w)
    s.srmc_set_own_control()
    s.srmc_solve()
    o = orc.Oracle(w)
    o.set_own_control()
    o.solve_full(0)
    x = s.centres()
    xn = x.cpu().numpy()
    for i in range(w.N):
        gy, gz = s.evaluate(i, x)
        ry, rz = o.eval(i, xn)
        _check(w, gy.cpu().numpy(), gz.cpu().numpy(), ry, rz, where=f"step {i}")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_own_control_cos_without_z_in_driver(dev, orc, prec):
    _own_parity(dev, orc, W.cfg2(C=12, N=6, M=384, precision=prec))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_own_control_with_z_in_driver(dev, orc, prec):
    _own_parity(dev, orc, W.cfg3(C=3, N=4, M=200, precision=prec))
    _own_parity(dev, orc, W.logistic_paper(d=3, N=4, C=3, M=160, precision=prec))


def test_own_control_state(dev):
    torch, srmc = dev
    w = W.cfg2(C=6, N=4, M=128)
    plain = srmc.Solver(w)
    plain.srmc_solve()
    s = srmc.Solver(w)
    s.srmc_set_control(CT.control_rows(w, CT.closed_form_z(w)))
    s.srmc_set_own_control()                       # replaces the rows
    with pytest.raises(srmc.SrmcError) as e:
        s.srmc_read_control()
    assert e.value.status == 5
    s.srmc_solve()
    y_own = s.evaluate(0, s.centres())[0]
    assert not torch.equal(y_own, plain.evaluate(0, plain.centres())[0])
    s.srmc_clear_control()
    s.srmc_solve()
    assert torch.equal(s.evaluate(0, s.centres())[0], plain.evaluate(0, plain.centres())[0])
    lp0 = srmc.Solver(W.cfg2(C=4, N=3, M=64, basis="lp0"))
    with pytest.raises(srmc.SrmcError) as e:
        lp0.srmc_set_own_control()
    assert e.value.status == 4


def test_own_control_cuts_the_spread_on_gpu(dev):
    # d = 1 (the case pinned on the oracle): the fitted z are accurate enough
    # there for the own control to remove much of the later steps' noise
    torch, srmc = dev
    w0 = W.cos_model("v", d=1, N=10, C=8, a=2.0, M=2000, s0=0.5, lam=0.5, kap=0.5, kapz=0.0)
    ys = {"plain": [], "own": []}
    for seed in range(8):
        w = w0.replace(seed=seed + 40)
        for name in ("plain", "own"):
            s = srmc.Solver(w)
            if name == "own":
                s.srmc_set_own_control()
            s.srmc_solve()
            y, _ = s.evaluate(0, s.centres())
            ys[name].append(y.cpu().numpy())
    sp = np.std(np.array(ys["plain"]), axis=0, ddof=1)
    so = np.std(np.array(ys["own"]), axis=0, ddof=1)
    cells = np.stack(np.unravel_index(np.arange(w0.K), w0.cells[::-1]), 1)[:, ::-1]
    inner = np.all((cells > 0) & (cells < np.array(w0.cells) - 1), axis=1)
    assert np.mean(so[inner]) < 0.6 * np.mean(sp[inner]), (np.mean(so[inner]), np.mean(sp[inner]))
    dm = np.abs(np.mean(ys["plain"], axis=0) - np.mean(ys["own"], axis=0))[inner]
    assert np.mean(dm) < 3 * np.mean(np.sqrt(sp ** 2 + so ** 2)[inner]) / np.sqrt(8)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_controls_on_equal_probability_strata(dev, orc, prec):
    # control rows in the centred basis of equal-probability cells (median
    # centre, quantile unit) and the run's own control
    w = W.cfg2(C=7, N=5, M=256, precision=prec).replace(strata="prob")
    _cv_parity(dev, orc, w, CT.closed_form_z(w))
    _own_parity(dev, orc, w)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_controls_with_exact_dynamics(dev, orc, prec):
    # the controls use dW_j, the first normal block of each exact step
    w = W.cfg2(C=6, N=4, M=256, precision=prec).replace(b=[0.1, 0.0], theta=[1.5, 0.5], dynamics="exact")
    _cv_parity(dev, orc, w, CT.random_smooth_z(w, seed=6))
    _own_parity(dev, orc, w)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_controls_with_non_diagonal_sigma(dev, orc, prec):
    # correlated coordinates: the controls still use dW_j, the step's increments
    w = W.cfg2(C=6, N=4, M=256, precision=prec, kapz=0.2).replace(sigma=[[0.3, 0.12], [-0.1, 0.25]])
    _cv_parity(dev, orc, w, CT.random_smooth_z(w, seed=7))
    _own_parity(dev, orc, w)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_controls_with_quadratic_polynomials(dev, orc, prec):
    w = W.cfg2(C=6, N=4, M=256, precision=prec, basis="lp2")
    _cv_parity(dev, orc, w, CT.closed_form_z(w))
    _own_parity(dev, orc, w)


def test_cfg5_learned_control_full_size_teacher_forced(dev, orc):
    # the learned control at full size, as the CV half of the benchmark runs
    # it: coarse M = 256 solve -> network trained on it -> sigma grad u_theta
    # tabulated as binary16 control rows -> M = 1024 solve on 8^6 strata.  The
    # oracle gets the same rows (read back and rounded to binary16, the form
    # the FP32 kernel reads) and the GPU's tables of the later steps, and
    # refits 128 sampled strata of steps 0, N/2 and N-1.
    torch, srmc = dev
    w = W.cfg5(M=1024)
    coarse = srmc.Solver(W.cfg5(M=256, seed=w.seed + 100))
    coarse.srmc_solve()
    net = srmc.MLP(w.d + 1, seed=1)
    net.srmc_mlp_fit(coarse, n_data=1 << 18, iters=300, batch=8192, lr=3e-3, seed=2)
    coarse.close()
    s = srmc.Solver(w)
    net.srmc_cv_tabulate(s)
    s.srmc_solve()
    net.close()
    rows = s.srmc_read_control().astype(np.float16).astype(np.float64)
    assert np.any(rows != 0)
    res = T.teacher_forced(torch, orc, s, [0, w.N // 2, w.N - 1], 128, control=rows)
    print(w.name, "learned control", {i: tuple("%.2e" % v for v in e) for i, e in res.items()})
    T.assert_within(w, res)
    s.close()
