"""GPU kernels of the learned control variate through the C ABI, against the
FP64 oracle MLP that rounds to bfloat16 at the same points, and the trained
network's gain over the plain scheme."""
import math

import numpy as np
import pytest

from paper_2407_21085_gb300 import workloads as W
from tests import controls as CT
from tests.test_oracle_cv import _params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21085_gb300 import srmc
    return torch, srmc


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-30))


@pytest.mark.parametrize("nin", [2, 7, 9])
def test_mlp_eval_vs_oracle(dev, orc, nin):
    torch, srmc = dev
    prm = _params(nin, 64, seed=nin)
    net = srmc.MLP(nin)
    net.srmc_mlp_set_params(prm)
    assert np.array_equal(net.srmc_mlp_get_params(), prm)
    rng = np.random.default_rng(1)
    n = 203                                            # ragged: 12 full tiles + 11 rows
    a = rng.normal(size=(n, nin)).astype(np.float32)
    at = torch.from_numpy(a).cuda()
    u = torch.empty(n, dtype=torch.float32, device="cuda")
    g = torch.empty((n, nin), dtype=torch.float32, device="cuda")
    net.srmc_mlp_eval(at, u, g)
    ur, gr = orc.mlp_eval(prm, nin, 64, a.astype(np.float64), bf16_round=True)
    assert np.max(np.abs(u.cpu().numpy() - ur)) < 2e-3 * (1 + np.max(np.abs(ur)))
    assert _rel(g.cpu().numpy(), gr) < 1e-2
    # and close to the unrounded FP64 network (bf16 tolerance)
    u0, g0 = orc.mlp_eval(prm, nin, 64, a.astype(np.float64))
    assert _rel(u.cpu().numpy(), u0) < 3e-2 and _rel(g.cpu().numpy(), g0) < 3e-2


@pytest.mark.parametrize("nin", [3, 7])
def test_mlp_loss_gradient_vs_oracle(dev, orc, nin):
    torch, srmc = dev
    prm = _params(nin, 64, seed=10 + nin)
    net = srmc.MLP(nin)
    net.srmc_mlp_set_params(prm)
    rng = np.random.default_rng(2)
    n = 1000
    a = rng.normal(size=(n, nin)).astype(np.float32)
    y = rng.normal(size=n).astype(np.float32)
    grad = torch.zeros(net.P, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.srmc_mlp_loss_grad(torch.from_numpy(a).cuda(), torch.from_numpy(y).cuda(), grad, loss)
    lr_, gr = orc.mlp_loss_grad(prm, nin, 64, a.astype(np.float64), y.astype(np.float64), bf16_round=True)
    g = grad.cpu().numpy()
    assert abs(loss.item() - lr_) < 1e-3 * (1 + lr_)
    H = 64
    parts = {"W1": (0, H * nin), "b1": (H * nin, H * nin + H), "W2": (H * nin + H, H * nin + H + H * H),
             "b2": (H * nin + H + H * H, H * nin + 2 * H + H * H), "w3": (H * nin + 2 * H + H * H, net.P - 1),
             "b3": (net.P - 1, net.P)}
    for name, (s, e) in parts.items():
        assert _rel(g[s:e], gr[s:e]) < 2e-2, (name, _rel(g[s:e], gr[s:e]))


@pytest.mark.parametrize("strata", ["size", "prob"])
def test_tabulated_control_rows_vs_oracle(dev, orc, strata):
    # Control rows from the network on the GPU vs the same rows computed from
    # the oracle's network at the same points (basis centre, +- half a basis
    # unit per axis: h/4 for equal-size cells).
    torch, srmc = dev
    w = W.cos_model("tab", d=3, N=4, C=3, a=2.0, M=64, s0=0.35, lam=0.2, kap=0.5).replace(strata=strata)
    prm = _params(4, 64, seed=21)
    net = srmc.MLP(4)
    net.srmc_mlp_set_params(prm)
    s = srmc.Solver(w)
    net.srmc_cv_tabulate(s)
    got = s.srmc_read_control()

    def fn(t, X):
        A = np.column_stack([np.full(len(X), np.float32(t)), X]).astype(np.float32).astype(np.float64)
        _, g = orc.mlp_eval(prm, 4, 64, A, bf16_round=True)
        return 0.35 * g[:, 1:]
    want = CT.control_rows(w, fn)
    assert _rel(got, want) < 2e-2, _rel(got, want)


def test_fit_reduces_the_loss(dev):
    torch, srmc = dev
    w = W.cfg2(C=16, N=8, M=256)
    coarse = srmc.Solver(w)
    coarse.srmc_solve()
    net = srmc.MLP(3, seed=5)
    curve = torch.zeros(600, dtype=torch.float32, device="cuda")
    net.srmc_mlp_fit(coarse, n_data=1 << 16, iters=600, batch=4096, lr=3e-3, seed=11, loss_curve=curve)
    c = curve.cpu().numpy()
    assert np.all(np.isfinite(c))
    assert c[-50:].mean() < 0.05 * c[:5].mean(), (c[:5], c[-50:].mean())


def test_trained_control_reduces_the_spread(dev):
    # The learned control: coarse run (M = 256) -> train u_theta on (t_i, x, y_i(x))
    # -> tabulate sigma grad u_theta -> CV solves.  Across seeds the CV fits
    # spread less than the plain ones at the same M, with the same mean.
    torch, srmc = dev
    w0 = W.cfg2(C=16, N=10, M=1024)
    coarse = srmc.Solver(w0.replace(M=256, seed=999))
    coarse.srmc_solve()
    net = srmc.MLP(3, seed=3)
    net.srmc_mlp_fit(coarse, n_data=1 << 17, iters=1500, batch=8192, lr=3e-3, seed=12)
    ys = {"plain": [], "cv": []}
    for seed in range(6):
        w = w0.replace(seed=seed + 20)
        for name in ("plain", "cv"):
            s = srmc.Solver(w)
            if name == "cv":
                net.srmc_cv_tabulate(s)
            s.srmc_solve()
            y, _ = s.evaluate(0, s.centres())
            ys[name].append(y.cpu().numpy())
    sp = np.std(np.array(ys["plain"]), axis=0, ddof=1).mean()
    sc = np.std(np.array(ys["cv"]), axis=0, ddof=1).mean()
    assert sc < 0.6 * sp, (sc, sp)
    dm = np.abs(np.mean(ys["plain"], axis=0) - np.mean(ys["cv"], axis=0)).mean()
    assert dm < 3 * math.sqrt(sp ** 2 + sc ** 2) / math.sqrt(6)
