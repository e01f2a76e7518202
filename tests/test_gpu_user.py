"""User models (g and f given as source, compiled at run time by NVRTC)
through the C ABI, against the oracle running the same source compiled as
plain C, and against the built-in model they restate."""
import numpy as np
import pytest

from paper_2407_21085_gb300 import workloads as W
from tests import controls as CT
from tests import user_models as U
from tests.test_gpu_parity import _check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21085_gb300 import srmc
    return torch, srmc


def _quad(d, prec, **kw):
    return W.cos_model("user", d=d, N=4, C=6 if d < 3 else 3, a=2.0, M=256, s0=0.4, lam=0.5, kap=0.4,
                       precision=prec, **kw).replace(model="user", user_source=U.QUAD, params=[0.7, -0.4])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_user_model_vs_oracle(dev, orc, prec, d):
    # every fitted step at every stratum centre (g itself, i = N, is the
    # user's function and is not evaluated by the library)
    torch, srmc = dev
    w = _quad(d, prec)
    s = srmc.Solver(w)
    s.srmc_solve()
    o = orc.Oracle(w)
    o.solve_full(0)
    x = s.centres()
    xn = x.cpu().numpy()
    for i in range(w.N):
        gy, gz = s.evaluate(i, x)
        ry, rz = o.eval(i, xn)
        _check(w, gy.cpu().numpy(), gz.cpu().numpy(), ry, rz, where=f"step {i}")
    st = s.srmc_stats()
    assert st["nonfinite"] == 0 and st["fallbacks"] == o.fallbacks == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_user_cos_matches_the_builtin_kernel(dev, prec):
    # the same arithmetic as source and built in: FP64 agrees to rounding
    # order, FP32 within the FP32 tolerance (the built-in form takes the SFU
    # cosine, the user source the libm one)
    torch, srmc = dev
    w = W.cfg2(C=8, N=5, M=512, precision=prec)
    a = srmc.Solver(w)
    b = srmc.Solver(w.replace(model="user", user_source=U.COS))
    a.srmc_solve()
    b.srmc_solve()
    x = a.centres()
    for i in range(w.N):
        (ya, za), (yb, zb) = a.evaluate(i, x), b.evaluate(i, x)
        ya, yb, za, zb = (t.cpu().numpy() for t in (ya, yb, za, zb))
        tol = 1e-11 if prec == "fp64" else 1e-4
        assert np.max(np.abs(ya - yb) / (1 + np.abs(yb))) < tol
        assert np.max(np.abs(za - zb) / (1 + np.abs(zb))) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_user_model_with_controls(dev, orc, prec):
    from tests.test_gpu_cv import _cv_parity, _own_parity
    w = _quad(2, prec)
    _cv_parity(dev, orc, w, CT.random_smooth_z(w, seed=8, scale=0.2))
    _own_parity(dev, orc, w)


def test_user_model_errors(dev):
    torch, srmc = dev
    bad = _quad(2, "fp32").replace(user_source="SRMC_USER srmc_real srmc_user_g(this is not C")
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Solver(bad)
    assert e.value.status == 1 and "user model" in str(e.value)
    s = srmc.Solver(_quad(2, "fp32"))
    s.srmc_solve()
    with pytest.raises(srmc.SrmcError) as e:
        s.closed_form_error()
    assert e.value.status == 4
    x = s.centres()
    with pytest.raises(srmc.SrmcError) as e:
        s.evaluate(s.w.N, x)
    assert e.value.status == 4
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Batch([s])
    assert e.value.status == 4
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Solver(_quad(2, "fp32").replace(strata="prob"))
    assert e.value.status == 4


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("d", [1, 2])
def test_user_dynamics_vs_oracle(dev, orc, prec, d):
    # the user's drift b(t, x) and diffusion sigma(t, x) in the Euler step
    torch, srmc = dev
    w = _quad(d, prec).replace(user_source=U.QUAD_DYN, user_dynamics=True)
    s = srmc.Solver(w)
    s.srmc_solve()
    o = orc.Oracle(w)
    o.solve_full(0)
    x = s.centres()
    xn = x.cpu().numpy()
    for i in range(w.N):
        gy, gz = s.evaluate(i, x)
        ry, rz = o.eval(i, xn)
        _check(w, gy.cpu().numpy(), gz.cpu().numpy(), ry, rz, where=f"step {i}")
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Solver(W.cfg2(C=4, N=2, M=64).replace(user_dynamics=True))    # not a user model
    assert e.value.status == 1
