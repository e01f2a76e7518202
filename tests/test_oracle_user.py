"""Pins of the oracle's user-model path (g and f supplied as source, compiled
as plain C): the cos family restated as a user model reproduces the built-in
model, and a model without closed form agrees with the brute-force
restatement (which evaluates the same g and f restated in Python)."""
import numpy as np

from paper_2407_21085_gb300 import workloads as W
from tests import controls as CT
from tests import brute_force as bf
from tests import user_models as U


def test_user_cos_reproduces_the_builtin_model(orc):
    w = W.cfg2(C=6, N=4, M=200, kapz=0.0, precision="fp64")
    a, b = orc.Oracle(w), orc.Oracle(w.replace(model="user", user_source=U.COS))
    a.solve_full(0)
    b.solve_full(0)
    x = CT.centres(w)
    for i in range(w.N):
        (ya, za), (yb, zb) = a.eval(i, x), b.eval(i, x)
        assert np.max(np.abs(ya - yb)) < 1e-13 and np.max(np.abs(za - zb)) < 1e-13


def test_user_model_brute_force_tiny(orc):
    for d, C, M in ((1, 3, 6), (2, 2, 7)):
        w = W.cos_model("user", d=d, N=3, C=C, a=1.0, M=M, s0=0.5, lam=0.5, kap=0.4, seed=11,
                        instance=3).replace(model="user", user_source=U.QUAD, params=[0.7, -0.4])
        y_and_z = bf.solve(w)[1]
        o = orc.Oracle(w)
        o.solve_full(1)
        x = np.random.default_rng(3).uniform(-2, 2, size=(20, d))
        worst = 0.0
        for i in range(w.N):
            y, z = o.eval(i, x)
            for a in range(len(x)):
                yb, zb = y_and_z(i, x[a])
                worst = max(worst, abs(y[a] - yb), float(np.max(np.abs(z[a] - zb))))
        assert worst < 1e-10, (d, worst)


def test_user_dynamics_brute_force_tiny(orc):
    # the user's own drift b(t, x) and diffusion sigma(t, x) in the Euler step
    for d, C, M in ((1, 3, 6), (2, 2, 7)):
        w = W.cos_model("userdyn", d=d, N=3, C=C, a=1.0, M=M, s0=0.5, lam=0.5, kap=0.4, seed=12,
                        instance=4).replace(model="user", user_source=U.QUAD_DYN, params=[0.7, -0.4],
                                            user_dynamics=True)
        y_and_z = bf.solve(w)[1]
        o = orc.Oracle(w)
        o.solve_full(1)
        x = np.random.default_rng(4).uniform(-2, 2, size=(20, d))
        worst = 0.0
        for i in range(w.N):
            y, z = o.eval(i, x)
            for a in range(len(x)):
                yb, zb = y_and_z(i, x[a])
                worst = max(worst, abs(y[a] - yb), float(np.max(np.abs(z[a] - zb))))
        assert worst < 1e-10, (d, worst)
        # the dynamics are in use: the same source without them differs
        o2 = orc.Oracle(w.replace(user_dynamics=False))
        o2.solve_full(1)
        assert np.max(np.abs(o2.eval(0, x)[0] - o.eval(0, x)[0])) > 1e-6
