"""GPU solves through the C ABI against the FP64 CPU oracle on the same
Philox streams.

Tolerances: |dy| <= tol (1 + |y|) and |dz| <= tol (1 + |z|) (per component)
at every stratum centre and at the 2d points a quarter cell off each centre,
tol = 1e-10 in the FP64 form and 1e-4 in the FP32 form.
Full-size workloads are checked step by step at depth: the oracle refits
sampled strata of steps 0, N/2 and N-1 from the GPU's own tables of the later
steps (teacher forcing, tests/teacher.py), at centres and off-centre points."""
import math

import numpy as np
import pytest

from paper_2407_21085_gb300 import workloads as W
from tests import teacher as T

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-4


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21085_gb300 import srmc
    return torch, srmc


def _check(w, gy, gz, ry, rz, where=""):
    tol = TOL64 if w.precision == "fp64" else TOL32
    ey = np.abs(gy - ry) / (1 + np.abs(ry))
    ez = np.abs(gz - rz) / (1 + np.abs(rz))
    assert np.max(ey) <= tol and np.max(ez) <= tol, (where, np.max(ey), np.max(ez))
    return np.max(ey), np.max(ez)


def _full_parity(dev, orc, w, block_threads=0, points=None):
    # default points: every stratum's centre and the 2d points a quarter cell
    # (half a basis unit) off it along each axis, so that slopes are compared too
    torch, srmc = dev
    s = srmc.Solver(w, block_threads=block_threads)
    s.srmc_solve()
    if points is None:
        points = T.probe_points(w, np.arange(w.K))
    x = torch.from_numpy(points).cuda()
    xn = x.cpu().numpy()
    o = orc.Oracle(w)
    o.solve_full(0)
    worst = (0.0, 0.0)
    for i in range(w.N + 1):
        gy, gz = s.evaluate(i, x)
        ry, rz = o.eval(i, xn)
        e = _check(w, gy.cpu().numpy(), gz.cpu().numpy(), ry, rz, where=f"step {i}")
        worst = (max(worst[0], e[0]), max(worst[1], e[1]))
    st = s.srmc_stats()
    assert st["nonfinite"] == 0 and st["fallbacks"] == o.fallbacks == 0
    return s, worst


# ---- whole backward solves at sizes the oracle finishes in seconds ----------

def test_cfg1_full_fp64(dev, orc):
    # d=1, K=32 on [-4,4], N=10, M=1000 (ragged: 1000 = 3*256 + 232), LP1, FP64
    _full_parity(dev, orc, W.cfg1())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("basis", ["lp1", "lp0"])
def test_cfg2_family_reduced(dev, orc, prec, basis):
    # d=2 cos model (s0=0.3, lam=0.2, kap=0.5), N=8.  The FP32 paths differ
    # from the FP64 ones by rounding, so now and then a path lands on the other
    # side of a cell edge; with LP0 the fitted y jumps there by ~|grad u| h, and
    # one such path moves its stratum's z fit by ~ jump dt |dW_i| / (dt M).
    # M is chosen so that one edge flip stays inside the FP32 tolerance.
    if prec == "fp32" and basis == "lp0":
        w = W.cfg2(C=8, N=8, M=4096, precision=prec, basis=basis)
    else:
        w = W.cfg2(C=16, N=8, M=512, precision=prec, basis=basis)
    _full_parity(dev, orc, w)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cfg3_family_reduced_with_z_in_driver(dev, orc, prec):
    # d=4, kapz = 0.2 (the driver reads z_j), 4^4 strata on [-3.5,3.5]^4, N=4, M=256
    _full_parity(dev, orc, W.cfg3(C=4, N=4, M=256, precision=prec))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_active_truncation(dev, orc, prec):
    w = W.cfg2(C=8, N=6, M=300, precision=prec, kapz=0.3).replace(Cy=0.8, Cz=0.5)
    _full_parity(dev, orc, w)


@pytest.mark.parametrize("d,C,N,M", [(3, 5, 3, 96), (5, 2, 3, 64), (6, 2, 3, 128), (7, 2, 2, 40), (8, 2, 2, 64)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_other_dimensions(dev, orc, d, C, N, M, prec):
    w = W.cos_model(f"d{d}", d=d, N=N, C=C, a=2.0, M=M, s0=0.3, lam=0.2, kap=0.5, kapz=0.1,
                    precision=prec)
    _full_parity(dev, orc, w)


@pytest.mark.parametrize("d,N,M", [(9, 3, 64), (10, 2, 48), (11, 3, 40)])
@pytest.mark.parametrize("model", ["cos", "cos_z", "logistic", "logistic_lp0"])
def test_wide_dimensions(dev, orc, d, N, M, model):
    # d = 9..11 (the paper's d = 11 experiments of Sec. 5.2): FP32 form,
    # 2^d strata; the cos model with and without z in its driver, and the
    # paper's logistic model (driver sum z (y - (2 + d)/(2d))) with LP1 and LP0
    if model.startswith("logistic"):
        w = W.logistic_paper(d=d, N=N, C=2, M=M, basis="lp0" if model.endswith("lp0") else "lp1")
    else:
        w = W.cos_model(f"d{d}", d=d, N=N, C=2, a=2.0, M=M, s0=0.3, lam=0.2, kap=0.5,
                        kapz=0.1 if model == "cos_z" else 0.0)
    _full_parity(dev, orc, w)


@pytest.mark.parametrize("d,N,M", [(12, 3, 48), (15, 2, 40), (19, 3, 64)])
@pytest.mark.parametrize("model", ["cos", "cos_z", "logistic", "logistic_lp0"])
def test_dimensions_12_to_19(dev, orc, d, N, M, model):
    # d = 12..19 (the paper's Tables LP1d12 to LP1d15_19): 2 cells in the first
    # three dimensions and one (the whole line) in the others, so that the
    # oracle solves in full while every coordinate is simulated, located and
    # fitted (the kernels hold their shared memory dynamically from d = 12)
    cells = [2, 2, 2] + [1] * (d - 3)
    if model.startswith("logistic"):
        w = W.logistic_paper(d=d, N=N, C=2, M=M, basis="lp0" if model.endswith("lp0") else "lp1")
    else:
        w = W.cos_model(f"d{d}", d=d, N=N, C=2, a=2.0, M=M, s0=0.3, lam=0.2, kap=0.5,
                        kapz=0.1 if model == "cos_z" else 0.0)
    _full_parity(dev, orc, w.replace(cells=cells))


# Non-diagonal constant diffusion matrices (correlated coordinates; the Euler
# step adds sum_r sigma_lr dW_r to coordinate l): no row is proportional to
# another and none is symmetric, so a transposed or diagonal-only step fails.
SIGMA_DENSE = {
    2: [[0.3, 0.12], [-0.1, 0.25]],
    3: [[0.3, 0.1, 0.0], [0.15, 0.25, -0.08], [0.0, -0.12, 0.35]],
    6: [[0.3 if l == r else 0.05 * ((l + 2 * r) % 5 - 2) for r in range(6)] for l in range(6)],
}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["cos_z_d2", "cos_drift_d3", "logistic_d3", "affine_d2", "cos_d6", "lp0_d2"])
def test_non_diagonal_sigma(dev, orc, prec, case):
    if case == "cos_z_d2":
        w = W.cfg2(C=4, N=4, M=256, kapz=0.2)
    elif case == "cos_drift_d3":
        w = W.cos_model("d3", d=3, N=3, C=3, a=2.0, M=128, s0=0.3, lam=0.2, kap=0.5).replace(
            b=[0.1, 0.0, -0.2], theta=[0.5, 0.0, 0.0])
    elif case == "logistic_d3":
        w = W.logistic_paper(d=3, N=3, C=3, M=128)
    elif case == "affine_d2":
        w = W.affine(d=2, N=3, C=3, M=64, g0=0.5, gv=[0.3, -0.2], f0=0.1, fv=[0.05, 0.02], a=-0.3,
                     s0=0.3)
    elif case == "cos_d6":
        w = W.cos_model("d6", d=6, N=3, C=2, a=2.0, M=64, s0=0.3, lam=0.2, kap=0.5)
    else:
        w = W.cfg2(C=4, N=4, M=512, basis="lp0")
    _full_parity(dev, orc, w.replace(sigma=SIGMA_DENSE[w.d], precision=prec))


# q != d: a d x q sigma (fewer or more Brownian components than coordinates)
SIGMA_DQ = {
    (2, 1): [[0.3], [-0.2]],
    (1, 2): [[0.25, -0.2]],
    (3, 2): [[0.3, 0.05], [-0.1, 0.25], [0.08, 0.2]],
    (2, 3): [[0.25, 0.1, -0.05], [0.0, 0.2, 0.15]],
    (4, 3): [[0.3 if l == r else 0.04 * (l - r) for r in range(3)] for l in range(4)],
}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["cos_z_d2_q1", "cos_z_d1_q2", "logistic_d3_q2", "affine_d2_q3", "lp0_d4_q3"])
def test_q_not_d(dev, orc, prec, case):
    if case == "cos_z_d2_q1":
        w, dq = W.cfg2(C=4, N=4, M=256, kapz=0.2), (2, 1)
    elif case == "cos_z_d1_q2":
        w, dq = W.cfg1(C=8, N=4, M=256).replace(params=[0.5, 0.3, 0.2, 0.4]), (1, 2)
    elif case == "logistic_d3_q2":
        w, dq = W.logistic_paper(d=3, N=3, C=3, M=128), (3, 2)
    elif case == "affine_d2_q3":
        w, dq = W.affine(d=2, N=3, C=3, M=64, g0=0.5, gv=[0.3, -0.2], f0=0.1, fv=[0.05, 0.02], a=-0.3), (2, 3)
    else:
        w, dq = W.cos_model("d4", d=4, N=3, C=2, a=2.0, M=512, s0=0.3, lam=0.2, kap=0.5, basis="lp0"), (4, 3)
    _full_parity(dev, orc, w.replace(q=dq[1], sigma=SIGMA_DQ[dq], precision=prec))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_controls_with_q_not_d(dev, orc, prec):
    from tests import controls as CT
    from tests.test_gpu_cv import _cv_parity, _own_parity
    w = W.cfg2(C=6, N=4, M=256, precision=prec, kapz=0.2).replace(q=1, sigma=SIGMA_DQ[(2, 1)])
    _cv_parity(dev, orc, w, CT.random_smooth_z(w, seed=8))
    _own_parity(dev, orc, w)


def test_q_not_d_limits(dev):
    torch, srmc = dev
    w = W.cfg2(C=4, N=2, M=64).replace(q=1, sigma=SIGMA_DQ[(2, 1)])
    bad = [W.cos_model("d5", d=5, N=2, C=1, a=2.0, M=64, s0=0.3, lam=0.2, kap=0.5).replace(
               q=2, sigma=[[0.3, 0.0]] * 5),
           w.replace(b=[0.1, 0.0]),                              # the cos drift term needs q == d
           w.replace(theta=[1.0, 1.0], dynamics="exact")]
    for b in bad:
        with pytest.raises(srmc.SrmcError) as e:
            srmc.Solver(b)
        assert e.value.status == 4, b.name
    s = srmc.Solver(w)
    net = srmc.MLP(3)
    with pytest.raises(srmc.SrmcError) as e:
        net.srmc_cv_tabulate(s)
    assert e.value.status == 4
    net.close()
    s.close()


def test_non_diagonal_sigma_limits(dev):
    torch, srmc = dev
    dense = W.cfg2(C=4, N=2, M=64).replace(sigma=SIGMA_DENSE[2])
    bad = [dense.replace(theta=[1.0, 1.0], dynamics="exact"), dense.replace(strata="prob"),
           dense.replace(basis="lp2"),
           W.cos_model("d9", d=9, N=2, C=1, a=2.0, M=64, s0=0.3, lam=0.2, kap=0.5).replace(
               sigma=[[0.3 if l == r else (0.01 if r == l + 1 else 0.0) for r in range(9)] for l in range(9)])]
    for w in bad:
        with pytest.raises(srmc.SrmcError) as e:
            srmc.Solver(w)
        assert e.value.status == 4, w.name
    s = srmc.Solver(dense)
    s.srmc_solve()
    with pytest.raises(srmc.SrmcError) as e:
        s.closed_form_error()
    assert e.value.status == 4
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Batch([s])
    assert e.value.status == 4
    s.close()


def test_d19_teacher_forced(dev, orc):
    # d = 19 at the M of the paper's d = 19 row (3200 paths per stratum, dt = 0.2)
    # on 2^10 strata (2 cells in ten dimensions), with z in the driver: steps 0,
    # 2 and 4 on 64 strata.  The smooth cos model is used here: the paper's
    # logistic solution is nearly a step in sum x at d = 19, so its LP1 fits of
    # neighbouring cells differ by O(1) at a shared edge, and a single path whose
    # FP32 position falls on the other side of an edge than its FP64 twin (about
    # one in 1e8 path-steps) moves a fit by ~1e-3.  The logistic driver's own
    # code path is checked by the whole-solve parity above (small M, no flips).
    w = W.cos_model("d19", d=19, N=5, C=2, a=2.0, M=3200, s0=0.3, lam=0.2, kap=0.5,
                    kapz=0.1).replace(cells=[2] * 10 + [1] * 9)
    _deep(dev, orc, w, n_strata=64)


def test_wide_dimensions_limits(dev):
    # d >= 9: FP32, equal-size strata, Euler dynamics, no controls
    torch, srmc = dev
    w = W.cos_model("d9", d=9, N=2, C=2, a=2.0, M=64, s0=0.3, lam=0.2, kap=0.5)
    for bad in (w.replace(precision="fp64"), w.replace(strata="prob"),
                w.replace(theta=[1.0] * 9, dynamics="exact"), w.replace(basis="lp2")):
        with pytest.raises(srmc.SrmcError) as e:
            srmc.Solver(bad)
        assert e.value.status == 4
    s = srmc.Solver(w)
    for call in (s.srmc_set_own_control,
                 lambda: s.srmc_set_control(np.zeros((w.N, w.K, w.d, w.d + 1)))):
        with pytest.raises(srmc.SrmcError) as e:
            call()
        assert e.value.status == 4
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Batch([s])
    assert e.value.status == 4
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Solver(W.cos_model("d20", d=20, N=2, C=1, a=2.0, M=64, s0=0.3, lam=0.2, kap=0.5))
    assert e.value.status == 1


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uneven_cells_in_morton_order(dev, orc, prec):
    # d = 3 and 4 with different cell counts per dimension (3, 7, 5 and
    # 2, 9, 3, 4 cells on boxes of different widths): the step launches solve
    # the strata in Morton order of cells with 2, 3, 3 and 1, 4, 2, 2 bits,
    # so every stratum must still be solved once and land in its own row.
    for cells, a in (([3, 7, 5], [2.0, 3.0, 2.5]), ([2, 9, 3, 4], [1.5, 3.0, 2.0, 2.0])):
        w = W.cos_model("uneven", d=len(cells), N=3, C=2, a=2.0, M=64, s0=0.3, lam=0.2, kap=0.5,
                        kapz=0.1, precision=prec)
        w = w.replace(cells=cells, lo=[-v for v in a], hi=list(a), name=f"uneven_{len(cells)}")
        _full_parity(dev, orc, w)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_equal_probability_strata(dev, orc, prec):
    # nu(H_k) = 1/K (assumption HS, example ii): cos model in d = 1, 2, 3 (with
    # z in the driver, LP0 too) and the paper's logistic model in d = 2.
    cases = [W.cfg1(C=9, N=5, M=300).replace(strata="prob"),
             W.cfg2(C=7, N=5, M=384, kapz=0.2).replace(strata="prob"),
             W.cos_model("p3", d=3, N=3, C=4, a=1.0, M=200, s0=0.3, lam=0.2, kap=0.5,
                         kapz=0.1).replace(strata="prob", cells=[3, 5, 4]),
             W.logistic_paper(d=2, N=4, C=5, M=300).replace(strata="prob")]
    if prec == "fp64":
        cases.append(W.cfg2(C=6, N=4, M=256, basis="lp0").replace(strata="prob"))
    for w in cases:
        _full_parity(dev, orc, w.replace(precision=prec))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_per_stratum_path_counts(dev, orc, prec):
    # M_k varying with the stratum (the minimum p = 3, a ragged 257, and
    # random counts up to 600), with and without z in the driver; the path-step
    # count of the solve is sum_k M_k N (N+1) / 2.
    rng = np.random.default_rng(9)
    for w in (W.cfg2(C=6, N=4, M=300, precision=prec), W.cfg3(C=2, N=3, M=64, precision=prec)):
        Ms = rng.integers(w.d + 1, 600, size=w.K).tolist()
        Ms[0], Ms[1] = w.d + 1, 257
        w = w.replace(M_strata=Ms)
        s, _ = _full_parity(dev, orc, w)
        assert s.srmc_stats()["path_steps"] == w.path_steps()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dynamics", ["euler", "exact"])
def test_affine_drift_dynamics(dev, orc, prec, dynamics):
    # Drift b - theta x (Ornstein-Uhlenbeck) moved by the Euler scheme (Alg. 2)
    # or by the exact transition (Alg. 1, two normal blocks per step); the cos
    # model's driver then carries -(1/s0) b(x).z.  d = 1, 2 and 3 (one axis
    # without mean reversion), with z in the driver through kapz too.
    cases = [W.cfg1(C=8, N=5, M=300).replace(b=[0.3], theta=[1.2]),
             W.cfg2(C=6, N=4, M=256, kapz=0.2).replace(b=[0.1, -0.2], theta=[0.8, 2.5]),
             W.cos_model("ou3", d=3, N=3, C=3, a=2.0, M=200, s0=0.3, lam=0.2, kap=0.5)
              .replace(b=[0.0, 0.2, -0.1], theta=[0.0, 1.0, 3.0])]
    for w in cases:
        _full_parity(dev, orc, w.replace(precision=prec, dynamics=dynamics))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_quadratic_local_polynomials(dev, orc, prec):
    # LP2: [1, u, u_a u_b] in the centred coordinates, d = 1, 2, 3; cos model
    # with z in the driver, and the paper's logistic model
    cases = [W.cfg1(C=8, N=5, M=300),
             W.cfg2(C=6, N=4, M=256, kapz=0.2),
             W.cos_model("q3", d=3, N=3, C=3, a=2.0, M=300, s0=0.3, lam=0.2, kap=0.5, kapz=0.1),
             W.logistic_paper(d=2, N=4, C=4, M=300)]
    for w in cases:
        _full_parity(dev, orc, w.replace(basis="lp2", precision=prec))


def test_quadratic_local_polynomials_limits(dev):
    torch, srmc = dev
    w = W.cfg3(C=2, N=2, M=64).replace(basis="lp2")            # d = 4
    for bad in (w, W.cfg2(C=4, N=2, M=64, basis="lp2").replace(strata="prob"),
                W.cfg2(C=4, N=2, M=64, basis="lp2").replace(theta=[1.0, 1.0], dynamics="exact")):
        with pytest.raises(srmc.SrmcError) as e:
            srmc.Solver(bad)
        assert e.value.status == 4
    s = srmc.Solver(W.cfg2(C=4, N=2, M=64, basis="lp2"))
    net = srmc.MLP(3)
    with pytest.raises(srmc.SrmcError) as e:
        net.srmc_cv_tabulate(s)
    assert e.value.status == 4
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Batch([s])
    assert e.value.status == 4


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_paper_logistic_model(dev, orc, prec):
    # The test BSDE of Sec. 5.1 (driver uses sum z), d=3, strata on [-6.5,6.5]^3
    _full_parity(dev, orc, W.logistic_paper(d=3, N=4, C=3, M=200, precision=prec))


# ---- edge cases -------------------------------------------------------------

@pytest.mark.parametrize("M,bt", [(37, 32), (3, 32), (33, 64), (257, 256)])
def test_ragged_and_minimal_M(dev, orc, M, bt):
    # M not a multiple of the block, and M equal to the basis dimension (d+1 = 3)
    _full_parity(dev, orc, W.cfg2(C=4, N=3, M=M, precision="fp64"), block_threads=bt)


def test_single_stratum_and_single_step(dev, orc):
    # K = 1: one cell covering R (nu_k = nu); N = 1: only the terminal step
    _full_parity(dev, orc, W.cfg1(C=1, N=1, M=500))
    _full_parity(dev, orc, W.cfg1(C=1, N=3, M=500))


def test_block_size_does_not_change_results(dev, orc):
    torch, srmc = dev
    w = W.cfg2(C=8, N=4, M=640, precision="fp64")
    vals = []
    for bt in (32, 96, 256):
        s = srmc.Solver(w, block_threads=bt)
        s.srmc_solve()
        y, z = s.evaluate(0, s.centres())
        vals.append((y.cpu().numpy(), z.cpu().numpy()))
    for y, z in vals[1:]:
        assert np.max(np.abs(y - vals[0][0])) < 1e-12 and np.max(np.abs(z - vals[0][1])) < 1e-12


def test_deterministic(dev):
    torch, srmc = dev
    w = W.cfg2(C=16, N=6, M=1024, precision="fp32")
    out = []
    for _ in range(2):
        s = srmc.Solver(w)
        s.srmc_solve()
        t = s.srmc_table()
        y, z = s.evaluate(0, s.centres())
        out.append((y.cpu().numpy(), z.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_one_pass_equals_two_passes(dev, prec, tol):
    # A driver without z is solved in one pass over each cloud (f_i added to
    # the Y response in phase A); kapz = 1e-300 selects the z-reading kernel,
    # which regenerates the cloud for f_i after the Z fit (phase B), on a
    # driver whose z term vanishes in rounding.  Both must give the same fits.
    torch, srmc = dev
    for w in (W.cfg2(C=12, N=6, M=384, precision=prec),
              W.cfg2(C=12, N=6, M=384, precision=prec, basis="lp0"),
              W.cos_model("d6", d=6, N=3, C=2, a=2.0, M=96, s0=0.3, lam=0.2, kap=0.5, precision=prec)):
        lam, kap, _, s0 = w.params
        w2 = w.replace(params=[lam, kap, 1e-300, s0])
        a, b = srmc.Solver(w), srmc.Solver(w2)
        a.srmc_solve()
        b.srmc_solve()
        x = a.centres()
        for i in range(w.N):
            ya, za = (t.cpu().numpy() for t in a.evaluate(i, x))
            yb, zb = (t.cpu().numpy() for t in b.evaluate(i, x))
            assert np.max(np.abs(ya - yb) / (1 + np.abs(yb))) <= tol, (w.name, w.basis, i)
            assert np.max(np.abs(za - zb) / (1 + np.abs(zb))) <= tol, (w.name, w.basis, i)
        a.close()
        b.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_exact_affine_fit(dev, prec, tol):
    # sigma = 0: y_i is affine and LP1 must reproduce it (exact up to rounding)
    torch, srmc = dev
    from tests.test_oracle_scheme import _affine_truth
    gv, fv = [0.3, -0.7], [0.2, 0.05]
    w = W.affine(d=2, N=5, C=3, M=64, g0=0.4, gv=gv, f0=-0.3, fv=fv, a=0.6, b=[0.5, -0.25],
                 s0=0.0, precision=prec)
    s = srmc.Solver(w)
    s.srmc_solve()
    truth = _affine_truth(2, 5, 1.0, 0.4, gv, -0.3, fv, 0.6, [0.5, -0.25])
    x = np.random.default_rng(0).uniform(-3, 3, size=(64, 2))
    for i in range(w.N):
        y, _ = s.evaluate(i, torch.from_numpy(x).cuda())
        want = truth[i][0] + x @ truth[i][1]
        assert np.max(np.abs(y.cpu().numpy() - want)) < tol * (1 + np.max(np.abs(want)))


def test_invalid_arguments(dev):
    torch, srmc = dev
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Solver(W.cfg2(M=2))                 # M < d + 1
    assert e.value.status == 1
    bad = W.cfg2(M=64)
    bad.sigma = [[0.3, float("nan")], [0.0, 0.3]]
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Solver(bad)                         # non-finite sigma
    assert e.value.status == 1
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Solver(W.cfg2(M=64), block_threads=48)
    assert e.value.status == 1
    w4 = W.cfg2(C=2, N=2, M=64)
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Solver(w4.replace(M_strata=[64, 2, 64, 64]))   # one M_k below d + 1
    assert e.value.status == 1
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Solver(w4.replace(strata="bogus"))               # unknown strata kind
    assert e.value.status == 1
    s = srmc.Solver(W.cfg2(C=4, N=5, M=64))
    with pytest.raises(srmc.SrmcError) as e:
        s.srmc_solve_step(2)                     # steps 3, 4 not solved yet
    assert e.value.status == 5
    s.srmc_solve_step(4)
    s.srmc_solve_step(3)
    s.srmc_solve_step(2)
    empty = torch.empty((0, 2), dtype=torch.float64, device="cuda")
    y = torch.empty(0, dtype=torch.float64, device="cuda")
    s.srmc_eval(2, empty, y)                     # n = 0 is a no-op


# ---- full-size workloads: teacher-forced steps at every depth ----------------
# The GPU's own FP64 tables of the later steps are given to the oracle, which
# refits ~256 sampled strata of a step from them; compared at the centres and
# at 2d off-centre points (tests/teacher.py).  Steps 0, N/2 and N-1.

def _deep(dev, orc, w, n_strata=256, steps=None, block_threads=0):
    torch, srmc = dev
    s = srmc.Solver(w, block_threads=block_threads)
    s.srmc_solve()
    torch.cuda.synchronize()
    steps = steps if steps is not None else [0, w.N // 2, w.N - 1]
    res = T.teacher_forced(torch, orc, s, steps, n_strata)
    print(w.name, w.precision, "(y, z all points; y, z centres):",
          {i: tuple("%.2e" % v for v in e) for i, e in res.items()})
    T.assert_within(w, res)
    assert s.srmc_stats()["nonfinite"] == 0
    s.close()
    return res


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_cfg2_full_size_teacher_forced(dev, orc, prec):
    # 64x64 strata on [-4,4]^2, N=20, M=4096, LP1: the launch configuration of
    # the d = 2 benchmark line
    _deep(dev, orc, W.cfg2(precision=prec))


def test_cfg2_lp0_full_size_teacher_forced(dev, orc):
    _deep(dev, orc, W.cfg2(basis="lp0", precision="fp64"))


def test_cfg3_full_size_teacher_forced(dev, orc):
    # 12^4 strata on [-3.5,3.5]^4, N=50, M=16384, kapz=0.2 (z in the driver),
    # FP32 paths + FP64 solves
    _deep(dev, orc, W.cfg3())


def test_cfg3_shape_fp64_teacher_forced(dev, orc):
    # the all-FP64 form on cfg3's strata, N and driver with M = 1024 (the FP64
    # form runs at the GB300's FP64 rate, far below its FP32 rate)
    _deep(dev, orc, W.cfg3(M=1024, precision="fp64"), n_strata=128)


def test_cfg5_full_size_teacher_forced(dev, orc):
    # 8^6 = 262144 strata on [-3,3]^6, N = 40, M = 4096, FP32: the benchmark's
    # headline launch configuration
    _deep(dev, orc, W.cfg5())


def test_cfg2_shape_equal_probability_teacher_forced(dev, orc):
    # cfg2's launch configuration with equal-probability strata
    _deep(dev, orc, W.cfg2().replace(strata="prob"))


def test_graph_solve_equals_step_launches(dev):
    # srmc_solve replays a captured graph of the N launches; srmc_solve_step
    # launches them one by one: the tables must be identical.
    torch, srmc = dev
    w = W.cfg2(C=8, N=5, M=300)
    a = srmc.Solver(w)
    a.srmc_solve()
    a.srmc_solve()                               # a second replay of the same graph
    b = srmc.Solver(w)
    for i in range(w.N - 1, -1, -1):
        b.srmc_solve_step(i)
    t = a.srmc_table()
    ny, nz = w.N * w.K * t["ry"], w.N * w.K * t["rz"]
    ya, za = torch.empty(ny, dtype=torch.float64, device="cuda"), torch.empty(nz, dtype=torch.float64, device="cuda")
    yb, zb = torch.empty_like(ya), torch.empty_like(za)
    a.srmc_read_table(ya, za)
    b.srmc_read_table(yb, zb)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb) and torch.equal(za, zb)


def _tables(torch, s):
    t = s.srmc_table()
    w = s.w
    y = torch.empty((w.N, w.K, t["ry"]), dtype=torch.float64, device="cuda")
    z = torch.empty((w.N, w.K, t["rz"]), dtype=torch.float64, device="cuda")
    s.srmc_read_table(y, z)
    torch.cuda.synchronize()
    return y, z


def test_set_rows_teacher_forcing_on_the_gpu(dev):
    # srmc_set_rows installs another solver's rows: (1) a fresh solver given all
    # of A's rows holds A's tables bit for bit, and refitting its step i from A's
    # rows of the later steps (same precision, same streams) gives A's step i bit
    # for bit; (2) an FP32 solver given the FP64 solver's rows of the later steps
    # fits every step within the FP32 bound of the FP64 fit (teacher forcing on
    # the GPU, the per-step precision check of the bench).
    torch, srmc = dev
    w64 = W.cfg2(C=8, N=6, M=512, kapz=0.1, precision="fp64", name="cfg2_set_rows")
    a = srmc.Solver(w64)
    a.srmc_solve()
    ya, za = _tables(torch, a)
    b = srmc.Solver(w64)
    with pytest.raises(srmc.SrmcError):
        b.srmc_solve_step(0)                     # steps > 0 are neither solved nor installed
    for i in range(w64.N - 1, -1, -1):
        b.srmc_set_rows(i, ya[i], za[i])
    yb, zb = _tables(torch, b)
    assert torch.equal(ya, yb) and torch.equal(za, zb)
    for i in range(w64.N - 1, -1, -1):
        b.srmc_solve_step(i)
        yb, zb = _tables(torch, b)
        assert torch.equal(ya[i], yb[i]) and torch.equal(za[i], zb[i]), i
        b.srmc_set_rows(i, ya[i], za[i])
    c = srmc.Solver(w64.replace(precision="fp32"))
    for i in range(w64.N - 1, -1, -1):
        c.srmc_set_rows(i, ya[i], za[i])
    x = T.probe_points(w64, np.arange(w64.K))
    xt = torch.from_numpy(x).cuda()
    for i in range(w64.N - 1, -1, -1):
        c.srmc_solve_step(i)
        gy, gz = (t.cpu().numpy() for t in c.evaluate(i, xt))
        ry, rz = (t.cpu().numpy() for t in a.evaluate(i, xt))
        _check(w64.replace(precision="fp32"), gy, gz, ry, rz, where=f"step {i}")
        c.srmc_set_rows(i, ya[i], za[i])
    for s in (a, b, c):
        s.close()


@pytest.mark.parametrize("model", ["cos", "logistic"])
def test_closed_form_error_kernel(dev, model):
    # The on-device error reduction equals the same statistics computed on the
    # host from srmc_eval at the centres and the closed form of the model.
    torch, srmc = dev
    if model == "cos":
        w = W.cfg2(C=16, N=6, M=512, kapz=0.1)
    else:
        w = W.logistic_paper(d=2, N=5, C=8, M=400)
    s = srmc.Solver(w)
    s.srmc_solve()
    err = s.closed_form_error()
    x = s.centres()
    xn = x.cpu().numpy()
    for i in range(w.N):
        y, z = s.evaluate(i, x)
        y, z = y.cpu().numpy(), z.cpu().numpy()
        t = i * w.dt
        if model == "cos":
            lam, s0 = w.params[0], w.params[3]
            sv = xn.sum(1) / math.sqrt(w.d)
            u = math.exp(lam * (1 - t)) * np.cos(sv)
            zs = np.repeat((-s0 * math.exp(lam * (1 - t)) * np.sin(sv) / math.sqrt(w.d))[:, None], w.d, 1)
        else:
            om = np.exp(t + xn.sum(1))
            u = om / (1 + om)
            zs = np.repeat((om / (1 + om) ** 2)[:, None], w.d, 1)
        want = [np.max(np.abs(y - u)), np.mean((y - u) ** 2), np.max(np.abs(z - zs)),
                np.mean(np.sum((z - zs) ** 2, axis=1))]
        assert np.allclose(err[i], want, rtol=1e-9, atol=1e-14), (i, err[i], want)
    # at inner strata the fit is close to the closed form (scheme + time-discretisation
    # error); the semi-infinite outer strata are evaluated at their nominal centre
    cells = np.stack(np.unravel_index(np.arange(w.K), w.cells[::-1]), 1)[:, ::-1]
    inner = np.all((cells > 0) & (cells < np.array(w.cells) - 1), axis=1)
    y0, _ = s.evaluate(0, x)
    u0 = (math.exp(w.params[0]) * np.cos(xn.sum(1) / math.sqrt(w.d)) if model == "cos"
          else np.exp(xn.sum(1)) / (1 + np.exp(xn.sum(1))))
    assert np.max(np.abs(y0.cpu().numpy() - u0)[inner]) < 0.1


@pytest.mark.parametrize("model", ["cos", "logistic"])
def test_point_error_kernel(dev, model):
    # Sums of squared errors against the closed form at given points per step
    # (the ingredients of the indicators of Sec. 5.1, eq. mse) equal the same
    # sums on the host from srmc_eval and the closed forms; the points are
    # drawn from nu (logistic, mu = 1) like the paper's R_{i,m}, plus exact
    # cell edges and far-out points of the semi-infinite cells.
    torch, srmc = dev
    if model == "cos":
        w = W.cfg2(C=16, N=6, M=512, kapz=0.1)
    else:
        w = W.logistic_paper(d=2, N=5, C=8, M=400)
    s = srmc.Solver(w)
    s.srmc_solve()
    rng = np.random.default_rng(5)
    n = 1000
    U = rng.uniform(size=(w.N, n, w.d))
    X = np.log(U / (1 - U))
    X[:, :3] = np.array(w.lo) + (np.array(w.hi) - np.array(w.lo)) / np.array(w.cells)   # an exact edge
    X[:, 3:6] = 1e3
    xt = torch.from_numpy(X).cuda()
    out = torch.empty((w.N, 2), dtype=torch.float64, device="cuda")
    s.srmc_point_error(xt, out)
    got = out.cpu().numpy()
    for i in range(w.N):
        y, z = s.evaluate(i, xt[i].contiguous())
        y, z = y.cpu().numpy(), z.cpu().numpy()
        t, xi = i * w.dt, X[i]
        if model == "cos":
            lam, s0 = w.params[0], w.params[3]
            sv = xi.sum(1) / math.sqrt(w.d)
            u = math.exp(lam * (1 - t)) * np.cos(sv)
            zs = np.repeat((-s0 * math.exp(lam * (1 - t)) * np.sin(sv) / math.sqrt(w.d))[:, None], w.d, 1)
        else:
            om = np.exp(np.minimum(t + xi.sum(1), 700.0))
            u = om / (1 + om)
            zs = np.repeat((om / (1 + om) ** 2)[:, None], w.d, 1)
        want = [np.sum((y - u) ** 2), np.sum((z - zs) ** 2)]
        assert np.allclose(got[i], want, rtol=1e-9, atol=1e-12), (i, got[i], want)
    with pytest.raises(srmc.SrmcError):
        srmc.Solver(W.affine(d=1, N=2, C=2, M=8, g0=0, gv=[1], f0=0, fv=[0], a=0)).srmc_point_error(xt, out)
