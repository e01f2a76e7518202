"""The batched form (many instances per launch) through the C ABI: every
instance's tables must equal those of its own single-instance solve, and
every instance must match the FP64 oracle (teacher-forced steps)."""
import numpy as np
import pytest

from paper_2407_21085_gb300 import workloads as W
from tests import controls as CT
from tests import teacher as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21085_gb300 import srmc
    return torch, srmc


def _tables(torch, s):
    t = s.srmc_table()
    w = s.w
    y = torch.empty(w.N * w.K * t["ry"], dtype=torch.float64, device="cuda")
    z = torch.empty(w.N * w.K * t["rz"], dtype=torch.float64, device="cuda")
    s.srmc_read_table(y, z)
    torch.cuda.synchronize()
    return y.cpu().numpy(), z.cpu().numpy()


def _instances():
    # a small heterogeneous mix: d = 1, 2, 3; different N, M, strata, models
    ws = W.cfg4_instances(n=12, seed=4)
    return [w.replace(cells=[max(4, c // 4) for c in w.cells], M=min(w.M, 512)) for w in ws] + [
        W.cfg3(C=3, N=3, M=256), W.logistic_paper(d=2, N=5, C=4, M=300),
        W.cfg2(C=6, N=4, M=300, kapz=0.2), W.cfg2(C=5, N=3, M=257, basis="lp0")]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_equals_single_solves(dev, mode):
    # mode 0: rounds of multi-instance launches; mode 1: one graph branch per
    # instance; mode 2: one persistent launch per kernel variant
    torch, srmc = dev
    ws = _instances()
    single = []
    for w in ws:
        s = srmc.Solver(w, block_threads=256)
        s.srmc_solve()
        single.append(_tables(torch, s))
    solvers = [srmc.Solver(w, block_threads=256) for w in ws]
    b = srmc.Batch(solvers)
    b.srmc_batch_set_mode(mode)
    assert b.srmc_batch_mode() == mode
    b.srmc_batch_solve()
    b.srmc_batch_solve()                       # graph replay
    assert b.srmc_batch_stats() == 0
    for a, s in enumerate(solvers):
        y, z = _tables(torch, s)
        assert np.array_equal(y, single[a][0]) and np.array_equal(z, single[a][1]), ws[a].name


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_instances_against_the_oracle(dev, orc, mode):
    # every batched instance against the FP64 oracle directly: teacher-forced
    # steps 0, N/2 and N-1 on up to 48 sampled strata each, at centres and
    # off-centre points, within the FP32 bound 1e-4 (1 + |v|)
    torch, srmc = dev
    ws = _instances()
    solvers = [srmc.Solver(w, block_threads=256) for w in ws]
    b = srmc.Batch(solvers)
    b.srmc_batch_set_mode(mode)
    b.srmc_batch_solve()
    torch.cuda.synchronize()
    for w, s in zip(ws, solvers):
        res = T.teacher_forced(torch, orc, s, [0, w.N // 2, w.N - 1], 48)
        T.assert_within(w, res, where=f"batched mode {mode}")


def test_full_size_batch_instances_against_the_oracle(dev, orc):
    # the first 32 instances of the 256-instance batched workload at full
    # size, solved together by the persistent strategy; the largest instance
    # of each dimension checked
    # against the oracle by teacher forcing (steps 0, N/2, N-1; 32 strata)
    torch, srmc = dev
    ws = W.cfg4_instances()[:32]
    solvers = [srmc.Solver(w) for w in ws]
    b = srmc.Batch(solvers)
    b.srmc_batch_set_mode(2)                  # the persistent strategy
    b.srmc_batch_solve()
    assert b.srmc_batch_stats() == 0
    for d in (1, 2, 3):
        a = max((r for r in range(len(ws)) if ws[r].d == d), key=lambda r: ws[r].path_steps())
        res = T.teacher_forced(torch, orc, solvers[a], [0, ws[a].N // 2, ws[a].N - 1], 32)
        print(ws[a].name, ws[a].d, ws[a].K, ws[a].N, ws[a].M, res)
        T.assert_within(ws[a], res, where="full-size batch")


def test_tuned_batch_matches_within_rounding(dev):
    torch, srmc = dev
    ws = _instances()[:8]
    ref = []
    for w in ws:
        s = srmc.Solver(w)
        s.srmc_solve()
        ref.append(_tables(torch, s))
    solvers = [srmc.Solver(w) for w in ws]
    b = srmc.Batch(solvers)
    threads = b.srmc_batch_tune()
    assert threads and all(t in (64, 128, 256) for t in threads)
    ms = b.srmc_batch_strategy_ms()                 # the tuner keeps the fastest strategy
    assert all(v > 0 for v in ms) and b.srmc_batch_mode() == int(np.argmin(ms))
    b.srmc_batch_solve()
    for a, s in enumerate(solvers):
        y, z = _tables(torch, s)
        # a different block size changes only the order of the FP32 moment sums
        assert np.max(np.abs(y - ref[a][0])) < 1e-4 * (1 + np.max(np.abs(ref[a][0])))


def test_batch_rejects_fp64(dev):
    torch, srmc = dev
    s = srmc.Solver(W.cfg1(C=4, N=2, M=64))
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Batch([s])
    assert e.value.status == 4


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_with_controls_equals_single_solves(dev, mode):
    # instances with tabulated control rows, with the run's own control (the
    # cos model without z in its driver then runs the z-evaluating variant)
    # and without control, in one batch
    torch, srmc = dev
    ws = [W.cfg2(C=6, N=4, M=300), W.cfg2(C=5, N=5, M=200), W.cfg3(C=3, N=3, M=256),
          W.logistic_paper(d=2, N=4, C=4, M=300), W.cfg2(C=4, N=3, M=128)]
    how = ["rows", "own", "own", "own", "none"]

    def make(w, h):
        s = srmc.Solver(w, block_threads=256)
        if h == "rows":
            s.srmc_set_control(CT.control_rows(w, CT.closed_form_z(w)))
        elif h == "own":
            s.srmc_set_own_control()
        return s
    single = []
    for w, h in zip(ws, how):
        s = make(w, h)
        s.srmc_solve()
        single.append(_tables(torch, s))
    solvers = [make(w, h) for w, h in zip(ws, how)]
    b = srmc.Batch(solvers)
    b.srmc_batch_set_mode(mode)
    b.srmc_batch_solve()
    for a, s in enumerate(solvers):
        y, z = _tables(torch, s)
        assert np.array_equal(y, single[a][0]) and np.array_equal(z, single[a][1]), (ws[a].name, how[a])


def test_batch_rejects_equal_probability_strata(dev):
    torch, srmc = dev
    s = srmc.Solver(W.cfg2(C=4, N=2, M=64).replace(strata="prob"))
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Batch([s])
    assert e.value.status == 4


def test_batch_rejects_exact_dynamics(dev):
    torch, srmc = dev
    s = srmc.Solver(W.cfg2(C=4, N=2, M=64).replace(theta=[1.0, 1.0], dynamics="exact"))
    with pytest.raises(srmc.SrmcError) as e:
        srmc.Batch([s])
    assert e.value.status == 4
