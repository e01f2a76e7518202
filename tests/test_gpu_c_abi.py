"""The C ABI from plain C: tests/c/abi_consumer.c is compiled with gcc
against include/srmc.h and libsrmc.so alone (no Python binding, no torch) and
its output is compared with the oracle on the same problem."""
import os
import subprocess

import numpy as np
import pytest

from paper_2407_21085_gb300 import workloads as W
from tests import controls as CT
from tests.test_gpu_parity import _check

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def consumer(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21085_gb300 import build
    lib = build.build()
    cuda_inc = build._cuda_include(build._nvcc())
    cuda_lib = os.path.join(os.path.dirname(cuda_inc), "lib64")
    exe = str(tmp_path_factory.mktemp("c") / "abi_consumer")
    subprocess.run(["gcc", "-O2", "-std=c11", os.path.join(ROOT, "tests", "c", "abi_consumer.c"),
                    "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, "-L", os.path.dirname(lib),
                    "-Wl,-rpath," + os.path.dirname(lib), "-lsrmc", "-L", cuda_lib, "-Wl,-rpath," + cuda_lib,
                    "-lcudart", "-lm", "-o", exe], check=True)
    return exe


def _run(consumer, d, N, C, a, M, s0, lam, kap, prec):
    r = subprocess.run([consumer] + [str(v) for v in (d, N, C, a, M, s0, lam, kap, prec)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "path-steps" in r.stderr
    return np.array([[float(v) for v in line.split()] for line in r.stdout.strip().splitlines()])


# d=2 cos model, 16x16 strata on [-4,4]^2, N=8, M=512: the reduced cfg2 problem,
# whose FP32 paths cross a cell edge differently from the FP64 ones rarely enough
# that one such crossing stays inside the FP32 tolerance (see test_gpu_parity)
CASE = dict(d=2, N=8, C=16, a=4.0, M=512, s0=0.3, lam=0.2, kap=0.5)


@pytest.mark.parametrize("prec", [64, 32])
def test_c_consumer_matches_the_oracle(consumer, orc, prec):
    c = CASE
    rows = _run(consumer, prec=prec, **c)
    w = W.cos_model("c_abi", precision="fp64" if prec == 64 else "fp32", seed=1, instance=0, **c)
    o = orc.Oracle(w)
    o.solve_full(0)
    x = CT.centres(w)
    for i in range(w.N):
        sel = rows[:, 0] == i
        assert np.array_equal(rows[sel, 1], np.arange(w.K))
        ry, rz = o.eval(i, x)
        _check(w, rows[sel, 2], rows[sel, 3:], ry, rz, where=f"C consumer step {i}")


@pytest.mark.parametrize("prec", [64, 32])
def test_c_consumer_equals_the_python_binding(consumer, prec):
    # the same library entry points on the same problem: the tables, and so
    # the printed values (17 significant digits), agree bit for bit
    import torch
    from paper_2407_21085_gb300 import srmc
    c = dict(CASE, N=4, C=8, M=300)
    rows = _run(consumer, prec=prec, **c)
    w = W.cos_model("c_abi", precision="fp64" if prec == 64 else "fp32", seed=1, instance=0, **c)
    s = srmc.Solver(w)
    s.srmc_solve()
    x = s.centres()
    for i in range(w.N):
        gy, gz = s.evaluate(i, x)
        sel = rows[:, 0] == i
        assert np.array_equal(rows[sel, 2], gy.cpu().numpy())
        assert np.array_equal(rows[sel, 3:], gz.cpu().numpy())
    torch.cuda.synchronize()
