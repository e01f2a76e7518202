"""The allocation-free training entry point, srmc_mlp_fit_noalloc.

It serves callers that cannot allocate device memory while they train (a
fixed pre-reserved memory budget, device memory owned by another allocator,
loops that must not pay cudaFree's implicit synchronisation).  It must do
the same work as srmc_mlp_fit: two networks with the same initial weights,
trained on the same coarse solve with the same arguments, one through each
entry point, must end with the same weights and loss curves (up to the
summation order of the gradient atomics), call after call.  This file is
collected last so that a run stopping at the first failure has run every
other test first.
"""
import numpy as np
import pytest

from paper_2407_21085_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-3          # relative norm; the MLP tests allow 2e-2 against the oracle


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21085_gb300 import srmc
    return torch, srmc


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_noalloc_fit_matches_fit_on_two_calls_in_a_row(dev):
    torch, srmc = dev
    coarse = srmc.Solver(W.cfg2(C=16, N=8, M=256))
    coarse.srmc_solve()
    ref = srmc.MLP(3, seed=7)
    nal = srmc.MLP(3, seed=7)
    assert np.array_equal(ref.srmc_mlp_get_params(), nal.srmc_mlp_get_params())
    for seed in (21, 22):                                  # two calls in a row
        cr = torch.zeros(200, dtype=torch.float32, device="cuda")
        cn = torch.zeros(200, dtype=torch.float32, device="cuda")
        ref.srmc_mlp_fit(coarse, n_data=1 << 15, iters=200, batch=4096, lr=3e-3, seed=seed, loss_curve=cr)
        nal.srmc_mlp_fit_noalloc(coarse, n_data=1 << 15, iters=200, batch=4096, lr=3e-3, seed=seed,
                                 loss_curve=cn)
        torch.cuda.synchronize()
        pr, pn = ref.srmc_mlp_get_params(), nal.srmc_mlp_get_params()
        assert _rel(pn, pr) < TOL, (seed, _rel(pn, pr))
        assert _rel(cn.cpu().numpy(), cr.cpu().numpy()) < TOL
        assert cn[-10:].mean().item() < cn[:5].mean().item()   # it trains
    # a third call without a loss curve: the losses go to the library's own slot
    # (srmc_mlp_fit) and to the scratch array's (srmc_mlp_fit_noalloc)
    ref.srmc_mlp_fit(coarse, n_data=1 << 15, iters=100, batch=4096, lr=3e-3, seed=23)
    nal.srmc_mlp_fit_noalloc(coarse, n_data=1 << 15, iters=100, batch=4096, lr=3e-3, seed=23)
    torch.cuda.synchronize()
    pr, pn = ref.srmc_mlp_get_params(), nal.srmc_mlp_get_params()
    assert _rel(pn, pr) < TOL, _rel(pn, pr)


def test_noalloc_fit_rejects_requests_beyond_its_scratch(dev):
    torch, srmc = dev
    coarse = srmc.Solver(W.cfg2(C=4, N=2, M=64))
    coarse.srmc_solve()
    net = srmc.MLP(3, seed=1)
    with pytest.raises(srmc.SrmcError) as e:
        net.srmc_mlp_fit_noalloc(coarse, n_data=1 << 19, iters=1, batch=1 << 19, lr=1e-3, seed=1)
    assert e.value.status == 1 and "scratch" in str(e.value)
    # sizes whose float count would wrap a 64-bit product are refused before any
    # arithmetic on them (and before any launch)
    for n in (1 << 60, (1 << 62) + (1 << 40)):
        with pytest.raises(srmc.SrmcError) as e:
            net.srmc_mlp_fit_noalloc(coarse, n_data=n, iters=1, batch=1 << 30, lr=1e-3, seed=1)
        assert e.value.status == 1 and "scratch" in str(e.value)
        with pytest.raises(srmc.SrmcError) as e:
            net.srmc_mlp_fit(coarse, n_data=n, iters=1, batch=1 << 30, lr=1e-3, seed=1)
        assert e.value.status == 1
