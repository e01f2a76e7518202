"""GPU parity of the method's primitives, called through the C ABI.

Integer and index results are compared bit for bit; floating-point ones
within bounds derived from the precision of each form."""
import math

import numpy as np
import pytest

from paper_2407_21085_gb300 import workloads as W
from tests import controls as CT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21085_gb300 import srmc
    return torch, srmc


def _u32_tensor(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.uint32).view(np.int32)).cuda()


def test_philox_bit_exact(dev, orc):
    torch, srmc = dev
    rng = np.random.default_rng(0)
    n = 20000
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    key = (0xA4093822, 0x299F31D0)
    out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    srmc.srmc_philox(_u32_tensor(torch, ctr), key, out)
    got = out.cpu().numpy().view(np.uint32)
    for a in list(range(50)) + list(rng.integers(0, n, 300)):
        assert tuple(got[a]) == orc.philox4x32_10(ctr[a], key)
    # published known answer
    one = _u32_tensor(torch, np.array([[0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]]))
    o1 = torch.empty((1, 4), dtype=torch.int32, device="cuda")
    srmc.srmc_philox(one, key, o1)
    assert list(o1.cpu().numpy().view(np.uint32)[0]) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_normals(dev, orc):
    torch, srmc = dev
    rng = np.random.default_rng(1)
    # special words, random words, and words of both tails (p < 2^-11: inside
    # the tail piece of the FP32 transform)
    words = np.concatenate([np.array([0, 1, 2, 255, 256, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 1], dtype=np.uint64),
                            rng.integers(0, 2 ** 32, 20000, dtype=np.uint64),
                            rng.integers(0, 2 ** 21, 64, dtype=np.uint64),
                            2 ** 32 - 1 - rng.integers(0, 2 ** 21, 64, dtype=np.uint64)]).astype(np.uint32)
    w_t = _u32_tensor(torch, words)
    o64 = torch.empty(len(words), dtype=torch.float64, device="cuda")
    o32 = torch.empty(len(words), dtype=torch.float32, device="cuda")
    srmc.srmc_normals(w_t, o64, o32)
    g64, g32 = o64.cpu().numpy(), o32.cpu().numpy().astype(np.float64)
    ref = np.array([orc.normal_from_word(int(v)) for v in words])
    # FP64: a few ulps of the value
    assert np.all(np.abs(g64 - ref) <= 1e-14 * np.maximum(1.0, np.abs(ref)))
    # FP32: 8 float ulps of the value plus the effect of rounding U to float
    tol = 8 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64) + 2e-7
    assert np.all(np.abs(g32 - ref) <= tol), np.max(np.abs(g32 - ref) - tol)
    # the upper half is the mirror of the lower half: xi(~w) = -xi(w)
    comp = _u32_tensor(torch, ~words)
    c64 = torch.empty(len(words), dtype=torch.float64, device="cuda")
    c32 = torch.empty(len(words), dtype=torch.float32, device="cuda")
    srmc.srmc_normals(comp, c64, c32)
    assert np.array_equal(c64.cpu().numpy(), -g64)
    assert np.array_equal(c32.cpu().numpy(), -o32.cpu().numpy())
    # FP32 words are taken in pairs (the packed form of the step kernels); a
    # single word takes the scalar form.  Both must give the same bits, for
    # central words, tail words (w >= 6 in the erfinv reduction) and pairs
    # mixing the two: the first eight words, every tail word, 40 others.
    p = (np.minimum(words, ~words).astype(np.float64) + 0.5) * 2.0 ** -32
    tail = np.nonzero(4 * p * (1 - p) <= np.exp(-6.0) * (1 + 1e-6))[0]
    pick = np.unique(np.concatenate([np.arange(8), tail, rng.integers(8, len(words), 40)]))
    assert len(tail) > 20
    bits = o32.cpu().numpy().view(np.uint32)
    one = torch.empty(1, dtype=torch.float32, device="cuda")
    for a in pick:
        srmc.srmc_normals(_u32_tensor(torch, words[a:a + 1]), None, one)
        assert one.cpu().numpy().view(np.uint32)[0] == bits[a], (int(words[a]), a)


def _edge_points(w, rng, n_random=4000):
    d = w.d
    pts = [rng.uniform(np.array(w.lo) - 1.5, np.array(w.hi) + 1.5, size=(n_random, d))]
    h = (np.array(w.hi) - np.array(w.lo)) / np.array(w.cells)
    for l in range(d):
        for c in range(0, w.cells[l] + 1):
            e = w.lo[l] + c * h[l]
            for delta in (0.0, np.spacing(max(abs(e), 1.0)), -np.spacing(max(abs(e), 1.0))):
                p = rng.uniform(np.array(w.lo), np.array(w.hi), size=(1, d))
                p[0, l] = e + delta
                pts.append(p)
    return np.concatenate(pts)


@pytest.mark.parametrize("make", [W.cfg1, W.cfg2, W.cfg3,
                                  lambda **k: W.cos_model("c5", d=6, N=4, C=8, a=3.0, M=8, s0=0.3,
                                                           lam=0.2, kap=0.5)])
def test_locate_bit_exact_fp64_and_fp32(dev, orc, make):
    torch, srmc = dev
    w = make()
    s = srmc.Solver(w.replace(M=max(w.d + 1, 8)))
    rng = np.random.default_rng(2)
    x = _edge_points(w, rng)
    k = torch.empty(len(x), dtype=torch.int64, device="cuda")
    s.srmc_locate(torch.from_numpy(x).cuda(), k)
    got = k.cpu().numpy()
    want = np.array([orc.locate(w, p) for p in x])
    assert np.array_equal(got, want)
    # FP32 decision: floor((x - lo) * r) in float on both sides
    xf = x.astype(np.float32)
    s.srmc_locate(torch.from_numpy(xf).cuda(), k)
    got32 = k.cpu().numpy()
    r = [np.float32(w.cells[l] / (w.hi[l] - w.lo[l])) for l in range(w.d)]
    stride = np.cumprod([1] + list(w.cells[:-1]))
    want32 = np.array([sum(orc.locate_dim_f32(p[l], w.lo[l], r[l], w.cells[l]) * stride[l]
                           for l in range(w.d)) for p in xf])
    assert np.array_equal(got32, want32)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_start_points(dev, orc, prec):
    torch, srmc = dev
    w = W.cfg3(precision=prec)
    s = srmc.Solver(w)
    rng = np.random.default_rng(3)
    for (i, k) in [(0, 0), (49, w.K - 1), (17, int(rng.integers(0, w.K))), (3, 1234)]:
        m0 = int(rng.integers(0, 1000))
        x = torch.empty((257, w.d), dtype=torch.float64, device="cuda")
        s.srmc_start_points(i, k, m0, x)
        got = x.cpu().numpy()
        want = np.array([orc.start_point(w, i, k, m0 + a) for a in range(257)])
        if prec == "fp64":
            assert np.allclose(got, want, rtol=1e-13, atol=1e-13)
        else:
            assert np.allclose(got, want, rtol=2e-6, atol=2e-6)
        kk = torch.empty(257, dtype=torch.int64, device="cuda")
        s.srmc_locate(x, kk)
        inside = np.mean(kk.cpu().numpy() == k)
        # single-precision draws may round onto an edge with probability ~1e-6
        assert inside == 1.0 if prec == "fp64" else inside >= 0.99


# ---- equal-probability strata (assumption HS, example ii) --------------------

def _prob_workloads():
    return [W.cfg1().replace(strata="prob", cells=[9]),
            W.cfg3(C=5, N=4).replace(strata="prob", cells=[3, 7, 5, 4])]


@pytest.mark.parametrize("n", [0, 1])
def test_prob_locate_bit_exact_fp64_and_fp32(dev, orc, n):
    # FP64: the oracle's edge scan and the kernel's CDF guess + one edge
    # comparison take the same decision everywhere, exact edges and their
    # neighbouring doubles included.  FP32: the kernel's decision equals the
    # cell of x among the edges rounded to float.
    torch, srmc = dev
    w = _prob_workloads()[n]
    s = srmc.Solver(w.replace(M=max(w.d + 1, 8)))
    rng = np.random.default_rng(7)
    pts = [rng.logistic(size=(3000, w.d)) * 1.5]
    for l in range(w.d):
        for c in range(1, w.cells[l]):
            e = orc.cell_edges(w, l, c)[0]
            for v in (e, np.nextafter(e, -np.inf), np.nextafter(e, np.inf)):
                p = rng.logistic(size=(1, w.d))
                p[0, l] = v
                pts.append(p)
    big = np.zeros((4, w.d)); big[0] = 1e300; big[1] = -1e300; big[2] = np.inf; big[3] = -np.inf
    pts.append(big)
    x = np.concatenate(pts)
    k = torch.empty(len(x), dtype=torch.int64, device="cuda")
    s.srmc_locate(torch.from_numpy(x).cuda(), k)
    assert np.array_equal(k.cpu().numpy(), np.array([orc.locate(w, p) for p in x]))
    xf = x.astype(np.float32)
    s.srmc_locate(torch.from_numpy(xf).cuda(), k)
    stride = np.cumprod([1] + list(w.cells[:-1]))
    want = np.zeros(len(xf), dtype=np.int64)
    for l in range(w.d):
        ef = np.array([np.float32(orc.cell_edges(w, l, c)[0]) for c in range(1, w.cells[l])])
        want += np.searchsorted(ef, xf[:, l], side="right") * stride[l]
    assert np.array_equal(k.cpu().numpy(), want)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_prob_start_points_and_centres(dev, orc, prec):
    torch, srmc = dev
    w = _prob_workloads()[1].replace(precision=prec)
    s = srmc.Solver(w)
    c = s.centres().cpu().numpy()
    assert np.allclose(c, CT.centres(w), rtol=1e-15, atol=1e-15)
    assert np.allclose(c, np.array([orc.stratum_centre(w, k) for k in range(w.K)]), rtol=1e-15, atol=1e-15)
    rng = np.random.default_rng(8)
    for (i, k) in [(0, 0), (3, w.K - 1), (2, int(rng.integers(0, w.K)))]:
        x = torch.empty((257, w.d), dtype=torch.float64, device="cuda")
        s.srmc_start_points(i, k, 5, x)
        want = np.array([orc.start_point(w, i, k, 5 + a) for a in range(257)])
        tol = 1e-13 if prec == "fp64" else 2e-6
        assert np.allclose(x.cpu().numpy(), want, rtol=tol, atol=tol)
