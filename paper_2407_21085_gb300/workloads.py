"""Seeded, synthetic SRMC workloads.

This module only describes inputs: the forward SDE coefficients, the model and
its parameters, the strata, the basis, M, the seed and the truncation levels.
It holds none of the scheme's arithmetic, so both the CUDA path and the CPU
oracle can be driven from it.

The BSDE family used by the benchmark workloads (the "cos" model):
    X = x + s0 W (q = d, sigma = s0 I, b = 0),
    u(t, x) = exp(lam (T - t)) cos(s),  s = sum_l x_l / sqrt(d),
    g(x) = cos(s),
    f(t, x, y, z) = (lam + s0^2/2) y + kap (y^2 - u^2)
                    + kapz (|z|^2 - s0^2 exp(2 lam (T - t)) sin^2 s),
whose exact solution is (y, z) = (u, s0 grad u) because the kap and kapz terms
vanish at the solution.  The paper's own test BSDE of Sec. 5.1 is the
"logistic" model.  The "affine" model gives exact fits for tests.
"""
from __future__ import annotations

import dataclasses
import math
import random
from dataclasses import dataclass, field
from typing import List, Optional


@dataclass
class Workload:
    name: str
    d: int
    N: int
    cells: List[int]
    lo: List[float]
    hi: List[float]
    M: int
    model: str = "cos"             # "cos" | "logistic" | "affine"
    params: List[float] = field(default_factory=list)
    q: int = 0                     # 0 -> q = d
    T: float = 1.0
    b: List[float] = field(default_factory=list)
    sigma: List[List[float]] = field(default_factory=list)
    mu: float = 1.0
    basis: str = "lp1"             # "lp0" | "lp1"
    precision: str = "fp32"        # "fp32" | "fp64"  (CUDA path only)
    seed: int = 1
    instance: int = 0
    Cy: float = 0.0                # <= 0: no truncation of y
    Cz: float = 0.0                # <= 0: no truncation of z
    strata: str = "size"           # "size": equal cells on [lo, hi); "prob": nu(H_k) = 1/K
    M_strata: Optional[List[int]] = None   # paths of each stratum (overrides M), [K]
    theta: List[float] = field(default_factory=list)   # drift b_l - theta_l x_l (empty: 0)
    dynamics: str = "euler"        # "euler" (Alg. 2) | "exact" (Alg. 1)
    user_source: Optional[str] = None   # model "user": srmc_user_g / srmc_user_f as source
    user_dynamics: bool = False    # the user source also defines srmc_user_b / srmc_user_sigma

    def __post_init__(self):
        if self.q == 0:
            self.q = self.d
        if not self.b:
            self.b = [0.0] * self.d
        if not self.sigma:
            self.sigma = [[0.0] * self.q for _ in range(self.d)]

    @property
    def K(self) -> int:
        return int(math.prod(self.cells))

    @property
    def dt(self) -> float:
        return self.T / self.N

    def path_steps(self) -> int:
        """Stratum-path-steps of one full backward solve: (sum_k M_k) N (N+1) / 2."""
        paths = sum(self.M_strata) if self.M_strata is not None else self.K * self.M
        return paths * self.N * (self.N + 1) // 2

    def replace(self, **kw) -> "Workload":
        w = dataclasses.replace(self, **kw)
        return w


def cos_model(name, d, N, C, a, M, s0, lam, kap, kapz=0.0, basis="lp1", precision="fp32",
              seed=1, instance=0, truncate=True) -> Workload:
    """Cos-family BSDE on the box [-a, a]^d cut into C cells per dimension.
    Truncation levels: C_y = 2 e^{lam T} (|u| <= e^{lam T}, so it is inactive
    at the solution) and C_z = C_y / sqrt(dt) as in the paper's a.s. bounds."""
    T = 1.0
    Cy = 2.0 * math.exp(lam * T) if truncate else 0.0
    Cz = Cy / math.sqrt(T / N) if truncate else 0.0
    sigma = [[s0 if l == r else 0.0 for r in range(d)] for l in range(d)]
    return Workload(name=name, d=d, N=N, cells=[C] * d, lo=[-a] * d, hi=[a] * d, M=M,
                    model="cos", params=[lam, kap, kapz, s0], T=T, sigma=sigma,
                    basis=basis, precision=precision, seed=seed, instance=instance,
                    Cy=Cy, Cz=Cz)


# The five workloads of the benchmark plan ----------------------------------
def cfg1(**kw) -> Workload:
    """d=1, 32 strata on [-4,4], N=10, M=1000, LP1, FP64."""
    args = dict(name="cfg1_d1_K32_N10_M1000", d=1, N=10, C=32, a=4.0, M=1000, s0=0.4,
                lam=0.5, kap=0.3, kapz=0.0, precision="fp64", instance=1)
    args.update(kw)
    return cos_model(**args)


def cfg2(**kw) -> Workload:
    """d=2, 64x64 strata on [-4,4]^2, N=20, M=4096, LP1 (LP0 variant too)."""
    args = dict(name="cfg2_d2_K4096_N20_M4096", d=2, N=20, C=64, a=4.0, M=4096, s0=0.3,
                lam=0.2, kap=0.5, kapz=0.0, precision="fp32", instance=2)
    args.update(kw)
    return cos_model(**args)


def cfg3(**kw) -> Workload:
    """d=4, 12^4 strata on [-3.5,3.5]^4, N=50, M=16384, LP1, z-term 0.2."""
    args = dict(name="cfg3_d4_K20736_N50_M16384", d=4, N=50, C=12, a=3.5, M=16384, s0=0.3,
                lam=0.2, kap=0.5, kapz=0.2, precision="fp32", instance=3)
    args.update(kw)
    return cos_model(**args)


def cfg5(**kw) -> Workload:
    """d=6, 8^6 strata on [-3,3]^6, N=40, M=4096 (plain) / 1024 (CV), LP1."""
    args = dict(name="cfg5_d6_K262144_N40_M4096", d=6, N=40, C=8, a=3.0, M=4096, s0=0.3,
                lam=0.2, kap=0.5, kapz=0.0, precision="fp32", instance=5)
    args.update(kw)
    return cos_model(**args)


def cfg4_instances(n: int = 256, seed: int = 4) -> List[Workload]:
    """The batched workload: n instances with d in {1,2,3}, 16..64 cells per
    dimension on [-4,4]^d, N in {10,20,40}, M in {1024,4096}, s0 ~ U[0.2,0.5],
    lam ~ U[0,1], kap ~ U[0,0.5], drawn from a fixed seed."""
    rng = random.Random(seed)
    out = []
    for r in range(n):
        d = rng.choice([1, 2, 3])
        if d == 1:
            C = rng.choice([16, 32, 64])
        elif d == 2:
            C = rng.choice([16, 24, 32, 48, 64])
        else:
            C = rng.choice([16, 20, 24])
        N = rng.choice([10, 20, 40])
        M = rng.choice([1024, 4096])
        s0 = rng.uniform(0.2, 0.5)
        lam = rng.uniform(0.0, 1.0)
        kap = rng.uniform(0.0, 0.5)
        out.append(cos_model(name=f"cfg4_inst{r}", d=d, N=N, C=C, a=4.0, M=M, s0=s0, lam=lam,
                             kap=kap, kapz=0.0, precision="fp32", seed=seed, instance=r))
    return out


def logistic_paper(d: int, N: int, C: int, M: int, basis="lp1", seed=1, instance=0,
                   precision="fp32") -> Workload:
    """The paper's test BSDE (Sec. 5.1): X = W, mu = 1, T = 1, strata on
    [-6.5, 6.5]^d.  g is bounded by 1 and |z_l| <= 1/4, so the truncation
    levels are set to 2 and 2 / sqrt(dt) (inactive at the solution)."""
    sigma = [[1.0 if l == r else 0.0 for r in range(d)] for l in range(d)]
    T = 1.0
    return Workload(name=f"paper_logistic_d{d}_N{N}_C{C}_M{M}", d=d, N=N, cells=[C] * d,
                    lo=[-6.5] * d, hi=[6.5] * d, M=M, model="logistic", params=[], T=T,
                    sigma=sigma, basis=basis, precision=precision, seed=seed,
                    instance=instance, Cy=2.0, Cz=2.0 / math.sqrt(T / N))


def affine(d: int, N: int, C: int, M: int, g0: float, gv, f0: float, fv, a: float,
           b=None, s0: float = 0.0, basis="lp1", precision="fp64", seed=7,
           lo=-2.0, hi=2.0) -> Workload:
    """Affine model: g(x) = g0 + gv.x, f(t,x,y,z) = f0 + fv.x + a y, constant
    drift b and diffusion s0 I, no truncation."""
    sigma = [[s0 if l == r else 0.0 for r in range(d)] for l in range(d)]
    params = [g0] + list(gv) + [f0] + list(fv) + [a]
    return Workload(name=f"affine_d{d}_N{N}", d=d, N=N, cells=[C] * d, lo=[lo] * d,
                    hi=[hi] * d, M=M, model="affine", params=params,
                    b=list(b) if b is not None else [0.0] * d, sigma=sigma, basis=basis,
                    precision=precision, seed=seed, Cy=0.0, Cz=0.0)


ALL = {"cfg1": cfg1, "cfg2": cfg2, "cfg3": cfg3, "cfg5": cfg5}
