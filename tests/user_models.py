"""User-model sources (srmc_user_g / srmc_user_f over srmc_real) for the
tests: compiled as plain C by the oracle and as CUDA by the library."""

# The cos family of the benchmarks restated as a user model: prm = {lam, kap,
# kapz, s0} (kapz unused), u = e^{lam (T - t)} cos(sum x / sqrt(d)), T = 1.
COS = r"""
SRMC_USER srmc_real srmc_user_g(const srmc_real *x, int d, const double *prm)
{
    srmc_real s = 0;
    for (int l = 0; l < d; ++l) s += x[l];
    return cos(s / sqrt((srmc_real)d));
}

SRMC_USER srmc_real srmc_user_f(srmc_real t, const srmc_real *x, srmc_real y, const srmc_real *z,
                                 int d, const double *prm)
{
    const srmc_real lam = (srmc_real)prm[0], kap = (srmc_real)prm[1], s0 = (srmc_real)prm[3];
    srmc_real s = 0;
    for (int l = 0; l < d; ++l) s += x[l];
    s = s / sqrt((srmc_real)d);
    const srmc_real u = exp(lam * ((srmc_real)1 - t)) * cos(s);
    return (lam + s0 * s0 / 2) * y + kap * (y * y - u * u);
}
"""

# A driver with z and x in it and no closed form (parity only): prm = {a, c}.
QUAD = r"""
SRMC_USER srmc_real srmc_user_g(const srmc_real *x, int d, const double *prm)
{
    srmc_real v = 0;
    for (int l = 0; l < d; ++l) v += x[l] * x[l];
    return (srmc_real)1 / ((srmc_real)1 + v);
}

SRMC_USER srmc_real srmc_user_f(srmc_real t, const srmc_real *x, srmc_real y, const srmc_real *z,
                                 int d, const double *prm)
{
    srmc_real zx = 0;
    for (int l = 0; l < d; ++l) zx += z[l] * x[l];
    return (srmc_real)prm[0] * y * ((srmc_real)1 - y) + (srmc_real)prm[1] * zx * t;
}
"""


def quad_g(x, prm):
    """QUAD's g restated in Python (for the brute-force restatement)."""
    return 1.0 / (1.0 + float(sum(v * v for v in x)))


def quad_f(t, x, y, z, prm):
    """QUAD's f restated in Python."""
    return prm[0] * y * (1.0 - y) + prm[1] * float(sum(a * b for a, b in zip(z, x))) * t


PY = {QUAD: (quad_g, quad_f)}


# QUAD with its own dynamics: a mean-reverting drift with a time-dependent
# level and a state-dependent diffusion (prm = {a, c}).
QUAD_DYN = QUAD + r"""
SRMC_USER srmc_real srmc_user_b(srmc_real t, const srmc_real *x, int l, int d, const double *prm)
{
    return -(srmc_real)0.5 * x[l] + (srmc_real)0.1 * sin(t + (srmc_real)l);
}

SRMC_USER srmc_real srmc_user_sigma(srmc_real t, const srmc_real *x, int l, int d, const double *prm)
{
    return (srmc_real)0.3 * ((srmc_real)1 + (srmc_real)0.2 * cos(x[l]));
}
"""


def quad_dyn_b(t, x, l, prm):
    import math
    return -0.5 * x[l] + 0.1 * math.sin(t + l)


def quad_dyn_sigma(t, x, l, prm):
    import math
    return 0.3 * (1.0 + 0.2 * math.cos(x[l]))


PY[QUAD_DYN] = (quad_g, quad_f, quad_dyn_b, quad_dyn_sigma)
