"""Teacher-forced step parity: the GPU's own FP64 tables of the later steps
are handed to the oracle (orc_set_rows_centred), which then fits sampled
strata of a step i from exactly the functions the GPU's fit of step i read,
so one step is compared at any depth of a full-size backward solve, not only
near the horizon.  Both sides draw the same Philox streams.

y and z are compared at the stratum centre and at 2d points a quarter cell
(half a basis unit) off the centre along each axis, so the slopes of the LP1
fits are compared as well as their intercepts.
"""
from __future__ import annotations

import numpy as np

from tests import controls as CT

TOL64 = 1e-10           # |dy| / (1 + |y|), |dz| / (1 + |z|) in the FP64 form
TOL32 = 1e-4            # the same in the FP32 form, at the stratum centres
# FP32 at the off-centre probe points: a path whose FP32 position falls on the
# other side of a cell edge than its FP64 twin changes its response by some
# delta; in the centred LP1 basis (u nearly uniform on [-1, 1], Gram ~ M
# diag(1, 1/3, ..)) that moves the intercept by ~delta/M and each slope by up to
# ~3 delta/M, so the value half a unit off the centre moves by up to
# (1 + 3/2) delta/M: 2.5 times the centre's bound.
TOL32_OFF = 2.5 * TOL32


def probe_points(w, ks):
    """[(1 + 2d) n][d]: for each stratum k of ks its centre and the points
    centre +- (unit_l / 2) e_l (a quarter cell for equal-size strata)."""
    ctr = CT.centres(w)[ks]
    unit = CT.cell_units(w)[ks]
    pts = [ctr]
    for l in range(w.d):
        for sgn in (-1.0, 1.0):
            p = ctr.copy()
            p[:, l] += sgn * unit[:, l] / 2
            pts.append(p)
    return np.concatenate(pts)


def gpu_tables(torch, s):
    """The solver's FP64 tables as device tensors [N][K][ry], [N][K][rz]."""
    t = s.srmc_table()
    w = s.w
    Y = torch.empty((w.N, w.K, t["ry"]), dtype=torch.float64, device="cuda")
    Z = torch.empty((w.N, w.K, t["rz"]), dtype=torch.float64, device="cuda")
    s.srmc_read_table(Y, Z)
    torch.cuda.synchronize()
    return Y, Z


def errors(gy, gz, ry, rz):
    """(max y error, max z error), each |d| / (1 + |reference|)."""
    if gy.size == 0:
        return 0.0, 0.0
    return (float(np.max(np.abs(gy - ry) / (1 + np.abs(ry)))),
            float(np.max(np.abs(gz - rz) / (1 + np.abs(rz)))))


def teacher_forced(torch, orc, s, steps, n_strata, seed=0, nthreads=0, control=None):
    """Compare the solved GPU solver s with the oracle at the given steps on
    n_strata sampled strata each; returns {i: (err_y, err_z, err_y_centres,
    err_z_centres)} (not asserted): the first two over all probe points, the
    last two at the centres alone.  control: the control rows [N][K][q][p]
    (centred basis) the GPU solver used, given to the oracle too."""
    w = s.w
    Y, Z = gpu_tables(torch, s)
    o = orc.Oracle(w)
    if control is not None:
        o.set_control(control)
    lo = min(steps)
    for j in range(lo + 1, w.N):
        o.set_rows_centred(j, Y[j].cpu().numpy(), Z[j].cpu().numpy())
    del Y, Z
    rng = np.random.default_rng(seed)
    out = {}
    # increasing i: a fit of step i reads rows of steps > i only, which are
    # still the GPU's (the oracle writes the sampled rows of step i itself)
    for i in sorted(set(steps)):
        ks = np.sort(rng.choice(w.K, size=min(n_strata, w.K), replace=False))
        o.fit_many(i, ks, nthreads)
        pts = probe_points(w, ks)
        centre = np.arange(len(pts)) < len(ks)
        # keep the points that lie in a fitted stratum (all of them for
        # equal-size strata; an off-centre point of an equal-probability cell
        # could leave it)
        fitted = set(int(k) for k in ks)
        keep = np.array([orc.locate(w, x) in fitted for x in pts])
        pts, centre = pts[keep], centre[keep]
        gy, gz = (t.cpu().numpy() for t in s.evaluate(i, torch.from_numpy(pts).cuda()))
        ry, rz = o.eval(i, pts)
        out[i] = errors(gy, gz, ry, rz) + errors(gy[centre], gz[centre], ry[centre], rz[centre])
    o.close()
    return out


def assert_within(w, res, where=""):
    """Centres within TOL64 / TOL32; all probe points within TOL64 (FP64) or
    TOL32_OFF (FP32: one edge flip weighs more on the slopes)."""
    tol = TOL64 if w.precision == "fp64" else TOL32
    tol_all = TOL64 if w.precision == "fp64" else TOL32_OFF
    for i, e in res.items():
        assert max(e[2], e[3]) <= tol, (where, w.name, w.precision, i, e, "centres")
        assert max(e[0], e[1]) <= tol_all, (where, w.name, w.precision, i, e, "probe points")
