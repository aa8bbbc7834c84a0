"""Oracle of the binary diagnostics (Sec. 4, the merger analysis) -- TEST INFRASTRUCTURE.

Only the test suite, the smoke check and the benchmark's CPU leg may use this module.  Plain
numpy in FP64, written from the paper's definitions:

* effective acceleration in the frame rotating about the z axis at Omega:
  g_eff = g + Omega^2 (x, y, 0)  (the centrifugal term, r the vector from the axis);
* q_s = g_eff . (x - x_s) / |x - x_s| for the stars s = 1 (accretor), 2 (donor);
* a cell belongs to the accretor if min(q_1, 0) < min(q_2, 0), to the donor if
  min(q_1, 0) > min(q_2, 0), to neither otherwise (in particular when q_1 >= 0 and q_2 >= 0);
  a cell closer to x_s than the critical radius rc_s (a quarter of the star's Roche-lobe radius)
  belongs to star s whatever q says (the accretor's radius is tested first);
* per star, with m = rho dx^3: mass M_s = sum m, the first moment sum m x, the force
  F_s = sum m g and the torque about x_s, T_s = sum (x - x_s) x m g.
  The torque on the orbit is x_1 x F_1 + x_2 x F_2.

Every floating-point step is a single IEEE operation in the order written below (numpy does not
fuse them), so a kernel that performs the same correctly rounded operations in the same order
takes the same membership decisions.
"""
import numpy as np


def membership(x, g, omega, x1, x2, rc1, rc2):
    """0 = neither, 1 = accretor, 2 = donor, for every point (x, g: (n, 3) arrays)."""
    x = np.asarray(x, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    w2 = omega * omega
    gex = g[:, 0] + w2 * x[:, 0]
    gey = g[:, 1] + w2 * x[:, 1]
    gez = g[:, 2]
    q = []
    d2s = []
    for c in (x1, x2):
        dx, dy, dz = x[:, 0] - c[0], x[:, 1] - c[1], x[:, 2] - c[2]
        d2 = (dx * dx + dy * dy) + dz * dz
        dot = (gex * dx + gey * dy) + gez * dz
        with np.errstate(invalid="ignore", divide="ignore"):
            q.append(np.where(d2 > 0.0, dot / np.sqrt(d2), 0.0))   # q = 0 at the centre itself
        d2s.append(d2)
    m1, m2 = np.minimum(q[0], 0.0), np.minimum(q[1], 0.0)
    out = np.where(m1 < m2, 1, np.where(m1 > m2, 2, 0)).astype(np.int8)
    out[d2s[1] < rc2 * rc2] = 2
    out[d2s[0] < rc1 * rc1] = 1
    return out


def star_sums(x, m, g, member, x1, x2):
    """Per star (rows 0, 1): M, sum m x (3), F (3), T about x_s (3), cell count."""
    x = np.asarray(x, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    out = np.zeros((2, 11))
    for k, c in enumerate((x1, x2)):
        sel = member == k + 1
        f = m[sel, None] * g[sel]
        out[k, 0] = m[sel].sum()
        out[k, 1:4] = (m[sel, None] * x[sel]).sum(0)
        out[k, 4:7] = f.sum(0)
        out[k, 7:10] = np.cross(x[sel] - np.asarray(c), f).sum(0)
        out[k, 10] = sel.sum()
    return out


def roche_lobe_radius(q, a):
    """Eggleton's volume-equivalent Roche-lobe radius for mass ratio q = M_star / M_other."""
    q23 = q ** (2.0 / 3.0)
    return a * 0.49 * q23 / (0.6 * q23 + np.log(1.0 + q ** (1.0 / 3.0)))


def iterate(x, m, g, omega, x1, x2, n_iter=5):
    """The diagnostics' fixed-point iteration: classify with the current centres, then move each
    centre to its star's centre of mass; the critical radii are a quarter of the point-mass Roche
    lobes of the previous iteration's masses (none in the first).  Returns the last membership,
    the last sums and the centres used."""
    x1 = np.asarray(x1, dtype=np.float64)
    x2 = np.asarray(x2, dtype=np.float64)
    rc1 = rc2 = 0.0
    for _ in range(n_iter):
        mem = membership(x, g, omega, x1, x2, rc1, rc2)
        sums = star_sums(x, m, g, mem, x1, x2)
        c1, c2 = x1, x2
        if sums[0, 0] > 0:
            x1 = sums[0, 1:4] / sums[0, 0]
        if sums[1, 0] > 0:
            x2 = sums[1, 1:4] / sums[1, 0]
        a = np.linalg.norm(x1 - x2)
        if sums[0, 0] > 0 and sums[1, 0] > 0:
            rc1 = 0.25 * roche_lobe_radius(sums[0, 0] / sums[1, 0], a)
            rc2 = 0.25 * roche_lobe_radius(sums[1, 0] / sums[0, 0], a)
    return mem, sums, c1, c2
