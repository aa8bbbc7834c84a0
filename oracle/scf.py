"""Oracle of the self-consistent-field (SCF) iteration for a synchronously rotating binary
(Sec. 4.1, "The Initial Stellar Model") -- TEST INFRASTRUCTURE.

Only the test suite, the smoke check and the benchmark's CPU leg may use this module.  Plain numpy
in FP64 around the oracle's own gravity solve (oracle.solve), following the paper's seven steps
in their order:

  (1) scale each star's density so that it has its prescribed mass;
  (2) put the centre of mass at the centre of the rotating frame;
  (3) Omega = J0 (M1 + M2) / (M1 M2 a^2), a the separation of the stars' centres of mass;
  (4) C1 = K (1 + n) rho_1^(1/n) + phi_1 (accretor: its largest density and the effective
      potential there) and C2 = (1 - f) phi_C + f phi_L1 (donor: effective potential at its centre
      and at the inner Lagrange point L1; f the donor's Roche filling factor);
  (5) a new K from the donor's centre;
  (6) rho = ((C - phi_eff) / (K (n + 1)))^n in each star's region;
  (7) solve for the potential and repeat,

with phi_eff = phi - Omega^2 r^2 / 2 (r the distance from the rotation axis).

Readings where the text is garbled or silent (each listed with the design notes):

* phi_eff carries Omega^2: the printed "Omega r^2 / 2" lacks the square of the centrifugal
  potential of a frame rotating at Omega.
* K = (C2 - phi_C) / ((n + 1) rho_2^(1/n)): the printed C2 phi_2 / ((n + 1) rho_2^(1/n)) does not
  balance dimensionally; this is the hydrostatic relation K (1 + n) rho^(1/n) + phi_eff = C2 at
  the donor's centre.
* rho = ((C - phi_eff) / (K (n + 1)))^n where C - phi_eff > 0 (the printed phi_eff - C has the
  opposite sign of the hydrostatic relation), the atmosphere density elsewhere.
* Step (2): the rotation axis is placed through the current centre of mass (a shift of the
  frame, not of the density, which on a fixed octree would need an interpolation the paper does
  not describe).  The stars lie on the x axis, so the axis is the line parallel to z through the
  centre of mass.
* Regions: the accretor is the star material (density above the atmosphere) on the -x side of
  the plane x = x_L1, the donor on the +x side; step (6) fills a star only inside the ball about
  its centre of mass that reaches the plane of L1 (beyond the outer Lagrange points phi_eff drops
  below C again).  Steps (1)-(4) use the plane of the previous iteration.
* Centres: rho_1, phi_1 and rho_2, phi_C are taken at the cell of largest density of each star
  (the first in canonical leaf order on a tie); L1 is the cell of largest phi_eff among the leaf
  cells touching the x axis between the two centres of mass (again the first on a tie), and
  x_L1 its centre.
* The solve of step (7) comes after the mass scaling of step (1) of the next iteration, so that
  the potential of steps (2)-(6) belongs to the density they work on (one solve per iteration, as
  in the paper).  In the printed order the potential of step (4) belongs to the density before
  its rescaling; on these binaries the masses then swing by factors of 3 and the iteration
  diverges within a few steps (measured), while this order converges.
* The inputs (prescribed masses, J0, the starting K) are the caller's; the tests take J0 of the
  Kepler orbit at the initial separation and K of the initial accretor.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# the entries of the state, in the order the CUDA library stores them (fmm_scf_iterate)
STATE_KEYS = ("K", "Omega", "C1", "C2", "x_L1", "phi_L1", "X1x", "X1y", "X1z", "X2x", "X2y",
              "X2z", "Xcmx", "Xcmy", "Xcmz", "a", "M1_raw", "M2_raw", "rho1", "rho2", "phi1",
              "phiC")


@dataclass
class ScfProblem:
    x: np.ndarray          # (n, 3) leaf-cell centres, canonical leaf order
    vol: np.ndarray        # (n,) cell volumes
    axis: np.ndarray       # indices of the leaf cells touching the x axis
    M1: float              # accretor mass
    M2: float              # donor mass
    n: float               # polytropic index
    f: float               # donor Roche filling factor
    J0: float              # orbital angular momentum held fixed
    rho_floor: float       # atmosphere density


def axis_cells(x: np.ndarray, dx: np.ndarray) -> np.ndarray:
    """Leaf cells whose closure touches the x axis (|y|, |z| <= dx / 2)."""
    return np.nonzero((np.abs(x[:, 1]) <= 0.5 * dx) & (np.abs(x[:, 2]) <= 0.5 * dx))[0]


def phi_eff(P: ScfProblem, phi: np.ndarray, omega: float, xcm: np.ndarray) -> np.ndarray:
    r2 = (P.x[:, 0] - xcm[0]) ** 2 + (P.x[:, 1] - xcm[1]) ** 2
    return phi - 0.5 * omega * omega * r2


def _first_argmax(v: np.ndarray, sel: np.ndarray) -> int:
    idx = np.nonzero(sel)[0]
    return int(idx[np.argmax(v[idx])])


def l1_point(P: ScfProblem, pe: np.ndarray, X1: np.ndarray, X2: np.ndarray):
    """(x_L1, phi_eff at L1): the axis cell between the two centres with the largest phi_eff."""
    xa = P.x[P.axis, 0]
    lo, hi = min(X1[0], X2[0]), max(X1[0], X2[0])
    cand = P.axis[(xa > lo) & (xa < hi)]
    j = int(cand[np.argmax(pe[cand])])
    return float(P.x[j, 0]), float(pe[j])


def initial_state(P: ScfProblem, rho: np.ndarray, phi: np.ndarray, K0: float) -> dict:
    """The state before the first iteration: the initial density's centres, Omega of the Kepler
    orbit of the initial separation, and the L1 plane of the initial potential (the stars are
    split for it by the plane x = 0, midway in the centre-of-mass frame of the input)."""
    m = rho * P.vol
    star = rho > P.rho_floor
    r1, r2 = star & (P.x[:, 0] < 0.0), star & (P.x[:, 0] >= 0.0)
    X1 = (m[r1, None] * P.x[r1]).sum(0) / m[r1].sum()
    X2 = (m[r2, None] * P.x[r2]).sum(0) / m[r2].sum()
    xcm = (P.M1 * X1 + P.M2 * X2) / (P.M1 + P.M2)
    a = float(np.linalg.norm(X1 - X2))
    omega = float(np.sqrt((P.M1 + P.M2) / a ** 3))
    xl1, pl1 = l1_point(P, phi_eff(P, phi, omega, xcm), X1, X2)
    s = dict.fromkeys(STATE_KEYS, 0.0)
    s.update(K=K0, Omega=omega, x_L1=xl1, phi_L1=pl1, a=a)
    for k in range(3):
        s["X1" + "xyz"[k]], s["X2" + "xyz"[k]], s["Xcm" + "xyz"[k]] = X1[k], X2[k], xcm[k]
    return s


def scale_masses(P: ScfProblem, rho: np.ndarray, x_l1: float):
    """Step (1): each star's material (density above the atmosphere, on its side of the plane of
    L1) multiplied so that its mass is the prescribed one.  Returns the scaled density and the
    two masses before the scaling."""
    m = rho * P.vol
    star = rho > P.rho_floor
    reg1 = star & (P.x[:, 0] < x_l1)
    reg2 = star & (P.x[:, 0] >= x_l1)
    M1_raw, M2_raw = float(m[reg1].sum()), float(m[reg2].sum())
    out = rho.copy()
    out[reg1] *= P.M1 / M1_raw
    out[reg2] *= P.M2 / M2_raw
    return out, (M1_raw, M2_raw)


def step(P: ScfProblem, rho: np.ndarray, phi: np.ndarray, st: dict, raw=(0.0, 0.0)):
    """Steps (2)-(6) of one SCF iteration on the (mass-scaled) density rho whose potential is
    phi; raw: the masses before the scaling (kept in the state).  Returns the new density and the
    new state."""
    n = P.n
    m = rho * P.vol
    star = rho > P.rho_floor
    reg1 = star & (P.x[:, 0] < st["x_L1"])
    reg2 = star & (P.x[:, 0] >= st["x_L1"])
    # (2) the stars' centres of mass and the rotation axis through the system's
    X1 = (m[reg1, None] * P.x[reg1]).sum(0) / m[reg1].sum()
    X2 = (m[reg2, None] * P.x[reg2]).sum(0) / m[reg2].sum()
    xcm = (P.M1 * X1 + P.M2 * X2) / (P.M1 + P.M2)
    # (3) the orbital frequency at the current separation with J0 held fixed
    a = float(np.linalg.norm(X1 - X2))
    omega = P.J0 * (P.M1 + P.M2) / (P.M1 * P.M2 * a * a)
    # (4) the integration constants
    pe = phi_eff(P, phi, omega, xcm)
    i1, i2 = _first_argmax(rho, reg1), _first_argmax(rho, reg2)
    rho1, rho2 = rho[i1], rho[i2]
    phi1, phiC = pe[i1], pe[i2]
    xl1, pl1 = l1_point(P, pe, X1, X2)
    C2 = (1.0 - P.f) * phiC + P.f * pl1
    # (5) the polytropic constant from the donor's centre, which C1 takes
    K = (C2 - phiC) / ((n + 1.0) * rho2 ** (1.0 / n))
    C1 = K * (1.0 + n) * rho1 ** (1.0 / n) + phi1
    # (6) the new density, each star inside its ball up to the plane of L1
    d1, d2 = abs(xl1 - X1[0]), abs(xl1 - X2[0])
    in1 = (P.x[:, 0] < xl1) & (np.linalg.norm(P.x - X1, axis=1) < d1)
    in2 = (P.x[:, 0] >= xl1) & (np.linalg.norm(P.x - X2, axis=1) < d2)
    c = np.where(in1, C1, C2)
    h = (c - pe) / (K * (n + 1.0))
    ok = (in1 | in2) & (h > 0.0)
    new = np.full_like(rho, P.rho_floor)
    new[ok] = np.maximum(h[ok] ** n, P.rho_floor)
    out = dict(K=K, Omega=omega, C1=C1, C2=C2, x_L1=xl1, phi_L1=pl1, a=a, M1_raw=raw[0],
               M2_raw=raw[1], rho1=rho1, rho2=rho2, phi1=phi1, phiC=phiC)
    for k in range(3):
        out["X1" + "xyz"[k]], out["X2" + "xyz"[k]], out["Xcm" + "xyz"[k]] = X1[k], X2[k], xcm[k]
    return new, out


def run(tree, P: ScfProblem, rho0: np.ndarray, K0: float, n_iter: int, theta: float = 0.5):
    """The whole iteration with the oracle's own gravity solve: the initial solve, then per
    iteration the mass scaling (1), the solve (7) of the scaled density, steps (2)-(6).  Returns
    per iteration the scaled density, its potential, the new density and the state."""
    import oracle as O
    phi = O.solve(tree, rho0, theta)[0]
    st = initial_state(P, rho0, phi, K0)
    rho = rho0
    out = []
    for _ in range(n_iter):
        scaled, raw = scale_masses(P, rho, st["x_L1"])
        phi = O.solve(tree, scaled, theta)[0]
        rho, st = step(P, scaled, phi, st, raw)
        out.append({"scaled": scaled, "phi": phi, "rho": rho, "state": st})
    return st, out
