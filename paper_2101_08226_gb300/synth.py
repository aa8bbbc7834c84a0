"""Seeded synthetic inputs for the gravity solve: density fields and refinement flags.

This module is shared by the CUDA path's tests and benchmark and by the oracle's tests.  It holds
no arithmetic of the multipole method itself; it only produces the inputs the method consumes:

* stellar density profiles on the unit box [-1/2, 1/2]^3 (G = 1 code units, Sec. 2.8):
  Lane-Emden polytropes (the n = 3/2 stationary star of Sec. 3.5 and the binary components of
  Sec. 4), the n = 1 polytrope and the uniform sphere of Sec. 3.4;
* the density-threshold refinement flags that define the octree of 8^3-cell subgrids
  (a subgrid is refined when its sampled maximum density exceeds a fraction of the peak; this is
  the simplified form of the density criterion of Sec. 2.7);
* the per-step multiplicative noise that emulates the per-timestep re-solve;
* splitmix64, the counter-based generator that draws the batched-tree parameters.

Geometry conventions used here (and by both solvers): a level-l subgrid with integer position
(i, j, k) in [0, 2^l)^3 covers [-1/2 + i/2^l, -1/2 + (i+1)/2^l] x ...; its 8^3 cells have width
dx_l = 1 / (8 * 2^l) and are numbered (a*8 + b)*8 + c with c (the z index) fastest.
Dense per-level flags are indexed (i * 2^l + j) * 2^l + k.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

SUBGRID_N = 8
FLOOR_DEFAULT = 1e-10


# --------------------------------------------------------------------------------------------
# Lane-Emden profiles
# --------------------------------------------------------------------------------------------
@functools.lru_cache(maxsize=8)
def lane_emden_table(n: float, h: float = 1e-4) -> Tuple[np.ndarray, float]:
    """Tabulate the Lane-Emden solution theta(xi) for index n on a uniform grid of step h.

    theta'' = -theta^n - (2/xi) theta', theta(0) = 1, theta'(0) = 0, integrated with classical RK4
    from a series start (theta ~ 1 - xi^2/6 + n xi^4/120) until theta changes sign.  Returns the
    table of theta on xi = 0, h, 2h, ... (clipped at 0 past the surface) and the surface xi_1,
    located by linear interpolation of the last step.
    """
    def rhs(xi: float, t: float, dt: float) -> Tuple[float, float]:
        return dt, -(max(t, 0.0) ** n) - 2.0 * dt / xi

    xi = h
    t = 1.0 - xi * xi / 6.0 + n * xi ** 4 / 120.0
    dt = -xi / 3.0 + n * xi ** 3 / 30.0
    vals = [1.0, t]
    while True:
        k1t, k1d = rhs(xi, t, dt)
        k2t, k2d = rhs(xi + 0.5 * h, t + 0.5 * h * k1t, dt + 0.5 * h * k1d)
        k3t, k3d = rhs(xi + 0.5 * h, t + 0.5 * h * k2t, dt + 0.5 * h * k2d)
        k4t, k4d = rhs(xi + h, t + h * k3t, dt + h * k3d)
        t_new = t + h / 6.0 * (k1t + 2 * k2t + 2 * k3t + k4t)
        dt = dt + h / 6.0 * (k1d + 2 * k2d + 2 * k3d + k4d)
        if t_new <= 0.0:
            xi1 = xi + h * t / (t - t_new)
            vals.append(0.0)
            break
        t = t_new
        xi += h
        vals.append(t)
    return np.asarray(vals, dtype=np.float64), float(xi1)


def lane_emden_theta(n: float, xi: np.ndarray) -> np.ndarray:
    """theta_n(xi) by linear interpolation of the RK4 table (0 beyond the surface)."""
    tab, xi1 = lane_emden_table(float(n))
    h = 1e-4
    xi = np.asarray(xi, dtype=np.float64)
    out = np.interp(xi / h, np.arange(tab.size, dtype=np.float64), tab, right=0.0)
    out[xi >= xi1] = 0.0
    return out


# --------------------------------------------------------------------------------------------
# Stars and fields
# --------------------------------------------------------------------------------------------
@dataclass(frozen=True)
class Star:
    """A spherically symmetric, radially non-increasing density profile.

    kind: "polytrope" (Lane-Emden index n, rho = rho_c * theta(xi_1 r / R)^n),
          "uniform" (rho = rho_c for r < R),
          "n1" (closed-form n = 1 polytrope, rho = rho_c sin(k r)/(k r), k = pi / R).
    """
    center: Tuple[float, float, float]
    radius: float
    rho_c: float
    kind: str = "polytrope"
    n: float = 1.5

    def rho_of_r(self, r: np.ndarray) -> np.ndarray:
        r = np.asarray(r, dtype=np.float64)
        if self.kind == "polytrope":
            _, xi1 = lane_emden_table(float(self.n))
            out = self.rho_c * lane_emden_theta(self.n, xi1 * r / self.radius) ** self.n
        elif self.kind == "uniform":
            out = np.where(r < self.radius, self.rho_c, 0.0)
        elif self.kind == "n1":
            kr = math.pi * r / self.radius
            with np.errstate(invalid="ignore", divide="ignore"):
                s = np.where(kr > 0, np.sin(kr) / np.where(kr > 0, kr, 1.0), 1.0)
            out = np.where(r < self.radius, self.rho_c * s, 0.0)
        else:
            raise ValueError(f"unknown star kind {self.kind!r}")
        return np.where(r < self.radius, out, 0.0)

    def rho(self, x: np.ndarray) -> np.ndarray:
        d = np.asarray(x, dtype=np.float64) - np.asarray(self.center)
        return self.rho_of_r(np.sqrt(np.einsum("...i,...i->...", d, d)))


@dataclass(frozen=True)
class Field:
    """Sum of stars on a density floor: rho = max(sum_s rho_s, floor * rho_peak)."""
    stars: Tuple[Star, ...]
    floor: float = FLOOR_DEFAULT

    @property
    def rho_peak(self) -> float:
        return max(s.rho_c for s in self.stars)

    def rho(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        tot = np.zeros(x.shape[:-1], dtype=np.float64)
        for s in self.stars:
            tot += s.rho(x)
        return np.maximum(tot, self.floor * self.rho_peak)

    def upper_bound_in_box(self, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
        """An upper bound of rho over boxes [lo, hi] (rows), from the monotone radial profiles."""
        tot = np.zeros(lo.shape[0], dtype=np.float64)
        for s in self.stars:
            c = np.asarray(s.center)
            q = np.clip(c, lo, hi)
            tot += s.rho_of_r(np.linalg.norm(q - c, axis=1))
        return np.maximum(tot, self.floor * self.rho_peak)


def binary_field(q: float, r1: float, r2: float, a: float, floor: float = FLOOR_DEFAULT,
                 n: float = 1.5, axis=(1.0, 0.0, 0.0), offset=(0.0, 0.0, 0.0)) -> Field:
    """Two equal-index polytropes along `axis` with their centre of mass at `offset` (default:
    on the x axis, centre of mass at the origin).

    The accretor (radius r1) has rho_c = 1; the donor's central density follows from the
    equal-index mass scaling M ~ rho_c R^3, so M2/M1 = q.
    """
    rc2 = q * (r1 / r2) ** 3
    u = np.asarray(axis, dtype=np.float64)
    u = u / np.linalg.norm(u)
    o = np.asarray(offset, dtype=np.float64)
    c1 = o - a * q / (1.0 + q) * u
    c2 = o + a / (1.0 + q) * u
    return Field((Star(tuple(float(v) for v in c1), r1, 1.0, "polytrope", n),
                  Star(tuple(float(v) for v in c2), r2, rc2, "polytrope", n)), floor)


def single_polytrope_field(radius: float = 0.3, center=(0.0, 0.0, 0.0), rho_c: float = 1.0,
                           floor: float = FLOOR_DEFAULT, n: float = 1.5) -> Field:
    return Field((Star(tuple(center), radius, rho_c, "polytrope", n),), floor)


def uniform_sphere_field(radius: float = 0.25, mass: float = 1.0, floor_abs: float = 1e-10,
                         center=(0.0, 0.0, 0.0)) -> Field:
    """Uniform sphere of Sec. 3.4 (R = 0.25, M = 1) on an absolute ambient density."""
    rho_s = mass / (4.0 / 3.0 * math.pi * radius ** 3)
    return Field((Star(tuple(center), radius, rho_s, "uniform"),), floor_abs / rho_s)


def n1_polytrope_field(radius: float = 0.25, rho_c: float = 1.0, floor: float = FLOOR_DEFAULT,
                       center=(0.0, 0.0, 0.0)) -> Field:
    return Field((Star(tuple(center), radius, rho_c, "n1"),), floor)


# --------------------------------------------------------------------------------------------
# Geometry of subgrids and cells (no solver arithmetic)
# --------------------------------------------------------------------------------------------
def flags_size(max_level: int) -> int:
    """Number of dense flags for levels 0 .. max_level-1."""
    return sum(8 ** l for l in range(max_level))


def flags_offset(level: int) -> int:
    return sum(8 ** l for l in range(level))


def cell_centres(level: int, ijk: np.ndarray) -> np.ndarray:
    """Cell centres of subgrids at one level; ijk (S,3) -> (S*512, 3) in canonical cell order."""
    ijk = np.asarray(ijk, dtype=np.int64).reshape(-1, 3)
    dx = 1.0 / (SUBGRID_N * (1 << level))
    a = np.arange(SUBGRID_N)
    la, lb, lc = np.meshgrid(a, a, a, indexing="ij")
    loc = np.stack([la.ravel(), lb.ravel(), lc.ravel()], axis=1)  # (512,3), c fastest
    g = ijk[:, None, :] * SUBGRID_N + loc[None, :, :]
    return (-0.5 + (g + 0.5) * dx).reshape(-1, 3)


def leaf_cell_centres(leaves: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """leaves: (S, 4) rows (level, i, j, k) in canonical leaf order -> centres (S*512,3), dx (S*512,)."""
    leaves = np.asarray(leaves, dtype=np.int64).reshape(-1, 4)
    xs = np.empty((leaves.shape[0] * 512, 3))
    dxs = np.empty(leaves.shape[0] * 512)
    for lev in np.unique(leaves[:, 0]):
        sel = np.nonzero(leaves[:, 0] == lev)[0]
        c = cell_centres(int(lev), leaves[sel, 1:]).reshape(len(sel), 512, 3)
        xs.reshape(-1, 512, 3)[sel] = c
        dxs.reshape(-1, 512)[sel] = 1.0 / (SUBGRID_N * (1 << int(lev)))
    return xs, dxs


def leaf_density(fld: Field, leaves: np.ndarray) -> np.ndarray:
    """rho point-sampled at the leaf-cell centres, in canonical leaf order."""
    x, _ = leaf_cell_centres(leaves)
    out = np.empty(x.shape[0])
    step = 1 << 22
    for s in range(0, x.shape[0], step):
        out[s:s + step] = fld.rho(x[s:s + step])
    return out


def refinement_flags(fld: Field, max_level: int, refine_frac: float, graded: bool = False) -> np.ndarray:
    """Dense flags: position p at level l (< max_level) is flagged iff the density exceeds
    refine_frac * rho_peak somewhere in the subgrid's volume.  Each star's profile is radial and
    non-increasing, so its maximum over the box is its value at the box point closest to the
    star's centre; the flag tests that maximum star by star (and the floor).  Point samples at
    coarse cell centres would miss a star that lies between them, while in an evolved field the
    coarse cells carry the mass of the finer ones.

    graded: the mass-based form of the density criterion (Sec. 2.7) -- a cell of density rho
    belongs at the deepest level l with rho > rho_r 8^(l - max_level), rho_r = refine_frac *
    rho_peak (cells of about equal mass: one level per factor 8 in density), so a level-l subgrid
    is refined iff its maximum density exceeds rho_r 8^(l + 1 - max_level)."""
    out = np.zeros(flags_size(max_level), dtype=np.uint8)
    for lev in range(max_level):
        thr = refine_frac * fld.rho_peak * (8.0 ** (lev + 1 - max_level) if graded else 1.0)
        floor_hit = fld.floor * fld.rho_peak > thr
        n = 1 << lev
        ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        ijk = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)
        lo = -0.5 + ijk / n
        hi = lo + 1.0 / n
        hit = np.full(ijk.shape[0], floor_hit)
        for st in fld.stars:
            c = np.asarray(st.center)
            q = np.clip(c, lo, hi)
            hit |= st.rho_of_r(np.linalg.norm(q - c, axis=1)) > thr
        off = flags_offset(lev)
        out[off:off + ijk.shape[0]] = hit.astype(np.uint8)
    return out


def uniform_flags(depth: int) -> np.ndarray:
    """Flags that refine everything down to `depth` (a uniform octree of 8^depth leaf subgrids)."""
    return np.ones(flags_size(depth), dtype=np.uint8)


# --------------------------------------------------------------------------------------------
# Seeded generators
# --------------------------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix64(state: int) -> Tuple[int, int]:
    """One step of splitmix64 (Steele, Lea and Flood 2014): returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state, out = splitmix64(self.state)
        return out

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] inclusive."""
        return lo + int(self.uniform() * (hi - lo + 1)) if hi > lo else lo


def perturbed_density(rho0: np.ndarray, step: int, amplitude: float = 1e-3,
                      floor_value: float = 0.0, seed_base: int = 20210120) -> np.ndarray:
    """rho_k = max(rho0 * (1 + amplitude * u), floor) with u ~ U[-1, 1] per cell, seed seed_base + step."""
    rng = np.random.Generator(np.random.PCG64(seed_base + step))
    u = rng.uniform(-1.0, 1.0, size=rho0.shape)
    return np.maximum(rho0 * (1.0 + amplitude * u), floor_value)


# --------------------------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    max_level: int
    flags: np.ndarray
    field: Field
    theta: float = 0.5
    meta: dict = field(default_factory=dict)


def workload_uniform_polytrope(depth: int = 2, theta: float = 0.5) -> Workload:
    """Uniform octree of depth `depth`; one n = 3/2 polytrope, R = 0.3, centred, on a 1e-10 floor."""
    return Workload(f"uniform_d{depth}_polytrope", depth, uniform_flags(depth),
                    single_polytrope_field(0.3), theta, {"depth": depth})


def workload_binary(levels: int = 4, q: float = 0.7, r1: float = 0.1, r2: float = 0.085,
                    a: float = 0.35, refine_frac: float = 1e-4, theta: float = 0.5,
                    axis=(1.0, 0.0, 0.0), offset=(0.0, 0.0, 0.0)) -> Workload:
    """AMR tree with `levels` refinement levels around a binary of two n = 3/2 polytropes."""
    fld = binary_field(q, r1, r2, a, axis=axis, offset=offset)
    return Workload(f"binary_q{q}_L{levels}", levels, refinement_flags(fld, levels, refine_frac),
                    fld, theta, {"q": q, "r1": r1, "r2": r2, "a": a, "refine_frac": refine_frac,
                                 "axis": tuple(axis), "offset": tuple(offset)})


def roche_lobe_radius(q: float, a: float) -> float:
    """Eggleton's volume-equivalent Roche-lobe radius of a star of mass ratio q = M_star / M_other
    at separation a (an approximation accurate to 1 % for all q)."""
    q23 = q ** (2.0 / 3.0)
    return a * 0.49 * q23 / (0.6 * q23 + math.log(1.0 + q ** (1.0 / 3.0)))


def polytrope_k(radius: float, rho_c: float, n: float = 1.5) -> float:
    """K of the Lane-Emden polytrope p = K rho^(1 + 1/n) of index n with this radius and central
    density (G = 1): R = xi_1 sqrt((n + 1) K rho_c^(1/n - 1) / (4 pi))."""
    _, xi1 = lane_emden_table(float(n))
    return 4.0 * math.pi * radius ** 2 * rho_c ** (1.0 - 1.0 / n) / ((n + 1.0) * xi1 ** 2)


def kepler_j0(m1: float, m2: float, a: float) -> float:
    """Orbital angular momentum of two point masses on a circular Kepler orbit of separation a
    (G = 1): J = m1 m2 / (m1 + m2) a^2 Omega, Omega^2 = (m1 + m2) / a^3."""
    return m1 * m2 * math.sqrt(a / (m1 + m2))


def workload_paper_binary(levels: int = 9, theta: float = 0.34, refine_frac: float = 1e-4,
                          graded: bool = False) -> Workload:
    """The merger models' binary in the paper's proportions (Sec. 4): a domain 40 code lengths wide
    mapped to the unit box, 9 refinement levels (finest spacing 1/4096 of the box), accretor 50
    finest cells across, donor of half the accretor's mass filling its Roche lobe (spherical
    stand-in of the lobe's volume-equivalent radius), separation 0.96 code lengths (6e-2 solar
    radii), theta = 0.34 as for the paper's interacting binaries.  Refinement: every subgrid whose
    volume reaches a density above refine_frac * rho_peak is refined, to the deepest level; with
    graded, one level per factor 8 in density below refine_frac * rho_peak (refinement_flags)."""
    a = 0.96 / 40.0
    q = 0.5
    r1 = 25.0 / 4096.0
    r2 = roche_lobe_radius(q, a)
    fld = binary_field(q, r1, r2, a)
    name = f"paper_binary_{'graded_' if graded else ''}L{levels}"
    return Workload(name, levels, refinement_flags(fld, levels, refine_frac, graded), fld, theta,
                    {"q": q, "r1": r1, "r2": r2, "a": a, "refine_frac": refine_frac, "graded": graded})


def workload_scf_binary(levels: int = 3, q: float = 0.5, r1: float = 0.1, a0: float = 0.45,
                        n: float = 1.5, f: float = 0.8385) -> Workload:
    """The starting model of the self-consistent-field iteration (Sec. 4.1): two n = 3/2
    polytropes of equal polytropic constant on the x axis (donor radius r1 q^(-1/3), the equal-K
    mass-radius relation of n = 3/2), mass ratio q, separation a0, density floor 1e-10 of the
    accretor's central density, refined where the density exceeds 1e-4 of the peak; f is the
    donor's Roche filling factor as placed (0.8385 for these stars at this separation)."""
    fld = binary_field(q, r1, r1 * q ** (-1.0 / 3.0), a0, n=n)
    return Workload(f"scf_binary_L{levels}", levels, refinement_flags(fld, levels, 1e-4), fld, 0.5,
                    {"q": q, "r1": r1, "a0": a0, "n": n, "f": f})


def scf_inputs(w: Workload, leaves: np.ndarray):
    """(fmm_scf_params as a dict, the initial density, K0) for workload_scf_binary: prescribed
    masses = the initial stars' masses on the grid (material at x < 0 and x >= 0), J0 of the
    Kepler orbit at the initial separation, K0 of the initial accretor."""
    x, dx = leaf_cell_centres(leaves)
    rho0 = leaf_density(w.field, leaves)
    floor = w.field.floor * w.field.rho_peak
    m = rho0 * dx ** 3
    star = rho0 > floor
    M1 = float(m[star & (x[:, 0] < 0)].sum())
    M2 = float(m[star & (x[:, 0] >= 0)].sum())
    params = {"M1": M1, "M2": M2, "n": w.meta["n"], "f": w.meta["f"],
              "J0": kepler_j0(M1, M2, w.meta["a0"]), "rho_floor": floor, "theta": w.theta}
    return params, rho0, polytrope_k(w.meta["r1"], 1.0, w.meta["n"])


def workload_uniform_sphere(depth: int, theta: float = 0.5) -> Workload:
    return Workload(f"uniform_sphere_d{depth}", depth, uniform_flags(depth),
                    uniform_sphere_field(), theta, {"depth": depth})


def batched_workloads(n_trees: int = 64, seed_base: int = 20210120, theta: float = 0.5,
                      refine_frac: float = 1e-4) -> List[Workload]:
    """Independent trees of uneven depth: levels ~ U{2..5}; single or binary (50/50);
    q ~ U[0.3, 1]; a ~ U[0.25, 0.5]; R1 ~ U[0.08, 0.12], R2 = R1 q^(1/3); stars resampled when
    they overlap or leave [-0.45, 0.45]^3."""
    out = []
    for t in range(n_trees):
        g = SplitMix64(seed_base + t)
        levels = g.randint(2, 5)
        binary = g.uniform() < 0.5
        while True:
            q = g.uniform(0.3, 1.0)
            a = g.uniform(0.25, 0.5)
            r1 = g.uniform(0.08, 0.12)
            r2 = r1 * q ** (1.0 / 3.0)
            dxmax = 1.0 / (SUBGRID_N * (1 << levels))
            if not binary:
                break
            x1 = -a * q / (1.0 + q)
            x2 = a / (1.0 + q)
            if a >= r1 + r2 + dxmax and x1 - r1 >= -0.45 and x2 + r2 <= 0.45:
                break
        if binary:
            fld = binary_field(q, r1, r2, a)
        else:
            fld = single_polytrope_field(r1)
        out.append(Workload(f"tree{t}", levels, refinement_flags(fld, levels, refine_frac), fld,
                            theta, {"binary": binary, "q": q, "a": a, "r1": r1}))
    return out
