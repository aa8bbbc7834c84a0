"""The binary of the SCF tests (Sec. 4.1): two n = 3/2 polytropes of equal polytropic constant on
the x axis, mass ratio 0.5, accretor radius 0.1 (donor 0.1 * 0.5^(-1/3), the equal-K mass-radius
relation of n = 3/2), separation 0.45, density floor 1e-10 of the accretor's central density, on
the 3-level tree refined where the density exceeds 1e-4 of the peak (75,776 leaf cells).  The
prescribed masses are the initial stars' masses on the grid, J0 that of the Kepler orbit at the
initial separation, K0 the accretor's polytropic constant, and the filling factor 0.8385, the
donor's as initially placed.  Inputs only: no step of the iteration is computed here."""
from paper_2101_08226_gb300 import synth

LEVELS, Q, R1, A0, N, F = 3, 0.5, 0.1, 0.45, 1.5, 0.8385


def workload():
    fld = synth.binary_field(Q, R1, R1 * Q ** (-1.0 / 3.0), A0)
    return fld, synth.refinement_flags(fld, LEVELS, 1e-4)


def inputs(fld, leaves):
    """(params dict of fmm_scf_params, the initial density, K0)."""
    x, dx = synth.leaf_cell_centres(leaves)
    rho0 = synth.leaf_density(fld, leaves)
    floor = fld.floor * fld.rho_peak
    m = rho0 * dx ** 3
    star = rho0 > floor
    M1 = float(m[star & (x[:, 0] < 0)].sum())
    M2 = float(m[star & (x[:, 0] >= 0)].sum())
    params = {"M1": M1, "M2": M2, "n": N, "f": F, "J0": synth.kepler_j0(M1, M2, A0),
              "rho_floor": floor, "theta": 0.5}
    return params, rho0, synth.polytrope_k(R1, 1.0, N)


def oracle_problem(params, leaves):
    from oracle import scf as S
    x, dx = synth.leaf_cell_centres(leaves)
    return S.ScfProblem(x, dx ** 3, S.axis_cells(x, dx), params["M1"], params["M2"], params["n"],
                        params["f"], params["J0"], params["rho_floor"])
