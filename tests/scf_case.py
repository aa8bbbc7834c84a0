"""The binary of the SCF tests (Sec. 4.1): synth.workload_scf_binary at 3 levels (75,776 leaf
cells) -- two n = 3/2 polytropes of equal polytropic constant, mass ratio 0.5, accretor radius
0.1, separation 0.45 -- with synth.scf_inputs (prescribed masses of the initial stars, J0 of the
Kepler orbit, K0 of the initial accretor, filling factor 0.8385).  Inputs only."""
from paper_2101_08226_gb300 import synth

LEVELS = 3
_W = synth.workload_scf_binary(LEVELS)
A0 = _W.meta["a0"]


def workload():
    return _W.field, _W.flags


def inputs(fld, leaves):
    """(params dict of fmm_scf_params, the initial density, K0)."""
    return synth.scf_inputs(_W, leaves)


def oracle_problem(params, leaves):
    from oracle import scf as S
    x, dx = synth.leaf_cell_centres(leaves)
    return S.ScfProblem(x, dx ** 3, S.axis_cells(x, dx), params["M1"], params["M2"], params["n"],
                        params["f"], params["J0"], params["rho_floor"])
