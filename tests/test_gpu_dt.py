"""GPU parity of the time-derivative solve (Sec. 2.1: dphi/dt from the FMM with d rho/dt as the
source, on rho's expansion centres) against the oracle, and the cancellation it exists for:
sum_i s_i phi_i = sum_i m_i (dphi/dt)_i.

The source has both signs, so a cell's dphi/dt is a sum with cancellation and its rounding error
scales with the sum of the absolute terms, not with the result: the FP64 bar is per cell,
|d_i| <= 1e-12 |psi_i|, where psi is the same operator applied to |s| (computed by the oracle)."""
import numpy as np
import pytest

import oracle as O
from paper_2101_08226_gb300 import _lib, api, build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _tiny_amr():
    fl = np.zeros(synth.flags_size(3), dtype=np.uint8)
    fl[0] = 1
    fl[synth.flags_offset(1)] = 1
    fl[synth.flags_offset(2) + (1 * 4 + 1) * 4] = 1
    return 3, fl, synth.binary_field(0.7, 0.1, 0.085, 0.35)


CASES = {
    "root_only": lambda: (0, np.zeros(0, np.uint8), synth.single_polytrope_field(0.3)),
    "uniform_d2": lambda: (2, synth.uniform_flags(2), synth.single_polytrope_field(0.3)),
    "tiny_amr": _tiny_amr,
    "tilted_binary_L3": lambda: (lambda w: (w.max_level, w.flags, w.field))(
        synth.workload_binary(3, axis=(1.0, 0.6, 0.3), offset=(0.02, -0.03, 0.05))),
}


def _setup(case, seed=7):
    max_level, flags, fld = CASES[case]()
    a = api.Tree(max_level, flags)
    b = O.Tree(max_level, flags)
    assert np.array_equal(a.subgrids(), b.subgrids())
    rho = synth.leaf_density(fld, b.leaves())
    rhodot = rho * np.random.default_rng(seed).uniform(-1.0, 1.0, rho.size)
    return a, b, rho, rhodot


def _gpu(a, rho, rhodot, theta, precision="fp64"):
    phi, g, pd, net = a.solve_dt(torch.from_numpy(rho).cuda(), torch.from_numpy(rhodot).cuda(),
                                 theta, precision)
    return phi.cpu().numpy(), g.cpu().numpy(), pd.cpu().numpy(), net.cpu().numpy()


def _rel(a, ref, absref):
    return float((np.abs(a - ref) / np.abs(absref)).max())


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("theta", [0.5, 0.34])
def test_dt_fp64_matches_oracle_every_cell(case, theta):
    a, b, rho, rhodot = _setup(case)
    ref = O.solve_dt(b, rho, rhodot, theta)
    absref = O.solve_dt(b, rho, np.abs(rhodot), theta)
    _, _, pd, _ = _gpu(a, rho, rhodot, theta)
    assert _rel(pd, ref, absref) <= FP64_TOL


@pytest.mark.parametrize("case", ["tiny_amr", "tilted_binary_L3"])
def test_dt_mixed_within_tolerance(case):
    a, b, rho, rhodot = _setup(case)
    ref = O.solve_dt(b, rho, rhodot, 0.5)
    _, _, pd, _ = _gpu(a, rho, rhodot, 0.5, "mixed")
    assert np.abs(pd - ref).max() / np.abs(ref).max() <= MIXED_TOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dt_solve_leaves_the_rho_solve_unchanged(precision):
    a, _, rho, rhodot = _setup("tilted_binary_L3")
    p0, g0, n0 = (x.cpu().numpy() for x in a.solve(torch.from_numpy(rho).cuda(), 0.5, precision))
    phi, g, _, net = _gpu(a, rho, rhodot, 0.5, precision)
    assert np.array_equal(phi, p0) and np.array_equal(g, g0) and np.array_equal(net, n0)


def test_dt_of_rho_is_phi_and_energy_terms_cancel():
    a, b, rho, rhodot = _setup("tilted_binary_L3")
    phi, _, pd_rho, _ = _gpu(a, rho, rho, 0.5)
    assert np.abs(pd_rho - phi).max() <= 1e-13 * np.abs(phi).max()
    phi, _, pd, _ = _gpu(a, rho, rhodot, 0.5)
    _, m = O.leaf_masses(b, rho)
    _, s = O.leaf_masses(b, rhodot)
    lhs, rhs = (s * phi).sum(), (m * pd).sum()
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(s) * np.abs(phi)).sum()


def test_dt_graph_equals_direct_launches_and_forest_slices():
    a, _, rho, rhodot = _setup("tiny_amr")
    a.set_graphs(False)
    ref = _gpu(a, rho, rhodot, 0.5)
    a.set_graphs(True)
    for _ in range(2):
        got = _gpu(a, rho, rhodot, 0.5)
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)
    # a forest: each tree's slice equals its own solve
    t2, _, rho2, rhodot2 = _setup("tilted_binary_L3", seed=8)
    f = api.Forest([a, t2])
    n, off = f.forest_info()
    phi, g, pd, net = _gpu(f, np.concatenate([rho, rho2]), np.concatenate([rhodot, rhodot2]), 0.5)
    assert np.array_equal(pd[: off[1] * 512], ref[2])
    assert np.array_equal(pd[off[1] * 512:], _gpu(t2, rho2, rhodot2, 0.5)[2])


def test_dt_invalid_source_reported():
    a, _, rho, rhodot = _setup("tiny_amr")
    bad = rhodot.copy()
    bad[17] = np.nan
    with pytest.raises(_lib.FmmError) as e:
        _gpu(a, rho, bad, 0.5)
    assert e.value.code == _lib.FMM_ERR_NONFINITE
    _, _, pd, _ = _gpu(a, rho, rhodot, 0.5)   # status cleared; tree still usable
    assert np.isfinite(pd).all()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dt_paper_binary_sampled(precision):
    """9 levels, theta = 0.34, 2.07M leaf cells; the oracle evaluates sampled cells one by one."""
    w = synth.workload_paper_binary()
    a = api.Tree(w.max_level, w.flags)
    b = O.Tree(w.max_level, w.flags)
    rho = synth.leaf_density(w.field, b.leaves())
    rhodot = rho * np.random.default_rng(21).uniform(-1.0, 1.0, rho.size)
    _, _, pd, _ = _gpu(a, rho, rhodot, w.theta, precision)
    idx = np.random.default_rng(22).choice(rho.size, 40, replace=False)
    ref = O.solve_dt(b, rho, rhodot, w.theta, idx=idx)
    scale = np.abs(ref).max()
    if precision == "fp64":
        absref = O.solve_dt(b, rho, np.abs(rhodot), w.theta, idx=idx)
        assert _rel(pd[idx], ref, absref) <= FP64_TOL
    else:
        assert np.abs(pd[idx] - ref).max() / scale <= MIXED_TOL
