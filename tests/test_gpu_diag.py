"""Binary diagnostics on the GPU against the oracle (Sec. 4): the membership decision is taken
with the same correctly rounded FP64 operations in the same order on both sides, so it must
agree cell for cell; the per-star sums agree to FP64 round-off (different summation order)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import diagnostics as D
from paper_2101_08226_gb300 import _lib, api, build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _case(w):
    t = api.Tree(w.max_level, w.flags)
    b = O.Tree(w.max_level, w.flags)
    rho = synth.leaf_density(w.field, b.leaves())
    r = torch.from_numpy(rho).cuda()
    phi, g, net = t.solve(r, w.theta, "fp64")
    x, m = O.leaf_masses(b, rho)
    s1, s2 = w.field.stars
    return t, r, g, x, m, g.cpu().numpy(), np.array(s1.center), np.array(s2.center)


def _scale(x, m, g):
    return (m * np.linalg.norm(x, axis=1) * np.linalg.norm(g, axis=1)).sum() + (m * np.abs(g).sum(1)).sum()


@pytest.mark.parametrize("which", ["binary_L4", "paper_binary_L9"])
def test_membership_and_sums_match_oracle(which):
    w = synth.workload_binary(4) if which == "binary_L4" else synth.workload_paper_binary()
    t, r, g, x, m, gh, c1, c2 = _case(w)
    a = float(np.linalg.norm(c2 - c1))
    for omega, rc1, rc2 in ((0.0, 0.0, 0.0), (math.sqrt(1.0 / a ** 3), 0.1 * a, 0.08 * a)):
        sums, mem = t.binary_diagnostics(r, g, omega, c1, c2, rc1, rc2, member=True)
        ref_mem = D.membership(x, gh, omega, c1, c2, rc1, rc2)
        assert np.array_equal(mem.cpu().numpy(), ref_mem)
        ref = D.star_sums(x, m, gh, ref_mem, c1, c2)
        assert np.array_equal(sums[:, 10], ref[:, 10])     # cell counts
        assert np.abs(sums[:, :10] - ref[:, :10]).max() <= 1e-13 * _scale(x, m, gh)
        assert (ref[:, 10] > 0).all()


def test_iteration_matches_oracle():
    w = synth.workload_binary(4)
    t, r, g, x, m, gh, c1, c2 = _case(w)
    a = float(np.linalg.norm(c2 - c1))
    omega = math.sqrt(1.2 / a ** 3)
    sums, mem, (d1, d2), t_orb = t.binary_iterate(r, g, omega, c1 + 0.01, c2 - 0.01)
    # the centres come from sums whose order differs by a rounding, so a decision could only
    # differ for a cell within ~1e-16 of a tie
    rmem, rsums, e1, e2 = D.iterate(x, m, gh, omega, c1 + 0.01, c2 - 0.01)
    assert np.array_equal(mem.cpu().numpy(), rmem)
    assert np.abs(np.asarray(d1) - e1).max() < 1e-12 and np.abs(np.asarray(d2) - e2).max() < 1e-12
    assert np.abs(sums[:, :10] - rsums[:, :10]).max() <= 1e-12 * _scale(x, m, gh)
    ref_torb = np.cross(e1, rsums[0, 4:7]) + np.cross(e2, rsums[1, 4:7])
    assert np.abs(t_orb - ref_torb).max() <= 1e-12 * _scale(x, m, gh)


def test_forest_rejected():
    w = synth.workload_binary(3)
    t1, t2 = api.Tree(w.max_level, w.flags), api.Tree(w.max_level, w.flags)
    f = api.Forest([t1, t2])
    n = f.n_leaf_cells
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.FmmError):
        f.binary_diagnostics(z, torch.zeros((n, 3), dtype=torch.float64, device="cuda"), 0.0,
                             (0, 0, 0), (0.1, 0, 0))
