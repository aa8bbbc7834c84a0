"""The level passes as persistent launches (fmm_set_persistent): the upward octant phases and the
downward level phases each run in one cooperative launch whose blocks meet at a grid-wide barrier
between phases.  Every item is the same device function as in the per-phase launches, so phi, g
and the net sums are the same bit for bit -- for every precision, with and without CUDA graphs,
on a single tree, a deep AMR tree and a forest of uneven trees -- and both agree with the FP64
oracle.  A barrier wait bounded to one cycle runs out, is reported as FMM_ERR_TIMEOUT, and the
next solve with the default limit is correct again."""
import numpy as np
import pytest

import oracle as O
from paper_2101_08226_gb300 import _lib, api, build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


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
    return 3, fl, synth.binary_field(0.7, 0.1, 0.085, 0.35, axis=(1.0, 0.6, 0.3))


CASES = {
    "tiny_amr": _tiny_amr,
    "uniform_d2": lambda: (2, synth.uniform_flags(2), synth.single_polytrope_field(0.3)),
    "binary_L4": lambda: (lambda w: (w.max_level, w.flags, w.field))(synth.workload_binary(4)),
}


def _outputs(tree, rho, theta, precision):
    phi, g, net = tree.solve(rho, theta, precision)
    return phi.cpu().numpy(), g.cpu().numpy(), net.cpu().numpy()


@pytest.mark.parametrize("case", list(CASES))
def test_persistent_equals_per_phase_launches(case):
    max_level, flags, fld = CASES[case]()
    a, b = api.Tree(max_level, flags), O.Tree(max_level, flags)
    rho_h = synth.leaf_density(fld, b.leaves())
    rho = torch.from_numpy(rho_h).cuda()
    phi_o, g_o, _ = O.solve(b, rho_h, 0.5)
    for precision in ("fp64", "df64", "mixed"):
        for graphs in (True, False):
            a.set_graphs(graphs)
            a.set_persistent(False)
            ref = _outputs(a, rho, 0.5, precision)
            a.set_persistent(True)
            got = _outputs(a, rho, 0.5, precision)
            for x, y in zip(got, ref):
                assert np.array_equal(x, y), (case, precision, graphs)
    a.set_graphs(True)
    phi, g, _ = _outputs(a, rho, 0.5, "fp64")
    assert np.abs(phi - phi_o).max() <= FP64_TOL * np.abs(phi_o).max()
    assert np.abs(g - g_o).max() <= FP64_TOL * np.abs(g_o).max()


def test_persistent_forest_equals_per_phase_launches():
    ws = synth.batched_workloads(8)
    trees = [api.Tree(w.max_level, w.flags) for w in ws]
    f = api.Forest(trees)
    rho = torch.from_numpy(np.concatenate([synth.leaf_density(w.field, t.leaves())
                                           for w, t in zip(ws, trees)])).cuda()
    for precision in ("fp64", "mixed"):
        f.set_persistent(False)
        ref = _outputs(f, rho, 0.5, precision)
        f.set_persistent(True)
        got = _outputs(f, rho, 0.5, precision)
        for x, y in zip(got, ref):
            assert np.array_equal(x, y), precision


def test_barrier_timeout_reported_and_recovered():
    w = synth.workload_binary(4)
    a = api.Tree(w.max_level, w.flags)
    rho = torch.from_numpy(synth.leaf_density(w.field, a.leaves())).cuda()
    ref = _outputs(a, rho, 0.5, "fp64")
    a.set_persistent(True)
    # one cycle: a block that reaches the first barrier before the last one arrives gives up
    a.set_wait_limit(1)
    with pytest.raises(_lib.FmmError) as e:
        a.solve(rho, 0.5, "fp64")
    assert e.value.code == _lib.FMM_ERR_TIMEOUT
    a.set_wait_limit(0)
    got = _outputs(a, rho, 0.5, "fp64")
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)
