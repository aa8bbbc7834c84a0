"""The mixed path's refined targets, whose partners' FP32 moments are staged in shared memory one
parity class at a time (bulk asynchronous copies on an mbarrier): the same pairs as the FP64
path, so against the FP64 oracle per cell within the mixed tolerance; at theta = 0.34 every class
holds more than one 64-pair correction chunk; refined level-1 subgrids lie on the domain
boundary, so their absent neighbours take the zero-filled branch; a wait limit that runs out is
reported as FMM_ERR_TIMEOUT and leaves the tree usable.  Both staging kernels: the one whose warps
meet at every class (variant 0) and the pipelined one with a copy-issuing warp and full / empty
barriers per buffer (variant 3)."""
import numpy as np
import pytest

import oracle as O
from paper_2101_08226_gb300 import _lib, api, build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _inf(a, ref):
    return float(np.abs(np.asarray(a) - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("theta", [0.34, 0.5, 0.7])
@pytest.mark.parametrize("case", ["uniform_d2", "binary_L3"])
def test_staged_refined_targets_match_oracle(case, theta, variant):
    if case == "uniform_d2":
        ml, fl, fld = 2, synth.uniform_flags(2), synth.single_polytrope_field(0.3)
    else:
        w = synth.workload_binary(3, axis=(1.0, 0.6, 0.3), offset=(0.02, -0.03, 0.05))
        ml, fl, fld = w.max_level, w.flags, w.field
    a, b = api.Tree(ml, fl), O.Tree(ml, fl)
    rho = synth.leaf_density(fld, b.leaves())
    phi_o, g_o, _ = O.solve(b, rho, theta)
    a.set_variant(theta, variant)
    phi, g, net = a.solve(torch.from_numpy(rho).cuda(), theta, "mixed")
    assert _inf(phi.cpu().numpy(), phi_o) <= MIXED_TOL
    assert _inf(g.cpu().numpy(), g_o) <= MIXED_TOL


@pytest.mark.parametrize("variant", [0, 3])
def test_wait_timeout_reported_and_recovered(variant):
    w = synth.workload_binary(3)
    a, b = api.Tree(w.max_level, w.flags), O.Tree(w.max_level, w.flags)
    rho = synth.leaf_density(w.field, b.leaves())
    a.set_variant(0.5, variant)
    r = torch.from_numpy(rho).cuda()
    phi_o, g_o, _ = O.solve(b, rho, 0.5)
    a.solve(r, 0.5, "mixed")  # checks the status word
    # one cycle: the first class's copies cannot have landed when the wait first tests (variant
    # 0); the copy-issuing warp of variant 3 gives up on its first wait for a buffer to empty
    a.set_wait_limit(1)
    with pytest.raises(_lib.FmmError) as e:
        a.solve(r, 0.5, "mixed")
    assert e.value.code == _lib.FMM_ERR_TIMEOUT
    a.set_wait_limit(0)
    phi, g, _ = a.solve(r, 0.5, "mixed")
    assert _inf(phi.cpu().numpy(), phi_o) <= MIXED_TOL
    assert _inf(g.cpu().numpy(), g_o) <= MIXED_TOL
