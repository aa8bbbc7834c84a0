"""The mixed-precision path (FP32 pair arithmetic, FP64 moments, correction sums and reductions)
on the 0.9M-cell 5-level binary at the three opening angles of its configuration, and the
13.5M-cell 7-level binary at the paper's smallest opening angle, against the FP64 oracle.

Bars (Sec. 2.2's opening angles; the paper uses theta = 0.5 and 0.34):
* every sampled cell, theta <= 0.5: |d phi_i| <= MIXED_TOL |phi_i| and
  |d g_i| <= MIXED_TOL max(|g_i|, G_FLOOR max|g|) -- a per-cell relative bar with a floor for the
  cells where g is small (star centres, the saddle between the stars, the far atmosphere): there
  g is a sum of terms of order max|g| that cancel, and FP32 rounding of those terms leaves an
  absolute error of a few 1e-7 max|g| (measured: per-cell 1e-5 holds down to |g| = 0.1 max|g| on
  every workload; below, 2e-5 of the cell's own |g| at worst);
* theta = 0.7, where the centre-of-mass series diverges in places (the expansion centre of a
  partner can come closer than the target's own cells), the bar is relative to the largest value;
* net force and net torque of the mixed solve at most MIXED_FORCE_TOL and MIXED_TORQUE_TOL of
  S = sum |x| |m g|: each target sums its pairs in FP32 on its own, so the two halves of a pair
  cancel only to FP32 rounding of sums whose terms are far larger than their result; the FP64
  path cancels to round-off (1e-13, test_gpu_parity.py).  Measured: force up to 5e-7 S (the
  9-level merger binary at theta = 0.34), torque up to 1e-8 S.
The samples are random leaf cells, one cell of every leaf level, and leaf cells next to refined
neighbours (targets whose partners cross a refinement boundary)."""
import numpy as np
import pytest

import oracle as O
from paper_2101_08226_gb300 import api, build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5
G_FLOOR = 0.1
MIXED_FORCE_TOL = 2e-6
MIXED_TORQUE_TOL = 1e-7


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def sample_cells(rows, n_leaf, n_random, seed):
    """Random leaf cells, the middle cell of every leaf level, and cells of leaf subgrids that
    have a refined same-level neighbour (refinement-boundary targets)."""
    leaves = rows[rows[:, 4] == 1]
    lev = np.repeat(leaves[:, 0], 512)
    rng = np.random.default_rng(seed)
    idx = [rng.choice(n_leaf, n_random, replace=False)]
    for l in np.unique(lev):
        cand = np.nonzero(lev == l)[0]
        idx.append(cand[len(cand) // 2:len(cand) // 2 + 1])
    refined = {(int(r[0]), int(r[1]), int(r[2]), int(r[3])) for r in rows if r[4] == 0}
    bnd = []
    for k, r in enumerate(leaves):
        l, i, j, kk = (int(v) for v in r[:4])
        if any((l, i + a, j + b, kk + c) in refined
               for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)):
            bnd.append(k)
    bnd = np.array(bnd)
    if bnd.size:
        pick = rng.choice(bnd, min(8, bnd.size), replace=False)
        idx.append((pick[:, None] * 512 + rng.integers(0, 512, (pick.size, 4))).ravel())
    return np.unique(np.concatenate(idx))


def check_sample(phi, g, net, ps, gs, idx, theta):
    gmax = np.abs(g).max()
    if theta <= 0.5:
        d_phi = np.abs(phi[idx] - ps) / np.abs(ps)
        gn = np.linalg.norm(gs, axis=1)
        d_g = np.linalg.norm(g[idx] - gs, axis=1) / np.maximum(gn, G_FLOOR * gmax)
        assert d_phi.max() <= MIXED_TOL, d_phi.max()
        assert d_g.max() <= MIXED_TOL, d_g.max()
    else:
        assert np.abs(phi[idx] - ps).max() <= MIXED_TOL * np.abs(ps).max()
        assert np.abs(g[idx] - gs).max() <= MIXED_TOL * gmax
    assert np.abs(net[:3]).max() <= MIXED_FORCE_TOL * net[6]
    assert np.abs(net[3:6]).max() <= MIXED_TORQUE_TOL * net[6]


@pytest.fixture(scope="module")
def binary5():
    w = synth.workload_binary(5)
    a = api.Tree(w.max_level, w.flags)
    b = O.Tree(w.max_level, w.flags)
    assert np.array_equal(a.subgrids(), b.subgrids())
    rho = synth.leaf_density(w.field, b.leaves())
    return a, b, rho


@pytest.mark.parametrize("theta", [0.35, 0.5, 0.7])
def test_mixed_binary5_sampled_against_oracle(binary5, theta):
    a, b, rho = binary5
    phi, g, net = (x.cpu().numpy() for x in a.solve(torch.from_numpy(rho).cuda(), theta, "mixed"))
    idx = sample_cells(a.subgrids(), rho.size, 96, int(theta * 100))
    ps, gs = O.sample(b, rho, theta, idx)
    check_sample(phi, g, net, ps, gs, idx, theta)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_binary7_theta034_sampled_against_oracle(precision):
    """The 13.5M-cell 7-level binary (mass ratio 0.6, density contrast 1e10) at theta = 0.34."""
    w = synth.workload_binary(7, q=0.6, a=0.3)
    a = api.Tree(w.max_level, w.flags)
    b = O.Tree(w.max_level, w.flags)
    rho = synth.leaf_density(w.field, b.leaves())
    phi, g, net = (x.cpu().numpy() for x in a.solve(torch.from_numpy(rho).cuda(), 0.34, precision))
    idx = sample_cells(a.subgrids(), rho.size, 48, 34)
    ps, gs = O.sample(b, rho, 0.34, idx)
    if precision == "fp64":
        d_phi = np.abs(phi[idx] - ps) / np.abs(ps)
        d_g = np.linalg.norm(g[idx] - gs, axis=1) / np.maximum(np.linalg.norm(gs, axis=1),
                                                                 1e-6 * np.abs(g).max())
        assert d_phi.max() <= 1e-12 and d_g.max() <= 1e-12
        assert np.abs(net[:6]).max() <= 1e-13 * net[6]
    else:
        check_sample(phi, g, net, ps, gs, idx, 0.34)
