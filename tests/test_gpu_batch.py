"""Forests: independent trees solved by one set of launches.

Each tree's slice of a forest solve must equal the tree's own solve bit for bit (the kernels do
the same arithmetic per cell wherever the tree sits in the forest; the net sums, whose reduction
layout depends on the number of trees, to round-off), the per-tree entry point must
equal the concatenated one, and the batched workload of 64 seeded trees of uneven depth must
match the oracle tree by tree.
"""
import numpy as np
import pytest

import oracle as O
from paper_2101_08226_gb300 import api, build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _small_trees():
    fl = np.zeros(synth.flags_size(3), dtype=np.uint8)
    fl[0] = 1
    fl[synth.flags_offset(1)] = 1
    fl[synth.flags_offset(2) + (1 * 4 + 1) * 4] = 1
    w = synth.workload_binary(3, axis=(1.0, 0.6, 0.3), offset=(0.02, -0.03, 0.05))
    specs = [(3, fl, synth.binary_field(0.7, 0.1, 0.085, 0.35)),
             (0, np.zeros(0, np.uint8), synth.single_polytrope_field(0.3)),
             (w.max_level, w.flags, w.field),
             (1, synth.uniform_flags(1), synth.single_polytrope_field(0.2, center=(0.1, 0, 0)))]
    trees = [api.Tree(m, f) for m, f, _ in specs]
    rhos = [synth.leaf_density(fld, t.leaves()) for t, (_, _, fld) in zip(trees, specs)]
    return trees, rhos


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forest_slices_equal_individual_solves(precision):
    trees, rhos = _small_trees()
    f = api.Forest(trees)
    n, off = f.forest_info()
    r = torch.from_numpy(np.concatenate(rhos)).cuda()
    phi, g, net = f.solve(r, 0.5, precision)
    phi, g, net = phi.cpu().numpy(), g.cpu().numpy(), net.cpu().numpy().reshape(n, 7)
    for k, (t, rho) in enumerate(zip(trees, rhos)):
        p1, g1, n1 = t.solve(torch.from_numpy(rho).cuda(), 0.5, precision)
        sl = slice(off[k] * 512, off[k + 1] * 512)
        assert np.array_equal(phi[sl], p1.cpu().numpy())
        assert np.array_equal(g[sl], g1.cpu().numpy())
        # the reduction's block layout depends on the number of trees: F and T equal to FP64
        # round-off, the normalisation S (summed in FP32 per thread) to FP32 round-off
        n1 = n1.cpu().numpy()
        assert np.abs(net[k][:6] - n1[:6]).max() <= 1e-14 * n1[6]
        assert abs(net[k][6] - n1[6]) <= 1e-6 * n1[6]
    rs = [torch.from_numpy(x).cuda() for x in rhos]
    phis, gs, net2 = f.solve_batch(rs, 0.5, precision)
    for k in range(n):
        sl = slice(off[k] * 512, off[k + 1] * 512)
        assert np.array_equal(phis[k].cpu().numpy(), phi[sl])
        assert np.array_equal(gs[k].cpu().numpy(), g[sl])
    assert np.array_equal(net2.cpu().numpy().reshape(n, 7), net)


def test_batched_64_trees_match_oracle():
    """64 seeded trees, levels 2..5, single stars or binaries: FP64 within 1e-12 of the oracle
    (every cell for trees up to 3 levels, 48 sampled cells for deeper ones), mixed within 1e-5,
    net force and torque at round-off for every tree."""
    ws = synth.batched_workloads(64)
    trees = [api.Tree(w.max_level, w.flags) for w in ws]
    rhos = [synth.leaf_density(w.field, t.leaves()) for w, t in zip(ws, trees)]
    f = api.Forest(trees)
    n, off = f.forest_info()
    r = torch.from_numpy(np.concatenate(rhos)).cuda()
    phi64, g64, net64 = (x.cpu().numpy() for x in f.solve(r, 0.5, "fp64"))
    phi32, g32, _ = (x.cpu().numpy() for x in f.solve(r, 0.5, "mixed"))
    net64 = net64.reshape(n, 7)
    for k, (w, rho) in enumerate(zip(ws, rhos)):
        assert np.abs(net64[k, :6]).max() <= 1e-13 * net64[k, 6]
        sl = slice(off[k] * 512, off[k + 1] * 512)
        ot = O.Tree(w.max_level, w.flags)
        if w.max_level <= 3:
            ps, gs, _ = O.solve(ot, rho, 0.5)
            idx = np.arange(rho.size)
        else:
            idx = np.random.default_rng(k).choice(rho.size, 48, replace=False)
            ps, gs = O.sample(ot, rho, 0.5, idx)
        p, gg = phi64[sl][idx], g64[sl][idx]
        assert (np.abs(p - ps) / np.abs(ps)).max() <= FP64_TOL
        gn = np.linalg.norm(gs, axis=1)
        assert (np.linalg.norm(gg - gs, axis=1) / np.maximum(gn, 1e-6 * gn.max())).max() <= FP64_TOL
        assert np.abs(phi32[sl][idx] - ps).max() / np.abs(ps).max() <= MIXED_TOL
        assert np.abs(g32[sl][idx] - gs).max() / np.abs(gs).max() <= MIXED_TOL
