"""GPU parity: the CUDA solve against the oracle on the same seeded inputs.

FP64 path: every leaf cell, max_i |d_i| / max(|ref_i|, 1e-6 max|ref|) <= 1e-12 for phi and for
the acceleration vectors.  Mixed path: against the FP64 oracle, |d|_inf / |ref|_inf and the
mass-weighted RMS relative error, for g within MIXED_G_TOL and for phi within MIXED_PHI_TOL.  Full-size
workloads are checked on sampled leaf cells that the oracle evaluates one by one, and through the
net force and torque, which vanish at any size.
"""
import numpy as np
import pytest

import oracle as O
from paper_2101_08226_gb300 import _lib, api, build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_G_TOL = 1e-5
MIXED_PHI_TOL = 1e-5
CONS_TOL = 1e-13
MIXED_FORCE_TOL = 2e-6     # net force / S of the mixed path (FP32 pair sums), measured <= 5e-7
MIXED_TORQUE_TOL = 1e-7    # net torque / S of the mixed path, measured <= 1e-8
G_FLOOR = 0.1              # per-cell mixed bar on g: relative to max(|g_i|, G_FLOOR max|g|)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def rel_err(a, ref):
    a = np.asarray(a)
    ref = np.asarray(ref)
    if ref.ndim == 2:
        d = np.linalg.norm(a - ref, axis=1)
        r = np.linalg.norm(ref, axis=1)
    else:
        d = np.abs(a - ref)
        r = np.abs(ref)
    return float((d / np.maximum(r, 1e-6 * r.max())).max())


def gpu_solve(tree, rho, theta, precision="fp64", amc=True):
    r = torch.from_numpy(rho).cuda()
    phi, g, net = tree.solve(r, theta, precision, amc)
    return phi.cpu().numpy(), g.cpu().numpy(), net.cpu().numpy()


def both_trees(max_level, flags):
    a = api.Tree(max_level, flags)
    b = O.Tree(max_level, flags)
    assert np.array_equal(a.subgrids(), b.subgrids())
    return a, b


def tiny_amr_flags():
    fl = np.zeros(synth.flags_size(3), dtype=np.uint8)
    fl[0] = 1
    fl[synth.flags_offset(1)] = 1
    fl[synth.flags_offset(2) + (1 * 4 + 1) * 4] = 1
    return 3, fl


CASES = {
    "root_only": lambda: (0, np.zeros(0, np.uint8), synth.single_polytrope_field(0.3)),
    "uniform_d1": lambda: (1, synth.uniform_flags(1), synth.single_polytrope_field(0.3)),
    "uniform_d2": lambda: (2, synth.uniform_flags(2), synth.single_polytrope_field(0.3)),
    "tiny_amr": lambda: tiny_amr_flags() + (synth.binary_field(0.7, 0.1, 0.085, 0.35),),
    "tilted_binary_L3": lambda: (lambda w: (w.max_level, w.flags, w.field))(
        synth.workload_binary(3, axis=(1.0, 0.6, 0.3), offset=(0.02, -0.03, 0.05))),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("theta", [0.5, 0.34, 0.7])
def test_fp64_matches_oracle_every_cell(case, theta):
    max_level, flags, fld = CASES[case]()
    a, b = both_trees(max_level, flags)
    rho = synth.leaf_density(fld, b.leaves())
    phi_o, g_o, cnt = O.solve(b, rho, theta)
    assert a.counts(theta) == cnt
    phi, g, net = gpu_solve(a, rho, theta)
    assert rel_err(phi, phi_o) <= FP64_TOL
    assert rel_err(g, g_o) <= FP64_TOL


def test_fp64_correction_off_matches_oracle():
    max_level, flags, fld = CASES["tilted_binary_L3"]()
    a, b = both_trees(max_level, flags)
    rho = synth.leaf_density(fld, b.leaves())
    phi_o, g_o, _ = O.solve(b, rho, 0.5, amc=False)
    phi, g, _ = gpu_solve(a, rho, 0.5, amc=False)
    assert rel_err(phi, phi_o) <= FP64_TOL and rel_err(g, g_o) <= FP64_TOL


def test_fp64_conservation_and_reduction():
    max_level, flags, fld = CASES["tilted_binary_L3"]()
    a, b = both_trees(max_level, flags)
    rho = synth.leaf_density(fld, b.leaves())
    x, m = O.leaf_masses(b, rho)
    phi, g, net = gpu_solve(a, rho, 0.5)
    f = m[:, None] * g
    ref = np.concatenate([f.sum(0), np.cross(x, f).sum(0),
                          [(np.linalg.norm(x, axis=1) * np.linalg.norm(f, axis=1)).sum()]])
    assert abs(net[6] - ref[6]) <= 1e-6 * ref[6]   # the normalisation is formed in FP32
    assert np.abs(net[:6] - ref[:6]).max() <= 1e-14 * ref[6]
    assert np.abs(net[:3]).max() <= CONS_TOL * net[6]
    assert np.abs(net[3:6]).max() <= CONS_TOL * net[6]
    _, g0, net0 = gpu_solve(a, rho, 0.5, amc=False)
    assert np.abs(net0[3:6]).max() > 1e6 * np.abs(net[3:6]).max()


def test_fp64_deterministic():
    max_level, flags, fld = CASES["tiny_amr"]()
    a, b = both_trees(max_level, flags)
    rho = synth.leaf_density(fld, b.leaves())
    p1, g1, n1 = gpu_solve(a, rho, 0.5)
    p2, g2, n2 = gpu_solve(a, rho, 0.5)
    assert np.array_equal(p1, p2) and np.array_equal(g1, g2) and np.array_equal(n1, n2)


def test_single_source_pair_coverage_on_gpu():
    max_level, flags, _ = CASES["tiny_amr"]()
    a, b = both_trees(max_level, flags)
    x, dx = synth.leaf_cell_centres(b.leaves())
    n = x.shape[0]
    for j in np.random.default_rng(4).choice(n, 6, replace=False):
        rho = np.zeros(n)
        rho[j] = 1.0 / dx[j] ** 3
        phi_o, g_o, _ = O.solve(b, rho, 0.5)
        phi, g, _ = gpu_solve(a, rho, 0.5)
        assert phi[j] == 0.0
        assert rel_err(phi, phi_o) <= FP64_TOL and rel_err(g, g_o) <= FP64_TOL


@pytest.mark.parametrize("case", ["uniform_d2", "tilted_binary_L3"])
@pytest.mark.parametrize("theta", [0.35, 0.5, 0.7])
def test_mixed_within_tolerance(case, theta):
    max_level, flags, fld = CASES[case]()
    a, b = both_trees(max_level, flags)
    rho = synth.leaf_density(fld, b.leaves())
    phi_o, g_o, _ = O.solve(b, rho, theta)
    phi, g, net = gpu_solve(a, rho, theta, "mixed")
    _, m = O.leaf_masses(b, rho)
    gn = np.linalg.norm(g_o, axis=1)
    w = m / m.sum()
    g_inf = np.abs(g - g_o).max() / np.abs(g_o).max()
    g_rms = np.sqrt((w * (np.linalg.norm(g - g_o, axis=1) / gn) ** 2).sum())
    phi_inf = np.abs(phi - phi_o).max() / np.abs(phi_o).max()
    phi_rms = np.sqrt((w * ((phi - phi_o) / phi_o) ** 2).sum())
    assert g_inf <= MIXED_G_TOL and g_rms <= MIXED_G_TOL
    assert phi_inf <= MIXED_PHI_TOL and phi_rms <= MIXED_PHI_TOL
    # FP32 pair sums on each side of a pair: conservation to FP32 rounding, not to round-off
    assert np.abs(net[:3]).max() <= MIXED_FORCE_TOL * net[6]
    assert np.abs(net[3:6]).max() <= MIXED_TORQUE_TOL * net[6]


def test_invalid_density_reported():
    a = api.Tree(1, synth.uniform_flags(1))
    n = a.n_leaf_cells
    for bad in (np.nan, -1.0, np.inf):
        rho = np.ones(n)
        rho[n // 3] = bad
        with pytest.raises(_lib.FmmError) as e:
            gpu_solve(a, rho, 0.5)
        assert e.value.code == _lib.FMM_ERR_NONFINITE
    phi, g, net = gpu_solve(a, np.ones(n), 0.5)   # status cleared; tree still usable
    assert np.isfinite(phi).all()


def test_host_entry_point_equals_device_entry_point():
    max_level, flags, fld = CASES["tiny_amr"]()
    a, b = both_trees(max_level, flags)
    rho = synth.leaf_density(fld, b.leaves())
    p1, g1, n1 = gpu_solve(a, rho, 0.5)
    p2, g2, n2 = a.solve_host(rho, 0.5)
    assert np.array_equal(p1, p2) and np.array_equal(g1, g2) and np.array_equal(n1, n2)
    r = torch.from_numpy(rho).cuda()
    net = a.net_force_torque(r, torch.from_numpy(g1).cuda()).cpu().numpy()
    assert np.array_equal(net, n1)


def mixed_per_cell(phi, g, net, ps, gs, idx):
    """The mixed path's bar at theta <= 0.5, per sampled cell: |d phi_i| <= 1e-5 |phi_i| and
    |d g_i| <= 1e-5 max(|g_i|, G_FLOOR max|g|); net force and torque to FP32 rounding."""
    assert (np.abs(phi[idx] - ps) / np.abs(ps)).max() <= MIXED_PHI_TOL
    gn = np.linalg.norm(gs, axis=1)
    d_g = np.linalg.norm(g[idx] - gs, axis=1) / np.maximum(gn, G_FLOOR * np.abs(g).max())
    assert d_g.max() <= MIXED_G_TOL
    assert np.abs(net[:3]).max() <= MIXED_FORCE_TOL * net[6]
    assert np.abs(net[3:6]).max() <= MIXED_TORQUE_TOL * net[6]


@pytest.mark.parametrize("levels,precision", [(5, "fp64"), (5, "mixed"), (6, "fp64"), (6, "mixed"),
                                              (7, "fp64"), (7, "mixed")])
def test_full_size_sampled(levels, precision):
    """The 5-level q = 0.7 binary (about 0.9M cells), the same field refined to 6 levels, and the
    7-level q = 0.6 binary (13.5M cells): the oracle evaluates a sample of leaf cells one by
    one."""
    if levels == 7:
        w = synth.workload_binary(7, q=0.6, a=0.3)
    else:
        w = synth.workload_binary(levels)
    a, b = both_trees(w.max_level, w.flags)
    rho = synth.leaf_density(w.field, b.leaves())
    phi, g, net = gpu_solve(a, rho, 0.5, precision)
    idx = np.random.default_rng(levels).choice(rho.size, 64, replace=False)
    # include cells of every leaf level
    lev = np.repeat(b.leaves()[:, 0], 512)
    extra = [int(np.nonzero(lev == l)[0][len(np.nonzero(lev == l)[0]) // 2]) for l in np.unique(lev)]
    idx = np.unique(np.concatenate([idx, extra]))
    ps, gs = O.sample(b, rho, 0.5, idx)
    if precision == "fp64":
        d_phi = np.abs(phi[idx] - ps) / np.abs(ps)
        d_g = np.linalg.norm(g[idx] - gs, axis=1) / np.maximum(np.linalg.norm(gs, axis=1),
                                                                 1e-6 * np.abs(g).max())
        assert d_phi.max() <= FP64_TOL and d_g.max() <= FP64_TOL
        assert np.abs(net[:6]).max() <= CONS_TOL * net[6]
    else:
        mixed_per_cell(phi, g, net, ps, gs, idx)


@pytest.mark.parametrize("graded", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_paper_binary_sampled(precision, graded):
    """The merger binary in the paper's proportions: 9 levels, theta = 0.34, 2.07M leaf cells
    (graded: the mass-based refinement, leaves on levels 2 to 9, 1.04M cells); the oracle
    evaluates sampled leaf cells one by one."""
    w = (synth.workload_paper_binary(graded=True, refine_frac=0.125) if graded
         else synth.workload_paper_binary())
    a, b = both_trees(w.max_level, w.flags)
    rho = synth.leaf_density(w.field, b.leaves())
    phi, g, net = gpu_solve(a, rho, w.theta, precision)
    lev = np.repeat(b.leaves()[:, 0], 512)
    idx = np.random.default_rng(9).choice(rho.size, 48, replace=False)
    extra = [int(np.nonzero(lev == l)[0][len(np.nonzero(lev == l)[0]) // 2]) for l in np.unique(lev)]
    idx = np.unique(np.concatenate([idx, extra]))
    ps, gs = O.sample(b, rho, w.theta, idx)
    if precision == "fp64":
        d_phi = np.abs(phi[idx] - ps) / np.abs(ps)
        d_g = np.linalg.norm(g[idx] - gs, axis=1) / np.maximum(np.linalg.norm(gs, axis=1),
                                                                 1e-6 * np.abs(g).max())
        assert d_phi.max() <= FP64_TOL and d_g.max() <= FP64_TOL
        assert np.abs(net[:6]).max() <= CONS_TOL * net[6]
    else:
        mixed_per_cell(phi, g, net, ps, gs, idx)


# ---- df64: FP64 results with the pair arithmetic in double-float on the FP32 pipes; the FP64
# path's per-cell bar at the paper's opening angles.  At theta = 0.7 the centre-of-mass series
# diverges on these trees (terms far larger than a cell's potential cancel), which amplifies the
# ~2^-44 operation error of double-float: there the bar is 1e-12 of the largest value.
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("theta", [0.5, 0.34, 0.7])
def test_df64_matches_oracle_every_cell(case, theta):
    max_level, flags, fld = CASES[case]()
    a, b = both_trees(max_level, flags)
    rho = synth.leaf_density(fld, b.leaves())
    phi_o, g_o, _ = O.solve(b, rho, theta)
    phi, g, net = gpu_solve(a, rho, theta, "df64")
    if theta < 0.6:
        assert rel_err(phi, phi_o) <= FP64_TOL
        assert rel_err(g, g_o) <= FP64_TOL
    else:
        assert np.abs(phi - phi_o).max() <= FP64_TOL * np.abs(phi_o).max()
        assert np.abs(g - g_o).max() <= FP64_TOL * np.abs(g_o).max()


def test_df64_conservation_and_correction_off():
    max_level, flags, fld = CASES["tilted_binary_L3"]()
    a, b = both_trees(max_level, flags)
    rho = synth.leaf_density(fld, b.leaves())
    phi, g, net = gpu_solve(a, rho, 0.5, "df64")
    assert np.abs(net[:3]).max() <= CONS_TOL * net[6]
    assert np.abs(net[3:6]).max() <= CONS_TOL * net[6]
    phi_o, g_o, _ = O.solve(b, rho, 0.5, amc=False)
    phi, g, _ = gpu_solve(a, rho, 0.5, "df64", amc=False)
    assert rel_err(phi, phi_o) <= FP64_TOL and rel_err(g, g_o) <= FP64_TOL


@pytest.mark.parametrize("which", ["binary_L5", "paper_binary_L9"])
def test_df64_full_size_sampled(which):
    w = synth.workload_binary(5) if which == "binary_L5" else synth.workload_paper_binary()
    a, b = both_trees(w.max_level, w.flags)
    rho = synth.leaf_density(w.field, b.leaves())
    phi, g, net = gpu_solve(a, rho, w.theta, "df64")
    idx = np.random.default_rng(5).choice(rho.size, 48, replace=False)
    lev = np.repeat(b.leaves()[:, 0], 512)
    extra = [int(np.nonzero(lev == l)[0][len(np.nonzero(lev == l)[0]) // 2]) for l in np.unique(lev)]
    idx = np.unique(np.concatenate([idx, extra]))
    ps, gs = O.sample(b, rho, w.theta, idx)
    d_phi = np.abs(phi[idx] - ps) / np.abs(ps)
    d_g = np.linalg.norm(g[idx] - gs, axis=1) / np.maximum(np.linalg.norm(gs, axis=1),
                                                             1e-6 * np.abs(g).max())
    assert d_phi.max() <= FP64_TOL and d_g.max() <= FP64_TOL
    assert np.abs(net[:6]).max() <= CONS_TOL * net[6]


def test_df64_rejected_for_time_derivative():
    a = api.Tree(1, synth.uniform_flags(1))
    r = torch.ones(a.n_leaf_cells, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.FmmError):
        a.solve_dt(r, r, 0.5, "df64")


@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed"])
def test_massless_field_gives_exact_zeros(precision):
    """The degenerate input: no mass anywhere.  Every cell's centre of mass falls back to its
    geometric centre, every moment and expansion is zero, and phi, g and the net sums come out
    as exact zeros (no NaN from a 0/0 centre of mass or a zero correction weight)."""
    max_level, flags, _ = CASES["tiny_amr"]()
    a = api.Tree(max_level, flags)
    n = a.n_leaf_cells
    for theta in (0.34, 0.5):
        phi, g, net = gpu_solve(a, np.zeros(n), theta, precision)
        assert (phi == 0.0).all() and (g == 0.0).all() and (net == 0.0).all()


def test_one_leaf_level_tree_and_forest_of_one():
    """Small degenerate shapes: a tree whose root is its only subgrid (no refined cell, no
    multipole partner beyond the root's own cells) and a forest holding one tree solve as the
    tree alone does, bit for bit."""
    a = api.Tree(0, np.zeros(0, np.uint8))
    b = O.Tree(0, np.zeros(0, np.uint8))
    rho = synth.leaf_density(synth.single_polytrope_field(0.3), b.leaves())
    phi, g, net = gpu_solve(a, rho, 0.5)
    phi_o, g_o, _ = O.solve(b, rho, 0.5)
    assert rel_err(phi, phi_o) <= FP64_TOL and rel_err(g, g_o) <= FP64_TOL
    f = api.Forest([a])
    p2, g2, n2 = gpu_solve(f, rho, 0.5)
    assert np.array_equal(p2, phi) and np.array_equal(g2, g) and np.array_equal(n2, net)


def test_pipelined_host_solves_equal_device_solves():
    """fmm_solve_host_async: a sequence of host-buffer solves on different densities, pipelined over
    two device slots and three streams, gives every step's phi, g and net sums bit for bit as the
    device entry point does, whichever slot the step used."""
    w = synth.workload_binary(4)
    a = api.Tree(w.max_level, w.flags)
    rho0 = synth.leaf_density(w.field, a.leaves())
    floor = w.field.floor * w.field.rho_peak
    steps = [np.ascontiguousarray(synth.perturbed_density(rho0, k, floor_value=floor)) for k in range(5)]
    n = rho0.size
    pinned = [torch.from_numpy(r).pin_memory() for r in steps]
    pins = [(torch.empty(n, dtype=torch.float64).pin_memory(),
             torch.empty((n, 3), dtype=torch.float64).pin_memory(),
             torch.empty(7, dtype=torch.float64).pin_memory()) for _ in steps]
    for k in range(len(steps)):
        a.solve_host_async(pinned[k].numpy(), 0.5, "fp64", pins[k][0].numpy(), pins[k][1].numpy(),
                           pins[k][2].numpy())
    a.sync_status()
    for k, r in enumerate(steps):
        phi, g, net = gpu_solve(a, r, 0.5)
        assert np.array_equal(pins[k][0].numpy(), phi) and np.array_equal(pins[k][1].numpy(), g)
        assert np.array_equal(pins[k][2].numpy(), net)
