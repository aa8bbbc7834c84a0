"""CUDA-graph replay of the solve: the same results bit for bit as launching the kernels one by
one, for any buffers a call passes, and on any caller stream."""
import numpy as np
import pytest

from paper_2101_08226_gb300 import api, build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def workload():
    w = synth.workload_binary(3, axis=(1.0, 0.6, 0.3), offset=(0.02, -0.03, 0.05))
    t = api.Tree(w.max_level, w.flags)
    return t, synth.leaf_density(w.field, t.leaves())


def run(tree, rho, theta, precision, graphs):
    tree.set_graphs(graphs)
    phi, g, net = tree.solve(torch.from_numpy(rho).cuda(), theta, precision, True)
    torch.cuda.synchronize()
    return phi.cpu().numpy(), g.cpu().numpy(), net.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_equals_direct_launches(precision):
    tree, rho = workload()
    ref = run(tree, rho, 0.5, precision, False)
    for _ in range(2):   # capture, then replay
        got = run(tree, rho, 0.5, precision, True)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)


def test_graph_follows_the_buffers_of_each_call():
    tree, rho = workload()
    rng = np.random.default_rng(3)
    rhos = [rho, rho * rng.uniform(0.5, 1.5, rho.size), rho[::-1].copy()]
    refs = [run(tree, r, 0.5, "fp64", False) for r in rhos]
    tree.set_graphs(True)
    outs = []
    for r in rhos:   # one graph, three different sets of buffers, no synchronisation between
        outs.append(tree.solve(torch.from_numpy(r).cuda(), 0.5, "fp64", True, check_status=False))
    tree.sync_status()
    for (phi, g, net), (p0, g0, n0) in zip(outs, refs):
        assert np.array_equal(phi.cpu().numpy(), p0)
        assert np.array_equal(g.cpu().numpy(), g0)
        assert np.array_equal(net.cpu().numpy(), n0)


def test_graph_per_configuration():
    tree, rho = workload()
    for theta in (0.5, 0.35, 0.5, 0.7):
        for precision in ("fp64", "mixed"):
            ref = run(tree, rho, theta, precision, False)
            got = run(tree, rho, theta, precision, True)
            for a, b in zip(got, ref):
                assert np.array_equal(a, b)


def test_graph_on_a_side_stream_and_profiled():
    tree, rho = workload()
    ref = run(tree, rho, 0.5, "mixed", False)
    tree.set_graphs(True)
    tree.set_profiling(True)
    r = torch.from_numpy(rho).cuda()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            phi, g, net = tree.solve(r, 0.5, "mixed", True, check_status=False)
        tree.sync_status()
        ms = tree.phase_times()
    s.synchronize()
    tree.set_profiling(False)
    assert np.array_equal(phi.cpu().numpy(), ref[0]) and np.array_equal(g.cpu().numpy(), ref[1])
    assert (ms > 0).all()
    # the leaf kernel starts beside the upward pass and ends inside the interaction phase; the
    # staging kernel runs inside the interaction phase
    assert ms[5] <= ms[0] + ms[1] + 0.01 and ms[4] <= ms[1] + 0.01
    assert ms[6] <= ms[1] + 0.01


def test_batch_in_place_through_graph():
    ws = synth.batched_workloads(3)
    trees = [api.Tree(w.max_level, w.flags) for w in ws]
    forest = api.Forest(trees)
    rhos = [torch.from_numpy(synth.leaf_density(w.field, t.leaves())).cuda()
            for w, t in zip(ws, trees)]
    forest.set_graphs(False)
    ref = forest.solve_batch(rhos, 0.5, "fp64", True)
    forest.set_graphs(True)
    for _ in range(2):
        phis, gs, net = forest.solve_batch(rhos, 0.5, "fp64", True)
        for a, b in zip(phis + gs + [net], ref[0] + ref[1] + [ref[2]]):
            assert torch.equal(a, b)
