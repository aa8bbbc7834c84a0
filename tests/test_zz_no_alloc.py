"""The allocation-free net force and torque entry point, checked against the workspace one.

Callers that cannot allocate device memory -- code inside a framework that owns all device memory
through its own pool, or a latency-critical loop where cudaMalloc and the device synchronisation
it can imply are not acceptable -- use fmm_net_force_torque_points_static, whose partial sums
live in a fixed device array of the library.  Its result must match fmm_net_force_torque, which
reduces the same field through the tree's workspace, on consecutive calls (the second call
reuses the array the first one left behind).  This file is collected last, so a failure here
leaves every other test already run.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2101_08226_gb300 import _lib, api, build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
NORM_TOL = 1e-6   # the normalisation S is formed from FP32 terms in both reductions


def _tiny_amr():
    fl = np.zeros(synth.flags_size(3), dtype=np.uint8)
    fl[0] = 1
    fl[synth.flags_offset(1)] = 1
    fl[synth.flags_offset(2) + (1 * 4 + 1) * 4] = 1
    return 3, fl


@pytest.mark.parametrize("which", ["tiny_amr", "binary_L4"])
def test_static_scratch_net_matches_workspace_net(which):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    if which == "tiny_amr":
        max_level, flags = _tiny_amr()
        fld = synth.binary_field(0.7, 0.1, 0.085, 0.35, axis=(1.0, 0.6, 0.3))
    else:
        w = synth.workload_binary(4)
        max_level, flags, fld = w.max_level, w.flags, w.field
    tree = api.Tree(max_level, flags)
    rho = synth.leaf_density(fld, tree.leaves())
    r = torch.from_numpy(rho).cuda()
    _, g, _ = tree.solve(r, 0.5, "fp64")
    ref = tree.net_force_torque(r, g).cpu().numpy()
    x, dx = synth.leaf_cell_centres(tree.leaves())
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    md = torch.from_numpy(rho * dx ** 3).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    n = x.shape[0]
    assert n > 4096  # several blocks and a partial last block
    for _ in range(2):
        out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
        rc = _lib.lib().fmm_net_force_torque_points_static(n, xd.data_ptr(), md.data_ptr(),
                                                           g.data_ptr(), out.data_ptr(), stream)
        assert rc == _lib.FMM_OK, _lib.lib().fmm_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[6] - ref[6]) <= NORM_TOL * ref[6]
        assert np.abs(got[:6] - ref[:6]).max() <= FP64_TOL * ref[6]
        # and against plain FP64 sums of the same points, formed on the host by numpy
        f = (rho * dx ** 3)[:, None] * g.cpu().numpy()
        host = np.concatenate([f.sum(0), np.cross(x, f).sum(0),
                               [(np.linalg.norm(x, axis=1) * np.linalg.norm(f, axis=1)).sum()]])
        assert abs(got[6] - host[6]) <= NORM_TOL * host[6]
        assert np.abs(got[:6] - host[:6]).max() <= FP64_TOL * host[6]


def test_static_scratch_empty_point_set():
    """n = 0 launches no partial-sum block; the sums are exact zeros, also right after a call that
    left partial sums in the shared array."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    stream = torch.cuda.current_stream().cuda_stream
    n = 5000
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.uniform(-0.5, 0.5, (n, 3))).cuda()
    m = torch.from_numpy(rng.uniform(0.0, 1.0, n)).cuda()
    g = torch.from_numpy(rng.normal(size=(n, 3))).cuda()
    out = torch.empty(7, dtype=torch.float64, device="cuda")
    assert _lib.lib().fmm_net_force_torque_points_static(n, x.data_ptr(), m.data_ptr(), g.data_ptr(),
                                                         out.data_ptr(), stream) == _lib.FMM_OK
    for _ in range(2):
        out.fill_(float("nan"))
        rc = _lib.lib().fmm_net_force_torque_points_static(0, x.data_ptr(), m.data_ptr(), g.data_ptr(),
                                                           out.data_ptr(), stream)
        assert rc == _lib.FMM_OK, _lib.lib().fmm_last_error()
        torch.cuda.synchronize()
        assert (out.cpu().numpy() == 0.0).all()


def test_static_scratch_rejects_sizes_beyond_its_capacity():
    # rejected on the host before any device work, so the pointers are never dereferenced
    p = C.c_void_p(256)
    rc = _lib.lib().fmm_net_force_torque_points_static(_lib.FMM_NET_STATIC_MAX_POINTS + 1,
                                                       p, p, p, p, None)
    assert rc == _lib.FMM_ERR_ARG
    assert b"FMM_NET_STATIC_MAX_POINTS" in _lib.lib().fmm_last_error()
