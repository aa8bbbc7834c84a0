"""The bounds-checked build of the library (libocto_fmm_bc.so, -DFMM_BOUNDS_CHECK): every index the
kernels read from the library's tables (neighbours, children, leaf ordinals, work lists, pair
lists, stencil and staging tables) is range-checked before the access it leads to, and a failed
check is reported as FMM_ERR_BOUNDS instead of being made.  On valid trees no check may fire: the
solves of every precision, every mixed launch variant, the time-derivative solve and a forest
report FMM_OK and give the normal build's results; so do the persistent level passes."""
import ctypes as C

import numpy as np
import pytest

from paper_2101_08226_gb300 import _lib, api, build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return _lib.load(build.LIB_BC)


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


def _tree(L, max_level, flags):
    h = C.c_void_p()
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    assert L.fmm_build_tree(int(max_level), flags.ctypes.data_as(C.c_void_p), int(flags.size),
                            C.byref(h)) == 0
    return h


def _solve(L, h, rho, theta, precision, variant=None, rhodot=None, persistent=False):
    n = rho.numel()
    assert L.fmm_set_persistent(h, int(persistent)) == 0
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    net = torch.empty(7, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    if variant is not None:
        assert L.fmm_set_variant(h, theta, variant) == 0
    if rhodot is None:
        rc = L.fmm_solve(h, rho.data_ptr(), theta, api.PRECISIONS[precision], 1, phi.data_ptr(),
                         g.data_ptr(), net.data_ptr(), st)
        out = (phi, g, net)
    else:
        pd = torch.empty(n, dtype=torch.float64, device="cuda")
        rc = L.fmm_solve_dt(h, rho.data_ptr(), rhodot.data_ptr(), theta, api.PRECISIONS[precision], 1,
                            phi.data_ptr(), g.data_ptr(), pd.data_ptr(), net.data_ptr(), st)
        out = (phi, g, pd)
    assert rc == 0, L.fmm_last_error()
    rc = L.fmm_sync_status(h, st)
    assert rc == 0, (rc, L.fmm_last_error())
    return [x.cpu().numpy() for x in out]


@pytest.mark.parametrize("case", list(CASES))
def test_no_check_fires_and_results_agree(checked, case):
    max_level, flags, fld = CASES[case]()
    plain = _lib.lib()
    hc, hp = _tree(checked, max_level, flags), _tree(plain, max_level, flags)
    try:
        leaves = api.Tree(max_level, flags).leaves()
        rho = torch.from_numpy(synth.leaf_density(fld, leaves)).cuda()
        rhodot = rho * torch.from_numpy(np.random.default_rng(2).uniform(-1, 1, rho.numel())).cuda()
        runs = [(p, th, None, None, False) for p in ("fp64", "df64", "mixed") for th in (0.34, 0.5, 0.7)]
        variants = range(_lib.FMM_MIXED_VARIANTS) if case == "tiny_amr" else range(0, _lib.FMM_MIXED_VARIANTS, 7)
        runs += [("mixed", 0.5, v, None, False) for v in variants]
        runs += [("fp64", 0.5, None, rhodot, False), ("mixed", 0.5, None, rhodot, False)]
        runs += [(p, 0.5, None, None, True) for p in ("fp64", "df64", "mixed")]  # persistent level passes
        for precision, theta, variant, rd, pers in runs:
            got = _solve(checked, hc, rho, theta, precision, variant, rd, pers)
            ref = _solve(plain, hp, rho, theta, precision, variant, rd, pers)
            for a, b in zip(got, ref):
                assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), (precision, theta, variant)
    finally:
        checked.fmm_destroy(hc)
        plain.fmm_destroy(hp)


def test_forest_no_check_fires(checked):
    ws = synth.batched_workloads(6)
    hs = [_tree(checked, w.max_level, w.flags) for w in ws]
    f = C.c_void_p()
    arr = (C.c_void_p * len(hs))(*hs)
    assert checked.fmm_build_forest(arr, len(hs), C.byref(f)) == 0
    rho = torch.from_numpy(np.concatenate([synth.leaf_density(w.field, api.Tree(w.max_level, w.flags).leaves())
                                           for w in ws])).cuda()
    for precision in ("fp64", "mixed"):
        phi, g, net = _solve(checked, f, rho, 0.5, precision)
        assert np.isfinite(phi).all() and np.isfinite(g).all()
    checked.fmm_destroy(f)
    for h in hs:
        checked.fmm_destroy(h)
