"""Host-side checks of the CUDA library (no GPU needed): it loads and exports every entry point
that include/octo_fmm.h declares; its tree, stencils and interaction counts equal the oracle's
bit for bit; arguments are validated."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2101_08226_gb300 import _lib, api, build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(fmm_\w+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    decl = _declared()
    assert len(decl) >= 13
    for name in decl:
        assert hasattr(L, name), name
    assert set(decl) == set(_lib.EXPORTS)


def _trees():
    yield "uniform_d2", 2, synth.uniform_flags(2)
    yield "uniform_d1", 1, synth.uniform_flags(1)
    yield "root_only", 0, np.zeros(0, np.uint8)
    w = synth.workload_binary(4)
    yield "binary_L4", w.max_level, w.flags
    w = synth.workload_binary(3, axis=(1.0, 0.6, 0.3), offset=(0.02, -0.03, 0.05))
    yield "tilted_L3", w.max_level, w.flags
    rng = np.random.default_rng(5)
    for r in range(3):
        fl = (rng.uniform(size=synth.flags_size(5)) < 0.02).astype(np.uint8)
        fl[0] = 1
        yield f"random{r}", 5, fl


@pytest.mark.parametrize("name,max_level,flags", list(_trees()), ids=[t[0] for t in _trees()])
def test_tree_equals_oracle_tree(name, max_level, flags):
    a = api.Tree(max_level, flags).subgrids()
    b = O.Tree(max_level, flags).subgrids()
    assert a.shape == b.shape and np.array_equal(a, b)


def test_large_binary_tree_equals_oracle_tree():
    w = synth.workload_binary(7, q=0.6, a=0.3)
    a = api.Tree(w.max_level, w.flags)
    b = O.Tree(w.max_level, w.flags)
    sa, sb = a.subgrids(), b.subgrids()
    assert np.array_equal(sa, sb)
    assert sa.shape[0] > 10000


def test_nine_level_paper_binary_tree_equals_oracle_tree():
    """The deepest tree the paper uses (9 refinement levels), built both ways."""
    w = synth.workload_paper_binary()
    a = api.Tree(w.max_level, w.flags)
    b = O.Tree(w.max_level, w.flags)
    assert np.array_equal(a.subgrids(), b.subgrids())
    assert a.subgrids()[:, 0].max() == 9


@pytest.mark.parametrize("theta", [0.34, 0.35, 0.4, 0.5, 0.6, 0.7, 0.9, 0.999])
def test_stencil_equals_oracle(theta):
    for p in range(8):
        assert np.array_equal(api.stencil(theta, p), O.stencil(theta, p))


def test_counts_equal_oracle_counts():
    cases = [(2, synth.uniform_flags(2), (0.5, 0.35, 0.7))]
    w = synth.workload_binary(3, axis=(1.0, 0.6, 0.3), offset=(0.02, -0.03, 0.05))
    cases.append((w.max_level, w.flags, (0.5, 0.7)))
    fl = np.zeros(synth.flags_size(3), dtype=np.uint8)
    fl[0] = 1
    fl[synth.flags_offset(1)] = 1
    fl[synth.flags_offset(2) + (1 * 4 + 1) * 4] = 1
    cases.append((3, fl, (0.5, 0.34)))
    cases.append((0, np.zeros(0, np.uint8), (0.5,)))
    for max_level, flags, thetas in cases:
        ta = api.Tree(max_level, flags)
        tb = O.Tree(max_level, flags)
        rho = np.ones(tb.n_leaf_cells)
        for th in thetas:
            _, _, cb = O.solve(tb, rho, th)
            assert ta.counts(th) == cb, (max_level, th)


def test_argument_errors():
    with pytest.raises(_lib.FmmError) as e:
        api.Tree(2, np.ones(3, np.uint8))
    assert e.value.code == _lib.FMM_ERR_ARG
    with pytest.raises(_lib.FmmError) as e:
        api.Tree(10, np.ones(synth.flags_size(10), np.uint8))
    assert e.value.code == _lib.FMM_ERR_ARG
    t = api.Tree(1, synth.uniform_flags(1))
    for th in (0.2, 0.3399, 1.0, float("nan")):
        with pytest.raises(_lib.FmmError) as e:
            t.counts(th)
        assert e.value.code == _lib.FMM_ERR_THETA
        with pytest.raises(_lib.FmmError):
            api.stencil(th, 0)
    n = C.c_int32()
    assert _lib.lib().fmm_stencil(0.5, 8, None, 0, C.byref(n)) == _lib.FMM_ERR_ARG
    assert _lib.lib().fmm_solve(None, None, 0.5, 0, 1, None, None, None, None) == _lib.FMM_ERR_ARG
    assert _lib.lib().fmm_solve(t._h, None, 0.5, 0, 1, None, None, None, None) == _lib.FMM_ERR_ARG
    assert _lib.lib().fmm_solve(t._h, C.c_void_p(16), 0.5, 7, 1, C.c_void_p(16), C.c_void_p(16),
                                None, None) == _lib.FMM_ERR_ARG
    assert _lib.lib().fmm_solve(t._h, C.c_void_p(16), 0.2, 0, 1, C.c_void_p(16), C.c_void_p(16),
                                None, None) == _lib.FMM_ERR_THETA
    assert b"theta" in _lib.lib().fmm_last_error()
    assert _lib.lib().fmm_set_wait_limit(None, 0) == _lib.FMM_ERR_ARG
    assert _lib.lib().fmm_set_wait_limit(t._h, -1) == _lib.FMM_ERR_ARG
    assert _lib.lib().fmm_set_wait_limit(t._h, 0) == _lib.FMM_OK
    assert _lib.lib().fmm_set_variant(None, 0.5, 0) == _lib.FMM_ERR_ARG
    assert _lib.lib().fmm_set_variant(t._h, 0.5, -1) == _lib.FMM_ERR_ARG
    assert _lib.lib().fmm_set_variant(t._h, 0.5, _lib.FMM_MIXED_VARIANTS) == _lib.FMM_ERR_ARG
    assert _lib.lib().fmm_set_variant(t._h, 0.2, 0) == _lib.FMM_ERR_THETA
    v = C.c_int32()
    assert _lib.lib().fmm_autotune(t._h, None, 0.5, 1, 1, None, None, 3, None, C.byref(v),
                                   None) == _lib.FMM_ERR_ARG
    assert _lib.lib().fmm_autotune(t._h, C.c_void_p(16), 0.5, 1, 1, C.c_void_p(16), C.c_void_p(16),
                                   0, None, C.byref(v), None) == _lib.FMM_ERR_ARG


def test_forest_is_the_disjoint_union():
    trees = [api.Tree(2, synth.uniform_flags(2)), api.Tree(0, np.zeros(0, np.uint8))]
    w = synth.workload_binary(3, axis=(1.0, 0.6, 0.3), offset=(0.02, -0.03, 0.05))
    trees.append(api.Tree(w.max_level, w.flags))
    f = api.Forest(trees)
    n, off = f.forest_info()
    assert n == 3
    sizes = [t.info() for t in trees]
    assert list(np.diff(off)) == [s[1] for s in sizes]
    ns, nl, depth = f.info()
    assert ns == sum(s[0] for s in sizes) and nl == sum(s[1] for s in sizes)
    assert depth == max(s[2] for s in sizes)
    for th in (0.5, 0.35):
        tot = {}
        for t in trees:
            for k, v in t.counts_by_type(th).items():
                tot[k] = tot.get(k, 0) + v
        assert f.counts_by_type(th) == tot
    # a forest of forests flattens
    f2 = api.Forest([f, trees[0]])
    assert f2.forest_info()[0] == 4
