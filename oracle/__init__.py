"""Oracle for the octree FMM gravity solve -- TEST INFRASTRUCTURE ONLY.

Python handle on the plain C oracle (octo_oracle.c): a slow, obviously correct FP64 restatement of
the paper's gravity solve (Sec. 2.2) plus the exact O(N^2) point-mass sum.  Only `tests/`, the
smoke check and the benchmark's CPU-baseline leg may import this package; the CUDA library never
does, and the two share no code.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Tuple

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
        L.oracle_tree_build.restype = vp
        L.oracle_tree_build.argtypes = [i32, vp, i64]
        L.oracle_tree_free.argtypes = [vp]
        L.oracle_tree_free.restype = None
        L.oracle_tree_depth.argtypes = [vp]
        L.oracle_tree_depth.restype = i32
        L.oracle_tree_n_subgrids.argtypes = [vp]
        L.oracle_tree_n_subgrids.restype = i64
        L.oracle_tree_n_leaf_subgrids.argtypes = [vp]
        L.oracle_tree_n_leaf_subgrids.restype = i64
        L.oracle_tree_subgrids.argtypes = [vp, vp]
        L.oracle_tree_subgrids.restype = None
        L.oracle_stencil.argtypes = [dbl, i32, vp, i32]
        L.oracle_stencil.restype = i32
        L.oracle_fmm_solve.argtypes = [vp, vp, dbl, i32, i32, vp, vp, vp]
        L.oracle_fmm_solve.restype = None
        L.oracle_fmm_sample.argtypes = [vp, vp, dbl, i32, i32, i64, vp, vp, vp, vp]
        L.oracle_fmm_sample.restype = None
        L.oracle_fmm_sample_given.argtypes = [vp, vp, vp, dbl, i32, i32, i64, vp, vp, vp]
        L.oracle_fmm_sample_given.restype = None
        L.oracle_inner_moments.argtypes = [vp, vp, i32, vp]
        L.oracle_inner_moments.restype = None
        L.oracle_direct.argtypes = [i64, vp, vp, i32, vp, vp]
        L.oracle_direct.restype = None
        L.oracle_dtensors.argtypes = [vp, vp]
        L.oracle_dtensors.restype = None
        L.oracle_point_moments.argtypes = [i64, vp, vp, vp]
        L.oracle_point_moments.restype = None
        L.oracle_m2l.argtypes = [vp, vp, i32, vp, vp]
        L.oracle_m2l.restype = None
        L.oracle_local_eval.argtypes = [vp, vp, vp, vp]
        L.oracle_local_eval.restype = None
        L.oracle_fmm_sample_dt.argtypes = [vp, vp, vp, dbl, i32, i64, vp, vp]
        L.oracle_fmm_sample_dt.restype = None
        L.oracle_m2l_source.argtypes = [vp, vp, vp, vp]
        L.oracle_m2l_source.restype = None
        L.oracle_max_threads.argtypes = []
        L.oracle_max_threads.restype = i32
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Tree:
    """Octree of 8^3-cell subgrids built by the oracle from dense per-level refinement flags."""

    def __init__(self, max_level: int, flags: np.ndarray):
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        self._flags = flags
        h = lib().oracle_tree_build(int(max_level), _p(flags), int(flags.size))
        if not h:
            raise ValueError("oracle: invalid tree arguments")
        self._h = C.c_void_p(h)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.oracle_tree_free(self._h)
            self._h = None

    @property
    def depth(self) -> int:
        return lib().oracle_tree_depth(self._h)

    def subgrids(self) -> np.ndarray:
        """(n, 5) rows (level, i, j, k, is_leaf), by level then Morton key."""
        n = lib().oracle_tree_n_subgrids(self._h)
        out = np.empty((n, 5), dtype=np.int32)
        lib().oracle_tree_subgrids(self._h, _p(out))
        return out

    def leaves(self) -> np.ndarray:
        """(n_leaf_subgrids, 4) rows (level, i, j, k) in canonical leaf order."""
        s = self.subgrids()
        return s[s[:, 4] == 1][:, :4].copy()

    @property
    def n_leaf_cells(self) -> int:
        return int(lib().oracle_tree_n_leaf_subgrids(self._h)) * 512


def stencil(theta: float, parity: int) -> np.ndarray:
    """(n, 3) same-level interaction offsets for a cell of the given parity (x<<2|y<<1|z)."""
    n = lib().oracle_stencil(float(theta), int(parity), None, 0)
    out = np.empty((max(n, 1), 3), dtype=np.int32)
    lib().oracle_stencil(float(theta), int(parity), _p(out), n)
    return out[:n]


def solve(tree: Tree, rho: np.ndarray, theta: float, amc: bool = True,
          nthreads: int = 0) -> Tuple[np.ndarray, np.ndarray, dict]:
    rho = _f64(rho)
    n = tree.n_leaf_cells
    assert rho.shape == (n,)
    phi = np.empty(n)
    g = np.empty((n, 3))
    cnt = np.zeros(3, dtype=np.int64)
    lib().oracle_fmm_solve(tree._h, _p(rho), float(theta), int(bool(amc)), int(nthreads),
                           _p(phi), _p(g), _p(cnt))
    return phi, g, {"m2l": int(cnt[0]), "p2p_same": int(cnt[1]), "p2p_mixed": int(cnt[2])}


def sample(tree: Tree, rho: np.ndarray, theta: float, idx: np.ndarray, amc: bool = True,
           nthreads: int = 0, with_counts: bool = False):
    """phi, g at the listed leaf cells (and, with_counts, the interactions evaluated)."""
    rho = _f64(rho)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    phi = np.empty(idx.size)
    g = np.empty((idx.size, 3))
    cnt = np.zeros(3, dtype=np.int64)
    lib().oracle_fmm_sample(tree._h, _p(rho), float(theta), int(bool(amc)), int(nthreads),
                            int(idx.size), _p(idx), _p(phi), _p(g), _p(cnt))
    if with_counts:
        return phi, g, {"m2l": int(cnt[0]), "p2p_same": int(cnt[1]), "p2p_mixed": int(cnt[2])}
    return phi, g


def sample_given(tree: Tree, rho: np.ndarray, inner_mom: np.ndarray, theta: float,
                 idx: np.ndarray, amc: bool = True, nthreads: int = 0):
    """phi, g at the listed leaf cells with the refined cells' multipoles taken from inner_mom
    ((n_refined_cells, 40), as inner_moments returns them) instead of formed from rho."""
    rho = _f64(rho)
    inner_mom = _f64(inner_mom)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    phi = np.empty(idx.size)
    g = np.empty((idx.size, 3))
    lib().oracle_fmm_sample_given(tree._h, _p(rho), _p(inner_mom), float(theta), int(bool(amc)),
                                  int(nthreads), int(idx.size), _p(idx), _p(phi), _p(g))
    return phi, g


def solve_dt(tree: Tree, rho: np.ndarray, src: np.ndarray, theta: float, idx=None,
             nthreads: int = 0) -> np.ndarray:
    """dphi/dt (Sec. 2.1): the rho solve's operator applied to the source density src (d rho/dt),
    at every leaf cell or at the listed ones."""
    rho = _f64(rho)
    src = _f64(src)
    n = tree.n_leaf_cells
    assert rho.shape == (n,) and src.shape == (n,)
    if idx is None:
        out = np.empty(n)
        lib().oracle_fmm_sample_dt(tree._h, _p(rho), _p(src), float(theta), int(nthreads), n, None,
                                   _p(out))
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        out = np.empty(idx.size)
        lib().oracle_fmm_sample_dt(tree._h, _p(rho), _p(src), float(theta), int(nthreads),
                                   int(idx.size), _p(idx), _p(out))
    return out


def m2l_source(XA, XB, smB) -> np.ndarray:
    """Expansion (40 numbers) at centre XA due to source moments smB (S0, S1[3], S2[9], S3[27])
    about XB."""
    L = np.zeros(40)
    lib().oracle_m2l_source(_p(_f64(XA)), _p(_f64(XB)), _p(_f64(smB)), _p(L))
    return L


def inner_moments(tree: Tree, rho: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """(n_refined_cells, 40): m, X[3], M2[9], M3[27] of every cell of every refined subgrid."""
    rho = _f64(rho)
    s = tree.subgrids()
    n_inner = int((s[:, 4] == 0).sum())
    out = np.empty((n_inner * 512, 40))
    lib().oracle_inner_moments(tree._h, _p(rho), int(nthreads), _p(out))
    return out


def direct(x: np.ndarray, m: np.ndarray, nthreads: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    x = _f64(x)
    m = _f64(m)
    n = m.size
    phi = np.empty(n)
    g = np.empty((n, 3))
    lib().oracle_direct(int(n), _p(x), _p(m), int(nthreads), _p(phi), _p(g))
    return phi, g


def dtensors(R) -> Tuple[float, np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    R = _f64(R)
    out = np.empty(121)
    lib().oracle_dtensors(_p(R), _p(out))
    return (out[0], out[1:4].copy(), out[4:13].reshape(3, 3).copy(),
            out[13:40].reshape(3, 3, 3).copy(), out[40:121].reshape(3, 3, 3, 3).copy())


def point_moments(x: np.ndarray, m: np.ndarray) -> np.ndarray:
    x = _f64(x)
    m = _f64(m)
    out = np.empty(40)
    lib().oracle_point_moments(int(m.size), _p(x), _p(m), _p(out))
    return out


def m2l(momA: np.ndarray, momB: np.ndarray, amc: bool = True) -> Tuple[np.ndarray, np.ndarray]:
    momA = _f64(momA)
    momB = _f64(momB)
    L = np.zeros(40)
    ac = np.zeros(3)
    lib().oracle_m2l(_p(momA), _p(momB), int(bool(amc)), _p(L), _p(ac))
    return L, ac


def local_eval(L: np.ndarray, X: np.ndarray, y: np.ndarray) -> Tuple[float, np.ndarray]:
    L = _f64(L)
    X = _f64(X)
    y = _f64(y)
    out = np.empty(4)
    lib().oracle_local_eval(_p(L), _p(X), _p(y), _p(out))
    return out[0], out[1:4].copy()


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def leaf_masses(tree: Tree, rho: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Leaf-cell centres and point masses (rho * dx^3), for direct sums in tests."""
    from paper_2101_08226_gb300 import synth
    x, dx = synth.leaf_cell_centres(tree.leaves())
    return x, _f64(rho) * dx ** 3
