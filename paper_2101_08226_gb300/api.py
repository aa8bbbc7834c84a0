"""Thin Python API over the C ABI.  PyTorch provides device memory and streams only; every step
of the solve runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes as C
from typing import Optional, Tuple

import numpy as np

from . import _lib
from ._lib import check, lib

PRECISIONS = {"fp64": _lib.FMM_FP64, "mixed": _lib.FMM_MIXED, "df64": _lib.FMM_DF64}


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


# the entries of the SCF state (octo_fmm.h, FMM_SCF_STATE), in order
SCF_STATE_KEYS = ("K", "Omega", "C1", "C2", "x_L1", "phi_L1", "X1x", "X1y", "X1z", "X2x", "X2y",
                  "X2z", "Xcmx", "Xcmy", "Xcmz", "a", "M1_raw", "M2_raw", "rho1", "rho2", "phi1",
                  "phiC")


def _scf_params(p: dict):
    return _lib.ScfParams(float(p["M1"]), float(p["M2"]), float(p["n"]), float(p["f"]),
                          float(p["J0"]), float(p["rho_floor"]), float(p.get("theta", 0.5)),
                          PRECISIONS[p.get("precision", "fp64")])


def measure_fma_rate(bits: int, reps: int = 5, stream=None) -> Tuple[float, float]:
    """fmm_measure_fma_rate: (TFLOP/s of fused multiply-adds at 2 flops each, ms per launch) of the
    FP64 (bits = 64) or FP32 (bits = 32; _lib.FMM_FMA_F32X2: packed pairs, one instruction per
    two FMAs) pipes of the current device."""
    tf, ms = C.c_double(), C.c_double()
    check(lib().fmm_measure_fma_rate(int(bits), int(reps), C.byref(tf), C.byref(ms),
                                     _stream_handle(stream)))
    return tf.value, ms.value


def stencil(theta: float, parity: int) -> np.ndarray:
    n = C.c_int32(0)
    check(lib().fmm_stencil(float(theta), int(parity), None, 0, C.byref(n)))
    out = np.empty((max(n.value, 1), 3), dtype=np.int32)
    check(lib().fmm_stencil(float(theta), int(parity), _p(out), n.value, C.byref(n)))
    return out[:n.value]


class Tree:
    """Octree of 8^3-cell subgrids owned by the CUDA library (fmm_build_tree / fmm_destroy)."""

    def __init__(self, max_level: int, flags: np.ndarray):
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        h = C.c_void_p()
        check(lib().fmm_build_tree(int(max_level), _p(flags), int(flags.size), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().fmm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forest_info(self) -> Tuple[int, np.ndarray]:
        """(number of trees, leaf-subgrid offsets [n_trees + 1])."""
        n = C.c_int32()
        check(lib().fmm_forest_info(self._h, C.byref(n), None))
        off = np.zeros(n.value + 1, dtype=np.int64)
        check(lib().fmm_forest_info(self._h, C.byref(n), _p(off)))
        return n.value, off

    def info(self) -> Tuple[int, int, int]:
        ns, nl, d = C.c_int64(), C.c_int64(), C.c_int32()
        check(lib().fmm_tree_info(self._h, C.byref(ns), C.byref(nl), C.byref(d)))
        return ns.value, nl.value, d.value

    @property
    def n_leaf_cells(self) -> int:
        return self.info()[1] * 512

    def subgrids(self) -> np.ndarray:
        out = np.empty((self.info()[0], 5), dtype=np.int32)
        check(lib().fmm_tree_subgrids(self._h, _p(out)))
        return out

    def leaves(self) -> np.ndarray:
        s = self.subgrids()
        return s[s[:, 4] == 1][:, :4].copy()

    def counts(self, theta: float) -> dict:
        out = np.zeros(3, dtype=np.int64)
        check(lib().fmm_interaction_counts(self._h, float(theta), _p(out)))
        return {"m2l": int(out[0]), "p2p_same": int(out[1]), "p2p_mixed": int(out[2])}

    def counts_by_type(self, theta: float) -> dict:
        out = np.zeros(6, dtype=np.int64)
        check(lib().fmm_interaction_counts_by_type(self._h, float(theta), _p(out)))
        keys = ("m2l_leaf_leaf", "m2l_leaf_refined", "m2l_refined_leaf", "m2l_refined_refined",
                "p2p_same", "p2p_mixed")
        return dict(zip(keys, (int(v) for v in out)))

    def partition(self, n_ranks: int, cut_level: int) -> np.ndarray:
        """fmm_partition: the rank of every subgrid (-1: kept by every rank)."""
        out = np.empty(self.info()[0], dtype=np.int32)
        check(lib().fmm_partition(self._h, int(n_ranks), int(cut_level), _p(out)))
        return out

    def ghosts(self, owner: np.ndarray, rank: int) -> np.ndarray:
        """fmm_ghosts: the subgrids other ranks own whose data `rank` reads."""
        owner = np.ascontiguousarray(owner, dtype=np.int32)
        n = C.c_int64()
        check(lib().fmm_ghosts(self._h, _p(owner), int(rank), None, 0, C.byref(n)))
        out = np.empty(max(n.value, 1), dtype=np.int32)
        check(lib().fmm_ghosts(self._h, _p(owner), int(rank), _p(out), n.value, C.byref(n)))
        return out[:n.value]

    def last_launches(self) -> int:
        n = C.c_int32()
        check(lib().fmm_last_launches(self._h, C.byref(n)))
        return n.value

    def solve(self, rho, theta: float, precision: str = "fp64", amc: bool = True, phi=None,
              g=None, net=None, stream=None, check_status: bool = True):
        """rho: CUDA float64 tensor [n_leaf].  Returns (phi, g, net) CUDA tensors."""
        import torch
        n = self.n_leaf_cells
        assert rho.is_cuda and rho.dtype == torch.float64 and rho.is_contiguous() and rho.numel() == n
        if phi is None:
            phi = torch.empty(n, dtype=torch.float64, device=rho.device)
        if g is None:
            g = torch.empty((n, 3), dtype=torch.float64, device=rho.device)
        if net is None:
            net = torch.empty(7 * self.forest_info()[0], dtype=torch.float64, device=rho.device)
        sh = _stream_handle(stream)
        check(lib().fmm_solve(self._h, rho.data_ptr(), float(theta), PRECISIONS[precision],
                              int(bool(amc)), phi.data_ptr(), g.data_ptr(),
                              net.data_ptr() if net is not False else None, sh))
        if check_status:
            check(lib().fmm_sync_status(self._h, sh))
        return phi, g, net

    def solve_dt(self, rho, rhodot, theta: float, precision: str = "fp64", amc: bool = True,
                 phi=None, g=None, phidot=None, net=None, stream=None, check_status: bool = True):
        """fmm_solve_dt: (phi, g, phidot, net) for CUDA float64 tensors rho and rhodot [n_leaf]."""
        import torch
        n = self.n_leaf_cells
        for x in (rho, rhodot):
            assert x.is_cuda and x.dtype == torch.float64 and x.is_contiguous() and x.numel() == n
        phi = torch.empty(n, dtype=torch.float64, device=rho.device) if phi is None else phi
        g = torch.empty((n, 3), dtype=torch.float64, device=rho.device) if g is None else g
        phidot = torch.empty(n, dtype=torch.float64, device=rho.device) if phidot is None else phidot
        if net is None:
            net = torch.empty(7 * self.forest_info()[0], dtype=torch.float64, device=rho.device)
        sh = _stream_handle(stream)
        check(lib().fmm_solve_dt(self._h, rho.data_ptr(), rhodot.data_ptr(), float(theta),
                                 PRECISIONS[precision], int(bool(amc)), phi.data_ptr(), g.data_ptr(),
                                 phidot.data_ptr(), net.data_ptr() if net is not False else None, sh))
        if check_status:
            check(lib().fmm_sync_status(self._h, sh))
        return phi, g, phidot, net

    def binary_diagnostics(self, rho, g, omega: float, x1, x2, rc1: float = 0.0, rc2: float = 0.0,
                           member: bool = False, stream=None):
        """One pass of fmm_binary_diagnostics.  Returns the (2, 11) per-star sums (M, sum m x,
        F, T about x_s, cell count) as a host array, and the membership tensor if asked."""
        import torch
        n = self.n_leaf_cells
        assert rho.numel() == n and g.numel() == 3 * n
        out = torch.empty(22, dtype=torch.float64, device=rho.device)
        mem = torch.empty(n, dtype=torch.int8, device=rho.device) if member else None
        c1 = (C.c_double * 3)(*[float(v) for v in x1])
        c2 = (C.c_double * 3)(*[float(v) for v in x2])
        sh = _stream_handle(stream)
        check(lib().fmm_binary_diagnostics(self._h, rho.data_ptr(), g.data_ptr(), float(omega), c1,
                                           c2, float(rc1), float(rc2), out.data_ptr(),
                                           mem.data_ptr() if mem is not None else None, sh))
        res = out.cpu().numpy().reshape(2, 11)
        return (res, mem) if member else res

    def binary_iterate(self, rho, g, omega: float, x1, x2, n_iter: int = 5, stream=None):
        """fmm_binary_iterate: n_iter diagnostics passes, each with the centres and critical radii
        the library derives on the device from the previous pass.  Returns the last pass's (2, 11)
        sums, its membership tensor, the centres it used and the orbital torque, as host arrays."""
        import torch
        n = self.n_leaf_cells
        assert rho.numel() == n and g.numel() == 3 * n
        dev = rho.device
        out = torch.empty(22, dtype=torch.float64, device=dev)
        cen = torch.empty(6, dtype=torch.float64, device=dev)
        torb = torch.empty(3, dtype=torch.float64, device=dev)
        mem = torch.empty(n, dtype=torch.int8, device=dev)
        c1 = (C.c_double * 3)(*[float(v) for v in x1])
        c2 = (C.c_double * 3)(*[float(v) for v in x2])
        check(lib().fmm_binary_iterate(self._h, rho.data_ptr(), g.data_ptr(), float(omega), c1, c2,
                                       int(n_iter), out.data_ptr(), cen.data_ptr(), torb.data_ptr(),
                                       mem.data_ptr(), _stream_handle(stream)))
        cen = cen.cpu().numpy()
        return (out.cpu().numpy().reshape(2, 11), mem, (cen[:3], cen[3:]), torb.cpu().numpy())

    def scf_init(self, params: dict, rho, K0: float, stream=None):
        """fmm_scf_init: the solve of the initial density and the initial SCF state.  params:
        M1, M2, n, f, J0, rho_floor, theta, precision ("fp64" / "mixed" / "df64").  Returns
        (phi, g) of the initial solve."""
        import torch
        n = self.n_leaf_cells
        assert rho.is_cuda and rho.dtype == torch.float64 and rho.numel() == n
        phi = torch.empty(n, dtype=torch.float64, device=rho.device)
        g = torch.empty((n, 3), dtype=torch.float64, device=rho.device)
        check(lib().fmm_scf_init(self._h, C.byref(_scf_params(params)), rho.data_ptr(), float(K0),
                                 phi.data_ptr(), g.data_ptr(), _stream_handle(stream)))
        return phi, g

    def scf_iterate(self, params: dict, rho, n_iter: int, phi=None, g=None, stream=None):
        """fmm_scf_iterate: n_iter SCF iterations on the CUDA float64 density rho (updated in
        place).  Returns (state dict, history array (n_iter, FMM_SCF_STATE), phi, g)."""
        import torch
        n = self.n_leaf_cells
        assert rho.is_cuda and rho.dtype == torch.float64 and rho.numel() == n
        dev = rho.device
        phi = torch.empty(n, dtype=torch.float64, device=dev) if phi is None else phi
        g = torch.empty((n, 3), dtype=torch.float64, device=dev) if g is None else g
        state = torch.empty(_lib.FMM_SCF_STATE, dtype=torch.float64, device=dev)
        hist = torch.empty((max(n_iter, 1), _lib.FMM_SCF_STATE), dtype=torch.float64, device=dev)
        check(lib().fmm_scf_iterate(self._h, C.byref(_scf_params(params)), int(n_iter),
                                    rho.data_ptr(), phi.data_ptr(), g.data_ptr(), state.data_ptr(),
                                    hist.data_ptr(), _stream_handle(stream)))
        st = state.cpu().numpy()
        return dict(zip(SCF_STATE_KEYS, (float(v) for v in st))), hist.cpu().numpy()[:n_iter], phi, g

    def sync_status(self, stream=None):
        check(lib().fmm_sync_status(self._h, _stream_handle(stream)))

    def solve_host(self, rho: np.ndarray, theta: float, precision: str = "fp64", amc: bool = True,
                   phi: Optional[np.ndarray] = None, g: Optional[np.ndarray] = None,
                   net: Optional[np.ndarray] = None, stream=None):
        """Host buffers in and out (the copies are part of the call)."""
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        n = self.n_leaf_cells
        assert rho.size == n
        phi = np.empty(n) if phi is None else phi
        g = np.empty((n, 3)) if g is None else g
        net = np.empty(7 * self.forest_info()[0]) if net is None else net
        check(lib().fmm_solve_host(self._h, _p(rho), float(theta), PRECISIONS[precision],
                                   int(bool(amc)), _p(phi), _p(g), _p(net),
                                   _stream_handle(stream)))
        return phi, g, net

    def solve_host_async(self, rho: np.ndarray, theta: float, precision: str, phi: np.ndarray,
                         g: np.ndarray, net: Optional[np.ndarray] = None, amc: bool = True,
                         stream=None):
        """fmm_solve_host_async: enqueue one host-buffer solve of a pipelined sequence; the buffers
        (pinned, contiguous float64) must stay untouched until sync_status()."""
        n = self.n_leaf_cells
        assert rho.size == n and phi.size == n and g.size == 3 * n
        for a in (rho, phi, g) + ((net,) if net is not None else ()):
            assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
        check(lib().fmm_solve_host_async(self._h, _p(rho), float(theta), PRECISIONS[precision],
                                         int(bool(amc)), _p(phi), _p(g),
                                         _p(net) if net is not None else None,
                                         _stream_handle(stream)))

    def net_force_torque(self, rho, g, stream=None):
        import torch
        net = torch.empty(7 * self.forest_info()[0], dtype=torch.float64, device=rho.device)
        sh = _stream_handle(stream)
        check(lib().fmm_net_force_torque(self._h, rho.data_ptr(), g.data_ptr(), net.data_ptr(), sh))
        check(lib().fmm_sync_status(self._h, sh))
        return net

    def set_profiling(self, on: bool = True):
        check(lib().fmm_set_profiling(self._h, int(bool(on))))

    def set_graphs(self, on: bool = True):
        """Replay one captured CUDA graph per solve configuration (the default), or launch the
        kernels one by one."""
        check(lib().fmm_set_graphs(self._h, int(bool(on))))

    def set_persistent(self, on: bool = True):
        """Level passes as one persistent, level-ordered launch per direction, or one launch per
        phase (the default) (fmm_set_persistent)."""
        check(lib().fmm_set_persistent(self._h, int(bool(on))))

    def set_variant(self, theta: float, variant: int):
        """Launch variant of the mixed path for this tree and theta (fmm_set_variant)."""
        check(lib().fmm_set_variant(self._h, float(theta), int(variant)))

    def autotune(self, rho, theta: float, precision: str = "mixed", amc: bool = True, reps: int = 5,
                 stream=None):
        """fmm_autotune on the CUDA float64 density rho: returns (chosen variant, median ms per
        variant, phi, g of the chosen variant)."""
        import torch
        n = self.n_leaf_cells
        assert rho.is_cuda and rho.dtype == torch.float64 and rho.is_contiguous() and rho.numel() == n
        phi = torch.empty(n, dtype=torch.float64, device=rho.device)
        g = torch.empty((n, 3), dtype=torch.float64, device=rho.device)
        ms = np.zeros(_lib.FMM_MIXED_VARIANTS, dtype=np.float32)
        v = C.c_int32()
        check(lib().fmm_autotune(self._h, rho.data_ptr(), float(theta), PRECISIONS[precision],
                                 int(bool(amc)), phi.data_ptr(), g.data_ptr(), int(reps), _p(ms),
                                 C.byref(v), _stream_handle(stream)))
        n_var = _lib.FMM_MIXED_VARIANTS if precision == "mixed" else 1
        return v.value, ms[:n_var], phi, g

    def set_wait_limit(self, cycles: int = 0):
        """Limit, in SM clock cycles, of the staging kernel's wait for each parity class's
        copies (0: the default, about a second); a wait that runs out is reported by the next
        status check as FMM_ERR_TIMEOUT."""
        check(lib().fmm_set_wait_limit(self._h, int(cycles)))

    def phase_times(self) -> np.ndarray:
        """ms of the last profiled solve: upward, interactions, downward, reductions, then the
        end of the leaf kernel to the end of the interactions, the leaf kernel, and (mixed) the
        refined targets' kernel on the second stream (fmm_phase_times)."""
        out = np.zeros(7, dtype=np.float32)
        check(lib().fmm_phase_times(self._h, _p(out), 7))
        return out


class Forest(Tree):
    """Independent trees solved together (fmm_build_forest): per-cell arrays are the trees'
    arrays back to back, net sums 7 per tree."""

    def __init__(self, trees):
        arr = (C.c_void_p * len(trees))(*[t._h for t in trees])
        h = C.c_void_p()
        check(lib().fmm_build_forest(arr, len(trees), C.byref(h)))
        self._h = h

    def solve_batch(self, rhos, theta: float, precision: str = "fp64", amc: bool = True,
                    phis=None, gs=None, net=None, stream=None, check_status: bool = True):
        """One device buffer per tree (fmm_solve_batch)."""
        import torch
        n, off = self.forest_info()
        sizes = (off[1:] - off[:-1]) * 512
        dev = rhos[0].device
        phis = phis or [torch.empty(int(m), dtype=torch.float64, device=dev) for m in sizes]
        gs = gs or [torch.empty((int(m), 3), dtype=torch.float64, device=dev) for m in sizes]
        if net is None:
            net = torch.empty(7 * n, dtype=torch.float64, device=dev)
        P = C.c_void_p * n
        sh = _stream_handle(stream)
        check(lib().fmm_solve_batch(self._h, P(*[r.data_ptr() for r in rhos]), float(theta),
                                    PRECISIONS[precision], int(bool(amc)),
                                    P(*[p.data_ptr() for p in phis]), P(*[x.data_ptr() for x in gs]),
                                    net.data_ptr(), sh))
        if check_status:
            check(lib().fmm_sync_status(self._h, sh))
        return phis, gs, net
