"""The self-consistent-field iteration on the GPU (fmm_scf_init / fmm_scf_iterate, Sec. 4.1)
against the oracle's iteration (oracle/scf.py with the oracle's gravity solve) on the same binary
and inputs: the FP64 iteration follows the oracle's state after every iteration and its
densities; the mixed-precision solves converge to the same model within the mixed path's error."""
import numpy as np
import pytest

import oracle as O
import scf_case
from oracle import scf as S
from paper_2101_08226_gb300 import _lib, api, build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_ITER = 6


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


@pytest.fixture(scope="module")
def case():
    fld, flags = scf_case.workload()
    t = api.Tree(scf_case.LEVELS, flags)
    b = O.Tree(scf_case.LEVELS, flags)
    assert np.array_equal(t.subgrids(), b.subgrids())
    params, rho0, K0 = scf_case.inputs(fld, b.leaves())
    P = scf_case.oracle_problem(params, b.leaves())
    st, out = S.run(b, P, rho0, K0, N_ITER)
    return t, params, rho0, K0, out


def test_scf_fp64_follows_oracle(case):
    t, params, rho0, K0, out = case
    r = torch.from_numpy(rho0.copy()).cuda()
    t.scf_init(dict(params, precision="fp64"), r, K0)
    state, hist, phi, g = t.scf_iterate(dict(params, precision="fp64"), r, N_ITER)
    for k in range(N_ITER):
        ref = out[k]["state"]
        got = dict(zip(api.SCF_STATE_KEYS, hist[k]))
        for key in api.SCF_STATE_KEYS:
            scale = max(abs(ref[key]), 1e-6 if key.startswith(("X", "x")) else 0.0)
            assert abs(got[key] - ref[key]) <= 1e-9 * scale, (k, key, got[key], ref[key])
    rho = r.cpu().numpy()
    assert np.abs(rho - out[-1]["rho"]).max() <= 1e-9 * out[-1]["rho"].max()
    assert state == dict(zip(api.SCF_STATE_KEYS, (float(v) for v in hist[-1])))
    # the last solve's potential is that of the last scaled density
    assert np.abs(phi.cpu().numpy() - out[-1]["phi"]).max() <= 1e-9 * np.abs(out[-1]["phi"]).max()


def test_scf_continues_across_calls(case):
    """Two calls of 3 iterations end where one call of 6 does (the state lives on the device)."""
    t, params, rho0, K0, out = case
    p = dict(params, precision="fp64")
    r = torch.from_numpy(rho0.copy()).cuda()
    t.scf_init(p, r, K0)
    t.scf_iterate(p, r, 3)
    state, _, _, _ = t.scf_iterate(p, r, 3)
    ref = out[5]["state"]
    for key in ("K", "Omega", "C1", "C2", "x_L1"):
        assert abs(state[key] - ref[key]) <= 1e-9 * abs(ref[key])


def test_scf_mixed_converges_to_the_same_model(case):
    t, params, rho0, K0, out = case
    p = dict(params, precision="mixed")
    r = torch.from_numpy(rho0.copy()).cuda()
    t.scf_init(p, r, K0)
    state, _, _, _ = t.scf_iterate(p, r, N_ITER)
    ref = out[-1]["state"]
    for key in ("K", "Omega", "C1", "C2", "a"):
        assert abs(state[key] - ref[key]) <= 1e-4 * abs(ref[key]), (key, state[key], ref[key])
    assert state["x_L1"] == ref["x_L1"]


def test_scf_argument_checks(case):
    t, params, rho0, K0, out = case
    fld, flags = scf_case.workload()
    fresh = api.Tree(scf_case.LEVELS, flags)
    r = torch.from_numpy(rho0.copy()).cuda()
    with pytest.raises(_lib.FmmError) as e:   # no initial state yet
        fresh.scf_iterate(dict(params, precision="fp64"), r, 1)
    assert e.value.code == _lib.FMM_ERR_STATE
    with pytest.raises(_lib.FmmError) as e:
        fresh.scf_init(dict(params, f=1.5), r, K0)
    assert e.value.code == _lib.FMM_ERR_ARG
    f = api.Forest([fresh, t])
    with pytest.raises(_lib.FmmError) as e:
        f.scf_init(dict(params), torch.zeros(f.n_leaf_cells, dtype=torch.float64, device="cuda"), K0)
    assert e.value.code == _lib.FMM_ERR_ARG
