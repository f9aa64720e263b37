"""The remaining paper-shaped workloads, at full size, on the GPU:

* 500^3 with 2.5e6 nonzeros and cores (50,50,50), (25,50,100), (10,50,250), (250,50,10): all four
  methods, FP64 against the oracle (fit within 1e-9 at every pass) and the mixed form against
  the FP64 path (fit within 1e-4);
* 2000^3 with 4e7 nonzeros, core 100^3: HOOI and MP in the mixed form against the FP64 path
  (fit within 1e-4), and the oracle's own core and fit from the mixed factors."""
import numpy as np
import pytest

from oracle import tucker_oracle as O
from paper_0711_2023_gb300 import synth

pytestmark = pytest.mark.gpu

CORES_500 = [(50, 50, 50), (25, 50, 100), (10, 50, 250), (250, 50, 10)]


@pytest.fixture(scope="module")
def t500(tucker_lib):
    X = synth.random_sparse_tensor((500, 500, 500), 2_500_000, synth.config_seed(3))
    return X, tucker_lib.tucker_tensor_create(X.idx, X.val, X.dims)


def run(tk, alg, T, J, C_raw, precision, sweeps):
    if alg == "hosvd":
        return tk.tucker_hosvd(T, J, precision=precision)
    if alg == "hooi":
        return tk.tucker_hooi(T, J, tol=-np.inf, max_iter=sweeps, precision=precision)
    if alg == "sp":
        return tk.tucker_sp(T, J, C_raw, tol=-np.inf, max_iter=sweeps, precision=precision)
    return tk.tucker_mp(T, J, tol=-np.inf, max_iter=sweeps, precision=precision)


def oracle(alg, X, J, C_raw, sweeps):
    if alg == "hosvd":
        return O.hosvd(X.dims, X.idx, X.val, J)
    if alg == "hooi":
        return O.hooi(X.dims, X.idx, X.val, J, -np.inf, sweeps)
    if alg == "sp":
        return O.sp(X.dims, X.idx, X.val, J, C_raw, -np.inf, sweeps)
    return O.mp(X.dims, X.idx, X.val, J, -np.inf, sweeps)


@pytest.mark.parametrize("J", CORES_500)
@pytest.mark.parametrize("alg", ["hosvd", "hooi", "sp", "mp"])
def test_500cube_core_ratios(tucker_lib, t500, alg, J):
    X, T = t500
    C_raw = synth.uniform_matrix(500, J[2], synth.config_seed(4))
    g64 = run(tucker_lib, alg, T, J, C_raw, "fp64", 2)
    gmx = run(tucker_lib, alg, T, J, C_raw, "mixed", 2)
    r = oracle(alg, X, J, C_raw, 2)
    assert g64["iters"] == r["iters"] == gmx["iters"]
    for a, b in zip(g64["fit_history"], r["fit_history"]):
        assert abs(a - b) <= 1e-9, (alg, J, g64["fit_history"], r["fit_history"])
    for a, b in zip(gmx["fit_history"], g64["fit_history"]):
        assert abs(a - b) <= 1e-4, (alg, J, gmx["fit_history"], g64["fit_history"])


@pytest.fixture(scope="module")
def t2000(tucker_lib):
    X = synth.random_sparse_tensor((2000, 2000, 2000), 40_000_000, synth.config_seed(2))
    return X, tucker_lib.tucker_tensor_create(X.idx, X.val, X.dims)


@pytest.mark.parametrize("alg,sweeps", [("hooi", 2), ("mp", 1)])
def test_2000cube_mixed_vs_fp64(tucker_lib, t2000, alg, sweeps):
    X, T = t2000
    J = (100, 100, 100)
    gmx = run(tucker_lib, alg, T, J, None, "mixed", sweeps)
    g64 = run(tucker_lib, alg, T, J, None, "fp64", sweeps)
    for a, b in zip(gmx["fit_history"], g64["fit_history"]):
        assert abs(a - b) <= 1e-4, (gmx["fit_history"], g64["fit_history"])
    U = [u.cpu().numpy() for u in gmx["U"]]
    for u in U:
        assert np.abs(u.T @ u - np.eye(100)).max() <= 1e-12
    if alg == "hooi":
        # the oracle's core and fit from the mixed form's factors
        G = O.core(X.dims, X.idx, X.val, U)
        fit = O.fit_from_core(O.norm2(X.val), G)
        assert abs(fit - gmx["fit"]) <= 1e-6
