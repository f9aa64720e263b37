"""The remaining paper-shaped workloads, at full size, on the GPU:

* 500^3 with 2.5e6 nonzeros and cores (50,50,50), (25,50,100), (10,50,250), (250,50,10): all four
  methods, FP64 against the oracle (fit within 1e-9 at every pass) and the mixed form against
  the FP64 path (fit within 1e-4);
* 2000^3 with 4e7 nonzeros, core 100^3: HOOI and MP in the mixed form against the FP64 path
  (fit within 1e-4), and the oracle's own core and fit from the mixed factors;
* the same tensor in the benchmark's launch configuration (one HOOI pass and one MP pass from
  the HO-SVD start of B and C, FP64): the oracle's core and fit from the returned factors, the
  first factor against the leading eigenspace of the matrix the start defines, and the last
  factor against the leading eigenspace of the matrix built from the returned factors."""
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


def check_core_fit(X, g, tol_fit=1e-9):
    U = [u.cpu().numpy() for u in g["U"]]
    for u in U:
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() <= 1e-12
    G = O.core(X.dims, X.idx, X.val, U)
    assert np.abs(G - g["G"].cpu().numpy()).max() <= 1e-11 * np.abs(G).max()
    fit = O.fit_from_core(O.norm2(X.val), G)
    assert abs(fit - g["fit"]) <= tol_fit, (fit, g["fit"])
    return U


def check_leading(M, V):
    """V (orthonormal columns) spans the leading eigenspace of the PSD matrix M: the trace of
    V^T M V equals the sum of the J largest eigenvalues."""
    w = np.linalg.eigvalsh(M)[::-1]
    Jn = V.shape[1]
    top = np.trace(V.T @ M @ V)
    assert abs(top - w[:Jn].sum()) <= 1e-11 * w[:Jn].sum()


@pytest.fixture(scope="module")
def hosvd_start_2000(tucker_lib, t2000):
    X, T = t2000
    g = tucker_lib.tucker_hosvd(T, (100, 100, 100))
    return [None, g["U"][1].cpu().numpy(), g["U"][2].cpu().numpy()]


def test_2000cube_hooi_fp64_one_pass(tucker_lib, t2000, hosvd_start_2000):
    X, T = t2000
    J = (100, 100, 100)
    init = hosvd_start_2000
    g = tucker_lib.tucker_hooi(T, J, tol=-np.inf, max_iter=1, init=init)
    assert g["iters"] == 1
    U = check_core_fit(X, g)
    # A from the start's B, C; C from the returned A, B (Figure hooi3)
    Y0 = O.ttmc(X.dims, X.idx, X.val, 0, [None, init[1], init[2]])
    check_leading(O.gram(O.unfold_dense(Y0, 0)), U[0])
    W = O.ttmc(X.dims, X.idx, X.val, 2, U)
    check_leading(O.gram(O.unfold_dense(W, 2)), U[2])


def test_2000cube_mp_fp64_one_pass(tucker_lib, t2000, hosvd_start_2000):
    X, T = t2000
    J = (100, 100, 100)
    init = hosvd_start_2000
    g = tucker_lib.tucker_mp(T, J, tol=-np.inf, max_iter=1, init=init)
    assert g["iters"] == 1
    U = check_core_fit(X, g)
    # C from the returned A, B: Gram((X x_2 B^T)_(3)) + Gram((X x_1 A^T)_(3)) (Figure mp3)
    M3 = O.gram(O.unfold_dense(O.ttm(X.dims, X.idx, X.val, 1, U[1]), 2))
    M3 += O.gram(O.unfold_dense(O.ttm(X.dims, X.idx, X.val, 0, U[0]), 2))
    check_leading(M3, U[2])
