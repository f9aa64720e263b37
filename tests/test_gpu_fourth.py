"""Fourth-order methods on the GPU (Figures HO-SVDn and hooin with N = 4, sp4, mp4) against
the oracle: the order-4 HOOI projection for every output mode, all four methods pass by pass on
ragged tensors, exact recovery of planted tensors, and the paper's fourth-order workload (100^4,
10% density, core 20^4) checked through the core and fit of the returned factors."""
import numpy as np
import pytest

from oracle import tucker_oracle as O
from paper_0711_2023_gb300 import synth

pytestmark = pytest.mark.gpu


def rand_factor(n, j, seed):
    Q, _ = np.linalg.qr(synth.uniform_matrix(n, j, seed) - 0.5)
    return Q


@pytest.fixture(scope="module")
def ragged4(tucker_lib):
    X = synth.random_sparse_tensor_n((13, 9, 11, 7), 1500, synth.config_seed(41))
    return X, tucker_lib.tucker4_tensor_create(X.idx, X.val, X.dims)


def test_ttmc4_every_mode(tucker_lib, ragged4):
    X, T = ragged4
    J = (3, 4, 2, 5)
    U = [rand_factor(X.dims[a], J[a], 70 + a) for a in range(4)]
    for n in range(4):
        Y = tucker_lib.tucker4_ttmc(T, n, U).cpu().numpy()
        ref = O.unfold_dense(O.ttmc_n(X.dims, X.idx, X.val, n, U), n)
        assert np.abs(Y - ref).max() <= 1e-12 * np.abs(ref).max(), n


def run_gpu(tk, alg, T, J, sweeps, tol, D_raw=None, init=None):
    if alg == "hosvd":
        return tk.tucker4_hosvd(T, J)
    if alg == "hooi":
        return tk.tucker4_hooi(T, J, tol=tol, max_iter=sweeps, init=init)
    if alg == "sp":
        return tk.tucker4_sp(T, J, D_raw, tol=tol, max_iter=sweeps)
    return tk.tucker4_mp(T, J, tol=tol, max_iter=sweeps, init=init)


def run_oracle(alg, X, J, sweeps, tol, D_raw=None, init=None):
    if alg == "hosvd":
        return O.hosvd_n(X.dims, X.idx, X.val, J)
    if alg == "hooi":
        return O.hooi_n(X.dims, X.idx, X.val, J, tol, sweeps, init=init)
    if alg == "sp":
        return O.sp4(X.dims, X.idx, X.val, J, D_raw, tol, sweeps)
    return O.mp4(X.dims, X.idx, X.val, J, tol, sweeps, init=init)


@pytest.mark.parametrize("alg", ["hosvd", "hooi", "sp", "mp"])
@pytest.mark.parametrize("tol", [-np.inf, 1e-4])
def test_methods_vs_oracle(tucker_lib, ragged4, alg, tol):
    X, T = ragged4
    J = (3, 4, 2, 3)
    D_raw = synth.uniform_matrix(X.dims[3], J[3], 88)
    g = run_gpu(tucker_lib, alg, T, J, 4, tol, D_raw)
    r = run_oracle(alg, X, J, 4, tol, D_raw)
    assert g["iters"] == r["iters"], (g["fit_history"], r["fit_history"])
    for a, b in zip(g["fit_history"], r["fit_history"]):
        assert abs(a - b) <= 1e-9, (alg, g["fit_history"], r["fit_history"])
    for u in g["U"]:
        u = u.cpu().numpy()
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() <= 1e-12


@pytest.mark.parametrize("alg", ["hosvd", "hooi", "sp", "mp"])
def test_exact_recovery_planted(tucker_lib, alg):
    core, support = (3, 2, 3, 2), (6, 5, 7, 4)
    X, G, F = synth.planted_tensor_n((9, 8, 10, 7), core, support, 123)
    T = tucker_lib.tucker4_tensor_create(X.idx, X.val, X.dims)
    D_raw = synth.uniform_matrix(7, 2, 89)
    g = run_gpu(tucker_lib, alg, T, core, 10, 1e-12, D_raw)
    assert g["fit"] >= 1 - 1e-7
    for a in range(4):
        assert O.subspace_distance(g["U"][a].cpu().numpy(), F[a]) <= 1e-6


def test_errors(tucker_lib, ragged4):
    import ctypes
    X, T = ragged4
    with pytest.raises(tucker_lib.TuckerError):                 # SP needs its random D
        tucker_lib._run4("tucker4_sp", T, (2, 2, 2, 2), -np.inf, 2, None)
    bad = X.idx.copy()
    bad[3, 5] = X.dims[3]                                        # index out of range
    with pytest.raises(tucker_lib.TuckerError) as e:
        tucker_lib.tucker4_tensor_create(bad, X.val, X.dims)
    assert e.value.status == tucker_lib.TUCKER_EINVAL
    # the mixed form is not offered for order four
    o = tucker_lib.tucker4_opts()
    o.precision, o.tol, o.max_iter = tucker_lib.TUCKER_MIXED, 1e-4, 2
    r = tucker_lib.tucker4_result()
    st = tucker_lib._lib().tucker4_hooi(T.handle, (ctypes.c_int32 * 4)(2, 2, 2, 2),
                                        ctypes.byref(o), ctypes.byref(r))
    assert st == tucker_lib.TUCKER_EINVAL


# ---- the paper's fourth-order workload ----------------------------------------------------------

@pytest.fixture(scope="module")
def paper4(tucker_lib):
    X = synth.random_sparse_tensor_n((100, 100, 100, 100), 10_000_000, synth.config_seed(400))
    return X, tucker_lib.tucker4_tensor_create(X.idx, X.val, X.dims)


def check_core_fit(X, g):
    U = [u.cpu().numpy() for u in g["U"]]
    G = O.core_n(X.dims, X.idx, X.val, U)
    assert np.abs(G - g["G"].cpu().numpy()).max() <= 1e-11 * np.abs(G).max()
    assert abs(O.fit_from_core(O.norm2(X.val), G) - g["fit"]) <= 1e-9
    return U


@pytest.mark.parametrize("alg", ["hosvd", "hooi", "sp", "mp"])
def test_paper_workload_100x4(tucker_lib, paper4, alg):
    X, T = paper4
    J = (20, 20, 20, 20)
    D_raw = synth.uniform_matrix(100, 20, synth.config_seed(401))
    g = run_gpu(tucker_lib, alg, T, J, 2, -np.inf, D_raw)
    U = check_core_fit(X, g)
    if alg == "hooi":
        # the last factor spans the leading eigenspace of Gram(Z_(4)) built from A, B, C
        Z = O.unfold_dense(O.ttmc_n(X.dims, X.idx, X.val, 3, U), 3)
        M = O.gram(Z)
        w = np.linalg.eigvalsh(M)[::-1]
        assert abs(np.trace(U[3].T @ M @ U[3]) - w[:20].sum()) <= 1e-11 * w[:20].sum()
    # paper rows for core 20^4 (Section 4.3 results table), two passes from the start
    assert 3.85 <= 100 * g["fit"] <= 3.95
