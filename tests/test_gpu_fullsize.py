"""Full-size checks on the 1000^3 workload (1e7 nonzeros, core 50^3) for all four methods.  The oracle cannot run every pass at this size, so it checks
what it can compute directly from the GPU's output: the core and fit of the returned factors
(which must equal the GPU's own), and that the last factor updated spans the leading
eigenspace of the matrix the method defines for it (built by the oracle from the other
returned factors)."""
import numpy as np
import pytest

from oracle import tucker_oracle as O
from paper_0711_2023_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS, NNZ, J = (1000, 1000, 1000), 10_000_000, (50, 50, 50)


@pytest.fixture(scope="module")
def big(tucker_lib):
    X = synth.random_sparse_tensor(DIMS, NNZ, synth.config_seed(1))
    T = tucker_lib.tucker_tensor_create(X.idx, X.val, X.dims)
    return X, T


def check_core_fit(X, g):
    U = [u.cpu().numpy() for u in g["U"]]
    for u in U:
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() <= 1e-12
    G = O.core(X.dims, X.idx, X.val, U)
    assert np.abs(G - g["G"].cpu().numpy()).max() <= 1e-11 * np.abs(G).max()
    fit = O.fit_from_core(O.norm2(X.val), G)
    assert abs(fit - g["fit"]) <= 1e-9
    return U


def check_leading(M, V):
    w = np.linalg.eigvalsh(M)[::-1]
    Jn = V.shape[1]
    top = np.trace(V.T @ M @ V)
    assert abs(top - w[:Jn].sum()) <= 1e-11 * w[:Jn].sum()


def test_hooi_fullsize(tucker_lib, big):
    X, T = big
    g = tucker_lib.tucker_hooi(T, J, tol=-np.inf, max_iter=2)
    U = check_core_fit(X, g)
    W = O.ttmc(X.dims, X.idx, X.val, 2, U)            # [[X; A^T, B^T, I]]
    check_leading(O.gram(O.unfold_dense(W, 2)), U[2])


def test_mp_fullsize(tucker_lib, big):
    X, T = big
    g = tucker_lib.tucker_mp(T, J, tol=-np.inf, max_iter=1)
    U = check_core_fit(X, g)
    Ya = O.ttm(X.dims, X.idx, X.val, 1, U[1])          # X x_2 B^T
    Yb = O.ttm(X.dims, X.idx, X.val, 0, U[0])          # X x_1 A^T
    M3 = O.gram(O.unfold_dense(Ya, 2)) + O.gram(O.unfold_dense(Yb, 2))
    check_leading(M3, U[2])


def test_hosvd_fullsize(tucker_lib, big):
    X, T = big
    g = tucker_lib.tucker_hosvd(T, J)
    U = check_core_fit(X, g)
    check_leading(O.unfolding_gram(X.dims, X.idx, X.val, 0), U[0])


def test_sp_fullsize(tucker_lib, big):
    X, T = big
    C_raw = synth.uniform_matrix(DIMS[2], J[2], synth.config_seed(2))
    g = tucker_lib.tucker_sp(T, J, C_raw, tol=-np.inf, max_iter=2)
    assert g["iters"] == 2
    U = check_core_fit(X, g)
    # C, the last factor of a pass, from B: Gram((X x_2 B^T)_(3)) (Figure sp3)
    Y = O.ttm(X.dims, X.idx, X.val, 1, U[1])
    check_leading(O.gram(O.unfold_dense(Y, 2)), U[2])
