"""GPU parity of each hot-path step, called through the C ABI, against the FP64 oracle on the
same seeded inputs.  Sizes span several tiles and ragged tails; index work is bit-exact and
FP64 arithmetic agrees to 1e-12 relative (different but fixed summation orders)."""
import itertools

import numpy as np
import pytest

from oracle import tucker_oracle as O
from paper_0711_2023_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-12


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def ragged(tucker_lib):
    X = synth.random_sparse_tensor((67, 45, 83), 9000, 101)
    T = tucker_lib.tucker_tensor_create(X.idx, X.val, X.dims)
    return X, T


def check_orderings(tucker_lib, X, T):
    for order in itertools.permutations(range(3)):
        g = tucker_lib.tucker_ordering(T, *order)
        r = O.csf_ordering(X.dims, X.idx, X.val, order)
        assert g["nfibers"] == r["nfibers"]
        np.testing.assert_array_equal(g["root_ptr"], r["root_ptr"])
        np.testing.assert_array_equal(g["fiber_idx"], r["fiber_idx"])
        np.testing.assert_array_equal(g["fiber_ptr"], r["fiber_ptr"])
        np.testing.assert_array_equal(g["leaf_idx"], r["leaf_idx"])
        assert g["val"].tobytes() == r["val"].tobytes()


def test_orderings_bit_exact(tucker_lib, ragged):
    X, T = ragged
    check_orderings(tucker_lib, X, T)


@pytest.mark.parametrize("dims,nnz", [((64, 64, 32), 30000), ((256, 256, 512), 40000)])
def test_orderings_bit_exact_nine_bit_pass(tucker_lib, dims, nnz):
    """Keys of 17 and 25 bits: the radix sort's last pass takes 9 bits (as it does for the
    33-bit keys of a 2000^3 tensor), both in the canonical sort and in every ordering."""
    X = synth.random_sparse_tensor(dims, nnz, 211)
    T = tucker_lib.tucker_tensor_create(X.idx, X.val, X.dims)
    check_orderings(tucker_lib, X, T)


def test_duplicates_and_device_input(tucker_lib):
    import torch
    X = synth.random_sparse_tensor((9, 8, 7), 120, 7)
    idx = np.concatenate([X.idx, X.idx[:, :30]], axis=1)
    val = np.concatenate([X.val, 0.5 * X.val[:30]])
    T = tucker_lib.tucker_tensor_create(torch.from_numpy(idx).cuda(), torch.from_numpy(val).cuda(),
                                        X.dims)
    ci, cv = O.canonical_coo(X.dims, idx, val)
    nnz, n2 = T.info()
    assert nnz == ci.shape[1]
    assert abs(n2 - O.norm2(cv)) <= RTOL * O.norm2(cv)
    g = tucker_lib.tucker_ordering(T, 0, 1, 2)
    assert g["val"].tobytes() == cv.tobytes()


def test_norm2(tucker_lib, ragged):
    X, T = ragged
    nnz, n2 = T.info()
    assert nnz == X.nnz
    assert abs(n2 - O.norm2(X.val)) <= RTOL * O.norm2(X.val)


def test_unfolding_gram(tucker_lib, ragged):
    X, T = ragged
    for n in range(3):
        M = tucker_lib.tucker_unfolding_gram(T, n).cpu().numpy()
        assert rel_err(M, O.unfolding_gram(X.dims, X.idx, X.val, n)) <= RTOL


@pytest.mark.parametrize("J", [(5, 17, 33), (70, 9, 40), (16, 16, 16)])
def test_ttmc(tucker_lib, ragged, J):
    X, T = ragged
    U = [synth.uniform_matrix(X.dims[a], J[a], 200 + a) - 0.5 for a in range(3)]
    for n in range(3):
        m, o = O.other_modes(n)
        Y = tucker_lib.tucker_ttmc(T, n, U[m], U[o]).cpu().numpy()
        ref = O.unfold_dense(O.ttmc(X.dims, X.idx, X.val, n, U), n)
        # oracle column order is (p, q) row-major, as is the library's
        assert rel_err(Y, ref) <= RTOL


@pytest.mark.parametrize("Jm", [3, 40, 130])
def test_slice_proj(tucker_lib, ragged, Jm):
    X, T = ragged
    for n, m in itertools.permutations(range(3), 2):
        o = 3 - n - m
        U = synth.uniform_matrix(X.dims[m], Jm, 300 + m) - 0.5
        Y = tucker_lib.tucker_slice_proj(T, n, m, U).cpu().numpy()
        ref = O.ttm(X.dims, X.idx, X.val, m, U)           # dense, mode m has size Jm
        # library column index: i_o * Jm + p
        ref_n = np.moveaxis(ref, (n, o, m), (0, 1, 2)).reshape(X.dims[n], -1)
        assert rel_err(Y, ref_n) <= RTOL


@pytest.mark.parametrize("rows,K1,K2", [(1, 7, 0), (100, 333, 0), (130, 1000, 77), (65, 64, 64)])
def test_gram(tucker_lib, rows, K1, K2):
    Y1 = synth.uniform_matrix(rows, K1, 400) - 0.5
    Y2 = synth.uniform_matrix(rows, K2, 401) - 0.5 if K2 else None
    M = tucker_lib.tucker_gram(Y1, Y2).cpu().numpy()
    ref = O.gram(Y1) + (O.gram(Y2) if K2 else 0)
    assert rel_err(M, ref) <= RTOL
    assert np.array_equal(M, M.T)


def spiked_psd(n, J, seed, gap=0.5):
    """PSD matrix with a clear gap after the J-th eigenvalue (well-posed subspace)."""
    Q, _ = np.linalg.qr(synth.uniform_matrix(n, n, seed) - 0.5)
    w = np.concatenate([np.linspace(10.0, 2.0, J), gap * np.linspace(1.0, 0.0, n - J)])
    return (Q * w) @ Q.T


# (100, 10) and (157, 60) solve all eigenpairs at once; the others run the subspace iteration
# with blocks of k = J + max(16, J / 2) = 36, 75, 300 and 384 columns, whose Cholesky-QR
# factorisations take 3, 5, 19 and 24 block rows of 16 (384 is the largest the cluster
# factorisation takes)
@pytest.mark.parametrize("n,J", [(100, 10), (157, 60), (400, 20), (700, 50), (1000, 200),
                                 (1000, 256)])
def test_eig_topk(tucker_lib, n, J):
    M = spiked_psd(n, J, 500 + n)
    U, lam = tucker_lib.tucker_eig_topk(M, J)
    U, lam = U.cpu().numpy(), lam.cpu().numpy()
    V, w = O.leading_eigvecs(M, J)
    np.testing.assert_allclose(lam, w[:J], rtol=1e-11)
    assert O.subspace_distance(U, V) <= 1e-9
    assert np.abs(U.T @ U - np.eye(J)).max() <= 1e-12
    # simple eigenvalues: columns agree one by one after the shared sign rule
    assert np.abs(U - V).max() <= 1e-8


@pytest.mark.parametrize("n", [120, 400])   # all-eigenpairs path and subspace path
def test_eig_topk_clusters_and_outlier(tucker_lib, n):
    """Spectra the small eigensolver's first-order refinement cannot split on its own: an exact
    triple, a pair 1e-9 apart, a pair 1e-6 apart (these go to the FP64 Jacobi fallback when they
    matter at the tolerance), under an outlier 1e4 times the bulk, with a clear gap after J."""
    J = 24
    Q, _ = np.linalg.qr(synth.uniform_matrix(n, n, 900 + n) - 0.5)
    w = np.concatenate([[1e4], [7.0, 7.0, 7.0], [5.0, 5.0 + 5e-9], [3.0, 3.0 + 3e-6],
                        np.linspace(2.5, 1.0, J - 8), 0.1 * np.linspace(1.0, 0.0, n - J)])
    M = (Q * w) @ Q.T
    M = 0.5 * (M + M.T)
    tucker_lib.tucker_profile_enable(True)
    U, lam = tucker_lib.tucker_eig_topk(M, J)
    rot = tucker_lib.tucker_profile_query("syev_cluster_rotations")[0]
    fb = tucker_lib.tucker_profile_query("syev_fallback")[0]
    tucker_lib.tucker_profile_enable(False)
    if n == 120:
        # all eigenpairs of M by one small eigenproblem: its clusters are split by the Jacobi
        # rotations inside the refinement, without the FP64 Jacobi fallback
        assert rot >= 1 and fb == 0, (rot, fb)
    U, lam = U.cpu().numpy(), lam.cpu().numpy()
    V, wr = O.leading_eigvecs(M, J)
    np.testing.assert_allclose(lam, wr[:J], rtol=1e-11, atol=1e-12 * wr[0])
    # The J-subspace is well posed (gap 0.9 after J).  The subspace path locks at residual
    # 3e-13 * theta_1 = 3e-9 here, so by Davis-Kahan sin(angle) <= 3e-9 / 0.9.
    assert O.subspace_distance(U, V) <= 1e-8
    assert np.abs(U.T @ U - np.eye(J)).max() <= 1e-12
    # within a cluster any orthonormal basis is right: check each column is an eigenvector
    res = np.linalg.norm(M @ U - U * lam, axis=0)
    assert res.max() <= 1e-11 * wr[0]


def test_eig_topk_warm_start_and_uniform_tensor_gram(tucker_lib):
    X = synth.random_sparse_tensor((300, 280, 260), 200000, 601)
    M = O.unfolding_gram(X.dims, X.idx, X.val, 0)
    J = 20
    V, w = O.leading_eigvecs(M, J)
    U, lam = tucker_lib.tucker_eig_topk(M, J)
    U = U.cpu().numpy()
    # near-degenerate bulk spectrum: compare what the method's fit depends on (the trace)
    assert abs(np.trace(U.T @ M @ U) - w[:J].sum()) <= 1e-12 * w[:J].sum()
    U2, _ = tucker_lib.tucker_eig_topk(M, J, U0=U)
    U2 = U2.cpu().numpy()
    assert abs(np.trace(U2.T @ M @ U2) - w[:J].sum()) <= 1e-12 * w[:J].sum()


def test_core(tucker_lib, ragged):
    X, T = ragged
    J = (7, 12, 5)
    U = [np.linalg.qr(synth.uniform_matrix(X.dims[a], J[a], 700 + a) - 0.5)[0] for a in range(3)]
    G, g2 = tucker_lib.tucker_core(T, *U)
    ref = O.core(X.dims, X.idx, X.val, U)
    assert rel_err(G.cpu().numpy(), ref) <= RTOL
    assert abs(g2 - np.sum(ref ** 2)) <= RTOL * np.sum(ref ** 2)


def test_errors(tucker_lib):
    import torch
    with pytest.raises(tucker_lib.TuckerError) as e:
        tucker_lib.tucker_tensor_create(np.array([[0], [0], [5]], dtype=np.int32),
                                        np.array([1.0]), (2, 2, 2))
    assert e.value.status == tucker_lib.TUCKER_EINVAL
    Z = tucker_lib.tucker_tensor_create(np.array([[0], [1], [1]], dtype=np.int32),
                                        np.array([0.0]), (2, 2, 2))
    with pytest.raises(tucker_lib.TuckerError) as e:
        tucker_lib.tucker_hosvd(Z, (1, 1, 1))
    assert e.value.status == tucker_lib.TUCKER_EEMPTY
    X = synth.random_sparse_tensor((5, 6, 7), 50, 3)
    T = tucker_lib.tucker_tensor_create(X.idx, X.val, X.dims)
    with pytest.raises(tucker_lib.TuckerError):
        tucker_lib.tucker_hooi(T, (6, 2, 2))              # J_1 > I_1
    with pytest.raises(tucker_lib.TuckerError):
        tucker_lib.tucker_sp(T, (2, 2, 2), None)          # SP needs its random C
    torch.cuda.synchronize()
