"""Pins of the oracle's order-N and fourth-order methods (Figures HO-SVDn, hooin, sp4, mp4)
against what the definitions and the paper fix, independently of the oracle's own code: brute
force on dense copies of tiny tensors (einsum), the figures' slice sums written out literally,
exact recovery of planted tensors, the reconstruction fit, reduction to the third-order methods,
and the paper's fourth-order results table."""
import json
import os

import numpy as np
import pytest

from oracle import tucker_oracle as O
from paper_0711_2023_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rand_factor(n, j, seed):
    Q, _ = np.linalg.qr(synth.uniform_matrix(n, j, seed) - 0.5)
    return Q


def tiny4(seed=3):
    X = synth.random_sparse_tensor_n((5, 4, 6, 3), 120, seed)
    return X, O.to_dense_n(X.dims, X.idx, X.val)


def test_generator_and_n_forms_match_third_order():
    X = synth.random_sparse_tensor((9, 7, 8), 200, 11)
    Xn = synth.random_sparse_tensor_n((9, 7, 8), 200, 11)
    assert np.array_equal(X.idx, Xn.idx) and np.array_equal(X.val, Xn.val)
    J = (3, 2, 4)
    a, b = O.hooi(X.dims, X.idx, X.val, J, -np.inf, 3), O.hooi_n(X.dims, X.idx, X.val, J, -np.inf, 3)
    assert np.allclose(a["fit_history"], b["fit_history"], rtol=0, atol=1e-14)
    a, b = O.hosvd(X.dims, X.idx, X.val, J), O.hosvd_n(X.dims, X.idx, X.val, J)
    assert abs(a["fit"] - b["fit"]) <= 1e-14
    i3, v3 = O.canonical_coo(X.dims, X.idx, X.val)
    i4, v4 = O.canonical_coo_n(X.dims, X.idx, X.val)
    assert np.array_equal(i3, i4) and np.array_equal(v3, v4)


def test_primitives_bruteforce():
    X, D = tiny4()
    U = [rand_factor(X.dims[a], 2 + a % 2, 30 + a) for a in range(4)]
    # single products on each mode
    for m in range(4):
        sub = "abcd"
        ref = np.einsum(f"abcd,{sub[m]}z->" + sub.replace(sub[m], "z"), D, U[m])
        assert np.abs(O.ttm_n(X.dims, X.idx, X.val, m, U[m]) - ref).max() <= 1e-13
    # projections on all modes but n, the core, unfolding Grams
    ref = np.einsum("abcd,bq,cr,ds->aqrs", D, U[1], U[2], U[3])
    assert np.abs(O.ttmc_n(X.dims, X.idx, X.val, 0, U) - ref).max() <= 1e-13
    ref = np.einsum("abcd,ap,cr,ds->pbrs", D, U[0], U[2], U[3])
    assert np.abs(O.ttmc_n(X.dims, X.idx, X.val, 1, U) - ref).max() <= 1e-13
    G = np.einsum("abcd,ap,bq,cr,ds->pqrs", D, *U)
    assert np.abs(O.core_n(X.dims, X.idx, X.val, U) - G).max() <= 1e-13
    for n in range(4):
        Dn = np.moveaxis(D, n, 0).reshape(D.shape[n], -1)
        assert np.abs(O.unfolding_gram_n(X.dims, X.idx, X.val, n) - Dn @ Dn.T).max() <= 1e-13


def test_sp4_slice_sums_written_out():
    # The four matrices of Figure sp4, each summed literally over its slices, equal the Grams
    # of the single-mode projections the oracle uses.
    X, D = tiny4(5)
    U = [rand_factor(X.dims[a], 2, 40 + a) for a in range(4)]
    I1, I2, I3, I4 = X.dims
    M14 = sum(D[:, i, j, :] @ U[3] @ U[3].T @ D[:, i, j, :].T for i in range(I2) for j in range(I3))
    M21 = sum(D[:, :, i, j].T @ U[0] @ U[0].T @ D[:, :, i, j] for i in range(I3) for j in range(I4))
    M32 = sum(D[i, :, :, j].T @ U[1] @ U[1].T @ D[i, :, :, j] for i in range(I1) for j in range(I4))
    M43 = sum(D[i, j, :, :].T @ U[2] @ U[2].T @ D[i, j, :, :] for i in range(I1) for j in range(I2))
    for (n, m), M in zip(O.SP4_PAIRS, (M14, M21, M32, M43)):
        Y = O.ttm_n(X.dims, X.idx, X.val, m, U[m])
        assert np.abs(O.gram(O.unfold_dense(Y, n)) - M).max() <= 1e-12


def test_mp4_matrices_written_out():
    X, D = tiny4(7)
    U = [rand_factor(X.dims[a], 2, 50 + a) for a in range(4)]
    I1, I2, I3, I4 = X.dims
    A, B, C, Dm = U
    P = lambda F: F @ F.T  # noqa: E731
    M1 = (sum(D[:, :, i, j] @ P(B) @ D[:, :, i, j].T for i in range(I3) for j in range(I4))
          + sum(D[:, i, :, j] @ P(C) @ D[:, i, :, j].T for i in range(I2) for j in range(I4))
          + sum(D[:, i, j, :] @ P(Dm) @ D[:, i, j, :].T for i in range(I2) for j in range(I3)))
    M2 = (sum(D[:, :, i, j].T @ P(A) @ D[:, :, i, j] for i in range(I3) for j in range(I4))
          + sum(D[i, :, :, j] @ P(C) @ D[i, :, :, j].T for i in range(I1) for j in range(I4))
          + sum(D[i, :, j, :] @ P(Dm) @ D[i, :, j, :].T for i in range(I1) for j in range(I3)))
    M3 = (sum(D[:, i, :, j].T @ P(A) @ D[:, i, :, j] for i in range(I2) for j in range(I4))
          + sum(D[i, :, :, j].T @ P(B) @ D[i, :, :, j] for i in range(I1) for j in range(I4))
          + sum(D[i, j, :, :] @ P(Dm) @ D[i, j, :, :].T for i in range(I1) for j in range(I2)))
    M4 = (sum(D[:, i, j, :].T @ P(A) @ D[:, i, j, :] for i in range(I2) for j in range(I3))
          + sum(D[i, :, j, :].T @ P(B) @ D[i, :, j, :] for i in range(I1) for j in range(I3))
          + sum(D[i, j, :, :].T @ P(C) @ D[i, j, :, :] for i in range(I1) for j in range(I2)))
    for n, M in enumerate((M1, M2, M3, M4)):
        assert np.abs(O.mp4_matrix(X.dims, X.idx, X.val, n, U) - M).max() <= 1e-12


def test_mp4_start_is_three_unfolding_grams():
    # Each of the three slice sums of the pseudo HO-SVD start equals X_(n) X_(n)^T, so the start
    # matrix is 3 X_(n) X_(n)^T and its leading eigenvectors are HO-SVD's.
    X, _ = tiny4(9)
    for n in (1, 2, 3):
        M = O.mp4_init_matrix(X.dims, X.idx, X.val, n)
        assert np.abs(M - 3.0 * O.unfolding_gram_n(X.dims, X.idx, X.val, n)).max() <= 1e-12


def run4(alg, X, J, sweeps=20, tol=1e-10, init=None):
    if alg == "hosvd":
        return O.hosvd_n(X.dims, X.idx, X.val, J)
    if alg == "hooi":
        return O.hooi_n(X.dims, X.idx, X.val, J, tol, sweeps, init=init)
    if alg == "sp":
        D_raw = synth.uniform_matrix(X.dims[3], J[3], 77)
        return O.sp4(X.dims, X.idx, X.val, J, D_raw, tol, sweeps)
    return O.mp4(X.dims, X.idx, X.val, J, tol, sweeps, init=init)


@pytest.mark.parametrize("alg", ["hosvd", "hooi", "sp", "mp"])
def test_exact_recovery_planted_4d(alg):
    core, support = (3, 2, 3, 2), (6, 5, 7, 4)
    X, G, F = synth.planted_tensor_n((9, 8, 10, 7), core, support, 123)
    r = run4(alg, X, core)
    assert r["fit"] >= 1 - 1e-7
    for a in range(4):
        assert O.subspace_distance(r["U"][a], F[a]) <= 1e-9
        assert np.abs(r["U"][a].T @ r["U"][a] - np.eye(core[a])).max() <= 1e-13
    assert abs(O.fit_explicit_n(X.dims, X.idx, X.val, r["G"], r["U"]) - 1.0) <= 1e-10


@pytest.mark.parametrize("alg", ["hosvd", "hooi", "sp", "mp"])
def test_fit_identity_equals_reconstruction_4d(alg):
    X, _ = tiny4(13)
    r = run4(alg, X, (3, 2, 4, 2), sweeps=3)
    assert abs(r["fit"] - O.fit_explicit_n(X.dims, X.idx, X.val, r["G"], r["U"])) <= 1e-10


def test_hooi_n_fit_monotone():
    X = synth.random_sparse_tensor_n((8, 7, 9, 6), 800, 17)
    r = O.hooi_n(X.dims, X.idx, X.val, (3, 3, 2, 2), -np.inf, 8)
    h = r["fit_history"]
    assert all(b >= a - 1e-13 for a, b in zip(h, h[1:]))


def test_singleton_fourth_mode_reduces_to_third_order():
    # I_4 = 1, J_4 = 1: the fourth factor is [1] and HOOI / HO-SVD of the order-4 tensor are the
    # third-order methods of X[:, :, :, 0].
    X3 = synth.random_sparse_tensor((9, 8, 7), 150, 19)
    idx4 = np.vstack([X3.idx, np.zeros((1, X3.nnz), dtype=np.int32)])
    dims4 = X3.dims + (1,)
    J = (3, 2, 4)
    for f3, fn in ((lambda: O.hosvd(X3.dims, X3.idx, X3.val, J),
                    lambda: O.hosvd_n(dims4, idx4, X3.val, J + (1,))),
                   (lambda: O.hooi(X3.dims, X3.idx, X3.val, J, -np.inf, 4),
                    lambda: O.hooi_n(dims4, idx4, X3.val, J + (1,), -np.inf, 4))):
        a, b = f3(), fn()
        assert np.allclose(a["fit_history"], b["fit_history"], rtol=0, atol=1e-13)
        assert np.abs(a["G"] - b["G"][..., 0]).max() <= 1e-12


def test_paper_table_fourth_order():
    """Statistical pin: the 100^4, 10% density, core 20^4 rows of the paper's fourth-order
    results table.  MP starts from the HO-SVD factors, which test_mp4_start_is_three_unfolding
    _grams shows equal to its pseudo HO-SVD start."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_fits_100x4.json")))
    X = synth.random_sparse_tensor_n((100, 100, 100, 100), 10_000_000, synth.config_seed(400))
    J = (20, 20, 20, 20)
    h = O.hosvd_n(X.dims, X.idx, X.val, J)
    fits = {"hosvd": 100 * h["fit"]}
    start = [None] + h["U"][1:]
    fits["hooi"] = 100 * O.hooi_n(X.dims, X.idx, X.val, J, 1e-4, 50, init=start)["fit"]
    D_raw = synth.uniform_matrix(100, 20, synth.config_seed(401))
    fits["sp"] = 100 * O.sp4(X.dims, X.idx, X.val, J, D_raw, 1e-4, 50)["fit"]
    fits["mp"] = 100 * O.mp4(X.dims, X.idx, X.val, J, 1e-4, 50, init=start)["fit"]
    for alg, f in fits.items():
        assert abs(f - gold["fit_percent"][alg]) <= gold["tolerance_pp"], (alg, fits)
    assert fits["hooi"] > fits["mp"] > fits["sp"] > fits["hosvd"]


def test_planted_mistakes_are_caught_4d():
    X, D = tiny4(21)
    U = [rand_factor(X.dims[a], 2, 60 + a) for a in range(4)]
    # 1. an MP4 pass that drops one of its three slice sums: the written-out matrices differ
    M1 = O.mp4_matrix(X.dims, X.idx, X.val, 0, U)
    short = sum(O.gram(O.unfold_dense(O.ttm_n(X.dims, X.idx, X.val, m, U[m]), 0)) for m in (1, 2))
    assert np.abs(M1 - short).max() > 1e-6
    # 2. projecting on the wrong mode in SP4's first step: the slice sums of Figure sp4 differ
    good = O.gram(O.unfold_dense(O.ttm_n(X.dims, X.idx, X.val, 3, U[3]), 0))
    bad = O.gram(O.unfold_dense(O.ttm_n(X.dims, X.idx, X.val, 2, rand_factor(6, 2, 63)), 0))
    assert np.abs(good - bad).max() > 1e-6
    # 3. a core whose last mode is projected with the factor's rows reversed: brute force fails
    G = np.einsum("abcd,ap,bq,cr,ds->pqrs", D, *U)
    assert np.abs(O.core_n(X.dims, X.idx, X.val, U) - G).max() <= 1e-13
    Ubad = U[:3] + [U[3][::-1].copy()]
    assert np.abs(O.core_n(X.dims, X.idx, X.val, Ubad) - G).max() > 1e-6
