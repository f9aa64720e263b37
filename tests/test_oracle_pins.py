"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics, not by the
oracle itself: brute force on tiny tensors, the matricization identity, exact recovery of
planted low-rank tensors, the reduction to a truncated SVD when I3 = 1 (Eckart-Young), the
reconstruction-based fit, orthonormality, HOOI's monotone fit, invariances, the paper's
printed fits (statistical pin), and planted mistakes that every pin set must catch."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import tucker_oracle as O
from paper_0711_2023_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny(dims=(4, 5, 6), nnz=40, seed=11):
    return synth.random_sparse_tensor(dims, nnz, seed)


def rand_factor(I, J, seed):
    return synth.uniform_matrix(I, J, seed) - 0.5


# ---- primitives by brute force -------------------------------------------------------------

def test_nmode_product_bruteforce():
    X = tiny()
    for n in range(3):
        A = rand_factor(3, X.dims[n], 100 + n)          # J x I_n
        Y = O.nmode_product_sparse(X.dims, X.idx, X.val, n, A)
        ref_shape = list(X.dims)
        ref_shape[n] = 3
        ref = np.zeros(ref_shape)
        for t in range(X.nnz):                          # eq. 1, one nonzero at a time
            i = [int(X.idx[a][t]) for a in range(3)]
            for j in range(3):
                out = list(i)
                out[n] = j
                ref[tuple(out)] += X.val[t] * A[j, i[n]]
        np.testing.assert_allclose(Y, ref, rtol=1e-13, atol=1e-14)


def test_matricization_identity():
    """Y = X x_n A  <=>  Y_(n) = A X_(n) (Section 2)."""
    X = tiny()
    D = O.to_dense(X.dims, X.idx, X.val)
    for n in range(3):
        A = rand_factor(2, X.dims[n], 7 + n)
        Y = O.nmode_product_sparse(X.dims, X.idx, X.val, n, A)
        np.testing.assert_allclose(O.unfold_dense(Y, n), A @ O.unfold_dense(D, n), rtol=1e-13,
                                   atol=1e-14)


def test_ttmc_bruteforce():
    X = tiny()
    U = [rand_factor(X.dims[a], 2 + a, 40 + a) for a in range(3)]
    for n in range(3):
        m, o = O.other_modes(n)
        Y = O.ttmc(X.dims, X.idx, X.val, n, U)
        ref = np.zeros(Y.shape)
        for t in range(X.nnz):
            i = [int(X.idx[a][t]) for a in range(3)]
            for p in range(U[m].shape[1]):
                for q in range(U[o].shape[1]):
                    out = list(i)
                    out[m], out[o] = p, q
                    ref[tuple(out)] += X.val[t] * U[m][i[m], p] * U[o][i[o], q]
        np.testing.assert_allclose(Y, ref, rtol=1e-13, atol=1e-14)


def test_core_bruteforce():
    X = tiny()
    U = [rand_factor(X.dims[a], 2 + a, 50 + a) for a in range(3)]
    G = O.core(X.dims, X.idx, X.val, U)
    ref = np.zeros(G.shape)
    for t in range(X.nnz):
        i, j, k = (int(X.idx[a][t]) for a in range(3))
        ref += X.val[t] * np.einsum("p,q,r->pqr", U[0][i], U[1][j], U[2][k])
    np.testing.assert_allclose(G, ref, rtol=1e-13, atol=1e-14)


def test_unfolding_gram_bruteforce():
    X = tiny()
    D = O.to_dense(X.dims, X.idx, X.val)
    for n in range(3):
        M = O.unfolding_gram(X.dims, X.idx, X.val, n)
        ref = np.zeros((X.dims[n], X.dims[n]))
        for a, b in itertools.product(range(X.dims[n]), repeat=2):
            ref[a, b] = np.sum(np.take(D, a, axis=n) * np.take(D, b, axis=n))
        np.testing.assert_allclose(M, ref, rtol=1e-13, atol=1e-14)


def test_slice_sums_equal_projection_gram():
    """sum_j X_{:j:} C C^T X_{:j:}^T (Figure sp3) = Gram((X x_3 C^T)_(1)), slice by slice."""
    X = tiny()
    D = O.to_dense(X.dims, X.idx, X.val)
    C = rand_factor(X.dims[2], 3, 77)
    ref = sum(D[:, j, :] @ C @ C.T @ D[:, j, :].T for j in range(X.dims[1]))
    Y = O.ttm(X.dims, X.idx, X.val, 2, C)
    np.testing.assert_allclose(O.gram(O.unfold_dense(Y, 0)), ref, rtol=1e-12, atol=1e-13)


def test_pseudo_hosvd_matrix_is_twice_unfolding_gram():
    X = tiny((6, 7, 5), 60, 3)
    for n in (1, 2):
        M = O.mp_init_matrix(X.dims, X.idx, X.val, n)
        np.testing.assert_allclose(M, 2 * O.unfolding_gram(X.dims, X.idx, X.val, n), rtol=1e-13)


def test_csf_ordering_bruteforce():
    X = tiny((5, 4, 6), 50, 9)
    for order in itertools.permutations(range(3)):
        n, m, o = order
        r = O.csf_ordering(X.dims, X.idx, X.val, order)
        ent = sorted((int(X.idx[n][t]), int(X.idx[m][t]), int(X.idx[o][t]), t)
                     for t in range(X.nnz))
        assert [e[2] for e in ent] == r["leaf_idx"].tolist()
        assert [X.val[e[3]] for e in ent] == r["val"].tolist()
        fibers = []
        for e in ent:
            if not fibers or fibers[-1][:2] != e[:2]:
                fibers.append(e[:2])
        assert r["nfibers"] == len(fibers)
        assert [f[1] for f in fibers] == r["fiber_idx"].tolist()
        for i in range(X.dims[n] + 1):
            assert r["root_ptr"][i] == sum(1 for f in fibers if f[0] < i)


def test_duplicates_summed_in_order():
    idx = np.array([[1, 0, 1, 1], [2, 0, 2, 1], [0, 0, 0, 3]], dtype=np.int32)
    val = np.array([0.1, 0.2, 0.7, 0.3])
    i2, v2 = O.canonical_coo((2, 3, 4), idx, val)
    assert i2.T.tolist() == [[0, 0, 0], [1, 1, 3], [1, 2, 0]]
    assert v2.tolist() == [0.2, 0.3, 0.1 + 0.7]


# ---- eigenvectors --------------------------------------------------------------------------

def test_leading_eigvecs_against_svd():
    rng = synth.uniform_matrix(30, 50, 5) - 0.5
    M = rng @ rng.T
    V, w = O.leading_eigvecs(M, 7)
    U, s, _ = np.linalg.svd(rng)                      # a different routine (gesdd)
    np.testing.assert_allclose(w[:7], s[:7] ** 2, rtol=1e-12)
    np.testing.assert_allclose(np.abs(V.T @ U[:, :7]), np.eye(7), atol=1e-10)
    np.testing.assert_allclose(M @ V, V * w[:7], atol=1e-11 * w[0])
    assert np.all(np.diff(w) <= 0)


def test_sign_rule():
    V = np.array([[0.1, -0.9], [-0.8, 0.3], [0.8, 0.2]])
    S = O.sign_fix(V)
    assert S[1, 0] == 0.8 and S[2, 0] == -0.8        # tie: first row wins, made positive
    assert S[0, 1] == 0.9


# ---- method-level pins ---------------------------------------------------------------------

ALGS = ["hosvd", "hooi", "sp", "mp"]


def run(alg, X, J, tol=1e-4, max_iter=50, seed=123):
    if alg == "hosvd":
        return O.hosvd(X.dims, X.idx, X.val, J)
    if alg == "hooi":
        return O.hooi(X.dims, X.idx, X.val, J, tol, max_iter)
    if alg == "sp":
        return O.sp(X.dims, X.idx, X.val, J, synth.uniform_matrix(X.dims[2], J[2], seed), tol,
                    max_iter)
    return O.mp(X.dims, X.idx, X.val, J, tol, max_iter)


@pytest.mark.parametrize("alg", ALGS)
def test_exact_recovery_planted(alg):
    """X = G x1 A x2 B x3 C with exact multilinear rank J: every method must give fit 1."""
    dims, core = (14, 12, 10), (3, 4, 2)
    X, G, F = synth.planted_tensor(dims, core, (8, 7, 6), seed=21)
    r = run(alg, X, core, tol=-np.inf, max_iter=3)
    assert r["fit"] >= 1 - 1e-7
    assert O.fit_explicit(X.dims, X.idx, X.val, r["G"], r["U"]) >= 1 - 1e-12
    for a in range(3):
        assert O.subspace_distance(r["U"][a], F[a]) <= 1e-10


@pytest.mark.parametrize("alg", ALGS)
def test_third_mode_singleton_is_truncated_svd(alg):
    """With I3 = 1 the tensor is a matrix; J = (J, J, 1) must give its truncated SVD and the
    Eckart-Young fit 1 - sqrt(sum_{i>J} s_i^2) / |X| (the 2-D case of Section 2)."""
    X = synth.random_sparse_tensor((12, 9, 1), 60, 31)
    D = O.to_dense(X.dims, X.idx, X.val)[:, :, 0]
    Jm = 4
    r = run(alg, X, (Jm, Jm, 1), tol=-np.inf, max_iter=4)
    U, s, Vt = np.linalg.svd(D)
    expect = 1 - np.sqrt(np.sum(s[Jm:] ** 2)) / np.linalg.norm(s)
    assert abs(r["fit"] - expect) <= 1e-12
    assert O.subspace_distance(r["U"][0], U[:, :Jm]) <= 1e-10
    assert O.subspace_distance(r["U"][1], Vt[:Jm].T) <= 1e-10


@pytest.mark.parametrize("alg", ALGS)
def test_fit_identity_equals_reconstruction(alg):
    X = synth.random_sparse_tensor((7, 5, 6), 70, 41)
    r = run(alg, X, (3, 2, 4), max_iter=5)
    assert abs(r["fit"] - O.fit_explicit(X.dims, X.idx, X.val, r["G"], r["U"])) <= 1e-10


@pytest.mark.parametrize("alg", ALGS)
def test_orthonormal_factors(alg):
    X = synth.random_sparse_tensor((20, 18, 16), 500, 43)
    r = run(alg, X, (5, 4, 6), max_iter=5)
    for U in r["U"]:
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() <= 1e-13


def test_hooi_fit_monotone():
    X = synth.random_sparse_tensor((30, 25, 20), 1500, 47)
    r = O.hooi(X.dims, X.idx, X.val, (5, 5, 5), tol=-np.inf, max_iter=8)
    h = r["fit_history"]
    assert all(h[t + 1] >= h[t] - 1e-13 for t in range(len(h) - 1))
    assert len(h) == 8


@pytest.mark.parametrize("alg", ALGS)
def test_scaling_invariance(alg):
    X = synth.random_sparse_tensor((15, 14, 13), 400, 53)
    Xs = synth.CooTensor(X.dims, X.idx, 3.0 * X.val)
    r, rs = run(alg, X, (4, 3, 5), max_iter=4), run(alg, Xs, (4, 3, 5), max_iter=4)
    assert abs(r["fit"] - rs["fit"]) <= 1e-12
    np.testing.assert_allclose(rs["G"], 3.0 * r["G"], rtol=1e-9, atol=1e-12)


def test_stop_rules():
    X = synth.random_sparse_tensor((40, 40, 40), 6400, 59)
    J = (6, 6, 6)
    for alg in ("hooi", "mp"):
        r = run(alg, X, J, tol=1e-4, max_iter=50)
        h = [0.0] + r["fit_history"]
        d = np.diff(h)
        assert d[-1] < 1e-4 and np.all(d[:-1] >= 1e-4)
    r = run("sp", X, J, tol=1e-4, max_iter=50)
    g = r["gnorm_history"]
    dg = [1 - g[t - 1] / g[t] for t in range(1, len(g))]
    assert dg[-1] < 1e-4 and all(x >= 1e-4 for x in dg[:-1])
    r = run("hooi", X, J, tol=-np.inf, max_iter=3)
    assert r["iters"] == 3


def test_mp_start_spans_hosvd():
    X = synth.random_sparse_tensor((25, 20, 15), 800, 61)
    for n, J in ((1, 4), (2, 5)):
        A = O.leading_eigvecs(O.mp_init_matrix(X.dims, X.idx, X.val, n), J)[0]
        B = O.leading_eigvecs(O.unfolding_gram(X.dims, X.idx, X.val, n), J)[0]
        assert O.subspace_distance(A, B) <= 1e-12


def test_ranking_and_paper_table_250():
    """Statistical pin: the 250^3, 10% density, core 25^3 rows of the paper's results table."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_fits_250.json")))
    X = synth.random_sparse_tensor((250, 250, 250), 1_562_500, synth.config_seed(250))
    J = (25, 25, 25)
    fits = {}
    for alg in ALGS:
        r = run(alg, X, J, seed=synth.config_seed(251))
        fits[alg] = 100 * r["fit"]
        assert abs(fits[alg] - gold["fit_percent"][alg]) <= gold["tolerance_pp"], (alg, fits)
    assert fits["hooi"] > fits["mp"] > fits["sp"] > fits["hosvd"]


# ---- planted mistakes: each must break at least one pin --------------------------------------

def test_planted_mistakes_are_caught(monkeypatch):
    X = synth.random_sparse_tensor((7, 5, 6), 70, 41)
    D = O.to_dense(X.dims, X.idx, X.val)

    # 1. fit without the square root: the reconstruction pin fails
    good = O.fit_from_core
    monkeypatch.setattr(O, "fit_from_core", lambda nX2, G: 1 - (max(0, nX2 - np.sum(G ** 2))) / nX2)
    r = O.hosvd(X.dims, X.idx, X.val, (3, 2, 4))
    assert abs(r["fit"] - O.fit_explicit(X.dims, X.idx, X.val, r["G"], r["U"])) > 1e-6
    monkeypatch.setattr(O, "fit_from_core", good)

    # 2. smallest instead of leading eigenvectors: the Eckart-Young pin fails
    good_eig = O.leading_eigvecs
    monkeypatch.setattr(O, "leading_eigvecs",
                        lambda M, J: (np.linalg.eigh(M)[1][:, :J], np.linalg.eigh(M)[0]))
    Xm = synth.random_sparse_tensor((12, 9, 1), 60, 31)
    Dm = O.to_dense(Xm.dims, Xm.idx, Xm.val)[:, :, 0]
    s = np.linalg.svd(Dm, compute_uv=False)
    r = O.hosvd(Xm.dims, Xm.idx, Xm.val, (4, 4, 1))
    assert abs(r["fit"] - (1 - np.sqrt(np.sum(s[4:] ** 2)) / np.linalg.norm(s))) > 1e-3
    monkeypatch.setattr(O, "leading_eigvecs", good_eig)

    # 3. a transposed factor in the core (A^T applied to mode 2): brute force fails
    U = [rand_factor(X.dims[a], 3, 60 + a) for a in range(3)]
    U[1] = rand_factor(X.dims[1], 3, 70)
    good_core = O.core

    def bad_core(dims, idx, val, U):
        T = O.ttmc(dims, idx, val, 0, U)
        return O.nmode_product_dense(T, 0, np.asarray(U[0])[::-1].T)
    ref = np.einsum("ijk,ip,jq,kr->pqr", D, U[0], U[1], U[2])
    assert np.abs(bad_core(X.dims, X.idx, X.val, U) - ref).max() > 1e-6
    assert np.abs(good_core(X.dims, X.idx, X.val, U) - ref).max() <= 1e-13

    # 4. the two non-output factors swapped inside the projection (equal shapes, so only
    #    the values can tell): the brute-force TTMc pin fails
    X6 = synth.random_sparse_tensor((6, 6, 6), 50, 17)
    D6 = O.to_dense(X6.dims, X6.idx, X6.val)
    V = [rand_factor(6, 3, 80 + a) for a in range(3)]
    ref = np.einsum("ijk,jq,kr->iqr", D6, V[1], V[2])
    assert np.abs(O.ttmc(X6.dims, X6.idx, X6.val, 0, V) - ref).max() <= 1e-13
    swapped = O.ttmc(X6.dims, X6.idx, X6.val, 0, [V[0], V[2], V[1]])
    assert np.abs(swapped - ref).max() > 1e-6
