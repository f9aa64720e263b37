"""GPU parity of the mixed-precision form: FP32 projections written as BF16 hi/lo splits, the
tcgen05 BF16x3 Gram, and the four methods with TUCKER_MIXED against the FP64 oracle.

Tolerances come from the arithmetic: a BF16 split y = hi + lo keeps 16 significant bits, so a
split product misses at most ~2^-16 of |y_i||y_j| (the lo*lo term and the rounding of lo); FP32
accumulation over a K chunk of at most 4096 adds ~K * 2^-24 relative.  Fits must agree with the
FP64 oracle within 1e-4, subspaces within 1e-3 where the eigen-gap makes them well posed."""
import numpy as np
import pytest

from oracle import tucker_oracle as O
from paper_0711_2023_gb300 import synth

pytestmark = pytest.mark.gpu


def split_to_f64(hi, lo):
    return hi.double().cpu().numpy(), lo.double().cpu().numpy()


@pytest.mark.parametrize("rows,K,K2", [(1, 64, 0), (100, 100, 0), (128, 1000, 0), (129, 5000, 0),
                                       (300, 700, 333), (257, 4096 * 2 + 64, 0)])
def test_gram_bf16x3(tucker_lib, rows, K, K2):
    import torch
    def split_input(K, seed):
        Y = torch.from_numpy(synth.uniform_matrix(rows, K, seed) - 0.5).float().cuda()
        ld = tucker_lib.gram_ld(K)
        hi = torch.zeros((rows, ld), dtype=torch.bfloat16, device="cuda")
        lo = torch.zeros((rows, ld), dtype=torch.bfloat16, device="cuda")
        hi[:, :K] = Y.to(torch.bfloat16)
        lo[:, :K] = (Y - hi[:, :K].float()).to(torch.bfloat16)
        return hi, lo
    t1 = split_input(K, 900 + rows)
    t2 = split_input(K2, 901 + rows) if K2 else None
    M = tucker_lib.tucker_gram_bf16x3(t1, t2, K, K2 if K2 else None).cpu().numpy()
    H, L = split_to_f64(*t1)
    ref = H @ H.T + H @ L.T + L @ H.T
    if t2 is not None:
        H2, L2 = split_to_f64(*t2)
        ref += H2 @ H2.T + H2 @ L2.T + L2 @ H2.T
    scale = np.abs(H).max() ** 2 * (K + K2)
    assert np.abs(M - ref).max() <= 2e-6 * scale
    assert np.array_equal(M, M.T)
    # and against the unsplit FP64 product: the split keeps ~16 bits
    Y64 = H + L
    full = Y64 @ Y64.T + ((H2 + L2) @ (H2 + L2).T if t2 is not None else 0)
    assert np.abs(M - full).max() <= 1e-4 * scale


@pytest.fixture(scope="module")
def ragged(tucker_lib):
    X = synth.random_sparse_tensor((67, 45, 83), 9000, 101)
    return X, tucker_lib.tucker_tensor_create(X.idx, X.val, X.dims)


@pytest.mark.parametrize("J", [(5, 17, 33), (70, 9, 40), (12, 48, 64)])   # scalar and float4 rows
def test_ttmc_mixed(tucker_lib, ragged, J):
    X, T = ragged
    U = [(synth.uniform_matrix(X.dims[a], J[a], 200 + a) - 0.5).astype(np.float32)
         for a in range(3)]
    for n in range(3):
        m, o = O.other_modes(n)
        hi, lo, Y32 = tucker_lib.tucker_ttmc_mixed(T, n, U[m], U[o], split=True, fp32=True)
        ref = O.unfold_dense(O.ttmc(X.dims, X.idx, X.val, n, [u.astype(np.float64) for u in U]), n)
        K = ref.shape[1]
        H, L = split_to_f64(hi, lo)
        tol = 1e-5 * np.abs(ref).max()
        assert np.abs(Y32.cpu().numpy() - ref).max() <= tol
        assert np.abs(H[:, :K] + L[:, :K] - ref).max() <= tol
        assert not H[:, K:].any() and not L[:, K:].any()


@pytest.mark.parametrize("Jm", [3, 40, 64, 100, 130])   # scalar and float4 row paths
def test_slice_proj_mixed(tucker_lib, ragged, Jm):
    X, T = ragged
    for n, m in [(0, 2), (1, 0), (2, 1), (0, 1)]:
        o = 3 - n - m
        U = (synth.uniform_matrix(X.dims[m], Jm, 300 + m) - 0.5).astype(np.float32)
        hi, lo = tucker_lib.tucker_slice_proj_mixed(T, n, m, U)
        ref = O.ttm(X.dims, X.idx, X.val, m, U.astype(np.float64))
        ref_n = np.moveaxis(ref, (n, o, m), (0, 1, 2)).reshape(X.dims[n], -1)
        K = ref_n.shape[1]
        H, L = split_to_f64(hi, lo)
        assert np.abs(H[:, :K] + L[:, :K] - ref_n).max() <= 1e-5 * np.abs(ref_n).max()
        assert not H[:, K:].any() and not L[:, K:].any()


def test_slice_proj_mixed_empty_fibers(tucker_lib):
    """Rows and columns with no fiber must come out as zeros (gap filling)."""
    idx = np.array([[0, 0, 2, 4], [1, 3, 3, 0], [2, 0, 5, 5]], dtype=np.int32)
    val = np.array([1.0, 2.0, 3.0, 4.0])
    T = tucker_lib.tucker_tensor_create(idx, val, (5, 4, 6))
    U = (synth.uniform_matrix(6, 3, 5) - 0.5).astype(np.float32)
    hi, lo = tucker_lib.tucker_slice_proj_mixed(T, 0, 2, U)   # rows i1, columns (i2, p)
    ref = O.ttm((5, 4, 6), idx, val, 2, U.astype(np.float64)).reshape(5, -1)
    H, L = split_to_f64(hi, lo)
    # a BF16 hi/lo pair keeps about 16 significant bits of the FP32 value
    assert np.abs(H[:, :12] + L[:, :12] - ref).max() <= 2e-5 * np.abs(ref).max()
    assert (H[:, :12][ref == 0] == 0).all() and (L[:, :12][ref == 0] == 0).all()
    assert not H[:, 12:].any()


def gpu_run(tk, alg, T, J, tol, max_iter, C_raw=None):
    if alg == "hosvd":
        return tk.tucker_hosvd(T, J, precision="mixed")
    if alg == "hooi":
        return tk.tucker_hooi(T, J, tol=tol, max_iter=max_iter, precision="mixed")
    if alg == "sp":
        return tk.tucker_sp(T, J, C_raw, tol=tol, max_iter=max_iter, precision="mixed")
    return tk.tucker_mp(T, J, tol=tol, max_iter=max_iter, precision="mixed")


def oracle_run(alg, X, J, tol, max_iter, C_raw=None):
    if alg == "hosvd":
        return O.hosvd(X.dims, X.idx, X.val, J)
    if alg == "hooi":
        return O.hooi(X.dims, X.idx, X.val, J, tol, max_iter)
    if alg == "sp":
        return O.sp(X.dims, X.idx, X.val, J, C_raw, tol, max_iter)
    return O.mp(X.dims, X.idx, X.val, J, tol, max_iter)


@pytest.mark.parametrize("alg", ["hosvd", "hooi", "sp", "mp"])
def test_methods_mixed_fit(tucker_lib, alg):
    X = synth.random_sparse_tensor((420, 390, 360), 300_000, synth.config_seed(9))
    J = (20, 9, 33)
    C_raw = synth.uniform_matrix(360, 33, synth.config_seed(10))
    T = tucker_lib.tucker_tensor_create(X.idx, X.val, X.dims)
    g = gpu_run(tucker_lib, alg, T, J, -np.inf, 3, C_raw)
    r = oracle_run(alg, X, J, -np.inf, 3, C_raw)
    assert g["iters"] == r["iters"]
    for a, b in zip(g["fit_history"], r["fit_history"]):
        assert abs(a - b) <= 1e-4
    for u in g["U"]:
        u = u.cpu().numpy()
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() <= 1e-12


@pytest.mark.parametrize("alg", ["hosvd", "hooi", "sp", "mp"])
def test_methods_mixed_planted(tucker_lib, alg):
    dims, core = (300, 260, 240), (6, 5, 4)
    X, G, F = synth.planted_tensor(dims, core, (40, 36, 30), seed=23)
    C_raw = synth.uniform_matrix(dims[2], core[2], 6)
    T = tucker_lib.tucker_tensor_create(X.idx, X.val, X.dims)
    g = gpu_run(tucker_lib, alg, T, core, -np.inf, 3, C_raw)
    assert g["fit"] >= 1 - 1e-4
    for a in range(3):
        assert O.subspace_distance(g["U"][a].cpu().numpy(), F[a]) <= 1e-3
