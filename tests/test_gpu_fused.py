"""The fused slice projection + tensor-core Gram of the mixed form (Figures sp3, mp3: the slice
sums sum_k X_k U U^T X_k^T = Gram((X x_m U^T)_(n)), the projection built in shared memory and never
written to memory), through tucker_gram_fused, against the FP64 projection Gram of the oracle
and against the two-kernel path (projection to memory, then the BF16x3 Gram).

Bars as for the BF16x3 Gram: the split y = hi + lo keeps ~16 bits, so entries agree with the
FP64 Gram within 1e-4 of max|y|^2 K, and with the two-kernel path (same FP32 projection values,
other summation chunks) within 2e-6 of it."""
import numpy as np
import pytest

from oracle import tucker_oracle as O
from paper_0711_2023_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPES = [((1, 40, 30), 300), ((50, 33, 61), 4000), ((128, 70, 40), 9000), ((129, 45, 83), 9000),
          ((200, 31, 17), 2500), ((256, 60, 50), 30000)]


def factor32(n, j, seed):
    return (synth.uniform_matrix(n, j, seed) - 0.5).astype(np.float32)


def proj64(X, n, m, U):
    """(X x_m U^T)_(n) in FP64 from the FP32 factor, columns (i_o, p) like the library's."""
    o = 3 - n - m
    Y = O.ttm(X.dims, X.idx, X.val, m, U.astype(np.float64))
    return np.moveaxis(Y, (n, o, m), (0, 1, 2)).reshape(X.dims[n], -1)


@pytest.mark.parametrize("dims,nnz", SHAPES)
@pytest.mark.parametrize("two", [False, True])
def test_fused_gram(tucker_lib, dims, nnz, two):
    X = synth.random_sparse_tensor(dims, nnz, synth.config_seed(sum(dims)))
    T = tucker_lib.tucker_tensor_create(X.idx, X.val, X.dims)
    n, m1, m2 = 0, 1, 2
    J1, J2 = 7, 12
    U1, U2 = factor32(dims[m1], J1, 301), factor32(dims[m2], J2, 302)
    M = tucker_lib.tucker_gram_fused(T, n, m1, U1, m2 if two else None, U2 if two else None)
    M = M.cpu().numpy()
    Y1 = proj64(X, n, m1, U1)
    ref = Y1 @ Y1.T
    K = Y1.shape[1]
    ymax = np.abs(Y1).max()
    if two:
        Y2 = proj64(X, n, m2, U2)
        ref += Y2 @ Y2.T
        K += Y2.shape[1]
        ymax = max(ymax, np.abs(Y2).max())
    scale = ymax ** 2 * K
    assert np.array_equal(M, M.T)
    assert np.abs(M - ref).max() <= 1e-4 * scale
    # the two-kernel path: projection written split, then the tensor-core Gram
    h1, l1 = tucker_lib.tucker_slice_proj_mixed(T, n, m1, U1)
    t2 = tucker_lib.tucker_slice_proj_mixed(T, n, m2, U2) if two else None
    M2 = tucker_lib.tucker_gram_bf16x3((h1, l1), t2, dims[2] * J1,
                                       dims[1] * J2 if two else None).cpu().numpy()
    assert np.abs(M - M2).max() <= 2e-6 * scale


def test_fused_gram_empty_slices(tucker_lib):
    # every second slice of the projecting term's slice mode is empty, and some rows are empty
    X = synth.random_sparse_tensor((90, 40, 50), 6000, synth.config_seed(303))
    keep = (X.idx[2] % 2 == 0) & (X.idx[0] % 7 != 3)
    idx, val = X.idx[:, keep], X.val[keep]
    T = tucker_lib.tucker_tensor_create(idx, val, X.dims)
    U = factor32(40, 9, 304)
    M = tucker_lib.tucker_gram_fused(T, 0, 1, U).cpu().numpy()
    Y = O.ttm(X.dims, idx, val, 1, U.astype(np.float64))
    Y = np.moveaxis(Y, (0, 2, 1), (0, 1, 2)).reshape(90, -1)
    assert np.abs(M - Y @ Y.T).max() <= 1e-4 * np.abs(Y).max() ** 2 * Y.shape[1]
    assert np.all(M[3::7] == 0.0)


def test_fused_gram_rejects_large_modes(tucker_lib):
    X = synth.random_sparse_tensor((257, 10, 10), 500, synth.config_seed(305))
    T = tucker_lib.tucker_tensor_create(X.idx, X.val, X.dims)
    with pytest.raises(tucker_lib.TuckerError) as e:
        tucker_lib.tucker_gram_fused(T, 0, 1, factor32(10, 3, 306))
    assert e.value.status == tucker_lib.TUCKER_EINVAL
