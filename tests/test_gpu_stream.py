"""Slice Projection and Multislice Projection on tensors streamed from pinned host memory
(the out-of-core form the paper designed SP and MP for, Section 3 "Slice Projection"), against
the in-memory GPU path and the oracle.  Small device budgets force many chunks, including single
slices larger than a chunk."""
import numpy as np
import pytest

from oracle import tucker_oracle as O
from paper_0711_2023_gb300 import synth

pytestmark = pytest.mark.gpu
BUDGET_MIN = 1 << 16


@pytest.fixture(scope="module")
def small(tucker_lib):
    X = synth.random_sparse_tensor((60, 50, 40), 20_000, synth.config_seed(61))
    # duplicates: the first 500 coordinates once more, with other values
    idx = np.hstack([X.idx, X.idx[:, :500]])
    val = np.concatenate([X.val, synth.uniform_matrix(1, 500, 62)[0]])
    S = tucker_lib.tucker_stream_create(idx, val, X.dims, BUDGET_MIN)
    T = tucker_lib.tucker_tensor_create(idx, val, X.dims)
    return X, idx, val, S, T


def test_build(tucker_lib, small):
    X, idx, val, S, T = small
    nnz, n2, chunks = tucker_lib.tucker_stream_info(S)
    nnz_t, n2_t = tucker_lib.tucker_tensor_info(T)
    ci, cv = O.canonical_coo(X.dims, idx, val)
    assert nnz == nnz_t == cv.shape[0]
    assert abs(n2 - O.norm2(cv)) <= 1e-12 * n2 and abs(n2 - n2_t) <= 1e-12 * n2
    assert chunks > 10


@pytest.mark.parametrize("alg", ["sp", "mp"])
@pytest.mark.parametrize("tol", [-np.inf, 1e-4])
def test_streamed_vs_in_memory_and_oracle(tucker_lib, small, alg, tol):
    X, idx, val, S, T = small
    J = (5, 4, 6)
    C_raw = synth.uniform_matrix(40, 6, 63)
    if alg == "sp":
        gs = tucker_lib.tucker_sp_streamed(S, J, C_raw, tol=tol, max_iter=4)
        gm = tucker_lib.tucker_sp(T, J, C_raw, tol=tol, max_iter=4)
        r = O.sp(X.dims, idx, val, J, C_raw, tol, 4)
    else:
        gs = tucker_lib.tucker_mp_streamed(S, J, tol=tol, max_iter=4)
        gm = tucker_lib.tucker_mp(T, J, tol=tol, max_iter=4)
        r = O.mp(X.dims, idx, val, J, tol, 4)
    assert gs["iters"] == gm["iters"] == r["iters"]
    for a, b, c in zip(gs["fit_history"], gm["fit_history"], r["fit_history"]):
        assert abs(a - b) <= 1e-12 and abs(a - c) <= 1e-9
    for u in gs["U"]:
        u = u.cpu().numpy()
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() <= 1e-12
    assert gs["bytes_streamed"] > 0


def test_mp_streamed_with_start(tucker_lib, small):
    X, idx, val, S, T = small
    J = (5, 4, 6)
    start = tucker_lib.tucker_hosvd(T, J)["U"]
    init = [None, start[1], start[2]]
    gs = tucker_lib.tucker_mp_streamed(S, J, tol=-np.inf, max_iter=2, init=init)
    r = O.mp(X.dims, idx, val, J, -np.inf, 2, init=[None] + [u.cpu().numpy() for u in start[1:]])
    for a, b in zip(gs["fit_history"], r["fit_history"]):
        assert abs(a - b) <= 1e-9


def test_slices_larger_than_a_chunk(tucker_lib):
    # mode-1 slices of ~1700 nonzeros against a budget that holds ~580 per chunk
    X = synth.random_sparse_tensor((30, 200, 200), 50_000, synth.config_seed(64))
    S = tucker_lib.tucker_stream_create(X.idx, X.val, X.dims, BUDGET_MIN)
    J = (4, 6, 5)
    gs = tucker_lib.tucker_mp_streamed(S, J, tol=-np.inf, max_iter=2)
    r = O.mp(X.dims, X.idx, X.val, J, -np.inf, 2)
    for a, b in zip(gs["fit_history"], r["fit_history"]):
        assert abs(a - b) <= 1e-9


def test_500cube_streamed_mp(tucker_lib):
    X = synth.random_sparse_tensor((500, 500, 500), 2_500_000, synth.config_seed(3))
    import torch
    S = tucker_lib.tucker_stream_create(torch.from_numpy(X.idx).cuda(),
                                        torch.from_numpy(X.val).cuda(), X.dims, 32 << 20)
    T = tucker_lib.tucker_tensor_create(X.idx, X.val, X.dims)
    assert tucker_lib.tucker_stream_info(S)[2] >= 8
    J = (50, 50, 50)
    gs = tucker_lib.tucker_mp_streamed(S, J, tol=-np.inf, max_iter=2)
    gm = tucker_lib.tucker_mp(T, J, tol=-np.inf, max_iter=2)
    for a, b in zip(gs["fit_history"], gm["fit_history"]):
        assert abs(a - b) <= 1e-10


def test_stream_errors(tucker_lib, small):
    X, idx, val, S, T = small
    with pytest.raises(tucker_lib.TuckerError):
        tucker_lib.tucker_stream_create(idx, val, X.dims, BUDGET_MIN - 1)
    bad = X.idx.copy()
    bad[2, 7] = 40
    with pytest.raises(tucker_lib.TuckerError) as e:
        tucker_lib.tucker_stream_create(bad, X.val, X.dims, BUDGET_MIN)
    assert e.value.status == tucker_lib.TUCKER_EINVAL
    with pytest.raises(tucker_lib.TuckerError):          # SP needs its random C
        tucker_lib._run_streamed("tucker_sp_streamed", S, (2, 2, 2), -np.inf, 2, None)
