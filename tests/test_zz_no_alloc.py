"""The allocation-free Gram entry point (for callers that cannot let the library allocate device
memory while they run) against the allocating one, through the C ABI, on two calls in a row:
the second call must not see anything of the first one's contents in the shared fixed scratch.
Collected last so that a run stopping at the first failure has run every other test."""
import numpy as np
import pytest

from paper_0711_2023_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-12   # same bar as the other FP64 Gram tests (different split counts, fixed orders)


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_gram_noalloc_matches_gram_twice(tucker_lib):
    # call 1: one term, several tiles with a ragged tail
    Y1 = synth.uniform_matrix(300, 1000, 11) - 0.5
    M_ref = tucker_lib.tucker_gram(Y1).cpu().numpy()
    M_new = tucker_lib.tucker_gram_noalloc(Y1).cpu().numpy()
    assert rel_err(M_new, M_ref) <= RTOL
    assert np.array_equal(M_new, M_new.T)
    # call 2: smaller and two terms; stale partials of call 1 must not leak in
    A = synth.uniform_matrix(100, 257, 12) - 0.5
    B = synth.uniform_matrix(100, 64, 13) - 0.5
    M_ref = tucker_lib.tucker_gram(A, B).cpu().numpy()
    M_new = tucker_lib.tucker_gram_noalloc(A, B).cpu().numpy()
    assert rel_err(M_new, M_ref) <= RTOL
    assert np.array_equal(M_new, M_new.T)


def test_gram_noalloc_largest_size(tucker_lib):
    # rows = 1448 is the largest the fixed scratch allows: one K split whose partial tiles fill
    # the array almost to its end
    Y = synth.uniform_matrix(1448, 4096, 14) - 0.5
    M_ref = tucker_lib.tucker_gram(Y).cpu().numpy()
    for _ in range(2):
        M_new = tucker_lib.tucker_gram_noalloc(Y).cpu().numpy()
        assert rel_err(M_new, M_ref) <= RTOL
        assert np.array_equal(M_new, M_new.T)


def test_gram_noalloc_rejects_oversize(tucker_lib):
    import torch
    Y = torch.zeros((1449, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(tucker_lib.TuckerError) as e:
        tucker_lib.tucker_gram_noalloc(Y)
    assert e.value.status == tucker_lib.TUCKER_EINVAL
