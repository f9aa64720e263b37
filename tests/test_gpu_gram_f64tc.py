"""The FP64 products on the BF16 tensor cores (error-free slicing, exact integer level sums):
the Gram that the FP64 form of every method uses for Y_(n) Y_(n)^T (Figures hooi3, sp3, mp3),
through tucker_gram, and the general product of the eigensolver, through tucker_gemm.

Pins independent of the library: integer-valued inputs, whose slices hold every bit, must give
the exact integer Gram bit for bit (a single inexact FP32 accumulation in the tensor cores, or a
wrong slice pair, level weight or scale, breaks it); inputs whose slice digits are all at their
largest magnitude must give the exact sum of the kept slice products (computed in rationals),
which pins the FP32 accumulators at their 2^24 bound; real inputs must match the FP64 product
within 1e-13 of max |M| over ragged tiles, one and two terms, zero rows, rows whose magnitudes
differ by 2^200, and a K long enough to be split across CTAs."""
import numpy as np
import pytest

from oracle import tucker_oracle as O
from paper_0711_2023_gb300 import synth

pytestmark = pytest.mark.gpu


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("rows,K1,K2", [(1, 1, 0), (63, 31, 0), (130, 33, 65), (300, 1000, 0),
                                        (257, 5000, 3000)])
def test_integer_inputs_exact(tucker_lib, rows, K1, K2):
    u1 = synth.uniform_matrix(rows, K1, 900 + rows)
    Y1 = np.floor(u1 * 2001.0) - 1000.0                   # integers in [-1000, 1000]
    Y2 = None
    if K2:
        Y2 = np.floor(synth.uniform_matrix(rows, K2, 901 + rows) * 129.0) - 64.0
    M = tucker_lib.tucker_gram(Y1, Y2).cpu().numpy()
    I1 = Y1.astype(np.int64)
    ref = I1 @ I1.T
    if K2:
        I2 = Y2.astype(np.int64)
        ref = ref + I2 @ I2.T
    assert np.array_equal(M, ref.astype(np.float64))


@pytest.mark.parametrize("rows,K1,K2", [(7, 13, 0), (128, 64, 0), (200, 777, 333),
                                        (513, 4000, 0), (1000, 20000, 0)])
def test_real_inputs(tucker_lib, rows, K1, K2):
    Y1 = synth.uniform_matrix(rows, K1, 910 + rows) - 0.5
    Y2 = synth.uniform_matrix(rows, K2, 911 + rows) - 0.5 if K2 else None
    M = tucker_lib.tucker_gram(Y1, Y2).cpu().numpy()
    ref = O.gram(Y1) + (O.gram(Y2) if K2 else 0)
    assert rel_err(M, ref) <= 1e-13
    assert np.array_equal(M, M.T)


def test_row_scales_and_zero_rows(tucker_lib):
    rows, K = 150, 2000
    Y = synth.uniform_matrix(rows, K, 920) - 0.5
    scale = 2.0 ** np.linspace(-100, 100, rows)
    Y = Y * scale[:, None]
    Y[[3, 77, 149]] = 0.0
    M = tucker_lib.tucker_gram(Y).cpu().numpy()
    ref = O.gram(Y)
    # each entry against its own row and column scale: |dM_ij| <= 1e-13 |y_i| |y_j|
    n = np.linalg.norm(Y, axis=1)
    bound = 1e-13 * np.outer(n, n)
    assert np.all(np.abs(M - ref) <= bound)
    assert np.all(M[[3, 77, 149]] == 0.0) and np.all(M[:, [3, 77, 149]] == 0.0)


def test_long_k_split(tucker_lib):
    # K long enough to be split into several K ranges, whose integer partials are summed
    rows, K = 256, 200_000
    Y = synth.uniform_matrix(rows, K, 930) - 0.5
    M = tucker_lib.tucker_gram(Y).cpu().numpy()
    assert rel_err(M, O.gram(Y)) <= 1e-13
    # the same Gram from two half-width terms (different K split points): equal within rounding
    M2 = tucker_lib.tucker_gram(Y[:, :K // 2].copy(), Y[:, K // 2:].copy()).cpu().numpy()
    assert rel_err(M2, M) <= 1e-14


def _digit_value(digits):
    """The value with these 8-bit slices at scale exponent 0: Z 2^-(8 S),
    Z = sum_s q_s 256^(S-1-s) (exact in FP64 when Z has at most 53 significant bits)."""
    from fractions import Fraction
    S = len(digits)
    Z = sum(d * 256 ** (S - 1 - s) for s, d in enumerate(digits))
    y = Fraction(Z, 2 ** (8 * S))
    assert float(y) == y
    return float(y)


def _kept_pairs(S):
    """The slice pairs the tensor-core product sums: s + t < S, and for even S the square pair
    (S/2, S/2) of level S."""
    pairs = [(s, t) for s in range(S) for t in range(S) if s + t < S]
    return pairs + ([(S // 2, S // 2)] if S % 2 == 0 else [])


def _kept_sum(qa, qb):
    """sum over the kept pairs of qa_s qb_t 2^-(8 (s + t + 2)), exactly."""
    from fractions import Fraction
    return sum(Fraction(qa[s] * qb[t], 2 ** (8 * (s + t + 2))) for s, t in _kept_pairs(len(qa)))


def _max_digit_columns(K, qa, qb):
    """Columns with slices qa, except every 16th with qb: with qa odd and qb even, every
    16-column MMA step adds an odd number to each level, so a dropped low bit shows."""
    ya, yb = _digit_value(qa), _digit_value(qb)
    is_b = np.arange(K) % 16 == 0
    return np.where(is_b, yb, ya), int(is_b.sum())


def test_max_digit_accumulation_exact(tucker_lib):
    # Slice digits near their largest magnitude (127, and 126 in every 16th column) and every
    # row of one sign, so each level's FP32 accumulator climbs to just below 2^24 before it is
    # read out: a rounding in the tensor cores' accumulation, or a readout chunk one stage too
    # long, moves a level sum and the result.  K spans several level-0 chunks (1024 columns)
    # and a ragged stage.  Expected: the exact sum of the kept slice products, in rationals.
    qa, qb = [127] * 6, [126] * 6
    K = 4 * 1024 + 77
    row, nb = _max_digit_columns(K, qa, qb)
    sign = np.array([1.0, -1.0, 1.0, 1.0, -1.0])
    M = tucker_lib.tucker_gram(np.outer(sign, row)).cpu().numpy()
    T = float((K - nb) * _kept_sum(qa, qa) + nb * _kept_sum(qb, qb))
    ref = np.outer(sign, sign) * T
    assert np.all(np.abs(M - ref) <= 2.0 * np.spacing(T)), (M[0, 0], T)


def test_gemm_max_digit_accumulation_exact(tucker_lib):
    # The same for the 7-slice product of tucker_gemm (last digit 124: the values stay within
    # 53 bits).
    qa, qb = [127] * 6 + [124], [126] * 6 + [124]
    K = 2 * 1024 + 45
    col, nb = _max_digit_columns(K, qa, qb)
    A = np.outer(np.array([1.0, -1.0, 1.0]), col)
    B = np.outer(col, np.ones(2))
    C = tucker_lib.tucker_gemm(A, B).cpu().numpy()
    T = float((K - nb) * _kept_sum(qa, qa) + nb * _kept_sum(qb, qb))
    ref = np.array([[T, T], [-T, -T], [T, T]])
    assert np.all(np.abs(C - ref) <= 2.0 * np.spacing(T)), (C[0, 0], T)


def test_empty_k(tucker_lib):
    import torch
    Y = torch.zeros((5, 0), dtype=torch.float64, device="cuda")
    M = tucker_lib.tucker_gram(Y).cpu().numpy()
    assert np.array_equal(M, np.zeros((5, 5)))


# ---- the general product C = A B (eight slices), used by the eigensolver for M V ------------

@pytest.mark.parametrize("m,K,n", [(1, 1, 1), (130, 33, 65), (300, 2000, 150), (2000, 2000, 7)])
def test_gemm_integer_inputs_exact(tucker_lib, m, K, n):
    A = np.floor(synth.uniform_matrix(m, K, 940 + m) * 2001.0) - 1000.0
    B = np.floor(synth.uniform_matrix(K, n, 941 + n) * 257.0) - 128.0
    C = tucker_lib.tucker_gemm(A, B).cpu().numpy()
    ref = A.astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(C, ref.astype(np.float64))


@pytest.mark.parametrize("m,K,n", [(7, 13, 3), (257, 1000, 150), (1000, 3000, 64)])
def test_gemm_real_inputs(tucker_lib, m, K, n):
    A = synth.uniform_matrix(m, K, 950 + m) - 0.5
    B = synth.uniform_matrix(K, n, 951 + n) - 0.5
    C = tucker_lib.tucker_gemm(A, B).cpu().numpy()
    ref = A @ B
    # per entry against its row and column scales
    bound = 1e-15 * np.outer(np.abs(A).max(axis=1), np.abs(B).max(axis=0)) * K
    assert np.all(np.abs(C - ref) <= bound)


def test_gemm_diagonal_dominant(tucker_lib):
    # The eigensolver's case: a Gram-like M whose diagonal is ~240x its off-diagonal entries,
    # times orthonormal columns.  Column errors must stay far below 1e-13 of the diagonal, the
    # accuracy the FP64 eigensolver's locking test needs.
    n, k = 1000, 40
    M = synth.uniform_matrix(n, n, 960) * 28.0
    M = 0.5 * (M + M.T) + 6700.0 * np.eye(n)
    V, _ = np.linalg.qr(synth.uniform_matrix(n, k, 961) - 0.5)
    C = tucker_lib.tucker_gemm(M, V).cpu().numpy()
    err = np.linalg.norm(C - M @ V, axis=0).max()
    assert err <= 1e-14 * 6700.0


def test_gemm_empty_k(tucker_lib):
    import torch
    A = torch.zeros((4, 0), dtype=torch.float64, device="cuda")
    B = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    assert np.array_equal(tucker_lib.tucker_gemm(A, B).cpu().numpy(), np.zeros((4, 3)))


# ---- the HOOI projection with its rank updates on the tensor cores ---------------------------

@pytest.mark.parametrize("J", [(50, 60, 70), (33, 64, 100)])
def test_ttmc_tensor_cores(tucker_lib, J):
    # sizes above the dispatch threshold (J_m J_o >= 2048, >= 4096 fibers): every mode's
    # projection runs as per-slice products on the tensor cores
    X = synth.random_sparse_tensor((200, 150, 180), 200_000, synth.config_seed(970))
    # empty slices of mode 0: rows of Y_(1) that must come out zero
    keep = X.idx[0] % 9 != 4
    idx, val = X.idx[:, keep], X.val[keep]
    T = tucker_lib.tucker_tensor_create(idx, val, X.dims)
    U = [synth.uniform_matrix(X.dims[a], J[a], 971 + a) - 0.5 for a in range(3)]
    for n in range(3):
        m, o = O.other_modes(n)
        Y = tucker_lib.tucker_ttmc(T, n, U[m], U[o]).cpu().numpy()
        ref = O.unfold_dense(O.ttmc(X.dims, idx, val, n, U), n)
        assert rel_err(Y, ref) <= 1e-13, n
    Y0 = tucker_lib.tucker_ttmc(T, 0, U[1], U[2]).cpu().numpy()
    assert np.all(Y0[4::9] == 0.0)
