"""Plain FP64 CPU oracle of the four sparse third-order Tucker methods (HO-SVD, HOOI, SP, MP).

TEST INFRASTRUCTURE ONLY.  This module is the correctness reference for the GPU library.  Only
the test suite, the smoke check and the benchmark's CPU-baseline leg may import it; the product
path never calls it and it shares no code with the CUDA library.

Everything here is written straight from the paper's definitions (Section 2, "Notation") and
algorithm figures (Section 3).  It is deliberately plain: sparse tensors are scipy COO/CSR
matrices of an unfolding, intermediate tensors are dense numpy arrays, every product is one
library matmul/tensordot call, eigenvectors come from numpy.linalg.eigh.  No blocking, fusion
or reordering beyond what the definitions state.

Conventions (readings of the paper where it is silent or MATLAB-specific):
  * indices are 0-based and tensors/cores row-major (the paper is 1-based and column-major);
  * duplicate coordinates are summed, in stable-sort order (MATLAB sparse() sums them);
  * "leading eigenvectors of M M^T" (SP, MP) is taken as leading eigenvectors of M: every M
    here is a sum of Gram matrices, symmetric positive semi-definite, so M M^T = M^2 has the
    same eigenvectors in the same order;
  * eigenvector sign rule: in every column the entry of largest magnitude is positive (lowest
    row index on a tie);
  * fit = 1 - sqrt(max(0, |X|^2 - |G|^2)) / |X| (equal to the reconstruction-based fit of the
    fit equation when the factors are orthonormal and G is the projected core);
    fit_explicit() evaluates the reconstruction itself on small tensors;
  * stop tests are signed: HOOI and MP stop when fit_t - fit_{t-1} < tol with fit_0 = 0; SP
    stops when Delta_G(t) = 1 - |G^(t-1)| / |G^(t)| < tol, tested from t = 2; max_iter
    counts passes of the main loop;
  * SP's random C is drawn outside (seeded U[0,1] matrix) and its columns normalised here.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sps

MODES = (0, 1, 2)


def other_modes(n):
    """The two modes other than n, in increasing order (m < o)."""
    return tuple(a for a in MODES if a != n)


# ----------------------------------------------------------------------------------------------
# Sparse tensor handling (the role of the paper's sort + slice step, appendix functions
# sort_index / slice): duplicates, mode orderings.
# ----------------------------------------------------------------------------------------------

def canonical_coo(dims, idx, val):
    """Sum duplicate coordinates.  Returns (idx, val) sorted by (i1, i2, i3); duplicates are
    added in their original COO order."""
    idx = np.asarray(idx, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    order = np.lexsort((idx[2], idx[1], idx[0]))        # stable
    idx, val = idx[:, order], val[order]
    if idx.shape[1] == 0:
        return idx, val
    new = np.ones(idx.shape[1], dtype=bool)
    new[1:] = np.any(idx[:, 1:] != idx[:, :-1], axis=0)
    starts = np.flatnonzero(new)
    seg = np.cumsum(new) - 1
    sums = np.zeros(starts.shape[0])
    np.add.at(sums, seg, val)            # unbuffered, in order: duplicates add in COO order
    return idx[:, starts], sums


def csf_ordering(dims, idx, val, order):
    """Compressed ordering of the nonzeros for the mode triple order = (n, m, o): nonzeros
    stably sorted by (i_n, i_m, i_o); a fiber is a run sharing (i_n, i_m).

    Returns a dict with
      perm       int64 [nnz]   position in the input COO of each sorted nonzero
      root_ptr   int64 [I_n+1] first fiber of each i_n
      fiber_idx  int32 [F]     i_m of each fiber
      fiber_ptr  int64 [F+1]   first nonzero of each fiber
      leaf_idx   int32 [nnz]   i_o of each sorted nonzero
      val        f64  [nnz]    values in sorted order
    This is the compressed form of the paper's sorted slice files (appendix sort_index/slice)."""
    n, m, o = order
    idx = np.asarray(idx, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    perm = np.lexsort((idx[o], idx[m], idx[n]))          # stable: ties keep COO order
    a, b, c = idx[n][perm], idx[m][perm], idx[o][perm]
    nnz = perm.shape[0]
    newf = np.ones(nnz, dtype=bool)
    if nnz:
        newf[1:] = (a[1:] != a[:-1]) | (b[1:] != b[:-1])
    fstart = np.flatnonzero(newf)
    F = fstart.shape[0]
    fiber_ptr = np.append(fstart, nnz).astype(np.int64)
    fiber_root = a[fstart]
    root_ptr = np.searchsorted(fiber_root, np.arange(dims[n] + 1), side="left").astype(np.int64)
    return dict(perm=perm, root_ptr=root_ptr, fiber_idx=b[fstart].astype(np.int32),
                fiber_ptr=fiber_ptr, leaf_idx=c.astype(np.int32), val=val[perm], nfibers=F)


def norm2(val):
    """|X|_F^2 (Section 2, fit equation): sum of squared nonzeros."""
    v = np.asarray(val, dtype=np.float64)
    return float(np.dot(v, v))


def to_dense(dims, idx, val):
    X = np.zeros(dims)
    np.add.at(X, (idx[0], idx[1], idx[2]), val)
    return X


# ----------------------------------------------------------------------------------------------
# n-mode products and matricization (Section 2, eq. 1 and the matricization paragraph)
# ----------------------------------------------------------------------------------------------

def unfold_sparse(dims, idx, val, n):
    """X_(n) as a scipy CSR matrix of size I_n x (I_m I_o).  The column order (i_m * I_o + i_o)
    differs from the paper's (lower mode fastest); Gram matrices do not depend on it."""
    m, o = other_modes(n)
    idx = np.asarray(idx, dtype=np.int64)
    cols = idx[m] * dims[o] + idx[o]
    return sps.csr_matrix((np.asarray(val, dtype=np.float64), (idx[n], cols)),
                          shape=(dims[n], dims[m] * dims[o]))


def unfold_dense(T, n):
    """Mode-n matricization of a dense 3-way array (columns in row-major order of the rest)."""
    return np.moveaxis(T, n, 0).reshape(T.shape[n], -1)


def nmode_product_sparse(dims, idx, val, n, A):
    """Y = X x_n A for sparse X and dense A (J x I_n): y_{..j..} = sum_{i_n} x_{..i_n..} a_{j i_n}
    (eq. 1).  Returns a dense array with mode n of size J."""
    A = np.asarray(A, dtype=np.float64)
    rest = other_modes(n)
    idx = np.asarray(idx, dtype=np.int64)
    rows = idx[rest[0]] * dims[rest[1]] + idx[rest[1]]
    Xm = sps.csr_matrix((np.asarray(val, dtype=np.float64), (rows, idx[n])),
                        shape=(dims[rest[0]] * dims[rest[1]], dims[n]))
    Z = np.asarray(Xm @ A.T)                              # (I_r0 I_r1) x J
    Z = Z.reshape(dims[rest[0]], dims[rest[1]], A.shape[0])
    return np.moveaxis(Z, 2, n)


def nmode_product_dense(T, n, A):
    """Y = T x_n A for a dense array T (eq. 1)."""
    return np.moveaxis(np.tensordot(np.asarray(A, dtype=np.float64), T, axes=(1, n)), 0, n)


def ttm(dims, idx, val, m, U):
    """Single projection Y = X x_m U^T (U is I_m x J_m): a dense tensor with mode m of size J_m.
    This is the slice projection of SP and MP: sum over slices of X_slice U U^T X_slice^T
    equals Y_(n) Y_(n)^T for the mode n that indexes the rows."""
    return nmode_product_sparse(dims, idx, val, m, np.asarray(U).T)


def ttmc(dims, idx, val, n, U):
    """Y = X x_m U_m^T x_o U_o^T for the two modes m, o other than n (HOOI's U, V, W tensors of
    Figure hooi3, and the Z tensor of Figure hooin).  U is the list of three factors (U[n] is
    not used).  Returns the dense tensor with modes m, o of sizes J_m, J_o."""
    m, o = other_modes(n)
    T = nmode_product_sparse(dims, idx, val, o, np.asarray(U[o]).T)
    return nmode_product_dense(T, m, np.asarray(U[m]).T)


def gram(Yn):
    """M = Y_(n) Y_(n)^T for a matricized Y_(n)."""
    Yn = np.asarray(Yn, dtype=np.float64)
    return Yn @ Yn.T


def unfolding_gram(dims, idx, val, n):
    """M_n = X_(n) X_(n)^T (Figure HO-SVD3)."""
    Xn = unfold_sparse(dims, idx, val, n)
    return np.asarray((Xn @ Xn.T).todense())


def core(dims, idx, val, U):
    """G = [[X; A^T, B^T, C^T]] (Tucker operator of Section 2 applied with transposed factors)."""
    T = ttmc(dims, idx, val, 0, U)
    return nmode_product_dense(T, 0, np.asarray(U[0]).T)


# ----------------------------------------------------------------------------------------------
# Leading eigenvectors
# ----------------------------------------------------------------------------------------------

def sign_fix(V):
    """Make the entry of largest magnitude of every column positive (first such row on ties)."""
    V = np.array(V, dtype=np.float64, copy=True)
    if V.size == 0:
        return V
    piv = np.argmax(np.abs(V), axis=0)
    s = np.sign(V[piv, np.arange(V.shape[1])])
    s[s == 0] = 1.0
    return V * s


def leading_eigvecs(M, J):
    """J leading eigenvectors of the symmetric matrix M (largest eigenvalues first), sign-fixed,
    and all eigenvalues in descending order.  numpy.linalg.eigh (LAPACK syevd) is the library
    eigensolver used as this step."""
    M = np.asarray(M, dtype=np.float64)
    M = 0.5 * (M + M.T)
    w, V = np.linalg.eigh(M)
    w, V = w[::-1], V[:, ::-1]
    return sign_fix(V[:, :J]), w


# ----------------------------------------------------------------------------------------------
# Fit (Section 2, fit equation) and stop tests (Delta_fit equation, Delta_G equation)
# ----------------------------------------------------------------------------------------------

def fit_from_core(nX2, G):
    g2 = float(np.sum(np.asarray(G) ** 2))
    return 1.0 - np.sqrt(max(0.0, nX2 - g2)) / np.sqrt(nX2)


def fit_explicit(dims, idx, val, G, U):
    """fit = 1 - |X - Xhat|_F / |X|_F with Xhat = [[G; A, B, C]] built densely (small only)."""
    X = to_dense(dims, idx, val)
    Xh = nmode_product_dense(nmode_product_dense(nmode_product_dense(
        np.asarray(G), 0, U[0]), 1, U[1]), 2, U[2])
    return 1.0 - np.linalg.norm((X - Xh).ravel()) / np.linalg.norm(X.ravel())


def _result(G, U, nX2, fits, extra=None):
    r = dict(G=np.asarray(G), U=[np.asarray(u) for u in U], fit=fits[-1], iters=len(fits),
             fit_history=list(fits), normX2=nX2)
    if extra:
        r.update(extra)
    return r


def _prep(dims, idx, val):
    idx, val = canonical_coo(dims, idx, val)
    nX2 = norm2(val)
    if nX2 == 0.0:
        raise ValueError("empty tensor: |X| = 0 makes the fit undefined")
    return idx, val, nX2


def _check_core(dims, J):
    for a in MODES:
        if not (1 <= J[a] <= dims[a]):
            raise ValueError("core size out of range")


# ----------------------------------------------------------------------------------------------
# The four methods
# ----------------------------------------------------------------------------------------------

def hosvd(dims, idx, val, J):
    """Figure HO-SVD3: A, B, C <- leading eigenvectors of X_(n) X_(n)^T; G <- [[X; A^T,B^T,C^T]]."""
    _check_core(dims, J)
    idx, val, nX2 = _prep(dims, idx, val)
    U = [leading_eigvecs(unfolding_gram(dims, idx, val, n), J[n])[0] for n in MODES]
    G = core(dims, idx, val, U)
    return _result(G, U, nX2, [fit_from_core(nX2, G)])


def hooi_update(dims, idx, val, n, U, Jn):
    """One factor update of Figure hooi3: the projection Y = X x_m U_m^T x_o U_o^T with the
    newest other factors, and the J_n leading eigenvectors of Y_(n) Y_(n)^T.  Returns (U_n, Y)."""
    Y = ttmc(dims, idx, val, n, U)
    return leading_eigvecs(gram(unfold_dense(Y, n)), Jn)[0], Y


def hooi(dims, idx, val, J, tol=1e-4, max_iter=50, init=None):
    """Figure hooi3 with the Delta_fit stop test.  B, C start from HO-SVD (or `init`); A is
    not initialised.  Each pass: U = [[X; I, B^T, C^T]] -> A; V = [[X; A^T, I, C^T]] -> B;
    W = [[X; A^T, B^T, I]] -> C (each with the newest factors); then G and the fit."""
    _check_core(dims, J)
    idx, val, nX2 = _prep(dims, idx, val)
    U = [None, None, None]
    for n in (1, 2):
        if init is not None and init[n] is not None:
            U[n] = np.asarray(init[n], dtype=np.float64)
        else:
            U[n] = leading_eigvecs(unfolding_gram(dims, idx, val, n), J[n])[0]
    fits, old = [], 0.0
    G = None
    for _ in range(max_iter):
        for n in MODES:
            U[n], Y = hooi_update(dims, idx, val, n, U, J[n])
        G = nmode_product_dense(Y, 2, U[2].T)             # W x_3 C^T = [[X; A^T, B^T, C^T]]
        f = fit_from_core(nX2, G)
        fits.append(f)
        if f - old < tol:
            break
        old = f
    return _result(G, U, nX2, fits)


def sp_initial_C(C_raw):
    """Figure sp3 initialisation: the random matrix with its columns normalised to unit length."""
    C = np.array(C_raw, dtype=np.float64, copy=True)
    return C / np.linalg.norm(C, axis=0)


def sp(dims, idx, val, J, C_raw, tol=1e-4, max_iter=50):
    """Figure sp3 with the Delta_G stop test.  Each pass:
       M13 = sum_j X_{:j:} C C^T X_{:j:}^T = Gram((X x_3 C^T)_(1)) -> A
       M21 = sum_k X_{::k}^T A A^T X_{::k} = Gram((X x_1 A^T)_(2)) -> B
       M32 = sum_i X_{i::}^T B B^T X_{i::} = Gram((X x_2 B^T)_(3)) -> C
    then G = [[X; A^T, B^T, C^T]]."""
    _check_core(dims, J)
    idx, val, nX2 = _prep(dims, idx, val)
    U = [None, None, sp_initial_C(C_raw)]
    fits, gnorms = [], []
    G = None
    for t in range(max_iter):
        for n, m in ((0, 2), (1, 0), (2, 1)):
            Y = ttm(dims, idx, val, m, U[m])
            U[n] = leading_eigvecs(gram(unfold_dense(Y, n)), J[n])[0]
        G = core(dims, idx, val, U)
        gn = float(np.linalg.norm(G.ravel()))
        fits.append(fit_from_core(nX2, G))
        gnorms.append(gn)
        if t >= 1 and (1.0 - gnorms[-2] / gn) < tol:
            break
    return _result(G, U, nX2, fits, dict(gnorm_history=gnorms))


def mp_init_matrix(dims, idx, val, n):
    """Pseudo HO-SVD matrix of Figure mp3, as written: the sum of the slice Gram sums over the
    two other slicing modes, e.g. M_2 = sum_i X_{i::} X_{i::}^T + sum_k X_{::k}^T X_{::k}."""
    m, o = other_modes(n)
    idx = np.asarray(idx, dtype=np.int64)
    M = np.zeros((dims[n], dims[n]))
    for s in (m, o):                       # slice on mode s; the remaining free mode is r
        r = o if s == m else m
        order = np.argsort(idx[s], kind="stable")          # group the nonzeros by slice
        bounds = np.searchsorted(idx[s][order], np.arange(dims[s] + 1))
        for t in range(dims[s]):           # slice X_t: rows i_n, columns i_r, at i_s = t
            sel = order[bounds[t]:bounds[t + 1]]
            Xt = sps.csr_matrix((val[sel], (idx[n][sel], idx[r][sel])), shape=(dims[n], dims[r]))
            M += np.asarray((Xt @ Xt.T).todense())
    return M


def mp_term(dims, idx, val, n, m, Um):
    """One slice sum of Figure mp3 for output mode n: sum over the slices of X along the third
    mode of X_s U_m U_m^T X_s^T, i.e. Gram((X x_m U_m^T)_(n))."""
    return gram(unfold_dense(ttm(dims, idx, val, m, Um), n))


def mp_update(dims, idx, val, n, U, Jn):
    """One factor update of Figure mp3: the J_n leading eigenvectors of the sum, over the two
    other modes m, of the slice sums Gram((X x_m U_m^T)_(n))."""
    M = np.zeros((dims[n], dims[n]))
    for m in other_modes(n):
        M += mp_term(dims, idx, val, n, m, U[m])
    return leading_eigvecs(M, Jn)[0]


def mp(dims, idx, val, J, tol=1e-4, max_iter=50, init=None):
    """Figure mp3 with the Delta_fit stop test.  Pseudo HO-SVD initialisation of B and C (or
    `init`, as in hooi), then
    each pass
       M1 = Gram((X x_2 B^T)_(1)) + Gram((X x_3 C^T)_(1)) -> A
       M2 = Gram((X x_1 A^T)_(2)) + Gram((X x_3 C^T)_(2)) -> B
       M3 = Gram((X x_2 B^T)_(3)) + Gram((X x_1 A^T)_(3)) -> C
    (the slice sums of Figure mp3, e.g. sum_k X_{::k} B B^T X_{::k}^T = Gram((X x_2 B^T)_(1)));
    then G and the fit."""
    _check_core(dims, J)
    idx, val, nX2 = _prep(dims, idx, val)
    U = [None, None, None]
    for n in (1, 2):
        if init is not None and init[n] is not None:
            U[n] = np.asarray(init[n], dtype=np.float64)
        else:
            U[n] = leading_eigvecs(mp_init_matrix(dims, idx, val, n), J[n])[0]
    fits, old = [], 0.0
    G = None
    for _ in range(max_iter):
        for n in MODES:
            U[n] = mp_update(dims, idx, val, n, U, J[n])
        G = core(dims, idx, val, U)
        f = fit_from_core(nX2, G)
        fits.append(f)
        if f - old < tol:
            break
        old = f
    return _result(G, U, nX2, fits)


def subspace_distance(U, V):
    """|U U^T - V V^T|_2 for two matrices with orthonormal columns."""
    U = np.asarray(U)
    V = np.asarray(V)
    return float(np.linalg.norm(U @ U.T - V @ V.T, 2))


# ----------------------------------------------------------------------------------------------
# Tensors of arbitrary order N (Figures HO-SVDn and hooin) and the fourth-order forms of Slice
# Projection and Multislice Projection (Figures sp4 and mp4).  idx is N x nnz.  For N = 3 these
# functions compute what the third-order ones above do.
# ----------------------------------------------------------------------------------------------

def canonical_coo_n(dims, idx, val):
    """Sum duplicate coordinates of an order-N COO tensor; returns (idx, val) sorted
    lexicographically by (i_1, ..., i_N), duplicates added in their original COO order."""
    idx = np.asarray(idx, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    order = np.lexsort(tuple(idx[a] for a in reversed(range(idx.shape[0]))))
    idx, val = idx[:, order], val[order]
    if idx.shape[1] == 0:
        return idx, val
    new = np.ones(idx.shape[1], dtype=bool)
    new[1:] = np.any(idx[:, 1:] != idx[:, :-1], axis=0)
    starts = np.flatnonzero(new)
    sums = np.zeros(starts.shape[0])
    np.add.at(sums, np.cumsum(new) - 1, val)
    return idx[:, starts], sums


def to_dense_n(dims, idx, val):
    X = np.zeros(dims)
    np.add.at(X, tuple(np.asarray(i) for i in idx), val)
    return X


def _rest(N, n):
    return tuple(a for a in range(N) if a != n)


def unfolding_gram_n(dims, idx, val, n):
    """X_(n) X_(n)^T of an order-N sparse tensor (Figure HO-SVDn)."""
    idx = np.asarray(idx, dtype=np.int64)
    rest = _rest(len(dims), n)
    cols = np.zeros(idx.shape[1], dtype=np.int64)
    for a in rest:
        cols = cols * dims[a] + idx[a]
    ncol = int(np.prod([dims[a] for a in rest]))
    Xn = sps.csr_matrix((np.asarray(val, dtype=np.float64), (idx[n], cols)),
                        shape=(dims[n], ncol))
    return np.asarray((Xn @ Xn.T).todense())


def ttm_n(dims, idx, val, m, U):
    """Y = X x_m U^T for an order-N sparse X (eq. 1): a dense N-way array with mode m of size
    J_m.  (Figures sp4 and mp4: the slice sums over the other modes equal Gram(Y_(n)).)"""
    U = np.asarray(U, dtype=np.float64)
    idx = np.asarray(idx, dtype=np.int64)
    N = len(dims)
    rest = _rest(N, m)
    rows = np.zeros(idx.shape[1], dtype=np.int64)
    for a in rest:
        rows = rows * dims[a] + idx[a]
    nrow = int(np.prod([dims[a] for a in rest]))
    Xm = sps.csr_matrix((np.asarray(val, dtype=np.float64), (rows, idx[m])), shape=(nrow, dims[m]))
    Z = np.asarray(Xm @ U)                                   # (prod rest) x J_m
    Z = Z.reshape([dims[a] for a in rest] + [U.shape[1]])
    return np.moveaxis(Z, N - 1, m)


def ttmc_n(dims, idx, val, n, U):
    """Z = [[X; U_1^T, ..., I_n, ..., U_N^T]] (Figure hooin): every mode but n projected onto
    its factor.  One sparse product on the last projected mode, dense products for the rest."""
    N = len(dims)
    rest = _rest(N, n)
    T = ttm_n(dims, idx, val, rest[-1], U[rest[-1]])
    for a in rest[:-1]:
        T = nmode_product_dense(T, a, np.asarray(U[a]).T)
    return T


def core_n(dims, idx, val, U):
    """G = [[X; U_1^T, ..., U_N^T]] for an order-N tensor."""
    T = ttmc_n(dims, idx, val, 0, U)
    return nmode_product_dense(T, 0, np.asarray(U[0]).T)


def fit_explicit_n(dims, idx, val, G, U):
    """fit = 1 - |X - [[G; U_1, ..., U_N]]|_F / |X|_F, reconstructed densely (small only)."""
    X = to_dense_n(dims, idx, val)
    Xh = np.asarray(G)
    for a in range(len(dims)):
        Xh = nmode_product_dense(Xh, a, U[a])
    return 1.0 - np.linalg.norm((X - Xh).ravel()) / np.linalg.norm(X.ravel())


def _prep_n(dims, idx, val, J):
    N = len(dims)
    for a in range(N):
        if not (1 <= J[a] <= dims[a]):
            raise ValueError("core size out of range")
    idx, val = canonical_coo_n(dims, idx, val)
    nX2 = norm2(val)
    if nX2 == 0.0:
        raise ValueError("empty tensor: |X| = 0 makes the fit undefined")
    return idx, val, nX2


def hosvd_n(dims, idx, val, J):
    """Figure HO-SVDn: A^(n) <- J_n leading eigenvectors of X_(n) X_(n)^T for every n, then the
    core."""
    idx, val, nX2 = _prep_n(dims, idx, val, J)
    U = [leading_eigvecs(unfolding_gram_n(dims, idx, val, n), J[n])[0] for n in range(len(dims))]
    G = core_n(dims, idx, val, U)
    return _result(G, U, nX2, [fit_from_core(nX2, G)])


def hooi_n(dims, idx, val, J, tol=1e-4, max_iter=50, init=None):
    """Figure hooin with the Delta_fit stop test: A^(2..N) from HO-SVD (or `init`), then per pass
    for n = 1..N: Z = [[X; A^(1)T, ..., I_n, ..., A^(N)T]] with the newest factors and
    A^(n) <- J_n leading eigenvectors of Z_(n) Z_(n)^T; then G and the fit."""
    idx, val, nX2 = _prep_n(dims, idx, val, J)
    N = len(dims)
    U = [None] * N
    for n in range(1, N):
        if init is not None and init[n] is not None:
            U[n] = np.asarray(init[n], dtype=np.float64)
        else:
            U[n] = leading_eigvecs(unfolding_gram_n(dims, idx, val, n), J[n])[0]
    fits, old, G = [], 0.0, None
    for _ in range(max_iter):
        for n in range(N):
            Z = ttmc_n(dims, idx, val, n, U)
            U[n] = leading_eigvecs(gram(unfold_dense(Z, n)), J[n])[0]
        G = nmode_product_dense(Z, N - 1, U[N - 1].T)   # the last Z projected on the last mode
        f = fit_from_core(nX2, G)
        fits.append(f)
        if f - old < tol:
            break
        old = f
    return _result(G, U, nX2, fits)


# Figure sp4: A from the slices on modes 2, 3 projected with D (M14), B from those on 3, 4 with
# A (M21), C from those on 1, 4 with B (M32), D from those on 1, 2 with C (M43): 0-based pairs
# (updated mode, projecting mode).
SP4_PAIRS = ((0, 3), (1, 0), (2, 1), (3, 2))


def sp4(dims, idx, val, J, D_raw, tol=1e-4, max_iter=50):
    """Figure sp4 with the Delta_G stop test.  D starts as the random matrix with normalised
    columns; each pass M_nm = sum over the slices of X_s U_m U_m^T X_s^T = Gram((X x_m U_m^T)_(n))
    for the pairs of SP4_PAIRS in order, U_n <- J_n leading eigenvectors of M_nm; then G."""
    if len(dims) != 4:
        raise ValueError("sp4 takes a fourth-order tensor")
    idx, val, nX2 = _prep_n(dims, idx, val, J)
    U = [None, None, None, sp_initial_C(D_raw)]
    fits, gnorms, G = [], [], None
    for t in range(max_iter):
        for n, m in SP4_PAIRS:
            Y = ttm_n(dims, idx, val, m, U[m])
            U[n] = leading_eigvecs(gram(unfold_dense(Y, n)), J[n])[0]
        G = core_n(dims, idx, val, U)
        gn = float(np.linalg.norm(G.ravel()))
        fits.append(fit_from_core(nX2, G))
        gnorms.append(gn)
        if t >= 1 and (1.0 - gnorms[-2] / gn) < tol:
            break
    return _result(G, U, nX2, fits, dict(gnorm_history=gnorms))


def mp4_init_matrix(dims, idx, val, n):
    """Pseudo HO-SVD matrix of Figure mp4, as written: for mode n, the sum over the three ways of
    choosing a second free mode r of the slice Gram sums sum_s X_s X_s^T, the slices X_s being
    the I_n x I_r matrices obtained by fixing the two remaining modes."""
    idx = np.asarray(idx, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    N = len(dims)
    M = np.zeros((dims[n], dims[n]))
    for r in _rest(N, n):
        fixed = [a for a in range(N) if a not in (n, r)]
        key = idx[fixed[0]] * dims[fixed[1]] + idx[fixed[1]]
        order = np.argsort(key, kind="stable")
        bounds = np.searchsorted(key[order], np.arange(dims[fixed[0]] * dims[fixed[1]] + 1))
        for t in range(dims[fixed[0]] * dims[fixed[1]]):
            sel = order[bounds[t]:bounds[t + 1]]
            if sel.size == 0:
                continue
            Xt = sps.csr_matrix((val[sel], (idx[n][sel], idx[r][sel])), shape=(dims[n], dims[r]))
            M += np.asarray((Xt @ Xt.T).todense())
    return M


def mp4_matrix(dims, idx, val, n, U):
    """The matrix M_n of a pass of Figure mp4: the sum, over the three other modes m, of the
    slice sums sum_s X_s U_m U_m^T X_s^T = Gram((X x_m U_m^T)_(n))."""
    M = np.zeros((dims[n], dims[n]))
    for m in _rest(len(dims), n):
        M += gram(unfold_dense(ttm_n(dims, idx, val, m, U[m]), n))
    return M


def mp4_update(dims, idx, val, n, U, Jn):
    """One factor update of Figure mp4: the J_n leading eigenvectors of mp4_matrix."""
    return leading_eigvecs(mp4_matrix(dims, idx, val, n, U), Jn)[0]


def mp4(dims, idx, val, J, tol=1e-4, max_iter=50, init=None):
    """Figure mp4 with the Delta_fit stop test: B, C, D from the pseudo HO-SVD matrices (or
    `init`), then per pass A, B, C, D by mp4_update with the newest factors; then G, fit."""
    if len(dims) != 4:
        raise ValueError("mp4 takes a fourth-order tensor")
    idx, val, nX2 = _prep_n(dims, idx, val, J)
    U = [None] * 4
    for n in (1, 2, 3):
        if init is not None and init[n] is not None:
            U[n] = np.asarray(init[n], dtype=np.float64)
        else:
            U[n] = leading_eigvecs(mp4_init_matrix(dims, idx, val, n), J[n])[0]
    fits, old, G = [], 0.0, None
    for _ in range(max_iter):
        for n in range(4):
            U[n] = mp4_update(dims, idx, val, n, U, J[n])
        G = core_n(dims, idx, val, U)
        f = fit_from_core(nX2, G)
        fits.append(f)
        if f - old < tol:
            break
        old = f
    return _result(G, U, nX2, fits)
