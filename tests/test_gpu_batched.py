"""Batched HOOI and MP over independent tensors drawn like the batched workload (each dim
uniform in [30, 300], density log-uniform in [1%, 20%], each core dim uniform in [4, 32] and at
most its tensor dim): every result must equal the single-tensor call bit for bit (same kernels,
same inputs), and eight of them (the largest, at the recipe's full sizes) must match the FP64
oracle (1e-9 in fit; mixed form 1e-4)."""
import numpy as np
import pytest

from oracle import tucker_oracle as O
from paper_0711_2023_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch(tucker_lib):
    cfgs = synth.batched_configs(20, synth.config_seed(5))
    Xs, Ts, Js = [], [], []
    for t, (dims, nnz, core) in enumerate(cfgs):
        X = synth.random_sparse_tensor(dims, nnz, synth.config_seed(100 + t))
        Xs.append(X)
        Ts.append(tucker_lib.tucker_tensor_create(X.idx, X.val, X.dims))
        Js.append(core)
    return Xs, Ts, Js


_ORACLE = {}


def oracle_fits(method, X, J, t):
    """The oracle's fit history for tensor t (computed once for both precision forms)."""
    if (method, t) not in _ORACLE:
        f = O.hooi if method == "hooi" else O.mp
        _ORACLE[(method, t)] = f(X.dims, X.idx, X.val, J, -np.inf, 3)["fit_history"]
    return _ORACLE[(method, t)]


@pytest.mark.parametrize("method", ["hooi", "mp"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_equals_single(tucker_lib, batch, method, precision):
    Xs, Ts, Js = batch
    fb = getattr(tucker_lib, f"tucker_{method}_batched")
    fs = getattr(tucker_lib, f"tucker_{method}")
    res = fb(Ts, Js, tol=-np.inf, max_iter=3, precision=precision)
    for t in (0, 7, 13, 19):
        one = fs(Ts[t], Js[t], tol=-np.inf, max_iter=3, precision=precision)
        assert res[t]["fit_history"] == one["fit_history"]
        assert np.array_equal(res[t]["G"].cpu().numpy(), one["G"].cpu().numpy())
        for a in range(3):
            assert np.array_equal(res[t]["U"][a].cpu().numpy(), one["U"][a].cpu().numpy())
    tol = 1e-9 if precision == "fp64" else 1e-4
    largest = sorted(range(len(Xs)), key=lambda t: -Xs[t].nnz)[:8]
    for t in largest:
        ref = oracle_fits(method, Xs[t], Js[t], t)
        for a, b in zip(res[t]["fit_history"], ref):
            assert abs(a - b) <= tol, (t, Xs[t].dims, Xs[t].nnz, res[t]["fit_history"], ref)
