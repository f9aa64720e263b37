"""The kernel-variant autotuner of the mixed projections: decisions are taken once per shape
class, report both variants' times, and later calls reuse them (same bits); with tuning
disabled new classes use the default variant."""
import numpy as np
import pytest
import torch

from paper_0711_2023_gb300 import synth

pytestmark = pytest.mark.gpu


def make(tk, dims, nnz, seed):
    X = synth.random_sparse_tensor(dims, nnz, synth.config_seed(seed))
    return tk.tucker_tensor_create(torch.from_numpy(X.idx).cuda(), torch.from_numpy(X.val).cuda(),
                                   X.dims)


def test_autotune_decisions_and_reuse(tucker_lib):
    tk = tucker_lib
    tk.tucker_autotune_enable(True)
    T = make(tk, (230, 210, 190), 90_000, 31)
    J = (36, 40, 44)                      # HOOI tiles of 64 columns: both TTMc variants apply
    # modes above 256 rows: MP's mixed Grams take the projection kernels (smaller modes use the
    # fused projection + Gram, which has no variants)
    T2 = make(tk, (300, 280, 270), 200_000, 33)
    n0 = tk.tucker_autotune_count()
    r1 = tk.tucker_hooi(T, J, tol=-np.inf, max_iter=2, precision="mixed")
    r1mp = tk.tucker_mp(T2, J, tol=-np.inf, max_iter=2, precision="mixed")
    n1 = tk.tucker_autotune_count()
    assert n1 > n0
    fams = set()
    for i in range(n1):
        d = tk.tucker_autotune_decision(i)
        assert d["family"] in (1, 2) and d["variant"] in (0, 1)
        assert d["ms_kept"] > 0 and d["ms_other"] > 0 and d["ms_kept"] <= d["ms_other"]
        fams.add(d["family"])
    assert fams == {1, 2}
    # the same shape classes again: no new decisions, identical results
    r2 = tk.tucker_hooi(T, J, tol=-np.inf, max_iter=2, precision="mixed")
    r2mp = tk.tucker_mp(T2, J, tol=-np.inf, max_iter=2, precision="mixed")
    assert tk.tucker_autotune_count() == n1
    assert r2["fit_history"] == r1["fit_history"] and r2mp["fit_history"] == r1mp["fit_history"]
    for a in range(3):
        assert torch.equal(r1["U"][a], r2["U"][a])
    with pytest.raises(tk.TuckerError):
        tk.tucker_autotune_decision(n1)


def test_autotune_disabled_uses_default(tucker_lib):
    tk = tucker_lib
    tk.tucker_autotune_enable(False)
    try:
        T = make(tk, (150, 170, 160), 60_000, 32)
        n0 = tk.tucker_autotune_count()
        r = tk.tucker_hooi(T, (52, 48, 40), tol=-np.inf, max_iter=2, precision="mixed")
        assert tk.tucker_autotune_count() == n0
        assert 0.0 < r["fit"] < 1.0
    finally:
        tk.tucker_autotune_enable(True)
