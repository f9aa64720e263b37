"""The opt-in profiling interface: timed kernel records, the eigensolver's counters, the launch
counter, and that switching profiling off leaves the library usable (records without events,
the counters, must not leave a CUDA error behind for the next launch to report)."""
import numpy as np
import pytest
import torch

from paper_0711_2023_gb300 import synth

pytestmark = pytest.mark.gpu


def make(tk, dims, nnz, seed):
    X = synth.random_sparse_tensor(dims, nnz, synth.config_seed(seed))
    return tk.tucker_tensor_create(torch.from_numpy(X.idx).cuda(), torch.from_numpy(X.val).cuda(),
                                   X.dims)


def test_profile_records_and_counters(tucker_lib):
    tk = tucker_lib
    T = make(tk, (300, 280, 260), 60_000, 11)
    J = (20, 20, 20)
    tk.tucker_profile_enable(True)
    n0 = tk.tucker_launch_count()
    r = tk.tucker_hooi(T, J, tol=-np.inf, max_iter=2)
    torch.cuda.synchronize()
    assert tk.tucker_launch_count() > n0
    n, ms, fl, by = tk.tucker_profile_query("gram_f64_tc")
    assert n == 6 and ms > 0 and fl > 0 and by > 0   # three modes, two passes
    n, ms, fl, by = tk.tucker_profile_query("gram_ozaki")
    assert n == 6 and ms > 0 and fl > 0 and by > 0   # its tensor-core kernel
    n, ms, _, _ = tk.tucker_profile_query("eig_topk")
    assert n == 6 + 2 and ms > 0                      # plus the HO-SVD start of B and C
    n_out, _, outer, _ = tk.tucker_profile_query("eig_outer")
    assert n_out == 8 and outer >= 8
    n_s, ms_s, steps, _ = tk.tucker_profile_query("syev_steps")
    assert n_s >= 8 and ms_s == 0 and steps >= 2 * n_s
    assert tk.tucker_profile_query("no_such_record") == (0, 0.0, 0.0, 0.0)
    tk.tucker_profile_enable(False)
    # nothing recorded once off, and the next calls still run
    r2 = tk.tucker_hooi(T, J, tol=-np.inf, max_iter=2)
    assert tk.tucker_profile_query("gram_f64_tc")[0] == 0
    assert r2["fit_history"] == r["fit_history"]
    T2 = make(tk, (50, 40, 30), 5_000, 12)
    tk.tucker_hosvd(T2, (5, 5, 5))
