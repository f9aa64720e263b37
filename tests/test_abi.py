"""The C ABI library builds, loads without a GPU, and exports every function that
include/tucker.h declares.  No compute call is made here."""
import ctypes

from paper_0711_2023_gb300 import build, tucker


def test_library_builds_and_exports_header_functions():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = tucker.header_functions()
    assert "tucker_hooi" in names and "tucker_eig_topk" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # every declared function also has a binding of the same name
    assert not [n for n in names if not hasattr(tucker, n)]


def test_strerror_is_host_only():
    lib = tucker._lib()
    assert lib.tucker_strerror(tucker.TUCKER_EINVAL).decode() == "invalid argument"
    assert lib.tucker_strerror(tucker.TUCKER_EEMPTY).decode().startswith("empty tensor")
    assert lib.tucker_strerror(12345).decode() == "unknown status"


def test_null_arguments_rejected_without_gpu():
    lib = tucker._lib()
    out = ctypes.c_void_p()
    assert lib.tucker_tensor_create(None, None, ctypes.byref(out)) == tucker.TUCKER_EINVAL
    coo = tucker.tucker_coo()
    coo.dims[0], coo.dims[1], coo.dims[2] = 0, 3, 3           # empty mode: invalid
    assert lib.tucker_tensor_create(ctypes.byref(coo), None, ctypes.byref(out)) == tucker.TUCKER_EINVAL
    assert lib.tucker_hooi(None, None, None, None) == tucker.TUCKER_EINVAL
