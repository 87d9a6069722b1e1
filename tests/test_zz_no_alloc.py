"""kde_exact_noalloc, called through the C-ABI with ctypes.

This entry point is for callers that may not allocate device memory while
they call into the library (for instance while a CUDA graph is being
captured, or when all device memory belongs to the application's own
allocator).  It keeps its accumulators in a fixed array inside the library,
so it must give the same numbers as kde_exact, call after call, even though
every call reuses that array.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _lib():
    import paper_2107_02736_gb300 as pkg
    lib = pkg.load_library()
    fn = lib.kde_exact_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return pkg, lib


def _close(got, want, rel=1e-5, floor=1e-6):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    mask = want >= floor
    err = np.abs(got - want) / np.maximum(want, 1e-300)
    assert np.all(err[mask] <= rel), err[mask].max()
    assert np.all(np.abs(got[~mask] - want[~mask]) <= rel * floor)


@pytest.mark.parametrize("kernel,h", [("gaussian", 2.5), ("laplacian", 9.0)])
def test_exact_noalloc_matches_exact_on_consecutive_calls(kernel, h):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    pkg, lib = _lib()
    rng = np.random.default_rng(0)
    n, d = 5000, 16
    X = rng.standard_normal((n, d)).astype(np.float32)
    index = pkg.KDEIndex(torch.from_numpy(X).cuda(), kernel, h)
    # two calls in a row with different query sets and sizes: the shared
    # array must not carry the first call's sums into the second.  The
    # reference is kde_exact's CUDA-core path (the path this call runs) and
    # the FP64 oracle.
    for call, nq in enumerate((300, 177)):
        Yh = rng.standard_normal((nq, d)).astype(np.float32)
        Y = torch.from_numpy(Yh).cuda()
        want = index.exact(Y, path="cuda").cpu().numpy()
        out = torch.full((nq,), float("nan"), device="cuda")
        st = lib.kde_exact_noalloc(index._h, ctypes.c_void_p(Y.data_ptr()), nq,
                                   ctypes.c_void_p(out.data_ptr()), None)
        assert st == 0, lib.kde_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        _close(got, want)
        _close(got, oracle.exact(X, Yh, kernel, h))
    index.close()


def test_exact_noalloc_rejects_oversized_batch():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    pkg, lib = _lib()
    X = torch.zeros((64, 8), device="cuda")
    index = pkg.KDEIndex(X, "gaussian", 1.0)
    Y = torch.zeros((65537, 8), device="cuda")
    out = torch.zeros(65537, device="cuda")
    st = lib.kde_exact_noalloc(index._h, ctypes.c_void_p(Y.data_ptr()), 65537,
                               ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1
    assert b"65536" in lib.kde_last_error()
    index.close()
