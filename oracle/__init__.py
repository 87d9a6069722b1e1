"""FP64 CPU oracle for the DEANN estimator (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module.  The GPU
library never imports it and shares no code with it.  The arithmetic lives in
``oracle.c``; this module compiles it with gcc and wraps it with ctypes, taking
and returning numpy arrays.

Citations are to the DEANN paper (Karppa, Aumueller, Pagh, arXiv 2107.02736):
the KDE definition (Section 2), Algorithm 1 (DEANN), Lemma RS (random
sampling), the IVF index of Section 4 and Algorithm 2 (permuted sampling).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

GAUSSIAN, EXPONENTIAL, LAPLACIAN = 0, 1, 2
KERNELS = {"gaussian": GAUSSIAN, "exponential": EXPONENTIAL, "laplacian": LAPLACIAN}

OK, EINVAL, ELIMIT = 0, 1, 4


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (OpenMP if gcc offers it)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", src, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, u64, u32, f64 = (ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                   ctypes.c_uint32, ctypes.c_double)
        lib.or_num_threads.restype = i32
        lib.or_set_num_threads.argtypes = [i32]
        lib.or_philox4x32_10.argtypes = [P, P, P]
        lib.or_draw_index.argtypes = [u64, u64, u32, u32, i64]
        lib.or_draw_index.restype = i64
        lib.or_kernel_value.argtypes = [i32, P, P, i32, f64]
        lib.or_kernel_value.restype = f64
        lib.or_exact.argtypes = [P, i64, i32, P, i64, i32, f64, P]
        lib.or_exact_grad.argtypes = [P, i64, i32, P, i64, i32, f64, P, P]
        lib.or_knn.argtypes = [P, i64, i32, P, i64, i32, P, P]
        lib.or_nearest_centroid.argtypes = [P, i64, i32, P, i32, P, P]
        lib.or_kmeans.argtypes = [P, i64, i32, i32, u64, i32, P, P, P]
        lib.or_kmeans.restype = i32
        lib.or_ivf_search.argtypes = [P, i64, i32, P, i32, P, P, i64, i32, i32, P, P, P]
        lib.or_deann.argtypes = [P, i64, i32, P, i64, i32, f64, P, i32, i32, u64, u64,
                                 i32, P, P]
        lib.or_deann.restype = i32
        lib.or_rs.argtypes = [P, i64, i32, P, i64, i32, f64, i32, u64, u64, P, P]
        lib.or_rs.restype = i32
        lib.or_deann_grad.argtypes = [P, i64, i32, P, i64, i32, f64, P, i32, i32, u64,
                                      u64, P, P, P, P]
        lib.or_deann_grad.restype = i32
        lib.or_deannp.argtypes = [P, i64, i32, P, i64, i32, f64, P, P, i32, i32, i64, P, P]
        lib.or_deannp.restype = i32
        lib.or_feistel_perm.argtypes = [u64, i64, i64]
        lib.or_feistel_perm.restype = i64
        lib.or_loo_exact.argtypes = [P, i64, i32, P, i64, i32, f64, P, P, P]
        lib.or_loo_exact.restype = i32
        lib.or_fit_bandwidth.argtypes = [P, i64, i32, P, i64, i32, f64, P, i32, i32, u64, i32,
                                         f64, P, P]
        lib.or_fit_bandwidth.restype = i32
        lib.or_mean_shift.argtypes = [P, i64, i32, P, i32, P, P, i64, f64, i32, i32, i32, u64,
                                      u64, i32, P]
        lib.or_mean_shift.restype = i32
        _lib = lib
        return lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _kern(kernel):
    return KERNELS[kernel] if isinstance(kernel, str) else int(kernel)


def _check(status, what):
    if status == EINVAL:
        raise OracleError(f"{what}: invalid argument")
    if status == ELIMIT:
        raise OracleError(f"{what}: draw cap reached")
    if status != OK:
        raise OracleError(f"{what}: status {status}")


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_num_threads(t: int) -> None:
    _load().or_set_num_threads(int(t))


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def draw_index(seed: int, qid: int, t: int, n: int, stream: int = 0) -> int:
    return int(_load().or_draw_index(seed, qid, t, stream, n))


def kernel_value(kernel, x, y, h):
    x, y = _f32(x), _f32(y)
    return float(_load().or_kernel_value(_kern(kernel), _ptr(x), _ptr(y), x.shape[-1], h))


def exact(X, Y, kernel, h):
    """Exact KDE (Section 2 definition), FP64."""
    X, Y = _f32(X), _f32(Y)
    out = np.zeros(Y.shape[0], dtype=np.float64)
    _load().or_exact(_ptr(X), X.shape[0], X.shape[1], _ptr(Y), Y.shape[0], _kern(kernel),
                     float(h), _ptr(out))
    return out


def exact_grad(X, Y, kernel, h):
    X, Y = _f32(X), _f32(Y)
    dY = np.zeros(Y.shape, dtype=np.float64)
    dl = np.zeros(Y.shape[0], dtype=np.float64)
    _load().or_exact_grad(_ptr(X), X.shape[0], X.shape[1], _ptr(Y), Y.shape[0],
                          _kern(kernel), float(h), _ptr(dY), _ptr(dl))
    return dY, dl


def knn(X, Y, k):
    X, Y = _f32(X), _f32(Y)
    nbr = np.zeros((Y.shape[0], k), dtype=np.int32)
    d2 = np.zeros((Y.shape[0], k), dtype=np.float64)
    _load().or_knn(_ptr(X), X.shape[0], X.shape[1], _ptr(Y), Y.shape[0], k, _ptr(nbr),
                   _ptr(d2))
    return nbr, d2


def nearest_centroid(X, C):
    X, C = _f32(X), _f32(C)
    a = np.zeros(X.shape[0], dtype=np.int32)
    d2 = np.zeros(X.shape[0], dtype=np.float64)
    _load().or_nearest_centroid(_ptr(X), X.shape[0], X.shape[1], _ptr(C), C.shape[0],
                                _ptr(a), _ptr(d2))
    return a, d2


def kmeans(X, L, seed, iters=20):
    """The inverted file's k-means (Philox-stream-1 initial points, `iters`
    Lloyd iterations with farthest-point reseeding, final assignment).
    Returns (centroids float32 L x d, assignment int32, mean squared distance
    of each assignment, status: OK, or ELIMIT when the initial draws ran out)."""
    X = _f32(X)
    n, d = X.shape
    C = np.zeros((L, d), dtype=np.float32)
    a = np.zeros(n, dtype=np.int32)
    obj = np.zeros(iters + 1, dtype=np.float64)
    st = _load().or_kmeans(_ptr(X), n, d, int(L), int(seed) & (2**64 - 1), int(iters), _ptr(C),
                           _ptr(a), _ptr(obj))
    if st == EINVAL:
        raise OracleError("kmeans: invalid arguments")
    return C, a, obj, st


def ivf_search(X, C, assign, Y, nprobe, k):
    X, C, Y, assign = _f32(X), _f32(C), _f32(Y), _i32(assign)
    nq = Y.shape[0]
    probes = np.zeros((nq, nprobe), dtype=np.int32)
    nbr = np.zeros((nq, k), dtype=np.int32)
    d2 = np.zeros((nq, k), dtype=np.float64)
    _load().or_ivf_search(_ptr(X), X.shape[0], X.shape[1], _ptr(C), C.shape[0],
                          _ptr(assign), _ptr(Y), nq, nprobe, k, _ptr(probes), _ptr(nbr),
                          _ptr(d2))
    return probes, nbr, d2


def deann(X, Y, kernel, h, nbr, m, seed, qid_offset=0, mode=0, return_samples=False):
    """DEANN estimate (Algorithm 1) from given neighbour sets (nq x k, -1 pads)."""
    X, Y = _f32(X), _f32(Y)
    nq = Y.shape[0]
    if nbr is None:
        nbr = np.zeros((nq, 0), dtype=np.int32)
    nbr = _i32(nbr).reshape(nq, -1)
    k = nbr.shape[1]
    out = np.zeros(nq, dtype=np.float64)
    samples = np.zeros((nq, m), dtype=np.int32) if return_samples else None
    st = _load().or_deann(_ptr(X), X.shape[0], X.shape[1], _ptr(Y), nq, _kern(kernel),
                          float(h), _ptr(nbr) if k > 0 else None, k, m, seed, qid_offset,
                          mode, _ptr(out), _ptr(samples))
    _check(st, "deann")
    return (out, samples) if return_samples else out


def rs(X, Y, kernel, h, m, seed, qid_offset=0, return_samples=False):
    """Random sampling (Lemma RS): mean kernel value over m draws with repetition."""
    X, Y = _f32(X), _f32(Y)
    nq = Y.shape[0]
    out = np.zeros(nq, dtype=np.float64)
    samples = np.zeros((nq, m), dtype=np.int32) if return_samples else None
    st = _load().or_rs(_ptr(X), X.shape[0], X.shape[1], _ptr(Y), nq, _kern(kernel),
                       float(h), m, seed, qid_offset, _ptr(out), _ptr(samples))
    _check(st, "rs")
    return (out, samples) if return_samples else out


def deann_grad(X, Y, kernel, h, nbr, m, seed, qid_offset=0, gout=None):
    """Pathwise gradient of the DEANN estimate with X_1 and S held fixed.

    Returns (out, dY, dlogh_per_query); dY and dlogh are scaled by gout."""
    X, Y = _f32(X), _f32(Y)
    nq = Y.shape[0]
    if nbr is None:
        nbr = np.zeros((nq, 0), dtype=np.int32)
    nbr = _i32(nbr).reshape(nq, -1)
    k = nbr.shape[1]
    g = None if gout is None else np.ascontiguousarray(gout, dtype=np.float64)
    out = np.zeros(nq, dtype=np.float64)
    dY = np.zeros(Y.shape, dtype=np.float64)
    dl = np.zeros(nq, dtype=np.float64)
    st = _load().or_deann_grad(_ptr(X), X.shape[0], X.shape[1], _ptr(Y), nq,
                               _kern(kernel), float(h), _ptr(nbr) if k > 0 else None, k,
                               m, seed, qid_offset, _ptr(g), _ptr(out), _ptr(dY), _ptr(dl))
    _check(st, "deann_grad")
    return out, dY, dl


def mean_shift(X, C, assign, Y, h, k, m, nprobe, seed, steps, qid_offset=0):
    """Gaussian mean-shift steps y <- y + h^2 grad KDE~(y) / KDE~(y) with the
    DEANN estimate: step s searches the exported inverted file (C, assign)
    for X_1 (none when k = 0) and draws S with seed + s.  Returns the moved
    queries (FP32, as the iterate is held) and the estimate at the start of
    the last step."""
    X, C, assign = _f32(X), _f32(C), _i32(assign)
    Yo = np.array(_f32(Y), dtype=np.float32, copy=True, order="C")
    nq = Yo.shape[0]
    est = np.zeros(nq, dtype=np.float64)
    st = _load().or_mean_shift(_ptr(X), X.shape[0], X.shape[1], _ptr(C), C.shape[0],
                               _ptr(assign), _ptr(Yo), nq, float(h), int(k), int(m),
                               int(nprobe), int(seed), int(qid_offset), int(steps), _ptr(est))
    _check(st, "mean_shift")
    return Yo, est


def loo_exact(X, zid, kernel, h):
    """Exact leave-one-out log-likelihood l(h) (up to a constant) at the
    training points X[zid] and dl/dlog h; returns (l, dl, points used)."""
    X = _f32(X)
    zid = _i32(zid)
    ll = np.zeros(1)
    dll = np.zeros(1)
    used = np.zeros(1, dtype=np.int64)
    st = _load().or_loo_exact(_ptr(X), X.shape[0], X.shape[1], _ptr(zid), zid.size,
                              _kern(kernel), float(h), _ptr(ll), _ptr(dll), _ptr(used))
    _check(st, "loo_exact")
    return float(ll[0]), float(dll[0]), int(used[0])


def fit_bandwidth(X, zid, kernel, h0, nbr, m, seed, iters, lr):
    """Gradient ascent on log h of the leave-one-out likelihood with the
    DEANN estimate (X_1 rows in nbr, which should hold each training point
    itself).  Returns (h_trace[iters + 1], ll_trace[iters])."""
    X = _f32(X)
    zid = _i32(zid)
    nz = zid.size
    nbr = _i32(nbr).reshape(nz, -1)
    ht = np.zeros(iters + 1)
    lt = np.zeros(max(iters, 1))
    st = _load().or_fit_bandwidth(_ptr(X), X.shape[0], X.shape[1], _ptr(zid), nz, _kern(kernel),
                                  float(h0), _ptr(nbr), nbr.shape[1], m, seed, iters, float(lr),
                                  _ptr(ht), _ptr(lt))
    _check(st, "fit_bandwidth")
    return ht, lt[:iters]


def feistel_perm(seed: int, n: int, idx=None):
    """The keyed permutation of [0, n) used as Algorithm 2's random
    permutation (Feistel network with cycle walking); returns pi(idx) for the
    given indices (all of [0, n) by default) as int32."""
    lib = _load()
    idx = range(n) if idx is None else idx
    return np.array([lib.or_feistel_perm(seed, n, int(i)) for i in idx], dtype=np.int32)


def deannp(X, Y, kernel, h, perm, nbr, m, ell0=0):
    """DEANNP: DEANN with permuted random sampling (Algorithm 2): query q uses
    the window perm[(ell0 + q m + t) mod n], t < m, minus the members of X_1."""
    X, Y, perm = _f32(X), _f32(Y), _i32(perm)
    nq = Y.shape[0]
    if nbr is None:
        nbr = np.zeros((nq, 0), dtype=np.int32)
    nbr = _i32(nbr).reshape(nq, -1)
    k = nbr.shape[1]
    out = np.zeros(nq, dtype=np.float64)
    ell = np.zeros(1, dtype=np.int64)
    st = _load().or_deannp(_ptr(X), X.shape[0], X.shape[1], _ptr(Y), nq, _kern(kernel),
                           float(h), _ptr(perm), _ptr(nbr) if k > 0 else None, k, m,
                           int(ell0), _ptr(out), _ptr(ell))
    _check(st, "deannp")
    return out, int(ell[0])
