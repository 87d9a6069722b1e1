"""DEANN kernel-density estimation on GB300 (sm_103a).

Thin Python binding of the C-ABI library ``libdeann_gb300.so``
(``include/deann_gb300.h``).  This module only marshals arguments: every step
of the estimator runs in the library's CUDA kernels.  Importing it never
falls back to a CPU path; when the library is missing it raises.

Paper: Karppa, Aumueller, Pagh, "DEANN: Speeding up Kernel-Density Estimation
using Approximate Nearest Neighbor Search" (arXiv 2107.02736).

Arrays are torch tensors (float32 / int32, C-contiguous).  CUDA tensors are
passed as device pointers and the work is enqueued on torch's current stream;
CPU tensors go through the library's host-pointer path (copy in, compute,
copy out, synchronise).
"""
from __future__ import annotations

import ctypes
import os
import numpy as np

import torch

from . import build as _build_mod

__all__ = ["KDEIndex", "DeannKDE", "GraphedQuery", "BatchServer", "KDEError", "library_path",
           "load_library", "GAUSSIAN", "EXPONENTIAL", "LAPLACIAN"]

GAUSSIAN, EXPONENTIAL, LAPLACIAN = 0, 1, 2
_KERNELS = {"gaussian": GAUSSIAN, "exponential": EXPONENTIAL, "laplacian": LAPLACIAN}
_STATUS = {0: "KDE_OK", 1: "KDE_EINVAL", 2: "KDE_ENOMEM", 3: "KDE_ECUDA", 4: "KDE_ELIMIT",
           5: "KDE_ESTATE"}

_lib = None


class KDEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("sample_mode", ctypes.c_int32),
                ("kmeans_iters", ctypes.c_int32), ("exact_path", ctypes.c_int32),
                ("query_id_offset", ctypes.c_uint64), ("stream", ctypes.c_void_p),
                ("dev_query_id_offset", ctypes.c_void_p), ("dev_active_rows", ctypes.c_void_p)]


STAGES = ["stage", "coarse", "plan", "scan", "select", "estimate", "exact", "grad"]


class _Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("timed", ctypes.c_int64 * 8),
                ("calls", ctypes.c_int64 * 8), ("launches", ctypes.c_int64 * 8)]


def library_path() -> str:
    return _build_mod.LIB


def load_library():
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(
            f"DEANN CUDA library not found at {path}; build it with "
            "`python -m paper_2107_02736_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    P, i64, i32, u64, f32 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                             ctypes.c_uint64, ctypes.c_float)
    O = ctypes.POINTER(_Opts)
    sig = {
        "kde_build": [P, i64, i32, i32, f32, i32, u64, O, ctypes.POINTER(ctypes.c_void_p)],
        "kde_set_bandwidth": [P, f32],
        "kde_set_scan_tile": [P, i32, i32],
        "kde_set_phase_window": [P, i64],
        "kde_index_info": [P, P, P, P, P, P, P],
        "kde_export_ivf": [P, P, P],
        "kde_search": [P, P, i64, i32, i32, P, P, O],
        "kde_query": [P, P, i64, i32, i32, i32, u64, P, P, O],
        "kde_query_with_neighbors": [P, P, i64, P, i32, i32, u64, P, O],
        "kde_query_rs": [P, P, i64, i32, u64, P, O],
        "kde_exact": [P, P, i64, P, O],
        "kde_sample_indices": [P, i64, P, i32, i32, u64, P, O],
        "kde_grad_with_neighbors": [P, P, i64, P, i32, i32, u64, P, P, P, P, O],
        "kde_grad": [P, P, i64, i32, i32, i32, u64, P, P, P, O],
        "kde_mean_shift": [P, P, i64, i32, i32, i32, i32, u64, P, O],
        "kde_sync": [P, O],
        "kde_stats": [P, P, O],
        "kde_reserve": [P, i64, i32, i32, i32, O],
        "kde_prepare_permuted": [P, P, O],
        "kde_fit_bandwidth": [P, P, i64, i32, i32, i32, u64, i32, f32, P, P, P, O],
        "kde_index_view": [P, ctypes.POINTER(ctypes.c_void_p)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.kde_profile_enable.argtypes = [P, i32]
    lib.kde_profile_enable.restype = ctypes.c_int
    lib.kde_profile_read.argtypes = [P, ctypes.POINTER(_Profile), i32, O]
    lib.kde_profile_read.restype = ctypes.c_int
    lib.kde_free.argtypes = [P]
    lib.kde_free.restype = None
    lib.kde_strerror.argtypes = [ctypes.c_int]
    lib.kde_strerror.restype = ctypes.c_char_p
    lib.kde_last_error.argtypes = []
    lib.kde_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        msg = _lib.kde_last_error().decode(errors="replace")
        raise KDEError(status, msg)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _f32(t, device=None):
    t = torch.as_tensor(t, dtype=torch.float32, device=device)
    return t.contiguous()


def _i32(t, device=None):
    t = torch.as_tensor(t, dtype=torch.int32, device=device)
    return t.contiguous()


class KDEIndex:
    """An index over a dataset X (n x d) for one kernel and bandwidth.

    ``nlist = 1`` makes every query scan all points (brute-force kNN as the
    ANN); ``nlist > 1`` builds an IVF-flat index with GPU k-means.
    """

    def __init__(self, X, kernel="gaussian", h=1.0, nlist=1, seed=0, kmeans_iters=20,
                 device=None):
        lib = load_library()
        X = _f32(X, device=device)
        if X.dim() != 2:
            raise ValueError("X must be n x d")
        self._device = X.device if X.is_cuda else torch.device("cuda", torch.cuda.current_device())
        kern = _KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        opts = self._opts(kmeans_iters=kmeans_iters)
        handle = ctypes.c_void_p()
        with torch.cuda.device(self._device):
            _check(lib.kde_build(_ptr(X), X.shape[0], X.shape[1], kern, float(h), int(nlist),
                                 int(seed) & (2**64 - 1), ctypes.byref(opts),
                                 ctypes.byref(handle)))
        self._h = handle
        self.n, self.d = X.shape
        self.kernel = kern
        self.nlist = int(nlist)

    # -- plumbing ----------------------------------------------------------
    def _opts(self, precision=0, sample_mode=0, qid_offset=0, kmeans_iters=0, host=False,
              exact_path=0):
        o = _Opts()
        o.precision = int(precision)
        o.sample_mode = int(sample_mode)
        o.kmeans_iters = int(kmeans_iters)
        o.exact_path = int(exact_path)
        o.query_id_offset = int(qid_offset)
        o.stream = None if host else torch.cuda.current_stream().cuda_stream
        return o

    def _prep(self, Y):
        Y = _f32(Y)
        if Y.dim() != 2 or Y.shape[1] != self.d:
            raise ValueError(f"Y must be nq x {self.d}")
        return Y

    def view(self) -> "KDEIndex":
        """A second handle on this index (kde_index_view): the same data, its
        own scratch, so that it can serve work on another stream at the same
        time.  This index must outlive the view."""
        handle = ctypes.c_void_p()
        with torch.cuda.device(self._device):
            _check(_lib.kde_index_view(self._h, ctypes.byref(handle)))
        v = KDEIndex.__new__(KDEIndex)
        v._h, v._device, v.n, v.d = handle, self._device, self.n, self.d
        v.kernel, v.nlist, v._base = self.kernel, self.nlist, self
        return v

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.kde_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def device(self):
        return self._device

    @property
    def h(self) -> float:
        h = ctypes.c_float()
        _check(_lib.kde_index_info(self._h, None, None, None, None, ctypes.byref(h), None))
        return h.value

    @property
    def max_list(self) -> int:
        v = ctypes.c_int64()
        _check(_lib.kde_index_info(self._h, None, None, None, None, None, ctypes.byref(v)))
        return v.value

    def set_bandwidth(self, h: float):
        _check(_lib.kde_set_bandwidth(self._h, float(h)))

    def set_scan_tile(self, precision: int, tile: int):
        """kde_set_scan_tile: the most queries a tensor-core list-scan tile
        takes for this precision (1 or 2); 0 = automatic."""
        _check(_lib.kde_set_scan_tile(self._h, int(precision), int(tile)))

    def set_phase_window(self, nbytes: int):
        """kde_set_phase_window: the bytes of X one phase of the query
        estimator reads (0 = per-query gathers always)."""
        _check(_lib.kde_set_phase_window(self._h, int(nbytes)))

    def tune_scan_tile(self, Y, k, m, nprobe, precision, tiles=(0, 96, 64, 48, 32), reps=3,
                       seed=0):
        """Times kde_query on the sample queries Y at each scan tile (CUDA
        events on the current stream, one untimed call first) and keeps the
        fastest for `precision` (kde_set_scan_tile).  Returns ({tile: ms per
        call}, the tile kept); 0 stands for the automatic tile."""
        times = {}
        for t in tiles:
            self.set_scan_tile(precision, t)
            self.query(Y, k, m, nprobe=nprobe, seed=seed, precision=precision)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                self.query(Y, k, m, nprobe=nprobe, seed=seed, precision=precision)
            e1.record()
            e1.synchronize()
            times[int(t)] = e0.elapsed_time(e1) / reps
        best = min(times, key=times.get)
        self.set_scan_tile(precision, best)
        return times, best

    def export_ivf(self):
        """(centroids nlist x d float32, assign n int32) as CPU tensors."""
        C = torch.empty((self.nlist, self.d), dtype=torch.float32)
        a = torch.empty(self.n, dtype=torch.int32)
        with torch.cuda.device(self._device):
            _check(_lib.kde_export_ivf(self._h, _ptr(C), _ptr(a)))
        return C, a

    def prepare_permuted(self, return_perm=False):
        """Algorithm 2's preprocessing (random permutation pi and the
        permuted dataset copy) for sample_mode=2; returns pi as an int32 CUDA
        tensor when asked."""
        perm = (torch.empty(self.n, dtype=torch.int32, device=self._device)
                if return_perm else None)
        with torch.cuda.device(self._device):
            _check(_lib.kde_prepare_permuted(self._h, _ptr(perm), ctypes.byref(self._opts())))
        return perm

    def fit_bandwidth(self, zid, k, m, nprobe=1, seed=0, iters=20, lr=0.5, precision=0,
                      sample_mode=0):
        """Gradient ascent on log h of the leave-one-out likelihood at the
        training points X[zid] with the DEANN estimate and its adjoint.
        Returns (h_trace, ll_trace, X_1 rows) as CPU arrays; the index keeps the
        final h."""
        zid = _i32(zid).cpu().contiguous()
        nz = zid.numel()
        ht = np.zeros(iters + 1, dtype=np.float32)
        lt = np.zeros(max(iters, 1), dtype=np.float64)
        nb = torch.empty((nz, k + 1), dtype=torch.int32)
        with torch.cuda.device(self._device):
            _check(_lib.kde_fit_bandwidth(
                self._h, _ptr(zid), nz, int(k), int(m), int(nprobe), int(seed) & (2**64 - 1),
                int(iters), float(lr), ht.ctypes.data_as(ctypes.c_void_p),
                lt.ctypes.data_as(ctypes.c_void_p), _ptr(nb),
                ctypes.byref(self._opts(precision, sample_mode, host=True))))
        return ht, lt[:iters], nb.numpy()

    def sync(self):
        with torch.cuda.device(self._device):
            _check(_lib.kde_sync(self._h, ctypes.byref(self._opts())))

    def margin_failures(self) -> int:
        v = ctypes.c_int64()
        with torch.cuda.device(self._device):
            _check(_lib.kde_stats(self._h, ctypes.byref(v), ctypes.byref(self._opts())))
        return v.value

    def profile(self, on: bool = True):
        _check(_lib.kde_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, reset: bool = True) -> dict:
        """{stage: {ms, timed, calls, launches}} since the last reset."""
        p = _Profile()
        with torch.cuda.device(self._device):
            _check(_lib.kde_profile_read(self._h, ctypes.byref(p), 1 if reset else 0,
                                         ctypes.byref(self._opts())))
        return {name: dict(ms=p.ms[i], timed=p.timed[i], calls=p.calls[i],
                           launches=p.launches[i]) for i, name in enumerate(STAGES)}

    def reserve(self, nq, k=0, m=0, nprobe=1, precision=0):
        with torch.cuda.device(self._device):
            _check(_lib.kde_reserve(self._h, int(nq), int(k), int(m), int(nprobe),
                                    ctypes.byref(self._opts(precision))))

    # -- the path ------------------------------------------------------------
    def search(self, Y, k, nprobe=1, precision=0):
        Y = self._prep(Y)
        nq = Y.shape[0]
        nbr = torch.empty((nq, k), dtype=torch.int32, device=Y.device)
        d2 = torch.empty((nq, k), dtype=torch.float32, device=Y.device)
        with torch.cuda.device(self._device):
            _check(_lib.kde_search(self._h, _ptr(Y), nq, int(k), int(nprobe), _ptr(nbr),
                                   _ptr(d2), ctypes.byref(self._opts(precision,
                                                                     host=not Y.is_cuda))))
        return nbr, d2

    def query(self, Y, k, m, nprobe=1, seed=0, precision=0, sample_mode=0, qid_offset=0,
              return_neighbors=False, dev_qid=None, dev_active=None):
        """DEANN estimates (Algorithm 1).  dev_qid: optional int64 CUDA tensor
        of one element added to qid_offset on the device (graph replays).
        dev_active: optional int64 CUDA tensor of one element A; only rows
        below A are served (their neighbours -1 and estimates unspecified
        past it)."""
        Y = self._prep(Y)
        nq = Y.shape[0]
        out = torch.empty(nq, dtype=torch.float32, device=Y.device)
        nbr = (torch.empty((nq, k), dtype=torch.int32, device=Y.device)
               if return_neighbors and k > 0 else None)
        o = self._opts(precision, sample_mode, qid_offset, host=not Y.is_cuda)
        if dev_qid is not None:
            o.dev_query_id_offset = dev_qid.data_ptr()
        if dev_active is not None:
            o.dev_active_rows = dev_active.data_ptr()
        with torch.cuda.device(self._device):
            _check(_lib.kde_query(self._h, _ptr(Y), nq, int(k), int(m), int(nprobe),
                                  int(seed) & (2**64 - 1), _ptr(out), _ptr(nbr),
                                  ctypes.byref(o)))
        return (out, nbr) if return_neighbors else out

    def query_batches(self, Ys, k, m, nprobe=1, seed=0, precision=0):
        """Uneven batches served by one call over their concatenation (one
        launch per stage for all of them); batch b keeps the sample streams it
        would get alone with qid_offset = its start row.  Returns a list."""
        sizes = [int(y.shape[0]) for y in Ys]
        out = self.query(torch.cat([self._prep(y) for y in Ys]), k, m, nprobe=nprobe,
                         seed=seed, precision=precision)
        return list(torch.split(out, sizes))

    def query_with_neighbors(self, Y, nbr, m, seed=0, sample_mode=0, qid_offset=0):
        Y = self._prep(Y)
        nq = Y.shape[0]
        nbr = _i32(nbr, device=Y.device).reshape(nq, -1)
        k = nbr.shape[1]
        out = torch.empty(nq, dtype=torch.float32, device=Y.device)
        with torch.cuda.device(self._device):
            _check(_lib.kde_query_with_neighbors(
                self._h, _ptr(Y), nq, _ptr(nbr) if k > 0 else None, k, int(m),
                int(seed) & (2**64 - 1), _ptr(out),
                ctypes.byref(self._opts(0, sample_mode, qid_offset, host=not Y.is_cuda))))
        return out

    def query_rs(self, Y, m, seed=0, qid_offset=0, sample_mode=0):
        """Random sampling; sample_mode=2 gives RSP (Algorithm 2)."""
        Y = self._prep(Y)
        nq = Y.shape[0]
        out = torch.empty(nq, dtype=torch.float32, device=Y.device)
        with torch.cuda.device(self._device):
            _check(_lib.kde_query_rs(self._h, _ptr(Y), nq, int(m), int(seed) & (2**64 - 1),
                                     _ptr(out), ctypes.byref(self._opts(
                                         0, sample_mode, qid_offset, host=not Y.is_cuda))))
        return out

    def exact(self, Y, path="auto"):
        """Exact KDE.  path: "auto" (tensor cores when their accuracy guard
        allows), "cuda" (FP32 difference form on CUDA cores) or "tensor"."""
        Y = self._prep(Y)
        nq = Y.shape[0]
        out = torch.empty(nq, dtype=torch.float32, device=Y.device)
        code = {"auto": 0, "cuda": 1, "tensor": 2}[path]
        with torch.cuda.device(self._device):
            _check(_lib.kde_exact(self._h, _ptr(Y), nq, _ptr(out), ctypes.byref(
                self._opts(host=not Y.is_cuda, exact_path=code))))
        return out

    def sample_indices(self, nbr, m, seed=0, nq=None, sample_mode=0, qid_offset=0,
                       device=None):
        if nbr is None:
            if nq is None:
                raise ValueError("nq is required without nbr")
            dev = device if device is not None else self._device
            k = 0
            nbr_t = None
        else:
            nbr_t = _i32(nbr, device=device)
            nq = nbr_t.shape[0]
            nbr_t = nbr_t.reshape(nq, -1)
            k = nbr_t.shape[1]
            dev = nbr_t.device
        S = torch.empty((nq, m), dtype=torch.int32, device=dev)
        with torch.cuda.device(self._device):
            _check(_lib.kde_sample_indices(
                self._h, int(nq), _ptr(nbr_t) if k > 0 else None, k, int(m),
                int(seed) & (2**64 - 1), _ptr(S),
                ctypes.byref(self._opts(0, sample_mode, qid_offset,
                                        host=S.device.type == "cpu"))))
        return S

    def mean_shift(self, Y, steps, k, m, nprobe=1, seed=0, precision=0, qid_offset=0):
        """Runs `steps` Gaussian mean-shift updates on a copy of Y; returns
        (moved queries, estimate at the start of the last step)."""
        Y = self._prep(Y).clone()
        nq = Y.shape[0]
        est = torch.empty(nq, dtype=torch.float32, device=Y.device)
        with torch.cuda.device(self._device):
            _check(_lib.kde_mean_shift(self._h, _ptr(Y), nq, int(steps), int(k), int(m),
                                       int(nprobe), int(seed) & (2**64 - 1), _ptr(est),
                                       ctypes.byref(self._opts(precision, 0, qid_offset,
                                                               host=not Y.is_cuda))))
        return Y, est

    def grad(self, Y, k, m, nprobe=1, seed=0, gout=None, precision=0, sample_mode=0,
             qid_offset=0):
        """(dY, dlogh) of the DEANN estimate (kde_grad: the search and the
        sample of kde_query with the same arguments, held fixed); dlogh is the
        device-side sum over the queries (a 0-d tensor)."""
        Y = self._prep(Y)
        nq = Y.shape[0]
        g = None if gout is None else _f32(gout, device=Y.device)
        dY = torch.empty((nq, self.d), dtype=torch.float32, device=Y.device)
        dl = torch.empty((), dtype=torch.float32, device=Y.device)
        with torch.cuda.device(self._device):
            _check(_lib.kde_grad(self._h, _ptr(Y), nq, int(k), int(m), int(nprobe),
                                 int(seed) & (2**64 - 1), _ptr(g), _ptr(dY), _ptr(dl),
                                 ctypes.byref(self._opts(precision, sample_mode, qid_offset,
                                                         host=not Y.is_cuda))))
        return dY, dl

    def grad_with_neighbors(self, Y, nbr, m, seed=0, gout=None, sample_mode=0, qid_offset=0):
        """(out, dY, dlogh_per_query) of the estimate with X_1 and S fixed."""
        Y = self._prep(Y)
        nq = Y.shape[0]
        if nbr is None:
            nbr_t, k = None, 0
        else:
            nbr_t = _i32(nbr, device=Y.device).reshape(nq, -1)
            k = nbr_t.shape[1]
        g = None if gout is None else _f32(gout, device=Y.device)
        out = torch.empty(nq, dtype=torch.float32, device=Y.device)
        dY = torch.empty((nq, self.d), dtype=torch.float32, device=Y.device)
        dl = torch.empty(nq, dtype=torch.float32, device=Y.device)
        with torch.cuda.device(self._device):
            _check(_lib.kde_grad_with_neighbors(
                self._h, _ptr(Y), nq, _ptr(nbr_t) if k > 0 else None, k, int(m),
                int(seed) & (2**64 - 1), _ptr(g), _ptr(out), _ptr(dY), _ptr(dl),
                ctypes.byref(self._opts(0, sample_mode, qid_offset, host=not Y.is_cuda))))
        return out, dY, dl


class GraphedQuery:
    """kde_query of a fixed capacity captured once in a CUDA graph.

    The index's scratch is reserved before the capture, so the captured call
    allocates nothing.  Each replay serves one batch of at most `capacity`
    queries: the batch is copied into the static input, its size is written
    to a device scalar that marks the rows past it inactive (they get no
    probes, neighbours or samples), and the batch's first query id to another
    that the estimator reads, so every replay draws the sample streams the
    direct call with that qid_offset would draw (with sample_mode=2, the permuted windows of Algorithm 2 that
    follow on from the previous batch's).  With neighbors=True the replay
    also returns the neighbour ids (X_1) that a backward pass needs.
    """

    def __init__(self, index: KDEIndex, capacity, k, m, nprobe=1, seed=0, precision=0,
                 sample_mode=0, neighbors=False):
        self.index, self.capacity = index, int(capacity)
        self.neighbors = bool(neighbors) and k > 0
        dev = index.device
        self.Y = torch.zeros((self.capacity, index.d), dtype=torch.float32, device=dev)
        self.qid = torch.zeros(1, dtype=torch.int64, device=dev)
        # no active row until a batch arrives: the warm-up call below only loads
        # the kernels (its rows would be zero vectors)
        self.active = torch.zeros(1, dtype=torch.int64, device=dev)
        index.reserve(self.capacity, k, m, nprobe, precision)
        args = dict(k=k, m=m, nprobe=nprobe, seed=seed, precision=precision,
                    sample_mode=sample_mode, dev_qid=self.qid, dev_active=self.active,
                    return_neighbors=self.neighbors)
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):  # first launches (module loading) outside the capture
            index.query(self.Y, **args)
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        self.nbr = None
        with torch.cuda.graph(self.graph, capture_error_mode="relaxed"):
            res = index.query(self.Y, **args)
        self.out, self.nbr = res if self.neighbors else (res, None)

    def __call__(self, Yb, qid_offset=0):
        nb = int(Yb.shape[0])
        if nb > self.capacity:
            raise ValueError(f"batch of {nb} exceeds the captured capacity {self.capacity}")
        self.Y[:nb].copy_(Yb, non_blocking=True)
        self.qid.fill_(int(qid_offset))
        self.active.fill_(nb)
        self.graph.replay()
        return (self.out[:nb], self.nbr[:nb]) if self.neighbors else self.out[:nb]


class BatchServer:
    """Serves uneven batches with CUDA graphs captured per power-of-two
    capacity class (16 ... max_batch); the query ids run on across batches.

    With streams > 1 consecutive batches go round-robin to that many CUDA
    streams, each with its own view of the index (its own scratch) and its
    own graphs, so that small batches, which leave most of the GPU idle, run
    side by side.  A batch's results stay valid until its stream serves again
    (`streams` calls later); copy them out before then.  Work on the caller's
    stream before a call is ordered before the batch, and the caller's stream
    waits for the batch's stream when it uses the result (sync()).
    With neighbors=True each call returns (estimates, neighbour ids) and
    backward() runs the adjoint of the last batch served (its sets fixed) on
    that batch's stream.  With tune_sample (queries of the workload) the
    tensor-core scan's tile is measured and kept before any graph is
    captured (KDEIndex.tune_scan_tile; tile_times holds the timings)."""

    def __init__(self, index: KDEIndex, k, m, nprobe=1, seed=0, precision=0, max_batch=8192,
                 sample_mode=0, neighbors=False, streams=1, tune_sample=None):
        self.index, self.args = index, dict(k=k, m=m, nprobe=nprobe, seed=seed,
                                            precision=precision, sample_mode=sample_mode,
                                            neighbors=neighbors)
        self.max_batch = int(max_batch)
        # the scan tile is fixed inside a captured graph: tune it (on sample
        # queries of the workload) before the lanes take their views
        self.tile_times = None
        if tune_sample is not None and precision in (1, 2):
            self.tile_times, _ = index.tune_scan_tile(tune_sample, k, m, nprobe, precision)
        cap = 16
        while cap < self.max_batch:
            cap *= 2
        dev = index.device
        self.lanes = []
        for i in range(max(1, int(streams))):
            ix = index if i == 0 else index.view()
            # the scratch for the largest capacity class up front, so that every
            # graph of the lane is captured on the same buffer
            ix.reserve(cap, k, m, nprobe, precision)
            self.lanes.append({"index": ix, "graphs": {},
                               "stream": (torch.cuda.current_stream(dev) if i == 0 and streams <= 1
                                          else torch.cuda.Stream(device=dev))})
        self.turn = 0
        self.next_qid = 0
        self.last_qid = 0
        self.last_lane = self.lanes[0]

    @property
    def graphs(self):
        """Capacity classes captured so far (over all lanes)."""
        caps = {}
        for lane in self.lanes:
            caps.update(lane["graphs"])
        return caps

    def _graph(self, lane, nb):
        cap = 16
        while cap < nb:
            cap *= 2
        if cap not in lane["graphs"]:
            with torch.cuda.stream(lane["stream"]):
                lane["graphs"][cap] = GraphedQuery(lane["index"], cap, **self.args)
        return lane["graphs"][cap]

    def __call__(self, Yb, out=None):
        """Serves one batch; returns the graph's result views.  With `out`
        given (a float32 tensor of the batch's length), the estimates are
        copied there on the batch's stream, so they survive the lane's next
        batch."""
        nb = int(Yb.shape[0])
        if nb > self.max_batch:
            raise ValueError(f"batch of {nb} exceeds max_batch {self.max_batch}")
        lane = self.lanes[self.turn % len(self.lanes)]
        self.turn += 1
        caller = torch.cuda.current_stream(self.index.device)
        lane["stream"].wait_stream(caller)
        g = self._graph(lane, nb)
        with torch.cuda.stream(lane["stream"]):
            res = g(Yb, self.next_qid)
            if out is not None:
                out.copy_(res[0] if isinstance(res, tuple) else res)
        self.last_qid, self.last_lane = self.next_qid, lane
        self.next_qid += nb
        return res

    @property
    def last_stream(self):
        """The stream of the last batch served: its results (and those of
        backward()) are written there."""
        return self.last_lane["stream"]

    def sync(self):
        """Makes the caller's stream wait for every lane's work."""
        caller = torch.cuda.current_stream(self.index.device)
        for lane in self.lanes:
            caller.wait_stream(lane["stream"])

    def backward(self, Yb, nbr, gout=None):
        """(estimate, dY, dlogh per query) of the last batch served, from its
        neighbour ids and its regenerated sample streams.  They are computed
        on the batch's stream (last_stream): read them there, or after
        sync()."""
        a, lane = self.args, self.last_lane
        with torch.cuda.stream(lane["stream"]):
            return lane["index"].grad_with_neighbors(Yb, nbr, a["m"], seed=a["seed"], gout=gout,
                                                     sample_mode=a["sample_mode"],
                                                     qid_offset=self.last_qid)


class DeannKDE(torch.autograd.Function):
    """out = DEANN estimate of KDE(Y) with bandwidth exp(log_h).

    Forward runs kde_query (IVF search and estimator).  Backward runs
    kde_grad with the same arguments: the library repeats the deterministic
    search, regenerates the sample from the same Philox stream, recomputes the
    kernel values and returns d/dY and the device-reduced d/dlog h of the
    estimate with the neighbour set and the sample held fixed.  Nothing but
    the queries and log h is saved.
    """

    @staticmethod
    def forward(ctx, Y, log_h, index: KDEIndex, k: int, m: int, nprobe: int, seed: int,
                precision: int = 0):
        h = float(torch.exp(log_h.detach()).item())
        index.set_bandwidth(h)
        out = index.query(Y.detach(), k, m, nprobe=nprobe, seed=seed, precision=precision)
        ctx.index, ctx.args, ctx.h = index, (k, m, nprobe, seed, precision), h
        ctx.save_for_backward(Y.detach())
        return out

    @staticmethod
    def backward(ctx, gout):
        (Y,) = ctx.saved_tensors
        k, m, nprobe, seed, precision = ctx.args
        ctx.index.set_bandwidth(ctx.h)
        dY, dl = ctx.index.grad(Y, k, m, nprobe=nprobe, seed=seed, gout=gout.contiguous(),
                                precision=precision)
        return dY, dl.to(gout.dtype), None, None, None, None, None, None
