"""The precision, differentiation and batched workloads at their full sizes.

Each workload is generated at the size its configuration names, served
through the C-ABI in the launch configuration a user would run, and sampled
outputs are checked one by one against the FP64 oracle:

* sparse image-like data, n = 1,000,000, d = 784, 10,000 queries, Gaussian
  kernel with the mean exact KDE near 1e-4: BF16 and FP32 scans with FP32
  rescoring, k = 200, m = 2,000, 2,048 lists, nprobe = 32;
* the anisotropic mixture, n = 200,000, d = 64, 50,000 queries, Gaussian
  h = 1: forward and adjoint on every query, FP64 central differences
  (step 1e-3 h) and the oracle's analytic gradient on 256 of them, and
  mean-shift steps;
* unit-norm power-law vectors, n = 4,000,000, d = 300, 100,000 queries in 64
  batches of 16 to 8,192, exponential kernel with the mean exact KDE near
  1e-3: BF16 scan, k = 200, m = 2,000, 4,096 lists, batches served by
  CUDA-graph replays, the backward pass on every tenth batch.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads
from test_gpu_parity import assert_kde_close, assert_neighbours_match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2107_02736_gb300 as p
    p.load_library()
    return p


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bisect_h(index, Yv, target):
    """log h bisected until the mean exact KDE of Yv is within 1 % of target."""
    lo, hi = math.log(1e-3), math.log(1e3)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        index.set_bandwidth(math.exp(mid))
        mu = float(index.exact(Yv).double().mean())
        if abs(mu / target - 1.0) <= 0.01:
            break
        lo, hi = (lo, mid) if mu > target else (mid, hi)
    return math.exp(mid), mu


def _grad_check(X, Y, kernel, h, nbr, m, seed, qids, est, dY, dl):
    """GPU estimate and adjoint of rows qids against the oracle (query id =
    row), value 1e-5, gradient 1e-4 relative in the vector norm."""
    for q in qids:
        w_out, w_dY, w_dl = oracle.deann_grad(X, Y[q:q + 1], kernel, h, nbr[q:q + 1], m, seed,
                                              qid_offset=int(q))
        assert_kde_close(est[q:q + 1], w_out)
        assert np.linalg.norm(dY[q] - w_dY[0]) <= 1e-4 * np.linalg.norm(w_dY[0]) + 1e-12
        assert abs(dl[q] - w_dl[0]) <= 1e-4 * abs(w_dl[0]) + 1e-12


def test_sparse_image_full_size_precision_form(pkg):
    sp = workloads.CONFIGS[3]
    X, Y, Yv = workloads.sparse_image()
    assert X.shape == (1_000_000, 784) and Y.shape == (10_000, 784)
    k, m, L, P = sp["k"], sp["m"], sp["nlist"], sp["nprobe"]
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0, nlist=L, seed=1)
    h, mu = _bisect_h(index, _dev(Yv[:1000]), sp["target_mu"])
    C, assign = (a.numpy() for a in index.export_ivf())
    Yd = _dev(Y)
    o16, n16 = index.query(Yd, k, m, nprobe=P, seed=2, precision=1, return_neighbors=True)
    o32, n32 = index.query(Yd, k, m, nprobe=P, seed=2, precision=0, return_neighbors=True)
    o16, o32 = o16.cpu().numpy(), o32.cpu().numpy()
    n16, n32 = n16.cpu().numpy(), n32.cpu().numpy()
    assert index.margin_failures() == 0
    # the BF16 scan's certified band returns the FP32 scan's neighbours
    assert np.array_equal(np.sort(n16, 1), np.sort(n32, 1))
    assert_kde_close(o16, o32)
    qs = np.sort(np.random.default_rng(3).choice(Y.shape[0], 16, replace=False))
    _, want, want_d2 = oracle.ivf_search(X, C, assign, Y[qs], P, k)
    assert_neighbours_match(X, Y[qs], n16[qs], want, want_d2)
    for q in qs:
        v = oracle.deann(X, Y[q:q + 1], "gaussian", h, n16[q:q + 1], m, 2, qid_offset=int(q))
        assert_kde_close(o16[q:q + 1], v)
    ex = index.exact(Yd).cpu().numpy()
    assert_kde_close(ex[qs[:8]], oracle.exact(X, Y[qs[:8]], "gaussian", h))
    index.close()


def test_aniso_full_size_gradients(pkg):
    sp = workloads.CONFIGS[4]
    w = workloads.make(4)
    X, Y = w.X, w.Y
    assert X.shape == (200_000, 64) and Y.shape == (50_000, 64)
    h, k, m, L, P = w.h, sp["k"], sp["m"], sp["nlist"], sp["nprobe"]
    index = pkg.KDEIndex(_dev(X), "gaussian", h, nlist=L, seed=1)
    C, assign = (a.numpy() for a in index.export_ivf())
    Yd = _dev(Y)
    out, nbr = index.query(Yd, k, m, nprobe=P, seed=5, return_neighbors=True)
    est, dY, dl = index.grad_with_neighbors(Yd, nbr, m, seed=5)
    out, nbr = out.cpu().numpy(), nbr.cpu().numpy()
    est, dY, dl = (t.cpu().numpy().astype(np.float64) for t in (est, dY, dl))
    assert_kde_close(est, out)
    qs = np.sort(np.random.default_rng(4).choice(Y.shape[0], 256, replace=False))
    _, want, want_d2 = oracle.ivf_search(X, C, assign, Y[qs], P, k)
    assert_neighbours_match(X, Y[qs], nbr[qs], want, want_d2)
    _grad_check(X, Y, "gaussian", h, nbr, m, 5, qs, est, dY, dl)
    # FP64 central differences (step 1e-3 h) of the estimator with its sets
    # fixed: |x - (y +- st e_j)|^2 = |x - y|^2 -+ 2 st (x_j - y_j) + st^2
    n, d = X.shape
    st = 1e-3 * h
    for q in qs:
        _, S = oracle.deann(X, Y[q:q + 1], "gaussian", h, nbr[q:q + 1], m, 5,
                            qid_offset=int(q), return_samples=True)
        ids = np.unique(nbr[q][nbr[q] >= 0])
        def f(rows, sign):  # kernel sums at y + sign st e_j for every j
            diff = X[rows].astype(np.float64) - Y[q].astype(np.float64)
            D = (diff ** 2).sum(1)
            return np.exp(-(D[None, :] - sign * 2 * st * diff.T + st * st) / (2 * h * h)).sum(1)
        fp = (f(ids, 1) + (n - ids.size) / m * f(S[0], 1)) / n
        fm = (f(ids, -1) + (n - ids.size) / m * f(S[0], -1)) / n
        fd = (fp - fm) / (2 * st)
        assert np.linalg.norm(dY[q] - fd) <= 1e-3 * np.linalg.norm(fd), q
    # two mean-shift steps on every query; sampled rows against the oracle's
    Yg, _ = index.mean_shift(Yd, 2, k, m, nprobe=P, seed=7)
    Yg = Yg.cpu().numpy()
    for q in qs[:16]:
        yo, _ = oracle.mean_shift(X, C, assign, Y[q:q + 1], h, k, m, P, 7, steps=2,
                                  qid_offset=int(q))
        yo = yo.astype(np.float64)
        moved = np.linalg.norm(yo[0] - Y[q])
        assert np.linalg.norm(Yg[q] - yo[0]) <= 1e-4 * max(moved, 1e-3), q
    index.close()


def test_unit_powerlaw_full_size_batched_form(pkg):
    sp = workloads.CONFIGS[5]
    X, Y, Yv = workloads.unit_powerlaw()
    assert X.shape == (4_000_000, 300) and Y.shape == (100_000, 300)
    sizes = workloads.uneven_batches()
    assert sizes.size == 64 and sizes.sum() == Y.shape[0]
    assert sizes.min() == 16 and sizes.max() == 8192
    k, m, L, P = sp["k"], sp["m"], sp["nlist"], sp["nprobe"]
    index = pkg.KDEIndex(_dev(X), "exponential", 1.0, nlist=L, seed=1)
    h, mu = _bisect_h(index, _dev(Yv[:1000]), sp["target_mu"])
    C, assign = (a.numpy() for a in index.export_ivf())
    Yd = _dev(Y)
    whole, nbr = index.query(Yd, k, m, nprobe=P, seed=9, precision=1, return_neighbors=True)
    whole, nbr = whole.cpu().numpy(), nbr.cpu().numpy()
    assert index.margin_failures() == 0
    server = pkg.BatchServer(index, k, m, nprobe=P, seed=9, precision=1, max_batch=8192,
                             neighbors=True)
    start, checked = 0, []
    for b, nb in enumerate(sizes):
        nb = int(nb)
        Yb = Yd[start:start + nb]
        got, ids = server(Yb)
        # a replay draws the streams of the batch's global query ids
        assert np.array_equal(got.cpu().numpy(), whole[start:start + nb]), b
        assert np.array_equal(np.sort(ids.cpu().numpy(), 1), np.sort(nbr[start:start + nb], 1))
        if b % 10 == 0:  # the backward pass on every tenth batch
            est, dY, dl = server.backward(Yb, ids)
            est, dY, dl = (t.cpu().numpy().astype(np.float64) for t in (est, dY, dl))
            assert_kde_close(est, whole[start:start + nb])
            r = nb // 2
            q = start + r
            w_out, w_dY, w_dl = oracle.deann_grad(X, Y[q:q + 1], "exponential", h,
                                                  nbr[q:q + 1], m, 9, qid_offset=q)
            assert_kde_close(est[r:r + 1], w_out)
            assert np.linalg.norm(dY[r] - w_dY[0]) <= 1e-4 * np.linalg.norm(w_dY[0])
            assert abs(dl[r] - w_dl[0]) <= 1e-4 * abs(w_dl[0])
            checked.append(q)
        start += nb
    classes = {1 << max(4, int(nb - 1).bit_length()) for nb in sizes}
    assert len(checked) == 7 and set(server.graphs) == classes
    assert index.margin_failures() == 0  # the capacity's padding rows are inactive
    qs = np.sort(np.concatenate([[0, Y.shape[0] - 1],
                                 np.random.default_rng(5).choice(Y.shape[0], 14,
                                                                 replace=False)]))
    _, want, want_d2 = oracle.ivf_search(X, C, assign, Y[qs], P, k)
    assert_neighbours_match(X, Y[qs], nbr[qs], want, want_d2)
    for q in qs:
        v = oracle.deann(X, Y[q:q + 1], "exponential", h, nbr[q:q + 1], m, 9,
                         qid_offset=int(q))
        assert_kde_close(whole[q:q + 1], v)
    ex = index.exact(Yd[qs[:8]]).cpu().numpy()
    assert_kde_close(ex, oracle.exact(X, Y[qs[:8]], "exponential", h))
    index.close()
