"""The five synthetic workloads through the C-ABI, checked against the oracle.

The low-dimensional workload runs at full size on every query.  The
1M-point d=128 workload runs at full size in the launch configuration the
benchmark times (k = 1280, m = 4000, nprobe = 4, 10k queries, every scan
precision; DEANNP with m = 8000), and at the earlier k = 1536, nprobe = 8,
and sampled queries are checked one by one.
The others run here at reduced n with their own dimension, kernel and
parameters (their full sizes are in test_gpu_full_size.py).
"""
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


def test_low_dim_brute_force_full(pkg):
    """n = 10,000, d = 16, 1,000 queries, Gaussian h = 2, brute-force kNN,
    k = 50, m = 500, seed 0; exact KDE for every query."""
    w = workloads.make(1)
    assert w.X.shape == (10_000, 16) and w.Y.shape == (1_000, 16)
    index = pkg.KDEIndex(_dev(w.X), "gaussian", 2.0, nlist=1)
    out, nbr = index.query(_dev(w.Y), 50, 500, nprobe=1, seed=0, return_neighbors=True)
    nbr = nbr.cpu().numpy()
    want_nbr, want_d2 = oracle.knn(w.X, w.Y, 50)
    assert_neighbours_match(w.X, w.Y, nbr, want_nbr, want_d2)
    assert_kde_close(out.cpu().numpy(), oracle.deann(w.X, w.Y, "gaussian", 2.0, nbr, 500, 0))
    ex = oracle.exact(w.X, w.Y, "gaussian", 2.0)
    assert_kde_close(index.exact(_dev(w.Y)).cpu().numpy(), ex)
    assert_kde_close(index.query_rs(_dev(w.Y), 500, seed=0).cpu().numpy(),
                     oracle.rs(w.X, w.Y, "gaussian", 2.0, 500, 0))


@pytest.fixture(scope="module")
def embed(pkg):
    X, Y, _ = workloads.mixture_embed()
    index = pkg.KDEIndex(_dev(X), "gaussian", 12.85, nlist=1024, seed=1)
    C, assign = index.export_ivf()
    return X, Y, index, C.numpy(), assign.numpy()


@pytest.mark.parametrize("sched", [(1280, 4000, 4), (1536, 4000, 8)])
@pytest.mark.parametrize("precision", [1, 0, 2])
def test_embed_full_size_sampled(embed, precision, sched):
    X, Y, index, C, assign = embed
    (k, m, P), h = sched, 12.85
    out, nbr = index.query(_dev(Y), k, m, nprobe=P, seed=3, precision=precision,
                           return_neighbors=True)
    out, nbr = out.cpu().numpy(), nbr.cpu().numpy()
    rng = np.random.default_rng(precision)
    qs = np.sort(rng.choice(Y.shape[0], 24, replace=False))
    _, want, want_d2 = oracle.ivf_search(X, C, assign, Y[qs], P, k)
    assert_neighbours_match(X, Y[qs], nbr[qs], want, want_d2)
    # the estimator's stream of query row q is qid = q
    for q in qs:
        v = oracle.deann(X, Y[q:q + 1], "gaussian", h, nbr[q:q + 1], m, 3, qid_offset=int(q))
        assert_kde_close(out[q:q + 1], v)
    assert index.margin_failures() == 0


def test_embed_full_size_deannp_sampled(embed):
    """DEANNP (Algorithm 2) at full size: the 1M-entry permutation is
    bit-exact and sampled estimates match the oracle's windows."""
    X, Y, index, _, _ = embed
    k, m, P, h = 1280, 8000, 4, 12.85
    perm = index.prepare_permuted(return_perm=True).cpu().numpy()
    want_perm = oracle.feistel_perm(1, X.shape[0])
    assert np.array_equal(perm, want_perm)
    out, nbr = index.query(_dev(Y), k, m, nprobe=P, precision=1, sample_mode=2,
                           return_neighbors=True)
    out, nbr = out.cpu().numpy(), nbr.cpu().numpy()
    n = X.shape[0]
    for q in np.arange(0, Y.shape[0], 417)[:24]:
        v, _ = oracle.deannp(X, Y[q:q + 1], "gaussian", h, want_perm, nbr[q:q + 1], m,
                             ell0=(int(q) * m) % n)
        assert_kde_close(out[q:q + 1], v)


def test_embed_full_size_exact_sampled(embed):
    X, Y, index, _, _ = embed
    ex = index.exact(_dev(Y)).cpu().numpy()
    qs = np.arange(0, Y.shape[0], 625)  # 16 queries
    assert_kde_close(ex[qs], oracle.exact(X, Y[qs], "gaussian", 12.85))


def test_sparse_image_reduced(pkg):
    """d = 784 sparse [0, 1] data: BF16 and FP32 scans give the same
    neighbours; estimates match the oracle."""
    X, Y, _ = workloads.sparse_image(n=30_000, nq=200)
    h = 1.3
    index = pkg.KDEIndex(_dev(X), "gaussian", h, nlist=64, seed=2)
    C, assign = index.export_ivf()
    o16, n16 = index.query(_dev(Y), 200, 2000, nprobe=8, seed=1, precision=1,
                           return_neighbors=True)
    o32, n32 = index.query(_dev(Y), 200, 2000, nprobe=8, seed=1, precision=0,
                           return_neighbors=True)
    n16, n32 = n16.cpu().numpy(), n32.cpu().numpy()
    assert np.array_equal(np.sort(n16, 1), np.sort(n32, 1))
    _, want, want_d2 = oracle.ivf_search(X, C.numpy(), assign.numpy(), Y, 8, 200)
    assert_neighbours_match(X, Y, n16, want, want_d2)
    assert_kde_close(o16.cpu().numpy(), oracle.deann(X, Y, "gaussian", h, n16, 2000, 1))
    assert index.margin_failures() == 0


def test_aniso_gradient_and_mean_shift(pkg):
    """d = 64 anisotropic mixture, Gaussian h = 1: forward and adjoint against
    the oracle's analytic gradient and FP64 central differences (step 1e-3 h),
    and mean-shift steps against the oracle's."""
    X, Y, _ = workloads.mixture_aniso(n=20_000, nq=64)
    h, k, m, P = 1.0, 100, 1000, 8
    index = pkg.KDEIndex(_dev(X), "gaussian", h, nlist=64, seed=3)
    C, assign = index.export_ivf()
    C, assign = C.numpy(), assign.numpy()
    out, nbr = index.query(_dev(Y), k, m, nprobe=P, seed=5, return_neighbors=True)
    nbr = nbr.cpu().numpy()
    est, dY, dl = index.grad_with_neighbors(_dev(Y), _dev(nbr), m, seed=5)
    w_out, w_dY, w_dl = oracle.deann_grad(X, Y, "gaussian", h, nbr, m, 5)
    assert_kde_close(est.cpu().numpy(), w_out)
    assert_kde_close(out.cpu().numpy(), w_out)
    dY = dY.cpu().numpy().astype(np.float64)
    for q in range(Y.shape[0]):
        assert np.linalg.norm(dY[q] - w_dY[q]) <= 1e-4 * np.linalg.norm(w_dY[q]) + 1e-12
    assert np.allclose(dl.cpu().numpy(), w_dl, rtol=1e-4, atol=1e-12)
    # central differences of the oracle estimator with the same sets, 8 queries
    _, S = oracle.deann(X, Y, "gaussian", h, nbr, m, 5, return_samples=True)
    step = 1e-3 * h
    for q in range(8):
        ids = np.unique(nbr[q][nbr[q] >= 0])
        def f(y):
            k1 = np.exp(-((X[ids].astype(np.float64) - y) ** 2).sum(1) / (2 * h * h)).sum()
            k2 = np.exp(-((X[S[q]].astype(np.float64) - y) ** 2).sum(1) / (2 * h * h)).sum()
            n = X.shape[0]
            return (k1 + (n - ids.size) / m * k2) / n
        y0 = Y[q].astype(np.float64)
        fd = np.array([(f(y0 + step * e) - f(y0 - step * e)) / (2 * step)
                       for e in np.eye(X.shape[1])])
        assert np.linalg.norm(dY[q] - fd) <= 1e-3 * np.linalg.norm(fd)
    # two mean-shift steps against the oracle's driver (search + adjoint, seed + step)
    Yg, eg = index.mean_shift(_dev(Y[:16]), 2, k, m, nprobe=P, seed=7)
    Yo, eo = oracle.mean_shift(X, C, assign, Y[:16], h, k, m, P, 7, steps=2)
    assert_kde_close(eg.cpu().numpy(), eo)
    Yo = Yo.astype(np.float64)
    moved = np.linalg.norm(Yo - Y[:16], axis=1)
    err = np.linalg.norm(Yg.cpu().numpy() - Yo, axis=1)
    assert np.all(err <= 1e-4 * np.maximum(moved, 1e-3)), (err, moved)


def test_unit_powerlaw_uneven_batches(pkg):
    """d = 300 unit vectors, exponential kernel, BF16 scan: uneven batches
    served one call each (query-id offsets) or all in one call give identical
    results, and spot checks match the oracle."""
    X, Y, _ = workloads.unit_powerlaw(n=40_000, nq=2_000, n_centres=200)
    h = 0.2
    sizes = workloads.uneven_batches(total=2_000, nbatch=8, lo=16, hi=800, seed=1)
    index = pkg.KDEIndex(_dev(X), "exponential", h, nlist=128, seed=4)
    Yd = _dev(Y)
    whole, nbr = index.query(Yd, 200, 2000, nprobe=8, seed=9, precision=1,
                             return_neighbors=True)
    whole, nbr = whole.cpu().numpy(), nbr.cpu().numpy()
    start, parts = 0, []
    for b in sizes:
        parts.append(index.query(Yd[start:start + b], 200, 2000, nprobe=8, seed=9, precision=1,
                                 qid_offset=start).cpu().numpy())
        start += int(b)
    assert np.array_equal(np.concatenate(parts), whole)
    C, assign = index.export_ivf()
    qs = np.array([0, 17, 555, 1999])
    _, want, want_d2 = oracle.ivf_search(X, C.numpy(), assign.numpy(), Y[qs], 8, 200)
    assert_neighbours_match(X, Y[qs], nbr[qs], want, want_d2)
    for q in qs:
        v = oracle.deann(X, Y[q:q + 1], "exponential", h, nbr[q:q + 1], 2000, 9,
                         qid_offset=int(q))
        assert_kde_close(whole[q:q + 1], v)


def test_graph_replays_serve_uneven_batches(pkg):
    """Batches of uneven size served by CUDA-graph replays (one graph per
    power-of-two capacity) give exactly the direct calls' results, each batch
    on its own sample streams (query ids continue across batches); one query
    of every batch, with the neighbour set the replay returned, matches the
    oracle's estimate from the same stream."""
    X, Y, _ = workloads.unit_powerlaw(n=30_000, nq=1_500, n_centres=100)
    h = 0.2
    index = pkg.KDEIndex(_dev(X), "exponential", h, nlist=64, seed=5)
    C, assign = index.export_ivf()
    sizes = workloads.uneven_batches(total=1_500, nbatch=9, lo=16, hi=600, seed=3)
    server = pkg.BatchServer(index, 100, 1000, nprobe=4, seed=11, precision=1, max_batch=1024,
                             neighbors=True)
    Yd = _dev(Y)
    start = 0
    for b in sizes:
        b = int(b)
        got, ids = server(Yd[start:start + b])
        got, ids = got.clone(), ids.clone()
        want = index.query(Yd[start:start + b], 100, 1000, nprobe=4, seed=11, precision=1,
                           qid_offset=start)
        assert torch.equal(got, want), b
        r = b // 3
        q = start + r
        nb = ids[r:r + 1].cpu().numpy()
        _, w_nb, w_d2 = oracle.ivf_search(X, C.numpy(), assign.numpy(), Y[q:q + 1], 4, 100)
        assert_neighbours_match(X, Y[q:q + 1], nb, w_nb, w_d2)
        assert_kde_close(got[r:r + 1].cpu().numpy(),
                         oracle.deann(X, Y[q:q + 1], "exponential", h, nb, 1000, 11,
                                      qid_offset=q))
        start += b
    assert len(server.graphs) >= 3


def test_batch_server_tunes_the_scan_tile_before_capture(pkg):
    """BatchServer(tune_sample=...) times the scan tiles on the sample before
    any graph is captured; the views the lanes take start with the tile kept,
    and the served batches equal direct calls."""
    X, Y, _ = workloads.unit_powerlaw(n=20_000, nq=900, n_centres=80)
    index = pkg.KDEIndex(_dev(X), "exponential", 0.2, nlist=32, seed=5)
    Yd = _dev(Y)
    server = pkg.BatchServer(index, 80, 600, nprobe=3, seed=2, precision=2, max_batch=512,
                             streams=2, tune_sample=Yd[:256])
    assert server.tile_times and set(server.tile_times) >= {0, 32}
    res = torch.empty(Y.shape[0], dtype=torch.float32, device="cuda")
    start = 0
    for nb in (17, 300, 64, 419):
        server(Yd[start:start + nb], out=res[start:start + nb])
        start += nb
    server.sync()
    torch.cuda.synchronize()
    want = index.query(Yd[:start], 80, 600, nprobe=3, seed=2, precision=2)
    assert torch.equal(res[:start], want)



def test_graph_replays_with_the_phased_estimator(pkg):
    """Graphs of every capacity take the phased estimator (forced here by a
    4 MiB window on a 36 MB dataset: fifteen windows of 2,048 rows), rows
    past the batch inactive; each served batch equals the direct call of its
    size, and the whole set in one call (the windows do not depend on the
    batch size)."""
    X, Y, _ = workloads.unit_powerlaw(n=30_000, nq=1_500, n_centres=100)
    index = pkg.KDEIndex(_dev(X), "exponential", 0.2, nlist=64, seed=5)
    index.set_phase_window(4 << 20)
    server = pkg.BatchServer(index, 100, 1000, nprobe=4, seed=11, precision=1, max_batch=1024)
    Yd = _dev(Y)
    start, parts = 0, []
    for b in (300, 17, 700, 260, 90):
        got = server(Yd[start:start + b]).clone()
        want = index.query(Yd[start:start + b], 100, 1000, nprobe=4, seed=11, precision=1,
                           qid_offset=start)
        assert torch.equal(got, want), b
        parts.append(got)
        start += b
    whole = index.query(Yd[:start], 100, 1000, nprobe=4, seed=11, precision=1)
    assert torch.equal(torch.cat(parts), whole)

def _data_small(n=3000, d=8, nq=40, seed=0):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, d)).astype(np.float32),
            rng.standard_normal((nq, d)).astype(np.float32))


def test_batches_on_several_streams_equal_direct_calls(pkg):
    """Uneven batches served round-robin on three streams, each with its own
    view of the index (own scratch and graphs), give exactly the direct calls'
    results, and the backward passes on their lanes match the oracle's
    gradient with the same sets."""
    X, Y, _ = workloads.unit_powerlaw(n=30_000, nq=2_000, n_centres=100)
    h, k, m = 0.2, 100, 1000
    index = pkg.KDEIndex(_dev(X), "exponential", h, nlist=64, seed=5)
    sizes = workloads.uneven_batches(total=2_000, nbatch=12, lo=16, hi=700, seed=4)
    server = pkg.BatchServer(index, k, m, nprobe=4, seed=11, precision=2, max_batch=1024,
                             neighbors=True, streams=3)
    Yd = _dev(Y)
    res = torch.empty(Y.shape[0], dtype=torch.float32, device="cuda")
    start, grads = 0, []
    for b, nb in enumerate(sizes):
        nb = int(nb)
        Yb = Yd[start:start + nb]
        _, ids = server(Yb, out=res[start:start + nb])
        if b % 4 == 0:
            est, dY, dl = server.backward(Yb, ids)
            with torch.cuda.stream(server.last_stream):  # where both were written
                grads.append((start, nb, ids.clone(), dY.clone()))
        start += nb
    server.sync()
    torch.cuda.synchronize()
    want = index.query(Yd, k, m, nprobe=4, seed=11, precision=2)
    assert torch.equal(res, want)
    assert len(server.lanes) == 3 and len(server.graphs) >= 3
    for start, nb, ids, dY in grads:
        r = nb // 2
        q = start + r
        _, w_dY, _ = oracle.deann_grad(X, Y[q:q + 1], "exponential", h,
                                       ids[r:r + 1].cpu().numpy(), m, 11, qid_offset=q)
        assert np.linalg.norm(dY[r].cpu().numpy() - w_dY[0]) <= 1e-4 * np.linalg.norm(w_dY[0])


def test_index_views_share_data_and_keep_their_own_state(pkg):
    """A view answers like its index, keeps its own bandwidth and error
    state, and a second view of a view is refused."""
    X, Y = _data_small()
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.5, nlist=8, seed=2)
    v = index.view()
    a = index.query(_dev(Y), 20, 300, nprobe=3, seed=4, precision=1)
    b = v.query(_dev(Y), 20, 300, nprobe=3, seed=4, precision=1)
    assert torch.equal(a, b) and v.h == index.h
    v.set_bandwidth(3.0)
    assert v.h == 3.0 and index.h == 1.5
    bad = torch.tensor([[0, 5000]], dtype=torch.int32)
    with pytest.raises(pkg.KDEError, match="EINVAL"):
        v.query_with_neighbors(torch.from_numpy(Y[:1]), bad, 10)
    index.sync()  # the index's own error words are clean
    with pytest.raises(pkg.KDEError, match="EINVAL"):
        v.view()
    v.close()
    assert torch.equal(index.query(_dev(Y), 20, 300, nprobe=3, seed=4, precision=1), a)


def test_graphs_stay_valid_when_the_scratch_grows(pkg):
    """A graph captured while the index's scratch was small is replayed after
    larger calls (other shapes, the FP32 scan) made the library allocate a
    bigger buffer: the outgrown buffer is kept, so the replay still gives the
    direct call's result."""
    X, Y, _ = workloads.unit_powerlaw(n=30_000, nq=3_000, n_centres=100)
    index = pkg.KDEIndex(_dev(X), "exponential", 0.2, nlist=64, seed=5)
    Yd = _dev(Y)
    small = pkg.GraphedQuery(index, 64, 50, 500, nprobe=4, seed=2, precision=1)
    got = small(Yd[:40], qid_offset=7).clone()
    # calls that need much more scratch than the graph's capacity
    index.query(Yd, 400, 4000, nprobe=16, seed=1, precision=0)
    index.query(Yd, 400, 4000, nprobe=16, seed=1, precision=1)
    again = small(Yd[:40], qid_offset=7).clone()
    want = index.query(Yd[:40], 50, 500, nprobe=4, seed=2, precision=1, qid_offset=7)
    assert torch.equal(got, want) and torch.equal(again, want)


def test_device_active_rows(pkg):
    """A device-side row count A serves rows below A exactly as a call on
    those rows alone; rows past it get no neighbours (-1) and, through a
    served graph of a larger capacity, add no selection overflow."""
    X, Y, _ = workloads.unit_powerlaw(n=30_000, nq=700, n_centres=100)
    index = pkg.KDEIndex(_dev(X), "exponential", 0.2, nlist=64, seed=5)
    Yd = _dev(Y)
    for A in (700, 413, 1, 0):
        act = torch.tensor([A], dtype=torch.int64, device="cuda")
        out, nbr = index.query(Yd, 100, 1000, nprobe=4, seed=11, precision=1,
                               return_neighbors=True, dev_active=act)
        assert torch.all(nbr[A:] == -1)
        if A:
            want, wnbr = index.query(Yd[:A], 100, 1000, nprobe=4, seed=11, precision=1,
                                     return_neighbors=True)
            assert torch.equal(out[:A], want)
            assert torch.equal(torch.sort(nbr[:A], 1)[0], torch.sort(wnbr, 1)[0])
    index.sync()
    # zero rows in a 1024-row capacity: padding rows used to be zero vectors
    server = pkg.BatchServer(index, 100, 1000, nprobe=4, seed=11, precision=1, max_batch=1024)
    got = server(Yd[:513]).clone()
    assert torch.equal(got, index.query(Yd[:513], 100, 1000, nprobe=4, seed=11, precision=1))
    assert index.margin_failures() == 0


def test_powerlaw_nn_contribution_map(pkg):
    """The Lemma's power-law construction: DEANN with the exact top k (the
    first k ids) matches the oracle draw for draw, and across 8,192 query ids
    the spread of the estimate is the exact ((n - k)/n) sigma / sqrt(m)."""
    X, y, h = workloads.powerlaw_nn(n=50_000, d=16)
    n = X.shape[0]
    index = pkg.KDEIndex(_dev(X), "gaussian", h, nlist=1)
    Kv = np.exp(-((X.astype(np.float64) - y) ** 2).sum(1) / (2 * h * h))
    for k, m in ((0, 2000), (16, 500), (128, 200)):
        Y = np.repeat(y[None], 64, axis=0)
        nbr = np.tile(np.arange(max(k, 1), dtype=np.int32), (64, 1))[:, :k]
        got = (index.query_with_neighbors(_dev(Y), _dev(nbr), m, seed=4).cpu().numpy() if k
               else index.query_rs(_dev(Y), m, seed=4).cpu().numpy())
        want = (oracle.deann(X, Y, "gaussian", h, nbr, m, 4) if k
                else oracle.rs(X, Y, "gaussian", h, m, 4))
        assert_kde_close(got, want)
        R = 8192
        Yr = np.repeat(y[None], R, axis=0)
        nbr_r = np.tile(np.arange(max(k, 1), dtype=np.int32), (R, 1))[:, :k]
        est = (index.query_with_neighbors(_dev(Yr), _dev(nbr_r), m, seed=5) if k
               else index.query_rs(_dev(Yr), m, seed=5)).cpu().numpy().astype(np.float64)
        var = ((n - k) / n) ** 2 * Kv[k:].var() / m
        assert abs(est.var(ddof=1) / var - 1) < 0.1
        assert abs(est.mean() - Kv.mean()) < 6 * np.sqrt(var / R)
