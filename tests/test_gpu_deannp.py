"""DEANNP and RSP (Algorithm 2, permuted sampling) on the GPU vs the oracle.

The permutation pi is integer work and must match the oracle's Feistel
permutation bit for bit, and so must the window ids; estimates follow the
same bar as DEANN (relative 1e-5 for values >= 1e-6).  The query with global
id qid reads the window that starts at (qid m) mod n, which is the oracle's
running index ell0 + q m with ell0 = (qid_offset m) mod n.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from test_gpu_parity import _bandwidth, _data, _dev, assert_kde_close

pytestmark = pytest.mark.gpu

SEED = 0x9E3779B97F4A7C15


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2107_02736_gb300 as p
    p.load_library()
    return p


def _window_ids(perm, nbr, qid0, m):
    """Oracle-side window ids (the kept ids, -1 for dropped X_1 members)."""
    n = perm.size
    out = np.empty((nbr.shape[0], m), np.int32)
    for q in range(nbr.shape[0]):
        ell = ((qid0 + q) * m) % n
        ids = perm[(ell + np.arange(m)) % n]
        members = set(int(v) for v in nbr[q] if v >= 0)
        out[q] = np.where(np.isin(ids, list(members)), -1, ids)
    return out


@pytest.mark.parametrize("n", [1, 2, 5, 3000, 4096, 65537])
def test_permutation_bit_exact(pkg, n):
    X, _ = _data(n, 4, 1, seed=n)
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0, seed=SEED)
    perm = index.prepare_permuted(return_perm=True).cpu().numpy()
    assert np.array_equal(perm, oracle.feistel_perm(SEED, n))
    # idempotent: a second call keeps the same permutation
    assert np.array_equal(index.prepare_permuted(return_perm=True).cpu().numpy(), perm)


def test_window_ids_bit_exact(pkg):
    """Windows span several 1024-entry chunks, wrap at n, and drop X_1
    members (duplicates and -1 padding in the neighbour rows)."""
    n, nq, k, m = 3000, 40, 30, 2500
    X, Y = _data(n, 8, nq, seed=4)
    nbr, _ = oracle.knn(X, Y, k)
    nbr[::3, 5] = nbr[::3, 4]
    nbr[1::4, -3:] = -1
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0, seed=7)
    index.prepare_permuted()
    perm = oracle.feistel_perm(7, n)
    qoff = (1 << 40) + 3
    got = index.sample_indices(_dev(nbr), m, sample_mode=2, qid_offset=qoff).cpu().numpy()
    assert np.array_equal(got, _window_ids(perm, nbr, qoff, m))


@pytest.mark.parametrize("d", [3, 17, 128])
@pytest.mark.parametrize("kernel", ["gaussian", "exponential", "laplacian"])
def test_deannp_with_neighbors(pkg, d, kernel):
    n, nq, k, m = 3000, 70, 25, 700
    X, Y = _data(n, d, nq, seed=d + 1)
    h = _bandwidth(d) if kernel == "gaussian" else _bandwidth(d) * 0.5
    if kernel == "laplacian":
        h = 0.5 * d
    nbr, _ = oracle.knn(X, Y, k)
    index = pkg.KDEIndex(_dev(X), kernel, h, seed=11)
    index.prepare_permuted()
    perm = oracle.feistel_perm(11, n)
    for qoff in (0, 5, (1 << 33) + 17):
        got = index.query_with_neighbors(_dev(Y), _dev(nbr), m, sample_mode=2,
                                         qid_offset=qoff).cpu().numpy()
        want, _ = oracle.deannp(X, Y, kernel, h, perm, nbr, m, ell0=(qoff * m) % n)
        assert_kde_close(got, want)


def test_deannp_full_window_is_exact(pkg):
    n, nq, k = 2000, 30, 40
    X, Y = _data(n, 16, nq, seed=2)
    h = _bandwidth(16)
    nbr, _ = oracle.knn(X, Y, k)
    index = pkg.KDEIndex(_dev(X), "gaussian", h, seed=3)
    index.prepare_permuted()
    got = index.query_with_neighbors(_dev(Y), _dev(nbr), n, sample_mode=2, qid_offset=9)
    assert_kde_close(got.cpu().numpy(), oracle.exact(X, Y, "gaussian", h))


def test_rsp_and_consecutive_windows(pkg):
    """RSP: k = 0 windows; n / m consecutive query ids of one query point
    cover X once, so their mean is the exact KDE."""
    n, m = 3000, 250
    X, Y = _data(n, 16, 12, seed=5)
    h = _bandwidth(16)
    index = pkg.KDEIndex(_dev(X), "exponential", h, seed=21)
    index.prepare_permuted()
    perm = oracle.feistel_perm(21, n)
    got = index.query_rs(_dev(Y), m, sample_mode=2, qid_offset=4).cpu().numpy()
    want, _ = oracle.deannp(X, Y, "exponential", h, perm, None, m, ell0=(4 * m) % n)
    assert_kde_close(got, want)
    Yrep = np.repeat(Y[:1], n // m, axis=0)
    rep = index.query_rs(_dev(Yrep), m, sample_mode=2).cpu().numpy().astype(np.float64)
    exact = oracle.exact(X, Y[:1], "exponential", h)[0]
    assert abs(rep.mean() - exact) <= 1e-5 * exact


def test_deannp_query_end_to_end(pkg):
    X, Y, _ = workloads.mixture_iso(n=10_000, d=16, nq=200)
    index = pkg.KDEIndex(_dev(X), "gaussian", 2.0, nlist=16, seed=1)
    index.prepare_permuted()
    perm = oracle.feistel_perm(1, 10_000)
    for precision in (0, 1):
        out, nbr = index.query(_dev(Y), 50, 900, nprobe=4, precision=precision,
                               sample_mode=2, qid_offset=77, return_neighbors=True)
        nbr = nbr.cpu().numpy()
        want, _ = oracle.deannp(X, Y, "gaussian", 2.0, perm, nbr, 900, ell0=(77 * 900) % 10_000)
        assert_kde_close(out.cpu().numpy(), want)


def test_deannp_graph_batches_follow_on(pkg):
    """BatchServer with sample_mode=2: each batch's windows follow on from the
    previous batch's (the running index of Algorithm 2)."""
    n, m, k = 5000, 300, 20
    X, Y = _data(n, 16, 100, seed=8)
    h = _bandwidth(16)
    index = pkg.KDEIndex(_dev(X), "gaussian", h, nlist=4, seed=2)
    index.prepare_permuted()
    server = pkg.BatchServer(index, k, m, nprobe=4, sample_mode=2, max_batch=64)
    outs = [server(_dev(Y[a:b])).clone() for a, b in ((0, 30), (30, 37), (37, 100))]
    got = torch.cat(outs).cpu().numpy()
    direct = index.query(_dev(Y), k, m, nprobe=4, sample_mode=2).cpu().numpy()
    assert np.array_equal(got, direct)


def test_deannp_argument_errors(pkg):
    X, Y = _data(500, 4, 3, seed=1)
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0)
    nbr = np.zeros((3, 2), np.int32)
    with pytest.raises(pkg.KDEError) as e:
        index.query_with_neighbors(_dev(Y), _dev(nbr), 10, sample_mode=2)
    assert e.value.status == 5  # not prepared
    index.prepare_permuted()
    with pytest.raises(pkg.KDEError) as e:
        index.query_with_neighbors(_dev(Y), _dev(nbr), 501, sample_mode=2)
    assert e.value.status == 1  # m > n
    with pytest.raises(pkg.KDEError) as e:
        index.grad_with_neighbors(_dev(Y), _dev(nbr), 10, sample_mode=2)
    assert e.value.status == 1
    with pytest.raises(pkg.KDEError) as e:
        index.query_rs(_dev(Y), 10, sample_mode=3)
    assert e.value.status == 1


# --------------------------------------------- windows shared by many queries --
# With A = nq / P >= 16 queries per window (P = n / gcd(n, m)) the estimator
# runs as dense (queries x window rows) tiles.
@pytest.mark.parametrize("n,m,nq", [(4096, 512, 300),    # P = 8, A = 37: one query tile
                                    (2000, 1000, 300),   # P = 2, A = 150: three query tiles
                                    (3001, 3001, 40),    # P = 1: the full window
                                    (6000, 1500, 200)])  # P = 4, A = 50
@pytest.mark.parametrize("kernel", ["gaussian", "exponential", "laplacian"])
def test_tiled_windows_match_oracle(pkg, n, m, nq, kernel):
    d = 17 if kernel != "gaussian" else 128
    X, Y = _data(n, d, nq, seed=n + nq)
    h = _bandwidth(d) if kernel != "laplacian" else 0.5 * d
    k = 50
    nbr, _ = oracle.knn(X, Y, k)
    nbr[::5, 3] = nbr[::5, 2]   # duplicates count once
    nbr[2::7, -4:] = -1         # padding
    index = pkg.KDEIndex(_dev(X), kernel, h, seed=31)
    index.prepare_permuted()
    perm = oracle.feistel_perm(31, n)
    for qoff in (0, 123457):
        got = index.query_with_neighbors(_dev(Y), _dev(nbr), m, sample_mode=2,
                                         qid_offset=qoff).cpu().numpy()
        want, _ = oracle.deannp(X, Y, kernel, h, perm, nbr, m, ell0=(qoff * m) % n)
        assert_kde_close(got, want)
    # host pointers take the same path
    got_h = index.query_with_neighbors(torch.from_numpy(Y), torch.from_numpy(nbr), m,
                                       sample_mode=2).numpy()
    want0, _ = oracle.deannp(X, Y, kernel, h, perm, nbr, m, ell0=0)
    assert_kde_close(got_h, want0)


def test_tiled_windows_rsp_and_search(pkg):
    n, m, nq = 8192, 1024, 400  # P = 8, A = 50
    X, Y, _ = workloads.mixture_iso(n=n, d=16, nq=nq)
    index = pkg.KDEIndex(_dev(X), "gaussian", 2.0, nlist=8, seed=4)
    index.prepare_permuted()
    perm = oracle.feistel_perm(4, n)
    got = index.query_rs(_dev(Y), m, sample_mode=2, qid_offset=3).cpu().numpy()
    want, _ = oracle.deannp(X, Y, "gaussian", 2.0, perm, None, m, ell0=(3 * m) % n)
    assert_kde_close(got, want)
    out, nbr = index.query(_dev(Y), 40, m, nprobe=4, sample_mode=2, precision=1,
                           return_neighbors=True)
    want, _ = oracle.deannp(X, Y, "gaussian", 2.0, perm, nbr.cpu().numpy(), m, ell0=0)
    assert_kde_close(out.cpu().numpy(), want)


def test_tiled_windows_under_graph_replays(pkg):
    n, m, k = 4096, 512, 20  # P = 8; capacity 256 gives A = 32
    X, Y = _data(n, 32, 600, seed=12)
    h = _bandwidth(32)
    index = pkg.KDEIndex(_dev(X), "gaussian", h, nlist=4, seed=6)
    index.prepare_permuted()
    g = pkg.GraphedQuery(index, 256, k, m, nprobe=4, sample_mode=2)
    for off, (a, b) in ((0, (0, 256)), (256, (256, 512)), (1000, (100, 356))):
        got = g(_dev(Y[a:b]), qid_offset=off).clone()
        want = index.query(_dev(Y[a:b]), k, m, nprobe=4, sample_mode=2, qid_offset=off)
        assert torch.equal(got, want)
