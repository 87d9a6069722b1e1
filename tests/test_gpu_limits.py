"""Edge cases and maximum sizes through the C-ABI, against the oracle: the
widest rows (d = 4096; 1024 for the adjoint), the most probes and lists,
a one-point dataset, sample counts around the estimator's 1,024-sample
chunks, k = n, and the permuted-window tiles with rows too wide to keep
the query tile resident."""
import math

import numpy as np
import pytest
import torch

import oracle
from test_gpu_parity import (_bandwidth, _data, _dev, assert_kde_close,
                             assert_neighbours_match)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2107_02736_gb300 as p
    p.load_library()
    return p


def test_widest_rows(pkg):
    n, d, nq = 600, 4096, 40
    X, Y = _data(n, d, nq, seed=9)
    h = _bandwidth(d)
    index = pkg.KDEIndex(_dev(X), "gaussian", h, nlist=1)
    want = oracle.exact(X, Y, "gaussian", h)
    assert_kde_close(index.exact(_dev(Y), path="cuda").cpu().numpy(), want)
    assert_kde_close(index.exact(_dev(Y), path="tensor").cpu().numpy(), want)
    wn, wd2 = oracle.knn(X, Y, 50)
    for prec in (0, 1):
        nbr, _ = index.search(_dev(Y), 50, nprobe=1, precision=prec)
        assert_neighbours_match(X, Y, nbr.cpu().numpy(), wn, wd2)
        out, nb = index.query(_dev(Y), 50, 1025, nprobe=1, precision=prec, seed=2,
                              return_neighbors=True)
        assert_kde_close(out.cpu().numpy(),
                         oracle.deann(X, Y, "gaussian", h, nb.cpu().numpy(), 1025, 2))
    # DEANNP on the tiled path with the query tile streamed (d > 320)
    index.prepare_permuted()
    perm = oracle.feistel_perm(0, n)
    got = index.query_with_neighbors(_dev(Y), _dev(wn), 300, sample_mode=2).cpu().numpy()
    assert_kde_close(got, oracle.deannp(X, Y, "gaussian", h, perm, wn, 300, ell0=0)[0])


@pytest.mark.parametrize("d", [300, 1024])
def test_adjoint_wide_rows(pkg, d):
    n, nq, k, m = 2000, 30, 20, 300
    X, Y = _data(n, d, nq, seed=d)
    h = _bandwidth(d)
    nbr, _ = oracle.knn(X, Y, k)
    index = pkg.KDEIndex(_dev(X), "gaussian", h)
    out, dY, dl = index.grad_with_neighbors(_dev(Y), _dev(nbr), m, seed=3)
    wo, wdY, wdl = oracle.deann_grad(X, Y, "gaussian", h, nbr, m, 3)
    assert_kde_close(out.cpu().numpy(), wo)
    err = np.linalg.norm(dY.cpu().numpy() - wdY, axis=1) / np.linalg.norm(wdY, axis=1)
    assert err.max() <= 1e-4
    assert np.allclose(dl.cpu().numpy(), wdl, rtol=1e-4, atol=1e-9)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_most_probes(pkg, precision):
    X, Y = _data(30_000, 8, 50, seed=4)
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0, nlist=512, seed=3)
    C, assign = index.export_ivf()
    nbr, _ = index.search(_dev(Y), 100, nprobe=256, precision=precision)
    _, want, wd2 = oracle.ivf_search(X, C.numpy(), assign.numpy(), Y, 256, 100)
    assert_neighbours_match(X, Y, nbr.cpu().numpy(), want, wd2)


def test_most_lists(pkg):
    X, Y = _data(16_384, 4, 40, seed=5)
    index = pkg.KDEIndex(_dev(X), "gaussian", 0.5, nlist=8192, seed=1)
    C, assign = index.export_ivf()
    # every point sits in the list of its nearest centroid
    near, _ = oracle.nearest_centroid(X, C.numpy())
    assert np.mean(near == assign.numpy()) > 0.999
    nbr, _ = index.search(_dev(Y), 20, nprobe=16, precision=1)
    _, want, wd2 = oracle.ivf_search(X, C.numpy(), assign.numpy(), Y, 16, 20)
    assert_neighbours_match(X, Y, nbr.cpu().numpy(), want, wd2)


def test_one_point_dataset(pkg):
    X = np.array([[0.5, -1.0, 2.0]], np.float32)
    Y = np.array([[0.0, 0.0, 0.0], [0.5, -1.0, 2.0], [3.0, 1.0, -1.0]], np.float32)
    index = pkg.KDEIndex(_dev(X), "exponential", 1.3)
    want = oracle.exact(X, Y, "exponential", 1.3)
    assert_kde_close(index.exact(_dev(Y)).cpu().numpy(), want)
    assert_kde_close(index.query(_dev(Y), 1, 10, nprobe=1).cpu().numpy(), want)  # k' = n
    assert_kde_close(index.query_rs(_dev(Y), 7).cpu().numpy(), want)            # every draw is x_0
    S = index.sample_indices(None, 5, nq=3).cpu().numpy()
    assert np.array_equal(S, np.zeros((3, 5), np.int32))


@pytest.mark.parametrize("m", [1, 1023, 1024, 1025, 2049])
@pytest.mark.parametrize("mode", [0, 1])
def test_sample_counts_around_chunks(pkg, m, mode):
    X, Y = _data(5000, 16, 20, seed=m)
    h = _bandwidth(16)
    nbr, _ = oracle.knn(X, Y, 40)
    index = pkg.KDEIndex(_dev(X), "gaussian", h)
    got = index.query_with_neighbors(_dev(Y), _dev(nbr), m, seed=6, sample_mode=mode)
    assert_kde_close(got.cpu().numpy(), oracle.deann(X, Y, "gaussian", h, nbr, m, 6, mode=mode))
    S = index.sample_indices(_dev(nbr), m, seed=6, sample_mode=mode).cpu().numpy()
    _, want = oracle.deann(X, Y, "gaussian", h, nbr, m, 6, mode=mode, return_samples=True)
    assert np.array_equal(S, want)


def test_k_equals_n_at_the_largest_k(pkg):
    X, Y = _data(2048, 8, 30, seed=8)
    index = pkg.KDEIndex(_dev(X), "laplacian", 3.0, nlist=4, seed=2)
    out = index.query(_dev(Y), 2048, 100, nprobe=4, precision=1)
    assert_kde_close(out.cpu().numpy(), oracle.exact(X, Y, "laplacian", 3.0))


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_largest_k_search_and_estimate(pkg, precision):
    """k = 2048 of n = 30,000 through the IVF: neighbours against the oracle's
    search of the same lists, estimates against the oracle with them."""
    X, Y = _data(30_000, 16, 40, seed=13)
    h = _bandwidth(16)
    index = pkg.KDEIndex(_dev(X), "gaussian", h, nlist=64, seed=3)
    C, assign = index.export_ivf()
    out, nbr = index.query(_dev(Y), 2048, 700, nprobe=16, precision=precision, seed=4,
                           return_neighbors=True)
    nbr = nbr.cpu().numpy()
    _, want, wd2 = oracle.ivf_search(X, C.numpy(), assign.numpy(), Y, 16, 2048)
    assert_neighbours_match(X, Y, nbr, want, wd2)
    assert_kde_close(out.cpu().numpy(), oracle.deann(X, Y, "gaussian", h, nbr, 700, 4))
    assert index.margin_failures() == 0


@pytest.mark.parametrize("kernel", ["gaussian", "laplacian"])
def test_deannp_tiles_with_streamed_queries(pkg, kernel):
    n, d, m, nq = 3000, 400, 1500, 64  # n / gcd(n, m) = 2 classes of 32 queries
    X, Y = _data(n, d, nq, seed=12)
    h = _bandwidth(d) if kernel == "gaussian" else 0.5 * d
    nbr, _ = oracle.knn(X, Y, 25)
    index = pkg.KDEIndex(_dev(X), kernel, h, seed=4)
    index.prepare_permuted()
    perm = oracle.feistel_perm(4, n)
    got = index.query_with_neighbors(_dev(Y), _dev(nbr), m, sample_mode=2, qid_offset=5)
    want, _ = oracle.deannp(X, Y, kernel, h, perm, nbr, m, ell0=(5 * m) % n)
    assert_kde_close(got.cpu().numpy(), want)
