"""GPU path vs the FP64 oracle, element by element, through the C-ABI.

Bars: sample indices and neighbour ids bit-exact (neighbour sets may differ
only among candidates whose oracle distance is within 1e-6 max(1, d_k) of the
k-th distance d_k); KDE values >= 1e-6 within 1e-5 relative error (FP32 path
vs FP64 oracle); gradients within 1e-4 relative (vector norm).
Sizes span several 64-row tiles with ragged tails.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

REL = 1e-5
FLOOR = 1e-6


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2107_02736_gb300 as p
    p.load_library()
    return p


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def assert_kde_close(got, want, rel=REL, floor=FLOOR):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert np.all(np.isfinite(got))
    mask = want >= floor
    err = np.abs(got - want) / np.maximum(np.abs(want), 1e-300)
    assert np.all(err[mask] <= rel), f"max rel err {err[mask].max():.3e} (bar {rel})"
    small = ~mask
    assert np.all(np.abs(got[small] - want[small]) <= rel * floor + 1e-12)


def assert_neighbours_match(X, Y, got_nbr, want_nbr, want_d2):
    """Sets equal except among near-ties at the k-th distance."""
    for q in range(got_nbr.shape[0]):
        g = got_nbr[q][got_nbr[q] >= 0]
        w = want_nbr[q][want_nbr[q] >= 0]
        assert g.size == w.size
        if np.array_equal(np.sort(g), np.sort(w)):
            continue
        dk = want_d2[q][w.size - 1]
        tol = 1e-6 * max(1.0, dk)
        extra = np.setdiff1d(g, w)
        missing = np.setdiff1d(w, g)
        d_extra = ((X[extra].astype(np.float64) - Y[q]) ** 2).sum(1)
        d_missing = ((X[missing].astype(np.float64) - Y[q]) ** 2).sum(1)
        assert np.all(np.abs(d_extra - dk) <= tol), (q, d_extra, dk)
        assert np.all(np.abs(d_missing - dk) <= tol), (q, d_missing, dk)


def _data(n, d, nq, seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    X = (scale * rng.standard_normal((n, d))).astype(np.float32)
    Y = (scale * rng.standard_normal((nq, d))).astype(np.float32)
    return X, Y


def _bandwidth(d, scale=1.0):
    # puts typical kernel values well inside (0, 1)
    return 0.6 * scale * math.sqrt(d)


# ----------------------------------------------------------------- sampling --
@pytest.mark.parametrize("mode", [0, 1])
def test_sample_indices_bit_exact(pkg, mode):
    n, k, m = 1000, 40, 700
    X, Y = _data(n, 4, 37)
    rng = np.random.default_rng(1)
    nbr = rng.integers(-1, n, size=(37, k)).astype(np.int32)
    nbr[:, 5] = nbr[:, 6]  # duplicates
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0)
    for qoff in (0, 12345, 2**40 + 7):
        got = index.sample_indices(_dev(nbr), m, seed=99, sample_mode=mode,
                                   qid_offset=qoff).cpu().numpy()
        _, want = oracle.deann(X, Y, "gaussian", 1.0, nbr, m, 99, qid_offset=qoff, mode=mode,
                               return_samples=True)
        assert np.array_equal(got, want)
    # random sampling draws (k = 0)
    got = index.sample_indices(None, m, seed=5, nq=37).cpu().numpy()
    _, want = oracle.rs(X, Y, "gaussian", 1.0, m, 5, return_samples=True)
    assert np.array_equal(got, want)


def test_sample_indices_host_pointers(pkg):
    X, Y = _data(500, 3, 9)
    nbr = np.tile(np.arange(30, dtype=np.int32), (9, 1))
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0)
    got = index.sample_indices(torch.from_numpy(nbr), 2500, seed=3, device="cpu").numpy()
    _, want = oracle.deann(X, Y, "gaussian", 1.0, nbr, 2500, 3, return_samples=True)
    assert np.array_equal(got, want)


# ----------------------------------------------------------------- estimates --
@pytest.mark.parametrize("d", [1, 3, 16, 17, 128, 784])
@pytest.mark.parametrize("kernel", ["gaussian", "exponential", "laplacian"])
def test_query_with_neighbors(pkg, d, kernel):
    n, nq, k, m = 3000, 70, 25, 300
    X, Y = _data(n, d, nq, seed=d)
    h = _bandwidth(d) if kernel == "gaussian" else _bandwidth(d) * 0.5
    if kernel == "laplacian":
        h = 0.5 * d
    nbr, _ = oracle.knn(X, Y, k)
    index = pkg.KDEIndex(_dev(X), kernel, h)
    got = index.query_with_neighbors(_dev(Y), _dev(nbr), m, seed=7).cpu().numpy()
    want = oracle.deann(X, Y, kernel, h, nbr, m, 7)
    assert_kde_close(got, want)
    got1 = index.query_with_neighbors(_dev(Y), _dev(nbr), m, seed=7, sample_mode=1)
    want1 = oracle.deann(X, Y, kernel, h, nbr, m, 7, mode=1)
    assert_kde_close(got1.cpu().numpy(), want1)


@pytest.mark.parametrize("kernel", ["gaussian", "exponential", "laplacian"])
def test_rs(pkg, kernel):
    X, Y = _data(2000, 16, 50, seed=3)
    h = 3.0 if kernel != "laplacian" else 10.0
    index = pkg.KDEIndex(_dev(X), kernel, h)
    got = index.query_rs(_dev(Y), 1000, seed=11).cpu().numpy()
    assert_kde_close(got, oracle.rs(X, Y, kernel, h, 1000, 11))


def test_full_neighbour_set_is_exact(pkg):
    X, Y = _data(300, 5, 20, seed=4)
    nbr = np.tile(np.arange(300, dtype=np.int32), (20, 1))
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.5)
    got = index.query_with_neighbors(_dev(Y), _dev(nbr), 50, seed=0).cpu().numpy()
    assert_kde_close(got, oracle.exact(X, Y, "gaussian", 1.5))


def test_m_zero_and_padding(pkg):
    X, Y = _data(400, 6, 10, seed=5)
    nbr, _ = oracle.knn(X, Y, 12)
    nbr = np.concatenate([nbr, -np.ones((10, 4), np.int32), nbr[:, :3]], axis=1)
    index = pkg.KDEIndex(_dev(X), "exponential", 2.0)
    got = index.query_with_neighbors(_dev(Y), _dev(nbr), 0, seed=0).cpu().numpy()
    assert_kde_close(got, oracle.deann(X, Y, "exponential", 2.0, nbr, 0, 0))


# --------------------------------------------------------------------- exact --
@pytest.mark.parametrize("d", [1, 3, 16, 17, 128])
@pytest.mark.parametrize("kernel", ["gaussian", "exponential", "laplacian"])
def test_exact(pkg, d, kernel):
    n, nq = 5000, 130
    X, Y = _data(n, d, nq, seed=10 + d)
    h = _bandwidth(d) if kernel != "laplacian" else 0.7 * d
    index = pkg.KDEIndex(_dev(X), kernel, h)
    want = oracle.exact(X, Y, kernel, h)
    got = index.exact(_dev(Y)).cpu().numpy()
    assert_kde_close(got, want)
    got_c = index.exact(_dev(Y), path="cuda").cpu().numpy()
    assert_kde_close(got_c, want)
    if kernel != "laplacian":
        got_t = index.exact(_dev(Y), path="tensor").cpu().numpy()
        assert_kde_close(got_t, want)
    # host-pointer path: same numbers up to the order of the FP64 atomics
    got_h = index.exact(torch.from_numpy(Y)).numpy()
    assert np.allclose(got, got_h, rtol=1e-6, atol=0)


@pytest.mark.parametrize("which,h", [("embed128", 12.8), ("unit300", 0.35), ("sparse784", 1.3)])
def test_exact_tensor_cores_on_workload_shapes(pkg, which, h):
    """The three-way BF16 split keeps FP32-level accuracy on the workloads'
    own geometry (norms far from zero, d up to 784, ragged tiles) inside its
    accuracy guard, max |x - mean|^2 <= 8 (2 h^2)."""
    if which == "embed128":
        X, Y, _ = workloads.mixture_embed(n=20000, nq=200, n_centres=50)
    elif which == "unit300":
        X, Y, _ = workloads.unit_powerlaw(n=20000, nq=150, n_centres=60)
    else:
        X, Y, _ = workloads.sparse_image(n=6000, nq=100)
    index = pkg.KDEIndex(_dev(X), "gaussian", h)
    assert_kde_close(index.exact(_dev(Y), path="tensor").cpu().numpy(),
                     oracle.exact(X, Y, "gaussian", h))
    index.close()
    if which == "embed128":
        index = pkg.KDEIndex(_dev(X), "exponential", h)
        assert_kde_close(index.exact(_dev(Y), path="tensor").cpu().numpy(),
                         oracle.exact(X, Y, "exponential", h))


def test_exact_auto_path_respects_accuracy_guard(pkg):
    """A bandwidth far below the data's spread sends the automatic path to the
    CUDA cores (2 launches per call) instead of the tensor cores (3)."""
    X, Y, _ = workloads.unit_powerlaw(n=5000, nq=50, n_centres=20)
    for h, want_launches in ((0.05, 2), (0.5, 3)):
        index = pkg.KDEIndex(_dev(X), "gaussian", h)
        index.profile_read(reset=True)
        got = index.exact(_dev(Y)).cpu().numpy()
        assert index.profile_read(reset=True)["exact"]["launches"] == want_launches
        assert_kde_close(got, oracle.exact(X, Y, "gaussian", h))
        index.close()


# ---------------------------------------------------------------- ANN search --
@pytest.mark.parametrize("d", [2, 16, 33])
def test_brute_force_search(pkg, d):
    n, nq, k = 4100, 90, 50
    X, Y = _data(n, d, nq, seed=20 + d)
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0)
    nbr, d2 = index.search(_dev(Y), k, nprobe=1)
    want, want_d2 = oracle.knn(X, Y, k)
    assert_neighbours_match(X, Y, nbr.cpu().numpy(), want, want_d2)
    d2 = d2.cpu().numpy()
    assert np.allclose(d2, np.sort(d2, axis=1))
    same = nbr.cpu().numpy() == want
    assert np.allclose(d2[same], want_d2[same], rtol=1e-6, atol=1e-6)


def test_search_with_ties(pkg):
    """Integer grid data: many exactly equal distances, broken by lower id."""
    rng = np.random.default_rng(3)
    X = rng.integers(-2, 3, size=(3000, 3)).astype(np.float32)
    Y = rng.integers(-2, 3, size=(40, 3)).astype(np.float32)
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0)
    nbr, _ = index.search(_dev(Y), 30)
    want, _ = oracle.knn(X, Y, 30)
    assert np.array_equal(nbr.cpu().numpy(), want)


def test_ivf_build_assignment_and_search(pkg):
    X, Y, _ = workloads.mixture_iso(n=6000, d=16, nq=80)
    index = pkg.KDEIndex(_dev(X), "gaussian", 2.0, nlist=24, seed=3)
    C, assign = index.export_ivf()
    C, assign = C.numpy(), assign.numpy()
    # final assignment: nearest centroid, up to near-ties
    a_or, d_or = oracle.nearest_centroid(X, C)
    diff = np.flatnonzero(a_or != assign)
    if diff.size:
        d_got = ((X[diff].astype(np.float64) - C[assign[diff]]) ** 2).sum(1)
        assert np.all(d_got <= d_or[diff] * (1 + 1e-5) + 1e-6)
    counts = np.bincount(assign, minlength=24)
    assert counts.sum() == 6000 and np.all(counts > 0)
    for P in (1, 3, 24):
        nbr, d2 = index.search(_dev(Y), 40, nprobe=P)
        _, want, want_d2 = oracle.ivf_search(X, C, assign, Y, P, 40)
        assert_neighbours_match(X, Y, nbr.cpu().numpy(), want, want_d2)


@pytest.mark.parametrize("L", [16, 64])
def test_kmeans_build_matches_oracle(pkg, L):
    """The IVF build's k-means against the oracle's: the same Philox initial
    points and Lloyd iterations (GPU assignment distances in FP32, the oracle's
    in FP64) end with the same lists and centroids, up to points whose two
    nearest centroids are nearly equidistant."""
    X, _, _ = workloads.mixture_iso(n=20000, d=16, nq=16)
    index = pkg.KDEIndex(_dev(X), "gaussian", 2.0, nlist=L, seed=3)
    C, a = (t.numpy() for t in index.export_ivf())
    Co, ao, _, st = oracle.kmeans(X, L, 3, iters=20)
    assert st == oracle.OK
    assert np.mean(a == ao) >= 0.999

    def objective(C, a):
        return np.mean(((X.astype(np.float64) - C[a].astype(np.float64)) ** 2).sum(1))
    assert abs(objective(C, a) / objective(Co, ao) - 1.0) <= 1e-4
    same = [l for l in range(L)
            if np.array_equal(np.flatnonzero(a == l), np.flatnonzero(ao == l))]
    assert len(same) >= 0.9 * L
    assert np.allclose(C[same], Co[same], rtol=0.0, atol=1e-5)


def test_query_end_to_end(pkg):
    X, Y, _ = workloads.mixture_iso(n=10_000, d=16, nq=200)
    index = pkg.KDEIndex(_dev(X), "gaussian", 2.0, nlist=16, seed=1)
    C, assign = index.export_ivf()
    out, nbr = index.query(_dev(Y), 50, 500, nprobe=4, seed=0, return_neighbors=True)
    nbr = nbr.cpu().numpy()
    _, want, want_d2 = oracle.ivf_search(X, C.numpy(), assign.numpy(), Y, 4, 50)
    assert_neighbours_match(X, Y, nbr, want, want_d2)
    assert_kde_close(out.cpu().numpy(), oracle.deann(X, Y, "gaussian", 2.0, nbr, 500, 0))
    assert index.margin_failures() == 0


@pytest.mark.parametrize("which", ["iso16", "embed128", "unit300", "sparse784"])
def test_bf16_tensor_core_scan(pkg, which):
    """precision=BF16: the tcgen05 scan ranks candidates in BF16; after FP32
    rescoring the neighbours match the oracle's IVF search as tightly as the
    FP32 path does."""
    if which == "iso16":
        X, Y, _ = workloads.mixture_iso(n=7000, d=16, nq=300)
    elif which == "embed128":
        X, Y, _ = workloads.mixture_embed(n=9000, nq=300, n_centres=30)
    elif which == "unit300":
        X, Y, _ = workloads.unit_powerlaw(n=6000, nq=200, n_centres=40)
    else:
        X, Y, _ = workloads.sparse_image(n=5000, nq=120)
    index = pkg.KDEIndex(_dev(X), "gaussian", 2.0, nlist=12, seed=2)
    C, assign = index.export_ivf()
    for P, k in ((1, 25), (3, 60), (12, 100)):
        nbr, d2 = index.search(_dev(Y), k, nprobe=P, precision=1)
        _, want, want_d2 = oracle.ivf_search(X, C.numpy(), assign.numpy(), Y, P, k)
        assert_neighbours_match(X, Y, nbr.cpu().numpy(), want, want_d2)
        f32, _ = index.search(_dev(Y), k, nprobe=P, precision=0)
        assert np.array_equal(np.sort(f32.cpu().numpy(), 1), np.sort(nbr.cpu().numpy(), 1))
    assert index.margin_failures() == 0
    out, nb = index.query(_dev(Y), 30, 300, nprobe=3, seed=9, precision=1, return_neighbors=True)
    assert_kde_close(out.cpu().numpy(),
                     oracle.deann(X, Y, "gaussian", 2.0, nb.cpu().numpy(), 300, 9))


@pytest.mark.parametrize("precision", [1, 2])
def test_bf16_scan_many_queries_per_list(pkg, precision):
    """Hundreds of queries probing the same lists: several CTAs per list, ragged
    last query group and ragged last 128-point tile."""
    X, Y, _ = workloads.mixture_iso(n=3000, d=32, nq=900, n_centres=3)
    index = pkg.KDEIndex(_dev(X), "gaussian", 2.0, nlist=5, seed=4)
    C, assign = index.export_ivf()
    nbr, _ = index.search(_dev(Y), 64, nprobe=2, precision=precision)
    _, want, want_d2 = oracle.ivf_search(X, C.numpy(), assign.numpy(), Y, 2, 64)
    assert_neighbours_match(X, Y, nbr.cpu().numpy(), want, want_d2)


@pytest.mark.parametrize("which", ["iso16", "embed128", "unit300", "sparse784"])
@pytest.mark.parametrize("kernel", ["gaussian", "exponential", "laplacian"])
def test_split_scan_matches_oracle(pkg, which, kernel):
    """The three-way split BF16 scan (precision 2): its distances are used
    without rescoring the neighbours' rows, so the sorted neighbours, their
    distances and the estimates (the neighbours' kernel values come from the
    scan) must match the oracle as the rescored paths do; sets equal the FP32
    scan's."""
    if which == "iso16":
        X, Y, _ = workloads.mixture_iso(n=7000, d=16, nq=300)
        h = 2.0
    elif which == "embed128":
        X, Y, _ = workloads.mixture_embed(n=9000, nq=300, n_centres=30)
        h = 6.0
    elif which == "unit300":
        X, Y, _ = workloads.unit_powerlaw(n=6000, nq=200, n_centres=40)
        h = 0.3
    else:
        X, Y, _ = workloads.sparse_image(n=5000, nq=120)
        h = 1.5
    if kernel == "laplacian":
        h *= 3.0
    index = pkg.KDEIndex(_dev(X), kernel, h, nlist=12, seed=2)
    C, assign = index.export_ivf()
    for P, k in ((1, 25), (3, 60), (12, 100)):
        nbr, d2 = index.search(_dev(Y), k, nprobe=P, precision=2)
        _, want, want_d2 = oracle.ivf_search(X, C.numpy(), assign.numpy(), Y, P, k)
        assert_neighbours_match(X, Y, nbr.cpu().numpy(), want, want_d2)
        # the split's error is absolute, on the scale of the centred operands:
        # bounded against each query's k-th distance
        d2 = d2.cpu().numpy().astype(np.float64)
        scale = np.maximum(np.where(want >= 0, want_d2, 0.0).max(1, keepdims=True), 1.0)
        ok = want >= 0
        assert np.all((np.abs(d2 - want_d2) <= 1e-5 * scale)[ok])
        f32, _ = index.search(_dev(Y), k, nprobe=P, precision=0)
        assert np.array_equal(np.sort(f32.cpu().numpy(), 1), np.sort(nbr.cpu().numpy(), 1))
    assert index.margin_failures() == 0
    out, nb = index.query(_dev(Y), 30, 300, nprobe=3, seed=9, precision=2, return_neighbors=True)
    assert_kde_close(out.cpu().numpy(),
                     oracle.deann(X, Y, kernel, h, nb.cpu().numpy(), 300, 9))
    # the neighbour part alone (m = 0): s1 / n from the scan's values
    out0, nb0 = index.query(_dev(Y), 60, 0, nprobe=3, precision=2, return_neighbors=True)
    assert_kde_close(out0.cpu().numpy(),
                     oracle.deann(X, Y, kernel, h, nb0.cpu().numpy(), 0, 0))


def test_split_scan_rejects_wide_rows(pkg):
    X, Y = _data(400, 1200, 3, seed=2)
    index = pkg.KDEIndex(_dev(X), "gaussian", 30.0, nlist=4)
    with pytest.raises(pkg.KDEError, match="EINVAL"):
        index.search(_dev(Y), 5, nprobe=1, precision=2)
    assert index.search(_dev(Y), 5, nprobe=1, precision=1)[0].shape == (3, 5)


def test_query_k_equals_n_is_exact(pkg):
    X, Y = _data(700, 4, 15, seed=8)
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.2)
    out = index.query(_dev(Y), 700, 100, nprobe=1, seed=0).cpu().numpy()
    assert_kde_close(out, oracle.exact(X, Y, "gaussian", 1.2))


def test_query_rs_via_k0(pkg):
    X, Y = _data(900, 8, 33, seed=9)
    index = pkg.KDEIndex(_dev(X), "exponential", 2.0, nlist=4)
    a = index.query(_dev(Y), 0, 400, seed=17).cpu().numpy()
    assert_kde_close(a, oracle.rs(X, Y, "exponential", 2.0, 400, 17))


def test_host_and_device_paths_agree(pkg):
    X, Y, _ = workloads.mixture_iso(n=5000, d=16, nq=64)
    index = pkg.KDEIndex(torch.from_numpy(X), "gaussian", 2.0, nlist=8)
    a = index.query(_dev(Y), 30, 200, nprobe=2, seed=4).cpu().numpy()
    b = index.query(torch.from_numpy(Y), 30, 200, nprobe=2, seed=4).numpy()
    assert np.array_equal(a, b)


# ------------------------------------------------------------------ gradient --
@pytest.mark.parametrize("kernel", ["gaussian", "exponential", "laplacian"])
@pytest.mark.parametrize("d", [3, 16, 64])
def test_gradient_matches_oracle(pkg, kernel, d):
    n, nq, k, m = 2500, 40, 30, 400
    X, Y = _data(n, d, nq, seed=30 + d)
    h = _bandwidth(d) if kernel != "laplacian" else 0.6 * d
    nbr, _ = oracle.knn(X, Y, k)
    rng = np.random.default_rng(2)
    gout = rng.uniform(0.5, 2.0, size=nq).astype(np.float32)
    index = pkg.KDEIndex(_dev(X), kernel, h)
    out, dY, dl = index.grad_with_neighbors(_dev(Y), _dev(nbr), m, seed=6, gout=_dev(gout))
    w_out, w_dY, w_dl = oracle.deann_grad(X, Y, kernel, h, nbr, m, 6, gout=gout)
    assert_kde_close(out.cpu().numpy(), w_out)
    dY = dY.cpu().numpy().astype(np.float64)
    for q in range(nq):
        nrm = np.linalg.norm(w_dY[q])
        assert np.linalg.norm(dY[q] - w_dY[q]) <= 1e-4 * nrm + 1e-9
    dl = dl.cpu().numpy()
    assert np.all(np.abs(dl - w_dl) <= 1e-4 * np.abs(w_dl) + 1e-9)


def test_gradient_with_padding_and_repeated_ids(pkg):
    """Neighbour rows with -1 padding between valid ids (the hash-set path,
    rows taken in row order) and rows with a repeated id (the sorted,
    deduplicated path): both give the oracle's gradient, k' counting each id
    once."""
    n, nq, k, m, d = 2500, 36, 30, 400, 16
    X, Y = _data(n, d, nq, seed=71)
    h = _bandwidth(d)
    nbr, _ = oracle.knn(X, Y, k)
    nbr[0::3, 4] = -1
    nbr[0::3, 11] = -1
    nbr[1::3, 7] = nbr[1::3, 2]
    index = pkg.KDEIndex(_dev(X), "gaussian", h)
    out, dY, dl = index.grad_with_neighbors(_dev(Y), _dev(nbr), m, seed=8)
    w_out, w_dY, w_dl = oracle.deann_grad(X, Y, "gaussian", h, nbr, m, 8)
    assert_kde_close(out.cpu().numpy(), w_out)
    dY = dY.cpu().numpy().astype(np.float64)
    for q in range(nq):
        assert np.linalg.norm(dY[q] - w_dY[q]) <= 1e-4 * np.linalg.norm(w_dY[q]) + 1e-9
    assert np.all(np.abs(dl.cpu().numpy() - w_dl) <= 1e-4 * np.abs(w_dl) + 1e-9)
    # the forward estimate with the same rows (sorted path: s1 computed here)
    assert_kde_close(index.query_with_neighbors(_dev(Y), _dev(nbr), m, seed=8).cpu().numpy(),
                     w_out)


@pytest.mark.parametrize("kernel,precision", [("gaussian", 1), ("exponential", 0),
                                              ("laplacian", 0), ("gaussian", 2)])
def test_grad_entry_point_matches_oracle(pkg, kernel, precision):
    """kde_grad (search + adjoint in one call, dlogh reduced on the device)
    against the oracle: the IVF search re-run from the exported index, then
    the pathwise gradient with those sets; dlogh is the sum over queries."""
    X, Y, _ = workloads.mixture_iso(n=6000, d=24, nq=70)
    h = 3.0 if kernel != "laplacian" else 12.0
    k, m, P = 40, 300, 3
    index = pkg.KDEIndex(_dev(X), kernel, h, nlist=16, seed=2)
    C, assign = (a.numpy() for a in index.export_ivf())
    rng = np.random.default_rng(8)
    gout = rng.uniform(0.5, 2.0, size=Y.shape[0]).astype(np.float32)
    dY, dl = index.grad(_dev(Y), k, m, nprobe=P, seed=4, gout=_dev(gout), precision=precision,
                        qid_offset=11)
    _, nbr, d2 = oracle.ivf_search(X, C, assign, Y, P, k)
    got_nbr = index.query(_dev(Y), k, m, nprobe=P, seed=4, precision=precision,
                          return_neighbors=True)[1].cpu().numpy()
    assert_neighbours_match(X, Y, got_nbr, nbr, d2)
    # the oracle's gradient with the GPU's sets (equal up to distance ties)
    w_out, w_dY, w_dl = oracle.deann_grad(X, Y, kernel, h, got_nbr, m, 4, qid_offset=11,
                                          gout=gout)
    dY = dY.cpu().numpy().astype(np.float64)
    for q in range(Y.shape[0]):
        assert np.linalg.norm(dY[q] - w_dY[q]) <= 1e-4 * np.linalg.norm(w_dY[q]) + 1e-9
    assert dl.dim() == 0
    assert math.isclose(dl.item(), w_dl.sum(), rel_tol=1e-4, abs_tol=1e-9)
    # host pointers give the same result
    dYh, dlh = index.grad(torch.from_numpy(Y), k, m, nprobe=P, seed=4,
                          gout=torch.from_numpy(gout), precision=precision, qid_offset=11)
    assert np.array_equal(dYh.numpy(), dY.astype(np.float32))
    assert dlh.item() == dl.item()
    # an empty batch has dlogh = 0
    dY0, dl0 = index.grad(_dev(Y[:0]), k, m, nprobe=P)
    assert dY0.shape == (0, X.shape[1]) and dl0.item() == 0.0


def test_grad_entry_point_k0_is_the_rs_gradient(pkg):
    X, Y = _data(1500, 8, 20, seed=12)
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.5, nlist=4)
    dY, dl = index.grad(_dev(Y), 0, 500, seed=3)
    _, w_dY, w_dl = oracle.deann_grad(X, Y, "gaussian", 1.5, None, 500, 3)
    assert np.allclose(dY.cpu().numpy(), w_dY, rtol=1e-4, atol=1e-4 * np.abs(w_dY).max())
    assert math.isclose(dl.item(), w_dl.sum(), rel_tol=1e-4)


def test_autograd_function(pkg):
    X, Y, _ = workloads.mixture_aniso(n=4000, d=64, nq=32)
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0, nlist=8)
    Yt = _dev(Y).requires_grad_(True)
    log_h = torch.zeros((), device="cuda", requires_grad=True)
    out = pkg.DeannKDE.apply(Yt, log_h, index, 20, 200, 3, 5)
    out.sum().backward()
    nbr = index.search(_dev(Y), 20, nprobe=3)[0].cpu().numpy()
    _, w_dY, w_dl = oracle.deann_grad(X, Y, "gaussian", 1.0, nbr, 200, 5)
    assert np.allclose(Yt.grad.cpu().numpy(), w_dY, rtol=1e-4, atol=1e-4 * np.abs(w_dY).max())
    assert math.isclose(log_h.grad.item(), w_dl.sum(), rel_tol=1e-4)
    # the backward pass used the forward's neighbour sets: the same gradient
    # as the adjoint given the neighbour ids the forward returned
    _, nbr_fwd = index.query(_dev(Y), 20, 200, nprobe=3, seed=5, return_neighbors=True)
    _, dY2, _ = index.grad_with_neighbors(_dev(Y), nbr_fwd, 200, seed=5)
    assert np.array_equal(Yt.grad.cpu().numpy(), dY2.cpu().numpy())


# --------------------------------------------------------------- edge cases --
def test_empty_batch_and_argument_errors(pkg):
    X, Y = _data(100, 4, 5)
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0)
    assert index.query(_dev(Y[:0]), 5, 10).numel() == 0
    with pytest.raises(pkg.KDEError, match="EINVAL"):
        index.query(_dev(Y), 101, 10)
    with pytest.raises(pkg.KDEError, match="EINVAL"):
        index.query(_dev(Y), 5, 10, nprobe=2)
    with pytest.raises(pkg.KDEError, match="EINVAL"):
        index.query(_dev(Y), 0, 0)


def test_bad_neighbour_id_reported(pkg):
    X, Y = _data(100, 4, 3)
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0)
    nbr = np.array([[1, 2], [3, 100], [4, 5]], np.int32)
    with pytest.raises(pkg.KDEError, match="EINVAL"):
        index.query_with_neighbors(torch.from_numpy(Y), torch.from_numpy(nbr), 10)
    # the device path flags it asynchronously; kde_sync reports it
    out = index.query_with_neighbors(_dev(Y), _dev(nbr), 10)
    with pytest.raises(pkg.KDEError, match="EINVAL"):
        index.sync()
    assert np.isnan(out.cpu().numpy()[1])
    index.sync()  # cleared


def test_draw_cap_reported(pkg):
    """k' = n - 1 of n = 1000 and m = 10 needs ~10^4 draws, above 64 m + 4096:
    the bounded draw loop gives up with KDE_ELIMIT (no hang)."""
    X, Y = _data(1000, 2, 2)
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0)
    nbr = np.tile(np.arange(999, dtype=np.int32), (2, 1))
    with pytest.raises(pkg.KDEError, match="ELIMIT"):
        index.query_with_neighbors(torch.from_numpy(Y), torch.from_numpy(nbr), 10)


# ------------------------------------------------------ bandwidth fitting ---
@pytest.mark.parametrize("kernel", ["gaussian", "exponential", "laplacian"])
def test_fit_bandwidth_matches_oracle_trace(pkg, kernel):
    """The library's gradient-ascent loop on the leave-one-out likelihood
    follows the oracle's trace step by step, given the same X_1 rows."""
    X, _, _ = workloads.mixture_iso(n=4000, d=8, nq=1)
    zid = np.arange(0, 4000, 17, dtype=np.int32)
    h0 = {"gaussian": 1.0, "exponential": 1.0, "laplacian": 3.0}[kernel]
    index = pkg.KDEIndex(_dev(X), kernel, h0, nlist=16, seed=2)
    ht, lt, nb = index.fit_bandwidth(zid, 30, 300, nprobe=4, seed=5, iters=8, lr=0.3)
    assert np.all(nb[:, 0] == zid)
    wh, wl = oracle.fit_bandwidth(X, zid, kernel, h0, nb, 300, 5, 8, 0.3)
    # FP32 estimates against FP64: each step moves log h by lr * g, and g
    # carries about 1e-6 relative error
    assert np.allclose(ht, wh, rtol=1e-4)
    assert np.allclose(lt, wl, rtol=1e-5, atol=1e-5)
    assert index.h == pytest.approx(float(ht[-1]))


def test_fit_bandwidth_reaches_exact_optimum(pkg):
    """Run to convergence, the fitted h lies at the exact leave-one-out
    maximiser (the oracle's exact l(h) on a grid)."""
    X, _, _ = workloads.mixture_iso(n=3000, d=4, nq=1)
    zid = np.arange(0, 3000, 10, dtype=np.int32)
    index = pkg.KDEIndex(_dev(X), "gaussian", 0.5, nlist=8, seed=3)
    ht, _, _ = index.fit_bandwidth(zid, 100, 2000, nprobe=8, seed=1, iters=60, lr=0.4)
    hs = np.exp(np.linspace(np.log(0.2), np.log(3.0), 120))
    ll = [oracle.loo_exact(X, zid, "gaussian", h)[0] for h in hs]
    h_star = hs[int(np.argmax(ll))]
    assert abs(np.log(np.mean(ht[-10:]) / h_star)) < 0.05


def test_fit_bandwidth_argument_errors(pkg):
    X, _, _ = workloads.mixture_iso(n=500, d=4, nq=1)
    index = pkg.KDEIndex(_dev(X), "gaussian", 1.0)
    with pytest.raises(pkg.KDEError):
        index.fit_bandwidth(np.array([0, 500], np.int32), 5, 10)   # id out of range
    with pytest.raises(pkg.KDEError):
        index.fit_bandwidth(np.array([0, 1], np.int32), 2048, 10)  # k > 2047
    with pytest.raises(pkg.KDEError):
        index.fit_bandwidth(np.array([0, 1], np.int32), 5, 10, sample_mode=2)


def test_scan_tile_changes_speed_only(pkg):
    """The tensor-core scan's query tile (kde_set_scan_tile) changes how the
    probing queries are grouped, not a single distance: estimates, neighbour
    sets and distances are the same bits for every tile, and the tuner keeps
    one of the tiles it timed.  Bad tiles and the FP32 scan are refused."""
    X, Y, _ = workloads.mixture_embed(n=20_000, nq=700, n_centres=40)
    index = pkg.KDEIndex(_dev(X), "gaussian", 6.0, nlist=16, seed=3)
    Yd = _dev(Y)
    for prec in (1, 2):
        want = index.query(Yd, 60, 500, nprobe=3, seed=4, precision=prec)
        wn, wd = index.search(Yd, 30, nprobe=3, precision=prec)
        for tile in (16, 48, 128):
            index.set_scan_tile(prec, tile)
            assert torch.equal(index.query(Yd, 60, 500, nprobe=3, seed=4, precision=prec), want)
            gn, gd = index.search(Yd, 30, nprobe=3, precision=prec)
            assert torch.equal(gn, wn) and torch.equal(gd, wd)
        times, best = index.tune_scan_tile(Yd, 60, 500, 3, prec, tiles=(0, 64, 32), reps=1)
        assert set(times) == {0, 64, 32} and best in times
        assert torch.equal(index.query(Yd, 60, 500, nprobe=3, seed=4, precision=prec), want)
        index.set_scan_tile(prec, 0)
    for prec, tile in ((0, 64), (1, 40), (2, 144), (1, -16)):
        with pytest.raises(pkg.KDEError):
            index.set_scan_tile(prec, tile)


@pytest.mark.parametrize("which,kernel,precision", [("iso16", "gaussian", 2),
                                                    ("embed128", "exponential", 1),
                                                    ("iso40", "laplacian", 0)])
def test_phased_estimator_matches_oracle(pkg, which, kernel, precision):
    """kde_query's phased order (kde_set_phase_window): every query's draws
    sorted by the window of X they fall in and gathered window by window.  A
    window of a small fraction of X forces 7-10 windows of a power of two of
    rows here, the last one shorter (57 of 2,048 rows with d = 40).  Against the FP64 oracle on the same neighbours and
    Philox draws, and against the per-query gathers (only the order of the
    sample sum's terms differs); two phased calls give the same bits."""
    if which == "iso16":
        X, Y, _ = workloads.mixture_iso(n=20_000, d=16, nq=300)
        h, window, m = 2.0, 131_072, 700
    elif which == "embed128":
        X, Y, _ = workloads.mixture_embed(n=9_000, nq=300, n_centres=30)
        h, window, m = 6.0, 600_000, 1000
    else:
        X, Y, _ = workloads.mixture_iso(n=12_345, d=40, nq=280)
        h, window, m = 9.0, 330_000, 700
    index = pkg.KDEIndex(_dev(X), kernel, h, nlist=12, seed=2)
    Yd = _dev(Y)
    index.set_phase_window(0)
    direct = index.query(Yd, 60, m, nprobe=3, seed=5, precision=precision).cpu().numpy()
    index.set_phase_window(window)
    out, nb = index.query(Yd, 60, m, nprobe=3, seed=5, precision=precision,
                          return_neighbors=True)
    again = index.query(Yd, 60, m, nprobe=3, seed=5, precision=precision)
    assert torch.equal(out, again)
    out = out.cpu().numpy()
    assert_kde_close(out, direct)
    assert_kde_close(out, oracle.deann(X, Y, kernel, h, nb.cpu().numpy(), m, 5))
    with pytest.raises(pkg.KDEError):
        index.set_phase_window(-1)


def test_phased_estimator_whole_dataset_as_neighbours(pkg):
    """k = n with the phased order on: no query samples (k' = n), every run
    is empty and the estimate is s1 / n, the exact KDE."""
    X, Y = _data(1500, 16, 260, seed=12)
    index = pkg.KDEIndex(_dev(X), "gaussian", 2.5, nlist=4)
    index.set_phase_window(16_384)
    out = index.query(_dev(Y), 1500, 400, nprobe=4, seed=0).cpu().numpy()
    assert_kde_close(out, oracle.exact(X, Y, "gaussian", 2.5))
