"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these tests touches the GPU library.  Each pin is chosen so that a
plausible slip in the oracle (a dropped term, a wrong sign or index, a wrong
norm, a missing rejection, k in place of k') fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from conftest import load_kat

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ----
def test_philox_known_answers():
    """Published Philox4x32-10 known-answer vectors (Salmon et al., SC'11)."""
    rows = load_kat(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = oracle.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == want


def test_draw_index_power_of_two_is_top_bits():
    """For n = 2^j the multiply-high mapping floor(u n / 2^64) keeps the top j
    bits of u, and u is built from the first two output words."""
    for j in (1, 5, 17, 30):
        for t in range(50):
            r = oracle.philox4x32_10([t, 7, 0, 0], [123, 0])
            u = (int(r[1]) << 32) | int(r[0])
            assert oracle.draw_index(123, 7, t, 1 << j) == u >> (64 - j)


def test_draw_index_range_and_uniformity():
    n = 10
    counts = np.zeros(n)
    for t in range(20000):
        i = oracle.draw_index(5, 3, t, n)
        assert 0 <= i < n
        counts[i] += 1
    chi2 = ((counts - 2000.0) ** 2 / 2000.0).sum()
    assert chi2 < 40.0  # 9 dof; p ~ 1e-5
    big = (1 << 31) - 1
    assert all(0 <= oracle.draw_index(9, 1, t, big) < big for t in range(200))
    assert all(oracle.draw_index(9, 1, t, 1) == 0 for t in range(20))


def test_streams_are_distinct():
    a = [oracle.draw_index(1, 0, t, 1 << 30) for t in range(64)]
    b = [oracle.draw_index(1, 1, t, 1 << 30) for t in range(64)]
    c = [oracle.draw_index(2, 0, t, 1 << 30) for t in range(64)]
    d = [oracle.draw_index(1, 0, t, 1 << 30, stream=1) for t in range(64)]
    assert len({tuple(a), tuple(b), tuple(c), tuple(d)}) == 4


# ---------------------------------------------------------------- kernels ---
def test_kernel_values_345_triangle():
    """x - y = (3, 4): Euclidean distance 5, L1 distance 7."""
    y = np.array([0.5, -1.0, 2.0], np.float32)
    x = y + np.array([3.0, 4.0, 0.0], np.float32)
    h = 2.0
    assert math.isclose(oracle.kernel_value("gaussian", x, y, h), math.exp(-25 / 8), rel_tol=1e-12)
    assert math.isclose(oracle.kernel_value("exponential", x, y, h), math.exp(-2.5), rel_tol=1e-12)
    assert math.isclose(oracle.kernel_value("laplacian", x, y, h), math.exp(-3.5), rel_tol=1e-12)


def _powerlaw_dataset(n, d, alpha, beta, seed=0):
    """Points whose squared distances to y are alpha ((i+1)/n)^beta along random
    directions (Lemma NN-contribution, Section 3.3)."""
    rng = np.random.default_rng(seed)
    y = rng.standard_normal(d)
    dirs = rng.standard_normal((n, d))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    r = np.sqrt(alpha * ((np.arange(n) + 1.0) / n) ** beta)
    X = y + r[:, None] * dirs
    return X, y


def test_exact_powerlaw_closed_form():
    """With h^2 = (alpha/2) n^-beta the i-th nearest point contributes
    exp(-(i+1)^beta) (proof of Lemma NN-contribution)."""
    n, d, alpha, beta = 400, 6, 3.0, 0.5
    X, y = _powerlaw_dataset(n, d, alpha, beta)
    # keep everything in float64 -> float32 consistently: use the float32 points
    X32, y32 = X.astype(np.float32), y.astype(np.float32)
    h = math.sqrt(alpha / 2 * n ** (-beta))
    got = oracle.exact(X32, y32[None], "gaussian", h)[0]
    # distances of the float32 points, computed independently
    d2 = ((X32.astype(np.float64) - y32.astype(np.float64)) ** 2).sum(1)
    want_rounded = np.exp(-d2 / (2 * h * h)).mean()
    want_closed = np.mean(np.exp(-((np.arange(n) + 1.0) ** beta)))
    assert math.isclose(got, want_rounded, rel_tol=1e-12)
    assert math.isclose(got, want_closed, rel_tol=1e-5)


def test_exact_limits():
    """h -> infinity: every summand -> 1; h -> 0: only points at distance 0."""
    rng = np.random.default_rng(1)
    X = rng.standard_normal((300, 5)).astype(np.float32)
    Y = np.concatenate([X[:3], rng.standard_normal((2, 5)).astype(np.float32)])
    for kern in ("gaussian", "exponential", "laplacian"):
        big = oracle.exact(X, Y, kern, 1e9)
        assert np.all(np.abs(big - 1.0) < 1e-7)
        small = oracle.exact(X, Y, kern, 1e-4)
        assert np.allclose(small[:3], 1.0 / 300, rtol=1e-12)
        assert np.all(small[3:] < 1e-300)


@pytest.mark.parametrize("kern,metric", [("gaussian", "euclidean"),
                                         ("exponential", "euclidean"),
                                         ("exponential", "manhattan")])
def test_exact_matches_sklearn_kde_ratios(kern, metric):
    """scikit-learn's KernelDensity (exact tree evaluation, zero tolerances)
    agrees up to its normalising constant: compare ratios between queries."""
    sk = pytest.importorskip("sklearn.neighbors")
    rng = np.random.default_rng(2)
    X = rng.standard_normal((500, 4)).astype(np.float32)
    Y = rng.standard_normal((6, 4)).astype(np.float32)
    h = 0.8
    ours_kern = "laplacian" if metric == "manhattan" else kern
    ours = oracle.exact(X, Y, ours_kern, h)
    kde = sk.KernelDensity(kernel=kern, bandwidth=h, metric=metric, algorithm="kd_tree",
                           atol=0.0, rtol=0.0).fit(X.astype(np.float64))
    ls = kde.score_samples(Y.astype(np.float64))
    assert np.allclose(np.log(ours) - np.log(ours[0]), ls - ls[0], atol=1e-9)


def test_exact_values_in_unit_interval():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((200, 7)).astype(np.float32)
    Y = rng.standard_normal((20, 7)).astype(np.float32) * 2
    for kern in ("gaussian", "exponential", "laplacian"):
        v = oracle.exact(X, Y, kern, 1.3)
        assert np.all((v >= 0) & (v <= 1))


# -------------------------------------------------------------- neighbours --
def _cdist2(A, B):
    from scipy.spatial.distance import cdist
    return cdist(A.astype(np.float64), B.astype(np.float64), "sqeuclidean")


def test_knn_matches_library_sort():
    rng = np.random.default_rng(4)
    X = rng.integers(-3, 4, size=(400, 3)).astype(np.float32)   # many exact ties
    Y = rng.integers(-3, 4, size=(25, 3)).astype(np.float32)
    k = 37
    nbr, d2 = oracle.knn(X, Y, k)
    D = _cdist2(Y, X)
    for q in range(Y.shape[0]):
        order = np.lexsort((np.arange(X.shape[0]), D[q]))[:k]
        assert np.array_equal(nbr[q], order)
        assert np.allclose(d2[q], D[q, order], rtol=0, atol=1e-9)


def test_knn_pads_when_k_exceeds_n():
    X = np.eye(3, dtype=np.float32)
    nbr, d2 = oracle.knn(X, X[:1], 5)
    assert list(nbr[0, 3:]) == [-1, -1] and np.all(np.isinf(d2[0, 3:]))


def test_nearest_centroid_matches_library_argmin():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((500, 6)).astype(np.float32)
    C = rng.standard_normal((17, 6)).astype(np.float32)
    a, _ = oracle.nearest_centroid(X, C)
    assert np.array_equal(a, np.argmin(_cdist2(X, C), axis=1))


def _first_distinct_draws(seed, n, L):
    """Initial k-means points from the Philox block itself (the known-answer
    pinned function): draw t of stream 1, query id 0, index floor(u n / 2^64)."""
    ids, seen, t = [], set(), 0
    while len(ids) < L:
        r = oracle.philox4x32_10([t, 0, 0, 1], [seed & 0xffffffff, seed >> 32])
        u = (int(r[1]) << 32) | int(r[0])
        i = (u * n) >> 64
        t += 1
        if i not in seen:
            seen.add(i)
            ids.append(i)
    return np.array(ids)


def test_kmeans_initial_points_are_the_first_distinct_draws():
    X = np.random.default_rng(30).standard_normal((97, 3)).astype(np.float32)
    for seed, L in ((1, 7), (2 ** 40 + 5, 30), (9, 97)):
        C0, _, _, st = oracle.kmeans(X, L, seed, iters=0)
        assert st == oracle.OK
        assert np.array_equal(C0, X[_first_distinct_draws(seed, 97, L)])


@pytest.mark.parametrize("L", [6, 12])
def test_kmeans_matches_sklearn_lloyd(L):
    """From the same initial centroids, the iterations are Lloyd's algorithm:
    scikit-learn's KMeans (algorithm="lloyd", one run, the same number of
    iterations) ends with the same labels and centroids."""
    sklearn_cluster = pytest.importorskip("sklearn.cluster")
    rng = np.random.default_rng(31)
    centres = rng.standard_normal((6, 8)) * 5.0
    X = (centres[rng.integers(0, 6, 3000)] + rng.standard_normal((3000, 8))).astype(np.float32)
    C0, _, _, _ = oracle.kmeans(X, L, 4, iters=0)
    C, a, _, _ = oracle.kmeans(X, L, 4, iters=20)
    assert np.bincount(a, minlength=L).min() > 0  # no empty list: plain Lloyd
    km = sklearn_cluster.KMeans(n_clusters=L, init=C0.astype(np.float64), n_init=1, max_iter=20,
                                tol=0.0, algorithm="lloyd").fit(X.astype(np.float64))
    assert np.array_equal(km.labels_, a)
    assert np.allclose(km.cluster_centers_, C, atol=1e-5)


def test_kmeans_objective_never_increases():
    rng = np.random.default_rng(32)
    X = rng.standard_normal((4000, 10)).astype(np.float32) * rng.uniform(0.5, 3.0, 10)
    _, _, obj, _ = oracle.kmeans(X, 40, 5, iters=25)
    assert np.all(np.diff(obj) <= 1e-6 * obj[:-1])
    assert obj[-1] < 0.8 * obj[0]


def test_kmeans_one_point_per_list():
    X = np.random.default_rng(33).standard_normal((50, 4)).astype(np.float32)
    C, a, obj, _ = oracle.kmeans(X, 50, 6, iters=3)
    assert obj[0] == 0.0 and obj[-1] == 0.0
    assert np.array_equal(C[a], X) and np.unique(a).size == 50


def test_kmeans_reseeds_an_empty_list_with_the_farthest_point():
    """Initial points at the same place leave a list empty (its twin with the
    lower id takes every point); the list then takes the point farthest from
    its centroid, and no list stays empty."""
    base = np.array([[0, 0], [10, 0], [0, 10]], dtype=np.float32)
    X = np.repeat(base, 20, axis=0)
    X = np.vstack([X, [[40.0, 40.0]]]).astype(np.float32)  # row 60: the outlier
    n = X.shape[0]
    for seed in range(200):
        ids = _first_distinct_draws(seed, n, 4)
        if len({tuple(X[i]) for i in ids}) == 3 and 60 not in ids:
            break
    else:
        pytest.fail("no seed with a repeated initial place")
    C, a, obj, _ = oracle.kmeans(X, 4, seed, iters=5)
    assert np.bincount(a, minlength=4).min() > 0
    assert np.sum(a == a[60]) == 1 and np.array_equal(C[a[60]], X[60])
    assert obj[-1] == 0.0


def test_ivf_full_probe_equals_brute_force():
    """nprobe = nlist scans every list: the IVF search is the exact kNN."""
    rng = np.random.default_rng(6)
    X = rng.standard_normal((600, 5)).astype(np.float32)
    C = rng.standard_normal((12, 5)).astype(np.float32)
    assign, _ = oracle.nearest_centroid(X, C)
    Y = rng.standard_normal((30, 5)).astype(np.float32)
    _, nbr, d2 = oracle.ivf_search(X, C, assign, Y, 12, 20)
    nb, db = oracle.knn(X, Y, 20)
    assert np.array_equal(nbr, nb) and np.allclose(d2, db)


def test_ivf_partial_probe_brute_force():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((300, 4)).astype(np.float32)
    C = rng.standard_normal((10, 4)).astype(np.float32)
    assign = rng.integers(0, 10, size=300).astype(np.int32)   # any list layout
    Y = rng.standard_normal((15, 4)).astype(np.float32)
    P, k = 3, 25
    probes, nbr, d2 = oracle.ivf_search(X, C, assign, Y, P, k)
    DC, DX = _cdist2(Y, C), _cdist2(Y, X)
    for q in range(15):
        pq = np.lexsort((np.arange(10), DC[q]))[:P]
        assert np.array_equal(probes[q], pq)
        cand = np.flatnonzero(np.isin(assign, pq))
        order = cand[np.lexsort((cand, DX[q, cand]))]
        want = np.full(k, -1)
        want[: min(k, order.size)] = order[:k]
        assert np.array_equal(nbr[q], want)


# --------------------------------------------------------------- DEANN -------
def _small_problem(seed=8, n=150, d=3, nq=4):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32)
    Y = (0.5 * rng.standard_normal((nq, d))).astype(np.float32)
    return X, Y


def test_deann_full_neighbour_set_is_exact():
    """k' = n: X_2 is empty and Algorithm 1 returns KDE_X(y) (Lemma
    composition with B empty); duplicates and -1 padding do not count."""
    X, Y = _small_problem()
    n = X.shape[0]
    rng = np.random.default_rng(0)
    nbr = np.stack([np.concatenate([rng.permutation(n), [-1, 3, 3, -1]]) for _ in Y])
    for kern in ("gaussian", "exponential", "laplacian"):
        got = oracle.deann(X, Y, kern, 0.9, nbr, m=50, seed=1)
        assert np.allclose(got, oracle.exact(X, Y, kern, 0.9), rtol=1e-13, atol=0)


def test_deann_k0_is_rs():
    """k = 0: Algorithm 1 falls back to random sampling (Section 3.2)."""
    X, Y = _small_problem()
    a, sa = oracle.deann(X, Y, "gaussian", 0.7, None, m=64, seed=11, return_samples=True)
    b, sb = oracle.rs(X, Y, "gaussian", 0.7, m=64, seed=11, return_samples=True)
    assert np.array_equal(sa, sb) and np.allclose(a, b, rtol=1e-14)


def test_deann_m0_discards_far_points():
    """m = 0: only the neighbours' exact contribution, divided by n."""
    X, Y = _small_problem()
    n = X.shape[0]
    nbr, _ = oracle.knn(X, Y, 10)
    got = oracle.deann(X, Y, "exponential", 0.6, nbr, m=0, seed=3)
    for q in range(Y.shape[0]):
        sub = oracle.exact(X[nbr[q]], Y[q:q + 1], "exponential", 0.6)[0]
        assert math.isclose(got[q], sub * 10 / n, rel_tol=1e-13)


def test_deann_samples_avoid_neighbours_and_are_in_range():
    X, Y = _small_problem(n=60)
    nbr, _ = oracle.knn(X, Y, 20)
    _, S = oracle.deann(X, Y, "gaussian", 1.0, nbr, m=200, seed=5, return_samples=True)
    for q in range(Y.shape[0]):
        assert S[q].min() >= 0 and S[q].max() < 60
        assert not np.isin(S[q], nbr[q]).any()
        # accepted draws are the stream's draws with X_1 members removed, in order
        draws = [oracle.draw_index(5, q, t, 60) for t in range(2000)]
        kept = [i for i in draws if i not in set(nbr[q].tolist())][:200]
        assert np.array_equal(S[q], kept)


def test_deann_values_in_unit_interval():
    X, Y = _small_problem(n=120, d=4, nq=30)
    nbr, _ = oracle.knn(X, Y, 15)
    for kern in ("gaussian", "exponential", "laplacian"):
        v = oracle.deann(X, Y, kern, 0.5, nbr, m=40, seed=2)
        assert np.all((v >= 0) & (v <= 1))


def _unbiased_check(X, y, kern, h, nbr_row, m, mode=0, reps=10_000):
    Yrep = np.repeat(y[None], reps, axis=0)
    nbr = np.repeat(np.asarray(nbr_row, np.int32)[None], reps, axis=0)
    est = oracle.deann(X, Yrep, kern, h, nbr, m=m, seed=77, mode=mode)
    mu = oracle.exact(X, y[None], kern, h)[0]
    se = est.std(ddof=1) / math.sqrt(reps)
    return abs(est.mean() - mu), se, mu


@pytest.mark.parametrize("which", ["good", "random", "adversarial", "duplicates"])
@pytest.mark.parametrize("mode", [0, 1])
def test_deann_unbiased_for_any_neighbour_set(which, mode):
    """Corollary "unbiased": the mean over 10^4 independent streams is within
    5 standard errors of the exact KDE, however poor the neighbour set."""
    rng = np.random.default_rng(9)
    X = rng.standard_normal((200, 3)).astype(np.float32)
    y = np.zeros(3, np.float32)
    d2 = ((X.astype(np.float64) - y) ** 2).sum(1)
    k = 50
    if which == "good":
        row = np.argsort(d2)[:k]
    elif which == "random":
        row = rng.choice(200, k, replace=False)
    elif which == "adversarial":
        row = np.argsort(-d2)[:k]
    else:
        base = np.argsort(d2)[:30]
        row = np.concatenate([base, base[:15], [-1] * 5])
    err, se, mu = _unbiased_check(X, y, "gaussian", 0.8, row, m=8, mode=mode)
    assert err < 5 * se + 1e-15, (err, se, mu)


def test_missing_rejection_would_be_biased():
    """Sanity of the unbiasedness test: a sampler that ignores X_1 (k' not
    subtracted, draws from all of X) is detected as biased."""
    rng = np.random.default_rng(9)
    X = rng.standard_normal((200, 3)).astype(np.float32)
    y = np.zeros(3, np.float32)
    d2 = ((X.astype(np.float64) - y) ** 2).sum(1)
    row = np.argsort(d2)[:50]
    reps = 10_000
    Yrep = np.repeat(y[None], reps, axis=0)
    nbr = np.repeat(row[None].astype(np.int32), reps, axis=0)
    s1 = oracle.exact(X[row], y[None], "gaussian", 0.8)[0] * 50
    rs = oracle.rs(X, Yrep, "gaussian", 0.8, m=8, seed=77)
    wrong = (s1 + 150 * rs) / 200          # RS over all of X, scaled as if over X_2
    mu = oracle.exact(X, y[None], "gaussian", 0.8)[0]
    se = wrong.std(ddof=1) / math.sqrt(reps)
    assert abs(wrong.mean() - mu) > 5 * se
    good = oracle.deann(X, Yrep, "gaussian", 0.8, nbr, m=8, seed=77)
    assert abs(good.mean() - mu) < 5 * good.std(ddof=1) / math.sqrt(reps)


def test_deann_draw_cap():
    """k' = n - 1 of n = 1000 with m = 10 needs ~10^4 draws, above the cap
    64 m + 4096: the oracle reports the cap instead of looping."""
    rng = np.random.default_rng(0)
    X = rng.standard_normal((1000, 2)).astype(np.float32)
    nbr = np.arange(999, dtype=np.int32)[None]
    with pytest.raises(oracle.OracleError, match="cap"):
        oracle.deann(X, X[:1], "gaussian", 1.0, nbr, m=10, seed=0)


def test_deann_rejects_out_of_range_neighbour():
    X, Y = _small_problem()
    with pytest.raises(oracle.OracleError):
        oracle.deann(X, Y[:1], "gaussian", 1.0, np.array([[0, 150]]), m=4, seed=0)


def test_rs_chernoff_bound_on_worst_case_input():
    """Lemma RS proof: Pr[Z > (1+eps) mu] <= exp(-eps^2 m tau / 3).  Worst-case
    input (the tightness example after the proof): a tau fraction of X sits on
    y (kernel value 1), the rest far away (kernel value ~0)."""
    n, tau, m, eps = 1000, 0.05, 400, 0.5
    X = np.full((n, 2), 1e3, np.float32)
    X[: int(tau * n)] = 0.0
    reps = 4000
    Y = np.zeros((reps, 2), np.float32)
    est = oracle.rs(X, Y, "gaussian", 1.0, m=m, seed=21)
    mu = tau
    assert abs(est.mean() - mu) < 5 * est.std(ddof=1) / math.sqrt(reps)
    fail_hi = np.mean(est > (1 + eps) * mu)
    fail_lo = np.mean(est < (1 - eps) * mu)
    assert fail_hi <= math.exp(-eps * eps * m * tau / 3)
    assert fail_lo <= math.exp(-eps * eps * m * tau / 2)


# ------------------------------------------------------------- gradients ----
@pytest.mark.parametrize("kern", ["gaussian", "exponential", "laplacian"])
def test_gradient_matches_central_differences(kern):
    """Pathwise derivative with X_1 and S held fixed vs FP64 central finite
    differences of the same estimator (step 1e-3 h)."""
    rng = np.random.default_rng(12)
    X = rng.standard_normal((300, 4)).astype(np.float32)
    Y = (0.3 * rng.standard_normal((3, 4))).astype(np.float32)
    h = 0.9
    nbr, _ = oracle.knn(X, Y, 20)
    out, dY, dl = oracle.deann_grad(X, Y, kern, h, nbr, m=30, seed=4)
    assert np.allclose(out, oracle.deann(X, Y, kern, h, nbr, m=30, seed=4), rtol=1e-13)
    # step 1e-3 h; the Laplacian kernel has kinks where x_j = y_j, so it takes a
    # step small enough not to cross one
    step = 1e-3 * h if kern != "laplacian" else 1e-7 * h
    # derivative in y along each axis; the query is float32, so difference the
    # estimator through a float64 shift of the data instead (translation
    # invariance: K(x, y + e) = K(x - e, y)).
    for j in range(4):
        e = np.zeros(4)
        e[j] = step
        fp = _deann64(X, Y, kern, h, nbr, 30, 4, shift=e)
        fm = _deann64(X, Y, kern, h, nbr, 30, 4, shift=-e)
        fd = (fp - fm) / (2 * step)
        assert np.allclose(dY[:, j], fd, rtol=1e-3, atol=1e-6 * np.abs(dY).max())
    fp = _deann64(X, Y, kern, h * math.exp(1e-3), nbr, 30, 4)
    fm = _deann64(X, Y, kern, h * math.exp(-1e-3), nbr, 30, 4)
    assert np.allclose(dl, (fp - fm) / 2e-3, rtol=1e-3)


def _deann64(X, Y, kern, h, nbr, m, seed, shift=None):
    """The estimator in float64 for finite differences: same neighbour set and
    sample indices (taken from the oracle), values from numpy."""
    _, S = oracle.deann(X, Y, kern, h, nbr, m=m, seed=seed, return_samples=True)
    n = X.shape[0]
    out = np.zeros(Y.shape[0])
    for q in range(Y.shape[0]):
        y = Y[q].astype(np.float64) + (0 if shift is None else shift)
        def K(idx):
            diff = X[idx].astype(np.float64) - y
            if kern == "gaussian":
                return np.exp(-(diff ** 2).sum(1) / (2 * h * h))
            if kern == "exponential":
                return np.exp(-np.sqrt((diff ** 2).sum(1)) / h)
            return np.exp(-np.abs(diff).sum(1) / h)
        nb = np.unique(nbr[q][nbr[q] >= 0])
        out[q] = (K(nb).sum() + (n - nb.size) / m * K(S[q]).sum()) / n
    return out


def test_exact_gradient_symmetry_and_fd():
    """Symmetric dataset {+a, -a}: the density gradient vanishes at 0; and the
    exact gradient matches central differences elsewhere."""
    a = np.array([[1.0, 2.0, -0.5]], np.float32)
    X = np.concatenate([a, -a])
    g, _ = oracle.exact_grad(X, np.zeros((1, 3), np.float32), "gaussian", 1.1)
    assert np.allclose(g, 0, atol=1e-15)
    rng = np.random.default_rng(13)
    X = rng.standard_normal((100, 3)).astype(np.float32)
    y = np.array([[0.2, -0.1, 0.4]], np.float32)
    g, dl = oracle.exact_grad(X, y, "gaussian", 0.7)
    step = 1e-4
    for j in range(3):
        e = np.zeros(3, np.float32)
        e[j] = 1
        Xp = (X.astype(np.float64) - step * e).astype(np.float64)
        Xm = (X.astype(np.float64) + step * e).astype(np.float64)
        f = lambda Z: np.exp(-((Z - y.astype(np.float64)) ** 2).sum(1) / (2 * 0.49)).mean()
        assert math.isclose(g[0, j], (f(Xp) - f(Xm)) / (2 * step), rel_tol=1e-6)


# ----------------------------------------------------------- DEANNP / RSP ---
def test_deannp_full_window_is_exact():
    """m = n: the window covers every point once; the members of X_1 are
    dropped, so m' = n - k' and DEANNP returns the exact KDE for any
    permutation and starting index."""
    X, Y = _small_problem(n=90)
    nbr, _ = oracle.knn(X, Y, 12)
    perm = np.random.default_rng(1).permutation(90).astype(np.int32)
    out, ell = oracle.deannp(X, Y, "gaussian", 0.8, perm, nbr, m=90, ell0=37)
    assert ell == 37
    assert np.allclose(out, oracle.exact(X, Y, "gaussian", 0.8), rtol=1e-13)


def test_deannp_unbiased_over_all_permutations():
    """Brute force over every permutation of a 6-point dataset: with m > k'
    the window always keeps a point, and the mean of the DEANNP estimate over
    the uniform permutation is the exact KDE (each kept window is a uniform
    sample without replacement from X minus X_1)."""
    import itertools
    rng = np.random.default_rng(5)
    X = rng.standard_normal((6, 2)).astype(np.float32)
    Y = rng.standard_normal((1, 2)).astype(np.float32)
    nbr = np.array([[4, 1]], np.int32)
    vals = []
    for p in itertools.permutations(range(6)):
        out, _ = oracle.deannp(X, Y, "gaussian", 0.9, np.array(p, np.int32), nbr,
                               m=3, ell0=2)
        vals.append(out[0])
    assert math.isclose(np.mean(vals), oracle.exact(X, Y, "gaussian", 0.9)[0],
                        rel_tol=1e-12)
    # and the estimator is not trivially exact on each permutation
    assert np.std(vals) > 1e-3 * np.mean(vals)


def test_deannp_rejects_window_longer_than_n():
    X, Y = _small_problem(n=30, nq=2)
    perm = np.arange(30, dtype=np.int32)
    with pytest.raises(Exception):
        oracle.deannp(X, Y, "gaussian", 0.8, perm, None, m=31)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 100, 1000, 4097, 65536])
def test_feistel_perm_is_a_bijection(n):
    """The keyed Feistel permutation with cycle walking maps [0, n) onto
    itself one-to-one for any n, and different keys give different orders."""
    a = oracle.feistel_perm(11, n)
    assert a.min() >= 0 and a.max() < n
    assert np.array_equal(np.sort(a), np.arange(n))
    if n >= 100:
        b = oracle.feistel_perm(12, n)
        assert not np.array_equal(a, b)
        assert not np.array_equal(a, np.arange(n))


def test_feistel_perm_is_roughly_uniform():
    """Position of element 0 across keys is spread over [0, n) (a chi-square
    test on 8 bins over 4000 keys, n = 64)."""
    pos = np.array([np.where(oracle.feistel_perm(s, 64) == 0)[0][0] for s in range(4000)])
    counts = np.bincount(pos // 8, minlength=8)
    chi2 = ((counts - 500.0) ** 2 / 500.0).sum()
    assert chi2 < 30.0  # 7 dof: p ~ 1e-4


def test_rsp_consecutive_windows_cover_dataset():
    """RSP (Algorithm 2) with m | n: n/m consecutive calls for the same query
    read disjoint windows covering X, so their mean is the exact KDE, and the
    running index returns to its start."""
    X, Y = _small_problem(n=120, nq=1)
    perm = np.random.default_rng(2).permutation(120).astype(np.int32)
    Yrep = np.repeat(Y, 6, axis=0)
    out, ell = oracle.deannp(X, Yrep, "exponential", 0.5, perm, None, m=20, ell0=7)
    assert ell == 7
    assert math.isclose(out.mean(), oracle.exact(X, Y, "exponential", 0.5)[0], rel_tol=1e-13)


# ------------------------------------------------------ bandwidth fitting ---
def _mixture_2d(n=240, seed=21):
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((3, 2)) * 3.0
    X = (c[rng.integers(0, 3, n)] + rng.standard_normal((n, 2))).astype(np.float32)
    return X


def test_loo_shortcut_equals_deleting_the_point():
    """KDE_{-z}(z) = (n KDE(z) - 1) / (n - 1): recompute the KDE over X with z
    removed, for each kernel."""
    X = _mixture_2d(60)
    for kern in ("gaussian", "exponential", "laplacian"):
        full = oracle.exact(X, X[:7], kern, 0.9)
        for j in range(7):
            rest = np.delete(X, j, axis=0)
            loo = oracle.exact(rest, X[j:j + 1], kern, 0.9)[0]
            assert math.isclose((60 * full[j] - 1.0) / 59.0, loo, rel_tol=1e-12)


def test_loo_likelihood_is_the_normalised_gaussian_density():
    """For the Gaussian kernel l(h) - (d/2) log(2 pi) is the mean log of the
    textbook leave-one-out density (1/(n-1)) sum_{i != j} N(z_j; x_i, h^2 I)."""
    X = _mixture_2d(80)
    zid = np.arange(0, 80, 3, dtype=np.int32)
    h = 0.7
    ll, _, used = oracle.loo_exact(X, zid, "gaussian", h)
    assert used == zid.size
    Xd = X.astype(np.float64)
    logs = []
    for j in zid:
        d2 = ((np.delete(Xd, j, axis=0) - Xd[j]) ** 2).sum(1)
        p = np.exp(-d2 / (2 * h * h)).sum() / (79 * (2 * math.pi * h * h))
        logs.append(math.log(p))
    assert math.isclose(ll - math.log(2 * math.pi), np.mean(logs), rel_tol=1e-12, abs_tol=1e-12)


@pytest.mark.parametrize("kern", ["gaussian", "exponential", "laplacian"])
def test_loo_derivative_matches_central_differences(kern):
    X = _mixture_2d(120)
    zid = np.arange(0, 120, 2, dtype=np.int32)
    h, eps = 0.8, 1e-5
    _, dll, _ = oracle.loo_exact(X, zid, kern, h)
    lp, _, _ = oracle.loo_exact(X, zid, kern, h * math.exp(eps))
    lm, _, _ = oracle.loo_exact(X, zid, kern, h * math.exp(-eps))
    assert math.isclose(dll, (lp - lm) / (2 * eps), rel_tol=1e-6, abs_tol=1e-8)


def test_fit_with_all_points_as_neighbours_is_exact_and_converges():
    """X_1 = X makes the estimate exact: the first step follows the exact
    gradient, and the ascent ends at the maximiser of the exact l(h), found
    independently by golden-section search."""
    X = _mixture_2d(150)
    n = X.shape[0]
    zid = np.arange(0, n, 3, dtype=np.int32)
    nbr = np.tile(np.arange(n, dtype=np.int32), (zid.size, 1))
    h0, lr = 0.3, 0.5  # every training point keeps a held-out density for h >= 0.2
    ht, lt = oracle.fit_bandwidth(X, zid, "gaussian", h0, nbr, 50, 5, 40, lr)
    ll0, dll0, _ = oracle.loo_exact(X, zid, "gaussian", h0)
    assert math.isclose(lt[0], ll0, rel_tol=1e-12)
    assert math.isclose(ht[1], h0 * math.exp(lr * dll0), rel_tol=1e-12)
    f = lambda lh: -oracle.loo_exact(X, zid, "gaussian", math.exp(lh))[0]
    a, b = math.log(0.2), math.log(5.0)
    g = (math.sqrt(5) - 1) / 2
    for _ in range(80):
        c, d = b - g * (b - a), a + g * (b - a)
        if f(c) < f(d):
            b = d
        else:
            a = c
    h_star = math.exp((a + b) / 2)
    assert math.isclose(ht[-1], h_star, rel_tol=1e-3)
    assert np.all(np.diff(lt) > -1e-12)  # the likelihood never decreases on this path
    assert oracle.loo_exact(X, zid, "gaussian", 0.2)[2] == zid.size


def test_fit_with_sampling_tracks_the_exact_optimum():
    """With k near neighbours (plus the point itself) and m samples, the
    noisy ascent still settles near the exact maximiser."""
    X = _mixture_2d(600, seed=3)
    n = X.shape[0]
    zid = np.arange(0, n, 5, dtype=np.int32)
    nb, _ = oracle.knn(X, X[zid], 40)  # holds the point itself first
    ht, _ = oracle.fit_bandwidth(X, zid, "gaussian", 0.3, nb, 400, 9, 60, 0.5)
    f = lambda h: oracle.loo_exact(X, zid, "gaussian", h)[0]
    hs = np.exp(np.linspace(math.log(0.1), math.log(3.0), 200))
    h_star = hs[int(np.argmax([f(h) for h in hs]))]
    assert abs(math.log(np.mean(ht[-20:]) / h_star)) < 0.1


# ------------------------------------- nearest-neighbour contribution lemma ---
def _powerlaw(n=20_000, d=16):
    import workloads
    return workloads.powerlaw_nn(n=n, d=d)


def test_powerlaw_construction_gives_the_closed_form():
    """At y = 0 with h^2 = (alpha/2) n^-beta the Gaussian KDE is
    (1/n) sum_i exp(-(i + 1)^beta) (the Lemma's proof)."""
    X, y, h = _powerlaw()
    n = X.shape[0]
    want = np.exp(-np.sqrt(np.arange(n) + 1.0)).mean()
    assert math.isclose(oracle.exact(X, y[None], "gaussian", h)[0], want, rel_tol=1e-6)


def test_powerlaw_top_neighbours_dominate():
    """Lemma part (a): the first Theta(log^(1/beta) n) neighbours carry all but
    a vanishing part of the KDE; the fraction grows with the constant."""
    X, y, h = _powerlaw()
    n = X.shape[0]
    tot = oracle.exact(X, y[None], "gaussian", h)[0] * n
    fr = []
    for c in (0.5, 1.0, 2.0):
        k = int(math.ceil(c * math.log(n) ** 2))  # 1/beta = 2
        fr.append(oracle.exact(X[:k], y[None], "gaussian", h)[0] * k / tot)
    assert fr[0] > 0.99 and fr[1] > 0.999 and fr[2] > 0.99998
    assert fr[0] < fr[1] < fr[2] < 1.0


def test_powerlaw_bandwidth_limits():
    """Lemma part (b): h^2 <= (alpha/2) n^-beta / ln(1/tau) gives KDE <= tau.
    Part (c) as its proof derives it for K = exp(-r^2/(2h^2)): the AM-GM step
    bounds the KDE below by exp(-alpha/(2 beta h^2)), so
    h^2 >= alpha / (2 beta ln(1/(1 - delta))) gives KDE >= 1 - delta.  The
    printed condition h^2 >= ln(1/(1 - delta)) alpha/(2 beta) (logarithm in the
    numerator) does not: it fails here for delta = 0.1."""
    X, y, h = _powerlaw()
    n, alpha, beta = X.shape[0], 1.0, 0.5
    for tau in (0.1, 1e-2, 1e-4):
        hb = math.sqrt(alpha / 2 * n ** -beta / math.log(1 / tau))
        assert oracle.exact(X, y[None], "gaussian", hb)[0] <= tau
    for delta in (0.5, 0.1, 0.01):
        hc = math.sqrt(alpha / (2 * beta * math.log(1 / (1 - delta))))
        kde = oracle.exact(X, y[None], "gaussian", hc)[0]
        assert kde >= 1 - delta
        # the AM-GM bound itself
        assert kde >= math.exp(-alpha / (2 * beta * hc * hc)) - 1e-12
    printed = math.sqrt(math.log(1 / 0.9) * alpha / (2 * beta))
    assert oracle.exact(X, y[None], "gaussian", printed)[0] < 0.9


def test_deann_variance_formula_given_the_neighbours():
    """With X_1 fixed the estimate's variance is ((n - k)/n)^2 sigma^2 / m,
    sigma^2 the population variance of K over X minus X_1 (draws with
    repetition): 4,000 seeds against the formula (chi-square, 4,000 dof)."""
    X, y, h = _powerlaw(n=2000, d=8)
    n, k, m = 2000, 20, 50
    Kv = np.exp(-((X.astype(np.float64) - y) ** 2).sum(1) / (2 * h * h))
    rest = Kv[k:]
    var = ((n - k) / n) ** 2 * rest.var() / m
    Y = np.repeat(y[None], 4000, axis=0)
    nbr = np.tile(np.arange(k, dtype=np.int32), (4000, 1))
    est = oracle.deann(X, Y, "gaussian", h, nbr, m, 3)
    s2 = est.var(ddof=1)
    # 4,000 draws: s2 / var within +-8 % (about 5 standard errors of the
    # variance for the kurtosis of these kernel values)
    assert abs(s2 / var - 1) < 0.08
    assert math.isclose(est.mean(), Kv.mean(), rel_tol=6 * math.sqrt(var / 4000) / Kv.mean())


# ------------------------------------------------------------- mean shift ----
def _mixture_small(n=300, d=4, nq=6, seed=31):
    rng = np.random.default_rng(seed)
    centres = rng.normal(0.0, 3.0, (4, d))
    X = (centres[rng.integers(0, 4, n)] + rng.normal(0.0, 1.0, (n, d))).astype(np.float32)
    Y = (centres[rng.integers(0, 4, nq)] + rng.normal(0.0, 1.5, (nq, d))).astype(np.float32)
    return X, Y


def test_mean_shift_step_is_the_weighted_mean_of_neighbours_and_samples():
    """For the Gaussian kernel grad K = K (x - y) / h^2, so one step
    y + h^2 grad(est)/est lands on sum_i w_i K_i x_i / sum_i w_i K_i over X_1 and
    S, with w = 1/n on X_1 and (n - k')/(n m) per sample.  X_1 comes from the
    IVF search (pinned by brute force) and S from the stream (pinned by the
    published known answers); the weighted mean is formed here in numpy.  A
    dropped h^2, a wrong sign of the gradient or weights without the (n - k')
    factor each move the result off the weighted mean."""
    X, Y = _mixture_small()
    n = X.shape[0]
    C, assign, _, _ = oracle.kmeans(X, 8, seed=2)
    h, k, m, P, seed = 1.3, 20, 40, 3, 11
    moved, est = oracle.mean_shift(X, C, assign, Y, h, k, m, P, seed, steps=1, qid_offset=5)
    _, nbr, _ = oracle.ivf_search(X, C, assign, Y, P, k)
    _, S = oracle.deann(X, Y, "gaussian", h, nbr, m, seed, qid_offset=5, return_samples=True)
    X64 = X.astype(np.float64)
    for q in range(Y.shape[0]):
        ids = np.unique(nbr[q][nbr[q] >= 0])
        y = Y[q].astype(np.float64)
        K1 = np.exp(-((X64[ids] - y) ** 2).sum(1) / (2 * h * h))
        K2 = np.exp(-((X64[S[q]] - y) ** 2).sum(1) / (2 * h * h))
        w1, w2 = 1.0 / n, (n - ids.size) / (n * m)
        num = w1 * (K1[:, None] * X64[ids]).sum(0) + w2 * (K2[:, None] * X64[S[q]]).sum(0)
        den = w1 * K1.sum() + w2 * K2.sum()
        assert est[q] == pytest.approx(den, rel=1e-12)
        want = (num / den).astype(np.float32)
        assert np.allclose(moved[q], want, rtol=0, atol=2e-6 * (1 + np.abs(want).max()))
        assert np.abs(moved[q] - Y[q]).max() > 1e-3  # the step did move the query


def test_mean_shift_with_every_point_as_neighbour_is_the_textbook_step():
    """With one list and k = n the estimate is the exact KDE (no sampling),
    and a step is the classical Gaussian mean-shift update sum K x / sum K over
    all of X (Fukunaga-Hostetler; Comaniciu-Meer)."""
    X, Y = _mixture_small(n=120, nq=4, seed=5)
    n = X.shape[0]
    C = X.astype(np.float64).mean(0, keepdims=True).astype(np.float32)
    assign = np.zeros(n, dtype=np.int32)
    h = 2.0
    moved, _ = oracle.mean_shift(X, C, assign, Y, h, n, 50, 1, 3, steps=3)
    y = Y.astype(np.float64)
    X64 = X.astype(np.float64)
    for _ in range(3):
        K = np.exp(-((X64[None, :, :] - y[:, None, :]) ** 2).sum(2) / (2 * h * h))
        y = ((K @ X64) / K.sum(1, keepdims=True)).astype(np.float32).astype(np.float64)
    assert np.allclose(moved, y, rtol=0, atol=1e-5)


def test_mean_shift_converges_to_the_centre_of_a_symmetric_set():
    """Points c +- a e_j (j < d) are symmetric about c, so c is a stationary
    point of the KDE; with h well above a it is the only mode, and the exact
    (k = n) flow started anywhere nearby ends at c.  Started at c, it stays."""
    d, a, h = 3, 1.0, 2.5
    c = np.array([0.5, -1.25, 2.0])
    X = np.concatenate([c + a * np.eye(d), c - a * np.eye(d)]).astype(np.float32)
    n = X.shape[0]
    C = c[None, :].astype(np.float32)
    assign = np.zeros(n, dtype=np.int32)
    Y = np.array([c + [0.4, -0.3, 0.2], c - [0.5, 0.1, 0.6], c], dtype=np.float32)
    moved, _ = oracle.mean_shift(X, C, assign, Y, h, n, 10, 1, 0, steps=60)
    assert np.abs(moved - c).max() < 1e-5
    still, _ = oracle.mean_shift(X, C, assign, Y[2:], h, n, 10, 1, 0, steps=5)
    assert np.abs(still[0] - c).max() < 1e-6


def test_mean_shift_steps_redraw_with_seed_plus_step():
    """Two steps with seed s equal one step with seed s followed by one step
    with seed s + 1 from the moved queries (sets redrawn every step)."""
    X, Y = _mixture_small(seed=9)
    C, assign, _, _ = oracle.kmeans(X, 6, seed=1)
    args = (1.1, 15, 30, 2)
    two, _ = oracle.mean_shift(X, C, assign, Y, *args, 7, steps=2)
    one, _ = oracle.mean_shift(X, C, assign, Y, *args, 7, steps=1)
    again, _ = oracle.mean_shift(X, C, assign, one, *args, 8, steps=1)
    assert np.array_equal(two, again)
    other, _ = oracle.mean_shift(X, C, assign, one, *args, 7, steps=1)
    assert not np.array_equal(two, other)
