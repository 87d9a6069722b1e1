"""The seeded synthetic inputs follow their stated recipes (CPU only, reduced
sizes): shapes and seeds, the sparse data's zero fraction and Beta(2, 5)
nonzeros, unit norms, the share of uniform queries inside the bounding box,
the power-law construction's distances, and the uneven batch sizes."""
import numpy as np

import workloads


def test_seeds_make_the_inputs_reproducible():
    a = workloads.mixture_iso(n=500, d=4, nq=20)
    b = workloads.mixture_iso(n=500, d=4, nq=20)
    for u, v in zip(a, b):
        assert u.dtype == np.float32 and np.array_equal(u, v)
    # test and validation queries come from their own streams
    assert not np.array_equal(a[1], a[2][:20])


def test_mixture_iso_centres_and_spread():
    X, _, _ = workloads.mixture_iso(n=20_000, d=16, nq=10, n_centres=10)
    rng = np.random.default_rng(1001)
    centres = 4.0 * rng.standard_normal((10, 16))
    d2 = ((X[:, None, :].astype(np.float64) - centres[None]) ** 2).sum(2)
    resid = np.sqrt(d2.min(1))
    # sigma = 1 in 16 dimensions: distance to the own centre ~ sqrt(16)
    assert abs(np.mean(resid ** 2) / 16.0 - 1.0) < 0.05


def test_sparse_image_zero_fraction_and_values():
    X, Y, _ = workloads.sparse_image(n=20_000, nq=100)
    assert X.shape == (20_000, 784)
    nz = X[X != 0]
    assert abs((X == 0).mean() - 0.80) < 0.01       # masks with p in {0.05, 0.35}
    assert nz.min() > 0 and nz.max() < 1
    assert abs(nz.mean() - 2.0 / 7.0) < 0.005        # Beta(2, 5) mean
    assert abs(nz.var() - 10.0 / (49.0 * 8.0)) < 0.002  # Beta(2, 5) variance


def test_unit_powerlaw_is_unit_norm_with_decaying_spectrum():
    X, Y, _ = workloads.unit_powerlaw(n=20_000, nq=200, n_centres=100)
    assert X.shape == (20_000, 300)
    assert np.allclose(np.linalg.norm(X, axis=1), 1.0, atol=1e-5)
    assert np.allclose(np.linalg.norm(Y, axis=1), 1.0, atol=1e-5)
    var = X.astype(np.float64).var(0)
    assert var[:10].mean() > 20 * var[-50:].mean()   # variance along i ~ 1/i


def test_mixture_embed_uniform_queries_in_the_box():
    X, Y, _ = workloads.mixture_embed(n=20_000, nq=1_000, n_centres=50)
    lo, hi = X.min(0), X.max(0)
    # 10 % of the queries are uniform in the box: far from every centre
    rng = np.random.default_rng(1002)
    centres = 3.0 * rng.standard_normal((50, 128))
    d = np.sqrt(((Y[:, None, :].astype(np.float64) - centres[None]) ** 2).sum(2)).min(1)
    far = d > 30.0                                    # mixture points lie ~ sigma sqrt(128) <= 17
    assert abs(far.mean() - 0.10) < 0.02
    inside = (Y[far] >= lo) & (Y[far] <= hi)
    assert inside.all()


def test_powerlaw_construction_distances():
    X, y, h = workloads.powerlaw_nn(n=5_000, d=8, alpha=1.0, beta=0.5)
    i = np.arange(5_000)
    want = ((i + 1) / 5_000.0) ** 0.5
    got = ((X.astype(np.float64) - y) ** 2).sum(1)
    assert np.allclose(got, want, rtol=1e-5)
    assert np.isclose(h * h, 0.5 * 5_000 ** -0.5)


def test_uneven_batches():
    b = workloads.uneven_batches()
    assert b.size == 64 and b.sum() == 100_000
    assert b.min() == 16 and b.max() == 8192 and np.all((b >= 16) & (b <= 8192))
    small = workloads.uneven_batches(total=2_000, nbatch=8, lo=16, hi=800, seed=1)
    assert small.sum() == 2_000 and small.min() >= 16 and small.max() <= 800
