"""Seeded synthetic workloads for the DEANN query path.

This module only draws random inputs (datasets, query sets and batch sizes).
It holds none of the estimator's arithmetic, so both the GPU library's tests
and benchmark and the FP64 oracle may use it.

The paper's own datasets (ALOI, MNIST, SVHN, ...) are not available; these
generators stand in for them with the same kinds of shape:

* ``mixture_iso`` -- low-dimensional mixture of isotropic Gaussians (10
  centres ~ N(0, 16 I), sigma = 1), the low-d case.
* ``mixture_embed`` -- 1,000 centres ~ N(0, 9 I) in d = 128, per-cluster
  sigma ~ U[0.5, 1.5]; queries 90 % from the mixture, 10 % uniform in the
  dataset's bounding box.  Stands in for dense ~100-d embeddings.
* ``sparse_image`` -- d = 784 entries in [0, 1], about 80 % exact zeros:
  10 latent clusters, each with a per-coordinate Bernoulli mask probability
  drawn from {0.05, 0.35}, nonzeros ~ Beta(2, 5).  Stands in for 784-d
  image-like data.
* ``mixture_aniso`` -- 50 anisotropic Gaussians in d = 64, centres ~ N(0, 4 I),
  x = c_j + A_j z with A_j entries ~ N(0, 1/d).
* ``unit_powerlaw`` -- 5,000 centres ~ N(0, diag(i^-1)) in d = 300, points
  c_j + N(0, 0.25 diag(i^-1)), normalised to unit norm.

Seeds: data 1000 + cfg, test queries 2000 + cfg, validation queries 3000 + cfg.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    X: np.ndarray            # n x d float32 dataset
    Y: np.ndarray            # test queries, float32
    Yval: np.ndarray         # validation queries (bandwidth fitting / tuning)
    kernel: str
    h: float | None          # None: fit so that the mean exact KDE hits target_mu
    target_mu: float | None
    params: dict


def _mixture_iso(rng, n, d, centres, sigma):
    lab = rng.integers(0, centres.shape[0], size=n)
    return (centres[lab] + sigma * rng.standard_normal((n, d), dtype=np.float32)).astype(np.float32)


def mixture_iso(n=10_000, d=16, nq=1_000, n_centres=10, seed=1001):
    """Low-d mixture: centres ~ N(0, 16 I), sigma = 1, equal weights; queries from
    the same mixture."""
    rng = np.random.default_rng(seed)
    centres = (4.0 * rng.standard_normal((n_centres, d))).astype(np.float32)
    X = _mixture_iso(rng, n, d, centres, 1.0)
    qr = np.random.default_rng(seed + 1000)
    Y = _mixture_iso(qr, nq, d, centres, 1.0)
    vr = np.random.default_rng(seed + 2000)
    Yval = _mixture_iso(vr, nq, d, centres, 1.0)
    return X, Y, Yval


def _embed_points(rng, n, centres, sig, chunk=1 << 18):
    d = centres.shape[1]
    out = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        lab = rng.integers(0, centres.shape[0], size=e - s)
        z = rng.standard_normal((e - s, d), dtype=np.float32)
        out[s:e] = centres[lab] + sig[lab, None] * z
    return out


def _embed_queries(rng, nq, centres, sig, lo, hi):
    nmix = int(round(0.9 * nq))
    Ym = _embed_points(rng, nmix, centres, sig)
    Yu = (lo + (hi - lo) * rng.random((nq - nmix, centres.shape[1]), dtype=np.float32))
    Y = np.concatenate([Ym, Yu.astype(np.float32)], axis=0)
    return Y[rng.permutation(nq)]


def mixture_embed(n=1_000_000, d=128, nq=10_000, n_centres=1_000, seed=1002):
    """Dense-embedding stand-in: 1,000 centres ~ N(0, 9 I), per-cluster sigma ~
    U[0.5, 1.5]; queries 90 % mixture, 10 % uniform in the bounding box."""
    rng = np.random.default_rng(seed)
    centres = (3.0 * rng.standard_normal((n_centres, d))).astype(np.float32)
    sig = rng.uniform(0.5, 1.5, size=n_centres).astype(np.float32)
    X = _embed_points(rng, n, centres, sig)
    lo, hi = X.min(axis=0), X.max(axis=0)
    Y = _embed_queries(np.random.default_rng(seed + 1000), nq, centres, sig, lo, hi)
    Yval = _embed_queries(np.random.default_rng(seed + 2000), nq, centres, sig, lo, hi)
    return X, Y, Yval


def _sparse_points(rng, n, probs, chunk=1 << 16):
    d = probs.shape[1]
    out = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        lab = rng.integers(0, probs.shape[0], size=e - s)
        mask = rng.random((e - s, d), dtype=np.float32) < probs[lab]
        blk = np.zeros((e - s, d), dtype=np.float32)
        # Beta(2, 5) values are drawn for the nonzero entries only
        blk[mask] = rng.beta(2.0, 5.0, size=int(mask.sum())).astype(np.float32)
        out[s:e] = blk
    return out


def sparse_image(n=1_000_000, d=784, nq=10_000, n_clusters=10, seed=1003):
    """784-d image-like stand-in: per-cluster Bernoulli masks with coordinate
    probabilities drawn from {0.05, 0.35}, nonzeros ~ Beta(2, 5)."""
    rng = np.random.default_rng(seed)
    probs = np.where(rng.random((n_clusters, d)) < 0.5, 0.05, 0.35).astype(np.float32)
    X = _sparse_points(rng, n, probs)
    Y = _sparse_points(np.random.default_rng(seed + 1000), nq, probs)
    Yval = _sparse_points(np.random.default_rng(seed + 2000), nq, probs)
    return X, Y, Yval


def _aniso_points(rng, n, centres, A, chunk=1 << 16):
    d = centres.shape[1]
    out = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        lab = rng.integers(0, centres.shape[0], size=e - s)
        z = rng.standard_normal((e - s, d), dtype=np.float32)
        out[s:e] = centres[lab] + np.einsum("nij,nj->ni", A[lab], z)
    return out


def mixture_aniso(n=200_000, d=64, nq=50_000, n_clusters=50, seed=1004):
    """50 anisotropic Gaussians: centres ~ N(0, 4 I), x = c_j + A_j z,
    A_j entries ~ N(0, 1/d), z ~ N(0, I)."""
    rng = np.random.default_rng(seed)
    centres = (2.0 * rng.standard_normal((n_clusters, d))).astype(np.float32)
    A = (rng.standard_normal((n_clusters, d, d)) / np.sqrt(d)).astype(np.float32)
    X = _aniso_points(rng, n, centres, A)
    Y = _aniso_points(np.random.default_rng(seed + 1000), nq, centres, A)
    Yval = _aniso_points(np.random.default_rng(seed + 2000), nq, centres, A)
    return X, Y, Yval


def _unit_points(rng, n, centres, scale, chunk=1 << 17):
    d = centres.shape[1]
    out = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        lab = rng.integers(0, centres.shape[0], size=e - s)
        z = rng.standard_normal((e - s, d), dtype=np.float32)
        p = centres[lab] + 0.5 * scale * z
        p /= np.linalg.norm(p, axis=1, keepdims=True)
        out[s:e] = p
    return out


def unit_powerlaw(n=4_000_000, d=300, nq=100_000, n_centres=5_000, seed=1005):
    """Unit-norm power-law-spectrum mixture: centres ~ N(0, diag(i^-1)),
    points c_j + N(0, 0.25 diag(i^-1)), normalised to unit norm."""
    rng = np.random.default_rng(seed)
    scale = (1.0 / np.sqrt(np.arange(1, d + 1, dtype=np.float64))).astype(np.float32)
    centres = (rng.standard_normal((n_centres, d)).astype(np.float32) * scale)
    X = _unit_points(rng, n, centres, scale)
    Y = _unit_points(np.random.default_rng(seed + 1000), nq, centres, scale)
    Yval = _unit_points(np.random.default_rng(seed + 2000), nq, centres, scale)
    return X, Y, Yval


def powerlaw_nn(n=1_000_000, d=32, alpha=1.0, beta=0.5, seed=1006):
    """The construction of the Lemma on the contribution of nearest
    neighbours: around the query y = 0, point i (in index order) lies at squared
    distance alpha ((i + 1) / n)^beta in a uniformly random direction.  With
    h^2 = (alpha / 2) n^-beta its Gaussian kernel value is exp(-(i + 1)^beta).
    Returns (X [n x d] float32, y [d] float32, h)."""
    rng = np.random.default_rng(seed)
    r = np.sqrt(alpha * ((np.arange(n, dtype=np.float64) + 1.0) / n) ** beta)
    u = rng.standard_normal((n, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    X = (u * r[:, None]).astype(np.float32)
    h = float(np.sqrt(alpha / 2.0 * n ** (-beta)))
    return X, np.zeros(d, dtype=np.float32), h


def uneven_batches(total=100_000, nbatch=64, lo=16, hi=8192, seed=5005):
    """Batch sizes log-uniform in [lo, hi], forced to include lo and hi, adjusted
    to sum to ``total``."""
    rng = np.random.default_rng(seed)
    b = np.exp(rng.uniform(np.log(lo), np.log(hi), size=nbatch))
    b = np.clip(np.round(b), lo, hi).astype(np.int64)
    b[0], b[1] = lo, hi
    inner = np.arange(2, nbatch)
    for _ in range(10_000):
        diff = total - int(b.sum())
        if diff == 0:
            break
        j = inner[rng.integers(0, inner.size)]
        step = int(np.sign(diff)) * min(abs(diff), 64)
        b[j] = int(np.clip(b[j] + step, lo, hi))
    assert int(b.sum()) == total, "could not balance the batch sizes"
    return b


CONFIGS = {
    1: dict(name="mixture_iso n=10k d=16", gen=mixture_iso, kernel="gaussian", h=2.0,
            target_mu=None, k=50, m=500, nlist=1, nprobe=1),
    2: dict(name="mixture_embed n=1M d=128", gen=mixture_embed, kernel="gaussian", h=None,
            target_mu=1e-3, k=100, m=1000, nlist=1024, nprobe=16),
    3: dict(name="sparse_image n=1M d=784", gen=sparse_image, kernel="gaussian", h=None,
            target_mu=1e-4, k=200, m=2000, nlist=2048, nprobe=32),
    4: dict(name="mixture_aniso n=200k d=64", gen=mixture_aniso, kernel="gaussian", h=1.0,
            target_mu=None, k=100, m=1000, nlist=512, nprobe=8),
    5: dict(name="unit_powerlaw n=4M d=300", gen=unit_powerlaw, kernel="exponential",
            h=None, target_mu=1e-3, k=200, m=2000, nlist=4096, nprobe=16),
}


def make(cfg: int, scale: float = 1.0, nq: int | None = None, **over) -> Workload:
    """Build config ``cfg``; ``scale`` shrinks n (and the query count) for tests."""
    spec = dict(CONFIGS[cfg])
    spec.update(over)
    gen = spec.pop("gen")
    defaults = gen.__defaults__
    names = gen.__code__.co_varnames[: gen.__code__.co_argcount]
    kw = dict(zip(names, defaults))
    kw["n"] = max(64, int(kw["n"] * scale))
    if nq is not None:
        kw["nq"] = nq
    else:
        kw["nq"] = max(16, int(kw["nq"] * min(1.0, scale * 10)))
    X, Y, Yval = gen(**kw)
    return Workload(name=spec.pop("name"), X=X, Y=Y, Yval=Yval, kernel=spec.pop("kernel"),
                    h=spec.pop("h"), target_mu=spec.pop("target_mu"), params=spec)
