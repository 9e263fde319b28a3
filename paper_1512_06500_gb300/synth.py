"""Seeded synthetic workloads shaped like the face-recognition sets of Section 4.

This module only draws random inputs: class means, per-sample noise, clipping,
labels and held-out splits. It contains none of the discriminant-analysis
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

Layout: a sample set is returned as a C-contiguous float64 array of shape
(n, d). Read as a column-major d x n matrix with leading dimension d, this is
the paper's data matrix X = [chi_1 .. chi_n] (Section 1), one sample per
column, each sample contiguous in memory.

The face databases of Section 4 (AR, Yale, Extended YaleB, FERET, ORL,
CMU-PIE) are not available; these generators stand in for their shapes:
d pixels, k classes, n_j training images per class, t = k - 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """One synthetic EDA problem: training set, labels and a held-out split."""
    X: np.ndarray            # (n, d) float64, sample i = row i
    labels: np.ndarray       # (n,) int32 in [0, k)
    k: int
    Xtest: np.ndarray        # (m, d) float64
    ytest: np.ndarray        # (m,) int32
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return self.X.shape[1]

    @property
    def n(self) -> int:
        return self.X.shape[0]


def _labels(rng, counts, shuffle):
    lab = np.repeat(np.arange(len(counts), dtype=np.int32), counts)
    if shuffle:
        lab = lab[rng.permutation(lab.size)]
    return lab.astype(np.int32)


def gaussian_clusters(d, k, n_per_class, noise=0.3, seed=0, n_test_per_class=0,
                      shuffle=True, clip=True, name=""):
    """Class means m_j ~ N(0, 1) per pixel; samples m_j + N(0, noise^2), clipped to [0, 1].

    n_per_class is an int (balanced) or a length-k sequence (uneven classes).
    Labels are shuffled so that the input order is not class-major.
    """
    rng = np.random.default_rng(seed)
    counts = np.full(k, int(n_per_class)) if np.isscalar(n_per_class) else np.asarray(n_per_class, int)
    assert counts.shape == (k,) and counts.min() >= 1
    means = rng.standard_normal((k, d))
    lab = _labels(rng, counts, shuffle)
    X = means[lab] + noise * rng.standard_normal((lab.size, d))
    if clip:
        np.clip(X, 0.0, 1.0, out=X)
    tcounts = np.full(k, int(n_test_per_class))
    ylab = _labels(rng, tcounts, False)
    Xt = means[ylab] + noise * rng.standard_normal((ylab.size, d))
    if clip:
        np.clip(Xt, 0.0, 1.0, out=Xt)
    return Problem(np.ascontiguousarray(X), lab, k, np.ascontiguousarray(Xt), ylab, name,
                   {"generator": "gaussian_clusters", "noise": noise, "seed": seed})


def dct_basis(side, modes):
    """Orthonormal 2-D DCT-II images of a side x side grid, lowest frequencies first.

    Frequencies (u, v) are ordered by u + v, then u. Returns (side*side, modes).
    """
    x = np.arange(side)
    def c1(u):
        s = np.sqrt((1.0 if u == 0 else 2.0) / side)
        return s * np.cos(np.pi * (x + 0.5) * u / side)
    pairs = sorted(((u, v) for u in range(side) for v in range(side) if u + v < 2 * modes + 2),
                   key=lambda p: (p[0] + p[1], p[0]))[:modes]
    B = np.empty((side * side, modes))
    for i, (u, v) in enumerate(pairs):
        B[:, i] = np.outer(c1(u), c1(v)).ravel()
    return B


def lowrank_images(d, k, n_per_class, rank=20, noise=0.05, seed=0, n_test_per_class=0, shuffle=True, name=""):
    """Smooth low-rank class means 0.5 + B a_j (B: `rank` lowest DCT modes), plus N(0, noise^2).

    a_j ~ N(0, s^2 I) with s = 0.3 sqrt(d / rank), so the mean image has pixel RMS about 0.3.
    No clipping.
    """
    side = int(round(np.sqrt(d)))
    assert side * side == d, "lowrank_images wants a square image size"
    rng = np.random.default_rng(seed)
    B = dct_basis(side, rank)
    s = 0.3 * np.sqrt(d / rank)
    A = s * rng.standard_normal((k, rank))
    means = 0.5 + A @ B.T
    counts = np.full(k, int(n_per_class))
    lab = _labels(rng, counts, shuffle)
    X = means[lab] + noise * rng.standard_normal((lab.size, d))
    ylab = _labels(rng, np.full(k, int(n_test_per_class)), False)
    Xt = means[ylab] + noise * rng.standard_normal((ylab.size, d))
    return Problem(np.ascontiguousarray(X), lab, k, np.ascontiguousarray(Xt), ylab, name,
                   {"generator": "lowrank_images", "rank": rank, "noise": noise, "seed": seed})


# The workload shapes. tau is the scale target (largest c^2 * lambda_max of the two Grams).
CONFIGS = {
    "d256_k8":    dict(d=256,   k=8,   n_j=6,  t=7,   b=1,  tau=10.0, test=5, gen="clusters"),
    "d4096_k40":  dict(d=4096,  k=40,  n_j=5,  t=39,  b=8,  tau=10.0, test=5, gen="clusters"),
    "d16384_k100": dict(d=16384, k=100, n_j=7, t=99,  b=16, tau=20.0, test=3, gen="clusters"),
    "d65536_k200": dict(d=65536, k=200, n_j=10, t=199, b=32, tau=20.0, test=3, gen="lowrank"),
    # CMU-PIE-sized images (486 x 640 pixels), 10 classes of 8 training images (Section 4, Table 4.6)
    "d311040_k10": dict(d=311040, k=10, n_j=8, t=9, b=8, tau=10.0, test=3, gen="clusters"),
}


def config_problem(name, split=0):
    """The named workload with seed 1000 * (index + 1) + split."""
    c = CONFIGS[name]
    seed = 1000 * (list(CONFIGS).index(name) + 1) + split
    if c["gen"] == "lowrank":
        return lowrank_images(c["d"], c["k"], c["n_j"], seed=seed, n_test_per_class=c["test"], name=name)
    return gaussian_clusters(c["d"], c["k"], c["n_j"], seed=seed, n_test_per_class=c["test"], name=name)


# The batched workload: 64 independent problems, d in {1024, 4096, 16384}, k ~ U[10, 100],
# n_j ~ U[3, 10] per class, t = k - 1, scale target tau = 10.
BATCHED = dict(count=64, seed=5000, tau=10.0)


def batched_problems(count=64, seed=5000, d_choices=(1024, 4096, 16384), k_range=(10, 100), nj_range=(3, 10)):
    """Independent problems of uneven size: d from d_choices, k ~ U[k_range], n_j ~ U[nj_range] per class."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        d = int(rng.choice(d_choices))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        nj = rng.integers(nj_range[0], nj_range[1] + 1, size=k)
        out.append(gaussian_clusters(d, k, nj, seed=int(rng.integers(1 << 31)), n_test_per_class=3,
                                     name=f"batch{p}"))
    return out


def start_block(d, b, seed=0):
    """A seeded Gaussian d x b block, returned as (b, d) C-contiguous (column-major d x b)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((b, d)))
