"""Seeded synthetic inputs for KL-NMF (the only code shared by the oracle and the CUDA path).

This module draws random numbers and nothing else: it holds none of the
factorisation arithmetic.  Every generator returns float32 arrays, so the FP64
oracle (which promotes them exactly) and the GPU path start from bit-identical
values.

Shapes and value distributions stand in for the paper's workloads (Section 4:
dense face-image matrices and sparse term-count matrices), which are public
datasets not available here.  The recipes:

* ``plain_small``      N=256  T=512   R=16:  W0,H0 ~ Gamma(0.5, 1), V ~ Poisson(W0 H0).
* ``plain_large``      N=4096 T=16384 R=128: W0,H0 ~ Gamma(0.3, 1), W0 H0 rescaled to
                       mean 2, V ~ Poisson(W0 H0).
* ``precision_large``  N=8192 T=32768 R=512: W0 ~ Gamma(0.5), H0 ~ Gamma(0.5) with 70 %
                       of its entries set to zero, V = W0 H0 + |N(0, 0.01)| (no zeros).
* ``diff_form``        N=1024 R=64 T=4096:   W0,H0 ~ Gamma(0.5), V ~ Poisson(W0 H0).
* ``batched``          512 problems, N ~ logU[64, 2048], T ~ logU[128, 8192],
                       R ~ U{8, 16, 32, 64}, each V ~ Poisson(W0 H0), Gamma(0.5) truth.

* ``sparse_tdt2``      36771 terms x 10212 documents, 0.35 % non-zeros, R=64 (the shape
                       of the TDT2 term counts of Section 4.2);
* ``sparse_newsgroup`` 61188 x 18774, 0.2 % non-zeros, R=64 (the Newsgroup counts):
                       synthetic term-document counts, one dominant topic per document
                       (70 % of its tokens from the topic's Zipf(1.1) vocabulary, the rest
                       from a background Zipf(1.1)), log-normal document lengths tuned to
                       the target density, returned as CSR (rows = terms).

The starting guess is W, H ~ U(0.1, 1) in every case.  ``custom`` builds the same
kind of problem at any (N, T, R) for tests, ``sparse_custom`` the sparse kind.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_CONFIG_IDS = {"plain_small": 1, "plain_large": 2, "precision_large": 3,
               "diff_form": 4, "batched": 5, "sparse_tdt2": 6, "sparse_newsgroup": 7,
               "sparse_custom": 8, "custom": 99}


@dataclass
class Problem:
    """One NMF problem: data V (N x T), truth factors and a starting guess."""
    name: str
    V: np.ndarray          # float32 N x T, row-major
    W0: np.ndarray         # float32 N x R truth (used only to build V)
    H0: np.ndarray         # float32 R x T truth
    W: np.ndarray          # float32 N x R starting guess
    H: np.ndarray          # float32 R x T starting guess
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.V.shape[0], self.V.shape[1], self.W.shape[1]


def _rng(seed: int, name: str, stream: int = 0) -> np.random.Generator:
    return np.random.default_rng([int(seed), _CONFIG_IDS[name], int(stream)])


def _init(rng: np.random.Generator, N: int, T: int, R: int):
    W = rng.uniform(0.1, 1.0, size=(N, R)).astype(np.float32)
    H = rng.uniform(0.1, 1.0, size=(R, T)).astype(np.float32)
    return W, H


def _poisson_rows(rng: np.random.Generator, lam: np.ndarray) -> np.ndarray:
    """Poisson draws, row by row to bound the float64 temporaries."""
    out = np.empty(lam.shape, dtype=np.float32)
    step = max(1, (1 << 22) // max(1, lam.shape[1]))
    for i in range(0, lam.shape[0], step):
        out[i:i + step] = rng.poisson(lam[i:i + step]).astype(np.float32)
    return out


def custom(N: int, T: int, R: int, seed: int = 0, shape: float = 0.5,
           mean: float | None = None, noise: str = "poisson",
           zero_frac_H0: float = 0.0, name: str = "custom") -> Problem:
    """A KL-NMF problem of any size.

    ``noise='poisson'``: V ~ Poisson(W0 H0).  ``noise='abs_normal'``:
    V = W0 H0 + |N(0, 0.01)|.  ``noise='exact'``: V = W0 H0 (an exact factorisation,
    rounded to float32).  ``mean`` rescales W0 H0 to that mean before the noise.
    """
    g_truth = _rng(seed, name, 0)
    W0 = g_truth.gamma(shape, 1.0, size=(N, R))
    H0 = g_truth.gamma(shape, 1.0, size=(R, T))
    if zero_frac_H0 > 0.0:
        H0 = H0 * (g_truth.random(size=(R, T)) >= zero_frac_H0)
    Z0 = W0 @ H0
    if mean is not None:
        k = mean / max(float(Z0.mean()), 1e-300)
        W0 = W0 * k
        Z0 = Z0 * k
    g_noise = _rng(seed, name, 1)
    if noise == "poisson":
        V = _poisson_rows(g_noise, Z0)
    elif noise == "abs_normal":
        V = (Z0 + np.abs(g_noise.normal(0.0, 0.01, size=Z0.shape))).astype(np.float32)
    elif noise == "exact":
        V = Z0.astype(np.float32)
    else:
        raise ValueError(f"unknown noise model {noise!r}")
    W, H = _init(_rng(seed, name, 2), N, T, R)
    meta = {"zero_fraction": float(np.mean(V == 0)), "mean_V": float(V.mean())}
    return Problem(name, np.ascontiguousarray(V), W0.astype(np.float32),
                   H0.astype(np.float32), W, H, seed, meta)


def plain_small(seed: int = 0) -> Problem:
    """N=256 T=512 R=16, Gamma(0.5) truth, Poisson counts."""
    return custom(256, 512, 16, seed, shape=0.5, name="plain_small")


def plain_large(seed: int = 0, N: int = 4096, T: int = 16384, R: int = 128) -> Problem:
    """N=4096 T=16384 R=128, Gamma(0.3) truth rescaled to mean count 2, Poisson counts."""
    return custom(N, T, R, seed, shape=0.3, mean=2.0, name="plain_large")


def precision_large(seed: int = 0, N: int = 8192, T: int = 32768, R: int = 512) -> Problem:
    """N=8192 T=32768 R=512 spectrogram-like data: sparse H0, |N(0, 0.01)| floor."""
    g_truth = _rng(seed, "precision_large", 0)
    W0 = g_truth.gamma(0.5, 1.0, size=(N, R)).astype(np.float32)
    H0 = g_truth.gamma(0.5, 1.0, size=(R, T)).astype(np.float32)
    H0 *= (g_truth.random(size=(R, T)) >= 0.7).astype(np.float32)
    V = W0 @ H0                                  # float32 GEMM: builds the data only
    g_noise = _rng(seed, "precision_large", 1)
    step = max(1, (1 << 22) // T)
    for i in range(0, N, step):
        V[i:i + step] += np.abs(g_noise.normal(0.0, 0.01, size=(min(step, N - i), T))
                                ).astype(np.float32)
    W, H = _init(_rng(seed, "precision_large", 2), N, T, R)
    meta = {"zero_fraction": 0.0, "mean_V": float(V.mean())}
    return Problem("precision_large", V, W0, H0, W, H, seed, meta)


def diff_form(seed: int = 0) -> Problem:
    """N=1024 R=64 T=4096, Gamma(0.5) truth, Poisson counts (W is held fixed there)."""
    return custom(1024, 4096, 64, seed, shape=0.5, name="diff_form")


def batched_shapes(count: int = 512, seed: int = 0,
                   n_range=(64, 2048), t_range=(128, 8192), ranks=(8, 16, 32, 64)):
    """(N, T, R) of each problem: N, T log-uniform, R uniform over ``ranks``."""
    g = _rng(seed, "batched", 0)
    N = np.exp(g.uniform(np.log(n_range[0]), np.log(n_range[1]), size=count)).astype(np.int64)
    T = np.exp(g.uniform(np.log(t_range[0]), np.log(t_range[1]), size=count)).astype(np.int64)
    R = g.choice(np.asarray(ranks, dtype=np.int64), size=count)
    return [(int(n), int(t), int(r)) for n, t, r in zip(N, T, R)]


def batched(count: int = 512, seed: int = 0, **kw) -> list[Problem]:
    """``count`` independent problems with the shapes of ``batched_shapes``."""
    out = []
    for i, (n, t, r) in enumerate(batched_shapes(count, seed, **kw)):
        p = custom(n, t, r, seed=seed * 100003 + i, shape=0.5, name="batched")
        out.append(p)
    return out


@dataclass
class SparseProblem:
    """A term-document count matrix V (N x T) in CSR and a starting guess."""
    name: str
    N: int
    T: int
    row_ptr: np.ndarray    # int64 N + 1
    col_idx: np.ndarray    # int32 nnz, ascending within a row
    vals: np.ndarray       # float32 nnz (counts >= 1)
    W: np.ndarray          # float32 N x R starting guess
    H: np.ndarray          # float32 R x T starting guess
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.vals.size)

    def dense(self) -> np.ndarray:
        """V as a dense float32 array (small cases only)."""
        V = np.zeros((self.N, self.T), dtype=np.float32)
        rows = np.repeat(np.arange(self.N), np.diff(self.row_ptr))
        V[rows, self.col_idx] = self.vals
        return V


def _zipf_cdf(n: int, exponent: float) -> np.ndarray:
    p = (np.arange(n, dtype=np.float64) + 1.0) ** -exponent
    return np.cumsum(p / p.sum())


def _draw_counts(g: np.random.Generator, N: int, T: int, R: int, mean_len: float):
    """Token draws -> (term, doc) count pairs, sorted by term then document."""
    lens = np.maximum(1, np.round(g.lognormal(np.log(mean_len), 0.8, size=T))).astype(np.int64)
    doc = np.repeat(np.arange(T, dtype=np.int64), lens)
    topic = g.integers(0, R, size=T)[doc]
    cdf = _zipf_cdf(N, 1.1)
    rank = np.minimum(np.searchsorted(cdf, g.random(doc.size)), N - 1)
    perms = np.stack([g.permutation(N) for _ in range(R + 1)])     # row R: background
    from_topic = g.random(doc.size) < 0.7
    term = np.where(from_topic, perms[topic, rank], perms[R, rank])
    key, cnt = np.unique(term * T + doc, return_counts=True)
    return key // T, key % T, cnt


def sparse_custom(N: int, T: int, R: int, density: float, seed: int = 0,
                  name: str = "sparse_custom") -> SparseProblem:
    """Synthetic term-document counts with about density * N * T non-zeros (module doc)."""
    target = density * N * T
    mean_len = 1.3 * target / T
    for _ in range(2):                   # one correction of the length scale for repeats
        rows, cols, cnt = _draw_counts(_rng(seed, name, 0), N, T, R, mean_len)
        mean_len *= target / max(1, rows.size)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    W, H = _init(_rng(seed, name, 2), N, T, R)
    meta = {"density": rows.size / (N * T), "nnz": int(rows.size),
            "mean_count": float(cnt.mean())}
    return SparseProblem(name, N, T, row_ptr, cols.astype(np.int32), cnt.astype(np.float32),
                         W, H, seed, meta)


def sparse_tdt2(seed: int = 0, R: int = 64) -> SparseProblem:
    """36771 x 10212 term counts at 0.35 % non-zeros (TDT2's shape, Section 4.2)."""
    return sparse_custom(36771, 10212, R, 0.0035, seed, name="sparse_tdt2")


def sparse_newsgroup(seed: int = 0, R: int = 64) -> SparseProblem:
    """61188 x 18774 term counts at 0.2 % non-zeros (Newsgroup's shape, Section 4.2)."""
    return sparse_custom(61188, 18774, R, 0.002, seed, name="sparse_newsgroup")
