"""Seeded synthetic inputs shaped like the paper's radio-map workloads.

This module only draws inputs: measurement locations, their embeddings, the
received-signal-strength observations, the evaluation grid and the Gaussian
random directions z_k that the preconditioner fit consumes (Eq. 12, the
random-directions equation of Sec. IV-B).  It contains none of the method's
arithmetic (no kernel, no solve, no CCCP), so the CPU oracle and the CUDA path
can both be fed from it without sharing any computation.

Input recipe (the paper's own embedding and field generator are described in
prose only, Sec. V-A):

* locations x_i in a square of side ``side`` metres, uniform, or 70 % uniform
  plus 30 % in five Gaussian blobs (sigma 50 m) whose centres are uniform in the
  square; blob draws outside the square are redrawn;
* embedding q(x) = sqrt(2/d) cos(W x/side + b), a seeded Gaussian random-feature
  map with W_t ~ N(0, ell^-2 I_2), ell = 0.1, and b_t ~ U[0, 2 pi), so |q| ~ 1;
* RSS in dBm from ``n_tx`` transmitters at uniform positions, 20 dBm each:
  free-space loss at d0 = 1 m plus log-distance loss with exponent ``eta``,
  and i.i.d. log-normal shadowing N(0, shadow_db^2) per (point, transmitter);
  powers add in milliwatts;
* y = (RSS - mean) / std (ddof 0); the noiseless field on the grid is kept
  for RMSE/NMSE;
* grid: m x m cell centres ((j + 1/2) side / m), embedded with the same map.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SPEED_OF_LIGHT = 299_792_458.0


@dataclasses.dataclass
class Instance:
    """One regression problem: embeddings, observations and a query grid."""

    X: np.ndarray        # n x 2 locations in metres
    Q: np.ndarray        # n x d embeddings, float64, row-major
    y: np.ndarray        # n standardised observations
    y_mu: float          # mean of the raw RSS (dBm)
    y_sigma: float       # std of the raw RSS (dB)
    Xg: np.ndarray       # M x 2 grid locations
    Qg: np.ndarray       # M x d grid embeddings
    rss_grid: np.ndarray  # M noiseless field values at the grid (dBm)
    lam: float           # ridge parameter lambda
    scale: float         # kernel scale s in G_ij = exp(s q_i . q_j)
    seed: int

    @property
    def n(self) -> int:
        return self.Q.shape[0]

    @property
    def d(self) -> int:
        return self.Q.shape[1]


def _locations(rng: np.random.Generator, n: int, side: float, layout: str) -> np.ndarray:
    if layout == "uniform":
        return rng.uniform(0.0, side, size=(n, 2))
    if layout == "clustered":
        n_blob = int(round(0.3 * n))
        n_uni = n - n_blob
        centres = rng.uniform(0.0, side, size=(5, 2))
        pts = [rng.uniform(0.0, side, size=(n_uni, 2))]
        which = rng.integers(0, 5, size=n_blob)
        blob = centres[which] + rng.normal(0.0, 50.0, size=(n_blob, 2))
        bad = (blob < 0.0) | (blob > side)
        bad = bad.any(axis=1)
        while bad.any():
            k = int(bad.sum())
            blob[bad] = centres[which[bad]] + rng.normal(0.0, 50.0, size=(k, 2))
            bad = ((blob < 0.0) | (blob > side)).any(axis=1)
        pts.append(blob)
        out = np.concatenate(pts, axis=0)
        return out[rng.permutation(n)]
    raise ValueError(f"unknown layout {layout!r}")


class FeatureMap:
    """Seeded Gaussian random-feature embedding of 2-D locations."""

    def __init__(self, rng: np.random.Generator, d: int, side: float, ell: float = 0.1):
        self.W = rng.normal(0.0, 1.0 / ell, size=(d, 2))
        self.b = rng.uniform(0.0, 2.0 * math.pi, size=d)
        self.side = side
        self.d = d

    def __call__(self, X: np.ndarray) -> np.ndarray:
        Xt = X / self.side
        return np.sqrt(2.0 / self.d) * np.cos(Xt @ self.W.T + self.b)


def _rss_dbm(X: np.ndarray, tx: np.ndarray, freq_hz: float, eta: float,
             shadow: np.ndarray | None, p_tx_dbm: float = 20.0) -> np.ndarray:
    d0 = 1.0
    fspl_d0 = 20.0 * math.log10(4.0 * math.pi * freq_hz * d0 / SPEED_OF_LIGHT)
    dist = np.sqrt(((X[:, None, :] - tx[None, :, :]) ** 2).sum(axis=2))
    pl = fspl_d0 + 10.0 * eta * np.log10(np.maximum(dist, d0) / d0)
    p = p_tx_dbm - pl
    if shadow is not None:
        p = p + shadow
    return 10.0 * np.log10((10.0 ** (p / 10.0)).sum(axis=1))


def make_instance(n: int, d: int, lam: float, *, n_tx: int = 3, seed: int = 0,
                  layout: str = "uniform", side: float = 1000.0,
                  freq_hz: float = 2.4e9, eta: float = 3.0, shadow_db: float = 6.0,
                  grid: int = 64, scale: float | None = None,
                  ell: float = 0.1) -> Instance:
    """Draw one seeded instance; ``scale`` defaults to 1/sqrt(d)."""
    rng = np.random.default_rng(seed)
    X = _locations(rng, n, side, layout)
    fmap = FeatureMap(rng, d, side, ell)
    Q = np.ascontiguousarray(fmap(X), dtype=np.float64)
    tx = rng.uniform(0.0, side, size=(n_tx, 2))
    shadow = rng.normal(0.0, shadow_db, size=(n, n_tx))
    rss = _rss_dbm(X, tx, freq_hz, eta, shadow)
    mu = float(rss.mean())
    sig = float(rss.std())
    if sig == 0.0:
        sig = 1.0
    y = (rss - mu) / sig
    c = (np.arange(grid) + 0.5) * side / grid
    gx, gy = np.meshgrid(c, c, indexing="xy")
    Xg = np.stack([gx.ravel(), gy.ravel()], axis=1)
    Qg = np.ascontiguousarray(fmap(Xg), dtype=np.float64)
    rss_grid = _rss_dbm(Xg, tx, freq_hz, eta, None)
    if scale is None:
        scale = 1.0 / math.sqrt(d)
    return Instance(X=X, Q=Q, y=np.ascontiguousarray(y), y_mu=mu, y_sigma=sig,
                    Xg=Xg, Qg=Qg, rss_grid=rss_grid, lam=float(lam),
                    scale=float(scale), seed=seed)


def directions(n: int, n_r: int, seed: int) -> np.ndarray:
    """Gaussian directions z_k ~ N(0, I_n), returned as an n x N_r array
    (column k is z_k), row-major float64."""
    rng = np.random.default_rng(seed + 7_919)
    return np.ascontiguousarray(rng.standard_normal(size=(n, n_r)))


def random_vector(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed + 104_729)
    return rng.standard_normal(size=n)


def default_num_directions(n: int) -> int:
    """The number of random directions N_r.  The paper gives only the shape of
    its schedule (O(sqrt n) for small n, linear for large n, Sec. V-A); this
    reading takes max(2 sqrt(n), n/64), at most n and 1024: 64 at n = 1024,
    128 at n = 4096, 256 at n = 16384, 1024 at n = 65536.  The constants are
    measured: the fit's cost grows like n N_r^2 + N_r^3 while the PCG products
    fall slowly with N_r, and each product costs ~n^2 d, so larger N_r pays
    only at the largest n."""
    return int(min(n, 1024, max(math.ceil(2.0 * math.sqrt(n)), math.ceil(n / 64.0))))


# Configurations of the workloads (sizes and field parameters).
CONFIGS = {
    "n1024_fp64": dict(n=1024, d=16, lam=1e-3, n_tx=3, layout="uniform", grid=64, tol=1e-8),
    "n16384_d32": dict(n=16384, d=32, lam=1e-4, n_tx=8, layout="clustered", grid=512, tol=1e-6),
    "n65536_d64": dict(n=65536, d=64, lam=1e-4, n_tx=8, layout="uniform", grid=512, tol=1e-6),
    "batch256": dict(count=256, n_lo=512, n_hi=8192, d_choices=(16, 32), lam_lo=1e-5, lam_hi=1e-2,
               tx_lo=1, tx_hi=8, f_lo=0.7e9, f_hi=6e9, layout="uniform", tol=1e-6),
}


def batch_specs(count: int, seed: int, cfg: dict | None = None) -> list:
    """Parameters of the batching workload: per instance n log-uniform in
    [n_lo, n_hi], d uniform over d_choices, lambda log-uniform, 1-8
    transmitters and a carrier frequency uniform in [f_lo, f_hi] (a pure
    offset of the standardised y).  Returns dicts for make_instance."""
    c = dict(CONFIGS["batch256"]) if cfg is None else cfg
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(math.floor(math.exp(rng.uniform(math.log(c["n_lo"]), math.log(c["n_hi"])))))
        d = int(rng.choice(np.asarray(c["d_choices"])))
        lam = float(10.0 ** rng.uniform(math.log10(c["lam_lo"]), math.log10(c["lam_hi"])))
        n_tx = int(rng.integers(c["tx_lo"], c["tx_hi"] + 1))
        freq = float(rng.uniform(c["f_lo"], c["f_hi"]))
        out.append(dict(n=n, d=d, lam=lam, n_tx=n_tx, freq_hz=freq, seed=int(seed * 1000 + k),
                        layout=c["layout"]))
    return out
