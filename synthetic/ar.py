"""Seeded synthetic AR(p) series: the inputs every test, the benchmark and the oracle share.

This module only *makes inputs*. It holds none of the least-squares arithmetic of the solver or of the
oracle, and imports neither of them.

Model (Def. "Autoregressive Model of Order p", Section 3):

    Y_t = phi_1 Y_{t-1} + ... + phi_p Y_{t-p} + W_t,    W_t i.i.d., mean 0, variance 1.

The paper draws "randomly obtained" stationary coefficients and simulates with a zero constant and unit
variance (Section 4.1); it does not say how. The reading used here:

* characteristic roots r_k: floor(p/2) complex-conjugate pairs with modulus ~ U[lo, hi] and angle ~ U(0, pi),
  plus one real root (modulus ~ U[lo, hi], random sign) when p is odd. Every |r_k| > 1, so the process is
  stationary;
* coefficients from 1 - sum_j phi_j z^j = prod_k (1 - z / r_k), expanded in 60-digit decimal arithmetic and
  rounded once to float64 (a float64 expansion loses all accuracy at p ~ 200 through cancellation);
* simulation as a cascade of real first/second-order recursive sections, one per real root / conjugate pair
  (numerically stable where the expanded direct-form recursion is not), with a 1,000-sample burn-in;
* innovations N(0, 1), or Student-t(5) scaled by sqrt(3/5) to unit variance.

Seeds: numpy PCG64 from SeedSequence([config_id, series_index, BASE_SEED]).
"""
from __future__ import annotations

import decimal
import math
from dataclasses import dataclass

import numpy as np
import scipy.signal

BASE_SEED = 2112_12994
BURN_IN = 1000


@dataclass
class ARSeries:
    y: np.ndarray            # float64, length n (burn-in already discarded)
    phi_true: np.ndarray     # float64, length p: the generating coefficients
    inv_roots: np.ndarray    # complex128, length p: 1/r_k (all inside the unit disc)
    seed: tuple              # the SeedSequence entropy used


def rng_for(config_id: int, series_index: int = 0, base_seed: int = BASE_SEED) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([config_id, series_index, base_seed])))


def draw_inverse_roots(rng: np.random.Generator, p: int, lo: float, hi: float) -> np.ndarray:
    """Inverse characteristic roots a_k = 1/r_k with |r_k| ~ U[lo, hi] (lo > 1)."""
    if not (1.0 < lo <= hi):
        raise ValueError("root moduli must satisfy 1 < lo <= hi")
    out = []
    for _ in range(p // 2):
        mod = rng.uniform(lo, hi)
        ang = rng.uniform(0.0, math.pi)
        a = np.exp(-1j * ang) / mod
        out.extend([a, np.conj(a)])
    if p % 2:
        mod = rng.uniform(lo, hi)
        sign = 1.0 if rng.uniform() < 0.5 else -1.0
        out.append(complex(sign / mod, 0.0))
    return np.asarray(out, dtype=np.complex128)


def _sections(inv_roots: np.ndarray):
    """Real factors of prod_k (1 - a_k z): ('2', 2 Re a, |a|^2) per conjugate pair, ('1', a) per real root."""
    secs = []
    k = 0
    while k < len(inv_roots):
        a = inv_roots[k]
        if abs(a.imag) > 0.0 and k + 1 < len(inv_roots) and inv_roots[k + 1] == np.conj(a):
            secs.append(("2", 2.0 * a.real, a.real * a.real + a.imag * a.imag))
            k += 2
        else:
            secs.append(("1", float(a.real)))
            k += 1
    return secs


def coefficients_from_inverse_roots(inv_roots: np.ndarray) -> np.ndarray:
    """phi with 1 - sum_j phi_j z^j = prod_k (1 - a_k z), expanded with 60 significant digits."""
    ctx = decimal.Context(prec=60)
    poly = [decimal.Decimal(1)]
    for sec in _sections(inv_roots):
        if sec[0] == "2":
            fac = [decimal.Decimal(1), -decimal.Decimal(sec[1]), decimal.Decimal(sec[2])]
        else:
            fac = [decimal.Decimal(1), -decimal.Decimal(sec[1])]
        new = [decimal.Decimal(0)] * (len(poly) + len(fac) - 1)
        for i, c in enumerate(poly):
            for j, f in enumerate(fac):
                new[i + j] = ctx.add(new[i + j], ctx.multiply(c, f))
        poly = new
    return np.array([-float(c) for c in poly[1:]], dtype=np.float64)


def simulate(inv_roots: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Run innovations w through the cascade 1 / prod_k (1 - a_k z^-1), one real section at a time."""
    rows = []
    for sec in _sections(inv_roots):
        if sec[0] == "2":
            rows.append([1.0, 0.0, 0.0, 1.0, -sec[1], sec[2]])
        else:
            rows.append([1.0, 0.0, 0.0, 1.0, -sec[1], 0.0])
    if not rows:
        return np.array(w, dtype=np.float64, copy=True)
    return scipy.signal.sosfilt(np.asarray(rows, dtype=np.float64), np.asarray(w, dtype=np.float64))


def innovations(rng: np.random.Generator, count: int, kind: str = "normal") -> np.ndarray:
    if kind == "normal":
        return rng.standard_normal(count)
    if kind == "t5":
        return rng.standard_t(5, size=count) * math.sqrt(3.0 / 5.0)
    raise ValueError(f"unknown innovation kind {kind!r}")


def log10_spectral_bound(inv_roots: np.ndarray, grid: int = 4096) -> float:
    """log10(max S / min S) of the AR spectral density S(w) = 1/|prod_k (1 - a_k e^{iw})|^2.

    It bounds kappa(X^T X) for long series; used only to pick or reject seeds.
    """
    w = np.linspace(0.0, math.pi, grid)
    z = np.exp(1j * w)
    logmag = np.zeros_like(w)
    for a in inv_roots:
        logmag += np.log10(np.abs(1.0 - a * z) ** 2)
    return float(logmag.max() - logmag.min())


def ar_series(n: int, p: int, *, config_id: int = 0, series_index: int = 0, root_lo: float = 1.2,
              root_hi: float = 3.0, noise: str = "normal", base_seed: int = BASE_SEED,
              max_log10_bound: float | None = None, max_tries: int = 1000) -> ARSeries:
    """A stationary AR(p) series of length n (after burn-in) from a reproducible seed.

    With max_log10_bound set, seeds (config_id, series_index + k, base_seed), k = 0, 1, ..., are tried until
    the spectral bound of the drawn roots is at most 10**max_log10_bound.
    """
    if n < 1 or p < 0:
        raise ValueError("need n >= 1 and p >= 0")
    for k in range(max_tries):
        idx = series_index + k
        rng = rng_for(config_id, idx, base_seed)
        inv = draw_inverse_roots(rng, p, root_lo, root_hi)
        if max_log10_bound is not None and p > 0 and log10_spectral_bound(inv) > max_log10_bound:
            continue
        w = innovations(rng, n + BURN_IN, noise)
        y = simulate(inv, w)[BURN_IN:]
        phi = coefficients_from_inverse_roots(inv) if p > 0 else np.zeros(0)
        return ARSeries(y=np.ascontiguousarray(y), phi_true=phi, inv_roots=inv, seed=(config_id, idx, base_seed))
    raise RuntimeError("no seed met the spectral bound")


def batch_shapes(count: int, *, config_id: int, n_lo: float, n_hi: float, p_lo: int, p_hi: int,
                 p_log_uniform: bool = False, base_seed: int = BASE_SEED):
    """(n_i, p_i) for a batch: n log-uniform in [n_lo, n_hi]; p uniform (or log-uniform) integer in [p_lo, p_hi]."""
    rng = rng_for(config_id, 10**9, base_seed)
    n = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(np.int64)
    if p_log_uniform:
        p = np.floor(np.exp(rng.uniform(math.log(max(p_lo, 1)), math.log(p_hi + 1), size=count))).astype(np.int64)
        p = np.clip(p, p_lo, p_hi)
    else:
        p = rng.integers(p_lo, p_hi + 1, size=count).astype(np.int64)
    n = np.maximum(n, p + 2)
    return n, p


def lsar_uniforms(p_bar: int, c: int, *, config_id: int, series_index: int = 0,
                  base_seed: int = BASE_SEED) -> np.ndarray:
    """The random draws of a leverage-sampling sweep over lags 1..p_bar: row h-1 holds the c uniforms in [0, 1)
    that pick the sampled rows at lag h (inverse-CDF sampling with replacement). Passed to the sampler as input."""
    rng = rng_for(config_id, 2 * 10**9 + series_index, base_seed)
    return np.ascontiguousarray(rng.random((p_bar, c)))


def with_outliers(y: np.ndarray, count: int, *, config_id: int, series_index: int = 0,
                  base_seed: int = BASE_SEED) -> np.ndarray:
    """A copy of y with `count` distinct positions, drawn uniformly, replaced by y + U[-3, 3] + N(0, 100): the
    outlier workload of the paper's Section 4.2 (1,000 such points in two million)."""
    rng = rng_for(config_id, 3 * 10**9 + series_index, base_seed)
    out = np.array(y, dtype=np.float64, copy=True)
    pos = rng.choice(out.size, size=count, replace=False)
    out[pos] += rng.uniform(-3.0, 3.0, size=count) + rng.normal(0.0, 10.0, size=count)
    return out


def srht_draws(m: int, c: int, *, config_id: int, series_index: int = 0, base_seed: int = BASE_SEED):
    """The random draws of a sampled randomised Hadamard transform on m rows padded to m2 = 2^ceil(log2 m): m2
    signs +-1 (the diagonal D) and c row indices uniform in [0, m2) with replacement (the sampling S)."""
    rng = rng_for(config_id, 4 * 10**9 + series_index, base_seed)
    m2 = 1 << max(0, (m - 1).bit_length())
    signs = np.where(rng.random(m2) < 0.5, -1.0, 1.0)
    rows = rng.integers(0, m2, size=c)
    return signs, rows


def rh_draws(n_rows: int, c: int, k: int, min_rows: int, *, config_id: int, series_index: int = 0,
             base_seed: int = BASE_SEED):
    """The random draws of a Repeated Halving run on n_rows rows: per halving level j (while the level has more
    than min_rows rows) the floor(n_j / 2) positions the next level keeps (a uniform subset, increasing), a
    k x r_j Gaussian sketch with N(0, 1/k) entries (r_j: rows of the approximation one level down, the deepest
    level's own rows or c), and c uniforms for the leverage sampling. Returns (keep, gauss, unif), lists
    indexed by level."""
    rng = rng_for(config_id, 5 * 10**9 + series_index, base_seed)
    sizes = [n_rows]
    while sizes[-1] > min_rows:
        sizes.append(sizes[-1] // 2)
    levels = len(sizes) - 1
    keep = [np.sort(rng.choice(sizes[j], size=sizes[j + 1], replace=False)).astype(np.int64)
            for j in range(levels)]
    gauss = [rng.standard_normal((k, sizes[-1] if j == levels - 1 else c)) / math.sqrt(k) for j in range(levels)]
    unif = [rng.random(c) for _ in range(levels)]
    return keep, gauss, unif
