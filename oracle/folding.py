"""TEST INFRASTRUCTURE ONLY -- oracle of the cleartext check of the folding polynomial.

Plain numpy restatement of the probabilistic-folding experiment of arxiv 2601.17561:
  - Section 4.1.2 defines a (k, N_f, P_f)-folding polynomial f through two probabilities over
    negative scores x_i drawn from a law D:  p1 bounds Pr(sum_{i<k} f(x_i) outside N_f), and p2
    bounds Pr(min_{x in P} f(x) + sum_{0<i<k} f(x_i) outside P_f);
  - Appendix C.2 prints the degree-7 polynomial for k = 16, N_f = [-0.13, 0.33], P_f = [0.4, 3.8]
    and validates it with 1e12 experiments: the sum of 16 values of f over D, and the minimum and
    the maximum of f over P each plus a sum of 15 values over D;
  - Section 6.1 approximates D (negative scores of real iris pairs) by the normal law N(0.008, 0.034^2).

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference legs of `bench.py` may
import this module.  It shares no code with the CUDA library.

Random numbers.  Both sides draw from one counter-based generator implemented separately from its
published definition: Philox4x64-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC 2011).  Trial t of a run keyed by `seed` uses the blocks at counters
(t, j, 0, 0), j = 0, 1, ..., with key (seed, 0); block j gives words 4j..4j+3.  Normal deviates come
in pairs from consecutive words (a, b) by the Box-Muller transform (Box and Muller, 1958):
u1 = (a + 1/2) 2^-64, u2 = b 2^-64, r = sqrt(-2 ln u1), (z0, z1) = (r cos 2 pi u2, r sin 2 pi u2).
Normal n = 2p + e of a trial comes from pair p (words 2p, 2p+1); normals 0..k-1 are the x_i of the
sum over k values, normals k..2k-2 the y_i of the sum over k-1 values (the paper draws them
independently).

Readings (the paper is silent or garbled here):
  - P, the positive-score interval, is never stated.  The functions take it as a parameter.
  - The appendix assigns p1 ~ 5.3e-11 and p2 ~ 5.4e-10, while its counts give 53 outliers (per
    1e12) for the sum over 16 negatives (the p1 event of Section 4.1.2) and 542 for the sums with a
    positive (the p2 event): the two names are swapped there.  This module names the events by the
    definition.
  - The paper counts the minimum and the maximum experiment of a trial separately; so does this
    module (four counters: each of the two values below P_f or above it).

Parity status: every function here is pinned by `tests/test_folding_pins.py` (numpy's Philox for
the generator, the normal law's moments and CDF for the deviates, closed forms and brute force for
the range and the convolution, the convolution for the Monte Carlo).
"""
from __future__ import annotations

import numpy as np

# Appendix C.2: the 16x folding polynomial, coefficients of x^0 .. x^7.
PAPER_FOLD_COEF = (0.004105, -0.173510, -2.528271, 24.347349, 124.161550, -412.746212, 376.961251, 106.553952)
PAPER_K = 16
PAPER_NF = (-0.13, 0.33)
PAPER_PF = (0.4, 3.8)
# Section 6.1: negative scores ~ N(0.008, 0.034^2); Appendix C.2 designs f against N(0.008, 0.06^2).
PAPER_D = (0.008, 0.034)
PAPER_D_DESIGN = (0.008, 0.06)

# ------------------------------------------------------------------ Philox4x64-10 (SC 2011)
_M0, _M1 = np.uint64(0xD2E7470EE14C6C93), np.uint64(0xCA5A826395121157)
_W0, _W1 = np.uint64(0x9E3779B97F4A7C15), np.uint64(0xBB67AE8584CAA73B)
_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo64(a, b):
    """(hi, lo) 64-bit halves of the 128-bit product a*b, by schoolbook over 32-bit halves."""
    a = np.asarray(a, np.uint64)
    b = np.asarray(b, np.uint64)
    a0, a1 = a & _LO32, a >> _S32
    b0, b1 = b & _LO32, b >> _S32
    p00, p01, p10, p11 = a0 * b0, a0 * b1, a1 * b0, a1 * b1
    mid = (p00 >> _S32) + (p01 & _LO32) + (p10 & _LO32)
    hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
    return hi, a * b


def philox4x64(ctr, key):
    """Philox4x64 with 10 rounds: ctr = 4 uint64 arrays (broadcast), key = (k0, k1).

    Round: (h0, l0) = M0 c0, (h1, l1) = M1 c2; c <- (h1 ^ c1 ^ k0, l1, h0 ^ c3 ^ k1, l0); then the
    key is bumped by the Weyl constants (W0, W1).  Returns the 4 output words."""
    c = [np.asarray(x, np.uint64) for x in ctr]
    k0, k1 = np.uint64(key[0]), np.uint64(key[1])
    with np.errstate(over="ignore"):
        for _ in range(10):
            h0, l0 = _mulhilo64(_M0, c[0])
            h1, l1 = _mulhilo64(_M1, c[2])
            c = [h1 ^ c[1] ^ k0, l1, h0 ^ c[3] ^ k1, l0]
            k0 = k0 + _W0
            k1 = k1 + _W1
    return c


def trial_words(seed: int, trials, n_words: int) -> np.ndarray:
    """Words 0..n_words-1 of every trial in `trials` (uint64 [len(trials)][n_words])."""
    t = np.asarray(trials, np.uint64)
    nb = (n_words + 3) // 4
    out = np.empty((t.size, nb * 4), np.uint64)
    zero = np.zeros_like(t)
    for j in range(nb):
        w = philox4x64([t, np.full_like(t, j), zero, zero], (seed, 0))
        for i in range(4):
            out[:, 4 * j + i] = w[i]
    return out[:, :n_words]


def box_muller(a, b):
    """Pairs of standard normals from word pairs (a, b): the textbook transform on
    u1 = (a + 1/2) 2^-64 in (0, 1) and u2 = b 2^-64 in [0, 1).  ln u1 is taken as log1p(-(1 - u1))
    with 1 - u1 = (~a + 1/2) 2^-64 when u1 >= 1/2, so that no digit of u1 is lost near 1."""
    a = np.asarray(a, np.uint64)
    b = np.asarray(b, np.uint64)
    top = a >= np.uint64(1 << 63)
    with np.errstate(divide="ignore"):
        ln_lo = np.log((a.astype(np.float64) + 0.5) * 2.0 ** -64)
        ln_hi = np.log1p(-((~a).astype(np.float64) + 0.5) * 2.0 ** -64)
    r = np.sqrt(-2.0 * np.where(top, ln_hi, ln_lo))
    th = 2.0 * np.pi * (b.astype(np.float64) * 2.0 ** -64)
    return r * np.cos(th), r * np.sin(th)


def trial_normals(seed: int, trials, k: int) -> np.ndarray:
    """The 2k standard normals of every trial (float64 [len(trials)][2k])."""
    w = trial_words(seed, trials, 2 * k)
    z0, z1 = box_muller(w[:, 0::2], w[:, 1::2])
    z = np.empty((w.shape[0], 2 * k))
    z[:, 0::2] = z0
    z[:, 1::2] = z1
    return z


# ------------------------------------------------------------------ the folding polynomial

def poly(coef, x):
    """f(x) = sum_i coef[i] x^i (coef from x^0 upwards), in float64."""
    return np.polynomial.polynomial.polyval(np.asarray(x, np.float64), np.asarray(coef, np.float64))


def poly_range(coef, lo: float, hi: float):
    """(min, max) of f over [lo, hi]: the extremes lie at the ends or at real roots of f' inside."""
    c = np.asarray(coef, np.float64)
    xs = [lo, hi]
    if len(c) > 2:
        for r in np.polynomial.polynomial.polyroots(np.polynomial.polynomial.polyder(c)):
            if abs(r.imag) < 1e-12 and lo < r.real < hi:
                xs.append(r.real)
    v = poly(c, np.array(xs))
    return float(v.min()), float(v.max())


def fold_mc(coef, mu, sigma, k, pos, nf, pf, seed, trial0, n_trials, hist=None):
    """The experiments of Appendix C.2 for trials trial0 .. trial0 + n_trials - 1.

    Returns dict(sk, sk1, counts, hist): per trial S_k = sum_{i<k} f(x_i) and
    S_{k-1} = sum_{i<k-1} f(y_i) with x, y ~ N(mu, sigma^2) (float64); counts = [S_k < nf_lo,
    S_k > nf_hi, fmin + S_{k-1} < pf_lo, fmin + S_{k-1} > pf_hi, fmax + S_{k-1} < pf_lo,
    fmax + S_{k-1} > pf_hi] with (fmin, fmax) the range of f over P = pos; hist = (lo, hi, n_bins)
    gives the histograms of S_k and S_{k-1} with an underflow bin first and an overflow bin last."""
    trials = np.arange(trial0, trial0 + n_trials, dtype=np.uint64)
    z = trial_normals(seed, trials, k)
    fx = poly(coef, mu + sigma * z)
    sk = fx[:, :k].sum(axis=1)
    sk1 = fx[:, k:2 * k - 1].sum(axis=1)
    fmin, fmax = poly_range(coef, *pos)
    counts = np.array([(sk < nf[0]).sum(), (sk > nf[1]).sum(),
                       (fmin + sk1 < pf[0]).sum(), (fmin + sk1 > pf[1]).sum(),
                       (fmax + sk1 < pf[0]).sum(), (fmax + sk1 > pf[1]).sum()], np.int64)
    out = dict(sk=sk, sk1=sk1, counts=counts, fmin=fmin, fmax=fmax)
    if hist is not None:
        lo, hi, nb = hist
        out["hist"] = np.stack([histogram(s, lo, hi, nb) for s in (sk, sk1)])
    return out


def histogram(s, lo, hi, nb):
    """Counts of s per bin: [below lo, nb equal bins of [lo, hi), at or above hi]."""
    i = np.floor((np.asarray(s) - lo) * (nb / (hi - lo)))
    i = np.clip(i, -1, nb).astype(np.int64) + 1
    return np.bincount(i, minlength=nb + 2)


# ------------------------------------------------------------------ exact law of the sums

def sum_law(coef, mu, sigma, k, h=2e-5, span=12.0, n_x=4_000_000):
    """Distribution of S_k = sum of k independent f(x), x ~ N(mu, sigma^2), on a grid of step h.

    The law of f(x) is binned from the exact normal masses of n_x cells of [mu - span sigma,
    mu + span sigma] (each cell's mass put at the grid point nearest f(cell centre)); its k-fold
    convolution is a power of its discrete Fourier transform (zero-padded, so no wrap-around).
    Returns (grid, pmf): grid[i] = k y0 + i h.  The grid rounding moves each term by at most h/2,
    so S_k by at most k h / 2."""
    from scipy.special import ndtr
    xs = np.linspace(mu - span * sigma, mu + span * sigma, n_x + 1)
    mass = np.diff(ndtr((xs - mu) / sigma))
    y = poly(coef, 0.5 * (xs[1:] + xs[:-1]))
    y0 = np.floor(y.min() / h) * h
    idx = np.rint((y - y0) / h).astype(np.int64)
    p1 = np.bincount(idx, weights=mass)
    n = 1
    while n < k * len(p1):
        n *= 2
    pk = np.fft.irfft(np.fft.rfft(p1, n) ** k, n)
    return k * y0 + np.arange(n) * h, np.maximum(pk, 0.0)


def law_mass(grid, pmf, lo, hi):
    """Pr(lo <= S < hi) from a law on a grid: each grid point's mass stands for its whole cell
    [g - h/2, g + h/2) (the grid rounds every term to the nearest point), so a cell that straddles
    lo or hi contributes the fraction inside."""
    h = grid[1] - grid[0]
    a = np.clip((grid + 0.5 * h - lo) / h, 0.0, 1.0)      # fraction of the cell at or above lo
    b = np.clip((hi - (grid - 0.5 * h)) / h, 0.0, 1.0)    # fraction of the cell below hi
    return float((pmf * np.clip(a + b - 1.0, 0.0, 1.0)).sum())


def tail_probs(grid, pmf, lo, hi):
    """(Pr(S < lo), Pr(S > hi)) from a law on a grid (cells as in law_mass)."""
    return law_mass(grid, pmf, -np.inf, lo), law_mass(grid, pmf, hi, np.inf)
