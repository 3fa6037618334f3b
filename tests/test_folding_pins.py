"""Pins for the oracle of the cleartext folding-polynomial check (Section 4.1.2 definition,
Appendix C.2 experiments): numpy's own Philox for the generator, closed forms of the Box-Muller
map and of the normal law, brute force for the polynomial and its range, closed forms for the
convolution law, the law for the Monte Carlo, and the paper's printed outlier rate.  CPU only."""
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.special import ndtr

from oracle import folding as F

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


# ----------------------------------------------------------------------------- generator

@pytest.mark.parametrize("ctr,key", [((0, 0, 0, 0), (0, 0)), ((5, 7, 0, 0), (123, 456)),
                                     ((2**64 - 1, 3, 2**63, 9), (2**64 - 1, 2**40 + 1)),
                                     ((123456789, 0, 0, 0), (0x9E3779B97F4A7C15, 0))])
def test_philox_matches_numpy(ctr, key):
    """numpy's Philox is Philox4x64-10; it advances its 256-bit counter before each block."""
    c = sum(int(w) << (64 * i) for i, w in enumerate(ctr))
    g = np.random.Philox(counter=(c - 1) % 2**256, key=key[0] | (key[1] << 64))
    want = [int(x) for x in g.random_raw(4)]
    got = [int(np.asarray(w)) for w in F.philox4x64(ctr, key)]
    assert got == want


def test_trial_words_layout():
    """Trial t, block j sits at counter (t, j, 0, 0) with key (seed, 0)."""
    w = F.trial_words(99, [0, 7, 2**40], 10)
    for r, t in enumerate([0, 7, 2**40]):
        for j in range(3):
            g = np.random.Philox(counter=((t | (j << 64)) - 1) % 2**256, key=99)
            blk = [int(x) for x in g.random_raw(4)]
            assert [int(x) for x in w[r, 4 * j:4 * j + 4][:max(0, min(4, 10 - 4 * j))]] == blk[:max(0, min(4, 10 - 4 * j))]


def test_box_muller_closed_forms():
    """a = 0 gives u1 = 2^-65 (the largest radius, sqrt(130 ln 2)); u2 = 1/4 turns it to the
    sine; a = 2^63 gives u1 = 1/2 + 2^-65 (radius sqrt(2 ln 2) to 1e-15); the top word gives a
    radius of about 2^-32."""
    z0, z1 = F.box_muller(np.array([0, 1 << 63, 2**64 - 1], np.uint64), np.array([0, 1 << 62, 0], np.uint64))
    assert z0[0] == pytest.approx(np.sqrt(130 * np.log(2)), rel=1e-14) and abs(z1[0]) < 1e-12
    assert abs(z0[1]) < 1e-12 and z1[1] == pytest.approx(np.sqrt(2 * np.log(2)), rel=1e-12)
    assert z0[2] == pytest.approx(2.0**-32, rel=1e-9)           # 1 - u1 = 2^-65


def test_normals_follow_the_normal_law():
    z = F.trial_normals(5, np.arange(1 << 14), 16).ravel()        # 2^19 deviates
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    zs = np.sort(z)
    ks = np.max(np.abs(ndtr(zs) - np.arange(1, n + 1) / n))
    assert ks < 1.95 / np.sqrt(n)                                  # KS test at the 0.1% level
    # pairs are independent: the sample correlation of z0 and z1 vanishes
    zz = F.trial_normals(6, np.arange(1 << 14), 16)
    assert abs(np.corrcoef(zz[:, 0::2].ravel(), zz[:, 1::2].ravel())[0, 1]) < 5 / np.sqrt(n / 2)


# ----------------------------------------------------------------------------- the polynomial

def test_paper_polynomial_and_brute_force():
    """Exact rational evaluation of the printed coefficients (x^0 first) at a few points; the
    constant term is the printed 0.004105 and f stays near 0 around 0 (Appendix C.2)."""
    C = [Fraction(s) for s in ("0.004105", "-0.173510", "-2.528271", "24.347349", "124.161550",
                               "-412.746212", "376.961251", "106.553952")]
    assert F.PAPER_FOLD_COEF == tuple(float(c) for c in C)
    for x in ("0", "1", "-1", "0.25", "-0.233", "0.5"):
        want = sum(c * Fraction(x) ** i for i, c in enumerate(C))
        assert F.poly(F.PAPER_FOLD_COEF, float(Fraction(x))) == pytest.approx(float(want), rel=1e-13, abs=1e-15)
    xs = np.linspace(-0.1, 0.1, 2001)
    assert np.abs(F.poly(F.PAPER_FOLD_COEF, xs)).max() < 0.02


@pytest.mark.parametrize("lo,hi", [(-0.25, 0.2), (0.257, 0.496), (-0.3, 1.0), (0.1, 0.1), (-0.1, -0.05)])
def test_poly_range_brute_force(lo, hi):
    xs = np.linspace(lo, hi, 200001)
    v = F.poly(F.PAPER_FOLD_COEF, xs)
    mn, mx = F.poly_range(F.PAPER_FOLD_COEF, lo, hi)
    assert mn <= v.min() + 1e-15 and mx >= v.max() - 1e-15
    step = (hi - lo) / 200000
    assert v.min() - mn < 1e-6 + 50 * step ** 2 and mx - v.max() < 1e-6 + 50 * step ** 2


# ----------------------------------------------------------------------------- the law of the sums

@pytest.mark.parametrize("k", [1, 5, 16])
def test_sum_law_linear_is_normal(k):
    """f(x) = x: S_k ~ N(k mu, k sigma^2)."""
    mu, sd = 0.008, 0.034
    g, p = F.sum_law((0.0, 1.0), mu, sd, k, h=1e-5, n_x=400_000)
    assert p.sum() == pytest.approx(1.0, abs=1e-12)
    for t in (-3.0, -1.0, 2.0, 4.0):
        x = k * mu + t * np.sqrt(k) * sd
        lo, _ = F.tail_probs(g, p, x, np.inf)
        assert lo == pytest.approx(ndtr(t), rel=2e-3, abs=1e-7)


def test_sum_law_square_is_chi_square():
    """f(x) = x^2 over N(0, sigma^2): Pr(f(x) > c) = 2 Phi(-sqrt(c) / sigma)."""
    sd = 0.05
    g, p = F.sum_law((0.0, 0.0, 1.0), 0.0, sd, 1, h=1e-7, n_x=400_000)
    for c in (1e-4, 1e-3, 9e-3):
        _, hi = F.tail_probs(g, p, -np.inf, c)
        assert hi == pytest.approx(2 * ndtr(-np.sqrt(c) / sd), rel=5e-3)


def test_monte_carlo_follows_the_law():
    """2^16 oracle trials of the paper's polynomial against the exact law of S_16 and S_15:
    chi-square over the bins that hold at least 20 expected trials, and a moderate tail count."""
    n = 1 << 16
    mu, sd = F.PAPER_D
    r = F.fold_mc(F.PAPER_FOLD_COEF, mu, sd, 16, (0.3, 0.45), F.PAPER_NF, F.PAPER_PF, seed=11, trial0=0,
                  n_trials=n, hist=(-0.05, 0.15, 40))
    for row, k in ((0, 16), (1, 15)):
        g, p = F.sum_law(F.PAPER_FOLD_COEF, mu, sd, k)
        edges = np.concatenate([[-np.inf], np.linspace(-0.05, 0.15, 41), [np.inf]])
        want = np.array([F.law_mass(g, p, a, b) for a, b in zip(edges[:-1], edges[1:])]) * n
        got = r["hist"][row]
        m = want >= 20
        chi2 = (((got[m] - want[m]) ** 2) / want[m]).sum()
        assert chi2 < m.sum() + 5 * np.sqrt(2 * m.sum())
        lo, hi = F.tail_probs(g, p, -np.inf, 0.06)
        s = r["sk"] if k == 16 else r["sk1"]
        assert abs((s > 0.06).sum() - n * hi) < 5 * np.sqrt(n * hi) + 1


def test_paper_outlier_rate_under_the_normal_law():
    """Appendix C.2 found 53 sums of 16 outside N_f in 1e12 trials; with D = N(0.008, 0.034^2)
    (Section 6.1) the exact probability must be of the same order (within a factor of 2 either way:
    the normal law only approximates the real scores)."""
    gd = _golden("fold_design_paper.txt")
    g, p = F.sum_law(F.PAPER_FOLD_COEF, gd["d_mean"], gd["d_sd"], 16)
    lo, hi = F.tail_probs(g, p, *F.PAPER_NF)
    rate = gd["n_f_outliers"] / gd["trials"]
    assert rate / 2 < lo + hi < rate * 2
