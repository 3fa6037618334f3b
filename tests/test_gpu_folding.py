"""GPU parity of the folding-polynomial check (icm_fold_mc, Section 4.1.2 definition, Appendix C.2
experiments) against the oracle on the same Philox streams.

Tolerance.  The kernel computes the deviates, f and the sums in fp32, the oracle in fp64.  Per
deviate: u1 (or 1 - u1) is rounded to 24 bits and ln u1 = log1p(.) + e ln 2 is evaluated with one
rounding per step, so ln u1 and the radius r = sqrt(-2 ln u1) carry relative errors below 3e-7;
u2 is rounded to a multiple of 2^-23, so the angle errs by at most 3.7e-7 rad; with r <= 9.5,
|dz| <= 9.5 (3e-7 + 3.7e-7) < 7e-6, the score moves by sigma |dz| < 2.4e-7 (sigma = 0.034) and f by
at most |f'| 2.4e-7 <= 2.4e-6 over |x| <= 0.4; the fp32 coefficients and Horner rounding add below
3e-6, and each partial sum of |S| < 8 rounds by at most ulp(8) = 9.5e-7.  A sum over n <= 63
values therefore differs by at most n 6.4e-6 <= 4e-4 = TOL.  A trial whose oracle sum lies within
TOL of a threshold or bin edge may be decided either way, so counts and histograms are compared up
to those trials, and exactly against the GPU's own fp32 sums."""
import numpy as np
import pytest
import torch

from oracle import folding as F
from paper_2601_17561_gb300 import build as B
from paper_2601_17561_gb300 import folding as G

pytestmark = pytest.mark.gpu
TOL = 4e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _run(n, **kw):
    r = G.fold_mc(n, **kw)
    torch.cuda.synchronize()
    return (r.counts.cpu().numpy(), None if r.hist is None else r.hist.cpu().numpy(),
            None if r.sums is None else r.sums.cpu().numpy())


@pytest.mark.parametrize("k,n,trial0", [(16, 3000, 12345), (1, 517, 0), (2, 1000, 7), (31, 700, 99),
                                        (16, 300, 2**40 + 3), (15, 300, 2**63 + 5)])
def test_per_trial_sums_match_oracle(k, n, trial0):
    """Every trial's S_k and S_{k-1}; ragged trial counts, odd k, counters above 2^32 and 2^63."""
    law = G.NEG_LAW
    _, _, s = _run(n, k=k, seed=7, trial0=trial0, want_sums=True)
    o = F.fold_mc(F.PAPER_FOLD_COEF, *law, k, (0.3, 0.45), F.PAPER_NF, F.PAPER_PF, 7, trial0, n)
    assert np.abs(s[:, 0] - o["sk"]).max() < TOL
    assert np.abs(s[:, 1] - o["sk1"]).max() < TOL
    if k == 1:
        assert np.all(s[:, 1] == 0)


def _ambiguous(x, edges):
    x = np.asarray(x)[:, None]
    return np.any(np.abs(x - np.asarray(edges)[None, :]) < TOL, axis=1)


def test_counts_and_histograms_match_oracle():
    """Thresholds inside the bulk of the laws and a narrow P (f varies by 0.004 over it) so that
    all six counters are large."""
    n, seed, t0 = (1 << 16) + 77, 3, 1000
    nf, pos = (0.0, 0.03), (0.3, 0.3005)
    fmin, fmax = F.poly_range(F.PAPER_FOLD_COEF, *pos)
    pf = (fmin + 0.01, fmin + 0.02)
    hist = (-0.02, 0.08, 50)
    c, h, s = _run(n, nf=nf, pf=pf, pos=pos, seed=seed, trial0=t0, hist=hist, want_sums=True)
    o = F.fold_mc(F.PAPER_FOLD_COEF, *F.PAPER_D, 16, pos, nf, pf, seed, t0, n, hist=hist)
    assert np.all(o["counts"] > 1000) and np.all(o["counts"] < n - 1000)
    # against the oracle, up to trials within TOL of a threshold
    amb_k = _ambiguous(o["sk"], nf).sum()
    amb_1 = _ambiguous(o["sk1"], [pf[0] - fmin, pf[1] - fmin, pf[0] - fmax, pf[1] - fmax]).sum()
    assert np.all(np.abs(c[:2] - o["counts"][:2]) <= amb_k)
    assert np.all(np.abs(c[2:] - o["counts"][2:]) <= amb_1)
    edges = np.linspace(hist[0], hist[1], hist[2] + 1)
    for row, key in ((0, "sk"), (1, "sk1")):
        assert h[row].sum() == n
        assert np.abs(h[row] - o["hist"][row]).sum() <= 2 * _ambiguous(o[key], edges).sum()
    # exactly against the GPU's own fp32 sums
    from paper_2601_17561_gb300 import icm as C
    lmin, lmax = C.icm_fold_poly_range(G.FOLD_COEF_K16, *pos)   # the range the kernel was given
    f32 = np.float32
    sk, sk1 = s[:, 0], s[:, 1]
    mn, mx = f32(lmin) + sk1, f32(lmax) + sk1
    own = [(sk < f32(nf[0])).sum(), (sk > f32(nf[1])).sum(), (mn < f32(pf[0])).sum(), (mn > f32(pf[1])).sum(),
           (mx < f32(pf[0])).sum(), (mx > f32(pf[1])).sum()]
    assert list(c) == own
    scale = f32(hist[2] / (hist[1] - hist[0]))
    for row, v in ((0, sk), (1, sk1)):
        b = np.floor(np.clip((v - f32(hist[0])) * scale, f32(-1), f32(hist[2]))).astype(np.int64) + 1
        assert np.array_equal(np.bincount(b, minlength=hist[2] + 2), h[row])


def test_ranges_continue_one_run():
    """Consecutive trial ranges with accumulate give the single run's counts, histogram and sums."""
    n, hist = 100_000, (-0.02, 0.08, 64)
    kw = dict(nf=(0.0, 0.03), pf=(0.69, 2.65), seed=9, hist=hist)
    c, h, s = _run(n, want_sums=True, **kw)
    r = G.fold_mc(n // 3, trial0=0, **kw)
    G.fold_mc(n - n // 3, trial0=n // 3, out=r, accumulate=True, **kw)
    torch.cuda.synchronize()
    assert np.array_equal(r.counts.cpu().numpy(), c) and np.array_equal(r.hist.cpu().numpy(), h)
    _, _, s2 = _run(n - n // 3, trial0=n // 3, want_sums=True, **kw)
    assert np.array_equal(s2, s[n // 3:])


@pytest.mark.parametrize("coef", [(0.25,), (0.0, 1.0), tuple(np.random.default_rng(4).normal(0, 0.5, 16))])
def test_other_degrees(coef):
    """Degree 0 (S_k = k c0), degree 1 (S_k = sum x_i) and degree 15 (the second kernel instance)."""
    n = 2000
    _, _, s = _run(n, coef=coef, seed=5, want_sums=True)
    o = F.fold_mc(coef, *F.PAPER_D, 16, (0.3, 0.45), F.PAPER_NF, F.PAPER_PF, 5, 0, n)
    scale = max(1.0, float(np.abs(o["sk"]).max()))
    assert np.abs(s[:, 0] - o["sk"]).max() < TOL * scale
    assert np.abs(s[:, 1] - o["sk1"]).max() < TOL * scale


def test_zero_trials_and_overwrite():
    r = G.fold_mc(5000, nf=(0.0, 0.03), hist=(-0.02, 0.08, 8))
    G.fold_mc(0, nf=(0.0, 0.03), hist=(-0.02, 0.08, 8), out=r)
    torch.cuda.synchronize()
    assert int(r.counts.abs().sum()) == 0 and int(r.hist.sum()) == 0


def test_full_size_against_the_exact_law():
    """2^32 trials of the paper's experiment in the benchmark's launch configuration: the
    histograms of S_16 and S_15 against the exact laws (chi-square over bins with at least 20
    expected trials), and the paper's N_f outliers against their exact expectation (Poisson)."""
    n, hist = 1 << 32, (-0.05, 0.15, 40)
    pos = (0.3, 0.45)
    c, h, _ = _run(n, pos=pos, seed=2026, hist=hist)
    edges = np.concatenate([[-np.inf], np.linspace(hist[0], hist[1], hist[2] + 1), [np.inf]])
    for row, k in ((0, 16), (1, 15)):
        g, p = F.sum_law(F.PAPER_FOLD_COEF, *F.PAPER_D, k)
        want = np.array([F.law_mass(g, p, a, b) for a, b in zip(edges[:-1], edges[1:])]) * n
        m = want >= 20
        chi2 = (((h[row][m] - want[m]) ** 2) / want[m]).sum()
        assert chi2 < m.sum() + 5 * np.sqrt(2 * m.sum()), (k, chi2, m.sum())
        if k == 16:
            lo, hi = F.tail_probs(g, p, *F.PAPER_NF)
            lam = n * (lo + hi)
            assert c[0] + c[1] <= lam + 6 * np.sqrt(lam) + 6
