"""Cleartext check of a folding polynomial on the GPU (icm_fold_mc): the Monte Carlo experiments
that validate the folding design (Section 4.1.2 definition, Appendix C.2 experiments).  Argument
marshalling only; the trials run in the library's kernel.

The constants below restate the paper's parameters: the degree-7 folding polynomial for k = 16
with N_f = [-0.13, 0.33] and P_f = [0.4, 3.8] (Appendix C.2), and the law of negative scores
N(0.008, 0.034^2) (Section 6.1).  The positive-score interval P is not given in the paper; callers
pass their own.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import icm as C

# Appendix C.2: coefficients of x^0 .. x^7.
FOLD_COEF_K16 = (0.004105, -0.173510, -2.528271, 24.347349, 124.161550, -412.746212, 376.961251, 106.553952)
FOLD_K = 16
N_F = (-0.13, 0.33)
P_F = (0.4, 3.8)
NEG_LAW = (0.008, 0.034)        # Section 6.1


@dataclass
class FoldMcResult:
    counts: torch.Tensor          # int64 [6] on the device (see icm_fold_mc)
    hist: torch.Tensor | None     # int64 [2][n_bins + 2]
    sums: torch.Tensor | None     # float32 [n_trials][2]


def fold_mc(n_trials: int, *, coef=FOLD_COEF_K16, k: int = FOLD_K, law=NEG_LAW, nf=N_F, pf=P_F,
            pos=(0.3, 0.45), seed: int = 1, trial0: int = 0, hist=None, want_sums: bool = False,
            out: FoldMcResult | None = None, accumulate: bool = False, stream=None) -> FoldMcResult:
    """Enqueue trials trial0 .. trial0 + n_trials - 1 on `stream`; hist = (lo, hi, n_bins)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    nb = 0 if hist is None else int(hist[2])
    if out is None:
        out = FoldMcResult(torch.zeros(6, dtype=torch.int64, device=dev),
                           torch.zeros(2, nb + 2, dtype=torch.int64, device=dev) if nb else None,
                           torch.empty(n_trials, 2, dtype=torch.float32, device=dev) if want_sums else None)
    cf = (ctypes.c_double * len(coef))(*coef)
    a = C.icm_fold_mc_args(coef=ctypes.cast(cf, ctypes.c_void_p), degree=len(coef) - 1, k=k, mu=law[0],
                           sigma=law[1], nf_lo=nf[0], nf_hi=nf[1], pf_lo=pf[0], pf_hi=pf[1], pos_lo=pos[0],
                           pos_hi=pos[1], hist_lo=hist[0] if nb else 0.0, hist_hi=hist[1] if nb else 0.0,
                           n_bins=nb, accumulate=int(accumulate), seed=seed, trial0=trial0, n_trials=n_trials)
    C.icm_fold_mc(a, out.counts, out.hist, out.sums, stream)
    return out
