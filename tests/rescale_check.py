"""Comparison of the library's rescaling by Q' with the oracle's exact rounded division.

The oracle computes x' = round(x / Q') mod Q on the exact integers (Section 2.2.2, Maintenance).
The CUDA kernel obtains the quotient by fast base conversion: its integer correction is the
nearest integer to sum_i yh_i / q_i, summed as L - L_q fixed-point fractions each short by less
than 2^-64, so it may round the other way only when x / Q' lies within (L - L_q) 2^-64 of a
half-integer.  There (and only there) the two results may differ by one unit modulo Q; every
other coefficient must be identical.
"""
import numpy as np

import oracle as O


def check_rescaled(P, got: np.ndarray, C: np.ndarray, max_window_frac: float = 1e-6) -> int:
    """Assert that `got` ([L_q][...] residues from the GPU) is the rescaling of the oracle's
    residues C ([L][...]): equal everywhere outside the fixed-point window, equal or one unit
    away inside it.  Returns the number of coefficients inside the window (expected: almost
    always 0; at most `max_window_frac` of all coefficients, plus one)."""
    want = O.rescale(P, C)
    assert got.shape == want.shape, (got.shape, want.shape)
    Lq = P.n_limbs_q
    g = got.reshape(Lq, -1)
    w = want.reshape(Lq, -1)
    num, den = O.rescale_half_distance(P, C)
    num = num.reshape(-1)
    bound = (P.n_limbs - Lq) * den                 # distance < (L - L_q) 2^-64  <=>  num 2^64 < bound
    window = np.array([int(n) << 64 for n in num], dtype=object) < bound
    window = window.astype(bool)
    differ = np.any(g != w, axis=0)
    assert not np.any(differ & ~window), \
        f"{int(np.sum(differ & ~window))} rescaled coefficients differ outside the rounding window"
    n_win = int(np.sum(window))
    assert n_win <= max_window_frac * g.shape[1] + 1, n_win
    for c in np.nonzero(window)[0]:
        # one unit away modulo Q, or equal
        ok = False
        for d in (0, 1, -1):
            if all(int(g[j, c]) == (int(w[j, c]) + d) % int(P.q[j]) for j in range(Lq)):
                ok = True
        assert ok, f"coefficient {c}: rescaled value is more than one unit from round(x / Q')"
    return n_win
