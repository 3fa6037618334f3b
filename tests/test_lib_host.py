"""Host-side checks of libicm that need no GPU: the library builds and loads, exports every
entry point that include/icm.h declares, and its parameter logic (primes, bounds, layout sizes)
agrees with the oracle's independent reading."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2601_17561_gb300 import build as B
from paper_2601_17561_gb300 import icm as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return C.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "icm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(icm_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def _params(**kw):
    base = dict(O.TINY)
    base.update(kw)
    return C.icm_params(log_n_db=base["log_n_db"], log_n_q=base["log_n_q"], n_limbs=base["n_limbs"],
                        n_limbs_q=base["n_limbs_q"], prime_bits=base["prime_bits"], code_bits=12800, d2=1 << 14,
                        rho=31, fold_k=16, hamming_weight=512, log2_delta=base["log2_delta"], noise_eta=21,
                        seed=base["seed"])


@pytest.mark.parametrize("cfg", [O.TINY, O.PAPER])
def test_primes_agree_with_oracle_rule(lib, cfg):
    ctx = C.icm_ctx_create(_params(**cfg))
    try:
        got = C.icm_ctx_primes(ctx, cfg["n_limbs"])
    finally:
        C.icm_ctx_destroy(ctx)
    assert got == O.primes(cfg["prime_bits"], cfg["n_limbs"])


@pytest.mark.parametrize("cfg", [O.TINY, O.PAPER])
def test_crt_moduli_cover_the_product_range(lib, cfg):
    """The CRT forms' small moduli: odd, below 2^8, pairwise coprime, and their product exceeds
    twice the largest |sum of K centred residue products| (so the CRT value is the exact integer),
    with at least 2 bits to spare (|C| / M <= 1/8, against a fixed-point error below 2^-12 in the
    recombination's rounded quotient)."""
    import math
    ctx = C.icm_ctx_create(_params(**cfg))
    try:
        mods = C.icm_ctx_crt_moduli(ctx)
        q = C.icm_ctx_primes(ctx, cfg["n_limbs"])
    finally:
        C.icm_ctx_destroy(ctx)
    K = (1 << 14) + (1 << cfg["log_n_q"])
    assert all(m % 2 == 1 and 3 <= m < 256 for m in mods)
    assert all(math.gcd(a, b) == 1 for i, a in enumerate(mods) for b in mods[i + 1:])
    bound = K * ((max(q) - 1) // 2) ** 2
    assert math.prod(mods) > 2 * bound * 4
    # greedy from 255 down: dropping the smallest modulus no longer covers the range with margin
    assert math.prod(mods[:-1]) < 2 * (bound + 1) * 4 * 2
    if cfg is O.PAPER:
        assert len(mods) == 18


@pytest.mark.parametrize("cfg", [O.TINY, O.PAPER])
def test_crt_recombination_rule(lib, cfg):
    """The recombination's rule, in exact integers over the library's moduli: with
    y_i = (M/m_i)^-1 mod m_i, sum_i c_i y_i (M/m_i) - kappa M recovers every centred C with
    |C| <= M/8 (the margin the moduli are chosen with, C at +-M/8 included) when kappa is rounded
    from the fixed-point sum sum_i c_i round(2^19 y_i / m_i), which stays below 2^32."""
    import math
    ctx = C.icm_ctx_create(_params(**cfg))
    try:
        mods = C.icm_ctx_crt_moduli(ctx)
    finally:
        C.icm_ctx_destroy(ctx)
    M = math.prod(mods)
    yinv = [pow((M // m) % m, -1, m) for m in mods]
    r19 = [((y << 19) + m // 2) // m for m, y in zip(mods, yinv)]
    rng = np.random.default_rng(11)
    cases = [M // 8, -(M // 8), 0, 1, -1] + [int(v) for v in rng.integers(-(1 << 62), 1 << 62, size=300)]
    cases += [(M // 8) * int(f) // 1000 for f in rng.integers(-1000, 1001, size=300)]
    for Cv in cases:
        c = [Cv % m for m in mods]
        T = sum(ci * ri for ci, ri in zip(c, r19))
        assert T < 1 << 32
        kappa = (T + (1 << 18)) >> 19
        assert sum(ci * yi * (M // m) for ci, yi, m in zip(c, yinv, mods)) - kappa * M == Cv


@pytest.mark.parametrize("cfg", [O.TINY, O.PAPER])
def test_slot_database_size(lib, cfg):
    """A slot-encoded chunk holds N_db/2 templates per block (one per slot), all blocks full:
    M = N_db + ceil(n_db / (N_db/2)) N_db rows of L x K words."""
    ctx = C.icm_ctx_create(_params(**cfg))
    try:
        N = 1 << cfg["log_n_db"]
        K = (1 << 14) + (1 << cfg["log_n_q"])
        for n_db in (1, N // 2, N // 2 + 1, 3 * N + 5):
            nbytes, m = C.icm_db_bytes_slots(ctx, n_db)
            blocks = -(-n_db // (N // 2))
            assert m == N + blocks * N
            assert nbytes == cfg["n_limbs"] * m * K * 8
    finally:
        C.icm_ctx_destroy(ctx)


def test_bounds_rejected(lib):
    # Delta too large: the message wraps modulo Q_db
    with pytest.raises(C.IcmError) as e:
        C.icm_ctx_create(_params(log2_delta=45))
    assert e.value.status == C.ICM_EBOUND
    # Delta too small: noise exceeds Q' Delta / 2 when Q' is a single small prime
    with pytest.raises(C.IcmError) as e:
        C.icm_ctx_create(_params(n_limbs=2, log2_delta=2, prime_bits=30))
    assert e.value.status == C.ICM_EBOUND
    # unsupported / invalid
    with pytest.raises(C.IcmError) as e:
        C.icm_ctx_create(_params(n_limbs_q=3, n_limbs=5))
    assert e.value.status == C.ICM_EUNSUPPORTED
    with pytest.raises(C.IcmError) as e:
        C.icm_ctx_create(_params(prime_bits=61))
    assert e.value.status == C.ICM_EINVAL
    assert C.icm_status_str(C.ICM_EBOUND) == "bound violated"


@pytest.mark.parametrize("n_db", [0, 1, 256, 4066, 4067, 4096, 4097, 3 * 4096, 3 * 4096 + 17])
def test_db_layout_sizes_match_oracle(lib, n_db):
    ctx = C.icm_ctx_create(_params())
    try:
        nbytes, m = C.icm_db_bytes(ctx, n_db)
        ct = C.icm_query_ct_bytes(ctx, 4)
        op = C.icm_query_op_bytes(ctx, 4, C.ICM_FORM_U64)
    finally:
        C.icm_ctx_destroy(ctx)
    ids = O.db_layout(n_db, 1 << 12, 31)
    assert m == len(ids)
    K = (1 << 14) + (1 << 12)
    assert nbytes == 3 * m * K * 8
    assert ct == 1 * 4 * 31 * K * 8 and op == 3 * 4 * 31 * K * 8


def test_paper_shape_sizes(lib):
    """Section 6.2.1 sizes: 7 * 2^14 templates in 7 full blocks of N_db = 2^14 rows plus the a-part
    (M = 131072), K = 2^14 + 2^13; 8 u64 limbs -> 206 GB resident."""
    ctx = C.icm_ctx_create(_params(**O.PAPER))
    try:
        nbytes, m = C.icm_db_bytes(ctx, 7 * (1 << 14))
    finally:
        C.icm_ctx_destroy(ctx)
    assert m == 131072
    assert nbytes == 8 * 131072 * 24576 * 8


# ----------------------------------------------------------------------------- folding-polynomial check

@pytest.mark.parametrize("lo,hi", [(0.3, 0.45), (-0.25, 0.2), (-0.3, 1.0), (0.1, 0.1), (-0.1, -0.05), (0.257, 0.496)])
def test_fold_poly_range_agrees_with_oracle(lib, lo, hi):
    """The library's range of f over P (ends and sign changes of f') against the oracle's
    (roots of f' by numpy's companion matrix)."""
    from oracle import folding as F
    from paper_2601_17561_gb300 import folding as G
    got = C.icm_fold_poly_range(G.FOLD_COEF_K16, lo, hi)
    want = F.poly_range(F.PAPER_FOLD_COEF, lo, hi)
    assert got == pytest.approx(want, rel=1e-12, abs=1e-15)
    # a quartic with two interior minima and one interior maximum
    q = (0.0, 0.0, -2.0, 0.0, 1.0)                      # x^4 - 2 x^2: min -1 at +-1, max 0 at 0
    assert C.icm_fold_poly_range(q, -1.5, 1.2) == pytest.approx(F.poly_range(q, -1.5, 1.2), abs=1e-12)


def _mc_args(**kw):
    from paper_2601_17561_gb300 import folding as G
    coef = kw.pop("coef", G.FOLD_COEF_K16)
    cf = (ctypes.c_double * len(coef))(*coef)
    base = dict(coef=ctypes.cast(cf, ctypes.c_void_p), degree=len(coef) - 1, k=16, mu=0.008, sigma=0.034,
                nf_lo=-0.13, nf_hi=0.33, pf_lo=0.4, pf_hi=3.8, pos_lo=0.3, pos_hi=0.45, hist_lo=0.0, hist_hi=0.0,
                n_bins=0, accumulate=0, seed=1, trial0=0, n_trials=16)
    base.update(kw)
    return C.icm_fold_mc_args(**base), cf


@pytest.mark.parametrize("bad", [dict(degree=16), dict(k=0), dict(k=33), dict(sigma=0.0), dict(sigma=float("nan")),
                                 dict(nf_lo=1.0, nf_hi=0.0), dict(pf_lo=4.0), dict(pos_lo=0.5, pos_hi=0.4),
                                 dict(n_bins=8193), dict(n_bins=10, hist_lo=1.0, hist_hi=1.0),
                                 dict(trial0=2**64 - 4, n_trials=8)])
def test_fold_mc_rejects_bad_arguments(lib, bad):
    """Rejected before any device work (no GPU needed): bad degree, k, law, intervals, histogram
    and a trial range that wraps around 2^64."""
    import torch
    if torch.cuda.is_available():                               # real buffers where a GPU exists
        buf = torch.zeros(2 * 8200, dtype=torch.int64, device="cuda")
        counts, hist, odd = buf.data_ptr(), buf.data_ptr() + 64, buf.data_ptr() + 4
    else:                                                       # never dereferenced: rejected first
        counts, hist, odd = 8, 16, 12
    a, keep = _mc_args(**bad)
    with pytest.raises(C.IcmError) as e:
        C.icm_fold_mc(a, counts, hist if a.n_bins else None, None, 0)
    assert e.value.status == C.ICM_EINVAL
    a, keep = _mc_args()
    with pytest.raises(C.IcmError) as e:
        C.icm_fold_mc(a, None, None, None, 0)                   # no counts buffer
    assert e.value.status == C.ICM_EINVAL
    with pytest.raises(C.IcmError) as e:
        C.icm_fold_mc(a, odd, None, None, 0)                    # misaligned counts
    assert e.value.status == C.ICM_EINVAL


# ----------------------------------------------------------------------------- p^2 form (plain product)

def test_p2_form_workspace_and_moduli(lib):
    """ICM_FORM_I8_P2 takes moduli p^2 of odd p <= 253 (the paper's Q = prod p^2, Section 6.2.2) and
    two int8 digit planes of the right operand; other moduli are rejected before any device work."""
    assert C.icm_ppmm_workspace_bytes(C.ICM_FORM_I8_P2, 3, 100, 37, 1000) == 3 * 2 * 37 * 1024
    for bad in ([127 * 127 + 2], [255 * 255], [1], [127 * 127, 35], [2 * 2], [254 * 254]):
        with pytest.raises(C.IcmError) as e:
            C.icm_ppmm(C.ICM_FORM_I8_P2, bad, len(bad), None, None, None, 0, 0, 0, stream=0)
        assert e.value.status == C.ICM_EINVAL, bad


def test_paper_p2_modulus():
    """Section 6.2.2: Q = prod of p^2 over the primes 127 <= p <= 253 gives 24 moduli, 48 int8
    matrices per operand, and about 2^357 (the paper's target; the product is 2^360.8)."""
    ps = [p for p in range(127, 254) if all(p % d for d in range(2, int(p ** 0.5) + 1))]
    assert len(ps) == 24 and 2 * len(ps) == 48
    bits = sum(2 * np.log2(p) for p in ps)
    assert 357 <= bits < 362


def test_p2_digit_split_exhaustive():
    """The p^2 form's digit split, as the kernels compute it (x1 = round(x * fl(1/p)) in fp32, x0 =
    x - p x1, one correction step): for every odd p <= 253 and every residue of p^2, |x0| <= (p-1)/2,
    |x1| <= 126 (int8 operands) and x0 + p x1 is the centred lift x."""
    worst = 0
    for p in range(3, 254, 2):
        q = p * p
        v = np.arange(q, dtype=np.int64)
        x = np.where(v > q // 2, v - q, v)
        ip = np.float32(1.0) / np.float32(p)
        x1 = np.rint(x.astype(np.float32) * ip).astype(np.int64)
        x0 = x - x1 * p
        h = (p - 1) // 2
        hi, lo = x0 > h, x0 < -h
        x0 = np.where(hi, x0 - p, np.where(lo, x0 + p, x0))
        x1 = np.where(hi, x1 + 1, np.where(lo, x1 - 1, x1))
        assert np.all(np.abs(x0) <= h) and np.all(x0 + p * x1 == x), p
        worst = max(worst, int(np.abs(x1).max()))
    assert worst == 126
