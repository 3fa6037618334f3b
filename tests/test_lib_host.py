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
