"""GPU parity of the slot-encoded database and of the normalisation (Section 2.2.1 Ecd_slot,
Section 2.3, Algorithm 2's ct (.) mu) against the oracle (oracle/slots.py).

Ring 2^11 for the database (1,024 templates per block), the paper's query side (N_q = 2^13,
K = 24,576), four primes below 2^60 (L_q = 2), Delta 2^60, database slot scale 2^16, mu scale
2^36; 1,500 templates (two blocks, the second partial) and one query eye (31 rotations).

Rounding of fp64 values to integers (the encoding of the database entries and of mu) is the one
step where two correct implementations may differ: only where the unrounded value lies within a
hair of a half-integer.  The tests count those positions from the oracle's unrounded values
(expected: none) and require bit-identical integers, database rows, CCMM and rescaled residues
(the rescaling's own window rule) and normalised ciphertexts; decoded distances must be within
2^-10 of the fp64 cleartext distances."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import slots as OS
from paper_2601_17561_gb300 import build as B
from paper_2601_17561_gb300 import engine as E
from paper_2601_17561_gb300 import icm as C
from paper_2601_17561_gb300 import synth

from rescale_check import check_rescaled

pytestmark = pytest.mark.gpu

CFG = dict(log_n_db=11, log_n_q=13, n_limbs=4, n_limbs_q=2, prime_bits=60, log2_delta=60, seed=7)
S_DB, S_MU = 16, 36
N_DB = 1500
# fp64 evaluations of the same rounded quantity agree to ~1e-15 of its magnitude (database
# entries below 2^13, mu coefficients below 2^23): windows of 1e-8 and 1e-6 around the
# half-integers hold every value two correct evaluations could round differently
TIE_W, TIE_MU = 1e-8, 1e-6


def _u64(t: torch.Tensor, shape):
    n = int(np.prod(shape))
    return t[: n * 8].view(torch.int64).cpu().numpy().view(np.uint64).reshape(shape)


def _from_digit_form(z: np.ndarray, q) -> np.ndarray:
    B_ = np.uint64(0x8080808080808080)
    c = (z ^ B_) - B_
    out = np.empty_like(z)
    for l, ql in enumerate(q):
        cl = c[l].view(np.int64)
        out[l] = np.where(cl < 0, (cl + np.int64(ql)).view(np.uint64), c[l])
    return out


def _ties(x: np.ndarray, tie: float) -> int:
    f = np.abs(x - np.floor(x) - 0.5)
    return int(np.sum(f < tie))


@pytest.fixture(scope="module")
def setup():
    B.build()
    P = O.Params(h=16, **CFG)
    N = P.ndb
    W = synth.make_workload(n_eyes=1, n_db=N_DB, seed=8, planted_frac=0.05)
    # oracle
    w_un = OS.slot_db_messages(W.db_codes, W.db_masks, N, P.d2, S_DB, unrounded=True)
    msg = np.rint(w_un).astype(np.int64)
    ids = OS.slot_layout(N_DB, N)
    rows = np.zeros((len(ids), P.d2), np.int64)
    rows[N:] = msg
    A = O.db_rows_from_messages(P, rows, ids)
    Bq = O.query_extend(P, O.query_encrypt(P, W.q_codes, W.q_masks, W.eye_ids))
    Cm = O.ppmm(P.q, A, Bq)
    R = O.rescale(P, Cm)
    rc, rm = O.rotated_templates(W.q_codes, W.q_masks, P.rho)
    num, den = O.hd_counts(rc, rm, O.unpack(W.db_codes), O.unpack(W.db_masks))
    mu_un = OS.mu_polys(den, N_DB, N, S_MU, unrounded=True)
    mu = np.rint(mu_un).astype(np.int64)
    norm = OS.normalize(P, R, mu)
    # GPU
    eng = E.Engine(hamming_weight=16, **CFG).keygen()
    db = eng.encrypt_db_slots(W.db_codes, W.db_masks, log2_scale=S_DB)
    ct = eng.encrypt_query(W.q_codes, W.q_masks, W.eye_ids)
    torch.cuda.synchronize()
    return dict(P=P, W=W, A=A, Cm=Cm, R=R, num=num, den=den, mu=mu, norm=norm, eng=eng, db=db, ct=ct,
                ties_w=_ties(w_un, TIE_W), ties_mu=_ties(mu_un, TIE_MU))


def test_no_rounding_ties_in_the_workload(setup):
    """The oracle's unrounded database entries and mu coefficients keep clear of half-integers,
    so the bit-exact comparisons below are well defined."""
    assert setup["ties_w"] == 0 and setup["ties_mu"] == 0


def test_slot_database_rows_bit_exact(setup):
    P, db = setup["P"], setup["db"]
    L, M, K = P.n_limbs, db.m_rows, P.K
    assert M == setup["A"].shape[1]
    got = _from_digit_form(_u64(db.buf, (L, M, K)), P.q)
    assert np.array_equal(got, setup["A"])


@pytest.mark.parametrize("form,variant", [("u64", None), ("f16_crt", 2)])
def test_slot_ccmm_and_rescale(setup, form, variant):
    """The CCMM of the slot-encoded chunk (any form; the fp16 CRT form on the tcgen05 kernel) is
    bit-exact to the oracle's, and its rescaling by Q' follows the rescaling rule."""
    P, eng, db = setup["P"], setup["eng"], setup["db"]
    if variant is not None:
        C.icm_ctx_set_variant(eng.ctx, variant)
    try:
        q = eng.prepare(setup["ct"], 1, form)
        s = eng.match(db, q)
        torch.cuda.synchronize()
        C.icm_device_status(True)
    finally:
        C.icm_ctx_set_variant(eng.ctx, 0)
    assert np.array_equal(s.residues(), setup["Cm"])
    r = eng.rescale(s)
    torch.cuda.synchronize()
    assert check_rescaled(P, r.residues(), setup["Cm"]) == 0
    setup["rescaled_" + form] = r


def _normalized(setup):
    eng, W = setup["eng"], setup["W"]
    r = setup.get("rescaled_u64")
    if r is None:
        s = eng.match(setup["db"], eng.prepare(setup["ct"], 1, "u64"))
        r = eng.rescale(s)
    qm = torch.from_numpy(np.ascontiguousarray(W.q_masks)).to(eng.device)
    dm = torch.from_numpy(np.ascontiguousarray(W.db_masks)).to(eng.device)
    out = eng.normalize(r, qm, dm, S_MU)
    torch.cuda.synchronize()
    return r, out


def test_normalize_bit_exact(setup):
    """ct (.) mu of every block (mask overlaps, mu encoding, negacyclic NTT products) equals the
    oracle's schoolbook products with the oracle's mu."""
    P = setup["P"]
    _, out = _normalized(setup)
    want = setup["norm"]
    got = _u64(out, want.shape)
    assert np.array_equal(got, want)


def test_decoded_distances_within_tolerance(setup):
    """Decrypted and decoded (FFT) normalised scores give fractional Hamming distances within 2^-10
    of the fp64 cleartext distances for every (rotation, template) pair, and within 1e-9 of the
    oracle's own decoding of the same ciphertexts."""
    P, eng = setup["P"], setup["eng"]
    r, out = _normalized(setup)
    hd = eng.decrypt_slots(r, out, S_MU).cpu().numpy()
    ref = O.fractional_hd(setup["num"], setup["den"])
    assert hd.shape == ref.shape
    err = np.abs(hd - ref).max()
    assert err < 2.0 ** -10
    assert err < 1e-4
    s_or = OS.decoded_scores(P, setup["norm"], S_DB, S_MU)[:, :N_DB]
    assert np.abs(hd - OS.hd_from_scores(s_or)).max() < 1e-9


def test_slot_argument_checks(setup):
    eng, W = setup["eng"], setup["W"]
    s = eng.match(setup["db"], eng.prepare(setup["ct"], 1, "u64"))
    with pytest.raises(C.IcmError):              # integer decryption does not apply to slot scores
        eng.decrypt(s)
    qm = torch.from_numpy(np.ascontiguousarray(W.q_masks)).to(eng.device)
    dm = torch.from_numpy(np.ascontiguousarray(W.db_masks)).to(eng.device)
    with pytest.raises(C.IcmError):              # normalisation wants the rescaled result
        C.icm_normalize_bytes(s.handle)
    r = eng.rescale(s)
    with pytest.raises(C.IcmError) as e:         # Delta 2^16 2^44 exceeds Q / 4
        eng.normalize(r, qm, dm, 44)
    assert e.value.status == C.ICM_EBOUND
    with pytest.raises(C.IcmError):              # database slot scale out of range
        eng.encrypt_db_slots(W.db_codes[:10], W.db_masks[:10], log2_scale=25)
    torch.cuda.synchronize()
