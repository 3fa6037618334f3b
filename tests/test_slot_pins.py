"""Pins for the oracle of the slot-encoded database and of the normalisation (oracle/slots.py):
closed forms of Ecd_slot (Section 2.2.1), the evaluation definition of Dcd, the ring
homomorphism between the negacyclic product and slot-wise products, brute-force negacyclic
products, and the whole chain (slot-encoded database, CCMM, rescaling, normalisation, decryption,
decoding) against the fp64 cleartext distances within 2^-10.  CPU only."""
import numpy as np
import pytest

import oracle as O
from oracle import slots as OS
from paper_2601_17561_gb300 import synth

# ring 2^11 for the database (1,024 templates per block), the paper's query side, four primes
# below 2^60 (L_q = 2): Delta 2^60, database slot scale 2^16, mu scale 2^36 (2^112 < Q / 2)
N3 = O.Params(log_n_db=11, log_n_q=13, n_limbs=4, n_limbs_q=2, prime_bits=60, h=16, log2_delta=60, seed=7)
S_DB, S_MU = 16, 36


def test_slot_exponents_cover_the_odd_residues():
    """{5^j} (j < N/2) and their negatives are the N odd residues modulo 2N, and 5^j = 1 mod 4
    (so the slots are the roots zeta^r with r = 1 mod 4)."""
    for N in (4, 16, 2048):
        e = OS.slot_exponents(N)
        assert len(set(e.tolist())) == N // 2
        assert all(v % 4 == 1 for v in e)
        both = set(e.tolist()) | {(-v) % (2 * N) for v in e}
        assert both == set(range(1, 2 * N, 2))


def test_encode_of_monomials_closed_form():
    """P = X^m has slots zeta^(5^j m): encoding those values gives back the unit vector e_m."""
    for N in (8, 64):
        e = OS.slot_exponents(N)
        for m in (0, 1, N // 2 - 1, N // 2, N - 1):
            z = np.exp(1j * np.pi * (e * m % (2 * N)) / N)
            p = OS.encode(z, N)
            want = np.zeros(N)
            want[m] = 1.0
            assert np.abs(p - want).max() < 1e-12, (N, m)


def test_encode_of_constant_slots_is_the_constant_polynomial():
    for N in (16, 2048):
        p = OS.encode(np.full(N // 2, 0.75), N)
        want = np.zeros(N)
        want[0] = 0.75
        assert np.abs(p - want).max() < 1e-12


def test_decode_inverts_encode():
    """Dcd by plain evaluation of P at zeta^(5^j) recovers the slots that Ecd was given (complex
    and real inputs; the two functions use independent formulas)."""
    rng = np.random.default_rng(1)
    for N in (16, 2048):
        z = rng.normal(size=N // 2) + 1j * rng.normal(size=N // 2)
        assert np.abs(OS.decode(OS.encode(z, N), N) - z).max() < 1e-9
        r = rng.normal(size=N // 2)
        assert np.abs(OS.decode_real(OS.encode(r, N), N) - r).max() < 1e-9


def test_negacyclic_mulmod_brute_force_and_monomials():
    rng = np.random.default_rng(2)
    q = (1 << 59) + 55           # any odd modulus below 2^62 works for the schoolbook product
    N = 8
    a = rng.integers(0, q, N, dtype=np.uint64)
    b = rng.integers(0, q, N, dtype=np.uint64)
    want = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            v = int(a[i]) * int(b[j])
            if k < N:
                want[k] += v
            else:
                want[k - N] -= v
    assert [int(x) for x in O.negacyclic_mulmod(a, b, q)] == [w % q for w in want]
    # X^i X^j = X^(i+j), with X^N = -1
    N = 64
    for i, j in ((0, 5), (3, 60), (63, 63), (32, 32)):
        x = np.zeros(N, np.uint64); x[i] = 1
        y = np.zeros(N, np.uint64); y[j] = 1
        got = O.negacyclic_mulmod(x, y, q)
        want = np.zeros(N, np.uint64)
        k = i + j
        want[k % N] = 1 if k < N else q - 1
        assert np.array_equal(got, want)
    # commutative
    a = rng.integers(0, q, N, dtype=np.uint64)
    b = rng.integers(0, q, N, dtype=np.uint64)
    assert np.array_equal(O.negacyclic_mulmod(a, b, q), O.negacyclic_mulmod(b, a, q))


def test_slot_product_is_the_ring_product():
    """The canonical embedding is a ring homomorphism: Dcd(a * b) = Dcd(a) Dcd(b) slot-wise for
    integer polynomials multiplied in Z[X]/(X^N + 1) (computed modulo a prime large enough that
    nothing wraps).  Pins the negacyclic product and the choice of roots together."""
    rng = np.random.default_rng(3)
    N = 256
    q = O.primes(60, 1)[0]
    a = rng.integers(-1000, 1000, N)
    b = rng.integers(-1000, 1000, N)
    c = O.negacyclic_mulmod(a % q, b % q, q).astype(object)
    c = np.array([int(v) - q if int(v) > q // 2 else int(v) for v in c], np.float64)
    za, zb, zc = OS.decode(a, N), OS.decode(b, N), OS.decode(c, N)
    assert np.abs(zc - za * zb).max() < 1e-6 * np.abs(za * zb).max()


def test_slot_db_messages_single_template_closed_form():
    """One template in block 0 sits in slot 0, at zeta^1: its column k encodes to
    round(2^s (2/N) c'[k] cos(pi n / N)) for every coefficient n."""
    W = synth.make_workload(n_eyes=1, n_db=1, seed=4, planted_frac=0.0)
    N, s = 64, 10
    msg = OS.slot_db_messages(W.db_codes, W.db_masks, N, 1 << 14, s)
    assert msg.shape == (N, 1 << 14)
    c = O.cprime(O.unpack(W.db_codes), O.unpack(W.db_masks), 1 << 14)[0].astype(np.float64)
    n = np.arange(N)
    want = np.rint((2.0 ** s) * (2.0 / N) * np.cos(np.pi * n / N)[:, None] * c[None, :]).astype(np.int64)
    assert np.array_equal(msg, want)


def test_slot_db_messages_decode_to_the_templates():
    """Real parts of Dcd(W / 2^s) give back every template's c' within the rounding bound
    sum_n |e_n| <= N / 2 of the scaled coefficients (2 blocks, the second one partial)."""
    N, s, n_db = 64, 12, 40
    W = synth.make_workload(n_eyes=1, n_db=n_db, seed=5, planted_frac=0.0)
    msg = OS.slot_db_messages(W.db_codes, W.db_masks, N, 1 << 14, s)
    V = OS.slot_values(W.db_codes, W.db_masks, N, 1 << 14)
    assert V.shape == (2, N // 2, 1 << 14)
    for t in range(2):
        got = OS.decode_real(msg[t * N:(t + 1) * N].astype(np.float64) / 2.0 ** s, N)
        assert np.abs(got - V[t]).max() <= (N / 2) / 2.0 ** s
    assert not V[1, n_db - N // 2:].any()          # missing templates are empty slots


def test_mu_values():
    den = np.array([[10, 0, 4], [1, 2, 3]])
    v = OS.mu_values(den, 3, 8)
    assert v.shape == (2, 1, 4)
    assert np.allclose(v[0, 0], [0.1, 0.0, 0.25, 0.0])
    assert np.allclose(v[1, 0], [1.0, 0.5, 1 / 3, 0.0])


@pytest.fixture(scope="module")
def chain():
    """Slot-encoded database of 1,500 templates (two blocks of 1,024, the second partial), one
    query eye (31 rotations), CCMM, rescaling by Q', the oracle's own mask overlaps."""
    P, N = N3, N3.ndb
    n_db = 1500
    W = synth.make_workload(n_eyes=1, n_db=n_db, seed=8, planted_frac=0.05)
    msg = OS.slot_db_messages(W.db_codes, W.db_masks, N, P.d2, S_DB)
    ids = OS.slot_layout(n_db, N)
    rows = np.zeros((len(ids), P.d2), np.int64)
    rows[N:] = msg
    A = O.db_rows_from_messages(P, rows, ids)
    B = O.query_extend(P, O.query_encrypt(P, W.q_codes, W.q_masks, W.eye_ids))
    R = O.rescale(P, O.ppmm(P.q, A, B))
    rc, rm = O.rotated_templates(W.q_codes, W.q_masks, P.rho)
    num, den = O.hd_counts(rc, rm, O.unpack(W.db_codes), O.unpack(W.db_masks))
    return P, n_db, R, num, den


def test_slot_database_decodes_to_the_inner_products(chain):
    """Before the normalisation: decrypting and decoding every block (mu = 1, the constant
    polynomial) gives the cleartext inner products <c'_q, c'_db> within 0.25.  The database
    rounding dominates: each scaled coefficient is off by at most 1/2, so each slot by a sum of N
    independent terms of deviation sqrt(N / 12) / 2^16 = 2.0e-4, and an inner product sums ~11,500
    of them: deviation 0.021, and 0.25 is 12 deviations."""
    P, n_db, R, num, den = chain
    N = P.ndb
    nb = OS.slot_blocks(n_db, N)
    one = np.zeros((R.shape[1], nb, N), np.int64)
    one[:, :, 0] = 1
    z = OS.decoded_scores(P, OS.normalize(P, R, one), S_DB, 0)[:, :n_db]
    inner = O.inner_from_counts(num, den)
    assert np.abs(z - inner).max() < 0.25


def test_normalised_scores_within_paper_tolerance(chain):
    """The whole chain: normalised, decrypted and decoded scores give fractional Hamming
    distances within 2^-10 of the fp64 cleartext ones, for every (rotation, template) pair."""
    P, n_db, R, num, den = chain
    mu = OS.mu_polys(den, n_db, P.ndb, S_MU)
    s = OS.decoded_scores(P, OS.normalize(P, R, mu), S_DB, S_MU)[:, :n_db]
    hd = OS.hd_from_scores(s)
    ref = O.fractional_hd(num, den)
    err = np.abs(hd - ref).max()
    assert err < 2.0 ** -10
    assert err < 1e-4               # what the scales give (the tolerance is far above)
