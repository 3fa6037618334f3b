"""Pins for the oracle: each oracle function checked against something other than itself --
published vectors, closed forms, brute force on tiny inputs, exact algebraic identities and the
decrypt(encrypt) identity.  CPU only."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2601_17561_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# a small parameter set: same code layout (d2 = 2^14), small rings so every check runs in seconds
SMALL = O.Params(log_n_db=6, log_n_q=5, n_limbs=3, n_limbs_q=1, prime_bits=50, h=16, log2_delta=26, seed=7)
SMALL2 = O.Params(log_n_db=6, log_n_q=5, n_limbs=4, n_limbs_q=2, prime_bits=60, h=16, log2_delta=60, seed=9)


def _golden_ints(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [int(x) for x in f.read().split("\n") if x and not x.startswith("#")]


# ----------------------------------------------------------------------------- generator

def test_splitmix64_published_vector():
    want = _golden_ints("splitmix64_seed1234567.txt")
    got = [O.lib().orc_sm64(1234567, i) for i in range(len(want))]
    assert got == want


def test_stream_keys_distinct():
    keys = {O.lib().orc_stream_key(1, k, a, b) for k in range(1, 7) for a in range(20) for b in range(8)}
    assert len(keys) == 6 * 20 * 8


def test_uniform_mod_range_and_uniformity():
    q = (1 << 50) - 27
    L = O.lib()
    assert L.orc_uniform_mod(0, q) == 0
    assert L.orc_uniform_mod((1 << 64) - 1, q) == q - 1
    xs = np.array([L.orc_uniform_mod(L.orc_sm64(5, i), q) for i in range(20000)], dtype=np.float64)
    assert xs.max() < q and xs.min() >= 0
    hist, _ = np.histogram(xs / q, bins=20, range=(0, 1))
    chi2 = ((hist - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 60  # 19 dof, p ~ 1e-6


def test_cbd_distribution():
    L = O.lib()
    ws = [L.orc_sm64(11, i) for i in range(40000)]
    e = np.array([L.orc_cbd(w, 21) for w in ws])
    # closed form for one word: popcount of 21 bits minus popcount of the next 21 bits
    w0 = ws[0]
    assert e[0] == bin(w0 & ((1 << 21) - 1)).count("1") - bin((w0 >> 21) & ((1 << 21) - 1)).count("1")
    assert e.min() >= -21 and e.max() <= 21
    assert abs(e.mean()) < 0.05
    assert abs(e.var() - 10.5) < 0.3   # Var = eta / 2


def test_secret_hamming_weight():
    for n, h in [(64, 16), (4096, 512), (16384, 512)]:
        s = np.zeros(n, np.int8)
        O.lib().orc_secret(O.lib().orc_stream_key(3, 1, 0, 0), n, h, s.ctypes.data)
        assert (s != 0).sum() == h
        assert set(np.unique(s)) <= {-1, 0, 1}


# ----------------------------------------------------------------------------- primes

def test_primes_rule():
    sympy = pytest.importorskip("sympy")
    for bits, count, two_n in [(50, 3, 1 << 17), (60, 8, 1 << 17), (20, 4, 64)]:
        ps = O.primes(bits, count, two_n)
        assert len(ps) == count and ps == sorted(ps, reverse=True)
        assert all(sympy.isprime(p) and p % two_n == 1 and p < (1 << bits) for p in ps)
        # nothing skipped between 2^bits and the last prime
        c = ((1 << bits) - 2) // two_n
        found = [c2 * two_n + 1 for c2 in range(c, ps[-1] // two_n - 1, -1) if sympy.isprime(c2 * two_n + 1)]
        assert found == ps


# ----------------------------------------------------------------------------- cleartext

def test_rotation_moves_single_bit():
    bits = np.zeros(O.CODE_BITS, np.uint8)
    row, col, b = 5, 3, 2
    bits[(row * 200 + col) * 4 + b] = 1
    for r in [0, 7, 15, 22, 30]:
        s = r - 15
        out = O.rotate(bits, r)
        assert out.sum() == 1
        # x_s[row, col', b] = x[row, (col' + s) mod 200, b]  =>  the bit lands at col' = col - s
        assert out[(row * 200 + (col - s) % 200) * 4 + b] == 1
    assert np.array_equal(O.rotate(bits, 15), bits)


def _brute_counts(c1, m1, c2, m2):
    num = sum(1 for i in range(len(c1)) if (c1[i] ^ c2[i]) and m1[i] and m2[i])
    den = sum(1 for i in range(len(c1)) if m1[i] and m2[i])
    return num, den


def test_hd_counts_brute_force_and_masked_identity():
    rng = np.random.default_rng(0)
    qc = rng.integers(0, 2, (3, O.CODE_BITS), dtype=np.uint8)
    qm = (rng.random((3, O.CODE_BITS)) < 0.9).astype(np.uint8)
    dc = rng.integers(0, 2, (4, O.CODE_BITS), dtype=np.uint8)
    dm = (rng.random((4, O.CODE_BITS)) < 0.9).astype(np.uint8)
    num, den = O.hd_counts(qc, qm, dc, dm)
    inner = O.inner_from_counts(num, den)
    for a in range(3):
        ca = O.cprime(qc[a], qm[a], O.CODE_BITS).astype(np.int64)
        for b in range(4):
            n, d = _brute_counts(qc[a], qm[a], dc[b], dm[b])
            assert (num[a, b], den[a, b]) == (n, d)
            cb = O.cprime(dc[b], dm[b], O.CODE_BITS).astype(np.int64)
            # Section 2.1.3: 2 <c1 xor c2, m1 and m2> = ||m1 and m2|| - <c1', c2'>
            assert 2 * n == d - int(ca @ cb)
            assert inner[a, b] == int(ca @ cb)


def test_cprime_values():
    c = np.array([0, 1, 0, 1], np.uint8)
    m = np.array([0, 0, 1, 1], np.uint8)
    assert O.cprime(c, m, 6).tolist() == [0, 0, 1, -1, 0, 0]


def test_decision_equivalence_and_zero_overlap():
    rng = np.random.default_rng(1)
    den = rng.integers(0, 13000, (31, 50)).astype(np.int32)
    num = (rng.random((31, 50)) * (den + 1)).astype(np.int32)
    num = np.minimum(num, den)
    t = 0.375
    hd = O.fractional_hd(num, den)
    score = (den - 2.0 * num) / np.where(den > 0, den, 1)
    nz = den > 0
    # Eq. (2): dist < t  <=>  score > 1 - 2t
    assert np.array_equal((hd < t)[nz], (score > 1 - 2 * t)[nz])
    assert np.all(hd[~nz] == 1.0)
    mb = O.match_bits(num, den, t, rho=31)
    assert np.array_equal(mb[0], ((hd < t) & nz).any(axis=0))


# ----------------------------------------------------------------------------- ring / encryption

def _conv_negacyclic(s, a, q):
    """Independent route: full linear convolution, then X^N = -1."""
    N = len(a)
    full = np.convolve(s.astype(object), a.astype(object))
    out = [0] * N
    for i, v in enumerate(full):
        if i < N:
            out[i] += v
        else:
            out[i - N] -= v
    return np.array([int(v) % q for v in out], dtype=np.uint64)


def test_negacyclic_against_convolution():
    rng = np.random.default_rng(2)
    q = SMALL.q[0]
    for N in [8, 64]:
        s = np.zeros(N, np.int8)
        idx = rng.choice(N, 5, replace=False)
        s[idx] = rng.choice([-1, 1], 5)
        a = np.array([int(x) % q for x in rng.integers(0, 1 << 62, N)], np.uint64)
        assert np.array_equal(O.negacyclic_mul(s, a, q), _conv_negacyclic(s, a, q))
    # X * X^(N-1) = X^N = -1
    N = 16
    s = np.zeros(N, np.int8); s[1] = 1
    a = np.zeros(N, np.uint64); a[N - 1] = 1
    out = O.negacyclic_mul(s, a, q)
    assert out[0] == q - 1 and out[1:].sum() == 0


def _centered(x, q):
    x = int(x) % q
    return x - q if x > q // 2 else x


@pytest.mark.parametrize("P", [SMALL, SMALL2])
def test_query_encrypt_decrypts_to_message(P):
    W = synth.make_workload(n_eyes=2, n_db=4, seed=3)
    ct = O.query_encrypt(P, W.q_codes, W.q_masks, W.eye_ids)
    cp = O.query_cprime(W.q_codes, W.q_masks, P.rho, P.d2)
    Q = P.Q
    delta = 1 << P.log2_delta
    nblk = P.d2 // P.nq
    for j in [0, 33]:
        # CRT the Lq limbs into residues mod Q (Python integers), then b + s_t * a per block
        def col(k0, k1):
            vals = []
            for k in range(k0, k1):
                x = 0
                for l in range(P.n_limbs_q):
                    ql = P.q[l]
                    Ml = Q // ql
                    x += int(ct[l, j, k]) * Ml * pow(Ml, -1, ql)
                vals.append(x % Q)
            return np.array(vals, dtype=object)
        a = col(P.d2, P.K)
        for t in sorted({0, 1, nblk // 2, nblk - 1}):
            s = O.secret(P, "q", t)
            b = col(t * P.nq, (t + 1) * P.nq)
            sa = np.convolve(s.astype(object), a)
            sa_red = [sa[i] - (sa[i + P.nq] if i + P.nq < len(sa) else 0) for i in range(P.nq)]
            dec = [_centered(int(b[i]) + int(sa_red[i]), Q) for i in range(P.nq)]
            msg = cp[j, t * P.nq:(t + 1) * P.nq].astype(np.int64)
            err = np.array(dec, dtype=object) - msg.astype(object) * delta
            assert max(abs(int(e)) for e in err) <= P.eta


def test_query_extend_is_centered_crt():
    P = SMALL2
    rng = np.random.default_rng(4)
    n = 200
    ins = np.stack([np.array([int(x) % P.q[l] for x in rng.integers(0, 1 << 62, n)], np.uint64)
                    for l in range(P.n_limbs_q)])
    ins[:, 0] = 0
    ins[:, 1] = [q - 1 for q in P.q[:P.n_limbs_q]]          # -1 mod Q
    out = O.query_extend(P, ins.reshape(P.n_limbs_q, 1, n))
    Q = P.Q
    for i in range(n):
        x = 0
        for l in range(P.n_limbs_q):
            Ml = Q // P.q[l]
            x += int(ins[l, i]) * Ml * pow(Ml, -1, P.q[l])
        x %= Q
        xc = x - Q if x > Q // 2 else x
        for l in range(P.n_limbs):
            assert int(out[l, 0, i]) == xc % P.q[l]
    assert int(out[P.n_limbs_q, 0, 1]) == P.q[P.n_limbs_q] - 1


@pytest.mark.parametrize("P", [SMALL, SMALL2])
def test_db_rows_decrypt_to_gadget_message(P):
    W = synth.make_workload(n_eyes=1, n_db=70, seed=5)
    ids = O.db_layout(70, P.ndb, P.rho)
    sel = np.array([0, 1, P.ndb - 1] + [P.ndb + r for r in (0, 1, 65, 69)], np.int64)
    rows = O.db_rows(P, W.db_codes, W.db_masks, ids)
    sub = O.db_rows(P, W.db_codes, W.db_masks, sel)
    pos = {int(r): x for x, r in enumerate(ids)}
    for x, r in enumerate(sel):
        assert np.array_equal(sub[:, x], rows[:, pos[int(r)]])      # row selection is consistent
    # dense definition of S_q (vertical stack of Neg(s_{q,t})) for M_db * S_q
    nqb = P.d2 // P.nq
    Sq = np.zeros((P.d2, P.nq), np.int64)
    for t in range(nqb):
        s = O.secret(P, "q", t).astype(np.int64)
        for k in range(P.nq):
            for j in range(P.nq):
                Sq[t * P.nq + k, j] = s[k - j] if k >= j else -s[P.nq + k - j]
    cb, mb = O.unpack(W.db_codes), O.unpack(W.db_masks)
    Qp = P.Qp
    A = rows[:, :P.ndb, :]                          # a-part rows in order 0..ndb-1
    for r in (0, 1, 65, 69):
        t, i = divmod(r, P.ndb)
        s = O.secret(P, "db", t)
        c = O.cprime(cb[r], mb[r], P.d2).astype(np.int64)
        Wrow = np.concatenate([c, c @ Sq])
        brow = rows[:, pos[P.ndb + r], :]
        for l in range(P.n_limbs):
            ql = P.q[l]
            for k in range(0, P.K, 97):
                a_col = A[l, :, k]
                sa = _conv_negacyclic(s, a_col, ql)[i]
                e = _centered(int(brow[l, k]) + int(sa) - (Qp % ql) * int(Wrow[k]), ql)
                assert abs(e) <= P.eta


# ----------------------------------------------------------------------------- CCMM

def test_ppmm_bigint_and_extremes():
    rng = np.random.default_rng(6)
    q = O.primes(60, 2)
    L, M, N, K = 2, 5, 3, 7
    A = np.stack([np.array([[int(x) % q[l] for x in r] for r in rng.integers(0, 1 << 62, (M, K))], np.uint64) for l in range(L)])
    B = np.stack([np.array([[int(x) % q[l] for x in r] for r in rng.integers(0, 1 << 62, (N, K))], np.uint64) for l in range(L)])
    C = O.ppmm(q, A, B)
    for l in range(L):
        for j in range(N):
            for i in range(M):
                assert int(C[l, j, i]) == sum(int(A[l, i, k]) * int(B[l, j, k]) for k in range(K)) % q[l]
    # all-extreme operands, deep K (accumulator stress): (q-1)^2 * K mod q = K mod q
    K = 1 << 15
    A = np.full((1, 2, K), q[0] - 1, np.uint64)
    B = np.full((1, 3, K), q[0] - 1, np.uint64)
    assert np.all(O.ppmm(q, A, B) == K % q[0])
    # identity
    K = 6
    I = np.eye(K, dtype=np.uint64)[None]
    B = np.array([[[int(x) % q[0] for x in r] for r in rng.integers(0, 1 << 62, (4, K))]], np.uint64)
    assert np.array_equal(O.ppmm(q, I, B)[0], B[0])


def test_ppmm_composite_square_moduli():
    """The same product modulo the paper's p^2 moduli (Section 6.2.2) and an odd composite square:
    Python big integers on random operands, and the (q-1)^2 K closed form with K across the
    oracle's 64-term reduction."""
    rng = np.random.default_rng(16)
    q = [127 ** 2, 251 ** 2, 9 ** 2]
    L, M, N, K = 3, 6, 4, 131
    A = np.stack([rng.integers(0, ql, (M, K)).astype(np.uint64) for ql in q])
    B = np.stack([rng.integers(0, ql, (N, K)).astype(np.uint64) for ql in q])
    C = O.ppmm(q, A, B)
    for l in range(L):
        for j in range(N):
            for i in range(M):
                assert int(C[l, j, i]) == sum(int(A[l, i, k]) * int(B[l, j, k]) for k in range(K)) % q[l]
    K = 70_000
    for ql in q:
        C = O.ppmm([ql], np.full((1, 2, K), ql - 1, np.uint64), np.full((1, 2, K), ql - 1, np.uint64))
        assert np.all(C == K % ql)


def test_crt_decode_closed_form():
    P = SMALL2
    scale = P.Qp * (1 << P.log2_delta)
    ns = [0, 1, -1, 12800, -12800, 4321]
    eps = [0, scale // 3, -(scale // 3), 17, -17, scale // 2 - 1]
    vals = [n * scale + e for n, e in zip(ns, eps)]
    D = np.array([[v % ql for v in vals] for ql in P.q], np.uint64)
    got, worst = O.crt_decode(P, D)
    assert got.tolist() == ns
    assert worst <= 0.5


@pytest.mark.parametrize("P", [SMALL, SMALL2])
def test_ccmm_decrypts_to_cleartext_inner_products(P):
    """End to end on the oracle alone: Dec(CCMM(Enc(M_db), Enc(M_q))) rounds to M_db M_q exactly
    (closed form <c'_db, c'_q>, Section 2.1.3), and the fold commutes with decryption."""
    n_db = 70
    W = synth.make_workload(n_eyes=2, n_db=n_db, seed=8, planted_frac=0.1)
    ct = O.query_encrypt(P, W.q_codes, W.q_masks, W.eye_ids)
    B = O.query_extend(P, ct)
    ids = O.db_layout(n_db, P.ndb, P.rho)
    A = O.db_rows(P, W.db_codes, W.db_masks, ids)
    C = O.ppmm(P.q, A, B)
    rc, rm = O.rotated_templates(W.q_codes, W.q_masks, P.rho)
    num, den = O.hd_counts(rc, rm, O.unpack(W.db_codes), O.unpack(W.db_masks))
    inner = O.inner_from_counts(num, den)
    dec = np.zeros((C.shape[1], n_db), np.int64)
    for j in range(C.shape[1]):
        b_ids, nums, worst = O.decrypt_column(P, C[:, j, :], ids)
        real = b_ids < n_db
        dec[j, b_ids[real]] = nums[real]
        assert np.all(nums[~real] == 0)
        assert worst < 1e-3
    assert np.array_equal(dec, inner)
    # fold: decrypt(fold(C)) equals the cleartext fold of the numerators (negacyclic shifts)
    F = O.fold(P, C, ids, n_eyes=2, n_real=n_db)
    N = P.ndb
    groups = [list(range(g, min(g + P.fold_k, P.rho))) for g in range(0, P.rho, P.fold_k)]
    for e in range(2):
        for g, grp in enumerate(groups):
            b_ids, nums, _ = O.decrypt_column(P, F[:, e * len(groups) + g, :], ids)
            for x, r in enumerate(b_ids):
                if r >= n_db:
                    continue
                t, i = divmod(int(r), N)
                want = 0
                for rr in grp:
                    src = i - rr
                    v = 0
                    sign = 1
                    if src < 0:
                        src += N
                        sign = -1
                    gsrc = t * N + src
                    if gsrc < n_db:
                        v = inner[e * P.rho + rr, gsrc]
                    want += sign * v
                assert nums[x] == want


# ----------------------------------------------------------------------------- rescaling

def _from_residues(res, moduli):
    """Test-side Chinese remaindering: the integer in [0, prod moduli) with the given residues,
    found by Garner-style incremental lifting (a different route from the oracle's sum formula)."""
    x, m = 0, 1
    for r, qj in zip(res, moduli):
        t = ((int(r) - x) * pow(m, -1, qj)) % qj
        x, m = x + m * t, m * qj
    return x


@pytest.mark.parametrize("P", [SMALL, SMALL2])
def test_rescale_is_rounded_division(P):
    """Rescaling by Q' (Section 2.2.2, Maintenance: divide by the dropped modulus factor and
    round).  Checked by what characterises the nearest integer, not by the oracle's formula:
    (i) for random x, the result x' is the unique class modulo Q with |x - Q' x'| <= (Q' - 1) / 2
    (centred modulo Q Q'); (ii) closed forms: k Q' + e rounds to k for every |e| <= (Q' - 1) / 2,
    including both edges next to the (never reached) half-integer; (iii) the ends of [0, Q Q')."""
    rng = np.random.default_rng(3)
    Qdb, Qp, Q = P.Qdb, P.Qp, P.Q
    Lq = P.n_limbs_q
    xs = [int.from_bytes(rng.bytes(64), "little") % Qdb for _ in range(400)]
    ks = [0, 1, 2, Q // 3, Q - 1]
    h = (Qp - 1) // 2
    es = [0, 1, -1, h, -h, h - 1, -(h - 1), Qp // 3]
    closed = [(k, e) for k in ks for e in es]
    xs_closed = [(k * Qp + e) % Qdb for k, e in closed]
    xs_all = xs + xs_closed + [0, Qdb - 1]
    C = np.array([[x % ql for x in xs_all] for ql in P.q], np.uint64)
    got = O.rescale(P, C)
    assert got.shape == (Lq, len(xs_all))
    moduli = [int(v) for v in P.q[:Lq]]
    xp = [_from_residues(got[:, i], moduli) for i in range(len(xs_all))]
    # (i) nearest-integer property for every input
    for x, y in zip(xs_all, xp):
        d = (x - Qp * y) % Qdb
        if d > Qdb // 2:
            d -= Qdb
        assert abs(d) <= h, (x, y)
    # (ii) closed forms
    for (k, e), y in zip(closed, xp[len(xs):len(xs) + len(closed)]):
        assert y == k % Q, (k, e)
    # (iii) the ends: 0 -> 0 and Q Q' - 1 (just below Q x Q') -> Q = 0 mod Q
    assert xp[-2] == 0 and xp[-1] == 0
    # the exact half-distance that the GPU parity tests use: zero never occurs (Q' odd), and the
    # edges e = +-(Q' - 1)/2 sit at the smallest possible distance 1 / (2 Q')
    num, den = O.rescale_half_distance(P, C)
    assert den == 2 * Qp and min(num) >= 1
    for (k, e), n in zip(closed, num[len(xs):len(xs) + len(closed)]):
        if abs(e) == h and (k * Qp + e) % Qdb == k * Qp + e:
            assert n == 1


@pytest.mark.parametrize("P", [SMALL, SMALL2])
def test_rescaled_ccmm_decrypts_exactly(P):
    """Dec at modulus Q of the rescaled CCMM result, divided by Delta and rounded, gives the
    cleartext inner products <c'_db, c'_q> exactly (the rescaling error, at most (1 + h) / 2 per
    coefficient, stays far below Delta / 2), and rescaling commutes with the fold up to the same
    error: both orders decrypt to the cleartext fold."""
    n_db = 70
    W = synth.make_workload(n_eyes=2, n_db=n_db, seed=8, planted_frac=0.1)
    B = O.query_extend(P, O.query_encrypt(P, W.q_codes, W.q_masks, W.eye_ids))
    ids = O.db_layout(n_db, P.ndb, P.rho)
    C = O.ppmm(P.q, O.db_rows(P, W.db_codes, W.db_masks, ids), B)
    R = O.rescale(P, C)
    assert R.shape == (P.n_limbs_q,) + C.shape[1:]
    rc, rm = O.rotated_templates(W.q_codes, W.q_masks, P.rho)
    num, den = O.hd_counts(rc, rm, O.unpack(W.db_codes), O.unpack(W.db_masks))
    inner = O.inner_from_counts(num, den)
    dec = np.zeros((R.shape[1], n_db), np.int64)
    for j in range(R.shape[1]):
        b_ids, nums, worst = O.decrypt_column(P, R[:, j, :], ids, rescaled=True)
        real = b_ids < n_db
        dec[j, b_ids[real]] = nums[real]
        assert worst < 1e-3
    assert np.array_equal(dec, inner)
    # fold then rescale, and rescale then fold (the fold is linear per limb): same decryption
    F0 = O.fold(P, C, ids, n_eyes=2, n_real=n_db)
    F1 = O.rescale(P, F0)
    Pq = O.Params(**{**P.__dict__, "n_limbs": P.n_limbs_q})
    F2 = O.fold(Pq, R, ids, n_eyes=2, n_real=n_db)
    for col in range(F1.shape[1]):
        b1, n1, _ = O.decrypt_column(P, F1[:, col, :], ids, rescaled=True)
        b2, n2, _ = O.decrypt_column(P, F2[:, col, :], ids, rescaled=True)
        _, n0, _ = O.decrypt_column(P, F0[:, col, :], ids)
        real = b1 < n_db                      # the fold writes the tail rows of a partial block as zero
        assert np.array_equal(b1, b2) and np.array_equal(n1[real], n2[real])
        assert np.array_equal(n1[real], n0[real])
