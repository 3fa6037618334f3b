"""GPU parity: every stage of the CUDA path against the oracle on the same seeded inputs.

Tiny workload (ring degree 2^12, three primes below 2^50, 4 eyes x 31 rotations, 256 database
templates): query ciphertext, extended query operand, encrypted database, CCMM residues and fold
residues must be bit-identical to the oracle's; decrypted numerators must equal the cleartext
inner products <c'_db, c'_q> exactly (so decoded distances equal the FP64 cleartext distances and
match bits are identical)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_17561_gb300 import build as B
from paper_2601_17561_gb300 import engine as E
from paper_2601_17561_gb300 import synth

pytestmark = pytest.mark.gpu


def _u64(t: torch.Tensor, shape):
    n = int(np.prod(shape))
    return t[: n * 8].view(torch.int64).cpu().numpy().view(np.uint64).reshape(shape)


@pytest.fixture(scope="module")
def tiny():
    B.build()
    P = O.Params(**O.TINY)
    W = synth.make_workload(**synth.TINY)
    ids = O.db_layout(W.db_codes.shape[0], P.ndb, P.rho)
    ct = O.query_encrypt(P, W.q_codes, W.q_masks, W.eye_ids)
    Bq = O.query_extend(P, ct)
    A = O.db_rows(P, W.db_codes, W.db_masks, ids)
    Cm = O.ppmm(P.q, A, Bq)
    F = O.fold(P, Cm, ids, n_eyes=W.q_codes.shape[0], n_real=W.db_codes.shape[0])
    rc, rm = O.rotated_templates(W.q_codes, W.q_masks, P.rho)
    num, den = O.hd_counts(rc, rm, O.unpack(W.db_codes), O.unpack(W.db_masks))
    return dict(P=P, W=W, ids=ids, ct=ct, Bq=Bq, A=A, C=Cm, F=F, num=num, den=den,
                inner=O.inner_from_counts(num, den))


@pytest.fixture(scope="module")
def gpu_run(tiny):
    P, W = tiny["P"], tiny["W"]
    eng = E.Engine(**E.TINY).keygen()
    db = eng.encrypt_db(W.db_codes, W.db_masks, chunk_id=0)
    ct = eng.encrypt_query(W.q_codes, W.q_masks, W.eye_ids)
    q = eng.prepare(ct, W.q_codes.shape[0], "u64")
    s = eng.match(db, q)
    f = eng.fold(s)
    dec = eng.decrypt(s)
    fdec = eng.decrypt(f)
    torch.cuda.synchronize()
    return dict(eng=eng, db=db, ct=ct, q=q, s=s, f=f, dec=dec.cpu().numpy(), fdec=fdec.cpu().numpy())


def test_primes(tiny, gpu_run):
    assert gpu_run["eng"].primes == tiny["P"].q


def test_query_ciphertext_bit_exact(tiny, gpu_run):
    got = _u64(gpu_run["ct"], tiny["ct"].shape)
    assert np.array_equal(got, tiny["ct"])


def test_query_operand_bit_exact(tiny, gpu_run):
    got = _u64(gpu_run["q"].buf, tiny["Bq"].shape)
    assert np.array_equal(got, tiny["Bq"])


def _from_digit_form(z: np.ndarray, q) -> np.ndarray:
    """The database's storage word holds the signed balanced base-256 digits of the centred lift
    (bytes in two's complement): lift = (z xor 0x80..80) - 0x80..80 (mod 2^64)."""
    B = np.uint64(0x8080808080808080)
    c = (z ^ B) - B                                      # wraps modulo 2^64
    out = np.empty_like(z)
    for l, ql in enumerate(q):
        cl = c[l].view(np.int64)
        out[l] = np.where(cl < 0, (cl + np.int64(ql)).view(np.uint64), c[l])
    return out


def test_database_bit_exact(tiny, gpu_run):
    A = tiny["A"]
    assert gpu_run["db"].m_rows == A.shape[1]
    got = _from_digit_form(_u64(gpu_run["db"].buf, A.shape), tiny["P"].q)
    assert np.array_equal(got, A)


def test_ccmm_bit_exact(tiny, gpu_run):
    got = gpu_run["s"].residues()
    assert got.shape == tiny["C"].shape
    assert np.array_equal(got, tiny["C"])


@pytest.mark.parametrize("form", ["i8_digits", "i8_crt", "f16_crt"])
def test_ccmm_tensor_forms_bit_exact(tiny, gpu_run, form):
    """The tensor-core forms give the same residues as the oracle (and the u64 form)."""
    eng, W = gpu_run["eng"], tiny["W"]
    q = eng.prepare(gpu_run["ct"], W.q_codes.shape[0], form)
    s = eng.match(gpu_run["db"], q)
    torch.cuda.synchronize()
    assert np.array_equal(s.residues(), tiny["C"])


def test_fold_bit_exact(tiny, gpu_run):
    got = gpu_run["f"].residues()
    assert got.shape == tiny["F"].shape
    assert np.array_equal(got, tiny["F"])


def test_decrypted_numerators_exact(tiny, gpu_run):
    assert np.array_equal(gpu_run["dec"], tiny["inner"])


def test_decoded_distance_and_match_bits(tiny, gpu_run):
    """Decoded fractional HD (numerator from the ciphertext, overlap ||m1 and m2|| from the
    plaintext masks, Section 3) equals the FP64 cleartext HD; match bits are identical."""
    num, den = tiny["num"], tiny["den"]
    hd_clear = O.fractional_hd(num, den)
    dec_num = (den.astype(np.int64) - gpu_run["dec"]) // 2          # <c1 xor c2, m1 and m2>
    assert np.array_equal((den.astype(np.int64) - gpu_run["dec"]) % 2, np.zeros_like(den, dtype=np.int64))
    hd_dec = O.fractional_hd(dec_num, den)
    assert np.max(np.abs(hd_dec - hd_clear)) <= 2.0 ** -10
    assert np.array_equal(O.match_bits(dec_num, den), O.match_bits(num, den))
    # planted near-duplicates are found
    mb = O.match_bits(num, den)
    for row, (eye, _) in tiny["W"].planted.items():
        assert mb[eye, row]


def test_folded_decryption_is_cleartext_fold(tiny, gpu_run):
    P, inner = tiny["P"], tiny["inner"]
    n_db = inner.shape[1]
    groups = [list(range(g, min(g + P.fold_k, P.rho))) for g in range(0, P.rho, P.fold_k)]
    want = np.zeros((4 * len(groups), n_db), np.int64)
    for e in range(4):
        for g, grp in enumerate(groups):
            for r in grp:
                for i in range(n_db):
                    src = i - r
                    if src >= 0:
                        want[e * len(groups) + g, i] += inner[e * P.rho + r, src]
                    # wrapped sources are padding coefficients of the block (zero message)
    assert np.array_equal(gpu_run["fdec"], want)


# ------------------------------------------------------------------ plain modular product

def _rand_res(rng, q, shape):
    return np.stack([np.array(rng.integers(0, 1 << 62, size=shape, dtype=np.int64) % q_l, dtype=np.uint64)
                     for q_l in q])


FORMS = ["u64", "i8_digits", "i8_crt", "f16_crt"]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (64, 64, 16), (65, 63, 17), (130, 37, 1000), (300, 5, 2049),
                                   (7, 129, 64), (64, 1, 0), (0, 3, 5), (257, 70, 33)])
def test_ppmm_ragged(form, M, N, K):
    B.build()
    rng = np.random.default_rng(M * 1000 + N * 10 + K)
    q = [O.primes(60, 1)[0], O.primes(50, 1)[0], O.primes(31, 1, 64)[0]]
    A = _rand_res(rng, q, (M, K))
    Bm = _rand_res(rng, q, (N, K))
    want = O.ppmm(q, A, Bm)
    dA = torch.from_numpy(A.view(np.int64)).cuda()
    dB = torch.from_numpy(Bm.view(np.int64)).cuda()
    got = E.ppmm(form, q, dA, dB).cpu().numpy().view(np.uint64)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("kind", ["minus_one", "digits_min"])
def test_ppmm_extremes(form, kind):
    """Deep K with operands at the accumulator limits.  minus_one: every residue q - 1.  digits_min:
    the centred lift has its seven low balanced digits at -128, so every int8 digit product is
    2^14 and a shift sums up to 7 pairs per column (the int32 accumulators must be chunked)."""
    B.build()
    q = O.primes(60, 2)
    K = 24576
    if kind == "minus_one":
        xc = [-1, -1]
    else:
        v = -sum(128 * 256 ** t for t in range(7))
        xc = [v, v]
    A = np.stack([np.full((70, K), (x % q_l), np.uint64) for x, q_l in zip(xc, q)])
    Bm = np.stack([np.full((9, K), (x % q_l), np.uint64) for x, q_l in zip(xc, q)])
    got = E.ppmm(form, q, torch.from_numpy(A.view(np.int64)).cuda(),
                 torch.from_numpy(Bm.view(np.int64)).cuda()).cpu().numpy().view(np.uint64)
    for l, q_l in enumerate(q):
        assert np.all(got[l] == (xc[l] * xc[l] * K) % q_l)


def _crt_edge_depth(q):
    """Even K as deep as the CRT forms allow before the small-modulus count grows: the product M
    of the greedy moduli (odd, pairwise coprime, from 255 down) covering 2^3 K ((q-1)/2)^2 stays
    that of K = 2^14, so |C| / M for operands at the largest centred lift approaches 1/8, the
    recombination's design limit."""
    import math
    h = (max(q) - 1) // 2
    need = 8 * (1 << 14) * h * h
    mods, M = [], 1
    for v in range(255, 2, -2):
        if M > need:
            break
        if all(math.gcd(v, m) == 1 for m in mods):
            mods.append(v)
            M *= v
    K = (M // (8 * h * h)) * 63 // 64
    return min(K - K % 2, 131070), len(mods)


@pytest.mark.parametrize("form", ["i8_crt", "f16_crt"])
@pytest.mark.parametrize("sign", [1, -1])
def test_ppmm_crt_range_edge(form, sign):
    """Every operand at the largest centred lift (q-1)/2, against +-(q-1)/2, at a depth K where
    |C| / M is close to 1/8 (58-bit primes, 17 moduli): C = +-K ((q-1)/2)^2 is recombined exactly
    (the fp32 quotient of the recombination still rounds to the right integer)."""
    B.build()
    q = O.primes(58, 2)
    K, r = _crt_edge_depth(q)
    assert r == 17 and K > 1 << 15
    xa = [(q_l - 1) // 2 for q_l in q]
    xb = [sign * x for x in xa]
    A = np.stack([np.full((70, K), x % q_l, np.uint64) for x, q_l in zip(xa, q)])
    Bm = np.stack([np.full((9, K), x % q_l, np.uint64) for x, q_l in zip(xb, q)])
    got = E.ppmm(form, q, torch.from_numpy(A.view(np.int64)).cuda(),
                 torch.from_numpy(Bm.view(np.int64)).cuda()).cpu().numpy().view(np.uint64)
    for l, q_l in enumerate(q):
        assert np.all(got[l] == (xa[l] * xb[l] * K) % q_l)


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_ccmm_tcgen05_variant_bit_exact(tiny, gpu_run, variant):
    """Every tcgen05 kernel variant of the fp16 CRT form (tensor-memory accumulators, one modulus
    on up to 512 columns per block; two ring depths, with or without the wave bound between
    blocks) gives the oracle's residues, and no kernel gave up a bounded wait."""
    from paper_2601_17561_gb300 import icm as C
    eng, W = gpu_run["eng"], tiny["W"]
    C.icm_ctx_set_variant(eng.ctx, variant)
    try:
        q = eng.prepare(gpu_run["ct"], W.q_codes.shape[0], "f16_crt")
        s = eng.match(gpu_run["db"], q)
        torch.cuda.synchronize()
        C.icm_device_status(True)
        assert np.array_equal(s.residues(), tiny["C"])
    finally:
        C.icm_ctx_set_variant(eng.ctx, 0)


@pytest.mark.parametrize("variant", [1, 2])
def test_tcgen05_bounded_wait_runs_out(tiny, gpu_run, variant):
    """Failure detection on the device without a fault: with a 20 ms wait bound and the query
    producer's copies withheld (test-only switch), the MMA issuers' waits run out; the kernel
    records ICM_ETIMEOUT in the device status word, drains its own copies, frees its tensor memory
    and returns (no trap, the context stays usable).  The status word reports the timeout once and
    is then clear, and the next normal launch gives the oracle's residues."""
    from paper_2601_17561_gb300 import icm as C
    eng, W = gpu_run["eng"], tiny["W"]
    C.icm_device_status(True)
    C.icm_ctx_set_variant(eng.ctx, variant)
    try:
        q = eng.prepare(gpu_run["ct"], W.q_codes.shape[0], "f16_crt")
        C.icm_ctx_set_device_wait(eng.ctx, 20_000_000, True)
        try:
            s = eng.match(gpu_run["db"], q)
            torch.cuda.synchronize()
        finally:
            C.icm_ctx_set_device_wait(eng.ctx, 0, False)
        with pytest.raises(C.IcmError) as e:
            C.icm_device_status(True)
        assert e.value.status == C.ICM_ETIMEOUT
        C.icm_device_status(True)                       # cleared: no error any more
        s = eng.match(gpu_run["db"], q)
        torch.cuda.synchronize()
        C.icm_device_status(True)
        assert np.array_equal(s.residues(), tiny["C"])
    finally:
        C.icm_ctx_set_variant(eng.ctx, 0)


def test_ccmm_tcgen05_two_column_rounds_ragged_rows(tiny):
    """tcgen05 variant on 20 eyes (620 columns: two column rounds, the second with a ragged
    column tile) against 300 codes (a ragged last row tile): identical to the mma.sync variant
    everywhere and to the oracle's product on sampled rows, including the ragged tail."""
    from paper_2601_17561_gb300 import icm as C
    P = tiny["P"]
    W = synth.make_workload(n_eyes=20, n_db=300, seed=11, planted_frac=0.05)
    eng = E.Engine(**E.TINY).keygen()
    db = eng.encrypt_db(W.db_codes, W.db_masks)
    ct = eng.encrypt_query(W.q_codes, W.q_masks, W.eye_ids)
    res = {}
    try:
        for v in (256, 1, 2, 3):
            C.icm_ctx_set_variant(eng.ctx, v)
            q = eng.prepare(ct, 20, "f16_crt")
            s = eng.match(db, q)
            torch.cuda.synchronize()
            res[v] = s.residues()
    finally:
        C.icm_ctx_set_variant(eng.ctx, 0)
    C.icm_device_status(True)
    for v in (1, 2, 3):
        assert np.array_equal(res[v], res[256]), v
    ids = O.db_layout(300, P.ndb, P.rho)
    A = O.db_rows(P, W.db_codes, W.db_masks, ids)
    Bq = O.query_extend(P, O.query_encrypt(P, W.q_codes, W.q_masks, W.eye_ids))
    M = A.shape[1]
    rows = np.unique(np.concatenate([np.arange(0, 8), np.arange(M // 2, M // 2 + 8), np.arange(M - 24, M)]))
    ref = O.ppmm(P.q, np.ascontiguousarray(A[:, rows, :]), Bq)
    assert np.array_equal(res[1][:, :, rows], ref)


@pytest.mark.parametrize("n_eyes", [17, 32, 34])
def test_ccmm_tcgen05_launch_rounds(tiny, n_eyes):
    """All column rounds of a launch in one persistent kernel: 17 eyes (527 columns: a second
    round of 15 columns with no second column tile, where the tile-1 producer and issuer take part
    without copies or MMAs), 32 eyes (992 columns: two rounds of two column tiles, the last ragged)
    and 34 eyes (1,054 columns: a full 1,024-column launch, then a 30-column launch), against 300
    codes (a ragged last row tile): every tcgen05 variant identical to the mma.sync variant
    everywhere and to the oracle's product on sampled rows."""
    from paper_2601_17561_gb300 import icm as C
    P = tiny["P"]
    W = synth.make_workload(n_eyes=n_eyes, n_db=300, seed=13, planted_frac=0.05)
    eng = E.Engine(**E.TINY).keygen()
    db = eng.encrypt_db(W.db_codes, W.db_masks)
    ct = eng.encrypt_query(W.q_codes, W.q_masks, W.eye_ids)
    res = {}
    try:
        for v in (256, 1, 2, 3):
            C.icm_ctx_set_variant(eng.ctx, v)
            q = eng.prepare(ct, n_eyes, "f16_crt")
            s = eng.match(db, q)
            torch.cuda.synchronize()
            res[v] = s.residues()
            del s, q
    finally:
        C.icm_ctx_set_variant(eng.ctx, 0)
    C.icm_device_status(True)
    for v in (1, 2, 3):
        assert np.array_equal(res[v], res[256]), v
    ids = O.db_layout(300, P.ndb, P.rho)
    A = O.db_rows(P, W.db_codes, W.db_masks, ids)
    M = A.shape[1]
    rows = np.unique(np.concatenate([np.arange(0, 4), np.arange(M - 12, M)]))
    Bq = O.query_extend(P, O.query_encrypt(P, W.q_codes, W.q_masks, W.eye_ids))
    ref = O.ppmm(P.q, np.ascontiguousarray(A[:, rows, :]), Bq)
    assert np.array_equal(res[1][:, :, rows], ref)


def test_ccmm_tcgen05_odd_modulus_count():
    """56-bit primes give 17 CRT moduli (an odd count, so the waves of persistent tiles do not
    split evenly over row tiles): residues of the tcgen05 variants equal the mma.sync variant's
    everywhere and the oracle's product on sampled rows."""
    from paper_2601_17561_gb300 import icm as C
    prm = dict(O.TINY)
    prm.update(prime_bits=56, seed=5)
    P = O.Params(**prm)
    W = synth.make_workload(n_eyes=8, n_db=140, seed=12, planted_frac=0.05)
    eprm = dict(E.TINY)
    eprm.update(prime_bits=56, seed=5)
    eng = E.Engine(**eprm).keygen()
    assert eng.primes == P.q
    assert len(C.icm_ctx_crt_moduli(eng.ctx)) == 17
    db = eng.encrypt_db(W.db_codes, W.db_masks)
    ct = eng.encrypt_query(W.q_codes, W.q_masks, W.eye_ids)
    res = {}
    try:
        for v in (256, 1, 2, 3):
            C.icm_ctx_set_variant(eng.ctx, v)
            q = eng.prepare(ct, 8, "f16_crt")
            s = eng.match(db, q)
            torch.cuda.synchronize()
            res[v] = s.residues()
    finally:
        C.icm_ctx_set_variant(eng.ctx, 0)
    C.icm_device_status(True)
    assert all(np.array_equal(res[v], res[256]) for v in (1, 2, 3))
    ids = O.db_layout(140, P.ndb, P.rho)
    A = O.db_rows(P, W.db_codes, W.db_masks, ids)
    Bq = O.query_extend(P, O.query_encrypt(P, W.q_codes, W.q_masks, W.eye_ids))
    M = A.shape[1]
    rows = np.unique(np.concatenate([np.arange(0, 8), np.arange(M - 16, M)]))
    ref = O.ppmm(P.q, np.ascontiguousarray(A[:, rows, :]), Bq)
    assert np.array_equal(res[1][:, :, rows], ref)


def test_decrypt_max_error_matches_oracle(tiny, gpu_run):
    """The decoder's reported pre-rounding error -- the largest |x - round(x)| over all (column,
    real row) outputs, x = decrypted coefficient / (Q' Delta) -- equals the oracle's exact
    big-integer value over the same outputs (up to the fp32 of the report), lies far below 1/2,
    and comes with the same numerators as the plain decryption."""
    P, W, eng = tiny["P"], tiny["W"], gpu_run["eng"]
    dec, err = eng.decrypt(gpu_run["s"], with_error=True)
    torch.cuda.synchronize()
    assert np.array_equal(dec.cpu().numpy(), gpu_run["dec"])
    e_gpu = float(err.cpu()[0])
    ids, Cm = tiny["ids"], tiny["C"]
    n_real = W.db_codes.shape[0]
    a_pos = np.array([np.where(ids == i)[0][0] for i in range(P.ndb)])
    b_pos = np.array([np.where(ids == P.ndb + r)[0][0] for r in range(n_real)])
    worst = 0.0
    for j in range(Cm.shape[1]):
        D = O.decrypt_rows(P, Cm[:, j, a_pos], Cm[:, j, b_pos], np.arange(n_real))
        _, w = O.crt_decode(P, D)
        worst = max(worst, w)
    print(f"max pre-rounding error: GPU {e_gpu:.6e}, oracle {worst:.6e} (numerator units)")
    assert 0 < worst < 1e-3
    assert abs(e_gpu - worst) <= 1e-6 * worst


# ----------------------------------------------------------------------------- rescaling by Q'

def test_rescale_bit_exact(tiny, gpu_run):
    """Rescaling by Q' on the GPU against the oracle's exact round(x / Q') mod Q (Section 2.2.2,
    Maintenance), for the CCMM result and for the folded scores: identical everywhere except where
    x / Q' lies within the kernel's fixed-point window (L - L_q) 2^-64 of a half-integer, where one
    unit either way is allowed (and that window holds no coefficient of this workload).  The fold
    of the rescaled scores equals the oracle's fold of the oracle's rescaling."""
    from rescale_check import check_rescaled
    P, eng = tiny["P"], gpu_run["eng"]
    r = eng.rescale(gpu_run["s"])
    rf = eng.rescale(gpu_run["f"])
    fr = eng.fold(r)
    torch.cuda.synchronize()
    assert r.shape[0] == P.n_limbs_q
    n_win = check_rescaled(P, r.residues(), tiny["C"])
    n_win_f = check_rescaled(P, rf.residues(), tiny["F"])
    print(f"coefficients in the rounding window: {n_win} (CCMM), {n_win_f} (fold)")
    assert n_win == 0 and n_win_f == 0
    R = O.rescale(P, tiny["C"])
    Pq = O.Params(**{**O.TINY, "n_limbs": P.n_limbs_q})
    W = tiny["W"]
    assert np.array_equal(fr.residues(), O.fold(Pq, R, tiny["ids"], n_eyes=W.q_codes.shape[0],
                                               n_real=W.db_codes.shape[0]))


def test_rescaled_decryption_exact(tiny, gpu_run):
    """Decryption at modulus Q with scale Delta of the rescaled CCMM result gives the cleartext
    inner products exactly; the rescaled fold decrypts like the full-level fold."""
    eng = gpu_run["eng"]
    dec = eng.decrypt(eng.rescale(gpu_run["s"]))
    fdec = eng.decrypt(eng.rescale(gpu_run["f"]))
    torch.cuda.synchronize()
    assert np.array_equal(dec.cpu().numpy(), tiny["inner"])
    assert np.array_equal(fdec.cpu().numpy(), gpu_run["fdec"])


def test_rescale_rejects_misuse(gpu_run):
    from paper_2601_17561_gb300 import icm as C
    eng = gpu_run["eng"]
    r = eng.rescale(gpu_run["s"])
    with pytest.raises(C.IcmError) as e:
        eng.rescale(r)
    assert e.value.status == C.ICM_EINVAL
    small = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(C.IcmError) as e:
        C.icm_rescale(eng.ctx, gpu_run["s"].handle, small, 8)
    assert e.value.status == C.ICM_ENOMEM


def test_match_launch_count(tiny, gpu_run):
    """icm_match_launches: one launch for the u64 and digit forms; for the CRT forms a product and
    a recombination launch per column round (1,024 columns on tcgen05, 512 on mma.sync) and limb
    group (the tiny residue scratch holds all three limbs in one group)."""
    from paper_2601_17561_gb300 import icm as C
    eng, db = gpu_run["eng"], gpu_run["db"]
    n_eyes = tiny["W"].q_codes.shape[0]                          # 124 columns: one round
    assert C.icm_match_launches(eng.ctx, db.handle, n_eyes, C.FORMS["u64"]) == 1
    assert C.icm_match_launches(eng.ctx, db.handle, n_eyes, C.FORMS["i8_digits"]) == 1
    assert C.icm_match_launches(eng.ctx, db.handle, n_eyes, C.FORMS["f16_crt"]) == 2
    assert C.icm_match_launches(eng.ctx, db.handle, 20, C.FORMS["i8_crt"]) == 4     # 620 columns: 2 rounds of 512
    assert C.icm_match_launches(eng.ctx, db.handle, 40, C.FORMS["f16_crt"]) == 4    # 1,240 columns: 2 of 1,024
    assert C.icm_match_launches(eng.ctx, db.handle, 0, C.FORMS["f16_crt"]) == 0


@pytest.mark.parametrize("n_eyes,form", [(4, "u64"), (3, "f16_crt"), (1, "f16_crt")])
def test_match_host_buffers(tiny, gpu_run, n_eyes, form):
    """icm_match_host (host ciphertext in, host folded scores out; the eyes run in two parts whose
    copies overlap the other part's product) gives the oracle's folded residues for an even, an
    odd and a single-eye batch."""
    from paper_2601_17561_gb300 import icm as C
    P, W = tiny["P"], tiny["W"]
    eng, db = gpu_run["eng"], gpu_run["db"]
    ct = eng.encrypt_query(W.q_codes[:n_eyes], W.q_masks[:n_eyes], W.eye_ids[:n_eyes])
    h_ct = ct.cpu().pin_memory()
    G = (P.rho + P.fold_k - 1) // P.fold_k
    L, M = P.n_limbs, db.m_rows
    h_fo = torch.zeros(L * n_eyes * G * M * 8, dtype=torch.uint8).pin_memory()
    f = C.FORMS[form]
    wsb = C.icm_match_host_workspace_bytes(eng.ctx, db.handle, n_eyes, f)
    ws = torch.empty(wsb, dtype=torch.uint8, device=eng.device)
    st = torch.cuda.Stream()
    C.icm_match_host(eng.ctx, db.handle, h_ct, n_eyes, f, h_fo, ws, wsb, stream=st)
    st.synchronize()
    got = h_fo.view(torch.int64).numpy().view(np.uint64).reshape(L, n_eyes * G, M)
    want = O.fold(P, tiny["C"][:, : n_eyes * P.rho], tiny["ids"], n_eyes=n_eyes, n_real=W.db_codes.shape[0])
    assert np.array_equal(got, want)
