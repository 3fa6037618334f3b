"""TEST INFRASTRUCTURE ONLY -- the oracle for the encrypted 1:N iris matching hot path.

Plain, slow, obviously correct CPU implementation of what arxiv 2601.17561 ("Private Iris
Recognition with High-Performance FHE") computes on its CCMM + fold path.  Only `tests/`,
`__graft_entry__.smoke()` and the CPU-baseline / reference legs of `bench.py` may import this
package.  It shares no code with the CUDA library (`paper_2601_17561_gb300`); both receive the
same packed templates from `paper_2601_17561_gb300.synth`, which holds no method arithmetic.

Heavy exact loops (encryption, the u128 schoolbook product, decryption sums, popcounts) live in
`icm_oracle.c`; this module holds the cleartext iris rules, the prime rule, the big-integer CRT
decoding and the fold, each written from the passage it cites.  Readings of passages where the
paper is silent are listed beside the functions that take them.

`slots.py` holds the slot-encoded database variant and the normalisation of the scores (Section
2.2.1 Ecd_slot, Section 2.3, Algorithm 2), pinned by `tests/test_slot_pins.py`.

Parity status: every function here is pinned by `tests/test_oracle_pins.py` (no function is
"parity unpinned").
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "icm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

ROWS, COLS, PLANES = 16, 200, 4          # iris code layout of the synthetic templates
CODE_BITS = ROWS * COLS * PLANES


# ------------------------------------------------------------------------------ build / load

def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, OpenMP).  Building the checker is not using it."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        u64, i32, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        _lib.orc_sm64.restype = u64
        _lib.orc_sm64.argtypes = [u64, u64]
        _lib.orc_stream_key.restype = u64
        _lib.orc_stream_key.argtypes = [u64, u64, u64, u64]
        _lib.orc_uniform_mod.restype = u64
        _lib.orc_uniform_mod.argtypes = [u64, u64]
        _lib.orc_cbd.restype = i32
        _lib.orc_cbd.argtypes = [u64, i32]
        _lib.orc_secret.restype = None
        _lib.orc_secret.argtypes = [u64, i32, i32, vp]
        _lib.orc_query_encrypt.restype = i32
        _lib.orc_query_encrypt.argtypes = [i32, vp, i32, i32, i32, i32, ctypes.c_uint, u64, i32, i32, vp, vp, vp]
        _lib.orc_query_extend.restype = i32
        _lib.orc_query_extend.argtypes = [i32, i32, vp, ctypes.c_size_t, vp, vp]
        _lib.orc_db_rows.restype = i32
        _lib.orc_db_rows.argtypes = [i32, i32, vp, i32, i32, i32, i32, i32, u64, u64, vp, i32, vp, vp]
        _lib.orc_ppmm.restype = None
        _lib.orc_ppmm.argtypes = [i32, vp, i32, i32, i32, vp, vp, vp]
        _lib.orc_decrypt_rows.restype = None
        _lib.orc_decrypt_rows.argtypes = [i32, vp, i32, i32, u64, vp, i32, vp, vp, vp]
        _lib.orc_hd_counts.restype = None
        _lib.orc_hd_counts.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, vp]
        _lib.orc_negacyclic_mul.restype = None
        _lib.orc_negacyclic_mul.argtypes = [vp, vp, i32, u64, vp]
        _lib.orc_negacyclic_mulmod.restype = None
        _lib.orc_negacyclic_mulmod.argtypes = [vp, vp, i32, u64, vp]
        _lib.orc_omp_threads.restype = i32
        _lib.orc_omp_threads.argtypes = []
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    return int(lib().orc_omp_threads())


# ------------------------------------------------------------------------------ parameters

def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (first twelve prime bases)."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def primes(bits: int, count: int, two_n: int = 1 << 17):
    """RNS prime chain (reading of Table 1 / Section 6: the paper fixes only the chain's size):
    the `count` largest primes below 2^bits that are 1 mod two_n, in decreasing order."""
    out = []
    c = ((1 << bits) - 2) // two_n
    while len(out) < count:
        cand = c * two_n + 1
        if is_prime(cand):
            out.append(cand)
        c -= 1
    return out


@dataclasses.dataclass
class Params:
    """CKKS / CCMM parameters as the oracle reads them (Section 2.3, Section 6.2.1, Table 1)."""
    log_n_db: int
    log_n_q: int
    n_limbs: int
    n_limbs_q: int
    prime_bits: int
    d2: int = 1 << 14
    rho: int = 31
    fold_k: int = 16
    h: int = 512
    log2_delta: int = 26
    eta: int = 21
    seed: int = 1

    @property
    def ndb(self):
        return 1 << self.log_n_db

    @property
    def nq(self):
        return 1 << self.log_n_q

    @property
    def K(self):
        return self.d2 + self.nq

    @property
    def q(self):
        return primes(self.prime_bits, self.n_limbs)

    @property
    def Q(self):
        return _prod(self.q[: self.n_limbs_q])

    @property
    def Qp(self):
        return _prod(self.q[self.n_limbs_q:])

    @property
    def Qdb(self):
        return _prod(self.q)


def _prod(xs):
    r = 1
    for x in xs:
        r *= x
    return r


TINY = dict(log_n_db=12, log_n_q=12, n_limbs=3, n_limbs_q=1, prime_bits=50, log2_delta=26, seed=1)
PAPER = dict(log_n_db=14, log_n_q=13, n_limbs=8, n_limbs_q=2, prime_bits=60, log2_delta=60, seed=2)


# ------------------------------------------------------------------------------ cleartext

def unpack(packed: np.ndarray) -> np.ndarray:
    """Packed templates (LSB-first bytes) -> bits, shape (n, CODE_BITS)."""
    packed = np.atleast_2d(packed)
    return np.unpackbits(packed, axis=1, bitorder="little")[:, :CODE_BITS].astype(np.uint8)


def rotate(bits: np.ndarray, r: int, rho: int = 31) -> np.ndarray:
    """Rotation r of a template (Section 2.1.2: code and mask are both rotated by a small
    offset).  Reading: shift s = r - (rho-1)/2 along the 200-column axis of the 16x200x4 layout,
    x_s[row, col, b] = x[row, (col + s) mod 200, b]; written with explicit indices."""
    s = r - (rho - 1) // 2
    out = np.empty_like(bits)
    for row in range(ROWS):
        for col in range(COLS):
            src = (row * COLS + (col + s) % COLS) * PLANES
            dst = (row * COLS + col) * PLANES
            out[..., dst:dst + PLANES] = bits[..., src:src + PLANES]
    return out


def cprime(code_bits: np.ndarray, mask_bits: np.ndarray, d2: int) -> np.ndarray:
    """Masked bit-vector c' = m - 2 (c AND m) in {-1, 0, 1} (Section 2.1.3), zero-padded to d2
    (the paper pads each database entry with zeroes, Section 2.3)."""
    c = code_bits.astype(np.int8)
    m = mask_bits.astype(np.int8)
    v = m - 2 * (c & m)
    out = np.zeros(v.shape[:-1] + (d2,), dtype=np.int8)
    out[..., : v.shape[-1]] = v
    return out


def query_cprime(q_codes: np.ndarray, q_masks: np.ndarray, rho: int, d2: int) -> np.ndarray:
    """Query matrix M_q as columns (d3 = n_eyes * rho, d2): column e*rho + r is c' of rotation r
    of eye e (Section 3.1: a query is rho rotated codes with their masks)."""
    cb, mb = unpack(q_codes), unpack(q_masks)
    n_eyes = cb.shape[0]
    out = np.zeros((n_eyes * rho, d2), dtype=np.int8)
    for e in range(n_eyes):
        for r in range(rho):
            out[e * rho + r] = cprime(rotate(cb[e], r, rho), rotate(mb[e], r, rho), d2)
    return out


def rotated_templates(q_codes, q_masks, rho):
    """(n_eyes * rho, CODE_BITS) rotated code and mask bits, column order e*rho + r."""
    cb, mb = unpack(q_codes), unpack(q_masks)
    rc = np.stack([rotate(cb[e], r, rho) for e in range(cb.shape[0]) for r in range(rho)])
    rm = np.stack([rotate(mb[e], r, rho) for e in range(mb.shape[0]) for r in range(rho)])
    return rc, rm


def _words(bits: np.ndarray) -> np.ndarray:
    packed = np.packbits(bits, axis=1, bitorder="little")
    pad = (-packed.shape[1]) % 8
    if pad:
        packed = np.concatenate([packed, np.zeros((packed.shape[0], pad), np.uint8)], axis=1)
    return np.ascontiguousarray(packed).view(np.uint64)


def hd_counts(qc_bits, qm_bits, dc_bits, dm_bits):
    """num = <c1 XOR c2, m1 AND m2>, den = ||m1 AND m2||_1 for every (query column, db row)
    pair (Section 2.1.1, Eq. (1))."""
    a, b = _words(qc_bits), _words(qm_bits)
    c, d = _words(dc_bits), _words(dm_bits)
    na, nb, w = a.shape[0], c.shape[0], a.shape[1]
    num = np.zeros((na, nb), np.int32)
    den = np.zeros((na, nb), np.int32)
    lib().orc_hd_counts(na, nb, w, _p(a), _p(b), _p(c), _p(d), _p(num), _p(den))
    return num, den


def inner_from_counts(num, den):
    """<c1', c2'> = ||m1 AND m2|| - 2 <c1 XOR c2, m1 AND m2> (Section 2.1.3 identity)."""
    return den.astype(np.int64) - 2 * num.astype(np.int64)


def fractional_hd(num, den):
    """dist = num / den (Eq. (1)); reading for den == 0: distance 1.0 (no match)."""
    num = np.asarray(num, dtype=np.float64)
    den = np.asarray(den, dtype=np.float64)
    out = np.ones_like(num)
    nz = den > 0
    out[nz] = num[nz] / den[nz]
    return out


def match_bits(num, den, t: float = 0.375, rho: int = 31):
    """Per (eye, db row): min over rotations of dist < t (Section 2.1.2, strict).  num/den are
    (n_eyes * rho, n_db); the comparison uses exact integers: num < t * den."""
    n_cols, n_db = num.shape
    n_eyes = n_cols // rho
    tn, td = _as_fraction(t)
    hit = (num.astype(np.int64) * td < tn * den.astype(np.int64)) & (den > 0)
    return hit.reshape(n_eyes, rho, n_db).any(axis=1)


def _as_fraction(t):
    from fractions import Fraction
    f = Fraction(t).limit_denominator(1 << 20)
    return f.numerator, f.denominator


# ------------------------------------------------------------------------------ encryption

def query_encrypt(P: Params, q_codes, q_masks, eye_ids) -> np.ndarray:
    """MSRLWE query ciphertext modulo Q (Section 2.3): [Lq][d3][K] residues, column j = b then a."""
    cp = np.ascontiguousarray(query_cprime(q_codes, q_masks, P.rho, P.d2))
    n_eyes = cp.shape[0] // P.rho
    out = np.zeros((P.n_limbs_q, cp.shape[0], P.K), np.uint64)
    q = np.array(P.q[: P.n_limbs_q], np.uint64)
    ids = np.ascontiguousarray(np.asarray(eye_ids, np.uint64))
    rc = lib().orc_query_encrypt(P.n_limbs_q, _p(q), P.nq, P.d2, P.h, P.eta, P.log2_delta, P.seed,
                                 n_eyes, P.rho, _p(ids), _p(cp), _p(out))
    assert rc == 0
    return out


def query_extend(P: Params, ct_q: np.ndarray) -> np.ndarray:
    """Centred lift from mod Q to every limb: [Lq][d3][K] -> [L][d3][K]."""
    Lq = ct_q.shape[0]
    flat = np.ascontiguousarray(ct_q.reshape(Lq, -1))
    out = np.zeros((P.n_limbs, flat.shape[1]), np.uint64)
    q = np.array(P.q, np.uint64)
    rc = lib().orc_query_extend(P.n_limbs, Lq, _p(q), flat.shape[1], _p(flat), _p(out))
    assert rc == 0
    return out.reshape((P.n_limbs,) + ct_q.shape[1:])


def db_layout(n_real: int, ndb: int, rho: int):
    """Logical ids of the rows of one database chunk, in storage order (reading of Section 2.3
    padding and of the fold's wrap-around, Algorithm 2): the a-part rows 0..ndb-1, then every
    real b-row r (id ndb + r), then for a partial last block the tail coefficients
    [ndb - rho + 1, ndb) of that block (encryptions of zero), which the negacyclic shift of the
    fold reads for its wrap-around."""
    ids = list(range(ndb)) + [ndb + r for r in range(n_real)]
    rem = n_real % ndb
    if rem:
        t = n_real // ndb
        lo = max(rem, ndb - (rho - 1))
        ids += [ndb + t * ndb + i for i in range(lo, ndb)]
    return np.array(ids, dtype=np.int64)


def db_rows(P: Params, db_codes, db_masks, row_ids, chunk: int = 0) -> np.ndarray:
    """Selected rows of the encrypted database chunk (Section 6.2.1), [L][n_rows][K].
    db_codes/db_masks: the chunk's templates; logical b-row r uses template r (padding rows,
    r >= number of templates, encrypt zero)."""
    row_ids = np.ascontiguousarray(np.asarray(row_ids, np.int64))
    n_tpl = db_codes.shape[0]
    cp = np.zeros((len(row_ids), P.d2), np.int32)
    sel = [(x, int(r) - P.ndb) for x, r in enumerate(row_ids) if r >= P.ndb and int(r) - P.ndb < n_tpl]
    if sel:
        idx = np.array([r for _, r in sel])
        cb, mb = unpack(db_codes[idx]), unpack(db_masks[idx])
        cp[[x for x, _ in sel]] = cprime(cb, mb, P.d2)
    return db_rows_from_messages(P, cp, row_ids, chunk)


def db_rows_from_messages(P: Params, msg: np.ndarray, row_ids, chunk: int = 0) -> np.ndarray:
    """Selected rows of an encrypted database chunk (Section 6.2.1) whose message matrix rows are
    given: msg [n_rows][d2] integers (|m| < 2^21) for the selected rows in row_ids order (rows of
    a-part ids are ignored).  [L][n_rows][K]."""
    row_ids = np.ascontiguousarray(np.asarray(row_ids, np.int64))
    msg = np.ascontiguousarray(msg, np.int32)
    assert msg.shape == (len(row_ids), P.d2)
    out = np.zeros((P.n_limbs, len(row_ids), P.K), np.uint64)
    q = np.array(P.q, np.uint64)
    rc = lib().orc_db_rows(P.n_limbs, P.n_limbs_q, _p(q), P.ndb, P.nq, P.d2, P.h, P.eta, P.seed, chunk,
                           _p(row_ids), len(row_ids), _p(msg), _p(out))
    assert rc == 0
    return out


def secret(P: Params, kind: str, t: int) -> np.ndarray:
    """Sparse ternary secret s_{db,t} (kind 'db', degree N_db) or s_{q,t} (kind 'q', degree N_q)."""
    n = P.ndb if kind == "db" else P.nq
    key = lib().orc_stream_key(P.seed, 1 if kind == "db" else 2, t, 0)
    s = np.zeros(n, np.int8)
    lib().orc_secret(key, n, P.h, _p(s))
    return s


def negacyclic_mul(s: np.ndarray, a: np.ndarray, q: int) -> np.ndarray:
    """s * a in Z_q[X]/(X^N + 1) for a sparse ternary s (Section 2.2.1 plaintext ring)."""
    s = np.ascontiguousarray(s, np.int8)
    a = np.ascontiguousarray(a, np.uint64)
    out = np.zeros_like(a)
    lib().orc_negacyclic_mul(_p(s), _p(a), len(a), q, _p(out))
    return out


# ------------------------------------------------------------------------------ CCMM / fold / decrypt

def negacyclic_mulmod(a: np.ndarray, b: np.ndarray, q: int) -> np.ndarray:
    """a * b in Z_q[X]/(X^N + 1) for residues a, b in [0, q) (Section 2.2.1 plaintext ring)."""
    a = np.ascontiguousarray(a, np.uint64)
    b = np.ascontiguousarray(b, np.uint64)
    assert a.shape == b.shape and a.ndim == 1
    out = np.zeros_like(a)
    lib().orc_negacyclic_mulmod(_p(a), _p(b), len(a), q, _p(out))
    return out


def ppmm(q, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """C[l][j][i] = sum_k A[l][i][k] B[l][j][k] mod q_l (u128 schoolbook, Section 2.3)."""
    A = np.ascontiguousarray(A, np.uint64)
    B = np.ascontiguousarray(B, np.uint64)
    L, M, K = A.shape
    N = B.shape[1]
    C = np.zeros((L, N, M), np.uint64)
    qa = np.array(q[:L], np.uint64)
    lib().orc_ppmm(L, _p(qa), M, N, K, _p(A), _p(B), _p(C))
    return C


def fold(P: Params, C: np.ndarray, row_ids: np.ndarray, n_eyes: int, n_real: int) -> np.ndarray:
    """Linear, key-free part of the fold of Algorithm 2: for eye e and group g of k = fold_k
    consecutive rotations, ct'_{e,g} = sum_{r in g} X^r * ct_{e,r}, on the a-part polynomial and
    on every b-block polynomial (reading: the shift is the global rotation index r; the keyed
    slot rotation Rot is replaced by the negacyclic monomial shift, and f is not applied).
    (X^r p)[i] = p[i-r] for i >= r and -p[N+i-r] for i < r.  C: [L][n_eyes*rho][M] in the chunk's
    row layout; output [L][n_eyes*G][M] in the same layout.  Reading for padded blocks: the tail
    coefficients of a partial block (logical b-rows >= n_real, padding entries with no template)
    are inputs of the wrap-around only and are not produced (zero)."""
    L, ncol, M = C.shape
    N = P.ndb
    groups = [list(range(g, min(g + P.fold_k, P.rho))) for g in range(0, P.rho, P.fold_k)]
    pos = {int(r): x for x, r in enumerate(row_ids)}
    out = np.zeros((L, n_eyes * len(groups), M), np.uint64)
    q = P.q
    for x, rid in enumerate(row_ids):
        rid = int(rid)
        if rid >= N + n_real:
            continue  # tail coefficient of a partial block: not produced
        blk_base = 0 if rid < N else N + ((rid - N) // N) * N
        i = rid - blk_base
        srcs = []
        ok = True
        for r in range(P.rho):
            if i >= r:
                src, sgn = blk_base + i - r, 1
            else:
                src, sgn = blk_base + N + i - r, -1
            if src not in pos:
                ok = False
                break
            srcs.append((pos[src], sgn))
        if not ok:
            continue  # a source row outside the given row set (partial row sets only)
        for l in range(L):
            ql = int(q[l])
            for e in range(n_eyes):
                for g, grp in enumerate(groups):
                    acc = 0
                    for r in grp:
                        sx, sgn = srcs[r]
                        acc += sgn * int(C[l, e * P.rho + r, sx])
                    out[l, e * len(groups) + g, x] = acc % ql
    return out


def crt_decode(P: Params, D: np.ndarray) -> np.ndarray:
    """Decode decrypted residues D [L][...] (Section 2.2.2 Dec, then the rounding of Section 2:
    floor(x + 1/2)): CRT to [0, Q_db), centre to (-Q_db/2, Q_db/2], divide by Q' * Delta and round
    to the nearest integer.  Returns (numerators, max |x - Q'Delta * numerator| / (Q'Delta))."""
    q = [int(v) for v in P.q]
    Qdb = P.Qdb
    scale = P.Qp * (1 << P.log2_delta)
    L = D.shape[0]
    flat = D.reshape(L, -1)
    coeffs = [(Qdb // qi) * pow(Qdb // qi, -1, qi) for qi in q]
    nums = np.zeros(flat.shape[1], np.int64)
    worst = 0.0
    for c in range(flat.shape[1]):
        x = sum(int(flat[l, c]) * coeffs[l] for l in range(L)) % Qdb
        if x > Qdb // 2:
            x -= Qdb
        n = (2 * x + scale) // (2 * scale)
        nums[c] = n
        err = abs(x - n * scale) / scale
        worst = max(worst, err)
    return nums.reshape(D.shape[1:]), worst


def crt_value(P: Params, C: np.ndarray) -> np.ndarray:
    """The integers x in [0, Q_db) whose residues modulo q_0 .. q_{L-1} are C [L][...] (Chinese
    remainder theorem, x = sum_l C_l (Q_db / q_l) ((Q_db / q_l)^-1 mod q_l) mod Q_db), as an object
    array of Python integers shaped like C[0]."""
    q = [int(v) for v in P.q]
    Qdb = P.Qdb
    L = C.shape[0]
    flat = np.ascontiguousarray(C.reshape(L, -1), np.uint64)
    x = np.zeros(flat.shape[1], dtype=object)
    for l in range(L):
        hat = Qdb // q[l]
        x = x + flat[l].astype(object) * (hat * pow(hat, -1, q[l]))
    return (x % Qdb).reshape(C.shape[1:])


def rescale(P: Params, C: np.ndarray) -> np.ndarray:
    """Rescaling by Q' (Section 2.2.2, Maintenance: RS divides by a factor of the modulus and
    rounds to the nearest integer).  The dropped factor is Q' = q_{L_q} ... q_{L-1}, so each
    coefficient x of Z_{Q Q'} (residues C [L][...]) becomes x' = round(x / Q') mod Q, returned as
    its residues [L_q][...] modulo q_0 .. q_{L_q - 1}.  Computed on the exact integers:
    round(x / Q') = floor((2x + Q') / (2Q')); Q' is odd, so x / Q' is never a half-integer and the
    rounding has no ties.  Any representative of x modulo Q Q' gives the same x' modulo Q."""
    Lq = P.n_limbs_q
    Qp, Q = P.Qp, P.Q
    x = crt_value(P, C).reshape(-1)
    xr = ((2 * x + Qp) // (2 * Qp)) % Q
    out = np.zeros((Lq, x.shape[0]), np.uint64)
    for j in range(Lq):
        out[j] = (xr % int(P.q[j])).astype(np.uint64)
    return out.reshape((Lq,) + C.shape[1:])


def rescale_half_distance(P: Params, C: np.ndarray) -> np.ndarray:
    """For every coefficient x (residues C [L][...]): the exact distance of x / Q' from the
    nearest half-integer, as the pair (|2 (x mod Q') - Q'|, 2 Q') of Python integers (distance =
    first / second).  Test support: a fast rescaling that estimates the quotient in fixed point may
    round either way only where this distance is below its stated error bound."""
    Qp = P.Qp
    y = crt_value(P, C) % Qp
    return np.abs(2 * y - Qp), 2 * Qp


def crt_decode_q(P: Params, D: np.ndarray) -> tuple:
    """crt_decode at the rescaled level: residues D [L_q][...] modulo Q, centred, divided by Delta
    and rounded (the scores after rescaling by Q' carry the scale Delta)."""
    q = [int(v) for v in P.q[: P.n_limbs_q]]
    Q = P.Q
    scale = 1 << P.log2_delta
    Lq = D.shape[0]
    flat = D.reshape(Lq, -1)
    coeffs = [(Q // qi) * pow(Q // qi, -1, qi) for qi in q]
    nums = np.zeros(flat.shape[1], np.int64)
    worst = 0.0
    for c in range(flat.shape[1]):
        x = sum(int(flat[l, c]) * coeffs[l] for l in range(Lq)) % Q
        if x > Q // 2:
            x -= Q
        n = (2 * x + scale) // (2 * scale)
        nums[c] = n
        worst = max(worst, abs(x - n * scale) / scale)
    return nums.reshape(D.shape[1:]), worst


def decrypt_rows(P: Params, Ca: np.ndarray, Cb: np.ndarray, b_rows) -> np.ndarray:
    """Residues of Dec = Cb + S_db * Ca for the given logical b-rows of one result column."""
    b_rows = np.ascontiguousarray(np.asarray(b_rows, np.int64))
    Ca = np.ascontiguousarray(Ca, np.uint64)
    Cb = np.ascontiguousarray(Cb, np.uint64)
    L = Ca.shape[0]
    D = np.zeros((L, len(b_rows)), np.uint64)
    q = np.array(P.q, np.uint64)
    lib().orc_decrypt_rows(L, _p(q), P.ndb, P.h, P.seed, _p(b_rows), len(b_rows), _p(Ca), _p(Cb), _p(D))
    return D


def decrypt_column(P: Params, Ccol: np.ndarray, row_ids, rescaled: bool = False) -> tuple:
    """Decrypt every b-row of one result column Ccol [L][M] (chunk row layout; [L_q][M] modulo Q
    with scale Delta when `rescaled`).  Returns (logical b-row ids, numerators, worst relative
    error)."""
    row_ids = np.asarray(row_ids, np.int64)
    a_pos = np.array([np.where(row_ids == i)[0][0] for i in range(P.ndb)])
    b_sel = np.where(row_ids >= P.ndb)[0]
    Ca = Ccol[:, a_pos]
    Cb = Ccol[:, b_sel]
    b_ids = row_ids[b_sel] - P.ndb
    D = decrypt_rows(P, Ca, Cb, b_ids)
    nums, worst = crt_decode_q(P, D) if rescaled else crt_decode(P, D)
    return b_ids, nums, worst
