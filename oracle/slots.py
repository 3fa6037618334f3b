"""TEST INFRASTRUCTURE ONLY -- oracle of the slot-encoded database and of the normalisation.

Plain fp64 / exact-integer CPU restatement of three passages of arxiv 2601.17561:

* Section 2.2.1 (Encoding and decoding): Ecd_slot maps N/2 complex slot values x_j to the
  rounded real polynomial Delta * P of degree < N with P(zeta^(5^j)) = x_j, zeta = exp(I pi / N);
  Dcd is its inverse up to rounding.
* Section 2.3: the CCMM also accepts a slot-encoded database matrix M_db, and the result then has
  the database's encoding (each result ciphertext of ring degree N_db carries one block of the
  database).
* Algorithm 2: every result ciphertext is multiplied by the plaintext
  mu = Ecd((1 / ||m_q AND m_db||_1)_j) before the fold, so that its slots hold the normalised
  scores <c'_q, c'_db> / ||m_q AND m_db||_1 = 1 - 2 HD (Section 2.1.3 identity).

Readings (where the paper leaves the choice open):
* One template per slot, in the slot's real part; the N/2 templates t*N/2 .. t*N/2 + N/2 - 1 of
  block t fill its N/2 slots, missing templates give 0.  (A slot holding two templates as real
  and imaginary part would be scaled by one complex factor, not by two real ones, so the
  slot-wise normalisation needs one template per slot; the paper's conjugate-invariant encoding
  would hold N real values per ciphertext but needs the arithmetic of that subring.)
* Rounding to integers is round-half-to-even of the fp64 value (numpy.rint).
* mu uses 1 / ||m_q AND m_db||_1 for every real template with a non-empty overlap and 0 for empty
  overlaps and for missing templates.
* The normalisation multiplies the result after the rescaling by Q' (modulus Q, scale Delta times
  the database scale); both ciphertext parts of every block are multiplied by its mu, so the
  shared a-part of a result column becomes one a-part per block.  No rescaling follows: decoding
  divides by the product of the three scales.

Every function here is pinned by tests/test_slot_pins.py.
"""
from __future__ import annotations

import functools

import numpy as np

from . import Params, crt_decode_q  # noqa: F401  (crt_decode_q: same CRT rule, exact integers)
from . import lib, _p, negacyclic_mulmod, secret, unpack, CODE_BITS


# ------------------------------------------------------------------------------ Ecd_slot / Dcd

def slot_exponents(N: int) -> np.ndarray:
    """e_j = 5^j mod 2N for j < N/2: slot j is the value of P at zeta^(e_j) (Section 2.2.1)."""
    e = np.zeros(N // 2, np.int64)
    v = 1
    for j in range(N // 2):
        e[j] = v
        v = v * 5 % (2 * N)
    return e


@functools.lru_cache(maxsize=4)
def _angles(N: int) -> np.ndarray:
    """(e_j * n mod 2N) as exact integers, [N][N/2]: zeta^(e_j n) = exp(I pi angle / N)."""
    e = slot_exponents(N)
    n = np.arange(N, dtype=np.int64)
    return (n[:, None] * e[None, :]) % (2 * N)


@functools.lru_cache(maxsize=4)
def _cos(N: int) -> np.ndarray:
    """C[n][j] = cos(pi (e_j n mod 2N) / N) = Re zeta^(e_j n)."""
    return np.cos(np.pi * _angles(N).astype(np.float64) / N)


def encode(z: np.ndarray, N: int) -> np.ndarray:
    """Real coefficients of P with P(zeta^(5^j)) = z_j (unrounded, scale 1).  z: [N/2] or
    [N/2][cols] complex or real.  Since P is real it also takes the conjugate values at
    zeta^(-5^j), and {5^j, -5^j mod 2N} are all the odd residues modulo 2N, so inverting the
    evaluation at every odd power of zeta gives
        p_n = (1/N) sum_{odd r} P(zeta^r) zeta^(-r n) = (2/N) Re sum_j z_j zeta^(-5^j n)."""
    z = np.asarray(z)
    ang = _angles(N).astype(np.float64) * (np.pi / N)          # [N][N/2]
    if np.iscomplexobj(z):
        # Re(z zeta^(-a)) = Re(z) cos(a) + Im(z) sin(a)
        return (2.0 / N) * (np.cos(ang) @ z.real + np.sin(ang) @ z.imag)
    return (2.0 / N) * (_cos(N) @ z)


def decode(p: np.ndarray, N: int) -> np.ndarray:
    """Slot values z_j = P(zeta^(5^j)) = sum_n p_n zeta^(5^j n) of a real polynomial (Section
    2.2.1 Dcd before the division by the scale), by plain evaluation.  p: [N] or [N][cols]."""
    ang = _angles(N).astype(np.float64) * (np.pi / N)
    p = np.asarray(p, np.float64)
    return np.cos(ang).T @ p + 1j * (np.sin(ang).T @ p)


def decode_real(p: np.ndarray, N: int) -> np.ndarray:
    """Real parts of the slot values: Re z_j = sum_n p_n cos(pi (5^j n mod 2N) / N)."""
    return _cos(N).T @ np.asarray(p, np.float64)


def ecd(z: np.ndarray, N: int, log2_scale: int) -> np.ndarray:
    """Ecd_slot at scale 2^log2_scale: round(2^s P) (round half to even), int64."""
    return np.rint(encode(z, N) * float(2 ** log2_scale)).astype(np.int64)


def ecd_unrounded(z: np.ndarray, N: int, log2_scale: int) -> np.ndarray:
    """2^s P before rounding (the tests use it to find values within a hair of a half-integer,
    where two correct fp64 evaluations may round to different neighbours)."""
    return encode(z, N) * float(2 ** log2_scale)


# ------------------------------------------------------------------------------ slot-encoded database

def slot_blocks(n_db: int, N: int) -> int:
    """Blocks of N/2 templates (one template per slot)."""
    return (n_db + N // 2 - 1) // (N // 2)


def slot_values(db_codes, db_masks, N: int, d2: int) -> np.ndarray:
    """Masked bit-vectors c' (Section 2.1.3) arranged by slot: V[t][j][k] = c'_{t N/2 + j}[k]
    (0 for missing templates and padding entries), int8 [n_blocks][N/2][d2]."""
    n_db = db_codes.shape[0]
    nb = slot_blocks(n_db, N)
    V = np.zeros((nb * (N // 2), d2), np.int8)
    c, m = unpack(db_codes).astype(np.int8), unpack(db_masks).astype(np.int8)
    V[:n_db, :CODE_BITS] = m - 2 * (c & m)
    return V.reshape(nb, N // 2, d2)


def slot_db_messages(db_codes, db_masks, N: int, d2: int, log2_scale: int, unrounded: bool = False):
    """Message matrix of the slot-encoded database: rows t N + n (block t, coefficient n) hold the
    coefficients of Ecd_slot of the column of block t's slot values, for every entry k < d2:
    W[t N + n][k] = round(2^s (2/N) sum_j V[t][j][k] cos(pi (5^j n mod 2N) / N)), [n_blocks N][d2]
    int64 (or the fp64 values before rounding)."""
    V = slot_values(db_codes, db_masks, N, d2)
    nb = V.shape[0]
    out = np.zeros((nb * N, d2), np.float64 if unrounded else np.int64)
    for t in range(nb):
        w = ecd_unrounded(V[t].astype(np.float64), N, log2_scale)
        out[t * N:(t + 1) * N] = w if unrounded else np.rint(w).astype(np.int64)
    return out


def slot_layout(n_db: int, N: int) -> np.ndarray:
    """Row ids of a slot-encoded chunk in storage order: the a-part rows 0..N-1, then every
    coefficient row of every block (all blocks are full: n_blocks N b-rows)."""
    nb = slot_blocks(n_db, N)
    return np.arange(N + nb * N, dtype=np.int64)


# ------------------------------------------------------------------------------ normalisation

def mu_values(den: np.ndarray, n_db: int, N: int) -> np.ndarray:
    """Slot values of mu for every result column j and block t: 1 / den[j][t N/2 + i] for real
    templates with den > 0, else 0.  den: [d3][n_db] mask overlaps.  [d3][n_blocks][N/2] fp64."""
    d3 = den.shape[0]
    nb = slot_blocks(n_db, N)
    v = np.zeros((d3, nb * (N // 2)), np.float64)
    d = den.astype(np.float64)
    v[:, :n_db] = np.where(den > 0, 1.0 / np.where(den > 0, d, 1.0), 0.0)
    return v.reshape(d3, nb, N // 2)


def mu_polys(den: np.ndarray, n_db: int, N: int, log2_scale: int, unrounded: bool = False):
    """mu = Ecd_slot(1 / ||m_q AND m_db||) per (column, block) at scale 2^s: [d3][n_blocks][N]."""
    v = mu_values(den, n_db, N)
    d3, nb, _ = v.shape
    w = ecd_unrounded(v.reshape(d3 * nb, N // 2).T, N, log2_scale).T.reshape(d3, nb, N)
    return w if unrounded else np.rint(w).astype(np.int64)


def normalize(P: Params, R: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """ct <- ct (.) mu for every block (Algorithm 2): R [L_q][d3][M] rescaled result of a
    slot-encoded chunk (rows: a-part 0..N-1, then block t's N b-rows), mu [d3][n_blocks][N]
    integers.  Out [L_q][d3][n_blocks][2][N] residues: (a mu, b_t mu) in Z_q[X]/(X^N + 1)."""
    Lq, d3, M = R.shape
    N = P.ndb
    nb = (M - N) // N
    q = [int(v) for v in P.q[:Lq]]
    out = np.zeros((Lq, d3, nb, 2, N), np.uint64)
    for l in range(Lq):
        for j in range(d3):
            a = R[l, j, :N]
            for t in range(nb):
                m = np.array([int(x) % q[l] for x in mu[j, t]], np.uint64)
                out[l, j, t, 0] = negacyclic_mulmod(a, m, q[l])
                out[l, j, t, 1] = negacyclic_mulmod(R[l, j, N + t * N:N + (t + 1) * N], m, q[l])
    return out


def decrypt_normalized(P: Params, out: np.ndarray) -> np.ndarray:
    """Dec = a' s_{db,t} + b' (Section 2.2.2) of every normalised block, as centred integers modulo
    Q (exact, Python ints): [d3][n_blocks][N] object array."""
    Lq, d3, nb, _, N = out.shape
    q = [int(v) for v in P.q[:Lq]]
    Q = 1
    for v in q:
        Q *= v
    coef = [(Q // qi) * pow(Q // qi, -1, qi) for qi in q]
    res = np.empty((d3, nb, N), dtype=object)
    for t in range(nb):
        s = secret(P, "db", t)
        for j in range(d3):
            limbs = []
            for l in range(Lq):
                sa = np.zeros(N, np.uint64)
                lib().orc_negacyclic_mul(_p(np.ascontiguousarray(s)), _p(np.ascontiguousarray(out[l, j, t, 0])), N,
                                         q[l], _p(sa))
                b = out[l, j, t, 1]
                limbs.append([(int(sa[i]) + int(b[i])) % q[l] for i in range(N)])
            for i in range(N):
                x = sum(limbs[l][i] * coef[l] for l in range(Lq)) % Q
                res[j, t, i] = x - Q if x > Q // 2 else x
    return res


def decoded_scores(P: Params, out: np.ndarray, log2_scale_db: int, log2_scale_mu: int) -> np.ndarray:
    """Normalised scores: real parts of Dcd(Dec(ct)) / (Delta 2^s_db 2^s_mu), one per slot:
    [d3][n_blocks * N/2] fp64 (slot t N/2 + j is template t N/2 + j)."""
    dec = decrypt_normalized(P, out)
    d3, nb, N = dec.shape
    scale = float(2 ** (P.log2_delta + log2_scale_db + log2_scale_mu))
    vals = np.array([[float(x) / scale for x in row] for row in dec.reshape(d3 * nb, N)])
    z = decode_real(vals.T, N).T                                   # [d3 * nb][N/2]
    return z.reshape(d3, nb * (N // 2))


def hd_from_scores(s: np.ndarray) -> np.ndarray:
    """Fractional Hamming distance from a normalised score: s = <c'_q, c'_db> / ||m_q AND m_db||
    = 1 - 2 HD (Section 2.1.3), so HD = (1 - s) / 2."""
    return (1.0 - np.asarray(s, np.float64)) / 2.0
