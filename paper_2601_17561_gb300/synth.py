"""Seeded synthetic iris templates: the only inputs shared by the CUDA path and the oracle.

This module draws iris codes and masks and nothing else.  It holds none of the matching or
encryption arithmetic: no masked bit-vector map, no rotation of queries, no Hamming distance,
no sampling of keys, noise or ciphertext randomness.  Both the library and the oracle receive
the same packed templates from here and do everything else on their own.

Workload shapes follow the paper's setup (Section 6.1): uniform binary iris codes and Bernoulli
masks.  The code length (12,800 bits on a 16 x 200 x 4 layout) and the mask rate (0.9) are the
synthetic stand-in for the ND-IRIS-0405 templates, which are not available here.

Bit packing: bit b of a template lives in byte b // 8 at bit position b % 8 (LSB first).
Bit index b = (row * 200 + col) * 4 + plane on the 16 x 200 x 4 layout.
"""
from __future__ import annotations

import dataclasses
import numpy as np

CODE_ROWS, CODE_COLS, CODE_PLANES = 16, 200, 4
CODE_BITS = CODE_ROWS * CODE_COLS * CODE_PLANES  # 12,800
CODE_BYTES = CODE_BITS // 8                      # 1,600


def _pack(bits: np.ndarray) -> np.ndarray:
    """(n, CODE_BITS) of {0,1} -> (n, CODE_BYTES) uint8, LSB first."""
    return np.packbits(bits.astype(np.uint8), axis=1, bitorder="little")


def _unpack(packed: np.ndarray) -> np.ndarray:
    return np.unpackbits(packed, axis=1, bitorder="little")[:, :CODE_BITS]


def iris_templates(n: int, rng: np.random.Generator, p_mask: float = 0.9):
    """n independent templates: codes ~ Bernoulli(0.5), masks ~ Bernoulli(p_mask)."""
    codes = rng.integers(0, 2, size=(n, CODE_BITS), dtype=np.uint8)
    masks = (rng.random(size=(n, CODE_BITS)) < p_mask).astype(np.uint8)
    return _pack(codes), _pack(masks)


def _column_roll(bits: np.ndarray, shift: int) -> np.ndarray:
    """Data-generation helper: roll one template's columns so that the copy sits at a
    rotation offset of the original (used only to plant near-duplicates)."""
    cube = bits.reshape(CODE_ROWS, CODE_COLS, CODE_PLANES)
    return np.roll(cube, -shift, axis=1).reshape(-1)


@dataclasses.dataclass
class Workload:
    """One matching job: query eyes against a database (one or several chunks)."""
    q_codes: np.ndarray          # (n_eyes, CODE_BYTES) uint8
    q_masks: np.ndarray
    eye_ids: np.ndarray          # (n_eyes,) uint64, keys the per-eye encryption randomness
    db_codes: np.ndarray         # (n_db, CODE_BYTES) uint8
    db_masks: np.ndarray
    planted: dict                # db row -> (eye, offset) for planted near-duplicates
    chunks: list                 # [(row_start, n_rows)] database chunks


def make_workload(n_eyes: int, n_db: int, seed: int, planted_frac: float = 0.0,
                  flip_rate: float = 0.2, p_mask: float = 0.9, chunk_sizes=None,
                  max_offset: int = 15) -> Workload:
    """Seeded workload.  A fraction `planted_frac` of database rows are noisy copies of a
    uniformly chosen query eye: columns rolled by a uniform offset in [-max_offset, max_offset],
    each code bit flipped with probability `flip_rate`, and a fresh mask."""
    rng = np.random.default_rng(seed)
    q_codes, q_masks = iris_templates(n_eyes, rng, p_mask)
    db_codes, db_masks = iris_templates(n_db, rng, p_mask)
    planted = {}
    n_plant = int(round(planted_frac * n_db))
    if n_plant and n_eyes:
        rows = rng.choice(n_db, size=n_plant, replace=False)
        qbits = _unpack(q_codes)
        dbits = _unpack(db_codes)
        for row in np.sort(rows):
            eye = int(rng.integers(0, n_eyes))
            off = int(rng.integers(-max_offset, max_offset + 1))
            copy = _column_roll(qbits[eye], off)
            flips = (rng.random(CODE_BITS) < flip_rate).astype(np.uint8)
            dbits[row] = copy ^ flips
            planted[int(row)] = (eye, off)
        db_codes = _pack(dbits)
    if chunk_sizes is None:
        chunks = [(0, n_db)]
    else:
        assert sum(chunk_sizes) == n_db
        starts = np.cumsum([0] + list(chunk_sizes[:-1]))
        chunks = [(int(s), int(c)) for s, c in zip(starts, chunk_sizes)]
    eye_ids = np.arange(1, n_eyes + 1, dtype=np.uint64) + np.uint64(seed) * np.uint64(1 << 20)
    return Workload(q_codes, q_masks, eye_ids, db_codes, db_masks, planted, chunks)


def uneven_chunk_sizes(n_chunks: int, base: int, seed: int):
    """Chunk sizes floor(base * U[0.5, 1.5]) (the batching form's uneven database split)."""
    rng = np.random.default_rng(seed)
    return [int(base * u) for u in rng.uniform(0.5, 1.5, size=n_chunks)]


# Named workload recipes (sizes from the paper's experiment, Section 6; tiny = a small case
# that the oracle finishes in seconds).
TINY = dict(n_eyes=4, n_db=256, seed=1, planted_frac=0.05)
PAPER = dict(n_eyes=32, n_db=7 * (1 << 14), seed=2, planted_frac=0.05)
