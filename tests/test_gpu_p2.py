"""GPU parity of the paper's own modulus family in icm_ppmm (ICM_FORM_I8_P2, Section 6.2.2: Q is the
product of p^2 over the primes 127 <= p <= 253, and a product modulo p^2 becomes int8 products of
base-p digits) against the oracle's u128 schoolbook product, bit for bit."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_17561_gb300 import build as B
from paper_2601_17561_gb300 import engine as E

pytestmark = pytest.mark.gpu

PAPER_P = [p for p in range(127, 254) if all(p % d for d in range(2, int(p ** 0.5) + 1))]   # 24 primes


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _rand(rng, q, shape):
    return np.stack([rng.integers(0, q_l, size=shape, dtype=np.int64).astype(np.uint64) for q_l in q])


def _run(q, A, Bm):
    got = E.ppmm("i8_p2", q, torch.from_numpy(A.view(np.int64)).cuda(), torch.from_numpy(Bm.view(np.int64)).cuda())
    return got.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (64, 64, 16), (65, 63, 17), (130, 37, 1000), (300, 5, 2049),
                                   (7, 129, 64), (64, 1, 0), (0, 3, 5), (257, 70, 33)])
def test_p2_ragged(M, N, K):
    """Ragged row and column tiles and K slabs; the largest and smallest paper primes, and odd
    composite and small bases."""
    q = [127 ** 2, 251 ** 2, 9 ** 2, 197 ** 2, 253 ** 2]
    rng = np.random.default_rng(M * 1000 + N * 10 + K)
    A, Bm = _rand(rng, q, (M, K)), _rand(rng, q, (N, K))
    assert np.array_equal(_run(q, A, Bm), O.ppmm(q, A, Bm))


@pytest.mark.parametrize("kind", ["half", "minus_one", "half_below"])
def test_p2_extremes_deep_k(kind):
    """K = 70,000 crosses the int32 chunk of the digit passes (65,504 columns).  half: every residue
    (q - 1) / 2, whose digits reach |x1| = (p - 1) / 2 with x0 = (p - 1) / 2; half_below: (q + 1) / 2,
    the most negative centred lift; minus_one: q - 1 (digits (-1, 0))."""
    q = [251 ** 2, 127 ** 2, 253 ** 2]
    K = 70_000
    pick = {"half": lambda ql: (ql - 1) // 2, "half_below": lambda ql: (ql + 1) // 2, "minus_one": lambda ql: ql - 1}[kind]
    A = np.stack([np.full((70, K), pick(ql), np.uint64) for ql in q])
    Bm = np.stack([np.full((9, K), pick(ql), np.uint64) for ql in q])
    got = _run(q, A, Bm)
    for l, ql in enumerate(q):
        assert np.all(got[l] == (int(pick(ql)) ** 2 * K) % ql)


def test_p2_paper_slice_sampled():
    """The paper's per-GPU CCMM unit (one database slice of 2^14 rows x K = 24,576 against 992 query
    columns), the first 8 of its 24 moduli, in the benchmark's launch configuration: 24 sampled rows
    (first, last, tile edges, random) in every column and modulus equal the oracle's."""
    q = [p * p for p in PAPER_P[:8]]
    M, N, K = 1 << 14, 992, 24576
    g = torch.Generator(device="cuda").manual_seed(11)
    dA = torch.stack([torch.randint(0, ql, (M, K), device="cuda", dtype=torch.int64, generator=g) for ql in q])
    dB = torch.stack([torch.randint(0, ql, (N, K), device="cuda", dtype=torch.int64, generator=g) for ql in q])
    dC = E.ppmm("i8_p2", q, dA, dB)
    torch.cuda.synchronize()
    rows = np.unique(np.concatenate([[0, 1, 127, 128, 129, M - 129, M - 128, M - 1],
                                     np.random.default_rng(3).integers(0, M, 16)]))
    A = dA[:, torch.from_numpy(rows).cuda(), :].cpu().numpy().view(np.uint64)
    Bm = dB.cpu().numpy().view(np.uint64)
    got = dC[:, :, torch.from_numpy(rows).cuda()].cpu().numpy().view(np.uint64)
    del dA, dB, dC
    torch.cuda.empty_cache()
    assert np.array_equal(got, O.ppmm(q, A, Bm))
