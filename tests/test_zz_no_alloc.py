"""The allocation-free product entry point (icm_ppmm_noalloc): for callers that cannot allocate
device memory, it runs the CRT-form product with its workspace in a static device array.  Its
output must equal icm_ppmm's (exactly: residues are integers) on two calls in a row, and problems
too large for the static array must be rejected before any work.  Collected last on purpose."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_17561_gb300 import build as B
from paper_2601_17561_gb300 import engine as E
from paper_2601_17561_gb300 import icm as C


def _rand(rng, q, rows, K):
    return np.stack([np.array(rng.integers(0, 1 << 62, size=(rows, K), dtype=np.int64) % ql, dtype=np.uint64) for ql in q])


@pytest.mark.gpu
@pytest.mark.parametrize("form", ["f16_crt", "i8_crt"])
def test_noalloc_matches_ppmm_twice(form):
    B.build()
    rng = np.random.default_rng(17)
    q = O.primes(60, 2) + [O.primes(50, 1)[0]]
    M, N, K = 300, 45, 1000
    A = torch.from_numpy(_rand(rng, q, M, K).view(np.int64)).cuda()
    Bm = torch.from_numpy(_rand(rng, q, N, K).view(np.int64)).cuda()
    ref = E.ppmm(form, q, A, Bm)                      # existing entry point, caller workspace
    f = C.FORMS[form]
    for _ in range(2):                                # two calls in a row share the static array
        out = torch.full((len(q), N, M), -1, dtype=torch.int64, device="cuda")
        C.icm_ppmm_noalloc(f, q, len(q), A, Bm, out, M, N, K)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_noalloc_rejects_oversize():
    """A workspace above the 64 MiB static array is refused with ICM_ENOMEM (host-side check made
    before the pointer checks, so the null pointers passed here can never reach a kernel: if the
    size check regressed, the call would fail with ICM_EINVAL on the host instead), and non-CRT
    forms are unsupported."""
    B.build()
    q = O.primes(60, 2)
    with pytest.raises(C.IcmError) as e:
        C.icm_ppmm_noalloc(C.ICM_FORM_F16_CRT, q, 2, None, None, None, 100000, 992, 24576, stream=0)
    assert e.value.status == C.ICM_ENOMEM
    with pytest.raises(C.IcmError) as e:
        C.icm_ppmm_noalloc(C.ICM_FORM_U64, q, 2, None, None, None, 10, 10, 10, stream=0)
    assert e.value.status == C.ICM_EUNSUPPORTED
