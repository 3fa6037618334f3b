"""Run one matching pass of a named synthetic workload through the library (CLI).

    python -m paper_2601_17561_gb300.run --workload mid --form f16_crt --passes 2

Workloads: tiny (4 eyes x 256 codes, ring 2^12, 3 primes < 2^50), mid (32 eyes x 2,000 codes,
same ring and primes: about 3 GB on the device, sized for profiler captures), slice (32 eyes x
4,096 codes with the paper's query side -- N_q = 2^13, d = 2^14, K = 24,576, primes < 2^60, so
18 CRT moduli -- but N_db = 2^12 and 2 primes: M = 8,192 rows, 3.2 GB, the paper's tile shape
and wave order at a profiler-sized scale), paper (32 eyes x 114,688 codes, N_db = 2^14,
N_q = 2^13, 8 primes < 2^60), slots (a slot-encoded database of 1,024 templates in one block of
N_db = 2^11, the paper's query side for 32 eyes, 4 primes < 2^60: 3.2 GB).  Each pass prepares the
query, runs the CCMM and the fold (and, with --rescale, the rescaling by Q'); for `slots` a pass
is the query preparation, the CCMM, the rescaling and the normalisation by the mask overlaps.

    python -m paper_2601_17561_gb300.run --fold-trials 268435456

runs the cleartext check of the paper's folding polynomial instead (Appendix C.2 experiments on
N(0.008, 0.034^2) scores, positive interval [0.3, 0.45]) and prints the six outlier counts.
"""
from __future__ import annotations

import argparse
import sys
import time

import torch

from . import build as B
from . import engine as E
from . import icm as C
from . import synth

WORKLOADS = {
    "tiny": (E.TINY, dict(n_eyes=4, n_db=256, seed=1, planted_frac=0.05)),
    "mid": (E.TINY, dict(n_eyes=32, n_db=2000, seed=3, planted_frac=0.05)),
    "slice": (dict(log_n_db=12, log_n_q=13, n_limbs=2, n_limbs_q=1, prime_bits=60, log2_delta=40, seed=4),
              dict(n_eyes=32, n_db=4096, seed=4, planted_frac=0.05)),
    "paper": (E.PAPER, dict(n_eyes=32, n_db=7 * (1 << 14), seed=2, planted_frac=0.05)),
    "slots": (dict(log_n_db=11, log_n_q=13, n_limbs=4, n_limbs_q=2, prime_bits=60, log2_delta=60, seed=9),
              dict(n_eyes=32, n_db=1024, seed=9, planted_frac=0.05)),
}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="tiny", choices=sorted(WORKLOADS))
    ap.add_argument("--form", default="f16_crt", choices=["u64", "i8_digits", "i8_crt", "f16_crt"])
    ap.add_argument("--passes", type=int, default=1)
    ap.add_argument("--variant", type=int, default=None,
                    help="CRT product kernel: 1 = tcgen05, 128 / 256 = mma.sync column tile (default: library's)")
    ap.add_argument("--fold-trials", type=int, default=0, help="run the folding-polynomial check instead")
    ap.add_argument("--rescale", action="store_true", help="also rescale the CCMM result by Q' each pass")
    a = ap.parse_args(argv)
    B.build()
    if a.fold_trials:
        from . import folding as FD
        for i in range(a.passes):
            t0 = time.perf_counter()
            r = FD.fold_mc(a.fold_trials, seed=1 + i)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            print(f"pass {i}: {dt * 1e3:.1f} ms, {a.fold_trials / dt:.3e} trials/s, counts "
                  f"{[int(x) for x in r.counts.cpu()]}", flush=True)
        return 0
    params, wl = WORKLOADS[a.workload]
    W = synth.make_workload(**wl)
    eng = E.Engine(**params).keygen()
    if a.variant is not None:
        C.icm_ctx_set_variant(eng.ctx, a.variant)
    ct = eng.encrypt_query(W.q_codes, W.q_masks, W.eye_ids)
    if a.workload == "slots":
        db = eng.encrypt_db_slots(W.db_codes, W.db_masks, log2_scale=16)
        qm = torch.from_numpy(W.q_masks.copy()).to(eng.device)
        dm = torch.from_numpy(W.db_masks.copy()).to(eng.device)
        torch.cuda.synchronize()
        for i in range(a.passes):
            t0 = time.perf_counter()
            r = eng.rescale(eng.match(db, eng.prepare(ct, wl["n_eyes"], a.form)))
            eng.normalize(r, qm, dm, 36)
            torch.cuda.synchronize()
            print(f"pass {i}: {(time.perf_counter() - t0) * 1e3:.1f} ms (slots, {a.form})", flush=True)
        return 0
    db = eng.encrypt_db(W.db_codes, W.db_masks)
    torch.cuda.synchronize()
    for i in range(a.passes):
        t0 = time.perf_counter()
        q = eng.prepare(ct, wl["n_eyes"], a.form)
        s = eng.match(db, q)
        eng.fold(s)
        if a.rescale:
            eng.rescale(s)
        torch.cuda.synchronize()
        print(f"pass {i}: {(time.perf_counter() - t0) * 1e3:.1f} ms ({a.workload}, {a.form})", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
