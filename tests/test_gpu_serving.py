"""GPU tests of the serving form: eyes submitted one by one are batched by the request loop; each
eye's folded scores are bit-identical whether it ran alone or inside a mixed batch, equal the
direct (non-serving) path, and, on sampled eyes, the oracle's fold of the oracle's CCMM.  Batches
are admitted by device memory: a workspace of one full batch runs one batch at a time, the default
workspace runs two at once, and a workspace a little above one full batch admits a second, smaller
batch."""
import threading
import time

import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_17561_gb300 import build as B
from paper_2601_17561_gb300 import engine as E
from paper_2601_17561_gb300 import icm as C
from paper_2601_17561_gb300 import synth

pytestmark = pytest.mark.gpu
N_EYES = 7


@pytest.fixture(scope="module")
def setup():
    B.build()
    W = synth.make_workload(n_eyes=N_EYES, n_db=320, seed=9, planted_frac=0.05, chunk_sizes=[120, 200])
    eng = E.Engine(**E.TINY).keygen()
    dbs = [eng.encrypt_db(W.db_codes[s:s + n], W.db_masks[s:s + n], chunk_id=c) for c, (s, n) in enumerate(W.chunks)]
    ct = eng.encrypt_query(W.q_codes, W.q_masks, W.eye_ids)
    # direct path, one eye at a time: prepare + grouped CCMM + fold, flattened in the server's order
    direct = []
    for e in range(N_EYES):
        cte = eng.encrypt_query(W.q_codes[e:e + 1], W.q_masks[e:e + 1], W.eye_ids[e:e + 1])
        q = eng.prepare(cte, 1, "f16_crt")
        outs = [eng.fold(s) for s in eng.match_batch(dbs, q)]
        direct.append(np.concatenate([f.residues().reshape(-1) for f in outs]))
    torch.cuda.synchronize()
    # oracle, sampled eyes: the fold of the u128 product of every chunk, flattened the same way
    P = O.Params(**O.TINY)
    oracle = {}
    for e in (0, N_EYES - 1):
        Bq = O.query_extend(P, O.query_encrypt(P, W.q_codes[e:e + 1], W.q_masks[e:e + 1], W.eye_ids[e:e + 1]))
        parts = []
        for c, (s0, n) in enumerate(W.chunks):
            ids = O.db_layout(n, P.ndb, P.rho)
            A = O.db_rows(P, W.db_codes[s0:s0 + n], W.db_masks[s0:s0 + n], ids, chunk=c)
            parts.append(O.fold(P, O.ppmm(P.q, A, Bq), ids, n_eyes=1, n_real=n).reshape(-1))
        oracle[e] = np.concatenate(parts)
    return dict(W=W, eng=eng, dbs=dbs, ct=ct, direct=direct, oracle=oracle)


def test_direct_path_matches_oracle(setup):
    for e, want in setup["oracle"].items():
        assert np.array_equal(setup["direct"][e], want), e


def test_alone_and_mixed_results_identical(setup):
    eng, dbs = setup["eng"], setup["dbs"]
    srv = E.Server(eng, dbs, form="f16_crt", max_eyes=4, window_us=3000)
    cts = srv.eye_cts(setup["ct"], N_EYES)
    alone = []
    for e in range(N_EYES):
        out = np.zeros(srv.out_words, np.uint64)
        t = srv.submit(cts[e], out)
        srv.wait(t)
        alone.append(out)
    _, batches_alone, _ = srv.stats()
    assert batches_alone == N_EYES
    # mixed: submit every eye from two threads with Poisson gaps, then wait for all
    outs = [np.zeros(srv.out_words, np.uint64) for _ in range(N_EYES)]
    tickets = [None] * N_EYES
    rng = np.random.default_rng(3)

    def producer(idx):
        for e in idx:
            time.sleep(float(rng.exponential(0.0005)))
            tickets[e] = srv.submit(cts[e], outs[e])

    th = [threading.Thread(target=producer, args=(list(range(i, N_EYES, 2)),)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    lat = [srv.wait(t) for t in tickets]
    done, batches, mean_batch = srv.stats()
    srv.close()
    assert done == 2 * N_EYES
    assert batches - batches_alone < N_EYES and mean_batch > 1.0      # eyes were batched together
    assert all(x > 0 for x in lat)
    for e in range(N_EYES):
        assert np.array_equal(alone[e], setup["direct"][e])
        assert np.array_equal(outs[e], setup["direct"][e])
    for e, want in setup["oracle"].items():
        assert np.array_equal(outs[e], want), e


def _burst(srv, cts, n):
    """Submit n eyes (cycling through cts) as fast as possible, wait for all; outputs in order."""
    outs = [np.zeros(srv.out_words, np.uint64) for _ in range(n)]
    tickets = [srv.submit(cts[i % len(cts)], outs[i]) for i in range(n)]
    for t in tickets:
        srv.wait(t)
    return outs


@pytest.mark.parametrize("ws_batches,window_us,n", [(1.0, 10_000_000, 32), (1.5, 0, 40), (None, 0, 40)])
def test_admission_by_memory(setup, ws_batches, window_us, n):
    """Batches of up to 16 eyes, n eyes submitted back to back.  The pool never holds more than its
    size.  With one full batch of workspace and a long window (so every batch is full) only one
    batch is ever in flight: the second waits for the first one's memory.  With 1.5 full batches a
    second batch in flight is a partial one; with the default workspace (two full batches) at most
    two run at once.  Every result equals the direct path's."""
    eng, dbs = setup["eng"], setup["dbs"]
    probe = E.Server(eng, dbs, form="f16_crt", max_eyes=16, window_us=0)
    full = probe.memory()[1]
    probe.close()
    ws = None if ws_batches is None else int(full * ws_batches)
    srv = E.Server(eng, dbs, form="f16_crt", max_eyes=16, window_us=window_us, ws_bytes=ws)
    cts = srv.eye_cts(setup["ct"], N_EYES)
    outs = _burst(srv, cts, n)
    pool, full2, peak_bytes, peak_batches = srv.memory()
    done, batches, mean_batch = srv.stats()
    srv.close()
    print(f"workspace {ws_batches or 2.0} full batches: {batches} batches (mean {mean_batch:.1f} eyes), "
          f"peak {peak_batches} in flight, peak {peak_bytes / full:.2f} full batches reserved")
    assert full2 == full and 0 < peak_bytes <= pool and done == n and 1 <= peak_batches <= 2
    if ws_batches == 1.0:
        assert peak_batches == 1 and batches == 2 and peak_bytes == full
    elif ws_batches == 1.5 and peak_batches == 2:
        assert peak_bytes < 2 * full
    for i in range(n):
        assert np.array_equal(outs[i], setup["direct"][i % N_EYES]), i


def test_bounded_wait_and_admission(setup):
    eng, dbs = setup["eng"], setup["dbs"]
    srv = E.Server(eng, dbs, form="f16_crt", max_eyes=32, window_us=200000, max_pending=2)
    cts = srv.eye_cts(setup["ct"], 3)
    outs = [np.zeros(srv.out_words, np.uint64) for _ in range(3)]
    t0 = srv.submit(cts[0], outs[0])
    # the batch waits for its window, so a zero-length wait must time out, not block
    with pytest.raises(C.IcmError) as ex:
        srv.wait(t0, timeout_ms=0)
    assert ex.value.status == C.ICM_ETIMEOUT
    t1 = srv.submit(cts[1], outs[1])
    with pytest.raises(C.IcmError) as ex:               # admission bound of 2 waiting eyes
        srv.submit(cts[2], outs[2])
    assert ex.value.status == C.ICM_ENOMEM
    srv.wait(t0)
    srv.wait(t1)
    srv.close()
    assert np.array_equal(outs[0], setup["direct"][0]) and np.array_equal(outs[1], setup["direct"][1])
