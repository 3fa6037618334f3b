"""The N > 1 path on CPU: two gloo ranks, each with its own encrypted database shard (own a-part
stream) and the same query batch, computed with the oracle; no data moves between ranks except
the test's own gathers.  The union of the ranks' decrypted scores must equal the cleartext inner
products of the common queries against the union of the shards, and the job time is the maximum
over ranks."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2601_17561_gb300 import shard

CFG = dict(log_n_db=6, log_n_q=5, n_limbs=3, n_limbs_q=1, prime_bits=50, log2_delta=26, seed=11)
N_EYES, N_DB, WORLD = 2, 40, 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P = O.Params(h=16, **CFG)
        W, Wq = shard.shard_workload(rank, N_EYES, N_DB, seed=5)
        ids = O.db_layout(N_DB, P.ndb, P.rho)
        A = O.db_rows(P, W.db_codes, W.db_masks, ids, chunk=shard.chunk_id(rank))
        B = O.query_extend(P, O.query_encrypt(P, Wq.q_codes, Wq.q_masks, Wq.eye_ids))
        C = O.ppmm(P.q, A, B)
        dec = np.zeros((C.shape[1], N_DB), np.int64)
        for j in range(C.shape[1]):
            b_ids, nums, _ = O.decrypt_column(P, C[:, j, :], ids)
            real = b_ids < N_DB
            dec[j, b_ids[real]] = nums[real]
        queries = [None] * world
        dist.all_gather_object(queries, (Wq.q_codes.tobytes(), Wq.q_masks.tobytes(), Wq.eye_ids.tobytes()))
        shards = [None] * world
        dist.all_gather_object(shards, (W.db_codes, W.db_masks, dec, A[:, : P.ndb, :8].copy()))
        t = shard.job_time_ms(10.0 * (rank + 1), dist)
        if rank == 0:
            out_q.put((queries, shards, t, Wq.q_codes, Wq.q_masks))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_the_database():
    O.build()
    ctx = mp.get_context("spawn")
    out_q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, WORLD, port, out_q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    queries, shards, t, q_codes, q_masks = out_q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # every rank matched the same query batch
    assert all(q == queries[0] for q in queries)
    # the shards differ, and so do their a-parts (chunk ids key the a-part streams)
    assert not np.array_equal(shards[0][0], shards[1][0])
    assert not np.array_equal(shards[0][3], shards[1][3])
    # union of the ranks' decrypted scores == cleartext inner products against the union
    P = O.Params(h=16, **CFG)
    codes = np.concatenate([s[0] for s in shards])
    masks = np.concatenate([s[1] for s in shards])
    rc, rm = O.rotated_templates(q_codes, q_masks, P.rho)
    num, den = O.hd_counts(rc, rm, O.unpack(codes), O.unpack(masks))
    want = O.inner_from_counts(num, den)
    got = np.concatenate([s[2] for s in shards], axis=1)
    assert np.array_equal(got, want)
    # the job time is the slowest rank's; the rate counts every rank's comparisons
    assert t == 10.0 * WORLD
    assert shard.job_rate(WORLD, N_EYES * N_DB, t) == WORLD * N_EYES * N_DB / (t / 1e3)


def _fold_rank_main(rank, world, port, n, out_q):
    """One rank of a sharded folding check: its consecutive trial range, counters summed."""
    import torch
    from oracle import folding as F
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t0, cnt = shard.trial_range(rank, world, n)
        fmin, fmax = F.poly_range(F.PAPER_FOLD_COEF, 0.3, 0.3005)
        r = F.fold_mc(F.PAPER_FOLD_COEF, *F.PAPER_D, 16, (0.3, 0.3005), (0.0, 0.03), (fmin + 0.01, fmin + 0.02),
                      seed=21, trial0=t0, n_trials=cnt, hist=(-0.02, 0.08, 20))
        counts = shard.job_sum(torch.from_numpy(r["counts"]), dist).numpy()
        hist = shard.job_sum(torch.from_numpy(r["hist"]), dist).numpy()
        sums = [None] * world
        dist.all_gather_object(sums, (t0, cnt, r["sk"], r["sk1"]))
        if rank == 0:
            out_q.put((counts, hist, sums))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_the_folding_trials():
    """The folding check's N > 1 path: each rank runs its own consecutive trial range (an odd total,
    so the ranges differ in length); the summed counters and histograms, and the ranks' per-trial
    sums in rank order, equal the single run's."""
    from oracle import folding as F
    n = 6001
    ctx = mp.get_context("spawn")
    out_q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_fold_rank_main, args=(r, WORLD, port, n, out_q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    counts, hist, sums = out_q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [(s[0], s[1]) for s in sums] == [(0, 3001), (3001, 3000)]
    fmin, fmax = F.poly_range(F.PAPER_FOLD_COEF, 0.3, 0.3005)
    one = F.fold_mc(F.PAPER_FOLD_COEF, *F.PAPER_D, 16, (0.3, 0.3005), (0.0, 0.03), (fmin + 0.01, fmin + 0.02),
                    seed=21, trial0=0, n_trials=n, hist=(-0.02, 0.08, 20))
    assert np.array_equal(counts, one["counts"]) and np.array_equal(hist, one["hist"])
    assert np.array_equal(np.concatenate([s[2] for s in sums]), one["sk"])
    assert np.array_equal(np.concatenate([s[3] for s in sums]), one["sk1"])
    assert shard.trial_range(3, 4, 10) == (8, 2) and shard.trial_range(0, 4, 10) == (0, 3)


def test_trial_ranges_tile_the_run():
    """For every world size (also more ranks than trials) the ranks' ranges are consecutive, cover
    [0, n) exactly and differ in length by at most one."""
    for n in (0, 1, 7, 6001, 2**33 + 5):
        for world in (1, 2, 3, 8, 13):
            rs = [shard.trial_range(r, world, n) for r in range(world)]
            assert rs[0][0] == 0 and sum(c for _, c in rs) == n
            assert all(rs[i][0] + rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            assert max(c for _, c in rs) - min(c for _, c in rs) <= 1


def _lib_rank_main(rank, world, port, n_db, out_q):
    """One rank's host-side view of its shard through the library (no GPU work): context, primes,
    CRT moduli, the shard's stored rows and bytes, and its per-step match footprint."""
    from paper_2601_17561_gb300 import engine as E
    from paper_2601_17561_gb300 import icm as C
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = dict(E.PAPER)
        ctx = C.icm_ctx_create(C.icm_params(log_n_db=p["log_n_db"], log_n_q=p["log_n_q"], n_limbs=p["n_limbs"],
                                            n_limbs_q=p["n_limbs_q"], prime_bits=p["prime_bits"], code_bits=12800,
                                            d2=1 << 14, rho=31, fold_k=16, hamming_weight=512,
                                            log2_delta=p["log2_delta"], noise_eta=21, seed=p["seed"]))
        try:
            nbytes, m_rows = C.icm_db_bytes(ctx, n_db)
            view = (C.icm_ctx_primes(ctx, p["n_limbs"]), C.icm_ctx_crt_moduli(ctx), n_db, m_rows, nbytes,
                    C.icm_query_ct_bytes(ctx, 32), shard.chunk_id(rank))
        finally:
            C.icm_ctx_destroy(ctx)
        views = [None] * world
        dist.all_gather_object(views, view)
        if rank == 0:
            out_q.put(views)
    finally:
        dist.destroy_process_group()


def test_two_ranks_library_host_view():
    """The N > 1 path through the library's host side on two gloo ranks: every rank's context has
    the same primes and CRT moduli (the query batch is common), each rank's shard of 7 x 2^14
    templates is laid out as 7 full blocks (M = 8 x 2^14 rows, 206 GB at the paper shape), and the
    query ciphertext a rank receives is the same size on every rank."""
    from paper_2601_17561_gb300 import build as B
    B.build()
    n_db = 7 * (1 << 14)
    ctx = mp.get_context("spawn")
    out_q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_lib_rank_main, args=(r, WORLD, port, n_db, out_q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    views = out_q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(v[0] == views[0][0] and v[1] == views[0][1] for v in views)
    assert len(views[0][1]) == 18
    for v in views:
        assert v[2] == n_db and v[3] == 8 * (1 << 14)
        assert v[4] == 8 * v[3] * ((1 << 14) + (1 << 13)) * 8
        assert v[5] == views[0][5] == 2 * 32 * 31 * ((1 << 14) + (1 << 13)) * 8
    assert [v[6] for v in views] == list(range(WORLD))            # every shard its own a-part stream
