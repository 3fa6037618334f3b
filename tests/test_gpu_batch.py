"""GPU tests of the batching form: several database chunks of uneven size (each its own MSRLWE
database with its own a-part) against one query batch in one grouped launch, captured in a CUDA
graph; results must equal the per-chunk path and the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_17561_gb300 import build as B
from paper_2601_17561_gb300 import engine as E
from paper_2601_17561_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [100, 4200, 333]


@pytest.fixture(scope="module")
def setup():
    B.build()
    W = synth.make_workload(n_eyes=3, n_db=sum(SIZES), seed=4, planted_frac=0.05, chunk_sizes=SIZES)
    eng = E.Engine(**E.TINY).keygen()
    dbs = [eng.encrypt_db(W.db_codes[s:s + n], W.db_masks[s:s + n], chunk_id=c) for c, (s, n) in enumerate(W.chunks)]
    ct = eng.encrypt_query(W.q_codes, W.q_masks, W.eye_ids)
    q = eng.prepare(ct, 3, "u64")
    ref = [eng.match(d, q).residues() for d in dbs]      # per-chunk u64 form
    torch.cuda.synchronize()
    return dict(W=W, eng=eng, dbs=dbs, ct=ct, ref=ref)


@pytest.mark.parametrize("form", ["f16_crt", "i8_crt", "u64"])
def test_grouped_launch_equals_per_chunk(setup, form):
    eng, dbs = setup["eng"], setup["dbs"]
    q = eng.prepare(setup["ct"], 3, form)
    outs = eng.match_batch(dbs, q)
    torch.cuda.synchronize()
    for s, ref in zip(outs, setup["ref"]):
        assert np.array_equal(s.residues(), ref)


def test_nonzero_chunk_against_oracle(setup):
    """Chunk 2 (own a-part stream) on sampled rows: a-part rows, every b-row and the tail rows."""
    W, ref = setup["W"], setup["ref"][2]
    P = O.Params(**O.TINY)
    start, n = W.chunks[2]
    ids = O.db_layout(n, P.ndb, P.rho)
    sel = np.concatenate([np.arange(0, 64), np.arange(len(ids) - (len(ids) - P.ndb), len(ids))])
    A = O.db_rows(P, W.db_codes[start:start + n], W.db_masks[start:start + n], ids[sel], chunk=2)
    Bq = O.query_extend(P, O.query_encrypt(P, W.q_codes, W.q_masks, W.eye_ids))
    want = O.ppmm(P.q, A, Bq)
    assert np.array_equal(ref[:, :, sel], want)


def test_graph_replay_and_fold(setup):
    eng, dbs = setup["eng"], setup["dbs"]
    st = torch.cuda.Stream()
    plan = eng.plan(dbs, 3, "f16_crt", setup["ct"], st)
    plan.launch(st)
    st.synchronize()
    first = [plan.folded_residues(i) for i in range(len(dbs))]
    plan.launch(st)
    st.synchronize()
    P = O.Params(**O.TINY)
    for i, d in enumerate(dbs):
        again = plan.folded_residues(i)
        assert np.array_equal(first[i], again)
        ids = O.db_layout(d.n_real, P.ndb, P.rho)
        assert np.array_equal(first[i], O.fold(P, setup["ref"][i], ids, 3, d.n_real))


def test_autotune_keeps_results(setup):
    eng, dbs = setup["eng"], setup["dbs"]
    q = eng.prepare(setup["ct"], 3, "f16_crt")
    best, ms = eng.autotune(dbs, q)
    # the fp16 form with an even K times the tcgen05 variants 1-3 (slots 2-4 of the fixed order
    # 128, 256, 1, 2, 3) and not the mma.sync tiles
    assert best in (1, 2, 3) and all(m > 0 for m in ms[2:5]) and ms[0] == 0 and ms[1] == 0
    outs = eng.match_batch(dbs, q)
    torch.cuda.synchronize()
    for s, ref in zip(outs, setup["ref"]):
        assert np.array_equal(s.residues(), ref)


@pytest.mark.parametrize("n_eyes", [1, 2])
def test_small_batches(setup, n_eyes):
    """Batches of 1 and 2 eyes: the same eyes give the same columns as in the 3-eye batch (eye ids
    key the encryption randomness)."""
    W, eng, dbs = setup["W"], setup["eng"], setup["dbs"]
    ct = eng.encrypt_query(W.q_codes[:n_eyes], W.q_masks[:n_eyes], W.eye_ids[:n_eyes])
    q = eng.prepare(ct, n_eyes, "f16_crt")
    outs = eng.match_batch(dbs, q)
    torch.cuda.synchronize()
    for s, ref in zip(outs, setup["ref"]):
        assert np.array_equal(s.residues(), ref[:, : n_eyes * 31, :])


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_grouped_tcgen05_variant(setup, variant):
    """tcgen05 variants over uneven chunks (ragged row tiles, partial column tile)."""
    from paper_2601_17561_gb300 import icm as C
    eng, dbs = setup["eng"], setup["dbs"]
    C.icm_ctx_set_variant(eng.ctx, variant)
    try:
        q = eng.prepare(setup["ct"], 3, "f16_crt")
        outs = eng.match_batch(dbs, q)
        torch.cuda.synchronize()
        C.icm_device_status(True)
        for s, ref in zip(outs, setup["ref"]):
            assert np.array_equal(s.residues(), ref)
    finally:
        C.icm_ctx_set_variant(eng.ctx, 0)


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_graph_replay_tcgen05_variant(setup, variant):
    """The tcgen05 variants captured in the plan's CUDA graph (the wave variants as cooperative
    launches with their counter reset by a memset node): two replays give the oracle's folded
    scores."""
    from paper_2601_17561_gb300 import icm as C
    eng, dbs = setup["eng"], setup["dbs"]
    C.icm_ctx_set_variant(eng.ctx, variant)
    try:
        st = torch.cuda.Stream()
        plan = eng.plan(dbs, 3, "f16_crt", setup["ct"], st)
        P = O.Params(**O.TINY)
        for _ in range(2):
            plan.launch(st)
            st.synchronize()
            C.icm_device_status(True)
            for i, d in enumerate(dbs):
                ids = O.db_layout(d.n_real, P.ndb, P.rho)
                assert np.array_equal(plan.folded_residues(i), O.fold(P, setup["ref"][i], ids, 3, d.n_real))
        del plan
    finally:
        C.icm_ctx_set_variant(eng.ctx, 0)
