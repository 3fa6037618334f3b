#!/usr/bin/env python3
"""Benchmark of the encrypted 1:N iris matching hot path on GB300.

One step = one pass of the whole hot path over one query batch: basis extension of the query
ciphertext (and its tensor-core planes), the CCMM against the resident encrypted database, and
the fold.  Workload (Section 6): 32 query eyes x 31 rotations against 7 x 2^14 = 114,688 database
iris codes, N_db = 2^14, N_q = 2^13, d = 2^14, eight primes below 2^60 (L_q = 2); synthetic
templates (uniform codes, Bernoulli(0.9) masks, 5% planted noisy copies).  The encrypted database
(206 GB) is built once before timing and stays resident; it exceeds L2 many times over, so no L2
flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--form F] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank matches the same query batch against
its own database of 114,688 codes (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "iris comparisons/s (32 eyes × 7·2^14 DB, 1 GB300), int8-TC vs u64 form; % INT8 peak"
UNIT = "comparisons/s"
N_EYES, N_DB = 32, 7 * (1 << 14)
WORKLOAD = ("paper-shaped CCMM + fold: 32 eyes x 31 rotations vs 114,688 codes (7 blocks of N_db=2^14), "
            "N_q=2^13, d=2^14, K=24,576, 8 primes < 2^60 (L_q=2), Delta=2^60")
DTYPE = {"u64": "u64", "i8_digits": "int8", "i8_crt": "int8", "f16_crt": "f16"}
# DRAM bytes (read + write) of the dominant kernel per CCMM call, keyed by (form, tcgen05
# variant), from one-pass ncu captures of the current kernels on the 8,192-row slice of this shape
# (2 limbs) scaled by 64 (16x the row tiles, 4x the limbs: the traffic of a wave of co-resident
# tiles does not depend on M, and the waves grow with row tiles x limbs x rounds); the int8 CRT
# figure scales one 512-column round by 2 rounds.  Absent (null) for a kernel changed since.
NCU_TRAFFIC = {
    ("f16_crt", 2): 64 * (22_524_419_072 + 299_334_656),
    ("i8_crt", 0): 2 * 64 * (12_100_983_040 + 155_742_464),
    ("u64", 0): 64 * (96_624_647_000 + 141_553_920),
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling (200 ms) during the timed region."""

    def __init__(self, dev: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(dev)], stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ------------------------------------------------------------------------------ CPU oracle legs

def oracle_sample(seconds_target: float, seed: int = 0):
    """Time the oracle on a bounded sample of the same workload: basis extension of the whole
    query operand, the u128 schoolbook product for a sample of database rows against all 992
    columns and 8 limbs, and the fold of those rows.  Uniform random residues stand in for the
    operands (the oracle's arithmetic does not depend on their values).  Returns
    (comparisons/s extrapolated to the whole workload, threads, sample description, seconds)."""
    import numpy as np
    import oracle as O

    P = O.Params(**O.PAPER)
    q = P.q
    rng = np.random.default_rng(seed)
    n_cols = N_EYES * P.rho
    M_total = P.ndb + N_DB
    ct = np.stack([rng.integers(0, q[l], size=(n_cols, P.K), dtype=np.uint64) for l in range(P.n_limbs_q)])
    t0 = time.perf_counter()
    Bq = O.query_extend(P, ct)
    t_ext = time.perf_counter() - t0

    def rows(S):
        return np.stack([rng.integers(0, q[l], size=(S, P.K), dtype=np.uint64) for l in range(P.n_limbs)])

    # calibrate the row count
    S = 4
    A = rows(S)
    t0 = time.perf_counter()
    O.ppmm(q, A, Bq)
    t4 = time.perf_counter() - t0
    S = max(4, min(4096, int(S * max(seconds_target - t_ext, 1.0) / max(t4, 1e-3))))
    A = rows(S)
    t0 = time.perf_counter()
    C = O.ppmm(q, A, Bq)
    t_mm = time.perf_counter() - t0
    # fold of the sampled rows (a-part coefficients 30..S-1 have every source present)
    ids = np.arange(S, dtype=np.int64)
    t0 = time.perf_counter()
    O.fold(P, C, ids, N_EYES, 0)
    t_fold = time.perf_counter() - t0
    t_full = t_ext + (t_mm + t_fold) * M_total / S
    value = N_EYES * N_DB / t_full
    sample = (f"oracle basis extension of the full query ({n_cols} cols x {P.K} x 2 limbs) + u128 schoolbook "
              f"PPMM of {S} of {M_total} database rows x {n_cols} cols x 8 limbs + fold of those rows, "
              f"extrapolated linearly in rows; uniform random residues")
    return value, O.threads(), sample, t_ext + t_mm + t_fold


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    times, vals = [], []
    threads, sample = None, None
    for i in range(args.warmup + args.steps):
        v, threads, sample, secs = oracle_sample(seconds_target=6.0, seed=i)
        if i >= args.warmup:
            vals.append(v)
            times.append(secs)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": N_EYES * N_DB / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "oracle u128 schoolbook (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ batching and serving forms

def run_batching(args, dev):
    """Batching form: 7 database chunks of floor(2^14 U[0.5, 1.5]) codes (seeded), each its own
    MSRLWE database with its own a-part; query batches of 1, 3, 8, 17 and 32 eyes, each pass one
    CUDA-graph replay of query preparation + grouped CCMM (one persistent launch per column round
    over every limb, chunk and tile) + folds.  Four primes below 2^60 (L_q = 2) so that the seven
    a-parts fit in HBM (180 GB); N_db = 2^14, N_q = 2^13, K = 24,576."""
    import torch
    from paper_2601_17561_gb300 import engine as E
    from paper_2601_17561_gb300 import synth
    sizes = synth.uneven_chunk_sizes(7, 1 << 14, seed=4)
    W = synth.make_workload(n_eyes=32, n_db=sum(sizes), seed=4, planted_frac=0.05, chunk_sizes=sizes)
    params = dict(E.PAPER)
    params.update(n_limbs=4, n_limbs_q=2)
    eng = E.Engine(**params).keygen()
    dbs = [eng.encrypt_db(W.db_codes[s:s + n], W.db_masks[s:s + n], chunk_id=c) for c, (s, n) in enumerate(W.chunks)]
    torch.cuda.synchronize()
    st = torch.cuda.Stream(device=dev)
    out = {}
    for n_eyes in (1, 3, 8, 17, 32):
        ct = eng.encrypt_query(W.q_codes[:n_eyes], W.q_masks[:n_eyes], W.eye_ids[:n_eyes])
        q = eng.prepare(ct, n_eyes, args.form)
        best, ms = eng.autotune(dbs, q)
        plan = eng.plan(dbs, n_eyes, args.form, ct, st)
        plan.launch(st)
        st.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(1, args.steps)
        a.record(st)
        for _ in range(reps):
            plan.launch(st)
        b.record(st)
        st.synchronize()
        t = a.elapsed_time(b) / reps
        out[str(n_eyes)] = {"ms_per_batch": t, "comparisons_per_s": n_eyes * sum(sizes) / (t / 1e3),
                            "variant": best}
        del plan, q, ct
        torch.cuda.empty_cache()
    line = {"metric": "batching form: iris comparisons/s per query batch (7 uneven chunks, one graph per batch)",
            "unit": "comparisons/s", "n_gpus": 1, "data": "synthetic", "dtype": DTYPE[args.form],
            "config": {"workload": "7 chunks of floor(2^14 U[0.5,1.5]) codes (seed 4): " + ",".join(map(str, sizes)) +
                       f"; 4 primes < 2^60; form {args.form}", "form": args.form},
            "batches": out}
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args, dev):
    """Serving form: a resident encrypted database of 2^17 codes (8 primes), query eyes submitted
    one by one at Poisson rates; the request loop admits them by free device memory, batches up to
    32 eyes per launch and overlaps consecutive batches (two batch slots where the memory left
    beside the database holds two full batches).  Each rate submits for --seconds or until
    --serving-eyes eyes, whichever comes first, then drains.  Reports eyes/s and p50/p99 latency
    (submission to result) per rate; checks sampled results bit-exact against the direct
    (non-serving) path."""
    import numpy as np
    import torch
    from paper_2601_17561_gb300 import engine as E
    from paper_2601_17561_gb300 import icm as C
    from paper_2601_17561_gb300 import synth
    n_db = 1 << 17
    pool = 64
    W = synth.make_workload(n_eyes=pool, n_db=n_db, seed=5, planted_frac=0.05)
    eng = E.Engine(**E.PAPER).keygen()
    db = eng.encrypt_db(W.db_codes, W.db_masks)
    ct = eng.encrypt_query(W.q_codes, W.q_masks, W.eye_ids)
    torch.cuda.synchronize()
    best = None
    if args.form in ("i8_crt", "f16_crt"):
        qt = eng.prepare(eng.encrypt_query(W.q_codes[:32], W.q_masks[:32], W.eye_ids[:32]), 32, args.form)
        best, _ = eng.autotune([db], qt)
        del qt
        torch.cuda.empty_cache()
    # reference for two sampled eyes through the direct path (before the server takes its pool)
    refs = {}
    for e in (0, pool - 1):
        cte = eng.encrypt_query(W.q_codes[e:e + 1], W.q_masks[e:e + 1], W.eye_ids[e:e + 1])
        qq = eng.prepare(cte, 1, args.form)
        refs[e] = eng.fold(eng.match(db, qq)).residues().reshape(-1)
        del qq, cte
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    cfg1 = C.icm_server_cfg(max_eyes=32, window_us=args.window_us, form=C.FORMS[args.form], max_batches=1)
    full = C.icm_server_device_bytes(eng.ctx, [db.handle], cfg1)
    free = torch.cuda.mem_get_info(dev)[0]
    margin = 4 << 30
    ws_bytes = min(2 * full, max(full, free - margin))
    srv = E.Server(eng, [db], form=args.form, max_eyes=32, window_us=args.window_us, ws_bytes=ws_bytes)
    cts = srv.eye_cts(ct, pool)
    rng = np.random.default_rng(5)
    rates = [float(x) for x in args.rates.split(",")]
    results = {}
    ok = True
    for lam in rates:
        b0 = srv.stats()
        outs, tickets = [], []
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < args.seconds and n < args.serving_eyes:
            e = n % pool
            o = np.zeros(srv.out_words, np.uint64)
            tickets.append((e, srv.submit(cts[e], o)))
            outs.append(o)
            n += 1
            time.sleep(float(rng.exponential(1.0 / lam)))
        t_sub = time.perf_counter() - t0
        lat = [srv.wait(t) for _, t in tickets]
        wall = time.perf_counter() - t0
        for (e, _), o in zip(tickets, outs):
            if e in refs and not np.array_equal(o, refs[e]):
                ok = False
        b1 = srv.stats()
        lat = np.array(lat)
        results[str(lam)] = {"eyes": n, "offered_eyes_per_s": n / t_sub, "eyes_per_s": n / wall,
                             "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                             "batches": int(b1[1] - b0[1]), "mean_batch": n / max(1, int(b1[1] - b0[1]))}
    pool_bytes, full_bytes, peak_bytes, peak_batches = srv.memory()
    srv.close()
    sat = max(r["eyes_per_s"] for r in results.values())
    line = {"metric": "serving form: p50/p99 latency and eyes/s at Poisson arrival rates", "unit": "ms",
            "n_gpus": 1, "data": "synthetic", "dtype": DTYPE[args.form],
            "config": {"workload": "resident database of 2^17 codes (M = 147,456), 8 primes < 2^60; "
                       f"<= 32 eyes per launch, window {args.window_us} us, up to {args.seconds} s or "
                       f"{args.serving_eyes} eyes per rate", "form": args.form, "variant": best},
            "memory": {"pool_bytes": pool_bytes, "full_batch_bytes": full_bytes, "peak_reserved_bytes": peak_bytes,
                       "peak_batches_in_flight": peak_batches},
            "rates": results, "max_served_eyes_per_s": sat, "sampled_results_bit_exact": ok}
    print(json.dumps(line), flush=True)
    return 0


def _exact_hd(q_codes, q_masks, db_codes, db_masks, rho, dev):
    """Cleartext fractional Hamming distances of every (eye x rotation, template) pair, from the
    packed bits with exact fp64 matrix products on the device (a check, not the measured path):
    HD = (||m AND m'|| - <c', c''>) / (2 ||m AND m'||) with c' = m - 2 (c AND m)."""
    import numpy as np
    import torch

    def bits(x):
        t = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
        b = (t.unsqueeze(-1) >> torch.arange(8, device=dev, dtype=torch.uint8)) & 1
        return b.reshape(t.shape[0], -1)[:, :12800]

    qc, qm = bits(q_codes).view(-1, 16, 200, 4), bits(q_masks).view(-1, 16, 200, 4)
    cols_c, cols_m = [], []
    for e in range(qc.shape[0]):
        for r in range(rho):
            sft = r - (rho - 1) // 2
            cols_c.append(torch.roll(qc[e], shifts=-sft, dims=1).reshape(-1))
            cols_m.append(torch.roll(qm[e], shifts=-sft, dims=1).reshape(-1))
    qc, qm = torch.stack(cols_c).double(), torch.stack(cols_m).double()
    dc, dm = bits(db_codes).double(), bits(db_masks).double()
    qcp = qm - 2 * qc * qm
    dcp = dm - 2 * dc * dm
    den = qm @ dm.T
    inner = qcp @ dcp.T
    hd = torch.where(den > 0, (den - inner) / (2 * den.clamp(min=1)), torch.ones_like(den))
    return hd


def run_slots(args, dev):
    """Slot-encoded database and normalisation (Section 2.2.1 Ecd_slot, Section 2.3, Algorithm 2's
    ct (.) mu) on the paper's query side: 32 eyes x 31 rotations against 2^15 templates in 4
    blocks of N_db/2 = 8,192 (one template per slot), N_db = 2^14, N_q = 2^13, 8 primes < 2^60
    (L_q = 2), Delta 2^60, database slot scale 2^16, mu scale 2^36.  One step: query preparation,
    CCMM (fp16 CRT form, tcgen05 kernel), rescaling by Q', normalisation; CUDA events on the
    launching stream around each part.  The decoded distances of all pairs are compared with the
    exact cleartext distances."""
    import numpy as np
    import torch
    from paper_2601_17561_gb300 import engine as E
    from paper_2601_17561_gb300 import icm as C
    from paper_2601_17561_gb300 import synth
    n_db, n_eyes, s_db, s_mu = 1 << 15, 32, 16, 36
    W = synth.make_workload(n_eyes=n_eyes, n_db=n_db, seed=6, planted_frac=0.05)
    eng = E.Engine(**E.PAPER).keygen()
    t0 = time.perf_counter()
    db = eng.encrypt_db_slots(W.db_codes, W.db_masks, log2_scale=s_db)
    torch.cuda.synchronize()
    enc_s = time.perf_counter() - t0
    ct = eng.encrypt_query(W.q_codes, W.q_masks, W.eye_ids)
    qm = torch.from_numpy(np.ascontiguousarray(W.q_masks)).to(dev)
    dm = torch.from_numpy(np.ascontiguousarray(W.db_masks)).to(dev)
    st = torch.cuda.Stream(device=dev)
    q = eng.prepare(ct, n_eyes, "f16_crt", stream=st)
    mws = eng.match_workspace(db, n_eyes, "f16_crt")
    s = eng.match(db, q, stream=st, ws=mws)
    r = eng.rescale(s, stream=st)
    ob, wb = C.icm_normalize_bytes(r.handle)
    out, ws = E._u8(ob, dev), E._u8(wb, dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    with torch.cuda.stream(st):
        for _ in range(max(1, args.warmup)):
            eng.prepare(ct, n_eyes, "f16_crt", stream=st, out=q.buf)
            eng.match(db, q, stream=st, out=s.buf, ws=mws)
            eng.rescale(s, stream=st, out=r.buf)
            eng.normalize(r, qm, dm, s_mu, stream=st, out=out, ws=ws)
        st.synchronize()
        for e in ev:
            e[0].record(st)
            eng.prepare(ct, n_eyes, "f16_crt", stream=st, out=q.buf)
            eng.match(db, q, stream=st, out=s.buf, ws=mws)
            e[1].record(st)
            eng.rescale(s, stream=st, out=r.buf)
            e[2].record(st)
            eng.normalize(r, qm, dm, s_mu, stream=st, out=out, ws=ws)
            e[3].record(st)
        st.synchronize()
    ccmm = statistics.median(e[0].elapsed_time(e[1]) for e in ev)
    resc = statistics.median(e[1].elapsed_time(e[2]) for e in ev)
    norm = statistics.median(e[2].elapsed_time(e[3]) for e in ev)
    step = statistics.median(e[0].elapsed_time(e[3]) for e in ev)
    C.icm_device_status(True)
    hd = eng.decrypt_slots(r, out, s_mu)
    ref = _exact_hd(W.q_codes, W.q_masks, W.db_codes, W.db_masks, 31, dev)
    err = float((hd - ref).abs().max())
    torch.cuda.synchronize()
    L_q, d3, N = eng.Lq, n_eyes * 31, 1 << 14
    nb = n_db // (N // 2)
    M = N + nb * N
    # normalisation bytes: rescaled scores read (a-parts and b-rows), normalised pairs written
    nbytes = L_q * d3 * M * 8 + L_q * d3 * nb * 2 * N * 8
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    line = {"metric": "slot-encoded database + normalisation: iris comparisons/s and decoded-HD error",
            "value": n_eyes * 31 * n_db / (step / 1e3), "unit": "comparisons/s (rotations x templates)",
            "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": max(1, args.warmup),
            "ms_per_step": step, "data": "synthetic", "dtype": "f16 CCMM, u64 NTT, f64 FFT",
            "config": {"workload": "32 eyes x 31 rotations vs 2^15 templates, slot-encoded (4 blocks of 8,192), "
                                   "N_db = 2^14, N_q = 2^13, 8 primes < 2^60 (L_q = 2), Delta 2^60, "
                                   f"slot scale 2^{s_db}, mu scale 2^{s_mu}", "form": "f16_crt",
                       "database_gb": round(db.buf.numel() / 1e9, 1)},
            "parts_ms": {"prepare_and_ccmm": ccmm, "rescale": resc, "normalize": norm},
            "normalize_roofline": {"bound": "hbm", "bytes": nbytes, "achieved": nbytes / (norm / 1e3) / 1e9,
                                   "peak": hbm, "unit": "GB/s", "frac": nbytes / (norm / 1e3) / 1e9 / hbm,
                                   "peak_source": "of measured: MEASURED_PEAKS.json hbm_gbs",
                                   "note": "rescaled scores read once, normalised pairs written once; the "
                                           "NTTs run in shared memory"},
            "database_encode_s": enc_s,
            "decode": {"hd_error_max": err, "hd_tolerance": 2.0 ** -10, "pairs": n_eyes * 31 * n_db,
                       "reference": "exact cleartext distances (fp64 integer matrix products on the device)"}}
    print(json.dumps(line), flush=True)
    return 0


def run_p2(args, dev):
    """The paper's own modulus family on its per-GPU CCMM unit (Section 6.2.2; Table 2 times it at
    259 ms on an RTX-5090): Q = prod p^2 over the 24 primes 127 <= p <= 253 (2^360.8), one database
    slice of 2^14 rows x K = 24,576 against 32 eyes x 31 rotations = 992 columns; every modulus is
    two int8 passes (x0 y0 over K, x0 y1 + x1 y0 over 2K).  One step = three icm_ppmm calls of 8
    moduli; random residues below 127^2 so one operand pair serves every modulus."""
    import torch
    from paper_2601_17561_gb300 import engine as E
    from paper_2601_17561_gb300 import icm as C
    ps = [p for p in range(127, 254) if all(p % d for d in range(2, int(p ** 0.5) + 1))]
    M, N, K = 1 << 14, 992, 24576
    g = torch.Generator(device=dev).manual_seed(1)
    A = torch.randint(0, 127 * 127, (8, M, K), device=dev, dtype=torch.int64, generator=g)
    Bm = torch.randint(0, 127 * 127, (8, N, K), device=dev, dtype=torch.int64, generator=g)
    Cm = torch.empty((8, N, M), device=dev, dtype=torch.int64)
    groups = [[p * p for p in ps[i:i + 8]] for i in (0, 8, 16)]
    ws_bytes = C.icm_ppmm_workspace_bytes(C.ICM_FORM_I8_P2, 8, M, N, K)
    ws = E._u8(ws_bytes, dev)
    st = torch.cuda.Stream(device=dev)

    def step():
        for q in groups:
            C.icm_ppmm(C.ICM_FORM_I8_P2, q, 8, A, Bm, Cm, M, N, K, ws, ws_bytes, st)

    with torch.cuda.stream(st):
        for _ in range(max(1, args.warmup)):
            step()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(args.steps):
            step()
        b.record(st)
        st.synchronize()
    ms = a.elapsed_time(b) / args.steps
    ops = 2.0 * M * N * 3 * K * len(ps)
    peak = 2.0 * C.icm_probe_peak(1)
    line = {"metric": "paper's p^2 modulus family: ms per CCMM slice (2^14 rows x 24,576 x 992, 24 moduli p^2)",
            "value": ms, "unit": "ms", "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "data": "synthetic", "dtype": "s8",
            "config": {"workload": "one database slice: M = 16,384, K = 24,576, N = 992; Q = prod p^2, 127 <= p <= 253 "
                                   "(24 moduli, 2^360.8); 3 x icm_ppmm of 8 moduli", "form": "i8_p2"},
            "paper_ms_rtx5090": 259.0,
            "roofline": {"bound": "tensor", "kernel": "k_ppmm_p2", "achieved": ops / (ms / 1e3) / 1e12,
                         "peak": peak / 1e12, "unit": "TOP/s", "frac": ops / (ms / 1e3) / peak,
                         "peak_source": "measured in this run: int8 mma.sync.m16n8k32 issue-bound probe "
                                        "(no tcgen05 int8 on sm_103a)",
                         "ops": "2 x M x N x 3K x 24 int8 operations (passes of K and 2K per modulus)"}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ GPU arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="icm", choices=["icm", "reference"])
    ap.add_argument("--form", default="f16_crt", choices=["u64", "i8_digits", "i8_crt", "f16_crt"])
    ap.add_argument("--form-steps", type=int, default=3, help="timed steps of each compared form")
    ap.add_argument("--form-warmup", type=int, default=1, help="warm-up steps of each compared form")
    ap.add_argument("--compare-forms", default="i8_crt,u64",
                    help="comma list of other forms, each timed (--form-warmup, --form-steps) on the same "
                         "workload ('' to skip; i8_digits takes ~33 s per step)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--variant", default="auto",
                    help="CRT product kernel: auto (autotuner), 128 / 256 (mma.sync) or 1..3 (tcgen05)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fold-trials", type=int, default=1 << 33,
                    help="trials of the folding-polynomial check reported beside the step (0: skip)")
    ap.add_argument("--workload", default="paper", choices=["paper", "batching", "serving", "p2", "slots"],
                    help="paper: the headline CCMM step; batching / serving: the query-batching and "
                         "request-loop forms; p2: the paper's p^2 modulus family on one CCMM slice; "
                         "slots: the slot-encoded database and the normalisation "
                         "(one JSON line each, not the headline)")
    ap.add_argument("--rates", default="16,32,64,128,256,512", help="serving: Poisson arrival rates (eyes/s)")
    ap.add_argument("--seconds", type=float, default=20.0, help="serving: longest submission time per rate")
    ap.add_argument("--serving-eyes", type=int, default=320, help="serving: most eyes submitted per rate")
    ap.add_argument("--window-us", type=int, default=20000, help="serving: batching window")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import numpy as np
    import torch
    import torch.distributed as dist

    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2601_17561_gb300 import build as B
    B.build()
    if args.workload == "batching":
        return run_batching(args, dev)
    if args.workload == "serving":
        return run_serving(args, dev)
    if args.workload == "p2":
        return run_p2(args, dev)
    if args.workload == "slots":
        return run_slots(args, dev)
    from paper_2601_17561_gb300 import engine as E
    from paper_2601_17561_gb300 import icm as C
    from paper_2601_17561_gb300 import shard

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- setup (untimed): resident encrypted database shard and the query ciphertext
    W, Wq = shard.shard_workload(rank, N_EYES, N_DB, seed=2)
    eng = E.Engine(**E.PAPER).keygen()
    db = eng.encrypt_db(W.db_codes, W.db_masks, chunk_id=shard.chunk_id(rank))
    ct = eng.encrypt_query(Wq.q_codes, Wq.q_masks, Wq.eye_ids)
    torch.cuda.synchronize()
    st = torch.cuda.Stream(device=dev)
    comps = N_EYES * N_DB

    # kernel variant of the CRT forms: autotuned on this workload (untimed) or fixed
    tune = None
    if args.form in ("i8_crt", "f16_crt"):
        if args.variant == "auto":
            qt = eng.prepare(ct, N_EYES, args.form)
            best, ms = eng.autotune([db], qt)
            tune = {"chosen": best, "ms": {name: t for name, t in zip(C.VARIANTS.values(), ms) if t > 0}}
            del qt
        else:
            C.icm_ctx_set_variant(eng.ctx, int(args.variant))
            tune = {"chosen": int(args.variant)}

    def timed_form(form: str, steps: int, warmup: int):
        """warmup (>= 1) untimed steps, barrier, then `steps` steps timed with CUDA events on the
        launching stream; also the per-launch time of the CCMM kernel."""
        f = C.FORMS[form]
        op = E._u8(C.icm_query_op_bytes(eng.ctx, N_EYES, f), dev)
        sc = E._u8(eng.scores_bytes(db, N_EYES, False), dev)
        fo = E._u8(eng.scores_bytes(db, N_EYES, True), dev)
        mw = eng.match_workspace(db, N_EYES, form)
        evs = []
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            if warmup == 0:
                st.synchronize()
                barrier()
                t_start.record(st)
            for i in range(warmup + steps):
                if i == warmup and warmup > 0:
                    st.synchronize()
                    barrier()
                    t_start.record(st)
                e1, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                q = eng.prepare(ct, N_EYES, f, stream=st, out=op)
                e1.record(st)
                s = eng.match(db, q, stream=st, out=sc, ws=mw)
                e2.record(st)
                eng.fold(s, stream=st, out=fo)
                if i >= warmup:
                    evs.append((e1, e2))
            t_end.record(st)
        st.synchronize()
        total_ms = t_start.elapsed_time(t_end)
        gemm_ms = [a.elapsed_time(b) for a, b in evs]
        del op, sc, fo, mw
        return total_ms, gemm_ms

    # ---- headline: K timed steps of the chosen form
    clocks = Clocks(local)
    total_ms, gemm_ms = timed_form(args.form, args.steps, max(args.warmup, 1))
    clk = clocks.stop()
    barrier()
    ms_per_step = shard.job_time_ms(total_ms, dist if ws > 1 else None, dev) / args.steps
    value = shard.job_rate(ws, comps, ms_per_step)

    # ---- end to end through the C ABI with host buffers, right after the headline steps (the
    # same conditions: before the long compared forms heat the GPU)
    f = C.FORMS[args.form]
    ct_bytes = C.icm_query_ct_bytes(eng.ctx, N_EYES)
    fo_bytes = eng.scores_bytes(db, N_EYES, True)
    h_ct = torch.empty(ct_bytes, dtype=torch.uint8, pin_memory=True)
    h_ct.copy_(ct[:ct_bytes].cpu())
    h_fo = torch.empty(fo_bytes, dtype=torch.uint8, pin_memory=True)
    wsb = C.icm_match_host_workspace_bytes(eng.ctx, db.handle, N_EYES, f)
    wsbuf = E._u8(wsb, dev)
    with torch.cuda.stream(st):
        C.icm_match_host(eng.ctx, db.handle, h_ct, N_EYES, f, h_fo, wsbuf, wsb, stream=st)
        st.synchronize()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(args.e2e_steps):
            C.icm_match_host(eng.ctx, db.handle, h_ct, N_EYES, f, h_fo, wsbuf, wsb, stream=st)
        b.record(st)
        st.synchronize()
    e2e_ms = a.elapsed_time(b) / args.e2e_steps
    te = shard.job_time_ms(e2e_ms, dist if ws > 1 else None, dev)
    e2e = {"value": shard.job_rate(ws, comps, te), "unit": UNIT, "h2d_bytes_per_step": ct_bytes,
           "d2h_bytes_per_step": fo_bytes, "ms_per_step": te}
    del wsbuf

    # ---- roofline of the dominant kernel (the CCMM product)
    M, K, L, n_cols = db.m_rows, eng.K, eng.L, N_EYES * 31
    peaks = measured_peaks()

    def form_roofline(form: str, gemm_avg_s: float, variant):
        """Roofline of the CCMM kernel of `form` from its CUDA-event time per launch."""
        tc = form == "f16_crt" and variant in (1, 2, 3)
        if form == "u64":
            ops = 4.0 * M * n_cols * K * L                 # IMAD.WIDE per launch (2 x 2 30-bit limb products)
            sm_max = peaks.get("sm_max_mhz", 2070.0)
            peak = 152 * 32 * sm_max * 1e6                  # 152 SMs x 32 IMAD.WIDE/clk x max SM clock
            roof = {"bound": "alu", "achieved": ops / gemm_avg_s / 1e9, "peak": peak / 1e9, "unit": "Gop/s",
                    "peak_source": "derived: 152 SMs x 32 IMAD.WIDE per clock x max SM clock",
                    "imad_wide_probe_gops": C.icm_probe_peak(0) / 1e9}
        else:
            kp = (K + 31) // 32 * 32
            # products per modular MAC: 64 digit pairs, or one per CRT modulus
            pairs = 64 if form == "i8_digits" else len(C.icm_ctx_crt_moduli(eng.ctx))
            ops = 2.0 * pairs * M * n_cols * kp * L
            if form == "f16_crt":
                # fp16 and bf16 share the dense tensor rate; the CCMM launch runs for seconds, so
                # the sustained (power-capped) figure is the denominator
                peak = peaks.get("bf16_tflops_sustained")
                src = "of measured: MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS, seconds-long loop); fp16 rate = bf16"
                if peak is None:
                    peak, src = 1700.0, "of fallback: 1.7 PFLOP/s bf16 sustained"
                roof = {"bound": "tensor", "achieved": ops / gemm_avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "peak_source": src, "mma_sync_fp16_probe_tflops": 2.0 * C.icm_probe_peak(2) / 1e12}
            else:
                peak = 2.0 * C.icm_probe_peak(1)
                roof = {"bound": "tensor", "achieved": ops / gemm_avg_s / 1e12, "peak": peak / 1e12, "unit": "TOP/s",
                        "peak_source": "measured in this run: int8 mma.sync.m16n8k32 issue-bound probe "
                                       "(no tcgen05 int8 on sm_103a)"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["traffic"] = NCU_TRAFFIC.get((form, variant if tc else 0))
        if roof["traffic"] is not None:
            roof["traffic_note"] = ("DRAM bytes per CCMM call: one-pass ncu capture on the 8,192-row slice of "
                                    "this shape, scaled x64 (profiles/)")
        roof["kernel"] = {"u64": "k_ppmm_u64", "i8_digits": "k_ppmm_digits", "i8_crt": "k_crt_p1<int8> + k_crt_combine",
                          "f16_crt": f"k_crt_tc ({C.VARIANTS[variant]}) + k_crt_combine" if tc
                          else "k_crt_p1<fp16> + k_crt_combine"}.get(form)
        roof["ms_per_launch"] = gemm_avg_s * 1e3
        return roof

    roof = form_roofline(args.form, statistics.mean(gemm_ms) / 1e3, tune["chosen"] if tune else None)

    # ---- rescaling by Q' of the step's CCMM result (not part of the timed step): HBM-bound, reads
    # L words and writes L_q words per coefficient
    rs, decode = None, None
    if eng.L > eng.Lq:
        with torch.cuda.stream(st):
            q1 = eng.prepare(ct, N_EYES, C.FORMS[args.form], stream=st)
            s1 = eng.match(db, q1, stream=st)
            out = E._u8(C.icm_rescale_bytes(s1.handle), dev)
            eng.rescale(s1, stream=st, out=out)                         # warm-up
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5
            a.record(st)
            for _ in range(reps):
                eng.rescale(s1, stream=st, out=out)
            b.record(st)
            st.synchronize()
        rms = a.elapsed_time(b) / reps
        rbytes = (L + eng.Lq) * n_cols * M * 8
        rpeak = peaks.get("hbm_gbs", 6800.0)
        rs = {"kernel": "k_rescale", "ms_per_launch": rms, "bytes": rbytes, "achieved_gbs": rbytes / (rms / 1e3) / 1e9,
              "peak_gbs": rpeak, "frac": rbytes / (rms / 1e3) / 1e9 / rpeak,
              "peak_source": "of measured: MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "of fallback: 6.8 TB/s"}
        # decoded-score error of that CCMM result: the decoder's largest pre-rounding distance
        # |x - round(x)| (numerator units), and the same in fractional-HD units over a lower bound
        # of every pair's mask overlap ||m_q & m_db|| >= |m_q| + |m_db| - code bits (any rotation)
        import numpy as np
        dec1, err1 = eng.decrypt(s1, stream=st, with_error=True)
        st.synchronize()
        e_num = float(err1.cpu()[0])
        wq = np.unpackbits(Wq.q_masks, axis=1).sum(axis=1)
        wd = np.unpackbits(W.db_masks, axis=1).sum(axis=1)
        den_lb = max(1, int(wq.min()) + int(wd.min()) - W.db_masks.shape[1] * 8)
        decode = {"pre_rounding_max": e_num, "unit": "numerator units (decrypted / (Q' Delta))",
                  "pre_rounding_max_hd": e_num / (2.0 * den_lb), "mask_overlap_lower_bound": den_lb,
                  "hd_error_max": 0.0 if e_num < 0.5 else None, "hd_tolerance": 2.0 ** -10,
                  "note": "numerators round exactly while pre_rounding_max < 1/2, so decoded distances equal "
                          "the FP64 cleartext distances (all pairs checked against the oracle in "
                          "tests/test_gpu_paper_scale.py); the bound includes the decoder's fixed-point error"}
        del q1, s1, out, dec1, err1

    # ---- cleartext folding-polynomial check (not part of the timed step): the paper's 1e12-trial
    # experiment, scaled down; one trial draws 31 scores (8 Philox4x64-10 blocks)
    fd = None
    if args.fold_trials > 0:
        from paper_2601_17561_gb300 import folding as FD
        # weak scaling: every rank runs fold_trials trials of one run, its own consecutive range
        t0, n_local = shard.trial_range(rank, ws, ws * args.fold_trials)
        with torch.cuda.stream(st):
            r = FD.fold_mc(1 << 26, seed=1, stream=st)                   # warm-up
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            FD.fold_mc(n_local, seed=2, trial0=t0, out=r, stream=st)
            b.record(st)
            st.synchronize()
        fms = shard.job_time_ms(a.elapsed_time(b), dist, dev)
        rate = ws * args.fold_trials / (fms / 1e3)
        imadw = 8 * 10 * 2 * 4                                           # 32x32->64 partial products per trial
        ipeak = C.icm_probe_peak(0)
        fd = {"kernel": "k_fold_mc<7>", "trials": ws * args.fold_trials, "ms": fms, "trials_per_s": rate,
              "counts": [int(x) for x in shard.job_sum(r.counts, dist).cpu()], "k": FD.FOLD_K, "n_f": FD.N_F,
              "p_f": FD.P_F, "law": FD.NEG_LAW, "positive_interval": (0.3, 0.45),
              "roofline": {"bound": "alu", "achieved": imadw * rate / ws / 1e9, "peak": ipeak / 1e9, "unit": "Gop/s",
                           "frac": imadw * rate / ws / ipeak,
                           "peak_source": "measured in this run: IMAD.WIDE issue-bound probe (icm_probe_peak 0)",
                           "ops": "Philox 64x64->128 products as 4 IMAD.WIDE each, 640 per trial"}}
        del r

    # ---- other forms on the same workload: warm-up step(s), then timed steps, each with the
    # roofline of its own CCMM kernel
    forms = {args.form: {"value": value, "ms_per_step": ms_per_step, "steps": args.steps,
                         "roofline_frac": roof["frac"]}}
    for other in [x for x in args.compare_forms.split(",") if x and x != args.form]:
        tot, gm = timed_form(other, args.form_steps, max(args.form_warmup, 1))
        fms = shard.job_time_ms(tot, dist if ws > 1 else None, dev) / args.form_steps
        forms[other] = {"value": shard.job_rate(ws, comps, fms), "ms_per_step": fms, "gemm_ms": statistics.mean(gm),
                        "steps": args.form_steps, "warmup": max(args.form_warmup, 1),
                        "roofline": form_roofline(other, statistics.mean(gm) / 1e3, None)}


    # kernels per step: query basis extension (+ residue planes), the product's launches as the
    # library reports them (CRT forms: a product and a recombination launch per column round and
    # limb group), fold
    launches_per_step = 1 + (1 if args.form != "u64" else 0) + \
        C.icm_match_launches(eng.ctx, db.handle, N_EYES, C.FORMS[args.form]) + 1
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 1), "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.form], "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": args.form, "database_gb": round(db.buf.numel() / 1e9, 1),
                       "l2": "inputs larger than L2 (206 GB resident database), no flush",
                       "parallelism": "replicas" if ws == 1 else f"weak: {ws} database shards, same query"},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "clocks": clk,
            "forms": forms, "variant": tune, "rescale": rs, "decode": decode, "fold_design": fd}

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, thr, sample, _ = oracle_sample(seconds_target=15.0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
