"""Convenience layer over the C ABI: PyTorch device buffers sized by the library and handles that
keep them alive.  Every computation is a libicm call; this module only allocates and marshals."""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import icm as C

# Named parameter sets.  TINY: ring degree 2^12, three primes below 2^50, Delta = 2^26.
# PAPER: N_db = 2^14, N_q = 2^13, d = 2^14 (Section 6.2.1), eight primes below 2^60.
TINY = dict(log_n_db=12, log_n_q=12, n_limbs=3, n_limbs_q=1, prime_bits=50, log2_delta=26, seed=1)
PAPER = dict(log_n_db=14, log_n_q=13, n_limbs=8, n_limbs_q=2, prime_bits=60, log2_delta=60, seed=2)


def _u8(nbytes: int, device) -> torch.Tensor:
    # 256-byte alignment comes from the caching allocator; round the size up to 16 bytes
    return torch.empty(max(16, (nbytes + 15) // 16 * 16), dtype=torch.uint8, device=device)


@dataclasses.dataclass
class Db:
    handle: object
    buf: torch.Tensor
    n_real: int
    m_rows: int
    chunk_id: int

    def __del__(self):
        if self.handle is not None:
            C.icm_db_destroy(self.handle)
            self.handle = None


@dataclasses.dataclass
class Query:
    handle: object
    buf: torch.Tensor
    n_eyes: int
    form: int

    def __del__(self):
        if self.handle is not None:
            C.icm_query_destroy(self.handle)
            self.handle = None


@dataclasses.dataclass
class Scores:
    handle: object
    buf: torch.Tensor
    shape: tuple          # (L, n_cols, M)
    n_eyes: int
    folded: bool
    db: Db

    def residues(self) -> np.ndarray:
        L, n, M = self.shape
        return self.buf[: L * n * M * 8].view(torch.int64).cpu().numpy().view(np.uint64).reshape(L, n, M)

    def __del__(self):
        if self.handle is not None:
            C.icm_scores_destroy(self.handle)
            self.handle = None


class Engine:
    """One library context (parameters, primes, secrets) on the current CUDA device."""

    def __init__(self, log_n_db, log_n_q, n_limbs, n_limbs_q, prime_bits, log2_delta, seed, rho=31, fold_k=16,
                 hamming_weight=512, noise_eta=21, d2=1 << 14, code_bits=12800, device="cuda"):
        self.device = torch.device(device)
        self.params = C.icm_params(log_n_db=log_n_db, log_n_q=log_n_q, n_limbs=n_limbs, n_limbs_q=n_limbs_q,
                                   prime_bits=prime_bits, code_bits=code_bits, d2=d2, rho=rho, fold_k=fold_k,
                                   hamming_weight=hamming_weight, log2_delta=log2_delta, noise_eta=noise_eta,
                                   seed=seed)
        self.ctx = C.icm_ctx_create(self.params)
        self.keyed = False
        self.L = n_limbs
        self.Lq = n_limbs_q
        self.rho = rho
        self.fold_k = fold_k
        self.K = d2 + (1 << log_n_q)

    def keygen(self):
        with torch.cuda.device(self.device):
            C.icm_keygen(self.ctx)
        self.keyed = True
        return self

    @property
    def primes(self):
        return C.icm_ctx_primes(self.ctx, self.L)

    def __del__(self):
        if getattr(self, "ctx", None) is not None:
            C.icm_ctx_destroy(self.ctx)
            self.ctx = None

    # -------------------------------------------------------------------- setup
    def encrypt_db(self, codes: np.ndarray, masks: np.ndarray, chunk_id: int = 0, stream=None) -> Db:
        codes = np.ascontiguousarray(codes, np.uint8)
        masks = np.ascontiguousarray(masks, np.uint8)
        n = codes.shape[0]
        nbytes, m_rows = C.icm_db_bytes(self.ctx, n)
        buf = _u8(nbytes, self.device)
        h = C.icm_db_encrypt(self.ctx, codes, masks, n, chunk_id, buf, nbytes, stream)
        return Db(h, buf, n, m_rows, chunk_id)

    def encrypt_db_slots(self, codes: np.ndarray, masks: np.ndarray, log2_scale: int = 16, chunk_id: int = 0,
                         stream=None) -> Db:
        """Slot-encoded database chunk (one template per slot, N_db/2 per block)."""
        codes = np.ascontiguousarray(codes, np.uint8)
        masks = np.ascontiguousarray(masks, np.uint8)
        n = codes.shape[0]
        nbytes, m_rows = C.icm_db_bytes_slots(self.ctx, n)
        buf = _u8(nbytes, self.device)
        h = C.icm_db_encrypt_slots(self.ctx, codes, masks, n, log2_scale, chunk_id, buf, nbytes, stream)
        return Db(h, buf, n, m_rows, chunk_id)

    def encrypt_query(self, codes: np.ndarray, masks: np.ndarray, eye_ids, stream=None) -> torch.Tensor:
        codes = np.ascontiguousarray(codes, np.uint8)
        masks = np.ascontiguousarray(masks, np.uint8)
        ids = np.ascontiguousarray(np.asarray(eye_ids, np.uint64))
        n = codes.shape[0]
        nbytes = C.icm_query_ct_bytes(self.ctx, n)
        buf = _u8(nbytes, self.device)
        C.icm_query_encrypt(self.ctx, codes, masks, ids, n, buf, nbytes, stream)
        return buf

    # -------------------------------------------------------------------- hot path
    def prepare(self, ct: torch.Tensor, n_eyes: int, form="u64", stream=None, out: torch.Tensor = None) -> Query:
        f = C.FORMS[form] if isinstance(form, str) else form
        nbytes = C.icm_query_op_bytes(self.ctx, n_eyes, f)
        buf = out if out is not None else _u8(nbytes, self.device)
        h = C.icm_query_prepare(self.ctx, ct, n_eyes, f, buf, nbytes, stream)
        return Query(h, buf, n_eyes, f)

    def scores_bytes(self, db: Db, n_eyes: int, folded: bool) -> int:
        return C.icm_scores_bytes(self.ctx, db.handle, n_eyes, folded)

    def match_workspace(self, db: Db, n_eyes: int, form) -> torch.Tensor:
        f = C.FORMS[form] if isinstance(form, str) else form
        n = C.icm_match_workspace_bytes(self.ctx, db.handle, n_eyes, f)
        return _u8(n, self.device) if n else None

    def match(self, db: Db, q: Query, stream=None, out: torch.Tensor = None, ws: torch.Tensor = None) -> Scores:
        nbytes = C.icm_scores_bytes(self.ctx, db.handle, q.n_eyes, 0)
        buf = out if out is not None else _u8(nbytes, self.device)
        wsb = C.icm_match_workspace_bytes(self.ctx, db.handle, q.n_eyes, q.form)
        if wsb and ws is None:
            ws = _u8(wsb, self.device)
        h = C.icm_match(self.ctx, db.handle, q.handle, buf, nbytes, ws, wsb, stream)
        return Scores(h, buf, C.icm_scores_shape(h), q.n_eyes, False, db)

    def fold(self, s: Scores, stream=None, out: torch.Tensor = None) -> Scores:
        nbytes = C.icm_scores_bytes(self.ctx, s.db.handle, s.n_eyes, 1)
        buf = out if out is not None else _u8(nbytes, self.device)
        h = C.icm_fold(self.ctx, s.handle, buf, nbytes, stream)
        return Scores(h, buf, C.icm_scores_shape(h), s.n_eyes, True, s.db)

    def rescale(self, s: Scores, stream=None, out: torch.Tensor = None) -> Scores:
        """Scores at modulus Q_db -> scores at the query modulus Q (L_q limbs, scale Delta)."""
        nbytes = C.icm_rescale_bytes(s.handle)
        buf = out if out is not None else _u8(nbytes, self.device)
        h = C.icm_rescale(self.ctx, s.handle, buf, nbytes, stream)
        return Scores(h, buf, C.icm_scores_shape(h), s.n_eyes, s.folded, s.db)

    def normalize(self, s: Scores, q_masks: torch.Tensor, db_masks: torch.Tensor, log2_scale_mu: int = 36,
                  stream=None, out: torch.Tensor = None, ws: torch.Tensor = None) -> torch.Tensor:
        """ct (.) mu of every block of rescaled slot-encoded scores; q_masks / db_masks: device
        uint8 packed masks.  Returns the [L_q][n_cols][n_blocks][2][N_db] residues (bytes)."""
        ob, wb = C.icm_normalize_bytes(s.handle)
        out = out if out is not None else _u8(ob, self.device)
        ws = ws if ws is not None else _u8(wb, self.device)
        C.icm_normalize(self.ctx, s.handle, q_masks, db_masks, log2_scale_mu, out, ob, ws, wb, stream)
        return out

    def decrypt_slots(self, s: Scores, norm: torch.Tensor, log2_scale_mu: int = 36, stream=None) -> torch.Tensor:
        """Decoded fractional Hamming distances [n_cols][n_db] (device fp64) of normalised blocks."""
        n = s.shape[1] * s.db.n_real
        out = torch.empty(max(n, 1), dtype=torch.float64, device=self.device)
        C.icm_decrypt_slots(self.ctx, s.handle, norm, norm.numel(), log2_scale_mu, out, n, stream)
        return out[:n].view(s.shape[1], s.db.n_real)

    # -------------------------------------------------------------------- batching form
    def match_batch(self, dbs, q: Query, stream=None, outs=None, ws: torch.Tensor = None):
        """CCMM of one query batch against several database chunks in one grouped launch."""
        sizes = [C.icm_scores_bytes(self.ctx, d.handle, q.n_eyes, 0) for d in dbs]
        outs = outs if outs is not None else [_u8(n, self.device) for n in sizes]
        wsb = C.icm_match_batch_workspace_bytes(self.ctx, [d.handle for d in dbs], q.n_eyes, q.form)
        if wsb and ws is None:
            ws = _u8(wsb, self.device)
        hs = C.icm_match_batch(self.ctx, [d.handle for d in dbs], q.handle, outs, sizes, ws, wsb, stream)
        return [Scores(h, b, C.icm_scores_shape(h), q.n_eyes, False, d) for h, b, d in zip(hs, outs, dbs)]

    def autotune(self, dbs, q: Query, stream=None):
        sizes = [C.icm_scores_bytes(self.ctx, d.handle, q.n_eyes, 0) for d in dbs]
        outs = [_u8(n, self.device) for n in sizes]
        wsb = C.icm_match_batch_workspace_bytes(self.ctx, [d.handle for d in dbs], q.n_eyes, q.form)
        ws = _u8(wsb, self.device) if wsb else None
        return C.icm_autotune(self.ctx, [d.handle for d in dbs], q.handle, outs, sizes, ws, wsb, stream)

    def plan(self, dbs, n_eyes: int, form, ct: torch.Tensor, stream):
        """Capture prepare + grouped CCMM + folds on fixed buffers into a CUDA graph."""
        return Plan(self, dbs, n_eyes, form, ct, stream)

    def decrypt(self, s: Scores, stream=None, with_error: bool = False):
        """Decrypted numerators [n_cols][n_db] (device int64); with_error=True also returns the
        largest pre-rounding distance |x - round(x)| (device fp32, numerator units)."""
        n = s.shape[1] * s.db.n_real
        out = torch.empty(max(n, 1), dtype=torch.int64, device=self.device)
        if not with_error:
            C.icm_decrypt_scores(self.ctx, s.handle, out, n, stream)
            return out[:n].view(s.shape[1], s.db.n_real)
        err = torch.empty(1, dtype=torch.float32, device=self.device)
        C.icm_decrypt_scores_max_error(self.ctx, s.handle, out, n, err, stream)
        return out[:n].view(s.shape[1], s.db.n_real), err


class Plan:
    """A CUDA graph of one batch pass (query preparation, grouped CCMM, folds) on fixed buffers."""

    def __init__(self, eng: Engine, dbs, n_eyes: int, form, ct: torch.Tensor, stream):
        f = C.FORMS[form] if isinstance(form, str) else form
        self.eng, self.dbs, self.n_eyes, self.form, self.ct = eng, dbs, n_eyes, f, ct
        dev = eng.device
        self.op_bytes = C.icm_query_op_bytes(eng.ctx, n_eyes, f)
        self.op = _u8(self.op_bytes, dev)
        self.sc_bytes = [C.icm_scores_bytes(eng.ctx, d.handle, n_eyes, 0) for d in dbs]
        self.fo_bytes = [C.icm_scores_bytes(eng.ctx, d.handle, n_eyes, 1) for d in dbs]
        self.scores = [_u8(n, dev) for n in self.sc_bytes]
        self.folded = [_u8(n, dev) for n in self.fo_bytes]
        self.ws_bytes = C.icm_match_batch_workspace_bytes(eng.ctx, [d.handle for d in dbs], n_eyes, f)
        self.ws = _u8(self.ws_bytes, dev) if self.ws_bytes else None
        self.handle = C.icm_plan_create(eng.ctx, [d.handle for d in dbs], n_eyes, f, ct, self.op, self.op_bytes,
                                        self.scores, self.sc_bytes, self.folded, self.fo_bytes, self.ws, self.ws_bytes,
                                        stream)

    def launch(self, stream=None):
        C.icm_plan_launch(self.handle, stream)

    def folded_residues(self, i: int) -> np.ndarray:
        L = self.eng.L
        groups = (self.eng.rho + self.eng.fold_k - 1) // self.eng.fold_k
        M = self.dbs[i].m_rows
        n = L * self.n_eyes * groups * M
        return self.folded[i][: n * 8].view(torch.int64).cpu().numpy().view(np.uint64).reshape(L, self.n_eyes * groups, M)

    def __del__(self):
        if getattr(self, "handle", None) is not None:
            C.icm_plan_destroy(self.handle)
            self.handle = None


class Server:
    """Serving loop over resident chunks (icm_server_*): submit one eye at a time, wait per ticket."""

    def __init__(self, eng: Engine, dbs, form="f16_crt", max_eyes=32, window_us=2000, max_pending=0,
                 max_batches=0, ws_bytes=None):
        """ws_bytes: device workspace (default: icm_server_device_bytes, max_batches full batches)."""
        f = C.FORMS[form] if isinstance(form, str) else form
        self.eng, self.dbs = eng, dbs
        cfg = C.icm_server_cfg(max_eyes=max_eyes, window_us=window_us, form=f, max_pending=max_pending,
                               max_batches=max_batches)
        nbytes = C.icm_server_device_bytes(eng.ctx, [d.handle for d in dbs], cfg)
        if ws_bytes is not None:
            nbytes = ws_bytes
        self.ws = _u8(nbytes, eng.device)
        torch.cuda.synchronize()
        self.handle = C.icm_server_create(eng.ctx, [d.handle for d in dbs], cfg, self.ws, nbytes)
        self.ct_words, self.out_words = C.icm_server_eye_words(self.handle)

    def eye_cts(self, ct: torch.Tensor, n_eyes: int) -> list:
        """Split a device wire ciphertext of n_eyes eyes into per-eye host arrays [Lq][rho][K]."""
        Lq = self.ct_words // (self.eng.rho * self.eng.K)
        full = ct[: Lq * n_eyes * self.eng.rho * self.eng.K * 8].view(torch.int64).cpu().numpy().view(np.uint64)
        full = full.reshape(Lq, n_eyes, self.eng.rho, self.eng.K)
        return [np.ascontiguousarray(full[:, e]) for e in range(n_eyes)]

    def submit(self, ct_eye: np.ndarray, out: np.ndarray) -> int:
        assert ct_eye.size == self.ct_words and out.size == self.out_words
        return C.icm_server_submit(self.handle, ct_eye, out)

    def wait(self, ticket: int, timeout_ms: int = 600000) -> float:
        return C.icm_server_wait(self.handle, ticket, timeout_ms)

    def stats(self):
        return C.icm_server_stats(self.handle)

    def memory(self):
        """(pool bytes, bytes of one full batch, peak reserved bytes, peak batches in flight)"""
        return C.icm_server_memory(self.handle)

    def close(self, timeout_ms: int = 600000):
        if self.handle is not None:
            C.icm_server_destroy(self.handle, timeout_ms)
            self.handle = None

    def __del__(self):
        self.close()


def ppmm(form, q, A: torch.Tensor, B: torch.Tensor, stream=None) -> torch.Tensor:
    """Plain modular product on device tensors (int64 views of u64 residues):
    A [L][M][K], B [L][N][K] -> C [L][N][M]."""
    f = C.FORMS[form] if isinstance(form, str) else form
    L, M, K = A.shape
    N = B.shape[1]
    Cm = torch.empty((L, N, M), dtype=torch.int64, device=A.device)
    ws_bytes = C.icm_ppmm_workspace_bytes(f, L, M, N, K)
    ws = _u8(ws_bytes, A.device) if ws_bytes else None
    C.icm_ppmm(f, q, L, A, B, Cm, M, N, K, ws, ws_bytes, stream)
    return Cm
