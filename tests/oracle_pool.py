"""The CPU oracle on every host core, for GPU parity tests at full frame sizes.

A spawn-context process pool (never fork: the parent holds a CUDA context) runs one video stream per task.
Tasks name their inputs by recipe (shape, frame index, seed), so frames are generated in the worker by the
same seeded generator the GPU side used, and only the results travel back: the digest of every frame, a
SHA-256 (hashlib) of every ciphertext, and the full ciphertext of the frames asked for."""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import multiprocessing as mp
import os

_POOL = None


def pool() -> cf.ProcessPoolExecutor:
    global _POOL
    if _POOL is None:
        _POOL = cf.ProcessPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)),
                                       mp_context=mp.get_context("spawn"))
    return _POOL


def _frame(recipe):
    import synth_inputs as si
    kind, shape, t, seed = recipe
    if kind == "gradient":
        return si.gradient_frame(*shape, t=t, seed=seed)
    return si.uniform_frame(*shape, seed=seed)


def stream_job(key: bytes, recipes, full: set, encrypt: set | None = None, n: int = 32):
    """Encrypt frames recipes[0], recipes[1], ... in order on one oracle stream.  Frames whose index is in
    `encrypt` (None = all) are encrypted; the others only advance the chaining state (digest + LHCS_m).
    Returns {index: (H, sha256(E) or None, E if index in full else None)}."""
    import oracle
    st = oracle.Stream.from_key(key, n=n)
    out = {}
    for q, rc in enumerate(recipes):
        F = _frame(rc)
        if encrypt is None or q in encrypt:
            E, H = st.encrypt(F)
            out[q] = (H, hashlib.sha256(E.tobytes()).digest(), E if q in full else None)
        else:
            out[q] = (st.advance(F), None, None)
    return out
