"""Autotuner of the permutation's tile shapes and of the clip pipeline's work split.

Per frame shape (height, width, channels) it chooses, by timing:

* P, the strip width of the column pass: each CTA holds a full-height strip of P pixel columns in shared
  memory.  Wide strips amortise the per-row work; narrow ones let two or more CTAs share an SM and hide
  memory latency.  Every power-of-two P whose strip fits is timed.
* RB, the rows per CTA of the row pass (bands of whole rows staged in shared memory), at the chosen P.
* ST and RT, the threads per CTA of the column pass (256 or 512) and of the row pass (128 or 256), at the
  chosen P and RB.

Each candidate is timed as the batched encrypt + decrypt permutation launches per frame of a batch of up to
30 frames (CUDA events the library records on the launch stream, median of several runs); the fastest is
installed with ``fhd_set_strip_width`` / ``fhd_set_row_band`` / ``fhd_set_cta_threads``.  Outputs are
bit-identical for every choice (the GPU tests check this).

The clip pipeline's work split (worker warp layout, clips in flight, worker window) is tuned by
``bench.py --tune``, which times the headline under each setting and stores the best here.

Two tables, both keyed by the GPU name: ``tuned.json`` beside this file holds the choices measured on the
GPUs this library was tuned on (committed with it, so a fresh machine of the same kind starts from them),
and ``_build/autotune.json`` holds this machine's own measurements of shapes not in the first."""
from __future__ import annotations

import json
import os
import statistics

import torch

from . import _lib

HERE = os.path.dirname(os.path.abspath(__file__))
COMMITTED = os.path.join(HERE, "tuned.json")
DEFAULT_CACHE = os.path.join(HERE, "_build", "autotune.json")
SMEM_LIMIT = 232448


def candidates(h: int, w: int, C: int):
    out = []
    P = 1
    while P <= 128:
        smem = (h * P * C + 15) & ~15
        if smem <= SMEM_LIMIT and (P == 1 or P // 2 < w):
            out.append(P)
        P *= 2
    return out


def row_band_candidates(h: int, w: int, C: int):
    pitch = (w * C + 15) & ~15
    return [rb for rb in (1, 2, 4, 8, 16) if rb <= h and 2 * rb * pitch + 4 * rb * C <= SMEM_LIMIT]


def _key(h, w, C):
    return f"{h}x{w}x{C}"


def _gpu_name() -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device())


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _shapes_of(table: dict, gpu: str) -> dict:
    return table.get(gpu, {}).get("shapes", {})


def time_shape(h: int, w: int, C: int, P: int, RB: int = 0, reps: int = 3, frames: int = 8, ST: int = 0,
               RT: int = 0) -> float:
    """Milliseconds per frame of the batched encrypt + decrypt permutation launches at strip width P, row
    band RB (0: the built-in band) and threads per CTA ST, RT of the two passes (0: the defaults).

    The frames go through encrypt_frames / decrypt_frames exactly as in production; only the permutation
    launches are timed (CUDA events the library records on the launch stream).  A large worker count keeps
    the chaotic chains short: the permutation kernels do not depend on it."""
    dev = torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device=dev)
    g.manual_seed(h * 7919 + w * 31 + C)
    key = bytes(range(32))
    enc = _lib.Cipher(key, n_workers=1024)
    dec = _lib.Cipher(key, n_workers=1024)
    sid, rid = enc.open_stream(), dec.open_stream()
    F = [torch.randint(0, 256, (h, w, C), dtype=torch.uint8, device=dev, generator=g) for _ in range(frames)]
    E = [torch.empty_like(f) for f in F]
    R = [torch.empty_like(f) for f in F]
    Hd = [torch.empty(32, dtype=torch.uint8, device=dev) for _ in F]
    _lib.fhd_set_strip_width(h, w, C, P)
    _lib.fhd_set_row_band(h, w, C, RB)
    _lib.fhd_set_cta_threads(h, w, C, ST, RT)
    try:
        def once():
            enc.encrypt_frames([(sid, F[k], E[k], Hd[k]) for k in range(frames)])
            dec.decrypt_frames([(rid, E[k], R[k], Hd[k]) for k in range(frames)])
        once()
        enc.profile(True)
        dec.profile(True)
        ts = []
        for _ in range(reps):
            once()
            t = enc.profile_read()["encrypt"][0] + dec.profile_read()["decrypt"][0]
            ts.append(t / frames)
        torch.cuda.synchronize()
        if not all(torch.equal(R[k], F[k]) for k in range(frames)):
            raise RuntimeError(f"strip width {P}, row band {RB}, CTA threads {ST}/{RT} failed the round trip "
                               f"for {h}x{w}x{C}")
        return statistics.median(ts)
    finally:
        _lib.fhd_set_strip_width(h, w, C, 0)
        _lib.fhd_set_row_band(h, w, C, 0)
        _lib.fhd_set_cta_threads(h, w, C, 0, 0)
        enc.close()
        dec.close()


def batch_frames(h: int, w: int, C: int) -> int:
    """Frames per timed batch: a 30-frame clip where it fits in about 1.5 GB, so that the wave count per
    launch, which decides the best strip width, is the one of a clip's launch (timing 8 frames picked 64 at
    1080p, where 16 is the fastest for 30 frames)."""
    return max(4, min(30, int(1.5e9 // (h * w * C))))


CTA_CANDIDATES = ((512, 256), (256, 256), (512, 128))


def tune_shape(h: int, w: int, C: int, reps: int = 7) -> dict:
    """Time every strip width, then every row band at the best width, then the CTA shapes of the two passes:
    {"P", "RB", "ST", "RT", "ms", "rb_ms", "cta_ms"}."""
    n = batch_frames(h, w, C)
    times = {P: time_shape(h, w, C, P, 0, reps, frames=n) for P in candidates(h, w, C)}
    best = min(times, key=times.get)
    rb_times = {RB: time_shape(h, w, C, best, RB, reps, frames=n) for RB in row_band_candidates(h, w, C)}
    rb = min(rb_times, key=rb_times.get) if rb_times else 0
    cta_times = {(st, rt): time_shape(h, w, C, best, rb, reps, frames=n, ST=st, RT=rt) for st, rt in CTA_CANDIDATES}
    st, rt = min(cta_times, key=cta_times.get)
    return {"P": best, "RB": rb, "ST": st, "RT": rt, "ms": {str(p): t for p, t in times.items()},
            "rb_ms": {str(r): t for r, t in rb_times.items()},
            "cta_ms": {f"{a}/{b}": t for (a, b), t in cta_times.items()}}


def _install(h, w, C, entry):
    _lib.fhd_set_strip_width(h, w, C, int(entry.get("P", 0)))
    _lib.fhd_set_row_band(h, w, C, int(entry.get("RB", 0)))
    _lib.fhd_set_cta_threads(h, w, C, int(entry.get("ST", 0)), int(entry.get("RT", 0)))


def tune(shapes, cache_path: str = DEFAULT_CACHE, force: bool = False, committed: str = COMMITTED) -> dict:
    """Install the tile shapes of every shape: from the committed table for this GPU, else this machine's
    cache, else by timing (recorded in the cache).  force=True times every shape again.  Returns
    {shape key: {"P", "RB", "ST", "RT", "source"}} (0: the library's default)."""
    gpu = _gpu_name()
    fixed = {} if force else _shapes_of(load_cache(committed), gpu)
    cache = load_cache(cache_path)
    table = cache.setdefault(gpu, {}).setdefault("shapes", {})
    changed = False
    out = {}
    for (h, w, C) in shapes:
        k = _key(h, w, C)
        if k in fixed:
            entry, src = fixed[k], "committed"
        elif not force and k in table and "ST" in table[k]:
            entry, src = table[k], "cache"
        else:
            entry, src = tune_shape(h, w, C), "timed"
            table[k] = entry
            changed = True
        _install(h, w, C, entry)
        out[k] = {"P": int(entry["P"]), "RB": int(entry.get("RB", 0)), "ST": int(entry.get("ST", 0)),
                  "RT": int(entry.get("RT", 0)), "source": src}
    if changed:
        save_cache(cache, cache_path)
    return out


def apply_cache(cache_path: str = DEFAULT_CACHE, committed: str = COMMITTED) -> dict:
    """Install every recorded choice for this GPU (no timing); the committed table wins."""
    gpu = _gpu_name()
    merged = dict(_shapes_of(load_cache(cache_path), gpu))
    merged.update(_shapes_of(load_cache(committed), gpu))
    for k, v in merged.items():
        h, w, C = (int(x) for x in k.split("x"))
        _install(h, w, C, v)
    return merged


def pipeline_defaults(committed: str = COMMITTED) -> dict | None:
    """The clip pipeline's tuned work split for this GPU ({"layout", "inflight", "worker_window", ...}), if
    recorded."""
    return load_cache(committed).get(_gpu_name(), {}).get("pipeline")


def record(shapes: dict | None = None, pipeline: dict | None = None, committed: str = COMMITTED):
    """Write tuned shapes ({key: entry}) and/or the pipeline's work split into the committed table."""
    table = load_cache(committed)
    ent = table.setdefault(_gpu_name(), {})
    if shapes:
        ent.setdefault("shapes", {}).update(shapes)
    if pipeline:
        ent["pipeline"] = pipeline
    save_cache(table, committed)
