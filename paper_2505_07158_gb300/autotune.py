"""Autotuner for the strip width of the fused permutation kernels.

The column pass of the confusion + XOR gives each CTA a full-height strip of
P pixel columns held in shared memory.  Wide strips amortise the per-row gather
overhead; narrow strips let two or more CTAs share an SM and hide memory
latency.  The best P depends on the frame shape, so it is measured: for each
(height, width, channels) every power-of-two P whose strip fits shared memory
is timed (encrypt + decrypt per frame of a batch of up to 30 frames, CUDA
events, median of several runs), the fastest is installed in the library with ``fhd_set_strip_width``
and remembered in a JSON cache keyed by the GPU name.

The chosen P only changes the schedule: outputs are bit-identical for every P
(the GPU tests check this)."""
from __future__ import annotations

import json
import os
import statistics

import torch

from . import _lib

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
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


def time_shape(h: int, w: int, C: int, P: int, reps: int = 3, frames: int = 8) -> float:
    """Milliseconds per frame of the batched encrypt + decrypt permutation launches at strip width P.

    The frames go through encrypt_frames / decrypt_frames exactly as in
    production; only the permutation launches are timed (CUDA events the
    library records on the launch stream).  A large worker count keeps the
    chaotic chains short: the permutation kernels do not depend on it."""
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
            raise RuntimeError(f"strip width {P} failed the round trip for {h}x{w}x{C}")
        return statistics.median(ts)
    finally:
        _lib.fhd_set_strip_width(h, w, C, 0)
        enc.close()
        dec.close()


def batch_frames(h: int, w: int, C: int) -> int:
    """Frames per timed batch: a 30-frame clip where it fits in about 1.5 GB, so that the wave count per
    launch, which decides the best strip width, is the one of a clip's launch (timing 8 frames picked 64 at
    1080p, where 16 is the fastest for 30 frames)."""
    return max(4, min(30, int(1.5e9 // (h * w * C))))


def tune_shape(h: int, w: int, C: int, reps: int = 7) -> tuple[int, dict]:
    n = batch_frames(h, w, C)
    times = {P: time_shape(h, w, C, P, reps, frames=n) for P in candidates(h, w, C)}
    best = min(times, key=times.get)
    return best, times


def tune(shapes, cache_path: str = DEFAULT_CACHE, force: bool = False) -> dict:
    """Tune (or fetch from the cache) every shape and install the choices."""
    cache = load_cache(cache_path)
    gpu = _gpu_name()
    table = cache.setdefault(gpu, {})
    changed = False
    for (h, w, C) in shapes:
        k = _key(h, w, C)
        if force or k not in table:
            best, times = tune_shape(h, w, C)
            table[k] = {"P": best, "ms": {str(p): t for p, t in times.items()}}
            changed = True
        _lib.fhd_set_strip_width(h, w, C, table[k]["P"])
    if changed:
        save_cache(cache, cache_path)
    return {k: v["P"] for k, v in table.items()}


def apply_cache(cache_path: str = DEFAULT_CACHE):
    """Install every cached choice for this GPU (no timing)."""
    table = load_cache(cache_path).get(_gpu_name(), {})
    for k, v in table.items():
        h, w, C = (int(x) for x in k.split("x"))
        _lib.fhd_set_strip_width(h, w, C, v["P"])
    return table
