"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no cipher arithmetic: it only draws frames, keys, bit flips
and arrival times, so that the CUDA library and the CPU oracle can be fed the
same bytes.  The paper's videos (Akiyo, Coastguard, Hall, Rhinos, Train,
Waterfall; Sec. III) are not available; these generators stand in for them
with the paper's frame shapes:

* ``uniform``: i.i.d. uniform bytes.
* ``gradient``: a smooth 2-D gradient per channel,
  ``255 * (a_c * i / h + (1 - a_c) * ((j + 2 t) mod w) / w)`` with
  ``a_c = (c + 1) / (C + 1)`` (0.25, 0.5, 0.75 for RGB), shifted 2 pixels per
  frame index ``t`` to mimic motion, plus Gaussian noise of sigma 8, rounded
  half-to-even and clipped to [0, 255].
"""
from __future__ import annotations

import numpy as np

PAPER_SIZES = {
    "vga": (480, 640),
    "sd": (480, 720),
    "720p": (720, 1280),
    "1080p": (1080, 1920),
    "4k": (2160, 3840),
    "8k": (4320, 7680),
}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_frame(h: int, w: int, C: int = 3, seed: int = 0) -> np.ndarray:
    return rng(seed).integers(0, 256, size=(h, w, C), dtype=np.uint8)


def gradient_frame(h: int, w: int, C: int = 3, t: int = 0, seed: int = 0, sigma: float = 8.0) -> np.ndarray:
    g = rng(seed * 1_000_003 + t)
    i = np.arange(h, dtype=np.float64)[:, None]
    j = np.arange(w, dtype=np.float64)[None, :]
    out = np.empty((h, w, C), np.uint8)
    for c in range(C):
        a = (c + 1) / (C + 1)
        base = 255.0 * (a * i / h + (1.0 - a) * ((j + 2 * t) % w) / w)
        noisy = base + g.normal(0.0, sigma, size=(h, w))
        out[:, :, c] = np.clip(np.rint(noisy), 0, 255).astype(np.uint8)
    return out


def clip(n_frames: int, h: int, w: int, C: int = 3, seed: int = 0) -> np.ndarray:
    """A moving gradient+noise clip, shape (n_frames, h, w, C)."""
    return np.stack([gradient_frame(h, w, C, t, seed) for t in range(n_frames)])


def key(seed: int) -> bytes:
    return rng(seed ^ 0x5EED).integers(0, 256, size=32, dtype=np.uint8).tobytes()


def bit_flip(frame: np.ndarray, seed: int):
    """Copy of ``frame`` with one seeded bit flipped; returns (copy, (i, j, c, bit))."""
    g = rng(seed ^ 0xF11F)
    h, w, C = frame.shape
    i, j, c, b = int(g.integers(h)), int(g.integers(w)), int(g.integers(C)), int(g.integers(8))
    out = frame.copy()
    out[i, j, c] ^= np.uint8(1 << b)
    return out, (i, j, c, b)


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process on [0, duration_s)."""
    g = rng(seed ^ 0xA771)
    ts, t = [], 0.0
    while True:
        t += g.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return np.asarray(ts)
        ts.append(t)
