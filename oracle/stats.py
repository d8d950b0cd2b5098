"""CPU oracle of the paper's frame statistics (Sec. III, and NPCR/UACI of Sec. IV-B) -- TEST INFRASTRUCTURE.

Only ``tests/`` and the CPU-baseline leg of ``bench.py`` may use this module;
the product library never calls it and shares no code with it.  Every
function follows its equation literally in binary64 (numpy), per channel of
an H x W x C uint8 frame, with the sums written the way the paper writes
them; random block and pair positions are inputs (the caller draws them).
All functions are pinned by ``tests/test_oracle_stats.py`` against closed
forms and the statistics of uniform random frames.
"""
from __future__ import annotations

import numpy as np


def histogram(frame, c: int) -> np.ndarray:
    """Sec. III-A: z_i = number of pixels of channel c with intensity i, i = 0..255."""
    F = np.asarray(frame, dtype=np.uint8)
    return np.bincount(F[:, :, c].reshape(-1), minlength=256).astype(np.int64)


def histogram_variance(z) -> float:
    """Sec. III-A, Eq. (4): var(Z) = 1/256^2 sum_i sum_j 1/2 (z_i - z_j)^2."""
    z = np.asarray(z, dtype=np.float64)
    total = 0.0
    for i in range(256):
        d = z[i] - z
        total += float(np.sum(0.5 * d * d))
    return total / (256.0 * 256.0)


def chi_square(z) -> float:
    """Sec. III-A, Eq. (5): chi^2 = sum_i (z_i - N/256)^2 / (N/256), N the pixel count of the channel."""
    z = np.asarray(z, dtype=np.float64)
    N = float(np.sum(z))
    e = N / 256.0
    return float(np.sum((z - e) ** 2 / e))


def entropy(z) -> float:
    """Sec. III-C, Eq. (10): H(m) = sum_i p(m_i) log2(1/p(m_i)) over the 256 intensity levels
    (log base 2: a uniform 256-level source has entropy 8, as the paper states)."""
    z = np.asarray(z, dtype=np.float64)
    N = float(np.sum(z))
    H = 0.0
    for zi in z:
        if zi > 0:
            p = zi / N
            H += p * np.log2(1.0 / p)
    return float(H)


def local_entropy(frame, c: int, blocks, bs: int) -> float:
    """Sec. III-C, Eq. (11): mean of the information entropies of k non-overlapping bs x bs blocks; blocks[k] =
    (row, column) of a block's top-left pixel (the paper draws k = 30 blocks of 44 x 44 at random)."""
    F = np.asarray(frame, dtype=np.uint8)
    blocks = np.asarray(blocks).reshape(-1, 2)
    total = 0.0
    for (r, q) in blocks:
        blk = F[r:r + bs, q:q + bs, c:c + 1]
        total += entropy(histogram(blk, 0))
    return total / len(blocks)


DIRECTIONS = {"horizontal": (0, 1), "vertical": (1, 0), "diagonal": (1, 1)}


def correlation(frame, c: int, pairs, direction: str) -> float:
    """Sec. III-B, Eqs. (6)-(9): r = cov(x, y) / sqrt(D(x) D(y)) with E, D, cov normalised by the number of
    pairs; pair k is x = F[i, j, c], y = the adjacent pixel in `direction`; pairs[k] = (i, j)."""
    F = np.asarray(frame, dtype=np.uint8)
    di, dj = DIRECTIONS[direction]
    pairs = np.asarray(pairs).reshape(-1, 2)
    x = np.array([float(F[i, j, c]) for i, j in pairs])
    y = np.array([float(F[i + di, j + dj, c]) for i, j in pairs])
    N = float(len(pairs))
    Ex = np.sum(x) / N
    Ey = np.sum(y) / N
    cov = np.sum((x - Ex) * (y - Ey)) / N
    Dx = np.sum((x - Ex) ** 2) / N
    Dy = np.sum((y - Ey) ** 2) / N
    return float(cov / np.sqrt(Dx * Dy))


def npcr_uaci(a, b, c: int):
    """Sec. IV-B, Eqs. (14)-(15): NPCR = 100 sum D(i,j) / (w h), D(i,j) = 1 where the two frames differ;
    UACI = 100 sum |a - b| / (w h 255); channel c."""
    A = np.asarray(a, dtype=np.uint8)[:, :, c].astype(np.int64)
    B = np.asarray(b, dtype=np.uint8)[:, :, c].astype(np.int64)
    wh = A.size
    changed = int(np.count_nonzero(A != B))
    absdiff = int(np.sum(np.abs(A - B)))
    return 100.0 * changed / wh, 100.0 * absdiff / (wh * 255.0)
