"""Pins for the oracle's SHA-256 and sub-frame digest fold (Sec. II-A).

SHA-256 is pinned to Python's ``hashlib`` (an independent implementation of
FIPS 180-4); the fold is pinned to the XOR of ``hashlib`` digests of the byte
ranges, with the partition recomputed here in Python integers."""
import hashlib

import numpy as np
import pytest

import oracle
import synth_inputs as si


@pytest.mark.parametrize("length", list(range(0, 200)) + [255, 256, 300, 1000, 4095, 4096, 65537])
def test_sha256_matches_hashlib(length):
    msg = si.rng(length).integers(0, 256, size=length, dtype=np.uint8).tobytes()
    assert oracle.sha256(msg) == hashlib.sha256(msg).digest()


def test_sha256_padding_boundaries():
    # 55/56 bytes: last length that fits in one padding block / first that needs two.
    for n in (55, 56, 63, 64, 119, 120, 127, 128):
        msg = bytes((7 * k + 3) & 0xFF for k in range(n))
        assert oracle.sha256(msg) == hashlib.sha256(msg).digest(), n


def test_sha256_large():
    msg = si.rng(99).integers(0, 256, size=3 * 1024 * 1024 + 17, dtype=np.uint8).tobytes()
    assert oracle.sha256(msg) == hashlib.sha256(msg).digest()


def _fold(frame_bytes: bytes, n: int) -> bytes:
    N = len(frame_bytes)
    acc = bytearray(32)
    for i in range(n):
        lo, hi = (N * i) // n, (N * (i + 1)) // n
        d = hashlib.sha256(frame_bytes[lo:hi]).digest()
        acc = bytearray(a ^ b for a, b in zip(acc, d))
    return bytes(acc)


@pytest.mark.parametrize("shape,n", [((1, 1, 1), 1), ((1, 1, 1), 32), ((3, 5, 3), 4), ((17, 23, 3), 32),
                                     ((64, 64, 3), 6), ((37, 41, 1), 12), ((2, 3, 4), 7)])
def test_frame_digest_is_xor_of_subframe_hashes(shape, n):
    f = si.uniform_frame(*shape, seed=sum(shape) + n)
    assert oracle.frame_digest(f, n) == _fold(f.tobytes(), n)


def test_frame_digest_n1_is_plain_sha256():
    f = si.gradient_frame(48, 64, 3, t=2, seed=1)
    assert oracle.frame_digest(f, 1) == hashlib.sha256(f.tobytes()).digest()


def test_frame_digest_cancellation_quirk():
    # Identical sub-frames cancel in the XOR fold: a flat frame whose N bytes
    # split into an even number of equal ranges digests to zero.
    f = np.full((16, 16, 3), 77, np.uint8)
    assert oracle.frame_digest(f, 8) == bytes(32)
    assert oracle.frame_digest(f, 3) == hashlib.sha256(bytes([77]) * 256).digest()
