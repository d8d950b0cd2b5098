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


def _tree(frame_bytes: bytes, n: int) -> bytes:
    N = len(frame_bytes)
    cat = b"".join(hashlib.sha256(frame_bytes[(N * i) // n:(N * (i + 1)) // n]).digest() for i in range(n))
    return hashlib.sha256(cat).digest()


@pytest.mark.parametrize("shape,n", [((1, 1, 1), 1), ((1, 1, 1), 32), ((3, 5, 3), 4), ((17, 23, 3), 32),
                                     ((64, 64, 3), 6), ((37, 41, 1), 12), ((2, 3, 4), 7), ((45, 64, 3), 3)])
def test_tree_digest_is_hash_of_concatenated_subframe_hashes(shape, n):
    """Tree mode (an option of this implementation): SHA-256 over the n sub-frame digests in order, pinned
    to hashlib with the partition recomputed in Python integers; n = 3 makes 96 bytes (a half block)."""
    f = si.uniform_frame(*shape, seed=3 * sum(shape) + n)
    assert oracle.frame_digest(f, n, "tree") == _tree(f.tobytes(), n)


def test_tree_digest_n1_is_double_sha256():
    f = si.gradient_frame(48, 64, 3, t=5, seed=2)
    assert oracle.frame_digest(f, 1, "tree") == hashlib.sha256(hashlib.sha256(f.tobytes()).digest()).digest()


def test_tree_digest_has_no_cancellation_and_sees_the_order():
    # The flat frame of the quirk above: the fold gives zero, the tree digest does not; swapping two
    # different sub-frames leaves the fold unchanged but changes the tree digest.
    f = np.full((16, 16, 3), 77, np.uint8)
    assert oracle.frame_digest(f, 8, "tree") == _tree(f.tobytes(), 8) != bytes(32)
    g = si.uniform_frame(8, 8, 3, seed=4)
    half = g.size // 2
    sw = np.concatenate([g.reshape(-1)[half:], g.reshape(-1)[:half]]).reshape(g.shape)
    assert oracle.frame_digest(sw, 2) == oracle.frame_digest(g, 2)
    assert oracle.frame_digest(sw, 2, "tree") != oracle.frame_digest(g, 2, "tree")


def test_stream_digest_mode_only_changes_the_digest_path():
    """A stream in tree mode encrypts exactly like the paper's path run with the tree digest as H: the
    digest mode selects how H is computed, nothing else."""
    key = si.key(31)
    F = si.gradient_frame(24, 40, 3, t=0, seed=31)
    E_tree, H_tree = oracle.Stream.from_key(key, digest_mode="tree").encrypt(F)
    assert H_tree == oracle.frame_digest(F, oracle.DEFAULT_N, "tree")
    ref = oracle.Stream.from_key(key)
    D, B = ref.frame_keystream(H_tree, *F.shape)
    assert np.array_equal(E_tree, oracle.permute_encrypt(F, D, B))
    assert np.array_equal(oracle.Stream.from_key(key).decrypt(E_tree, H_tree), F)
