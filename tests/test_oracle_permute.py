"""Pins for the bit-level confusion + XOR (Sec. II-C, Algos 3-7) and its inverse.

The oracle scatters bits through the paper's [8w x h] bit matrices; here an
independent formulation (numpy ``unpackbits(bitorder='little')`` + ``np.roll``
per row and per pixel column + ``packbits``) must agree, the map must be a
bijection of bit positions on tiny frames, and the special cases (D = 0,
B = 0; byte-aligned shifts) reduce to identity, plain XOR and byte rolls."""
import numpy as np
import pytest

import oracle
import synth_inputs as si


def np_encrypt(F, D, B):
    h, w, C = F.shape
    Bf = B.reshape(h, w, C)
    E = np.empty_like(F)
    for c in range(C):
        bits = np.unpackbits(F[:, :, c], axis=1, bitorder="little")
        for i in range(h):
            bits[i] = np.roll(bits[i], int(D[c * h + i]) % (8 * w))
        for j in range(w):
            bits[:, 8 * j: 8 * j + 8] = np.roll(bits[:, 8 * j: 8 * j + 8], int(D[C * h + c * w + j]) % h, axis=0)
        bits ^= np.unpackbits(Bf[:, :, c], axis=1, bitorder="little")
        E[:, :, c] = np.packbits(bits, axis=1, bitorder="little")
    return E


def _rand(h, w, C, seed):
    g = si.rng(seed)
    F = g.integers(0, 256, size=(h, w, C), dtype=np.uint8)
    D = g.integers(0, 65536, size=C * (h + w), dtype=np.uint16)
    B = g.integers(0, 256, size=h * w * C, dtype=np.uint8)
    return F, D, B


SHAPES = [(1, 1, 1), (1, 1, 3), (1, 8, 3), (8, 1, 3), (3, 5, 3), (4, 4, 1), (7, 9, 3), (16, 13, 4), (37, 53, 3), (64, 96, 3)]


@pytest.mark.parametrize("shape", SHAPES)
def test_matches_numpy_formulation(shape):
    F, D, B = _rand(*shape, seed=sum(shape))
    assert np.array_equal(oracle.permute_encrypt(F, D, B), np_encrypt(F, D, B))


@pytest.mark.parametrize("shape", SHAPES)
def test_decrypt_inverts(shape):
    F, D, B = _rand(*shape, seed=3 * sum(shape))
    E = oracle.permute_encrypt(F, D, B)
    assert np.array_equal(oracle.permute_decrypt(E, D, B), F)


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 1), (3, 2, 3), (4, 5, 2), (5, 3, 3)])
def test_bit_permutation_is_bijective(shape):
    h, w, C = shape
    _, D, _ = _rand(h, w, C, seed=11 * sum(shape))
    B0 = np.zeros(h * w * C, np.uint8)
    nbits = h * w * C * 8
    seen = set()
    for q in range(nbits):
        F = np.zeros(h * w * C, np.uint8)
        F[q // 8] = 1 << (q % 8)
        E = oracle.permute_encrypt(F.reshape(h, w, C), D, B0).reshape(-1)
        bits = np.unpackbits(E, bitorder="little")
        assert bits.sum() == 1
        p = int(np.flatnonzero(bits)[0])
        assert (p // 8) % C == (q // 8) % C   # the channel is preserved
        seen.add(p)
    assert len(seen) == nbits


def test_zero_keystream_is_identity_and_xor_only():
    F, _, B = _rand(9, 11, 3, seed=4)
    D0 = np.zeros(3 * (9 + 11), np.uint16)
    assert np.array_equal(oracle.permute_encrypt(F, D0, np.zeros_like(B)), F)
    assert np.array_equal(oracle.permute_encrypt(F, D0, B), F ^ B.reshape(F.shape))


def test_byte_aligned_shifts_are_byte_rolls():
    h, w, C = 6, 10, 3
    F, D, B = _rand(h, w, C, seed=5)
    D[: C * h] = (D[: C * h] // 8) * 8          # whole-byte horizontal shifts
    D[C * h:] = 0                               # no vertical shift
    E = oracle.permute_encrypt(F, D, np.zeros_like(B))
    for c in range(C):
        for i in range(h):
            q = (int(D[c * h + i]) % (8 * w)) // 8
            assert np.array_equal(E[i, :, c], np.roll(F[i, :, c], q))


def test_vertical_only_is_column_roll():
    h, w, C = 7, 5, 3
    F, D, B = _rand(h, w, C, seed=6)
    D[: C * h] = 0
    E = oracle.permute_encrypt(F, D, np.zeros_like(B))
    for c in range(C):
        for j in range(w):
            assert np.array_equal(E[:, j, c], np.roll(F[:, j, c], int(D[C * h + c * w + j]) % h))
