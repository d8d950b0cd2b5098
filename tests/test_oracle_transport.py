"""Pins of the masked digest transport (an option of this implementation: Sec. V sends the frame hashes
encrypted over the public channel without giving the mechanism).

The transmitted digest is H xor M with M = SHA-256("FHDMASK1" || LE64 bit patterns of the chaining state
x, y, z, w and of gamma) taken before the frame.  Pinned to hashlib and struct; the keystream still
derives from H, so the ciphertext equals the plain-transport one; the receiver unmasks with its own state."""
import hashlib
import struct

import numpy as np

import oracle
import synth_inputs as si


def _mask(state, gamma) -> bytes:
    return hashlib.sha256(b"FHDMASK1" + struct.pack("<5d", *[float(v) for v in state], float(gamma))).digest()


def test_mask_is_sha256_of_tag_and_state_bits():
    s = oracle.Stream.from_key(si.key(41))
    assert s.digest_mask() == _mask(s.state, s.gamma)
    s2 = oracle.Stream(( -0.0, 1e-300, 17.25, -3.5, -1.1))   # signed zero and a tiny value: raw bit patterns
    assert s2.digest_mask() == _mask((-0.0, 1e-300, 17.25, -3.5), -1.1)


def test_masked_transport_round_trip_and_ciphertext():
    key = si.key(42)
    frames = [si.gradient_frame(20, 36, 3, t=t, seed=42) for t in range(3)]
    tx, plain = oracle.Stream.from_key(key, transport="masked"), oracle.Stream.from_key(key)
    rx = oracle.Stream.from_key(key, transport="masked")
    masks = []
    for F in frames:
        M = tx.digest_mask()
        assert M == _mask(tx.state, tx.gamma)
        masks.append(M)
        E, Htx = tx.encrypt(F)
        E0, H = plain.encrypt(F)
        assert np.array_equal(E, E0)                       # the keystream comes from H, not from H xor M
        assert Htx == bytes(a ^ b for a, b in zip(H, M)) != H
        assert np.array_equal(rx.decrypt(E, Htx), F)
    assert len(set(masks)) == len(masks)                   # a fresh mask per frame: the state advances


def test_unmasked_receiver_cannot_use_the_transmitted_digest():
    key = si.key(43)
    F = si.gradient_frame(20, 36, 3, t=0, seed=43)
    E, Htx = oracle.Stream.from_key(key, transport="masked").encrypt(F)
    wrong = oracle.Stream.from_key(key).decrypt(E, Htx)
    assert np.mean(wrong != F) > 0.9
