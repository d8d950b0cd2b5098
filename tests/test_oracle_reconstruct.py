"""Pins for key expansion and the initial-condition reconstruction (Sec. II-A, Fig. 1a).

Hand-derived worked examples live in ``golden/reconstruct_worked_examples.txt``;
properties below follow from the definition (integer part from the two low
bytes mod u, a 48-bit fraction XORed with six digest bytes)."""
import math
import os
import struct

import numpy as np
import pytest

import oracle
import synth_inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "reconstruct_worked_examples.txt")


def _examples():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v, hb, u, want = line.split()[:4]
        out.append((float(v), bytes.fromhex(hb), int(u), float.fromhex(want)))
    return out


@pytest.mark.parametrize("v,hb,u,want", _examples())
def test_worked_examples(v, hb, u, want):
    got = oracle.reconstruct(v, hb, u)
    assert got == want, (got.hex(), want.hex())


def test_identity_when_digest_is_zero():
    g = si.rng(5)
    for _ in range(500):
        u = int(g.integers(1, 65536))
        ip = int(g.integers(0, u))
        frac = int(g.integers(0, 1 << 48)) * 2.0 ** -48
        if ip >= 32:  # keep int + frac exactly representable (<= 53 bits)
            frac = math.floor(frac * 2 ** 20) * 2.0 ** -20
        v = ip + frac
        assert oracle.reconstruct(v, bytes(8), u) == v


def test_integer_and_fraction_fields():
    g = si.rng(6)
    for _ in range(2000):
        u = int(g.integers(1, 32))          # int' < 32: v' = int' + frac' is exact
        v = float(g.uniform(-1e4, 1e4))
        hb = g.integers(0, 256, size=8, dtype=np.uint8).tobytes()
        got = oracle.reconstruct(v, hb, u)
        a = abs(v)
        I = int(a)
        F48 = int((a - I) * 2 ** 48)
        ip = ((I & 0xFFFF) ^ (hb[0] | hb[1] << 8)) % u
        fr = F48 ^ int.from_bytes(hb[2:8], "little")
        assert 0.0 <= got < u
        assert math.floor(got) == ip
        assert (got - ip) * 2 ** 48 == fr


def test_nonfinite_and_huge_inputs_map_to_digest_only():
    hb = bytes([5, 0, 0, 0, 0, 0, 0, 0x40])
    for v in (float("nan"), float("inf"), 2.0 ** 60):
        assert oracle.reconstruct(v, hb, 20) == 5.0 + 0.25


def test_key_to_ic_hand_examples():
    ic = oracle.key_to_ic(bytes(32))
    assert ic == (0.0, 0.0, 0.0, 0.0, -1.52)
    k = bytearray(32)
    k[7] = 0x80            # k0 = 2^63 -> (k0 >> 11) * 2^-53 = 1/2
    ic = oracle.key_to_ic(bytes(k))
    assert ic[0] == 10.0 and ic[1:4] == (0.0, 0.0, 0.0)
    assert ic[4] == -1.52 + 0.73     # 1.46 * 1/2 is exact halving
    k[8 + 7] = 0x80        # k1 = 2^63 too: the gamma XOR cancels
    ic = oracle.key_to_ic(bytes(k))
    assert ic[:2] == (10.0, 10.0) and ic[4] == -1.52


def test_key_to_ic_ranges():
    for s in range(300):
        x, y, z, w, gamma = oracle.key_to_ic(si.key(s))
        assert 0 <= x < 20 and 0 <= y < 20 and 0 <= z < 40 and 0 <= w < 20
        assert -1.52 <= gamma <= -0.06


def test_master_reconstructs_then_iterates():
    # Algorithm 1: IR[0] is one RK4 step from the reconstructed ICs; IR[t] one
    # step from IR[t-1]; the new chaining state is the last iterate.
    H = si.rng(8).integers(0, 256, size=32, dtype=np.uint8).tobytes()
    v = (3.5, 11.25, 30.0, 7.0)
    gamma = -1.0
    IR, ns = oracle.master(v, H, gamma, n=5)
    s0 = [oracle.reconstruct(v[m], H[8 * m: 8 * m + 8], (20, 20, 40, 20)[m]) for m in range(4)]
    assert np.array_equal(IR[0], oracle.rk4_step(s0, gamma))
    for t in range(1, 10):
        assert np.array_equal(IR[t], oracle.rk4_step(IR[t - 1], gamma))
    assert np.array_equal(ns, IR[-1])
