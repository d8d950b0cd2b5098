"""Whole-cipher properties of the oracle (Algorithm 1 and its inverse).

* decrypt(encrypt(x)) == x over a chained clip;
* no diffusion (Sec. VI-A item 4): one ciphertext byte flip changes at most
  two plaintext bytes, in the same row and channel;
* differential test (Sec. IV-B, Eqs. (6)-(8)): a one-bit plaintext flip gives
  NPCR/UACI near the ideal values 100*255/256 % and 100*(65535/768)/255 %
  (the expectations for independent uniform bytes), and passes the paper's
  512x512 critical values N* = 99.5893 %, U in (33.3730, 33.5541) %;
* frame chaining (Sec. VI-A): a one-bit flip in frame t changes frame t+1's
  ciphertext even though frame t+1 itself is unchanged;
* key sensitivity (Sec. IV-A): x0 + 1e-14 fails to decrypt.  Under the
  readings taken (RK4 with h = 0.01, no transient, the six low mantissa
  bytes) a 1e-14 change only reaches the low mantissa bytes within a frame, so
  about 25-85 % of the bytes come out wrong, not the 99.6 % of unrelated
  frames; a change in a high key bit gives the full 99.6 %."""
import math

import numpy as np
import pytest

import oracle
import synth_inputs as si

NPCR_IDEAL = 100.0 * 255.0 / 256.0
UACI_IDEAL = 100.0 * (65535.0 / 768.0) / 255.0


def npcr_uaci(a, b):
    a = a.astype(np.int32)
    b = b.astype(np.int32)
    npcr = [100.0 * np.mean(a[:, :, c] != b[:, :, c]) for c in range(a.shape[2])]
    uaci = [100.0 * np.mean(np.abs(a[:, :, c] - b[:, :, c])) / 255.0 for c in range(a.shape[2])]
    return npcr, uaci


def test_round_trip_chained_clip():
    key = si.key(1)
    frames = si.clip(3, 36, 52, 3, seed=1)
    enc = oracle.Stream.from_key(key, n=6)
    dec = oracle.Stream.from_key(key, n=6)
    for F in frames:
        E, H = enc.encrypt(F)
        assert not np.array_equal(E, F)
        assert H == oracle.frame_digest(F, 6)
        assert np.array_equal(dec.decrypt(E, H), F)
    assert np.array_equal(enc.state, dec.state)


def test_locality_no_diffusion():
    key = si.key(2)
    F = si.uniform_frame(24, 40, 3, seed=2)
    E, H = oracle.Stream.from_key(key, n=4).encrypt(F)
    g = si.rng(2)
    for _ in range(20):
        i, j, c = int(g.integers(24)), int(g.integers(40)), int(g.integers(3))
        E2 = E.copy()
        E2[i, j, c] ^= np.uint8(1 << int(g.integers(8)))
        P = oracle.Stream.from_key(key, n=4).decrypt(E2, H)
        diff = np.argwhere(P != F)
        assert 1 <= len(diff) <= 2
        assert len(set(diff[:, 0])) == 1 and len(set(diff[:, 2])) == 1 and diff[0, 2] == c


@pytest.mark.parametrize("size,seed", [(256, 0), (512, 1)])
def test_npcr_uaci_one_bit_flip(size, seed):
    key = si.key(seed)
    F = si.uniform_frame(size, size, 3, seed=seed)
    F2, _ = si.bit_flip(F, seed)
    E1, _ = oracle.Stream.from_key(key).encrypt(F)
    E2, _ = oracle.Stream.from_key(key).encrypt(F2)
    npcr, uaci = npcr_uaci(E1, E2)
    n = size * size
    sd_npcr = 100.0 * math.sqrt((1 / 256) * (255 / 256) / n)
    sd_uaci = 100.0 * (math.sqrt(65535 * 65537 / 18 / 65536 * (1 - 0) ) / 255.0) / math.sqrt(n)
    for v in npcr:
        assert abs(v - NPCR_IDEAL) < 6 * sd_npcr
    for v in uaci:
        assert abs(v - UACI_IDEAL) < 6 * sd_uaci
    if size == 512:
        # Paper's critical values for 512x512 frames (Sec. IV-B).
        assert min(npcr) > 99.5893 - 3 * sd_npcr
        assert all(33.3730 - 3 * sd_uaci < v < 33.5541 + 3 * sd_uaci for v in uaci)


def test_next_frame_sensitivity():
    key = si.key(3)
    f0, f1 = si.clip(2, 64, 64, 3, seed=3)
    f0b, _ = si.bit_flip(f0, 3)
    a, b = oracle.Stream.from_key(key), oracle.Stream.from_key(key)
    a.encrypt(f0)
    b.encrypt(f0b)
    e1a, _ = a.encrypt(f1)
    e1b, _ = b.encrypt(f1)
    npcr, _ = npcr_uaci(e1a, e1b)
    assert min(npcr) > 99.0


def test_key_sensitivity():
    key = si.key(4)
    F = si.gradient_frame(64, 64, 3, seed=4)
    ic = oracle.key_to_ic(key)
    E, H = oracle.Stream(ic).encrypt(F)
    assert np.array_equal(oracle.Stream(ic).decrypt(E, H), F)
    for m in range(4):
        bad = list(ic)
        bad[m] += 1e-14
        P = oracle.Stream(bad).decrypt(E, H)
        npcr, _ = npcr_uaci(P, F)
        assert min(npcr) > 20.0, (m, npcr)
    k = bytearray(key)
    k[6] ^= 0x10                      # bit 52 of k0: x0 moves by u_x * 2^-12
    P = oracle.Stream.from_key(bytes(k)).decrypt(E, H)
    npcr, _ = npcr_uaci(P, F)
    assert all(abs(v - NPCR_IDEAL) < 1.0 for v in npcr), npcr


@pytest.mark.parametrize("mode", ["xor", "tree"])
def test_chaining_step_alone_leaves_the_state_encryption_leaves(mode):
    """Stream.advance (digest + LHCS_m only) leaves the chaining state that a full encryption of the same
    frame leaves: the next frame then encrypts to the same ciphertext.  A wrong worker count, step, digest
    mode or a skipped reconstruction in advance() would change that next ciphertext."""
    key = si.key(3)
    frames = si.clip(3, 24, 40, 3, seed=4)
    full = oracle.Stream.from_key(key, n=5, digest_mode=mode)
    short = oracle.Stream.from_key(key, n=5, digest_mode=mode)
    for F in frames[:2]:
        _, H = full.encrypt(F)
        assert short.advance(F) == H
        assert np.array_equal(full.state, short.state)
    E_full, _ = full.encrypt(frames[2])
    E_short, _ = short.encrypt(frames[2])
    assert np.array_equal(E_full, E_short)
    skipped = oracle.Stream.from_key(key, n=5, digest_mode=mode)
    skipped.advance(frames[0])
    assert not np.array_equal(skipped.encrypt(frames[2])[0], E_full)


def _channel_stats(h, keys, size=512):
    from oracle import stats
    F = si.gradient_frame(size, size, 3, t=0, seed=3)
    F2, _ = si.bit_flip(F, 3)
    chi, uaci = [], []
    for key in keys:
        E = oracle.Stream.from_key(key, h=h).encrypt(F)[0]
        E2 = oracle.Stream.from_key(key, h=h).encrypt(F2)[0]
        chi.append([stats.chi_square(stats.histogram(E, c)) for c in range(3)])
        uaci.append([stats.npcr_uaci(E, E2, c)[1] for c in range(3)])
    return np.mean(chi, axis=0), np.mean(uaci, axis=0)


def test_default_step_meets_the_papers_statistics():
    """The RK4 step is a reading (the paper names no integrator): it is the one whose ciphertexts meet the
    paper's Sec. III-A chi^2 bar (< 293.25 per channel, 512x512) and Sec. IV-B UACI interval
    (33.3730 %, 33.5541 %), as the paper's own ciphertexts do.  Means over four keys of a 512x512 gradient
    frame and its one-bit flip; ideal values 255 and 33.4635 %.  With h = 0.001 the third channel's
    ciphertext is biased: consecutive iterates of the same trajectory feed each worker pair, and at that
    step the XOR of their sixth mantissa byte is far from uniform."""
    keys = [si.key(700 + k) for k in range(4)]
    chi, uaci = _channel_stats(oracle.DEFAULT_H, keys)
    assert oracle.DEFAULT_H == 0.01
    assert (chi < 293.25).all(), chi
    assert ((uaci > 33.3730) & (uaci < 33.5541)).all(), uaci
    _, uaci_small = _channel_stats(0.001, keys)
    assert uaci_small[2] < 33.3730, uaci_small
