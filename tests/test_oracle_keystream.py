"""Pins for the worker data generation (Sec. II-B, Algorithm 2).

* two identically seeded systems cancel: that worker's D and B slices are 0;
* a system seeded at the origin (an equilibrium of Eq. (1)) contributes zero
  bytes, so the worker's stream is the other system's mantissa bytes alone --
  compared here with bytes taken by ``struct`` from the oracle's trajectory,
  with the slice bounds recomputed in Python integers;
* perturbing worker p's seeds changes only worker p's slices."""
import struct

import numpy as np
import pytest

import oracle
import synth_inputs as si


def _slices(L, n):
    return [((L * i) // n, (L * (i + 1)) // n) for i in range(n)]


def _ir(n, seed):
    g = si.rng(seed)
    return np.column_stack([g.uniform(0, 20, 2 * n), g.uniform(0, 20, 2 * n), g.uniform(0, 40, 2 * n), g.uniform(0, 20, 2 * n)])


@pytest.mark.parametrize("h,w,C,n", [(8, 8, 3, 4), (5, 7, 1, 3), (30, 40, 3, 32), (1, 1, 3, 2)])
def test_equal_seeds_cancel(h, w, C, n):
    IR = _ir(n, 1)
    p = n // 2
    IR[2 * p + 1] = IR[2 * p]
    D, B = oracle.keystream(IR, -1.0, h, w, C, n)
    d0, d1 = _slices(C * (h + w), n)[p]
    b0, b1 = _slices(h * w * C, n)[p]
    assert np.all(D[d0:d1] == 0) and np.all(B[b0:b1] == 0)
    others = np.concatenate([D[:d0], D[d1:]])
    if others.size > 8:
        assert np.any(others != 0)


@pytest.mark.parametrize("h,w,C,n", [(8, 8, 3, 4), (5, 7, 1, 3), (20, 31, 3, 6), (2, 3, 4, 5)])
def test_origin_partner_exposes_single_stream(h, w, C, n):
    gamma = -0.9
    IR = _ir(n, 2)
    IR[1::2] = 0.0                      # second system of every worker at the origin
    D, B = oracle.keystream(IR, gamma, h, w, C, n)
    dsl, bsl = _slices(C * (h + w), n), _slices(h * w * C, n)
    for i in range(n):
        (d0, d1), (b0, b1) = dsl[i], bsl[i]
        need = 2 * (d1 - d0) + (b1 - b0)
        steps = -(-need // 24)
        traj = oracle.rk4_trajectory(IR[2 * i], gamma, steps)
        S = bytearray()
        for t in range(steps):
            for m in range(4):
                S += struct.pack("<d", traj[t, m])[:6]
        exp_D = [S[2 * k] | S[2 * k + 1] << 8 for k in range(d1 - d0)]
        exp_B = list(S[2 * (d1 - d0): 2 * (d1 - d0) + (b1 - b0)])
        assert list(D[d0:d1]) == exp_D
        assert list(B[b0:b1]) == exp_B


def test_workers_are_independent():
    h, w, C, n = 12, 9, 3, 6
    IR = _ir(n, 3)
    D, B = oracle.keystream(IR, -1.2, h, w, C, n)
    IR2 = IR.copy()
    IR2[2 * 4, 1] += 1e-9
    D2, B2 = oracle.keystream(IR2, -1.2, h, w, C, n)
    dsl, bsl = _slices(C * (h + w), n), _slices(h * w * C, n)
    for i in range(n):
        (d0, d1), (b0, b1) = dsl[i], bsl[i]
        same = np.array_equal(D[d0:d1], D2[d0:d1]) and np.array_equal(B[b0:b1], B2[b0:b1])
        assert same == (i != 4)


def test_workers_fed_from_one_master_trajectory_are_shifted_copies():
    """Documented consequence of the reading of Algorithm 2 (pair i starts at IR[2i] and IR[2i+1]):
    IR holds consecutive iterates of one trajectory of Eq. (1), and the workers iterate the same map,
    so chain 2i+1 is chain 2i one step ahead and worker i's byte stream is worker 0's stream shifted by
    2i steps (48 i bytes).  The D/B slices then come from one sequence.  With a small step (h = 0.001)
    the XOR of adjacent iterates leaves the sixth extracted byte (mantissa bits 40-47) far from uniform;
    at the default step (0.01) it is uniform."""
    key = si.key(21)
    ic = oracle.key_to_ic(key)
    F = si.gradient_frame(64, 96, 3, seed=21)
    IR, _ = oracle.master(np.array(ic[:4]), oracle.frame_digest(F), ic[4])
    IR = np.asarray(IR).reshape(-1, 4)
    assert np.array_equal(oracle.rk4_step(IR[0], ic[4]), IR[1])

    def stream(i, steps):
        a = oracle.rk4_trajectory(IR[2 * i], ic[4], steps)
        b = oracle.rk4_trajectory(IR[2 * i + 1], ic[4], steps)
        x = (a.view(np.uint64) ^ b.view(np.uint64)) & np.uint64(0xFFFFFFFFFFFF)
        return np.stack([(x >> np.uint64(8 * k)) & np.uint64(255) for k in range(6)], axis=-1).reshape(-1)

    s0 = stream(0, 2000)
    for i in (1, 5):
        assert np.array_equal(stream(i, 1000)[:24 * 900], s0[48 * i:48 * i + 24 * 900])

    def sixth_chi2(h):   # a pair one step of h apart on one trajectory, as IR[0] and IR[1] are
        a = oracle.rk4_trajectory(IR[0], ic[4], 2000, h)
        b = oracle.rk4_trajectory(oracle.rk4_step(IR[0], ic[4], h), ic[4], 2000, h)
        x = (a.view(np.uint64) ^ b.view(np.uint64)) >> np.uint64(40) & np.uint64(255)
        z = np.bincount(x.reshape(-1).astype(np.int64), minlength=256)
        e = z.sum() / 256.0
        return ((z - e) ** 2 / e).sum()

    assert sixth_chi2(0.001) > 1000.0                        # uniform bytes would give ~255
    assert sixth_chi2(oracle.DEFAULT_H) < 330.0


def _records(IR0, gamma, R, h):
    """Records r = 0..R-1 of one trajectory from s_1 = IR0: the 24 stream bytes of s_{r+2} xor s_{r+3}
    (x, y, z, w in turn, six low mantissa bytes each, least significant first)."""
    S = oracle.rk4_trajectory(IR0, gamma, R + 1, h)          # s_2 .. s_{R+2}
    x = (S.view(np.uint64)[:-1] ^ S.view(np.uint64)[1:]) & np.uint64(0xFFFFFFFFFFFF)
    return np.stack([(x >> np.uint64(8 * k)) & np.uint64(255) for k in range(6)], axis=-1).astype(np.uint8).reshape(-1)


@pytest.mark.parametrize("h,w,C,n", [(16, 16, 3, 32), (1, 16, 3, 32), (7, 5, 1, 4), (9, 33, 3, 1), (2, 2, 1, 64),
                                     (32, 48, 3, 32), (3, 8, 3, 7)])
def test_keystream_is_windows_of_one_trajectory(h, w, C, n):
    """The identity the one-trajectory keystream route computes, checked against the oracle's Algorithm 2:
    with R = ceil((48 (n - 1) + 2 ceil(L_D / n) + ceil(N / n)) / 24) records of the frame's LHCS_m trajectory
    continued from IR[0], worker i's slice of D (16-bit little-endian pairs) and then its slice of B are the
    record bytes from 48 i on.  Shapes with one worker, slices shorter than 16 bytes and n > the number of
    rows are included."""
    key = si.key(30 + n)
    ic = oracle.key_to_ic(key)
    H = oracle.sha256(bytes(si.rng(n).integers(0, 256, 64, dtype=np.uint8)))
    IR, _ = oracle.master(np.array(ic[:4]), H, ic[4], n=n)
    D0, B0 = oracle.keystream(IR, ic[4], h, w, C, n=n)
    LD, LB = C * (h + w), h * w * C
    R = -(-(48 * (n - 1) + 2 * -(-LD // n) + -(-LB // n)) // 24)
    G = _records(np.asarray(IR).reshape(-1, 4)[0], ic[4], R, oracle.DEFAULT_H)
    D1, B1 = np.zeros(LD, np.uint16), np.zeros(LB, np.uint8)
    for i, ((d0, d1), (b0, b1)) in enumerate(zip(_slices(LD, n), _slices(LB, n))):
        src = G[48 * i:48 * i + 2 * (d1 - d0) + (b1 - b0)]
        assert src.size == 2 * (d1 - d0) + (b1 - b0)       # R records cover every worker's window
        D1[d0:d1] = src[0:2 * (d1 - d0):2].astype(np.uint16) | (src[1:2 * (d1 - d0):2].astype(np.uint16) << 8)
        B1[b0:b1] = src[2 * (d1 - d0):]
    assert np.array_equal(D0, D1)
    assert np.array_equal(B0, B1)
