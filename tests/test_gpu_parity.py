"""GPU path vs the CPU oracle, step by step and end to end, bit-exact.

Every step of the hot path is called through the C ABI (via the ctypes
binding) on seeded synthetic inputs and compared element by element with the
oracle: sub-frame SHA-256 fold (Sec. II-A), reconstruction + LHCS_m
(Algorithm 1), worker keystream (Algorithm 2), the fused confusion + XOR and
its inverse (Algos 3-7), and whole frames through encrypt_frames /
decrypt_frames.  Integer and index work must match bit for bit; the
binary64 chaotic states too (the iteration is reproduced with round-to-nearest
intrinsics and no contraction, so the tolerance is zero)."""
import numpy as np
import pytest
import torch

import oracle
import synth_inputs as si
from gpu_util import d16, dev, host, host_u16, to_dev

pytestmark = pytest.mark.gpu

fhd = pytest.importorskip("paper_2505_07158_gb300")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


# ---- K1: sub-frame SHA-256 + fold ----

@pytest.mark.parametrize("nbytes,n,count", [(0, 1, 1), (1, 1, 3), (55, 1, 2), (56, 1, 2), (63, 1, 1), (64, 1, 1),
                                            (119, 1, 1), (120, 1, 1), (300, 7, 3), (1000, 32, 2),
                                            (196608, 32, 2), (6220800, 32, 1), (921600, 6, 1), (12345, 12, 4)])
def test_frame_digest(nbytes, n, count):
    data = si.rng(nbytes + n).integers(0, 256, size=nbytes * count, dtype=np.uint8)
    got = host(fhd.fhd_frame_digest(to_dev(data), n=n, count=count))
    for k in range(count):
        assert bytes(got[k]) == oracle.frame_digest(data[k * nbytes:(k + 1) * nbytes], n), k


def test_frame_digest_all_lengths_unaligned():
    # count buffers of odd size laid end to end: every start offset mod 16.
    for nbytes in range(0, 140):
        data = si.rng(nbytes).integers(0, 256, size=nbytes * 17, dtype=np.uint8)
        got = host(fhd.fhd_frame_digest(to_dev(data), n=1, count=17))
        for k in range(17):
            assert bytes(got[k]) == oracle.sha256(data[k * nbytes:(k + 1) * nbytes].tobytes())


# ---- K2a: reconstruction + LHCS_m ----

@pytest.mark.parametrize("n", [1, 6, 32, 100])
def test_master(n):
    g = si.rng(n)
    for trial in range(3):
        v = [float(g.uniform(-50, 50)) for _ in range(4)]
        gamma = float(g.uniform(-1.52, -0.06))
        H = g.integers(0, 256, size=32, dtype=np.uint8)
        IR_ref, ns_ref = oracle.master(v, H.tobytes(), gamma, n=n)
        st = to_dev(np.array(v + [gamma], np.float64))
        IR = fhd.fhd_master(st, to_dev(H), n_workers=n)
        assert np.array_equal(host(IR), IR_ref)
        assert np.array_equal(host(st)[:4], ns_ref)


# ---- K2b: worker keystream ----

@pytest.mark.parametrize("h,w,C,n", [(1, 1, 1, 1), (3, 5, 3, 2), (8, 8, 3, 32), (17, 23, 3, 6), (64, 96, 3, 32),
                                     (256, 256, 3, 32), (37, 53, 4, 12), (2, 2, 1, 40), (1080, 1920, 3, 32)])
def test_keystream(h, w, C, n):
    g = si.rng(h * w + n)
    IR = np.column_stack([g.uniform(0, 20, 2 * n), g.uniform(0, 20, 2 * n), g.uniform(0, 40, 2 * n),
                          g.uniform(0, 20, 2 * n)])
    gamma = -0.83
    D_ref, B_ref = oracle.keystream(IR, gamma, h, w, C, n)
    D, B = fhd.fhd_keystream(to_dev(IR), gamma, h, w, C, n_workers=n)
    assert np.array_equal(host_u16(D), D_ref)
    assert np.array_equal(host(B), B_ref)


# ---- K3 / K4: fused confusion + XOR and inverse ----

SHAPES = [(1, 1, 1), (1, 1, 3), (1, 8, 3), (8, 1, 3), (3, 5, 3), (2, 2, 4), (7, 9, 3), (16, 13, 1), (37, 53, 3),
          (64, 129, 3), (100, 1000, 3), (33, 300, 4), (480, 640, 3), (1080, 1920, 3),
          # planar RGB route (w % 4 == 0): one group per row, a few groups, a wide row
          (5, 4, 3), (3, 12, 3), (17, 36, 3), (2, 4096, 3)]


def _rand(h, w, C, seed):
    g = si.rng(seed)
    return (g.integers(0, 256, size=(h, w, C), dtype=np.uint8), g.integers(0, 65536, size=C * (h + w), dtype=np.uint16),
            g.integers(0, 256, size=h * w * C, dtype=np.uint8))


@pytest.mark.parametrize("shape", SHAPES)
def test_permute_encrypt(shape):
    F, D, B = _rand(*shape, seed=sum(shape))
    E = fhd.fhd_permute_encrypt(to_dev(F), d16(D), to_dev(B))
    assert np.array_equal(host(E), oracle.permute_encrypt(F, D, B))


@pytest.mark.parametrize("shape", SHAPES)
def test_permute_decrypt(shape):
    F, D, B = _rand(*shape, seed=7 * sum(shape))
    E = oracle.permute_encrypt(F, D, B)
    P = fhd.fhd_permute_decrypt(to_dev(E), d16(D), to_dev(B))
    assert np.array_equal(host(P), F)


@pytest.mark.parametrize("P", [1, 2, 8, 32])
def test_permute_strip_overrides(P):
    h, w, C = 45, 77, 3
    fhd.fhd_set_strip_width(h, w, C, P)
    try:
        assert fhd.fhd_strip_width(h, w, C) == P
        F, D, B = _rand(h, w, C, seed=P)
        E = fhd.fhd_permute_encrypt(to_dev(F), d16(D), to_dev(B))
        assert np.array_equal(host(E), oracle.permute_encrypt(F, D, B))
        Pd = fhd.fhd_permute_decrypt(E, d16(D), to_dev(B))
        assert np.array_equal(host(Pd), F)
    finally:
        fhd.fhd_set_strip_width(h, w, C, 0)


# ---- whole frames through encrypt_frames / decrypt_frames ----

def test_config1_frame_and_bit_flip():
    """256x256x3 uniform frame, fixed key: bit-exact vs oracle, round trip, NPCR/UACI."""
    key = si.key(0)
    F = si.uniform_frame(256, 256, 3, seed=0)
    F2, _ = si.bit_flip(F, 0)
    outs = []
    for frame in (F, F2):
        c = fhd.Cipher(key)
        sid = c.open_stream()
        E, H = c.encrypt(sid, to_dev(frame))
        E_ref, H_ref = oracle.Stream.from_key(key).encrypt(frame)
        assert bytes(host(H)) == H_ref
        assert np.array_equal(host(E), E_ref)
        d = fhd.Cipher(key)
        P = d.decrypt(d.open_stream(), E, H)
        assert np.array_equal(host(P), frame)
        outs.append(host(E).astype(np.int32))
    npcr = [100 * np.mean(outs[0][:, :, c] != outs[1][:, :, c]) for c in range(3)]
    assert all(abs(v - 100 * 255 / 256) < 0.2 for v in npcr)


def test_chained_clip_in_one_call_and_per_frame():
    key = si.key(1)
    clip = si.clip(5, 72, 128, 3, seed=1)
    ref = oracle.Stream.from_key(key)
    refs = [ref.encrypt(f) for f in clip]
    # one call, all frames of one stream
    c = fhd.Cipher(key)
    sid = c.open_stream()
    srcs = [to_dev(f) for f in clip]
    dsts = [torch.empty_like(s) for s in srcs]
    digs = [torch.empty(32, dtype=torch.uint8, device=dev()) for _ in clip]
    c.encrypt_frames([(sid, s, d, g) for s, d, g in zip(srcs, dsts, digs)])
    for (E_ref, H_ref), d, g in zip(refs, dsts, digs):
        assert bytes(host(g)) == H_ref
        assert np.array_equal(host(d), E_ref)
    # one call per frame gives the same
    c2 = fhd.Cipher(key)
    sid2 = c2.open_stream()
    for f, (E_ref, H_ref) in zip(clip, refs):
        E, H = c2.encrypt(sid2, to_dev(f))
        assert np.array_equal(host(E), E_ref) and bytes(host(H)) == H_ref
    # decrypt in one call
    r = fhd.Cipher(key)
    rid = r.open_stream()
    outs = [torch.empty_like(s) for s in srcs]
    r.decrypt_frames([(rid, d, o, g) for d, o, g in zip(dsts, outs, digs)])
    for o, f in zip(outs, clip):
        assert np.array_equal(host(o), f)
    assert c.export_state(sid) == r.export_state(rid) == c2.export_state(sid2)


def test_mixed_batch_streams_and_sizes():
    """Frames of several streams (own keys) and sizes in one call == each alone."""
    shapes = [(48, 64, 3), (30, 50, 3), (64, 64, 1), (20, 36, 4), (48, 64, 3), (30, 50, 3)]
    keys = [si.key(10 + k) for k in range(3)]
    owner = [0, 1, 2, 0, 1, 2]
    frames = [si.uniform_frame(*s, seed=40 + k) for k, s in enumerate(shapes)]
    c = fhd.Cipher(si.key(99))
    sids = [c.open_stream(k) for k in keys]
    items, outs, digs = [], [], []
    for f, o in zip(frames, owner):
        s = to_dev(f)
        outs.append(torch.empty_like(s))
        digs.append(torch.empty(32, dtype=torch.uint8, device=dev()))
        items.append((sids[o], s, outs[-1], digs[-1]))
    c.encrypt_frames(items)
    refs = [oracle.Stream.from_key(k) for k in keys]
    for f, o, out, dg in zip(frames, owner, outs, digs):
        E_ref, H_ref = refs[o].encrypt(f)
        assert np.array_equal(host(out), E_ref) and bytes(host(dg)) == H_ref


@pytest.mark.parametrize("n", [1, 6, 12, 33])
def test_worker_counts(n):
    key = si.key(n)
    F = si.gradient_frame(40, 56, 3, seed=n)
    c = fhd.Cipher(key, n_workers=n)
    E, H = c.encrypt(c.open_stream(), to_dev(F))
    E_ref, H_ref = oracle.Stream.from_key(key, n=n).encrypt(F)
    assert bytes(host(H)) == H_ref and np.array_equal(host(E), E_ref)


def test_raw_key_and_state_resume():
    ic = (1.25, 2.5, 3.75, 4.0, -1.0)
    frames = si.clip(3, 32, 40, 3, seed=5)
    c = fhd.Cipher(ic=ic)
    sid = c.open_stream()
    c.encrypt(sid, to_dev(frames[0]))
    state = c.export_state(sid)
    E1, H1 = c.encrypt(sid, to_dev(frames[1]))
    c2 = fhd.Cipher(ic=(0, 0, 0, 0, -0.5))
    s2 = c2.open_stream()
    c2.import_state(s2, state)
    E2, H2 = c2.encrypt(s2, to_dev(frames[1]))
    assert np.array_equal(host(E1), host(E2)) and bytes(host(H1)) == bytes(host(H2))
    ref = oracle.Stream(ic)
    ref.encrypt(frames[0])
    E_ref, _ = ref.encrypt(frames[1])
    assert np.array_equal(host(E1), E_ref)


def test_edge_cases_and_errors():
    c = fhd.Cipher(si.key(3))
    sid = c.open_stream()
    c.encrypt_frames([])                       # empty batch: no-op
    src = torch.zeros((4, 4, 3), dtype=torch.uint8, device=dev())
    dig = torch.empty(32, dtype=torch.uint8, device=dev())
    with pytest.raises(fhd.FhdError) as e:
        c.encrypt_frames([(sid + 7, src, torch.empty_like(src), dig)])
    assert e.value.code == fhd.FHD_ERR_BAD_STREAM
    with pytest.raises(fhd.FhdError) as e:
        c.encrypt_frames([(sid, src, src, dig)])
    assert e.value.code == fhd.FHD_ERR_INVALID_ARG
    zero = torch.zeros((0, 4, 3), dtype=torch.uint8, device=dev())
    with pytest.raises(fhd.FhdError) as e:
        c.encrypt_frames([(sid, zero, torch.empty_like(zero), dig)])
    assert e.value.code == fhd.FHD_ERR_INVALID_ARG
    c5 = torch.zeros((2, 2, 5), dtype=torch.uint8, device=dev())
    with pytest.raises(fhd.FhdError):
        c.encrypt_frames([(sid, c5, torch.empty_like(c5), dig)])
    # a 1x1 frame and a flat frame (digest cancellation) still round-trip
    for F in (np.array([[[7]]], np.uint8), np.full((16, 16, 3), 77, np.uint8)):
        key = si.key(4)
        a = fhd.Cipher(key)
        E, H = a.encrypt(a.open_stream(), to_dev(F))
        E_ref, H_ref = oracle.Stream.from_key(key).encrypt(F)
        assert np.array_equal(host(E), E_ref) and bytes(host(H)) == H_ref
        b = fhd.Cipher(key)
        assert np.array_equal(host(b.decrypt(b.open_stream(), E, H)), F)
    c.sync_status()


def test_receiver_side_verification():
    """The decrypted frame re-hashes to the transmitted digest; a flipped
    ciphertext byte or a wrong digest is caught."""
    key = si.key(31)
    frames = [si.gradient_frame(48, 64, 3, t=t, seed=31) for t in range(3)]
    enc, dec = fhd.Cipher(key, n_workers=6), fhd.Cipher(key, n_workers=6)
    sid, rid = enc.open_stream(), dec.open_stream()
    srcs = [to_dev(f) for f in frames]
    E = [torch.empty_like(s) for s in srcs]
    R = [torch.empty_like(s) for s in srcs]
    H = [torch.empty(32, dtype=torch.uint8, device=dev()) for _ in srcs]
    enc.encrypt_frames([(sid, s, e, h) for s, e, h in zip(srcs, E, H)])
    E[1].view(-1)[100] ^= 1                      # damage frame 1 in transit
    dec.decrypt_frames([(rid, e, r, h) for e, r, h in zip(E, R, H)])
    Hbad = H[2].clone()
    Hbad[0] ^= 0x80
    ok = dec.verify_frames([(rid, e, r, h) for e, r, h in zip(E, R, [H[0], H[1], Hbad])])
    assert host(ok).tolist() == [1, 0, 0]


# ---- the single-pass encryption (gather route) against the two passes and the oracle ----

GATHER_SHAPES = [(1, 16, 3), (2, 32, 3), (37, 48, 3), (64, 112, 3), (200, 320, 3), (480, 640, 3),
                 (720, 1280, 3), (3, 4096, 3)]


@pytest.mark.parametrize("shape", GATHER_SHAPES)
@pytest.mark.parametrize("P", [0, 16, 32, 64, 128])
def test_single_pass_encrypt_matches_two_passes_and_oracle(shape, P):
    """Every strip width the single pass takes (0 = the built-in choice), full and tail strips
    (w % P != 0), one-row and one-strip frames: bit-exact with the oracle and with the two-pass route."""
    h, w, C = shape
    if P and (h * P * C + 15) // 16 * 16 > 232448:
        pytest.skip("strip does not fit shared memory")
    F, D, B = _rand(h, w, C, seed=h + w + P)
    ref = oracle.permute_encrypt(F, D, B)
    if P:
        fhd.fhd_set_strip_width(h, w, C, P)
    try:
        outs = {}
        for route in ("single_pass", "two_pass"):
            fhd.fhd_set_encrypt_route(route)
            outs[route] = host(fhd.fhd_permute_encrypt(to_dev(F), d16(D), to_dev(B)))
    finally:
        fhd.fhd_set_encrypt_route("two_pass")
        fhd.fhd_set_strip_width(h, w, C, 0)
    assert np.array_equal(outs["single_pass"], ref)
    assert np.array_equal(outs["two_pass"], ref)


def test_single_pass_in_a_mixed_batch_of_streams():
    """A batch whose frames all take the single pass (several sizes, strip widths and streams, chained
    frames of one stream), and the same batch with one frame that does not (w % 16 != 0), which sends
    the whole batch through the two passes: both equal the oracle streams."""
    fhd.fhd_set_encrypt_route("single_pass")
    try:
        _mixed_batches_match_oracle()
    finally:
        fhd.fhd_set_encrypt_route("two_pass")


@pytest.mark.parametrize("shape", [(1080, 1920, 3), (2160, 3840, 3)])
def test_single_pass_encrypt_full_size(shape):
    F, D, B = _rand(*shape, seed=sum(shape))
    fhd.fhd_set_encrypt_route("single_pass")
    try:
        E = host(fhd.fhd_permute_encrypt(to_dev(F), d16(D), to_dev(B)))
    finally:
        fhd.fhd_set_encrypt_route("two_pass")
    assert np.array_equal(E, oracle.permute_encrypt(F, D, B))


def _mixed_batches_match_oracle():
    for shapes in ([(48, 64, 3), (30, 96, 3), (16, 16, 3), (72, 160, 3)],
                   [(48, 64, 3), (30, 96, 3), (20, 36, 3), (72, 160, 3)]):
        keys = [si.key(900 + k) for k in range(3)]
        c = fhd.Cipher(keys[0], n_workers=5)
        sids = [c.open_stream(k) for k in keys]
        refs = [oracle.Stream.from_key(k, n=5) for k in keys]
        items, frames = [], []
        for t, s in enumerate(shapes):
            st = t % 3 if t < 3 else 0           # frames 0 and 3 are consecutive frames of stream 0
            F = si.gradient_frame(*s, t=t, seed=31)
            frames.append((st, F))
            items.append((sids[st], to_dev(F), torch.empty(s, dtype=torch.uint8, device=dev()),
                          torch.empty(32, dtype=torch.uint8, device=dev())))
        c.encrypt_frames(items)
        torch.cuda.synchronize()
        for (st, F), it in zip(frames, items):
            E_ref, H_ref = refs[st].encrypt(F)
            assert bytes(host(it[3])) == H_ref
            assert np.array_equal(host(it[2]), E_ref)
        c.close()


@pytest.mark.parametrize("RB", [1, 3, 7, 16, 64])
def test_permute_row_band_overrides(RB):
    """Every row band the autotuner may install (including bands taller than the frame, ragged last
    bands and the byte-wise route of w % 4 != 0) gives the oracle's bytes both ways."""
    for h, w, C in [(45, 64, 3), (45, 77, 3), (20, 36, 4)]:
        fhd.fhd_set_row_band(h, w, C, RB)
        try:
            assert fhd.fhd_row_band(h, w, C) == RB
            F, D, B = _rand(h, w, C, seed=RB + w)
            E = fhd.fhd_permute_encrypt(to_dev(F), d16(D), to_dev(B))
            assert np.array_equal(host(E), oracle.permute_encrypt(F, D, B)), (h, w, C)
            Pd = fhd.fhd_permute_decrypt(E, d16(D), to_dev(B))
            assert np.array_equal(host(Pd), F), (h, w, C)
        finally:
            fhd.fhd_set_row_band(h, w, C, 0)


@pytest.mark.parametrize("st,rt", [(256, 128), (256, 256), (512, 128)])
def test_permute_cta_thread_overrides(st, rt):
    """Every CTA shape the autotuner may install for the two passes gives the oracle's bytes both ways: the
    column-word route (h % 4 == 0), the byte-scatter route (h % 4 != 0) and the byte-wise row route
    (w % 4 != 0), full and tail strips, at 1080p too."""
    for h, w, C in [(44, 64, 3), (45, 77, 3), (20, 36, 4), (48, 100, 1), (1080, 1920, 3)]:
        fhd.fhd_set_cta_threads(h, w, C, st, rt)
        try:
            assert fhd.fhd_cta_threads(h, w, C) == (st, rt)
            F, D, B = _rand(h, w, C, seed=st + rt + w)
            E = fhd.fhd_permute_encrypt(to_dev(F), d16(D), to_dev(B))
            assert np.array_equal(host(E), oracle.permute_encrypt(F, D, B)), (h, w, C)
            Pd = fhd.fhd_permute_decrypt(E, d16(D), to_dev(B))
            assert np.array_equal(host(Pd), F), (h, w, C)
        finally:
            fhd.fhd_set_cta_threads(h, w, C, 0, 0)
