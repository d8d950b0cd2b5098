"""The persistent batch kernel (one launch for every step of a batch) against the oracle.

* A round trip (sender encrypts, receiver decrypts the ciphertexts) of mixed shapes and streams, with a
  stream that has two frames in the batch, for both digest modes and both transports: ciphertexts,
  digests, decrypted frames and the chaining states after the launch equal the oracle's.
* One direction at a time (encrypt_frames_persistent, then decrypt_frames_persistent).
* The round trip captured in a CUDA graph and replayed: every replay is the next frame of every stream.
* A withheld dependency (the test hook holds one frame's digest back): the bounded waits run out, both
  handles report FHD_ERR_TIMEOUT, the launch ends within the limit, and the device keeps working."""
import time

import numpy as np
import pytest
import torch

import oracle
import synth_inputs as si
from gpu_util import dev, host, to_dev

pytestmark = pytest.mark.gpu

fhd = pytest.importorskip("paper_2505_07158_gb300")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_07158_gb300 import batching  # noqa: E402

SHAPES = [(48, 64, 3), (30, 50, 3), (64, 64, 1), (20, 36, 4), (72, 160, 3), (16, 16, 3), (37, 53, 3)]


def _batch(keys, shapes, n, mode="xor", transport="plain", seed=0):
    enc = fhd.Cipher(keys[0], n_workers=n, digest_mode=mode, digest_transport=transport)
    dec = fhd.Cipher(keys[0], n_workers=n, digest_mode=mode, digest_transport=transport)
    # streams: one per key; the last frame belongs to stream 0 again (two frames of one stream)
    sids = [enc.open_stream(k) for k in keys]
    rids = [dec.open_stream(k) for k in keys]
    enc_items, dec_items, frames, owner = [], [], [], []
    for t, s in enumerate(shapes):
        st = t if t < len(keys) else 0
        F = si.gradient_frame(*s, t=t, seed=seed)
        Fd = to_dev(F)
        E = torch.empty_like(Fd)
        R = torch.empty_like(Fd)
        H = torch.empty(32, dtype=torch.uint8, device=dev())
        enc_items.append((sids[st], Fd, E, H))
        dec_items.append((rids[st], E, R, H))
        frames.append(F)
        owner.append(st)
    return enc, dec, enc_items, dec_items, frames, owner


@pytest.mark.parametrize("n,mode,transport", [(5, "xor", "plain"), (32, "xor", "plain"), (7, "tree", "plain"),
                                              (6, "xor", "masked")])
def test_round_trip_matches_oracle(n, mode, transport):
    keys = [si.key(1300 + k) for k in range(len(SHAPES) - 1)]
    enc, dec, ei, di, frames, owner = _batch(keys, SHAPES, n, mode, transport, seed=n)
    enc.round_trip_persistent(dec, ei, di)
    torch.cuda.synchronize()
    enc.sync_status()
    dec.sync_status()
    refs = [oracle.Stream.from_key(k, n=n, digest_mode=mode, transport=transport) for k in keys]
    for k, F in enumerate(frames):
        E_ref, H_ref = refs[owner[k]].encrypt(F)
        assert np.array_equal(host(ei[k][2]), E_ref), k
        # the receiver unmasks the transmitted digest in place: the buffer ends with H itself
        assert bytes(host(ei[k][3])) == (H_ref if transport == "plain" else oracle.frame_digest(F, n, mode)), k
        assert np.array_equal(host(di[k][2]), F), k
    for st, ref in enumerate(refs):
        sent = np.frombuffer(enc.export_state(ei[[o for o in range(len(owner)) if owner[o] == st][0]][0])[:32],
                             dtype=np.float64)
        assert np.array_equal(sent, ref.state), st
    enc.close()
    dec.close()


def test_one_direction_at_a_time():
    keys = [si.key(1400 + k) for k in range(len(SHAPES) - 1)]
    enc, dec, ei, di, frames, owner = _batch(keys, SHAPES, 9, seed=3)
    enc.encrypt_frames_persistent(ei)
    dec.decrypt_frames_persistent(di)
    torch.cuda.synchronize()
    enc.sync_status()
    dec.sync_status()
    refs = [oracle.Stream.from_key(k, n=9) for k in keys]
    for k, F in enumerate(frames):
        E_ref, H_ref = refs[owner[k]].encrypt(F)
        assert np.array_equal(host(ei[k][2]), E_ref), k
        assert bytes(host(ei[k][3])) == H_ref, k
        assert np.array_equal(host(di[k][2]), F), k
    enc.close()
    dec.close()


def test_graph_replays_are_the_next_frames():
    shapes = SHAPES[:-1]
    keys = [si.key(1500 + k) for k in range(len(shapes))]
    enc, dec, ei, di, frames, owner = _batch(keys, shapes, 8, seed=5)
    call = batching.PersistentRoundTrip(enc, dec, ei, di, graph=True)
    refs = [oracle.Stream.from_key(k, n=8) for k in keys]
    for rep in range(3):
        call.replay()
        torch.cuda.synchronize()
        for k, F in enumerate(frames):
            E_ref, H_ref = refs[k].encrypt(F)
            assert np.array_equal(host(ei[k][2]), E_ref), (rep, k)
            assert bytes(host(ei[k][3])) == H_ref
            assert np.array_equal(host(di[k][2]), F)
    enc.sync_status()
    dec.sync_status()
    enc.close()
    dec.close()


def test_withheld_dependency_times_out_and_the_device_recovers():
    keys = [si.key(1600 + k) for k in range(len(SHAPES) - 1)]
    enc, dec, ei, di, frames, owner = _batch(keys, SHAPES, 5, seed=7)
    enc.set_persistent_limits(timeout_ns=50_000_000, hold_frame=2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    enc.round_trip_persistent(dec, ei, di)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    for c in (enc, dec):
        with pytest.raises(fhd.FhdError) as exc:
            c.sync_status()
        assert exc.value.code == fhd.FHD_ERR_TIMEOUT
    assert elapsed < 5.0
    # the device and the library still work: a fresh pair of handles round-trips the batch correctly
    enc.close()
    dec.close()
    enc, dec, ei, di, frames, owner = _batch(keys, SHAPES, 5, seed=7)
    enc.round_trip_persistent(dec, ei, di)
    torch.cuda.synchronize()
    enc.sync_status()
    dec.sync_status()
    for k, F in enumerate(frames):
        assert np.array_equal(host(di[k][2]), F), k
    enc.close()
    dec.close()


def test_long_streams_and_mixed_sizes_within_a_stream():
    """Streams with many frames in one launch, whose frames differ in size (a stream's first frame the
    largest, so its LHCS_m task must be queued ahead of its later, smaller frames' worker warps), with the
    maximum of 64 frames: every ciphertext and digest equals the oracle's, and every frame round-trips."""
    sizes = [(40, 64, 3), (24, 32, 3), (16, 16, 3), (8, 48, 1)]
    keys = [si.key(1700 + k) for k in range(3)]
    enc = fhd.Cipher(keys[0], n_workers=6)
    dec = fhd.Cipher(keys[0], n_workers=6)
    sids = [enc.open_stream(k) for k in keys]
    rids = [dec.open_stream(k) for k in keys]
    ei, di, frames, owner = [], [], [], []
    for t in range(64):
        st = 0 if t < 30 else (1 if t < 50 else 2)      # 30, 20 and 14 frames
        s = sizes[0] if t in (0, 30, 50) else sizes[(t * 7) % 4]
        F = si.gradient_frame(*s, t=t, seed=17)
        Fd = to_dev(F)
        E, R = torch.empty_like(Fd), torch.empty_like(Fd)
        H = torch.empty(32, dtype=torch.uint8, device=dev())
        ei.append((sids[st], Fd, E, H))
        di.append((rids[st], E, R, H))
        frames.append(F)
        owner.append(st)
    enc.round_trip_persistent(dec, ei, di)
    torch.cuda.synchronize()
    enc.sync_status()
    dec.sync_status()
    refs = [oracle.Stream.from_key(k, n=6) for k in keys]
    for k, F in enumerate(frames):
        E_ref, H_ref = refs[owner[k]].encrypt(F)
        assert np.array_equal(host(ei[k][2]), E_ref), k
        assert bytes(host(ei[k][3])) == H_ref, k
        assert np.array_equal(host(di[k][2]), F), k
    with pytest.raises(fhd.FhdError):       # more than 64 frames in one launch
        enc.round_trip_persistent(dec, ei + ei[:1], di + di[:1])
    enc.close()
    dec.close()


@pytest.fixture
def ks_route():
    """Set the process-wide keystream route for one test and restore the default afterwards."""
    yield fhd.fhd_set_keystream_route
    fhd.fhd_set_keystream_route("trajectory")


@pytest.mark.parametrize("ks", ["pairs", "trajectory"])
def test_round_trip_under_both_keystream_routes(ks_route, ks):
    """The persistent round trip with the worker-pair keystream tasks and with the one-trajectory tasks (a
    trajectory task per frame and side, then emission tasks of 180,224 bytes of B each): frames of one to
    sixteen emission tasks, one whose size is not a multiple of 16 and one of a single task, all equal to
    the oracle."""
    ks_route(ks)
    shapes = [(480, 640, 3), (16, 16, 3), (720, 1280, 3), (30, 50, 3), (481, 641, 3)]
    keys = [si.key(1800 + k) for k in range(len(shapes) - 1)]
    enc, dec, ei, di, frames, owner = _batch(keys, shapes, 32, seed=21)
    enc.round_trip_persistent(dec, ei, di)
    torch.cuda.synchronize()
    enc.sync_status()
    dec.sync_status()
    refs = [oracle.Stream.from_key(k, n=32) for k in keys]
    for k, F in enumerate(frames):
        E_ref, H_ref = refs[owner[k]].encrypt(F)
        assert np.array_equal(host(ei[k][2]), E_ref), k
        assert bytes(host(ei[k][3])) == H_ref, k
        assert np.array_equal(host(di[k][2]), F), k
    enc.close()
    dec.close()
