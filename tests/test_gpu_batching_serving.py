"""Batched mixed-resolution launches, CUDA-graph replay and the serving loop.

Each frame's result must be the same alone and in the mix: graph replays of a
mixed batch are compared with the CPU oracle stream by stream, and every
frame the continuous-batching server produced is compared (by a digest of the
ciphertext) with the same stream encrypted alone, one frame per call."""
import ctypes

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

from paper_2505_07158_gb300 import batching, serving  # noqa: E402


def test_graphed_mixed_batch_matches_oracle():
    shapes = [(48, 64, 3), (30, 50, 3), (64, 64, 1), (20, 36, 4), (72, 40, 3), (16, 16, 3)]
    keys = [si.key(200 + k) for k in range(len(shapes))]
    frames = [to_dev(si.uniform_frame(*s, seed=300 + k)) for k, s in enumerate(shapes)]
    enc = fhd.Cipher(si.key(1))
    enc_items, dec_items, dec = batching.mixed_batch(shapes, keys, enc, frames)
    g_enc = batching.GraphedCall(enc, enc_items, encrypt=True)
    g_dec = batching.GraphedCall(dec, dec_items, encrypt=False)
    refs = [oracle.Stream.from_key(k) for k in keys]
    for rep in range(2):            # two replays = the first two frames of every stream
        g_enc.replay()
        g_dec.replay()
        torch.cuda.synchronize()
        for k, (sid, F, E, H) in enumerate(enc_items):
            E_ref, H_ref = refs[k].encrypt(host(F))
            assert np.array_equal(host(E), E_ref), (rep, k)
            assert bytes(host(H)) == H_ref
            assert np.array_equal(host(dec_items[k][2]), host(F))


def test_concurrent_cuda_streams_share_one_handle():
    keys = [si.key(400 + k) for k in range(4)]
    c = fhd.Cipher(keys[0])
    sids = [c.open_stream(k) for k in keys]
    lanes = [torch.cuda.Stream() for _ in range(2)]
    frames = [[to_dev(si.gradient_frame(40, 64, 3, t=t, seed=k)) for t in range(3)] for k in range(4)]
    outs = [[None] * 3 for _ in range(4)]
    for t in range(3):
        for k in range(4):
            E = torch.empty_like(frames[k][t])
            H = torch.empty(32, dtype=torch.uint8, device=dev())
            lane = lanes[k % 2]
            c.encrypt_frames([(sids[k], frames[k][t], E, H)], stream=lane)
            outs[k][t] = E
    torch.cuda.synchronize()
    for k in range(4):
        ref = oracle.Stream.from_key(keys[k])
        for t in range(3):
            E_ref, _ = ref.encrypt(host(frames[k][t]))
            assert np.array_equal(host(outs[k][t]), E_ref)


def test_served_results_equal_alone():
    shapes_avail = [(64, 96, 3), (48, 64, 3), (32, 48, 1)]
    nstreams = 8
    g = si.rng(7)
    shapes = [shapes_avail[int(g.integers(3))] for _ in range(nstreams)]
    keys = [si.key(500 + k) for k in range(nstreams)]
    pool = {s: [to_dev(si.gradient_frame(*s, t=t, seed=9)) for t in range(5)] for s in set(shapes)}
    stats, srv = serving.run(keys, shapes, pool, fps=60.0, duration=1.5, seed=3, n_workers=8, fingerprint=True)
    assert stats["completed_frames"] == stats["offered_frames"] > 0
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    srv.close()
    # the same streams alone, one frame per call
    alone = fhd.Cipher(keys[0], n_workers=8)
    for s in range(nstreams):
        sid = alone.open_stream(keys[s])
        seqs = sorted(q for (st, q) in srv.prints if st == s)
        assert seqs == list(range(len(seqs)))
        for q in seqs:
            src = pool[shapes[s]][(s * 7 + q) % 5]
            E, _ = alone.encrypt(sid, src)
            d = bytes(host(fhd.fhd_frame_digest(E.view(-1), n=256)).reshape(-1))
            assert d == srv.prints[(s, q)], (s, q)


def test_budget_admission_limits_in_flight_bytes():
    shapes = [(64, 64, 3)] * 4
    keys = [si.key(600 + k) for k in range(4)]
    pool = {(64, 64, 3): [to_dev(si.uniform_frame(64, 64, 3, seed=1))]}
    one = serving.frame_footprint(64, 64, 3, 8)
    stats, srv = serving.run(keys, shapes, pool, fps=200.0, duration=0.5, seed=1, n_workers=8,
                             budget_bytes=2 * one)
    assert srv.peak <= 2 * one
    assert stats["completed_frames"] == stats["offered_frames"]
    srv.close()


def test_event_ordered_frames_across_cuda_streams():
    """Consecutive frames of one stream on alternating CUDA streams, ordered only
    at the chaining step with events, equal the oracle's sequential encryption."""
    key = si.key(700)
    c = fhd.Cipher(key, n_workers=6)
    sid = c.open_stream()
    lanes = [torch.cuda.Stream() for _ in range(3)]
    frames = [to_dev(si.gradient_frame(56, 72, 3, t=t, seed=70)) for t in range(7)]
    outs, last = [], None
    for t, F in enumerate(frames):
        E = torch.empty_like(F)
        H = torch.empty(32, dtype=torch.uint8, device=dev())
        ev = torch.cuda.Event()
        c.encrypt_frames([(sid, F, E, H)], stream=lanes[t % 3], master_event=ev,
                         wait_events=[last] if last is not None else [])
        last = ev
        outs.append((E, H))
    torch.cuda.synchronize()
    ref = oracle.Stream.from_key(key, n=6)
    for F, (E, H) in zip(frames, outs):
        E_ref, H_ref = ref.encrypt(host(F))
        assert np.array_equal(host(E), E_ref) and bytes(host(H)) == H_ref


def test_receiver_starts_before_ciphertext_arrives():
    """decrypt_frames(data_events=...): the chaotic stage runs on the digests while the
    ciphertext is still on its way; the inverse permutation waits for the data event.  The
    sender's stream delays the ciphertext copy behind a fixed-length sleep kernel, so a
    permutation that did not wait would read the zero-filled receive buffer."""
    shapes = [(96, 128, 3), (60, 100, 3)]
    key = si.key(610)
    frames = [to_dev(si.gradient_frame(*s, t=t, seed=611)) for t, s in enumerate(shapes)]
    snd, rcv = fhd.Cipher(key), fhd.Cipher(key)
    sid, rid = snd.open_stream(), rcv.open_stream()
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    E = [torch.empty_like(f) for f in frames]
    wire = [torch.zeros_like(f) for f in frames]       # the receiver's ciphertext buffers
    H = torch.empty((len(frames), 32), dtype=torch.uint8, device=dev())
    R = [torch.empty_like(f) for f in frames]
    digests_ready, data_ready = torch.cuda.Event(), torch.cuda.Event()
    torch.cuda.synchronize()
    snd.encrypt_frames([(sid, frames[k], E[k], H[k]) for k in range(len(frames))], stream=sa,
                       digest_event=digests_ready, keystream_event=torch.cuda.Event())
    with torch.cuda.stream(sa):
        torch.cuda._sleep(20_000_000)                   # ~10 ms: the ciphertext is late
        for k in range(len(frames)):
            wire[k].copy_(E[k])
        data_ready.record(sa)
    rx_keys = torch.cuda.Event()
    rcv.decrypt_frames([(rid, wire[k], R[k], H[k]) for k in range(len(frames))], stream=sb,
                       wait_events=[digests_ready], data_events=[data_ready], keystream_event=rx_keys)
    torch.cuda.synchronize()
    assert rx_keys.query()
    ref = oracle.Stream.from_key(key)
    for k in range(len(frames)):
        E_ref, H_ref = ref.encrypt(host(frames[k]))
        assert np.array_equal(host(E[k]), E_ref), k
        assert bytes(host(H[k])) == H_ref
        assert torch.equal(R[k], frames[k]), k
    with pytest.raises(ValueError):
        rcv.decrypt_frames([(rid, wire[0], R[0], H[0])], stream=sb, data_events=[torch.cuda.Event()])


def test_worker_gate_holds_only_the_workers():
    """worker_wait_events gate the worker kernel alone: with the gate held by a ~10 ms sleep on
    another CUDA stream, the digest stage and LHCS_m finish before it, the workers start after it,
    and the ciphertext and digest are the oracle's."""
    key = si.key(630)
    F = to_dev(si.gradient_frame(120, 160, 3, t=0, seed=631))
    c = fhd.Cipher(key)
    sid = c.open_stream()
    E, H = torch.empty_like(F), torch.empty(32, dtype=torch.uint8, device=dev())
    other, s = torch.cuda.Stream(), torch.cuda.Stream()
    origin, gate = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    c.profile(True)
    origin.record(s)
    other.wait_event(origin)
    with torch.cuda.stream(other):
        torch.cuda._sleep(20_000_000)
        gate.record(other)
    c.encrypt_frames([(sid, F, E, H)], stream=s, master_event=torch.cuda.Event(), worker_wait_events=[gate])
    torch.cuda.synchronize()
    spans = {k: (a, b) for k, a, b in c.profile_spans(origin)}
    c.profile(False)
    gate_ms = origin.elapsed_time(gate)
    assert gate_ms > 1.0
    assert spans["sha"][1] < gate_ms and spans["master"][1] < gate_ms
    assert spans["keystream"][0] >= gate_ms - 1e-3
    E_ref, H_ref = oracle.Stream.from_key(key).encrypt(host(F))
    assert np.array_equal(host(E), E_ref) and bytes(host(H)) == H_ref
    # a nonzero count with a null list is an argument error, caught before anything is enqueued
    hk = fhd._lib.FhdSchedule()
    hk.n_worker_waits = 1
    arr, n = c._frames([(sid, F, E, H)])
    assert fhd._lib.load().encrypt_frames_sched(c._handle(), n, arr, None, ctypes.byref(hk)) == fhd.FHD_ERR_INVALID_ARG


def test_worker_gate_on_the_receiver_and_a_null_schedule():
    """The worker gate on decrypt_frames holds the receiver's workers behind an event (its LHCS_m runs
    first); encrypt_frames_sched / decrypt_frames_sched with a NULL schedule behave as the plain calls."""
    key = si.key(660)
    F = to_dev(si.gradient_frame(72, 96, 3, t=0, seed=661))
    snd, rcv = fhd.Cipher(key), fhd.Cipher(key)
    sid, rid = snd.open_stream(), rcv.open_stream()
    E, R = torch.empty_like(F), torch.empty_like(F)
    H = torch.empty(32, dtype=torch.uint8, device=dev())
    snd.encrypt_frames([(sid, F, E, H)])
    torch.cuda.synchronize()
    other, s = torch.cuda.Stream(), torch.cuda.Stream()
    origin, gate = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rcv.profile(True)
    origin.record(s)
    other.wait_event(origin)
    with torch.cuda.stream(other):
        torch.cuda._sleep(20_000_000)
        gate.record(other)
    rcv.decrypt_frames([(rid, E, R, H)], stream=s, master_event=torch.cuda.Event(), worker_wait_events=[gate])
    torch.cuda.synchronize()
    spans = {k: (a, b) for k, a, b in rcv.profile_spans(origin)}
    rcv.profile(False)
    gate_ms = origin.elapsed_time(gate)
    assert spans["master"][1] < gate_ms <= spans["keystream"][0] + 1e-3
    assert torch.equal(R, F)
    # NULL schedule through the C ABI: the next frame of both streams, checked against the oracle
    lib = fhd._lib.load()
    F2 = to_dev(si.gradient_frame(72, 96, 3, t=1, seed=661))
    E2, R2 = torch.empty_like(F2), torch.empty_like(F2)
    H2 = torch.empty(32, dtype=torch.uint8, device=dev())
    arr, n = snd._frames([(sid, F2, E2, H2)])
    assert lib.encrypt_frames_sched(snd._handle(), n, arr, None, None) == fhd.FHD_OK
    arr, n = rcv._frames([(rid, E2, R2, H2)])
    assert lib.decrypt_frames_sched(rcv._handle(), n, arr, None, None) == fhd.FHD_OK
    torch.cuda.synchronize()
    ref = oracle.Stream.from_key(key)
    ref.encrypt(host(F))
    E_ref, H_ref = ref.encrypt(host(F2))
    assert np.array_equal(host(E2), E_ref) and bytes(host(H2)) == H_ref
    assert torch.equal(R2, F2)


@pytest.mark.parametrize("ks,counts", [("trajectory", (7, 5)), ("pairs", (6, 4))])
def test_launch_count_per_call(ks, counts):
    """fhd_launch_count counts every kernel: digest (SHA + fold), LHCS_m, the keystream (trajectory and
    emission, or the worker pairs), and the two permutation passes on encryption; LHCS_m, the keystream
    and the two passes on decryption."""
    fhd.fhd_set_keystream_route(ks)
    try:
        key = si.key(620)
        F = to_dev(si.uniform_frame(40, 56, 3, seed=621))
        snd, rcv = fhd.Cipher(key), fhd.Cipher(key)
        sid, rid = snd.open_stream(), rcv.open_stream()
        E, R = torch.empty_like(F), torch.empty_like(F)
        H = torch.empty(32, dtype=torch.uint8, device=dev())
        l0 = fhd.fhd_launch_count()
        snd.encrypt_frames([(sid, F, E, H)])
        l1 = fhd.fhd_launch_count()
        rcv.decrypt_frames([(rid, E, R, H)])
        l2 = fhd.fhd_launch_count()
        torch.cuda.synchronize()
        assert (l1 - l0, l2 - l1) == counts
        assert torch.equal(R, F)
    finally:
        fhd.fhd_set_keystream_route("trajectory")


def test_sm_partition_matches_single_stream():
    """The SM partition (LHCS_m on its own SMs, the rest on the others; or three ways, the digest stage on
    SMs of its own too) changes where kernels run, not what they compute: a mixed batch encrypted in every
    mode is byte-identical, and all match the oracle."""
    shapes = [(60, 100, 3), (32, 48, 1), (96, 128, 3)]
    key = si.key(630)
    frames = [to_dev(si.gradient_frame(*s, t=t, seed=631)) for t, s in enumerate(shapes)]
    outs = []
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for mode in (1, 0, 2):   # LHCS_m on its own SMs; no partition; LHCS_m and the digest stage on their own
        c = fhd.Cipher(key)
        try:
            c.set_partition(mode)
        except fhd.FhdError as exc:   # a device or driver without green contexts: that mode is not run
            assert exc.code == fhd.FHD_ERR_CUDA and mode, exc
            outs.append(None)
            continue
        sid = c.open_stream()
        chain, bulk = c.partition()
        if mode == 1 and chain:
            assert bulk > chain and (chain + bulk) == sms
        if mode == 2 and chain:
            assert bulk > chain and chain + bulk < sms     # the digest stage's SMs are in neither
        if mode == 0:
            assert (chain, bulk) == (0, 0)
        E = [torch.empty_like(f) for f in frames]
        H = torch.empty((len(frames), 32), dtype=torch.uint8, device=dev())
        s = torch.cuda.Stream()
        c.encrypt_frames([(sid, frames[k], E[k], H[k]) for k in range(len(frames))], stream=s)
        torch.cuda.synchronize()
        outs.append(([host(e) for e in E], host(H)))
    base = outs[1]   # no partition
    for other in (0, 2):
        if outs[other] is None:
            continue
        for k in range(len(frames)):
            assert np.array_equal(base[0][k], outs[other][0][k]), (other, k)
        assert np.array_equal(base[1], outs[other][1])
    with pytest.raises(fhd.FhdError):
        fhd.Cipher(key).set_partition(3)
    ref = oracle.Stream.from_key(key)
    for k in range(len(frames)):
        E_ref, H_ref = ref.encrypt(host(frames[k]))
        assert np.array_equal(base[0][k], E_ref), k


def test_more_than_one_descriptor_group():
    """260 frames of one stream in one call (two groups of at most 256 descriptors): the groups
    reuse the scratch, so each group's LHCS_m must wait for the previous group's keystream; with the
    SM partition they run on different internal streams."""
    key = si.key(640)
    F = 260
    frames = torch.stack([to_dev(si.uniform_frame(8, 16, 3, seed=641 + t)) for t in range(F)])
    snd, rcv = fhd.Cipher(key), fhd.Cipher(key)
    sid, rid = snd.open_stream(), rcv.open_stream()
    E, R = torch.empty_like(frames), torch.empty_like(frames)
    H = torch.empty((F, 32), dtype=torch.uint8, device=dev())
    snd.encrypt_frames([(sid, frames[t], E[t], H[t]) for t in range(F)])
    rcv.decrypt_frames([(rid, E[t], R[t], H[t]) for t in range(F)])
    torch.cuda.synchronize()
    assert torch.equal(R, frames)
    ref = oracle.Stream.from_key(key)
    for t in range(F):
        E_ref, H_ref = ref.encrypt(host(frames[t]))
        if t in (0, 255, 256, 259):
            assert np.array_equal(host(E[t]), E_ref), t
            assert bytes(host(H[t])) == H_ref, t


@pytest.mark.parametrize("layout", ["latency", "throughput"])
@pytest.mark.parametrize("cta", [1, 4, 8])
def test_worker_layouts_match_oracle(layout, cta):
    """Both warp layouts of the worker kernel (six chains per warp with constant lanes, eight with
    selects), with 1, 4 or 8 worker warps per CTA (a CTA's last warps idle when the batch's warp count is
    not a multiple), produce the oracle's bytes, for worker counts that fill and do not fill the last
    warp."""
    shapes = [(40, 56, 3), (24, 40, 1)]
    for n in (5, 8, 32):
        key = si.key(650 + n)
        frames = [to_dev(si.uniform_frame(*s, seed=651 + n + k)) for k, s in enumerate(shapes)]
        c = fhd.Cipher(key, n_workers=n)
        c.set_layout(layout)
        c.set_worker_cta(cta)
        d = fhd.Cipher(key, n_workers=n)
        d.set_layout(layout)
        d.set_worker_cta(cta)
        sid, rid = c.open_stream(), d.open_stream()
        E = [torch.empty_like(f) for f in frames]
        R = [torch.empty_like(f) for f in frames]
        H = torch.empty((len(frames), 32), dtype=torch.uint8, device=dev())
        c.encrypt_frames([(sid, frames[k], E[k], H[k]) for k in range(len(frames))])
        d.decrypt_frames([(rid, E[k], R[k], H[k]) for k in range(len(frames))])
        torch.cuda.synchronize()
        ref = oracle.Stream.from_key(key, n=n)
        for k in range(len(frames)):
            E_ref, H_ref = ref.encrypt(host(frames[k]))
            assert np.array_equal(host(E[k]), E_ref), (layout, n, k)
            assert bytes(host(H[k])) == H_ref
            assert torch.equal(R[k], frames[k])
    with pytest.raises(KeyError):
        c.set_layout("fast")



@pytest.mark.parametrize("mix", [1, 3, 8])
def test_integer_worker_mix_matches_oracle(mix):
    """Worker warps stepping on the integer pipes (cipher_set_int_mix: mix of every 8 warps of the
    eight-chain layout) produce the oracle's bytes, mixed with binary64 warps in one launch or alone, for
    worker counts that fill and do not fill the last warp, at 1, 4 and 8 warps per CTA."""
    shapes = [(40, 56, 3), (24, 40, 1)]
    for n, cta in ((5, 1), (32, 4), (12, 8)):
        key = si.key(670 + n + mix)
        frames = [to_dev(si.uniform_frame(*s, seed=671 + n + k)) for k, s in enumerate(shapes)]
        c, d = fhd.Cipher(key, n_workers=n), fhd.Cipher(key, n_workers=n)
        for x in (c, d):
            x.set_layout("throughput")
            x.set_worker_cta(cta)
            x.set_int_mix(mix)
        sid, rid = c.open_stream(), d.open_stream()
        E = [torch.empty_like(f) for f in frames]
        R = [torch.empty_like(f) for f in frames]
        H = torch.empty((len(frames), 32), dtype=torch.uint8, device=dev())
        for t in range(2):   # two frames per stream: the chaining state after integer-pipe workers
            c.encrypt_frames([(sid, frames[k], E[k], H[k]) for k in range(len(frames))])
            d.decrypt_frames([(rid, E[k], R[k], H[k]) for k in range(len(frames))])
            torch.cuda.synchronize()
            if t == 0:
                ref = oracle.Stream.from_key(key, n=n)
            for k in range(len(frames)):
                E_ref, H_ref = ref.encrypt(host(frames[k]))
                assert np.array_equal(host(E[k]), E_ref), (mix, n, t, k)
                assert bytes(host(H[k])) == H_ref
                assert torch.equal(R[k], frames[k])
    with pytest.raises(fhd.FhdError):
        c.set_int_mix(9)


@pytest.mark.parametrize("smem", [28000, 60000])
def test_worker_smem_cap_matches_oracle(smem):
    """A cap on worker CTAs per SM (dynamic shared memory each worker CTA requests, above the default
    48 KB limit too) changes placement only: the oracle's bytes, both layouts."""
    key = si.key(695)
    frames = [to_dev(si.uniform_frame(40, 56, 3, seed=696)), to_dev(si.uniform_frame(24, 40, 1, seed=697))]
    ref = oracle.Stream.from_key(key, n=12)
    E_ref = [ref.encrypt(host(f)) for f in frames]
    for layout in ("latency", "throughput"):
        c = fhd.Cipher(key, n_workers=12)
        c.set_layout(layout)
        c.set_worker_smem(smem)
        sid = c.open_stream()
        E = [torch.empty_like(f) for f in frames]
        H = torch.empty((len(frames), 32), dtype=torch.uint8, device=dev())
        c.encrypt_frames([(sid, frames[k], E[k], H[k]) for k in range(len(frames))])
        torch.cuda.synchronize()
        for k in range(len(frames)):
            assert np.array_equal(host(E[k]), E_ref[k][0]), (layout, k)
            assert bytes(host(H[k])) == E_ref[k][1]
    with pytest.raises(fhd.FhdError):
        c.set_worker_smem(232449)


def test_integer_worker_mix_full_1080p_frame():
    """One 1080p frame (n = 32: 8 worker warps of 8 chains, about 8,100 RK4 steps each) with every worker
    warp on the integer pipes, and with half of them: the oracle's ciphertext and digest."""
    key = si.key(690)
    F = si.gradient_frame(1080, 1920, 3, t=0, seed=691)
    E_ref, H_ref = oracle.Stream.from_key(key).encrypt(F)
    for mix in (8, 4):
        c = fhd.Cipher(key)
        c.set_layout("throughput")
        c.set_int_mix(mix)
        sid = c.open_stream()
        E, H = c.encrypt(sid, to_dev(F))
        torch.cuda.synchronize()
        assert bytes(host(H)) == H_ref, mix
        assert np.array_equal(host(E), E_ref), mix