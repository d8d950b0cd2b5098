"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

* the 30-frame 1920x1080x3 gradient clip encrypted in one encrypt_frames call
  and decrypted in one decrypt_frames call on two CUDA streams ordered by
  events (the bench's step), with both worker layouts: every frame's digest,
  and the sender's and receiver's chaining state after the clip, against the
  oracle; the full ciphertext of frames 0, 14 and 29 against the oracle's
  bit-matrix confusion; the round trip;
* one 7680x4320x3 frame (the stress size): full ciphertext and digest
  against the oracle, and the round trip."""
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


@pytest.mark.parametrize("layout", ["latency", "throughput"])
def test_clip_1080p_30_frames_one_call(layout):
    """As bench.py runs it: the sender on one CUDA stream records a digests-ready event, the
    receiver on another starts its chaotic stage on it and its inverse permutation on the
    ciphertext event; both worker layouts."""
    key = si.key(0)
    clip = si.clip(30, 1080, 1920, 3, seed=0)
    enc = fhd.Cipher(key)
    enc.set_layout(layout)
    sid = enc.open_stream()
    srcs = [to_dev(f) for f in clip]
    dsts = [torch.empty_like(s) for s in srcs]
    digs = [torch.empty(32, dtype=torch.uint8, device=dev()) for _ in srcs]
    tx, rx = torch.cuda.Stream(), torch.cuda.Stream()
    digests_ready, cipher_ready = torch.cuda.Event(), torch.cuda.Event()
    torch.cuda.synchronize()
    enc.encrypt_frames([(sid, s, d, g) for s, d, g in zip(srcs, dsts, digs)], stream=tx, digest_event=digests_ready)
    cipher_ready.record(tx)
    dec = fhd.Cipher(key)
    dec.set_layout(layout)
    rid = dec.open_stream()
    outs = [torch.empty_like(s) for s in srcs]
    dec.decrypt_frames([(rid, d, o, g) for d, o, g in zip(dsts, outs, digs)], stream=rx,
                       wait_events=[digests_ready], data_events=[cipher_ready])
    torch.cuda.synchronize()
    # oracle: digest + LHCS_m chain for every frame; full frames for a sample
    ref = oracle.Stream.from_key(key)
    for t, F in enumerate(clip):
        H = oracle.frame_digest(F)
        assert bytes(host(digs[t])) == H, t
        if t in (0, 14, 29):
            E_ref, H_ref = ref.encrypt(F)
            assert H_ref == H and np.array_equal(host(dsts[t]), E_ref), t
        else:
            ref.frame_keystream(H, 1080, 1920, 3)      # advances the chain like encrypt does
    st = np.frombuffer(enc.export_state(sid), dtype=np.float64)[:4]
    assert np.array_equal(st, ref.state)
    assert np.array_equal(np.frombuffer(dec.export_state(rid), dtype=np.float64)[:4], ref.state)
    assert all(torch.equal(o, s) for o, s in zip(outs, srcs))


def test_one_8k_frame():
    key = si.key(8)
    F = si.gradient_frame(4320, 7680, 3, t=3, seed=8)
    c = fhd.Cipher(key)
    E, H = c.encrypt(c.open_stream(), to_dev(F))
    E_ref, H_ref = oracle.Stream.from_key(key).encrypt(F)
    assert bytes(host(H)) == H_ref
    assert np.array_equal(host(E), E_ref)
    d = fhd.Cipher(key)
    assert torch.equal(d.decrypt(d.open_stream(), E, H), to_dev(F))
