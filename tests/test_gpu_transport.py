"""Masked digest transport (an option of this library: Sec. V sends the frame hashes encrypted without
giving the mechanism), GPU against the oracle.

Encryption writes H xor M, M = SHA-256("FHDMASK1" || LE64 bits of the chaining state before the frame and of
gamma); decryption unmasks with its own chaining state and leaves H in the digest buffer.  Checked bit for
bit: chained frames of two streams in one batch, the tree digest combined with the mask, the split
sender/receiver schedule (digests_done then follows LHCS_m, which writes the masked digest), and the
receiver-side check after decryption."""
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


@pytest.mark.parametrize("digest_mode", ["xor", "tree"])
def test_masked_transport_batch_matches_oracle(digest_mode):
    keys = [si.key(720), si.key(721)]
    shapes = [(64, 96, 3), (64, 96, 3), (40, 56, 3)]
    enc = fhd.Cipher(keys[0], digest_mode=digest_mode, digest_transport="masked")
    dec = fhd.Cipher(keys[0], digest_mode=digest_mode, digest_transport="masked")
    sids = [enc.open_stream(), enc.open_stream(keys[1])]
    rids = [dec.open_stream(), dec.open_stream(keys[1])]
    refs = [oracle.Stream.from_key(k, digest_mode=digest_mode, transport="masked") for k in keys]
    plain = [oracle.Stream.from_key(k, digest_mode=digest_mode) for k in keys]
    for t, sh in enumerate(shapes):
        F = [to_dev(si.gradient_frame(*sh, t=t, seed=722 + q)) for q in range(2)]
        E = [torch.empty_like(f) for f in F]
        R = [torch.empty_like(f) for f in F]
        H = torch.empty((2, 32), dtype=torch.uint8, device=dev())
        enc.encrypt_frames([(sids[q], F[q], E[q], H[q]) for q in range(2)])
        torch.cuda.synchronize()
        Htx = host(H).copy()
        dec.decrypt_frames([(rids[q], E[q], R[q], H[q]) for q in range(2)])
        torch.cuda.synchronize()
        for q in range(2):
            E_ref, Htx_ref = refs[q].encrypt(host(F[q]))
            _, H_ref = plain[q].encrypt(host(F[q]))
            assert np.array_equal(host(E[q]), E_ref), (t, q)
            assert bytes(Htx[q]) == Htx_ref != H_ref
            assert bytes(host(H)[q]) == H_ref             # the receiver left the unmasked digest
            assert torch.equal(R[q], F[q])
        ok = dec.verify_frames([(rids[q], E[q], R[q], H[q]) for q in range(2)])
        assert host(ok).tolist() == [1, 1]


def test_masked_digest_event_follows_lhcs_m():
    """encrypt_frames_split in masked mode records digests_done after LHCS_m (which writes H xor M); a
    receiver gated on it decrypts correctly while the sender's keystream and permutation still run."""
    key = si.key(730)
    frames = [to_dev(si.gradient_frame(96, 128, 3, t=t, seed=731)) for t in range(2)]
    snd = fhd.Cipher(key, digest_transport="masked")
    rcv = fhd.Cipher(key, digest_transport="masked")
    sid, rid = snd.open_stream(), rcv.open_stream()
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    E = [torch.empty_like(f) for f in frames]
    R = [torch.empty_like(f) for f in frames]
    H = torch.empty((2, 32), dtype=torch.uint8, device=dev())
    ready, data = torch.cuda.Event(), torch.cuda.Event()
    torch.cuda.synchronize()
    snd.encrypt_frames([(sid, frames[k], E[k], H[k]) for k in range(2)], stream=sa, digest_event=ready,
                       keystream_event=torch.cuda.Event())
    data.record(sa)
    rcv.decrypt_frames([(rid, E[k], R[k], H[k]) for k in range(2)], stream=sb, wait_events=[ready],
                       data_events=[data])
    torch.cuda.synchronize()
    for k in range(2):
        assert torch.equal(R[k], frames[k]), k


def test_unknown_transport_is_rejected():
    lib = fhd._lib.load()
    p = fhd._lib._params()
    p.digest_transport = 5
    h = ctypes.c_void_p()
    assert lib.cipher_init(bytes(32), ctypes.byref(p), ctypes.byref(h)) == fhd.FHD_ERR_INVALID_ARG
    assert b"digest_transport" in lib.cipher_last_error(None)
