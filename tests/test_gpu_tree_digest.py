"""The tree digest option (an option of this library, not of the paper), GPU against the oracle.

In tree mode H = SHA-256(h_1 || ... || h_n), the n sub-frame digests concatenated in order, instead of the
paper's XOR fold (Sec. II-A).  Checked bit for bit against the oracle: the standalone digest entry point
(n even and odd, so the 32 n digest bytes end on a whole or a half SHA-256 block), whole chained frames
through encrypt_frames, the receiver-side check in each mode, and the flat frame whose fold cancels."""
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


@pytest.mark.parametrize("nbytes,n,count", [(0, 1, 1), (1, 1, 2), (64, 1, 1), (300, 3, 3), (1000, 32, 2),
                                            (12345, 33, 2), (196608, 32, 2), (6220800, 32, 1), (921600, 1024, 1)])
def test_tree_frame_digest(nbytes, n, count):
    data = si.rng(nbytes + 7 * n).integers(0, 256, size=nbytes * count, dtype=np.uint8)
    got = host(fhd.fhd_frame_digest(to_dev(data), n=n, count=count, mode="tree"))
    for k in range(count):
        assert bytes(got[k]) == oracle.frame_digest(data[k * nbytes:(k + 1) * nbytes], n, "tree"), k


def test_flat_frame_digest_cancels_only_in_xor_mode():
    f = np.full((16, 16, 3), 77, np.uint8)
    xor = bytes(host(fhd.fhd_frame_digest(to_dev(f), n=8))[0])
    tree = bytes(host(fhd.fhd_frame_digest(to_dev(f), n=8, mode="tree"))[0])
    assert xor == bytes(32)
    assert tree == oracle.frame_digest(f, 8, "tree") != bytes(32)


@pytest.mark.parametrize("n", [32, 5])
def test_tree_mode_cipher_matches_oracle_and_verifies(n):
    """Three chained frames of one stream encrypted in tree mode: ciphertexts and digests equal the
    oracle's in tree mode; decryption (which takes H as given) restores the frames; the receiver-side
    check passes in tree mode and fails in XOR mode, whose recomputed H differs."""
    key = si.key(700 + n)
    shapes = [(96, 128, 3), (96, 128, 3), (61, 77, 3)]
    frames = [to_dev(si.gradient_frame(*sh, t=t, seed=701)) for t, sh in enumerate(shapes)]
    enc = fhd.Cipher(key, n_workers=n, digest_mode="tree")
    dec = fhd.Cipher(key, n_workers=n, digest_mode="tree")
    plain = fhd.Cipher(key, n_workers=n)
    sid, rid = enc.open_stream(), dec.open_stream()
    ref = oracle.Stream.from_key(key, n=n, digest_mode="tree")
    for k, F in enumerate(frames):
        E = torch.empty_like(F)
        H = torch.empty(32, dtype=torch.uint8, device=dev())
        enc.encrypt_frames([(sid, F, E, H)])
        R = torch.empty_like(F)
        dec.decrypt_frames([(rid, E, R, H)])
        torch.cuda.synchronize()
        E_ref, H_ref = ref.encrypt(host(F))
        assert np.array_equal(host(E), E_ref), k
        assert bytes(host(H)) == H_ref
        assert torch.equal(R, F), k
        assert int(host(dec.verify_frames([(rid, E, R, H)]))[0]) == 1
        assert int(host(plain.verify_frames([(plain.open_stream(), E, R, H)]))[0]) == 0


def test_unknown_digest_mode_is_rejected():
    import ctypes
    lib = fhd._lib.load()
    p = fhd._lib._params()
    p.digest_mode = 7
    h = ctypes.c_void_p()
    assert lib.cipher_init(bytes(32), ctypes.byref(p), ctypes.byref(h)) == fhd.FHD_ERR_INVALID_ARG
    assert b"digest_mode" in lib.cipher_last_error(None)
