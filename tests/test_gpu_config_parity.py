"""Bit-exact parity with the CPU oracle at the frame sizes of the batched and served workloads.

* The 64-frame mixed batch (16 each of 640x480, 1280x720, 1920x1080, 3840x2160, RGB; one video stream and
  key per frame; the autotuned strip widths installed) is captured as one CUDA graph per direction and
  replayed twice, then as one persistent round-trip launch in a CUDA graph and replayed twice more, as the
  benchmark does.  Every frame's transmitted digest and ciphertext on all four replays (each replay is the
  next frame of every stream) equal the oracle's: ciphertexts compared by SHA-256 of their bytes for all
  64 frames, byte for byte for one frame of each size; every decrypted frame equals its plaintext.
* The continuous-batching server (8 streams over 1920x1080 / 1280x720 / 640x480 RGB, Poisson arrivals,
  32 workers, 20 GB budget) keeps a copy of every frame it serves; every served digest equals the oracle's,
  and the first, a middle and the last frame of every stream equal the oracle's ciphertext byte for byte
  (the oracle advances the chaining state through the frames in between).

The oracle runs on every host core (spawned processes, one video stream per task)."""
import hashlib

import numpy as np
import pytest
import torch

import oracle_pool
import synth_inputs as si
from gpu_util import dev, host, to_dev

pytestmark = pytest.mark.gpu

fhd = pytest.importorskip("paper_2505_07158_gb300")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_07158_gb300 import autotune, batching, serving  # noqa: E402

MIXED = [(480, 640, 3), (720, 1280, 3), (1080, 1920, 3), (2160, 3840, 3)]
SERVE = [(1080, 1920, 3), (720, 1280, 3), (480, 640, 3)]


def _sha(t: torch.Tensor) -> bytes:
    return hashlib.sha256(host(t).tobytes()).digest()


def test_mixed64_graph_replays_match_oracle_at_full_sizes():
    shapes = [s for s in MIXED for _ in range(16)]
    recipes = [("gradient", s, k, 11) for k, s in enumerate(shapes)]
    keys = [si.key(1000 + k) for k in range(len(shapes))]
    full = {16 * q for q in range(4)}                     # the first frame of each size, compared in full
    jobs = [oracle_pool.pool().submit(oracle_pool.stream_job, keys[k], [recipes[k]] * 4,
                                      {0, 1, 2, 3} if k in full else set())
            for k in range(len(shapes))]
    autotune.tune(MIXED)
    frames = [to_dev(si.gradient_frame(*s, t=k, seed=11)) for k, s in enumerate(shapes)]
    enc = fhd.Cipher(keys[0], n_workers=32)
    enc_items, dec_items, dec = batching.mixed_batch(shapes, keys, enc, frames, dev())
    g_enc = batching.GraphedCall(enc, enc_items, encrypt=True)
    g_dec = batching.GraphedCall(dec, dec_items, encrypt=False)
    persistent = None
    got = []
    for rep in range(4):
        if rep < 2:      # the seven-kernel batched calls, one graph per direction
            g_enc.replay()
            g_dec.replay()
        else:            # the persistent round trip (one launch), captured in a graph
            if persistent is None:
                persistent = batching.PersistentRoundTrip(enc, dec, enc_items, dec_items, graph=True)
            persistent.replay()
        torch.cuda.synchronize()
        rec = []
        for k, (sid, F, E, H) in enumerate(enc_items):
            assert torch.equal(dec_items[k][2], F), (rep, k)
            rec.append((bytes(host(H)), _sha(E), host(E) if k in full else None))
        got.append(rec)
    enc.sync_status()
    dec.sync_status()
    for k, job in enumerate(jobs):
        ref = job.result()
        for rep in range(4):
            H_ref, sha_ref, E_ref = ref[rep]
            H, sha, E = got[rep][k]
            assert H == H_ref, (rep, k, shapes[k])
            if E_ref is not None:
                assert np.array_equal(E, E_ref), (rep, k, shapes[k], int(np.count_nonzero(E != E_ref)))
            assert sha == sha_ref, (rep, k, shapes[k])
    enc.close()
    dec.close()


def test_served_frames_match_oracle_at_serving_sizes():
    nstreams = 8
    shapes = [SERVE[s % 3] for s in range(nstreams)]
    keys = [si.key(5000 + s) for s in range(nstreams)]
    pool = {s: [to_dev(si.gradient_frame(*s, t=t, seed=5)) for t in range(4)] for s in SERVE}
    stats, srv = serving.run(keys, shapes, pool, fps=30.0, duration=0.6, seed=17, n_workers=32,
                             budget_bytes=20 << 30, keep=True)
    srv.close()
    assert stats["completed_frames"] == stats["offered_frames"] > 0
    jobs = {}
    for s in range(nstreams):
        seqs = sorted(q for (st, q) in srv.kept if st == s)
        assert seqs == list(range(len(seqs)))
        if not seqs:
            continue
        sample = {0, len(seqs) // 2, len(seqs) - 1}
        # the server's source of frame q of stream s: pool[shape][(7 s + q) % 4] (gradient frame t of seed 5)
        recipes = [("gradient", shapes[s], (7 * s + q) % 4, 5) for q in seqs]
        jobs[s] = (oracle_pool.pool().submit(oracle_pool.stream_job, keys[s], recipes, sample, sample), sample)
    checked = 0
    for s, (job, sample) in jobs.items():
        ref = job.result()
        for q, (H_ref, _, E_ref) in ref.items():
            E, H = srv.kept[(s, q)]
            assert bytes(host(H)) == H_ref, (s, q)
            if q in sample:
                assert np.array_equal(host(E), E_ref), (s, q, shapes[s])
                checked += 1
    assert checked >= 2 * nstreams
