"""The one-trajectory keystream route (Sec. II-B, Algorithm 2) on the GPU, bit-exact against the oracle.

Worker pair i starts from LHCS_m's iterates IR[2i] and IR[2i+1] and iterates the same map, so the route
computes each frame's trajectory once and copies each worker's window of it into D and B.  These tests take
IR from the oracle's LHCS_m (so it is one trajectory) and compare D and B element by element with the
oracle's Algorithm 2, over shapes with one worker, the maximum worker count, slices shorter than a 16-byte
chunk, a B buffer at an odd address and a full 1080p frame; then whole batches of mixed shapes and streams
through encrypt_frames / decrypt_frames under both routes."""
import numpy as np
import pytest
import torch

import oracle
import synth_inputs as si
from gpu_util import dev, host, host_u16, to_dev

pytestmark = pytest.mark.gpu

fhd = pytest.importorskip("paper_2505_07158_gb300")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture
def route():
    """Set the process-wide keystream route for one test and restore the default afterwards."""
    yield fhd.fhd_set_keystream_route
    fhd.fhd_set_keystream_route("trajectory")


def _master_ir(n, seed):
    g = si.rng(seed)
    v = [float(g.uniform(0, 20)), float(g.uniform(0, 20)), float(g.uniform(0, 40)), float(g.uniform(0, 20))]
    gamma = float(g.uniform(-1.52, -0.06))
    H = g.integers(0, 256, size=32, dtype=np.uint8).tobytes()
    IR, _ = oracle.master(v, H, gamma, n=n)
    return np.ascontiguousarray(IR), gamma


@pytest.mark.parametrize("h,w,C,n", [(1, 1, 1, 1), (3, 5, 3, 2), (8, 8, 3, 32), (17, 23, 3, 6), (64, 96, 3, 32),
                                     (256, 256, 3, 32), (37, 53, 4, 12), (2, 2, 1, 40), (1, 16, 3, 1024),
                                     (5, 7, 3, 1024), (40, 56, 3, 1), (1080, 1920, 3, 32)])
def test_keystream_trajectory_matches_oracle(h, w, C, n):
    IR, gamma = _master_ir(n, h * w + n)
    D_ref, B_ref = oracle.keystream(IR, gamma, h, w, C, n)
    D, B = fhd.fhd_keystream(to_dev(IR), gamma, h, w, C, n_workers=n, trajectory=True)
    assert np.array_equal(host_u16(D), D_ref)
    assert np.array_equal(host(B), B_ref)


@pytest.mark.parametrize("offset", [1, 3, 8, 15])
def test_keystream_trajectory_unaligned_B(offset):
    """B at an address that is not a multiple of 16: every chunk is written byte by byte."""
    h, w, C, n = 30, 50, 3, 32
    IR, gamma = _master_ir(n, 7 + offset)
    D_ref, B_ref = oracle.keystream(IR, gamma, h, w, C, n)
    buf = torch.full((h * w * C + 32,), 0xA5, dtype=torch.uint8, device=dev())
    D, B = fhd.fhd_keystream(to_dev(IR), gamma, h, w, C, n_workers=n, trajectory=True,
                             B_out=buf[offset:offset + h * w * C])
    assert np.array_equal(host_u16(D), D_ref)
    out = host(buf)
    assert np.array_equal(out[offset:offset + h * w * C], B_ref)
    assert (out[:offset] == 0xA5).all() and (out[offset + h * w * C:] == 0xA5).all()   # nothing outside B


def test_keystream_trajectory_equals_pairs_on_lhcs_iterates():
    """The two routes agree on IR written by the GPU's own LHCS_m (fhd_master)."""
    n, h, w, C = 32, 120, 200, 3
    g = si.rng(5)
    st = to_dev(np.array([3.0, 4.0, 17.0, 9.0, -0.9], np.float64))
    IR = fhd.fhd_master(st, to_dev(g.integers(0, 256, size=32, dtype=np.uint8)), n_workers=n)
    D0, B0 = fhd.fhd_keystream(IR, -0.9, h, w, C, n_workers=n)
    D1, B1 = fhd.fhd_keystream(IR, -0.9, h, w, C, n_workers=n, trajectory=True)
    assert torch.equal(D0, D1) and torch.equal(B0, B1)


@pytest.mark.parametrize("ks", ["trajectory", "pairs"])
def test_batches_of_mixed_shapes_and_streams_under_both_routes(route, ks):
    """Thirteen frames of three streams and five shapes in one call (three trajectory warps, whose frames need
    different numbers of records), then their decryption; ciphertexts and digests equal the oracle's."""
    route(ks)
    shapes = [(48, 64, 3), (30, 50, 3), (64, 64, 1), (20, 36, 4), (1, 16, 3), (48, 64, 3), (30, 50, 3),
              (120, 160, 3), (64, 64, 1), (20, 36, 4), (1, 16, 3), (48, 64, 3), (30, 50, 3)]
    keys = [si.key(60 + k) for k in range(3)]
    owner = [k % 3 for k in range(len(shapes))]
    frames = [si.uniform_frame(*s, seed=80 + k) for k, s in enumerate(shapes)]
    enc, dec = fhd.Cipher(si.key(1)), fhd.Cipher(si.key(1))
    sids = [enc.open_stream(k) for k in keys]
    rids = [dec.open_stream(k) for k in keys]
    srcs = [to_dev(f) for f in frames]
    outs = [torch.empty_like(s) for s in srcs]
    digs = [torch.empty(32, dtype=torch.uint8, device=dev()) for _ in srcs]
    enc.encrypt_frames([(sids[o], s, e, d) for o, s, e, d in zip(owner, srcs, outs, digs)])
    refs = [oracle.Stream.from_key(k) for k in keys]
    for f, o, e, d in zip(frames, owner, outs, digs):
        E_ref, H_ref = refs[o].encrypt(f)
        assert np.array_equal(host(e), E_ref) and bytes(host(d)) == H_ref
    back = [torch.empty_like(s) for s in srcs]
    dec.decrypt_frames([(rids[o], e, b, d) for o, e, b, d in zip(owner, outs, back, digs)])
    for f, b in zip(frames, back):
        assert np.array_equal(host(b), f)


def test_full_clip_frame_under_both_routes(route):
    """A chained 1080p stream, three frames per call: the routes give the same ciphertexts and digests, and the
    first two frames equal the oracle's."""
    key = si.key(4)
    clip = si.clip(3, 1080, 1920, 3, seed=4)
    got = {}
    for ks in ("pairs", "trajectory"):
        route(ks)
        c = fhd.Cipher(key)
        sid = c.open_stream()
        srcs = [to_dev(clip[t]) for t in range(3)]
        outs = [torch.empty_like(s) for s in srcs]
        digs = [torch.empty(32, dtype=torch.uint8, device=dev()) for _ in srcs]
        c.encrypt_frames([(sid, s, e, d) for s, e, d in zip(srcs, outs, digs)])
        got[ks] = [(host(e), bytes(host(d))) for e, d in zip(outs, digs)]
    for (ea, da), (eb, db) in zip(got["pairs"], got["trajectory"]):
        assert np.array_equal(ea, eb) and da == db
    ref = oracle.Stream.from_key(key)
    for t in range(2):
        E_ref, H_ref = ref.encrypt(clip[t])
        assert np.array_equal(got["trajectory"][t][0], E_ref) and got["trajectory"][t][1] == H_ref
