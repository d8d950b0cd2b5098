"""Batched launches of mixed-resolution frames, captured into a CUDA graph.

One ``encrypt_frames`` / ``decrypt_frames`` call already covers every frame
of a batch -- frames of different streams and resolutions -- with one launch
per step of the cipher (sub-frame SHA-256, LHCS_m, worker keystream, fused
confusion + XOR), each launch walking a per-frame descriptor table.
:class:`GraphedCall` captures such a call once and replays it: the
descriptors (buffer pointers, shapes, strip widths chosen by the autotuner)
are baked into the graph, the caller refreshes the buffers' contents between
replays, and each replay advances the chaining state of every stream in the
batch exactly like a direct call would.
"""
from __future__ import annotations

from typing import Sequence

import torch

from . import _lib


class GraphedCall:
    """A fixed batch of frames (``(stream_id, src, dst, digest)`` tuples) as a CUDA graph."""

    def __init__(self, cipher: "_lib.Cipher", items: Sequence, encrypt: bool = True,
                 stream: torch.cuda.Stream | None = None):
        self.cipher = cipher
        self.items = list(items)
        self.encrypt = encrypt
        self.stream = stream or torch.cuda.Stream()
        fn = cipher.encrypt_frames if encrypt else cipher.decrypt_frames
        sids = sorted({it[0] for it in self.items})
        # One uncaptured run sizes the scratch of this CUDA stream; the chaining
        # state it advances is put back so the first replay is the first call.
        saved = {sid: cipher.export_state(sid) for sid in sids}
        torch.cuda.synchronize()
        fn(self.items, stream=self.stream)
        self.stream.synchronize()
        for sid, st in saved.items():
            cipher.import_state(sid, st)
        self.graph = torch.cuda.CUDAGraph()
        l0 = _lib.fhd_launch_count()
        with torch.cuda.graph(self.graph, stream=self.stream):
            fn(self.items, stream=self.stream)
        torch.cuda.synchronize()
        # the library counts the kernels it launches, captured ones included
        self.kernels_per_replay = _lib.fhd_launch_count() - l0

    def replay(self):
        self.graph.replay()


def mixed_batch(shapes: Sequence[tuple], keys: Sequence[bytes], cipher: "_lib.Cipher", frames,
                device=None):
    """Open one stream per frame (own key) and allocate outputs: -> (enc_items, dec_items, decrypt cipher)."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    dec = _lib.Cipher(keys[0], n_workers=cipher.n_workers, digest_mode=cipher.digest_mode,
                      digest_transport=cipher.digest_transport)
    enc_items, dec_items = [], []
    for shape, key, F in zip(shapes, keys, frames):
        sid = cipher.open_stream(key)
        rid = dec.open_stream(key)
        E = torch.empty_like(F)
        R = torch.empty_like(F)
        H = torch.empty(32, dtype=torch.uint8, device=device)
        enc_items.append((sid, F, E, H))
        dec_items.append((rid, E, R, H))
    return enc_items, dec_items, dec


class PersistentRoundTrip:
    """A fixed mixed batch encrypted by ``sender`` and decrypted by ``receiver`` in ONE persistent kernel
    launch per replay (``cipher_round_trip_persistent``), optionally captured in a CUDA graph.

    ``enc_items`` are ``(stream_id, src, dst, digest)`` of the sender; ``dec_items`` the receiver's, frame k
    being the ciphertext and digest of enc_items[k].  The uncaptured first call sizes the handles' scratch and
    the launch's counters; the chaining states it advanced are put back, so the first replay is the first
    call."""

    def __init__(self, sender: "_lib.Cipher", receiver: "_lib.Cipher", enc_items: Sequence, dec_items: Sequence,
                 stream: torch.cuda.Stream | None = None, graph: bool = True):
        self.sender, self.receiver = sender, receiver
        self.enc_items, self.dec_items = list(enc_items), list(dec_items)
        self.stream = stream or torch.cuda.Stream()
        saved = [(c, sid, c.export_state(sid)) for c, items in ((sender, self.enc_items), (receiver, self.dec_items))
                 for sid in sorted({it[0] for it in items})]
        torch.cuda.synchronize()
        self._call()
        self.stream.synchronize()
        for c, sid, st in saved:
            c.import_state(sid, st)
        self.graph = None
        if graph:
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=self.stream):
                self._call()
            torch.cuda.synchronize()
        self.kernels_per_replay = 1

    def _call(self):
        self.sender.round_trip_persistent(self.receiver, self.enc_items, self.dec_items, stream=self.stream)

    def replay(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            with torch.cuda.stream(self.stream):
                self._call()
