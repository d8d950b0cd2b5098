"""ctypes binding of ``libfhdcipher.so`` (argument marshalling only).

Every entry point of ``include/fhdcipher.h`` is exposed under the same name.
Tensors are CUDA ``torch.uint8`` (frames, digests, B), ``torch.uint16``-sized
``torch.int16`` (D) or ``torch.float64`` (states, iterates); their device
pointers are handed to the library, which enqueues its kernels on the current
torch CUDA stream (or the stream given).  There is no CPU path: if the
library cannot be loaded the import of this module raises."""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Iterable, Sequence

import torch

from . import build as _build

FHD_OK = 0
FHD_ERR_INVALID_ARG = -1
FHD_ERR_OOM = -2
FHD_ERR_BAD_STREAM = -3
FHD_ERR_TIMEOUT = -5
FHD_ERR_CUDA = -6
FHD_ERR_STATE = -7
FHD_ERR_TOO_LARGE = -8
FHD_STATE_BYTES = 48

# Every symbol the header declares (checked by the CPU test-suite).
EXPORTS = (
    "cipher_init", "cipher_init_raw", "cipher_open_stream", "cipher_open_stream_key", "cipher_close_stream",
    "encrypt_frames", "decrypt_frames", "cipher_export_state", "cipher_import_state", "cipher_sync_status",
    "cipher_last_error", "cipher_destroy", "fhd_frame_digest", "fhd_master", "fhd_keystream",
    "fhd_permute_encrypt", "fhd_permute_decrypt", "fhd_strip_width", "fhd_set_strip_width", "fhd_version",
    "cipher_profile", "cipher_profile_read", "fhd_launch_count", "encrypt_frames_ex", "decrypt_frames_ex",
    "cipher_reserve", "fhd_frame_scratch_bytes", "fhd_frame_digest_noalloc", "cipher_verify_frames",
    "decrypt_frames_split", "encrypt_frames_split", "cipher_profile_spans", "cipher_set_partition",
    "cipher_get_partition", "cipher_set_layout", "fhd_stats_histogram", "fhd_stats_npcr_uaci",
    "fhd_stats_correlation", "fhd_stats_local_entropy", "encrypt_frames_sched", "decrypt_frames_sched",
    "fhd_frame_digest_tree", "fhd_fp64_probe", "fhd_set_encrypt_route", "encrypt_frames_persistent",
    "decrypt_frames_persistent", "cipher_round_trip_persistent", "cipher_set_persistent_limits",
    "cipher_set_worker_cta", "cipher_persistent_trace", "fhd_row_band", "fhd_set_row_band", "fhd_build_flags",
    "fhd_bounds_report", "fhd_bounds_site_name", "fhd_bounds_selftest", "cipher_set_int_mix", "fhd_binary64_check",
    "cipher_set_worker_smem", "fhd_set_cta_threads", "fhd_cta_threads", "fhd_set_keystream_route",
    "fhd_keystream_trajectory",
)
FHD_BUILD_BOUNDS_CHECK = 1
KERNEL_KINDS = ("sha", "master", "keystream", "encrypt", "decrypt")


class FhdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fhdcipher error {code}: {msg}")
        self.code = code


class FhdParams(ctypes.Structure):
    _fields_ = [("n_workers", ctypes.c_uint32), ("rk4_h", ctypes.c_double), ("u_bound", ctypes.c_uint32 * 4),
                ("digest_mode", ctypes.c_uint32), ("digest_transport", ctypes.c_uint32)]


# How the frame digest H is formed from the n sub-frame digests: "xor" is the paper's fold (Sec. II-A),
# "tree" (an option of this library) is SHA-256 of the sub-frame digests concatenated in order.
DIGEST_MODES = {"xor": 0, "tree": 1}
# How the digest travels: "plain" as computed, or "masked" (an option of this library) as H xor M with M
# derived from the stream's chaining state; the receiver unmasks it in place.
TRANSPORTS = {"plain": 0, "masked": 1}


class FhdFrame(ctypes.Structure):
    _fields_ = [("stream_id", ctypes.c_uint32), ("height", ctypes.c_uint32), ("width", ctypes.c_uint32),
                ("channels", ctypes.c_uint32), ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p),
                ("digest", ctypes.c_void_p)]


class FhdSchedule(ctypes.Structure):
    """``fhd_schedule``: the ordering hooks of one call (event lists and output events)."""
    _fields_ = [("key_waits", ctypes.c_void_p), ("n_key_waits", ctypes.c_uint32),
                ("worker_waits", ctypes.c_void_p), ("n_worker_waits", ctypes.c_uint32),
                ("data_events", ctypes.c_void_p), ("n_data", ctypes.c_uint32),
                ("digests_done", ctypes.c_void_p), ("master_done", ctypes.c_void_p),
                ("keystream_done", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None


def checked_requested() -> bool:
    """True when FHD_CHECKED=1 asks for the checked build (range checks of every computed index)."""
    return os.environ.get("FHD_CHECKED", "0") not in ("", "0")


def load(path: str | None = None) -> ctypes.CDLL:
    """Load (building first if needed) the in-tree library: the checked build when FHD_CHECKED=1."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(path or _build.build(checked=checked_requested()))
        P, u32, u64, dbl, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
        PP = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "cipher_init": (i32, [P, P, PP]),
            "cipher_init_raw": (i32, [dbl, dbl, dbl, dbl, dbl, P, PP]),
            "cipher_open_stream": (i32, [P, ctypes.POINTER(u32)]),
            "cipher_open_stream_key": (i32, [P, P, ctypes.POINTER(u32)]),
            "cipher_close_stream": (i32, [P, u32]),
            "encrypt_frames": (i32, [P, u32, P, P]),
            "decrypt_frames": (i32, [P, u32, P, P]),
            "cipher_export_state": (i32, [P, u32, P, ctypes.c_size_t]),
            "cipher_import_state": (i32, [P, u32, P, ctypes.c_size_t]),
            "cipher_sync_status": (i32, [P, P]),
            "cipher_last_error": (ctypes.c_char_p, [P]),
            "cipher_destroy": (None, [P]),
            "fhd_frame_digest": (i32, [P, u64, u32, u32, P, P]),
            "fhd_frame_digest_noalloc": (i32, [P, u64, u32, u32, P, P]),
            "fhd_frame_digest_tree": (i32, [P, u64, u32, u32, P, P]),
            "fhd_master": (i32, [P, P, P, P, P]),
            "fhd_keystream": (i32, [P, dbl, P, u32, u32, u32, P, P, P]),
            "fhd_keystream_trajectory": (i32, [P, dbl, P, u32, u32, u32, P, P, P]),
            "fhd_permute_encrypt": (i32, [P, P, u32, u32, u32, P, P, P]),
            "fhd_permute_decrypt": (i32, [P, P, u32, u32, u32, P, P, P]),
            "fhd_strip_width": (u32, [u32, u32, u32]),
            "fhd_set_strip_width": (i32, [u32, u32, u32, u32]),
            "fhd_row_band": (u32, [u32, u32, u32]),
            "fhd_set_row_band": (i32, [u32, u32, u32, u32]),
            "fhd_set_cta_threads": (i32, [u32, u32, u32, u32, u32]),
            "fhd_cta_threads": (i32, [u32, u32, u32, ctypes.POINTER(u32), ctypes.POINTER(u32)]),
            "fhd_version": (ctypes.c_char_p, []),
            "cipher_profile": (i32, [P, i32]),
            "cipher_profile_read": (i32, [P, P, P]),
            "fhd_launch_count": (ctypes.c_uint64, []),
            "encrypt_frames_ex": (i32, [P, u32, P, P, P, u32, P]),
            "decrypt_frames_ex": (i32, [P, u32, P, P, P, u32, P]),
            "decrypt_frames_split": (i32, [P, u32, P, P, P, u32, P, u32, P, P]),
            "encrypt_frames_split": (i32, [P, u32, P, P, P, u32, P, P, P]),
            "encrypt_frames_sched": (i32, [P, u32, P, P, P]),
            "decrypt_frames_sched": (i32, [P, u32, P, P, P]),
            "cipher_profile_spans": (i32, [P, P, u32, P, P, P, P]),
            "cipher_set_partition": (i32, [P, i32]),
            "cipher_get_partition": (i32, [P, P, P]),
            "cipher_set_layout": (i32, [P, i32]),
            "fhd_stats_histogram": (i32, [P, u32, u32, u32, u32, P, P, P]),
            "fhd_stats_npcr_uaci": (i32, [P, P, u32, u32, u32, u32, P, P, P]),
            "fhd_stats_correlation": (i32, [P, u32, u32, u32, u32, P, u32, P, P, P, P]),
            "fhd_stats_local_entropy": (i32, [P, u32, u32, u32, u32, P, u32, u32, P, P, P]),
            "cipher_reserve": (i32, [P, P, u64]),
            "cipher_verify_frames": (i32, [P, u32, P, P, P]),
            "fhd_frame_scratch_bytes": (u64, [u32, u32, u32, u32]),
            "fhd_fp64_probe": (i32, [u32, u32, P, ctypes.POINTER(u64), P]),
            "fhd_set_encrypt_route": (i32, [i32]),
            "fhd_set_keystream_route": (i32, [i32]),
            "encrypt_frames_persistent": (i32, [P, u32, P, P]),
            "decrypt_frames_persistent": (i32, [P, u32, P, P]),
            "cipher_round_trip_persistent": (i32, [P, P, u32, P, P, P]),
            "cipher_set_persistent_limits": (i32, [P, u64, i32]),
            "cipher_set_worker_cta": (i32, [P, u32]),
            "cipher_persistent_trace": (i32, [P, u32, P]),
            "fhd_build_flags": (u32, []),
            "cipher_set_int_mix": (i32, [P, u32]),
            "cipher_set_worker_smem": (i32, [P, u32]),
            "fhd_binary64_check": (i32, [u64, u64, P, P]),
            "fhd_bounds_report": (i32, [ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u64),
                                        ctypes.POINTER(u64)]),
            "fhd_bounds_site_name": (ctypes.c_char_p, [u32]),
            "fhd_bounds_selftest": (i32, [ctypes.POINTER(u32), ctypes.POINTER(u32), P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def library_path() -> str:
    return _build.CHECKED_LIB if checked_requested() else _build.LIB


def _check(code: int, handle=None):
    if code != FHD_OK:
        msg = load().cipher_last_error(handle).decode(errors="replace")
        raise FhdError(code, msg)


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _params(n_workers=32, rk4_h=0.01, u_bound=(20, 20, 40, 20), digest_mode="xor", transport="plain") -> FhdParams:
    p = FhdParams()
    p.n_workers = n_workers
    p.rk4_h = rk4_h
    for m in range(4):
        p.u_bound[m] = u_bound[m]
    p.digest_mode = DIGEST_MODES[digest_mode]
    p.digest_transport = TRANSPORTS[transport]
    return p


def _frame_tensor(t: torch.Tensor, what: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.uint8 or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous CUDA uint8 tensor")
    if t.dim() != 3:
        raise ValueError(f"{what} must have shape (height, width, channels)")
    return t


def _digest_tensor(t: torch.Tensor):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.uint8 or not t.is_contiguous() or t.numel() != 32:
        raise ValueError("digest must be a contiguous CUDA uint8 tensor of 32 bytes")
    return t


class Cipher:
    """A cipher handle: key, protocol parameters and device-resident streams."""

    def __init__(self, key: bytes | None = None, ic: Sequence[float] | None = None, n_workers: int = 32,
                 rk4_h: float = 0.01, u_bound=(20, 20, 40, 20), digest_mode: str = "xor",
                 digest_transport: str = "plain"):
        lib = load()
        self.params = _params(n_workers, rk4_h, u_bound, digest_mode, digest_transport)
        self.digest_mode = digest_mode
        self.digest_transport = digest_transport
        self.n_workers = n_workers
        h = ctypes.c_void_p()
        if ic is not None:
            x0, y0, z0, w0, g = (float(v) for v in ic)
            code = lib.cipher_init_raw(x0, y0, z0, w0, g, ctypes.byref(self.params), ctypes.byref(h))
        else:
            if key is None or len(key) != 32:
                raise ValueError("key must be 32 bytes (or pass ic=)")
            kb = (ctypes.c_uint8 * 32).from_buffer_copy(bytes(key))
            code = lib.cipher_init(kb, ctypes.byref(self.params), ctypes.byref(h))
        _check(code)
        self._h = h

    def _handle(self):
        if self._h is None:
            raise RuntimeError("cipher closed")
        return self._h

    def open_stream(self, key: bytes | None = None) -> int:
        sid = ctypes.c_uint32()
        if key is None:
            code = load().cipher_open_stream(self._handle(), ctypes.byref(sid))
        else:
            kb = (ctypes.c_uint8 * 32).from_buffer_copy(bytes(key))
            code = load().cipher_open_stream_key(self._handle(), kb, ctypes.byref(sid))
        _check(code, self._h)
        return sid.value

    def close_stream(self, sid: int):
        _check(load().cipher_close_stream(self._handle(), sid), self._h)

    @staticmethod
    def _frames(items) -> ctypes.Array:
        items = list(items)
        arr = (FhdFrame * max(len(items), 1))()
        for k, (sid, src, dst, digest) in enumerate(items):
            _frame_tensor(src, "src")
            _frame_tensor(dst, "dst")
            _digest_tensor(digest)
            if src.shape != dst.shape:
                raise ValueError("src and dst shapes differ")
            h, w, c = src.shape
            arr[k] = FhdFrame(sid, h, w, c, src.data_ptr(), dst.data_ptr(), digest.data_ptr())
        return arr, len(items)

    @staticmethod
    def _events(events):
        for ev in events:
            if not ev.cuda_event:
                raise ValueError("wait event was never recorded")
        return (ctypes.c_void_p * max(len(events), 1))(*[ev.cuda_event for ev in events])

    @staticmethod
    def _out_event(ev, stream):
        if ev is None:
            return ctypes.c_void_p()
        if not ev.cuda_event:
            # torch creates the CUDA event on first record; the library re-records it.
            ev.record(stream if stream is not None else torch.cuda.current_stream())
        return ctypes.c_void_p(ev.cuda_event)

    def _run(self, plain, sched, items, stream, encrypt, key_waits=(), worker_waits=(), data_events=(),
             digest_event=None, master_event=None, keystream_event=None):
        arr, n = self._frames(items)
        if not (key_waits or worker_waits or data_events) and digest_event is None and master_event is None \
                and keystream_event is None:
            _check(plain(self._handle(), n, arr, _stream_ptr(stream)), self._h)
            return
        lists = [self._events(list(x)) for x in (key_waits, worker_waits, data_events)]
        hk = FhdSchedule(ctypes.cast(lists[0], ctypes.c_void_p), len(key_waits),
                         ctypes.cast(lists[1], ctypes.c_void_p), len(worker_waits),
                         ctypes.cast(lists[2], ctypes.c_void_p), len(data_events),
                         self._out_event(digest_event if encrypt else None, stream),
                         self._out_event(master_event, stream), self._out_event(keystream_event, stream))
        _check(sched(self._handle(), n, arr, _stream_ptr(stream), ctypes.byref(hk)), self._h)

    def encrypt_frames(self, items: Iterable, stream=None, master_event=None, wait_events=(), digest_event=None,
                       keystream_event=None, worker_wait_events=()):
        """items: (stream_id, src, dst, digest) tuples; digest (32 B) is written.

        The chaining-state kernel first waits on ``wait_events`` and
        ``master_event`` is recorded right after it; ``digest_event`` is
        recorded once the digests are written, before the chaining-state
        kernel; the worker kernel waits on ``worker_wait_events`` and
        ``keystream_event`` is recorded after it, before the permutation (all
        torch.cuda.Event's)."""
        lib = load()
        self._run(lib.encrypt_frames, lib.encrypt_frames_sched, items, stream, True, key_waits=tuple(wait_events),
                  worker_waits=tuple(worker_wait_events), digest_event=digest_event, master_event=master_event,
                  keystream_event=keystream_event)

    def decrypt_frames(self, items: Iterable, stream=None, master_event=None, wait_events=(), data_events=(),
                       keystream_event=None, worker_wait_events=()):
        """items: (stream_id, src, dst, digest) tuples; digest (32 B) is read.

        ``wait_events`` gate the chaining-state kernel (it reads the digests);
        ``worker_wait_events`` gate the worker kernel; ``data_events`` gate
        the inverse permutation, the first kernel that reads the ciphertext
        ``src``, so the chaotic stage can run while the ciphertext is still
        being produced; ``keystream_event`` is recorded after the worker
        kernel."""
        lib = load()
        self._run(lib.decrypt_frames, lib.decrypt_frames_sched, items, stream, False, key_waits=tuple(wait_events),
                  worker_waits=tuple(worker_wait_events), data_events=tuple(data_events), master_event=master_event,
                  keystream_event=keystream_event)

    def encrypt_frames_persistent(self, items: Iterable, stream=None):
        """encrypt_frames as one persistent kernel launch (at most 64 frames)."""
        arr, n = self._frames(items)
        _check(load().encrypt_frames_persistent(self._handle(), n, arr, _stream_ptr(stream)), self._h)

    def decrypt_frames_persistent(self, items: Iterable, stream=None):
        """decrypt_frames as one persistent kernel launch (at most 64 frames)."""
        arr, n = self._frames(items)
        _check(load().decrypt_frames_persistent(self._handle(), n, arr, _stream_ptr(stream)), self._h)

    def round_trip_persistent(self, receiver: "Cipher", enc_items: Iterable, dec_items: Iterable, stream=None):
        """This handle encrypts enc_items and ``receiver`` decrypts dec_items, frame k of dec_items being the
        ciphertext (and digest) of frame k of enc_items, in one persistent kernel launch."""
        ea, n = self._frames(enc_items)
        da, m = self._frames(dec_items)
        if n != m:
            raise ValueError("enc_items and dec_items differ in length")
        _check(load().cipher_round_trip_persistent(self._handle(), receiver._handle(), n, ea, da,
                                                   _stream_ptr(stream)), self._h)

    PTRACE = ("digest", "master", "keystream", "rows", "strips", "rx_master", "rx_keystream", "rx_rows", "rx_strips")

    def persistent_trace(self, count: int):
        """Timeline of the last persistent launch: (count, 9) ms after its start, columns PTRACE (-1: never)."""
        import numpy as np
        out = np.zeros((count, 9), dtype=np.float64)
        _check(load().cipher_persistent_trace(self._handle(), count, ctypes.c_void_p(out.ctypes.data)), self._h)
        return out

    def set_persistent_limits(self, timeout_ns: int = 2_000_000_000, hold_frame: int = -1):
        """Wait limit of the persistent launches of this handle; hold_frame >= 0 (a test hook) withholds that
        frame's digest so that the waits on it run out."""
        _check(load().cipher_set_persistent_limits(self._handle(), int(timeout_ns), int(hold_frame)), self._h)

    def verify_frames(self, items: Iterable, stream=None) -> torch.Tensor:
        """Receiver-side check: 1 per frame whose decrypted ``dst`` re-hashes to its ``digest``."""
        arr, n = self._frames(items)
        ok = torch.zeros(max(n, 1), dtype=torch.uint8, device=torch.device("cuda", torch.cuda.current_device()))
        _check(load().cipher_verify_frames(self._handle(), n, arr, ctypes.c_void_p(ok.data_ptr()),
                                           _stream_ptr(stream)), self._h)
        return ok[:n]

    def reserve(self, nbytes: int, stream=None):
        """Pre-size this CUDA stream's scratch so later calls on it never allocate."""
        _check(load().cipher_reserve(self._handle(), _stream_ptr(stream), int(nbytes)), self._h)

    def encrypt(self, sid: int, src: torch.Tensor, stream=None):
        dst = torch.empty_like(src)
        dig = torch.empty(32, dtype=torch.uint8, device=src.device)
        self.encrypt_frames([(sid, src, dst, dig)], stream)
        return dst, dig

    def decrypt(self, sid: int, src: torch.Tensor, digest: torch.Tensor, stream=None):
        dst = torch.empty_like(src)
        self.decrypt_frames([(sid, src, dst, digest)], stream)
        return dst

    def export_state(self, sid: int) -> bytes:
        buf = (ctypes.c_uint8 * FHD_STATE_BYTES)()
        _check(load().cipher_export_state(self._handle(), sid, buf, FHD_STATE_BYTES), self._h)
        return bytes(buf)

    def import_state(self, sid: int, data: bytes):
        buf = (ctypes.c_uint8 * FHD_STATE_BYTES).from_buffer_copy(bytes(data))
        _check(load().cipher_import_state(self._handle(), sid, buf, FHD_STATE_BYTES), self._h)

    def sync_status(self, stream=None):
        _check(load().cipher_sync_status(self._handle(), _stream_ptr(stream)), self._h)

    def profile(self, enable: bool = True):
        """Record CUDA events around every kernel this handle launches."""
        _check(load().cipher_profile(self._handle(), 1 if enable else 0), self._h)

    def profile_read(self) -> dict:
        """{kind: (ms, launches)} since the last read (synchronises on the events)."""
        ms = (ctypes.c_double * 5)()
        n = (ctypes.c_uint32 * 5)()
        _check(load().cipher_profile_read(self._handle(), ms, n), self._h)
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_KINDS)}

    def profile_spans(self, origin) -> list:
        """[(kind, start_ms, end_ms)] of the launches recorded since the last
        ``profile_read``, relative to ``origin`` (a recorded timing event)."""
        if not origin.cuda_event:
            raise ValueError("origin event was never recorded")
        lib = load()
        count = ctypes.c_uint32()
        _check(lib.cipher_profile_spans(self._handle(), ctypes.c_void_p(origin.cuda_event), 0, None, None, None,
                                        ctypes.byref(count)), self._h)
        n = count.value
        kinds = (ctypes.c_int32 * max(n, 1))()
        t0 = (ctypes.c_double * max(n, 1))()
        t1 = (ctypes.c_double * max(n, 1))()
        _check(lib.cipher_profile_spans(self._handle(), ctypes.c_void_p(origin.cuda_event), n, kinds, t0, t1,
                                        ctypes.byref(count)), self._h)
        return [(KERNEL_KINDS[kinds[i]], t0[i], t1[i]) for i in range(min(n, count.value))]

    def set_partition(self, enable):
        """Run LHCS_m on its own small SM partition (green contexts; True or 1), LHCS_m and the digest stage
        each on their own (2), or neither (False or 0)."""
        mode = int(enable) if not isinstance(enable, bool) else (1 if enable else 0)
        _check(load().cipher_set_partition(self._handle(), mode), self._h)

    def set_layout(self, layout: str):
        """Worker warp layout: "latency" (six chains per warp) or "throughput" (eight)."""
        _check(load().cipher_set_layout(self._handle(), {"latency": 0, "throughput": 1}[layout]), self._h)

    def set_worker_cta(self, warps: int):
        """Worker warps per CTA of the worker kernel (1, 2, 4 or 8); same results for every value."""
        _check(load().cipher_set_worker_cta(self._handle(), int(warps)), self._h)

    def set_worker_smem(self, nbytes: int):
        """Dynamic shared memory per worker CTA (a cap on worker CTAs per SM); same results for every value."""
        _check(load().cipher_set_worker_smem(self._handle(), int(nbytes)), self._h)

    def set_int_mix(self, per8: int):
        """Eight-chain worker warps per 8 that step on the integer pipes (0..8); same results for every value."""
        _check(load().cipher_set_int_mix(self._handle(), int(per8)), self._h)

    def partition(self) -> tuple:
        """(SMs of the LHCS_m partition, SMs of the rest); (0, 0) when off."""
        a, b = ctypes.c_uint32(), ctypes.c_uint32()
        _check(load().cipher_get_partition(self._handle(), ctypes.byref(a), ctypes.byref(b)), self._h)
        return a.value, b.value

    def last_error(self) -> str:
        return load().cipher_last_error(self._h).decode(errors="replace")

    def close(self):
        if self._h is not None:
            load().cipher_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- one call per step of the hot path ----

def fhd_frame_digest(data: torch.Tensor, n: int = 32, count: int = 1, out: torch.Tensor | None = None, stream=None,
                     mode: str = "xor"):
    """Frame digest of ``count`` equal buffers laid end to end: the XOR of the n sub-frame SHA-256 digests
    (mode "xor", the paper's), or SHA-256 of those digests concatenated in order (mode "tree")."""
    if data.numel() % max(count, 1):
        raise ValueError("data size must be a multiple of count")
    fn = {"xor": load().fhd_frame_digest, "tree": load().fhd_frame_digest_tree}[mode]
    if not data.is_cuda or data.dtype != torch.uint8 or not data.is_contiguous():
        raise ValueError("data must be a contiguous CUDA uint8 tensor")
    nbytes = data.numel() // max(count, 1)
    if out is None:
        out = torch.empty((count, 32), dtype=torch.uint8, device=data.device)
    ptr = data.data_ptr() if data.numel() else 0
    _check(fn(ctypes.c_void_p(ptr), nbytes, n, count, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


# ---- frame statistics (Sec. III and IV-B) ----

def _frames4(frames: torch.Tensor) -> torch.Tensor:
    if not frames.is_cuda or frames.dtype != torch.uint8 or not frames.is_contiguous():
        raise ValueError("frames must be a contiguous CUDA uint8 tensor")
    if frames.dim() == 3:
        frames = frames.unsqueeze(0)
    if frames.dim() != 4:
        raise ValueError("frames must be (count, height, width, channels) or (height, width, channels)")
    return frames


def _vp(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p()


def fhd_stats_histogram(frames: torch.Tensor, stream=None):
    """(hist uint32 [count, C, 256], stats float64 [count, C, 3] = histogram variance, chi^2, entropy)."""
    f = _frames4(frames)
    n, h, w, c = f.shape
    hist = torch.empty((n, c, 256), dtype=torch.int32, device=f.device)
    st = torch.empty((n, c, 3), dtype=torch.float64, device=f.device)
    _check(load().fhd_stats_histogram(_vp(f), n, h, w, c, _vp(hist), _vp(st), _stream_ptr(stream)))
    return hist, st


def fhd_stats_npcr_uaci(a: torch.Tensor, b: torch.Tensor, stream=None):
    """(counts int64 [count, C, 2] = changed pixels and sum |a - b|, out float64 [count, C, 2] = NPCR, UACI %)."""
    fa, fb = _frames4(a), _frames4(b)
    if fa.shape != fb.shape:
        raise ValueError("a and b shapes differ")
    n, h, w, c = fa.shape
    counts = torch.empty((n, c, 2), dtype=torch.int64, device=fa.device)
    out = torch.empty((n, c, 2), dtype=torch.float64, device=fa.device)
    _check(load().fhd_stats_npcr_uaci(_vp(fa), _vp(fb), n, h, w, c, _vp(counts), _vp(out), _stream_ptr(stream)))
    return counts, out


def fhd_stats_correlation(frames: torch.Tensor, pairs: torch.Tensor, stream=None):
    """pairs int32 [count, 3, npairs, 2] (row, column of x; directions horizontal, vertical, diagonal) ->
    (sums int64 [count, C, 3, 5], r float64 [count, C, 3], status int32 [1])."""
    f = _frames4(frames)
    n, h, w, c = f.shape
    if not pairs.is_cuda or pairs.dtype != torch.int32 or not pairs.is_contiguous() or pairs.dim() != 4 \
            or pairs.shape[0] != n or pairs.shape[1] != 3 or pairs.shape[3] != 2:
        raise ValueError("pairs must be a contiguous CUDA int32 tensor [count, 3, npairs, 2]")
    sums = torch.empty((n, c, 3, 5), dtype=torch.int64, device=f.device)
    r = torch.empty((n, c, 3), dtype=torch.float64, device=f.device)
    status = torch.zeros(1, dtype=torch.int32, device=f.device)
    _check(load().fhd_stats_correlation(_vp(f), n, h, w, c, _vp(pairs), pairs.shape[2], _vp(sums), _vp(r),
                                        _vp(status), _stream_ptr(stream)))
    return sums, r, status


def fhd_stats_local_entropy(frames: torch.Tensor, blocks: torch.Tensor, block: int, stream=None):
    """blocks int32 [count, k, 2] (top-left row, column) -> (out float64 [count, C], status int32 [1])."""
    f = _frames4(frames)
    n, h, w, c = f.shape
    if not blocks.is_cuda or blocks.dtype != torch.int32 or not blocks.is_contiguous() or blocks.dim() != 3 \
            or blocks.shape[0] != n or blocks.shape[2] != 2:
        raise ValueError("blocks must be a contiguous CUDA int32 tensor [count, k, 2]")
    out = torch.empty((n, c), dtype=torch.float64, device=f.device)
    status = torch.zeros(1, dtype=torch.int32, device=f.device)
    _check(load().fhd_stats_local_entropy(_vp(f), n, h, w, c, _vp(blocks), blocks.shape[1], block, _vp(out),
                                          _vp(status), _stream_ptr(stream)))
    return out, status


ROUTES = {"two_pass": 0, "single_pass": 1}


def fhd_set_encrypt_route(route: str = "two_pass"):
    """Encryption's confusion + XOR: "two_pass" (row pass + column pass, the default) or "single_pass" (one
    gather pass where the batch allows it)."""
    _check(load().fhd_set_encrypt_route(ROUTES[route]))


KS_ROUTES = {"pairs": 0, "trajectory": 1}


def fhd_set_keystream_route(route: str = "trajectory") -> str:
    """Keystream route (bit-identical either way): "trajectory" (the default; one LHCS_m trajectory per frame,
    each worker's window of it copied into D and B) or "pairs" (the n worker pairs as 2n chains).  Returns the
    previous route."""
    old = load().fhd_set_keystream_route(KS_ROUTES[route])
    if old < 0:
        _check(old)
    return {v: k for k, v in KS_ROUTES.items()}[old]


def fhd_fp64_probe(warps_per_subpartition: int, iters: int, sink: torch.Tensor, stream=None) -> int:
    """Launch the binary64 pipe probe; returns the binary64 lane-operations it executes."""
    if not sink.is_cuda or sink.dtype != torch.float64:
        raise ValueError("sink must be a CUDA float64 tensor (one element per SM)")
    ops = ctypes.c_uint64()
    _check(load().fhd_fp64_probe(warps_per_subpartition, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ops),
                                 _stream_ptr(stream)))
    return int(ops.value)


def fhd_frame_digest_noalloc(data: torch.Tensor, out: torch.Tensor, n: int = 32, count: int = 1, stream=None):
    """fhd_frame_digest into a caller-provided ``out`` (count x 32 bytes); the library allocates nothing."""
    if data.numel() % max(count, 1):
        raise ValueError("data size must be a multiple of count")
    if not data.is_cuda or data.dtype != torch.uint8 or not data.is_contiguous():
        raise ValueError("data must be a contiguous CUDA uint8 tensor")
    if not out.is_cuda or out.dtype != torch.uint8 or not out.is_contiguous() or out.numel() < 32 * count:
        raise ValueError("out must be a contiguous CUDA uint8 tensor of count x 32 bytes")
    nbytes = data.numel() // max(count, 1)
    ptr = data.data_ptr() if data.numel() else 0
    _check(load().fhd_frame_digest_noalloc(ctypes.c_void_p(ptr), nbytes, n, count, ctypes.c_void_p(out.data_ptr()),
                                           _stream_ptr(stream)))
    return out


def fhd_master(state5: torch.Tensor, H: torch.Tensor, n_workers=32, rk4_h=0.01, u_bound=(20, 20, 40, 20),
               IR: torch.Tensor | None = None, stream=None):
    """Reconstruct + 2n LHCS_m steps; ``state5`` (float64 x5, CUDA) is updated in place."""
    assert state5.is_cuda and state5.dtype == torch.float64 and state5.numel() == 5
    if IR is None:
        IR = torch.empty((2 * n_workers, 4), dtype=torch.float64, device=state5.device)
    p = _params(n_workers, rk4_h, u_bound)
    _check(load().fhd_master(ctypes.c_void_p(state5.data_ptr()), ctypes.c_void_p(H.data_ptr()), ctypes.byref(p),
                             ctypes.c_void_p(IR.data_ptr()), _stream_ptr(stream)))
    return IR


def fhd_keystream(IR: torch.Tensor, gamma: float, height: int, width: int, channels: int, n_workers=32,
                  rk4_h=0.01, stream=None, trajectory=False, B_out=None):
    """Worker pairs -> (D int16[C*(h+w)] holding uint16 bits, B uint8[h*w*C]).  trajectory=True takes the
    one-trajectory route (fhd_keystream_trajectory: IR must be LHCS_m's iterates, as fhd_master writes them).
    B_out: a uint8 device buffer of h*w*C bytes to write B into (any alignment)."""
    assert IR.is_cuda and IR.dtype == torch.float64 and IR.is_contiguous()
    D = torch.empty(channels * (height + width), dtype=torch.int16, device=IR.device)
    if B_out is None:
        B = torch.empty(height * width * channels, dtype=torch.uint8, device=IR.device)
    else:
        assert B_out.is_cuda and B_out.dtype == torch.uint8 and B_out.is_contiguous()
        assert B_out.numel() == height * width * channels
        B = B_out
    p = _params(n_workers, rk4_h)
    fn = load().fhd_keystream_trajectory if trajectory else load().fhd_keystream
    _check(fn(ctypes.c_void_p(IR.data_ptr()), float(gamma), ctypes.byref(p), height, width, channels,
              ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(B.data_ptr()), _stream_ptr(stream)))
    return D, B


def _permute(fn, src, D, B, out, stream):
    _frame_tensor(src, "src")
    h, w, c = src.shape
    if out is None:
        out = torch.empty_like(src)
    _check(fn(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(out.data_ptr()), h, w, c,
              ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(B.data_ptr()), _stream_ptr(stream)))
    return out


def fhd_permute_encrypt(src: torch.Tensor, D: torch.Tensor, B: torch.Tensor, out=None, stream=None):
    return _permute(load().fhd_permute_encrypt, src, D, B, out, stream)


def fhd_permute_decrypt(src: torch.Tensor, D: torch.Tensor, B: torch.Tensor, out=None, stream=None):
    return _permute(load().fhd_permute_decrypt, src, D, B, out, stream)


def fhd_strip_width(height: int, width: int, channels: int) -> int:
    return int(load().fhd_strip_width(height, width, channels))


def fhd_set_strip_width(height: int, width: int, channels: int, P: int):
    _check(load().fhd_set_strip_width(height, width, channels, P))


def fhd_row_band(height: int, width: int, channels: int) -> int:
    return int(load().fhd_row_band(height, width, channels))


def fhd_set_row_band(height: int, width: int, channels: int, RB: int):
    _check(load().fhd_set_row_band(height, width, channels, RB))


def fhd_set_cta_threads(height: int, width: int, channels: int, strip_threads: int = 0, row_threads: int = 0):
    """Threads per CTA of the permutation passes for one frame shape (column pass 256/512, row pass 128/256;
    0 keeps the default)."""
    _check(load().fhd_set_cta_threads(height, width, channels, strip_threads, row_threads))


def fhd_cta_threads(height: int, width: int, channels: int) -> tuple:
    """(column-pass, row-pass) threads per CTA in effect for a frame shape."""
    a, b = ctypes.c_uint32(), ctypes.c_uint32()
    _check(load().fhd_cta_threads(height, width, channels, ctypes.byref(a), ctypes.byref(b)))
    return int(a.value), int(b.value)


def fhd_frame_scratch_bytes(n_workers: int, height: int, width: int, channels: int) -> int:
    return int(load().fhd_frame_scratch_bytes(n_workers, height, width, channels))


def fhd_launch_count() -> int:
    return int(load().fhd_launch_count())


def fhd_binary64_check(pairs: int, seed: int = 1, stream=None) -> dict:
    """Integer-pipe binary64 multiply and add against the binary64 instructions on `pairs` generated operand
    pairs: {"bad_mul", "bad_add", "fast_mul", "fast_add"}."""
    out = (ctypes.c_uint64 * 4)()
    _check(load().fhd_binary64_check(pairs, seed, out, _stream_ptr(stream)))
    return {"bad_mul": int(out[0]), "bad_add": int(out[1]), "fast_mul": int(out[2]), "fast_add": int(out[3])}


def fhd_build_flags() -> int:
    """FHD_BUILD_BOUNDS_CHECK when the loaded library is the checked build."""
    return int(load().fhd_build_flags())


def fhd_bounds_report() -> dict:
    """Read and clear the checked build's bounds records: {"count", "site", "site_name", "index", "limit"}
    (count 0 in the default build)."""
    cnt, site, idx, lim = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint64()
    lib = load()
    _check(lib.fhd_bounds_report(ctypes.byref(cnt), ctypes.byref(site), ctypes.byref(idx), ctypes.byref(lim)))
    return {"count": int(cnt.value), "site": int(site.value),
            "site_name": lib.fhd_bounds_site_name(site.value).decode(), "index": int(idx.value),
            "limit": int(lim.value)}


def fhd_bounds_site_name(site: int) -> str:
    return load().fhd_bounds_site_name(site).decode()


def fhd_bounds_selftest(stream=None) -> tuple[int, int]:
    """Checked build: the permutation on a frame whose descriptor is one row short of its buffers; returns
    (failed checks, first site)."""
    cnt, site = ctypes.c_uint32(), ctypes.c_uint32()
    _check(load().fhd_bounds_selftest(ctypes.byref(cnt), ctypes.byref(site), _stream_ptr(stream)))
    return int(cnt.value), int(site.value)


def fhd_version() -> str:
    return load().fhd_version().decode()
