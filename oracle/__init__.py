"""CPU oracle of the arXiv 2505.07158 video cipher -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it.  ``oracle.c`` is plain single-threaded C compiled with
``-ffp-contract=off`` so that every binary64 multiply and add is rounded on its
own, as the chaotic iteration requires; this module builds it with ``gcc`` on
first use and wraps it with numpy-friendly functions.

Functions with no independent pin would say "parity unpinned" here; every
function below is pinned by ``tests/test_oracle_*.py`` (see the test
docstrings for what pins which step).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Paper defaults: sigma, rho, beta fixed in Eq. (1); n = 32 workers on the
# Xeon + RTX 3090 platform (Tab. speedEvaluation).  Integrator step and the
# reconstruction upper bounds are readings (the paper gives no values).
DEFAULT_N = 32
DEFAULT_H = 0.01
DEFAULT_U = (20, 20, 40, 20)

CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        u32, u64, dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        lib.oracle_sha256.argtypes = [P, u64, P]
        lib.oracle_frame_digest.argtypes = [P, u64, u32, P]
        lib.oracle_frame_digest_tree.argtypes = [P, u64, u32, P]
        lib.oracle_key_to_ic.argtypes = [P, P, P]
        lib.oracle_reconstruct.argtypes = [dbl, P, u32]
        lib.oracle_reconstruct.restype = dbl
        lib.oracle_rk4_step.argtypes = [P, dbl, dbl]
        lib.oracle_master.argtypes = [P, P, P, dbl, dbl, u32, P, P]
        lib.oracle_keystream.argtypes = [P, u32, dbl, dbl, u32, u32, u32, P, P]
        lib.oracle_permute_encrypt.argtypes = [P, u32, u32, u32, P, P, P]
        lib.oracle_permute_decrypt.argtypes = [P, u32, u32, u32, P, P, P]
        lib.oracle_frame_keystream.argtypes = [P, dbl, dbl, u32, P, P, u32, u32, u32, P, P]
        lib.oracle_encrypt_frame.argtypes = [P, dbl, dbl, u32, P, P, u32, u32, u32, P, P, u32, u32]
        lib.oracle_decrypt_frame.argtypes = [P, dbl, dbl, u32, P, P, u32, u32, u32, P, P, u32]
        lib.oracle_digest_mask.argtypes = [P, dbl, P]
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def _u32x4(u) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(u, dtype=np.uint32).reshape(4))


def sha256(msg) -> bytes:
    """FIPS 180-4 SHA-256 of a byte string."""
    m = _u8(np.frombuffer(bytes(msg), dtype=np.uint8)) if isinstance(msg, (bytes, bytearray)) else _u8(msg).reshape(-1)
    out = np.zeros(32, np.uint8)
    buf = m if m.size else np.zeros(1, np.uint8)
    _load().oracle_sha256(_ptr(buf), m.size, _ptr(out))
    return out.tobytes()


DIGEST_MODES = {"xor": 0, "tree": 1}
# How the digest travels (Sec. V sends it encrypted, mechanism not given): "plain" as computed, or "masked"
# (an option of this implementation) XORed with a mask derived from the stream's chaining state.
TRANSPORTS = {"plain": 0, "masked": 1}


def frame_digest(frame, n: int = DEFAULT_N, mode: str = "xor") -> bytes:
    """Sec. II-A: XOR of the SHA-256 digests of the n sub-frames (mode "xor").  Mode "tree", an option of
    this implementation rather than the paper's: SHA-256 of the n sub-frame digests concatenated in order."""
    f = _u8(frame).reshape(-1)
    out = np.zeros(32, np.uint8)
    buf = f if f.size else np.zeros(1, np.uint8)
    fn = _load().oracle_frame_digest_tree if DIGEST_MODES[mode] == 1 else _load().oracle_frame_digest
    fn(_ptr(buf), f.size, n, _ptr(out))
    return out.tobytes()


def key_to_ic(key: bytes, u=DEFAULT_U):
    """256-bit key -> (x0, y0, z0, w0, gamma)."""
    k = _u8(np.frombuffer(bytes(key), dtype=np.uint8))
    assert k.size == 32
    ic = np.zeros(5, np.float64)
    _load().oracle_key_to_ic(_ptr(k), _ptr(_u32x4(u)), _ptr(ic))
    return tuple(float(v) for v in ic)


def reconstruct(v: float, hb: bytes, u: int) -> float:
    """Sec. II-A, Fig. 1a: one initial condition from 8 digest bytes."""
    b = _u8(np.frombuffer(bytes(hb), dtype=np.uint8))
    assert b.size == 8
    return float(_load().oracle_reconstruct(float(v), _ptr(b), int(u)))


def rk4_step(state, gamma: float, h: float = DEFAULT_H) -> np.ndarray:
    """One RK4 step of Eq. (1); returns the new (x, y, z, w)."""
    s = np.ascontiguousarray(np.asarray(state, np.float64).reshape(4).copy())
    _load().oracle_rk4_step(_ptr(s), float(gamma), float(h))
    return s


def rk4_trajectory(state, gamma: float, steps: int, h: float = DEFAULT_H) -> np.ndarray:
    """States after steps 1..steps, shape (steps, 4)."""
    s = np.ascontiguousarray(np.asarray(state, np.float64).reshape(4).copy())
    out = np.zeros((steps, 4), np.float64)
    lib = _load()
    for t in range(steps):
        lib.oracle_rk4_step(_ptr(s), float(gamma), float(h))
        out[t] = s
    return out


def master(state, H: bytes, gamma: float, n: int = DEFAULT_N, h: float = DEFAULT_H, u=DEFAULT_U):
    """Algorithm 1: reconstruct from H, iterate LHCS_m 2n times -> (IR (2n,4), new state)."""
    v = np.ascontiguousarray(np.asarray(state, np.float64).reshape(4))
    Hb = _u8(np.frombuffer(bytes(H), dtype=np.uint8))
    IR = np.zeros((2 * n, 4), np.float64)
    ns = np.zeros(4, np.float64)
    _load().oracle_master(_ptr(v), _ptr(Hb), _ptr(_u32x4(u)), float(gamma), float(h), n, _ptr(IR), _ptr(ns))
    return IR, ns


def keystream(IR, gamma: float, hgt: int, wid: int, C: int, n: int = DEFAULT_N, h: float = DEFAULT_H):
    """Algorithm 2 for all n workers -> (D uint16 [C*(h+w)], B uint8 [h*w*C])."""
    ir = np.ascontiguousarray(np.asarray(IR, np.float64).reshape(2 * n, 4))
    D = np.zeros(max(C * (hgt + wid), 1), np.uint16)
    B = np.zeros(max(hgt * wid * C, 1), np.uint8)
    _load().oracle_keystream(_ptr(ir), n, float(gamma), float(h), hgt, wid, C, _ptr(D), _ptr(B))
    return D[: C * (hgt + wid)], B[: hgt * wid * C]


def permute_encrypt(F, D, B) -> np.ndarray:
    """Algos 3-7 on the bit matrices: frame (h, w, C) uint8 -> encrypted frame."""
    F = _u8(F)
    h, w, C = F.shape
    D = np.ascontiguousarray(np.asarray(D, np.uint16))
    B = _u8(B).reshape(-1)
    assert D.size == C * (h + w) and B.size == h * w * C
    E = np.zeros_like(F)
    _load().oracle_permute_encrypt(_ptr(F), h, w, C, _ptr(D), _ptr(B), _ptr(E))
    return E


def permute_decrypt(E, D, B) -> np.ndarray:
    """Inverse of :func:`permute_encrypt`."""
    E = _u8(E)
    h, w, C = E.shape
    D = np.ascontiguousarray(np.asarray(D, np.uint16))
    B = _u8(B).reshape(-1)
    assert D.size == C * (h + w) and B.size == h * w * C
    F = np.zeros_like(E)
    _load().oracle_permute_decrypt(_ptr(E), h, w, C, _ptr(D), _ptr(B), _ptr(F))
    return F


class Stream:
    """One video stream's chaining state (Sec. II-A): x, y, z, w and gamma.

    The first frame reconstructs from the key's x0..w0; every later frame from
    x_2n..w_2n of the previous frame's LHCS_m run (Algorithm 1)."""

    def __init__(self, ic, n: int = DEFAULT_N, h: float = DEFAULT_H, u=DEFAULT_U, digest_mode: str = "xor",
                 transport: str = "plain"):
        ic = tuple(float(v) for v in ic)
        self.state = np.array(ic[:4], np.float64)
        self.gamma = ic[4]
        self.n, self.h, self.u = n, h, _u32x4(u)
        self.digest_mode = DIGEST_MODES[digest_mode]
        self.masked = TRANSPORTS[transport]

    @classmethod
    def from_key(cls, key: bytes, n: int = DEFAULT_N, h: float = DEFAULT_H, u=DEFAULT_U, digest_mode: str = "xor",
                 transport: str = "plain"):
        return cls(key_to_ic(key, u), n, h, u, digest_mode, transport)

    def digest_mask(self) -> bytes:
        """The mask M of the next frame's transmitted digest (masked transport, an option of this
        implementation): SHA-256 of "FHDMASK1" and the LE64 bit patterns of the chaining state and gamma."""
        M = np.zeros(32, np.uint8)
        _load().oracle_digest_mask(_ptr(self.state), self.gamma, _ptr(M))
        return M.tobytes()

    def frame_keystream(self, H: bytes, hgt: int, wid: int, C: int):
        """Advance the chain by one frame; return that frame's (D, B)."""
        Hb = _u8(np.frombuffer(bytes(H), dtype=np.uint8))
        D = np.zeros(max(C * (hgt + wid), 1), np.uint16)
        B = np.zeros(max(hgt * wid * C, 1), np.uint8)
        _load().oracle_frame_keystream(_ptr(self.state), self.gamma, self.h, self.n, _ptr(self.u),
                                       _ptr(Hb), hgt, wid, C, _ptr(D), _ptr(B))
        return D[: C * (hgt + wid)], B[: hgt * wid * C]

    def encrypt(self, F):
        """Algorithm 1 for one frame: returns (E, H)."""
        F = _u8(F)
        h, w, C = F.shape
        E = np.zeros_like(F)
        H = np.zeros(32, np.uint8)
        _load().oracle_encrypt_frame(_ptr(self.state), self.gamma, self.h, self.n, _ptr(self.u),
                                     _ptr(F), h, w, C, _ptr(E), _ptr(H), self.digest_mode, self.masked)
        return E, H.tobytes()

    def advance(self, F):
        """The chaining step of Algorithm 1 alone: the state after frame F (its digest H, then 2n LHCS_m
        steps from the state reconstructed from H), without the worker keystream or the confusion, which
        do not feed the state.  Returns the frame's digest H (as computed, not masked)."""
        H = frame_digest(F, self.n, "tree" if self.digest_mode == 1 else "xor")
        _, ns = master(self.state, H, self.gamma, self.n, self.h, self.u)
        self.state = np.array(ns, np.float64)
        return H

    def decrypt(self, E, H: bytes):
        """Inverse of :meth:`encrypt` given the transmitted digest H."""
        E = _u8(E)
        h, w, C = E.shape
        Hb = _u8(np.frombuffer(bytes(H), dtype=np.uint8))
        F = np.zeros_like(E)
        _load().oracle_decrypt_frame(_ptr(self.state), self.gamma, self.h, self.n, _ptr(self.u),
                                     _ptr(E), h, w, C, _ptr(Hb), _ptr(F), self.masked)
        return F
