"""Continuous-batching serving loop for many video streams.

Frames of many streams arrive over time (Poisson processes at the streams'
frame rates).  The loop, polled on the host:

* admits arrived frames while their HBM footprint fits the budget (input,
  output and the per-frame keystream scratch: about 3N + 2C(h+w) + 96n bytes
  for an N-byte frame with n workers), otherwise they wait;
* groups the admitted frames into a batch and launches it with one
  ``encrypt_frames`` call on a free *lane* (one of several CUDA streams) --
  requests that arrive while other batches are on the GPU go into the next
  batch, and batches on different lanes overlap on the device;
* orders each video stream's frames on the device with CUDA events: a batch
  waits only for the chaining-state kernel (LHCS_m) of the streams' previous
  frames, so the digest, keystream and permutation of consecutive frames of
  one stream overlap, while the chaining state (x, y, z, w, gamma) stays on
  the device and advances in order;
* pre-allocates scratch per lane and output buffers (an allocation while
  work is in flight would synchronise the device);
* retires batches when their completion event fires, releasing the budget,
  and records each frame's latency (completion - arrival).

The paper's real-time criterion is a frame finished within 1000/FPS ms of its
arrival; the fraction that is not is its delay rate (Sec. V).  ``plain``
mode processes the same arrivals one frame per call on one CUDA stream, in
arrival order, for comparison.
"""
from __future__ import annotations

import collections
import dataclasses
import statistics
import time

import numpy as np
import torch

from . import _lib


@dataclasses.dataclass
class Frame:
    stream: int          # index into the server's video streams
    seq: int             # frame number within the stream
    arrival: float       # seconds since the start of the run
    nbytes: int = 0
    done: float = -1.0
    batch: int = -1


def frame_footprint(h: int, w: int, C: int, n: int) -> int:
    N = h * w * C
    return 3 * N + 2 * C * (h + w) + 96 * n + 64


class Server:
    """Serve a set of video streams with continuous batching.

    The lanes are CUDA streams whose calls wait on each other's chaining events; run the process with
    CUDA_DEVICE_MAX_CONNECTIONS=32 (set before CUDA starts) so that each lane has its own hardware queue.
    With the default 8, a lane held by an event wait stalls the lanes that share its queue (measured on the
    32-stream workload at 60 fps: p99 44.9 ms with 8 queues, 14.5 ms with 32)."""

    def __init__(self, keys, shapes, frame_pool, n_workers: int = 32, budget_bytes: int = 20 << 30,
                 lanes: int = 16, slots_per_lane: int = 1, max_batch: int = 64, fingerprint: bool = False,
                 outputs_per_shape: int = 32, partition: bool = False, keep: bool = False):
        self.n = n_workers
        self.cipher = _lib.Cipher(keys[0], n_workers=n_workers)
        # The lanes already overlap the frames of all streams; the SM partition would add two internal
        # CUDA streams per lane, more than a context's hardware queues, and lanes would then wait on
        # each other (measured: p50 12 -> 31 ms at 30 fps).  Off unless asked for.
        if not partition:
            self.cipher.set_partition(False)
        self.sids = [self.cipher.open_stream(k) for k in keys]
        self.shapes = list(shapes)
        self.pool = frame_pool               # shape -> list of device frames (inputs)
        self.budget = budget_bytes
        self.used = 0
        self.peak = 0
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.lanes = [torch.cuda.Stream() for _ in range(lanes)]
        self.slots = slots_per_lane
        self.max_batch = max_batch
        # Scratch and outputs are allocated up front: an allocation while work
        # is in flight would synchronise the device and stall every lane.
        per_lane = max(_lib.fhd_frame_scratch_bytes(n_workers, *sh) for sh in set(shapes)) * min(max_batch, 8)
        for ln in self.lanes:
            self.cipher.reserve(per_lane, stream=ln)
        self.free_out = {sh: [(torch.empty(sh, dtype=torch.uint8, device=self.dev),
                               torch.empty(32, dtype=torch.uint8, device=self.dev)) for _ in range(outputs_per_shape)]
                         for sh in set(shapes)}
        self.inflight = [collections.deque() for _ in range(lanes)]   # (done event, frames, outs)
        self.waiting = collections.deque()
        self.last_master = {}                 # video stream -> event after its latest chaining step
        self.done = []
        self.batches = 0
        self.batch_sizes = []
        self.fingerprint = fingerprint
        self.prints = {}                      # (stream, seq) -> digest of the ciphertext
        self.keep = keep
        self.kept = {}                        # (stream, seq) -> (ciphertext, transmitted digest) copies
        self._rr = 0

    def submit(self, fr: Frame):
        h, w, C = self.shapes[fr.stream]
        fr.nbytes = frame_footprint(h, w, C, self.n)
        self.waiting.append(fr)

    def _retire(self, now_fn):
        for q in self.inflight:
            while q and q[0][0].query():
                ev, frames, outs = q.popleft()
                t = now_fn()
                for fr in frames:
                    fr.done = t
                    self.used -= fr.nbytes
                self.done.extend(frames)
                for fr, (E, H) in zip(frames, outs):
                    if self.fingerprint:
                        d = _lib.fhd_frame_digest(E.view(-1), n=256)
                        self.prints[(fr.stream, fr.seq)] = bytes(d.cpu().numpy().reshape(-1))
                    if self.keep:               # before the buffers are reused (checks of served output)
                        self.kept[(fr.stream, fr.seq)] = (E.clone(), H.clone())
                    self.free_out[self.shapes[fr.stream]].append((E, H))

    def _free_lane(self):
        for k in range(len(self.lanes)):
            lane = (self._rr + k) % len(self.lanes)
            if len(self.inflight[lane]) < self.slots:
                self._rr = lane + 1
                return lane
        return None

    def _launch(self, lane: int) -> bool:
        q = self.waiting
        take = []
        # (a frame larger than the whole budget is admitted alone so it cannot block its stream)
        while q and len(take) < self.max_batch and (self.used + q[0].nbytes <= self.budget or self.used == 0):
            fr = q.popleft()
            self.used += fr.nbytes
            take.append(fr)
        if not take:
            return False
        self.peak = max(self.peak, self.used)
        s = self.lanes[lane]
        items, outs = [], []
        for fr in take:
            sh = self.shapes[fr.stream]
            pool = self.pool[sh]
            src = pool[(fr.stream * 7 + fr.seq) % len(pool)]
            free = self.free_out[sh]
            E, H = free.pop() if free else (torch.empty_like(src), torch.empty(32, dtype=torch.uint8, device=self.dev))
            items.append((self.sids[fr.stream], src, E, H))
            outs.append((E, H))
            fr.batch = self.batches
        # Order only the chaining step after each stream's previous frame.
        waits = []
        for st in {fr.stream for fr in take}:
            ev = self.last_master.get(st)
            if ev is not None and ev not in waits and not ev.query():
                waits.append(ev)
        master = torch.cuda.Event()
        self.cipher.encrypt_frames(items, stream=s, master_event=master, wait_events=waits)
        for st in {fr.stream for fr in take}:
            self.last_master[st] = master
        done = torch.cuda.Event()
        done.record(s)
        self.inflight[lane].append((done, take, outs))
        self.batches += 1
        self.batch_sizes.append(len(take))
        return True

    def poll(self, now_fn):
        self._retire(now_fn)
        while self.waiting:
            lane = self._free_lane()
            if lane is None or not self._launch(lane):
                break

    def drain(self, now_fn):
        while self.waiting or any(self.inflight):
            self.poll(now_fn)
            time.sleep(0.0002)

    def close(self):
        torch.cuda.synchronize()
        self.cipher.close()


def arrivals(rates, duration: float, seed: int):
    """Merged Poisson arrival trace: list of (time, stream, seq) sorted by time."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for s, r in enumerate(rates):
        t, k = g.exponential(1.0 / r), 0
        while t < duration:
            out.append((t, s, k))
            k += 1
            t += g.exponential(1.0 / r)
    out.sort()
    return out


def latency_stats(frames, fps: float):
    lat = [1000.0 * (f.done - f.arrival) for f in frames if f.done >= 0]
    if not lat:
        return {}
    lat.sort()
    q = lambda p: lat[min(len(lat) - 1, int(round(p * (len(lat) - 1))))]
    return {"frames": len(lat), "p50_ms": q(0.5), "p99_ms": q(0.99), "max_ms": lat[-1],
            "mean_ms": statistics.fmean(lat), "delay_rate": sum(1 for x in lat if x > 1000.0 / fps) / len(lat)}


def run(keys, shapes, frame_pool, fps: float, duration: float, seed: int = 0, n_workers: int = 32,
        budget_bytes: int = 20 << 30, lanes: int | None = None, mode: str = "served", fingerprint: bool = False,
        keep: bool = False):
    """Replay a Poisson arrival trace in real time; returns (stats, server).  keep=True keeps a copy of
    every served frame's ciphertext and digest in ``server.kept``."""
    trace = arrivals([fps] * len(shapes), duration, seed)
    if mode == "plain":
        srv = Server(keys, shapes, frame_pool, n_workers, budget_bytes, lanes=1, slots_per_lane=1, max_batch=1,
                     fingerprint=fingerprint, keep=keep)
    else:
        srv = Server(keys, shapes, frame_pool, n_workers, budget_bytes, lanes=lanes or 16, fingerprint=fingerprint,
                     keep=keep)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    k = 0
    while k < len(trace) or srv.waiting or any(srv.inflight):
        t = now()
        while k < len(trace) and trace[k][0] <= t:
            at, s, seq = trace[k]
            srv.submit(Frame(s, seq, at))
            k += 1
        srv.poll(now)
        if k < len(trace) and not any(srv.inflight):
            time.sleep(max(0.0, min(0.0005, trace[k][0] - now())))
        if mode == "plain" and now() > duration + 2.0:
            break                      # the plain loop cannot keep up: stop counting
    elapsed = now()
    stats = latency_stats(srv.done, fps)
    total_bytes = sum(np.prod(shapes[f.stream]) for f in srv.done)
    stats.update({"mode": mode, "fps_per_stream": fps, "streams": len(shapes), "seconds": elapsed,
                  "offered_frames": len(trace), "completed_frames": len(srv.done),
                  "frames_per_s": len(srv.done) / elapsed, "GB_per_s": 2 * total_bytes / elapsed / 1e9,
                  "batches": srv.batches,
                  "mean_batch": statistics.fmean(srv.batch_sizes) if srv.batch_sizes else 0.0,
                  "peak_budget_fraction": srv.peak / budget_bytes, "lanes": len(srv.lanes)})
    return stats, srv
