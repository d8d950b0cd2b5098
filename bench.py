#!/usr/bin/env python3
"""Benchmark of the cipher's hot path on GB300.

Workload (one "step"): the 30-frame 1920x1080x3 uint8 clip (smooth 2-D
gradients + Gaussian noise sigma 8, shifted 2 px per frame) of one video
stream is encrypted (digest -> LHCS_m -> keystream, by default from one LHCS_m
trajectory per frame -> confusion + XOR, Algorithm 1) and then decrypted
(inverse), one library call each.  The
metric is round-tripped 1080p frames per second (30 frames per step).
Inputs are resident in HBM when the timed region starts and are larger than
L2 (30 x 6.2 MB frames + outputs + keystream ~ 560 MB).

Also reported: an end-to-end number through the same public API with pinned
host buffers (host->device copy of the plaintext and device->host copy of the
decrypted frames and digests inside the timed region), the plain one-frame-
per-call path, per-kernel times from CUDA events recorded on the launch
stream, the roofline of the dominant kernel, and the CPU oracle timed on a
bounded sample.

``--impl reference`` times the CPU oracle (single-threaded C) on the same
workload and metric instead.  Multi-GPU: one process per GPU (torchrun); each
rank encrypts its own clip (independent streams, no data exchange).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# One hardware queue per CUDA stream: with the default 8, the slots' streams (two callers' CUDA streams per
# clip in flight plus the library's internal chain and bulk streams) share queues, and a stream held by an
# event wait stalls unrelated streams queued behind it.  Read when the CUDA context is created.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth_inputs as si  # noqa: E402

FRAMES, HGT, WID, CH = 30, 1080, 1920, 3
N_WORKERS = 32
HBM_PEAK_FALLBACK = 6800.0
# FP64 pipe, used only when the in-run probe (run_fp64_probe) cannot run: 1.684 binary64 lane-ops per clock
# per SM (an earlier probe with one warp per sub-partition), x 152 SMs x 2.07 GHz maximum SM clock.
FP64_PEAK_TOPS_FALLBACK = 1.684 * 152 * 2.07e9 / 1e12
RK4_FP64_OPS = 104      # per chain step: 4 x 13 (Eq. 1) + 3 x 8 (stages) + 4 x 7 (combination)
# DRAM bytes (read + write) per 1080p frame of one launch, from ncu captures (cold caches, writes still in L2
# at kernel end not counted): the worker kernel on a 4-frame clip, the four permutation passes on the 30-frame
# clip (row + column pass of each direction, divided by 30); None where no capture of the current kernel exists.
TRAFFIC_PER_FRAME = {"keystream": (29952 + 0) / 4,
                     "encrypt": (186890496 + 130175232 + 374881536 + 156594944) / 30,
                     "decrypt": (411278336 + 127123200 + 186961664 + 125687808) / 30, "sha": None, "master": None}
# The one-trajectory keystream route, per 1080p frame: trajectory_kernel on a 4-frame clip (24,064 bytes read,
# none written: the records stay in L2) plus emit_kernel on the 30-frame clip (5,954,048 read, 126,382,848
# written), both from ncu captures.
TRAFFIC_TRAJ_PER_FRAME = (24064 + 0) / 4 + (5954048 + 126382848) / 30


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=120)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-oracle sample")
    ap.add_argument("--frames", type=int, default=30, help="frames per step (30 = the clip; smaller for ncu)")
    ap.add_argument("--dry-run", action="store_true",
                    help="multi-process skeleton only (gloo, no GPU): ranks, barrier, max-over-ranks, one line")
    ap.add_argument("--no-probe", action="store_true", help="skip the binary64 peak probe (profiling runs)")
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed regions of --steps steps each; value is the median region")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="length of each serving run (60 s: the full workload)")
    ap.add_argument("--no-extras", action="store_true", help="skip the mixed-batch, serving and stress measurements")
    ap.add_argument("--no-stress", action="store_true", help="skip the 256 x 8K stress round trip")
    ap.add_argument("--extras", default=",".join(EXTRAS),
                    help="comma list of the other workloads to run: " + ",".join(EXTRAS))
    ap.add_argument("--encrypt-route", default="two_pass", choices=["two_pass", "single_pass"],
                    help="route of the encryption's confusion + XOR in the headline")
    ap.add_argument("--keystream-route", default="trajectory", choices=["trajectory", "pairs"],
                    help="route of the keystream: one LHCS_m trajectory per frame (default) or the n worker pairs")
    ap.add_argument("--gate", default="chain", choices=["permute", "keystream", "chain", "window"],
                    help="what the next clip's LHCS_m waits for besides the chaining state (see round_trip)")
    ap.add_argument("--partition", action="store_true",
                    help="run LHCS_m on its own 8-SM partition (green contexts) instead of beside the workers")
    ap.add_argument("--digest-partition", action="store_true",
                    help="also run the digest stage on its own 8-SM partition (three-way split; implies --partition)")
    ap.add_argument("--no-partition", action="store_true", help="(the default) LHCS_m on the same SMs as the rest")
    ap.add_argument("--layout", default=None, choices=["latency", "throughput"],
                    help="worker warp layout (default: the tuned table's, else throughput)")
    ap.add_argument("--worker-cta", type=int, default=1, choices=[1, 2, 4, 8], help="worker warps per CTA")
    ap.add_argument("--inflight", type=int, default=None,
                    help="clips in flight on separate buffers: later clips' digest stage and LHCS_m overlap earlier "
                         "clips' keystreams (default: the tuned table's, else 5)")
    ap.add_argument("--worker-smem", type=int, default=None,
                    help="dynamic shared memory per worker CTA, a cap on worker CTAs per SM (default: the tuned "
                         "table's, else 0: none)")
    ap.add_argument("--int-mix", type=int, default=None, choices=range(9), metavar="0..8",
                    help="worker warps per 8 (throughput layout) that step on the integer pipes beside the "
                         "binary64 ones (default: the tuned table's, else 0)")
    ap.add_argument("--worker-window", type=int, default=None,
                    help="clip k's workers (both sides) wait for the workers of clip k - W, so about W clips' "
                         "workers share the FP64 pipes while later clips' digests and LHCS_m run ahead "
                         "(0: no gate; needs more clips in flight than W; default: the tuned table's, else 3)")
    ap.add_argument("--tune", default=None, metavar="OUT.json",
                    help="time the tile shapes of every workload's frame sizes and the clip pipeline's work split "
                         "(layout, clips in flight, worker window) and write the table to OUT.json "
                         "(the library's tuned.json format); prints it and exits")
    ap.add_argument("--copy-streams", type=int, default=None, choices=[1, 2, 4],
                    help="end-to-end run: CUDA streams per copy direction, clips taking them in turn (default: "
                         "the tuned table's, else 2)")
    ap.add_argument("--e2e-out-buffers", type=int, default=2,
                    help="end-to-end run: pinned host buffers the decrypted clips are copied into, in turn "
                         "(0: one per clip in flight)")
    ap.add_argument("--spans", default=None,
                    help="write the timed region's launch timeline (sender and receiver, ms from its start) as JSON")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.idx)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        time.sleep(0.15)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- binary64 peak

def run_fp64_probe(fhd, torch, dev, gpu_index, iters=16384, reps=5, warps=(1, 2, 3, 4, 6, 8)):
    """The binary64 pipe's rate on this GPU, measured in this run: the library's probe kernel (one CTA per
    SM, k warps per sub-partition, eight independent fma chains per lane), each k timed with CUDA events
    (best of `reps` launches) while nvidia-smi samples the SM clock.  Returns the per-k rates, the peak
    (the best rate, in binary64 Top/s) and the lane-ops per clock per SM at the sampled median clock."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(sms, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    rows = {}
    with ClockSampler(gpu_index) as clk:
        for k in warps:
            for _ in range(2):
                fhd.fhd_fp64_probe(k, iters, sink, stream)
            best = None
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ops = fhd.fhd_fp64_probe(k, iters, sink, stream)
                b.record(stream)
                b.synchronize()
                ms = a.elapsed_time(b)
                best = ms if best is None else min(best, ms)
            rows[k] = {"ms": best, "lane_ops": ops, "tops": ops / (best / 1000.0) / 1e12}
    clocks = clk.summary()
    mhz = clocks.get("sm_mhz")
    for r in rows.values():
        r["lane_ops_per_clk_per_sm"] = (r["tops"] * 1e12 / (mhz * 1e6 * sms)) if mhz else None
    kbest = max(rows, key=lambda k: rows[k]["tops"])
    return {"peak_tops": rows[kbest]["tops"], "best_warps_per_subpartition": kbest,
            "lane_ops_per_clk_per_sm": rows[kbest]["lane_ops_per_clk_per_sm"], "sms": sms,
            "per_warps_per_subpartition": {str(k): v for k, v in rows.items()}, "clocks": clocks,
            "kernel": "fp64_probe_kernel: one CTA per SM, 4k warps, 8 independent __fma_rn chains per lane, "
                      f"{iters} steps; best of {reps} launches per k, CUDA events"}


# ---------------------------------------------------------------- work model

def worker_steps(h, w, C, n):
    """RK4 steps of every worker chain of one frame (both chains of a pair)."""
    LD, LB = C * (h + w), h * w * C
    total = 0
    for p in range(n):
        nd = (LD * (p + 1)) // n - (LD * p) // n
        nb = (LB * (p + 1)) // n - (LB * p) // n
        total += -(-(2 * nd + nb) // 24)
    return 2 * total


def traj_steps(h, w, C, n):
    """RK4 steps of one frame's trajectory in the one-trajectory keystream route: records R (the bound the
    library sizes them by) need the states up to s_{R+2}, and s_1 .. s_2n are LHCS_m's iterates."""
    LD, LB = C * (h + w), h * w * C
    R = (48 * (n - 1) + 2 * -(-LD // n) + -(-LB // n) + 23) // 24
    return R + 2 - 2 * n


RK4_FP64_INSTR = 27     # binary64 instructions one warp issues per RK4 step of its chains (six-chain layout)


def sha_blocks(N, n):
    blocks = 0
    for i in range(n):
        L = (N * (i + 1)) // n - (N * i) // n
        blocks += L // 64 + (1 if (L % 64) + 9 <= 64 else 2)
    return blocks


# ---------------------------------------------------------------- CPU oracle

def _oracle_worker(idx: int, conn):
    """One host core: its own video stream (own key) round-tripped through the oracle, one chained
    frame per request; replies whether the round trip was exact."""
    import oracle
    key = si.key(1000 + idx)
    enc, dec = oracle.Stream.from_key(key, n=N_WORKERS), oracle.Stream.from_key(key, n=N_WORKERS)
    frames = [si.gradient_frame(HGT, WID, CH, t=t, seed=idx) for t in range(2)]
    t = 0
    while True:
        msg = conn.recv()
        if msg is None:
            break
        F = frames[t % 2]
        E, H = enc.encrypt(F)
        P = dec.decrypt(E, H)
        t += 1
        conn.send(bool(np.array_equal(P, F)))


class OraclePool:
    """The oracle, as it stands, on every host core: one spawned process per core, each with its own
    stream; a step round-trips one chained 1080p frame on every core (independent streams)."""

    def __init__(self, cores: int | None = None):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.cores = cores or os.cpu_count() or 1
        self.pipes, self.procs = [], []
        for i in range(self.cores):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(i, b), daemon=True)
            p.start()
            self.pipes.append(a)
            self.procs.append(p)

    def step(self) -> bool:
        for a in self.pipes:
            a.send(1)
        return all(a.recv() for a in self.pipes)

    def close(self):
        for a in self.pipes:
            a.send(None)
        for p in self.procs:
            p.join(timeout=30)


def cpu_oracle_sample(seconds: float, rank: int):
    """Round trips on every host core (one oracle stream per core) until the budget is spent:
    (frames/s, frames, seconds, cores)."""
    pool = OraclePool()
    try:
        ok = pool.step()                        # warm-up: first frame of every stream
        done, t0 = 0, time.perf_counter()
        while True:
            ok = pool.step() and ok
            done += pool.cores
            el = time.perf_counter() - t0
            if el >= seconds:
                break
        assert ok
        return done / el, done, el, pool.cores
    finally:
        pool.close()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    pool = OraclePool()
    try:
        ok = True
        for _ in range(args.warmup):
            ok = pool.step() and ok
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ok = pool.step() and ok
        el = time.perf_counter() - t0
    finally:
        pool.close()
    assert ok, "oracle round trip not exact"
    fps = pool.cores * args.steps / el
    line = {
        "impl": "reference", "metric": "1080p RGB frames/s (encrypt + decrypt round trip)", "value": fps,
        "unit": "frames/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "1920x1080x3 gradient+noise frames, n=32, one stream per host core",
                   "sample": f"each step round-trips one chained frame on each of {pool.cores} host cores "
                             "(independent streams, own keys)",
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": pool.cores, "kind": "oracle",
                         "sample": f"{args.steps} steps x {pool.cores} chained 1080p frame round trips, "
                                   "single-threaded C oracle per core"},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm

def run_ours(args):
    global FRAMES
    FRAMES = args.frames
    import torch
    import torch.distributed as dist

    import paper_2505_07158_gb300 as fhd

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_2505_07158_gb300 import autotune
    tuned = autotune.tune([(HGT, WID, CH)])
    # the clip pipeline's work split: flags, else the tuned table for this GPU, else the built-in defaults
    # (the worker-pair route has its own record in the table)
    pipe = autotune.pipeline_defaults() or {}
    if args.keystream_route == "pairs":
        pipe = pipe.get("pairs_route") or pipe
    split_source = {}
    for name, attr, default in (("layout", "layout", "throughput"), ("inflight", "inflight", 5),
                                ("worker_window", "worker_window", 3), ("int_mix", "int_mix", 0),
                                ("worker_smem", "worker_smem", 0), ("copy_streams", "copy_streams", 2)):
        if getattr(args, attr) is None:
            setattr(args, attr, pipe.get(name, default))
            split_source[name] = "tuned table" if name in pipe else "built-in default"
        else:
            split_source[name] = "flag"
    fhd.fhd_set_encrypt_route(args.encrypt_route)
    fhd.fhd_set_keystream_route(args.keystream_route)
    clip = si.clip(FRAMES, HGT, WID, CH, seed=rank)
    host = torch.from_numpy(clip).pin_memory()
    key = si.key(rank)
    enc, dec = fhd.Cipher(key, n_workers=N_WORKERS), fhd.Cipher(key, n_workers=N_WORKERS)
    if args.digest_partition and not args.no_partition:
        enc.set_partition(2)
        dec.set_partition(2)
    elif not args.partition or args.no_partition:
        enc.set_partition(False)
        dec.set_partition(False)
    enc.set_layout(args.layout)
    dec.set_layout(args.layout)
    enc.set_worker_cta(args.worker_cta)
    dec.set_worker_cta(args.worker_cta)
    enc.set_int_mix(args.int_mix)
    dec.set_int_mix(args.int_mix)
    enc.set_worker_smem(args.worker_smem)
    dec.set_worker_smem(args.worker_smem)
    sid, rid = enc.open_stream(), dec.open_stream()
    stream = torch.cuda.current_stream()

    class Slot:
        """Buffers and CUDA streams of one clip in flight: the sender encrypts on `tx`, the receiver
        decrypts on `rx`; the receiver's chaotic stage waits for the digests, its inverse permutation
        for the ciphertext, and the slot is reused once its previous receiver has finished."""

        def __init__(self):
            # The clip's frames are views of one contiguous tensor each way, so that the end-to-end step moves
            # its input and its result with one copy each.
            self.src_all = host.to(dev)
            self.dec_all = torch.empty_like(self.src_all)
            self.srcs = [self.src_all[t] for t in range(FRAMES)]
            self.encs = [torch.empty_like(x) for x in self.srcs]
            self.decs = [self.dec_all[t] for t in range(FRAMES)]
            self.digs = torch.empty((FRAMES, 32), dtype=torch.uint8, device=dev)
            self.tx, self.rx = torch.cuda.Stream(), torch.cuda.Stream()
            self.enc_items = [(sid, self.srcs[t], self.encs[t], self.digs[t]) for t in range(FRAMES)]
            self.dec_items = [(rid, self.encs[t], self.decs[t], self.digs[t]) for t in range(FRAMES)]
            self.digests_ready, self.cipher_ready = torch.cuda.Event(), torch.cuda.Event()
            self.enc_master, self.dec_master, self.rx_done = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()
            self.dec_done, self.enc_ks, self.dec_ks = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()
            self.h2d_done = torch.cuda.Event()
            self.used = False
            self.e2e_used = False
            self.host_out = torch.empty_like(host).pin_memory() if args.e2e_out_buffers <= 0 else None
            self.host_dig = torch.empty((FRAMES, 32), dtype=torch.uint8).pin_memory()
            self.index = len(slots)

    slots = []
    for _ in range(max(1, args.inflight)):
        slots.append(Slot())
    # Decrypted clips go to a ring of pinned host buffers (a consumer reads each before its turn comes round
    # again), or to one buffer per clip in flight.
    n_out = max(0, args.e2e_out_buffers)
    host_outs = [torch.empty_like(host).pin_memory() for _ in range(n_out)]
    e2e_out_used = set()
    # The end-to-end copies run on two streams of their own, one per direction, so that a copy waiting for
    # its slot to come free never sits in a compute stream.  A clip's host-to-device copy waits only for the
    # slot's previous encryption to have read its frames, so it runs a round trip ahead; the sender waits
    # for that copy and for the slot's previous receiver and copy-out (the ciphertext, digest and output
    # buffers are reused); the copy-out waits for the receiver.
    # With several copy streams per direction, the clips take them in turn; a clip's copy-out stream is the
    # one of its host buffer (clips that share a buffer share its stream, so their copies stay in order).
    h2ds = [torch.cuda.Stream() for _ in range(args.copy_streams)]
    d2hs = [torch.cuda.Stream() for _ in range(args.copy_streams)]
    clip_no = [0]
    WW = args.worker_window if 0 < args.worker_window < len(slots) else 0
    KEEP = max(2, WW)
    last = [None] * KEEP     # slots of the previous clips, oldest first: the chaining state advances clip after clip

    def round_trip(sl, e2e=False):
        prev, prev2 = last[-1], last[-2]
        if e2e:
            k_clip = clip_no[0]
            clip_no[0] += 1
            if n_out:
                ob = k_clip % n_out
                out_buf, d2h = host_outs[ob], d2hs[ob % len(d2hs)]
                e2e_out_used.add(ob)
            else:
                out_buf, d2h = sl.host_out, d2hs[sl.index % len(d2hs)]
            h2d = h2ds[k_clip % len(h2ds)]
            if sl.used:
                h2d.wait_event(sl.cipher_ready)
            with torch.cuda.stream(h2d):
                sl.src_all.copy_(host, non_blocking=True)
            sl.h2d_done.record(h2d)
            sl.tx.wait_event(sl.h2d_done)
        if sl.used:
            sl.tx.wait_event(sl.rx_done)
        # The digest stage (integer work) of this clip runs at once, during the previous clip's keystreams
        # (binary64 work).  This clip's LHCS_m waits for the chaining state and, by --gate, for:
        #   permute:   the previous clip's ciphertext and decrypted frames (all of its work);
        #   keystream: the previous clip's two keystreams (its permutations overlap this LHCS_m);
        #   chain:     nothing more (this clip's chaotic stage overlaps the previous clip's);
        #   window:    the keystreams of the clip before the previous one (at most two clips' keystreams
        #              share the FP64 pipes, while a third clip's digest stage and LHCS_m run ahead).
        # Events of this clip's own slot would alias (they are re-recorded by this very round trip), so with
        # too few clips in flight a gate falls back to `permute`.
        gate = args.gate
        if gate == "window" and (prev2 is None or prev2 is sl):
            gate = "chain"
        if prev is sl:
            gate = "permute"
        if prev is None:
            ew, dw = [], []
        elif gate == "permute":
            ew, dw = [prev.enc_master, prev.cipher_ready], [prev.dec_done]
        elif gate == "keystream":
            ew, dw = [prev.enc_master, prev.enc_ks, prev.dec_ks], [prev.dec_master, prev.enc_ks, prev.dec_ks]
        elif gate == "window":
            ew = [prev.enc_master, prev2.enc_ks, prev2.dec_ks]
            dw = [prev.dec_master, prev2.enc_ks, prev2.dec_ks]
        else:
            ew, dw = [prev.enc_master], [prev.dec_master]
        # Worker window: this clip's workers start once the workers of clip k - W are done; its digest stage
        # and LHCS_m do not wait, so they run while W clips' workers fill the FP64 pipes.
        wslot = last[-WW] if WW else None
        if wslot is sl:
            wslot = None
        ewk, dwk = ([wslot.enc_ks], [wslot.dec_ks]) if wslot is not None else ([], [])
        enc.encrypt_frames(sl.enc_items, sl.tx, wait_events=ew, master_event=sl.enc_master,
                           digest_event=sl.digests_ready, keystream_event=sl.enc_ks, worker_wait_events=ewk)
        sl.cipher_ready.record(sl.tx)
        dec.decrypt_frames(sl.dec_items, sl.rx, wait_events=[sl.digests_ready] + dw, master_event=sl.dec_master,
                           data_events=[sl.cipher_ready], keystream_event=sl.dec_ks, worker_wait_events=dwk)
        sl.dec_done.record(sl.rx)             # before the copy-out: gates the next clip's receiver
        if e2e:
            d2h.wait_event(sl.dec_done)
            with torch.cuda.stream(d2h):
                out_buf.copy_(sl.dec_all, non_blocking=True)
                sl.host_dig.copy_(sl.digs, non_blocking=True)
            sl.e2e_used = True
            sl.rx_done.record(d2h)
        else:
            sl.rx_done.record(sl.rx)
        sl.used = True
        last.append(sl)
        del last[:-KEEP]

    def timed_steps(nsteps, inflight, e2e=False):
        """K round trips with up to `inflight` clips in flight; device time between two events on
        `stream` (every slot stream waits on the first, the second waits on every slot)."""
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev0.record(stream)
        for sl in slots[:inflight]:
            sl.tx.wait_event(ev0)
            sl.rx.wait_event(ev0)
        for k in range(nsteps):
            round_trip(slots[k % inflight], e2e)
        for sl in slots[:inflight]:
            stream.wait_event(sl.rx_done)
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        barrier()
        return ev0, ev0.elapsed_time(ev1), wall

    INF = len(slots)
    for k in range(max(args.warmup, 3)):
        round_trip(slots[k % INF])
    torch.cuda.synchronize()
    verified = all(torch.equal(sl.decs[t], sl.srcs[t]) for sl in slots if sl.used for t in range(FRAMES))

    # ---- one clip in flight (the sender's next clip waits for the receiver), when the headline has more
    ms_one = timed_steps(args.steps, 1)[1] if INF > 1 else None

    # ---- the binary64 peak of this GPU, measured in this run (the keystream roofline's denominator)
    fp64 = {"skipped": "--no-probe"}
    if not args.no_probe:
        try:
            fp64 = run_fp64_probe(fhd, torch, dev, local)
        except Exception as exc:   # noqa: BLE001 -- report, fall back to the recorded figure
            fp64 = {"error": repr(exc)}

    # ---- device-resident timed region, repeated; per-kernel events on the launch streams in every
    # repeat.  value = the median repeat (its spans and kernel sums feed the rooflines); min and max reported.
    from paper_2505_07158_gb300 import replicas
    enc.profile(True)
    dec.profile(True)
    reps = []
    l0 = fhd.fhd_launch_count()
    with ClockSampler(local) as clk:
        for r in range(max(1, args.repeats)):
            origin, ms_r, _ = timed_steps(args.steps, INF)
            if r == 0:
                launches = fhd.fhd_launch_count() - l0
            es, ds = enc.profile_spans(origin), dec.profile_spans(origin)
            pr = {}
            for c in (enc, dec):
                for k, (ms, n) in c.profile_read().items():
                    a = pr.setdefault(k, [0.0, 0])
                    a[0] += ms
                    a[1] += n
            reps.append((replicas.max_over_ranks(ms_r, device=dev), es, ds, pr))
    enc.profile(False)
    dec.profile(False)
    order = sorted(range(len(reps)), key=lambda i: reps[i][0])
    ms_total, enc_spans, dec_spans, prof = reps[order[len(order) // 2]]
    rep_values = [world * FRAMES * args.steps / (r[0] / 1000.0) for r in reps]
    spans = enc_spans + dec_spans
    if args.spans and rank == 0:
        with open(args.spans, "w") as fh:
            json.dump({"ms_total": ms_total, "steps": args.steps, "inflight": INF,
                       "sender": enc_spans, "receiver": dec_spans}, fh)
    ms_step = ms_total / args.steps
    value = replicas.job_throughput(FRAMES * args.steps, ms_total, world)
    ms_one = replicas.max_over_ranks(ms_one, device=dev) if ms_one is not None else ms_total

    def busy_ms(kind):
        """Union of the launch spans of one kind of kernel (ms)."""
        iv = sorted((a, b) for k, a, b in spans if k == kind)
        tot, cur = 0.0, None
        for a, b in iv:
            if cur is None or a > cur[1]:
                if cur is not None:
                    tot += cur[1] - cur[0]
                cur = [a, b]
            else:
                cur[1] = max(cur[1], b)
        return tot + (cur[1] - cur[0] if cur else 0.0)

    # ---- end to end through the public API with pinned host buffers
    # Repeated like the device-resident region (the pipeline's placement varies from region to region): the
    # median repeat is the value, min and max reported.
    round_trip(slots[0], e2e=True)
    torch.cuda.synchronize()
    e2e_reps = []
    for _ in range(max(1, args.repeats)):
        _, e2e_dev_ms, e2e_wall = timed_steps(args.steps, INF, e2e=True)
        e2e_reps.append((replicas.max_over_ranks(max(e2e_dev_ms, 1000 * e2e_wall) / args.steps, device=dev),
                         e2e_dev_ms / args.steps, 1000 * e2e_wall / args.steps))
    e2e_values = [world * FRAMES / (r[0] / 1000.0) for r in e2e_reps]   # in the order the regions ran
    e2e_reps.sort()
    e2e_ms, e2e_dev, e2e_wall_ms = e2e_reps[len(e2e_reps) // 2]
    e2e_parts = {"device_ms_per_step": e2e_dev, "wall_ms_per_step": e2e_wall_ms,
                 "repeats": {"n": len(e2e_reps), "value": "median",
                             "min": world * FRAMES / (e2e_reps[-1][0] / 1000.0),
                             "max": world * FRAMES / (e2e_reps[0][0] / 1000.0), "values": e2e_values}}
    e2e_ok = (all(torch.equal(host_outs[b], host) for b in e2e_out_used) if n_out else
              all(torch.equal(sl.host_out, host) for sl in slots if sl.e2e_used))

    # ---- plain path: one call per frame (the paper's per-frame loop), one CUDA stream
    sl0 = slots[0]
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for t in range(FRAMES):
        enc.encrypt_frames([sl0.enc_items[t]], stream)
        dec.decrypt_frames([sl0.dec_items[t]], stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    plain_fps = FRAMES / (ev0.elapsed_time(ev1) / 1000.0)

    # ---- every kernel alone: one call each way for the clip on one CUDA stream, nothing else running
    # (the per-kernel rooflines of the kernels that overlap others in the timed run)
    torch.cuda.synchronize()
    enc.profile(True)
    dec.profile(True)
    enc.encrypt_frames(sl0.enc_items, stream)
    dec.decrypt_frames(sl0.dec_items, stream)
    torch.cuda.synchronize()
    alone = {}
    for c in (enc, dec):
        for k, (ms, n) in c.profile_read().items():
            a = alone.setdefault(k, [0.0, 0])
            a[0] += ms
            a[1] += n
    enc.profile(False)
    dec.profile(False)
    alone_ok = all(torch.equal(sl0.decs[t], sl0.srcs[t]) for t in range(FRAMES))
    # the clip's encryption alone on a fresh stream through each route of the confusion + XOR (the single
    # gather pass and the row pass + column pass): launch time of each, and equal ciphertexts
    routes = {}
    for route in ("single_pass", "two_pass"):
        fhd.fhd_set_encrypt_route(route)
        try:
            tmp = fhd.Cipher(key, n_workers=N_WORKERS)
            tmp.set_partition(False)
            tmp.set_layout(args.layout)
            tsid = tmp.open_stream()
            outs = [torch.empty_like(x) for x in sl0.srcs]
            items = [(tsid, sl0.srcs[t], outs[t], torch.empty(32, dtype=torch.uint8, device=dev))
                     for t in range(FRAMES)]
            tmp.profile(True)
            tmp.encrypt_frames(items, stream)
            torch.cuda.synchronize()
            ms_r, n_r = tmp.profile_read()["encrypt"]
            tmp.close()
        finally:
            fhd.fhd_set_encrypt_route(args.encrypt_route)
        routes[route] = {"ms": ms_r / max(n_r, 1), "launches": n_r, "outs": outs}
    routes_equal = all(torch.equal(a, b) for a, b in zip(routes["single_pass"]["outs"], routes["two_pass"]["outs"]))

    # ---- roofline of the dominant kernel (largest share of device time)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", HBM_PEAK_FALLBACK)
    N = HGT * WID * CH
    per_step_frames = FRAMES
    kern = {}
    busy = sum(v[0] for v in prof.values()) or 1.0
    for k, (ms, n) in prof.items():
        if n:
            kern[k] = {"ms_per_step": ms / args.steps, "launches_per_step": n / args.steps,
                       "avg_launch_ms": ms / n, "share": ms / busy}
    chain_steps = worker_steps(HGT, WID, CH, N_WORKERS) * per_step_frames   # per keystream launch (one per call)
    master_steps = 2 * N_WORKERS * per_step_frames

    if "peak_tops" in fp64:
        fp64_peak = fp64["peak_tops"]
        fp64_source = (f"fp64_probe leg of this run: binary64 lane-ops/s of the library's probe kernel at "
                       f"{fp64['best_warps_per_subpartition']} warps per sub-partition (best of 1-8)")
    else:
        fp64_peak = FP64_PEAK_TOPS_FALLBACK
        fp64_source = "fallback: 1.684 lane-op/clk/SM x 152 SMs x 2.07 GHz (probe did not run)"

    def fp64_roof(k, steps_per_launch):
        # Launches of one kind overlap (sender and receiver, clips in flight): achieved = algorithmic
        # ops of all its launches / the union of their spans; per launch for reference.
        n_l = kern[k]["launches_per_step"] * args.steps
        busy = busy_ms(k)
        ach = n_l * steps_per_launch * RK4_FP64_OPS / (busy / 1000.0) / 1e12
        ms = kern[k]["avg_launch_ms"]
        tpf = TRAFFIC_PER_FRAME.get(k)
        return {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": ach / fp64_peak, "traffic": tpf * per_step_frames if tpf is not None else None,
                "peak_source": fp64_source,
                "per_launch_units": f"{steps_per_launch} RK4 chain steps x {RK4_FP64_OPS} binary64 ops",
                "busy_ms_per_step": busy / args.steps,
                "achieved_per_launch": steps_per_launch * RK4_FP64_OPS / (ms / 1000.0) / 1e12,
                "timing": "ops of all launches / union of their CUDA-event spans (launches overlap)"}

    def hbm_roof(k):
        ms = alone[k][0] / alone[k][1]          # launch alone (see above)
        ach = 2 * N * per_step_frames / (ms / 1000.0) / 1e9
        tpf = TRAFFIC_PER_FRAME.get(k)
        return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": tpf * per_step_frames if tpf is not None else None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback",
                "per_launch_units": f"{per_step_frames} frames x 2N bytes (one frame read + one frame written)",
                "timing": "one launch with nothing else running (in the timed run it overlaps the keystreams)",
                "ms_per_launch_alone": ms, "ms_per_launch_in_timed_run": kern[k]["avg_launch_ms"]}

    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    def traj_roof(k):
        # One chain per frame, strictly sequential: the launch lasts its longest chain, whose warp issues 27
        # binary64 instructions per step back to back on one sub-partition's binary64 pipe.  achieved = the
        # binary64 lane-operations that warp issues per second (steps x 27 x 32 / launch time alone), peak =
        # one sub-partition's share of the measured binary64 peak: frac is how close the chain runs to the
        # pipe's own rate.  The whole GPU's binary64 fraction (algorithmic ops of all launches over the union
        # of their spans) is reported beside it.
        steps = traj_steps(HGT, WID, CH, N_WORKERS)
        ms = alone[k][0] / alone[k][1]
        sp_peak = fp64_peak * 1e12 / (sms * 4) / 1e9
        ach = steps * RK4_FP64_INSTR * 32 / (ms / 1000.0) / 1e9
        n_l = kern[k]["launches_per_step"] * args.steps
        gpu_ach = n_l * steps * per_step_frames * RK4_FP64_OPS / (busy_ms(k) / 1000.0) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": sp_peak, "unit": "Gop/s (binary64 lane-ops, one sub-partition)",
                "frac": ach / sp_peak, "traffic": TRAFFIC_TRAJ_PER_FRAME * per_step_frames,
                "peak_source": fp64_source + f", divided by {sms} SMs x 4 sub-partitions",
                "per_launch_units": f"{per_step_frames} frames x one trajectory of {steps} RK4 steps "
                                    f"({RK4_FP64_INSTR} binary64 warp instructions each) + the D/B emission",
                "timing": "one launch (trajectory + emission) with nothing else running",
                "ms_per_launch_alone": ms, "ms_per_launch_in_timed_run": kern[k]["avg_launch_ms"],
                "step_cycles_alone": (ms / 1000.0) * (clocks_mhz or 0) * 1e6 / steps if clocks_mhz else None,
                "gpu_binary64_frac": gpu_ach / fp64_peak,
                "gpu_binary64_note": f"{steps} steps x {RK4_FP64_OPS} ops per frame, all launches over the union "
                                     "of their spans, against the whole GPU's measured peak: the route needs "
                                     "one chain per frame, so the pipes stay mostly idle"}

    roofs = {}
    clocks_mhz = clk.summary().get("sm_mhz")
    if "keystream" in kern:
        roofs["keystream"] = (traj_roof("keystream") if args.keystream_route == "trajectory"
                              else fp64_roof("keystream", chain_steps))
    if "master" in kern:
        roofs["master"] = fp64_roof("master", master_steps)
        roofs["master"]["achieved_per_launch_alone"] = (master_steps * RK4_FP64_OPS /
                                                         (alone["master"][0] / alone["master"][1] / 1000.0) / 1e12)
    if "encrypt" in kern:
        roofs["encrypt"] = hbm_roof("encrypt")
    if "decrypt" in kern:
        roofs["decrypt"] = hbm_roof("decrypt")
    if "sha" in kern:
        ms = alone["sha"][0] / alone["sha"][1]
        blocks = sha_blocks(N, N_WORKERS) * per_step_frames
        ach = N * per_step_frames / (ms / 1000.0) / 1e9
        roofs["sha"] = {"bound": "latency", "achieved": ach, "unit": "GB/s hashed",
                        "compressions_per_launch": blocks,
                        "note": f"{N_WORKERS} sequential messages per frame: one thread each"}
    dominant = max(kern, key=lambda k: kern[k]["share"]) if kern else None

    extras = {} if (args.no_extras or world > 1) else run_extras(args, rank, fhd, torch)

    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            v, n_done, el, cores = cpu_oracle_sample(args.cpu_seconds, 0)
            cpu = {"value": v, "unit": "frames/s", "cores": cores, "kind": "oracle",
                   "sample": f"{n_done} 1080p frame round trips in {el:.1f} s on {cores} host cores, one chained "
                             f"stream per core, single-threaded C oracle each (bit-matrix confusion, RK4 in binary64)"}
        clocks = clk.summary()
        line = {
            "metric": "1080p RGB frames/s (encrypt + decrypt round trip)", "value": value, "unit": "frames/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
            "repeats": {"n": len(rep_values), "steps_each": args.steps, "value": "median",
                        "min": min(rep_values), "max": max(rep_values), "values": rep_values},
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8+f64",
            "data": "synthetic",
            "config": {"workload": "30-frame 1920x1080x3 gradient+noise clip (sigma 8, 2 px/frame), one stream "
                                   "per GPU, n=32 workers, RK4 h=0.01; per step encrypt_frames on the sender's CUDA stream and "
                                   "decrypt_frames on the receiver's (its chaotic stage waits for the digests, its "
                                   "inverse permutation for the ciphertext)",
                       "clips_in_flight": INF, "next_clip_gate": args.gate, "worker_window": WW,
                       "int_mix_per8": args.int_mix, "worker_smem_bytes": args.worker_smem,
                       "worker_layout": args.layout, "worker_warps_per_cta": args.worker_cta,
                       "encrypt_route": args.encrypt_route, "keystream_route": args.keystream_route,
                       "e2e_copy_streams_per_direction": args.copy_streams,
                       "e2e_host_out_buffers": n_out or "one per clip in flight",
                       "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS"),
                       "sm_partition": {"lhcs_m_sms": enc.partition()[0], "other_sms": enc.partition()[1],
                                        "digest_stage_own_sms": bool(args.digest_partition and not args.no_partition)},
                       "frames_per_step": FRAMES * world, "l2": "inputs larger than L2 (~560 MB live per step)",
                       "parallelism": f"replicas x{world} (independent streams)",
                       "strip_width": tuned[f"{HGT}x{WID}x{CH}"]["P"], "row_band": tuned[f"{HGT}x{WID}x{CH}"]["RB"],
                       "permute_cta_threads": list(fhd.fhd_cta_threads(HGT, WID, CH)),
                       "tile_source": tuned[f"{HGT}x{WID}x{CH}"]["source"], "work_split_source": split_source},
            "verified_round_trip": bool(verified) and bool(e2e_ok) and bool(alone_ok),
            "kernels_alone_ms": {k: v[0] / v[1] for k, v in alone.items() if v[1]},
            "e2e": {"value": world * FRAMES / (e2e_ms / 1000.0), "unit": "frames/s",
                    "h2d_bytes_per_step": FRAMES * N, "d2h_bytes_per_step": FRAMES * N + FRAMES * 32, **e2e_parts},
            "plain_per_frame_fps": plain_fps,
            "one_clip_in_flight": ({"value": world * FRAMES / (ms_one / args.steps / 1000.0), "unit": "frames/s",
                                    "ms_per_step": ms_one / args.steps} if INF > 1 else None),
            "gpu_launches": int(launches),
            "clocks": clocks,
            "roofline": dict(roofs[dominant], kernel=dominant) if dominant in roofs else None,
            "fp64_probe": fp64,
            "roofline_fused_encrypt": roofs.get("encrypt"),
            "encrypt_routes_alone": {"single_pass_ms": routes["single_pass"]["ms"], "single_pass_launches": routes["single_pass"]["launches"],
                                     "two_pass_ms": routes["two_pass"]["ms"], "two_pass_launches": routes["two_pass"]["launches"],
                                     "ciphertexts_equal": bool(routes_equal),
                                     "frames": FRAMES, "note": "one encrypt_frames call of the clip on a fresh stream each"},
            "kernels": kern,
            "kernel_roofs": roofs,
            "cpu_baseline": cpu,
            **extras,
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


MIXED = [(480, 640, 3), (720, 1280, 3), (1080, 1920, 3), (2160, 3840, 3)]
SERVE_RES = [(480, 640, 3), (720, 1280, 3), (1080, 1920, 3)]


EXTRAS = ("batched", "serving", "sweep", "digest", "stats", "stress")


def run_extras(args, rank, fhd, torch):
    """The other workloads, by --extras: the batched mixed-resolution launches (64 frames), the serving loop,
    the worker-count sweep, the digest modes, the frame statistics and the 8K stress round trip."""
    want = set(args.extras.split(",")) if args.extras else set()
    out = {}
    if "batched" in want:
        out["batched_mixed64"] = run_batched(rank, fhd, torch)
    if "serving" in want:
        out["serving"] = run_serving(args, rank, fhd, torch)
    if "sweep" in want:
        out["worker_count_sweep"] = run_n_sweep(rank, fhd, torch)
    if "digest" in want:
        out["digest_modes"] = run_digest_modes(rank, fhd, torch)
    if "stats" in want:
        out["frame_statistics"] = run_stats(rank, fhd, torch)
    if "stress" in want and not args.no_stress:
        out["stress_8k"] = run_stress(rank, fhd, torch)
    return out


def run_batched(rank, fhd, torch):
    """64 frames, 16 each of VGA, 720p, 1080p, 4K, one stream (own key) per frame: the seven-kernel batched
    calls as one CUDA graph per direction, the same frames one call per frame, and the persistent round trip
    (one launch for both sides) in a CUDA graph."""
    from paper_2505_07158_gb300 import autotune, batching
    dev = torch.device("cuda", torch.cuda.current_device())
    autotune.tune(MIXED)
    shapes = [s for s in MIXED for _ in range(16)]
    frames = [torch.from_numpy(si.gradient_frame(*s, t=k, seed=rank + 11)).to(dev) for k, s in enumerate(shapes)]
    keys = [si.key(1000 * (rank + 1) + k) for k in range(len(shapes))]
    enc = fhd.Cipher(keys[0], n_workers=N_WORKERS)
    enc_items, dec_items, dec = batching.mixed_batch(shapes, keys, enc, frames, dev)
    g_enc = batching.GraphedCall(enc, enc_items, encrypt=True)
    g_dec = batching.GraphedCall(dec, dec_items, encrypt=False)
    g_enc.replay(); g_dec.replay()
    torch.cuda.synchronize()
    ok = all(torch.equal(it[2], fr) for it, fr in zip(dec_items, frames))
    reps = 3
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        g_enc.replay()
        g_dec.replay()
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    nbytes = sum(int(np.prod(s)) for s in shapes)
    # the same 64 frames one call per frame (plain path)
    torch.cuda.synchronize()
    a.record()
    for ei, di in zip(enc_items, dec_items):
        enc.encrypt_frames([ei])
        dec.decrypt_frames([di])
    b.record()
    b.synchronize()
    plain_ms = a.elapsed_time(b)
    # the same batch as one persistent round-trip launch (sender and receiver), captured in a CUDA graph
    pers = batching.PersistentRoundTrip(enc, dec, enc_items, dec_items, graph=True)
    pers.replay()
    torch.cuda.synchronize()
    pers_ok = all(torch.equal(it[2], fr) for it, fr in zip(dec_items, frames))
    a.record()
    for _ in range(reps):
        pers.replay()
    b.record()
    b.synchronize()
    pers_ms = a.elapsed_time(b) / reps
    enc.sync_status()
    dec.sync_status()
    # timeline of the last launch: per frame size, when its digests, LHCS_m, keystreams and last
    # permutation task were done (median over the 16 frames of the size; ms after the launch's start)
    tr = enc.persistent_trace(len(shapes))
    timeline = {}
    for q, s in enumerate(MIXED):
        t = tr[16 * q:16 * q + 16]
        done = np.maximum(t[:, 3:5].max(axis=1), t[:, 7:9].max(axis=1))
        timeline[f"{s[0]}x{s[1]}x{s[2]}"] = {
            "digest": float(np.median(t[:, 0])), "lhcs_m": float(np.median(t[:, 1])),
            "keystreams": float(np.median(np.maximum(t[:, 2], t[:, 6]))), "round_trip_done": float(np.median(done)),
            "round_trip_done_max": float(done.max())}
    res = {
        "workload": "64 frames (16 x 640x480, 720p, 1080p, 2160p x3 uint8), one stream and key per frame, "
                    "encrypt + decrypt as two CUDA-graph replays",
        "frames_per_s": len(shapes) / (ms / 1000.0), "GB_per_s": 2 * nbytes / (ms / 1000.0) / 1e9,
        "ms_per_batch_round_trip": ms, "plain_per_frame_frames_per_s": len(shapes) / (plain_ms / 1000.0),
        "kernels_per_replay": g_enc.kernels_per_replay + g_dec.kernels_per_replay, "round_trip_ok": bool(ok),
        "persistent": {"frames_per_s": len(shapes) / (pers_ms / 1000.0), "ms_per_batch_round_trip": pers_ms,
                       "GB_per_s": 2 * nbytes / (pers_ms / 1000.0) / 1e9, "kernels_per_replay": 1,
                       "round_trip_ok": bool(pers_ok), "speedup_vs_graph_replays": ms / pers_ms,
                       "timeline_ms": timeline,
                       "note": "cipher_round_trip_persistent: one launch for both sides, captured in a CUDA graph"},
        "strip_widths": {f"{h}x{w}x{c}": fhd.fhd_strip_width(h, w, c) for (h, w, c) in MIXED}}
    enc.close(); dec.close()
    del frames, enc_items, dec_items, g_enc, g_dec, pers
    torch.cuda.empty_cache()
    return res


def run_serving(args, rank, fhd, torch):
    """32 streams, resolutions drawn from VGA / 720p / 1080p, Poisson arrivals at 24, 30 and 60 fps."""
    from paper_2505_07158_gb300 import serving
    dev = torch.device("cuda", torch.cuda.current_device())
    g = si.rng(77 + rank)
    sshapes = [SERVE_RES[int(g.integers(3))] for _ in range(32)]
    skeys = [si.key(5000 + 100 * rank + k) for k in range(32)]
    pool = {s: [torch.from_numpy(si.gradient_frame(*s, t=t, seed=5)).to(dev) for t in range(4)] for s in SERVE_RES}
    serve = {}
    for fps in (24.0, 30.0, 60.0):
        st, srv = serving.run(skeys, sshapes, pool, fps=fps, duration=args.serve_seconds, seed=int(fps),
                              n_workers=N_WORKERS, budget_bytes=20 << 30)
        srv.close()
        serve[f"{int(fps)}fps"] = st
    st, srv = serving.run(skeys, sshapes, pool, fps=30.0, duration=min(args.serve_seconds, 3.0), seed=30,
                          n_workers=N_WORKERS, budget_bytes=20 << 30, mode="plain")
    srv.close()
    serve["plain_30fps"] = st
    res = {"workload": f"32 streams, resolutions uniform over 640x480 / 1280x720 / 1920x1080 x3, "
                                  f"Poisson arrivals, 20 GB HBM budget, {args.serve_seconds:g} s per rate "
                                  f"(plain: one frame per call, one CUDA stream)", **serve}
    del pool
    torch.cuda.empty_cache()
    return res


def run_stats(rank, fhd, torch, frames=30, reps=10):
    """Frame statistics (Sec. III, IV-B) over a 30-frame 1080p batch: the streaming passes against HBM
    (histogram statistics read N bytes per frame, NPCR/UACI 2N), and the sampled ones (10,000 pairs per
    direction, 30 blocks of 44 x 44 per frame) as latencies.  Inputs are device-generated uniform frames,
    larger than L2 (187 MB per batch)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device=dev)
    g.manual_seed(rank + 31)
    a = torch.randint(0, 256, (frames, HGT, WID, CH), dtype=torch.uint8, device=dev, generator=g)
    b = torch.randint(0, 256, (frames, HGT, WID, CH), dtype=torch.uint8, device=dev, generator=g)
    pairs = torch.stack([torch.randint(0, HGT - 1, (frames, 3, 10000), device=dev, generator=g),
                         torch.randint(0, WID - 1, (frames, 3, 10000), device=dev, generator=g)], dim=-1).int()
    cells = [(44 * i, 44 * j) for i in range(HGT // 44) for j in range(WID // 44)]
    pick = torch.stack([torch.randperm(len(cells), device=dev, generator=g)[:30] for _ in range(frames)])
    blocks = torch.tensor(cells, dtype=torch.int32, device=dev)[pick]
    calls = {"histogram_variance_chi2_entropy": (lambda: fhd.fhd_stats_histogram(a), a.numel()),
             "npcr_uaci": (lambda: fhd.fhd_stats_npcr_uaci(a, b), 2 * a.numel()),
             "correlation_10000_pairs_x3": (lambda: fhd.fhd_stats_correlation(a, pairs), None),
             "local_entropy_30_blocks": (lambda: fhd.fhd_stats_local_entropy(a, blocks, 44), None)}
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", HBM_PEAK_FALLBACK)
    res = {"workload": f"{frames} x 1920x1080x3 uint8 (device-generated uniform), statistics per frame and channel"}
    for name, (fn, nbytes) in calls.items():
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        r = {"ms_per_batch": ms, "frames_per_s": frames / (ms / 1000.0)}
        if nbytes:
            ach = nbytes / (ms / 1000.0) / 1e9
            r["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                             "bytes_per_batch": nbytes}
        res[name] = r
    _, st = fhd.fhd_stats_histogram(a[:1])
    res["uniform_frame_0"] = {"chi2": st[0, :, 1].tolist(), "entropy": st[0, :, 2].tolist()}
    return res


def run_n_sweep(rank, fhd, torch, ns=(32, 128, 512), steps=3):
    """The same 30-frame 1080p round trip with other worker counts n.  n is a protocol parameter both ends
    must share (Sec. V): more workers mean more, shorter sub-frame messages and chaotic chains."""
    dev = torch.device("cuda", torch.cuda.current_device())
    clip = torch.from_numpy(si.clip(FRAMES, HGT, WID, CH, seed=rank + 3)).to(dev)
    res = {}
    for n in ns:
        key = si.key(700 + n)
        enc, dec = fhd.Cipher(key, n_workers=n), fhd.Cipher(key, n_workers=n)
        sid, rid = enc.open_stream(), dec.open_stream()
        E = torch.empty_like(clip)
        R = torch.empty_like(clip)
        H = torch.empty((FRAMES, 32), dtype=torch.uint8, device=dev)
        ei = [(sid, clip[t], E[t], H[t]) for t in range(FRAMES)]
        di = [(rid, E[t], R[t], H[t]) for t in range(FRAMES)]
        enc.encrypt_frames(ei); dec.decrypt_frames(di)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            enc.encrypt_frames(ei)
            dec.decrypt_frames(di)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        res[str(n)] = {"frames_per_s": FRAMES / (ms / 1000.0), "ms_per_step": ms,
                       "round_trip_ok": bool(torch.equal(R, clip))}
        enc.close(); dec.close()
    return {"workload": "30-frame 1080p clip round trip (as the headline) with n workers", **res}


def run_digest_modes(rank, fhd, torch, reps=10, steps=3):
    """The frame digest and its transport.  Modes: the paper's XOR fold sent as computed; the tree digest
    (SHA-256 of the concatenated sub-frame digests); the fold sent masked (H xor M, M from the chaining
    state; both options of this library).  Per mode: the digest stage alone on the 30-frame 1080p clip, the
    clip's round trip on one CUDA stream (as the n sweep) with its LHCS_m time, the receiver-side check, and
    the digests of encrypt_frames against the standalone digest entry point (the oracle comparisons of
    every mode are in the GPU tests)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    clip_np = si.clip(FRAMES, HGT, WID, CH, seed=rank + 5)
    clip = torch.from_numpy(clip_np).to(dev)
    flat = clip.reshape(-1)
    res, ok = {}, True
    for name, mode, transport in (("xor", "xor", "plain"), ("tree", "tree", "plain"), ("xor_masked", "xor", "masked")):
        dig = fhd.fhd_frame_digest(flat, n=N_WORKERS, count=FRAMES, mode=mode)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fhd.fhd_frame_digest(flat, n=N_WORKERS, count=FRAMES, out=dig, mode=mode)
        b.record()
        b.synchronize()
        digest_ms = a.elapsed_time(b) / reps
        key = si.key(900 + rank)
        enc = fhd.Cipher(key, n_workers=N_WORKERS, digest_mode=mode, digest_transport=transport)
        dec = fhd.Cipher(key, n_workers=N_WORKERS, digest_mode=mode, digest_transport=transport)
        sid, rid = enc.open_stream(), dec.open_stream()
        E, R = torch.empty_like(clip), torch.empty_like(clip)
        H = torch.empty((FRAMES, 32), dtype=torch.uint8, device=dev)
        ei = [(sid, clip[t], E[t], H[t]) for t in range(FRAMES)]
        di = [(rid, E[t], R[t], H[t]) for t in range(FRAMES)]
        enc.encrypt_frames(ei); dec.decrypt_frames(di)
        torch.cuda.synchronize()
        # the receiver leaves the unmasked digest H in place: it must equal the standalone digest
        ok = ok and torch.equal(H, dig)
        enc.profile(True)
        dec.profile(True)
        a.record()
        for _ in range(steps):
            enc.encrypt_frames(ei)
            dec.decrypt_frames(di)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        prof = [c.profile_read() for c in (enc, dec)]
        enc.profile(False)
        dec.profile(False)
        verified = dec.verify_frames(di)
        res[name] = {"digest_ms_per_clip": digest_ms, "round_trip_frames_per_s": FRAMES / (ms / 1000.0),
                     "lhcs_m_ms_per_clip_each_side": sum(p["master"][0] for p in prof) / (2 * steps),
                     "round_trip_ok": bool(torch.equal(R, clip)), "verify_ok": bool(int(verified.min()) == 1)}
        enc.close(); dec.close()
    return {"workload": "30 x 1080p clip: the digest stage alone (n = 32), and the round trip on one CUDA stream",
            **res, "digests_match_standalone_digest": bool(ok)}


def run_stress(rank, fhd, torch, frames=256):
    """256 frames of 7680x4320x3 (uniform and gradient+noise halves, generated on the device), one stream,
    encrypt then decrypt in one call each; round trip, digests against the standalone digest entry point,
    permutation rooflines (an 8K frame against the oracle is in the GPU tests)."""
    from paper_2505_07158_gb300 import autotune
    dev = torch.device("cuda", torch.cuda.current_device())
    h, w, C = 4320, 7680, 3
    autotune.tune([(h, w, C)])
    g = torch.Generator(device=dev)
    g.manual_seed(8000 + rank)
    src = []
    ii = torch.arange(h, device=dev, dtype=torch.float32)[:, None]
    jj = torch.arange(w, device=dev, dtype=torch.float32)[None, :]
    for t in range(frames):
        if t < frames // 2:
            src.append(torch.randint(0, 256, (h, w, C), dtype=torch.uint8, device=dev, generator=g))
        else:
            chans = []
            for c in range(C):
                a = (c + 1) / (C + 1)
                base = 255.0 * (a * ii / h + (1 - a) * torch.remainder(jj + 2 * t, w) / w)
                noisy = base + 8.0 * torch.randn((h, w), device=dev, generator=g)
                chans.append(torch.clamp(torch.round(noisy), 0, 255).to(torch.uint8))
            src.append(torch.stack(chans, dim=-1).contiguous())
    key = si.key(9000 + rank)
    enc, dec = fhd.Cipher(key, n_workers=N_WORKERS), fhd.Cipher(key, n_workers=N_WORKERS)
    sid, rid = enc.open_stream(), dec.open_stream()
    E = [torch.empty_like(x) for x in src]
    R = [torch.empty_like(x) for x in src]
    Hd = torch.empty((frames, 32), dtype=torch.uint8, device=dev)
    # scratch for the batch is sized by a first call on a throwaway stream of the same handles
    tmp_s, tmp_r = enc.open_stream(), dec.open_stream()
    enc.encrypt_frames([(tmp_s, src[k], E[k], Hd[k]) for k in range(min(frames, 256))])
    dec.decrypt_frames([(tmp_r, E[k], R[k], Hd[k]) for k in range(min(frames, 256))])
    torch.cuda.synchronize()
    enc.profile(True)
    dec.profile(True)
    a, b, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    a.record()
    enc.encrypt_frames([(sid, src[k], E[k], Hd[k]) for k in range(frames)])
    b.record()
    dec.decrypt_frames([(rid, E[k], R[k], Hd[k]) for k in range(frames)])
    c2.record()
    c2.synchronize()
    pe, pd = enc.profile_read(), dec.profile_read()
    enc.profile(False)
    dec.profile(False)
    ok = all(torch.equal(R[k], src[k]) for k in range(frames))
    N = h * w * C
    digest_ok = all(torch.equal(Hd[k], fhd.fhd_frame_digest(src[k].view(-1), n=N_WORKERS)[0]) for k in (0, frames - 1))
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", HBM_PEAK_FALLBACK)
    enc_ms, dec_ms = a.elapsed_time(b), b.elapsed_time(c2)
    perm_e, perm_d = pe["encrypt"][0], pd["decrypt"][0]
    res = {"workload": f"{frames} x 7680x4320x3 uint8 (uniform / gradient+noise halves, device-generated), one stream, "
                       "encrypt then decrypt, one call each",
           "round_trip_ok": bool(ok), "digests_match_standalone_digest": bool(digest_ok),
           "encrypt_ms": enc_ms, "decrypt_ms": dec_ms,
           "frames_per_s_round_trip": frames / ((enc_ms + dec_ms) / 1000.0),
           "kernel_ms": {"encrypt": {k: v[0] for k, v in pe.items() if v[1]},
                         "decrypt": {k: v[0] for k, v in pd.items() if v[1]}},
           "permute_encrypt_roofline": {"bound": "hbm", "achieved": 2 * N * frames / (perm_e / 1000.0) / 1e9,
                                        "peak": hbm, "unit": "GB/s",
                                        "frac": 2 * N * frames / (perm_e / 1000.0) / 1e9 / hbm},
           "permute_decrypt_roofline": {"bound": "hbm", "achieved": 2 * N * frames / (perm_d / 1000.0) / 1e9,
                                        "peak": hbm, "unit": "GB/s",
                                        "frac": 2 * N * frames / (perm_d / 1000.0) / 1e9 / hbm},
           "strip_width": fhd.fhd_strip_width(h, w, C)}
    enc.close()
    dec.close()
    del src, E, R
    torch.cuda.empty_cache()
    return res


def free_port() -> int:
    import socket
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def launch_ranks(n: int) -> int:
    """--gpus N without a launcher: start N copies of this command, one process per GPU (RANK = LOCAL_RANK =
    index, WORLD_SIZE = N, rendezvous on 127.0.0.1), and return the worst exit code.  Rank 0 prints the
    JSON line; the other ranks print nothing."""
    port = free_port()
    procs = []
    for r in range(n):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(n), LOCAL_WORLD_SIZE=str(n),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__), *sys.argv[1:]], env=env))
    return max(p.wait() for p in procs)


def run_dry(args):
    """The multi-process skeleton without a GPU (gloo): barrier, max-over-ranks of a per-rank time, one JSON
    line from rank 0 with the job-level count of ranks."""
    import torch
    import torch.distributed as dist
    from paper_2505_07158_gb300 import replicas
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        dist.init_process_group("gloo")
    ranks = torch.ones(1)
    if world > 1:
        dist.all_reduce(ranks)
    ms = replicas.max_over_ranks(1.0 + rank)
    if rank == 0:
        print(json.dumps({"dry_run": True, "n_gpus": world, "ranks_seen": int(ranks.item()), "max_ms": ms,
                          "value": replicas.job_throughput(FRAMES, ms, world)}))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def pick_trajectory_split(results):
    """The clips-in-flight / copy-streams candidate to keep: the best end-to-end value among those whose
    device-resident value is within 1 % of the best (the headline's limit is the stream's LHCS_m chain, so
    the device-resident values of the deeper pipelines tie).  results: {(inflight, copy_streams): (value,
    e2e)}, None for a failed run."""
    ok = {k: v for k, v in results.items() if v}
    top = max(v[0] for v in ok.values())
    near = [k for k, v in ok.items() if v[0] >= 0.99 * top]
    return max(near, key=lambda k: (ok[k][1], ok[k][0]))


def tune_trajectory_pipeline(inflights=(8, 10, 12, 16), copy_streams=(1, 2)):
    """The one-trajectory route's work split: the headline at each clips-in-flight / copy-streams candidate,
    each in its own process (120 steps, median of three timed regions)."""
    results = {}
    for inf in inflights:
        for cs in copy_streams:
            cmd = [sys.executable, os.path.abspath(__file__), "--no-extras", "--no-cpu-baseline", "--no-probe",
                   "--repeats", "3", "--keystream-route", "trajectory", "--inflight", str(inf),
                   "--copy-streams", str(cs)]
            r = subprocess.run(cmd, capture_output=True, text=True)
            lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
            d = json.loads(lines[-1]) if r.returncode == 0 and lines else None
            results[(inf, cs)] = (d["value"], d["e2e"]["value"]) if d else None
            print(f"pipeline trajectory inflight={inf} copy_streams={cs}: {results[(inf, cs)]}", flush=True)
    inf, cs = pick_trajectory_split(results)
    return {"keystream_route": "trajectory", "inflight": inf, "copy_streams": cs, "worker_window": 0,
            "frames_per_s": results[(inf, cs)][0], "e2e_frames_per_s": results[(inf, cs)][1],
            "candidates": {f"inflight {a}, copy streams {b}": v for (a, b), v in results.items()},
            "how": "bench.py headline, 120 steps, median of 3 timed regions per candidate, one process each "
                   "(frames/s, e2e frames/s); kept: the best e2e within 1 % of the best frames/s"}


def run_tune(args):
    """Tile shapes of every workload's frame sizes (timed afresh), then the clip pipeline's work split: the
    headline under each candidate setting, each in its own process (a bench run of 15 steps, median of three
    timed regions); the table goes to args.tune."""
    import torch
    from paper_2505_07158_gb300 import autotune
    torch.cuda.set_device(0)
    shapes = [(HGT, WID, CH)] + MIXED + SERVE_RES + [(4320, 7680, 3)]
    tuned = autotune.tune(sorted(set(shapes)), force=True)
    cache = autotune.load_cache()
    gpu = autotune._gpu_name()
    entries = {k: cache[gpu]["shapes"][k] for k in tuned}
    if args.keystream_route == "trajectory":
        pipeline = tune_trajectory_pipeline()
        pipeline["pairs_route"] = (autotune.pipeline_defaults() or {}).get("pairs_route")
        table = {gpu: {"shapes": entries, "pipeline": pipeline}}
        with open(args.tune, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        print(json.dumps(table))
        return 0
    grid = [("throughput", i, w) for i in (3, 4, 5, 6) for w in (2, 3, 4) if w < i] + [("latency", 5, 3)]
    results = {}
    for layout, inflight, window in grid:
        cmd = [sys.executable, os.path.abspath(__file__), "--no-extras", "--no-cpu-baseline", "--no-probe",
               "--steps", "15", "--repeats", "3", "--layout", layout, "--inflight", str(inflight),
               "--worker-window", str(window)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
        v = json.loads(lines[-1])["value"] if r.returncode == 0 and lines else None
        results[f"{layout}/{inflight}/{window}"] = v
        print(f"pipeline {layout} inflight={inflight} window={window}: {v}", flush=True)
    best = max((k for k in results if results[k]), key=lambda k: results[k])
    layout, inflight, window = best.split("/")
    # then the cap on worker CTAs per SM (dynamic shared memory per worker CTA) at the best split
    smem_results = {}
    for smem in (0, 24000, 28000, 32000, 38000):
        cmd = [sys.executable, os.path.abspath(__file__), "--no-extras", "--no-cpu-baseline", "--no-probe",
               "--steps", "15", "--repeats", "3", "--layout", layout, "--inflight", inflight,
               "--worker-window", window, "--worker-smem", str(smem)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
        smem_results[str(smem)] = json.loads(lines[-1])["value"] if r.returncode == 0 and lines else None
        print(f"pipeline {best} worker_smem={smem}: {smem_results[str(smem)]}", flush=True)
    best_smem = max((k for k in smem_results if smem_results[k]), key=lambda k: smem_results[k])
    pipeline = {"layout": layout, "inflight": int(inflight), "worker_window": int(window),
                "worker_smem": int(best_smem), "worker_smem_candidates": smem_results,
                "frames_per_s": max(results[best], smem_results[best_smem] or 0), "candidates": results,
                "how": "bench.py headline, 15 steps, median of 3 timed regions per candidate, one process each"}
    table = {gpu: {"shapes": entries, "pipeline": pipeline}}
    with open(args.tune, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print(json.dumps(table))
    return 0


def main():
    args = parse()
    if args.tune:
        return run_tune(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return launch_ranks(args.gpus)
    if args.dry_run:
        return run_dry(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
