"""bench.py --gpus N started without a launcher starts N ranks itself (one process per GPU, rendezvous on
127.0.0.1) and prints one JSON line from rank 0.  Exercised on CPU with --dry-run (gloo, no CUDA): the
line must count both ranks and carry the slowest rank's time."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gpus_2_starts_two_ranks_and_prints_one_line():
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--dry-run"],
                       capture_output=True, text=True, env=env, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    rec = json.loads(lines[0])
    assert rec["n_gpus"] == 2 and rec["ranks_seen"] == 2
    assert rec["max_ms"] == 2.0          # rank r reports 1 + r ms: the maximum is rank 1's


def test_work_split_flags_parse_and_default_to_the_tuned_table():
    """The placement and integer-mix flags parse, reject values out of range, and default to None (the tuned
    table's value, else the built-in default, is filled in at run time)."""
    sys.path.insert(0, ROOT)
    import bench
    old = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
        assert a.worker_smem is None and a.int_mix is None and a.inflight is None and a.worker_window is None
        sys.argv = ["bench.py", "--worker-smem", "28000", "--int-mix", "3", "--digest-partition"]
        a = bench.parse()
        assert a.worker_smem == 28000 and a.int_mix == 3 and a.digest_partition
        sys.argv = ["bench.py", "--int-mix", "9"]
        try:
            bench.parse()
            raise AssertionError("--int-mix 9 accepted")
        except SystemExit:
            pass
    finally:
        sys.argv = old


def test_tuned_table_carries_the_pipeline_split():
    """The committed tuned table holds, for the GPU it was measured on, the clip pipeline's split that the
    bench applies: layout, clips in flight, worker window and the cap on worker CTAs per SM."""
    with open(os.path.join(ROOT, "paper_2505_07158_gb300", "tuned.json")) as f:
        table = json.load(f)
    pipe = table["NVIDIA GB300"]["pipeline"]
    assert pipe["layout"] in ("latency", "throughput")
    assert pipe["worker_window"] < pipe["inflight"]
    assert 0 <= pipe["worker_smem"] <= 232448


def test_tuned_table_records_both_keystream_routes_and_the_trajectory_pick():
    """The table's pipeline record is the one-trajectory route's (clips in flight, copy streams), with the
    worker-pair route's own record beside it; the tuner's pick keeps the best end-to-end value among the
    candidates within 1 % of the best device-resident value, skipping failed runs."""
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "paper_2505_07158_gb300", "tuned.json")) as f:
        pipe = json.load(f)["NVIDIA GB300"]["pipeline"]
    assert pipe["keystream_route"] == "trajectory" and pipe["copy_streams"] in (1, 2, 4)
    pairs = pipe["pairs_route"]
    assert pairs["layout"] in ("latency", "throughput") and pairs["worker_window"] < pairs["inflight"]
    res = {(8, 1): (14000.0, 12000.0), (12, 2): (14460.0, 13400.0), (16, 2): (14470.0, 10000.0),
           (10, 1): None, (12, 1): (14300.0, 13900.0)}
    assert bench.pick_trajectory_split(res) == (12, 2)      # (12, 1) is more than 1 % below the best value
    res[(12, 1)] = (14400.0, 13900.0)
    assert bench.pick_trajectory_split(res) == (12, 1)
    sys.argv, old = ["bench.py"], sys.argv
    try:
        assert bench.parse().copy_streams is None            # filled in from the table at run time
    finally:
        sys.argv = old
