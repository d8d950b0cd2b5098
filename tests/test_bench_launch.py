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
