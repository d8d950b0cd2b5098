"""The checked build on the GPU: every computed index of the kernels' memory accesses range-checked.

`libfhdcipher_checked.so` is the library compiled with -DFHD_BOUNDS_CHECK: an access whose index fails its
check is counted in a device-side record and skipped, nothing traps.  Two things are checked here:

* a descriptor that declares one row fewer than its buffers hold (every buffer is allocated at full size,
  so no access can leave its allocation) makes the checks of the permutation fail, and the record names the
  pass and the extent;
* every GPU test of this suite (the parity tests of the digest, chaining, worker, permutation, persistent,
  batching, serving and statistics kernels, at every size they cover) passes under the checked build with
  no failed check (the autouse fixture of conftest reads the record after each test) -- run in a child
  process with FHD_CHECKED=1, so that it loads the checked library."""
import os
import subprocess
import sys

import pytest
import torch

import paper_2505_07158_gb300 as fhd

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PERMUTE_SITES = {20, 21, 22, 23, 30, 31, 32, 33}


def _checked():
    return fhd.fhd_build_flags() & fhd.FHD_BUILD_BOUNDS_CHECK


def test_selftest_records_and_skips_the_accesses_past_the_declared_extent():
    if not _checked():
        pytest.skip("default build: the checked build's tests run in the child process below")
    torch.cuda.init()
    count, site = fhd.fhd_bounds_selftest()
    # the last of 16 rows of a 16 x 64 x 3 frame: its loads in the row pass at least (one per 16-byte
    # vector of the 192-byte row), and the column pass's accesses of that row
    assert count >= 12, count
    assert site in PERMUTE_SITES, (site, fhd.fhd_bounds_site_name(site))
    assert fhd.fhd_bounds_report()["count"] == 0   # the self-test took its reading: the records are clear


def test_gpu_suite_under_the_checked_build():
    if _checked():
        pytest.skip("already the checked build")
    env = dict(os.environ, FHD_CHECKED="1")
    cmd = [sys.executable, "-m", "pytest", "-m", "gpu", "-x", "-q", "-p", "no:cacheprovider", "tests"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-25:])
    assert r.returncode == 0, tail
    assert " passed" in tail and "failed" not in tail, tail
