"""The C-ABI library loads and exports every symbol include/fhdcipher.h declares
(no GPU needed: only host-side logic is exercised here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fhdcipher.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2505_07158_gb300 as fhd
    return fhd.load()


def test_header_declares_the_documented_api():
    import paper_2505_07158_gb300 as fhd
    assert declared_functions() == sorted(fhd.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    import paper_2505_07158_gb300 as fhd
    out = subprocess.run(["nm", "-D", "--defined-only", fhd.library_path()], capture_output=True, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for name in declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_checked_build_exports_the_same_symbols():
    """The checked build (-DFHD_BOUNDS_CHECK) is the same library with range checks: every declared symbol,
    and a build flag that says which build it is (the default library's says 0)."""
    import paper_2505_07158_gb300 as fhd
    from paper_2505_07158_gb300 import build as b
    path = b.build(checked=True)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for name in declared_functions():
        assert name in exported, name
    checked = ctypes.CDLL(path)
    checked.fhd_build_flags.restype = ctypes.c_uint32
    assert checked.fhd_build_flags() == fhd.FHD_BUILD_BOUNDS_CHECK
    if not fhd.checked_requested():
        assert fhd.fhd_build_flags() == 0


def test_cta_threads_overrides_on_the_host(lib):
    import paper_2505_07158_gb300 as fhd
    assert fhd.fhd_cta_threads(1080, 1920, 3) == (512, 256)
    assert lib.fhd_set_cta_threads(1080, 1920, 3, 300, 0) == fhd.FHD_ERR_INVALID_ARG
    assert lib.fhd_set_cta_threads(1080, 1920, 3, 0, 64) == fhd.FHD_ERR_INVALID_ARG
    assert lib.fhd_set_cta_threads(0, 1920, 3, 256, 128) == fhd.FHD_ERR_INVALID_ARG
    fhd.fhd_set_cta_threads(37, 41, 3, 256, 0)
    assert fhd.fhd_cta_threads(37, 41, 3) == (256, 256)
    fhd.fhd_set_cta_threads(37, 41, 3, 0, 0)
    assert fhd.fhd_cta_threads(37, 41, 3) == (512, 256)


def test_int_mix_and_binary64_check_arguments(lib):
    import paper_2505_07158_gb300 as fhd
    assert lib.cipher_set_int_mix(None, 1) == fhd.FHD_ERR_INVALID_ARG
    assert lib.cipher_set_worker_smem(None, 0) == fhd.FHD_ERR_INVALID_ARG
    assert lib.fhd_binary64_check(16, 1, None, None) == fhd.FHD_ERR_INVALID_ARG
    out = (ctypes.c_uint64 * 4)()
    assert lib.fhd_binary64_check(0, 1, out, None) == fhd.FHD_ERR_INVALID_ARG
    assert lib.fhd_binary64_check((1 << 40) + 1, 1, out, None) == fhd.FHD_ERR_INVALID_ARG


def test_bounds_calls_without_a_device(lib):
    """Host-side behaviour of the bounds calls: site names, and the default build's report (all zero, no
    device call) and self-test (refused: not a checked build)."""
    import paper_2505_07158_gb300 as fhd
    assert fhd.fhd_bounds_site_name(33) == "column pass: frame store"
    assert fhd.fhd_bounds_site_name(9999) == "unknown site"
    if fhd.fhd_build_flags() == 0:
        assert fhd.fhd_bounds_report() == {"count": 0, "site": 0, "site_name": "unknown site", "index": 0,
                                           "limit": 0}
        assert lib.fhd_bounds_selftest(None, None, None) == fhd.FHD_ERR_STATE


def test_host_side_argument_checks(lib):
    import paper_2505_07158_gb300 as fhd
    out = ctypes.c_void_p()
    assert lib.cipher_init(None, None, ctypes.byref(out)) == fhd.FHD_ERR_INVALID_ARG
    assert lib.encrypt_frames(None, 1, None, None) == fhd.FHD_ERR_INVALID_ARG
    assert lib.cipher_open_stream(None, None) == fhd.FHD_ERR_INVALID_ARG
    assert lib.fhd_permute_encrypt(None, None, 4, 4, 3, None, None, None) == fhd.FHD_ERR_INVALID_ARG
    assert b"null" in lib.cipher_last_error(None)
    assert lib.fhd_set_strip_width(0, 4, 3, 8) == fhd.FHD_ERR_INVALID_ARG
    ops = ctypes.c_uint64()
    assert lib.fhd_fp64_probe(1, 16, None, ctypes.byref(ops), None) == fhd.FHD_ERR_INVALID_ARG
    assert lib.fhd_fp64_probe(9, 16, ctypes.c_void_p(16), ctypes.byref(ops), None) == fhd.FHD_ERR_INVALID_ARG
    assert lib.fhd_fp64_probe(1, 0, ctypes.c_void_p(16), ctypes.byref(ops), None) == fhd.FHD_ERR_INVALID_ARG


def test_strip_width_fits_shared_memory(lib):
    import paper_2505_07158_gb300 as fhd
    assert fhd.fhd_strip_width(1080, 1920, 3) == 64
    assert fhd.fhd_strip_width(2160, 3840, 3) == 32
    assert fhd.fhd_strip_width(4320, 7680, 3) == 16
    assert fhd.fhd_strip_width(1, 1, 1) == 1
    assert fhd.fhd_strip_width(12288, 16384, 4) >= 1
    for h, w, c in [(480, 640, 3), (720, 1280, 3), (3, 5, 3), (12288, 7, 4), (12288, 16384, 3)]:
        P = fhd.fhd_strip_width(h, w, c)
        assert P >= 1 and ((h * P * c + 15) & ~15) <= 232448


def test_host_side_checks_of_the_stream_ordering_and_placement_calls(lib):
    """The split entry points, the SM-partition and layout switches and the profile spans reject a
    null handle before touching a device, and report it through cipher_last_error."""
    import paper_2505_07158_gb300 as fhd
    ev = (ctypes.c_void_p * 1)()
    n = ctypes.c_uint32()
    assert lib.encrypt_frames_split(None, 1, None, None, None, 0, None, None, None) == fhd.FHD_ERR_INVALID_ARG
    assert lib.decrypt_frames_split(None, 1, None, None, None, 0, ev, 1, None, None) == fhd.FHD_ERR_INVALID_ARG
    assert lib.encrypt_frames_ex(None, 1, None, None, None, 0, None) == fhd.FHD_ERR_INVALID_ARG
    hk = fhd._lib.FhdSchedule()
    assert lib.encrypt_frames_sched(None, 1, None, None, ctypes.byref(hk)) == fhd.FHD_ERR_INVALID_ARG
    assert lib.decrypt_frames_sched(None, 1, None, None, None) == fhd.FHD_ERR_INVALID_ARG
    assert lib.cipher_set_partition(None, 1) == fhd.FHD_ERR_INVALID_ARG
    assert lib.cipher_get_partition(None, ctypes.byref(n), ctypes.byref(n)) == fhd.FHD_ERR_INVALID_ARG
    assert lib.cipher_set_layout(None, 0) == fhd.FHD_ERR_INVALID_ARG
    assert lib.cipher_profile_spans(None, None, 0, None, None, None, ctypes.byref(n)) == fhd.FHD_ERR_INVALID_ARG
    assert b"null" in lib.cipher_last_error(None)


def test_protocol_parameters_are_checked_before_any_device_work(lib):
    """cipher_init / cipher_init_raw validate fhd_params (worker count, step, bounds, digest mode and
    transport) before they select a device, so the errors are the same with and without a GPU."""
    import paper_2505_07158_gb300 as fhd
    from paper_2505_07158_gb300 import _lib
    h = ctypes.c_void_p()
    bad = []
    p = _lib._params(); p.digest_mode = 7; bad.append((p, b"digest_mode"))
    p = _lib._params(); p.digest_transport = 3; bad.append((p, b"digest_transport"))
    p = _lib._params(n_workers=4096); bad.append((p, b"n_workers"))
    p = _lib._params(rk4_h=2.0); bad.append((p, b"rk4_h"))
    p = _lib._params(u_bound=(20, 20, 70000, 20)); bad.append((p, b"u_bound"))
    for params, word in bad:
        assert lib.cipher_init(bytes(32), ctypes.byref(params), ctypes.byref(h)) == fhd.FHD_ERR_INVALID_ARG
        assert word in lib.cipher_last_error(None)
        assert lib.cipher_init_raw(1.0, 2.0, 3.0, 4.0, -1.0, ctypes.byref(params), ctypes.byref(h)) == \
            fhd.FHD_ERR_INVALID_ARG
    assert set(_lib.DIGEST_MODES.values()) == {0, 1} and set(_lib.TRANSPORTS.values()) == {0, 1}


def test_digest_calls_reject_more_than_2_32_sub_frames(lib):
    """count * n is the hash kernel's 32-bit message count: beyond 2^32 - 1 the allocating digest calls
    return FHD_ERR_TOO_LARGE before any allocation or launch (so this needs no GPU)."""
    import paper_2505_07158_gb300 as fhd
    dig = ctypes.create_string_buffer(32)
    for fn in (lib.fhd_frame_digest, lib.fhd_frame_digest_tree, lib.fhd_frame_digest_noalloc):
        assert fn(None, 0, 4, 1 << 31, dig, None) == fhd.FHD_ERR_TOO_LARGE
        assert b"exceeds" in lib.cipher_last_error(None)


def test_digest_wrappers_reject_a_size_that_count_does_not_divide():
    import torch
    import paper_2505_07158_gb300 as fhd
    data = torch.zeros(10, dtype=torch.uint8)
    with pytest.raises(ValueError, match="multiple of count"):
        fhd.fhd_frame_digest(data, n=2, count=3)
    with pytest.raises(ValueError, match="multiple of count"):
        fhd._lib.fhd_frame_digest_noalloc(data, torch.zeros(96, dtype=torch.uint8), n=2, count=3)


def test_host_side_checks_of_the_persistent_and_tuning_calls(lib):
    """The persistent launches, their limits and trace, the worker CTA size, the encryption route and the
    row-band override reject bad arguments before any device work."""
    import paper_2505_07158_gb300 as fhd
    assert lib.encrypt_frames_persistent(None, 1, None, None) == fhd.FHD_ERR_INVALID_ARG
    assert lib.decrypt_frames_persistent(None, 1, None, None) == fhd.FHD_ERR_INVALID_ARG
    assert lib.cipher_round_trip_persistent(None, None, 1, None, None, None) == fhd.FHD_ERR_INVALID_ARG
    assert lib.cipher_set_persistent_limits(None, 10**9, -1) == fhd.FHD_ERR_INVALID_ARG
    assert lib.cipher_persistent_trace(None, 1, None) == fhd.FHD_ERR_INVALID_ARG
    assert lib.cipher_set_worker_cta(None, 4) == fhd.FHD_ERR_INVALID_ARG
    assert lib.fhd_set_encrypt_route(7) == fhd.FHD_ERR_INVALID_ARG
    assert lib.fhd_set_keystream_route(7) == fhd.FHD_ERR_INVALID_ARG
    assert lib.fhd_set_keystream_route(-1) == fhd.FHD_ERR_INVALID_ARG
    assert lib.fhd_set_keystream_route(0) == 1       # the default is the trajectory route
    assert fhd.fhd_set_keystream_route("trajectory") == "pairs"
    assert fhd.fhd_set_keystream_route("trajectory") == "trajectory"
    assert lib.fhd_set_row_band(0, 16, 3, 2) == fhd.FHD_ERR_INVALID_ARG
    assert lib.fhd_set_row_band(16, 16, 3, 65) == fhd.FHD_ERR_INVALID_ARG
    assert lib.fhd_row_band(0, 16, 3) == 0
    assert lib.fhd_set_row_band(24, 24, 3, 3) == fhd.FHD_OK
    assert lib.fhd_row_band(24, 24, 3) == 3
    assert lib.fhd_set_row_band(24, 24, 3, 0) == fhd.FHD_OK
    assert lib.fhd_row_band(24, 24, 3) == 16
