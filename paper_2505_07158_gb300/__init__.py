"""GB300-native implementation of the diffusion-free bit-level video cipher of
arXiv 2505.07158 ("Real-Time Bit-Level Encryption of Full High-Definition
Video Without Diffusion").

The compute path is the C-ABI library ``libfhdcipher.so`` (hand-written CUDA
for sm_103a, declared in ``include/fhdcipher.h``); this package is its thin
binding plus the batching/serving layers above it.  PyTorch provides device
memory and streams only."""
from ._lib import (  # noqa: F401
    EXPORTS, FHD_ERR_BAD_STREAM, FHD_ERR_CUDA, FHD_ERR_INVALID_ARG, FHD_ERR_OOM, FHD_ERR_STATE, FHD_ERR_TIMEOUT,
    FHD_ERR_TOO_LARGE, FHD_OK, FHD_STATE_BYTES, Cipher, FhdError, fhd_frame_digest, fhd_keystream, fhd_master,
    fhd_frame_scratch_bytes, fhd_launch_count, fhd_permute_decrypt, fhd_permute_encrypt, KERNEL_KINDS, fhd_set_strip_width, fhd_strip_width, fhd_row_band, fhd_set_row_band, fhd_version, library_path,
    load, fhd_stats_histogram, fhd_stats_npcr_uaci, fhd_stats_correlation, fhd_stats_local_entropy, fhd_fp64_probe,
    fhd_set_encrypt_route, fhd_set_keystream_route, fhd_build_flags, fhd_bounds_report, fhd_bounds_site_name, fhd_bounds_selftest,
    FHD_BUILD_BOUNDS_CHECK, checked_requested, fhd_binary64_check, fhd_set_cta_threads, fhd_cta_threads,
)
