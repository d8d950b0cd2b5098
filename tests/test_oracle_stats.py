"""Pins of the statistics oracle (oracle/stats.py) against closed forms and known distributions.

* histogram variance (Eq. 4), chi^2 (Eq. 5), entropy (Eq. 10) of a constant frame and of a frame
  holding every level equally often: closed forms;
* chi^2 of uniform random frames follows the chi^2 distribution with 255 degrees of freedom
  (mean 255; Sec. III-A's critical value 293.25 is its 95 % point);
* local Shannon entropy (Eq. 11) of blocks holding every level once is 8, and of 1936-pixel blocks of
  uniform random bytes averages the paper's ideal 7.902469317 (Sec. III-C) with the spread of the
  plug-in estimator;
* correlation (Eqs. 6-9) of ramps is +1 / -1, of independent uniform pairs ~0;
* NPCR/UACI (Eqs. 14-15) of identical frames 0/0, of complementary frames 100 % and 50.196 %, of
  independent uniform frames 255/256 = 99.609 % and 33.464 % (the standard expected values)."""
import numpy as np
import pytest

from oracle import stats

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _all_levels(h, w, C, seed=0):
    """h*w a multiple of 256: every level equally often in every channel, shuffled."""
    g = np.random.default_rng(seed)
    F = np.empty((h, w, C), dtype=np.uint8)
    for c in range(C):
        v = np.tile(np.arange(256, dtype=np.uint8), h * w // 256)
        g.shuffle(v)
        F[:, :, c] = v.reshape(h, w)
    return F


def test_histogram_counts():
    F = np.zeros((3, 5, 2), dtype=np.uint8)
    F[0, :, 0] = 7
    F[1:, 2, 1] = 255
    z0, z1 = stats.histogram(F, 0), stats.histogram(F, 1)
    assert z0[7] == 5 and z0[0] == 10 and z0.sum() == 15
    assert z1[255] == 2 and z1[0] == 13


def test_constant_frame_closed_forms():
    h, w = 48, 64
    N = h * w
    F = np.full((h, w, 1), 200, dtype=np.uint8)
    z = stats.histogram(F, 0)
    assert stats.chi_square(z) == pytest.approx(255.0 * N, rel=1e-14)
    assert stats.entropy(z) == 0.0
    # population variance of (N, 0, ..., 0): N^2/256 - (N/256)^2 = 255 N^2 / 256^2
    assert stats.histogram_variance(z) == pytest.approx(255.0 * N * N / 65536.0, rel=1e-14)


def test_every_level_equally_often():
    F = _all_levels(64, 64, 3)
    for c in range(3):
        z = stats.histogram(F, c)
        assert stats.chi_square(z) == 0.0
        assert stats.histogram_variance(z) == 0.0
        assert stats.entropy(z) == 8.0


def test_two_levels_entropy_one_bit():
    F = np.zeros((16, 16, 1), dtype=np.uint8)
    F[:8] = 9
    assert stats.entropy(stats.histogram(F, 0)) == pytest.approx(1.0, abs=1e-15)


def test_chi_square_of_random_frames_follows_chi2_255():
    g = np.random.default_rng(11)
    vals = [stats.chi_square(stats.histogram(g.integers(0, 256, (128, 128, 1), dtype=np.uint8), 0))
            for _ in range(300)]
    # mean 255, standard deviation sqrt(2*255) ~ 22.6; the mean of 300 is within ~4 of 255
    assert abs(np.mean(vals) - 255.0) < 6.0
    above = np.mean(np.array(vals) > 293.25)      # the 95 % point the paper quotes
    assert 0.01 < above < 0.10


def test_local_entropy_closed_form_and_paper_ideal():
    F = _all_levels(32, 32, 1, seed=3)            # 16 x 16 blocks do not each hold every level ...
    blk = np.tile(np.arange(256, dtype=np.uint8).reshape(16, 16), (2, 2))[:, :, None]
    assert stats.local_entropy(blk, 0, [(0, 0), (0, 16), (16, 0), (16, 16)], 16) == 8.0   # ... these do
    g = np.random.default_rng(5)
    means = []
    for _ in range(40):
        R = g.integers(0, 256, (44 * 6, 44 * 5, 1), dtype=np.uint8)
        blocks = [(44 * i, 44 * j) for i in range(6) for j in range(5)]      # 30 non-overlapping blocks
        means.append(stats.local_entropy(R, 0, blocks, 44))
    # Sec. III-C: ideal 7.902469317 for k = 30, T_B = 1936.  The spread of the 30-block mean of ideal random
    # blocks is sqrt(2 * 255) / (2 * 1936 * ln 2) / sqrt(30) ~ 0.0015 (plug-in entropy estimator), so the
    # acceptance interval the paper quotes, (7.901515798, 7.903422936), holds only about half of them; it is
    # not used as a pin.
    assert abs(np.mean(means) - 7.902469317) < 6e-4
    assert 0.0008 < np.std(means) < 0.0025
    assert F.shape == (32, 32, 1)


def test_correlation_of_ramps_and_noise():
    h, w = 64, 64
    ramp = np.add.outer(np.arange(h), np.arange(w)).astype(np.uint8)[:, :, None]      # i + j < 256
    pairs = [(i, j) for i in range(0, h - 1, 3) for j in range(0, w - 1, 2)]
    for d in ("horizontal", "vertical", "diagonal"):
        assert stats.correlation(ramp, 0, pairs, d) == pytest.approx(1.0, abs=1e-12)
    # anti-correlated pairs: y = 255 - x across a horizontal pair of a frame built for it
    A = np.zeros((4, 64, 1), dtype=np.uint8)
    A[:, 0::2, 0] = np.arange(32) * 7
    A[:, 1::2, 0] = 255 - np.arange(32) * 7
    assert stats.correlation(A, 0, [(i, j) for i in range(4) for j in range(0, 63, 2)], "horizontal") == \
        pytest.approx(-1.0, abs=1e-12)
    g = np.random.default_rng(7)
    R = g.integers(0, 256, (200, 200, 1), dtype=np.uint8)
    p = np.stack([g.integers(0, 199, 10000), g.integers(0, 199, 10000)], axis=1)
    for d in ("horizontal", "vertical", "diagonal"):
        assert abs(stats.correlation(R, 0, p, d)) < 0.04        # ~N(0, 1/100) for independent pairs


def test_npcr_uaci_closed_forms_and_expectations():
    F = _all_levels(64, 64, 2, seed=9)
    assert stats.npcr_uaci(F, F, 0) == (0.0, 0.0)
    npcr, uaci = stats.npcr_uaci(F, 255 - F, 1)
    # every level equally often: mean |2a - 255| = 128 -> UACI = 100 * 128 / 255
    assert npcr == 100.0 and uaci == pytest.approx(100.0 * 128.0 / 255.0, rel=1e-14)
    g = np.random.default_rng(13)
    A = g.integers(0, 256, (512, 512, 1), dtype=np.uint8)
    B = g.integers(0, 256, (512, 512, 1), dtype=np.uint8)
    npcr, uaci = stats.npcr_uaci(A, B, 0)
    # E[NPCR] = 100 * 255/256; E|a - b| = (256^2 - 1) / (3 * 256) -> E[UACI] = 100 * 85.332 / 255
    assert npcr == pytest.approx(100.0 * 255.0 / 256.0, abs=0.05)
    assert uaci == pytest.approx(100.0 * (65535.0 / 768.0) / 255.0, abs=0.15)
