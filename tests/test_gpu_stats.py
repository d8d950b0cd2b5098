"""GPU frame statistics (Sec. III, Sec. IV-B) against the oracle.

Histograms and NPCR/UACI are exact: the counts are integers and the percentages are one binary64
division on both sides, so they are compared for equality.  Histogram variance, chi^2, entropy,
correlation and local entropy are finished by different formulas on the two sides (the oracle sums
the paper's expressions literally, the kernels work from exact integer sums), so they are compared
within 1e-12 relative.  The shapes cover the 16-byte and the byte-wise streaming paths (frame sizes
that are and are not multiples of 16 * C), one to four channels, and batches of frames."""
import numpy as np
import pytest
import torch

from oracle import stats as ostats
import synth_inputs as si
from gpu_util import dev, host, to_dev

pytestmark = pytest.mark.gpu

fhd = pytest.importorskip("paper_2505_07158_gb300")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

SHAPES = [(1, 1, 1), (7, 9, 3), (37, 53, 3), (16, 16, 4), (64, 100, 1), (480, 640, 3), (1080, 1920, 3)]


def _batch(shape, count, seed):
    g = si.rng(seed)
    frames = g.integers(0, 256, size=(count, *shape), dtype=np.uint8)
    if count > 1:          # one smooth frame: a skewed histogram and correlated neighbours
        h, w, C = shape
        ramp = (np.add.outer(np.arange(h), 2 * np.arange(w)) % 256).astype(np.uint8)
        frames[0] = ramp[:, :, None].repeat(C, axis=2)
    return frames


@pytest.mark.parametrize("shape", SHAPES)
def test_histogram_statistics(shape):
    count = 3 if shape[0] * shape[1] < 10 ** 6 else 2
    F = _batch(shape, count, seed=sum(shape))
    hist, st = fhd.fhd_stats_histogram(to_dev(F))
    hist, st = host(hist), host(st)
    for f in range(count):
        for c in range(shape[2]):
            z = ostats.histogram(F[f], c)
            assert np.array_equal(hist[f, c].astype(np.int64), z), (f, c)
            assert st[f, c, 0] == pytest.approx(ostats.histogram_variance(z), rel=1e-12, abs=1e-12)
            assert st[f, c, 1] == pytest.approx(ostats.chi_square(z), rel=1e-12, abs=1e-12)
            assert st[f, c, 2] == pytest.approx(ostats.entropy(z), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("shape", SHAPES)
def test_npcr_uaci_exact(shape):
    count = 2
    A = _batch(shape, count, seed=3 * sum(shape))
    B = A.copy()
    g = si.rng(5 + sum(shape))
    mask = g.random(B.shape) < 0.5
    B[mask] = g.integers(0, 256, size=int(mask.sum()), dtype=np.uint8)
    counts, out = fhd.fhd_stats_npcr_uaci(to_dev(A), to_dev(B))
    counts, out = host(counts), host(out)
    for f in range(count):
        for c in range(shape[2]):
            npcr, uaci = ostats.npcr_uaci(A[f], B[f], c)
            assert out[f, c, 0] == npcr and out[f, c, 1] == uaci, (f, c)
            a = A[f][:, :, c].astype(np.int64)
            b = B[f][:, :, c].astype(np.int64)
            assert counts[f, c, 0] == np.count_nonzero(a != b) and counts[f, c, 1] == np.abs(a - b).sum()


@pytest.mark.parametrize("shape", [(37, 53, 3), (480, 640, 3), (64, 100, 1), (16, 16, 4)])
def test_correlation(shape):
    h, w, C = shape
    count, npairs = 2, 10000
    F = _batch(shape, count, seed=7 * sum(shape))
    g = si.rng(9 + sum(shape))
    pairs = np.stack([g.integers(0, h - 1, (count, 3, npairs)), g.integers(0, w - 1, (count, 3, npairs))],
                     axis=-1).astype(np.int32)
    sums, r, status = fhd.fhd_stats_correlation(to_dev(F), torch.from_numpy(pairs).to(dev()))
    r = host(r)
    assert int(host(status)[0]) == 0
    for f in range(count):
        for c in range(C):
            for d, name in enumerate(("horizontal", "vertical", "diagonal")):
                ref = ostats.correlation(F[f], c, pairs[f, d], name)
                assert r[f, c, d] == pytest.approx(ref, rel=1e-12, abs=1e-12), (f, c, name)
    # a pair whose neighbour leaves the frame is reported
    pairs[0, 0, 0] = (0, w - 1)
    _, _, status = fhd.fhd_stats_correlation(to_dev(F), torch.from_numpy(pairs).to(dev()))
    assert int(host(status)[0]) & 1


@pytest.mark.parametrize("shape", [(88, 132, 3), (480, 640, 3), (1080, 1920, 3)])
def test_local_entropy(shape):
    h, w, C = shape
    count, bs, k = 2, 44, 30
    F = _batch(shape, count, seed=11 * sum(shape))
    g = si.rng(13 + sum(shape))
    grid = [(44 * i, 44 * j) for i in range(h // 44) for j in range(w // 44)]
    blocks = np.stack([np.array(grid)[g.choice(len(grid), size=min(k, len(grid)), replace=False)]
                       for _ in range(count)]).astype(np.int32)
    out, status = fhd.fhd_stats_local_entropy(to_dev(F), torch.from_numpy(blocks).to(dev()), bs)
    out = host(out)
    assert int(host(status)[0]) == 0
    for f in range(count):
        for c in range(C):
            ref = ostats.local_entropy(F[f], c, blocks[f], bs)
            assert out[f, c] == pytest.approx(ref, rel=1e-12, abs=1e-12), (f, c)
    blocks[1, 0] = (h - 10, 0)
    _, status = fhd.fhd_stats_local_entropy(to_dev(F), torch.from_numpy(blocks).to(dev()), bs)
    assert int(host(status)[0]) & 1


def test_statistics_of_the_ciphertext():
    """The cipher's output measured with the GPU statistics: a 1080p gradient frame and the same frame
    with one bit flipped encrypt to frames that pass the paper's bars -- entropy above 7.999 and chi^2
    below 293.25 per channel (Sec. III-A, III-C), NPCR at the value of independent uniform frames and UACI
    inside (33.3730, 33.5541) % (Sec. IV-B) -- while the plaintext is far from uniform.  (With the RK4 step
    read as 0.001 one channel's chi^2 and UACI failed: the finding that fixed the step at 0.01.)"""
    key = si.key(21)
    F = si.gradient_frame(1080, 1920, 3, t=0, seed=21)
    F2 = F.copy()
    F2[500, 700, 1] ^= 1
    c1, c2 = fhd.Cipher(key), fhd.Cipher(key)
    E1, _ = c1.encrypt(c1.open_stream(), to_dev(F))
    E2, _ = c2.encrypt(c2.open_stream(), to_dev(F2))
    _, st = fhd.fhd_stats_histogram(torch.stack([E1, E2]))
    st = host(st)
    assert (st[:, :, 2] > 7.999).all()
    assert (st[:, :, 1] < 293.25).all(), st[:, :, 1]
    _, out = fhd.fhd_stats_npcr_uaci(E1, E2)
    out = host(out)[0]
    assert ((out[:, 0] > 99.55) & (out[:, 0] < 99.67)).all()
    assert ((out[:, 1] > 33.3730) & (out[:, 1] < 33.5541)).all(), out[:, 1]
    _, so = fhd.fhd_stats_histogram(to_dev(F))
    assert (host(so)[0, :, 2] < 7.99).all()          # the plaintext is far from uniform
