"""The seeded input generators: reproducibility and the stated statistics."""
import numpy as np

import workloads as W


def test_gaussian_field_statistics_and_seed():
    a = W.gaussian_field((1, 64, 64), (1, 1, 1), 1.5, 0.1, 123)
    b = W.gaussian_field((1, 64, 64), (1, 1, 1), 1.5, 0.1, 123)
    c = W.gaussian_field((1, 64, 64), (1, 1, 1), 1.5, 0.1, 124)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert abs(a.mean()) < 1e-12 and abs(a.std() - 1.5) < 1e-12
    f = a.reshape(64, 64)
    # correlation at lag l should be near exp(-1/2) = 0.61 for l = ell
    lag = int(round(0.1 * 64))
    r = np.mean(f * np.roll(f, lag, axis=1)) / np.mean(f * f)
    assert 0.4 < r < 0.8


def test_layered_channels_structure():
    n = 64
    lnk = W.layered_channels(n, 16, 8, 2, 1e4, 7).reshape(n, n, n)
    ch = np.isclose(lnk, np.log(1e4))
    assert ch.sum() == 8 * 2 * 2 * n  # non-overlapping channels through x
    assert np.all(ch.all(axis=2) == ch.any(axis=2))  # x-aligned
    other = lnk[~ch].reshape(-1)
    assert len(np.unique(np.round(other, 12))) <= 16


def test_workload_shapes():
    w = W.heat2d(64)
    assert w.n == 4096 and w.steps == 20 and w.dt == 0.05
    w3 = W.channels3d(32, steps=2)
    assert w3.n == 32**3 and w3.dim == 3 and w3.dt == 8 / 32
    sizes, sig = W.ensemble_sizes()
    assert sizes.min() >= 64 and sizes.max() <= 512 and len(sizes) == 512
    assert sig.min() >= 0.5 and sig.max() <= 2.5
