"""Pins for the oracle's randomised labels: a permutation, counts kept, uniform, seed-dependent."""
import numpy as np
from scipy.stats import chisquare


def test_permutation_for_awkward_sizes(orc):
    for n in (1, 2, 3, 5, 17, 1000, 4096, 4097, 65537, (1 << 20) + 7):
        p = orc.label_perm(n, 12345)
        assert p.shape == (n,)
        assert np.array_equal(np.sort(p), np.arange(n, dtype=np.uint32))


def test_labels_keep_their_counts(orc):
    t = np.random.default_rng(0).integers(0, 3, 100_000).astype(np.uint8)
    s = orc.shuffle_labels(t, 7)
    assert np.array_equal(np.bincount(t, minlength=3), np.bincount(s, minlength=3))
    assert np.mean(s != t) > 0.3  # actually moved
    assert np.array_equal(s, t[orc.label_perm(t.shape[0], 7)])


def test_uniform_images_over_seeds(orc):
    # image of position 0 and of position 9 over 4000 seeds: uniform on [0, 10)
    n = 10
    img0 = np.array([orc.label_perm(n, s)[0] for s in range(4000)])
    img9 = np.array([orc.label_perm(n, s)[9] for s in range(4000)])
    for img in (img0, img9):
        assert chisquare(np.bincount(img, minlength=n)).pvalue > 1e-4


def test_seeds_differ_and_no_identity(orc):
    a, b = orc.label_perm(10_000, 1), orc.label_perm(10_000, 2)
    assert np.mean(a != b) > 0.99
    assert np.mean(a == np.arange(10_000)) < 0.01
    # adjacent positions land far apart (no local structure left)
    assert np.median(np.abs(np.diff(a.astype(np.int64)))) > 1000
