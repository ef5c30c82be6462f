"""Pins of the oracle's random stream (Philox4x32-10, Salmon et al. SC'11)."""
import numpy as np
from scipy import stats

from conftest import read_golden


def test_known_answer_vectors(kpo):
    rows = read_golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = kpo.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_counter_sensitivity(kpo):
    """Changing any counter or key word changes every output word."""
    base = kpo.philox4x32_10([3, 5, 7, 1], [11, 13])
    for i in range(4):
        ctr = [3, 5, 7, 1]
        ctr[i] ^= 1
        assert np.all(kpo.philox4x32_10(ctr, [11, 13]) != base)
    assert np.all(kpo.philox4x32_10([3, 5, 7, 1], [11, 12]) != base)


def test_uniformity_chi2(kpo):
    """Top 8 bits of 4 * 4096 words are uniform over 256 cells."""
    words = np.concatenate([kpo.philox4x32_10([i, 17, 3, 0], [99, 7])
                            for i in range(4096)])
    counts = np.bincount(words >> 24, minlength=256)
    p = stats.chisquare(counts).pvalue
    assert p > 1e-4
