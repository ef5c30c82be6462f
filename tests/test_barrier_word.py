"""The grid barrier's one-word arithmetic (kp_device.cuh, team_sync): every
block but block 0 adds 1 and block 0 adds 2^31 - (nb - 1), in any order;
the top bit must flip with the last arrival and only then, and the low 31
bits must come back to 0, phase after phase, for every team size the
launches use (one block up to KP_MAX_GRID)."""
import numpy as np
import pytest


def arrivals(nb, rng):
    order = rng.permutation(nb)
    return [(0x80000000 - (nb - 1)) if b == 0 else 1 for b in order]


@pytest.mark.parametrize("nb", [1, 2, 3, 304, 456, 8192])
def test_top_bit_flips_with_the_last_arrival_only(nb):
    rng = np.random.default_rng(nb)
    word = 0
    for _ in range(4):
        top = word & 0x80000000
        adds = arrivals(nb, rng)
        for i, a in enumerate(adds):
            word = (word + a) & 0xFFFFFFFF
            flipped = (word & 0x80000000) != top
            assert flipped == (i == nb - 1), (nb, i)
        assert word & 0x7FFFFFFF == 0


def test_a_stale_low_part_would_flip_early():
    """Why the reset and import paths write the word: with low bits left
    over (a launch that stopped mid-phase) the bit could flip before the
    last arrival, so a context whose wait expired is poisoned instead."""
    nb, word = 8, 5
    top = word & 0x80000000
    early = False
    for i, a in enumerate([0x80000000 - (nb - 1)] + [1] * (nb - 1)):
        word = (word + a) & 0xFFFFFFFF
        if (word & 0x80000000) != top and i < nb - 1:
            early = True
    assert early
