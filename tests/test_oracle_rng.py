"""Pins of the oracle's counter-based generator (vacancies of Sec. 3.2)."""
import numpy as np
import pytest

from oracle import philox


def _numpy_block(counter, key):
    """First raw block of numpy's independent Philox4x64-10.  numpy advances the
    256-bit counter by one before producing a block, so the block belongs to
    counter + 1."""
    bg = np.random.Philox(counter=np.array(counter, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    return [int(x) for x in bg.random_raw(4)]


def _plus_one(counter):
    c = [int(x) for x in counter]
    for i in range(4):
        c[i] = (c[i] + 1) & ((1 << 64) - 1)
        if c[i] != 0:
            break
    return c


@pytest.mark.parametrize("counter,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([5, 7, 9, 11], [123, 456]),
    ([2**64 - 1, 3, 0, 0], [161109784, 1]),      # carry into word 1
    ([2**64 - 1, 2**64 - 1, 2**64 - 1, 5], [2**64 - 1, 2**63]),
    ([1234567, 999, 3, 0], [161109784, 2]),
])
def test_philox_matches_numpy(counter, key):
    assert list(philox.philox4x64_10(_plus_one(counter), key)) == _numpy_block(counter, key)


def test_threshold_edges():
    assert philox.vacancy_threshold(0.0) == 0
    assert philox.vacancy_threshold(0.5) == 2**63
    assert philox.vacancy_threshold(1.0) == 2**64
    assert philox.vacancy_threshold(0.25) == 2**62
    with pytest.raises(ValueError):
        philox.vacancy_threshold(1.5)


def test_vacancy_fraction_binomial():
    # 20 000 Bernoulli(0.05) draws: the count must fall within 4 sigma of n p.
    n, p = 20000, 0.05
    masks = [philox.vacancy_mask(161109784, 0, s, 400, p) for s in range(n // 400)]
    cnt = int(np.sum([m.sum() for m in masks]))
    sigma = np.sqrt(n * p * (1 - p))
    assert abs(cnt - n * p) < 4 * sigma


def test_masks_independent_across_levels_and_samples():
    # Two independent Bernoulli(p) masks agree on a site with prob. 1 - 2p(1-p).
    p, n = 0.3, 4000
    a = philox.vacancy_mask(7, 0, 0, n, p)
    b = philox.vacancy_mask(7, 1, 0, n, p)
    c = philox.vacancy_mask(7, 0, 1, n, p)
    q = 1 - 2 * p * (1 - p)
    sig = np.sqrt(n * q * (1 - q))
    for x in (b, c):
        agree = int((a == x).sum())
        assert abs(agree - n * q) < 4 * sig


def test_p_zero_and_one():
    assert philox.vacancy_mask(1, 0, 0, 64, 0.0).sum() == 0
    assert philox.vacancy_mask(1, 0, 0, 64, 1.0).sum() == 64


def test_uniform_params_range_and_mean():
    u = philox.uniform_params(20150921, 4000, -2.0, 2.0)
    assert u.min() >= -2.0 and u.max() < 2.0
    # mean of U(-2, 2): 0, sd of the mean 4/sqrt(12)/sqrt(n)
    assert abs(u.mean()) < 4 * (4 / np.sqrt(12)) / np.sqrt(4000)
