"""Philox4x64-10 counter-based generator, written from its published definition
(J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplications whose
high halves are xored into the other counter words, with a Weyl-sequence key
schedule.

Used for the i.i.d. Bernoulli(p) vacancies of Sec. 3.2 (each site removed with
probability p independently of all others).

Counter/key layout (the build's reading; the paper's MATLAB runs were unseeded):
    key     = (seed, stream)            stream 1 = vacancies, 2 = model parameters
    counter = (site, sample, level, 0)
A site is vacant iff word 0 of the output block is < floor(p * 2**64), an
integer comparison, so masks are bit-exact across implementations.

Pinned against ``numpy.random.Philox`` (an independent implementation of the
same generator) in tests/test_oracle_rng.py.
"""
from __future__ import annotations

import math

import numpy as np

_MASK64 = (1 << 64) - 1
# Round multipliers and Weyl key increments of Philox4x64 (Salmon et al.).
_M0 = 0xD2E7470EE14C6C93
_M1 = 0xCA5A826395121157
_W0 = 0x9E3779B97F4A7C15
_W1 = 0xBB67AE8584CAA73B

STREAM_VACANCY = 1
STREAM_PARAMS = 2


def philox4x64_10(counter, key):
    """One Philox4x64-10 block: four 64-bit words from a 256-bit counter and a
    128-bit key.  Pure Python integers, one round at a time."""
    c0, c1, c2, c3 = (int(x) & _MASK64 for x in counter)
    k0, k1 = (int(x) & _MASK64 for x in key)
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> 64, p0 & _MASK64
        hi1, lo1 = p1 >> 64, p1 & _MASK64
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + _W0) & _MASK64
        k1 = (k1 + _W1) & _MASK64
    return c0, c1, c2, c3


def vacancy_threshold(p: float) -> int:
    """floor(p * 2**64) as an exact integer (ldexp is exact in binary64)."""
    if not (0.0 <= p <= 1.0):
        raise ValueError("p must lie in [0, 1]")
    return int(math.floor(math.ldexp(float(p), 64)))


def vacancy_mask(seed: int, level: int, sample: int, n_sites: int, p: float) -> np.ndarray:
    """u8[n_sites]: 1 where the site is removed (Sec. 3.2), 0 where it is kept."""
    thr = vacancy_threshold(p)
    out = np.zeros(n_sites, dtype=np.uint8)
    for site in range(n_sites):
        w0 = philox4x64_10((site, sample, level, 0), (seed, STREAM_VACANCY))[0]
        out[site] = 1 if w0 < thr else 0
    return out


def uniform_params(model_seed: int, count: int, lo: float, hi: float) -> np.ndarray:
    """float64[count] uniform on [lo, hi) from 53-bit fractions of word 0:
    u = (w0 >> 11) * 2**-53, value = lo + (hi - lo) * u.  Used to draw the
    TMDC-shaped model's on-site energies and hopping blocks."""
    out = np.empty(count, dtype=np.float64)
    for i in range(count):
        w0 = philox4x64_10((i, 0, 0, 0), (model_seed, STREAM_PARAMS))[0]
        u = math.ldexp(float(w0 >> 11), -53)
        out[i] = lo + (hi - lo) * u
    return out
