"""CPU emulation of the GPU path's bidiagonal kernels for graphene's small
matrices, lane by lane, in float64: the sublattice masks and ranks, the
column assembly from the kept sites' three bonds, the Golub-Kahan left/right
reflector steps, and the right step's row sums by the half-warp
reduce-scatter (16 lanes) and by the 64-thread mapping (two 32-lane warps).
The spectra of the resulting (d, e^2) tridiagonals are compared with the
oracle's eigenvalues of the dense H(k) of the same cell and k-point.  This
checks the method and its index mappings without a GPU; the kernels
themselves are checked against the oracle by the GPU tests."""
import math

import numpy as np
import pytest

from oracle import idos as oidos
from synthetic import model_params, workload


def neighbours(N, m):
    """Bond partners of site m = 2 (i + N j) + s, and whether m is a B site."""
    cell, s = m >> 1, m & 1
    i, j = cell % N, cell // N
    if s == 0:
        im, jm = (i + N - 1) % N, (j + N - 1) % N
        return [2 * (i + N * j) + 1, 2 * (im + N * j) + 1, 2 * (i + N * jm) + 1], False
    ip, jp = (i + 1) % N, (j + 1) % N
    return [2 * (i + N * j), 2 * (ip + N * j), 2 * (i + N * jp)], True


def bond_phase(N, K, kidx, b):
    """exp(i pi num / (3 N K)) of bond b at k-point kidx (i1 = kidx % K fastest)."""
    i1, i2 = kidx % K, kidx // K
    U1, U2 = 2 * i1 - K + 1, 2 * i2 - K + 1
    c1 = -2 if b == 1 else 1
    c2 = -2 if b == 2 else 1
    num = (U1 * c1 + U2 * c2) % (6 * N * K)
    x = num / (3 * N * K)
    return complex(math.cos(math.pi * x), math.sin(math.pi * x))


def popc(x):
    return bin(x & 0xFFFFFFFF).count("1")


def block_columns(N, K, kidx, mask, t, width):
    """Sublattice split from 32-bit ballot words over the kept indices, and
    the lane-held columns of the q x p block M (p <= q)."""
    n_sites = 2 * N * N
    act = [m for m in range(n_sites) if not mask[m]]
    inv = [-1] * n_sites
    for i, m in enumerate(act):
        inv[m] = i
    n = len(act)
    words = [0] * 4
    for idx in range(n):
        if act[idx] & 1 == 0:
            words[idx >> 5] |= 1 << (idx & 31)
    live = [((1 << min(32, max(0, n - 32 * w))) - 1) for w in range(4)]
    n_a = sum(popc(x) for x in words)
    n_b = n - n_a
    colm = [live[w] & ~words[w] if n_a >= n_b else words[w] for w in range(4)]
    rowm = [live[w] & ~colm[w] for w in range(4)]
    p, q = min(n_a, n_b), n - min(n_a, n_b)
    m = np.zeros((width, width), complex)   # m[lane][row]
    for c in range(p):
        cum, ic = 0, -1
        for w in range(4):
            pc = popc(colm[w])
            if ic < 0 and c < cum + pc:
                mm = colm[w]
                for _ in range(c - cum):
                    mm &= mm - 1
                ic = 32 * w + ((mm & -mm).bit_length() - 1)
            cum += pc
        nb, from_b = neighbours(N, act[ic])
        for b in range(3):
            ai = inv[nb[b]]
            if ai >= 0 and (rowm[ai >> 5] >> (ai & 31)) & 1:
                rw = sum(popc(rowm[w]) for w in range(ai >> 5)) + popc(rowm[ai >> 5] & ((1 << (ai & 31)) - 1))
                ph = t * bond_phase(N, K, kidx, b)
                m[c, rw] += ph if from_b else ph.conjugate()
    return m, p, q, n


def householder(alpha, sigma2):
    aa = abs(alpha)
    phs = alpha / aa if aa > 0 else 1.0
    sigma = math.sqrt(sigma2)
    return sigma, phs, 1.0 / (sigma * (sigma + aa))


def reduce_scatter(vals, lanes):
    """vals[lane][row] over `lanes` lanes and rows: recursive halving by lane
    bit (a lane with the bit set keeps the upper half); lane l ends with row l."""
    cur = vals.copy()
    width = lanes
    off = lanes // 2
    while off >= 1:
        half = width // 2
        nxt = np.zeros((lanes, half), complex)
        for l in range(lanes):
            pa = l ^ off
            bit, pbit = (l & off) != 0, (pa & off) != 0
            for tt in range(half):
                kept = cur[l, tt + half] if bit else cur[l, tt]
                sent = cur[pa, tt] if pbit else cur[pa, tt + half]
                nxt[l, tt] = kept + sent
        cur, width, off = nxt, half, off // 2
    return cur[:, 0]


def golub_kahan(m, p, q, n, eps, row_sums):
    e2 = np.zeros(max(n - 1, 0))
    for j in range(p):
        rest = sum(abs(m[j, r]) ** 2 for r in range(j + 1, q))
        sa = abs(m[j, j]) ** 2 + rest
        e2[2 * j] = sa
        if rest > 1e-30:
            sigma, phs, tau = householder(m[j, j], sa)
            v = np.zeros(m.shape[1], complex)
            v[j] = m[j, j] + phs * sigma
            v[j + 1:q] = m[j, j + 1:q]
            for c in range(j + 1, p):
                s = np.vdot(v, m[c]) * tau
                m[c] -= v * s
        if j + 1 >= p:
            break
        z = np.array([np.conj(m[c, j]) if j < c < p else 0 for c in range(m.shape[0])])
        rz = sum(abs(z[c]) ** 2 for c in range(j + 2, p))
        sb = abs(z[j + 1]) ** 2 + rz
        e2[2 * j + 1] = sb
        if rz > 1e-30:
            sigma, phs, tau = householder(z[j + 1], sb)
            u = z.copy()
            u[j + 1] = z[j + 1] + phs * sigma
            prod = np.array([[m[c, r] * u[c] if j < r < q else 0 for r in range(m.shape[1])]
                             for c in range(m.shape[0])])
            x = row_sums(prod)
            for c in range(j + 1, p):
                for r in range(j + 1, q):
                    m[c, r] -= x[r] * tau * np.conj(u[c])
    return np.full(n, eps), e2


def half_warp_sums(prod):
    """16 lanes, 16 rows: one reduce-scatter."""
    return reduce_scatter(prod, 16)


def cta_sums(prod):
    """64 lanes (two warps of 32), 64 rows: per warp a reduce-scatter over
    each 32-row half, the two warps' sums added."""
    x = np.zeros(64, complex)
    for warp in range(2):
        part = prod[32 * warp: 32 * warp + 32]
        for h in range(2):
            x[32 * h: 32 * h + 32] += reduce_scatter(part[:, 32 * h: 32 * h + 32], 32)
    return x


def spectrum(d, e2):
    if d.size == 0:
        return d
    T = np.diag(d) + np.diag(np.sqrt(e2), 1) + np.diag(np.sqrt(e2), -1)
    return np.linalg.eigvalsh(T)


@pytest.mark.parametrize("N,width,sums,trials", [(1, 16, half_warp_sums, 4), (2, 16, half_warp_sums, 8),
                                                 (3, 16, half_warp_sums, 6), (4, 16, half_warp_sums, 6),
                                                 (5, 64, cta_sums, 2), (6, 64, cta_sums, 2)])
def test_emulated_kernels_match_oracle_spectra(N, width, sums, trials):
    w = workload("graphene_mlmc")
    prm = model_params(w)
    rng = np.random.default_rng(31 + N)
    K = 2
    for trial in range(trials):
        eps = [0.0, 0.37][trial % 2]
        prm_t = dict(prm, eps_onsite=eps)
        mask = (rng.random(2 * N * N) < [0.0, 0.1, 0.3, 0.6][trial % 4]).astype(np.uint8)
        if mask.all():
            continue
        kidx = trial % (K * K)
        m, p, q, n = block_columns(N, K, kidx, mask, prm["t"], width)
        d, e2 = golub_kahan(m, p, q, n, eps, sums)
        ref = oidos.band_energies(N, K, mask, prm_t)[kidx]
        got = spectrum(d, e2)
        assert got.shape == ref.shape
        assert np.max(np.abs(got - ref)) < 1e-9
