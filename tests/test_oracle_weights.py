"""Pins of the oracle's guide weights (eq. wts), CPU only."""
import numpy as np
import pytest

from oracle import nlpr, cloops


def test_weights_vectorised_equals_bruteforce_patches():
    rng = np.random.default_rng(20)
    G = rng.random((6, 7, 2))
    for K, S in [(0, 1), (1, 1), (1, 2)]:
        a = nlpr.weights(G, K, S, 0.6)
        b = nlpr.weights_bruteforce(G, K, S, 0.6)
        c = cloops.weights(G, K, S, 0.6)
        assert np.abs(a - b).max() < 1e-14
        assert np.abs(a - c).max() < 1e-14


def test_weights_impulse_closed_form():
    # Guide = a at the origin, 0 elsewhere.  Then ||P_{i tau}(G)||^2 = a^2 (1[i in P] +
    # 1[i - tau in P]) with P = [-K,K]^2 taken mod (H, W); this fixes the i - tau and
    # i - k index conventions of Sec. II-B.
    H, W, a, h = 9, 10, 0.7, 0.5
    G = np.zeros((H, W, 1)); G[0, 0, 0] = a
    for K, S in [(0, 2), (1, 2)]:
        om = nlpr.weights(G, K, S, h)
        for t, tau in enumerate(nlpr.search_offsets(S)):
            for i1 in range(H):
                for i2 in range(W):
                    def inP(y, x):
                        yy = (y + K) % H; xx = (x + K) % W
                        return int(yy <= 2 * K and xx <= 2 * K)
                    n = inP(i1, i2) + inP(i1 - tau[0], i2 - tau[1])
                    assert abs(om[t, i1, i2] - np.exp(-n * a * a / (h * h))) < 1e-15


def test_weights_range_constant_and_symmetry():
    rng = np.random.default_rng(21)
    H, W, K, S = 8, 9, 1, 2
    G = rng.random((H, W, 3))
    om = nlpr.weights(G, K, S, 0.4)
    assert np.all(om > 0) and np.all(om <= 1)
    # omega = 1 for a constant guide
    assert np.all(nlpr.weights(np.full((H, W, 2), 0.3), K, S, 0.4) == 1.0)
    # omega_{i, tau} = omega_{i - tau, -tau}
    offs = nlpr.search_offsets(S)
    idx = {tau: t for t, tau in enumerate(offs)}
    for t, tau in enumerate(offs):
        tm = idx[(-tau[0], -tau[1])]
        shifted = np.roll(om[tm], shift=(tau[0], tau[1]), axis=(0, 1))   # (i) -> om[tm](i - tau)
        assert np.abs(om[t] - shifted).max() < 1e-14
