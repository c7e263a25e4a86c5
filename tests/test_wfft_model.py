"""CPU model of the register-resident DFT's index algebra (the CUDA passes in csrc/k_wfft.cuh).

A line of N = 32 P points is held by 32 lanes, lane l owning points l + 32 j (j < P).  The forward
transform is a P-point DFT per lane, the twist w_N^{l k1}, and a radix-2 decimation-in-frequency
transform across the lanes; lane l then holds frequency k1 + P rev5(l) in slot k1.  The inverse
applies the adjoint of each step in reverse order.  These tests check, in NumPy and against
numpy.fft, that ordering, that the adjoint returns natural order, and that a per-frequency
factor stored in the slot-major order of both axes filters an image exactly as the
natural-order factor does.  That is the layout the host builds for f (position q holds
frequency q / 32 + P rev5(q mod 32)).  The GPU tests check the kernels themselves."""
import numpy as np
import pytest


def rev5(l):
    return int(f"{l:05b}"[::-1], 2)


def slot_freq(q, P):
    """Frequency held at slot-major position q = k1 * 32 + l of a line of 32 P points."""
    return q // 32 + P * rev5(q % 32)


def small_dft(v, inverse):
    F = len(v)
    s = 1 if inverse else -1
    k = np.arange(F)
    return np.exp(s * 2j * np.pi * np.outer(k, k) / F) @ v


def lane_forward(x, P):
    """x (natural order, 32 P) -> v[l, k1]."""
    N = 32 * P
    w = np.exp(-2j * np.pi * np.arange(N) / N)
    v = np.array([[x[l + 32 * j] for j in range(P)] for l in range(32)], dtype=complex)
    v = np.array([small_dft(v[l], False) for l in range(32)])
    for l in range(32):
        v[l] *= w[(l * np.arange(P)) % N]
    for h in (16, 8, 4, 2, 1):                   # radix-2 stages across lanes
        nv = v.copy()
        for l in range(32):
            up = bool(l & h)
            o = v[l ^ h]
            tw = w[(l & (h - 1)) * (16 * P // h)] if up else 1.0
            nv[l] = ((o - v[l]) if up else (v[l] + o)) * tw
        v = nv
    return v


def lane_inverse(v, P):
    """Adjoint of lane_forward (unnormalised inverse): v[l, k1] -> natural order x."""
    N = 32 * P
    w = np.exp(-2j * np.pi * np.arange(N) / N)
    v = v.copy()
    for h in (1, 2, 4, 8, 16):
        m = v.copy()
        for l in range(32):
            if l & h:
                m[l] = v[l] * np.conj(w[(l & (h - 1)) * (16 * P // h)])
        nv = v.copy()
        for l in range(32):
            o = m[l ^ h]
            nv[l] = (o - m[l]) if (l & h) else (m[l] + o)
        v = nv
    for l in range(32):
        v[l] *= np.conj(w[(l * np.arange(P)) % N])
    v = np.array([small_dft(v[l], True) for l in range(32)])
    x = np.zeros(N, dtype=complex)
    for l in range(32):
        for j in range(P):
            x[l + 32 * j] = v[l, j]
    return x


def to_slot_major(v):
    """v[l, k1] -> array indexed by position q = k1 * 32 + l."""
    P = v.shape[1]
    return np.array([v[q % 32, q // 32] for q in range(32 * P)])


def from_slot_major(y, P):
    return np.array([[y[k1 * 32 + l] for k1 in range(P)] for l in range(32)])


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 8, 10, 12, 16])
def test_forward_is_the_dft_in_slot_major_order(P):
    rng = np.random.default_rng(P)
    N = 32 * P
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    y = to_slot_major(lane_forward(x, P))
    X = np.fft.fft(x)
    assert np.abs(y - X[[slot_freq(q, P) for q in range(N)]]).max() <= 1e-10 * np.abs(X).max()
    # the positions hold every frequency once
    assert sorted(slot_freq(q, P) for q in range(N)) == list(range(N))


@pytest.mark.parametrize("P", [1, 3, 5, 12, 16])
def test_adjoint_returns_natural_order(P):
    rng = np.random.default_rng(100 + P)
    N = 32 * P
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    back = lane_inverse(lane_forward(x, P), P) / N
    assert np.abs(back - x).max() <= 1e-12 * np.abs(x).max()


@pytest.mark.parametrize("PH,PW", [(1, 2), (3, 2)])
def test_slot_major_factor_filters_like_the_natural_factor(PH, PW):
    # rows forward -> columns forward * fT * columns inverse -> rows inverse, with fT[q][r] =
    # f(u(r), v(q)) in slot-major order on both axes, against ifft2(f * fft2(z))
    rng = np.random.default_rng(7)
    H, W = 32 * PH, 32 * PW
    z = rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))
    f = rng.uniform(0.5, 2.0, (H, W))
    ref = np.fft.ifft2(f * np.fft.fft2(z))
    Y = np.array([to_slot_major(lane_forward(z[y], PW)) for y in range(H)])     # rows, slot-major in x
    out = np.empty_like(Y)
    for q in range(W):
        col = to_slot_major(lane_forward(Y[:, q], PH))                             # slot-major in y
        fT = np.array([f[slot_freq(r, PH), slot_freq(q, PW)] for r in range(H)])
        out[:, q] = lane_inverse(from_slot_major(col * fT, PH), PH)
    X = np.array([lane_inverse(from_slot_major(out[y], PW), PW) for y in range(H)]) / (H * W)
    assert np.abs(X - ref).max() <= 1e-12 * np.abs(ref).max()
