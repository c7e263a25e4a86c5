"""Pins of the oracle's operators and identities (CPU only).

Each check compares the oracle with something other than itself: a library routine,
an adjoint identity, a brute-force patch extraction, or an identity the paper states.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import nlpr


def _rng(s=0):
    return np.random.default_rng(s)


def _inner(a, b):
    return float((a * b).sum())


def test_blur_matches_library_convolution():
    # B is circular convolution with the centred kernel (Sec. I-A): equals
    # scipy.ndimage.convolve with wrap boundaries, for an asymmetric kernel.
    rng = _rng(1)
    A = rng.standard_normal((9, 11, 2))
    k = rng.standard_normal((5, 3))
    B = nlpr.blur(A, k)
    for c in range(2):
        ref = ndi.convolve(A[:, :, c], k, mode="wrap")
        assert np.abs(B[:, :, c] - ref).max() < 1e-13


def test_blur_matches_fft_convolution():
    rng = _rng(2)
    A = rng.standard_normal((8, 12, 1))
    k = rng.standard_normal((3, 5))
    f = np.zeros((8, 12))
    for a in range(3):
        for b in range(5):
            f[(a - 1) % 8, (b - 2) % 12] = k[a, b]
    ref = np.fft.ifft2(np.fft.fft2(A[:, :, 0]) * np.fft.fft2(f)).real
    assert np.abs(nlpr.blur(A, k)[:, :, 0] - ref).max() < 1e-13


@pytest.mark.parametrize("shape", [(6, 6, 2), (8, 10, 3)])
def test_adjoints(shape):
    rng = _rng(3)
    H, W, L = shape
    x = rng.standard_normal(shape)
    y = rng.standard_normal(shape)
    k = rng.standard_normal((3, 5))
    # <Bx, y> = <x, B^T y>
    a, b = _inner(nlpr.blur(x, k), y), _inner(x, nlpr.blur_t(y, k))
    assert abs(a - b) <= 1e-13 * (abs(a) + 1)
    # <D_{tau k} x, y> = <x, D_{tau k}^T y>
    for tau in [(1, -2), (0, 1), (-2, 2)]:
        for kk in [(0, 0), (1, -1), (-1, 1)]:
            a = _inner(nlpr.diff_op(x, tau, kk), y)
            b = _inner(x, nlpr.diff_op_t(y, tau, kk))
            assert abs(a - b) <= 1e-13 * (abs(a) + 1)
    # <S x, z> = <x, S^T z> and <SBx, z> = <x, B^T S^T z>
    d = 2
    z = rng.standard_normal((H // d, W // d, L))
    a = _inner(nlpr.decimate(x, d), z)
    b = _inner(x, nlpr.decimate_t(z, d, H, W))
    assert abs(a - b) <= 1e-13 * (abs(a) + 1)
    a = _inner(nlpr.decimate(nlpr.blur(x, k), d), z)
    b = _inner(x, nlpr.blur_t(nlpr.decimate_t(z, d, H, W), k))
    assert abs(a - b) <= 1e-13 * (abs(a) + 1)


def test_sampling_mask_properties():
    # S^T S S^T = S^T and (S^T S)^2 = S^T S  (eq. maskprop)
    rng = _rng(4)
    H, W, d = 12, 8, 4
    z = rng.standard_normal((H // d, W // d, 2))
    st = nlpr.decimate_t(z, d, H, W)
    assert np.array_equal(nlpr.decimate_t(nlpr.decimate(st, d), d, H, W), st)
    m = nlpr.sampling_mask(H, W, d)
    assert np.array_equal(m * m, m)
    assert m.sum() == (H // d) * (W // d)
    x = rng.standard_normal((H, W, 2))
    assert np.array_equal(nlpr.decimate_t(nlpr.decimate(x, d), d, H, W), m[:, :, None] * x)


def test_shift_identity():
    # (d_{tau k} * X)(i) = (d_{tau k0} * X)(i - k)   (Sec. III, after eq. differencemat)
    rng = _rng(5)
    X = rng.standard_normal((7, 9, 2))
    for tau in [(1, 2), (-2, 0)]:
        d0 = nlpr.diff_op(X, tau, (0, 0))
        for k in [(1, 1), (-1, 2), (2, -2)]:
            assert np.array_equal(nlpr.diff_op(X, tau, k), nlpr.shift(d0, k))


def test_diff_op_is_patch_difference():
    # ||P_{i tau}(X)||_1 = sum_c sum_k |D_{tau k} X(i, c)|, with P_{i tau} by brute-force
    # patch extraction (Sec. II-B) and D by eq. differencemat.
    rng = _rng(6)
    X = rng.standard_normal((6, 6, 2))
    K = 1
    for tau in nlpr.search_offsets(2):
        Ds = [nlpr.diff_op(X, tau, k) for k in nlpr.patch_offsets(K)]
        for i in [(0, 0), (2, 5), (5, 3)]:
            p = nlpr.patch_diff(X, i, tau, K)
            lhs = np.abs(p).sum()
            rhs = sum(np.abs(D[i[0], i[1], :]).sum() for D in Ds)
            assert abs(lhs - rhs) < 1e-12
            # entries match one to one in the (k, c) ordering of Lambda
            flat = np.concatenate([D[i[0], i[1], :] for D in Ds])
            assert np.allclose(p, flat, atol=1e-14, rtol=0)


def test_nlpr_matches_patch_loops():
    rng = _rng(7)
    X = rng.standard_normal((6, 5, 2))
    K, S = 1, 1
    om = rng.random((len(nlpr.search_offsets(S)), 6, 5))
    ref = 0.0
    for t, tau in enumerate(nlpr.search_offsets(S)):
        for i1 in range(6):
            for i2 in range(5):
                ref += om[t, i1, i2] * np.abs(nlpr.patch_diff(X, (i1, i2), tau, K)).sum()
    assert abs(nlpr.nlpr(X, om, K, S) - ref) <= 1e-12 * ref


def test_index_sets():
    assert len(nlpr.search_offsets(3)) == 48
    assert len(nlpr.search_offsets(5)) == 120
    assert len(nlpr.search_offsets(2)) == 24
    assert (0, 0) not in nlpr.search_offsets(2)
    assert len(nlpr.patch_offsets(2)) == 25
    # W is symmetric: tau in W <=> -tau in W
    W = set(nlpr.search_offsets(3))
    assert all((-a, -b) in W for (a, b) in W)


def test_soft_threshold_is_the_prox():
    # S(v, mu) = argmin_q |q| + (q - v)^2 / (2 mu)   (eq. Qj_update_problem -> eq. Qj_main),
    # checked by a dense grid search and by the subgradient condition.
    rng = _rng(8)
    for _ in range(40):
        v = rng.uniform(-3, 3)
        mu = rng.uniform(0.01, 2)
        grid = np.linspace(-4, 4, 800001)
        q_grid = grid[np.argmin(np.abs(grid) + (grid - v) ** 2 / (2 * mu))]
        q = nlpr.soft(v, mu)
        assert abs(q - q_grid) < 2e-5
        if q != 0:
            assert abs(np.sign(q) + (q - v) / mu) < 1e-12
        else:
            assert abs(v) <= mu
    # special cases
    assert nlpr.soft(0.5, 0.0) == 0.5
    assert nlpr.soft(-0.2, 0.3) == 0.0


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = _rng(9)
    x = np.concatenate([rng.random(20000), rng.random(2000) * 1e-30, np.exp(-rng.random(2000) * 100),
                        [1.0, 0.5, 2 ** -126, 2 ** -130, 0.0]])
    x32 = x.astype(np.float32)
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    got = nlpr.round_bf16(x32.astype(np.float64))
    assert np.array_equal(ref, got)
