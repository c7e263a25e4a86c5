"""CPU model of the FP64 soft-threshold clamp of the latent pass (SymBound<double> in
csrc/common.cuh).

The FP64 latent pass takes clamp(u, -mu, mu) (eq. Qj_main: Sigma' = -clamp(v, -mu, mu)) on the
IEEE-754 bit patterns instead of with two FP64 min/max operations: with the bound's sign bit
cleared, |u| <= mu holds exactly when the magnitude bits of u, read as an unsigned 64-bit
integer, are at most those of mu, and then the result is u, else mu with the sign of u.  These
tests restate that rule in NumPy and check it against np.clip on random, special and adjacent
values, so a wrong mask, a signed comparison or a dropped sign would fail.  The GPU tests check
the kernel itself against the oracle (FP64 within 1e-11)."""
import numpy as np

MAG = np.uint64(0x7FFFFFFFFFFFFFFF)
SIGN = np.uint64(0x8000000000000000)


def bit_clamp(u, m):
    ub = np.asarray(u, dtype=np.float64).view(np.uint64)
    mb = np.asarray(m, dtype=np.float64).view(np.uint64) & MAG
    other = (mb | (ub & SIGN)).view(np.float64)
    return np.where((ub & MAG) <= mb, u, other)


def check(u, m):
    got = bit_clamp(u, m)
    want = np.clip(u, -np.abs(m), np.abs(m))
    assert np.array_equal(got, want)
    # a zero result (u = +-0, or a zero bound) carries the sign of u
    z = want == 0
    assert np.array_equal(np.signbit(got[z]), np.signbit(np.asarray(u)[z]))


def test_random_values_across_magnitudes():
    rng = np.random.default_rng(5)
    n = 200_000
    u = rng.standard_normal(n) * 10.0 ** rng.integers(-300, 300, n)
    m = np.abs(rng.standard_normal(n)) * 10.0 ** rng.integers(-300, 300, n)
    check(u, m)
    # magnitudes of the same order, where most entries sit near the bound
    u = rng.standard_normal(n) * 1e-3
    m = np.abs(rng.standard_normal(n)) * 1e-3
    check(u, m)


def test_adjacent_doubles_at_the_bound():
    rng = np.random.default_rng(6)
    m = np.abs(rng.standard_normal(5000)) + 1e-12
    for u in (m, -m, np.nextafter(m, np.inf), -np.nextafter(m, np.inf), np.nextafter(m, 0.0),
              -np.nextafter(m, 0.0)):
        check(u, m)


def test_special_values():
    tiny = np.finfo(np.float64).tiny
    den = tiny / 4.0                                     # subnormal
    vals = np.array([0.0, -0.0, den, -den, tiny, -tiny, 1.0, -1.0, 1e308, -1e308, np.inf, -np.inf])
    U, M = np.meshgrid(vals, np.abs(vals))
    check(U.ravel(), M.ravel())
    # a bound of -0 acts as +0: every value clamps to a zero carrying its own sign
    u = np.array([3.0, -3.0, 0.0, -0.0])
    got = bit_clamp(u, np.full(4, -0.0))
    assert np.all(got == 0.0)
    assert np.array_equal(np.signbit(got), np.signbit(u))
