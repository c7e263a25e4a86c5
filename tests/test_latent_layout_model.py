"""CPU model of the interleaved rows of the latent pass's shifted shared tiles (csrc/k_latent.cuh).

The tiles read at shifted columns (X(m - tau) and the H_tau tiles) keep element x of a row at
word (x mod VEC) tpr + x / VEC, tpr = W / VEC.  The thread owning columns x0 .. x0 + VEC - 1
(x0 = VEC tcol) finds the element x0 + q, circular in the row, at
(q mod VEC) tpr + (tcol + floor(q / VEC)) mod tpr with a single wrap.  These tests check that
formula against the direct definition for every thread, every shift of the search windows the
kernels take (|tau2| <= S, W >= 2S + 1, W a multiple of VEC) and both element widths, and that a
warp's accesses for a fixed j hit distinct banks within each row."""
import pytest


def wrap1(a, n):
    assert -n <= a < 2 * n, "one wrap must suffice"
    return a + n if a < 0 else (a - n if a >= n else a)


def ishift(vec, tcol, q, tpr):
    lv = vec.bit_length() - 1
    return (q & (vec - 1)) * tpr + wrap1(tcol + (q >> lv), tpr)


def direct(vec, tcol, q, W):
    x = (vec * tcol + q) % W
    return (x % vec) * (W // vec) + x // vec


@pytest.mark.parametrize("vec", [8, 4])
def test_shifted_positions_equal_the_definition(vec):
    for S in range(1, 8):
        for W in range(vec, 4 * (2 * S + 1) + 2 * vec, vec):
            if W < 2 * S + 1:
                continue
            tpr = W // vec
            for tcol in range(tpr):
                for j in range(vec):
                    for t2 in range(-S, S + 1):
                        for q in (j - t2, j + t2):
                            assert ishift(vec, tcol, q, tpr) == direct(vec, tcol, q, W)


@pytest.mark.parametrize("vec,W", [(8, 256), (8, 384), (4, 128)])
def test_warp_accesses_of_a_row_hit_distinct_banks(vec, W):
    # 4-byte words for FP32 (VEC 8), two banks per 8-byte word for FP64 (VEC 4)
    tpr = W // vec
    words = 1 if vec == 8 else 2
    for j in range(vec):
        for t2 in range(-3, 4):
            for w0 in range(0, tpr, 32):
                lanes = range(w0, min(w0 + 32, tpr))
                pos = [ishift(vec, t, j - t2, tpr) for t in lanes]
                assert len(set(pos)) == len(pos)
                banks = [(p * words + h) % 32 for p in pos for h in range(words)]
                # a warp-wide access is split in 128-byte wavefronts: count them
                waves = max(banks.count(b) for b in set(banks))
                assert waves <= words + 1
