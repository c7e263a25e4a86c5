"""FP64 CPU oracle for guided nonlocal patch regularisation (NLPR) multiband fusion.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py may import this module.  The product (the CUDA library and its
Python binding) never calls it, and it shares no code with the CUDA path.

What it computes, in the paper's order and notation:
  * operators S, B, B^T, D_{tau k}, D_{tau k}^T and the patch operators P_i, P_{i tau}
    (Sec. I-A eq. model; Sec. II-B; Sec. III eq. differencemat);
  * guide weights omega_{i tau} (Sec. II-B eq. wts) by explicit patch differences;
  * the NLPR regulariser phi (eq. reg1) and the objective (eq. mainoptim);
  * the ADMM of Sec. IV for the splitting of eq. fusionoptim: X update
    (eqs. x_linear_system_main and inv), P1 update (eq. Qh_update), P2 update
    (eq. Qm_update), Q update (eq. Qj_main) and the dual updates
    (eqs. dualvar1_main, dualvar2_main, dualvar3_main).  Q and Sigma are both stored;
  * a variant that is not the paper's: the same objective with only P2 = X and Q = D X split,
    so the X system keeps S B and is solved as one dense d^2 x d^2 system per alias class of
    the DFT grid (FUSE-type direct solve of the S B term); admm(..., x_update="sb").

Readings where the paper is silent or inconsistent:
  * threshold mu = lambda2 * omega / rho (eq. Qj_main) and the objective
    l(X) + lambda2 * phi(X) (eq. mainoptim); the 1/2 in front of lambda2 in
    eqs. ouroptim/fusionoptim is not used;
  * W = [-S, S]^2 without tau = 0 (D_{0k} = 0, so it changes nothing);
  * zero initialisation of P1, P2, Q, Lambda1, Lambda2, Sigma;
  * circular blur with the kernel centred at the origin; decimation keeps pixels
    with i1 = 0 and i2 = 0 (mod d);
  * unnormalised forward DFT (numpy convention).

Layout: an image with L bands is an array of shape (H, W, L); band c is A[:, :, c] =
A_c, and the paper's n_h x L matrix is A.reshape(H * W, L) (row i = pixel (i1, i2),
row-major).  The shift convention is shift(A, j)(i) = A(i - j), indices mod (H, W).
"""
from __future__ import annotations

import dataclasses
import numpy as np

# --------------------------------------------------------------------------------------
# index sets
# --------------------------------------------------------------------------------------


def search_offsets(S: int) -> list[tuple[int, int]]:
    """W = [-S, S]^2 minus (0, 0), row-major (tau1 outer).  Sec. II-B."""
    return [(a, b) for a in range(-S, S + 1) for b in range(-S, S + 1) if (a, b) != (0, 0)]


def patch_offsets(K: int) -> list[tuple[int, int]]:
    """P = [-K, K]^2, row-major (k1 outer).  |P| = (2K+1)^2.  Sec. II-B."""
    return [(a, b) for a in range(-K, K + 1) for b in range(-K, K + 1)]


# --------------------------------------------------------------------------------------
# linear operators (Sec. I-A eq. model, Sec. III eq. differencemat)
# --------------------------------------------------------------------------------------


def shift(A: np.ndarray, j) -> np.ndarray:
    """shift(A, j)(i) = A(i - j) with circular indices (periodic domain, Sec. II-B)."""
    return np.roll(A, shift=(int(j[0]), int(j[1])), axis=(0, 1))


def blur(A: np.ndarray, kern: np.ndarray) -> np.ndarray:
    """B A: circular convolution with the centred kernel b, (b (*) A)(i) = sum_j b(j) A(i - j)."""
    bh, bw = kern.shape
    rh, rw = bh // 2, bw // 2
    out = np.zeros_like(A)
    for u in range(-rh, rh + 1):
        for v in range(-rw, rw + 1):
            out += kern[u + rh, v + rw] * shift(A, (u, v))
    return out


def blur_t(A: np.ndarray, kern: np.ndarray) -> np.ndarray:
    """B^T A: (B^T A)(i) = sum_j b(j) A(i + j)."""
    bh, bw = kern.shape
    rh, rw = bh // 2, bw // 2
    out = np.zeros_like(A)
    for u in range(-rh, rh + 1):
        for v in range(-rw, rw + 1):
            out += kern[u + rh, v + rw] * shift(A, (-u, -v))
    return out


def decimate(A: np.ndarray, d: int) -> np.ndarray:
    """S A: keep the pixels with i1 = 0 and i2 = 0 (mod d)."""
    return A[::d, ::d]


def decimate_t(Y: np.ndarray, d: int, H: int, W: int) -> np.ndarray:
    """S^T Y: zero-filled upsampling back onto the H x W grid."""
    out = np.zeros((H, W) + Y.shape[2:], dtype=Y.dtype)
    out[::d, ::d] = Y
    return out


def sampling_mask(H: int, W: int, d: int) -> np.ndarray:
    """Diagonal of S^T S as an (H, W) 0/1 array."""
    m = np.zeros((H, W))
    m[::d, ::d] = 1.0
    return m


def diff_op(X: np.ndarray, tau, k) -> np.ndarray:
    """D_{tau k} X (i, c) = X_c(i - k) - X_c(i - tau - k).  Eq. differencemat."""
    return shift(X, k) - shift(X, (tau[0] + k[0], tau[1] + k[1]))


def diff_op_t(Y: np.ndarray, tau, k) -> np.ndarray:
    """D_{tau k}^T Y (i, c) = Y_c(i + k) - Y_c(i + k + tau)  (adjoint of diff_op)."""
    return shift(Y, (-k[0], -k[1])) - shift(Y, (-(tau[0] + k[0]), -(tau[1] + k[1])))


def mat(A: np.ndarray) -> np.ndarray:
    """The paper's n_h x L matrix of an (H, W, L) image."""
    return A.reshape(A.shape[0] * A.shape[1], A.shape[2])


def img(M: np.ndarray, H: int, W: int) -> np.ndarray:
    return M.reshape(H, W, M.shape[1])


# --------------------------------------------------------------------------------------
# patches, weights and the regulariser (Sec. II-B eqs. reg1, wts)
# --------------------------------------------------------------------------------------


def patch(A: np.ndarray, i, K: int) -> np.ndarray:
    """P_i(A): the values A_c(i - k) for (k, c) in Lambda = [-K,K]^2 x [1, L], k-major."""
    H, W, L = A.shape
    vals = []
    for k in patch_offsets(K):
        for c in range(L):
            vals.append(A[(i[0] - k[0]) % H, (i[1] - k[1]) % W, c])
    return np.array(vals)


def patch_diff(A: np.ndarray, i, tau, K: int) -> np.ndarray:
    """P_{i tau}(A) = P_i(A) - P_{i - tau}(A)."""
    H, W, _ = A.shape
    j = ((i[0] - tau[0]) % H, (i[1] - tau[1]) % W)
    return patch(A, i, K) - patch(A, j, K)


def weights(G: np.ndarray, K: int, S: int, h: float) -> np.ndarray:
    """omega[t, i1, i2] = exp(-||P_{i tau_t}(G)||_2^2 / h^2) for every pixel i (eq. wts).

    The squared norm sums (G_c(i - k) - G_c(i - tau - k))^2 over k in P and every band c;
    the loop over pixels is vectorised with circular shifts."""
    offs = search_offsets(S)
    H, W, _ = G.shape
    out = np.empty((len(offs), H, W))
    for t, tau in enumerate(offs):
        acc = np.zeros((H, W))
        for k in patch_offsets(K):
            diff = shift(G, k) - shift(G, (tau[0] + k[0], tau[1] + k[1]))
            acc += (diff * diff).sum(axis=2)
        out[t] = np.exp(-acc / (h * h))
    return out


def weights_bruteforce(G: np.ndarray, K: int, S: int, h: float) -> np.ndarray:
    """Same as weights() by pure-Python patch extraction per pixel (tiny inputs only)."""
    offs = search_offsets(S)
    H, W, _ = G.shape
    out = np.empty((len(offs), H, W))
    for t, tau in enumerate(offs):
        for i1 in range(H):
            for i2 in range(W):
                p = patch_diff(G, (i1, i2), tau, K)
                out[t, i1, i2] = np.exp(-float(np.dot(p, p)) / (h * h))
    return out


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 value (ties to even), returned as float64.

    bfloat16 keeps 8 significant bits and the float32 exponent range; subnormal
    spacing is 2^-133."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                      # x = m * 2^e, 0.5 <= |m| < 1
    e = np.maximum(e, -125)
    ulp = np.ldexp(1.0, e - 8)
    return np.rint(x / ulp) * ulp


def nlpr(X: np.ndarray, omega: np.ndarray, K: int, S: int) -> float:
    """phi(X) = sum_i sum_tau omega_{i tau} ||P_{i tau}(X)||_1  (eq. reg1)."""
    total = 0.0
    for t, tau in enumerate(search_offsets(S)):
        acc = np.zeros(X.shape[:2])
        for k in patch_offsets(K):
            acc += np.abs(diff_op(X, tau, k)).sum(axis=2)
        total += float((omega[t] * acc).sum())
    return total


def objective(X, Yl, Yh, kern, d, R, E, omega, K, S, lam1, lam2, mask=None) -> float:
    """l(X) + lambda2 phi(X), with l(X) = 1/2||Yl - SBXE||^2 + lambda1/2 ||Yh - XER||^2
    (eq. mainoptim).  mask (H, W) 0/1 with d = 1: S keeps the pixels where mask is 1 and Yl is
    given at full resolution (its values elsewhere do not enter)."""
    H, W, _ = X.shape
    if mask is not None:
        m = mat(mask[:, :, None].astype(float))
        r1 = m * (mat(Yl) - mat(blur(X, kern)) @ E)
    else:
        SBXE = mat(decimate(blur(X, kern), d)) @ E
        r1 = mat(Yl) - SBXE
    r2 = mat(Yh) - mat(X) @ E @ R
    return 0.5 * float((r1 * r1).sum()) + 0.5 * lam1 * float((r2 * r2).sum()) \
        + lam2 * nlpr(X, omega, K, S)


# --------------------------------------------------------------------------------------
# X update (eqs. x_linear_system_main, inv)
# --------------------------------------------------------------------------------------


def filter_image(taps: dict, H: int, W: int) -> np.ndarray:
    """The H x W filter whose circular convolution applies the given taps {j: value}."""
    f = np.zeros((H, W))
    for (a, b), v in taps.items():
        f[a % H, b % W] += v
    return f


def blur_taps(kern: np.ndarray) -> dict:
    bh, bw = kern.shape
    return {(u - bh // 2, v - bw // 2): float(kern[u, v]) for u in range(bh) for v in range(bw)}


def x_denominator(H: int, W: int, kern: np.ndarray, K: int, S: int) -> np.ndarray:
    """1 + |b^(w)|^2 + |P| sum_tau |d^_{tau k0}(w)|^2 on the H x W DFT grid (eq. inv)."""
    bhat = np.fft.fft2(filter_image(blur_taps(kern), H, W))
    acc = np.zeros((H, W))
    for tau in search_offsets(S):
        dhat = np.fft.fft2(filter_image({(0, 0): 1.0, tau: -1.0}, H, W))
        acc += np.abs(dhat) ** 2
    npatch = (2 * K + 1) ** 2
    return 1.0 + np.abs(bhat) ** 2 + npatch * acc


def solve_x(C: np.ndarray, denom: np.ndarray) -> np.ndarray:
    """X_c = IDFT( DFT(C_c) / denom ) for every band c (eq. inv)."""
    Ch = np.fft.fft2(C, axes=(0, 1))
    return np.fft.ifft2(Ch / denom[:, :, None], axes=(0, 1)).real


def x_system_matrix(H: int, W: int, kern: np.ndarray, K: int, S: int) -> np.ndarray:
    """Dense n_h x n_h matrix I + B^T B + sum_{tau,k} D_{tau k}^T D_{tau k} of
    eq. x_linear_system_main, built column by column from the operators (tiny inputs)."""
    n = H * W
    A = np.zeros((n, n))
    offs, poffs = search_offsets(S), patch_offsets(K)
    for col in range(n):
        e = np.zeros((H, W, 1))
        e.flat[col] = 1.0
        y = e + blur_t(blur(e, kern), kern)
        for tau in offs:
            for k in poffs:
                y = y + diff_op_t(diff_op(e, tau, k), tau, k)
        A[:, col] = y.reshape(n)
    return A


def solve_x_dense(C: np.ndarray, kern: np.ndarray, K: int, S: int) -> np.ndarray:
    H, W, L = C.shape
    A = x_system_matrix(H, W, kern, K, S)
    return np.linalg.solve(A, mat(C)).reshape(H, W, L)


# --------------------------------------------------------------------------------------
# Alternative X update with S B kept in the X system (FUSE-type per-frequency systems)
# --------------------------------------------------------------------------------------
#
# Not the paper's splitting: there P1 = B X moves S into the per-pixel P1 update and the X
# system is diagonal in the DFT basis (eq. inv).  Here only P2 = X and Q = D X are split, so the
# X subproblem keeps the data term 1/2 ||Y_l - S B X E||^2 and its normal equations are
#   B^T S^T S B X (E E^T) + rho (I + sum D^T D) X = B^T S^T Y_l E^T + rho (P2 + Lambda2
#                                                    + sum D^T (Q + Sigma)).
# With E E^T = V diag(e) V^T, band c' of X V solves
#   (I + sum D^T D + (e_c'/rho) B^T S^T S B) x = (rhs V)_c' / rho.
# S^T S keeps the lattice i1 = i2 = 0 (mod d), whose DFT couples frequency (u, v) with its d^2
# aliases (u + a H/d, v + b W/d):  (S^T S y)^(w) = d^-2 sum_{w' ~ w} y^(w').  Each alias class
# is therefore one d^2 x d^2 system  diag(g) + (gamma / d^2) conj(b^) b^T  with
# g = 1 + |P| sum_tau |d^_{tau 0}|^2 (the same filter sum as eq. inv) and gamma = e_c'/rho.


def sb_spectra(H: int, W: int, kern: np.ndarray, K: int, S: int):
    """b^(w) (complex) and g(w) = 1 + |P| sum_tau |d^_{tau 0}(w)|^2 on the H x W DFT grid."""
    bhat = np.fft.fft2(filter_image(blur_taps(kern), H, W))
    g = x_denominator(H, W, np.zeros((1, 1)), K, S)      # a zero blur leaves 1 + |P| sum |d^|^2
    return bhat, g


def solve_x_sb_band(c: np.ndarray, bhat: np.ndarray, g: np.ndarray, d: int, gamma: float) -> np.ndarray:
    """x with (I + sum D^T D + gamma B^T S^T S B) x = c for one (H, W) band: one dense
    d^2 x d^2 solve per alias class of the DFT grid."""
    H, W = c.shape
    h, w = H // d, W // d
    # class (u0, v0) holds the frequencies (u0 + a h, v0 + b w), a, b in [0, d): index arrays
    # of shape (h w, d^2), one row per class
    a = np.arange(d)
    U = (np.arange(h)[:, None, None, None] + h * a[None, None, :, None]) + np.zeros((1, w, 1, d), int)
    V = (np.arange(w)[None, :, None, None] + w * a[None, None, None, :]) + np.zeros((h, 1, d, 1), int)
    U, V = U.reshape(h * w, d * d), V.reshape(h * w, d * d)
    ch = np.fft.fft2(c)
    bv = bhat[U, V]
    A = np.zeros((h * w, d * d, d * d), dtype=complex)
    A[:, np.arange(d * d), np.arange(d * d)] = g[U, V]
    A += (gamma / d ** 2) * np.conj(bv)[:, :, None] * bv[:, None, :]
    xh = np.empty_like(ch)
    xh[U, V] = np.linalg.solve(A, ch[U, V][:, :, None])[:, :, 0]
    return np.fft.ifft2(xh).real


def solve_x_sb(C: np.ndarray, su) -> np.ndarray:
    """X update of the S B-in-X variant: C is the right-hand side divided by rho, (H, W, L_s)."""
    e, V = np.linalg.eigh(su.E @ su.E.T)
    Crot = img(mat(C) @ V, su.H, su.W)
    bhat, g = sb_spectra(su.H, su.W, su.kern, su.K, su.S)
    Xrot = np.stack([solve_x_sb_band(Crot[:, :, j], bhat, g, su.d, e[j] / su.rho) for j in range(su.L_s)],
                    axis=-1)
    return img(mat(Xrot) @ V.T, su.H, su.W)


def rhs_sb(st, su, dtsum_fn=None) -> np.ndarray:
    """B^T S^T Y_l E^T / rho + P2 + Lambda2 + sum D^T (Q + Sigma)."""
    dts = (dtsum_fn or dt_sum)(st.Q, st.Sig, su.K, su.S)
    return blur_t(su.SYlEt, su.kern) / su.rho + st.P2 + st.Lam2 + dts


# --------------------------------------------------------------------------------------
# proximal step (eq. Qj_main)
# --------------------------------------------------------------------------------------


def soft(x, mu):
    """S(x, mu) = sign(x) max(|x| - mu, 0), componentwise."""
    return np.sign(x) * np.maximum(np.abs(x) - mu, 0.0)


# --------------------------------------------------------------------------------------
# ADMM (Sec. IV)
# --------------------------------------------------------------------------------------


@dataclasses.dataclass
class State:
    P1: np.ndarray
    P2: np.ndarray
    Lam1: np.ndarray
    Lam2: np.ndarray
    Q: np.ndarray        # (|W|, |P|, H, W, L_s)
    Sig: np.ndarray      # (|W|, |P|, H, W, L_s)
    X: np.ndarray | None = None
    t: int = 0

    @staticmethod
    def zeros(H, W, L_s, K, S):
        nW, nP = len(search_offsets(S)), len(patch_offsets(K))
        z = lambda: np.zeros((H, W, L_s))
        return State(z(), z(), z(), z(), np.zeros((nW, nP, H, W, L_s)),
                     np.zeros((nW, nP, H, W, L_s)))

    def copy(self):
        return State(*(None if a is None else a.copy() for a in
                       (self.P1, self.P2, self.Lam1, self.Lam2, self.Q, self.Sig, self.X)),
                     t=self.t)


@dataclasses.dataclass
class Setup:
    """The per-problem constants of Sec. IV (all float64)."""
    H: int
    W: int
    L_s: int
    d: int
    K: int
    S: int
    lam1: float
    lam2: float
    rho: float
    kern: np.ndarray
    E: np.ndarray           # (L_s, L_l)
    R: np.ndarray           # (L_l, L_h)
    omega: np.ndarray       # (|W|, H, W)
    denom: np.ndarray       # eq. inv
    inv_p1: np.ndarray      # (E E^T + rho I)^{-1}          (eq. Qh_update)
    F: np.ndarray           # (I + lambda1/rho E R R^T E^T)^{-1}  (eq. Qm_update)
    SYlEt: np.ndarray       # S^T Y_l E^T  (H, W, L_s)
    YhRtEt: np.ndarray      # Y_h R^T E^T  (H, W, L_s)
    mask: np.ndarray        # diag(S^T S) as (H, W)


def setup(Yl, Yh, kern, d, R, E, K, S, lam1, lam2, rho, omega, mask=None) -> Setup:
    """Yl: (H/d, W/d, L_l), Yh: (H, W, L_h), E: (L_s, L_l), R: (L_l, L_h).

    mask: optional (H, W) 0/1 array with d = 1 for a general sampling operator S that keeps the
    pixels where mask is 1 (for example a random inpainting mask); Yl is then (H, W, L_l) and
    S^T S = diag(mask), S^T Y_l = mask * Y_l.  Eq. Qh_update holds for any such S."""
    H, W = Yh.shape[:2]
    L_s = E.shape[0]
    inv_p1 = np.linalg.inv(E @ E.T + rho * np.eye(L_s))
    F = np.linalg.inv(np.eye(L_s) + (lam1 / rho) * (E @ R @ R.T @ E.T))
    if mask is not None:
        if d != 1:
            raise ValueError("a sampling mask needs d = 1")
        smask = np.asarray(mask, dtype=float)
        SYlEt = smask[:, :, None] * img(mat(Yl) @ E.T, H, W)
    else:
        smask = sampling_mask(H, W, d)
        SYlEt = decimate_t(img(mat(Yl) @ E.T, H // d, W // d), d, H, W)
    YhRtEt = img(mat(Yh) @ R.T @ E.T, H, W)
    return Setup(H, W, L_s, d, K, S, lam1, lam2, rho, kern, E, R, omega,
                 x_denominator(H, W, kern, K, S), inv_p1, F, SYlEt, YhRtEt, smask)


def dt_sum(Q: np.ndarray, Sig: np.ndarray, K: int, S: int) -> np.ndarray:
    """sum_{tau, k} D_{tau k}^T (Q_{tau k} + Sigma_{tau k}), explicit (tau, k) loops."""
    out = np.zeros(Q.shape[2:])
    for t, tau in enumerate(search_offsets(S)):
        for kk, k in enumerate(patch_offsets(K)):
            out += diff_op_t(Q[t, kk] + Sig[t, kk], tau, k)
    return out


def rhs(st: State, su: Setup, dtsum_fn=None) -> np.ndarray:
    """C = B^T(P1 + Lambda1) + P2 + Lambda2 + sum D^T(Q + Sigma)  (after eq.
    x_linear_system_main)."""
    dts = (dtsum_fn or dt_sum)(st.Q, st.Sig, su.K, su.S)
    return blur_t(st.P1 + st.Lam1, su.kern) + st.P2 + st.Lam2 + dts


def update_p1(X, st: State, su: Setup):
    """Eq. Qh_update: S^T S (rho BX + S^T Yl E^T - rho Lambda1)(E E^T + rho I)^{-1}
    + (I - S^T S)(BX - Lambda1).  Returns (P1, BX)."""
    BX = blur(X, su.kern)
    m = su.mask[:, :, None]
    sampled = img(mat(su.rho * BX + su.SYlEt - su.rho * st.Lam1) @ su.inv_p1, su.H, su.W)
    return m * sampled + (1.0 - m) * (BX - st.Lam1), BX


def update_p2(X, st: State, su: Setup):
    """Eq. Qm_update: (-Lambda2 + X + lambda1/rho Yh R^T E^T) F."""
    return img(mat(-st.Lam2 + X + (su.lam1 / su.rho) * su.YhRtEt) @ su.F, su.H, su.W)


def update_q(X, st: State, su: Setup) -> np.ndarray:
    """Eq. Qj_main: Q_{tau k} = S(D_{tau k} X - Sigma_{tau k}, lambda2 omega_{i tau} / rho)."""
    Q = np.empty_like(st.Q)
    for t, tau in enumerate(search_offsets(su.S)):
        mu = (su.lam2 * su.omega[t] / su.rho)[:, :, None]
        for kk, k in enumerate(patch_offsets(su.K)):
            Q[t, kk] = soft(diff_op(X, tau, k) - st.Sig[t, kk], mu)
    return Q


def update_sigma(X, Q, st: State, su: Setup) -> np.ndarray:
    """Eq. dualvar3_main: Sigma_{tau k} - (D_{tau k} X - Q_{tau k})."""
    Sig = np.empty_like(st.Sig)
    for t, tau in enumerate(search_offsets(su.S)):
        for kk, k in enumerate(patch_offsets(su.K)):
            Sig[t, kk] = st.Sig[t, kk] - (diff_op(X, tau, k) - Q[t, kk])
    return Sig


def admm_step_sb(st: State, su: Setup, latent_fn=None, dtsum_fn=None) -> State:
    """One iteration of the S B-in-X variant: X (solve_x_sb), P2, Q, Sigma, Lambda2; P1 and
    Lambda1 are not variables of this splitting and stay zero."""
    X = solve_x_sb(rhs_sb(st, su, dtsum_fn), su)
    P2 = update_p2(X, st, su)
    if latent_fn is not None:
        Q, Sig = latent_fn(X, st, su)
    else:
        Q = update_q(X, st, su)
        Sig = update_sigma(X, Q, st, su)
    Lam2 = st.Lam2 - (X - P2)           # eq. dualvar2_main
    return State(st.P1, P2, st.Lam1, Lam2, Q, Sig, X, st.t + 1)


def admm_step(st: State, su: Setup, x_solver=None, latent_fn=None, dtsum_fn=None) -> State:
    """One ADMM iteration t -> t+1 in the order X, P1, P2, Q, duals (Sec. IV)."""
    C = rhs(st, su, dtsum_fn)
    X = x_solver(C) if x_solver is not None else solve_x(C, su.denom)
    P1, BX = update_p1(X, st, su)
    P2 = update_p2(X, st, su)
    if latent_fn is not None:
        Q, Sig = latent_fn(X, st, su)
    else:
        Q = update_q(X, st, su)
        Sig = update_sigma(X, Q, st, su)
    Lam1 = st.Lam1 - (BX - P1)          # eq. dualvar1_main
    Lam2 = st.Lam2 - (X - P2)           # eq. dualvar2_main
    return State(P1, P2, Lam1, Lam2, Q, Sig, X, st.t + 1)


def residuals(prev: State, st: State, su: Setup) -> tuple[float, float]:
    """ADMM residual norms of the iteration prev -> st (scaled form of the splitting of eq.
    fusionoptim: constraint A X = z with A = (B; I; D_{tau k}) and z = (P1, P2, Q)):
      primal  ||A X - z||        = sqrt(||B X - P1||^2 + ||X - P2||^2 + sum ||D_{tau k} X - Q||^2)
      dual    rho ||A^T (z - z_prev)|| = rho ||B^T dP1 + dP2 + sum D^T dQ||
    at the new iterates (X, z) = (st.X, st.P1, st.P2, st.Q).  Not printed in the paper, which
    monitors the objective; the standard ADMM stopping quantities."""
    X = st.X
    r2 = float(((blur(X, su.kern) - st.P1) ** 2).sum() + ((X - st.P2) ** 2).sum())
    for t, tau in enumerate(search_offsets(su.S)):
        for kk, k in enumerate(patch_offsets(su.K)):
            r2 += float(((diff_op(X, tau, k) - st.Q[t, kk]) ** 2).sum())
    s = blur_t(st.P1 - prev.P1, su.kern) + (st.P2 - prev.P2) + dt_sum(st.Q - prev.Q, np.zeros_like(st.Q),
                                                                        su.K, su.S)
    return float(np.sqrt(r2)), float(su.rho * np.sqrt((s * s).sum()))


def quantize_state(Sig: np.ndarray, omega: np.ndarray, lam2: float, rho: float, levels: int) -> np.ndarray:
    """Sigma as stored in `levels`-step fixed point relative to its own threshold.

    After any update Sigma_{tau k}(i) = -clamp(v, -mu, mu) with mu = lambda2 omega_{i tau}/rho
    (eqs. Qj_main, dualvar3_main), so |Sigma| <= mu and the code rint(Sigma levels / mu) lies in
    [-levels, levels]; the stored value is code mu / levels (0 where mu = 0).  This storage is
    not the paper's: it is the reduced-precision state option of the solver."""
    out = np.zeros_like(Sig)
    for t in range(Sig.shape[0]):
        mu = (lam2 * omega[t] / rho)[None, :, :, None]
        safe = np.where(mu > 0, mu, 1.0)
        code = np.where(mu > 0, np.clip(np.rint(Sig[t] / safe * levels), -levels, levels), 0.0)
        out[t] = code * mu / levels
    return out


def admm(Yl, Yh, kern, d, R, E, K, S, lam1, lam2, rho, omega, iters, state=None,
         x_solver=None, fast=False, callback=None, inplace=False, state_levels=None, mask=None,
         x_update="paper"):
    """Run `iters` ADMM iterations from `state` (zero initialisation by default).

    Images in (H, W, L) layout.  fast=True uses the C loops of oracle/loops.c for the
    Q/Sigma updates and the D^T sum (same arithmetic, explicit loops); with inplace=True those
    loops overwrite Q and Sigma in place (the old values are not needed once C is formed),
    so large problems hold one copy of the latent variables.
    state_levels: Sigma enters the Q and Sigma updates as stored in fixed point
    (quantize_state); the right-hand side still sums the exact Q + Sigma of the last update.
    mask: general sampling operator (see setup).
    x_update: "paper" (the splitting of eq. fusionoptim) or "sb" (S B kept in the X system,
    admm_step_sb; lattice sampling only).
    Returns (X, state, setup)."""
    if x_update not in ("paper", "sb"):
        raise ValueError("x_update is 'paper' or 'sb'")
    if x_update == "sb" and mask is not None:
        raise ValueError("the S B-in-X update needs the regular lattice")
    su = setup(Yl, Yh, kern, d, R, E, K, S, lam1, lam2, rho, omega, mask)
    if state is not None:
        st = state if inplace else state.copy()
    else:
        st = State.zeros(su.H, su.W, su.L_s, K, S)
    latent_fn = dtsum_fn = None
    if fast:
        from . import cloops
        latent_fn = cloops.latent_update_inplace if inplace else cloops.latent_update
        dtsum_fn = cloops.dt_sum
    if state_levels:
        exact_fn = latent_fn

        def latent_fn(X, s, u):
            sq = dataclasses.replace(s, Sig=quantize_state(s.Sig, u.omega, u.lam2, u.rho, state_levels))
            if exact_fn is not None:
                return exact_fn(X, sq, u)
            Q = update_q(X, sq, u)
            return Q, update_sigma(X, Q, sq, u)
    for _ in range(iters):
        if x_update == "sb":
            st = admm_step_sb(st, su, latent_fn, dtsum_fn)
        else:
            st = admm_step(st, su, x_solver, latent_fn, dtsum_fn)
        if callback is not None:
            callback(st, su)
    X = st.X if st.X is not None else np.zeros((su.H, su.W, su.L_s))
    return X, st, su


# --------------------------------------------------------------------------------------
# layout helpers for planar (L, H, W) inputs
# --------------------------------------------------------------------------------------


def to_hwl(A: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.moveaxis(np.asarray(A, dtype=np.float64), 0, -1))


def to_lhw(A: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.moveaxis(A, -1, 0))
