"""Pins of the S B-in-X variant of the oracle (CPU only).

The variant keeps the data term 1/2 ||Y_l - S B X E||^2 in the X subproblem (only P2 = X and
Q = D X are split) and solves it as one d^2 x d^2 system per alias class of the DFT grid.  Each
pin checks it against something built independently of that Fourier form:
  * the band solve against the dense n_h x n_h operator system I + sum D^T D + gamma B^T S^T S B
    assembled column by column from the spatial operators;
  * the full X update for a generic (non-orthonormal) E against the Kronecker form of its normal
    equations;
  * the iteration's limit against the Chambolle-Pock minimiser of the same objective (the
    paper's ADMM and the variant minimise the same convex function)."""
import numpy as np
import pytest

from oracle import nlpr
from test_oracle_convergence import DenseProblem, _tiny


def _operator_matrix(fn, H, W):
    n = H * W
    cols = []
    for j in range(n):
        e = np.zeros((H, W, 1))
        e.flat[j] = 1.0
        cols.append(fn(e).reshape(n))
    return np.stack(cols, axis=1)


def _sb_system(H, W, kern, d, K, S, gamma):
    def fn(e):
        y = e.copy()
        for tau in nlpr.search_offsets(S):
            for k in nlpr.patch_offsets(K):
                y = y + nlpr.diff_op_t(nlpr.diff_op(e, tau, k), tau, k)
        sb = nlpr.decimate_t(nlpr.decimate(nlpr.blur(e, kern), d), d, H, W)
        return y + gamma * nlpr.blur_t(sb, kern)
    return _operator_matrix(fn, H, W)


@pytest.mark.parametrize("H,W,d,K,S,kshape", [(8, 8, 2, 1, 1, (3, 3)), (8, 12, 4, 1, 2, (3, 5)),
                                               (6, 6, 1, 0, 1, (3, 3)), (12, 8, 2, 0, 2, (5, 3)),
                                               (9, 6, 3, 1, 1, (3, 3))])
def test_band_solve_matches_dense_operator_system(H, W, d, K, S, kshape):
    rng = np.random.default_rng(70 + H + W + d)
    kern = rng.random(kshape)
    kern /= kern.sum()
    c = rng.standard_normal((H, W))
    gamma = 3.7
    bhat, g = nlpr.sb_spectra(H, W, kern, K, S)
    x = nlpr.solve_x_sb_band(c, bhat, g, d, gamma)
    A = _sb_system(H, W, kern, d, K, S, gamma)
    xd = np.linalg.solve(A, c.reshape(-1)).reshape(H, W)
    assert np.abs(x - xd).max() <= 1e-12 * np.abs(xd).max()


def test_d1_band_solve_is_a_per_frequency_division():
    # S = I: the alias classes are single frequencies and the system is diagonal,
    # 1 + |P| sum |d^|^2 + gamma |b^|^2 (eq. inv's filter with the blur term weighted by gamma).
    rng = np.random.default_rng(77)
    H, W, K, S, gamma = 7, 10, 1, 2, 0.4
    kern = rng.random((3, 3))
    kern /= kern.sum()
    c = rng.standard_normal((H, W))
    bhat, g = nlpr.sb_spectra(H, W, kern, K, S)
    x = nlpr.solve_x_sb_band(c, bhat, g, 1, gamma)
    den = nlpr.x_denominator(H, W, np.zeros((1, 1)), K, S) + gamma * np.abs(bhat) ** 2
    xr = np.fft.ifft2(np.fft.fft2(c) / den).real
    assert np.abs(x - xr).max() <= 1e-13 * np.abs(xr).max()


def test_x_update_with_generic_E_matches_kronecker_normal_equations():
    # B^T S^T S B X (E E^T) + rho (I + sum D^T D) X = rho C, in row-major vec form
    # (kron(Msb, E E^T) + rho kron(Md, I)) vec(X) = rho vec(C).
    rng = np.random.default_rng(78)
    H, W, d, K, S, L_l, L_s, rho = 4, 6, 2, 1, 1, 4, 3, 0.35
    E = rng.standard_normal((L_s, L_l))                 # not orthonormal: E E^T has spread
    R = rng.random((L_l, 2))
    kern = rng.random((3, 3))
    kern /= kern.sum()
    Yl = rng.standard_normal((H // d, W // d, L_l))
    Yh = rng.standard_normal((H, W, 2))
    om = np.ones((len(nlpr.search_offsets(S)), H, W))
    su = nlpr.setup(Yl, Yh, kern, d, R, E, K, S, 1.0, 0.1, rho, om)
    C = rng.standard_normal((H, W, L_s))
    X = nlpr.solve_x_sb(C, su)

    def sb(e):
        return nlpr.blur_t(nlpr.decimate_t(nlpr.decimate(nlpr.blur(e, kern), d), d, H, W), kern)

    def dd(e):
        y = e.copy()
        for tau in nlpr.search_offsets(S):
            for k in nlpr.patch_offsets(K):
                y = y + nlpr.diff_op_t(nlpr.diff_op(e, tau, k), tau, k)
        return y
    Msb, Md = _operator_matrix(sb, H, W), _operator_matrix(dd, H, W)
    M = np.kron(Msb, E @ E.T) + rho * np.kron(Md, np.eye(L_s))
    xv = np.linalg.solve(M, rho * C.reshape(-1))
    assert np.abs(X.reshape(-1) - xv).max() <= 1e-12 * np.abs(xv).max()


def test_right_hand_side_is_the_gradient_balance_of_the_x_subproblem():
    # At the X update the gradient of 1/2||Y_l - S B X E||^2 + rho/2||X - P2 - Lambda2||^2
    # + rho/2 sum ||D X - Q - Sigma||^2 vanishes (checked with the operators, not the solve).
    rng = np.random.default_rng(79)
    H, W, d, K, S, L_l, L_s, rho = 8, 8, 2, 1, 1, 4, 2, 0.5
    E = np.linalg.qr(rng.standard_normal((L_l, L_s)))[0].T
    R = rng.random((L_l, 2))
    kern = rng.random((3, 3))
    kern /= kern.sum()
    Yl = rng.standard_normal((H // d, W // d, L_l))
    Yh = rng.standard_normal((H, W, 2))
    om = rng.random((len(nlpr.search_offsets(S)), H, W))
    su = nlpr.setup(Yl, Yh, kern, d, R, E, K, S, 1.0, 0.1, rho, om)
    st = nlpr.State.zeros(H, W, L_s, K, S)
    st.P2 = rng.standard_normal((H, W, L_s))
    st.Lam2 = rng.standard_normal((H, W, L_s))
    st.Q = rng.standard_normal(st.Q.shape)
    st.Sig = rng.standard_normal(st.Sig.shape)
    X = nlpr.solve_x_sb(nlpr.rhs_sb(st, su), su)
    r = nlpr.img(nlpr.mat(Yl) - nlpr.mat(nlpr.decimate(nlpr.blur(X, kern), d)) @ E, H // d, W // d)
    grad = -nlpr.img(nlpr.mat(nlpr.blur_t(nlpr.decimate_t(r, d, H, W), kern)) @ E.T, H, W)
    grad = grad + rho * (X - st.P2 - st.Lam2)
    for t, tau in enumerate(nlpr.search_offsets(S)):
        for kk, k in enumerate(nlpr.patch_offsets(K)):
            grad = grad + rho * nlpr.diff_op_t(nlpr.diff_op(X, tau, k) - st.Q[t, kk] - st.Sig[t, kk], tau, k)
    assert np.abs(grad).max() <= 1e-11 * (1 + np.abs(X).max())


@pytest.mark.slow
def test_sb_variant_limit_matches_chambolle_pock_objective():
    Yl, Yh, kern, R, E, G = _tiny(30, d=2)
    K, S, lam1, lam2, rho, h = 1, 1, 0.8, 0.02, 0.5, 0.5
    om = nlpr.weights(G, K, S, h)
    X, st, su = nlpr.admm(Yl, Yh, kern, 2, R, E, K, S, lam1, lam2, rho, om, 6000, fast=True, x_update="sb")
    dp = DenseProblem(Yl, Yh, kern, 2, R, E, K, S, lam1, lam2, om)
    f_sb = dp.objective(X.reshape(-1))
    f_cp = dp.objective(dp.chambolle_pock(20000))
    assert abs(f_sb - f_cp) <= 1e-10 * abs(f_cp)
    assert np.abs(X - st.P2).max() < 1e-9                  # the split's primal residual vanishes
    assert not st.P1.any() and not st.Lam1.any()             # not variables of this splitting


@pytest.mark.slow
def test_sb_variant_limit_is_the_unique_minimiser():
    Yl, Yh, kern, R, E, G = _tiny(31, d=1, E_identity=True, H=5, W=6, center=0.6)
    K, S, lam1, lam2, rho, h = 1, 1, 0.5, 0.03, 0.1, 0.5
    om = nlpr.weights(G, K, S, h)
    X, _, _ = nlpr.admm(Yl, Yh, kern, 1, R, E, K, S, lam1, lam2, rho, om, 3000, fast=True, x_update="sb")
    dp = DenseProblem(Yl, Yh, kern, 1, R, E, K, S, lam1, lam2, om)
    assert np.abs(X.reshape(-1) - dp.chambolle_pock(20000)).max() < 1e-10


def test_sb_variant_rejects_a_mask():
    Yl, Yh, kern, R, E, G = _tiny(32, d=1)
    om = nlpr.weights(G, 1, 1, 0.5)
    with pytest.raises(ValueError):
        nlpr.admm(Yl, Yh, kern, 1, R, E, 1, 1, 0.5, 0.01, 0.1, om, 1, x_update="sb",
                  mask=np.ones(Yh.shape[:2]))
