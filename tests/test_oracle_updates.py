"""Pins of the oracle's ADMM sub-steps (CPU only): each closed form of Sec. IV is checked
against an independent solve of its subproblem."""
import numpy as np
import pytest

from oracle import nlpr, cloops


def _rng(s=0):
    return np.random.default_rng(s)


def _kernel(rng, bh=3, bw=3):
    k = rng.random((bh, bw)) + 0.1
    return k / k.sum()


@pytest.mark.parametrize("HW,K,S,asym", [((6, 6), 1, 1, False), ((8, 6), 1, 2, True), ((6, 8), 0, 1, True)])
def test_x_update_matches_dense_solve(HW, K, S, asym):
    # The per-frequency division (eq. inv) solves the n_h x n_h system of
    # eq. x_linear_system_main, built densely from the spatial operators.
    rng = _rng(10)
    H, W = HW
    kern = rng.random((3, 5)) if asym else _kernel(rng)
    C = rng.standard_normal((H, W, 2))
    Xf = nlpr.solve_x(C, nlpr.x_denominator(H, W, kern, K, S))
    Xd = nlpr.solve_x_dense(C, kern, K, S)
    assert np.abs(Xf - Xd).max() <= 1e-12 * np.abs(Xd).max()
    A = nlpr.x_system_matrix(H, W, kern, K, S)
    res = np.linalg.norm(A @ nlpr.mat(Xf) - nlpr.mat(C)) / np.linalg.norm(C)
    assert res < 1e-12


def test_filter_magnitude_identity():
    # |d^_{tau k}| = |d^_{tau k0}| so sum_{tau,k} |d^_{tau k}|^2 = |P| sum_tau |d^_{tau k0}|^2.
    H, W, K, S = 8, 10, 1, 2
    lit = np.zeros((H, W))
    for tau in nlpr.search_offsets(S):
        for k in nlpr.patch_offsets(K):
            f = nlpr.filter_image({k: 1.0, (tau[0] + k[0], tau[1] + k[1]): -1.0}, H, W)
            lit += np.abs(np.fft.fft2(f)) ** 2
    kern = np.zeros((1, 1)); kern[0, 0] = 0.0
    den = nlpr.x_denominator(H, W, kern, K, S)
    assert np.abs((1.0 + lit) - den).max() < 1e-11


def _vec_map(fn, shape_in):
    """Dense matrix of a linear map on arrays of the given shape (C order)."""
    n = int(np.prod(shape_in))
    cols = []
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        cols.append(np.asarray(fn(e.reshape(shape_in))).ravel())
    return np.stack(cols, axis=1)


def _problem(rng, H=8, W=8, L_l=4, L_h=2, L_s=3, d=2):
    E = np.linalg.qr(rng.standard_normal((L_l, L_s)))[0].T * rng.uniform(0.5, 2.0)   # generic E
    R = rng.random((L_l, L_h))
    Yl = rng.standard_normal((H // d, W // d, L_l))
    Yh = rng.standard_normal((H, W, L_h))
    return E, R, Yl, Yh


def test_p1_update_solves_its_subproblem():
    # eq. Qh_update = argmin_P1 1/2||Yl - S P1 E||^2 + rho/2 ||P1 - BX + Lambda1||^2
    # (eq. P1_update_problem), the latter solved as a generic dense least-squares problem.
    rng = _rng(11)
    H, W, d, rho = 8, 8, 2, 0.37
    E, R, Yl, Yh = _problem(rng, H, W, d=d)
    L_s = E.shape[0]
    kern = _kernel(rng)
    om = rng.random((8, H, W))
    su = nlpr.setup(Yl, Yh, kern, d, R, E, 1, 1, 0.8, 0.1, rho, om)
    st = nlpr.State.zeros(H, W, L_s, 1, 1)
    st.Lam1 = rng.standard_normal((H, W, L_s))
    X = rng.standard_normal((H, W, L_s))
    P1, BX = nlpr.update_p1(X, st, su)
    A = _vec_map(lambda P: nlpr.mat(nlpr.decimate(P, d)) @ E, (H, W, L_s))
    n = A.shape[1]
    lhs = np.vstack([A, np.sqrt(rho) * np.eye(n)])
    V = nlpr.blur(X, kern) - st.Lam1
    rhs = np.concatenate([Yl.reshape(-1), np.sqrt(rho) * V.reshape(-1)])
    ref = np.linalg.lstsq(lhs, rhs, rcond=None)[0].reshape(H, W, L_s)
    assert np.abs(P1 - ref).max() <= 1e-10 * np.abs(ref).max()


def test_p2_update_solves_its_subproblem():
    # eq. Qm_update = argmin_P2 lambda1/2 ||Yh - P2 E R||^2 + rho/2 ||P2 + Lambda2 - X||^2
    rng = _rng(12)
    H, W, d, rho, lam1 = 6, 6, 2, 0.21, 0.9
    E, R, Yl, Yh = _problem(rng, H, W, d=d)
    L_s = E.shape[0]
    om = rng.random((8, H, W))
    su = nlpr.setup(Yl, Yh, _kernel(rng), d, R, E, 1, 1, lam1, 0.1, rho, om)
    st = nlpr.State.zeros(H, W, L_s, 1, 1)
    st.Lam2 = rng.standard_normal((H, W, L_s))
    X = rng.standard_normal((H, W, L_s))
    P2 = nlpr.update_p2(X, st, su)
    A = _vec_map(lambda P: nlpr.mat(P) @ E @ R, (H, W, L_s))
    n = A.shape[1]
    lhs = np.vstack([np.sqrt(lam1) * A, np.sqrt(rho) * np.eye(n)])
    rhs = np.concatenate([np.sqrt(lam1) * Yh.reshape(-1), np.sqrt(rho) * (X - st.Lam2).reshape(-1)])
    ref = np.linalg.lstsq(lhs, rhs, rcond=None)[0].reshape(H, W, L_s)
    assert np.abs(P2 - ref).max() <= 1e-10 * np.abs(ref).max()


def test_q_update_is_the_prox_of_the_weighted_l1():
    # Q_{tau k}(i,c) minimises lambda2 w |q| + rho/2 (q - (D X - Sigma))^2 per entry;
    # checked entrywise by the optimality condition.
    rng = _rng(13)
    H, W, L_s, K, S = 6, 7, 2, 1, 1
    om = rng.random((8, H, W))
    E = np.eye(L_s); R = rng.random((L_s, 1))
    su = nlpr.setup(np.zeros((H, W, L_s)), np.zeros((H, W, 1)), np.ones((1, 1)), 1, R, E,
                    K, S, 1.0, 0.3, 0.2, om)
    st = nlpr.State.zeros(H, W, L_s, K, S)
    st.Sig = rng.standard_normal(st.Sig.shape) * 0.3
    X = rng.standard_normal((H, W, L_s))
    Q = nlpr.update_q(X, st, su)
    for t, tau in enumerate(nlpr.search_offsets(S)):
        for kk, k in enumerate(nlpr.patch_offsets(K)):
            v = nlpr.diff_op(X, tau, k) - st.Sig[t, kk]
            mu = (0.3 * om[t] / 0.2)[:, :, None] * np.ones_like(v)
            q = Q[t, kk]
            nz = q != 0
            assert np.all(np.abs(np.sign(q[nz]) + (q[nz] - v[nz]) / mu[nz]) < 1e-12)
            assert np.all(np.abs(v[~nz]) <= mu[~nz] + 1e-15)


def test_c_loops_match_numpy():
    rng = _rng(14)
    H, W, L, K, S = 7, 9, 3, 1, 2
    G = rng.standard_normal((H, W, 2))
    om_np = nlpr.weights(G, K, S, 1.7)
    om_c = cloops.weights(G, K, S, 1.7)
    assert np.abs(om_np - om_c).max() < 1e-14
    su = nlpr.setup(np.zeros((H, W, L)), np.zeros((H, W, 1)), np.ones((1, 1)), 1,
                    rng.random((L, 1)), np.eye(L), K, S, 1.0, 0.4, 0.3, om_np)
    st = nlpr.State.zeros(H, W, L, K, S)
    st.Sig = rng.standard_normal(st.Sig.shape) * 0.2
    st.Q = rng.standard_normal(st.Q.shape) * 0.2
    X = rng.standard_normal((H, W, L))
    Qn = nlpr.update_q(X, st, su)
    Sn = nlpr.update_sigma(X, Qn, st, su)
    Qc, Sc = cloops.latent_update(X, st, su)
    assert np.abs(Qn - Qc).max() < 1e-14 and np.abs(Sn - Sc).max() < 1e-14
    assert np.abs(nlpr.dt_sum(st.Q, st.Sig, K, S) - cloops.dt_sum(st.Q, st.Sig, K, S)).max() < 1e-12


def test_first_two_iterates_closed_form():
    # From zero initialisation (all variables 0): X^1 = 0, P1^1 = S^T S (S^T Yl E^T)
    # (E E^T + rho I)^{-1}, Lambda1^1 = P1^1, P2^1 = (lambda1/rho Yh R^T E^T) F,
    # Lambda2^1 = P2^1, Q^1 = Sigma^1 = 0; then X^2 solves the dense system with right side
    # B^T(2 P1^1) + 2 P2^1.  Pins the update order and the dual signs of Sec. IV.
    rng = _rng(15)
    H, W, d, K, S, lam1, lam2, rho = 6, 6, 2, 1, 1, 0.7, 0.05, 0.3
    E, R, Yl, Yh = _problem(rng, H, W, L_l=3, L_h=2, L_s=2, d=d)
    kern = _kernel(rng)
    om = rng.random((8, H, W))
    X1, st1, su = nlpr.admm(Yl, Yh, kern, d, R, E, K, S, lam1, lam2, rho, om, 1)
    assert np.abs(X1).max() < 1e-15
    L_s = E.shape[0]
    m = nlpr.sampling_mask(H, W, d)[:, :, None]
    SYlEt = np.zeros((H, W, L_s)); SYlEt[::d, ::d] = (Yl.reshape(-1, Yl.shape[2]) @ E.T).reshape(H // d, W // d, L_s)
    P1 = (m * SYlEt).reshape(-1, L_s) @ np.linalg.inv(E @ E.T + rho * np.eye(L_s))
    P2 = (lam1 / rho) * Yh.reshape(-1, Yh.shape[2]) @ R.T @ E.T @ np.linalg.inv(
        np.eye(L_s) + (lam1 / rho) * E @ R @ R.T @ E.T)
    assert np.allclose(nlpr.mat(st1.P1), P1, atol=1e-12) and np.allclose(nlpr.mat(st1.Lam1), P1, atol=1e-12)
    assert np.allclose(nlpr.mat(st1.P2), P2, atol=1e-12) and np.allclose(nlpr.mat(st1.Lam2), P2, atol=1e-12)
    assert not st1.Q.any() and not st1.Sig.any()
    X2, _, _ = nlpr.admm(Yl, Yh, kern, d, R, E, K, S, lam1, lam2, rho, om, 1, state=st1)
    C = nlpr.blur_t(2 * P1.reshape(H, W, L_s), kern) + 2 * P2.reshape(H, W, L_s)
    ref = nlpr.solve_x_dense(C, kern, K, S)
    assert np.abs(X2 - ref).max() <= 1e-12 * np.abs(ref).max()


def test_inplace_latent_loops_match():
    rng = _rng(16)
    H, W, L, K, S = 8, 10, 2, 1, 1
    su = nlpr.setup(np.zeros((H, W, L)), np.zeros((H, W, 1)), np.ones((1, 1)), 1,
                    rng.random((L, 1)), np.eye(L), K, S, 1.0, 0.4, 0.3, rng.random((8, H, W)))
    st = nlpr.State.zeros(H, W, L, K, S)
    st.Sig = rng.standard_normal(st.Sig.shape) * 0.2
    X = rng.standard_normal((H, W, L))
    Qa, Sa = cloops.latent_update(X, st, su)
    st2 = st.copy()
    Qb, Sb = cloops.latent_update_inplace(X, st2, su)
    assert np.array_equal(Qa, Qb) and np.array_equal(Sa, Sb) and Sb is st2.Sig


def test_fixed_point_state_storage():
    # codes are integers in [-levels, levels], |Sigma| <= mu is kept, mu = 0 stores 0, and with
    # very fine steps the fixed-point run equals the exact one
    rng = np.random.default_rng(61)
    H, W, L, K, S = 6, 8, 2, 1, 1
    nW, nP = len(nlpr.search_offsets(S)), len(nlpr.patch_offsets(K))
    om = rng.random((nW, H, W))
    om[0, 0, 0] = 0.0
    lam2, rho, lev = 0.3, 0.5, 32767
    mu = lam2 * om / rho
    Sig = -np.clip(rng.standard_normal((nW, nP, H, W, L)), -mu[:, None, :, :, None], mu[:, None, :, :, None])
    q = nlpr.quantize_state(Sig, om, lam2, rho, lev)
    codes = np.divide(q * lev, mu[:, None, :, :, None], out=np.zeros_like(q), where=mu[:, None, :, :, None] > 0)
    assert np.allclose(codes, np.rint(codes), atol=1e-6) and np.abs(np.rint(codes)).max() <= lev
    assert np.all(np.abs(q - Sig) <= mu[:, None, :, :, None] / (2 * lev) * (1 + 1e-12))
    assert np.all(q[0, :, 0, 0, :] == 0.0)
    assert np.array_equal(nlpr.quantize_state(q, om, lam2, rho, lev), q) or \
        np.abs(nlpr.quantize_state(q, om, lam2, rho, lev) - q).max() <= 1e-15
    Yl = rng.random((3, 4, 3)); Yh = rng.random((H, W, 1))
    E = np.linalg.qr(rng.standard_normal((3, L)))[0].T
    R = rng.random((3, 1)); R /= R.sum()
    kern = np.ones((3, 3)) / 9.0
    omega = nlpr.weights(Yh, K, S, 0.5)
    args = (Yl, Yh, kern, 2, R, E, K, S, 0.8, 0.05, 0.3, omega, 6)
    X0, _, _ = nlpr.admm(*args)
    X1, _, _ = nlpr.admm(*args, state_levels=2 ** 40)
    X2, _, _ = nlpr.admm(*args, state_levels=lev)
    assert np.abs(X1 - X0).max() <= 1e-11
    assert 0 < np.abs(X2 - X0).max() <= 1e-4 * np.abs(X0).max()


def test_sampling_mask_generalises_the_lattice():
    # S given as a 0/1 mask (d = 1, Y_l at full resolution): the lattice pattern of d = 2 with
    # Y_l placed on it reproduces the regular d = 2 run exactly, and an all-ones mask the d = 1 run
    rng = _rng(71)
    H, W, d = 8, 12, 2
    E, R, Yl, Yh = _problem(rng, H, W, d=d)
    kern = _kernel(rng)
    om = nlpr.weights(Yh, 1, 1, 0.5)
    args = (kern, d, R, E, 1, 1, 0.8, 0.05, 0.3, om, 5)
    X_reg, _, _ = nlpr.admm(Yl, Yh, *args)
    mask = nlpr.sampling_mask(H, W, d)
    Yl_full = nlpr.decimate_t(Yl, d, H, W) + 7.0 * (1.0 - mask)[:, :, None]   # off-mask values unused
    X_mask, _, _ = nlpr.admm(Yl_full, Yh, kern, 1, R, E, 1, 1, 0.8, 0.05, 0.3, om, 5, mask=mask)
    assert np.abs(X_mask - X_reg).max() <= 1e-12 * np.abs(X_reg).max()
    Yl1 = rng.random((H, W, Yl.shape[2]))
    X1, _, _ = nlpr.admm(Yl1, Yh, kern, 1, R, E, 1, 1, 0.8, 0.05, 0.3, om, 4)
    X1m, _, _ = nlpr.admm(Yl1, Yh, kern, 1, R, E, 1, 1, 0.8, 0.05, 0.3, om, 4, mask=np.ones((H, W)))
    assert np.abs(X1m - X1).max() <= 1e-12 * np.abs(X1).max()


def test_p1_update_with_a_random_mask_solves_its_subproblem():
    # eq. P1_update_problem with S = the rows of I at a random set of pixels
    rng = _rng(72)
    H, W, rho = 8, 8, 0.37
    E, R, _, Yh = _problem(rng, H, W, d=1)
    L_s = E.shape[0]
    kern = _kernel(rng)
    mask = (rng.random((H, W)) < 0.3).astype(float)
    Yl = rng.random((H, W, E.shape[1]))
    su = nlpr.setup(Yl, Yh, kern, 1, R, E, 1, 1, 0.8, 0.1, rho, rng.random((8, H, W)), mask)
    st = nlpr.State.zeros(H, W, L_s, 1, 1)
    st.Lam1 = rng.standard_normal((H, W, L_s))
    X = rng.standard_normal((H, W, L_s))
    P1, _ = nlpr.update_p1(X, st, su)
    keep = mask.reshape(-1) > 0
    A = _vec_map(lambda P: nlpr.mat(P)[keep] @ E, (H, W, L_s))
    n = A.shape[1]
    lhs = np.vstack([A, np.sqrt(rho) * np.eye(n)])
    V = nlpr.blur(X, kern) - st.Lam1
    rhs = np.concatenate([nlpr.mat(Yl)[keep].reshape(-1), np.sqrt(rho) * V.reshape(-1)])
    ref = np.linalg.lstsq(lhs, rhs, rcond=None)[0].reshape(H, W, L_s)
    assert np.abs(P1 - ref).max() <= 1e-10 * np.abs(ref).max()


def _cg(apply_A, b, tol=1e-15, maxit=5000):
    """Plain conjugate gradients for a symmetric positive definite operator (matrix-free)."""
    x = np.zeros_like(b)
    r = b - apply_A(x)
    p = r.copy()
    rr = float((r * r).sum())
    b2 = float((b * b).sum())
    for _ in range(maxit):
        Ap = apply_A(p)
        alpha = rr / float((p * Ap).sum())
        x += alpha * p
        r -= alpha * Ap
        rn = float((r * r).sum())
        if rn <= tol * tol * b2:
            break
        p = r + (rn / rr) * p
        rr = rn
    return x


@pytest.mark.parametrize("H,W,K,S", [(16, 20, 1, 2), (18, 15, 2, 1)])
def test_x_update_matches_matrix_free_cg(H, W, K, S):
    # eq. x_linear_system_main solved by CG with the spatial operators (the paper's rejected
    # splitting solves this system iteratively); the per-frequency division of eq. inv agrees.
    rng = _rng(31)
    kern = rng.random((5, 3))
    kern /= kern.sum()
    C = rng.standard_normal((H, W, 2))

    def A(x):
        y = x + nlpr.blur_t(nlpr.blur(x, kern), kern)
        for tau in nlpr.search_offsets(S):
            for k in nlpr.patch_offsets(K):
                y = y + nlpr.diff_op_t(nlpr.diff_op(x, tau, k), tau, k)
        return y
    Xcg = _cg(A, C)
    Xf = nlpr.solve_x(C, nlpr.x_denominator(H, W, kern, K, S))
    assert np.abs(Xf - Xcg).max() <= 1e-12 * np.abs(Xcg).max()


@pytest.mark.parametrize("H,W,d,K,S", [(16, 24, 4, 1, 1), (18, 12, 3, 1, 2)])
def test_sb_band_solve_matches_matrix_free_cg(H, W, d, K, S):
    # the S B-in-X system I + sum D^T D + gamma B^T S^T S B, by CG with the spatial operators
    rng = _rng(32)
    kern = rng.random((3, 5))
    kern /= kern.sum()
    c = rng.standard_normal((H, W))
    gamma = 2.3

    def A(x):
        x3 = x[:, :, None]
        y = x3.copy()
        for tau in nlpr.search_offsets(S):
            for k in nlpr.patch_offsets(K):
                y = y + nlpr.diff_op_t(nlpr.diff_op(x3, tau, k), tau, k)
        sb = nlpr.decimate_t(nlpr.decimate(nlpr.blur(x3, kern), d), d, H, W)
        return (y + gamma * nlpr.blur_t(sb, kern))[:, :, 0]
    xcg = _cg(A, c)
    bhat, g = nlpr.sb_spectra(H, W, kern, K, S)
    x = nlpr.solve_x_sb_band(c, bhat, g, d, gamma)
    assert np.abs(x - xcg).max() <= 1e-12 * np.abs(xcg).max()
