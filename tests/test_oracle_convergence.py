"""Theorem 1 pins (CPU only): the oracle's ADMM converges to a minimiser of
l(X) + lambda2 phi(X), checked against an independent primal-dual (Chambolle-Pock)
solver built here from dense matrices written from the definitions, against a gradient
method on the Huber-smoothed objective (within the smoothing bound), and against the
special cases lambda2 = 0 (least squares) and lambda2 -> infinity (constant bands)."""
import numpy as np
import pytest

from oracle import nlpr


def _dense_ops(H, W, kern, d, K, S):
    """Dense pixel-space matrices written from index arithmetic: B, S, D_{tau k}."""
    n = H * W
    pix = lambda a, b: (a % H) * W + (b % W)
    B = np.zeros((n, n))
    rh, rw = kern.shape[0] // 2, kern.shape[1] // 2
    for i1 in range(H):
        for i2 in range(W):
            for u in range(-rh, rh + 1):
                for v in range(-rw, rw + 1):
                    B[pix(i1, i2), pix(i1 - u, i2 - v)] += kern[u + rh, v + rw]
    rows = [pix(a, b) for a in range(0, H, d) for b in range(0, W, d)]
    Sm = np.zeros((len(rows), n))
    Sm[np.arange(len(rows)), rows] = 1.0
    Ds = []
    for tau in nlpr.search_offsets(S):
        for k in nlpr.patch_offsets(K):
            D = np.zeros((n, n))
            for i1 in range(H):
                for i2 in range(W):
                    D[pix(i1, i2), pix(i1 - k[0], i2 - k[1])] += 1.0
                    D[pix(i1, i2), pix(i1 - tau[0] - k[0], i2 - tau[1] - k[1])] -= 1.0
            Ds.append((tau, D))
    return B, Sm, Ds


class DenseProblem:
    def __init__(self, Yl, Yh, kern, d, R, E, K, S, lam1, lam2, omega):
        H, W = Yh.shape[:2]
        self.H, self.W, self.Ls = H, W, E.shape[0]
        B, Sm, Ds = _dense_ops(H, W, kern, d, K, S)
        Ls = self.Ls
        self.M1 = np.kron(Sm @ B, E.T)                       # vec_row(S B X E)
        self.y1 = Yl.reshape(-1)
        self.M2 = np.kron(np.eye(H * W), (E @ R).T)          # vec_row(X E R)
        self.y2 = Yh.reshape(-1)
        self.lam1 = lam1
        offs = nlpr.search_offsets(S)
        blocks, wts = [], []
        nP = len(nlpr.patch_offsets(K))
        for j, (tau, D) in enumerate(Ds):
            t = j // nP
            blocks.append(np.kron(D, np.eye(Ls)))
            wts.append(np.repeat(lam2 * omega[t].reshape(-1), Ls))
        self.Kop = np.vstack(blocks)
        self.w = np.concatenate(wts)

    def objective(self, x):
        r1 = self.M1 @ x - self.y1
        r2 = self.M2 @ x - self.y2
        return 0.5 * r1 @ r1 + 0.5 * self.lam1 * r2 @ r2 + float(self.w @ np.abs(self.Kop @ x))

    def chambolle_pock(self, iters):
        A = self.M1.T @ self.M1 + self.lam1 * self.M2.T @ self.M2
        b = self.M1.T @ self.y1 + self.lam1 * self.M2.T @ self.y2
        L = np.linalg.norm(self.Kop, 2)
        T = Sg = 0.99 / L
        Pinv = np.linalg.inv(A + np.eye(A.shape[0]) / T)
        x = np.zeros(A.shape[0]); xbar = x.copy(); y = np.zeros(self.Kop.shape[0])
        xs = np.zeros_like(x)
        for it in range(iters):
            y = np.clip(y + Sg * (self.Kop @ xbar), -self.w, self.w)
            xn = Pinv @ (b + (x - T * (self.Kop.T @ y)) / T)
            xbar = 2 * xn - x
            x = xn
        return x


def _tiny(seed, d=2, E_identity=False, H=6, W=6, center=0.0):
    rng = np.random.default_rng(seed)
    L_l, L_h = 3, 2
    L_s = L_l if E_identity else 2
    E = np.eye(L_l) if E_identity else np.linalg.qr(rng.standard_normal((L_l, L_s)))[0].T
    R = rng.random((L_l, L_h)); R /= R.sum(axis=0)
    k = rng.random((3, 3)) + 0.5; kern = (1.0 - center) * k / k.sum()
    kern[1, 1] += center            # |b^| >= 2 center - 1 > 0 when center > 1/2
    Z = rng.random((H, W, L_l))
    Yh = np.einsum("hwl,lk->hwk", Z, R) + 0.01 * rng.standard_normal((H, W, L_h))
    Yl = nlpr.decimate(nlpr.blur(Z, kern), d) + 0.01 * rng.standard_normal((H // d, W // d, L_l))
    G = Yh
    return Yl, Yh, kern, R, E, G


@pytest.mark.slow
def test_admm_limit_matches_chambolle_pock_objective():
    Yl, Yh, kern, R, E, G = _tiny(30, d=2)
    K, S, lam1, lam2, rho, h = 1, 1, 0.8, 0.02, 0.5, 0.5
    om = nlpr.weights(G, K, S, h)
    X, st, su = nlpr.admm(Yl, Yh, kern, 2, R, E, K, S, lam1, lam2, rho, om, 6000, fast=True)
    dp = DenseProblem(Yl, Yh, kern, 2, R, E, K, S, lam1, lam2, om)
    f_admm = dp.objective(X.reshape(-1))
    f_or = nlpr.objective(X, Yl, Yh, kern, 2, R, E, om, K, S, lam1, lam2)
    assert abs(f_admm - f_or) <= 1e-12 * abs(f_or)             # objective definitions agree
    x_cp = dp.chambolle_pock(20000)
    f_cp = dp.objective(x_cp)
    assert abs(f_admm - f_cp) <= 1e-10 * abs(f_cp)
    # primal residuals of the splitting are small at the limit
    BX = nlpr.blur(X, kern)
    assert np.abs(BX - st.P1).max() < 1e-9 and np.abs(X - st.P2).max() < 1e-9
    # a gradient method on the Huber-smoothed objective (|x| -> x^2/(2 delta) within delta):
    # 0 <= |x| - huber(x) <= delta/2, so its minimiser lies within sum(w) delta/2 of the minimum
    opt = pytest.importorskip("scipy.optimize")
    A = dp.M1.T @ dp.M1 + dp.lam1 * dp.M2.T @ dp.M2
    b = dp.M1.T @ dp.y1 + dp.lam1 * dp.M2.T @ dp.y2
    c0 = 0.5 * dp.y1 @ dp.y1 + 0.5 * dp.lam1 * dp.y2 @ dp.y2
    gaps = []
    for delta in (1e-2, 1e-3, 1e-4):
        def fg(x, delta=delta):
            kx = dp.Kop @ x
            hub = np.where(np.abs(kx) <= delta, kx * kx / (2 * delta), np.abs(kx) - delta / 2)
            g = A @ x - b + dp.Kop.T @ (dp.w * np.clip(kx / delta, -1.0, 1.0))
            return 0.5 * x @ A @ x - b @ x + c0 + dp.w @ hub, g
        r = opt.minimize(fg, np.zeros(A.shape[0]), jac=True, method="L-BFGS-B",
                         options=dict(maxiter=200000, maxfun=400000, gtol=1e-13, ftol=1e-16, maxcor=30))
        gap = dp.objective(r.x) - f_admm
        assert -1e-10 * abs(f_admm) <= gap <= dp.w.sum() * delta / 2
        gaps.append(gap)
    assert gaps[2] < gaps[1] < gaps[0]


@pytest.mark.slow
def test_admm_limit_unique_minimiser_strictly_convex():
    # d = 1, E = I and a blur with nonvanishing spectrum: the data term is strictly convex,
    # so the minimiser is unique and the iterates themselves must agree.
    Yl, Yh, kern, R, E, G = _tiny(31, d=1, E_identity=True, H=5, W=6, center=0.6)
    assert np.abs(np.fft.fft2(nlpr.filter_image(nlpr.blur_taps(kern), 5, 6))).min() > 0.05
    K, S, lam1, lam2, rho, h = 1, 1, 0.5, 0.03, 0.1, 0.5
    om = nlpr.weights(G, K, S, h)
    X, _, _ = nlpr.admm(Yl, Yh, kern, 1, R, E, K, S, lam1, lam2, rho, om, 3000, fast=True)
    dp = DenseProblem(Yl, Yh, kern, 1, R, E, K, S, lam1, lam2, om)
    x_cp = dp.chambolle_pock(20000)
    assert np.abs(X.reshape(-1) - x_cp).max() < 1e-10


@pytest.mark.slow
def test_anisotropic_tv_ablation_limit_matches_chambolle_pock():
    # K = 0, omega = 1 on the 4-neighbour offsets and 0 on the diagonals of the 3x3 window:
    # phi is anisotropic TV (the paper's local-regulariser ablation); same CP comparison.
    Yl, Yh, kern, R, E, G = _tiny(34, d=2)
    K, S, lam1, lam2, rho = 0, 1, 0.8, 0.03, 0.5
    H, W = Yh.shape[:2]
    om = np.zeros((len(nlpr.search_offsets(S)), H, W))
    for t, tau in enumerate(nlpr.search_offsets(S)):
        if abs(tau[0]) + abs(tau[1]) == 1:
            om[t] = 1.0
    X, _, _ = nlpr.admm(Yl, Yh, kern, 2, R, E, K, S, lam1, lam2, rho, om, 6000, fast=True)
    dp = DenseProblem(Yl, Yh, kern, 2, R, E, K, S, lam1, lam2, om)
    f_admm = dp.objective(X.reshape(-1))
    # phi is the sum of |X_c(i) - X_c(i - e)| over both axes and both signs of e
    tv = sum(np.abs(X - nlpr.shift(X, e)).sum() for e in ((1, 0), (-1, 0), (0, 1), (0, -1)))
    f_def = nlpr.objective(X, Yl, Yh, kern, 2, R, E, np.zeros_like(om), K, S, lam1, 0.0) + lam2 * tv
    assert abs(f_admm - f_def) <= 1e-12 * abs(f_def)
    f_cp = dp.objective(dp.chambolle_pock(20000))
    assert abs(f_admm - f_cp) <= 1e-10 * abs(f_cp)


def test_lambda2_zero_is_least_squares():
    # lambda2 = 0: the ADMM limit minimises l(X) alone; compare with a dense least squares.
    Yl, Yh, kern, R, E, G = _tiny(32, d=1, E_identity=True, H=5, W=5, center=0.6)
    K, S, lam1, rho = 1, 1, 0.7, 0.1
    om = nlpr.weights(G, K, S, 0.5)
    X, _, _ = nlpr.admm(Yl, Yh, kern, 1, R, E, K, S, lam1, 0.0, rho, om, 2500, fast=True)
    dp = DenseProblem(Yl, Yh, kern, 1, R, E, K, S, lam1, 0.0, om)
    A = np.vstack([dp.M1, np.sqrt(lam1) * dp.M2])
    y = np.concatenate([dp.y1, np.sqrt(lam1) * dp.y2])
    ref = np.linalg.lstsq(A, y, rcond=None)[0]
    assert np.abs(X.reshape(-1) - ref).max() < 1e-9


def test_lambda2_huge_gives_constant_bands():
    # lambda2 -> infinity forces D X = 0, i.e. X constant per band (W generates Z^2);
    # the limit is the least-squares fit over constant images.
    Yl, Yh, kern, R, E, G = _tiny(33, d=2)
    K, S, lam1, rho = 1, 1, 0.9, 1.0
    om = nlpr.weights(G, K, S, 0.5)
    X, _, _ = nlpr.admm(Yl, Yh, kern, 2, R, E, K, S, lam1, 1e8, rho, om, 600, fast=True)
    H, W, Ls = X.shape
    dp = DenseProblem(Yl, Yh, kern, 2, R, E, K, S, lam1, 0.0, om)
    Cmat = np.kron(np.ones((H * W, 1)), np.eye(Ls))     # vec_row(1 a^T) = Cmat a
    A = np.vstack([dp.M1 @ Cmat, np.sqrt(lam1) * dp.M2 @ Cmat])
    y = np.concatenate([dp.y1, np.sqrt(lam1) * dp.y2])
    a = np.linalg.lstsq(A, y, rcond=None)[0]
    assert np.abs(X - a[None, None, :]).max() < 1e-8


def test_objective_plateaus():
    # The objective stabilises (Sec. V, convergence plot): late changes are tiny.
    Yl, Yh, kern, R, E, G = _tiny(34, d=2)
    K, S = 1, 1
    om = nlpr.weights(G, K, S, 0.5)
    vals = []
    cb = lambda st, su: vals.append(nlpr.objective(st.X, Yl, Yh, kern, 2, R, E, om, K, S, 0.8, 0.02))
    nlpr.admm(Yl, Yh, kern, 2, R, E, K, S, 0.8, 0.02, 0.5, om, 2000, fast=True, callback=cb)
    assert abs(vals[-1] - vals[-100]) <= 1e-4 * abs(vals[-1])
    tail = np.array(vals[-500:])
    assert np.all(np.diff(tail) <= 1e-12 * abs(vals[-1]))        # monotone tail


def test_residuals_follow_the_dual_updates_and_vanish_at_the_limit():
    # primal residual = size of the scaled-dual change of the same iteration (eqs. dualvar1_main,
    # dualvar2_main, dualvar3_main: Lambda1 - (B X - P1), Lambda2 - (X - P2), Sigma - (D X - Q));
    # both residuals -> 0 as the iterates converge (Theorem 1).
    Yl, Yh, kern, R, E, G = _tiny(35, d=2)
    K, S, lam1, lam2, rho = 1, 1, 0.8, 0.02, 0.5
    om = nlpr.weights(G, K, S, 0.5)
    su = nlpr.setup(Yl, Yh, kern, 2, R, E, K, S, lam1, lam2, rho, om)
    st = nlpr.State.zeros(su.H, su.W, su.L_s, K, S)
    from oracle import cloops
    hist = []
    for t in range(3000):
        nxt = nlpr.admm_step(st, su, latent_fn=cloops.latent_update, dtsum_fn=cloops.dt_sum)
        if t in (0, 1, 10, 2999):
            rp, rd = nlpr.residuals(st, nxt, su)
            dl = np.sqrt(((nxt.Lam1 - st.Lam1) ** 2).sum() + ((nxt.Lam2 - st.Lam2) ** 2).sum()
                         + ((nxt.Sig - st.Sig) ** 2).sum())
            assert abs(rp - dl) <= 1e-12 * max(dl, 1e-300)
            # dual residual another way: C = A^T (z + Lambda) and Lambda' - Lambda = -(A X' - z'),
            # so A^T (z' - z) = C' - C + A^T r' with r' = A X' - z'
            X = nxt.X
            Atr = nlpr.blur_t(nlpr.blur(X, kern) - nxt.P1, kern) + (X - nxt.P2)
            for ti, tau in enumerate(nlpr.search_offsets(S)):
                for kk, k in enumerate(nlpr.patch_offsets(K)):
                    Atr = Atr + nlpr.diff_op_t(nlpr.diff_op(X, tau, k) - nxt.Q[ti, kk], tau, k)
            sv = nlpr.rhs(nxt, su) - nlpr.rhs(st, su) + Atr
            rd2 = rho * np.sqrt((sv * sv).sum())
            assert abs(rd - rd2) <= 1e-9 * max(rd2, 1e-300)
            hist.append((rp, rd))
        st = nxt
    assert hist[0][0] > 1e-3 and hist[0][1] > 1e-3
    assert hist[-1][0] < 1e-6 * hist[0][0] and hist[-1][1] < 1e-4 * hist[0][1]
