"""Pins of the oracle's reverse pass (oracle/grad.py): central finite differences of the FP64
forward in every input direction (Y_l, Y_h, lambda1, lambda2, rho), on tiny problems whose
soft-threshold active set is stable under the step."""
import numpy as np
import pytest

from oracle import nlpr, grad


def _tiny(seed, d=2):
    rng = np.random.default_rng(seed)
    H, W, L_l, L_h, L_s = 6, 8, 3, 2, 2
    E = np.linalg.qr(rng.standard_normal((L_l, L_s)))[0].T
    R = rng.random((L_l, L_h)); R /= R.sum(axis=0)
    k = rng.random((3, 3)) + 0.5; kern = k / k.sum()
    Yh = rng.random((H, W, L_h))
    Yl = rng.random((H // d, W // d, L_l))
    om = nlpr.weights(Yh, 1, 1, 0.5)
    return dict(Yl=Yl, Yh=Yh, kern=kern, d=d, R=R, E=E, K=1, S=1, lam1=0.8, lam2=0.05, rho=0.3,
                omega=om)


def _loss(p, Wt, iters):
    X, _, _ = nlpr.admm(p["Yl"], p["Yh"], p["kern"], p["d"], p["R"], p["E"], p["K"], p["S"], p["lam1"],
                        p["lam2"], p["rho"], p["omega"], iters)
    return float((Wt * X).sum())


@pytest.mark.parametrize("iters", [1, 2, 5])
def test_reverse_pass_matches_central_differences(iters):
    p = _tiny(40)
    rng = np.random.default_rng(41)
    Wt = rng.standard_normal((6, 8, 2))
    X, g = grad.unrolled_grad(p["Yl"], p["Yh"], p["kern"], p["d"], p["R"], p["E"], p["K"], p["S"], p["lam1"],
                              p["lam2"], p["rho"], p["omega"], iters, lambda X: Wt)
    h = 1e-6
    for key in ("Yl", "Yh"):
        dirn = rng.standard_normal(p[key].shape)
        q_plus = dict(p); q_plus[key] = p[key] + h * dirn
        q_minus = dict(p); q_minus[key] = p[key] - h * dirn
        fd = (_loss(q_plus, Wt, iters) - _loss(q_minus, Wt, iters)) / (2 * h)
        an = float((g[key] * dirn).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (key, fd, an)
    for key in ("lam1", "lam2", "rho"):
        q_plus = dict(p); q_plus[key] = p[key] + h
        q_minus = dict(p); q_minus[key] = p[key] - h
        fd = (_loss(q_plus, Wt, iters) - _loss(q_minus, Wt, iters)) / (2 * h)
        assert abs(fd - g[key]) <= 1e-6 * max(1.0, abs(g[key])), (key, fd, g[key])


def test_reverse_pass_with_identity_subspace_and_no_decimation():
    p = _tiny(42, d=1)
    p["E"] = np.eye(3)
    p["Yl"] = np.random.default_rng(43).random((6, 8, 3))
    rng = np.random.default_rng(44)
    Wt = rng.standard_normal((6, 8, 3))
    iters = 3
    X, g = grad.unrolled_grad(p["Yl"], p["Yh"], p["kern"], p["d"], p["R"], p["E"], p["K"], p["S"], p["lam1"],
                              p["lam2"], p["rho"], p["omega"], iters, lambda X: Wt)
    h = 1e-6
    for key in ("Yl", "Yh", "rho", "lam2"):
        if key in ("Yl", "Yh"):
            dirn = rng.standard_normal(p[key].shape)
            qp = dict(p); qp[key] = p[key] + h * dirn
            qm = dict(p); qm[key] = p[key] - h * dirn
            an = float((g[key] * dirn).sum())
        else:
            qp = dict(p); qp[key] = p[key] + h
            qm = dict(p); qm[key] = p[key] - h
            an = g[key]
        fd = (_loss(qp, Wt, iters) - _loss(qm, Wt, iters)) / (2 * h)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (key, fd, an)


def test_weight_and_guide_gradients_match_central_differences():
    # omega enters only through mu = lambda2 omega / rho; the guide only through omega (eq. wts)
    p = _tiny(45)
    rng = np.random.default_rng(46)
    Wt = rng.standard_normal((6, 8, 2))
    iters = 4
    G = rng.random((6, 8, 2))                       # a guide other than Y_h
    h_w = 0.5
    p["omega"] = nlpr.weights(G, p["K"], p["S"], h_w)
    X, g = grad.unrolled_grad(p["Yl"], p["Yh"], p["kern"], p["d"], p["R"], p["E"], p["K"], p["S"], p["lam1"],
                              p["lam2"], p["rho"], p["omega"], iters, lambda X: Wt)
    h = 1e-6
    d_om = rng.standard_normal(p["omega"].shape)
    qp = dict(p); qp["omega"] = p["omega"] + h * d_om
    qm = dict(p); qm["omega"] = p["omega"] - h * d_om
    fd = (_loss(qp, Wt, iters) - _loss(qm, Wt, iters)) / (2 * h)
    an = float((g["omega"] * d_om).sum())
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)
    # <omega_bar, omega> = lambda2 dL/dlambda2 (mu depends on lambda2 omega only)
    assert abs(float((g["omega"] * p["omega"]).sum()) - p["lam2"] * g["lam2"]) <= 1e-9 * max(1.0, abs(an))
    Gb = grad.weights_vjp(G, p["K"], p["S"], h_w, g["omega"])
    d_g = rng.standard_normal(G.shape)
    qp = dict(p); qp["omega"] = nlpr.weights(G + h * d_g, p["K"], p["S"], h_w)
    qm = dict(p); qm["omega"] = nlpr.weights(G - h * d_g, p["K"], p["S"], h_w)
    fd = (_loss(qp, Wt, iters) - _loss(qm, Wt, iters)) / (2 * h)
    an = float((Gb * d_g).sum())
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_weights_vjp_matches_central_differences_of_the_weights():
    # the guide step alone: L = <V, omega(G)> for a random V
    rng = np.random.default_rng(47)
    G = rng.random((7, 9, 2))
    K, S, hw = 1, 2, 0.7
    V = rng.standard_normal((len(nlpr.search_offsets(S)), 7, 9))
    Gb = grad.weights_vjp(G, K, S, hw, V)
    d = rng.standard_normal(G.shape)
    e = 1e-6
    fd = (float((V * nlpr.weights(G + e * d, K, S, hw)).sum()) -
          float((V * nlpr.weights(G - e * d, K, S, hw)).sum())) / (2 * e)
    assert abs(fd - float((Gb * d).sum())) <= 1e-7 * max(1.0, abs(fd))


def test_reverse_pass_with_a_sampling_mask():
    # a random sampling mask (d = 1): dL/dY_l vanishes off the mask and matches central differences
    p = _tiny(48, d=1)
    rng = np.random.default_rng(49)
    mask = (rng.random((6, 8)) < 0.4).astype(float)
    p["Yl"] = rng.random((6, 8, 3))
    Wt = rng.standard_normal((6, 8, 2))
    iters = 4

    def loss(q):
        X, _, _ = nlpr.admm(q["Yl"], q["Yh"], q["kern"], 1, q["R"], q["E"], q["K"], q["S"], q["lam1"],
                            q["lam2"], q["rho"], q["omega"], iters, mask=mask)
        return float((Wt * X).sum())

    X, g = grad.unrolled_grad(p["Yl"], p["Yh"], p["kern"], 1, p["R"], p["E"], p["K"], p["S"], p["lam1"],
                              p["lam2"], p["rho"], p["omega"], iters, lambda X: Wt, mask=mask)
    assert not g["Yl"][mask == 0].any()
    h = 1e-6
    for key in ("Yl", "Yh", "rho"):
        if key == "rho":
            qp = dict(p); qp[key] = p[key] + h
            qm = dict(p); qm[key] = p[key] - h
            an = g[key]
        else:
            dirn = rng.standard_normal(p[key].shape)
            qp = dict(p); qp[key] = p[key] + h * dirn
            qm = dict(p); qm[key] = p[key] - h * dirn
            an = float((g[key] * dirn).sum())
        fd = (loss(qp) - loss(qm)) / (2 * h)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (key, fd, an)
