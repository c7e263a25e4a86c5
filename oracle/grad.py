"""FP64 reverse pass of K unrolled ADMM iterations (TEST INFRASTRUCTURE ONLY; see nlpr.py).

Given dL/dX for the X of the last iteration, returns the gradients of L with respect to Y_l,
Y_h, lambda1, lambda2, rho and the weights omega through the whole unrolled ADMM of Sec. IV from
zero initialisation; weights_vjp carries dL/domega back to the guide through eq. wts.  Written on the oracle's own variables (P1, Lambda1, P2, Lambda2, Q, Sigma):
each update of Sec. IV is differentiated as printed, in reverse order:

  Sigma' = Sigma - (D X - Q')          (eq. dualvar3_main)
  Lambda2' = Lambda2 - (X - P2')       (eq. dualvar2_main)
  Lambda1' = Lambda1 - (B X - P1')     (eq. dualvar1_main)
  Q' = S(D X - Sigma, lambda2 omega / rho)                       (eq. Qj_main)
  P2' = (X - Lambda2 + lambda1/rho Yh R^T E^T) F                  (eq. Qm_update)
  P1' = mask (rho B X + S^T Yl E^T - rho Lambda1)(E E^T + rho I)^{-1}
        + (1 - mask)(B X - Lambda1)                               (eq. Qh_update)
  X = A^{-1} C,  A = I + B^T B + sum D^T D symmetric             (eq. x_linear_system_main)
  C = B^T (P1 + Lambda1) + P2 + Lambda2 + sum D^T (Q + Sigma)

Derivative of the soft threshold at |v| = mu: the a.e. derivative with the kink counted as
outside the dead zone (dQ/dv = 1, dQ/dmu = -sign(v)); both sides of every comparison use
the same rule.
"""
from __future__ import annotations

import numpy as np

from . import nlpr


def forward_tape(Yl, Yh, kern, d, R, E, K, S, lam1, lam2, rho, omega, iters, mask=None):
    """Forward ADMM from zero state keeping every input state and X (images (H, W, L))."""
    su = nlpr.setup(Yl, Yh, kern, d, R, E, K, S, lam1, lam2, rho, omega, mask)
    st = nlpr.State.zeros(su.H, su.W, su.L_s, K, S)
    tape = []
    for _ in range(iters):
        nxt = nlpr.admm_step(st, su)
        tape.append((st, nxt.X))
        st = nxt
    return tape, su, st


def backward(tape, su: nlpr.Setup, Yl, Yh, Xbar_last):
    """Gradients (dict) of L with dL/dX_last = Xbar_last."""
    H, W, Ls = su.H, su.W, su.L_s
    offs, poffs = nlpr.search_offsets(su.S), nlpr.patch_offsets(su.K)
    mask = su.mask[:, :, None]
    lam1, lam2, rho = su.lam1, su.lam2, su.rho
    G = su.E @ su.R                              # (L_s, L_h)
    D9b = (lam1 / rho) * su.YhRtEt               # (H, W, L_s)
    # adjoints of the state that leaves the current iteration
    z = lambda: np.zeros((H, W, Ls))
    P1b, L1b, P2b, L2b = z(), z(), z(), z()
    Qb = np.zeros_like(tape[0][0].Q)
    Sb = np.zeros_like(tape[0][0].Sig)
    D9ab, D9bb = z(), z()
    Fb = np.zeros((Ls, Ls))
    M1b = np.zeros((Ls, Ls))
    rho_b = 0.0
    S_mu = 0.0                                   # sum mubar * omega
    omega_b = np.zeros_like(su.omega)            # dL/domega (mu = lambda2 omega / rho)
    last = len(tape) - 1
    for t in range(last, -1, -1):
        st, X = tape[t]
        BX = nlpr.blur(X, su.kern)
        Xb = Xbar_last.copy() if t == last else z()
        BXb = z()
        if t != last:
            # Sigma' = Sigma - D X + Q'
            Qpb = Qb.copy()
            for ti, tau in enumerate(offs):
                for ki, k in enumerate(poffs):
                    Xb -= nlpr.diff_op_t(Sb[ti, ki], tau, k)
            Qpb += Sb
            Sig_in_b = Sb.copy()
            # Lambda2' = Lambda2 - X + P2'
            L2_in_b = L2b.copy()
            Xb -= L2b
            P2pb = P2b + L2b
            # Lambda1' = Lambda1 - B X + P1'
            L1_in_b = L1b.copy()
            BXb -= L1b
            P1pb = P1b + L1b
            # Q' = soft(D X - Sigma, mu)
            for ti, tau in enumerate(offs):
                mu = (lam2 * su.omega[ti] / rho)[:, :, None]
                for ki, k in enumerate(poffs):
                    v = nlpr.diff_op(X, tau, k) - st.Sig[ti, ki]
                    outside = np.abs(v) >= mu
                    vb = Qpb[ti, ki] * outside
                    mub = (-Qpb[ti, ki] * np.sign(v) * outside).sum(axis=2)
                    S_mu += float((mub * su.omega[ti]).sum())
                    omega_b[ti] += mub * (lam2 / rho)
                    Xb += nlpr.diff_op_t(vb, tau, k)
                    Sig_in_b[ti, ki] -= vb
            # P2' = a2 F
            a2 = X - st.Lam2 + D9b
            a2b = nlpr.img(nlpr.mat(P2pb) @ su.F.T, H, W)
            Xb += a2b
            L2_in_b -= a2b
            D9bb += a2b
            Fb += nlpr.mat(a2).T @ nlpr.mat(P2pb)
            # P1'
            a1 = rho * BX + su.SYlEt - rho * st.Lam1
            a1b = nlpr.img(nlpr.mat(mask * P1pb) @ su.inv_p1.T, H, W) * mask
            BXb += rho * a1b + (1.0 - mask) * P1pb
            L1_in_b += -rho * a1b - (1.0 - mask) * P1pb
            D9ab += a1b
            M1b += nlpr.mat(mask * a1).T @ nlpr.mat(mask * P1pb)
            rho_b += float((a1b * (BX - st.Lam1)).sum())
        else:
            Sig_in_b = np.zeros_like(Sb)
            L1_in_b, L2_in_b = z(), z()
        # B X
        Xb += nlpr.blur_t(BXb, su.kern)
        # X = A^{-1} C (A symmetric)
        Cb = nlpr.solve_x(Xb, su.denom)
        # C = B^T(P1 + Lambda1) + P2 + Lambda2 + sum D^T(Q + Sigma)
        BCb = nlpr.blur(Cb, su.kern)
        P1b = BCb
        L1b = L1_in_b + BCb
        P2b = Cb
        L2b = L2_in_b + Cb
        Qb = np.empty_like(Qb)
        Sb = Sig_in_b.copy()
        for ti, tau in enumerate(offs):
            for ki, k in enumerate(poffs):
                DCb = nlpr.diff_op(Cb, tau, k)
                Qb[ti, ki] = DCb
                Sb[ti, ki] += DCb
    # parameters
    g = {}
    g["lam2"] = S_mu / rho
    rho_b += -lam2 * S_mu / rho ** 2
    GGt = G @ G.T
    rho_b += float((Fb * ((lam1 / rho ** 2) * su.F @ GGt @ su.F)).sum())
    lam1_b = float((Fb * (-(1.0 / rho) * su.F @ GGt @ su.F)).sum())
    rho_b += float((M1b * (-su.inv_p1 @ su.inv_p1)).sum())
    rho_b += float((D9bb * (-D9b / rho)).sum())
    lam1_b += float((D9bb * (D9b / lam1)).sum())
    g["rho"] = rho_b
    g["lam1"] = lam1_b
    g["Yh"] = (lam1 / rho) * nlpr.img(nlpr.mat(D9bb) @ G, H, W)           # (H, W, L_h)
    g["Yl"] = nlpr.img(nlpr.mat(nlpr.decimate(D9ab, su.d)) @ su.E, H // su.d, W // su.d)
    g["omega"] = omega_b                                                     # (|W|, H, W)
    return g


def weights_vjp(G, K, S, h, omega_bar):
    """dL/dG (H, W, L_guide) for a loss that depends on the guide G only through
    omega = nlpr.weights(G, K, S, h) (eq. wts), given dL/domega (|W|, H, W):
      omega_tau(i) = exp(-dist_tau(i) / h^2),  dist_tau(i) = sum_k ||D_{tau k} G(i)||^2,
      dL/dG = sum_tau sum_k D_{tau k}^T ( -2/h^2 omega_bar_tau omega_tau  D_{tau k} G )."""
    omega = nlpr.weights(G, K, S, h)
    Gb = np.zeros_like(G)
    for t, tau in enumerate(nlpr.search_offsets(S)):
        a = (-2.0 / (h * h)) * omega_bar[t] * omega[t]
        for k in nlpr.patch_offsets(K):
            Gb += nlpr.diff_op_t(a[:, :, None] * nlpr.diff_op(G, tau, k), tau, k)
    return Gb


def unrolled_grad(Yl, Yh, kern, d, R, E, K, S, lam1, lam2, rho, omega, iters, Xbar_fn, mask=None):
    """Runs the forward tape and the reverse pass; Xbar_fn(X_last) gives dL/dX_last.
    Returns (X_last, grads)."""
    tape, su, _ = forward_tape(Yl, Yh, kern, d, R, E, K, S, lam1, lam2, rho, omega, iters, mask)
    X_last = tape[-1][1]
    return X_last, backward(tape, su, Yl, Yh, Xbar_fn(X_last))
