"""Writes the small text fixtures of tests/golden/ from oracle/ only (no CUDA path).

tiny_admm.json: a 6x8 problem (L_l=3, L_h=2, L_s=2, d=2, 3x3 blur, K=1, S=1) with its
inputs and the oracle's X after 1, 2 and 7 ADMM iterations of Sec. IV from zero
initialisation (threshold lambda2*omega/rho, eq. Qj_main), and after 1 and 7 iterations of
the variant that keeps S B in the X system (x_update="sb").  Regression fixture: the paper
prints no worked example, so these values are the oracle's, pinned by the oracle tests.

Run:  python tests/golden/make_golden.py
"""
import json
import pathlib
import sys

import numpy as np

ROOT = pathlib.Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))
from oracle import nlpr  # noqa: E402


def tiny_problem():
    rng = np.random.default_rng(2210)
    H, W, d, L_l, L_h, L_s = 6, 8, 2, 3, 2, 2
    E = np.linalg.qr(rng.standard_normal((L_l, L_s)))[0].T
    R = rng.random((L_l, L_h)); R /= R.sum(axis=0)
    k = rng.random((3, 3)) + 0.5; kern = k / k.sum()
    Yh = rng.random((H, W, L_h))
    Yl = rng.random((H // d, W // d, L_l))
    return dict(H=H, W=W, d=d, K=1, S=1, lam1=0.8, lam2=0.05, rho=0.3, h=0.5,
                E=E, R=R, kern=kern, Yh=Yh, Yl=Yl)


def main():
    p = tiny_problem()
    om = nlpr.weights(p["Yh"], p["K"], p["S"], p["h"])
    out = {k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    out["layout"] = "images (H, W, L); omega (|W|, H, W)"
    out["omega"] = om.tolist()
    st = None
    done = 0
    for n in (1, 2, 7):
        X, st, _ = nlpr.admm(p["Yl"], p["Yh"], p["kern"], p["d"], p["R"], p["E"], p["K"], p["S"],
                             p["lam1"], p["lam2"], p["rho"], om, n - done, state=st)
        done = n
        out[f"X_{n}"] = X.tolist()
    for n in (1, 7):
        X, _, _ = nlpr.admm(p["Yl"], p["Yh"], p["kern"], p["d"], p["R"], p["E"], p["K"], p["S"],
                            p["lam1"], p["lam2"], p["rho"], om, n, x_update="sb")
        out[f"Xsb_{n}"] = X.tolist()
    path = pathlib.Path(__file__).with_name("tiny_admm.json")
    path.write_text(json.dumps(out))
    print("wrote", path)


if __name__ == "__main__":
    main()
