"""Regression of the oracle against tests/golden/tiny_admm.json (written from oracle/ by
tests/golden/make_golden.py)."""
import json
import pathlib

import numpy as np

from oracle import nlpr

GOLD = pathlib.Path(__file__).with_name("golden") / "tiny_admm.json"


def test_oracle_reproduces_golden():
    g = json.loads(GOLD.read_text())
    a = {k: np.array(v) if isinstance(v, list) else v for k, v in g.items()}
    om = nlpr.weights(a["Yh"], a["K"], a["S"], a["h"])
    assert np.abs(om - a["omega"]).max() < 1e-14
    X, st, _ = nlpr.admm(a["Yl"], a["Yh"], a["kern"], a["d"], a["R"], a["E"], a["K"], a["S"],
                         a["lam1"], a["lam2"], a["rho"], om, 7)
    assert np.abs(X - a["X_7"]).max() <= 1e-12 * np.abs(a["X_7"]).max()


def test_oracle_sb_variant_reproduces_golden():
    g = json.loads(GOLD.read_text())
    a = {k: np.array(v) if isinstance(v, list) else v for k, v in g.items()}
    om = np.array(a["omega"])
    for n in (1, 7):
        X, _, _ = nlpr.admm(a["Yl"], a["Yh"], a["kern"], a["d"], a["R"], a["E"], a["K"], a["S"],
                            a["lam1"], a["lam2"], a["rho"], om, n, x_update="sb")
        ref = a[f"Xsb_{n}"]
        assert np.abs(X - ref).max() <= 1e-12 * np.abs(ref).max()
