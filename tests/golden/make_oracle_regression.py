"""Writes oracle_regression.json: values of the FP64 oracle (and only the oracle) on two
tiny seeded cases, stored so that a later change of the oracle's arithmetic shows up as a
failing regression test and has to be justified by the passage of the paper it follows.
These are not paper values and pin nothing by themselves; the pins are the closed-form,
invariant and finite-difference tests of the oracle.

Run from the repository root:  python tests/golden/make_oracle_regression.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pm  # noqa: E402
from paper_2211_09815_gb300 import inputs  # noqa: E402

CASES = {
    "za_8_16_4": dict(box=24.0, n_mesh=16, n_ptcl=8, n_steps=4, lpt_order=1),
    "lpt2_8_16_4": dict(box=24.0, n_mesh=16, n_ptcl=8, n_steps=4, lpt_order=2),
}


def evaluate(case):
    cfg = pm.PMConfig(**case)
    th = inputs.THETA_FIDUCIAL
    om = inputs.white_noise(cfg.n_ptcl, 1).astype(np.float64)
    target = pm.forward(inputs.white_noise(cfg.n_ptcl, 2).astype(np.float64), th, cfg)["delta"]
    loss, adj, fwd = pm.loss_and_gradient(om, th, target, cfg)
    _, pk, _ = pm.power_spectrum(fwd["delta"], cfg.box)
    g = adj["grad_omega"]
    return {
        "loss": loss,
        "grad_omega_norm": float(np.linalg.norm(g)),
        "grad_omega_first": [float(v) for v in g[:8]],
        "grad_theta": [float(v) for v in adj["grad_theta"]],
        "final_disp_rms": float(np.sqrt(np.mean(fwd["s"] ** 2))),
        "pk": [float(v) for v in pk],
    }


if __name__ == "__main__":
    out = {name: evaluate(case) for name, case in CASES.items()}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json"), "w") as f:
        json.dump({"cases": CASES, "values": out}, f, indent=1)
