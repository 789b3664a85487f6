"""Writes kirkwood_series.json: the Kirkwood series G_pol (kcal/mol) of the two
Kirkwood-type sphere workloads, from the oracle's closed form only (Sec. 4.2
test problem: charges inside a dielectric sphere in an ionic solvent).

Run from the repository root: python tests/golden/make_kirkwood_series.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import closed_forms as cf  # noqa: E402
from oracle import KCAL_PER_E2_A  # noqa: E402
from paper_1709_08070_gb300 import inputs  # noqa: E402

CASES = {
    "kirkwood_sphere": dict(R=20.0, n_charges=50, charge_ball=16.0),
    "kirkwood_sphere_large": dict(R=60.0, n_charges=50, charge_ball=48.0),
}
EPS_IN, EPS_OUT, KAPPA = 2.0, 80.0, 0.1257


def main():
    out = {"eps_in": EPS_IN, "eps_out": EPS_OUT, "kappa": KAPPA, "unit": "kcal/mol", "workloads": {}}
    for name, c in CASES.items():
        z, q = inputs.kirkwood_charges(c["n_charges"], c["charge_ball"])
        g = cf.kirkwood_energy(c["R"], z, q, EPS_IN, EPS_OUT, KAPPA) * KCAL_PER_E2_A
        out["workloads"][name] = dict(c, gpol_kcal=g)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "kirkwood_series.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
