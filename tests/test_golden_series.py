"""The stored Kirkwood series energies (tests/golden/kirkwood_series.json,
read by bench.py) equal the oracle's closed form on the same seeded charges."""
import json
import os

import numpy as np

import oracle
from oracle import closed_forms as cf
from paper_1709_08070_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def test_stored_series_energies_are_current():
    with open(os.path.join(HERE, "golden", "kirkwood_series.json")) as f:
        g = json.load(f)
    assert set(g["workloads"]) == {"kirkwood_sphere", "kirkwood_sphere_large"}
    for name, c in g["workloads"].items():
        z, q = inputs.kirkwood_charges(c["n_charges"], c["charge_ball"])
        e = cf.kirkwood_energy(c["R"], z, q, g["eps_in"], g["eps_out"], g["kappa"]) * oracle.KCAL_PER_E2_A
        np.testing.assert_allclose(c["gpol_kcal"], e, rtol=1e-12)
