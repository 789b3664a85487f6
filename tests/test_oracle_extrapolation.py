"""Pins of the extrapolated tube treatment (tau -> 0 by Richardson on tau and
tau/2, the regularisation error read as linear in tau), against the Born
closed form (Sec. 4.2):

* with the full Jacobian, the extrapolated energy is far closer to the closed
  form than either solve (h = 0.25: 2.5 % and 1.3 % -> below 0.1 %);
* its error falls as h^2 (h = 0.25 -> 0.125 divides it by about 4), while
  the tau = h error alone falls only as h.
"""
import numpy as np

import oracle
from oracle import closed_forms as cf


def _born(h):
    R = 2.0
    g = oracle.sphere_nodes(R, h=h, eps=3 * h)
    w = oracle.jacobian_weights(g)
    z, q = np.zeros((1, 3)), np.ones(1)
    P = oracle.Phys(1.0, 80.0, 0.1257, h, 0)
    exact = cf.born_energy(R, 1.0, 1.0, 80.0, 0.1257)
    _, Gx, G1, G2 = oracle.extrapolated_energy(g["xs"], g["nrm"], w, P, z, q, 1.0, tol=1e-9)
    assert Gx == 2.0 * G2 - G1
    return (G1 - exact) / exact, (Gx - exact) / exact


def test_extrapolated_born_energy_is_second_order():
    e1a, exa = _born(0.25)
    e1b, exb = _born(0.125)
    print("tau = h: %.3e -> %.3e; extrapolated: %.3e -> %.3e" % (e1a, e1b, exa, exb))
    assert abs(exa) < 1e-3 and abs(exa) < 0.05 * abs(e1a)
    assert abs(exb) < 0.35 * abs(exa)          # second order in h
    assert abs(e1b) > 0.4 * abs(e1a)           # the tau = h error alone is first order
