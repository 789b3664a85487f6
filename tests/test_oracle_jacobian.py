"""Pins of the full Jacobian J = 1 - d lap(d) + d^2 sigma2(Hess d) (Sec. 2.2,
with the sum of the Hessian's 2x2 principal minors as the last term), which
the paper's runs replace by J = 1.

* Sphere: the weights J delta_eps(d) h^3 integrate the constant 1 to the exact
  area 4 pi R^2 (the J = 1 weights give 4 pi (R^2 + c eps^2), c = 1/3 - 2/pi^2).
* Level sets built from analytic distance functions on a grid: J = 1 for a
  plane, a/(a + d) for a cylinder of radius a and (R/(R + d))^2 for a sphere,
  to second order in h (central-difference Hessian).
"""
import numpy as np
import pytest

import oracle

C_EPS = 1.0 / 3.0 - 2.0 / np.pi ** 2


@pytest.mark.parametrize("h", [0.25, 0.125])
def test_sphere_area_is_exact_with_full_jacobian(h):
    R, eps = 2.0, 3 * h
    g = oracle.sphere_nodes(R, h=h, eps=eps, origin=(0.013, -0.021, 0.007))
    A = 4 * np.pi * R * R
    a1 = g["w"].sum() / A - 1.0
    aj = oracle.jacobian_weights(g).sum() / A - 1.0
    assert abs(a1 - C_EPS * eps * eps / (R * R)) < 0.1 * C_EPS * eps * eps / (R * R)
    assert abs(aj) < 5e-4 and abs(aj) < 0.05 * abs(a1), (a1, aj)


def _band(phi_fn, h, half):
    """Band of an analytic distance on a cube of (2 half + 1)^3 nodes, restricted
    to nodes whose second-difference stencil lies inside the box (a level-set
    box leaves a margin of several cells around its band)."""
    n = 2 * half + 1
    g = oracle.make_grid((-half, -half, -half), (n, n, n), h)
    X = oracle.grid_coords(g)
    phi = phi_fn(X)
    b = oracle.ls_band(g, phi, 2 * h)
    keep = np.all(np.abs(b["ijk"]) < half, axis=1)
    return {k: v[keep] for k, v in b.items()}


def test_levelset_jacobian_of_a_plane_is_one():
    b = _band(lambda X: 0.31 * X[..., 0] - 0.52 * X[..., 1] + 0.795 * X[..., 2] - 0.2, 0.25, 16)
    assert b["w"].size > 100
    assert np.max(np.abs(oracle.jacobian(b) - 1.0)) < 1e-12
    assert np.max(np.abs(b["sig2"])) < 1e-10


@pytest.mark.parametrize("shape", ["cylinder", "sphere"])
def test_levelset_jacobian_converges_to_closed_form(shape):
    a = 2.0
    errs = []
    for h in (0.2, 0.1):
        if shape == "cylinder":
            b = _band(lambda X: np.sqrt(X[..., 0] ** 2 + X[..., 1] ** 2 + 0.0) - a, h, int(3.5 / h))
            exact = a / (a + b["d"])
        else:
            b = _band(lambda X: np.sqrt((X ** 2).sum(-1)) - a, h, int(3.5 / h))
            exact = (a / (a + b["d"])) ** 2
        errs.append(np.max(np.abs(oracle.jacobian(b) - exact)))
    # second order: halving h divides the error by about 4
    assert errs[1] < 0.35 * errs[0] and errs[1] < 2e-3, errs


def test_levelset_sphere_area_with_full_jacobian():
    R, h = 2.0, 0.125
    b = _band(lambda X: np.sqrt(((X - np.array([0.03, -0.02, 0.01])) ** 2).sum(-1)) - R, h, int(3.5 / h))
    A = 4 * np.pi * R * R
    a1 = b["w"].sum() / A - 1.0
    aj = oracle.jacobian_weights(b).sum() / A - 1.0
    assert abs(aj) < 0.1 * abs(a1), (a1, aj)


def test_born_energy_with_jacobian_does_not_depend_on_the_band_width():
    """With J = 1 the Born energy drifts as the band widens (the O(eps^2) area
    bias); with the full J it does not, and it is closer to the closed form."""
    from oracle import closed_forms as cf
    R, h = 2.0, 0.25
    exact = cf.born_energy(R, 1.0, 1.0, 80.0, 0.1257)
    z, q = np.zeros((1, 3)), np.ones(1)
    P = oracle.Phys(1.0, 80.0, 0.1257, h, 0)
    err = {}
    for k in (3, 4):
        g = oracle.sphere_nodes(R, h=h, eps=k * h)
        b = oracle.rhs(g["xs"], g["nrm"], z, q, 1.0)
        for name, w in (("one", g["w"]), ("full", oracle.jacobian_weights(g))):
            x, *_ = oracle.gmres(g["xs"], g["nrm"], w, P, b, tol=1e-10)
            G = oracle.gpol(q, oracle.psi_rxn(g["xs"], g["nrm"], w, z, P, x))
            err[(name, k)] = (G - exact) / exact
    assert abs(err[("full", 3)] - err[("full", 4)]) < 0.1 * abs(err[("one", 3)] - err[("one", 4)]), err
    assert abs(err[("full", 3)]) < abs(err[("one", 3)]) and abs(err[("full", 4)]) < abs(err[("one", 4)]), err
