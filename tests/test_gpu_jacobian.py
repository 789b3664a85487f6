"""Full Jacobian J (ibim_set_jacobian / ibim_get_jacobian) against the oracle.

Spheres: J, the Laplacian of d at each node and the J weights must equal the
oracle's analytic values; with J the weights integrate 1 to the exact area.
Level sets: J from the central-difference Hessian of phi must equal the
oracle's on the shared node set (both sides build phi independently; it
agrees to round-off).  A Born solve with the J weights must match the
oracle's FP64 solve with the same weights, and mode 0 restores the J = 1
weights exactly.
"""
import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from paper_1709_08070_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1709_08070_gb300 import ibim  # noqa: E402


def _perm(gpu_ijk, orc_ijk):
    key = {tuple(v): i for i, v in enumerate(orc_ijk)}
    return np.array([key[tuple(v)] for v in gpu_ijk])


def test_sphere_jacobian_weights_and_area():
    R, h = 2.0, 0.25
    eps = 3 * h
    ctx = ibim.Context.sphere(R, h=h, band_eps=eps)
    g = oracle.sphere_nodes(R, h=h, eps=eps)
    n1 = ctx.nodes()
    perm = _perm(n1["ijk"], g["ijk"])
    np.testing.assert_allclose(ctx.curvature(), g["curv"][perm], rtol=1e-13, atol=0)
    J = ctx.jacobian()
    np.testing.assert_allclose(J, oracle.jacobian(g)[perm], rtol=1e-12, atol=1e-14)
    ctx.set_jacobian(1)
    nJ = ctx.nodes()
    np.testing.assert_allclose(nJ["w"], oracle.jacobian_weights(g)[perm], rtol=1e-12, atol=0)
    A = 4 * np.pi * R * R
    a1 = n1["w"].sum() / A - 1.0
    aJ = ctx.area() / A - 1.0
    print("sphere area error: J = 1 %.3e, full J %.3e" % (a1, aJ))
    assert abs(aJ) < 5e-4 and abs(aJ) < 0.05 * abs(a1)
    ctx.set_jacobian(0)
    assert np.array_equal(ctx.nodes()["w"], n1["w"])
    ctx.close()


def test_levelset_jacobian_matches_oracle():
    z, r, q = inputs.globule_atoms(40, seed=21)
    probe, h, eps = 1.4, 0.5, 1.0
    ctx = ibim.Context.molecule(z, r, None, probe=probe, h=h, band_eps=eps)
    gr, phi_o, _ = oracle.ls_ses(z, r, probe, h, eps)
    bo = oracle.ls_band(gr, phi_o, eps)
    bg = ctx.nodes()
    ko = {tuple(v): i for i, v in enumerate(bo["ijk"])}
    common = [(j, ko[tuple(v)]) for j, v in enumerate(bg["ijk"]) if tuple(v) in ko]
    jg = np.array([a for a, _ in common])
    jo = np.array([b for _, b in common])
    assert len(jg) > 0.99 * len(bg["w"])
    Jg = ctx.jacobian()[jg]
    Jo = oracle.jacobian(bo)[jo]
    err = np.max(np.abs(Jg - Jo))
    print("level-set J: range [%.3f, %.3f], max |GPU - oracle| %.2e" % (Jo.min(), Jo.max(), err))
    assert err < 1e-7, err
    ctx.set_jacobian(1)
    wJ = ctx.nodes()["w"][jg]
    np.testing.assert_allclose(wJ, oracle.jacobian_weights(bo)[jo], rtol=0, atol=1e-7 * h ** 3)
    ctx.close()


def test_born_solve_with_jacobian_matches_oracle_and_is_more_accurate():
    R, h = 2.0, 0.25
    eps = 3 * h
    ctx = ibim.Context.sphere(R, h=h, band_eps=eps)
    ctx.set_charges(np.zeros((1, 3)), np.ones(1))
    g = oracle.sphere_nodes(R, h=h, eps=eps)
    P = ibim.Phys(1.0, 80.0, 0.1257, h, 0)
    Po = oracle.Phys(1.0, 80.0, 0.1257, h, 0)
    exact = cf.born_energy(R, 1.0, 1.0, 80.0, 0.1257)
    d = torch.empty(2 * ctx.N, dtype=torch.float64, device="cuda")
    i1 = ctx.solve(P, d, precision=ibim.IBIM_F64, tol=1e-10, restart=64, maxit=300)
    ctx.set_jacobian(1)
    iJ = ctx.solve(P, d, precision=ibim.IBIM_F64, tol=1e-10, restart=64, maxit=300)
    z, q = np.zeros((1, 3)), np.ones(1)
    wJ = oracle.jacobian_weights(g)
    b = oracle.rhs(g["xs"], g["nrm"], z, q, 1.0)
    x, *_ = oracle.gmres(g["xs"], g["nrm"], wJ, Po, b, tol=1e-10)
    Go = oracle.gpol(q, oracle.psi_rxn(g["xs"], g["nrm"], wJ, z, Po, x))
    e1, eJ = (i1["gpol"] - exact) / exact, (iJ["gpol"] - exact) / exact
    print("Born energy error: J = 1 %.3e, full J %.3e (oracle with J %.3e)" % (e1, eJ, (Go - exact) / exact))
    assert abs(iJ["gpol"] - Go) < 1e-8 * abs(Go)
    assert abs(eJ) < abs(e1)
    f32 = ctx.solve(P, d, precision=ibim.IBIM_F32C, tol=1e-8, restart=64, maxit=300, certify=1)
    assert abs(f32["gpol"] - Go) < 1e-5 * abs(Go)
    ctx.close()


def test_caller_nodes_keep_their_weights():
    xs, nr, w = inputs.sphere_cloud(500, radius=4.0, seed=3)
    ctx = ibim.Context.from_nodes(xs, nr, w, h=0.3)
    ctx.set_jacobian(0)
    with pytest.raises(ibim.IbimError) as e:
        ctx.set_jacobian(1)
    assert e.value.status == 7  # IBIM_ERR_STATE
    with pytest.raises(ibim.IbimError):
        ctx.jacobian()
    np.testing.assert_array_equal(ctx.nodes()["w"], w)
    ctx.close()
