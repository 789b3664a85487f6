"""Extrapolated tube treatment (ibim_solve_extrapolated) against the oracle's
and against the closed forms.

Born sphere (full Jacobian): the GPU's p* = 2 p(tau/2) - p(tau) and G* must
equal the oracle's extrapolation (FP64 to 1e-8, certified FP32 to 1e-5) and
lie within 1e-3 of the closed form.  Kirkwood sphere (80k nodes): the
extrapolated energy must be closer to the series solution than the tau = h
solve.
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


def test_born_extrapolation_matches_oracle_and_closed_form():
    R, h = 2.0, 0.25
    ctx = ibim.Context.sphere(R, h=h, band_eps=3 * h)
    ctx.set_charges(np.zeros((1, 3)), np.ones(1))
    ctx.set_jacobian(1)
    g = oracle.sphere_nodes(R, h=h, eps=3 * h)
    perm = _perm(ctx.nodes()["ijk"], g["ijk"])
    N = ctx.N
    z, q = np.zeros((1, 3)), np.ones(1)
    Po = oracle.Phys(1.0, 80.0, 0.1257, h, 0)
    po, Go, G1, G2 = oracle.extrapolated_energy(g["xs"], g["nrm"], oracle.jacobian_weights(g), Po, z, q, 1.0)
    exact = cf.born_energy(R, 1.0, 1.0, 80.0, 0.1257)
    P = ibim.Phys(1.0, 80.0, 0.1257, h, 0)
    d = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    info = ctx.solve_extrapolated(P, d, precision=ibim.IBIM_F64, tol=1e-10, restart=64, maxit=400)
    p = d.cpu().numpy()
    pref = np.concatenate([po[:N][perm], po[N:][perm]])
    err_p = np.linalg.norm(p - pref) / np.linalg.norm(pref)
    print("Born extrapolated: G* %.8e (oracle %.8e), |p - p_oracle| %.2e, vs closed form %.2e (tau = h: %.2e), "
          "iters %d" % (info["gpol"], Go, err_p, (info["gpol"] - exact) / exact, (G1 - exact) / exact, info["iters"]))
    assert err_p < 1e-8
    assert abs(info["gpol"] - Go) < 1e-8 * abs(Go)
    assert abs(info["gpol"] - exact) < 1e-3 * abs(exact)
    i32 = ctx.solve_extrapolated(P, d, precision=ibim.IBIM_F32C, tol=1e-6, restart=64, maxit=400, certify=1)
    assert i32["converged"] and abs(i32["gpol"] - Go) < 1e-5 * abs(Go)
    ctx.close()


def test_kirkwood_extrapolation_is_closer_to_the_series():
    R, h = 20.0, 0.5
    ctx = ibim.Context.sphere(R, h=h, band_eps=2 * h)
    z, q = inputs.kirkwood_charges(50, 16.0)
    ctx.set_charges(z, q)
    P = ibim.Phys(2.0, 80.0, 0.1257, h, 0)
    series = cf.kirkwood_energy(R, z, q, 2.0, 80.0, 0.1257)
    d = torch.empty(2 * ctx.N, dtype=torch.float64, device="cuda")
    opts = dict(precision=ibim.IBIM_F32C, tol=1e-7, restart=64, maxit=400, certify=1)
    e1 = (ctx.solve(P, d, **opts)["gpol"] - series) / series
    ctx.set_jacobian(1)
    eJ = (ctx.solve(P, d, **opts)["gpol"] - series) / series
    info = ctx.solve_extrapolated(P, d, **opts)
    ex = (info["gpol"] - series) / series
    print("Kirkwood energy error vs series: J = 1 %.3e, full J %.3e, full J + extrapolated %.3e (iters %d)"
          % (e1, eJ, ex, info["iters"]))
    assert info["converged"]
    assert abs(ex) < 0.5 * abs(eJ) and abs(ex) < 0.5 * abs(e1)
    ctx.close()
