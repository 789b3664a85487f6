"""Batched solve (ibim_solve_batch) against one-molecule solves.

Molecules of uneven size and screening constant (analytic spheres, small
level-set globules, one caller-given node cloud) are solved together in one
batch with the FP32 operator, and each one alone with ibim_solve at the same
tolerance; the solutions and energies must agree to the FP32 tolerance, and
each batched energy must agree with the FP64 solve of the same molecule to
1e-4.
"""
import numpy as np
import pytest

from paper_1709_08070_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1709_08070_gb300 import ibim  # noqa: E402


def _molecules():
    mols = []
    for R, h, kappa in ((2.0, 0.25, 0.1257), (4.0, 0.5, 0.0), (6.0, 0.5, 0.2)):
        ctx = ibim.Context.sphere(R, h=h, band_eps=2 * h)
        z, q = inputs.kirkwood_charges(n=3, ball_radius=0.6 * R, seed=int(R * 10))
        ctx.set_charges(z, q)
        mols.append((ctx, ibim.Phys(2.0, 80.0, kappa, h, 0)))
    for n_atoms, kappa in ((40, 0.05), (120, 0.15)):
        z, r, q = inputs.globule_atoms(n_atoms, seed=100 + n_atoms)
        ctx = ibim.Context.molecule(z, r, q, probe=1.4, h=0.5)
        mols.append((ctx, ibim.Phys(1.0, 80.0, kappa, 0.5, 0)))
    xs, nr, w = inputs.sphere_cloud(3000, radius=5.0, seed=7)
    ctx = ibim.Context.from_nodes(xs, nr, w, h=0.3)
    ctx.set_charges(np.array([[0.5, 0.0, 0.0]]), np.array([1.0]))
    mols.append((ctx, ibim.Phys(4.0, 80.0, 0.1, 0.3, 0)))
    return mols


def test_batch_matches_single_solves():
    mols = _molecules()
    try:
        ctxs = [c for c, _ in mols]
        physs = [p for _, p in mols]
        outs = [torch.empty(2 * c.N, dtype=torch.float64, device="cuda") for c in ctxs]
        infos = ibim.ibim_solve_batch(ctxs, physs, outs, precision=ibim.IBIM_F32C, tol=1e-8, restart=64, maxit=400)
        for (ctx, P), d, info in zip(mols, outs, infos):
            assert info["converged"] and info["relres"] < 1e-8, info
            ref = torch.empty_like(d)
            i1 = ctx.solve(P, ref, precision=ibim.IBIM_F32C, tol=1e-8, restart=64, maxit=400)
            a, b = d.cpu().numpy(), ref.cpu().numpy()
            err = np.linalg.norm(a - b) / np.linalg.norm(b)
            print("batch N=%d iters %d vs %d, rel diff %.2e, G %.6f vs %.6f" %
                  (ctx.N, info["iters"], i1["iters"], err, info["gpol"], i1["gpol"]))
            assert err < 1e-5
            assert abs(info["gpol"] - i1["gpol"]) <= 1e-5 * abs(i1["gpol"])
            d64 = torch.empty_like(d)
            i64 = ctx.solve(P, d64, precision=ibim.IBIM_F64, tol=1e-8, restart=64, maxit=400)
            assert abs(info["gpol"] - i64["gpol"]) <= 1e-4 * abs(i64["gpol"])
    finally:
        for c, _ in mols:
            c.close()


def test_batch_from_caller_starts():
    """start = 3: each molecule starts from the vector in its output buffer.
    From the converged solutions the batch stops at once with the same
    energies; from a perturbed solution it needs fewer iterations than from
    zero and reaches the same solution."""
    mols = _molecules()[:4]
    try:
        ctxs = [c for c, _ in mols]
        physs = [p for _, p in mols]
        opts = dict(precision=ibim.IBIM_F32C, tol=1e-7, restart=64, maxit=400)
        ref = [torch.empty(2 * c.N, dtype=torch.float64, device="cuda") for c in ctxs]
        i0 = ibim.ibim_solve_batch(ctxs, physs, ref, **opts)
        outs = [r.clone() for r in ref]
        i1 = ibim.ibim_solve_batch(ctxs, physs, outs, start=3, **opts)
        for a, b, r, o in zip(i0, i1, ref, outs):
            assert b["converged"] and b["iters"] <= 2, b
            assert abs(a["gpol"] - b["gpol"]) <= 1e-6 * abs(a["gpol"])
        gen = torch.Generator(device="cuda").manual_seed(5)
        outs = [r * (1.0 + 0.05 * torch.randn(r.shape, dtype=torch.float64, device="cuda", generator=gen))
                for r in ref]
        i2 = ibim.ibim_solve_batch(ctxs, physs, outs, start=3, **opts)
        for a, b, r, o in zip(i0, i2, ref, outs):
            err = float(torch.linalg.norm(o - r) / torch.linalg.norm(r))
            print("batch start=3 perturbed: iters %d (zero start %d), rel diff %.1e" % (b["iters"], a["iters"], err))
            assert b["converged"] and b["iters"] < a["iters"] and err < 1e-5
    finally:
        for c, _ in mols:
            c.close()


def test_batch_rejects_unsupported_options():
    ctx = ibim.Context.sphere(2.0, h=0.25)
    ctx.set_charges(np.zeros((1, 3)), np.ones(1))
    d = torch.empty(2 * ctx.N, dtype=torch.float64, device="cuda")
    P = ibim.Phys(1.0, 80.0, 0.1257, 0.25, 0)
    with pytest.raises(ibim.IbimError) as e:
        ibim.ibim_solve_batch([ctx], [P], [d], precision=ibim.IBIM_F64)
    assert e.value.status == 1
    with pytest.raises(ibim.IbimError) as e:
        ibim.ibim_solve_batch([ctx], [P], [d], start=1)
    assert e.value.status == 1
    with pytest.raises(ibim.IbimError) as e:
        ibim.ibim_solve_batch([ctx, ctx], [P, P], [d, d])
    assert e.value.status == 1
    ctx.close()
