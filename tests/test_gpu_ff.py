"""The float-float operator (IBIM_FF) against the FP64 oracle, and the
certified FP32 solve that uses it.

IBIM_FF evaluates the discrete system of Sec. 2.2 (regularisation of
Sec. 2.2.1) with every quantity held as an unevaluated sum of two floats.  It
must reproduce the oracle to the plain FP64 path's bar, 1e-10 of max |y| per
element and output block, on tiny and ragged caller clouds, both tube rules,
kappa = 0, a molecule far from the origin and a large sphere (where the
power-of-two grid of the coordinates is coarsest).  A certified FP32 solve
(certify = 1) reports the residual the oracle computes for its solution, as
the plain FP64 certification (certify = 2) does.
"""
import numpy as np
import pytest

import oracle
from paper_1709_08070_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1709_08070_gb300 import ibim  # noqa: E402

TOL = 1e-10


def _worst_blocks(y, yo, N):
    out = []
    for blk in (slice(0, N), slice(N, 2 * N)):
        out += [float(np.linalg.norm(y[blk] - yo[blk]) / np.linalg.norm(yo[blk])),
                float(np.max(np.abs(y[blk] - yo[blk])) / np.max(np.abs(yo[blk])))]
    return out


def _match(gpu_ijk, orc_ijk):
    ko = {tuple(v): i for i, v in enumerate(orc_ijk)}
    return np.array([ko[tuple(v)] for v in gpu_ijk], dtype=np.int64)


@pytest.mark.parametrize("symmetric", [1, 0])
def test_ff_tiny_and_ragged_caller_clouds(symmetric):
    """Both float-float kernels (symmetric, one-directional) on clouds with fewer
    nodes than a chunk, a ragged last chunk and tile, and several tiles."""
    for n in (1, 2, 3, 33, 257, 1000, 3001):
        xs, nr, w = inputs.sphere_cloud(n, radius=3.0, seed=100 + n)
        ctx = ibim.Context.from_nodes(xs, nr, w, h=0.25)
        try:
            ctx.set_ff_kernel(symmetric)
            for rule in (0, 1):
                P = ibim.Phys(2.0, 80.0, 0.1257, 0.3, rule)
                Po = oracle.Phys(2.0, 80.0, 0.1257, 0.3, rule)
                p = inputs.random_vector(2 * n, seed=n)
                y = ctx.matvec_host(P, p, precision=ibim.IBIM_FF)
                e = _worst_blocks(y, oracle.matvec(xs, nr, w, Po, p), n)
                print("ff (symmetric %d) cloud n=%d rule %d: %s" % (symmetric, n, rule,
                                                                   " ".join("%.1e" % v for v in e)))
                assert max(e) < TOL, (n, rule, e)
        finally:
            ctx.close()


def test_ff_kernels_on_the_kirkwood_sphere_rows():
    """The 80k-node sphere: 2,048 oracle rows for both float-float kernels, and
    the two kernels against each other on every row."""
    R, h = 20.0, 0.5
    ctx = ibim.Context.sphere(R, h=h, band_eps=2 * h)
    try:
        g = oracle.sphere_nodes(R, h=h, eps=2 * h)
        perm = _match(ctx.nodes()["ijk"], g["ijk"])
        N = ctx.N
        P = ibim.Phys(2.0, 80.0, 0.1257, h, 0)
        Po = oracle.Phys(2.0, 80.0, 0.1257, h, 0)
        p = inputs.random_vector(2 * N, seed=64)
        rows = inputs.random_rows(N, 2048, seed=65)
        y1o, y2o = oracle.matvec_rows(g["xs"], g["nrm"], g["w"], Po, p, perm[rows])
        outs = []
        for symmetric in (1, 0):
            ctx.set_ff_kernel(symmetric)
            y = ctx.matvec_host(P, np.concatenate([p[:N][perm], p[N:][perm]]), precision=ibim.IBIM_FF)
            e = _worst_blocks(np.concatenate([y[:N][rows], y[N:][rows]]), np.concatenate([y1o, y2o]), 2048)
            print("ff (symmetric %d) kirkwood rows: %s" % (symmetric, " ".join("%.1e" % v for v in e)))
            assert max(e) < TOL, (symmetric, e)
            outs.append(y)
        assert max(_worst_blocks(outs[0], outs[1], N)) < TOL
    finally:
        ctx.close()


@pytest.mark.parametrize("kappa,tau_k,rule,eps_in", [(0.2, 1.0, 1, 2.0), (0.0, 0.5, 0, 1.0), (0.1257, 1.0, 0, 4.0)])
def test_ff_born_sphere_every_row(kappa, tau_k, rule, eps_in):
    R, h = 2.0, 0.25
    ctx = ibim.Context.sphere(R, h=h, band_eps=3 * h)
    try:
        g = oracle.sphere_nodes(R, h=h, eps=3 * h)
        perm = _match(ctx.nodes()["ijk"], g["ijk"])
        N = ctx.N
        P = ibim.Phys(eps_in, 80.0, kappa, tau_k * h, rule)
        Po = oracle.Phys(eps_in, 80.0, kappa, tau_k * h, rule)
        p = inputs.random_vector(2 * N, seed=61)
        yo = oracle.matvec(g["xs"], g["nrm"], g["w"], Po, p)
        y = ctx.matvec_host(P, np.concatenate([p[:N][perm], p[N:][perm]]), precision=ibim.IBIM_FF)
        e = _worst_blocks(y, np.concatenate([yo[:N][perm], yo[N:][perm]]), N)
        print("ff born kappa %g tau %gh rule %d: %s" % (kappa, tau_k, rule, " ".join("%.1e" % v for v in e)))
        assert max(e) < TOL, e
    finally:
        ctx.close()


def test_ff_sphere_far_from_the_origin_and_a_large_sphere():
    """A sphere centred 400 A from the origin (coordinates are taken relative
    to the centroid), and a 40 A sphere (about 320k nodes, the coarsest grid
    of the hi parts here): sampled rows against the oracle."""
    for R, h, centre, nrows in ((6.0, 0.25, (400.0, -250.0, 125.0), 0), (40.0, 0.5, (0.0, 0.0, 0.0), 512)):
        ctx = ibim.Context.sphere(R, centre=centre, h=h, band_eps=2 * h)
        try:
            g = oracle.sphere_nodes(R, centre=centre, h=h, eps=2 * h)
            perm = _match(ctx.nodes()["ijk"], g["ijk"])
            N = ctx.N
            P = ibim.Phys(2.0, 80.0, 0.1257, h, 0)
            Po = oracle.Phys(2.0, 80.0, 0.1257, h, 0)
            p = inputs.random_vector(2 * N, seed=62)
            y = ctx.matvec_host(P, np.concatenate([p[:N][perm], p[N:][perm]]), precision=ibim.IBIM_FF)
            if nrows:
                rows = inputs.random_rows(N, nrows, seed=63)  # library rows
                y1o, y2o = oracle.matvec_rows(g["xs"], g["nrm"], g["w"], Po, p, perm[rows])
                e = _worst_blocks(np.concatenate([y[:N][rows], y[N:][rows]]), np.concatenate([y1o, y2o]), nrows)
            else:
                yo = oracle.matvec(g["xs"], g["nrm"], g["w"], Po, p)
                e = _worst_blocks(y, np.concatenate([yo[:N][perm], yo[N:][perm]]), N)
            print("ff sphere R=%g centre %s N=%d: %s" % (R, centre, N, " ".join("%.1e" % v for v in e)))
            assert max(e) < TOL, (R, e)
        finally:
            ctx.close()


def test_certified_solve_reports_the_oracle_residual():
    """Born sphere, FP32 GMRES to 1e-6: with certify = 1 (float-float check)
    and certify = 2 (plain FP64 check) the reported residual is the oracle's
    residual of the returned vector, and the two certified solutions agree."""
    R, h = 2.0, 0.25
    ctx = ibim.Context.sphere(R, h=h, band_eps=3 * h)
    try:
        g = oracle.sphere_nodes(R, h=h, eps=3 * h)
        perm = _match(ctx.nodes()["ijk"], g["ijk"])
        N = ctx.N
        z, q = np.array([[0.2, -0.1, 0.3]]), np.array([1.0])
        ctx.set_charges(z, q)
        P = ibim.Phys(1.0, 80.0, 0.1257, h, 0)
        Po = oracle.Phys(1.0, 80.0, 0.1257, h, 0)
        b = oracle.rhs(g["xs"], g["nrm"], z, q, 1.0)
        sols = []
        for certify in (1, 2):
            d = torch.empty(2 * N, dtype=torch.float64, device="cuda")
            info = ctx.solve(P, d, precision=ibim.IBIM_F32C, tol=1e-6, restart=64, maxit=300, certify=certify)
            x = d.cpu().numpy()
            xo = np.empty_like(x)
            xo[:N][perm] = x[:N]
            xo[N:][perm] = x[N:]
            r = b - oracle.matvec(g["xs"], g["nrm"], g["w"], Po, xo)
            res = np.linalg.norm(r) / np.linalg.norm(b)
            print("certify %d: reported %.6e, oracle %.6e, FP64-accurate applications %d"
                  % (certify, info["relres"], res, info["matvecs_f64"]))
            assert info["converged"] and res < 1e-6
            assert abs(info["relres"] - res) <= 1e-9, (certify, info["relres"], res)
            assert 1 <= info["matvecs_f64"] <= 2
            sols.append(x)
        assert np.max(np.abs(sols[0] - sols[1])) <= 1e-6 * np.max(np.abs(sols[1]))
    finally:
        ctx.close()


@pytest.mark.parametrize("tol", [1e-8, 1e-10])
def test_certified_solve_below_the_fp32_accuracy(tol):
    """Born sphere, FP32 GMRES certified to tolerances at and below the FP32
    operator's own accuracy (about 1e-8 of |A p|): the refinement on the
    correction equation reaches them with the one-directional kernel and with
    every symmetric variant (whose applications also vary by about 1e-8), and
    the reported residual is the oracle's residual of the returned vector."""
    R, h = 2.0, 0.25
    ctx = ibim.Context.sphere(R, h=h, band_eps=3 * h)
    try:
        g = oracle.sphere_nodes(R, h=h, eps=3 * h)
        perm = _match(ctx.nodes()["ijk"], g["ijk"])
        N = ctx.N
        z, q = np.array([[0.2, -0.1, 0.3]]), np.array([1.0])
        ctx.set_charges(z, q)
        P = ibim.Phys(1.0, 80.0, 0.1257, h, 0)
        Po = oracle.Phys(1.0, 80.0, 0.1257, h, 0)
        b = oracle.rhs(g["xs"], g["nrm"], z, q, 1.0)
        d = torch.empty(2 * N, dtype=torch.float64, device="cuda")
        sym = [v for v, vi in enumerate(ibim.ibim_f32_variants()) if vi[3]]
        for v in [0] + sym:
            ctx.set_f32_variant(v, 0)
            info = ctx.solve(P, d, precision=ibim.IBIM_F32C, tol=tol, restart=64, maxit=400, certify=1)
            x = d.cpu().numpy()
            xo = np.empty_like(x)
            xo[:N][perm] = x[:N]
            xo[N:][perm] = x[N:]
            r = b - oracle.matvec(g["xs"], g["nrm"], g["w"], Po, xo)
            res = np.linalg.norm(r) / np.linalg.norm(b)
            print("tol %g variant %d: iterations %d, cycles %d, FP64-accurate applications %d, reported %.6e, "
                  "oracle %.6e" % (tol, v, info["iters"], info["cycles"], info["matvecs_f64"], info["relres"], res))
            assert info["converged"] and res < tol
            assert abs(info["relres"] - res) <= 1e-11
            assert info["iters"] <= 150 and info["matvecs_f64"] <= 6
    finally:
        ctx.close()
