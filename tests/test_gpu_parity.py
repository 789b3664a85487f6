"""GPU parity: the sm_103a library (through its C ABI) against the FP64 oracle.

Each side builds its own geometry from the same parameters; nodes are matched
through their integer grid coordinates.  Tolerances (relative 2-norm of the
difference over each output block):
  FP64 operator 1e-10, FP32 compensated operator 1e-5, energies 1e-4 (FP32).
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

F64, F32 = ibim.IBIM_F64, ibim.IBIM_F32C
BORN = dict(R=2.0, h=0.25, k=3)
KIRK = dict(R=20.0, h=0.5, k=2)


def _phys(eps_in=1.0, eps_out=80.0, kappa=0.1257, tau=0.25, rule=0):
    return ibim.Phys(eps_in, eps_out, kappa, tau, rule), oracle.Phys(eps_in, eps_out, kappa, tau, rule)


def _match(gpu_ijk, orc_ijk):
    """perm with gpu node j == oracle node perm[j]."""
    lo = np.minimum(gpu_ijk.min(0), orc_ijk.min(0)).astype(np.int64)
    span = (np.maximum(gpu_ijk.max(0), orc_ijk.max(0)) - lo + 1).astype(np.int64)

    def key(a):
        a = a.astype(np.int64) - lo
        return (a[:, 2] * span[1] + a[:, 1]) * span[0] + a[:, 0]

    ko, kg = key(orc_ijk), key(gpu_ijk)
    order = np.argsort(ko)
    pos = np.searchsorted(ko[order], kg)
    perm = order[pos]
    assert np.array_equal(ko[perm], kg)
    return perm


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.fixture(scope="module")
def born():
    ctx = ibim.Context.sphere(BORN["R"], h=BORN["h"], band_eps=BORN["k"] * BORN["h"])
    g = oracle.sphere_nodes(BORN["R"], h=BORN["h"], eps=BORN["k"] * BORN["h"])
    gn = ctx.nodes()
    perm = _match(gn["ijk"], g["ijk"])
    yield ctx, g, gn, perm
    ctx.close()


def test_sphere_geometry_matches_oracle(born):
    ctx, g, gn, perm = born
    assert ctx.N == g["w"].size
    assert np.unique(perm).size == perm.size
    np.testing.assert_allclose(gn["xs"], g["xs"][perm], rtol=0, atol=1e-13)
    np.testing.assert_allclose(gn["nrm"], g["nrm"][perm], rtol=0, atol=1e-14)
    np.testing.assert_allclose(gn["w"], g["w"][perm], rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(gn["d"], g["d"][perm], rtol=0, atol=1e-13)
    assert ctx.area() == pytest.approx(oracle.area(g["w"]), rel=1e-13)


def _both_blocks(y, yo, N):
    return _rel(y[:N], yo[:N]), _rel(y[N:], yo[N:]), _rel(y, yo)


@pytest.mark.parametrize("kappa,tau_k,rule,eps_in", [(0.1257, 1.0, 0, 1.0), (0.1257, 0.5, 0, 1.0),
                                                     (0.0, 1.0, 0, 1.0), (0.2, 1.0, 1, 2.0)])
def test_operator_all_rows_born(born, kappa, tau_k, rule, eps_in):
    ctx, g, gn, perm = born
    N = ctx.N
    P, Po = _phys(eps_in, 80.0, kappa, tau_k * BORN["h"], rule)
    p_orc = inputs.random_vector(2 * N, seed=5)
    y_orc = oracle.matvec(g["xs"], g["nrm"], g["w"], Po, p_orc)
    p_gpu = np.concatenate([p_orc[:N][perm], p_orc[N:][perm]])
    y_ref = np.concatenate([y_orc[:N][perm], y_orc[N:][perm]])
    din = _dev(p_gpu)
    dout = torch.empty_like(din)
    ctx.matvec(P, din, dout, precision=F64)
    torch.cuda.synchronize()
    r64 = _both_blocks(dout.cpu().numpy(), y_ref, N)
    assert max(r64) < 1e-10, r64
    ctx.matvec(P, din, dout, precision=F32)
    torch.cuda.synchronize()
    r32 = _both_blocks(dout.cpu().numpy(), y_ref, N)
    assert max(r32) < 1e-5, r32


def test_operator_host_entry_point(born):
    ctx, g, gn, perm = born
    N = ctx.N
    P, Po = _phys()
    p = inputs.random_vector(2 * N, seed=9)
    y_dev = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    ctx.matvec(P, _dev(p), y_dev, precision=F64)
    y_host = ctx.matvec_host(P, p, precision=F64)
    np.testing.assert_array_equal(y_host, y_dev.cpu().numpy())


def test_rhs_energy_area(born):
    ctx, g, gn, perm = born
    N = ctx.N
    z, q = inputs.kirkwood_charges(n=5, ball_radius=1.5, seed=3)
    ctx.set_charges(z, q)
    dg = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    ctx.rhs(1.0, dg)
    torch.cuda.synchronize()
    go = oracle.rhs(g["xs"], g["nrm"], z, q, 1.0)
    gref = np.concatenate([go[:N][perm], go[N:][perm]])
    assert max(_both_blocks(dg.cpu().numpy(), gref, N)) < 1e-12
    P, Po = _phys()
    p_orc = inputs.random_vector(2 * N, seed=6, scale=1e-2)
    p_gpu = np.concatenate([p_orc[:N][perm], p_orc[N:][perm]])
    psi = torch.empty(len(q), dtype=torch.float64, device="cuda")
    G = ctx.energy(P, _dev(p_gpu), psi)
    psi_o = oracle.psi_rxn(g["xs"], g["nrm"], g["w"], z, Po, p_orc)
    np.testing.assert_allclose(psi.cpu().numpy(), psi_o, rtol=1e-11, atol=1e-14 * np.abs(psi_o).max())
    assert G == pytest.approx(oracle.gpol(q, psi_o), rel=1e-11)


def test_born_solve_fp64_matches_oracle_and_closed_form(born):
    ctx, g, gn, perm = born
    N = ctx.N
    z, q = np.zeros((1, 3)), np.ones(1)
    ctx.set_charges(z, q)
    P, Po = _phys(tau=BORN["h"])
    dp = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    info = ctx.solve(P, dp, precision=F64, tol=1e-10, restart=64, maxit=300)
    assert info["converged"] and info["relres"] < 1e-10
    b = oracle.rhs(g["xs"], g["nrm"], z, q, 1.0)
    x, it, rr, ok = oracle.gmres(g["xs"], g["nrm"], g["w"], Po, b, tol=1e-12)
    xg = dp.cpu().numpy()
    xref = np.concatenate([x[:N][perm], x[N:][perm]])
    assert _rel(xg, xref) < 1e-8
    Go = oracle.gpol(q, oracle.psi_rxn(g["xs"], g["nrm"], g["w"], z, Po, x))
    assert info["gpol"] == pytest.approx(Go, rel=1e-9)
    Gs = cf.born_energy(BORN["R"])
    assert abs(info["gpol"] - Gs) / abs(Gs) < 0.05
    assert info["gpol_kcal"] == pytest.approx(info["gpol"] * oracle.KCAL_PER_E2_A, rel=1e-12)


@pytest.mark.parametrize("start", [0, 1])
def test_born_solve_fp32_certified(born, start):
    ctx, g, gn, perm = born
    N = ctx.N
    ctx.set_charges(np.zeros((1, 3)), np.ones(1))
    P, Po = _phys(tau=BORN["h"])
    d64 = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    i64 = ctx.solve(P, d64, precision=F64, tol=1e-8, restart=64, maxit=300, start=start)
    d32 = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    i32 = ctx.solve(P, d32, precision=F32, tol=1e-6, restart=64, maxit=300, start=start, certify=1)
    assert i32["converged"] and i32["relres"] < 1e-6
    # restarts use the FP32 operator; the FP64 operator only checks convergence
    assert 1 <= i32["matvecs_f64"] <= 2, i32
    assert abs(i32["gpol"] - i64["gpol"]) / abs(i64["gpol"]) < 1e-4
    # the certified residual is the oracle's residual of the returned vector
    x = d32.cpu().numpy()
    inv = np.empty_like(perm)
    inv[perm] = np.arange(N)
    xo = np.concatenate([x[:N][inv], x[N:][inv]])
    b = oracle.rhs(g["xs"], g["nrm"], np.zeros((1, 3)), np.ones(1), 1.0)
    r = b - oracle.matvec(g["xs"], g["nrm"], g["w"], Po, xo)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-6


def test_from_nodes_tiny_and_ragged():
    """Caller-given node clouds: N = 1, 2, 3, 257 (one target tile plus one), 1000."""
    for n in (1, 2, 3, 257, 1000):
        xs, nr, w = inputs.sphere_cloud(n, radius=3.0, seed=n)
        ctx = ibim.Context.from_nodes(xs, nr, w, h=0.25)
        P, Po = _phys(tau=0.3)
        p = inputs.random_vector(2 * n, seed=n + 1)
        yo = oracle.matvec(xs, nr, w, Po, p)
        y = ctx.matvec_host(P, p, precision=F64)
        assert _rel(y, yo) < 1e-10, n
        y32 = ctx.matvec_host(P, p, precision=F32)
        assert _rel(y32, yo) < 1e-5, n
        ctx.close()


def test_kirkwood_full_size_sampled_rows():
    """The 80k-node Kirkwood sphere, in the launch configuration the benchmark
    uses: 2048 seeded rows of both operators against the oracle's rows."""
    ctx = ibim.Context.sphere(KIRK["R"], h=KIRK["h"], band_eps=KIRK["k"] * KIRK["h"])
    g = oracle.sphere_nodes(KIRK["R"], h=KIRK["h"], eps=KIRK["k"] * KIRK["h"])
    gn = ctx.nodes()
    perm = _match(gn["ijk"], g["ijk"])
    N = ctx.N
    assert N > 70000
    P, Po = _phys(2.0, 80.0, 0.1257, KIRK["h"])
    p_orc = inputs.random_vector(2 * N, seed=21)
    p_gpu = np.concatenate([p_orc[:N][perm], p_orc[N:][perm]])
    rows_gpu = inputs.random_rows(N, 2048, seed=22)
    y1o, y2o = oracle.matvec_rows(g["xs"], g["nrm"], g["w"], Po, p_orc, perm[rows_gpu])
    din = _dev(p_gpu)
    dout = torch.empty_like(din)
    for prec, tol in ((F64, 1e-10), (F32, 1e-5)):
        ctx.matvec(P, din, dout, precision=prec)
        y = dout.cpu().numpy()
        e1 = _rel(y[:N][rows_gpu], y1o)
        e2 = _rel(y[N:][rows_gpu], y2o)
        assert max(e1, e2) < tol, (prec, e1, e2)
    ctx.close()


def test_kirkwood_energy_fp32_vs_fp64_and_series():
    ctx = ibim.Context.sphere(KIRK["R"], h=KIRK["h"], band_eps=KIRK["k"] * KIRK["h"])
    z, q = inputs.kirkwood_charges()
    ctx.set_charges(z, q)
    N = ctx.N
    P, _ = _phys(2.0, 80.0, 0.1257, KIRK["h"])
    d32 = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    i32 = ctx.solve(P, d32, precision=F32, tol=1e-6, restart=64, maxit=400)
    assert i32["converged"]
    G64 = ctx.energy(P, d32, precision=F64)
    assert G64 == pytest.approx(i32["gpol"], rel=1e-12)
    Gs = cf.kirkwood_energy(KIRK["R"], z, q, 2.0, 80.0, 0.1257)
    assert abs(i32["gpol"] - Gs) / abs(Gs) < 0.02
    ctx.close()


def test_solve_reports_not_converged():
    ctx = ibim.Context.sphere(BORN["R"], h=BORN["h"], band_eps=BORN["k"] * BORN["h"])
    ctx.set_charges(np.zeros((1, 3)), np.ones(1))
    P, _ = _phys()
    dp = torch.empty(2 * ctx.N, dtype=torch.float64, device="cuda")
    with pytest.raises(ibim.IbimError) as e:
        ctx.solve(P, dp, precision=F64, tol=1e-14, restart=2, maxit=2)
    assert e.value.status == 5
    info = ctx.solve(P, dp, precision=F64, tol=1e-14, restart=2, maxit=2, allow_not_converged=True)
    assert info["iters"] == 2 and not info["converged"]
    ctx.close()


def test_kirkwood_fp32_all_rows_against_fp64():
    """All 2N rows of the FP32 operator against the FP64 operator (itself
    checked against the oracle above) on the 80k-node sphere, whose lattice
    symmetry puts many pairs within rounding of the tube boundary: the FP32
    path must decide those ties as FP64 does (no row may stand out)."""
    ctx = ibim.Context.sphere(KIRK["R"], h=KIRK["h"], band_eps=KIRK["k"] * KIRK["h"])
    N = ctx.N
    for kappa in (0.1257, 0.0):
        P, _ = _phys(2.0, 80.0, kappa, KIRK["h"])
        p = _dev(inputs.random_vector(2 * N, seed=1))
        y64 = torch.empty_like(p)
        y32 = torch.empty_like(p)
        ctx.matvec(P, p, y64, precision=F64)
        ctx.matvec(P, p, y32, precision=F32)
        a, b = y64.cpu().numpy(), y32.cpu().numpy()
        r = _both_blocks(b, a, N)
        worst = np.max(np.abs(b - a)) / np.max(np.abs(a))
        print("kirkwood all rows kappa=%g: rel %.2e %.2e %.2e, worst row %.2e" % (kappa, *r, worst))
        assert max(r) < 1e-6, r
        assert worst < 1e-5, worst
    ctx.close()


def test_every_fp32_variant_matches_fp64():
    """Each compiled FP32 pair-kernel variant (targets per thread, register
    budget, CTA size) and a reduced persistent grid give the same operator as
    the FP64 path on a sphere with several target and source tiles."""
    ctx = ibim.Context.sphere(6.0, h=0.25, band_eps=0.5)
    N = ctx.N
    P, _ = _phys(2.0, 80.0, 0.1257, 0.25)
    p = _dev(inputs.random_vector(2 * N, seed=2))
    y64 = torch.empty_like(p)
    ctx.matvec(P, p, y64, precision=F64)
    a = y64.cpu().numpy()
    y32 = torch.empty_like(p)
    for v, (tpt, minb, nthr, sym) in enumerate(ibim.ibim_f32_variants()):
        for bps in (0, 1):
            ctx.set_f32_variant(v, bps)
            ctx.matvec(P, p, y32, precision=F32)
            torch.cuda.synchronize()
            r = _both_blocks(y32.cpu().numpy(), a, N)
            assert max(r) < 1e-6, (v, tpt, minb, nthr, sym, bps, r)
    ctx.close()


def _block_radii(xs):
    nb = len(xs) // 32
    b = xs[:nb * 32].reshape(nb, 32, 3)
    return np.sqrt(((b - b.mean(axis=1, keepdims=True)) ** 2).sum(axis=2).max(axis=1))


def test_built_geometries_have_compact_32_node_blocks():
    """Built geometries are reordered into compact aligned 32-node blocks (the
    pair kernels' chunks): on the 80k sphere no block is wider than a few grid
    cells and on a level-set globule nearly none is, while the node set is
    unchanged."""
    ctx = ibim.Context.sphere(KIRK["R"], h=KIRK["h"], band_eps=KIRK["k"] * KIRK["h"])
    n = ctx.nodes()
    r = _block_radii(n["xs"])
    assert r.max() < 2.5, r.max()
    ijk = n["ijk"].astype(np.int64)
    assert len({tuple(v) for v in ijk}) == ctx.N  # a permutation of distinct grid nodes
    ctx.close()
    z, rad, q = inputs.globule_atoms(300, seed=11)
    ctx = ibim.Context.molecule(z, rad, q, probe=1.4, h=0.5)
    r = _block_radii(ctx.nodes()["xs"])
    frac = float(np.mean(r > 3.0))
    print("block radius: globule max %.2f median %.2f, %.1f %% above 3 A" % (r.max(), np.median(r), 100 * frac))
    # a few blocks hold a small detached piece of surface together with nodes
    # of its neighbourhood (leaves are cut by count); nearly all are compact
    assert np.median(r) < 1.5 and frac < 0.03, (np.median(r), frac)
    ctx.close()


def test_symmetric_kernel_all_rows_against_fp64():
    """The symmetric FP32 kernel (each unordered pair evaluated once for both
    directions) on every row of the 80k sphere and of a level-set globule,
    against the FP64 operator: same bar as the one-directional kernel."""
    sym = [v for v, info in enumerate(ibim.ibim_f32_variants()) if info[3]]
    assert sym
    z, r, q = inputs.globule_atoms(300, seed=9)
    for ctx in (ibim.Context.sphere(KIRK["R"], h=KIRK["h"], band_eps=KIRK["k"] * KIRK["h"]),
                ibim.Context.molecule(z, r, q, probe=1.4, h=0.5)):
        N = ctx.N
        for kappa in (0.1257, 0.0):
            P, _ = _phys(2.0, 80.0, kappa, 0.5)
            p = _dev(inputs.random_vector(2 * N, seed=1))
            y64 = torch.empty_like(p)
            ctx.matvec(P, p, y64, precision=F64)
            a = y64.cpu().numpy()
            for v in sym:
                for bps in (0, 1):
                    ctx.set_f32_variant(v, bps)
                    y32 = torch.empty_like(p)
                    ctx.matvec(P, p, y32, precision=F32)
                    b = y32.cpu().numpy()
                    rr = _both_blocks(b, a, N)
                    worst = np.max(np.abs(b - a)) / np.max(np.abs(a))
                    print("symmetric v%d bps %d N %d kappa %g: rel %.2e %.2e %.2e worst %.2e" % (v, bps, N, kappa,
                                                                                            *rr, worst))
                    assert max(rr) < 1e-6 and worst < 1e-5, (v, bps, N, kappa, rr, worst)
        ctx.close()


def test_symmetric_kernel_small_ragged_and_repeated():
    """Symmetric variants on node counts with fewer steps than CTAs, a single
    tile and a ragged last tile, against FP64; repeated calls agree to the
    FP32 rounding of one tile's reverse partial (the atomic order of the
    reverse sums is the only run-to-run change; a segment counter that was not
    reset would drop a tenth of the steps)."""
    sym = [v for v, info in enumerate(ibim.ibim_f32_variants()) if info[3]]
    P, _ = _phys(2.0, 80.0, 0.1257, 0.3)
    for n in (40, 700, 5000):
        xs, nr, w = inputs.sphere_cloud(n, radius=4.0 + n / 2000.0, seed=n)
        ctx = ibim.Context.from_nodes(xs, nr, w, h=0.3)
        N = ctx.N
        p = _dev(inputs.random_vector(2 * N, seed=5))
        y64 = torch.empty_like(p)
        ctx.matvec(P, p, y64, precision=F64)
        a = y64.cpu().numpy()
        for v in sym:
            ctx.set_f32_variant(v, 0)
            outs = []
            for _ in range(3):
                y32 = torch.empty_like(p)
                ctx.matvec(P, p, y32, precision=F32)
                outs.append(y32.cpu().numpy())
            r = _both_blocks(outs[0], a, N)
            assert max(r) < 1e-6, (n, v, r)
            for o in outs[1:]:
                assert np.max(np.abs(o - outs[0])) <= 1e-8 * np.max(np.abs(outs[0])), (n, v)
        ctx.close()
