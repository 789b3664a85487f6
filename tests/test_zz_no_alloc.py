"""The allocation-free operator entry point against the oracle and the
context-based entry point.

ibim_matvec_noalloc serves callers that cannot allocate device memory (for
example code running where cudaMalloc is not allowed, or under an allocator
owned by another runtime).  It takes its working memory from a fixed static
device array, so two back-to-back calls must each give the product of their
own inputs, matching ibim_matvec with IBIM_F32C to the FP32 tolerance of the
other tests.  The caller's nodes here are the oracle's own sphere nodes, so
the FP64 oracle's rows are the reference; at the 80k-node Kirkwood size
(inside the entry point's node limit) the nodes are passed in coordinate-
bisection order, the order a caller should use.  This file is collected last
on purpose.
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

TOL_F32 = 1e-5  # relative 2-norm per output block, and worst element / max |y| per block


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _worst(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _check_blocks(y, yo, N, what):
    for blk in (slice(0, N), slice(N, 2 * N)):
        r, w = _rel(y[blk], yo[blk]), _worst(y[blk], yo[blk])
        assert r < TOL_F32 and w < TOL_F32, (what, r, w)


def test_noalloc_matches_oracle_and_context_on_two_calls():
    import __graft_entry__
    __graft_entry__.build()
    R, h = 6.0, 0.25
    g = oracle.sphere_nodes(R, h=h, eps=2 * h)
    N = g["w"].size
    assert 256 < N <= ibim.IBIM_NOALLOC_MAX_NODES
    ctx = ibim.Context.from_nodes(g["xs"], g["nrm"], g["w"], h=h)
    try:
        dx, dn, dw = _dev(g["xs"]), _dev(g["nrm"]), _dev(g["w"])
        P = ibim.Phys(2.0, 80.0, 0.1257, h, 0)
        Po = oracle.Phys(2.0, 80.0, 0.1257, h, 0)
        stream = torch.cuda.current_stream().cuda_stream
        outs = []
        for call, seed in enumerate((31, 32)):
            p_h = inputs.random_vector(2 * N, seed=seed)
            p = _dev(p_h)
            y_ref = torch.empty_like(p)
            ctx.matvec(P, p, y_ref, precision=ibim.IBIM_F32C)
            y = torch.full_like(p, float("nan"))
            ibim.ibim_matvec_noalloc(N, dx, dn, dw, P, p, y, stream)
            a, b = y.cpu().numpy(), y_ref.cpu().numpy()
            assert np.all(np.isfinite(a)), call
            _check_blocks(a, b, N, ("context", call))
            _check_blocks(a, oracle.matvec(g["xs"], g["nrm"], g["w"], Po, p_h), N, ("oracle", call))
            outs.append(a)
        assert _rel(outs[0], outs[1]) > 1e-2  # the second call did not return the first call's result
    finally:
        ctx.close()


def test_noalloc_at_kirkwood_size_against_oracle_rows_and_fp64():
    """80,358 nodes (R = 20, h = 0.5, band 2h), the size the entry point's
    chunk frames are for: 2048 seeded rows against the oracle, every row
    against the FP64 and FP32 operators of a context on the same nodes."""
    R, h = 20.0, 0.5
    g = oracle.sphere_nodes(R, h=h, eps=2 * h)
    perm = inputs.bisection_order(g["xs"])
    xs, nrm, w = g["xs"][perm], g["nrm"][perm], g["w"][perm]
    N = w.size
    assert 70000 < N <= ibim.IBIM_NOALLOC_MAX_NODES
    P = ibim.Phys(2.0, 80.0, 0.1257, h, 0)
    Po = oracle.Phys(2.0, 80.0, 0.1257, h, 0)
    p_h = inputs.random_vector(2 * N, seed=33)
    p = _dev(p_h)
    y = torch.full_like(p, float("nan"))
    ibim.ibim_matvec_noalloc(N, _dev(xs), _dev(nrm), _dev(w), P, p, y)
    a = y.cpu().numpy()
    assert np.all(np.isfinite(a))
    rows = inputs.random_rows(N, 2048, seed=34)
    y1o, y2o = oracle.matvec_rows(xs, nrm, w, Po, p_h, rows)
    for got, ref in ((a[:N][rows], y1o), (a[N:][rows], y2o)):
        assert _rel(got, ref) < TOL_F32 and _worst(got, ref) < TOL_F32, (_rel(got, ref), _worst(got, ref))
    ctx = ibim.Context.from_nodes(xs, nrm, w, h=h)
    try:
        for prec in (ibim.IBIM_F64, ibim.IBIM_F32C):
            yc = torch.empty_like(p)
            ctx.matvec(P, p, yc, precision=prec)
            _check_blocks(a, yc.cpu().numpy(), N, prec)
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_limit_and_overlapping_vectors():
    P = ibim.Phys(1.0, 80.0, 0.1257, 0.25, 0)
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ibim.IbimError) as e:
        ibim.ibim_matvec_noalloc(ibim.IBIM_NOALLOC_MAX_NODES + 1, d, d, d, P, d, d[4:])
    assert e.value.status == 1
    assert "IBIM_NOALLOC_MAX_NODES" in str(e.value)
    # two nodes: partly overlapping 2N-vectors are rejected, adjacent ones accepted
    xs = _dev([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0]])
    nr = _dev([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    w = _dev([0.01, 0.02])
    buf = torch.ones(8, dtype=torch.float64, device="cuda")
    for d_in, d_out in ((buf[0:4], buf[3:7]), (buf[3:7], buf[0:4]), (buf[0:4], buf[1:5])):
        with pytest.raises(ibim.IbimError) as e:
            ibim.ibim_matvec_noalloc(2, xs, nr, w, P, d_in, d_out)
        assert e.value.status == 1 and "overlap" in str(e.value)
    ibim.ibim_matvec_noalloc(2, xs, nr, w, P, buf[0:4], buf[4:8])
    y = buf[4:8].cpu().numpy()
    yo = oracle.matvec(xs.cpu().numpy(), nr.cpu().numpy(), w.cpu().numpy(), oracle.Phys(1.0, 80.0, 0.1257, 0.25, 0),
                       np.ones(4))
    np.testing.assert_allclose(y, yo, rtol=1e-5, atol=0)
