"""The allocation-free operator entry point against the context-based one.

ibim_matvec_noalloc serves callers that cannot allocate device memory (for
example code running where cudaMalloc is not allowed, or under an allocator
owned by another runtime).  It takes its working memory from a fixed static
device array, so two back-to-back calls must each give the product of their
own inputs, matching ibim_matvec with IBIM_F32C to the FP32 tolerance of the
other tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1709_08070_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1709_08070_gb300 import ibim  # noqa: E402

TOL_F32 = 1e-5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_context_matvec_on_two_calls():
    import __graft_entry__
    __graft_entry__.build()
    R, h = 6.0, 0.25
    ctx = ibim.Context.sphere(R, h=h, band_eps=2 * h)
    try:
        N = ctx.N
        assert 256 < N <= ibim.IBIM_NOALLOC_MAX_NODES
        nodes = ctx.nodes()
        dx = torch.from_numpy(nodes["xs"]).cuda().contiguous()
        dn = torch.from_numpy(nodes["nrm"]).cuda().contiguous()
        dw = torch.from_numpy(nodes["w"]).cuda().contiguous()
        P = ibim.Phys(2.0, 80.0, 0.1257, h, 0)
        stream = torch.cuda.current_stream().cuda_stream
        outs = []
        for call, seed in enumerate((31, 32)):
            p = torch.from_numpy(inputs.random_vector(2 * N, seed=seed)).cuda()
            y_ref = torch.empty_like(p)
            ctx.matvec(P, p, y_ref, precision=ibim.IBIM_F32C)
            y = torch.full_like(p, float("nan"))
            ibim.ibim_matvec_noalloc(N, dx, dn, dw, P, p, y, stream)
            a, b = y.cpu().numpy(), y_ref.cpu().numpy()
            assert np.all(np.isfinite(a)), call
            assert _rel(a[:N], b[:N]) < TOL_F32, call
            assert _rel(a[N:], b[N:]) < TOL_F32, call
            outs.append(a)
        assert _rel(outs[0], outs[1]) > 1e-2  # the second call did not return the first call's result
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    P = ibim.Phys(1.0, 80.0, 0.1257, 0.25, 0)
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ibim.IbimError) as e:
        ibim.ibim_matvec_noalloc(ibim.IBIM_NOALLOC_MAX_NODES + 1, d, d, d, P, d, d[4:])
    assert e.value.status == 1
    assert "IBIM_NOALLOC_MAX_NODES" in str(e.value)
