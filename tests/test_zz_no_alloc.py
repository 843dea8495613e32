"""The allocation-free pose query (forward + backward in one call, saved state in a
file-scope device array), for callers that cannot allocate device memory.  Checked through
the C ABI against the allocating entry points, on two calls in a row.  Collected last, so a
run that stops at the first failure has run every other test first."""
import numpy as np
import pytest
import torch

from synthetic import bumpy_plane, random_poses

pytestmark = pytest.mark.gpu

C1 = dict(nx=100, ny=100, n_yaw=36, res=0.1, length=0.6, width=0.4)


@pytest.fixture(scope="module")
def seb():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2503_02412_gb300 as seb

    return seb


def reference(seb, p, te, tp, g, st):
    n = tp.shape[0]
    out = torch.empty(n, 5, device="cuda")
    fl = torch.empty(n, dtype=torch.uint8, device="cuda")
    sv = torch.empty(n, seb.abi.SEB_QUERY_SAVED, device="cuda")
    gp = torch.empty(n, 3, device="cuda")
    seb.abi.seb_query_poses(p, te.data_ptr(), 3, -2, tp.data_ptr(), n, out.data_ptr(), fl.data_ptr(), sv.data_ptr(), st)
    seb.abi.seb_query_poses_backward(p, te.data_ptr(), 3, -2, tp.data_ptr(), sv.data_ptr(), g.data_ptr(), gp.data_ptr(),
                                     n, st)
    return out, fl, gp


def noalloc(seb, p, te, tp, g, st):
    n = tp.shape[0]
    out = torch.empty(n, 5, device="cuda")
    fl = torch.empty(n, dtype=torch.uint8, device="cuda")
    gp = torch.empty(n, 3, device="cuda")
    seb.abi.seb_query_poses_grad_noalloc(p, te.data_ptr(), 3, -2, tp.data_ptr(), n, g.data_ptr(), out.data_ptr(),
                                         fl.data_ptr(), gp.data_ptr(), st)
    return out, fl, gp


def _compare_twice(seb, p, te, cases, origin=(3, -2)):
    st = torch.cuda.current_stream().cuda_stream
    for seed, n in cases:  # each call reuses the scratch the previous one left
        tp = torch.from_numpy(random_poses(seed, n, 100, 100, 0.1, 3, origin=origin)).cuda()
        g = torch.randn(n, 5, device="cuda", generator=torch.Generator("cuda").manual_seed(seed))
        ro, rf, rg = reference(seb, p, te, tp, g, st)
        no, nf, ng = noalloc(seb, p, te, tp, g, st)
        torch.cuda.synchronize()
        assert torch.equal(rf, nf)
        fin = torch.isfinite(ro)
        assert torch.equal(fin, torch.isfinite(no))
        assert torch.allclose(no[fin], ro[fin], rtol=1e-5, atol=1e-6)
        assert torch.allclose(ng, rg, rtol=1e-5, atol=1e-6)


def test_noalloc_matches_allocating_query_twice(seb):
    """Two calls in a row on the grouped kernels (fewer than 65,536 poses), then the largest
    batch the scratch takes (65,536 poses: the one-pose-per-thread kernels, every record of the
    array written and read) and a smaller batch after it."""
    p = seb.SebParams(**C1).c()
    te = torch.from_numpy(bumpy_plane(31)).cuda()
    _compare_twice(seb, p, te, ((1, 5000), (2, 777), (3, 65536), (4, 1000)))


def test_noalloc_ellipse_footprint(seb):
    """The paper's elliptical footprint: the lattice comes from the same tables as the
    allocating query's."""
    p = seb.SebParams(**dict(C1, shape="ellipse", length=0.8, width=0.5)).c()
    te = torch.from_numpy(bumpy_plane(33)).cuda()
    _compare_twice(seb, p, te, ((5, 3000), (6, 65536)))


def test_noalloc_rejects_batches_beyond_the_scratch(seb):
    p = seb.SebParams(**C1).c()
    te = torch.from_numpy(bumpy_plane(32)).cuda()
    n = 65537
    tp = torch.zeros(n, 3, device="cuda")
    g = torch.zeros(n, 5, device="cuda")
    with pytest.raises(seb.abi.SebError) as ei:
        noalloc(seb, p, te, tp, g, torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == seb.abi.SEB_ERR_INVALID_ARG
    assert "65536-pose scratch" in str(ei.value)
