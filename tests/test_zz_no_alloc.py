"""fe_sparsity_build_noalloc: the sparsity build for callers that must not allocate device memory.

Such callers (code whose device memory is a budget owned by another runtime, or code that cannot
afford cudaMalloc's latency and device-wide synchronisation) pass every buffer in; the kernels'
scratch is a fixed static device array.  This checks, through the C ABI, that two calls in a row
(different meshes, so the shared scratch is reused) give exactly the pattern and lookup table of
fe_sparsity_build, that calls after the first allocate nothing, and that the size query, the
size limits and the buffer-extent checks behave as documented.  The file
is named to be collected last; it also runs alone in a fresh process.
"""
import numpy as np
import pytest

from tests import problems as PB

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_01809_gb300 import build
    build.build()
    from paper_1501_01809_gb300 import fe
    return torch, fe


def _reference(pr):
    """Pattern and lookup table from the allocating entry point, on the same maps."""
    g = PB.GpuProblem(pr)
    nr, nc, nnz, rp, ci = g.fe.sparsity_csr(g.sparsity())
    nd = pr.cmap.shape[1]
    lut = g.fe.sparsity_lut(g.sparsity(), pr.mesh.ncell, nd, nd)
    return rp.cpu().numpy(), ci.cpu().numpy(), lut.cpu().numpy()


def _noalloc(torch, fe, pr):
    dev = torch.device("cuda", 0)
    m = torch.from_numpy(np.ascontiguousarray(pr.cmap)).to(dev)
    nd = pr.cmap.shape[1]
    rowptr = torch.full((pr.nnodes + 1,), -1, dtype=torch.int64, device=dev)
    lut = torch.full((pr.mesh.ncell * nd * nd,), 255, dtype=torch.uint8, device=dev)
    nnz = fe.sparsity_build_noalloc(m, m, pr.nnodes, pr.nnodes, rowptr, None, lut)  # size query
    colidx = torch.full((nnz,), -1, dtype=torch.int32, device=dev)
    nnz2 = fe.sparsity_build_noalloc(m, m, pr.nnodes, pr.nnodes, rowptr, colidx, lut)
    torch.cuda.synchronize()
    assert nnz2 == nnz
    return rowptr.cpu().numpy(), colidx.cpu().numpy(), lut.cpu().numpy()


def test_two_calls_match_the_allocating_build(env):
    torch, fe = env
    for dim, p, n, jit in [(3, 2, 6, 0.2), (2, 2, 13, 0.2)]:
        pr = PB.make(dim, p, n, jit, seed=3)
        want = _reference(pr)
        got = _noalloc(torch, fe, pr)
        for a, b in zip(got, want):
            np.testing.assert_array_equal(a, b)


def test_unaligned_map_and_table(env):
    """A map 4 bytes past an 8-byte boundary and a lookup table at an odd address (views into larger
    tensors): the row pass takes its one-at-a-time loads and byte stores; the result is the same."""
    torch, fe = env
    pr = PB.make(3, 2, 5, 0.2, seed=5)
    want = _reference(pr)
    dev = torch.device("cuda", 0)
    nd = pr.cmap.shape[1]
    flat = torch.empty(pr.cmap.size + 1, dtype=torch.int32, device=dev)
    m = flat[1:].view(pr.cmap.shape)
    m.copy_(torch.from_numpy(np.ascontiguousarray(pr.cmap)))
    lbig = torch.full((pr.mesh.ncell * nd * nd + 1,), 255, dtype=torch.uint8, device=dev)
    lut = lbig[1:]
    assert m.data_ptr() % 8 == 4 and lut.data_ptr() % 2 == 1
    rowptr = torch.empty(pr.nnodes + 1, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    nnz = fe.sparsity_build_noalloc(m, m, pr.nnodes, pr.nnodes, rowptr, None, lut)
    colidx = torch.empty(nnz, dtype=torch.int32, device=dev)
    fe.sparsity_build_noalloc(m, m, pr.nnodes, pr.nnodes, rowptr, colidx, lut)
    torch.cuda.synchronize()
    for a, b in zip((rowptr.cpu().numpy(), colidx.cpu().numpy(), lut.cpu().numpy()), want):
        np.testing.assert_array_equal(a, b)


def test_second_call_allocates_nothing(env):
    """After the first call (module loaded, scratch address looked up), a further build changes
    neither torch's allocator statistics nor the device's free memory."""
    torch, fe = env
    pr = PB.make(3, 2, 5, 0.2, seed=4)
    dev = torch.device("cuda", 0)
    m = torch.from_numpy(np.ascontiguousarray(pr.cmap)).to(dev)
    nd = pr.cmap.shape[1]
    rowptr = torch.empty(pr.nnodes + 1, dtype=torch.int64, device=dev)
    lut = torch.empty(pr.mesh.ncell * nd * nd, dtype=torch.uint8, device=dev)
    nnz = fe.sparsity_build_noalloc(m, m, pr.nnodes, pr.nnodes, rowptr, None, lut)
    colidx = torch.empty(nnz, dtype=torch.int32, device=dev)
    fe.sparsity_build_noalloc(m, m, pr.nnodes, pr.nnodes, rowptr, colidx, lut)
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(dev), torch.cuda.memory_reserved(dev), torch.cuda.mem_get_info(dev)[0])
    for _ in range(2):
        assert fe.sparsity_build_noalloc(m, m, pr.nnodes, pr.nnodes, rowptr, colidx, lut) == nnz
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(dev), torch.cuda.memory_reserved(dev), torch.cuda.mem_get_info(dev)[0])
    assert after == before, (before, after)


def test_small_colidx_and_limits_are_rejected(env):
    torch, fe = env
    pr = PB.make(2, 1, 8, 0.0)
    dev = torch.device("cuda", 0)
    m = torch.from_numpy(pr.cmap).to(dev)
    rowptr = torch.empty(pr.nnodes + 1, dtype=torch.int64, device=dev)
    lut = torch.empty(pr.mesh.ncell * 9, dtype=torch.uint8, device=dev)
    small = torch.empty(10, dtype=torch.int32, device=dev)
    with pytest.raises(fe.FeError) as ei:
        fe.sparsity_build_noalloc(m, m, pr.nnodes, pr.nnodes, rowptr, small, lut)
    assert ei.value.code == fe.FE_EINVAL and "colidx holds" in str(ei.value)
    big_rows = (1 << 18) + 1
    rp_big = torch.empty(big_rows + 1, dtype=torch.int64, device=dev)
    with pytest.raises(fe.FeError) as ei:
        fe.sparsity_build_noalloc(m, m, big_rows, big_rows, rp_big, None, lut)
    assert ei.value.code == fe.FE_EUNSUPPORTED and "static scratch" in str(ei.value)
    # buffers too small for the stated sizes are refused before any device work
    with pytest.raises(ValueError, match="rowptr holds"):
        fe.sparsity_build_noalloc(m, m, pr.nnodes + 5, pr.nnodes + 5, rowptr, None, lut)
    with pytest.raises(ValueError, match="lut holds"):
        fe.sparsity_build_noalloc(m, m, pr.nnodes, pr.nnodes, rowptr, None, lut[:-1])
    with pytest.raises(ValueError, match="equal ncell"):
        fe.sparsity_build_noalloc(m, m[:-1], pr.nnodes, pr.nnodes, rowptr, None, lut)
