"""libfe builds for sm_103a, loads without a GPU, and exports every entry point of include/fe.h."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fe_[a-z0-9_]+)\s*\(", src)) - {"fe_alloc_fn", "fe_free_fn"})


@pytest.fixture(scope="module")
def lib():
    from paper_1501_01809_gb300 import build
    build.build()
    from paper_1501_01809_gb300 import fe
    return fe.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["fe_ctx_create", "fe_set_create", "fe_map_create", "fe_dat_create", "fe_sparsity_build",
                 "fe_sparsity_csr", "fe_mat_create", "fe_kernel_create", "fe_assemble_mat", "fe_assemble_vec",
                 "fe_action", "fe_sync", "fe_last_error"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol(lib):
    from paper_1501_01809_gb300 import fe
    assert sorted(fe.SYMBOLS) == _declared()


def test_host_only_calls_without_gpu(lib):
    from paper_1501_01809_gb300 import fe
    assert fe.version().startswith("libfe")
    assert isinstance(lib.fe_last_error(), bytes)
    # a NULL handle is rejected with FE_EHANDLE, never a crash
    assert lib.fe_set_create(None, 4, None) == fe.FE_EHANDLE
    assert lib.fe_sync(None) == fe.FE_EHANDLE
    assert b"invalid" in lib.fe_last_error()


def test_generated_local_kernels_are_current():
    from paper_1501_01809_gb300 import build, codegen
    with open(build.GEN) as fh:
        assert fh.read() == codegen.generate(check=False)


def test_no_cpu_fallback(lib):
    """Without a CUDA device the product path fails loudly: the binding refuses to make a context,
    the C ABI reports a CUDA error for one, and buffers on the host are refused before any call."""
    import torch
    from paper_1501_01809_gb300 import fe
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        fe.ctx_create(0)
    import ctypes as C
    out = C.c_void_p()
    assert lib.fe_ctx_create(0, None, C.byref(out)) == fe.FE_ECUDA and not out.value
    host = torch.zeros((4, 3), dtype=torch.int32)
    with pytest.raises(TypeError, match="CUDA tensor"):
        fe.map_create(None, None, None, host)
    with pytest.raises(TypeError, match="CUDA tensor"):
        fe.sparsity_build_noalloc(host, host, 4, 4, torch.zeros(5, dtype=torch.int64), None,
                                  torch.zeros(36, dtype=torch.uint8))


def test_noalloc_sources_name_no_allocator():
    """fe_sparsity_build_noalloc and the sparsity launchers it calls (fe_sparsity.cu) name no
    device allocation or free routine: their scratch is the static array only."""
    csrc = os.path.join(ROOT, "paper_1501_01809_gb300", "csrc")
    pat = re.compile(r"\b(cudaMalloc\w*|cudaFree\w*|cuMemAlloc\w*|cuMemFree\w*|dev_alloc|dev_free|malloc|free)\s*\(")
    for name in ("fe_noalloc.cu", "fe_sparsity.cu"):
        src = re.sub(r"//[^\n]*|/\*.*?\*/", "", open(os.path.join(csrc, name)).read(), flags=re.S)
        assert not pat.findall(src), (name, pat.findall(src))
