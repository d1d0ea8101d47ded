"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads without a
GPU, and exports every function that include/ecc.h declares. No compute calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ecc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(ecc_[a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def so_path():
    from paper_1705_02045_gb300 import build
    return build.build_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ecc_create", "ecc_destroy", "ecc_compute", "ecc_stream_begin",
                     "ecc_stream_push_slab", "ecc_stream_finish", "ecc_submit", "ecc_poll",
                     "ecc_last_error", "ecc_result_free", "ecc_compute_batch"]:
        assert required in names


def test_library_exports_every_declared_symbol(so_path):
    lib = ctypes.CDLL(so_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_signatures_cover_the_header(so_path):
    from paper_1705_02045_gb300 import ecc
    assert set(declared_functions()) <= set(ecc._SIGNATURES)


def test_create_without_gpu_fails_cleanly(so_path):
    """With no visible GPU, ecc_create reports ECC_ERR_CUDA instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    from paper_1705_02045_gb300 import ecc
    with pytest.raises(ecc.EccError) as ei:
        ecc.ecc_create(device=0)
    assert ei.value.status == ecc.ECC_ERR_CUDA


def test_built_for_sm_103a_only():
    """The build passes exactly one -gencode, for sm_103a."""
    from paper_1705_02045_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
