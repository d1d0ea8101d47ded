"""The allocation-free entry point (ecc_compute_device_noalloc), for callers that
cannot allocate device memory. Its curves must equal the oracle's element by
element -- the curve is integer, so exactly -- in both cell conventions, and
equal those of the regular device entry point (ecc_compute_device), on two
calls in a row, since the second call reuses the scratch the first one left
behind. Runs alone in a fresh process as well as after the other tests."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1705_02045_gb300 import ecc, synth

pytestmark = pytest.mark.gpu

CASES = [
    # (shape, dtype, bins, generator): rows 16-byte aligned (bit-sliced kernel)
    # and not aligned (generic kernel), 2D/3D/4D, both dtypes
    ((40, 48, 64), np.uint8, 256, lambda s: synth.smooth_u8(s, 2.0, synth.SEED_BASE + 71)),
    ((23, 37, 29), np.uint16, 16384,
     lambda s: synth.two_phase_u16(s, 1.5, synth.SEED_BASE + 72)),
    ((300, 200), np.uint8, 256, lambda s: synth.uniform_u8(s, synth.SEED_BASE + 73)),
    ((5, 6, 7, 8), np.uint16, 65536,
     lambda s: synth.uniform_int(s, 65536, synth.SEED_BASE + 74, np.uint16)),
]

CONV_NAME = {ecc.ECC_CONV_V: "V", ecc.ECC_CONV_T: "T"}


@pytest.mark.parametrize("conv", [ecc.ECC_CONV_V, ecc.ECC_CONV_T])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{np.dtype(c[1]).name}")
def test_noalloc_equals_oracle_and_compute_device_twice(case, conv):
    import torch
    shape, dtype, bins, gen = case
    host = gen(shape).astype(dtype)
    expect = oracle.ecc_int(host, bins, CONV_NAME[conv])
    img = torch.from_numpy(host).cuda()
    h = ecc.ecc_create(device=0, convention=conv)
    try:
        want = torch.empty(bins, dtype=torch.int64, device="cuda")
        ecc.ecc_compute_device(h, img, bins, want)
        torch.cuda.synchronize()
        assert ecc.ecc_device_status(h) == ecc.ECC_OK
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(want.cpu().numpy(), expect)
    for _ in range(2):
        got = torch.full((bins,), -7, dtype=torch.int64, device="cuda")
        assert ecc.ecc_compute_device_noalloc(img, bins, got, convention=conv) == ecc.ECC_OK
        assert np.array_equal(got.cpu().numpy(), expect)
        assert torch.equal(got, want)


def test_noalloc_limits_and_errors():
    import torch
    lib = ecc.load()
    img = torch.zeros((4, 4, 16), dtype=torch.uint8, device="cuda")
    curve = torch.empty(70000, dtype=torch.int64, device="cuda")
    # bins beyond the fixed scratch
    assert ecc.ecc_compute_device_noalloc(img, 65537, curve) == ecc.ECC_ERR_ARG
    # a value >= bins
    img[1, 2, 3] = 200
    assert ecc.ecc_compute_device_noalloc(img, 100, curve) == ecc.ECC_ERR_VALUE
    # float images are not taken
    f = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    assert ecc.ecc_compute_device_noalloc(f, 256, curve) == ecc.ECC_ERR_DTYPE
    # rejected before anything is enqueued: a uint16 image at an odd address,
    # a host image, a host curve
    raw = torch.zeros(2 * 64 + 2, dtype=torch.uint8, device="cuda")
    dims = (C.c_int64 * 1)(64)
    assert lib.ecc_compute_device_noalloc(C.c_void_p(raw.data_ptr() + 1), dims, 1, ecc.ECC_U16,
                                          256, ecc.ECC_CONV_V, C.c_void_p(curve.data_ptr()),
                                          None) == ecc.ECC_ERR_ARG
    host = np.zeros(64, np.uint8)
    assert lib.ecc_compute_device_noalloc(host.ctypes.data_as(C.c_void_p), dims, 1, ecc.ECC_U8,
                                          256, ecc.ECC_CONV_V, C.c_void_p(curve.data_ptr()),
                                          None) == ecc.ECC_ERR_ARG
    host_curve = np.zeros(256, np.int64)
    assert lib.ecc_compute_device_noalloc(C.c_void_p(raw.data_ptr()), dims, 1, ecc.ECC_U8,
                                          256, ecc.ECC_CONV_V,
                                          host_curve.ctypes.data_as(C.c_void_p),
                                          None) == ecc.ECC_ERR_ARG
    # the next good call is unaffected by the failed ones
    img[1, 2, 3] = 0
    assert ecc.ecc_compute_device_noalloc(img, 256, curve) == ecc.ECC_OK
    got = curve[:256].cpu().numpy()
    assert np.array_equal(got, np.r_[np.ones(256, np.int64)])
    assert hasattr(lib, "ecc_compute_device_noalloc")
    assert isinstance(lib.ecc_compute_device_noalloc, C._CFuncPtr)
