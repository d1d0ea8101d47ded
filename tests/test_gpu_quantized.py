"""GPU parity of the value transform path (ecc_compute_quantized, Sec. 3
"Other Ranges of Gray Values"): float32 images shifted, scaled and rounded
into codes 0..bins-1, then the integer kernels. Compared element by element
with the oracle's transform + cell enumeration; codes are decided in float32
on both sides."""
import numpy as np
import pytest

import oracle
from paper_1705_02045_gb300 import ecc, synth

pytestmark = pytest.mark.gpu

S = synth.SEED_BASE + 1300


def _img(shape, seed, spread=1.6):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=shape) * spread).astype(np.float32)


CASES = [  # shape, bins (256 / 16384 / 65536 take the bit-sliced kernel in 1-3D)
    ((1000,), 256), ((37, 41), 256), ((9, 21, 40), 256), ((5, 33, 530), 16384),
    ((4, 17, 70), 65536), ((6, 7, 8, 9), 16384), ((11, 13, 15), 1000), ((8, 9), 37),
    ((3, 1, 1100), 256),
]


@pytest.mark.parametrize("conv", [0, 1])
@pytest.mark.parametrize("shape,bins", CASES, ids=str)
def test_quantized_matches_oracle(conv, shape, bins):
    img = _img(shape, S + len(shape) + bins)
    lo, hi = -2.0, 2.5  # values beyond both ends: clamped codes
    h = ecc.ecc_create(device=0, convention=conv)
    try:
        got = ecc.ecc_compute_quantized(h, img, lo, hi, bins)
    finally:
        ecc.ecc_destroy(h)
    want = oracle.ecc_quantized(img, lo, hi, bins, "V" if conv == 0 else "T")
    assert np.array_equal(got, want)


def test_quantized_device_input_and_unaligned():
    import torch
    img = _img((7, 19, 33), S + 1)
    h = ecc.ecc_create(device=0)
    try:
        d = torch.from_numpy(img).cuda()
        got = ecc.ecc_compute_quantized(h, d, -1.0, 1.0, 256)
        # a device view starting 4 bytes in (not 16-byte aligned): scalar loads
        buf = torch.zeros(img.size + 1, dtype=torch.float32, device="cuda")
        buf[1:].copy_(torch.from_numpy(img.ravel()))
        got_u = ecc.ecc_compute_quantized(h, buf[1:].view(img.shape), -1.0, 1.0, 256)
    finally:
        ecc.ecc_destroy(h)
    want = oracle.ecc_quantized(img, -1.0, 1.0, 256)
    assert np.array_equal(got, want) and np.array_equal(got_u, want)


def test_quantized_float32_rounding_decides_codes():
    """0.7f * 10 rounds to 7.0 in float32: the code is 7 on both sides."""
    img = np.array([[0.7, 0.3, 0.1], [0.69, 0.71, 0.05]], np.float32)
    h = ecc.ecc_create(device=0)
    try:
        got = ecc.ecc_compute_quantized(h, img, 0.0, 1.0, 10)
    finally:
        ecc.ecc_destroy(h)
    assert oracle.quantize_f32(img, 0.0, 1.0, 10).tolist() == [[7, 3, 1], [6, 7, 0]]
    assert np.array_equal(got, oracle.ecc_quantized(img, 0.0, 1.0, 10))


def test_quantized_transform_relation_mid_size():
    """32^4 float field (1 M voxels): bit-exact against the oracle, and the
    paper's relation to the exact float curve at the top value of each bin."""
    img = synth.grf_f32((32, 32, 32, 32), 3.0, S + 2)
    lo, hi, bins = float(img.min()), float(img.max()), 4096
    h = ecc.ecc_create(device=0)
    try:
        got = ecc.ecc_compute_quantized(h, img, lo, hi, bins)
        t, chi = ecc.ecc_compute(h, img)
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(got, oracle.ecc_quantized(img, lo, hi, bins))
    codes = oracle.quantize_f32(img, lo, hi, bins).ravel()
    vals = img.ravel()
    top = np.full(bins, -np.inf, np.float32)
    np.maximum.at(top, codes, vals)
    top = np.maximum.accumulate(top)
    for k in range(0, bins, 97):
        i = np.searchsorted(t, top[k], side="right") - 1
        assert got[k] == (chi[i] if i >= 0 else 0)


def test_quantized_errors_and_empty():
    h = ecc.ecc_create(device=0)
    try:
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_compute_quantized(h, np.array([0.5, np.nan], np.float32), 0.0, 1.0, 8)
        assert ei.value.status == ecc.ECC_ERR_VALUE
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_compute_quantized(h, np.zeros(4, np.float32), 1.0, 1.0, 8)
        assert ei.value.status == ecc.ECC_ERR_ARG
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_compute_quantized(h, np.zeros(4, np.float32), 0.0, 1.0, 70000)
        assert ei.value.status == ecc.ECC_ERR_ARG
        with pytest.raises(TypeError):
            ecc.ecc_compute_quantized(h, np.zeros(4, np.float64), 0.0, 1.0, 8)
        empty = ecc.ecc_compute_quantized(h, np.zeros((0, 5), np.float32), 0.0, 1.0, 8)
        assert empty.tolist() == [0] * 8
        # the handle still works after the errors
        img = _img((5, 6, 7), S + 3)
        assert np.array_equal(ecc.ecc_compute_quantized(h, img, -1.0, 1.0, 256),
                              oracle.ecc_quantized(img, -1.0, 1.0, 256))
    finally:
        ecc.ecc_destroy(h)
