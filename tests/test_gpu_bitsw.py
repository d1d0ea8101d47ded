"""GPU parity of the warp-column layout of the bit-sliced contribution kernel
(forced with ECC_KERNEL=bits, ECC_BITS_LAYOUT=columns) against the CPU oracle.

A warp holds 32 rows of one 32-voxel word each and owns the middle 30 of both,
so the shapes put image edges at every position relative to the 30-voxel
tiles (widths and heights 1, 2, 29..33, 59..61, 89..91, 512), rows whose
start is or is not 16 bytes aligned (16-byte chunk loads and the 4-byte word
path), device images at odd byte offsets, single planes, plane spans that
cross warp columns, both cell conventions and the three bin counts."""
import os

import numpy as np
import pytest

import oracle
from paper_1705_02045_gb300 import ecc, synth

pytestmark = pytest.mark.gpu

S = synth.SEED_BASE + 1900


def _columns(**kw):
    env = {"ECC_KERNEL": "bits", "ECC_BITS_LAYOUT": "columns"}
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return ecc.ecc_create(device=0, **kw)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


def _run(img, bins, conv):
    h = _columns(bins=bins, convention=conv)
    try:
        return ecc.ecc_compute(h, img)
    finally:
        ecc.ecc_destroy(h)


U8_SHAPES = [(1,), (2,), (31,), (64,), (1, 1), (1, 30), (2, 31), (30, 30), (31, 32),
             (29, 61), (33, 59), (60, 60), (61, 91), (89, 90), (3, 1, 1), (4, 2, 33),
             (5, 31, 29), (6, 30, 60), (7, 32, 61), (3, 59, 90), (2, 91, 89), (9, 17, 512),
             (4, 64, 48), (3, 61, 50), (40, 3, 7)]


@pytest.mark.parametrize("conv", [0, 1])
@pytest.mark.parametrize("shape", U8_SHAPES, ids=str)
def test_columns_u8_uniform(conv, shape):
    img = synth.uniform_u8(shape, S + len(shape) + shape[-1])
    want = oracle.ecc_int(img, 256, "V" if conv == 0 else "T")
    assert np.array_equal(_run(img, 256, conv), want)


@pytest.mark.parametrize("conv", [0, 1])
@pytest.mark.parametrize("shape", [(21, 30, 64), (9, 50, 100), (40, 40, 32), (12, 61, 91)],
                         ids=str)
def test_columns_u8_smooth(conv, shape):
    """Plateaus of a smoothed, requantised field: the index tie-break decides."""
    img = synth.smooth_u8(shape, 2.0, S + 7)
    assert np.array_equal(_run(img, 256, conv), oracle.ecc_int(img, 256, "V" if conv == 0 else "T"))


@pytest.mark.parametrize("conv", [0, 1])
@pytest.mark.parametrize("shape", [(9, 21, 40), (5, 33, 61), (3, 7, 160), (8, 8), (4, 31, 90)],
                         ids=str)
def test_columns_u16_14bit(conv, shape):
    """Noisy two-phase 14-bit data: most words take the dense deposit path."""
    img = synth.two_phase_u16(shape, 1.5, S + 11)
    assert np.array_equal(_run(img, 16384, conv),
                          oracle.ecc_int(img, 16384, "V" if conv == 0 else "T"))


@pytest.mark.parametrize("conv", [0, 1])
@pytest.mark.parametrize("shape", [(6, 9, 24), (3, 31, 33)], ids=str)
def test_columns_u16_full_range(conv, shape):
    """65536 bins: global-memory histogram."""
    img = synth.uniform_int(shape, 65536, S + 12, np.uint16)
    assert np.array_equal(_run(img, 65536, conv),
                          oracle.ecc_int(img, 65536, "V" if conv == 0 else "T"))


@pytest.mark.parametrize("offset", [1, 2, 3, 5, 8, 13])
@pytest.mark.parametrize("dtype", ["u8", "u16"])
def test_columns_device_rows_at_any_offset(offset, dtype):
    """Device images at byte offsets that are not 16-byte aligned: the
    4-byte word load path (uint16 images at even offsets)."""
    import torch
    if dtype == "u8":
        img, bins, eb = synth.smooth_u8((7, 33, 64), 2.0, S + 15), 256, 1
    else:
        img, bins, eb = synth.two_phase_u16((5, 31, 32), 1.5, S + 16), 16384, 2
        offset *= 2
    buf = torch.zeros(img.nbytes + offset, dtype=torch.uint8, device="cuda")
    buf[offset:].copy_(torch.from_numpy(img.view(np.uint8).reshape(-1)))
    view = buf[offset:]
    if eb == 2:
        view = view.view(torch.uint16)
    view = view.view(img.shape)
    h = _columns(bins=bins)
    try:
        got = ecc.ecc_compute(h, view)
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(got, oracle.ecc_int(img, bins, "V"))


def test_columns_full_size_512_cube_slab():
    """64 planes of the 512^3 benchmark image (smoothed, sigma = 4) against
    the oracle, in both conventions."""
    img = synth.smooth_u8((64, 512, 512), 4.0, synth.SEED_BASE + 1)
    for conv in (0, 1):
        assert np.array_equal(_run(img, 256, conv),
                              oracle.ecc_int(img, 256, "V" if conv == 0 else "T"))


def test_columns_stream_slabs():
    """Streamed slabs (planes resident only in the ring, collars kept on the
    device) through the warp-column kernel."""
    img = synth.two_phase_u16((37, 40, 70), 1.5, S + 21)
    h = _columns(bins=16384, slab_depth=8, ring_bytes=1 << 20)
    try:
        s = ecc.ecc_stream_begin(h, img.shape, np.uint16)
        z = 0
        for n in (5, 8, 1, 13, 10):
            ecc.ecc_stream_push_slab(h, s, img[z:z + n], z)
            z += n
        got = ecc.ecc_stream_finish(h, s)
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(got, oracle.ecc_int(img, 16384, "V"))
