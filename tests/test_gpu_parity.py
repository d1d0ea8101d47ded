"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by
element (integers: bit-exact; float pairs: exact keys and exact int64 chi).

Cases span several tiles with ragged tails in every axis, the degenerate
shapes (single voxel, a single row or column, empty), prime extents, both cell
conventions, every dtype and both histogram paths (shared memory for up to
16384 bins, global memory above).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1705_02045_gb300 import ecc, synth

pytestmark = pytest.mark.gpu

S = synth.SEED_BASE


@pytest.fixture(scope="module")
def hV(lib):
    h = ecc.ecc_create(device=0, convention=ecc.ECC_CONV_V)
    yield h
    ecc.ecc_destroy(h)


@pytest.fixture(scope="module")
def hT(lib):
    h = ecc.ecc_create(device=0, convention=ecc.ECC_CONV_T)
    yield h
    ecc.ecc_destroy(h)


def _handle(hV, hT, conv):
    return hV if conv == "V" else hT


INT_SHAPES = [(1,), (7,), (1000,), (100003,), (1, 1), (1, 50), (50, 1), (33, 65),
              (1, 1, 1), (2, 3, 4), (17, 9, 33), (31, 37, 41), (5, 70, 3),
              (2, 2, 2, 2), (3, 5, 7, 9), (7, 6, 35, 5), (4, 9, 3, 66)]


@pytest.mark.parametrize("conv", ["V", "T"])
@pytest.mark.parametrize("shape", INT_SHAPES, ids=str)
def test_u8_uniform(hV, hT, conv, shape):
    img = synth.uniform_u8(shape, S + 10 + len(shape))
    got = ecc.ecc_compute(_handle(hV, hT, conv), img)
    assert np.array_equal(got, oracle.ecc_int(img, 256, conv))


@pytest.mark.parametrize("conv", ["V", "T"])
@pytest.mark.parametrize("shape", [(40, 45), (19, 40, 37), (6, 11, 10, 13)], ids=str)
def test_u8_smooth_with_ties(hV, hT, conv, shape):
    """Smooth, requantised fields have plateaus: the index tie-break matters."""
    img = synth.smooth_u8(shape, 1.5, S + 20)
    got = ecc.ecc_compute(_handle(hV, hT, conv), img)
    assert np.array_equal(got, oracle.ecc_int(img, 256, conv))


@pytest.mark.parametrize("shape", [(3, 5), (9, 8, 7), (4, 5, 6, 3)], ids=str)
def test_few_levels_many_ties(hV, shape):
    img = synth.uniform_int(shape, 3, S + 30, np.uint8)
    assert np.array_equal(ecc.ecc_compute(hV, img), oracle.ecc_int(img, 256, "V"))


def test_small_bins(lib):
    h = ecc.ecc_create(device=0, bins=8)
    try:
        img = synth.uniform_int((13, 14, 15), 8, S + 31, np.uint8)
        got = ecc.ecc_compute(h, img)
        assert got.shape == (8,)
        assert np.array_equal(got, oracle.ecc_int(img, 8, "V"))
    finally:
        ecc.ecc_destroy(h)


@pytest.mark.parametrize("shape", [(21, 33, 40), (5, 6, 7, 8)], ids=str)
def test_u16_14bit_smem_histogram(lib, shape):
    h = ecc.ecc_create(device=0, bins=16384)
    try:
        img = synth.two_phase_u16(shape, 2.0, S + 40)
        assert np.array_equal(ecc.ecc_compute(h, img), oracle.ecc_int(img, 16384, "V"))
    finally:
        ecc.ecc_destroy(h)


@pytest.mark.parametrize("conv", ["V", "T"])
def test_u16_full_range_global_histogram(hV, hT, conv):
    img = synth.uniform_int((9, 40, 35), 65536, S + 41, np.uint16)
    got = ecc.ecc_compute(_handle(hV, hT, conv), img)
    assert got.shape == (65536,)
    assert np.array_equal(got, oracle.ecc_int(img, 65536, conv))


@pytest.mark.parametrize("conv", ["V", "T"])
@pytest.mark.parametrize("shape", [(1,), (9,), (9, 13), (8, 9, 10), (6, 7, 8, 9), (3, 40, 2, 35)],
                         ids=str)
def test_f32_pairs(hV, hT, conv, shape):
    img = synth.grf_f32(shape, 1.2, S + 50)
    t, chi = ecc.ecc_compute(_handle(hV, hT, conv), img)
    t_ref, chi_ref = oracle.ecc_pairs_float(img, conv)
    assert np.array_equal(t, t_ref)
    assert np.array_equal(chi, chi_ref)


@pytest.mark.parametrize("conv", ["V", "T"])
@pytest.mark.parametrize("shape,kind", [
    ((3, 4, 5, 130), "u8"), ((5, 9, 6, 129), "u8"), ((2, 5, 9, 257), "u16"),
    ((4, 3, 3, 128), "f32"), ((3, 2, 7, 300), "f32"), ((6, 5, 11, 140), "f32")], ids=str)
def test_4d_several_x_tiles(hV, hT, conv, shape, kind):
    """4D rows wider than one 128-voxel tile, ragged in x, y and z: shared
    histogram (u8), global histogram (u16, 65536 bins) and pairs (f32)."""
    h = _handle(hV, hT, conv)
    if kind == "u8":
        img = synth.uniform_u8(shape, S + 55)
        assert np.array_equal(ecc.ecc_compute(h, img), oracle.ecc_int(img, 256, conv))
    elif kind == "u16":
        img = synth.uniform_int(shape, 65536, S + 56, np.uint16)
        assert np.array_equal(ecc.ecc_compute(h, img), oracle.ecc_int(img, 65536, conv))
    else:
        img = synth.grf_f32(shape, 1.5, S + 57)
        t, chi = ecc.ecc_compute(h, img)
        t_ref, chi_ref = oracle.ecc_pairs_float(img, conv)
        assert np.array_equal(t, t_ref) and np.array_equal(chi, chi_ref)


@pytest.mark.parametrize("conv", ["V", "T"])
@pytest.mark.parametrize("shape,kind", [
    ((4, 23, 9, 40), "u8"), ((3, 20, 6, 31), "u8"), ((2, 1, 5, 33), "u8"),
    ((3, 31, 5, 70), "u16_14"), ((2, 11, 33, 9), "u16"),
    ((3, 21, 31, 33), "f32"), ((4, 10, 7, 20), "f32"), ((2, 12, 3, 62), "f32")], ids=str)
def test_4d_several_z_tiles(hV, hT, conv, shape, kind):
    """4D images whose z extent crosses the 4D kernel's blocks of own
    z-slices (exact multiples, ragged tails, a single slice), in every value
    mode: shared histogram (u8, 14-bit u16), global histogram (65536 bins)
    and pairs (f32)."""
    h = _handle(hV, hT, conv)
    if kind == "u8":
        img = synth.smooth_u8(shape, 1.5, S + 58)
        assert np.array_equal(ecc.ecc_compute(h, img), oracle.ecc_int(img, 256, conv))
    elif kind == "u16_14":
        img = synth.two_phase_u16(shape, 1.5, S + 59)
        h14 = ecc.ecc_create(device=0, bins=16384, convention=0 if conv == "V" else 1)
        try:
            got = ecc.ecc_compute(h14, img)
        finally:
            ecc.ecc_destroy(h14)
        assert np.array_equal(got, oracle.ecc_int(img, 16384, conv))
    elif kind == "u16":
        img = synth.uniform_int(shape, 65536, S + 60, np.uint16)
        assert np.array_equal(ecc.ecc_compute(h, img), oracle.ecc_int(img, 65536, conv))
    else:
        img = synth.grf_f32(shape, 1.5, S + 61)
        t, chi = ecc.ecc_compute(h, img)
        t_ref, chi_ref = oracle.ecc_pairs_float(img, conv)
        assert np.array_equal(t, t_ref) and np.array_equal(chi, chi_ref)


@pytest.mark.parametrize("conv", ["V", "T"])
def test_f32_4d_full_size_equals_oracle(tmp_path, conv):
    """The 128^4 float field of the benchmark (Gaussian random field, sigma = 3
    per axis), element by element against the oracle over the whole image:
    every (threshold, chi) pair, computed on the host cores in chunks of 8
    planes whose maps are merged by value."""
    import oracle_pool
    d = synth.grf_f32_torch((128, 128, 128, 128), 3.0, synth.SEED_BASE + 4).contiguous()
    h = ecc.ecc_create(device=0, convention=ecc.ECC_CONV_V if conv == "V" else ecc.ECC_CONV_T)
    try:
        t, chi = ecc.ecc_compute(h, d)
    finally:
        ecc.ecc_destroy(h)
    host = d.cpu().numpy()
    del d
    path = tmp_path / "grf4.raw"
    host.tofile(path)
    t_ref, chi_ref = oracle_pool.ecc_pairs_float_parallel(path, host.shape, 8, conv=conv)
    assert len(t) == len(t_ref)
    assert np.array_equal(t, t_ref) and np.array_equal(chi, chi_ref)


@pytest.mark.parametrize("conv", ["V", "T"])
@pytest.mark.parametrize("shape", [(20, 48, 64, 72), (70, 240, 256)], ids=str)
def test_f32_host_image_chunked_upload(tmp_path, conv, shape):
    """Float images of 16 MB or more in host memory are uploaded in plane
    chunks while the pairs kernel runs on the chunks already there: the pairs
    equal the oracle's (4D and 3D, both conventions)."""
    import oracle_pool
    img = synth.grf_f32(shape, 2.0, S + 59)
    assert img.nbytes >= 16 << 20
    h = ecc.ecc_create(device=0, convention=ecc.ECC_CONV_V if conv == "V" else ecc.ECC_CONV_T)
    try:
        t, chi = ecc.ecc_compute(h, img)
        t2, chi2 = ecc.ecc_compute(h, img)  # the buffer reused after its readers
    finally:
        ecc.ecc_destroy(h)
    path = tmp_path / "f.raw"
    img.tofile(path)
    t_ref, chi_ref = oracle_pool.ecc_pairs_float_parallel(path, shape, 4, conv=conv)
    assert np.array_equal(t, t_ref) and np.array_equal(chi, chi_ref)
    assert np.array_equal(t2, t_ref) and np.array_equal(chi2, chi_ref)


@pytest.mark.parametrize("conv", ["V", "T"])
def test_f32_4d_noise_past_1024_radix_tiles(tmp_path, conv):
    """4D i.i.d. uniform floats, 64^4: more than half the voxels carry a
    non-zero change, so the (key, change) pairs exceed 1024 radix tiles of
    1024 pairs several times over and the digit offsets carry across tile
    chunks, and the segment and
    non-zero compactions run on many blocks. Element by element against the
    oracle."""
    import oracle_pool
    shape = (64, 64, 64, 64)
    img = np.random.default_rng(S + 58).random(size=shape, dtype=np.float32)
    h = ecc.ecc_create(device=0, convention=ecc.ECC_CONV_V if conv == "V" else ecc.ECC_CONV_T)
    try:
        t, chi = ecc.ecc_compute(h, img)
    finally:
        ecc.ecc_destroy(h)
    path = tmp_path / "noise4.raw"
    img.tofile(path)
    t_ref, chi_ref = oracle_pool.ecc_pairs_float_parallel(path, shape, 4, conv=conv)
    assert len(t_ref) > 4 * 1024 * 1024
    assert np.array_equal(t, t_ref) and np.array_equal(chi, chi_ref)


def test_f32_4d_full_size_properties(lib):
    """The 128^4 float field of the benchmark: thresholds strictly
    ascending, chi = 1 at the top (the full box is contractible), and the
    value transform of the same image through the integer 4D path agrees with
    the pairs at the top value of every 512th bin."""
    d = synth.grf_f32_torch((128, 128, 128, 128), 3.0, synth.SEED_BASE + 4).contiguous()
    lo, hi, bins = float(d.min()), float(d.max()), 4096
    h = ecc.ecc_create(device=0)
    try:
        t, chi = ecc.ecc_compute(h, d)
        q = ecc.ecc_compute_quantized(h, d, lo, hi, bins)
    finally:
        ecc.ecc_destroy(h)
    assert np.all(np.diff(t) > 0) and chi[-1] == 1 and q[-1] == 1
    import torch
    vals = d.reshape(-1)
    codes = torch.from_numpy(oracle.quantize_f32(vals.cpu().numpy(), lo, hi, bins)).cuda()
    top = torch.full((bins,), float("-inf"), device="cuda")
    top = top.scatter_reduce(0, codes, vals, reduce="amax")
    top = torch.cummax(top, 0).values.cpu().numpy()
    for k in range(0, bins, 512):
        i = np.searchsorted(t, top[k], side="right") - 1
        assert q[k] == (chi[i] if i >= 0 else 0)


def test_f32_ties_and_signed_zero(hV):
    rng = np.random.default_rng(S + 51)
    img = (rng.integers(-3, 4, size=(10, 11, 12)) * 0.5).astype(np.float32)
    img[img == 0] = np.where(rng.random(np.sum(img == 0)) < 0.5, -0.0, 0.0)
    t, chi = ecc.ecc_compute(hV, img)
    t_ref, chi_ref = oracle.ecc_pairs_float(img, "V")
    assert np.array_equal(t, t_ref) and np.array_equal(chi, chi_ref)
    assert not np.any(np.signbit(t[t == 0]))


def test_golden_fixtures(hV, hT, lib):
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_small.json")
    for rec in json.load(open(path)):
        img = np.array(rec["values"], dtype=rec["dtype"]).reshape(rec["shape"])
        for conv in ("V", "T"):
            h = _handle(hV, hT, conv)
            if rec["dtype"] == "float32":
                t, chi = ecc.ecc_compute(h, img)
                assert [[float(a), int(b)] for a, b in zip(t, chi)] == rec["pairs_" + conv]
            else:
                hb = ecc.ecc_create(device=0, bins=rec["bins"],
                                    convention=0 if conv == "V" else 1)
                try:
                    curve = ecc.ecc_compute(hb, img)
                finally:
                    ecc.ecc_destroy(hb)
                a = np.diff(np.r_[0, curve])
                nz = np.flatnonzero(a)
                assert [[int(x), int(a[x])] for x in nz] == rec["vcec_" + conv], rec["name"]


# ---- edge cases and errors -------------------------------------------------

def test_empty_image(hV):
    got = ecc.ecc_compute(hV, np.zeros((0, 5, 5), np.uint8))
    assert got.shape == (256,) and not got.any()
    t, chi = ecc.ecc_compute(hV, np.zeros((4, 0), np.float32))
    assert t.size == 0 and chi.size == 0


def test_value_out_of_range(lib):
    h = ecc.ecc_create(device=0, bins=16)
    try:
        img = np.zeros((4, 5, 6), np.uint8)
        img[2, 3, 4] = 16
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_compute(h, img)
        assert ei.value.status == ecc.ECC_ERR_VALUE
        # the handle stays usable
        img[2, 3, 4] = 15
        assert np.array_equal(ecc.ecc_compute(h, img), oracle.ecc_int(img, 16, "V"))
    finally:
        ecc.ecc_destroy(h)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_nan_inf_rejected(hV, bad):
    img = np.zeros((3, 4, 5), np.float32)
    img[1, 2, 3] = bad
    with pytest.raises(ecc.EccError) as ei:
        ecc.ecc_compute(hV, img)
    assert ei.value.status == ecc.ECC_ERR_VALUE


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("pos", [(0, 0, 0, 0), (2, 11, 6, 39), (1, 10, 3, 30), (1, 9, 0, 31),
                                 (0, 5, 6, 1)], ids=str)
def test_4d_nan_inf_rejected(hV, bad, pos):
    """A NaN or an infinity anywhere in a 4D float image (corners, the edges
    of the 30-voxel x tiles and of the blocks of own z-slices, the last
    volume) is an error of the whole call; the handle stays usable."""
    img = synth.grf_f32((3, 12, 7, 40), 1.5, S + 62)
    good = img.copy()
    img[pos] = bad
    with pytest.raises(ecc.EccError) as ei:
        ecc.ecc_compute(hV, img)
    assert ei.value.status == ecc.ECC_ERR_VALUE
    t, chi = ecc.ecc_compute(hV, good)
    t_ref, chi_ref = oracle.ecc_pairs_float(good, "V")
    assert np.array_equal(t, t_ref) and np.array_equal(chi, chi_ref)


@pytest.mark.parametrize("conv", ["V", "T"])
def test_4d_signed_zeros(hV, hT, conv):
    """+0.0 and -0.0 are one value (ties between them broken by the linear
    index): a 4D field with many zeros of both signs against the oracle."""
    rng = np.random.default_rng(S + 63)
    shape = (4, 11, 9, 37)
    img = rng.choice(np.array([-1.5, -0.0, 0.0, 0.75], np.float32), size=shape)
    img[0, 0, 0, :8] = -0.0
    t, chi = ecc.ecc_compute(_handle(hV, hT, conv), img)
    t_ref, chi_ref = oracle.ecc_pairs_float(img, conv)
    assert np.array_equal(t, t_ref) and np.array_equal(chi, chi_ref)


def test_bad_arguments(hV):
    lib = ecc.load()
    import ctypes as C
    r = ecc.ecc_result()
    dims = (C.c_int64 * 5)(2, 2, 2, 2, 2)
    buf = np.zeros(32, np.uint8)
    p = buf.ctypes.data_as(C.c_void_p)
    assert lib.ecc_compute(hV, p, dims, 5, ecc.ECC_U8, C.byref(r)) == ecc.ECC_ERR_ARG
    assert lib.ecc_compute(hV, p, dims, 0, ecc.ECC_U8, C.byref(r)) == ecc.ECC_ERR_ARG
    neg = (C.c_int64 * 2)(2, -1)
    assert lib.ecc_compute(hV, p, neg, 2, ecc.ECC_U8, C.byref(r)) == ecc.ECC_ERR_ARG
    assert lib.ecc_compute(hV, p, dims, 2, 9, C.byref(r)) == ecc.ECC_ERR_DTYPE
    assert lib.ecc_compute(hV, None, dims, 2, ecc.ECC_U8, C.byref(r)) == ecc.ECC_ERR_ARG
    assert "NULL" in ecc.ecc_last_error(hV)


# ---- device pointers --------------------------------------------------------

def test_device_tensor_input(hV):
    import torch
    img = synth.smooth_u8((33, 40, 50), 2.0, S + 60)
    t = torch.from_numpy(img).cuda()
    assert np.array_equal(ecc.ecc_compute(hV, t), oracle.ecc_int(img, 256, "V"))


def test_compute_device_on_torch_stream(hV):
    import torch
    img = synth.uniform_int((20, 30, 40), 16384, S + 61, np.uint16)
    d = torch.from_numpy(img).cuda()
    curve = torch.empty(16384, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    ecc.ecc_compute_device(hV, d, 16384, curve, stream=s)
    s.synchronize()
    assert ecc.ecc_device_status(hV) == ecc.ECC_OK
    assert np.array_equal(curve.cpu().numpy(), oracle.ecc_int(img, 16384, "V"))


def test_device_status_reports_bad_value(lib):
    import torch
    h = ecc.ecc_create(device=0)
    try:
        img = torch.zeros((4, 4, 4), dtype=torch.uint8, device="cuda")
        img[1, 1, 1] = 200
        curve = torch.empty(100, dtype=torch.int64, device="cuda")
        ecc.ecc_compute_device(h, img, 100, curve)
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_device_status(h)
        assert ei.value.status == ecc.ECC_ERR_VALUE
        assert ecc.ecc_device_status(h) == ecc.ECC_OK  # flag cleared
    finally:
        ecc.ecc_destroy(h)


# ---- the benchmark workloads at full size ----------------------------------

def test_full_size_2d_512_uniform(hV):
    img = synth.uniform_u8((512, 512), S + 0)
    assert np.array_equal(ecc.ecc_compute(hV, img), oracle.ecc_int(img, 256, "V"))


def test_full_size_3d_512_smooth_device_path(hV):
    """The 512^3 smoothed uint8 workload in the launch configuration the
    benchmark times (device-resident image, ecc_compute_device)."""
    import torch
    img = synth.smooth_u8((512, 512, 512), 4.0, S + 1)
    d = torch.from_numpy(img).cuda()
    curve = torch.empty(256, dtype=torch.int64, device="cuda")
    ecc.ecc_compute_device(hV, d, 256, curve)
    torch.cuda.synchronize()
    assert ecc.ecc_device_status(hV) == ecc.ECC_OK
    got = curve.cpu().numpy()
    want = np.zeros(256, np.int64)
    # oracle in z-ranges of cells (chunk decomposition; bounded host memory)
    for lo in range(0, 513, 128):
        want += oracle.vcec_int_zrange(img, 256, lo, min(lo + 128, 513), "V")
    assert np.array_equal(got, oracle.ecc_from_vcec(want))


@pytest.mark.parametrize("shape,dtype,bins", [
    ((96, 400, 500), np.uint16, 16384),   # 38 MB: 2 chunks, the last cut in halves
    ((2, 4096, 2048), np.uint8, 256),     # 16 MB in 2 planes: 2 chunks
    ((20, 30, 100, 300), np.uint8, 256),  # 4D, generic kernel, chunked
    ((70, 300, 800), np.uint8, 200),      # bins the bit-sliced kernel does not take
], ids=str)
def test_large_host_image_chunked_upload(shape, dtype, bins):
    """Host images of 16 MB and more are uploaded in plane chunks overlapping
    the kernels (each chunk's launches take its planes but the last, plus the
    previous chunk's last plane): the curve equals the one of the same bytes
    on the device (uploaded whole) and the oracle's."""
    import torch
    rng = np.random.default_rng(S + 77)
    img = rng.integers(0, bins, size=shape).astype(dtype)
    h = ecc.ecc_create(device=0, bins=bins)
    try:
        got = ecc.ecc_compute(h, img)
        raw = torch.from_numpy(img.view(np.int16) if dtype == np.uint16 else img).cuda()
        d = raw.view(torch.uint16) if dtype == np.uint16 else raw
        ref = ecc.ecc_compute(h, d)
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(got, ref)
    assert got[-1] == 1
    assert np.array_equal(got, oracle.ecc_int(img, bins, "V"))


def test_large_host_image_value_error_in_a_late_chunk():
    img = synth.smooth_u8((64, 512, 512), 2.0, S + 79).astype(np.uint16)
    img[50, 7, 9] = 300
    h = ecc.ecc_create(device=0, bins=256)
    try:
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_compute(h, img)
        assert ei.value.status == ecc.ECC_ERR_VALUE
        img[50, 7, 9] = 3
        assert ecc.ecc_compute(h, img)[-1] == 1
    finally:
        ecc.ecc_destroy(h)
