"""GPU parity of the bit-sliced contribution kernel (forced with ECC_KERNEL=bits)
against the CPU oracle and against the generic kernel (ECC_KERNEL=generic).

Eligible images: 1-3D, uint8 with 256 bins or uint16 with 16384 / 65536 bins,
rows a multiple of 16 bytes. Shapes cover row groups of 1..32 lanes, rows wider
than 1024 voxels (overlapping warps), ragged tails in y and z, single planes,
tile edges, and both cell conventions."""
import os

import numpy as np
import pytest

import oracle
from paper_1705_02045_gb300 import ecc, synth

pytestmark = pytest.mark.gpu

S = synth.SEED_BASE + 900


def _handle(kernel, layout=None, **kw):
    env = {"ECC_KERNEL": kernel}
    if layout:
        env["ECC_BITS_LAYOUT"] = layout
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


def _both(img, bins, conv, layout=None):
    hb = _handle("bits", layout, bins=bins, convention=conv)
    hg = _handle("generic", bins=bins, convention=conv)
    try:
        return ecc.ecc_compute(hb, img), ecc.ecc_compute(hg, img)
    finally:
        ecc.ecc_destroy(hb)
        ecc.ecc_destroy(hg)


U8_SHAPES = [(16,), (4096,), (1, 16), (5, 32), (40, 48), (17, 9, 48), (33, 31, 64),
             (3, 40, 512), (2, 15, 496), (7, 20, 1024), (4, 10, 1056), (3, 17, 2048),
             (2, 5, 3072), (1, 1, 16), (29, 3, 16)]


@pytest.mark.parametrize("conv", [0, 1])
@pytest.mark.parametrize("shape", U8_SHAPES, ids=str)
def test_bits_u8_uniform(conv, shape):
    img = synth.uniform_u8(shape, S + len(shape) + shape[-1])
    got, gen = _both(img, 256, conv)
    want = oracle.ecc_int(img, 256, "V" if conv == 0 else "T")
    assert np.array_equal(got, want)
    assert np.array_equal(gen, want)


@pytest.mark.parametrize("conv", [0, 1])
@pytest.mark.parametrize("shape", [(21, 30, 64), (9, 50, 1040), (40, 40, 32)], ids=str)
def test_bits_u8_smooth(conv, shape):
    img = synth.smooth_u8(shape, 2.0, S + 7)
    got, _ = _both(img, 256, conv)
    assert np.array_equal(got, oracle.ecc_int(img, 256, "V" if conv == 0 else "T"))


@pytest.mark.parametrize("layout", ["rows", "columns"])
@pytest.mark.parametrize("shape", [(9, 21, 40), (5, 33, 520), (3, 7, 1600), (8, 8)], ids=str)
def test_bits_u16_14bit(shape, layout):
    img = synth.two_phase_u16(shape, 1.5, S + 11)
    got, gen = _both(img, 16384, 0, layout)
    want = oracle.ecc_int(img, 16384, "V")
    assert np.array_equal(got, want) and np.array_equal(gen, want)


@pytest.mark.parametrize("layout", ["rows", "columns"])
@pytest.mark.parametrize("conv", [0, 1])
def test_bits_u16_full_range(conv, layout):
    img = synth.uniform_int((6, 9, 24), 65536, S + 12, np.uint16)
    got, _ = _both(img, 65536, conv, layout)
    assert np.array_equal(got, oracle.ecc_int(img, 65536, "V" if conv == 0 else "T"))


def test_bits_few_levels_ties():
    img = synth.uniform_int((13, 19, 64), 2, S + 13, np.uint8)
    got, _ = _both(img, 256, 0)
    assert np.array_equal(got, oracle.ecc_int(img, 256, "V"))


@pytest.mark.parametrize("layout", ["rows", "columns"])
def test_bits_rejects_values_above_14_bits(layout):
    img = synth.two_phase_u16((4, 5, 16), 1.5, S + 14)
    img[2, 3, 7] = 20000
    h = _handle("bits", layout, bins=16384)
    try:
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_compute(h, img)
        assert ei.value.status == ecc.ECC_ERR_VALUE
    finally:
        ecc.ecc_destroy(h)


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_bits_unaligned_device_rows(offset):
    """Device images whose rows start at any byte: the bit-sliced kernel's
    4-byte funnel-shift load path (no staging copy)."""
    import torch
    img = synth.smooth_u8((9, 10, 48), 2.0, S + 15)
    buf = torch.zeros(img.size + offset, dtype=torch.uint8, device="cuda")
    view = buf[offset:].view(img.shape)
    view.copy_(torch.from_numpy(img))
    h = _handle("bits")
    try:
        assert np.array_equal(ecc.ecc_compute(h, view), oracle.ecc_int(img, 256, "V"))
    finally:
        ecc.ecc_destroy(h)


@pytest.mark.parametrize("conv", [0, 1])
@pytest.mark.parametrize("shape", [(5, 7, 37), (2, 333), (3, 9, 1100), (4, 3, 2077), (35,)],
                         ids=str)
def test_bits_odd_widths(conv, shape):
    """Row widths that are not a multiple of 16 bytes, in row groups and in
    overlapping warps."""
    img = synth.uniform_u8(shape, S + 17 + shape[-1])
    got, _ = _both(img, 256, conv)
    assert np.array_equal(got, oracle.ecc_int(img, 256, "V" if conv == 0 else "T"))


def test_bits_u16_odd_width_unaligned():
    import torch
    img = synth.two_phase_u16((4, 5, 47), 1.5, S + 18)
    if not hasattr(torch, "uint16"):
        pytest.skip("torch has no uint16")
    buf = torch.zeros(img.size + 1, dtype=torch.int16, device="cuda")
    buf[1:].copy_(torch.from_numpy(np.ascontiguousarray(img).ravel().view(np.int16)).cuda())
    view = buf[1:].view(torch.uint16).view(img.shape)
    h = _handle("bits", bins=16384)
    try:
        assert np.array_equal(ecc.ecc_compute(h, view), oracle.ecc_int(img, 16384, "V"))
    finally:
        ecc.ecc_destroy(h)


def test_bits_stream_slabs():
    """Streaming through the ring with the bit-sliced kernel on every slab."""
    img = synth.two_phase_u16((45, 30, 64), 2.0, S + 16)
    h = _handle("bits", bins=16384, slab_depth=8)
    try:
        s = ecc.ecc_stream_begin(h, img.shape, img.dtype)
        z = 0
        for n in (3, 8, 20, 14):
            ecc.ecc_stream_push_slab(h, s, img[z:z + n], z)
            z += n
        got = ecc.ecc_stream_finish(h, s)
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(got, oracle.ecc_int(img, 16384, "V"))


@pytest.mark.parametrize("conv", [0, 1])
def test_bits_full_size_512_cube(tmp_path, conv):
    """The 512^3 smoothed uint8 benchmark image: bit-sliced == generic == the
    oracle over the whole image (one process per host core, 16-plane chunks)."""
    import oracle_pool
    img = synth.smooth_u8((512, 512, 512), 4.0, synth.SEED_BASE + 1)
    got, gen = _both(img, 256, conv)
    assert np.array_equal(got, gen)
    assert got[-1] == 1
    path = tmp_path / "cube.raw"
    img.tofile(path)
    want = oracle_pool.ecc_int_parallel(path, img.shape, np.uint8, 256, planes_per_task=16,
                                        conv="V" if conv == 0 else "T")
    assert np.array_equal(got, want)


def test_tuner_picks_and_caches_a_launch_shape(tmp_path):
    """The first image of a shape class tunes the bit-sliced launch shape
    (extra timed launches) and writes the choice to the cache file; a new
    handle on the same file reuses it (exactly one launch: the contribution
    kernel, whose last block also writes the curve). Results are the oracle's
    either way."""
    path = str(tmp_path / "tune.jsonl").encode()
    img = synth.smooth_u8((40, 60, 64), 2.0, S + 19)
    want = oracle.ecc_int(img, 256, "V")
    h = ecc.ecc_create(device=0, tuner_cache=path)
    try:
        assert np.array_equal(ecc.ecc_compute(h, img), want)
        tuned_launches = ecc.ecc_launch_count(h)
    finally:
        ecc.ecc_destroy(h)
    lines = open(path.decode()).read().strip().splitlines()
    assert len(lines) == 1 and '"warps"' in lines[0] and '"zc"' in lines[0]
    assert '"hist": 0' in lines[0] or '"hist": 2' in lines[0]
    assert '"layout": 1' in lines[0] or '"layout": 2' in lines[0]
    assert tuned_launches > 2
    h = ecc.ecc_create(device=0, tuner_cache=path)
    try:
        assert np.array_equal(ecc.ecc_compute(h, img), want)
        assert ecc.ecc_launch_count(h) == 1
    finally:
        ecc.ecc_destroy(h)


def test_plane_512_uniform_u8_matches_oracle():
    """The 2D 512 x 512 i.i.d. uniform uint8 image of the benchmark, both
    conventions, device and host input."""
    import torch
    img = synth.uniform_u8((512, 512), synth.SEED_BASE + 0)
    for conv in (0, 1):
        h = ecc.ecc_create(device=0, convention=conv)
        try:
            got_h = ecc.ecc_compute(h, img)
            got_d = ecc.ecc_compute(h, torch.from_numpy(img).cuda())
        finally:
            ecc.ecc_destroy(h)
        want = oracle.ecc_int(img, 256, "V" if conv == 0 else "T")
        assert np.array_equal(got_h, want) and np.array_equal(got_d, want)


def test_full_size_14bit_volume_streamed_resident_generic(tmp_path):
    """The 3072 x 3072 x 1536 14-bit two-phase volume of the benchmark (27 GiB):
    streamed from pinned host memory in 64-plane slabs through a 4 GiB ring,
    resident with the bit-sliced kernel, and resident with the generic kernel
    give the same curve, which is 0 below the minimum and 1 at the top, and
    equals the oracle's over the whole volume (one process per host core,
    4-plane chunks of a raw copy of the volume, Sec. 3 chunk additivity)."""
    import torch
    import oracle_pool
    shape = (1536, 3072, 3072)
    host = torch.empty(shape, dtype=torch.int16, pin_memory=True)
    hview = host.numpy().view(np.uint16)
    for z0, slab in synth.two_phase_u16_slabs(shape, 6.0, synth.SEED_BASE + 2, 64):
        hview[z0:z0 + slab.shape[0]] = slab
    h = ecc.ecc_create(device=0, bins=16384, slab_depth=64, ring_bytes=4 << 30)
    try:
        s = ecc.ecc_stream_begin(h, shape, np.uint16)
        hu = host.view(torch.uint16)
        for z0 in range(0, shape[0], 64):
            ecc.ecc_stream_push_slab(h, s, hu[z0:z0 + 64], z0)
        streamed = ecc.ecc_stream_finish(h, s)
        d = hu.cuda()
        resident = ecc.ecc_compute(h, d)
    finally:
        ecc.ecc_destroy(h)
    hg = _handle("generic", bins=16384)
    try:
        generic = ecc.ecc_compute(hg, d)
    finally:
        ecc.ecc_destroy(hg)
    lo = int(d.view(torch.int16).min().item())  # values are 14-bit
    del d
    assert np.array_equal(streamed, resident) and np.array_equal(resident, generic)
    assert resident[-1] == 1 and not np.any(resident[:lo])
    path = tmp_path / "vol.raw"
    hview.tofile(path)
    del hview, hu, host
    want = oracle_pool.ecc_int_parallel(path, shape, np.uint16, 16384, planes_per_task=4)
    assert np.array_equal(resident, want)


def test_1d_longer_than_2_pow_31():
    """A 1D uint8 image of 2^31 + 12345 voxels (64-bit indexing throughout):
    chi(K_t) is the number of runs of {f <= t}, i.e. the voxels <= t minus the
    adjacent pairs whose larger value is <= t (the run count the oracle is
    pinned to in 1D)."""
    import torch
    n = (1 << 31) + 12345
    g = torch.Generator(device="cuda").manual_seed(synth.SEED_BASE + 90)
    d = torch.randint(0, 256, (n,), generator=g, device="cuda", dtype=torch.int16).to(torch.uint8)
    torch.cuda.synchronize()
    h = ecc.ecc_create(device=0)
    try:
        got = ecc.ecc_compute(h, d)
    finally:
        ecc.ecc_destroy(h)
    c1 = torch.bincount(d.long(), minlength=256)
    pair_max = torch.maximum(d[1:], d[:-1]).long()
    c2 = torch.bincount(pair_max, minlength=256)
    want = (torch.cumsum(c1, 0) - torch.cumsum(c2, 0)).cpu().numpy()
    assert np.array_equal(got, want)
    assert got[-1] == 1
