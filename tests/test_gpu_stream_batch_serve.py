"""GPU parity of the streamed, batched and served paths against the CPU oracle,
and their host-side error handling (wrong slab order, missing planes, values
out of range, unknown requests, a memory cap smaller than the request mix)."""
import numpy as np
import pytest

import oracle
from paper_1705_02045_gb300 import ecc, synth

pytestmark = pytest.mark.gpu

S = synth.SEED_BASE + 500


def _push_all(h, s, img, sizes):
    z = 0
    for n in sizes:
        ecc.ecc_stream_push_slab(h, s, img[z:z + n], z)
        z += n
    assert z == img.shape[0]


# ---- streaming --------------------------------------------------------------

@pytest.mark.parametrize("conv", [0, 1])
def test_stream_3d_u8_uneven_slabs_small_ring(lib, conv):
    img = synth.smooth_u8((40, 33, 37), 1.5, S + 1)
    plane = 33 * 37
    # ring of 13 planes: 2 slots of depth 4 (+2 collar planes each)
    h = ecc.ecc_create(device=0, slab_depth=4, ring_bytes=13 * plane, convention=conv)
    try:
        s = ecc.ecc_stream_begin(h, img.shape, img.dtype)
        _push_all(h, s, img, [1, 5, 3, 9, 22])
        got = ecc.ecc_stream_finish(h, s)
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(got, oracle.ecc_int(img, 256, "V" if conv == 0 else "T"))


def test_stream_4d_u16_14bit(lib):
    img = synth.two_phase_u16((12, 5, 6, 7), 1.5, S + 2)
    h = ecc.ecc_create(device=0, slab_depth=3, bins=16384)
    try:
        s = ecc.ecc_stream_begin(h, img.shape, img.dtype)
        _push_all(h, s, img, [2, 2, 7, 1])
        got = ecc.ecc_stream_finish(h, s)
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(got, oracle.ecc_int(img, 16384, "V"))


@pytest.mark.parametrize("shape", [(50, 70), (31,)], ids=str)
def test_stream_1d_2d(lib, shape):
    img = synth.uniform_u8(shape, S + 3)
    h = ecc.ecc_create(device=0, slab_depth=8)
    try:
        s = ecc.ecc_stream_begin(h, img.shape, img.dtype)
        _push_all(h, s, img, [shape[0] // 3, shape[0] - shape[0] // 3])
        got = ecc.ecc_stream_finish(h, s)
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(got, oracle.ecc_int(img, 256, "V"))


def test_stream_equals_resident_larger(lib):
    """Streamed in slabs of 16 through a 3-slot ring == resident, bit for bit."""
    img = synth.two_phase_u16((100, 160, 144), 3.0, S + 4)
    h = ecc.ecc_create(device=0, slab_depth=16, bins=16384)
    try:
        resident = ecc.ecc_compute(h, img)
        s = ecc.ecc_stream_begin(h, img.shape, img.dtype)
        _push_all(h, s, img, [37, 37, 26])
        streamed = ecc.ecc_stream_finish(h, s)
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(streamed, resident)
    assert resident[-1] == 1
    sub = img[:, :40, :50]
    assert np.array_equal(ecc_sub(sub), oracle.ecc_int(sub, 16384, "V"))


def ecc_sub(sub):
    h = ecc.ecc_create(device=0, bins=16384)
    try:
        return ecc.ecc_compute(h, np.ascontiguousarray(sub))
    finally:
        ecc.ecc_destroy(h)


def test_stream_pinned_host_buffer(lib):
    import torch
    img = synth.smooth_u8((20, 64, 64), 2.0, S + 5)
    h = ecc.ecc_create(device=0, slab_depth=5)
    try:
        s = ecc.ecc_stream_begin(h, img.shape, img.dtype)
        buf = torch.empty((5, 64, 64), dtype=torch.uint8).pin_memory()
        for z in range(0, 20, 5):
            buf.copy_(torch.from_numpy(img[z:z + 5]))
            ecc.ecc_stream_push_slab(h, s, buf, z)  # buffer reused right after
        got = ecc.ecc_stream_finish(h, s)
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(got, oracle.ecc_int(img, 256, "V"))


def test_stream_device_slabs(lib):
    """Slabs pushed from device memory (a CUDA tensor reused for every slab,
    as the call returns once its copies are done), 14-bit values, uneven
    slabs; the curve is the oracle's."""
    import torch
    img = synth.two_phase_u16((23, 40, 70), 1.5, S + 6)
    h = ecc.ecc_create(device=0, bins=16384, slab_depth=4)
    try:
        s = ecc.ecc_stream_begin(h, img.shape, img.dtype)
        buf = torch.empty((7, 40, 70), dtype=torch.int16, device="cuda")
        z = 0
        for n in (7, 3, 7, 6):
            buf[:n].copy_(torch.from_numpy(img[z:z + n].view(np.int16)))
            torch.cuda.synchronize()
            ecc.ecc_stream_push_slab(h, s, buf[:n].view(torch.uint16), z)
            z += n
        got = ecc.ecc_stream_finish(h, s)
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(got, oracle.ecc_int(img, 16384, "V"))


def test_stream_errors(lib):
    img = synth.uniform_u8((10, 8, 8), S + 6)
    h = ecc.ecc_create(device=0, slab_depth=4)
    try:
        s = ecc.ecc_stream_begin(h, img.shape, img.dtype)
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_stream_push_slab(h, s, img[3:5], 3)  # not the next plane
        assert ei.value.status == ecc.ECC_ERR_STATE
        ecc.ecc_stream_push_slab(h, s, img[0:4], 0)
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_stream_finish(h, s)  # planes 4..9 missing
        assert ei.value.status == ecc.ECC_ERR_STATE
        # the handle still works, and a value error is reported at finish
        h2 = ecc.ecc_create(device=0, bins=100)
        try:
            s2 = ecc.ecc_stream_begin(h2, img.shape, img.dtype)
            bad = img.copy()
            bad[7, 3, 3] = 200
            _push_all(h2, s2, bad, [5, 5])
            with pytest.raises(ecc.EccError) as ei:
                ecc.ecc_stream_finish(h2, s2)
            assert ei.value.status == ecc.ECC_ERR_VALUE
        finally:
            ecc.ecc_destroy(h2)
        s3 = ecc.ecc_stream_begin(h, img.shape, img.dtype)
        _push_all(h, s3, img, [10])
        assert np.array_equal(ecc.ecc_stream_finish(h, s3), oracle.ecc_int(img, 256, "V"))
        with pytest.raises(ecc.EccError):
            ecc.ecc_stream_begin(h, (4, 4), np.float32)
    finally:
        ecc.ecc_destroy(h)


# ---- batching ---------------------------------------------------------------

def _mixed_images(n, seed, max2d=120, max3d=40):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        if rng.random() < 0.5:
            shape = tuple(int(x) for x in rng.integers(1, max2d, size=2))
        else:
            shape = tuple(int(x) for x in rng.integers(1, max3d, size=3))
        if rng.random() < 0.6:
            out.append((synth.smooth_u8(shape, 1.0, seed + i), 256))
        else:
            out.append((synth.smooth_int(shape, 1.0, 16383, seed + i, np.uint16), 16384))
    return out


def test_batch_mixed_matches_oracle(lib):
    import torch
    imgs = _mixed_images(60, S + 10)
    imgs.append((np.zeros((0, 7), np.uint8), 256))
    imgs.append((np.full((1, 1, 1), 5, np.uint8), 256))
    arrays = [a for a, _ in imgs]
    bins = [b for _, b in imgs]
    # a few as device tensors
    for i in range(0, len(arrays), 7):
        arrays[i] = torch.from_numpy(arrays[i]).cuda()
    h = ecc.ecc_create(device=0)
    try:
        res = ecc.ecc_compute_batch(h, arrays, bins)
    finally:
        ecc.ecc_destroy(h)
    for (img, b), r in zip(imgs, res):
        assert not isinstance(r, Exception), r
        assert np.array_equal(r, oracle.ecc_int(img, b, "V"))


def test_batch_bad_entries_do_not_spoil_the_rest(lib):
    good = synth.smooth_u8((20, 30, 40), 2.0, S + 11)
    four_d = np.zeros((2, 2, 2, 2), np.uint8)
    too_big = good.copy()
    too_big[3, 3, 3] = 200
    h = ecc.ecc_create(device=0)
    try:
        res = ecc.ecc_compute_batch(h, [good, four_d, too_big, good], [256, 256, 100, 256])
    finally:
        ecc.ecc_destroy(h)
    want = oracle.ecc_int(good, 256, "V")
    assert np.array_equal(res[0], want) and np.array_equal(res[3], want)
    assert isinstance(res[1], ecc.EccError) and res[1].status == ecc.ECC_ERR_ARG
    assert isinstance(res[2], ecc.EccError) and res[2].status == ecc.ECC_ERR_VALUE


def test_batch_more_than_one_launch_worth(lib):
    """1100 images: more than one work list (1024 images), same answers."""
    rng = np.random.default_rng(S + 12)
    imgs = [rng.integers(0, 256, size=(int(rng.integers(1, 9)), int(rng.integers(1, 9))),
                         dtype=np.uint8) for _ in range(1100)]
    h = ecc.ecc_create(device=0)
    try:
        res = ecc.ecc_compute_batch(h, imgs)
    finally:
        ecc.ecc_destroy(h)
    for img, r in zip(imgs, res):
        assert np.array_equal(r, oracle.ecc_int(img, 256, "V"))


def test_batch_results_live_in_shared_blocks(lib):
    """2500 images (three launches of up to 1024, alternating between the two
    slots; host images staged once and read by both): the curves of three
    calls kept alive together (each call's results in pinned blocks the
    library shares between them), then the first call's dropped and the
    blocks reused by a fourth call; every curve is the oracle's, also after
    the handle is destroyed."""
    import torch
    rng = np.random.default_rng(S + 14)
    imgs, bins = [], []
    for i in range(2500):
        shape = tuple(int(x) for x in rng.integers(1, 10, size=int(rng.integers(1, 4))))
        if i % 3 == 0:
            imgs.append(rng.integers(0, 16384, size=shape).astype(np.uint16))
            bins.append(16384)
        else:
            imgs.append(rng.integers(0, 256, size=shape).astype(np.uint8))
            bins.append(256)
    want = [oracle.ecc_int(img, b, "V") for img, b in zip(imgs, bins)]
    arrays = [torch.from_numpy(a).cuda() if i % 11 == 0 else a for i, a in enumerate(imgs)]
    h = ecc.ecc_create(device=0)
    try:
        kept = [ecc.ecc_compute_batch(h, arrays, bins) for _ in range(3)]
        for res in kept:
            assert all(np.array_equal(r, w) for r, w in zip(res, want))
        del kept[0]
        kept.append(ecc.ecc_compute_batch(h, arrays, bins))
    finally:
        ecc.ecc_destroy(h)
    for res in kept:
        assert len(res) == len(want)
        assert all(np.array_equal(r, w) for r, w in zip(res, want))


def test_batch_profiling_records_graphs(lib):
    """With profiling on, a batched call records its graphs: the span from the
    first start to the last end is positive and at most their summed time
    plus the gaps (the two slots' graphs overlap or follow each other)."""
    rng = np.random.default_rng(S + 15)
    imgs = [rng.integers(0, 256, size=(12, 40, 64), dtype=np.uint8) for _ in range(1500)]
    h = ecc.ecc_create(device=0)
    try:
        ecc.ecc_set_profiling(h, True)
        ecc.ecc_profile_read(h)
        res = ecc.ecc_compute_batch(h, imgs)
        total, count = ecc.ecc_profile_read(h)
        span = ecc.ecc_profile_span(h)
    finally:
        ecc.ecc_destroy(h)
    assert count == 2 and total > 0 and 0 < span
    assert np.array_equal(res[0], oracle.ecc_int(imgs[0], 256, "V"))


# ---- serving ----------------------------------------------------------------

def test_serve_alone_equals_in_the_mix(lib):
    imgs = _mixed_images(80, S + 20, max2d=200, max3d=48)
    h = ecc.ecc_create(device=0, bins=16384)  # one bin count for both dtypes
    try:
        alone = [ecc.ecc_compute(h, img) for img, _ in imgs]
        ids = [ecc.ecc_submit(h, img) for img, _ in imgs]
        got = {}
        for rid in ids:
            st, curve = ecc.ecc_poll(h, rid, timeout_us=60_000_000)
            assert st == ecc.ECC_OK
            got[rid] = curve
        lat = [ecc.ecc_request_latency_us(h, rid) for rid in ids]
    finally:
        ecc.ecc_destroy(h)
    for (img, _), rid, a in zip(imgs, ids, alone):
        assert np.array_equal(got[rid], a)
        assert np.array_equal(a, oracle.ecc_int(img, 16384, "V"))
    assert all(x > 0 for x in lat)


def test_serve_memory_cap_admits_gradually(lib):
    imgs = [synth.smooth_u8((24, 64, 64), 2.0, S + 30 + i) for i in range(12)]
    one = 24 * 64 * 64 + 8 * (2 * 256 + 1)
    h = ecc.ecc_create(device=0, mem_cap_bytes=3 * one)  # three requests at a time
    try:
        ids = [ecc.ecc_submit(h, img) for img in imgs]
        for img, rid in zip(imgs, ids):
            st, curve = ecc.ecc_poll(h, rid, timeout_us=60_000_000)
            assert st == ecc.ECC_OK
            assert np.array_equal(curve, oracle.ecc_int(img, 256, "V"))
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_submit(h, np.zeros((80, 80, 80), np.uint8))  # larger than the cap
        assert ei.value.status == ecc.ECC_ERR_OOM
    finally:
        ecc.ecc_destroy(h)


def test_serve_poll_states(lib):
    h = ecc.ecc_create(device=0)
    try:
        img = synth.uniform_u8((30, 30, 30), S + 40)
        rid = ecc.ecc_submit(h, img)
        st, _ = ecc.ecc_poll(h, rid, timeout_us=0)
        assert st in (ecc.ECC_OK, ecc.ECC_PENDING)
        if st == ecc.ECC_PENDING:
            st, curve = ecc.ecc_poll(h, rid, timeout_us=60_000_000)
            assert st == ecc.ECC_OK
        with pytest.raises(ecc.EccError):
            ecc.ecc_poll(h, rid, timeout_us=0)  # already retired
        with pytest.raises(ecc.EccError):
            ecc.ecc_poll(h, 987654321, timeout_us=0)
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_submit(h, np.zeros((3, 3), np.float32))
        assert ei.value.status == ecc.ECC_ERR_DTYPE
    finally:
        ecc.ecc_destroy(h)


def test_destroy_with_requests_in_flight(lib):
    h = ecc.ecc_create(device=0)
    for i in range(20):
        ecc.ecc_submit(h, synth.uniform_u8((40, 40, 40), S + 50 + i))
    ecc.ecc_destroy(h)  # cancels cleanly


def test_serve_streams_requests_larger_than_the_ring(lib):
    """Requests larger than the ring go through it in z-slabs (3D: planes of
    dims[0]; 2D: rows) while the small requests around them are batched; every
    result equals the one-shot computation and the oracle."""
    big3 = synth.two_phase_u16((60, 40, 130), 1.5, S + 50)        # 624000 B
    big2 = synth.smooth_int((700, 500), 2.0, 16383, S + 51, np.uint16)  # 700000 B
    small = _mixed_images(24, S + 52, max2d=150, max3d=40)
    order = [(big3, 16384)] + small[:12] + [(big2, 16384)] + small[12:]
    h = ecc.ecc_create(device=0, bins=16384, ring_bytes=256 * 1024, slab_depth=8,
                       mem_cap_bytes=64 << 20)
    try:
        alone = [ecc.ecc_compute(h, img) for img, _ in order]
        ids = [ecc.ecc_submit(h, img) for img, _ in order]
        got = []
        for rid in ids:
            st, curve = ecc.ecc_poll(h, rid, timeout_us=120_000_000)
            assert st == ecc.ECC_OK
            got.append(curve)
    finally:
        ecc.ecc_destroy(h)
    for (img, _), a, g in zip(order, alone, got):
        assert np.array_equal(g, a)
    assert np.array_equal(got[0], oracle.ecc_int(big3, 16384, "V"))
    assert np.array_equal(got[13], oracle.ecc_int(big2, 16384, "V"))


def test_serve_streamed_request_errors(lib):
    """A value >= bins inside a streamed request fails that request only; a
    ring that cannot fit under the cap is refused at submit."""
    bad = synth.two_phase_u16((30, 40, 130), 1.5, S + 53)
    bad[17, 5, 9] = 20000
    ok = synth.smooth_u8((20, 30, 40), 2.0, S + 54)
    h = ecc.ecc_create(device=0, bins=16384, ring_bytes=128 * 1024, slab_depth=4,
                       mem_cap_bytes=16 << 20)
    try:
        r_bad = ecc.ecc_submit(h, bad)
        r_ok = ecc.ecc_submit(h, ok)
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_poll(h, r_bad, timeout_us=120_000_000)
        assert ei.value.status == ecc.ECC_ERR_VALUE
        st, curve = ecc.ecc_poll(h, r_ok, timeout_us=120_000_000)
        assert st == ecc.ECC_OK and np.array_equal(curve, oracle.ecc_int(ok, 16384, "V"))
    finally:
        ecc.ecc_destroy(h)
    h = ecc.ecc_create(device=0, ring_bytes=1 << 20, mem_cap_bytes=512 * 1024)
    try:
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_submit(h, np.zeros((64, 128, 256), np.uint8))  # 2 MiB, ring over the cap
        assert ei.value.status == ecc.ECC_ERR_OOM
    finally:
        ecc.ecc_destroy(h)


# ---- out-of-core from a file ---------------------------------------------------

@pytest.mark.parametrize("dtype,bins", [(np.uint8, 256), (np.uint16, 16384)])
def test_stream_file_matches_oracle(lib, tmp_path, dtype, bins):
    """A raw image after a 123-byte header, streamed in slabs of 4 planes
    through a small ring (many slabs, both pinned buffers in turn)."""
    if dtype == np.uint8:
        img = synth.smooth_u8((37, 29, 45), 2.0, S + 60)
    else:
        img = synth.two_phase_u16((37, 29, 45), 1.5, S + 61)
    path = tmp_path / "vol.raw"
    with open(path, "wb") as f:
        f.write(b"h" * 123)
        f.write(np.ascontiguousarray(img).tobytes())
    h = ecc.ecc_create(device=0, bins=bins, slab_depth=4, ring_bytes=1 << 20)
    try:
        got = ecc.ecc_stream_file(h, path, img.shape, img.dtype, offset=123)
        whole = ecc.ecc_compute(h, img)
    finally:
        ecc.ecc_destroy(h)
    want = oracle.ecc_int(img, bins, "V")
    assert np.array_equal(got, want) and np.array_equal(whole, want)


@pytest.mark.parametrize("shape", [(300,), (40, 70), (1, 5, 6)], ids=str)
def test_stream_file_1d_2d_single_plane(lib, tmp_path, shape):
    img = synth.uniform_u8(shape, S + 62 + len(shape))
    path = tmp_path / "img.raw"
    img.tofile(path)
    h = ecc.ecc_create(device=0, slab_depth=3)
    try:
        got = ecc.ecc_stream_file(h, path, img.shape, img.dtype)
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(got, oracle.ecc_int(img, 256, "V"))


def test_stream_file_errors(lib, tmp_path):
    img = synth.uniform_u8((6, 7, 8), S + 63)
    path = tmp_path / "short.raw"
    img[:5].tofile(path)  # one plane short
    h = ecc.ecc_create(device=0, slab_depth=2)
    try:
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_stream_file(h, path, img.shape, img.dtype)
        assert ei.value.status == ecc.ECC_ERR_ARG
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_stream_file(h, tmp_path / "missing.raw", img.shape, img.dtype)
        assert ei.value.status == ecc.ECC_ERR_ARG
        bad = img.astype(np.uint16)
        bad[3, 2, 1] = 300
        p2 = tmp_path / "bad.raw"
        bad.tofile(p2)
        h2 = ecc.ecc_create(device=0, bins=256, slab_depth=2)
        try:
            with pytest.raises(ecc.EccError) as ei:
                ecc.ecc_stream_file(h2, p2, bad.shape, bad.dtype)
            assert ei.value.status == ecc.ECC_ERR_VALUE
        finally:
            ecc.ecc_destroy(h2)
        # the handle still works
        img.tofile(path)
        assert np.array_equal(ecc.ecc_stream_file(h, path, img.shape, img.dtype),
                              oracle.ecc_int(img, 256, "V"))
    finally:
        ecc.ecc_destroy(h)


def test_serve_concurrent_submitters(lib):
    """Four client threads submit and poll at once (ecc_submit / ecc_poll may be
    called concurrently); every result is the oracle's, and a bad request in
    one thread reports its own error to that thread."""
    import threading
    imgs = _mixed_images(48, S + 80, max2d=120, max3d=32)
    h = ecc.ecc_create(device=0, bins=16384)
    results, errors = {}, []

    def client(k):
        try:
            mine = imgs[k::4]
            ids = [ecc.ecc_submit(h, img) for img, _ in mine]
            for (img, _), rid in zip(mine, ids):
                st, curve = ecc.ecc_poll(h, rid, timeout_us=120_000_000)
                results[id(img)] = (img, curve)
            if k == 0:
                try:
                    ecc.ecc_submit(h, np.zeros((3, 3), np.float32))
                    errors.append("no error")
                except ecc.EccError as e:
                    if e.status != ecc.ECC_ERR_DTYPE or "ECC_U8" not in str(e):
                        errors.append(f"unexpected {e.status} {e}")
        except Exception as e:  # pragma: no cover - reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    try:
        for t in threads:
            t.start()
        for t in threads:
            t.join()
    finally:
        ecc.ecc_destroy(h)
    assert not errors, errors
    assert len(results) == len(imgs)
    for img, curve in results.values():
        assert np.array_equal(curve, oracle.ecc_int(img, 16384, "V"))


def test_serve_borrowed_matches_oracle(lib):
    """Borrowed submissions: pinned images are read in place (the call does not
    wait for their copies), a pageable one in the same stream is copied; the
    binding keeps a pinned image alive that the caller dropped at once."""
    import torch
    imgs = _mixed_images(40, S + 90, max2d=160, max3d=36)
    pinned = [torch.from_numpy(img).pin_memory() for img, _ in imgs]
    extra = synth.smooth_int((20, 30, 40), 1.0, 16383, S + 91, np.uint16)
    h = ecc.ecc_create(device=0, bins=16384)
    try:
        ids = [ecc.ecc_submit_borrowed(h, t) for t in pinned]
        ids.append(ecc.ecc_submit_borrowed(h, extra))  # pageable: copied
        ids.append(ecc.ecc_submit_borrowed(h, torch.from_numpy(extra.copy()).pin_memory()))
        got = []
        for rid in ids:
            st, curve = ecc.ecc_poll(h, rid, timeout_us=120_000_000)
            assert st == ecc.ECC_OK
            got.append(curve)
        assert not [k for k in ecc._borrowed if k[0] == h.value]
    finally:
        ecc.ecc_destroy(h)
    for (img, _), g in zip(imgs, got):
        assert np.array_equal(g, oracle.ecc_int(img, 16384, "V"))
    want = oracle.ecc_int(extra, 16384, "V")
    assert np.array_equal(got[-2], want) and np.array_equal(got[-1], want)


def test_serve_borrowed_over_cap_and_streamed(lib):
    """Borrowed pinned images under a cap of three requests (admitted later,
    copied from the caller's buffer) and two requests larger than the ring
    (slabs read from the caller's buffer), against the oracle."""
    import torch
    small = [synth.smooth_u8((24, 64, 64), 2.0, S + 95 + i) for i in range(9)]
    big3 = synth.two_phase_u16((60, 40, 130), 1.5, S + 96)
    big2 = synth.smooth_int((700, 500), 2.0, 16383, S + 97, np.uint16)
    order = [big3] + small[:5] + [big2] + small[5:]
    one = 24 * 64 * 64 + 8 * (2 * 16384 + 1)
    h = ecc.ecc_create(device=0, bins=16384, ring_bytes=256 * 1024, slab_depth=8,
                       mem_cap_bytes=3 * one)
    try:
        bufs = [torch.from_numpy(img).pin_memory() for img in order]
        ids = [ecc.ecc_submit_borrowed(h, t) for t in bufs]
        got = []
        for rid in ids:
            st, curve = ecc.ecc_poll(h, rid, timeout_us=120_000_000)
            assert st == ecc.ECC_OK
            got.append(curve)
    finally:
        ecc.ecc_destroy(h)
    for img, g in zip(order, got):
        assert np.array_equal(g, oracle.ecc_int(img, 16384, "V"))


def test_serve_borrowed_many_requests_two_threads(lib):
    """300 borrowed requests from two threads: more than the copies the
    library keeps in flight at a time (64), so submitters wait for room and
    the request loop batches requests as their copies finish; every curve is
    the oracle's and the binding has let go of every image."""
    import threading
    import torch
    rng = np.random.default_rng(S + 120)
    imgs = []
    for i in range(300):
        shape = tuple(int(x) for x in rng.integers(2, 24, size=int(rng.integers(1, 4))))
        imgs.append(torch.from_numpy(synth.smooth_u8(shape, 1.0, S + 121 + i)).pin_memory())
    h = ecc.ecc_create(device=0)
    ids = [None] * len(imgs)
    errors = []

    def client(k):
        try:
            for i in range(k, len(imgs), 2):
                ids[i] = ecc.ecc_submit_borrowed(h, imgs[i])
        except Exception as e:  # pragma: no cover - reported below
            errors.append(repr(e))

    try:
        threads = [threading.Thread(target=client, args=(k,)) for k in range(2)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors
        got = []
        for rid in ids:
            st, curve = ecc.ecc_poll(h, rid, timeout_us=120_000_000)
            assert st == ecc.ECC_OK
            got.append(curve)
        assert not [k for k in ecc._borrowed if k[0] == h.value]
    finally:
        ecc.ecc_destroy(h)
    for t, g in zip(imgs, got):
        assert np.array_equal(g, oracle.ecc_int(t.numpy(), 256, "V"))


def test_batch_many_large_histograms(lib):
    """80 images with 16384 bins each (10.5 MB of curves, copied out of the
    pinned arena by several threads) plus small ones: every curve is the
    oracle's and lands in its own slot of the result list."""
    rng = np.random.default_rng(S + 130)
    imgs, bins = [], []
    for i in range(100):
        shape = tuple(int(x) for x in rng.integers(2, 14, size=int(rng.integers(1, 4))))
        if i % 5 == 4:
            imgs.append(synth.smooth_u8(shape, 1.0, S + 131 + i))
            bins.append(256)
        else:
            imgs.append(synth.smooth_int(shape, 1.0, 16383, S + 131 + i, np.uint16))
            bins.append(16384)
    h = ecc.ecc_create(device=0)
    try:
        res = ecc.ecc_compute_batch(h, imgs, bins)
    finally:
        ecc.ecc_destroy(h)
    assert len(res) == len(imgs)
    for img, b, r in zip(imgs, bins, res):
        assert np.array_equal(r, oracle.ecc_int(img, b, "V"))


@pytest.mark.parametrize("borrowed", [False, True])
def test_serve_device_images(lib, borrowed):
    """Requests whose images are CUDA tensors, through ecc_submit and
    ecc_submit_borrowed: under a cap of a few requests (the rest wait for
    admission), and two larger than the ring (streamed from device memory);
    every curve is the oracle's."""
    import torch
    submit = ecc.ecc_submit_borrowed if borrowed else ecc.ecc_submit
    small = [synth.smooth_u8((24, 64, 64), 2.0, S + 140 + i) for i in range(9)]
    big3 = synth.two_phase_u16((60, 40, 130), 1.5, S + 150)
    big2 = synth.smooth_int((700, 500), 2.0, 16383, S + 151, np.uint16)
    order = small[:4] + [big3] + small[4:] + [big2]
    one = 24 * 64 * 64 + 8 * (2 * 16384 + 1)
    h = ecc.ecc_create(device=0, bins=16384, ring_bytes=256 * 1024, slab_depth=8,
                       mem_cap_bytes=3 * one)
    try:
        dev = [torch.from_numpy(img.view(np.int16) if img.dtype == np.uint16 else img).cuda()
               for img in order]
        dev = [d.view(torch.uint16) if img.dtype == np.uint16 else d for d, img in zip(dev, order)]
        torch.cuda.synchronize()
        ids = [submit(h, d) for d in dev]
        got = []
        for rid in ids:
            st, curve = ecc.ecc_poll(h, rid, timeout_us=120_000_000)
            assert st == ecc.ECC_OK
            got.append(curve)
    finally:
        ecc.ecc_destroy(h)
    for img, g in zip(order, got):
        assert np.array_equal(g, oracle.ecc_int(img, 16384, "V"))
