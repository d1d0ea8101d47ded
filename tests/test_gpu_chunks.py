"""GPU parity of the chunk entry point (ecc_compute_vcec_chunk): an image cut
along dims[0] into chunks, each computed from its own planes plus the
one-plane collars (as a worker holding only that part would), gives partial
VCECs whose sum equals the oracle's VCEC of the whole image (Sec. 3,
"Parallel Computations" and "Post-Processing"). Random partitions with
single-plane and empty chunks, 1-4D, both dtypes and conventions, host and
device planes."""
import numpy as np
import pytest

import oracle
from paper_1705_02045_gb300 import ecc, synth

pytestmark = pytest.mark.gpu

S = synth.SEED_BASE + 2100

CASES = [
    ((1000,), np.uint8, 256, lambda s: synth.uniform_u8(s, S + 1)),
    ((50, 70), np.uint8, 256, lambda s: synth.smooth_u8(s, 1.5, S + 2)),
    ((37, 40, 64), np.uint8, 256, lambda s: synth.smooth_u8(s, 2.0, S + 3)),
    ((29, 33, 61), np.uint16, 16384, lambda s: synth.two_phase_u16(s, 1.5, S + 4)),
    ((11, 7, 9, 10), np.uint16, 65536,
     lambda s: synth.uniform_int(s, 65536, S + 5, np.uint16)),
    ((9, 6, 7, 130), np.uint8, 256, lambda s: synth.smooth_u8(s, 1.0, S + 6)),
]


def _cuts(n0, rng):
    inner = sorted(set(int(x) for x in rng.integers(0, n0 + 1, size=min(n0, 5))))
    cuts = sorted(set([0, n0] + inner))
    if n0 >= 3:  # a single-plane chunk and an empty one
        cuts = sorted(set(cuts + [1, 2]))
    return list(zip(cuts[:-1], cuts[1:])) + [(cuts[-1], cuts[-1])]


@pytest.mark.parametrize("conv", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{np.dtype(c[1]).name}")
def test_chunk_vcecs_add_up_to_the_oracle(case, conv):
    import torch
    shape, dtype, bins, gen = case
    img = gen(shape).astype(dtype)
    rng = np.random.default_rng(S + sum(shape))
    h = ecc.ecc_create(device=0, bins=bins, convention=conv)
    try:
        total = np.zeros(bins, np.int64)
        for k, (lo, hi) in enumerate(_cuts(shape[0], rng)):
            p_lo, p_hi = max(lo - 1, 0), min(hi + 1, shape[0])
            part = np.ascontiguousarray(img[p_lo:p_hi])
            if k % 2:
                part = torch.from_numpy(part).cuda()
            total += ecc.ecc_compute_vcec_chunk(h, part, shape, lo, hi, bins)
    finally:
        ecc.ecc_destroy(h)
    assert np.array_equal(total, oracle.vcec_int(img, bins, "V" if conv == 0 else "T"))
    assert np.array_equal(np.cumsum(total), oracle.ecc_int(img, bins, "V" if conv == 0 else "T"))


def test_chunk_errors():
    img = synth.uniform_u8((6, 8, 16), S + 7)
    h = ecc.ecc_create(device=0)
    try:
        for lo, hi in [(-1, 2), (3, 7), (4, 3)]:
            with pytest.raises(ecc.EccError) as ei:
                ecc.ecc_compute_vcec_chunk(h, img, img.shape, lo, hi, 256)
            assert ei.value.status == ecc.ECC_ERR_ARG
        bad = img.copy()
        bad[2, 3, 4] = 200
        hb = ecc.ecc_create(device=0, bins=100)
        try:
            with pytest.raises(ecc.EccError) as ei:
                ecc.ecc_compute_vcec_chunk(hb, bad[1:4], bad.shape, 2, 3, 100)
            assert ei.value.status == ecc.ECC_ERR_VALUE
        finally:
            ecc.ecc_destroy(hb)
        # the handle still computes whole images correctly afterwards
        assert np.array_equal(ecc.ecc_compute(h, img), oracle.ecc_int(img, 256, "V"))
    finally:
        ecc.ecc_destroy(h)
