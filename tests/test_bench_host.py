"""Host-side logic of the benchmark: a served curve spans the handle's default
bins (65536 for uint16 images) while the batched call of the same image uses
the request's bins; the benchmark accepts the served curve when it equals the
batched one and then holds its last value. The oracle fixes that property:
thresholds past the largest gray value add no cells (Sec. 3, the curve as
the running sum of the VCEC)."""
import numpy as np

import bench
import oracle
from paper_1705_02045_gb300 import synth


def test_served_curve_comparison_against_the_oracle():
    img = synth.two_phase_u16((6, 20, 24), 1.5, synth.SEED_BASE + 2200)  # 14-bit values
    assert int(img.max()) < 16384
    for conv in ("V", "T"):
        small = oracle.ecc_int(img, 16384, conv)
        large = oracle.ecc_int(img, 65536, conv)
        assert np.array_equal(large[:16384], small)
        assert bench._same_curve(large, small)
        # a change past the batched bins, one inside them, a shorter curve
        late = large.copy()
        late[20000] += 1
        assert not bench._same_curve(late, small)
        early = large.copy()
        early[int(img.min())] -= 1
        assert not bench._same_curve(early, small)
        assert not bench._same_curve(small[:100], small)
