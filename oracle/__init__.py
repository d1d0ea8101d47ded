"""CPU oracle for Euler characteristic curves of gray-scale images.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import this package:
only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) use it. The CUDA library never calls it and
shares no code with it.

The oracle is the plain definition written out (Heiss & Wagner, Sec. 2 and 3):
enumerate every cell of the cubical complex of the image, give each cell its
filtration value, histogram (-1)^dim by value, prefix-sum. It never uses
neighbour masks, tie-breaks or the per-voxel block decomposition that the GPU
path uses, so a mistake in that decomposition cannot hide in both.

Pinning status of each public function is stated in its docstring and in the
pin tests (``tests/test_oracle_pins.py``). Functions with no independent pin
say "parity unpinned".
"""
from .ecc_oracle import (  # noqa: F401
    SENTINEL_INT,
    cells_V,
    cells_T,
    vcec_int,
    vcec_int_zrange,
    ecc_int,
    ecc_from_vcec,
    ecc_pairs_float,
    vcec_float_zrange,
    merge_vcec_float,
    pairs_from_vcec_float,
    quantize_f32,
    ecc_quantized,
    cell_counts,
)
