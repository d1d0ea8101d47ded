"""Write tests/golden/oracle_small.json: small seeded images and their curves.

Calls only the CPU oracle (oracle/) and the seeded generators; nothing here
comes from the CUDA path. The paper's own worked example (the bone slice of
its Fig. 1, with chi = 8, -17, -7, -3, 1 at t = 0, 12, 25, 38, 52) cannot be a
fixture: the image itself is not part of the paper's text.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1705_02045_gb300 import synth  # noqa: E402

CASES = [
    # name, shape, dtype, bins, generator
    ("u8_1d_uniform", (37,), "uint8", 256, lambda s: synth.uniform_u8(s, 1)),
    ("u8_2d_uniform", (13, 17), "uint8", 256, lambda s: synth.uniform_u8(s, 2)),
    ("u8_3d_smooth", (9, 10, 11), "uint8", 256, lambda s: synth.smooth_u8(s, 1.5, 3)),
    ("u16_3d_two_phase", (8, 9, 7), "uint16", 16384, lambda s: synth.two_phase_u16(s, 1.5, 4)),
    ("u8_4d_uniform", (4, 3, 5, 4), "uint8", 8, lambda s: synth.uniform_int(s, 8, 5, np.uint8)),
    ("f32_3d_grf", (6, 7, 5), "float32", 0, lambda s: synth.grf_f32(s, 1.0, 6)),
]


def main():
    out = []
    for name, shape, dtype, bins, gen in CASES:
        img = gen(shape).astype(dtype)
        rec = {"name": name, "shape": list(shape), "dtype": dtype,
               "values": img.ravel().tolist()}
        for conv in ("V", "T"):
            if dtype == "float32":
                t, chi = oracle.ecc_pairs_float(img, conv)
                rec["pairs_" + conv] = [[float(a), int(b)] for a, b in zip(t, chi)]
            else:
                a = oracle.vcec_int(img, bins, conv)
                nz = np.flatnonzero(a)
                rec["bins"] = bins
                # sparse VCEC (t, a_t) keeps the 14-bit fixture small
                rec["vcec_" + conv] = [[int(t), int(a[t])] for t in nz]
        out.append(rec)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json")
    with open(path, "w") as f:
        f.write("[\n" + ",\n".join(json.dumps(r) for r in out) + "\n]\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
