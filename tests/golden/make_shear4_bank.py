"""Writes shear4_bank_64x64.json: sampled values of the oracle's filter bank for a 2D
system at the maximum shear level 4 (64 x 64 grid, one scale, R = 65).

The oracle builds these filters by explicit upsampling by 16, convolution, shearing
and downsampling of finite arrays; that takes minutes, too long for the test suites,
so this script (which calls only oracle/) stores what the library's bank is compared
with: the frame bound A, every filter's norm, and the real spectrum at 12 seeded
frequencies per filter (half spectrum, k1 <= 32).

    python tests/golden/make_shear4_bank.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import shearlet_oracle as O  # noqa: E402

DIMS, J, LEVELS = (64, 64), 1, (4,)


def main() -> None:
    s = O.build_system(DIMS, J, LEVELS)
    rng = np.random.default_rng(2024)
    nh = DIMS[1] // 2 + 1
    filters = []
    for j in range(s.R):
        m = s.meta[j]
        k0 = rng.integers(0, DIMS[0], 12)
        k1 = rng.integers(0, nh, 12)
        ph = s.psi_hat(j)
        filters.append({"scale": int(m.scale), "cone": int(m.cone), "k": [int(v) for v in m.k],
                        "norm": float(s.norms[j]),
                        "samples": [[int(a), int(b), float(ph[a, b])] for a, b in zip(k0, k1)]})
    out = {"dims": list(DIMS), "nScales": J, "shearLevels": list(LEVELS), "R": int(s.R),
           "A": float(s.A), "filters": filters,
           "source": "oracle/shearlet_oracle.py build_system, written by make_shear4_bank.py"}
    head = {k: v for k, v in out.items() if k != "filters"}
    with open(os.path.join(HERE, "shear4_bank_64x64.json"), "w") as f:  # one filter per line
        f.write(json.dumps(head)[:-1] + ', "filters": [\n')
        f.write(",\n".join(json.dumps(fl, separators=(",", ":")) for fl in filters))
        f.write("\n]}\n")


if __name__ == "__main__":
    main()
