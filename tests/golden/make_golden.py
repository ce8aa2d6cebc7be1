"""Write tests/golden/small_volumes.json from the CPU oracle alone.

The fixture pins the oracle across machines (x86 here, Arm on the GPU
host): each case is a seeded tiny volume and its exact moments (Eq. 2),
stored as decimal strings.  Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2012_08099_gb300 import synth  # noqa: E402

CASES = [
    ("u8", (4, 4, 4), 101, 3),
    ("u8", (3, 5, 7), 102, 6),
    ("u16", (5, 4, 6), 103, 8),
    ("u16", (2, 9, 3), 104, 4),
]


def main():
    out = []
    for dt, shape, seed, K in CASES:
        vol = synth.uniform_volume(shape, np.uint8 if dt == "u8" else np.uint16, seed=seed)
        out.append({
            "dtype": dt, "shape_zyx": list(shape), "seed": seed, "K": K,
            "moments": [str(v) for v in oracle.moments(vol, K, nthreads=1)],
        })
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "small_volumes.json")
    with open(path, "w") as f:
        json.dump({"source": "oracle.moments (Eq. 2), uniform seeded volumes", "cases": out}, f,
                  indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
