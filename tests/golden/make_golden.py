"""Write the stored expected values under tests/golden/ (calls only oracle/).

tori_seed.json: the two-tori workload (R = 1, r = 0.3, 32 x 32 quads, B at a
seeded random rotation and +2.5 along x) must not intersect; its seed is the
first one for which the oracle's brute-force D_min (Section 3, Eq. 1) is
positive.  Run from the repository root:  python tests/golden/make_golden.py
"""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2411_11244_gb300 import synth  # noqa: E402


def main():
    seed = 0
    while True:
        A, B, xa, xb = synth.config_tori(seed)
        r = oracle.brute(A, xa, B, xb)
        if r.d > 0.0:
            break
        seed += 1
    out = {
        "source": "oracle brute force, Section 3 Eq. 1; workload: two tori R=1 r=0.3 32x32 quads, offset 2.5",
        "seed": seed,
        "d_min": r.d,
        "witness": [r.ta, r.tb],
    }
    with open(os.path.join(os.path.dirname(__file__), "tori_seed.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(out)


if __name__ == "__main__":
    main()
