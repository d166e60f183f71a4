"""Write stored expected values for inputs too large to run the oracle inside a test.

Calls only the CPU oracle (``oracle/``) on the seeded synthetic inputs of
``paper_2404_05708_gb300.workloads``.  Each record keeps a SHA-256 of the
input arrays so a test can tell whether it regenerated the very same curves.

    python tests/golden/make_golden.py            # all records
"""
import hashlib
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2404_05708_gb300 import workloads  # noqa: E402


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(a.tobytes())
    return h.hexdigest()


def long_pair_record():
    p, q = workloads.warped_long_pair(200_000, 200_000, dim=3, seed=3)
    t = time.time()
    d2 = oracle.dfd2_linear(p, q)
    return {
        "name": "warped_long_pair_200k_d3",
        "generator": "workloads.warped_long_pair(200000, 200000, dim=3, seed=3)",
        "sha256": digest(p, q),
        "delta2_f64": d2,
        "delta_f64": math.sqrt(d2),
        "method": "oracle.dfd2_linear (Alg. 5, float64)",
        "oracle_seconds": round(time.time() - t, 1),
    }


def main():
    out = os.path.join(HERE, "long_pair_200k.json")
    rec = long_pair_record()
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec, indent=1))


if __name__ == "__main__":
    main()
