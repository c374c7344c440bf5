"""Writes the stored expected values under tests/golden/.

Calls only ``oracle/`` (and the seeded generators in ``workloads/``); no GPU
code is imported.  Run from the repository root:

    python tests/golden/make_golden.py
"""

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import field as F  # noqa: E402
from oracle import tft as T  # noqa: E402
from workloads import config1_inputs  # noqa: E402


def main():
    a, b, _ = config1_inputs()
    c = T.schoolbook(F.P998244353, [int(v) for v in a], [int(v) for v in b])
    with open(os.path.join(HERE, "config1_product.txt"), "w") as fh:
        fh.write("# schoolbook product of the two length-500 operands of the\n"
                 "# p = 998244353 workload (seed 0), written by "
                 "make_golden.py from oracle.tft.schoolbook\n")
        for v in c:
            fh.write(f"{v}\n")


if __name__ == "__main__":
    main()
