"""Write the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle as orc  # noqa: E402
from paper_1408_1664_gb300 import datagen  # noqa: E402


def main():
    ds, d = datagen.config_small()
    out = orc.edge_posteriors(ds.data, ds.arity, d)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "small_n12_d3_posteriors.txt")
    with open(path, "w") as f:
        f.write("# Edge posteriors P(u->v|D), row u, column v, of the n=12 binary, d=3,\n"
                "# m=200, seed 0 workload (datagen.config_small), BDeu ess=1, q=rho=1.\n"
                "# Written by tests/golden/make_golden.py from the CPU oracle only.\n"
                "# First line: log P(D).  Then the n x n matrix.\n")
        f.write(f"{out['log_PD']:.17g}\n")
        for row in out["post"]:
            f.write(" ".join(f"{x:.17g}" for x in row) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
