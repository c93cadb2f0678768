"""Writes the stored oracle regression values under tests/golden/.

Calls only the CPU oracle (oracle/) and the seeded input generators; nothing
here touches the CUDA path.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2103_07512_gb300 import inputs as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    tok, g = I.small_population(seed=0)
    r64, _, _ = oracle.fitness(tok.ops, tok.imm, tok.tree_off, tok.order, g.W, g.H,
                               g.xlo, g.xhi, g.ylo, g.yhi)
    with open(os.path.join(HERE, "small_population_rmse.txt"), "w") as f:
        f.write("# RMSE vs Pagie (Eq. 1) of the 50-tree RHH population (depth 2-6, seed 0)\n")
        f.write("# on the 64x64 grid over [-5,5]^2, binary64 oracle; written by make_golden.py\n")
        for v in r64:
            f.write(f"{float(v)!r}\n")


if __name__ == "__main__":
    main()
